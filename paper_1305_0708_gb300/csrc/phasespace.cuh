// On-device phase-space generation, cuts and redraws (FP64).
//
// Random numbers: Philox4x64-10 (Salmon, Moraes, Dror, Shaw, SC'11), one
// counter per (event, attempt, block): counter = (event, attempt, block, 0),
// key = (seed, 0), ten rounds with the Weyl key schedule.  Each 64-bit word
// gives two 32-bit deviates w (low half first), mapped to (w + 1/2) 2^-32 in
// (0, 1), as the paper's generator delivers 32-bit deviates (App. B): uniform i
// of a draw is half i % 2 of word (i % 8) / 2 of block i / 8.
//
// Generators: two-body at fixed sqrt(s) with cos(theta), phi uniform;
// massless RAMBO (Kleiss, Stirling, Ellis 1986) with the massive rescaling;
// g g > t t~ > (b W+)(b~ W-) > ... with sqrt(s) uniform, Breit-Wigner
// sampled t, t~, W+, W- virtualities (the paper's Eq. 16, App. A.2) and
// isotropic two-body decays.  A point that fails the cuts (the paper's
// Eqs. 8-11 in form: pT, |eta|, Delta R) is redrawn with the next attempt,
// which keeps the result independent of the launch shape (Sect. 3 and App. A
// note that on a GPU each thread has one try per point; here each thread
// loops until its own point passes).
#pragma once
#include <cstdint>

#include "dfloat.cuh"
#include "me_internal.h"

namespace me {

struct Philox {
  static __host__ __device__ __forceinline__ void mulhilo(uint64_t a, uint64_t b, uint64_t& hi, uint64_t& lo) {
#ifdef __CUDA_ARCH__
    // the 128-bit product from four 32 x 32-bit partial products with one carry chain
    // (the lower and upper halves share their partial products)
    const uint32_t a0 = (uint32_t)a, a1 = (uint32_t)(a >> 32), b0 = (uint32_t)b, b1 = (uint32_t)(b >> 32);
    uint32_t r0, r1, r2, r3;
    asm("{\n\t"
        "mul.lo.u32 %0, %4, %6;\n\t"
        "mul.hi.u32 %1, %4, %6;\n\t"
        "mad.lo.cc.u32 %1, %4, %7, %1;\n\t"
        "madc.hi.u32 %2, %4, %7, 0;\n\t"
        "mad.lo.cc.u32 %1, %5, %6, %1;\n\t"
        "madc.hi.cc.u32 %2, %5, %6, %2;\n\t"
        "madc.hi.u32 %3, %5, %7, 0;\n\t"
        "mad.lo.cc.u32 %2, %5, %7, %2;\n\t"
        "addc.u32 %3, %3, 0;\n\t"
        "}"
        : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3)
        : "r"(a0), "r"(a1), "r"(b0), "r"(b1));
    lo = ((uint64_t)r1 << 32) | r0;
    hi = ((uint64_t)r3 << 32) | r2;
#else
    hi = (uint64_t)(((unsigned __int128)a * b) >> 64);
    lo = a * b;
#endif
  }
  static __host__ __device__ __forceinline__ void block(uint64_t c0, uint64_t c1, uint64_t c2, uint64_t c3,
                                                        uint64_t k0, uint64_t k1, uint64_t out[4]) {
    const uint64_t M0 = 0xD2E7470EE14C6C93ull, M1 = 0xCA5A826395121157ull;
    const uint64_t W0 = 0x9E3779B97F4A7C15ull, W1 = 0xBB67AE8584CAA73Bull;
#pragma unroll  // unrolled: the Weyl key increments fold into constants
    for (int r = 0; r < 10; ++r) {
      uint64_t h0, l0, h1, l1;
      mulhilo(M0, c0, h0, l0);
      mulhilo(M1, c2, h1, l1);
      const uint64_t n0 = h1 ^ c1 ^ k0, n2 = h0 ^ c3 ^ k1;
      c0 = n0; c1 = l1; c2 = n2; c3 = l0;
      k0 += W0; k1 += W1;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
  }
};

__host__ __device__ __forceinline__ double unit32(uint32_t w) { return ((double)w + 0.5) * 0x1p-32; }
__host__ __device__ __forceinline__ uint32_t half32(uint64_t x, int h) { return (uint32_t)(h ? x >> 32 : x); }

// ---------------------------------------------------------------------------
// Adaptive grid (VEGAS, Lepage 1978) over the generator's uniforms: in
// dimension d a uniform y lies in bin i = floor(N y) and maps to
// x = e_i + (N y - i)(e_{i+1} - e_i); the Jacobian N (e_{i+1} - e_i) multiplies
// the weight and the bin is recorded for the histogram of the refinement.
// ---------------------------------------------------------------------------
__host__ __device__ __forceinline__ double vg_map(const KinDev& kin, int d, double y, double& jac, uint8_t* bins) {
  const int N = kin.vg_bins;
  const double t = y * N;
  int i = (int)t;
  i = i < N - 1 ? i : N - 1;
  const double* e = kin.vg_edges + (size_t)d * (N + 1);
  const double lo = e[i], w = e[i + 1] - lo;
  jac *= N * w;
  if (bins) bins[d] = (uint8_t)i;
  return lo + (t - i) * w;
}

__host__ __device__ __forceinline__ df vg_map_df(const KinDev& kin, int d, df y, df& jac, uint8_t* bins) {
  const int N = kin.vg_bins;
  const df t = y * (float)N;  // N <= 256: exact in FP32
  int i = (int)floorf(t.hi);
  if ((float)i == t.hi && t.lo < 0.0f) --i;
  i = i < 0 ? 0 : (i < N - 1 ? i : N - 1);
  const double* e = kin.vg_edges + (size_t)d * (N + 1);
  const df lo = from_double(e[i]), w = from_double(e[i + 1]) - lo;
  jac = jac * (w * (float)N);
  if (bins) bins[d] = (uint8_t)i;
  return lo + (t + (float)(-i)) * w;
}

// uniforms u[NU] for (event, attempt)
template <int NU>
__host__ __device__ __forceinline__ void draw_uniforms(uint64_t seed, uint64_t event, uint64_t attempt, double (&u)[NU]) {
#pragma unroll
  for (int j = 0; j < (NU + 7) / 8; ++j) {
    uint64_t o[4];
    Philox::block(event, attempt, (uint64_t)j, 0ull, seed, 0ull, o);
#pragma unroll
    for (int q = 0; q < 8; ++q)
      if (8 * j + q < NU) u[8 * j + q] = unit32(half32(o[q / 2], q & 1));
  }
}

__host__ __device__ __forceinline__ void set4(double* p, double e, double x, double y, double z) {
  p[0] = e; p[1] = x; p[2] = y; p[3] = z;
}

// isotropic unit vector from cos(theta) = 2a - 1, phi = 2 pi b
__host__ __device__ __forceinline__ void direction(double a, double b, double& nx, double& ny, double& nz) {
  const double c = 2.0 * a - 1.0;
  const double s = sqrt(fmax(1.0 - c * c, 0.0));
  double sp, cp;
  sincospi(2.0 * b, &sp, &cp);
  nx = s * cp; ny = s * sp; nz = c;
}

// two-body decay at rest of mass M into (m1, m2): |p*| and the momenta along +-n
__host__ __device__ __forceinline__ double kallen_sqrt(double a, double b, double c) {
  const double l = a * a + b * b + c * c - 2.0 * (a * b + b * c + c * a);
  return sqrt(fmax(l, 0.0));
}

// boost pstar out of the rest frame of a system with lab momentum P and mass M
__host__ __device__ __forceinline__ void boost_from_rest(double* p, const double* P, double M) {
  const double pp = P[1] * p[1] + P[2] * p[2] + P[3] * p[3];
  const double e = (P[0] * p[0] + pp) / M;
  const double f = (pp / (P[0] + M) + p[0]) / M;
  p[0] = e;
  p[1] += f * P[1];
  p[2] += f * P[2];
  p[3] += f * P[3];
}

// ---------------------------------------------------------------------------
// generators; each returns false if the draw is outside the kinematic limits
// ---------------------------------------------------------------------------
template <int NEXT>
__host__ __device__ __forceinline__ void beams(double (&p)[NEXT][4], double w) {
  set4(p[0], 0.5 * w, 0.0, 0.0, 0.5 * w);
  set4(p[1], 0.5 * w, 0.0, 0.0, -0.5 * w);
}

template <int NEXT>
__host__ __device__ __forceinline__ bool gen_two_body(const KinDev& kin, const double* u, double (&p)[NEXT][4],
                                                      double& wps, double& shat) {
  const double w = kin.sqrt_s;
  beams<NEXT>(p, w);
  double nx, ny, nz;
  direction(u[0], u[1], nx, ny, nz);
  const double E = 0.5 * w;
  set4(p[NEXT - 1], E, E * nx, E * ny, E * nz);
  set4(p[NEXT - 2], E, -E * nx, -E * ny, -E * nz);
  wps = 1.0 / (8.0 * 3.14159265358979323846);
  shat = w * w;
  return true;
}

// RAMBO (Kleiss, Stirling, Ellis 1986): NF massless momenta at total energy w
// from 4 NF uniforms, in q[0..NF-1]
template <int NF>
__host__ __device__ __forceinline__ void rambo_massless_core(double w, const double* u, double (*q)[4]) {
  double Q0 = 0, Q1 = 0, Q2 = 0, Q3 = 0;
#pragma unroll
  for (int k = 0; k < NF; ++k) {
    double nx, ny, nz;
    direction(u[4 * k + 0], u[4 * k + 1], nx, ny, nz);
    const double q0 = -log(u[4 * k + 2] * u[4 * k + 3]);
    set4(q[k], q0, q0 * nx, q0 * ny, q0 * nz);
    Q0 += q0; Q1 += q[k][1]; Q2 += q[k][2]; Q3 += q[k][3];
  }
  const double M = sqrt(Q0 * Q0 - Q1 * Q1 - Q2 * Q2 - Q3 * Q3);
  const double iM = 1.0 / M;
  const double b1 = -Q1 * iM, b2 = -Q2 * iM, b3 = -Q3 * iM;
  const double gam = Q0 * iM, a = 1.0 / (1.0 + gam), x = w * iM;
#pragma unroll
  for (int k = 0; k < NF; ++k) {
    double* r = q[k];
    const double bq = b1 * r[1] + b2 * r[2] + b3 * r[3];
    const double q0 = r[0];
    const double c = q0 + a * bq;
    r[0] = x * (gam * q0 + bq);
    r[1] = x * (r[1] + b1 * c);
    r[2] = x * (r[2] + b2 * c);
    r[3] = x * (r[3] + b3 * c);
  }
}

// massive rescaling of NF massless momenta q at total energy w to masses m[]:
// sum_k sqrt(m_k^2 + xi^2 E_k^2) = w by Newton's method; returns the weight factor
// xi^(2 NF - 3) prod_k(|p_k| / E_k) w / sum_k(|p_k|^2 / E_k)
template <int NF>
__host__ __device__ __forceinline__ double rambo_massive_rescale(double w, const double* m, double (*q)[4]) {
  double E0[NF];
  double msum = 0;
#pragma unroll
  for (int k = 0; k < NF; ++k) { E0[k] = q[k][0]; msum += m[k]; }
  double xi = sqrt(fmax(1.0 - (msum / w) * (msum / w), 0.0));
  for (int it = 0; it < 40; ++it) {
    double f = -w, df = 0;
#pragma unroll
    for (int k = 0; k < NF; ++k) {
      const double Ek = sqrt(m[k] * m[k] + xi * xi * E0[k] * E0[k]);
      f += Ek;
      df += xi * E0[k] * E0[k] / Ek;
    }
    xi -= f / df;
  }
  double prod = 1.0, sum = 0.0;
#pragma unroll
  for (int k = 0; k < NF; ++k) {
    const double ak = xi * E0[k];
    const double Ek = sqrt(m[k] * m[k] + ak * ak);
    prod *= ak / Ek;
    sum += ak * ak / Ek;
    q[k][0] = Ek;
    q[k][1] *= xi; q[k][2] *= xi; q[k][3] *= xi;
  }
  return pow(xi, 2 * NF - 3) * prod * w / sum;
}

// RAMBO: massless momenta, then (if any mass) the Kleiss-Stirling-Ellis rescaling
template <int NEXT>
__host__ __device__ __forceinline__ bool gen_rambo(const KinDev& kin, const double* u, double (&p)[NEXT][4],
                                                   double& wps, double& shat) {
  constexpr int NF = NEXT - 2;
  const double w = kin.sqrt_s;
  beams<NEXT>(p, w);
  rambo_massless_core<NF>(w, u, p + 2);
  // massless volume (2pi)^(4-3n) (pi/2)^(n-1) w^(2n-4) / ((n-1)! (n-2)!)
  wps = kin.rambo_volume;
  shat = w * w;
  if (kin.massive) wps *= rambo_massive_rescale<NF>(w, kin.mass + 2, p + 2);
  return true;
}

__host__ __device__ __forceinline__ double bw_draw(double m, double g, double t0, double t1, double uu, double& jac) {
  const double th = t0 + (t1 - t0) * uu;
  const double s = m * m + m * g * tan(th);
  const double d = s - m * m;
  jac = (t1 - t0) * (d * d + m * m * g * g) / (m * g) * (1.0 / (2.0 * 3.14159265358979323846));
  return s;
}

// Resonance-mapped RAMBO (App. A.2): legs 2 and 3 are the decay products of a
// resonance R (kin.bw_mass[0], kin.bw_width[0]); dPhi_n = dPhi_{n-1}(R, 4..) ds/(2 pi)
// dPhi_2(R -> 2 3), s Breit-Wigner mapped (Eq. 16 range), RAMBO with the resonance
// mass for (R, legs 4..), isotropic decay at rest.  Uniforms: 4 per RAMBO particle
// of (R, 4, ...), then theta, then the decay direction of leg 2.
template <int NEXT>
__host__ __device__ __forceinline__ bool gen_rambo_bw(const KinDev& kin, const double* u, double (&p)[NEXT][4],
                                                      double& wps, double& shat) {
  constexpr int NR = NEXT - 3;  // RAMBO particles: the resonance and legs 4..NEXT-1
  const double w = kin.sqrt_s;
  double jac;
  const double s = bw_draw(kin.bw_mass[0], kin.bw_width[0], kin.bw_t0[0], kin.bw_t1[0], u[4 * NR], jac);
  if (!(s > 0.0)) return false;
  const double M = sqrt(s);
  if (!(M < w)) return false;
  beams<NEXT>(p, w);
  double q[NR][4];
  rambo_massless_core<NR>(w, u, q);
  double m[NR];
#pragma unroll
  for (int k = 0; k < NR; ++k) m[k] = k == 0 ? M : 0.0;
  const double fac = rambo_massive_rescale<NR>(w, m, q);
  double nx, ny, nz;
  direction(u[4 * NR + 1], u[4 * NR + 2], nx, ny, nz);
  const double kd = 0.5 * M;
  set4(p[2], kd, kd * nx, kd * ny, kd * nz);
  set4(p[3], kd, -kd * nx, -kd * ny, -kd * nz);
  boost_from_rest(p[2], q[0], M);
  boost_from_rest(p[3], q[0], M);
#pragma unroll
  for (int k = 1; k < NR; ++k) set4(p[3 + k], q[k][0], q[k][1], q[k][2], q[k][3]);
  wps = kin.rambo_volume * fac * jac * kd / (4.0 * 3.14159265358979323846 * M);
  shat = w * w;
  return true;
}

// The paper's parametrisation at fixed energy (Eq. 13, App. A.1; Eq. 17; App. A.2), in FP64:
// n objects (kin.n_obj), each one leg or a Breit-Wigner resonance decaying isotropically into two
// massless legs.  dPhi_n = (2 pi)^(4 - 3n) 2^-n prod dy_i d^2 pT_i delta^4(P - sum p): the first n - 2
// objects take y uniform in [-y_max, y_max], the first n - 1 take ln(pT^2 + m^2) uniform over their pT
// range and phi uniform, the last pT balances; P+- = sum mT exp(+-y) = sqrt_s then fixes the last two
// rapidities (a quadratic in mT_a exp(y_a), one of its two roots drawn; Jacobian
// 2 mT_a mT_b |sinh(y_b - y_a)|).  Uniforms, in order: resonance virtualities, free rapidities,
// (pT, phi) pairs, the root, the resonances' decay directions: 3 per final leg - 3 in all.
template <int NEXT>
__host__ __device__ __forceinline__ bool gen_ypt(const KinDev& kin, const double* u, double (&p)[NEXT][4],
                                                 double& wps, double& shat) {
  constexpr int NF = NEXT - 2;  // objects never outnumber the final legs
  constexpr double kPi_ = 3.14159265358979323846;
  const int n = kin.n_obj;
  const double w = kin.sqrt_s;
  beams<NEXT>(p, w);
  double m2[NF], px[NF], py[NF], y[NF];
  double wt = 1.0;
  int k = 0;
#pragma unroll
  for (int j = 0; j < NF; ++j) {
    m2[j] = 0.0;
    px[j] = py[j] = y[j] = 0.0;
    if (j >= n) continue;
    if (kin.obj_legs[j][1] >= 0) {
      double jac;
      const double sr = bw_draw(kin.obj_res_mass[j], kin.obj_res_width[j], kin.obj_t0[j], kin.obj_t1[j], u[k++], jac);
      if (!(sr > 0.0)) return false;
      m2[j] = sr;
      wt *= jac;
    } else {
      m2[j] = kin.obj_mass[j] * kin.obj_mass[j];
    }
  }
#pragma unroll
  for (int j = 0; j < NF - 2; ++j) {
    if (j >= n - 2) continue;
    y[j] = (2.0 * u[k++] - 1.0) * kin.obj_y_max[j];
    wt *= 2.0 * kin.obj_y_max[j];
  }
  double sx = 0.0, sy = 0.0;
#pragma unroll
  for (int j = 0; j < NF - 1; ++j) {
    if (j >= n - 1) continue;
    const double l0 = log(kin.obj_pt_min[j] * kin.obj_pt_min[j] + m2[j]);
    const double l1 = log(kin.obj_pt_max[j] * kin.obj_pt_max[j] + m2[j]);
    const double l = l0 + u[k++] * (l1 - l0);
    const double e = exp(l);
    const double pt = sqrt(fmax(e - m2[j], 0.0));
    double sp, cp;
    sincospi(2.0 * u[k++], &sp, &cp);
    px[j] = pt * cp;
    py[j] = pt * sp;
    sx += px[j];
    sy += py[j];
    wt *= kPi_ * e * (l1 - l0);
  }
  // light-cone components P+- = mT exp(+-y); E = (P+ + P-)/2 and pz = (P+ - P-)/2 are formed from
  // them so that the balance sum P+- = sqrt_s also holds for the stored momenta
  double mt[NF], lp[NF], lm[NF];
  double ap = w, am = w;
#pragma unroll
  for (int j = 0; j < NF; ++j) {
    if (j == n - 1) { px[j] = -sx; py[j] = -sy; }
    mt[j] = sqrt(px[j] * px[j] + py[j] * py[j] + m2[j]);
    lp[j] = lm[j] = 0.0;
    if (j < n - 2) {
      const double ey = exp(y[j]);
      lp[j] = mt[j] * ey;
      lm[j] = mt[j] / ey;
      ap -= lp[j];
      am -= lm[j];
    }
  }
  if (!(ap > 0.0 && am > 0.0)) return false;
  double a = 0.0, b = 0.0;
#pragma unroll
  for (int j = 0; j < NF; ++j) {
    if (j == n - 2) a = mt[j];
    if (j == n - 1) b = mt[j];
  }
  const double msq = ap * am, c = msq + a * a - b * b, d = c * c - 4.0 * msq * a * a;
  if (!(d >= 0.0)) return false;
  // the larger root without cancellation, the smaller one from the product of the roots a^2 ap / am
  const double big = (c + sqrt(d)) / (2.0 * am);
  const double x = u[k++] < 0.5 ? big : a * a * ap / (am * big);
  const double z = ap - x;
  if (!(x > 0.0 && z > 0.0)) return false;
  const double ya = log(x / a), yb = log(z / b);
  const double r = (z * a) / (x * b);  // exp(y_b - y_a): Jacobian 2 mT_a mT_b |sinh(y_b - y_a)|
  const double jac = a * b * fabs(r - 1.0 / r);
  if (!(jac > 0.0)) return false;
  wt *= 4.0 / jac;
  double ymax_a = 0.0, ymax_b = 0.0, ptmin_b = 0.0, ptmax_b = 0.0, ptb = 0.0;
#pragma unroll
  for (int j = 0; j < NF; ++j) {
    if (j == n - 2) { y[j] = ya; ymax_a = kin.obj_y_max[j]; lp[j] = x; lm[j] = a * a / x; }
    if (j == n - 1) {
      y[j] = yb;
      lp[j] = z;
      lm[j] = b * b / z;
      ymax_b = kin.obj_y_max[j];
      ptmin_b = kin.obj_pt_min[j];
      ptmax_b = kin.obj_pt_max[j];
      ptb = sqrt(px[j] * px[j] + py[j] * py[j]);
    }
  }
  if (!(fabs(ya) <= ymax_a && fabs(yb) <= ymax_b && ptb >= ptmin_b && ptb <= ptmax_b)) return false;
  // (2 pi)^(4 - 3n) 2^-n
  double f = 1.0;
#pragma unroll
  for (int j = 0; j < NF; ++j)
    if (j < n) f *= 1.0 / (2.0 * (2.0 * kPi_) * (2.0 * kPi_) * (2.0 * kPi_));
  wt *= f * (2.0 * kPi_) * (2.0 * kPi_) * (2.0 * kPi_) * (2.0 * kPi_);
#pragma unroll
  for (int j = 0; j < NF; ++j) {
    if (j >= n) continue;
    const double e = 0.5 * (lp[j] + lm[j]), pz = 0.5 * (lp[j] - lm[j]);
    const int l0 = kin.obj_legs[j][0], l1 = kin.obj_legs[j][1];
    if (l1 < 0) {
#pragma unroll
      for (int q = 2; q < NEXT; ++q)
        if (q == l0) set4(p[q], e, px[j], py[j], pz);
      continue;
    }
    const double M = sqrt(m2[j]);
    const double P[4] = {e, px[j], py[j], pz};
    double nx, ny, nz;
    direction(u[k], u[k + 1], nx, ny, nz);
    k += 2;
    const double kd = 0.5 * M;
    double d1[4] = {kd, kd * nx, kd * ny, kd * nz}, d2[4] = {kd, -kd * nx, -kd * ny, -kd * nz};
    boost_from_rest(d1, P, M);
    boost_from_rest(d2, P, M);
#pragma unroll
    for (int q = 2; q < NEXT; ++q) {
      if (q == l0) set4(p[q], d1[0], d1[1], d1[2], d1[3]);
      if (q == l1) set4(p[q], d2[0], d2[1], d2[2], d2[3]);
    }
    wt *= kd / (4.0 * kPi_ * M);
  }
  wps = wt;
  shat = w * w;
  return true;
}

// g g > t t~ > (b (e+ ve)) (b~ (e- ve~)); legs g g b e+ ve b~ e- ve~
template <int NEXT>
__host__ __device__ __forceinline__ bool gen_ttbar(const KinDev& kin, const double* u, double (&p)[NEXT][4],
                                                   double& wps, double& shat) {
  if constexpr (NEXT != 8) {
    return false;
  } else {
    const double rs = kin.sqrt_s_min + (kin.sqrt_s_max - kin.sqrt_s_min) * u[0];
    shat = rs * rs;
    double jt, jtb, jwp, jwm;
    const double st = bw_draw(kin.bw_mass[0], kin.bw_width[0], kin.bw_t0[0], kin.bw_t1[0], u[1], jt);
    const double stb = bw_draw(kin.bw_mass[0], kin.bw_width[0], kin.bw_t0[0], kin.bw_t1[0], u[2], jtb);
    const double swp = bw_draw(kin.bw_mass[1], kin.bw_width[1], kin.bw_t0[1], kin.bw_t1[1], u[3], jwp);
    const double swm = bw_draw(kin.bw_mass[1], kin.bw_width[1], kin.bw_t0[1], kin.bw_t1[1], u[4], jwm);
    if (!(st > 0 && stb > 0 && swp > 0 && swm > 0)) return false;
    const double mt = sqrt(st), mtb = sqrt(stb), mwp = sqrt(swp), mwm = sqrt(swm);
    if (!(mwp <= mt && mwm <= mtb && mt + mtb <= rs)) return false;
    beams<NEXT>(p, rs);
    const double inv4pi = 1.0 / (4.0 * 3.14159265358979323846);
    double nx, ny, nz;
    // production in the CM frame
    const double kp = kallen_sqrt(shat, st, stb) / (2.0 * rs);
    direction(u[5], u[6], nx, ny, nz);
    double T[4], TB[4];
    set4(T, sqrt(st + kp * kp), kp * nx, kp * ny, kp * nz);
    set4(TB, sqrt(stb + kp * kp), -kp * nx, -kp * ny, -kp * nz);
    // t -> b W+
    const double kt = (st - swp) / (2.0 * mt);
    direction(u[7], u[8], nx, ny, nz);
    double WP[4];
    set4(p[2], kt, kt * nx, kt * ny, kt * nz);
    set4(WP, sqrt(swp + kt * kt), -kt * nx, -kt * ny, -kt * nz);
    boost_from_rest(p[2], T, mt);
    boost_from_rest(WP, T, mt);
    // W+ -> e+ ve
    const double kw = 0.5 * mwp;
    direction(u[9], u[10], nx, ny, nz);
    set4(p[3], kw, kw * nx, kw * ny, kw * nz);
    set4(p[4], kw, -kw * nx, -kw * ny, -kw * nz);
    boost_from_rest(p[3], WP, mwp);
    boost_from_rest(p[4], WP, mwp);
    // t~ -> b~ W-
    const double ktb = (stb - swm) / (2.0 * mtb);
    direction(u[11], u[12], nx, ny, nz);
    double WM[4];
    set4(p[5], ktb, ktb * nx, ktb * ny, ktb * nz);
    set4(WM, sqrt(swm + ktb * ktb), -ktb * nx, -ktb * ny, -ktb * nz);
    boost_from_rest(p[5], TB, mtb);
    boost_from_rest(WM, TB, mtb);
    // W- -> e- ve~
    const double kw2 = 0.5 * mwm;
    direction(u[13], u[14], nx, ny, nz);
    set4(p[6], kw2, kw2 * nx, kw2 * ny, kw2 * nz);
    set4(p[7], kw2, -kw2 * nx, -kw2 * ny, -kw2 * nz);
    boost_from_rest(p[6], WM, mwm);
    boost_from_rest(p[7], WM, mwm);
    wps = (kp * inv4pi / rs) * jt * jtb * jwp * jwm * (kt * inv4pi / mt) * (kw * inv4pi / mwp) *
          (ktb * inv4pi / mtb) * (kw2 * inv4pi / mwm);
    return true;
  }
}

// ---------------------------------------------------------------------------
// cuts: pT > pt_min, |eta| < eta_max, Delta R > dr_min over kin.cut_legs.
// pT and |eta| (as |pz| < sinh(eta_max) pT) are exact FP64 comparisons.  A pair
// is separated when its azimuthal or its pseudorapidity distance alone exceeds
// dr_min; both tests run first in FP32 and decide only outside a 1e-5 relative
// guard band around the boundary (FP32 rounding and the approximate reciprocal
// square roots of the mixed path stay below 1e-6 here), else the same test runs
// in FP64.  Only pairs close in both evaluate Delta R with asinh
// and atan2 in FP64.  The decision therefore equals the FP64 one.
// ---------------------------------------------------------------------------
// returns +1 (certainly x > y), -1 (certainly x < y) or 0 (undecided) for float estimates
__host__ __device__ __forceinline__ int fcmp(float x, float y, float scale) {
  const float band = 1e-5f * scale;
  if (x > y + band) return 1;
  if (x < y - band) return -1;
  return 0;
}

template <int NEXT>
__host__ __device__ __forceinline__ bool pass_cuts(const KinDev& kin, const double (&p)[NEXT][4]) {
  const uint32_t mask = kin.cut_mask;
  if (mask == 0) return true;
  // loops run over every leg with compile-time indices (registers, no local memory)
  double pt2[NEXT];
  float ptf[NEXT], af[NEXT], rf[NEXT];
#pragma unroll
  for (int i = 2; i < NEXT; ++i) {
    if (!((mask >> i) & 1u)) continue;
    const double* q = p[i];
    pt2[i] = q[1] * q[1] + q[2] * q[2];
    if (!(pt2[i] > kin.pt_min * kin.pt_min)) return false;
    if (!(q[3] * q[3] < kin.sinh2_eta_max * pt2[i])) return false;
    const float p2f = (float)pt2[i], zf = (float)q[3];
    ptf[i] = sqrtf(p2f);
    const float ip = 1.0f / ptf[i];
    af[i] = zf * ip;                          // sinh(eta)
    rf[i] = sqrtf(p2f + zf * zf) * ip;        // cosh(eta)
  }
  const float cdr = kin.f_cdr, chd = kin.f_chd, shd = kin.f_shd;
#pragma unroll
  for (int i = 2; i < NEXT; ++i) {
#pragma unroll
    for (int j = i + 1; j < NEXT; ++j) {
      if (!((mask >> i) & 1u) || !((mask >> j) & 1u)) continue;
      const double* qi = p[i];
      const double* qj = p[j];
      // |d_phi| > dr_min  <=>  pT_i . pT_j < cos(dr_min) |pT_i| |pT_j|
      const float dotf = (float)qi[1] * (float)qj[1] + (float)qi[2] * (float)qj[2];
      const float ptijf = ptf[i] * ptf[j];
      int c = fcmp(dotf, cdr * ptijf, ptijf);
      if (c == 0) {
        const double dot = qi[1] * qj[1] + qi[2] * qj[2];
        c = dot < kin.cos_dr * sqrt(pt2[i] * pt2[j]) ? -1 : 1;
      }
      if (c < 0) continue;
      // eta_i - eta_j > dr_min  <=>  sinh(eta_i) > sinh(eta_j) cosh(dr) + cosh(eta_j) sinh(dr), and i <-> j
      const float sc = fabsf(af[i]) + fabsf(af[j]) + rf[i] + rf[j];
      int e1 = fcmp(af[i], af[j] * chd + rf[j] * shd, sc);
      int e2 = fcmp(af[j], af[i] * chd + rf[i] * shd, sc);
      if (e1 == 0 || e2 == 0) {
        const double ipi = 1.0 / sqrt(pt2[i]), ipj = 1.0 / sqrt(pt2[j]);
        const double ai = qi[3] * ipi, aj = qj[3] * ipj;
        const double ri = sqrt(pt2[i] + qi[3] * qi[3]) * ipi, rj = sqrt(pt2[j] + qj[3] * qj[3]) * ipj;
        e1 = ai > aj * kin.cosh_dr + rj * kin.sinh_dr ? 1 : -1;
        e2 = aj > ai * kin.cosh_dr + ri * kin.sinh_dr ? 1 : -1;
      }
      if (e1 > 0 || e2 > 0) continue;
      // close in both: Delta R^2 = d_eta^2 + d_phi^2 in FP64
      const double ipi = 1.0 / sqrt(pt2[i]), ipj = 1.0 / sqrt(pt2[j]);
      const double deta = asinh(qi[3] * ipi) - asinh(qj[3] * ipj);
      const double dot = qi[1] * qj[1] + qi[2] * qj[2];
      const double cross = qi[1] * qj[2] - qi[2] * qj[1];
      const double dphi = atan2(fabs(cross), dot);
      if (!(deta * deta + dphi * dphi > kin.dr_min * kin.dr_min)) return false;
    }
  }
  return true;
}

// The paper's selection (Eqs. 8-11), kin.cut_mode == 1 (with the y/pT generator), in FP64: per leg
// class, jets |eta| < jet_eta
// and pT > jet_pt with min(pT_i, pT_j) Delta R_ij > jet_ptij for every pair of jets; b jets and
// charged leptons pT and |eta| only (not isolated).
template <int NEXT>
__host__ __device__ __forceinline__ bool pass_paper_cuts(const KinDev& kin, const double (&p)[NEXT][4]) {
  if (kin.cut_mode != 1) return true;
  double pt[NEXT], eta[NEXT], phi[NEXT];
#pragma unroll
  for (int i = 2; i < NEXT; ++i) {
    const int cl = kin.leg_class[i];
    if (cl == 0) continue;
    pt[i] = sqrt(p[i][1] * p[i][1] + p[i][2] * p[i][2]);
    if (!(pt[i] > 0.0)) return false;
    eta[i] = asinh(p[i][3] / pt[i]);
    phi[i] = atan2(p[i][2], p[i][1]);
    const double ptmin = cl == 1 ? kin.jet_pt : (cl == 2 ? kin.b_pt : kin.lep_pt);
    const double etamax = cl == 1 ? kin.jet_eta : (cl == 2 ? kin.b_eta : kin.lep_eta);
    if (!(pt[i] > ptmin && fabs(eta[i]) < etamax)) return false;
  }
#pragma unroll
  for (int i = 2; i < NEXT; ++i) {
#pragma unroll
    for (int j = i + 1; j < NEXT; ++j) {
      if (kin.leg_class[i] != 1 || kin.leg_class[j] != 1) continue;
      const double deta = eta[i] - eta[j];
      double dphi = fabs(phi[i] - phi[j]);
      if (dphi > 3.14159265358979323846) dphi = 2.0 * 3.14159265358979323846 - dphi;
      if (!(fmin(pt[i], pt[j]) * sqrt(deta * deta + dphi * dphi) > kin.jet_ptij)) return false;
    }
  }
  return true;
}

// Generator kind as a template argument: kKindAny reads kin.kind at run time;
// a fixed kind compiles only that generator (smaller code, fewer registers).  The y/pT
// generator is compiled only where it is the fixed kind (k_ps, k_gen): the fused kernels,
// which dispatch at run time and hold the |M|^2 program's registers, leave it out.
// kKindRamboMassive is RAMBO with the massive rescaling; ME_PS_RAMBO as a fixed
// kind on the mixed path is massless RAMBO.  The grid map runs where `bins` is
// not null (the caller passes null unless kin carries a grid).
constexpr int kKindAny = -1;
constexpr int kKindRamboMassive = 100 + ME_PS_RAMBO;

// one draw (attempt `att`) for `event`: false if outside the kinematic limits or the cuts
template <int NEXT, int KIND = kKindAny>
__host__ __device__ __forceinline__ bool draw_point(const KinDev& kin, uint64_t seed, uint64_t event, int att,
                                                    double (&p)[NEXT][4], double& wps, double& shat,
                                                    uint8_t* bins = nullptr) {
  bool ok;
  double jac = 1.0;
  const int kind = KIND == kKindAny ? kin.kind : KIND == kKindRamboMassive ? ME_PS_RAMBO : KIND;
  if (kind == ME_PS_TWO_BODY) {
    double u[2];
    draw_uniforms<2>(seed, event, (uint64_t)att, u);
#pragma unroll
    for (int d = 0; d < 2; ++d)  // compile-time indices keep u in registers
      if (bins && d < kin.vg_dims) u[d] = vg_map(kin, d, u[d], jac, bins);
    ok = gen_two_body<NEXT>(kin, u, p, wps, shat);
  } else if (kind == ME_PS_RAMBO || kind == ME_PS_RAMBO_BW) {
    double u[4 * (NEXT - 2)];
    draw_uniforms<4 * (NEXT - 2)>(seed, event, (uint64_t)att, u);
#pragma unroll
    for (int d = 0; d < 4 * (NEXT - 2); ++d)
      if (bins && d < kin.vg_dims) u[d] = vg_map(kin, d, u[d], jac, bins);
    if (kind == ME_PS_RAMBO) ok = gen_rambo<NEXT>(kin, u, p, wps, shat);
    else if constexpr (NEXT >= 5) ok = gen_rambo_bw<NEXT>(kin, u, p, wps, shat);
    else ok = false;
  } else if (KIND == ME_PS_YPT && kind == ME_PS_YPT) {
    constexpr int NU = 3 * (NEXT - 2) - 3;
    double u[NU];
    draw_uniforms<NU>(seed, event, (uint64_t)att, u);
#pragma unroll
    for (int d = 0; d < NU; ++d)
      if (bins && d < kin.vg_dims) u[d] = vg_map(kin, d, u[d], jac, bins);
    ok = gen_ypt<NEXT>(kin, u, p, wps, shat);
  } else {
    double u[16];
    draw_uniforms<16>(seed, event, (uint64_t)att, u);
#pragma unroll
    for (int d = 0; d < 16; ++d)
      if (bins && d < kin.vg_dims) u[d] = vg_map(kin, d, u[d], jac, bins);
    ok = gen_ttbar<NEXT>(kin, u, p, wps, shat);
  }
  wps *= jac;
  if (kind == ME_PS_YPT) return ok && pass_cuts<NEXT>(kin, p) && pass_paper_cuts<NEXT>(kin, p);
  return ok && pass_cuts<NEXT>(kin, p);
}

// ---------------------------------------------------------------------------
// Mixed-precision phase space: RAMBO in double-float arithmetic (FP32 pairs,
// ~2^-48 relative) on the FP32 pipe, the same formulas and draw order as
// gen_rambo; the tt~ chain in double-float below.
// ---------------------------------------------------------------------------
template <int NEXT>
__host__ __device__ __forceinline__ void rambo_df(const KinDev& kin, uint64_t seed, uint64_t event, int att,
                                         df (&p)[NEXT][4], df& jac, uint8_t* bins = nullptr) {
  constexpr int NF = NEXT - 2;
  const df w = df{kin.sqrt_s_f[0], kin.sqrt_s_f[1]};
  const df hw = df{w.hi * 0.5f, w.lo * 0.5f};
  const df z = df{0.0f, 0.0f};
  p[0][0] = hw; p[0][1] = z; p[0][2] = z; p[0][3] = hw;
  p[1][0] = hw; p[1][1] = z; p[1][2] = z; p[1][3] = -hw;
  df Q0 = z, Q1 = z, Q2 = z, Q3 = z;
  uint64_t o[4];  // Philox block k / 2: uniforms 4k .. 4k+3 are words 2 (k % 2) and 2 (k % 2) + 1
#pragma unroll 1  // one copy of the per-particle code: the unrolled form overflows the instruction cache
  for (int k = 0; k < NF; ++k) {
    if ((k & 1) == 0) Philox::block(event, (uint64_t)att, (uint64_t)(k >> 1), 0ull, seed, 0ull, o);
    const uint64_t wa = (k & 1) ? o[2] : o[0], wb = (k & 1) ? o[3] : o[1];
    df u0 = unit_df32((uint32_t)wa), u1 = unit_df32((uint32_t)(wa >> 32));
    df u2 = unit_df32((uint32_t)wb), u3 = unit_df32((uint32_t)(wb >> 32));
    if (bins) {
      u0 = vg_map_df(kin, 4 * k + 0, u0, jac, bins);
      u1 = vg_map_df(kin, 4 * k + 1, u1, jac, bins);
      u2 = vg_map_df(kin, 4 * k + 2, u2, jac, bins);
      u3 = vg_map_df(kin, 4 * k + 3, u3, jac, bins);
    }
    const df c = df{u0.hi * 2.0f, u0.lo * 2.0f} + (-1.0f);
    const df sn = df_sqrt((dfs(1.0f) - c) * (dfs(1.0f) + c));
    df sp, cp;
    df_sincospi(df{u1.hi * 2.0f, u1.lo * 2.0f}, sp, cp);
    const df q0 = -df_log(u2 * u3);
    const df qs = q0 * sn;
    p[2 + k][0] = q0;
    p[2 + k][1] = qs * cp;
    p[2 + k][2] = qs * sp;
    p[2 + k][3] = q0 * c;
    Q0 = sadd(Q0, p[2 + k][0]); Q1 = sadd(Q1, p[2 + k][1]); Q2 = sadd(Q2, p[2 + k][2]); Q3 = sadd(Q3, p[2 + k][3]);
  }
  const df M = df_sqrt(ssub(ssub(ssub(sqr(Q0), sqr(Q1)), sqr(Q2)), sqr(Q3)));
  const df iM = dfs(1.0f) / M;
  const df b1 = -(Q1 * iM), b2 = -(Q2 * iM), b3 = -(Q3 * iM);
  const df gam = Q0 * iM;
  const df a = dfs(1.0f) / (gam + 1.0f);
  const df x = w * iM;
#pragma unroll 1
  for (int k = 0; k < NF; ++k) {
    df* q = p[2 + k];
    const df bq = sadd(sadd(b1 * q[1], b2 * q[2]), b3 * q[3]);
    const df q0 = q[0];
    const df c = sadd(q0, a * bq);
    q[0] = x * sadd(gam * q0, bq);
    q[1] = x * sadd(q[1], b1 * c);
    q[2] = x * sadd(q[2], b2 * c);
    q[3] = x * sadd(q[3], b3 * c);
  }
}

// approximate 1/sqrt(x) and x/y (the device's fast forms; plain IEEE on the host)
__host__ __device__ __forceinline__ float approx_rsqrt(float x) {
#ifdef __CUDA_ARCH__
  return rsqrtf(x);
#else
  return 1.0f / sqrtf(x);
#endif
}
__host__ __device__ __forceinline__ float approx_div(float x, float y) {
#ifdef __CUDA_ARCH__
  return __fdividef(x, y);
#else
  return x / y;
#endif
}

// Massive RAMBO rescaling in double-float: the massless momenta of rambo_df are
// scaled so that every final particle gets its mass at fixed total energy w
// (the same equation as gen_rambo: sum_k sqrt(m_k^2 + xi^2 E_k^2) = w).  xi is
// found by Newton's method in FP32 from the same start, then refined by two
// double-float Newton steps (quadratic convergence: FP32 accuracy squared is
// below the double-float rounding).  Massless particles take e_k = xi E_k exactly.  Returns the factor of the weight,
// xi^(2n-3) prod_k(|p_k|/E_k) w / sum_k(|p_k|^2/E_k).
template <int NEXT>
__host__ __device__ __forceinline__ df massive_rescale_df(const KinDev& kin, df (&p)[NEXT][4],
                                                         const df* mass = nullptr) {
  constexpr int NF = NEXT - 2;
  const df w = df{kin.sqrt_s_f[0], kin.sqrt_s_f[1]};
  df E0[NF], m2[NF];
  float msum = 0.0f;
#pragma unroll
  for (int k = 0; k < NF; ++k) {
    E0[k] = p[2 + k][0];
    const df m = mass ? mass[k] : from_double(kin.mass[2 + k]);
    m2[k] = sqr(m);
    msum += m.hi;
  }
  const float r = msum / w.hi;
  float xf = sqrtf(fmaxf(1.0f - r * r, 0.0f));
  // FP32 stage with approximate square roots and quotients, until the step falls below 2^-22 x
  // (at most 12 iterations): it only starts the double-float steps, which square its error.
  // Massless particles (m = 0, the same in every thread) contribute x E exactly.
  for (int it = 0; it < 12; ++it) {
    float f = -w.hi, d = 0.0f;
#pragma unroll
    for (int k = 0; k < NF; ++k) {
      const float e = E0[k].hi;
      if (m2[k].hi == 0.0f) {
        f += xf * e;
        d += e;
      } else {
        const float q = m2[k].hi + xf * xf * e * e;
        const float rq = approx_rsqrt(q);
        f += q * rq;
        d += xf * e * e * rq;
      }
    }
    const float dx = approx_div(f, d);
    xf -= dx;
    if (fabsf(dx) <= 0x1p-22f * xf) break;
  }
  df X = dfs(xf);
#pragma unroll
  for (int it = 0; it < 2; ++it) {
    df f = -w, d = dfs(0.0f);
#pragma unroll
    for (int k = 0; k < NF; ++k) {
      const df ak = X * E0[k];
      if (m2[k].hi == 0.0f) {  // e_k = x E_k
        f = f + ak;
        d = d + E0[k];
      } else {
        const df ek = df_sqrt(m2[k] + sqr(ak));
        f = f + ek;
        d = d + (ak * E0[k]) / ek;
      }
    }
    X = X - f / d;
  }
  df prod = dfs(1.0f), sum = dfs(0.0f);
#pragma unroll
  for (int k = 0; k < NF; ++k) {
    const df ak = X * E0[k];
    if (m2[k].hi == 0.0f) {  // |p_k| / e_k = 1, |p_k|^2 / e_k = |p_k|
      sum = sum + ak;
      p[2 + k][0] = ak;
    } else {
      const df ek = df_sqrt(m2[k] + sqr(ak));
      prod = prod * (ak / ek);
      sum = sum + sqr(ak) / ek;
      p[2 + k][0] = ek;
    }
    p[2 + k][1] = p[2 + k][1] * X;
    p[2 + k][2] = p[2 + k][2] * X;
    p[2 + k][3] = p[2 + k][3] * X;
  }
  df xp = dfs(1.0f);
#pragma unroll
  for (int i = 0; i < 2 * NF - 3; ++i) xp = xp * X;
  return ((xp * prod) * w) / sum;
}

// Delta R test of the pairs in `close` (bit k NF + l: legs k + 2 and l + 2, not
// certainly separated by their azimuth or pseudorapidity distance alone) in FP32
// with the guard band, then the FP64 cuts for any undecided point.  Kept out of line: a few lanes of most
// warps take it, and inlined its code and registers slow the common path.
// Returns the decision.
template <int NEXT>
__device__ __noinline__ bool cuts_close_pairs(const KinDev& kin, const df (&p)[NEXT][4], uint64_t close,
                                              bool undecided) {
  constexpr int NF = NEXT - 2;
  const float dr2 = kin.f_dr2;
  while (close && !undecided) {
    const int b = __ffsll((long long)close) - 1;
    close &= close - 1;
    const int k = b / NF, l = b - (b / NF) * NF;
    const df* qi = p[k + 2];
    const df* qj = p[l + 2];
    const float xi = qi[1].hi, yi = qi[2].hi, xj = qj[1].hi, yj = qj[2].hi;
    const float deta = asinhf(qi[3].hi * rsqrtf(xi * xi + yi * yi)) - asinhf(qj[3].hi * rsqrtf(xj * xj + yj * yj));
    const float dphi = atan2f(fabsf(xi * yj - yi * xj), xi * xj + yi * yj);
    const float r2 = deta * deta + dphi * dphi;
    const int r = fcmp(r2, dr2, dr2 + r2);
    if (r < 0) return false;
    undecided |= (r == 0);
  }
  if (!undecided) return true;
  double pd[NEXT][4];
#pragma unroll
  for (int k = 0; k < NEXT; ++k) {
#pragma unroll
    for (int m = 0; m < 4; ++m) pd[k][m] = to_double(p[k][m]);
  }
  return pass_cuts<NEXT>(kin, pd);
}

// cuts on double-float momenta: FP32 estimates decide outside a 1e-5 guard band;
// a point with any undecided test is decided by the FP64 cuts on its momenta.
// The per-leg quantities and the pair pre-tests (azimuth, then pseudorapidity
// through sinh/cosh) stay in registers; pairs not certainly separated by one of them
// go to cuts_close_pairs.
template <int NEXT>
__host__ __device__ __forceinline__ bool pass_cuts_df(const KinDev& kin, const df (&p)[NEXT][4]) {
  const uint32_t mask = kin.cut_mask;
  if (mask == 0) return true;
  constexpr int NF = NEXT - 2;
  const float ptmin2 = kin.f_ptmin2, sh2 = kin.f_sinh2;
  const float cdr = kin.f_cdr, chd = kin.f_chd, shd = kin.f_shd;
  float px[NF], py[NF], pt[NF], a[NF], r[NF];  // a = sinh(eta), r = cosh(eta)
  bool undecided = false;
#pragma unroll
  for (int k = 0; k < NF; ++k) {
    px[k] = p[k + 2][1].hi;
    py[k] = p[k + 2][2].hi;
    pt[k] = 1.0f; a[k] = 0.0f; r[k] = 1.0f;
    if (!((mask >> (k + 2)) & 1u)) continue;
    const float z = p[k + 2][3].hi;
    const float pt2 = px[k] * px[k] + py[k] * py[k];
    int c = fcmp(pt2, ptmin2, ptmin2);
    if (c < 0) return false;
    undecided |= (c == 0);
    c = fcmp(z * z, sh2 * pt2, sh2 * pt2 + z * z);
    if (c > 0) return false;
    undecided |= (c == 0);
    // approximate reciprocal square roots (relative error below 3e-7, inside the band)
    const float ip = rsqrtf(pt2);
    const float p2 = pt2 + z * z;
    pt[k] = pt2 * ip;
    a[k] = z * ip;
    r[k] = p2 * rsqrtf(p2) * ip;
  }
  uint64_t close = 0;
#pragma unroll
  for (int k = 0; k < NF; ++k) {
#pragma unroll
    for (int l = k + 1; l < NF; ++l) {
      if (!((mask >> (k + 2)) & 1u) || !((mask >> (l + 2)) & 1u)) continue;
      // |d_phi| > dr_min  <=>  pT_k . pT_l < cos(dr_min) |pT_k| |pT_l|
      const float ptkl = pt[k] * pt[l];
      const int c = fcmp(px[k] * px[l] + py[k] * py[l], cdr * ptkl, ptkl);
      if (c < 0) continue;
      // eta_k - eta_l > dr_min  <=>  sinh(eta_k) > sinh(eta_l) cosh(dr) + cosh(eta_l) sinh(dr), and k <-> l
      const float sc = fabsf(a[k]) + fabsf(a[l]) + r[k] + r[l];
      const int e1 = fcmp(a[k], a[l] * chd + r[l] * shd, sc);
      const int e2 = fcmp(a[l], a[k] * chd + r[k] * shd, sc);
      if (e1 > 0 || e2 > 0) continue;
      close |= 1ull << (k * NF + l);  // Delta R decides (also where a pre-test was in its band)
    }
  }
  if (!undecided && !close) return true;
#ifdef __CUDA_ARCH__
  return cuts_close_pairs<NEXT>(kin, p, close, undecided);
#else
  double pd[NEXT][4];
  for (int k = 0; k < NEXT; ++k)
    for (int m = 0; m < 4; ++m) pd[k][m] = to_double(p[k][m]);
  return pass_cuts<NEXT>(kin, pd);
#endif
}

// ---------------------------------------------------------------------------
// g g > t t~ > (b W+)(b~ W-) in double-float: the formulas and uniforms of
// gen_ttbar (sqrt(s) uniform, Breit-Wigner t, t~, W+, W- virtualities from
// s = m^2 + m G tan(theta), isotropic two-body decays boosted to the lab).  The
// two-body momentum uses the factorised Kallen function
// lambda(s, m1^2, m2^2) = (s - (m1 + m2)^2)(s - (m1 - m2)^2), with
// s - (m1 +- m2)^2 = (rs - m1 -+ m2)(rs + m1 +- m2), which keeps its relative
// accuracy near threshold; the Breit-Wigner Jacobian uses 1 + tan^2.
// ---------------------------------------------------------------------------
__host__ __device__ __forceinline__ void direction_df(df a, df b, df& nx, df& ny, df& nz) {
  const df c = df{a.hi * 2.0f, a.lo * 2.0f} + (-1.0f);
  const df sn = df_sqrt((dfs(1.0f) - c) * (dfs(1.0f) + c));
  df sp, cp;
  df_sincospi(df{b.hi * 2.0f, b.lo * 2.0f}, sp, cp);
  nx = sn * cp;
  ny = sn * sp;
  nz = c;
}

__host__ __device__ __forceinline__ void boost_from_rest_df(df* p, const df* P, df M) {
  const df pp = (P[1] * p[1] + P[2] * p[2]) + P[3] * p[3];
  const df iM = dfs(1.0f) / M;
  const df e = (P[0] * p[0] + pp) * iM;
  const df f = (pp / (P[0] + M) + p[0]) * iM;
  p[0] = e;
  p[1] = p[1] + f * P[1];
  p[2] = p[2] + f * P[2];
  p[3] = p[3] + f * P[3];
}

// s = m^2 + m G tan(theta), theta = t0 + (t1 - t0) u in (-pi/2, pi/2); jac = (t1 - t0) m G (1 + tan^2) / (2 pi)
__host__ __device__ __forceinline__ df bw_draw_df(double m, double g, double t0, double t1, df u, df& jac) {
  const df T0 = from_double(t0), dT = from_double(t1) - T0;
  const df th = T0 + dT * u;
  df x = th * df{kInvPiHi, kInvPiLo};  // theta / pi in (-1/2, 1/2)
  if (x.hi < 0.0f) x = x + 2.0f;        // sin and cos of pi x have period 2
  df sn, cs;
  df_sincospi(x, sn, cs);
  const df t = sn / cs;
  const df M = from_double(m), mg = M * from_double(g);
  jac = (dT * mg) * (sqr(t) + 1.0f) * df{kInv2PiHi, kInv2PiLo};
  return sqr(M) + mg * t;
}

__host__ __device__ __forceinline__ void set4_df(df* p, df e, df x, df y, df z) {
  p[0] = e; p[1] = x; p[2] = y; p[3] = z;
}

// |p*| of the two-body decay of mass rs into masses m1, m2
__host__ __device__ __forceinline__ df two_body_k(df rs, df m1, df m2) {
  const df a = (rs - m1) - m2, b = (rs + m1) + m2, c = (rs - m1) + m2, d = (rs + m1) - m2;
  return df_sqrt((a * b) * (c * d)) / df{rs.hi * 2.0f, rs.lo * 2.0f};
}

template <int NEXT>
__host__ __device__ __forceinline__ bool ttbar_df(const KinDev& kin, uint64_t seed, uint64_t event, int att,
                                                  df (&p)[NEXT][4], double& wps, double& shat, df& jac,
                                                  uint8_t* bins = nullptr) {
  if constexpr (NEXT != 8) {
    return false;
  } else {
    df u[16];
#pragma unroll
    for (int j = 0; j < 2; ++j) {
      uint64_t o[4];
      Philox::block(event, (uint64_t)att, (uint64_t)j, 0ull, seed, 0ull, o);
#pragma unroll
      for (int q = 0; q < 8; ++q) u[8 * j + q] = unit_df32(half32(o[q / 2], q & 1));
    }
#pragma unroll
    for (int d = 0; d < 16; ++d)
      if (bins && d < kin.vg_dims) u[d] = vg_map_df(kin, d, u[d], jac, bins);
    const df rmin = from_double(kin.sqrt_s_min);
    const df rs = rmin + (from_double(kin.sqrt_s_max) - rmin) * u[0];
    df jt, jtb, jwp, jwm;
    const df st = bw_draw_df(kin.bw_mass[0], kin.bw_width[0], kin.bw_t0[0], kin.bw_t1[0], u[1], jt);
    const df stb = bw_draw_df(kin.bw_mass[0], kin.bw_width[0], kin.bw_t0[0], kin.bw_t1[0], u[2], jtb);
    const df swp = bw_draw_df(kin.bw_mass[1], kin.bw_width[1], kin.bw_t0[1], kin.bw_t1[1], u[3], jwp);
    const df swm = bw_draw_df(kin.bw_mass[1], kin.bw_width[1], kin.bw_t0[1], kin.bw_t1[1], u[4], jwm);
    if (!(st.hi > 0.0f && stb.hi > 0.0f && swp.hi > 0.0f && swm.hi > 0.0f)) return false;
    const df mt = df_sqrt(st), mtb = df_sqrt(stb), mwp = df_sqrt(swp), mwm = df_sqrt(swm);
    // kinematic limits, decided in FP64 on the double-float values (as gen_ttbar)
    if (!(to_double(mwp) <= to_double(mt) && to_double(mwm) <= to_double(mtb) &&
          to_double(mt) + to_double(mtb) <= to_double(rs)))
      return false;
    const df z = dfs(0.0f), hw = df{rs.hi * 0.5f, rs.lo * 0.5f};
    set4_df(p[0], hw, z, z, hw);
    set4_df(p[1], hw, z, z, -hw);
    df nx, ny, nz;
    // production in the CM frame
    const df kp = two_body_k(rs, mt, mtb);
    direction_df(u[5], u[6], nx, ny, nz);
    df T[4], TB[4];
    set4_df(T, df_sqrt(st + sqr(kp)), kp * nx, kp * ny, kp * nz);
    set4_df(TB, df_sqrt(stb + sqr(kp)), -(kp * nx), -(kp * ny), -(kp * nz));
    // t -> b W+
    const df kt = (st - swp) / df{mt.hi * 2.0f, mt.lo * 2.0f};
    direction_df(u[7], u[8], nx, ny, nz);
    df WP[4];
    set4_df(p[2], kt, kt * nx, kt * ny, kt * nz);
    set4_df(WP, df_sqrt(swp + sqr(kt)), -(kt * nx), -(kt * ny), -(kt * nz));
    boost_from_rest_df(p[2], T, mt);
    boost_from_rest_df(WP, T, mt);
    // W+ -> e+ ve
    const df kw = df{mwp.hi * 0.5f, mwp.lo * 0.5f};
    direction_df(u[9], u[10], nx, ny, nz);
    set4_df(p[3], kw, kw * nx, kw * ny, kw * nz);
    set4_df(p[4], kw, -(kw * nx), -(kw * ny), -(kw * nz));
    boost_from_rest_df(p[3], WP, mwp);
    boost_from_rest_df(p[4], WP, mwp);
    // t~ -> b~ W-
    const df ktb = (stb - swm) / df{mtb.hi * 2.0f, mtb.lo * 2.0f};
    direction_df(u[11], u[12], nx, ny, nz);
    df WM[4];
    set4_df(p[5], ktb, ktb * nx, ktb * ny, ktb * nz);
    set4_df(WM, df_sqrt(swm + sqr(ktb)), -(ktb * nx), -(ktb * ny), -(ktb * nz));
    boost_from_rest_df(p[5], TB, mtb);
    boost_from_rest_df(WM, TB, mtb);
    // W- -> e- ve~
    const df kw2 = df{mwm.hi * 0.5f, mwm.lo * 0.5f};
    direction_df(u[13], u[14], nx, ny, nz);
    set4_df(p[6], kw2, kw2 * nx, kw2 * ny, kw2 * nz);
    set4_df(p[7], kw2, -(kw2 * nx), -(kw2 * ny), -(kw2 * nz));
    boost_from_rest_df(p[6], WM, mwm);
    boost_from_rest_df(p[7], WM, mwm);
    // (kp / (4 pi rs)) (kt / (4 pi mt)) (kw / (4 pi mW+)) (ktb / (4 pi mt~)) (kw2 / (4 pi mW-)) x Jacobians
    const df i4p = df{kInv4PiHi, kInv4PiLo};
    const df w1 = (kp / rs) * (kt / mt), w2 = (kw / mwp) * (ktb / mtb), w3 = kw2 / mwm;
    const df i4p2 = sqr(i4p);
    const df jac = (jt * jtb) * (jwp * jwm);
    const df wt = ((((w1 * w2) * w3) * jac) * (i4p2 * i4p2)) * i4p;
    wps = to_double(wt);
    shat = to_double(sqr(rs));
    return true;
  }
}

// resonance-mapped RAMBO in double-float (gen_rambo_bw's formulas and uniforms)
template <int NEXT>
__host__ __device__ __forceinline__ bool rambo_bw_df(const KinDev& kin, uint64_t seed, uint64_t event, int att,
                                                     df (&p)[NEXT][4], double& wps, df& jac, uint8_t* bins) {
  constexpr int NR = NEXT - 3;
  uint64_t o[4];
  // uniforms 4 NR, 4 NR + 1, 4 NR + 2: block NR / 2, words 2 (NR % 2) and 2 (NR % 2) + 1
  Philox::block(event, (uint64_t)att, (uint64_t)(NR / 2), 0ull, seed, 0ull, o);
  constexpr int WB = 2 * (NR % 2);
  df ub = unit_df32((uint32_t)o[WB]), ud0 = unit_df32((uint32_t)(o[WB] >> 32)), ud1 = unit_df32((uint32_t)o[WB + 1]);
  if (bins) {
    ub = vg_map_df(kin, 4 * NR, ub, jac, bins);
    ud0 = vg_map_df(kin, 4 * NR + 1, ud0, jac, bins);
    ud1 = vg_map_df(kin, 4 * NR + 2, ud1, jac, bins);
  }
  df jbw;
  const df s = bw_draw_df(kin.bw_mass[0], kin.bw_width[0], kin.bw_t0[0], kin.bw_t1[0], ub, jbw);
  if (!(s.hi > 0.0f)) return false;
  const df M = df_sqrt(s);
  if (!(to_double(M) < kin.sqrt_s)) return false;
  df q[NR + 2][4];
  rambo_df<NR + 2>(kin, seed, event, att, q, jac, bins);
  df masses[NR];
#pragma unroll
  for (int k = 0; k < NR; ++k) masses[k] = k == 0 ? M : dfs(0.0f);
  const df fac = massive_rescale_df<NR + 2>(kin, q, masses);
  df nx, ny, nz;
  direction_df(ud0, ud1, nx, ny, nz);
  const df kd = df{M.hi * 0.5f, M.lo * 0.5f};
#pragma unroll
  for (int mu = 0; mu < 4; ++mu) {
    p[0][mu] = q[0][mu];
    p[1][mu] = q[1][mu];
  }
  set4_df(p[2], kd, kd * nx, kd * ny, kd * nz);
  set4_df(p[3], kd, -(kd * nx), -(kd * ny), -(kd * nz));
  boost_from_rest_df(p[2], q[2], M);
  boost_from_rest_df(p[3], q[2], M);
#pragma unroll
  for (int k = 1; k < NR; ++k) {
#pragma unroll
    for (int mu = 0; mu < 4; ++mu) p[3 + k][mu] = q[2 + k][mu];
  }
  wps = kin.rambo_volume * to_double(((fac * jbw) * (kd / M)) * df{kInv4PiHi, kInv4PiLo});
  return true;
}

// the generators that run in FP64 on the mixed path too (two-body, y/pT), their momenta split into
// double-floats
template <int NEXT, int KIND>
__host__ __device__ __forceinline__ bool draw_point_fp64_df(const KinDev& kin, uint64_t seed, uint64_t event, int att,
                                                         df (&p)[NEXT][4], double& wps, double& shat, uint8_t* bins) {
  double pd[NEXT][4];
  const bool ok = draw_point<NEXT, KIND>(kin, seed, event, att, pd, wps, shat, bins);
  if (ok) {
#pragma unroll
    for (int k = 0; k < NEXT; ++k) {
#pragma unroll
      for (int m = 0; m < 4; ++m) p[k][m] = from_double(pd[k][m]);
    }
  }
  return ok;
}

// one mixed-precision draw: double-float RAMBO (massless, with the massive
// rescaling, or resonance-mapped) or tt~ chain; the two-body and y/pT generators in
// FP64 split into double-floats
template <int NEXT, int KIND = kKindAny>
__host__ __device__ __forceinline__ bool draw_point_df(const KinDev& kin, uint64_t seed, uint64_t event, int att,
                                              df (&p)[NEXT][4], double& wps, double& shat,
                                              uint8_t* bins = nullptr) {
  df jac = dfs(1.0f);
  const int kind = KIND == kKindAny ? kin.kind : KIND == kKindRamboMassive ? ME_PS_RAMBO : KIND;
  const bool massive = KIND == kKindAny ? kin.massive != 0 : KIND == kKindRamboMassive;
  if (kind == ME_PS_RAMBO) {
    rambo_df<NEXT>(kin, seed, event, att, p, jac, bins);
    wps = kin.rambo_volume;
    if (massive) wps *= to_double(massive_rescale_df<NEXT>(kin, p));
    if (bins) wps *= to_double(jac);
    shat = kin.shat_fixed;
    return pass_cuts_df<NEXT>(kin, p);
  }
  if (kind == ME_PS_RAMBO_BW) {
    if constexpr (NEXT >= 5) {
      const bool ok = rambo_bw_df<NEXT>(kin, seed, event, att, p, wps, jac, bins);
      if (bins) wps *= to_double(jac);
      shat = kin.shat_fixed;
      return ok && pass_cuts_df<NEXT>(kin, p);
    } else {
      return false;
    }
  }
  if (kind == ME_PS_TTBAR) {
    const bool ok = ttbar_df<NEXT>(kin, seed, event, att, p, wps, shat, jac, bins);
    if (bins) wps *= to_double(jac);
    return ok && pass_cuts_df<NEXT>(kin, p);
  }
  return draw_point_fp64_df<NEXT, KIND>(kin, seed, event, att, p, wps, shat, bins);
}

}  // namespace me
