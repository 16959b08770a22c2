// Device library of helicity wavefunctions and vertex functions (the role of
// the paper's HEGET functions, Sect. 4 and App. C), written for sm_103a.
//
// Differences from the paper's layout: the four-momentum is not carried in
// the wavefunction (the compiler keeps every line's momentum once per event,
// in FP64, and passes it explicitly); every factor i of a vertex or
// propagator is tracked by the compiler and folded into the colour
// coefficients, so these functions compute real-coupling ("stripped")
// expressions only; the propagator denominator arrives as a precomputed
// complex reciprocal so that the mixed-precision path can form it in FP64.
//
// Conventions: metric (+,-,-,-); chiral basis, gamma^mu = [[0, s^mu],
// [sb^mu, 0]] with s^mu = (1, sigma), sb^mu = (1, -sigma); P_L keeps the
// upper two components.  Spinors: u(p,l), v(p,l) helicity spinors, rows
// ubar = u^dagger gamma^0.  Vectors carry an upper index.
//
// All functions are templated on the real type R (double: FP64 path, float:
// mixed path) and are __host__ __device__ so they compile for either side.
#pragma once
#include <cstdint>

#define ME_HD __host__ __device__ __forceinline__

namespace me {

template <class R>
struct cx {
  R re, im;
};

template <class R> ME_HD cx<R> mk(R a, R b) { return cx<R>{a, b}; }
template <class R> ME_HD cx<R> operator+(cx<R> a, cx<R> b) { return {a.re + b.re, a.im + b.im}; }
template <class R> ME_HD cx<R> operator-(cx<R> a, cx<R> b) { return {a.re - b.re, a.im - b.im}; }
template <class R> ME_HD cx<R> operator-(cx<R> a) { return {-a.re, -a.im}; }
template <class R> ME_HD cx<R> operator*(cx<R> a, cx<R> b) {
  return {a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re};
}
template <class R> ME_HD cx<R> operator*(R s, cx<R> a) { return {s * a.re, s * a.im}; }
template <class R> ME_HD cx<R> operator*(cx<R> a, R s) { return {s * a.re, s * a.im}; }
template <class R> ME_HD cx<R> conj(cx<R> a) { return {a.re, -a.im}; }
template <class R> ME_HD cx<R> mul_i(cx<R> a) { return {-a.im, a.re}; }
template <class R> ME_HD R abs2(cx<R> a) { return a.re * a.re + a.im * a.im; }

// four-component objects: spinor (column or row) or vector (upper index)
template <class R>
struct W4 {
  cx<R> c[4];
};

template <class R>
struct P4 {
  R e, x, y, z;
};

template <class R> ME_HD P4<R> p4(const double* p) { return P4<R>{(R)p[0], (R)p[1], (R)p[2], (R)p[3]}; }
template <class R> ME_HD P4<R> operator+(P4<R> a, P4<R> b) { return P4<R>{a.e + b.e, a.x + b.x, a.y + b.y, a.z + b.z}; }
template <class R> ME_HD P4<R> neg(P4<R> k) { return P4<R>{-k.e, -k.x, -k.y, -k.z}; }
template <class R> ME_HD R msq(P4<R> k) { return k.e * k.e - k.x * k.x - k.y * k.y - k.z * k.z; }

// ---------------------------------------------------------------------------
// external wavefunctions (massless and massive fermions, massless/massive vectors, scalars)
// ---------------------------------------------------------------------------
// sqrt(E + pz) computed without cancellation for pz < 0; zero only for p along -z.
template <class R> ME_HD R kplus(P4<R> p) {
  return p.z >= R(0) ? p.e + p.z : (p.x * p.x + p.y * p.y) / (p.e - p.z);
}

// Column spinor of a massless fermion line entering its vertex:
//   incoming fermion  -> u(p, hel)      outgoing antifermion -> v(p, hel)
template <class R> ME_HD W4<R> ext_column_massless(P4<R> p, int hel, bool incoming) {
  W4<R> w;
  const R kp = kplus(p);
  cx<R> a, b;  // (s, (px + i py)/s) = sqrt(2E) xi_+ ; ((-px + i py)/s, s) = sqrt(2E) xi_-
  if (kp > R(0)) {
    const R s = sqrt(kp), is = R(1) / s;
    if ((incoming && hel < 0) || (!incoming && hel > 0)) {  // xi_- in the upper (left) slot
      a = mk(-p.x * is, p.y * is);
      b = mk(s, R(0));
    } else {
      a = mk(s, R(0));
      b = mk(p.x * is, p.y * is);
    }
  } else {  // p along -z: xi_+ = (0, 1), xi_- = (-1, 0)
    const R s = sqrt(R(2) * p.e);
    if ((incoming && hel < 0) || (!incoming && hel > 0)) {
      a = mk(-s, R(0));
      b = mk(R(0), R(0));
    } else {
      a = mk(R(0), R(0));
      b = mk(s, R(0));
    }
  }
  const cx<R> z = mk(R(0), R(0));
  if (incoming) {
    if (hel < 0) { w.c[0] = a; w.c[1] = b; w.c[2] = z; w.c[3] = z; }  // u(p,-) = (xi_-, 0)
    else         { w.c[0] = z; w.c[1] = z; w.c[2] = a; w.c[3] = b; }  // u(p,+) = (0, xi_+)
  } else {
    if (hel > 0) { w.c[0] = -a; w.c[1] = -b; w.c[2] = z; w.c[3] = z; }  // v(p,+) = (-xi_-, 0)
    else         { w.c[0] = z; w.c[1] = z; w.c[2] = -a; w.c[3] = -b; }  // v(p,-) = (0, -xi_+)
  }
  return w;
}

// Row spinor of a massless fermion line leaving its vertex:
//   outgoing fermion -> ubar(p, hel)      incoming antifermion -> vbar(p, hel)
template <class R> ME_HD W4<R> ext_row_massless(P4<R> p, int hel, bool incoming) {
  // ubar(p,h) = u(p,h)^dag gamma^0; vbar likewise: row = (lower^*, upper^*)
  W4<R> col = ext_column_massless(p, hel, !incoming);
  W4<R> w;
  w.c[0] = conj(col.c[2]);
  w.c[1] = conj(col.c[3]);
  w.c[2] = conj(col.c[0]);
  w.c[3] = conj(col.c[1]);
  return w;
}

// Two-component helicity eigenstates xi_+-(p) of p^.sigma, with the phases of the massless forms
// above: xi_+ = (cos th/2, e^{i ph} sin th/2), xi_- = (-e^{-i ph} sin th/2, cos th/2); along -z
// xi_+ = (0, 1), xi_- = (-1, 0); at rest the spin states along +z.
template <class R> ME_HD void helicity_xi(P4<R> p, R r, cx<R> xp[2], cx<R> xm[2]) {
  const R rp = p.z >= R(0) ? r + p.z : (p.x * p.x + p.y * p.y) / (r - p.z);
  if (r > R(0) && rp > R(0)) {
    const R n = R(1) / sqrt(R(2) * r * rp);
    xp[0] = mk(rp * n, R(0));
    xp[1] = mk(p.x * n, p.y * n);
    xm[0] = mk(-p.x * n, p.y * n);
    xm[1] = mk(rp * n, R(0));
  } else if (r > R(0)) {
    xp[0] = mk(R(0), R(0)); xp[1] = mk(R(1), R(0));
    xm[0] = mk(R(-1), R(0)); xm[1] = mk(R(0), R(0));
  } else {
    xp[0] = mk(R(1), R(0)); xp[1] = mk(R(0), R(0));
    xm[0] = mk(R(0), R(0)); xm[1] = mk(R(1), R(0));
  }
}

// Column spinor of a massive fermion line entering its vertex, helicity basis:
//   incoming fermion     u(p, l) = (sqrt(E - l|p|) xi_l, sqrt(E + l|p|) xi_l)
//   outgoing antifermion v(p, l) = (-l sqrt(E + l|p|) xi_-l, l sqrt(E - l|p|) xi_-l)
// E - |p| is formed as m^2 / (E + |p|) (no cancellation at high energy).
template <class R> ME_HD W4<R> ext_column_massive(P4<R> p, int hel, bool incoming, R mass) {
  const R r = sqrt(p.x * p.x + p.y * p.y + p.z * p.z);
  const R wp = sqrt(p.e + r), wm = mass / wp;  // sqrt(E + |p|), sqrt(E - |p|)
  cx<R> xp[2], xm[2];
  helicity_xi(p, r, xp, xm);
  const R l = (R)hel;
  W4<R> w;
  if (incoming) {
    const cx<R>* x = hel > 0 ? xp : xm;
    const R a = hel > 0 ? wm : wp, b = hel > 0 ? wp : wm;
    w.c[0] = a * x[0]; w.c[1] = a * x[1]; w.c[2] = b * x[0]; w.c[3] = b * x[1];
  } else {
    const cx<R>* x = hel > 0 ? xm : xp;
    const R a = hel > 0 ? wp : wm, b = hel > 0 ? wm : wp;
    w.c[0] = (-l * a) * x[0]; w.c[1] = (-l * a) * x[1]; w.c[2] = (l * b) * x[0]; w.c[3] = (l * b) * x[1];
  }
  return w;
}

// Row spinor of a massive fermion line leaving its vertex (ubar outgoing, vbar incoming)
template <class R> ME_HD W4<R> ext_row_massive(P4<R> p, int hel, bool incoming, R mass) {
  W4<R> col = ext_column_massive(p, hel, !incoming, mass);
  W4<R> w;
  w.c[0] = conj(col.c[2]);
  w.c[1] = conj(col.c[3]);
  w.c[2] = conj(col.c[0]);
  w.c[3] = conj(col.c[1]);
  return w;
}

// Polarisation vector eps(k, hel) (incoming) or eps^*(k, hel) (outgoing).
// eps(+-1) = (0, -+ e_theta - i e_phi)/sqrt2, eps(0) = (|k|, E k^)/m.
template <class R> ME_HD W4<R> ext_vector(P4<R> k, int hel, bool incoming, R mass) {
  W4<R> w;
  const R pt2 = k.x * k.x + k.y * k.y;
  const R pt = sqrt(pt2);
  const R ak = sqrt(pt2 + k.z * k.z);
  if (hel == 0) {
    const R im = R(1) / mass;
    const R f = k.e / (ak * mass);
    w.c[0] = mk(ak * im, R(0));
    w.c[1] = mk(f * k.x, R(0));
    w.c[2] = mk(f * k.y, R(0));
    w.c[3] = mk(f * k.z, R(0));
    return w;
  }
  R cth, sth, cph, sph;
  if (pt > R(0)) {
    cth = k.z / ak; sth = pt / ak; cph = k.x / pt; sph = k.y / pt;
  } else {
    cth = k.z >= R(0) ? R(1) : R(-1); sth = R(0); cph = R(1); sph = R(0);
  }
  const R r = R(0.70710678118654752440);
  const R l = (R)hel;
  const R sgn = incoming ? R(1) : R(-1);  // conjugation flips the imaginary parts
  w.c[0] = mk(R(0), R(0));
  w.c[1] = mk(-l * cth * cph * r, sgn * sph * r);
  w.c[2] = mk(-l * cth * sph * r, -sgn * cph * r);
  w.c[3] = mk(l * sth * r, R(0));
  return w;
}

// Transverse polarisation of a massless external vector in the helicity basis:
// eps(+-1) above has a zero time component and a real z component.  It is
// carried as PV (two complex and one real number), and the vertex functions
// below take it beside W4 and skip its zero and real parts (IEEE arithmetic
// would not let the compiler drop products with the literal zeros of a W4).
template <class R>
struct PV {
  cx<R> c1, c2;
  R c3;
};

template <class R> ME_HD PV<R> ext_pol(P4<R> k, int hel, bool incoming) {
  const R pt2 = k.x * k.x + k.y * k.y;
  const R pt = sqrt(pt2);
  const R ak = sqrt(pt2 + k.z * k.z);
  R cth, sth, cph, sph;
  if (pt > R(0)) {
    cth = k.z / ak; sth = pt / ak; cph = k.x / pt; sph = k.y / pt;
  } else {
    cth = k.z >= R(0) ? R(1) : R(-1); sth = R(0); cph = R(1); sph = R(0);
  }
  const R r = R(0.70710678118654752440);
  const R l = (R)hel;
  const R sgn = incoming ? R(1) : R(-1);
  PV<R> w;
  w.c1 = mk(-l * cth * cph * r, sgn * sph * r);
  w.c2 = mk(-l * cth * sph * r, -sgn * cph * r);
  w.c3 = l * sth * r;
  return w;
}

// ---------------------------------------------------------------------------
// FFV: Gamma = Vslash (gL P_L + gR P_R)
// ---------------------------------------------------------------------------
// V.sigma = [[V0-V3, -V1+iV2], [-V1-iV2, V0+V3]],  V.sigmabar = [[V0+V3, V1-iV2], [V1+iV2, V0-V3]]
template <class R> ME_HD void vsig(const W4<R>& V, cx<R> m[4]) {
  m[0] = V.c[0] - V.c[3];
  m[1] = -V.c[1] + mul_i(V.c[2]);
  m[2] = -V.c[1] - mul_i(V.c[2]);
  m[3] = V.c[0] + V.c[3];
}
template <class R> ME_HD void vsigbar(const W4<R>& V, cx<R> m[4]) {
  m[0] = V.c[0] + V.c[3];
  m[1] = V.c[1] - mul_i(V.c[2]);
  m[2] = V.c[1] + mul_i(V.c[2]);
  m[3] = V.c[0] - V.c[3];
}

// Which halves of a four-spinor can be non-zero.  A massless line of definite
// chirality keeps one half zero exactly: a left-chiral column spinor has only
// its upper (P_L) half, its Dirac adjoint only the lower half.  The compiler
// knows the half of every spinor and instantiates these functions so that the
// zero half is neither read nor computed (IEEE arithmetic would not let the
// compiler drop products with zeros on its own).
enum : int { kUp = 0, kLo = 1, kAll = 2 };

// Gamma psi for a column spinor: (gR (V.s) psi_lo, gL (V.sb) psi_up)
template <class R, int H = kAll>
ME_HD W4<R> ffv_col(const W4<R>& psi, const W4<R>& V, R gl, R gr, bool has_l, bool has_r) {
  W4<R> o;
  const cx<R> z = mk(R(0), R(0));
  if (H != kUp && has_r) {
    cx<R> m[4];
    vsig(V, m);
    o.c[0] = gr * (m[0] * psi.c[2] + m[1] * psi.c[3]);
    o.c[1] = gr * (m[2] * psi.c[2] + m[3] * psi.c[3]);
  } else { o.c[0] = z; o.c[1] = z; }
  if (H != kLo && has_l) {
    cx<R> m[4];
    vsigbar(V, m);
    o.c[2] = gl * (m[0] * psi.c[0] + m[1] * psi.c[1]);
    o.c[3] = gl * (m[2] * psi.c[0] + m[3] * psi.c[1]);
  } else { o.c[2] = z; o.c[3] = z; }
  return o;
}

// row Gamma: (gL row_lo (V.sb), gR row_up (V.s))
template <class R, int H = kAll>
ME_HD W4<R> ffv_row(const W4<R>& row, const W4<R>& V, R gl, R gr, bool has_l, bool has_r) {
  W4<R> o;
  const cx<R> z = mk(R(0), R(0));
  if (H != kUp && has_l) {
    cx<R> m[4];
    vsigbar(V, m);
    o.c[0] = gl * (row.c[2] * m[0] + row.c[3] * m[2]);
    o.c[1] = gl * (row.c[2] * m[1] + row.c[3] * m[3]);
  } else { o.c[0] = z; o.c[1] = z; }
  if (H != kLo && has_r) {
    cx<R> m[4];
    vsig(V, m);
    o.c[2] = gr * (row.c[0] * m[0] + row.c[1] * m[2]);
    o.c[3] = gr * (row.c[0] * m[1] + row.c[1] * m[3]);
  } else { o.c[2] = z; o.c[3] = z; }
  return o;
}

// ffv_col with a PV: V.s = [[-V3, -V1+iV2], [-V1-iV2, V3]], V.sb = [[V3, V1-iV2], [V1+iV2, -V3]]
template <class R, int H = kAll>
ME_HD W4<R> ffv_col(const W4<R>& psi, const PV<R>& V, R gl, R gr, bool has_l, bool has_r) {
  W4<R> o;
  const cx<R> z = mk(R(0), R(0));
  if (H != kUp && has_r) {
    const cx<R> m1 = -V.c1 + mul_i(V.c2), m2 = -V.c1 - mul_i(V.c2);
    o.c[0] = gr * ((-V.c3) * psi.c[2] + m1 * psi.c[3]);
    o.c[1] = gr * (m2 * psi.c[2] + V.c3 * psi.c[3]);
  } else { o.c[0] = z; o.c[1] = z; }
  if (H != kLo && has_l) {
    const cx<R> m1 = V.c1 - mul_i(V.c2), m2 = V.c1 + mul_i(V.c2);
    o.c[2] = gl * (V.c3 * psi.c[0] + m1 * psi.c[1]);
    o.c[3] = gl * (m2 * psi.c[0] + (-V.c3) * psi.c[1]);
  } else { o.c[2] = z; o.c[3] = z; }
  return o;
}

// ffv_row with a PV
template <class R, int H = kAll>
ME_HD W4<R> ffv_row(const W4<R>& row, const PV<R>& V, R gl, R gr, bool has_l, bool has_r) {
  W4<R> o;
  const cx<R> z = mk(R(0), R(0));
  if (H != kUp && has_l) {
    const cx<R> m1 = V.c1 - mul_i(V.c2), m2 = V.c1 + mul_i(V.c2);
    o.c[0] = gl * (row.c[2] * V.c3 + row.c[3] * m2);
    o.c[1] = gl * (row.c[2] * m1 + row.c[3] * (-V.c3));
  } else { o.c[0] = z; o.c[1] = z; }
  if (H != kLo && has_r) {
    const cx<R> m1 = -V.c1 + mul_i(V.c2), m2 = -V.c1 - mul_i(V.c2);
    o.c[2] = gr * (row.c[0] * (-V.c3) + row.c[1] * m2);
    o.c[3] = gr * (row.c[0] * m1 + row.c[1] * V.c3);
  } else { o.c[2] = z; o.c[3] = z; }
  return o;
}

// row Gamma column; HR, HC: halves of the row and the column
template <class R, int HR = kAll, int HC = kAll, class VV>
ME_HD cx<R> ffv_amp(const W4<R>& row, const W4<R>& col, const VV& V, R gl, R gr, bool has_l, bool has_r) {
  const W4<R> g = ffv_col<R, HC>(col, V, gl, gr, has_l, has_r);
  // g has the half opposite to HC; only the overlap with the row contributes
  constexpr bool up = (HC != kUp) && (HR != kLo);   // g upper half (from psi_lo) meets row upper half
  constexpr bool lo = (HC != kLo) && (HR != kUp);
  cx<R> a = mk(R(0), R(0));
  if (up) a = a + row.c[0] * g.c[0] + row.c[1] * g.c[1];
  if (lo) a = a + row.c[2] * g.c[2] + row.c[3] * g.c[3];
  return a;
}

// ---------------------------------------------------------------------------
// FFS: Gamma = S (gL P_L + gR P_R)   (P_L: the upper half)
// ---------------------------------------------------------------------------
template <class R, int H = kAll>
ME_HD W4<R> ffs_col(const W4<R>& psi, cx<R> S, R gl, R gr, bool has_l, bool has_r) {
  W4<R> o;
  const cx<R> z = mk(R(0), R(0));
  if (H != kLo && has_l) { const cx<R> f = gl * S; o.c[0] = f * psi.c[0]; o.c[1] = f * psi.c[1]; }
  else { o.c[0] = z; o.c[1] = z; }
  if (H != kUp && has_r) { const cx<R> f = gr * S; o.c[2] = f * psi.c[2]; o.c[3] = f * psi.c[3]; }
  else { o.c[2] = z; o.c[3] = z; }
  return o;
}

// row (gL P_L + gR P_R) S: (gL S row_up, gR S row_lo)
template <class R, int H = kAll>
ME_HD W4<R> ffs_row(const W4<R>& row, cx<R> S, R gl, R gr, bool has_l, bool has_r) {
  return ffs_col<R, H>(row, S, gl, gr, has_l, has_r);
}

// row (gL P_L + gR P_R) col
template <class R, int HR = kAll, int HC = kAll>
ME_HD cx<R> ffs_scalar(const W4<R>& row, const W4<R>& col, R gl, R gr, bool has_l, bool has_r) {
  cx<R> a = mk(R(0), R(0));
  if (has_l && HR != kLo && HC != kLo) a = a + gl * (row.c[0] * col.c[0] + row.c[1] * col.c[1]);
  if (has_r && HR != kUp && HC != kUp) a = a + gr * (row.c[2] * col.c[2] + row.c[3] * col.c[3]);
  return a;
}

// J^mu = row gamma^mu (gL P_L + gR P_R) col = gL row_lo sb^mu col_up + gR row_up s^mu col_lo
template <class R, int HR = kAll, int HC = kAll>
ME_HD W4<R> ffv_current(const W4<R>& row, const W4<R>& col, R gl, R gr, bool has_l, bool has_r) {
  W4<R> J;
  cx<R> s0 = mk(R(0), R(0)), s1 = s0, s2 = s0, s3 = s0;
  if (has_l && HR != kUp && HC != kLo) {  // a = row_lo, b = col_up, sigmabar: (1, -sigma)
    const cx<R> a0 = row.c[2], a1 = row.c[3], b0 = col.c[0], b1 = col.c[1];
    const cx<R> t00 = a0 * b0, t11 = a1 * b1, t01 = a0 * b1, t10 = a1 * b0;
    s0 = s0 + gl * (t00 + t11);
    s1 = s1 - gl * (t01 + t10);
    s2 = s2 - gl * mul_i(t10 - t01);
    s3 = s3 - gl * (t00 - t11);
  }
  if (has_r && HR != kLo && HC != kUp) {  // a = row_up, b = col_lo, sigma: (1, sigma)
    const cx<R> a0 = row.c[0], a1 = row.c[1], b0 = col.c[2], b1 = col.c[3];
    const cx<R> t00 = a0 * b0, t11 = a1 * b1, t01 = a0 * b1, t10 = a1 * b0;
    s0 = s0 + gr * (t00 + t11);
    s1 = s1 + gr * (t01 + t10);
    s2 = s2 + gr * mul_i(t10 - t01);
    s3 = s3 + gr * (t00 - t11);
  }
  J.c[0] = s0; J.c[1] = s1; J.c[2] = s2; J.c[3] = s3;
  return J;
}

// ---------------------------------------------------------------------------
// propagators (numerators times the reciprocal denominator inv = 1/(q^2 - m^2 + i m w))
// INV is cx<R> for a line with a width and R for a massless line (a real
// reciprocal: IEEE arithmetic would not let the compiler drop the products with
// its zero imaginary part).  The real diagonal entries of q.sigma, q.sigmabar
// multiply as reals for the same reason.
// ---------------------------------------------------------------------------
// (qslash + m) x inv for a column with non-zero half HX;  q is the momentum along the fermion arrow
template <class R, int HX = kAll, class INV>
ME_HD W4<R> prop_col(const W4<R>& x, P4<R> q, R m, INV inv) {
  // q.sigma = [[q0-q3, -q1+iq2], [-q1-iq2, q0+q3]],  q.sigmabar = [[q0+q3, q1-iq2], [q1+iq2, q0-q3]]
  const R qm = q.e - q.z, qp = q.e + q.z;
  const cx<R> s01 = mk(-q.x, q.y), s10 = mk(-q.x, -q.y), b01 = mk(q.x, -q.y), b10 = mk(q.x, q.y);
  const cx<R> z = mk(R(0), R(0));
  W4<R> o;
  if (HX != kUp) {
    o.c[0] = (qm * x.c[2] + s01 * x.c[3]) * inv;
    o.c[1] = (s10 * x.c[2] + qp * x.c[3]) * inv;
  } else { o.c[0] = z; o.c[1] = z; }
  if (HX != kLo) {
    o.c[2] = (qp * x.c[0] + b01 * x.c[1]) * inv;
    o.c[3] = (b10 * x.c[0] + qm * x.c[1]) * inv;
  } else { o.c[2] = z; o.c[3] = z; }
  if (m != R(0)) {
    for (int k = 0; k < 4; ++k) o.c[k] = o.c[k] + (m * x.c[k]) * inv;
  }
  return o;
}

// x (qslash + m) inv for a row with non-zero half HX
template <class R, int HX = kAll, class INV>
ME_HD W4<R> prop_row(const W4<R>& x, P4<R> q, R m, INV inv) {
  const R qm = q.e - q.z, qp = q.e + q.z;
  const cx<R> s01 = mk(-q.x, q.y), s10 = mk(-q.x, -q.y), b01 = mk(q.x, -q.y), b10 = mk(q.x, q.y);
  const cx<R> z = mk(R(0), R(0));
  W4<R> o;
  // (x_up, x_lo) [[0, q.s], [q.sb, 0]] = (x_lo q.sb, x_up q.s)
  if (HX != kUp) {
    o.c[0] = (x.c[2] * qp + x.c[3] * b10) * inv;
    o.c[1] = (x.c[2] * b01 + x.c[3] * qm) * inv;
  } else { o.c[0] = z; o.c[1] = z; }
  if (HX != kLo) {
    o.c[2] = (x.c[0] * qm + x.c[1] * s10) * inv;
    o.c[3] = (x.c[0] * s01 + x.c[1] * qp) * inv;
  } else { o.c[2] = z; o.c[3] = z; }
  if (m != R(0)) {
    for (int k = 0; k < 4; ++k) o.c[k] = o.c[k] + (m * x.c[k]) * inv;
  }
  return o;
}

template <class R> ME_HD cx<R> mdot(const W4<R>& a, const W4<R>& b) {
  return a.c[0] * b.c[0] - a.c[1] * b.c[1] - a.c[2] * b.c[2] - a.c[3] * b.c[3];
}
template <class R> ME_HD cx<R> mdot(P4<R> q, const W4<R>& b) {
  return q.e * b.c[0] - q.x * b.c[1] - q.y * b.c[2] - q.z * b.c[3];
}
// with a PV (time component zero, z component real)
template <class R> ME_HD cx<R> mdot(const W4<R>& a, const PV<R>& b) {
  return -(a.c[1] * b.c1 + a.c[2] * b.c2 + a.c[3] * b.c3);
}
template <class R> ME_HD cx<R> mdot(const PV<R>& a, const W4<R>& b) { return mdot(b, a); }
template <class R> ME_HD cx<R> mdot(const PV<R>& a, const PV<R>& b) {
  const cx<R> t = a.c1 * b.c1 + a.c2 * b.c2;
  return mk(-(t.re + a.c3 * b.c3), -t.im);
}
template <class R> ME_HD cx<R> mdot(P4<R> q, const PV<R>& b) {
  const cx<R> t = q.x * b.c1 + q.y * b.c2;
  return mk(-(t.re + q.z * b.c3), -t.im);
}

// acc + v_mu s for component MU of a W4 or a PV (nothing for the zero time component of a PV)
template <int MU, class R> ME_HD cx<R> add_comp(cx<R> acc, const W4<R>& v, cx<R> s) { return acc + v.c[MU] * s; }
template <int MU, class R> ME_HD cx<R> add_comp(cx<R> acc, const PV<R>& v, cx<R> s) {
  if constexpr (MU == 0) return acc;
  else if constexpr (MU == 1) return acc + v.c1 * s;
  else if constexpr (MU == 2) return acc + v.c2 * s;
  else return acc + v.c3 * s;
}

// vector propagator numerator g^{mu nu} - q^mu q^nu / mc2 applied to X, times inv
template <class R, class INV>
ME_HD W4<R> prop_vec(const W4<R>& X, P4<R> q, INV inv, bool massive, cx<R> inv_mc2) {
  W4<R> o;
  if (massive) {
    const cx<R> f = mdot(q, X) * inv_mc2;
    o.c[0] = (X.c[0] - q.e * f) * inv;
    o.c[1] = (X.c[1] - q.x * f) * inv;
    o.c[2] = (X.c[2] - q.y * f) * inv;
    o.c[3] = (X.c[3] - q.z * f) * inv;
  } else {
    for (int k = 0; k < 4; ++k) o.c[k] = X.c[k] * inv;
  }
  return o;
}

// ---------------------------------------------------------------------------
// VVV (all momenta incoming):  g [ g^{12}(k1-k2)^3 + g^{23}(k2-k3)^1 + g^{31}(k3-k1)^2 ]
// ---------------------------------------------------------------------------
template <class R, class VA, class VB>
ME_HD W4<R> vvv_current(const VA& V1, P4<R> k1, const VB& V2, P4<R> k2, R g) {
  const P4<R> k3 = {-(k1.e + k2.e), -(k1.x + k2.x), -(k1.y + k2.y), -(k1.z + k2.z)};
  const P4<R> d12 = {k1.e - k2.e, k1.x - k2.x, k1.y - k2.y, k1.z - k2.z};
  const P4<R> d23 = {k2.e - k3.e, k2.x - k3.x, k2.y - k3.y, k2.z - k3.z};
  const P4<R> d31 = {k3.e - k1.e, k3.x - k1.x, k3.y - k1.y, k3.z - k1.z};
  const cx<R> v12 = mdot(V1, V2), a = mdot(d23, V1), b = mdot(d31, V2);
  W4<R> o;
  o.c[0] = g * add_comp<0>(add_comp<0>(d12.e * v12, V2, a), V1, b);
  o.c[1] = g * add_comp<1>(add_comp<1>(d12.x * v12, V2, a), V1, b);
  o.c[2] = g * add_comp<2>(add_comp<2>(d12.y * v12, V2, a), V1, b);
  o.c[3] = g * add_comp<3>(add_comp<3>(d12.z * v12, V2, a), V1, b);
  return o;
}

template <class R, class VA, class VB, class VC>
ME_HD cx<R> vvv_amp(const VA& V1, P4<R> k1, const VB& V2, P4<R> k2, const VC& V3, R g) {
  return mdot(vvv_current<R>(V1, k1, V2, k2, g), V3);
}

// VVVV pairing current: V_p (V_a . V_b)
template <class R> ME_HD W4<R> vec_times(const W4<R>& v, cx<R> d) {
  W4<R> o;
  for (int k = 0; k < 4; ++k) o.c[k] = v.c[k] * d;
  return o;
}
template <class R> ME_HD W4<R> vec_times(const PV<R>& v, cx<R> d) {
  W4<R> o;
  o.c[0] = mk(R(0), R(0));
  o.c[1] = v.c1 * d;
  o.c[2] = v.c2 * d;
  o.c[3] = v.c3 * d;
  return o;
}
template <class R, class VP, class VA, class VB> ME_HD W4<R> v4_term(const VP& Vp, const VA& Va, const VB& Vb) {
  return vec_times<R>(Vp, mdot(Va, Vb));
}

template <class R> ME_HD W4<R> w4_sub(const W4<R>& a, const W4<R>& b, R g) {
  W4<R> o;
  for (int k = 0; k < 4; ++k) o.c[k] = g * (a.c[k] - b.c[k]);
  return o;
}

// electroweak quartic current: g (a + b - 2 p), with a, b, p the currents of the three metric pairings
template <class R> ME_HD W4<R> w4_quartic(const W4<R>& a, const W4<R>& b, const W4<R>& p, R g) {
  W4<R> o;
  for (int k = 0; k < 4; ++k) o.c[k] = g * (a.c[k] + b.c[k] - R(2) * p.c[k]);
  return o;
}

template <class R> ME_HD W4<R> w4_scale(const W4<R>& a, cx<R> s) {
  W4<R> o;
  for (int k = 0; k < 4; ++k) o.c[k] = a.c[k] * s;
  return o;
}

}  // namespace me
