// Process unit for NGLUON gluons (compiled once per gluon count with -DNGLUON=n).
// Kernels: k_eval_gluon (|M|^2 from momenta in HBM) and, for the Monte Carlo
// step, the generic phase-space kernel k_ps followed by k_me_gluon.  One thread
// block evaluates one event at a time (grid-stride over events, one resident
// wave of blocks); its two halves run two helicities of the non-root legs side
// by side, and after each such pair the block forms the colour sum of the
// pair's 8 amplitude rows (2 helicities x 2 root helicities x re/im).
//
// Colour sum, Eq. 6 with the exact integer matrix C_num = den C:
//   FP64 path:  y = C_num x on the FP64 CUDA cores, then x . y;
//   mixed path: on the tensor cores (tcgen05).  Every row x of the pair is scaled
//   by a power of two per helicity and split into FP16 hi + lo parts (22 bits);
//   the off-diagonal part of C_num has integer entries below 2048 and is exact in
//   FP16.  One thread issues D = C_off [x_hi | x_lo]^T as tcgen05.mma (M = 128
//   colour rows, N = 16 = 8 rows x hi/lo, K = 16 per instruction, FP32
//   accumulation in tensor memory), both operands K-major in shared memory; the
//   commit arrives on an mbarrier, four warps read D back with tcgen05.ld; the
//   constant diagonal of C_num (3641 for six gluons, not exact in FP16) is added
//   on the CUDA cores in that epilogue, which also forms x . (D_hi + D_lo + c x).
#include <algorithm>
#include <cstdint>
#include <cstring>
#include <cuda_fp16.h>

#include "gluon.cuh"
#include "process_common.cuh"

#define ME_STR2(x) #x
#define ME_STR(x) ME_STR2(x)
#define ME_CAT2(a, b) a##b
#define ME_CAT(a, b) ME_CAT2(a, b)
#include ME_STR(ME_CAT(gluon_tables, NGLUON).h)

#ifdef __CUDA_ARCH__
#define ME_GTN(a) ME_CAT(a, NGLUON)
#else
#define ME_GTN(a) ME_CAT(ME_CAT(a, NGLUON), _h)
#endif

namespace me {
namespace gluon {
namespace ME_CAT(g, NGLUON) {  // one namespace per gluon count: the units link together

using T = ME_CAT(Tables, NGLUON);
constexpr int NG = NGLUON;
constexpr int NHEL = 1 << (NG - 1);        // helicities of the non-root legs
// Helicities evaluated side by side (one per kThreads-thread part of a block) and
// the amplitude rows they produce (helicity, root helicity, re/im).  FP32: two, so
// that the 8 rows of a pair fill one n8 tensor-core tile; FP64: one (its shared
// memory allows two blocks per SM only at one helicity per block).
template <class R>
struct Cfg {
  static constexpr int HP = sizeof(R) == 4 ? 2 : 1;
  static constexpr int THREADS = HP * kThreads;
  static constexpr int NROW = 4 * HP;
};
constexpr int NROW = Cfg<float>::NROW;     // rows of the tensor-core colour step
constexpr int MT = 128;                    // colour rows of the tcgen05 tile (C zero padded)
constexpr int NT = 2 * NROW;               // its columns: the pair's rows, hi parts then lo parts
constexpr int KP = (T::NAMP + 31) / 32 * 32;  // colour columns padded to whole K-steps of 16
constexpr int XLD = KP + 4;                // FP32 row stride: epilogue reads hit 32 distinct banks
static_assert(T::NAMP <= MT, "the colour basis fits one tcgen05 tile");
constexpr float kDiag = ME_CAT(kColourDiag, NGLUON);
static_assert(ME_CAT(kColourOffFitsHalf, NGLUON), "off-diagonal colour integers must be exact in FP16");
static_assert(NROW == 8, "one n8 MMA tile per helicity pair");
static_assert(T::NAMP % 2 == 0, "amplitude rows are converted in pairs");

struct Traits {
  static constexpr int NEXT = NG;
  struct Params {
    double GS;
  };
};

__host__ __device__ __forceinline__ const int32_t* cur_meta() { return ME_GTN(kCurMeta); }
__host__ __device__ __forceinline__ const float* colour() { return ME_GTN(kColour); }

// Shared-memory storage of currents and momenta: 16-byte aligned with vector
// loads and stores.  A current slot holds the four complex components and the
// two contractions e_r = eps0_r . J with the root polarisations (the amplitude
// needs only these scalars, see amp_scalar); its stride is 48 B (FP32), not a
// power of two, so gathers at data-dependent indices spread over the banks.
template <class R>
struct alignas(16) JS {
  R v[12];
};
template <class R>
struct alignas(16) KS {
  R v[4];
};

__device__ __forceinline__ W4<float> ldj(const JS<float>& j) {
  const float4 u = reinterpret_cast<const float4*>(j.v)[0], w = reinterpret_cast<const float4*>(j.v)[1];
  return W4<float>{{{u.x, u.y}, {u.z, u.w}, {w.x, w.y}, {w.z, w.w}}};
}
__device__ __forceinline__ void stj(JS<float>& j, const W4<float>& a) {
  reinterpret_cast<float4*>(j.v)[0] = make_float4(a.c[0].re, a.c[0].im, a.c[1].re, a.c[1].im);
  reinterpret_cast<float4*>(j.v)[1] = make_float4(a.c[2].re, a.c[2].im, a.c[3].re, a.c[3].im);
}
__device__ __forceinline__ W4<double> ldj(const JS<double>& j) {
  const double2* q = reinterpret_cast<const double2*>(j.v);
  const double2 a = q[0], b = q[1], c = q[2], d = q[3];
  return W4<double>{{{a.x, a.y}, {b.x, b.y}, {c.x, c.y}, {d.x, d.y}}};
}
__device__ __forceinline__ void stj(JS<double>& j, const W4<double>& a) {
  double2* q = reinterpret_cast<double2*>(j.v);
#pragma unroll
  for (int k = 0; k < 4; ++k) q[k] = make_double2(a.c[k].re, a.c[k].im);
}
// e_r = eps0_r . J of a current slot, r = 0, 1
__device__ __forceinline__ void lde(const JS<float>& j, cx<float>& e0, cx<float>& e1) {
  const float4 u = reinterpret_cast<const float4*>(j.v)[2];
  e0 = cx<float>{u.x, u.y};
  e1 = cx<float>{u.z, u.w};
}
__device__ __forceinline__ void ste(JS<float>& j, cx<float> e0, cx<float> e1) {
  reinterpret_cast<float4*>(j.v)[2] = make_float4(e0.re, e0.im, e1.re, e1.im);
}
__device__ __forceinline__ void lde(const JS<double>& j, cx<double>& e0, cx<double>& e1) {
  const double2* q = reinterpret_cast<const double2*>(j.v);
  const double2 a = q[4], b = q[5];
  e0 = cx<double>{a.x, a.y};
  e1 = cx<double>{b.x, b.y};
}
__device__ __forceinline__ void ste(JS<double>& j, cx<double> e0, cx<double> e1) {
  double2* q = reinterpret_cast<double2*>(j.v);
  q[4] = make_double2(e0.re, e0.im);
  q[5] = make_double2(e1.re, e1.im);
}

__device__ __forceinline__ P4<float> ldk(const KS<float>& k) {
  const float4 u = *reinterpret_cast<const float4*>(k.v);
  return P4<float>{u.x, u.y, u.z, u.w};
}
__device__ __forceinline__ void stk(KS<float>& k, const P4<float>& p) {
  *reinterpret_cast<float4*>(k.v) = make_float4(p.e, p.x, p.y, p.z);
}
__device__ __forceinline__ P4<double> ldk(const KS<double>& k) {
  const double2* q = reinterpret_cast<const double2*>(k.v);
  const double2 a = q[0], b = q[1];
  return P4<double>{a.x, a.y, b.x, b.y};
}
__device__ __forceinline__ void stk(KS<double>& k, const P4<double>& p) {
  double2* q = reinterpret_cast<double2*>(k.v);
  q[0] = make_double2(p.e, p.x);
  q[1] = make_double2(p.y, p.z);
}

template <class R>
struct Shared {
  KS<R> K[T::NCUR];       // outgoing momenta of every current (externals first)
  KS<R> EK[T::NCUR];      // eps0_0 . K and eps0_1 . K (two complex numbers) of every current
  R invp2[T::NCUR];
  JS<R> J[Cfg<R>::HP][T::NCUR];  // currents of the helicities being evaluated
  JS<R> ext[NG - 1][2];          // polarisation vectors of legs 1..NG-1, helicity -1 / +1
  W4<R> eps0[2];                 // root polarisation, both helicities
  R X[Cfg<R>::NROW][XLD];        // amplitude rows, row 4 h + 2 r + (0: re, 1: im)
  unsigned emax[2];              // largest biased FP32 exponent in the rows of each helicity
  R red[Cfg<R>::THREADS / 32];
};

// Tensor-core operands of the mixed path (dynamic shared memory after Shared<float>), K-major
// without swizzle: an element (row r, column k) of an operand sits at byte
//   (r / 8) * (KP / 8) * 128 + (k / 8) * 128 + (r % 8) * 16 + (k % 8) * 2,
// i.e. 8 x 16-byte core matrices, 128 B apart along K (the descriptor's leading-dimension
// offset) and (KP / 8) * 128 B apart between groups of 8 rows (its stride-dimension offset).
struct alignas(128) TcShared {
  __half C[MT * KP];     // C_num with zero diagonal, zero padded to MT x KP
  __half X[NT * KP];     // rows 0..7: high FP16 parts of the pair's scaled rows; 8..15: low parts
  uint64_t mbar;         // completion of the pair's MMAs (tcgen05.commit)
  uint32_t tmem;         // tensor-memory address of the 128 x 32 FP32 accumulator
  uint32_t uses;         // completed pairs (the parity of the next wait)
  int failed;            // a wait ran out (the kernel reports it and stops using the tensor cores)
};
__device__ __forceinline__ uint32_t tc_off(int r, int k) {
  return (uint32_t)((r >> 3) * (KP / 8) * 128 + (k >> 3) * 128 + (r & 7) * 16 + (k & 7) * 2);
}

// ---------------------------------------------------------------------------
// tcgen05 helpers (inline PTX)
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// shared-memory matrix descriptor: start address, leading (K) and stride (8-row group) byte
// offsets, descriptor version 1, no swizzle
__device__ __forceinline__ uint64_t tc_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((addr & 0x3FFFFu) >> 4) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
         ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}
// kind::f16 instruction descriptor: FP32 accumulator, FP16 A and B, both K-major, N >> 3, M >> 4
constexpr uint32_t kTcIdesc = (1u << 4) | ((uint32_t)(NT >> 3) << 17) | ((uint32_t)(MT >> 4) << 24);
constexpr uint32_t kTmemCols = 32;  // allocation granule (the accumulator uses NT columns)

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t done;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.b32 %0, 1, 0, p;\n}\n"
      : "=r"(done)
      : "r"(smem_addr(bar)), "r"(parity)
      : "memory");
  return done != 0;
}
// bounded wait for a phase of the mbarrier: false if it did not complete within about 0.1 s
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity) {
  for (int it = 0; it < (1 << 20); ++it) {
    if (mbar_try_wait(bar, parity)) return true;
    __nanosleep(64);
  }
  return false;
}

// scale 2^es with es = 141 - emax puts every value of the rows below 2^15
__device__ __forceinline__ int scale_exp(unsigned emax) {
  const int es = 141 - (int)emax;
  return es > 126 ? 126 : es;
}
__device__ __forceinline__ float pow2f(int e) { return __int_as_float((e + 127) << 23); }

__device__ __forceinline__ unsigned exp_bits(float x) { return (__float_as_uint(x) >> 23) & 0xffu; }

// colour sum of the pair on the tensor cores; returns this thread's share of sum_rows x . C x
__device__ float colour_pair(Shared<float>& sh, TcShared* tcp) {
  TcShared& tc = *tcp;
  const int tid = threadIdx.x;
  // FP16 hi/lo split of the scaled rows (columns beyond NAMP are zero), in the operand layout
  for (int i = tid; i < NROW * (KP / 2); i += blockDim.x) {
    const int n = i / (KP / 2), k = 2 * (i % (KP / 2));
    const float s = pow2f(scale_exp(sh.emax[n >> 2]));
    float x0 = 0.0f, x1 = 0.0f;
    if (k < T::NAMP) {
      x0 = sh.X[n][k] * s;
      x1 = sh.X[n][k + 1] * s;
    }
    const __half2 h = __floats2half2_rn(x0, x1);
    const float2 hf = __half22float2(h);
    *reinterpret_cast<__half2*>(reinterpret_cast<char*>(tc.X) + tc_off(n, k)) = h;
    *reinterpret_cast<__half2*>(reinterpret_cast<char*>(tc.X) + tc_off(n + NROW, k)) =
        __floats2half2_rn(x0 - hf.x, x1 - hf.y);
  }
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // the operands, visible to the tensor cores
  __syncthreads();
  const uint32_t parity = tc.uses & 1u;
  const bool run = !tc.failed;
  if (tid == 0 && run) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t a0 = smem_addr(tc.C), b0 = smem_addr(tc.X);
#pragma unroll
    for (int kk = 0; kk < KP / 16; ++kk) {  // two core matrices (16 columns) per step
      const uint64_t a = tc_desc(a0 + 256u * kk, 128u, (KP / 8) * 128u);
      const uint64_t b = tc_desc(b0 + 256u * kk, 128u, (KP / 8) * 128u);
      asm volatile(
          "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
          " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tc.tmem),
          "l"(a), "l"(b), "r"(kTcIdesc), "r"((uint32_t)(kk > 0))
          : "memory");
    }
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                     smem_addr(&tc.mbar))
                 : "memory");
  }
  // block-uniform outcome: tcgen05.ld below is a whole-warp instruction
  const bool ok = __syncthreads_and(run && mbar_wait_bounded(&tc.mbar, parity)) != 0;
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  float part = 0.0f;
  const int warp = tid >> 5, lane = tid & 31;
  // D[m][n]: colour row m = 32 warp + lane, columns n (hi parts) and n + NROW (lo parts)
  if (warp < MT / 32 && ok) {
    uint32_t r[NT];
    const uint32_t taddr = tc.tmem + ((uint32_t)(32 * warp) << 16);
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr)
        : "memory");
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
    const int m = 32 * warp + lane;
    if (m < T::NAMP) {
#pragma unroll
      for (int n = 0; n < NROW; ++n) {
        const float is = pow2f(-scale_exp(sh.emax[n >> 2]));
        const float x = sh.X[n][m];
        part += x * fmaf(__uint_as_float(r[n]) + __uint_as_float(r[n + NROW]), is, kDiag * x);
      }
    }
  }
  if (run && !ok && tid == 0) {
    // the MMAs did not complete in time: wait once more (bounded) for them before the tensor memory
    // can be released, and stop using the tensor cores in this block
    mbar_wait_bounded(&tc.mbar, parity);
    tc.failed = 1;
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (tid == 0) tc.uses += 1u;
  if (tid < 2) sh.emax[tid] = 0u;  // next use is behind at least one more barrier
  return part;
}

// colour sum of the pair on the FP64 CUDA cores (C symmetric: column reads are row reads)
__device__ double colour_pair(Shared<double>& sh, const float* sC) {
  double part = 0.0;
  for (int i = threadIdx.x; i < Cfg<double>::NROW * T::NAMP; i += blockDim.x) {
    const int n = i / T::NAMP, m = i % T::NAMP;
    double y = 0.0;
    for (int l = 0; l < T::NAMP; ++l) y += (double)sC[l * T::NAMP + m] * sh.X[n][l];
    part += sh.X[n][m] * y;
  }
  __syncthreads();
  return part;
}

// Vertex sum of current i of tuple size S, amputated: the three-gluon terms
// V3(P_t, Q_t) and the four-gluon terms V4(P_i, M_ij, Q_j) of its prefixes
// P_t = J(s[:t]), suffixes Q_t = J(s[t:]) and middles M_ij = J(s[i:j]) (table
// kPQM, slot-major).  Each prefix is loaded once; with kc the current's own
// outgoing momentum, k(Q_t) = kc - k(P_t), so the three-gluon vertex (legs P, Q, X
// with kx = -kc) needs the prefix momentum only.
template <int S, class R>
__device__ __forceinline__ W4<R> vertex_sum(const JS<R>* J, const KS<R>* K, const P4<R>& kc, int i, R g, R g2) {
  constexpr int NP = S - 1, CNT = T::COUNT[S], OFF = T::PQM_OFF[S];
  const int16_t* ix = ME_GTN(kPQM) + OFF + i;
  W4<R> s;
#pragma unroll
  for (int k = 0; k < 4; ++k) s.c[k] = mk(R(0), R(0));
#pragma unroll
  for (int t = 1; t <= NP; ++t) {
    const int pa = ix[(t - 1) * CNT];
    const W4<R> Pj = ldj(J[pa]);
    const P4<R> k1 = ldk(K[pa]);
    {
      const W4<R> Qj = ldj(J[ix[(NP + t - 1) * CNT]]);
      // d12 = k1 - k2 = 2 k1 - kc, d2x = k2 - kx = 2 kc - k1, dx1 = kx - k1 = -(kc + k1)
      const P4<R> d12 = {R(2) * k1.e - kc.e, R(2) * k1.x - kc.x, R(2) * k1.y - kc.y, R(2) * k1.z - kc.z};
      const P4<R> d2x = {R(2) * kc.e - k1.e, R(2) * kc.x - k1.x, R(2) * kc.y - k1.y, R(2) * kc.z - k1.z};
      const P4<R> dx1 = {-(kc.e + k1.e), -(kc.x + k1.x), -(kc.y + k1.y), -(kc.z + k1.z)};
      const cx<R> j12 = mdot(Pj, Qj), av = mdot(d2x, Pj), bv = mdot(dx1, Qj);
      W4<R> o;
      o.c[0] = d12.e * j12 + Qj.c[0] * av + Pj.c[0] * bv;
      o.c[1] = d12.x * j12 + Qj.c[1] * av + Pj.c[1] * bv;
      o.c[2] = d12.y * j12 + Qj.c[2] * av + Pj.c[2] * bv;
      o.c[3] = d12.z * j12 + Qj.c[3] * av + Pj.c[3] * bv;
      acc(s, o, g);
    }
#pragma unroll
    for (int j = t + 1; j <= NP; ++j) {
      const int ma = ix[(2 * NP + (t - 1) * (2 * NP - t) / 2 + (j - t - 1)) * CNT];
      acc(s, v4(Pj, ldj(J[ma]), ldj(J[ix[(NP + j - 1) * CNT]])), g2);
    }
  }
  return s;
}

// currents of tuple sizes S..NG-2, one phase per size, a barrier after each
template <int S, class R>
__device__ __forceinline__ void current_phases(Shared<R>& sh, JS<R>* J, int lt, R g, R g2) {
  if constexpr (S <= NG - 2) {
    constexpr int CNT = T::COUNT[S], ST = T::START[S];
    for (int i = lt; i < CNT; i += kThreads) {
      const int c = ST + i;
      W4<R> s = vertex_sum<S, R>(J, sh.K, ldk(sh.K[c]), i, g, g2);
      const R f = sh.invp2[c];
#pragma unroll
      for (int k = 0; k < 4; ++k) s.c[k] = f * s.c[k];
      stj(J[c], s);
      ste(J[c], mdot(sh.eps0[0], s), mdot(sh.eps0[1], s));
    }
    __syncthreads();
    current_phases<S + 1, R>(sh, J, lt, g, g2);
  }
}

// Amplitudes of ordering a for both root helicities, from scalars only.  The
// amplitude is eps0_r . S with S the amputated vertex sum of the full tuple s;
// contracting each vertex term with eps0_r first gives, with e_r(J) = eps0_r . J
// and E_r(k) = eps0_r . k (momenta outgoing, kx = -(k1 + k2)):
//   three-gluon:  eps0.V3 = (E(k1) - E(k2)) (J1.J2) + e(J2) (k2 - kx).J1 + e(J1) (kx - k1).J2
//   four-gluon:   eps0.V4 = 2 (J1.J3) e(J2) - (J1.J2) e(J3) - (J2.J3) e(J1)
// (the vertices of v3 and v4 above), so that no four-vector sum is formed.  The
// terms use the prefixes P_t = J(s[:t]), suffixes Q_t = J(s[t:]) and middles
// M_ij = J(s[i:j]) of s: V3(P_t, Q_t) and V4(P_i, M_ij, Q_j).  Each prefix is
// loaded once; momentum conservation gives k(Q_t) = p0 - k(P_t), with p0 the root's
// physical momentum, so kx = -p0, and transversality eps0 . p0 = 0 gives
// E(k(Q_t)) = -E(k(P_t)).
template <class R>
__device__ __forceinline__ void amp_scalar(const JS<R>* J, const KS<R>* K, const KS<R>* EK, const P4<R>& p0, int a,
                                           R g, R g2, cx<R>& A0, cx<R>& A1) {
  constexpr int NP = NG - 2, CNT = T::NAMP, OFF = T::PQM_OFF[NG - 1];
  const int16_t* ix = ME_GTN(kPQM) + OFF + a;
  cx<R> s30 = mk(R(0), R(0)), s31 = s30, s40 = s30, s41 = s30;
#pragma unroll
  for (int i = 1; i <= NP; ++i) {
    const int pa = ix[(i - 1) * CNT];
    const W4<R> Pj = ldj(J[pa]);
    cx<R> ep0, ep1;
    lde(J[pa], ep0, ep1);
    const P4<R> k1 = ldk(K[pa]), q1 = ldk(EK[pa]);
    {
      const int qa = ix[(NP + i - 1) * CNT];
      const W4<R> Qj = ldj(J[qa]);
      cx<R> eq0, eq1;
      lde(J[qa], eq0, eq1);
      const P4<R> d2x = {R(2) * p0.e - k1.e, R(2) * p0.x - k1.x, R(2) * p0.y - k1.y, R(2) * p0.z - k1.z};
      const P4<R> dx1 = {-(k1.e + p0.e), -(k1.x + p0.x), -(k1.y + p0.y), -(k1.z + p0.z)};
      const cx<R> j12 = mdot(Pj, Qj), av = mdot(d2x, Pj), bv = mdot(dx1, Qj);
      s30 = s30 + mk(R(2) * q1.e, R(2) * q1.x) * j12 + eq0 * av + ep0 * bv;
      s31 = s31 + mk(R(2) * q1.y, R(2) * q1.z) * j12 + eq1 * av + ep1 * bv;
    }
#pragma unroll
    for (int j = i + 1; j <= NP; ++j) {
      const int ma = ix[(2 * NP + (i - 1) * (2 * NP - i) / 2 + (j - i - 1)) * CNT];
      const int qa = ix[(NP + j - 1) * CNT];
      const W4<R> Mj = ldj(J[ma]), Qj = ldj(J[qa]);
      cx<R> em0, em1, eq0, eq1;
      lde(J[ma], em0, em1);
      lde(J[qa], eq0, eq1);
      const cx<R> j13 = mdot(Pj, Qj), j12 = mdot(Pj, Mj), j23 = mdot(Mj, Qj);
      const cx<R> t13 = j13 + j13;
      s40 = s40 + t13 * em0 - j12 * eq0 - j23 * ep0;
      s41 = s41 + t13 * em1 - j12 * eq1 - j23 * ep1;
    }
  }
  A0 = R(2) * (g * s30 + g2 * s40);
  A1 = R(2) * (g * s31 + g2 * s41);
}

// |M|^2 of one event, computed by the whole block.  p: physical momenta (leg-major).
template <class R, class CS>
__device__ double event_block(const R (&p)[NG][4], R gs, Shared<R>& sh, CS cs) {
  constexpr int HP = Cfg<R>::HP;
  const int tid = threadIdx.x, hs = tid / kThreads, lt = tid % kThreads;
  // (1) momenta of the currents (externals are legs 1..NG-1; incoming legs carry -p),
  // the polarisation vectors of every leg for both helicities
  if (tid < NG - 1) {
    const int leg = tid + 1;
    const R sg = leg < 2 ? R(-1) : R(1);
    stk(sh.K[tid], P4<R>{sg * p[leg][0], sg * p[leg][1], sg * p[leg][2], sg * p[leg][3]});
  }
  if (tid >= 32 && tid < 32 + 2 * (NG - 1)) {
    const int leg = (tid - 32) / 2 + 1, h = tid & 1;
    const P4<R> k = {p[leg][0], p[leg][1], p[leg][2], p[leg][3]};
    stj(sh.ext[leg - 1][h], ext_vector<R>(k, h ? 1 : -1, leg < 2, R(0)));
  }
  if (tid >= 64 && tid < 66) {
    const P4<R> k0 = {p[0][0], p[0][1], p[0][2], p[0][3]};
    sh.eps0[tid - 64] = ext_vector<R>(k0, (tid - 64) ? 1 : -1, true, R(0));
  }
  __syncthreads();
  // composite momenta, 1/P^2, and the root contractions of every momentum and external vector
  for (int c = tid; c < T::NCUR; c += blockDim.x) {
    P4<R> k;
    if (c < NG - 1) {
      k = ldk(sh.K[c]);
    } else {
      const int mask = cur_meta()[4 * c];
      k = P4<R>{R(0), R(0), R(0), R(0)};
      for (int l = 1; l < NG; ++l)
        if ((mask >> l) & 1) k = k + ldk(sh.K[l - 1]);
      stk(sh.K[c], k);
      sh.invp2[c] = R(1) / msq(k);
    }
    const cx<R> q0 = mdot(k, sh.eps0[0]), q1 = mdot(k, sh.eps0[1]);
    stk(sh.EK[c], P4<R>{q0.re, q0.im, q1.re, q1.im});
  }
  if (tid >= 64 && tid < 64 + 2 * (NG - 1)) {
    JS<R>& x = sh.ext[(tid - 64) / 2][tid & 1];
    const W4<R> v = ldj(x);
    ste(x, mdot(sh.eps0[0], v), mdot(sh.eps0[1], v));
  }
  const R g = gs, g2 = gs * gs;
  JS<R>* J = sh.J[hs];
  __syncthreads();
  // external currents of the first helicity (later ones are set during the colour step)
  if (lt < NG - 1) J[lt] = sh.ext[lt][(hs >> lt) & 1];
  __syncthreads();
  R part = R(0);
  for (int hp = 0; hp < NHEL / HP; ++hp) {
    // (2a) currents, phase by phase
    current_phases<2, R>(sh, J, lt, g, g2);
    // (2b) amplitudes for both root helicities -> rows 4 hs .. 4 hs + 3
    unsigned e = 0u;
    const P4<R> p0 = {p[0][0], p[0][1], p[0][2], p[0][3]};
    for (int a = lt; a < T::NAMP; a += kThreads) {
      cx<R> a0, a1;
      amp_scalar<R>(J, sh.K, sh.EK, p0, a, g, g2, a0, a1);
      sh.X[4 * hs + 0][a] = a0.re;
      sh.X[4 * hs + 1][a] = a0.im;
      sh.X[4 * hs + 2][a] = a1.re;
      sh.X[4 * hs + 3][a] = a1.im;
      if constexpr (sizeof(R) == 4)
        e = max(max(max(e, exp_bits(a0.re)), max(exp_bits(a0.im), exp_bits(a1.re))), exp_bits(a1.im));
    }
    if constexpr (sizeof(R) == 4) {
      e = __reduce_max_sync(0xffffffffu, e);
      if ((lt & 31) == 0) atomicMax(&sh.emax[hs], e);
    }
    __syncthreads();
    // external currents of the next pair: J is not read again before the colour step's barriers
    if (lt < NG - 1 && hp + 1 < NHEL / HP) J[lt] = sh.ext[lt][((HP * (hp + 1) + hs) >> lt) & 1];
    // (2c) colour quadratic form of the pair's rows
    part += colour_pair(sh, cs);
  }
  // (3) block sum
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) part += __shfl_down_sync(0xffffffffu, part, o);
  if ((tid & 31) == 0) sh.red[tid >> 5] = part;
  __syncthreads();
  double tot = 0.0;
  if (tid == 0)
    for (int w = 0; w < (int)(blockDim.x / 32); ++w) tot += (double)sh.red[w];
  __syncthreads();
  // initial average 1/(4 * 8 * 8) and the colour denominator
  return tot * (1.0 / (256.0 * (double)T::DEN));
}

// colour operand in shared memory: FP16 C_off for the tensor cores, FP32 C_num for FP64
template <class R>
struct ColourSmem;
template <>
struct ColourSmem<float> {
  static constexpr size_t bytes = sizeof(TcShared);
  // the colour operand in the tcgen05 layout, the mbarrier, and the block's tensor memory (warp 0)
  static __device__ TcShared* load(unsigned char* p) {
    TcShared& tc = *reinterpret_cast<TcShared*>(p);
    for (int i = threadIdx.x; i < MT * KP; i += blockDim.x) {
      const int m = i / KP, k = i % KP;
      const float v = (m < T::NAMP && k < T::NAMP && m != k) ? colour()[m * T::NAMP + k] : 0.0f;
      *reinterpret_cast<__half*>(reinterpret_cast<char*>(tc.C) + tc_off(m, k)) = __float2half_rn(v);
    }
    if (threadIdx.x < 32) {
      asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(&tc.tmem)),
                   "r"(kTmemCols)
                   : "memory");
      asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (threadIdx.x == 0) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(&tc.mbar)), "r"(1) : "memory");
      asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
      tc.uses = 0u;
      tc.failed = 0;
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");  // the kernel's barrier follows
    return &tc;
  }
  // release the tensor memory (warp 0); every MMA has completed by now.  Returns whether the
  // block's tensor-core waits all finished in time.
  static __device__ bool release(TcShared* tcp) {
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    const bool ok = !tcp->failed;
    if (threadIdx.x < 32) {
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tcp->tmem), "r"(kTmemCols) : "memory");
    }
    return ok;
  }
};
template <>
struct ColourSmem<double> {
  static constexpr size_t bytes = sizeof(float) * T::NAMP * T::NAMP;
  static __device__ const float* load(unsigned char* p) {
    float* sC = reinterpret_cast<float*>(p);
    for (int i = threadIdx.x; i < T::NAMP * T::NAMP; i += blockDim.x) sC[i] = colour()[i];
    return sC;
  }
  static __device__ bool release(const float*) { return true; }
};

template <class R>
constexpr size_t shared_offset() {
  return (sizeof(Shared<R>) + 127) / 128 * 128;
}

template <class R>
__device__ __forceinline__ Shared<R>& setup(unsigned char* smem) {
  Shared<R>& sh = *reinterpret_cast<Shared<R>*>(smem);
  if (threadIdx.x < 2) sh.emax[threadIdx.x] = 0u;
  return sh;
}

template <class R>
constexpr int min_blocks() {
  return sizeof(R) == 4 ? 3 : 2;
}

template <class R>
__global__ void __launch_bounds__(Cfg<R>::THREADS, min_blocks<R>())
    k_eval_gluon(const double* __restrict__ mom, int64_t n, double* __restrict__ out, double gs) {
  extern __shared__ __align__(128) unsigned char smem[];
  Shared<R>& sh = setup<R>(smem);
  const auto cs = ColourSmem<R>::load(smem + shared_offset<R>());
  __shared__ R p[NG][4];
  __syncthreads();
  for (int64_t i = blockIdx.x; i < n; i += gridDim.x) {
    if (threadIdx.x < NG * 4) p[threadIdx.x / 4][threadIdx.x % 4] = (R)mom[(int64_t)threadIdx.x * n + i];
    __syncthreads();
    const double m2 = event_block<R>(p, (R)gs, sh, cs);
    if (threadIdx.x == 0) out[i] = m2;
    __syncthreads();
  }
  if (!ColourSmem<R>::release(cs) && threadIdx.x == 0) {
    // a tensor-core wait ran out in this block: its results are not to be trusted
    for (int64_t i = blockIdx.x; i < n; i += gridDim.x) out[i] = __longlong_as_double(0x7ff8000000000000ll);
  }
}

template <class R, bool MIXED>
__global__ void __launch_bounds__(Cfg<R>::THREADS, min_blocks<R>())
    k_me_gluon(KinDev kin, StepArgs a, double gs) {
  const int64_t m = a.m, out_stride = a.out_stride;
  const void* __restrict__ ws = a.ws;
  double* __restrict__ partials = a.partials;
  double* __restrict__ me2_out = a.me2_out;
  double* __restrict__ mom_out = a.mom_out;
  const int nslots = a.nslots;
  extern __shared__ __align__(128) unsigned char smem[];
  Shared<R>& sh = setup<R>(smem);
  const auto cs = ColourSmem<R>::load(smem + shared_offset<R>());
  __shared__ R p[NG][4];
  __syncthreads();
  const float* ph = reinterpret_cast<const float*>(ws);
  const float* pl = ph + (int64_t)NG * 4 * m;
  const double* pd = reinterpret_cast<const double*>(ws);
  const double* wps_a = reinterpret_cast<const double*>(MIXED ? (const void*)(pl + (int64_t)NG * 4 * m)
                                                              : (const void*)(pd + (int64_t)NG * 4 * m));
  const double* shat_a = wps_a + m;
  const int32_t* tries_a = reinterpret_cast<const int32_t*>(shat_a + m);
  double sw = 0.0, sw2 = 0.0;
  int64_t ntries = 0;
  for (int64_t i = blockIdx.x; i < m; i += gridDim.x) {
    const int t = threadIdx.x;
    if (t < NG * 4) {
      const int64_t idx = (int64_t)t * m + i;
      double v;
      if (MIXED) v = to_double(df{ph[idx], pl[idx]});
      else v = pd[idx];
      p[t / 4][t % 4] = (R)v;
      if (mom_out) mom_out[(int64_t)t * out_stride + i] = v;
    }
    __syncthreads();
    // mixed path: k_ps stored the weight factor as a double-float pair in the weight slot
    const float2 wf = reinterpret_cast<const float2*>(wps_a)[i];
    const double wps = MIXED ? 0.0 : wps_a[i], shat = shat_a[i];
    const bool ok = MIXED ? wf.x > 0.0f : wps > 0.0;
    double m2 = 0.0;
    if (ok) m2 = event_block<R>(p, (R)gs, sh, cs);
    if (t == 0) {
      const double w = !ok ? 0.0
                           : MIXED ? m2 * ((double)wf.x + (double)wf.y)
                                   : (kin.wfactor > 0.0 ? m2 * kin.wfactor
                                                        : wps * m2 * kin.s_ident / (2.0 * shat) * kGeV2pb);
      sw += w;
      sw2 = fma(w, w, sw2);
      ntries += tries_a[i];
      if (me2_out) me2_out[i] = m2;
      if (a.vg_w) a.vg_w[i] = w;
    }
    __syncthreads();
  }
  // a tensor-core wait that ran out is reported like an exhausted bounded loop (ME_ERR_TIMEOUT)
  if (!ColourSmem<R>::release(cs) && threadIdx.x == 0) atomicOr(a.status, 1);
  if (threadIdx.x == 0) {
    // this block's sums, and zeros in the slots of blocks the one-wave grid did not launch
    for (int b = blockIdx.x; b < nslots; b += gridDim.x) {
      const bool own = b == (int)blockIdx.x;
      partials[3 * b + 0] = own ? sw : 0.0;
      partials[3 * b + 1] = own ? sw2 : 0.0;
      partials[3 * b + 2] = own ? (double)ntries : 0.0;
    }
  }
}

template <class R>
size_t smem_bytes() {
  return shared_offset<R>() + ColourSmem<R>::bytes;
}

// dynamic shared memory opt-in, and the number of blocks of one resident wave (capped by `cap`)
template <class R, class K>
cudaError_t prepare(K kern, int cap, int& grid) {
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_bytes<R>());
  if (e != cudaSuccess) return e;
  if ((e = cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, 100)) != cudaSuccess) return e;
  int dev = 0, n_sm = 0, per_sm = 0;
  if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
  if ((e = cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
  if constexpr (sizeof(R) == 4) {
    // the occupancy calculator answers one block per SM for any kernel that allocates tensor memory,
    // whatever it allocates; blocks of 32 columns do run side by side, so count the limits here:
    // registers (per-warp allocation in units of 256), shared memory, threads, tensor-memory columns
    cudaFuncAttributes fa;
    int regs = 0, smem_sm = 0, reserved = 0, threads_sm = 0;
    if ((e = cudaFuncGetAttributes(&fa, kern)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&regs, cudaDevAttrMaxRegistersPerMultiprocessor, dev)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev)) != cudaSuccess)
      return e;
    if ((e = cudaDeviceGetAttribute(&reserved, cudaDevAttrReservedSharedMemoryPerBlock, dev)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&threads_sm, cudaDevAttrMaxThreadsPerMultiProcessor, dev)) != cudaSuccess)
      return e;
    const int warps = (Cfg<R>::THREADS + 31) / 32;
    const int regs_warp = (fa.numRegs * 32 + 255) / 256 * 256;
    const int by_regs = regs / (regs_warp * warps);
    const int by_smem = smem_sm / (int)(fa.sharedSizeBytes + smem_bytes<R>() + (size_t)reserved);
    const int by_threads = threads_sm / Cfg<R>::THREADS;
    const int by_tmem = 512 / (int)kTmemCols;
    per_sm = std::min(std::min(by_regs, by_smem), std::min(by_threads, by_tmem));
  } else if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, Cfg<R>::THREADS, smem_bytes<R>())) !=
             cudaSuccess) {
    return e;
  }
  if (per_sm < 1) return cudaErrorInvalidConfiguration;
  grid = n_sm * per_sm < cap ? n_sm * per_sm : cap;
  if (grid < 1) grid = 1;
  return cudaSuccess;
}

cudaError_t launch_eval(int prec, const double* mom, int64_t n, double* out, const double* params, cudaStream_t s,
                        int grid) {
  cudaError_t e;
  int g = 0;
  if (prec == ME_FP64) {
    if ((e = prepare<double>(k_eval_gluon<double>, grid, g)) != cudaSuccess) return e;
    k_eval_gluon<double><<<g, Cfg<double>::THREADS, smem_bytes<double>(), s>>>(mom, n, out, params[0]);
  } else {
    if ((e = prepare<float>(k_eval_gluon<float>, grid, g)) != cudaSuccess) return e;
    k_eval_gluon<float><<<g, Cfg<float>::THREADS, smem_bytes<float>(), s>>>(mom, n, out, params[0]);
  }
  return cudaGetLastError();
}

cudaError_t launch_step(int prec, const KinDev* kin, const StepArgs* a, const double* params, cudaStream_t s,
                        int grid_ps, int grid_me, cudaEvent_t ev_mid) {
  cudaError_t e;
  int g = 0;
  if ((e = launch_ps<Traits>(prec, kin, a, grid_ps, s)) != cudaSuccess) return e;
  if (ev_mid) cudaEventRecord(ev_mid, s);
  if (prec == ME_FP64) {
    if ((e = prepare<double>(k_me_gluon<double, false>, grid_me, g)) != cudaSuccess) return e;
    k_me_gluon<double, false><<<g, Cfg<double>::THREADS, smem_bytes<double>(), s>>>(*kin, *a, params[0]);
  } else {
    if ((e = prepare<float>(k_me_gluon<float, true>, grid_me, g)) != cudaSuccess) return e;
    k_me_gluon<float, true><<<g, Cfg<float>::THREADS, smem_bytes<float>(), s>>>(*kin, *a, params[0]);
  }
  return cudaGetLastError();
}

// the fused single-kernel step is not provided for gluon processes: the generic
// phase-space kernel without amplitudes serves me_generate
struct NoME {
  static constexpr int NEXT = NG;
  struct Params {
    double unused;
  };
  using ParamsMx = Params;
  static ParamsMx mixed_params(const Params& p) { return p; }
  static __host__ __device__ double eval64(const double (&)[NG][4], const Params&) { return 0.0; }
  static __host__ __device__ float evalmx(const df (&)[NG][4], const ParamsMx&) { return 0.0f; }
};

cudaError_t launch_xsec(int prec, const KinDev* kin, uint64_t seed, uint64_t offset, int64_t n, const double* params,
                        double* partials, double* me2_out, double* mom_out, double* wps_out, double* shat_out,
                        int32_t* tries_out, int* status, int eval_me, cudaStream_t s, int grid) {
  (void)params;
  if (eval_me || partials || me2_out) return cudaErrorNotSupported;
  if (kin->kind == ME_PS_YPT) {
    if (prec == ME_FP64)
      k_gen<NoME, false, ME_PS_YPT><<<grid, kThreads, 0, s>>>(*kin, seed, offset, n, mom_out, wps_out, shat_out,
                                                              tries_out, status);
    else
      k_gen<NoME, true, ME_PS_YPT><<<grid, kThreads, 0, s>>>(*kin, seed, offset, n, mom_out, wps_out, shat_out,
                                                             tries_out, status);
    return cudaGetLastError();
  }
  typename NoME::Params prm{0.0};
  if (prec == ME_FP64)
    k_xsec<NoME, false><<<grid, kThreads, 0, s>>>(*kin, seed, offset, n, prm, nullptr, nullptr, mom_out, wps_out,
                                                  shat_out, tries_out, status, 0);
  else
    k_xsec<NoME, true><<<grid, kThreads, 0, s>>>(*kin, seed, offset, n, prm, nullptr, nullptr, mom_out, wps_out,
                                                 shat_out, tries_out, status, 0);
  return cudaGetLastError();
}

}  // namespace g<NGLUON>
}  // namespace gluon
}  // namespace me

extern "C" void ME_CAT(me_register_gluon, NGLUON)(me::ProcessDesc* d) {
  d->n_ext = NGLUON;
  d->events_per_block = 1;
  d->launch_eval = me::gluon::ME_CAT(g, NGLUON)::launch_eval;
  d->launch_xsec = me::gluon::ME_CAT(g, NGLUON)::launch_xsec;
  d->launch_step = me::gluon::ME_CAT(g, NGLUON)::launch_step;
}
