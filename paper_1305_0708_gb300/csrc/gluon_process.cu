// Process unit for NGLUON gluons (compiled once per gluon count with -DNGLUON=n).
// Kernels: k_eval_gluon (|M|^2 from momenta in HBM) and, for the Monte Carlo
// step, the generic phase-space kernel k_ps followed by k_me_gluon.  One thread
// block evaluates one event at a time (grid-stride over events).
#include <cstdint>
#include <cstring>

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

struct Traits {
  static constexpr int NEXT = NG;
  struct Params {
    double GS;
  };
};

__host__ __device__ __forceinline__ const int32_t* cur_meta() { return ME_GTN(kCurMeta); }
__host__ __device__ __forceinline__ const int16_t* cur_terms() { return ME_GTN(kCurTerms); }
__host__ __device__ __forceinline__ const int32_t* amp_meta() { return ME_GTN(kAmpMeta); }
__host__ __device__ __forceinline__ const int16_t* amp_terms() { return ME_GTN(kAmpTerms); }
__host__ __device__ __forceinline__ const int32_t* phases() { return ME_GTN(kPhase); }
__host__ __device__ __forceinline__ const float* colour() { return ME_GTN(kColour); }

template <class R>
struct Shared {
  P4<R> K[T::NCUR];       // outgoing momenta of every current (externals first)
  R invp2[T::NCUR];
  W4<R> J[T::NCUR];       // currents of the helicity being evaluated
  W4<R> eps0[2];          // root polarisation, both helicities
  cx<R> A[2][T::NAMP];    // amplitudes of both root helicities
  R red[kThreads / 32];
};

// |M|^2 of one event, computed by the whole block.  p: physical momenta (leg-major).
template <class R>
__device__ double event_block(const R (&p)[NG][4], R gs, Shared<R>& sh, const float* sC) {
  const int tid = threadIdx.x;
  // (1) momenta of the currents: externals are legs 1..NG-1; incoming legs carry -p
  if (tid < NG - 1) {
    const int leg = tid + 1;
    const R sg = leg < 2 ? R(-1) : R(1);
    sh.K[tid] = P4<R>{sg * p[leg][0], sg * p[leg][1], sg * p[leg][2], sg * p[leg][3]};
  }
  if (tid < 2) {
    const P4<R> k0 = {p[0][0], p[0][1], p[0][2], p[0][3]};
    sh.eps0[tid] = ext_vector<R>(k0, tid ? 1 : -1, true, R(0));
  }
  __syncthreads();
  for (int c = NG - 1 + tid; c < T::NCUR; c += blockDim.x) {
    const int mask = cur_meta()[4 * c];
    P4<R> k = {R(0), R(0), R(0), R(0)};
    for (int l = 1; l < NG; ++l)
      if ((mask >> l) & 1) k = k + sh.K[l - 1];
    sh.K[c] = k;
    sh.invp2[c] = R(1) / msq(k);
  }
  __syncthreads();
  const R g = gs, g2 = gs * gs;
  R part = R(0);
  for (int hl = 0; hl < (1 << (NG - 1)); ++hl) {
    // (2a) external polarisation vectors of legs 1..NG-1 for this helicity
    if (tid < NG - 1) {
      const int leg = tid + 1;
      const int hel = ((hl >> tid) & 1) ? 1 : -1;
      const P4<R> k = {p[leg][0], p[leg][1], p[leg][2], p[leg][3]};
      sh.J[tid] = ext_vector<R>(k, hel, leg < 2, R(0));
    }
    __syncthreads();
    // (2b) currents, phase by phase
    for (int ph = 0; ph < T::NPHASE; ++ph) {
      const int start = phases()[2 * ph], count = phases()[2 * ph + 1];
      for (int i = tid; i < count; i += blockDim.x) {
        const int c = start + i;
        W4<R> s = entry_sum<R>(cur_meta() + 4 * c, cur_terms(), sh.J, sh.K, g, g2);
        const R f = sh.invp2[c];
#pragma unroll
        for (int k = 0; k < 4; ++k) s.c[k] = f * s.c[k];
        sh.J[c] = s;
      }
      __syncthreads();
    }
    // (2c) amplitudes for both root helicities
    for (int a = tid; a < T::NAMP; a += blockDim.x) {
      const W4<R> s = entry_sum<R>(amp_meta() + 4 * a, amp_terms(), sh.J, sh.K, g, g2);
      sh.A[0][a] = R(2) * mdot(sh.eps0[0], s);
      sh.A[1][a] = R(2) * mdot(sh.eps0[1], s);
    }
    __syncthreads();
    // (2d) colour quadratic form: sum_kl C_kl Re(A_k^* A_l), row k per thread
    for (int k = tid; k < T::NAMP; k += blockDim.x) {
      R y0r = R(0), y0i = R(0), y1r = R(0), y1i = R(0);
      const float* row = sC + k * T::NAMP;
      for (int l = 0; l < T::NAMP; ++l) {
        const R c = (R)row[l];
        y0r += c * sh.A[0][l].re;
        y0i += c * sh.A[0][l].im;
        y1r += c * sh.A[1][l].re;
        y1i += c * sh.A[1][l].im;
      }
      part += sh.A[0][k].re * y0r + sh.A[0][k].im * y0i + sh.A[1][k].re * y1r + sh.A[1][k].im * y1i;
    }
    __syncthreads();
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

__device__ __forceinline__ void load_colour(float* sC) {
  for (int i = threadIdx.x; i < T::NAMP * T::NAMP; i += blockDim.x) sC[i] = colour()[i];
  __syncthreads();
}

template <class R>
__global__ void __launch_bounds__(kThreads) k_eval_gluon(const double* __restrict__ mom, int64_t n,
                                                         double* __restrict__ out, double gs) {
  extern __shared__ __align__(16) unsigned char smem[];
  Shared<R>& sh = *reinterpret_cast<Shared<R>*>(smem);
  float* sC = reinterpret_cast<float*>(smem + sizeof(Shared<R>));
  load_colour(sC);
  __shared__ R p[NG][4];
  for (int64_t i = blockIdx.x; i < n; i += gridDim.x) {
    if (threadIdx.x < NG * 4) p[threadIdx.x / 4][threadIdx.x % 4] = (R)mom[(int64_t)threadIdx.x * n + i];
    __syncthreads();
    const double m2 = event_block<R>(p, (R)gs, sh, sC);
    if (threadIdx.x == 0) out[i] = m2;
    __syncthreads();
  }
}

template <class R, bool MIXED>
__global__ void __launch_bounds__(kThreads) k_me_gluon(KinDev kin, int64_t m, const void* __restrict__ ws, double gs,
                                                       double* __restrict__ partials, double* __restrict__ me2_out,
                                                       double* __restrict__ mom_out, int64_t out_stride) {
  extern __shared__ __align__(16) unsigned char smem[];
  Shared<R>& sh = *reinterpret_cast<Shared<R>*>(smem);
  float* sC = reinterpret_cast<float*>(smem + sizeof(Shared<R>));
  load_colour(sC);
  __shared__ R p[NG][4];
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
    const double wps = wps_a[i], shat = shat_a[i];
    const bool ok = wps > 0.0;
    double m2 = 0.0;
    if (ok) m2 = event_block<R>(p, (R)gs, sh, sC);
    if (t == 0) {
      const double w = !ok ? 0.0 : (kin.wfactor > 0.0 ? m2 * kin.wfactor
                                                       : wps * m2 * kin.s_ident / (2.0 * shat) * kGeV2pb);
      sw += w;
      sw2 = fma(w, w, sw2);
      ntries += tries_a[i];
      if (me2_out) me2_out[i] = m2;
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    partials[3 * blockIdx.x + 0] = sw;
    partials[3 * blockIdx.x + 1] = sw2;
    partials[3 * blockIdx.x + 2] = (double)ntries;
  }
}

template <class R>
size_t smem_bytes() {
  return sizeof(Shared<R>) + sizeof(float) * T::NAMP * T::NAMP;
}

template <class R, class K>
cudaError_t prepare(K kern) {
  return cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_bytes<R>());
}

cudaError_t launch_eval(int prec, const double* mom, int64_t n, double* out, const double* params, cudaStream_t s,
                        int grid) {
  cudaError_t e;
  if (prec == ME_FP64) {
    if ((e = prepare<double>(k_eval_gluon<double>)) != cudaSuccess) return e;
    k_eval_gluon<double><<<grid, kThreads, smem_bytes<double>(), s>>>(mom, n, out, params[0]);
  } else {
    if ((e = prepare<float>(k_eval_gluon<float>)) != cudaSuccess) return e;
    k_eval_gluon<float><<<grid, kThreads, smem_bytes<float>(), s>>>(mom, n, out, params[0]);
  }
  return cudaGetLastError();
}

cudaError_t launch_step(int prec, const KinDev* kin, uint64_t seed, uint64_t offset, int64_t m, const double* params,
                        void* ws, double* partials, double* me2_out, double* mom_out, int64_t out_stride, int* status,
                        cudaStream_t s, int grid_ps, int grid_me, cudaEvent_t ev_mid) {
  cudaError_t e;
  if (prec == ME_FP64) k_ps<Traits, false><<<grid_ps, kThreads, 0, s>>>(*kin, seed, offset, m, ws, status);
  else k_ps<Traits, true><<<grid_ps, kThreads, 0, s>>>(*kin, seed, offset, m, ws, status);
  if (ev_mid) cudaEventRecord(ev_mid, s);
  if (prec == ME_FP64) {
    if ((e = prepare<double>(k_me_gluon<double, false>)) != cudaSuccess) return e;
    k_me_gluon<double, false><<<grid_me, kThreads, smem_bytes<double>(), s>>>(*kin, m, ws, params[0], partials,
                                                                              me2_out, mom_out, out_stride);
  } else {
    if ((e = prepare<float>(k_me_gluon<float, true>)) != cudaSuccess) return e;
    k_me_gluon<float, true><<<grid_me, kThreads, smem_bytes<float>(), s>>>(*kin, m, ws, params[0], partials, me2_out,
                                                                           mom_out, out_stride);
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
  static __host__ __device__ double eval64(const double (&)[NG][4], const Params&) { return 0.0; }
  static __host__ __device__ double evalmx(const df (&)[NG][4], const Params&) { return 0.0; }
};

cudaError_t launch_xsec(int prec, const KinDev* kin, uint64_t seed, uint64_t offset, int64_t n, const double* params,
                        double* partials, double* me2_out, double* mom_out, double* wps_out, double* shat_out,
                        int32_t* tries_out, int* status, int eval_me, cudaStream_t s, int grid) {
  (void)params;
  if (eval_me || partials || me2_out) return cudaErrorNotSupported;
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
  d->launch_eval = me::gluon::ME_CAT(g, NGLUON)::launch_eval;
  d->launch_xsec = me::gluon::ME_CAT(g, NGLUON)::launch_xsec;
  d->launch_step = me::gluon::ME_CAT(g, NGLUON)::launch_step;
}
