// Kernels shared by every generated process unit.  A generated unit defines a
// traits struct P with NEXT (number of legs), Params, and two per-event
// evaluators: eval64 (FP64 path: FP64 momenta, FP64 amplitudes) and evalmx
// (mixed path: double-float momenta, FP32 amplitudes, double-float resonant
// invariants).  MIXED selects the path.
//
//   k_eval : one event per thread, momenta read coalesced from the
//            structure-of-arrays buffer into registers, |M|^2 written out.
//   k_xsec : the fused hot path of one Monte Carlo step, per tile of kThreads
//            points: (1) phase space with redraws through a shared-memory work
//            queue -- round r draws attempt r for every point still open, the
//            failures are compacted into the next round's queue, so warps stay
//            full instead of idling while single lanes redraw; accepted momenta
//            land in shared memory; (2) every thread evaluates |M|^2 of its own
//            point, forms the weight and accumulates (sum w, sum w^2, tries);
//            per block a fixed-order shuffle + shared-memory reduction writes one
//            partial, so the totals are deterministic for a given launch shape.
//            Each point's draws depend only on (seed, event, attempt).
// Both use a grid-stride loop over a grid sized in multiples of the SM count.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include "dfloat.cuh"
#include "heget.cuh"
#include "me_internal.h"
#include "phasespace.cuh"

// 1/(a + i b) formed in FP64 (a, b carry the cancellation-prone q^2 - m^2);
// the mixed path rounds the pair to FP32 first and inverts in FP32.
template <class R>
__host__ __device__ __forceinline__ me::cx<R> inv_den(double a, double b);
template <>
__host__ __device__ __forceinline__ me::cx<double> inv_den<double>(double a, double b) {
  const double d = 1.0 / (a * a + b * b);
  return me::mk(a * d, -b * d);
}
template <>
__host__ __device__ __forceinline__ me::cx<float> inv_den<float>(double a, double b) {
  const float fa = (float)a, fb = (float)b;
  const float d = 1.0f / (fa * fa + fb * fb);
  return me::mk(fa * d, -fb * d);
}
__host__ __device__ __forceinline__ me::cx<float> inv_den_f(float a, float b) {
  const float d = 1.0f / (a * a + b * b);
  return me::mk(a * d, -b * d);
}

namespace me {
constexpr double kGeV2pb = 0.3893793721e9;

__host__ __device__ __forceinline__ P4<float> p4f(const df* p) {
  return P4<float>{to_float(p[0]), to_float(p[1]), to_float(p[2]), to_float(p[3])};
}

// fixed-order block sum of three doubles into out[blockIdx.x * 3 + {0,1,2}]
__device__ __forceinline__ void block_reduce3(double a, double b, double c, double* out) {
  __shared__ double sm[3][kThreads / 32];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    a += __shfl_down_sync(0xffffffffu, a, o);
    b += __shfl_down_sync(0xffffffffu, b, o);
    c += __shfl_down_sync(0xffffffffu, c, o);
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) { sm[0][warp] = a; sm[1][warp] = b; sm[2][warp] = c; }
  __syncthreads();
  if (threadIdx.x == 0) {
    double s0 = 0, s1 = 0, s2 = 0;
    for (int w = 0; w < kThreads / 32; ++w) { s0 += sm[0][w]; s1 += sm[1][w]; s2 += sm[2][w]; }
    out[3 * blockIdx.x + 0] = s0;
    out[3 * blockIdx.x + 1] = s1;
    out[3 * blockIdx.x + 2] = s2;
  }
}

template <class P, bool MIXED>
__global__ void __launch_bounds__(kThreads) k_eval(const double* __restrict__ mom, int64_t n,
                                                   double* __restrict__ out, typename P::Params prm) {
  constexpr int NEXT = P::NEXT;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    if constexpr (MIXED) {
      df pm[NEXT][4];
#pragma unroll
      for (int k = 0; k < NEXT; ++k) {
#pragma unroll
        for (int m = 0; m < 4; ++m) pm[k][m] = from_double(__ldg(mom + ((int64_t)(k * 4 + m)) * n + i));
      }
      out[i] = P::evalmx(pm, prm);
    } else {
      double pm[NEXT][4];
#pragma unroll
      for (int k = 0; k < NEXT; ++k) {
#pragma unroll
        for (int m = 0; m < 4; ++m) pm[k][m] = __ldg(mom + ((int64_t)(k * 4 + m)) * n + i);
      }
      out[i] = P::eval64(pm, prm);
    }
  }
}

template <class P, bool MIXED>
__global__ void __launch_bounds__(kThreads) k_xsec(KinDev kin, uint64_t seed, uint64_t offset, int64_t n,
                                                   typename P::Params prm, double* __restrict__ partials,
                                                   double* __restrict__ me2_out, double* __restrict__ mom_out,
                                                   double* __restrict__ wps_out, double* __restrict__ shat_out,
                                                   int32_t* __restrict__ tries_out, int* status, int eval_me) {
  constexpr int NEXT = P::NEXT;
  // accepted momenta of the tile: FP64 (hi) or double-float (hi, lo) per component
  __shared__ double s_pd[MIXED ? 1 : NEXT * 4][kThreads];
  __shared__ float s_ph[MIXED ? NEXT * 4 : 1][kThreads];
  __shared__ float s_pl[MIXED ? NEXT * 4 : 1][kThreads];
  __shared__ double s_wps[kThreads], s_shat[kThreads];
  __shared__ int s_tries[kThreads];
  __shared__ int s_q[2][kThreads];
  __shared__ int s_qn[2];
  double sw = 0.0, sw2 = 0.0, nt = 0.0;
  const int64_t ntiles = (n + kThreads - 1) / kThreads;
  for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const int64_t base = tile * kThreads;
    const int cnt = (int)((n - base) < kThreads ? (n - base) : kThreads);
    if (threadIdx.x == 0) { s_qn[0] = 0; s_qn[1] = 0; }
    if (threadIdx.x < cnt) { s_wps[threadIdx.x] = 0.0; s_tries[threadIdx.x] = kin.max_attempts; }
    __syncthreads();
    int cur = 0;
    for (int att = 0;; ++att) {
      const int nitems = (att == 0) ? cnt : s_qn[cur];
      if (nitems == 0) break;
      if (att >= kin.max_attempts) {
        if (threadIdx.x == 0) atomicOr(status, 1);
        break;
      }
      const int nxt = cur ^ 1;
      for (int j = threadIdx.x; j < nitems; j += kThreads) {
        const int ev = (att == 0) ? j : s_q[cur][j];
        const uint64_t event = offset + (uint64_t)(base + ev);
        double wps = 0.0, shat = 1.0;
        bool ok;
        if constexpr (MIXED) {
          df pm[NEXT][4];
          ok = draw_point_df<NEXT>(kin, seed, event, att, pm, wps, shat);
          if (ok) {
#pragma unroll
            for (int k = 0; k < NEXT; ++k) {
#pragma unroll
              for (int m = 0; m < 4; ++m) { s_ph[k * 4 + m][ev] = pm[k][m].hi; s_pl[k * 4 + m][ev] = pm[k][m].lo; }
            }
          }
        } else {
          double pm[NEXT][4];
          ok = draw_point<NEXT>(kin, seed, event, att, pm, wps, shat);
          if (ok) {
#pragma unroll
            for (int k = 0; k < NEXT; ++k) {
#pragma unroll
              for (int m = 0; m < 4; ++m) s_pd[k * 4 + m][ev] = pm[k][m];
            }
          }
        }
        if (ok) {
          s_wps[ev] = wps;
          s_shat[ev] = shat;
          s_tries[ev] = att + 1;
        } else {
          s_q[nxt][atomicAdd(&s_qn[nxt], 1)] = ev;
        }
      }
      __syncthreads();
      if (threadIdx.x == 0) s_qn[cur] = 0;
      cur = nxt;
      __syncthreads();
    }
    if (threadIdx.x < cnt) {
      const int ev = threadIdx.x;
      const int64_t i = base + ev;
      const double wps = s_wps[ev], shat = s_shat[ev];
      const int tries = s_tries[ev];
      const bool ok = wps > 0.0;
      double m2 = 0.0;
      if constexpr (MIXED) {
        df pm[NEXT][4];
#pragma unroll
        for (int k = 0; k < NEXT; ++k) {
#pragma unroll
          for (int m = 0; m < 4; ++m) pm[k][m] = df{s_ph[k * 4 + m][ev], s_pl[k * 4 + m][ev]};
        }
        if (eval_me && ok) m2 = P::evalmx(pm, prm);
        if (mom_out) {
#pragma unroll
          for (int k = 0; k < NEXT; ++k) {
#pragma unroll
            for (int m = 0; m < 4; ++m) mom_out[((int64_t)(k * 4 + m)) * n + i] = to_double(pm[k][m]);
          }
        }
      } else {
        double pm[NEXT][4];
#pragma unroll
        for (int k = 0; k < NEXT; ++k) {
#pragma unroll
          for (int m = 0; m < 4; ++m) pm[k][m] = s_pd[k * 4 + m][ev];
        }
        if (eval_me && ok) m2 = P::eval64(pm, prm);
        if (mom_out) {
#pragma unroll
          for (int k = 0; k < NEXT; ++k) {
#pragma unroll
            for (int m = 0; m < 4; ++m) mom_out[((int64_t)(k * 4 + m)) * n + i] = pm[k][m];
          }
        }
      }
      const double w = ok ? wps * m2 * kin.s_ident / (2.0 * shat) * kGeV2pb : 0.0;
      sw += w;
      sw2 += w * w;
      nt += (double)tries;
      if (me2_out) me2_out[i] = m2;
      if (wps_out) wps_out[i] = wps;
      if (shat_out) shat_out[i] = shat;
      if (tries_out) tries_out[i] = tries;
    }
    __syncthreads();
  }
  if (partials) block_reduce3(sw, sw2, nt, partials);
}

template <class P>
cudaError_t launch_eval(int prec, const double* mom, int64_t n, double* out, const double* params, cudaStream_t s,
                        int grid) {
  typename P::Params prm;
  memcpy(&prm, params, sizeof(prm));
  if (prec == ME_FP64) k_eval<P, false><<<grid, kThreads, 0, s>>>(mom, n, out, prm);
  else k_eval<P, true><<<grid, kThreads, 0, s>>>(mom, n, out, prm);
  return cudaGetLastError();
}

template <class P>
cudaError_t launch_xsec(int prec, const KinDev* kin, uint64_t seed, uint64_t offset, int64_t n, const double* params,
                        double* partials, double* me2_out, double* mom_out, double* wps_out, double* shat_out,
                        int32_t* tries_out, int* status, int eval_me, cudaStream_t s, int grid) {
  typename P::Params prm;
  memcpy(&prm, params, sizeof(prm));
  if (prec == ME_FP64)
    k_xsec<P, false><<<grid, kThreads, 0, s>>>(*kin, seed, offset, n, prm, partials, me2_out, mom_out, wps_out,
                                               shat_out, tries_out, status, eval_me);
  else
    k_xsec<P, true><<<grid, kThreads, 0, s>>>(*kin, seed, offset, n, prm, partials, me2_out, mom_out, wps_out,
                                              shat_out, tries_out, status, eval_me);
  return cudaGetLastError();
}
}  // namespace me

#define ME_DEFINE_PROCESS(TAG, NEXT_, NPARAM)                                       \
  extern "C" void me_register_##TAG(me::ProcessDesc* d) {                           \
    static_assert(sizeof(me::TAG::Traits::Params) == NPARAM * sizeof(double), "parameter block"); \
    d->n_ext = NEXT_;                                                               \
    d->launch_eval = me::launch_eval<me::TAG::Traits>;                              \
    d->launch_xsec = me::launch_xsec<me::TAG::Traits>;                              \
  }
