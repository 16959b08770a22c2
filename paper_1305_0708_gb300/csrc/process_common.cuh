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
#include <type_traits>
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

// parameter block of a kernel: FP64 values (FP64 path) or the host-converted FP32 /
// double-float values of the mixed path
template <class P, bool MIXED>
using PrmT = typename std::conditional<MIXED, typename P::ParamsMx, typename P::Params>::type;

__host__ __device__ __forceinline__ P4<float> p4f(const df* p) {
  return P4<float>{to_float(p[0]), to_float(p[1]), to_float(p[2]), to_float(p[3])};
}

// fixed-order block sum of three doubles into out[slot * 3 + {0,1,2}] (slot: the block's index by default)
__device__ __forceinline__ void block_reduce3(double a, double b, double c, double* out, int64_t slot = -1) {
  if (slot < 0) slot = blockIdx.x;
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
    out[3 * slot + 0] = s0;
    out[3 * slot + 1] = s1;
    out[3 * slot + 2] = s2;
  }
}

template <class P, bool MIXED>
__global__ void __launch_bounds__(kThreads) k_eval(const double* __restrict__ mom, int64_t n,
                                                   double* __restrict__ out, PrmT<P, MIXED> prm) {
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

// shared memory of one tile of the fused step: accepted momenta (FP64, or double-float
// hi and lo), weights, draws and the redraw queue
template <class P, bool MIXED>
struct XsecTileSmem {
  double pd[MIXED ? 1 : P::NEXT * 4][kThreads];
  float ph[MIXED ? P::NEXT * 4 : 1][kThreads];
  float pl[MIXED ? P::NEXT * 4 : 1][kThreads];
  double wps[kThreads], shat[kThreads];
  int tries[kThreads];
  int q[2][kThreads];
  int qn[2];
};

// a thread's Monte Carlo sums (the mixed path sums FP32 weights as double-floats)
struct XsecSums {
  double sw = 0.0, sw2 = 0.0, nt = 0.0;
  df swf = df{0.0f, 0.0f}, sw2f = df{0.0f, 0.0f};
};

// One tile of the fused step: points [base, base + cnt) (cnt <= kThreads) of a step over
// events offset + i whose optional outputs have n points per component.  Phase space with
// redraws through the shared-memory queue, then every thread evaluates |M|^2 of its own
// point and adds its weight to acc.  Ends with a block barrier.
template <class P, bool MIXED>
__device__ __forceinline__ void xsec_tile(const KinDev& kin, uint64_t seed, uint64_t offset, int64_t n, int64_t base,
                                          int cnt, const PrmT<P, MIXED>& prm, double* __restrict__ me2_out,
                                          double* __restrict__ mom_out, double* __restrict__ wps_out,
                                          double* __restrict__ shat_out, int32_t* __restrict__ tries_out, int* status,
                                          int eval_me, XsecTileSmem<P, MIXED>& sm, XsecSums& acc) {
  constexpr int NEXT = P::NEXT;
  if (threadIdx.x == 0) { sm.qn[0] = 0; sm.qn[1] = 0; }
  if (threadIdx.x < cnt) { sm.wps[threadIdx.x] = 0.0; sm.tries[threadIdx.x] = kin.max_attempts; }
  __syncthreads();
  int cur = 0;
  for (int att = 0;; ++att) {
    const int nitems = (att == 0) ? cnt : sm.qn[cur];
    if (nitems == 0) break;
    if (att >= kin.max_attempts) {
      if (threadIdx.x == 0) atomicOr(status, 1);
      break;
    }
    const int nxt = cur ^ 1;
    for (int j = threadIdx.x; j < nitems; j += kThreads) {
      const int ev = (att == 0) ? j : sm.q[cur][j];
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
            for (int m = 0; m < 4; ++m) { sm.ph[k * 4 + m][ev] = pm[k][m].hi; sm.pl[k * 4 + m][ev] = pm[k][m].lo; }
          }
        }
      } else {
        double pm[NEXT][4];
        ok = draw_point<NEXT>(kin, seed, event, att, pm, wps, shat);
        if (ok) {
#pragma unroll
          for (int k = 0; k < NEXT; ++k) {
#pragma unroll
            for (int m = 0; m < 4; ++m) sm.pd[k * 4 + m][ev] = pm[k][m];
          }
        }
      }
      if (ok) {
        sm.wps[ev] = wps;
        sm.shat[ev] = shat;
        sm.tries[ev] = att + 1;
      } else {
        sm.q[nxt][atomicAdd(&sm.qn[nxt], 1)] = ev;
      }
    }
    __syncthreads();
    if (threadIdx.x == 0) sm.qn[cur] = 0;
    cur = nxt;
    __syncthreads();
  }
  if (threadIdx.x < cnt) {
    const int ev = threadIdx.x;
    const int64_t i = base + ev;
    const double wps = sm.wps[ev], shat = sm.shat[ev];
    const int tries = sm.tries[ev];
    const bool ok = wps > 0.0;
    double m2 = 0.0;
    if constexpr (MIXED) {
      df pm[NEXT][4];
#pragma unroll
      for (int k = 0; k < NEXT; ++k) {
#pragma unroll
        for (int m = 0; m < 4; ++m) pm[k][m] = df{sm.ph[k * 4 + m][ev], sm.pl[k * 4 + m][ev]};
      }
      const float m2f = (eval_me && ok) ? P::evalmx(pm, prm) : 0.0f;
      m2 = (double)m2f;
      if (mom_out) {
#pragma unroll
        for (int k = 0; k < NEXT; ++k) {
#pragma unroll
          for (int m = 0; m < 4; ++m) mom_out[((int64_t)(k * 4 + m)) * n + i] = to_double(pm[k][m]);
        }
      }
      if (ok) {
        const df wf = kin.wfactor > 0.0 ? from_double(kin.wfactor)
                                        : (from_double(wps) * from_double(kin.s_ident * (0.5 * kGeV2pb))) /
                                              from_double(shat);
        const float w = m2f * wf.hi;
        acc.swf = acc.swf + w;
        acc.sw2f = acc.sw2f + two_prod(w, w);
      }
    } else {
      double pm[NEXT][4];
#pragma unroll
      for (int k = 0; k < NEXT; ++k) {
#pragma unroll
        for (int m = 0; m < 4; ++m) pm[k][m] = sm.pd[k * 4 + m][ev];
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
    if constexpr (!MIXED) {
      const double w = ok ? wps * m2 * kin.s_ident / (2.0 * shat) * kGeV2pb : 0.0;
      acc.sw += w;
      acc.sw2 += w * w;
    }
    acc.nt += (double)tries;
    if (me2_out) me2_out[i] = m2;
    if (wps_out) wps_out[i] = wps;
    if (shat_out) shat_out[i] = shat;
    if (tries_out) tries_out[i] = tries;
  }
  __syncthreads();
}

template <class P, bool MIXED>
__device__ __forceinline__ void finish_sums(XsecSums& acc) {
  if constexpr (MIXED) {
    acc.sw = to_double(acc.swf);
    acc.sw2 = to_double(acc.sw2f);
  }
}

template <class P, bool MIXED>
__global__ void __launch_bounds__(kThreads) k_xsec(KinDev kin, uint64_t seed, uint64_t offset, int64_t n,
                                                   PrmT<P, MIXED> prm, double* __restrict__ partials,
                                                   double* __restrict__ me2_out, double* __restrict__ mom_out,
                                                   double* __restrict__ wps_out, double* __restrict__ shat_out,
                                                   int32_t* __restrict__ tries_out, int* status, int eval_me) {
  __shared__ XsecTileSmem<P, MIXED> sm;
  XsecSums acc;
  const int64_t ntiles = (n + kThreads - 1) / kThreads;
  for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const int64_t base = tile * kThreads;
    const int cnt = (int)((n - base) < kThreads ? (n - base) : kThreads);
    xsec_tile<P, MIXED>(kin, seed, offset, n, base, cnt, prm, me2_out, mom_out, wps_out, shat_out, tries_out, status,
                        eval_me, sm, acc);
  }
  finish_sums<P, MIXED>(acc);
  if (partials) block_reduce3(acc.sw, acc.sw2, acc.nt, partials);
}

// ---------------------------------------------------------------------------
// k_serve: the persistent kernel of the request server.  Each block claims queue
// items (one tile of one request each) until the host closes the queue, runs the
// fused step on the tile's points, writes the tile's partial sums, and the block
// that completes the last tile of a request sums its partials in tile order and
// publishes the totals to the host.  A block that has waited spin_limit times
// (about 1 us each) for an item that was neither published nor closed sets
// timed_out and returns: the host sees the kernel end and fails the requests left.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t ld_acquire_sys_u32(const uint32_t* p) {
  uint32_t v;
#ifdef __CUDA_ARCH__
  asm volatile("ld.acquire.sys.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
#else
  v = *p;
#endif
  return v;
}
__device__ __forceinline__ void st_release_sys_u32(uint32_t* p, uint32_t v) {
#ifdef __CUDA_ARCH__
  asm volatile("st.release.sys.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
#else
  *p = v;
#endif
}

template <class P, bool MIXED>
__global__ void __launch_bounds__(kThreads) k_serve(ServeCtl c, PrmT<P, MIXED> prm) {
  __shared__ XsecTileSmem<P, MIXED> sm;
  __shared__ KinDev s_kin;
  __shared__ ServeItem s_it;
  __shared__ ServeReq s_rq;
  __shared__ int s_state, s_kin_idx, s_last;
  if (threadIdx.x == 0) s_kin_idx = -1;
  for (;;) {
    __syncthreads();  // the previous item is done with every shared buffer
    if (threadIdx.x == 0) {
      const uint32_t idx = atomicAdd(c.claim, 1u);
#ifdef __CUDA_ARCH__
      asm volatile("st.relaxed.sys.global.u32 [%0], %1;" ::"l"(c.claimed), "r"(idx + 1u) : "memory");
#endif
      int state = -2;
      for (uint64_t it = 0; it <= c.spin_limit; ++it) {
        if (idx < ld_acquire_sys_u32(c.published)) {
          state = (int)idx;
          break;
        }
        if (ld_acquire_sys_u32(c.closed)) {  // the host publishes every item before it closes
          state = idx < ld_acquire_sys_u32(c.published) ? (int)idx : -1;
          break;
        }
#ifdef __CUDA_ARCH__
        __nanosleep(1000);
#endif
      }
      if (state == -2) {
        st_release_sys_u32(c.timed_out, 1u);
      } else if (state >= 0) {
        s_it = c.items[state];
        s_rq = c.reqs[s_it.req];
      }
      s_state = state;
    }
    __syncthreads();
    if (s_state < 0) return;
    const ServeItem it = s_it;
    if (it.kin != s_kin_idx) {
      const uint32_t* src = reinterpret_cast<const uint32_t*>(c.kins + it.kin);
      uint32_t* dst = reinterpret_cast<uint32_t*>(&s_kin);
      for (int w = threadIdx.x; w < (int)(sizeof(KinDev) / 4); w += kThreads) dst[w] = src[w];
      __syncthreads();
      if (threadIdx.x == 0) s_kin_idx = it.kin;
    }
    XsecSums acc;
    const int64_t end = it.first + it.count;
    for (int64_t base = it.first; base < end; base += kThreads) {
      const int cnt = (int)((end - base) < kThreads ? (end - base) : kThreads);
      xsec_tile<P, MIXED>(s_kin, it.seed, it.offset, it.n, base, cnt, prm, s_rq.me2, s_rq.mom, nullptr, nullptr,
                          nullptr, s_rq.status, 1, sm, acc);
    }
    finish_sums<P, MIXED>(acc);
    block_reduce3(acc.sw, acc.sw2, acc.nt, s_rq.partials, it.tile);
    if (threadIdx.x == 0) {
      __threadfence();
      s_last = atomicAdd(s_rq.tiles_done, 1u) + 1u == (uint32_t)s_rq.tiles;
    }
    __syncthreads();
    if (s_last) {
      // the request's tile partials in a fixed order: thread t sums tiles t, t + kThreads, ...,
      // then the block's fixed-order reduction (the same for every run of the request)
      __threadfence();
      double t0 = 0.0, t1 = 0.0, t2 = 0.0;
      for (int k = threadIdx.x; k < s_rq.tiles; k += kThreads) {
        t0 += __ldcg(s_rq.partials + 3 * k);
        t1 += __ldcg(s_rq.partials + 3 * k + 1);
        t2 += __ldcg(s_rq.partials + 3 * k + 2);
      }
      __shared__ double s_tot[3];
      block_reduce3(t0, t1, t2, s_tot, 0);
      if (threadIdx.x == 0) {
        s_rq.totals[0] = s_tot[0];
        s_rq.totals[1] = s_tot[1];
        s_rq.totals[2] = s_tot[2];
        s_rq.totals[3] = (double)__ldcg(s_rq.status);
        *s_rq.tiles_done = 0u;
        __threadfence_system();
        st_release_sys_u32(s_rq.done, 1u);
      }
    }
  }
}

// ---------------------------------------------------------------------------
// Two-kernel Monte Carlo step (xsec_step): k_ps draws the accepted points of a
// chunk (the same work-queue redraws as k_xsec, without the amplitude code, so
// it runs at high occupancy) into a workspace; k_me evaluates |M|^2, forms the
// weights and writes one partial per block.  Workspace layout per chunk of m
// points: momenta [NEXT*4][m] as FP64 (FP64 path) or as two FP32 arrays hi, lo
// (mixed path), then wps [m] (FP64 path: FP64 phase-space weight; mixed path: the
// whole weight factor w_PS s_ident / (2 s) in pb GeV^2 as an FP32 hi/lo pair), shat [m]
// (FP64) and tries [m] (int32).  The mixed k_me thus forms each weight in FP32 and sums
// a thread's weights as double-floats; the per-block and final sums are FP64.
// ---------------------------------------------------------------------------
// k_ps: each block owns a contiguous range of events and a circular queue of
// redraws.  Every round takes up to kThreads items -- first the carried-over
// redraws, then new events -- so rounds stay full until the range runs out; a
// failed draw is appended with its next attempt number.  Accepted points are
// written straight to their event's slot in the workspace.
// KIND fixes the generator at compile time and GRID whether the adaptive-grid
// code is compiled in (used where kin carries a grid); launch_ps picks the
// instantiation.
template <class P, bool MIXED, int KIND, bool GRID>
__global__ void __launch_bounds__(kThreads, 4) k_ps(KinDev kin, StepArgs a) {
  const uint64_t seed = a.seed, offset = a.offset;
  const int64_t m = a.m;
  void* __restrict__ ws = a.ws;
  int* status = a.status;
  constexpr int NEXT = P::NEXT;
  constexpr int QCAP = 4 * kThreads;  // power of two; holds at most 2 kThreads items at any time
  float* ph = reinterpret_cast<float*>(ws);
  float* pl = ph + (int64_t)NEXT * 4 * m;
  double* pd = reinterpret_cast<double*>(ws);
  double* wps_a = reinterpret_cast<double*>(MIXED ? (void*)(pl + (int64_t)NEXT * 4 * m) : (void*)(pd + (int64_t)NEXT * 4 * m));
  double* shat_a = wps_a + m;
  int32_t* tries_a = reinterpret_cast<int32_t*>(shat_a + m);
  __shared__ int64_t s_ev[QCAP];
  __shared__ int s_att[QCAP];
  __shared__ int s_head, s_tail;
  const int64_t per = (m + gridDim.x - 1) / gridDim.x;
  const int64_t b0 = (int64_t)blockIdx.x * per < m ? (int64_t)blockIdx.x * per : m;  // empty range past m
  const int64_t b1 = b0 + per < m ? b0 + per : m;
  if (threadIdx.x == 0) { s_head = 0; s_tail = 0; }
  __syncthreads();
  int64_t next_new = b0;
  while (true) {
    const int head = s_head, tail = s_tail;
    const int carried = tail - head;
    const int take_c = carried < kThreads ? carried : kThreads;
    const int64_t left = b1 - next_new;
    const int take_n = (int)((kThreads - take_c) < left ? (kThreads - take_c) : left);
    if (take_c + take_n == 0) break;
    int64_t ev = -1;
    int att = 0;
    if ((int)threadIdx.x < take_c) {
      ev = s_ev[(head + threadIdx.x) & (QCAP - 1)];
      att = s_att[(head + threadIdx.x) & (QCAP - 1)];
    } else if ((int)threadIdx.x < take_c + take_n) {
      ev = next_new + (threadIdx.x - take_c);
    }
    __syncthreads();  // every item read before the queue moves
    if (threadIdx.x == 0) s_head = head + take_c;
    next_new += take_n;
    if (ev >= 0) {
      double wps = 0.0, shat = 1.0;
      bool ok;
      uint8_t vbins[GRID ? kGridMaxDims : 1];  // grid steps: bin of every mapped uniform
      uint8_t* vb = GRID && kin.vg_bins ? vbins : nullptr;
      // Every lane stores its point's slots, accepted or not: a warp's stores then fill whole
      // 32-byte sectors, and the redraw of a rejected point (one of the next few rounds, through the
      // queue) overwrites its slots while their lines are still in L2.  Stores from lanes that skip
      // them leave partly written sectors, which L2 completes with reads from DRAM.
      if constexpr (MIXED) {
        df q[NEXT][4] = {};
        ok = draw_point_df<NEXT, KIND>(kin, seed, offset + (uint64_t)ev, att, q, wps, shat, vb);
#pragma unroll
        for (int k = 0; k < NEXT; ++k) {
#pragma unroll
          for (int mu = 0; mu < 4; ++mu) {
            ph[(int64_t)(k * 4 + mu) * m + ev] = q[k][mu].hi;
            pl[(int64_t)(k * 4 + mu) * m + ev] = q[k][mu].lo;
          }
        }
      } else {
        double q[NEXT][4] = {};
        ok = draw_point<NEXT, KIND>(kin, seed, offset + (uint64_t)ev, att, q, wps, shat, vb);
#pragma unroll
        for (int k = 0; k < NEXT; ++k) {
#pragma unroll
          for (int mu = 0; mu < 4; ++mu) pd[(int64_t)(k * 4 + mu) * m + ev] = q[k][mu];
        }
      }
      if (GRID && a.vg_idx && (ok || att + 1 >= kin.max_attempts))
        for (int d = 0; d < kin.vg_dims; ++d) a.vg_idx[(int64_t)d * m + ev] = ok ? vbins[d] : (uint8_t)0;
      if (ok) {
        if constexpr (MIXED) {
          // weight factor w_PS s_ident / (2 s) GeV^2->pb as a double-float pair in the weight slot
          // fixed-energy generators without a grid have a constant factor
          constexpr bool kConstW = !GRID && (KIND == ME_PS_RAMBO || KIND == ME_PS_TWO_BODY);
          const df wf = kConstW || kin.wfactor > 0.0 ? from_double(kin.wfactor)
                                          : (from_double(wps) * from_double(kin.s_ident * (0.5 * kGeV2pb))) /
                                                from_double(shat);
          float2* wf_a = reinterpret_cast<float2*>(wps_a);
          wf_a[ev] = make_float2(wf.hi, wf.lo);
        } else {
          wps_a[ev] = wps;
        }
        shat_a[ev] = shat;
        tries_a[ev] = att + 1;
      } else {
        // exhausted: the final zero weight; otherwise placeholders that the redraw overwrites
        const bool last = att + 1 >= kin.max_attempts;
        wps_a[ev] = 0.0;
        shat_a[ev] = 1.0;
        tries_a[ev] = last ? att + 1 : 0;
        if (last) {
          atomicOr(status, 1);
        } else {
          const int pos = atomicAdd(&s_tail, 1);
          s_ev[pos & (QCAP - 1)] = ev;
          s_att[pos & (QCAP - 1)] = att + 1;
        }
      }
    }
    __syncthreads();
  }
}

template <class P, bool MIXED>
__global__ void __launch_bounds__(kThreads) k_me(KinDev kin, StepArgs a, PrmT<P, MIXED> prm) {
  const int64_t m = a.m, out_stride = a.out_stride;
  const void* __restrict__ ws = a.ws;
  double* __restrict__ partials = a.partials;
  double* __restrict__ me2_out = a.me2_out;
  double* __restrict__ mom_out = a.mom_out;
  constexpr int NEXT = P::NEXT;
  const float* ph = reinterpret_cast<const float*>(ws);
  const float* pl = ph + (int64_t)NEXT * 4 * m;
  const double* pd = reinterpret_cast<const double*>(ws);
  const double* wps_a = reinterpret_cast<const double*>(MIXED ? (const void*)(pl + (int64_t)NEXT * 4 * m)
                                                              : (const void*)(pd + (int64_t)NEXT * 4 * m));
  const double* shat_a = wps_a + m;
  const int32_t* tries_a = reinterpret_cast<const int32_t*>(shat_a + m);
  double sw = 0.0, sw2 = 0.0;
  df swf = dfs(0.0f), sw2f = dfs(0.0f);  // mixed path: per-thread sums as double-floats
  int64_t ntries = 0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x) {
    double m2 = 0.0;
    if constexpr (MIXED) {
      // FP32 |M|^2 times the double-float weight factor written by k_ps; no FP64 per point
      const float wf = reinterpret_cast<const float2*>(wps_a)[i].x;
      const bool ok = wf > 0.0f;
      df q[NEXT][4];
#pragma unroll
      for (int k = 0; k < NEXT; ++k) {
#pragma unroll
        for (int mu = 0; mu < 4; ++mu)
          q[k][mu] = df{__ldg(ph + (int64_t)(k * 4 + mu) * m + i), __ldg(pl + (int64_t)(k * 4 + mu) * m + i)};
      }
      const float m2f = ok ? P::evalmx(q, prm) : 0.0f;
      if (mom_out) {
#pragma unroll
        for (int k = 0; k < NEXT; ++k) {
#pragma unroll
          for (int mu = 0; mu < 4; ++mu) mom_out[(int64_t)(k * 4 + mu) * out_stride + i] = to_double(q[k][mu]);
        }
      }
      const float w = m2f * wf;
      swf = swf + w;
      sw2f = sw2f + two_prod(w, w);
      ntries += tries_a[i];
      if (me2_out) me2_out[i] = (double)m2f;
      if (a.vg_w) a.vg_w[i] = (double)w;
    } else {
      const double wps = wps_a[i], shat = shat_a[i];
      const bool ok = wps > 0.0;
      double q[NEXT][4];
#pragma unroll
      for (int k = 0; k < NEXT; ++k) {
#pragma unroll
        for (int mu = 0; mu < 4; ++mu) q[k][mu] = __ldg(pd + (int64_t)(k * 4 + mu) * m + i);
      }
      if (ok) m2 = P::eval64(q, prm);
      if (mom_out) {
#pragma unroll
        for (int k = 0; k < NEXT; ++k) {
#pragma unroll
          for (int mu = 0; mu < 4; ++mu) mom_out[(int64_t)(k * 4 + mu) * out_stride + i] = q[k][mu];
        }
      }
      // constant weight factor for fixed-energy generators (one FP64 multiply per point)
      const double w = !ok ? 0.0 : (kin.wfactor > 0.0 ? m2 * kin.wfactor
                                                       : wps * m2 * kin.s_ident / (2.0 * shat) * kGeV2pb);
      sw += w;
      sw2 = fma(w, w, sw2);
      ntries += tries_a[i];
      if (me2_out) me2_out[i] = m2;
      if (a.vg_w) a.vg_w[i] = w;
    }
  }
  if constexpr (MIXED) {
    sw = to_double(swf);
    sw2 = to_double(sw2f);
  }
  block_reduce3(sw, sw2, (double)ntries, partials);
}

// ---------------------------------------------------------------------------
// k_me_mx: the mixed-path |M|^2 kernel with its inputs staged through shared
// memory.  The helicity program holds ~255 registers, so only 8 warps fit on an
// SM and the global loads of a point's 8*NEXT + 2 words stall them; here every
// thread copies the next tile's words of its own point with cp.async (4-byte
// copies: no alignment condition on the chunk size) while it evaluates the
// current one.  A thread reads only the column it copied itself, so no block
// barrier is needed between the stages.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void cp_async4(void* smem_dst, const void* gmem_src) {
#ifdef __CUDA_ARCH__
  const uint32_t d = (uint32_t)__cvta_generic_to_shared(smem_dst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(d), "l"(gmem_src));
#endif
}
__device__ __forceinline__ void cp_async_commit() {
#ifdef __CUDA_ARCH__
  asm volatile("cp.async.commit_group;\n" ::);
#endif
}
template <int N>
__device__ __forceinline__ void cp_async_wait() {
#ifdef __CUDA_ARCH__
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N));
#endif
}

template <class P>
constexpr int me_mx_words() {
  return 8 * P::NEXT + 2;  // momenta hi and lo, weight factor (hi), tries
}
template <class P>
constexpr size_t me_mx_smem() {
  return 2 * sizeof(float) * (size_t)me_mx_words<P>() * kThreads;
}

template <class P>
__global__ void __launch_bounds__(kThreads) k_me_mx(KinDev kin, StepArgs a, PrmT<P, true> prm) {
  const int64_t m = a.m, out_stride = a.out_stride;
  const void* __restrict__ ws = a.ws;
  double* __restrict__ partials = a.partials;
  double* __restrict__ me2_out = a.me2_out;
  double* __restrict__ mom_out = a.mom_out;
  constexpr int NEXT = P::NEXT, NW = me_mx_words<P>();
  extern __shared__ __align__(16) float s_stage[];  // [2][NW][kThreads]
  const float* ph = reinterpret_cast<const float*>(ws);
  const float* pl = ph + (int64_t)NEXT * 4 * m;
  const float2* wf_a = reinterpret_cast<const float2*>(pl + (int64_t)NEXT * 4 * m);
  const int32_t* tries_a = reinterpret_cast<const int32_t*>(reinterpret_cast<const double*>(wf_a) + 2 * m);
  const int64_t ntiles = (m + kThreads - 1) / kThreads;
  const int tid = threadIdx.x;
  auto stage = [&](int64_t tile, int b) {
    const int64_t i = tile * kThreads + tid;
    float* dst = s_stage + (size_t)b * NW * kThreads + tid;
    if (i < m) {
#pragma unroll
      for (int c = 0; c < 4 * NEXT; ++c) {
        cp_async4(dst + c * kThreads, ph + (int64_t)c * m + i);
        cp_async4(dst + (4 * NEXT + c) * kThreads, pl + (int64_t)c * m + i);
      }
      cp_async4(dst + 8 * NEXT * kThreads, &wf_a[i].x);
      cp_async4(dst + (8 * NEXT + 1) * kThreads, tries_a + i);
    }
    cp_async_commit();
  };
  df swf = dfs(0.0f), sw2f = dfs(0.0f);
  int64_t ntries = 0;
  int b = 0;
  if ((int64_t)blockIdx.x < ntiles) stage(blockIdx.x, 0);
  for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    if (tile + gridDim.x < ntiles) stage(tile + gridDim.x, b ^ 1);
    else cp_async_commit();  // an empty group keeps the wait count uniform
    cp_async_wait<1>();      // this thread's copies of the current tile have landed
    const int64_t i = tile * kThreads + tid;
    if (i < m) {
      const float* src = s_stage + (size_t)b * NW * kThreads + tid;
      const float wf = src[8 * NEXT * kThreads];
      const bool ok = wf > 0.0f;
      df q[NEXT][4];
#pragma unroll
      for (int k = 0; k < NEXT; ++k) {
#pragma unroll
        for (int mu = 0; mu < 4; ++mu)
          q[k][mu] = df{src[(k * 4 + mu) * kThreads], src[(4 * NEXT + k * 4 + mu) * kThreads]};
      }
      const float m2f = ok ? P::evalmx(q, prm) : 0.0f;
      if (mom_out) {
#pragma unroll
        for (int k = 0; k < NEXT; ++k) {
#pragma unroll
          for (int mu = 0; mu < 4; ++mu) mom_out[(int64_t)(k * 4 + mu) * out_stride + i] = to_double(q[k][mu]);
        }
      }
      const float w = m2f * wf;
      swf = swf + w;
      sw2f = sw2f + two_prod(w, w);
      ntries += __float_as_int(src[(8 * NEXT + 1) * kThreads]);
      if (me2_out) me2_out[i] = (double)m2f;
      if (a.vg_w) a.vg_w[i] = (double)w;
    }
    b ^= 1;
  }
  cp_async_wait<0>();
  block_reduce3(to_double(swf), to_double(sw2f), (double)ntries, partials);
}

// k_ps for the generator of kin (the kinds the host accepts for NEXT legs).  The
// mixed path has one kernel per generator, massless and massive RAMBO apart, with
// and without the grid code; the FP64 path one per generator with the grid code.
template <class P, bool MIXED, bool GRID>
cudaError_t launch_ps_kind(const KinDev* kin, const StepArgs* a, int grid, cudaStream_t s) {
  constexpr int N = P::NEXT;
  switch (kin->kind) {
    case ME_PS_TWO_BODY:
      if constexpr (N == 4) {
        k_ps<P, MIXED, ME_PS_TWO_BODY, GRID><<<grid, kThreads, 0, s>>>(*kin, *a);
        return cudaSuccess;
      }
      break;
    case ME_PS_RAMBO:
      if constexpr (MIXED) {
        if (kin->massive) {
          k_ps<P, MIXED, kKindRamboMassive, GRID><<<grid, kThreads, 0, s>>>(*kin, *a);
          return cudaSuccess;
        }
      }
      k_ps<P, MIXED, ME_PS_RAMBO, GRID><<<grid, kThreads, 0, s>>>(*kin, *a);
      return cudaSuccess;
    case ME_PS_RAMBO_BW:
      if constexpr (N >= 5) {
        k_ps<P, MIXED, ME_PS_RAMBO_BW, GRID><<<grid, kThreads, 0, s>>>(*kin, *a);
        return cudaSuccess;
      }
      break;
    case ME_PS_TTBAR:
      if constexpr (N == 8) {
        k_ps<P, MIXED, ME_PS_TTBAR, GRID><<<grid, kThreads, 0, s>>>(*kin, *a);
        return cudaSuccess;
      }
      break;
    case ME_PS_YPT:  // one instantiation with the grid code (it runs without a grid as well)
      k_ps<P, MIXED, ME_PS_YPT, true><<<grid, kThreads, 0, s>>>(*kin, *a);
      return cudaSuccess;
    default:
      break;
  }
  return cudaErrorInvalidValue;
}

template <class P>
cudaError_t launch_ps(int prec, const KinDev* kin, const StepArgs* a, int grid, cudaStream_t s) {
  if (prec == ME_FP64) return launch_ps_kind<P, false, true>(kin, a, grid, s);
  return kin->vg_bins ? launch_ps_kind<P, true, true>(kin, a, grid, s) : launch_ps_kind<P, true, false>(kin, a, grid, s);
}

template <class P>
cudaError_t launch_step(int prec, const KinDev* kin, const StepArgs* a, const double* params, cudaStream_t s,
                        int grid_ps, int grid_me, cudaEvent_t ev_mid) {
  typename P::Params prm;
  memcpy(&prm, params, sizeof(prm));
  cudaError_t e0 = launch_ps<P>(prec, kin, a, grid_ps, s);
  if (e0 != cudaSuccess) return e0;
  if (ev_mid) cudaEventRecord(ev_mid, s);
  if (prec == ME_FP64) {
    k_me<P, false><<<grid_me, kThreads, 0, s>>>(*kin, *a, prm);
  } else {
    cudaError_t e = cudaFuncSetAttribute(k_me_mx<P>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)me_mx_smem<P>());
    if (e != cudaSuccess) return e;
    k_me_mx<P><<<grid_me, kThreads, me_mx_smem<P>(), s>>>(*kin, *a, P::mixed_params(prm));
  }
  return cudaGetLastError();
}

template <class P>
cudaError_t launch_eval(int prec, const double* mom, int64_t n, double* out, const double* params, cudaStream_t s,
                        int grid) {
  typename P::Params prm;
  memcpy(&prm, params, sizeof(prm));
  if (prec == ME_FP64) k_eval<P, false><<<grid, kThreads, 0, s>>>(mom, n, out, prm);
  else k_eval<P, true><<<grid, kThreads, 0, s>>>(mom, n, out, P::mixed_params(prm));
  return cudaGetLastError();
}

// k_gen: phase-space points only, for a generator compiled as a fixed kind (the y/pT
// generator, which the fused kernels leave out): each thread redraws its own point until
// it passes, up to kin.max_attempts; outputs as k_xsec without |M|^2.
template <class P, bool MIXED, int KIND>
__global__ void __launch_bounds__(kThreads) k_gen(KinDev kin, uint64_t seed, uint64_t offset, int64_t n,
                                                  double* __restrict__ mom_out, double* __restrict__ wps_out,
                                                  double* __restrict__ shat_out, int32_t* __restrict__ tries_out,
                                                  int* status) {
  constexpr int NEXT = P::NEXT;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    double wps = 0.0, shat = 1.0;
    double q[NEXT][4];
    int att = 0;
    bool ok = false;
    for (; att < kin.max_attempts && !ok; ++att) ok = draw_point<NEXT, KIND>(kin, seed, offset + (uint64_t)i, att, q, wps, shat);
    if (!ok) {
      atomicOr(status, 1);
      wps = 0.0;
    }
    if (MIXED && ok) {  // the mixed path's momenta are the double-float split of the FP64 draw
#pragma unroll
      for (int k = 0; k < NEXT; ++k)
#pragma unroll
        for (int m = 0; m < 4; ++m) q[k][m] = to_double(from_double(q[k][m]));
    }
    if (mom_out)
#pragma unroll
      for (int k = 0; k < NEXT; ++k)
#pragma unroll
        for (int m = 0; m < 4; ++m) mom_out[(int64_t)(k * 4 + m) * n + i] = q[k][m];
    if (wps_out) wps_out[i] = wps;
    if (shat_out) shat_out[i] = shat;
    if (tries_out) tries_out[i] = ok ? att : kin.max_attempts;
  }
}

template <class P>
cudaError_t launch_serve(int prec, const ServeCtl* ctl, const double* params, cudaStream_t s, int grid) {
  typename P::Params prm;
  memcpy(&prm, params, sizeof(prm));
  if (prec == ME_FP64) k_serve<P, false><<<grid, kThreads, 0, s>>>(*ctl, prm);
  else k_serve<P, true><<<grid, kThreads, 0, s>>>(*ctl, P::mixed_params(prm));
  return cudaGetLastError();
}

template <class P>
int serve_blocks_per_sm(int prec) {
  int b = 0;
  const cudaError_t e = prec == ME_FP64
                            ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_serve<P, false>, kThreads, 0)
                            : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_serve<P, true>, kThreads, 0);
  return e == cudaSuccess ? b : 0;
}

template <class P>
cudaError_t launch_xsec(int prec, const KinDev* kin, uint64_t seed, uint64_t offset, int64_t n, const double* params,
                        double* partials, double* me2_out, double* mom_out, double* wps_out, double* shat_out,
                        int32_t* tries_out, int* status, int eval_me, cudaStream_t s, int grid) {
  typename P::Params prm;
  memcpy(&prm, params, sizeof(prm));
  if (kin->kind == ME_PS_YPT) {  // points only (the fused kernel does not compile this generator)
    if (eval_me) return cudaErrorNotSupported;
    if (prec == ME_FP64)
      k_gen<P, false, ME_PS_YPT><<<grid, kThreads, 0, s>>>(*kin, seed, offset, n, mom_out, wps_out, shat_out,
                                                           tries_out, status);
    else
      k_gen<P, true, ME_PS_YPT><<<grid, kThreads, 0, s>>>(*kin, seed, offset, n, mom_out, wps_out, shat_out,
                                                          tries_out, status);
    return cudaGetLastError();
  }
  if (prec == ME_FP64)
    k_xsec<P, false><<<grid, kThreads, 0, s>>>(*kin, seed, offset, n, prm, partials, me2_out, mom_out, wps_out,
                                               shat_out, tries_out, status, eval_me);
  else
    k_xsec<P, true><<<grid, kThreads, 0, s>>>(*kin, seed, offset, n, P::mixed_params(prm), partials, me2_out,
                                              mom_out, wps_out, shat_out, tries_out, status, eval_me);
  return cudaGetLastError();
}
}  // namespace me

#define ME_DEFINE_PROCESS(TAG, NEXT_, NPARAM)                                       \
  extern "C" void me_register_##TAG(me::ProcessDesc* d) {                           \
    static_assert(sizeof(me::TAG::Traits::Params) == NPARAM * sizeof(double), "parameter block"); \
    d->n_ext = NEXT_;                                                               \
    d->launch_eval = me::launch_eval<me::TAG::Traits>;                              \
    d->launch_xsec = me::launch_xsec<me::TAG::Traits>;                              \
    d->launch_step = me::launch_step<me::TAG::Traits>;                              \
    d->launch_serve = me::launch_serve<me::TAG::Traits>;                            \
    d->serve_blocks_per_sm = me::serve_blocks_per_sm<me::TAG::Traits>;              \
  }
