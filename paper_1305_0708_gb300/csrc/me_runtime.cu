// C-ABI runtime: handles, parameter resolution, workspace, launches and the
// deterministic Monte Carlo reduction.  Declarations and contracts: include/me.h.
#include <cmath>
#include <complex>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include <cuda.h>

#include "runtime_internal.h"

namespace me {
// generated registry (registry.cu)
int registry_size();
ProcessDesc* registry_entry(int i);
}  // namespace me

namespace me {
namespace rt {

thread_local std::string g_err;

me_status fail(me_status st, const std::string& msg) {
  g_err = msg;
  return st;
}

me_status cuda_fail(cudaError_t e, const char* where) {
  return fail(ME_ERR_CUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

}  // namespace rt
}  // namespace me

using namespace me::rt;

namespace {

const double kPi = 3.14159265358979323846;

me_params default_params() {
  me_params p;
  p.alpha = 1.0 / 128.0;
  p.sw2 = 0.2312;
  p.mZ = 91.1876;
  p.wZ = 2.4952;
  p.mW = 80.4;
  p.wW = 2.085;
  p.alpha_s = 0.118;
  p.mt = 175.0;
  p.wt = 1.50;
  p.mH = 125.0;
  p.wH = 0.0;
  p.complex_mass = 0;
  p.reserved_ = 0;
  return p;
}

// numerical value of a coupling / mass parameter name used by the generated code.  The couplings
// that carry a vector-boson mass (W W H, Z Z H, H H H, H H H H, t t H) are complex: the programs
// take them as name.re and name.im.  With the complex-mass option (Sect. 7.11) mu_V^2 = m_V^2 -
// i m_V Gamma_V enters those couplings and v = 2 mu_W / g, and the W is tied to the Z by
// mu_W^2 = c_W^2 mu_Z^2 (MW = c_W mZ, WW = c_W wZ in the propagators too).
bool coupling_value(const std::string& name, const me_params& p, double& v) {
  const double e = std::sqrt(4 * kPi * p.alpha);
  const double sw = std::sqrt(p.sw2), cw = std::sqrt(1 - p.sw2);
  const double g = e / sw, gz = e / (sw * cw), gs = std::sqrt(4 * kPi * p.alpha_s);
  const bool cms = p.complex_mass != 0;
  const double mW = cms ? cw * p.mZ : p.mW, wW = cms ? cw * p.wZ : p.wW;
  using C = std::complex<double>;
  const C muW = cms ? std::sqrt(C(mW * mW, -mW * wW)) : C(mW);
  const C muZ = cms ? std::sqrt(C(p.mZ * p.mZ, -p.mZ * p.wZ)) : C(p.mZ);
  const C vev = 2.0 * muW / g;
  struct F { const char* f; double q, t3; };
  static const F ferm[] = {{"u", 2.0 / 3, 0.5}, {"c", 2.0 / 3, 0.5}, {"t", 2.0 / 3, 0.5}, {"d", -1.0 / 3, -0.5},
                           {"s", -1.0 / 3, -0.5}, {"b", -1.0 / 3, -0.5}, {"e-", -1.0, -0.5}, {"mu-", -1.0, -0.5},
                           {"ve", 0.0, 0.5}, {"vm", 0.0, 0.5}};
  const size_t dot = name.find('.');
  if (dot != std::string::npos) {
    const std::string n = name.substr(0, dot), part = name.substr(dot + 1);
    if (part != "re" && part != "im") return false;
    C z;
    if (n == "GWWH") z = g * muW;
    else if (n == "GZZH") z = gz * muZ;
    else if (n == "GHHH") z = -3 * p.mH * p.mH / vev;
    else if (n == "GHHHH") z = -3 * p.mH * p.mH / (vev * vev);
    else if (n == "GHTT") z = -p.mt / vev;
    else return false;
    v = part == "re" ? z.real() : z.imag();
    return true;
  }
  const std::string& n = name;
  if (n == "ZERO" || n == "0") { v = 0; return true; }
  if (n == "GS") { v = gs; return true; }
  if (n == "GS2") { v = gs * gs; return true; }
  if (n == "GW") { v = g / std::sqrt(2.0); return true; }
  if (n == "GWWA") { v = e; return true; }
  if (n == "GWWZ") { v = g * cw; return true; }
  if (n == "GWWWW") { v = -g * g; return true; }
  if (n == "GWWAA") { v = g * g * sw * sw; return true; }
  if (n == "GWWAZ") { v = g * g * sw * cw; return true; }
  if (n == "GWWZZ") { v = g * g * cw * cw; return true; }
  if (n == "GWWHH") { v = g * g / 2; return true; }
  if (n == "GZZHH") { v = gz * gz / 2; return true; }
  if (n == "MT") { v = p.mt; return true; }
  if (n == "WT") { v = p.wt; return true; }
  if (n == "MZ") { v = p.mZ; return true; }
  if (n == "WZ") { v = p.wZ; return true; }
  if (n == "MW") { v = mW; return true; }
  if (n == "WW") { v = wW; return true; }
  if (n == "MH") { v = p.mH; return true; }
  if (n == "WH") { v = p.wH; return true; }
  for (const F& f : ferm) {
    const std::string s(f.f);
    if (n == "GA_" + s) { v = e * f.q; return true; }
    if (n == "GZL_" + s) { v = gz * (f.t3 - f.q * p.sw2); return true; }
    if (n == "GZR_" + s) { v = gz * (-f.q * p.sw2); return true; }
  }
  return false;
}

std::string normalise(const char* s) {
  std::string out;
  bool space = false;
  for (const char* c = s; *c; ++c) {
    if (*c == ' ' || *c == '\t' || *c == '\n') {
      space = !out.empty();
      continue;
    }
    if (space) out.push_back(' ');
    space = false;
    out.push_back(*c);
  }
  return out;
}

}  // namespace


namespace {

// fixed-order sum of the per-block partials (one block; deterministic)
__global__ void k_reduce_partials(const double* __restrict__ partials, int nblocks, double* __restrict__ acc) {
  __shared__ double sm[3][256];
  double s0 = 0, s1 = 0, s2 = 0;
  for (int b = threadIdx.x; b < nblocks; b += blockDim.x) {
    s0 += partials[3 * b + 0];
    s1 += partials[3 * b + 1];
    s2 += partials[3 * b + 2];
  }
  sm[0][threadIdx.x] = s0;
  sm[1][threadIdx.x] = s1;
  sm[2][threadIdx.x] = s2;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o) {
      sm[0][threadIdx.x] += sm[0][threadIdx.x + o];
      sm[1][threadIdx.x] += sm[1][threadIdx.x + o];
      sm[2][threadIdx.x] += sm[2][threadIdx.x + o];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    acc[0] = sm[0][0];
    acc[1] = sm[1][0];
    acc[2] = sm[2][0];
  }
}

}  // namespace

namespace me {
namespace rt {

// Asynchronous steps: the same fixed-order reduction, added to a caller's device accumulator
// (sum w, sum w^2, tries, steps with an exhausted point); the status word is consumed.
__global__ void k_reduce_partials_add(const double* __restrict__ partials, int nblocks, double* __restrict__ acc,
                                      int* __restrict__ status) {
  __shared__ double sm[3][256];
  double s0 = 0, s1 = 0, s2 = 0;
  for (int b = threadIdx.x; b < nblocks; b += blockDim.x) {
    s0 += partials[3 * b + 0];
    s1 += partials[3 * b + 1];
    s2 += partials[3 * b + 2];
  }
  sm[0][threadIdx.x] = s0;
  sm[1][threadIdx.x] = s1;
  sm[2][threadIdx.x] = s2;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o) {
      sm[0][threadIdx.x] += sm[0][threadIdx.x + o];
      sm[1][threadIdx.x] += sm[1][threadIdx.x + o];
      sm[2][threadIdx.x] += sm[2][threadIdx.x + o];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    acc[0] += sm[0][0];
    acc[1] += sm[1][0];
    acc[2] += sm[2][0];
    if (*status) {
      acc[3] += 1.0;
      *status = 0;
    }
  }
}

cudaError_t launch_reduce(const double* partials, int nblocks, double* acc, cudaStream_t s) {
  k_reduce_partials<<<1, 256, 0, s>>>(partials, nblocks, acc);
  return cudaGetLastError();
}

int grid_for(me_handle h, int64_t n) {
  const int64_t per = h->desc->events_per_block > 0 ? h->desc->events_per_block : me::kThreads;
  const int64_t need = (n + per - 1) / per;
  const int64_t cap = (int64_t)h->n_sm * 8;  // grid-stride beyond 8 blocks per SM
  return (int)std::max<int64_t>(1, std::min(need, cap));
}

me_status make_kin(me_handle h, const me_kin* kin, me::KinDev& k) {
  if (kin->kind < ME_PS_TWO_BODY || kin->kind > ME_PS_YPT) return fail(ME_ERR_ARG, "kin->kind: unknown generator");
  const int next = h->desc->n_ext;
  if (kin->kind == ME_PS_TWO_BODY && next != 4) return fail(ME_ERR_ARG, "two-body generator needs 4 legs");
  if (kin->kind == ME_PS_TTBAR && next != 8) return fail(ME_ERR_ARG, "ttbar generator needs 8 legs");
  if (kin->kind == ME_PS_RAMBO && (next < 4 || next > 10)) return fail(ME_ERR_ARG, "RAMBO supports 2 to 8 final legs");
  if (kin->kind == ME_PS_RAMBO_BW && (next < 5 || next > 10))
    return fail(ME_ERR_ARG, "resonance RAMBO supports 3 to 8 final legs");
  if (kin->kind == ME_PS_RAMBO_BW && !(kin->res_mass > 0 && kin->res_width > 0 && kin->res_mass < kin->sqrt_s))
    return fail(ME_ERR_ARG, "kin: resonance mass and width must be positive, mass below sqrt_s");
  if (kin->kind == ME_PS_YPT) {
    if (kin->n_obj < 2 || kin->n_obj > 8 || next > 10) return fail(ME_ERR_ARG, "kin: y/pT generator needs 2..8 objects");
    uint32_t seen = 0;
    for (int j = 0; j < kin->n_obj; ++j) {
      for (int q = 0; q < 2; ++q) {
        const int l = kin->obj_legs[j][q];
        if (q == 1 && l == -1) continue;
        if (l < 2 || l >= next || ((seen >> l) & 1u)) return fail(ME_ERR_ARG, "kin->obj_legs: not a partition of the final legs");
        seen |= 1u << l;
      }
      const bool res = kin->obj_legs[j][1] >= 0;
      if (res && !(kin->obj_res_mass[j] > 0 && kin->obj_res_width[j] > 0 && kin->obj_res_mass[j] < kin->sqrt_s))
        return fail(ME_ERR_ARG, "kin: a resonance object needs a positive mass below sqrt_s and a positive width");
      if (!res && !(kin->obj_mass[j] >= 0)) return fail(ME_ERR_ARG, "kin->obj_mass must be >= 0");
      if (!(kin->obj_y_max[j] > 0 && kin->obj_pt_max[j] > kin->obj_pt_min[j] && kin->obj_pt_min[j] >= 0))
        return fail(ME_ERR_ARG, "kin: object ranges need y_max > 0 and 0 <= pt_min < pt_max");
      if (!res && kin->obj_mass[j] == 0 && j < kin->n_obj - 1 && !(kin->obj_pt_min[j] > 0))
        return fail(ME_ERR_ARG, "kin: a massless object with a generated pT needs pt_min > 0 (Eq. 17 maps ln pT^2)");
    }
    if (seen != (((1u << next) - 1u) & ~3u)) return fail(ME_ERR_ARG, "kin->obj_legs: every final leg belongs to one object");
  }
  if (kin->cut_mode != 0 && kin->cut_mode != 1) return fail(ME_ERR_ARG, "kin->cut_mode must be 0 or 1");
  if (kin->cut_mode == 1 && kin->kind != ME_PS_YPT)
    return fail(ME_ERR_ARG, "kin->cut_mode 1 (the paper's selection) goes with the y/pT generator");
  if (kin->cut_mode == 1) {
    for (int i = 0; i < 16; ++i)
      if (kin->leg_class[i] < 0 || kin->leg_class[i] > 3 || (kin->leg_class[i] && (i < 2 || i >= next)))
        return fail(ME_ERR_ARG, "kin->leg_class: 0..3 on final legs only");
  }
  if (kin->n_cut_legs < 0 || kin->n_cut_legs > 8) return fail(ME_ERR_ARG, "kin->n_cut_legs out of range");
  for (int i = 0; i < kin->n_cut_legs; ++i)
    if (kin->cut_legs[i] < 2 || kin->cut_legs[i] >= next) return fail(ME_ERR_ARG, "kin->cut_legs: not a final-state leg");
  if (kin->kind != ME_PS_TTBAR && !(kin->sqrt_s > 0)) return fail(ME_ERR_ARG, "kin->sqrt_s must be positive");
  if (kin->kind == ME_PS_TTBAR && !(kin->sqrt_s_max > kin->sqrt_s_min && kin->sqrt_s_min > 0))
    return fail(ME_ERR_ARG, "kin->sqrt_s_min/max invalid");
  std::memset(&k, 0, sizeof(k));
  k.kind = kin->kind;
  k.max_attempts = kin->max_attempts > 0 ? kin->max_attempts : 10000;
  k.sqrt_s = kin->sqrt_s;
  k.sqrt_s_min = kin->sqrt_s_min;
  k.sqrt_s_max = kin->sqrt_s_max;
  double msum = 0;
  for (int i = 0; i < 16; ++i) {
    k.mass[i] = (kin->kind == ME_PS_RAMBO && i < next) ? kin->mass[i] : 0.0;
    if (i >= 2 && i < next) msum += k.mass[i];
  }
  if (kin->kind == ME_PS_RAMBO && !(msum < kin->sqrt_s)) return fail(ME_ERR_ARG, "kin: masses exceed sqrt_s");
  k.massive = msum > 0.0 ? 1 : 0;
  k.n_cut_legs = kin->n_cut_legs;
  k.cut_mask = 0;
  for (int i = 0; i < 8; ++i) k.cut_legs[i] = kin->cut_legs[i];
  for (int i = 0; i < kin->n_cut_legs; ++i) k.cut_mask |= 1u << kin->cut_legs[i];
  k.pt_min = kin->pt_min;
  k.eta_max = kin->eta_max;
  k.dr_min = kin->dr_min;
  k.s_ident = kin->s_ident > 0 ? kin->s_ident : 1.0;
  // RAMBO volume of the particles RAMBO draws (the resonance counts as one for RAMBO_BW)
  const int nf = kin->kind == ME_PS_RAMBO_BW ? next - 3 : next - 2;
  double fact = 1;
  for (int i = 2; i <= nf - 1; ++i) fact *= i;  // (n-1)!
  double fact2 = 1;
  for (int i = 2; i <= nf - 2; ++i) fact2 *= i;  // (n-2)!
  const double w = kin->sqrt_s;
  k.rambo_volume = std::pow(2 * kPi, 4 - 3 * nf) * std::pow(kPi / 2, nf - 1) * std::pow(w, 2 * nf - 4) / (fact * fact2);
  const double sh = std::sinh(kin->eta_max);
  k.sinh2_eta_max = kin->n_cut_legs > 0 ? sh * sh : 0.0;
  k.cos_dr = std::cos(kin->dr_min);
  k.cosh_dr = std::cosh(kin->dr_min);
  k.sinh_dr = std::sinh(kin->dr_min);
  const me_params& p = h->params;
  k.bw_mass[0] = p.mt;
  k.bw_width[0] = p.wt;
  // the W of the programs: tied to the Z under the complex-mass option
  const double cw = std::sqrt(1 - p.sw2);
  k.bw_mass[1] = p.complex_mass ? cw * p.mZ : p.mW;
  k.bw_width[1] = p.complex_mass ? cw * p.wZ : p.wW;
  if (kin->kind == ME_PS_RAMBO_BW) {
    k.bw_mass[0] = kin->res_mass;
    k.bw_width[0] = kin->res_width;
  }
  for (int r = 0; r < 2; ++r) {
    const double x = std::min(20.0, k.bw_mass[r] / k.bw_width[r]);
    k.bw_t0[r] = -std::atan(x);
    k.bw_t1[r] = std::atan(x);
  }
  if (kin->kind == ME_PS_TTBAR && !(p.wt > 0 && k.bw_width[1] > 0)) return fail(ME_ERR_ARG, "ttbar generator needs widths");
  k.sqrt_s_f[0] = (float)kin->sqrt_s;
  k.sqrt_s_f[1] = (float)(kin->sqrt_s - (double)k.sqrt_s_f[0]);
  k.shat_fixed = kin->sqrt_s * kin->sqrt_s;
  k.f_ptmin2 = (float)(k.pt_min * k.pt_min);
  k.f_sinh2 = (float)k.sinh2_eta_max;
  k.f_cdr = (float)k.cos_dr;
  k.f_chd = (float)k.cosh_dr;
  k.f_shd = (float)k.sinh_dr;
  k.f_dr2 = (float)(k.dr_min * k.dr_min);
  k.n_obj = kin->kind == ME_PS_YPT ? kin->n_obj : 0;
  k.cut_mode = kin->cut_mode;
  for (int j = 0; j < 8; ++j) {
    k.obj_legs[j][0] = kin->obj_legs[j][0];
    k.obj_legs[j][1] = j < k.n_obj ? kin->obj_legs[j][1] : -1;
    k.obj_mass[j] = kin->obj_mass[j];
    k.obj_res_mass[j] = kin->obj_res_mass[j];
    k.obj_res_width[j] = kin->obj_res_width[j];
    if (j < k.n_obj && kin->obj_legs[j][1] >= 0) {
      const double x = std::min(20.0, kin->obj_res_mass[j] / kin->obj_res_width[j]);
      k.obj_t0[j] = -std::atan(x);
      k.obj_t1[j] = std::atan(x);
    }
    k.obj_y_max[j] = kin->obj_y_max[j];
    k.obj_pt_min[j] = kin->obj_pt_min[j];
    k.obj_pt_max[j] = kin->obj_pt_max[j];
  }
  for (int i = 0; i < 16; ++i) k.leg_class[i] = kin->cut_mode == 1 ? kin->leg_class[i] : 0;
  k.jet_pt = kin->jet_pt;
  k.jet_eta = kin->jet_eta;
  k.jet_ptij = kin->jet_ptij;
  k.b_pt = kin->b_pt;
  k.b_eta = kin->b_eta;
  k.lep_pt = kin->lep_pt;
  k.lep_eta = kin->lep_eta;
  if (kin->cut_mode == 1) k.cut_mask = 0;  // the per-class selection replaces the uniform cuts
  const double gev2pb = 0.3893793721e9;
  if (kin->kind == ME_PS_TWO_BODY)
    k.wfactor = (1.0 / (8.0 * kPi)) * k.s_ident * gev2pb / (2.0 * k.shat_fixed);
  else if (kin->kind == ME_PS_RAMBO && !k.massive)
    k.wfactor = k.rambo_volume * k.s_ident * gev2pb / (2.0 * k.shat_fixed);
  else
    k.wfactor = 0.0;
  return ME_OK;
}

me_status ensure_workspace(me_handle h, int nblocks) {
  cudaError_t e;
  if (!h->d_acc) {
    if ((e = cudaMalloc(&h->d_acc, 4 * sizeof(double))) != cudaSuccess) return fail(ME_ERR_OOM, "workspace");
    if ((e = cudaMalloc(&h->d_status, sizeof(int))) != cudaSuccess) return fail(ME_ERR_OOM, "workspace");
    if ((e = cudaMemset(h->d_status, 0, sizeof(int))) != cudaSuccess) return cuda_fail(e, "cudaMemset");
    if ((e = cudaMallocHost(&h->h_acc, 4 * sizeof(double))) != cudaSuccess) return fail(ME_ERR_OOM, "pinned");
  }
  if (nblocks > h->partials_cap) {
    if (h->d_partials) cudaFree(h->d_partials);
    h->d_partials = nullptr;
    if ((e = cudaMalloc(&h->d_partials, (size_t)nblocks * 3 * sizeof(double))) != cudaSuccess)
      return fail(ME_ERR_OOM, "workspace partials");
    h->partials_cap = nblocks;
  }
  return ME_OK;
}

size_t ws_bytes(int n_ext, int64_t m) { return (size_t)m * (32 * (size_t)n_ext + 20); }

int grid_ps_for(me_handle h, int64_t m) {
  // phase space: 4 resident blocks per SM, each with a contiguous range of points
  return (int)std::max<int64_t>(1, std::min<int64_t>((m + me::kThreads - 1) / me::kThreads, (int64_t)h->n_sm * 4));
}

}  // namespace rt
}  // namespace me

namespace {

me_status ensure_points_ws(me_handle h, int64_t m) {
  const size_t need = ws_bytes(h->desc->n_ext, m);
  if (need <= h->ws_cap) return ME_OK;
  if (h->d_ws) cudaFree(h->d_ws);
  h->d_ws = nullptr;
  h->ws_cap = 0;
  if (cudaMalloc(&h->d_ws, need) != cudaSuccess) return fail(ME_ERR_OOM, "workspace for phase-space points");
  h->ws_cap = need;
  return ME_OK;
}

me_status check_handle(me_handle h) {
  if (!h || !h->desc) return fail(ME_ERR_ARG, "null handle");
  return ME_OK;
}

}  // namespace

// ---------------------------------------------------------------------------
// Scratch of xsec_step_noalloc: a file-scope device array, so that callers that
// must not allocate device memory can still run a Monte Carlo step.  Every GPU
// that loads this library holds it (about 100 KB) until the process exits.
// ---------------------------------------------------------------------------
namespace {

constexpr int kNoAllocMaxBlocks = 4096;  // one partial (3 doubles) per block of the fused kernel

struct NoAllocScratch {
  double partials[kNoAllocMaxBlocks * 3];
  double acc[4];
  int status;
};

__device__ __align__(256) NoAllocScratch g_noalloc_scratch;

constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mu;
struct NoAllocSlot {
  unsigned long long ctx_id;  // context the address belongs to (0: not looked up yet)
  NoAllocScratch* ptr;
};
NoAllocSlot g_noalloc_slot[kMaxDevices] = {};

// Unique id of the calling thread's current context (driver entry points taken through the runtime,
// so the library needs no link dependency on the driver library).  0 if it cannot be had.
unsigned long long current_context_id() {
  typedef CUresult (*GetCurrent)(CUcontext*);
  typedef CUresult (*GetId)(CUcontext, unsigned long long*);
  static GetCurrent get_current = nullptr;
  static GetId get_id = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      get_current = reinterpret_cast<GetCurrent>(f);
    f = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      get_id = reinterpret_cast<GetId>(f);
  });
  CUcontext ctx = nullptr;
  unsigned long long id = 0;
  if (!get_current || !get_id || get_current(&ctx) != CUDA_SUCCESS || !ctx || get_id(ctx, &id) != CUDA_SUCCESS)
    return 0;
  return id;
}

// Device address of the scratch array for the current device.  Host code may
// not use &g_noalloc_scratch (that is a host-side stand-in); the address is
// looked up with the device current, once per device and context: a context
// made anew (after cudaDeviceReset, say) reloads the module, so the address is
// looked up again.  Call after a CUDA call has made the device's context
// current (the runtime does that on first use).
me_status noalloc_scratch(int device, NoAllocScratch** out) {
  if (device < 0 || device >= kMaxDevices) return fail(ME_ERR_ARG, "xsec_step_noalloc: device index out of range");
  const unsigned long long ctx = current_context_id();
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  NoAllocSlot& slot = g_noalloc_slot[device];
  if (!slot.ptr || ctx == 0 || slot.ctx_id != ctx) {
    void* ptr = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress");
    slot.ptr = static_cast<NoAllocScratch*>(ptr);
    slot.ctx_id = ctx;
  }
  *out = slot.ptr;
  return ME_OK;
}

}  // namespace

namespace me {
namespace rt {

me_status run_step(me_handle h, KinDev& k, uint64_t seed, uint64_t counter_offset, int64_t n_accept, void* stream,
                   me_xsec_acc* acc, double* me2_out, double* momenta_out, GridHook* grid, double* acc_dev) {
  me_status st;
  if (n_accept == 0) return ME_OK;
  std::lock_guard<std::mutex> lock(h->mu);
  const int64_t m0 = std::min<int64_t>(n_accept, kChunk);
  const int64_t nchunks = (n_accept + kChunk - 1) / kChunk;
  const int grid_me = grid_for(h, m0);
  const int grid_ps = grid_ps_for(h, m0);
  if ((st = ensure_workspace(h, (int)(grid_me * nchunks))) != ME_OK) return st;
  if ((st = ensure_points_ws(h, m0)) != ME_OK) return st;
  if (grid && (st = grid->ensure(m0)) != ME_OK) return st;
  cudaStream_t s = (cudaStream_t)stream;
  cudaError_t e;
  for (int64_t c = 0; c < nchunks; ++c) {
    const int64_t first = c * kChunk;
    const int64_t m = std::min<int64_t>(kChunk, n_accept - first);
    if (h->timing && !acc_dev) cudaEventRecord(h->ev[0], s);
    me::StepArgs a{seed, counter_offset + (uint64_t)first, m, h->d_ws, h->d_status,
                   h->d_partials + 3 * (size_t)grid_me * c, grid_me, me2_out ? me2_out + first : nullptr,
                   momenta_out ? momenta_out + first : nullptr, n_accept,
                   grid ? grid->idx : nullptr, grid ? grid->w : nullptr};
    e = h->desc->launch_step(h->prec, &k, &a, h->cvals.data(), s, grid_ps, grid_me,
                             h->timing && !acc_dev ? h->ev[1] : nullptr);
    if (e != cudaSuccess) return cuda_fail(e, "xsec_step launch");
    if (grid && (e = launch_vg_hist(m, grid->dims, grid->bins, grid->idx, grid->w, grid->hist, s)) != cudaSuccess)
      return cuda_fail(e, "grid histogram");
    if (h->timing && !acc_dev) {
      cudaEventRecord(h->ev[2], s);
      if ((e = cudaEventSynchronize(h->ev[2])) != cudaSuccess) return cuda_fail(e, "xsec_step timing");
      float a = 0, b = 0;
      cudaEventElapsedTime(&a, h->ev[0], h->ev[1]);
      cudaEventElapsedTime(&b, h->ev[1], h->ev[2]);
      h->t_ps += a;
      h->t_me += b;
    }
  }
  if (acc_dev) {  // asynchronous: the sums stay on the device
    k_reduce_partials_add<<<1, 256, 0, s>>>(h->d_partials, (int)(grid_me * nchunks), acc_dev, h->d_status);
    if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(e, "xsec_step_async reduce");
    return ME_OK;
  }
  k_reduce_partials<<<1, 256, 0, s>>>(h->d_partials, (int)(grid_me * nchunks), h->d_acc);
  if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(e, "xsec_step reduce");
  if ((e = cudaMemcpyAsync(h->h_acc, h->d_acc, 3 * sizeof(double), cudaMemcpyDeviceToHost, s)) != cudaSuccess)
    return cuda_fail(e, "xsec_step copy");
  int status = 0;
  if ((e = cudaMemcpyAsync(&h->h_acc[3], h->d_status, sizeof(int), cudaMemcpyDeviceToHost, s)) != cudaSuccess)
    return cuda_fail(e, "xsec_step copy");
  if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return cuda_fail(e, "xsec_step sync");
  std::memcpy(&status, &h->h_acc[3], sizeof(int));
  if (status) {
    cudaMemsetAsync(h->d_status, 0, sizeof(int), s);
    cudaStreamSynchronize(s);
    return fail(ME_ERR_TIMEOUT, "xsec_step: a point exhausted its phase-space redraws");
  }
  acc->sum_w += h->h_acc[0];
  acc->sum_w2 += h->h_acc[1];
  acc->n_acc += n_accept;
  acc->n_try += (int64_t)llround(h->h_acc[2]);
  return ME_OK;
}

}  // namespace rt
}  // namespace me

extern "C" {

int32_t me_n_processes(void) { return me::registry_size(); }

const char* me_process_name(int32_t i) {
  if (i < 0 || i >= me::registry_size()) return nullptr;
  return me::registry_entry(i)->name;
}

me_status me_create(const char* process, const me_params* params, int32_t prec, me_handle* out) {
  if (!process || !out) return fail(ME_ERR_ARG, "me_create: null argument");
  if (prec != ME_FP64 && prec != ME_MIXED) return fail(ME_ERR_ARG, "me_create: unknown precision");
  if (params && (params->reserved_ != 0 || (params->complex_mass != 0 && params->complex_mass != 1)))
    return fail(ME_ERR_ARG, "me_create: complex_mass must be 0 or 1 and reserved_ 0");
  *out = nullptr;
  const std::string want = normalise(process);
  me::ProcessDesc* d = nullptr;
  for (int i = 0; i < me::registry_size(); ++i)
    if (normalise(me::registry_entry(i)->name) == want) d = me::registry_entry(i);
  if (!d) return fail(ME_ERR_PROCESS, "process not compiled into this library: " + want);
  me_handle h = new me_handle_s();
  h->desc = d;
  h->params = params ? *params : default_params();
  h->prec = prec;
  for (int k = 0; k < d->n_params; ++k) {
    double v;
    if (!coupling_value(d->param_names[k], h->params, v)) {
      delete h;
      return fail(ME_ERR_PROCESS, std::string("unknown coupling ") + d->param_names[k]);
    }
    h->cvals.push_back(v);
  }
  if (h->cvals.empty()) h->cvals.push_back(0.0);
  cudaError_t e = cudaGetDevice(&h->device);
  if (e != cudaSuccess) { delete h; return cuda_fail(e, "cudaGetDevice"); }
  e = cudaDeviceGetAttribute(&h->n_sm, cudaDevAttrMultiProcessorCount, h->device);
  if (e != cudaSuccess) { delete h; return cuda_fail(e, "cudaDeviceGetAttribute"); }
  *out = h;
  return ME_OK;
}

me_status me_eval(me_handle h, const double* momenta, int64_t n, double* out, void* stream) {
  me_status st = check_handle(h);
  if (st != ME_OK) return st;
  if (n < 0) return fail(ME_ERR_ARG, "me_eval: n < 0");
  if (n == 0) return ME_OK;
  if (!momenta || !out) return fail(ME_ERR_ARG, "me_eval: null buffer");
  cudaError_t e = h->desc->launch_eval(h->prec, momenta, n, out, h->cvals.data(), (cudaStream_t)stream, grid_for(h, n));
  if (e != cudaSuccess) return cuda_fail(e, "me_eval launch");
  return ME_OK;
}

me_status me_eval_host(me_handle h, const double* momenta, int64_t n, double* out, void* stream) {
  me_status st = check_handle(h);
  if (st != ME_OK) return st;
  if (n < 0) return fail(ME_ERR_ARG, "me_eval_host: n < 0");
  if (n == 0) return ME_OK;
  if (!momenta || !out) return fail(ME_ERR_ARG, "me_eval_host: null buffer");
  cudaStream_t s = (cudaStream_t)stream;
  cudaPointerAttributes am{}, ao{};
  cudaError_t e = cudaPointerGetAttributes(&am, momenta);
  if (e == cudaSuccess) e = cudaPointerGetAttributes(&ao, out);
  if (e != cudaSuccess) return cuda_fail(e, "me_eval_host: cudaPointerGetAttributes");
  if (am.type == cudaMemoryTypeDevice || ao.type == cudaMemoryTypeDevice)
    return fail(ME_ERR_ARG, "me_eval_host: device buffer (use me_eval)");
  std::lock_guard<std::mutex> lock(h->mu);
  const bool mapped = am.type == cudaMemoryTypeHost && am.devicePointer && ao.type == cudaMemoryTypeHost &&
                      ao.devicePointer;
  if (mapped) {
    // page-locked, mapped host memory: the kernel reads the momenta and writes |M|^2 over the
    // CPU-GPU link itself, no staging copy
    e = h->desc->launch_eval(h->prec, (const double*)am.devicePointer, n, (double*)ao.devicePointer,
                             h->cvals.data(), s, grid_for(h, n));
    if (e != cudaSuccess) return cuda_fail(e, "me_eval_host launch");
    e = cudaStreamSynchronize(s);
    return e == cudaSuccess ? ME_OK : cuda_fail(e, "me_eval_host");
  }
  // other host memory: chunks of kHostChunk points through two device buffers, alternating
  // between the caller's stream and a second one, so that one chunk's copies overlap the
  // other's evaluation
  const int rows = h->desc->n_ext * 4;
  const int64_t cm = std::min<int64_t>(n, kHostChunk);
  if (!h->s_aux) {
    for (int b = 0; b < 2; ++b) {
      if ((e = cudaMalloc(&h->d_stage[b], sizeof(double) * rows * kHostChunk)) != cudaSuccess ||
          (e = cudaMalloc(&h->d_stage_out[b], sizeof(double) * kHostChunk)) != cudaSuccess ||
          (e = cudaEventCreateWithFlags(&h->ev_aux[b], cudaEventDisableTiming)) != cudaSuccess)
        return cuda_fail(e, "me_eval_host: staging");
    }
    if ((e = cudaStreamCreateWithFlags(&h->s_aux, cudaStreamNonBlocking)) != cudaSuccess)
      return cuda_fail(e, "me_eval_host: stream");
  }
  // the second stream starts after the work already queued on the caller's stream
  if ((e = cudaEventRecord(h->ev_aux[0], s)) != cudaSuccess || (e = cudaStreamWaitEvent(h->s_aux, h->ev_aux[0], 0)))
    return cuda_fail(e, "me_eval_host: order");
  const int64_t nchunk = (n + cm - 1) / cm;
  for (int64_t c = 0; c < nchunk && e == cudaSuccess; ++c) {
    const int b = (int)(c & 1);
    cudaStream_t sc = b ? h->s_aux : s;
    const int64_t first = c * cm, m = std::min<int64_t>(cm, n - first);
    e = cudaMemcpy2DAsync(h->d_stage[b], sizeof(double) * m, momenta + first, sizeof(double) * n, sizeof(double) * m,
                          rows, cudaMemcpyHostToDevice, sc);
    if (e == cudaSuccess)
      e = h->desc->launch_eval(h->prec, h->d_stage[b], m, h->d_stage_out[b], h->cvals.data(), sc, grid_for(h, m));
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(out + first, h->d_stage_out[b], sizeof(double) * m, cudaMemcpyDeviceToHost, sc);
  }
  cudaError_t e2 = cudaStreamSynchronize(h->s_aux);
  cudaError_t e3 = cudaStreamSynchronize(s);
  if (e == cudaSuccess) e = e2 != cudaSuccess ? e2 : e3;
  return e == cudaSuccess ? ME_OK : cuda_fail(e, "me_eval_host");
}

me_status me_generate(me_handle h, uint64_t seed, uint64_t counter_offset, int64_t n, const me_kin* kin,
                      double* momenta, double* weight, double* shat, int32_t* tries, void* stream) {
  me_status st = check_handle(h);
  if (st != ME_OK) return st;
  if (!kin) return fail(ME_ERR_ARG, "me_generate: null kin");
  if (n < 0) return fail(ME_ERR_ARG, "me_generate: n < 0");
  me::KinDev k;
  if ((st = make_kin(h, kin, k)) != ME_OK) return st;
  if (n == 0) return ME_OK;
  std::lock_guard<std::mutex> lock(h->mu);
  if ((st = ensure_workspace(h, 1)) != ME_OK) return st;
  cudaError_t e = h->desc->launch_xsec(h->prec, &k, seed, counter_offset, n, h->cvals.data(), nullptr, nullptr,
                                       momenta, weight, shat, tries, h->d_status, 0, (cudaStream_t)stream,
                                       grid_for(h, n));
  if (e != cudaSuccess) return cuda_fail(e, "me_generate launch");
  return ME_OK;
}

me_status xsec_step(me_handle h, uint64_t seed, uint64_t counter_offset, int64_t n_accept, const me_kin* kin,
                    void* stream, me_xsec_acc* acc, double* me2_out, double* momenta_out) {
  me_status st = check_handle(h);
  if (st != ME_OK) return st;
  if (!kin || !acc) return fail(ME_ERR_ARG, "xsec_step: null argument");
  if (n_accept < 0) return fail(ME_ERR_ARG, "xsec_step: n_accept < 0");
  me::KinDev k;
  if ((st = make_kin(h, kin, k)) != ME_OK) return st;
  return me::rt::run_step(h, k, seed, counter_offset, n_accept, stream, acc, me2_out, momenta_out, nullptr, nullptr);
}

me_status xsec_step_async(me_handle h, uint64_t seed, uint64_t counter_offset, int64_t n_accept, const me_kin* kin,
                          void* stream, double* acc_dev) {
  me_status st = check_handle(h);
  if (st != ME_OK) return st;
  if (!kin || !acc_dev) return fail(ME_ERR_ARG, "xsec_step_async: null argument");
  if (n_accept < 0) return fail(ME_ERR_ARG, "xsec_step_async: n_accept < 0");
  cudaPointerAttributes at{};
  cudaError_t e = cudaPointerGetAttributes(&at, acc_dev);
  if (e != cudaSuccess) return cuda_fail(e, "xsec_step_async: cudaPointerGetAttributes");
  if (at.type != cudaMemoryTypeDevice && at.type != cudaMemoryTypeManaged)
    return fail(ME_ERR_ARG, "xsec_step_async: acc_dev is not device memory");
  me::KinDev k;
  if ((st = make_kin(h, kin, k)) != ME_OK) return st;
  return me::rt::run_step(h, k, seed, counter_offset, n_accept, stream, nullptr, nullptr, nullptr, nullptr, acc_dev);
}

me_status xsec_step_noalloc(me_handle h, uint64_t seed, uint64_t counter_offset, int64_t n_accept,
                            const me_kin* kin, void* stream, me_xsec_acc* acc, double* me2_out,
                            double* momenta_out) {
  me_status st = check_handle(h);
  if (st != ME_OK) return st;
  if (!kin || !acc) return fail(ME_ERR_ARG, "xsec_step_noalloc: null argument");
  if (n_accept < 0) return fail(ME_ERR_ARG, "xsec_step_noalloc: n_accept < 0");
  if (h->desc->events_per_block == 1)
    return fail(ME_ERR_ARG, std::string("xsec_step_noalloc: not available for ") + h->desc->name +
                                " (its |M|^2 kernel takes one event per block and has no fused step)");
  if (kin->kind == ME_PS_YPT)
    return fail(ME_ERR_ARG, "xsec_step_noalloc: the y/pT generator is not compiled into the fused step");
  me::KinDev k;
  if ((st = make_kin(h, kin, k)) != ME_OK) return st;
  if (n_accept == 0) return ME_OK;
  const int grid = grid_for(h, n_accept);
  if (grid > kNoAllocMaxBlocks)
    return fail(ME_ERR_ARG, "xsec_step_noalloc: launch needs " + std::to_string(grid) +
                                " blocks, beyond the static scratch maximum of " + std::to_string(kNoAllocMaxBlocks));
  int device = 0;
  cudaError_t e = cudaGetDevice(&device);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
  NoAllocScratch* scr = nullptr;
  if ((st = noalloc_scratch(device, &scr)) != ME_OK) return st;
  cudaStream_t s = (cudaStream_t)stream;
  // the status flag keeps the previous call's value: clear it; partials and totals are overwritten
  if ((e = cudaMemsetAsync(&scr->status, 0, sizeof(int), s)) != cudaSuccess) return cuda_fail(e, "cudaMemsetAsync");
  e = h->desc->launch_xsec(h->prec, &k, seed, counter_offset, n_accept, h->cvals.data(), scr->partials, me2_out,
                           momenta_out, nullptr, nullptr, nullptr, &scr->status, 1, s, grid);
  if (e != cudaSuccess) return cuda_fail(e, "xsec_step_noalloc launch");
  k_reduce_partials<<<1, 256, 0, s>>>(scr->partials, grid, scr->acc);
  if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(e, "xsec_step_noalloc reduce");
  double tot[3];
  int status = 0;
  if ((e = cudaMemcpyAsync(tot, scr->acc, sizeof(tot), cudaMemcpyDeviceToHost, s)) != cudaSuccess)
    return cuda_fail(e, "xsec_step_noalloc copy");
  if ((e = cudaMemcpyAsync(&status, &scr->status, sizeof(int), cudaMemcpyDeviceToHost, s)) != cudaSuccess)
    return cuda_fail(e, "xsec_step_noalloc copy");
  if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return cuda_fail(e, "xsec_step_noalloc sync");
  if (status) return fail(ME_ERR_TIMEOUT, "xsec_step_noalloc: a point exhausted its phase-space redraws");
  acc->sum_w += tot[0];
  acc->sum_w2 += tot[1];
  acc->n_acc += n_accept;
  acc->n_try += (int64_t)llround(tot[2]);
  return ME_OK;
}

me_status me_step_timing(me_handle h, int32_t enable, double* ms_ps, double* ms_me) {
  me_status st = check_handle(h);
  if (st != ME_OK) return st;
  std::lock_guard<std::mutex> lock(h->mu);
  if (ms_ps) *ms_ps = h->t_ps;
  if (ms_me) *ms_me = h->t_me;
  h->t_ps = h->t_me = 0.0;
  if (enable && !h->ev[0]) {
    for (int i = 0; i < 3; ++i) {
      cudaError_t e = cudaEventCreate(&h->ev[i]);
      if (e != cudaSuccess) return cuda_fail(e, "cudaEventCreate");
    }
  }
  h->timing = enable != 0;
  return ME_OK;
}

me_status me_xsec_estimate(const me_xsec_acc* acc, double* sigma, double* error) {
  if (!acc || !sigma || !error) return fail(ME_ERR_ARG, "me_xsec_estimate: null argument");
  if (acc->n_try <= 0) return fail(ME_ERR_STATE, "me_xsec_estimate: empty accumulator");
  const double n = (double)acc->n_try;
  const double mean = acc->sum_w / n;
  const double var = std::max(acc->sum_w2 / n - mean * mean, 0.0);
  *sigma = mean;
  *error = std::sqrt(var / std::max(n - 1.0, 1.0));
  return ME_OK;
}

me_status me_info(me_handle h, me_info_t* info) {
  me_status st = check_handle(h);
  if (st != ME_OK) return st;
  if (!info) return fail(ME_ERR_ARG, "me_info: null argument");
  std::memset(info, 0, sizeof(*info));
  const me::ProcessDesc* d = h->desc;
  info->n_ext = d->n_ext;
  info->n_hel = d->n_hel;
  info->n_hel_live = d->n_hel_live;
  info->n_colour = d->n_colour;
  info->n_diagrams = d->n_diagrams;
  for (int i = 0; i < d->n_ext && i < 16; ++i) info->pdg[i] = d->pdg[i];
  info->flops_amp = d->flops_amp;
  info->flops_fp64 = d->flops_fp64;
  info->flops_colour = d->flops_colour;
  return ME_OK;
}

void me_destroy(me_handle h) {
  if (!h) return;
  if (h->d_partials) cudaFree(h->d_partials);
  if (h->d_acc) cudaFree(h->d_acc);
  if (h->d_status) cudaFree(h->d_status);
  if (h->h_acc) cudaFreeHost(h->h_acc);
  if (h->d_ws) cudaFree(h->d_ws);
  for (int b = 0; b < 2; ++b) {
    if (h->d_stage[b]) cudaFree(h->d_stage[b]);
    if (h->d_stage_out[b]) cudaFree(h->d_stage_out[b]);
    if (h->ev_aux[b]) cudaEventDestroy(h->ev_aux[b]);
  }
  if (h->s_aux) cudaStreamDestroy(h->s_aux);
  for (int i = 0; i < 3; ++i)
    if (h->ev[i]) cudaEventDestroy(h->ev[i]);
  delete h;
}

const char* me_last_error(void) { return g_err.c_str(); }

}  // extern "C"
