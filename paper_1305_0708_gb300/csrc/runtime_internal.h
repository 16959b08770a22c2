// Runtime internals shared by the C-ABI entry points (me_runtime.cu) and the
// request server (me_server.cu): the handle, argument checks and launch sizing.
#pragma once
#include <mutex>
#include <string>
#include <vector>

#include "me.h"
#include "me_internal.h"

struct me_handle_s {
  me::ProcessDesc* desc = nullptr;
  me_params params;
  int prec = ME_FP64;
  std::vector<double> cvals;
  int device = 0;
  int n_sm = 0;
  // workspace (lazy)
  double* d_partials = nullptr;
  int partials_cap = 0;
  double* d_acc = nullptr;    // 3 doubles
  int* d_status = nullptr;
  double* h_acc = nullptr;    // pinned, 3 doubles + status
  void* d_ws = nullptr;       // phase-space points of one chunk (k_ps -> k_me)
  size_t ws_cap = 0;
  // me_eval_host staging for host memory the device cannot address (lazy): two
  // momentum buffers [n_ext*4][kHostChunk], two |M|^2 buffers, a second stream
  double* d_stage[2] = {nullptr, nullptr};
  double* d_stage_out[2] = {nullptr, nullptr};
  cudaStream_t s_aux = nullptr;
  cudaEvent_t ev_aux[2] = {nullptr, nullptr};
  // optional per-kernel timing of xsec_step (CUDA events on the call's stream)
  bool timing = false;
  cudaEvent_t ev[3] = {nullptr, nullptr, nullptr};
  double t_ps = 0.0, t_me = 0.0;
  std::mutex mu;
};

namespace me {
namespace rt {

constexpr int64_t kChunk = 1 << 20;      // points per k_ps / k_me pair of xsec_step
constexpr int64_t kHostChunk = 1 << 17;  // points per staged chunk of me_eval_host

me_status fail(me_status st, const std::string& msg);
me_status cuda_fail(cudaError_t e, const char* where);
// device form of the generator and cut parameters; checks them against the process
me_status make_kin(me_handle h, const me_kin* kin, KinDev& k);
// blocks of the |M|^2 kernel and of the phase-space kernel for a chunk of m points
int grid_for(me_handle h, int64_t n);
int grid_ps_for(me_handle h, int64_t m);
// bytes of the phase-space workspace between k_ps and k_me for m points
size_t ws_bytes(int n_ext, int64_t m);
// fixed-order sum of nblocks partials (3 doubles each) into acc[0..2]
cudaError_t launch_reduce(const double* partials, int nblocks, double* acc, cudaStream_t s);

// the adaptive-grid part of a Monte Carlo step: per-chunk bins and weights, the histogram
struct GridHook {
  int dims = 0, bins = 0;
  uint8_t* idx = nullptr;  // [dims][chunk]
  double* w = nullptr;     // [chunk]
  double* hist = nullptr;  // [dims][bins]
  virtual me_status ensure(int64_t chunk) = 0;  // buffers for chunks of up to `chunk` points
  virtual ~GridHook() = default;
};
// adds sum of w^2 per (dimension, bin) of m points to hist (me_grid.cu)
cudaError_t launch_vg_hist(int64_t m, int dims, int bins, const uint8_t* idx, const double* w, double* hist,
                           cudaStream_t s);
// one Monte Carlo step of n_accept points in chunks (xsec_step, and with a grid xsec_step_grid)
// acc_dev != nullptr: asynchronous step, sums added on the device to acc_dev (no host sync)
me_status run_step(me_handle h, KinDev& k, uint64_t seed, uint64_t counter_offset, int64_t n_accept, void* stream,
                   me_xsec_acc* acc, double* me2_out, double* momenta_out, GridHook* grid, double* acc_dev);

}  // namespace rt
}  // namespace me
