// Internal types shared by the runtime and the generated process units.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include "me.h"

namespace me {

// Phase-space description as the kernels use it: the user's me_kin plus the
// quantities derived once on the host.
struct KinDev {
  int32_t kind;
  int32_t max_attempts;
  double sqrt_s, sqrt_s_min, sqrt_s_max;
  double mass[16];
  int32_t n_cut_legs;
  int32_t cut_legs[8];
  double pt_min, eta_max, dr_min, s_ident;
  double rambo_volume;   // massless n-body volume with the (2 pi) factors of Eq. 5
  double sinh2_eta_max;  // sinh(eta_max)^2
  double cos_dr, cosh_dr, sinh_dr;
  double bw_mass[2], bw_width[2], bw_t0[2], bw_t1[2];  // top, W (ttbar); [0] the resonance of RAMBO_BW
  int32_t massive;       // any final-state mass (RAMBO)
  uint32_t cut_mask;     // bit k set: leg k is cut
  // FP32 / double-float copies formed on the host (no FP64 arithmetic per draw)
  float sqrt_s_f[2];     // sqrt_s as (hi, lo)
  double shat_fixed;     // sqrt_s^2
  float f_ptmin2, f_sinh2, f_cdr, f_chd, f_shd, f_dr2;
  double wfactor;        // constant weight factor W_PS s_ident pb / (2 s): fixed-energy generators, else 0
  // adaptive grid over the generator's uniforms (VEGAS); vg_bins == 0: none
  int32_t vg_dims, vg_bins;
  const double* vg_edges;  // device [vg_dims][vg_bins + 1]
  // ME_PS_YPT objects (me.h) with the Breit-Wigner range of each resonance object
  int32_t n_obj, cut_mode;
  int32_t obj_legs[8][2];
  int32_t leg_class[16];
  double obj_mass[8], obj_res_mass[8], obj_res_width[8], obj_t0[8], obj_t1[8];
  double obj_y_max[8], obj_pt_min[8], obj_pt_max[8];
  double jet_pt, jet_eta, jet_ptij, b_pt, b_eta, lep_pt, lep_eta;
};

constexpr int kGridMaxDims = 32, kGridMaxBins = 256;

constexpr int kThreads = 128;

// Entry points of one compiled process.
// Per-chunk arguments of the Monte Carlo step kernels, in one struct so that a
// captured CUDA graph of a step can be pointed at the next chunk by rewriting
// one kernel argument.
struct StepArgs {
  uint64_t seed, offset;  // Philox key and the counter of the chunk's first point
  int64_t m;              // points of the chunk
  void* ws;               // phase-space workspace of the chunk (k_ps -> |M|^2 kernel)
  int* status;            // set to 1 if a point exhausts its redraws
  double* partials;       // 3 doubles (sum w, sum w^2, tries) per block of the |M|^2 kernel
  int nslots;             // partial slots reserved for the chunk (>= blocks launched)
  double* me2_out;        // optional |M|^2 per point
  double* mom_out;        // optional momenta, SoA [n_ext][4] with stride out_stride
  int64_t out_stride;
  uint8_t* vg_idx;        // grid steps: [vg_dims][m] bin of every uniform of each accepted point
  double* vg_w;           // grid steps: [m] weight of each point
};

// Persistent serving (request server, persistent mode).  A lane's kernel claims
// items (tiles of requests) one at a time from a queue that the host fills while the
// kernel runs.  Items, the per-request records, the kinematics table and the control
// words live in page-locked host memory mapped into the device; the host writes an
// item and its request record before it publishes the item by raising `published`
// (release), and the kernel reads `published` with acquire semantics.
struct ServeItem {
  uint64_t seed, offset;  // request key; counter of the request's first point
  int64_t n;              // points of the request (stride of its momentum output)
  int64_t first;          // index of the tile's first point within the request
  int32_t count;          // points of the tile
  int32_t req;            // request record
  int32_t tile;           // partial slot of the tile within the request
  int32_t kin;            // index into the kinematics table
};

struct ServeReq {
  double* partials;        // device, 3 doubles per tile
  double* me2;             // device [n] or null
  double* mom;             // device [n_ext * 4][n] or null
  int* status;             // device: set to 1 if a point exhausts its redraws
  uint32_t* tiles_done;    // device counter, zero between requests
  int32_t tiles;           // tiles of the request
  int32_t pad_;
  double* totals;          // mapped host [4]: sum w, sum w^2, draws, redraw status
  uint32_t* done;          // mapped host: set to 1 (release) once totals hold the request's sums
};

struct ServeCtl {
  const ServeItem* items;      // mapped host
  const uint32_t* published;   // mapped host: items [0, published) are complete
  const uint32_t* closed;      // mapped host: nonzero once no further item will be published
  uint32_t* claim;             // device: next item index to hand out
  const ServeReq* reqs;        // mapped host
  const KinDev* kins;          // mapped host
  uint32_t* timed_out;         // mapped host: set to 1 by a block whose wait ran out
  uint32_t* claimed;           // mapped host: a recent claim index + 1 (how far the blocks have got)
  uint64_t spin_limit;         // waits of about 1 us a block may spend on one claim
  int32_t tile_points;         // points per item (a multiple of kThreads)
};

struct ProcessDesc {
  const char* name;
  int n_ext;
  int n_params;
  const char* const* param_names;
  int n_hel, n_hel_live, n_colour, n_diagrams;
  double flops_amp, flops_fp64, flops_colour;
  const int* pdg;
  int events_per_block;  // events one block of the |M|^2 kernel takes at a time (0: kThreads)
  cudaError_t (*launch_eval)(int prec, const double* mom, int64_t n, double* out, const double* params,
                             cudaStream_t s, int grid);
  cudaError_t (*launch_xsec)(int prec, const KinDev* kin, uint64_t seed, uint64_t offset, int64_t n,
                             const double* params, double* partials, double* me2_out, double* mom_out,
                             double* wps_out, double* shat_out, int32_t* tries_out, int* status,
                             int eval_me, cudaStream_t s, int grid);
  cudaError_t (*launch_step)(int prec, const KinDev* kin, const StepArgs* a, const double* params, cudaStream_t s,
                             int grid_ps, int grid_me, cudaEvent_t ev_mid);
  // persistent serving kernel (null for processes without one); blocks_per_sm: resident blocks of it
  cudaError_t (*launch_serve)(int prec, const ServeCtl* ctl, const double* params, cudaStream_t s, int grid);
  int (*serve_blocks_per_sm)(int prec);
};

}  // namespace me
