// Adaptive grids (VEGAS; G. P. Lepage, J. Comput. Phys. 27 (1978) 192) for the
// Monte Carlo step -- the role of the BASES / gBASES integrator the paper uses
// for its cross sections (Sect. 6).  Contract: include/me.h (me_grid_*,
// xsec_step_grid).
//
// A grid holds, per uniform variable the phase-space generator draws, N bin
// edges on [0, 1].  xsec_step_grid maps every uniform through the grid on the
// device (k_ps), multiplies the weight by the map's Jacobian, records each
// accepted point's bins and weight, and adds w^2 per (dimension, bin) to the
// grid's histogram (k_vg_hist).  me_grid_refine forms the new edges on the host:
// smoothing of the bin sums over neighbours, normalisation, the damping
// ((1 - r) / ln(1 / r))^alpha, and equal shares of the damped weights per new bin.
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "runtime_internal.h"

using me::rt::cuda_fail;
using me::rt::fail;

namespace {

// uniforms a draw of the generator uses (the grid's dimensions)
int grid_dims_for(int kind, int n_ext) {
  if (kind == ME_PS_TWO_BODY) return 2;
  if (kind == ME_PS_RAMBO) return 4 * (n_ext - 2);
  if (kind == ME_PS_RAMBO_BW) return 4 * (n_ext - 2) - 1;
  if (kind == ME_PS_YPT) return 3 * (n_ext - 2) - 3;
  return 15;
}

__global__ void __launch_bounds__(256) k_vg_hist(int64_t m, int dims, int bins, const uint8_t* __restrict__ idx,
                                                 const double* __restrict__ w, double* __restrict__ hist) {
  extern __shared__ double s_hist[];  // [dims][bins]
  for (int j = threadIdx.x; j < dims * bins; j += blockDim.x) s_hist[j] = 0.0;
  __syncthreads();
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x) {
    const double w2 = w[i] * w[i];
    if (w2 == 0.0) continue;
    for (int d = 0; d < dims; ++d) {
      int b = idx[(int64_t)d * m + i];
      b = b < bins ? b : bins - 1;
      atomicAdd(&s_hist[d * bins + b], w2);
    }
  }
  __syncthreads();
  for (int j = threadIdx.x; j < dims * bins; j += blockDim.x)
    if (s_hist[j] != 0.0) atomicAdd(&hist[j], s_hist[j]);
}

// new edges of one dimension from its bin sums d (host; see the file header)
void refine_dimension(const double* x, const double* d, int N, double alpha, double* out) {
  double any = 0.0;
  for (int i = 0; i < N; ++i) any += d[i];
  if (!(any > 0.0)) {
    std::memcpy(out, x, sizeof(double) * (N + 1));
    return;
  }
  std::vector<double> sm(N), m(N);
  if (N == 1) {
    sm[0] = d[0];
  } else {
    for (int i = 0; i < N; ++i) {
      if (i == 0) sm[i] = 0.5 * (d[0] + d[1]);
      else if (i == N - 1) sm[i] = 0.5 * (d[N - 2] + d[N - 1]);
      else sm[i] = (d[i - 1] + d[i] + d[i + 1]) / 3.0;
    }
  }
  double total_sm = 0.0;
  for (double v : sm) total_sm += v;
  double total = 0.0;
  for (int i = 0; i < N; ++i) {
    const double r = sm[i] / total_sm;
    m[i] = r >= 1.0 ? 1.0 : (r > 0.0 ? std::pow((1.0 - r) / std::log(1.0 / r), alpha) : 0.0);
    total += m[i];
  }
  out[0] = 0.0;
  out[N] = 1.0;
  double before = 0.0;  // damped weight of the old bins left of bin j
  int j = 0;
  for (int e = 1; e < N; ++e) {
    const double target = total * e / N;
    while (j < N - 1 && before + m[j] < target) before += m[j++];
    double f = m[j] > 0.0 ? (target - before) / m[j] : 0.0;
    f = f < 0.0 ? 0.0 : (f > 1.0 ? 1.0 : f);
    out[e] = x[j] + f * (x[j + 1] - x[j]);
  }
}

}  // namespace

struct me_grid_s : me::rt::GridHook {
  int device = 0, kind = 0, n_ext = 0;
  double* d_edges = nullptr;
  int64_t cap = 0;
  std::vector<double> edges;  // host copy [dims][bins + 1]

  me_status ensure(int64_t chunk) override {
    if (chunk <= cap) return ME_OK;
    if (idx) cudaFree(idx);
    if (w) cudaFree(w);
    idx = nullptr;
    w = nullptr;
    cap = 0;
    if (cudaMalloc(&idx, (size_t)dims * chunk) != cudaSuccess) return fail(ME_ERR_OOM, "grid: bin buffer");
    if (cudaMalloc(&w, sizeof(double) * chunk) != cudaSuccess) return fail(ME_ERR_OOM, "grid: weight buffer");
    cap = chunk;
    return ME_OK;
  }
  me_status upload() {
    const cudaError_t e = cudaMemcpy(d_edges, edges.data(), sizeof(double) * edges.size(), cudaMemcpyHostToDevice);
    return e == cudaSuccess ? ME_OK : cuda_fail(e, "grid: edges upload");
  }
  ~me_grid_s() override {
    if (idx) cudaFree(idx);
    if (w) cudaFree(w);
    if (hist) cudaFree(hist);
    if (d_edges) cudaFree(d_edges);
  }
};

namespace me {
namespace rt {

cudaError_t launch_vg_hist(int64_t m, int dims, int bins, const uint8_t* idx, const double* w, double* hist,
                           cudaStream_t s) {
  const size_t smem = sizeof(double) * (size_t)dims * bins;
  const int64_t blocks = std::min<int64_t>((m + 255) / 256, 1024);
  k_vg_hist<<<(int)std::max<int64_t>(blocks, 1), 256, smem, s>>>(m, dims, bins, idx, w, hist);
  return cudaGetLastError();
}

}  // namespace rt
}  // namespace me

extern "C" {

me_status me_grid_create(me_handle h, const me_kin* kin, int32_t n_bins, me_grid* out) {
  if (!h || !h->desc || !kin || !out) return fail(ME_ERR_ARG, "me_grid_create: null argument");
  *out = nullptr;
  me::KinDev k;
  me_status st = me::rt::make_kin(h, kin, k);
  if (st != ME_OK) return st;
  const int dims = grid_dims_for(k.kind, h->desc->n_ext);
  if (n_bins < 1 || n_bins > me::kGridMaxBins) return fail(ME_ERR_ARG, "me_grid_create: n_bins must be 1..256");
  if (dims > me::kGridMaxDims) return fail(ME_ERR_ARG, "me_grid_create: too many dimensions");
  if ((size_t)dims * n_bins * sizeof(double) > 48 * 1024)
    return fail(ME_ERR_ARG, "me_grid_create: dims * n_bins above 6144 (histogram in shared memory)");
  auto g = new me_grid_s();
  g->dims = dims;
  g->bins = n_bins;
  g->kind = k.kind;
  g->n_ext = h->desc->n_ext;
  cudaGetDevice(&g->device);
  g->edges.resize((size_t)dims * (n_bins + 1));
  for (int d = 0; d < dims; ++d)
    for (int i = 0; i <= n_bins; ++i) g->edges[(size_t)d * (n_bins + 1) + i] = (double)i / n_bins;
  cudaError_t e = cudaMalloc(&g->d_edges, sizeof(double) * g->edges.size());
  if (e == cudaSuccess) e = cudaMalloc(&g->hist, sizeof(double) * dims * n_bins);
  if (e == cudaSuccess) e = cudaMemset(g->hist, 0, sizeof(double) * dims * n_bins);
  if (e != cudaSuccess) {
    delete g;
    return fail(ME_ERR_OOM, "me_grid_create: device buffers");
  }
  if ((st = g->upload()) != ME_OK) {
    delete g;
    return st;
  }
  *out = g;
  return ME_OK;
}

me_status me_grid_info(me_grid g, int32_t* n_dims, int32_t* n_bins) {
  if (!g) return fail(ME_ERR_ARG, "me_grid_info: null grid");
  if (n_dims) *n_dims = g->dims;
  if (n_bins) *n_bins = g->bins;
  return ME_OK;
}

me_status me_grid_get_edges(me_grid g, double* edges) {
  if (!g || !edges) return fail(ME_ERR_ARG, "me_grid_get_edges: null argument");
  std::memcpy(edges, g->edges.data(), sizeof(double) * g->edges.size());
  return ME_OK;
}

me_status me_grid_set_edges(me_grid g, const double* edges) {
  if (!g || !edges) return fail(ME_ERR_ARG, "me_grid_set_edges: null argument");
  const int N = g->bins;
  for (int d = 0; d < g->dims; ++d) {
    const double* e = edges + (size_t)d * (N + 1);
    if (e[0] != 0.0 || e[N] != 1.0) return fail(ME_ERR_ARG, "me_grid_set_edges: edges must run from 0 to 1");
    for (int i = 0; i < N; ++i)
      if (!(e[i + 1] > e[i])) return fail(ME_ERR_ARG, "me_grid_set_edges: edges must increase");
  }
  std::memcpy(g->edges.data(), edges, sizeof(double) * g->edges.size());
  return g->upload();
}

me_status me_grid_get_hist(me_grid g, double* hist) {
  if (!g || !hist) return fail(ME_ERR_ARG, "me_grid_get_hist: null argument");
  const cudaError_t e = cudaMemcpy(hist, g->hist, sizeof(double) * g->dims * g->bins, cudaMemcpyDeviceToHost);
  return e == cudaSuccess ? ME_OK : cuda_fail(e, "me_grid_get_hist");
}

me_status me_grid_clear_hist(me_grid g) {
  if (!g) return fail(ME_ERR_ARG, "me_grid_clear_hist: null grid");
  const cudaError_t e = cudaMemset(g->hist, 0, sizeof(double) * g->dims * g->bins);
  return e == cudaSuccess ? ME_OK : cuda_fail(e, "me_grid_clear_hist");
}

me_status me_grid_refine(me_grid g, double alpha) {
  if (!g) return fail(ME_ERR_ARG, "me_grid_refine: null grid");
  if (!(alpha > 0.0)) return fail(ME_ERR_ARG, "me_grid_refine: alpha must be positive");
  std::vector<double> d((size_t)g->dims * g->bins);
  me_status st = me_grid_get_hist(g, d.data());
  if (st != ME_OK) return st;
  std::vector<double> out(g->edges.size());
  const int N = g->bins;
  for (int k = 0; k < g->dims; ++k)
    refine_dimension(g->edges.data() + (size_t)k * (N + 1), d.data() + (size_t)k * N, N, alpha,
                     out.data() + (size_t)k * (N + 1));
  g->edges = out;
  if ((st = g->upload()) != ME_OK) return st;
  return me_grid_clear_hist(g);
}

me_status xsec_step_grid(me_handle h, me_grid g, uint64_t seed, uint64_t counter_offset, int64_t n_accept,
                         const me_kin* kin, void* stream, me_xsec_acc* acc, double* me2_out, double* momenta_out) {
  if (!h || !h->desc || !g || !kin || !acc) return fail(ME_ERR_ARG, "xsec_step_grid: null argument");
  if (n_accept < 0) return fail(ME_ERR_ARG, "xsec_step_grid: n_accept < 0");
  me::KinDev k;
  me_status st = me::rt::make_kin(h, kin, k);
  if (st != ME_OK) return st;
  if (k.kind != g->kind || h->desc->n_ext != g->n_ext)
    return fail(ME_ERR_ARG, "xsec_step_grid: grid made for another generator or process");
  k.vg_dims = g->dims;
  k.vg_bins = g->bins;
  k.vg_edges = g->d_edges;
  k.wfactor = 0.0;  // the Jacobian makes every weight differ
  return me::rt::run_step(h, k, seed, counter_offset, n_accept, stream, acc, me2_out, momenta_out, g, nullptr);
}

me_status me_vegas_refine_edges(const double* edges, const double* hist, int32_t n_dims, int32_t n_bins, double alpha,
                                double* out) {
  if (!edges || !hist || !out) return fail(ME_ERR_ARG, "me_vegas_refine_edges: null argument");
  if (n_dims < 1 || n_bins < 1 || !(alpha > 0.0)) return fail(ME_ERR_ARG, "me_vegas_refine_edges: bad size or alpha");
  for (int k = 0; k < n_dims; ++k)
    refine_dimension(edges + (size_t)k * (n_bins + 1), hist + (size_t)k * n_bins, n_bins, alpha,
                     out + (size_t)k * (n_bins + 1));
  return ME_OK;
}

void me_grid_destroy(me_grid g) { delete g; }

}  // extern "C"
