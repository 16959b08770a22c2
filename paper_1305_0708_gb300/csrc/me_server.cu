// Request server: continuous batching of Monte Carlo steps on one GPU.
// Contract and semantics: include/me_server.h.
//
// Design.  One scheduler thread owns all device work.  Every admitted request
// owns its result buffers (partials of every chunk, the |M|^2 and momentum
// arrays if kept, a 4-double accumulator and a status word), taken from a
// dedicated stream-ordered memory pool; every slot owns a CUDA stream and the
// phase-space workspace of one chunk.  The loop (1) admits waiting requests in
// arrival order while they fit in the budget, (2) gives every free slot the
// next chunk of the admitted requests in round-robin order (a request may run
// on several slots at once; chunk c writes only its own partials and array
// range), (3) when the last chunk of a request is seen complete, sums its
// partials in a fixed order and copies the sums to pinned staging on that
// slot's stream, and (4) marks the request done when that copy completes.
// Chunk sizes per process come from the autotuner (me_server_warm, or the
// first request of a process).
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <thread>
#include <utility>
#include <vector>

#include "me_server.h"
#include "runtime_internal.h"

using me::rt::cuda_fail;
using me::rt::fail;

namespace {

constexpr uint64_t kDefaultCap = 40ull << 30;
constexpr int64_t kChunkMin = 1 << 12, kChunkMax = 1 << 20;
constexpr size_t kWsMaxBytes = 512ull << 20;  // largest slot workspace the autotuner may ask for

double now_ms(std::chrono::steady_clock::time_point t0) {
  return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
}

struct Proc {
  me_handle h = nullptr;
  int64_t chunk = 0;  // 0: not tuned yet
  // persistent mode: the process has a persistent kernel; its autotuned tile (points per
  // queue item) and resident blocks per SM
  bool serve = false;
  int64_t tile = 0;
  int bps = 0;
};

// lane capacities (page-locked host memory of every lane)
constexpr uint32_t kLaneItems = 1u << 18;
constexpr int kLaneReqs = 1024;
constexpr int kLaneKins = 32;

enum class RState { Waiting, Active, Final, Done };

struct Request {
  int64_t id = 0;
  me_request r{};
  std::string process;
  Proc* proc = nullptr;
  me::KinDev kin{};
  RState state = RState::Waiting;
  int64_t chunk = 0, nchunks = 0, next_chunk = 0, chunks_done = 0;
  int grid_me = 0, grid_ps = 0;
  uint64_t need = 0;   // device bytes of its buffers
  size_t ws_need = 0;  // slot workspace bytes of one of its chunks
  uint64_t bytes = 0;  // bytes held against the budget (need, once admitted)
  bool failed = false;
  double* d_partials = nullptr;
  double* d_acc = nullptr;  // 3 sums + 1 spare
  int* d_status = nullptr;
  double* d_me2 = nullptr;
  double* d_mom = nullptr;
  int stage = -1;  // pinned staging slot index
  cudaEvent_t ready = nullptr;
  me_request_result res{};
  // persistent mode
  struct Lane* lane = nullptr;
  int lane_slot = -1, lane_kin = -1;
  int64_t tiles = 0, tiles_published = 0;
};

// A persistent lane: one slot's persistent kernel for one process at a time, fed through a
// queue in page-locked host memory mapped into the device (layout: me_internal.h).
struct Lane {
  me::ServeItem* items = nullptr;  // [kLaneItems]
  me::ServeReq* reqs = nullptr;    // [kLaneReqs]
  me::KinDev* kins = nullptr;      // [kLaneKins]
  uint32_t* ctl = nullptr;         // [0] published, [1] closed, [2] timed_out, [3] claim hint
  double* totals = nullptr;        // [kLaneReqs][4]
  uint32_t* done = nullptr;        // [kLaneReqs]
  me::ServeCtl dctl{};             // device view (pointers as the kernel sees them)
  uint32_t* d_claim = nullptr;
  uint32_t* d_tiles_done = nullptr;
  const Proc* proc = nullptr;
  int grid = 0;
  bool running = false, closed = false;
  uint32_t n_items = 0;
  int n_kins = 0;
  size_t rr = 0;
  std::vector<int> free_req;
  std::vector<Request*> in;        // requests with a record in this lane
  cudaEvent_t ev_end = nullptr;
  std::map<std::pair<const Proc*, int>, cudaGraphExec_t> graphs;  // by (process, grid)
};

// The step of one process and generator kind on one slot as an instantiated CUDA
// graph (the phase-space kernel compiled for that generator and the |M|^2 kernel,
// captured once); a chunk rewrites the two kernels' (KinDev, StepArgs) arguments
// in the executable graph and launches it.
struct SlotGraph {
  bool ok = false;
  cudaGraph_t g = nullptr;
  cudaGraphExec_t exec = nullptr;
  cudaGraphNode_t node_ps = nullptr, node_me = nullptr;
  cudaKernelNodeParams p_ps{}, p_me{};  // as captured; p_me.kernelParams[2] is the parameter block
};

struct Slot {
  cudaStream_t stream = nullptr;
  cudaEvent_t ev = nullptr;
  void* ws = nullptr;
  size_t ws_cap = 0;
  Request* req = nullptr;  // request whose chunk (or final reduction) is in flight
  bool final = false;
  std::map<std::pair<const Proc*, int>, SlotGraph> graphs;  // by (process, generator kind)
  std::unique_ptr<Lane> lane;  // persistent mode
};

// host stores and loads that order the mapped queue against the device's acquire/release
inline void store_release(uint32_t* p, uint32_t v) { __atomic_store_n(p, v, __ATOMIC_RELEASE); }
inline uint32_t load_acquire(const uint32_t* p) { return __atomic_load_n(p, __ATOMIC_ACQUIRE); }

template <class T>
cudaError_t mapped_alloc(T** host, size_t count) {
  cudaError_t e = cudaHostAlloc((void**)host, sizeof(T) * count, cudaHostAllocMapped | cudaHostAllocPortable);
  if (e == cudaSuccess) std::memset((void*)*host, 0, sizeof(T) * count);
  return e;
}
template <class T>
T* dev_view(T* host) {
  void* d = nullptr;
  return cudaHostGetDevicePointer(&d, (void*)host, 0) == cudaSuccess ? static_cast<T*>(d) : nullptr;
}

cudaError_t lane_init(Lane& L, uint64_t spin_limit) {
  cudaError_t e = mapped_alloc(&L.items, kLaneItems);
  if (e == cudaSuccess) e = mapped_alloc(&L.reqs, kLaneReqs);
  if (e == cudaSuccess) e = mapped_alloc(&L.kins, kLaneKins);
  if (e == cudaSuccess) e = mapped_alloc(&L.ctl, 4);
  if (e == cudaSuccess) e = mapped_alloc(&L.totals, 4 * (size_t)kLaneReqs);
  if (e == cudaSuccess) e = mapped_alloc(&L.done, kLaneReqs);
  if (e == cudaSuccess) e = cudaMalloc(&L.d_claim, sizeof(uint32_t));
  if (e == cudaSuccess) e = cudaMalloc(&L.d_tiles_done, sizeof(uint32_t) * kLaneReqs);
  if (e == cudaSuccess) e = cudaMemset(L.d_tiles_done, 0, sizeof(uint32_t) * kLaneReqs);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&L.ev_end, cudaEventDisableTiming);
  if (e != cudaSuccess) return e;
  L.dctl.items = dev_view(L.items);
  L.dctl.reqs = dev_view(L.reqs);
  L.dctl.kins = dev_view(L.kins);
  uint32_t* c = dev_view(L.ctl);
  L.dctl.published = c;
  L.dctl.closed = c + 1;
  L.dctl.timed_out = c + 2;
  L.dctl.claimed = c + 3;
  L.dctl.claim = L.d_claim;
  L.dctl.spin_limit = spin_limit;
  if (!L.dctl.items || !L.dctl.reqs || !L.dctl.kins || !c) return cudaErrorInvalidValue;
  for (int i = kLaneReqs - 1; i >= 0; --i) L.free_req.push_back(i);
  return cudaSuccess;
}

void lane_free(Lane& L) {
  for (auto& kv : L.graphs)
    if (kv.second) cudaGraphExecDestroy(kv.second);
  L.graphs.clear();
  if (L.items) cudaFreeHost(L.items);
  if (L.reqs) cudaFreeHost(L.reqs);
  if (L.kins) cudaFreeHost(L.kins);
  if (L.ctl) cudaFreeHost(L.ctl);
  if (L.totals) cudaFreeHost(L.totals);
  if (L.done) cudaFreeHost(L.done);
  if (L.d_claim) cudaFree(L.d_claim);
  if (L.d_tiles_done) cudaFree(L.d_tiles_done);
  if (L.ev_end) cudaEventDestroy(L.ev_end);
  L = Lane{};
}

// queue reset for a new kernel (no kernel of the lane running)
void lane_reset(Lane& L) {
  L.ctl[0] = L.ctl[1] = L.ctl[2] = L.ctl[3] = 0u;
  L.n_items = 0;
  L.n_kins = 0;
  L.closed = false;
  L.rr = 0;
}

// record of request slot r of the lane, pointing the kernel at the request's buffers
void lane_record(Lane& L, int r, double* partials, double* me2, double* mom, int* status, int64_t tiles) {
  me::ServeReq& q = L.reqs[r];
  q.partials = partials;
  q.me2 = me2;
  q.mom = mom;
  q.status = status;
  q.tiles_done = L.d_tiles_done + r;
  q.tiles = (int32_t)tiles;
  q.totals = dev_view(L.totals) + 4 * r;
  q.done = dev_view(L.done) + r;
  L.done[r] = 0u;
}

// kinematics table index of kin in the lane (added if new; -1 if the table is full)
int lane_kin(Lane& L, const me::KinDev& k) {
  for (int i = 0; i < L.n_kins; ++i)
    if (std::memcmp(&L.kins[i], &k, sizeof(k)) == 0) return i;
  if (L.n_kins >= kLaneKins) return -1;
  L.kins[L.n_kins] = k;
  return L.n_kins++;
}

// item of tile t (points [t * tile, ...)) of a request
me::ServeItem lane_item(uint64_t seed, uint64_t offset, int64_t n, int64_t tile, int64_t t, int req, int kin) {
  me::ServeItem it{};
  it.seed = seed;
  it.offset = offset;
  it.n = n;
  it.first = t * tile;
  it.count = (int32_t)std::min<int64_t>(tile, n - it.first);
  it.req = req;
  it.tile = (int32_t)t;
  it.kin = kin;
  return it;
}

// The lane's kernel for process p with `grid` blocks as a captured graph: the claim counter
// reset and the persistent kernel (first use per process and grid only).
cudaGraphExec_t lane_graph(Lane& L, const Proc* p, int grid, int64_t tile, cudaStream_t st) {
  const auto key = std::make_pair(p, grid);
  auto it = L.graphs.find(key);
  if (it != L.graphs.end()) return it->second;
  me::ServeCtl c = L.dctl;
  c.tile_points = (int32_t)tile;
  cudaGraph_t g = nullptr;
  cudaGraphExec_t ex = nullptr;
  if (cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal) == cudaSuccess) {
    cudaError_t e1 = cudaMemsetAsync(L.d_claim, 0, sizeof(uint32_t), st);
    cudaError_t e2 = e1 == cudaSuccess ? p->h->desc->launch_serve(p->h->prec, &c, p->h->cvals.data(), st, grid) : e1;
    cudaError_t e3 = cudaStreamEndCapture(st, &g);
    if (e2 != cudaSuccess || e3 != cudaSuccess || !g || cudaGraphInstantiate(&ex, g, 0) != cudaSuccess) ex = nullptr;
    if (g) cudaGraphDestroy(g);
  }
  cudaGetLastError();
  L.graphs[key] = ex;
  return ex;
}

// Start the lane's kernel: the captured graph, or the two operations directly if no graph
// could be made; ev_end marks its end.
cudaError_t lane_launch(Lane& L, const Proc* p, int grid, int64_t tile, cudaStream_t st, bool* as_graph) {
  cudaGraphExec_t ex = lane_graph(L, p, grid, tile, st);
  cudaError_t e;
  *as_graph = ex != nullptr;
  if (ex) {
    e = cudaGraphLaunch(ex, st);
  } else {
    me::ServeCtl c = L.dctl;
    c.tile_points = (int32_t)tile;
    e = cudaMemsetAsync(L.d_claim, 0, sizeof(uint32_t), st);
    if (e == cudaSuccess) e = p->h->desc->launch_serve(p->h->prec, &c, p->h->cvals.data(), st, grid);
  }
  if (e == cudaSuccess) e = cudaEventRecord(L.ev_end, st);
  return e;
}

}  // namespace

struct me_server_s {
  me_server_config cfg{};
  int device = 0;
  std::chrono::steady_clock::time_point t0;
  cudaMemPool_t pool = nullptr;
  cudaStream_t admin = nullptr;  // allocations, frees and result copies
  std::vector<Slot> slots;
  double* h_stage = nullptr;     // pinned: 8 doubles per admitted request
  std::vector<int> free_stage;

  std::mutex mu;                 // guards everything below and the request states
  std::condition_variable cv_submit, cv_done;
  bool stop = false;
  int64_t next_id = 1;
  std::deque<Request*> incoming;           // submitted, not yet seen by the scheduler
  std::deque<Request*> waiting;            // seen, not admitted
  std::vector<Request*> active;            // admitted, chunks left or in flight
  std::map<int64_t, std::unique_ptr<Request>> all;
  std::map<std::pair<const void*, int>, std::unique_ptr<Proc>> procs;
  std::mutex proc_mu;                      // process cache and autotuning
  me_server_stats st{};
  uint64_t req_bytes = 0;  // budget held by admitted requests' buffers (until the client collects them)
  std::thread worker;
  size_t rr = 0;

  int n_sms = 0;
  bool persistent_step();
  void lane_collect(Lane& L);
  bool lane_place(Request* q);
  void run();
  bool admit(Request* q);
  bool launch_chunk(Slot& sl, Request* q);
  bool grow_workspaces(size_t need);
  SlotGraph& graph_for(Slot& sl, Request* q, const me::StepArgs& sa);
  void finish(Request* q, me_status status);
  void release(Request* q);
};

namespace {

me_status tune_chunk(me_handle h, const me::KinDev& kin, cudaStream_t s, int64_t* out) {
  // candidates from 2^12 to 2^20 points (x4 apart, until one launch takes 50 ms): time per
  // point of one k_ps/k_me pair, then the smallest chunk within 15 % of the best (small
  // chunks interleave requests more finely)
  const int n_ext = h->desc->n_ext;
  std::vector<int64_t> cand;
  for (int64_t c = kChunkMin; c <= kChunkMax; c *= 4)
    if (me::rt::ws_bytes(n_ext, c) <= kWsMaxBytes) cand.push_back(c);
  if (cand.empty()) return fail(ME_ERR_ARG, "server: process too large for the slot workspace");
  const int64_t cmax = cand.back();
  void* ws = nullptr;
  double* part = nullptr;
  int* status = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaError_t e = cudaMalloc(&ws, me::rt::ws_bytes(n_ext, cmax));
  if (e == cudaSuccess) e = cudaMalloc(&part, 3 * sizeof(double) * (size_t)me::rt::grid_for(h, cmax));
  if (e == cudaSuccess) e = cudaMalloc(&status, sizeof(int));
  if (e == cudaSuccess) e = cudaMemsetAsync(status, 0, sizeof(int), s);
  if (e == cudaSuccess) e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  std::vector<double> per_point;
  for (size_t i = 0; e == cudaSuccess && i < cand.size(); ++i) {
    const int64_t m = cand[i];
    const int gm = me::rt::grid_for(h, m), gp = me::rt::grid_ps_for(h, m);
    float best = 0.0f;
    for (int rep = 0; rep < 3 && e == cudaSuccess; ++rep) {  // first repetition warms up
      e = cudaEventRecord(e0, s);
      if (e == cudaSuccess) {
        const me::StepArgs sa{12345u, (uint64_t)rep * (uint64_t)m, m, ws, status, part, gm, nullptr, nullptr, m};
        e = h->desc->launch_step(h->prec, &kin, &sa, h->cvals.data(), s, gp, gm, nullptr);
      }
      if (e == cudaSuccess) e = cudaEventRecord(e1, s);
      if (e == cudaSuccess) e = cudaEventSynchronize(e1);
      float ms = 0.0f;
      if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
      if (rep == 1 || (rep == 2 && ms < best)) best = ms;
    }
    per_point.push_back((double)best / (double)m);
    if (best > 50.0f) break;  // launch overhead is long amortised: larger chunks only coarsen interleaving
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (ws) cudaFree(ws);
  if (part) cudaFree(part);
  if (status) cudaFree(status);
  if (e != cudaSuccess) return cuda_fail(e, "server autotune");
  double best = per_point[0];
  for (double v : per_point) best = v < best ? v : best;
  for (size_t i = 0; i < per_point.size(); ++i)
    if (per_point[i] <= 1.15 * best) {
      *out = cand[i];
      return ME_OK;
    }
  *out = cmax;
  return ME_OK;
}

// Persistent mode: the tile (points per queue item) and resident blocks per SM of a process's
// persistent kernel, by timing it on a temporary lane whose queue holds one request of 2^18
// points, fully published and closed before the launch (so no block waits): tiles of 256, 1024
// and 4096 points at one block per SM and at the most that fit; the fastest per point wins, and
// the smallest tile within 5 % of it (finer tiles interleave requests more finely).
me_status tune_serve(Proc* p, const me::KinDev& kin, int n_sms, cudaStream_t s) {
  me_handle h = p->h;
  const int bmax = h->desc->serve_blocks_per_sm(h->prec);
  if (bmax < 1) return fail(ME_ERR_CUDA, "server: the persistent kernel does not fit on an SM");
  const int64_t n = 1 << 18;
  const int64_t tiles_max = n / 256;
  Lane L;
  double* part = nullptr;
  int* status = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaError_t e = lane_init(L, 1u << 20);
  if (e == cudaSuccess) e = cudaMalloc(&part, 3 * sizeof(double) * (size_t)tiles_max);
  if (e == cudaSuccess) e = cudaMalloc(&status, sizeof(int));
  if (e == cudaSuccess) e = cudaMemsetAsync(status, 0, sizeof(int), s);
  if (e == cudaSuccess) e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  double best = 0.0;
  int64_t best_tile = 1024;
  int best_b = bmax;
  std::vector<std::pair<double, std::pair<int64_t, int>>> runs;
  const std::vector<int> blocks = bmax > 1 ? std::vector<int>{1, bmax} : std::vector<int>{1};
  for (int64_t tile : {256, 1024, 4096}) {
    for (int b : blocks) {
      float tbest = 0.0f;
      for (int rep = 0; rep < 2 && e == cudaSuccess; ++rep) {  // first repetition warms up
        lane_reset(L);
        const int64_t tiles = (n + tile - 1) / tile;
        lane_record(L, 0, part, nullptr, nullptr, status, tiles);
        const int k = lane_kin(L, kin);
        for (int64_t t = 0; t < tiles; ++t) L.items[L.n_items++] = lane_item(777u, (uint64_t)rep * n, n, tile, t, 0, k);
        store_release(&L.ctl[0], L.n_items);
        store_release(&L.ctl[1], 1u);
        me::ServeCtl c = L.dctl;
        c.tile_points = (int32_t)tile;
        e = cudaEventRecord(e0, s);
        if (e == cudaSuccess) e = cudaMemsetAsync(L.d_claim, 0, sizeof(uint32_t), s);
        if (e == cudaSuccess) e = h->desc->launch_serve(h->prec, &c, h->cvals.data(), s, n_sms * b);
        if (e == cudaSuccess) e = cudaEventRecord(e1, s);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        float ms = 0.0f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
        if (e == cudaSuccess && load_acquire(&L.done[0]) != 1u) e = cudaErrorUnknown;
        if (rep == 1) tbest = ms;
      }
      if (e != cudaSuccess) break;
      runs.push_back({(double)tbest, {tile, b}});
    }
  }
  if (part) cudaFree(part);
  if (status) cudaFree(status);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  lane_free(L);
  if (e != cudaSuccess) return cuda_fail(e, "server persistent autotune");
  best = runs[0].first;
  for (auto& r : runs) best = r.first < best ? r.first : best;
  for (auto& r : runs)
    if (r.first <= 1.05 * best) {
      best_tile = r.second.first;
      best_b = r.second.second;
      break;
    }
  p->tile = best_tile;
  p->bps = best_b;
  return ME_OK;
}

// process handle (cached per process and precision) with its chunk tuned for kin
me_status get_proc(me_server s, const char* process, int32_t prec, const me_kin* kin, Proc** out, cudaStream_t st) {
  me_handle h = nullptr;
  me_status r = me_create(process, nullptr, prec, &h);
  if (r != ME_OK) return r;
  std::lock_guard<std::mutex> lock(s->proc_mu);
  auto key = std::make_pair((const void*)h->desc, (int)prec);
  auto it = s->procs.find(key);
  Proc* p;
  if (it == s->procs.end()) {
    auto np = std::make_unique<Proc>();
    np->h = h;
    p = np.get();
    s->procs.emplace(key, std::move(np));
  } else {
    me_destroy(h);
    p = it->second.get();
  }
  if (p->chunk == 0) {
    me::KinDev k;
    if ((r = me::rt::make_kin(p->h, kin, k)) != ME_OK) return r;
    if (s->cfg.persistent && p->h->desc->launch_serve) {
      if ((r = tune_serve(p, k, s->n_sms, st)) != ME_OK) return r;
      p->serve = true;
      p->chunk = p->tile;
    } else {
      int64_t c = 0;
      if ((r = tune_chunk(p->h, k, st, &c)) != ME_OK) return r;
      p->chunk = c;
    }
  }
  *out = p;
  return ME_OK;
}

}  // namespace

// buffers of an admitted request; false if they do not fit now
bool me_server_s::admit(Request* q) {
  const int n_ext = q->proc->h->desc->n_ext;
  const uint64_t bytes = q->need;
  if (st.bytes_in_use + bytes > cfg.mem_cap_bytes || free_stage.empty()) return false;
  q->bytes = bytes;
  cudaError_t e = cudaSuccess;
  auto alloc = [&](void** p, size_t b) {
    if (e == cudaSuccess && b) e = cudaMallocFromPoolAsync(p, b, pool, admin);
  };
  alloc((void**)&q->d_partials, 3 * sizeof(double) * (size_t)q->grid_me * (size_t)q->nchunks);
  alloc((void**)&q->d_acc, 4 * sizeof(double));
  alloc((void**)&q->d_status, 16);
  if (q->r.want_me2) alloc((void**)&q->d_me2, sizeof(double) * (size_t)q->r.n);
  if (q->r.want_momenta) alloc((void**)&q->d_mom, sizeof(double) * 4 * (size_t)n_ext * (size_t)q->r.n);
  if (e == cudaSuccess) e = cudaMemsetAsync(q->d_status, 0, sizeof(int), admin);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&q->ready, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventRecord(q->ready, admin);
  q->stage = free_stage.back();
  free_stage.pop_back();
  st.bytes_in_use += bytes;
  req_bytes += bytes;
  st.bytes_peak = st.bytes_in_use > st.bytes_peak ? st.bytes_in_use : st.bytes_peak;
  ++st.admitted;
  q->res.t_admit_ms = now_ms(t0);
  if (e != cudaSuccess) {
    finish(q, ME_ERR_OOM);
    return true;
  }
  q->state = RState::Active;
  if (q->tiles > 0) q->next_chunk = q->nchunks;  // persistent: no chunk launches
  active.push_back(q);
  return true;
}

// every slot's phase-space workspace to at least `need` bytes (stream-ordered: a slot with a
// chunk in flight frees its old workspace after that chunk); the budget counts them
bool me_server_s::grow_workspaces(size_t need) {
  for (Slot& sl : slots) {
    if (sl.ws_cap >= need) continue;
    if (st.bytes_in_use - sl.ws_cap + need > cfg.mem_cap_bytes) return false;
    if (sl.ws) cudaFreeAsync(sl.ws, sl.stream);
    st.bytes_in_use -= sl.ws_cap;
    sl.ws = nullptr;
    sl.ws_cap = 0;
    if (cudaMallocFromPoolAsync(&sl.ws, need, pool, sl.stream) != cudaSuccess) return false;
    sl.ws_cap = need;
    st.bytes_in_use += need;
    st.bytes_peak = st.bytes_in_use > st.bytes_peak ? st.bytes_in_use : st.bytes_peak;
  }
  return true;
}

// Capture the step of q's process on this slot (first use only).  Its two kernel
// nodes are told apart by their dependencies (the phase-space kernel has none).
SlotGraph& me_server_s::graph_for(Slot& sl, Request* q, const me::StepArgs& sa) {
  const std::pair<const Proc*, int> key(q->proc, q->kin.kind);
  auto it = sl.graphs.find(key);
  if (it != sl.graphs.end()) return it->second;
  SlotGraph& sg = sl.graphs[key];
  me_handle h = q->proc->h;
  cudaGraph_t g = nullptr;
  cudaError_t e = cudaStreamBeginCapture(sl.stream, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) return sg;
  const cudaError_t el = h->desc->launch_step(h->prec, &q->kin, &sa, h->cvals.data(), sl.stream, q->grid_ps,
                                              q->grid_me, nullptr);
  e = cudaStreamEndCapture(sl.stream, &g);
  if (el != cudaSuccess || e != cudaSuccess || !g) {
    if (g) cudaGraphDestroy(g);
    cudaGetLastError();
    return sg;
  }
  size_t n = 0;
  cudaGraphGetNodes(g, nullptr, &n);
  std::vector<cudaGraphNode_t> nodes(n);
  if (n) cudaGraphGetNodes(g, nodes.data(), &n);
  int nk = 0;
  for (cudaGraphNode_t nd : nodes) {
    cudaGraphNodeType t;
    if (cudaGraphNodeGetType(nd, &t) != cudaSuccess || t != cudaGraphNodeTypeKernel) continue;
    ++nk;
    size_t ndep = 0;
    cudaGraphNodeGetDependencies(nd, nullptr, nullptr, &ndep);
    if (ndep == 0) sg.node_ps = nd;
    else sg.node_me = nd;
  }
  if (nk != 2 || !sg.node_ps || !sg.node_me || cudaGraphKernelNodeGetParams(sg.node_ps, &sg.p_ps) != cudaSuccess ||
      cudaGraphKernelNodeGetParams(sg.node_me, &sg.p_me) != cudaSuccess ||
      cudaGraphInstantiate(&sg.exec, g, 0) != cudaSuccess) {
    cudaGraphDestroy(g);
    cudaGetLastError();
    sg = SlotGraph{};
    return sg;
  }
  sg.g = g;
  sg.ok = true;
  return sg;
}

bool me_server_s::launch_chunk(Slot& sl, Request* q) {
  const int64_t c = q->next_chunk++;
  const int64_t first = c * q->chunk;
  const int64_t m = std::min<int64_t>(q->chunk, q->r.n - first);
  me_handle h = q->proc->h;
  cudaError_t e = cudaStreamWaitEvent(sl.stream, q->ready, 0);
  const me::StepArgs sa{q->r.seed, q->r.counter_offset + (uint64_t)first, m, sl.ws, q->d_status,
                        q->d_partials + 3 * (size_t)q->grid_me * (size_t)c, q->grid_me,
                        q->d_me2 ? q->d_me2 + first : nullptr, q->d_mom ? q->d_mom + first : nullptr, q->r.n};
  SlotGraph& sg = graph_for(sl, q, sa);
  if (e == cudaSuccess && sg.ok) {
    // the chunk's arguments into the executable graph, then one launch
    me::KinDev kin = q->kin;
    me::StepArgs args = sa;
    void* a_ps[2] = {&kin, &args};
    void* a_me[3] = {&kin, &args, sg.p_me.kernelParams[2]};
    cudaKernelNodeParams pp = sg.p_ps, pm = sg.p_me;
    pp.kernelParams = a_ps;
    pm.kernelParams = a_me;
    e = cudaGraphExecKernelNodeSetParams(sg.exec, sg.node_ps, &pp);
    if (e == cudaSuccess) e = cudaGraphExecKernelNodeSetParams(sg.exec, sg.node_me, &pm);
    if (e == cudaSuccess) e = cudaGraphLaunch(sg.exec, sl.stream);
    if (e == cudaSuccess) ++st.graph_launches;
  } else if (e == cudaSuccess) {
    e = h->desc->launch_step(h->prec, &q->kin, &sa, h->cvals.data(), sl.stream, q->grid_ps, q->grid_me, nullptr);
  }
  if (e == cudaSuccess) e = cudaEventRecord(sl.ev, sl.stream);
  if (c == 0) q->res.t_start_ms = now_ms(t0);
  ++st.launches;
  if (e != cudaSuccess) {
    me::rt::fail(ME_ERR_CUDA, std::string("server launch: ") + cudaGetErrorString(e));
    q->next_chunk = q->nchunks;  // launch nothing more for this request
    return false;
  }
  sl.req = q;
  sl.final = false;
  return true;
}

void me_server_s::finish(Request* q, me_status status) {
  q->res.status = status;
  q->res.done = 1;
  q->res.t_done_ms = now_ms(t0);
  q->state = RState::Done;
  ++st.completed;
  if (status == ME_OK) st.points_done += q->r.n;
  for (size_t i = 0; i < active.size(); ++i)
    if (active[i] == q) {
      active.erase(active.begin() + (long)i);
      break;
    }
  cv_done.notify_all();
}

void me_server_s::release(Request* q) {
  auto fr = [&](void* p) {
    if (p) cudaFreeAsync(p, admin);
  };
  fr(q->d_partials);
  fr(q->d_acc);
  fr(q->d_status);
  fr(q->d_me2);
  fr(q->d_mom);
  q->d_partials = q->d_acc = q->d_me2 = q->d_mom = nullptr;
  q->d_status = nullptr;
  if (q->ready) cudaEventDestroy(q->ready);
  q->ready = nullptr;
  if (q->stage >= 0) free_stage.push_back(q->stage);
  q->stage = -1;
  if (q->bytes) {
    st.bytes_in_use -= q->bytes;
    req_bytes -= q->bytes;
  }
  q->bytes = 0;
}

// completed requests of a lane: the kernel published their sums (done flag, acquire)
void me_server_s::lane_collect(Lane& L) {
  for (size_t i = 0; i < L.in.size();) {
    Request* q = L.in[i];
    if (load_acquire(&L.done[q->lane_slot]) != 1u) {
      ++i;
      continue;
    }
    const double* t = L.totals + 4 * q->lane_slot;
    q->res.acc.sum_w = t[0];
    q->res.acc.sum_w2 = t[1];
    q->res.acc.n_acc = q->r.n;
    q->res.acc.n_try = (int64_t)llround(t[2]);
    L.free_req.push_back(q->lane_slot);
    q->lane = nullptr;
    q->lane_slot = -1;
    L.in.erase(L.in.begin() + (long)i);
    finish(q, t[3] != 0.0 ? ME_ERR_TIMEOUT : ME_OK);
  }
}

// a lane for an admitted persistent request: a running lane of its process that is still open
// and has room, else an idle slot whose persistent kernel is started now (graph launch)
bool me_server_s::lane_place(Request* q) {
  Lane* L = nullptr;
  int kin = -1;
  for (Slot& sl : slots) {
    Lane& c = *sl.lane;
    if (!c.running || c.closed || c.proc != q->proc || c.free_req.empty()) continue;
    int64_t unpublished = 0;  // queue room the lane's requests still need
    for (Request* x : c.in) unpublished += x->tiles - x->tiles_published;
    if ((int64_t)c.n_items + unpublished + q->tiles > (int64_t)kLaneItems) continue;
    if ((kin = lane_kin(c, q->kin)) < 0) continue;
    L = &c;
    break;
  }
  if (!L) {
    Slot* free_slot = nullptr;
    int running = 0;
    for (Slot& sl : slots) {
      if (sl.lane->running) ++running;
      else if (!free_slot && !sl.req) free_slot = &sl;
    }
    if (!free_slot || q->tiles > (int64_t)kLaneItems) return false;
    Lane& c = *free_slot->lane;
    lane_reset(c);
    c.proc = q->proc;
    // the SMs' resident blocks of this kernel, shared among the lanes running
    c.grid = std::max(1, n_sms * q->proc->bps / (running + 1));
    bool as_graph = false;
    const cudaError_t e = lane_launch(c, q->proc, c.grid, q->proc->tile, free_slot->stream, &as_graph);
    if (e != cudaSuccess) {
      me::rt::fail(ME_ERR_CUDA, std::string("server lane launch: ") + cudaGetErrorString(e));
      finish(q, ME_ERR_CUDA);
      return true;
    }
    c.running = true;
    ++st.lane_launches;
    if (as_graph) ++st.graph_launches;
    kin = lane_kin(c, q->kin);
    L = &c;
  }
  const int slot = L->free_req.back();
  L->free_req.pop_back();
  lane_record(*L, slot, q->d_partials, q->d_me2, q->d_mom, q->d_status, q->tiles);
  q->lane = L;
  q->lane_slot = slot;
  q->lane_kin = kin;
  q->tiles_published = 0;
  q->res.t_start_ms = now_ms(t0);
  L->in.push_back(q);
  return true;
}

// One pass of the persistent lanes: ends of kernels, completed requests, placement of
// admitted requests, publication of tiles a little ahead of the blocks' claims (round-robin
// over a lane's requests), and closing of lanes with nothing left to publish.
bool me_server_s::persistent_step() {
  bool progress = false;
  for (Slot& sl : slots) {
    Lane& L = *sl.lane;
    if (!L.running || cudaEventQuery(L.ev_end) == cudaErrorNotReady) continue;
    cudaGetLastError();
    progress = true;
    L.running = false;
    lane_collect(L);
    const bool timed_out = load_acquire(&L.ctl[2]) != 0u;
    if (timed_out) ++st.lane_timeouts;
    for (Request* q : L.in) {
      L.free_req.push_back(q->lane_slot);
      q->lane = nullptr;
      q->lane_slot = -1;
      me::rt::fail(timed_out ? ME_ERR_TIMEOUT : ME_ERR_CUDA,
                   timed_out ? "server: a persistent kernel's wait for work ran out"
                             : "server: a persistent kernel ended before its requests");
      finish(q, timed_out ? ME_ERR_TIMEOUT : ME_ERR_CUDA);
    }
    L.in.clear();
    L.proc = nullptr;
  }
  for (Slot& sl : slots)
    if (sl.lane->running) lane_collect(*sl.lane);
  for (Request* q : std::vector<Request*>(active)) {
    if (stop || q->state != RState::Active || q->tiles == 0 || q->lane) continue;
    if (cudaEventQuery(q->ready) == cudaErrorNotReady) continue;  // its buffers are still being set up
    if (lane_place(q)) progress = true;
  }
  if (cfg.inject_feeder_stall) return progress;
  for (Slot& sl : slots) {
    Lane& L = *sl.lane;
    if (!L.running || L.closed) continue;
    const uint32_t claimed = __atomic_load_n(&L.ctl[3], __ATOMIC_RELAXED);
    const uint32_t window = (uint32_t)(2 * L.grid + 8);
    const uint32_t target = std::min<uint32_t>(kLaneItems, claimed + window);
    const uint32_t before = L.n_items;
    bool more = true;
    while (more && L.n_items < target) {
      more = false;
      for (size_t k = 0; k < L.in.size() && L.n_items < target; ++k) {
        Request* q = L.in[(L.rr + k) % L.in.size()];
        if (q->tiles_published >= q->tiles) continue;
        L.items[L.n_items++] = lane_item(q->r.seed, q->r.counter_offset, q->r.n, q->proc->tile, q->tiles_published++,
                                         q->lane_slot, q->lane_kin);
        more = true;
      }
      L.rr = L.in.empty() ? 0 : (L.rr + 1) % L.in.size();
    }
    if (L.n_items != before) {
      store_release(&L.ctl[0], L.n_items);
      st.lane_items += L.n_items - before;
      progress = true;
    }
    // nothing left to publish and no admitted request of its process that this lane could still
    // take: close (a request that does not fit the lane's remaining queue goes to a new lane)
    bool left = false;
    int64_t unpublished = 0;
    for (Request* q : L.in) {
      left = left || q->tiles_published < q->tiles;
      unpublished += q->tiles - q->tiles_published;
    }
    for (Request* q : active)
      left = left || (q->state == RState::Active && q->tiles && !q->lane && q->proc == L.proc &&
                      (int64_t)L.n_items + unpublished + q->tiles <= (int64_t)kLaneItems && !L.free_req.empty());
    if (!left || stop) {
      store_release(&L.ctl[1], 1u);
      L.closed = true;
      progress = true;
    }
  }
  return progress;
}

void me_server_s::run() {
  cudaSetDevice(device);
  std::unique_lock<std::mutex> lock(mu);
  while (true) {
    bool progress = false;
    // new arrivals: resolve the process (tuning it on first use) and size the request
    while (!stop && !incoming.empty()) {
      Request* q = incoming.front();
      incoming.pop_front();
      lock.unlock();
      Proc* p = nullptr;
      me_status r = get_proc(this, q->process.c_str(), q->r.precision, &q->r.kin, &p, admin);
      lock.lock();
      if (r != ME_OK) {
        finish(q, r);
        continue;
      }
      q->proc = p;
      me::rt::make_kin(p->h, &q->r.kin, q->kin);  // checked at submit
      if (cfg.persistent && p->serve && q->kin.kind != ME_PS_YPT &&
          (q->r.n + p->tile - 1) / p->tile <= (int64_t)kLaneItems / 2) {
        // a persistent lane takes it in tiles; its partials are one per tile
        const int n_ext = p->h->desc->n_ext;
        q->chunk = p->tile;
        q->tiles = (q->r.n + p->tile - 1) / p->tile;
        q->nchunks = q->tiles;
        q->grid_me = 1;
        q->res.chunk = p->tile;
        q->ws_need = 0;
        q->need = 64 + 3 * sizeof(double) * (uint64_t)q->tiles + (q->r.want_me2 ? 8ull * (uint64_t)q->r.n : 0) +
                  (q->r.want_momenta ? 32ull * (uint64_t)n_ext * (uint64_t)q->r.n : 0);
        waiting.push_back(q);
        progress = true;
        continue;
      }
      q->chunk = std::min<int64_t>(p->chunk, q->r.n);
      q->nchunks = (q->r.n + q->chunk - 1) / q->chunk;
      // one launch shape per process (its autotuned chunk), so that its captured graph serves
      // every request; a shorter chunk leaves blocks without points
      q->grid_me = me::rt::grid_for(p->h, p->chunk);
      q->grid_ps = me::rt::grid_ps_for(p->h, p->chunk);
      q->res.chunk = q->chunk;
      const int n_ext = p->h->desc->n_ext;
      q->ws_need = me::rt::ws_bytes(n_ext, q->chunk);
      q->need = 64 + 3 * sizeof(double) * (uint64_t)q->grid_me * (uint64_t)q->nchunks +
                (q->r.want_me2 ? 8ull * (uint64_t)q->r.n : 0) +
                (q->r.want_momenta ? 32ull * (uint64_t)n_ext * (uint64_t)q->r.n : 0);
      waiting.push_back(q);
      progress = true;
    }
    bool inflight = false;
    for (Slot& sl : slots) inflight = inflight || sl.req || (sl.lane && sl.lane->running);
    // admission, first come first served; a request that does not fit even with nothing
    // else admitted is refused
    while (!stop && !waiting.empty()) {
      Request* q = waiting.front();
      if (!grow_workspaces(q->ws_need) || !admit(q)) {
        // it cannot fit beside the slot workspaces alone: nothing runs, and no finished request
        // still holds buffers that its client has yet to collect
        if (active.empty() && !inflight && req_bytes == 0) {
          waiting.pop_front();
          finish(q, ME_ERR_OOM);
          progress = true;
          continue;
        }
        break;
      }
      waiting.pop_front();
      progress = true;
    }
    // completions
    for (Slot& sl : slots) {
      if (!sl.req || cudaEventQuery(sl.ev) == cudaErrorNotReady) continue;
      Request* q = sl.req;
      sl.req = nullptr;
      progress = true;
      if (sl.final) {
        const double* hs = h_stage + 8 * q->stage;
        int status = 0;
        std::memcpy(&status, hs + 3, sizeof(int));
        q->res.acc.sum_w = hs[0];
        q->res.acc.sum_w2 = hs[1];
        q->res.acc.n_acc = q->r.n;
        q->res.acc.n_try = (int64_t)llround(hs[2]);
        finish(q, status ? ME_ERR_TIMEOUT : ME_OK);
        continue;
      }
      if (++q->chunks_done < q->nchunks) continue;
      if (q->failed) {
        finish(q, ME_ERR_CUDA);
        continue;
      }
      // fixed-order sum of all chunks' partials, then the sums and status to pinned staging
      double* hs = h_stage + 8 * q->stage;
      cudaError_t e = me::rt::launch_reduce(q->d_partials, (int)(q->grid_me * q->nchunks), q->d_acc, sl.stream);
      if (e == cudaSuccess) e = cudaMemcpyAsync(hs, q->d_acc, 3 * sizeof(double), cudaMemcpyDeviceToHost, sl.stream);
      if (e == cudaSuccess) e = cudaMemcpyAsync(hs + 3, q->d_status, sizeof(int), cudaMemcpyDeviceToHost, sl.stream);
      if (e == cudaSuccess) e = cudaEventRecord(sl.ev, sl.stream);
      if (e != cudaSuccess) {
        finish(q, ME_ERR_CUDA);
        continue;
      }
      q->state = RState::Final;
      sl.req = q;
      sl.final = true;
    }
    if (cfg.persistent && persistent_step()) progress = true;
    // free slots take the next chunk, round-robin over the admitted requests
    for (Slot& sl : slots) {
      if (stop || sl.req || (sl.lane && sl.lane->running)) continue;
      Request* pick = nullptr;
      for (size_t k = 0; k < active.size() && !pick; ++k) {
        Request* q = active[(rr + k) % active.size()];
        if (q->state == RState::Active && q->next_chunk < q->nchunks && q->ws_need <= sl.ws_cap) {
          pick = q;
          rr = (rr + k + 1) % active.size();
        }
      }
      if (!pick) continue;
      progress = true;
      if (!launch_chunk(sl, pick)) {
        // the failed chunk and the ones never launched count as done; the request
        // finishes with an error once its chunks on other slots have drained
        pick->failed = true;
        pick->chunks_done += 1 + (pick->nchunks - pick->next_chunk);
        pick->next_chunk = pick->nchunks;
        if (pick->chunks_done >= pick->nchunks) finish(pick, ME_ERR_CUDA);
      }
    }
    inflight = false;
    for (Slot& sl : slots) inflight = inflight || sl.req || (sl.lane && sl.lane->running);
    // admitted persistent requests whose buffers are still being set up: poll, do not sleep
    for (Request* q : active) inflight = inflight || (q->tiles && !q->lane && q->state == RState::Active);
    st.waiting = (int64_t)waiting.size();
    st.active = (int64_t)active.size();
    if (stop && !inflight) {
      // requests not yet run are dropped at shutdown
      for (Request* q : incoming) finish(q, ME_ERR_STATE);
      incoming.clear();
      for (Request* q : waiting) finish(q, ME_ERR_STATE);
      waiting.clear();
      for (Request* q : std::vector<Request*>(active)) finish(q, ME_ERR_STATE);
      break;
    }
    if (!progress) {
      if (inflight) {
        lock.unlock();
        std::this_thread::sleep_for(std::chrono::microseconds(cfg.persistent ? 5 : 20));
        lock.lock();
      } else {
        cv_submit.wait_for(lock, std::chrono::milliseconds(2));
      }
    }
  }
}

extern "C" {

me_status me_server_create(const me_server_config* cfg, me_server* out) {
  if (!out) return fail(ME_ERR_ARG, "me_server_create: null out");
  *out = nullptr;
  me_server_config c{};
  if (cfg) c = *cfg;
  if (c.mem_cap_bytes == 0) c.mem_cap_bytes = kDefaultCap;
  if (c.n_slots == 0) c.n_slots = 4;
  if (c.max_requests == 0) c.max_requests = 4096;
  if (c.n_slots < 1 || c.n_slots > 16) return fail(ME_ERR_ARG, "me_server_create: n_slots must be 1..16");
  if (c.max_requests < 1 || c.max_requests > 65536)
    return fail(ME_ERR_ARG, "me_server_create: max_requests must be 1..65536");
  if (c.spin_limit_us == 0) c.spin_limit_us = 500000;
  if (c.persistent != 0 && c.persistent != 1) return fail(ME_ERR_ARG, "me_server_create: persistent must be 0 or 1");
  if (c.spin_limit_us < 1 || c.spin_limit_us > 10000000)
    return fail(ME_ERR_ARG, "me_server_create: spin_limit_us must be 1..10^7");
  auto s = std::make_unique<me_server_s>();
  s->cfg = c;
  s->t0 = std::chrono::steady_clock::now();
  s->st.mem_cap_bytes = c.mem_cap_bytes;
  cudaError_t e = cudaGetDevice(&s->device);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
  cudaMemPoolProps props{};
  props.allocType = cudaMemAllocationTypePinned;
  props.location.type = cudaMemLocationTypeDevice;
  props.location.id = s->device;
  if ((e = cudaMemPoolCreate(&s->pool, &props)) != cudaSuccess) return cuda_fail(e, "cudaMemPoolCreate");
  uint64_t keep = c.mem_cap_bytes;  // freed blocks stay in the pool up to the budget
  cudaMemPoolSetAttribute(s->pool, cudaMemPoolAttrReleaseThreshold, &keep);
  if ((e = cudaStreamCreateWithFlags(&s->admin, cudaStreamNonBlocking)) != cudaSuccess)
    return cuda_fail(e, "cudaStreamCreate");
  if ((e = cudaDeviceGetAttribute(&s->n_sms, cudaDevAttrMultiProcessorCount, s->device)) != cudaSuccess)
    return cuda_fail(e, "cudaDeviceGetAttribute");
  s->slots.resize(c.n_slots);
  for (Slot& sl : s->slots) {
    if ((e = cudaStreamCreateWithFlags(&sl.stream, cudaStreamNonBlocking)) != cudaSuccess)
      return cuda_fail(e, "cudaStreamCreate");
    if ((e = cudaEventCreateWithFlags(&sl.ev, cudaEventDisableTiming)) != cudaSuccess)
      return cuda_fail(e, "cudaEventCreate");
    sl.lane = std::make_unique<Lane>();
    if (c.persistent && (e = lane_init(*sl.lane, (uint64_t)c.spin_limit_us)) != cudaSuccess)
      return fail(ME_ERR_OOM, "me_server_create: lane queues");
  }
  if ((e = cudaMallocHost(&s->h_stage, 8 * sizeof(double) * (size_t)c.max_requests)) != cudaSuccess)
    return fail(ME_ERR_OOM, "me_server_create: pinned staging");
  for (int i = c.max_requests - 1; i >= 0; --i) s->free_stage.push_back(i);
  me_server_s* raw = s.release();
  raw->worker = std::thread([raw] { raw->run(); });
  *out = raw;
  return ME_OK;
}

me_status me_server_warm(me_server s, const char* process, int32_t precision, const me_kin* kin, int64_t* chunk) {
  if (!s || !process || !kin) return fail(ME_ERR_ARG, "me_server_warm: null argument");
  cudaSetDevice(s->device);
  cudaStream_t st = nullptr;
  cudaError_t e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
  if (e != cudaSuccess) return cuda_fail(e, "cudaStreamCreate");
  Proc* p = nullptr;
  me_status r = get_proc(s, process, precision, kin, &p, st);
  cudaStreamDestroy(st);
  if (r == ME_OK && chunk) *chunk = p->chunk;
  return r;
}

me_status me_server_submit(me_server s, const me_request* r, int64_t* ticket) {
  if (!s || !r || !ticket || !r->process) return fail(ME_ERR_ARG, "me_server_submit: null argument");
  if (r->n < 1) return fail(ME_ERR_ARG, "me_server_submit: n must be >= 1");
  if (r->precision != ME_FP64 && r->precision != ME_MIXED) return fail(ME_ERR_ARG, "me_server_submit: precision");
  // argument checks on a throw-away handle (no device work)
  me_handle h = nullptr;
  me_status st = me_create(r->process, nullptr, r->precision, &h);
  if (st != ME_OK) return st;
  me::KinDev k;
  st = me::rt::make_kin(h, &r->kin, k);
  const int n_ext = h->desc->n_ext;
  me_destroy(h);
  if (st != ME_OK) return st;
  const uint64_t arrays = (r->want_me2 ? 8ull * (uint64_t)r->n : 0) +
                          (r->want_momenta ? 32ull * (uint64_t)n_ext * (uint64_t)r->n : 0);
  if (arrays + me::rt::ws_bytes(n_ext, kChunkMax) > s->cfg.mem_cap_bytes)
    return fail(ME_ERR_OOM, "me_server_submit: request larger than the memory budget");
  auto q = std::make_unique<Request>();
  q->r = *r;
  q->process = r->process;
  q->r.process = nullptr;
  {
    std::lock_guard<std::mutex> lock(s->mu);
    q->id = s->next_id++;
    q->res.t_submit_ms = now_ms(s->t0);
    *ticket = q->id;
    s->incoming.push_back(q.get());
    s->all.emplace(q->id, std::move(q));
    ++s->st.submitted;
  }
  s->cv_submit.notify_one();
  return ME_OK;
}

me_status me_server_poll(me_server s, int64_t ticket, me_request_result* res) {
  if (!s || !res) return fail(ME_ERR_ARG, "me_server_poll: null argument");
  std::lock_guard<std::mutex> lock(s->mu);
  auto it = s->all.find(ticket);
  if (it == s->all.end()) return fail(ME_ERR_ARG, "me_server_poll: unknown ticket");
  *res = it->second->res;
  return ME_OK;
}

me_status me_server_wait(me_server s, int64_t ticket, double timeout_s, me_request_result* res, double* me2_host,
                         double* momenta_host) {
  if (!s) return fail(ME_ERR_ARG, "me_server_wait: null server");
  std::unique_lock<std::mutex> lock(s->mu);
  auto it = s->all.find(ticket);
  if (it == s->all.end()) return fail(ME_ERR_ARG, "me_server_wait: unknown ticket");
  Request* q = it->second.get();
  auto done = [q] { return q->state == RState::Done; };
  if (timeout_s < 0) s->cv_done.wait(lock, done);
  else if (!s->cv_done.wait_for(lock, std::chrono::duration<double>(timeout_s), done))
    return fail(ME_ERR_TIMEOUT, "me_server_wait: request not finished");
  if (res) *res = q->res;
  const me_status st = (me_status)q->res.status;
  cudaError_t e = cudaSuccess;
  if (st == ME_OK) {
    cudaSetDevice(s->device);
    const int n_ext = q->proc->h->desc->n_ext;
    if (me2_host && q->d_me2)
      e = cudaMemcpyAsync(me2_host, q->d_me2, 8 * (size_t)q->r.n, cudaMemcpyDeviceToHost, s->admin);
    if (e == cudaSuccess && momenta_host && q->d_mom)
      e = cudaMemcpyAsync(momenta_host, q->d_mom, 32 * (size_t)n_ext * (size_t)q->r.n, cudaMemcpyDeviceToHost,
                          s->admin);
  }
  s->release(q);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s->admin);
  s->all.erase(it);
  s->cv_submit.notify_one();  // freed budget: the scheduler may admit a waiting request
  if (e != cudaSuccess) return cuda_fail(e, "me_server_wait copy");
  if (st != ME_OK) return fail(st, "me_server_wait: request failed");
  return ME_OK;
}

me_status me_server_get_stats(me_server s, me_server_stats* out) {
  if (!s || !out) return fail(ME_ERR_ARG, "me_server_get_stats: null argument");
  std::lock_guard<std::mutex> lock(s->mu);
  *out = s->st;
  return ME_OK;
}

void me_server_destroy(me_server s) {
  if (!s) return;
  {
    std::lock_guard<std::mutex> lock(s->mu);
    s->stop = true;
  }
  s->cv_submit.notify_all();
  if (s->worker.joinable()) s->worker.join();
  cudaSetDevice(s->device);
  for (auto& kv : s->all) s->release(kv.second.get());
  for (Slot& sl : s->slots) {
    if (sl.stream) cudaStreamSynchronize(sl.stream);
    for (auto& kv : sl.graphs) {
      if (kv.second.exec) cudaGraphExecDestroy(kv.second.exec);
      if (kv.second.g) cudaGraphDestroy(kv.second.g);
    }
    if (sl.ws) cudaFreeAsync(sl.ws, sl.stream);
    if (sl.stream) cudaStreamSynchronize(sl.stream);
    if (sl.lane) lane_free(*sl.lane);
    if (sl.ev) cudaEventDestroy(sl.ev);
    if (sl.stream) cudaStreamDestroy(sl.stream);
  }
  if (s->admin) {
    cudaStreamSynchronize(s->admin);
    cudaStreamDestroy(s->admin);
  }
  if (s->pool) cudaMemPoolDestroy(s->pool);
  if (s->h_stage) cudaFreeHost(s->h_stage);
  for (auto& kv : s->procs) me_destroy(kv.second->h);
  delete s;
}

}  // extern "C"
