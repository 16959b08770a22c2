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
};

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
};

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
  std::thread worker;
  size_t rr = 0;

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
    int64_t c = 0;
    if ((r = tune_chunk(p->h, k, st, &c)) != ME_OK) return r;
    p->chunk = c;
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
  st.bytes_peak = st.bytes_in_use > st.bytes_peak ? st.bytes_in_use : st.bytes_peak;
  ++st.admitted;
  q->res.t_admit_ms = now_ms(t0);
  if (e != cudaSuccess) {
    finish(q, ME_ERR_OOM);
    return true;
  }
  q->state = RState::Active;
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
  if (q->bytes) st.bytes_in_use -= q->bytes;
  q->bytes = 0;
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
    for (Slot& sl : slots) inflight = inflight || sl.req;
    // admission, first come first served; a request that does not fit even with nothing
    // else admitted is refused
    while (!stop && !waiting.empty()) {
      Request* q = waiting.front();
      if (!grow_workspaces(q->ws_need) || !admit(q)) {
        if (active.empty() && !inflight) {  // it cannot fit beside the slot workspaces alone
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
    // free slots take the next chunk, round-robin over the admitted requests
    for (Slot& sl : slots) {
      if (stop || sl.req) continue;
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
    for (Slot& sl : slots) inflight = inflight || sl.req;
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
        std::this_thread::sleep_for(std::chrono::microseconds(20));
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
  s->slots.resize(c.n_slots);
  for (Slot& sl : s->slots) {
    if ((e = cudaStreamCreateWithFlags(&sl.stream, cudaStreamNonBlocking)) != cudaSuccess)
      return cuda_fail(e, "cudaStreamCreate");
    if ((e = cudaEventCreateWithFlags(&sl.ev, cudaEventDisableTiming)) != cudaSuccess)
      return cuda_fail(e, "cudaEventCreate");
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
