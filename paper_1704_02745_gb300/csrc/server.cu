// server.cu -- continuous-batching solve server of libpb (pb_server_*,
// pb_batch_*): many MD snapshots (arXiv:1704.02745 Sec. 1: PB over thousands
// to millions of snapshots) solved together on one GPU.
//
// A worker thread owns the server's CUDA work.  Each round it
//   1. admits queued requests (pb_plan_admission) into resident grids --
//      one per trajectory, reused snapshot after snapshot, so a solve starts
//      from the trajectory's last solution -- evicting idle grids LRU when the
//      device-memory budget requires;
//   2. queues the setup kernels of the admitted snapshots on four setup
//      streams (each after the last work on its grid only, so they run beside
//      the running graph and beside each other), then the start of their
//      solves on the compute stream after them (no host round trip);
//   3. rebuilds the batch's work list when the active set changed: the
//      stencil tiles of every active grid, largest first, each grid's partial
//      sums at its own offset, so its reductions are summed in a fixed order
//      whatever else runs;
//   4. queues a captured device graph of `ticks` phase ticks over the whole
//      batch (finished grids are skipped by their convergence mask) and a copy
//      of all grids' scalars;
//   5. while that graph runs, reads the scalars the previous round's graph
//      left, queues the energy (and phi) of the solves that finished in it on
//      the copy stream, beside the running graph, and hands out the results
//      queued one round earlier.
// Everything the host uploads comes from pinned staging in two sets, one
// per round in flight, so no copy waits for the graph ahead of it and the
// GPU never idles on the host between rounds.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <unordered_set>
#include <vector>

#include "pb.h"
#include "pb_host.h"
#include "pb_internal.cuh"
#include "solve.cuh"

using namespace pb;

// ---------------------------------------------------------------------------
// Admission planner (pure host logic).

extern "C" int pb_plan_admission(size_t budget, const pb_slot_state *slots, int n_slots,
                                 const int64_t *req_traj, const int *req_dims,
                                 const size_t *req_bytes, int n_reqs, int *admit, int *evict) {
  std::vector<char> busy(n_slots), gone(n_slots, 0);
  size_t used = 0;
  for (int j = 0; j < n_slots; j++) {
    busy[j] = slots[j].busy != 0;
    used += slots[j].bytes;
    evict[j] = 0;
  }
  int n_admit = 0;
  bool blocked = false;  // a request needing new memory did not fit: no overtaking
  for (int i = 0; i < n_reqs; i++) {
    admit[i] = -2;
    const int64_t tr = req_traj[i];
    const int *dm = req_dims + 3 * i;
    // an idle resident grid of this trajectory with the same dims, most recent first
    int own = -1;
    if (tr >= 0)
      for (int j = 0; j < n_slots; j++)
        if (!gone[j] && !busy[j] && slots[j].trajectory_id == tr && slots[j].nx == dm[0] &&
            slots[j].ny == dm[1] && slots[j].nz == dm[2] &&
            (own < 0 || slots[j].last_used > slots[own].last_used))
          own = j;
    if (own >= 0) {
      admit[i] = own;
      busy[own] = 1;
      n_admit++;
      continue;
    }
    if (blocked) continue;
    // new memory: idle grids of this trajectory with other dims go first, then
    // idle grids least recently used first
    const size_t need = req_bytes[i];
    if (tr >= 0)
      for (int j = 0; j < n_slots; j++)
        if (!gone[j] && !busy[j] && slots[j].trajectory_id == tr) {
          gone[j] = 1;
          evict[j] = 1;
          used -= slots[j].bytes;
        }
    while (used + need > budget) {
      int lru = -1;
      for (int j = 0; j < n_slots; j++)
        if (!gone[j] && !busy[j] && (lru < 0 || slots[j].last_used < slots[lru].last_used)) lru = j;
      if (lru < 0) break;
      gone[lru] = 1;
      evict[lru] = 1;
      used -= slots[lru].bytes;
    }
    if (used + need > budget) {
      blocked = true;
      continue;
    }
    used += need;
    admit[i] = -1;
    n_admit++;
  }
  return n_admit;
}

// ---------------------------------------------------------------------------
// Server state.

namespace {

constexpr int MAX_SLOTS = 1024;  // resident grids (device scalar / descriptor arrays)
constexpr int MAX_QUEUE = 1 << 20;

struct Request {
  uint64_t ticket;
  int64_t traj;
  pb_grid_desc desc;
  std::vector<double> xyz, q, r;
  double *phi_out;
  bool phi_pinned = false;  // phi_out is page-locked: the device copies into it directly
  std::chrono::steady_clock::time_point t_submit;
  size_t bytes;
};

struct Slot {
  pb_grid *g = nullptr;
  int64_t traj = -1;
  size_t bytes = 0;
  bool busy = false;
  bool pending = false;       // busy, its setup queued and not yet seen complete
  bool stopping = false;      // cancelled while on the device: its scalars were set to DONE
  bool has_solution = false;  // x64[xbuf] holds a solution of this trajectory
  uint64_t last_used = 0;
  uint64_t solved_at = 0;     // clock of that solution
  int xbuf = 0;               // which x64 buffer holds it
  Request req;
  bool warm = false;
  uint64_t first_round = 0;   // round whose graph first runs the current solve
};

// A finished solve whose energy (and phi) are queued behind the running graph.
struct Finishing {
  Request req;
  Scal S;
  bool warm = false;
  double *energy = nullptr;  // pinned
  double *phi = nullptr;     // pinned staging, n doubles (phi requested into pageable memory)
  size_t n = 0;
  bool zero_phi = false;     // phi requested and the solution is 0 (b = 0)
};

// Pinned host staging of one round.
struct Stage {
  Inst *inst = nullptr;   // descriptors of slots [0, MAX_SLOTS)
  Item *items = nullptr;  // stencil items, then update items
  size_t cap_items = 0;
  int *counts = nullptr;  // 2 ints
  int *start = nullptr;   // slots whose solves start
  Scal *scal = nullptr;   // scalars of all slots after the round's graph
  double *energy = nullptr;
  double *phi = nullptr;
  size_t cap_phi = 0;
  double *d_energy = nullptr;      // device: the energies of the round's finished solves
  cudaEvent_t ev_graph = nullptr;  // after the graph and the scalar copy
  cudaEvent_t ev_done = nullptr;   // after the energy (and phi) copies
};

}  // namespace

struct pb_server {
  pb_ctx *ctx = nullptr;      // internal context: the caller's device, the server's stream
  pb_ctx *parent = nullptr;   // the caller's context (counters)
  size_t budget = 0;
  pb_solve_opts opts{};
  int mode = MODE_F32_REFINE, coef = COEF_PACKED;
  // host side
  std::thread worker;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  bool stop = false;
  std::deque<Request> queue;
  std::unordered_map<uint64_t, pb_result> done;
  std::unordered_set<uint64_t> outstanding;  // submitted, result not yet returned by a poll
  std::unordered_set<uint64_t> cancelled;    // cancelled after admission: stop, report PB_ERR_CANCELLED
  uint64_t next_ticket = 1, completed = 0, clock = 0;
  int n_active = 0, n_resident = 0;
  size_t bytes_resident = 0;
  // worker-only state
  cudaStream_t stream = nullptr;
  std::vector<Slot> slots;  // index = device slot
  std::vector<int> free_slots;
  Scal *d_scal = nullptr, *h_scal = nullptr;
  int *h_stop = nullptr;  // pinned {PH_DONE, PB_ERR_CANCELLED}: written into a stopped grid's scalars
  Inst *d_inst = nullptr;
  int *d_counts = nullptr, *d_list = nullptr, *d_err = nullptr;
  int *d_rlist = nullptr;  // instances waiting for a residual pass
  Item *d_st = nullptr;
  double *d_st_part = nullptr, *d_rs_part = nullptr;
  size_t cap_st = 0, cap_rs = 0;
  cudaStream_t copy_stream = nullptr;  // result copies, beside the next round's graph
  // setups of admitted snapshots, several at once and beside the running graph
  static constexpr int SETUP_STREAMS = 4;
  cudaStream_t setup_stream[SETUP_STREAMS] = {};
  // per slot: ev_energy after the last solve's energy (its atoms may then be
  // replaced), ev_idle after every read of the grid (creation, or the energy
  // and phi read-out of its last solve), ev_ready after the next snapshot's
  // setup (setup stream)
  std::vector<cudaEvent_t> ev_idle, ev_ready, ev_energy;
  cudaGraphExec_t graph = nullptr;
#ifndef PB_SERVER_TICKS
#define PB_SERVER_TICKS 8
#endif
  int ticks = PB_SERVER_TICKS;
  Stage stage[2];
  uint64_t round = 0;
  // kernel measurement (pb_server_profile_begin/end)
  std::atomic<bool> profiling{false};
  pb_kernel_profile prof{};
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  KernelGrid kg{};
  std::string worker_error;
  // tile plan of the batch (pb_server_set_plan, pb_server_autotune)
  pb_batch_plan plan{32, 100, 3};
  pb_batch_plan plan_next{32, 100, 3};  // requested, applied by the worker (under mu)
  bool plan_requested = false;
  int tune_state = 0;                   // 0 idle, 1 requested, 2 done (under mu)
  pb_server_tune_info tune_out{};
  std::condition_variable cv_tune;
};

namespace {

double since(std::chrono::steady_clock::time_point t0) {
  return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
}

bool cuda_ok(cudaError_t e, pb_server *s, const char *what) {
  if (e == cudaSuccess) return true;
  s->worker_error = std::string(what) + ": " + cudaGetErrorString(e);
  return false;
}

// Grow a device array (contents not kept).
template <typename T>
bool grow(T **p, size_t *cap, size_t need) {
  if (need <= *cap) return true;
  size_t n = std::max(need, *cap * 2);
  if (*p) cudaFree(*p);
  *p = nullptr;
  if (pb_dalloc((void **)p, n * sizeof(T))) {
    *cap = 0;
    return false;
  }
  *cap = n;
  return true;
}

void fail_request(pb_server *s, const Request &rq, int status) {
  pb_result r;
  memset(&r, 0, sizeof(r));
  r.status = status;
  r.info.status = status;
  r.seconds = since(rq.t_submit);
  std::lock_guard<std::mutex> lk(s->mu);
  if (s->cancelled.erase(rq.ticket)) r.status = r.info.status = PB_ERR_CANCELLED;
  s->done[rq.ticket] = r;
  s->completed++;
  s->cv_done.notify_all();
}

// Release the grid of a slot.
void evict_slot(pb_server *s, int j) {
  Slot &sl = s->slots[j];
  if (sl.g) {
    sl.g->scal = nullptr;  // a slot of the server's array, not the grid's own
    pb_grid_release(sl.g);
  }
  sl = Slot();
  s->free_slots.push_back(j);
}

// Admit queued requests and queue their setups; returns their slots, which
// stay pending (out of the batch) until their setups are seen complete.
std::vector<int> admit(pb_server *s) {
  std::vector<Request> cand;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    if (!s->cancelled.empty()) {  // cancelled before admission: leave the queue now
      std::deque<Request> keep;
      for (auto &r : s->queue) {
        if (!s->cancelled.erase(r.ticket)) {
          keep.push_back(std::move(r));
          continue;
        }
        pb_result res;
        memset(&res, 0, sizeof(res));
        res.status = res.info.status = PB_ERR_CANCELLED;
        res.seconds = since(r.t_submit);
        s->done[r.ticket] = res;
        s->completed++;
      }
      s->queue.swap(keep);
      s->cv_done.notify_all();
    }
    const size_t look = std::min<size_t>(s->queue.size(), 4096);
    for (size_t i = 0; i < look; i++) cand.push_back(s->queue[i]);
  }
  std::vector<int> started;
  if (cand.empty()) return started;
  std::vector<int> idx;  // occupied slot indices
  std::vector<pb_slot_state> st;
  for (int j = 0; j < (int)s->slots.size(); j++)
    if (s->slots[j].g) {
      idx.push_back(j);
      const Slot &sl = s->slots[j];
      st.push_back(pb_slot_state{sl.traj, sl.g->d.nx, sl.g->d.ny, sl.g->d.nz, sl.bytes,
                                 sl.busy ? 1 : 0, sl.last_used});
    }
  std::vector<int64_t> traj(cand.size());
  std::vector<int> dims(3 * cand.size());
  std::vector<size_t> bytes(cand.size());
  for (size_t i = 0; i < cand.size(); i++) {
    traj[i] = cand[i].traj;
    dims[3 * i] = cand[i].desc.nx;
    dims[3 * i + 1] = cand[i].desc.ny;
    dims[3 * i + 2] = cand[i].desc.nz;
    bytes[i] = cand[i].bytes;
  }
  std::vector<int> adm(cand.size()), ev(st.size());
  pb_plan_admission(s->budget, st.data(), (int)st.size(), traj.data(), dims.data(), bytes.data(),
                    (int)cand.size(), adm.data(), ev.data());
  for (size_t k = 0; k < st.size(); k++)
    if (ev[k]) evict_slot(s, idx[k]);
  std::vector<uint64_t> taken;
  for (size_t i = 0; i < cand.size(); i++) {
    if (adm[i] == -2) continue;
    Request &rq = cand[i];
    int j;
    if (adm[i] >= 0) {
      j = idx[adm[i]];
      if (!s->slots[j].g) continue;  // evicted after an allocation failure: replan later
    } else {
      if (s->free_slots.empty()) continue;  // all slots in use: stays queued
      j = s->free_slots.back();
      pb_grid *g = nullptr;
      auto create = [&]() -> bool {
        if (pb_grid_create(s->ctx, &rq.desc, true, &g) || pb_ensure_workspace(g, s->mode)) {
          if (g) pb_grid_release(g);
          g = nullptr;
          return false;
        }
        pb_batch_plan_grid(g, s->kg, s->plan.min_planes, s->plan.height_pct);
        return true;
      };
      if (!create()) {
        // The device refused memory the budget model allows: free every idle
        // grid and try once more; if that fails too, the request fails with
        // PB_ERR_OOM (never retried forever) and the server goes on.
        for (int k = 0; k < (int)s->slots.size(); k++)
          if (k != j && s->slots[k].g && !s->slots[k].busy) evict_slot(s, k);
        if (!create()) {
          fail_request(s, rq, PB_ERR_OOM);
          taken.push_back(rq.ticket);
          continue;
        }
      }
      s->free_slots.erase(std::find(s->free_slots.begin(), s->free_slots.end(), j));
      g->scal = s->d_scal + j;
      g->own_scal = false;
      cudaEventRecord(s->ev_idle[j], s->stream);  // its workspace clears
      cudaEventRecord(s->ev_energy[j], s->stream);
      Slot &sl = s->slots[j];
      sl.g = g;
      sl.traj = rq.traj;
      sl.bytes = rq.bytes;
      sl.has_solution = false;
    }
    Slot &sl = s->slots[j];
    // this snapshot's setup stream waits for the energy of the grid's last
    // solve (the setup replaces the atoms it reads); the read-out of that
    // solve's phi may still run beside the setup kernels
    cudaStream_t sst = s->setup_stream[started.size() % pb_server::SETUP_STREAMS];
    cudaStreamWaitEvent(sst, s->ev_energy[j], 0);
    // a new grid of a trajectory starts from the trajectory's latest solution
    // held by an idle grid of the same dims, if any (device-to-device copy)
    if (adm[i] == -1 && s->opts.warm_start && rq.traj >= 0) {
      int src = -1;
      for (int k = 0; k < (int)s->slots.size(); k++) {
        const Slot &o = s->slots[k];
        if (k != j && o.g && o.traj == rq.traj && o.has_solution && !o.busy &&
            o.g->d.nx == rq.desc.nx && o.g->d.ny == rq.desc.ny && o.g->d.nz == rq.desc.nz &&
            (src < 0 || o.solved_at > s->slots[src].solved_at))
          src = k;
      }
      if (src >= 0) {
        const Slot &o = s->slots[src];
        const double *from = o.xbuf ? o.g->x64b : o.g->x64;
        cudaStreamWaitEvent(sst, s->ev_idle[j], 0);
        cudaStreamWaitEvent(sst, s->ev_idle[src], 0);
        cudaMemcpyAsync(sl.g->x64, from, sl.g->n_pad * sizeof(double), cudaMemcpyDeviceToDevice,
                        sst);
        cudaMemsetAsync(s->d_scal + j, 0, sizeof(Scal), s->stream);
        sl.has_solution = true;
        sl.solved_at = o.solved_at;
      }
    }
    sl.busy = true;
    sl.pending = true;
    sl.first_round = s->round;  // reset again when the solve starts
    sl.last_used = ++s->clock;
    sl.warm = s->opts.warm_start && sl.has_solution;
    if (pb_run_setup(sl.g, (int)rq.q.size(), rq.xyz.data(), rq.q.data(), rq.r.data(), false, sst)) {
      sl.busy = false;
      fail_request(s, rq, PB_ERR_CUDA);
      taken.push_back(rq.ticket);
      continue;
    }
    cudaStreamWaitEvent(sst, s->ev_idle[j], 0);  // the last solve's phi is read out
    if (!sl.warm) {  // cold start: phi0 = 0 in both solution buffers
      cudaMemsetAsync(sl.g->x64, 0, sl.g->n_pad * sizeof(double), sst);
      cudaMemsetAsync(sl.g->x64b, 0, sl.g->n_pad * sizeof(double), sst);
    }
    cudaEventRecord(s->ev_ready[j], sst);
    sl.req = std::move(rq);
    taken.push_back(sl.req.ticket);
    started.push_back(j);
  }
  if (!taken.empty()) {
    std::lock_guard<std::mutex> lk(s->mu);
    std::deque<Request> rest;
    for (auto &r : s->queue)
      if (std::find(taken.begin(), taken.end(), r.ticket) == taken.end()) rest.push_back(std::move(r));
    s->queue.swap(rest);
  }
  return started;
}

// Kernel grid of the batch for a plan's stencil occupancy (the two builds of
// the FP32 packed stencil pass: three or two CTAs per SM).
KernelGrid batch_kernel_grid(const pb_server *s, const pb_batch_plan &P) {
  KernelGrid kg = kernel_grid(s->mode, s->coef, s->ctx->num_sms, P.occupancy == 2);
  kg.tile_update = 1;
  return kg;
}

// Re-plan every resident grid (between graph launches: the tile plan holds no
// state across launches).
void replan_all(pb_server *s) {
  for (auto &sl : s->slots)
    if (sl.g) pb_batch_plan_grid(sl.g, s->kg, s->plan.min_planes, s->plan.height_pct);
}

// Upload the descriptors, work lists and partial offsets of the active grids.
// Host staging capacity for n items (pinned; the set is idle when called).
bool stage_items(Stage &st, size_t n) {
  if (n <= st.cap_items) return true;
  const size_t cap = std::max(n, 2 * st.cap_items);
  if (st.items) cudaFreeHost(st.items);
  st.items = nullptr;
  st.cap_items = 0;
  if (cudaMallocHost((void **)&st.items, cap * sizeof(Item)) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  st.cap_items = cap;
  return true;
}

bool rebuild_batch(pb_server *s, Stage &sg, bool *graph_stale) {
  std::vector<Item> st;
  std::vector<int> active;
  for (int j = 0; j < (int)s->slots.size(); j++)
    if (s->slots[j].g && s->slots[j].busy && !s->slots[j].pending) active.push_back(j);
  int st_off = 0, rs_off = 0, hi = 0;
  for (int j : active) {
    pb_grid *g = s->slots[j].g;
    Inst &I = sg.inst[j];
    if (pb_make_inst(g, &s->opts, s->mode, s->coef, I)) return false;
    I.s = s->d_scal + j;
    I.ap = nullptr;  // the update pass forms Ap again from p (k_update_tile)
    I.st_base = st_off;
    I.rs_base = rs_off;
    rs_off += g->n_rs;
    for (int t = 0; t < g->n_st; t++) st.push_back(Item{j, t});
    st_off += g->n_st;
    hi = j + 1;
  }
  // the fast builds of the tile passes serve a batch with no grid that wraps
  bool fast = s->mode != MODE_F64 && s->coef == COEF_PACKED;
  for (int j : active) fast = fast && !s->slots[j].g->d.periodic;
  if (s->kg.fast != (fast ? 1 : 0)) {
    s->kg.fast = fast ? 1 : 0;
    *graph_stale = true;
  }
  // descriptors of slots [0, hi): the idle ones among them are never read
  if (hi > 0) {
    if (!cuda_ok(cudaMemcpyAsync(s->d_inst, sg.inst, hi * sizeof(Inst), cudaMemcpyHostToDevice,
                                 s->stream), s, "upload descriptors"))
      return false;
    s->ctx->stats->h2d += hi * sizeof(Inst);
  }
  // Largest items first: the phase kernels take items in list order, so the
  // small ones fill in at the end of each launch.  (The order changes no
  // result: each item's partial sum has a fixed place.)
  auto st_cost = [&](const Item &it) {
    const pb_grid *g = s->slots[it.inst].g;
    const int bz = it.tile / (g->tiles_x * g->tiles_y);
    return (long)g->W * g->H * (std::min(g->tz, g->d.nz - bz * g->tz) + 2);
  };
  std::stable_sort(st.begin(), st.end(),
                   [&](const Item &a, const Item &b) { return st_cost(a) > st_cost(b); });
  const double *old_rs = s->d_rs_part;
  if (!grow(&s->d_rs_part, &s->cap_rs, 2 * (size_t)std::max(rs_off, 1))) {
    s->worker_error = "out of device memory for the partial sums";
    return false;
  }
  if (s->d_rs_part != old_rs) *graph_stale = true;
  const size_t old_st = s->cap_st;
  Item *ost = s->d_st;
  if (!grow(&s->d_st, &s->cap_st, std::max<size_t>(st.size(), 1))) {
    s->worker_error = "out of device memory for the work lists";
    return false;
  }
  // partials follow the item capacity
  if (s->cap_st != old_st || s->d_st != ost) {
    cudaFree(s->d_st_part);
    s->d_st_part = nullptr;
    pb_dalloc((void **)&s->d_st_part, 2 * sizeof(double) * s->cap_st);
    *graph_stale = true;
  }
  if (!s->d_st_part) {
    s->worker_error = "out of device memory for the partial sums";
    return false;
  }
  if (!stage_items(sg, st.size())) {
    s->worker_error = "out of pinned host memory for the work lists";
    return false;
  }
  std::copy(st.begin(), st.end(), sg.items);
  sg.counts[0] = (int)st.size();
  sg.counts[1] = 0;
  if (!st.empty() && !cuda_ok(cudaMemcpyAsync(s->d_st, sg.items, st.size() * sizeof(Item),
                                              cudaMemcpyHostToDevice, s->stream), s, "items"))
    return false;
  if (!cuda_ok(cudaMemcpyAsync(s->d_counts, sg.counts, 2 * sizeof(int), cudaMemcpyHostToDevice,
                               s->stream), s, "counts"))
    return false;
  s->ctx->stats->h2d += st.size() * sizeof(Item) + 2 * sizeof(int);
  return true;
}

bool run_graph(pb_server *s, bool stale) {
  if (stale && s->graph) {
    cudaGraphExecDestroy(s->graph);
    s->graph = nullptr;
  }
  if (!s->graph) {
    Batch B;
    B.inst = s->d_inst;
    B.st_items = s->d_st;
    B.ch_items = nullptr;
    B.n_items = s->d_counts;
    B.work = (unsigned *)(s->d_counts + 4);
    B.resid_pending = s->d_counts + 2;
    B.resid_list = s->d_rlist;
    B.rs_part = s->d_rs_part;
    B.st_part = s->d_st_part;
    B.ch_part = nullptr;
    B.error = s->d_err;
    cudaGraph_t g;
    if (!cuda_ok(cudaStreamBeginCapture(s->stream, cudaStreamCaptureModeThreadLocal), s, "capture"))
      return false;
    for (int t = 0; t < s->ticks; t++) launch_tick(B, s->mode, s->coef, s->kg, s->stream);
    if (!cuda_ok(cudaStreamEndCapture(s->stream, &g), s, "capture")) return false;
    const cudaError_t e = cudaGraphInstantiate(&s->graph, g, 0);
    cudaGraphDestroy(g);
    if (!cuda_ok(e, s, "instantiate")) return false;
  }
  if (!cuda_ok(cudaGraphLaunch(s->graph, s->stream), s, "graph launch")) return false;
  s->ctx->stats->launches += 3ull * s->ticks;
  return true;
}

// Queue the energy (and phi) of the solves that finished in the previous
// round's graph, and free their slots.  The host has seen that graph finish,
// and the running graph only skips these grids (their phase is DONE), so the
// energy kernels and the device-to-host copies run on the copy stream, beside
// the running graph.  Phi is copied by the copy engine straight from the
// padded solution (a pitched copy, rows of nx of px doubles), into page-locked
// caller memory or else the round's pinned staging: no kernel, so the copy
// does not wait for SMs that the graph's persistent kernels hold.  A grid's
// next setup waits for its energy (ev_energy), its next solve for the copy of
// its phi as well (ev_idle).
// snap: the scalars the previous round's graph left; sg: this round's
// staging set (idle: its last copies were waited for).
bool queue_finished(pb_server *s, Stage &sg, const Scal *snap, const std::vector<int> &fin,
                    std::vector<Finishing> &out) {
  size_t stage_total = 0;
  for (int j : fin) {
    const Slot &sl = s->slots[j];
    if (sl.req.phi_out && !sl.req.phi_pinned)
      stage_total += (size_t)sl.g->d.nx * sl.g->d.ny * sl.g->d.nz;
  }
  if (stage_total > sg.cap_phi) {
    if (sg.phi) cudaFreeHost(sg.phi);
    sg.phi = nullptr;
    sg.cap_phi = 0;
    if (cudaMallocHost((void **)&sg.phi, stage_total * sizeof(double)) != cudaSuccess) {
      cudaGetLastError();
      s->worker_error = "out of pinned host memory for phi";
      return false;
    }
    sg.cap_phi = stage_total;
  }
  struct Copy { double *dst; const double *src; int slot; const pb_grid *g; };
  std::vector<Copy> copies;
  size_t stage_off = 0;
  for (size_t k = 0; k < fin.size(); k++) {
    Slot &sl = s->slots[fin[k]];
    pb_grid *g = sl.g;
    const Scal &S = snap[fin[k]];
    Finishing f;
    f.S = S;
    f.warm = sl.warm;
    f.energy = sg.energy + k;
    *f.energy = 0.0;
    const size_t n = (size_t)g->d.nx * g->d.ny * g->d.nz;
    const bool no_result = S.status == PB_ERR_ARG || S.status == PB_ERR_CANCELLED;
    if (!no_result && S.outer == -1 && sl.req.phi_out) {  // phi = 0, energy 0
      f.zero_phi = true;
      f.n = n;
    }
    bool copied = false;
    if (!no_result && S.outer != -1) {
      const double *x = S.xbuf ? g->x64b : g->x64;
      launch_energy(g->xyzq, g->n_atoms, g->d.nx, g->d.ny, g->d.nz, g->g.px, g->d.periodic, g->d.h,
                    g->d.origin[0], g->d.origin[1], g->d.origin[2], x,
                    g->scratch + SCR_ENERGY_PART, sg.d_energy + k, s->copy_stream);
      s->ctx->stats->launches += g->n_atoms > 0 ? 2 : 1;
      if (sl.req.phi_out) {
        if (sl.req.phi_pinned) {
          copies.push_back(Copy{sl.req.phi_out, x, fin[k], g});
        } else {
          f.phi = sg.phi + stage_off;
          f.n = n;
          stage_off += n;
          copies.push_back(Copy{f.phi, x, fin[k], g});
        }
        s->ctx->stats->d2h += n * sizeof(double);
        copied = true;
      }
    } else {
      cudaMemsetAsync(sg.d_energy + k, 0, sizeof(double), s->copy_stream);
    }
    cudaEventRecord(s->ev_energy[fin[k]], s->copy_stream);
    if (!copied) cudaEventRecord(s->ev_idle[fin[k]], s->copy_stream);
    f.req = std::move(sl.req);
    out.push_back(std::move(f));
    sl.busy = false;
    sl.stopping = false;
    sl.has_solution = S.status == PB_OK && S.outer != -1;
    sl.xbuf = S.xbuf;
    sl.last_used = ++s->clock;
    sl.solved_at = sl.last_used;
    sl.req = Request();
  }
  cudaMemcpyAsync(sg.energy, sg.d_energy, fin.size() * sizeof(double), cudaMemcpyDeviceToHost,
                  s->copy_stream);
  s->ctx->stats->d2h += fin.size() * sizeof(double);
  for (const Copy &c : copies) {
    const size_t row = (size_t)c.g->d.nx * sizeof(double);
    cudaMemcpy2DAsync(c.dst, row, c.src, (size_t)c.g->g.px * sizeof(double), row,
                      (size_t)c.g->d.ny * c.g->d.nz, cudaMemcpyDeviceToHost, s->copy_stream);
    cudaEventRecord(s->ev_idle[c.slot], s->copy_stream);  // after the copy of its phi
  }
  return cuda_ok(cudaEventRecord(sg.ev_done, s->copy_stream), s, "event");
}

// Hand out the results of finished solves (their copies have landed).
void publish(pb_server *s, std::vector<Finishing> &fin) {
  if (fin.empty()) return;
  for (auto &f : fin) {
    if (f.phi) memcpy(f.req.phi_out, f.phi, f.n * sizeof(double));
    if (f.zero_phi) memset(f.req.phi_out, 0, f.n * sizeof(double));
  }
  std::lock_guard<std::mutex> lk(s->mu);
  for (auto &f : fin) {
    const Scal &S = f.S;
    pb_result r;
    memset(&r, 0, sizeof(r));
    r.status = S.status;
    if (s->cancelled.erase(f.req.ticket)) {  // cancelled before its result was handed out
      r.status = r.info.status = PB_ERR_CANCELLED;
      r.seconds = since(f.req.t_submit);
      s->done[f.req.ticket] = r;
      s->completed++;
      continue;
    }
    r.energy = S.status == PB_ERR_ARG ? 0.0 : *f.energy;
    r.info.status = S.status;
    r.info.iterations = S.total_iter;
    r.info.outer_steps = S.outer < 0 ? 0 : S.outer;
    r.info.relres = S.relres;
    r.info.relres_true = S.outer == -1 ? 0.0 : S.relres_true;
    r.seconds = since(f.req.t_submit);
    r.warm_started = f.warm ? 1 : 0;
    s->done[f.req.ticket] = r;
    s->completed++;
  }
  fin.clear();
  s->cv_done.notify_all();
}

// Algorithmic bytes of one launch (which: 4 residual, 1 stencil, 2 update
// pass) over the active grids, from their phases.
double launch_bytes(pb_server *s, const std::vector<int> &active, int which) {
  const bool f64 = s->mode == MODE_F64;
  double b = 0;
  for (int j : active) {
    const pb_grid *g = s->slots[j].g;
    const double n = (double)g->d.nx * g->d.ny * g->d.nz;
    const int ph = s->h_scal[j].phase;
    if (which == 4) {
      if (ph == PH_RESID) b += n * 37;
    } else if (which == 1) {
      if (ph == PH_INNER || ph == PH_START) b += n * (f64 ? 41 : 21);
    } else if (ph == PH_INNER) {
      b += n * (f64 ? 25 : 13);  // p, code, z read; z written
    }
  }
  return b;
}

// Measurement ticks: each kernel on its own between events, phases read
// before each launch.
bool run_profiled(pb_server *s, const std::vector<int> &active, pb_kernel_profile &prof,
                  int ticks) {
  Batch B;
  B.inst = s->d_inst;
  B.st_items = s->d_st;
  B.ch_items = nullptr;
  B.n_items = s->d_counts;
  B.work = (unsigned *)(s->d_counts + 4);
  B.resid_pending = s->d_counts + 2;
  B.resid_list = s->d_rlist;
  B.rs_part = s->d_rs_part;
  B.st_part = s->d_st_part;
  B.ch_part = nullptr;
  B.error = s->d_err;
  const int hi = *std::max_element(active.begin(), active.end()) + 1;
  for (int t = 0; t < 3 * ticks; t++) {
    const int which = t % 3 == 0 ? 4 : t % 3 == 1 ? 1 : 2;
    cudaMemcpyAsync(s->h_scal, s->d_scal, hi * sizeof(Scal), cudaMemcpyDeviceToHost, s->stream);
    if (!cuda_ok(cudaStreamSynchronize(s->stream), s, "profile")) return false;
    const double bytes = launch_bytes(s, active, which);
    cudaEventRecord(s->ev0, s->stream);
    if (!cuda_ok(launch_phase(B, s->mode, s->coef, s->kg, which, s->stream), s, "launch"))
      return false;
    cudaEventRecord(s->ev1, s->stream);
    if (!cuda_ok(cudaEventSynchronize(s->ev1), s, "profile")) return false;
    float ms = 0;
    cudaEventElapsedTime(&ms, s->ev0, s->ev1);
    s->ctx->stats->launches += 1;
    if (which == 1 && prof.first_stencil < 64) prof.first_bytes_stencil[prof.first_stencil++] = bytes;
    if (which == 2 && prof.first_update < 64) prof.first_bytes_update[prof.first_update++] = bytes;
    if (bytes <= 0) continue;  // nothing of this kind was active
    if (which == 4) {
      prof.ms_resid += ms;
      prof.bytes_resid += bytes;
      prof.launches_resid++;
    } else if (which == 1) {
      prof.ms_stencil += ms;
      prof.bytes_stencil += bytes;
      prof.launches_stencil++;
    } else {
      prof.ms_update += ms;
      prof.bytes_update += bytes;
      prof.launches_update++;
    }
  }
  return true;
}

// The batch autotuner: time the stencil and update passes of candidate plans
// on the live batch (each applied to all active grids, two ticks each; the
// four fastest again with three ticks), keep the fastest.  Runs between
// graph launches in the worker; the solves advance during the timed ticks.
bool tune_batch(pb_server *s, Stage &sg, const std::vector<int> &active, bool *graph_stale) {
  std::vector<pb_batch_plan> cand{s->plan};
  for (int occ : {3, 2})
    for (int hp : {100, 67})
      for (int mp : {16, 32, 64, 128, 1 << 20}) {
        const pb_batch_plan c{mp, hp, occ};
        bool dup = false;
        for (const auto &x : cand)
          dup |= x.min_planes == c.min_planes && x.height_pct == c.height_pct && x.occupancy == c.occupancy;
        if (!dup) cand.push_back(c);
      }
  auto measure = [&](const pb_batch_plan &c, int ticks, double *gbs) -> bool {
    if (!cuda_ok(cudaStreamSynchronize(s->stream), s, "tune")) return false;
    s->plan = c;
    s->kg = batch_kernel_grid(s, c);
    replan_all(s);
    if (!rebuild_batch(s, sg, graph_stale)) return false;
    pb_kernel_profile p{};
    if (!run_profiled(s, active, p, ticks)) return false;
    const double ms = p.ms_stencil + p.ms_update, b = p.bytes_stencil + p.bytes_update;
    *gbs = ms > 0 ? b / ms / 1e6 : 0.0;
    return true;
  };
  std::vector<double> score(cand.size(), 0.0);
  for (size_t k = 0; k < cand.size(); k++)
    if (!measure(cand[k], 2, &score[k])) return false;
  const double first_default = score[0];
  std::vector<size_t> order(cand.size());
  for (size_t k = 0; k < order.size(); k++) order[k] = k;
  std::stable_sort(order.begin(), order.end(), [&](size_t a, size_t b) { return score[a] > score[b]; });
  // the four fastest, and the default, timed again: the kept plan is the
  // fastest of these second timings
  std::vector<size_t> again(order.begin(), order.begin() + std::min<size_t>(4, order.size()));
  if (std::find(again.begin(), again.end(), (size_t)0) == again.end()) again.push_back(0);
  size_t best = 0;
  double best_gbs = -1, default_gbs = first_default;
  for (size_t k : again) {
    double g = 0;
    if (!measure(cand[k], 3, &g)) return false;
    if (k == 0) default_gbs = g;
    if (g > best_gbs) {
      best_gbs = g;
      best = k;
    }
  }
  if (!cuda_ok(cudaStreamSynchronize(s->stream), s, "tune")) return false;
  s->plan = cand[best];
  s->kg = batch_kernel_grid(s, s->plan);
  replan_all(s);
  *graph_stale = true;
  std::lock_guard<std::mutex> lk(s->mu);
  s->tune_out.plan = s->plan;
  s->tune_out.candidates = (int)cand.size();
  s->tune_out.gbs_default = default_gbs;
  s->tune_out.gbs_best = best_gbs;
  s->plan_next = s->plan;
  s->plan_requested = false;
  s->tune_state = 2;
  s->cv_tune.notify_all();
  return true;
}

void worker_main(pb_server *s) {
  cudaSetDevice(s->ctx->device);
  bool active_changed = true, graph_stale = true;
  bool prev_graph = false;             // the previous round ran a graph: its scalars are unread
  std::vector<int> prev_active;        // ... over these slots
  std::vector<Finishing> finishing;    // results queued in the previous round
  std::vector<int> pending;            // admitted, setups not yet seen complete
  while (true) {
    {
      std::unique_lock<std::mutex> lk(s->mu);
      const bool any_busy = std::any_of(s->slots.begin(), s->slots.end(),
                                        [](const Slot &x) { return x.g && x.busy; });
      if (!any_busy && s->queue.empty() && !prev_graph && finishing.empty())
        s->cv_work.wait_for(lk, std::chrono::milliseconds(50),
                            [&] { return s->stop || !s->queue.empty(); });
      if (s->stop) break;
    }
    Stage &sg = s->stage[s->round & 1], &sp = s->stage[(s->round & 1) ^ 1];
    for (int j : admit(s)) pending.push_back(j);
    // Snapshots whose setups have completed join the batch now; the others
    // stay out of it, so the running solves never wait for a setup.  With
    // nothing else to run, wait for the oldest setup.
    std::vector<int> started;
    if (!pending.empty() && !prev_graph && finishing.empty() &&
        std::none_of(s->slots.begin(), s->slots.end(),
                     [](const Slot &x) { return x.g && x.busy && !x.pending; }))
      cudaEventSynchronize(s->ev_ready[pending.front()]);
    for (size_t k = 0; k < pending.size();) {
      const int j = pending[k];
      const cudaError_t q = cudaEventQuery(s->ev_ready[j]);
      if (q == cudaErrorNotReady) {
        k++;
        continue;
      }
      if (q != cudaSuccess) cuda_ok(q, s, "setup");
      s->slots[j].pending = false;
      s->slots[j].first_round = s->round;
      started.push_back(j);
      pending.erase(pending.begin() + k);
    }
    if (!s->worker_error.empty()) break;
    // Cancellations: a snapshot whose setup just completed does not start;
    // a running solve is stopped before this round's graph (its scalars say
    // DONE, so the phase kernels skip it and it leaves the batch as a finished
    // solve would, with no energy).
    {
      std::unordered_set<uint64_t> cx;
      {
        std::lock_guard<std::mutex> lk(s->mu);
        cx = s->cancelled;
      }
      if (!cx.empty()) {
        for (size_t k = 0; k < started.size();) {
          Slot &sl = s->slots[started[k]];
          if (cx.count(sl.req.ticket)) {
            fail_request(s, sl.req, PB_ERR_CANCELLED);
            sl.busy = false;
            sl.req = Request();
            started.erase(started.begin() + k);
          } else {
            k++;
          }
        }
        for (int j = 0; j < (int)s->slots.size(); j++) {
          Slot &sl = s->slots[j];
          if (sl.g && sl.busy && !sl.pending && !sl.stopping && cx.count(sl.req.ticket)) {
            cudaMemcpyAsync(&s->d_scal[j].phase, &s->h_stop[0], sizeof(int), cudaMemcpyHostToDevice,
                            s->stream);
            cudaMemcpyAsync(&s->d_scal[j].status, &s->h_stop[1], sizeof(int), cudaMemcpyHostToDevice,
                            s->stream);
            s->ctx->stats->h2d += 2 * sizeof(int);
            sl.stopping = true;
          }
        }
      }
    }
    if (!started.empty()) active_changed = true;
    if (active_changed) {
      // descriptors first: the start kernel reads each grid's error word and
      // ||b||^2 through its descriptor
      if (!rebuild_batch(s, sg, &graph_stale)) break;
      if (!started.empty()) {
        std::copy(started.begin(), started.end(), sg.start);
        cudaMemcpyAsync(s->d_list, sg.start, started.size() * sizeof(int), cudaMemcpyHostToDevice,
                        s->stream);
        launch_start(s->d_inst, s->d_list, (int)started.size(), s->d_counts + 2, s->d_rlist,
                     s->stream);
        s->ctx->stats->launches += 1;
        s->ctx->stats->h2d += started.size() * sizeof(int);
      }
      active_changed = false;
    }
    std::vector<int> active;
    for (int j = 0; j < (int)s->slots.size(); j++)
      if (s->slots[j].g && s->slots[j].busy && !s->slots[j].pending) active.push_back(j);
    {
      std::lock_guard<std::mutex> lk(s->mu);
      s->n_active = (int)active.size();
      s->n_resident = 0;
      s->bytes_resident = 0;
      for (auto &x : s->slots)
        if (x.g) { s->n_resident++; s->bytes_resident += x.bytes; }
    }
    // a plan set by pb_server_set_plan, or the autotuner on this batch
    bool want_plan = false, want_tune = false;
    {
      std::lock_guard<std::mutex> lk(s->mu);
      want_plan = s->plan_requested;
      want_tune = s->tune_state == 1 && !active.empty();
      if (want_plan) {
        s->plan = s->plan_next;
        s->plan_requested = false;
      }
    }
    if (want_plan) {
      if (!cuda_ok(cudaStreamSynchronize(s->stream), s, "plan")) break;
      s->kg = batch_kernel_grid(s, s->plan);
      replan_all(s);
      graph_stale = true;
      if (!active.empty() && !rebuild_batch(s, sg, &graph_stale)) break;
    }
    if (want_tune) {
      if (!tune_batch(s, sg, active, &graph_stale)) break;
      if (!rebuild_batch(s, sg, &graph_stale)) break;
    }
    bool ran = false;
    if (!active.empty()) {
      if (s->profiling.load()) {
        if (!run_profiled(s, active, s->prof, s->ticks)) break;
      } else {
        if (!run_graph(s, graph_stale)) break;
        graph_stale = false;
      }
      const int hi = *std::max_element(active.begin(), active.end()) + 1;
      cudaMemcpyAsync(sg.scal, s->d_scal, hi * sizeof(Scal), cudaMemcpyDeviceToHost, s->stream);
      cudaMemcpyAsync(sg.counts + 2, s->d_err, sizeof(int), cudaMemcpyDeviceToHost, s->stream);
      s->ctx->stats->d2h += hi * sizeof(Scal) + sizeof(int);
      if (!cuda_ok(cudaEventRecord(sg.ev_graph, s->stream), s, "event")) break;
      ran = true;
    }
    // The previous round, while this round's graph runs: hand out the results
    // queued then, and queue those of the solves its graph finished.
    if (!finishing.empty()) {
      if (!cuda_ok(cudaEventSynchronize(sp.ev_done), s, "round")) break;
      publish(s, finishing);
    }
    if (prev_graph) {
      if (!cuda_ok(cudaEventSynchronize(sp.ev_graph), s, "round")) break;
      if (sp.counts[2] & 2) {
        // A pipeline wait gave up in that graph (bounded device wait): the
        // grid whose tile was abandoned can no longer finish, and the error
        // word does not say which.  Fail every solve on the device with
        // PB_ERR_TIMEOUT, release their grids, clear the word, go on.
        if (!cuda_ok(cudaStreamSynchronize(s->stream), s, "round")) break;
        for (int j = 0; j < (int)s->slots.size(); j++) {
          Slot &sl = s->slots[j];
          if (sl.g && sl.busy && !sl.pending) {
            fail_request(s, sl.req, PB_ERR_TIMEOUT);
            evict_slot(s, j);
          }
        }
        if (!cuda_ok(cudaMemsetAsync(s->d_err, 0, 4 * sizeof(int), s->stream), s, "clear error")) break;
        active_changed = true;
        prev_graph = false;
        prev_active.clear();
        s->round++;
        continue;
      }
      std::vector<int> fin;
      for (int j : prev_active) {
        const Slot &sl = s->slots[j];
        // a pending slot's scalars are those of its previous solve
        if (sl.g && sl.busy && !sl.pending && sl.first_round < s->round &&
            sp.scal[j].phase == PH_DONE)
          fin.push_back(j);
      }
      if (!fin.empty()) {
        if (!queue_finished(s, sg, sp.scal, fin, finishing)) break;
        active_changed = true;
      }
    }
    prev_graph = ran;
    prev_active.swap(active);
    s->round++;
  }
  // hand out what was queued, fail what is left
  cudaStreamSynchronize(s->stream);
  cudaStreamSynchronize(s->copy_stream);
  publish(s, finishing);
  std::lock_guard<std::mutex> lk(s->mu);
  for (auto &rq : s->queue) {
    pb_result r;
    memset(&r, 0, sizeof(r));
    r.status = r.info.status = s->stop ? PB_ERR_BUSY : PB_ERR_CUDA;
    s->done[rq.ticket] = r;
  }
  s->queue.clear();
  for (auto &sl : s->slots)
    if (sl.g && sl.busy) {
      pb_result r;
      memset(&r, 0, sizeof(r));
      r.status = r.info.status = s->stop ? PB_ERR_BUSY : PB_ERR_CUDA;
      s->done[sl.req.ticket] = r;
      sl.busy = false;
    }
  s->stop = true;
  s->cv_done.notify_all();
  s->cv_tune.notify_all();
}

}  // namespace

// ---------------------------------------------------------------------------
// C ABI

extern "C" pb_status pb_server_create(pb_ctx *ctx, size_t budget, const pb_solve_opts *opts,
                                      pb_server **out) {
  if (!ctx || !out) return pb_fail(PB_ERR_ARG, "pb_server_create: NULL argument");
  *out = nullptr;
  pb_solve_opts o;
  if (opts) {
    o = *opts;
  } else {
    memset(&o, 0, sizeof(o));
    o.precond = PB_PRECOND_JACOBI;
    o.precision = PB_PREC_F32_REFINE;
    o.rel_tol = 1e-6;
    o.max_iter = 100000;
    o.inner_tol = 1e-3;
    o.max_outer = 20;
    o.warm_start = 1;
  }
  if (o.precision < PB_PREC_F64 || o.precision > PB_PREC_F32_REFINE || !(o.rel_tol > 0) ||
      (o.precision == PB_PREC_F32_REFINE && (!(o.inner_tol > 0) || o.max_outer < 1)))
    return pb_fail(PB_ERR_ARG, "pb_server_create: bad solve options");
  if (o.precond != PB_PRECOND_NONE && o.precond != PB_PRECOND_JACOBI)
    return pb_fail(PB_ERR_ARG, "pb_server_create: the server runs CG or Jacobi-PCG");
  if (o.precision != PB_PREC_F32_REFINE) o.max_outer = 1;
  if (o.max_iter <= 0) o.max_iter = 100000;
  if (cudaSetDevice(ctx->device) != cudaSuccess) return pb_fail(PB_ERR_CUDA, "cudaSetDevice");
  pb_server *s = new pb_server();
  s->parent = ctx;
  s->budget = budget;
  s->opts = o;
  s->mode = o.precision == PB_PREC_F64 ? MODE_F64 : o.precision == PB_PREC_F32 ? MODE_F32
                                                                                : MODE_F32_REFINE;
  s->coef = COEF_PACKED;
  s->kg = kernel_grid(s->mode, s->coef, ctx->num_sms, false);
  s->kg.tile_update = 1;
  s->slots.resize(MAX_SLOTS);
  for (int j = MAX_SLOTS - 1; j >= 0; j--) s->free_slots.push_back(j);
  bool ok = cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking) == cudaSuccess;
  // every grid of the server works on the server's stream
  s->ctx = new pb_ctx();
  s->ctx->device = ctx->device;
  s->ctx->stream = s->stream;
  s->ctx->own_stream = false;
  s->ctx->num_sms = ctx->num_sms;
  s->ctx->stats = ctx->stats;
  ok = ok && cudaMallocHost((void **)&s->ctx->host_scal, sizeof(Scal) * 64) == cudaSuccess;
  ok = ok && !pb_dalloc((void **)&s->d_scal, MAX_SLOTS * sizeof(Scal));
  ok = ok && !pb_dalloc((void **)&s->d_inst, MAX_SLOTS * sizeof(Inst));
  // item counts, residual passes pending, work counters
  ok = ok && !pb_dalloc((void **)&s->d_counts, PB_COUNTS * sizeof(int));
  ok = ok && cudaMemset(s->d_counts, 0, PB_COUNTS * sizeof(int)) == cudaSuccess;
  ok = ok && !pb_dalloc((void **)&s->d_list, MAX_SLOTS * sizeof(int));
  ok = ok && !pb_dalloc((void **)&s->d_rlist, MAX_SLOTS * sizeof(int));
  ok = ok && !pb_dalloc((void **)&s->d_err, 4 * sizeof(int));
  ok = ok && cudaMallocHost((void **)&s->h_scal, MAX_SLOTS * sizeof(Scal)) == cudaSuccess;
  ok = ok && cudaMallocHost((void **)&s->h_stop, 2 * sizeof(int)) == cudaSuccess;
  if (ok) {
    s->h_stop[0] = PH_DONE;
    s->h_stop[1] = PB_ERR_CANCELLED;
  }
  ok = ok && cudaMemset(s->d_scal, 0, MAX_SLOTS * sizeof(Scal)) == cudaSuccess;
  ok = ok && cudaMemset(s->d_err, 0, 4 * sizeof(int)) == cudaSuccess;
  ok = ok && cudaEventCreate(&s->ev0) == cudaSuccess && cudaEventCreate(&s->ev1) == cudaSuccess;
#ifndef PB_SETUP_PRIORITY
#define PB_SETUP_PRIORITY 1
#endif
#ifndef PB_COPY_PRIORITY
#define PB_COPY_PRIORITY 1
#endif
  {
    // setups first: a snapshot waiting for its setup is a slot the batch lacks;
    // and a finished solve's energy and phi copy, whose grid the trajectory's
    // next snapshot waits for (the graph's persistent kernels would otherwise
    // keep the energy kernels off the SMs until the graph ends)
    int least = 0, greatest = 0;
    cudaDeviceGetStreamPriorityRange(&least, &greatest);
    const int prio = PB_SETUP_PRIORITY ? greatest : least;
    for (auto &x : s->setup_stream)
      ok = ok && cudaStreamCreateWithPriority(&x, cudaStreamNonBlocking, prio) == cudaSuccess;
    ok = ok && cudaStreamCreateWithPriority(&s->copy_stream, cudaStreamNonBlocking,
                                            PB_COPY_PRIORITY ? greatest : least) == cudaSuccess;
  }
  s->ev_idle.assign(MAX_SLOTS, nullptr);
  s->ev_ready.assign(MAX_SLOTS, nullptr);
  s->ev_energy.assign(MAX_SLOTS, nullptr);
  for (int j = 0; ok && j < MAX_SLOTS; j++)
    ok = cudaEventCreateWithFlags(&s->ev_idle[j], cudaEventDisableTiming) == cudaSuccess &&
         cudaEventCreateWithFlags(&s->ev_ready[j], cudaEventDisableTiming) == cudaSuccess &&
         cudaEventCreateWithFlags(&s->ev_energy[j], cudaEventDisableTiming) == cudaSuccess;
  for (Stage &sg : s->stage) {
    ok = ok && cudaMallocHost((void **)&sg.inst, MAX_SLOTS * sizeof(Inst)) == cudaSuccess;
    ok = ok && cudaMallocHost((void **)&sg.counts, 4 * sizeof(int)) == cudaSuccess;
    ok = ok && cudaMallocHost((void **)&sg.start, MAX_SLOTS * sizeof(int)) == cudaSuccess;
    ok = ok && cudaMallocHost((void **)&sg.scal, MAX_SLOTS * sizeof(Scal)) == cudaSuccess;
    ok = ok && cudaMallocHost((void **)&sg.energy, MAX_SLOTS * sizeof(double)) == cudaSuccess;
    ok = ok && !pb_dalloc((void **)&sg.d_energy, MAX_SLOTS * sizeof(double));
    ok = ok && cudaEventCreateWithFlags(&sg.ev_graph, cudaEventDisableTiming) == cudaSuccess;
    ok = ok && cudaEventCreateWithFlags(&sg.ev_done, cudaEventDisableTiming) == cudaSuccess;
  }
  if (!ok) {
    pb_server_destroy(s);
    return pb_fail(PB_ERR_OOM, "pb_server_create: device allocation failed");
  }
  s->worker = std::thread(worker_main, s);
  *out = s;
  return PB_OK;
}

extern "C" pb_status pb_pinned_alloc(size_t bytes, void **out) {
  if (!out) return pb_fail(PB_ERR_ARG, "pb_pinned_alloc: NULL out");
  *out = nullptr;
  if (cudaHostAlloc(out, bytes > 0 ? bytes : 1, cudaHostAllocDefault) != cudaSuccess) {
    cudaGetLastError();
    *out = nullptr;
    return pb_fail(PB_ERR_OOM, "pb_pinned_alloc: cudaHostAlloc failed");
  }
  return PB_OK;
}

extern "C" pb_status pb_pinned_free(void *p) {
  if (p && cudaFreeHost(p) != cudaSuccess) return pb_fail(PB_ERR_CUDA, "pb_pinned_free: cudaFreeHost failed");
  return PB_OK;
}

extern "C" pb_status pb_server_destroy(pb_server *s) {
  if (!s) return PB_OK;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stop = true;
  }
  s->cv_work.notify_all();
  if (s->worker.joinable()) s->worker.join();
  cudaSetDevice(s->parent->device);
  if (s->stream) cudaStreamSynchronize(s->stream);
  if (s->copy_stream) cudaStreamSynchronize(s->copy_stream);
  for (auto x : s->setup_stream)
    if (x) cudaStreamSynchronize(x);
  for (int j = 0; j < (int)s->slots.size(); j++)
    if (s->slots[j].g) {
      s->slots[j].g->scal = nullptr;
      pb_grid_release(s->slots[j].g);
      s->slots[j].g = nullptr;
    }
  if (s->graph) cudaGraphExecDestroy(s->graph);
  void *ptrs[] = {s->d_scal, s->d_inst, s->d_counts, s->d_list, s->d_err, s->d_st,
                  s->d_st_part, s->d_rs_part, s->d_rlist};
  for (void *p : ptrs)
    if (p) cudaFree(p);
  if (s->h_scal) cudaFreeHost(s->h_scal);
  if (s->h_stop) cudaFreeHost(s->h_stop);
  for (Stage &sg : s->stage) {
    void *hp[] = {sg.inst, sg.items, sg.counts, sg.start, sg.scal, sg.energy, sg.phi};
    for (void *p : hp)
      if (p) cudaFreeHost(p);
    if (sg.d_energy) cudaFree(sg.d_energy);
    if (sg.ev_graph) cudaEventDestroy(sg.ev_graph);
    if (sg.ev_done) cudaEventDestroy(sg.ev_done);
  }
  if (s->ev0) cudaEventDestroy(s->ev0);
  if (s->ev1) cudaEventDestroy(s->ev1);
  if (s->stream) cudaStreamDestroy(s->stream);
  if (s->copy_stream) cudaStreamDestroy(s->copy_stream);
  for (auto x : s->setup_stream)
    if (x) cudaStreamDestroy(x);
  for (auto e : s->ev_idle)
    if (e) cudaEventDestroy(e);
  for (auto e : s->ev_ready)
    if (e) cudaEventDestroy(e);
  for (auto e : s->ev_energy)
    if (e) cudaEventDestroy(e);
  if (s->ctx) {
    if (s->ctx->host_scal) cudaFreeHost(s->ctx->host_scal);
    delete s->ctx;
  }
  delete s;
  return PB_OK;
}

extern "C" pb_status pb_batch_submit(pb_server *s, const pb_request *req, uint64_t *ticket) {
  if (!s || !req || !ticket) return pb_fail(PB_ERR_ARG, "pb_batch_submit: NULL argument");
  pb_status st = pb_check_desc(&req->desc);
  if (st) return st;
  if (req->desc.eps_model != PB_EPS_MIDPOINT)
    return pb_fail(PB_ERR_ARG, "pb_batch_submit: the server solves with the packed midpoint dielectric");
  if ((st = pb_check_atoms(req->n_atoms, req->xyz, req->q, req->radius))) return st;
  Request rq;
  rq.traj = req->trajectory_id < 0 ? -1 : req->trajectory_id;
  rq.desc = req->desc;
  rq.desc.coef = PB_COEF_PACKED;
  rq.xyz.assign(req->xyz, req->xyz + 3 * (size_t)req->n_atoms);
  rq.q.assign(req->q, req->q + req->n_atoms);
  rq.r.assign(req->radius, req->radius + req->n_atoms);
  rq.phi_out = req->phi_out;
  if (rq.phi_out) {
    cudaPointerAttributes pa;
    if (cudaPointerGetAttributes(&pa, rq.phi_out) == cudaSuccess)
      rq.phi_pinned = pa.type == cudaMemoryTypeHost;
    else
      cudaGetLastError();
  }
  rq.t_submit = std::chrono::steady_clock::now();
  rq.bytes = pb_grid_bytes(&rq.desc, s->opts.precision);
  if (rq.bytes > s->budget) return pb_fail(PB_ERR_ARG, "request larger than the memory budget");
  std::lock_guard<std::mutex> lk(s->mu);
  if (s->stop) return pb_fail(PB_ERR_BUSY, "server stopped: " + s->worker_error);
  if (s->queue.size() >= MAX_QUEUE) return pb_fail(PB_ERR_BUSY, "queue full");
  rq.ticket = s->next_ticket++;
  *ticket = rq.ticket;
  s->outstanding.insert(rq.ticket);
  s->queue.push_back(std::move(rq));
  s->cv_work.notify_all();
  return PB_OK;
}

extern "C" pb_status pb_batch_poll(pb_server *s, uint64_t ticket, int timeout_ms, pb_result *res) {
  if (!s || !res) return pb_fail(PB_ERR_ARG, "pb_batch_poll: NULL argument");
  std::unique_lock<std::mutex> lk(s->mu);
  if (!s->outstanding.count(ticket)) return pb_fail(PB_ERR_NOT_FOUND, "unknown or returned ticket");
  auto ready = [&] { return s->done.count(ticket) > 0; };
  if (!ready()) {
    if (timeout_ms == 0) return pb_fail(PB_ERR_TIMEOUT, "not ready");
    if (timeout_ms < 0) s->cv_done.wait(lk, [&] { return ready() || s->stop; });
    else
      s->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms),
                          [&] { return ready() || s->stop; });
    if (!ready()) {
      if (s->stop) return pb_fail(PB_ERR_CUDA, "server stopped: " + s->worker_error);
      return pb_fail(PB_ERR_TIMEOUT, "not ready");
    }
  }
  *res = s->done[ticket];
  s->done.erase(ticket);
  s->outstanding.erase(ticket);
  return PB_OK;  // a result was handed out: its own outcome is res->status
}

extern "C" pb_status pb_batch_cancel(pb_server *s, uint64_t ticket, int *cancelled) {
  if (!s) return pb_fail(PB_ERR_ARG, "pb_batch_cancel: NULL server");
  if (cancelled) *cancelled = 0;
  std::lock_guard<std::mutex> lk(s->mu);
  if (!s->outstanding.count(ticket)) return pb_fail(PB_ERR_NOT_FOUND, "unknown or returned ticket");
  if (s->done.count(ticket)) return PB_OK;  // finished already: its result stands
  s->cancelled.insert(ticket);  // the worker drops it from the queue, or stops it on the device
  if (cancelled) *cancelled = 1;
  s->cv_work.notify_all();
  return PB_OK;
}

extern "C" pb_status pb_server_stats(pb_server *s, int *queued, int *active, int *resident,
                                     size_t *bytes, uint64_t *completed) {
  if (!s) return pb_fail(PB_ERR_ARG, "pb_server_stats: NULL server");
  std::lock_guard<std::mutex> lk(s->mu);
  if (queued) *queued = (int)s->queue.size();
  if (active) *active = s->n_active;
  if (resident) *resident = s->n_resident;
  if (bytes) *bytes = s->bytes_resident;
  if (completed) *completed = s->completed;
  return PB_OK;
}

extern "C" pb_status pb_server_set_plan(pb_server *s, const pb_batch_plan *plan) {
  if (!s || !plan) return pb_fail(PB_ERR_ARG, "pb_server_set_plan: NULL argument");
  if (plan->min_planes < 1 || plan->height_pct < 1 || plan->height_pct > 100 ||
      (plan->occupancy != 2 && plan->occupancy != 3))
    return pb_fail(PB_ERR_ARG, "pb_server_set_plan: min_planes >= 1, height_pct 1..100, occupancy 2 or 3");
  std::lock_guard<std::mutex> lk(s->mu);
  s->plan_next = *plan;
  s->plan_requested = true;
  s->cv_work.notify_all();
  return PB_OK;
}

extern "C" pb_status pb_server_autotune(pb_server *s, int timeout_ms, pb_server_tune_info *out) {
  if (!s) return pb_fail(PB_ERR_ARG, "pb_server_autotune: NULL server");
  if (out) memset(out, 0, sizeof(*out));
  std::unique_lock<std::mutex> lk(s->mu);
  if (s->stop) return pb_fail(PB_ERR_CUDA, "server stopped: " + s->worker_error);
  s->tune_state = 1;
  s->cv_work.notify_all();
  auto done = [&] { return s->tune_state == 2 || s->stop; };
  if (timeout_ms < 0) s->cv_tune.wait(lk, done);
  else s->cv_tune.wait_for(lk, std::chrono::milliseconds(timeout_ms), done);
  if (s->tune_state != 2) {
    if (s->stop) return pb_fail(PB_ERR_CUDA, "server stopped: " + s->worker_error);
    return pb_fail(PB_ERR_TIMEOUT, "no batch has been tuned yet (the tuning runs once solves are active)");
  }
  if (out) *out = s->tune_out;
  s->tune_state = 0;
  return PB_OK;
}

extern "C" pb_status pb_server_profile_begin(pb_server *s) {
  if (!s) return pb_fail(PB_ERR_ARG, "pb_server_profile_begin: NULL server");
  std::lock_guard<std::mutex> lk(s->mu);
  memset(&s->prof, 0, sizeof(s->prof));
  s->profiling.store(true);
  return PB_OK;
}

extern "C" pb_status pb_server_profile_end(pb_server *s, pb_kernel_profile *out) {
  if (!s || !out) return pb_fail(PB_ERR_ARG, "pb_server_profile_end: NULL argument");
  s->profiling.store(false);
  std::lock_guard<std::mutex> lk(s->mu);
  *out = s->prof;
  return PB_OK;
}
