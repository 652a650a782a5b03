// Solve server: continuous batching of CG solves on one GPU.
//
// jqcd_serve_submit queues a request (thread-safe, never blocks on the GPU).
// Requests go to one of three lanes by lattice size: at most 65,536 sites
// per parity (small), at most 524,288 (medium), larger (large).  Each lane
// has its own BatchEngine, stream and scheduler thread, and loops:
//   admit queued requests while a slot is free and the device memory of all
//   slot buffers of all lanes, plus what this request adds, fits the byte
//   budget -> advance every admitted solve of the lane together by a few
//   batched iterations -> queue the reconstruction of the solves that
//   finished and the copy of x to the caller's buffer -> report the requests
//   whose copy has completed (latency recorded).
// The smaller a lane's lattices, the higher its stream priority, so the
// block scheduler starts its kernels ahead of waiting blocks of the larger
// lanes': a solve iterates at its own pace instead of in lockstep with the
// iterations of much larger ones, and the lanes' work overlaps on the GPU.  Sources and solutions move on each engine's copy stream, so with
// pinned host buffers they overlap the iterations of other requests.
// Requests that arrive while others iterate join their lane at the next
// iteration boundary; their work shares the same kernel launches (and, on
// the same gauge field, the same link loads).  Admission is FIFO per lane: a
// request that does not fit waits until earlier ones finish.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <thread>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "batch_engine.h"
#include "serve.h"

namespace jqcd {

namespace {
double wall() {
  return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}
constexpr int kItersPerStep = 8;
#ifndef JQCD_SERVE_LANES
#define JQCD_SERVE_LANES 3
#endif
constexpr int kLanes = JQCD_SERVE_LANES;
// largest sites per parity of each lane but the last: 16^3x32, then 32^3x32
constexpr int64_t kLaneMaxVhAll[2] = {65536, 524288};
constexpr const int64_t *kLaneMaxVh = kLaneMaxVhAll;

int lane_of(int64_t vh) {
  int l = 0;
  while (l < kLanes - 1 && vh > kLaneMaxVh[l]) ++l;
  return l;
}
}  // namespace

struct ServeTicket {
  jqcd_request req;
  GaugeEntry *G = nullptr;
  double t_submit = 0.0, t_admit = 0.0, t_done = 0.0;
  int state = 0;  // 0 queued, 1 running, 2 finished
  jqcd_status status = JQCD_PENDING;
  jqcd_solve_info info{};
  size_t footprint = 0;
  int slot = -1;
  int lane = 0;
};

struct ServeLane {
  cudaStream_t stream = nullptr;
  std::unique_ptr<BatchEngine> engine;
  std::thread thread;
  std::deque<uint64_t> queue;          // waiting tickets, FIFO (guarded by Server::mu)
  std::map<int, uint64_t> slot_ticket;  // engine slot -> ticket (guarded by Server::mu)
  size_t alloc = 0;  // device bytes of this lane's slot buffers, admissions in flight included
};

struct Server {
  int device = 0;
  int sm_count = 152;
  int hp = PREC_F16N;
  size_t budget = 0;
  int max_queue = 0;
  ServeLane lanes[kLanes];
  std::mutex mu;
  std::condition_variable cv;
  bool stop = false;
  double stop_deadline = 0.0;  // drain limit after stop (seconds on wall())
  bool failed = false;
  std::string error;
  uint64_t next_ticket = 1;
  std::map<uint64_t, std::unique_ptr<ServeTicket>> tickets;
  size_t peak_alloc = 0;                            // peak device bytes of slot buffers
  int peak_active = 0;
  int peak_queue = 0;                               // most requests waiting at once
  double t_first = 0.0, t_last = 0.0;
  std::vector<double> latencies;
  int64_t rejected = 0;

  size_t total_alloc() const {  // caller holds mu
    size_t a = 0;
    for (const ServeLane &L : lanes) a += L.alloc;
    return a;
  }
  int total_active() const {  // caller holds mu
    int n = 0;
    for (const ServeLane &L : lanes) n += (int)L.slot_ticket.size();
    return n;
  }
  int total_queued() const {  // caller holds mu
    int n = 0;
    for (const ServeLane &L : lanes) n += (int)L.queue.size();
    return n;
  }
  void fail(const std::string &msg) {  // caller holds mu
    failed = true;
    error = msg;
    for (auto &kv : tickets)
      if (kv.second->state != 2) {
        kv.second->state = 2;
        kv.second->status = JQCD_ECUDA;
      }
    cv.notify_all();
  }
  void loop(int lane);
};

void Server::loop(int li) {
  cudaSetDevice(device);
  ServeLane &L = lanes[li];
  BatchEngine *engine = L.engine.get();
  std::vector<int> finished;
  for (;;) {
    std::vector<std::pair<uint64_t, ServeTicket *>> admit;
    {
      std::unique_lock<std::mutex> lk(mu);
      if (failed) return;  // the other lane hit an error
      const bool idle = engine->running() == 0;
      if (idle && L.queue.empty()) {
        if (engine->draining() == 0) {
          if (stop) return;
          cv.wait_for(lk, std::chrono::milliseconds(2));
          continue;
        }
        cv.wait_for(lk, std::chrono::microseconds(200));  // results still on their way to the host
      }
      if (stop && wall() > stop_deadline) {  // drain took too long: give up
        for (auto &kv : tickets)
          if (kv.second->lane == li && kv.second->state != 2) {
            kv.second->state = 2;
            kv.second->status = JQCD_ETIMEOUT;
          }
        failed = true;
        error = "requests still running at the stop deadline";
        cv.notify_all();
        return;
      }
      // FIFO admission: a free slot and a device-memory budget that covers
      // every slot buffer of all lanes plus what this request adds
      while (!L.queue.empty()) {
        ServeTicket *T = tickets[L.queue.front()].get();
        if (T->footprint > budget) {  // can never fit
          T->state = 2;
          T->status = JQCD_ENOMEM;
          T->t_done = wall();
          ++rejected;
          L.queue.pop_front();
          continue;
        }
        int64_t extra = 0;
        int slot = engine->pick_slot(T->G->g.vh, &extra);
        if (slot < 0) break;
        if ((int64_t)total_alloc() + extra > (int64_t)budget) {
          // idle slots may be holding buffers from earlier, larger requests
          engine->release_idle(slot);
          L.alloc = engine->allocated_bytes();
          slot = engine->pick_slot(T->G->g.vh, &extra);
          if (slot < 0 || (int64_t)total_alloc() + extra > (int64_t)budget) break;
        }
        L.alloc += (size_t)extra;  // reserved until the admission has allocated it
        T->slot = slot;
        admit.push_back({L.queue.front(), T});
        L.queue.pop_front();
        break;  // one admission per pass: pick_slot sees the new slot state next time
      }
    }
    cudaError_t e = cudaSuccess;
    for (auto &a : admit) {
      ServeTicket *T = a.second;
      nvtxRangePushA(li == 0 ? "serve admit (small lane)" : li == 1 ? "serve admit (medium lane)" : "serve admit");
      e = engine->admit(T->slot, T->G, T->req.params, T->req.b);
      nvtxRangePop();
      std::lock_guard<std::mutex> lk(mu);
      L.alloc = engine->allocated_bytes();
      if (e) break;
      T->state = 1;
      T->t_admit = wall();
      L.slot_ticket[T->slot] = a.first;
      peak_alloc = std::max(peak_alloc, total_alloc());
      peak_active = std::max(peak_active, total_active());
    }
    // keep admitting while requests fit before spending time on iterations
    if (!e && !admit.empty()) {
      std::lock_guard<std::mutex> lk(mu);
      if (!L.queue.empty() && (int)L.slot_ticket.size() < engine->max_slots()) {
        int64_t extra = 0;
        const int slot = engine->pick_slot(tickets[L.queue.front()]->G->g.vh, &extra);
        if (slot >= 0 && (int64_t)total_alloc() + extra <= (int64_t)budget) continue;
      }
    }
    nvtxRangePushA(li == 0 ? "serve iterate (small lane)" : li == 1 ? "serve iterate (medium lane)" : "serve iterate");
    if (!e && engine->running() > 0) e = engine->run(kItersPerStep);
    finished.clear();
    if (!e) e = engine->poll(&finished);
    nvtxRangePop();
    // finished solves: reconstruction queued, x copied to the caller's buffer
    // on the copy stream while the other requests keep iterating
    for (int slot : finished) {
      if (e) break;
      ServeTicket *T;
      {
        std::lock_guard<std::mutex> lk(mu);
        T = tickets[L.slot_ticket[slot]].get();
      }
      e = engine->collect_async(slot, T->req.x);
    }
    // requests whose result has reached the host are done
    std::vector<std::pair<int, uint64_t>> drained;
    if (!e) {
      std::lock_guard<std::mutex> lk(mu);
      for (auto &kv : L.slot_ticket)
        if (engine->drained(kv.first)) drained.push_back(kv);
    }
    for (auto &d : drained) {
      if (e) break;
      jqcd_solve_info inf;
      engine->finish(d.first, &inf);
      std::lock_guard<std::mutex> lk(mu);
      ServeTicket *T = tickets[d.second].get();
      T->t_done = wall();
      inf.seconds = T->t_done - T->t_submit;
      T->info = inf;
      T->status = inf.status;
      T->state = 2;
      L.slot_ticket.erase(d.first);
      latencies.push_back(T->t_done - T->t_submit);
      t_last = T->t_done;
    }
    if (e) {
      std::lock_guard<std::mutex> lk(mu);
      fail(cudaGetErrorString(e));
      return;
    }
  }
}

Server *serve_create(int device, int sm_count, int hp, size_t budget, int max_slots, int max_queue,
                     std::string *err) {
  std::unique_ptr<Server> S(new Server());
  S->device = device;
  S->sm_count = sm_count;
  S->hp = hp;
  S->budget = budget;
  S->max_queue = max_queue;
  int least = 0, greatest = 0;
  cudaError_t e = cudaDeviceGetStreamPriorityRange(&least, &greatest);
  for (int li = 0; li < kLanes && !e; ++li) {
    ServeLane &L = S->lanes[li];
    // lane 0 the greatest priority, the last lane the least (numerically, greater is lower)
    const int prio = greatest + (least - greatest) * li / (kLanes - 1);
    e = cudaStreamCreateWithPriority(&L.stream, cudaStreamNonBlocking, prio);
    if (e) break;
    L.engine.reset(new BatchEngine(hp, max_slots, L.stream, sm_count));
    e = L.engine->init();
  }
  if (e) {
    *err = cudaGetErrorString(e);
    for (ServeLane &L : S->lanes) {
      L.engine.reset();
      if (L.stream) cudaStreamDestroy(L.stream);
    }
    return nullptr;
  }
  Server *raw = S.get();
  for (int li = 0; li < kLanes; ++li) S->lanes[li].thread = std::thread([raw, li] { raw->loop(li); });
  return S.release();
}

jqcd_status serve_submit(Server *S, GaugeEntry *G, const jqcd_request &r, uint64_t *ticket) {
  std::unique_ptr<ServeTicket> T(new ServeTicket());
  T->req = r;
  T->G = G;
  T->t_submit = wall();
  T->footprint = SlotBuffers::footprint(G->g.vh, S->hp);
  T->lane = lane_of(G->g.vh);
  std::lock_guard<std::mutex> lk(S->mu);
  if (S->failed) return JQCD_ECUDA;
  if (S->stop) return JQCD_EINVAL;
  if (S->max_queue > 0 && S->total_queued() >= S->max_queue) return JQCD_EBUSY;
  const uint64_t id = S->next_ticket++;
  if (S->t_first == 0.0) S->t_first = T->t_submit;
  const int lane = T->lane;
  S->tickets[id] = std::move(T);
  S->lanes[lane].queue.push_back(id);
  S->peak_queue = std::max(S->peak_queue, S->total_queued());
  *ticket = id;
  S->cv.notify_all();
  return JQCD_OK;
}

jqcd_status serve_poll(Server *S, uint64_t ticket, jqcd_solve_info *info, bool forget) {
  std::lock_guard<std::mutex> lk(S->mu);
  auto it = S->tickets.find(ticket);
  if (it == S->tickets.end()) return JQCD_ENOTFOUND;
  ServeTicket *T = it->second.get();
  if (T->state != 2) return JQCD_PENDING;
  if (info) *info = T->info;
  const jqcd_status st = T->status;
  if (forget) S->tickets.erase(it);
  return st;
}

bool serve_uses_gauge(Server *S, const GaugeEntry *G) {
  std::lock_guard<std::mutex> lk(S->mu);
  for (auto &kv : S->tickets)
    if (kv.second->G == G && kv.second->state != 2) return true;
  return false;
}

jqcd_status serve_destroy(Server *S, jqcd_serve_stats *stats, std::string *err) {
  {
    std::lock_guard<std::mutex> lk(S->mu);
    S->stop = true;
    S->stop_deadline = wall() + 300.0;
    S->cv.notify_all();
  }
  for (ServeLane &L : S->lanes)
    if (L.thread.joinable()) L.thread.join();
  jqcd_status st = S->failed ? JQCD_ECUDA : JQCD_OK;
  if (S->failed) *err = S->error;
  if (stats) {
    memset(stats, 0, sizeof *stats);
    std::vector<double> l = S->latencies;
    std::sort(l.begin(), l.end());
    auto pct = [&](double q) -> double {
      if (l.empty()) return 0.0;
      size_t k = (size_t)std::ceil(q * l.size()) - 1;
      return l[std::min(k, l.size() - 1)];
    };
    stats->completed = (int64_t)l.size();
    stats->rejected = S->rejected;
    stats->p50_s = pct(0.50);
    stats->p99_s = pct(0.99);
    double sum = 0;
    for (double v : l) sum += v;
    stats->mean_s = l.empty() ? 0.0 : sum / l.size();
    stats->wall_s = S->t_last > S->t_first ? S->t_last - S->t_first : 0.0;
    stats->solves_per_s = stats->wall_s > 0 ? l.size() / stats->wall_s : 0.0;
    stats->peak_hbm_bytes = (double)S->peak_alloc;
    stats->peak_active = S->peak_active;
    stats->peak_queue = S->peak_queue;
  }
  for (ServeLane &L : S->lanes) {
    L.engine.reset();
    if (L.stream) cudaStreamDestroy(L.stream);
  }
  delete S;
  return st;
}

}  // namespace jqcd
