// Request serving for the solver (mg_submit / mg_poll).
//
// Requests (xCFC solves or div-B cleanings of any size) enter a FIFO queue.
// A fixed number of worker slots, each a host thread with its own CUDA
// stream, take them as they free up, so requests that arrive while others
// run are admitted and their kernels overlap on the device.  Hierarchies are
// cached per grid descriptor and reused; the solution of each stream id is
// kept resident on the device and used as the next initial guess of that
// stream (the paper reuses the previous time step's metric the same way,
// Sec. 4.2.1).  Device memory of cached hierarchies and resident solutions
// stays within the HBM budget given at creation: idle hierarchies, then the
// resident solutions of streams with nothing in flight, are evicted least
// recently used first; a request that still cannot fit waits for a running
// request to release memory, or fails with MG_ERR_OOM when none runs.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "mg.h"
#include "mg_internal.h"

namespace {

double now_ms() {
  using namespace std::chrono;
  return duration<double, std::milli>(steady_clock::now().time_since_epoch()).count();
}

bool desc_equal(const mg_grid_desc& a, const mg_grid_desc& b) {
  if (a.ndim != b.ndim || a.geom != b.geom || a.precision != b.precision || a.nu1 != b.nu1 ||
      a.nu2 != b.nu2 || a.max_cycles != b.max_cycles || a.tol != b.tol || a.mixed_deriv != b.mixed_deriv ||
      a.stall_window != b.stall_window || a.accel_depth != b.accel_depth || a.cycle != b.cycle ||
      a.divb_variant != b.divb_variant)
    return false;
  for (int d = 0; d < a.ndim; ++d)
    if (a.n[d] != b.n[d] || a.lo[d] != b.lo[d] || a.hi[d] != b.hi[d]) return false;
  return true;
}

long cells_of(const mg_grid_desc& d) {
  long c = 1;
  for (int k = 0; k < d.ndim; ++k) c *= d.n[k];
  return c;
}

enum { QUEUED = 0, RUNNING = 1, DONE = 2 };

struct Job {
  uint64_t ticket;
  mg_request req;
  int state = QUEUED;
  mg_result res{};
  double t_submit = 0, t_start = 0;
  cudaEvent_t ready = nullptr;   // recorded on the submitter's stream
};

struct Cached {
  mg_grid_desc desc;
  mg_hierarchy* h;
  size_t bytes;  // with the patch of AMR requests
  bool busy;
  uint64_t last;
  bool amr;      // serves AMR requests (its bytes count their patch)
};

// Resident solution of a stream id: psi, alpha, beta[3], X[3] back to back.
struct Warm {
  mg_grid_desc desc{};
  double* buf = nullptr;
  size_t bytes = 0;
  bool valid = false;
  uint64_t last = 0;  // use stamp (eviction order)
};

}  // namespace

struct mg_server {
  int device = 0;
  size_t budget = 0, used = 0;
  int slots = 1, max_queue = 1;
  std::mutex mu;
  std::condition_variable cv_work, cv_free;
  std::deque<Job*> queue;
  std::unordered_map<uint64_t, Job*> jobs;
  std::vector<Cached> cache;
  std::unordered_map<uint64_t, Warm> warm;
  std::vector<std::thread> workers;
  std::vector<cudaStream_t> streams;
  std::unordered_map<uint64_t, int> running_ids;  // stream ids with a job in flight
  int creating = 0;  // hierarchies being created (memory counted, not yet cached)
  bool stop = false;
  uint64_t next_ticket = 1, clock = 0;
};

namespace {

// Device bytes of the refined patch an AMR request adds to its hierarchy
// (five ghosted arrays of the patch and its tables; an estimate with room
// for the row padding).
size_t amr_patch_bytes(const mg_grid_desc& d, const mg_amr_arrays& a) {
  size_t cells = 1, side = 0;
  for (int k = 0; k < d.ndim; ++k) {
    const size_t m = 2 * (size_t)std::max(a.box_hi[k] - a.box_lo[k], 1) + 2 + (k == 0 ? 8 : 0);
    cells *= m;
    side += m;
  }
  return 5 * sizeof(double) * cells + 16 * sizeof(double) * side + (1 << 16);
}

// Free the resident solution of one stream id that has nothing in flight
// (own_id counts as free: its request is the caller), least recently used
// first and own_id last.  Called with the lock held; false if none.
bool evict_warm(mg_server* S, uint64_t own_id) {
  uint64_t victim = 0;
  bool found = false, victim_own = false;
  for (auto& kv : S->warm) {
    if (!kv.second.buf) continue;
    const bool own = kv.first == own_id;
    if (!own && S->running_ids[kv.first] != 0) continue;
    const bool better = !found || (victim_own && !own) ||
                        (victim_own == own && kv.second.last < S->warm[victim].last);
    if (better) {
      victim = kv.first;
      victim_own = own;
      found = true;
    }
  }
  if (!found) return false;
  Warm& w = S->warm[victim];
  cudaFree(w.buf);
  S->used -= w.bytes;
  w.buf = nullptr;
  w.bytes = 0;
  w.valid = false;
  return true;
}

// Take an idle cached hierarchy for desc, or create one within the budget
// (evicting idle hierarchies, then resident solutions of idle streams,
// least recently used first).  Called with the lock held; may release it
// while waiting or allocating.  Waits only while another request holds
// memory it will release; otherwise a request that cannot fit fails with
// MG_ERR_OOM.  Returns null on error.
mg_hierarchy* acquire(mg_server* S, std::unique_lock<std::mutex>& lk, const mg_grid_desc& d, cudaStream_t st,
                      uint64_t own_id, size_t extra, int* status) {
  size_t need = 0;
  if (mg_hierarchy_bytes(&d, &need) != MG_OK) {
    *status = MG_ERR_INVALID;
    return nullptr;
  }
  need += extra;  // the patch an AMR request adds, counted with its hierarchy
  for (;;) {
    for (Cached& c : S->cache)
      if (!c.busy && c.amr == (extra > 0) && desc_equal(c.desc, d)) {
        c.busy = true;
        gmg::hier_set_stream(c.h, st);
        return c.h;
      }
    while (S->used + need > S->budget) {
      int victim = -1;
      for (int q = 0; q < (int)S->cache.size(); ++q)
        if (!S->cache[q].busy && (victim < 0 || S->cache[q].last < S->cache[victim].last)) victim = q;
      if (victim >= 0) {
        mg_destroy_hierarchy(S->cache[victim].h);
        S->used -= S->cache[victim].bytes;
        S->cache.erase(S->cache.begin() + victim);
        continue;
      }
      if (!evict_warm(S, own_id)) break;
    }
    if (S->used + need <= S->budget) break;
    if (S->stop) {
      *status = MG_ERR_BUSY;
      return nullptr;
    }
    int holders = S->creating;
    for (const Cached& c : S->cache) holders += c.busy ? 1 : 0;
    if (holders == 0) {
      *status = gmg::set_last_error(MG_ERR_OOM,
                                    "request does not fit the HBM budget beside the resident solutions of "
                                    "running streams, and no running request will release memory");
      return nullptr;
    }
    S->cv_free.wait(lk);  // a running request will release memory
  }
  S->used += need;
  S->creating += 1;
  lk.unlock();
  mg_hierarchy* h = nullptr;
  int st2 = mg_create_hierarchy(&d, (void*)st, &h);
  lk.lock();
  S->creating -= 1;
  if (st2 != MG_OK) {
    S->used -= need;
    S->cv_free.notify_all();
    *status = st2;
    return nullptr;
  }
  gmg::hier_set_host_loop(h, true);  // concurrent slots: host cycle loops (see hier_set_host_loop)
  S->cache.push_back(Cached{d, h, need, true, S->clock++, extra > 0});
  return h;
}

void release(mg_server* S, mg_hierarchy* h) {
  for (Cached& c : S->cache)
    if (c.h == h) {
      c.busy = false;
      c.last = S->clock++;
    }
  S->cv_free.notify_all();
}

// Device copies between a request's metric fields and a resident buffer.
void copy_fields(const mg_request& r, double* buf, long n, bool to_request, cudaStream_t st) {
  double* f[8] = {r.io.psi, r.io.alpha, r.io.beta[0], r.io.beta[1], r.io.beta[2], r.io.X[0], r.io.X[1], r.io.X[2]};
  const int nf = (r.flags & MG_CFC_PSI_ONLY) ? 1 : 8;
  for (int q = 0; q < nf; ++q) {
    if (!f[q]) continue;
    if (to_request)
      cudaMemcpyAsync(f[q], buf + (long)q * n, sizeof(double) * n, cudaMemcpyDeviceToDevice, st);
    else
      cudaMemcpyAsync(buf + (long)q * n, f[q], sizeof(double) * n, cudaMemcpyDeviceToDevice, st);
  }
}

void run_job(mg_server* S, Job* J, cudaStream_t st, std::unique_lock<std::mutex>& lk) {
  const mg_request& r = J->req;
  int status = MG_OK;
  // the request's inputs were produced on the submitter's stream
  if (J->ready) cudaStreamWaitEvent(st, J->ready, 0);
  mg_hierarchy* h = acquire(S, lk, r.desc, st, r.stream_id, r.kind == MG_REQ_AMR ? amr_patch_bytes(r.desc, r.amr) : 0,
                            &status);
  if (!h) {
    J->res.status = status;
    return;
  }
  const long n = cells_of(r.desc);
  // warm start from the stream's resident solution
  Warm* w = nullptr;
  if (r.kind == MG_REQ_CFC && r.stream_id) {
    auto it = S->warm.find(r.stream_id);
    if (it != S->warm.end() && it->second.valid && desc_equal(it->second.desc, r.desc)) w = &it->second;
  }
  double* wbuf = w ? w->buf : nullptr;
  if (w) w->last = S->clock++;
  lk.unlock();
  if (wbuf) {
    copy_fields(r, wbuf, n, true, st);
    J->res.warm_started = 1;
  }
  if (r.kind == MG_REQ_CFC) {
    mg_cfc_sources src = r.src;
    mg_cfc_fields io = r.io;
    status = mg_solve_cfc(h, &src, &io, r.flags & MG_CFC_PSI_ONLY, &J->res.cfc);
  } else if (r.kind == MG_REQ_AMR) {
    const mg_amr_arrays& a = r.amr;
    status = mg_solve_scalar_amr(h, a.box_lo, a.box_hi, MG_EQ_PSI, MG_BC_ROBIN, r.src.U, a.A2, nullptr, nullptr,
                                 a.Up, a.A2p, nullptr, nullptr, a.u, a.up, &J->res.cfc.eq[1]);
  } else {
    double* B[3] = {r.B[0], r.B[1], r.B[2]};
    status = mg_clean_divB(h, B, r.phi, 0, &J->res.divb);
  }
  lk.lock();
  // keep the solution resident for the stream (within the budget)
  if (r.kind == MG_REQ_CFC && r.stream_id && status == MG_OK) {
    const size_t bytes = sizeof(double) * 8 * (size_t)n;
    Warm& ww = S->warm[r.stream_id];
    if (ww.buf && ww.bytes != bytes) {
      cudaFree(ww.buf);
      S->used -= ww.bytes;
      ww.buf = nullptr;
    }
    if (!ww.buf && S->used + bytes <= S->budget) {
      if (cudaMalloc(&ww.buf, bytes) == cudaSuccess) {
        ww.bytes = bytes;
        S->used += bytes;
      } else {
        ww.buf = nullptr;
      }
    }
    if (ww.buf) {
      ww.desc = r.desc;
      ww.last = S->clock++;
      copy_fields(r, ww.buf, n, false, st);
      cudaStreamSynchronize(st);
      ww.valid = true;
    }
  }
  release(S, h);
  J->res.status = status;
}

void worker(mg_server* S, int slot) {
  cudaSetDevice(S->device);
  cudaStream_t st = S->streams[slot];
  std::unique_lock<std::mutex> lk(S->mu);
  // first queued job whose stream id has nothing in flight (the requests of
  // one stream are solved in order, each warm-started from the previous)
  auto pick = [&]() -> std::deque<Job*>::iterator {
    for (auto it = S->queue.begin(); it != S->queue.end(); ++it) {
      const uint64_t id = (*it)->req.stream_id;
      if (id == 0 || S->running_ids[id] == 0) return it;
    }
    return S->queue.end();
  };
  for (;;) {
    S->cv_work.wait(lk, [&] { return (S->stop && S->queue.empty()) || pick() != S->queue.end(); });
    if (S->queue.empty()) return;  // stopping and drained
    auto it = pick();
    Job* J = *it;
    S->queue.erase(it);
    const uint64_t id = J->req.stream_id;
    if (id) S->running_ids[id] += 1;
    J->state = RUNNING;
    J->t_start = now_ms();
    run_job(S, J, st, lk);
    const double t = now_ms();
    J->res.latency_ms = t - J->t_submit;
    J->res.queue_ms = J->t_start - J->t_submit;
    J->state = DONE;
    if (id) S->running_ids[id] -= 1;
    S->cv_work.notify_all();
  }
}

}  // namespace

extern "C" {

int mg_server_create(size_t hbm_budget, int max_slots, int max_queue, mg_server** out) {
  if (!out || max_slots < 1 || max_slots > 64 || max_queue < 1 || hbm_budget == 0)
    return gmg::set_last_error(MG_ERR_INVALID, "need budget > 0, 1 <= max_slots <= 64, max_queue >= 1");
  mg_server* S = new (std::nothrow) mg_server();
  if (!S) return MG_ERR_OOM;
  if (cudaGetDevice(&S->device) != cudaSuccess) {
    delete S;
    return gmg::set_last_error(MG_ERR_CUDA, "no current CUDA device");
  }
  S->budget = hbm_budget;
  S->slots = max_slots;
  S->max_queue = max_queue;
  for (int q = 0; q < max_slots; ++q) {
    // non-blocking streams: concurrent with each other and never tied to
    // the legacy stream (which must not depend on a capturing stream); each
    // request waits on an event recorded on its submitter's stream
    cudaStream_t st;
    if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) {
      for (cudaStream_t s2 : S->streams) cudaStreamDestroy(s2);
      delete S;
      return gmg::set_last_error(MG_ERR_CUDA, "stream creation failed");
    }
    S->streams.push_back(st);
  }
  for (int q = 0; q < max_slots; ++q) S->workers.emplace_back(worker, S, q);
  *out = S;
  return MG_OK;
}

int mg_server_destroy(mg_server* S) {
  if (!S) return MG_OK;
  {
    std::lock_guard<std::mutex> lk(S->mu);
    S->stop = true;
    for (Job* J : S->queue) {
      J->res.status = MG_ERR_BUSY;
      J->state = DONE;
    }
    S->queue.clear();
  }
  S->cv_work.notify_all();
  S->cv_free.notify_all();
  for (std::thread& t : S->workers) t.join();
  for (Cached& c : S->cache) mg_destroy_hierarchy(c.h);
  for (auto& kv : S->warm)
    if (kv.second.buf) cudaFree(kv.second.buf);
  for (cudaStream_t st : S->streams) cudaStreamDestroy(st);
  for (auto& kv : S->jobs) {
    if (kv.second->ready) cudaEventDestroy(kv.second->ready);
    delete kv.second;
  }
  delete S;
  return MG_OK;
}

int mg_submit(mg_server* S, const mg_request* req, uint64_t* ticket) {
  if (!S || !req || !ticket) return gmg::set_last_error(MG_ERR_INVALID, "null argument");
  if (req->kind != MG_REQ_CFC && req->kind != MG_REQ_DIVB && req->kind != MG_REQ_AMR)
    return gmg::set_last_error(MG_ERR_INVALID, "bad kind");
  size_t need = 0;
  int st = mg_hierarchy_bytes(&req->desc, &need);
  if (st) return st;
  if (req->kind == MG_REQ_AMR) need += amr_patch_bytes(req->desc, req->amr);
  if (need > S->budget) return gmg::set_last_error(MG_ERR_OOM, "request larger than the server's HBM budget");
  std::lock_guard<std::mutex> lk(S->mu);
  if (S->stop) return gmg::set_last_error(MG_ERR_BUSY, "server stopping");
  if ((int)S->queue.size() >= S->max_queue) return gmg::set_last_error(MG_ERR_BUSY, "queue full");
  Job* J = new (std::nothrow) Job();
  if (!J) return MG_ERR_OOM;
  if (cudaEventCreateWithFlags(&J->ready, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventRecord(J->ready, (cudaStream_t)req->wait_stream) != cudaSuccess) {
    if (J->ready) cudaEventDestroy(J->ready);
    delete J;
    return gmg::set_last_error(MG_ERR_CUDA, "recording the request's ready event failed");
  }
  J->ticket = S->next_ticket++;
  J->req = *req;
  J->t_submit = now_ms();
  S->jobs[J->ticket] = J;
  S->queue.push_back(J);
  *ticket = J->ticket;
  S->cv_work.notify_one();
  return MG_OK;
}

int mg_poll(mg_server* S, uint64_t ticket, int* done, mg_result* out) {
  if (!S || !done) return gmg::set_last_error(MG_ERR_INVALID, "null argument");
  std::lock_guard<std::mutex> lk(S->mu);
  auto it = S->jobs.find(ticket);
  if (it == S->jobs.end()) return gmg::set_last_error(MG_ERR_NOTFOUND, "unknown or already collected ticket");
  Job* J = it->second;
  *done = J->state == DONE;
  if (!*done) return MG_OK;
  if (out) *out = J->res;
  const int status = J->res.status;
  S->jobs.erase(it);
  if (J->ready) cudaEventDestroy(J->ready);
  delete J;
  return status;
}

}  // extern "C"
