// bm_server.cu -- request loop: flood-scenario runs of different mesh sizes are
// submitted at any time, admitted while their HBM footprint fits the budget, kept
// resident, and stepped together (continuous batching: one launch per step over
// every running member, each with its own dt and end time).  Finished runs are
// copied out, their memory is freed and waiting runs are admitted in their place.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <limits>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "bm_internal.h"
#include "bm_state.h"

namespace bm {
size_t state_footprint(const bm_mesh* m, int precision);
bm_status batch_set_end(bm_batch* b, const double* t_end_host);
bm_status batch_enqueue(bm_batch* b, int64_t n);
bm_status batch_member_flags(bm_batch* b, std::vector<int>* flags);
}  // namespace bm

namespace {

using Clock = std::chrono::steady_clock;

struct Request {
  uint64_t ticket = 0;
  const bm_mesh* mesh = nullptr;
  bm_params prm{};
  std::vector<double> hydro_t, hydro_q;
  std::vector<double> H, qx, qy;  // input, then result (caller order)
  double t_end = 0.0;
  double h_arrival = -1.0;        // flood tracking threshold (< 0: no tracking)
  std::vector<double> track[5];   // the tracking record at the end (caller order)
  size_t footprint = 0;
  Clock::time_point submitted, finished;
  bm_state* state = nullptr;
  bm_status status = BM_OK;
  std::string error;
  int64_t steps = 0;
  bool done = false;
};

}  // namespace

struct bm_server {
  bm_server_opts opts{};
  std::mutex mu;
  std::condition_variable cv;
  std::deque<std::shared_ptr<Request>> queue;         // submitted, not admitted
  std::vector<std::shared_ptr<Request>> running;      // resident on the device
  std::map<uint64_t, std::shared_ptr<Request>> all;   // every ticket not yet polled
  uint64_t next_ticket = 1;
  size_t resident_bytes = 0;
  bool stop = false;
  std::thread worker;
  // statistics
  int64_t completed = 0;
  double cell_updates = 0.0;
  double busy_s = 0.0;
  int device = 0;
};

namespace {

using namespace bm;

// Device work of the server runs on the worker thread only.
void admit(bm_server* sv, std::vector<std::shared_ptr<Request>>* fresh) {
  std::unique_lock<std::mutex> lk(sv->mu);
  while (!sv->queue.empty()) {
    auto r = sv->queue.front();
    const bool fits = sv->resident_bytes + r->footprint <= sv->opts.hbm_budget_bytes;
    const bool slot = sv->opts.max_slots <= 0 ||
                      static_cast<int>(sv->running.size() + fresh->size()) < sv->opts.max_slots;
    if (!(fits && slot)) break;
    sv->queue.pop_front();
    sv->resident_bytes += r->footprint;
    fresh->push_back(r);
  }
}

void finish(bm_server* sv, const std::shared_ptr<Request>& r, bm_status st, const std::string& err) {
  if (r->state) {
    if (st == BM_OK) {
      bm_status d = bm_state_download(r->state, r->H.data(), r->qx.data(), r->qy.data(), nullptr);
      if (d == BM_OK && r->h_arrival >= 0.0) {
        for (auto& v : r->track) v.assign(r->H.size(), 0.0);
        d = bm_state_download_track(r->state, r->track[0].data(), r->track[1].data(), r->track[2].data(),
                                    r->track[3].data(), r->track[4].data());
      }
      if (d != BM_OK) {
        st = d;
      }
      int64_t steps = 0;
      bm_state_stats(r->state, nullptr, nullptr, &steps, nullptr, nullptr);
      r->steps = steps;
    }
    bm_state_destroy(r->state);
    r->state = nullptr;
  }
  std::lock_guard<std::mutex> lk(sv->mu);
  r->finished = Clock::now();
  r->status = st;
  r->error = err;
  r->done = true;
  sv->resident_bytes -= std::min(sv->resident_bytes, r->footprint);
  sv->completed += 1;
  sv->cell_updates += static_cast<double>(r->steps) * static_cast<double>(r->mesh->h.n_cells);
  sv->cv.notify_all();
}

void worker_loop(bm_server* sv) {
  cudaSetDevice(sv->device);
  cudaStream_t stream = nullptr;
  cudaStreamCreateWithFlags(&stream, cudaStreamNonBlocking);
  bm_batch* batch = nullptr;
  std::vector<bm_state*> members;
  const int rounds = std::max(1, sv->opts.steps_per_round);
  for (;;) {
    {
      std::unique_lock<std::mutex> lk(sv->mu);
      sv->cv.wait(lk, [&] { return sv->stop || !sv->queue.empty() || !sv->running.empty(); });
      if (sv->stop && sv->running.empty()) break;
      if (sv->stop) {
        // drop queued work; running members are finished below with BM_EBUSY
        for (auto& r : sv->queue) {
          r->status = BM_EBUSY;
          r->error = "server destroyed before the run was admitted";
          r->done = true;
        }
        sv->queue.clear();
      }
    }
    const auto t0 = Clock::now();
    // admit as many waiting runs as the budget allows (continuous batching)
    std::vector<std::shared_ptr<Request>> fresh;
    if (!sv->stop) admit(sv, &fresh);
    bool changed = false;
    for (auto& r : fresh) {
      bm_params p = r->prm;
      p.hydro_t = r->hydro_t.data();
      p.hydro_q = r->hydro_q.data();
      bm_state* s = nullptr;
      bm_status st = bm_state_init(r->mesh, &p, r->H.data(), r->qx.data(), r->qy.data(), &s);
      if (st == BM_OK && r->h_arrival >= 0.0) st = bm_state_track(s, r->h_arrival);
      if (st != BM_OK && s) {
        bm_state_destroy(s);
        s = nullptr;
      }
      if (st == BM_OK) {
        r->state = s;
        std::lock_guard<std::mutex> lk(sv->mu);
        sv->running.push_back(r);
        changed = true;
      } else {
        finish(sv, r, st, bm_last_error());
      }
    }
    std::vector<std::shared_ptr<Request>> run;
    {
      std::lock_guard<std::mutex> lk(sv->mu);
      run = sv->running;
    }
    if (run.empty()) continue;
    if (changed || !batch) {
      if (batch) bm_batch_destroy(batch);
      batch = nullptr;
      members.clear();
      std::vector<double> te;
      for (auto& r : run) {
        members.push_back(r->state);
        te.push_back(r->t_end);
      }
      bm_status st = bm_batch_create(members.data(), static_cast<int32_t>(members.size()), &batch);
      if (st == BM_OK) st = bm_batch_set_stream(batch, stream);
      if (st == BM_OK && sv->opts.ctas_per_sm > 0) st = bm_batch_set_launch(batch, sv->opts.ctas_per_sm);
      if (st == BM_OK) st = batch_set_end(batch, te.data());  // each member stops at its own t_end
      if (st != BM_OK) {
        const std::string err = bm_last_error();
        for (auto& r : run) finish(sv, r, st, err);
        std::lock_guard<std::mutex> lk(sv->mu);
        sv->running.clear();
        if (batch) bm_batch_destroy(batch);
        batch = nullptr;
        continue;
      }
    }
    if (sv->stop) {
      for (auto& r : run) finish(sv, r, BM_EBUSY, "server destroyed while the run was in flight");
      std::lock_guard<std::mutex> lk(sv->mu);
      sv->running.clear();
      continue;
    }
    // one round: `rounds` steps of every running member, then read their flags
    std::vector<int> flags;
    bm_status st = batch_enqueue(batch, rounds);
    if (st == BM_OK) st = batch_member_flags(batch, &flags);
    std::vector<std::shared_ptr<Request>> keep;
    bool changed_now = false;
    for (size_t k = 0; k < run.size(); ++k) {
      if (st != BM_OK) {
        finish(sv, run[k], st, bm_last_error());
        changed_now = true;
        continue;
      }
      const int f = flags[k];
      if (f >> 1) {
        const int code = f >> 1;
        finish(sv, run[k], (code & 1) ? BM_ENONFINITE : (code & 2) ? BM_ENEGDEPTH : BM_ETIMEOUT,
               (code & 1)   ? "the step produced a non-finite value"
               : (code & 2) ? "a depth fell below -h_min"
                            : "a step's data copies did not arrive in time");
        changed_now = true;
      } else if (!(f & 1)) {
        finish(sv, run[k], BM_OK, "");
        changed_now = true;
      } else {
        keep.push_back(run[k]);
      }
    }
    {
      std::lock_guard<std::mutex> lk(sv->mu);
      // runs admitted by this thread only: keep == the still-running subset of `run`
      sv->running = keep;
      sv->busy_s += std::chrono::duration<double>(Clock::now() - t0).count();
    }
    if (changed_now) {
      if (batch) bm_batch_destroy(batch);
      batch = nullptr;
    }
  }
  if (batch) bm_batch_destroy(batch);
  cudaStreamDestroy(stream);
}

}  // namespace

extern "C" {

void bm_server_opts_default(bm_server_opts* o) {
  if (!o) return;
  std::memset(o, 0, sizeof(*o));
  o->hbm_budget_bytes = 0;
  o->max_slots = 0;
  o->precision = BM_FP32_BULK;
  o->steps_per_round = 64;
  o->ctas_per_sm = 0;
}

bm_status bm_server_create(const bm_server_opts* opts, bm_server** out) {
  clear_error();
  if (!out) return fail(BM_EINVAL, "bm_server_create: out is NULL");
  *out = nullptr;
  bm_server* sv = new (std::nothrow) bm_server();
  if (!sv) return fail(BM_ENOMEM, "bm_server_create: out of host memory");
  bm_server_opts_default(&sv->opts);
  if (opts) sv->opts = *opts;
  if (sv->opts.steps_per_round <= 0) sv->opts.steps_per_round = 64;
  if (sv->opts.precision != BM_FP64 && sv->opts.precision != BM_FP32_BULK) {
    delete sv;
    return fail(BM_EINVAL, "bm_server_create: precision must be BM_FP64 or BM_FP32_BULK");
  }
  cudaGetDevice(&sv->device);
  if (sv->opts.hbm_budget_bytes == 0) {
    size_t fr = 0, tot = 0;
    cudaError_t e = cudaMemGetInfo(&fr, &tot);
    if (e != cudaSuccess) {
      delete sv;
      return fail(BM_ECUDA, std::string("bm_server_create: ") + cudaGetErrorString(e));
    }
    sv->opts.hbm_budget_bytes = static_cast<uint64_t>(0.8 * static_cast<double>(fr));
  }
  try {
    sv->worker = std::thread(worker_loop, sv);
  } catch (...) {
    delete sv;
    return fail(BM_ENOMEM, "bm_server_create: cannot start the worker thread");
  }
  *out = sv;
  return BM_OK;
}

void bm_server_destroy(bm_server* sv) {
  if (!sv) return;
  {
    std::lock_guard<std::mutex> lk(sv->mu);
    sv->stop = true;
  }
  sv->cv.notify_all();
  if (sv->worker.joinable()) sv->worker.join();
  delete sv;
}

bm_status bm_submit(bm_server* sv, const bm_mesh* mesh, const bm_params* prm, const double* H, const double* qx,
                    const double* qy, double t_end, uint64_t* ticket) {
  return bm_submit_tracked(sv, mesh, prm, H, qx, qy, t_end, -1.0, ticket);
}

bm_status bm_submit_tracked(bm_server* sv, const bm_mesh* mesh, const bm_params* prm, const double* H,
                            const double* qx, const double* qy, double t_end, double h_arrival, uint64_t* ticket) {
  clear_error();
  if (std::isnan(h_arrival) || std::isinf(h_arrival))
    return fail(BM_EINVAL, "bm_submit_tracked: h_arrival must be finite (< 0: no tracking)");
  if (!sv || !mesh || !H || !ticket) return fail(BM_EINVAL, "bm_submit: NULL argument");
  bm_status st = check_params(prm);
  if (st != BM_OK) return st;
  if (!std::isfinite(t_end) || !(t_end > 0)) return fail(BM_EINVAL, "bm_submit: t_end must be finite and > 0");
  if (prm->precision != sv->opts.precision) return fail(BM_EINVAL, "bm_submit: precision differs from the server's");
  auto r = std::make_shared<Request>();
  const size_t n = static_cast<size_t>(mesh->h.n_cells);
  r->mesh = mesh;
  r->prm = *prm;
  r->hydro_t.assign(prm->hydro_t, prm->hydro_t + prm->hydro_n);
  r->hydro_q.assign(prm->hydro_q, prm->hydro_q + prm->hydro_n);
  r->H.assign(H, H + n);
  r->qx.assign(n, 0.0);
  r->qy.assign(n, 0.0);
  if (qx) std::copy(qx, qx + n, r->qx.begin());
  if (qy) std::copy(qy, qy + n, r->qy.begin());
  r->t_end = t_end;
  r->h_arrival = h_arrival;
  r->footprint = state_footprint(mesh, prm->precision);
  if (h_arrival >= 0.0)  // the record: arrival time (double) and four maxima per padded cell
    r->footprint += static_cast<size_t>(mesh->h.n_tiles) * kTile * (8 + 4 * (prm->precision == BM_FP64 ? 8 : 4));
  r->submitted = Clock::now();
  {
    std::lock_guard<std::mutex> lk(sv->mu);
    if (sv->stop) return fail(BM_EBUSY, "bm_submit: server is shutting down");
    if (r->footprint > sv->opts.hbm_budget_bytes)
      return fail(BM_ENOMEM, "bm_submit: the run's footprint exceeds the server's HBM budget");
    r->ticket = sv->next_ticket++;
    sv->queue.push_back(r);
    sv->all[r->ticket] = r;
    *ticket = r->ticket;
  }
  sv->cv.notify_all();
  return BM_OK;
}

bm_status bm_poll(bm_server* sv, uint64_t ticket, double* H, double* qx, double* qy, double* latency_s) {
  clear_error();
  if (!sv) return fail(BM_EINVAL, "bm_poll: server is NULL");
  std::shared_ptr<Request> r;
  {
    std::lock_guard<std::mutex> lk(sv->mu);
    auto it = sv->all.find(ticket);
    if (it == sv->all.end()) return fail(BM_EINVAL, "bm_poll: unknown or already collected ticket");
    r = it->second;
    if (!r->done) return fail(BM_EAGAIN, "bm_poll: not finished yet");
    sv->all.erase(it);
  }
  if (latency_s) *latency_s = std::chrono::duration<double>(r->finished - r->submitted).count();
  if (r->status != BM_OK) return fail(r->status, "bm_poll: run failed: " + r->error);
  const size_t n = r->H.size();
  if (H) std::copy(r->H.begin(), r->H.end(), H);
  if (qx) std::copy(r->qx.begin(), r->qx.begin() + n, qx);
  if (qy) std::copy(r->qy.begin(), r->qy.begin() + n, qy);
  return BM_OK;
}

bm_status bm_poll_track(bm_server* sv, uint64_t ticket, double* t_arrival, double* h_max, double* u_max,
                        double* q_max, double* tau_max) {
  clear_error();
  if (!sv) return fail(BM_EINVAL, "bm_poll_track: server is NULL");
  std::shared_ptr<Request> r;
  {
    std::lock_guard<std::mutex> lk(sv->mu);
    auto it = sv->all.find(ticket);
    if (it == sv->all.end()) return fail(BM_EINVAL, "bm_poll_track: unknown or already collected ticket");
    r = it->second;
    if (!r->done) return fail(BM_EAGAIN, "bm_poll_track: not finished yet");
  }
  if (r->status != BM_OK) return fail(r->status, "bm_poll_track: run failed: " + r->error);
  if (r->h_arrival < 0.0) return fail(BM_EINVAL, "bm_poll_track: the run was submitted without tracking");
  double* outs[5] = {t_arrival, h_max, u_max, q_max, tau_max};
  for (int k = 0; k < 5; ++k)
    if (outs[k]) std::copy(r->track[k].begin(), r->track[k].end(), outs[k]);
  return BM_OK;
}

bm_status bm_server_wait(bm_server* sv, uint64_t ticket, double timeout_s) {
  clear_error();
  if (!sv) return fail(BM_EINVAL, "bm_server_wait: server is NULL");
  std::unique_lock<std::mutex> lk(sv->mu);
  auto it = sv->all.find(ticket);
  if (it == sv->all.end()) return fail(BM_EINVAL, "bm_server_wait: unknown or already collected ticket");
  auto r = it->second;
  const bool ok = sv->cv.wait_for(lk, std::chrono::duration<double>(timeout_s), [&] { return r->done; });
  return ok ? BM_OK : fail(BM_ETIMEOUT, "bm_server_wait: timed out");
}

bm_status bm_server_stats(bm_server* sv, int64_t* queued, int64_t* running, int64_t* completed,
                          double* cell_updates, double* resident_bytes) {
  clear_error();
  if (!sv) return fail(BM_EINVAL, "bm_server_stats: server is NULL");
  std::lock_guard<std::mutex> lk(sv->mu);
  if (queued) *queued = static_cast<int64_t>(sv->queue.size());
  if (running) *running = static_cast<int64_t>(sv->running.size());
  if (completed) *completed = sv->completed;
  if (cell_updates) *cell_updates = sv->cell_updates;
  if (resident_bytes) *resident_bytes = static_cast<double>(sv->resident_bytes);
  return BM_OK;
}

}  // extern "C"
