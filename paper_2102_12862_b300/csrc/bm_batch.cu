// bm_batch.cu -- batches of independent states stepped by one launch per step.
//
// The launch's work list packs every member's tiles; each CTA reads its member's
// descriptor (pointers, sizes, parameters) and the CTA that completes the launch
// finalizes every member, so every member advances with its own dt.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <functional>
#include <limits>
#include <map>
#include <memory>
#include <string>
#include <vector>

#include "bm_internal.h"
#include "bm_state.h"

struct bm_batch {
  std::vector<bm_state*> members;
  std::vector<long long> epochs;  // the members' descriptor epochs the batch was made with
  int prec = BM_FP64;
  bm::DBuf<unsigned char> descs;  // member descriptors, one after another
  size_t dsz = 0;                 // bytes per descriptor
  bm::StepList list;
  // run_until: a work list of the members still running, once enough have finished
  // (a finished member's tiles would still be staged by every launch)
  std::unique_ptr<bm::StepList> sub;
  std::map<int, cudaGraphExec_t> sub_graphs;
  int sub_grid = 0;
  int shape = 0;                  // the launch shape (CTAs per SM; 0 = occupancy)
  bm::DBuf<bm::Ctl*> ctlp;        // device pointers to the members' control blocks
  bm::DBuf<double> t_end;         // per-member end times (run_until)
  bm::DBuf<int> flags;            // per member: active | status << 1
  int* hflags = nullptr;          // pinned
  cudaStream_t stream = nullptr;
  cudaStream_t own = nullptr;
  std::map<int, cudaGraphExec_t> graphs;
  int grid = 0;
  ~bm_batch() {
    for (auto& kv : graphs) cudaGraphExecDestroy(kv.second);
    for (auto& kv : sub_graphs) cudaGraphExecDestroy(kv.second);
    if (hflags) cudaFreeHost(hflags);
    if (own) cudaStreamDestroy(own);
  }
};

namespace bm {
bm_status autotune_shape(std::vector<bm_state*> states, int steps, int start_ctas, int start_static, int* best,
                         int* best_static,
                         double* best_ms, const std::function<bm_status(int, int)>& set_shape,
                         const std::function<int(int)>& grid_of,
                         const std::function<bm_status(int)>& run_steps, cudaStream_t st,
                         const std::vector<int>& slot_cands, const std::function<bm_status(int)>& set_slots,
                         int start_claim, const std::function<bm_status(int)>& set_claim);
namespace {

// Set every member's end time (+inf = plain stepping) from a device array.
__global__ void batch_set_t_end(Ctl* const* ctl, const double* t_end, int n) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n) return;
  Ctl* c = ctl[k];
  const double te = t_end[k];
  c->t_end = te;
  double dt = c->dt_cfl;
  int clipped = 0;
  if (dt >= te - c->t) {
    dt = te - c->t;
    clipped = 1;
  }
  c->dt = dt;
  c->dt_f = static_cast<float>(dt);
  c->clipped = clipped;
  c->active = c->t < te ? 1 : 0;
}

__global__ void batch_flags(Ctl* const* ctl, int n, int* flags) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k < n) flags[k] = ctl[k]->active | (ctl[k]->status << 1);
}

// One batch step: the members' own kernels before and after it (sources, species, bed
// evolution) around the one step launch, for the members of the list launched (a member
// left out of a run_until list takes no step, so its species and bed are left alone).
void launch_batch(bm_batch* b, cudaStream_t st) {
  const StepList& l = b->sub ? *b->sub : b->list;
  for (bm_state* m : l.members) state_pre_step(m, st);
  launch_work(b->prec, l, b->sub ? b->sub_grid : b->grid, 0, st);
  for (bm_state* m : l.members) state_post_step(m, st);
}

bm_status batch_graph(bm_batch* b, int k, cudaGraphExec_t* out) {
  auto& graphs = b->sub ? b->sub_graphs : b->graphs;
  auto it = graphs.find(k);
  if (it != graphs.end()) {
    *out = it->second;
    return BM_OK;
  }
  cudaGraph_t g = nullptr;
  BM_CUDA(cudaStreamBeginCapture(b->own, cudaStreamCaptureModeThreadLocal));
  for (int i = 0; i < k; ++i) launch_batch(b, b->own);
  BM_CUDA(cudaStreamEndCapture(b->own, &g));
  cudaGraphExec_t ge = nullptr;
  cudaError_t e = cudaGraphInstantiate(&ge, g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) return fail(BM_ECUDA, std::string("cudaGraphInstantiate: ") + cudaGetErrorString(e));
  graphs[k] = ge;
  *out = ge;
  return BM_OK;
}

// Drop the run_until work list (the stream must be idle).
void drop_sub(bm_batch* b) {
  for (auto& kv : b->sub_graphs) cudaGraphExecDestroy(kv.second);
  b->sub_graphs.clear();
  b->sub.reset();
}

// Step only the members whose flag (b->hflags, as batch_read left it) is active.
bm_status use_active_members(bm_batch* b) {
  std::vector<bm_state*> act;
  std::vector<const void*> dptr;
  for (size_t k = 0; k < b->members.size(); ++k)
    if (b->hflags[k] & 1) {
      act.push_back(b->members[k]);
      dptr.push_back(b->descs.p + k * b->dsz);
    }
  drop_sub(b);
  if (act.empty()) return BM_OK;
  std::unique_ptr<StepList> l(new (std::nothrow) StepList());
  if (!l) return fail(BM_ENOMEM, "bm_batch_run_until: out of host memory");
  bm_status st = build_step_list(act, dptr, l.get());
  if (st != BM_OK) return st;
  l->static16 = b->list.static16;
  l->claim = b->list.claim;
  if (b->list.slots != l->slots) {
    l->slots = b->list.slots;
    st = list_occupancy(b->prec, l.get());
    if (st != BM_OK) return st;
  }
  b->sub_grid = step_grid(*l, b->shape);
  b->sub = std::move(l);
  return BM_OK;
}

}  // namespace

bm_status batch_enqueue(bm_batch* b, int64_t n) {
  constexpr int kChunk = 16;
  if (n <= 0) return BM_OK;
  for (size_t k = 0; k < b->members.size(); ++k)
    if (b->members[k]->desc_epoch != b->epochs[k])
      return fail(BM_EINVAL, "batch: a member's features changed after bm_batch_create (make the batch again)");
  ensure_list(b->sub ? b->sub.get() : &b->list, b->stream);
  cudaGraphExec_t gbig = nullptr, gone = nullptr;
  if (n >= kChunk) {
    bm_status st = batch_graph(b, kChunk, &gbig);
    if (st != BM_OK) return st;
  }
  if (n % kChunk) {
    bm_status st = batch_graph(b, 1, &gone);
    if (st != BM_OK) return st;
  }
  for (int64_t i = 0; i < n / kChunk; ++i) BM_CUDA(cudaGraphLaunch(gbig, b->stream));
  for (int64_t i = 0; i < n % kChunk; ++i) BM_CUDA(cudaGraphLaunch(gone, b->stream));
  return BM_OK;
}

bm_status batch_set_end(bm_batch* b, const double* t_end_host) {
  const int n = static_cast<int>(b->members.size());
  std::vector<double> te(n);
  for (int k = 0; k < n; ++k) {
    te[k] = t_end_host ? t_end_host[k] : std::numeric_limits<double>::infinity();
    b->members[k]->cur_t_end = te[k];
  }
  BM_CUDA(cudaMemcpyAsync(b->t_end.p, te.data(), n * sizeof(double), cudaMemcpyHostToDevice, b->stream));
  batch_set_t_end<<<(n + 127) / 128, 128, 0, b->stream>>>(b->ctlp.p, b->t_end.p, n);
  BM_CUDA(cudaGetLastError());
  // te is a host temporary: wait for the copy before it goes out of scope
  BM_CUDA(cudaStreamSynchronize(b->stream));
  return BM_OK;
}

// Per member: active | status << 1 (synchronises the batch's stream).
bm_status batch_member_flags(bm_batch* b, std::vector<int>* flags) {
  const int n = static_cast<int>(b->members.size());
  batch_flags<<<(n + 127) / 128, 128, 0, b->stream>>>(b->ctlp.p, n, b->flags.p);
  BM_CUDA(cudaMemcpyAsync(b->hflags, b->flags.p, n * sizeof(int), cudaMemcpyDeviceToHost, b->stream));
  BM_CUDA(cudaStreamSynchronize(b->stream));
  for (int k = 0; k < n; ++k)
    if ((b->hflags[k] >> 1) & 4) b->members[k]->last_list = nullptr;  // a launch gave up
  flags->assign(b->hflags, b->hflags + n);
  return BM_OK;
}

// Read every member's active flag and status; returns the first failing status.
bm_status batch_read(bm_batch* b, int* n_active) {
  const int n = static_cast<int>(b->members.size());
  batch_flags<<<(n + 127) / 128, 128, 0, b->stream>>>(b->ctlp.p, n, b->flags.p);
  BM_CUDA(cudaMemcpyAsync(b->hflags, b->flags.p, n * sizeof(int), cudaMemcpyDeviceToHost, b->stream));
  BM_CUDA(cudaStreamSynchronize(b->stream));
  int act = 0;
  bm_status worst = BM_OK;
  for (int k = 0; k < n; ++k) {
    act += b->hflags[k] & 1;
    const int st = b->hflags[k] >> 1;
    if (st & 4) b->members[k]->last_list = nullptr;  // a launch gave up: its lists are incomplete
    if (worst == BM_OK && (st & 1)) worst = fail(BM_ENONFINITE, "batch member " + std::to_string(k) +
                                                     ": the step produced a non-finite value");
    if (worst == BM_OK && (st & 2)) worst = fail(BM_ENEGDEPTH, "batch member " + std::to_string(k) +
                                                     ": a depth fell below -h_min");
    if (worst == BM_OK && (st & 4)) worst = fail(BM_ETIMEOUT, "batch member " + std::to_string(k) +
                                                     ": a step's data copies did not arrive in time");
  }
  if (n_active) *n_active = act;
  return worst;
}

}  // namespace bm

using namespace bm;

extern "C" {

bm_status bm_batch_create(bm_state* const* states, int32_t n, bm_batch** out) {
  clear_error();
  if (!out) return fail(BM_EINVAL, "bm_batch_create: out is NULL");
  *out = nullptr;
  if (!states || n < 1) return fail(BM_EINVAL, "bm_batch_create: need at least one state");
  const int prec = states[0] ? states[0]->prec : BM_FP64;
  for (int k = 0; k < n; ++k) {
    if (!states[k]) return fail(BM_EINVAL, "bm_batch_create: NULL state");
    if (states[k]->prec != prec) return fail(BM_EINVAL, "bm_batch_create: members must share one precision");
    for (int j = 0; j < k; ++j)
      if (states[j] == states[k]) return fail(BM_EINVAL, "bm_batch_create: a state appears twice");
  }
  bm_batch* b = new (std::nothrow) bm_batch();
  if (!b) return fail(BM_ENOMEM, "bm_batch_create: out of host memory");
  b->members.assign(states, states + n);
  for (int k = 0; k < n; ++k) b->epochs.push_back(states[k]->desc_epoch);
  b->prec = prec;
  std::vector<unsigned char> all, one;
  std::vector<Ctl*> ctls(n);
  for (int k = 0; k < n; ++k) {
    bm_state* s = states[k];
    cudaStreamSynchronize(s->stream);
    state_desc_bytes(s, &one);
    all.insert(all.end(), one.begin(), one.end());
    ctls[k] = s->ctl;
  }
  const size_t dsz = one.size();  // a multiple of 16: members' descriptors stay aligned
  b->dsz = dsz;
  cudaError_t e = b->descs.upload(all);
  if (e == cudaSuccess) {
    std::vector<const void*> dptr(n);
    for (int k = 0; k < n; ++k) dptr[k] = b->descs.p + k * dsz;
    bm_status lst = build_step_list(b->members, dptr, &b->list);
    if (lst != BM_OK) {
      delete b;
      return lst;
    }
  }
  if (e == cudaSuccess) e = b->ctlp.upload(ctls);
  if (e == cudaSuccess) e = b->t_end.alloc(n);
  if (e == cudaSuccess) e = b->flags.alloc(n);
  if (e == cudaSuccess) e = cudaMallocHost(&b->hflags, n * sizeof(int));
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&b->own, cudaStreamNonBlocking);
  if (e != cudaSuccess) {
    delete b;
    return fail(e == cudaErrorMemoryAllocation ? BM_ENOMEM : BM_ECUDA,
                std::string("bm_batch_create: ") + cudaGetErrorString(e));
  }
  b->stream = b->own;
  b->grid = step_grid(b->list, 0);
  bm_status st = batch_set_end(b, nullptr);
  if (st != BM_OK) {
    delete b;
    return st;
  }
  *out = b;
  return BM_OK;
}

void bm_batch_destroy(bm_batch* b) {
  if (!b) return;
  cudaStreamSynchronize(b->stream);
  delete b;
}

bm_status bm_batch_set_stream(bm_batch* b, void* stream) {
  clear_error();
  if (!b) return fail(BM_EINVAL, "bm_batch_set_stream: batch is NULL");
  BM_CUDA(cudaStreamSynchronize(b->stream));
  b->stream = stream ? static_cast<cudaStream_t>(stream) : cudaStreamLegacy;
  return BM_OK;
}

bm_status bm_batch_set_launch(bm_batch* b, int ctas_per_sm) {
  clear_error();
  if (!b) return fail(BM_EINVAL, "bm_batch_set_launch: batch is NULL");
  if (ctas_per_sm < 0 || ctas_per_sm > 64) return fail(BM_EINVAL, "bm_batch_set_launch: ctas_per_sm in [0, 64]");
  const int grid = step_grid(b->list, ctas_per_sm);
  b->shape = ctas_per_sm;
  if (grid != b->grid) {
    BM_CUDA(cudaStreamSynchronize(b->stream));
    for (auto& kv : b->graphs) cudaGraphExecDestroy(kv.second);
    b->graphs.clear();
    b->grid = grid;
  }
  return BM_OK;
}

bm_status bm_batch_set_schedule(bm_batch* b, int ctas_per_sm, int static_sixteenths) {
  clear_error();
  if (!b) return fail(BM_EINVAL, "bm_batch_set_schedule: batch is NULL");
  if (static_sixteenths < -1 || static_sixteenths > 16)
    return fail(BM_EINVAL, "bm_batch_set_schedule: static_sixteenths in [-1, 16]");
  if (static_sixteenths != b->list.static16) {
    BM_CUDA(cudaStreamSynchronize(b->stream));
    for (auto& kv : b->graphs) cudaGraphExecDestroy(kv.second);  // they carry the old share
    b->graphs.clear();
    b->list.static16 = static_sixteenths;
  }
  return bm_batch_set_launch(b, ctas_per_sm);
}

bm_status bm_batch_set_slots(bm_batch* b, int slots) {
  clear_error();
  if (!b) return fail(BM_EINVAL, "bm_batch_set_slots: batch is NULL");
  if (slots < 2 || slots > 4) return fail(BM_EINVAL, "bm_batch_set_slots: slots in {2, 3, 4}");
  if (slots == list_slots(b->list) && b->list.slots > 0) return BM_OK;
  BM_CUDA(cudaStreamSynchronize(b->stream));
  const int keep = b->list.slots;
  b->list.slots = slots;
  bm_status st = list_occupancy(b->prec, &b->list);
  if (st != BM_OK) {  // (the layout does not fit: keep the previous count)
    b->list.slots = keep;
    (void)list_occupancy(b->prec, &b->list);
    return st;
  }
  for (auto& kv : b->graphs) cudaGraphExecDestroy(kv.second);  // they carry the old kernel
  b->graphs.clear();
  drop_sub(b);  // the run_until list is built again with the new count
  b->grid = step_grid(b->list, b->shape);
  return BM_OK;
}

bm_status bm_batch_set_claim(bm_batch* b, int mode) {
  clear_error();
  if (!b) return fail(BM_EINVAL, "bm_batch_set_claim: batch is NULL");
  if (mode < -1 || mode > 3) return fail(BM_EINVAL, "bm_batch_set_claim: mode in {-1, 0, 1, 2, 3}");
  if (mode == b->list.claim) return BM_OK;
  BM_CUDA(cudaStreamSynchronize(b->stream));
  for (auto& kv : b->graphs) cudaGraphExecDestroy(kv.second);  // they carry the old mode
  b->graphs.clear();
  drop_sub(b);
  b->list.claim = mode;
  return BM_OK;
}

bm_status bm_batch_get_claim(bm_batch* b, int* mode) {
  clear_error();
  if (!b) return fail(BM_EINVAL, "bm_batch_get_claim: batch is NULL");
  if (mode) *mode = list_claim(b->prec, b->list);
  return BM_OK;
}

bm_status bm_batch_get_slots(bm_batch* b, int* slots) {
  clear_error();
  if (!b) return fail(BM_EINVAL, "bm_batch_get_slots: batch is NULL");
  if (slots) *slots = list_slots(b->list);
  return BM_OK;
}

bm_status bm_batch_get_schedule(bm_batch* b, int* ctas_per_sm, int* static_sixteenths) {
  clear_error();
  if (!b) return fail(BM_EINVAL, "bm_batch_get_schedule: batch is NULL");
  if (ctas_per_sm) *ctas_per_sm = b->shape;
  if (static_sixteenths) *static_sixteenths = b->list.static16;
  return BM_OK;
}

bm_status bm_batch_step_async(bm_batch* b, int64_t n_steps) {
  clear_error();
  if (!b) return fail(BM_EINVAL, "bm_batch_step: batch is NULL");
  if (n_steps < 0) return fail(BM_EINVAL, "bm_batch_step: n_steps must be >= 0");
  bool reset = false;
  for (bm_state* s : b->members) reset |= std::isfinite(s->cur_t_end);
  if (reset) {
    bm_status st = batch_set_end(b, nullptr);
    if (st != BM_OK) return st;
  }
  return batch_enqueue(b, n_steps);
}

bm_status bm_batch_sync(bm_batch* b) {
  clear_error();
  if (!b) return fail(BM_EINVAL, "bm_batch_sync: batch is NULL");
  return batch_read(b, nullptr);
}

bm_status bm_batch_step(bm_batch* b, int64_t n_steps) {
  bm_status st = bm_batch_step_async(b, n_steps);
  if (st != BM_OK) return st;
  return batch_read(b, nullptr);
}

bm_status bm_batch_run_until(bm_batch* b, const double* t_end) {
  clear_error();
  if (!b) return fail(BM_EINVAL, "bm_batch_run_until: batch is NULL");
  if (!t_end) return fail(BM_EINVAL, "bm_batch_run_until: t_end is NULL");
  for (size_t k = 0; k < b->members.size(); ++k)
    if (!std::isfinite(t_end[k])) return fail(BM_EINVAL, "bm_batch_run_until: t_end must be finite");
  bm_status st = batch_set_end(b, t_end);
  if (st != BM_OK) return st;
  int active = 0;
  st = batch_read(b, &active);
  int64_t chunk = 16;
  int64_t launched = 0;
  int listed = static_cast<int>(b->members.size());  // members of the launches' work list
  while (st == BM_OK && active > 0) {
    // once a quarter of the listed members have finished, list only the running ones
    if (4 * active <= 3 * listed) {
      st = use_active_members(b);
      if (st != BM_OK) break;
      listed = active;
    }
    st = batch_enqueue(b, chunk);
    if (st != BM_OK) break;
    launched += chunk;
    st = batch_read(b, &active);
    if (chunk < 512) chunk *= 2;
    if (launched > (int64_t(1) << 40)) {
      st = fail(BM_ETIMEOUT, "bm_batch_run_until: no progress");
      break;
    }
  }
  cudaStreamSynchronize(b->stream);
  drop_sub(b);
  return st;
}

bm_status bm_batch_info(const bm_batch* b, int32_t* n_members, int64_t* n_cells, int64_t* n_tiles) {
  clear_error();
  if (!b) return fail(BM_EINVAL, "bm_batch_info: batch is NULL");
  int64_t cells = 0;
  for (bm_state* s : b->members) cells += s->mesh->h.n_cells;
  if (n_members) *n_members = static_cast<int32_t>(b->members.size());
  if (n_cells) *n_cells = cells;
  if (n_tiles) *n_tiles = static_cast<int64_t>(b->list.n);
  return BM_OK;
}

bm_status bm_batch_autotune(bm_batch* b, int steps_per_trial, int* best_ctas_per_sm, double* ms_per_step) {
  clear_error();
  if (!b) return fail(BM_EINVAL, "bm_batch_autotune: batch is NULL");
  if (steps_per_trial < 1 || steps_per_trial > 10000) return fail(BM_EINVAL, "bm_batch_autotune: steps in [1, 10000]");
  BM_CUDA(cudaStreamSynchronize(b->stream));
  std::vector<double> keep;
  bool finite = false;
  for (bm_state* s : b->members) {
    keep.push_back(s->cur_t_end);
    finite |= std::isfinite(s->cur_t_end);
  }
  if (finite) {
    bm_status st = batch_set_end(b, nullptr);
    if (st != BM_OK) return st;
  }
  bm_status st = autotune_shape(
      b->members, steps_per_trial, b->shape, b->list.static16, best_ctas_per_sm, nullptr, ms_per_step,
      [&](int c, int s16) { return bm_batch_set_schedule(b, c, s16); },
      [&](int c) { return step_grid(b->list, c); }, [&](int n) { return batch_enqueue(b, n); }, b->stream,
      slot_candidates(b->list), [&](int k) { return bm_batch_set_slots(b, k); }, list_claim(b->prec, b->list),
      [&](int m) { return bm_batch_set_claim(b, m); });
  if (st == BM_OK && finite) st = batch_set_end(b, keep.data());
  return st;
}

}  // extern "C"
