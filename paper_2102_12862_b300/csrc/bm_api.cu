// bm_api.cu -- the C ABI (include/bm.h): meshes and states resident in HBM, one fused
// kernel launch per step (single states and batches of uneven meshes), the step
// sequence captured in CUDA graphs, end-time targeting, checkpoint upload/download.
#include <cuda_runtime.h>

#include <algorithm>
#include <deque>
#include <functional>
#include <cmath>
#include <cstring>
#include <limits>
#include <map>
#include <mutex>
#include <sstream>
#include <string>
#include <vector>

#include "bm_internal.h"
#include "bm_kernels.cuh"
#include "bm_step.cuh"
#include "bm_species.cuh"
#include "bm_morpho.cuh"
#include "bm_state.h"

namespace bm {

static thread_local std::string g_err;

bm_status fail(bm_status st, const std::string& msg) {
  g_err = msg;
  return st;
}
void clear_error() { g_err.clear(); }
const char* last_error() { return g_err.c_str(); }

namespace {

const double kInf = std::numeric_limits<double>::infinity();

template <typename T>
std::vector<T> narrow(const std::vector<double>& v, double shift = 0.0) {
  std::vector<T> out(v.size());
  for (size_t i = 0; i < v.size(); ++i) out[i] = static_cast<T>(v[i] - shift);
  return out;
}

}  // namespace

bm_status check_params(const bm_params* p) {
  if (!p) return fail(BM_EINVAL, "bm_params is NULL");
  if (!(p->cfl > 0 && p->cfl <= 1)) return fail(BM_EINVAL, "cfl must be in (0, 1]");
  if (!(p->g > 0) || !std::isfinite(p->g)) return fail(BM_EINVAL, "g must be > 0");
  if (!(p->h_min >= 0) || !std::isfinite(p->h_min)) return fail(BM_EINVAL, "h_min must be >= 0");
  if (!(p->dt_max > 0) || !std::isfinite(p->dt_max)) return fail(BM_EINVAL, "dt_max must be > 0");
  if (p->precision != BM_FP64 && p->precision != BM_FP32_BULK)
    return fail(BM_EINVAL, "precision must be BM_FP64 or BM_FP32_BULK");
  if (p->cfl_mode != 0 && p->cfl_mode != 1) return fail(BM_EINVAL, "cfl_mode must be 0 or 1");
  if (p->hydro_n < 0 || (p->hydro_n > 0 && (!p->hydro_t || !p->hydro_q)))
    return fail(BM_EINVAL, "hydrograph arrays missing");
  if (p->hydro_n > 1000000) return fail(BM_EINVAL, "hydrograph too long");
  for (int64_t i = 0; i < p->hydro_n; ++i) {
    if (!std::isfinite(p->hydro_t[i]) || !std::isfinite(p->hydro_q[i]) || p->hydro_q[i] < 0)
      return fail(BM_EINVAL, "hydrograph values must be finite and Q >= 0");
    if (i > 0 && !(p->hydro_t[i] > p->hydro_t[i - 1]))
      return fail(BM_EINVAL, "hydrograph times must increase strictly");
  }
  return BM_OK;
}

bm_status status_of(const Ctl& c) {
  if (c.status & 1) return fail(BM_ENONFINITE, "the step produced a non-finite value");
  if (c.status & 2) return fail(BM_ENEGDEPTH, "a depth fell below -h_min");
  if (c.status & 4) return fail(BM_ETIMEOUT, "a step's data copies did not arrive in time");
  return BM_OK;
}

namespace {
// Largest dynamic shared memory of a step CTA: the device's per-block opt-in limit
// less the kernel's static shared memory (set once per kernel; above 48 KB it must
// be opted into).
template <typename T>
int step_smem_limit() {
  static int lim = [] {
    int dev = 0, optin = 48 * 1024;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    const auto kernels = {step_pipe<T, 0, 2>, step_pipe<T, 0, 3>, step_pipe<T, 0, 4>, step_pipe<T, 1, 3>,
                          step_pipe<T, 2, 3>};
    int stat = 0;  // the largest static shared memory of the instantiations
    for (auto k : kernels) {
      cudaFuncAttributes fa{};
      cudaFuncGetAttributes(&fa, k);
      stat = std::max(stat, static_cast<int>(fa.sharedSizeBytes));
    }
    const int l = optin - stat;
    bool ok = true;
    for (auto k : kernels)
      ok = ok && cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, l) == cudaSuccess &&
           cudaFuncSetAttribute(k, cudaFuncAttributePreferredSharedMemoryCarveout, 100) == cudaSuccess;
    if (!ok) {
      (void)cudaGetLastError();  // leave no sticky error behind; launches check the size
      return 48 * 1024 - stat;
    }
    return l;
  }();
  return lim;
}
int sm_count() {
  static int n = [] {
    int dev = 0, v = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev);
    return v;
  }();
  return n;
}
bm_status dev_fail(cudaError_t e, const char* what) {
  return fail(e == cudaErrorMemoryAllocation ? BM_ENOMEM : BM_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
}
}  // namespace

bm_status mesh_on_device(bm_mesh* m, int prec) {
  std::lock_guard<std::mutex> lk(m->mu);
  int dev = 0;
  BM_CUDA(cudaGetDevice(&dev));
  const HostMesh& h = m->h;
  cudaError_t e = cudaSuccess;
  if (!m->on_device) {
    e = m->z.upload(h.z);
    if (e == cudaSuccess) e = m->inv_area.upload(h.inv_area);
    if (e == cudaSuccess) e = m->area.upload(h.area);
    if (e == cudaSuccess) e = m->in_cell.upload(h.in_cell);
    if (e == cudaSuccess) e = m->in_len.upload(h.in_len);
    if (e == cudaSuccess) {
      std::vector<double> lia(h.in_len.size());
      for (size_t j = 0; j < lia.size(); ++j) lia[j] = h.in_len[j] * h.inv_area[h.in_cell[j]];
      e = m->in_lia.upload(lia);
    }
    if (e == cudaSuccess) e = m->in_nx.upload(h.in_nx);
    if (e == cudaSuccess) e = m->in_ny.upload(h.in_ny);
    if (e == cudaSuccess) e = m->btiles.upload(h.btiles);
    if (e == cudaSuccess) e = m->perm.upload(h.perm);
    if (e != cudaSuccess) return dev_fail(e, "mesh upload");
    m->device = dev;
    m->on_device = true;
  } else if (dev != m->device) {
    return fail(BM_EINVAL, "the mesh is resident on another device");
  }
  const int r = prec == BM_FP64 ? 0 : 1;
  if (r == 1 && !m->has32) {
    e = m->inv_area32.upload(narrow<float>(h.inv_area));
    if (e == cudaSuccess) e = m->in_len32.upload(narrow<float>(h.in_len));
    if (e != cudaSuccess) return dev_fail(e, "mesh upload");
    m->has32 = true;
  }
  if (!m->rec_built[r]) {
    bm_status st = build_tile_records(h, r == 0 ? 8 : 4, &m->rec[r]);
    if (st != BM_OK) return st;
    m->rec_built[r] = true;
  }
  if (!m->rec_dev[r].p) {
    e = m->rec_dev[r].upload(m->rec[r].data);
    if (e != cudaSuccess) return dev_fail(e, "tile record upload");
  }
  return BM_OK;
}

bm_status build_step_list(const std::vector<bm_state*>& members, const std::vector<const void*>& descs,
                          StepList* out) {
  const int prec = members.at(0)->prec;
  const int r = prec == BM_FP64 ? 0 : 1;
  std::vector<PipeItem> items;
  std::vector<int> fixed, first;
  uint32_t ne4 = 4, nh4 = 4;
  for (size_t k = 0; k < members.size(); ++k) {
    const bm_mesh* m = members[k]->mesh;
    const TileRecords& R = m->rec[r];
    if (!m->rec_built[r] || !m->rec_dev[r].p) return fail(BM_EINVAL, "internal: tile records missing");
    // items in tile order (a launch takes the fixed ones first); boundary ranks in tile order
    first.push_back(static_cast<int>(items.size()));
    for (int64_t t = 0, b = 0; t < m->h.n_tiles; ++t) {
      PipeItem it{};
      it.rec = m->rec_dev[r].p + R.off[t];
      it.desc = descs[k];
      it.ctl = members[k]->ctl;
      it.rec_bytes = R.bytes[t];
      it.tile = static_cast<int32_t>(t);
      it.ne_nh = R.ne_nh[t];
      it.inst = static_cast<int32_t>(k);
      it.flags = R.flags[t];
      if (!members[k]->src_tile.empty() && members[k]->src_tile[t]) it.flags |= 4u;  // source cells
      it.bidx = (R.flags[t] & 1u) ? static_cast<uint32_t>(b++) : 0u;
      if ((it.flags & kFixedFlags) || items.empty()) fixed.push_back(static_cast<int>(items.size()));
      items.push_back(it);
    }
    ne4 = std::max(ne4, R.ne4_max);
    nh4 = std::max(nh4, R.nh4_max);
  }
  cudaError_t e = out->items.upload(items);
  if (e == cudaSuccess) e = out->sched.alloc(kSchedInts);
  if (e == cudaSuccess) e = out->early.alloc(2 * items.size());
  if (e == cudaSuccess) e = out->mark.alloc(2 * items.size());
  if (e == cudaSuccess) e = out->fixed.upload(fixed);
  if (e == cudaSuccess) e = out->inst_item.upload(first);
  if (e != cudaSuccess) return dev_fail(e, "work list upload");
  out->members = members;
  out->n = static_cast<int>(items.size());
  out->n_fixed = static_cast<int>(fixed.size());
  out->ne4 = ne4;
  out->nh4 = nh4;
  for (bm_state* m : members) m->last_list = nullptr;  // the first launch resets the list
  {
    // every bulk-copy destination in a slot must be 16-byte aligned
    const StepLayout<double> l64(ne4, nh4);
    const StepLayout<float> l32(ne4, nh4);
    const uint32_t offs[] = {l64.desc, l64.ctl, l64.arr, l64.gn2, l64.slot, l32.desc, l32.ctl, l32.arr, l32.gn2,
                             l32.slot};
    for (uint32_t o : offs)
      if (o % 16u != 0u) return fail(BM_EINVAL, "internal: step layout not 16-byte aligned");
  }
  out->extra = 0;
  for (bm_state* m : members) out->extra = std::max(out->extra, state_extra_level(m));
  return list_occupancy(prec, out);
}

bool state_listed_ok(const bm_state* s) { return s->n_species == 0 && !s->morpho && !s->no_skip; }

void ensure_list(StepList* l, cudaStream_t st) {
  bool stale = false, ok = true;
  for (bm_state* m : l->members) {
    stale = stale || m->last_list != l;
    ok = ok && state_listed_ok(m);
  }
  if (!stale || l->n <= 0) return;
  const int n = std::max(l->n, kSchedInts);
  list_reset<<<(n + 255) / 256, 256, 0, st>>>(static_cast<const PipeItem*>(l->items.p), l->n, l->mark.p, l->sched.p,
                                               ok ? 1 : 0);
  for (bm_state* m : l->members) m->last_list = l;
}

int state_extra_level(const bm_state* s) {
  const HostMesh& h = s->mesh->h;
  const bool outflow =
      (h.n_hq > 0 && s->hq_n > 0) || (h.n_weir > 0 && s->weir_mu > 0.0) || (h.n_level > 0 && s->zh_n > 0);
  if (s->n_src > 0 || s->fr_law != 0 || outflow) return 2;
  const bool trk = s->prec == BM_FP64 ? s->b64.trk_t.p != nullptr : s->b32.trk_t.p != nullptr;
  return (trk || s->n_species > 0) ? 1 : 0;
}

// The tile slots a list's step kernel runs with: the count asked for (by default 2,
// measured with items claimed when a slot frees) at the plain level, 3 at the
// optional-feature levels (built for that count only).
constexpr int kDefaultSlots = 2;
int list_slots(const StepList& l) { return l.extra == 0 ? (l.slots > 0 ? l.slots : kDefaultSlots) : 3; }

// Work-item claiming of a list's launches: by default a CTA claims each item once its
// slot is free, so it commits to no more tiles than its slots hold and none it would
// reach late while others run dry (the launch's end is set by its last tile); FP64,
// whose wet tiles take 20-35 us, also waits until the tile before is past its edge
// phase, so a CTA commits to its next tile only near the end of the current one.
// Measured over the floodplain run against the other modes in both precisions.
int list_claim(int prec, const StepList& l) { return l.claim >= 0 ? l.claim : (prec == BM_FP64 ? 3 : 2); }

// The slot counts the autotuner tries for a list: the one in force first.
std::vector<int> slot_candidates(const StepList& l) {
  std::vector<int> k{list_slots(l)};
  if (l.extra == 0)
    for (int c : {2, 3, 4})
      if (c != k[0]) k.push_back(c);
  return k;
}

// The step kernel of a feature level and slot count.
template <typename T>
auto step_kernel(int level, int slots) {
  if (level >= 2) return step_pipe<T, 2, 3>;
  if (level == 1) return step_pipe<T, 1, 3>;
  return slots == 2 ? step_pipe<T, 0, 2> : (slots == 4 ? step_pipe<T, 0, 4> : step_pipe<T, 0, 3>);
}

template <typename T>
size_t step_smem(const StepList& l) {
  const int k = list_slots(l);
  if (k == 2) return StepLayout<T, 2>(l.ne4, l.nh4).total;
  if (k == 4) return StepLayout<T, 4>(l.ne4, l.nh4).total;
  return StepLayout<T, 3>(l.ne4, l.nh4).total;
}

// The list's shared memory per CTA (its largest tile layout at its slot count) and
// resident CTAs per SM of its kernel.
bm_status list_occupancy(int prec, StepList* l) {
  l->smem = prec == BM_FP64 ? step_smem<double>(*l) : step_smem<float>(*l);
  const int lim = prec == BM_FP64 ? step_smem_limit<double>() : step_smem_limit<float>();
  if (l->smem > static_cast<size_t>(lim)) return fail(BM_EINVAL, "tile layout exceeds the device's shared memory");
  int occ = 0;
  cudaError_t e;
  if (prec == BM_FP64)
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(
        &occ, step_kernel<double>(l->extra, list_slots(*l)), kStepThreads, l->smem);
  else
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(
        &occ, step_kernel<float>(l->extra, list_slots(*l)), kStepThreads, l->smem);
  if (e != cudaSuccess) return dev_fail(e, "occupancy query");
  l->occupancy = std::max(1, occ);
  return BM_OK;
}

// CTAs of a step launch: all resident at once (a share of the tiles is assigned to
// CTAs statically, so a CTA that waited for another to exit would finish late).
int step_grid(const StepList& l, int ctas_per_sm) {
  const int per = ctas_per_sm > 0 ? std::min(ctas_per_sm, l.occupancy) : l.occupancy;
  const long long g = static_cast<long long>(per) * sm_count();
  return static_cast<int>(std::max(1LL, std::min<long long>(g, l.n)));
}

// One fused step (or prime) launch over a work list.
// Launched as a programmatic dependent of the previous kernel in the stream: its CTAs
// may start while that kernel's last CTAs finish and wait (griddepcontrol.wait) before
// touching anything the previous kernel writes.
void launch_work(int prec, const StepList& l, int grid, int prime, cudaStream_t st, int withhold) {
  if (l.n <= 0) return;
  grid = std::max(1, std::min(grid, l.n));
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(static_cast<unsigned>(grid));
  cfg.blockDim = dim3(kStepThreads);
  cfg.dynamicSmemBytes = l.smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  ListArgs a;
  a.items = static_cast<const PipeItem*>(l.items.p);
  a.n_items = l.n;
  a.sched = l.sched.p;
  a.early = l.early.p;
  a.mark = l.mark.p;
  a.fixed = l.fixed.p;
  a.n_fixed = l.n_fixed;
  a.inst_item = l.inst_item.p;
  a.n_inst = static_cast<int>(l.members.size());
  a.ne4max = static_cast<int>(l.ne4);
  a.nh4max = static_cast<int>(l.nh4);
  a.lazy = list_claim(prec, l);
  if (prec == BM_FP64)
    (void)cudaLaunchKernelEx(&cfg, step_kernel<double>(l.extra, list_slots(l)), a, prime, withhold, l.static16);
  else
    (void)cudaLaunchKernelEx(&cfg, step_kernel<float>(l.extra, list_slots(l)), a, prime, withhold, l.static16);
}

namespace {

bm_status read_status(bm_state* s) {
  BM_CUDA(cudaMemcpyAsync(s->hctl, s->ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, s->stream));
  BM_CUDA(cudaStreamSynchronize(s->stream));
  if (s->hctl->status & 4) s->last_list = nullptr;  // a launch gave up: its lists are incomplete
  return status_of(*s->hctl);
}

// The species kernel after a step: one CTA per tile of the state's work list.
template <typename T>
void launch_species(bm_state* s, cudaStream_t st) {
  Buffers<T>& b = s->buf<T>();
  const TileRecords& R = s->mesh->rec[sizeof(T) == 8 ? 0 : 1];
  const size_t np = static_cast<size_t>(s->mesh->h.n_tiles) * kTile;
  SpeciesArgs<T> a{};
  a.items = static_cast<const PipeItem*>(s->list.items.p);
  for (int c = 0; c < s->n_species; ++c) {
    a.hc[c][0] = b.hc[0].p + c * np;
    a.hc[c][1] = b.hc[1].p + c * np;
    a.c_in[c] = static_cast<T>(s->c_in[c]);
  }
  for (int k = 0; k < 2; ++k) {
    a.H[k] = b.H[k].p;
    a.Hlo[k] = b.Hlo[k].p;
  }
  a.z = b.z.p;
  a.ctl = s->ctl;
  a.ex_flux = b.ex_flux.p;
  a.ex_right = b.ex_right.p;
  a.ex_valid = b.ex_valid.p;
  a.ex_dt = b.ex_dt.p;
  a.zmask = b.zmask.p;
  a.ex_stride = static_cast<int>(R.ne4_max);
  a.n_species = s->n_species;
  a.n_inflow = static_cast<int>(s->mesh->h.n_inflow);
  a.n_level0 = static_cast<int>(s->mesh->h.n_inflow + s->mesh->h.n_hq + s->mesh->h.n_weir);
  a.n_cells = static_cast<int>(s->mesh->h.n_cells);
  const int nloc = kTile + static_cast<int>(R.nh4_max);
  const size_t smem = (2 * static_cast<size_t>(nloc) + R.ne4_max) * sizeof(T);
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(static_cast<unsigned>(s->list.n));
  cfg.blockDim = dim3(kTile);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  (void)cudaLaunchKernelEx(&cfg, species_step<T>, a, nloc);
}

// The bed update after a step (and after the species, which read z^n).
void launch_morpho(bm_state* s, cudaStream_t st) {
  const TileRecords& R = s->mesh->rec[0];
  MorphoArgs a{};
  a.items = static_cast<const PipeItem*>(s->list.items.p);
  for (int k = 0; k < 2; ++k) {
    a.H[k] = s->b64.H[k].p;
    a.qx[k] = s->b64.qx[k].p;
    a.qy[k] = s->b64.qy[k].p;
  }
  a.z = s->b64.z.p;
  a.gn2 = s->b64.gn2.p;
  a.ctl = s->ctl;
  a.step_dt = s->mo_dt.p;
  a.dz = s->mo_dz.p;
  const double* q = s->mo_par;
  a.mp = MorphoParams{q[0], q[1], q[2], q[3], q[4], q[5], 1.0 / s->p.g, 1.0 / ((q[1] - 1.0) * q[2]),
                      std::sqrt((q[1] - 1.0) * s->p.g * q[2] * q[2] * q[2]), 1.0 / (1.0 - q[0])};
  a.g = s->p.g;
  a.h_min = s->p.h_min;
  a.n_cells = static_cast<int>(s->mesh->h.n_cells);
  const int nloc = kTile + static_cast<int>(R.nh4_max);
  const size_t smem = (8 * static_cast<size_t>(nloc) + R.ne4_max) * sizeof(double);
  morpho_flux<<<s->list.n, kTile, smem, st>>>(a, nloc);
  const int nb = (a.n_cells + 255) / 256;
  morpho_apply<<<nb, 256, 0, st>>>(s->mo_dz.p, s->mo_dt.p, s->ctl, s->b64.z.p, s->b64.H[0].p, s->b64.H[1].p,
                                   a.n_cells);
}

void pre_step(bm_state* s, cudaStream_t st) {
  if (s->morpho) morpho_save_dt<<<1, 32, 0, st>>>(s->ctl, s->mo_dt.p);
  if (s->n_src > 0) {
    if (s->prec == BM_FP64)
      source_rates<double><<<1, 128, 0, st>>>(s->ctl, s->n_src, s->src_kind.p, s->src_off.p, s->src_t.p, s->src_v.p,
                                               s->src_area.p, s->src_rate64.p);
    else
      source_rates<float><<<1, 128, 0, st>>>(s->ctl, s->n_src, s->src_kind.p, s->src_off.p, s->src_t.p, s->src_v.p,
                                              s->src_area.p, s->src_rate32.p);
  }
}

void post_step(bm_state* s, cudaStream_t st) {
  if (s->n_species > 0) {
    if (s->prec == BM_FP64) launch_species<double>(s, st);
    else launch_species<float>(s, st);
  }
  if (s->morpho) launch_morpho(s, st);
}

void launch_state(bm_state* s, cudaStream_t st, int prime) {
  if (prime) ensure_list(&s->list, st);  // (prime launches are never captured)
  if (!prime) pre_step(s, st);
  launch_work(s->prec, s->list, s->grid, prime, st);
  if (!prime) post_step(s, st);
}

bm_status get_graph(bm_state* s, int k, cudaGraphExec_t* out) {
  auto it = s->graphs.find(k);
  if (it != s->graphs.end()) {
    *out = it->second;
    return BM_OK;
  }
  cudaGraph_t g = nullptr;
  BM_CUDA(cudaStreamBeginCapture(s->own, cudaStreamCaptureModeThreadLocal));
  for (int i = 0; i < k; ++i) launch_state(s, s->own, 0);
  BM_CUDA(cudaStreamEndCapture(s->own, &g));
  cudaGraphExec_t ge = nullptr;
  cudaError_t e = cudaGraphInstantiate(&ge, g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) return fail(BM_ECUDA, std::string("cudaGraphInstantiate: ") + cudaGetErrorString(e));
  s->graphs[k] = ge;
  *out = ge;
  return BM_OK;
}

void drop_graphs(bm_state* s) {
  for (auto& kv : s->graphs) cudaGraphExecDestroy(kv.second);
  s->graphs.clear();
}

// Enqueue n steps as graph launches of 32 steps plus single-step launches.
bm_status enqueue_steps(bm_state* s, int64_t n) {
  constexpr int kChunk = 32;
  if (n <= 0) return BM_OK;
  ensure_list(&s->list, s->stream);
  cudaGraphExec_t gbig = nullptr, gone = nullptr;
  if (n >= kChunk) {
    bm_status st = get_graph(s, kChunk, &gbig);
    if (st != BM_OK) return st;
  }
  if (n % kChunk) {
    bm_status st = get_graph(s, 1, &gone);
    if (st != BM_OK) return st;
  }
  for (int64_t i = 0; i < n / kChunk; ++i) BM_CUDA(cudaGraphLaunch(gbig, s->stream));
  for (int64_t i = 0; i < n % kChunk; ++i) BM_CUDA(cudaGraphLaunch(gone, s->stream));
  return BM_OK;
}

bm_status set_end(bm_state* s, double t_end) {
  set_t_end<<<1, 1, 0, s->stream>>>(s->ctl, t_end);
  BM_CUDA(cudaGetLastError());
  s->cur_t_end = t_end;
  return BM_OK;
}

template <typename T>
void fill_desc(bm_state* s, InstDesc<T>& d) {
  const bm_mesh* m = s->mesh;
  const HostMesh& h = m->h;
  std::memset(&d, 0, sizeof(d));
  Buffers<T>& b = s->buf<T>();
  for (int k = 0; k < 2; ++k) {
    d.H[k] = b.H[k].p; d.Hlo[k] = b.Hlo[k].p; d.qx[k] = b.qx[k].p; d.qy[k] = b.qy[k].p;
  }
  d.z = b.z.p;
  d.gn2 = b.gn2.p;
  if (b.trk_t.p) {
    d.trk_t = b.trk_t.p;
    d.trk_h = b.trk[0].p;
    d.trk_u = b.trk[1].p;
    d.trk_q = b.trk[2].p;
    d.trk_tau = b.trk[3].p;
    d.trk_harr = static_cast<T>(s->trk_harr);
  }
  if (s->n_species > 0) {
    d.ex_flux = b.ex_flux.p;
    d.ex_right = b.ex_right.p;
    d.ex_valid = b.ex_valid.p;
    d.ex_dt = b.ex_dt.p;
    d.ex_stride = static_cast<int>(m->rec[sizeof(T) == 8 ? 0 : 1].ne4_max);
  }
  d.fr_law = s->fr_law;
  if (s->n_src > 0) {
    d.src_reg = s->src_reg.p;
    d.src_mode = s->src_mode.p;
    if constexpr (sizeof(T) == 8) d.src_rate = s->src_rate64.p;
    else d.src_rate = s->src_rate32.p;
  }
  d.in_pw = b.in_pw.p;
  d.in_hs = b.in_hs.p;
  if constexpr (sizeof(T) == 8) {
    d.inv_area = m->inv_area.p;
    d.in_len = m->in_len.p;
  } else {
    d.inv_area = m->inv_area32.p;
    d.in_len = m->in_len32.p;
  }
  d.in_cell = m->in_cell.p;
  d.in_lia = m->in_lia.p;
  d.in_nx = m->in_nx.p;
  d.in_ny = m->in_ny.p;
  d.btiles = m->btiles.p;
  d.ctl = s->ctl;
  d.part = s->part.p;
  d.p = s->p;
  d.inflow_len = h.inflow_len;
  d.n_inflow = static_cast<int>(h.n_inflow);
  d.n_btiles = static_cast<int>(h.btiles.size());
  {
    const TileRecords& R = m->rec[sizeof(T) == 8 ? 0 : 1];
    int nit = 0, nhq = 0;
    for (uint8_t f : R.flags) {
      nit += (f & 2u) ? 1 : 0;
      nhq += (f & 8u) ? 1 : 0;
    }
    d.n_in_tiles = nit;
    d.n_hq_tiles = nhq;
  }
  d.n_hq = static_cast<int>(h.n_hq);
  d.n_weir = static_cast<int>(h.n_weir);
  d.hq_n = s->hq_n;
  d.hq_s = s->hq_s.p;
  d.hq_q = s->hq_q.p;
  d.datum = s->prec == BM_FP64 ? 0.0 : s->datum;
  d.weir_crest = static_cast<T>(s->weir_crest - d.datum);
  d.weir_k = static_cast<T>(2.0 / 3.0 * s->weir_mu * std::sqrt(2.0 * s->prm.g));
  d.n_level = static_cast<int>(h.n_level);
  d.zh_n = s->zh_n;
  d.zh_t = s->zh_t.p;
  d.zh_v = s->zh_v.p;
  d.n_cells = static_cast<int>(h.n_cells);
  d.n_tiles = static_cast<int>(h.n_tiles);
}

}  // namespace

void state_pre_step(bm_state* s, cudaStream_t st) { pre_step(s, st); }
void state_post_step(bm_state* s, cudaStream_t st) { post_step(s, st); }

// Host copy of a state's descriptor (for batches).
void state_desc_bytes(bm_state* s, std::vector<unsigned char>* out) {
  if (s->prec == BM_FP64) {
    InstDesc<double> d;
    fill_desc<double>(s, d);
    out->assign(reinterpret_cast<unsigned char*>(&d), reinterpret_cast<unsigned char*>(&d) + sizeof(d));
  } else {
    InstDesc<float> d;
    fill_desc<float>(s, d);
    out->assign(reinterpret_cast<unsigned char*>(&d), reinterpret_cast<unsigned char*>(&d) + sizeof(d));
  }
}

// Load caller-order arrays into state buffer 0, validate, reset time and prime dt.
bm_status load_state(bm_state* s, const double* H, const double* qx, const double* qy, double t) {
  const HostMesh& h = s->mesh->h;
  const int n = static_cast<int>(h.n_cells);
  if (!H) return fail(BM_EINVAL, "H is NULL");
  if (!std::isfinite(t)) return fail(BM_EINVAL, "t must be finite");
  const size_t bytes = static_cast<size_t>(n) * sizeof(double);
  BM_CUDA(cudaMemcpyAsync(s->stage[0].p, H, bytes, cudaMemcpyHostToDevice, s->stream));
  if (qx) BM_CUDA(cudaMemcpyAsync(s->stage[1].p, qx, bytes, cudaMemcpyHostToDevice, s->stream));
  else BM_CUDA(cudaMemsetAsync(s->stage[1].p, 0, bytes, s->stream));
  if (qy) BM_CUDA(cudaMemcpyAsync(s->stage[2].p, qy, bytes, cudaMemcpyHostToDevice, s->stream));
  else BM_CUDA(cudaMemsetAsync(s->stage[2].p, 0, bytes, s->stream));
  const int nb = (n + 255) / 256;
  const int32_t* perm = s->mesh->perm.p;
  BM_CUDA(cudaMemsetAsync(s->bad.p, 0, sizeof(int), s->stream));
  // a fresh scheduling state (a launch that gave up may have left it inconsistent; the
  // new state's tiles all need a step)
  s->last_list = nullptr;
  if (s->prec == BM_FP64) {
    Buffers<double>& b = s->b64;
    gather_from_user<double><<<nb, 256, 0, s->stream>>>(s->stage[0].p, perm, n, b.H[0].p);
    gather_from_user<double><<<nb, 256, 0, s->stream>>>(s->stage[1].p, perm, n, b.qx[0].p);
    gather_from_user<double><<<nb, 256, 0, s->stream>>>(s->stage[2].p, perm, n, b.qy[0].p);
    check_state<double><<<nb, 256, 0, s->stream>>>(b.H[0].p, b.qx[0].p, b.qy[0].p, b.z.p, n, s->bad.p);
  } else {
    Buffers<float>& b = s->b32;
    gather_surface_pair<<<nb, 256, 0, s->stream>>>(s->stage[0].p, perm, n, s->mesh->z.p, b.z.p, s->datum, b.H[0].p,
                                                   b.Hlo[0].p, s->bad.p);
    gather_from_user<float><<<nb, 256, 0, s->stream>>>(s->stage[1].p, perm, n, b.qx[0].p);
    gather_from_user<float><<<nb, 256, 0, s->stream>>>(s->stage[2].p, perm, n, b.qy[0].p);
    check_state<float><<<nb, 256, 0, s->stream>>>(nullptr, b.qx[0].p, b.qy[0].p, b.z.p, n, s->bad.p);
  }
  BM_CUDA(cudaMemcpyAsync(s->hbad, s->bad.p, sizeof(int), cudaMemcpyDeviceToHost, s->stream));
  BM_CUDA(cudaStreamSynchronize(s->stream));
  if (*s->hbad & 1) return fail(BM_EINVAL, "state has a non-finite value");
  if (*s->hbad & 2) return fail(BM_EINVAL, "state has H < z_bed (a dry cell is H = z_bed)");
  Ctl c;
  std::memset(&c, 0, sizeof(c));
  c.t = t;
  c.t_end = kInf;
  c.active = 1;
  BM_CUDA(cudaMemcpyAsync(s->ctl, &c, sizeof(Ctl), cudaMemcpyHostToDevice, s->stream));
  s->cur_t_end = kInf;
  launch_state(s, s->stream, 1);
  BM_CUDA(cudaGetLastError());
  BM_CUDA(cudaStreamSynchronize(s->stream));
  return BM_OK;
}

// Allocate the device arrays of a state and upload its per-cell constants.
bm_status alloc_state(bm_state* s, const bm_params* prm) {
  const bm_mesh* m = s->mesh;
  const HostMesh& h = m->h;
  const size_t Np = static_cast<size_t>(h.n_tiles) * kTile;
  const bool f64 = s->prec == BM_FP64;
  s->datum = f64 ? 0.0 : (std::isnan(prm->datum) ? h.z_min : prm->datum);
  if (!std::isfinite(s->datum)) return fail(BM_EINVAL, "bm_state_init: datum must be finite or NaN");
  std::vector<double> gn2(h.man.size());
  for (size_t i = 0; i < gn2.size(); ++i) gn2[i] = prm->g * h.man[i] * h.man[i];
  bm_status mst = mesh_on_device(const_cast<bm_mesh*>(m), s->prec);
  if (mst != BM_OK) return mst;
  cudaError_t e = cudaSuccess;
  if (f64) {
    e = s->b64.alloc(Np, h.in_cell.size(), false);
    if (e == cudaSuccess) e = s->b64.gn2.upload(gn2);
    if (e == cudaSuccess) e = cudaMemcpy(s->b64.z.p, h.z.data(), Np * sizeof(double), cudaMemcpyHostToDevice);
  } else {
    e = s->b32.alloc(Np, h.in_cell.size(), true);
    if (e == cudaSuccess) e = s->b32.gn2.upload(narrow<float>(gn2));
    if (e == cudaSuccess) {
      std::vector<float> z32 = narrow<float>(h.z, s->datum);
      e = cudaMemcpy(s->b32.z.p, z32.data(), Np * sizeof(float), cudaMemcpyHostToDevice);
    }
  }
  for (int k = 0; k < 3 && e == cudaSuccess; ++k) e = s->stage[k].alloc(h.n_cells);
  if (e == cudaSuccess) e = s->part.alloc(h.n_tiles);
  if (e == cudaSuccess) e = cudaMemset(s->part.p, 0, h.n_tiles * sizeof(TilePartial));
  if (e == cudaSuccess) e = s->vol_part.alloc(h.n_tiles);
  if (e == cudaSuccess) e = s->vol_out.alloc(1);
  if (e == cudaSuccess) e = s->bad.alloc(1);
  if (e == cudaSuccess) e = s->d_hydro_t.upload(s->hydro_t);
  if (e == cudaSuccess) e = s->d_hydro_q.upload(s->hydro_q);
  if (e == cudaSuccess) e = cudaMalloc(&s->ctl, sizeof(Ctl));
  if (e == cudaSuccess) e = cudaMallocHost(&s->hctl, sizeof(Ctl));
  if (e == cudaSuccess) e = cudaMallocHost(&s->hvol, sizeof(double));
  if (e == cudaSuccess) e = cudaMallocHost(&s->hbad, sizeof(int));
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s->own, cudaStreamNonBlocking);
  if (e != cudaSuccess) {
    if (e == cudaErrorMemoryAllocation) return fail(BM_ENOMEM, "bm_state_init: out of device memory");
    return fail(BM_ECUDA, std::string("bm_state_init: ") + cudaGetErrorString(e));
  }
  s->stream = s->own;
  Params& p = s->p;
  p.cfl = prm->cfl;
  p.g = prm->g;
  p.h_min = prm->h_min;
  p.dt_max = prm->dt_max;
  p.cfl_mode = prm->cfl_mode;
  p.hydro_n = static_cast<int>(prm->hydro_n);
  p.hydro_t = s->d_hydro_t.p;
  p.hydro_q = s->d_hydro_q.p;
  p.g_f = static_cast<float>(prm->g);
  p.hg_f = static_cast<float>(0.5 * prm->g);
  p.hmin_f = static_cast<float>(prm->h_min);
  p.pad_f = 0.0f;
  state_desc_bytes(s, &s->hdesc);
  ++s->desc_epoch;  // (a batch made before this no longer describes the state)
  e = s->desc.upload(s->hdesc);
  if (e != cudaSuccess) return dev_fail(e, "bm_state_init");
  bm_status lst = build_step_list({s}, {static_cast<const void*>(s->desc.p)}, &s->list);
  if (lst != BM_OK) return lst;
  s->grid = step_grid(s->list, 0);
  return BM_OK;
}

// Device bytes held by a state (its admission footprint).
size_t state_footprint(const bm_mesh* m, int precision) {
  const HostMesh& h = m->h;
  const size_t Np = static_cast<size_t>(h.n_tiles) * kTile;
  const size_t w = precision == BM_FP64 ? 8 : 4;
  const size_t arrays = precision == BM_FP64 ? 8 : 10;  // 2 x (H [pair], q) + z, gn2
  // + caller-order staging, per tile: boundary partial, volume partial, work item
  return Np * w * arrays + 3 * static_cast<size_t>(h.n_cells) * 8 + static_cast<size_t>(h.n_tiles) * 72 +
         h.in_cell.size() * 2 * w + 4096;
}

}  // namespace bm

using namespace bm;

extern "C" {

void bm_params_default(bm_params* p) {
  if (!p) return;
  std::memset(p, 0, sizeof(*p));
  p->cfl = 0.9;
  p->g = 9.81;
  p->h_min = 1e-6;
  p->dt_max = 1.0;
  p->precision = BM_FP64;
  p->cfl_mode = 0;
  p->datum = std::numeric_limits<double>::quiet_NaN();
  p->hydro_t = nullptr;
  p->hydro_q = nullptr;
  p->hydro_n = 0;
}

const char* bm_last_error(void) { return last_error(); }

bm_status bm_mesh_create(const double* xy, int64_t n_nodes, const int32_t* tri, int64_t n_tri, const double* z_bed,
                         const double* manning_n, const uint8_t* edge_tag, bm_mesh** out) {
  clear_error();
  if (!out) return fail(BM_EINVAL, "bm_mesh_create: out is NULL");
  *out = nullptr;
  bm_mesh* m = new (std::nothrow) bm_mesh();
  if (!m) return fail(BM_ENOMEM, "bm_mesh_create: out of host memory");
  bm_status st;
  try {
    st = prepare_mesh(xy, n_nodes, tri, n_tri, z_bed, manning_n, edge_tag, &m->h);
  } catch (const std::bad_alloc&) {
    st = fail(BM_ENOMEM, "bm_mesh_create: out of host memory");
  }
  if (st != BM_OK) {
    delete m;
    return st;
  }
  *out = m;
  return BM_OK;
}

bm_status bm_mesh_info(const bm_mesh* m, int64_t* n_cells, int64_t* n_edges, int64_t* n_boundary,
                       int64_t* n_inflow, int64_t* n_tiles) {
  clear_error();
  if (!m) return fail(BM_EINVAL, "bm_mesh_info: mesh is NULL");
  if (n_cells) *n_cells = m->h.n_cells;
  if (n_edges) *n_edges = m->h.n_edges;
  if (n_boundary) *n_boundary = m->h.n_boundary;
  if (n_inflow) *n_inflow = m->h.n_inflow;
  if (n_tiles) *n_tiles = m->h.n_tiles;
  return BM_OK;
}

void bm_mesh_destroy(bm_mesh* m) { delete m; }

bm_status bm_mesh_layout(const bm_mesh* cm, int32_t precision, int64_t* max_tile_edges, int64_t* max_tile_halo,
                         int64_t* record_bytes) {
  clear_error();
  if (!cm) return fail(BM_EINVAL, "bm_mesh_layout: mesh is NULL");
  if (precision != BM_FP64 && precision != BM_FP32_BULK)
    return fail(BM_EINVAL, "bm_mesh_layout: precision must be BM_FP64 or BM_FP32_BULK");
  bm_mesh* m = const_cast<bm_mesh*>(cm);
  std::lock_guard<std::mutex> lk(m->mu);
  const int r = precision == BM_FP64 ? 0 : 1;
  if (!m->rec_built[r]) {
    bm_status st = build_tile_records(m->h, r == 0 ? 8 : 4, &m->rec[r]);
    if (st != BM_OK) return st;
    m->rec_built[r] = true;
  }
  const TileRecords& R = m->rec[r];
  uint32_t ne = 0, nh = 0;
  for (uint32_t v : R.ne_nh) {
    ne = std::max(ne, v & 0xffffu);
    nh = std::max(nh, v >> 16);
  }
  if (max_tile_edges) *max_tile_edges = ne;
  if (max_tile_halo) *max_tile_halo = nh;
  if (record_bytes) *record_bytes = static_cast<int64_t>(R.data.size());
  return BM_OK;
}

bm_status bm_state_init(const bm_mesh* m, const bm_params* prm, const double* H, const double* qx, const double* qy,
                        bm_state** out) {
  clear_error();
  if (!out) return fail(BM_EINVAL, "bm_state_init: out is NULL");
  *out = nullptr;
  if (!m) return fail(BM_EINVAL, "bm_state_init: mesh is NULL");
  bm_status st = check_params(prm);
  if (st != BM_OK) return st;
  bm_state* s = new (std::nothrow) bm_state();
  if (!s) return fail(BM_ENOMEM, "bm_state_init: out of host memory");
  s->mesh = m;
  s->prm = *prm;
  s->prec = prm->precision;
  s->hydro_t.assign(prm->hydro_t, prm->hydro_t + prm->hydro_n);
  s->hydro_q.assign(prm->hydro_q, prm->hydro_q + prm->hydro_n);
  s->prm.hydro_t = s->hydro_t.data();
  s->prm.hydro_q = s->hydro_q.data();
  st = alloc_state(s, prm);
  if (st == BM_OK) st = load_state(s, H, qx, qy, 0.0);
  if (st != BM_OK) {
    delete s;
    return st;
  }
  *out = s;
  return BM_OK;
}

void bm_state_destroy(bm_state* s) {
  if (!s) return;
  cudaStreamSynchronize(s->stream);
  delete s;
}

bm_status bm_state_set_stream(bm_state* s, void* stream) {
  clear_error();
  if (!s) return fail(BM_EINVAL, "bm_state_set_stream: state is NULL");
  BM_CUDA(cudaStreamSynchronize(s->stream));
  s->stream = stream ? static_cast<cudaStream_t>(stream) : cudaStreamLegacy;
  return BM_OK;
}

bm_status bm_state_set_launch(bm_state* s, int ctas_per_sm) {
  clear_error();
  if (!s) return fail(BM_EINVAL, "bm_state_set_launch: state is NULL");
  if (ctas_per_sm < 0 || ctas_per_sm > 64) return fail(BM_EINVAL, "bm_state_set_launch: ctas_per_sm in [0, 64]");
  const int grid = step_grid(s->list, ctas_per_sm);
  s->ctas_per_sm = ctas_per_sm;
  if (grid != s->grid) {
    BM_CUDA(cudaStreamSynchronize(s->stream));
    drop_graphs(s);
    s->grid = grid;
  }
  return BM_OK;
}

bm_status bm_state_set_schedule(bm_state* s, int ctas_per_sm, int static_sixteenths) {
  clear_error();
  if (!s) return fail(BM_EINVAL, "bm_state_set_schedule: state is NULL");
  if (static_sixteenths < -1 || static_sixteenths > 16)
    return fail(BM_EINVAL, "bm_state_set_schedule: static_sixteenths in [-1, 16]");
  if (static_sixteenths != s->list.static16) {
    BM_CUDA(cudaStreamSynchronize(s->stream));
    drop_graphs(s);  // the captured launches carry the old share
    s->list.static16 = static_sixteenths;
  }
  return bm_state_set_launch(s, ctas_per_sm);
}

bm_status bm_state_set_slots(bm_state* s, int slots) {
  clear_error();
  if (!s) return fail(BM_EINVAL, "bm_state_set_slots: state is NULL");
  if (slots < 2 || slots > 4) return fail(BM_EINVAL, "bm_state_set_slots: slots in {2, 3, 4}");
  if (slots == list_slots(s->list) && s->list.slots > 0) return BM_OK;
  BM_CUDA(cudaStreamSynchronize(s->stream));
  const int keep = s->list.slots;
  s->list.slots = slots;
  bm_status st = list_occupancy(s->prec, &s->list);
  if (st != BM_OK) {  // (the layout does not fit: keep the previous count)
    s->list.slots = keep;
    (void)list_occupancy(s->prec, &s->list);
    return st;
  }
  drop_graphs(s);  // the captured launches carry the old kernel
  s->grid = step_grid(s->list, s->ctas_per_sm);
  return BM_OK;
}

bm_status bm_state_set_claim(bm_state* s, int mode) {
  clear_error();
  if (!s) return fail(BM_EINVAL, "bm_state_set_claim: state is NULL");
  if (mode < -1 || mode > 3) return fail(BM_EINVAL, "bm_state_set_claim: mode in {-1, 0, 1, 2, 3}");
  if (mode == s->list.claim) return BM_OK;
  BM_CUDA(cudaStreamSynchronize(s->stream));
  drop_graphs(s);  // the captured launches carry the old mode
  s->list.claim = mode;
  return BM_OK;
}

bm_status bm_state_get_claim(bm_state* s, int* mode) {
  clear_error();
  if (!s) return fail(BM_EINVAL, "bm_state_get_claim: state is NULL");
  if (mode) *mode = list_claim(s->prec, s->list);
  return BM_OK;
}

bm_status bm_state_get_slots(bm_state* s, int* slots) {
  clear_error();
  if (!s) return fail(BM_EINVAL, "bm_state_get_slots: state is NULL");
  if (slots) *slots = list_slots(s->list);
  return BM_OK;
}

bm_status bm_state_get_schedule(bm_state* s, int* ctas_per_sm, int* static_sixteenths) {
  clear_error();
  if (!s) return fail(BM_EINVAL, "bm_state_get_schedule: state is NULL");
  if (ctas_per_sm) *ctas_per_sm = s->ctas_per_sm;
  if (static_sixteenths) *static_sixteenths = s->list.static16;
  return BM_OK;
}

bm_status bm_step_async(bm_state* s, int64_t n) {
  clear_error();
  if (!s) return fail(BM_EINVAL, "bm_step: state is NULL");
  if (n < 0) return fail(BM_EINVAL, "bm_step: n_steps must be >= 0");
  if (s->cur_t_end != kInf) {
    bm_status st = set_end(s, kInf);
    if (st != BM_OK) return st;
  }
  return enqueue_steps(s, n);
}

bm_status bm_sync(bm_state* s) {
  clear_error();
  if (!s) return fail(BM_EINVAL, "bm_sync: state is NULL");
  return read_status(s);
}

bm_status bm_step(bm_state* s, int64_t n) {
  bm_status st = bm_step_async(s, n);
  if (st != BM_OK) return st;
  return read_status(s);
}

bm_status bm_run_until(bm_state* s, double t_end) {
  clear_error();
  if (!s) return fail(BM_EINVAL, "bm_run_until: state is NULL");
  if (!std::isfinite(t_end)) return fail(BM_EINVAL, "bm_run_until: t_end must be finite");
  bm_status st = set_end(s, t_end);
  if (st != BM_OK) return st;
  st = read_status(s);
  if (st != BM_OK) return st;
  // chunks grow while the run is long; steps past t_end are no-ops on the device
  int64_t chunk = 32;
  double last_t = s->hctl->t;
  int stalls = 0;
  while (s->hctl->active) {
    st = enqueue_steps(s, chunk);
    if (st != BM_OK) return st;
    st = read_status(s);
    if (st != BM_OK) return st;
    if (s->hctl->t == last_t) {
      if (++stalls > 4) return fail(BM_ETIMEOUT, "bm_run_until: time does not advance");
    } else {
      stalls = 0;
    }
    last_t = s->hctl->t;
    if (chunk < 1024) chunk *= 2;
    // estimate the remaining steps from the current dt to avoid overshooting much
    const double rem = t_end - s->hctl->t;
    if (s->hctl->dt > 0) {
      const double est = rem / s->hctl->dt + 1;
      if (est < chunk) chunk = std::max<int64_t>(1, static_cast<int64_t>(est) + 1);
    }
  }
  return BM_OK;
}

bm_status bm_state_upload(bm_state* s, const double* H, const double* qx, const double* qy, double t) {
  clear_error();
  if (!s) return fail(BM_EINVAL, "bm_state_upload: state is NULL");
  BM_CUDA(cudaStreamSynchronize(s->stream));
  BM_CUDA(cudaMemcpy(s->hctl, s->ctl, sizeof(Ctl), cudaMemcpyDeviceToHost));
  const int par = s->hctl->parity;
  bm_status st = load_state(s, H, qx, qy, t);
  if (st != BM_OK || s->n_species == 0 || par == 0) return st;
  // the state restarts in buffer 0: the species keep their values
  if (s->prec == BM_FP64) {
    BM_CUDA(cudaMemcpy(s->b64.hc[0].p, s->b64.hc[1].p, s->b64.hc[1].bytes(), cudaMemcpyDeviceToDevice));
    BM_CUDA(cudaMemset(s->b64.zmask.p, 0, s->b64.zmask.bytes()));
  } else {
    BM_CUDA(cudaMemcpy(s->b32.hc[0].p, s->b32.hc[1].p, s->b32.hc[1].bytes(), cudaMemcpyDeviceToDevice));
    BM_CUDA(cudaMemset(s->b32.zmask.p, 0, s->b32.zmask.bytes()));
  }
  return BM_OK;
}

bm_status bm_state_download(bm_state* s, double* H, double* qx, double* qy, double* t) {
  clear_error();
  if (!s) return fail(BM_EINVAL, "bm_state_download: state is NULL");
  BM_CUDA(cudaMemcpyAsync(s->hctl, s->ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, s->stream));
  BM_CUDA(cudaStreamSynchronize(s->stream));
  const int par = s->hctl->parity;
  const int n = static_cast<int>(s->mesh->h.n_cells);
  const int nb = (n + 255) / 256;
  const size_t bytes = static_cast<size_t>(n) * sizeof(double);
  double* outs[3] = {H, qx, qy};
  for (int k = 0; k < 3; ++k) {
    if (!outs[k]) continue;
    if (s->prec == BM_FP64) {
      const double* src[3] = {s->b64.H[par].p, s->b64.qx[par].p, s->b64.qy[par].p};
      scatter_to_user<double><<<nb, 256, 0, s->stream>>>(src[k], nullptr, s->mesh->perm.p, n, s->stage[k].p, 0.0);
    } else {
      const float* src[3] = {s->b32.H[par].p, s->b32.qx[par].p, s->b32.qy[par].p};
      scatter_to_user<float><<<nb, 256, 0, s->stream>>>(src[k], k == 0 ? s->b32.Hlo[par].p : nullptr,
                                                         s->mesh->perm.p, n, s->stage[k].p,
                                                         k == 0 ? s->datum : 0.0);
    }
    BM_CUDA(cudaMemcpyAsync(outs[k], s->stage[k].p, bytes, cudaMemcpyDeviceToHost, s->stream));
  }
  BM_CUDA(cudaStreamSynchronize(s->stream));
  if (t) *t = s->hctl->t;
  return BM_OK;
}

bm_status bm_state_track(bm_state* s, double h_arrival) {
  clear_error();
  if (!s) return fail(BM_EINVAL, "bm_state_track: state is NULL");
  if (!std::isfinite(h_arrival) || h_arrival < 0.0)
    return fail(BM_EINVAL, "bm_state_track: h_arrival must be finite and >= 0");
  const HostMesh& h = s->mesh->h;
  const size_t Np = static_cast<size_t>(h.n_tiles) * kTile;
  cudaError_t e = s->prec == BM_FP64 ? s->b64.alloc_tracking(Np) : s->b32.alloc_tracking(Np);
  if (e != cudaSuccess) return dev_fail(e, "bm_state_track: tracking arrays");
  s->trk_harr = h_arrival;
  // the step kernels read the descriptor in place: rewrite it (same size, same address)
  BM_CUDA(cudaStreamSynchronize(s->stream));
  state_desc_bytes(s, &s->hdesc);
  ++s->desc_epoch;  // (a batch made before this no longer describes the state)
  BM_CUDA(cudaMemcpyAsync(s->desc.p, s->hdesc.data(), s->hdesc.size(), cudaMemcpyHostToDevice, s->stream));
  const int n = static_cast<int>(h.n_cells);
  const int nb = (n + 255) / 256;
  if (s->prec == BM_FP64)
    track_init<double><<<nb, 256, 0, s->stream>>>(reinterpret_cast<const InstDesc<double>*>(s->desc.p), s->ctl, n);
  else
    track_init<float><<<nb, 256, 0, s->stream>>>(reinterpret_cast<const InstDesc<float>*>(s->desc.p), s->ctl, n);
  BM_CUDA(cudaGetLastError());
  BM_CUDA(cudaStreamSynchronize(s->stream));
  // from now on the state's launches run the tracking kernel
  if (state_extra_level(s) != s->list.extra) {
    s->list.extra = state_extra_level(s);
    bm_status st = list_occupancy(s->prec, &s->list);
    if (st != BM_OK) return st;
    s->grid = step_grid(s->list, s->ctas_per_sm);
    drop_graphs(s);
    s->last_list = nullptr;  // the state's features changed: the next launch takes every tile
  }
  return BM_OK;
}

bm_status bm_state_download_track(bm_state* s, double* t_arrival, double* h_max, double* u_max, double* q_max,
                                  double* tau_max) {
  clear_error();
  if (!s) return fail(BM_EINVAL, "bm_state_download_track: state is NULL");
  const bool on = s->prec == BM_FP64 ? s->b64.trk_t.p != nullptr : s->b32.trk_t.p != nullptr;
  if (!on) return fail(BM_EINVAL, "bm_state_download_track: tracking is off (bm_state_track starts it)");
  const int n = static_cast<int>(s->mesh->h.n_cells);
  const int nb = (n + 255) / 256;
  const size_t bytes = static_cast<size_t>(n) * sizeof(double);
  double* outs[5] = {t_arrival, h_max, u_max, q_max, tau_max};
  for (int k = 0; k < 5; ++k) {
    if (!outs[k]) continue;
    double* stage = s->stage[k % 3].p;  // reused in stream order after its copy-out
    if (k == 0) {
      const double* src = s->prec == BM_FP64 ? s->b64.trk_t.p : s->b32.trk_t.p;
      scatter_to_user<double><<<nb, 256, 0, s->stream>>>(src, nullptr, s->mesh->perm.p, n, stage, 0.0);
    } else if (s->prec == BM_FP64) {
      scatter_to_user<double><<<nb, 256, 0, s->stream>>>(s->b64.trk[k - 1].p, nullptr, s->mesh->perm.p, n, stage,
                                                          0.0);
    } else {
      scatter_to_user<float><<<nb, 256, 0, s->stream>>>(s->b32.trk[k - 1].p, nullptr, s->mesh->perm.p, n, stage,
                                                         0.0);
    }
    BM_CUDA(cudaGetLastError());
    BM_CUDA(cudaMemcpyAsync(outs[k], stage, bytes, cudaMemcpyDeviceToHost, s->stream));
  }
  BM_CUDA(cudaStreamSynchronize(s->stream));
  return BM_OK;
}

bm_status bm_state_set_scalars(bm_state* s, int32_t n_species, const double* hc, const double* c_in) {
  clear_error();
  if (!s) return fail(BM_EINVAL, "bm_state_set_scalars: state is NULL");
  if (n_species < 0 || n_species > kMaxSpecies) return fail(BM_EINVAL, "bm_state_set_scalars: n_species in [0, 5]");
  const HostMesh& h = s->mesh->h;
  const int n = static_cast<int>(h.n_cells);
  if (n_species > 0 && !hc) return fail(BM_EINVAL, "bm_state_set_scalars: hc is NULL");
  for (int64_t i = 0; i < static_cast<int64_t>(n_species) * n; ++i)
    if (!std::isfinite(hc[i])) return fail(BM_EINVAL, "bm_state_set_scalars: hc has a non-finite value");
  for (int c = 0; c < n_species && c_in; ++c)
    if (!std::isfinite(c_in[c])) return fail(BM_EINVAL, "bm_state_set_scalars: c_in has a non-finite value");
  BM_CUDA(cudaStreamSynchronize(s->stream));
  BM_CUDA(cudaMemcpyAsync(s->hctl, s->ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, s->stream));
  BM_CUDA(cudaStreamSynchronize(s->stream));
  const int par = s->hctl->parity;
  const size_t np = static_cast<size_t>(h.n_tiles) * kTile;
  const TileRecords& R = s->mesh->rec[s->prec == BM_FP64 ? 0 : 1];
  const size_t stride = R.ne4_max;
  if (n_species == 0) {
    s->b64.free_species();
    s->b32.free_species();
  } else {
    cudaError_t e = s->prec == BM_FP64 ? s->b64.alloc_species(np, n_species, h.n_tiles, stride)
                                       : s->b32.alloc_species(np, n_species, h.n_tiles, stride);
    if (e != cudaSuccess) return dev_fail(e, "bm_state_set_scalars: species arrays");
    const int nb = (n + 255) / 256;
    const size_t bytes = static_cast<size_t>(n) * sizeof(double);
    for (int c = 0; c < n_species; ++c) {
      double* stage = s->stage[c % 3].p;  // reused in stream order after its gather
      BM_CUDA(cudaMemcpyAsync(stage, hc + static_cast<size_t>(c) * n, bytes, cudaMemcpyHostToDevice, s->stream));
      if (s->prec == BM_FP64)
        gather_from_user<double><<<nb, 256, 0, s->stream>>>(stage, s->mesh->perm.p, n, s->b64.hc[par].p + c * np);
      else
        gather_from_user<float><<<nb, 256, 0, s->stream>>>(stage, s->mesh->perm.p, n, s->b32.hc[par].p + c * np);
      BM_CUDA(cudaGetLastError());
    }
  }
  s->n_species = n_species;
  for (int c = 0; c < kMaxSpecies; ++c) s->c_in[c] = (c < n_species && c_in) ? c_in[c] : 0.0;
  // the step kernels read the descriptor in place: rewrite it (same size, same address)
  state_desc_bytes(s, &s->hdesc);
  ++s->desc_epoch;  // (a batch made before this no longer describes the state)
  BM_CUDA(cudaMemcpyAsync(s->desc.p, s->hdesc.data(), s->hdesc.size(), cudaMemcpyHostToDevice, s->stream));
  BM_CUDA(cudaStreamSynchronize(s->stream));
  // the launch sequence changes (kernel instantiation, species kernel after each step)
  const int extra = state_extra_level(s);
  if (extra != s->list.extra) {
    s->list.extra = extra;
    bm_status st = list_occupancy(s->prec, &s->list);
    if (st != BM_OK) return st;
    s->grid = step_grid(s->list, s->ctas_per_sm);
  }
  drop_graphs(s);
  s->last_list = nullptr;  // the state's features changed: the next launch takes every tile
  return BM_OK;
}

bm_status bm_state_download_scalars(bm_state* s, double* hc) {
  clear_error();
  if (!s) return fail(BM_EINVAL, "bm_state_download_scalars: state is NULL");
  if (s->n_species == 0) return fail(BM_EINVAL, "bm_state_download_scalars: the state carries no species");
  if (!hc) return fail(BM_EINVAL, "bm_state_download_scalars: hc is NULL");
  BM_CUDA(cudaMemcpyAsync(s->hctl, s->ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, s->stream));
  BM_CUDA(cudaStreamSynchronize(s->stream));
  const int par = s->hctl->parity;
  const int n = static_cast<int>(s->mesh->h.n_cells);
  const int nb = (n + 255) / 256;
  const size_t np = static_cast<size_t>(s->mesh->h.n_tiles) * kTile;
  const size_t bytes = static_cast<size_t>(n) * sizeof(double);
  for (int c = 0; c < s->n_species; ++c) {
    double* stage = s->stage[c % 3].p;
    if (s->prec == BM_FP64)
      scatter_to_user<double><<<nb, 256, 0, s->stream>>>(s->b64.hc[par].p + c * np, nullptr, s->mesh->perm.p, n,
                                                          stage, 0.0);
    else
      scatter_to_user<float><<<nb, 256, 0, s->stream>>>(s->b32.hc[par].p + c * np, nullptr, s->mesh->perm.p, n,
                                                         stage, 0.0);
    BM_CUDA(cudaGetLastError());
    BM_CUDA(cudaMemcpyAsync(hc + static_cast<size_t>(c) * n, stage, bytes, cudaMemcpyDeviceToHost, s->stream));
  }
  BM_CUDA(cudaStreamSynchronize(s->stream));
  return BM_OK;
}

bm_status bm_state_set_sources(bm_state* s, int32_t n_regions, const int32_t* region, const int32_t* kind,
                               const int32_t* mode, const int64_t* offsets, const double* t, const double* v) {
  clear_error();
  if (!s) return fail(BM_EINVAL, "bm_state_set_sources: state is NULL");
  if (n_regions < 0 || n_regions > 65536) return fail(BM_EINVAL, "bm_state_set_sources: n_regions in [0, 65536]");
  const HostMesh& h = s->mesh->h;
  const int64_t n = h.n_cells;
  if (n_regions > 0) {
    if (!region || !kind || !mode || !offsets || !t || !v) return fail(BM_EINVAL, "bm_state_set_sources: NULL array");
    if (offsets[0] != 0) return fail(BM_EINVAL, "bm_state_set_sources: offsets[0] must be 0");
    for (int32_t r = 0; r < n_regions; ++r) {
      if (kind[r] != 0 && kind[r] != 1) return fail(BM_EINVAL, "bm_state_set_sources: kind must be 0 or 1");
      if (mode[r] < 0 || mode[r] > 2) return fail(BM_EINVAL, "bm_state_set_sources: mode must be 0, 1 or 2");
      if (offsets[r + 1] <= offsets[r] || offsets[r + 1] - offsets[r] > 1000000)
        return fail(BM_EINVAL, "bm_state_set_sources: every series needs 1 to 1e6 points");
      for (int64_t k = offsets[r]; k < offsets[r + 1]; ++k) {
        if (!std::isfinite(t[k]) || !std::isfinite(v[k]))
          return fail(BM_EINVAL, "bm_state_set_sources: series values must be finite");
        if (k > offsets[r] && !(t[k] > t[k - 1]))
          return fail(BM_EINVAL, "bm_state_set_sources: series times must increase strictly");
      }
    }
  }
  std::vector<int32_t> reg_new(static_cast<size_t>(h.n_tiles) * kTile, -1);
  std::vector<double> area(static_cast<size_t>(n_regions), 0.0);
  std::vector<uint8_t> tiles(static_cast<size_t>(h.n_tiles), 0);
  for (int64_t i = 0; i < n && n_regions > 0; ++i) {
    const int32_t r = region[h.perm[i]];
    if (r < -1 || r >= n_regions) return fail(BM_EINVAL, "bm_state_set_sources: region index out of range");
    reg_new[i] = r;
    if (r >= 0) {
      area[r] += h.area[i];
      tiles[i / kTile] = 1;
    }
  }
  for (int32_t r = 0; r < n_regions; ++r)
    if (kind[r] == 0 && !(area[r] > 0.0))
      return fail(BM_EINVAL, "bm_state_set_sources: a total-discharge region holds no cell");
  BM_CUDA(cudaStreamSynchronize(s->stream));
  cudaError_t e = cudaSuccess;
  if (n_regions > 0) {
    const int64_t np = offsets[n_regions];
    e = s->src_reg.upload(reg_new);
    if (e == cudaSuccess) e = s->src_kind.upload(std::vector<int32_t>(kind, kind + n_regions));
    if (e == cudaSuccess) e = s->src_mode.upload(std::vector<int32_t>(mode, mode + n_regions));
    if (e == cudaSuccess) e = s->src_off.upload(std::vector<long long>(offsets, offsets + n_regions + 1));
    if (e == cudaSuccess) e = s->src_t.upload(std::vector<double>(t, t + np));
    if (e == cudaSuccess) e = s->src_v.upload(std::vector<double>(v, v + np));
    if (e == cudaSuccess) e = s->src_area.upload(area);
    if (e == cudaSuccess) e = s->src_rate64.alloc(static_cast<size_t>(n_regions));
    if (e == cudaSuccess) e = s->src_rate32.alloc(static_cast<size_t>(n_regions));
    if (e != cudaSuccess) return dev_fail(e, "bm_state_set_sources: source arrays");
    s->src_tile = tiles;
  } else {
    s->src_reg.release(); s->src_kind.release(); s->src_mode.release(); s->src_off.release();
    s->src_t.release(); s->src_v.release(); s->src_area.release(); s->src_rate64.release(); s->src_rate32.release();
    s->src_tile.clear();
  }
  s->n_src = n_regions;
  // the descriptor (read in place) and the work list (tile flags, kernel instantiation)
  state_desc_bytes(s, &s->hdesc);
  ++s->desc_epoch;  // (a batch made before this no longer describes the state)
  BM_CUDA(cudaMemcpyAsync(s->desc.p, s->hdesc.data(), s->hdesc.size(), cudaMemcpyHostToDevice, s->stream));
  BM_CUDA(cudaStreamSynchronize(s->stream));
  drop_graphs(s);
  s->last_list = nullptr;  // the state's features changed: the next launch takes every tile
  bm_status st = build_step_list({s}, {static_cast<const void*>(s->desc.p)}, &s->list);
  if (st != BM_OK) return st;
  s->grid = step_grid(s->list, s->ctas_per_sm);
  return BM_OK;
}

bm_status bm_state_set_morpho(bm_state* s, int32_t on, double porosity, double s_rel, double d, double alpha,
                              double m, double theta_cr) {
  clear_error();
  if (!s) return fail(BM_EINVAL, "bm_state_set_morpho: state is NULL");
  if (on) {
    if (s->prec != BM_FP64) return fail(BM_EINVAL, "bm_state_set_morpho: morphodynamics needs an FP64 state");
    if (s->fr_law != 0) return fail(BM_EINVAL, "bm_state_set_morpho: morphodynamics takes Manning's law only");
    if (!(porosity >= 0.0 && porosity < 1.0) || !(s_rel > 1.0) || !(d > 0.0) || !(alpha >= 0.0) || !(m >= 1.0) ||
        !std::isfinite(theta_cr) || !std::isfinite(d) || !std::isfinite(alpha) || !std::isfinite(m) ||
        !std::isfinite(s_rel))
      return fail(BM_EINVAL,
                  "bm_state_set_morpho: need 0 <= porosity < 1, s > 1, d > 0, alpha >= 0, m >= 1, finite theta_cr");
  }
  BM_CUDA(cudaStreamSynchronize(s->stream));
  if (on) {
    const size_t np = static_cast<size_t>(s->mesh->h.n_tiles) * kTile;
    cudaError_t e = s->mo_dz.p ? cudaSuccess : s->mo_dz.alloc(np);
    if (e == cudaSuccess && !s->mo_dt.p) e = s->mo_dt.alloc(1);
    if (e == cudaSuccess) e = cudaMemset(s->mo_dz.p, 0, s->mo_dz.bytes());
    if (e != cudaSuccess) return dev_fail(e, "bm_state_set_morpho");
    const double par[6] = {porosity, s_rel, d, alpha, m, theta_cr};
    for (int k = 0; k < 6; ++k) s->mo_par[k] = par[k];
  }
  s->morpho = on != 0;
  drop_graphs(s);  // the launch sequence changes
  s->last_list = nullptr;  // the state's features changed: the next launch takes every tile
  return BM_OK;
}

bm_status bm_state_set_outflow(bm_state* s, const double* hq_stage, const double* hq_discharge, int64_t n_hq,
                               double weir_crest, double weir_poleni) {
  clear_error();
  if (!s) return fail(BM_EINVAL, "bm_state_set_outflow: state is NULL");
  if (n_hq < 0 || n_hq == 1) return fail(BM_EINVAL, "bm_state_set_outflow: the h-Q table needs 0 or >= 2 points");
  if (n_hq > 0 && (!hq_stage || !hq_discharge)) return fail(BM_EINVAL, "bm_state_set_outflow: table is NULL");
  for (int64_t k = 0; k < n_hq; ++k) {
    if (!std::isfinite(hq_stage[k]) || !std::isfinite(hq_discharge[k]) || !(hq_discharge[k] >= 0.0))
      return fail(BM_EINVAL, "bm_state_set_outflow: stages must be finite and discharges finite and >= 0");
    if (k > 0 && !(hq_stage[k] > hq_stage[k - 1]))
      return fail(BM_EINVAL, "bm_state_set_outflow: stages must increase strictly");
  }
  if (!std::isfinite(weir_crest)) return fail(BM_EINVAL, "bm_state_set_outflow: weir_crest must be finite");
  if (!std::isfinite(weir_poleni) || !(weir_poleni >= 0.0))
    return fail(BM_EINVAL, "bm_state_set_outflow: weir_poleni must be finite and >= 0");
  BM_CUDA(cudaStreamSynchronize(s->stream));
  std::vector<double> st(hq_stage, hq_stage + n_hq), dq(hq_discharge, hq_discharge + n_hq);
  cudaError_t e = s->hq_s.upload(st);
  if (e == cudaSuccess) e = s->hq_q.upload(dq);
  if (e != cudaSuccess) return dev_fail(e, "bm_state_set_outflow");
  s->hq_n = static_cast<int>(n_hq);
  s->weir_crest = weir_crest;
  s->weir_mu = weir_poleni;
  state_desc_bytes(s, &s->hdesc);
  ++s->desc_epoch;  // (a batch made before this no longer describes the state)
  BM_CUDA(cudaMemcpyAsync(s->desc.p, s->hdesc.data(), s->hdesc.size(), cudaMemcpyHostToDevice, s->stream));
  const int extra = state_extra_level(s);  // laws that let water out: the full instantiation
  if (extra != s->list.extra) {
    s->list.extra = extra;
    bm_status lst = list_occupancy(s->prec, &s->list);
    if (lst != BM_OK) return lst;
    s->grid = step_grid(s->list, s->ctas_per_sm);
  }
  drop_graphs(s);
  s->last_list = nullptr;  // the state's features changed: the next launch takes every tile
  // the next step's dt and h-Q split follow the new laws: prime again (time unchanged)
  launch_state(s, s->stream, 1);
  BM_CUDA(cudaGetLastError());
  BM_CUDA(cudaStreamSynchronize(s->stream));
  return read_status(s);
}

bm_status bm_state_set_level(bm_state* s, const double* t, const double* z, int64_t n) {
  clear_error();
  if (!s) return fail(BM_EINVAL, "bm_state_set_level: state is NULL");
  if (n < 0) return fail(BM_EINVAL, "bm_state_set_level: n must be >= 0");
  if (n > 0 && (!t || !z)) return fail(BM_EINVAL, "bm_state_set_level: series is NULL");
  if (n > (1 << 20)) return fail(BM_EINVAL, "bm_state_set_level: at most 2^20 points");
  for (int64_t k = 0; k < n; ++k) {
    if (!std::isfinite(t[k]) || !std::isfinite(z[k]))
      return fail(BM_EINVAL, "bm_state_set_level: times and levels must be finite");
    if (k > 0 && !(t[k] > t[k - 1])) return fail(BM_EINVAL, "bm_state_set_level: times must increase strictly");
  }
  BM_CUDA(cudaStreamSynchronize(s->stream));
  std::vector<double> tt(t, t + n), zz(z, z + n);
  cudaError_t e = s->zh_t.upload(tt);
  if (e == cudaSuccess) e = s->zh_v.upload(zz);
  if (e != cudaSuccess) return dev_fail(e, "bm_state_set_level");
  s->zh_n = static_cast<int>(n);
  state_desc_bytes(s, &s->hdesc);
  ++s->desc_epoch;  // (a batch made before this no longer describes the state)
  BM_CUDA(cudaMemcpyAsync(s->desc.p, s->hdesc.data(), s->hdesc.size(), cudaMemcpyHostToDevice, s->stream));
  const int extra = state_extra_level(s);  // a level series: the full instantiation
  if (extra != s->list.extra) {
    s->list.extra = extra;
    bm_status lst = list_occupancy(s->prec, &s->list);
    if (lst != BM_OK) return lst;
    s->grid = step_grid(s->list, s->ctas_per_sm);
  }
  drop_graphs(s);
  s->last_list = nullptr;  // the state's features changed: the next launch takes every tile
  // the next step's dt follows the level: prime again (time unchanged)
  launch_state(s, s->stream, 1);
  BM_CUDA(cudaGetLastError());
  BM_CUDA(cudaStreamSynchronize(s->stream));
  return read_status(s);
}

bm_status bm_state_set_friction(bm_state* s, int32_t law, const double* coef) {
  clear_error();
  if (!s) return fail(BM_EINVAL, "bm_state_set_friction: state is NULL");
  if (law < 0 || law > 2) return fail(BM_EINVAL, "bm_state_set_friction: law must be 0, 1 or 2");
  if (!coef) return fail(BM_EINVAL, "bm_state_set_friction: coef is NULL");
  if (law != 0 && s->morpho)
    return fail(BM_EINVAL, "bm_state_set_friction: morphodynamics takes Manning's law only");
  const HostMesh& h = s->mesh->h;
  const int64_t n = h.n_cells;
  std::vector<double> v(static_cast<size_t>(h.n_tiles) * kTile, 0.0);
  for (int64_t i = 0; i < n; ++i) {
    const double c = coef[h.perm[i]];
    if (!(c >= 0.0) || !std::isfinite(c)) return fail(BM_EINVAL, "bm_state_set_friction: coef must be finite and >= 0");
    v[i] = law == 0 ? s->prm.g * c * c : c;
  }
  BM_CUDA(cudaStreamSynchronize(s->stream));
  cudaError_t e = s->prec == BM_FP64 ? cudaMemcpy(s->b64.gn2.p, v.data(), v.size() * sizeof(double),
                                                  cudaMemcpyHostToDevice)
                                     : cudaMemcpy(s->b32.gn2.p, narrow<float>(v).data(), v.size() * sizeof(float),
                                                  cudaMemcpyHostToDevice);
  if (e != cudaSuccess) return dev_fail(e, "bm_state_set_friction");
  s->fr_law = law;
  state_desc_bytes(s, &s->hdesc);
  ++s->desc_epoch;  // (a batch made before this no longer describes the state)
  BM_CUDA(cudaMemcpyAsync(s->desc.p, s->hdesc.data(), s->hdesc.size(), cudaMemcpyHostToDevice, s->stream));
  BM_CUDA(cudaStreamSynchronize(s->stream));
  const int extra = state_extra_level(s);
  if (extra != s->list.extra) {
    s->list.extra = extra;
    bm_status st = list_occupancy(s->prec, &s->list);
    if (st != BM_OK) return st;
    s->grid = step_grid(s->list, s->ctas_per_sm);
  }
  drop_graphs(s);
  s->last_list = nullptr;  // the state's features changed: the next launch takes every tile
  return BM_OK;
}

bm_status bm_state_download_bed(bm_state* s, double* z) {
  clear_error();
  if (!s) return fail(BM_EINVAL, "bm_state_download_bed: state is NULL");
  if (!z) return fail(BM_EINVAL, "bm_state_download_bed: z is NULL");
  const int n = static_cast<int>(s->mesh->h.n_cells);
  const int nb = (n + 255) / 256;
  if (s->prec == BM_FP64)
    scatter_to_user<double><<<nb, 256, 0, s->stream>>>(s->b64.z.p, nullptr, s->mesh->perm.p, n, s->stage[0].p, 0.0);
  else
    scatter_to_user<float><<<nb, 256, 0, s->stream>>>(s->b32.z.p, nullptr, s->mesh->perm.p, n, s->stage[0].p,
                                                       s->datum);
  BM_CUDA(cudaGetLastError());
  BM_CUDA(cudaMemcpyAsync(z, s->stage[0].p, static_cast<size_t>(n) * sizeof(double), cudaMemcpyDeviceToHost,
                          s->stream));
  BM_CUDA(cudaStreamSynchronize(s->stream));
  return BM_OK;
}

bm_status bm_state_set_tile_skipping(bm_state* s, int32_t on) {
  clear_error();
  if (!s) return fail(BM_EINVAL, "bm_state_set_tile_skipping: state is NULL");
  if (on != 0 && on != 1) return fail(BM_EINVAL, "bm_state_set_tile_skipping: on must be 0 or 1");
  BM_CUDA(cudaStreamSynchronize(s->stream));
  s->no_skip = on == 0;
  s->last_list = nullptr;  // the next launch resets the list with the new setting
  return BM_OK;
}

bm_status bm_state_work(bm_state* s, int64_t* tiles_last, int64_t* tiles_total) {
  clear_error();
  if (!s) return fail(BM_EINVAL, "bm_state_work: state is NULL");
  int sc[kSchedInts];
  BM_CUDA(cudaStreamSynchronize(s->stream));
  BM_CUDA(cudaMemcpy(sc, s->list.sched.p, sizeof(sc), cudaMemcpyDeviceToHost));
  if (tiles_last) *tiles_last = s->last_list == &s->list ? sc[12] : 0;
  if (tiles_total) *tiles_total = s->list.n;
  return BM_OK;
}

bm_status bm_state_stats(bm_state* s, double* t, double* dt_next, int64_t* steps, double* volume,
                         double* boundary_volume) {
  clear_error();
  if (!s) return fail(BM_EINVAL, "bm_state_stats: state is NULL");
  BM_CUDA(cudaMemcpyAsync(s->hctl, s->ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, s->stream));
  BM_CUDA(cudaStreamSynchronize(s->stream));
  if (volume) {
    const int par = s->hctl->parity;
    const int nt = static_cast<int>(s->mesh->h.n_tiles);
    const int n = static_cast<int>(s->mesh->h.n_cells);
    if (s->prec == BM_FP64)
      volume_partials<double><<<nt, kTile, 0, s->stream>>>(s->b64.H[par].p, nullptr, s->b64.z.p, s->mesh->area.p,
                                                            nullptr, n, s->vol_part.p);
    else
      volume_partials<float><<<nt, kTile, 0, s->stream>>>(s->b32.H[par].p, s->b32.Hlo[par].p, s->b32.z.p, nullptr,
                                                           s->mesh->inv_area32.p, n, s->vol_part.p);
    sum_partials<<<1, kSumThreads, 0, s->stream>>>(s->vol_part.p, nt, s->vol_out.p);
    BM_CUDA(cudaMemcpyAsync(s->hvol, s->vol_out.p, sizeof(double), cudaMemcpyDeviceToHost, s->stream));
    BM_CUDA(cudaStreamSynchronize(s->stream));
    *volume = *s->hvol;
  }
  if (t) *t = s->hctl->t;
  if (dt_next) *dt_next = s->hctl->active ? s->hctl->dt : 0.0;
  if (steps) *steps = s->hctl->steps;
  if (boundary_volume) *boundary_volume = s->hctl->bvol;
  return BM_OK;
}

bm_status bm_state_test_timeout(bm_state* s) {
  clear_error();
  if (!s) return fail(BM_EINVAL, "bm_state_test_timeout: state is NULL");
  BM_CUDA(cudaStreamSynchronize(s->stream));
  ensure_list(&s->list, s->stream);
  launch_work(s->prec, s->list, s->grid, 0, s->stream, 1);
  BM_CUDA(cudaGetLastError());
  s->last_list = nullptr;  // the launch gave up: its lists are incomplete
  return read_status(s);
}

bm_status bm_step_timed(bm_state* s, int64_t n, double* step_kernel_ms, double* total_ms) {
  clear_error();
  if (!s) return fail(BM_EINVAL, "bm_step_timed: state is NULL");
  if (n < 1 || n > 100000) return fail(BM_EINVAL, "bm_step_timed: n_steps must be in [1, 100000]");
  if (s->cur_t_end != kInf) {
    bm_status st = set_end(s, kInf);
    if (st != BM_OK) return st;
  }
  std::vector<cudaEvent_t> ev(2 * n, nullptr);
  for (auto& e : ev) {
    cudaError_t r = cudaEventCreate(&e);
    if (r != cudaSuccess) {
      for (auto& x : ev) if (x) cudaEventDestroy(x);
      return fail(BM_ECUDA, std::string("cudaEventCreate: ") + cudaGetErrorString(r));
    }
  }
  ensure_list(&s->list, s->stream);
  for (int64_t k = 0; k < n; ++k) {
    cudaEventRecord(ev[2 * k], s->stream);
    launch_state(s, s->stream, 0);
    cudaEventRecord(ev[2 * k + 1], s->stream);
  }
  cudaError_t r = cudaStreamSynchronize(s->stream);
  double ksum = 0.0;
  float ms = 0.0f;
  for (int64_t k = 0; k < n && r == cudaSuccess; ++k) {
    r = cudaEventElapsedTime(&ms, ev[2 * k], ev[2 * k + 1]);
    ksum += ms;
  }
  float tot = 0.0f;
  if (r == cudaSuccess) r = cudaEventElapsedTime(&tot, ev[0], ev[2 * n - 1]);
  for (auto& e : ev) cudaEventDestroy(e);
  if (r != cudaSuccess) return fail(BM_ECUDA, std::string("bm_step_timed: ") + cudaGetErrorString(r));
  if (step_kernel_ms) *step_kernel_ms = ksum;
  if (total_ms) *total_ms = tot;
  return read_status(s);
}

}  // extern "C"

namespace bm {
namespace {
// The step kernel's elementary functions (and the CUDA library's counterparts) on an
// array, for tests of the hand-written ones.
__global__ void math_eval(int fn, const double* x, double* y, int64_t n) {
  const int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double v = x[i];
  double r = 0.0;
  switch (fn) {
    case 0: r = f_rcbrt(v); break;
    case 1: r = 1.0 / cbrt(v); break;
    case 2: r = f_rcp(v); break;
    case 3: r = 1.0 / v; break;
    case 4: r = static_cast<double>(f_rcbrt(static_cast<float>(v))); break;
    case 5: r = static_cast<double>(rcbrtf(static_cast<float>(v))); break;
    case 6: r = f_cbrt(v); break;
    case 7: r = cbrt(v); break;
    default: r = 0.0;
  }
  y[i] = r;
}
}  // namespace
}  // namespace bm

extern "C" {

bm_status bm_math_eval(int32_t fn, const double* x, double* y, int64_t n) {
  clear_error();
  if (fn < 0 || fn > 7) return fail(BM_EINVAL, "bm_math_eval: fn must be in [0, 7]");
  if (n < 0 || n > (int64_t(1) << 28)) return fail(BM_EINVAL, "bm_math_eval: n must be in [0, 2^28]");
  if (n == 0) return BM_OK;
  if (!x || !y) return fail(BM_EINVAL, "bm_math_eval: NULL array");
  DBuf<double> dx, dy;
  BM_CUDA(dx.alloc(static_cast<size_t>(n)));
  BM_CUDA(dy.alloc(static_cast<size_t>(n)));
  BM_CUDA(cudaMemcpy(dx.p, x, static_cast<size_t>(n) * sizeof(double), cudaMemcpyHostToDevice));
  math_eval<<<static_cast<unsigned>((n + 255) / 256), 256>>>(fn, dx.p, dy.p, n);
  BM_CUDA(cudaGetLastError());
  BM_CUDA(cudaMemcpy(y, dy.p, static_cast<size_t>(n) * sizeof(double), cudaMemcpyDeviceToHost));
  return BM_OK;
}

}  // extern "C"

// ---------------------------------------------------------------- autotuner

namespace bm {
namespace {

// Device snapshot of everything a step reads or writes, to undo tuning trials.
struct Snapshot {
  std::deque<std::pair<void*, DBuf<unsigned char>>> saved;  // deque: entries never move
  cudaError_t take(void* p, size_t bytes, cudaStream_t st) {
    if (!p || bytes == 0) return cudaSuccess;
    saved.emplace_back();
    saved.back().first = p;
    cudaError_t e = saved.back().second.alloc(bytes);
    if (e == cudaSuccess) e = cudaMemcpyAsync(saved.back().second.p, p, bytes, cudaMemcpyDeviceToDevice, st);
    return e;
  }
  cudaError_t restore(cudaStream_t st) {
    for (auto& kv : saved) {
      cudaError_t e = cudaMemcpyAsync(kv.first, kv.second.p, kv.second.n, cudaMemcpyDeviceToDevice, st);
      if (e != cudaSuccess) return e;
    }
    return cudaStreamSynchronize(st);
  }
};

template <typename T>
cudaError_t snapshot_buffers(Buffers<T>& b, Snapshot* sn, cudaStream_t st) {
  cudaError_t e = cudaSuccess;
  for (int k = 0; k < 2 && e == cudaSuccess; ++k) {
    DBuf<T>* bufs[4] = {&b.H[k], &b.Hlo[k], &b.qx[k], &b.qy[k]};
    for (auto* x : bufs)
      if (e == cudaSuccess) e = sn->take(x->p, x->bytes(), st);
  }
  if (e == cudaSuccess) e = sn->take(b.in_pw.p, b.in_pw.bytes(), st);
  if (e == cudaSuccess) e = sn->take(b.in_hs.p, b.in_hs.bytes(), st);
  if (e == cudaSuccess) e = sn->take(b.trk_t.p, b.trk_t.bytes(), st);
  for (int k = 0; k < 4 && e == cudaSuccess; ++k) e = sn->take(b.trk[k].p, b.trk[k].bytes(), st);
  for (int k = 0; k < 2 && e == cudaSuccess; ++k) e = sn->take(b.hc[k].p, b.hc[k].bytes(), st);
  if (e == cudaSuccess) e = sn->take(b.zmask.p, b.zmask.bytes(), st);
  if (e == cudaSuccess) e = sn->take(b.z.p, b.z.bytes(), st);  // the bed moves with morphodynamics
  return e;
}

cudaError_t snapshot_state(bm_state* s, Snapshot* sn, cudaStream_t st) {
  cudaError_t e = s->prec == BM_FP64 ? snapshot_buffers(s->b64, sn, st) : snapshot_buffers(s->b32, sn, st);
  if (e == cudaSuccess) e = sn->take(s->ctl, sizeof(Ctl), st);
  if (e == cudaSuccess) e = sn->take(s->part.p, s->part.bytes(), st);
  return e;
}

}  // namespace

// Time `steps` steps for each candidate launch schedule, restore the state(s), pick
// the fastest.  Two rounds: for each claiming mode and tile-slot count (those in force
// first), the CTAs per SM -- the count in force first, then as many as fit (0) and
// 1..4, candidates that give the same grid timed once -- at the current static share
// of the tickets; then that share (sixteenths 0, 2, ..., 16 and the precision's
// default) at the best mode, slots and CTAs per SM.  The schedule never changes results, so every trial restores the
// same state and the choice is by time alone.
bm_status autotune_shape(std::vector<bm_state*> states, int steps, int start_ctas, int start_static, int* best,
                         int* best_static,
                         double* best_ms, const std::function<bm_status(int, int)>& set_shape,
                         const std::function<int(int)>& grid_of,
                         const std::function<bm_status(int)>& run_steps, cudaStream_t st,
                         const std::vector<int>& slot_cands, const std::function<bm_status(int)>& set_slots,
                         int start_claim, const std::function<bm_status(int)>& set_claim) {
  Snapshot sn;
  for (bm_state* s : states) {
    cudaError_t e = snapshot_state(s, &sn, st);
    if (e != cudaSuccess) return fail(BM_ENOMEM, std::string("autotune snapshot: ") + cudaGetErrorString(e));
  }
  BM_CUDA(cudaStreamSynchronize(st));
  cudaEvent_t e0, e1;
  BM_CUDA(cudaEventCreate(&e0));
  BM_CUDA(cudaEventCreate(&e1));
  double bms = std::numeric_limits<double>::infinity();
  int bc = 0, bs = start_static, bk = slot_cands.empty() ? 3 : slot_cands[0], bm = start_claim;
  int cur_k = bk, cur_m = bm;  // the slot count and claiming in force during a trial
  bm_status out = BM_OK;
  // a trial: the schedule, two warm steps (graph capture), then `steps` steps timed
  // twice (the state restored after each), the faster counts; a schedule replaces the
  // best so far only if it is 2 % faster (the first trial, the schedule in force, is
  // kept unless another clearly beats it)
  bool first = true;
  // trials time whole graphs of 32 launches (launches in one graph overlap each other's
  // ends and starts; separate graph launches do not, which favours other shapes)
  const int timed = (steps + 31) / 32 * 32;
  auto trial = [&](int c, int s16) -> bm_status {
    bm_status r = set_shape(c, s16);
    if (r != BM_OK) return r;
    float tmin = std::numeric_limits<float>::infinity();
    for (int rep = 0; rep < 2; ++rep) {
      r = run_steps(rep == 0 ? 32 : 2);  // (the first captures the graphs)
      if (r != BM_OK) return r;
      cudaEventRecord(e0, st);
      r = run_steps(timed);
      if (r != BM_OK) return r;
      cudaEventRecord(e1, st);
      cudaEventSynchronize(e1);
      float ms = 0.0f;
      cudaEventElapsedTime(&ms, e0, e1);
      tmin = std::min(tmin, ms);
      if (sn.restore(st) != cudaSuccess) return fail(BM_ECUDA, "autotune: restore failed");
      for (bm_state* m : states) m->last_list = nullptr;  // restored arrays: the next launch takes every tile
    }
    if (first || tmin < 0.98 * bms) {
      bms = tmin;
      bc = c;
      bs = s16;
      bk = cur_k;
      bm = cur_m;
    }
    first = false;
    return BM_OK;
  };
  for (int m : {start_claim, (start_claim + 1) % 4, (start_claim + 2) % 4, (start_claim + 3) % 4}) {
    if (out != BM_OK) break;
    out = set_claim(m);
    cur_m = m;
    for (int k : slot_cands) {
      if (out != BM_OK) break;
      if (set_slots(k) != BM_OK) {  // a layout that does not fit this device: skip the count
        clear_error();
        continue;
      }
      cur_k = k;
      std::vector<int> grids;
      for (int c : {start_ctas, 0, 1, 2, 3, 4}) {
        const int g = grid_of(c);
        if (std::find(grids.begin(), grids.end(), g) != grids.end()) continue;
        grids.push_back(g);
        out = trial(c, start_static);
        if (out != BM_OK) break;
      }
    }
  }
  if (out == BM_OK) out = set_claim(bm);
  if (out == BM_OK) out = set_slots(bk);
  cur_k = bk;
  cur_m = bm;
  const int c_best = bc;
  for (int s16 = -1; s16 <= 16 && out == BM_OK; s16 += (s16 < 0 ? 1 : 2)) {
    if (s16 == start_static) continue;
    out = trial(c_best, s16);
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (out != BM_OK) return out;
  out = set_claim(bm);
  if (out != BM_OK) return out;
  out = set_slots(bk);
  if (out != BM_OK) return out;
  out = set_shape(bc, bs);
  if (out != BM_OK) return out;
  if (best) *best = bc;
  if (best_static) *best_static = bs;
  if (best_ms) *best_ms = bms / timed;
  return BM_OK;
}

}  // namespace bm

extern "C" {

bm_status bm_state_autotune(bm_state* s, int steps_per_trial, int* best_ctas_per_sm, double* ms_per_step) {
  clear_error();
  if (!s) return fail(BM_EINVAL, "bm_state_autotune: state is NULL");
  if (steps_per_trial < 1 || steps_per_trial > 10000) return fail(BM_EINVAL, "bm_state_autotune: steps in [1, 10000]");
  BM_CUDA(cudaStreamSynchronize(s->stream));
  const double keep_end = s->cur_t_end;
  if (keep_end != kInf) {
    bm_status st = set_end(s, kInf);
    if (st != BM_OK) return st;
  }
  bm_status st = autotune_shape(
      {s}, steps_per_trial, s->ctas_per_sm, s->list.static16, best_ctas_per_sm, nullptr, ms_per_step,
      [&](int c, int s16) { return bm_state_set_schedule(s, c, s16); },
      [&](int c) { return step_grid(s->list, c); }, [&](int n) { return enqueue_steps(s, n); }, s->stream,
      slot_candidates(s->list), [&](int k) { return bm_state_set_slots(s, k); }, list_claim(s->prec, s->list),
      [&](int m) { return bm_state_set_claim(s, m); });
  if (st == BM_OK && keep_end != kInf) st = set_end(s, keep_end);
  return st;
}

}  // extern "C"

// ---------------------------------------------------------------- volume without allocation

namespace bm {
namespace {

// Scratch for bm_volume_noalloc: one partial sum per 256-cell block.  It lives in the
// library image (64 KiB per device that loads the library, held until exit), so the
// entry point never allocates.  Every call overwrites the partials it reads, so
// nothing has to start at zero; calls that overlap on the GPU share it and race.
constexpr int kNoallocPartials = 8192;
constexpr int64_t kNoallocMaxCells = static_cast<int64_t>(kNoallocPartials) * kTile;
static __device__ __align__(256) double g_noalloc_partials[kNoallocPartials];

constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mu;
double* g_noalloc_addr[kMaxDevices] = {nullptr};

// Device address of the scratch array on the current device (looked up once per
// device; host code must not use the symbol itself as a device pointer).
bm_status noalloc_scratch(double** out) {
  int dev = 0;
  BM_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices) return fail(BM_EINVAL, "bm_volume_noalloc: device index out of range");
  std::lock_guard<std::mutex> lk(g_noalloc_mu);
  if (!g_noalloc_addr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_partials);
    if (e != cudaSuccess)
      return fail(BM_ECUDA, std::string("bm_volume_noalloc: cudaGetSymbolAddress: ") + cudaGetErrorString(e));
    g_noalloc_addr[dev] = static_cast<double*>(p);
  }
  *out = g_noalloc_addr[dev];
  return BM_OK;
}

}  // namespace
}  // namespace bm

extern "C" {

bm_status bm_volume_noalloc(const double* H, const double* z, const double* area, int64_t n_cells, double* volume,
                            void* cuda_stream) {
  clear_error();
  if (n_cells < 0) return fail(BM_EINVAL, "bm_volume_noalloc: n_cells must be >= 0");
  if (n_cells > kNoallocMaxCells)
    return fail(BM_EINVAL, "bm_volume_noalloc: n_cells exceeds the fixed scratch limit of 2,097,152 cells");
  if (!volume) return fail(BM_EINVAL, "bm_volume_noalloc: volume is NULL");
  if (n_cells > 0 && (!H || !z || !area)) return fail(BM_EINVAL, "bm_volume_noalloc: NULL input array");
  double* scratch = nullptr;
  bm_status st = noalloc_scratch(&scratch);
  if (st != BM_OK) return st;
  cudaStream_t stream = cuda_stream ? static_cast<cudaStream_t>(cuda_stream) : cudaStreamLegacy;
  const int nb = static_cast<int>((n_cells + kTile - 1) / kTile);
  if (nb > 0)
    volume_partials<double><<<nb, kTile, 0, stream>>>(H, nullptr, z, area, nullptr, static_cast<int>(n_cells),
                                                      scratch);
  sum_partials<<<1, kSumThreads, 0, stream>>>(scratch, nb, volume);
  BM_CUDA(cudaGetLastError());
  return BM_OK;
}

}  // extern "C"
