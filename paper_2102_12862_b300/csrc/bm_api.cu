// bm_api.cu -- the C ABI (include/bm.h): meshes and states resident in HBM, the step
// sequence captured in CUDA graphs, end-time targeting, checkpoint upload/download.
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>
#include <limits>
#include <map>
#include <sstream>
#include <string>
#include <vector>

#include "bm_internal.h"
#include "bm_kernels.cuh"

namespace bm {

static thread_local std::string g_err;

bm_status fail(bm_status st, const std::string& msg) {
  g_err = msg;
  return st;
}
void clear_error() { g_err.clear(); }

#define BM_CUDA(call)                                                                          \
  do {                                                                                         \
    cudaError_t e_ = (call);                                                                   \
    if (e_ != cudaSuccess) {                                                                   \
      std::ostringstream os_;                                                                  \
      os_ << #call << ": " << cudaGetErrorString(e_);                                          \
      return fail(BM_ECUDA, os_.str());                                                        \
    }                                                                                          \
  } while (0)

// Typed device buffer (owning).
template <typename T>
struct DBuf {
  T* p = nullptr;
  size_t n = 0;
  DBuf() = default;
  DBuf(const DBuf&) = delete;
  DBuf& operator=(const DBuf&) = delete;
  ~DBuf() { release(); }
  void release() {
    if (p) cudaFree(p);
    p = nullptr;
    n = 0;
  }
  cudaError_t alloc(size_t count) {
    release();
    n = count;
    if (count == 0) return cudaSuccess;
    return cudaMalloc(&p, count * sizeof(T));
  }
  cudaError_t upload(const std::vector<T>& v) {
    cudaError_t e = alloc(v.size());
    if (e != cudaSuccess || v.empty()) return e;
    return cudaMemcpy(p, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice);
  }
};

}  // namespace bm

using namespace bm;

struct bm_mesh {
  HostMesh h;
  int device = 0;
  // FP64 device copies
  DBuf<double> z, inv_area, area, enx, eny, elen, in_len;
  DBuf<uint64_t> slots;
  DBuf<int64_t> eoff;
  DBuf<int32_t> eL, eR, in_cell, perm;
};

struct bm_state {
  const bm_mesh* mesh = nullptr;
  bm_params prm{};
  Params p{};
  std::vector<double> hydro_t, hydro_q;
  DBuf<double> d_hydro_t, d_hydro_q;
  DBuf<double> gn2;  // g n^2 per cell (new order)
  DBuf<double> H[2], qx[2], qy[2], u[2], v[2], c[2];
  DBuf<double> stage[3];  // caller-order staging for upload/download
  DBuf<double> vol_part, vol_out;
  DBuf<TilePartial> part;
  DBuf<int> bad;
  Ctl* ctl = nullptr;       // device
  Ctl* hctl = nullptr;      // pinned host mirror
  double* hvol = nullptr;   // pinned
  cudaStream_t stream = nullptr;   // user stream (may be the default stream)
  cudaStream_t own = nullptr;      // private stream used for graph capture
  std::map<int, cudaGraphExec_t> graphs;
  double cur_t_end = std::numeric_limits<double>::infinity();
  StepArgs<double> sa{};
  FinalizeArgs<double> fa{};
  ~bm_state() {
    for (auto& kv : graphs) cudaGraphExecDestroy(kv.second);
    if (ctl) cudaFree(ctl);
    if (hctl) cudaFreeHost(hctl);
    if (hvol) cudaFreeHost(hvol);
    if (own) cudaStreamDestroy(own);
  }
};

namespace {

const double kInf = std::numeric_limits<double>::infinity();

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

bm_status read_status(bm_state* s) {
  BM_CUDA(cudaMemcpyAsync(s->hctl, s->ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, s->stream));
  BM_CUDA(cudaStreamSynchronize(s->stream));
  if (s->hctl->status & 1) return fail(BM_ENONFINITE, "the step produced a non-finite value");
  if (s->hctl->status & 2) return fail(BM_ENEGDEPTH, "a depth fell below -h_min");
  return BM_OK;
}

// Launch the two kernels of one step on `st`.
void enqueue_step(bm_state* s, cudaStream_t st) {
  const int nt = static_cast<int>(s->mesh->h.n_tiles);
  step_fp64<<<nt, kTile, 0, st>>>(s->sa);
  finalize<double><<<1, kFinThreads, 0, st>>>(s->fa, 1);
}

bm_status get_graph(bm_state* s, int k, cudaGraphExec_t* out) {
  auto it = s->graphs.find(k);
  if (it != s->graphs.end()) {
    *out = it->second;
    return BM_OK;
  }
  cudaGraph_t g = nullptr;
  BM_CUDA(cudaStreamBeginCapture(s->own, cudaStreamCaptureModeThreadLocal));
  for (int i = 0; i < k; ++i) enqueue_step(s, s->own);
  BM_CUDA(cudaStreamEndCapture(s->own, &g));
  cudaGraphExec_t ge = nullptr;
  cudaError_t e = cudaGraphInstantiate(&ge, g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) return fail(BM_ECUDA, std::string("cudaGraphInstantiate: ") + cudaGetErrorString(e));
  s->graphs[k] = ge;
  *out = ge;
  return BM_OK;
}

// Enqueue n steps as graph launches of 32 steps plus single-step launches.
bm_status enqueue_steps(bm_state* s, int64_t n) {
  constexpr int kChunk = 32;
  if (n <= 0) return BM_OK;
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
  gather_from_user<double><<<nb, 256, 0, s->stream>>>(s->stage[0].p, s->mesh->perm.p, n, s->H[0].p, 0.0);
  gather_from_user<double><<<nb, 256, 0, s->stream>>>(s->stage[1].p, s->mesh->perm.p, n, s->qx[0].p, 0.0);
  gather_from_user<double><<<nb, 256, 0, s->stream>>>(s->stage[2].p, s->mesh->perm.p, n, s->qy[0].p, 0.0);
  BM_CUDA(cudaMemsetAsync(s->bad.p, 0, sizeof(int), s->stream));
  check_state<double><<<nb, 256, 0, s->stream>>>(s->H[0].p, s->qx[0].p, s->qy[0].p, s->mesh->z.p, n, s->bad.p);
  int bad = 0;
  BM_CUDA(cudaMemcpyAsync(&bad, s->bad.p, sizeof(int), cudaMemcpyDeviceToHost, s->stream));
  BM_CUDA(cudaStreamSynchronize(s->stream));
  if (bad & 1) return fail(BM_EINVAL, "state has a non-finite value");
  if (bad & 2) return fail(BM_EINVAL, "state has H < z_bed (a dry cell is H = z_bed)");
  Ctl c{};
  c.t = t;
  c.dt = 0;
  c.t_end = kInf;
  c.bvol = 0;
  c.parity = 0;
  c.active = 1;
  c.pad0 = 0;
  BM_CUDA(cudaMemcpyAsync(s->ctl, &c, sizeof(Ctl), cudaMemcpyHostToDevice, s->stream));
  s->cur_t_end = kInf;
  prime_fp64<<<static_cast<int>(h.n_tiles), kTile, 0, s->stream>>>(s->sa);
  finalize<double><<<1, kFinThreads, 0, s->stream>>>(s->fa, 0);
  BM_CUDA(cudaGetLastError());
  BM_CUDA(cudaStreamSynchronize(s->stream));
  return BM_OK;
}

}  // namespace

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

const char* bm_last_error(void) { return g_err.c_str(); }

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
  cudaGetDevice(&m->device);
  cudaError_t e = cudaSuccess;
  const HostMesh& h = m->h;
  if (e == cudaSuccess) e = m->z.upload(h.z);
  if (e == cudaSuccess) e = m->inv_area.upload(h.inv_area);
  if (e == cudaSuccess) e = m->area.upload(h.area);
  if (e == cudaSuccess) e = m->slots.upload(h.slots);
  if (e == cudaSuccess) e = m->eoff.upload(h.eoff);
  if (e == cudaSuccess) e = m->eL.upload(h.eL);
  if (e == cudaSuccess) e = m->eR.upload(h.eR);
  if (e == cudaSuccess) e = m->enx.upload(h.enx);
  if (e == cudaSuccess) e = m->eny.upload(h.eny);
  if (e == cudaSuccess) e = m->elen.upload(h.elen);
  if (e == cudaSuccess) e = m->in_cell.upload(h.in_cell);
  if (e == cudaSuccess) e = m->in_len.upload(h.in_len);
  if (e == cudaSuccess) e = m->perm.upload(h.perm);
  if (e != cudaSuccess) {
    delete m;
    if (e == cudaErrorMemoryAllocation) return fail(BM_ENOMEM, "bm_mesh_create: out of device memory");
    return fail(BM_ECUDA, std::string("bm_mesh_create: ") + cudaGetErrorString(e));
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

bm_status bm_state_init(const bm_mesh* m, const bm_params* prm, const double* H, const double* qx, const double* qy,
                        bm_state** out) {
  clear_error();
  if (!out) return fail(BM_EINVAL, "bm_state_init: out is NULL");
  *out = nullptr;
  if (!m) return fail(BM_EINVAL, "bm_state_init: mesh is NULL");
  bm_status st = check_params(prm);
  if (st != BM_OK) return st;
  if (prm->precision != BM_FP64) return fail(BM_EINVAL, "bm_state_init: this build steps BM_FP64 states only");
  bm_state* s = new (std::nothrow) bm_state();
  if (!s) return fail(BM_ENOMEM, "bm_state_init: out of host memory");
  s->mesh = m;
  s->prm = *prm;
  s->hydro_t.assign(prm->hydro_t, prm->hydro_t + prm->hydro_n);
  s->hydro_q.assign(prm->hydro_q, prm->hydro_q + prm->hydro_n);
  s->prm.hydro_t = s->hydro_t.data();
  s->prm.hydro_q = s->hydro_q.data();
  const HostMesh& h = m->h;
  const size_t Np = static_cast<size_t>(h.n_tiles) * kTile;
  cudaError_t e = cudaSuccess;
  for (int b = 0; b < 2 && e == cudaSuccess; ++b) {
    e = s->H[b].alloc(Np);
    if (e == cudaSuccess) e = s->qx[b].alloc(Np);
    if (e == cudaSuccess) e = s->qy[b].alloc(Np);
    if (e == cudaSuccess) e = s->u[b].alloc(Np);
    if (e == cudaSuccess) e = s->v[b].alloc(Np);
    if (e == cudaSuccess) e = s->c[b].alloc(Np);
  }
  for (int k = 0; k < 3 && e == cudaSuccess; ++k) e = s->stage[k].alloc(h.n_cells);
  if (e == cudaSuccess) e = s->part.alloc(h.n_tiles);
  if (e == cudaSuccess) e = s->vol_part.alloc(h.n_tiles);
  if (e == cudaSuccess) e = s->vol_out.alloc(1);
  if (e == cudaSuccess) e = s->bad.alloc(1);
  if (e == cudaSuccess) {
    std::vector<double> gn2(h.man.size());
    for (size_t i = 0; i < gn2.size(); ++i) gn2[i] = prm->g * h.man[i] * h.man[i];
    e = s->gn2.upload(gn2);
  }
  if (e == cudaSuccess) e = s->d_hydro_t.upload(s->hydro_t);
  if (e == cudaSuccess) e = s->d_hydro_q.upload(s->hydro_q);
  if (e == cudaSuccess) e = cudaMalloc(&s->ctl, sizeof(Ctl));
  if (e == cudaSuccess) e = cudaMallocHost(&s->hctl, sizeof(Ctl));
  if (e == cudaSuccess) e = cudaMallocHost(&s->hvol, sizeof(double));
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s->own, cudaStreamNonBlocking);
  if (e != cudaSuccess) {
    delete s;
    if (e == cudaErrorMemoryAllocation) return fail(BM_ENOMEM, "bm_state_init: out of device memory");
    return fail(BM_ECUDA, std::string("bm_state_init: ") + cudaGetErrorString(e));
  }
  s->stream = s->own;
  // zero the padding cells once so they stay inert
  for (int b = 0; b < 2; ++b) {
    cudaMemset(s->H[b].p, 0, Np * sizeof(double));
    cudaMemset(s->qx[b].p, 0, Np * sizeof(double));
    cudaMemset(s->qy[b].p, 0, Np * sizeof(double));
    cudaMemset(s->u[b].p, 0, Np * sizeof(double));
    cudaMemset(s->v[b].p, 0, Np * sizeof(double));
    cudaMemset(s->c[b].p, 0, Np * sizeof(double));
  }
  Params& p = s->p;
  p.cfl = prm->cfl;
  p.g = prm->g;
  p.h_min = prm->h_min;
  p.dt_max = prm->dt_max;
  p.cfl_mode = prm->cfl_mode;
  p.hydro_n = static_cast<int>(prm->hydro_n);
  p.hydro_t = s->d_hydro_t.p;
  p.hydro_q = s->d_hydro_q.p;
  StepArgs<double>& a = s->sa;
  for (int b = 0; b < 2; ++b) {
    a.H[b] = s->H[b].p; a.qx[b] = s->qx[b].p; a.qy[b] = s->qy[b].p;
    a.u[b] = s->u[b].p; a.v[b] = s->v[b].p; a.c[b] = s->c[b].p;
  }
  a.z = m->z.p;
  a.gn2 = s->gn2.p;
  a.inv_area = m->inv_area.p;
  a.slots = m->slots.p;
  a.eoff = m->eoff.p;
  a.eL = m->eL.p;
  a.eR = m->eR.p;
  a.enx = m->enx.p;
  a.eny = m->eny.p;
  a.elen = m->elen.p;
  a.n_cells = static_cast<int>(h.n_cells);
  a.ctl = s->ctl;
  a.part = s->part.p;
  a.p = p;
  FinalizeArgs<double>& f = s->fa;
  f.H[0] = s->H[0].p;
  f.H[1] = s->H[1].p;
  f.z = m->z.p;
  f.inv_area = m->inv_area.p;
  f.in_cell = m->in_cell.p;
  f.in_len = m->in_len.p;
  f.n_inflow = static_cast<int>(h.n_inflow);
  f.inflow_len = h.inflow_len;
  f.n_tiles = static_cast<int>(h.n_tiles);
  f.ctl = s->ctl;
  f.part = s->part.p;
  f.p = p;
  st = load_state(s, H, qx, qy, 0.0);
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
  return load_state(s, H, qx, qy, t);
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
  double* srcs[3] = {s->H[par].p, s->qx[par].p, s->qy[par].p};
  for (int k = 0; k < 3; ++k) {
    if (!outs[k]) continue;
    scatter_to_user<double><<<nb, 256, 0, s->stream>>>(srcs[k], s->mesh->perm.p, n, s->stage[k].p, 0.0);
    BM_CUDA(cudaMemcpyAsync(outs[k], s->stage[k].p, bytes, cudaMemcpyDeviceToHost, s->stream));
  }
  BM_CUDA(cudaStreamSynchronize(s->stream));
  if (t) *t = s->hctl->t;
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
    volume_partials<double><<<nt, kTile, 0, s->stream>>>(s->H[par].p, s->mesh->z.p, s->mesh->area.p,
                                                          static_cast<int>(s->mesh->h.n_cells), 0.0, s->vol_part.p);
    sum_partials<<<1, kFinThreads, 0, s->stream>>>(s->vol_part.p, nt, s->vol_out.p);
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

bm_status bm_step_timed(bm_state* s, int64_t n, double* step_kernel_ms, double* total_ms) {
  clear_error();
  if (!s) return fail(BM_EINVAL, "bm_step_timed: state is NULL");
  if (n < 1 || n > 100000) return fail(BM_EINVAL, "bm_step_timed: n_steps must be in [1, 100000]");
  if (s->cur_t_end != kInf) {
    bm_status st = set_end(s, kInf);
    if (st != BM_OK) return st;
  }
  std::vector<cudaEvent_t> ev(2 * n);
  for (auto& e : ev) {
    cudaError_t r = cudaEventCreate(&e);
    if (r != cudaSuccess) {
      for (auto& x : ev) if (x) cudaEventDestroy(x);
      return fail(BM_ECUDA, std::string("cudaEventCreate: ") + cudaGetErrorString(r));
    }
  }
  const int nt = static_cast<int>(s->mesh->h.n_tiles);
  for (int64_t k = 0; k < n; ++k) {
    cudaEventRecord(ev[2 * k], s->stream);
    step_fp64<<<nt, kTile, 0, s->stream>>>(s->sa);
    cudaEventRecord(ev[2 * k + 1], s->stream);
    finalize<double><<<1, kFinThreads, 0, s->stream>>>(s->fa, 1);
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
