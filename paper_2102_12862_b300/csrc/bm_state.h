// bm_state.h -- host-side objects behind the opaque handles of include/bm.h.
#pragma once

#include <cuda_runtime.h>

#include <map>
#include <mutex>
#include <sstream>
#include <string>
#include <vector>

#include "bm_internal.h"

namespace bm {

#define BM_CUDA(call)                                                                          \
  do {                                                                                         \
    cudaError_t e_ = (call);                                                                   \
    if (e_ != cudaSuccess) {                                                                   \
      std::ostringstream os_;                                                                  \
      os_ << #call << ": " << cudaGetErrorString(e_);                                          \
      return ::bm::fail(BM_ECUDA, os_.str());                                                  \
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
  size_t bytes() const { return n * sizeof(T); }
};

// Per-precision state arrays of one instance (new cell numbering, padded).
template <typename T>
struct Buffers {
  DBuf<T> H[2], Hlo[2], qx[2], qy[2];
  DBuf<T> z, gn2, in_pw, in_hs;
  DBuf<double> trk_t;  // flood tracking (bm_state_track): front arrival time,
  DBuf<T> trk[4];      // maxima of depth, |u|, |q|, bed shear stress
  cudaError_t alloc_tracking(size_t np) {
    cudaError_t e = trk_t.p ? cudaSuccess : trk_t.alloc(np);
    for (int k = 0; k < 4 && e == cudaSuccess; ++k)
      if (!trk[k].p) e = trk[k].alloc(np);
    return e;
  }
  // passive species (bm_state_set_scalars): q_c = h phi_c of K species per state
  // buffer (species c at c * np), and the step kernel's exports per tile edge
  DBuf<T> hc[2];
  DBuf<T> ex_flux;
  DBuf<unsigned char> ex_right, ex_valid, zmask;  // zmask: per tile, species all zero per buffer
  DBuf<double> ex_dt;
  cudaError_t alloc_species(size_t np, int k, size_t n_tiles, size_t stride) {
    cudaError_t e = cudaSuccess;
    for (int b = 0; b < 2 && e == cudaSuccess; ++b) {
      e = hc[b].alloc(np * static_cast<size_t>(k));
      if (e == cudaSuccess) e = cudaMemset(hc[b].p, 0, hc[b].bytes());
    }
    if (e == cudaSuccess && !ex_flux.p) e = ex_flux.alloc(n_tiles * stride);
    if (e == cudaSuccess && !ex_right.p) e = ex_right.alloc(n_tiles * stride);
    if (e == cudaSuccess && !ex_valid.p) e = ex_valid.alloc(n_tiles);
    if (e == cudaSuccess && !ex_dt.p) e = ex_dt.alloc(1);
    if (e == cudaSuccess && !zmask.p) e = zmask.alloc(n_tiles);
    if (e == cudaSuccess) e = cudaMemset(zmask.p, 0, zmask.bytes());  // not known to be zero
    if (e == cudaSuccess) e = cudaMemset(ex_valid.p, 0, ex_valid.bytes());
    if (e == cudaSuccess) e = cudaMemset(ex_dt.p, 0xff, sizeof(double));  // -NaN: no step exported
    return e;
  }
  void free_species() {
    hc[0].release(); hc[1].release();
    ex_flux.release(); ex_right.release(); ex_valid.release(); ex_dt.release(); zmask.release();
  }
  cudaError_t alloc(size_t np, size_t n_inflow, bool pair) {
    cudaError_t e = cudaSuccess;
    for (int b = 0; b < 2 && e == cudaSuccess; ++b) {
      e = H[b].alloc(np);
      if (e == cudaSuccess && pair) e = Hlo[b].alloc(np);  // FP32-bulk keeps H as a pair
      if (e == cudaSuccess) e = qx[b].alloc(np);
      if (e == cudaSuccess) e = qy[b].alloc(np);
    }
    if (e == cudaSuccess) e = z.alloc(np);
    if (e == cudaSuccess) e = in_pw.alloc(n_inflow > 0 ? n_inflow : 1);
    if (e == cudaSuccess) e = in_hs.alloc(n_inflow > 0 ? n_inflow : 1);
    // zero everything once so padding cells stay inert
    for (int b = 0; b < 2 && e == cudaSuccess; ++b) {
      DBuf<T>* bufs[4] = {&H[b], &Hlo[b], &qx[b], &qy[b]};
      for (auto* x : bufs)
        if (e == cudaSuccess && x->p) e = cudaMemset(x->p, 0, x->bytes());
    }
    if (e == cudaSuccess) e = cudaMemset(in_pw.p, 0, in_pw.bytes());
    if (e == cudaSuccess) e = cudaMemset(in_hs.p, 0, in_hs.bytes());
    return e;
  }
  size_t bytes() const {
    size_t b = z.bytes() + gn2.bytes() + in_pw.bytes() + in_hs.bytes() + trk_t.bytes();
    for (int k = 0; k < 4; ++k) b += trk[k].bytes();
    b += hc[0].bytes() + hc[1].bytes() + ex_flux.bytes() + ex_right.bytes() + ex_valid.bytes() + ex_dt.bytes() + zmask.bytes();
    for (int k = 0; k < 2; ++k)
      b += H[k].bytes() + Hlo[k].bytes() + qx[k].bytes() + qy[k].bytes();
    return b;
  }
};

}  // namespace bm

struct bm_mesh {
  bm::HostMesh h;
  // Device data is created on first use by a state (bm_mesh_create needs no GPU).
  std::mutex mu;
  int device = -1;
  bool on_device = false;
  bm::DBuf<double> z, inv_area, area, in_len, in_lia, in_nx, in_ny;
  bm::DBuf<int32_t> in_cell, btiles, perm;
  bool has32 = false;  // FP32 copies for FP32-bulk states
  bm::DBuf<float> inv_area32, in_len32;
  // tile records, host and device, per precision (0: FP64, 1: FP32)
  bm::TileRecords rec[2];
  bool rec_built[2] = {false, false};
  bm::DBuf<unsigned char> rec_dev[2];
};

namespace bm {
// The work list of a step launch and the shared-memory layout it needs.
struct StepList {
  DBuf<PipeItem> items;
  DBuf<int> sched;  // the kernel's scheduling counters (kSchedInts; see step_pipe)
  DBuf<int> early;  // 2 x n: the items a launch lists for the next (front and back parts)
  DBuf<int> mark;   // 2 x n: per launch parity, the stamp of the launch an item is listed for
  DBuf<int> fixed;  // the items every launch takes (kFixedFlags, and item 0)
  DBuf<int> inst_item;  // per instance: its first item
  std::vector<bm_state*> members;
  int n = 0;
  int n_fixed = 0;
  uint32_t ne4 = 4, nh4 = 4;
  size_t smem = 0;
  int occupancy = 1;  // resident CTAs per SM at this shared-memory size
  int static16 = -1;  // static share of the tickets in sixteenths (-1: the precision's default)
  int slots = 0;      // tile slots of the step kernel asked for (2, 3, 4; 0 the default; levels
                      // 1 and 2 run 3)
  int claim = -1;     // work-item claiming: 0 ahead, 1 after each issue, 2 once a slot is free,
                      // 3 also once the tile before is past its edges; -1 the default
  int extra = 0;  // the step kernel's feature level the members need (0 none; 1 tracking or
                 // species; 2 also sources or log-law friction)
};
}  // namespace bm

struct bm_state {
  const bm_mesh* mesh = nullptr;
  bm_params prm{};
  bm::Params p{};
  int prec = BM_FP64;
  double datum = 0.0;  // FP32-bulk: H and z are stored as offsets from it
  std::vector<double> hydro_t, hydro_q;
  bm::DBuf<double> d_hydro_t, d_hydro_q;
  bm::Buffers<double> b64;
  bm::Buffers<float> b32;
  bm::DBuf<double> stage[3];  // caller-order staging for upload/download
  bm::DBuf<double> vol_part, vol_out;
  bm::DBuf<bm::TilePartial> part;
  bm::DBuf<int> bad;
  bm::DBuf<unsigned char> desc;   // one InstDesc<T> (device copy)
  std::vector<unsigned char> hdesc;  // host copy of the descriptor
  bm::StepList list;                 // the state's tiles as a work list of one instance
  // the work list whose launches stepped the state last (null: none since the state's
  // arrays or features changed); another list resets its scheduling state first
  const bm::StepList* last_list = nullptr;
  long long desc_epoch = 0;  // counts the rebuilds of the state's descriptor (feature setters)
  bool no_skip = false;  // bm_state_set_tile_skipping(s, 0): every launch takes every tile
  bm::Ctl* ctl = nullptr;   // device
  bm::Ctl* hctl = nullptr;  // pinned host mirror
  double* hvol = nullptr;   // pinned
  int* hbad = nullptr;      // pinned
  cudaStream_t stream = nullptr;  // stream the work is ordered on
  cudaStream_t own = nullptr;     // private stream, also used for graph capture
  std::map<int, cudaGraphExec_t> graphs;
  double cur_t_end = 0.0;
  int grid = 0;         // CTAs of the persistent step launch
  int ctas_per_sm = 0;  // launch shape (0: as many as fit)
  double trk_harr = 0.0;  // flood tracking: arrival threshold depth (tracking is on
                          // once the tracking arrays exist)
  // external sources (bm_state_set_sources): region of each cell (new numbering),
  // per region kind, mode, series and area; S_h per region (T of the precision);
  // per tile whether it holds a source cell (never quiet)
  int n_src = 0;
  bm::DBuf<int32_t> src_reg, src_kind, src_mode;
  bm::DBuf<long long> src_off;
  bm::DBuf<double> src_t, src_v, src_area, src_rate64;
  bm::DBuf<float> src_rate32;
  std::vector<uint8_t> src_tile;
  // bed evolution (bm_state_set_morpho; FP64): parameters, per-cell bed change of the
  // step, the dt of the step being taken
  int fr_law = 0;  // friction closure (bm_state_set_friction): 0 Manning, 1 Chezy, 2 Bezzola
  bool morpho = false;
  double mo_par[6] = {};  // porosity, s, d, alpha, m, theta_cr
  bm::DBuf<double> mo_dz, mo_dt;
  // outflow laws (bm_state_set_outflow): the h-Q relation's table (absolute stage,
  // discharge) and the weir's crest (absolute) and Poleni factor
  bm::DBuf<double> hq_s, hq_q;
  int hq_n = 0;
  double weir_crest = 0.0, weir_mu = 0.0;
  // the water-level series of the level edges (bm_state_set_level): times, absolute
  // surface elevations; zh_n = 0: the level edges are walls
  bm::DBuf<double> zh_t, zh_v;
  int zh_n = 0;
  int n_species = 0;                    // passive species carried (0: none)
  double c_in[bm::kMaxSpecies] = {};    // their concentration in the inflow
  template <typename T>
  bm::Buffers<T>& buf();
  ~bm_state() {
    for (auto& kv : graphs) cudaGraphExecDestroy(kv.second);
    if (ctl) cudaFree(ctl);
    if (hctl) cudaFreeHost(hctl);
    if (hvol) cudaFreeHost(hvol);
    if (hbad) cudaFreeHost(hbad);
    if (own) cudaStreamDestroy(own);
  }
};

template <>
inline bm::Buffers<double>& bm_state::buf<double>() { return b64; }
template <>
inline bm::Buffers<float>& bm_state::buf<float>() { return b32; }

namespace bm {
const char* last_error();
bm_status check_params(const bm_params* p);
bm_status status_of(const Ctl& c);
bm_status load_state(bm_state* s, const double* H, const double* qx, const double* qy, double t);
void state_desc_bytes(bm_state* s, std::vector<unsigned char>* out);
// Device data of a mesh for a precision (uploads on first use; thread-safe).
bm_status mesh_on_device(bm_mesh* m, int prec);
// Work list over the tiles of several states; descs[k] = device address of member k's
// descriptor.
bm_status build_step_list(const std::vector<bm_state*>& members, const std::vector<const void*>& descs,
                          StepList* out);
// Grid of a step launch for a launch shape (ctas_per_sm = 0: all that fit).
bm_status list_occupancy(int prec, StepList* l);
// The per-state kernels around a step launch: before it, the external sources' rates at
// t^n and the bed update's copy of dt^n; after it, the passive species' advection and
// the bed update (nothing for a state without those features).
void state_pre_step(bm_state* s, cudaStream_t st);
void state_post_step(bm_state* s, cudaStream_t st);
// The tile slots a list's kernel runs with, and the counts the autotuner tries.
int list_slots(const StepList& l);
int list_claim(int prec, const StepList& l);
std::vector<int> slot_candidates(const StepList& l);
// The step kernel's feature level a state needs (see StepList::extra).
int state_extra_level(const bm_state* s);
int step_grid(const StepList& l, int ctas_per_sm);
void launch_work(int prec, const StepList& l, int grid, int prime, cudaStream_t st, int withhold = 0);
// Whether launches may skip the tiles the previous launch did not list (no member
// carries passive species or bed evolution, whose kernels read every tile).
bool state_listed_ok(const bm_state* s);
// Before a launch of list l on stream st: unless every member was last stepped by l,
// reset l's scheduling state (counters, lists, marks), so the next launch takes every tile.
void ensure_list(StepList* l, cudaStream_t st);
}  // namespace bm
