// bm_internal.h -- internal data structures shared by the host mesh preparation,
// the C ABI and the CUDA kernels of the shallow-water step.
#pragma once

#include <cstddef>
#include <cstdint>
#include <string>
#include <vector>

#include "../../include/bm.h"

namespace bm {

// Cells are renumbered along a Hilbert curve and grouped in tiles of kTile
// consecutive cells; each tile owns the list of every edge incident to one of
// its cells, so one CTA evaluates each of those edges once (edges shared with
// another tile are evaluated by both; about 12 % of them on large meshes).
constexpr int kTile = 256;
// Passive species a state can carry (Section "Scalar advection-diffusion").
constexpr int kMaxSpecies = 5;
constexpr int kMaxTileEdges = 3 * kTile;

// Boundary codes stored in place of the right cell of an edge.  Edges with a boundary
// law are listed -- the inflow edges first, then the h-Q outflow edges, then the weir
// outflow edges, then the water-level edges -- and listed edge j is stored as kInflow - j.
constexpr int32_t kWall = -1;
constexpr int32_t kTransmissive = -2;
constexpr int32_t kInflow = -3;
constexpr int32_t kHqTag = -4;    // h-Q and weir edges before they are listed (mesh
constexpr int32_t kWeirTag = -5;  // preparation only)
constexpr int32_t kLevelTag = -6; // water-level edges before they are listed

// Set the thread-local error message and return the status.
bm_status fail(bm_status st, const std::string& msg);
void clear_error();

// Host-side mesh after preparation (new Hilbert numbering).
struct HostMesh {
  int64_t n_cells = 0, n_edges = 0, n_boundary = 0, n_inflow = 0;
  int64_t n_hq = 0, n_weir = 0;  // listed h-Q and weir outflow edges (after the inflow edges)
  int64_t n_level = 0;           // listed water-level edges (after the weir edges)
  int64_t n_tiles = 0;
  // per cell, new numbering (padded to n_tiles * kTile with inert cells)
  std::vector<int32_t> perm;        // new -> caller index (n_cells entries)
  std::vector<double> z, man, inv_area, area;
  std::vector<uint64_t> slots;      // 3 x 16 bit: (tile-local edge index << 1) | side (1 = right)
  // per tile edge lists (concatenated; tile t owns [eoff[t], eoff[t+1]))
  std::vector<int64_t> eoff;
  std::vector<int32_t> eL, eR;      // left cell (new id), right cell (new id) or boundary code
  std::vector<double> enx, eny, elen;
  // listed edges (inflow, h-Q, weir, level; one entry each): cell (new id), length, unit
  // normal (outward)
  std::vector<int32_t> in_cell;
  std::vector<double> in_len, in_nx, in_ny;
  // tiles whose edge list holds at least one boundary edge that can carry mass
  // (transmissive or listed; ascending)
  std::vector<int32_t> btiles;
  double inflow_len = 0;
  double z_min = 0;
};

bm_status prepare_mesh(const double* xy, int64_t n_nodes, const int32_t* tri, int64_t n_tri,
                       const double* z, const double* man, const uint8_t* tag, HostMesh* out);

#if defined(__CUDACC__)
#define BM_HD __host__ __device__ __forceinline__
#else
#define BM_HD inline
#endif

BM_HD uint32_t round4(uint32_t x) { return (x + 3u) & ~3u; }
BM_HD uint32_t align16(uint32_t x) { return (x + 15u) & ~15u; }

// Tile record: everything static one tile's step reads, as one contiguous block so a
// single bulk copy brings it into shared memory.  With ne4 / nh4 = the tile's edge /
// halo counts rounded up to a multiple of 4 and S = sizeof(T):
//   inv_area[kTile] T | slot[kTile] u32 | lr[ne4] u32 | nx[ne4] T | ny[ne4] T |
//   len[ne4] T | hidx[nh4] i32
// slot: the cell's three tile-local edge indices, 10 bits each (the side follows from
// lr: the cell is the edge's left cell iff the left index is the cell's).
// lr: left local index in bits 0..9, right local index or boundary code (signed) in
// bits 10..31.  Local index j < kTile is cell tile*kTile + j, j >= kTile is halo cell
// hidx[j - kTile] (another tile's cell, instance numbering).  Every segment is a
// multiple of 16 bytes, so records concatenate 16-byte aligned.
constexpr int kLocBits = 10;
constexpr int kMaxLocal = 1 << kLocBits;           // tile cells + halo cells
constexpr int32_t kMinCode = -(1 << 21);           // most negative code in lr
template <int S>
struct RecLayout {
  static BM_HD uint32_t ia() { return 0; }
  static BM_HD uint32_t slot() { return kTile * S; }
  static BM_HD uint32_t lr() { return kTile * S + kTile * 4; }
  static BM_HD uint32_t nx(uint32_t ne4) { return lr() + ne4 * 4; }
  static BM_HD uint32_t ny(uint32_t ne4) { return nx(ne4) + ne4 * S; }
  static BM_HD uint32_t len(uint32_t ne4) { return ny(ne4) + ne4 * S; }
  static BM_HD uint32_t hidx(uint32_t ne4) { return len(ne4) + ne4 * S; }
  static BM_HD uint32_t bytes(uint32_t ne4, uint32_t nh4) { return hidx(ne4) + nh4 * 4; }
};

// Tile records of one mesh in one precision (host side).
struct TileRecords {
  std::vector<unsigned char> data;   // concatenated records
  std::vector<uint64_t> off;         // byte offset of tile t's record
  std::vector<uint32_t> bytes;       // its size (multiple of 16)
  std::vector<uint32_t> ne_nh;       // edges | halo cells << 16
  std::vector<uint8_t> flags;        // bit 0: boundary edges that can carry mass (transmissive or
                                     // listed; walls do not count), bit 1: inflow edges, bit 3: h-Q
                                     // edges, bit 4: weir edges, bit 5: water-level edges
  uint32_t ne4_max = 0, nh4_max = 0;
};

// Build (and check) the tile records of a prepared mesh; S = 8 (FP64) or 4 (FP32).
bm_status build_tile_records(const HostMesh& m, int S, TileRecords* out);

// Device-side control block of one state (one instance).
struct Ctl {
  double t;        // current time t^n
  double dt;       // dt^n, the step the next launch takes (clipped to t_end)
  double t_end;    // run_until target (+inf for bm_step)
  double bvol;     // net boundary volume since init (FP64)
  double qscale;   // inflow: q_e = qscale * h_e^(5/3) when wsum > 0
  double quni;     // inflow: q_e = quni on every inflow edge when wsum == 0
  double Q;        // Q(t^n)
  double dt_cfl;   // dt^n before clipping to t_end
  long long steps;
  unsigned long long rmax_bits;  // max over cells of the Eq. 21 rate (bits of a double >= 0)
  unsigned int done;             // (unused)
  int parity;      // which state buffer holds U^n
  int active;      // 0 once t reached t_end
  int clipped;     // dt^n was clipped to t_end - t^n
  int wpos;        // wsum > 0
  int status;      // bit 0: non-finite value, bit 1: negative depth
  float dt_f;      // dt and quni rounded once for FP32-bulk steps
  float quni_f;
  double rb;            // max inflow-edge rate of Eq. 21 at t^{n+1} (written mid-launch)
  // (in_done, b_done: 8-byte aligned, counted together by a 64-bit atomicAdd)
  unsigned int in_done; // inflow tiles of the current launch that finished  } one 64-bit word
  unsigned int b_done;  // boundary tiles of the current launch that finished } (one atomic)
  double rb_out;        // max h-Q-edge rate of Eq. 21 at t^{n+1} (written mid-launch)
  unsigned int hq_done; // h-Q tiles of the current launch that finished
  unsigned int pad_u;
};

static_assert(sizeof(Ctl) % 16 == 0, "Ctl is bulk-copied: its size must be a multiple of 16");
static_assert(offsetof(Ctl, in_done) % 8 == 0 && offsetof(Ctl, b_done) == offsetof(Ctl, in_done) + 4,
              "in_done and b_done form one 8-byte word");

// One work item of a step launch: a tile of an instance, with the addresses its bulk
// copies read (the items of one instance are consecutive and in tile order, so item
// index = the instance's first item + tile; 48 bytes, 16-byte aligned).
struct PipeItem {
  const unsigned char* rec;  // the tile's record
  const void* desc;          // the instance's descriptor (InstDesc<T>)
  Ctl* ctl;                  // the instance's control block
  uint32_t rec_bytes;        // record size (multiple of 16)
  int32_t tile;
  uint32_t ne_nh;            // edges | halo cells << 16
  int32_t inst;              // instance index within the launch
  uint32_t flags;            // bit 0: the tile has boundary edges that can carry mass, bit 1:
                             // inflow edges, bit 2: source cells, bit 3: h-Q edges, bit 4: weir edges,
                             // bit 5: water-level edges
  uint32_t bidx;             // boundary tiles: rank among the instance's boundary tiles
};
static_assert(sizeof(PipeItem) == 48, "PipeItem layout");

// Work items every launch takes (the "fixed" items): those with any of these flags, and
// item 0 of a work list.  The others are taken only when the previous launch listed
// them (see step_pipe).  kFixedMark: their entries in the list marks.
constexpr uint32_t kFixedFlags = 63u;
constexpr int kFixedMark = 0x7fffffff;
// Launch stamps restart (with a full launch) before they reach this value (marks hold
// 2 x stamp + 1 at most, below kFixedMark).
constexpr int kStampMax = 1 << 29;
// Scheduling counters of a work list (int entries).
constexpr int kSchedInts = 16;

// Per-tile reduction slot written by the step kernel.
struct TilePartial {
  double bflux;  // sum over the tile's boundary edges of l * F_h (outward)
  double pad;
};

// Kernel parameters (plain values).
struct Params {
  double cfl, g, h_min, dt_max;
  int cfl_mode;
  int hydro_n;
  const double* hydro_t;
  const double* hydro_q;
  float g_f, hg_f, hmin_f, pad_f;  // g, g/2, h_min rounded once for FP32-bulk steps
};

}  // namespace bm
