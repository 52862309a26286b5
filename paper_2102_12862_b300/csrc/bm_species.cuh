// bm_species.cuh -- passive species advected with the water (BASEMENT v3, Section
// "Scalar advection-diffusion", Eq. 8 with the diffusion and source terms off).
//
// Unknowns q_c = h phi_c per cell and species.  The advective flux of a species through
// an edge is HLLC's contact-wave flux, the formula the tangential momentum uses with
// phi_c in place of the tangential velocity: l F_h phi_c of the upwind side of the
// contact -- the solver the numerics of that section name for the advective part.  The
// step kernel (its optional-output instantiation) exports, per tile edge, l F_h and the
// upwind side; this kernel, launched after each step, applies
//   q_c^{n+1} = q_c^n - dt / |Omega| sum_j (+-) l F_h phi_c,upwind
// with phi_c = q_c / h on U^n (0 where h <= 0), the inflow concentration on inflow
// edges, none from outside through water-level edges, nothing through walls, and
// q_c = 0 in a cell that ends the step dry.
#pragma once

#include "bm_kernels.cuh"
#include "bm_step.cuh"

namespace bm {

template <typename T>
struct SpeciesArgs {
  const PipeItem* items;          // the state's work list: one item per tile
  T* hc[kMaxSpecies][2];          // q_c per species and state buffer
  T c_in[kMaxSpecies];            // concentration of the water entering through inflow edges
  const T* H[2];
  const T* Hlo[2];                // FP32-bulk: low part of the surface pair (else null)
  const T* z;
  const Ctl* ctl;                 // after the step: U^{n+1} in buffer ctl->parity
  const T* ex_flux;               // the step's exports (see InstDesc)
  const unsigned char* ex_right;
  const unsigned char* ex_valid;
  const double* ex_dt;
  unsigned char* zmask;           // per tile: bit b set = q_c of every species is 0 in buffer b
  int ex_stride;
  int n_species;
  int n_cells;
  int n_inflow;                   // listed edges below n_inflow are inflow edges (outflow above)
  int n_level0;                   // listed edges from n_level0 on are water-level edges
};

// One CTA per work item (a 256-cell tile).  Dynamic shared memory: (2 nloc_max +
// ne4_max) values of T, nloc_max = 256 + the largest halo of the mesh.
// Launched as a programmatic dependent of the step: it waits for the whole step grid.
// A quiet tile (no flux: dry and at rest, U^{n+1} = U^n) whose species are zero in both
// buffers stays zero and is left alone: the dry floodplain costs two bytes per tile.
template <typename T>
__global__ void __launch_bounds__(kTile) species_step(const SpeciesArgs<T> a, int nloc_max) {
  grid_dep_wait();
  const double dt = *a.ex_dt;
  if (!(dt >= 0.0)) return;  // the instance did not step
  const PipeItem& it0 = a.items[blockIdx.x];
  const unsigned char zm = a.zmask[it0.tile];
  const bool valid = a.ex_valid[it0.tile] != 0;
  if (!valid && (zm & 3u) == 3u) return;
  using RL = RecLayout<sizeof(T)>;
  extern __shared__ __align__(16) unsigned char smem_sp[];
  T* hs = reinterpret_cast<T*>(smem_sp);  // 1 / h^n of the tile's and halo cells (0 where dry)
  T* ph = hs + nloc_max;                   // phi of the species being advected
  T* fs = ph + nloc_max;                   // its edge fluxes
  const PipeItem& it = a.items[blockIdx.x];
  const int tile = it.tile, tid = threadIdx.x;
  const unsigned char* rec = it.rec;
  const uint32_t nn = it.ne_nh;
  const int ne = static_cast<int>(nn & 0xffffu), nh = static_cast<int>(nn >> 16);
  const uint32_t ne4 = round4(static_cast<uint32_t>(ne));
  const int32_t* hidx = reinterpret_cast<const int32_t*>(rec + RL::hidx(ne4));
  const uint32_t* lr = reinterpret_cast<const uint32_t*>(rec + RL::lr());
  const int pn = a.ctl->parity, po = pn ^ 1;
  auto depth = [&](int buf, int g) -> T {
    const T lo = a.Hlo[buf] ? a.Hlo[buf][g] : T(0);
    return depth_of(a.H[buf][g], lo, a.z[g]);
  };
  auto cell = [&](int j) -> int { return j < kTile ? tile * kTile + j : hidx[j - kTile]; };
  // one reciprocal per cell for all species (FP64 division is slow on this part: a
  // Newton-refined hardware reciprocal, within 2 ulp of the quotient)
  for (int j = tid; j < kTile + nh; j += kTile) {
    const int g = cell(j);
    const T h = g < a.n_cells ? depth(po, g) : T(0);
    hs[j] = h > T(0) ? f_div(T(1), h) : T(0);
  }
  const int i = tile * kTile + tid;
  const bool own = i < a.n_cells;
  T hnew = T(0), ia = T(0);
  uint32_t sl = 0;
  if (own) {
    hnew = depth(pn, i);
    ia = reinterpret_cast<const T*>(rec + RL::ia())[tid];
    sl = reinterpret_cast<const uint32_t*>(rec + RL::slot())[tid];
  }
  const T tdt = static_cast<T>(dt);
  bool allz = true;  // every value this thread writes is zero
  __syncthreads();
  for (int c = 0; c < a.n_species; ++c) {
    for (int j = tid; j < kTile + nh; j += kTile) {
      const int g = cell(j);
      const T rh = hs[j];
      ph[j] = (g < a.n_cells && rh > T(0)) ? a.hc[c][po][g] * rh : T(0);
    }
    __syncthreads();
    for (int k = tid; k < ne; k += kTile) {
      T f = T(0);
      if (valid) {
        const size_t o = static_cast<size_t>(tile) * static_cast<size_t>(a.ex_stride) + k;
        const T fh = a.ex_flux[o];
        if (fh != T(0)) {
          const uint32_t w = lr[k];
          const int lL = static_cast<int>(w & (kMaxLocal - 1));
          const int R = static_cast<int32_t>(w) >> kLocBits;
          if (R <= kInflow && kInflow - R < a.n_inflow) {
            f = fh * a.c_in[c];  // the inflow brings its concentration
          } else if (R <= kInflow && kInflow - R >= a.n_level0) {
            // a water-level edge: the contact's upwind side, the water outside carrying none
            f = a.ex_right[o] ? T(0) : fh * ph[lL];
          } else {  // an outflow edge takes the inside cell's
            const int lR = R >= 0 ? R : lL;  // transmissive: the outside equals the inside
            f = fh * (a.ex_right[o] ? ph[lR] : ph[lL]);
          }
        }
      }
      fs[k] = f;
    }
    __syncthreads();
    if (own) {
      T sum = T(0);
#pragma unroll
      for (int q = 0; q < 3; ++q) {
        const int e = static_cast<int>((sl >> (kLocBits * q)) & (kMaxLocal - 1));
        const bool left = (lr[e] & (kMaxLocal - 1)) == static_cast<uint32_t>(tid);
        sum += left ? fs[e] : -fs[e];
      }
      const T v = hnew > T(0) ? a.hc[c][po][i] - tdt * ia * sum : T(0);
      a.hc[c][pn][i] = v;
      allz = allz && v == T(0);
    }
    __syncthreads();
  }
  allz = __syncthreads_and(allz) != 0;
  if (tid == 0) a.zmask[tile] = static_cast<unsigned char>(allz ? (zm | (1u << pn)) : (zm & ~(1u << pn)));
}

}  // namespace bm
