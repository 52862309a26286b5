// bm_kernels.cuh -- device code of the explicit shallow-water step (sm_103a).
//
// One step of one instance (BASEMENT v3, Section "Numerical solution",
// "Hydrodynamics"), processed tile by tile (256 consecutive Hilbert-ordered cells):
//   phase 0  stage the tile's cells (H, z, u, v, c) in shared memory;
//   phase 1  each tile edge once: modified states on max(z_L, z_R), HLLC flux in
//            the edge frame (Toro wave speeds), pre-balanced pressure correction,
//            wall / transmissive / discharge-inflow boundary states;
//   phase 2  each cell gathers its three edge contributions in local edge order
//            (Eq. 12), applies the split Manning friction (Eq. 2, Table 1, two
//            semi-implicit stages), zeroes q below h_min, writes U^{n+1} and reduces
//            lambda/rho of Eq. 21 for the next dt;
//   finalize the CTA that completes an instance's last tile reduces the instance's
//            partials in a fixed order (dt^{n+1}, t^{n+1}, boundary volume, inflow
//            split for t^{n+1}) -- no second launch, no spin-wait.
// One launch steps every instance of a work list (a batch of uneven meshes, each
// with its own dt); a single state is a batch of one.
#pragma once

#include <cuda_runtime.h>

#include <cfloat>
#include <cstdint>

#include "bm_internal.h"

namespace bm {

// Everything one instance's tiles need; lives in device memory.
template <typename T>
struct InstDesc {
  T* H[2];    // free surface (FP32-bulk: hi part of the offset from the datum)
  T* Hlo[2];  // FP32-bulk only: lo part of the free surface
  T* qx[2];
  T* qy[2];
  T* u[2];   // FP64 only: velocity of the cell (0 at or below h_min)
  T* v[2];
  T* c[2];   // FP64 only: sqrt(g max(0, h))
  const T* z;
  const T* gn2;       // g n^2
  const T* inv_area;  // 1 / |Omega_i|
  const uint64_t* slots;
  const int64_t* eoff;
  const int32_t* eL;
  const int32_t* eR;
  const T* enx;
  const T* eny;
  const T* elen;
  const int32_t* in_cell;  // inflow edge j: its cell
  const T* in_len;         //                its length
  T* in_pw;                //                h^(5/3) of the cell (0 at or below h_min)
  T* in_hs;                //                max(0, h) of the cell
  const int32_t* btiles;   // tiles with boundary edges
  Ctl* ctl;
  TilePartial* part;
  Params p;
  double inflow_len;
  int n_inflow;
  int n_btiles;
  int n_cells;
  int n_tiles;
};

// ------------------------------------------------------------------ helpers

// Deterministic block reductions (fixed shuffle tree, then warp 0 over warps).
template <int NT, typename V>
__device__ __forceinline__ V block_max(V x, V* sbuf) {
  for (int o = 16; o > 0; o >>= 1) x = fmax(x, __shfl_xor_sync(0xffffffffu, x, o));
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  __syncthreads();
  if (lane == 0) sbuf[w] = x;
  __syncthreads();
  if (w == 0) {
    x = lane < NT / 32 ? sbuf[lane] : V(0);
    for (int o = 16; o > 0; o >>= 1) x = fmax(x, __shfl_xor_sync(0xffffffffu, x, o));
  }
  return x;  // valid in thread 0
}

template <int NT>
__device__ __forceinline__ double block_sum(double x, double* sbuf) {
  for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  __syncthreads();
  if (lane == 0) sbuf[w] = x;
  __syncthreads();
  if (w == 0) {
    x = lane < NT / 32 ? sbuf[lane] : 0.0;
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
  }
  return x;  // valid in thread 0
}

__device__ __forceinline__ double hydrograph(const Params& p, double t) {
  if (p.hydro_n <= 0) return 0.0;
  if (t <= p.hydro_t[0]) return p.hydro_q[0];
  for (int i = 1; i < p.hydro_n; ++i) {
    if (t <= p.hydro_t[i]) {
      double w = (t - p.hydro_t[i - 1]) / (p.hydro_t[i] - p.hydro_t[i - 1]);
      return p.hydro_q[i - 1] + w * (p.hydro_q[i] - p.hydro_q[i - 1]);
    }
  }
  return p.hydro_q[p.hydro_n - 1];
}

// Elementary functions.  FP64: the IEEE-rounded library functions (the path the
// oracle is checked against at 1e-11).  FP32-bulk: the hardware approximations
// (MUFU reciprocal square root, reciprocal, base-2 logarithm and exponent), a few
// ulp each -- far inside that mode's 1e-4 m accuracy target and deterministic, so
// both sides of an edge still compute identical values.
__device__ __forceinline__ double f_sqrt(double x) { return sqrt(x); }
__device__ __forceinline__ double f_div(double a, double b) { return a / b; }
__device__ __forceinline__ double f_cbrt(double x) { return cbrt(x); }
__device__ __forceinline__ float f_sqrt(float x) { return x > 0.0f ? x * rsqrtf(x) : 0.0f; }
__device__ __forceinline__ float f_div(float a, float b) { return __fdividef(a, b); }
__device__ __forceinline__ float f_exp2(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ float f_cbrt(float x) { return f_exp2(__log2f(x) * (1.0f / 3.0f)); }  // x > 0

// h^(5/3) for h > 0, through the cube root.
template <typename T>
__device__ __forceinline__ T pow53(T h) {
  const T r = f_cbrt(h);
  return h * r * r;
}

// HLLC flux in the edge frame for the modified depths hL, hR (>= 0) with their
// celerities cL = sqrt(g hL), cR = sqrt(g hR); un/ut are normal/tangential
// velocities.  Wave speeds: two-rarefaction star estimates when both sides are
// wet, exact dry-front speeds when one side is dry.  pL, pR = g/2 h^2 are
// returned so the caller subtracts exactly the same values.
template <typename T>
__device__ __forceinline__ void hllc(T hL, T unL, T utL, T cL, T hR, T unR, T utR, T cR, T hg, T& F0, T& F1,
                                     T& F2, T& pL, T& pR) {
  const T half = T(0.5), quarter = T(0.25), two = T(2), zero = T(0);
  const T us = half * (unL + unR) + cL - cR;
  const T cs = half * (cL + cR) + quarter * (unL - unR);
  T SL = fmin(unL - cL, us - cs);
  T SR = fmax(unR + cR, us + cs);
  const bool ldry = !(hL > zero), rdry = !(hR > zero);
  SL = ldry ? unR - two * cR : (rdry ? unL - cL : SL);
  SR = ldry ? unR + cR : (rdry ? unL + two * cL : SR);
  pL = hg * hL * hL;
  pR = hg * hR * hR;
  const T FL0 = hL * unL, FL1 = FL0 * unL + pL, FL2 = FL0 * utL;
  const T FR0 = hR * unR, FR1 = FR0 * unR + pR, FR2 = FR0 * utR;
  const T rd = f_div(T(1), SR - SL);
  const T H0 = FL0 - SL * ((FR0 - FL0) - SR * (hR - hL)) * rd;
  const T H1 = FL1 - SL * ((FR1 - FL1) - SR * (FR0 - FL0)) * rd;
  // sign of the contact speed S* = num / den with den < 0 whenever a side is wet
  const T num = SL * hR * (unR - SR) - SR * hL * (unL - SL);
  const T H2 = H0 * (num <= zero ? utL : utR);
  if (SL >= zero) {
    F0 = FL0; F1 = FL1; F2 = FL2;
  } else if (SR <= zero) {
    F0 = FR0; F1 = FR1; F2 = FR2;
  } else {
    F0 = H0; F1 = H1; F2 = H2;
  }
  if (ldry && rdry) {
    F0 = zero; F1 = zero; F2 = zero;
  }
}

// Velocity (0 at or below h_min) and celerity sqrt(g max(0, h)) of a cell of depth h.
template <typename T>
__device__ __forceinline__ void cell_derived(T h, T qx, T qy, T hmin, T g, T& u, T& v, T& c) {
  u = T(0);
  v = T(0);
  if (h > hmin) {
    const T rh = f_div(T(1), h);
    u = qx * rh;
    v = qy * rh;
  }
  c = f_sqrt(g * fmax(T(0), h));
}

// The free surface H of an FP32-bulk cell is the unevaluated sum hi + lo of two
// floats (offset from the FP64 datum); FP64 cells have lo = 0.  Depths are formed
// as (hi - z) + lo, so near-equal hi and z cancel exactly (Sterbenz) and the lo
// part keeps what a single float would round away.
template <typename T>
__device__ __forceinline__ T depth_of(T hi, T lo, T z) {
  return (hi - z) + lo;
}

// (hi, lo) += d without rounding error in the pair: Knuth's TwoSum of hi and d,
// then Dekker's Fast2Sum renormalisation (|s| >= |lo + e| holds for these
// magnitudes).  Uses round-to-nearest intrinsics so nothing is contracted.
__device__ __forceinline__ void pair_add(float& hi, float& lo, float d) {
  const float s = __fadd_rn(hi, d);
  const float bp = __fsub_rn(s, hi);
  const float ap = __fsub_rn(s, bp);
  const float e = __fadd_rn(__fsub_rn(hi, ap), __fsub_rn(d, bp));
  const float t = __fadd_rn(lo, e);
  const float h2 = __fadd_rn(s, t);
  lo = __fsub_rn(t, __fsub_rn(h2, s));
  hi = h2;
}

// lambda_ij / rho_ij of Eq. 21 for one cell (max over its edges, cfl_mode 0) or
// sum_j l_ij lambda_ij / |Omega_i| (cfl_mode 1), from the tile's staged geometry.
template <typename T>
__device__ __forceinline__ T cell_rate(const T* nxs, const T* nys, const T* ls, const int (&idx)[3], T u, T v, T c,
                                       T ia, int cfl_mode) {
  T rmax = T(0), ssum = T(0);
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const T lam = fabs(u * nxs[idx[k]] + v * nys[idx[k]]) + c;  // |u.n| does not depend on the side
    const T ll = lam * ls[idx[k]];
    rmax = fmax(rmax, T(0.75) * ll * ia);
    ssum += ll;
  }
  return cfl_mode == 1 ? ssum * ia : rmax;
}

// Per-instance finalize, run by every thread of the CTA that completed the
// instance's last tile.  advance = 1 after a step, 0 after prime.
template <typename T>
__device__ void finalize_instance(const InstDesc<T>& a, int advance, double* sred, double* sbc) {
  Ctl* ctl = a.ctl;
  const int tid = threadIdx.x;
  double bs = 0.0;
  for (int j = tid; j < a.n_btiles; j += kTile) bs += __ldcg(&a.part[a.btiles[j]].bflux);
  bs = block_sum<kTile>(bs, sred);
  if (tid == 0) {
    if (advance) {
      const double dt = ctl->dt;
      ctl->bvol += -dt * bs;
      ctl->t = ctl->clipped ? ctl->t_end : ctl->t + dt;
      ctl->parity ^= 1;
      ctl->steps += 1;
    }
    sbc[0] = ctl->t;
  }
  __syncthreads();
  const double t = sbc[0];
  const double g = a.p.g;
  // inflow distribution at the new time (conveyance weights l h^(5/3))
  double wsum = 0.0;
  for (int j = tid; j < a.n_inflow; j += kTile)
    wsum += static_cast<double>(a.in_len[j]) * static_cast<double>(__ldcg(&a.in_pw[j]));
  wsum = block_sum<kTile>(wsum, sred);
  if (tid == 0) sbc[1] = wsum;
  __syncthreads();
  wsum = sbc[1];
  const double Q = hydrograph(a.p, t);
  const bool wpos = wsum > 0.0;
  const double qscale = wpos ? Q / wsum : 0.0;
  const double quni = (!wpos && a.inflow_len > 0.0) ? Q / a.inflow_len : 0.0;
  double rb = 0.0;
  for (int j = tid; j < a.n_inflow; j += kTile) {
    const double q = wpos ? qscale * static_cast<double>(__ldcg(&a.in_pw[j])) : quni;
    if (q > 0.0) {
      const double hs = static_cast<double>(__ldcg(&a.in_hs[j]));
      const double hb = fmax(hs, cbrt(q * q / g));
      const double lb = q / hb + sqrt(g * hb);
      const double ll = lb * static_cast<double>(a.in_len[j]) * static_cast<double>(a.inv_area[a.in_cell[j]]);
      rb = fmax(rb, a.p.cfl_mode == 0 ? 0.75 * ll : ll);
    }
  }
  rb = block_max<kTile, double>(rb, sred);
  if (tid == 0) {
    const double rcell = __longlong_as_double(static_cast<long long>(atomicExch(&ctl->rmax_bits, 0ull)));
    const double r = fmax(rcell, rb);
    double dtc = r > 0.0 ? a.p.cfl / r : a.p.dt_max;
    if (dtc > a.p.dt_max) dtc = a.p.dt_max;
    ctl->dt_cfl = dtc;
    double dt = dtc;
    int clipped = 0;
    if (dt >= ctl->t_end - t) {
      dt = ctl->t_end - t;
      clipped = 1;
    }
    ctl->dt = dt;
    ctl->dt_f = static_cast<float>(dt);
    ctl->clipped = clipped;
    ctl->active = t < ctl->t_end ? 1 : 0;
    ctl->Q = Q;
    ctl->qscale = qscale;
    ctl->quni = quni;
    ctl->quni_f = static_cast<float>(quni);
    ctl->wpos = wpos ? 1 : 0;
    ctl->done = 0u;
  }
}

// ------------------------------------------------------------------ step kernel

// Step constants in the working precision (read, not converted, per thread).
__device__ __forceinline__ void step_consts(const Ctl* c, const Params& p, double& dt, double& quni, double& g,
                                            double& hg, double& hmin) {
  dt = c->dt; quni = c->quni; g = p.g; hg = 0.5 * p.g; hmin = p.h_min;
}
__device__ __forceinline__ void step_consts(const Ctl* c, const Params& p, float& dt, float& quni, float& g,
                                            float& hg, float& hmin) {
  dt = c->dt_f; quni = c->quni_f; g = p.g_f; hg = p.hg_f; hmin = p.hmin_f;
}

// Shared memory of one CTA (dynamic): the tile's cells, its edges' geometry and
// fluxes, reduction scratch.
template <typename T>
struct TileSmem {
  T Hh[kTile], Hl[kTile], Z[kTile], U[kTile], V[kTile], C[kTile];
  T F[5][kMaxTileEdges];
  T Nx[kMaxTileEdges], Ny[kMaxTileEdges], Ln[kMaxTileEdges];
  int32_t Code[kMaxTileEdges];
  double red[kTile / 32];
  double bc[2];
  unsigned long long rbits;  // max Eq. 21 rate of the tile (bits of a value >= 0)
  int anyb;                  // the tile has boundary edges
};

// One (instance, tile) work item.  T = double: every array and operation in FP64;
// velocity and celerity of U^{n+1} are stored (kDerived) so the next step reads them
// instead of dividing again.  T = float (FP32-bulk): H is an FP32 pair, z an FP32
// offset from an FP64 datum; velocity and celerity are recomputed; the boundary
// volume is summed in FP64.  prime = 1: no update, only derived data, inflow
// weights and the dt of the current state (after init/upload).
template <typename T, bool kDerived>
__device__ __forceinline__ void tile_step(const InstDesc<T>& a, const int tile, const int prime, TileSmem<T>& sm) {
  constexpr bool kPair = sizeof(T) == 4;
  const int tid = threadIdx.x;
  const T zero = T(0);
  Ctl* ctl = a.ctl;
  // round 1: control block and the tile's edge range
  const int par = ctl->parity;
  T dt, quni, g, hg, hmin;
  step_consts(ctl, a.p, dt, quni, g, hg, hmin);
  const double qscale = ctl->qscale;
  const int wpos = ctl->wpos;
  const int64_t e0 = a.eoff[tile];
  const int ne = static_cast<int>(a.eoff[tile + 1] - e0);
  const T* __restrict__ HH = a.H[par];
  const T* __restrict__ HL = kPair ? a.Hlo[par] : nullptr;
  const T* __restrict__ QX0 = a.qx[par];
  const T* __restrict__ QY0 = a.qy[par];
  const T* __restrict__ Z = a.z;
  const int base = tile * kTile;
  const int i = base + tid;
  const bool valid = i < a.n_cells;

  // round 2: every load of the tile that depends only on the tile (cells, edges)
  T Hh = zero, Hl = zero, zi = zero, qxi = zero, qyi = zero, ui = zero, vi = zero, ci = zero, ia = zero, gn2 = zero;
  uint64_t sl = 0;
  if (valid) {
    Hh = HH[i]; zi = Z[i]; qxi = QX0[i]; qyi = QY0[i];
    if (kPair) Hl = HL[i];
    sl = a.slots[i];
    ia = a.inv_area[i];
    gn2 = a.gn2[i];
    if (kDerived && !prime) { ui = a.u[par][i]; vi = a.v[par][i]; ci = a.c[par][i]; }
  }
  // the first two edges of this thread (most tiles have fewer than 512 edges)
  int gL0 = 0, gR0 = kWall, gL1 = 0, gR1 = kWall;
  T nx0 = zero, ny0 = zero, l0 = zero, nx1 = zero, ny1 = zero, l1 = zero;
  if (!prime && tid < ne) {
    gL0 = a.eL[e0 + tid]; gR0 = a.eR[e0 + tid]; nx0 = a.enx[e0 + tid]; ny0 = a.eny[e0 + tid]; l0 = a.elen[e0 + tid];
  }
  if (!prime && tid + kTile < ne) {
    const int64_t e = e0 + tid + kTile;
    gL1 = a.eL[e]; gR1 = a.eR[e]; nx1 = a.enx[e]; ny1 = a.eny[e]; l1 = a.elen[e];
  }
  const T hi0 = depth_of(Hh, Hl, zi);
  if (!(kDerived && !prime) && valid) cell_derived<T>(hi0, qxi, qyi, hmin, g, ui, vi, ci);
  sm.Hh[tid] = Hh; sm.Hl[tid] = Hl; sm.Z[tid] = zi; sm.U[tid] = ui; sm.V[tid] = vi; sm.C[tid] = ci;
  double bsum = 0.0;
  bool sawb = false;  // this thread evaluated a boundary edge
  __syncthreads();

  // phase 1: edges of the tile (round 3: halo cells of other tiles)
  if (!prime) {
    auto edge = [&](const int k, const int gL, const int gR, const T nx, const T ny, const T l) {
      sm.Nx[k] = nx; sm.Ny[k] = ny; sm.Ln[k] = l; sm.Code[k] = gR;
      // surfaces and beds of both sides (the right side mirrors the left at a boundary)
      const int lL = gL - base;
      const bool inL = static_cast<unsigned>(lL) < static_cast<unsigned>(kTile);
      T HLh, HLl, zL;
      if (inL) {
        HLh = sm.Hh[lL]; HLl = sm.Hl[lL]; zL = sm.Z[lL];
      } else {
        HLh = HH[gL]; HLl = kPair ? HL[gL] : zero; zL = Z[gL];
      }
      const int lR = gR - base;
      const bool inR = gR >= 0 && static_cast<unsigned>(lR) < static_cast<unsigned>(kTile);
      T HRh = HLh, HRl = HLl, zR = zL;
      if (gR >= 0) {
        if (inR) {
          HRh = sm.Hh[lR]; HRl = sm.Hl[lR]; zR = sm.Z[lR];
        } else {
          HRh = HH[gR]; HRl = kPair ? HL[gR] : zero; zR = Z[gR];
        }
      }
      // modified states (hydrostatic reconstruction on the higher bed)
      const T zs = fmax(zL, zR);
      const T h1 = fmax(zero, depth_of(HLh, HLl, zs));
      const T h2 = fmax(zero, depth_of(HRh, HRl, zs));
      T F0 = zero, F2 = zero, GL = zero, GR = zero;
      // with both modified depths zero every contribution is exactly zero: skip the
      // flux (warps whose edges are all dry do no flux arithmetic); inflow edges
      // always impose their discharge
      if (h1 > zero || h2 > zero || gR <= kInflow) {
        T uL, vL, cL;
        if (inL) {
          uL = sm.U[lL]; vL = sm.V[lL]; cL = sm.C[lL];
        } else if (kDerived) {
          uL = a.u[par][gL]; vL = a.v[par][gL]; cL = a.c[par][gL];
        } else {
          cell_derived<T>(depth_of(HLh, HLl, zL), QX0[gL], QY0[gL], hmin, g, uL, vL, cL);
        }
        const T unL = uL * nx + vL * ny, utL = -uL * ny + vL * nx;
        T un2, ut2, c1, c2;
        if (gR >= 0) {
          T uR, vR, cR;
          if (inR) {
            uR = sm.U[lR]; vR = sm.V[lR]; cR = sm.C[lR];
          } else if (kDerived) {
            uR = a.u[par][gR]; vR = a.v[par][gR]; cR = a.c[par][gR];
          } else {
            cell_derived<T>(depth_of(HRh, HRl, zR), QX0[gR], QY0[gR], hmin, g, uR, vR, cR);
          }
          // the side with the higher bed keeps its own depth, hence its own celerity
          const bool lhi = zL >= zR;
          const T clo = f_sqrt(g * (lhi ? h2 : h1));
          c1 = lhi ? cL : clo;
          c2 = lhi ? clo : cR;
          un2 = uR * nx + vR * ny;
          ut2 = -uR * ny + vR * nx;
        } else {
          c1 = cL;
          c2 = cL;
          un2 = (gR == kWall) ? -unL : unL;  // wall: mirrored normal velocity
          ut2 = utL;
        }
        T F1, pL, pR;
        hllc<T>(h1, unL, utL, c1, h2, un2, ut2, c2, hg, F0, F1, F2, pL, pR);
        GL = F1 - pL;
        GR = F1 - pR;
        if (gR < 0) {
          if (gR == kWall) {
            F0 = zero; F2 = zero;  // impermeable, frictionless
          } else if (gR <= kInflow) {
            const int j = kInflow - gR;
            const T q = wpos ? static_cast<T>(qscale * static_cast<double>(a.in_pw[j])) : quni;
            if (q > zero) {
              const T hcr = f_cbrt(f_div(q * q, g));
              const T hb = fmax(h1, hcr);
              F0 = -q;
              GL = f_div(q * q, hb) + hg * hb * hb - pL;
            } else {
              F0 = zero;
              GL = zero;
            }
            F2 = zero;
          }
        }
      }
      if (gR < 0) {
        bsum += static_cast<double>(l * F0);
        sawb = true;
      }
      sm.F[0][k] = l * F0;
      sm.F[1][k] = l * (GL * nx - F2 * ny);
      sm.F[2][k] = l * (GL * ny + F2 * nx);
      sm.F[3][k] = l * (GR * nx - F2 * ny);
      sm.F[4][k] = l * (GR * ny + F2 * nx);
    };
    if (tid < ne) edge(tid, gL0, gR0, nx0, ny0, l0);
    if (tid + kTile < ne) edge(tid + kTile, gL1, gR1, nx1, ny1, l1);
    for (int k = tid + 2 * kTile; k < ne; k += kTile) {
      const int64_t e = e0 + k;
      edge(k, a.eL[e], a.eR[e], a.enx[e], a.eny[e], a.elen[e]);
    }
  } else {
    // prime: only the geometry and boundary codes are needed by phase 2
    for (int k = tid; k < ne; k += kTile) {
      sm.Nx[k] = a.enx[e0 + k]; sm.Ny[k] = a.eny[e0 + k]; sm.Ln[k] = a.elen[e0 + k]; sm.Code[k] = a.eR[e0 + k];
    }
  }
  __syncthreads();

  // phase 2: cells
  T rloc = zero;
  if (valid) {
    int idx[3], side[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      const unsigned p = static_cast<unsigned>((sl >> (16 * k)) & 0xffffu);
      idx[k] = static_cast<int>(p >> 1);
      side[k] = static_cast<int>(p & 1u);
    }
    T h = hi0, ux = qxi, uy = qyi;
    if (!prime) {
      T s0 = zero, s1 = zero, s2 = zero;
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        if (side[k] == 0) {
          s0 += sm.F[0][idx[k]]; s1 += sm.F[1][idx[k]]; s2 += sm.F[2][idx[k]];
        } else {
          s0 += -sm.F[0][idx[k]]; s1 += -sm.F[3][idx[k]]; s2 += -sm.F[4][idx[k]];
        }
      }
      const T r = dt * ia;
      if constexpr (kPair) {
        pair_add(Hh, Hl, -(r * s0));
      } else {
        Hh = Hh - r * s0;
      }
      ux = qxi - r * s1;
      uy = qyi - r * s2;
      h = depth_of(Hh, Hl, zi);
      if (h > hmin && gn2 > zero) {
        // split friction: two semi-implicit stages, Heun average
        const T cf = f_div(gn2, h * h * f_cbrt(h));
        const T k0 = cf * f_sqrt(ux * ux + uy * uy);
        const T d0 = f_div(T(1), T(1) + dt * k0);
        const T q1x = ux * d0, q1y = uy * d0;
        const T k1 = cf * f_sqrt(q1x * q1x + q1y * q1y);
        const T d1 = f_div(T(1), T(1) + dt * k1);
        ux = T(0.5) * (ux + q1x * d1);
        uy = T(0.5) * (uy + q1y * d1);
      }
      if (!(h > hmin)) { ux = zero; uy = zero; }
      const int dst = par ^ 1;
      a.H[dst][i] = Hh;
      if constexpr (kPair) a.Hlo[dst][i] = Hl;
      a.qx[dst][i] = ux;
      a.qy[dst][i] = uy;
      if (!isfinite(Hh) || !isfinite(ux) || !isfinite(uy)) atomicOr(&ctl->status, 1);
      // negative depth: below -h_min, beyond the rounding of the FP32 bed offset in FP32-bulk
      const T negtol = kPair ? hmin + T(4) * static_cast<T>(FLT_EPSILON) * fabs(zi) : hmin;
      if (h < -negtol) atomicOr(&ctl->status, 2);
    }
    const int out = prime ? par : (par ^ 1);
    T u, v, c;
    cell_derived<T>(h, ux, uy, hmin, g, u, v, c);
    if (kDerived) {
      a.u[out][i] = u;
      a.v[out][i] = v;
      a.c[out][i] = c;
    }
    if (h > hmin) rloc = cell_rate<T>(sm.Nx, sm.Ny, sm.Ln, idx, u, v, c, ia, a.p.cfl_mode);
    // inflow cells: conveyance weight and depth of the new state, for the finalize
    // and the next step's inflow flux
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      const int code = sm.Code[idx[k]];
      if (code <= kInflow) {
        const int j = kInflow - code;
        a.in_pw[j] = h > hmin ? pow53(h) : zero;
        a.in_hs[j] = fmax(zero, h);
      }
    }
  }
  // end of the tile: rate max (warp shuffle, then one shared atomic per warp) and
  // whether any thread saw a boundary edge
  T rw = rloc;
  for (int o = 16; o > 0; o >>= 1) rw = fmax(rw, __shfl_xor_sync(0xffffffffu, rw, o));
  const bool wb = __any_sync(0xffffffffu, sawb);
  if ((tid & 31) == 0) {
    if (rw > zero) atomicMax(&sm.rbits, static_cast<unsigned long long>(__double_as_longlong(static_cast<double>(rw))));
    if (wb) sm.anyb = 1;
  }
  __syncthreads();
  const int hasb = sm.anyb;
  const unsigned long long rbits = sm.rbits;
  // boundary volume partial (FP64, fixed order) only where the tile has boundary edges
  double bs = 0.0;
  if (hasb) bs = block_sum<kTile>(bsum, sm.red);
  int is_last = 0;
  if (tid == 0) {
    if (hasb) a.part[tile].bflux = bs;
    if (rbits) atomicMax(&ctl->rmax_bits, rbits);
    __threadfence();
    const unsigned prev = atomicAdd(&ctl->done, 1u);
    is_last = (prev == static_cast<unsigned>(a.n_tiles) - 1u) ? 1 : 0;
  }
  if (__syncthreads_or(is_last)) {
    __threadfence();
    finalize_instance<T>(a, prime ? 0 : 1, sm.red, sm.bc);
  }
  if (tid == 0) {  // every thread read them before the barrier above
    sm.rbits = 0ull;
    sm.anyb = 0;
  }
}

template <typename T>
constexpr int kMinBlocks = sizeof(T) == 8 ? 2 : 3;

// The step launch: a work list of (instance, tile) items over instance descriptors
// in device memory.  A single state is a list of one instance's tiles, so a run
// executes the same machine code alone and in a batch and gives bitwise the same
// result (separately compiled copies could contract multiply-adds differently).
template <typename T, bool kDerived>
__global__ void __launch_bounds__(kTile, kMinBlocks<T>) step_batch(const InstDesc<T>* __restrict__ descs,
                                                                    const WorkItem* __restrict__ work, int n_work,
                                                                    int prime) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  TileSmem<T>& sm = *reinterpret_cast<TileSmem<T>*>(smem_raw);
  __shared__ __align__(16) InstDesc<T> sdesc;
  static_assert(sizeof(InstDesc<T>) % 8 == 0, "descriptor copy works in 8-byte words");
  const int tid = threadIdx.x;
  if (tid == 0) {
    sm.rbits = 0ull;
    sm.anyb = 0;
  }
  int staged = -1;  // instance whose descriptor is in shared memory
  for (int w = blockIdx.x; w < n_work; w += gridDim.x) {
    const WorkItem wi = work[w];
    if (wi.inst != staged) {  // consecutive items usually belong to one instance
      __syncthreads();        // nobody still reads the previous descriptor
      const unsigned long long* src = reinterpret_cast<const unsigned long long*>(descs + wi.inst);
      unsigned long long* dstw = reinterpret_cast<unsigned long long*>(&sdesc);
      for (int k = tid; k < static_cast<int>(sizeof(InstDesc<T>) / 8); k += kTile) dstw[k] = src[k];
      staged = wi.inst;
      __syncthreads();
    }
    if (sdesc.ctl->active || prime) tile_step<T, kDerived>(sdesc, wi.tile, prime, sm);
  }
}

// Re-target the end time of one instance: dt is recomputed from the unclipped step.
__global__ void set_t_end(Ctl* ctl, double t_end) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  ctl->t_end = t_end;
  const double t = ctl->t;
  double dt = ctl->dt_cfl;
  int clipped = 0;
  if (dt >= t_end - t) {
    dt = t_end - t;
    clipped = 1;
  }
  ctl->dt = dt;
  ctl->dt_f = static_cast<float>(dt);
  ctl->clipped = clipped;
  ctl->active = t < t_end ? 1 : 0;
}

// V = sum |Omega_i| (H_i - z_i): per-tile partials, then one block in fixed order.
// FP32-bulk: H = hi + lo, and |Omega_i| = 1 / inv_area_i (the area the FP32 update
// uses), so V is the quantity that scheme conserves.
constexpr int kSumThreads = 1024;

template <typename R>
__global__ void __launch_bounds__(kTile) volume_partials(const R* Hh, const R* Hl, const R* z, const double* area,
                                                        const R* inv_area, int n, double* part) {
  __shared__ double sred[kTile / 32];
  const int i = blockIdx.x * kTile + threadIdx.x;
  double x = 0.0;
  if (i < n) {
    const double H = static_cast<double>(Hh[i]) + (Hl ? static_cast<double>(Hl[i]) : 0.0);
    const double A = area ? area[i] : 1.0 / static_cast<double>(inv_area[i]);
    x = A * (H - static_cast<double>(z[i]));
  }
  x = block_sum<kTile>(x, sred);
  if (threadIdx.x == 0) part[blockIdx.x] = x;
}

__global__ void __launch_bounds__(kSumThreads) sum_partials(const double* part, int n, double* out) {
  __shared__ double sred[kSumThreads / 32];
  double x = 0.0;
  for (int t = threadIdx.x; t < n; t += kSumThreads) x += part[t];
  x = block_sum<kSumThreads>(x, sred);
  if (threadIdx.x == 0) *out = x;
}

// Caller order <-> internal order.
template <typename R>
__global__ void gather_from_user(const double* user, const int32_t* perm, int n, R* out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = static_cast<R>(user[perm[i]]);
}

// FP32-bulk free surface: H - datum as an FP32 pair hi + lo; a dry cell (H <= z)
// gets exactly its FP32 bed offset so it stays exactly dry.  Also validates the
// FP64 input (bit 0: non-finite, bit 1: H < z).
__global__ void gather_surface_pair(const double* user, const int32_t* perm, int n, const double* zd, const float* zf,
                                    double datum, float* hi, float* lo, int* bad) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double H = user[perm[i]];
  if (!isfinite(H)) atomicOr(bad, 1);
  if (H < zd[i]) atomicOr(bad, 2);
  if (H <= zd[i]) {
    hi[i] = zf[i];
    lo[i] = 0.0f;
  } else {
    const double v = H - datum;
    const float h = static_cast<float>(v);
    hi[i] = h;
    lo[i] = static_cast<float>(v - static_cast<double>(h));
  }
}

template <typename R>
__global__ void scatter_to_user(const R* in, const R* lo, const int32_t* perm, int n, double* user, double shift) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) user[perm[i]] = shift + (static_cast<double>(in[i]) + (lo ? static_cast<double>(lo[i]) : 0.0));
}

// Validation of an uploaded state: flags non-finite entries and (FP64) H < z.
template <typename R>
__global__ void check_state(const R* H, const R* qx, const R* qy, const R* z, int n, int* bad) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) {
    const bool fin = isfinite(static_cast<double>(qx[i])) && isfinite(static_cast<double>(qy[i])) &&
                     (H == nullptr || isfinite(static_cast<double>(H[i])));
    if (!fin) atomicOr(bad, 1);
    if (H && fin && H[i] < z[i]) atomicOr(bad, 2);
  }
}

}  // namespace bm
