// bm_kernels.cuh -- device code of the explicit shallow-water step (sm_103a).
//
// One step (BASEMENT v3, Section "Numerical solution", "Hydrodynamics"):
//   phase 0  stage the tile's cells (H, z, u, v, c) in shared memory;
//   phase 1  each tile edge once: modified states on max(z_L, z_R), HLLC flux in
//            the edge frame (Toro wave speeds), pre-balanced pressure correction,
//            wall / transmissive / discharge-inflow boundary states;
//   phase 2  each cell gathers its three edge contributions in local edge order
//            (Eq. 12), applies the split Manning friction (Eq. 2, Table 1, two
//            semi-implicit stages), zeroes q below h_min, writes U^{n+1} and its
//            velocity / celerity, and reduces lambda/rho for the next dt (Eq. 21);
//   finalize one block reduces the tile partials in a fixed order: dt^{n+1},
//            t^{n+1}, boundary volume, inflow distribution for t^{n+1}.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

#include "bm_internal.h"

namespace bm {

template <typename R>
struct StepArgs {
  R* H[2];
  R* qx[2];
  R* qy[2];
  R* u[2];   // velocity of the cell (0 below h_min)
  R* v[2];
  R* c[2];   // sqrt(g max(0, h))
  const R* z;
  const R* gn2;       // g n^2
  const R* inv_area;  // 1 / |Omega_i|
  const uint64_t* slots;
  const int64_t* eoff;
  const int32_t* eL;
  const int32_t* eR;
  const R* enx;
  const R* eny;
  const R* elen;
  int n_cells;
  Ctl* ctl;
  TilePartial* part;
  Params p;
};

template <typename R>
struct FinalizeArgs {
  R* H[2];
  const R* z;
  const R* inv_area;
  const int32_t* in_cell;
  const R* in_len;
  int n_inflow;
  double inflow_len;
  int n_tiles;
  Ctl* ctl;
  const TilePartial* part;
  Params p;
};

// ------------------------------------------------------------------ helpers

// Deterministic block reductions (fixed shuffle tree, then warp 0 over warps).
template <int NT>
__device__ __forceinline__ double block_max(double x, double* sbuf) {
  for (int o = 16; o > 0; o >>= 1) x = fmax(x, __shfl_xor_sync(0xffffffffu, x, o));
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  __syncthreads();
  if (lane == 0) sbuf[w] = x;
  __syncthreads();
  if (w == 0) {
    x = lane < NT / 32 ? sbuf[lane] : 0.0;
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

// h^(5/3) for h > 0, through the cube root.
__device__ __forceinline__ double pow53(double h) {
  double r = cbrt(h);
  return h * r * r;
}

// HLLC flux in the edge frame for the modified depths hL, hR (>= 0) with their
// celerities cL = sqrt(g hL), cR = sqrt(g hR); un/ut are normal/tangential
// velocities.  Wave speeds: two-rarefaction star estimates when both sides are
// wet, exact dry-front speeds when one side is dry.  pL, pR = g/2 h^2 are
// returned so the caller subtracts exactly the same values.
__device__ __forceinline__ void hllc(double hL, double unL, double utL, double cL, double hR, double unR,
                                     double utR, double cR, double hg, double& F0, double& F1, double& F2,
                                     double& pL, double& pR) {
  const double us = 0.5 * (unL + unR) + cL - cR;
  const double cs = 0.5 * (cL + cR) + 0.25 * (unL - unR);
  double SL = fmin(unL - cL, us - cs);
  double SR = fmax(unR + cR, us + cs);
  const bool ldry = !(hL > 0.0), rdry = !(hR > 0.0);
  SL = ldry ? unR - 2.0 * cR : (rdry ? unL - cL : SL);
  SR = ldry ? unR + cR : (rdry ? unL + 2.0 * cL : SR);
  pL = hg * hL * hL;
  pR = hg * hR * hR;
  const double FL0 = hL * unL, FL1 = FL0 * unL + pL, FL2 = FL0 * utL;
  const double FR0 = hR * unR, FR1 = FR0 * unR + pR, FR2 = FR0 * utR;
  const double rd = 1.0 / (SR - SL);
  const double H0 = FL0 - SL * ((FR0 - FL0) - SR * (hR - hL)) * rd;
  const double H1 = FL1 - SL * ((FR1 - FL1) - SR * (FR0 - FL0)) * rd;
  // sign of the contact speed S* = num / den with den < 0 whenever a side is wet
  const double num = SL * hR * (unR - SR) - SR * hL * (unL - SL);
  const double H2 = H0 * (num <= 0.0 ? utL : utR);
  if (SL >= 0.0) {
    F0 = FL0; F1 = FL1; F2 = FL2;
  } else if (SR <= 0.0) {
    F0 = FR0; F1 = FR1; F2 = FR2;
  } else {
    F0 = H0; F1 = H1; F2 = H2;
  }
  if (ldry && rdry) {
    F0 = 0.0; F1 = 0.0; F2 = 0.0;
  }
}

// ------------------------------------------------------------------ step kernel (FP64)

__global__ void __launch_bounds__(kTile) step_fp64(const StepArgs<double> a) {
  Ctl* ctl = a.ctl;
  if (!ctl->active) return;
  const int par = ctl->parity;
  const double dt = ctl->dt;
  const double qscale = ctl->qscale, quni = ctl->quni;
  const int wpos = ctl->wpos;
  const double g = a.p.g, hg = 0.5 * a.p.g, hmin = a.p.h_min;

  const double* __restrict__ H0 = a.H[par];
  const double* __restrict__ QX0 = a.qx[par];
  const double* __restrict__ QY0 = a.qy[par];
  const double* __restrict__ U0 = a.u[par];
  const double* __restrict__ V0 = a.v[par];
  const double* __restrict__ C0 = a.c[par];
  const double* __restrict__ Z = a.z;

  __shared__ double sH[kTile], sZ[kTile], sU[kTile], sV[kTile], sC[kTile];
  __shared__ double sF[5][kMaxTileEdges];
  __shared__ double sred[kTile / 32];

  const int tile = blockIdx.x, tid = threadIdx.x;
  const int base = tile * kTile;
  const int i = base + tid;
  const bool valid = i < a.n_cells;
  double Hi = 0, zi = 0, qxi = 0, qyi = 0;
  if (valid) {
    Hi = H0[i]; zi = Z[i]; qxi = QX0[i]; qyi = QY0[i];
    sU[tid] = U0[i]; sV[tid] = V0[i]; sC[tid] = C0[i];
  } else {
    sU[tid] = 0; sV[tid] = 0; sC[tid] = 0;
  }
  sH[tid] = Hi;
  sZ[tid] = zi;
  __syncthreads();

  // phase 1: edges of the tile
  const int64_t e0 = a.eoff[tile];
  const int ne = static_cast<int>(a.eoff[tile + 1] - e0);
  double bsum = 0.0;
  for (int k = tid; k < ne; k += kTile) {
    const int64_t e = e0 + k;
    const int gL = a.eL[e], gR = a.eR[e];
    const double nx = a.enx[e], ny = a.eny[e], l = a.elen[e];
    double HL, zL, uL, vL, cL;
    const int lL = gL - base;
    if (static_cast<unsigned>(lL) < static_cast<unsigned>(kTile)) {
      HL = sH[lL]; zL = sZ[lL]; uL = sU[lL]; vL = sV[lL]; cL = sC[lL];
    } else {
      HL = H0[gL]; zL = Z[gL]; uL = U0[gL]; vL = V0[gL]; cL = C0[gL];
    }
    const double unL = uL * nx + vL * ny, utL = -uL * ny + vL * nx;
    double h1, h2, un2, ut2, c1, c2;
    if (gR >= 0) {
      double HR, zR, uR, vR, cR;
      const int lR = gR - base;
      if (static_cast<unsigned>(lR) < static_cast<unsigned>(kTile)) {
        HR = sH[lR]; zR = sZ[lR]; uR = sU[lR]; vR = sV[lR]; cR = sC[lR];
      } else {
        HR = H0[gR]; zR = Z[gR]; uR = U0[gR]; vR = V0[gR]; cR = C0[gR];
      }
      const double zs = fmax(zL, zR);
      h1 = fmax(0.0, HL - zs);
      h2 = fmax(0.0, HR - zs);
      // the side with the higher bed keeps its own depth, hence its own celerity
      const bool lhi = zL >= zR;
      const double clo = sqrt(g * (lhi ? h2 : h1));
      c1 = lhi ? cL : clo;
      c2 = lhi ? clo : cR;
      un2 = uR * nx + vR * ny;
      ut2 = -uR * ny + vR * nx;
    } else {
      h1 = fmax(0.0, HL - zL);
      h2 = h1;
      c1 = cL;
      c2 = cL;
      un2 = (gR == kWall) ? -unL : unL;  // wall: mirrored normal velocity
      ut2 = utL;
    }
    double F0, F1, F2, pL, pR;
    hllc(h1, unL, utL, c1, h2, un2, ut2, c2, hg, F0, F1, F2, pL, pR);
    double GL = F1 - pL, GR = F1 - pR;
    if (gR < 0) {
      if (gR == kWall) {
        F0 = 0.0; F2 = 0.0;  // impermeable, frictionless
      } else if (gR == kInflow) {
        const double h = HL - zL;
        const double q = wpos ? (h > hmin ? qscale * pow53(h) : 0.0) : quni;
        if (q > 0.0) {
          const double hcr = cbrt(q * q / g);
          const double hb = fmax(h1, hcr);
          F0 = -q;
          GL = q * q / hb + hg * hb * hb - pL;
        } else {
          F0 = 0.0;
          GL = 0.0;
        }
        F2 = 0.0;
      }
      bsum += l * F0;
    }
    sF[0][k] = l * F0;
    sF[1][k] = l * (GL * nx - F2 * ny);
    sF[2][k] = l * (GL * ny + F2 * nx);
    sF[3][k] = l * (GR * nx - F2 * ny);
    sF[4][k] = l * (GR * ny + F2 * nx);
  }
  __syncthreads();

  // phase 2: cells
  double rloc = 0.0;
  if (valid) {
    const uint64_t sl = a.slots[i];
    double s0 = 0.0, s1 = 0.0, s2 = 0.0;
    int idx[3], side[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      const unsigned p = static_cast<unsigned>((sl >> (16 * k)) & 0xffffu);
      idx[k] = static_cast<int>(p >> 1);
      side[k] = static_cast<int>(p & 1u);
      if (side[k] == 0) {
        s0 += sF[0][idx[k]]; s1 += sF[1][idx[k]]; s2 += sF[2][idx[k]];
      } else {
        s0 += -sF[0][idx[k]]; s1 += -sF[3][idx[k]]; s2 += -sF[4][idx[k]];
      }
    }
    const double ia = a.inv_area[i];
    const double r = dt * ia;
    const double Hn = Hi - r * s0;
    double ux = qxi - r * s1;
    double uy = qyi - r * s2;
    const double h = Hn - zi;
    const double gn2 = a.gn2[i];
    if (h > hmin && gn2 > 0.0) {
      // split friction: two semi-implicit stages, Heun average
      const double cf = gn2 / (h * h * cbrt(h));
      const double k0 = cf * sqrt(ux * ux + uy * uy);
      const double d0 = 1.0 / (1.0 + dt * k0);
      const double q1x = ux * d0, q1y = uy * d0;
      const double k1 = cf * sqrt(q1x * q1x + q1y * q1y);
      const double d1 = 1.0 / (1.0 + dt * k1);
      ux = 0.5 * (ux + q1x * d1);
      uy = 0.5 * (uy + q1y * d1);
    }
    const bool wet = h > hmin;
    if (!wet) { ux = 0.0; uy = 0.0; }
    const int dst = par ^ 1;
    a.H[dst][i] = Hn;
    a.qx[dst][i] = ux;
    a.qy[dst][i] = uy;
    double u = 0.0, v = 0.0;
    if (wet) {
      const double rh = 1.0 / h;
      u = ux * rh;
      v = uy * rh;
    }
    const double c = sqrt(g * fmax(0.0, h));
    a.u[dst][i] = u;
    a.v[dst][i] = v;
    a.c[dst][i] = c;
    if (!isfinite(Hn) || !isfinite(ux) || !isfinite(uy)) atomicOr(&ctl->status, 1);
    if (h < -hmin) atomicOr(&ctl->status, 2);
    // next dt (Eq. 21): lambda_ij / rho_ij = 3/4 lambda l / |Omega| (or sum l lambda / |Omega|)
    if (wet) {
      double ssum = 0.0;
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        const int64_t e = e0 + idx[k];
        const double lam = fabs(u * a.enx[e] + v * a.eny[e]) + c;  // |u.n| is side-independent
        const double ll = lam * a.elen[e];
        rloc = fmax(rloc, 0.75 * ll * ia);
        ssum += ll;
      }
      if (a.p.cfl_mode == 1) rloc = ssum * ia;
    }
  }
  const double rm = block_max<kTile>(rloc, sred);
  const double bs = block_sum<kTile>(bsum, sred);
  if (tid == 0) {
    a.part[tile].rmax = rm;
    a.part[tile].bflux = bs;
  }
}

// Derived cell data (u, v, c) and the dt partials of the current state; used after
// init/upload before the first step.
__global__ void __launch_bounds__(kTile) prime_fp64(const StepArgs<double> a) {
  __shared__ double sred[kTile / 32];
  const int par = a.ctl->parity;
  const int tile = blockIdx.x, tid = threadIdx.x;
  const int i = tile * kTile + tid;
  const double g = a.p.g, hmin = a.p.h_min;
  double rloc = 0.0;
  if (i < a.n_cells) {
    const double h = a.H[par][i] - a.z[i];
    const bool wet = h > hmin;
    double u = 0.0, v = 0.0;
    if (wet) {
      const double rh = 1.0 / h;
      u = a.qx[par][i] * rh;
      v = a.qy[par][i] * rh;
    }
    const double c = sqrt(g * fmax(0.0, h));
    a.u[par][i] = u;
    a.v[par][i] = v;
    a.c[par][i] = c;
    if (wet) {
      const uint64_t sl = a.slots[i];
      const double ia = a.inv_area[i];
      const int64_t e0 = a.eoff[tile];
      double ssum = 0.0;
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        const unsigned p = static_cast<unsigned>((sl >> (16 * k)) & 0xffffu);
        const int64_t e = e0 + (p >> 1);
        const double lam = fabs(u * a.enx[e] + v * a.eny[e]) + c;
        const double ll = lam * a.elen[e];
        rloc = fmax(rloc, 0.75 * ll * ia);
        ssum += ll;
      }
      if (a.p.cfl_mode == 1) rloc = ssum * ia;
    }
  }
  const double rm = block_max<kTile>(rloc, sred);
  if (tid == 0) {
    a.part[tile].rmax = rm;
    a.part[tile].bflux = 0.0;
  }
}

// ------------------------------------------------------------------ finalize

constexpr int kFinThreads = 1024;

// advance = 1 after a step (t += dt, boundary volume, parity flip); 0 after prime.
template <typename R>
__global__ void __launch_bounds__(kFinThreads) finalize(const FinalizeArgs<R> a, int advance) {
  __shared__ double sred[kFinThreads / 32];
  __shared__ double s_t, s_rm;
  __shared__ int s_par;
  Ctl* ctl = a.ctl;
  if (!ctl->active && advance) return;
  const int tid = threadIdx.x;
  double rm = 0.0, bs = 0.0;
  for (int t = tid; t < a.n_tiles; t += kFinThreads) {
    rm = fmax(rm, a.part[t].rmax);
    bs += a.part[t].bflux;
  }
  rm = block_max<kFinThreads>(rm, sred);
  bs = block_sum<kFinThreads>(bs, sred);
  if (tid == 0) {
    if (advance) {
      const double dt = ctl->dt;
      ctl->bvol += -dt * bs;
      ctl->t = ctl->clipped ? ctl->t_end : ctl->t + dt;
      ctl->parity ^= 1;
      ctl->steps += 1;
    }
    s_t = ctl->t;
    s_par = ctl->parity;
    s_rm = rm;
  }
  __syncthreads();
  const double t = s_t;
  const int par = s_par;
  const double g = a.p.g, hmin = a.p.h_min;
  // inflow distribution at the new time (conveyance weights l h^(5/3))
  double wsum = 0.0;
  for (int j = tid; j < a.n_inflow; j += kFinThreads) {
    const int cell = a.in_cell[j];
    const double h = static_cast<double>(a.H[par][cell]) - static_cast<double>(a.z[cell]);
    wsum += h > hmin ? static_cast<double>(a.in_len[j]) * pow53(h) : 0.0;
  }
  wsum = block_sum<kFinThreads>(wsum, sred);
  __shared__ double s_w;
  if (tid == 0) s_w = wsum;
  __syncthreads();
  wsum = s_w;
  const double Q = hydrograph(a.p, t);
  const bool wpos = wsum > 0.0;
  const double qscale = wpos ? Q / wsum : 0.0;
  const double quni = (!wpos && a.inflow_len > 0.0) ? Q / a.inflow_len : 0.0;
  double rb = 0.0;
  for (int j = tid; j < a.n_inflow; j += kFinThreads) {
    const int cell = a.in_cell[j];
    const double h = static_cast<double>(a.H[par][cell]) - static_cast<double>(a.z[cell]);
    const double q = wpos ? (h > hmin ? qscale * pow53(h) : 0.0) : quni;
    if (q > 0.0) {
      const double hs = fmax(0.0, h);
      const double hb = fmax(hs, cbrt(q * q / g));
      const double lb = q / hb + sqrt(g * hb);
      const double ll = lb * static_cast<double>(a.in_len[j]) * static_cast<double>(a.inv_area[cell]);
      rb = fmax(rb, a.p.cfl_mode == 0 ? 0.75 * ll : ll);
    }
  }
  rb = block_max<kFinThreads>(rb, sred);
  if (tid == 0) {
    const double r = fmax(s_rm, rb);
    double dtc = r > 0.0 ? a.p.cfl / r : a.p.dt_max;
    if (dtc > a.p.dt_max) dtc = a.p.dt_max;
    ctl->pad0 = dtc;  // unclipped dt, used when t_end changes
    double dt = dtc;
    int clipped = 0;
    if (dt >= ctl->t_end - t) {
      dt = ctl->t_end - t;
      clipped = 1;
    }
    ctl->dt = dt;
    ctl->clipped = clipped;
    ctl->active = t < ctl->t_end ? 1 : 0;
    ctl->Q = Q;
    ctl->qscale = qscale;
    ctl->quni = quni;
    ctl->wpos = wpos ? 1 : 0;
  }
}

// Re-target the end time: dt is recomputed from the unclipped CFL step.
__global__ void set_t_end(Ctl* ctl, double t_end) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  ctl->t_end = t_end;
  const double t = ctl->t;
  double dt = ctl->pad0;
  int clipped = 0;
  if (dt >= t_end - t) {
    dt = t_end - t;
    clipped = 1;
  }
  ctl->dt = dt;
  ctl->clipped = clipped;
  ctl->active = t < t_end ? 1 : 0;
}

// V = sum |Omega_i| (H_i - z_i): per-tile partials, then one block in fixed order.
template <typename R>
__global__ void __launch_bounds__(kTile) volume_partials(const R* H, const R* z, const double* area, int n,
                                                        double datum_shift, double* part) {
  __shared__ double sred[kTile / 32];
  const int i = blockIdx.x * kTile + threadIdx.x;
  double x = 0.0;
  if (i < n) x = area[i] * ((static_cast<double>(H[i]) - static_cast<double>(z[i])) + datum_shift);
  x = block_sum<kTile>(x, sred);
  if (threadIdx.x == 0) part[blockIdx.x] = x;
}

__global__ void __launch_bounds__(kFinThreads) sum_partials(const double* part, int n, double* out) {
  __shared__ double sred[kFinThreads / 32];
  double x = 0.0;
  for (int t = threadIdx.x; t < n; t += kFinThreads) x += part[t];
  x = block_sum<kFinThreads>(x, sred);
  if (threadIdx.x == 0) *out = x;
}

// Caller order <-> internal order.
template <typename R>
__global__ void gather_from_user(const double* user, const int32_t* perm, int n, R* out, double shift) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = static_cast<R>(user[perm[i]] - shift);
}

template <typename R>
__global__ void scatter_to_user(const R* in, const int32_t* perm, int n, double* user, double shift) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) user[perm[i]] = static_cast<double>(in[i]) + shift;
}

// Validation of an uploaded state: counts H < z and non-finite entries.
template <typename R>
__global__ void check_state(const R* H, const R* qx, const R* qy, const R* z, int n, int* bad) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) {
    const bool fin = isfinite(static_cast<double>(H[i])) && isfinite(static_cast<double>(qx[i])) &&
                     isfinite(static_cast<double>(qy[i]));
    if (!fin) atomicOr(bad, 1);
    if (fin && H[i] < z[i]) atomicOr(bad, 2);
  }
}

}  // namespace bm
