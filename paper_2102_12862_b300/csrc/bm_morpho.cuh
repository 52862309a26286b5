// bm_morpho.cuh -- bed evolution (BASEMENT v3, Section "Morphodynamics": Exner, Eq. 3
// with S_b = 0, updated by Eq. 13 with the HLL sediment flux of Eq. 14-16), solved
// synchronous-decoupled with the water: the same dt, every term from U^n and z^n.
//
// Bedload from Table 2's MPM-like closure,
//   |q_B| = alpha (theta - theta_cr)^m sqrt((s - 1) g d^3)  (0 for theta <= theta_cr),
//   theta = n^2 |u|^2 / ((s - 1) d h^(1/3))   (Manning's bed shear stress over
//                                               (rho_s - rho) g d),
// along the flow.  dq_B,n/dq_n of Eq. 16 is taken along the flow at fixed depth,
// d|q_B|/d|u| / h.  Walls carry no sediment, other boundary edges the inside cell's
// normal bedload.  The free surface moves with the bed (the water depth is kept).
// FP64 states only.
#pragma once

#include "bm_kernels.cuh"
#include "bm_step.cuh"

namespace bm {

struct MorphoParams {
  double porosity, s, d, alpha, m, theta_cr;
  // derived on the host: 1 / g, 1 / ((s - 1) d), sqrt((s - 1) g d^3), 1 / (1 - porosity)
  double inv_g, inv_sdd, scale, inv_solid;
};

struct MorphoArgs {
  const PipeItem* items;  // the state's work list: one item per tile
  const double* H[2];
  double* z;
  const double* qx[2];
  const double* qy[2];
  const double* gn2;      // g n^2 per cell
  const Ctl* ctl;         // after the step: U^{n+1} in buffer ctl->parity
  const double* step_dt;  // dt of the step that just ran (< 0: none)
  double* dz;             // per cell: the bed change of this step
  MorphoParams mp;
  double g, h_min;
  int n_cells;
};

// Before each step: the dt that step takes (-1 once the run ended).
__global__ void morpho_save_dt(const Ctl* ctl, double* step_dt) {
  if (threadIdx.x == 0 && blockIdx.x == 0) *step_dt = ctl->active ? ctl->dt : -1.0;
}

// Bedload vector and dq_B/dq of one cell (velocity desingularised below h_min).
__device__ __forceinline__ void bedload(const MorphoArgs& a, double h, double qx, double qy, double gn2,
                                        double& bx, double& by, double& bd) {
  bx = 0.0;
  by = 0.0;
  bd = 0.0;
  if (!(h > a.h_min)) return;
  // FP64 transcendentals are slow on this part: divisions as a times a refined
  // reciprocal, h^(-1/3) by Newton steps, and for the usual exponent 3/2 the powers
  // as x sqrt(x) and sqrt(x) (the library power for any other exponent)
  const double rh = f_rcp(h);
  const double u = qx * rh, v = qy * rh;
  const double sp = sqrt(u * u + v * v);
  if (sp == 0.0) return;
  const double theta = gn2 * a.mp.inv_g * sp * sp * f_rcbrt(h) * a.mp.inv_sdd;
  if (!(theta > a.mp.theta_cr)) return;
  const double scale = a.mp.scale;
  const double x = theta - a.mp.theta_cr;
  double xm, xm1;  // x^m, x^(m-1)
  if (a.mp.m == 1.5) {
    xm1 = sqrt(x);
    xm = x * xm1;
  } else {
    xm = pow(x, a.mp.m);
    xm1 = pow(x, a.mp.m - 1.0);
  }
  const double qb = a.mp.alpha * xm * scale;
  const double rsp = f_rcp(sp);
  bx = qb * u * rsp;
  by = qb * v * rsp;
  bd = a.mp.alpha * a.mp.m * xm1 * scale * (2.0 * theta * rsp) * rh;
}

// Eq. 16's two speeds for one cell on an edge.
__device__ __forceinline__ void morpho_speeds(double un, double c, double bd, double& l1, double& l2) {
  const double a = un - c;
  const double r = sqrt(a * a + 4.0 * bd * c * c);
  l1 = 0.5 * (a - r);
  l2 = 0.5 * (a + r);
}

// One CTA per work item (a 256-cell tile): the bed change of its cells into dz.
// Dynamic shared memory: 8 nloc_max + ne4_max doubles.
__global__ void __launch_bounds__(kTile) morpho_flux(const MorphoArgs a, int nloc_max) {
  const double dt = *a.step_dt;
  if (!(dt >= 0.0)) return;
  using RL = RecLayout<8>;
  extern __shared__ __align__(16) unsigned char smem_mo[];
  double* sh = reinterpret_cast<double*>(smem_mo);  // h, u, v, c, q_Bx, q_By, dq_B/dq, z
  double* su = sh + nloc_max;
  double* sv = su + nloc_max;
  double* sc = sv + nloc_max;
  double* sbx = sc + nloc_max;
  double* sby = sbx + nloc_max;
  double* sbd = sby + nloc_max;
  double* sz = sbd + nloc_max;
  double* fs = sz + nloc_max;  // per edge: l q_Bij, outward from the left cell
  const PipeItem& it = a.items[blockIdx.x];
  const int tile = it.tile, tid = threadIdx.x;
  const unsigned char* rec = it.rec;
  const int ne = static_cast<int>(it.ne_nh & 0xffffu), nh = static_cast<int>(it.ne_nh >> 16);
  const uint32_t ne4 = round4(static_cast<uint32_t>(ne));
  const int32_t* hidx = reinterpret_cast<const int32_t*>(rec + RL::hidx(ne4));
  const uint32_t* lr = reinterpret_cast<const uint32_t*>(rec + RL::lr());
  const double* enx = reinterpret_cast<const double*>(rec + RL::nx(ne4));
  const double* eny = reinterpret_cast<const double*>(rec + RL::ny(ne4));
  const double* eln = reinterpret_cast<const double*>(rec + RL::len(ne4));
  const int po = a.ctl->parity ^ 1;  // U^n
  bool wet = false;  // a tile or halo cell above h_min (else no edge of the tile moves sediment)
  for (int j = tid; j < kTile + nh; j += kTile) {
    const int g = j < kTile ? tile * kTile + j : hidx[j - kTile];
    double h = 0.0, u = 0.0, v = 0.0, c = 0.0, bx = 0.0, by = 0.0, bd = 0.0, zz = 0.0;
    if (g < a.n_cells) {
      zz = a.z[g];
      h = a.H[po][g] - zz;
      const double qx = a.qx[po][g], qy = a.qy[po][g];
      if (h > a.h_min) {
        const double rh = f_rcp(h);
        u = qx * rh;
        v = qy * rh;
        wet = true;
        bedload(a, h, qx, qy, a.gn2[g], bx, by, bd);
      }
      if (h > 0.0) c = sqrt(a.g * h);
    }
    sh[j] = h; su[j] = u; sv[j] = v; sc[j] = c; sbx[j] = bx; sby[j] = by; sbd[j] = bd; sz[j] = zz;
  }
  const int i = tile * kTile + tid;
  // every cell at or below h_min: u_n - c <= 0 and no bedload on both sides of every
  // edge, so lambda+ = 0 and every flux of Eq. 14 is zero
  if (!__syncthreads_or(wet)) {
    if (i < a.n_cells) a.dz[i] = 0.0;
    return;
  }
  for (int k = tid; k < ne; k += kTile) {
    const uint32_t w = lr[k];
    const int lL = static_cast<int>(w & (kMaxLocal - 1));
    const int R = static_cast<int32_t>(w) >> kLocBits;
    const double nx = enx[k], ny = eny[k];
    const double qL = sbx[lL] * nx + sby[lL] * ny;
    double f;
    if (R >= 0) {
      const double unL = su[lL] * nx + sv[lL] * ny, unR = su[R] * nx + sv[R] * ny;
      const double qR = sbx[R] * nx + sby[R] * ny;
      const double aL = unL - sc[lL], aR = unR - sc[R];
      if (sbd[lL] == 0.0 && sbd[R] == 0.0 && qL == 0.0 && qR == 0.0 && !(fmin(aL, aR) < 0.0 && fmax(aL, aR) > 0.0)) {
        // no transport on either side: Eq. 16 gives min(a, 0) and max(a, 0) exactly,
        // so one of lambda+, lambda- is zero unless a changes sign across the edge
        f = 0.0;
      } else {
        double a1, a2, b1, b2;
        morpho_speeds(unL, sc[lL], sbd[lL], a1, a2);
        morpho_speeds(unR, sc[R], sbd[R], b1, b2);
        const double lm = fmin(a1, b1), lp = fmax(a2, b2);
        f = lp - lm > 0.0 ? (lp * qL - lm * qR + lp * lm * (sz[R] - sz[lL])) * f_rcp(lp - lm) : 0.0;
      }
    } else {
      f = R == kWall ? 0.0 : qL;
    }
    fs[k] = eln[k] * f;
  }
  __syncthreads();
  if (i < a.n_cells) {
    const double ia = reinterpret_cast<const double*>(rec + RL::ia())[tid];
    const uint32_t sl = reinterpret_cast<const uint32_t*>(rec + RL::slot())[tid];
    double sum = 0.0;
#pragma unroll
    for (int q = 0; q < 3; ++q) {
      const int e = static_cast<int>((sl >> (kLocBits * q)) & (kMaxLocal - 1));
      const bool left = (lr[e] & (kMaxLocal - 1)) == static_cast<uint32_t>(tid);
      sum += left ? fs[e] : -fs[e];
    }
    a.dz[i] = -(dt * ia * sum) * a.mp.inv_solid;
  }
}

// The bed change applied: z += dz, and the new free surface with it.
__global__ void morpho_apply(const double* dz, const double* step_dt, const Ctl* ctl, double* z, double* H0,
                             double* H1, int n) {
  if (!(*step_dt >= 0.0)) return;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double* Hn = ctl->parity ? H1 : H0;
  z[i] += dz[i];
  Hn[i] += dz[i];
}

}  // namespace bm
