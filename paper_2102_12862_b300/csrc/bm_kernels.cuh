// bm_kernels.cuh -- device helpers of the explicit shallow-water step (sm_103a): the
// instance descriptor, deterministic block reductions, the HLLC flux, cell-derived
// quantities, the per-instance finalize (dt of Eq. 21, time, boundary volume, inflow
// split), and the small kernels around the step (end-time targeting, volume, user-order
// gather/scatter, state checks).  The step kernel itself is in bm_step.cuh.
#pragma once

#include <cuda_runtime.h>

#include <cfloat>
#include <cstdint>

#include "bm_internal.h"

namespace bm {

// Everything one instance's tiles need besides their tile records; lives in device
// memory and is bulk-copied into shared memory with each tile (size a multiple of 16).
template <typename T>
struct alignas(16) InstDesc {
  T* H[2];    // free surface (FP32-bulk: hi part of the offset from the datum)
  T* Hlo[2];  // FP32-bulk only: lo part of the free surface
  T* qx[2];
  T* qy[2];
  // flood tracking (null when off): front arrival time, maxima of depth, |u|, |q|
  // and bed shear stress per cell; the arrival threshold depth
  double* trk_t;
  T* trk_h;
  T* trk_u;
  T* trk_q;
  T* trk_tau;
  T trk_harr;
  const T* z;
  const T* gn2;       // g n^2
  const T* inv_area;  // 1 / |Omega_i|
  const int32_t* in_cell;  // listed edge j (inflow, h-Q, weir, level): its cell
  const double* in_lia;    //                l_j / |Omega| of its cell
  const T* in_len;         //                its length
  const double* in_nx;     //                its outward unit normal
  const double* in_ny;
  T* in_pw;                //                inflow: h^(5/3) of the cell (0 at or below h_min);
                           //                h-Q: the unit discharge leaving (at t^n)
  T* in_hs;                //                inflow: max(0, h) of the cell
  const int32_t* btiles;   // tiles with boundary edges (tile b's partial at part[b's rank])
  Ctl* ctl;
  TilePartial* part;
  Params p;
  double inflow_len;
  int n_inflow;
  int n_btiles;
  int n_in_tiles;          // tiles with inflow edges
  int n_cells;
  int n_tiles;
  // passive species (null when none): the step exports, per tile edge, l F_h and
  // whether the contact's right side is upwind; per tile whether it had fluxes (0:
  // quiet); the step's dt.  A second kernel advects the species with them.
  T* ex_flux;
  unsigned char* ex_right;
  unsigned char* ex_valid;
  double* ex_dt;
  int ex_stride;  // edges per tile in ex_flux / ex_right (the mesh's largest, rounded to 4)
  // external sources (null when none): region of each cell (-1: none), S_h of each
  // region at t^n (m/s, written before each step), its sink mode (0 Exact, 1
  // Available, 2 Infinity)
  const int32_t* src_reg;
  const T* src_rate;
  const int32_t* src_mode;
  // friction closure of Table 1: 0 Manning (gn2 = g n^2), 1 Chezy (gn2 holds K_s),
  // 2 Bezzola (gn2 holds y_R)
  int fr_law;
  // outflow laws: listed edges [n_inflow, n_inflow + n_hq) are h-Q edges, the next
  // n_weir weir edges.  The h-Q relation's table (absolute stage, discharge; hq_n = 0:
  // nothing leaves); the weir's crest (FP32-bulk: offset from the datum) and
  // (2/3) mu sqrt(2 g) of its Poleni factor mu (0: nothing leaves)
  int n_hq;
  int n_weir;
  int n_hq_tiles;          // tiles with h-Q edges
  int hq_n;
  const double* hq_s;
  const double* hq_q;
  double datum;            // FP32-bulk: the surface and the bed are offsets from it
  T weir_crest;
  T weir_k;
  // water-level edges: listed edges [n_inflow + n_hq + n_weir, + n_level).  The series
  // of the imposed surface Z_b(t) (absolute; zh_n = 0: the edges are walls)
  int n_level;
  int zh_n;
  const double* zh_t;
  const double* zh_v;
};

// ------------------------------------------------------------------ helpers

// Barrier over the first NT threads of the block (named barrier 1): the step kernel's
// compute warps synchronise without its copy warp.
template <int NT>
__device__ __forceinline__ void nbar() {
  asm volatile("bar.sync 1, %0;" ::"n"(NT) : "memory");
}
template <int NT>
__device__ __forceinline__ bool nbar_and(bool v) {
  uint32_t r;
  asm volatile(
      "{\n\t.reg .pred p, q;\n\tsetp.ne.u32 q, %1, 0;\n\t"
      "bar.red.and.pred p, 1, %2, q;\n\tselp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(r)
      : "r"(static_cast<uint32_t>(v)), "n"(NT)
      : "memory");
  return r != 0;
}
template <int NT>
__device__ __forceinline__ bool nbar_or(bool v) {
  uint32_t r;
  asm volatile(
      "{\n\t.reg .pred p, q;\n\tsetp.ne.u32 q, %1, 0;\n\t"
      "bar.red.or.pred p, 1, %2, q;\n\tselp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(r)
      : "r"(static_cast<uint32_t>(v)), "n"(NT)
      : "memory");
  return r != 0;
}

// Deterministic block reductions over the first NT threads (fixed shuffle tree, then
// warp 0 over warps).
template <int NT, typename V>
__device__ __forceinline__ V block_max(V x, V* sbuf) {
  for (int o = 16; o > 0; o >>= 1) x = fmax(x, __shfl_xor_sync(0xffffffffu, x, o));
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  nbar<NT>();
  if (lane == 0) sbuf[w] = x;
  nbar<NT>();
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
  nbar<NT>();
  if (lane == 0) sbuf[w] = x;
  nbar<NT>();
  if (w == 0) {
    x = lane < NT / 32 ? sbuf[lane] : 0.0;
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
  }
  return x;  // valid in thread 0
}

// Maximum of non-negative doubles over the first NT threads, returned to every
// thread.  Non-negative doubles order like their bit patterns, so the reduction runs
// on 64-bit integers (integer pipes, not the FP64 pipe; the result is exact).
template <int NT>
__device__ __forceinline__ double block_max_nonneg_all(double x, unsigned long long* sbuf) {
  unsigned long long v = static_cast<unsigned long long>(__double_as_longlong(x));
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long u = __shfl_xor_sync(0xffffffffu, v, o);
    v = u > v ? u : v;
  }
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  nbar<NT>();
  if (lane == 0) sbuf[w] = v;
  nbar<NT>();
  if (w == 0) {
    v = lane < NT / 32 ? sbuf[lane] : 0ull;
    for (int o = 16; o > 0; o >>= 1) {
      const unsigned long long u = __shfl_xor_sync(0xffffffffu, v, o);
      v = u > v ? u : v;
    }
    if (lane == 0) sbuf[NT / 32] = v;
  }
  nbar<NT>();
  return __longlong_as_double(static_cast<long long>(sbuf[NT / 32]));
}

// Sum over one warp in a fixed order (lane-strided partial sums, then a shuffle tree).
__device__ __forceinline__ double warp_sum(double x) {
  for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
  return x;
}

// Comparisons, minima and maxima of FP64 values on the integer pipes: B300 issues FP64
// instructions at 2 lanes per SM and cycle and integer ones at 64, and the wet-cell
// step is bound by its FP64 pipe, so every FP64 comparison or min / max moved off it
// is time saved.  okey is an order-preserving integer key of a double (for x, y not
// NaN: key(x) <= key(y) exactly when x <= y, except that -0 sorts below +0).  For
// non-NaN arguments the helpers equal the IEEE operations, up to which zero of a
// (-0, +0) pair fmin / fmax return; the float overloads are the FP32 operations.
__device__ __forceinline__ long long okey(double x) {
  const long long b = __double_as_longlong(x);
  return b ^ ((b >> 63) & 0x7fffffffffffffffLL);
}
__device__ __forceinline__ bool gt0(double x) { return __double_as_longlong(x) > 0; }  // x > 0
__device__ __forceinline__ bool gt0(float x) { return x > 0.0f; }
__device__ __forceinline__ bool ge0(double x) { return okey(x) >= -1; }  // x >= 0, -0 included
__device__ __forceinline__ bool ge0(float x) { return x >= 0.0f; }
__device__ __forceinline__ bool le0(double x) { return okey(x) <= 0; }  // x <= 0
__device__ __forceinline__ bool le0(float x) { return x <= 0.0f; }
__device__ __forceinline__ bool gt(double x, double y) { return okey(x) > okey(y); }  // x > y
__device__ __forceinline__ bool gt(float x, float y) { return x > y; }
__device__ __forceinline__ double pos(double x) { return gt0(x) ? x : 0.0; }  // max(0, x)
__device__ __forceinline__ float pos(float x) { return fmaxf(0.0f, x); }
__device__ __forceinline__ double dmax(double x, double y) { return okey(x) >= okey(y) ? x : y; }
__device__ __forceinline__ float dmax(float x, float y) { return fmaxf(x, y); }
__device__ __forceinline__ double dmin(double x, double y) { return okey(x) <= okey(y) ? x : y; }
__device__ __forceinline__ float dmin(float x, float y) { return fminf(x, y); }
// the larger of two non-negative values (their bit patterns order like the values)
__device__ __forceinline__ double nmax(double x, double y) {
  return __double_as_longlong(x) >= __double_as_longlong(y) ? x : y;
}
__device__ __forceinline__ float nmax(float x, float y) { return fmaxf(x, y); }
__device__ __forceinline__ bool finite(double x) {
  return (__double_as_longlong(x) & 0x7ff0000000000000LL) != 0x7ff0000000000000LL;
}
__device__ __forceinline__ bool finite(float x) { return isfinite(x); }

// Elementary functions.  FP64: the IEEE-rounded library square root; division as a
// times the Newton-refined reciprocal f_rcp below; cube roots through f_rcbrt below.
// FP32-bulk: the hardware approximations (MUFU reciprocal square root, reciprocal,
// base-2 logarithm and exponent), a few ulp each -- far inside that mode's 1e-4 m
// accuracy target.  All are deterministic, so both sides of an edge still compute
// identical values.
//
// 1/x for FP64 by Newton-Raphson on f(r) = 1/r - x: from the hardware estimate
// (rcp.approx.ftz.f64), e = 1 - x r, r <- r + r e, which squares the relative error at
// each step (two steps reach the double's precision); within 2 ulp of the rounded
// reciprocal for normal x (no special-case path: 0 and infinities give NaN).
__device__ __forceinline__ double f_rcp(double x) {
  double r;
  asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(r) : "d"(x));
  double e = fma(-x, r, 1.0);
  r = fma(r, e, r);
  e = fma(-x, r, 1.0);
  return fma(r, e, r);
}
__device__ __forceinline__ double f_sqrt(double x) { return sqrt(x); }
__device__ __forceinline__ double f_div(double a, double b) { return a * f_rcp(b); }
__device__ __forceinline__ float f_sqrt(float x) { return x > 0.0f ? x * rsqrtf(x) : 0.0f; }
__device__ __forceinline__ float f_div(float a, float b) { return __fdividef(a, b); }
__device__ __forceinline__ float f_exp2(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// x^(-1/3) for x > 0.  FP32-bulk: 2^(-log2(x)/3) from the hardware approximations.
// FP64: that single-precision estimate refined by two Newton-Raphson steps on
// f(r) = r^-3 - x, r <- r (4 - x r^3) / 3, which converge quadratically (about 21
// correct bits -> 41 -> the full double) without a division or a library cube root;
// outside [1e-30, 1e30] (beyond the estimate's range) it falls back to 1 / cbrt(x).
__device__ __forceinline__ float f_rcbrt(float x) { return f_exp2(__log2f(x) * (-1.0f / 3.0f)); }
__device__ __forceinline__ double f_rcbrt(double x) {
  if (!(okey(x) >= okey(1e-30) && okey(x) <= okey(1e30))) return 1.0 / cbrt(x);
  double r = static_cast<double>(f_rcbrt(static_cast<float>(x)));
  constexpr double kThird = 1.0 / 3.0;
  r = r * fma(-x, r * r * r, 4.0) * kThird;
  r = r * fma(-x, r * r * r, 4.0) * kThird;
  return r;
}
// Cube root of x > 0: x r^2 with r = x^(-1/3).
__device__ __forceinline__ float f_cbrt(float x) { return f_exp2(__log2f(x) * (1.0f / 3.0f)); }
__device__ __forceinline__ double f_cbrt(double x) {
  const double r = f_rcbrt(x);
  return x * r * r;
}

// h^(5/3) for h > 0: h^2 h^(-1/3).
template <typename T>
__device__ __forceinline__ T pow53(T h) {
  return h * h * f_rcbrt(h);
}

// HLLC flux in the edge frame for the modified depths hL, hR (>= 0) with their
// celerities cL = sqrt(g hL), cR = sqrt(g hR); un/ut are normal/tangential
// velocities.  Wave speeds: two-rarefaction star estimates when both sides are
// wet, exact dry-front speeds when one side is dry.  pL, pR = g/2 h^2 are
// returned so the caller subtracts exactly the same values; right: the flux carries
// the right side's tangential velocity (and passive species), else the left's.
template <typename T>
__device__ __forceinline__ void hllc(T hL, T unL, T utL, T cL, T hR, T unR, T utR, T cR, T hg, T& F0, T& F1,
                                     T& F2, T& pL, T& pR, bool& right) {
  const T half = T(0.5), quarter = T(0.25), two = T(2), zero = T(0);
  const T us = half * (unL + unR) + cL - cR;
  const T cs = half * (cL + cR) + quarter * (unL - unR);
  T SL = dmin(unL - cL, us - cs);
  T SR = dmax(unR + cR, us + cs);
  const bool ldry = !gt0(hL), rdry = !gt0(hR);
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
  const T H2 = H0 * (le0(num) ? utL : utR);
  // the side whose tangential velocity (and passive species) the flux carries
  right = ge0(SL) ? false : (le0(SR) ? true : !le0(num));
  if (ge0(SL)) {
    F0 = FL0; F1 = FL1; F2 = FL2;
  } else if (le0(SR)) {
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
  if (gt(h, hmin)) {
    const T rh = f_div(T(1), h);
    u = qx * rh;
    v = qy * rh;
  }
  c = f_sqrt(g * pos(h));
}

// The free surface H of an FP32-bulk cell is the unevaluated sum hi + lo of two
// floats (offset from the FP64 datum); FP64 cells have lo = 0.  Depths are formed
// as (hi - z) + lo, so near-equal hi and z cancel exactly (Sterbenz) and the lo
// part keeps what a single float would round away; FP64 forms H - z, as the
// oracle does (adding a zero lo would cost an instruction and could flip the sign
// of a zero depth).
__device__ __forceinline__ float depth_of(float hi, float lo, float z) { return (hi - z) + lo; }
__device__ __forceinline__ double depth_of(double hi, double, double z) { return hi - z; }

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
    rmax = nmax(rmax, T(0.75) * ll * ia);
    ssum += ll;
  }
  return cfl_mode == 1 ? ssum * ia : rmax;
}

// FP64 -> FP32 by integer operations (the mantissa truncated, magnitudes below the FP32
// normal range to 0, above it and NaN to infinity): relative error below 2^-23 with no
// conversion instruction, for the rate screen below.
__device__ __forceinline__ float f32_trunc(double x) {
  const unsigned long long b = static_cast<unsigned long long>(__double_as_longlong(x));
  const unsigned hi = static_cast<unsigned>(b >> 32);
  const int e = static_cast<int>((hi >> 20) & 0x7ffu) - 896;  // the FP32 biased exponent
  const unsigned m = static_cast<unsigned>(b >> 29) & 0x7fffffu;
  const unsigned mag = e <= 0 ? 0u : (e >= 255 ? 0x7f800000u : (static_cast<unsigned>(e) << 23) | m);
  return __uint_as_float((hi & 0x80000000u) | mag);
}

// A single-precision screen of a wet FP64 cell's Eq. 21 rate (cell_rate of its depth
// h and discharge (qx, qy)): inputs truncated to FP32, the hardware reciprocal and
// reciprocal square root; relative error below 1e-5 of the FP64 rate.
__device__ __forceinline__ float cell_rate_screen(const double* nxs, const double* nys, const double* ls,
                                                  const int (&idx)[3], double h, double qx, double qy, double ia,
                                                  float g, int cfl_mode) {
  const float hf = f32_trunc(h), rh = __frcp_rn(hf);
  const float u = f32_trunc(qx) * rh, v = f32_trunc(qy) * rh, c = f_sqrt(g * hf), iaf = f32_trunc(ia);
  float rmax = 0.0f, ssum = 0.0f;
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const float ll = (fabsf(u * f32_trunc(nxs[idx[k]]) + v * f32_trunc(nys[idx[k]])) + c) * f32_trunc(ls[idx[k]]);
    rmax = fmaxf(rmax, 0.75f * ll * iaf);
    ssum += ll;
  }
  return cfl_mode == 1 ? ssum * iaf : rmax;
}

// ------------------------------------------------------------------ flood tracking

// The hydrodynamic module's "Flood" outputs per cell: the time the water front
// arrives (the first time the depth exceeds a threshold) and the running maxima of
// the depth h, the flow velocity |u| = |q| / h, the specific discharge |q| and the
// bed shear stress, Manning's rho g n^2 |u|^2 / h^(1/3) (= rho g h S_f with Eq. 2's
// friction slope; |u| and the stress are 0 at or below h_min).
constexpr double kRhoWater = 1000.0;  // density of water, kg / m^3

// The dimensionless friction coefficient c_f of Table 1's logarithmic closures (Eq. 2:
// S_f = u |u| / (g h c_f^2)): Chezy (r = K_s) c_f = 6.25 + ln(h / K_s) for h > K_s,
// else 6.25; Bezzola (r = y_R) 2.5 sqrt(1 - y_R / h) ln(10.9 h / y_R) for h / y_R > 2,
// 1.25 sqrt(h / y_R) ln(10.9 h / y_R) for 0.5 <= h / y_R <= 2, 1.5 below.
template <typename T>
__device__ __forceinline__ T closure_cf(int law, T h, T r) {
  if (law == 1) return h > r ? T(6.25) + log(h / r) : T(6.25);
  const T x = h / r;
  if (x > T(2)) return T(2.5) * sqrt(T(1) - r / h) * log(T(10.9) * h / r);
  if (x >= T(0.5)) return T(1.25) * sqrt(x) * log(T(10.9) * h / r);
  return T(1.5);
}

template <typename T>
__device__ __forceinline__ void track_values(T h, T qx, T qy, T gn2, T hmin, int law, T& q, T& u, T& tau) {
  q = f_sqrt(qx * qx + qy * qy);
  u = T(0);
  tau = T(0);
  if (h > hmin) {
    u = f_div(q, h);
    if (law == 0) {
      tau = static_cast<T>(kRhoWater) * gn2 * u * u * f_rcbrt(h);  // rho g n^2 u^2 / h^(1/3)
    } else {
      const T cf = closure_cf<T>(law, h, gn2);  // gn2 holds K_s or y_R
      tau = static_cast<T>(kRhoWater) * u * u / (cf * cf);  // rho u^2 / c_f^2
    }
  }
}

// A cell's record before this step's update (loaded early, so the loads overlap the
// update's arithmetic).
template <typename T>
struct TrackRecord {
  double t;
  T h, u, q, tau;
};
template <typename T>
__device__ __forceinline__ TrackRecord<T> track_load(const InstDesc<T>& a, int i) {
  return TrackRecord<T>{a.trk_t[i], a.trk_h[i], a.trk_u[i], a.trk_q[i], a.trk_tau[i]};
}
// Fold the cell's state U^{n+1} (depth h, discharge qx, qy) at time t into its record;
// stores only what changes.
template <typename T, bool kLaws>
__device__ __forceinline__ void track_update(const InstDesc<T>& a, int i, const TrackRecord<T>& r, T h, T qx, T qy,
                                             T gn2, T hmin, double t) {
  T q, u, tau;
  track_values<T>(h, qx, qy, gn2, hmin, kLaws ? a.fr_law : 0, q, u, tau);
  if (isnan(r.t) && h > a.trk_harr) a.trk_t[i] = t;
  if (h > r.h) a.trk_h[i] = h;
  if (u > r.u) a.trk_u[i] = u;
  if (q > r.q) a.trk_q[i] = q;
  if (tau > r.tau) a.trk_tau[i] = tau;
}

// Start the record from the instance's current state (cells 0..n-1, tile order).
template <typename T>
__global__ void track_init(const InstDesc<T>* d, const Ctl* ctl, int n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const InstDesc<T>& a = *d;
  const int par = ctl->parity;
  const T lo = sizeof(T) == 4 ? a.Hlo[par][i] : T(0);
  const T h = depth_of(a.H[par][i], lo, a.z[i]);
  const T hmin = sizeof(T) == 8 ? static_cast<T>(a.p.h_min) : static_cast<T>(a.p.hmin_f);
  T q, u, tau;
  track_values<T>(h, a.qx[par][i], a.qy[par][i], a.gn2[i], hmin, a.fr_law, q, u, tau);
  a.trk_t[i] = h > a.trk_harr ? ctl->t : static_cast<double>(NAN);
  a.trk_h[i] = h;
  a.trk_u[i] = u;
  a.trk_q[i] = q;
  a.trk_tau[i] = tau;
}

// The per-instance work at the end of a step is split three ways so that little of
// it remains on the launch's critical path (B300 executes FP64 at 2 lanes per SM and
// cycle, so FP64 chains and reductions in one CTA are slow; sums are finished in warp
// 0 in a fixed order, maxima run on integer bit patterns).  Each runs in the kTile
// compute threads of one CTA; cs is the control block as it was when the launch began
// (t, dt, t_end, clipped, parity, bvol do not change during a launch).  The time the
// step reaches: t^{n+1} after a step (advance = 1), t^n after prime (advance = 0).
__device__ __forceinline__ double new_time(const Ctl& cs, int advance) {
  return advance ? (cs.clipped ? cs.t_end : cs.t + cs.dt) : cs.t;
}

// Boundary volume: run by the CTA that completes the instance's last boundary tile.
template <typename T>
__device__ __noinline__ void finalize_boundary(const InstDesc<T>& a, const Ctl& cs, double* scratch) {
  const int tid = threadIdx.x;
  double bs = 0.0;
  for (int j = tid; j < a.n_btiles; j += kTile) bs += __ldcg(&a.part[j].bflux);
  scratch[tid] = bs;
  nbar<kTile>();
  if (tid < 32) {
    bs = 0.0;
    for (int k = tid; k < kTile; k += 32) bs += scratch[k];
    bs = warp_sum(bs);
    if (tid == 0) {
      a.ctl->bvol = cs.bvol - cs.dt * bs;
      atomicAnd(reinterpret_cast<unsigned long long*>(&a.ctl->in_done), 0x00000000ffffffffull);  // b_done = 0
    }
  }
  nbar<kTile>();
}

// Knuth's TwoSum: s = a + b rounded, e its rounding error (s + e == a + b exactly).
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = a + b;
  const float bb = s - a;
  e = (a - (s - bb)) + (b - bb);
}

// Inflow at the new time: Q(t), the conveyance-weighted split of Q (sum of l h^(5/3))
// and the largest inflow-edge rate lambda_b l / |Omega| of Eq. 21.  Run by the CTA that
// completes the instance's last inflow tile (only inflow tiles read the split, and
// they are all done).  B300 runs FP64 on two lanes per SM and cycle, and this runs on
// one SM, so the FP64 work is only what the result needs.  FP64: the weight sum in
// FP64, the split's two divisions once, and the exact rate of the few edges whose
// single-precision screen (inputs truncated by integer operations) can reach the
// maximum, which is therefore the exact FP64 maximum.  FP32-bulk (whose cell rates are
// single precision): the weight sum as an exact FP32 pair sum (products split by FMA,
// TwoSum), the rate the largest single-precision edge rate.  Every global load is
// issued first.  sred: 9 doubles, sbc: 4, scratch: kTile.
template <typename T>
__device__ __noinline__ void finalize_inflow(const InstDesc<T>& a, const Ctl& cs, int advance, double* sred,
                                             double* sbc, double* scratch) {
  constexpr bool k64 = sizeof(T) == 8;
  Ctl* ctl = a.ctl;
  const int tid = threadIdx.x;
  const double g = a.p.g;
  unsigned long long* ured = reinterpret_cast<unsigned long long*>(sred);
  auto f32 = [](T x) -> float {
    if constexpr (k64) return f32_trunc(x);
    else return x;
  };
  constexpr int U = 4;
  const int ni = a.n_inflow;
  T pwv[U], lv[U], hsv[U];
  double liad[U];
#pragma unroll
  for (int u = 0; u < U; ++u) {
    const int j = tid + u * kTile;
    const bool in = j < ni;
    pwv[u] = in ? __ldcg(&a.in_pw[j]) : T(0);
    lv[u] = in ? a.in_len[j] : T(0);
    hsv[u] = in ? __ldcg(&a.in_hs[j]) : T(0);
    liad[u] = in ? a.in_lia[j] : 0.0;
  }
  // Q(t): the thread of the hydrograph segment that contains t evaluates it
  const int nq = a.p.hydro_n;
  if (tid == 0 && nq <= 0) sbc[0] = 0.0;
  if (tid <= nq && nq > 0) {
    const double t = new_time(cs, advance);
    const double* ht = a.p.hydro_t;
    const double* hq = a.p.hydro_q;
    for (int i = tid; i <= nq; i += kTile) {
      if (i == 0) {
        if (t <= ht[0]) sbc[0] = hq[0];
      } else if (i == nq) {
        if (t > ht[nq - 1]) sbc[0] = hq[nq - 1];
      } else if (t > ht[i - 1] && t <= ht[i]) {
        const double wgt = (t - ht[i - 1]) / (ht[i] - ht[i - 1]);
        sbc[0] = hq[i - 1] + wgt * (hq[i] - hq[i - 1]);
      }
    }
  }
  // the weight sum W = sum of l h^(5/3), thread 0 then the split: q_e = qscale h_e^(5/3)
  // where some inflow cell is wet, else the uniform quni on every inflow edge
  if constexpr (k64) {
    double wsum = 0.0;
#pragma unroll
    for (int u = 0; u < U; ++u) wsum += lv[u] * pwv[u];
    for (int j = tid + U * kTile; j < ni; j += kTile) wsum += a.in_len[j] * __ldcg(&a.in_pw[j]);
    scratch[tid] = wsum;
    nbar<kTile>();
    if (tid < 32) {
      wsum = 0.0;
      for (int k = tid; k < kTile; k += 32) wsum += scratch[k];
      scratch[tid] = warp_sum(wsum);  // (lane 0's is the sum)
    }
  } else {
    float hi = 0.0f, lo = 0.0f;
    auto add = [&](float x, float y) {  // (hi, lo) += x * y, exactly up to the pair's rounding
      const float p = x * y, e = fmaf(x, y, -p);
      float s2, e2;
      two_sum(hi, p, s2, e2);
      hi = s2;
      lo += e2 + e;
    };
#pragma unroll
    for (int u = 0; u < U; ++u) add(lv[u], pwv[u]);
    for (int j = tid + U * kTile; j < ni; j += kTile) add(a.in_len[j], __ldcg(&a.in_pw[j]));
    for (int o = 16; o > 0; o >>= 1) {
      const float h2 = __shfl_xor_sync(0xffffffffu, hi, o), l2 = __shfl_xor_sync(0xffffffffu, lo, o);
      float s2, e2;
      two_sum(hi, h2, s2, e2);
      hi = s2;
      lo += l2 + e2;
    }
    float* sp = reinterpret_cast<float*>(scratch);
    if ((tid & 31) == 0) {
      sp[2 * (tid >> 5)] = hi;
      sp[2 * (tid >> 5) + 1] = lo;
    }
    nbar<kTile>();
    if (tid == 0) {
      hi = sp[0];
      lo = sp[1];
      for (int w = 1; w < kTile / 32; ++w) {
        float s2, e2;
        two_sum(hi, sp[2 * w], s2, e2);
        hi = s2;
        lo += sp[2 * w + 1] + e2;
      }
      scratch[0] = static_cast<double>(hi) + static_cast<double>(lo);
    }
  }
  if (tid == 0) {
    const double Q = sbc[0], wsum = scratch[0];
    const bool wpos = wsum > 0.0;
    sbc[1] = wpos ? Q / wsum : 0.0;
    sbc[2] = (!wpos && a.inflow_len > 0.0) ? Q / a.inflow_len : 0.0;
    reinterpret_cast<int*>(&sbc[3])[0] = wpos ? 1 : 0;
  }
  nbar<kTile>();
  const float qscf = f32_trunc(sbc[1]), qunf = f32_trunc(sbc[2]);
  const bool wpos = reinterpret_cast<const int*>(&sbc[3])[0] != 0;
  const float gf = a.p.g_f;
  const float facf = a.p.cfl_mode == 0 ? 0.75f : 1.0f;
  // the edges' single-precision rates (FP64: a screen within 1e-5 of the rate)
  auto screen = [&](float pw, float hs, float lia) {
    const float q = wpos ? qscf * pw : qunf;
    const float hbf = fmaxf(hs, f_cbrt(fmaxf(q, 1e-30f) * q / gf));
    return q > 0.0f ? (q / hbf + sqrtf(gf * hbf)) * lia * facf : 0.0f;
  };
  float scr[U];
  float rbf = 0.0f;
#pragma unroll
  for (int u = 0; u < U; ++u) {
    scr[u] = tid + u * kTile < ni ? screen(f32(pwv[u]), f32(hsv[u]), f32_trunc(liad[u])) : 0.0f;
    rbf = fmaxf(rbf, scr[u]);
  }
  for (int j = tid + U * kTile; j < ni; j += kTile)
    rbf = fmaxf(rbf, screen(f32(__ldcg(&a.in_pw[j])), f32(__ldcg(&a.in_hs[j])), f32_trunc(a.in_lia[j])));
  // the largest (non-negative floats order as their bits)
  {
    unsigned v = __reduce_max_sync(0xffffffffu, __float_as_uint(rbf));
    if ((tid & 31) == 0) reinterpret_cast<unsigned*>(scratch)[32 + (tid >> 5)] = v;
    nbar<kTile>();
    v = __reduce_max_sync(0xffffffffu, reinterpret_cast<const unsigned*>(scratch)[32 + (tid & 7)]);
    rbf = __uint_as_float(v);
  }
  double rb;
  if constexpr (k64) {
    auto exact = [&](double pw, double hs, double lia) {
      const double q = wpos ? sbc[1] * pw : sbc[2];
      if (!(q > 0.0)) return 0.0;
      const double hb = fmax(hs, f_cbrt(q * q / g));
      return (q / hb + sqrt(g * hb)) * lia * (a.p.cfl_mode == 0 ? 0.75 : 1.0);
    };
    const float thr = rbf * (1.0f - 1e-4f);
    rb = 0.0;
#pragma unroll
    for (int u = 0; u < U; ++u)
      if (tid + u * kTile < ni && scr[u] >= thr && rbf > 0.0f) rb = fmax(rb, exact(pwv[u], hsv[u], liad[u]));
    for (int j = tid + U * kTile; j < ni; j += kTile) {
      const double pw = __ldcg(&a.in_pw[j]), hs = __ldcg(&a.in_hs[j]), lia = a.in_lia[j];
      if (screen(f32(pw), f32(hs), f32_trunc(lia)) >= thr && rbf > 0.0f) rb = fmax(rb, exact(pw, hs, lia));
    }
    rb = block_max_nonneg_all<kTile>(rb, ured);
  } else {
    rb = static_cast<double>(rbf);
  }
  if (tid == 0) {
    ctl->rb = rb;
    ctl->Q = sbc[0];
    ctl->qscale = sbc[1];
    ctl->quni = sbc[2];
    ctl->quni_f = static_cast<float>(sbc[2]);
    ctl->wpos = wpos ? 1 : 0;
    atomicAnd(reinterpret_cast<unsigned long long*>(&ctl->in_done), 0xffffffff00000000ull);  // in_done = 0
  }
  nbar<kTile>();
}

// ------------------------------------------------------------------ outflow laws

// The boundary state of an outflow edge (h-Q relation, weir; Section "Boundary
// conditions", standard outflows) that lets the unit discharge q > 0 leave a cell of
// depth h and outward normal velocity un: the depth h_b on the cell's outgoing
// characteristic, q / h_b + 2 sqrt(g h_b) = w = un + 2 sqrt(g h), on its subcritical
// branch (u_b <= sqrt(g h_b)).  q is first capped at the critical discharge
// w^3 / (27 g), the largest the invariant admits (h_b is then the critical depth
// (w / 3)^2 / g).  Returns h_b, or -1 with q = 0 when nothing can leave (w <= 0).
// Newton's method on s = sqrt(h_b) for f(s) = 2 sqrt(g) s + q / s^2 - w, convex in s,
// from s = max(sqrt(h), the minimum of f): from the right of the root it descends
// monotonically, from its left the first step lands to its right.  IEEE division and
// square roots: the edges are few, and the iteration converges to the last bits.
template <typename T>
__device__ __noinline__ T outflow_state(T h, T un, T g, T& q) {
  const T w = un + T(2) * sqrt(g * h);
  if (!(w > T(0))) {
    q = T(0);
    return T(-1);
  }
  const T qmax = w * w * w / (T(27) * g);
  if (q >= qmax) {
    q = qmax;
    const T w3 = w / T(3);
    return w3 * w3 / g;
  }
  const T sg = sqrt(g);
  T s = fmax(sqrt(h), cbrt(q / sg));
  const T eps = sizeof(T) == 8 ? T(1e-16) : T(1e-7);
  for (int it = 0; it < 100; ++it) {
    const T f = T(2) * sg * s + q / (s * s) - w;
    const T df = T(2) * sg - T(2) * q / (s * s * s);
    if (!(df > T(0))) break;
    const T ds = f / df;
    s -= ds;
    if (fabs(ds) <= eps * s) break;
  }
  return s * s;
}

// Poleni's weir discharge per unit crest width leaving a cell with surface (Hh, Hl),
// bed z and depth h: (2/3) mu sqrt(2 g) eta^(3/2) = weir_k eta^(3/2), eta the head of
// the surface over the crest, a crest below the bed taken at the bed (free overfall);
// 0 for a dry cell or water at or below the crest.
template <typename T>
__device__ __forceinline__ T weir_discharge(const InstDesc<T>& a, T Hh, T Hl, T z, T h, T hmin) {
  const T eta = depth_of(Hh, Hl, fmax(a.weir_crest, z));
  return (h > hmin && eta > T(0)) ? a.weir_k * eta * sqrt(eta) : T(0);
}

// The largest Eq. 21 rate of a cell's weir edges at its new state (surface (Hh, Hl),
// bed z, depth h, velocity (u, v)): the boundary state's u_b + sqrt(g h_b), times
// l / |Omega| (and 3/4 for Eq. 21's rho = 4 |Omega| / (3 l)); 0 if nothing leaves.
template <typename T>
__device__ __noinline__ T weir_rate(const InstDesc<T>& a, const uint32_t* sLR, const T* sNx, const T* sNy,
                                    const T* sLn, const int (&idx)[3], T Hh, T Hl, T z, T h, T u, T v, T ia) {
  const T g = static_cast<T>(a.p.g), hmin = static_cast<T>(a.p.h_min);
  T r = T(0);
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const int e = idx[k];
    const int code = static_cast<int32_t>(sLR[e]) >> kLocBits;
    if (code > kInflow || kInflow - code < a.n_inflow + a.n_hq ||
        kInflow - code >= a.n_inflow + a.n_hq + a.n_weir)
      continue;
    T q = weir_discharge<T>(a, Hh, Hl, z, h, hmin);
    const T hb = q > T(0) ? outflow_state<T>(h, u * sNx[e] + v * sNy[e], g, q) : T(-1);
    if (hb > T(0)) r = fmax(r, (q / hb + sqrt(g * hb)) * sLn[e] * ia * (a.p.cfl_mode == 0 ? T(0.75) : T(1)));
  }
  return r;
}

// ------------------------------------------------------------------ water-level edges

// The imposed water surface Z_b(t) of the level edges (Section "Boundary conditions",
// the zhydrograph of the standard inflows and outflows): piecewise linear through
// (zh_t, zh_v), constant beyond its ends (zh_n >= 1).
template <typename T>
__device__ __forceinline__ double level_at(const InstDesc<T>& a, double t) {
  const int n = a.zh_n;
  if (t <= a.zh_t[0]) return a.zh_v[0];
  for (int k = 1; k < n; ++k)
    if (t <= a.zh_t[k]) {
      const double w = (t - a.zh_t[k - 1]) / (a.zh_t[k] - a.zh_t[k - 1]);
      return a.zh_v[k - 1] + w * (a.zh_v[k] - a.zh_v[k - 1]);
    }
  return a.zh_v[n - 1];
}

// Z_b(t) as the state stores a surface: FP64 as is (lo = 0); FP32-bulk as the pair of
// floats (hi, lo) of its offset from the datum, rounded the way an uploaded surface is,
// so still water at the imposed level has exactly the boundary's depth.
template <typename T>
__device__ __forceinline__ void level_pair(const InstDesc<T>& a, double t, T& hi, T& lo) {
  const double v = level_at(a, t) - a.datum;
  hi = static_cast<T>(v);
  lo = static_cast<T>(v - static_cast<double>(hi));
}

// The boundary state of a level edge of a cell with bed z, depth h >= 0 and outward
// normal velocity un: the imposed surface over the cell's bed, h_b = max(0, Z_b - z),
// with the normal velocity that keeps the cell's outgoing Riemann invariant,
// u_b = un + 2 sqrt(g h) - 2 sqrt(g h_b) (u_b = 0 next to a cell at or below h_min: the
// boundary water floods it as a dam break); c_b = sqrt(g h_b).  The tangential
// velocity is the cell's.
template <typename T>
__device__ __forceinline__ void level_state(T zh_hi, T zh_lo, T z, T h, T un, T g, T hmin, T& hb, T& ub, T& cb) {
  hb = fmax(T(0), depth_of(zh_hi, zh_lo, z));
  cb = sqrt(g * hb);
  ub = h > hmin ? un + T(2) * sqrt(g * h) - T(2) * cb : T(0);
}

// The largest Eq. 21 rate of a cell's level edges at its new state (bed z, depth h,
// velocity (u, v)) under the surface pair (zh_hi, zh_lo) of the new time: the boundary
// state's |u_b| + sqrt(g h_b), times l / |Omega| (and 3/4 for Eq. 21's
// rho = 4 |Omega| / (3 l)); dry cells count too (u_b = 0 there).
template <typename T>
__device__ __noinline__ T level_rate(const InstDesc<T>& a, const uint32_t* sLR, const T* sNx, const T* sNy,
                                     const T* sLn, const int (&idx)[3], T zh_hi, T zh_lo, T z, T h, T u, T v,
                                     T ia) {
  const T g = static_cast<T>(a.p.g), hmin = static_cast<T>(a.p.h_min);
  const int j0 = a.n_inflow + a.n_hq + a.n_weir;
  T r = T(0);
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const int e = idx[k];
    const int code = static_cast<int32_t>(sLR[e]) >> kLocBits;
    if (code > kInflow || kInflow - code < j0) continue;
    T hb, ub, cb;
    level_state<T>(zh_hi, zh_lo, z, fmax(T(0), h), u * sNx[e] + v * sNy[e], g, hmin, hb, ub, cb);
    const T lb = fabs(ub) + cb;
    if (lb > T(0)) r = fmax(r, lb * sLn[e] * ia * (a.p.cfl_mode == 0 ? T(0.75) : T(1)));
  }
  return r;
}

// The rating curve of the h-Q relation: piecewise linear through (hq_s, hq_q), constant
// beyond its ends; 0 without a table.
template <typename T>
__device__ __forceinline__ double rating_curve(const InstDesc<T>& a, double S) {
  const int n = a.hq_n;
  if (n <= 0) return 0.0;
  if (S <= a.hq_s[0]) return a.hq_q[0];
  for (int k = 1; k < n; ++k) {
    if (S <= a.hq_s[k]) {
      const double w = (S - a.hq_s[k - 1]) / (a.hq_s[k] - a.hq_s[k - 1]);
      return a.hq_q[k - 1] + w * (a.hq_q[k] - a.hq_q[k - 1]);
    }
  }
  return a.hq_q[n - 1];
}

// h-Q outflow at the new time: the stage S (length-weighted mean surface over the h-Q
// edges whose cell is wet), Q = the rating curve at S, its conveyance split over those
// edges, q_e = Q h_e^(5/3) / sum_f l_f h_f^(5/3) (stored for the next step's fluxes),
// and the largest h-Q-edge rate of Eq. 21 (the boundary state's u_b + sqrt(g h_b)).
// Run, in FP64, by the CTA that completes the instance's last h-Q tile (the state of
// every h-Q cell at the new time is in memory).  sred: 9 doubles, sbc: 4.
template <typename T>
__device__ __noinline__ void finalize_hq(const InstDesc<T>& a, const Ctl& cs, int advance, double* sred,
                                         double* sbc) {
  constexpr bool kPair = sizeof(T) == 4;
  const int tid = threadIdx.x;
  const int b = advance ? (cs.parity ^ 1) : cs.parity;  // the buffer holding the new state
  const int j0 = a.n_inflow, j1 = a.n_inflow + a.n_hq;
  const double g = a.p.g, hmin = a.p.h_min;
  auto depth = [&](int i, double* Habs) {
    const double Hh = static_cast<double>(__ldcg(&a.H[b][i]));
    const double Hl = kPair ? static_cast<double>(__ldcg(&a.Hlo[b][i])) : 0.0;
    *Habs = (a.datum + Hh) + Hl;
    return (Hh - static_cast<double>(a.z[i])) + Hl;
  };
  double sl = 0.0, sH = 0.0, sw = 0.0;
  for (int j = j0 + tid; j < j1; j += kTile) {
    double Habs;
    const double h = depth(a.in_cell[j], &Habs);
    if (h > hmin) {
      const double l = static_cast<double>(a.in_len[j]);
      sl += l;
      sH += l * Habs;
      sw += l * pow53(h);
    }
  }
  sl = block_sum<kTile>(sl, sred);
  if (tid == 0) sbc[0] = sl;
  sH = block_sum<kTile>(sH, sred);
  if (tid == 0) sbc[1] = sH;
  sw = block_sum<kTile>(sw, sred);
  if (tid == 0) {
    sbc[2] = sw;
    sbc[3] = sbc[0] > 0.0 ? rating_curve(a, sbc[1] / sbc[0]) : 0.0;
  }
  nbar<kTile>();
  const double Q = sbc[3], W = sbc[2];
  const double fac = a.p.cfl_mode == 0 ? 0.75 : 1.0;
  double rb = 0.0;
  for (int j = j0 + tid; j < j1; j += kTile) {
    const int i = a.in_cell[j];
    double Habs;
    const double h = depth(i, &Habs);
    double q = (h > hmin && W > 0.0) ? Q * pow53(h) / W : 0.0;
    a.in_pw[j] = static_cast<T>(q);
    if (q > 0.0) {
      const double un = (static_cast<double>(__ldcg(&a.qx[b][i])) * a.in_nx[j] +
                         static_cast<double>(__ldcg(&a.qy[b][i])) * a.in_ny[j]) / h;
      const double hb = outflow_state<double>(h, un, g, q);
      if (hb > 0.0) rb = fmax(rb, (q / hb + sqrt(g * hb)) * a.in_lia[j] * fac);
    }
  }
  rb = block_max_nonneg_all<kTile>(rb, reinterpret_cast<unsigned long long*>(sred));
  if (tid == 0) {
    a.ctl->rb_out = rb;
    a.ctl->hq_done = 0u;
  }
  nbar<kTile>();
}

// The step itself: run (thread 0 only) by the CTA that completes the instance's last
// tile, after the inflow, h-Q and boundary parts (their CTAs counted their tiles after
// them).  dt^{n+1} from the maximum cell rate and inflow / h-Q rate (Eq. 21), then time,
// parity and step count.
template <typename T>
__device__ __forceinline__ void finalize_step(const InstDesc<T>& a, const Ctl& cs, int advance) {
  Ctl* ctl = a.ctl;
  const double t = new_time(cs, advance);
  const double rcell = __longlong_as_double(static_cast<long long>(__ldcg(&ctl->rmax_bits)));
  const double rb = fmax(a.n_in_tiles > 0 ? __ldcg(&ctl->rb) : 0.0, a.n_hq_tiles > 0 ? __ldcg(&ctl->rb_out) : 0.0);
  if (advance) {
    ctl->t = t;
    ctl->parity = cs.parity ^ 1;
    ctl->steps = cs.steps + 1;
  }
  if (a.n_in_tiles == 0) {
    ctl->Q = 0.0;
    ctl->qscale = 0.0;
    ctl->quni = 0.0;
    ctl->quni_f = 0.0f;
    ctl->wpos = 0;
  }
  ctl->rmax_bits = 0ull;
  const double r = fmax(rcell, rb);
  double dtc = r > 0.0 ? a.p.cfl / r : a.p.dt_max;
  if (dtc > a.p.dt_max) dtc = a.p.dt_max;
  ctl->dt_cfl = dtc;
  double dt = dtc;
  int clipped = 0;
  if (dt >= cs.t_end - t) {
    dt = cs.t_end - t;
    clipped = 1;
  }
  ctl->dt = dt;
  ctl->dt_f = static_cast<float>(dt);
  ctl->clipped = clipped;
  ctl->active = t < cs.t_end ? 1 : 0;
  ctl->done = 0u;
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

// External sources (Section "External inflow/outflow discharge"): S_h of every region
// at t^n -- its series v(t), piecewise linear through its points and constant beyond
// the ends, as a total discharge over the region's area (kind 0, m^3/s) or an
// intensity (kind 1, mm/h).  Launched before each step; nothing once the run ended.
template <typename T>
__global__ void source_rates(const Ctl* ctl, int n_regions, const int32_t* kind, const long long* off,
                             const double* ts, const double* vs, const double* area, T* rate) {
  if (!ctl->active) return;
  const double t = ctl->t;
  for (int r = threadIdx.x; r < n_regions; r += blockDim.x) {
    const long long a = off[r], b = off[r + 1];
    double v = vs[a];
    if (t > ts[a]) {
      v = vs[b - 1];
      for (long long k = a + 1; k < b; ++k)
        if (t <= ts[k]) {
          const double w = (t - ts[k - 1]) / (ts[k] - ts[k - 1]);
          v = vs[k - 1] + w * (vs[k] - vs[k - 1]);
          break;
        }
    }
    rate[r] = static_cast<T>(kind[r] == 0 ? v / area[r] : v / 3.6e6);
  }
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
  // the state's own bed: the datum plus the bed's FP32 offset, formed as a download
  // forms a dry cell's surface (it may round either way of the FP64 bed).  Below both
  // beds is an error.  Dry: exactly on the FP64 bed (an FP64 dry cell) or at or below
  // the state's own bed (a downloaded dry cell uploads as dry, not as a film of the
  // rounding); a film between the two beds (a downloaded wet cell thinner than the
  // bed's rounding) stays the film it was
  const double Hb = datum + static_cast<double>(zf[i]);
  if (H < zd[i] && H < Hb) atomicOr(bad, 2);
  if (H == zd[i] || H <= Hb) {
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
