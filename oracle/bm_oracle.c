/*
 * bm_oracle.c -- plain, serial, FP64 CPU oracle for the explicit finite-volume
 * time step of the 2D shallow-water equations of BASEMENT v3 (arXiv 2102.12862,
 * Section "Numerical solution", subsection "Hydrodynamics").
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may link, import or call
 * this file; only the tests, the smoke check and the CPU-baseline leg of the
 * benchmark do.  It shares no code, header, table or helper with the CUDA path.
 *
 * It is written as an EDGE loop (each edge visited once, in the caller's cell
 * numbering), deliberately unlike the tiled GPU kernel, and is compiled with
 * -O2 -ffp-contract=off so every operation rounds once, in source order.
 *
 * What one step computes (all in the unknowns of Eq. 1 / Eq. 10: H, q_x, q_y):
 *   0. dt from Eq. 21 on U^n (rho_ij = 4|Omega_i|/(3 l_ij), lambda = |u.n| + sqrt(g h)),
 *      clipped by dt_max (parameter list of the hydrodynamic module) and t_end.
 *   1. per edge: modified states (hydrostatic reconstruction on max(z_L, z_R),
 *      the bed treatment named in the "Hydrodynamics" numerics subsection), HLLC
 *      flux (Toro 2001 ch. 10, named in the same subsection) in the edge frame,
 *      pre-balanced pressure correction 1/2 g h*^2 of each side.
 *   2. boundary edges: wall (mirror), transmissive (zero gradient), discharge
 *      inflow, the outflows h-Q relation (rating curve) and weir (Poleni), and the
 *      water level (zhydrograph: a boundary state under an imposed surface)
 *      (Section "Boundary conditions": standard inflow / outflow / wall).
 *   3. conservative update, Eq. 12.
 *   4. Manning friction (Eq. 2, Table 1) split off and integrated with a
 *      two-stage semi-implicit Runge-Kutta (Heun) step.
 *   5. q := 0 on cells whose depth is below the minimum water depth.
 * Optional: external sources in step 3 (orc_set_sources), the bed update of the
 * morphodynamic module (orc_set_morpho), flood tracking after each step (orc_track),
 * passive species advected with each step (orc_run_scalars).
 *
 * Readings where the paper is silent are the same as in the design notes:
 * modified-state form, Toro wave speeds, h_min, friction stages, rho_ij, the
 * inflow distribution, wall mass flux exactly zero.
 *
 * Pinned by tests/test_oracle_*.py (closed forms, invariants, paper values; the
 * inflow split by a channel held at its normal flow and hand-computed boundary wave
 * speeds; the speeds of Eq. 16 by the waves of the coupled shallow-water-Exner
 * system); the wet/dry threshold logic by Ritter's dry-bed dam break, the lake at rest
 * with dry islands and wet/dry mass conservation (h_min's value is a reading).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_OK 0
#define ORC_EINVAL 1
#define ORC_ENOMEM 2

/* parameters of one run (hydrodynamic module parameter list) */
typedef struct {
  double cfl;      /* Eq. 21 coefficient, default 0.9 */
  double g;        /* gravity, 9.81 */
  double h_min;    /* minimum water depth */
  double dt_max;   /* upper limit of the time step */
  int cfl_mode;    /* 0: Eq. 21 literally; 1: dt <= |Omega_i| / sum_j l_ij lambda_ij */
  const double *hydro_t, *hydro_q; /* inflow hydrograph Q(t), piecewise linear */
  int64_t hydro_n;
} orc_params;

typedef struct {
  int64_t n_cells, n_edges;
  /* per edge: left cell, right cell (>= 0) or boundary code -1 - tag; unit
   * normal pointing from left to right; length. left < right for interior edges. */
  int64_t *eL, *eR;
  double *nx, *ny, *len;
  /* per cell */
  double *area, *z, *man;
  int64_t *cedge;        /* 3 per cell: edge index of local edge k */
  /* per edge, filled each step: flux contribution to the left and to the right
   * cell, already multiplied by the edge length */
  double *cL, *cR;       /* 3 per edge */
  double *qin;           /* per edge: imposed unit discharge on inflow edges */
  double inflow_len;     /* total length of the inflow boundary */
  /* outflow boundaries (orc_set_outflow): the h-Q relation's table of stage (strictly
   * increasing) and discharge (tag 3); the weir's crest elevation and Poleni
   * coefficient (tag 4); per edge the unit discharge leaving through it */
  int64_t hq_n;
  double *hq_s, *hq_q;
  double weir_crest, weir_mu;
  /* water-level boundary (zhydrograph, tag 5; orc_set_level): the water surface
   * elevation Z_b(t), piecewise linear through (zh_t[k], zh_v[k]), constant beyond the
   * ends (zh_n = 0: the level edges are walls); zh_now = Z_b at the current step */
  int64_t zh_n;
  double *zh_t, *zh_v;
  double zh_now;
  double *qout;
  orc_params p;
  double *ht, *hq;
  /* external sources (orc_set_sources): region of each cell (-1: none); per region
   * kind, mode, area and a piecewise-linear series (src_off[r] .. src_off[r+1]) */
  int32_t src_n;
  int32_t *src_reg, *src_kind, *src_mode;
  int64_t *src_off;
  double *src_t, *src_v, *src_area, *src_rate;
  double src_vol; /* volume the sources added (negative: removed) since they were set */
  /* morphodynamics (orc_set_morpho): on/off, porosity p, relative density s, grain
   * diameter d, MPM-like alpha, m, theta_cr; per cell bedload vector and dq_B/dq; per
   * edge l q_Bij (outward from the left cell); bed volume through the boundary */
  int morpho;
  double mp_p, mp_s, mp_d, mp_alpha, mp_m, mp_thcr;
  double *qbx, *qby, *qbd, *fb;
  double bed_bvol;
  /* friction closure (orc_set_friction): 0 Manning (man = n), 1 Chezy (man = K_s),
   * 2 Bezzola (man = y_R) */
  int fr_law;
} orc_mesh;

/* ---------- mesh topology (independent, plain) ---------- */

typedef struct { int64_t a, b, t; int k; } orc_half;

static int cmp_half(const void* x, const void* y) {
  const orc_half* u = (const orc_half*)x;
  const orc_half* v = (const orc_half*)y;
  if (u->a != v->a) return u->a < v->a ? -1 : 1;
  if (u->b != v->b) return u->b < v->b ? -1 : 1;
  if (u->t != v->t) return u->t < v->t ? -1 : 1;
  return u->k - v->k;
}

void orc_destroy(orc_mesh* m) {
  if (!m) return;
  free(m->eL); free(m->eR); free(m->nx); free(m->ny); free(m->len);
  free(m->area); free(m->z); free(m->man); free(m->cedge);
  free(m->cL); free(m->cR); free(m->qin); free(m->ht); free(m->hq);
  free(m->qout); free(m->hq_s); free(m->hq_q); free(m->zh_t); free(m->zh_v);
  free(m->src_reg); free(m->src_kind); free(m->src_mode); free(m->src_off);
  free(m->src_t); free(m->src_v); free(m->src_area); free(m->src_rate);
  free(m->qbx); free(m->qby); free(m->qbd); free(m->fb);
  free(m);
}

/*
 * Build the finite-volume mesh of Section "Domain discretization": cells are
 * triangles, l_ij and n_ij (unit, pointing from i to j) per edge, |Omega_i| per
 * cell.  Clockwise triangles are reoriented; their edge tags follow the edges.
 * edge_tag[3t+k] tags edge (v_k, v_{k+1}) of the triangle as given: 0 wall,
 * 1 transmissive, 2 inflow, 3 h-Q outflow, 4 weir outflow (their laws are set by
 * orc_set_outflow; until then they let nothing out), 5 water level (zhydrograph; its
 * series is set by orc_set_level, until then a wall).  Returns ORC_EINVAL on any
 * malformed input.
 */
int orc_create(int64_t n_nodes, const double* xy, int64_t n_tri, const int32_t* tri,
               const double* z, const double* man, const uint8_t* edge_tag,
               const orc_params* p, orc_mesh** out) {
  *out = NULL;
  if (n_tri <= 0 || n_nodes < 3) return ORC_EINVAL;
  orc_mesh* m = (orc_mesh*)calloc(1, sizeof(orc_mesh));
  if (!m) return ORC_ENOMEM;
  m->n_cells = n_tri;
  m->p = *p;
  int64_t N = n_tri;
  m->area = (double*)malloc(N * sizeof(double));
  m->z = (double*)malloc(N * sizeof(double));
  m->man = (double*)malloc(N * sizeof(double));
  m->cedge = (int64_t*)malloc(3 * N * sizeof(int64_t));
  int32_t* v = (int32_t*)malloc(3 * N * sizeof(int32_t));
  uint8_t* tg = (uint8_t*)malloc(3 * N);
  orc_half* hs = (orc_half*)malloc(3 * N * sizeof(orc_half));
  if (!m->area || !m->z || !m->man || !m->cedge || !v || !tg || !hs) {
    free(v); free(tg); free(hs); orc_destroy(m); return ORC_ENOMEM;
  }
  int rc = ORC_OK;
  for (int64_t t = 0; t < N && rc == ORC_OK; ++t) {
    int32_t a = tri[3 * t], b = tri[3 * t + 1], c = tri[3 * t + 2];
    if (a < 0 || b < 0 || c < 0 || a >= n_nodes || b >= n_nodes || c >= n_nodes) { rc = ORC_EINVAL; break; }
    double ax = xy[2 * a], ay = xy[2 * a + 1], bx = xy[2 * b], by = xy[2 * b + 1];
    double cx = xy[2 * c], cy = xy[2 * c + 1];
    double twice = (bx - ax) * (cy - ay) - (cx - ax) * (by - ay);
    if (twice < 0) { /* clockwise: swap v1, v2; edge k of the new triangle is old edge 2,1,0 */
      v[3 * t] = a; v[3 * t + 1] = c; v[3 * t + 2] = b;
      tg[3 * t] = edge_tag[3 * t + 2]; tg[3 * t + 1] = edge_tag[3 * t + 1]; tg[3 * t + 2] = edge_tag[3 * t];
      twice = -twice;
    } else {
      v[3 * t] = a; v[3 * t + 1] = b; v[3 * t + 2] = c;
      tg[3 * t] = edge_tag[3 * t]; tg[3 * t + 1] = edge_tag[3 * t + 1]; tg[3 * t + 2] = edge_tag[3 * t + 2];
    }
    if (!(twice > 0)) { rc = ORC_EINVAL; break; }
    m->area[t] = 0.5 * twice;
    m->z[t] = z[t];
    m->man[t] = man[t];
    if (!(man[t] >= 0) || !isfinite(z[t])) { rc = ORC_EINVAL; break; }
    for (int k = 0; k < 3; ++k) {
      int64_t p0 = v[3 * t + k], p1 = v[3 * t + (k + 1) % 3];
      hs[3 * t + k].a = p0 < p1 ? p0 : p1;
      hs[3 * t + k].b = p0 < p1 ? p1 : p0;
      hs[3 * t + k].t = t;
      hs[3 * t + k].k = k;
    }
  }
  if (rc != ORC_OK) { free(v); free(tg); free(hs); orc_destroy(m); return rc; }
  qsort(hs, 3 * N, sizeof(orc_half), cmp_half);
  /* count edges */
  int64_t ne = 0;
  for (int64_t i = 0; i < 3 * N;) {
    int64_t j = i + 1;
    while (j < 3 * N && hs[j].a == hs[i].a && hs[j].b == hs[i].b) ++j;
    if (j - i > 2) { rc = ORC_EINVAL; break; }
    ++ne; i = j;
  }
  if (rc != ORC_OK) { free(v); free(tg); free(hs); orc_destroy(m); return rc; }
  m->n_edges = ne;
  m->eL = (int64_t*)malloc(ne * sizeof(int64_t));
  m->eR = (int64_t*)malloc(ne * sizeof(int64_t));
  m->nx = (double*)malloc(ne * sizeof(double));
  m->ny = (double*)malloc(ne * sizeof(double));
  m->len = (double*)malloc(ne * sizeof(double));
  m->cL = (double*)malloc(3 * ne * sizeof(double));
  m->cR = (double*)malloc(3 * ne * sizeof(double));
  m->qin = (double*)calloc(ne, sizeof(double));
  m->qout = (double*)calloc(ne, sizeof(double));
  if (!m->eL || !m->eR || !m->nx || !m->ny || !m->len || !m->cL || !m->cR || !m->qin || !m->qout) {
    free(v); free(tg); free(hs); orc_destroy(m); return ORC_ENOMEM;
  }
  int64_t e = 0;
  m->inflow_len = 0;
  for (int64_t i = 0; i < 3 * N; ++e) {
    int64_t j = i + 1;
    while (j < 3 * N && hs[j].a == hs[i].a && hs[j].b == hs[i].b) ++j;
    /* the lower cell index is the left cell; the normal is computed from the left
     * cell's counter-clockwise traversal of the edge: outward = (dy, -dx) / l */
    int64_t tl = hs[i].t; int kl = hs[i].k;
    int64_t p0 = v[3 * tl + kl], p1 = v[3 * tl + (kl + 1) % 3];
    double dx = xy[2 * p1] - xy[2 * p0], dy = xy[2 * p1 + 1] - xy[2 * p0 + 1];
    double l = sqrt(dx * dx + dy * dy);
    m->eL[e] = tl;
    m->nx[e] = dy / l;
    m->ny[e] = -dx / l;
    m->len[e] = l;
    m->cedge[3 * tl + kl] = e;
    if (j - i == 2) {
      int64_t tr = hs[i + 1].t; int kr = hs[i + 1].k;
      int64_t q0 = v[3 * tr + kr], q1 = v[3 * tr + (kr + 1) % 3];
      if (!(q0 == p1 && q1 == p0)) { rc = ORC_EINVAL; } /* both traverse the edge the same way */
      m->eR[e] = tr;
      m->cedge[3 * tr + kr] = e;
    } else {
      uint8_t tag = tg[3 * tl + kl];
      if (tag > 5) rc = ORC_EINVAL;
      m->eR[e] = -1 - (int64_t)tag;
      if (tag == 2) m->inflow_len += l;
    }
    i = j;
  }
  free(v); free(tg); free(hs);
  if (rc != ORC_OK) { orc_destroy(m); return rc; }
  if (p->hydro_n > 0) {
    m->ht = (double*)malloc(p->hydro_n * sizeof(double));
    m->hq = (double*)malloc(p->hydro_n * sizeof(double));
    if (!m->ht || !m->hq) { orc_destroy(m); return ORC_ENOMEM; }
    memcpy(m->ht, p->hydro_t, p->hydro_n * sizeof(double));
    memcpy(m->hq, p->hydro_q, p->hydro_n * sizeof(double));
    m->p.hydro_t = m->ht; m->p.hydro_q = m->hq;
  }
  *out = m;
  return ORC_OK;
}

/* ---------- point-wise pieces (exported for the pins) ---------- */

/* Q(t): piecewise linear through (hydro_t, hydro_q), constant beyond the ends; 0 if empty */
double orc_hydrograph(const orc_params* p, double t) {
  if (p->hydro_n <= 0) return 0.0;
  if (t <= p->hydro_t[0]) return p->hydro_q[0];
  for (int64_t i = 1; i < p->hydro_n; ++i) {
    if (t <= p->hydro_t[i]) {
      double w = (t - p->hydro_t[i - 1]) / (p->hydro_t[i] - p->hydro_t[i - 1]);
      return p->hydro_q[i - 1] + w * (p->hydro_q[i] - p->hydro_q[i - 1]);
    }
  }
  return p->hydro_q[p->hydro_n - 1];
}

/*
 * HLLC flux of the 1D shallow-water Riemann problem in the edge frame (normal
 * velocity un, tangential velocity ut passively carried by the contact wave),
 * Toro 2001 ch. 10 as named in the "Hydrodynamics" numerics subsection.
 * Wave speeds: two-rarefaction estimates for wet/wet, dry-front speeds if one
 * side has zero depth.  Writes (F_h, F_n, F_t).
 */
/* Wave-speed bounds (S_L, S_R) of the HLL family: star values from the
 * two-rarefaction approximation for a wet/wet problem, exact dry-front speeds if
 * one side is dry.  They must bracket the exact Riemann waves. */
void orc_wave_speeds(double hL, double uL, double hR, double uR, double g, double* SL, double* SR) {
  double cL = sqrt(g * hL), cR = sqrt(g * hR);
  if (hL <= 0) {
    *SL = uR - 2 * cR; *SR = uR + cR;
  } else if (hR <= 0) {
    *SL = uL - cL; *SR = uL + 2 * cL;
  } else {
    double us = 0.5 * (uL + uR) + cL - cR;
    double cs = 0.5 * (cL + cR) + 0.25 * (uL - uR);
    *SL = fmin(uL - cL, us - cs);
    *SR = fmax(uR + cR, us + cs);
  }
}

void orc_hllc(double hL, double uL, double vL, double hR, double uR, double vR, double g,
              double* F) {
  if (hL <= 0 && hR <= 0) { F[0] = 0; F[1] = 0; F[2] = 0; return; }
  double SL, SR;
  orc_wave_speeds(hL, uL, hR, uR, g, &SL, &SR);
  /* physical fluxes of the left and right state; the pressure 1/2 g h^2 is the
   * same expression as the correction the caller subtracts */
  double pL = 0.5 * g * hL * hL, pR = 0.5 * g * hR * hR;
  double FL0 = hL * uL, FL1 = hL * uL * uL + pL, FL2 = hL * uL * vL;
  double FR0 = hR * uR, FR1 = hR * uR * uR + pR, FR2 = hR * uR * vR;
  if (SL >= 0) { F[0] = FL0; F[1] = FL1; F[2] = FL2; return; }
  if (SR <= 0) { F[0] = FR0; F[1] = FR1; F[2] = FR2; return; }
  /* HLL state-flux: F_L - S_L (F_R - F_L - S_R (U_R - U_L)) / (S_R - S_L) */
  double d = SR - SL;
  double H0 = FL0 - SL * ((FR0 - FL0) - SR * (hR - hL)) / d;
  double H1 = FL1 - SL * ((FR1 - FL1) - SR * (hR * uR - hL * uL)) / d;
  /* contact speed decides which tangential velocity is advected */
  double Ss = (SL * hR * (uR - SR) - SR * hL * (uL - SL)) / (hR * (uR - SR) - hL * (uL - SL));
  F[0] = H0;
  F[1] = H1;
  F[2] = H0 * (Ss >= 0 ? vL : vR);
}

/*
 * Friction split step (Eq. 2 with Manning c_f, Table 1): dq/dt = -k(q) q with
 * k(q) = g n^2 |q| / h^(7/3), h frozen.  Two semi-implicit (linearly implicit)
 * Euler stages combined as Heun's RK2: q1 = q0/(1+dt k(q0)), q2 = q1/(1+dt k(q1)),
 * q = (q0 + q2)/2.  Skipped when h <= h_min or n = 0.
 */
/* the two semi-implicit stages and their Heun average for dq/dt = -c |q| q */
static void friction_stages(double c, double dt, double* qx, double* qy) {
  double q0x = *qx, q0y = *qy;
  double k0 = c * sqrt(q0x * q0x + q0y * q0y);
  double q1x = q0x / (1 + dt * k0), q1y = q0y / (1 + dt * k0);
  double k1 = c * sqrt(q1x * q1x + q1y * q1y);
  double q2x = q1x / (1 + dt * k1), q2y = q1y / (1 + dt * k1);
  *qx = 0.5 * (q0x + q2x);
  *qy = 0.5 * (q0y + q2y);
}

void orc_friction(double h, double n, double g, double dt, double h_min, double* qx, double* qy) {
  if (!(h > h_min) || n == 0) return;
  double c = g * n * n / pow(h, 7.0 / 3.0);
  friction_stages(c, dt, qx, qy);
}

/*
 * The friction closures of Table 1 as the dimensionless coefficient c_f of Eq. 2
 * (S_f = u |u| / (g h c_f^2)): Chezy c_f = 6.25 + ln(h / K_s) for h > K_s, else 6.25;
 * Bezzola c_f = 2.5 sqrt(1 - y_R / h) ln(10.9 h / y_R) for h / y_R > 2,
 * 1.25 sqrt(h / y_R) ln(10.9 h / y_R) for 0.5 <= h / y_R <= 2, 1.5 below.  (Manning,
 * c_f = h^(1/6) / (n sqrt(g)), and Strickler, the same with n = 1 / k_str, go through
 * orc_friction's own form.)
 */
double orc_cf(int law, double h, double r) {
  if (law == 1) return h > r ? 6.25 + log(h / r) : 6.25;
  const double x = h / r;
  if (x > 2.0) return 2.5 * sqrt(1.0 - r / h) * log(10.9 * h / r);
  if (x >= 0.5) return 1.25 * sqrt(x) * log(10.9 * h / r);
  return 1.5;
}

/* the friction split step of orc_friction with a Table 1 closure other than Manning:
 * k(q) = |q| / (h^2 c_f^2), the same two semi-implicit stages */
void orc_friction_cf(double h, double cf, double dt, double h_min, double* qx, double* qy) {
  if (!(h > h_min)) return;
  double c = 1.0 / (h * h * cf * cf);
  friction_stages(c, dt, qx, qy);
}

/* select the friction closure; coef (n_cells, caller order) replaces the per-cell
 * coefficient: n (Manning), K_s (Chezy) or y_R (Bezzola), all > 0 or 0 for none */
int orc_set_friction(orc_mesh* m, int law, const double* coef) {
  if (law < 0 || law > 2) return ORC_EINVAL;
  for (int64_t i = 0; i < m->n_cells; ++i)
    if (!(coef[i] >= 0)) return ORC_EINVAL;
  memcpy(m->man, coef, sizeof(double) * (size_t)m->n_cells);
  m->fr_law = law;
  return ORC_OK;
}

/* cell velocity of the unmodified state: q/h where h > h_min, else 0 */
static void cell_velocity(const orc_mesh* m, const double* H, const double* qx, const double* qy,
                          int64_t i, double* u, double* w) {
  double h = H[i] - m->z[i];
  if (h > m->p.h_min) { *u = qx[i] / h; *w = qy[i] / h; }
  else { *u = 0; *w = 0; }
}

/* conveyance weight of an inflow edge of length l whose cell holds depth h: l h^(5/3)
 * (Manning's uniform-flow discharge per unit width grows as h^(5/3)), 0 when dry */
static double inflow_weight(double l, double h, double h_min) {
  return h > h_min ? l * pow(h, 5.0 / 3.0) : 0.0;
}

/* inflow: unit discharge per inflow edge at time t, conveyance-weighted */
static double level_at(const orc_mesh* m, double t);
static void inflow_discharge(orc_mesh* m, const double* H, double t) {
  if (m->zh_n > 0) m->zh_now = level_at(m, t);  /* the water level at t as well */
  double Q = orc_hydrograph(&m->p, t);
  double W = 0;
  for (int64_t e = 0; e < m->n_edges; ++e) {
    if (m->eR[e] != -3) continue;
    double h = H[m->eL[e]] - m->z[m->eL[e]];
    W += inflow_weight(m->len[e], h, m->p.h_min);
  }
  for (int64_t e = 0; e < m->n_edges; ++e) {
    if (m->eR[e] != -3) { m->qin[e] = 0; continue; }
    double h = H[m->eL[e]] - m->z[m->eL[e]];
    if (W > 0) {
      double w = inflow_weight(m->len[e], h, m->p.h_min);
      m->qin[e] = Q * w / (m->len[e] * W);
    } else {
      m->qin[e] = m->inflow_len > 0 ? Q / m->inflow_len : 0.0;
    }
  }
}

/* depth at an inflow edge: the cell depth or the critical depth of q_e, the larger */
static double inflow_depth(double hc, double q, double g) {
  double hcr = cbrt(q * q / g);
  return hc > hcr ? hc : hcr;
}

/*
 * Outflow laws (Section "Boundary conditions", standard outflows; the appendix's
 * parameter list: the h-Q relation's table, the weir's height and Poleni factor).
 *
 * h-Q relation: the discharge Q leaving through the whole h-Q boundary is the rating
 * curve at its stage S, the length-weighted mean free surface over its edges whose
 * cell is wet; Q is split over those edges like the inflow, by conveyance l h^(5/3).
 * Rating curve: piecewise linear through (hq_s[k], hq_q[k]), constant beyond the ends.
 *
 * Weir: Poleni's law per unit crest width, q = (2/3) mu sqrt(2 g) eta^(3/2), with eta
 * the head of the cell's free surface over the crest; a crest below the cell's bed is
 * taken at the bed (free overfall), so eta never exceeds the depth.
 *
 * Either way the edge's flux is the physical flux of a boundary state that lets q leave
 * (outflow_state): the depth h_b on the outgoing characteristic of the cell (Riemann
 * invariant u_n + 2 sqrt(g h) of the cell, subcritical branch) that carries q at u_b =
 * q / h_b, and the cell's tangential velocity: (q, q u_b + g h_b^2 / 2, q u_t), less
 * the cell's own pressure g h^2 / 2 (pre-balanced form).  Water at rest sees a lower
 * boundary depth and accelerates towards the outlet; water arriving faster than the law
 * lets it out sees a higher one and is partly reflected.  An edge that lets nothing out
 * (head at or below the crest, dry cell) is a wall.
 */
static double rating(const orc_mesh* m, double S) {
  if (m->hq_n <= 0) return 0.0;
  if (S <= m->hq_s[0]) return m->hq_q[0];
  for (int64_t k = 1; k < m->hq_n; ++k) {
    if (S <= m->hq_s[k]) {
      double w = (S - m->hq_s[k - 1]) / (m->hq_s[k] - m->hq_s[k - 1]);
      return m->hq_q[k - 1] + w * (m->hq_q[k] - m->hq_q[k - 1]);
    }
  }
  return m->hq_q[m->hq_n - 1];
}

/* The boundary depth h_b of an outflow edge whose cell holds depth h and outward normal
 * velocity un, for a unit discharge *q > 0 leaving: q / h_b + 2 sqrt(g h_b) = w with
 * w = un + 2 sqrt(g h), on the subcritical branch (u_b <= sqrt(g h_b)).  *q is first
 * capped at the critical discharge w^3 / (27 g), the largest the invariant admits (then
 * h_b is the critical depth, (w / 3)^2 / g).  Returns h_b, or -1 if nothing can leave
 * (w <= 0: then *q = 0).  Newton's method on s = sqrt(h_b), from the right of the root
 * or stepping past it to the right (f(s) = 2 sqrt(g) s + q / s^2 - w is convex). */
static double outflow_state(double h, double un, double g, double* q) {
  const double w = un + 2.0 * sqrt(g * h), sg = sqrt(g);
  if (!(w > 0)) { *q = 0; return -1.0; }
  const double qmax = w * w * w / (27.0 * g);
  if (*q >= qmax) { *q = qmax; return (w / 3.0) * (w / 3.0) / g; }
  const double sm = cbrt(*q / sg); /* f's minimum */
  double s = sqrt(h) > sm ? sqrt(h) : sm;
  for (int it = 0; it < 100; ++it) {
    double f = 2.0 * sg * s + *q / (s * s) - w;
    double df = 2.0 * sg - 2.0 * *q / (s * s * s);
    if (!(df > 0)) break;
    double ds = f / df;
    s -= ds;
    if (fabs(ds) <= 1e-16 * s) break;
  }
  return s * s;
}

static double poleni(double mu, double g, double eta) {
  return (2.0 / 3.0) * mu * sqrt(2.0 * g) * eta * sqrt(eta);
}

static void outflow_discharge(orc_mesh* m, const double* H) {
  const double hmin = m->p.h_min;
  double sl = 0, sH = 0, W = 0;
  for (int64_t e = 0; e < m->n_edges; ++e) {
    if (m->eR[e] != -4) continue;
    int64_t i = m->eL[e];
    double h = H[i] - m->z[i];
    if (!(h > hmin)) continue;
    sl += m->len[e];
    sH += m->len[e] * H[i];
    W += inflow_weight(m->len[e], h, hmin);
  }
  double Q = sl > 0 ? rating(m, sH / sl) : 0.0;
  for (int64_t e = 0; e < m->n_edges; ++e) {
    m->qout[e] = 0;
    int64_t i = m->eL[e];
    double h = H[i] - m->z[i];
    if (!(h > hmin)) continue;
    if (m->eR[e] == -4 && W > 0) {
      m->qout[e] = Q * inflow_weight(m->len[e], h, hmin) / (m->len[e] * W);
    } else if (m->eR[e] == -5) {
      double crest = m->weir_crest > m->z[i] ? m->weir_crest : m->z[i];
      double eta = H[i] - crest;
      if (eta > 0) m->qout[e] = poleni(m->weir_mu, m->p.g, eta);
    }
  }
}

/*
 * The outflow laws of a mesh with h-Q (tag 3) or weir (tag 4) edges: n_hq >= 2
 * (stage, discharge) pairs, stage strictly increasing, discharge >= 0 (n_hq = 0: the
 * h-Q edges let nothing out); the weir's crest elevation and Poleni coefficient
 * mu >= 0.  Returns ORC_EINVAL on a malformed table.
 */
int orc_set_outflow(orc_mesh* m, int64_t n_hq, const double* stage, const double* q, double crest, double mu) {
  if (n_hq < 0 || n_hq == 1 || !(mu >= 0) || !isfinite(crest)) return ORC_EINVAL;
  for (int64_t k = 0; k < n_hq; ++k) {
    if (!isfinite(stage[k]) || !(q[k] >= 0) || !isfinite(q[k])) return ORC_EINVAL;
    if (k > 0 && !(stage[k] > stage[k - 1])) return ORC_EINVAL;
  }
  free(m->hq_s); free(m->hq_q);
  m->hq_s = m->hq_q = NULL;
  m->hq_n = 0;
  if (n_hq > 0) {
    m->hq_s = (double*)malloc(n_hq * sizeof(double));
    m->hq_q = (double*)malloc(n_hq * sizeof(double));
    if (!m->hq_s || !m->hq_q) return ORC_ENOMEM;
    memcpy(m->hq_s, stage, n_hq * sizeof(double));
    memcpy(m->hq_q, q, n_hq * sizeof(double));
  }
  m->hq_n = n_hq;
  m->weir_crest = crest;
  m->weir_mu = mu;
  return ORC_OK;
}

/* unit discharge through every edge at the state H and time t (>0 entering on inflow
 * edges, >0 leaving on outflow edges, 0 elsewhere) -- exported for the pins */
void orc_boundary_discharge(orc_mesh* m, const double* H, double t, double* q_in, double* q_out) {
  inflow_discharge(m, H, t);
  outflow_discharge(m, H);
  memcpy(q_in, m->qin, m->n_edges * sizeof(double));
  memcpy(q_out, m->qout, m->n_edges * sizeof(double));
}

/*
 * Water-level boundary (Section "Boundary conditions": zhydrograph, "water surface
 * elevation" as input, among the standard inflows and outflows).  The paper gives no
 * formula.  Reading: the edge's flux is the HLLC flux between the inside cell and a
 * boundary state: depth h_b = max(0, Z_b(t^n) - z_i), the imposed surface over the
 * inside cell's bed; normal velocity on the cell's outgoing characteristic, the
 * Riemann invariant u_n + 2 sqrt(g h) carried from the cell, u_b = u_n + 2 sqrt(g h) -
 * 2 sqrt(g h_b) (for h_b < h exactly the state the 1-rarefaction reaches from the
 * cell); the cell's tangential velocity.  A dry inside cell carries no invariant: the
 * boundary water is at rest there (u_b = 0), so the level floods the cell as a dam
 * break.  Still water at the imposed level gives the cell's own state (no flux beyond
 * its pressure).  Eq. 21 takes the boundary state's |u_b| + sqrt(g h_b) on the edge.
 */
static double level_at(const orc_mesh* m, double t) {
  if (t <= m->zh_t[0]) return m->zh_v[0];
  for (int64_t k = 1; k < m->zh_n; ++k)
    if (t <= m->zh_t[k]) {
      double w = (t - m->zh_t[k - 1]) / (m->zh_t[k] - m->zh_t[k - 1]);
      return m->zh_v[k - 1] + w * (m->zh_v[k] - m->zh_v[k - 1]);
    }
  return m->zh_v[m->zh_n - 1];
}

/* the boundary state's depth and normal velocity of a level edge of cell i (depth h,
 * outward normal velocity un) */
static void level_state(const orc_mesh* m, int64_t i, double h, double un, double* hb, double* ub) {
  const double g = m->p.g;
  *hb = fmax(0.0, m->zh_now - m->z[i]);
  *ub = h > m->p.h_min ? un + 2.0 * sqrt(g * h) - 2.0 * sqrt(g * *hb) : 0.0;
}

/* The water-level series of the level edges (tag 5): n >= 1 points (t strictly
 * increasing, levels finite); n = 0 turns the edges back into walls.  ORC_EINVAL on
 * malformed input. */
int orc_set_level(orc_mesh* m, int64_t n, const double* t, const double* v) {
  if (n < 0) return ORC_EINVAL;
  for (int64_t k = 0; k < n; ++k) {
    if (!isfinite(t[k]) || !isfinite(v[k])) return ORC_EINVAL;
    if (k > 0 && !(t[k] > t[k - 1])) return ORC_EINVAL;
  }
  free(m->zh_t); free(m->zh_v);
  m->zh_t = m->zh_v = NULL;
  m->zh_n = 0;
  if (n > 0) {
    m->zh_t = (double*)malloc(n * sizeof(double));
    m->zh_v = (double*)malloc(n * sizeof(double));
    if (!m->zh_t || !m->zh_v) return ORC_ENOMEM;
    memcpy(m->zh_t, t, n * sizeof(double));
    memcpy(m->zh_v, v, n * sizeof(double));
  }
  m->zh_n = n;
  return ORC_OK;
}

/* Eq. 21: dt = CFL * min_i min_j rho_ij / lambda_ij on wet cells (or, cfl_mode 1,
 * CFL * min_i |Omega_i| / sum_j l_ij lambda_ij); inflow and outflow edges add their
 * own boundary wave speed.  Returns +inf if nothing constrains dt.  Requires qin and
 * qout. */
double orc_cfl(const orc_mesh* m, const double* H, const double* qx, const double* qy) {
  const double g = m->p.g;
  double best = INFINITY;
  for (int64_t i = 0; i < m->n_cells; ++i) {
    double h = H[i] - m->z[i];
    int wet = h > m->p.h_min;
    double u = 0, w = 0, c = 0;
    if (wet) { u = qx[i] / h; w = qy[i] / h; c = sqrt(g * h); }
    double sum = 0;
    for (int k = 0; k < 3; ++k) {
      int64_t e = m->cedge[3 * i + k];
      double sgn = (m->eL[e] == i) ? 1.0 : -1.0;
      double nx = sgn * m->nx[e], ny = sgn * m->ny[e];
      double lam = wet ? fabs(u * nx + w * ny) + c : 0.0;
      if (m->eR[e] == -3 && m->qin[e] > 0) {
        double hb = inflow_depth(h > 0 ? h : 0.0, m->qin[e], g);
        double lb = m->qin[e] / hb + sqrt(g * hb);
        if (m->p.cfl_mode == 0) {
          double rho = 4.0 * m->area[i] / (3.0 * m->len[e]);
          if (rho / lb < best) best = rho / lb;
        } else {
          double r = m->area[i] / (m->len[e] * lb);
          if (r < best) best = r;
        }
      }
      if (m->eR[e] == -6 && m->zh_n > 0) {
        /* water-level edge: the boundary state's |u_b| + sqrt(g h_b) */
        double hb, ub;
        level_state(m, i, h > 0 ? h : 0.0, u * nx + w * ny, &hb, &ub);
        double lb = fabs(ub) + sqrt(g * hb);
        if (lb > 0) {
          if (m->p.cfl_mode == 0) {
            double rho = 4.0 * m->area[i] / (3.0 * m->len[e]);
            if (rho / lb < best) best = rho / lb;
          } else {
            double r = m->area[i] / (m->len[e] * lb);
            if (r < best) best = r;
          }
        }
      }
      if ((m->eR[e] == -4 || m->eR[e] == -5) && m->qout[e] > 0) {
        /* outflow edge: the boundary state's u_b + sqrt(g h_b) */
        double q = m->qout[e];
        double hb = outflow_state(h, u * nx + w * ny, g, &q);
        double lb = hb > 0 ? q / hb + sqrt(g * hb) : 0.0;
        if (m->p.cfl_mode == 0) {
          double rho = 4.0 * m->area[i] / (3.0 * m->len[e]);
          if (rho / lb < best) best = rho / lb;
        } else {
          double r = m->area[i] / (m->len[e] * lb);
          if (r < best) best = r;
        }
      }
      if (lam > 0) {
        double rho = 4.0 * m->area[i] / (3.0 * m->len[e]);
        if (m->p.cfl_mode == 0 && rho / lam < best) best = rho / lam;
      }
      sum += m->len[e] * lam;
    }
    if (m->p.cfl_mode == 1 && sum > 0) {
      double r = m->area[i] / sum;
      if (r < best) best = r;
    }
  }
  return best;
}

/*
 * External sources and sinks (Section "External inflow/outflow discharge"): S_h [m/s]
 * over regions of cells, added explicitly to the continuity equation (the S term of
 * Eq. 12, evaluated at t^n).  Region r has a series v_r(t), piecewise linear through
 * its points and constant beyond the ends; kind 0: a total discharge [m^3/s] spread
 * over the region's area A_r, S_h = v / A_r; kind 1: an intensity [mm/h] per square
 * metre, S_h = v / 3.6e6.  v > 0 adds water, v < 0 takes it.  mode 0 (Exact): the
 * depth changes by dt S_h as prescribed (it may fall below zero: the run then fails);
 * mode 1 (Available): a sink takes at most the water the cell holds after the
 * fluxes (the depth stops at 0); mode 2 (Infinity): the region takes all water its
 * cells hold (depth 0, whatever v).  Sources add mass only, no momentum.
 * n_regions = 0 removes them.  Returns ORC_EINVAL on malformed input.
 */
int orc_set_sources(orc_mesh* m, int32_t n_regions, const int32_t* reg, const int32_t* kind, const int32_t* mode,
                    const int64_t* off, const double* t, const double* v) {
  free(m->src_reg); free(m->src_kind); free(m->src_mode); free(m->src_off);
  free(m->src_t); free(m->src_v); free(m->src_area); free(m->src_rate);
  m->src_reg = NULL; m->src_kind = NULL; m->src_mode = NULL; m->src_off = NULL;
  m->src_t = NULL; m->src_v = NULL; m->src_area = NULL; m->src_rate = NULL;
  m->src_n = 0;
  m->src_vol = 0.0;
  if (n_regions <= 0) return ORC_OK;
  const int64_t n = m->n_cells, np = off[n_regions];
  m->src_reg = (int32_t*)malloc(sizeof(int32_t) * (size_t)n);
  m->src_kind = (int32_t*)malloc(sizeof(int32_t) * (size_t)n_regions);
  m->src_mode = (int32_t*)malloc(sizeof(int32_t) * (size_t)n_regions);
  m->src_off = (int64_t*)malloc(sizeof(int64_t) * (size_t)(n_regions + 1));
  m->src_t = (double*)malloc(sizeof(double) * (size_t)(np + 1));
  m->src_v = (double*)malloc(sizeof(double) * (size_t)(np + 1));
  m->src_area = (double*)calloc((size_t)n_regions, sizeof(double));
  m->src_rate = (double*)calloc((size_t)n_regions, sizeof(double));
  if (!m->src_reg || !m->src_kind || !m->src_mode || !m->src_off || !m->src_t || !m->src_v || !m->src_area ||
      !m->src_rate)
    return ORC_ENOMEM;
  memcpy(m->src_reg, reg, sizeof(int32_t) * (size_t)n);
  memcpy(m->src_kind, kind, sizeof(int32_t) * (size_t)n_regions);
  memcpy(m->src_mode, mode, sizeof(int32_t) * (size_t)n_regions);
  memcpy(m->src_off, off, sizeof(int64_t) * (size_t)(n_regions + 1));
  memcpy(m->src_t, t, sizeof(double) * (size_t)np);
  memcpy(m->src_v, v, sizeof(double) * (size_t)np);
  for (int64_t i = 0; i < n; ++i)
    if (reg[i] >= 0) m->src_area[reg[i]] += m->area[i];
  m->src_n = n_regions;
  return ORC_OK;
}

/*
 * Morphodynamics (Section "Morphodynamics", Eq. 3 with S_b = 0, solved with the update
 * of Eq. 13 and the HLL sediment flux of Eq. 14-16, synchronous-decoupled: the same dt,
 * every term from U^n and z^n).  Bedload magnitude from the MPM-like closure (Table 2):
 *   |q_B| = alpha (theta - theta_cr)^m sqrt((s - 1) g d^3)  (0 for theta <= theta_cr),
 *   theta = tau_b / ((rho_s - rho) g d) = n^2 |u|^2 / ((s - 1) d h^(1/3))
 * (Manning's bed shear stress rho g n^2 |u|^2 / h^(1/3)), directed along the flow
 * (no slope or curvature corrections).  dq_B,n/dq_n of Eq. 16 is taken along the
 * flow at fixed depth: d|q_B|/d|u| / h = alpha m (theta - theta_cr)^(m-1)
 * sqrt((s - 1) g d^3) (2 theta / |u|) / h.  u_n and c = sqrt(g h) of each cell on the
 * edge; walls carry no sediment, other boundary edges the inside cell's normal bedload.
 * The bed change moves the free surface with it (H += dz): the water depth, hence the
 * water volume, is kept.  on = 0 turns it off.
 */
int orc_set_morpho(orc_mesh* m, int on, double porosity, double s, double d, double alpha, double mexp,
                   double theta_cr) {
  m->morpho = 0;
  if (!on) return ORC_OK;
  if (!(porosity >= 0 && porosity < 1) || !(s > 1) || !(d > 0) || !(alpha >= 0) || !(mexp >= 1)) return ORC_EINVAL;
  if (!m->qbx) {
    m->qbx = (double*)calloc((size_t)m->n_cells, sizeof(double));
    m->qby = (double*)calloc((size_t)m->n_cells, sizeof(double));
    m->qbd = (double*)calloc((size_t)m->n_cells, sizeof(double));
    m->fb = (double*)calloc((size_t)m->n_edges, sizeof(double));
    if (!m->qbx || !m->qby || !m->qbd || !m->fb) return ORC_ENOMEM;
  }
  m->mp_p = porosity; m->mp_s = s; m->mp_d = d; m->mp_alpha = alpha; m->mp_m = mexp; m->mp_thcr = theta_cr;
  m->morpho = 1;
  return ORC_OK;
}

/* bedload vector and dq_B/dq of every cell from U^n, z^n */
static void morpho_cells(orc_mesh* m, const double* H, const double* qx, const double* qy) {
  const double g = m->p.g, sd = m->mp_s - 1.0, d = m->mp_d;
  const double scale = sqrt(sd * g * d * d * d);
  for (int64_t i = 0; i < m->n_cells; ++i) {
    double u, v;
    cell_velocity(m, H, qx, qy, i, &u, &v);
    const double h = H[i] - m->z[i];
    const double sp = sqrt(u * u + v * v);
    m->qbx[i] = 0; m->qby[i] = 0; m->qbd[i] = 0;
    if (!(h > m->p.h_min) || sp == 0) continue;
    const double theta = m->man[i] * m->man[i] * sp * sp / (sd * d * cbrt(h));
    if (!(theta > m->mp_thcr)) continue;
    const double qb = m->mp_alpha * pow(theta - m->mp_thcr, m->mp_m) * scale;
    m->qbx[i] = qb * u / sp;
    m->qby[i] = qb * v / sp;
    m->qbd[i] = m->mp_alpha * m->mp_m * pow(theta - m->mp_thcr, m->mp_m - 1.0) * scale * (2.0 * theta / sp) / h;
  }
}

/* the two speeds of Eq. 16 for one cell on an edge */
static void morpho_speeds(double un, double c, double dqb, double* l1, double* l2) {
  const double a = un - c;
  const double r = sqrt(a * a + 4.0 * dqb * c * c);
  *l1 = 0.5 * (a - r);
  *l2 = 0.5 * (a + r);
}

/* the speeds of Eq. 16 of cell i on an edge of unit normal (nx, ny): u_n = u.n and
 * c = sqrt(g h) of the cell's own (unmodified) state, dq_B,n/dq_n from morpho_cells */
static void cell_edge_speeds(const orc_mesh* m, const double* H, const double* qx, const double* qy, int64_t i,
                             double nx, double ny, double* l1, double* l2) {
  double u, v;
  cell_velocity(m, H, qx, qy, i, &u, &v);
  const double c = sqrt(m->p.g * fmax(0.0, H[i] - m->z[i]));
  morpho_speeds(u * nx + v * ny, c, m->qbd[i], l1, l2);
}

/* l q_Bij of every edge (Eq. 14, 15), outward from the left cell */
static void morpho_edges(orc_mesh* m, const double* H, const double* qx, const double* qy) {
  for (int64_t e = 0; e < m->n_edges; ++e) {
    const int64_t L = m->eL[e], R = m->eR[e];
    const double nx = m->nx[e], ny = m->ny[e];
    const double qL = m->qbx[L] * nx + m->qby[L] * ny;
    double f;
    if (R >= 0) {
      double a1, a2, b1, b2;
      cell_edge_speeds(m, H, qx, qy, L, nx, ny, &a1, &a2);
      cell_edge_speeds(m, H, qx, qy, R, nx, ny, &b1, &b2);
      const double lm = fmin(a1, b1), lp = fmax(a2, b2);
      const double qR = m->qbx[R] * nx + m->qby[R] * ny;
      f = lp - lm > 0 ? (lp * qL - lm * qR + lp * lm * (m->z[R] - m->z[L])) / (lp - lm) : 0.0;
    } else {
      f = R == -1 ? 0.0 : qL; /* wall; transmissive / inflow / outflow: the inside cell's bedload */
    }
    m->fb[e] = m->len[e] * f;
  }
}

/* S_h of every region at time t (m/s) */
static void source_rates(orc_mesh* m, double t) {
  for (int32_t r = 0; r < m->src_n; ++r) {
    const int64_t a = m->src_off[r], b = m->src_off[r + 1];
    double v = m->src_v[a];
    if (t > m->src_t[a]) {
      v = m->src_v[b - 1];
      for (int64_t k = a + 1; k < b; ++k)
        if (t <= m->src_t[k]) {
          double w = (t - m->src_t[k - 1]) / (m->src_t[k] - m->src_t[k - 1]);
          v = m->src_v[k - 1] + w * (m->src_v[k] - m->src_v[k - 1]);
          break;
        }
    }
    m->src_rate[r] = m->src_kind[r] == 0 ? v / m->src_area[r] : v / 3.6e6;
  }
}

/*
 * One explicit step from (t, H, qx, qy) to t + dt, in place.  t_end clips dt
 * (pass +inf for none).  bvol accumulates the net volume that entered through
 * the boundary (positive = inflow).  Returns dt (0 if t >= t_end).
 */
double orc_step(orc_mesh* m, double* H, double* qx, double* qy, double* t, double t_end,
                double* bvol) {
  const double g = m->p.g, hmin = m->p.h_min;
  if (!(*t < t_end)) return 0.0;
  /* 0. time step from U^n (Eq. 21) */
  inflow_discharge(m, H, *t);
  outflow_discharge(m, H);
  double mcfl = orc_cfl(m, H, qx, qy);
  double dt = isinf(mcfl) ? m->p.dt_max : m->p.cfl * mcfl;
  if (dt > m->p.dt_max) dt = m->p.dt_max;
  int clipped = 0;
  if (dt >= t_end - *t) { dt = t_end - *t; clipped = 1; }
  /* 1.-2. edge fluxes */
  double bflux = 0; /* sum over boundary edges of l * F_h (outward) */
  for (int64_t e = 0; e < m->n_edges; ++e) {
    int64_t L = m->eL[e], R = m->eR[e];
    double nx = m->nx[e], ny = m->ny[e], l = m->len[e];
    double uL, vL; cell_velocity(m, H, qx, qy, L, &uL, &vL);
    double unL = uL * nx + vL * ny, utL = -uL * ny + vL * nx;
    double F[3];
    if (R >= 0) {
      double zs = fmax(m->z[L], m->z[R]);
      double hLs = fmax(0.0, H[L] - zs), hRs = fmax(0.0, H[R] - zs);
      double uR, vR; cell_velocity(m, H, qx, qy, R, &uR, &vR);
      double unR = uR * nx + vR * ny, utR = -uR * ny + vR * nx;
      orc_hllc(hLs, unL, utL, hRs, unR, utR, g, F);
      double pL = 0.5 * g * hLs * hLs, pR = 0.5 * g * hRs * hRs;
      double GL = F[1] - pL, GR = F[1] - pR;
      m->cL[3 * e] = l * F[0];
      m->cL[3 * e + 1] = l * (GL * nx - F[2] * ny);
      m->cL[3 * e + 2] = l * (GL * ny + F[2] * nx);
      m->cR[3 * e] = -l * F[0];
      m->cR[3 * e + 1] = -l * (GR * nx - F[2] * ny);
      m->cR[3 * e + 2] = -l * (GR * ny + F[2] * nx);
    } else {
      double hs = fmax(0.0, H[L] - m->z[L]);
      double p = 0.5 * g * hs * hs;
      double Fh, Gn, Ft;
      /* an outflow edge (h-Q, weir) lets q_e leave through its boundary state */
      double qo = (R == -4 || R == -5) ? m->qout[e] : 0.0;
      double hbo = qo > 0 ? outflow_state(hs, unL, g, &qo) : -1.0;
      if (R == -1 || ((R == -4 || R == -5) && !(hbo > 0)) || (R == -6 && m->zh_n == 0)) {
        /* wall: mirrored normal velocity, impermeable (also an outflow edge that lets
         * nothing out) */
        orc_hllc(hs, unL, utL, hs, -unL, utL, g, F);
        Fh = 0; Gn = F[1] - p; Ft = 0;
      } else if (R == -6) { /* water level: HLLC with the boundary state */
        double hb, ub;
        level_state(m, L, hs, unL, &hb, &ub);
        orc_hllc(hs, unL, utL, hb, ub, utL, g, F);
        Fh = F[0]; Gn = F[1] - p; Ft = F[2];
      } else if (R == -2) { /* transmissive: the outside state equals the inside state */
        orc_hllc(hs, unL, utL, hs, unL, utL, g, F);
        Fh = F[0]; Gn = F[1] - p; Ft = F[2];
      } else if (R == -3) { /* inflow: imposed unit discharge q_e entering along -n */
        double q = m->qin[e];
        if (q > 0) {
          double hb = inflow_depth(hs, q, g);
          Fh = -q; Gn = q * q / hb + 0.5 * g * hb * hb - p; Ft = 0;
        } else { Fh = 0; Gn = 0; Ft = 0; }
      } else { /* outflow: q_e leaves along n at the boundary state's depth */
        Fh = qo; Gn = qo * (qo / hbo) + 0.5 * g * hbo * hbo - p; Ft = qo * utL;
      }
      m->cL[3 * e] = l * Fh;
      m->cL[3 * e + 1] = l * (Gn * nx - Ft * ny);
      m->cL[3 * e + 2] = l * (Gn * ny + Ft * nx);
      bflux += l * Fh;
    }
  }
  /* morphodynamics: bedload fluxes from U^n, z^n (before the state is overwritten) */
  if (m->morpho) {
    morpho_cells(m, H, qx, qy);
    morpho_edges(m, H, qx, qy);
  }
  /* 3.-5. cell update (Eq. 12 with the external source), friction, dry clean-up */
  if (m->src_n > 0) source_rates(m, *t);
  for (int64_t i = 0; i < m->n_cells; ++i) {
    double s0 = 0, s1 = 0, s2 = 0;
    for (int k = 0; k < 3; ++k) {
      int64_t e = m->cedge[3 * i + k];
      const double* c = (m->eL[e] == i) ? &m->cL[3 * e] : &m->cR[3 * e];
      s0 += c[0]; s1 += c[1]; s2 += c[2];
    }
    double r = dt / m->area[i];
    double Hn = H[i] - r * s0;
    double ux = qx[i] - r * s1;
    double uy = qy[i] - r * s2;
    if (m->src_n > 0 && m->src_reg[i] >= 0) {
      const int32_t rg = m->src_reg[i];
      const double Hf = Hn, add = dt * m->src_rate[rg];
      if (m->src_mode[rg] == 2 || (m->src_mode[rg] == 1 && (Hn - m->z[i]) + add < 0))
        Hn = m->z[i]; /* the sink empties the cell */
      else
        Hn = Hn + add;
      m->src_vol += m->area[i] * (Hn - Hf);
    }
    double h = Hn - m->z[i];
    if (m->fr_law == 0)
      orc_friction(h, m->man[i], g, dt, hmin, &ux, &uy);
    else if (m->man[i] > 0 && h > hmin)
      orc_friction_cf(h, orc_cf(m->fr_law, h, m->man[i]), dt, hmin, &ux, &uy);
    if (!(h > hmin)) { ux = 0; uy = 0; }
    H[i] = Hn; qx[i] = ux; qy[i] = uy;
  }
  if (m->morpho) {
    /* Eq. 13 (S_b = 0); the free surface moves with the bed */
    for (int64_t i = 0; i < m->n_cells; ++i) {
      double sum = 0;
      for (int k = 0; k < 3; ++k) {
        int64_t e = m->cedge[3 * i + k];
        sum += (m->eL[e] == i) ? m->fb[e] : -m->fb[e];
      }
      const double dz = -(dt / m->area[i] * sum) / (1.0 - m->mp_p);
      m->z[i] += dz;
      H[i] += dz;
    }
    for (int64_t e = 0; e < m->n_edges; ++e)
      if (m->eR[e] < 0) m->bed_bvol += dt * m->fb[e];
  }
  *bvol += -dt * bflux;
  *t = clipped ? t_end : *t + dt;
  return dt;
}

/* run up to n_steps steps, stopping early at t_end; returns the number taken */
int64_t orc_run(orc_mesh* m, double* H, double* qx, double* qy, double* t, double t_end,
                int64_t n_steps, double* bvol) {
  int64_t s = 0;
  for (; s < n_steps; ++s) {
    if (!(*t < t_end)) break;
    orc_step(m, H, qx, qy, t, t_end, bvol);
  }
  return s;
}

/*
 * Flood tracking (the hydrodynamic module's "Flood" outputs: water front arrival
 * time, maximum water depth, maximum flow velocity, maximum specific discharge and
 * maximum bed shear stress), updated from the state (H, qx, qy) at time t.  Per cell:
 *   h = H - z,  |q| = sqrt(qx^2 + qy^2),
 *   |u| = |q| / h and tau = rho g n^2 |u|^2 / h^(1/3) where h > h_min, else 0
 *   (Manning, Eq. 2 / Table 1: the bed shear stress rho g h S_f with
 *   S_f = n^2 |u|^2 / h^(4/3); under a logarithmic closure rho |u|^2 / c_f^2),
 *   arrival = the first t at which h > h_arr (NaN until then),
 *   the maxima of h, |u|, |q|, tau over the calls.
 * init != 0 starts the record from this state.
 */
void orc_track(const orc_mesh* m, const double* H, const double* qx, const double* qy, double t, double h_arr,
               double rho, int init, double* arr, double* hmax, double* umax, double* qmax, double* taumax) {
  const double g = m->p.g, hmin = m->p.h_min;
  for (int64_t i = 0; i < m->n_cells; ++i) {
    const double h = H[i] - m->z[i];
    const double q = sqrt(qx[i] * qx[i] + qy[i] * qy[i]);
    double u = 0, tau = 0;
    if (h > hmin) {
      u = q / h;
      if (m->fr_law == 0) {
        tau = rho * g * m->man[i] * m->man[i] * u * u / cbrt(h);
      } else { /* rho g h S_f = rho u^2 / c_f^2 (Eq. 2) with the law's c_f */
        double cf = orc_cf(m->fr_law, h, m->man[i]);
        tau = rho * u * u / (cf * cf);
      }
    }
    if (init) {
      arr[i] = h > h_arr ? t : NAN;
      hmax[i] = h; umax[i] = u; qmax[i] = q; taumax[i] = tau;
    } else {
      if (isnan(arr[i]) && h > h_arr) arr[i] = t;
      if (h > hmax[i]) hmax[i] = h;
      if (u > umax[i]) umax[i] = u;
      if (q > qmax[i]) qmax[i] = q;
      if (tau > taumax[i]) taumax[i] = tau;
    }
  }
}

/* orc_run with flood tracking after every step */
int64_t orc_run_tracked(orc_mesh* m, double* H, double* qx, double* qy, double* t, double t_end, int64_t n_steps,
                        double* bvol, double h_arr, double rho, double* arr, double* hmax, double* umax, double* qmax,
                        double* taumax) {
  int64_t s = 0;
  for (; s < n_steps; ++s) {
    if (!(*t < t_end)) break;
    orc_step(m, H, qx, qy, t, t_end, bvol);
    orc_track(m, H, qx, qy, *t, h_arr, rho, 0, arr, hmax, umax, qmax, taumax);
  }
  return s;
}

/*
 * Passive scalar advection (Section "Scalar advection-diffusion", Eq. 8 without the
 * diffusion and source terms): K species with unknowns q_c = h phi_c (hc: K x n,
 * species-major).  The advective flux of a species is HLLC's contact-wave flux, the
 * formula the tangential momentum uses with phi_c in place of the tangential velocity:
 * F_c = F_h phi_c of the upwind side of the contact (S* >= 0: left) -- the scheme the
 * "Scalar advection-diffusion" numerics subsection names for the advective part.
 * phi_c = q_c / h where h = H - z > 0, else 0.  Walls carry nothing; a transmissive
 * edge carries F_h phi_c of the inside cell; an inflow edge brings q_e l c_in[c]; an
 * outflow edge (h-Q, weir) takes its mass flux F_h (the discharge its boundary state
 * lets out) times phi_c of the inside cell.
 * A cell that ends the step dry (h <= 0) keeps no scalar.  One step of the water
 * (orc_step) and the species together; returns the number of steps taken.
 */
int64_t orc_run_scalars(orc_mesh* m, double* H, double* qx, double* qy, double* t, double t_end, int64_t n_steps,
                        double* bvol, int K, double* hc, const double* c_in) {
  const double g = m->p.g;
  const int64_t n = m->n_cells, ne = m->n_edges;
  double* phi = (double*)malloc(sizeof(double) * (size_t)(K * n + K * ne + 1));
  if (!phi) return -1;
  double* fl = phi + K * n; /* per edge and species: l * F_c (outward from the left cell) */
  int64_t s = 0;
  for (; s < n_steps; ++s) {
    if (!(*t < t_end)) break;
    for (int64_t i = 0; i < n; ++i) {
      double h = H[i] - m->z[i];
      for (int c = 0; c < K; ++c) phi[c * n + i] = h > 0 ? hc[c * n + i] / h : 0.0;
    }
    inflow_discharge(m, H, *t); /* q_e of this step (orc_step computes the same) */
    outflow_discharge(m, H);
    for (int64_t e = 0; e < ne; ++e) {
      int64_t L = m->eL[e], R = m->eR[e];
      double nx = m->nx[e], ny = m->ny[e], l = m->len[e];
      double uL, vL; cell_velocity(m, H, qx, qy, L, &uL, &vL);
      double unL = uL * nx + vL * ny;
      for (int c = 0; c < K; ++c) {
        double F[3], f;
        double pL = phi[c * n + L];
        if (R >= 0) {
          double zs = fmax(m->z[R], m->z[L]); /* the higher bed of the two */
          double hLs = fmax(0.0, H[L] - zs), hRs = fmax(0.0, H[R] - zs);
          double uR, vR; cell_velocity(m, H, qx, qy, R, &uR, &vR);
          double unR = uR * nx + vR * ny;
          orc_hllc(hLs, unL, pL, hRs, unR, phi[c * n + R], g, F);
          f = F[2];
        } else if (R == -1) {
          f = 0; /* wall */
        } else if (R == -2) {
          double hs = fmax(0.0, H[L] - m->z[L]);
          orc_hllc(hs, unL, pL, hs, unL, pL, g, F);
          f = F[2];
        } else if (R == -3) {
          double q = m->qin[e];
          f = q > 0 ? -q * c_in[c] : 0.0;
        } else if (R == -6) {
          /* water level: the step's HLLC with the boundary state, upwinded at the contact;
           * the water outside carries no species */
          double hs = fmax(0.0, H[L] - m->z[L]), hb, ub;
          if (m->zh_n > 0) {
            m->zh_now = level_at(m, *t);
            level_state(m, L, hs, unL, &hb, &ub);
            orc_hllc(hs, unL, pL, hb, ub, 0.0, g, F);
            f = F[2];
          } else {
            f = 0; /* a wall until its series is set */
          }
        } else { /* outflow: the inside cell's scalar leaves with the edge's mass flux */
          double q = m->qout[e];
          double hs = fmax(0.0, H[L] - m->z[L]);
          double hb = q > 0 ? outflow_state(hs, unL, g, &q) : -1.0;
          f = hb > 0 ? q * pL : 0.0;
        }
        fl[c * ne + e] = l * f;
      }
    }
    double dt = orc_step(m, H, qx, qy, t, t_end, bvol);
    for (int64_t i = 0; i < n; ++i) {
      double r = dt / m->area[i];
      for (int c = 0; c < K; ++c) {
        double sum = 0;
        for (int k = 0; k < 3; ++k) {
          int64_t e = m->cedge[3 * i + k];
          sum += (m->eL[e] == i) ? fl[c * ne + e] : -fl[c * ne + e];
        }
        double v = hc[c * n + i] - r * sum;
        hc[c * n + i] = (H[i] - m->z[i] > 0) ? v : 0.0;
      }
    }
  }
  free(phi);
  return s;
}

double orc_source_volume(const orc_mesh* m) { return m->src_vol; }
/* sediment volume (solid, per Eq. 3's flux) that left through the boundary */
double orc_bed_outflow(const orc_mesh* m) { return m->bed_bvol; }
void orc_bed(const orc_mesh* m, double* z) { memcpy(z, m->z, m->n_cells * sizeof(double)); }

/* V = sum_i |Omega_i| (H_i - z_i), fixed order */
double orc_volume(const orc_mesh* m, const double* H) {
  double v = 0;
  for (int64_t i = 0; i < m->n_cells; ++i) v += m->area[i] * (H[i] - m->z[i]);
  return v;
}

/* next dt that orc_step would take from this state (Eq. 21 with dt_max), no clipping */
double orc_next_dt(orc_mesh* m, const double* H, const double* qx, const double* qy, double t) {
  inflow_discharge(m, H, t);
  outflow_discharge(m, H);
  double mcfl = orc_cfl(m, H, qx, qy);
  double dt = isinf(mcfl) ? m->p.dt_max : m->p.cfl * mcfl;
  return dt > m->p.dt_max ? m->p.dt_max : dt;
}

/* accessors for tests */

/* Eq. 16's (lambda_1, lambda_2) of cell i for the unit normal (nx, ny) at the state
 * (H, qx, qy), as the bed flux of a step from that state uses them (bed evolution must
 * be on: orc_set_morpho).  Returns ORC_EINVAL when it is off or i is out of range. */
int orc_morpho_speeds(orc_mesh* m, const double* H, const double* qx, const double* qy, int64_t i, double nx,
                      double ny, double* l1, double* l2) {
  if (!m->morpho || i < 0 || i >= m->n_cells) return ORC_EINVAL;
  morpho_cells(m, H, qx, qy);
  cell_edge_speeds(m, H, qx, qy, i, nx, ny, l1, l2);
  return ORC_OK;
}
int64_t orc_n_edges(const orc_mesh* m) { return m->n_edges; }
void orc_cell_area(const orc_mesh* m, double* out) { memcpy(out, m->area, m->n_cells * sizeof(double)); }
void orc_edges(const orc_mesh* m, int64_t* L, int64_t* R, double* nx, double* ny, double* len) {
  memcpy(L, m->eL, m->n_edges * sizeof(int64_t));
  memcpy(R, m->eR, m->n_edges * sizeof(int64_t));
  memcpy(nx, m->nx, m->n_edges * sizeof(double));
  memcpy(ny, m->ny, m->n_edges * sizeof(double));
  memcpy(len, m->len, m->n_edges * sizeof(double));
}
