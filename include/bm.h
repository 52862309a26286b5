/*
 * bm.h -- C ABI of the B300-native explicit finite-volume shallow-water step.
 *
 * The method is the hydrodynamic module of BASEMENT v3 (arXiv 2102.12862):
 * unknowns U = (H, q_x, q_y) per triangle (Eq. 1, Eq. 10), the explicit update of
 * Eq. 12 with an HLLC edge flux and the modified-state bed treatment (Section
 * "Numerical solution", subsection "Hydrodynamics"), Manning friction (Eq. 2,
 * Table 1) integrated after splitting, and the time step of Eq. 21.
 *
 * Conventions for every entry point:
 *  - Returns a bm_status; BM_OK is 0.  On failure bm_last_error() returns a
 *    thread-local message.  No C++ exception crosses the ABI.
 *  - Handles are opaque.  Input arrays are host pointers owned by the caller; the
 *    library copies them before returning.  Output arrays are caller-allocated
 *    host buffers.  All per-cell arrays are in the caller's triangle order (the
 *    library renumbers cells internally along a Hilbert curve).
 *  - Device work is ordered on the state's CUDA stream (bm_state_set_stream).
 *  - Handles are not thread-safe; use one handle from one thread at a time.
 */
#ifndef BM_H
#define BM_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  BM_OK = 0,
  BM_EINVAL = 1,      /* invalid argument or malformed mesh */
  BM_ENOMEM = 2,      /* host or device allocation failed, or admission budget exceeded */
  BM_ECUDA = 3,       /* a CUDA runtime call failed (message has the CUDA error) */
  BM_ENONFINITE = 4,  /* the step produced a NaN or infinity */
  BM_ENEGDEPTH = 5,   /* a depth fell below -h_min */
  BM_ETIMEOUT = 6,    /* a bounded device wait gave up */
  BM_EAGAIN = 7,      /* result not ready yet (bm_poll) */
  BM_EBUSY = 8        /* resource in use */
} bm_status;

enum { BM_FP64 = 0, BM_FP32_BULK = 1 };
enum { BM_TAG_WALL = 0, BM_TAG_TRANSMISSIVE = 1, BM_TAG_INFLOW = 2 };

typedef struct bm_mesh bm_mesh;
typedef struct bm_state bm_state;
typedef struct bm_server bm_server;

/*
 * Run parameters: the hydrodynamic module's parameter list (CFL, minimum water
 * depth, upper limit of the time step) plus the discharge hydrograph of the
 * standard inflow boundary.
 *   cfl       Eq. 21 coefficient, in (0, 1]; default 0.9.
 *   g         gravity [m/s^2]; default 9.81.
 *   h_min     minimum water depth [m]: below it a cell is dry (velocity 0,
 *             excluded from Eq. 21, q set to 0 after the step); default 1e-6.
 *   dt_max    upper limit of the time step [s]; default 1.
 *   precision BM_FP64 (every array and operation in FP64) or BM_FP32_BULK
 *             (state, bed and geometry as FP32 offsets from an FP64 datum;
 *             thresholds and mass accumulators in FP64).
 *   cfl_mode  0: Eq. 21 as printed (rho_ij = 4|Omega_i|/(3 l_ij));
 *             1: dt <= CFL |Omega_i| / sum_j l_ij lambda_ij (positivity bound).
 *   datum     FP32_BULK only: FP64 reference elevation; NaN = min(z_bed).
 *   hydro_t, hydro_q, hydro_n  Q(t) [m^3/s] of the inflow boundary, piecewise
 *             linear in t, constant outside; copied; hydro_n = 0 means Q = 0.
 *             hydro_t must be strictly increasing and hydro_q >= 0.
 */
typedef struct {
  double cfl;
  double g;
  double h_min;
  double dt_max;
  int32_t precision;
  int32_t cfl_mode;
  double datum;
  const double* hydro_t;
  const double* hydro_q;
  int64_t hydro_n;
} bm_params;

/* Fill *p with the defaults listed above. */
void bm_params_default(bm_params* p);

/* Thread-local description of the last failure in this thread ("" if none). */
const char* bm_last_error(void);

/*
 * Build a finite-volume mesh (Section "Domain discretization": conforming
 * triangulation, edge lengths l_ij, unit normals n_ij, cell areas |Omega_i|).
 *   xy        2*n_nodes doubles, node coordinates (x0, y0, x1, y1, ...).
 *   tri       3*n_tri node indices; clockwise triangles are reoriented.
 *   z_bed     n_tri bed elevations (one per cell).
 *   manning_n n_tri Manning coefficients n >= 0 (Table 1); 0 = frictionless.
 *   edge_tag  3*n_tri tags; tag[3t+k] applies to the edge (tri[3t+k],
 *             tri[3t+(k+1)%3]) when it is on the boundary: 0 wall, 1 transmissive
 *             (zero gradient), 2 discharge inflow, 3 h-Q relation outflow, 4 weir
 *             outflow (the last two let nothing out until bm_state_set_outflow
 *             sets their laws), 5 water level (a wall until bm_state_set_level sets
 *             its series).  Ignored on interior edges.
 * Errors: BM_EINVAL for n_tri < 1, indices out of range, area <= 0, an edge
 * shared by more than two triangles or traversed twice in one direction, a tag
 * outside {0,1,2,3,4,5} on a boundary edge, n < 0 or a non-finite input.
 * *out receives the handle (NULL on failure); free with bm_mesh_destroy.
 * Host work only: the mesh is copied to the device by the first state created on
 * it (and stays on that device), so this call needs no GPU.
 */
bm_status bm_mesh_create(const double* xy, int64_t n_nodes, const int32_t* tri, int64_t n_tri,
                         const double* z_bed, const double* manning_n, const uint8_t* edge_tag,
                         bm_mesh** out);

/* Sizes of a mesh: cells, edges, boundary edges, inflow edges, tiles (NULL pointers skipped). */
bm_status bm_mesh_info(const bm_mesh* m, int64_t* n_cells, int64_t* n_edges, int64_t* n_boundary,
                       int64_t* n_inflow, int64_t* n_tiles);

/*
 * Tile layout of a mesh for a precision (BM_FP64 or BM_FP32_BULK): the step reads
 * each tile of 256 Hilbert-ordered cells as one record (inverse areas, edge slots,
 * edge codes and geometry, halo list).  Builds and checks the records on the host
 * (no GPU needed; cached in the mesh) and reports the largest edge list and halo of a
 * tile and the records' total size in bytes (NULL pointers skipped).
 * Errors: BM_EINVAL for a bad precision or an inconsistent layout, BM_ENOMEM.
 */
bm_status bm_mesh_layout(const bm_mesh* m, int32_t precision, int64_t* max_tile_edges, int64_t* max_tile_halo,
                         int64_t* record_bytes);
void bm_mesh_destroy(bm_mesh* m);

/*
 * Create a device-resident state on a mesh (Section "Initial conditions",
 * region-defined: free-surface elevation H and discharge q per cell).
 *   H, qx, qy  n_tri doubles each; qx/qy may be NULL for zeros.  H < z_bed is
 *              rejected (a dry cell is H = z_bed); FP32_BULK accepts a surface down
 *              to its own bed, the datum plus the bed's FP32 offset (what it returns
 *              for a dry cell), so a downloaded state uploads again: a cell exactly on
 *              the FP64 bed or at or below its own bed is dry, a film above its own
 *              bed keeps its depth.  The time starts at 0.
 * The mesh must outlive the state.  Allocates device memory.
 */
bm_status bm_state_init(const bm_mesh* m, const bm_params* p, const double* H, const double* qx,
                        const double* qy, bm_state** out);
void bm_state_destroy(bm_state* s);

/* Order all later device work of this state on `cuda_stream` (a cudaStream_t; NULL =
 * the legacy default stream).  Until this is called the state uses a private
 * non-blocking stream.  Waits for work already queued on the previous stream. */
bm_status bm_state_set_stream(bm_state* s, void* cuda_stream);

/* Take n_steps explicit steps (dt from Eq. 21 each step, dt_max applied).  Blocks
 * until done; returns BM_ENONFINITE / BM_ENEGDEPTH if the device flagged it, or
 * BM_ETIMEOUT if a step's data copies did not arrive within about a second. */
bm_status bm_step(bm_state* s, int64_t n_steps);

/* Enqueue n_steps steps on the state's stream and return at once (no status check). */
bm_status bm_step_async(bm_state* s, int64_t n_steps);

/* Wait for the state's stream and report the device status (as bm_step). */
bm_status bm_sync(bm_state* s);

/* Step until t == t_end exactly (the last dt is clipped to t_end - t). */
bm_status bm_run_until(bm_state* s, double t_end);

/* Replace the state and time (checkpoint resume); arrays as in bm_state_init. */
bm_status bm_state_upload(bm_state* s, const double* H, const double* qx, const double* qy, double t);

/* Copy the state to host arrays (caller order); any pointer may be NULL. */
bm_status bm_state_download(bm_state* s, double* H, double* qx, double* qy, double* t);

/*
 * Flood tracking (the hydrodynamic module's "Flood" outputs), updated in the step
 * kernel with every step from the call on, per cell: the water front arrival time
 * (the first t^{n+1} at which the depth h = H - z exceeds h_arrival; NaN until then)
 * and the running maxima of h, of the flow velocity |u| = |q| / h, of the specific
 * discharge |q| = sqrt(q_x^2 + q_y^2) and of the bed shear stress of the friction law
 * in force (Eq. 2; rho = 1000 kg/m^3): rho g n^2 |u|^2 / h^(1/3) under Manning's law
 * (law 0, the default), rho |u|^2 / c_f^2 under Chezy's or Bezzola's (laws 1 and 2, see
 * bm_state_set_friction); |u| and the stress are 0 where h <= h_min.
 * bm_state_track starts (or restarts) the record from the current state: arrival = t
 * where h > h_arrival, maxima = the current values.  It allocates the five tracking
 * arrays on first use (5 values per cell) and blocks.  h_arrival must be finite and
 * >= 0 (BM_EINVAL).  Uploading a state does not restart the record; batches created
 * after the call track their member (the batch copies the member's descriptor).
 * bm_state_download_track copies the record to host arrays in the caller's cell order
 * (any pointer may be NULL); BM_EINVAL while tracking was never started.  FP32-bulk
 * states keep the maxima in single precision (the arrival time in double).
 */
bm_status bm_state_track(bm_state* s, double h_arrival);
bm_status bm_state_download_track(bm_state* s, double* t_arrival, double* h_max, double* u_max, double* q_max,
                                  double* tau_max);

/*
 * Passive species (Section "Scalar advection-diffusion", Eq. 8 with the diffusion and
 * source terms off): up to 5 concentrations phi_c carried by the water, advected with
 * every step from the call on.  The unknowns are q_c = h phi_c per cell; the flux of
 * a species through an edge is the edge's HLLC mass flux times phi_c of the upwind
 * side of the contact wave (the step kernel's own decision), phi_c = q_c / h where
 * h > 0, else 0; walls carry nothing, a transmissive edge carries the inside value,
 * and the water entering through inflow edges carries c_in[c].  A cell that ends a
 * step dry keeps no species (q_c = 0).  External sources (bm_state_set_sources) change
 * the water only: with Eq. 8's source term off, rain and other sources bring no species
 * (they dilute) and sinks take none (they concentrate).
 * bm_state_set_scalars sets the species: hc holds n_species * n_cells values of q_c
 * (species-major, caller cell order, finite; BM_EINVAL otherwise), c_in n_species
 * inflow concentrations (NULL: 0).  n_species in [0, 5]; 0 removes them.  It
 * allocates 2 * n_species values per cell plus, per tile edge, one exported flux and
 * one byte, and blocks.  From then on every step launches a second kernel after the
 * step kernel (one CTA per tile); in a batch, after the batch's step launch, one such
 * kernel per member with species.  Set species before bm_batch_create on a batch
 * member: a batch made earlier refuses to step (BM_EINVAL).  Uploading a
 * state keeps the species' values.  bm_state_download_scalars copies q_c back
 * (n_species * n_cells, caller order); BM_EINVAL when the state carries none.
 * FP32-bulk states keep q_c in single precision.
 */
bm_status bm_state_set_scalars(bm_state* s, int32_t n_species, const double* hc, const double* c_in);
bm_status bm_state_download_scalars(bm_state* s, double* hc);

/*
 * External sources and sinks (Section "External inflow/outflow discharge"): S_h [m/s]
 * over regions of cells, added explicitly to the continuity equation (the S term of
 * Eq. 12, evaluated at t^n) with every step from the call on.
 * region: n_cells entries (caller order), the region of each cell in [0, n_regions)
 * or -1.  Per region r: kind[r] 0 = total discharge [m^3/s] spread over the region's
 * area (S_h = v / A_r), 1 = intensity [mm/h] (S_h = v / 3.6e6); mode[r] 0 = Exact
 * (the depth changes by dt S_h as prescribed; a sink larger than the water ends the
 * run with BM_ENEGDEPTH), 1 = Available (a sink takes at most the
 * water the cell holds after the step's fluxes), 2 = Infinity (the region takes all
 * the water its cells hold, whatever v); its series v(t) is the points
 * (t[k], v[k]) for k in [offsets[r], offsets[r+1]) (times strictly increasing),
 * piecewise linear and constant beyond the ends; v > 0 adds water, v < 0 takes it.
 * Sources add mass, not momentum.  n_regions in [0, 65536]; 0 removes them.  BM_EINVAL
 * on malformed input and on a total-discharge region with no cell.  A state may carry
 * passive species too: the sources' water carries none (see bm_state_set_scalars).
 * Blocks.  Every step launches a one-block kernel before the step kernel
 * (S_h at t^n); in a batch, one per member with sources before the batch's step launch.
 * Set sources before bm_batch_create on a batch member (a batch made earlier refuses to
 * step, BM_EINVAL).
 */
bm_status bm_state_set_sources(bm_state* s, int32_t n_regions, const int32_t* region, const int32_t* kind,
                               const int32_t* mode, const int64_t* offsets, const double* t, const double* v);

/*
 * Bed evolution (Section "Morphodynamics": Exner, Eq. 3 with S_b = 0, updated by Eq. 13
 * with the HLL sediment flux of Eq. 14-16), stepped with the water from the call on
 * (synchronous-decoupled: the same dt, every term from U^n and z^n).  Bedload from
 * Table 2's MPM-like closure: |q_B| = alpha (theta - theta_cr)^m sqrt((s - 1) g d^3),
 * theta = n^2 |u|^2 / ((s - 1) d h^(1/3)) (Manning's bed shear stress), along the flow;
 * dq_B,n/dq_n of Eq. 16 along the flow at fixed depth.  Walls carry no sediment, other
 * boundary edges the inside cell's normal bedload.  The free surface moves with the
 * bed, so the water depth and volume are kept.  on = 0 stops it (the bed stays as it
 * is).  FP64 states only; 0 <= porosity < 1, s > 1, d > 0 [m], alpha >= 0, m >= 1,
 * theta_cr finite (BM_EINVAL otherwise).  Every step launches three more kernels (the
 * step's dt saved before it; the bed fluxes, one CTA per tile, and the update after
 * it), in a batch for each member with morphodynamics around the batch's step launch;
 * set it before bm_batch_create on a batch member (a batch made earlier refuses to step).
 * Blocks.  bm_state_download_bed copies the bed elevation (caller order) to z.
 */
/*
 * Friction closure (Table 1, used in Eq. 2's S_f = u |u| / (g h c_f^2) by the split
 * friction step): law 0 Manning with coef = n (the default, set from bm_params at
 * init; Strickler is Manning with n = 1 / k_str), 1 Chezy with coef = K_s [m]
 * (c_f = 6.25 + ln(h / K_s) for h > K_s, else 6.25), 2 Bezzola with coef = y_R [m]
 * (c_f = 2.5 sqrt(1 - y_R/h) ln(10.9 h / y_R) for h / y_R > 2, 1.25 sqrt(h / y_R)
 * ln(10.9 h / y_R) for 0.5 <= h / y_R <= 2, 1.5 below).  coef: n_cells values,
 * caller order, finite and >= 0 (0: no friction in that cell).  Laws 1 and 2 run in
 * the step kernel's optional-feature instantiation; flood tracking records the bed
 * shear stress of the law in force (rho u^2 / c_f^2); bed evolution takes Manning's law
 * only (BM_EINVAL either way round).  Blocks.
 */
bm_status bm_state_set_friction(bm_state* s, int32_t law, const double* coef);

bm_status bm_state_set_morpho(bm_state* s, int32_t on, double porosity, double s_rel, double d, double alpha,
                              double m, double theta_cr);

/*
 * Outflow laws of the mesh's h-Q (tag 3) and weir (tag 4) edges (Section "Boundary
 * conditions", standard outflows; the appendix's parameter lists: the H-Q relation;
 * the weir height and Poleni factor).
 *   h-Q relation: the discharge Q leaving through all h-Q edges together is the rating
 *     curve -- piecewise linear through (hq_stage[k], hq_discharge[k]), k < n_hq,
 *     constant beyond its ends -- at the stage S, the length-weighted mean free
 *     surface over the h-Q edges whose cell is wet (h > h_min); Q is split over those
 *     edges by conveyance, q_e = Q h_e^(5/3) / sum_f l_f h_f^(5/3).  n_hq = 0: nothing.
 *   weir: q_e = (2/3) mu sqrt(2 g) eta^(3/2) per unit width (Poleni), eta the head of
 *     the cell's free surface over the crest elevation weir_crest (a crest below the
 *     cell's bed counts from the bed: free overfall); mu = weir_poleni (0: nothing).
 * Each outflow edge's flux is that of the boundary state on the cell's outgoing
 * characteristic (u_n + 2 sqrt(g h) carried from the cell) that carries q_e, with q_e
 * first capped at the critical discharge (u_n + 2 sqrt(g h))^3 / (27 g); that state's
 * u_b + sqrt(g h_b) enters Eq. 21; an edge that lets nothing out is a wall.  Passive
 * species leave with the inside cell's concentration, bedload as on a transmissive
 * edge.  Stages and crest are absolute elevations [m], discharges [m^3/s] >= 0 and
 * finite, stages strictly increasing, n_hq = 0 or >= 2, weir_poleni finite >= 0
 * (BM_EINVAL otherwise; the arrays are copied).  Re-primes the state: the next step's
 * dt and h-Q split follow the new laws; time and step count are kept.  Set it before
 * bm_batch_create on a batch member (the batch copies the member's laws then); served
 * requests (bm_submit) take none (their h-Q and weir edges are walls).  Blocks.
 */
bm_status bm_state_set_outflow(bm_state* s, const double* hq_stage, const double* hq_discharge, int64_t n_hq,
                               double weir_crest, double weir_poleni);

/*
 * The water-level series of the mesh's level edges (tag 5; Section "Boundary
 * conditions": the zhydrograph of the standard inflows and outflows, whose input is
 * the water surface elevation, and the appendix's parameter list).  The imposed
 * surface Z_b(t) is piecewise linear through (t[k], z[k]), k < n, constant beyond its
 * ends; n = 0 turns the level edges back into walls.  A level edge's flux is HLLC's
 * between its cell (depth h, outward normal velocity u_n) and the boundary state of
 * depth h_b = max(0, Z_b(t^n) - z_cell), normal velocity
 * u_b = u_n + 2 sqrt(g h) - 2 sqrt(g h_b) (the cell's outgoing Riemann invariant; 0 next
 * to a cell at or below h_min) and the cell's tangential velocity; that state's
 * |u_b| + sqrt(g h_b) at Z_b(t^{n+1}) enters Eq. 21.  The condition fixes the state of
 * subcritical flow; which boundary type suits the flow regime is the user's choice.
 * Passive species leave with the cell's concentration and enter with none; bedload
 * leaves as on a transmissive edge.  Times and levels finite, times strictly
 * increasing, n <= 2^20 (BM_EINVAL otherwise; the arrays are copied).  Re-primes the
 * state: the next step's dt follows the level; time and step count are kept.  Set it
 * before bm_batch_create on a batch member (the batch reads the member's series);
 * served requests (bm_submit) take none (their level edges are walls).  Blocks.
 */
bm_status bm_state_set_level(bm_state* s, const double* t, const double* z, int64_t n);
bm_status bm_state_download_bed(bm_state* s, double* z);

/*
 * The work of the state's last step launch: the tiles (of 256 cells) it took (0 before
 * the first launch, or when the state changed since) and the state's tiles in all.  A
 * launch takes the tiles with boundary edges that carry mass, inflow, outflow or source
 * cells, and those the previous launch listed (the tiles that were not quiet, and the
 * tiles next to them); a skipped tile is dry and at rest, with no changed neighbour, so
 * its step would copy it through unchanged.  The first launch after the state or its
 * features changed, or after it was stepped in a batch, takes every tile, and so does
 * every launch of a state with passive species or bed evolution, and a launch after one
 * that listed most tiles.  Results do not depend on it.  Blocks (waits for the state's
 * stream).
 */
bm_status bm_state_work(bm_state* s, int64_t* tiles_last, int64_t* tiles_total);

/*
 * Tile skipping (on = 1, the default) or not (on = 0: every launch takes every tile, as
 * a state with passive species does).  Results are bitwise the same either way; the
 * switch exists to show that, and to time the step without it.  on must be 0 or 1
 * (BM_EINVAL).  Takes effect from the next launch.
 */
bm_status bm_state_set_tile_skipping(bm_state* s, int32_t on);

/*
 * Scalars of the state: time, the dt the next step will take, steps taken,
 * water volume V = sum |Omega_i| (H_i - z_i) (FP64, fixed summation order), and
 * the net volume that entered through the boundary since init/upload.
 */
bm_status bm_state_stats(bm_state* s, double* t, double* dt_next, int64_t* steps, double* volume,
                         double* boundary_volume);

/*
 * Diagnostic timing: take n_steps steps as plain kernel launches (no graph) with a
 * CUDA event pair around every launch of the step kernel on the state's stream.
 * *step_kernel_ms receives the summed duration of the step-kernel launches and
 * *total_ms the time from the first to the last event; either may be NULL.  The
 * state advances exactly as bm_step would.
 */
bm_status bm_step_timed(bm_state* s, int64_t n_steps, double* step_kernel_ms, double* total_ms);

/*
 * Diagnostics for tests of the failure path (the paper has no counterpart: the bounded
 * waits belong to this library's step kernel): one step launch in
 * which every CTA's copy warp withholds the halo copies of its first tile, so the
 * compute warps' bounded wait for them runs out after about a second.  Every CTA then
 * retires the copies it did issue and exits without writing the state; the call blocks
 * and returns BM_ETIMEOUT with the state, time and step count unchanged.  The status
 * stays set in the state: re-upload it (bm_state_upload) before stepping it again.
 */
bm_status bm_state_test_timeout(bm_state* s);

/*
 * Launch shape of the state's step kernel, whose CTAs stay resident and loop over
 * the 256-cell tiles: ctas_per_sm = 0 launches as many CTAs per SM as fit (the
 * default), k > 0 launches k per SM, at most as many as fit (every CTA of the launch
 * is resident from its start: a share of the tiles is assigned to CTAs statically).
 * Results do not depend on it.  Chosen by the autotuner or by hand.
 */
bm_status bm_state_set_launch(bm_state* s, int ctas_per_sm);

/*
 * The step kernel's schedule: the launch shape (as bm_state_set_launch) and the static
 * share of the work tickets, static_sixteenths / 16 of them handed to the CTAs in a
 * fixed round-robin (known a step ahead, no atomic), the rest from a launch-wide
 * counter (balancing uneven tiles); -1 = the precision's default (FP64 0/16, FP32-bulk
 * 4/16), at least one ticket per CTA is static (two when claiming ahead, see
 * bm_state_set_claim).  Results do not depend on it (the
 * reductions are order-free).  BM_EINVAL outside [-1, 16].  get returns both.
 */
bm_status bm_state_set_schedule(bm_state* s, int ctas_per_sm, int static_sixteenths);
bm_status bm_state_get_schedule(bm_state* s, int* ctas_per_sm, int* static_sixteenths);

/*
 * Tile slots of the step kernel's pipeline: how many 256-cell tiles a CTA's copy warp
 * may stage in shared memory ahead of its compute warps (2, 3 or 4; default 2).  More
 * slots hide more copy latency but take more shared memory, so fewer CTAs may fit an
 * SM.  The plain step is compiled for each count; a state with optional features
 * (tracking, species, sources, log-law friction, outflow or level laws) runs 3 slots
 * whatever the setting, and get reports the count in force.  Results do not depend
 * on it.  BM_EINVAL outside {2, 3, 4}, or when that layout does not fit the device's
 * shared memory (the count in force is kept).  Chosen by the autotuner or by hand.
 */
bm_status bm_state_set_slots(bm_state* s, int slots);
bm_status bm_state_get_slots(bm_state* s, int* slots);

/*
 * How the step kernel's CTAs claim work items: 0 ahead (the copy warp reads the next
 * items and requests the next tickets a step or two before it needs them, hiding their
 * latency), 1 the next item right after each issue (no tickets ahead), 2 each item once
 * its slot is free (a CTA commits to no more tiles than its slots hold, so the launch's
 * last tiles are not queued behind long ones), 3 as 2 and only once the tile before is
 * past its edge phase (a CTA commits to its next tile near the end of the current one),
 * -1 the precision's default (FP64 3, FP32-bulk 2).  With modes 1-3 a CTA's static
 * tickets may be one.  Results do not depend on it.  BM_EINVAL outside {-1, 0, 1, 2, 3};
 * get reports the mode in force.
 */
bm_status bm_state_set_claim(bm_state* s, int mode);
bm_status bm_state_get_claim(bm_state* s, int* mode);

/*
 * Autotuner: time steps_per_trial steps (rounded up to whole graphs of 32 launches, as
 * bm_step runs them) for each schedule, in two rounds -- for each
 * claiming mode (bm_state_set_claim, the one in force first) and tile-slot count (2, 3,
 * 4 for the plain step, the count in force first; 3 only with optional features) the
 * launch shapes (as many CTAs per SM as fit, and 1, 2, 3, 4 CTAs
 * per SM; shapes giving the same grid are timed once) at the current static share,
 * then the static shares 0, 2, ..., 16 sixteenths and the default at the best slots
 * and shape -- undo the trial steps (the state is snapshotted in device memory and
 * restored), keep the fastest schedule and report its shape and time per step
 * (bm_state_get_schedule, bm_state_get_slots and bm_state_get_claim give the rest).  A schedule replaces
 * the one in force only if it is 2 % faster.  Allocates a temporary device copy of the
 * state.  Results do not depend on it.  The tile size is fixed at compile time:
 * 256-cell tiles of one cell per thread (8 compute warps and 1 copy warp; the tile
 * records are built for that size).
 */
bm_status bm_state_autotune(bm_state* s, int steps_per_trial, int* best_ctas_per_sm, double* ms_per_step);

/*
 * Batches: many independent states (uneven meshes, same precision) stepped by ONE
 * kernel launch per step through a packed (member, tile) work list; each member
 * keeps its own dt, time and status.  The member handles stay valid and owned by
 * the caller; while they are in a batch, step them only through the batch (their
 * stats / download may be read after bm_batch_sync).  Creating a batch allocates a
 * little device memory (descriptors, work list); the members' data is not copied.
 * Members may carry any feature (tracking, species, sources, friction closures,
 * outflow and level laws, bed evolution): the batch's step launch runs the lowest
 * instantiation that serves them all, and each member's own kernels (sources' rates
 * before, species and bed update after) run around it.  A member's features must be
 * set before the batch is made: stepping a batch whose member changed a feature since
 * returns BM_EINVAL ("make the batch again").
 */
typedef struct bm_batch bm_batch;
bm_status bm_batch_create(bm_state* const* states, int32_t n_states, bm_batch** out);
void bm_batch_destroy(bm_batch* b);
bm_status bm_batch_info(const bm_batch* b, int32_t* n_members, int64_t* n_cells, int64_t* n_tiles);
/* Order the batch's launches on a stream (NULL = the legacy default stream). */
bm_status bm_batch_set_stream(bm_batch* b, void* cuda_stream);
/* Launch shape, as bm_state_set_launch; the autotuner as bm_state_autotune. */
bm_status bm_batch_set_launch(bm_batch* b, int ctas_per_sm);
bm_status bm_batch_set_schedule(bm_batch* b, int ctas_per_sm, int static_sixteenths);
bm_status bm_batch_get_schedule(bm_batch* b, int* ctas_per_sm, int* static_sixteenths);
bm_status bm_batch_set_slots(bm_batch* b, int slots);
bm_status bm_batch_get_slots(bm_batch* b, int* slots);
bm_status bm_batch_set_claim(bm_batch* b, int mode);
bm_status bm_batch_get_claim(bm_batch* b, int* mode);
bm_status bm_batch_autotune(bm_batch* b, int steps_per_trial, int* best_ctas_per_sm, double* ms_per_step);
/* Every member takes n_steps steps with its own dt (Eq. 21); blocks; returns the
 * first member's BM_ENONFINITE / BM_ENEGDEPTH if any. */
bm_status bm_batch_step(bm_batch* b, int64_t n_steps);
bm_status bm_batch_step_async(bm_batch* b, int64_t n_steps);
bm_status bm_batch_sync(bm_batch* b);
/* Member k runs until exactly t_end[k] (n_states finite values); finished members
 * idle while the others continue (once a quarter of the listed members have
 * finished, the launches list only the running ones; blocks, allocating a work list
 * each time). */
bm_status bm_batch_run_until(bm_batch* b, const double* t_end);

/*
 * Request server (continuous batching).  Runs are submitted at any time from any
 * thread; a worker thread admits them while the sum of their device footprints
 * (state arrays, not the mesh) fits hbm_budget_bytes and at most max_slots are
 * resident, steps every resident run together (one launch per step, each run with
 * its own dt; a run stops exactly at its t_end), copies finished runs out, frees
 * their memory and admits waiting runs.  A run's result is the same as that of
 * bm_state_init + bm_run_until(t_end) on its own, whatever else is running.
 *   hbm_budget_bytes  0 = 80 % of the free device memory at creation.
 *   max_slots         0 = no limit.
 *   precision         every run of a server uses this precision.
 *   steps_per_round   steps between the worker's admissions / completion checks.
 *   ctas_per_sm       launch shape of the batched step (bm_state_set_launch).
 * Meshes are owned by the caller and must outlive the runs that use them.
 */
typedef struct {
  uint64_t hbm_budget_bytes;
  int32_t max_slots;
  int32_t precision;
  int32_t steps_per_round;
  int32_t ctas_per_sm;
} bm_server_opts;

void bm_server_opts_default(bm_server_opts* o);
bm_status bm_server_create(const bm_server_opts* opts, bm_server** out);
/* Stops the worker; runs not finished yet complete with BM_EBUSY. */
void bm_server_destroy(bm_server* sv);
/*
 * Submit a run: mesh, parameters (copied; precision must be the server's), initial
 * H, qx, qy (n_cells doubles each, copied; qx/qy may be NULL) and the end time
 * t_end > 0 (the run starts at t = 0).  Non-blocking; *ticket identifies the run.
 * BM_ENOMEM if the run alone exceeds the budget; BM_EINVAL for bad arguments.
 */
bm_status bm_submit(bm_server* sv, const bm_mesh* mesh, const bm_params* p, const double* H, const double* qx,
                    const double* qy, double t_end, uint64_t* ticket);
/*
 * BM_EAGAIN while the run is queued or running.  When finished: copies the final
 * state (caller order; NULL pointers skipped) and the time from submission to
 * completion, forgets the ticket and returns BM_OK, or the run's failure status.
 */
bm_status bm_poll(bm_server* sv, uint64_t ticket, double* H, double* qx, double* qy, double* latency_s);
/*
 * bm_submit with flood tracking (see bm_state_track): h_arrival >= 0 starts the record
 * when the run is admitted (its footprint counts the record); h_arrival < 0 is
 * bm_submit.  bm_poll_track copies the finished run's record (caller order, any
 * pointer may be NULL) and leaves the ticket for bm_poll: call it first.  BM_EAGAIN
 * while the run is not finished, BM_EINVAL for an unknown ticket or a run submitted
 * without tracking, the run's error if it failed.
 */
bm_status bm_submit_tracked(bm_server* sv, const bm_mesh* mesh, const bm_params* p, const double* H,
                            const double* qx, const double* qy, double t_end, double h_arrival, uint64_t* ticket);
bm_status bm_poll_track(bm_server* sv, uint64_t ticket, double* t_arrival, double* h_max, double* u_max,
                        double* q_max, double* tau_max);
/* Block until the run has finished (or timeout_s elapsed: BM_ETIMEOUT); then bm_poll. */
bm_status bm_server_wait(bm_server* sv, uint64_t ticket, double timeout_s);
/* Queued, running and completed runs, cell-updates done, device bytes admitted. */
bm_status bm_server_stats(bm_server* sv, int64_t* queued, int64_t* running, int64_t* completed,
                          double* cell_updates, double* resident_bytes);

/*
 * Water volume V = sum_i area_i (H_i - z_i) over caller-owned device arrays, computed
 * without allocating any device memory.  The paper has no counterpart: this exists
 * for callers that cannot call cudaMalloc -- applications whose device memory is
 * entirely handed to their own pool allocator (a stray cudaMalloc would fail or
 * fragment it) and loops that cannot afford cudaMalloc/cudaFree's implicit device
 * synchronisation.  It runs the library's volume reduction with its partial sums
 * in a fixed scratch array compiled into the library (64 KiB, held on every device
 * that loads the library until the process exits).
 *   H, z, area  n_cells doubles each, device memory, any cell order.
 *   volume      device pointer receiving the result (one double).
 *   cuda_stream the stream the two kernels are queued on (NULL = legacy default);
 *               the call returns without waiting for them.
 * Limits and behaviour: n_cells up to 2,097,152 (BM_EINVAL beyond, before any device
 * work); n_cells = 0 writes 0.  The first call on a device looks the scratch array up
 * (cudaGetSymbolAddress) with that device current; make that first call before any
 * stream capture.  All calls share the one array and it keeps the last call's
 * partials; every call overwrites what it reads, so nothing needs clearing, but two
 * calls whose kernels overlap on the GPU race and can return wrong sums -- order
 * them on one stream or synchronise in between.
 */
bm_status bm_volume_noalloc(const double* H, const double* z, const double* area, int64_t n_cells, double* volume,
                            void* cuda_stream);

/* Diagnostics: evaluate one of the step kernel's hand-written elementary functions, or
 * the CUDA library function it stands in for, on n host values (copied to the device
 * and back; synchronous).  fn: 0 x^(-1/3) as the FP64 step computes it (Newton steps
 * from a single-precision estimate), 1 the library's 1/cbrt(x), 2 1/x as the FP64 step
 * computes it (Newton steps from the hardware reciprocal estimate), 3 the IEEE
 * division 1/x, 4 x^(-1/3) as the FP32-bulk step computes it (hardware base-2
 * logarithm and exponent), 5 the library's rcbrtf, 6 x^(1/3) as the FP64 step computes
 * it, 7 the library's cbrt.  x, y: n doubles each (host memory, caller-owned; FP32
 * functions see x rounded to float).  BM_EINVAL for fn outside [0, 7], n outside
 * [0, 2^28] or NULL arrays; BM_ECUDA / BM_ENOMEM from the device. */
bm_status bm_math_eval(int32_t fn, const double* x, double* y, int64_t n);

#ifdef __cplusplus
}
#endif
#endif /* BM_H */
