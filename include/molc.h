/*
 * molc.h — C ABI of libmolc: the high-order sweep of the method of long characteristics (MOLC / ray tracing)
 * for the backward-Euler multigroup Boltzmann transport equation, on one GB300 (sm_103a) GPU.
 *
 * Paper: J. M. Coale and D. Y. Anistratov, "Multilevel method for thermal radiative transfer problems with
 * method of long characteristics for the Boltzmann transport equation" — Sec. 3 (the MOLC / ray-tracing
 * scheme, Eqs. 10-16) and Sec. 2 (the moments E_g, F_g and the Eddington tensor, Eqs. 4 and 7).
 *
 * Conventions shared by every entry point:
 *  - Units: lengths in cm, time in shakes, opacity in cm^-1, intensities (B, boundary, I) in one intensity unit;
 *    E is (1/c) x intensity.
 *  - Cell index i = iy * nx + ix; per-group arrays are [G][ny*nx] row-major ("[g][cell]").
 *  - "device" pointers are CUDA device memory of the device current when molc_create() ran; the caller owns
 *    them (allocates and frees).  "host" pointers are ordinary host memory, read during the call only.
 *  - Entry points that take a stream are asynchronous on that stream (NULL = legacy default stream), perform
 *    no device allocation and no host synchronisation, and return MOLC_ERR_CUDA if a launch fails.  Errors the
 *    kernels detect (non-finite or negative inputs) are recorded in a per-plan device status word that
 *    molc_device_status() reads; kernels never trap.
 *  - Every entry point returns a molc_status; on failure molc_last_error() gives a message (thread-local).
 *  - A plan is not thread-safe: calls on one plan must be serialised by the caller (one stream at a time).
 */
#ifndef MOLC_H
#define MOLC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st *molc_stream; /* a cudaStream_t */

typedef enum {
  MOLC_OK = 0,
  MOLC_ERR_INVALID_ARG = 1,      /* a host-checkable argument is wrong (sizes, NULLs, quadrature structure) */
  MOLC_ERR_OUT_OF_MEMORY = 2,    /* molc_create could not allocate the plan's device tables */
  MOLC_ERR_CUDA = 3,             /* a CUDA runtime call or kernel launch failed */
  MOLC_ERR_NONFINITE_INPUT = 4,  /* device status: kappa, B or the boundary held NaN/Inf or a negative value */
  MOLC_ERR_TIMEOUT = 5,          /* device status: a bounded wait of the tiled FP32 sweep gave up (an item's
                                    upstream items or its staged data did not arrive within ~1 s); that step's
                                    results are void */
  MOLC_ERR_INTERNAL = 6,
  MOLC_ERR_RANGE = 7             /* device status: a scaled value exceeds the range of an FP32 state (cannot
                                    happen for finite inputs: the state's power-of-two scale follows
                                    max(B, boundary) at every sweep) */
} molc_status;

typedef enum { MOLC_FP64 = 0, MOLC_FP32 = 1 } molc_precision;

/* Characteristic-grid construction (Sec. 3, last paragraph before the results).
 *  MOLC_RAYS_UNIFORM: per azimuth, n = ceil(L_perp / spacing) parallel characteristics of equal width
 *                     w = L_perp / n (L_perp = projected width of the domain), centred at (k + 1/2) w.
 *  MOLC_RAYS_PAPER:   the paper's rule: the gaps between the projections of all grid vertices are the initial
 *                     characteristics (no characteristic crosses a vertex); each is halved until w <= spacing. */
typedef enum { MOLC_RAYS_UNIFORM = 0, MOLC_RAYS_PAPER = 1 } molc_layout;

/* flags for molc_create */
#define MOLC_AREA_RENORM 1u /* scale A_{k,s} per (cell, azimuth) so that sum over C(i,m) of A = cell area */
#define MOLC_HOST_ONLY 2u   /* build the characteristic grid on the host only (no device memory, no GPU needed):
                               only molc_plan_get_info, molc_intensity_count, molc_intensity_bytes,
                               molc_tracks_export, molc_plan_retile (the tiles are re-cut on the host) and
                               molc_destroy accept such a plan; every other call that takes it returns
                               MOLC_ERR_INVALID_ARG */
#define MOLC_FACES 8u       /* also accumulate the face moments of Eq. 16 in every molc_sweep (device memory for
                               6 FP64 sums per (face, group); FP64 reductions per segment, so sweeps are slower);
                               read them with molc_face_moments */
#define MOLC_AUTOTUNE 4u    /* time launch configurations of the FP32 sweep on this plan during molc_create and
                               keep the fastest: the compiled staging depths of the bundle sweep
                               (molc_plan_info.fp32_sweep_depth), or for a tiled plan the planner's tile side,
                               groups per work item and block size and their neighbours (fp32_tile_cells,
                               fp32_tile_groups, fp32_block_threads).  Temporary device memory of about one FP32
                               state.  The choice changes no segment update, only speed (a tiled plan's moment
                               summation order follows its tiles).  With a tuning cache set (molc_tune_cache) a
                               recorded choice is applied without timing. */
#define MOLC_BALANCE 16u    /* also evaluate the per-ray discrete balance of every sweep in FP64 (a check, not part
                               of the result; FP64 work per update, so sweeps are slower); read the largest
                               relative residual with molc_ray_balance.  Not with MOLC_FACES. */
#define MOLC_TILED 32u      /* sweep FP32 with the tiled kernel: the characteristics cut into per-tile pieces, one
                               persistent launch over (tile, quadrant, group tile) work items in wavefront order, the
                               cell moments summed in shared memory (no second pass over the state).  Ignored with
                               MOLC_FACES or MOLC_BALANCE, with more than 8 polar cosines, or when no tile keeps a work
                               item within shared memory (molc_plan_info.fp32_tile_items == 0 then).  Same segment
                               updates, bit for bit, as the default FP32 sweep; different moment summation order. */

typedef struct {
  int nx, ny;               /* material cells (>= 1) */
  double x0, y0, lx, ly;    /* domain [x0, x0+lx] x [y0, y0+ly], cm (lx, ly > 0) */
} molc_grid;

/* Angular quadrature, host arrays of n directions with mu > 0 (the upper hemisphere; each direction also
 * stands for its mirror through the x-y plane, so the weights sum to 4 pi).  (cos_phi, sin_phi) is the
 * in-plane direction.  Required structure: every direction has an opposite one with (cos_phi, sin_phi)
 * exactly negated and the same mu and w, and every azimuth carries the same list of polar cosines. */
typedef struct {
  int n;
  const double *mu;
  const double *cos_phi;
  const double *sin_phi;
  const double *w;
} molc_quadrature;

typedef struct {
  int G;                    /* number of frequency groups (>= 1) */
  const double *edges;      /* host, G+1 group edges in keV, or NULL (metadata only) */
} molc_groups;

typedef struct molc_plan molc_plan; /* opaque; owns the device characteristic grid and sweep workspace */

/* Cell moments, all device [G][ny*nx] FP64, caller-owned (Sec. 2: E_g = (1/c) int I dOmega,
 * F_g = int Omega I dOmega; Eq. 7 / Eq. 15: N_g = int Omega Omega I dOmega).  Cell averages. */
typedef struct {
  double *E, *Fx, *Fy, *Nxx, *Nxy, *Nyy;
} molc_moments;

typedef struct {
  int G, nx, ny;
  int n_dir;                /* directions (both senses, all polar cosines) */
  int n_azim_pairs;         /* distinct characteristic families: azimuth phi with phi + pi */
  int n_polar;              /* polar cosines per azimuth */
  int64_t n_tracks;         /* characteristics summed over azimuth pairs */
  int64_t n_track_segments; /* segments summed over azimuth pairs (each walked by 2 senses x n_polar) */
  int64_t n_segments;       /* segments summed over all directions (= 2 n_polar n_track_segments) */
  int64_t n_updates;        /* segment x direction x group updates per sweep (= n_segments G) */
  int fp32_groups_per_warp; /* groups per chunk of the FP32 sweep (chunks run one after another) */
  size_t device_bytes;      /* device memory the plan holds */
  int fp32_sweep_depth;     /* staging depth of the FP32 sweep (steps of look-ahead; MOLC_AUTOTUNE picks it) */
  int n_faces;              /* MOLC_FACES: (nx + 1) ny x-faces then nx (ny + 1) y-faces; else 0 */
  int n_split_cells;        /* FP32 moments: cells crossed by more than 256 segment entries, summed in parts and
                               combined by one more kernel launch per sweep (0: no such launch) */
  int fp32_tile_cells;      /* tiled FP32 sweep (plans without MOLC_FACES / MOLC_BALANCE): tile side in cells, or 0
                               when the plan sweeps FP32 without tiles */
  int fp32_tile_groups;     /* tiled FP32 sweep: groups per work item */
  int fp32_tile_items;      /* tiled FP32 sweep: work items per step (tiles x 4 quadrants x group tiles) */
  int fp32_sweep_blocks;    /* tiled FP32 sweep: blocks of its persistent launch */
  int fp32_block_threads;   /* tiled FP32 sweep: threads of one such block */
  int tuned_from_cache;     /* MOLC_AUTOTUNE: 1 when the configuration came from the tuning cache (nothing timed) */
} molc_plan_info;

/* Configuration of a tiled FP32 sweep (no counterpart in the paper: how the sweep's work is cut for the GPU).
 * tile_cells: tile side in cells (the characteristic pieces one work item stages in shared memory);
 * tile_groups: groups per work item (rays per warp = 32 / tile_groups); block_threads: threads of a block of the
 * persistent launch (a multiple of 32, at most 512).  0 in any field: the library's choice. */
typedef struct {
  int tile_cells, tile_groups, block_threads;
} molc_tile_config;

/* Gauss-Legendre (n_polar nodes on mu in (0,1), weights summing to 1) x Chebyshev (phi_j = (j-1/2) 2 pi / n_azim,
 * equal weights) product set, omega = 4 pi w_p / n_azim, direction order m = p * n_azim + j.  n_azim must be a
 * positive multiple of 4; cos/sin are built by exact reflection from the first octant so the set is exactly
 * symmetric.  Host output arrays of n_polar * n_azim entries.  (A substitute for the paper's Abu-Shumays set,
 * Sec. 4, whose table is not available.) */
molc_status molc_quadrature_product(int n_polar, int n_azim, double *mu, double *cos_phi, double *sin_phi,
                                    double *w);

/* Build the characteristic grid on the host (Sec. 3) and upload it to the current CUDA device.
 * ray_spacing: h_moc in cm (> 0).  flags: MOLC_AREA_RENORM, MOLC_HOST_ONLY, MOLC_AUTOTUNE, MOLC_FACES, MOLC_BALANCE,
 * MOLC_TILED (see above) or 0.  groups->G fixes the group count of every later call.  Larger grids are planned on
 * up to one host thread per hardware thread (the threads end before the call returns; the plan is the same as
 * from one thread).  On success *out owns device memory until molc_destroy(). */
molc_status molc_create(const molc_grid *grid, const molc_quadrature *quad, const molc_groups *groups,
                        double ray_spacing, molc_layout layout, unsigned flags, molc_plan **out);

molc_status molc_plan_get_info(const molc_plan *plan, molc_plan_info *info);

/* The opaque intensity state I^{n-1} of one precision (the previous step's segment averages in the source Q of Eq.
 * 11): one element per (segment, direction, group) (FP64: 8 bytes, FP32: 4, laid out for the sweep kernel with a
 * little padding) holding the deviation of the segment average from the cell's Planck intensity, followed by that
 * reference Planck intensity per (group, cell) in FP64 and a small header. The FP32 state works in units scaled by
 * a power of two that maps max(B, boundary) near 2^100 (set by molc_intensity_init from B, and reset by any sweep
 * whose max(B, boundary) has moved by more than ~2^8 from it, the stored deviations being rescaled exactly as they
 * are read), which keeps intensities down to ~1e-68 of that maximum in the normal FP32 range. molc_intensity_count
 * gives the elements, molc_intensity_bytes the bytes to allocate (256-byte aligned device memory). The layout is
 * private to the library; use export/import to read or write segment averages. */
int64_t molc_intensity_count(const molc_plan *plan);
size_t molc_intensity_bytes(const molc_plan *plan, molc_precision prec);

/* I^{n-1} := B_g of the segment's cell on every segment, direction and group (the state before the first step: Eq.
 * 11's I^{n-1} for a medium starting in equilibrium), and the state's scale. I: device, molc_intensity_bytes(prec).
 * B: device [G][cell], finite and >= 0. Allocation-free (memsets, a copy and two small kernels). */
molc_status molc_intensity_init(molc_plan *plan, molc_precision prec, void *I, const double *B,
                                molc_stream stream);

/* One backward-Euler step of the high-order sweep (Sec. 3, Eqs. 11-15), for every azimuth pair,
 * characteristic, sense, polar cosine and group:
 *   kappa~ = kappa + 1/(c dt),  Q = kappa B + I^{n-1}/(c dt),  tau = kappa~ l / sin(zeta),
 *   I_{s+1} = I_s e^-tau + (Q/kappa~)(1 - e^-tau),  Ibar = alpha I_s + (1 - alpha) I_{s+1},
 * I^{n-1} is the previous step's segment average on the same segment, direction and group, and is replaced in
 * place by this step's Ibar.  Entering intensity: bnd[edge][g] (isotropic per edge; edges left, right,
 * bottom, top).  Writes the cell moments E, Fx, Fy, Nxx, Nxy, Nyy of every group into *out (the areas
 * A = l w of Eq. 14 weight the segment averages).
 *   prec   MOLC_FP64: all arithmetic in FP64.  MOLC_FP32: segment arithmetic in FP32; each cell's moment sums
 *          in FP32 within runs of at most 8 segments of one azimuth pair and as two-word FP32 sums (hi + lo,
 *          about 48 significant bits) across the runs, then the cell assembly in FP64.
 *   kappa, B  device [G][cell] FP64;  c (cm/sh) > 0, dt (sh) > 0;  I: device state of precision prec;
 *   bnd    device [4][G] FP64;  out: device pointers, each [G][cell] FP64, overwritten.
 * Asynchronous on `stream`; no allocation. */
molc_status molc_sweep(molc_plan *plan, molc_precision prec, const double *kappa, const double *B, double c,
                       double dt, void *I, const double *bnd, const molc_moments *out, molc_stream stream);

/* Allocation-free variant of molc_sweep (the paper has no counterpart: it is an engineering entry point).
 * Same arguments, semantics and results as molc_sweep, but the per-sweep workspace (the FP64 moment
 * accumulators; for MOLC_FP32 the cell tables, and with a MOLC_TILED plan also the work-item flags, quadrant
 * moment partials and the boundary buffer of the characteristic pieces) comes from one fixed 64 MiB array
 * compiled into the library instead of from the plan.  It is meant for callers that must not allocate device memory, or must
 * know all of it in advance, once they are running: an embedding whose device memory is fully handed to
 * another allocator, or a time-stepping loop run under a fixed memory budget.  Neither this call nor its
 * set-up calls cudaMalloc, cudaFree or any other allocating routine.
 *  - Limit: the workspace is 48 bytes per (cell, group) for MOLC_FP64 (the accumulators) and 20 bytes per
 *    (cell, group) for MOLC_FP32 (the cell tables; groups padded to the plan's group chunk); a MOLC_TILED plan
 *    needs about 220 bytes per (cell, group) plus (polar cosines + 2) x 4 bytes per (characteristic piece,
 *    group); each part is rounded up to 256 bytes.  A plan that needs more than 64 MiB (e.g. more than ~1.4M
 *    cell-groups in FP64, ~3.3M in FP32, ~0.25M tiled) is rejected with MOLC_ERR_INVALID_ARG and nothing is
 *    launched.  molc_sweep has no such limit.
 *  - Set-up: the first call on each device (with the plan's device current) looks up the array's device
 *    address with cudaGetSymbolAddress, which also loads the library's kernels on that device if that has
 *    not happened yet; later calls reuse the cached address.  Make that first call before any stream
 *    capture.
 *  - The FP64 accumulators must start at zero; every FP64 call clears them itself (cudaMemsetAsync on
 *    `stream`) before its kernels run, so nothing needs to be zeroed by the caller.  The FP32 cell tables are
 *    fully rewritten by every call; a tiled FP32 call also clears its control words, work-item flags and
 *    arrival counts (a few KB) before its kernels run.
 *  - There is ONE array per device, shared by every plan and stream in the process: calls that can overlap in
 *    time on the same device (different streams, or different host threads) race on it and give wrong
 *    results.  Serialise them, e.g. issue them all on one stream.
 *  - Sweep-kernel timing (molc_kernel_timing) does not record this call.
 *  - A FP32 plan with cells crossed by more than 256 characteristic segments (very fine ray spacing) also sums
 *    per-part partials in a buffer of its own, allocated by molc_create, as molc_sweep does. */
molc_status molc_sweep_static_scratch(molc_plan *plan, molc_precision prec, const double *kappa,
                                      const double *B, double c, double dt, void *I, const double *bnd,
                                      const molc_moments *out, molc_stream stream);

/* ---- Batched FP32 sweep of many independent instances (Eqs. 7, 11-15 for each; plans of any sizes, group counts
 * and quadratures on one device): every step runs as one launch of each kernel over the work of all instances (the
 * scale update over several blocks per instance, one prep launch, one sweep launch per distinct (polar count,
 * staging depth) and one moment launch per polar count, in order on the caller's stream), with the sweep blocks of
 * all instances scheduled longest first; batches of MOLC_TILED plans run one prep and one persistent tiled sweep
 * launch instead.  Built for many uneven problems in one time-stepping loop, where per-instance launches would
 * leave most of the GPU idle. The paper sweeps one problem; this is the production packaging of the same
 * per-instance sweep (results are bit-identical to molc_sweep + molc_closure per instance). */
typedef struct molc_batch molc_batch;

/* Per-instance arguments, as for molc_sweep (device pointers) plus optional Eddington factors. */
typedef struct {
  const double *kappa, *B;      /* device [G][cell] */
  double c, dt;                 /* > 0 */
  void *I;                      /* device FP32 state of this instance's plan (molc_intensity_init'ed) */
  const double *bnd;            /* device [4][G] */
  molc_moments out;             /* device, each [G][cell] */
  double *fxx, *fxy, *fyy;      /* device [G][cell] (f = N / (c E), as molc_closure), or all NULL */
} molc_sweep_args;

/* Builds a batch (no counterpart in the paper: block maps over the instances). plans: host array of n (>= 1) plans
 * created on the current device (not MOLC_HOST_ONLY, MOLC_FACES or MOLC_BALANCE, at most 8 polar cosines, either
 * all tiled or none; MOLC_ERR_INVALID_ARG otherwise); the batch keeps pointers to them (destroy the batch first).
 * Builds the block maps (device). */
molc_status molc_batch_create(molc_plan *const *plans, int n, molc_batch **out);

/* Record the per-instance arguments of Eqs. 11-15 (and 7) (host array of n, copied to the device synchronously).
 * Call again whenever a buffer changes; molc_batch_sweep uses the last recorded arguments. */
molc_status molc_batch_bind(molc_batch *batch, const molc_sweep_args *args);

/* One backward-Euler step (Eqs. 11-15) of every instance: molc_sweep_closure in FP32 for the instances bound with
 * factor outputs, molc_sweep for the others. Asynchronous on `stream`; no allocation and no host synchronisation,
 * so a step (or several) can be captured in a CUDA graph and replayed. Device status words are per plan
 * (molc_device_status). */
molc_status molc_batch_sweep(molc_batch *batch, molc_stream stream);

/* Frees the batch (no counterpart in the paper). */
void molc_batch_destroy(molc_batch *batch);

/* Eddington factors of each cell and group, f = N / (c E) (Eq. 7 with the cell averages of Eq. 15):
 * fxx, fxy, fyy device [G][cell]; f_zz = 1 - f_xx - f_yy.  f_grey: device [3][cell] or NULL, the
 * E-weighted spectral average <f>_E = sum_g f_g E_g / sum_g E_g (Sec. 2, Eq. 8) of xx, xy, yy.
 * A cell with E = 0 gets f = 0. */
molc_status molc_closure(const molc_plan *plan, const molc_moments *m, double c, double *fxx, double *fxy,
                         double *fyy, double *f_grey, molc_stream stream);

/* Per-ray discrete balance of the sweeps of a plan created with MOLC_BALANCE (Eqs. 11-13: the transport equation
 * integrated along each characteristic, which the exact attenuation of Eq. 12 satisfies segment by segment).
 * For every characteristic k, direction and group of the sweep,
 *   R = I_in - I_out + sum_s (Q_s - kappa~_s Ibar_s) l_s / sin zeta
 * is formed in FP64 from the values the sweep itself computed (in the sweep's working precision), and divided by
 * S, the sum of the magnitudes of its terms written segment by segment in the variables the sweep rounds
 * (|I_in,s|, |I_out,s|, their deviations from the cell's B, |Q_s| l_s / sin zeta, kappa~_s |Ibar_s| l_s / sin zeta,
 * and the cell-to-cell steps of B that the deviation form adds at each crossing): a few units of the working
 * precision's rounding (FP64 ~1e-16, FP32 ~1e-7) when the sweep's arithmetic is consistent.  Rays with S below
 * 1e-30 of max(B, boundary) of the sweep carry no radiation at the working precision and are left out.
 * *max_rel_residual
 * := the largest |R| / S over all characteristics, directions and groups of the molc_sweep or molc_sweep_closure
 * calls since the last molc_sweep or molc_sweep_closure began (0 before any; molc_sweep_static_scratch on such a
 * plan adds its rays without starting a new record).  Synchronises with the device.
 * MOLC_ERR_INVALID_ARG for a plan created without MOLC_BALANCE. */
molc_status molc_ray_balance(const molc_plan *plan, double *max_rel_residual);

/* One backward-Euler step and the Eddington factors of its moments in one call (Eqs. 7, 11-15): the same as
 * molc_sweep followed by molc_closure(plan, out, c, fxx, fxy, fyy, NULL, stream), bit for bit, with the factors
 * formed where each cell's moments are assembled (no second pass over the moments).  fxx, fxy, fyy: device
 * [G][cell], caller-owned, all non-NULL (else MOLC_ERR_INVALID_ARG).  Other arguments, errors and
 * asynchrony as molc_sweep; the grey average is not formed (molc_closure gives it). */
molc_status molc_sweep_closure(molc_plan *plan, molc_precision prec, const double *kappa, const double *B, double c,
                               double dt, void *I, const double *bnd, const molc_moments *out, double *fxx,
                               double *fxy, double *fyy, molc_stream stream);

/* Face-average moments of the last molc_sweep in precision prec (plans created with MOLC_FACES), the
 * quantities of the face Eddington tensor (Eq. 16): for every face f and group, with I_{k,s} the intensity at
 * the upwind face of each segment whose upwind face is f (F(f, m)) and w_k its characteristic's width,
 *   E_f = (1/(c |f|)) sum_m sum_{F(f,m)} omega_m w_k I,  F_f = (1/|f|) sum omega w Omega I,
 *   N_f = (1/|f|) sum omega w Omega Omega I  (f_f = N_f / (c E_f) is the face tensor of Eq. 16).
 * |f| = hy on x-faces, hx on y-faces.  Faces: x-face (i, j) on the line x = x0 + i hx in row j is number
 * j (nx + 1) + i; y-face (i, j) on y = y0 + j hy in column i is (nx + 1) ny + j nx + i.  A segment entering
 * through a vertex counts on the x-face of the cell it enters.  I: the state the sweep used (for its scale);
 * out: device, each [G][n_faces] FP64.  Not produced by molc_batch_sweep. */
molc_status molc_face_moments(const molc_plan *plan, molc_precision prec, const void *I, double c,
                              const molc_moments *out, molc_stream stream);

/* Spectrum-averaged coefficients of the effective grey problem (Sec. 2, Eqs. 8-9), per cell from the group
 * moments and opacities:
 *   out[0] = <kappa>_E = sum_g kappa_g E_g / sum_g E_g,
 *   out[1] = <kappa>_B = sum_g kappa_g B_g / sum_g B_g (the emission average of the grey energy balance, Eq. 6),
 *   out[2], out[3] = K_R = diag(<kappa>_|Fx|, <kappa>_|Fy|), <u>_|Fa| = sum_g u_g |F_a,g| / sum_g |F_a,g|,
 *   out[4], out[5] = eta = sum_g (kappa_g - K_R) F_g / sum_g E_g (x and y components).
 * m: device moments [G][cell] (E, Fx, Fy used); kappa, B: device [G][cell]; out: device [6][cell] FP64.  A
 * cell whose denominator is zero gets 0.  Asynchronous on `stream`. */
molc_status molc_grey_coefficients(const molc_plan *plan, const molc_moments *m, const double *kappa,
                                   const double *B, double *out, molc_stream stream);

/* Canonical intensity layout: [n_segments][g_count] FP64 segment averages (Ibar of Eq. 12), direction-major in
 * quadrature order; within a direction, characteristics by increasing offset along (-sin phi, cos phi) and segments
 * in traversal order. export: canon := I (groups g_begin .. g_begin+g_count-1). import: I := canon for the same
 * groups, with B (device [G][cell]) as the new reference Planck intensity of those groups. Device memory. */
molc_status molc_intensity_export(const molc_plan *plan, molc_precision prec, const void *I, int g_begin,
                                  int g_count, double *canon, molc_stream stream);
molc_status molc_intensity_import(molc_plan *plan, molc_precision prec, void *I, int g_begin, int g_count,
                                  const double *canon, const double *B, molc_stream stream);

/* The characteristic grid of Sec. 3 in the canonical order (host arrays): dir_ray_off[n_dir+1],
 * ray_seg_off[rays+1], width[rays], entry[rays] (edge 0..3), cell[n_segments], len[n_segments] (in-plane l),
 * area[n_segments] (A after renormalisation). rays = 2 n_polar n_tracks. */
molc_status molc_tracks_export(const molc_plan *plan, int64_t *dir_ray_off, int64_t *ray_seg_off, double *width,
                               int *entry, int *cell, double *len, double *area);

/* Kernel timing for benchmarks (no counterpart in the paper): while enabled, every molc_sweep records CUDA events
 * around its three kernels (input preparation, the sweep itself, the cell moments; at most 4096 calls are kept).
 * molc_kernel_time synchronises with the last recorded event, returns the summed elapsed milliseconds of the sweep
 * kernel and the number of timed calls, and clears the record; molc_kernel_time_parts does the same with
 * parts_ms[3] = {preparation, sweep, moments}. Disabled by default; enabling creates the events (no device memory
 * allocation). */
molc_status molc_kernel_timing(molc_plan *plan, int enable);
molc_status molc_kernel_time(molc_plan *plan, double *total_ms, int *launches);
molc_status molc_kernel_time_parts(molc_plan *plan, double *parts_ms, int *launches);

/* Re-cut the tiled FP32 sweep of a plan (one created without MOLC_FACES / MOLC_BALANCE and with at most 8 polar
 * cosines) with the given configuration, replacing its device tables (no counterpart in the paper).  The FP32
 * intensity layout changes with the configuration: states made for the old one must be re-initialised
 * (molc_intensity_init) or re-imported, and batches of the plan re-created.  Synchronises with the device.
 * MOLC_ERR_INVALID_ARG if the configuration does not fit a block's shared memory (the plan then keeps the
 * library's default configuration). */
molc_status molc_plan_retile(molc_plan *plan, const molc_tile_config *cfg);

/* Tuning cache of MOLC_AUTOTUNE (no counterpart in the paper), process-wide: from this call on, molc_create with
 * MOLC_AUTOTUNE first looks the plan up in the JSON file `path` (host path, read during the call; later plans
 * reread and rewrite it).  An entry for the same plan signature (grid, directions, groups, ray spacing, layout
 * and the flags that change the sweep), the same kind of device (name, SM count, compute capability) and the same
 * library build is applied without timing (molc_plan_info.tuned_from_cache = 1); otherwise the plan is tuned and
 * its entry added, the file rewritten whole through a temporary file and a rename (a file that cannot be
 * written leaves the plan tuned and the file unchanged).  The file need not exist.  path = NULL or "" switches the
 * cache off.  *n_entries (may be NULL) receives the number of entries read.  MOLC_ERR_INVALID_ARG, with the
 * earlier setting kept, if the file exists but cannot be read or is not a cache this library wrote. */
molc_status molc_tune_cache(const char *path, int *n_entries);

/* FP64 fused multiply-add throughput of the current device, in FLOP/s (2 per FMA): the bound of the plain FP64
 * sweep's arithmetic (no counterpart in the paper; a measurement for the roofline).  Runs a kernel of independent
 * FMA chains on every SM four times (the first as warm-up) on the legacy default stream, timed with CUDA events;
 * synchronises with the device.  No device memory is allocated. */
molc_status molc_fp64_fma_rate(double *flops_per_s);

/* Read and clear the plan's device status word (error reporting, no counterpart in the paper; synchronises with the
 * device). *code = MOLC_OK or the first error the kernels recorded. */
molc_status molc_device_status(molc_plan *plan, int *code);

/* Message of the last failure on the calling thread ("" if none; no counterpart in the paper). */
const char *molc_last_error(void);

/* Frees the plan and its device memory (no counterpart in the paper). */
void molc_destroy(molc_plan *plan);

#ifdef __cplusplus
}
#endif
#endif /* MOLC_H */
