/*
 * vpmc.h -- C ABI of the GB300-native aperture-aware proton Monte Carlo engine.
 *
 * The engine transports independent proton histories (one identical model
 * per history, paper Sec. 2.A) through an optional range shifter and a brass
 * aperture block (Sec. 2.B: 30 mm brass; in the aperture slab a
 * crossing-number test decides at every step whether the particle is in the
 * opening -- straight flight -- or in brass -- brass physics) and a voxelised
 * CT grid, and scores deposited energy into a dose grid or into per-spot
 * influence-matrix columns (Sec. 2.C, sparse matrices) for robust scenarios
 * (Sec. 2.E: stopping-power-ratio scaling and isocentre shifts).
 *
 * Conventions for every entry point:
 *   - Units: mm, MeV, mrad for spot divergence; coordinates are the CT
 *     grid's (patient) frame.  Grids are x-fastest.
 *   - The caller owns every input; the library copies geometry, polygons,
 *     spots and scenarios during the call, so they may be freed on return.
 *   - Device work is enqueued on the context's CUDA stream.  Calls that return
 *     sizes or statistics synchronise that stream; the others are
 *     asynchronous (documented per call).
 *   - Errors: a vpmc_status is returned and a message is kept per thread
 *     (vpmc_last_error).  No C++ exception crosses this boundary.  A kernel
 *     that meets an inconsistent state (iteration cap of a history, box
 *     overflow) records it in a device status word that the host reads.
 *   - Nothing here allocates memory that the caller must free, except the
 *     CSR buffers of vpmc_influence_matrix (vpmc_free_csr), unless the caller
 *     supplies their allocator (vpmc_set_csr_allocator).
 */
#ifndef VPMC_H
#define VPMC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct vpmc_ctx vpmc_ctx; /* opaque; one per (CUDA device, stream, CT) */

typedef enum {
    VPMC_OK = 0,
    VPMC_ERR_ARG = -1,         /* invalid argument (message says which)       */
    VPMC_ERR_CUDA = -2,        /* a CUDA runtime call failed                  */
    VPMC_ERR_OOM = -3,         /* device memory exhausted                     */
    VPMC_ERR_TIMEOUT = -4,     /* a history reached the iteration cap         */
    VPMC_ERR_STATE = -5,       /* call out of order (e.g. beam not set)       */
    VPMC_ERR_DEVICE_FLAG = -6  /* a kernel latched an error in its status word */
} vpmc_status;

/* Four-segment piecewise-linear HU -> (mass density g/cc, stopping-power
 * ratio to water) curve: 5 knots, HU ascending.  HU is clamped to
 * [hu[0], 3071]; above hu[4] the last segment is extended. */
typedef struct { double hu[5], density[5], spr[5]; } vpmc_hu_curve;

/* Regular grid: n voxels per axis of size d (mm); origin = corner of voxel
 * (0,0,0).  Arrays on it are x-fastest: index = x + nx*(y + ny*z). */
typedef struct { int nx, ny, nz; double dx, dy, dz; double origin[3]; } vpmc_grid;

/* One field (Sec. 2.B, 2.D).  dir = beam axis w (unit), bev_x = first
 * beam's-eye-view axis u (unit, orthogonal to w); second axis v = w x u.
 * Positions along the beam are t (mm) relative to the isocentre, downstream
 * positive; devices are placed by the distance of their downstream face to
 * the isocentre (paper: aperture 150 mm, range shifter 190 mm).  The source
 * plane is t = -source_to_iso_mm and must lie upstream of every device.
 * Range shifter: PMMA slab of water-equivalent thickness rs_wet_mm (geometric
 * thickness = rs_wet_mm / SPR_PMMA(150 MeV)) and radius rs_radius_mm.
 * Aperture: brass block of thickness ap_thickness_mm whose opening is the
 * polygon poly_xy (n_vertices (u, v) pairs in mm, any orientation, simple)
 * at the block's downstream face; at most 4096 vertices over all beams of a
 * context.  ap_sad_mm = 0: walls parallel to the beam axis (Sec. 2.B).
 * ap_sad_mm > 0: divergent walls (the authors' next step, Sec. 4): each wall
 * is the plane through the virtual source at t = -ap_sad_mm on the beam
 * axis and one polygon edge, so the opening at depth t is the polygon
 * scaled by (t + ap_sad_mm) / (t_dn + ap_sad_mm); the source must lie
 * upstream of the block.  The learned aperture surrogate (vpmc_opts.surrogate)
 * is trained on parallel walls and is refused for divergent blocks. */
typedef struct {
    double dir[3], bev_x[3], iso[3];
    double source_to_iso_mm;
    int rs_present;
    double rs_wet_mm, rs_radius_mm, rs_down_to_iso_mm;
    int ap_present;
    double ap_thickness_mm, ap_down_to_iso_mm;
    const double* poly_xy;
    int n_vertices;
    double ap_sad_mm;
} vpmc_beam;

/* One pencil-beam spot (Sec. 2.D.2): mono-energetic (energy_mev <= 250),
 * position (x_mm, y_mm) and Gaussian sigma_mm at the isocentre plane in BEV
 * coordinates, per-plane angular sigma div_mrad, n_hist histories (< 2^32).
 * weight multiplies every deposit of the spot in vpmc_run_spots (dose per
 * history x weight); vpmc_influence_matrix ignores it. */
typedef struct {
    int beam;
    double energy_mev, x_mm, y_mm, sigma_mm, div_mrad;
    int64_t n_hist;
    double weight;
} vpmc_spot;

/* Robust scenario (Sec. 2.E): isocentre shift (patient frame) and SPR scale. */
typedef struct { double shift_mm[3]; double spr_scale; } vpmc_scenario;

/* Per-history record (optional output of vpmc_run_spots). */
typedef struct {
    int64_t q_dep;    /* fixed-point sum of the history's grid deposits (2^-frac_bits MeV) */
    int32_t fate;     /* 0 stopped, 1 nuclear, 2 left the grid / missed, 3 absorbed in range
                         shifter, 4 absorbed in aperture, 5 iteration cap reached */
    int32_t steps;    /* condensed-history steps */
    float e_dep;      /* energy scored in the grid, MeV */
    float e_end;      /* kinetic energy when it left the simulation, MeV */
    float pos[3];     /* end position, patient frame, mm */
    float pad;
} vpmc_history_record;

typedef struct {
    uint64_t seed;          /* Philox key: (seed low word, spot index ^ seed high word)  */
    int mcs;                /* Highland multiple scattering on/off                        */
    int straggling;         /* Bohr straggling on/off                                     */
    int nuclear;            /* nuclear removal (1.2 %/cm x density) on/off                */
    int frac_bits;          /* fixed-point scale of deposits, 2^-frac_bits MeV (default 24) */
    /* Autotuned launch: the first dose (or influence-matrix) call of a
     * context times a few launch configurations on a sample of its
     * histories (up to 24 per thread of the largest block, about 3.3e6 on
     * 152 SMs); the choice is kept by the context and, for later contexts
     * on the same device with the same grids, field devices and fixed launch
     * options, by the process.  Results do not depend on the choice. */
    int aggregate;          /* -1 autotuned, 0 plain atomics, 1 warp-aggregated atomics   */
    int block_size;         /* 0 autotuned, else patient-kernel threads per block (multiple of 32, <= 896) */
    int blocks_per_sm;      /* 0 autotuned                                                */
    int chunk;              /* histories taken per warp refill (0 = default)              */
    vpmc_history_record* history_out;  /* device buffer or NULL                          */
    int64_t history_cap;    /* records for global history index < history_cap            */
    int range_rejection;    /* 1 (default): a brass proton whose longest possible remaining
                               path (1.2 x residual CSDA range) cannot reach the opening or
                               a face of the block is absorbed at once; the patient sees the
                               same histories either way                                 */
    int surrogate;          /* 0 (default): plain aperture transport.  1: each proton that
                               enters the brass within the learned surrogate's training
                               domain takes one network draw for its state on the block's
                               exit plane instead of condensed-history stepping (needs
                               vpmc_surrogate_set_weights or _train first); the others
                               use the plain path                                         */
    int64_t timeout_iters;  /* iterations a history may take in each transport kernel before
                               it is stopped as an error (0 = default 200,000; at most
                               2^31 - 1).  A history that reaches it ends with fate 5, its
                               remaining energy goes to e_leak, and the kernel latches bit 0
                               of the device status word: the call (or, for an asynchronous
                               call, the next call on the context) returns VPMC_ERR_TIMEOUT */
} vpmc_opts;

/* Totals of one call.  Energies in MeV (fixed-point sums, unweighted). */
typedef struct {
    int64_t histories, steps, errors;
    double e_in, e_dep, e_leak, e_rs, e_aperture, e_nuc;
    float ms;               /* device time of the transport launch(es), CUDA events */
    int64_t launches;       /* kernels this call launched (autotuning included) */
    int64_t ovf_records;    /* influence matrix: deposits outside their column's dense box */
    int64_t steps_rs;       /* condensed-history steps in the range shifter (included in steps) */
    int64_t steps_aperture; /* condensed-history steps in the brass block (included in steps) */
    float ms_devices;       /* device time of the beam-line kernels (source, range shifter, aperture,
                               surrogate draws) within ms, CUDA events; 0 for vpmc_run_spots_noalloc */
    float ms_patient;       /* device time of the patient kernel within ms, CUDA events; 0 for
                               vpmc_run_spots_noalloc */
    int64_t scratch_bytes;  /* influence matrix: dense column scratch the call filled, summed over its
                               waves (each byte is zeroed once and read three times to build the CSR) */
} vpmc_stats;

/* Sparse influence matrix of one scenario: rows = scoring voxels (x-fastest),
 * columns = spot indices; row_ptr int64[n_rows+1], col int32[nnz] sorted
 * within each row, val float32[nnz] = dose per primary proton (Gy).  All three
 * buffers are device memory allocated by the library. */
typedef struct {
    int64_t n_rows, n_cols, nnz;
    int64_t* row_ptr;
    int32_t* col;
    float* val;
} vpmc_csr;

/* Fill opts with defaults: seed 1234, all physics on, frac_bits 24,
 * autotuned launch, no records, brass range rejection on, iteration cap
 * 200,000. */
void vpmc_default_opts(vpmc_opts* opts);

/* Create a context (Sec. 2.A physics tables; Sec. 2.D.3 patient CT).
 * hu: int16 CT on ct's grid, host pointer (hu_on_device = 0) or device
 * pointer of the current device (hu_on_device = 1); copied.  dose_grid: the
 * scoring grid; it must have the CT's origin and extent (its voxel size may
 * differ); dose is dose-to-medium with the volume-weighted mean density of
 * the overlapping CT voxels.  cuda_stream: a cudaStream_t (NULL = legacy
 * default stream).  Builds the stopping-power/range tables (Bethe-Bloch,
 * FP64 on the host, stored FP32), the HU lookup table and the scoring-voxel
 * densities; synchronises the stream.  On error *out is NULL. */
vpmc_status vpmc_create_geometry(vpmc_ctx** out, const int16_t* hu, int hu_on_device, const vpmc_grid* ct,
                                 const vpmc_hu_curve* curve, const vpmc_grid* dose_grid, void* cuda_stream);

/* Set beam entry beam_id (0..63) (Sec. 2.B: range shifter and aperture
 * geometry, crossing-number opening).  Copies the polygon and builds its BEV
 * classification raster.  Synchronous.  An energy-layer-specific (dynamic)
 * aperture (the authors' future work, Sec. 4) is one entry per (field,
 * energy layer): the same field geometry with that layer's opening, the
 * layer's spots referring to it; spots must be sorted by entry for
 * vpmc_influence_matrix.  VPMC_ERR_ARG (the entry keeps its previous state)
 * for dir and bev_x not orthonormal, a polygon of fewer than 3 vertices, a
 * non-finite vertex, or one that is not simple: two edges that are not
 * neighbours touch or cross, or two neighbouring edges overlap or a vertex
 * repeats. */
vpmc_status vpmc_set_aperture(vpmc_ctx* ctx, int beam_id, const vpmc_beam* beam);

/* Dose of a set of spots in one scenario (Sec. 2.C, 2.D): transports every
 * history, accumulates 64-bit fixed-point sums and writes dose_dev (device
 * float32 array on the scoring grid, caller-owned) = sum over deposits of
 * dE * weight / (rho * V) in Gy.  scen may be NULL (nominal).  Asynchronous
 * on the context stream unless stats_out is non-NULL, in which case it
 * synchronises, fills the totals and returns VPMC_ERR_TIMEOUT or
 * VPMC_ERR_DEVICE_FLAG when a kernel latched its status word.  An
 * asynchronous call leaves that word to the next call on the context, which
 * first waits for the earlier call's work and, if the word is set, returns
 * that error without running (the earlier call's dose is then not valid).
 * Spot errors: VPMC_ERR_STATE for a beam id that was not set,
 * VPMC_ERR_ARG for an energy outside (0.5, 250] MeV (NaN included), n_hist
 * outside [0, 2^32), a negative or non-finite sigma, divergence or weight. */
vpmc_status vpmc_run_spots(vpmc_ctx* ctx, const vpmc_spot* spots, int n_spots, const vpmc_scenario* scen,
                           const vpmc_opts* opts, float* dose_dev, vpmc_stats* stats_out);

/* The dose of vpmc_run_spots computed without allocating any memory in the
 * call.  The paper has no counterpart: this serves callers that cannot let a
 * call allocate device memory -- serving loops where the implicit
 * device-wide synchronisation of cudaMalloc/cudaFree would stall other
 * streams, and hosts whose memory pool owns all device memory.  The context
 * (vpmc_create_geometry, vpmc_set_aperture) must already exist; it is the
 * only allocation, made once at set-up.  Scratch (64-bit accumulator, work
 * items, beam-line hand-off buffer, counters, status word) lives in one fixed
 * device array of about 29 MiB that every GPU loading the library holds until
 * the process exits; its limits are 2,097,152 scoring voxels and 16,384 spots
 * with histories per call (VPMC_ERR_ARG beyond them).  The first call on a
 * device resolves that array's device address (cudaGetSymbolAddress).  All
 * calls on a device share the array and clear it at their start: calls that
 * overlap on the GPU (other streams, other threads) race and corrupt each
 * other.  The work list is copied from host stack memory during the call, so
 * a stream that is capturing is refused (VPMC_ERR_STATE).  Arguments, output
 * and the status rules (stats_out, and the latched status word read by the
 * next call on the same device) are those of vpmc_run_spots, with the plain
 * aperture only (opts->surrogate = 1 is VPMC_ERR_ARG); the launch
 * configuration is the context's tuned one (or opts') without autotuning. */
vpmc_status vpmc_run_spots_noalloc(vpmc_ctx* ctx, const vpmc_spot* spots, int n_spots, const vpmc_scenario* scen,
                                   const vpmc_opts* opts, float* dose_dev, vpmc_stats* stats_out);

/* Influence matrices for n_scen scenarios (Sec. 2.C sparse matrices, Sec.
 * 2.E 13 robust scenarios): every (scenario, spot) column in one persistent
 * launch, unweighted; column j of scenario s = dose per primary of spot j;
 * entries below rel_threshold x the column maximum are dropped.  Spots must
 * be sorted by beam id.  out: array of n_scen vpmc_csr filled with
 * library-allocated device buffers (free with vpmc_free_csr).  Synchronous. */
vpmc_status vpmc_influence_matrix(vpmc_ctx* ctx, const vpmc_spot* spots, int n_spots, const vpmc_scenario* scen,
                                  int n_scen, const vpmc_opts* opts, float rel_threshold, vpmc_csr* out,
                                  vpmc_stats* stats_out);

/* Free the device buffers of n CSR matrices and zero the structs.  Only for
 * buffers the library allocated (no allocator set with
 * vpmc_set_csr_allocator when they were made). */
vpmc_status vpmc_free_csr(vpmc_csr* csr, int n);

/* Allocator of the CSR buffers vpmc_influence_matrix returns: alloc(bytes,
 * user) returns device memory of the context's device, at least 16-byte
 * aligned, or NULL (the call then fails with VPMC_ERR_OOM).  It is called on
 * the calling thread during vpmc_influence_matrix, three times per scenario
 * (row_ptr, col, val; never with bytes = 0), and what it returns belongs to
 * the caller: the library never frees it, also when the call fails, and
 * vpmc_free_csr must not be used on it.  alloc = NULL restores allocation by
 * the library.  Lets a caller take the matrices in its own memory pool
 * without a copy and without device-wide allocation calls in the loop.
 * VPMC_ERR_ARG: ctx NULL. */
typedef void* (*vpmc_alloc_fn)(size_t bytes, void* user);
vpmc_status vpmc_set_csr_allocator(vpmc_ctx* ctx, vpmc_alloc_fn alloc, void* user);

/* ------------------------------------------------------------------------
 * Learned aperture surrogate.  The paper has no counterpart: its aperture
 * module (Sec. 2.B) reads the brass block's effect from pre-computed brass
 * transport.  Here a small network, trained on tracks of this library's own
 * plain aperture transport, draws the state of a proton that enters the
 * brass near the opening on the block's exit plane in one step.
 *
 * Network: 6 inputs -> 128 -> 128 (ReLU) -> 45 outputs.  Outputs: a
 * transmission logit, then a 4-component diagonal Gaussian mixture over five
 * exit quantities (mixture logits [4], means [4 x 5], log widths [4 x 5]).
 * Weights and activations are BF16, sums FP32, on the tensor cores.
 * Parameters: VPMC_SUR_NPARAMS FP32 values, row-major (outputs x inputs):
 * W1 [128 x 6], b1 [128], W2 [128 x 128], b2 [128], W3 [45 x 128], b3 [45].
 *
 * Inputs of a proton at (x, y) on the block's entrance plane, with direction d
 * and energy E.  n is the unit vector from the nearest boundary point of the
 * opening to the proton; t = (-n_y, n_x).
 *   x0 = min(dist, 12 mm) / 6 mm - 1
 *   x1 = (E - 135 MeV) / 95 MeV
 *   x2 = (d . n) / 0.04,  x3 = (d . t) / 0.04
 *   x4 = 8 mm x (boundary curvature there) - 1
 *   x5 = (brass CSDA range of E) / (block thickness) - 1
 * Targets of a transmitted proton:
 *   y0 = 5 (E_in - E_out) / E_in
 *   y1 = (exit - entry) . n - T (d_in . n) / d_in,z
 *   y2 = (exit - entry) . t - T (d_in . t) / d_in,z
 *   y3 = (d_out - d_in) . n / 0.05,  y4 = (d_out - d_in) . t / 0.05
 * Training domain: E in [40, 230] MeV, |d . n| and |d . t| <= 0.12,
 * curvature in [-0.001, 0.26] / mm, block thickness 30 mm, and |x5| >= 0.06
 * (away from the stopping threshold, where the exit energy has a sharp
 * edge that the mixture does not follow).  Only beams with a range shifter
 * use the network: without one, the nearly parallel, mono-energetic beam
 * makes the few protons that escape through the wall stand out, and the
 * network's dose error there exceeded 1 % of the maximum.  With
 * opts->surrogate = 1, a brass entry outside this domain takes the plain
 * path.  A brass entry whose 1.2 x CSDA range is below both its edge distance
 * and the thickness is absorbed without a draw.
 * ------------------------------------------------------------------------ */
#define VPMC_SUR_NPARAMS 23213

/* Load the network's parameters (host array of VPMC_SUR_NPARAMS floats,
 * copied) and reset the Adam state.  Synchronous. */
vpmc_status vpmc_surrogate_set_weights(vpmc_ctx* ctx, const float* params);

/* Fresh parameters: He-normal weights (the output layer scaled by 0.1 / sqrt 2),
 * zero biases, from a seeded generator on the host.  Resets the Adam state.
 * Synchronous. */
vpmc_status vpmc_surrogate_init(vpmc_ctx* ctx, uint64_t seed);

/* Copy the current parameters to a host array of VPMC_SUR_NPARAMS floats. */
vpmc_status vpmc_surrogate_get_weights(vpmc_ctx* ctx, float* params);

/* Training or evaluation tracks.  Each beam_ids[g] must be set, with an
 * aperture and no range shifter.  tracks_per_beam histories per beam start on
 * its entrance plane near the opening.  Track h of list entry g is global
 * index i = g * tracks_per_beam + h, with Philox key (seed low word,
 * g ^ seed high word).  Its start, from counter (h, 0, slot, 0):
 *   slot 0: E = 40 + 190 u0 MeV, angle phi = 2 pi u1, edge distance d = d_hi u2^2,
 *           where d_hi = min(12 mm, 1.2 R) if 1.2 x brass CSDA range R is
 *           below the thickness, else 12 mm; the proton starts at radius
 *           r_c + d at angle phi, r_c the largest vertex radius;
 *   slot 5: incidence direction cosines along the radial and tangential
 *           directions, 0.04 x (first Box-Muller pair), clamped to +-0.12;
 *   slot 3: the nuclear free path.
 * Outputs are caller-owned device arrays of n = n_beams x tracks_per_beam
 * rows: feat_dev [n x 6] (inputs), target_dev [n x 5] (targets, zero unless
 * transmitted), label_dev [n] (1: left through the exit plane).
 * use_surrogate = 0: the plain aperture transport with opts' physics.
 * use_surrogate = 1: one network draw per track (Philox slots 4 and 5 at the
 * entry step); the targets are the drawn ones.  Synchronous. */
vpmc_status vpmc_surrogate_tracks(vpmc_ctx* ctx, const int* beam_ids, int n_beams, int64_t tracks_per_beam,
                                  const vpmc_opts* opts, int use_surrogate, float* feat_dev, float* target_dev,
                                  int32_t* label_dev);

/* Network outputs for n input rows.  feat_dev: [n x 6] device.
 * z_dev: [n x 45] device, caller-owned.  Both 16-byte aligned (VPMC_ERR_ARG
 * otherwise): a tile's rows are moved in 16-byte pieces.  Synchronous. */
vpmc_status vpmc_surrogate_forward(vpmc_ctx* ctx, const float* feat_dev, int64_t n, float* z_dev);

/* Mean loss over n tracks at the current parameters, and its gradient.
 * Loss of one track: softplus(z0) - label z0, plus (label = 1 only) the
 * mixture's negative log-likelihood of its targets.  grad_dev: device array
 * of VPMC_SUR_NPARAMS floats, parameter order.  Synchronous. */
vpmc_status vpmc_surrogate_gradient(vpmc_ctx* ctx, const float* feat_dev, const float* target_dev,
                                    const int32_t* label_dev, int64_t n, float* grad_dev, double* loss);

/* Adam training (beta 0.9 / 0.999, eps 1e-8) over n tracks: minibatches of
 * `batch` rows, `epochs` passes, each in its own batch order.  Learning rate
 * follows a cosine from lr to lr_min over all steps.  epoch_loss: optional
 * host array [epochs], the mean loss of each pass.  A pass whose loss is not
 * finite stops the training with VPMC_ERR_STATE (the parameters are then
 * not usable).  Synchronous. */
vpmc_status vpmc_surrogate_train(vpmc_ctx* ctx, const float* feat_dev, const float* target_dev,
                                 const int32_t* label_dev, int64_t n, int batch, int epochs, float lr, float lr_min,
                                 float* epoch_loss);

/* ------------------------------------------------------------------------
 * Robust spot-weight optimisation over the scenarios' influence matrices
 * (Sec. 2.E: robust optimisation over 13 scenarios, evaluated by the target
 * indices of Table 3).  The paper's optimiser is an in-house trial-and-error
 * procedure; this one minimises the worst case over the scenarios of
 *   f(d) = w_under/|T| sum_T max(0, D_p - d)^2 + w_over/|T| sum_T max(0, d - over_frac D_p)^2
 *        + w_ring/|R| sum_R max(0, d - ring_frac D_p)^2,      d = A_s x,
 * with Adam on the spot weights x, clamped at zero after each step.
 * T and R are the voxels of class 1 (target) and 2 (ring).
 * ------------------------------------------------------------------------ */
typedef struct {
    float prescription;     /* D_p, in the matrices' dose units x weight units */
    float w_under, w_over, w_ring;
    float over_frac;        /* target overdose above over_frac * D_p */
    float ring_frac;        /* ring overdose above ring_frac * D_p */
    float lr;               /* Adam step, in units of the mean initial weight */
    int iterations;
} vpmc_opt_params;

/* mats: n_scen CSR (device buffers, e.g. from vpmc_influence_matrix), all of
 * the same shape, at most 28,000 columns and 2^31 - 1 rows; row_ptr must be
 * non-decreasing from 0 to nnz (not checked); entries whose column lies
 * outside [0, n_cols) are skipped.  voxel_class_dev: uint8 [n_rows], device
 * (1 target, 2 ring, other values ignored; at least one target voxel).
 * x_dev: float [n_cols], device: the initial weights (finite, >= 0) in, the
 * optimised weights out.  history: optional host float [iterations], the
 * worst-case objective before each step.  ms: optional host float [2]: device
 * time of the iterations, then of the setup (CUDA events).  stream: a
 * cudaStream_t (NULL = legacy default).
 * Only target and ring voxels enter the objective, so the call first copies
 * their rows of every matrix into a compact form (scratch of about 6 bytes
 * per such entry, allocated and freed by the call), then iterates on those.
 * The gradient is summed in 64-bit fixed point, so repeated calls with the
 * same inputs give the same bits.  Synchronous. */
vpmc_status vpmc_robust_optimize(const vpmc_csr* mats, int n_scen, const uint8_t* voxel_class_dev,
                                 const vpmc_opt_params* params, float* x_dev, float* history, float* ms,
                                 void* stream);

/* dose_dev[i] = sum_j A_ij x_j for one CSR matrix (device float
 * [n_rows], caller-owned): the dose of the weights x.  Synchronous. */
vpmc_status vpmc_weights_dose(const vpmc_csr* mat, const float* x_dev, float* dose_dev, void* stream);

/* Target indices (Table 3) of the dose A_s x of each scenario:
 *   out[4 s + 0] V100 (fraction of T with d >= D_p)
 *   out[4 s + 1] min_T d / D_p
 *   out[4 s + 2] CI100 = |{d >= D_p}| / |T|
 *   out[4 s + 3] RHI100 = max_T d / D_p
 * out is a host array.  Synchronous. */
vpmc_status vpmc_target_indices(const vpmc_csr* mats, int n_scen, const uint8_t* voxel_class_dev,
                                float prescription, const float* x_dev, double* out, void* stream);

/* ------------------------------------------------------------------------
 * Measurement.  The paper has no counterpart.
 * ------------------------------------------------------------------------ */

/* The current device's rate of 64-bit atomic adds resolved in L2: the
 * secondary bound of the transport's scoring, which adds each
 * condensed-history step's fixed-point deposit to a voxel with one such add.
 * 4 x SMs blocks of 1024 threads each make `iters` adds of 1 to entries of a
 * device buffer of n_entries 64-bit words (a power of two in [32, 2^26];
 * 2^22 words, 32 MiB, stay in L2), chosen by a hash of (thread, iteration),
 * results unused.  One untimed pass, then a timed one between CUDA events
 * on `stream` (a cudaStream_t, NULL = legacy default).  Outputs: adds_per_s
 * (timed pass), adds_out (adds of the timed pass) and sum_out (the buffer's
 * sum after both passes: 2 x adds_out when every add landed); the last two
 * may be NULL.  The call allocates and frees its buffer.  Synchronous. */
vpmc_status vpmc_measure_l2_atomics(int64_t n_entries, int iters, double* adds_per_s, int64_t* adds_out,
                                    int64_t* sum_out, void* stream);

/* Destroy a context and free its device memory. */
void vpmc_destroy(vpmc_ctx* ctx);

/* Message of the last error raised on the calling thread ("" if none). */
const char* vpmc_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* VPMC_H */
