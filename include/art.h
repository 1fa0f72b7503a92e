/*
 * art.h -- C ABI of libart, a GB300 (sm_103a) implementation of the diffuse
 * radiation ray-tracing scheme of Tanaka, Yoshikawa, Okamoto & Hasegawa (2014),
 * "A new ray-tracing scheme for 3D diffuse radiation transfer on highly
 * parallel architectures" (PASJ), and of the photo-ionization iteration it
 * drives.
 *
 * Conventions shared by every entry point:
 *   - Fields are 3D arrays of nz * ny * nx cells, x fastest ([z][y][x]); with
 *     nu_bins > 1 the bin index is outermost ([bin][z][y][x]).  Lengths inside
 *     the library are in cell widths, so kappa is the absorption coefficient
 *     times the cell width (optical depth per cell width).
 *   - The caller owns every input and output buffer.  The context owns its
 *     device memory (field copies in sweep-axis layouts, ray-plane buffers,
 *     per-class J partials, tables).  Nothing is retained from caller buffers
 *     after a call returns, except that device-pointer inputs are read
 *     stream-ordered on the given stream: keep them alive until that stream
 *     has been synchronized.
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *     stream).  Calls that take host buffers synchronize that stream before
 *     returning; calls on device buffers return without synchronizing.
 *   - Every call returns an art_status and never aborts; the text of the last
 *     error of a context is available from art_last_error().  A context is not
 *     thread-safe; separate contexts are independent.
 *   - Floating-point buffers are float (4 bytes) for ART_FP32 contexts and
 *     double (8 bytes) for ART_FP64 contexts.
 */
#ifndef ART_H
#define ART_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct art_ctx art_ctx;

typedef enum {
    ART_OK = 0,
    ART_E_INVALID = 1,        /* bad argument or input value */
    ART_E_CUDA = 2,           /* a CUDA call failed (message names it) */
    ART_E_OOM = 3,            /* device or host allocation failed */
    ART_E_NOT_CONVERGED = 4,  /* iteration hit max_iter before tol */
    ART_E_TIMEOUT = 5,        /* a bounded device wait gave up */
    ART_E_STATE = 6           /* call out of order (e.g. sweep before fields) */
} art_status;

enum { ART_FP32 = 0, ART_FP64 = 1 };
/* ART_AVG_PAPER: Eq. (path_averaged_intensity): the cell average of the
 * incoming intensity, J = J^in + S (Eq. mean_intensity).
 * ART_AVG_EXACT: the exact path average of I over each segment,
 * S + (I_in - S) phi(dtau), in place of the paper's I_in phi + S, which
 * counts the local emission as absorbed locally and also propagates it.
 * J = S + (1/N_d) sum_n <(I_in - S) phi> and J^in = J - S (with emissivity
 * inputs, J^in = J where kappa = 0).  Gamma stays 4 pi sum_b G_b J^in_b. */
enum { ART_AVG_PAPER = 0, ART_AVG_EXACT = 1 };
/* ART_FIELDS_S: inputs are (kappa, S), Eq. (rt).  ART_FIELDS_EPS: inputs are
 * (kappa, eps) with eps the emissivity times the cell width (S = eps/kappa);
 * kappa = 0 is then allowed and the transfer step adds eps * ds. */
enum { ART_FIELDS_S = 0, ART_FIELDS_EPS = 1 };

typedef struct {
    int nx, ny, nz;   /* cells per axis, each >= 1 */
    double dx_cm;     /* cell width in cm (used by the ionization side only) */
} art_grid;

typedef struct {
    int precision;    /* ART_FP32 (default) or ART_FP64 */
    int averaging;    /* ART_AVG_PAPER (default) or ART_AVG_EXACT */
    int field_form;   /* ART_FIELDS_S (default) or ART_FIELDS_EPS */
    int tile_b;       /* ray-plane tile along the fastest transverse axis; 0 = auto */
    int tile_c;       /* ray-plane tile along the other transverse axis;  0 = auto */
    int slab;         /* slabs per launch along the sweep axis;           0 = auto */
    int dir_split;    /* direction groups per octant class (J partials);  0 = auto */
    double tie_tol;   /* dominant-axis tie tolerance (relative), default 1e-12 */
    int variant;      /* sweep-kernel variant (1-based index of the compiled table); 0 = auto */
    int persistent;   /* slab-block launches as a fixed grid of CTAs taking work items
                         from a queue: 1 = on, -1 = off, 0 = auto (on for batches) */
    int graph;        /* 1: art_sweep replays the launches of one sweep as a CUDA graph
                         (captured on the first call and again whenever the output
                         pointers, band integrals or variant change); 0 = plain launches */
    int dir_begin, dir_end;  /* direction shard: sweep only RING indices [dir_begin, dir_end)
                                (single-grid contexts); 0, 0 = all directions.  J_in and
                                gamma are then this shard's additive share (still divided by
                                the full N_d), and the J output is not available */
    int early_launch;        /* slab-block launches after the first of a sweep may start while
                                the previous one drains (programmatic dependent launch): they
                                stage fields and tables, then wait before touching the
                                intensity planes.  1 or 0 = on (default), -1 = off */
} art_options;

/* Statistics of one sweep, fixed at art_create. */
typedef struct {
    int64_t segments;        /* exact number of (ray, cell) pairs with ds > 0, all bins */
    int32_t n_dirs;          /* 12 N_side^2 */
    int32_t n_classes;       /* non-empty (dominant axis, octant) classes */
    int32_t launches;        /* kernel launches per sweep and bin (sweep + reduce); a sweep launch
                                covers bins_per_launch bins */
    int32_t ctas_per_launch; /* CTAs of one slab-block launch */
    int32_t tile_b, tile_c, slab, dir_split;
    int64_t device_bytes;    /* device memory owned by the context */
    int32_t variant;         /* sweep-kernel variant in use (1-based) */
    int32_t group;           /* directions processed per exchange barrier */
    int32_t n_grids;         /* grids in the context (1 outside batches) */
    int32_t work_items;      /* (class, tile, direction group) items per slab-block launch */
    int32_t persistent;      /* 1 if launches take work items from a queue */
    int32_t bins_per_launch; /* bins one sweep launch covers: the wavefront sweep takes all bins
                                in one launch when their buffers fit in a quarter of the free
                                device memory at setup (at most 8), else 1 */
} art_sweep_stats;

/* Fill `opt` with defaults (FP32, paper averaging, (kappa, S) inputs, auto
 * tiles, tie_tol 1e-12).  Never fails for a non-NULL pointer. */
art_status art_options_default(art_options *opt);

/*
 * Create a context for one grid, angular resolution and number of frequency
 * bins.  Directions are the 12 n_side^2 HEALPix pixel centres (Sec. 2.3,
 * Gorski et al. 2005, RING order); each is swept by the family of parallel
 * rays of Sec. 2.2 (Fig. parallel_ray): lines spaced one cell width apart on
 * planes normal to the direction's dominant axis, through cell centres.
 * Allocates all device memory of the sweep.  Errors: ART_E_INVALID (dims < 1,
 * n_side < 1, nu_bins < 1, bad options), ART_E_OOM, ART_E_CUDA.
 * On success *out owns the context; release it with art_destroy().
 */
art_status art_create(const art_grid *grid, int n_side, int nu_bins, const art_options *opt,
                      art_ctx **out);

/*
 * Create a context for a batch of n_grids independent grids (the many-problem
 * mode: e.g. several sub-volumes or snapshots solved together).  grids[g] and
 * n_side[g] give each grid's cells and angular resolution; grids may differ in
 * both.  One sweep covers every grid: each slab-block launch carries the work
 * items (direction class x ray-plane tile x direction group) of all grids, so
 * small grids fill the GPU together.  Field and output arrays are the grids'
 * [bin][z][y][x] arrays concatenated grid after grid inside each bin:
 * [bin][grid g cells ... ] with grid g starting at cell offset
 * sum_{h<g} nx_h ny_h nz_h.  Results are identical to sweeping each grid in
 * its own context.  Errors as art_create, plus ART_E_INVALID for n_grids < 1
 * or > 4096 and for more than 2^31 cells in total.
 */
art_status art_batch_create(const art_grid *grids, const int *n_side, int n_grids, int nu_bins,
                            const art_options *opt, art_ctx **out);

/*
 * Time every compiled sweep-kernel variant of the context's precision on the
 * fields already set (reps sweeps each after one warm-up, on `stream`,
 * synchronizing it), in both launch forms (one CTA per work item, or the
 * persistent work queue) unless art_options.persistent fixed one, and keep
 * the fastest; *best_variant (may be NULL) receives its 1-based index.  Outputs of the timing sweeps go to internal
 * buffers.  Rebuilds the context's tables (direction groups chosen per
 * variant as at creation unless options fixed them).  Errors: ART_E_STATE (no
 * fields set), ART_E_OOM, ART_E_CUDA.
 */
art_status art_autotune(art_ctx *ctx, int reps, int *best_variant, void *stream);

/*
 * Fixed-order sum of n_parts FP32 partial fields (device [n_parts][n], part
 * order = the order of the sum, with Kahan compensation) into out (device
 * [n]); used to combine the J_in shares of direction shards (one per rank) so
 * that the result does not depend on how a collective would order the sum.
 * Stream-ordered.  Errors: ART_E_INVALID, ART_E_CUDA.
 */
art_status art_sum_partials(const float *parts, int n_parts, int64_t n, float *out, void *stream);

/* Release a context and all its device memory.  NULL is accepted. */
art_status art_destroy(art_ctx *ctx);

/* Text of the last error on this context ("" if none).  The pointer stays
 * valid until the next call on the context. */
const char *art_last_error(const art_ctx *ctx);

/*
 * Host-only (no GPU needed): exact number of (ray, cell) pairs with path
 * length > 0 in one sweep of one bin, from the per-slab segment tables the
 * sweep uses.  Errors: ART_E_INVALID (dims < 1, n_side < 1, NULL out).
 */
art_status art_count_segments(const art_grid *grid, int n_side, double tie_tol, int64_t *out);

/* Sweep statistics (segment count, launch shape, memory). */
art_status art_get_stats(const art_ctx *ctx, art_sweep_stats *st);

/*
 * Set the absorption coefficient (per cell width) and the source function S
 * (ART_FIELDS_S) or emissivity per cell width (ART_FIELDS_EPS) for every bin:
 * two arrays of nu_bins * nz * ny * nx values ([bin][z][y][x]).  on_device = 0:
 * host arrays, copied and validated synchronously; on_device = 1: device
 * arrays, read stream-ordered on `stream`.  Validation (both cases): every
 * value finite, kappa >= 0; failures return ART_E_INVALID and leave the
 * previous fields in place.
 */
art_status art_set_fields(art_ctx *ctx, const void *kappa, const void *src, int on_device,
                          void *stream);

/*
 * Band integrals G_b = int_bin sigma(nu)/(h nu) dnu, one per bin, used by the
 * Gamma output of art_sweep: Gamma^diff_in = 4 pi sum_b G_b J^in_b (the
 * non-local part of Eq. gamma_diff).  Host array of nu_bins doubles.  Without
 * this call G_b = 0.
 */
art_status art_set_band(art_ctx *ctx, const double *G);

/*
 * The straightforward layout of Sec. 3.1, kept to measure the ray grouping
 * (benchmark only): one thread per light-ray of a direction marches the whole
 * box and deposits (|n_a| / N_d) ds Ibar_in into J_in of every cell it
 * crosses (the same per-segment arithmetic and geometry as art_sweep).
 * Rays of one direction share cells, so mode 0 makes one launch per
 * direction with float atomicAdd deposits (results vary in the last bits
 * with the order of the atomics), and mode 1 four launches per direction,
 * one per ray group of starting columns (j mod 2, k mod 2), which visit no
 * cell twice, with plain read-modify-write deposits.  Directions run one
 * after another; the launches are captured once as a CUDA graph (per mode
 * and output pointer) and replayed on an internal stream ordered with
 * `stream`.  J_in: device [z][y][x] floats, overwritten with J^in.  Single
 * grid, FP32, one bin, ART_FIELDS_S, all directions, vacuum boundary, after
 * art_set_fields, on a context created with a slab-block kernel variant
 * (art_options.variant 1-15: it marches that kernel's segment tables).
 * Errors: ART_E_INVALID, ART_E_STATE (no fields, or a wavefront context),
 * ART_E_CUDA.
 */
art_status art_ablation_sweep(art_ctx *ctx, int mode, float *J_in, void *stream);

/*
 * Boundary intensity of the diffuse sweep: every ray of every direction
 * enters the box with intensity I_bc[b] in bin b (isotropic, uniform over the
 * faces), instead of the vacuum boundary I = 0 of Eq. (rad_tr2) with
 * I(0) = 0.  The formal solution then carries I_bc e^-tau into the box (the
 * incident-radiation boundary of Sec. 4.3).  Host array of nu_bins doubles,
 * each finite and >= 0; NULL restores vacuum.  Applies to the following
 * art_sweep calls (a captured graph is re-captured).  Errors: ART_E_INVALID.
 */
art_status art_set_boundary_intensity(art_ctx *ctx, const double *I_bc);

/*
 * Host-only: G = int_{nu_lo}^{nu_hi} sigma(nu)/(h nu) dnu for the hydrogenic
 * threshold power law sigma(nu) = sigma0 (nu/nu0)^-3, the band integral of
 * Eq. (gamma_diff) (nu_lo = nu0, nu_hi = nu0 + k_B T/h for the rectangular
 * recombination spectrum of Sec. 2.2).  Errors: ART_E_INVALID (non-positive
 * or non-finite arguments, nu_hi < nu_lo, NULL out).
 */
art_status art_band_integral(double sigma0, double h, double nu0, double nu_lo, double nu_hi,
                             double *G);

/*
 * One diffuse-radiation sweep (Sec. 2.2, Eqs. rt to mean_intensity, and
 * Eq. gamma_diff):
 *   J_in  = (1/N_d) sum_i Ibar^{ave,in}(n_i)          [bin][z][y][x]
 *   J     = J_in + S  (S = eps/kappa for ART_FIELDS_EPS where kappa > 0,
 *                      J = J_in where kappa = 0)       [bin][z][y][x]
 *   gamma = 4 pi sum_b G_b J_in_b                      [z][y][x]
 * Each output pointer may be NULL (not written).  on_device selects device or
 * host output buffers.  The sweep marches every ray with vacuum entry
 * intensity; Ibar^{ave,in} is the path-length-weighted average over the rays
 * that cross a cell, which equals the Delta-tau weighting of
 * Eq. (averaged_intensity) because kappa is constant inside a cell.
 * Deterministic: repeated calls give bit-identical outputs.  Errors:
 * ART_E_STATE (no fields set), ART_E_CUDA.
 */
art_status art_sweep(art_ctx *ctx, void *J, void *J_in, void *gamma, int on_device, void *stream);

/*
 * Read and clear the context's sweep error word, synchronizing `stream`.  The
 * wavefront sweep (the default for FP32 contexts with the paper's averaging)
 * hands ray intensities between thread blocks through device memory, and
 * every wait for an upstream block is bounded in time (art_sweep_set_wait);
 * a wait that runs out ends the sweep early and leaves its outputs invalid.
 * art_sweep with device outputs returns without waiting, so a caller checks
 * here; art_sweep with host outputs, art_sweep_stream and the iterations check
 * on their own.  Returns ART_OK, ART_E_TIMEOUT (a wait ran out) or ART_E_CUDA
 * (an index check of a checked build failed).  Errors: ART_E_INVALID (NULL).
 */
art_status art_sweep_check(art_ctx *ctx, void *stream);

/*
 * Bound of every wait of the wavefront sweep (seconds, default 2) and a test
 * hook: stall_unit >= 0 names a unit (CTA tile) that computes but never
 * publishes its progress (by its ticket: unit u of bin b of a launch that
 * holds several bins is b * ctas_per_launch + u, art_sweep_stats), so the
 * tiles downstream of it wait until the bound
 * and the sweep reports ART_E_TIMEOUT through art_sweep_check; -1 (the
 * default) disables the hook.  Errors: ART_E_INVALID (NULL ctx, bound not in
 * (0, 60], stall_unit < -1).
 */
art_status art_sweep_set_wait(art_ctx *ctx, double seconds, int stall_unit);

/*
 * Profiling counters of the wavefront sweep (a library built with
 * ART_WAVE_STATS=1; zeros in other builds and in contexts that use the
 * slab-block sweep).  out[4] receives, summed over the sweep launches since
 * the last call: out[0] warp cycles spent at the per-step block barriers,
 * out[1] warp cycles in the units (tiles), out[2] cycles lane 0 spent polling
 * upstream progress flags, out[3] the number of those polls; the counters are
 * then cleared.  Synchronizes the device.  Errors: ART_E_INVALID (NULL),
 * ART_E_CUDA.
 */
art_status art_wave_counters(art_ctx *ctx, long long *out);

/*
 * The sweeps of n_sets independent field sets held in host memory, streamed
 * through the device: the host-to-device copy and validation of set k + 1 and
 * the device-to-host copy of set k - 1 run on the library's own copy streams
 * while set k is swept on `stream` (double-buffered input staging and output
 * slots).  kappa[k], src[k]: host arrays as art_set_fields takes them with
 * on_device = 0; J[k], J_in[k], gamma[k]: host outputs as art_sweep writes
 * them (any of the three pointer arrays may be NULL: not written).  Page-
 * locked host memory lets the copies overlap; pageable memory works, slower.
 * Each set is checked as art_set_fields checks it before it is swept; the
 * first invalid set ends the call with ART_E_INVALID (the sets before it are
 * swept and written, the rest are not).  Returns once every output is in host
 * memory.  The outputs are bit-identical to art_set_fields + art_sweep per
 * set, and the last set swept remains the context's fields.  Errors:
 * ART_E_INVALID (null arrays or pointers, n_sets < 0, an invalid set, J on a
 * direction shard), ART_E_OOM, ART_E_CUDA.
 */
art_status art_sweep_stream(art_ctx *ctx, int n_sets, const void *const *kappa, const void *const *src,
                            void *const *J, void *const *J_in, void *const *gamma, void *stream);

/* Hydrogen rate coefficients at the (fixed) gas temperature and the spectral
 * constants of the recombination radiation (Sec. 2.2, App. B). */
typedef struct {
    double alphaA, alphaB;  /* case-A and case-B radiative recombination, cm^3/s */
    double gcoll;           /* collisional ionization of HI, cm^3/s */
    double sigma0;          /* HI photo-ionization cross section at nu0, cm^2 */
    double h, nu0, dnu;     /* Planck constant (erg s), threshold (Hz), k_B T/h (Hz) */
} art_chem;

/* A point source: position in cell widths (box [0, nx] x [0, ny] x [0, nz]),
 * ionizing photons per second (monochromatic at nu0 unless per-bin rates are
 * given). */
typedef struct {
    double x, y, z;
    double Q;
} art_source;

/* Starts of art_iterate_ionization. */
enum { ART_WARM_NONE = 0, ART_WARM_COARSE = 1, ART_WARM_SURROGATE = 2 };

typedef struct {
    int32_t iterations;     /* iterations run */
    int32_t converged;      /* 1 if the residual fell below tol */
    double residual;        /* last max_cells |n_e^(i) - n_e^(i-1)| / n_e^(i) */
    double seconds;         /* wall time of the call */
} art_iter_report;

/*
 * Photo-ionization rate per neutral atom from point sources (Sec. 2.1,
 * App. A, Eq. pc_gamma), by long characteristics: for every cell and source
 * (index order) the ray from the source to the cell centre is marched,
 * tau_b = sum kappa_b ds over the cells before the target cell, [r_in, r_out]
 * is the ray's passage through the target cell (r_in = 0 in the source's own
 * cell; the first cell is the one containing source + 1e-6 * direction), and
 *   Gamma += Q_b e^-tau_b (1 - e^-dtau_b) / (n_HI (4 pi/3)(r_out^3 - r_in^3) dx^3)
 * with n_HI = kappa_b/(sigma_b dx) (absorbed photons = in - out; App. A prints
 * out - in).  kappa: device [bin][z][y][x] floats per cell width; sigma: host
 * array of nu_bins cross sections (cm^2); src: host array of n_src sources;
 * Qb: host [n_src][nu_bins] photons/s per bin, or NULL to put each source's
 * Q in bin 0; gamma: device [z][y][x] floats, s^-1.  Uses grid.dx_cm.
 * Arithmetic is FP32 (positions as integer cell + FP32 fraction; the
 * per-bin constant 3 Q_b sigma_b / (4 pi dx^2) formed in FP64 on the host);
 * e^-tau is off by a relative ~u sum_c T_c |kappa_c - kappa_c+1| over the
 * ray's plane crossings at distances T_c (u = 2^-24).
 * Synchronizes `stream`.  Errors: ART_E_INVALID (null pointers, sources
 * outside the box, more than 4 bins, dx_cm <= 0, a bin constant beyond FP32
 * range), ART_E_OOM, ART_E_CUDA.
 */
art_status art_point_sources(art_ctx *ctx, const float *kappa, const double *sigma, const art_source *src,
                             const double *Qb, int n_src, float *gamma, void *stream);

/*
 * RT / ionization-balance fixed-point iteration (App. D) for hydrogen at a
 * fixed temperature, in the equilibrium (dt -> infinity) limit of the BDF
 * update of App. B.  Each iteration:
 *   kappa = n_HI sigma0 dx,  eps = h nu0 (alpha_A - alpha_B) n_e n_HII dx / (4 pi dnu)
 *   (the rectangular recombination spectrum of Sec. 2.2, swept at nu0);
 *   Gamma_point from art_point_sources; J^in from the diffuse sweep;
 *   g = Gamma_point + 4 pi G J^in, G = int sigma/(h nu) over [nu0, nu0 + dnu];
 *   the local term of Eq. (gamma_diff), (alpha_A - alpha_B) n_e n_HII / n_HI,
 *   taken at the new state, leaves alpha_B n_e n_HII = n_HI (Gamma_coll n_e + g),
 *   solved for the neutral fraction y in FP64 without cancellation;
 * until max_cells |n_e^(i) - n_e^(i-1)| / n_e^(i) < tol.
 * alpha_A == alpha_B selects the on-the-spot approximation (Sec. 2.1, Eq.
 * on_the_spot): the recombination emissivity vanishes, the source function is
 * neglected, J^in = 0 and no sweep runs, leaving case-B recombination
 * against the point sources (and collisions).
 * The context must be FP32 with one bin and ART_FIELDS_EPS inputs.
 * nH: device [z][y][x] doubles (cm^-3); y: device [z][y][x] doubles, the
 * initial neutral fraction on input and the result on output; src: host
 * array (src[i].Q photons/s, monochromatic at nu0 unless
 * art_set_source_spectrum gave bins); resid_hist: host array of max_iter
 * doubles or NULL; rep: may be NULL.  One host synchronization per iteration
 * (the residual).
 * warm_start (not in the paper, which iterates from its initial state):
 *   ART_WARM_NONE       the plain iteration from y;
 *   ART_WARM_COARSE     first solve the same problem on the mesh coarsened by
 *                       4 (N_side 4; n_H and y block means) to 1e-4 and start
 *                       from its neutral fraction;
 *   ART_WARM_SURROGATE  the coarse start, then early iterations take J^in
 *                       from the context's surrogate network (trained by
 *                       art_surrogate_train, art_net.h) until the residual
 *                       falls below 1e-3, judged against full sweeps and
 *                       abandoned for the coarse start if its error exceeds
 *                       0.3 (art_iterate_ionization_warm gives every option).
 * All three stop by the same rule at the same fixed point.  The warm starts
 * need grid dimensions divisible by 4.  Errors: ART_E_INVALID,
 * ART_E_STATE (ART_WARM_SURROGATE before art_surrogate_train),
 * ART_E_NOT_CONVERGED (y holds the last iterate), ART_E_OOM, ART_E_CUDA,
 * ART_E_TIMEOUT (a bounded wait of the sweep ran out).
 */
art_status art_iterate_ionization(art_ctx *ctx, const art_chem *chem, const double *nH, const art_source *src,
                                  int n_src, double tol, int max_iter, int warm_start, double *y,
                                  double *resid_hist, art_iter_report *rep, void *stream);

/*
 * Time-dependent mode (App. B-D) for hydrogen at the fixed temperature of
 * `chem`.  From t = 0 to t_end, in RT steps of
 *   dt = F min_cells dt_chem  (App. D; or dt_fixed when > 0),
 *   dt_chem = eps_e |n_e / n_e'| + eps_hi |n_HI / n_HI'|
 * evaluated at the state and rates at the start of the step.  Each step
 * iterates: the chemistry of every cell over dt from the state at t, at the
 * rates of the current iterate (the BDF update of App. B,
 * n_HI <- (C dtc + n_HI) / (1 + D dtc), C = alpha_B n_e n_HII,
 * D = Gamma_coll n_e + g, sub-cycled with dt_chem, the last sub-step cut to
 * end at dt), then the rates of the new iterate (point sources with the
 * source spectrum, the plane-parallel flux, the diffuse sweep), until
 * max_cells |n_e^(i) - n_e^(i-1)| / n_e^(i) < eps_iter.  g holds the
 * non-local rates; the local recombination term of Eq. gamma_diff cancels
 * the ground-state recombinations (alpha_B), and alpha_A == alpha_B is the
 * on-the-spot approximation (no sweep).  The energy equation of App. C is not
 * solved here: the temperature stays that of the rate constants
 * (art_evolve_thermal solves it).  FP64 chemistry,
 * one host synchronization per iteration.  nH, y: device [z][y][x] doubles;
 * y is the state at t = 0 on input and at t_end on output.  Errors:
 * ART_E_INVALID, ART_E_NOT_CONVERGED (max_steps before t_end, or a step that
 * reached max_iter: y holds the last state), ART_E_OOM, ART_E_CUDA.
 */
typedef struct {
    double t_end;      /* s */
    double F;          /* default 10 */
    double eps_iter;   /* default 1e-3 (App. D) */
    double eps_e;      /* default 0.2 */
    double eps_hi;     /* default 0.002 */
    double dt_fixed;   /* > 0: every step is dt_fixed (s); default 0 */
    int max_steps;     /* default 100000 */
    int max_iter;      /* per step, default 100 */
    int max_sub;       /* chemistry sub-steps per cell and step, default 1e6 */
} art_evolve_options;

typedef struct {
    int32_t steps;          /* RT steps taken */
    int32_t iterations;     /* chemistry / RT iterations over all steps */
    int32_t sweeps;         /* diffuse sweeps run */
    int32_t converged;      /* 1 if every step met eps_iter */
    int64_t sub_overflow;   /* (cell, iteration) pairs that ran out of sub-steps */
    double t;               /* time reached, s */
    double dt_min, dt_max;  /* smallest and largest step, s */
    double seconds;         /* wall time of the call */
} art_evolve_report;

art_status art_evolve_options_default(art_evolve_options *opt);
art_status art_evolve_ionization(art_ctx *ctx, const art_chem *chem, const double *nH, const art_source *src,
                                 int n_src, const art_evolve_options *opt, double *y, art_evolve_report *rep,
                                 void *stream);

/*
 * Energy equation of App. C for the time-dependent mode (art_evolve_thermal).
 * The paper takes its rate and cooling coefficients from the works of its
 * rate table without printing them; the library evaluates, T in K,
 * lambda = 2 * 157807 K / T:
 *   alpha_A(T), alpha_B(T)       Hui & Gnedin (1997) case-A / case-B fits
 *   Gamma_coll(T)                Cen (1992) collisional ionization of HI
 *   recombination cooling        Cen (1992) case A; Hui & Gnedin (1997) case B
 *   collisional ionization and excitation cooling of HI   Cen (1992)
 *   free-free cooling            1.42e-27 g_ff sqrt(T) n_e n_HII,
 *                                g_ff = 1.1 + 0.34 exp(-(5.5 - log10 T)^2 / 3)
 *   Compton cooling off the CMB  4 sigma_T a T_g^4 k_B (T - T_g) n_e / (m_e c),
 *                                T_g = 2.7255 (1 + z) K
 * Photo-heating per volume
 *   H = n_HI (sum_b Gamma_b e_bin[b] + Gamma^diff_in e_diff)
 *       + (alpha_A - alpha_B)(T) n_e n_HII e_diff,
 * the sources' and plane flux's rate per bin times the mean energy above
 * threshold of a photo-ionization in that bin, the transferred diffuse field,
 * and the local recombination photons that Eq. gamma_diff counts in
 * Gamma^diff (their ionizations cancel the ground-state recombinations, their
 * energy heats).  on_the_spot: alpha_A = alpha_B, no diffuse field and no
 * diffuse heating, case-B recombination cooling.
 */
typedef struct {
    int32_t on_the_spot;   /* 0 (default): the diffuse field is transferred */
    int32_t cool_mask;     /* cooling terms on: bit 0 recombination, 1 collisional ionization,
                              2 collisional excitation, 3 free-free, 4 Compton; default 31 */
    double e_bin[4];       /* erg per photo-ionization above threshold, per source-spectrum bin */
    double e_diff;         /* the same for the diffuse recombination band, erg */
    double z;              /* redshift of the CMB (Compton term), default 0 */
    double kB;             /* Boltzmann constant, erg/K, default 1.380649e-16 */
    double T_min, T_max;   /* temperature bracket, K; defaults 10 and 1e9 */
} art_thermal;

art_status art_thermal_default(art_thermal *th);

/*
 * The time-dependent mode of art_evolve_ionization with the energy equation
 * of App. C.  The temperature T (device [z][y][x] doubles, K; the state at
 * t = 0 on input and at t_end on output) is carried beside y.  In each
 * chemistry sub-step of a cell: the BDF update of y with alpha_B(T) and
 * Gamma_coll(T) at the sub-step's start, then the implicit update of the
 * specific energy u = 3 k_B T (1 + x) n_H / (2 rho) at the new composition,
 *   u' = u + (H(n') - C(n', u')) dtc / rho
 * (rho cancels: 1.5 k_B n_H ((1 + x') T' - (1 + x) T) = (H' - C(n', T')) dtc),
 * whose root T' is found by Newton's method from T on the analytic
 * derivative of the cooling fits, kept inside the bracket its iterates build
 * within [T_min, T_max] (bisection, or doubling / halving before both ends
 * are known, when a step leaves it).  The emissivity of the
 * diffuse field takes (alpha_A - alpha_B)(T) per cell, evaluated in FP32
 * like the field it scales; chem->alphaA, alphaB and gcoll are not used.  dt_chem is App. D's (n_e and n_HI only);
 * each RT step iterates until max_cells of |n_e^(i) - n_e^(i-1)| / n_e^(i)
 * and |u^(i) - u^(i-1)| / u^(i) is below eps_iter (App. D).  Point-source and
 * plane-flux heating come from the same kernels as their rates (FP32, the
 * sum over sources in FP64).  Errors: as art_evolve_ionization, and
 * ART_E_INVALID for a null th or T, kB <= 0, 0 < T_min < T_max violated, a
 * negative or non-finite energy, or an initial T outside [T_min, T_max].
 */
art_status art_evolve_thermal(art_ctx *ctx, const art_chem *chem, const art_thermal *th, const double *nH,
                              const art_source *src, int n_src, const art_evolve_options *opt, double *y,
                              double *T, art_evolve_report *rep, void *stream);

/*
 * Over-relaxation of the balance update in art_iterate_ionization (and its
 * warm-started form and coarse solve) on this context: each iteration sets
 *   y <- y_old + omega (y_balance - y_old),  clamped to [0, 1],
 * where y_balance is App. B's equilibrium at the iteration's rates.
 * omega = 1 (the default) is the paper's plain fixed-point iteration; a fixed
 * point of either form is a fixed point of the other, and the residual test
 * measures the relaxed change (|y_balance - y_old| is 1/omega of it).  Not in
 * the paper: on the clumpy 256^3 medium with 8 sources, omega = 1.3 takes 29
 * iterations instead of 41.  Errors: ART_E_INVALID unless 0 < omega < 2.
 */
art_status art_set_relaxation(art_ctx *ctx, double omega);

/*
 * Source spectrum of art_iterate_ionization on this context (App. A with
 * frequency bins): every point source emits Q * frac[b] photons/s in bin b,
 * absorbed with cross section sigma[b] (cm^2; kappa_b = n_HI sigma[b] dx);
 * Gamma sums over the bins (Eq. pc_gamma per bin).  The diffuse
 * recombination field keeps its band at nu0.  nbins = 0 restores the
 * default (one bin at chem->sigma0, frac 1).  1 <= nbins <= 4.  Errors:
 * ART_E_INVALID.
 */
art_status art_set_source_spectrum(art_ctx *ctx, int nbins, const double *sigma, const double *frac);

/*
 * Photo-ionization rate of a plane-parallel incident flux, the Test-3 setup
 * of Sec. 4.3 (a constant photon flux through one face of the box: a point
 * source at infinity).  The beam travels along +axis (dir = 1, entering at
 * coordinate 0) or -axis (dir = -1); axis 0, 1, 2 = x, y, z.  In bin b a cell
 * absorbs flux[b] dx^2 e^-tau (1 - e^-dtau) photons/s, tau summing kappa_b
 * over the cells before it along the beam and dtau = kappa_b, so per
 * neutral atom
 *   Gamma = sum_b flux[b] sigma[b] e^-tau (1 - e^-dtau) / dtau
 * (photon-conserving as App. A's point-source rate; no dependence on dx).
 * kappa: device [bin][z][y][x] floats per cell width; sigma, flux: host
 * arrays of nu_bins values (cm^2, photons/s/cm^2); gamma: device [z][y][x]
 * floats (s^-1), overwritten.  FP32, stream-ordered.  Errors: ART_E_INVALID
 * (null pointers, bad axis or dir, negative or non-finite values, more than
 * 4 bins, a rate beyond FP32 range), ART_E_CUDA.
 */
art_status art_plane_source(art_ctx *ctx, const float *kappa, const double *sigma, int axis, int dir,
                            const double *flux, float *gamma, void *stream);

/*
 * Adds a plane-parallel incident flux (as art_plane_source) to the point
 * sources of art_iterate_ionization on this context: flux photons/s/cm^2
 * along axis in direction dir, split over the source spectrum's bins like
 * the point sources' photons.  flux = 0 removes it.  Errors: ART_E_INVALID.
 */
art_status art_set_plane_source(art_ctx *ctx, int axis, int dir, double flux);

/* Per-kernel device time accumulated while profiling is enabled. */
typedef struct {
    double sweep_ms;          /* slab-block sweep kernels */
    int64_t sweep_launches;
    double reduce_ms;         /* partial-reduction kernels */
    int64_t reduce_launches;
} art_profile;

/*
 * Enable (1) or disable (0) per-kernel timing: while enabled, art_sweep
 * records CUDA events on its stream around the sweep launches of each bin and
 * around the reduction.  The events add a few microseconds per sweep.
 */
art_status art_profile_enable(art_ctx *ctx, int enable);

/*
 * Wait for the recorded events, add their durations into *out and, if
 * reset != 0, forget them.  Errors: ART_E_CUDA.
 */
art_status art_profile_read(art_ctx *ctx, art_profile *out, int reset);

/*
 * Issue-rate microbenchmark of the current device (about 15 ms): results per
 * clock per SM of MUFU ex2 (the one exponential of each segment), MUFU rcp,
 * scalar FP32 FFMA, and FP32 FMAs issued as packed FP32x2 instructions (two
 * per instruction, the form of the sweep's pair arithmetic), from clock64()
 * timings of independent chains with two 1024-thread CTAs per SM: per SM, the
 * window from the earliest start to the latest end of its CTAs; the median
 * over SMs, the better of two runs.  Used to state the sweep's arithmetic
 * roofline.  Errors: ART_E_INVALID (NULL output), ART_E_OOM, ART_E_CUDA.
 */
art_status art_measure_pipes(double *ex2_per_clk_sm, double *rcp_per_clk_sm,
                             double *ffma_per_clk_sm, double *ffma2_per_clk_sm);

/*
 * One FP32 sweep (kappa, S inputs, J^in output) that allocates no memory.
 * The paper has no counterpart: this entry point exists for callers that
 * cannot allocate device memory -- a simulation code that reserves the whole
 * device memory budget for its own arrays at start-up, or code calling from a
 * place where the implicit device-wide synchronization of cudaMalloc and
 * cudaFree would stall work it has in flight on other streams.
 *
 * kappa, S: device arrays of nz * ny * nx floats ([z][y][x]); J_in: device
 * array of the same size, written with J^in as art_sweep writes it (the same
 * kernels; results agree with art_sweep within FP32 rounding).  All working
 * memory is one file-scope device array of 12 MiB that every GPU loading the
 * library holds until the process exits; host-side tables are file-scope too.
 * Limits: each axis <= 64 cells, at most 32768 cells, 1 <= n_side <= 4, and
 * the grid's tables must fit the 12 MiB; otherwise ART_E_INVALID and a message
 * in errbuf (if errbuf != NULL, errlen bytes).  Inputs are not validated.
 *
 * The library's device code is loaded lazily: the first call on each device
 * loads the module that holds the scratch array (looking up its address with
 * cudaGetSymbolAddress), and only then are its 12 MiB reserved.  A caller that
 * reserves the device's memory for itself should therefore make a first call
 * (a 1 x 1 x 1 grid will do) before it does; a load that runs out of memory
 * returns ART_E_OOM.  The call copies its tables with cudaMemcpyAsync and
 * synchronizes `stream` once before launching its kernels on it (it returns
 * without waiting for them), so it must never be called on a stream that is
 * being captured: it checks, and returns ART_E_INVALID before queuing anything,
 * leaving the capture valid.  Every call uses the same scratch array and the array keeps the
 * last call's contents (nothing is carried over: each call writes every
 * element it reads), so calls that overlap on the GPU -- from several threads
 * or streams -- race and must be serialized by the caller.
 */
art_status art_sweep_noalloc(const art_grid *grid, int n_side, const float *kappa, const float *S,
                             float *J_in, void *stream, char *errbuf, size_t errlen);

#ifdef __cplusplus
}
#endif

#endif /* ART_H */
