/*
 * art_net.h -- C ABI of the 3D-convolution surrogate of libart: a small
 * network that predicts the diffuse mean intensity J^in of the sweep from
 * the solver's state, trained on the GPU on plain-sweep results, and the
 * RT / ionization-balance iteration it warm-starts.
 *
 * The paper iterates plain sweeps to convergence (App. D); the surrogate is
 * an addition of this library and has no counterpart in the paper.  What it
 * computes:
 *   - inputs per cell (4 channels): 0.25 ln kappa, 0.1 ln(eps/eps_ref),
 *     x = 1 - y, 0.1 ln(J_c/eps_ref); each logarithm clamped at ln(1e-30)
 *     below its reference; eps_ref = max eps; kappa and eps the sweep's
 *     absorption and emissivity per cell width (ART_FIELDS_EPS form) from the
 *     neutral fraction y; J_c the J^in of a sweep on the mesh coarsened by a
 *     factor f (block means times f), prolonged by injection;
 *   - network: four 3x3x3 convolutions with zero padding and per-layer
 *     dilations, channels 4 -> 32 -> 32 -> 32 -> 1, ReLU after the first
 *     three; BF16 weights and activations, FP32 accumulation (tensor cores);
 *   - prediction J^in = J_c exp(o); training target t = ln(J^in/J_c) on the
 *     plain sweep's J^in (logarithms clamped at ln eps_ref - 69); loss
 *     mean(w (o - t)^2) with cell weights w = J^in / mean J^in (or 1);
 *     optimizer Adam with bias-corrected moments and FP32
 *     master weights.
 * Parameters (FP32, "params layout"): for each layer l = 0..3, W_l as
 * [27][c_out][c_in] (tap t = 9 (dz+1) + 3 (dy+1) + (dx+1), offsets
 * d_l * (dx, dy, dz) from the output cell; x fastest in cell indices),
 * then b_l [c_out]; c_in/c_out = 4/32, 32/32, 32/32, 32/1; ART_NET_PARAMS
 * floats in total.
 * Grids passed to the network need nx * ny * nz a multiple of 128, with nx a
 * divisor of 128 (and 128/nx dividing ny) or a multiple of 128.
 * Conventions (ownership, streams, status codes) as in art.h.
 */
#ifndef ART_NET_H
#define ART_NET_H

#include "art.h"

#ifdef __cplusplus
extern "C" {
#endif

#define ART_NET_PARAMS 59713

typedef struct art_net art_net;

typedef struct {
    int dilation[4];      /* per layer; default {1, 2, 4, 8} */
    uint64_t seed;        /* He-normal initialisation (last layer x 0.1), default 1 */
    double lr, beta1, beta2, adam_eps;   /* Adam; default 1e-3, 0.9, 0.999, 1e-8 */
} art_net_options;

/* Defaults as stated above.  Never fails for a non-NULL pointer. */
art_status art_net_options_default(art_net_options *opt);

/* Create a network with freshly initialised weights (device memory for the
 * weights and optimizer state; activation workspace grows with the grids it
 * sees).  Errors: ART_E_INVALID (dilations outside 1..16), ART_E_OOM,
 * ART_E_CUDA. */
art_status art_net_create(const art_net_options *opt, art_net **out);

/* Release the network.  NULL is accepted. */
art_status art_net_destroy(art_net *net);

/* Text of the last error ("" if none). */
const char *art_net_last_error(const art_net *net);

/* Copy the FP32 master parameters to / from a host array of ART_NET_PARAMS
 * floats (params layout).  Setting resets the Adam moments and step count.
 * Synchronous.  Errors: ART_E_INVALID, ART_E_CUDA. */
art_status art_net_get_params(art_net *net, float *host);
art_status art_net_set_params(art_net *net, const float *host);

/*
 * Forward pass: X device [4][nz][ny][nx] floats (the input channels), o
 * device [nz][ny][nx] floats.  Stream-ordered on `stream`.  Errors:
 * ART_E_INVALID (grid shape, NULL), ART_E_OOM, ART_E_CUDA.
 */
art_status art_net_forward(art_net *net, int nx, int ny, int nz, const float *X, float *o, void *stream);

/*
 * Forward and backward pass on one sample (X as above, t device [nz][ny][nx]
 * targets, w device [nz][ny][nx] loss weights or NULL for 1): *loss (host)
 * receives mean(w (o - t)^2) and grads (host, may be NULL) the gradient of
 * the loss in every parameter (params layout).  Synchronizes `stream`.
 * Errors as art_net_forward.
 */
art_status art_net_gradients(art_net *net, int nx, int ny, int nz, const float *X, const float *t, const float *w,
                             double *loss, float *grads, void *stream);

/*
 * One Adam step on one sample (X, t, w as in art_net_gradients): forward,
 * backward, update of the master weights and of their BF16 copies.  *loss (host, may be NULL) receives the
 * loss before the step; reading it synchronizes `stream`.  Errors as
 * art_net_forward.
 */
art_status art_net_train_step(art_net *net, int nx, int ny, int nz, const float *X, const float *t, const float *w,
                              double *loss, void *stream);

/*
 * Synchronize `stream` and report whether any convolution kernel of the
 * network gave up a bounded wait since the last check: ART_E_TIMEOUT (the
 * error word is then cleared; outputs of those launches are undefined, the
 * network and the CUDA context stay usable) or ART_OK.  The convolution
 * kernels bound every wait on a shared-memory barrier to about one second,
 * then drain their copies, free tensor memory and return.
 */
art_status art_net_check(art_net *net, void *stream);

/*
 * Test hook for the bounded waits: while on != 0, the convolution kernels
 * issue no loads, so their waits run out (about one second per launch) and
 * the next art_net_check reports ART_E_TIMEOUT.  Off by default.
 */
art_status art_net_set_test_stall(art_net *net, int on);

/*
 * Output planes per work item of the convolution kernels: 1, 2 or 4 (planes
 * z, z + d, ... of one tile position share the loaded tap tiles), or 0 to
 * choose by grid and dilation (the default).  Results do not depend on it.
 * Errors: ART_E_INVALID.
 */
art_status art_net_set_plane_group(art_net *net, int planes);

/*
 * Training sample of the solver state y (device [z][y][x] doubles) on the
 * context's grid: kappa = y nH sigma0 dx and eps as in art_iterate_ionization,
 * a plain sweep for J^in and a coarse sweep (factor coarse_factor, N_side
 * coarse_nside) for J_c.  Outputs (device, any may be NULL): X [4][V] inputs,
 * t [V] target, jin [V] the sweep's J^in, jc [V] the prolonged coarse J^in.
 * The context must satisfy art_iterate_ionization's requirements, with grid
 * dimensions divisible by coarse_factor.  Stream-ordered.  Errors:
 * ART_E_INVALID, ART_E_OOM, ART_E_CUDA.
 */
art_status art_surrogate_sample(art_ctx *ctx, const art_chem *chem, const double *nH, const double *y,
                                int coarse_factor, int coarse_nside, float *X, float *t, float *jin, float *jc,
                                void *stream);

/*
 * Training data from the plain iteration: runs n_iter iterations of
 * art_iterate_ionization from the state y (device, updated in place) and
 * records, for every iteration k, the sample of the state the iteration
 * starts from: inputs X + k * 4V (layout [4][V]), target t + k * V and loss
 * weights w + k * V (J^in / mean J^in; w may be NULL), target and weights
 * taken on the J^in of that iteration's own sweep.  X, t, w are device arrays
 * of n_iter samples.  Stream-ordered except for one host
 * synchronization per iteration.  Errors as art_surrogate_sample, and
 * ART_E_INVALID under the on-the-spot approximation (no diffuse field).
 */
art_status art_surrogate_collect(art_ctx *ctx, const art_chem *chem, const double *nH, const art_source *src,
                                 int n_src, double *y, int n_iter, int coarse_factor, int coarse_nside, float *X,
                                 float *t, float *w, void *stream);

/*
 * Adam steps over a set of n_samples samples of one grid shape (X device
 * [n_samples][4][V], t and w device [n_samples][V], w may be NULL): `steps` steps, one sample per
 * step, in epochs of a permutation drawn from `seed` (splitmix64 keys,
 * deterministic).  loss_hist (host, may be NULL) receives the loss of every
 * step (reading it synchronizes once at the end).  Errors as
 * art_net_train_step.
 */
art_status art_net_train(art_net *net, int nx, int ny, int nz, int n_samples, const float *X, const float *t,
                         const float *w, int steps, uint64_t seed, double *loss_hist, void *stream);

typedef struct {
    int coarse_factor;     /* mesh coarsening of the coarse sweep, default 4 */
    int coarse_nside;      /* N_side of the coarse sweep, default 4 */
    int use_net;           /* 1 (default): J^in = J_c exp(net); 0: J^in = J_c (coarse sweep alone) */
    int phase1_max_iter;   /* surrogate iterations at most, default 40 */
    double phase1_tol;     /* surrogate phase ends below this residual, default 1e-3 */
    double judge_tol;      /* fall back when sum|J_s - J|/sum J exceeds this, default 0.3 */
    int coarse_solve;      /* 1 (default): start from the coarse-mesh solution (see below) */
    double coarse_tol;     /* residual of the coarse-mesh solve, default 1e-4 */
    int judge_after;       /* also judge after this many surrogate iterations, default 2; 0: only at the end */
} art_warm_options;

typedef struct {
    art_iter_report total;        /* all iterations, as art_iterate_ionization */
    int32_t surrogate_iterations; /* iterations that took J^in from the surrogate */
    int32_t plain_sweeps;         /* full sweeps run (judge included) */
    int32_t fell_back;            /* 1 if a judge restarted from the fallback state */
    double judge_error;           /* sum|J_s - J| / sum J at the last judge */
    int32_t coarse_iterations;    /* iterations of the coarse-mesh solve */
} art_warm_report;

/* Fill `opt` with the defaults above. */
art_status art_warm_options_default(art_warm_options *opt);

/*
 * The iteration of art_iterate_ionization (same arguments, same fixed point
 * and stopping rule), warm-started.  With coarse_solve, the whole RT /
 * balance problem is first solved on the mesh coarsened by coarse_factor
 * (N_side coarse_nside; n_H and y block means, sources at the same place) to
 * coarse_tol, and the fine iteration starts from that neutral fraction
 * (injection).  Then, while the residual is above phase1_tol (and for at
 * most phase1_max_iter iterations), J^in comes from the surrogate (coarse
 * sweep of the current state, corrected by the network when use_net) instead
 * of the full sweep.  One full sweep judges the surrogate on the current
 * state after judge_after surrogate iterations and again when the phase
 * ends; its exact J^in serves the next iteration.  If a judge's error
 * exceeds judge_tol the state is reset to the fallback state -- the
 * coarse-mesh start, or the caller's y without coarse_solve -- and
 * (fell_back = 1) plain iterations run to tol from there.  net may be NULL only with
 * use_net = 0.  Under the on-the-spot approximation (alpha_A == alpha_B)
 * there is no diffuse field: only the coarse-mesh solve runs before the
 * plain iterations.  Errors as art_iterate_ionization.
 */
art_status art_iterate_ionization_warm(art_ctx *ctx, art_net *net, const art_chem *chem, const double *nH,
                                       const art_source *src, int n_src, double tol, int max_iter,
                                       const art_warm_options *wopt, double *y, double *resid_hist,
                                       art_warm_report *rep, void *stream);

/* Training samples on a context's grid: X [n_samples][4][V], t and w
 * [n_samples][V] device floats (w may be NULL: weights 1), V = nx ny nz, as
 * art_surrogate_collect writes them. */
typedef struct {
    int nx, ny, nz;
    int n_samples;
    const float *X, *t, *w;
} art_dataset;

typedef struct {
    int steps;                /* Adam steps, one sample per step; default 0 = 8 epochs */
    uint64_t seed;            /* permutation seed of the epochs, default 1 */
    int reset;                /* 1: start from freshly initialised weights (net options) */
    art_net_options net;      /* network of the first call or of a reset (defaults as art_net_options_default) */
    void *stream;             /* cudaStream_t of the training launches, NULL = legacy default */
} art_train_opts;

typedef struct {
    int32_t steps;            /* steps run */
    double first_epoch_loss;  /* mean loss of the first min(n_samples, steps) steps */
    double last_epoch_loss;   /* mean loss of the last min(n_samples, steps) steps */
    double seconds;           /* wall time */
} art_train_report;

/* Defaults of art_train_opts.  Never fails for a non-NULL pointer. */
art_status art_train_opts_default(art_train_opts *opt);

/*
 * Train the context's surrogate network (the one ART_WARM_SURROGATE of
 * art_iterate_ionization uses) on a dataset of its grid: art_net_train's
 * seeded Adam epochs on a network the context owns, created by the first
 * call (or by reset) with opt->net.  The paper has no surrogate; this is the
 * warm start's learned part.  opt may be NULL (defaults), rep may be NULL.
 * Synchronizes opt->stream once.  Errors: ART_E_INVALID (NULL ctx or data,
 * a grid other than the context's, n_samples < 1, NULL X or t, steps < 0),
 * ART_E_OOM, ART_E_CUDA, ART_E_TIMEOUT (a bounded wait of the convolution
 * kernels ran out).
 */
art_status art_surrogate_train(art_ctx *ctx, const art_dataset *data, const art_train_opts *opt,
                               art_train_report *rep);

/* The context's surrogate network (owned by the context; NULL before
 * art_surrogate_train), e.g. to read or set its parameters.  Errors:
 * ART_E_INVALID (NULL ctx or out). */
art_status art_surrogate_network(art_ctx *ctx, art_net **out);

#ifdef __cplusplus
}
#endif

#endif /* ART_NET_H */
