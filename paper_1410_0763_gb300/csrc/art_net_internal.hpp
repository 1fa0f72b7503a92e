// art_net_internal.hpp -- surrogate entry points shared by the translation
// units of libart (private).
#pragma once
#include <cuda_runtime.h>

#include "art.h"
#include "art_net.h"

struct art_ctx;

// The coarse-mesh context (factor f, N_side nside_c) and the surrogate
// scratch of this context, created on first use.
art_status artnet_coarse(art_ctx *ctx, int f, int nside_c);
// Surrogate J^in on the context's grid from the solver fields kappa, eps (FP32
// per cell width) and the neutral fraction y: coarse sweep (factor f, N_side
// nside_c), inputs, and (use_net) the network.  Outputs, each optional:
// jin = J_c exp(o) (or J_c), X32 = inputs [4][V], jc_fine = prolonged J_c.
art_status artnet_surrogate(art_ctx *ctx, art_net *net, int use_net, int f, int nside_c, const float *kap,
                            const float *eps, const double *y, float *jin, float *X32, float *jc_fine,
                            cudaStream_t st);
// Training target from the sweep's J^in and the prolonged J_c of the last
// artnet_surrogate call on this context (its eps_ref).
art_status artnet_target(art_ctx *ctx, const float *jin, const float *jc_fine, float *t, cudaStream_t st);
// Loss weights w = J / mean(J) over the context's cells (synchronizes st).
art_status artnet_weights(art_ctx *ctx, const float *jin, float *w, cudaStream_t st);
// sum |a - b| / sum |b| over the context's cells (synchronizes st).
art_status artnet_l1(art_ctx *ctx, const float *a, const float *b, double *err, cudaStream_t st);
// Bounded-wait status of the network's last kernels (synchronizes st).
art_status artnet_check(art_net *n, cudaStream_t st);
const char *artnet_error(const art_net *n);
