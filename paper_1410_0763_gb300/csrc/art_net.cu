// art_net.cu -- the 3D-convolution surrogate (include/art_net.h): network
// object, tensor maps, forward / backward / Adam, and the surrogate's inputs
// on a sweep context (coarse sweep, features, prediction).
#include <cuda.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "art.h"
#include "art_net.h"
#include "art_ctx.hpp"
#include "art_net_internal.hpp"
#include "art_net_kernels.cuh"

using namespace artnet;

namespace {

// Layers in the params layout: (c_in, c_out) padded to the kernels' channel
// counts (16 or 32).
const LayerDev kLayers[4] = {
    {0, 3456, 4, 32, 16, 32},
    {3488, 31136, 32, 32, 32, 32},
    {31168, 58816, 32, 32, 32, 32},
    {58848, 59712, 32, 1, 32, 16},
};
static_assert(59713 == ART_NET_PARAMS, "parameter count");

typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                  const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn()
{
    static EncodeTiledFn fn = nullptr;
    if (!fn) {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiledFn>(p);
        cudaGetLastError();
    }
    return fn;
}

// Channels-last BF16 activations [nz][ny][nx][C]; box = one 128-voxel tile.
bool act_map(CUtensorMap *m, const void *base, int C, int nx, int ny, int nz)
{
    EncodeTiledFn enc = encode_fn();
    if (!enc) return false;
    const int bx = std::min(nx, TILE_M), by = TILE_M / bx;
    cuuint64_t dims[4] = {(cuuint64_t)C, (cuuint64_t)nx, (cuuint64_t)ny, (cuuint64_t)nz};
    cuuint64_t strides[3] = {(cuuint64_t)C * 2, (cuuint64_t)C * 2 * nx, (cuuint64_t)C * 2 * nx * ny};
    cuuint32_t box[4] = {(cuuint32_t)C, (cuuint32_t)bx, (cuuint32_t)by, 1};
    cuuint32_t es[4] = {1, 1, 1, 1};
    return enc(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, const_cast<void *>(base), dims, strides, box, es,
               CU_TENSOR_MAP_INTERLEAVE_NONE, C == 32 ? CU_TENSOR_MAP_SWIZZLE_64B : CU_TENSOR_MAP_SWIZZLE_32B,
               CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// Weights [27 * rows][K] BF16, box = one tap's [rows][K] block.
bool weight_map(CUtensorMap *m, const void *base, int K, int rows)
{
    EncodeTiledFn enc = encode_fn();
    if (!enc) return false;
    cuuint64_t dims[2] = {(cuuint64_t)K, (cuuint64_t)27 * rows};
    cuuint64_t strides[1] = {(cuuint64_t)K * 2};
    cuuint32_t box[2] = {(cuuint32_t)K, (cuuint32_t)rows};
    cuuint32_t es[2] = {1, 1};
    return enc(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void *>(base), dims, strides, box, es,
               CU_TENSOR_MAP_INTERLEAVE_NONE, K == 32 ? CU_TENSOR_MAP_SWIZZLE_64B : CU_TENSOR_MAP_SWIZZLE_32B,
               CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// Counter-based normal numbers for the initial weights: splitmix64 of
// (seed, index) -> two uniforms -> Box-Muller.
double normal_at(uint64_t seed, uint64_t i)
{
    auto mix = [](uint64_t z) {
        z += 0x9E3779B97F4A7C15ull;
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
        return z ^ (z >> 31);
    };
    const uint64_t a = mix(seed * 0x100000001B3ull + 2 * i), b = mix(seed * 0x100000001B3ull + 2 * i + 1);
    const double u1 = ((a >> 11) + 0.5) * (1.0 / 9007199254740992.0), u2 = (b >> 11) * (1.0 / 9007199254740992.0);
    return std::sqrt(-2.0 * std::log(u1)) * std::cos(2.0 * 3.14159265358979323846 * u2);
}

}  // namespace

struct art_net {
    art_net_options opt{};
    std::string err;
    float *params = nullptr, *m = nullptr, *v = nullptr, *grad = nullptr;
    int step = 0;
    bf16 *wf[4] = {}, *wd[4] = {};
    float *bias[4] = {};
    int *d_err = nullptr;
    CUtensorMap wmap_f[4], wmap_d[4];
    // activation workspace
    int nx = 0, ny = 0, nz = 0;
    long long V = 0;
    bf16 *X16 = nullptr, *h[3] = {}, *g16 = nullptr, *gA = nullptr, *gB = nullptr;
    float *o = nullptr, *part = nullptr, *pb = nullptr;
    double *lpart = nullptr, *loss = nullptr;
    CUtensorMap amap_X, amap_h[3], amap_g16, amap_gA, amap_gB;
    int sms = 152;
    int test_stall = 0;
    int plane_group = 0;   // output planes per convolution work item (0: by grid and dilation)
};

namespace {

art_status nfail(art_net *net, art_status st, const std::string &msg)
{
    if (net) net->err = msg;
    return st;
}

#define NCK(net, call)                                                                              \
    do {                                                                                            \
        cudaError_t e_ = (call);                                                                    \
        if (e_ != cudaSuccess)                                                                      \
            return nfail(net, e_ == cudaErrorMemoryAllocation ? ART_E_OOM : ART_E_CUDA,             \
                         std::string(#call) + ": " + cudaGetErrorString(e_));                       \
    } while (0)

template <typename T> cudaError_t nalloc(T **p, size_t n)
{
    return cudaMalloc(reinterpret_cast<void **>(p), std::max<size_t>(n * sizeof(T), 16));
}

void free_workspace(art_net *n)
{
    void *ptrs[] = {n->X16, n->h[0], n->h[1], n->h[2], n->g16, n->gA, n->gB, n->o, n->part, n->pb, n->lpart, n->loss};
    for (void *p : ptrs)
        if (p) cudaFree(p);
    n->X16 = n->h[0] = n->h[1] = n->h[2] = n->g16 = n->gA = n->gB = nullptr;
    n->o = n->part = n->pb = nullptr;
    n->lpart = n->loss = nullptr;
    n->V = 0;
    n->nx = n->ny = n->nz = 0;
}

bool shape_ok(int nx, int ny, int nz)
{
    if (nx < 1 || ny < 1 || nz < 1) return false;
    const long long V = (long long)nx * ny * nz;
    if (V % TILE_M != 0 || V > (1LL << 31)) return false;
    if (nx >= TILE_M) return nx % TILE_M == 0;
    if (TILE_M % nx != 0) return false;
    return ny % (TILE_M / nx) == 0;
}

art_status ensure_workspace(art_net *n, int nx, int ny, int nz)
{
    if (!shape_ok(nx, ny, nz))
        return nfail(n, ART_E_INVALID,
                     "surrogate grid: nx*ny*nz must be a multiple of 128, nx a divisor of 128 (with 128/nx dividing "
                     "ny) or a multiple of 128");
    if (n->nx == nx && n->ny == ny && n->nz == nz) return ART_OK;
    free_workspace(n);
    const long long V = (long long)nx * ny * nz;
    const long long nch = (V + WG_CHUNK - 1) / WG_CHUNK;
    const long long nb = (V + 255) / 256;
    if (nalloc(&n->X16, V * 16) != cudaSuccess || nalloc(&n->h[0], V * 32) != cudaSuccess ||
        nalloc(&n->h[1], V * 32) != cudaSuccess || nalloc(&n->h[2], V * 32) != cudaSuccess ||
        nalloc(&n->g16, V * 16) != cudaSuccess || nalloc(&n->gA, V * 32) != cudaSuccess ||
        nalloc(&n->gB, V * 32) != cudaSuccess || nalloc(&n->o, V) != cudaSuccess ||
        nalloc(&n->part, nch * 27 * 32 * 32) != cudaSuccess || nalloc(&n->pb, nch * 32) != cudaSuccess ||
        nalloc(&n->lpart, nb) != cudaSuccess || nalloc(&n->loss, 1) != cudaSuccess) {
        cudaGetLastError();
        free_workspace(n);
        return nfail(n, ART_E_OOM, "surrogate workspace allocation failed");
    }
    bool ok = act_map(&n->amap_X, n->X16, 16, nx, ny, nz);
    for (int i = 0; i < 3; ++i) ok = ok && act_map(&n->amap_h[i], n->h[i], 32, nx, ny, nz);
    ok = ok && act_map(&n->amap_g16, n->g16, 16, nx, ny, nz) && act_map(&n->amap_gA, n->gA, 32, nx, ny, nz) &&
         act_map(&n->amap_gB, n->gB, 32, nx, ny, nz);
    if (!ok) {
        free_workspace(n);
        return nfail(n, ART_E_CUDA, "cuTensorMapEncodeTiled failed for an activation map");
    }
    n->nx = nx;
    n->ny = ny;
    n->nz = nz;
    n->V = V;
    return ART_OK;
}

template <int CIN, int COUT, int MODE, int G>
art_status conv_g(art_net *n, const CUtensorMap &amap, const CUtensorMap &wmap, const ConvArgs &a, cudaStream_t st)
{
    using L = ConvSmem<CIN, COUT, G>;
    auto kern = conv_tc_kernel<CIN, COUT, MODE, G>;
    // at most two CTAs per SM whenever their TMEM allocations (2 G COUT
    // columns each) would not fit three times into the SM's 512 columns:
    // the shared-memory request is raised so a third cannot be resident
    constexpr int SMEM = (3 * L::NCOLS > 512 && L::BYTES < 80 * 1024) ? 80 * 1024 : L::BYTES;
    static bool attr = false;
    if (!attr) {
        NCK(n, cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM));
        attr = true;
    }
    const long long plane = (long long)a.nx * a.ny;
    const int nzg = (a.nz + G * a.dil - 1) / (G * a.dil) * a.dil;
    const long long items = plane / TILE_M * nzg;
    const int grid = (int)std::min<long long>(items, 2LL * n->sms);
    kern<<<grid, CONV_THREADS, SMEM, st>>>(amap, wmap, a);
    NCK(n, cudaGetLastError());
    return ART_OK;
}

// Planes per work item: 4 when the grid holds four planes at this dilation,
// else 2 or 1 (fewer planes beyond the grid to skip).
template <int CIN, int COUT, int MODE>
art_status conv(art_net *n, const CUtensorMap &amap, const CUtensorMap &wmap, const float *bias, const bf16 *mask,
                bf16 *out, float *out_f32, int dil, cudaStream_t st)
{
    ConvArgs a;
    a.bias = bias;
    a.mask = mask;
    a.out = out;
    a.out_f32 = out_f32;
    a.nx = n->nx;
    a.ny = n->ny;
    a.nz = n->nz;
    a.dil = dil;
    a.ntiles = (int)(n->V / TILE_M);
    a.err = n->d_err;
    a.test_stall = n->test_stall;
    const int g = n->plane_group > 0 ? n->plane_group : (n->nz >= 4 * dil ? 4 : (n->nz >= 2 * dil ? 2 : 1));
    if (g >= 4) return conv_g<CIN, COUT, MODE, 4>(n, amap, wmap, a, st);
    if (g == 2) return conv_g<CIN, COUT, MODE, 2>(n, amap, wmap, a, st);
    return conv_g<CIN, COUT, MODE, 1>(n, amap, wmap, a, st);
}

art_status pack_weights(art_net *n, cudaStream_t st)
{
    for (int l = 0; l < 4; ++l) {
        const LayerDev &L = kLayers[l];
        const int cnt = 27 * L.coutp * L.cinp;
        pack_kernel<<<(cnt + 255) / 256, 256, 0, st>>>(n->params, L, n->wf[l], n->bias[l], l > 0 ? n->wd[l] : nullptr);
        NCK(n, cudaGetLastError());
    }
    return ART_OK;
}

art_status forward16(art_net *n, float *o, cudaStream_t st)
{
    const int *d = n->opt.dilation;
    art_status s;
    if ((s = conv<16, 32, MODE_RELU>(n, n->amap_X, n->wmap_f[0], n->bias[0], nullptr, n->h[0], nullptr, d[0], st)))
        return s;
    if ((s = conv<32, 32, MODE_RELU>(n, n->amap_h[0], n->wmap_f[1], n->bias[1], nullptr, n->h[1], nullptr, d[1], st)))
        return s;
    if ((s = conv<32, 32, MODE_RELU>(n, n->amap_h[1], n->wmap_f[2], n->bias[2], nullptr, n->h[2], nullptr, d[2], st)))
        return s;
    return conv<32, 16, MODE_OUT>(n, n->amap_h[2], n->wmap_f[3], n->bias[3], nullptr, nullptr, o, d[3], st);
}

template <int CIN, int COUT>
art_status wgrad(art_net *n, const bf16 *g, const bf16 *a, int l, cudaStream_t st)
{
    const LayerDev &L = kLayers[l];
    const int nch = (int)((n->V + WG_CHUNK - 1) / WG_CHUNK);
    wgrad_kernel<CIN, COUT><<<dim3(nch, 27), 128, 0, st>>>(g, a, n->nx, n->ny, n->nz, n->opt.dilation[l], n->part);
    NCK(n, cudaGetLastError());
    bgrad_kernel<COUT><<<nch, COUT * 8, 0, st>>>(g, n->V, n->pb);
    NCK(n, cudaGetLastError());
    const int cnt = 27 * L.cout * L.cin + L.cout;
    gw_reduce_kernel<<<(cnt + 255) / 256, 256, 0, st>>>(n->part, n->pb, nch, L.coutp, L.cinp, L.cout, L.cin,
                                                         n->grad + L.w_off, n->grad + L.b_off);
    NCK(n, cudaGetLastError());
    return ART_OK;
}

// forward + loss + backward: gradients into n->grad, loss into n->loss (device)
art_status forward_backward(art_net *n, const float *t, const float *w, cudaStream_t st)
{
    art_status s;
    if ((s = forward16(n, n->o, st))) return s;
    const int nb = (int)((n->V + 255) / 256);
    loss_grad_kernel<<<nb, 256, 0, st>>>(n->o, t, w, n->V, n->g16, n->lpart);
    NCK(n, cudaGetLastError());
    sum_partials_kernel<<<1, 32, 0, st>>>(n->lpart, nb, 1.0 / (double)n->V, n->loss);
    NCK(n, cudaGetLastError());
    const int *d = n->opt.dilation;
    if ((s = wgrad<32, 16>(n, n->g16, n->h[2], 3, st))) return s;
    if ((s = conv<16, 32, MODE_DGRAD>(n, n->amap_g16, n->wmap_d[3], nullptr, n->h[2], n->gA, nullptr, d[3], st)))
        return s;
    if ((s = wgrad<32, 32>(n, n->gA, n->h[1], 2, st))) return s;
    if ((s = conv<32, 32, MODE_DGRAD>(n, n->amap_gA, n->wmap_d[2], nullptr, n->h[1], n->gB, nullptr, d[2], st)))
        return s;
    if ((s = wgrad<32, 32>(n, n->gB, n->h[0], 1, st))) return s;
    if ((s = conv<32, 32, MODE_DGRAD>(n, n->amap_gB, n->wmap_d[1], nullptr, n->h[0], n->gA, nullptr, d[1], st)))
        return s;
    return wgrad<16, 32>(n, n->gA, n->X16, 0, st);
}

art_status check_err(art_net *n, cudaStream_t st)
{
    int e = 0;
    NCK(n, cudaMemcpyAsync(&e, n->d_err, sizeof(int), cudaMemcpyDeviceToHost, st));
    NCK(n, cudaStreamSynchronize(st));
    if (e) {
        cudaMemsetAsync(n->d_err, 0, sizeof(int), st);
        return nfail(n, ART_E_TIMEOUT, "surrogate convolution: a bounded wait gave up (code " + std::to_string(e) + ")");
    }
    return ART_OK;
}

}  // namespace

// ---------------------------------------------------------------------------
// internal entry points (used by the warm-started iteration)
// ---------------------------------------------------------------------------
art_status artnet_input(art_net *n, int nx, int ny, int nz, void **X16)
{
    art_status s = ensure_workspace(n, nx, ny, nz);
    if (s) return s;
    *X16 = n->X16;
    return ART_OK;
}

art_status artnet_forward(art_net *n, float *o, cudaStream_t st) { return forward16(n, o, st); }

art_status artnet_check(art_net *n, cudaStream_t st) { return check_err(n, st); }
const char *artnet_error(const art_net *n) { return n ? n->err.c_str() : "null network"; }

art_status artnet_coarse(art_ctx *ctx, int f, int nside_c)
{
    const int nx = ctx->grid.nx, ny = ctx->grid.ny, nz = ctx->grid.nz;
    if (f < 1 || nx % f || ny % f || nz % f || nside_c < 1)
        return art_fail(ctx, ART_E_INVALID, "surrogate: grid dimensions must be divisible by the coarse factor");
    const long long V = ctx->ncell;
    const long long Vc = V / ((long long)f * f * f);
    art_sur_bufs &S = ctx->sur;
    if (!ctx->coarse || S.f != f || S.nside != nside_c) {
        if (ctx->coarse) art_destroy(ctx->coarse);
        ctx->coarse = nullptr;
        art_grid gc{nx / f, ny / f, nz / f, ctx->grid.dx_cm * f};
        art_options o;
        art_options_default(&o);
        o.field_form = ART_FIELDS_EPS;
        o.averaging = ctx->opt.averaging;   // the coarse sweep averages as the fine one
        art_status s = art_create(&gc, nside_c, 1, &o, &ctx->coarse);
        if (s != ART_OK) return art_fail(ctx, s, "surrogate: coarse sweep context could not be created");
        S.f = f;
        S.nside = nside_c;
        S.n = 0;   // coarse buffers follow the coarse mesh
    }
    if (S.n != V) {
        void *ptrs[] = {S.kc, S.ec, S.jc, S.o, S.eref, S.nHc, S.yc};
        for (void *p : ptrs)
            if (p) cudaFree(p);
        const int keep_f = S.f, keep_nside = S.nside;
        S = art_sur_bufs{};
        S.f = keep_f;
        S.nside = keep_nside;
        if (cudaMalloc(&S.kc, Vc * 4) != cudaSuccess || cudaMalloc(&S.ec, Vc * 4) != cudaSuccess ||
            cudaMalloc(&S.jc, Vc * 4) != cudaSuccess || cudaMalloc(&S.o, V * 4) != cudaSuccess ||
            cudaMalloc(&S.eref, 16) != cudaSuccess || cudaMalloc(&S.nHc, Vc * 8) != cudaSuccess ||
            cudaMalloc(&S.yc, Vc * 8) != cudaSuccess) {
            cudaGetLastError();
            return art_fail(ctx, ART_E_OOM, "surrogate: scratch allocation failed");
        }
        S.n = V;
    }
    return ART_OK;
}

art_status artnet_surrogate(art_ctx *ctx, art_net *net, int use_net, int f, int nside_c, const float *kap,
                            const float *eps, const double *y, float *jin, float *X32, float *jc_fine, cudaStream_t st)
{
    const int nx = ctx->grid.nx, ny = ctx->grid.ny, nz = ctx->grid.nz;
    art_status s = artnet_coarse(ctx, f, nside_c);
    if (s != ART_OK) return s;
    const long long V = ctx->ncell;
    const long long Vc = V / ((long long)f * f * f);
    art_sur_bufs &S = ctx->sur;
    const int nt = 256;
    restrict_kernel<<<(unsigned)((Vc + nt - 1) / nt), nt, 0, st>>>(kap, eps, nx, ny, nz, f, static_cast<float *>(S.kc),
                                                                   static_cast<float *>(S.ec));
    if (cudaGetLastError() != cudaSuccess) return art_fail(ctx, ART_E_CUDA, "surrogate: restrict launch failed");
    s = art_internal_layout(ctx->coarse, S.kc, S.ec, st);
    if (s == ART_OK) s = art_internal_sweep(ctx->coarse, nullptr, S.jc, nullptr, st);
    if (s != ART_OK) return art_fail(ctx, s, std::string("surrogate: coarse sweep: ") + art_last_error(ctx->coarse));
    unsigned int *eref = static_cast<unsigned int *>(S.eref);
    if (cudaMemsetAsync(eref, 0, sizeof(unsigned int), st) != cudaSuccess)
        return art_fail(ctx, ART_E_CUDA, "surrogate: memset failed");
    max_kernel<<<1024, nt, 0, st>>>(eps, V, eref);
    FeatArgs fa;
    fa.kap = kap;
    fa.eps = eps;
    fa.jc = static_cast<const float *>(S.jc);
    fa.y = y;
    fa.eref_bits = eref;
    fa.nx = nx;
    fa.ny = ny;
    fa.nz = nz;
    fa.f = f;
    fa.X16 = nullptr;
    if (jin && use_net) {
        if (!net) return art_fail(ctx, ART_E_INVALID, "surrogate: no network");
        void *x16 = nullptr;
        s = artnet_input(net, nx, ny, nz, &x16);
        if (s != ART_OK) return art_fail(ctx, s, std::string("surrogate: ") + artnet_error(net));
        fa.X16 = static_cast<bf16 *>(x16);
    }
    fa.X32 = X32;
    fa.jc_fine = jc_fine;
    features_kernel<<<(unsigned)((V + nt - 1) / nt), nt, 0, st>>>(fa);
    if (cudaGetLastError() != cudaSuccess) return art_fail(ctx, ART_E_CUDA, "surrogate: features launch failed");
    if (!jin) return ART_OK;
    float *o = nullptr;
    if (use_net) {
        s = artnet_forward(net, static_cast<float *>(S.o), st);
        if (s != ART_OK) return art_fail(ctx, s, std::string("surrogate: ") + artnet_error(net));
        o = static_cast<float *>(S.o);
    }
    predict_kernel<<<(unsigned)((V + nt - 1) / nt), nt, 0, st>>>(static_cast<const float *>(S.jc), o, nx, ny, nz, f, jin);
    if (cudaGetLastError() != cudaSuccess) return art_fail(ctx, ART_E_CUDA, "surrogate: predict launch failed");
    return ART_OK;
}

art_status artnet_target(art_ctx *ctx, const float *jin, const float *jc_fine, float *t, cudaStream_t st)
{
    const long long V = ctx->ncell;
    target_kernel<<<(unsigned)((V + 255) / 256), 256, 0, st>>>(jin, jc_fine, V,
                                                               static_cast<const unsigned int *>(ctx->sur.eref), t);
    if (cudaGetLastError() != cudaSuccess) return art_fail(ctx, ART_E_CUDA, "surrogate: target launch failed");
    return ART_OK;
}

art_status artnet_weights(art_ctx *ctx, const float *jin, float *w, cudaStream_t st)
{
    const long long V = ctx->ncell;
    const int nb = 256;
    double *part = nullptr;
    if (cudaMalloc(&part, nb * sizeof(double)) != cudaSuccess) {
        cudaGetLastError();
        return art_fail(ctx, ART_E_OOM, "surrogate: weight buffer");
    }
    sum_kernel<<<nb, 256, 0, st>>>(jin, V, part);
    weight_scale_kernel<<<(unsigned)((V + 255) / 256), 256, 0, st>>>(jin, V, part, nb, w);
    const cudaError_t e = cudaGetLastError();
    cudaStreamSynchronize(st);   // the partial buffer is freed below
    cudaFree(part);
    if (e != cudaSuccess) return art_fail(ctx, ART_E_CUDA, "surrogate: weight launch failed");
    return ART_OK;
}

art_status artnet_l1(art_ctx *ctx, const float *a, const float *b, double *err, cudaStream_t st)
{
    const int nb = 256;
    double *part = nullptr;
    if (cudaMalloc(&part, 2 * nb * sizeof(double)) != cudaSuccess) {
        cudaGetLastError();
        return art_fail(ctx, ART_E_OOM, "surrogate: judge buffer");
    }
    l1_kernel<<<nb, 256, 0, st>>>(a, b, ctx->ncell, part);
    std::vector<double> h(2 * nb);
    cudaError_t e = cudaMemcpyAsync(h.data(), part, h.size() * sizeof(double), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    cudaFree(part);
    if (e != cudaSuccess) return art_fail(ctx, ART_E_CUDA, std::string("surrogate: judge: ") + cudaGetErrorString(e));
    double s0 = 0.0, s1 = 0.0;
    for (int i = 0; i < nb; ++i) {
        s0 += h[2 * i];
        s1 += h[2 * i + 1];
    }
    *err = s1 > 0.0 ? s0 / s1 : (s0 > 0.0 ? INFINITY : 0.0);
    return ART_OK;
}

// ---------------------------------------------------------------------------
// C ABI
// ---------------------------------------------------------------------------
extern "C" {

art_status art_net_options_default(art_net_options *o)
{
    if (!o) return ART_E_INVALID;
    std::memset(o, 0, sizeof(*o));
    o->dilation[0] = 1;
    o->dilation[1] = 2;
    o->dilation[2] = 4;
    o->dilation[3] = 8;
    o->seed = 1;
    o->lr = 1e-3;
    o->beta1 = 0.9;
    o->beta2 = 0.999;
    o->adam_eps = 1e-8;
    return ART_OK;
}

art_status art_net_create(const art_net_options *opt, art_net **out)
{
    if (!out) return ART_E_INVALID;
    *out = nullptr;
    art_net_options o;
    if (opt) o = *opt;
    else art_net_options_default(&o);
    for (int l = 0; l < 4; ++l)
        if (o.dilation[l] < 1 || o.dilation[l] > 16) return ART_E_INVALID;
    if (!(o.lr > 0.0) || !(o.beta1 >= 0.0 && o.beta1 < 1.0) || !(o.beta2 >= 0.0 && o.beta2 < 1.0) || !(o.adam_eps >= 0.0))
        return ART_E_INVALID;
    if (!encode_fn()) return ART_E_CUDA;
    art_net *n = new (std::nothrow) art_net();
    if (!n) return ART_E_OOM;
    n->opt = o;
    int dev = 0;
    if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&n->sms, cudaDevAttrMultiProcessorCount, dev);
    cudaGetLastError();
    bool ok = nalloc(&n->params, ART_NET_PARAMS) == cudaSuccess && nalloc(&n->m, ART_NET_PARAMS) == cudaSuccess &&
              nalloc(&n->v, ART_NET_PARAMS) == cudaSuccess && nalloc(&n->grad, ART_NET_PARAMS) == cudaSuccess &&
              nalloc(&n->d_err, 1) == cudaSuccess;
    for (int l = 0; l < 4 && ok; ++l) {
        const LayerDev &L = kLayers[l];
        ok = nalloc(&n->wf[l], 27 * L.coutp * L.cinp) == cudaSuccess && nalloc(&n->bias[l], L.coutp) == cudaSuccess;
        if (ok && l > 0) ok = nalloc(&n->wd[l], 27 * L.coutp * L.cinp) == cudaSuccess;
    }
    if (!ok) {
        cudaGetLastError();
        art_net_destroy(n);
        return ART_E_OOM;
    }
    for (int l = 0; l < 4 && ok; ++l) {
        const LayerDev &L = kLayers[l];
        ok = weight_map(&n->wmap_f[l], n->wf[l], L.cinp, L.coutp);
        if (ok && l > 0) ok = weight_map(&n->wmap_d[l], n->wd[l], L.coutp, L.cinp);
    }
    if (!ok) {
        art_net_destroy(n);
        return ART_E_CUDA;
    }
    // He-normal initial weights, zero biases, last layer x 0.1
    std::vector<float> h(ART_NET_PARAMS, 0.f);
    for (int l = 0; l < 4; ++l) {
        const LayerDev &L = kLayers[l];
        const double sd = std::sqrt(2.0 / (27.0 * L.cin)) * (l == 3 ? 0.1 : 1.0);
        for (long long i = 0; i < 27LL * L.cout * L.cin; ++i)
            h[L.w_off + i] = (float)(sd * normal_at(o.seed, (uint64_t)(L.w_off + i)));
    }
    if (art_net_set_params(n, h.data()) != ART_OK || cudaMemset(n->d_err, 0, sizeof(int)) != cudaSuccess) {
        art_net_destroy(n);
        return ART_E_CUDA;
    }
    *out = n;
    return ART_OK;
}

art_status art_net_destroy(art_net *n)
{
    if (!n) return ART_OK;
    free_workspace(n);
    void *ptrs[] = {n->params, n->m, n->v, n->grad, n->d_err};
    for (void *p : ptrs)
        if (p) cudaFree(p);
    for (int l = 0; l < 4; ++l) {
        if (n->wf[l]) cudaFree(n->wf[l]);
        if (n->wd[l]) cudaFree(n->wd[l]);
        if (n->bias[l]) cudaFree(n->bias[l]);
    }
    delete n;
    return ART_OK;
}

const char *art_net_last_error(const art_net *n) { return artnet_error(n); }

art_status art_net_get_params(art_net *n, float *host)
{
    if (!n || !host) return ART_E_INVALID;
    NCK(n, cudaMemcpy(host, n->params, ART_NET_PARAMS * sizeof(float), cudaMemcpyDeviceToHost));
    return ART_OK;
}

art_status art_net_set_params(art_net *n, const float *host)
{
    if (!n || !host) return ART_E_INVALID;
    for (int i = 0; i < ART_NET_PARAMS; ++i)
        if (!std::isfinite(host[i])) return nfail(n, ART_E_INVALID, "art_net_set_params: non-finite parameter");
    NCK(n, cudaMemcpy(n->params, host, ART_NET_PARAMS * sizeof(float), cudaMemcpyHostToDevice));
    NCK(n, cudaMemset(n->m, 0, ART_NET_PARAMS * sizeof(float)));
    NCK(n, cudaMemset(n->v, 0, ART_NET_PARAMS * sizeof(float)));
    n->step = 0;
    art_status s = pack_weights(n, 0);
    if (s) return s;
    NCK(n, cudaDeviceSynchronize());
    return ART_OK;
}

art_status art_net_forward(art_net *n, int nx, int ny, int nz, const float *X, float *o, void *stream)
{
    if (!n) return ART_E_INVALID;
    if (!X || !o) return nfail(n, ART_E_INVALID, "art_net_forward: null pointer");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    art_status s = ensure_workspace(n, nx, ny, nz);
    if (s) return s;
    pack_input_kernel<<<(unsigned)((n->V + 255) / 256), 256, 0, st>>>(X, n->V, n->X16);
    NCK(n, cudaGetLastError());
    return forward16(n, o, st);
}

art_status art_net_gradients(art_net *n, int nx, int ny, int nz, const float *X, const float *t, const float *w,
                             double *loss, float *grads, void *stream)
{
    if (!n) return ART_E_INVALID;
    if (!X || !t || !loss) return nfail(n, ART_E_INVALID, "art_net_gradients: null pointer");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    art_status s = ensure_workspace(n, nx, ny, nz);
    if (s) return s;
    pack_input_kernel<<<(unsigned)((n->V + 255) / 256), 256, 0, st>>>(X, n->V, n->X16);
    NCK(n, cudaGetLastError());
    if ((s = forward_backward(n, t, w, st))) return s;
    NCK(n, cudaMemcpyAsync(loss, n->loss, sizeof(double), cudaMemcpyDeviceToHost, st));
    if (grads) NCK(n, cudaMemcpyAsync(grads, n->grad, ART_NET_PARAMS * sizeof(float), cudaMemcpyDeviceToHost, st));
    return check_err(n, st);
}

art_status art_net_check(art_net *n, void *stream)
{
    if (!n) return ART_E_INVALID;
    return check_err(n, static_cast<cudaStream_t>(stream));
}

art_status art_net_set_test_stall(art_net *n, int on)
{
    if (!n) return ART_E_INVALID;
    n->test_stall = on != 0;
    return ART_OK;
}

art_status art_net_set_plane_group(art_net *n, int planes)
{
    if (!n) return ART_E_INVALID;
    if (planes != 0 && planes != 1 && planes != 2 && planes != 4)
        return nfail(n, ART_E_INVALID, "art_net_set_plane_group: 0 (auto), 1, 2 or 4");
    n->plane_group = planes;
    return ART_OK;
}

art_status art_net_train(art_net *n, int nx, int ny, int nz, int n_samples, const float *X, const float *t,
                         const float *w, int steps, uint64_t seed, double *loss_hist, void *stream)
{
    if (!n) return ART_E_INVALID;
    if (!X || !t || n_samples < 1 || steps < 0) return nfail(n, ART_E_INVALID, "art_net_train: bad argument");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    art_status s = ensure_workspace(n, nx, ny, nz);
    if (s) return s;
    const long long V = n->V;
    double *d_hist = nullptr;
    if (loss_hist && steps > 0) NCK(n, cudaMalloc(&d_hist, (size_t)steps * sizeof(double)));
    std::vector<int> order(n_samples);
    for (int step = 0; step < steps; ++step) {
        const int k = step % n_samples;
        if (k == 0) {   // new epoch: order by splitmix64 keys of (seed, epoch, sample)
            const uint64_t epoch = (uint64_t)(step / n_samples);
            std::vector<std::pair<uint64_t, int>> key(n_samples);
            for (int i = 0; i < n_samples; ++i) {
                uint64_t z = seed * 0x9E3779B97F4A7C15ull + epoch * 0xD1B54A32D192ED03ull + (uint64_t)i;
                z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
                z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
                key[i] = {z ^ (z >> 31), i};
            }
            std::sort(key.begin(), key.end());
            for (int i = 0; i < n_samples; ++i) order[i] = key[i].second;
        }
        const int smp = order[k];
        pack_input_kernel<<<(unsigned)((V + 255) / 256), 256, 0, st>>>(X + (long long)smp * 4 * V, V, n->X16);
        if (cudaGetLastError() != cudaSuccess) {
            if (d_hist) cudaFree(d_hist);
            return nfail(n, ART_E_CUDA, "art_net_train: launch failed");
        }
        if ((s = forward_backward(n, t + (long long)smp * V, w ? w + (long long)smp * V : nullptr, st))) {
            if (d_hist) cudaFree(d_hist);
            return s;
        }
        if (d_hist) cudaMemcpyAsync(d_hist + step, n->loss, sizeof(double), cudaMemcpyDeviceToDevice, st);
        n->step += 1;
        const double c1 = 1.0 - std::pow(n->opt.beta1, n->step), c2 = 1.0 - std::pow(n->opt.beta2, n->step);
        adam_kernel<<<(ART_NET_PARAMS + 255) / 256, 256, 0, st>>>(n->params, n->m, n->v, n->grad, ART_NET_PARAMS,
                                                                  (float)n->opt.lr, (float)n->opt.beta1,
                                                                  (float)n->opt.beta2, (float)n->opt.adam_eps,
                                                                  (float)c1, (float)c2);
        if ((s = pack_weights(n, st))) {
            if (d_hist) cudaFree(d_hist);
            return s;
        }
    }
    if (d_hist) {
        cudaError_t e = cudaMemcpyAsync(loss_hist, d_hist, (size_t)steps * sizeof(double), cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        cudaFree(d_hist);
        if (e != cudaSuccess) return nfail(n, ART_E_CUDA, std::string("art_net_train: ") + cudaGetErrorString(e));
    }
    return check_err(n, st);
}

art_status art_net_train_step(art_net *n, int nx, int ny, int nz, const float *X, const float *t, const float *w,
                              double *loss, void *stream)
{
    if (!n) return ART_E_INVALID;
    if (!X || !t) return nfail(n, ART_E_INVALID, "art_net_train_step: null pointer");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    art_status s = ensure_workspace(n, nx, ny, nz);
    if (s) return s;
    pack_input_kernel<<<(unsigned)((n->V + 255) / 256), 256, 0, st>>>(X, n->V, n->X16);
    NCK(n, cudaGetLastError());
    if ((s = forward_backward(n, t, w, st))) return s;
    n->step += 1;
    const double c1 = 1.0 - std::pow(n->opt.beta1, n->step), c2 = 1.0 - std::pow(n->opt.beta2, n->step);
    adam_kernel<<<(ART_NET_PARAMS + 255) / 256, 256, 0, st>>>(n->params, n->m, n->v, n->grad, ART_NET_PARAMS,
                                                              (float)n->opt.lr, (float)n->opt.beta1,
                                                              (float)n->opt.beta2, (float)n->opt.adam_eps, (float)c1,
                                                              (float)c2);
    NCK(n, cudaGetLastError());
    if ((s = pack_weights(n, st))) return s;
    if (loss) {
        NCK(n, cudaMemcpyAsync(loss, n->loss, sizeof(double), cudaMemcpyDeviceToHost, st));
        return check_err(n, st);
    }
    return ART_OK;
}


art_status art_train_opts_default(art_train_opts *o)
{
    if (!o) return ART_E_INVALID;
    std::memset(o, 0, sizeof(*o));
    o->steps = 0;
    o->seed = 1;
    o->reset = 0;
    art_net_options_default(&o->net);
    o->stream = nullptr;
    return ART_OK;
}

art_status art_surrogate_train(art_ctx *ctx, const art_dataset *data, const art_train_opts *opt,
                               art_train_report *rep)
{
    if (!ctx) return ART_E_INVALID;
    if (!data || !data->X || !data->t || data->n_samples < 1)
        return art_fail(ctx, ART_E_INVALID, "art_surrogate_train: null dataset, no samples or null X / t");
    if (ctx->grids.size() != 1 || data->nx != ctx->grid.nx || data->ny != ctx->grid.ny || data->nz != ctx->grid.nz)
        return art_fail(ctx, ART_E_INVALID, "art_surrogate_train: the samples must be on the context's grid");
    art_train_opts o;
    if (opt) o = *opt;
    else art_train_opts_default(&o);
    if (o.steps < 0) return art_fail(ctx, ART_E_INVALID, "art_surrogate_train: steps must be >= 0");
    const int steps = o.steps > 0 ? o.steps : 8 * data->n_samples;
    const auto t0 = std::chrono::steady_clock::now();
    if (ctx->net && o.reset) {
        art_net_destroy(ctx->net);
        ctx->net = nullptr;
    }
    if (!ctx->net) {
        art_net *n = nullptr;
        const art_status s = art_net_create(&o.net, &n);
        if (s != ART_OK) return art_fail(ctx, s, "art_surrogate_train: network creation failed");
        ctx->net = n;
    }
    std::vector<double> hist(steps);
    art_status s = art_net_train(ctx->net, data->nx, data->ny, data->nz, data->n_samples, data->X, data->t, data->w,
                                 steps, o.seed, hist.data(), o.stream);
    if (s == ART_OK) s = art_net_check(ctx->net, o.stream);
    if (s != ART_OK) return art_fail(ctx, s, std::string("art_surrogate_train: ") + art_net_last_error(ctx->net));
    if (rep) {
        rep->steps = steps;
        const int ep = std::min(steps, data->n_samples);
        double m0 = 0.0, m1 = 0.0;
        for (int i = 0; i < ep; ++i) {
            m0 += hist[i];
            m1 += hist[steps - ep + i];
        }
        rep->first_epoch_loss = ep ? m0 / ep : 0.0;
        rep->last_epoch_loss = ep ? m1 / ep : 0.0;
        rep->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    }
    return ART_OK;
}

art_status art_surrogate_network(art_ctx *ctx, art_net **out)
{
    if (!ctx || !out) return ART_E_INVALID;
    *out = ctx->net;
    return ART_OK;
}

}  // extern "C"
