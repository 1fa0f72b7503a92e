// art_ablation.cu -- the straightforward thread-per-ray layout of Sec. 3.1,
// kept only to measure what the paper's ray grouping buys (Sec. 5 and its
// figure of performance gains from grouping): every light-ray of a direction
// is one thread that marches the whole box, depositing its path-averaged
// incoming intensity into the cells it crosses.  Rays of one direction share
// cells, so either
//   * mode 0: one launch per direction, deposits by float atomicAdd, or
//   * mode 1: four launches per direction, one per ray group -- the rays
//     starting from the 2D-interleaved columns (j mod 2, k mod 2) -- which
//     never visit a cell twice, so deposits are plain read-modify-writes.
// Directions run one after another on the stream; the launches of a sweep
// are captured once as a CUDA graph and replayed.  Same geometry (segment
// tables) and per-segment arithmetic as the production sweep, in FP32.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <string>
#include <vector>

#include "art.h"
#include "art_ctx.hpp"
#include "art_kernels.cuh"

using namespace art;

namespace {

struct RayArgs {
    const float2 *F;               // (kappa, S) of the direction's class, axis-a layout
    const SegEntry<float> *segs;   // the direction's slab table
    int sa, sb, sc, a;
    int Na, Nb, Nc, nx, ny;
    float w;                       // |n_a| / N_d
    int b_first, c_first, step;    // first starting column of the group and the column stride (1 or 2)
    int nb_rays, n_rays;
    float *jin;
};

// phi(x) = (1 - e^-x)/x times ds, and 1 - e^-x, as in the production sweep:
// the Maclaurin series below x = 1/4, the hardware base-2 exponential above.
__device__ __forceinline__ void ray_coef(float kap, float ds, float &dsph, float &xph)
{
    const float x = kap * ds;
    if (x < 0.25f) {
        float q = fmaf(x, -1.0f / 720.0f, 1.0f / 120.0f);
        q = fmaf(x, q, -1.0f / 24.0f);
        q = fmaf(x, q, 1.0f / 6.0f);
        q = fmaf(x, q, -0.5f);
        q = fmaf(x, q, 1.0f);
        dsph = ds * q;
        xph = x * q;
    } else {
        float e;
        asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(e) : "f"(-1.4426950408889634f * x));
        xph = 1.0f - e;
        dsph = xph / kap;
    }
}

template <bool ATOMIC> __global__ void __launch_bounds__(128) ray_kernel(const RayArgs p)
{
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= p.n_rays) return;
    int b = p.b_first + p.step * (r % p.nb_rays);
    int c = p.c_first + p.step * (r / p.nb_rays);
    float I = 0.0f;   // vacuum boundary
    for (int m = 0; m < p.Na; ++m) {
        const SegEntry<float> e = p.segs[m];
        const int nseg = (e.code & 3) + 1, cf = (e.code >> 2) & 1;
        const int shb = (e.code >> 3) & 1, shc = (e.code >> 4) & 1;
        const int pa = p.sa > 0 ? m : p.Na - 1 - m;
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            if (k >= nseg) break;
            // the ray's column during segment k
            const int cb = k == 0 ? b : (k == 1 ? b + (nseg == 3 ? 1 - cf : shb) : b + 1);
            const int cc = k == 0 ? c : (k == 1 ? c + (nseg == 3 ? cf : shc) : c + 1);
            const float ds = k == 0 ? e.ds1 : (k == 1 ? e.ds2 : e.ds3);
            if (cb < 0 || cc < 0 || cb >= p.Nb || cc >= p.Nc) continue;   // outside the box: vacuum
            const int pb = p.sb > 0 ? cb : p.Nb - 1 - cb;
            const int pc = p.sc > 0 ? cc : p.Nc - 1 - cc;
            const float2 f = p.F[((long long)pa * p.Nc + pc) * p.Nb + pb];
            float dsph, xph;
            ray_coef(f.x, ds, dsph, xph);
            const int x = p.a == 0 ? pa : pb;
            const int y = p.a == 1 ? pa : (p.a == 0 ? pb : pc);
            const int z = p.a == 2 ? pa : pc;
            float *dst = p.jin + ((long long)z * p.ny + y) * p.nx + x;
            const float dep = p.w * I * dsph;
            if (ATOMIC)
                atomicAdd(dst, dep);
            else
                *dst += dep;
            I = fmaf(f.y - I, xph, I);
        }
        b += nseg == 3 ? 1 : shb;
        c += nseg == 3 ? 1 : shc;
    }
}

struct AblationDir {
    int cls;
    long long seg_off;
    float w;
    int Tb, Tc;   // the ray family's total column shifts over the box depth
};

struct AblationPlan {
    std::vector<AblationDir> dirs;
    std::vector<ClassDev> classes;
    cudaGraphExec_t exec[2] = {nullptr, nullptr};
    void *key[2] = {nullptr, nullptr};
    cudaStream_t stream = nullptr;
    cudaEvent_t ev[2] = {nullptr, nullptr};
};

#define ACK(ctx, call)                                                                                \
    do {                                                                                              \
        cudaError_t e_ = (call);                                                                      \
        if (e_ != cudaSuccess) return art_fail(ctx, ART_E_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
    } while (0)

art_status build_plan(art_ctx *ctx, AblationPlan &P)
{
    std::vector<DirDev> dirs(ctx->nd);
    P.classes.resize(ctx->n_classes);
    ACK(ctx, cudaMemcpy(dirs.data(), ctx->d_dirs, dirs.size() * sizeof(DirDev), cudaMemcpyDeviceToHost));
    ACK(ctx, cudaMemcpy(P.classes.data(), ctx->d_classes, P.classes.size() * sizeof(ClassDev),
                        cudaMemcpyDeviceToHost));
    const size_t nsegs = ctx->segs_bytes / sizeof(SegEntry<float>);
    std::vector<SegEntry<float>> segs(nsegs);
    ACK(ctx, cudaMemcpy(segs.data(), ctx->d_segs, nsegs * sizeof(SegEntry<float>), cudaMemcpyDeviceToHost));
    const int nd_all = 12 * ctx->nside * ctx->nside;
    for (int c = 0; c < (int)P.classes.size(); ++c) {
        const ClassDev &C = P.classes[c];
        for (int d = C.dir_begin; d < C.dir_end; ++d) {
            AblationDir A;
            A.cls = c;
            A.seg_off = dirs[d].seg_off;
            A.w = (float)(dirs[d].na / nd_all);
            A.Tb = A.Tc = 0;
            for (int m = 0; m < C.Na; ++m) {
                const int code = segs[A.seg_off + m].code, nseg = (code & 3) + 1;
                A.Tb += nseg == 3 ? 1 : (code >> 3) & 1;
                A.Tc += nseg == 3 ? 1 : (code >> 4) & 1;
            }
            P.dirs.push_back(A);
        }
    }
    return ART_OK;
}

art_status launch_all(art_ctx *ctx, const AblationPlan &P, int mode, float *jin, cudaStream_t st)
{
    ACK(ctx, cudaMemsetAsync(jin, 0, ctx->ncell * sizeof(float), st));
    const float2 *fields = static_cast<const float2 *>(ctx->d_field);
    for (const AblationDir &A : P.dirs) {
        const ClassDev &C = P.classes[A.cls];
        RayArgs r;
        r.F = fields + (long long)C.a * ctx->ncell;
        r.segs = static_cast<const SegEntry<float> *>(ctx->d_segs) + A.seg_off;
        r.sa = C.sa;
        r.sb = C.sb;
        r.sc = C.sc;
        r.a = C.a;
        r.Na = C.Na;
        r.Nb = C.Nb;
        r.Nc = C.Nc;
        r.nx = C.nx;
        r.ny = C.ny;
        r.w = A.w;
        r.jin = jin;
        const int b_lo = -A.Tb, c_lo = -A.Tc;
        for (int g = 0; g < (mode == 0 ? 1 : 4); ++g) {
            if (mode == 0) {
                r.b_first = b_lo;
                r.c_first = c_lo;
                r.step = 1;
                r.nb_rays = C.Nb - b_lo;
                r.n_rays = r.nb_rays * (C.Nc - c_lo);
            } else {
                const int gb = g & 1, gc = g >> 1;
                r.b_first = b_lo + (((gb - b_lo) % 2) + 2) % 2;
                r.c_first = c_lo + (((gc - c_lo) % 2) + 2) % 2;
                r.step = 2;
                r.nb_rays = r.b_first < C.Nb ? (C.Nb - r.b_first + 1) / 2 : 0;
                const int nc_rays = r.c_first < C.Nc ? (C.Nc - r.c_first + 1) / 2 : 0;
                r.n_rays = r.nb_rays * nc_rays;
            }
            if (r.n_rays <= 0) continue;
            const int nt = 128;
            const unsigned nb = (unsigned)((r.n_rays + nt - 1) / nt);
            if (mode == 0)
                ray_kernel<true><<<nb, nt, 0, st>>>(r);
            else
                ray_kernel<false><<<nb, nt, 0, st>>>(r);
            ACK(ctx, cudaGetLastError());
        }
    }
    return ART_OK;
}

}  // namespace

void art_internal_ablation_free(art_ctx *ctx)
{
    AblationPlan *P = static_cast<AblationPlan *>(ctx->ablation);
    if (!P) return;
    for (cudaGraphExec_t &g : P->exec)
        if (g) cudaGraphExecDestroy(g);
    if (P->stream) cudaStreamDestroy(P->stream);
    for (cudaEvent_t e : P->ev)
        if (e) cudaEventDestroy(e);
    delete P;
    ctx->ablation = nullptr;
}

extern "C" art_status art_ablation_sweep(art_ctx *ctx, int mode, float *J_in, void *stream)
{
    if (!ctx) return ART_E_INVALID;
    if (mode != 0 && mode != 1) return art_fail(ctx, ART_E_INVALID, "art_ablation_sweep: mode 0 (atomics) or 1 (groups)");
    if (!J_in) return art_fail(ctx, ART_E_INVALID, "art_ablation_sweep: null output");
    if (ctx->grids.size() != 1 || ctx->prec != ART_FP32 || ctx->nbins != 1 || ctx->opt.field_form != ART_FIELDS_S ||
        ctx->opt.averaging != ART_AVG_PAPER || ctx->opt.dir_end > ctx->opt.dir_begin)
        return art_fail(ctx, ART_E_INVALID,
                        "art_ablation_sweep: single-grid FP32 contexts, one bin, ART_FIELDS_S, the paper's averaging, "
                        "all directions");
    if (!ctx->have_fields) return art_fail(ctx, ART_E_STATE, "art_ablation_sweep: call art_set_fields first");
    if (ctx->wave.on)
        return art_fail(ctx, ART_E_STATE,
                        "art_ablation_sweep: needs a slab-block context (art_options.variant 1-15), whose segment "
                        "tables it marches; this context uses the wavefront sweep");
    for (double v : ctx->i_bc)
        if (v != 0.0) return art_fail(ctx, ART_E_INVALID, "art_ablation_sweep: vacuum boundary only");
    AblationPlan *P = static_cast<AblationPlan *>(ctx->ablation);
    if (!P) {
        P = new AblationPlan();
        ctx->ablation = P;
        art_status s = build_plan(ctx, *P);
        if (s != ART_OK) return s;
        ACK(ctx, cudaStreamCreateWithFlags(&P->stream, cudaStreamNonBlocking));
        ACK(ctx, cudaEventCreateWithFlags(&P->ev[0], cudaEventDisableTiming));
        ACK(ctx, cudaEventCreateWithFlags(&P->ev[1], cudaEventDisableTiming));
    }
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (P->exec[mode] && P->key[mode] != J_in) {
        cudaGraphExecDestroy(P->exec[mode]);
        P->exec[mode] = nullptr;
    }
    if (!P->exec[mode]) {
        cudaGraph_t graph = nullptr;
        ACK(ctx, cudaStreamBeginCapture(P->stream, cudaStreamCaptureModeThreadLocal));
        const art_status s = launch_all(ctx, *P, mode, J_in, P->stream);
        const cudaError_t e = cudaStreamEndCapture(P->stream, &graph);
        if (s != ART_OK || e != cudaSuccess) {
            if (graph) cudaGraphDestroy(graph);
            cudaGetLastError();
            return s != ART_OK ? s : art_fail(ctx, ART_E_CUDA, std::string("graph capture: ") + cudaGetErrorString(e));
        }
        const cudaError_t ei = cudaGraphInstantiate(&P->exec[mode], graph, 0);
        cudaGraphDestroy(graph);
        if (ei != cudaSuccess) {
            P->exec[mode] = nullptr;
            return art_fail(ctx, ART_E_CUDA, std::string("graph instantiate: ") + cudaGetErrorString(ei));
        }
        P->key[mode] = J_in;
    }
    // order the replay after `stream`'s work and `stream`'s later work after it
    ACK(ctx, cudaEventRecord(P->ev[0], st));
    ACK(ctx, cudaStreamWaitEvent(P->stream, P->ev[0], 0));
    ACK(ctx, cudaGraphLaunch(P->exec[mode], P->stream));
    ACK(ctx, cudaEventRecord(P->ev[1], P->stream));
    ACK(ctx, cudaStreamWaitEvent(st, P->ev[1], 0));
    return ART_OK;
}
