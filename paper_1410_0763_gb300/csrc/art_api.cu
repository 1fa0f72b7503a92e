// art_api.cu -- C ABI of libart (see include/art.h): context set-up, device
// memory, launches of the slab-block sweep and the partial reduction.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "art.h"
#include "art_geometry.hpp"
#include "art_kernels.cuh"

using namespace art;

#include "art_ctx.hpp"

art_status art_fail(art_ctx *ctx, art_status st, const std::string &msg)
{
    if (ctx) ctx->err = msg;
    return st;
}

namespace {

art_status fail(art_ctx *ctx, art_status st, const std::string &msg) { return art_fail(ctx, st, msg); }

#define CK(ctx, call)                                                                             \
    do {                                                                                          \
        cudaError_t e_ = (call);                                                                  \
        if (e_ != cudaSuccess)                                                                    \
            return fail(ctx, e_ == cudaErrorMemoryAllocation ? ART_E_OOM : ART_E_CUDA,            \
                        std::string(#call) + ": " + cudaGetErrorString(e_));                      \
    } while (0)

template <typename T> art_status dev_alloc(art_ctx *ctx, T **p, size_t bytes)
{
    void *q = nullptr;
    cudaError_t e = cudaMalloc(&q, bytes ? bytes : 16);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(ctx, e == cudaErrorMemoryAllocation ? ART_E_OOM : ART_E_CUDA,
                    std::string("cudaMalloc(") + std::to_string(bytes) + "): " + cudaGetErrorString(e));
    }
    ctx->dev_bytes += (long long)bytes;
    *p = static_cast<T *>(q);
    return ART_OK;
}

template <typename real, int TB, int TC, int BLK, int NT, int KP, int MINB>
cudaError_t launch_sweep(const void *args, int nwork, cudaStream_t st)
{
    const SweepArgs<real> &a = *static_cast<const SweepArgs<real> *>(args);
    const size_t sm = SweepShape<TB, TC, BLK, NT, KP>::template bytes<real>();
    auto kern = sweep_block_kernel<real, TB, TC, BLK, NT, KP, MINB>;
    if (sm > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        if (e != cudaSuccess) return e;
    }
    kern<<<nwork, NT, sm, st>>>(a);
    return cudaGetLastError();
}

// Sweep-kernel variants compiled into the library: tile (b x c), slab block,
// threads, direction pairs per exchange group, min CTAs per SM.  Index + 1 is
// the value of art_options.variant that selects one (0 = default).
struct KVariant {
    int prec, tb, tc, blk, nt, kp, minb;
    cudaError_t (*launch)(const void *, int, cudaStream_t);
};
#define ART_V(real, pr, tb, tc, blk, nt, kp, mb) \
    {pr, tb, tc, blk, nt, kp, mb, &launch_sweep<real, tb, tc, blk, nt, kp, mb>}
const KVariant kVariants[] = {
    ART_V(float, ART_FP32, 32, 16, 4, 256, 2, 3),   //  1: default FP32
    ART_V(float, ART_FP32, 32, 8, 4, 256, 2, 3),    //  2
    ART_V(float, ART_FP32, 32, 16, 4, 256, 1, 4),   //  3
    ART_V(float, ART_FP32, 32, 16, 4, 256, 3, 2),   //  4
    ART_V(float, ART_FP32, 32, 16, 2, 256, 2, 3),   //  5
    ART_V(float, ART_FP32, 32, 16, 4, 128, 2, 4),   //  6
    ART_V(float, ART_FP32, 32, 32, 4, 512, 2, 1),   //  7
    ART_V(float, ART_FP32, 64, 16, 4, 512, 2, 1),   //  8
    ART_V(float, ART_FP32, 32, 16, 8, 256, 1, 2),   //  9
    ART_V(float, ART_FP32, 32, 8, 4, 128, 2, 5),    // 10
    ART_V(double, ART_FP64, 16, 16, 4, 128, 1, 1),  // 11: default FP64
};
#undef ART_V
const int kNumVariants = int(sizeof(kVariants) / sizeof(kVariants[0]));

struct HostTables {
    std::vector<ClassDev> classes;
    std::vector<DirDev> dirs;
    std::vector<SlabGeom> geo;    // concatenated per class-sorted direction
    std::vector<int> part_axis;
    std::vector<WorkItem> work;
    long long plane_elems = 0;
    long long seg_count = 0;
};

void build_tables(const art_ctx *ctx, const std::vector<double> &xyz, HostTables &t)
{
    const int dims[3] = {ctx->grid.nx, ctx->grid.ny, ctx->grid.nz};
    std::vector<Frame> fr(ctx->nd);
    for (int d = 0; d < ctx->nd; ++d) fr[d] = frame_of(&xyz[3 * d], ctx->opt.tie_tol);
    long long seg_off = 0, plane_off = 0;
    for (int cls = 0; cls < 24; ++cls) {
        std::vector<int> members;
        for (int d = 0; d < ctx->nd; ++d)
            if (fr[d].cls == cls) members.push_back(d);
        if (members.empty()) continue;
        // Order within the class: by column drift per slab block along b, then
        // c, then RING index.  Directions the kernel takes together then have
        // similar upstream cones.  The order is fixed, so sums stay deterministic.
        auto drift = [&](double q) { return (int)std::floor(q * ctx->BLK + 0.5); };
        std::stable_sort(members.begin(), members.end(), [&](int x, int y) {
            const int bx = drift(fr[x].qb), by = drift(fr[y].qb);
            if (bx != by) return bx < by;
            return drift(fr[x].qc) < drift(fr[y].qc);
        });
        const Frame &f0 = fr[members[0]];
        ClassDev C;
        C.a = f0.a;
        C.sa = f0.sa;
        C.sb = f0.sb;
        C.sc = f0.sc;
        C.Na = dims[f0.a];
        C.Nb = dims[f0.b];
        C.Nc = dims[f0.c];
        C.dir_begin = (int)t.dirs.size();
        C.dir_end = C.dir_begin + (int)members.size();
        C.part0 = (int)t.part_axis.size();
        const int split = std::min<int>(ctx->split, (int)members.size());
        for (int g = 0; g < ctx->split; ++g) t.part_axis.push_back(f0.a);
        (void)split;
        const int ci = (int)t.classes.size();
        t.classes.push_back(C);
        for (int d : members) {
            std::vector<SlabGeom> g;
            slab_geometry(fr[d], C.Na, g);
            DirDev D;
            D.seg_off = seg_off;
            D.plane_off = plane_off;
            D.na = fr[d].na;
            t.dirs.push_back(D);
            for (const SlabGeom &s : g) {
                t.geo.push_back(s);
                t.seg_count += (long long)s.nonzero * C.Nb * C.Nc;
            }
            seg_off += C.Na;
            plane_off += (long long)C.Nb * C.Nc;
        }
        for (int pc = 0; pc < C.Nc; pc += ctx->TC)
            for (int pb = 0; pb < C.Nb; pb += ctx->TB)
                for (int g = 0; g < ctx->split; ++g) t.work.push_back(WorkItem{ci, pb, pc, g});
    }
    t.plane_elems = plane_off;
}

template <typename real> std::vector<SegEntry<real>> pack_segs(const std::vector<SlabGeom> &geo)
{
    std::vector<SegEntry<real>> out(geo.size());
    for (size_t i = 0; i < geo.size(); ++i) {
        const SlabGeom &g = geo[i];
        out[i].ds1 = real(g.ds[0]);
        out[i].ds2 = real(g.ds[1]);
        out[i].ds3 = real(g.ds[2]);
        out[i].code = (g.nseg - 1) | (g.cfirst << 2) | (g.shb << 3) | (g.shc << 4);
    }
    return out;
}

template <typename real> art_status do_sweep(art_ctx *ctx, real *J, real *Jin, real *gam, cudaStream_t st)
{
    using v2 = typename Vec2<real>::type;
    const long long n = ctx->ncell;
    v2 *fields = static_cast<v2 *>(ctx->d_field);
    real *planes[2] = {static_cast<real *>(ctx->d_plane[0]), static_cast<real *>(ctx->d_plane[1])};
    for (int b = 0; b < ctx->nbins; ++b) {
        SweepArgs<real> a;
        a.field0 = fields + (0LL * ctx->nbins + b) * n;
        a.field1 = fields + (1LL * ctx->nbins + b) * n;
        a.field2 = fields + (2LL * ctx->nbins + b) * n;
        a.jpart = static_cast<real *>(ctx->d_jpart);
        a.nx = ctx->grid.nx;
        a.ny = ctx->grid.ny;
        a.nz = ctx->grid.nz;
        a.segs = static_cast<const SegEntry<real> *>(ctx->d_segs);
        a.dirs = ctx->d_dirs;
        a.classes = ctx->d_classes;
        a.work = ctx->d_work;
        a.ncell = n;
        a.split = ctx->split;
        a.field_form = ctx->opt.field_form;
        cudaEvent_t e0 = nullptr, e1 = nullptr, e2 = nullptr;
        if (ctx->profiling) {
            CK(ctx, cudaEventCreate(&e0));
            CK(ctx, cudaEventCreate(&e1));
            CK(ctx, cudaEventCreate(&e2));
            ctx->ev.push_back(e0);
            ctx->ev.push_back(e1);
            ctx->ev.push_back(e2);
            CK(ctx, cudaEventRecord(e0, st));
        }
        for (int k = 0; k < ctx->nblocks; ++k) {
            a.kblock = k;
            a.plane_in = planes[k & 1];
            a.plane_out = planes[(k + 1) & 1];
            CK(ctx, kVariants[ctx->variant].launch(&a, ctx->n_work, st));
        }
        if (ctx->profiling) CK(ctx, cudaEventRecord(e1, st));
        ReduceArgs<real> r;
        r.jpart = static_cast<const real *>(ctx->d_jpart);
        r.field_nat = fields + (2LL * ctx->nbins + b) * n;
        r.n_part = ctx->n_part;
        r.ncell = n;
        r.inv_nd = real(1.0 / ctx->nd);
        r.gamma_coef = real(4.0 * M_PI * ctx->G[b]);
        r.gamma_accum = b > 0;
        r.field_form = ctx->opt.field_form;
        r.Jin = Jin ? Jin + (long long)b * n : nullptr;
        r.J = J ? J + (long long)b * n : nullptr;
        r.gamma = gam;
        const int nt = 256;
        reduce_kernel<real><<<(unsigned)((n + nt - 1) / nt), nt, 0, st>>>(r);
        CK(ctx, cudaGetLastError());
        if (ctx->profiling) CK(ctx, cudaEventRecord(e2, st));
    }
    return ART_OK;
}

}  // namespace

art_status art_internal_sweep(art_ctx *ctx, void *J, void *J_in, void *gamma, cudaStream_t st)
{
    if (ctx->prec == ART_FP64)
        return do_sweep<double>(ctx, static_cast<double *>(J), static_cast<double *>(J_in),
                                static_cast<double *>(gamma), st);
    return do_sweep<float>(ctx, static_cast<float *>(J), static_cast<float *>(J_in), static_cast<float *>(gamma), st);
}

art_status art_internal_layout(art_ctx *ctx, const void *kd, const void *sd, cudaStream_t st)
{
    const long long nc = ctx->ncell;
    const int nt = 256;
    const unsigned lb = (unsigned)((nc + nt - 1) / nt);
    for (int b = 0; b < ctx->nbins; ++b) {
        if (ctx->prec == ART_FP64) {
            double2 *f = static_cast<double2 *>(ctx->d_field);
            const double *k = static_cast<const double *>(kd) + (long long)b * nc;
            const double *s = static_cast<const double *>(sd) + (long long)b * nc;
            layout_kernel<double><<<lb, nt, 0, st>>>(k, s, f + (0LL * ctx->nbins + b) * nc, f + (1LL * ctx->nbins + b) * nc,
                                                     f + (2LL * ctx->nbins + b) * nc, ctx->grid.nx, ctx->grid.ny, ctx->grid.nz);
        } else {
            float2 *f = static_cast<float2 *>(ctx->d_field);
            const float *k = static_cast<const float *>(kd) + (long long)b * nc;
            const float *s = static_cast<const float *>(sd) + (long long)b * nc;
            layout_kernel<float><<<lb, nt, 0, st>>>(k, s, f + (0LL * ctx->nbins + b) * nc, f + (1LL * ctx->nbins + b) * nc,
                                                    f + (2LL * ctx->nbins + b) * nc, ctx->grid.nx, ctx->grid.ny, ctx->grid.nz);
        }
        CK(ctx, cudaGetLastError());
    }
    ctx->have_fields = true;
    return ART_OK;
}

extern "C" {

art_status art_options_default(art_options *opt)
{
    if (!opt) return ART_E_INVALID;
    std::memset(opt, 0, sizeof(*opt));
    opt->precision = ART_FP32;
    opt->averaging = ART_AVG_PAPER;
    opt->field_form = ART_FIELDS_S;
    opt->tie_tol = 1e-12;
    return ART_OK;
}

art_status art_create(const art_grid *grid, int n_side, int nu_bins, const art_options *opt,
                      art_ctx **out)
{
    if (!out) return ART_E_INVALID;
    *out = nullptr;
    if (!grid || grid->nx < 1 || grid->ny < 1 || grid->nz < 1 || n_side < 1 || nu_bins < 1)
        return ART_E_INVALID;
    if ((long long)grid->nx * grid->ny * grid->nz > (1LL << 31) || n_side > 1024) return ART_E_INVALID;
    art_ctx *ctx = new (std::nothrow) art_ctx();
    if (!ctx) return ART_E_OOM;
    ctx->grid = *grid;
    ctx->nside = n_side;
    ctx->nbins = nu_bins;
    if (opt) ctx->opt = *opt;
    else art_options_default(&ctx->opt);
    if (!(ctx->opt.tie_tol >= 0.0) || ctx->opt.tie_tol > 1e-3) ctx->opt.tie_tol = 1e-12;
    if (ctx->opt.precision != ART_FP32 && ctx->opt.precision != ART_FP64) {
        delete ctx;
        return ART_E_INVALID;
    }
    if (ctx->opt.averaging != ART_AVG_PAPER ||
        (ctx->opt.field_form != ART_FIELDS_S && ctx->opt.field_form != ART_FIELDS_EPS)) {
        delete ctx;
        return ART_E_INVALID;
    }
    ctx->prec = ctx->opt.precision;
    ctx->rsz = ctx->prec == ART_FP64 ? 8 : 4;
    ctx->ncell = (long long)grid->nx * grid->ny * grid->nz;
    ctx->nd = 12 * n_side * n_side;
    ctx->G.assign(nu_bins, 0.0);

    // kernel variant
    {
        int pick = -1;
        if (ctx->opt.variant > 0) {
            pick = ctx->opt.variant - 1;
            if (pick >= kNumVariants || kVariants[pick].prec != ctx->prec) pick = -2;
        } else {
            // measured on GB300: the 32 x 8 tile wins below ~100^3 cells
            // (more CTAs per launch), the 32 x 16 tile above
            const int prefer = (ctx->prec == ART_FP32 && ctx->ncell < 100LL * 100 * 100 && !ctx->opt.tile_b &&
                                !ctx->opt.tile_c && !ctx->opt.slab)
                                   ? 1
                                   : -1;
            if (prefer >= 0) pick = prefer;
            for (int v = 0; v < kNumVariants && pick == -1; ++v) {
                const KVariant &k = kVariants[v];
                if (k.prec != ctx->prec) continue;
                if ((ctx->opt.tile_b && k.tb != ctx->opt.tile_b) || (ctx->opt.tile_c && k.tc != ctx->opt.tile_c) ||
                    (ctx->opt.slab && k.blk != ctx->opt.slab))
                    continue;
                pick = v;
            }
        }
        if (pick < 0) {
            delete ctx;
            return ART_E_INVALID;
        }
        const KVariant &k = kVariants[pick];
        ctx->variant = pick;
        ctx->TB = k.tb;
        ctx->TC = k.tc;
        ctx->BLK = k.blk;
        ctx->NT = k.nt;
        ctx->KP = k.kp;
    }

    std::vector<double> xyz;
    healpix_directions(n_side, xyz);
    // direction groups per class: enough CTAs to cover the GPU at least twice
    {
        int dev = 0, sms = 152;
        if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        cudaGetLastError();
        if (ctx->opt.dir_split > 0) {
            ctx->split = ctx->opt.dir_split;
        } else {
            ctx->split = 1;
            HostTables probe;
            build_tables(ctx, xyz, probe);
            const int base = (int)probe.work.size();
            const int per_class = std::max(1, ctx->nd / std::max<int>(1, (int)probe.classes.size()));
            while (base * ctx->split < 2 * sms && ctx->split * 2 <= per_class) ctx->split *= 2;
        }
    }
    HostTables t;
    build_tables(ctx, xyz, t);
    ctx->n_classes = (int)t.classes.size();
    ctx->n_part = (int)t.part_axis.size();
    ctx->n_work = (int)t.work.size();
    ctx->seg_count = t.seg_count;
    ctx->plane_elems = t.plane_elems;
    int maxNa = 0;
    for (const ClassDev &c : t.classes) maxNa = std::max(maxNa, c.Na);
    ctx->nblocks = (maxNa + ctx->BLK - 1) / ctx->BLK;

    const size_t rs = ctx->rsz, n = (size_t)ctx->ncell;
    art_status st;
#define ALLOC(ptr, bytes)                                      \
    do {                                                       \
        if ((st = dev_alloc(ctx, &(ptr), (bytes))) != ART_OK) { \
            art_ctx *c_ = ctx;                                 \
            std::string m_ = c_->err;                          \
            art_destroy(c_);                                   \
            (void)m_;                                          \
            return st;                                         \
        }                                                      \
    } while (0)
    ALLOC(ctx->d_field, 3 * (size_t)nu_bins * n * 2 * rs);
    ALLOC(ctx->d_plane[0], (size_t)ctx->plane_elems * rs);
    ALLOC(ctx->d_plane[1], (size_t)ctx->plane_elems * rs);
    ALLOC(ctx->d_jpart, (size_t)ctx->n_part * n * rs);
    ALLOC(ctx->d_segs, t.geo.size() * (ctx->prec == ART_FP64 ? sizeof(SegEntry<double>) : sizeof(SegEntry<float>)));
    ALLOC(ctx->d_dirs, t.dirs.size() * sizeof(DirDev));
    ALLOC(ctx->d_classes, t.classes.size() * sizeof(ClassDev));
    ALLOC(ctx->d_work, t.work.size() * sizeof(WorkItem));
    ALLOC(ctx->d_part_axis, t.part_axis.size() * sizeof(int));
    ALLOC(ctx->d_stage, 2 * (size_t)nu_bins * n * rs);
    ALLOC(ctx->d_out, (2 * (size_t)nu_bins + 1) * n * rs);
    ALLOC(ctx->d_flag, sizeof(int));
#undef ALLOC
    cudaError_t e = cudaSuccess;
    if (ctx->prec == ART_FP64) {
        auto s = pack_segs<double>(t.geo);
        e = cudaMemcpy(ctx->d_segs, s.data(), s.size() * sizeof(s[0]), cudaMemcpyHostToDevice);
    } else {
        auto s = pack_segs<float>(t.geo);
        e = cudaMemcpy(ctx->d_segs, s.data(), s.size() * sizeof(s[0]), cudaMemcpyHostToDevice);
    }
    if (e == cudaSuccess) e = cudaMemcpy(ctx->d_dirs, t.dirs.data(), t.dirs.size() * sizeof(DirDev), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(ctx->d_classes, t.classes.data(), t.classes.size() * sizeof(ClassDev), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(ctx->d_work, t.work.data(), t.work.size() * sizeof(WorkItem), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(ctx->d_part_axis, t.part_axis.data(), t.part_axis.size() * sizeof(int), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        art_destroy(ctx);
        return ART_E_CUDA;
    }
    *out = ctx;
    return ART_OK;
}

art_status art_band_integral(double sigma0, double h, double nu0, double nu_lo, double nu_hi, double *G)
{
    if (!G || !(sigma0 > 0.0) || !(h > 0.0) || !(nu0 > 0.0) || !(nu_lo > 0.0) || !(nu_hi >= nu_lo) ||
        !std::isfinite(sigma0 * h * nu0 * nu_lo * nu_hi))
        return ART_E_INVALID;
    // sigma/(h nu) = sigma0 nu0^3 / (h nu^4); its antiderivative is -sigma0 nu0^3 / (3 h nu^3)
    const double r_lo = nu0 / nu_lo, r_hi = nu0 / nu_hi;
    *G = sigma0 / (3.0 * h) * (r_lo * r_lo * r_lo - r_hi * r_hi * r_hi);
    return ART_OK;
}

art_status art_count_segments(const art_grid *grid, int n_side, double tie_tol, int64_t *out)
{
    if (!grid || !out || grid->nx < 1 || grid->ny < 1 || grid->nz < 1 || n_side < 1 || n_side > 1024)
        return ART_E_INVALID;
    const int dims[3] = {grid->nx, grid->ny, grid->nz};
    std::vector<double> xyz;
    healpix_directions(n_side, xyz);
    int64_t total = 0;
    std::vector<SlabGeom> g;
    for (size_t d = 0; d < xyz.size() / 3; ++d) {
        const Frame f = frame_of(&xyz[3 * d], tie_tol >= 0.0 ? tie_tol : 1e-12);
        slab_geometry(f, dims[f.a], g);
        for (const SlabGeom &s : g) total += (int64_t)s.nonzero * dims[f.b] * dims[f.c];
    }
    *out = total;
    return ART_OK;
}

art_status art_profile_enable(art_ctx *ctx, int enable)
{
    if (!ctx) return ART_E_INVALID;
    ctx->profiling = enable != 0;
    return ART_OK;
}

art_status art_profile_read(art_ctx *ctx, art_profile *out, int reset)
{
    if (!ctx || !out) return ART_E_INVALID;
    for (size_t i = 0; i + 2 < ctx->ev.size(); i += 3) {
        float a = 0.f, b = 0.f;
        CK(ctx, cudaEventSynchronize(ctx->ev[i + 2]));
        CK(ctx, cudaEventElapsedTime(&a, ctx->ev[i], ctx->ev[i + 1]));
        CK(ctx, cudaEventElapsedTime(&b, ctx->ev[i + 1], ctx->ev[i + 2]));
        out->sweep_ms += a;
        out->sweep_launches += ctx->nblocks;
        out->reduce_ms += b;
        out->reduce_launches += 1;
    }
    if (reset) {
        for (cudaEvent_t e : ctx->ev) cudaEventDestroy(e);
        ctx->ev.clear();
    }
    return ART_OK;
}

art_status art_destroy(art_ctx *ctx)
{
    if (!ctx) return ART_OK;
    for (cudaEvent_t e : ctx->ev) cudaEventDestroy(e);
    void *ptrs[] = {ctx->d_field, ctx->d_plane[0], ctx->d_plane[1], ctx->d_jpart, ctx->d_segs,
                    ctx->d_dirs, ctx->d_classes, ctx->d_work, ctx->d_part_axis, ctx->d_stage,
                    ctx->d_out, ctx->d_flag, ctx->it.nH, ctx->it.y, ctx->it.y0, ctx->it.gpt, ctx->it.kap,
                    ctx->it.eps, ctx->it.jin, ctx->it.resid, ctx->it.src};
    for (void *p : ptrs)
        if (p) cudaFree(p);
    delete ctx;
    return ART_OK;
}

const char *art_last_error(const art_ctx *ctx) { return ctx ? ctx->err.c_str() : "null context"; }

art_status art_get_stats(const art_ctx *ctx, art_sweep_stats *s)
{
    if (!ctx || !s) return ART_E_INVALID;
    s->segments = ctx->seg_count * ctx->nbins;
    s->n_dirs = ctx->nd;
    s->n_classes = ctx->n_classes;
    s->launches = ctx->nblocks + 1;
    s->ctas_per_launch = ctx->n_work;
    s->tile_b = ctx->TB;
    s->tile_c = ctx->TC;
    s->slab = ctx->BLK;
    s->dir_split = ctx->split;
    s->device_bytes = ctx->dev_bytes;
    s->variant = ctx->variant + 1;
    s->group = 2 * ctx->KP;
    return ART_OK;
}

art_status art_set_fields(art_ctx *ctx, const void *kappa, const void *src, int on_device, void *stream)
{
    if (!ctx) return ART_E_INVALID;
    if (!kappa || !src) return fail(ctx, ART_E_INVALID, "art_set_fields: null field pointer");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const long long n = ctx->ncell * ctx->nbins;
    const size_t bytes = (size_t)n * ctx->rsz;
    const void *kd = kappa, *sd = src;
    if (!on_device) {
        char *stage = static_cast<char *>(ctx->d_stage);
        CK(ctx, cudaMemcpyAsync(stage, kappa, bytes, cudaMemcpyHostToDevice, st));
        CK(ctx, cudaMemcpyAsync(stage + bytes, src, bytes, cudaMemcpyHostToDevice, st));
        kd = stage;
        sd = stage + bytes;
    }
    CK(ctx, cudaMemsetAsync(ctx->d_flag, 0, sizeof(int), st));
    const int nt = 256;
    const unsigned nb = (unsigned)std::min<long long>((n + nt - 1) / nt, 4096);
    if (ctx->prec == ART_FP64)
        validate_kernel<double><<<nb, nt, 0, st>>>(static_cast<const double *>(kd), static_cast<const double *>(sd), n, ctx->d_flag);
    else
        validate_kernel<float><<<nb, nt, 0, st>>>(static_cast<const float *>(kd), static_cast<const float *>(sd), n, ctx->d_flag);
    CK(ctx, cudaGetLastError());
    int flag = 0;
    CK(ctx, cudaMemcpyAsync(&flag, ctx->d_flag, sizeof(int), cudaMemcpyDeviceToHost, st));
    CK(ctx, cudaStreamSynchronize(st));
    if (flag & 1) return fail(ctx, ART_E_INVALID, "art_set_fields: kappa negative or not finite");
    if (flag & 2) return fail(ctx, ART_E_INVALID, "art_set_fields: source term not finite");
    return art_internal_layout(ctx, kd, sd, st);
}

art_status art_set_band(art_ctx *ctx, const double *G)
{
    if (!ctx) return ART_E_INVALID;
    if (!G) return fail(ctx, ART_E_INVALID, "art_set_band: null pointer");
    for (int b = 0; b < ctx->nbins; ++b) {
        if (!std::isfinite(G[b])) return fail(ctx, ART_E_INVALID, "art_set_band: non-finite band integral");
        ctx->G[b] = G[b];
    }
    return ART_OK;
}

art_status art_sweep(art_ctx *ctx, void *J, void *J_in, void *gamma, int on_device, void *stream)
{
    if (!ctx) return ART_E_INVALID;
    if (!ctx->have_fields) return fail(ctx, ART_E_STATE, "art_sweep: call art_set_fields first");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const long long nb = ctx->ncell * ctx->nbins;
    const size_t rs = ctx->rsz;
    char *o = static_cast<char *>(ctx->d_out);
    void *dJ = J, *dJin = J_in, *dG = gamma;
    if (!on_device) {
        dJ = J ? o : nullptr;
        dJin = J_in ? o + nb * rs : nullptr;
        dG = gamma ? o + 2 * nb * rs : nullptr;
    }
    art_status s;
    if (ctx->prec == ART_FP64)
        s = do_sweep<double>(ctx, static_cast<double *>(dJ), static_cast<double *>(dJin), static_cast<double *>(dG), st);
    else
        s = do_sweep<float>(ctx, static_cast<float *>(dJ), static_cast<float *>(dJin), static_cast<float *>(dG), st);
    if (s != ART_OK) return s;
    if (!on_device) {
        if (J) CK(ctx, cudaMemcpyAsync(J, dJ, nb * rs, cudaMemcpyDeviceToHost, st));
        if (J_in) CK(ctx, cudaMemcpyAsync(J_in, dJin, nb * rs, cudaMemcpyDeviceToHost, st));
        if (gamma) CK(ctx, cudaMemcpyAsync(gamma, dG, ctx->ncell * rs, cudaMemcpyDeviceToHost, st));
        CK(ctx, cudaStreamSynchronize(st));
    }
    return ART_OK;
}

}  // extern "C"
