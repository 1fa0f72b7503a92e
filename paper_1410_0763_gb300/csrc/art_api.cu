// art_api.cu -- C ABI of libart (see include/art.h): context set-up for one
// grid or a batch of grids, device memory, launches of the slab-block sweep
// (one CTA per work item, or persistent CTAs on a work queue; optionally
// replayed as a CUDA graph), the partial reduction and the variant autotuner.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "art.h"
#include "art_net.h"
#include "art_geometry.hpp"
#include "art_kernels.cuh"

using namespace art;

// The exact-average kernels live in art_sweep_exact.cu (one instantiation per
// variant of art_variants.inc).
template <typename real, int TB, int TC, int BLK, int NT, int KP, int MINB>
cudaError_t art_launch_exact(const cudaLaunchConfig_t &cfg, const SweepArgs<real> &a);
template <typename real, int TB, int TC, int BLK, int NT, int KP, int MINB> cudaError_t art_prepare_exact(int smem);

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

// Fixed-order Kahan sum of n_parts partial fields (direction shards).
__global__ void shard_sum_kernel(const float *__restrict__ parts, int n_parts, long long n, float *__restrict__ out)
{
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    float s = 0.f, c = 0.f;
    for (int k = 0; k < n_parts; ++k) kahan_add(s, c, parts[(long long)k * n + i]);
    out[i] = s - c;
}

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

template <typename T> void dev_free(art_ctx *ctx, T *&p, size_t &bytes)
{
    if (p) {
        cudaFree(p);
        ctx->dev_bytes -= (long long)bytes;
    }
    p = nullptr;
    bytes = 0;
}

// Launch one slab-block sweep.  The shared-memory attribute is set by
// prepare_sweep (outside any stream capture).  With `early`, the launch may
// begin while the previous kernel on the stream drains (programmatic
// dependent launch): its CTAs stage the fields and segment tables, which no
// kernel of the sweep writes, and wait for the previous launch to complete
// before they touch the intensity planes or the J partials.
template <typename real, int TB, int TC, int BLK, int NT, int KP, int MINB>
cudaError_t launch_sweep(const void *args, int nctas, cudaStream_t st, bool early)
{
    const SweepArgs<real> &a = *static_cast<const SweepArgs<real> *>(args);
    const size_t sm = SweepShape<TB, TC, BLK, NT, KP>::template bytes<real>();
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)nctas);
    cfg.blockDim = dim3(NT);
    cfg.dynamicSmemBytes = sm;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = early ? 1 : 0;
    if (a.averaging) return art_launch_exact<real, TB, TC, BLK, NT, KP, MINB>(cfg, a);
    if (a.counter) return cudaLaunchKernelEx(&cfg, sweep_queue_kernel<real, TB, TC, BLK, NT, KP, MINB>, a);
    return cudaLaunchKernelEx(&cfg, sweep_block_kernel<real, TB, TC, BLK, NT, KP, MINB>, a);
}

// Allow the variant's dynamic shared memory; returns its resident CTAs per SM
// (0 on error).
template <typename real, int TB, int TC, int BLK, int NT, int KP, int MINB> int prepare_sweep()
{
    const size_t sm = SweepShape<TB, TC, BLK, NT, KP>::template bytes<real>();
    auto kern = sweep_block_kernel<real, TB, TC, BLK, NT, KP, MINB>;
    auto qkern = sweep_queue_kernel<real, TB, TC, BLK, NT, KP, MINB>;
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm) != cudaSuccess ||
        cudaFuncSetAttribute(qkern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm) != cudaSuccess ||
        art_prepare_exact<real, TB, TC, BLK, NT, KP, MINB>((int)sm) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    int per_sm = 0;   // of the queue form, which sizes the persistent grid
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, qkern, NT, sm) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return per_sm;
}

// Sweep-kernel variants compiled into the library: tile (b x c), slab block,
// threads, direction pairs per exchange group, min CTAs per SM.  Index + 1 is
// the value of art_options.variant that selects one (0 = default).
struct KVariant {
    int prec, tb, tc, blk, nt, kp, minb;
    cudaError_t (*launch)(const void *, int, cudaStream_t, bool);
    int (*prepare)();
};
#define ART_V(real, pr, tb, tc, blk, nt, kp, mb)                                                   \
    {pr, tb, tc, blk, nt, kp, mb, &launch_sweep<real, tb, tc, blk, nt, kp, mb>,                      \
     &prepare_sweep<real, tb, tc, blk, nt, kp, mb>}
const KVariant kVariants[] = {
#define ART_VARIANT(real, pr, tb, tc, blk, nt, kp, mb) ART_V(real, pr, tb, tc, blk, nt, kp, mb),
#include "art_variants.inc"
#undef ART_VARIANT
};
#undef ART_V
const int kNumVariants = int(sizeof(kVariants) / sizeof(kVariants[0]));

struct HostTables {
    std::vector<ClassDev> classes;
    std::vector<DirDev> dirs;
    std::vector<SlabGeom> geo;    // concatenated per class-sorted direction
    std::vector<int> na;          // slabs of each direction, in table order
    std::vector<WorkItem> work;
    std::vector<art_grid_host> grids;
    long long plane_elems = 0;
    long long jpart_elems = 0;
    int max_blocks = 0;
    int min_per_class = 1 << 30;  // fewest directions in a non-empty class
};

// Tables of every grid for the context's tile, slab block and direction
// groups.  Segment-table, plane and J-partial offsets run across the grids of
// a batch; work items are ordered longest first, which the persistent queue
// hands out first.  Each (class, group, cell) partial is written by exactly
// one work item, so the order changes no result.
void build_tables(const art_ctx *ctx, HostTables &t)
{
    long long seg_off = 0, plane_off = 0, jpart_off = 0, cell_off = 0;
    std::vector<long long> cost;
    for (const art_grid_host &gin : ctx->grids) {
        art_grid_host gh = gin;
        const int dims[3] = {gh.g.nx, gh.g.ny, gh.g.nz};
        std::vector<double> xyz;
        healpix_directions(gh.nside, xyz);
        std::vector<Frame> fr(gh.nd);
        for (int d = 0; d < gh.nd; ++d) fr[d] = frame_of(&xyz[3 * d], ctx->opt.tie_tol);
        const bool ranged = ctx->opt.dir_end > ctx->opt.dir_begin;
        auto in_shard = [&](int d) { return !ranged || (d >= ctx->opt.dir_begin && d < ctx->opt.dir_end); };
        gh.cell_off = cell_off;
        gh.jpart_off = jpart_off;
        gh.seg_count = 0;
        int part = 0, maxNa = 0;
        for (int cls = 0; cls < 24; ++cls) {
            std::vector<int> members;
            for (int d = 0; d < gh.nd; ++d)
                if (fr[d].cls == cls && in_shard(d)) members.push_back(d);
            if (members.empty()) continue;
            t.min_per_class = std::min(t.min_per_class, (int)members.size());
            // Order within the class: by column drift per slab block along b,
            // then c, then RING index.  Directions the kernel takes together
            // then have similar upstream cones.  The order is fixed, so sums
            // stay deterministic.
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
            C.part0 = part;
            C.nx = dims[0];
            C.ny = dims[1];
            C.nz = dims[2];
            C.cell_off = gh.cell_off;
            C.jpart_off = gh.jpart_off + (long long)part * gh.ncell;
            C.ncell = gh.ncell;
            part += ctx->split;
            maxNa = std::max(maxNa, C.Na);
            const int ci = (int)t.classes.size();
            t.classes.push_back(C);
            for (int d : members) {
                std::vector<SlabGeom> g;
                slab_geometry(fr[d], C.Na, g);
                t.na.push_back(C.Na);
                DirDev D;
                D.seg_off = seg_off;
                D.plane_off = plane_off;
                D.na = fr[d].na;
                t.dirs.push_back(D);
                for (const SlabGeom &s : g) {
                    t.geo.push_back(s);
                    gh.seg_count += (long long)s.nonzero * C.Nb * C.Nc;
                }
                seg_off += C.Na;
                plane_off += (long long)C.Nb * C.Nc;
            }
            const long long ndir = (long long)members.size();
            for (int pc = 0; pc < C.Nc; pc += ctx->TC)
                for (int pb = 0; pb < C.Nb; pb += ctx->TB)
                    for (int g = 0; g < ctx->split; ++g) {
                        t.work.push_back(WorkItem{ci, pb, pc, g});
                        const long long nd_g = (ndir * (g + 1)) / ctx->split - (ndir * g) / ctx->split;
                        cost.push_back((nd_g + 1) * std::min(ctx->TB, C.Nb - pb) * std::min(ctx->TC, C.Nc - pc) *
                                       (long long)C.Na);
                    }
        }
        gh.n_part = part;
        gh.nblocks = (maxNa + ctx->BLK - 1) / ctx->BLK;
        t.max_blocks = std::max(t.max_blocks, gh.nblocks);
        jpart_off += (long long)part * gh.ncell;
        cell_off += gh.ncell;
        t.grids.push_back(gh);
    }
    std::vector<int> idx(t.work.size());
    for (size_t i = 0; i < idx.size(); ++i) idx[i] = (int)i;
    std::stable_sort(idx.begin(), idx.end(), [&](int x, int y) { return cost[x] > cost[y]; });
    std::vector<WorkItem> w(t.work.size());
    for (size_t i = 0; i < idx.size(); ++i) w[i] = t.work[idx[i]];
    t.work.swap(w);
    t.plane_elems = plane_off;
    t.jpart_elems = jpart_off;
}

// Segment entries of the tables; the code also carries, per slab, the column
// shifts that the direction still makes from this slab to the end of its slab
// block (the upstream cone the kernel must recompute), so the kernel reads
// them instead of summing them.  `na` holds each direction's slab count, in
// table order.
template <typename real>
std::vector<SegEntry<real>> pack_segs(const std::vector<SlabGeom> &geo, const std::vector<int> &na, int blk)
{
    std::vector<SegEntry<real>> out(geo.size());
    size_t base = 0;
    for (int n : na) {
        for (int m = n - 1; m >= 0; --m) {
            const SlabGeom &g = geo[base + m];
            const bool last_in_block = (m + 1) % blk == 0 || m + 1 == n;
            const int rb = g.shb + (last_in_block ? 0 : ((out[base + m + 1].code >> 5) & 15));
            const int rc = g.shc + (last_in_block ? 0 : ((out[base + m + 1].code >> 9) & 15));
            SegEntry<real> &e = out[base + m];
            e.ds1 = real(g.ds[0]);
            e.ds2 = real(g.ds[1]);
            e.ds3 = real(g.ds[2]);
            e.code = slab_code(g, rb, rc);
        }
        base += n;
    }
    return out;
}

template <typename real> art_status upload_gridinfo(art_ctx *ctx)
{
    std::vector<GridDev<real>> gi;
    for (const art_grid_host &g : ctx->grids)
        gi.push_back(GridDev<real>{g.cell_off, g.ncell, g.jpart_off, g.n_part, real(1.0 / g.nd)});
    CK(ctx, cudaMemcpy(ctx->d_gridinfo, gi.data(), gi.size() * sizeof(gi[0]), cudaMemcpyHostToDevice));
    return ART_OK;
}

// Select a kernel variant: build its tables and (re)allocate the buffers that
// depend on them.  Field, plane and staging buffers do not depend on it.
art_status setup_wave(art_ctx *ctx, int w);

art_status setup_variant(art_ctx *ctx, int variant)
{
    if (variant >= kNumVariants) return setup_wave(ctx, variant - kNumVariants);
    const KVariant &k = kVariants[variant];
    const int per_sm = k.prepare();
    if (per_sm < 1) return fail(ctx, ART_E_CUDA, "sweep kernel variant cannot be launched on this device");
    if (ctx->gexec) {
        cudaGraphExecDestroy(ctx->gexec);
        ctx->gexec = nullptr;
    }
    art_wave_free(ctx);
    ctx->variant = variant;
    ctx->TB = k.tb;
    ctx->TC = k.tc;
    ctx->BLK = k.blk;
    ctx->NT = k.nt;
    ctx->KP = k.kp;
    int dev = 0, sms = 152;
    if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaGetLastError();
    // direction groups per class: enough work items to cover the GPU twice
    ctx->split = 1;
    if (ctx->opt.dir_split > 0) {
        ctx->split = ctx->opt.dir_split;
    } else {
        HostTables probe;
        build_tables(ctx, probe);
        const int base = (int)probe.work.size();
        while (base * ctx->split < 2 * sms && ctx->split * 2 <= probe.min_per_class) ctx->split *= 2;
    }
    HostTables t;
    build_tables(ctx, t);
    ctx->grids = t.grids;
    ctx->n_classes = (int)t.classes.size();
    ctx->n_part = 0;
    ctx->seg_count = 0;
    for (const art_grid_host &g : ctx->grids) {
        ctx->n_part += g.n_part;
        ctx->seg_count += g.seg_count;
    }
    ctx->n_work = (int)t.work.size();
    ctx->nblocks = t.max_blocks;
    ctx->plane_elems = t.plane_elems;
    ctx->n_ctas = std::min(ctx->n_work, sms * per_sm);

    dev_free(ctx, ctx->d_jpart, ctx->jpart_bytes);
    dev_free(ctx, ctx->d_segs, ctx->segs_bytes);
    dev_free(ctx, ctx->d_dirs, ctx->dirs_bytes);
    dev_free(ctx, ctx->d_classes, ctx->classes_bytes);
    dev_free(ctx, ctx->d_work, ctx->work_bytes);
    dev_free(ctx, ctx->d_counter, ctx->counter_bytes);
    dev_free(ctx, ctx->d_gridinfo, ctx->gridinfo_bytes);
    const size_t jb = (size_t)t.jpart_elems * ctx->rsz;
    const size_t sb = t.geo.size() * (ctx->prec == ART_FP64 ? sizeof(SegEntry<double>) : sizeof(SegEntry<float>));
    const size_t db = t.dirs.size() * sizeof(DirDev), cb = t.classes.size() * sizeof(ClassDev);
    const size_t wb = t.work.size() * sizeof(WorkItem), qb = (size_t)std::max(1, ctx->nblocks) * sizeof(int);
    const size_t gb = ctx->grids.size() * sizeof(GridDev<double>);
    art_status s;
    if ((s = dev_alloc(ctx, &ctx->d_jpart, jb)) != ART_OK) return s;
    ctx->jpart_bytes = jb;
    if ((s = dev_alloc(ctx, &ctx->d_segs, sb)) != ART_OK) return s;
    ctx->segs_bytes = sb;
    if ((s = dev_alloc(ctx, &ctx->d_dirs, db)) != ART_OK) return s;
    ctx->dirs_bytes = db;
    if ((s = dev_alloc(ctx, &ctx->d_classes, cb)) != ART_OK) return s;
    ctx->classes_bytes = cb;
    if ((s = dev_alloc(ctx, &ctx->d_work, wb)) != ART_OK) return s;
    ctx->work_bytes = wb;
    if ((s = dev_alloc(ctx, &ctx->d_counter, qb)) != ART_OK) return s;
    ctx->counter_bytes = qb;
    if ((s = dev_alloc(ctx, &ctx->d_gridinfo, gb)) != ART_OK) return s;
    ctx->gridinfo_bytes = gb;
    if (ctx->prec == ART_FP64) {
        auto v = pack_segs<double>(t.geo, t.na, ctx->BLK);
        CK(ctx, cudaMemcpy(ctx->d_segs, v.data(), v.size() * sizeof(v[0]), cudaMemcpyHostToDevice));
        if ((s = upload_gridinfo<double>(ctx)) != ART_OK) return s;
    } else {
        auto v = pack_segs<float>(t.geo, t.na, ctx->BLK);
        CK(ctx, cudaMemcpy(ctx->d_segs, v.data(), v.size() * sizeof(v[0]), cudaMemcpyHostToDevice));
        if ((s = upload_gridinfo<float>(ctx)) != ART_OK) return s;
    }
    CK(ctx, cudaMemcpy(ctx->d_dirs, t.dirs.data(), db, cudaMemcpyHostToDevice));
    CK(ctx, cudaMemcpy(ctx->d_classes, t.classes.data(), cb, cudaMemcpyHostToDevice));
    CK(ctx, cudaMemcpy(ctx->d_work, t.work.data(), wb, cudaMemcpyHostToDevice));
    // ray-plane buffers of the slab-block launches
    const size_t pb = (size_t)std::max<long long>(1, ctx->plane_elems) * ctx->rsz;
    if (ctx->plane_bytes != pb) {
        dev_free(ctx, ctx->d_plane[0], ctx->plane_bytes_0);
        dev_free(ctx, ctx->d_plane[1], ctx->plane_bytes_1);
        if ((s = dev_alloc(ctx, &ctx->d_plane[0], pb)) != ART_OK) return s;
        ctx->plane_bytes_0 = pb;
        if ((s = dev_alloc(ctx, &ctx->d_plane[1], pb)) != ART_OK) return s;
        ctx->plane_bytes_1 = pb;
        ctx->plane_bytes = pb;
    }
    return ART_OK;
}

// Select wave variant w (art_wave.cu): its tables, buffers and J partials; the
// slab-block tables and planes are released.
art_status setup_wave(art_ctx *ctx, int w)
{
    if (ctx->prec != ART_FP32 || ctx->opt.averaging != ART_AVG_PAPER)
        return fail(ctx, ART_E_INVALID, "the wavefront sweep is FP32 with the paper's averaging");
    if (ctx->gexec) {
        cudaGraphExecDestroy(ctx->gexec);
        ctx->gexec = nullptr;
    }
    dev_free(ctx, ctx->d_jpart, ctx->jpart_bytes);
    dev_free(ctx, ctx->d_segs, ctx->segs_bytes);
    dev_free(ctx, ctx->d_dirs, ctx->dirs_bytes);
    dev_free(ctx, ctx->d_classes, ctx->classes_bytes);
    dev_free(ctx, ctx->d_work, ctx->work_bytes);
    dev_free(ctx, ctx->d_counter, ctx->counter_bytes);
    dev_free(ctx, ctx->d_gridinfo, ctx->gridinfo_bytes);
    dev_free(ctx, ctx->d_plane[0], ctx->plane_bytes_0);
    dev_free(ctx, ctx->d_plane[1], ctx->plane_bytes_1);
    ctx->plane_bytes = 0;
    art_status s = art_wave_setup(ctx, w);
    if (s != ART_OK) return s;
    ctx->variant = kNumVariants + w;
    ctx->TB = 8 * ctx->wave.wb;
    ctx->TC = 8 * ctx->wave.np * ctx->wave.wc;
    ctx->BLK = 0;
    ctx->KP = 0;
    ctx->split = 0;
    ctx->nblocks = 1;
    ctx->n_work = ctx->wave.n_units;
    ctx->n_ctas = ctx->wave.n_units;
    ctx->persistent = 0;
    ctx->plane_elems = 0;
    const size_t jb =
        (size_t)std::max<long long>(1, ctx->wave.jpart_floats) * ctx->wave.bins_per_launch * sizeof(float);
    if ((s = dev_alloc(ctx, &ctx->d_jpart, jb)) != ART_OK) return s;
    ctx->jpart_bytes = jb;
    const size_t gb = ctx->grids.size() * sizeof(GridDev<double>);
    if ((s = dev_alloc(ctx, &ctx->d_gridinfo, gb)) != ART_OK) return s;
    ctx->gridinfo_bytes = gb;
    return upload_gridinfo<float>(ctx);
}

// The wave variant for the context's largest class: the fewest direction
// slots that hold it, else the most (classes split into groups); -1 if the
// context cannot use the wavefront sweep.
int pick_wave(const art_ctx *ctx)
{
    if (ctx->prec != ART_FP32 || ctx->opt.averaging != ART_AVG_PAPER) return -1;
    int maxc = 0;
    long long largest = 0;
    for (const art_grid_host &g : ctx->grids) {
        std::vector<double> xyz;
        healpix_directions(g.nside, xyz);
        int cnt[24] = {0};
        const bool ranged = ctx->opt.dir_end > ctx->opt.dir_begin;
        for (int d = 0; d < g.nd; ++d)
            if (!ranged || (d >= ctx->opt.dir_begin && d < ctx->opt.dir_end))
                ++cnt[frame_of(&xyz[3 * d], ctx->opt.tie_tol).cls];
        for (int c = 0; c < 24; ++c) maxc = std::max(maxc, cnt[c]);
        largest = std::max(largest, (long long)g.g.nx * g.g.ny * g.g.nz);
    }
    return art_wave_default(maxc, largest);
}

template <typename real> art_status do_sweep(art_ctx *ctx, real *J, real *Jin, real *gam, cudaStream_t st)
{
    using v2 = typename Vec2<real>::type;
    const long long n = ctx->ncell;
    v2 *fields = static_cast<v2 *>(ctx->d_field);
    real *planes[2] = {static_cast<real *>(ctx->d_plane[0]), static_cast<real *>(ctx->d_plane[1])};
    for (int b = 0; b < ctx->nbins; ++b) {
        SweepArgs<real> a{};
        a.field0 = fields + (0LL * ctx->nbins + b) * n;
        a.field1 = fields + (1LL * ctx->nbins + b) * n;
        a.field2 = fields + (2LL * ctx->nbins + b) * n;
        a.jpart = static_cast<real *>(ctx->d_jpart);
        a.segs = static_cast<const SegEntry<real> *>(ctx->d_segs);
        a.dirs = ctx->d_dirs;
        a.classes = ctx->d_classes;
        a.work = ctx->d_work;
        a.n_work = ctx->n_work;
        a.split = ctx->split;
        a.field_form = ctx->opt.field_form;
        a.i_bc = real(ctx->i_bc[b]);
        a.averaging = ctx->opt.averaging;
        cudaEvent_t e0 = nullptr, e1 = nullptr, e2 = nullptr;
        if (ctx->profiling) {
            CK(ctx, cudaEventCreate(&e0));
            CK(ctx, cudaEventCreate(&e1));
            CK(ctx, cudaEventCreate(&e2));
            ctx->ev.push_back(e0);
            ctx->ev.push_back(e1);
            ctx->ev.push_back(e2);
        }
        if (ctx->persistent) CK(ctx, cudaMemsetAsync(ctx->d_counter, 0, ctx->counter_bytes, st));
        if (ctx->profiling) CK(ctx, cudaEventRecord(e0, st));
        // the wavefront sweeps bins_per_launch bins per launch (all of them, or one)
        const int wnb = ctx->wave.on ? ctx->wave.bins_per_launch : 1;
        if (ctx->wave.on && b % wnb == 0) {
            art_status ws = art_wave_launch(ctx, reinterpret_cast<const float2 *>(a.field0),
                                            reinterpret_cast<const float2 *>(a.field1),
                                            reinterpret_cast<const float2 *>(a.field2), n, b, st);
            if (ws != ART_OK) return ws;
        }
        for (int k = 0; k < ctx->nblocks && !ctx->wave.on; ++k) {
            a.kblock = k;
            a.plane_in = planes[k & 1];
            a.plane_out = planes[(k + 1) & 1];
            a.counter = ctx->persistent ? ctx->d_counter + k : nullptr;
            // the first launch of a bin follows kernels that write its inputs, so it starts only after them
            CK(ctx, kVariants[ctx->variant].launch(&a, ctx->persistent ? ctx->n_ctas : ctx->n_work, st,
                                                   k > 0 && ctx->early_launch));
        }
        if (ctx->profiling) CK(ctx, cudaEventRecord(e1, st));
        ReduceArgs<real> r{};
        r.jpart = static_cast<const real *>(ctx->d_jpart) +
                  (ctx->wave.on ? (long long)(b % wnb) * ctx->wave.jpart_floats : 0LL);
        r.field_nat = fields + (2LL * ctx->nbins + b) * n;
        r.grids = static_cast<const GridDev<real> *>(ctx->d_gridinfo);
        r.n_grids = (int)ctx->grids.size();
        r.total = n;
        r.gamma_coef = real(4.0 * M_PI * ctx->G[b]);
        r.gamma_accum = b > 0;
        r.field_form = ctx->opt.field_form;
        r.whole = ctx->opt.averaging == ART_AVG_EXACT && ctx->opt.field_form == ART_FIELDS_EPS;
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

art_status sweep_launches(art_ctx *ctx, void *J, void *J_in, void *gamma, cudaStream_t st)
{
    if (ctx->prec == ART_FP64)
        return do_sweep<double>(ctx, static_cast<double *>(J), static_cast<double *>(J_in),
                                static_cast<double *>(gamma), st);
    return do_sweep<float>(ctx, static_cast<float *>(J), static_cast<float *>(J_in), static_cast<float *>(gamma), st);
}

// Replay the launches of one sweep as a CUDA graph, captured on an internal
// stream and ordered after the work already queued on `st` and before
// anything queued on `st` later.  Captured again whenever the outputs change.
art_status sweep_graph(art_ctx *ctx, void *J, void *J_in, void *gamma, cudaStream_t st)
{
    if (!ctx->gstream) {
        CK(ctx, cudaStreamCreateWithFlags(&ctx->gstream, cudaStreamNonBlocking));
        CK(ctx, cudaEventCreateWithFlags(&ctx->gev[0], cudaEventDisableTiming));
        CK(ctx, cudaEventCreateWithFlags(&ctx->gev[1], cudaEventDisableTiming));
    }
    if (ctx->gexec && (ctx->g_key[0] != J || ctx->g_key[1] != J_in || ctx->g_key[2] != gamma)) {
        cudaGraphExecDestroy(ctx->gexec);
        ctx->gexec = nullptr;
    }
    if (!ctx->gexec) {
        cudaGraph_t graph = nullptr;
        CK(ctx, cudaStreamBeginCapture(ctx->gstream, cudaStreamCaptureModeThreadLocal));
        const art_status s = sweep_launches(ctx, J, J_in, gamma, ctx->gstream);
        const cudaError_t e = cudaStreamEndCapture(ctx->gstream, &graph);
        if (s != ART_OK || e != cudaSuccess) {
            if (graph) cudaGraphDestroy(graph);
            cudaGetLastError();
            return s != ART_OK ? s : fail(ctx, ART_E_CUDA, std::string("graph capture: ") + cudaGetErrorString(e));
        }
        const cudaError_t ei = cudaGraphInstantiate(&ctx->gexec, graph, 0);
        cudaGraphDestroy(graph);
        if (ei != cudaSuccess) {
            ctx->gexec = nullptr;
            return fail(ctx, ART_E_CUDA, std::string("graph instantiate: ") + cudaGetErrorString(ei));
        }
        ctx->g_key[0] = J;
        ctx->g_key[1] = J_in;
        ctx->g_key[2] = gamma;
    }
    CK(ctx, cudaEventRecord(ctx->gev[0], st));
    CK(ctx, cudaStreamWaitEvent(ctx->gstream, ctx->gev[0], 0));
    CK(ctx, cudaGraphLaunch(ctx->gexec, ctx->gstream));
    CK(ctx, cudaEventRecord(ctx->gev[1], ctx->gstream));
    CK(ctx, cudaStreamWaitEvent(st, ctx->gev[1], 0));
    return ART_OK;
}

art_status create_common(const art_grid *grids, const int *n_side, int n_grids, int nu_bins, const art_options *opt,
                         art_ctx **out)
{
    if (!out) return ART_E_INVALID;
    *out = nullptr;
    if (!grids || !n_side || n_grids < 1 || n_grids > 4096 || nu_bins < 1) return ART_E_INVALID;
    long long total = 0, largest = 0;
    for (int g = 0; g < n_grids; ++g) {
        const art_grid &gr = grids[g];
        if (gr.nx < 1 || gr.ny < 1 || gr.nz < 1 || n_side[g] < 1 || n_side[g] > 1024) return ART_E_INVALID;
        const long long c = (long long)gr.nx * gr.ny * gr.nz;
        if (c > (1LL << 31)) return ART_E_INVALID;
        total += c;
        largest = std::max(largest, c);
    }
    if (total > (1LL << 31)) return ART_E_INVALID;
    art_ctx *ctx = new (std::nothrow) art_ctx();
    if (!ctx) return ART_E_OOM;
    ctx->grid = grids[0];
    ctx->nside = n_side[0];
    ctx->nbins = nu_bins;
    if (opt) ctx->opt = *opt;
    else art_options_default(&ctx->opt);
    if (!(ctx->opt.tie_tol >= 0.0) || ctx->opt.tie_tol > 1e-3) ctx->opt.tie_tol = 1e-12;
    if ((ctx->opt.precision != ART_FP32 && ctx->opt.precision != ART_FP64) ||
        (ctx->opt.averaging != ART_AVG_PAPER && ctx->opt.averaging != ART_AVG_EXACT) ||
        (ctx->opt.field_form != ART_FIELDS_S && ctx->opt.field_form != ART_FIELDS_EPS) || ctx->opt.dir_split < 0 ||
        ctx->opt.dir_begin < 0 || ctx->opt.dir_end < 0 ||
        (ctx->opt.dir_end != 0 || ctx->opt.dir_begin != 0) &&
            (n_grids != 1 || ctx->opt.dir_begin >= ctx->opt.dir_end || ctx->opt.dir_end > 12 * n_side[0] * n_side[0])) {
        delete ctx;
        return ART_E_INVALID;
    }
    ctx->prec = ctx->opt.precision;
    ctx->rsz = ctx->prec == ART_FP64 ? 8 : 4;
    ctx->ncell = total;
    ctx->nd = 0;   // directions swept (all, or the shard)
    for (int g = 0; g < n_grids; ++g) {
        art_grid_host gh;
        gh.g = grids[g];
        gh.nside = n_side[g];
        gh.nd = 12 * n_side[g] * n_side[g];
        gh.ncell = (long long)grids[g].nx * grids[g].ny * grids[g].nz;
        ctx->grids.push_back(gh);
        ctx->nd += gh.nd;
    }
    if (ctx->opt.dir_end > ctx->opt.dir_begin) ctx->nd = ctx->opt.dir_end - ctx->opt.dir_begin;
    ctx->G.assign(nu_bins, 0.0);
    ctx->i_bc.assign(nu_bins, 0.0);
    ctx->persistent = ctx->opt.persistent > 0 ? 1 : (ctx->opt.persistent < 0 ? 0 : (n_grids > 1 ? 1 : 0));
    ctx->early_launch = ctx->opt.early_launch >= 0;

    int pick = -1;
    if (ctx->opt.variant > kNumVariants) {
        pick = ctx->opt.variant - 1;
        if (pick - kNumVariants >= art_wave_variants() || ctx->prec != ART_FP32 ||
            ctx->opt.averaging != ART_AVG_PAPER)
            pick = -2;
    } else if (ctx->opt.variant > 0) {
        pick = ctx->opt.variant - 1;
        if (pick >= kNumVariants || kVariants[pick].prec != ctx->prec) pick = -2;
    } else if (!ctx->opt.tile_b && !ctx->opt.tile_c && !ctx->opt.slab && !ctx->opt.dir_split &&
               ctx->opt.persistent == 0 && pick_wave(ctx) >= 0) {
        // the wavefront sweep, unless the options ask for a slab-block shape
        pick = kNumVariants + pick_wave(ctx);
    } else {
        // measured on GB300: the 32 x 8 tile with three direction pairs per
        // exchange (variant 15) wins for grids below ~100^3 cells (more CTAs
        // per launch), the 32 x 16 tile above
        if (ctx->prec == ART_FP32 && largest < 100LL * 100 * 100 && !ctx->opt.tile_b && !ctx->opt.tile_c &&
            !ctx->opt.slab)
            pick = 14;
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
    art_status st = setup_variant(ctx, pick);
    if (st != ART_OK) {
        art_destroy(ctx);
        return st;
    }
    const size_t rs = ctx->rsz, n = (size_t)ctx->ncell;
#define ALLOC(ptr, bytes)                                       \
    do {                                                        \
        if ((st = dev_alloc(ctx, &(ptr), (bytes))) != ART_OK) { \
            art_destroy(ctx);                                   \
            return st;                                          \
        }                                                       \
    } while (0)
    ALLOC(ctx->d_field, 3 * (size_t)nu_bins * n * 2 * rs);
    ALLOC(ctx->d_stage, 2 * (size_t)nu_bins * n * rs);
    ALLOC(ctx->d_out, (2 * (size_t)nu_bins + 1) * n * rs);
    ALLOC(ctx->d_flag, sizeof(int));
#undef ALLOC
    *out = ctx;
    return ART_OK;
}

}  // namespace

art_status art_internal_sweep(art_ctx *ctx, void *J, void *J_in, void *gamma, cudaStream_t st)
{
    return sweep_launches(ctx, J, J_in, gamma, st);
}

art_status art_internal_layout(art_ctx *ctx, const void *kd, const void *sd, cudaStream_t st)
{
    const long long nc = ctx->ncell;
    const int nt = 256;
    for (int b = 0; b < ctx->nbins; ++b) {
        for (const art_grid_host &g : ctx->grids) {
            const unsigned lb = (unsigned)((g.ncell + nt - 1) / nt);
            const long long off = (long long)b * nc + g.cell_off;
            if (ctx->prec == ART_FP64) {
                double2 *f = static_cast<double2 *>(ctx->d_field);
                layout_kernel<double><<<lb, nt, 0, st>>>(
                    static_cast<const double *>(kd) + off, static_cast<const double *>(sd) + off,
                    f + (0LL * ctx->nbins + b) * nc + g.cell_off, f + (1LL * ctx->nbins + b) * nc + g.cell_off,
                    f + (2LL * ctx->nbins + b) * nc + g.cell_off, g.g.nx, g.g.ny, g.g.nz);
            } else {
                float2 *f = static_cast<float2 *>(ctx->d_field);
                layout_kernel<float><<<lb, nt, 0, st>>>(
                    static_cast<const float *>(kd) + off, static_cast<const float *>(sd) + off,
                    f + (0LL * ctx->nbins + b) * nc + g.cell_off, f + (1LL * ctx->nbins + b) * nc + g.cell_off,
                    f + (2LL * ctx->nbins + b) * nc + g.cell_off, g.g.nx, g.g.ny, g.g.nz);
            }
            CK(ctx, cudaGetLastError());
        }
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

art_status art_create(const art_grid *grid, int n_side, int nu_bins, const art_options *opt, art_ctx **out)
{
    if (!grid) {
        if (out) *out = nullptr;
        return ART_E_INVALID;
    }
    return create_common(grid, &n_side, 1, nu_bins, opt, out);
}

art_status art_batch_create(const art_grid *grids, const int *n_side, int n_grids, int nu_bins,
                            const art_options *opt, art_ctx **out)
{
    return create_common(grids, n_side, n_grids, nu_bins, opt, out);
}

art_status art_autotune(art_ctx *ctx, int reps, int *best_variant, void *stream)
{
    if (!ctx) return ART_E_INVALID;
    if (!ctx->have_fields) return fail(ctx, ART_E_STATE, "art_autotune: call art_set_fields first");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (reps < 1) reps = 3;
    char *jin = static_cast<char *>(ctx->d_out) + (size_t)ctx->ncell * ctx->nbins * ctx->rsz;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    CK(ctx, cudaEventCreate(&e0));
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        return fail(ctx, ART_E_CUDA, "art_autotune: cudaEventCreate failed");
    }
    const bool keep_prof = ctx->profiling;
    ctx->profiling = false;
    int best = ctx->variant, best_pers = ctx->persistent;
    float best_ms = 3.0e38f;
    art_status s = ART_OK;
    // launch forms tried: both unless the options fixed one
    const int forms[2] = {1, 0};
    const int nforms = ctx->opt.persistent == 0 ? 2 : 1;
    const bool wave_ok = ctx->prec == ART_FP32 && ctx->opt.averaging == ART_AVG_PAPER;
    const int nv = kNumVariants + (wave_ok ? art_wave_variants() : 0);
    for (int v = 0; v < nv && s == ART_OK; ++v) {
        const bool wave = v >= kNumVariants;
        if (!wave && (kVariants[v].prec != ctx->prec || kVariants[v].prepare() < 1)) continue;
        if ((s = setup_variant(ctx, v)) != ART_OK) break;
        for (int f = 0; f < (wave ? 1 : nforms) && s == ART_OK; ++f) {
            if (nforms == 2 && !wave) ctx->persistent = forms[f];
            if ((s = sweep_launches(ctx, nullptr, jin, nullptr, st)) != ART_OK) break;   // warm-up
            if (cudaEventRecord(e0, st) != cudaSuccess) {
                s = fail(ctx, ART_E_CUDA, "art_autotune: cudaEventRecord failed");
                break;
            }
            for (int r = 0; r < reps && s == ART_OK; ++r) s = sweep_launches(ctx, nullptr, jin, nullptr, st);
            if (s != ART_OK) break;
            float ms = 0.f;
            if (cudaEventRecord(e1, st) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
                cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) {
                s = fail(ctx, ART_E_CUDA, "art_autotune: timing failed");
                break;
            }
            if (ms < best_ms) {
                best_ms = ms;
                best = v;
                best_pers = ctx->persistent;
            }
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    ctx->profiling = keep_prof;
    if (s != ART_OK) return s;
    if ((s = setup_variant(ctx, best)) != ART_OK) return s;
    if (best < kNumVariants) ctx->persistent = best_pers;
    if (best_variant) *best_variant = best + 1;
    return ART_OK;
}

art_status art_sum_partials(const float *parts, int n_parts, int64_t n, float *out, void *stream)
{
    if (!parts || !out || n_parts < 1 || n < 0) return ART_E_INVALID;
    if (n == 0) return ART_OK;
    const int nt = 256;
    shard_sum_kernel<<<(unsigned)((n + nt - 1) / nt), nt, 0, static_cast<cudaStream_t>(stream)>>>(parts, n_parts, n,
                                                                                                      out);
    return cudaGetLastError() == cudaSuccess ? ART_OK : ART_E_CUDA;
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
    if (ctx->gexec) cudaGraphExecDestroy(ctx->gexec);
    if (ctx->gstream) cudaStreamDestroy(ctx->gstream);
    for (cudaEvent_t e : ctx->gev)
        if (e) cudaEventDestroy(e);
    void *ptrs[] = {ctx->d_field, ctx->d_plane[0], ctx->d_plane[1], ctx->d_jpart, ctx->d_segs, ctx->d_dirs,
                    ctx->d_classes, ctx->d_work, ctx->d_counter, ctx->d_gridinfo, ctx->d_stage, ctx->d_out,
                    ctx->d_flag, ctx->it.nH, ctx->it.y, ctx->it.y0, ctx->it.gpt, ctx->it.kap, ctx->it.eps,
                    ctx->it.jin, ctx->it.jsur, ctx->it.resid, ctx->it.src, ctx->it.yit, ctx->it.evo,
                    ctx->it.hpt, ctx->it.Tit};
    for (void *p : ptrs)
        if (p) cudaFree(p);
    art_wave_free(ctx);
    void *sur[] = {ctx->sur.kc, ctx->sur.ec, ctx->sur.jc, ctx->sur.o, ctx->sur.eref, ctx->sur.nHc, ctx->sur.yc};
    for (void *p : sur)
        if (p) cudaFree(p);
    art_internal_ablation_free(ctx);
    {
        auto &R = ctx->sres;
        if (R.in) cudaStreamDestroy(R.in);
        if (R.out) cudaStreamDestroy(R.out);
        for (int b = 0; b < 2; ++b) {
            for (cudaEvent_t e : {R.ev_in[b], R.ev_lay[b], R.ev_sw[b], R.ev_out[b]})
                if (e) cudaEventDestroy(e);
            if (R.slot[b]) cudaFree(R.slot[b]);
        }
        if (R.stage2) cudaFree(R.stage2);
        if (R.d_flags) cudaFree(R.d_flags);
        if (R.h_flags) cudaFreeHost(R.h_flags);
    }
    if (ctx->coarse) art_destroy(ctx->coarse);
    if (ctx->net) art_net_destroy(ctx->net);
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
    s->launches = ctx->wave.on ? 2 : ctx->nblocks + 1;
    s->ctas_per_launch = ctx->persistent ? ctx->n_ctas : ctx->n_work;
    s->tile_b = ctx->TB;
    s->tile_c = ctx->TC;
    s->slab = ctx->BLK;
    s->dir_split = ctx->split;
    s->device_bytes = ctx->dev_bytes;
    s->variant = ctx->variant + 1;
    s->group = ctx->wave.on ? ctx->wave.dmax : 2 * ctx->KP;
    s->n_grids = (int32_t)ctx->grids.size();
    s->work_items = ctx->n_work;
    s->persistent = ctx->persistent;
    s->bins_per_launch = ctx->wave.on ? ctx->wave.bins_per_launch : 1;
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
        validate_kernel<double><<<nb, nt, 0, st>>>(static_cast<const double *>(kd), static_cast<const double *>(sd), n,
                                                   ctx->d_flag);
    else
        validate_kernel<float><<<nb, nt, 0, st>>>(static_cast<const float *>(kd), static_cast<const float *>(sd), n,
                                                  ctx->d_flag);
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
    for (int b = 0; b < ctx->nbins; ++b)
        if (!std::isfinite(G[b])) return fail(ctx, ART_E_INVALID, "art_set_band: non-finite band integral");
    for (int b = 0; b < ctx->nbins; ++b) ctx->G[b] = G[b];
    if (ctx->gexec) {   // the captured reduction holds the old coefficients
        cudaGraphExecDestroy(ctx->gexec);
        ctx->gexec = nullptr;
    }
    return ART_OK;
}

art_status art_set_boundary_intensity(art_ctx *ctx, const double *I_bc)
{
    if (!ctx) return ART_E_INVALID;
    for (int b = 0; I_bc && b < ctx->nbins; ++b)
        if (!std::isfinite(I_bc[b]) || I_bc[b] < 0.0)
            return fail(ctx, ART_E_INVALID, "art_set_boundary_intensity: intensities must be finite and >= 0");
    for (int b = 0; b < ctx->nbins; ++b) ctx->i_bc[b] = I_bc ? I_bc[b] : 0.0;
    if (ctx->gexec) {   // the captured launches hold the old value
        cudaGraphExecDestroy(ctx->gexec);
        ctx->gexec = nullptr;
    }
    return ART_OK;
}

art_status art_sweep_stream(art_ctx *ctx, int n_sets, const void *const *kappa, const void *const *src,
                            void *const *J, void *const *J_in, void *const *gamma, void *stream)
{
    if (!ctx) return ART_E_INVALID;
    if (n_sets < 0 || (n_sets > 0 && (!kappa || !src)))
        return fail(ctx, ART_E_INVALID, "art_sweep_stream: bad set count or null input arrays");
    if (J && ctx->opt.dir_end > ctx->opt.dir_begin)
        return fail(ctx, ART_E_INVALID, "art_sweep_stream: a direction shard has no J output (sum the J_in shares)");
    for (int k = 0; k < n_sets; ++k)
        if (!kappa[k] || !src[k] || (J && !J[k]) || (J_in && !J_in[k]) || (gamma && !gamma[k]))
            return fail(ctx, ART_E_INVALID, "art_sweep_stream: null field or output pointer");
    if (n_sets == 0) return ART_OK;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const long long nb = ctx->ncell * ctx->nbins;
    const size_t rs = ctx->rsz, fbytes = (size_t)nb * rs;
    const size_t jbytes = fbytes, gbytes = (size_t)ctx->ncell * rs;
    auto &R = ctx->sres;
    if (!R.in) {
        CK(ctx, cudaStreamCreateWithFlags(&R.in, cudaStreamNonBlocking));
        CK(ctx, cudaStreamCreateWithFlags(&R.out, cudaStreamNonBlocking));
        for (int b = 0; b < 2; ++b)
            for (cudaEvent_t *e : {&R.ev_in[b], &R.ev_lay[b], &R.ev_sw[b], &R.ev_out[b]})
                CK(ctx, cudaEventCreateWithFlags(e, cudaEventDisableTiming));
        const size_t ob = (2 * (size_t)ctx->nbins + 1) * ctx->ncell * rs;
        CK(ctx, cudaMalloc(&R.stage2, 2 * fbytes));
        CK(ctx, cudaMalloc(&R.slot[0], ob));
        CK(ctx, cudaMalloc(&R.slot[1], ob));
        CK(ctx, cudaMalloc(&R.d_flags, 2 * sizeof(int)));
        CK(ctx, cudaMallocHost(&R.h_flags, 2 * sizeof(int)));
        ctx->dev_bytes += (long long)(2 * fbytes + 2 * ob + 2 * sizeof(int));
    }
    char *stage[2] = {static_cast<char *>(ctx->d_stage), static_cast<char *>(R.stage2)};
    char *o = static_cast<char *>(ctx->d_out);
    void *dJ = J ? o : nullptr, *dJin = J_in ? o + nb * rs : nullptr, *dG = gamma ? o + 2 * nb * rs : nullptr;
    const int nt = 256;
    const unsigned vb = (unsigned)std::min<long long>((nb + nt - 1) / nt, 4096);
    art_status status = ART_OK;
    int k = 0;
    for (; k < n_sets; ++k) {
        const int b = k & 1;
        // host -> device into stage[b] once the layout of set k - 2 has read it; validate there
        CK(ctx, cudaStreamWaitEvent(R.in, R.ev_lay[b], 0));
        CK(ctx, cudaMemcpyAsync(stage[b], kappa[k], fbytes, cudaMemcpyHostToDevice, R.in));
        CK(ctx, cudaMemcpyAsync(stage[b] + fbytes, src[k], fbytes, cudaMemcpyHostToDevice, R.in));
        CK(ctx, cudaMemsetAsync(R.d_flags + b, 0, sizeof(int), R.in));
        if (ctx->prec == ART_FP64)
            validate_kernel<double><<<vb, nt, 0, R.in>>>(reinterpret_cast<const double *>(stage[b]),
                                                         reinterpret_cast<const double *>(stage[b] + fbytes), nb,
                                                         R.d_flags + b);
        else
            validate_kernel<float><<<vb, nt, 0, R.in>>>(reinterpret_cast<const float *>(stage[b]),
                                                        reinterpret_cast<const float *>(stage[b] + fbytes), nb,
                                                        R.d_flags + b);
        CK(ctx, cudaGetLastError());
        CK(ctx, cudaMemcpyAsync(R.h_flags + b, R.d_flags + b, sizeof(int), cudaMemcpyDeviceToHost, R.in));
        CK(ctx, cudaEventRecord(R.ev_in[b], R.in));
        // the host waits for this set's copy and check while the sweep of set k - 1 runs
        CK(ctx, cudaEventSynchronize(R.ev_in[b]));
        if (R.h_flags[b]) {
            status = fail(ctx, ART_E_INVALID, "art_sweep_stream: set " + std::to_string(k) +
                                                  ((R.h_flags[b] & 1) ? ": kappa negative or not finite"
                                                                      : ": source term not finite"));
            break;
        }
        CK(ctx, cudaStreamWaitEvent(st, R.ev_in[b], 0));
        if ((status = art_internal_layout(ctx, stage[b], stage[b] + fbytes, st)) != ART_OK) break;
        CK(ctx, cudaEventRecord(R.ev_lay[b], st));
        status = (ctx->opt.graph && !ctx->profiling) ? sweep_graph(ctx, dJ, dJin, dG, st)
                                                     : sweep_launches(ctx, dJ, dJin, dG, st);
        if (status != ART_OK) break;
        // results into slot b once the device -> host copy of set k - 2 has read it
        CK(ctx, cudaStreamWaitEvent(st, R.ev_out[b], 0));
        char *sl = static_cast<char *>(R.slot[b]);
        if (J) CK(ctx, cudaMemcpyAsync(sl, dJ, jbytes, cudaMemcpyDeviceToDevice, st));
        if (J_in) CK(ctx, cudaMemcpyAsync(sl + jbytes, dJin, jbytes, cudaMemcpyDeviceToDevice, st));
        if (gamma) CK(ctx, cudaMemcpyAsync(sl + 2 * jbytes, dG, gbytes, cudaMemcpyDeviceToDevice, st));
        CK(ctx, cudaEventRecord(R.ev_sw[b], st));
        CK(ctx, cudaStreamWaitEvent(R.out, R.ev_sw[b], 0));
        if (J) CK(ctx, cudaMemcpyAsync(J[k], sl, jbytes, cudaMemcpyDeviceToHost, R.out));
        if (J_in) CK(ctx, cudaMemcpyAsync(J_in[k], sl + jbytes, jbytes, cudaMemcpyDeviceToHost, R.out));
        if (gamma) CK(ctx, cudaMemcpyAsync(gamma[k], sl + 2 * jbytes, gbytes, cudaMemcpyDeviceToHost, R.out));
        CK(ctx, cudaEventRecord(R.ev_out[b], R.out));
    }
    CK(ctx, cudaStreamSynchronize(st));
    CK(ctx, cudaStreamSynchronize(R.out));
    CK(ctx, cudaStreamSynchronize(R.in));
    return status;
}

art_status art_sweep(art_ctx *ctx, void *J, void *J_in, void *gamma, int on_device, void *stream)
{
    if (!ctx) return ART_E_INVALID;
    if (!ctx->have_fields) return fail(ctx, ART_E_STATE, "art_sweep: call art_set_fields first");
    if (J && ctx->opt.dir_end > ctx->opt.dir_begin)
        return fail(ctx, ART_E_INVALID, "art_sweep: a direction shard has no J output (sum the J_in shares)");
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
    const art_status s = (ctx->opt.graph && !ctx->profiling) ? sweep_graph(ctx, dJ, dJin, dG, st)
                                                              : sweep_launches(ctx, dJ, dJin, dG, st);
    if (s != ART_OK) return s;
    if (!on_device) {
        if (J) CK(ctx, cudaMemcpyAsync(J, dJ, nb * rs, cudaMemcpyDeviceToHost, st));
        if (J_in) CK(ctx, cudaMemcpyAsync(J_in, dJin, nb * rs, cudaMemcpyDeviceToHost, st));
        if (gamma) CK(ctx, cudaMemcpyAsync(gamma, dG, ctx->ncell * rs, cudaMemcpyDeviceToHost, st));
        CK(ctx, cudaStreamSynchronize(st));
        return art_wave_status(ctx, st);
    }
    return ART_OK;
}

art_status art_sweep_check(art_ctx *ctx, void *stream)
{
    if (!ctx) return ART_E_INVALID;
    return art_wave_status(ctx, static_cast<cudaStream_t>(stream));
}

art_status art_sweep_set_wait(art_ctx *ctx, double seconds, int stall_unit)
{
    if (!ctx) return ART_E_INVALID;
    if (!(seconds > 0.0) || seconds > 60.0)
        return fail(ctx, ART_E_INVALID, "art_sweep_set_wait: the bound must be in (0, 60] seconds");
    if (stall_unit < -1) return fail(ctx, ART_E_INVALID, "art_sweep_set_wait: stall_unit must be >= -1");
    ctx->wave.wait_ns = (long long)(seconds * 1e9);
    ctx->wave.stall_unit = stall_unit;
    if (ctx->gexec) {   // the captured launch holds the old values
        cudaGraphExecDestroy(ctx->gexec);
        ctx->gexec = nullptr;
    }
    return ART_OK;
}

}  // extern "C"
