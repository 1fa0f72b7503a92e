// art_wave.cu -- host side of the wavefront sweep (art_wave.cuh): the unit,
// class and direction tables of a context, its device buffers, the launch of
// one bin, and the compiled kernel shapes.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "art.h"
#include "art_ctx.hpp"
#include "art_geometry.hpp"
#include "art_wave.cuh"

using namespace art;

namespace {

#define WCK(ctx, call)                                                                            \
    do {                                                                                          \
        cudaError_t e_ = (call);                                                                  \
        if (e_ != cudaSuccess)                                                                    \
            return art_fail(ctx, e_ == cudaErrorMemoryAllocation ? ART_E_OOM : ART_E_CUDA,        \
                            std::string(#call) + ": " + cudaGetErrorString(e_));                  \
    } while (0)

template <int WB, int WC, int DMAX, int NP, int MINB>
cudaError_t wave_launch(const WaveArgs &a, int n_units, cudaStream_t st)
{
    using Sh = WaveShape<WB, WC, DMAX, NP>;
    wave_kernel<WB, WC, DMAX, NP, MINB><<<(unsigned)n_units, Sh::NT, Sh::bytes, st>>>(a);
    return cudaGetLastError();
}

// Shared-memory attribute; returns resident CTAs per SM (0 on error).
template <int WB, int WC, int DMAX, int NP, int MINB> int wave_prepare()
{
    using Sh = WaveShape<WB, WC, DMAX, NP>;
    auto kern = wave_kernel<WB, WC, DMAX, NP, MINB>;
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Sh::bytes) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, Sh::NT, Sh::bytes) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return per_sm;
}

struct WVariant {
    int wb, wc, dmax, np, minb;   // np: pairs of rows per lane (a warp tile is 8 x 8 np columns)
    cudaError_t (*launch)(const WaveArgs &, int, cudaStream_t);
    int (*prepare)();
};

#define ART_WV(wb, wc, dm, np, mb) \
    {wb, wc, dm, np, mb, &wave_launch<wb, wc, dm, np, mb>, &wave_prepare<wb, wc, dm, np, mb>}
// Compiled shapes: warps along b and c, direction slots of a unit (classes
// with more directions are split into groups), pairs of rows per lane (a warp
// tile is 8 x 8 np columns), min CTAs per SM.
const WVariant kWave[] = {
    ART_WV(2, 2, 16, 1, 6),   // 16 x 16 columns; N_side 8 (26-37 directions per class: 3 groups)
    ART_WV(2, 2, 12, 1, 8),   // N_side 3-4 (3-11 directions per class)
    ART_WV(2, 2, 4, 1, 8),    // N_side 1-2 (1-4)
    ART_WV(2, 4, 16, 1, 3),   // 16 x 32 columns
    ART_WV(4, 2, 16, 1, 3),   // 32 x 16 columns
    ART_WV(2, 4, 12, 1, 4),   // 16 x 32 columns, 12 slots (more CTAs per SM)
    ART_WV(2, 2, 20, 1, 5),   // 16 x 16 columns, 20 slots: N_side 8 classes in 2 groups
    ART_WV(2, 2, 16, 2, 4),   // four rows per lane: 16 x 32 columns, 4 warps
    ART_WV(2, 1, 16, 2, 8),   // four rows per lane: 16 x 16 columns, 2 warps
    ART_WV(2, 2, 12, 2, 4),   // four rows per lane, 12 slots (the default from N_side 3 up)
    ART_WV(2, 2, 17, 2, 3),   // four rows per lane, 17 slots: N_side 8 classes of up to 34 in 2 groups
    ART_WV(2, 2, 19, 2, 3),   // four rows per lane, 19 slots: every N_side 8 class (up to 37) in 2 groups
};
#undef ART_WV
const int kNumWave = int(sizeof(kWave) / sizeof(kWave[0]));

struct WaveHost {
    std::vector<WaveClass> classes;
    std::vector<WaveUnit> units;   // ticket order
    std::vector<float4> rtab;      // run tables of the direction groups
    int n_groups = 0;
    std::vector<art_grid_host> grids;
    long long edge_floats = 0, jpart_floats = 0;
    int max_class = 0;
};

float int_bits(int v)
{
    float f;
    std::memcpy(&f, &v, sizeof f);
    return f;
}

// Segment pattern of a slab, the run it belongs to: 0 one segment; 1 / 2 two
// segments, hand-off along b / c; 3 / 4 three segments, b / c crossed first.
int run_of(const SlabGeom &g)
{
    if (g.nseg == 1) return 0;
    if (g.nseg == 2) return g.shc ? 2 : 1;
    return g.cfirst ? 4 : 3;
}

// Run table of one direction group (members' frames f[0..nd)): per slab the
// header of run ends and the entries sorted by run (stable: slot order within
// a run).
void build_run_table(const std::vector<const Frame *> &f, int Na, std::vector<float4> &out)
{
    const int nd = (int)f.size();
    std::vector<std::vector<SlabGeom>> geo(nd);
    for (int i = 0; i < nd; ++i) slab_geometry(*f[i], Na, geo[i]);
    std::vector<int> order(nd);
    for (int m = 0; m < Na; ++m) {
        int ends[5] = {0, 0, 0, 0, 0};
        for (int i = 0; i < nd; ++i) ++ends[run_of(geo[i][m])];
        for (int k = 1; k < 5; ++k) ends[k] += ends[k - 1];
        for (int i = 0; i < nd; ++i) order[i] = i;
        std::stable_sort(order.begin(), order.end(),
                         [&](int x, int y) { return run_of(geo[x][m]) < run_of(geo[y][m]); });
        out.push_back(make_float4(int_bits(ends[0]), int_bits(ends[1]), int_bits(ends[2]), int_bits(ends[3])));
        for (int i : order) {
            const SlabGeom &g = geo[i][m];
            for (int k = 0; k < 3; ++k) {
                const float ds = k < g.nseg ? float(g.ds[k]) : 0.0f;
                out.push_back(make_float4(ds, ds, ds * ds, ds * ds));
            }
            const float na = float(f[i]->na);
            out.push_back(make_float4(na, na, int_bits(i), 0.0f));
        }
    }
}

void build_wave(const art_ctx *ctx, const WVariant &v, WaveHost &t)
{
    const int TB = 8 * v.wb, TC = 8 * v.np * v.wc;
    long long jpart_off = 0, cell_off = 0;
    struct Raw {
        WaveUnit u;
        int ib, ic, grid, cls, grp, key;
        long long cost;
    };
    std::vector<Raw> raw;
    for (const art_grid_host &gin : ctx->grids) {
        art_grid_host gh = gin;
        const int dims[3] = {gh.g.nx, gh.g.ny, gh.g.nz};
        const long long strides[3] = {1, (long long)dims[0], (long long)dims[0] * dims[1]};
        std::vector<double> xyz;
        healpix_directions(gh.nside, xyz);
        std::vector<Frame> fr(gh.nd);
        for (int d = 0; d < gh.nd; ++d) fr[d] = frame_of(&xyz[3 * d], ctx->opt.tie_tol);
        const bool ranged = ctx->opt.dir_end > ctx->opt.dir_begin;
        auto in_shard = [&](int d) { return !ranged || (d >= ctx->opt.dir_begin && d < ctx->opt.dir_end); };
        gh.cell_off = cell_off;
        gh.jpart_off = jpart_off;
        gh.seg_count = 0;
        gh.nblocks = 1;
        int part = 0;
        for (int cls = 0; cls < 24; ++cls) {
            std::vector<int> members;
            for (int d = 0; d < gh.nd; ++d)
                if (fr[d].cls == cls && in_shard(d)) members.push_back(d);
            if (members.empty()) continue;
            const int n = (int)members.size();
            t.max_class = std::max(t.max_class, n);
            const Frame &f0 = fr[members[0]];
            WaveClass C{};
            C.a = f0.a;
            C.sa = f0.sa;
            C.sb = f0.sb;
            C.sc = f0.sc;
            C.Na = dims[f0.a];
            C.Nb = dims[f0.b];
            C.Nc = dims[f0.c];
            C.pub = 1;
            while (C.pub * 2 <= std::min(WAVE_PUB, C.Na / 16)) C.pub *= 2;
            C.cell_off = gh.cell_off;
            C.stride_a = strides[f0.a];
            C.stride_b = strides[f0.b];
            C.stride_c = strides[f0.c];
            const int ci = (int)t.classes.size();
            t.classes.push_back(C);
            const int G = (n + v.dmax - 1) / v.dmax;
            for (int g = 0; g < G; ++g) {
                const int lo = (int)((long long)n * g / G), hi = (int)((long long)n * (g + 1) / G);
                const int grp = t.n_groups++;
                const long long gtab = (long long)t.rtab.size();
                std::vector<const Frame *> gf;
                for (int i = lo; i < hi; ++i) {
                    gf.push_back(&fr[members[i]]);
                    std::vector<SlabGeom> geo;
                    slab_geometry(fr[members[i]], C.Na, geo);
                    for (const SlabGeom &s : geo) gh.seg_count += (long long)s.nonzero * C.Nb * C.Nc;
                }
                build_run_table(gf, C.Na, t.rtab);
                const long long jp = gh.jpart_off + (long long)part * gh.ncell;
                ++part;
                const int nib = (C.Nb + TB - 1) / TB, nic = (C.Nc + TC - 1) / TC;
                for (int ic = 0; ic < nic; ++ic)
                    for (int ib = 0; ib < nib; ++ib) {
                        Raw r{};
                        r.u.cls = ci;
                        r.u.grp = grp;
                        r.u.nd = hi - lo;
                        r.u.tab = gtab;
                        r.u.tb = ib * TB;
                        r.u.tc = ic * TC;
                        r.u.jpart = jp;
                        // output buffers only where a downstream tile reads them
                        r.u.eb = ib + 1 < nib ? 0 : -1;
                        r.u.ec = ic + 1 < nic ? 0 : -1;
                        r.ib = ib;
                        r.ic = ic;
                        r.grid = (int)t.grids.size();
                        r.cls = ci;
                        r.grp = g;
                        r.key = (int)raw.size();
                        r.cost = (long long)C.Na * (hi - lo);
                        raw.push_back(r);
                    }
            }
        }
        gh.n_part = part;
        jpart_off += (long long)part * gh.ncell;
        cell_off += gh.ncell;
        t.grids.push_back(gh);
    }
    t.jpart_floats = jpart_off;
    // Ticket order: by tile diagonal, so both upstream tiles of a unit come
    // first; within a diagonal the costliest units first.  (Putting the
    // direction groups of one tile side by side, to share their field reads
    // in L2, was measured: no less DRAM traffic, 3 % slower.)
    std::vector<int> idx(raw.size());
    for (size_t i = 0; i < idx.size(); ++i) idx[i] = (int)i;
    std::stable_sort(idx.begin(), idx.end(), [&](int x, int y) {
        const int dx = raw[x].ib + raw[x].ic, dy = raw[y].ib + raw[y].ic;
        if (dx != dy) return dx < dy;
        return raw[x].cost > raw[y].cost;
    });
    // raw units are laid out tile-row by tile-row per (class, group): the
    // upstream tiles are at key - 1 (along b) and key - nib (along c)
    std::vector<int> pos(raw.size());
    for (size_t i = 0; i < idx.size(); ++i) pos[idx[i]] = (int)i;
    t.units.resize(raw.size());
    long long eoff = 0;
    for (size_t i = 0; i < idx.size(); ++i) {
        const Raw &r = raw[idx[i]];
        WaveUnit u = r.u;
        const WaveClass &C = t.classes[u.cls];
        const int nib = (C.Nb + TB - 1) / TB;
        u.up_b = r.ib > 0 ? pos[r.key - 1] : -1;
        u.up_c = r.ic > 0 ? pos[r.key - nib] : -1;
        if (u.eb >= 0) {
            u.eb = eoff;
            eoff += (long long)C.Na * v.wc * v.dmax * 8 * v.np;
        }
        if (u.ec >= 0) {
            u.ec = eoff;
            eoff += (long long)C.Na * v.wb * v.dmax * 8;
        }
        t.units[i] = u;
    }
    t.edge_floats = eoff;
}

int bits_int(float f)
{
    int v;
    std::memcpy(&v, &f, sizeof v);
    return v;
}

// A run table block per slab: run ends in order and at most nd, the slots of
// its entries a permutation of 0 .. nd - 1 (the kernel indexes shared memory
// with both unchecked).
bool run_table_ok(const std::vector<float4> &rt, long long tab, int nd, int Na)
{
    std::vector<char> seen(nd);
    for (int m = 0; m < Na; ++m) {
        const long long b = tab + (long long)m * wv_block(nd);
        const float4 h = rt[b];
        const int e[6] = {0, bits_int(h.x), bits_int(h.y), bits_int(h.z), bits_int(h.w), nd};
        for (int k = 0; k < 5; ++k)
            if (e[k] > e[k + 1]) return false;
        std::fill(seen.begin(), seen.end(), 0);
        for (int i = 0; i < nd; ++i) {
            const int slot = bits_int(rt[b + 1 + (long long)WV_ENT * i + 3].z);
            if (slot < 0 || slot >= nd || seen[slot]) return false;
            seen[slot] = 1;
        }
    }
    return true;
}

// Invariants the kernel relies on: every upstream unit has a smaller ticket
// (so a wait is always on a unit that has started), the upstream tiles are the
// neighbours of the same (class, group), every buffer range lies inside its
// allocation, and the run tables are well formed.
bool wave_tables_ok(const WaveHost &t, const WVariant &v, std::string &why)
{
    const int TB = 8 * v.wb, TC = 8 * v.np * v.wc;
    std::vector<char> group_ok(t.n_groups, 0);
    for (size_t i = 0; i < t.units.size(); ++i) {
        const WaveUnit &u = t.units[i];
        if (u.cls < 0 || u.cls >= (int)t.classes.size() || u.nd < 1 || u.nd > v.dmax || u.grp < 0 ||
            u.grp >= t.n_groups) {
            why = "unit " + std::to_string(i) + ": class or direction range";
            return false;
        }
        const WaveClass &C = t.classes[u.cls];
        if (C.pub < 1 || (C.pub & (C.pub - 1)) || C.pub > WAVE_PUB) {
            why = "unit " + std::to_string(i) + ": publication interval";
            return false;
        }
        if (u.tab < 0 || u.tab + (long long)C.Na * wv_block(u.nd) > (long long)t.rtab.size()) {
            why = "unit " + std::to_string(i) + ": run table range";
            return false;
        }
        if (!group_ok[u.grp]) {
            if (!run_table_ok(t.rtab, u.tab, u.nd, C.Na)) {
                why = "unit " + std::to_string(i) + ": run table contents";
                return false;
            }
            group_ok[u.grp] = 1;
        }
        const int ups[2] = {u.up_b, u.up_c};
        for (int k = 0; k < 2; ++k) {
            const int q = ups[k];
            const bool edge = k == 0 ? u.tb == 0 : u.tc == 0;
            if (edge != (q < 0) || q >= (int)i) {
                why = "unit " + std::to_string(i) + ": upstream ticket order";
                return false;
            }
            if (q < 0) continue;
            const WaveUnit &w = t.units[q];
            const bool nb = k == 0 ? (w.tb + TB == u.tb && w.tc == u.tc) : (w.tc + TC == u.tc && w.tb == u.tb);
            const long long o = k == 0 ? w.eb : w.ec;
            const long long len = (long long)C.Na * (k == 0 ? v.wc * 8 * v.np : v.wb * 8) * v.dmax;
            if (!nb || w.cls != u.cls || w.grp != u.grp || w.nd != u.nd || o < 0 || o % 4 || o + len > t.edge_floats) {
                why = "unit " + std::to_string(i) + ": upstream tile or its buffer";
                return false;
            }
        }
        const long long ncell = (long long)C.Na * C.Nb * C.Nc;
        if (u.jpart < 0 || u.jpart + ncell > t.jpart_floats) {
            why = "unit " + std::to_string(i) + ": J partial range";
            return false;
        }
    }
    return true;
}

}  // namespace

int art_wave_variants() { return kNumWave; }

// Default shape for classes of at most maxc directions and a largest grid of
// `cells` cells (measured on GB300): 2 x 2 warps throughout; with 4 slots and
// two rows per lane when no class has more than 4 directions; below 100^3
// cells two rows per lane and 20 slots (more, smaller tiles); above, four rows
// per lane with 12 slots up to 12 directions per class, 17 up to 17, else 19
// (N_side 8, classes of 26-37: two groups each).
int art_wave_default(int maxc, long long cells)
{
    int dmax = 19, np = 2;
    if (maxc <= 4) dmax = 4, np = 1;
    else if (cells < 100LL * 100 * 100) dmax = 20, np = 1;
    else if (maxc <= 12) dmax = 12;
    else if (maxc <= 17) dmax = 17;
    for (int w = 0; w < kNumWave; ++w)
        if (kWave[w].wb == 2 && kWave[w].wc == 2 && kWave[w].dmax == dmax && kWave[w].np == np) return w;
    return 0;
}

// Direction slots of wave variant w (0 if out of range).
int art_wave_dmax(int w) { return w >= 0 && w < kNumWave ? kWave[w].dmax : 0; }

void art_wave_free(art_ctx *ctx)
{
    art_wave_state &W = ctx->wave;
    void *ptrs[] = {W.units, W.classes, W.rtab, W.edge, W.flags};
    for (void *p : ptrs)
        if (p) cudaFree(p);
    ctx->dev_bytes -= W.bytes;
    const long long wait_ns = W.wait_ns;
    const int stall = W.stall_unit;
    W = art_wave_state{};
    W.wait_ns = wait_ns;
    W.stall_unit = stall;
}

// Build the tables of wave variant w for the context's grids and allocate
// its buffers (the J partials are the context's d_jpart).
art_status art_wave_setup(art_ctx *ctx, int w)
{
    if (w < 0 || w >= kNumWave) return art_fail(ctx, ART_E_INVALID, "wave variant out of range");
    const WVariant &v = kWave[w];
    if (v.prepare() < 1) return art_fail(ctx, ART_E_CUDA, "wave kernel variant cannot be launched on this device");
    art_wave_free(ctx);
    WaveHost t;
    build_wave(ctx, v, t);
    std::string why;
    if (!wave_tables_ok(t, v, why)) return art_fail(ctx, ART_E_CUDA, "wave sweep tables inconsistent: " + why);
    art_wave_state &W = ctx->wave;
    W.variant = w;
    W.wb = v.wb;
    W.wc = v.wc;
    W.dmax = v.dmax;
    W.np = v.np;
    W.n_units = (int)t.units.size();
    W.edge_floats = t.edge_floats;
    W.jpart_floats = t.jpart_floats;
    ctx->grids = t.grids;
    ctx->n_classes = (int)t.classes.size();
    ctx->n_part = 0;
    ctx->seg_count = 0;
    for (const art_grid_host &g : ctx->grids) {
        ctx->n_part += g.n_part;
        ctx->seg_count += g.seg_count;
    }
    // All bins in one launch (the units of bin b after those of bin b - 1, so
    // no launch drains between bins) when their edge buffers and J partials
    // fit in a quarter of the free device memory; else one launch per bin.
    int nb = 1;
    if (ctx->nbins > 1 && ctx->nbins <= WV_MAXB) {
        size_t fr = 0, tot = 0;
        if (cudaMemGetInfo(&fr, &tot) == cudaSuccess) {
            const double extra = double(ctx->nbins - 1) * double(t.edge_floats + t.jpart_floats) * sizeof(float);
            if (extra <= 0.25 * double(fr)) nb = ctx->nbins;
        } else {
            cudaGetLastError();
        }
    }
    W.bins_per_launch = nb;
    const size_t ub = t.units.size() * sizeof(WaveUnit), cb = t.classes.size() * sizeof(WaveClass);
    const size_t sb = std::max<size_t>(16, t.rtab.size() * sizeof(float4));
    const size_t eb = std::max<size_t>(16, (size_t)t.edge_floats * nb * sizeof(float));
    // error word, ticket, progress flags of every bin, then (8-byte aligned) four counters of
    // ART_WAVE_STATS builds
    const size_t fb =
        ((size_t(W.n_units) * (v.wb + v.wc) * nb + 2) * sizeof(int) + 7) / 8 * 8 + 4 * sizeof(long long);
    struct {
        void **p;
        size_t b;
    } al[] = {{&W.units, ub}, {&W.classes, cb}, {&W.rtab, sb},
              {reinterpret_cast<void **>(&W.edge), eb}, {reinterpret_cast<void **>(&W.flags), fb}};
    for (auto &a : al) {
        const cudaError_t e = cudaMalloc(a.p, a.b ? a.b : 16);
        if (e != cudaSuccess) {
            cudaGetLastError();
            return art_fail(ctx, e == cudaErrorMemoryAllocation ? ART_E_OOM : ART_E_CUDA,
                            "wave sweep buffers (" + std::to_string(a.b) + " bytes): " + cudaGetErrorString(e));
        }
        W.bytes += (long long)a.b;
        ctx->dev_bytes += (long long)a.b;
    }
    W.flag_bytes = fb - 4 * sizeof(long long);   // cleared before every launch (the counters are not)
    W.stats = reinterpret_cast<long long *>(reinterpret_cast<char *>(W.flags) + W.flag_bytes);
    WCK(ctx, cudaMemcpy(W.units, t.units.data(), ub, cudaMemcpyHostToDevice));
    WCK(ctx, cudaMemcpy(W.classes, t.classes.data(), cb, cudaMemcpyHostToDevice));
    if (!t.rtab.empty()) WCK(ctx, cudaMemcpy(W.rtab, t.rtab.data(), t.rtab.size() * sizeof(float4), cudaMemcpyHostToDevice));
    W.rtab_len = (long long)t.rtab.size();
    WCK(ctx, cudaMemset(W.flags, 0, fb));
    W.on = true;
    return ART_OK;
}

// The wavefront sweep of bins b0 .. b0 + bins_per_launch - 1 (fields of bin
// b0 at f0, f1, f2, the next bins bin_cells elements further) into the
// context's J partials (bin b0 + k at k jpart_floats): clear the ticket and
// progress flags (the error word, flags[0], is kept until read), launch.
art_status art_wave_launch(art_ctx *ctx, const float2 *f0, const float2 *f1, const float2 *f2,
                           long long bin_cells, int b0, cudaStream_t st)
{
    art_wave_state &W = ctx->wave;
    const WVariant &v = kWave[W.variant];
    const int nb = W.bins_per_launch;
    if (nb < 1 || nb > WV_MAXB || b0 < 0 || b0 + nb > ctx->nbins)
        return art_fail(ctx, ART_E_INVALID, "wave sweep: bins of a launch out of range");
    WCK(ctx, cudaMemsetAsync(W.flags + 1, 0, W.flag_bytes - sizeof(int), st));
    WaveArgs a{};
    a.field0 = f0;
    a.field1 = f1;
    a.field2 = f2;
    a.n_bins = nb;
    a.bin_cells = bin_cells;
    for (int k = 0; k < nb; ++k) a.i_bc[k] = float(ctx->i_bc[b0 + k]);
    a.rtab = static_cast<const float4 *>(W.rtab);
    a.rtab_len = W.rtab_len;
    a.units = static_cast<const WaveUnit *>(W.units);
    a.classes = static_cast<const WaveClass *>(W.classes);
    a.jpart = static_cast<float *>(ctx->d_jpart);
    a.edge = W.edge;
    a.err = W.flags;
    a.ticket = W.flags + 1;
    a.flags = W.flags + 2;
    a.n_units = W.n_units;
    a.field_form = ctx->opt.field_form;
    a.stall_unit = W.stall_unit;
    a.wait_ns = W.wait_ns;
    a.edge_floats = W.edge_floats;
    a.jpart_floats = W.jpart_floats;
    a.stats = W.stats;
    if (W.n_units == 0) return ART_OK;
    WCK(ctx, v.launch(a, W.n_units * nb, st));
    return ART_OK;
}

// Read and clear the error word (synchronizes the stream).
art_status art_wave_status(art_ctx *ctx, cudaStream_t st)
{
    art_wave_state &W = ctx->wave;
    if (!W.on) return ART_OK;
    int err = 0;
    WCK(ctx, cudaMemcpyAsync(&err, W.flags, sizeof(int), cudaMemcpyDeviceToHost, st));
    WCK(ctx, cudaStreamSynchronize(st));
    if (err) WCK(ctx, cudaMemsetAsync(W.flags, 0, sizeof(int), st));
    if (err & 2) return art_fail(ctx, ART_E_CUDA, "wave sweep: an index check failed (checked build)");
    if (err & 1) return art_fail(ctx, ART_E_TIMEOUT, "wave sweep: a wait for an upstream tile ran out");
    return ART_OK;
}

// Enqueue a copy of the error word to host memory (read after the stream's
// next synchronization).
art_status art_wave_status_async(art_ctx *ctx, int *host, cudaStream_t st)
{
    art_wave_state &W = ctx->wave;
    *host = 0;
    if (!W.on) return ART_OK;
    WCK(ctx, cudaMemcpyAsync(host, W.flags, sizeof(int), cudaMemcpyDeviceToHost, st));
    return ART_OK;
}

// Counters of a build with ART_WAVE_STATS (a profiling aid): cycles warps
// spent at the step barriers, cycles in their units, cycles of lane 0 in the
// poll loops and the number of polls, summed over the launches since the last
// call; read and cleared.  Zeros in other builds.
extern "C" art_status art_wave_counters(art_ctx *ctx, long long *out)
{
    if (!ctx || !out) return ART_E_INVALID;
    for (int i = 0; i < 4; ++i) out[i] = 0;
    art_wave_state &W = ctx->wave;
    if (!W.on) return ART_OK;
    WCK(ctx, cudaDeviceSynchronize());
    WCK(ctx, cudaMemcpy(out, W.stats, 4 * sizeof(long long), cudaMemcpyDeviceToHost));
    WCK(ctx, cudaMemset(W.stats, 0, 4 * sizeof(long long)));
    return ART_OK;
}
