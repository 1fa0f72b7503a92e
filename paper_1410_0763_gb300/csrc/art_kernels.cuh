// art_kernels.cuh -- device kernels of the diffuse-radiation sweep.
//
// Sweep organisation (GB300 design; the paper's thread-per-ray layout with
// four ray groups, Sec. 3.1, is prior art and is not used):
//
//  * Directions are grouped into octant-axis classes (dominant axis and the
//    signs of the three components).  In a class's canonical frame (axes
//    mirrored so that all components are >= 0) all rays advance in +a, +b, +c.
//  * The ray family of a direction is represented by its "intensity plane":
//    at each a-plane u = m exactly one ray sits in every transverse column, at
//    the same fractional offset.  A slab m <= u < m+1 cuts every ray into the
//    same 1-3 segments (tabulated per direction and slab on the host), so each
//    cell of the slab receives exactly one segment of each kind: kind 1 from
//    the ray starting in its own column, kinds 2 and 3 from the rays starting
//    one column upstream.  Hence the cell's total chord length is exactly
//    1/|n_a| and the Delta-tau-weighted average of Eq. (averaged_intensity) is
//    |n_a| * sum_k ds_k Ibar_in_k (kappa is constant in a cell).
//  * A thread owns a transverse column; within a slab it computes the kinds
//    in order, receiving the intensity of kinds 2 and 3 from the upstream
//    neighbour through shared memory.  The deposit of a cell is summed in a
//    fixed order (kind 1, 2, 3) in registers: no atomics anywhere.
//  * A CTA owns a T_b x T_c tile of columns for BLK consecutive slabs and all
//    directions of its class (or a group of them), so the cell's J partial
//    stays in registers (Kahan-compensated) across directions.  Rays enter the
//    tile from upstream: the CTA also recomputes the upstream "cone" of
//    columns, at most BLK wide, starting from the plane values that the
//    previous launch stored.  Values in the cone that depend on columns
//    outside it are wrong but never reach the owned tile (a ray moves at most
//    one column per slab).  Rays enter the box with the boundary intensity
//    (0 for vacuum): the first slab block starts every column with it, and
//    columns outside the box keep it (their cells have kappa = S = 0).
//  * One launch per slab block; plane buffers ping-pong between launches.
//    Each class writes its J partial once per cell; a reduce kernel sums the
//    partials in fixed class order.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace art {

template <typename T> struct Vec2;
template <> struct Vec2<float> { using type = float2; };
template <> struct Vec2<double> { using type = double2; };

// Segment table entry of one (direction, slab).
// code bits: 0-1 nseg-1, 2 c-plane crossed first, 3 b-shift, 4 c-shift,
// 5-8 and 9-12 the b- and c-shifts from this slab to the end of its slab
// block (this slab included).
template <typename real> struct SegEntry {
    real ds1, ds2, ds3;
    int code;
};

struct ClassDev {
    int a, sa, sb, sc;
    int Na, Nb, Nc;
    int dir_begin, dir_end;   // into the class-sorted direction table
    int part0;                // first J partial of the class within its grid
    int nx, ny, nz;           // the grid of this class (natural layout)
    long long cell_off;       // first cell of the grid in the concatenated cell arrays
    long long jpart_off;      // first element of the class's J partials
    long long ncell;          // cells of the grid
};

// One grid of a batch, for the partial reduction.
template <typename real> struct GridDev {
    long long cell_off, ncell, jpart_off;
    int n_part;
    real inv_nd;
};

struct DirDev {
    long long seg_off;        // first SegEntry of this direction
    long long plane_off;      // first element of its plane (canonical [c][b])
    double na;                // |n_a|
};

struct WorkItem {
    int cls, pb, pc, group;   // class, tile origin (canonical b, c), direction group
};

template <typename real> struct alignas(4 * sizeof(real)) Quad {
    real x, y, z, w;
};

template <typename real> struct SweepArgs {
    const typename Vec2<real>::type *field0, *field1, *field2;   // (kappa, src), axis-a layouts, one bin
    const real *plane_in;
    real *plane_out;
    real *jpart;                 // J partials, natural [z][y][x] layout per grid
    const SegEntry<real> *segs;
    const DirDev *dirs;
    const ClassDev *classes;
    const WorkItem *work;
    int n_work;
    int *counter;                // persistent mode: work-queue head (0 before the launch); else null
    int split;
    int kblock;
    int field_form;
    real i_bc;                   // intensity of every ray where it enters the box (0: vacuum)
    int averaging;               // 0: the paper's cell average; 1: the exact path average
};

// ---------------------------------------------------------------------------
// Per-segment arithmetic
// ---------------------------------------------------------------------------
__device__ __forceinline__ float ex2_approx(float x)
{
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// Programmatic dependent launch: let the next kernel on the stream begin its
// CTAs now (they wait on grid_dep_wait before reading what this one writes),
// and wait for the previous kernel to complete and its writes to be visible.
// Both are no-ops for a launch made without the attribute.
__device__ __forceinline__ void grid_dep_launch() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }
__device__ __forceinline__ void grid_dep_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

__device__ __forceinline__ void kahan_add(float &s, float &c, float v)
{
    const float y = __fsub_rn(v, c);
    const float t = __fadd_rn(s, y);
    c = __fsub_rn(__fsub_rn(t, s), y);
    s = t;
}

__device__ __forceinline__ void kahan_add(double &s, double &c, double v)
{
    const double y = __dsub_rn(v, c);
    const double t = __dadd_rn(s, y);
    c = __dsub_rn(__dsub_rn(t, s), y);
    s = t;
}

// ---------------------------------------------------------------------------
// Pair arithmetic: two directions per operation.  FP32 uses the packed
// FP32x2 instructions of sm_100+ (one issue slot for two lanes); FP64 is
// component-wise.
// ---------------------------------------------------------------------------
template <typename real> struct PairOps;
template <> struct PairOps<float> {
    using T = float2;
    static __device__ __forceinline__ T mk(float a, float b) { return make_float2(a, b); }
    static __device__ __forceinline__ T splat(float a) { return make_float2(a, a); }
    static __device__ __forceinline__ T mul(T a, T b) { return __fmul2_rn(a, b); }
    static __device__ __forceinline__ T fma(T a, T b, T c) { return __ffma2_rn(a, b, c); }
};
template <> struct PairOps<double> {
    using T = double2;
    static __device__ __forceinline__ T mk(double a, double b) { return make_double2(a, b); }
    static __device__ __forceinline__ T splat(double a) { return make_double2(a, a); }
    static __device__ __forceinline__ T mul(T a, T b) { return make_double2(a.x * b.x, a.y * b.y); }
    static __device__ __forceinline__ T fma(T a, T b, T c)
    {
        return make_double2(::fma(a.x, b.x, c.x), ::fma(a.y, b.y, c.y));
    }
};

// Per-cell values used by every segment in the cell.
template <typename real> struct CellVals {
    real kap, src, k2, rk0, z;   // kappa, S or eps, -kappa log2 e, 1/kappa (0 if kappa = 0), [kappa == 0]
};

template <typename real> __device__ __forceinline__ CellVals<real> cell_vals(real kap, real src);
template <> __device__ __forceinline__ CellVals<float> cell_vals<float>(float kap, float src)
{
    CellVals<float> c;
    c.kap = kap;
    c.src = src;
    c.k2 = -1.4426950408889634f * kap;
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(kap));
    c.rk0 = kap > 0.0f ? r : 0.0f;
    c.z = kap > 0.0f ? 0.0f : 1.0f;
    return c;
}
template <> __device__ __forceinline__ CellVals<double> cell_vals<double>(double kap, double src)
{
    CellVals<double> c;
    c.kap = kap;
    c.src = src;
    c.k2 = 0.0;
    c.rk0 = 0.0;
    c.z = 0.0;
    return c;
}

// Coefficients of one segment for two directions at once (path lengths ds),
// x = kappa ds:  xph = x phi(x) = 1 - e^-x,  dsph = ds phi(x)
// (phi = (1 - e^-x)/x, the path-averaged attenuation of the segment, Sec. 2.2).
// FP32: below x = 1/4 the Maclaurin series sum_n (-x)^n/(n+1)! to n = 5
// (truncation < 6e-8 relative); above, 1 - 2^(-x log2 e) from the hardware
// base-2 exponential (relative error ~2^-22, < 1e-6 on 1 - e^-x there).
// dsph = xph / kappa, except ds itself where kappa = 0 (phi(0) = 1), so no
// division or select runs for it.
__device__ __forceinline__ void seg_coef2(const CellVals<float> &c, float2 ds, float2 &dsph, float2 &xph)
{
    using P = PairOps<float>;
    const float2 x = P::mul(P::splat(c.kap), ds);
    float2 q = P::fma(x, P::splat(-1.0f / 720.0f), P::splat(1.0f / 120.0f));
    q = P::fma(x, q, P::splat(-1.0f / 24.0f));
    q = P::fma(x, q, P::splat(1.0f / 6.0f));
    q = P::fma(x, q, P::splat(-0.5f));
    q = P::fma(x, q, P::splat(1.0f));
    const float2 arg = P::mul(P::splat(c.k2), ds);
    const float2 e = make_float2(ex2_approx(arg.x), ex2_approx(arg.y));
    const float2 om = P::fma(e, P::splat(-1.0f), P::splat(1.0f));
    const float2 xq = P::mul(x, q);
    xph.x = x.x < 0.25f ? xq.x : om.x;
    xph.y = x.y < 0.25f ? xq.y : om.y;
    dsph = P::fma(ds, P::splat(c.z), P::mul(xph, P::splat(c.rk0)));
}

__device__ __forceinline__ void seg_coef2(const CellVals<double> &c, double2 ds, double2 &dsph, double2 &xph)
{
    const double x0 = c.kap * ds.x, x1 = c.kap * ds.y;
    const double p0 = x0 > 0.0 ? -expm1(-x0) / x0 : 1.0;
    const double p1 = x1 > 0.0 ? -expm1(-x1) / x1 : 1.0;
    dsph = make_double2(ds.x * p0, ds.y * p1);
    xph = make_double2(x0 * p0, x1 * p1);
}

// ds^2 psi(x), psi = (1 - phi)/x (-> 1/2 at x = 0): the emission part of the
// exact path average with emissivity inputs, ds <I> = I_in dsph + eps ds^2 psi.
// FP32: the Maclaurin series of psi below x = 1/4, else (x - xph)/kappa^2.
__device__ __forceinline__ float2 seg_psids(const CellVals<float> &c, float2 ds, float2 xph)
{
    using P = PairOps<float>;
    const float2 x = P::mul(P::splat(c.kap), ds);
    float2 q = P::fma(x, P::splat(-1.0f / 5040.0f), P::splat(1.0f / 720.0f));
    q = P::fma(x, q, P::splat(-1.0f / 120.0f));
    q = P::fma(x, q, P::splat(1.0f / 24.0f));
    q = P::fma(x, q, P::splat(-1.0f / 6.0f));
    q = P::fma(x, q, P::splat(0.5f));
    const float2 small = P::mul(P::mul(ds, ds), q);
    const float r2 = c.rk0 * c.rk0;
    return make_float2(x.x < 0.25f ? small.x : (x.x - xph.x) * r2, x.y < 0.25f ? small.y : (x.y - xph.y) * r2);
}

__device__ __forceinline__ double2 seg_psids(const CellVals<double> &c, double2 ds, double2)
{
    const double x0 = c.kap * ds.x, x1 = c.kap * ds.y;
    auto psi = [](double x) {
        return x < 1e-3 ? 0.5 - x / 6.0 + x * x / 24.0 - x * x * x / 120.0 : (x + expm1(-x)) / (x * x);
    };
    return make_double2(ds.x * ds.x * psi(x0), ds.y * ds.y * psi(x1));
}

// Eq. (rt) for a pair: the deposit, then I = S + (I - S) e^-x (form 0) or
// I = I e^-x + eps ds phi (form 1, S = eps/kappa).  Deposit of the paper's
// average (avg 0): A += I_in dsph, the path-averaged incoming intensity times
// the segment length.  Exact path average (avg 1): A += (I_in - S) dsph with
// source-function inputs (J = S + the cell average), or the whole
// ds <I> = I_in dsph + eps ds^2 psi with emissivity inputs.
template <typename real>
__device__ __forceinline__ void seg_apply2(typename PairOps<real>::T &I, typename PairOps<real>::T &A, real src,
                                           typename PairOps<real>::T dsph, typename PairOps<real>::T xph, int form,
                                           int avg, const CellVals<real> &c, typename PairOps<real>::T ds)
{
    using P = PairOps<real>;
    if (avg == 0)
        A = P::fma(I, dsph, A);
    else if (form == 0)
        A = P::fma(P::fma(I, P::splat(real(1)), P::splat(-src)), dsph, A);
    else
        A = P::fma(P::splat(src), seg_psids(c, ds, xph), P::fma(I, dsph, A));
    if (form == 0) {
        const auto d = P::fma(I, P::splat(real(-1)), P::splat(src));
        I = P::fma(d, xph, I);
    } else {
        const auto t = P::fma(P::splat(src), dsph, I);
        I = P::fma(I, P::mul(xph, P::splat(real(-1))), t);
    }
}

// ---------------------------------------------------------------------------
// Slab-block sweep kernel.  Grid: one CTA per work item (class, tile, group).
// The CTA takes the directions of its group K = 2 KP at a time: for each slab
// the K directions share the cell loads and the exchange barriers, and each
// thread carries K independent intensity chains per column, two per packed
// operation.  A step in which a direction has no segment is an exact no-op
// (ds = 0, fetched from its own column), so all K run the same code.
// Shared memory: (kappa, src) of the region (tile + BLK + 1 upstream
// columns) for the BLK slabs, two exchange buffers of K planes (pairs
// interleaved) over the region, and the decoded segment tables of a chunk of
// directions.  Region columns outside the box hold kappa = S = 0 and their
// exchange slots are never written: rays there carry the boundary intensity.
// ---------------------------------------------------------------------------
template <typename real> struct DirSm {
    long long plane_off;
    real na;
    int d0b, d0c;    // column shifts over the slab block
};

// Decoded segment entry of a pair of directions (the two lanes of a packed
// operation) in one slab: path lengths (0 where a direction has no such
// segment) and, per exchange step, the offsets in elements of the
// pair-interleaved exchange buffer of the column that feeds each lane
// (12 bits each, 0 = its own column); bits 24 and 25 of off3 say whether
// either direction has a segment 2 or 3.
template <typename real> struct alignas(2 * sizeof(real)) PairSm {
    typename Vec2<real>::type ds1, ds2, ds3;
    int off2, off3;
};

template <int TB, int TC, int BLK, int NT, int KP> struct SweepShape {
    static constexpr int K = 2 * KP;
    static constexpr int HB = BLK + 1;
    static constexpr int WB = TB + HB, WC = TC + HB, NS = WB * WC;
    static constexpr int OPT = (TB * TC) / NT;
    static constexpr int MAXH = BLK * (TB + BLK) + TC * BLK;
    static constexpr int HPT = (MAXH + NT - 1) / NT;
    static constexpr int DCH = 8 * K;   // directions staged per chunk
    template <typename real> __host__ __device__ static constexpr size_t off_x()
    {
        return (size_t(BLK) * NS * sizeof(typename Vec2<real>::type) + 31) / 32 * 32;
    }
    template <typename real> __host__ __device__ static constexpr size_t off_t()
    {
        return (off_x<real>() + 2 * size_t(K) * NS * sizeof(real) + 31) / 32 * 32;
    }
    template <typename real> __host__ __device__ static constexpr size_t off_d()
    {
        return off_t<real>() + size_t(DCH / 2) * BLK * sizeof(PairSm<real>);
    }
    template <typename real> __host__ __device__ static constexpr size_t off_g()
    {
        return (off_d<real>() + size_t(DCH) * sizeof(DirSm<real>) + 15) / 16 * 16;
    }
    template <typename real> __host__ __device__ static constexpr size_t bytes()
    {
        return off_g<real>() + size_t(DCH / K) * BLK * sizeof(int4);
    }
};

template <typename real, int TB, int TC, int BLK, int NT, int KP, int AVG>
__device__ __forceinline__ void sweep_item(const SweepArgs<real> &p, int item, unsigned char *smem_raw)
{
    using v2 = typename Vec2<real>::type;
    using P = PairOps<real>;
    using pr = typename P::T;
    using Sh = SweepShape<TB, TC, BLK, NT, KP>;
    constexpr int HB = Sh::HB, WB = Sh::WB, WC = Sh::WC, NS = Sh::NS, OPT = Sh::OPT, HPT = Sh::HPT,
                  DCH = Sh::DCH, K = Sh::K;
    static_assert((TB * TC) % NT == 0, "owned columns must split evenly over threads");
    static_assert(WB * WC < 4096, "exchange offsets are packed in 12 bits");

    v2 *ks = reinterpret_cast<v2 *>(smem_raw);
    pr *xbuf = reinterpret_cast<pr *>(smem_raw + Sh::template off_x<real>());   // [2][KP][NS] pairs
    PairSm<real> *tsm = reinterpret_cast<PairSm<real> *>(smem_raw + Sh::template off_t<real>());
    DirSm<real> *dsm = reinterpret_cast<DirSm<real> *>(smem_raw + Sh::template off_d<real>());
    int4 *gsm = reinterpret_cast<int4 *>(smem_raw + Sh::template off_g<real>());

    const WorkItem w = p.work[item];
    const ClassDev C = p.classes[w.cls];
    const int m0 = p.kblock * BLK;
    if (m0 >= C.Na) return;
    const int Bp = min(BLK, C.Na - m0);
    const int Rb = w.pb - HB, Rc = w.pc - HB;   // origin of the smem region
    const v2 *__restrict__ F = (C.a == 0 ? p.field0 : (C.a == 1 ? p.field1 : p.field2)) + C.cell_off;
    const int tid = threadIdx.x;
    const int form = p.field_form;
    constexpr int avg = AVG;   // averaging mode, fixed per kernel instantiation

    // Stage the region's (kappa, src) for the BLK slabs (vacuum outside the
    // box) and clear the exchange buffers.
    for (int e = tid; e < BLK * WC * WB; e += NT) {
        const int rowi = e / WB, rb = e - rowi * WB;
        const int i = rowi / WC, rc = rowi - i * WC;
        const int gb = Rb + rb, gc = Rc + rc;
        v2 v;
        v.x = real(0);
        v.y = real(0);
        if (i < Bp && gb >= 0 && gc >= 0 && gb < C.Nb && gc < C.Nc) {
            const int am = m0 + i;
            const int pa = C.sa > 0 ? am : C.Na - 1 - am;
            const int pb = C.sb > 0 ? gb : C.Nb - 1 - gb;
            const int pc = C.sc > 0 ? gc : C.Nc - 1 - gc;
            v = F[((long long)pa * C.Nc + pc) * C.Nb + pb];
        }
        ks[e] = v;
    }
    // columns outside the box are never written: they carry the boundary intensity
    for (int e = tid; e < 2 * KP * NS; e += NT) xbuf[e] = P::splat(p.i_bc);

    int o_gb[OPT], o_gc[OPT], o_r[OPT];
    bool o_ok[OPT];
#pragma unroll
    for (int s = 0; s < OPT; ++s) {
        const int o = tid + s * NT;
        o_gb[s] = w.pb + o % TB;
        o_gc[s] = w.pc + o / TB;
        o_r[s] = (o / TB + HB) * WB + (o % TB + HB);
        o_ok[s] = o_gb[s] < C.Nb && o_gc[s] < C.Nc;
    }
    real js[OPT][BLK], jc[OPT][BLK];
#pragma unroll
    for (int s = 0; s < OPT; ++s)
#pragma unroll
        for (int i = 0; i < BLK; ++i) js[s][i] = jc[s][i] = real(0);

    const int nd = C.dir_end - C.dir_begin;
    const int d0 = C.dir_begin + (int)((long long)nd * w.group / p.split);
    const int d1 = C.dir_begin + (int)((long long)nd * (w.group + 1) / p.split);
    const bool first = p.kblock == 0;
    int xs = 0;

    int o_r2[OPT];
#pragma unroll
    for (int s = 0; s < OPT; ++s) o_r2[s] = 2 * o_r[s];

    for (int c0 = d0; c0 < d1; c0 += DCH) {
        const int cnt = min(DCH, d1 - c0);
        const int cntk = (cnt + K - 1) / K * K;   // padded with inactive directions
        __syncthreads();   // previous chunk's tables are no longer read
        for (int e = tid; e < (cntk / 2) * BLK; e += NT) {
            const int pl = e / BLK, i = e - pl * BLK;
            real ds[2][3];
            int o2[2], o3[2], ns[2];
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int dl = 2 * pl + h;
                ds[h][0] = ds[h][1] = ds[h][2] = real(0);
                o2[h] = o3[h] = 0;
                ns[h] = 1;   // inactive: one segment of length 0, own column
                if (dl < cnt && i < Bp) {
                    const SegEntry<real> g = p.segs[p.dirs[c0 + dl].seg_off + m0 + i];
                    const int nseg = (g.code & 3) + 1, cf = (g.code >> 2) & 1;
                    const int shb = (g.code >> 3) & 1, shc = (g.code >> 4) & 1;
                    if (nseg == 2) o2[h] = shc * WB + shb;
                    if (nseg == 3) {
                        o2[h] = cf * WB + (1 - cf);
                        o3[h] = (1 - cf) * WB + cf;
                    }
                    ds[h][0] = g.ds1;
                    ds[h][1] = nseg >= 2 ? g.ds2 : real(0);
                    ds[h][2] = nseg == 3 ? g.ds3 : real(0);
                    ns[h] = nseg;
                }
            }
            PairSm<real> q;
            q.ds1 = P::mk(ds[0][0], ds[1][0]);
            q.ds2 = P::mk(ds[0][1], ds[1][1]);
            q.ds3 = P::mk(ds[0][2], ds[1][2]);
            // lane a reads element 2 (c - off) of the exchange buffer, lane b element 2 (c - off) + 1
            q.off2 = (2 * o2[0]) | ((2 * o2[1]) << 12);
            q.off3 = (2 * o3[0]) | ((2 * o3[1]) << 12) | (int(max(ns[0], ns[1]) >= 2) << 24) |
                     (int(max(ns[0], ns[1]) >= 3) << 25);
            tsm[e] = q;
        }
        for (int dl = tid; dl < cnt; dl += NT) {
            const DirDev D = p.dirs[c0 + dl];
            DirSm<real> q;
            q.plane_off = D.plane_off;
            q.na = real(D.na);
            q.d0b = q.d0c = 0;
            dsm[dl] = q;
        }
        // per (group, slab): max segment count and the union of the
        // directions' remaining upstream cones at the start of the slab (the
        // table carries each direction's remaining shifts to the block end)
        for (int e = tid; e < (cntk / K) * BLK; e += NT) {
            const int grp = e / BLK, i = e - grp * BLK;
            int nsmax = 1, ub = 0, uc = 0;
            if (i < Bp) {
                int code[K];
#pragma unroll
                for (int k = 0; k < K; ++k) {
                    const int dl = grp * K + k;
                    code[k] = dl < cnt ? p.segs[p.dirs[c0 + dl].seg_off + m0 + i].code : 0;
                }
#pragma unroll
                for (int k = 0; k < K; ++k) {
                    ub = max(ub, (code[k] >> 5) & 15);
                    uc = max(uc, (code[k] >> 9) & 15);
                    nsmax = max(nsmax, (code[k] & 3) + 1);
                }
            }
            gsm[e] = make_int4(nsmax, ub, uc, 0);
        }
        __syncthreads();
        // the intensity planes and the J partials are shared with the previous launch
        grid_dep_wait();

        for (int g0 = 0; g0 < cnt; g0 += K) {
            const int kk = min(K, cnt - g0);
            const int4 *G = gsm + (g0 / K) * BLK;
            const int D0b = G[0].y, D0c = G[0].z;   // union cone of the group
            long long poff[K];
            pr na2[KP];   // |n_a| of the pair's directions, 0 for padding
#pragma unroll
            for (int kp = 0; kp < KP; ++kp) {
                real na[2];
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const int k = 2 * kp + h;
                    const DirSm<real> D = dsm[g0 + (k < kk ? k : 0)];
                    poff[k] = D.plane_off;
                    na[h] = k < kk ? D.na : real(0);
                }
                na2[kp] = P::mk(na[0], na[1]);
            }
            const int hw = TB + D0b;
            const int n1 = D0c * hw, nh = n1 + TC * D0b;
            int h_gb[HPT], h_gc[HPT], h_r[HPT];
            bool h_ok[HPT], h_w[HPT];
#pragma unroll
            for (int s = 0; s < HPT; ++s) {
                const int h = tid + s * NT;
                int gb = -1, gc = -1;
                if (h < n1) {
                    gc = w.pc - D0c + h / hw;
                    gb = w.pb - D0b + h % hw;
                } else if (h < nh) {
                    const int h2 = h - n1;
                    gc = w.pc + h2 / D0b;
                    gb = w.pb - D0b + h2 % D0b;
                }
                h_w[s] = ((tid & ~31) + s * NT) < nh;   // warp-uniform: this warp has halo work
                h_ok[s] = h < nh && gb >= 0 && gc >= 0 && gb < C.Nb && gc < C.Nc;
                h_gb[s] = gb;
                h_gc[s] = gc;
                h_r[s] = h_ok[s] ? (gc - Rc) * WB + (gb - Rb) : 0;
            }
            pr oI[OPT][KP], hI[HPT][KP];
#pragma unroll
            for (int kp = 0; kp < KP; ++kp) {
                const real *pa = p.plane_in + poff[2 * kp];
                const real *pb = p.plane_in + poff[2 * kp + 1];
                const bool va = !first && 2 * kp < kk, vb = !first && 2 * kp + 1 < kk;
#pragma unroll
                for (int s = 0; s < OPT; ++s) {
                    const long long ci = (long long)o_gc[s] * C.Nb + o_gb[s];
                    oI[s][kp] = P::mk(va && o_ok[s] ? pa[ci] : p.i_bc, vb && o_ok[s] ? pb[ci] : p.i_bc);
                }
#pragma unroll
                for (int s = 0; s < HPT; ++s) {
                    const long long ci = (long long)h_gc[s] * C.Nb + h_gb[s];
                    hI[s][kp] = P::mk(va && h_ok[s] ? pa[ci] : p.i_bc, vb && h_ok[s] ? pb[ci] : p.i_bc);
                }
            }

#pragma unroll
            for (int i = 0; i < BLK; ++i) {
                if (i < Bp) {
                    const int4 Gi = G[i];
                    PairSm<real> g[KP];
#pragma unroll
                    for (int kp = 0; kp < KP; ++kp) g[kp] = tsm[(g0 / 2 + kp) * BLK + i];
                    const v2 *ksi = ks + i * NS;
                    CellVals<real> oc[OPT], hc[HPT];
                    pr oA[OPT][KP];
                    bool h_act[HPT];
#pragma unroll
                    for (int s = 0; s < OPT; ++s) {
                        const v2 c = ksi[o_r[s]];
                        oc[s] = cell_vals<real>(c.x, c.y);
#pragma unroll
                        for (int kp = 0; kp < KP; ++kp) {
                            pr dsph, xph;
                            seg_coef2(oc[s], g[kp].ds1, dsph, xph);
                            oA[s][kp] = P::splat(real(0));
                            seg_apply2<real>(oI[s][kp], oA[s][kp], oc[s].src, dsph, xph, form, avg, oc[s],
                                             g[kp].ds1);
                        }
                    }
#pragma unroll
                    for (int s = 0; s < HPT; ++s) {
                        h_act[s] = h_w[s] && h_ok[s] && h_gb[s] >= w.pb - Gi.y && h_gc[s] >= w.pc - Gi.z;
                        hc[s] = cell_vals<real>(real(0), real(0));
                        if (h_w[s] && h_act[s]) {
                            const v2 c = ksi[h_r[s]];
                            hc[s] = cell_vals<real>(c.x, c.y);
#pragma unroll
                            for (int kp = 0; kp < KP; ++kp) {
                                pr dsph, xph, dummy = P::splat(real(0));
                                seg_coef2(hc[s], g[kp].ds1, dsph, xph);
                                seg_apply2<real>(hI[s][kp], dummy, hc[s].src, dsph, xph, form, 0, hc[s],
                                                 g[kp].ds1);
                            }
                        }
                    }
                    // Segments 2 and 3: publish the intensities, then each column
                    // takes the ray arriving from its upstream neighbour.
#pragma unroll
                    for (int step = 2; step <= 3; ++step) {
                        if (Gi.x < step) break;   // uniform
                        pr *X = xbuf + xs * KP * NS;
#pragma unroll
                        for (int kp = 0; kp < KP; ++kp) {
#pragma unroll
                            for (int s = 0; s < OPT; ++s) X[kp * NS + o_r[s]] = oI[s][kp];
#pragma unroll
                            for (int s = 0; s < HPT; ++s)
                                if (h_w[s] && h_act[s]) X[kp * NS + h_r[s]] = hI[s][kp];
                        }
                        __syncthreads();
#pragma unroll
                        for (int kp = 0; kp < KP; ++kp) {
                            // uniform: neither direction has this segment (a zero-length
                            // segment through an edge still moves the ray to the next column)
                            if (!((g[kp].off3 >> (22 + step)) & 1)) continue;
                            const int ow = step == 2 ? g[kp].off2 : g[kp].off3;
                            const int offa = ow & 4095, offb = (ow >> 12) & 4095;
                            const pr dsv = step == 2 ? g[kp].ds2 : g[kp].ds3;
                            const real *Xr = reinterpret_cast<const real *>(X + kp * NS);
#pragma unroll
                            for (int s = 0; s < OPT; ++s) {
                                pr dsph, xph;
                                seg_coef2(oc[s], dsv, dsph, xph);
                                pr Iin = P::mk(Xr[o_r2[s] - offa], Xr[o_r2[s] + 1 - offb]);
                                seg_apply2<real>(Iin, oA[s][kp], oc[s].src, dsph, xph, form, avg, oc[s], dsv);
                                oI[s][kp] = Iin;
                            }
#pragma unroll
                            for (int s = 0; s < HPT; ++s) {
                                if (h_w[s] && h_act[s]) {
                                    pr dsph, xph, dummy = P::splat(real(0));
                                    seg_coef2(hc[s], dsv, dsph, xph);
                                    pr Iin = P::mk(Xr[2 * h_r[s] - offa], Xr[2 * h_r[s] + 1 - offb]);
                                    seg_apply2<real>(Iin, dummy, hc[s].src, dsph, xph, form, 0, hc[s], dsv);
                                    hI[s][kp] = Iin;
                                }
                            }
                        }
                        xs ^= 1;
                    }
#pragma unroll
                    for (int s = 0; s < OPT; ++s) {
                        if (o_ok[s]) {
                            pr a2 = P::splat(real(0));
#pragma unroll
                            for (int kp = 0; kp < KP; ++kp) a2 = P::fma(oA[s][kp], na2[kp], a2);
                            kahan_add(js[s][i], jc[s][i], a2.x + a2.y);
                        }
                    }
                }
            }
#pragma unroll
            for (int kp = 0; kp < KP; ++kp) {
                real *pa = p.plane_out + poff[2 * kp];
                real *pb = p.plane_out + poff[2 * kp + 1];
#pragma unroll
                for (int s = 0; s < OPT; ++s) {
                    if (!o_ok[s]) continue;
                    const long long ci = (long long)o_gc[s] * C.Nb + o_gb[s];
                    if (2 * kp < kk) pa[ci] = oI[s][kp].x;
                    if (2 * kp + 1 < kk) pb[ci] = oI[s][kp].y;
                }
            }
        }
    }

    // grid fields of the class read here rather than kept live through the march
    const ClassDev *Cg = p.classes + w.cls;
    const int gnx = Cg->nx, gny = Cg->ny;
    real *J = p.jpart + Cg->jpart_off + (long long)w.group * Cg->ncell;
#pragma unroll
    for (int s = 0; s < OPT; ++s) {
        if (!o_ok[s]) continue;
        const int pb = C.sb > 0 ? o_gb[s] : C.Nb - 1 - o_gb[s];
        const int pc = C.sc > 0 ? o_gc[s] : C.Nc - 1 - o_gc[s];
#pragma unroll
        for (int i = 0; i < BLK; ++i) {
            if (i < Bp) {
                const int am = m0 + i;
                const int pa = C.sa > 0 ? am : C.Na - 1 - am;
                const int x = C.a == 0 ? pa : pb;
                const int y = C.a == 1 ? pa : (C.a == 0 ? pb : pc);
                const int z = C.a == 2 ? pa : pc;
                J[((long long)z * gny + y) * gnx + x] = js[s][i] - jc[s][i];
            }
        }
    }
    __syncthreads();   // shared memory is reused by the CTA's next work item
}

// One CTA per work item.  AVG: the averaging mode (0 the paper's, 1 exact),
// a separate instantiation so the paper's path keeps its own registers.
template <typename real, int TB, int TC, int BLK, int NT, int KP, int MINB, int AVG = 0>
__global__ void __launch_bounds__(NT, MINB) sweep_block_kernel(const SweepArgs<real> p)
{
    extern __shared__ __align__(32) unsigned char smem_raw[];
    grid_dep_launch();
    if ((int)blockIdx.x < p.n_work) sweep_item<real, TB, TC, BLK, NT, KP, AVG>(p, blockIdx.x, smem_raw);
}

// Persistent form: a fixed grid of CTAs taking work items from a queue
// (p.counter, zero before the launch).  Items write disjoint outputs, so the
// order in which CTAs take them changes no result.
template <typename real, int TB, int TC, int BLK, int NT, int KP, int MINB, int AVG = 0>
__global__ void __launch_bounds__(NT, MINB) sweep_queue_kernel(const SweepArgs<real> p)
{
    extern __shared__ __align__(32) unsigned char smem_raw[];
    __shared__ int s_item;
    grid_dep_launch();
    for (;;) {
        if (threadIdx.x == 0) s_item = atomicAdd(p.counter, 1);
        __syncthreads();
        const int item = s_item;
        __syncthreads();
        if (item >= p.n_work) break;
        sweep_item<real, TB, TC, BLK, NT, KP, AVG>(p, item, smem_raw);
    }
}

template <typename real> struct ReduceArgs {
    const real *jpart;
    const typename Vec2<real>::type *field_nat;    // (kappa, src) in [z][y][x], concatenated grids, one bin
    const GridDev<real> *grids;
    int n_grids;
    long long total;                               // cells of all grids
    real gamma_coef;     // 4 pi G_b
    int gamma_accum;     // add to gamma instead of overwriting
    int field_form;
    int whole;           // the partials sum to J (exact average, emissivity inputs): J^in = J - S
    real *Jin, *J, *gamma;   // concatenated grids
};

template <typename real> __global__ void reduce_kernel(const ReduceArgs<real> p)
{
    using v2 = typename Vec2<real>::type;
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= p.total) return;
    int lo = 0, hi = p.n_grids - 1;   // the grid holding cell i
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (p.grids[mid].cell_off <= i) lo = mid;
        else hi = mid - 1;
    }
    const GridDev<real> G = p.grids[lo];
    const long long l = i - G.cell_off;
    real s = real(0), c = real(0);
    for (int k = 0; k < G.n_part; ++k) kahan_add(s, c, p.jpart[G.jpart_off + (long long)k * G.ncell + l]);
    const real acc = (s - c) * G.inv_nd;
    real jin = acc;
    if (p.J || p.whole) {
        const v2 f = p.field_nat[i];
        real S = f.y;
        if (p.field_form == 1) S = f.x > real(0) ? f.y / f.x : real(0);
        if (p.whole) jin = acc - S;
        if (p.J) p.J[i] = p.whole ? acc : acc + S;
    }
    if (p.Jin) p.Jin[i] = jin;
    if (p.gamma) {
        const real g = p.gamma_coef * jin;
        p.gamma[i] = p.gamma_accum ? p.gamma[i] + g : g;
    }
}

// Fill the three axis layouts of (kappa, src) from [z][y][x] arrays.
template <typename real>
__global__ void layout_kernel(const real *kap, const real *src, typename Vec2<real>::type *f0,
                              typename Vec2<real>::type *f1, typename Vec2<real>::type *f2,
                              int nx, int ny, int nz)
{
    const long long n = (long long)nx * ny * nz;
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int x = (int)(i % nx);
    const int y = (int)((i / nx) % ny);
    const int z = (int)(i / ((long long)nx * ny));
    typename Vec2<real>::type v;
    v.x = kap[i];
    v.y = src[i];
    f2[i] = v;
    f1[((long long)y * nz + z) * nx + x] = v;
    f0[((long long)x * nz + z) * ny + y] = v;
}

// Input check: bit 0 = kappa negative or not finite, bit 1 = src not finite.
template <typename real>
__global__ void validate_kernel(const real *kap, const real *src, long long n, int *flag)
{
    int bad = 0;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const real k = kap[i], s = src[i];
        if (!(k >= real(0)) || isinf(k)) bad |= 1;
        if (isnan(s) || isinf(s)) bad |= 2;
    }
    if (bad) atomicOr(flag, bad);
}

}  // namespace art
