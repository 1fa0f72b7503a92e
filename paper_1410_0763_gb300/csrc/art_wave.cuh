// art_wave.cuh -- wavefront sweep kernel (FP32, the paper's cell average).
//
// The same discretization as the slab-block kernel of art_kernels.cuh (Sec. 2.2:
// per direction the family of parallel rays one cell apart, Eq. (rt) per
// segment, the Delta-tau (= Delta-s) weighted cell average of
// Eq. (averaged_intensity), the angle average of Eq. (mean_intensity)), laid out
// as a wavefront so that no ray segment is computed twice and one launch covers
// the whole sweep of a bin, or of every bin when their buffers fit:
//
//  * Directions are grouped into octant-axis classes; in a class's canonical
//    frame (axes mirrored so that every component is >= 0) rays advance in +a
//    (slab by slab), +b and +c.  Slab m of a direction cuts every ray into the
//    same 1-3 segments, so a cell receives at most one segment of each kind:
//    kind 1 from the ray that enters the slab in its own column, kind 2 from
//    the ray one column upstream along the axis crossed first, kind 3 from the
//    diagonal neighbour.
//  * A warp owns an 8 (b) x 8 NP (c) tile of ray columns and, at each step,
//    one slab of it; a lane owns 2 NP columns (neighbouring c rows, in NP
//    pairs), so it marches 2 NP cells per direction.  The intensity handed
//    from a column to its downstream neighbour moves inside the lane (between
//    its rows), by a warp shuffle, through shared memory at the warp's edges,
//    or through global memory at the CTA's edges.  The intensity of the ray
//    that sits in each column, per direction, is kept in shared memory between
//    slabs, so the direction loop stays rolled (small code).
//  * A CTA owns WB x WC warp tiles.  Warp (wb, wc) handles slab t - wb - wc at
//    step t, so everything it receives from the warps upstream of it was
//    written one step earlier (double-buffered by step parity): one barrier
//    per step, and every segment is computed once.
//  * A unit of work is (grid, class, direction group, CTA tile) over all slabs,
//    for one bin.  Units are numbered in an order in which every unit comes
//    after the two units upstream of it (the tile diagonal; bin by bin), and
//    a CTA takes the next number from a ticket counter when it starts.  A CTA waits only on units with
//    smaller tickets, which are running or done, so the waits always end.
//    Each warp row on a CTA's downstream faces publishes its progress every
//    C.pub slabs (release at GPU scope); the downstream warp polls only when
//    the last value it saw does not cover the slab it needs (then acquires).
//    Every wait is bounded in time; one that runs out sets an error word,
//    after which every CTA leaves its loop at the next step.
//  * Per slab, the directions of a group are listed in five runs by segment
//    pattern (one segment; two, hand-off along b or c; three, b or c crossed
//    first), so each run is a branch-free loop; the entry's slot names the
//    direction's ray states and hand-off buffers.
//  * Each unit writes the J partial of its (class, direction group) once per
//    cell: the FP32 sum over its directions (at most DMAX, in run order).
//    reduce_kernel sums the partials in fixed order with Kahan compensation.
//    Results are deterministic.
//  * The two cells of a pair share every segment length, so the arithmetic of
//    Eq. (rt) runs as packed FP32x2 instructions on both.
//  * Arithmetic per (warp, slab), chosen by ballot over the warp's cells:
//    every kappa below KAP_THIN2, KAP_THIN or KAP_THIN5 (series only, of
//    degree 2, 3 or 5 with economized coefficients, as a polynomial in the
//    segment length with per-cell coefficients), every kappa at or above
//    KAP_THICK (hardware exponential only), else both with a per-segment
//    select (series below x = 1/4).  The series path deposits
//    ds phi(x) directly, so kappa = 0 needs no special case; the exponential
//    path deposits 1 - e^-x and the cell's sum is scaled by 1/kappa once.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace art {

// A (grid, class) of the wavefront: canonical frame and natural strides.
struct WaveClass {
    int a, sa, sb, sc;
    int Na, Nb, Nc;
    int pub;                  // slabs between progress publications (a power of two)
    long long cell_off;       // first cell of the grid in the concatenated field arrays
    long long stride_a, stride_b, stride_c;   // natural-layout strides of axes a, b, c
};

// A unit of the wavefront: one CTA tile of one (grid, class, direction group).
struct WaveUnit {
    int cls;                  // WaveClass index
    int grp, nd;              // direction group (index over all classes), its directions (<= DMAX)
    int tb, tc;               // tile origin in canonical columns
    int up_b, up_c;           // unit index of the upstream tiles along b and c; -1 at the box edge
    int pad;
    long long tab;            // first float4 of the group's run table
    long long jpart;          // first element of the J partial this unit writes
    long long eb, ec;         // first float of its B-face and C-face output buffers
};

// Run table of a direction group: per slab a block of 1 + 4 nd float4.  The
// header (int4) holds the ends of five runs of entries, by segment pattern:
// one segment; two with the hand-off along b; two along c; three, b first;
// three, c first.  Entry = 4 float4: (ds_k, ds_k, ds_k^2, ds_k^2) for the
// segments k = 1..3 (zero past the pattern's count), then (|n_a|, |n_a|,
// direction slot as int bits, 0).  Packed pairs load straight into the
// register pairs of the FP32x2 arithmetic.
constexpr int WV_ENT = 4;   // float4 per entry

__host__ __device__ constexpr int wv_block(int nd) { return 1 + WV_ENT * nd; }

constexpr int WV_MAXB = 8;   // bins one launch can hold

struct WaveArgs {
    const float2 *field0, *field1, *field2;   // (kappa, S or eps), sweep-axis layouts, one bin
    const float4 *rtab;       // run tables of the direction groups
    long long rtab_len;       // float4 count (checked builds)
    const WaveUnit *units;    // in ticket order
    const WaveClass *classes;
    float *jpart;
    float *edge;              // B-face [Na][WC][DMAX][4] and C-face [Na][WB][DMAX][8] per unit
    int *flags;               // per unit: WC B-face then WB C-face progress counters (slabs published)
    int *ticket;              // next unit to take (0 before the launch)
    int *err;                 // bit 0: a wait ran out; bit 1: check failure (checked builds)
    int n_units;
    int field_form;           // 0: S, 1: eps
    int n_bins;               // bins in this launch (units of bin b take tickets b n_units ..)
    long long bin_cells;      // field elements from one bin to the next
    float i_bc[WV_MAXB];      // intensity of every ray where it enters the box, per bin
    int stall_unit;           // test hook: this unit never publishes its progress (-1: none)
    long long wait_ns;        // bound of every wait
    long long edge_floats;    // edge buffer of one bin (the bins' buffers follow each other)
    long long jpart_floats;   // J partials of one bin (likewise)
    long long *stats;         // counters of ART_WAVE_STATS builds: barrier, unit, poll-loop cycles, polls
};

// Thresholds of the per-warp arithmetic choice.  The series paths replace
// phi(x) = (1 - e^-x)/x by a polynomial of degree K whose coefficients are
// economized (Chebyshev) on the path's whole range x <= sqrt(3) kappa_max
// (wv_beta): degree 2 to KAP_THIN2 (x <= 0.0329), degree 3 to KAP_THIN (x <=
// 0.165), degree 5 to KAP_THIN5 (x <= 0.866); each approximation is within
// 2e-7 relative of phi there (with FP32 rounding of the coefficient
// polynomial, 2.8e-7 for degree 5; the plain Taylor series would reach only
// x = 0.017, 0.071 and 0.32 with the same degrees).  The mixed path takes a
// series below x = X_SERIES: of degree 4 economized on that range in the
// four-row shapes (within 1.2e-7, 1.8e-7 with FP32 rounding), the degree-5
// one in the two-row shapes; shapes with fewer than 96 registers a thread
// keep the x^5 Taylor series in x below X_SERIES_X (< 6e-8).  Exponential path: 1 - ex2.approx(-x log2
// e), whose absolute error (~2^-22) is below 2e-6 of a cell's deposit when
// kappa >= KAP_THICK, and below 5e-7 of a segment's deposit for x >= X_SERIES.
constexpr float KAP_THIN2 = 0.019f;
constexpr float KAP_THIN = 0.095f;
constexpr float KAP_THIN5 = 0.5f;
constexpr float KAP_THICK = 0.5f;
constexpr float X_SERIES = 0.4f;
constexpr float X_SERIES_X = 0.25f;
constexpr int MODE_THIN = 0, MODE_MIXED = 1, MODE_THICK = 2;

__device__ __forceinline__ float wv_ex2(float x)
{
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

__device__ __forceinline__ float wv_rcp(float x)
{
    float y;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

__device__ __forceinline__ long long wv_now()
{
    long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ int wv_ld_relaxed(const int *p)
{
    int v;
    asm volatile("ld.relaxed.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void wv_st_release(int *p, int v)
{
    asm volatile("st.release.gpu.global.s32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ unsigned wv_smem(const void *p)
{
    return static_cast<unsigned>(__cvta_generic_to_shared(p));
}

// Asynchronous global -> shared copies (L2 only for 16 bytes), completed by
// wv_cp_wait before the step's barrier.
__device__ __forceinline__ void wv_cp16(void *dst, const void *src)
{
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(wv_smem(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void wv_cp8(void *dst, const void *src)
{
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(wv_smem(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void wv_cp_wait()
{
    asm volatile("cp.async.wait_all;" ::: "memory");
}

// Poll a progress flag (relaxed loads), starting from the value v read
// earlier, until it reaches `target` or the wait runs out (or another CTA
// reported an error); a fence then makes the read that saw it an acquire.
// Returns the value seen, or -1 if the wait ran out.
__device__ __forceinline__ int wv_wait(const int *flag, int target, int v, const WaveArgs &p, long long *st)
{
    if (v < target) {
        const long long t0 = wv_now();
#ifdef ART_WAVE_STATS
        const long long c0 = clock64();
#endif
        for (;;) {
            __nanosleep(64);
#ifdef ART_WAVE_STATS
            ++st[1];
#endif
            v = wv_ld_relaxed(flag);
            if (v >= target) break;
            if (wv_ld_relaxed(p.err) != 0 || wv_now() - t0 > p.wait_ns) return -1;
        }
#ifdef ART_WAVE_STATS
        st[0] += clock64() - c0;
#endif
    }
    (void)st;
    asm volatile("fence.acq_rel.gpu;" ::: "memory");
    return v;
}

// Checked builds (ART_WAVE_CHECK) test every global index against its buffer
// before the access, record a failure in bit 1 of the error word and skip the
// access; plain builds compile the test away.
__device__ __forceinline__ bool wv_ok(bool cond, int *err)
{
#ifdef ART_WAVE_CHECK
    if (!cond) atomicOr(err, 2);
    return cond;
#else
    (void)err;
    return true;
#endif
}

__device__ __forceinline__ float2 f2s(float v) { return make_float2(v, v); }

// Per-cell values of a pair of the lane's cells (x: the first row, y: the
// second) for the current slab.  The two cells see the same segment lengths,
// so each FP32 operation of Eq. (rt) runs on both at once as one packed FP32x2
// instruction.
//
// Thin paths (every kappa below KAP_THIN2, KAP_THIN or KAP_THIN5: K = 2, 3 or
// 5): the deposit coefficient of a segment, ds phi(kappa ds) with phi to
// degree K, written as a polynomial in ds whose coefficients are the cell's:
// ds + ds^2 (c_1 + ds (c_2 + ... + ds c_K)), c_k = (-kappa)^k beta_k, where
// beta_k = 1/(k + 1)! for the Taylor series and wv_beta<K>(k) economized.
template <int K> struct WvThin {
    float2 c[K];   // c_1 .. c_K
    float2 nkap;   // -kappa
    float2 E;      // kappa S (S inputs) or eps: emission per unit length
};

// Mixed and thick paths.
struct WvCell2 {
    float2 nkap;  // -kappa per cell width (0 outside the box)
    float2 kap;   // kappa
    float2 E;     // kappa S (S inputs) or eps: emission per unit length
    float2 S;     // source function (exponential path only; kappa > 0 there)
    float2 k2;    // -kappa log2 e
    float2 rk;    // 1/kappa (0 where kappa = 0)
};

// Coefficient of one segment for both cells, from its table pair w = (ds, ds,
// ds^2, ds^2); independent of the intensities, so the coefficients of a
// direction's segments are evaluated side by side.  Thin and mixed paths:
// ds phi(x); thick path: 1 - e^-x (the cell's deposits are scaled by 1/kappa
// at the end).
template <int K> __device__ __forceinline__ float2 wv_coef(const WvThin<K> &c, const float4 &w)
{
    const float2 ds = make_float2(w.x, w.y), ds2 = make_float2(w.z, w.w);
    float2 q = __ffma2_rn(c.c[K - 1], ds, c.c[K - 2]);
#pragma unroll
    for (int k = K - 3; k >= 0; --k) q = __ffma2_rn(q, ds, c.c[k]);
    return __ffma2_rn(q, ds2, ds);
}

// Economized coefficients beta_k (k = 1 .. K; c_k = (-kappa)^k beta_k) of the
// series paths: the Taylor series of psi(x) = (phi(x) - 1)/x, whose x^(k-1)
// coefficient is (-1)^k/(k + 1)!, taken to degree K + 7, rewritten in the
// Chebyshev polynomials of the path's range [0, h], h = sqrt(3) kappa_max,
// and truncated to degree K - 1 (Chebyshev economization; each beta_k lies
// just below its Taylor value 1/(k + 1)!).  Rounded to FP32.
template <int K> __host__ __device__ constexpr float wv_beta(int k);
template <> __host__ __device__ constexpr float wv_beta<2>(int k)   // h = sqrt(3) KAP_THIN2
{
    return k == 1 ? 0.499994397f : 0.165303871f;
}
template <> __host__ __device__ constexpr float wv_beta<3>(int k)   // h = sqrt(3) KAP_THIN
{
    return k == 1 ? 0.499998897f : (k == 2 ? 0.166545019f : 0.0396740399f);
}
template <> __host__ __device__ constexpr float wv_beta<4>(int k)   // h = X_SERIES (mixed path)
{
    return k == 1 ? 0.499999762f : (k == 2 ? 0.166646942f : (k == 3 ? 0.0414167084f : 0.00730631594f));
}
template <> __host__ __device__ constexpr float wv_beta<5>(int k)   // h = sqrt(3) KAP_THIN5
{
    return k == 1 ? 0.499999851f
                  : (k == 2 ? 0.166658416f : (k == 3 ? 0.0415891334f : (k == 4 ? 0.00807498395f : 0.00102687033f)));
}

// The coefficients c_1 .. c_K of a pair of cells.
template <int K> __device__ __forceinline__ WvThin<K> wv_thin(float2 k, float2 src, int field_form)
{
    WvThin<K> c;
    const float2 nk = make_float2(-k.x, -k.y);
    float2 pw = nk;   // (-kappa)^j
#pragma unroll
    for (int j = 1; j <= K; ++j) {
        c.c[j - 1] = __fmul2_rn(pw, f2s(wv_beta<K>(j)));
        pw = __fmul2_rn(pw, nk);
    }
    c.nkap = nk;
    c.E = field_form ? src : __fmul2_rn(k, src);
    return c;
}

// Mixed path: per cell and segment, a series of degree K (per-cell
// coefficients; degree 4 economized on x < X_SERIES, or degree 5, economized
// on a range that covers it) for segments with x = kappa ds below X_SERIES,
// i.e. ds below the cell's threshold X_SERIES / kappa, else the exponential
// path.  (Four-row shapes take degree 4; in the two-row shapes degree 4
// spills registers, so they keep degree 5.)
template <int K> struct WvMixed {
    WvThin<K> t;     // c_1 .. c_K, -kappa, emission
    float2 k2;       // -kappa log2 e
    float2 rk, nrk;  // 1/kappa, -1/kappa (0 where kappa = 0)
    float2 th;       // X_SERIES / kappa (+inf where kappa = 0)
};

template <int K> __device__ __forceinline__ WvMixed<K> wv_mixed(float2 k, float2 src, int field_form)
{
    WvMixed<K> c;
    c.t = wv_thin<K>(k, src, field_form);
    c.k2 = __fmul2_rn(k, f2s(-1.4426950408889634f));
    c.rk = make_float2(k.x > 0.0f ? wv_rcp(k.x) : 0.0f, k.y > 0.0f ? wv_rcp(k.y) : 0.0f);
    c.nrk = make_float2(-c.rk.x, -c.rk.y);
    c.th = make_float2(k.x > 0.0f ? X_SERIES * c.rk.x : __int_as_float(0x7f800000),
                       k.y > 0.0f ? X_SERIES * c.rk.y : __int_as_float(0x7f800000));
    return c;
}

template <int K> __device__ __forceinline__ float2 wv_coef(const WvMixed<K> &c, const float4 &w)
{
    const float2 gs = wv_coef(c.t, w);
    const float2 arg = __fmul2_rn(c.k2, make_float2(w.x, w.y));
    const float2 e = make_float2(wv_ex2(arg.x), wv_ex2(arg.y));
    const float2 gm = __ffma2_rn(e, c.nrk, c.rk);   // (1 - e^-x) / kappa
    return make_float2(w.x < c.th.x ? gs.x : gm.x, w.y < c.th.y ? gs.y : gm.y);
}

template <int MODE> __device__ __forceinline__ float2 wv_coef(const WvCell2 &c, const float4 &w)
{
    const float2 dsv = make_float2(w.x, w.y);
    if (MODE == MODE_THICK) {
        const float2 arg = __fmul2_rn(c.k2, dsv);
        const float2 e = make_float2(wv_ex2(arg.x), wv_ex2(arg.y));
        return __ffma2_rn(e, f2s(-1.0f), f2s(1.0f));
    }
    const float2 x = __fmul2_rn(c.kap, dsv);
    float2 q = __ffma2_rn(x, f2s(-1.0f / 720.0f), f2s(1.0f / 120.0f));
    q = __ffma2_rn(x, q, f2s(-1.0f / 24.0f));
    q = __ffma2_rn(x, q, f2s(1.0f / 6.0f));
    q = __ffma2_rn(x, q, f2s(-0.5f));
    q = __ffma2_rn(x, q, f2s(1.0f));
    const float2 gs = __fmul2_rn(dsv, q);
    const float2 arg = __fmul2_rn(c.k2, dsv);
    const float2 e = make_float2(wv_ex2(arg.x), wv_ex2(arg.y));
    const float2 gm = __fmul2_rn(__ffma2_rn(e, f2s(-1.0f), f2s(1.0f)), c.rk);
    return make_float2(x.x < X_SERIES_X ? gs.x : gm.x, x.y < X_SERIES_X ? gs.y : gm.y);
}

// One segment with coefficient g and incoming intensities I (both cells):
// accumulates the deposits I g into A and returns the outgoing intensities,
// I + (eps - kappa I) ds phi(x) = I + (S - I)(1 - e^-x).
template <bool FIRST, int K>
__device__ __forceinline__ float2 wv_seg(const WvThin<K> &c, float2 I, float2 g, float2 &A)
{
    A = FIRST ? __fmul2_rn(I, g) : __ffma2_rn(I, g, A);
    return __ffma2_rn(__ffma2_rn(c.nkap, I, c.E), g, I);
}

template <int MODE, bool FIRST>
__device__ __forceinline__ float2 wv_seg(const WvCell2 &c, float2 I, float2 g, float2 &A)
{
    A = FIRST ? __fmul2_rn(I, g) : __ffma2_rn(I, g, A);
    if (MODE == MODE_THICK) return __ffma2_rn(__ffma2_rn(I, f2s(-1.0f), c.S), g, I);
    return __ffma2_rn(__ffma2_rn(c.nkap, I, c.E), g, I);
}

// Mode dispatch of the two helpers above (the thin path has its own type).
template <int MODE, class CO> struct WvOps;
template <int K> struct WvOps<MODE_THIN, WvThin<K>> {
    static __device__ __forceinline__ float2 coef(const WvThin<K> &c, const float4 &w) { return wv_coef(c, w); }
    template <bool F>
    static __device__ __forceinline__ float2 seg(const WvThin<K> &c, float2 I, float2 g, float2 &A)
    {
        return wv_seg<F>(c, I, g, A);
    }
};
template <int K> struct WvOps<MODE_MIXED, WvMixed<K>> {
    static __device__ __forceinline__ float2 coef(const WvMixed<K> &c, const float4 &w) { return wv_coef(c, w); }
    template <bool F>
    static __device__ __forceinline__ float2 seg(const WvMixed<K> &c, float2 I, float2 g, float2 &A)
    {
        return wv_seg<F>(c.t, I, g, A);
    }
};
template <int MODE> struct WvOps<MODE, WvCell2> {
    static __device__ __forceinline__ float2 coef(const WvCell2 &c, const float4 &w) { return wv_coef<MODE>(c, w); }
    template <bool F> static __device__ __forceinline__ float2 seg(const WvCell2 &c, float2 I, float2 g, float2 &A)
    {
        return wv_seg<MODE, F>(c, I, g, A);
    }
};

__device__ __forceinline__ void wv_sts(unsigned a, float v) { asm volatile("st.shared.f32 [%0], %1;" ::"r"(a), "f"(v) : "memory"); }
__device__ __forceinline__ float wv_lds(unsigned a)
{
    float v;
    asm volatile("ld.shared.f32 %0, [%1];" : "=f"(v) : "r"(a) : "memory");
    return v;
}
__device__ __forceinline__ void wv_sts2(unsigned a, float x, float y)
{
    asm volatile("st.shared.v2.f32 [%0], {%1, %2};" ::"r"(a), "f"(x), "f"(y) : "memory");
}
__device__ __forceinline__ float2 wv_lds2(unsigned a)
{
    float2 v;
    asm volatile("ld.shared.v2.f32 {%0, %1}, [%2];" : "=f"(v.x), "=f"(v.y) : "r"(a) : "memory");
    return v;
}

// The lane's rows in pairs (rows 2i, 2i + 1 in p[i]): each packed FP32x2
// instruction of a segment works on one pair.
template <int NP> struct WvRows {
    static_assert(NP == 1 || NP == 2, "two or four rows per lane");
    float2 p[NP];
};

// Per-lane exchange state of one step: shared-window byte addresses of this
// lane's slots for direction 0.  B-face slots hold the lane's 2 NP rows (the
// warp's 4 lanes of a column: 32 NP bytes per direction), C-face slots its
// column bl (8 lanes: 32 bytes per direction).
struct WvXch {
    unsigned bo, bi;   // B-face output / input rows
    unsigned co, ci;   // C-face output / input
    bool b0, b7, c0, c3;
    int nslot;         // direction slots (checked builds test table slots against it)
    int *err;
};

template <int NP> __device__ __forceinline__ void wv_sts_rows(unsigned a, const WvRows<NP> &v)
{
    if (NP == 1) {
        wv_sts2(a, v.p[0].x, v.p[0].y);
    } else {
        asm volatile("st.shared.v4.f32 [%0], {%1, %2, %3, %4};" ::"r"(a), "f"(v.p[0].x), "f"(v.p[0].y),
                     "f"(v.p[NP - 1].x), "f"(v.p[NP - 1].y)
                     : "memory");
    }
}

// The same stores, made by the lanes whose flag is set (a predicated store:
// no branch in the direction loop).
template <int NP> __device__ __forceinline__ void wv_sts_rows_if(bool f, unsigned a, const WvRows<NP> &v)
{
    if (NP == 1) {
        asm volatile("{\n\t.reg .pred q;\n\tsetp.ne.b32 q, %0, 0;\n\t@q st.shared.v2.f32 [%1], {%2, %3};\n\t}"
                     ::"r"((int)f), "r"(a), "f"(v.p[0].x), "f"(v.p[0].y)
                     : "memory");
    } else {
        asm volatile("{\n\t.reg .pred q;\n\tsetp.ne.b32 q, %0, 0;\n\t@q st.shared.v4.f32 [%1], {%2, %3, %4, %5};\n\t}"
                     ::"r"((int)f), "r"(a), "f"(v.p[0].x), "f"(v.p[0].y), "f"(v.p[NP - 1].x), "f"(v.p[NP - 1].y)
                     : "memory");
    }
}
__device__ __forceinline__ void wv_sts_if(bool f, unsigned a, float v)
{
    asm volatile("{\n\t.reg .pred q;\n\tsetp.ne.b32 q, %0, 0;\n\t@q st.shared.f32 [%1], %2;\n\t}"
                 ::"r"((int)f), "r"(a), "f"(v)
                 : "memory");
}

template <int NP> __device__ __forceinline__ WvRows<NP> wv_lds_rows(unsigned a)
{
    WvRows<NP> v;
    if (NP == 1) {
        v.p[0] = wv_lds2(a);
    } else {
        asm volatile("ld.shared.v4.f32 {%0, %1, %2, %3}, [%4];"
                     : "=f"(v.p[0].x), "=f"(v.p[0].y), "=f"(v.p[NP - 1].x), "=f"(v.p[NP - 1].y)
                     : "r"(a)
                     : "memory");
    }
    return v;
}

// Hand-off across a b-plane: each of the lane's rows takes the intensity that
// leaves the column one step upstream along b (the lane to the left, or the
// B-face input `in` at bl = 0, loaded beforehand); lanes at bl = 7 write
// theirs to the B-face output.
template <int NP> __device__ __forceinline__ void wv_xb(const WvXch &x, WvRows<NP> &v, int d, const WvRows<NP> &in)
{
    constexpr unsigned XBD = 4 * 4 * 2 * NP;   // bytes per direction: 4 lanes x 2 NP rows
    WvRows<NP> n;
#pragma unroll
    for (int i = 0; i < NP; ++i) {
        n.p[i].x = __shfl_up_sync(0xffffffffu, v.p[i].x, 1);
        n.p[i].y = __shfl_up_sync(0xffffffffu, v.p[i].y, 1);
    }
    if (NP == 1) {   // (the predicated form costs these shapes registers)
        if (x.b7) wv_sts_rows<NP>(x.bo + XBD * d, v);
    } else {
        wv_sts_rows_if<NP>(x.b7, x.bo + XBD * d, v);
    }
#pragma unroll
    for (int i = 0; i < NP; ++i) {
        v.p[i].x = x.b0 ? in.p[i].x : n.p[i].x;
        v.p[i].y = x.b0 ? in.p[i].y : n.p[i].y;
    }
}

// Hand-off across a c-plane: each row after the lane's first takes the row
// before it (registers); the first row takes the last row of the lane one step
// upstream along c (or the C-face input `in` at cl = 0, loaded beforehand);
// lanes at cl = 3 write their last row to the C-face output.
template <int NP> __device__ __forceinline__ void wv_xc(const WvXch &x, WvRows<NP> &v, int d, float in)
{
    const float last = v.p[NP - 1].y;
    const float n = __shfl_up_sync(0xffffffffu, last, 8);
    if (NP == 1) {
        if (x.c3) wv_sts(x.co + 32 * d, last);
    } else {
        wv_sts_if(x.c3, x.co + 32 * d, last);
    }
#pragma unroll
    for (int i = NP - 1; i >= 0; --i) {
        v.p[i].y = v.p[i].x;
        v.p[i].x = i > 0 ? v.p[i - 1].y : (x.c0 ? in : n);
    }
}

template <int NP> __device__ __forceinline__ WvRows<NP> wv_ld_xb(const WvXch &x, int d)
{
    return wv_lds_rows<NP>(x.bi + 4 * 4 * 2 * NP * d);
}
__device__ __forceinline__ float wv_ld_xc(const WvXch &x, int d) { return wv_lds(x.ci + 32 * d); }

__device__ __forceinline__ float4 wv_lds4(unsigned a)
{
    float4 v;
    asm volatile("ld.shared.v4.f32 {%0, %1, %2, %3}, [%4];" : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w) : "r"(a));
    return v;
}

// What one entry of a run needs from shared memory: its segment pairs, its
// |n_a| pair and slot, the ray states of the slot and the hand-off inputs.
template <int NP> struct WvEnt {
    float4 w0, w1, w2;
    float2 na;
    int slot;
    WvRows<NP> o, inb;
    float inc;
};

template <int NT, int NP, int NS, bool FC>
__device__ __forceinline__ WvEnt<NP> wv_ld_ent(unsigned rs, unsigned ent, int d, const WvXch &x)
{
    constexpr unsigned RSD = 8 * NP * NT;   // ray-state bytes per direction slot
    WvEnt<NP> E;
    const unsigned e = ent + 16 * WV_ENT * d;
    const float4 w3 = wv_lds4(e + 48);
    E.slot = __float_as_int(w3.z);
#ifdef ART_WAVE_CHECK
    if (!wv_ok(E.slot >= 0 && E.slot < x.nslot, x.err)) E.slot = 0;
#endif
    E.na = make_float2(w3.x, w3.y);
    E.w0 = wv_lds4(e);
    E.w1 = E.w2 = E.w0;
    if (NS >= 2) E.w1 = wv_lds4(e + 16);
    if (NS >= 3) E.w2 = wv_lds4(e + 32);
    E.o = wv_lds_rows<NP>(rs + RSD * E.slot);
    E.inc = 0.0f;
    if (NS == 3 || (NS == 2 && !FC)) E.inb = wv_ld_xb<NP>(x, E.slot);
    if (NS == 3 || (NS == 2 && FC)) E.inc = wv_ld_xc(x, E.slot);
    return E;
}

// One entry: the segment coefficients first (they do not depend on the
// intensities), then the chain of intensity updates and hand-offs; the ray
// states go back to the slot and the |n_a|-weighted deposits into acc.
template <int MODE, int NT, int NP, int NS, bool FC, class CO>
__device__ __forceinline__ void wv_ent(const CO (&c)[NP], unsigned rs, WvEnt<NP> &E, const WvXch &x,
                                       WvRows<NP> &acc)
{
    using Op = WvOps<MODE, CO>;
    constexpr unsigned RSD = 8 * NP * NT;
    float2 g1[NP], g2[NP], g3[NP];
#pragma unroll
    for (int i = 0; i < NP; ++i) {
        g1[i] = Op::coef(c[i], E.w0);
        if (NS >= 2) g2[i] = Op::coef(c[i], E.w1);
        if (NS >= 3) g3[i] = Op::coef(c[i], E.w2);
    }
    WvRows<NP> A;
    WvRows<NP> &o = E.o;
#pragma unroll
    for (int i = 0; i < NP; ++i) o.p[i] = Op::template seg<true>(c[i], o.p[i], g1[i], A.p[i]);
    if (NS >= 2) {
        if (FC) wv_xc<NP>(x, o, E.slot, E.inc);
        else wv_xb<NP>(x, o, E.slot, E.inb);
#pragma unroll
        for (int i = 0; i < NP; ++i) o.p[i] = Op::template seg<false>(c[i], o.p[i], g2[i], A.p[i]);
    }
    if (NS >= 3) {
        if (FC) wv_xb<NP>(x, o, E.slot, E.inb);
        else wv_xc<NP>(x, o, E.slot, E.inc);
#pragma unroll
        for (int i = 0; i < NP; ++i) o.p[i] = Op::template seg<false>(c[i], o.p[i], g3[i], A.p[i]);
    }
    wv_sts_rows<NP>(rs + RSD * E.slot, o);
#pragma unroll
    for (int i = 0; i < NP; ++i) acc.p[i] = __ffma2_rn(A.p[i], E.na, acc.p[i]);
}

// Two entries of one run in lockstep, statement by statement, so that their
// independent chains sit side by side for the scheduler; the same arithmetic
// and the same order of the deposit sums as two calls of wv_ent.
template <int MODE, int NT, int NP, int NS, bool FC, class CO>
__device__ __forceinline__ void wv_ent2(const CO (&c)[NP], unsigned rs, WvEnt<NP> &E, WvEnt<NP> &F,
                                        const WvXch &x, WvRows<NP> &acc)
{
    using Op = WvOps<MODE, CO>;
    constexpr unsigned RSD = 8 * NP * NT;
    float2 g1[NP], g2[NP], g3[NP], h1[NP], h2[NP], h3[NP];
#pragma unroll
    for (int i = 0; i < NP; ++i) {
        g1[i] = Op::coef(c[i], E.w0);
        h1[i] = Op::coef(c[i], F.w0);
        if (NS >= 2) g2[i] = Op::coef(c[i], E.w1);
        if (NS >= 2) h2[i] = Op::coef(c[i], F.w1);
        if (NS >= 3) g3[i] = Op::coef(c[i], E.w2);
        if (NS >= 3) h3[i] = Op::coef(c[i], F.w2);
    }
    WvRows<NP> A, B;
    WvRows<NP> &o = E.o, &q = F.o;
#pragma unroll
    for (int i = 0; i < NP; ++i) {
        o.p[i] = Op::template seg<true>(c[i], o.p[i], g1[i], A.p[i]);
        q.p[i] = Op::template seg<true>(c[i], q.p[i], h1[i], B.p[i]);
    }
    if (NS >= 2) {
        if (FC) {
            wv_xc<NP>(x, o, E.slot, E.inc);
            wv_xc<NP>(x, q, F.slot, F.inc);
        } else {
            wv_xb<NP>(x, o, E.slot, E.inb);
            wv_xb<NP>(x, q, F.slot, F.inb);
        }
#pragma unroll
        for (int i = 0; i < NP; ++i) {
            o.p[i] = Op::template seg<false>(c[i], o.p[i], g2[i], A.p[i]);
            q.p[i] = Op::template seg<false>(c[i], q.p[i], h2[i], B.p[i]);
        }
    }
    if (NS >= 3) {
        if (FC) {
            wv_xb<NP>(x, o, E.slot, E.inb);
            wv_xb<NP>(x, q, F.slot, F.inb);
        } else {
            wv_xc<NP>(x, o, E.slot, E.inc);
            wv_xc<NP>(x, q, F.slot, F.inc);
        }
#pragma unroll
        for (int i = 0; i < NP; ++i) {
            o.p[i] = Op::template seg<false>(c[i], o.p[i], g3[i], A.p[i]);
            q.p[i] = Op::template seg<false>(c[i], q.p[i], h3[i], B.p[i]);
        }
    }
    wv_sts_rows<NP>(rs + RSD * E.slot, o);
    wv_sts_rows<NP>(rs + RSD * F.slot, q);
#pragma unroll
    for (int i = 0; i < NP; ++i) acc.p[i] = __ffma2_rn(B.p[i], F.na, __ffma2_rn(A.p[i], E.na, acc.p[i]));
}

// One run of a slab's table: entries [d, d1), all with NS segments and, for
// NS >= 2, the first hand-off along c (FC) or b.  (Loading the next entry
// while computing the current one, in register-rich shapes, measured no
// faster.)
template <int MODE, int NT, int NP, int NS, bool FC, bool TWO, class CO>
__device__ __forceinline__ void wv_run(const CO (&c)[NP], unsigned rs, unsigned ent, int d, int d1,
                                       const WvXch &x, WvRows<NP> &acc)
{
    if (TWO) {
        // two entries side by side (independent chains for the scheduler)
#pragma unroll 1
        for (; d + 1 < d1; d += 2) {
            WvEnt<NP> E0 = wv_ld_ent<NT, NP, NS, FC>(rs, ent, d, x);
            WvEnt<NP> E1 = wv_ld_ent<NT, NP, NS, FC>(rs, ent, d + 1, x);
            wv_ent2<MODE, NT, NP, NS, FC>(c, rs, E0, E1, x, acc);
        }
    }
#pragma unroll 1
    for (; d < d1; ++d) {
        WvEnt<NP> E = wv_ld_ent<NT, NP, NS, FC>(rs, ent, d, x);
        wv_ent<MODE, NT, NP, NS, FC>(c, rs, E, x, acc);
    }
}

// All directions of the unit for one slab (table block at tb), for the lane's
// 2 NP cells: returns the cells' sums over the unit's directions of |n_a|
// times the deposits (at most DMAX directions, summed in FP32 in run order;
// the units' partials are summed with Kahan compensation by the reduction).
template <int MODE, int NT, int NP, bool TWO, class CO>
__device__ __forceinline__ WvRows<NP> wv_dirs(const CO (&c)[NP], unsigned rs, unsigned tb, int nd, const WvXch &x)
{
    WvRows<NP> acc;
#pragma unroll
    for (int i = 0; i < NP; ++i) acc.p[i] = f2s(0.0f);
    const float4 hf = wv_lds4(tb);
    int e1 = __float_as_int(hf.x), e2 = __float_as_int(hf.y), e3 = __float_as_int(hf.z), e4 = __float_as_int(hf.w);
#ifdef ART_WAVE_CHECK
    if (!wv_ok(0 <= e1 && e1 <= e2 && e2 <= e3 && e3 <= e4 && e4 <= nd && nd <= x.nslot, x.err))
        e1 = e2 = e3 = e4 = nd = 0;
#endif
    const unsigned ent = tb + 16;
    wv_run<MODE, NT, NP, 1, false, TWO && MODE == MODE_THIN>(c, rs, ent, 0, e1, x, acc);
    wv_run<MODE, NT, NP, 2, false, TWO && MODE == MODE_THIN>(c, rs, ent, e1, e2, x, acc);
    wv_run<MODE, NT, NP, 2, true, TWO && MODE == MODE_THIN>(c, rs, ent, e2, e3, x, acc);
    wv_run<MODE, NT, NP, 3, false, TWO && MODE == MODE_THIN>(c, rs, ent, e3, e4, x, acc);
    wv_run<MODE, NT, NP, 3, true, TWO && MODE == MODE_THIN>(c, rs, ent, e4, nd, x, acc);
    return acc;
}

// Shared-memory and edge-buffer shape of a kernel: WB x WC warps, each an
// 8 (b) x 4 R (c) tile of columns with R = 2 NP rows per lane.
template <int WB, int WC, int DMAX, int NP> struct WaveShape {
    static constexpr int NT = 32 * WB * WC;
    static constexpr int R = 2 * NP;                          // rows per lane
    static constexpr int TB = 8 * WB, TC = 4 * R * WC;
    static constexpr int RT = (WB + WC <= 4) ? 4 : ((WB + WC <= 8) ? 8 : 16);   // table ring (slabs)
    static constexpr int XBW = 4 * R;                         // B-face floats per warp and direction
    static constexpr int XB_PAR = (WB + 1) * WC * DMAX * XBW; // floats per parity
    static constexpr int XC_PAR = (WC + 1) * WB * DMAX * 8;
    static constexpr int TABS = wv_block(DMAX);               // float4 per slab of the table ring
    static constexpr size_t off_xb = size_t(RT) * TABS * 16;
    static constexpr size_t off_xc = off_xb + size_t(2) * XB_PAR * 4;
    static constexpr size_t off_fs = off_xc + size_t(2) * XC_PAR * 4;
    static constexpr size_t off_rs = off_fs + size_t(2) * NT * R * 8;
    static constexpr size_t bytes = off_rs + size_t(DMAX) * NT * R * 4;
    static constexpr long long edge_b(int Na) { return (long long)Na * WC * DMAX * XBW; }
    static constexpr long long edge_c(int Na) { return (long long)Na * WB * DMAX * 8; }
};

// Longest interval between progress publications, in slabs (each costs the
// publishing warp a GPU-scope release, and its consumer an acquire; a class
// publishes every Na/16 slabs, a power of two between 1 and this).
#ifndef ART_WAVE_PUB
#define ART_WAVE_PUB 16
#endif
constexpr int WAVE_PUB = ART_WAVE_PUB;
static_assert(WAVE_PUB >= 1 && (WAVE_PUB & (WAVE_PUB - 1)) == 0, "publication interval");

template <int WB, int WC, int DMAX, int NP, int MINB>
__global__ void __launch_bounds__(32 * WB * WC, MINB) wave_kernel(const WaveArgs p)
{
    using Sh = WaveShape<WB, WC, DMAX, NP>;
    constexpr int NT = Sh::NT, RT = Sh::RT, R = Sh::R, XBW = Sh::XBW;
    // shapes with at least 160 registers a thread take two degree-2-path entries at a time
    constexpr bool TWO = 65536 / (MINB * NT) >= 160;
    // the degree-2 and degree-5 series paths (kappa < KAP_THIN2, KAP_THIN5) and the coefficient
    // form of the mixed path in shapes with at least 96 registers a thread (the others take the
    // degree-3 path below KAP_THIN and the mixed path in x above it)
    constexpr bool THIN5 = 65536 / (MINB * NT) >= 96;
    extern __shared__ __align__(16) unsigned char wsm[];
    float4 *tab = reinterpret_cast<float4 *>(wsm);                  // [RT][TABS]: run-table blocks
    float *XB = reinterpret_cast<float *>(wsm + Sh::off_xb);        // [2][WB+1][WC][DMAX][XBW]
    float *XC = reinterpret_cast<float *>(wsm + Sh::off_xc);        // [2][WC+1][WB][DMAX][8]
    float2 *FS = reinterpret_cast<float2 *>(wsm + Sh::off_fs);      // [2][NT][R]: (kappa, src) of the lane's cells
    float *RS = reinterpret_cast<float *>(wsm + Sh::off_rs);        // [DMAX][NT][R]: ray states of its columns
    __shared__ int s_unit;
    __shared__ long long s_up[2];       // output buffers of the upstream units (B, C)

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int wb = warp % WB, wc = warp / WB;
    const int bl = lane & 7, cl = lane >> 3;
    if (tid == 0) s_unit = atomicAdd(p.ticket, 1);
    __syncthreads();
    const int ticket = s_unit;
    if (ticket >= p.n_units * p.n_bins) return;
    // all bins' units in one launch, bin by bin in ticket order: the units of
    // a bin wait only on units of the same bin, which have smaller tickets
    const int bin = ticket / p.n_units, u = ticket - bin * p.n_units;
    const float i_bc = p.i_bc[bin];
    float *const edge = p.edge + bin * p.edge_floats;
    int *const flags = p.flags + (long long)bin * p.n_units * (WB + WC);
    const WaveUnit U = p.units[u];
    const WaveClass C = p.classes[U.cls];
    const int Na = C.Na, nd = U.nd;
    const int j = U.tb + 8 * wb + bl;                          // canonical b column
    const int k0 = U.tc + 4 * R * wc + R * cl;                  // canonical c rows k0 .. k0 + R - 1
    const int pb = C.sb > 0 ? j : C.Nb - 1 - j;
    const int pc0 = C.sc > 0 ? k0 : C.Nc - 1 - k0;
    const int dpc = C.sc > 0 ? 1 : -1;                          // physical c step from one row to the next
    unsigned inmask = 0;                                        // rows of the lane inside the box
#pragma unroll
    for (int r = 0; r < R; ++r) inmask |= (j < C.Nb && k0 + r < C.Nc) ? 1u << r : 0u;
    // the lane's columns in the axis-a field layout [a][c][b] (row r at
    // F0 + r dpc Nb), and its cells of slab m in the natural layout of the J
    // partial (row r at J0 + r dpc stride_c + m jstep)
    const float2 *Fb = (C.a == 0 ? p.field0 : (C.a == 1 ? p.field1 : p.field2)) + bin * p.bin_cells + C.cell_off;
    const long long f0 = (long long)pc0 * C.Nb + pb;
    const int fslab = C.Nb * C.Nc, frow = dpc * C.Nb;
    const long long ja = C.sa > 0 ? 0 : (long long)(Na - 1) * C.stride_a;
    const long long jb0 = ja + (long long)pb * C.stride_b + (long long)pc0 * C.stride_c;
    const int jrow = (int)(dpc * C.stride_c);
    const int jstep = (int)(C.sa > 0 ? C.stride_a : -C.stride_a);
    bool jl_ok = true;
#pragma unroll
    for (int r = 0; r < R; ++r)
        if (inmask >> r & 1) {
            const long long j1 = U.jpart + jb0 + (long long)r * jrow, j2 = j1 + (long long)(Na - 1) * jstep;
            jl_ok = jl_ok && j1 >= 0 && j1 < p.jpart_floats && j2 >= 0 && j2 < p.jpart_floats;
        }
    jl_ok = wv_ok(jl_ok, p.err);
    float *J0 = p.jpart + bin * p.jpart_floats + U.jpart + (inmask ? jb0 : 0);
    const bool stalled = ticket == p.stall_unit;
    // ART_WAVE_STATS builds: cycles in the poll loops and polls (lane 0), cycles at the step
    // barriers and in the unit (every warp), added to p.stats when the unit ends
    long long st_poll[2] = {0, 0}, st_bar = 0;
#ifdef ART_WAVE_STATS
    const long long st_t0 = clock64();
    auto stats_out = [&]() {
        if (lane == 0 && p.stats) {
            atomicAdd(reinterpret_cast<unsigned long long *>(p.stats + 0), (unsigned long long)st_bar);
            atomicAdd(reinterpret_cast<unsigned long long *>(p.stats + 1), (unsigned long long)(clock64() - st_t0));
            atomicAdd(reinterpret_cast<unsigned long long *>(p.stats + 2), (unsigned long long)st_poll[0]);
            atomicAdd(reinterpret_cast<unsigned long long *>(p.stats + 3), (unsigned long long)st_poll[1]);
        }
    };
#endif

    if (tid == 0) s_up[0] = U.up_b >= 0 ? p.units[U.up_b].eb : -1;
    if (tid == 1) s_up[1] = U.up_c >= 0 ? p.units[U.up_c].ec : -1;
    // box-edge inputs carry the boundary intensity in both parities
    if (U.up_b < 0)
        for (int e = tid; e < WC * DMAX * XBW; e += NT) {
            XB[e] = i_bc;
            XB[Sh::XB_PAR + e] = i_bc;
        }
    if (U.up_c < 0)
        for (int e = tid; e < WB * DMAX * 8; e += NT) {
            XC[e] = i_bc;
            XC[Sh::XC_PAR + e] = i_bc;
        }
    // every ray enters the box with the boundary intensity
    for (int d = 0; d < nd; ++d)
#pragma unroll
        for (int r = 0; r < R; ++r) RS[(d * NT + tid) * R + r] = i_bc;

    // progress of the upstream warps last seen by this warp (uniform), and the
    // flag values lane 0 read in the previous step (used before polling again)
    int seen_b = 0, seen_c = 0, pref_b = 0, pref_c = 0;
    const int *up_flag_b = U.up_b >= 0 ? flags + (long long)U.up_b * (WB + WC) + wc : nullptr;
    const int *up_flag_c = U.up_c >= 0 ? flags + (long long)U.up_c * (WB + WC) + WC + wb : nullptr;

    // Stage what step t + 1 reads: the table of slab t + 1, this lane's fields
    // of its next slab, and (warps on the CTA's upstream edges) the upstream
    // CTA's edge intensities, into the parity that step t + 1 reads (t & 1).
    // Returns 0 if a wait ran out.
    auto stage = [&](int t) -> int {
        const int s1 = t + 1, rp = t & 1;
        if (s1 < Na) {
            const long long src = U.tab + (long long)s1 * wv_block(nd);
            for (int q = tid; q < wv_block(nd); q += NT)
                if (wv_ok(src + q < p.rtab_len, p.err)) wv_cp16(tab + (s1 & (RT - 1)) * Sh::TABS + q, p.rtab + src + q);
        }
        const int mn = s1 - wb - wc;
        if (mn >= 0 && mn < Na) {
            const long long fa = f0 + (long long)(C.sa > 0 ? mn : Na - 1 - mn) * fslab;
            float2 *dst = FS + ((s1 & 1) * NT + tid) * R;   // read at step s1
#pragma unroll
            for (int r = 0; r < R; ++r)
                if (inmask >> r & 1) wv_cp8(dst + r, Fb + fa + (long long)r * frow);
        }
        int ok = 1;
        if (wb == 0 && U.up_b >= 0) {
            const int s = s1 - wc;
            if (s >= 0 && s < Na) {
                if (s + 1 > seen_b) {
                    int v = 0;
                    if (lane == 0) v = wv_wait(up_flag_b, s + 1, pref_b, p, st_poll);
                    v = __shfl_sync(0xffffffffu, v, 0);
                    if (v < 0) ok = 0;
                    else seen_b = v;
                }
                // read ahead: the value is used by the next step that needs more than seen_b
                if (lane == 0 && seen_b < Na) pref_b = wv_ld_relaxed(up_flag_b);
                if (ok) {
                    const long long eb_up = s_up[0];
                    for (int dd = lane; dd < nd; dd += 32) {
                        const long long o = eb_up + (((long long)s * WC + wc) * DMAX + dd) * XBW;
                        if (wv_ok(eb_up >= 0 && o + XBW <= p.edge_floats, p.err)) {
                            float *dst = XB + rp * Sh::XB_PAR + (wc * DMAX + dd) * XBW;
#pragma unroll
                            for (int q = 0; q < XBW; q += 4) wv_cp16(dst + q, edge + o + q);
                        }
                    }
                }
            }
        }
        if (wc == 0 && U.up_c >= 0) {
            const int s = s1 - wb;
            if (s >= 0 && s < Na) {
                int okc = 1;
                if (s + 1 > seen_c) {
                    int v = 0;
                    if (lane == 0) v = wv_wait(up_flag_c, s + 1, pref_c, p, st_poll);
                    v = __shfl_sync(0xffffffffu, v, 0);
                    if (v < 0) okc = 0;
                    else seen_c = v;
                }
                if (lane == 0 && seen_c < Na) pref_c = wv_ld_relaxed(up_flag_c);
                if (okc) {
                    const long long ec_up = s_up[1];
                    for (int dd = lane; dd < nd; dd += 32) {
                        const long long o = ec_up + (((long long)s * WB + wb) * DMAX + dd) * 8;
                        if (wv_ok(ec_up >= 0 && o + 8 <= p.edge_floats, p.err)) {
                            float *dst = XC + rp * Sh::XC_PAR + (wb * DMAX + dd) * 8;
                            wv_cp16(dst, edge + o);
                            wv_cp16(dst + 4, edge + o + 4);
                        }
                    }
                }
                ok &= okc;
            }
        }
        return ok;
    };

    __syncthreads();   // s_up, ray states
    // A wait that ran out ends the unit: the decision is taken by the barrier
    // itself (__syncthreads_or), so every thread leaves the loop at the same step.
    int bad = stage(-1) ? 0 : 1;
    wv_cp_wait();
    int abort_ = __syncthreads_or(bad);

    const int T = Na + WB + WC - 2;
    const bool b_out = wb == WB - 1, c_out = wc == WC - 1;
    const int fl_b = u * (WB + WC) + wc, fl_c = u * (WB + WC) + WC + wb;
    const unsigned xb0 = wv_smem(XB), xc0 = wv_smem(XC);
    const unsigned rs0 = wv_smem(RS) + 4 * R * tid, tab0 = wv_smem(tab);
    for (int t = 0; t < T && !abort_; ++t) {
        const int m = t - wb - wc;
        // progress of the slabs written to global memory in earlier steps
        if (lane == 0 && !stalled && m - 1 >= 0 && m - 1 < Na && (m & (C.pub - 1)) == 0) {
            if (b_out) wv_st_release(flags + fl_b, m);
            if (c_out) wv_st_release(flags + fl_c, m);
        }
        if (!stage(t)) bad = 1;
        if (m >= 0 && m < Na) {
            const int par = t & 1;
            float2 kap[NP], src[NP];
            float kmax = 0.0f, kmin = __int_as_float(0x7f800000);
#pragma unroll
            for (int i = 0; i < NP; ++i) {
                const float4 f = reinterpret_cast<const float4 *>(FS + (par * NT + tid) * R)[i];
                const bool i0 = inmask >> (2 * i) & 1, i1 = inmask >> (2 * i + 1) & 1;
                kap[i] = make_float2(i0 ? f.x : 0.0f, i1 ? f.z : 0.0f);
                src[i] = make_float2(i0 ? f.y : 0.0f, i1 ? f.w : 0.0f);
                kmax = fmaxf(kmax, fmaxf(kap[i].x, kap[i].y));
                kmin = fminf(kmin, fminf(kap[i].x, kap[i].y));
            }
            // the mode of the warp, by vote on its cells' largest and smallest kappa
            const bool all_thin2 = THIN5 && __all_sync(0xffffffffu, kmax < KAP_THIN2);
            WvXch x;
            x.bo = xb0 + 4 * (par * Sh::XB_PAR + ((wb + 1) * WC + wc) * DMAX * XBW + R * cl);
            x.bi = xb0 + 4 * ((par ^ 1) * Sh::XB_PAR + (wb * WC + wc) * DMAX * XBW + R * cl);
            x.co = xc0 + 4 * (par * Sh::XC_PAR + ((wc + 1) * WB + wb) * DMAX * 8 + bl);
            x.ci = xc0 + 4 * ((par ^ 1) * Sh::XC_PAR + (wc * WB + wb) * DMAX * 8 + bl);
            x.b0 = bl == 0;
            x.b7 = bl == 7;
            x.c0 = cl == 0;
            x.c3 = cl == 3;
            x.nslot = DMAX;
            x.err = p.err;
            const unsigned tb = tab0 + 16 * (m & (RT - 1)) * Sh::TABS;
            const bool all_thin = __all_sync(0xffffffffu, kmax < KAP_THIN);
            const bool all_thick = __all_sync(0xffffffffu, kmin >= KAP_THICK);
            const bool all_thin5 = THIN5 && __all_sync(0xffffffffu, kmax < KAP_THIN5);
            WvRows<NP> js;
            // (code size decides which paths take two entries at a time: with the
            // degree-2 path's loop doubled and the others single, the modes of a mixed
            // bin still fit the instruction cache)
            if (THIN5 && all_thin2) {   // (the degree-2 and degree-5 paths: shapes with >= 96 registers)
                WvThin<2> c[NP];
#pragma unroll
                for (int i = 0; i < NP; ++i) c[i] = wv_thin<2>(kap[i], src[i], p.field_form);
                js = wv_dirs<MODE_THIN, NT, NP, TWO>(c, rs0, tb, nd, x);
            } else if (all_thin) {
                WvThin<3> c[NP];
#pragma unroll
                for (int i = 0; i < NP; ++i) c[i] = wv_thin<3>(kap[i], src[i], p.field_form);
                js = wv_dirs<MODE_THIN, NT, NP, false>(c, rs0, tb, nd, x);
            } else if (THIN5 && all_thin5) {
                WvThin<5> c[NP];
#pragma unroll
                for (int i = 0; i < NP; ++i) c[i] = wv_thin<5>(kap[i], src[i], p.field_form);
                js = wv_dirs<MODE_THIN, NT, NP, false>(c, rs0, tb, nd, x);
            } else if (THIN5 && !all_thick) {   // (the coefficient form needs the registers of THIN5 shapes)
                constexpr int KM = NP == 2 ? 4 : 5;   // the mixed path's series degree
                WvMixed<KM> c[NP];
#pragma unroll
                for (int i = 0; i < NP; ++i) c[i] = wv_mixed<KM>(kap[i], src[i], p.field_form);
                js = wv_dirs<MODE_MIXED, NT, NP, false>(c, rs0, tb, nd, x);
            } else {
                WvCell2 c[NP];
#pragma unroll
                for (int i = 0; i < NP; ++i) {
                    c[i].kap = kap[i];
                    c[i].nkap = make_float2(-kap[i].x, -kap[i].y);
                    c[i].rk = make_float2(kap[i].x > 0.0f ? wv_rcp(kap[i].x) : 0.0f,
                                          kap[i].y > 0.0f ? wv_rcp(kap[i].y) : 0.0f);
                    c[i].E = p.field_form ? src[i] : __fmul2_rn(kap[i], src[i]);
                    c[i].S = p.field_form ? __fmul2_rn(src[i], c[i].rk) : src[i];
                    c[i].k2 = __fmul2_rn(kap[i], f2s(-1.4426950408889634f));
                }
                if (all_thick) {
                    js = wv_dirs<MODE_THICK, NT, NP, false>(c, rs0, tb, nd, x);
#pragma unroll
                    for (int i = 0; i < NP; ++i) js.p[i] = __fmul2_rn(js.p[i], c[i].rk);
                } else {
                    js = wv_dirs<MODE_MIXED, NT, NP, false>(c, rs0, tb, nd, x);
                }
            }
            if (jl_ok) {
                float *Jm = J0 + (long long)m * jstep;
#pragma unroll
                for (int i = 0; i < NP; ++i) {
                    if (inmask >> (2 * i) & 1) Jm[(2 * i) * jrow] = js.p[i].x;
                    if (inmask >> (2 * i + 1) & 1) Jm[(2 * i + 1) * jrow] = js.p[i].y;
                }
            }
            // edge intensities of this slab to the downstream CTAs
            if ((b_out && U.eb >= 0) || (c_out && U.ec >= 0)) {
                __syncwarp();
                if (b_out && U.eb >= 0)
                    for (int dd = lane; dd < nd; dd += 32) {
                        const float *srcs = XB + par * Sh::XB_PAR + ((wb + 1) * WC + wc) * DMAX * XBW + dd * XBW;
                        const long long o = U.eb + (((long long)m * WC + wc) * DMAX + dd) * XBW;
                        if (wv_ok(o + XBW <= p.edge_floats, p.err))
#pragma unroll
                            for (int q = 0; q < XBW; q += 4)
                                *reinterpret_cast<float4 *>(edge + o + q) =
                                    *reinterpret_cast<const float4 *>(srcs + q);
                    }
                if (c_out && U.ec >= 0)
                    for (int dd = lane; dd < nd; dd += 32) {
                        const float *srcs = XC + par * Sh::XC_PAR + ((wc + 1) * WB + wb) * DMAX * 8 + dd * 8;
                        const long long o = U.ec + (((long long)m * WB + wb) * DMAX + dd) * 8;
                        if (wv_ok(o + 8 <= p.edge_floats, p.err)) {
                            *reinterpret_cast<float4 *>(edge + o) = *reinterpret_cast<const float4 *>(srcs);
                            *reinterpret_cast<float4 *>(edge + o + 4) = *reinterpret_cast<const float4 *>(srcs + 4);
                        }
                    }
            }
        }
        wv_cp_wait();
#ifdef ART_WAVE_STATS
        const long long tb0 = clock64();
#endif
        abort_ = __syncthreads_or(bad);
#ifdef ART_WAVE_STATS
        st_bar += clock64() - tb0;
#endif
    }
#ifdef ART_WAVE_STATS
    stats_out();
#endif
    (void)st_bar;
    if (abort_) {
        if (tid == 0) atomicOr(p.err, 1);
        return;
    }
    if (lane == 0 && !stalled) {
        if (b_out) wv_st_release(flags + fl_b, Na);
        if (c_out) wv_st_release(flags + fl_c, Na);
    }
}

}  // namespace art
