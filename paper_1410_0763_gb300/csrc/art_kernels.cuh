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
//    one column per slab).
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
// code bits: 0-1 nseg-1, 2 c-plane crossed first, 3 b-shift, 4 c-shift.
template <typename real> struct SegEntry {
    real ds1, ds2, ds3;
    int code;
};

struct ClassDev {
    int a, sa, sb, sc;
    int Na, Nb, Nc;
    int dir_begin, dir_end;   // into the class-sorted direction table
    int part0;                // first J partial of the class
};

struct DirDev {
    long long seg_off;        // first SegEntry of this direction
    long long plane_off;      // first element of its plane (canonical [c][b])
    double na;                // |n_a|
};

struct WorkItem {
    int cls, pb, pc, group;   // class, tile origin (canonical b, c), direction group
};

template <typename real> struct SweepArgs {
    const typename Vec2<real>::type *field[3];   // (kappa, src) in axis-a layout, one bin
    const real *plane_in;
    real *plane_out;
    typename Vec2<real>::type *jpart;            // [n_part][ncell] (sum, compensation)
    const SegEntry<real> *segs;
    const DirDev *dirs;
    const ClassDev *classes;
    const WorkItem *work;
    long long ncell;
    int split;
    int kblock;
    int field_form;
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

// phi(x) = (1 - e^-x)/x, phi(0) = 1 (the path-averaged attenuation of a
// segment, Sec. 2.2).  Below x = 0.5 the Maclaurin series
// sum_n (-x)^n/(n+1)! to n = 7 (truncation < 1.5e-8 relative); above, the
// hardware base-2 exponential (relative error ~2^-22) where 1 - e^-x loses
// at most ~2 bits.
__device__ __forceinline__ float phi_of(float x)
{
    float p = fmaf(x, -1.0f / 40320.0f, 1.0f / 5040.0f);
    p = fmaf(x, p, -1.0f / 720.0f);
    p = fmaf(x, p, 1.0f / 120.0f);
    p = fmaf(x, p, -1.0f / 24.0f);
    p = fmaf(x, p, 1.0f / 6.0f);
    p = fmaf(x, p, -0.5f);
    p = fmaf(x, p, 1.0f);
    const float e = ex2_approx(-1.4426950408889634f * x);
    const float q = __fdividef(1.0f - e, x);
    return x < 0.5f ? p : q;
}

__device__ __forceinline__ double phi_of(double x) { return x > 0.0 ? -expm1(-x) / x : 1.0; }

// One segment of Eq. (rt): deposit ds * I_in * phi(kappa ds) (the path-
// averaged incoming intensity times the segment length) into A, then advance
// I = S + (I - S) e^-dtau (field_form 0) or I = I e^-dtau + eps ds phi
// (field_form 1, S = eps/kappa).
template <typename real>
__device__ __forceinline__ void seg_step(real &I, real &A, real kap, real src, real ds, int form)
{
    const real x = kap * ds;
    const real ph = phi_of(x);
    const real dsph = ds * ph;
    A = fma(I, dsph, A);
    const real xph = x * ph;
    if (form == 0)
        I = fma(src - I, xph, I);
    else
        I = fma(-I, xph, fma(src, dsph, I));
}

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
// Slab-block sweep kernel.  Grid: one CTA per work item (class, tile, group).
// ---------------------------------------------------------------------------
template <typename real, int TB, int TC, int BLK, int NT>
__global__ void __launch_bounds__(NT) sweep_block_kernel(const SweepArgs<real> p)
{
    using v2 = typename Vec2<real>::type;
    constexpr int WB = TB + BLK, WC = TC + BLK, NS = WB * WC;
    static_assert((TB * TC) % NT == 0, "owned columns must split evenly over threads");
    constexpr int OPT = (TB * TC) / NT;
    constexpr int MAXH = BLK * (TB + BLK) + TC * BLK;
    constexpr int HPT = (MAXH + NT - 1) / NT;

    extern __shared__ __align__(16) unsigned char smem_raw[];
    v2 *ks = reinterpret_cast<v2 *>(smem_raw);                 // [BLK][NS] (kappa, src)
    real *xbuf = reinterpret_cast<real *>(ks + BLK * NS);      // [2][NS] exchange

    const WorkItem w = p.work[blockIdx.x];
    const ClassDev C = p.classes[w.cls];
    const int m0 = p.kblock * BLK;
    if (m0 >= C.Na) return;
    const int Bp = min(BLK, C.Na - m0);
    const int Rb = w.pb - BLK, Rc = w.pc - BLK;   // origin of the smem region
    const v2 *__restrict__ F = p.field[C.a];
    const int tid = threadIdx.x;

    // Stage kappa and src of the region (tile + BLK upstream columns) for the
    // BLK slabs; cells outside the box read as vacuum (0, 0).
    for (int e = tid; e < BLK * NS; e += NT) {
        const int i = e / NS, r = e - i * NS;
        const int gb = Rb + r % WB, gc = Rc + r / WB;
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

    int o_gb[OPT], o_gc[OPT], o_r[OPT];
    bool o_ok[OPT];
#pragma unroll
    for (int s = 0; s < OPT; ++s) {
        const int o = tid + s * NT;
        o_gb[s] = w.pb + o % TB;
        o_gc[s] = w.pc + o / TB;
        o_r[s] = (o / TB + BLK) * WB + (o % TB + BLK);
        o_ok[s] = o_gb[s] < C.Nb && o_gc[s] < C.Nc;
    }
    real js[OPT][BLK], jc[OPT][BLK];
#pragma unroll
    for (int s = 0; s < OPT; ++s)
#pragma unroll
        for (int i = 0; i < BLK; ++i) js[s][i] = jc[s][i] = real(0);
    __syncthreads();

    const int nd = C.dir_end - C.dir_begin;
    const int d0 = C.dir_begin + (int)((long long)nd * w.group / p.split);
    const int d1 = C.dir_begin + (int)((long long)nd * (w.group + 1) / p.split);
    const int form = p.field_form;
    int xs = 0;

    // Intensity fetched across a column boundary: vacuum outside the box,
    // harmless garbage outside the smem region (only cone cells that never
    // feed the owned tile read there).
    auto fetch = [&](const real *X, int gb, int gc) -> real {
        if (gb < 0 || gc < 0) return real(0);
        const int rb = gb - Rb, rc = gc - Rc;
        if (rb < 0 || rc < 0) return real(0);
        return X[rc * WB + rb];
    };

    for (int d = d0; d < d1; ++d) {
        const DirDev D = p.dirs[d];
        const SegEntry<real> *tab = p.segs + D.seg_off + m0;
        int D0b = 0, D0c = 0;
        for (int i = 0; i < Bp; ++i) {
            const int code = tab[i].code;
            D0b += (code >> 3) & 1;
            D0c += (code >> 4) & 1;
        }
        // upstream cone of this direction: top strip D0c rows of TB + D0b
        // columns, then TC rows of D0b columns
        const int hw = TB + D0b;
        const int n1 = D0c * hw, nh = n1 + TC * D0b;
        int h_gb[HPT], h_gc[HPT], h_r[HPT];
        bool h_ok[HPT];
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
            h_ok[s] = (h < nh) && gb >= 0 && gc >= 0 && gb < C.Nb && gc < C.Nc;
            h_gb[s] = gb;
            h_gc[s] = gc;
            h_r[s] = (gc - Rc) * WB + (gb - Rb);
        }
        const real *pin = p.plane_in + D.plane_off;
        real oI[OPT], hI[HPT];
#pragma unroll
        for (int s = 0; s < OPT; ++s)
            oI[s] = (p.kblock > 0 && o_ok[s]) ? pin[(long long)o_gc[s] * C.Nb + o_gb[s]] : real(0);
#pragma unroll
        for (int s = 0; s < HPT; ++s)
            hI[s] = (p.kblock > 0 && h_ok[s]) ? pin[(long long)h_gc[s] * C.Nb + h_gb[s]] : real(0);
        const real na = real(D.na);
        int Db = D0b, Dc = D0c;

#pragma unroll
        for (int i = 0; i < BLK; ++i) {
            if (i < Bp) {
                const SegEntry<real> g = tab[i];
                const int nseg = (g.code & 3) + 1;
                const int cfirst = (g.code >> 2) & 1;
                const int shb = (g.code >> 3) & 1, shc = (g.code >> 4) & 1;
                const v2 *ksi = ks + i * NS;
                bool h_act[HPT];
                real hk[HPT], hs[HPT], ok[OPT], os[OPT], oA[OPT];
#pragma unroll
                for (int s = 0; s < HPT; ++s) {
                    h_act[s] = h_ok[s] && h_gb[s] >= w.pb - Db && h_gc[s] >= w.pc - Dc;
                    hk[s] = hs[s] = real(0);
                    if (h_act[s]) {
                        const v2 v = ksi[h_r[s]];
                        hk[s] = v.x;
                        hs[s] = v.y;
                    }
                }
#pragma unroll
                for (int s = 0; s < OPT; ++s) {
                    const v2 v = ksi[o_r[s]];
                    ok[s] = v.x;
                    os[s] = v.y;
                    oA[s] = real(0);
                    seg_step(oI[s], oA[s], ok[s], os[s], g.ds1, form);
                }
#pragma unroll
                for (int s = 0; s < HPT; ++s) {
                    real dummy = real(0);
                    if (h_act[s]) seg_step(hI[s], dummy, hk[s], hs[s], g.ds1, form);
                }
                if (nseg >= 2) {
                    int ob, oc;
                    if (nseg == 2) {
                        ob = shb;
                        oc = shc;
                    } else {
                        ob = cfirst ? 0 : 1;
                        oc = cfirst;
                    }
                    for (int step = 2; step <= nseg; ++step) {
                        const real dsk = step == 2 ? g.ds2 : g.ds3;
                        real *X = xbuf + xs * NS;
#pragma unroll
                        for (int s = 0; s < OPT; ++s) X[o_r[s]] = oI[s];
#pragma unroll
                        for (int s = 0; s < HPT; ++s)
                            if (h_act[s]) X[h_r[s]] = hI[s];
                        __syncthreads();
#pragma unroll
                        for (int s = 0; s < OPT; ++s) {
                            real Iin = fetch(X, o_gb[s] - ob, o_gc[s] - oc);
                            seg_step(Iin, oA[s], ok[s], os[s], dsk, form);
                            oI[s] = Iin;
                        }
#pragma unroll
                        for (int s = 0; s < HPT; ++s) {
                            if (h_act[s]) {
                                real Iin = fetch(X, h_gb[s] - ob, h_gc[s] - oc);
                                real dummy = real(0);
                                seg_step(Iin, dummy, hk[s], hs[s], dsk, form);
                                hI[s] = Iin;
                            }
                        }
                        xs ^= 1;
                        // the third segment comes from the other neighbour
                        ob = 1 - ob;
                        oc = 1 - oc;
                    }
                }
#pragma unroll
                for (int s = 0; s < OPT; ++s)
                    if (o_ok[s]) kahan_add(js[s][i], jc[s][i], oA[s] * na);
                Db -= shb;
                Dc -= shc;
            }
        }
        real *pout = p.plane_out + D.plane_off;
#pragma unroll
        for (int s = 0; s < OPT; ++s)
            if (o_ok[s]) pout[(long long)o_gc[s] * C.Nb + o_gb[s]] = oI[s];
    }

    v2 *J = p.jpart + (long long)(C.part0 + w.group) * p.ncell;
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
                v2 v;
                v.x = js[s][i];
                v.y = jc[s][i];
                J[((long long)pa * C.Nc + pc) * C.Nb + pb] = v;
            }
        }
    }
}

// ---------------------------------------------------------------------------
// Sum the class partials (fixed order, Kahan) into J^in, J and Gamma.
// ---------------------------------------------------------------------------
template <typename real> struct ReduceArgs {
    const typename Vec2<real>::type *jpart;
    const typename Vec2<real>::type *field_nat;   // (kappa, src) in [z][y][x]
    const int *part_axis;
    int n_part;
    int nx, ny, nz;
    long long ncell;
    real inv_nd;
    real gamma_coef;     // 4 pi G_b
    int gamma_accum;     // add to gamma instead of overwriting
    int field_form;
    real *Jin, *J, *gamma;
};

template <typename real> __global__ void reduce_kernel(const ReduceArgs<real> p)
{
    using v2 = typename Vec2<real>::type;
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= p.ncell) return;
    const int x = (int)(i % p.nx);
    const int y = (int)((i / p.nx) % p.ny);
    const int z = (int)(i / ((long long)p.nx * p.ny));
    const long long idx[3] = {((long long)x * p.nz + z) * p.ny + y, ((long long)y * p.nz + z) * p.nx + x, i};
    real s = real(0), c = real(0);
    for (int k = 0; k < p.n_part; ++k) {
        const v2 v = p.jpart[(long long)k * p.ncell + idx[p.part_axis[k]]];
        kahan_add(s, c, v.x);
        kahan_add(s, c, -v.y);
    }
    const real jin = (s - c) * p.inv_nd;
    if (p.Jin) p.Jin[i] = jin;
    if (p.J) {
        const v2 f = p.field_nat[i];
        real S = f.y;
        if (p.field_form == 1) S = f.x > real(0) ? f.y / f.x : real(0);
        p.J[i] = jin + S;
    }
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
