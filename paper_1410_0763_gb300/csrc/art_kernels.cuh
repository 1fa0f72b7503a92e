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

template <typename real> struct alignas(4 * sizeof(real)) Quad {
    real x, y, z, w;
};

template <typename real> struct SweepArgs {
    const typename Vec2<real>::type *field0, *field1, *field2;   // (kappa, src), axis-a layouts, one bin
    const real *plane_in;
    real *plane_out;
    real *jpart;                 // [n_part][ncell] J partials, natural [z][y][x] layout
    const SegEntry<real> *segs;
    const DirDev *dirs;
    const ClassDev *classes;
    const WorkItem *work;
    long long ncell;
    int nx, ny, nz;
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

// Coefficients of one segment of optical depth x = kappa ds:
//   dsph = ds phi(x), xph = x phi(x) = 1 - e^-x,  phi(x) = (1 - e^-x)/x, phi(0) = 1
// (phi: the path-averaged attenuation of the segment, Sec. 2.2).  FP32: below
// x = 1/4 the Maclaurin series sum_n (-x)^n/(n+1)! to n = 5 (truncation
// < 6e-8 relative); above, 1 - 2^(-x log2 e) from the hardware base-2
// exponential (relative error ~2^-22, so < 1e-6 on 1 - e^-x there) and the
// per-cell reciprocal 1/kappa (no per-segment division).  k2 = -kappa log2 e
// and rk = 1/kappa are precomputed per cell.
__device__ __forceinline__ void seg_coef(float kap, float k2, float rk, float ds, float &dsph, float &xph)
{
    const float x = kap * ds;
    float q = fmaf(x, -1.0f / 720.0f, 1.0f / 120.0f);
    q = fmaf(x, q, -1.0f / 24.0f);
    q = fmaf(x, q, 1.0f / 6.0f);
    q = fmaf(x, q, -0.5f);
    q = fmaf(x, q, 1.0f);
    const float om = 1.0f - ex2_approx(k2 * ds);
    const bool small = x < 0.25f;
    dsph = small ? ds * q : om * rk;
    xph = small ? x * q : om;
}

__device__ __forceinline__ void seg_coef(double kap, double, double, double ds, double &dsph, double &xph)
{
    const double x = kap * ds;
    const double ph = x > 0.0 ? -expm1(-x) / x : 1.0;
    dsph = ds * ph;
    xph = x * ph;
}

// One segment of Eq. (rt): deposit ds * I_in * phi into A (the path-averaged
// incoming intensity times the segment length), then advance
// I = S + (I - S) e^-x (form 0) or I = I e^-x + eps ds phi (form 1, S = eps/kappa).
template <typename real>
__device__ __forceinline__ void seg_apply(real &I, real &A, real src, real dsph, real xph, int form)
{
    A = fma(I, dsph, A);
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
// The CTA takes the directions of its group K at a time: for each slab the K
// directions share the cell loads and the exchange barriers, and each thread
// carries K independent intensity chains per column.  Shared memory: (kappa,
// src) of the region (tile + BLK + 1 upstream columns) for the BLK slabs, two
// exchange buffers of K planes over the region, and the segment tables of a
// chunk of directions.  Region columns upstream of the box are never written
// and stay 0: rays there carry the vacuum boundary intensity.
// ---------------------------------------------------------------------------
template <typename real> struct DirSm {
    long long plane_off;
    real na;
    int d0b, d0c;    // column shifts over the slab block
};

template <int TB, int TC, int BLK, int NT, int K> struct SweepShape {
    static constexpr int HB = BLK + 1;
    static constexpr int WB = TB + HB, WC = TC + HB, NS = WB * WC;
    static constexpr int OPT = (TB * TC) / NT;
    static constexpr int MAXH = BLK * (TB + BLK) + TC * BLK;
    static constexpr int HPT = (MAXH + NT - 1) / NT;
    static constexpr int DCH = 8 * K;   // directions staged per chunk
    template <typename real> __host__ __device__ static constexpr size_t off_x()
    {
        return size_t(BLK) * NS * sizeof(typename Vec2<real>::type);
    }
    template <typename real> __host__ __device__ static constexpr size_t off_t()
    {
        return (off_x<real>() + 2 * size_t(K) * NS * sizeof(real) + 31) / 32 * 32;
    }
    template <typename real> __host__ __device__ static constexpr size_t off_d()
    {
        return off_t<real>() + size_t(DCH) * BLK * sizeof(SegEntry<real>);
    }
    template <typename real> __host__ __device__ static constexpr size_t bytes()
    {
        return off_d<real>() + size_t(DCH) * sizeof(DirSm<real>);
    }
};

__device__ __forceinline__ float rcp_or_zero(float k)
{
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(k));
    return k > 0.0f ? r : 0.0f;
}
__device__ __forceinline__ double rcp_or_zero(double k) { return k > 0.0 ? 1.0 / k : 0.0; }

template <typename real, int TB, int TC, int BLK, int NT, int K, int MINB>
__global__ void __launch_bounds__(NT, MINB) sweep_block_kernel(const SweepArgs<real> p)
{
    using v2 = typename Vec2<real>::type;
    using Sh = SweepShape<TB, TC, BLK, NT, K>;
    constexpr int HB = Sh::HB, WB = Sh::WB, WC = Sh::WC, NS = Sh::NS, OPT = Sh::OPT, HPT = Sh::HPT,
                  DCH = Sh::DCH;
    static_assert((TB * TC) % NT == 0, "owned columns must split evenly over threads");

    extern __shared__ __align__(32) unsigned char smem_raw[];
    v2 *ks = reinterpret_cast<v2 *>(smem_raw);
    real *xbuf = reinterpret_cast<real *>(smem_raw + Sh::template off_x<real>());   // [2][K][NS]
    SegEntry<real> *tsm = reinterpret_cast<SegEntry<real> *>(smem_raw + Sh::template off_t<real>());
    DirSm<real> *dsm = reinterpret_cast<DirSm<real> *>(smem_raw + Sh::template off_d<real>());

    const WorkItem w = p.work[blockIdx.x];
    const ClassDev C = p.classes[w.cls];
    const int m0 = p.kblock * BLK;
    if (m0 >= C.Na) return;
    const int Bp = min(BLK, C.Na - m0);
    const int Rb = w.pb - HB, Rc = w.pc - HB;   // origin of the smem region
    const v2 *__restrict__ F = C.a == 0 ? p.field0 : (C.a == 1 ? p.field1 : p.field2);
    const int tid = threadIdx.x;
    const int form = p.field_form;

    // Stage the region's (kappa, src) for the BLK slabs row by row (vacuum
    // outside the box), and clear the exchange buffers.
    {
        const int nrows = BLK * WC;
        for (int e = tid; e < nrows * WB; e += NT) {
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
    }
    for (int e = tid; e < 2 * K * NS; e += NT) xbuf[e] = real(0);

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

    for (int c0 = d0; c0 < d1; c0 += DCH) {
        const int cnt = min(DCH, d1 - c0);
        __syncthreads();   // previous chunk's tables are no longer read
        for (int e = tid; e < cnt * BLK; e += NT) {
            const int dl = e / BLK, i = e - dl * BLK;
            if (i < Bp) tsm[e] = p.segs[p.dirs[c0 + dl].seg_off + m0 + i];
        }
        for (int dl = tid; dl < cnt; dl += NT) {
            const DirDev D = p.dirs[c0 + dl];
            int sb = 0, sc = 0;
            for (int i = 0; i < Bp; ++i) {
                const int code = p.segs[D.seg_off + m0 + i].code;
                sb += (code >> 3) & 1;
                sc += (code >> 4) & 1;
            }
            DirSm<real> q;
            q.plane_off = D.plane_off;
            q.na = real(D.na);
            q.d0b = sb;
            q.d0c = sc;
            dsm[dl] = q;
        }
        __syncthreads();

        for (int g0 = 0; g0 < cnt; g0 += K) {
            const int kk = min(K, cnt - g0);
            // union cone of the group
            int D0b = 0, D0c = 0;
            int Dbk[K], Dck[K];   // remaining cone of each direction
            long long poff[K];
            real na[K];
#pragma unroll
            for (int k = 0; k < K; ++k) {
                const DirSm<real> D = dsm[g0 + (k < kk ? k : 0)];
                poff[k] = D.plane_off;
                na[k] = k < kk ? D.na : real(0);
                Dbk[k] = k < kk ? D.d0b : 0;
                Dck[k] = k < kk ? D.d0c : 0;
                D0b = max(D0b, Dbk[k]);
                D0c = max(D0c, Dck[k]);
            }
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
                h_ok[s] = h < nh && gb >= 0 && gc >= 0 && gb < C.Nb && gc < C.Nc;
                h_gb[s] = gb;
                h_gc[s] = gc;
                h_r[s] = h_ok[s] ? (gc - Rc) * WB + (gb - Rb) : 0;
            }
            real oI[OPT][K], hI[HPT][K];
#pragma unroll
            for (int k = 0; k < K; ++k) {
                const real *pin = p.plane_in + poff[k];
#pragma unroll
                for (int s = 0; s < OPT; ++s)
                    oI[s][k] = (!first && o_ok[s] && k < kk) ? pin[(long long)o_gc[s] * C.Nb + o_gb[s]] : real(0);
#pragma unroll
                for (int s = 0; s < HPT; ++s)
                    hI[s][k] = (!first && h_ok[s] && k < kk) ? pin[(long long)h_gc[s] * C.Nb + h_gb[s]] : real(0);
            }

#pragma unroll
            for (int i = 0; i < BLK; ++i) {
                if (i < Bp) {
                    SegEntry<real> g[K];
                    int nsmax = 1, Db = 0, Dc = 0;   // union of the remaining cones
#pragma unroll
                    for (int k = 0; k < K; ++k) {
                        g[k] = tsm[(g0 + (k < kk ? k : 0)) * BLK + i];
                        if (k >= kk) g[k].code = 0;   // inactive: one segment, ignored below
                        nsmax = max(nsmax, (g[k].code & 3) + 1);
                        Db = max(Db, Dbk[k]);
                        Dc = max(Dc, Dck[k]);
                        Dbk[k] -= (g[k].code >> 3) & 1;
                        Dck[k] -= (g[k].code >> 4) & 1;
                    }
                    const v2 *ksi = ks + i * NS;
                    real ok[OPT], os[OPT], ok2[OPT], ork[OPT], oA[OPT][K];
                    real hk[HPT], hs[HPT], hk2[HPT], hrk[HPT];
                    bool h_act[HPT], hw_act[HPT];
#pragma unroll
                    for (int s = 0; s < OPT; ++s) {
                        const v2 c = ksi[o_r[s]];
                        ok[s] = c.x;
                        os[s] = c.y;
                        ok2[s] = real(-1.4426950408889634) * c.x;
                        ork[s] = rcp_or_zero(c.x);
#pragma unroll
                        for (int k = 0; k < K; ++k) {
                            real dsph, xph;
                            seg_coef(ok[s], ok2[s], ork[s], g[k].ds1, dsph, xph);
                            oA[s][k] = real(0);
                            seg_apply(oI[s][k], oA[s][k], os[s], dsph, xph, form);
                        }
                    }
#pragma unroll
                    for (int s = 0; s < HPT; ++s) {
                        hw_act[s] = ((tid & ~31) + s * NT) < nh;
                        h_act[s] = h_ok[s] && h_gb[s] >= w.pb - Db && h_gc[s] >= w.pc - Dc;
                        hk[s] = hs[s] = hk2[s] = hrk[s] = real(0);
                        if (hw_act[s] && h_act[s]) {
                            const v2 c = ksi[h_r[s]];
                            hk[s] = c.x;
                            hs[s] = c.y;
                            hk2[s] = real(-1.4426950408889634) * c.x;
                            hrk[s] = rcp_or_zero(c.x);
#pragma unroll
                            for (int k = 0; k < K; ++k) {
                                real dsph, xph, dummy = real(0);
                                seg_coef(hk[s], hk2[s], hrk[s], g[k].ds1, dsph, xph);
                                seg_apply(hI[s][k], dummy, hs[s], dsph, xph, form);
                            }
                        }
                    }
                    for (int step = 2; step <= nsmax; ++step) {
                        real *X = xbuf + xs * K * NS;
#pragma unroll
                        for (int k = 0; k < K; ++k) {
#pragma unroll
                            for (int s = 0; s < OPT; ++s) X[k * NS + o_r[s]] = oI[s][k];
#pragma unroll
                            for (int s = 0; s < HPT; ++s)
                                if (hw_act[s] && h_act[s]) X[k * NS + h_r[s]] = hI[s][k];
                        }
                        __syncthreads();
#pragma unroll
                        for (int k = 0; k < K; ++k) {
                            const int ns = (g[k].code & 3) + 1;
                            if (ns < step) continue;   // uniform: this direction is done
                            const int cf = (g[k].code >> 2) & 1;
                            int ob, oc;
                            if (ns == 2) {
                                ob = (g[k].code >> 3) & 1;
                                oc = (g[k].code >> 4) & 1;
                            } else if (step == 2) {
                                ob = 1 - cf;
                                oc = cf;
                            } else {
                                ob = cf;
                                oc = 1 - cf;
                            }
                            const int off = oc * WB + ob;
                            const real dsk = step == 2 ? g[k].ds2 : g[k].ds3;
                            const real *Xk = X + k * NS;
#pragma unroll
                            for (int s = 0; s < OPT; ++s) {
                                real dsph, xph;
                                seg_coef(ok[s], ok2[s], ork[s], dsk, dsph, xph);
                                real Iin = Xk[o_r[s] - off];
                                seg_apply(Iin, oA[s][k], os[s], dsph, xph, form);
                                oI[s][k] = Iin;
                            }
#pragma unroll
                            for (int s = 0; s < HPT; ++s) {
                                if (hw_act[s] && h_act[s]) {
                                    real dsph, xph, dummy = real(0);
                                    seg_coef(hk[s], hk2[s], hrk[s], dsk, dsph, xph);
                                    real Iin = Xk[h_r[s] - off];
                                    seg_apply(Iin, dummy, hs[s], dsph, xph, form);
                                    hI[s][k] = Iin;
                                }
                            }
                        }
                        xs ^= 1;
                    }
#pragma unroll
                    for (int s = 0; s < OPT; ++s) {
                        if (o_ok[s]) {
                            real a = real(0);
#pragma unroll
                            for (int k = 0; k < K; ++k) a = fma(oA[s][k], na[k], a);
                            kahan_add(js[s][i], jc[s][i], a);
                        }
                    }
                }
            }
#pragma unroll
            for (int k = 0; k < K; ++k) {
                if (k < kk) {
                    real *pout = p.plane_out + poff[k];
#pragma unroll
                    for (int s = 0; s < OPT; ++s)
                        if (o_ok[s]) pout[(long long)o_gc[s] * C.Nb + o_gb[s]] = oI[s][k];
                }
            }
        }
    }

    real *J = p.jpart + (long long)(C.part0 + w.group) * p.ncell;
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
                J[((long long)z * p.ny + y) * p.nx + x] = js[s][i] - jc[s][i];
            }
        }
    }
}

// ---------------------------------------------------------------------------
// Sum the class partials (fixed order, Kahan) into J^in, J and Gamma.
// ---------------------------------------------------------------------------
template <typename real> struct ReduceArgs {
    const real *jpart;                             // [n_part][ncell], natural layout
    const typename Vec2<real>::type *field_nat;    // (kappa, src) in [z][y][x]
    int n_part;
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
    real s = real(0), c = real(0);
    for (int k = 0; k < p.n_part; ++k) kahan_add(s, c, p.jpart[(long long)k * p.ncell + i]);
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
