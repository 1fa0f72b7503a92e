// art_ion.cu -- point sources (long characteristics with the photon-conserving
// rate of App. A), the FP64 hydrogen ionization balance (App. B, equilibrium
// limit), the RT / balance fixed-point iteration (App. D) and the
// time-dependent mode with and without the energy equation (App. B-D) of
// Tanaka et al. (2014), on top of the diffuse-radiation sweep.
#include <cuda_runtime.h>

#include <chrono>
#include <cmath>
#include <cstring>
#include <string>
#include <type_traits>
#include <vector>

#include "art.h"
#include "art_ctx.hpp"
#include "art_net.h"
#include "art_net_internal.hpp"

namespace {

constexpr double kPi = 3.14159265358979323846;

#define ICK(ctx, call)                                                                               \
    do {                                                                                             \
        cudaError_t e_ = (call);                                                                     \
        if (e_ != cudaSuccess)                                                                       \
            return art_fail(ctx, e_ == cudaErrorMemoryAllocation ? ART_E_OOM : ART_E_CUDA,           \
                            std::string(#call) + ": " + cudaGetErrorString(e_));                     \
    } while (0)

// ---------------------------------------------------------------------------
// Point sources.  One thread per target cell; for each source (index order)
// the straight ray from the source to the cell centre is marched cell by
// cell, accumulating tau_b = sum kappa_b ds over the cells before the target
// cell; [r_in, r_out] is the ray's passage through the target cell (r_in = 0
// in the source's own cell).  Per bin (App. A, absorbed = in - out):
//   Ndot_abs = Q_b e^-tau (1 - e^-dtau),  dtau = kappa_b (r_out - r_in),
//   Gamma   += Ndot_abs / (n_HI 4pi/3 (r_out^3 - r_in^3) dx^3),  n_HI = kappa_b/(sigma_b dx)
// which, with r_out^3 - r_in^3 = (r_out - r_in)(r_out^2 + r_out r_in + r_in^2), is
//   Gamma   += 3 Q_b sigma_b / (4 pi dx^2) e^-tau phi(dtau) / (r_out^2 + r_out r_in + r_in^2),
// free of the cancellation of r_out^3 - r_in^3 far from the source.  The march
// and each source's rate are FP32: the source position is split into its integer cell and the fraction
// inside it, so every distance from the source to a plane or cell centre is
// an exact small integer plus a fraction (no cancellation near the source);
// the march keeps, per axis, the parametric distance to that axis' next plane
// (an O(1) number); the constant 3 Q_b sigma_b / (4 pi dx^2) is formed on
// the host in FP64, and the sources' rates are summed in FP64.
// ---------------------------------------------------------------------------
struct PtSrc {
    int si[3];       // cell containing the source
    float sf[3];     // position inside it, [0, 1)
    float coef[4];   // 3 Q_b sigma_b / (4 pi dx^2) per bin
};

struct PtArgs {
    const float *kappa;   // [bins][ncell], or one field scaled per bin (scaled != 0)
    const PtSrc *src;     // [nsrc]
    int nsrc, nbins;
    int nx, ny, nz;
    long long ncell;
    float *gamma;
    int scaled;           // kappa_b = kappa * kscale[b] (one field for all bins, one tau to march)
    float kscale[4];
    float *heat;          // photo-heating per neutral atom, sum_b Gamma_b ebin[b] (null: not computed)
    float ebin[4];        // erg above threshold per photo-ionization in bin b
};

constexpr int kMaxBins = 4;   // point-source kernels are compiled for 1-4 bins
#ifndef PT_UNROLL
#define PT_UNROLL 4                // march steps whose kappa loads are issued together
#endif

// phi(x) = (1 - e^-x)/x: its Maclaurin series to x^5 below x = 1/4, else direct
__device__ __forceinline__ float pt_phi(float x)
{
    if (x < 0.25f) {
        float q = fmaf(x, -1.0f / 720.0f, 1.0f / 120.0f);
        q = fmaf(x, q, -1.0f / 24.0f);
        q = fmaf(x, q, 1.0f / 6.0f);
        q = fmaf(x, q, -0.5f);
        return fmaf(x, q, 1.0f);
    }
    return (1.0f - __expf(-x)) / x;
}

// One march step: the kappa of the current cell and the path length in it,
// then the crossing of the nearest plane (one plane per step; a plane of
// another axis at the same place is crossed by the next step, with ds ~ 0).
template <int NK, typename IDX>
__device__ __forceinline__ void pt_step(const float *__restrict__ kappa, long long ncell, IDX &ci, float (&r)[3],
                                        const float (&dl)[3], const IDX (&dci)[3], float (&kv)[NK], float &dv)
{
    const float ds = fminf(r[0], fminf(r[1], r[2]));
#pragma unroll
    for (int b = 0; b < NK; ++b) kv[b] = __ldg(kappa + (long long)b * ncell + ci);
    dv = ds;
    r[0] -= ds;
    r[1] -= ds;
    r[2] -= ds;
    // the nearest plane's distance is now exactly 0
    if (r[0] <= 0.0f) {
        ci += dci[0];
        r[0] += dl[0];
    } else if (r[1] <= 0.0f) {
        ci += dci[1];
        r[1] += dl[1];
    } else {
        ci += dci[2];
        r[2] += dl[2];
    }
}

// Threads map to 8 x 4 x 4 bricks of cells (a warp is an 8 x 4 patch of one
// plane), so the rays of a warp have similar lengths and touch nearby cells.
template <int NB, bool SCALED, typename IDX>
__global__ void __launch_bounds__(128) point_source_kernel(const PtArgs p)
{
    const int bx = (p.nx + 7) >> 3, by = (p.ny + 3) >> 2;
    const int blk = blockIdx.x;
    const int tx = (blk % bx) * 8 + (threadIdx.x & 7);
    const int ty = ((blk / bx) % by) * 4 + ((threadIdx.x >> 3) & 3);
    const int tz = (blk / (bx * by)) * 4 + (threadIdx.x >> 5);
    if (tx >= p.nx || ty >= p.ny || tz >= p.nz) return;
    const IDX stride[3] = {(IDX)1, (IDX)p.nx, (IDX)p.nx * (IDX)p.ny};
    const IDX target = (IDX)tx + stride[1] * (IDX)ty + stride[2] * (IDX)tz;
    const int tc[3] = {tx, ty, tz};
    const int dims[3] = {p.nx, p.ny, p.nz};
    constexpr int U = PT_UNROLL;
    constexpr int NK = SCALED ? 1 : NB;   // kappa fields marched
    double g = 0.0, h = 0.0;              // the sums over sources, in index order, in FP64
    for (int a = 0; a < p.nsrc; ++a) {
        const PtSrc S = p.src[a];
        // source -> cell centre: integer part exact, plus the fractions
        float d[3];
#pragma unroll
        for (int k = 0; k < 3; ++k) d[k] = (float)(tc[k] - S.si[k]) + (0.5f - S.sf[k]);
        const float L2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
        if (L2 < 1e-12f) {
            d[0] = 1.0f;
            d[1] = d[2] = 0.0f;
        } else {
            const float il = rsqrtf(L2);
#pragma unroll
            for (int k = 0; k < 3; ++k) d[k] *= il;
        }
        // first cell: the one containing the source + 1e-6 d; the walk from it
        // to the target crosses |tc_k - cur_k| planes of each axis k, one per
        // step, and every cell on the way lies between the two
        IDX ci = 0;
        IDX dci[3];    // index step on crossing each axis' next plane
        float rn[3];   // 1/d
        float r[3];    // ray length from the current point to each axis' next plane (O(1))
        float dl[3];   // ray length between successive planes of each axis
        int n = 0;     // steps to the target cell
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            const int v = S.si[k] + (int)floorf(S.sf[k] + 1e-6f * d[k]);
            const int cur = v < 0 ? 0 : (v >= dims[k] ? dims[k] - 1 : v);
            ci += (IDX)cur * stride[k];
            n += abs(tc[k] - cur);
            const int stp = d[k] > 0.0f ? 1 : (d[k] < 0.0f ? -1 : 0);
            rn[k] = stp ? __frcp_rn(d[k]) : 0.0f;
            r[k] = stp ? ((float)(cur + (stp > 0) - S.si[k]) - S.sf[k]) * rn[k] : INFINITY;
            dl[k] = stp ? fabsf(rn[k]) : INFINITY;
            dci[k] = stp > 0 ? stride[k] : (IDX)0 - stride[k];
        }
        // March in rounds of U steps: first the U cells and path lengths (the
        // cell walk does not depend on kappa), with their kappa loads issued
        // together, then the U optical-depth updates in order.
        float tau[NK];
#pragma unroll
        for (int b = 0; b < NK; ++b) tau[b] = 0.0f;
        for (; n >= U; n -= U) {
            float kv[U][NK], dv[U];
#pragma unroll
            for (int u = 0; u < U; ++u) pt_step<NK, IDX>(p.kappa, p.ncell, ci, r, dl, dci, kv[u], dv[u]);
#pragma unroll
            for (int u = 0; u < U; ++u)
#pragma unroll
                for (int b = 0; b < NK; ++b) tau[b] = fmaf(kv[u][b], dv[u], tau[b]);
        }
        for (; n > 0; --n) {
            float kv[NK], dv;
            pt_step<NK, IDX>(p.kappa, p.ncell, ci, r, dl, dci, kv, dv);
#pragma unroll
            for (int b = 0; b < NK; ++b) tau[b] = fmaf(kv[b], dv, tau[b]);
        }
        {
            // passage through the target cell, exactly, from its faces
            float rin = 0.0f, rout = INFINITY;
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                if (d[k] == 0.0f) continue;
                const float t1 = ((float)(tc[k] - S.si[k]) - S.sf[k]) * rn[k];
                const float t2 = t1 + rn[k];
                rin = fmaxf(rin, fminf(t1, t2));
                rout = fminf(rout, fmaxf(t1, t2));
            }
            const float den = rout * rout + rout * rin + rin * rin;
            float ga = 0.0f, ha = 0.0f;
#pragma unroll
            for (int b = 0; b < NB; ++b) {
                const float kb = SCALED ? p.kappa[target] * p.kscale[b] : p.kappa[(long long)b * p.ncell + target];
                const float tb = SCALED ? tau[0] * p.kscale[b] : tau[b];
                const float rb = S.coef[b] * __expf(-tb) * pt_phi(kb * (rout - rin)) / den;
                ga += rb;
                ha = fmaf(rb, p.ebin[b], ha);
            }
            g += (double)ga;
            h += (double)ha;
        }
    }
    p.gamma[target] = (float)g;
    if (p.heat) p.heat[target] = (float)h;
}

// ---------------------------------------------------------------------------
// Plane-parallel incident flux (the Test-3 setup of Sec. 4.3: a constant
// photon flux F through one face, a point source at infinity).  One thread
// per transverse column marches along the beam; in bin b a cell absorbs
// F_b dx^2 e^-tau (1 - e^-dtau) photons per second, tau summing kappa_b over
// the cells before it and dtau = kappa_b, so per neutral atom
// (n_HI dx^3 = kappa_b dx^2 / sigma_b)
//   Gamma += F_b sigma_b e^-tau phi(dtau),  phi(x) = (1 - e^-x)/x.
// FP32; threads run along x where x is transverse, so loads coalesce.
// ---------------------------------------------------------------------------
struct PlaneArgs {
    const float *kappa;   // [bins][ncell], or one field scaled per bin (scaled != 0)
    long long ncell;
    int nx, ny, nz;
    int axis, dir;        // beam along +axis (dir 1, entering at coordinate 0) or -axis (dir -1)
    float coef[4];        // F_b sigma_b
    int scaled;
    float kscale[4];
    int accumulate;       // add to gamma (and heat) instead of overwriting it
    float *gamma;
    float *heat;          // photo-heating per neutral atom, sum_b Gamma_b ebin[b] (null: not computed)
    float ebin[4];
};

template <int NB, bool SCALED> __global__ void __launch_bounds__(128) plane_source_kernel(const PlaneArgs p)
{
    const int dims[3] = {p.nx, p.ny, p.nz};
    const long long stride[3] = {1, p.nx, (long long)p.nx * p.ny};
    const int u = p.axis == 0 ? 1 : 0, v = p.axis == 2 ? 1 : 2;   // transverse axes, u fastest
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (long long)dims[u] * dims[v]) return;
    const int pu = (int)(t % dims[u]), pv = (int)(t / dims[u]);
    const int na = dims[p.axis];
    const long long step = p.dir > 0 ? stride[p.axis] : -stride[p.axis];
    long long ci = pu * stride[u] + pv * stride[v] + (p.dir > 0 ? 0 : (long long)(na - 1) * stride[p.axis]);
    constexpr int NK = SCALED ? 1 : NB;
    float tau[NK];
#pragma unroll
    for (int b = 0; b < NK; ++b) tau[b] = 0.0f;
    for (int m = 0; m < na; ++m, ci += step) {
        float kc[NK];
#pragma unroll
        for (int b = 0; b < NK; ++b) kc[b] = __ldg(p.kappa + (long long)b * p.ncell + ci);
        float g = 0.0f, h = 0.0f;
#pragma unroll
        for (int b = 0; b < NB; ++b) {
            const float kb = SCALED ? kc[0] * p.kscale[b] : kc[b];
            const float tb = SCALED ? tau[0] * p.kscale[b] : tau[b];
            const float rb = p.coef[b] * __expf(-tb) * pt_phi(kb);
            g += rb;
            h = fmaf(rb, p.ebin[b], h);
        }
#pragma unroll
        for (int b = 0; b < NK; ++b) tau[b] += kc[b];
        p.gamma[ci] = p.accumulate ? p.gamma[ci] + g : g;
        if (p.heat) p.heat[ci] = p.accumulate ? p.heat[ci] + h : h;
    }
}

art_status launch_plane(art_ctx *ctx, const float *kappa, int nbins, int axis, int dir, const double *coef,
                        float *gamma, int accumulate, cudaStream_t st, const float *kscale = nullptr,
                        float *heat = nullptr, const double *ebin = nullptr)
{
    PlaneArgs a;
    a.heat = heat;
    for (int b = 0; b < 4; ++b) a.ebin[b] = heat && b < nbins ? (float)ebin[b] : 0.0f;
    a.kappa = kappa;
    a.ncell = ctx->ncell;
    a.nx = ctx->grid.nx;
    a.ny = ctx->grid.ny;
    a.nz = ctx->grid.nz;
    a.axis = axis;
    a.dir = dir;
    for (int b = 0; b < 4; ++b) {
        const double c = b < nbins ? coef[b] : 0.0;
        if (!(c >= 0.0) || !(c <= 3.0e38))
            return art_fail(ctx, ART_E_INVALID, "plane source: bad flux or a rate beyond FP32 range");
        a.coef[b] = (float)c;
        a.kscale[b] = kscale && b < nbins ? kscale[b] : 1.0f;
    }
    a.scaled = kscale != nullptr;
    a.accumulate = accumulate;
    a.gamma = gamma;
    const int dims[3] = {a.nx, a.ny, a.nz};
    const long long ncol = (long long)dims[axis == 0 ? 1 : 0] * dims[axis == 2 ? 1 : 2];
    const int nt = 128;
    const unsigned nb = (unsigned)((ncol + nt - 1) / nt);
    switch (nbins + (a.scaled ? 4 : 0)) {
    case 1: plane_source_kernel<1, false><<<nb, nt, 0, st>>>(a); break;
    case 2: plane_source_kernel<2, false><<<nb, nt, 0, st>>>(a); break;
    case 3: plane_source_kernel<3, false><<<nb, nt, 0, st>>>(a); break;
    case 4: plane_source_kernel<4, false><<<nb, nt, 0, st>>>(a); break;
    case 5: plane_source_kernel<1, true><<<nb, nt, 0, st>>>(a); break;
    case 6: plane_source_kernel<2, true><<<nb, nt, 0, st>>>(a); break;
    case 7: plane_source_kernel<3, true><<<nb, nt, 0, st>>>(a); break;
    case 8: plane_source_kernel<4, true><<<nb, nt, 0, st>>>(a); break;
    default: return art_fail(ctx, ART_E_INVALID, "plane source: 1 to 4 bins");
    }
    ICK(ctx, cudaGetLastError());
    return ART_OK;
}

// ---------------------------------------------------------------------------
// FP64 balance (App. B, dt -> infinity), hydrogen only.  With the local
// recombination term of Eq. (gamma_diff) at the same state,
//   alpha_B n_e n_HII = n_HI (Gamma_coll n_e + g),  g = Gamma_point + Gamma_diff,in,
// n_HI = y n_H, n_e = n_HII = x n_H, x = 1 - y:  a = alpha_B n_H, c = Gamma_coll n_H,
//   den = 2a + c + g + sqrt(4ag + (c + g)^2),  y = 2a/den,  x = (c + g + sqrt(.))/den
// (both without cancellation).  Writes y, the next sweep inputs
//   kappa = n_HI sigma0 dx,  eps' = 4 pi G eps dx = G h nu0 (alpha_A - alpha_B) n_e^2 dx / dnu
// (eps' makes the sweep return Gamma_diff,in directly), and the block maxima
// of |n_e^(i) - n_e^(i-1)| / n_e^(i) into an order-independent atomic max.
// ---------------------------------------------------------------------------
struct BalArgs {
    const double *nH;
    const float *gpt, *gdiff;   // may be null (prepare pass)
    double alphaB, gcoll;
    double kap_coef, eps_coef;  // sigma0 dx ; G h nu0 dalpha dx / dnu
    double *y;
    float *kap, *eps;
    unsigned long long *resid;
    long long ncell;
    int solve;                  // 0: only derive kappa, eps from y
    const double *T;            // non-null: eps takes (alpha_A - alpha_B)(T) per cell times eps_base
    double eps_base;            // G h nu0 dx / dnu
    double relax;               // y <- y_old + relax (y_balance - y_old), clamped to [0, 1]
};

// Temperature fits of the energy equation (App. C), T in K; sources in art.h.
// The powers of lambda = 2 T_HI / T and of T are taken as exp(a ln .) from one
// logarithm of T per evaluation.
constexpr double kLn2THI = 12.662275226919286;   // ln(2 * 157807)
__device__ __forceinline__ double th_alpha_A_ln(double lnl)
{
    return 1.269e-13 * exp(1.503 * lnl - 1.923 * log1p(exp(0.470 * (lnl - log(0.522)))));
}
__device__ __forceinline__ double th_alpha_B_ln(double lnl)
{
    return 2.753e-14 * exp(1.500 * lnl - 2.242 * log1p(exp(0.407 * (lnl - log(2.740)))));
}
__device__ __forceinline__ double th_alpha_B(double T) { return th_alpha_B_ln(kLn2THI - log(T)); }
// alpha_A - alpha_B in FP32, for the emissivity that the FP32 sweep takes (the
// difference is ~40 % of alpha_A near 1e4 K: no cancellation; ~1e-6 relative)
__device__ __forceinline__ float th_dalpha_f32(double T)
{
    const float lnl = (float)kLn2THI - logf((float)T);
    const float a = 1.269e-13f * expf(1.503f * lnl - 1.923f * log1pf(expf(0.470f * (lnl + 0.65008769f))));
    const float b = 2.753e-14f * expf(1.500f * lnl - 2.242f * log1pf(expf(0.407f * (lnl - 1.00795792f))));
    return a - b;
}
__device__ __forceinline__ double th_gamma_coll(double T)
{
    return 5.85e-11 * sqrt(T) * exp(-157809.1 / T) / (1.0 + sqrt(T / 1e5));
}

__global__ void balance_kernel(const BalArgs p)
{
    __shared__ double smax[32];
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    double r = 0.0;
    if (i < p.ncell) {
        const double nH = p.nH[i];
        const double yo = p.y[i];
        double y = yo, x = 1.0 - yo;
        if (p.solve) {
            const double g = (double)p.gpt[i] + (double)p.gdiff[i];
            const double a = p.alphaB * nH, c = p.gcoll * nH;
            const double sq = sqrt(4.0 * a * g + (c + g) * (c + g));
            const double den = 2.0 * a + c + g + sq;
            y = den > 0.0 ? 2.0 * a / den : 0.0;
            x = den > 0.0 ? (c + g + sq) / den : 1.0;
            if (p.relax != 1.0) {
                y = fmin(fmax(yo + p.relax * (y - yo), 0.0), 1.0);
                x = 1.0 - y;
            }
            const double ne_new = x * nH, ne_old = (1.0 - yo) * nH;
            r = ne_new > 0.0 ? fabs(ne_new - ne_old) / ne_new : (ne_old > 0.0 ? INFINITY : 0.0);
            p.y[i] = y;
        }
        p.kap[i] = (float)(y * nH * p.kap_coef);
        const double ec = p.T ? p.eps_base * (double)th_dalpha_f32(p.T[i]) : p.eps_coef;
        p.eps[i] = (float)(ec * (x * nH) * (x * nH));
    }
    if (!p.solve) return;
    // block max, then one atomic max on the bit pattern (r >= 0)
    for (int o = 16; o > 0; o >>= 1) r = fmax(r, __shfl_xor_sync(0xffffffffu, r, o));
    if ((threadIdx.x & 31) == 0) smax[threadIdx.x >> 5] = r;
    __syncthreads();
    if (threadIdx.x < 32) {
        r = threadIdx.x < (blockDim.x >> 5) ? smax[threadIdx.x] : 0.0;
        for (int o = 16; o > 0; o >>= 1) r = fmax(r, __shfl_xor_sync(0xffffffffu, r, o));
        if (threadIdx.x == 0) atomicMax(p.resid, (unsigned long long)__double_as_longlong(r));
    }
}

template <typename T> art_status ensure(art_ctx *ctx, T **p, size_t n)
{
    if (*p) return ART_OK;
    void *q = nullptr;
    cudaError_t e = cudaMalloc(&q, n * sizeof(T));
    if (e != cudaSuccess) {
        cudaGetLastError();
        return art_fail(ctx, e == cudaErrorMemoryAllocation ? ART_E_OOM : ART_E_CUDA,
                        std::string("cudaMalloc: ") + cudaGetErrorString(e));
    }
    ctx->dev_bytes += (long long)(n * sizeof(T));
    *p = static_cast<T *>(q);
    return ART_OK;
}

// Sources as the kernel reads them: integer cell + FP32 fraction, and per bin
// the rate constant 3 Q_b sigma_b / (4 pi dx^2) (Q_b = Qb[a][b], or Q_a times
// frac[b] when Qb is null).
art_status pack_sources(art_ctx *ctx, const art_source *src, int n_src, const double *Qb, const double *frac,
                        const double *sigma, int nbins, std::vector<PtSrc> &h)
{
    h.assign(n_src > 0 ? (size_t)n_src : 1, PtSrc{});
    const double dx = ctx->grid.dx_cm;
    const int dims[3] = {ctx->grid.nx, ctx->grid.ny, ctx->grid.nz};
    for (int a = 0; a < n_src; ++a) {
        const art_source &s = src[a];
        const double x[3] = {s.x, s.y, s.z};
        if (!std::isfinite(s.x) || !std::isfinite(s.y) || !std::isfinite(s.z) || !(s.Q >= 0.0) ||
            s.x < 0 || s.y < 0 || s.z < 0 || s.x > dims[0] || s.y > dims[1] || s.z > dims[2])
            return art_fail(ctx, ART_E_INVALID, "point source outside the box or with a bad luminosity");
        PtSrc &P = h[a];
        for (int k = 0; k < 3; ++k) {
            const double f = std::floor(x[k]);
            P.si[k] = (int)f;
            P.sf[k] = (float)(x[k] - f);
            if (P.sf[k] >= 1.0f) {   // a fraction that rounds up to a whole cell
                P.si[k] += 1;
                P.sf[k] = 0.0f;
            }
        }
        for (int b = 0; b < kMaxBins; ++b) {
            double q = 0.0;
            if (b < nbins) q = Qb ? Qb[(size_t)a * nbins + b] : s.Q * (frac ? frac[b] : (b == 0 ? 1.0 : 0.0));
            const double c = 3.0 * q * (b < nbins ? sigma[b] : 0.0) / (4.0 * kPi * dx * dx);
            if (!(q >= 0.0) || !(c <= 3.0e38))
                return art_fail(ctx, ART_E_INVALID, "point source: bad bin luminosity or a rate beyond FP32 range");
            P.coef[b] = (float)c;
        }
    }
    return ART_OK;
}

// Device room for n_src packed sources (at least one).
art_status source_buffer(art_ctx *ctx, int n_src)
{
    const int need = (int)(((size_t)(n_src > 0 ? n_src : 1) * sizeof(PtSrc) + sizeof(double) - 1) / sizeof(double));
    if (ctx->it.nsrc_cap >= need) return ART_OK;
    if (ctx->it.src) cudaFree(ctx->it.src);
    ctx->it.src = nullptr;
    ctx->it.nsrc_cap = need;
    return ensure(ctx, &ctx->it.src, (size_t)need);
}

template <typename IDX> void launch_points_t(const PtArgs &a, unsigned nb, int nt, cudaStream_t st)
{
    switch (a.nbins + (a.scaled ? 4 : 0)) {
    case 1: point_source_kernel<1, false, IDX><<<nb, nt, 0, st>>>(a); break;
    case 2: point_source_kernel<2, false, IDX><<<nb, nt, 0, st>>>(a); break;
    case 3: point_source_kernel<3, false, IDX><<<nb, nt, 0, st>>>(a); break;
    case 4: point_source_kernel<4, false, IDX><<<nb, nt, 0, st>>>(a); break;
    case 5: point_source_kernel<1, true, IDX><<<nb, nt, 0, st>>>(a); break;
    case 6: point_source_kernel<2, true, IDX><<<nb, nt, 0, st>>>(a); break;
    case 7: point_source_kernel<3, true, IDX><<<nb, nt, 0, st>>>(a); break;
    default: point_source_kernel<4, true, IDX><<<nb, nt, 0, st>>>(a); break;
    }
}

// Point-source rates into gamma (device), kappa per bin on the device, or
// (kscale != null) one kappa field scaled per bin.
art_status launch_points(art_ctx *ctx, const float *kappa, int nbins, const PtSrc *d_src, int n_src, float *gamma,
                         cudaStream_t st, const float *kscale = nullptr, float *heat = nullptr,
                         const double *ebin = nullptr)
{
    PtArgs a;
    a.heat = heat;
    for (int b = 0; b < 4; ++b) a.ebin[b] = heat && b < nbins ? (float)ebin[b] : 0.0f;
    a.kappa = kappa;
    a.src = d_src;
    a.nsrc = n_src;
    a.nbins = nbins;
    a.nx = ctx->grid.nx;
    a.ny = ctx->grid.ny;
    a.nz = ctx->grid.nz;
    a.ncell = ctx->ncell;
    a.gamma = gamma;
    a.scaled = kscale != nullptr;
    for (int b = 0; b < 4; ++b) a.kscale[b] = kscale && b < nbins ? kscale[b] : 1.0f;
    if (nbins < 1 || nbins > kMaxBins) return art_fail(ctx, ART_E_INVALID, "point sources: 1 to 4 bins");
    const int nt = 128;
    const unsigned nb = (unsigned)(((a.nx + 7) / 8) * (long long)((a.ny + 3) / 4) * ((a.nz + 3) / 4));
    if (ctx->ncell <= 0x7fffffffLL)
        launch_points_t<int>(a, nb, nt, st);
    else
        launch_points_t<long long>(a, nb, nt, st);
    ICK(ctx, cudaGetLastError());
    return ART_OK;
}

}  // namespace

extern "C" {

art_status art_point_sources(art_ctx *ctx, const float *kappa, const double *sigma, const art_source *src,
                             const double *Qb, int n_src, float *gamma, void *stream)
{
    if (!ctx) return ART_E_INVALID;
    if (ctx->grids.size() != 1) return art_fail(ctx, ART_E_INVALID, "art_point_sources: single-grid contexts only");
    if (!kappa || !sigma || !gamma || (n_src > 0 && !src) || n_src < 0)
        return art_fail(ctx, ART_E_INVALID, "art_point_sources: null argument");
    const int nbins = ctx->nbins;
    if (nbins > kMaxBins) return art_fail(ctx, ART_E_INVALID, "art_point_sources: at most 4 bins");
    if (!(ctx->grid.dx_cm > 0.0)) return art_fail(ctx, ART_E_INVALID, "art_point_sources: grid dx_cm must be > 0");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    for (int b = 0; b < nbins; ++b)
        if (!(sigma[b] >= 0.0)) return art_fail(ctx, ART_E_INVALID, "art_point_sources: bad cross section");
    std::vector<PtSrc> h_src;
    art_status s = pack_sources(ctx, src, n_src, Qb, nullptr, sigma, nbins, h_src);
    if (s != ART_OK) return s;
    if ((s = source_buffer(ctx, n_src)) != ART_OK) return s;
    const PtSrc *d_src = reinterpret_cast<const PtSrc *>(ctx->it.src);
    ICK(ctx, cudaMemcpyAsync(ctx->it.src, h_src.data(), h_src.size() * sizeof(PtSrc), cudaMemcpyHostToDevice, st));
    s = launch_points(ctx, kappa, nbins, d_src, n_src, gamma, st);
    if (s != ART_OK) return s;
    // host vectors are copied from: wait before they go out of scope
    ICK(ctx, cudaStreamSynchronize(st));
    return ART_OK;
}

}  // extern "C"

namespace {

art_status check_iteration_context(art_ctx *ctx, const art_chem *ch, const char *who)
{
    if (ctx->grids.size() != 1) return art_fail(ctx, ART_E_INVALID, std::string(who) + ": single-grid contexts only");
    if (!ch) return art_fail(ctx, ART_E_INVALID, std::string(who) + ": null chemistry");
    if (ctx->prec != ART_FP32 || ctx->nbins != 1 || ctx->opt.field_form != ART_FIELDS_EPS)
        return art_fail(ctx, ART_E_INVALID,
                        std::string(who) + ": needs an FP32 context with one bin and ART_FIELDS_EPS inputs");
    if (!(ctx->grid.dx_cm > 0.0) || !(ch->sigma0 > 0.0) || !(ch->h > 0.0) || !(ch->nu0 > 0.0) || !(ch->dnu > 0.0) ||
        !(ch->alphaB > 0.0) || !(ch->alphaA >= ch->alphaB) || !(ch->gcoll >= 0.0))
        return art_fail(ctx, ART_E_INVALID, std::string(who) + ": bad chemistry constants");
    return ART_OK;
}

// Balance-kernel arguments: kappa = y nH sigma0 dx and the recombination
// emissivity eps = G h nu0 (alpha_A - alpha_B) (x nH)^2 dx / dnu, scaled by
// the band integral G so that the sweep's J^in is Gamma_diff / (4 pi).
BalArgs balance_args(art_ctx *ctx, const art_chem *ch, const double *nH, double *y)
{
    double G = 0.0;
    art_band_integral(ch->sigma0, ch->h, ch->nu0, ch->nu0, ch->nu0 + ch->dnu, &G);
    art_iter_bufs &B = ctx->it;
    BalArgs ba;
    ba.nH = nH;
    ba.gpt = B.gpt;
    ba.gdiff = B.jin;
    ba.alphaB = ch->alphaB;
    ba.gcoll = ch->gcoll;
    ba.kap_coef = ch->sigma0 * ctx->grid.dx_cm;
    ba.eps_coef = G * ch->h * ch->nu0 * (ch->alphaA - ch->alphaB) * ctx->grid.dx_cm / ch->dnu;
    ba.y = y;
    ba.kap = B.kap;
    ba.eps = B.eps;
    ba.resid = B.resid;
    ba.ncell = ctx->ncell;
    ba.solve = 0;
    ba.T = nullptr;
    ba.eps_base = G * ch->h * ch->nu0 * ctx->grid.dx_cm / ch->dnu;
    ba.relax = ctx->relax;
    return ba;
}

// Block means over f^3 cells of two FP64 fields (coarse-mesh n_H and y).
__global__ void mean_d_kernel(const double *__restrict__ a, const double *__restrict__ b, int nx, int ny, int nz, int f,
                              double *__restrict__ ac, double *__restrict__ bc)
{
    const int cx = nx / f, cy = ny / f, cz = nz / f;
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (long long)cx * cy * cz) return;
    const int X = (int)(i % cx), Y = (int)((i / cx) % cy), Z = (int)(i / ((long long)cx * cy));
    double sa = 0.0, sb = 0.0;
    for (int k = 0; k < f; ++k)
        for (int j = 0; j < f; ++j)
            for (int l = 0; l < f; ++l) {
                const long long v = ((long long)(Z * f + k) * ny + (Y * f + j)) * nx + (long long)X * f + l;
                sa += a[v];
                sb += b[v];
            }
    const double inv = 1.0 / ((double)f * f * f);
    ac[i] = sa * inv;
    bc[i] = sb * inv;
}

// Every fine cell takes its coarse cell's value.
__global__ void inject_d_kernel(const double *__restrict__ c, int nx, int ny, int nz, int f, double *__restrict__ out)
{
    const long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= (long long)nx * ny * nz) return;
    const int x = (int)(v % nx), y = (int)((v / nx) % ny), z = (int)(v / ((long long)nx * ny));
    out[v] = c[((long long)(z / f) * (ny / f) + y / f) * (nx / f) + x / f];
}

// Where the iteration records training samples (art_surrogate_collect).
struct SampleSink {
    float *X, *t, *w;
    int n;
};

// The RT / balance fixed-point iteration; with `warm`, J^in comes from the
// surrogate until its phase ends, then from plain sweeps.  With `sink`, every
// plain iteration records the surrogate inputs of its starting state and the
// target from its sweep.
art_status iterate_impl(art_ctx *ctx, art_net *net, const art_chem *ch, const double *nH, const art_source *src,
                        int n_src, double tol, int max_iter, const art_warm_options *warm, double *y,
                        double *resid_hist, art_iter_report *rep, art_warm_report *wrep, cudaStream_t st,
                        SampleSink *sink = nullptr)
{
    if (!ctx) return ART_E_INVALID;
    art_status s = check_iteration_context(ctx, ch, "art_iterate_ionization");
    if (s != ART_OK) return s;
    if (!nH || !y || (n_src > 0 && !src) || n_src < 0 || max_iter < 1 || !(tol > 0.0))
        return art_fail(ctx, ART_E_INVALID, "art_iterate_ionization: bad argument");
    const auto t0 = std::chrono::steady_clock::now();
    const long long n = ctx->ncell;
    art_iter_bufs &B = ctx->it;
    if ((s = ensure(ctx, &B.gpt, n)) != ART_OK || (s = ensure(ctx, &B.kap, n)) != ART_OK ||
        (s = ensure(ctx, &B.eps, n)) != ART_OK || (s = ensure(ctx, &B.jin, n)) != ART_OK ||
        (s = ensure(ctx, &B.resid, 1)) != ART_OK)
        return s;
    if (warm && ((s = ensure(ctx, &B.y0, n)) != ART_OK || (s = ensure(ctx, &B.jsur, n)) != ART_OK)) return s;
    // source spectrum: Q_a frac_b photons/s in bin b, cross section sigma_b (default: one bin at sigma0)
    const int nbp = ctx->spec_bins > 0 ? ctx->spec_bins : 1;
    std::vector<double> sig(nbp), frac(nbp);
    std::vector<float> kscale(nbp);
    for (int b = 0; b < nbp; ++b) {
        sig[b] = ctx->spec_bins > 0 ? ctx->spec_sigma[b] : ch->sigma0;
        frac[b] = ctx->spec_bins > 0 ? ctx->spec_frac[b] : 1.0;
        kscale[b] = (float)(sig[b] / ch->sigma0);
    }
    double plane_coef[4] = {0, 0, 0, 0};   // F frac_b sigma_b of the plane-parallel flux
    for (int b = 0; b < nbp; ++b) plane_coef[b] = ctx->plane_flux * frac[b] * sig[b];
    std::vector<PtSrc> h_src;
    if ((s = pack_sources(ctx, src, n_src, nullptr, frac.data(), sig.data(), nbp, h_src)) != ART_OK) return s;
    if ((s = source_buffer(ctx, n_src)) != ART_OK) return s;
    const PtSrc *d_src = reinterpret_cast<const PtSrc *>(B.src);
    ICK(ctx, cudaMemcpyAsync(B.src, h_src.data(), h_src.size() * sizeof(PtSrc), cudaMemcpyHostToDevice, st));

    const int nt = 256;
    const unsigned nb = (unsigned)((n + nt - 1) / nt);
    int coarse_it = 0;
    if (warm && warm->coarse_solve) {
        // the whole problem on the coarse mesh; its neutral fraction starts the fine iteration
        const int f = warm->coarse_factor;
        if ((s = artnet_coarse(ctx, f, warm->coarse_nside)) != ART_OK) return s;
        art_sur_bufs &S = ctx->sur;
        const long long nc = n / ((long long)f * f * f);
        mean_d_kernel<<<(unsigned)((nc + nt - 1) / nt), nt, 0, st>>>(nH, y, ctx->grid.nx, ctx->grid.ny, ctx->grid.nz, f,
                                                                     S.nHc, S.yc);
        ICK(ctx, cudaGetLastError());
        std::vector<art_source> csrc(src, src + n_src);
        for (art_source &c : csrc) {
            c.x /= f;
            c.y /= f;
            c.z /= f;
        }
        ctx->coarse->spec_bins = ctx->spec_bins;
        ctx->coarse->plane_axis = ctx->plane_axis;   // a flux per area: the same on the coarse mesh
        ctx->coarse->plane_dir = ctx->plane_dir;
        ctx->coarse->plane_flux = ctx->plane_flux;
        ctx->coarse->relax = ctx->relax;
        for (int b = 0; b < 4; ++b) {
            ctx->coarse->spec_sigma[b] = ctx->spec_sigma[b];
            ctx->coarse->spec_frac[b] = ctx->spec_frac[b];
        }
        art_iter_report cr{};
        const art_status cs = iterate_impl(ctx->coarse, nullptr, ch, S.nHc, csrc.data(), n_src, warm->coarse_tol,
                                           max_iter, nullptr, S.yc, nullptr, &cr, nullptr, st);
        if (cs != ART_OK && cs != ART_E_NOT_CONVERGED)
            return art_fail(ctx, cs, std::string("warm start: coarse solve: ") + art_last_error(ctx->coarse));
        coarse_it = cr.iterations;
        inject_d_kernel<<<nb, nt, 0, st>>>(S.yc, ctx->grid.nx, ctx->grid.ny, ctx->grid.nz, f, y);
        ICK(ctx, cudaGetLastError());
    }
    // the state a failed judge falls back to: the coarse-mesh start (or the caller's y)
    if (warm) ICK(ctx, cudaMemcpyAsync(B.y0, y, n * sizeof(double), cudaMemcpyDeviceToDevice, st));
    BalArgs ba = balance_args(ctx, ch, nH, y);
    balance_kernel<<<nb, nt, 0, st>>>(ba);   // kappa, eps of the starting state
    ICK(ctx, cudaGetLastError());
    ba.solve = 1;

    // On-the-spot approximation (Sec. 2.1, Eq. on_the_spot): alpha_A = alpha_B
    // makes the recombination emissivity vanish, so the source function is
    // neglected and J^in = 0 exactly; no sweep (and no surrogate phase) runs.
    const bool otsa = ch->alphaA == ch->alphaB;
    if (otsa) ICK(ctx, cudaMemsetAsync(B.jin, 0, n * sizeof(float), st));
    bool phase1 = !otsa && warm != nullptr && warm->phase1_max_iter > 0;
    bool have_jin = false, judged_early = false;
    int it = 0, conv = 0, it1 = 0, sweeps = 0, fell_back = 0;
    double r = 0.0, judge = 0.0;
    for (it = 1; it <= max_iter; ++it) {
        if ((s = launch_points(ctx, B.kap, nbp, d_src, n_src, B.gpt, st, kscale.data())) != ART_OK)
            return s;
        if (ctx->plane_flux > 0.0 &&
            (s = launch_plane(ctx, B.kap, nbp, ctx->plane_axis, ctx->plane_dir, plane_coef, B.gpt, 1, st,
                              kscale.data())) != ART_OK)
            return s;
        if (otsa) {
            // J^in stays 0
        } else if (have_jin) {
            have_jin = false;   // J^in of this state came with the judge's sweep
        } else if (phase1) {
            s = artnet_surrogate(ctx, net, warm->use_net, warm->coarse_factor, warm->coarse_nside, B.kap, B.eps, y,
                                 B.jin, nullptr, nullptr, st);
            if (s != ART_OK) return s;
            ++it1;
        } else {
            if (sink && it <= sink->n) {
                const long long V = n;
                float *Xk = sink->X + (long long)(it - 1) * 4 * V;
                s = artnet_surrogate(ctx, nullptr, 0, warm->coarse_factor, warm->coarse_nside, B.kap, B.eps, y,
                                     nullptr, Xk, B.jsur, st);
                if (s != ART_OK) return s;
            }
            if ((s = art_internal_layout(ctx, B.kap, B.eps, st)) != ART_OK) return s;
            if ((s = art_internal_sweep(ctx, nullptr, B.jin, nullptr, st)) != ART_OK) return s;
            ++sweeps;
            if (sink && it <= sink->n) {
                if ((s = artnet_target(ctx, B.jin, B.jsur, sink->t + (long long)(it - 1) * n, st))) return s;
                if (sink->w && (s = artnet_weights(ctx, B.jin, sink->w + (long long)(it - 1) * n, st))) return s;
            }
        }
        ICK(ctx, cudaMemsetAsync(B.resid, 0, sizeof(unsigned long long), st));
        balance_kernel<<<nb, nt, 0, st>>>(ba);
        ICK(ctx, cudaGetLastError());
        unsigned long long bits = 0;
        int werr = 0;
        ICK(ctx, cudaMemcpyAsync(&bits, B.resid, sizeof(bits), cudaMemcpyDeviceToHost, st));
        if ((s = art_wave_status_async(ctx, &werr, st)) != ART_OK) return s;
        ICK(ctx, cudaStreamSynchronize(st));
        if (werr && (s = art_wave_status(ctx, st)) != ART_OK) return s;
        std::memcpy(&r, &bits, sizeof(r));
        if (resid_hist) resid_hist[it - 1] = r;
        if (!phase1 && r < tol) {
            conv = 1;
            break;
        }
        const bool end_phase = phase1 && (r < warm->phase1_tol || it1 >= warm->phase1_max_iter);
        const bool early = phase1 && !end_phase && !judged_early && warm->judge_after > 0 &&
                           it1 == warm->judge_after;
        if (end_phase || early) {
            // judge the surrogate against a full sweep on the current state
            if (warm->use_net && (s = artnet_check(net, st)) != ART_OK)
                return art_fail(ctx, s, std::string("surrogate network: ") + artnet_error(net));
            s = artnet_surrogate(ctx, net, warm->use_net, warm->coarse_factor, warm->coarse_nside, B.kap, B.eps, y,
                                 B.jsur, nullptr, nullptr, st);
            if (s != ART_OK) return s;
            if ((s = art_internal_layout(ctx, B.kap, B.eps, st)) != ART_OK) return s;
            if ((s = art_internal_sweep(ctx, nullptr, B.jin, nullptr, st)) != ART_OK) return s;
            ++sweeps;
            if ((s = artnet_l1(ctx, B.jsur, B.jin, &judge, st)) != ART_OK) return s;
            if (!(judge <= warm->judge_tol)) {
                phase1 = false;
                fell_back = 1;
                ICK(ctx, cudaMemcpyAsync(y, B.y0, n * sizeof(double), cudaMemcpyDeviceToDevice, st));
                ba.solve = 0;
                balance_kernel<<<nb, nt, 0, st>>>(ba);
                ICK(ctx, cudaGetLastError());
                ba.solve = 1;
            } else {
                have_jin = true;   // the next iteration takes the judge's exact J^in
                if (end_phase) phase1 = false;
                if (early) judged_early = true;
            }
        }
    }
    if (rep) {
        rep->iterations = conv ? it : max_iter;
        rep->converged = conv;
        rep->residual = r;
        rep->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    }
    if (wrep) {
        wrep->surrogate_iterations = it1;
        wrep->plain_sweeps = sweeps;
        wrep->fell_back = fell_back;
        wrep->judge_error = judge;
        wrep->coarse_iterations = coarse_it;
    }
    return conv ? ART_OK : art_fail(ctx, ART_E_NOT_CONVERGED, "art_iterate_ionization: max_iter reached");
}

// ---------------------------------------------------------------------------
// Time-dependent mode (App. B-D), hydrogen at the fixed temperature of the
// chemistry constants, FP64 per cell.  In one cell over dt at fixed rate g
// the BDF step of App. B,
//   n_HI <- (C dtc + n_HI) / (1 + D dtc),  C = alpha_B n_e n_HII,  D = Gamma_coll n_e + g,
// takes C and D at the start of the sub-step (hydrogen is the lowest
// ionization level, updated first) and is sub-cycled with the chemical
// timestep of App. D, dtc = eps_e |n_e/n_e'| + eps_HI |n_HI/n_HI'|, the last
// sub-step cut to end at dt.  alpha_B: the local recombination term of
// Eq. (gamma_diff) cancels the ground-state recombinations, as in the
// equilibrium balance; g = Gamma_point + Gamma^diff_in.
// ---------------------------------------------------------------------------
__device__ __forceinline__ double dtchem_of(double nH, double y, double alphaB, double gcoll, double g,
                                            double eps_e, double eps_hi)
{
    const double nHI = y * nH, ne = (1.0 - y) * nH;
    const double dHI = alphaB * ne * ne - (gcoll * ne + g) * nHI;   // dn_HI/dt = -dn_e/dt
    if (dHI == 0.0) return INFINITY;
    return eps_e * fabs(ne / dHI) + eps_hi * fabs(nHI / dHI);
}

struct ChemArgs {
    const double *nH;
    const float *gpt, *gdiff;
    const double *y_t;          // state at t
    double *y;                  // in: previous iterate at t + dt; out: the new one
    double alphaB, gcoll, dt, eps_e, eps_hi;
    int max_sub;
    long long ncell;
    unsigned long long *evo;    // [0] max residual, [1] min dt_chem, [2] cells out of sub-steps (double bits / count)
    int mode;                   // 0: min dt_chem of y_t; 1: chemistry over dt
};

__device__ __forceinline__ void block_reduce_bits(unsigned long long v, bool is_max, unsigned long long *dst)
{
    __shared__ unsigned long long sred[32];
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long w = __shfl_xor_sync(0xffffffffu, v, o);
        v = is_max ? (w > v ? w : v) : (w < v ? w : v);
    }
    if ((threadIdx.x & 31) == 0) sred[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x < 32) {
        const unsigned long long id = is_max ? 0ull : ~0ull;
        v = threadIdx.x < (blockDim.x >> 5) ? sred[threadIdx.x] : id;
        for (int o = 16; o > 0; o >>= 1) {
            const unsigned long long w = __shfl_xor_sync(0xffffffffu, v, o);
            v = is_max ? (w > v ? w : v) : (w < v ? w : v);
        }
        if (threadIdx.x == 0) {
            if (is_max) atomicMax(dst, v);
            else atomicMin(dst, v);
        }
    }
}

// Non-negative doubles order like their bit patterns, so max / min reduce on the bits.
__global__ void __launch_bounds__(256) chem_kernel(const ChemArgs p)
{
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const bool in = i < p.ncell;
    if (p.mode == 0) {
        double d = INFINITY;
        if (in) d = dtchem_of(p.nH[i], p.y_t[i], p.alphaB, p.gcoll, (double)p.gpt[i] + (double)p.gdiff[i], p.eps_e,
                              p.eps_hi);
        block_reduce_bits((unsigned long long)__double_as_longlong(d), false, p.evo + 1);
        return;
    }
    double r = 0.0;
    if (in) {
        const double nH = p.nH[i], g = (double)p.gpt[i] + (double)p.gdiff[i];
        double y = p.y_t[i], tau = 0.0;
        int n = 0;
        while (tau < p.dt && n < p.max_sub) {
            const double nHI = y * nH, ne = (1.0 - y) * nH;
            const double C = p.alphaB * ne * ne, D = p.gcoll * ne + g;
            double dtc = dtchem_of(nH, y, p.alphaB, p.gcoll, g, p.eps_e, p.eps_hi);
            const bool last = !(dtc < p.dt - tau);
            if (last) dtc = p.dt - tau;
            y = fmin((C * dtc + nHI) / (1.0 + D * dtc) / nH, 1.0);
            tau = last ? p.dt : tau + dtc;
            ++n;
        }
        if (tau < p.dt) atomicAdd(p.evo + 2, 1ull);
        const double ne_new = (1.0 - y) * nH, ne_old = (1.0 - p.y[i]) * nH;
        r = ne_new > 0.0 ? fabs(ne_new - ne_old) / ne_new : (ne_old > 0.0 ? INFINITY : 0.0);
        p.y[i] = y;
    }
    block_reduce_bits((unsigned long long)__double_as_longlong(r), true, p.evo);
}

art_status evolve_impl(art_ctx *ctx, const art_chem *ch, const double *nH, const art_source *src, int n_src,
                       const art_evolve_options *o, double *y, art_evolve_report *rep, cudaStream_t st)
{
    if (!ctx) return ART_E_INVALID;
    art_status s = check_iteration_context(ctx, ch, "art_evolve_ionization");
    if (s != ART_OK) return s;
    if (!nH || !y || !o || (n_src > 0 && !src) || n_src < 0 || !(o->t_end >= 0.0) || !std::isfinite(o->t_end) ||
        !(o->F > 0.0) || !(o->eps_iter > 0.0) || !(o->eps_e >= 0.0) || !(o->eps_hi >= 0.0) ||
        !(o->eps_e + o->eps_hi > 0.0) || !(o->dt_fixed >= 0.0) || o->max_steps < 1 || o->max_iter < 1 ||
        o->max_sub < 1)
        return art_fail(ctx, ART_E_INVALID, "art_evolve_ionization: bad argument");
    const auto t0 = std::chrono::steady_clock::now();
    const long long n = ctx->ncell;
    art_iter_bufs &B = ctx->it;
    if ((s = ensure(ctx, &B.gpt, n)) != ART_OK || (s = ensure(ctx, &B.kap, n)) != ART_OK ||
        (s = ensure(ctx, &B.eps, n)) != ART_OK || (s = ensure(ctx, &B.jin, n)) != ART_OK ||
        (s = ensure(ctx, &B.yit, n)) != ART_OK || (s = ensure(ctx, &B.evo, 3)) != ART_OK)
        return s;
    const int nbp = ctx->spec_bins > 0 ? ctx->spec_bins : 1;
    std::vector<double> sig(nbp), frac(nbp);
    std::vector<float> kscale(nbp);
    for (int b = 0; b < nbp; ++b) {
        sig[b] = ctx->spec_bins > 0 ? ctx->spec_sigma[b] : ch->sigma0;
        frac[b] = ctx->spec_bins > 0 ? ctx->spec_frac[b] : 1.0;
        kscale[b] = (float)(sig[b] / ch->sigma0);
    }
    double plane_coef[4] = {0, 0, 0, 0};
    for (int b = 0; b < nbp; ++b) plane_coef[b] = ctx->plane_flux * frac[b] * sig[b];
    std::vector<PtSrc> h_src;
    if ((s = pack_sources(ctx, src, n_src, nullptr, frac.data(), sig.data(), nbp, h_src)) != ART_OK) return s;
    if ((s = source_buffer(ctx, n_src)) != ART_OK) return s;
    const PtSrc *d_src = reinterpret_cast<const PtSrc *>(B.src);
    ICK(ctx, cudaMemcpyAsync(B.src, h_src.data(), h_src.size() * sizeof(PtSrc), cudaMemcpyHostToDevice, st));
    const bool otsa = ch->alphaA == ch->alphaB;
    if (otsa) ICK(ctx, cudaMemsetAsync(B.jin, 0, n * sizeof(float), st));
    ICK(ctx, cudaMemsetAsync(B.evo, 0, 3 * sizeof(unsigned long long), st));

    // photo-ionization rates of state ys into B.gpt (+ plane) and B.jin
    int sweeps = 0;
    auto rates = [&](double *ys) -> art_status {
        BalArgs ba = balance_args(ctx, ch, nH, ys);
        const int nt = 256;
        balance_kernel<<<(unsigned)((n + nt - 1) / nt), nt, 0, st>>>(ba);   // kappa, eps of the state
        ICK(ctx, cudaGetLastError());
        art_status r = launch_points(ctx, B.kap, nbp, d_src, n_src, B.gpt, st, kscale.data());
        if (r != ART_OK) return r;
        if (ctx->plane_flux > 0.0 &&
            (r = launch_plane(ctx, B.kap, nbp, ctx->plane_axis, ctx->plane_dir, plane_coef, B.gpt, 1, st,
                              kscale.data())) != ART_OK)
            return r;
        if (!otsa) {
            if ((r = art_internal_layout(ctx, B.kap, B.eps, st)) != ART_OK) return r;
            if ((r = art_internal_sweep(ctx, nullptr, B.jin, nullptr, st)) != ART_OK) return r;
            ++sweeps;
        }
        return ART_OK;
    };
    ChemArgs ca;
    ca.nH = nH;
    ca.gpt = B.gpt;
    ca.gdiff = B.jin;
    ca.y_t = y;
    ca.y = B.yit;
    ca.alphaB = ch->alphaB;
    ca.gcoll = ch->gcoll;
    ca.eps_e = o->eps_e;
    ca.eps_hi = o->eps_hi;
    ca.max_sub = o->max_sub;
    ca.ncell = n;
    ca.evo = B.evo;
    const int nt = 256;
    const unsigned nb = (unsigned)((n + nt - 1) / nt);
    double t = 0.0, dt_min = INFINITY, dt_max = 0.0;
    int steps = 0, iters = 0, unconverged = 0;
    unsigned long long overflow = 0;
    while (t < o->t_end && steps < o->max_steps) {
        if ((s = rates(y)) != ART_OK) return s;
        double dt = o->dt_fixed;
        if (!(dt > 0.0)) {
            const unsigned long long inf_bits = 0x7ff0000000000000ull;
            ICK(ctx, cudaMemcpyAsync(B.evo + 1, &inf_bits, sizeof(inf_bits), cudaMemcpyHostToDevice, st));
            ca.mode = 0;
            chem_kernel<<<nb, nt, 0, st>>>(ca);
            ICK(ctx, cudaGetLastError());
            unsigned long long bits = 0;
            ICK(ctx, cudaMemcpyAsync(&bits, B.evo + 1, sizeof(bits), cudaMemcpyDeviceToHost, st));
            ICK(ctx, cudaStreamSynchronize(st));
            double m;
            std::memcpy(&m, &bits, sizeof(m));
            dt = o->F * m;
        }
        const bool last = !(dt < o->t_end - t);
        if (last) dt = o->t_end - t;
        ca.dt = dt;
        ca.mode = 1;
        ICK(ctx, cudaMemcpyAsync(B.yit, y, n * sizeof(double), cudaMemcpyDeviceToDevice, st));
        int conv = 0;
        for (int k = 1; k <= o->max_iter; ++k) {
            ++iters;
            ICK(ctx, cudaMemsetAsync(B.evo, 0, sizeof(unsigned long long), st));
            chem_kernel<<<nb, nt, 0, st>>>(ca);
            ICK(ctx, cudaGetLastError());
            unsigned long long bits = 0;
            int werr = 0;
            ICK(ctx, cudaMemcpyAsync(&bits, B.evo, sizeof(bits), cudaMemcpyDeviceToHost, st));
            {
                const art_status ws = art_wave_status_async(ctx, &werr, st);
                if (ws != ART_OK) return ws;
            }
            ICK(ctx, cudaStreamSynchronize(st));
            if (werr) {
                const art_status ws = art_wave_status(ctx, st);
                if (ws != ART_OK) return ws;
            }
            double r;
            std::memcpy(&r, &bits, sizeof(r));
            if (r < o->eps_iter) {
                conv = 1;
                break;
            }
            if ((s = rates(B.yit)) != ART_OK) return s;
        }
        if (!conv) unconverged = 1;
        ICK(ctx, cudaMemcpyAsync(y, B.yit, n * sizeof(double), cudaMemcpyDeviceToDevice, st));
        dt_min = std::min(dt_min, dt);
        dt_max = std::max(dt_max, dt);
        t = last ? o->t_end : t + dt;
        ++steps;
    }
    ICK(ctx, cudaMemcpyAsync(&overflow, B.evo + 2, sizeof(overflow), cudaMemcpyDeviceToHost, st));
    ICK(ctx, cudaStreamSynchronize(st));
    if (rep) {
        rep->steps = steps;
        rep->iterations = iters;
        rep->sweeps = sweeps;
        rep->converged = !unconverged;
        rep->sub_overflow = (long long)overflow;
        rep->t = t;
        rep->dt_min = steps ? dt_min : 0.0;
        rep->dt_max = dt_max;
        rep->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    }
    if (t < o->t_end) return art_fail(ctx, ART_E_NOT_CONVERGED, "art_evolve_ionization: max_steps before t_end");
    if (unconverged) return art_fail(ctx, ART_E_NOT_CONVERGED, "art_evolve_ionization: a step reached max_iter");
    return ART_OK;
}

// ---------------------------------------------------------------------------
// Time-dependent mode with the energy equation (App. C).  Per cell and
// chemistry sub-step: the BDF update of App. B with alpha_B(T), Gamma_coll(T)
// at the sub-step's start, then the implicit update of the specific energy at
// the new composition; with e = rho u = 1.5 k_B T n_H (1 + x) it is the root T'
// of
//   f(T') = 1.5 k_B n_H (1 + x') T' + dtc C(n', T') - (e + H' dtc),
// found by a bracket-safeguarded Newton iteration (th_energy_step).
// ---------------------------------------------------------------------------
struct ThermParams {
    int otsa, cool_mask;
    double e_diff, kB, T_min, T_max;
    double compton, T_g;         // Compton coefficient per electron (erg/s/K) and CMB temperature
};

// Cooling rate C(n, T) (erg/s/cm^3) and dC/dT, each term's derivative from
// its logarithmic derivative d ln c / d ln T (rec A: 0.3 - 0.7 u/(1 + u),
// u = (T/1e6)^0.7; rec B: 1 - 1.970 + 3.720 * 0.376 v/(1 + v),
// v = (lambda/2.25)^0.376; collisional ionization: 0.5 + 157809.1/T - 0.5 w/(1 + w),
// w = sqrt(T/1e5); excitation: 118348/T - 0.5 w/(1 + w); free-free:
// 0.5 + 0.34 e^{-d^2/3} (2d / (3 ln 10)) / g_ff, d = log10 of 10^5.5 / T).
template <typename R>
__device__ __forceinline__ R th_cooling(const ThermParams &q, R nH, R y, R T, R &dC)
{
    const R nHI = y * nH, ne = (R(1) - y) * nH;
    const R lnT = log(T), iT = R(1) / T, sT = sqrt(T);
    const R w = sT * R(3.1622776601683794e-3), cden = R(1) + w;   // sqrt(T / 1e5)
    R c = R(0), d = R(0);
    if (q.cool_mask & 1) {
        R rc, g;
        if (q.otsa) {
            const R lnl = R(kLn2THI) - lnT;
            const R v = exp(R(0.376) * (lnl - R(0.81093021621632877)));   // (lambda / 2.25)^0.376
            rc = R(3.435e-30) * T * exp(R(1.970) * lnl - R(3.720) * log1p(v));
            g = R(1) - R(1.970) + R(3.720 * 0.376) * v / (R(1) + v);
        } else {
            const R u = exp(R(0.7) * (lnT - R(13.815510557964274)));     // (T / 1e6)^0.7
            rc = R(8.70e-27) * sT * exp(R(-0.2) * (lnT - R(6.907755278982137))) / (R(1) + u);
            g = R(0.3) - R(0.7) * u / (R(1) + u);
        }
        c += rc * ne * ne;
        d += rc * g * iT * ne * ne;
    }
    if (q.cool_mask & 2) {
        const R r = R(1.27e-21) * sT * exp(R(-157809.1) * iT) / cden;
        c += r * ne * nHI;
        d += r * (R(0.5) + R(157809.1) * iT - R(0.5) * w / cden) * iT * ne * nHI;
    }
    if (q.cool_mask & 4) {
        const R r = R(7.50e-19) * exp(R(-118348.0) * iT) / cden;
        c += r * ne * nHI;
        d += r * (R(118348.0) * iT - R(0.5) * w / cden) * iT * ne * nHI;
    }
    if (q.cool_mask & 8) {
        const R dd = R(5.5) - lnT * R(0.43429448190325176);   // 5.5 - log10 T
        const R e = R(0.34) * exp(-dd * dd / R(3)), gff = R(1.1) + e;
        const R r = R(1.42e-27) * gff * sT;
        c += r * ne * ne;
        d += r * (R(0.5) + e * dd * R(0.28952965460216784) / gff) * iT * ne * ne;   // 2 / (3 ln 10)
    }
    if (q.cool_mask & 16) {
        c += R(q.compton) * (T - R(q.T_g)) * ne;
        d += R(q.compton) * ne;
    }
    dC = d;
    return c;
}

// Newton's method from T on f(T) = A T + dt C(n', T) - B, f' = A + dt dC/dT,
// kept inside the bracket its iterates build (the largest T with f < 0 and the
// smallest with f > 0 so far, within [T_min, T_max]): a step that leaves it,
// or a non-positive f', bisects once both ends are known and otherwise doubles
// or halves T towards the sign change.  Stops when a step moves T by at most
// tol T, at a bound, or after max_it steps.
template <typename R>
__device__ R th_newton(const ThermParams &q, R nH, R y1, R A, R B, R dt, R T, R tol, int max_it)
{
    const R Tmin = R(q.T_min), Tmax = R(q.T_max);
    T = fmin(fmax(T, Tmin), Tmax);
    R lo = Tmin, hi = Tmax;
    bool have_lo = false, have_hi = false;
    for (int it = 0; it < max_it; ++it) {
        R dC;
        const R f = A * T + dt * th_cooling<R>(q, nH, y1, T, dC) - B;
        if (f == R(0)) return T;
        if (f < R(0)) {
            lo = T;
            have_lo = true;
        } else {
            hi = T;
            have_hi = true;
        }
        const R fp = A + dt * dC;
        R Tn = fp > R(0) ? T - f / fp : R(-1);
        if (!(Tn > lo && Tn < hi) || !(fp > R(0))) {
            if (have_lo && have_hi) Tn = R(0.5) * (lo + hi);
            else if (f < R(0)) Tn = fmin(R(2) * T, Tmax);
            else Tn = fmax(R(0.5) * T, Tmin);
        }
        if (fabs(Tn - T) <= tol * T) return Tn;
        T = Tn;
    }
    return T;
}

// The root in FP32 first (to 1e-5 T, ~3 cheap steps), then the FP64 iteration
// from there, which stops once a step moves T by at most 1e-12 T (Newton's
// error is then of order its square): usually one or two FP64 cooling
// evaluations per root instead of ~4.
__device__ double th_energy_step(const ThermParams &q, double nH, double y0, double T0, double y1, double H1,
                                 double dt)
{
    const double A = 1.5 * q.kB * nH * (2.0 - y1);
    const double B = 1.5 * q.kB * nH * (2.0 - y0) * T0 + H1 * dt;
    const float Tf = th_newton<float>(q, (float)nH, (float)y1, (float)A, (float)B, (float)dt, (float)T0, 1e-5f, 50);
    return th_newton<double>(q, nH, y1, A, B, dt, (double)Tf, 1e-12, 100);
}

struct ThermArgs {
    const double *nH;
    const float *gpt, *hpt, *gdiff;   // rates and heating per neutral atom
    const double *y_t, *T_t;          // state at t
    double *y, *T;                    // in: previous iterate at t + dt; out: the new one
    double dt, eps_e, eps_hi;
    int max_sub;
    long long ncell;
    unsigned long long *evo;          // as ChemArgs
    int mode;                         // 0: min dt_chem of the state at t; 1: chemistry and energy over dt
    ThermParams q;
};

__global__ void __launch_bounds__(256) thermal_kernel(const ThermArgs p)
{
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const bool in = i < p.ncell;
    if (p.mode == 0) {
        double d = INFINITY;
        if (in) {
            const double T = p.T_t[i];
            d = dtchem_of(p.nH[i], p.y_t[i], th_alpha_B(T), th_gamma_coll(T), (double)p.gpt[i] + (double)p.gdiff[i],
                          p.eps_e, p.eps_hi);
        }
        block_reduce_bits((unsigned long long)__double_as_longlong(d), false, p.evo + 1);
        return;
    }
    double r = 0.0;
    if (in) {
        const double nH = p.nH[i], gd = (double)p.gdiff[i];
        const double g = (double)p.gpt[i] + gd, hpt = (double)p.hpt[i];
        double y = p.y_t[i], T = p.T_t[i], tau = 0.0;
        int n = 0;
        while (tau < p.dt && n < p.max_sub) {
            const double lnl = kLn2THI - log(T);
            const double aB = th_alpha_B_ln(lnl), gc = th_gamma_coll(T);
            const double dal = p.q.otsa ? 0.0 : th_alpha_A_ln(lnl) - aB;
            const double nHI = y * nH, ne = (1.0 - y) * nH;
            const double C = aB * ne * ne, D = gc * ne + g;
            double dtc = dtchem_of(nH, y, aB, gc, g, p.eps_e, p.eps_hi);
            const bool last = !(dtc < p.dt - tau);
            if (last) dtc = p.dt - tau;
            const double y1 = fmin((C * dtc + nHI) / (1.0 + D * dtc) / nH, 1.0);
            const double ne1 = (1.0 - y1) * nH;
            const double H1 = y1 * nH * (hpt + gd * p.q.e_diff) + dal * ne1 * ne1 * p.q.e_diff;
            T = th_energy_step(p.q, nH, y, T, y1, H1, dtc);
            y = y1;
            tau = last ? p.dt : tau + dtc;
            ++n;
        }
        if (tau < p.dt) atomicAdd(p.evo + 2, 1ull);
        const double ne_new = (1.0 - y) * nH, ne_old = (1.0 - p.y[i]) * nH;
        const double re = ne_new > 0.0 ? fabs(ne_new - ne_old) / ne_new : (ne_old > 0.0 ? INFINITY : 0.0);
        const double u_new = (2.0 - y) * T, u_old = (2.0 - p.y[i]) * p.T[i];
        r = fmax(re, fabs(u_new - u_old) / u_new);
        p.y[i] = y;
        p.T[i] = T;
    }
    block_reduce_bits((unsigned long long)__double_as_longlong(r), true, p.evo);
}

__global__ void temperature_check_kernel(const double *__restrict__ T, long long n, double lo, double hi,
                                         unsigned long long *__restrict__ bad)
{
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n && !(T[i] >= lo && T[i] <= hi)) atomicAdd(bad, 1ull);
}

art_status evolve_thermal_impl(art_ctx *ctx, const art_chem *ch, const art_thermal *th, const double *nH,
                               const art_source *src, int n_src, const art_evolve_options *o, double *y, double *T,
                               art_evolve_report *rep, cudaStream_t st)
{
    if (!ctx) return ART_E_INVALID;
    art_status s = check_iteration_context(ctx, ch, "art_evolve_thermal");
    if (s != ART_OK) return s;
    if (!nH || !y || !T || !o || !th || (n_src > 0 && !src) || n_src < 0 || !(o->t_end >= 0.0) ||
        !std::isfinite(o->t_end) || !(o->F > 0.0) || !(o->eps_iter > 0.0) || !(o->eps_e >= 0.0) ||
        !(o->eps_hi >= 0.0) || !(o->eps_e + o->eps_hi > 0.0) || !(o->dt_fixed >= 0.0) || o->max_steps < 1 ||
        o->max_iter < 1 || o->max_sub < 1)
        return art_fail(ctx, ART_E_INVALID, "art_evolve_thermal: bad argument");
    if (!(th->kB > 0.0) || !(th->T_min > 0.0) || !(th->T_max > th->T_min) || !std::isfinite(th->T_max) ||
        !(th->e_diff >= 0.0) || !std::isfinite(th->e_diff) || !std::isfinite(th->z) || th->z <= -1.0)
        return art_fail(ctx, ART_E_INVALID, "art_evolve_thermal: bad thermal parameters");
    for (int b = 0; b < 4; ++b)
        if (!(th->e_bin[b] >= 0.0) || !std::isfinite(th->e_bin[b]))
            return art_fail(ctx, ART_E_INVALID, "art_evolve_thermal: bad bin energy");
    const auto t0 = std::chrono::steady_clock::now();
    const long long n = ctx->ncell;
    art_iter_bufs &B = ctx->it;
    if ((s = ensure(ctx, &B.gpt, n)) != ART_OK || (s = ensure(ctx, &B.kap, n)) != ART_OK ||
        (s = ensure(ctx, &B.eps, n)) != ART_OK || (s = ensure(ctx, &B.jin, n)) != ART_OK ||
        (s = ensure(ctx, &B.yit, n)) != ART_OK || (s = ensure(ctx, &B.evo, 3)) != ART_OK ||
        (s = ensure(ctx, &B.hpt, n)) != ART_OK || (s = ensure(ctx, &B.Tit, n)) != ART_OK)
        return s;
    const int nt = 256;
    const unsigned nb = (unsigned)((n + nt - 1) / nt);
    ICK(ctx, cudaMemsetAsync(B.evo, 0, 3 * sizeof(unsigned long long), st));
    temperature_check_kernel<<<nb, nt, 0, st>>>(T, n, th->T_min, th->T_max, B.evo + 2);
    ICK(ctx, cudaGetLastError());
    unsigned long long nbad = 0;
    ICK(ctx, cudaMemcpyAsync(&nbad, B.evo + 2, sizeof(nbad), cudaMemcpyDeviceToHost, st));
    ICK(ctx, cudaStreamSynchronize(st));
    if (nbad) return art_fail(ctx, ART_E_INVALID, "art_evolve_thermal: initial temperature outside [T_min, T_max]");

    const int nbp = ctx->spec_bins > 0 ? ctx->spec_bins : 1;
    std::vector<double> sig(nbp), frac(nbp), ebin(nbp);
    std::vector<float> kscale(nbp);
    for (int b = 0; b < nbp; ++b) {
        sig[b] = ctx->spec_bins > 0 ? ctx->spec_sigma[b] : ch->sigma0;
        frac[b] = ctx->spec_bins > 0 ? ctx->spec_frac[b] : 1.0;
        kscale[b] = (float)(sig[b] / ch->sigma0);
        ebin[b] = th->e_bin[b];
    }
    double plane_coef[4] = {0, 0, 0, 0};
    for (int b = 0; b < nbp; ++b) plane_coef[b] = ctx->plane_flux * frac[b] * sig[b];
    std::vector<PtSrc> h_src;
    if ((s = pack_sources(ctx, src, n_src, nullptr, frac.data(), sig.data(), nbp, h_src)) != ART_OK) return s;
    if ((s = source_buffer(ctx, n_src)) != ART_OK) return s;
    const PtSrc *d_src = reinterpret_cast<const PtSrc *>(B.src);
    ICK(ctx, cudaMemcpyAsync(B.src, h_src.data(), h_src.size() * sizeof(PtSrc), cudaMemcpyHostToDevice, st));
    const bool otsa = th->on_the_spot != 0;
    if (otsa) ICK(ctx, cudaMemsetAsync(B.jin, 0, n * sizeof(float), st));

    // rates and heating of state (ys, Ts) into B.gpt, B.hpt (+ plane) and B.jin
    int sweeps = 0;
    auto rates = [&](double *ys, double *Ts) -> art_status {
        BalArgs ba = balance_args(ctx, ch, nH, ys);
        ba.T = Ts;
        balance_kernel<<<nb, nt, 0, st>>>(ba);   // kappa, eps of the state
        ICK(ctx, cudaGetLastError());
        art_status r = launch_points(ctx, B.kap, nbp, d_src, n_src, B.gpt, st, kscale.data(), B.hpt, ebin.data());
        if (r != ART_OK) return r;
        if (ctx->plane_flux > 0.0 &&
            (r = launch_plane(ctx, B.kap, nbp, ctx->plane_axis, ctx->plane_dir, plane_coef, B.gpt, 1, st,
                              kscale.data(), B.hpt, ebin.data())) != ART_OK)
            return r;
        if (!otsa) {
            if ((r = art_internal_layout(ctx, B.kap, B.eps, st)) != ART_OK) return r;
            if ((r = art_internal_sweep(ctx, nullptr, B.jin, nullptr, st)) != ART_OK) return r;
            ++sweeps;
        }
        return ART_OK;
    };
    ThermArgs ta;
    ta.nH = nH;
    ta.gpt = B.gpt;
    ta.hpt = B.hpt;
    ta.gdiff = B.jin;
    ta.y_t = y;
    ta.T_t = T;
    ta.y = B.yit;
    ta.T = B.Tit;
    ta.eps_e = o->eps_e;
    ta.eps_hi = o->eps_hi;
    ta.max_sub = o->max_sub;
    ta.ncell = n;
    ta.evo = B.evo;
    ta.q.otsa = otsa ? 1 : 0;
    ta.q.cool_mask = th->cool_mask;
    ta.q.e_diff = otsa ? 0.0 : th->e_diff;
    ta.q.kB = th->kB;
    ta.q.T_min = th->T_min;
    ta.q.T_max = th->T_max;
    {
        // Compton cooling per electron: 4 sigma_T a T_g^4 k_B / (m_e c)
        const double sigma_T = 6.6524587e-25, a_rad = 7.5657e-15, m_e = 9.1093837e-28, c = 2.99792458e10;
        ta.q.T_g = 2.7255 * (1.0 + th->z);
        ta.q.compton = 4.0 * sigma_T * a_rad * std::pow(ta.q.T_g, 4.0) * th->kB / (m_e * c);
    }
    double t = 0.0, dt_min = INFINITY, dt_max = 0.0;
    int steps = 0, iters = 0, unconverged = 0;
    unsigned long long overflow = 0;
    while (t < o->t_end && steps < o->max_steps) {
        if ((s = rates(y, T)) != ART_OK) return s;
        double dt = o->dt_fixed;
        if (!(dt > 0.0)) {
            const unsigned long long inf_bits = 0x7ff0000000000000ull;
            ICK(ctx, cudaMemcpyAsync(B.evo + 1, &inf_bits, sizeof(inf_bits), cudaMemcpyHostToDevice, st));
            ta.mode = 0;
            thermal_kernel<<<nb, nt, 0, st>>>(ta);
            ICK(ctx, cudaGetLastError());
            unsigned long long bits = 0;
            ICK(ctx, cudaMemcpyAsync(&bits, B.evo + 1, sizeof(bits), cudaMemcpyDeviceToHost, st));
            ICK(ctx, cudaStreamSynchronize(st));
            double m;
            std::memcpy(&m, &bits, sizeof(m));
            dt = o->F * m;
        }
        const bool last = !(dt < o->t_end - t);
        if (last) dt = o->t_end - t;
        ta.dt = dt;
        ta.mode = 1;
        ICK(ctx, cudaMemcpyAsync(B.yit, y, n * sizeof(double), cudaMemcpyDeviceToDevice, st));
        ICK(ctx, cudaMemcpyAsync(B.Tit, T, n * sizeof(double), cudaMemcpyDeviceToDevice, st));
        int conv = 0;
        for (int k = 1; k <= o->max_iter; ++k) {
            ++iters;
            ICK(ctx, cudaMemsetAsync(B.evo, 0, sizeof(unsigned long long), st));
            thermal_kernel<<<nb, nt, 0, st>>>(ta);
            ICK(ctx, cudaGetLastError());
            unsigned long long bits = 0;
            int werr = 0;
            ICK(ctx, cudaMemcpyAsync(&bits, B.evo, sizeof(bits), cudaMemcpyDeviceToHost, st));
            {
                const art_status ws = art_wave_status_async(ctx, &werr, st);
                if (ws != ART_OK) return ws;
            }
            ICK(ctx, cudaStreamSynchronize(st));
            if (werr) {
                const art_status ws = art_wave_status(ctx, st);
                if (ws != ART_OK) return ws;
            }
            double r;
            std::memcpy(&r, &bits, sizeof(r));
            if (r < o->eps_iter) {
                conv = 1;
                break;
            }
            if ((s = rates(B.yit, B.Tit)) != ART_OK) return s;
        }
        if (!conv) unconverged = 1;
        ICK(ctx, cudaMemcpyAsync(y, B.yit, n * sizeof(double), cudaMemcpyDeviceToDevice, st));
        ICK(ctx, cudaMemcpyAsync(T, B.Tit, n * sizeof(double), cudaMemcpyDeviceToDevice, st));
        dt_min = std::min(dt_min, dt);
        dt_max = std::max(dt_max, dt);
        t = last ? o->t_end : t + dt;
        ++steps;
    }
    ICK(ctx, cudaMemcpyAsync(&overflow, B.evo + 2, sizeof(overflow), cudaMemcpyDeviceToHost, st));
    ICK(ctx, cudaStreamSynchronize(st));
    if (rep) {
        rep->steps = steps;
        rep->iterations = iters;
        rep->sweeps = sweeps;
        rep->converged = !unconverged;
        rep->sub_overflow = (long long)overflow;
        rep->t = t;
        rep->dt_min = steps ? dt_min : 0.0;
        rep->dt_max = dt_max;
        rep->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    }
    if (t < o->t_end) return art_fail(ctx, ART_E_NOT_CONVERGED, "art_evolve_thermal: max_steps before t_end");
    if (unconverged) return art_fail(ctx, ART_E_NOT_CONVERGED, "art_evolve_thermal: a step reached max_iter");
    return ART_OK;
}

}  // namespace

extern "C" {

art_status art_iterate_ionization(art_ctx *ctx, const art_chem *ch, const double *nH, const art_source *src,
                                  int n_src, double tol, int max_iter, int warm_start, double *y,
                                  double *resid_hist, art_iter_report *rep, void *stream)
{
    if (!ctx) return ART_E_INVALID;
    const cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (warm_start == ART_WARM_NONE)
        return iterate_impl(ctx, nullptr, ch, nH, src, n_src, tol, max_iter, nullptr, y, resid_hist, rep, nullptr, st);
    if (warm_start != ART_WARM_COARSE && warm_start != ART_WARM_SURROGATE)
        return art_fail(ctx, ART_E_INVALID, "art_iterate_ionization: warm_start must be ART_WARM_NONE, "
                                            "ART_WARM_COARSE or ART_WARM_SURROGATE");
    if (warm_start == ART_WARM_SURROGATE && !ctx->net)
        return art_fail(ctx, ART_E_STATE, "art_iterate_ionization: train the context's surrogate "
                                          "(art_surrogate_train) before ART_WARM_SURROGATE");
    art_warm_options w;
    art_warm_options_default(&w);
    if (warm_start == ART_WARM_COARSE) {
        w.use_net = 0;
        w.phase1_max_iter = 0;   // the coarse-mesh start, then plain iterations
    }
    art_warm_report wr{};
    return iterate_impl(ctx, warm_start == ART_WARM_SURROGATE ? ctx->net : nullptr, ch, nH, src, n_src, tol,
                        max_iter, &w, y, resid_hist, rep, &wr, st);
}

art_status art_evolve_options_default(art_evolve_options *o)
{
    if (!o) return ART_E_INVALID;
    o->t_end = 0.0;
    o->F = 10.0;
    o->eps_iter = 1e-3;
    o->eps_e = 0.2;
    o->eps_hi = 0.002;
    o->dt_fixed = 0.0;
    o->max_steps = 100000;
    o->max_iter = 100;
    o->max_sub = 1000000;
    return ART_OK;
}

art_status art_evolve_ionization(art_ctx *ctx, const art_chem *ch, const double *nH, const art_source *src,
                                 int n_src, const art_evolve_options *opt, double *y, art_evolve_report *rep,
                                 void *stream)
{
    return evolve_impl(ctx, ch, nH, src, n_src, opt, y, rep, static_cast<cudaStream_t>(stream));
}

art_status art_thermal_default(art_thermal *th)
{
    if (!th) return ART_E_INVALID;
    th->on_the_spot = 0;
    th->cool_mask = 31;
    for (int b = 0; b < 4; ++b) th->e_bin[b] = 0.0;
    th->e_diff = 0.0;
    th->z = 0.0;
    th->kB = 1.380649e-16;
    th->T_min = 10.0;
    th->T_max = 1e9;
    return ART_OK;
}

art_status art_evolve_thermal(art_ctx *ctx, const art_chem *ch, const art_thermal *th, const double *nH,
                              const art_source *src, int n_src, const art_evolve_options *opt, double *y, double *T,
                              art_evolve_report *rep, void *stream)
{
    return evolve_thermal_impl(ctx, ch, th, nH, src, n_src, opt, y, T, rep, static_cast<cudaStream_t>(stream));
}

art_status art_set_relaxation(art_ctx *ctx, double omega)
{
    if (!ctx) return ART_E_INVALID;
    if (!(omega > 0.0 && omega < 2.0)) return art_fail(ctx, ART_E_INVALID, "art_set_relaxation: 0 < omega < 2");
    ctx->relax = omega;
    return ART_OK;
}

art_status art_set_plane_source(art_ctx *ctx, int axis, int dir, double flux)
{
    if (!ctx) return ART_E_INVALID;
    if (axis < 0 || axis > 2 || (dir != 1 && dir != -1) || !(flux >= 0.0) || !std::isfinite(flux))
        return art_fail(ctx, ART_E_INVALID, "art_set_plane_source: axis 0-2, dir +-1, finite flux >= 0");
    ctx->plane_axis = axis;
    ctx->plane_dir = dir;
    ctx->plane_flux = flux;
    return ART_OK;
}

art_status art_plane_source(art_ctx *ctx, const float *kappa, const double *sigma, int axis, int dir,
                            const double *flux, float *gamma, void *stream)
{
    if (!ctx) return ART_E_INVALID;
    if (ctx->grids.size() != 1) return art_fail(ctx, ART_E_INVALID, "art_plane_source: single-grid contexts only");
    if (!kappa || !sigma || !flux || !gamma) return art_fail(ctx, ART_E_INVALID, "art_plane_source: null argument");
    if (axis < 0 || axis > 2 || (dir != 1 && dir != -1))
        return art_fail(ctx, ART_E_INVALID, "art_plane_source: axis 0-2 and dir +-1");
    const int nbins = ctx->nbins;
    if (nbins > kMaxBins) return art_fail(ctx, ART_E_INVALID, "art_plane_source: at most 4 bins");
    double coef[4] = {0, 0, 0, 0};
    for (int b = 0; b < nbins; ++b) {
        if (!(sigma[b] >= 0.0) || !(flux[b] >= 0.0) || !std::isfinite(sigma[b]) || !std::isfinite(flux[b]))
            return art_fail(ctx, ART_E_INVALID, "art_plane_source: bad cross section or flux");
        coef[b] = flux[b] * sigma[b];
    }
    const art_status s = launch_plane(ctx, kappa, nbins, axis, dir, coef, gamma, 0, static_cast<cudaStream_t>(stream));
    return s;
}

art_status art_set_source_spectrum(art_ctx *ctx, int nbins, const double *sigma, const double *frac)
{
    if (!ctx) return ART_E_INVALID;
    if (nbins == 0) {
        ctx->spec_bins = 0;
        return ART_OK;
    }
    if (nbins < 1 || nbins > kMaxBins || !sigma || !frac)
        return art_fail(ctx, ART_E_INVALID, "art_set_source_spectrum: 1 to 4 bins with cross sections and fractions");
    for (int b = 0; b < nbins; ++b)
        if (!(sigma[b] > 0.0) || !std::isfinite(sigma[b]) || !(frac[b] >= 0.0) || !std::isfinite(frac[b]))
            return art_fail(ctx, ART_E_INVALID, "art_set_source_spectrum: bad cross section or fraction");
    ctx->spec_bins = nbins;
    for (int b = 0; b < nbins; ++b) {
        ctx->spec_sigma[b] = sigma[b];
        ctx->spec_frac[b] = frac[b];
    }
    return ART_OK;
}

art_status art_warm_options_default(art_warm_options *o)
{
    if (!o) return ART_E_INVALID;
    o->coarse_factor = 4;
    o->coarse_nside = 4;
    o->use_net = 1;
    o->phase1_max_iter = 40;
    o->phase1_tol = 1e-3;
    o->judge_tol = 0.3;
    o->coarse_solve = 1;
    o->coarse_tol = 1e-4;
    o->judge_after = 2;
    return ART_OK;
}

art_status art_iterate_ionization_warm(art_ctx *ctx, art_net *net, const art_chem *ch, const double *nH,
                                       const art_source *src, int n_src, double tol, int max_iter,
                                       const art_warm_options *wopt, double *y, double *resid_hist,
                                       art_warm_report *rep, void *stream)
{
    if (!ctx) return ART_E_INVALID;
    art_warm_options w;
    if (wopt) w = *wopt;
    else art_warm_options_default(&w);
    if (w.coarse_factor < 1 || w.coarse_nside < 1 || w.phase1_max_iter < 0 || !(w.phase1_tol > 0.0) ||
        !(w.judge_tol >= 0.0) || (w.use_net && !net) || (w.coarse_solve && !(w.coarse_tol > 0.0)) ||
        w.judge_after < 0)
        return art_fail(ctx, ART_E_INVALID, "art_iterate_ionization_warm: bad warm-start options");
    art_iter_report r{};
    art_status s = iterate_impl(ctx, net, ch, nH, src, n_src, tol, max_iter, &w, y, resid_hist, &r, rep,
                                static_cast<cudaStream_t>(stream));
    if (rep) rep->total = r;
    return s;
}

art_status art_surrogate_sample(art_ctx *ctx, const art_chem *ch, const double *nH, const double *y,
                                int coarse_factor, int coarse_nside, float *X, float *t, float *jin, float *jc,
                                void *stream)
{
    if (!ctx) return ART_E_INVALID;
    art_status s = check_iteration_context(ctx, ch, "art_surrogate_sample");
    if (s != ART_OK) return s;
    if (!nH || !y) return art_fail(ctx, ART_E_INVALID, "art_surrogate_sample: null state");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const long long n = ctx->ncell;
    art_iter_bufs &B = ctx->it;
    if ((s = ensure(ctx, &B.kap, n)) != ART_OK || (s = ensure(ctx, &B.eps, n)) != ART_OK ||
        (s = ensure(ctx, &B.jin, n)) != ART_OK || (s = ensure(ctx, &B.jsur, n)) != ART_OK)
        return s;
    BalArgs ba = balance_args(ctx, ch, nH, const_cast<double *>(y));
    balance_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(ba);
    ICK(ctx, cudaGetLastError());
    float *jcf = jc ? jc : B.jsur;
    float *jf = jin ? jin : B.jin;
    if ((s = artnet_surrogate(ctx, nullptr, 0, coarse_factor, coarse_nside, B.kap, B.eps, y, nullptr, X, jcf, st)) !=
        ART_OK)
        return s;
    if ((s = art_internal_layout(ctx, B.kap, B.eps, st)) != ART_OK) return s;
    if ((s = art_internal_sweep(ctx, nullptr, jf, nullptr, st)) != ART_OK) return s;
    if (t && (s = artnet_target(ctx, jf, jcf, t, st)) != ART_OK) return s;
    return ART_OK;
}

art_status art_surrogate_collect(art_ctx *ctx, const art_chem *ch, const double *nH, const art_source *src, int n_src,
                                 double *y, int n_iter, int coarse_factor, int coarse_nside, float *X, float *t,
                                 float *w, void *stream)
{
    if (!ctx) return ART_E_INVALID;
    if (!X || !t || n_iter < 1) return art_fail(ctx, ART_E_INVALID, "art_surrogate_collect: bad argument");
    if (ch && ch->alphaA == ch->alphaB)
        return art_fail(ctx, ART_E_INVALID, "art_surrogate_collect: no diffuse field to learn under the on-the-spot approximation");
    art_warm_options wo;
    art_warm_options_default(&wo);
    wo.coarse_factor = coarse_factor;
    wo.coarse_nside = coarse_nside;
    wo.use_net = 0;
    wo.phase1_max_iter = 0;
    wo.coarse_solve = 0;
    SampleSink sink{X, t, w, n_iter};
    art_iter_report r{};
    const art_status s = iterate_impl(ctx, nullptr, ch, nH, src, n_src, 1e-300, n_iter, &wo, y, nullptr, &r, nullptr,
                                      static_cast<cudaStream_t>(stream), &sink);
    return s == ART_E_NOT_CONVERGED ? ART_OK : s;
}

}  // extern "C"
