// art_ion.cu -- point sources (long characteristics with the photon-conserving
// rate of App. A), the FP64 hydrogen ionization balance (App. B, equilibrium
// limit) and the RT / balance fixed-point iteration (App. D) of Tanaka et al.
// (2014), on top of the diffuse-radiation sweep.
#include <cuda_runtime.h>

#include <chrono>
#include <cmath>
#include <cstring>
#include <string>
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
//   Gamma   += 3 Q_b sigma_b e^-tau phi(dtau) / (4 pi dx^2 (r_out^2 + r_out r_in + r_in^2)),
// free of the cancellation of r_out^3 - r_in^3 far from the source.  The
// march is FP32 in relative form: it keeps, per axis, the parametric distance
// to that axis' next plane (an O(1) number, so rounding stays ~1e-7 absolute
// instead of growing with the distance from the source); crossings within
// 1e-6 of each other are taken together.  r_in and r_out come from the target
// cell's faces in FP64.
// ---------------------------------------------------------------------------
struct PtArgs {
    const float *kappa;   // [bins][ncell], or one field scaled per bin (scaled != 0)
    const double *src;    // [nsrc][4]: x, y, z, (unused)
    const double *Qb;     // [nsrc][bins]
    const double *sigma;  // [bins]
    int nsrc, nbins;
    int nx, ny, nz;
    long long ncell;
    double dx;
    float *gamma;
    int scaled;           // kappa_b = kappa * kscale[b] (one field for all bins, one tau to march)
    float kscale[4];
};

constexpr int kMaxBins = 4;   // point-source kernels are compiled for 1-4 bins
#ifndef PT_UNROLL
#define PT_UNROLL 4                // march steps whose kappa loads are issued together
#endif

template <int NB, bool SCALED> __global__ void __launch_bounds__(128) point_source_kernel(const PtArgs p)
{
    const long long cell = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (cell >= p.ncell) return;
    const int tx = (int)(cell % p.nx), ty = (int)((cell / p.nx) % p.ny), tz = (int)(cell / ((long long)p.nx * p.ny));
    const int dims[3] = {p.nx, p.ny, p.nz};
    const int maxsteps = p.nx + p.ny + p.nz + 4;
    double g = 0.0;
    for (int a = 0; a < p.nsrc; ++a) {
        const double s[3] = {p.src[4 * a], p.src[4 * a + 1], p.src[4 * a + 2]};
        const double c[3] = {tx + 0.5, ty + 0.5, tz + 0.5};
        double d[3] = {c[0] - s[0], c[1] - s[1], c[2] - s[2]};
        const double L2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
        if (L2 < 1e-24) {
            d[0] = 1.0;
            d[1] = d[2] = 0.0;
        } else {
            const double il = 1.0 / sqrt(L2);
            d[0] *= il;
            d[1] *= il;
            d[2] *= il;
        }
        // first cell: the one containing s + 1e-9 d
        int cur[3], stp[3];
        double rn[3];
        float r[3], dl[3];   // parametric distance to the next plane of each axis; plane spacing
        for (int k = 0; k < 3; ++k) {
            int v = (int)floor(s[k] + 1e-9 * d[k]);
            cur[k] = v < 0 ? 0 : (v >= dims[k] ? dims[k] - 1 : v);
            stp[k] = d[k] > 0.0 ? 1 : (d[k] < 0.0 ? -1 : 0);
            rn[k] = stp[k] ? 1.0 / d[k] : 0.0;
            r[k] = stp[k] > 0 ? (float)((cur[k] + 1 - s[k]) * rn[k])
                              : (stp[k] < 0 ? (float)((cur[k] - s[k]) * rn[k]) : INFINITY);
            dl[k] = stp[k] ? (float)fabs(rn[k]) : INFINITY;
        }
        // March in rounds of U steps: first the U cells and path lengths (the
        // cell walk does not depend on kappa), with their kappa loads issued
        // together, then the U optical-depth updates in order.
        constexpr int U = PT_UNROLL;
        constexpr int NK = SCALED ? 1 : NB;   // kappa fields marched
        float tau[NK];
#pragma unroll
        for (int b = 0; b < NK; ++b) tau[b] = 0.0f;
        const long long target = cell;
        int state = 0;   // 0 marching, 1 at the target cell, 2 left the box (cannot happen)
        int it = 0;
        while (state == 0 && it < maxsteps) {
            float kv[U][NK], dv[U];
            int nu = 0;
#pragma unroll
            for (int u = 0; u < U; ++u) {
                if (state == 0 && it < maxsteps) {
                    const long long ci = ((long long)cur[2] * p.ny + cur[1]) * p.nx + cur[0];
                    if (ci == target) {
                        state = 1;
                    } else {
                        const float ds = fminf(r[0], fminf(r[1], r[2]));
#pragma unroll
                        for (int b = 0; b < NK; ++b) kv[u][b] = __ldg(p.kappa + (long long)b * p.ncell + ci);
                        dv[u] = ds;
                        nu = u + 1;
                        ++it;
#pragma unroll
                        for (int k = 0; k < 3; ++k) {
                            r[k] -= ds;
                            if (r[k] <= 1e-6f) {   // this axis' plane is crossed here (ties within 1e-6 together)
                                cur[k] += stp[k];
                                if (cur[k] < 0 || cur[k] >= dims[k]) state = 2;
                                r[k] += dl[k];
                            }
                        }
                    }
                }
            }
#pragma unroll
            for (int u = 0; u < U; ++u)
                if (u < nu) {
#pragma unroll
                    for (int b = 0; b < NK; ++b) tau[b] = fmaf(kv[u][b], dv[u], tau[b]);
                }
        }
        if (state == 1) {
            const long long ci = target;
            {
                // passage through the target cell, exactly, from its faces
                double rin = 0.0, rout = INFINITY;
                for (int k = 0; k < 3; ++k) {
                    if (!stp[k]) continue;
                    const double t1 = (tx * (k == 0) + ty * (k == 1) + tz * (k == 2) - s[k]) * rn[k];
                    const double t2 = t1 + rn[k];
                    rin = fmax(rin, fmin(t1, t2));
                    rout = fmin(rout, fmax(t1, t2));
                }
                const double den = 4.0 * kPi * p.dx * p.dx * (rout * rout + rout * rin + rin * rin);
#pragma unroll
                for (int b = 0; b < NB; ++b) {
                    const double kb = SCALED ? (double)p.kappa[ci] * p.kscale[b]
                                             : (double)p.kappa[(long long)b * p.ncell + ci];
                    const double tb = SCALED ? (double)tau[0] * p.kscale[b] : (double)tau[b];
                    const double x = kb * (rout - rin);
                    const double ph = x > 0.0 ? -expm1(-x) / x : 1.0;
                    g += 3.0 * p.Qb[(long long)a * p.nbins + b] * p.sigma[b] * exp(-tb) * ph / den;
                }
            }
        }
    }
    p.gamma[cell] = (float)g;
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
};

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
            const double ne_new = x * nH, ne_old = (1.0 - yo) * nH;
            r = ne_new > 0.0 ? fabs(ne_new - ne_old) / ne_new : (ne_old > 0.0 ? INFINITY : 0.0);
            p.y[i] = y;
        }
        p.kap[i] = (float)(y * nH * p.kap_coef);
        p.eps[i] = (float)(p.eps_coef * (x * nH) * (x * nH));
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

art_status upload_sources(art_ctx *ctx, const art_source *src, int n_src, const double *Qb, int nbins,
                          std::vector<double> &h_src, std::vector<double> &h_q)
{
    h_src.assign(4 * (size_t)n_src, 0.0);
    h_q.assign((size_t)n_src * nbins, 0.0);
    for (int a = 0; a < n_src; ++a) {
        const art_source &s = src[a];
        if (!std::isfinite(s.x) || !std::isfinite(s.y) || !std::isfinite(s.z) || !(s.Q >= 0.0) ||
            s.x < 0 || s.y < 0 || s.z < 0 || s.x > ctx->grid.nx || s.y > ctx->grid.ny || s.z > ctx->grid.nz)
            return art_fail(ctx, ART_E_INVALID, "point source outside the box or with a bad luminosity");
        h_src[4 * a] = s.x;
        h_src[4 * a + 1] = s.y;
        h_src[4 * a + 2] = s.z;
        for (int b = 0; b < nbins; ++b) h_q[(size_t)a * nbins + b] = Qb ? Qb[(size_t)a * nbins + b] : (b == 0 ? s.Q : 0.0);
    }
    return ART_OK;
}

// Point-source rates into gamma (device), kappa per bin on the device, or
// (kscale != null) one kappa field scaled per bin.
art_status launch_points(art_ctx *ctx, const float *kappa, int nbins, const double *d_src, const double *d_q,
                         const double *d_sigma, int n_src, float *gamma, cudaStream_t st,
                         const float *kscale = nullptr)
{
    PtArgs a;
    a.kappa = kappa;
    a.src = d_src;
    a.Qb = d_q;
    a.sigma = d_sigma;
    a.nsrc = n_src;
    a.nbins = nbins;
    a.nx = ctx->grid.nx;
    a.ny = ctx->grid.ny;
    a.nz = ctx->grid.nz;
    a.ncell = ctx->ncell;
    a.dx = ctx->grid.dx_cm;
    a.gamma = gamma;
    a.scaled = kscale != nullptr;
    for (int b = 0; b < 4; ++b) a.kscale[b] = kscale && b < nbins ? kscale[b] : 1.0f;
    const int nt = 128;
    const unsigned nb = (unsigned)((ctx->ncell + nt - 1) / nt);
    if (a.scaled) {
        switch (nbins) {
        case 1: point_source_kernel<1, true><<<nb, nt, 0, st>>>(a); break;
        case 2: point_source_kernel<2, true><<<nb, nt, 0, st>>>(a); break;
        case 3: point_source_kernel<3, true><<<nb, nt, 0, st>>>(a); break;
        case 4: point_source_kernel<4, true><<<nb, nt, 0, st>>>(a); break;
        default: return art_fail(ctx, ART_E_INVALID, "point sources: 1 to 4 bins");
        }
    } else {
        switch (nbins) {
        case 1: point_source_kernel<1, false><<<nb, nt, 0, st>>>(a); break;
        case 2: point_source_kernel<2, false><<<nb, nt, 0, st>>>(a); break;
        case 3: point_source_kernel<3, false><<<nb, nt, 0, st>>>(a); break;
        case 4: point_source_kernel<4, false><<<nb, nt, 0, st>>>(a); break;
        default: return art_fail(ctx, ART_E_INVALID, "point sources: 1 to 4 bins");
        }
    }
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
    std::vector<double> h_src, h_q;
    art_status s = upload_sources(ctx, src, n_src, Qb, nbins, h_src, h_q);
    if (s != ART_OK) return s;
    for (int b = 0; b < nbins; ++b)
        if (!(sigma[b] >= 0.0)) return art_fail(ctx, ART_E_INVALID, "art_point_sources: bad cross section");
    const int cap = n_src > 0 ? n_src : 1;
    if (ctx->it.nsrc_cap < cap * (nbins + 4) + nbins) {
        if (ctx->it.src) cudaFree(ctx->it.src);
        ctx->it.src = nullptr;
        ctx->it.nsrc_cap = cap * (nbins + 4) + nbins;
        if ((s = ensure(ctx, &ctx->it.src, (size_t)ctx->it.nsrc_cap)) != ART_OK) return s;
    }
    double *d_src = ctx->it.src, *d_q = d_src + 4 * cap, *d_sig = d_q + (size_t)cap * nbins;
    if (n_src > 0) {
        ICK(ctx, cudaMemcpyAsync(d_src, h_src.data(), h_src.size() * sizeof(double), cudaMemcpyHostToDevice, st));
        ICK(ctx, cudaMemcpyAsync(d_q, h_q.data(), h_q.size() * sizeof(double), cudaMemcpyHostToDevice, st));
    }
    ICK(ctx, cudaMemcpyAsync(d_sig, sigma, nbins * sizeof(double), cudaMemcpyHostToDevice, st));
    s = launch_points(ctx, kappa, nbins, d_src, d_q, d_sig, n_src, gamma, st);
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
    std::vector<double> h_src, h_q;
    if ((s = upload_sources(ctx, src, n_src, nullptr, 1, h_src, h_q)) != ART_OK) return s;
    std::vector<double> h_qb((size_t)(n_src > 0 ? n_src : 1) * nbp, 0.0);
    for (int a = 0; a < n_src; ++a)
        for (int b = 0; b < nbp; ++b) h_qb[(size_t)a * nbp + b] = h_q[a] * frac[b];
    const int cap = n_src > 0 ? n_src : 1;
    const int need = cap * (4 + nbp) + nbp;
    if (B.nsrc_cap < need) {
        if (B.src) cudaFree(B.src);
        B.src = nullptr;
        B.nsrc_cap = need;
        if ((s = ensure(ctx, &B.src, (size_t)B.nsrc_cap)) != ART_OK) return s;
    }
    double *d_src = B.src, *d_q = d_src + 4 * cap, *d_sig = d_q + (size_t)cap * nbp;
    if (n_src > 0) {
        ICK(ctx, cudaMemcpyAsync(d_src, h_src.data(), h_src.size() * sizeof(double), cudaMemcpyHostToDevice, st));
        ICK(ctx, cudaMemcpyAsync(d_q, h_qb.data(), (size_t)n_src * nbp * sizeof(double), cudaMemcpyHostToDevice, st));
    }
    ICK(ctx, cudaMemcpyAsync(d_sig, sig.data(), nbp * sizeof(double), cudaMemcpyHostToDevice, st));

    const int nt = 256;
    const unsigned nb = (unsigned)((n + nt - 1) / nt);
    if (warm) ICK(ctx, cudaMemcpyAsync(B.y0, y, n * sizeof(double), cudaMemcpyDeviceToDevice, st));
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
    BalArgs ba = balance_args(ctx, ch, nH, y);
    balance_kernel<<<nb, nt, 0, st>>>(ba);   // kappa, eps of the starting state
    ICK(ctx, cudaGetLastError());
    ba.solve = 1;

    bool phase1 = warm != nullptr && warm->phase1_max_iter > 0;
    bool have_jin = false;
    int it = 0, conv = 0, it1 = 0, sweeps = 0, fell_back = 0;
    double r = 0.0, judge = 0.0;
    for (it = 1; it <= max_iter; ++it) {
        if ((s = launch_points(ctx, B.kap, nbp, d_src, d_q, d_sig, n_src, B.gpt, st, kscale.data())) != ART_OK)
            return s;
        if (have_jin) {
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
        ICK(ctx, cudaMemcpyAsync(&bits, B.resid, sizeof(bits), cudaMemcpyDeviceToHost, st));
        ICK(ctx, cudaStreamSynchronize(st));
        std::memcpy(&r, &bits, sizeof(r));
        if (resid_hist) resid_hist[it - 1] = r;
        if (!phase1 && r < tol) {
            conv = 1;
            break;
        }
        if (phase1 && (r < warm->phase1_tol || it1 >= warm->phase1_max_iter)) {
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
            phase1 = false;
            if (!(judge <= warm->judge_tol)) {
                fell_back = 1;
                ICK(ctx, cudaMemcpyAsync(y, B.y0, n * sizeof(double), cudaMemcpyDeviceToDevice, st));
                ba.solve = 0;
                balance_kernel<<<nb, nt, 0, st>>>(ba);
                ICK(ctx, cudaGetLastError());
                ba.solve = 1;
            } else {
                have_jin = true;
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

}  // namespace

extern "C" {

art_status art_iterate_ionization(art_ctx *ctx, const art_chem *ch, const double *nH, const art_source *src,
                                  int n_src, double tol, int max_iter, double *y, double *resid_hist,
                                  art_iter_report *rep, void *stream)
{
    return iterate_impl(ctx, nullptr, ch, nH, src, n_src, tol, max_iter, nullptr, y, resid_hist, rep, nullptr,
                        static_cast<cudaStream_t>(stream));
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
        !(w.judge_tol >= 0.0) || (w.use_net && !net) || (w.coarse_solve && !(w.coarse_tol > 0.0)))
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
