/*
 * oracle.c -- plain FP64 CPU oracle for the diffuse-radiation ray-tracing
 * scheme of Tanaka, Yoshikawa, Okamoto & Hasegawa (2014), "A new ray-tracing
 * scheme for 3D diffuse radiation transfer on highly parallel architectures".
 *
 * TEST INFRASTRUCTURE.  This library exists only to check the CUDA path.  Only
 * the test suite, the package smoke check and the benchmark's CPU-baseline leg
 * may load it.  It shares no code, header, table or constant with the CUDA
 * library; both sides receive the same seeded inputs and physical constants
 * from their caller.
 *
 * What it computes, in the paper's order:
 *   - directions: HEALPix RING pixel centres (Sec. 2.3; Gorski et al. 2005,
 *     Sec. 4, pixel-to-angle relations of the RING scheme);
 *   - the parallel-ray family of each direction (Sec. 2.2, Fig. parallel_ray;
 *     reading: a unit lattice of lines on planes normal to the dominant axis,
 *     offset to cell centres), each line marched cell by cell from where it
 *     enters the box with vacuum intensity, or with a given boundary
 *     intensity (the incident-radiation boundary of Sec. 4.3);
 *   - the per-segment transfer step, Eq. (rt); the path-averaged incoming
 *     intensity of a segment (the equation after Eq. (rt)); the Delta-tau
 *     weighted cell average, Eqs. (path_averaged_intensity) and
 *     (averaged_intensity); the angle average, Eq. (mean_intensity) and the
 *     definition of J^in that follows it;
 *   - the photo-ionization rate of the diffuse field, Eq. (gamma_diff);
 *   - point sources by long characteristics with the photon-conserving rate
 *     of App. A, Eq. (pc_gamma), with the absorbed count taken as in minus
 *     out (App. A prints out minus in; the sign is a typo);
 *   - a plane-parallel incident photon flux through one face (Test-3 setup,
 *     Sec. 4.3), absorbed cell by cell with the same photon-conserving rate;
 *   - the on-the-spot approximation (Sec. 2.1, Eq. on_the_spot) as the case
 *     alpha_A = alpha_B, where the recombination emissivity vanishes;
 *   - the hydrogen ionization balance of App. B in its dt -> infinity
 *     (equilibrium) limit, and the RT/balance fixed-point iteration of App. D
 *     with the electron-density convergence test;
 *   - the time-dependent mode: the BDF update of App. B sub-cycled with the
 *     chemical timestep of App. D, RT steps of F times the smallest of them,
 *     each iterated to convergence of n_e (fixed temperature); and with the
 *     energy equation of App. C: temperature-dependent rates, photo-heating
 *     and radiative cooling, the implicit update of the specific energy,
 *     each RT step iterated to convergence of n_e and u.
 *
 * Everything is FP64.  Summations run in a fixed order (directions in RING
 * order, rays in lattice order, sources in index order), so the oracle is
 * deterministic for a given thread count and bit-identical across thread
 * counts (directions are computed in parallel but added in RING order).
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

/* Crossing parameters closer than this (in cell widths along the dominant
 * axis) are one crossing: a ray through an edge or a corner steps across all
 * the planes it meets there at once, and no zero-length segment is emitted. */
#define ORC_TIE 1e-12

/* ------------------------------------------------------------------------ */
/* Directions: HEALPix RING scheme, pixel index -> unit vector.              */
/* Gorski et al. (2005), Sec. 4: north polar cap, equatorial belt, south    */
/* polar cap; ring index i, pixel-in-ring index j, z = cos(theta), phi.      */
/* ------------------------------------------------------------------------ */
int orc_n_dirs(int nside) { return 12 * nside * nside; }

void orc_healpix_vec(int nside, long p, double v[3])
{
    const double ns = (double)nside;
    const long npix = 12L * nside * nside;
    const long ncap = 2L * nside * (nside - 1);
    double z, phi;
    if (p < ncap) {
        double ph = 0.5 * (double)(p + 1);
        long i = (long)floor(sqrt(ph - sqrt(floor(ph)))) + 1;
        long j = p + 1 - 2 * i * (i - 1);
        z = 1.0 - (double)(i * i) / (3.0 * ns * ns);
        phi = M_PI / (2.0 * (double)i) * ((double)j - 0.5);
    } else if (p < npix - ncap) {
        long q = p - ncap;
        long i = q / (4 * nside) + nside;
        long j = q % (4 * nside) + 1;
        long s = (i - nside + 1) % 2;
        z = 4.0 / 3.0 - 2.0 * (double)i / (3.0 * ns);
        phi = M_PI / (2.0 * ns) * ((double)j - 0.5 * (double)s);
    } else {
        double ph = 0.5 * (double)(npix - p);
        long i = (long)floor(sqrt(ph - sqrt(floor(ph)))) + 1;
        long j = 4 * i + 1 - (npix - p - 2 * i * (i - 1));
        z = -1.0 + (double)(i * i) / (3.0 * ns * ns);
        phi = M_PI / (2.0 * (double)i) * ((double)j - 0.5);
    }
    double st = sqrt((1.0 - z) * (1.0 + z));
    v[0] = st * cos(phi);
    v[1] = st * sin(phi);
    v[2] = z;
}

int orc_healpix_dirs(int nside, double *out)
{
    if (nside < 1) return -1;
    long n = orc_n_dirs(nside);
    for (long p = 0; p < n; p++) orc_healpix_vec(nside, p, out + 3 * p);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Frame of one direction.  a = dominant axis (the lowest index among the    */
/* components within tie_tol of the largest magnitude), b < c the other two. */
/* The rays are the lines X_a = upwind + sa*u, X_b = j + 1/2 + qb*u,         */
/* X_c = k + 1/2 + qc*u with integer (j, k), u the distance along a from the */
/* upwind a-face, qb = n_b/|n_a|, qc = n_c/|n_a| (clamped to [-1, 1]); the   */
/* path length of a piece of ray is du / |n_a|.                              */
/* ------------------------------------------------------------------------ */
typedef struct {
    int dims[3];          /* nx, ny, nz */
    int a, b, c;          /* axes */
    int sa;               /* sign of n_a */
    double na, qb, qc;
    int Na, Nb, Nc;
} frame_t;

static double clamp1(double q) { return q > 1.0 ? 1.0 : (q < -1.0 ? -1.0 : q); }

static void frame_of(const int dims[3], const double n[3], double tie_tol, frame_t *f)
{
    double m = fabs(n[0]);
    if (fabs(n[1]) > m) m = fabs(n[1]);
    if (fabs(n[2]) > m) m = fabs(n[2]);
    int a = 0;
    for (int i = 0; i < 3; i++)
        if (fabs(n[i]) >= m - tie_tol * m) { a = i; break; }
    f->a = a;
    f->b = (a == 0) ? 1 : 0;
    f->c = (a == 2) ? 1 : 2;
    f->sa = n[a] >= 0.0 ? 1 : -1;
    f->na = fabs(n[a]);
    f->qb = clamp1(n[f->b] / f->na);
    f->qc = clamp1(n[f->c] / f->na);
    for (int i = 0; i < 3; i++) f->dims[i] = dims[i];
    f->Na = dims[a];
    f->Nb = dims[f->b];
    f->Nc = dims[f->c];
}

/* Range of u over which the ray (j, k) is inside the open box. */
static int ray_u_range(const frame_t *f, long j, long k, double *u0, double *u1)
{
    double lo = 0.0, hi = (double)f->Na;
    double xb0 = (double)j + 0.5, xc0 = (double)k + 0.5;
    const double q[2] = {f->qb, f->qc};
    const double x0[2] = {xb0, xc0};
    const int N[2] = {f->Nb, f->Nc};
    for (int t = 0; t < 2; t++) {
        if (q[t] == 0.0) {
            if (!(x0[t] > 0.0 && x0[t] < (double)N[t])) return 0;
            continue;
        }
        double ua = (0.0 - x0[t]) / q[t];
        double ub = ((double)N[t] - x0[t]) / q[t];
        if (ua > ub) { double s = ua; ua = ub; ub = s; }
        if (ua > lo) lo = ua;
        if (ub < hi) hi = ub;
    }
    if (hi - lo <= ORC_TIE) return 0;
    *u0 = lo;
    *u1 = hi;
    return 1;
}

/* Lattice index range that can contain rays meeting the box (generous). */
static void lattice_range(const frame_t *f, long *jlo, long *jhi, long *klo, long *khi)
{
    double sb = f->qb * f->Na, sc = f->qc * f->Na;
    *jlo = (long)floor(-0.5 - (sb > 0 ? sb : 0.0)) - 1;
    *jhi = (long)ceil((double)f->Nb - 0.5 - (sb < 0 ? sb : 0.0)) + 1;
    *klo = (long)floor(-0.5 - (sc > 0 ? sc : 0.0)) - 1;
    *khi = (long)ceil((double)f->Nc - 0.5 - (sc < 0 ? sc : 0.0)) + 1;
}

static long cell_index(const frame_t *f, long ia, long ib, long ic)
{
    long x[3];
    x[f->a] = ia;
    x[f->b] = ib;
    x[f->c] = ic;
    return (x[2] * f->dims[1] + x[1]) * f->dims[0] + x[0];
}

static long clampl(long v, long lo, long hi) { return v < lo ? lo : (v > hi ? hi : v); }

/* phi(x) = (1 - e^-x)/x with phi(0) = 1: the path-averaged attenuation of a
 * segment of optical depth x (Sec. 2.2, the equation after Eq. (rt)). */
static double phi_of(double x) { return x > 0.0 ? -expm1(-x) / x : 1.0; }

/* March one ray from where it enters the box to where it leaves.  For each
 * segment (a maximal piece inside one cell, length > 0) the callback receives
 * the cell index and the path length ds, in order along n. */
typedef void (*seg_fn)(void *ctx, long cell, double ds);

static int march_ray(const frame_t *f, long j, long k, seg_fn fn, void *ctx)
{
    double u0, u1;
    if (!ray_u_range(f, j, k, &u0, &u1)) return 0;
    const double xb0 = (double)j + 0.5, xc0 = (double)k + 0.5;
    const double q[2] = {f->qb, f->qc};
    const double x0[2] = {xb0, xc0};
    /* next crossing parameter per axis: a-planes sit at integer u */
    double pa = floor(u0 + ORC_TIE) + 1.0;
    double plane[2], un[2];
    for (int t = 0; t < 2; t++) {
        double x = x0[t] + q[t] * u0;
        if (q[t] > 0.0) {
            plane[t] = floor(x + ORC_TIE) + 1.0;
            un[t] = (plane[t] - x0[t]) / q[t];
        } else if (q[t] < 0.0) {
            plane[t] = ceil(x - ORC_TIE) - 1.0;
            un[t] = (plane[t] - x0[t]) / q[t];
        } else {
            plane[t] = 0.0;
            un[t] = INFINITY;
        }
    }
    int nseg = 0;
    double u = u0;
    while (u < u1 - ORC_TIE) {
        double ue = u1;
        if (pa < ue) ue = pa;
        if (un[0] < ue) ue = un[0];
        if (un[1] < ue) ue = un[1];
        if (ue - u > ORC_TIE) {
            double um = 0.5 * (u + ue);
            double xa = f->sa > 0 ? um : (double)f->Na - um;
            long ia = clampl((long)floor(xa), 0, f->Na - 1);
            long ib = clampl((long)floor(x0[0] + q[0] * um), 0, f->Nb - 1);
            long ic = clampl((long)floor(x0[1] + q[1] * um), 0, f->Nc - 1);
            fn(ctx, cell_index(f, ia, ib, ic), (ue - u) / f->na);
            nseg++;
        }
        if (pa <= ue + ORC_TIE) pa += 1.0;
        for (int t = 0; t < 2; t++) {
            if (un[t] <= ue + ORC_TIE) {
                plane[t] += (q[t] > 0.0) ? 1.0 : -1.0;
                un[t] = (plane[t] - x0[t]) / q[t];
            }
        }
        u = ue;
    }
    return nseg;
}

/* ------------------------------------------------------------------------ */
/* One direction of the sweep.                                               */
/* ------------------------------------------------------------------------ */
typedef struct {
    int nx, ny, nz;
    int nside;
    double tie_tol;
    int field_form;   /* 0: (kappa, S) inputs; 1: (kappa, emissivity) inputs */
    int nthreads;
    double i_bc;      /* intensity of every ray where it enters the box (0: vacuum) */
    int averaging;    /* 0: the paper's cell average (J = J^in + S); 1: the exact path average */
} orc_sweep_cfg;

typedef struct {
    const double *kappa, *src;  /* per cell: kappa per cell width; S or eps*dx */
    int form;
    int exact;                  /* exact path average instead of the paper's */
    double I;                   /* running intensity along the ray */
    double *A, *W;              /* per-cell accumulators of this direction */
    /* optional per-segment record */
    long *cells;
    double *ds, *Iin;
    int maxseg, nrec;
    long only_cell;             /* >= 0: accumulate A, W for this cell only */
    long long nseg;             /* segments marched */
} ray_ctx;

/* Eq. (rt) for one segment, with the path-averaged incoming intensity
 * Ibar_in = I_in (1 - e^-dtau)/dtau deposited with weight dtau; since kappa is
 * constant inside a cell, the dtau weights of Eq. (averaged_intensity) equal
 * ds weights, so A accumulates ds * Ibar_in and W accumulates ds. */
static void seg_update(void *vctx, long cell, double ds)
{
    ray_ctx *r = (ray_ctx *)vctx;
    const double kap = r->kappa[cell];
    const double x = kap * ds;
    const double e = exp(-x);
    const double ph = phi_of(x);
    const double Iin = r->I;
    if (r->A && (r->only_cell < 0 || r->only_cell == cell)) {
        /* paper: ds Ibar_in = ds I_in phi.  Exact: the path average of I over
         * the segment, S + (I_in - S) phi, less S (source-function inputs),
         * or in full, ds I_in phi + eps ds^2 psi with psi = (1 - phi)/x
         * (emissivity inputs, where kappa may vanish). */
        double dep = ds * Iin * ph;
        if (r->exact) {
            if (r->form == 0) {
                dep = ds * (Iin - r->src[cell]) * ph;
            } else {
                const double psi = x < 1e-3 ? 0.5 - x / 6.0 + x * x / 24.0 - x * x * x / 120.0
                                            : (x + expm1(-x)) / (x * x);
                dep += r->src[cell] * ds * ds * psi;
            }
        }
        r->A[r->only_cell < 0 ? cell : 0] += dep;
        r->W[r->only_cell < 0 ? cell : 0] += ds;
    }
    if (r->cells && r->nrec < r->maxseg) {
        r->cells[r->nrec] = cell;
        r->ds[r->nrec] = ds;
        r->Iin[r->nrec] = Iin;
    }
    r->nrec++;
    r->nseg++;
    if (r->form == 0) {
        const double S = r->src[cell];
        r->I = S + (Iin - S) * e;                 /* Eq. (rt) */
    } else {
        r->I = Iin * e + r->src[cell] * ds * ph;  /* Eq. (rt) with S = eps/kappa */
    }
}

static void make_frame(const orc_sweep_cfg *cfg, int d, frame_t *f)
{
    double n[3];
    const int dims[3] = {cfg->nx, cfg->ny, cfg->nz};
    orc_healpix_vec(cfg->nside, d, n);
    frame_of(dims, n, cfg->tie_tol, f);
}

/* Accumulate A (sum of ds * Ibar_in) and W (sum of ds) of direction d over
 * every ray of its family. */
static long long sweep_dir(const orc_sweep_cfg *cfg, const double *kappa, const double *src, int d,
                           double *A, double *W)
{
    frame_t f;
    make_frame(cfg, d, &f);
    long jlo, jhi, klo, khi;
    lattice_range(&f, &jlo, &jhi, &klo, &khi);
    ray_ctx r;
    memset(&r, 0, sizeof r);
    r.kappa = kappa;
    r.src = src;
    r.form = cfg->field_form;
    r.exact = cfg->averaging;
    r.A = A;
    r.W = W;
    r.only_cell = -1;
    for (long k = klo; k <= khi; k++)
        for (long j = jlo; j <= jhi; j++) {
            r.I = cfg->i_bc;   /* boundary intensity entering the box (0: vacuum) */
            march_ray(&f, j, k, seg_update, &r);
        }
    return r.nseg;
}

int orc_sweep_dir(const orc_sweep_cfg *cfg, const double *kappa, const double *src, int d,
                  double *A, double *W)
{
    long ncell = (long)cfg->nx * cfg->ny * cfg->nz;
    if (d < 0 || d >= orc_n_dirs(cfg->nside)) return -1;
    memset(A, 0, sizeof(double) * ncell);
    memset(W, 0, sizeof(double) * ncell);
    sweep_dir(cfg, kappa, src, d, A, W);
    return 0;
}

/* Sum over directions d0 <= d < d1, in RING order, of the per-cell average
 * incoming intensity A/W of Eq. (averaged_intensity) (not yet divided by N_d).
 * Returns the number of (cell, direction) pairs with W = 0 (expected: 0). */
long orc_sweep_range_count(const orc_sweep_cfg *cfg, const double *kappa, const double *src,
                           int d0, int d1, double *acc, long long *nseg)
{
    const long ncell = (long)cfg->nx * cfg->ny * cfg->nz;
    int nt = cfg->nthreads > 0 ? cfg->nthreads : 1;
    double *buf = (double *)malloc(sizeof(double) * ncell * 2 * (size_t)nt);
    if (!buf) return -1;
    long nzero = 0;
    long long segs = 0;
    memset(acc, 0, sizeof(double) * ncell);
    for (int dc = d0; dc < d1; dc += nt) {
        int cnt = (d1 - dc) < nt ? (d1 - dc) : nt;
#ifdef _OPENMP
#pragma omp parallel for schedule(static, 1) num_threads(nt) reduction(+ : segs)
#endif
        for (int t = 0; t < cnt; t++) {
            double *A = buf + (size_t)2 * t * ncell, *W = A + ncell;
            memset(A, 0, sizeof(double) * ncell * 2);
            segs += sweep_dir(cfg, kappa, src, dc + t, A, W);
        }
        for (int t = 0; t < cnt; t++) {
            const double *A = buf + (size_t)2 * t * ncell, *W = A + ncell;
            for (long i = 0; i < ncell; i++) {
                if (W[i] > 0.0) acc[i] += A[i] / W[i];
                else nzero++;
            }
        }
    }
    free(buf);
    if (nseg) *nseg = segs;
    return nzero;
}

long orc_sweep_range(const orc_sweep_cfg *cfg, const double *kappa, const double *src,
                     int d0, int d1, double *acc)
{
    return orc_sweep_range_count(cfg, kappa, src, d0, d1, acc, NULL);
}

/* Full sweep, Eq. (mean_intensity): J^in = (1/N_d) sum_i Ibar^{ave,in}(n_i),
 * J = J^in + S.  With emissivity inputs S = eps/kappa where kappa > 0; where
 * kappa = 0 only J^in is defined and J = J^in is returned.  Exact averaging:
 * with source-function inputs the sum is of (I_in - S) phi, so again
 * J = J^in + S; with emissivity inputs it is of the whole path average, so
 * J is the sum and J^in = J - S (J where kappa = 0). */
long orc_sweep(const orc_sweep_cfg *cfg, const double *kappa, const double *src,
               double *Jin, double *J)
{
    const long ncell = (long)cfg->nx * cfg->ny * cfg->nz;
    const int nd = orc_n_dirs(cfg->nside);
    long nzero = orc_sweep_range(cfg, kappa, src, 0, nd, Jin);
    if (nzero < 0) return nzero;
    for (long i = 0; i < ncell; i++) Jin[i] /= (double)nd;
    const int whole = cfg->averaging == 1 && cfg->field_form == 1;   /* Jin holds J */
    for (long i = 0; i < ncell; i++) {
        double S = src[i];
        if (cfg->field_form == 1) S = kappa[i] > 0.0 ? src[i] / kappa[i] : 0.0;
        if (whole) {
            if (J) J[i] = Jin[i];
            Jin[i] -= S;
        } else if (J) {
            J[i] = Jin[i] + S;
        }
    }
    return nzero;
}

/* Lattice description of direction d (for tests that enumerate rays). */
int orc_lattice(const orc_sweep_cfg *cfg, int d, long *range4, int *axes4, double *q3)
{
    frame_t f;
    if (d < 0 || d >= orc_n_dirs(cfg->nside)) return -1;
    make_frame(cfg, d, &f);
    lattice_range(&f, &range4[0], &range4[1], &range4[2], &range4[3]);
    axes4[0] = f.a;
    axes4[1] = f.b;
    axes4[2] = f.c;
    axes4[3] = f.sa;
    q3[0] = f.qb;
    q3[1] = f.qc;
    q3[2] = f.na;
    return 0;
}

/* Trace one lattice ray (j, k) of direction d.  Records up to maxseg segments
 * (cell, ds, incoming intensity) and returns the number of segments, the exit
 * intensity in *I_exit. */
int orc_trace_ray(const orc_sweep_cfg *cfg, const double *kappa, const double *src, int d,
                  long j, long k, long *cells, double *ds, double *Iin, int maxseg,
                  double *I_exit)
{
    frame_t f;
    if (d < 0 || d >= orc_n_dirs(cfg->nside)) return -1;
    make_frame(cfg, d, &f);
    ray_ctx r;
    memset(&r, 0, sizeof r);
    r.kappa = kappa;
    r.src = src;
    r.form = cfg->field_form;
    r.exact = cfg->averaging;
    r.cells = cells;
    r.ds = ds;
    r.Iin = Iin;
    r.maxseg = maxseg;
    r.only_cell = -1;
    r.I = cfg->i_bc;
    march_ray(&f, j, k, seg_update, &r);
    if (I_exit) *I_exit = r.I;
    return r.nrec;
}

/* J^in at selected cells, computed one by one: for every direction, every ray
 * of the family that can pass through the cell is traced from its entry point
 * and only its segment in that cell is kept. */
int orc_jin_cells(const orc_sweep_cfg *cfg, const double *kappa, const double *src,
                  const long *cells, int ncells, double *Jin)
{
    const int nd = orc_n_dirs(cfg->nside);
    const int dims[3] = {cfg->nx, cfg->ny, cfg->nz};
    int nt = cfg->nthreads > 0 ? cfg->nthreads : 1;
    int bad = 0;
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 1) num_threads(nt) reduction(+ : bad)
#endif
    for (int ci = 0; ci < ncells; ci++) {
        long cell = cells[ci];
        long x[3];
        x[0] = cell % dims[0];
        x[1] = (cell / dims[0]) % dims[1];
        x[2] = cell / ((long)dims[0] * dims[1]);
        double sum = 0.0;
        for (int d = 0; d < nd; d++) {
            frame_t f;
            make_frame(cfg, d, &f);
            /* u-interval of the cell along the ray family */
            double ucell = f.sa > 0 ? (double)x[f.a] : (double)(f.Na - 1 - x[f.a]);
            long jr[2], kr[2];
            const double qq[2] = {f.qb, f.qc};
            const long pc[2] = {x[f.b], x[f.c]};
            long *rr[2] = {jr, kr};
            for (int t = 0; t < 2; t++) {
                double s0 = qq[t] * ucell, s1 = qq[t] * (ucell + 1.0);
                double smin = s0 < s1 ? s0 : s1, smax = s0 < s1 ? s1 : s0;
                rr[t][0] = (long)floor((double)pc[t] - 0.5 - smax) - 1;
                rr[t][1] = (long)ceil((double)pc[t] + 0.5 - smin) + 1;
            }
            double A = 0.0, W = 0.0;
            ray_ctx r;
            memset(&r, 0, sizeof r);
            r.kappa = kappa;
            r.src = src;
            r.form = cfg->field_form;
            r.exact = cfg->averaging;
            r.A = &A;
            r.W = &W;
            r.only_cell = cell;
            for (long k = kr[0]; k <= kr[1]; k++)
                for (long j = jr[0]; j <= jr[1]; j++) {
                    r.I = cfg->i_bc;
                    march_ray(&f, j, k, seg_update, &r);
                }
            if (W > 0.0) sum += A / W;
            else bad++;
        }
        Jin[ci] = sum / (double)nd;
        if (cfg->averaging == 1 && cfg->field_form == 1 && kappa[cell] > 0.0)
            Jin[ci] -= src[cell] / kappa[cell];   /* the sum was the whole path average */
    }
    return bad;
}

/* ------------------------------------------------------------------------ */
/* Diffuse photo-ionization rate, Eq. (gamma_diff): the incoming part        */
/* 4 pi Jcal^in * int_{nu0}^{nu0+dnu} sigma(nu)/(h nu) dnu.                  */
/* sigma(nu) = sigma0 (nu/nu0)^-3 (hydrogenic threshold power law), so the  */
/* band integral has the closed form sigma0 nu0^3/(3h) (nu0^-3 - nu1^-3).    */
/* ------------------------------------------------------------------------ */
double orc_band_integral(double sigma0, double h, double nu0, double nu1)
{
    return sigma0 * nu0 * nu0 * nu0 / (3.0 * h) * (1.0 / (nu0 * nu0 * nu0) - 1.0 / (nu1 * nu1 * nu1));
}

/* ------------------------------------------------------------------------ */
/* Point sources: long characteristics, photon-conserving rate (Sec. 2.1,   */
/* App. A).  For each target cell and source, the ray from the source to    */
/* the cell centre is marched; tau sums kappa*ds over the cells before the  */
/* target cell, [r_in, r_out] is the ray's passage through the target cell  */
/* (r_in = 0 in the source's own cell).  Per bin b:                          */
/*   Ndot_abs = Q_b e^-tau (1 - e^-dtau),  dtau = kappa_b (r_out - r_in),    */
/*   Gamma   += Ndot_abs / (n_HI * 4pi/3 (r_out^3 - r_in^3) dx^3)            */
/* with n_HI = kappa_b/(sigma_b dx), written without the division by n_HI:   */
/*   Gamma += Q_b e^-tau sigma_b (r_out - r_in) phi(dtau)                    */
/*            / (4pi/3 (r_out^3 - r_in^3) dx^2).                             */
/* Positions are in cell widths, box [0, n]^3.                               */
/* ------------------------------------------------------------------------ */
static double pt_one(const int dims[3], const double *kappa_bins, long ncell, int nbins,
                     const double *sigma, const double *Qb, const double s[3], long target,
                     double dx)
{
    long tx = target % dims[0], ty = (target / dims[0]) % dims[1], tz = target / ((long)dims[0] * dims[1]);
    double c[3] = {tx + 0.5, ty + 0.5, tz + 0.5};
    double dvec[3] = {c[0] - s[0], c[1] - s[1], c[2] - s[2]};
    double L = sqrt(dvec[0] * dvec[0] + dvec[1] * dvec[1] + dvec[2] * dvec[2]);
    double n[3];
    if (L < 1e-12) { n[0] = 1.0; n[1] = 0.0; n[2] = 0.0; }
    else { n[0] = dvec[0] / L; n[1] = dvec[1] / L; n[2] = dvec[2] / L; }
    /* the first cell is the one containing s + 1e-9 n */
    long cur[3];
    for (int i = 0; i < 3; i++) {
        double p = s[i] + 1e-9 * n[i];
        long v = (long)floor(p);
        cur[i] = v < 0 ? 0 : (v >= dims[i] ? dims[i] - 1 : v);
    }
    double tnext[3], step[3];
    for (int i = 0; i < 3; i++) {
        if (n[i] > 1e-300) { tnext[i] = ((double)(cur[i] + 1) - s[i]) / n[i]; step[i] = 1.0 / n[i]; }
        else if (n[i] < -1e-300) { tnext[i] = ((double)cur[i] - s[i]) / n[i]; step[i] = -1.0 / n[i]; }
        else { tnext[i] = INFINITY; step[i] = INFINITY; }
    }
    double tau_buf[16];
    double *tau = nbins <= 16 ? tau_buf : (double *)calloc(nbins, sizeof(double));
    for (int b = 0; b < nbins; b++) tau[b] = 0.0;
    double t = 0.0, gamma = 0.0;
    for (;;) {
        double te = tnext[0];
        if (tnext[1] < te) te = tnext[1];
        if (tnext[2] < te) te = tnext[2];
        long cidx = (cur[2] * dims[1] + cur[1]) * dims[0] + cur[0];
        if (cidx == target) {
            double rin = t, rout = te;
            double vol = 4.0 * M_PI / 3.0 * (rout * rout * rout - rin * rin * rin);
            for (int b = 0; b < nbins; b++) {
                double dtau = kappa_bins[(size_t)b * ncell + cidx] * (rout - rin);
                gamma += Qb[b] * exp(-tau[b]) * sigma[b] * (rout - rin) * phi_of(dtau) / (vol * dx * dx);
            }
            break;
        }
        for (int b = 0; b < nbins; b++) tau[b] += kappa_bins[(size_t)b * ncell + cidx] * (te - t);
        /* advance every axis whose crossing coincides with te */
        int moved = 0;
        for (int i = 0; i < 3; i++) {
            if (tnext[i] <= te + 1e-12) {
                cur[i] += n[i] > 0 ? 1 : -1;
                tnext[i] += step[i];
                moved = 1;
            }
        }
        t = te;
        if (!moved || cur[0] < 0 || cur[1] < 0 || cur[2] < 0 || cur[0] >= dims[0] || cur[1] >= dims[1] ||
            cur[2] >= dims[2])
            break;   /* cannot happen for a target inside the box */
    }
    if (tau != tau_buf) free(tau);
    return gamma;
}

int orc_point_sources(int nx, int ny, int nz, int nbins, const double *kappa_bins, const double *sigma,
                      int nsrc, const double *pos, const double *Q, double dx, int nthreads,
                      double *gamma)
{
    const int dims[3] = {nx, ny, nz};
    const long ncell = (long)nx * ny * nz;
    int nt = nthreads > 0 ? nthreads : 1;
    (void)nt;
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 64) num_threads(nt)
#endif
    for (long i = 0; i < ncell; i++) {
        double g = 0.0;
        for (int a = 0; a < nsrc; a++)
            g += pt_one(dims, kappa_bins, ncell, nbins, sigma, Q + (size_t)a * nbins, pos + 3 * a, i, dx);
        gamma[i] = g;
    }
    return 0;
}

/* The same rates at selected target cells only (flat indices). */
int orc_point_sources_cells(int nx, int ny, int nz, int nbins, const double *kappa_bins, const double *sigma,
                            int nsrc, const double *pos, const double *Q, double dx, const long *cells,
                            int ncells, double *gamma)
{
    const int dims[3] = {nx, ny, nz};
    const long ncell = (long)nx * ny * nz;
    for (int c = 0; c < ncells; c++) {
        if (cells[c] < 0 || cells[c] >= ncell) return -1;
        double g = 0.0;
        for (int a = 0; a < nsrc; a++)
            g += pt_one(dims, kappa_bins, ncell, nbins, sigma, Q + (size_t)a * nbins, pos + 3 * a, cells[c], dx);
        gamma[c] = g;
    }
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Plane-parallel incident flux (the Test-3 setup of Sec. 4.3: a constant    */
/* photon flux F through one face of the box, i.e. a point source at         */
/* infinity).  The beam travels along +axis (dir = +1, entering at the face  */
/* coordinate 0) or -axis (dir = -1).  In bin b, the photons absorbed in a   */
/* cell per unit time are F_b dx^2 e^-tau (1 - e^-dtau), tau summing kappa_b */
/* over the cells before it along the beam and dtau = kappa_b of the cell;   */
/* per neutral atom (n_HI dx^3 = kappa_b dx^2 / sigma_b):                    */
/*   Gamma += F_b sigma_b e^-tau (1 - e^-dtau) / dtau.                       */
/* ------------------------------------------------------------------------ */
int orc_plane_source(int nx, int ny, int nz, int nbins, const double *kappa_bins, const double *sigma,
                     int axis, int dir, const double *F, double *gamma)
{
    const int dims[3] = {nx, ny, nz};
    const long stride[3] = {1, nx, (long)nx * ny};
    const long ncell = (long)nx * ny * nz;
    if (axis < 0 || axis > 2 || (dir != 1 && dir != -1)) return -1;
    const int u = axis == 0 ? 1 : 0, v = axis == 2 ? 1 : 2;   /* the two transverse axes */
    for (long i = 0; i < ncell; i++) gamma[i] = 0.0;
    for (int b = 0; b < nbins; b++) {
        const double *kap = kappa_bins + (size_t)b * ncell;
        for (int q = 0; q < dims[v]; q++)
            for (int p = 0; p < dims[u]; p++) {
                double tau = 0.0;
                for (int m = 0; m < dims[axis]; m++) {
                    const int a = dir > 0 ? m : dims[axis] - 1 - m;
                    const long cell = a * stride[axis] + p * stride[u] + q * stride[v];
                    const double dtau = kap[cell];
                    gamma[cell] += F[b] * sigma[b] * exp(-tau) * phi_of(dtau);
                    tau += dtau;
                }
            }
    }
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Ionization balance (App. B), hydrogen only, in the dt -> infinity limit:  */
/*   alpha_A n_e n_HII = n_HI (Gamma_coll n_e + Gamma_gamma),                */
/* Gamma_gamma = Gamma_point + Gamma^diff and Gamma^diff carries the local   */
/* term Delta_alpha n_e n_HII / n_HI of Eq. (gamma_diff).  Taking that term  */
/* at the same state as the rest, it moves to the left side and leaves       */
/*   alpha_B n_e n_HII = n_HI (Gamma_coll n_e + g),  g = non-local rates.    */
/* With n_HI = y n_H and n_e = n_HII = (1 - y) n_H, a = alpha_B n_H,         */
/* c = Gamma_coll n_H:  (a + c) y^2 - (2a + c + g) y + a = 0, whose root in  */
/* [0, 1] is y = 2a / (2a + c + g + sqrt(4 a g + (c + g)^2)) (no            */
/* cancellation: the neutral fraction y is computed directly).              */
/* ------------------------------------------------------------------------ */
void orc_balance_eq(long ncell, const double *nH, double alphaB, double gcoll, const double *g,
                    double *y)
{
    for (long i = 0; i < ncell; i++) {
        double a = alphaB * nH[i], c = gcoll * nH[i], gg = g[i];
        double disc = 4.0 * a * gg + (c + gg) * (c + gg);
        y[i] = (a > 0.0) ? 2.0 * a / (2.0 * a + c + gg + sqrt(disc)) : 0.0;
    }
}

/* ------------------------------------------------------------------------ */
/* RT / ionization-balance fixed-point iteration (App. D): repeat            */
/*   kappa = n_HI sigma0 dx,  eps = h nu0 dalpha n_e n_HII dx/(4 pi dnu)      */
/*   (Eq. for eps_nu/(h nu) with the rectangular spectrum, at nu0),          */
/*   J^in from the sweep (monochromatic at nu0, paper averaging),            */
/*   g = 4 pi G J^in + Gamma_point,  y <- balance,                           */
/* until max_cells |n_e^(i) - n_e^(i-1)| / n_e^(i) < tol.                    */
/* ------------------------------------------------------------------------ */
typedef struct {
    double alphaA, alphaB, gcoll;   /* cm^3/s at the (fixed) temperature */
    double sigma0;                  /* cm^2 at nu0 */
    double h, nu0, dnu;             /* erg s, Hz, Hz (dnu = k_B T / h) */
    double dx;                      /* cell width, cm */
} orc_chem;

int orc_iterate_bins(const orc_sweep_cfg *cfg, const orc_chem *ch, const double *nH, int nsrc,
                     const double *pos, const double *Q, int nb, const double *sigma_b,
                     const double *frac_b, double tol, int max_iter, double *y,
                     double *resid_hist, int *iters);
int orc_iterate_ext(const orc_sweep_cfg *cfg, const orc_chem *ch, const double *nH, int nsrc,
                    const double *pos, const double *Q, int nb, const double *sigma_b,
                    const double *frac_b, int pl_axis, int pl_dir, double pl_flux, double tol,
                    int max_iter, double *y, double *resid_hist, int *iters);

int orc_iterate(const orc_sweep_cfg *cfg, const orc_chem *ch, const double *nH, int nsrc,
                const double *pos, const double *Q, double tol, int max_iter, double *y,
                double *resid_hist, int *iters)
{
    const double one = 1.0;
    return orc_iterate_bins(cfg, ch, nH, nsrc, pos, Q, 1, &ch->sigma0, &one, tol, max_iter, y,
                            resid_hist, iters);
}

/* The iteration with point sources over nb frequency bins (App. A, Eq.
 * pc_gamma summed over bins): source a emits Q_a frac_b photons/s in bin b,
 * absorbed with cross section sigma_b (kappa_b = n_HI sigma_b dx); the
 * diffuse recombination field stays the band [nu0, nu0 + dnu] at sigma0. */
int orc_iterate_bins(const orc_sweep_cfg *cfg, const orc_chem *ch, const double *nH, int nsrc,
                     const double *pos, const double *Q, int nb, const double *sigma_b,
                     const double *frac_b, double tol, int max_iter, double *y,
                     double *resid_hist, int *iters)
{
    return orc_iterate_ext(cfg, ch, nH, nsrc, pos, Q, nb, sigma_b, frac_b, 0, 1, 0.0, tol, max_iter, y,
                           resid_hist, iters);
}

/* ... and, with pl_flux > 0, a plane-parallel incident flux of pl_flux
 * photons/s/cm^2 along axis pl_axis in direction pl_dir, split over the bins
 * like the point sources' photons (frac_b). */
int orc_iterate_ext(const orc_sweep_cfg *cfg, const orc_chem *ch, const double *nH, int nsrc,
                    const double *pos, const double *Q, int nb, const double *sigma_b,
                    const double *frac_b, int pl_axis, int pl_dir, double pl_flux, double tol,
                    int max_iter, double *y, double *resid_hist, int *iters)
{
    const long ncell = (long)cfg->nx * cfg->ny * cfg->nz;
    double *kap = (double *)malloc(sizeof(double) * ncell);
    double *kapb = (double *)malloc(sizeof(double) * ncell * nb);
    double *qb = (double *)malloc(sizeof(double) * (nsrc > 0 ? nsrc : 1) * nb);
    double *eps = (double *)malloc(sizeof(double) * ncell);
    double *jin = (double *)malloc(sizeof(double) * ncell);
    double *gpt = (double *)malloc(sizeof(double) * ncell);
    double *g = (double *)malloc(sizeof(double) * ncell);
    double *yn = (double *)malloc(sizeof(double) * ncell);
    double *gpl = (double *)malloc(sizeof(double) * ncell);
    double *fb = (double *)malloc(sizeof(double) * nb);
    if (!kap || !kapb || !qb || !eps || !jin || !gpt || !g || !yn || !gpl || !fb) return -1;
    for (int b = 0; b < nb; b++) fb[b] = pl_flux * frac_b[b];
    for (int a = 0; a < nsrc; a++)
        for (int b = 0; b < nb; b++) qb[a * nb + b] = Q[a] * frac_b[b];
    orc_sweep_cfg c = *cfg;
    c.field_form = 1;
    const double dalpha = ch->alphaA - ch->alphaB;
    const double G = orc_band_integral(ch->sigma0, ch->h, ch->nu0, ch->nu0 + ch->dnu);
    int it = 0, conv = 0;
    for (it = 1; it <= max_iter; it++) {
        for (long i = 0; i < ncell; i++) {
            double nHI = y[i] * nH[i], ne = (1.0 - y[i]) * nH[i];
            kap[i] = nHI * ch->sigma0 * ch->dx;
            eps[i] = ch->h * ch->nu0 * dalpha * ne * ne * ch->dx / (4.0 * M_PI * ch->dnu);
        }
        orc_sweep(&c, kap, eps, jin, NULL);
        for (int b = 0; b < nb; b++)
            for (long i = 0; i < ncell; i++) kapb[b * ncell + i] = y[i] * nH[i] * sigma_b[b] * ch->dx;
        orc_point_sources(cfg->nx, cfg->ny, cfg->nz, nb, kapb, sigma_b, nsrc, pos, qb, ch->dx, cfg->nthreads, gpt);
        if (pl_flux > 0.0) {
            if (orc_plane_source(cfg->nx, cfg->ny, cfg->nz, nb, kapb, sigma_b, pl_axis, pl_dir, fb, gpl) != 0)
                return -1;
            for (long i = 0; i < ncell; i++) gpt[i] += gpl[i];
        }
        for (long i = 0; i < ncell; i++) g[i] = 4.0 * M_PI * G * jin[i] + gpt[i];
        orc_balance_eq(ncell, nH, ch->alphaB, ch->gcoll, g, yn);
        double r = 0.0;
        for (long i = 0; i < ncell; i++) {
            double ne_new = (1.0 - yn[i]) * nH[i], ne_old = (1.0 - y[i]) * nH[i];
            double ri = fabs(ne_new - ne_old) / ne_new;
            if (ri > r) r = ri;
            y[i] = yn[i];
        }
        if (resid_hist) resid_hist[it - 1] = r;
        if (r < tol) { conv = 1; break; }
    }
    if (iters) *iters = conv ? it : max_iter;
    free(kap); free(kapb); free(qb); free(eps); free(jin); free(gpt); free(g); free(yn); free(gpl); free(fb);
    return conv ? 0 : 1;
}

/* ------------------------------------------------------------------------ */
/* Time-dependent mode (App. B-D), hydrogen only, at the fixed temperature   */
/* of the chemistry constants.                                              */
/*                                                                          */
/* One cell over dt at fixed photo-ionization rate g (App. B): the BDF step */
/*   n_HI <- (C dtc + n_HI) / (1 + D dtc),  C = alpha_B n_e n_HII,          */
/*   D = Gamma_coll n_e + g,  n_e = n_HII = n_H - n_HI,                     */
/* with C and D taken at the start of the sub-step (hydrogen is the lowest  */
/* ionization level, updated first), sub-cycled with the chemical timestep  */
/* of App. D, dtc = eps_e |n_e / n_e'| + eps_HI |n_HI / n_HI'|, the last    */
/* sub-step cut to end at dt.  alpha_B because the local recombination term */
/* of Eq. (gamma_diff) cancels the ground-state recombinations, as in the   */
/* equilibrium balance; g holds the non-local rates.                        */
/* ------------------------------------------------------------------------ */
static double dtchem_cell(double nH, double y, double alphaB, double gcoll, double g, double eps_e,
                          double eps_hi)
{
    const double nHI = y * nH, ne = (1.0 - y) * nH;
    const double dHI = alphaB * ne * ne - (gcoll * ne + g) * nHI;   /* dn_HI/dt = -dn_e/dt */
    if (dHI == 0.0) return INFINITY;
    return eps_e * fabs(ne / dHI) + eps_hi * fabs(nHI / dHI);
}

static int chem_cell(double nH, double y0, double alphaB, double gcoll, double g, double dt, double eps_e,
                     double eps_hi, int max_sub, double *y_out)
{
    double y = y0, tau = 0.0;
    int n = 0;
    while (tau < dt && n < max_sub) {
        const double nHI = y * nH, ne = (1.0 - y) * nH;
        const double C = alphaB * ne * ne, D = gcoll * ne + g;
        double dtc = dtchem_cell(nH, y, alphaB, gcoll, g, eps_e, eps_hi);
        const int last = !(dtc < dt - tau);
        if (last) dtc = dt - tau;
        y = (C * dtc + nHI) / (1.0 + D * dtc) / nH;
        if (y > 1.0) y = 1.0;
        tau = last ? dt : tau + dtc;
        n++;
    }
    *y_out = y;
    return n;
}

typedef struct {
    double F;          /* Delta t = F min_i Delta t_chem,i (App. D) */
    double eps_iter;   /* n_e convergence of the RT / chemistry iteration per step */
    double eps_e, eps_hi;
    double dt_fixed;   /* > 0: every step is dt_fixed instead */
    int max_steps, max_iter, max_sub;
} orc_evolve_opt;

/* Photo-ionization rates g of state y: point sources (+ plane flux) over the
 * bins and 4 pi G J^in from the sweep of the state's emissivity. */
static void rates_of(const orc_sweep_cfg *cfg, const orc_chem *ch, const double *nH, const double *y,
                     int nsrc, const double *pos, const double *qb, int nb, const double *sigma_b,
                     int pl_axis, int pl_dir, double pl_flux, const double *fb, double G,
                     double *kap, double *kapb, double *eps, double *jin, double *gpt, double *gpl, double *g)
{
    const long ncell = (long)cfg->nx * cfg->ny * cfg->nz;
    orc_sweep_cfg c = *cfg;
    c.field_form = 1;
    const double dalpha = ch->alphaA - ch->alphaB;
    for (long i = 0; i < ncell; i++) {
        double nHI = y[i] * nH[i], ne = (1.0 - y[i]) * nH[i];
        kap[i] = nHI * ch->sigma0 * ch->dx;
        eps[i] = ch->h * ch->nu0 * dalpha * ne * ne * ch->dx / (4.0 * M_PI * ch->dnu);
    }
    orc_sweep(&c, kap, eps, jin, NULL);
    for (int b = 0; b < nb; b++)
        for (long i = 0; i < ncell; i++) kapb[b * ncell + i] = y[i] * nH[i] * sigma_b[b] * ch->dx;
    orc_point_sources(cfg->nx, cfg->ny, cfg->nz, nb, kapb, sigma_b, nsrc, pos, qb, ch->dx, cfg->nthreads, gpt);
    if (pl_flux > 0.0) {
        orc_plane_source(cfg->nx, cfg->ny, cfg->nz, nb, kapb, sigma_b, pl_axis, pl_dir, fb, gpl);
        for (long i = 0; i < ncell; i++) gpt[i] += gpl[i];
    }
    for (long i = 0; i < ncell; i++) g[i] = 4.0 * M_PI * G * jin[i] + gpt[i];
}

/* Evolve y from t = 0 to t_end in RT steps: the rates of the state at t
 * give Delta t; then iterate {chemistry of every cell over Delta t from the
 * state at t, at the rates of the current iterate; the rates of the new
 * iterate} until max |n_e^(i) - n_e^(i-1)| / n_e^(i) < eps_iter (App. D).
 * Returns 0 when t_end is reached with every step converged, 1 if an
 * iteration hit max_iter (the last iterate is kept), 2 if max_steps ran out
 * first, -1 on allocation failure. */
int orc_evolve(const orc_sweep_cfg *cfg, const orc_chem *ch, const double *nH, int nsrc, const double *pos,
               const double *Q, int nb, const double *sigma_b, const double *frac_b, int pl_axis, int pl_dir,
               double pl_flux, const orc_evolve_opt *opt, double t_end, double *y, int *steps_out,
               int *iters_out, double *t_out, double *dt_hist)
{
    const long ncell = (long)cfg->nx * cfg->ny * cfg->nz;
    double *kap = malloc(sizeof(double) * ncell), *kapb = malloc(sizeof(double) * ncell * nb);
    double *eps = malloc(sizeof(double) * ncell), *jin = malloc(sizeof(double) * ncell);
    double *gpt = malloc(sizeof(double) * ncell), *gpl = malloc(sizeof(double) * ncell);
    double *g = malloc(sizeof(double) * ncell), *yp = malloc(sizeof(double) * ncell);
    double *yn = malloc(sizeof(double) * ncell);
    double *qb = malloc(sizeof(double) * (nsrc > 0 ? nsrc : 1) * nb), *fb = malloc(sizeof(double) * nb);
    if (!kap || !kapb || !eps || !jin || !gpt || !gpl || !g || !yp || !yn || !qb || !fb) return -1;
    for (int a = 0; a < nsrc; a++)
        for (int b = 0; b < nb; b++) qb[a * nb + b] = Q[a] * frac_b[b];
    for (int b = 0; b < nb; b++) fb[b] = pl_flux * frac_b[b];
    const double G = orc_band_integral(ch->sigma0, ch->h, ch->nu0, ch->nu0 + ch->dnu);
    double t = 0.0;
    int steps = 0, iters = 0, unconverged = 0;
    while (t < t_end && steps < opt->max_steps) {
        rates_of(cfg, ch, nH, y, nsrc, pos, qb, nb, sigma_b, pl_axis, pl_dir, pl_flux, fb, G, kap, kapb, eps,
                 jin, gpt, gpl, g);
        double dt;
        if (opt->dt_fixed > 0.0) {
            dt = opt->dt_fixed;
        } else {
            double m = INFINITY;
            for (long i = 0; i < ncell; i++) {
                const double d = dtchem_cell(nH[i], y[i], ch->alphaB, ch->gcoll, g[i], opt->eps_e, opt->eps_hi);
                if (d < m) m = d;
            }
            dt = opt->F * m;
        }
        const int last = !(dt < t_end - t);
        if (last) dt = t_end - t;
        for (long i = 0; i < ncell; i++) yp[i] = y[i];
        int conv = 0;
        for (int k = 1; k <= opt->max_iter; k++) {
            iters++;
            double r = 0.0;
            for (long i = 0; i < ncell; i++) {
                chem_cell(nH[i], y[i], ch->alphaB, ch->gcoll, g[i], dt, opt->eps_e, opt->eps_hi, opt->max_sub,
                          &yn[i]);
                const double ne_new = (1.0 - yn[i]) * nH[i], ne_old = (1.0 - yp[i]) * nH[i];
                const double ri = ne_new > 0.0 ? fabs(ne_new - ne_old) / ne_new : (ne_old > 0.0 ? INFINITY : 0.0);
                if (ri > r) r = ri;
            }
            for (long i = 0; i < ncell; i++) yp[i] = yn[i];
            if (r < opt->eps_iter) {
                conv = 1;
                break;
            }
            rates_of(cfg, ch, nH, yp, nsrc, pos, qb, nb, sigma_b, pl_axis, pl_dir, pl_flux, fb, G, kap, kapb,
                     eps, jin, gpt, gpl, g);
        }
        if (!conv) unconverged = 1;
        for (long i = 0; i < ncell; i++) y[i] = yp[i];
        if (dt_hist) dt_hist[steps] = dt;
        t = last ? t_end : t + dt;
        steps++;
    }
    if (steps_out) *steps_out = steps;
    if (iters_out) *iters_out = iters;
    if (t_out) *t_out = t;
    free(kap); free(kapb); free(eps); free(jin); free(gpt); free(gpl); free(g); free(yp); free(yn);
    free(qb); free(fb);
    if (t < t_end) return 2;
    return unconverged ? 1 : 0;
}

/* ------------------------------------------------------------------------ */
/* Energy equation (App. C) and temperature-dependent rates, hydrogen only. */
/*                                                                          */
/* The paper takes its rate and cooling coefficients from the works listed  */
/* in its rate table without printing them.  The fits used here, T in K,    */
/* lambda = 2 T_HI / T with T_HI = 157807 K (Hui & Gnedin 1997):            */
/*   alpha_A  case-A recombination   Hui & Gnedin (1997)                    */
/*   alpha_B  case-B recombination   Hui & Gnedin (1997)                    */
/*   Gamma_coll  collisional ionization of HI   Cen (1992)                  */
/*   recombination cooling, case A   Cen (1992); case B   Hui & Gnedin      */
/*   collisional ionization / excitation cooling of HI   Cen (1992)         */
/*   free-free cooling   1.42e-27 g_ff sqrt(T), g_ff of Spitzer's form      */
/*   Compton cooling off the CMB   4 sigma_T a T_g^4 k_B (T - T_g) / (m_e c) */
/*     per electron, T_g = 2.7255 (1 + z) K                                 */
/* ------------------------------------------------------------------------ */
#define ORC_T_HI 157807.0

double orc_alpha_A(double T)
{
    const double l = 2.0 * ORC_T_HI / T;
    return 1.269e-13 * pow(l, 1.503) / pow(1.0 + pow(l / 0.522, 0.470), 1.923);
}

double orc_alpha_B(double T)
{
    const double l = 2.0 * ORC_T_HI / T;
    return 2.753e-14 * pow(l, 1.500) / pow(1.0 + pow(l / 2.740, 0.407), 2.242);
}

double orc_gamma_coll(double T)
{
    return 5.85e-11 * sqrt(T) * exp(-157809.1 / T) / (1.0 + sqrt(T / 1e5));
}

/* cooling coefficients: erg cm^3 / s, times n_e n_HII (recombination,
 * free-free) or n_e n_HI (collisional ionization, excitation) */
double orc_cool_rec_A(double T) { return 8.70e-27 * sqrt(T) * pow(T / 1e3, -0.2) / (1.0 + pow(T / 1e6, 0.7)); }

double orc_cool_rec_B(double T)
{
    const double l = 2.0 * ORC_T_HI / T;
    return 3.435e-30 * T * pow(l, 1.970) / pow(1.0 + pow(l / 2.250, 0.376), 3.720);
}

double orc_cool_ci(double T) { return 1.27e-21 * sqrt(T) * exp(-157809.1 / T) / (1.0 + sqrt(T / 1e5)); }

double orc_cool_ce(double T) { return 7.50e-19 * exp(-118348.0 / T) / (1.0 + sqrt(T / 1e5)); }

double orc_cool_ff(double T)
{
    const double d = 5.5 - log10(T);
    return 1.42e-27 * (1.1 + 0.34 * exp(-d * d / 3.0)) * sqrt(T);
}

/* Compton coefficient per electron, erg/s/K: the cooling is c (T - T_g) n_e */
double orc_compton_coef(double z, double kB)
{
    const double sigma_T = 6.6524587e-25, a_rad = 7.5657e-15, m_e = 9.1093837e-28, c = 2.99792458e10;
    const double Tg = 2.7255 * (1.0 + z);
    return 4.0 * sigma_T * a_rad * Tg * Tg * Tg * Tg * kB / (m_e * c);
}

typedef struct {
    int on_the_spot;   /* alpha_A = alpha_B, no diffuse field, case-B recombination cooling */
    int cool_mask;     /* bit 0 recombination, 1 collisional ionization, 2 collisional excitation,
                          3 free-free, 4 Compton (31: all) */
    double e_bin[4];   /* mean energy above threshold per photo-ionization in source bin b, erg */
    double e_diff;     /* the same for the diffuse recombination band, erg */
    double z;          /* CMB redshift of the Compton term */
    double kB;         /* Boltzmann constant, erg/K */
    double T_min, T_max;   /* bracket of the temperature root, K */
} orc_thermal;

/* Cooling rate C(n, T), erg/s/cm^3, of hydrogen with neutral fraction y. */
double orc_cooling(const orc_thermal *th, double nH, double y, double T)
{
    const double nHI = y * nH, ne = (1.0 - y) * nH, nHII = ne;
    double c = 0.0;
    if (th->cool_mask & 1) c += (th->on_the_spot ? orc_cool_rec_B(T) : orc_cool_rec_A(T)) * ne * nHII;
    if (th->cool_mask & 2) c += orc_cool_ci(T) * ne * nHI;
    if (th->cool_mask & 4) c += orc_cool_ce(T) * ne * nHI;
    if (th->cool_mask & 8) c += orc_cool_ff(T) * ne * nHII;
    if (th->cool_mask & 16) {
        const double Tg = 2.7255 * (1.0 + th->z);
        c += orc_compton_coef(th->z, th->kB) * (T - Tg) * ne;
    }
    return c;
}

/* dC/dT of orc_cooling, from the logarithmic derivative of each fit:
 *   case-A recombination (Cen)   0.3 - 0.7 u / (1 + u),  u = (T/1e6)^0.7
 *   case-B recombination (H&G)   1 - 1.970 + 3.720 * 0.376 v / (1 + v),  v = (lambda/2.25)^0.376
 *   collisional ionization       0.5 + 157809.1/T - 0.5 w / (1 + w),  w = sqrt(T/1e5)
 *   collisional excitation       118348/T - 0.5 w / (1 + w)
 *   free-free                    0.5 + 0.34 e^{-d^2/3} (2d / (3 ln 10)) / g_ff,  d = 5.5 - log10 T
 * (d ln c / d ln T; dc/dT = c (d ln c / d ln T) / T), and the Compton term's
 * coefficient times n_e. */
double orc_cooling_deriv(const orc_thermal *th, double nH, double y, double T)
{
    const double nHI = y * nH, ne = (1.0 - y) * nH, nHII = ne;
    const double w = sqrt(T / 1e5);
    double d = 0.0;
    if (th->cool_mask & 1) {
        double c, g;
        if (th->on_the_spot) {
            const double v = pow(2.0 * ORC_T_HI / T / 2.250, 0.376);
            c = orc_cool_rec_B(T);
            g = 1.0 - 1.970 + 3.720 * 0.376 * v / (1.0 + v);
        } else {
            const double u = pow(T / 1e6, 0.7);
            c = orc_cool_rec_A(T);
            g = 0.3 - 0.7 * u / (1.0 + u);
        }
        d += c * g / T * ne * nHII;
    }
    if (th->cool_mask & 2) d += orc_cool_ci(T) * (0.5 + 157809.1 / T - 0.5 * w / (1.0 + w)) / T * ne * nHI;
    if (th->cool_mask & 4) d += orc_cool_ce(T) * (118348.0 / T - 0.5 * w / (1.0 + w)) / T * ne * nHI;
    if (th->cool_mask & 8) {
        const double dd = 5.5 - log10(T), e = 0.34 * exp(-dd * dd / 3.0);
        d += orc_cool_ff(T) * (0.5 + e * 2.0 * dd / (3.0 * log(10.0)) / (1.1 + e)) / T * ne * nHII;
    }
    if (th->cool_mask & 16) d += orc_compton_coef(th->z, th->kB) * ne;
    return d;
}

/* The implicit update of App. C for one cell over dt: the specific energy
 * u = 3 k_B T (1 + x) n_H / (2 rho) at t + dt solves
 *   u' = u + (H(n') - C(n', u')) dt / rho,
 * i.e. with e = rho u = 1.5 k_B T n_H (1 + x) (rho cancels):
 *   f(T') = 1.5 k_B n_H (1 + x') T' + dt C(n', T') - (e + H' dt) = 0.
 * Newton's method from T on f' = 1.5 k_B n_H (1 + x') + dt dC/dT, kept
 * inside the bracket its iterates build (the largest T with f < 0 and the
 * smallest with f > 0 seen so far, within [T_min, T_max]): a step that leaves
 * it, or a non-positive f', bisects the bracket once both ends are known and
 * otherwise doubles or halves T towards the sign change.  Stops when a step
 * moves T by at most 1e-12 T (Newton's error is then of order the square of
 * that), at a bound with f of the bound's sign, or after 100 steps.
 * Returns T'. */
static double energy_f(const orc_thermal *th, double nH, double y1, double A, double B, double dt, double T)
{
    return A * T + dt * orc_cooling(th, nH, y1, T) - B;
}

double orc_energy_step(const orc_thermal *th, double nH, double y0, double T0, double y1, double H1, double dt)
{
    const double A = 1.5 * th->kB * nH * (2.0 - y1);
    const double B = 1.5 * th->kB * nH * (2.0 - y0) * T0 + H1 * dt;
    double T = T0 < th->T_min ? th->T_min : (T0 > th->T_max ? th->T_max : T0);
    double lo = th->T_min, hi = th->T_max;
    int have_lo = 0, have_hi = 0;
    for (int it = 0; it < 100; it++) {
        const double f = energy_f(th, nH, y1, A, B, dt, T);
        if (f == 0.0) return T;
        if (f < 0.0) { lo = T; have_lo = 1; } else { hi = T; have_hi = 1; }
        const double fp = A + dt * orc_cooling_deriv(th, nH, y1, T);
        double Tn = fp > 0.0 ? T - f / fp : -1.0;
        if (!(Tn > lo && Tn < hi) || !(fp > 0.0)) {
            if (have_lo && have_hi) Tn = 0.5 * (lo + hi);
            else if (f < 0.0) Tn = 2.0 * T < th->T_max ? 2.0 * T : th->T_max;
            else Tn = 0.5 * T > th->T_min ? 0.5 * T : th->T_min;
        }
        if (fabs(Tn - T) <= 1e-12 * T) return Tn;   // quadratic: Tn is then exact to rounding
        T = Tn;
    }
    return T;
}

/* Chemical timestep of App. D at temperature T. */
static double dtchem_T(double nH, double y, double T, double g, double eps_e, double eps_hi)
{
    return dtchem_cell(nH, y, orc_alpha_B(T), orc_gamma_coll(T), g, eps_e, eps_hi);
}

/* One cell over dt: sub-steps of the chemical timestep; in each, the BDF
 * update of App. B with alpha_B(T) and Gamma_coll(T) at the sub-step's start,
 * then the implicit energy update at the new composition.  Heating per
 * volume H = n_HI (hpt + g_diff e_diff) + (alpha_A - alpha_B)(T) n_e n_HII
 * e_diff: the photo-heating of the point sources and the plane flux (hpt,
 * per neutral atom), of the transferred diffuse field, and of the local
 * recombination photons counted in Gamma^diff by Eq. (gamma_diff). */
int orc_thermal_cell(const orc_thermal *th, double nH, double y0, double T0, double gpt, double hpt, double gdiff,
                     double dt, double eps_e, double eps_hi, int max_sub, double *y_out, double *T_out)
{
    double y = y0, T = T0, tau = 0.0;
    int n = 0;
    const double g = gpt + gdiff;
    while (tau < dt && n < max_sub) {
        const double aB = orc_alpha_B(T), gc = orc_gamma_coll(T);
        const double dal = th->on_the_spot ? 0.0 : orc_alpha_A(T) - aB;
        const double nHI = y * nH, ne = (1.0 - y) * nH;
        const double Cc = aB * ne * ne, D = gc * ne + g;
        double dtc = dtchem_cell(nH, y, aB, gc, g, eps_e, eps_hi);
        const int last = !(dtc < dt - tau);
        if (last) dtc = dt - tau;
        double y1 = (Cc * dtc + nHI) / (1.0 + D * dtc) / nH;
        if (y1 > 1.0) y1 = 1.0;
        const double ne1 = (1.0 - y1) * nH;
        const double H1 = y1 * nH * (hpt + gdiff * th->e_diff) + dal * ne1 * ne1 * th->e_diff;
        T = orc_energy_step(th, nH, y, T, y1, H1, dtc);
        y = y1;
        tau = last ? dt : tau + dtc;
        n++;
    }
    *y_out = y;
    *T_out = T;
    return n;
}

/* Rates of state (y, T): kappa, the emissivity with (alpha_A - alpha_B)(T),
 * the point sources and plane flux (photo-ionization g and heating h per
 * neutral atom: the same rates with bin luminosities Q_b E_b), and the
 * diffuse rate 4 pi G J^in (zero on the spot). */
static void thermal_rates(const orc_sweep_cfg *cfg, const orc_chem *ch, const orc_thermal *th, const double *nH,
                          const double *y, const double *T, int nsrc, const double *pos, const double *qb,
                          const double *qh, int nb, const double *sigma_b, int pl_axis, int pl_dir, double pl_flux,
                          const double *fb, const double *fh, double G, double *kap, double *kapb, double *eps,
                          double *gdiff, double *gpt, double *hpt, double *tmp)
{
    const long ncell = (long)cfg->nx * cfg->ny * cfg->nz;
    for (long i = 0; i < ncell; i++) {
        const double nHI = y[i] * nH[i], ne = (1.0 - y[i]) * nH[i];
        kap[i] = nHI * ch->sigma0 * ch->dx;
        const double dal = orc_alpha_A(T[i]) - orc_alpha_B(T[i]);
        eps[i] = ch->h * ch->nu0 * dal * ne * ne * ch->dx / (4.0 * M_PI * ch->dnu);
    }
    if (th->on_the_spot) {
        for (long i = 0; i < ncell; i++) gdiff[i] = 0.0;
    } else {
        orc_sweep_cfg c = *cfg;
        c.field_form = 1;
        orc_sweep(&c, kap, eps, gdiff, NULL);
        for (long i = 0; i < ncell; i++) gdiff[i] *= 4.0 * M_PI * G;
    }
    for (int b = 0; b < nb; b++)
        for (long i = 0; i < ncell; i++) kapb[b * ncell + i] = y[i] * nH[i] * sigma_b[b] * ch->dx;
    orc_point_sources(cfg->nx, cfg->ny, cfg->nz, nb, kapb, sigma_b, nsrc, pos, qb, ch->dx, cfg->nthreads, gpt);
    orc_point_sources(cfg->nx, cfg->ny, cfg->nz, nb, kapb, sigma_b, nsrc, pos, qh, ch->dx, cfg->nthreads, hpt);
    if (pl_flux > 0.0) {
        orc_plane_source(cfg->nx, cfg->ny, cfg->nz, nb, kapb, sigma_b, pl_axis, pl_dir, fb, tmp);
        for (long i = 0; i < ncell; i++) gpt[i] += tmp[i];
        orc_plane_source(cfg->nx, cfg->ny, cfg->nz, nb, kapb, sigma_b, pl_axis, pl_dir, fh, tmp);
        for (long i = 0; i < ncell; i++) hpt[i] += tmp[i];
    }
}

/* Time-dependent mode with the energy equation: as orc_evolve, with the
 * temperature T carried beside y, the rates and the emissivity taken at
 * each cell's temperature, and the iteration of every RT step run until
 * both n_e and u converge (App. D: |x^(i) - x^(i-1)| < eps_iter x^(i) for
 * x = n_e, u).  Return codes as orc_evolve. */
int orc_evolve_thermal(const orc_sweep_cfg *cfg, const orc_chem *ch, const orc_thermal *th, const double *nH,
                       int nsrc, const double *pos, const double *Q, int nb, const double *sigma_b,
                       const double *frac_b, int pl_axis, int pl_dir, double pl_flux, const orc_evolve_opt *opt,
                       double t_end, double *y, double *T, int *steps_out, int *iters_out, double *t_out,
                       double *dt_hist)
{
    const long ncell = (long)cfg->nx * cfg->ny * cfg->nz;
    double *kap = malloc(sizeof(double) * ncell), *kapb = malloc(sizeof(double) * ncell * nb);
    double *eps = malloc(sizeof(double) * ncell), *gdiff = malloc(sizeof(double) * ncell);
    double *gpt = malloc(sizeof(double) * ncell), *hpt = malloc(sizeof(double) * ncell);
    double *tmp = malloc(sizeof(double) * ncell);
    double *yp = malloc(sizeof(double) * ncell), *Tp = malloc(sizeof(double) * ncell);
    double *yn = malloc(sizeof(double) * ncell), *Tn = malloc(sizeof(double) * ncell);
    const int ns = nsrc > 0 ? nsrc : 1;
    double *qb = malloc(sizeof(double) * ns * nb), *qh = malloc(sizeof(double) * ns * nb);
    double *fb = malloc(sizeof(double) * nb), *fh = malloc(sizeof(double) * nb);
    if (!kap || !kapb || !eps || !gdiff || !gpt || !hpt || !tmp || !yp || !Tp || !yn || !Tn || !qb || !qh || !fb ||
        !fh)
        return -1;
    for (int a = 0; a < nsrc; a++)
        for (int b = 0; b < nb; b++) {
            qb[a * nb + b] = Q[a] * frac_b[b];
            qh[a * nb + b] = Q[a] * frac_b[b] * th->e_bin[b];
        }
    for (int b = 0; b < nb; b++) {
        fb[b] = pl_flux * frac_b[b];
        fh[b] = pl_flux * frac_b[b] * th->e_bin[b];
    }
    const double G = orc_band_integral(ch->sigma0, ch->h, ch->nu0, ch->nu0 + ch->dnu);
    double t = 0.0;
    int steps = 0, iters = 0, unconverged = 0;
    while (t < t_end && steps < opt->max_steps) {
        thermal_rates(cfg, ch, th, nH, y, T, nsrc, pos, qb, qh, nb, sigma_b, pl_axis, pl_dir, pl_flux, fb, fh, G,
                      kap, kapb, eps, gdiff, gpt, hpt, tmp);
        double dt;
        if (opt->dt_fixed > 0.0) {
            dt = opt->dt_fixed;
        } else {
            double m = INFINITY;
            for (long i = 0; i < ncell; i++) {
                const double d = dtchem_T(nH[i], y[i], T[i], gpt[i] + gdiff[i], opt->eps_e, opt->eps_hi);
                if (d < m) m = d;
            }
            dt = opt->F * m;
        }
        const int last = !(dt < t_end - t);
        if (last) dt = t_end - t;
        for (long i = 0; i < ncell; i++) {
            yp[i] = y[i];
            Tp[i] = T[i];
        }
        int conv = 0;
        for (int k = 1; k <= opt->max_iter; k++) {
            iters++;
            double r = 0.0;
            for (long i = 0; i < ncell; i++) {
                orc_thermal_cell(th, nH[i], y[i], T[i], gpt[i], hpt[i], gdiff[i], dt, opt->eps_e, opt->eps_hi,
                                 opt->max_sub, &yn[i], &Tn[i]);
                const double ne_new = (1.0 - yn[i]) * nH[i], ne_old = (1.0 - yp[i]) * nH[i];
                const double re = ne_new > 0.0 ? fabs(ne_new - ne_old) / ne_new : (ne_old > 0.0 ? INFINITY : 0.0);
                const double u_new = (2.0 - yn[i]) * Tn[i], u_old = (2.0 - yp[i]) * Tp[i];
                const double ru = fabs(u_new - u_old) / u_new;
                if (re > r) r = re;
                if (ru > r) r = ru;
            }
            for (long i = 0; i < ncell; i++) {
                yp[i] = yn[i];
                Tp[i] = Tn[i];
            }
            if (r < opt->eps_iter) {
                conv = 1;
                break;
            }
            thermal_rates(cfg, ch, th, nH, yp, Tp, nsrc, pos, qb, qh, nb, sigma_b, pl_axis, pl_dir, pl_flux, fb, fh,
                          G, kap, kapb, eps, gdiff, gpt, hpt, tmp);
        }
        if (!conv) unconverged = 1;
        for (long i = 0; i < ncell; i++) {
            y[i] = yp[i];
            T[i] = Tp[i];
        }
        if (dt_hist) dt_hist[steps] = dt;
        t = last ? t_end : t + dt;
        steps++;
    }
    if (steps_out) *steps_out = steps;
    if (iters_out) *iters_out = iters;
    if (t_out) *t_out = t;
    free(kap); free(kapb); free(eps); free(gdiff); free(gpt); free(hpt); free(tmp); free(yp); free(Tp);
    free(yn); free(Tn); free(qb); free(qh); free(fb); free(fh);
    if (t < t_end) return 2;
    return unconverged ? 1 : 0;
}
