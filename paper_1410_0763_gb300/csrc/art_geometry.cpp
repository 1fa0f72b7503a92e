// art_geometry.cpp -- see art_geometry.hpp.
#include "art_geometry.hpp"

#include <algorithm>
#include <cmath>

namespace art {

static const double kPi = 3.14159265358979323846;

// HEALPix RING scheme, enumerated ring by ring from the north pole.  Ring r
// (1 .. 4N-1) has its centre at z_r; the polar rings hold 4r (4(4N-r))
// pixels with a half-pixel phi offset, the 2N+1 equatorial rings hold 4N
// pixels, every other one shifted by half a pixel (Gorski et al. 2005,
// Sec. 4: equal-area, iso-latitude pixels).
void healpix_directions(int nside, std::vector<double> &xyz)
{
    xyz.assign(36u * nside * nside, 0.0);
    healpix_directions_into(nside, xyz.data());
}

void healpix_directions_into(int nside, double *xyz)
{
    const int N = nside;
    long long p = 0;
    for (int r = 1; r <= 4 * N - 1; ++r) {
        double z, dphi, off;
        int count;
        if (r < N) {
            z = 1.0 - double(r) * r / (3.0 * N * N);
            count = 4 * r;
            dphi = kPi / (2.0 * r);
            off = 0.5;
        } else if (r <= 3 * N) {
            z = 2.0 * double(2 * N - r) / (3.0 * N);
            count = 4 * N;
            dphi = kPi / (2.0 * N);
            off = ((r - N + 1) & 1) ? 0.5 : 0.0;
        } else {
            const int rs = 4 * N - r;
            z = -(1.0 - double(rs) * rs / (3.0 * N * N));
            count = 4 * rs;
            dphi = kPi / (2.0 * rs);
            off = 0.5;
        }
        const double st = std::sqrt((1.0 - z) * (1.0 + z));
        for (int j = 1; j <= count; ++j, ++p) {
            const double ph = dphi * (j - off);
            xyz[3 * p] = st * std::cos(ph);
            xyz[3 * p + 1] = st * std::sin(ph);
            xyz[3 * p + 2] = z;
        }
    }
}

Frame frame_of(const double n[3], double tie_tol)
{
    Frame f;
    const double m = std::max(std::fabs(n[0]), std::max(std::fabs(n[1]), std::fabs(n[2])));
    f.a = 2;
    for (int i = 2; i >= 0; --i)
        if (std::fabs(n[i]) >= m - tie_tol * m) f.a = i;
    f.b = (f.a == 0) ? 1 : 0;
    f.c = (f.a == 2) ? 1 : 2;
    f.sa = n[f.a] >= 0.0 ? 1 : -1;
    f.sb = n[f.b] >= 0.0 ? 1 : -1;
    f.sc = n[f.c] >= 0.0 ? 1 : -1;
    f.na = std::fabs(n[f.a]);
    f.qb = std::min(std::fabs(n[f.b]) / f.na, 1.0);
    f.qc = std::min(std::fabs(n[f.c]) / f.na, 1.0);
    f.cls = f.a * 8 + (f.sa < 0 ? 4 : 0) + (f.sb < 0 ? 2 : 0) + (f.sc < 0 ? 1 : 0);
    return f;
}

// Crossings closer than kTie (cell widths along a) are one crossing: a ray
// through an edge or a corner steps across all those planes at once and no
// sliver segment is made.  This also absorbs the last-bit differences of
// components that are equal in exact arithmetic (e.g. |n_b| = |n_c|).
static const double kTie = 1e-12;

static double snap(double u)
{
    if (u <= kTie) return 0.0;
    if (u >= 1.0 - kTie) return 1.0;
    return u;
}

// In the canonical frame the rays sit at X_b = j + 1/2 + qb u.  The integer
// part F(m) = floor(1/2 + qb m) of the offset at plane m advances by 0 or 1
// per slab; it advances exactly when the ray meets a b-plane inside the slab,
// at u - m = (F(m+1) - 1/2 - qb m)/qb.  Deriving the crossing from F keeps the
// crossings and the column shifts of consecutive slabs consistent.
void slab_geometry(const Frame &f, int Na, std::vector<SlabGeom> &out)
{
    out.resize(Na);
    slab_geometry_into(f, Na, out.data());
}

void slab_geometry_into(const Frame &f, int Na, SlabGeom *out)
{
    for (int m = 0; m < Na; ++m) {
        SlabGeom g{};
        const double fb0 = std::floor(0.5 + f.qb * m), fb1 = std::floor(0.5 + f.qb * (m + 1));
        const double fc0 = std::floor(0.5 + f.qc * m), fc1 = std::floor(0.5 + f.qc * (m + 1));
        g.shb = fb1 > fb0 ? 1 : 0;
        g.shc = fc1 > fc0 ? 1 : 0;
        double ub = 2.0, uc = 2.0;
        if (g.shb) ub = snap((fb1 - 0.5 - f.qb * m) / f.qb);
        if (g.shc) uc = snap((fc1 - 0.5 - f.qc * m) / f.qc);
        if (g.shb && g.shc && std::fabs(ub - uc) <= kTie) uc = ub;   // through an edge
        const double inv = 1.0 / f.na;
        g.nseg = 1 + g.shb + g.shc;
        if (g.nseg == 1) {
            g.ds[0] = inv;
        } else if (g.nseg == 2) {
            const double u = g.shb ? ub : uc;
            g.ds[0] = u * inv;
            g.ds[1] = (1.0 - u) * inv;
        } else {
            g.cfirst = uc < ub ? 1 : 0;
            const double u1 = std::min(ub, uc), u2 = std::max(ub, uc);
            g.ds[0] = u1 * inv;
            g.ds[1] = (u2 - u1) * inv;
            g.ds[2] = (1.0 - u2) * inv;
        }
        g.nonzero = 0;
        for (int k = 0; k < g.nseg; ++k) g.nonzero += g.ds[k] > 0.0 ? 1 : 0;
        out[m] = g;
    }
}

}  // namespace art
