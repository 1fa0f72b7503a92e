// art_geometry.hpp -- host-side FP64 geometry of the parallel-ray sweep.
//
// Directions are HEALPix RING pixel centres (Sec. 2.3 of Tanaka et al. 2014;
// Gorski et al. 2005, Sec. 4).  Each direction is swept by the family of
// parallel rays of Sec. 2.2 (Fig. parallel_ray): lines one cell width apart on
// planes normal to the dominant axis a, through cell centres.  In the
// "canonical frame" of a direction the axes are mirrored so that every
// component of the direction is >= 0; there the ray in transverse column p at
// the a-plane u = m (m integer) sits at the same fractional offset
// frac(1/2 + q m) for every ray, so the pieces into which a slab
// m <= u < m+1 cuts a ray are the same for all rays of the direction.  The
// per-slab table below holds those pieces: up to three segments, in order,
// in the cells at transverse offsets (0,0), then (1,0) or (0,1), then (1,1)
// from the ray's starting column.
#pragma once
#include <cstdint>
#include <vector>

namespace art {

// Octant-axis class: dominant axis and the signs of the three components.
struct Frame {
    int a, b, c;       // dominant axis; the other two in increasing order
    int sa, sb, sc;    // +1 / -1: sign of n_a, n_b, n_c (a zero counts as +1)
    double na;         // |n_a|
    double qb, qc;     // |n_b|/|n_a|, |n_c|/|n_a|, clamped to [0, 1]
    int cls;           // a * 8 + (sa < 0) * 4 + (sb < 0) * 2 + (sc < 0)
};

struct SlabGeom {
    double ds[3];      // path length of segment 1, 2, 3 (cell widths); unused = 0
    int nseg;          // 1, 2 or 3
    int cfirst;        // nseg == 3: the c-plane is crossed before the b-plane
    int shb, shc;      // the ray moves to the next b (c) column during the slab
    int nonzero;       // segments with ds > 0
};

// HEALPix RING pixel centres, 12 nside^2 unit vectors (x, y, z), RING order.
void healpix_directions(int nside, std::vector<double> &xyz);
// The same into a caller array of 36 nside^2 doubles (no allocation).
void healpix_directions_into(int nside, double *xyz);

// Frame of direction n; a = the lowest axis whose |n_i| is within tie_tol
// (relative) of the largest component.
Frame frame_of(const double n[3], double tie_tol);

// Segments of every slab 0 <= m < Na of a direction in its canonical frame.
void slab_geometry(const Frame &f, int Na, std::vector<SlabGeom> &out);
// The same into a caller array of Na entries (no allocation).
void slab_geometry_into(const Frame &f, int Na, SlabGeom *out);

// Code word of a slab-block segment-table entry: bits 0-1 nseg - 1, 2 the
// c-plane first, 3 b-shift, 4 c-shift, 5-8 and 9-12 the b- and c-shifts from
// this slab to the end of its slab block (rb, rc; this slab included).
inline int slab_code(const SlabGeom &g, int rb, int rc)
{
    return (g.nseg - 1) | (g.cfirst << 2) | (g.shb << 3) | (g.shc << 4) | (rb << 5) | (rc << 9);
}

}  // namespace art
