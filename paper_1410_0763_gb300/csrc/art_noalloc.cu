// art_noalloc.cu -- art_sweep_noalloc: the diffuse-radiation sweep for callers
// that cannot allocate device memory (see include/art.h).  All working memory
// comes from one file-scope device array; host-side tables live in file-scope
// host arrays.  Nothing here calls cudaMalloc, cudaFree or any other
// allocating routine.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>
#include <cstring>

#include "art.h"
#include "art_geometry.hpp"
#include "art_kernels.cuh"

using namespace art;

namespace {

// Working memory of every call, on every device that loads the library.
constexpr size_t kScratchBytes = size_t(12) << 20;
static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

constexpr int kMaxDim = 64;            // cells per axis
constexpr long long kMaxCells = 32768; // cells in total (32^3)
constexpr int kMaxNside = 4;           // 192 directions
constexpr int kMaxDirs = 12 * kMaxNside * kMaxNside;
constexpr int kMaxSlabs = kMaxDirs * kMaxDim;
constexpr int kTB = 32, kTC = 8, kBLK = 4, kNT = 256, kKP = 2, kMINB = 3;
constexpr int kMaxWork = 24 * ((kMaxDim + kTB - 1) / kTB) * ((kMaxDim + kTC - 1) / kTC);

// Device address of g_scratch, looked up once per device.
constexpr int kMaxDevices = 64;
static void *g_scratch_dev[kMaxDevices];

// Host-side tables of the current call.
static double g_xyz[3 * kMaxDirs];
static Frame g_frame[kMaxDirs];
static int g_order[kMaxDirs];
static SegEntry<float> g_segs[kMaxSlabs];
static SlabGeom g_geo[kMaxDim];
static DirDev g_dirs[kMaxDirs];
static ClassDev g_classes[24];
static WorkItem g_work[kMaxWork];
static GridDev<float> g_grid;

size_t align256(size_t x) { return (x + 255) / 256 * 256; }

art_status reject(char *errbuf, size_t errlen, art_status st, const char *msg)
{
    if (errbuf && errlen) std::snprintf(errbuf, errlen, "%s", msg);
    return st;
}

}  // namespace

extern "C" art_status art_sweep_noalloc(const art_grid *grid, int n_side, const float *kappa, const float *S,
                                        float *J_in, void *stream, char *errbuf, size_t errlen)
{
    if (!grid || !kappa || !S || !J_in)
        return reject(errbuf, errlen, ART_E_INVALID, "art_sweep_noalloc: null argument");
    const int dims[3] = {grid->nx, grid->ny, grid->nz};
    const long long ncell = (long long)dims[0] * dims[1] * dims[2];
    if (dims[0] < 1 || dims[1] < 1 || dims[2] < 1 || n_side < 1)
        return reject(errbuf, errlen, ART_E_INVALID, "art_sweep_noalloc: dimensions and n_side must be >= 1");
    if (dims[0] > kMaxDim || dims[1] > kMaxDim || dims[2] > kMaxDim || ncell > kMaxCells || n_side > kMaxNside)
        return reject(errbuf, errlen, ART_E_INVALID,
                      "art_sweep_noalloc: grid or angular resolution above the fixed maximum "
                      "(each axis <= 64 cells, <= 32768 cells, n_side <= 4); use art_create/art_sweep");
    cudaStream_t st = static_cast<cudaStream_t>(stream);

    // The call synchronizes the stream after copying its tables, which a stream
    // capture does not allow: refuse before anything is queued, so that the
    // caller's capture stays valid.
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(st, &cap) != cudaSuccess) {
        cudaGetLastError();
        return reject(errbuf, errlen, ART_E_CUDA, "art_sweep_noalloc: cudaStreamIsCapturing failed");
    }
    if (cap != cudaStreamCaptureStatusNone)
        return reject(errbuf, errlen, ART_E_INVALID,
                      "art_sweep_noalloc: the stream is being captured; call it outside stream capture");

    // Device set-up, once per device: the device address of the scratch array.
    // The device module holding the array is loaded here, on the first call
    // (lazy loading), which is when its 12 MiB are reserved.
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices)
        return reject(errbuf, errlen, ART_E_CUDA, "art_sweep_noalloc: no usable current device");
    if (!g_scratch_dev[dev]) {
        void *ptr = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&ptr, g_scratch);
        if (e != cudaSuccess || !ptr) {
            cudaGetLastError();
            if (e == cudaErrorMemoryAllocation)
                return reject(errbuf, errlen, ART_E_OOM,
                              "art_sweep_noalloc: loading the library's device module (with its 12 MiB scratch "
                              "array) ran out of device memory; make the first call on each device before "
                              "reserving the device's memory");
            char msg[256];
            std::snprintf(msg, sizeof(msg), "art_sweep_noalloc: loading the device module / scratch address failed: %s",
                          cudaGetErrorString(e));
            return reject(errbuf, errlen, ART_E_CUDA, msg);
        }
        g_scratch_dev[dev] = ptr;
    }
    unsigned char *base = static_cast<unsigned char *>(g_scratch_dev[dev]);

    // Host tables: classes of directions, drift-sorted, with segment tables.
    const int nd = 12 * n_side * n_side;
    healpix_directions_into(n_side, g_xyz);
    for (int d = 0; d < nd; ++d) g_frame[d] = frame_of(&g_xyz[3 * d], 1e-12);
    int ncls = 0, nslab = 0, nwork = 0, ndir = 0;
    long long plane_elems = 0;
    auto drift = [](double q) { return (int)std::floor(q * kBLK + 0.5); };
    for (int cls = 0; cls < 24; ++cls) {
        int cnt = 0;
        for (int d = 0; d < nd; ++d)
            if (g_frame[d].cls == cls) g_order[cnt++] = d;
        if (!cnt) continue;
        for (int i = 1; i < cnt; ++i) {   // stable insertion sort by (drift b, drift c)
            const int v = g_order[i];
            int j = i - 1;
            while (j >= 0) {
                const int u = g_order[j];
                const int bu = drift(g_frame[u].qb), bv = drift(g_frame[v].qb);
                const bool after = bu > bv || (bu == bv && drift(g_frame[u].qc) > drift(g_frame[v].qc));
                if (!after) break;
                g_order[j + 1] = u;
                --j;
            }
            g_order[j + 1] = v;
        }
        const Frame &f0 = g_frame[g_order[0]];
        ClassDev C;
        C.a = f0.a;
        C.sa = f0.sa;
        C.sb = f0.sb;
        C.sc = f0.sc;
        C.Na = dims[f0.a];
        C.Nb = dims[f0.b];
        C.Nc = dims[f0.c];
        C.dir_begin = ndir;
        C.dir_end = ndir + cnt;
        C.part0 = ncls;
        C.nx = dims[0];
        C.ny = dims[1];
        C.nz = dims[2];
        C.cell_off = 0;
        C.jpart_off = (long long)ncls * ncell;
        C.ncell = ncell;
        for (int i = 0; i < cnt; ++i) {
            DirDev D;
            D.seg_off = nslab;
            D.plane_off = plane_elems;
            D.na = g_frame[g_order[i]].na;
            g_dirs[ndir++] = D;
            slab_geometry_into(g_frame[g_order[i]], C.Na, g_geo);
            // entries with the remaining column shifts to the end of each slab block (read by the kernel)
            for (int m = C.Na - 1; m >= 0; --m) {
                const SlabGeom &g = g_geo[m];
                SegEntry<float> &e = g_segs[nslab + m];
                const bool last = (m + 1) % kBLK == 0 || m + 1 == C.Na;
                const int nxt = last ? 0 : g_segs[nslab + m + 1].code;
                e.ds1 = float(g.ds[0]);
                e.ds2 = float(g.ds[1]);
                e.ds3 = float(g.ds[2]);
                e.code = slab_code(g, g.shb + ((nxt >> 5) & 15), g.shc + ((nxt >> 9) & 15));
            }
            nslab += C.Na;
            plane_elems += (long long)C.Nb * C.Nc;
        }
        for (int pc = 0; pc < C.Nc; pc += kTC)
            for (int pb = 0; pb < C.Nb; pb += kTB) g_work[nwork++] = WorkItem{ncls, pb, pc, 0};
        g_classes[ncls++] = C;
    }

    // Scratch layout; every region read by a launch is written earlier in the
    // same call (the first slab block does not read a plane), so no state
    // carries over between calls and nothing needs clearing.
    const size_t o_field = 0;
    const size_t o_plane0 = align256(o_field + 3 * size_t(ncell) * sizeof(float2));
    const size_t o_plane1 = align256(o_plane0 + size_t(plane_elems) * sizeof(float));
    const size_t o_jpart = align256(o_plane1 + size_t(plane_elems) * sizeof(float));
    const size_t o_segs = align256(o_jpart + size_t(ncls) * ncell * sizeof(float));
    const size_t o_dirs = align256(o_segs + size_t(nslab) * sizeof(SegEntry<float>));
    const size_t o_cls = align256(o_dirs + size_t(ndir) * sizeof(DirDev));
    const size_t o_work = align256(o_cls + size_t(ncls) * sizeof(ClassDev));
    const size_t o_grid = align256(o_work + size_t(nwork) * sizeof(WorkItem));
    const size_t need = align256(o_grid + sizeof(GridDev<float>));
    if (need > kScratchBytes)
        return reject(errbuf, errlen, ART_E_INVALID,
                      "art_sweep_noalloc: this grid needs more than the 12 MiB scratch array; use art_create/art_sweep");

    float2 *fld = reinterpret_cast<float2 *>(base + o_field);
    float *planes[2] = {reinterpret_cast<float *>(base + o_plane0), reinterpret_cast<float *>(base + o_plane1)};
    float *jpart = reinterpret_cast<float *>(base + o_jpart);
#define ART_NA_CK(call, what)                                                       \
    do {                                                                            \
        if ((call) != cudaSuccess) {                                                \
            cudaGetLastError();                                                     \
            return reject(errbuf, errlen, ART_E_CUDA, "art_sweep_noalloc: " what);  \
        }                                                                           \
    } while (0)
    ART_NA_CK(cudaMemcpyAsync(base + o_segs, g_segs, size_t(nslab) * sizeof(SegEntry<float>), cudaMemcpyHostToDevice, st),
              "copy of the segment tables failed");
    ART_NA_CK(cudaMemcpyAsync(base + o_dirs, g_dirs, size_t(ndir) * sizeof(DirDev), cudaMemcpyHostToDevice, st),
              "copy of the direction table failed");
    ART_NA_CK(cudaMemcpyAsync(base + o_cls, g_classes, size_t(ncls) * sizeof(ClassDev), cudaMemcpyHostToDevice, st),
              "copy of the class table failed");
    ART_NA_CK(cudaMemcpyAsync(base + o_work, g_work, size_t(nwork) * sizeof(WorkItem), cudaMemcpyHostToDevice, st),
              "copy of the work list failed");
    g_grid = GridDev<float>{0, ncell, 0, ncls, float(1.0 / nd)};
    ART_NA_CK(cudaMemcpyAsync(base + o_grid, &g_grid, sizeof(g_grid), cudaMemcpyHostToDevice, st),
              "copy of the grid record failed");
    // the host tables are reused by the next call: wait for the copies
    ART_NA_CK(cudaStreamSynchronize(st), "stream synchronize failed");

    const int nt = 256;
    layout_kernel<float><<<(unsigned)((ncell + nt - 1) / nt), nt, 0, st>>>(kappa, S, fld, fld + ncell, fld + 2 * ncell,
                                                                           dims[0], dims[1], dims[2]);
    ART_NA_CK(cudaGetLastError(), "layout kernel launch failed");

    SweepArgs<float> a{};
    a.field0 = fld;
    a.field1 = fld + ncell;
    a.field2 = fld + 2 * ncell;
    a.jpart = jpart;
    a.segs = reinterpret_cast<const SegEntry<float> *>(base + o_segs);
    a.dirs = reinterpret_cast<const DirDev *>(base + o_dirs);
    a.classes = reinterpret_cast<const ClassDev *>(base + o_cls);
    a.work = reinterpret_cast<const WorkItem *>(base + o_work);
    a.n_work = nwork;
    a.counter = nullptr;
    a.split = 1;
    a.field_form = ART_FIELDS_S;
    a.i_bc = 0.0f;   // vacuum boundary
    a.averaging = ART_AVG_PAPER;
    int maxNa = 0;
    for (int c = 0; c < ncls; ++c) maxNa = g_classes[c].Na > maxNa ? g_classes[c].Na : maxNa;
    const size_t sm = SweepShape<kTB, kTC, kBLK, kNT, kKP>::bytes<float>();
    auto kern = sweep_block_kernel<float, kTB, kTC, kBLK, kNT, kKP, kMINB>;
    if (sm > 48 * 1024)
        ART_NA_CK(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm),
                  "shared-memory attribute failed");
    for (int k = 0; k * kBLK < maxNa; ++k) {
        a.kblock = k;
        a.plane_in = planes[k & 1];
        a.plane_out = planes[(k + 1) & 1];
        kern<<<nwork, kNT, sm, st>>>(a);
        ART_NA_CK(cudaGetLastError(), "sweep kernel launch failed");
    }
    ReduceArgs<float> r{};
    r.jpart = jpart;
    r.field_nat = fld + 2 * ncell;
    r.grids = reinterpret_cast<const GridDev<float> *>(base + o_grid);
    r.n_grids = 1;
    r.total = ncell;
    r.gamma_coef = 0.0f;
    r.gamma_accum = 0;
    r.field_form = ART_FIELDS_S;
    r.whole = 0;
    r.Jin = J_in;
    r.J = nullptr;
    r.gamma = nullptr;
    reduce_kernel<float><<<(unsigned)((ncell + nt - 1) / nt), nt, 0, st>>>(r);
    ART_NA_CK(cudaGetLastError(), "reduce kernel launch failed");
#undef ART_NA_CK
    if (errbuf && errlen) errbuf[0] = '\0';
    return ART_OK;
}
