// art_ctx.hpp -- the context behind art_ctx* (private to libart).
#pragma once
#include <cuda_runtime.h>

#include <string>
#include <vector>

#include "art.h"
#include "art_kernels.cuh"

struct art_net;

// Device buffers of the RT / ionization-balance iteration (allocated on the
// first art_iterate_ionization call).
struct art_iter_bufs {
    long long ncell = 0;
    int nsrc_cap = 0;
    double *nH = nullptr, *y = nullptr, *y0 = nullptr;   // FP64 state
    float *gpt = nullptr, *kap = nullptr, *eps = nullptr, *jin = nullptr;
    float *jsur = nullptr;                                // surrogate J^in / prolonged J_c
    unsigned long long *resid = nullptr;
    double *src = nullptr;                                // packed point sources
    double *yit = nullptr;                                // time-dependent mode: the iterate at t + dt
    unsigned long long *evo = nullptr;                    // [3]: residual, min dt_chem (double bits), overflows
    float *hpt = nullptr;                                 // energy equation: photo-heating per neutral atom
    double *Tit = nullptr;                                // energy equation: the temperature iterate at t + dt
};

// One grid of a context (a context holds one grid, or a batch of them).
struct art_grid_host {
    art_grid g{};
    int nside = 0, nd = 0;
    long long ncell = 0;
    long long cell_off = 0;    // first cell in the concatenated [z][y][x] arrays
    long long jpart_off = 0;   // first element of its J partials
    int n_part = 0;            // J partials (classes x direction groups)
    int nblocks = 0;           // slab blocks of its longest axis
    long long seg_count = 0;   // segments per sweep and bin
};

// Scratch of the surrogate on this context's grid (coarse fields, coarse
// J^in, network output, eps_ref).
struct art_sur_bufs {
    long long n = 0;
    int f = 0, nside = 0;
    void *kc = nullptr, *ec = nullptr, *jc = nullptr, *o = nullptr, *eref = nullptr;
    double *nHc = nullptr, *yc = nullptr;   // coarse-mesh solve of the warm start
};

// Wavefront sweep (art_wave.cuh): tables and buffers of the selected shape.
struct art_wave_state {
    bool on = false;
    int variant = 0, wb = 0, wc = 0, dmax = 0, np = 1, n_units = 0;
    int bins_per_launch = 1;    // all of a sweep's bins in one launch when their buffers fit
    void *units = nullptr, *classes = nullptr, *rtab = nullptr;   // rtab: run tables of the direction groups
    long long rtab_len = 0;     // float4 count
    float *edge = nullptr;      // edge intensities handed between CTA tiles
    int *flags = nullptr;       // [0] error word, [1] ticket, then per-unit progress flags
    long long *stats = nullptr; // inside the flags allocation: counters of ART_WAVE_STATS builds
    size_t flag_bytes = 0;
    long long edge_floats = 0, jpart_floats = 0, bytes = 0;
    long long wait_ns = 2000000000LL;   // bound of every wait in the kernel
    int stall_unit = -1;                 // test hook (see art_wave_test_stall)
};

struct art_ctx {
    art_grid grid{};           // first grid (the only one outside batches)
    int nside = 0, nbins = 0;
    std::vector<art_grid_host> grids;
    int persistent = 0;        // sweep launches take work items from a queue
    int n_ctas = 0;            // CTAs of a persistent launch
    bool early_launch = true;  // slab-block launches after the first may start as the previous one drains
    int *d_counter = nullptr;  // queue heads, one per slab block
    void *d_gridinfo = nullptr;
    // CUDA graph of one sweep (device outputs), replayed while the outputs match
    cudaGraphExec_t gexec = nullptr;
    cudaStream_t gstream = nullptr;
    cudaEvent_t gev[2] = {nullptr, nullptr};
    void *g_key[3] = {nullptr, nullptr, nullptr};
    art_options opt{};
    std::string err;
    int prec = ART_FP32;
    size_t rsz = 4;           // bytes per real
    long long ncell = 0;
    int nd = 0;
    int TB = 0, TC = 0, BLK = 0, NT = 0, KP = 1, variant = 0, split = 1, nblocks = 0;
    int n_classes = 0, n_part = 0, n_work = 0;
    long long seg_count = 0;  // segments per sweep, one bin
    long long plane_elems = 0;
    std::vector<double> G;
    std::vector<double> i_bc;  // boundary intensity per bin (0: vacuum)
    bool have_fields = false;
    long long dev_bytes = 0;
    // device memory
    void *d_field = nullptr;   // [3][nbins][ncell] vec2
    void *d_plane[2] = {nullptr, nullptr};
    size_t plane_bytes = 0, plane_bytes_0 = 0, plane_bytes_1 = 0;
    void *d_jpart = nullptr;   // [n_part][ncell] real, natural layout
    void *d_segs = nullptr;
    art::DirDev *d_dirs = nullptr;
    art::ClassDev *d_classes = nullptr;
    art::WorkItem *d_work = nullptr;
    size_t jpart_bytes = 0, segs_bytes = 0, dirs_bytes = 0, classes_bytes = 0, work_bytes = 0,
           counter_bytes = 0, gridinfo_bytes = 0;
    void *d_stage = nullptr;   // [2][nbins][ncell] real: host-input staging
    void *d_out = nullptr;     // [2 nbins + 1][ncell] real: host-output staging
    int *d_flag = nullptr;
    // art_sweep_stream: copy streams, the second input staging buffer, two
    // output slots, per-slot validation flags (device and pinned host), events
    struct StreamRes {
        cudaStream_t in = nullptr, out = nullptr;
        cudaEvent_t ev_in[2] = {nullptr, nullptr}, ev_lay[2] = {nullptr, nullptr};
        cudaEvent_t ev_sw[2] = {nullptr, nullptr}, ev_out[2] = {nullptr, nullptr};
        void *stage2 = nullptr, *slot[2] = {nullptr, nullptr};
        int *d_flags = nullptr, *h_flags = nullptr;
    } sres;
    // profiling: event triples (before sweep launches, after them, after reduce)
    bool profiling = false;
    std::vector<cudaEvent_t> ev;
    art_iter_bufs it;
    int spec_bins = 0;          // point-source spectrum of the iteration (0: one bin at sigma0)
    double spec_sigma[4] = {0, 0, 0, 0}, spec_frac[4] = {0, 0, 0, 0};
    int plane_axis = 0, plane_dir = 1;   // plane-parallel incident flux of the iteration
    double plane_flux = 0.0;             // photons/s/cm^2 (0: none)
    double relax = 1.0;                  // over-relaxation factor of the balance update (1: plain)
    art_ctx *coarse = nullptr;  // coarse-mesh sweep of the surrogate
    void *ablation = nullptr;   // thread-per-ray comparison sweep (tables, graphs)
    art_sur_bufs sur;
    art_wave_state wave;
    art_net *net = nullptr;     // the context's surrogate (art_surrogate_train)
};


// internal entry points shared by the translation units of libart
art_status art_fail(art_ctx *ctx, art_status st, const std::string &msg);
void art_internal_ablation_free(art_ctx *ctx);
art_status art_internal_sweep(art_ctx *ctx, void *J, void *J_in, void *gamma, cudaStream_t st);
art_status art_internal_layout(art_ctx *ctx, const void *kappa, const void *src, cudaStream_t st);
// wavefront sweep (art_wave.cu)
int art_wave_variants();
int art_wave_dmax(int w);
int art_wave_default(int maxc, long long cells);   // default shape: class size, largest grid
void art_wave_free(art_ctx *ctx);
art_status art_wave_setup(art_ctx *ctx, int w);
art_status art_wave_launch(art_ctx *ctx, const float2 *f0, const float2 *f1, const float2 *f2,
                           long long bin_cells, int b0, cudaStream_t st);
art_status art_wave_status(art_ctx *ctx, cudaStream_t st);
art_status art_wave_status_async(art_ctx *ctx, int *host, cudaStream_t st);
