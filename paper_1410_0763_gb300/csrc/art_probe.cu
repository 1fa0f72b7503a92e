// art_probe.cu -- issue-rate microbenchmark of the pipes the sweep relies on:
// MUFU ex2 (one exponential per segment), MUFU rcp, FP32 FFMA and the packed
// FP32x2 FMA (counted as two FMAs) that the sweep's pair arithmetic uses.  Each CTA
// runs 8 independent chains per thread and records its SM and its first and
// last clock64() (a per-SM counter).  Per SM the window runs from the earliest
// start to the latest end of the CTAs it ran, so that CTAs which did not start
// together do not shorten it; the result per pipe is the median over SMs of
// operations per clock (two CTAs of 1024 threads resident per SM).
#include <cuda_runtime.h>

#include <algorithm>
#include <vector>

#include "art.h"

namespace {

// cyc[3 b] = first clock, cyc[3 b + 1] = last clock, cyc[3 b + 2] = SM of CTA b
template <int OP> __global__ void pipe_probe_kernel(float *out, long long *cyc, int iters)
{
    float a[8];
    float2 a2[8];
    for (int i = 0; i < 8; i++) {
        a[i] = (threadIdx.x + i) * 1e-3f;
        a2[i] = make_float2(a[i], a[i] + 0.5f);
    }
    __syncthreads();
    const long long t0 = clock64();
    for (int it = 0; it < iters; it++) {
#pragma unroll
        for (int i = 0; i < 8; i++) {
            if (OP == 3) {   // packed: two FP32 FMAs per instruction
                a2[i] = __ffma2_rn(a2[i], make_float2(1.0001f, 1.0001f), make_float2(0.5f, 0.5f));
                continue;
            }
            float y;
            if (OP == 0) {
                asm volatile("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(a[i] * -0.5f));
            } else if (OP == 1) {
                asm volatile("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(a[i] + 1.0f));
            } else {
                y = fmaf(a[i], 1.0001f, 0.5f);
            }
            a[i] = y;
        }
    }
    __syncthreads();
    const long long t1 = clock64();
    float s = 0.f;
    for (int i = 0; i < 8; i++) s += OP == 3 ? a2[i].x + a2[i].y : a[i];
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
    if (threadIdx.x == 0) {
        unsigned smid;
        asm volatile("mov.u32 %0, %%smid;" : "=r"(smid));
        cyc[3 * blockIdx.x] = t0;
        cyc[3 * blockIdx.x + 1] = t1;
        cyc[3 * blockIdx.x + 2] = smid;
    }
}

}  // namespace

extern "C" art_status art_measure_pipes(double *ex2_per_clk_sm, double *rcp_per_clk_sm,
                                        double *ffma_per_clk_sm, double *ffma2_per_clk_sm)
{
    if (!ex2_per_clk_sm || !rcp_per_clk_sm || !ffma_per_clk_sm || !ffma2_per_clk_sm) return ART_E_INVALID;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 1)
        return ART_E_CUDA;
    const int nt = 1024, per_sm = 2, nb = sms * per_sm, iters = 2048;
    float *out = nullptr;
    long long *cyc = nullptr;
    if (cudaMalloc(&out, sizeof(float) * nb * nt) != cudaSuccess) return ART_E_OOM;
    if (cudaMalloc(&cyc, sizeof(long long) * 3 * nb) != cudaSuccess) {
        cudaFree(out);
        return ART_E_OOM;
    }
    double *res[4] = {ex2_per_clk_sm, rcp_per_clk_sm, ffma_per_clk_sm, ffma2_per_clk_sm};
    std::vector<long long> h(3 * nb);
    art_status st = ART_OK;
    for (int op = 0; op < 4 && st == ART_OK; op++) {
        double best = 0.0;
        for (int rep = 0; rep < 2; rep++) {
            if (op == 0) pipe_probe_kernel<0><<<nb, nt>>>(out, cyc, iters);
            else if (op == 1) pipe_probe_kernel<1><<<nb, nt>>>(out, cyc, iters);
            else if (op == 2) pipe_probe_kernel<2><<<nb, nt>>>(out, cyc, iters);
            else pipe_probe_kernel<3><<<nb, nt>>>(out, cyc, iters);
            if (cudaDeviceSynchronize() != cudaSuccess ||
                cudaMemcpy(h.data(), cyc, sizeof(long long) * 3 * nb, cudaMemcpyDeviceToHost) != cudaSuccess) {
                st = ART_E_CUDA;
                break;
            }
            // per SM: CTAs run, earliest start, latest end
            int nsm_ids = 0;
            for (int b = 0; b < nb; b++) nsm_ids = std::max(nsm_ids, int(h[3 * b + 2]) + 1);
            std::vector<long long> lo(nsm_ids, 0), hi(nsm_ids, 0);
            std::vector<int> cnt(nsm_ids, 0);
            for (int b = 0; b < nb; b++) {
                const int s = int(h[3 * b + 2]);
                lo[s] = cnt[s] ? std::min(lo[s], h[3 * b]) : h[3 * b];
                hi[s] = cnt[s] ? std::max(hi[s], h[3 * b + 1]) : h[3 * b + 1];
                cnt[s]++;
            }
            std::vector<double> rate;
            for (int s = 0; s < nsm_ids; s++)
                if (cnt[s] && hi[s] > lo[s])
                    rate.push_back(double(cnt[s]) * nt * iters * 8 * (op == 3 ? 2 : 1) / double(hi[s] - lo[s]));
            if (rate.empty()) continue;
            std::nth_element(rate.begin(), rate.begin() + rate.size() / 2, rate.end());
            const double v = rate[rate.size() / 2];
            best = v > best ? v : best;
        }
        *res[op] = best;
    }
    cudaFree(out);
    cudaFree(cyc);
    return st;
}
