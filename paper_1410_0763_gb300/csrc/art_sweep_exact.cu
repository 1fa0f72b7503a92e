// art_sweep_exact.cu -- the sweep kernels with the exact path average
// (ART_AVG_EXACT), instantiated for every variant in a translation unit of
// their own so that they compile in parallel with the paper-average kernels.
#include <cuda_runtime.h>

#include "art.h"
#include "art_ctx.hpp"
#include "art_kernels.cuh"

using namespace art;

template <typename real, int TB, int TC, int BLK, int NT, int KP, int MINB>
cudaError_t art_launch_exact(const cudaLaunchConfig_t &cfg, const SweepArgs<real> &a)
{
    if (a.counter) return cudaLaunchKernelEx(&cfg, sweep_queue_kernel<real, TB, TC, BLK, NT, KP, MINB, 1>, a);
    return cudaLaunchKernelEx(&cfg, sweep_block_kernel<real, TB, TC, BLK, NT, KP, MINB, 1>, a);
}

template <typename real, int TB, int TC, int BLK, int NT, int KP, int MINB> cudaError_t art_prepare_exact(int smem)
{
    cudaError_t e = cudaFuncSetAttribute(sweep_block_kernel<real, TB, TC, BLK, NT, KP, MINB, 1>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(sweep_queue_kernel<real, TB, TC, BLK, NT, KP, MINB, 1>,
                                cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
}

#define ART_VARIANT(real, pr, tb, tc, blk, nt, kp, mb)                                                   \
    template cudaError_t art_launch_exact<real, tb, tc, blk, nt, kp, mb>(const cudaLaunchConfig_t &,     \
                                                                          const SweepArgs<real> &);      \
    template cudaError_t art_prepare_exact<real, tb, tc, blk, nt, kp, mb>(int);
#include "art_variants.inc"
#undef ART_VARIANT
