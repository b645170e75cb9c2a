// FP32 FMA throughput of the GPU (a measurement aid, no counterpart in the
// paper): the denominator of the scan kernel's ALU roofline, measured on the
// machine instead of taken from unit counts.  Every thread runs CHAINS
// independent FMA chains, so each SM sub-partition always has independent FMAs
// to issue; the grid fills every SM at full occupancy.
#include <cuda_runtime.h>
#include <stdint.h>

#include "cdc_host.h"

namespace cdc {

constexpr int FFMA_CHAINS = 8;   // independent chains per thread (covers the FMA latency)
constexpr int FFMA_UNROLL = 16;  // FMAs per chain per loop iteration
constexpr int FFMA_BLOCK = 256;

__global__ void __launch_bounds__(FFMA_BLOCK) ffma_kernel(float a, float b, int iters, float* sink) {
    float x[FFMA_CHAINS];
#pragma unroll
    for (int i = 0; i < FFMA_CHAINS; ++i) x[i] = (float)(threadIdx.x + i) * 1.0e-3f;
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int k = 0; k < FFMA_UNROLL; ++k) {
#pragma unroll
            for (int i = 0; i < FFMA_CHAINS; ++i) x[i] = fmaf(x[i], a, b);
        }
    }
    float s = 0.f;
#pragma unroll
    for (int i = 0; i < FFMA_CHAINS; ++i) s += x[i];
    if (s == -1.0f) sink[blockIdx.x] = s;  // never true for the arguments used; keeps the chains live
}

cudaError_t launch_ffma(int num_sms, int iters, float* sink, cudaStream_t st, double* fma_count) {
    int occ = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, ffma_kernel, FFMA_BLOCK, 0);
    if (e != cudaSuccess) return e;
    const int blocks = num_sms * (occ > 0 ? occ : 1);
    ffma_kernel<<<blocks, FFMA_BLOCK, 0, st>>>(0.99999994f, 1.0e-7f, iters, sink);
    *fma_count = (double)blocks * FFMA_BLOCK * (double)iters * FFMA_UNROLL * FFMA_CHAINS;
    return cudaGetLastError();
}

}  // namespace cdc
