// Shared-memory atomic throughput of this GPU, for the second roofline of the
// pair kernel: its histogram updates are `red.shared.add.u32`, one per pair
// binned through the table (to the thread's own column) and a few per chunk
// settled by span.  One block of 1024 threads per SM (its shared memory
// request keeps a second block off the SM) issues a fixed number of
// reductions, either each thread to its own word (distinct banks within a
// warp) or every thread to one word; the SM clock counter times the block.
#include <cuda_runtime.h>

#include "wtheta_internal.h"

namespace {

constexpr int kThreads = 1024;
constexpr int kIters = 4096;
constexpr int kSmem = 160 * 1024;  // more than half an SM's shared memory

__global__ void __launch_bounds__(kThreads) k_shared_atomics(int same_address,
                                                             unsigned long long* cycles,
                                                             unsigned* sink) {
    extern __shared__ unsigned words[];
    words[threadIdx.x] = 0;
    __syncthreads();
    const unsigned a =
        (unsigned)__cvta_generic_to_shared(&words[same_address ? 0 : threadIdx.x]);
    const long long t0 = clock64();
#pragma unroll 8
    for (int i = 0; i < kIters; ++i) asm volatile("red.shared.add.u32 [%0], 1;" ::"r"(a) : "memory");
    __syncthreads();
    const long long t1 = clock64();
    if (threadIdx.x == 0) {
        atomicAdd(cycles, (unsigned long long)(t1 - t0));
        atomicAdd(sink, words[0]);
    }
}

}  // namespace

extern "C" int wtheta_probe_shared_atomics(int32_t same_address, double* per_sm_per_clock) {
    if (!per_sm_per_clock || (same_address != 0 && same_address != 1)) return WTHETA_EINVAL;
    wtheta::DeviceInfo di;
    int rc = wtheta::device_info(&di);
    if (rc) return rc;
    unsigned long long* d = nullptr;
    if ((rc = wtheta::check_cuda(cudaFuncSetAttribute(
             k_shared_atomics, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmem))))
        return rc;
    if ((rc = wtheta::check_cuda(cudaMalloc(&d, 16)))) return rc;
    rc = wtheta::check_cuda(cudaMemset(d, 0, 16));
    for (int rep = 0; rep < 2 && !rc; ++rep) {  // the first launch warms up
        if (!rc) rc = wtheta::check_cuda(cudaMemset(d, 0, 16));
        k_shared_atomics<<<di.sm_count, kThreads, kSmem>>>(same_address, d, (unsigned*)(d + 1));
        wtheta::add_launches(1);
        if (!rc) rc = wtheta::check_cuda(cudaGetLastError());
        if (!rc) rc = wtheta::check_cuda(cudaDeviceSynchronize());
    }
    unsigned long long cyc = 0;
    if (!rc) rc = wtheta::check_cuda(cudaMemcpy(&cyc, d, 8, cudaMemcpyDeviceToHost));
    cudaFree(d);
    if (rc) return rc;
    // warp-wide reductions per SM per clock, averaged over the blocks (one per SM)
    const double warps = kThreads / 32.0;
    const double mean_cycles = (double)cyc / (double)di.sm_count;
    *per_sm_per_clock = warps * kIters / mean_cycles;
    return WTHETA_OK;
}
