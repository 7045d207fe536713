// probe.cu -- measured peaks of the units that bound the enumeration kernel: shared-memory
// 32-bit reductions (red.shared.add.u32) with conflict-free and with scattered addresses, and
// integer ALU issue. Each warp works on its own 2048-word table; every address is masked into
// it. The rates are lane-operations per second over the whole GPU, timed with CUDA events.
#include <cuda_runtime.h>

#include <string>

#include "isg_internal.h"

namespace isg {

constexpr int kProbeWords = 2048;   // words per warp table (power of two); two warps share one

// MODE 3: MODE 1's addresses, aggregated first: __match_any_sync, one leader lane per address
// adds the count (what a warp-aggregated histogram does per configuration).
// MODE 0: each lane adds to 32 words of its own bank (lane + 32 j), addresses held in registers,
// so the loop is nothing but reductions. MODE 1: 32 scattered per-lane addresses in registers
// (independent odd strides per lane), the same reductions with bank conflicts. MODE 2: integer
// ALU, four independent xor/add chains.
template <int MODE>
__global__ void __launch_bounds__(512) probe_kernel(int iters, unsigned* sink) {
    extern __shared__ unsigned tbl[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    unsigned* t = tbl + (warp >> 1) * kProbeWords;     // warps 2w and 2w+1 share table w
    for (int i = lane; i < kProbeWords; i += 32) t[i] = 0;
    __syncthreads();
    const uint32_t base = static_cast<uint32_t>(__cvta_generic_to_shared(t));
    unsigned x0 = lane, x1 = lane * 3u, x2 = lane * 5u, x3 = lane * 7u;
    if (MODE == 0 || MODE == 1 || MODE == 3) {
        uint32_t a[32];
        const unsigned s = ((lane * 2654435761u) >> 7) | 1u;
#pragma unroll
        for (int j = 0; j < 32; ++j)
            a[j] = base + 4u * (MODE == 0 ? (unsigned)(lane + 32 * j) : ((lane * 97u + j * s) & (kProbeWords - 1)));
        for (int i = 0; i < iters; i += 32) {
#pragma unroll
            for (int j = 0; j < 32; ++j) {
                if (MODE == 3) {
                    const unsigned peers = __match_any_sync(0xffffffffu, a[j]);
                    if (lane == __ffs(static_cast<int>(peers)) - 1)
                        asm volatile("red.shared.add.u32 [%0], %1;" ::"r"(a[j]), "r"((unsigned)__popc(peers)) : "memory");
                } else {
                    asm volatile("red.shared.add.u32 [%0], 1;" ::"r"(a[j]) : "memory");
                }
            }
        }
    } else {
        for (int i = 0; i < iters; ++i) {
            x0 = (x0 ^ x1) + i; x1 = (x1 ^ x2) + i; x2 = (x2 ^ x3) + i; x3 = (x3 ^ x0) + i;
        }
    }
    __syncthreads();
    unsigned tot = x0 + x1 + x2 + x3;
    for (int i = lane; i < kProbeWords; i += 32) tot += t[i];
    atomicAdd(sink, tot);
}

template <int MODE>
static double probe_rate(cudaStream_t s, unsigned* sink, int sms, double ops_per_iter) {
    const int threads = 512, iters = 1 << 16, per_sm = 3;   // 3 x 64 KB tables: 48 warps per SM
    const size_t smem = (size_t)(threads / 32) * kProbeWords * 4 / 2;
    ISG_CUDA(cudaFuncSetAttribute(probe_kernel<MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    probe_kernel<MODE><<<sms * per_sm, threads, smem, s>>>(iters, sink);      // warm-up
    ISG_CUDA(cudaGetLastError());
    cudaEvent_t e0, e1;
    ISG_CUDA(cudaEventCreate(&e0));
    ISG_CUDA(cudaEventCreate(&e1));
    ISG_CUDA(cudaEventRecord(e0, s));
    probe_kernel<MODE><<<sms * per_sm, threads, smem, s>>>(iters, sink);
    ISG_CUDA(cudaEventRecord(e1, s));
    ISG_CUDA(cudaEventSynchronize(e1));
    float ms = 0;
    ISG_CUDA(cudaEventElapsedTime(&ms, e0, e1));
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return (double)sms * per_sm * threads * iters * ops_per_iter / (ms * 1e-3);
}

}  // namespace isg

using namespace isg;

extern "C" isg_status isg_probe_peaks(void* stream, double* red_conflict_free, double* red_scattered, double* alu,
                                      double* match_aggregated) {
    return guarded([&] {
        cudaStream_t s = static_cast<cudaStream_t>(stream);
        int dev = 0, sms = 0;
        ISG_CUDA(cudaGetDevice(&dev));
        ISG_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
        unsigned* sink = nullptr;
        sink = static_cast<unsigned*>(scratch_alloc(4, s));
        const double r0 = probe_rate<0>(s, sink, sms, 1.0);
        const double r1 = probe_rate<1>(s, sink, sms, 1.0);
        const double r2 = probe_rate<2>(s, sink, sms, 8.0);
        const double r3 = match_aggregated ? probe_rate<3>(s, sink, sms, 1.0) : 0.0;
        ISG_CUDA(cudaFreeAsync(sink, s));
        ISG_CUDA(cudaStreamSynchronize(s));
        if (red_conflict_free) *red_conflict_free = r0;
        if (red_scattered) *red_scattered = r1;
        if (alu) *alu = r2;
        if (match_aggregated) *match_aggregated = r3;
    });
}
