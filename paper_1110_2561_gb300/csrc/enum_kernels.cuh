// enum_kernels.cuh -- the device code of the enumeration kernels (enumerate.cu holds their host
// side): the Gray walk of enum_core.cuh per lane, counting into privatised 32-bit shared-memory
// bins that a CTA-wide flush adds into the int64 table (arXiv:1110.2561, Sec. 2-3).
#pragma once
#include <cuda_runtime.h>

#include <cstdint>

#include "enum_core.cuh"

namespace isg {

// Counts one configuration at a shared-memory byte address. The address is an in/out operand so
// the compiler keeps the Gray chain of addresses in step with the reductions instead of
// computing the whole unrolled block of addresses ahead (which exhausts registers).
struct SmemSink {
    __device__ __forceinline__ void operator()(uint32_t& addr) const {
        asm volatile("red.shared.add.u32 [%0], 1;" : "+r"(addr) : : "memory");
    }
};

// Warp-aggregated counting: lanes holding the same address elect one lane, which adds the
// number of such lanes. Kept to measure against SmemSink: on GB300 match.any issues far more
// slowly than the reduction it saves.
struct MatchSink {
    __device__ __forceinline__ void operator()(uint32_t& addr) const {
        const unsigned peers = __match_any_sync(0xffffffffu, addr);
        const int leader = __ffs(static_cast<int>(peers)) - 1;
        if ((int)(threadIdx.x & 31) == leader) {
            const unsigned cnt = static_cast<unsigned>(__popc(peers));
            asm volatile("red.shared.add.u32 [%0], %1;" : "+r"(addr) : "r"(cnt) : "memory");
        }
    }
};

struct EnumArgs {
    const uint64_t* blob;
    int64_t* g;                     // public table (n_e * n_m int64)
    unsigned long long* counter;    // next task
    unsigned int* status;           // bit 0: a lane's tracked bin disagreed with its recomputation
    uint64_t prefix_base;           // first lane prefix
    uint64_t n_tasks;
    int32_t blob_words;
    int32_t copies;
    int32_t flush_rounds;
    int32_t copy_words;              // words of one histogram copy
    int32_t n_sub;                   // sub-tables per copy (1, or kLaneTables for lane tables)
    int32_t sub_off[kLaneTables];    // bin (e', m) of sub-table t is word sub_off[t] + e' stride + m,
    int32_t sub_m_lo[kLaneTables];   // for the columns m in [sub_m_lo[t], sub_m_hi[t]] only (the
    int32_t sub_m_hi[kLaneTables];   // other words of those rows may be another sub-table's)
    int32_t lane_word[32];           // lane l counts into the sub-table starting lane_word[l] words into its copy
    int32_t pad;
};

__device__ __forceinline__ void stage_blob(uint64_t* dst, const uint64_t* src, int words) {
    for (int i = threadIdx.x; i < words; i += blockDim.x) dst[i] = src[i];
}

// Programs up to this many words travel inside the kernel parameters (no host-to-device copy);
// every graph of up to 64 spins with at most two weight classes fits.
constexpr int kInlineProgramWords = 512;

struct EnumParams {
    EnumArgs a;                                 // a.blob == NULL: the program is in `program`
    uint64_t program[kInlineProgramWords];
};

// Add the CTA's privatised bins (every sub-table of every copy) into the public int64 table and
// clear them. Thread i takes bin (e', m) = (i / n_m, i % n_m) of every sub-table holding column m.
__device__ __forceinline__ void flush_bins(const ProgHeader* hd, uint32_t* hist, const EnumArgs& a, int64_t* g) {
    const int n_m = hd->n_m, R = hd->stride, nb = hd->n_e_c * n_m;
    for (int i = threadIdx.x; i < nb; i += blockDim.x) {
        const int ec = i / n_m, m = i - ec * n_m;
        unsigned long long s = 0;
        for (int c = 0; c < a.copies; ++c)
            for (int t = 0; t < a.n_sub; ++t)
                if (m >= a.sub_m_lo[t] && m <= a.sub_m_hi[t]) {
                    uint32_t& w = hist[c * a.copy_words + a.sub_off[t] + ec * R + m];
                    s += w;
                    w = 0;
                }
        if (s) {
            const int64_t e = (hd->e_lo + (int64_t)hd->G * ec + hd->S) / 2;
            atomicAdd(reinterpret_cast<unsigned long long*>(g + e * n_m + m), s);
        }
    }
}

template <int B, class Sink>
__global__ void __launch_bounds__(1024) enumerate_kernel(const __grid_constant__ EnumParams P) {
    const EnumArgs& a = P.a;
    extern __shared__ __align__(16) uint64_t smem[];
    stage_blob(smem, a.blob ? a.blob : P.program, a.blob_words);
    uint32_t* hist = reinterpret_cast<uint32_t*>(smem + ((a.blob_words + 1) & ~1));
    __shared__ int s_done;
    if (threadIdx.x == 0) s_done = 0;
    __syncthreads();
    const ProgHeader* hd = reinterpret_cast<const ProgHeader*>(smem);
    const ProgView v = make_view(smem);
    for (int i = threadIdx.x; i < a.copies * a.copy_words; i += blockDim.x) hist[i] = 0;
    __syncthreads();

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t base = static_cast<uint32_t>(
        __cvta_generic_to_shared(hist + (warp % a.copies) * a.copy_words + a.lane_word[lane]));
    Sink sink;
    bool done = false;
    for (;;) {
        for (int r = 0; r < a.flush_rounds; ++r) {
            unsigned long long t = 0;
            if (lane == 0) t = atomicAdd(a.counter, 1ull);
            t = __shfl_sync(0xffffffffu, t, 0);
            if (t >= a.n_tasks) { done = true; break; }
            uint64_t last_state;
            uint32_t last_idx;
            lane_walk<B>(v, a.prefix_base + t * 32 + lane, base, sink, last_state, last_idx);
            if (last_idx != base + bin_offset(v, last_state)) atomicOr(a.status, 1u);
        }
        if (done) s_done = 1;
        __syncthreads();
        flush_bins(hd, hist, a, a.g);
        __syncthreads();
        if (s_done) break;
    }
}

// Small graphs (fewer than 11 free spins): one thread per configuration, counted straight into
// the int64 table.
__global__ void enumerate_small_kernel(const __grid_constant__ EnumParams P, uint64_t s_lo, uint64_t s_hi) {
    const int words = P.a.blob_words;
    int64_t* g = P.a.g;
    extern __shared__ __align__(16) uint64_t smem[];
    stage_blob(smem, P.a.blob ? P.a.blob : P.program, words);
    __syncthreads();
    const ProgHeader* hd = reinterpret_cast<const ProgHeader*>(smem);
    const ProgView v = make_view(smem);
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t s = s_lo + (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; s < s_hi; s += stride) {
        const int64_t i = bin_offset(v, s) >> 2;
        const int64_t ec = i / hd->stride, m = i - ec * hd->stride;
        const int64_t e = (hd->e_lo + hd->G * ec + hd->S) / 2;
        atomicAdd(reinterpret_cast<unsigned long long*>(g + e * hd->n_m + m), 1ull);
    }
}

// Symmetry completion: out (=/+=) half(E, M) + half(E, -M), where half counts the configurations
// with spin N-1 up (a global flip keeps E and negates M).
__global__ void mirror_kernel(const int64_t* half, int64_t* out, int n_e, int n_m, int accumulate) {
    const int total = n_e * n_m;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < total; i += gridDim.x * blockDim.x) {
        const int e = i / n_m, m = i - e * n_m;
        const int64_t v = half[i] + half[(size_t)e * n_m + (n_m - 1 - m)];
        out[i] = accumulate ? out[i] + v : v;
    }
}

}  // namespace isg
