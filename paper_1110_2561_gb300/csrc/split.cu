// split.cu -- split-and-convolve enumeration on the device (the identity and the program layout
// are in split_internal.h): one CTA per configuration s of the boundary set S at a time.
//
// Per s (half of them: the other half are their global-flip mirrors), a CTA computes the boundary
// energy and up count, then for each component C_c the field
// S exerts on each of its spins, walks the 2^|C_c| configurations of C_c (up to 512 threads, each
// a reflected Gray walk over the low bits with its thread index in the top bits) into a 32-bit
// shared histogram, and convolves that histogram into the CTA's accumulator: the nonzero bins of
// both are listed, lanes hold a few accumulator bins in registers while the warps take the
// histogram bins in turn, and every product is a shared-memory reduction into the next
// accumulator.
// The accumulator, shifted by the boundary's bin, is added into the CTA's int64 table in shared
// memory, which is flushed to the output with 64-bit atomics at the end.
//
// The enumeration walks visit 2^(|S|-1) * sum_c 2^|C_c| configurations instead of 2^N; the
// convolutions are exact integer arithmetic, so the table equals the full enumeration's.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "isg_internal.h"
#include "nvtx_range.h"
#include "split_internal.h"

namespace isg {

DeviceInfo device_info();

struct SplitArgs {
    const uint64_t* blob;          // device program
    int blob_words;
    unsigned long long* table;     // (S + 1)(N + 1) counts, accumulated into
    unsigned int* status;          // bit 0: a walk lost track of its bin
    unsigned long long n_s;        // 2^|S|
};

__device__ __forceinline__ int warp_sum_i(int v) {
#pragma unroll
    for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// sum_t J_t (2 popc(m_t & bits) - popc(m_t)) over the classes' masks m_t = masks[t * stride]
__device__ __forceinline__ int split_field(const int64_t* cls, int ncl, const uint64_t* masks, int stride, uint64_t bits) {
    int f = 0;
    for (int t = 0; t < ncl; ++t) {
        const uint64_t m = masks[t * stride];
        f += (int)cls[t] * (2 * __popcll(m & bits) - __popcll(m));
    }
    return f;
}

// A warp's accumulator buffer of `words` bins. 32-bit counts: one word per bin. 64-bit counts: a
// plane of low words then a plane of high words (the same 8 bytes per bin), so that every update is
// a 32-bit shared atomic: 64-bit shared atomics are several times slower on this GPU, and far
// slower when lanes collide. An addition's carry out of the low word is detected from the value
// the atomic returns and added to the high word with the value's own high half.
template <class Acc>
struct AccBuf {
    uint32_t* lo;
    uint32_t* hi;
    __device__ AccBuf(void* base, int words)
        : lo(static_cast<uint32_t*>(base)), hi(sizeof(Acc) == 8 ? static_cast<uint32_t*>(base) + words : nullptr) {}
    __device__ Acc get(int i) const {
        if (sizeof(Acc) == 8) return (Acc)(((unsigned long long)hi[i] << 32) | lo[i]);
        return (Acc)lo[i];
    }
    __device__ void set(int i, Acc v) const {
        lo[i] = (uint32_t)v;
        if (sizeof(Acc) == 8) hi[i] = (uint32_t)((unsigned long long)v >> 32);
    }
    __device__ void add(int i, Acc v) const {
        if (sizeof(Acc) == 8) {
            const unsigned long long w = (unsigned long long)v;
            const uint32_t vl = (uint32_t)w, vh = (uint32_t)(w >> 32);
            const uint32_t old = atomicAdd(&lo[i], vl);
            const uint32_t up = vh + (uint32_t)(old + vl < old);
            if (up) atomicAdd(&hi[i], up);
        } else {
            atomicAdd(&lo[i], (uint32_t)v);
        }
    }
};

// The low block of a component walk: from its all-down state, steps T = 1 .. 2^B - 1 of the
// reflected Gray code, unrolled at compile time (the flipped bit and its direction are
// constants): one add and one shared reduction per configuration. The shared byte address `addr`
// of the current bin (e MC + m, MC the histogram's row stride) moves by +-G[k] = +-4 (h_k MC - 1)
// when low spin k flips (e by +-h_k, m by -+1), h_k the field on low spin k, constant over the
// block because low spins have no bond among them. The address is an in/out operand of the
// reduction, so the chain of addresses stays in step with the reductions.
template <int B, int T>
__device__ __forceinline__ void split_low_steps(uint32_t& addr, const int (&G)[B]) {
    if constexpr (T < (1 << B)) {
        constexpr int k = split_ctz(T);
        constexpr bool was_up = (split_gray(T - 1) >> k) & 1;
        addr += was_up ? (uint32_t)G[k] : (uint32_t)-G[k];
        asm volatile("red.shared.add.u32 [%0], 1;" : "+r"(addr) : : "memory");
        split_low_steps<B, T + 1>(addr, G);
    }
}

// A walker's configurations with a low block of B spins: the mid bits (L - B of them) in Gray
// order, and at each mid state the low block from all down, its fields in registers, checked once
// against the histogram's range (a bin outside it would be a bug: recorded in bad, not written).
// x, e, m: the walker's configuration and its bin at the low block's all-down state. With kFew
// (the register-rich kernel, see split_kernel) the low spins' records {class-0 mask, class-1 mask,
// constant} are held in registers for the whole walk, so their fields at each mid state cost two
// popcounts each and no shared-memory load (on the 8x8 torus those loads were about a tenth of
// the walk's shared-memory wavefronts).
template <int B, bool kFew, class Field>
__device__ __forceinline__ void split_walk_low(uint32_t& x, int& e, int& m, int L, int nc, int Sc, int MC, uint32_t hs,
                                               const Field& field, const uint4* wsp, int J0, int J1, bool& bad) {
    uint4 lr[kFew ? B : 1];
    if constexpr (kFew) {
#pragma unroll
        for (int j = 0; j < B; ++j) lr[j] = wsp[j];
    }
    auto low_field = [&](int j) -> int {
        if constexpr (kFew) return 2 * (J0 * __popc(lr[j].x & x) + J1 * __popc(lr[j].y & x)) + (int)lr[j].z;
        else return field(j, x);
    };
    for (uint32_t tm = 0; tm < (1u << (L - B)); ++tm) {
        if (tm) {
            const int k = B + __ffs(tm) - 1;         // the same spin in every walker
            const bool up = (x >> k) & 1;
            const int hk = field(k, x);
            e += up ? hk : -hk;
            m += up ? -1 : 1;
            x ^= 1u << k;
        }
        int G[B];
        int lo = e, hi = e;
#pragma unroll
        for (int j = 0; j < B; ++j) {
            const int h = low_field(j);
            lo -= h > 0 ? h : 0;
            hi -= h < 0 ? h : 0;
            G[j] = 4 * (h * MC - 1);
        }
        if (lo >= 0 && hi <= Sc && m + B <= nc) {
            uint32_t addr = hs + 4u * (uint32_t)(e * MC + m);
            asm volatile("red.shared.add.u32 [%0], 1;" : "+r"(addr) : : "memory");
            split_low_steps<B, 1>(addr, G);
        } else {
            bad = true;
        }
    }
}

// kFew: at most two coupling classes (every lattice here: J = 1, or +-J), so a spin's field is
// two masked popcounts of a 32-bit component word and a constant; otherwise a loop over classes.
//
// One CTA (256 or 512 threads, from the program header) per boundary configuration at a time, in a grid-stride loop:
// the CTA's buffers (split_warp_layout) hold one accumulator pair, the lists and a histogram, so
// large components do not cut the number of warps per SM.
// kMinCtas: CTAs of 512 threads the register budget leaves room for per SM. 2 (at most 64
// registers a thread) for launches whose shared memory fits two or more CTAs per SM; 1 (up to 128)
// for those held to one CTA per SM by their buffers, which then also keep the low spins' records
// of the component walks in registers.
template <class Acc, bool kFew, int kMinCtas>
__global__ void __launch_bounds__(kSplitThreads, kMinCtas == 1 ? 1 : 0) split_kernel(const __grid_constant__ SplitArgs a) {
    extern __shared__ __align__(16) unsigned char sm[];
    uint64_t* prog = reinterpret_cast<uint64_t*>(sm);
    for (int i = threadIdx.x; i < a.blob_words; i += blockDim.x) prog[i] = a.blob[i];
    __syncthreads();
    const SplitView v = split_view(prog);
    const SplitHeader& H = *v.h;
    const int ncl = H.n_cls, MO = H.MO;
    // the CTA's table as 32-bit low and high words: 32-bit shared atomics, the carry of a low-word
    // addition detected from the value it returned
    unsigned int* tlo = reinterpret_cast<unsigned int*>(sm + split_prog_bytes(a.blob_words));
    unsigned int* thi = tlo + H.n_bins;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nwarps = blockDim.x >> 5;
    const SplitWarpLayout WL = split_warp_layout(H, sizeof(Acc) == 8);
    unsigned char* cbase = sm + split_prog_bytes(a.blob_words) + split_table_bytes(H);
    const AccBuf<Acc> bufA(cbase + WL.acc_a, H.acc_words), bufB(cbase + WL.acc_b, H.acc_words);
    uint64_t* hlist = reinterpret_cast<uint64_t*>(cbase + WL.hlist);
    uint32_t* list = reinterpret_cast<uint32_t*>(cbase + WL.list);
    uint32_t* hist = reinterpret_cast<uint32_t*>(cbase + WL.hist);
    uint4* wsp = reinterpret_cast<uint4*>(cbase + WL.spins);      // per component spin: masks, constant, field
    int* sc = reinterpret_cast<int*>(cbase + WL.scalars);          // [0] list length, [1] histogram list length, [2] e_SS
    const int J0 = (int)v.cls[0], J1 = ncl > 1 ? (int)v.cls[1] : 0;
    for (int i = tid; i < 2 * H.n_bins; i += blockDim.x) tlo[i] = 0;
    __syncthreads();
    auto table_add = [&](int i, unsigned long long val) {
        const unsigned int vl = (unsigned int)val, vh = (unsigned int)(val >> 32);
        const unsigned int old = atomicAdd(&tlo[i], vl);
        const unsigned int carry = (unsigned int)(old + vl < old);
        if (vh + carry) atomicAdd(&thi[i], vh + carry);
    };

    bool bad = false;
    // The global flip (every spin reversed) keeps E and negates M, so the boundary configurations
    // with the top boundary bit set give the mirror images of the others: only s < n_s / 2 are
    // walked and each result is added at M and at -M.
    const unsigned long long n_walk = H.ns ? a.n_s >> 1 : a.n_s;
    for (unsigned long long s = blockIdx.x; s < n_walk; s += gridDim.x) {
        // boundary: sum_j S_j a_j = -2 E_SS over its own bonds (warp 0); up count
        if (warp == 0) {
            int part = 0;
            for (int j = lane; j < H.ns; j += 32) {
                const int f = split_field(v.cls, ncl, v.ss + (size_t)j * ncl, 1, s);
                part += ((s >> j) & 1) ? f : -f;
            }
            part = warp_sum_i(part);
            if (lane == 0) sc[2] = (-part / 2 + H.S_SS) / 2;
        }
        AccBuf<Acc> acc = bufA, out = bufB;
        int rows = 0;
        if (H.n_comp == 0 && tid == 0) acc.set(0, (Acc)1);     // every spin is boundary: the empty convolution
        for (int c = 0; c < H.n_comp; ++c) {
            const SplitComp cp = v.comp[c];
            const int nc = cp.nc, MC = cp.hstride;   // bin (e, m) at e MC + m; columns m > nc are padding
            const uint64_t* sp = v.spin + (size_t)cp.first * ncl * 2;
            // component spin records: the field from the boundary (both paths), and with few
            // classes {mask of class 0, mask of class 1, f - J0 deg0 - J1 deg1} so that
            // field(x) = 2 (J0 popc(m0 & x) + J1 popc(m1 & x)) + constant
            if (tid < nc) {
                const int f = split_field(v.cls, ncl, sp + (size_t)tid * ncl * 2 + 1, 2, s);
                uint32_t m0 = 0, m1 = 0;
                if (kFew) {
                    m0 = (uint32_t)sp[(size_t)tid * ncl * 2];
                    m1 = ncl > 1 ? (uint32_t)sp[((size_t)tid * ncl + 1) * 2] : 0u;
                }
                wsp[tid] = make_uint4(m0, m1, (uint32_t)(f - J0 * __popc(m0) - J1 * __popc(m1)), (uint32_t)f);
            }
            for (int i = tid; i < cp.h_words; i += blockDim.x) hist[i] = 0;
            __syncthreads();
            // internal field plus boundary field of component spin q at configuration x
            auto field = [&](int q, uint32_t xx) -> int {
                if (kFew) {
                    const uint4 r = wsp[q];
                    return 2 * (J0 * __popc(r.x & xx) + J1 * __popc(r.y & xx)) + (int)r.z;
                }
                return split_field(v.cls, ncl, sp + (size_t)q * ncl * 2, 2, xx) + (int)wsp[q].w;
            };
            auto twice_energy = [&](uint32_t xx) {        // 2 E_c = -sum_q S_q (internal_q + 2 f_q)
                int t2 = 0;
                for (int q = 0; q < nc; ++q) {
                    const int hq = field(q, xx) + (int)wsp[q].w;
                    t2 -= ((xx >> q) & 1) ? hq : -hq;
                }
                return t2;
            };
            // walk: 2^P walker threads, each the reflected Gray walk over the low L = nc - P bits
            // with its index in the top P bits
            const int P = split_walk_bits(nc, cp.low, H.cta_bits), L = nc - P;
            if (tid < (1 << P)) {
                uint32_t x = (uint32_t)tid << L;
                int e = (twice_energy(x) / 2 + cp.Sc) / 2;
                int m = __popc(x);
                if (cp.low) {
                    const uint32_t hs = (uint32_t)__cvta_generic_to_shared(hist);
                    constexpr bool kRegLow = kFew && kMinCtas == 1;
                    if (cp.low == kSplitLowLarge)
                        split_walk_low<kSplitLowLarge, kRegLow>(x, e, m, L, nc, cp.Sc, MC, hs, field, wsp, J0, J1, bad);
                    else split_walk_low<kSplitLow, kRegLow>(x, e, m, L, nc, cp.Sc, MC, hs, field, wsp, J0, J1, bad);
                } else {
                    // a bin outside the histogram (a bug) is recorded and skipped, never written
                    auto count = [&](int ee, int mm) {
                        if ((unsigned)ee <= (unsigned)cp.Sc && (unsigned)mm <= (unsigned)nc) atomicAdd(&hist[ee * MC + mm], 1u);
                        else bad = true;
                    };
                    count(e, m);
                    for (uint32_t t = 1; t < (1u << L); ++t) {
                        const int k = __ffs(t) - 1;                      // the same spin in every walker
                        const bool up = (x >> k) & 1;
                        const int hk = field(k, x);
                        e += up ? hk : -hk;
                        m += up ? -1 : 1;
                        x ^= 1u << k;
                        count(e, m);
                    }
                }
                // self-check (the first warp's walkers): the tracked bin of the last configuration
                // (low bits all down in the low-block walk), recomputed
                if (tid < 32 && (e != (twice_energy(x) / 2 + cp.Sc) / 2 || m != __popc(x))) bad = true;
            }
            if (c == 0) {
                for (int i = tid; i < H.acc_words; i += blockDim.x) acc.set(i, (Acc)0);
                if (tid == 0) { sc[0] = 0; sc[1] = 0; }
                __syncthreads();
                for (int i = tid; i < cp.h_words; i += blockDim.x) {
                    const int e1 = i / MC, m1 = i - e1 * MC;
                    if (m1 <= nc) acc.set(e1 * MO + m1, (Acc)hist[i]);
                }
            } else {
                if (tid == 0) { sc[0] = 0; sc[1] = 0; }
                __syncthreads();
                // nonzero bins of the accumulator and of the histogram (order free: the products
                // are summed), and the next accumulator cleared
                const int used = (rows + 1) * MO;
                for (int i = tid; i < used; i += blockDim.x)
                    if (acc.get(i) != 0) list[atomicAdd(&sc[0], 1)] = (uint32_t)i;
                for (int i = tid; i < cp.h_words; i += blockDim.x) {
                    const uint32_t hv = hist[i];
                    if (hv) {
                        const int e1 = i / MC, m1 = i - e1 * MC;
                        hlist[atomicAdd(&sc[1], 1)] = (uint64_t)(uint32_t)(e1 * MO + m1) | ((uint64_t)hv << 32);
                    }
                }
                for (int i = tid; i < H.acc_words; i += blockDim.x) out.set(i, (Acc)0);
                __syncthreads();
                const int nl = sc[0], nh = sc[1];
                // out[a + shift] += count * acc[a] over all pairs: lanes hold up to kRegs accumulator
                // bins in registers, warps take the histogram bins in turn, every product is a
                // shared-memory reduction into the next accumulator
                constexpr int kRegs = sizeof(Acc) == 8 ? 4 : 8;
                for (int ch = 0; ch < nl; ch += 32 * kRegs) {
                    uint32_t li[kRegs];
                    Acc av[kRegs];
#pragma unroll
                    for (int k = 0; k < kRegs; ++k) {
                        const int q = ch + lane + 32 * k;
                        li[k] = q < nl ? list[q] : 0u;
                        av[k] = q < nl ? acc.get(li[k]) : (Acc)0;
                    }
                    for (int j = warp; j < nh; j += nwarps) {
                        const uint64_t hw = hlist[j];
                        const uint32_t hs = (uint32_t)hw;
                        const Acc hv = (Acc)(hw >> 32);
#pragma unroll
                        for (int k = 0; k < kRegs; ++k)
                            if (av[k]) out.add(li[k] + hs, hv * av[k]);
                    }
                }
                const AccBuf<Acc> t = acc;
                acc = out;
                out = t;
            }
            rows += cp.Sc;
            __syncthreads();
        }
        // shift by the boundary's bin and add into the CTA's table (and at -M: the flip mirror)
        const int e_SS = sc[2], m_S = __popcll(s);
        const int used = H.EO * MO;
        for (int i = tid; i < used; i += blockDim.x) {
            const Acc val = acc.get(i);
            if (val) {
                const int e1 = i / MO, m1 = i - e1 * MO;
                const int row = (e_SS + e1) * (H.n + 1);
                table_add(row + m_S + m1, (unsigned long long)val);
                if (H.ns) table_add(row + H.n - m_S - m1, (unsigned long long)val);
            }
        }
        __syncthreads();                      // the buffers and scalars are reused by the next s
    }
    if (bad) atomicOr(a.status, 1u);
    for (int i = tid; i < H.n_bins; i += blockDim.x) {
        const unsigned long long val = ((unsigned long long)thi[i] << 32) | tlo[i];
        if (val) atomicAdd(&a.table[i], val);
    }
}

}  // namespace isg

using namespace isg;

namespace isg {

// The kernels' dynamic shared-memory limit, raised once per device to the maximum (a per-launch
// attribute call costs microseconds, which a batch of small launches would feel; and it must not
// happen while a stream is being captured).
void split_prepare_launches() {
    static std::mutex mu;
    static std::vector<char> raised;
    int dev = 0;
    ISG_CUDA(cudaGetDevice(&dev));
    std::lock_guard<std::mutex> lk(mu);
    if ((int)raised.size() <= dev) raised.resize(dev + 1, 0);
    if (raised[dev]) return;
    const int lim = (int)device_info().smem_optin;
    const void* kernels[] = {
        reinterpret_cast<const void*>(split_kernel<uint32_t, true, 2>), reinterpret_cast<const void*>(split_kernel<uint32_t, false, 2>),
        reinterpret_cast<const void*>(split_kernel<unsigned long long, true, 2>),
        reinterpret_cast<const void*>(split_kernel<unsigned long long, false, 2>),
        reinterpret_cast<const void*>(split_kernel<uint32_t, true, 1>), reinterpret_cast<const void*>(split_kernel<uint32_t, false, 1>),
        reinterpret_cast<const void*>(split_kernel<unsigned long long, true, 1>),
        reinterpret_cast<const void*>(split_kernel<unsigned long long, false, 1>)};
    for (const void* k : kernels) ISG_CUDA(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, lim));
    raised[dev] = 1;
}

// Enqueue the split kernel for a prepared plan: program at d_blob (device), table (device,
// (S + 1)(N + 1) counts) accumulated into, status bit 0 set if a walk's self-check fails.
void launch_split(const SplitPrepared& prep, const uint64_t* d_blob, unsigned long long* table, unsigned int* status,
                  void* stream, int share) {
    const SplitHeader& H = *reinterpret_cast<const SplitHeader*>(prep.blob.data());
    const bool u64 = prep.plan.use_u64;
    const DeviceInfo d = device_info();
    const size_t smem = split_smem_bytes((int)prep.blob.size(), H, u64, 1);
    if (smem > (size_t)d.smem_optin) fail(ISG_ERR_TOO_LARGE, "split buffers exceed shared memory");
    // a grid of the CTAs that can be resident at once (registers and shared memory), never more
    // than boundary configurations: the grid-stride loop over them then balances by itself
    const int threads = 1 << H.cta_bits;
    const unsigned long long n_s = 1ull << H.ns;
    const unsigned long long n_walk = H.ns ? n_s >> 1 : n_s;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    SplitArgs a{d_blob, (int)prep.blob.size(), table, status, n_s};
    split_prepare_launches();
    // the register-rich variant where the 64-register one cannot have two CTAs per SM anyway
    auto launch = [&](auto kernel2, auto kernel1) {
        int ctas_per_sm = kernel_occupancy(reinterpret_cast<const void*>(kernel2), threads, smem);
        const int occ1 = ctas_per_sm <= 1 ? kernel_occupancy(reinterpret_cast<const void*>(kernel1), threads, smem) : 0;
        ctas_per_sm = std::max(1, std::max(ctas_per_sm, occ1));
        const unsigned long long resident = (unsigned long long)d.sms * ctas_per_sm;
        const int grid = (int)std::max<unsigned long long>(
            1, std::min<unsigned long long>(n_walk, std::max<unsigned long long>(1, resident / std::max(1, share))));
        if (occ1 >= 1) kernel1<<<grid, threads, smem, s>>>(a);
        else kernel2<<<grid, threads, smem, s>>>(a);
    };
    const bool few = H.n_cls <= 2;
    if (u64) {
        if (few) launch(split_kernel<unsigned long long, true, 2>, split_kernel<unsigned long long, true, 1>);
        else launch(split_kernel<unsigned long long, false, 2>, split_kernel<unsigned long long, false, 1>);
    } else {
        if (few) launch(split_kernel<uint32_t, true, 2>, split_kernel<uint32_t, true, 1>);
        else launch(split_kernel<uint32_t, false, 2>, split_kernel<uint32_t, false, 1>);
    }
    ISG_CUDA(cudaGetLastError());
}

}  // namespace isg

extern "C" isg_status isg_enumerate_split_batch(int32_t n, const isg_graph* const* graphs, void* stream,
                                                int64_t* const* g_out, int32_t g_out_on_device) {
    NvtxRange nvtx("isg_enumerate_split_batch");
    isg_options o;
    isg_options_init(&o);
    o.split = 1;
    o.max_spins = 62;
    return isg_enumerate_batch(n, graphs, stream, g_out, g_out_on_device, &o);
}

extern "C" isg_status isg_enumerate_split(const isg_graph* graph, void* stream, int64_t* g_out, int32_t g_out_on_device,
                                          uint64_t boundary) {
    return guarded([&] {
        NvtxRange nvtx("isg_enumerate_split");
        if (!graph || !g_out) fail(ISG_ERR_INVALID, "graph or g_out is NULL");
        const std::shared_ptr<const SplitPrepared> prep = prepare_split(*graph, boundary, true, true);
        const std::vector<uint64_t>& blob = prep->blob;
        const SplitHeader& H = *reinterpret_cast<const SplitHeader*>(blob.data());
        cudaStream_t s = static_cast<cudaStream_t>(stream);
        const size_t table_bytes = sizeof(int64_t) * (size_t)H.n_bins;
        const size_t blob_bytes = blob.size() * 8;
        // scratch: [status 16][program][table if host output]
        const size_t o_blob = 16, o_tab = (o_blob + blob_bytes + 255) & ~(size_t)255;
        char* scratch = static_cast<char*>(scratch_alloc(o_tab + (g_out_on_device ? 0 : table_bytes), s));
        struct Free {
            char* p; cudaStream_t s;
            ~Free() { if (p) cudaFreeAsync(p, s); }
        } guard{scratch, s};
        unsigned long long* table = g_out_on_device ? reinterpret_cast<unsigned long long*>(g_out)
                                                    : reinterpret_cast<unsigned long long*>(scratch + o_tab);
        ISG_CUDA(cudaMemsetAsync(scratch, 0, 16, s));
        ISG_CUDA(cudaMemcpyAsync(scratch + o_blob, blob.data(), blob_bytes, cudaMemcpyHostToDevice, s));
        ISG_CUDA(cudaMemsetAsync(table, 0, table_bytes, s));
        // host output: the call's own status word, read below; device output: the device's word,
        // which isg_device_status reports
        unsigned int* status = g_out_on_device ? device_status_word() : reinterpret_cast<unsigned int*>(scratch);
        launch_split(*prep, reinterpret_cast<const uint64_t*>(scratch + o_blob), table, status, s);
        if (!g_out_on_device) {
            unsigned int word = 0;
            ISG_CUDA(cudaMemcpyAsync(g_out, table, table_bytes, cudaMemcpyDeviceToHost, s));
            ISG_CUDA(cudaMemcpyAsync(&word, scratch, sizeof word, cudaMemcpyDeviceToHost, s));
            ISG_CUDA(cudaStreamSynchronize(s));
            check_self_check_word(word, "split enumeration");
        }
    });
}
