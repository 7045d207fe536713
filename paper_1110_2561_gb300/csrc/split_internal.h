// split_internal.h -- split-and-convolve enumeration: the plan, the program layout shared by the
// host (planner, program builder, emulation) and the device kernel.
//
// The method (a variant of the paper's full enumeration, Sec. 3, that visits fewer than 2^N
// configurations): a boundary set S of spins is chosen whose removal leaves components C_1..C_k
// with no bond between different components. For a fixed configuration s of S the components are
// independent, so
//   g(E, M) = sum_s  delta(E_SS(s), M_S(s)) * conv_c h_c(. | s),
// where h_c(e_c, m_c | s) counts the configurations of C_c by their energy (bonds inside C_c and
// between C_c and S, the latter through the field S exerts on each spin of C_c) and up count, and
// conv is the 2-D convolution over (energy, up count). Bins: with S_c = sum |J| over the bonds
// touching C_c, e_c = (E_c + S_c) / 2 in [0, S_c], m_c in [0, |C_c|]; the S part has
// e_SS = (E_SS + S_SS) / 2, m_S = popcount(s); the table bin is (e_SS + sum e_c, m_S + sum m_c),
// which is the public bin ((E + S) / 2, up count) because every bond lies in S x S, inside one
// component, or between one component and S.
#pragma once
#include <cstddef>
#include <cstdint>
#include <memory>
#include <vector>

#include "../../include/isg.h"

#ifdef __CUDACC__
#define ISG_SPLIT_HD __host__ __device__
#else
#define ISG_SPLIT_HD
#endif

namespace isg {

constexpr int kSplitMaxClasses = 16;     // distinct signed couplings
constexpr int kSplitMaxComp = 64;
constexpr int kSplitMaxCompSpins = 30;   // a component's configurations fit a 32-bit word walk
constexpr int kSplitThreads = 512;       // threads of a split CTA (one boundary configuration at a time)
constexpr int kSplitWalkBits = 9;        // at most 2^9 = 512 walkers per component (one per thread)
constexpr int kSplitLow = 5;             // size of a component walk's low block ...
constexpr int kSplitLowLarge = 7;        // ... or of the larger one, where a component has room for it
constexpr int kSplitLowMinSpins = 12;    // components given a low block: at least this many spins
constexpr int kSplitLaneModelMinSpins = 16;   // components whose lane spins the conflict model may choose
// Warp instructions per configuration of the full enumeration (ncu on the 6x6 torus: 2.86 per 32
// configurations): the unit in which the planner compares a split with the full enumeration.
constexpr double kDirectWarpInstrPerConfig = 2.86 / 32;
// The fixed cost of one split launch among many (host enqueue, table clear, a small grid's ramp):
// about 20 us, in warp instructions of the whole GPU at full issue.
constexpr double kSplitLaunchWarpInstr = 2.5e7;

// Walker bits P of a component of nc spins: 2^P walkers (every thread of the CTA where the
// component is large enough: idle threads cost more than short walks), each walking
// 2^(nc - P) configurations, and at least its low block when it has one.
ISG_SPLIT_HD inline int split_walk_bits(int nc, int low, int cta_bits) {
    const int cap = nc - low;
    return cap < cta_bits ? (cap < 0 ? 0 : cap) : cta_bits;
}

// Low-block size wanted for a component of nc spins in CTAs of 2^cta_bits threads: the larger
// block where the component still has a bit for every thread above it (its mid states are then
// fewer per configuration: 1 in 128), else the smaller one from kSplitLowMinSpins spins, else
// none. The program builder falls back to a smaller block when no such independent set exists.
ISG_SPLIT_HD inline int split_low_want(int nc, int cta_bits) {
    return nc - kSplitLowLarge >= cta_bits ? kSplitLowLarge : (nc >= kSplitLowMinSpins ? kSplitLow : 0);
}

// Row stride of a component histogram: nc + 1, padded (by at most 10) so that the rows a walk
// uses, every rs-th one, lie a good bank distance apart. rs is the largest power of two dividing
// every energy step of the component (2 on the tori: all fields are even, so a walk keeps one
// parity of e). The walkers of a warp differ in five spins, so their bins differ by a few rows and
// columns; a row distance of 5-7, 9, 11, 13, 19, 21, 23 or 25-27 banks (mod 32) sends the common
// small offsets to distinct banks. With no such stride within reach (rs >= 4) the rows stay
// unpadded.
ISG_SPLIT_HD inline int split_hist_stride(int nc, int rs) {
    for (int s = nc + 1; s <= nc + 32; ++s) {
        const int r = (rs * s) & 31;
        if ((r >= 5 && r <= 7) || r == 9 || r == 11 || r == 13 || r == 19 || r == 21 || r == 23 || (r >= 25 && r <= 27))
            return s;
    }
    return nc + 1;
}

// Threads per split CTA: 256 (up to four CTAs per SM, so one waits at a barrier while others
// issue) when four CTAs' shared memory fits an SM, else 512.
inline int split_cta_bits(size_t cta_smem_bytes) { return 4 * (cta_smem_bytes + 1024) <= 233472 ? 8 : kSplitWalkBits; }

// Compile-time bit helpers for the unrolled low block (reflected Gray code: step t flips bit
// ctz(t); the state after step t is gray(t)).
ISG_SPLIT_HD constexpr int split_ctz(int x) { return (x & 1) ? 0 : 1 + split_ctz(x >> 1); }
ISG_SPLIT_HD constexpr int split_popc(int x) { return x ? (x & 1) + split_popc(x >> 1) : 0; }
ISG_SPLIT_HD constexpr int split_gray(int t) { return t ^ (t >> 1); }

// Program header (32-bit words at the start of the blob).
struct SplitHeader {
    int32_t n, ns, n_comp, n_cls;        // spins, boundary spins, components, coupling classes
    int32_t S_total, S_SS, EO, MO;       // sum |J|; S x S part; convolution rows (sum S_c + 1), row stride (sum |C_c| + 1)
    int32_t off_cls, off_ss, off_comp, off_spin;   // 64-bit word offsets of the sections below
    int32_t max_h, acc_words, n_bins;    // largest component histogram; accumulator words per buffer; (S+1)(N+1)
    int32_t cta_bits;                    // log2 of the threads of a CTA (8: 256, four CTAs per SM; 9: 512)
};
static_assert(sizeof(SplitHeader) == 64, "header is 8 words");

// Per component (four 64-bit words).
struct SplitComp {
    int32_t nc, Sc, first, h_words;      // spins, sum |J| touching it, index of its first spin record, (Sc+1) hstride
    int32_t low;                         // kSplitLow or kSplitLowLarge: local bits 0..low-1 are mutually unbonded (a low block); else 0
    int32_t hstride;                     // histogram row stride (>= nc + 1): bin (e, m) at e hstride + m
    int32_t reserved[2];
};

// Sections (64-bit words):
//   cls[n_cls]                 signed coupling of each class (int64)
//   ss[ns * n_cls]             for boundary spin j and class t: mask over boundary bits of its boundary
//                              neighbours with that coupling
//   comp[4 n_comp]             SplitComp records (four words each)
//   spin[(sum nc) * 2 n_cls]   for component spin k (components in order) and class t: mask over the
//                              component's own bits (internal neighbours), then mask over boundary bits
struct SplitView {
    const SplitHeader* h;
    const int64_t* cls;
    const uint64_t* ss;
    const SplitComp* comp;
    const uint64_t* spin;
};

ISG_SPLIT_HD inline SplitView split_view(const uint64_t* blob) {
    SplitView v;
    v.h = reinterpret_cast<const SplitHeader*>(blob);
    v.cls = reinterpret_cast<const int64_t*>(blob + v.h->off_cls);
    v.ss = blob + v.h->off_ss;
    v.comp = reinterpret_cast<const SplitComp*>(blob + v.h->off_comp);
    v.spin = blob + v.h->off_spin;
    return v;
}

// Field on a spin from the spins in `bits` that its masks select: sum_t J_t (2 popc(mask_t & bits)
// - popc(mask_t)), i.e. sum over those neighbours of J * S_j with S_j = +1 for a set bit.
ISG_SPLIT_HD inline int64_t split_popc64(uint64_t x) {
#ifdef __CUDA_ARCH__
    return __popcll(x);
#else
    return __builtin_popcountll(x);
#endif
}

struct SplitPlan {
    uint64_t boundary = 0;               // mask of boundary spins (graph indices)
    std::vector<int> S;                  // boundary spins, boundary bit j <-> S[j]
    std::vector<std::vector<int>> comps; // component spins, local bit k <-> comps[c][k]
    double visits = 0;                   // configurations walked: 2^(|S|-1) * sum 2^|C_c| (flip mirrors)
    double cost = 0, direct_cost = 0;    // model of the work, and of the full enumeration
    bool use_u64 = false;                // accumulator counts may exceed 31 bits
    int cta_bits = kSplitWalkBits;       // log2 of the threads per CTA
    int warps = 0;                       // warps per CTA whose buffers fit shared memory
};

// Host side (split_host.cpp).
// boundary = 0: the cheapest admissible boundary set; with require_gain, refused (TOO_LARGE) unless
// it is cheaper than the full enumeration under the work model.
SplitPlan plan_split(const struct ::isg_graph& g, uint64_t boundary, bool require_gain);
std::vector<uint64_t> build_split_program(const struct ::isg_graph& g, const SplitPlan& p, bool lane_model);
void emulate_split(const std::vector<uint64_t>& blob, int64_t* g_out);

// A plan and its program for one graph content and boundary argument (cached).
struct SplitPrepared {
    int n = 0;
    std::vector<int32_t> bi, bj;
    std::vector<int64_t> bJ;
    uint64_t boundary_arg = 0;
    bool require_gain = false;
    bool lane_model = false;
    SplitPlan plan;
    std::vector<uint64_t> blob;
};
// lane_model: the walkers' lane spins and row strides of components of at least
// kSplitLaneModelMinSpins spins chosen by the bank-conflict model (a search per component
// structure, cached); without it the component order and the fixed stride preference.
std::shared_ptr<const SplitPrepared> prepare_split(const struct ::isg_graph& g, uint64_t boundary, bool require_gain,
                                                   bool lane_model);

// Device side (split.cu): enqueue the split kernel for a prepared plan on `stream` (a
// cudaStream_t); program at d_blob, table (device) accumulated into, status bit 0 on a failed
// self-check. share > 1: the launch runs beside share - 1 others of its kind (a batch's parallel
// branches), so its grid takes a 1/share part of the CTAs the GPU holds at once (each CTA then
// walks more boundary configurations for its fixed costs, and the launches overlap).
void launch_split(const SplitPrepared& prep, const uint64_t* d_blob, unsigned long long* table, unsigned int* status,
                  void* stream, int share = 1);
// Set the split kernels' launch attributes on the current device (once; call before any capture).
void split_prepare_launches();

// Shared memory of the split kernel: the program, the CTA's table (32-bit low and high words per
// bin), then the CTA's working block (16-byte aligned): 32 component-spin records, scalars, two
// accumulators, the histogram's nonzero
// list (8-byte entries), the accumulator's nonzero list and a component histogram (4-byte
// entries). The 8-byte arrays come first so that they stay 8-byte aligned whatever the sizes.
struct SplitWarpLayout {
    size_t spins, scalars, acc_a, acc_b, hlist, list, hist, bytes;   // byte offsets within the block; its size
};
ISG_SPLIT_HD inline SplitWarpLayout split_warp_layout(const SplitHeader& h, bool u64) {
    SplitWarpLayout L;
    const size_t acc = (u64 ? 8 : 4) * (size_t)h.acc_words;
    L.spins = 0;                                      // 32 records of 16 bytes (component spins)
    L.scalars = 512;                                  // a few ints shared by the CTA
    L.acc_a = 768;
    L.acc_b = L.acc_a + ((acc + 7) & ~(size_t)7);
    L.hlist = L.acc_b + ((acc + 7) & ~(size_t)7);
    L.list = L.hlist + 8 * (size_t)h.max_h;
    L.hist = L.list + 4 * (size_t)h.acc_words;
    L.bytes = (L.hist + 4 * (size_t)h.max_h + 15) & ~(size_t)15;
    return L;
}
ISG_SPLIT_HD inline size_t split_prog_bytes(int blob_words) { return ((size_t)blob_words * 8 + 15) & ~(size_t)15; }
ISG_SPLIT_HD inline size_t split_table_bytes(const SplitHeader& h) { return (8 * (size_t)h.n_bins + 15) & ~(size_t)15; }
ISG_SPLIT_HD inline size_t split_warp_bytes(const SplitHeader& h, bool u64) { return split_warp_layout(h, u64).bytes; }
ISG_SPLIT_HD inline size_t split_smem_bytes(int blob_words, const SplitHeader& h, bool u64, int warps) {
    return split_prog_bytes(blob_words) + split_table_bytes(h) + (size_t)warps * split_warp_bytes(h, u64);
}

}  // namespace isg
