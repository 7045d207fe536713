// enum_core.cuh -- the per-thread Gray-code walk that visits 2^q configurations and counts each
// one into a histogram of (E, M) bins. Compiled twice: into the CUDA kernels (device) and into
// the host emulation that checks the same index arithmetic on the CPU.
//
// Method (arXiv:1110.2561): every configuration of N bit-packed spins is visited (Sec. 3, the
// nested loops over bit-vectors), its spin excess M comes from the number of up bits (Sec. 3a)
// and its energy from counting satisfied bonds with XOR / NOT / mask / popcount (Sec. 3b-3c).
// This walk orders the visits as a binary reflected Gray code, so consecutive configurations
// differ in one spin k and E changes by 2 S_k h_k with the local field h_k = sum_j J_kj S_j.
//
// Internal spin order. Positions 0..B-1 (the "low block") hold spins with no bond among
// themselves. Inside one low block the fields on those B spins come only from spins outside it,
// which stay fixed for 2^B consecutive visits; the bin address then moves by +-G_k per visit,
// with G_k a per-thread register and the sign known at compile time. A spin above the low block
// ("mid flip") is flipped every 2^B visits; its field is recomputed from the popcount of the
// configuration word against that spin's neighbour masks.
//
// Bin address. Reachable energies are E = e_lo + G e' with G >= 2 the energy stride of the graph
// (every single flip changes E by a multiple of G). The histogram stores bin (e', m) at byte
// offset 4 (e' R + m), m = number of up spins, R >= N + 1 the row stride. One unit of field moves
// the address by sE = 8 R / G bytes: dE = 2 S_k h_k gives de' = 2 S_k h_k / G, and dm = -S_k.
// R is padded so that lanes whose bins differ by a few rows and a few columns fall in different
// shared-memory banks (R = -1 mod 32, for instance, puts (e' + d, m + d) in the same bank). Lane
// tables instead take R a multiple of 32, so that a bin's bank depends on m alone, and count each
// lane into its own sub-table of the copy, offset so that the 32 lanes' banks differ (the walk
// only sees the lane's base address; enum_kernels.cuh and the planner lay the sub-tables out).
#pragma once
#include <cstdint>
#include <utility>

#if defined(__CUDACC__)
#define ISG_HD __host__ __device__ __forceinline__
#define ISG_CHD __host__ __device__
#else
#define ISG_HD inline
#define ISG_CHD
#endif

namespace isg {

constexpr int kMaxSpins = 64;
constexpr int kMaxClasses = 21;   // |J| <= 2^20 decomposes into at most 21 binary weights
constexpr int kMaxLow = 7;        // largest low block
// Lane tables: sub-tables per histogram copy when every lane's bank is fixed by its up count
// (the number of 5-bit lane values of the commonest popcount, C(5, 2))
constexpr int kLaneTables = 10;

// Per-spin record of a program, 48 bytes and 16-byte aligned, so a mid flip reads everything it
// needs about its spin with three 128-bit shared-memory loads.
struct alignas(16) SiteRec {
    uint64_t sgn;            // neighbours j with J_kj < 0
    uint64_t mask0;          // neighbours whose |J_kj| has weight class 0
    int32_t degw;            // sum_j |J_kj|
    int32_t A[kMaxLow];      // A[k] = -2 J_{k,this} sE for the low spins k (this spin outside the block)
};
static_assert(sizeof(SiteRec) == 48, "site record must be three 16-byte words");

// Program header, the first kHeaderWords words of a program blob (fields 32-bit unless noted).
struct ProgHeader {
    int32_t n;         // spins
    int32_t q;         // inner bits walked per thread: 2^q configurations per task lane
    int32_t b;         // low-block size
    int32_t nc;        // weight classes
    int32_t n_m;       // N + 1
    int32_t n_e_c;     // compact energy bins
    int32_t nbins_c;   // n_e_c * stride
    int32_t sE;        // address bytes per unit of field
    int32_t G;         // energy stride
    int32_t words;     // blob length in 64-bit words
    int64_t e_lo;      // energy of compact bin 0
    int64_t S;         // sum |J|; public bin e = (E + S) / 2
    int32_t off_site;  // word offsets: site records [n], extra class masks [n * (nc - 1)], weights [nc]
    int32_t off_maskx;
    int32_t off_w;
    int32_t stride;    // histogram row stride in bins (>= n_m), chosen against bank conflicts
    int32_t w0;        // weight of class 0
    int32_t pad;
};
constexpr int kHeaderWords = (int)(sizeof(ProgHeader) / 8);
static_assert(sizeof(ProgHeader) % 16 == 0, "program header must keep the site records 16-byte aligned");

// Read-only view of a program (in shared memory on the device, host memory in emulation).
struct ProgView {
    int n, q, b, nc, n_m, stride, sE, G, w0;
    int64_t e_lo;
    const SiteRec* site;     // [n]
    const uint64_t* maskx;   // [n * (nc - 1)] masks of classes 1.. (class c of spin k at k*(nc-1)+c-1)
    const int32_t* w;        // [nc] class weights
};

ISG_HD ProgView make_view(const uint64_t* blob) {
    const ProgHeader* h = reinterpret_cast<const ProgHeader*>(blob);
    ProgView v;
    v.n = h->n; v.q = h->q; v.b = h->b; v.nc = h->nc; v.n_m = h->n_m; v.stride = h->stride; v.sE = h->sE;
    v.G = h->G; v.w0 = h->w0;
    v.e_lo = h->e_lo;
    v.site = reinterpret_cast<const SiteRec*>(blob + h->off_site);
    v.maskx = blob + h->off_maskx;
    v.w = reinterpret_cast<const int32_t*>(blob + h->off_w);
    return v;
}

// The fields of one site record, read with three 128-bit loads on the device.
struct SiteVals {
    uint64_t sgn, mask0;
    int32_t degw;
    int32_t A[kMaxLow];
};

ISG_HD void load_site(const ProgView& p, int k, SiteVals& v) {
#if defined(__CUDA_ARCH__)
    const uint4* r = reinterpret_cast<const uint4*>(p.site + k);
    const uint4 a = r[0], b = r[1], c = r[2];
    v.sgn = (uint64_t)a.x | ((uint64_t)a.y << 32);
    v.mask0 = (uint64_t)a.z | ((uint64_t)a.w << 32);
    v.degw = (int32_t)b.x;
    v.A[0] = (int32_t)b.y; v.A[1] = (int32_t)b.z; v.A[2] = (int32_t)b.w;
    v.A[3] = (int32_t)c.x; v.A[4] = (int32_t)c.y; v.A[5] = (int32_t)c.z; v.A[6] = (int32_t)c.w;
#else
    const SiteRec& r = p.site[k];
    v.sgn = r.sgn;
    v.mask0 = r.mask0;
    v.degw = r.degw;
    for (int i = 0; i < kMaxLow; ++i) v.A[i] = r.A[i];
#endif
}

ISG_HD int popc64(uint64_t x) {
#if defined(__CUDA_ARCH__)
    return __popcll(x);
#else
    return __builtin_popcountll(x);
#endif
}

ISG_HD int ctz32(uint32_t x) {  // x != 0
#if defined(__CUDA_ARCH__)
    return __ffs(static_cast<int>(x)) - 1;
#else
    return __builtin_ctz(x);
#endif
}

// Compile-time helpers for the unrolled low block.
ISG_CHD constexpr int ctz_c(int u) { return (u & 1) ? 0 : 1 + ctz_c(u >> 1); }
ISG_CHD constexpr int gray_c(int u) { return u ^ (u >> 1); }

// Local field h_k = sum_j J_kj S_j of configuration st: a neighbour j with J_kj = +-w contributes
// +w when (bit_j XOR [J_kj < 0]) is 1 and -w otherwise (Sec. 3b: XOR, mask, count).
ISG_HD int field_of(const ProgView& p, const SiteVals& sv, uint64_t st, int k) {
    const uint64_t x = st ^ sv.sgn;
    int acc = p.w0 * popc64(x & sv.mask0);
#pragma unroll 1
    for (int c = 1; c < p.nc; ++c) acc += p.w[c] * popc64(x & p.maskx[k * (p.nc - 1) + c - 1]);
    return 2 * acc - sv.degw;
}

ISG_HD int field(const ProgView& p, uint64_t st, int k) {
    SiteVals sv;
    load_site(p, k, sv);
    return field_of(p, sv, st, k);
}

// Byte offset of the bin of configuration st, from scratch: E = -1/2 sum_k S_k h_k (Eq. 1 with
// each bond once), m = popcount (Sec. 3a).
ISG_HD uint32_t bin_offset(const ProgView& p, uint64_t st) {
    int64_t sum = 0;
#pragma unroll 1
    for (int k = 0; k < p.n; ++k) {
        const int h = field(p, st, k);
        sum += ((st >> k) & 1) ? h : -h;
    }
    const int64_t E = -sum / 2;
    const int64_t ec = (E - p.e_lo) / p.G;
    return static_cast<uint32_t>((ec * p.stride + popc64(st)) * 4);
}

// One Gray step inside a low block, fully resolved at compile time: step U flips spin k =
// ctz(U); its state before the flip is bit k of gray(U - 1), with spin B-1 inverted in ODD
// blocks (the reflected code starts those from low state 2^(B-1) instead of 0). Spin k going
// up -> down moves the address by +G_k, down -> up by -G_k; then the configuration is counted.
template <int B, bool ODD, int U, class Sink>
ISG_HD void low_step(uint32_t& idx, const int32_t (&Gk)[B], Sink& sink) {
    constexpr int k = ctz_c(U);
    constexpr int before = gray_c(U - 1) ^ (ODD ? (1 << (B - 1)) : 0);
    if constexpr (((before >> k) & 1) != 0) idx += static_cast<uint32_t>(Gk[k]);
    else idx -= static_cast<uint32_t>(Gk[k]);
    sink(idx);
}

template <int B, bool ODD, class Sink, int... U>
ISG_HD void low_steps(uint32_t& idx, const int32_t (&Gk)[B], Sink& sink, std::integer_sequence<int, U...>) {
    (low_step<B, ODD, U + 1>(idx, Gk, sink), ...);
}

// One low block: count the current configuration, then the 2^B - 1 Gray flips of the low spins,
// each followed by a count (a fold over a compile-time sequence, so every flip site, sign and
// register index is a constant).
template <int B, bool ODD, class Sink>
ISG_HD void low_block(uint32_t& idx, const int32_t (&Gk)[B], Sink& sink) {
    sink(idx);
    low_steps<B, ODD>(idx, Gk, sink, std::make_integer_sequence<int, (1 << B) - 1>{});
}

// Flip spin r (r >= B) of st: the address moves by S_r (h_r sE - 4) (dE = 2 S_r h_r, dm = -S_r),
// and every low spin k bonded to r sees its field change by -2 S_r J_kr.
template <int B>
ISG_HD void mid_flip_with(const ProgView& p, const SiteVals& sv, uint64_t& st, int r, uint32_t& idx, int32_t (&Gk)[B]) {
    const int h = field_of(p, sv, st, r);
    const bool up = (st >> r) & 1;
    const int32_t d = h * p.sE - 4;
    idx += static_cast<uint32_t>(up ? d : -d);
#pragma unroll
    for (int k = 0; k < B; ++k) Gk[k] += up ? sv.A[k] : -sv.A[k];
    st ^= 1ull << r;
}

template <int B>
ISG_HD void mid_flip(const ProgView& p, uint64_t& st, int r, uint32_t& idx, int32_t (&Gk)[B]) {
    SiteVals sv;
    load_site(p, r, sv);
    mid_flip_with<B>(p, sv, st, r, idx, Gk);
}

// Visit the 2^q configurations prefix * 2^q + inner, inner in Gray order, counting each through
// sink(byte offset). Returns the last configuration and its incrementally tracked offset so the
// caller can check them against a from-scratch recomputation.
template <int B, class Sink>
ISG_HD void lane_walk(const ProgView& p, uint64_t prefix, uint32_t base, Sink& sink, uint64_t& last_state,
                      uint32_t& last_idx) {
    uint64_t st = prefix << p.q;
    uint32_t idx = base + bin_offset(p, st);
    int32_t Gk[B];
#pragma unroll
    for (int k = 0; k < B; ++k) Gk[k] = field(p, st, k) * p.sE - 4;
    const uint32_t nblocks = 1u << (p.q - B);
    SiteVals svB;                     // spin B takes every other mid flip: its record stays in registers
    if (nblocks > 1) load_site(p, B, svB);
    for (uint32_t t = 0; t < nblocks; t += 2) {
        low_block<B, false>(idx, Gk, sink);
        st ^= 1ull << (B - 1);
        if (t + 1 < nblocks) {
            mid_flip_with<B>(p, svB, st, B, idx, Gk);
            low_block<B, true>(idx, Gk, sink);
            st ^= 1ull << (B - 1);
            if (t + 2 < nblocks) mid_flip<B>(p, st, B + ctz32(t + 2), idx, Gk);
        }
    }
    last_state = st;
    last_idx = idx;
}

}  // namespace isg
