// split_host.cpp -- split-and-convolve enumeration on the host side: choice of the boundary set,
// the device program, and an emulation of the split kernel's per-warp work (no CUDA calls here).
//
// A variant of the paper's full enumeration (Sec. 3): instead of visiting all 2^N configurations,
// a boundary set S is enumerated and, for each of its configurations, the components left by
// removing S are enumerated separately and their histograms convolved (the identity is written
// out in split_internal.h). The tables are identical to the full enumeration's.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <memory>
#include <mutex>
#include <numeric>
#include <string>
#include <unordered_map>
#include <vector>

#include "isg_internal.h"
#include "split_internal.h"

namespace isg {

namespace {

inline int ctz64(uint64_t x) { return __builtin_ctzll(x); }
inline int popc(uint64_t x) { return __builtin_popcountll(x); }
inline uint64_t low_mask(int n) { return n >= 64 ? ~0ull : ((1ull << n) - 1); }

std::vector<uint64_t> adjacency(const isg_graph& g) {
    std::vector<uint64_t> adj(g.n, 0);
    for (size_t b = 0; b < g.bi.size(); ++b) {
        adj[g.bi[b]] |= 1ull << g.bj[b];
        adj[g.bj[b]] |= 1ull << g.bi[b];
    }
    return adj;
}

// Connected components of the spins in `rem` (bit masks), by breadth-first growth, into out[]
// (at most 64 of them: one per spin); returns their number.
int components(const std::vector<uint64_t>& adj, uint64_t rem, uint64_t (&out)[64]) {
    int k = 0;
    while (rem) {
        uint64_t comp = rem & (~rem + 1), front = comp;
        while (front) {
            uint64_t nb = 0;
            for (uint64_t f = front; f; f &= f - 1) nb |= adj[ctz64(f)];
            front = nb & rem & ~comp;
            comp |= front;
        }
        out[k++] = comp;
        rem &= ~comp;
    }
    return k;
}

// Per spin i: the lowest set bit of gcd(|sum_j J_ij|, 2 gcd_j |J_ij|), the power-of-two part of
// every energy step a flip of i can make (Delta e = +-h_i, h_i = sum_j J_ij S_j); 0 for a spin
// with no bonds.
std::vector<uint32_t> spin_step_lowbits(const isg_graph& g) {
    std::vector<uint32_t> out(g.n, 0);
    for (int i = 0; i < g.n; ++i) {
        int64_t sum = 0, gq = 0;
        for (int j = 0; j < g.n; ++j) {
            const int64_t J = g.K[(size_t)i * g.n + j];
            if (!J) continue;
            sum += J;
            gq = std::gcd(gq, std::llabs(J));
        }
        const int64_t r = std::gcd(std::llabs(sum), 2 * gq);
        out[i] = (uint32_t)(r & -r);
    }
    return out;
}

// Row step of a component's histogram: the largest power of two dividing every energy step of
// its spins (1 when none can change the energy).
int component_row_step(const std::vector<uint32_t>& lowbits, uint64_t comp) {
    uint32_t any = 0;
    for (uint64_t r = comp; r; r &= r - 1) any |= lowbits[ctz64(r)];
    return any ? (int)(any & (~any + 1)) : 1;
}

// Per spin: the sum of |J| over its bonds and its neighbours grouped by |J|, so that the bond weight
// touching a set of spins is sum_i w_i - (weight inside the set) without a pass over all bonds.
struct WeightIndex {
    std::vector<int64_t> wsum;
    std::vector<std::vector<std::pair<uint64_t, int64_t>>> groups;   // (neighbour mask, |J|)
    std::vector<uint32_t> step_lowbits;                               // spin_step_lowbits
    explicit WeightIndex(const isg_graph& g) : wsum(g.n, 0), groups(g.n), step_lowbits(spin_step_lowbits(g)) {
        for (int i = 0; i < g.n; ++i)
            for (int j = 0; j < g.n; ++j) {
                const int64_t a = std::llabs(g.K[(size_t)i * g.n + j]);
                if (!a) continue;
                wsum[i] += a;
                auto it = std::find_if(groups[i].begin(), groups[i].end(), [&](const auto& p) { return p.second == a; });
                if (it == groups[i].end()) groups[i].push_back({1ull << j, a});
                else it->first |= 1ull << j;
            }
    }
    int64_t touching(uint64_t set) const {
        int64_t w = 0, twice_inside = 0;
        for (uint64_t r = set; r; r &= r - 1) {
            const int i = ctz64(r);
            w += wsum[i];
            for (const auto& p : groups[i]) twice_inside += p.second * popc(p.first & set);
        }
        return w - twice_inside / 2;
    }
};

// Modelled operations per configuration of a component walk: with a low block (assumed found)
// 2 per configuration (an add to the bin address and a reduction) plus its fields and the mid
// flip per 2^low configurations; without one a field and a checked count each.
static double walk_cost_per_config(int low, int n_cls) {
    return low ? 2 + (low * (6 + 3.0 * n_cls) + 24 + 3.0 * n_cls) / std::ldexp(1.0, low) : 8 + 3.0 * n_cls;
}

struct Candidate {
    uint64_t S = 0;
    int cta_bits = kSplitWalkBits;
    std::vector<uint64_t> comps;     // largest histogram first
    std::vector<int64_t> Sc;
    double cost = INFINITY, visits = 0;
    bool u64 = false;
    int warps = 0;
};

double ceil32(double x) { return std::ceil(x / 32.0); }

// Work model in warp instructions (see the kernel): per boundary configuration the boundary
// energy, per component its fields, a walk of 2^|C| configurations over 32 lanes, and the
// convolution of its histogram's nonzero bins with the accumulator's nonzero bins; then the
// shift-add of the accumulator into the table. Also checks the shared-memory layout fits.
void evaluate(const isg_graph& g, const WeightIndex& wi, int n_cls, Candidate& c) {
    const int ns = popc(c.S);
    c.cost = INFINITY;
    if (ns > 40) return;
    const size_t k = c.comps.size();
    if (k > (size_t)kSplitMaxComp) return;           // k = 0 (all spins boundary) is allowed
    std::vector<int> nc(k);
    c.Sc.assign(k, 0);
    std::vector<size_t> order(k);
    for (size_t i = 0; i < k; ++i) {
        nc[i] = popc(c.comps[i]);
        if (nc[i] > kSplitMaxCompSpins) return;
        c.Sc[i] = wi.touching(c.comps[i]);
        order[i] = i;
    }
    std::sort(order.begin(), order.end(), [&](size_t a, size_t b) {
        const int64_t ha = (c.Sc[a] + 1) * (nc[a] + 1), hb = (c.Sc[b] + 1) * (nc[b] + 1);
        return ha != hb ? ha > hb : c.comps[a] < c.comps[b];
    });
    std::vector<uint64_t> comps2(k);
    std::vector<int64_t> Sc2(k);
    std::vector<int> nc2(k);
    for (size_t i = 0; i < k; ++i) { comps2[i] = c.comps[order[i]]; Sc2[i] = c.Sc[order[i]]; nc2[i] = nc[order[i]]; }
    c.comps = comps2;
    c.Sc = Sc2;
    nc = nc2;
    int64_t EO = 1, MO = 1, hmax = 0;
    std::vector<int> hstride(k);
    for (size_t i = 0; i < k; ++i) {
        EO += c.Sc[i];
        MO += nc[i];
        hstride[i] = split_hist_stride(nc[i], component_row_step(wi.step_lowbits, c.comps[i]));
        hmax = std::max<int64_t>(hmax, (c.Sc[i] + 1) * hstride[i]);
    }
    const int inner = g.n - ns;
    c.u64 = inner > 31;
    const int64_t acc_words = (EO + 1) * MO;
    const size_t acc_bytes = c.u64 ? 8 : 4;
    const size_t per_cta = 768 + 12 * (size_t)hmax + 32 + (2 * acc_bytes + 4) * (size_t)acc_words;
    const size_t prog_bytes = 64 + 8 * ((size_t)n_cls * (1 + ns) + 4 * k + (size_t)(g.n - ns) * 2 * n_cls);
    const size_t table_bytes = 8 * (size_t)(g.S + 1) * (g.n + 1);
    const size_t budget = 227 * 1024 - 1024;
    if (prog_bytes + table_bytes + per_cta > budget) return;
    c.cta_bits = split_cta_bits(prog_bytes + table_bytes + per_cta);
    c.warps = (1 << c.cta_bits) / 32;
    // cost per boundary configuration
    double per_s = 40 + ceil32(ns) * (6 + 3.0 * n_cls);            // plus a few CTA barriers
    double nnz_acc = 0, rows = 1;
    double configs = 0;
    for (size_t i = 0; i < k; ++i) {
        const double hw = (double)(c.Sc[i] + 1) * hstride[i];       // histogram words, padding included
        const double walk = std::ldexp(1.0, nc[i]);
        configs += walk;
        // walkers: 2^P threads, each a from-scratch start and its walk (one warp also rechecks);
        const int low = split_low_want(nc[i], c.cta_bits);
        const double walkers = std::ldexp(1.0, split_walk_bits(nc[i], low, c.cta_bits));
        const double per_config = walk_cost_per_config(low, n_cls);
        per_s += ceil32(nc[i]) * (4 + 3.0 * n_cls) + ceil32(hw) * 2 + nc[i] * (4 + 3.0 * n_cls) +
                 ceil32(walkers) * (nc[i] * (4 + 3.0 * n_cls) + (walk / walkers) * per_config);
        const double nnz_h = std::min((double)(c.Sc[i] + 1) * (nc[i] + 1), walk);
        if (i == 0) {
            nnz_acc = nnz_h;
        } else {
            per_s += ceil32(hw) * 8 + ceil32(rows * MO) * 8 + std::ceil(nnz_acc / 256) * nnz_h * (3 + 8 * 3);
            nnz_acc = std::min(nnz_acc * nnz_h, (rows + c.Sc[i]) * (double)MO);
        }
        rows += c.Sc[i];
        per_s += ceil32(rows * MO) * 2;
    }
    per_s += ceil32((double)EO * MO) * 5;
    c.visits = std::ldexp(configs, ns > 0 ? ns - 1 : 0);         // half the boundary: flip mirrors
    // one CTA per walked boundary configuration: fewer of them than CTA slots (about two per SM)
    // leaves SMs idle, so the work counts at least one full wave
    const double n_walk = std::ldexp(1.0, ns > 0 ? ns - 1 : 0), wave = (c.cta_bits == 8 ? 4.0 : 2.0) * 152;
    c.cost = per_s * std::max(n_walk, wave);
}

}  // namespace

// The boundary search depends on a graph only through its bonds' endpoints and magnitudes and the
// number of distinct couplings: graphs that differ only in coupling signs (disorder realisations
// of one lattice) share it. record = 0 looks a structure up (0: unknown); record != 0 stores the
// boundary found for it.
static uint64_t structural_boundary(const isg_graph& g, int n_cls, uint64_t record) {
    struct Entry {
        int n, n_cls;
        std::vector<int32_t> bi, bj;
        std::vector<int64_t> aJ;
        uint64_t boundary;
    };
    static std::mutex mu;
    static std::unordered_multimap<uint64_t, Entry> cache;
    std::vector<int64_t> aJ(g.bJ.size());
    for (size_t k = 0; k < g.bJ.size(); ++k) aJ[k] = std::llabs(g.bJ[k]);
    uint64_t h = 1469598103934665603ull;
    auto mix = [&](uint64_t v) { for (int b = 0; b < 8; ++b) { h ^= (v >> (8 * b)) & 0xff; h *= 1099511628211ull; } };
    mix((uint64_t)g.n);
    mix((uint64_t)n_cls);
    for (size_t k = 0; k < aJ.size(); ++k) { mix((uint64_t)g.bi[k]); mix((uint64_t)g.bj[k]); mix((uint64_t)aJ[k]); }
    std::lock_guard<std::mutex> lk(mu);
    if (record) {
        if (cache.size() >= 1024) cache.clear();
        cache.emplace(h, Entry{g.n, n_cls, g.bi, g.bj, aJ, record});
        return record;
    }
    auto range = cache.equal_range(h);
    for (auto it = range.first; it != range.second; ++it) {
        const Entry& e = it->second;
        if (e.n == g.n && e.n_cls == n_cls && e.bi == g.bi && e.bj == g.bj && e.aJ == aJ) return e.boundary;
    }
    return 0;
}

// The boundary set: the caller's (boundary != 0), or the cheapest under the work model among
// (a) one or two windows of consecutive spin indices (cyclic), (b) the spins whose index lies in
// a set of residues modulo p (2 <= p <= 8), (c) the complement of a greedy maximal independent
// set. Windows and residues follow the lattices' index order, so rows, columns and layers are
// among the candidates.
SplitPlan plan_split(const isg_graph& g, uint64_t boundary, bool require_gain) {
    const int n = g.n;
    std::vector<int64_t> cls;
    for (int64_t J : g.bJ) cls.push_back(J);
    std::sort(cls.begin(), cls.end());
    cls.erase(std::unique(cls.begin(), cls.end()), cls.end());
    if ((int)cls.size() > kSplitMaxClasses)
        fail(ISG_ERR_TOO_LARGE, "the split enumeration supports at most 16 distinct couplings");
    const int n_cls = std::max<int>(1, (int)cls.size());
    const std::vector<uint64_t> adj = adjacency(g);
    const WeightIndex wi(g);
    const uint64_t all = low_mask(n);
    Candidate best;
    // The walks alone bound the work from below: per boundary configuration a component of nc
    // spins costs at least walk_floor[nc] (its walk at its cheapest, with the largest low block
    // any CTA size allows), and the model charges at least one wave of CTAs (two per SM of 512
    // threads). Candidates whose bound loses skip the full model.
    double walk_floor[kSplitMaxCompSpins + 1];
    for (int nc = 0; nc <= kSplitMaxCompSpins; ++nc)
        walk_floor[nc] = std::max(1.0, std::ldexp(1.0, nc) / 32) * walk_cost_per_config(split_low_want(nc, 8), n_cls);
    auto consider = [&](uint64_t S) {
        S &= all;
        uint64_t comps[64];
        const int k = components(adj, all & ~S, comps);
        double walk = 0;
        for (int i = 0; i < k; ++i) {
            const int nc = popc(comps[i]);
            if (nc > kSplitMaxCompSpins) return;
            walk += walk_floor[nc];
        }
        const int ns = popc(S);
        if (walk * std::max((double)(1ull << (ns > 0 ? ns - 1 : 0)), 2.0 * 152) >= best.cost) return;
        Candidate c;
        c.S = S;
        c.comps.assign(comps, comps + k);
        evaluate(g, wi, n_cls, c);
        if (c.cost < best.cost) best = std::move(c);
    };
    if (boundary) {
        if (boundary & ~all) fail(ISG_ERR_INVALID, "boundary mask names spins beyond N");
        consider(boundary);
        if (!std::isfinite(best.cost))
            fail(ISG_ERR_TOO_LARGE, "the given boundary leaves a component of more than 30 spins, more than 40 "
                                    "boundary spins, or buffers beyond shared memory");
    } else {
        // a boundary known from a graph of the same structure is tried first; the search runs
        // when there is none, or when these couplings reject it (buffers beyond shared memory)
        if (const uint64_t known = structural_boundary(g, n_cls, 0)) consider(known);
        if (!std::isfinite(best.cost)) {
            auto window = [&](int a, int w) {
                uint64_t m = 0;
                for (int i = 0; i < w; ++i) m |= 1ull << ((a + i) % n);
                return m;
            };
            for (int w = 1; w <= n / 2; ++w)
                for (int a = 0; a < n; ++a) {
                    const uint64_t w1 = window(a, w);
                    consider(w1);
                    for (int d = w + 1; d + w <= n; ++d) consider(w1 | window(a + d, w));
                }
            for (int p = 2; p <= 8 && p <= n; ++p)
                for (uint32_t W = 1; W + 1 < (1u << p); ++W) {
                    uint64_t S = 0;
                    for (int i = 0; i < n; ++i) if ((W >> (i % p)) & 1) S |= 1ull << i;
                    consider(S);
                }
            {
                std::vector<int> order(n);
                for (int i = 0; i < n; ++i) order[i] = i;
                std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return popc(adj[a]) < popc(adj[b]); });
                uint64_t I = 0, blocked = 0;
                for (int i : order)
                    if (!((blocked >> i) & 1)) { I |= 1ull << i; blocked |= adj[i] | (1ull << i); }
                consider(all & ~I);
            }
            if (!std::isfinite(best.cost)) fail(ISG_ERR_TOO_LARGE, "no boundary set gives components of at most 30 spins that fit");
            structural_boundary(g, n_cls, best.S);
        }
    }
    // searched or known from a graph of the same structure (planned before without the gain
    // requirement): either way a boundary that does not beat the full enumeration is refused
    if (!boundary && require_gain && best.cost >= std::ldexp(kDirectWarpInstrPerConfig, n))
        fail(ISG_ERR_TOO_LARGE, "no boundary set makes the split cheaper than the full enumeration for this graph");
    SplitPlan p;
    p.boundary = best.S;
    for (int i = 0; i < n; ++i) if ((best.S >> i) & 1) p.S.push_back(i);
    for (uint64_t c : best.comps) {
        std::vector<int> v;
        for (int i = 0; i < n; ++i) if ((c >> i) & 1) v.push_back(i);
        p.comps.push_back(v);
    }
    p.visits = best.visits;
    p.cost = best.cost;
    p.direct_cost = std::ldexp(kDirectWarpInstrPerConfig, n);
    p.use_u64 = best.u64;
    p.cta_bits = best.cta_bits;
    p.warps = best.warps;
    return p;
}

std::vector<uint64_t> build_split_program(const isg_graph& g, const SplitPlan& p, bool lane_model) {
    const int n = g.n, ns = (int)p.S.size(), k = (int)p.comps.size();
    std::vector<int64_t> cls;
    for (int64_t J : g.bJ) cls.push_back(J);
    std::sort(cls.begin(), cls.end());
    cls.erase(std::unique(cls.begin(), cls.end()), cls.end());
    if (cls.empty()) cls.push_back(1);
    const int n_cls = (int)cls.size();
    auto coupling = [&](int i, int j) { return g.K[(size_t)i * n + j]; };
    const std::vector<uint32_t> step_lowbits = spin_step_lowbits(g);
    int n_in = 0;
    for (const auto& c : p.comps) n_in += (int)c.size();
    if (n_in + ns != n) fail(ISG_ERR_INTERNAL, "split plan does not cover every spin");
    SplitHeader h{};
    h.n = n; h.ns = ns; h.n_comp = k; h.n_cls = n_cls;
    h.S_total = (int32_t)g.S;
    h.off_cls = 8;
    h.off_ss = h.off_cls + n_cls;
    h.off_comp = h.off_ss + ns * n_cls;
    h.off_spin = h.off_comp + 4 * k;                // a SplitComp record is four words
    std::vector<uint64_t> blob((size_t)h.off_spin + (size_t)n_in * 2 * n_cls, 0);
    int64_t S_SS = 0;
    for (int a = 0; a < ns; ++a)
        for (int b = a + 1; b < ns; ++b) S_SS += std::llabs(coupling(p.S[a], p.S[b]));
    for (int t = 0; t < n_cls; ++t) std::memcpy(&blob[h.off_cls + t], &cls[t], 8);
    for (int j = 0; j < ns; ++j)
        for (int t = 0; t < n_cls; ++t) {
            uint64_t m = 0;
            for (int l = 0; l < ns; ++l) if (l != j && coupling(p.S[j], p.S[l]) == cls[t]) m |= 1ull << l;
            blob[h.off_ss + (size_t)j * n_cls + t] = m;
        }
    // component energies and the planner's row strides: the largest component histogram is the
    // budget that a row stride chosen by the lane model may not exceed (the CTA's buffers, and so
    // its launch shape, stay as planned)
    auto comp_Sc = [&](const std::vector<int>& v) {
        int64_t Sc = 0;
        for (size_t a = 0; a < v.size(); ++a) {
            for (size_t b = a + 1; b < v.size(); ++b) Sc += std::llabs(coupling(v[a], v[b]));
            for (int j = 0; j < ns; ++j) Sc += std::llabs(coupling(v[a], p.S[j]));
        }
        return Sc;
    };
    auto comp_mask = [](const std::vector<int>& v) { uint64_t m = 0; for (int a : v) m |= 1ull << a; return m; };
    int64_t h_budget = 0;
    for (int c = 0; c < k; ++c)
        h_budget = std::max<int64_t>(h_budget, (comp_Sc(p.comps[c]) + 1) *
                                                   split_hist_stride((int)p.comps[c].size(),
                                                                     component_row_step(step_lowbits, comp_mask(p.comps[c]))));
    int64_t EO = 1, MO = 1, hmax = 0, sumSc = 0;
    int first = 0;
    for (int c = 0; c < k; ++c) {
        // a component of at least kSplitLowMinSpins spins gets a low block: kSplitLowLarge or
        // kSplitLow of its spins (split_low_want) with no bond among them (greedy, fewest bonds
        // inside the component first) as its lowest local bits, so a walk can hold their fields in
        // registers
        std::vector<int> v = p.comps[c];
        const int nc = (int)v.size();
        // `want` spins of the component outside `avoid` with no bond among them (greedy, fewest
        // bonds inside the component first), or fewer if there is no such set
        auto low_pick = [&](int want, uint64_t avoid) {
            std::vector<int> order, pick;
            for (int a : p.comps[c]) if (!((avoid >> a) & 1)) order.push_back(a);
            auto deg = [&](int a) { int d = 0; for (int b : p.comps[c]) d += b != a && coupling(a, b) != 0; return d; };
            std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return deg(a) < deg(b); });
            for (int a : order) {
                bool free = true;
                for (int b : pick) free = free && coupling(a, b) == 0;
                if (free) pick.push_back(a);
                if ((int)pick.size() == want) break;
            }
            return pick;
        };
        int low = 0;
        for (int want = split_low_want(nc, p.cta_bits); want > 0 && !low;
             want = want == kSplitLowLarge && nc >= kSplitLowMinSpins ? kSplitLow : 0) {
            const std::vector<int> pick = low_pick(want, 0);
            if ((int)pick.size() == want) {
                std::vector<int> v2(pick);
                for (int a : p.comps[c])
                    if (std::find(pick.begin(), pick.end(), a) == pick.end()) v2.push_back(a);
                v = v2;
                low = want;
            }
        }
        const int64_t Sc = comp_Sc(v);
        uint64_t cmask = comp_mask(v);
        int hstride = split_hist_stride(nc, component_row_step(step_lowbits, cmask));
        // The walkers of a warp differ in the five spins at local positions Lp .. Lp+4 (the low bits
        // of the thread index); for a large component the bank-conflict model (lanes.cpp, rows of 2
        // units of energy: bin e = E/2) chooses them and the row stride within the budget.
        const int P = split_walk_bits(nc, low, p.cta_bits), Lp = nc - P;
        if (lane_model && nc >= kSplitLaneModelMinSpins && P >= 5 && Lp >= low) {
            const int hi = (int)std::min<int64_t>(nc + 32, h_budget / (Sc + 1));
            const LaneChoice lc = choose_lanes_in(g, cmask, &v[Lp], nc + 1, hi, 2, false);
            bool ok = lc.valid;
            if (ok) {
                uint64_t lmask = 0;
                for (int t = 0; t < 5; ++t) lmask |= 1ull << lc.spins[t];
                const std::vector<int> pick = low ? low_pick(low, lmask) : std::vector<int>();
                ok = (int)pick.size() == low;
                if (ok) {
                    std::vector<int> v2(pick), rest;
                    for (int a : p.comps[c])
                        if (!((lmask >> a) & 1) && std::find(pick.begin(), pick.end(), a) == pick.end()) rest.push_back(a);
                    size_t r = 0;
                    while ((int)v2.size() < Lp) v2.push_back(rest[r++]);
                    for (int t = 0; t < 5; ++t) v2.push_back(lc.spins[t]);
                    while (r < rest.size()) v2.push_back(rest[r++]);
                    v = v2;
                    hstride = lc.stride;
                }
            }
        }
        for (int c2 = 0; c2 < k; ++c2)            // no bond may join two components
            if (c2 != c)
                for (int a : v) for (int b : p.comps[c2])
                    if (coupling(a, b)) fail(ISG_ERR_INTERNAL, "split components are not independent");
        SplitComp rec{nc, (int32_t)Sc, first, (int32_t)((Sc + 1) * hstride), low, hstride, {0, 0}};
        static_assert(sizeof(SplitComp) == 32, "component record is four words");
        std::memcpy(&blob[h.off_comp + 4 * (size_t)c], &rec, sizeof rec);
        for (int a = 0; a < nc; ++a)
            for (int t = 0; t < n_cls; ++t) {
                uint64_t im = 0, sm = 0;
                for (int b = 0; b < nc; ++b) if (b != a && coupling(v[a], v[b]) == cls[t]) im |= 1ull << b;
                for (int j = 0; j < ns; ++j) if (coupling(v[a], p.S[j]) == cls[t]) sm |= 1ull << j;
                const size_t o = h.off_spin + ((size_t)(first + a) * n_cls + t) * 2;
                blob[o] = im;
                blob[o + 1] = sm;
            }
        first += nc;
        EO += Sc;
        MO += nc;
        sumSc += Sc;
        hmax = std::max<int64_t>(hmax, (Sc + 1) * hstride);
    }
    if (S_SS + sumSc != g.S) fail(ISG_ERR_INTERNAL, "split bond weights do not add up to the graph's");
    h.S_SS = (int32_t)S_SS;
    h.EO = (int32_t)EO;
    h.MO = (int32_t)MO;
    h.max_h = (int32_t)hmax;
    h.acc_words = (int32_t)((EO + 1) * MO);
    h.n_bins = (int32_t)((g.S + 1) * (n + 1));
    h.cta_bits = p.cta_bits;
    std::memcpy(blob.data(), &h, sizeof h);
    return blob;
}

// The split kernel's work, warp by warp and lane by lane, on the host with every index checked
// (the device kernel follows the same steps; see split.cu).
void emulate_split(const std::vector<uint64_t>& blob, int64_t* g_out) {
    const SplitView v = split_view(blob.data());
    const SplitHeader& h = *v.h;
    // the device layout: 8-byte arrays at 8-byte aligned offsets, blocks at 16-byte multiples
    for (bool u64 : {false, true}) {
        const SplitWarpLayout L = split_warp_layout(h, u64);
        const size_t base = split_prog_bytes((int)blob.size()) + split_table_bytes(h);
        const size_t acc = (u64 ? 8 : 4) * (size_t)h.acc_words;
        if (base % 16 || L.bytes % 16 || L.spins % 16 || L.scalars < L.spins + 16 * 32 || L.scalars % 4 ||
            L.acc_a < L.scalars + 4 * 16 || L.acc_a % 8 || L.acc_b % 8 || L.hlist % 8 || L.list % 4 || L.hist % 4 ||
            L.acc_b < L.acc_a + acc || L.hlist < L.acc_b + acc || L.list < L.hlist + 8 * (size_t)h.max_h ||
            L.hist < L.list + 4 * (size_t)h.acc_words || L.bytes < L.hist + 4 * (size_t)h.max_h)
            fail(ISG_ERR_INTERNAL, "split kernel shared-memory layout misaligned or overlapping");
    }
    const int ncl = h.n_cls;
    auto field = [&](const uint64_t* masks, int stride, uint64_t bits) {   // sum_t J_t (2 popc(m & bits) - popc(m))
        int64_t f = 0;
        for (int t = 0; t < ncl; ++t) {
            const uint64_t m = masks[(size_t)t * stride];
            f += v.cls[t] * (2 * split_popc64(m & bits) - split_popc64(m));
        }
        return f;
    };
    std::vector<uint64_t> acc((size_t)h.acc_words), out((size_t)h.acc_words);
    std::vector<uint32_t> hist((size_t)h.max_h);
    std::vector<uint32_t> list((size_t)h.acc_words);
    const uint64_t n_s = 1ull << h.ns;
    const uint64_t n_walk = h.ns ? n_s >> 1 : n_s;   // the others are global-flip mirrors
    std::vector<uint64_t> hlist((size_t)h.max_h);
    for (uint64_t s = 0; s < n_walk; ++s) {
        int64_t two_neg_E = 0;                       // sum_j S_j a_j = -2 E_SS
        for (int j = 0; j < h.ns; ++j) {
            const int64_t a = field(v.ss + (size_t)j * ncl, 1, s);
            two_neg_E += ((s >> j) & 1) ? a : -a;
        }
        if (two_neg_E & 1) fail(ISG_ERR_INTERNAL, "odd boundary energy");
        const int64_t e_SS = (-two_neg_E / 2 + h.S_SS) / 2;
        const int m_S = split_popc64(s);
        if (e_SS < 0 || e_SS > h.S_SS) fail(ISG_ERR_INTERNAL, "boundary energy out of range");
        int64_t rows = 0;                            // accumulator rows in use - 1
        if (h.n_comp == 0) { std::fill(acc.begin(), acc.end(), 0); acc[0] = 1; }   // the empty convolution
        for (int c = 0; c < h.n_comp; ++c) {
            const SplitComp cp = v.comp[c];
            const int nc = cp.nc, MC = cp.hstride;
            if (MC < nc + 1 || (int64_t)(cp.Sc + 1) * MC != cp.h_words || cp.h_words > h.max_h)
                fail(ISG_ERR_INTERNAL, "component histogram stride or size inconsistent");
            const uint64_t* sp = v.spin + (size_t)cp.first * ncl * 2;
            std::vector<int64_t> f(nc);
            for (int a = 0; a < nc; ++a) f[a] = field(sp + (size_t)a * ncl * 2 + 1, 2, s);
            std::fill(hist.begin(), hist.end(), 0u);
            const int P = split_walk_bits(nc, cp.low, h.cta_bits), L = nc - P;
            auto count = [&](int64_t e, int m) {
                if (e < 0 || e > cp.Sc || m < 0 || m > nc) fail(ISG_ERR_INTERNAL, "component bin out of range");
                hist[(size_t)e * MC + m] += 1;
            };
            auto field_at = [&](int a, uint32_t x) {
                return field(sp + (size_t)a * ncl * 2, 2, x) + f[a];
            };
            for (int walker = 0; walker < (1 << P); ++walker) {
                uint32_t x = (uint32_t)walker << L;
                int64_t twoE = 0;                    // 2 E_c(x) = -sum_q S_q (internal field + 2 f_q)
                for (int a = 0; a < nc; ++a) {
                    const int64_t hin = field(sp + (size_t)a * ncl * 2, 2, x);
                    const int64_t sa = ((x >> a) & 1) ? 1 : -1;
                    twoE -= sa * (hin + 2 * f[a]);
                }
                if ((twoE / 2 + cp.Sc) & 1) fail(ISG_ERR_INTERNAL, "component energy parity");
                int64_t e = (twoE / 2 + cp.Sc) / 2;
                int m = split_popc64(x);
                if (cp.low) {
                    // mid bits walked in Gray order; at each mid state the low block (all down to
                    // start, its fields fixed) in its own Gray order
                    if ((cp.low != kSplitLow && cp.low != kSplitLowLarge) || L < cp.low)
                        fail(ISG_ERR_INTERNAL, "bad low block");
                    for (uint32_t tm = 0; tm < (1u << (L - cp.low)); ++tm) {
                        if (tm) {
                            const int kk = cp.low + __builtin_ctz(tm);
                            const bool up = (x >> kk) & 1;
                            const int64_t hk = field_at(kk, x);
                            e += up ? hk : -hk;
                            m += up ? -1 : 1;
                            x ^= 1u << kk;
                        }
                        // the kernel moves a histogram address by +-G_k = +-(h_k MC - 1) words per
                        // step from e MC + m; it is checked here against the tracked bin
                        int64_t hl[kSplitLowLarge], Gl[kSplitLowLarge];
                        for (int j = 0; j < cp.low; ++j) {
                            hl[j] = field_at(j, x);
                            Gl[j] = hl[j] * MC - 1;
                        }
                        count(e, m);
                        int64_t el = e, addr = e * MC + m;
                        for (int tl = 1; tl < (1 << cp.low); ++tl) {
                            const int kk = split_ctz(tl);
                            const bool was_up = (split_gray(tl - 1) >> kk) & 1;
                            el += was_up ? hl[kk] : -hl[kk];
                            addr += was_up ? Gl[kk] : -Gl[kk];
                            const int ml = m + split_popc(split_gray(tl));
                            if (addr != el * MC + ml) fail(ISG_ERR_INTERNAL, "low-block address lost its bin");
                            count(el, ml);
                        }
                    }
                } else {
                    for (uint32_t t = 0;; ++t) {
                        count(e, m);
                        if (t + 1 >= (1u << L)) break;
                        const int kk = __builtin_ctz(t + 1);
                        const bool up = (x >> kk) & 1;
                        const int64_t hk = field_at(kk, x);
                        e += up ? hk : -hk;
                        m += up ? -1 : 1;
                        x ^= 1u << kk;
                    }
                }
            }
            if (c == 0) {
                std::fill(acc.begin(), acc.end(), 0);
                for (int64_t e = 0; e <= cp.Sc; ++e)
                    for (int m = 0; m <= nc; ++m) acc[(size_t)e * h.MO + m] = hist[(size_t)e * MC + m];
            } else {
                const int64_t used = (rows + 1) * h.MO;
                size_t nl = 0, nh = 0;
                for (int64_t i = 0; i < used; ++i) if (acc[i]) list[nl++] = (uint32_t)i;
                for (int64_t i = 0; i < (int64_t)cp.h_words; ++i)
                    if (hist[i]) {
                        const int64_t e1 = i / MC, m1 = i % MC;
                        if (m1 > nc) fail(ISG_ERR_INTERNAL, "count in a histogram padding column");
                        hlist[nh++] = (uint64_t)(uint32_t)(e1 * h.MO + m1) | ((uint64_t)hist[i] << 32);
                    }
                std::fill(out.begin(), out.end(), 0);
                for (size_t q = 0; q < nl; ++q)
                    for (size_t j = 0; j < nh; ++j) {
                        const int64_t o = (int64_t)list[q] + (uint32_t)hlist[j];
                        if (o >= h.acc_words) fail(ISG_ERR_INTERNAL, "convolution out of range");
                        out[o] += (hlist[j] >> 32) * acc[list[q]];
                    }
                acc.swap(out);
            }
            rows += cp.Sc;
        }
        if (rows + 1 != h.EO) fail(ISG_ERR_INTERNAL, "accumulator rows");
        for (int64_t i = 0; i < (int64_t)h.EO * h.MO; ++i) {
            if (!acc[i]) continue;
            const int64_t e = e_SS + i / h.MO, m = m_S + i % h.MO;
            if (e > h.S_total || m > h.n) fail(ISG_ERR_INTERNAL, "table bin out of range");
            g_out[e * (h.n + 1) + m] += (int64_t)acc[i];
            if (h.ns) g_out[e * (h.n + 1) + (h.n - m)] += (int64_t)acc[i];
        }
    }
}

// Plans and programs of recent (graph, boundary) pairs: the boundary search costs milliseconds,
// the enumeration of a small lattice microseconds. The key is the graph's content (N and its bond
// list, compared in full on every hit), so graphs created separately share entries and a freed
// handle's address cannot alias another graph.
std::shared_ptr<const SplitPrepared> prepare_split(const isg_graph& g, uint64_t boundary, bool require_gain,
                                                   bool lane_model) {
    static std::mutex mu;
    static std::unordered_multimap<uint64_t, std::shared_ptr<const SplitPrepared>> cache;
    uint64_t h = 1469598103934665603ull;
    auto mix = [&](uint64_t v) { for (int b = 0; b < 8; ++b) { h ^= (v >> (8 * b)) & 0xff; h *= 1099511628211ull; } };
    mix((uint64_t)g.n);
    mix(boundary);
    mix(require_gain ? 1 : 0);
    mix(lane_model ? 1 : 0);
    for (size_t k = 0; k < g.bJ.size(); ++k) { mix((uint64_t)g.bi[k]); mix((uint64_t)g.bj[k]); mix((uint64_t)g.bJ[k]); }
    {
        std::lock_guard<std::mutex> lk(mu);
        auto range = cache.equal_range(h);
        for (auto it = range.first; it != range.second; ++it) {
            const SplitPrepared& e = *it->second;
            if (e.n == g.n && e.boundary_arg == boundary && e.require_gain == require_gain &&
                e.lane_model == lane_model && e.bi == g.bi && e.bj == g.bj && e.bJ == g.bJ)
                return it->second;
        }
    }
    auto e = std::make_shared<SplitPrepared>();
    e->n = g.n;
    e->bi = g.bi;
    e->bj = g.bj;
    e->bJ = g.bJ;
    e->boundary_arg = boundary;
    e->require_gain = require_gain;
    e->lane_model = lane_model;
    e->plan = plan_split(g, boundary, require_gain);
    e->blob = build_split_program(g, e->plan, lane_model);
    std::lock_guard<std::mutex> lk(mu);
    if (cache.size() >= 256) cache.clear();
    cache.emplace(h, e);
    return e;
}

}  // namespace isg

using namespace isg;

extern "C" {

isg_status isg_split_plan(const isg_graph* graph, uint64_t boundary, uint64_t* chosen, int32_t* n_components,
                          int32_t* largest_component, double* visits, double* work_ratio) {
    return guarded([&] {
        if (!graph) fail(ISG_ERR_INVALID, "graph is NULL");
        const std::shared_ptr<const SplitPrepared> e = prepare_split(*graph, boundary, false, false);
        const SplitPlan& p = e->plan;
        if (chosen) *chosen = p.boundary;
        if (n_components) *n_components = (int32_t)p.comps.size();
        if (largest_component) {
            int32_t mx = 0;
            for (const auto& c : p.comps) mx = std::max<int32_t>(mx, (int32_t)c.size());
            *largest_component = mx;
        }
        if (visits) *visits = p.visits;
        if (work_ratio) *work_ratio = p.cost / p.direct_cost;
    });
}

isg_status isg_debug_emulate_split(const isg_graph* graph, uint64_t boundary, int64_t* g_out) {
    return guarded([&] {
        if (!graph || !g_out) fail(ISG_ERR_INVALID, "NULL argument");
        // the program isg_enumerate_split runs (lane spins by the conflict model)
        const std::shared_ptr<const SplitPrepared> e = prepare_split(*graph, boundary, false, true);
        const std::vector<uint64_t>& blob = e->blob;
        std::memset(g_out, 0, sizeof(int64_t) * (size_t)(graph->S + 1) * (graph->n + 1));
        emulate_split(blob, g_out);
    });
}

}  // extern "C"
