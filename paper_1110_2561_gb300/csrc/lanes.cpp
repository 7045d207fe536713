// lanes.cpp -- which five spins carry a warp's lane index in the enumeration kernel, chosen by a
// model of the kernel's shared-memory bank conflicts (host only, no CUDA calls).
//
// The 32 lanes of a warp task walk the same inner configurations with the same task bits; they
// differ only in the five spins at internal positions q .. q+4 (the "lane spins", lane bit k on
// spin L_k). In one warp reduction the 32 bin addresses 4 (e' R + m) therefore differ by
//   de'(b) = (E(b) - E(0)) / G,  dm(b) = popcount(b)     (b = the lane's five bits),
// where E(b) - E(0) comes from the couplings among the lane spins and from the fields on them of
// their other neighbours (Eq. 1 restricted to the lane spins' bonds). The shared-memory pipe
// serves one distinct address per bank per wavefront and merges lanes that hit the same address,
// so a reduction costs as many wavefronts as its busiest bank holds distinct addresses -- a
// function of the offsets de'(b) R + dm(b) modulo 32 only (a common shift of all 32 addresses
// moves every bank alike).
//
// The enumeration visits every configuration once, so over a launch the states of the lane
// spins' neighbours run uniformly over all their values, whichever of them are inner or task
// spins. The expected wavefronts per reduction are thus a property of the lane set and the row
// stride R alone; the planner estimates them by sampling those neighbour states and picks the set
// and stride with the fewest, among compact candidate sets. (On the 6x6 torus a spin with its four
// neighbours as lane spins makes every reduction conflict-free at R = 45.)
#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <mutex>
#include <set>
#include <tuple>
#include <vector>

#include "isg_internal.h"

namespace isg {

namespace {

uint64_t splitmix(uint64_t& s) {
    s += 0x9E3779B97F4A7C15ull;
    uint64_t z = s;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

int popc(uint64_t x) { return __builtin_popcountll(x); }

// Expected wavefronts per warp reduction of lane set L[0..4] for every stride in `strides`, with
// histogram rows of `divisor` units of energy, estimated from `samples` uniform draws of the
// states of the lane spins' other neighbours (the
// draws come from `seed`; equal seeds give every candidate the same draws where their
// neighbourhoods coincide). Distinct addresses are distinct (e', m) pairs at every stride above
// 2 x 5, so the 32 lanes are merged once per draw and only their banks depend on the stride.
std::vector<double> lane_costs(const isg_graph& g, const int* L, const std::vector<int>& strides, int samples,
                               uint64_t seed, int64_t divisor) {
    const int n = g.n;
    uint64_t inL = 0;
    for (int k = 0; k < 5; ++k) inL |= 1ull << L[k];
    // the lane spins' couplings to every spin outside the set, whose states are drawn
    std::vector<std::pair<int, int64_t>> nb[5];
    for (int k = 0; k < 5; ++k)
        for (int j = 0; j < n; ++j) {
            const int64_t J = g.K[(size_t)L[k] * n + j];
            if (J && !((inL >> j) & 1)) nb[k].push_back({j, J});
        }
    // energy of the bonds among the lane spins for each lane value (s_k = 2 b_k - 1)
    int64_t ell[32];
    for (int b = 0; b < 32; ++b) {
        int64_t e = 0;
        for (int k = 0; k < 5; ++k)
            for (int k2 = k + 1; k2 < 5; ++k2) {
                const int64_t J = g.K[(size_t)L[k] * n + L[k2]];
                if (J) e -= J * (((b >> k) & 1) ? 1 : -1) * (((b >> k2) & 1) ? 1 : -1);
            }
        ell[b] = e;
    }
    std::vector<double> tot(strides.size(), 0.0);
    uint64_t rs = seed;
    int64_t de[32], dist_de[32];
    int dist_m[32];
    for (int smp = 0; smp < samples; ++smp) {
        const uint64_t state = splitmix(rs);            // spin j of the draw: bit j (n <= 64)
        int64_t h[5];
        for (int k = 0; k < 5; ++k) {
            int64_t a = 0;
            for (const auto& p : nb[k]) a += ((state >> p.first) & 1) ? p.second : -p.second;
            h[k] = a;
        }
        // E(b) = ell(b) - sum_k s_k h_k; differences from lane 0 are multiples of the divisor
        int64_t e0 = 0;
        int nd = 0;
        for (int b = 0; b < 32; ++b) {
            int64_t e = ell[b];
            for (int k = 0; k < 5; ++k) e -= (((b >> k) & 1) ? 1 : -1) * h[k];
            if (b == 0) e0 = e;
            de[b] = (e - e0) / divisor;
            const int m = popc((uint64_t)b);
            bool dup = false;
            for (int t = 0; t < nd; ++t) if (dist_de[t] == de[b] && dist_m[t] == m) { dup = true; break; }
            if (!dup) { dist_de[nd] = de[b]; dist_m[nd] = m; ++nd; }
        }
        for (size_t r = 0; r < strides.size(); ++r) {
            const int64_t R = strides[r];
            int cnt[32] = {0}, worst = 0;
            for (int t = 0; t < nd; ++t) {
                const int bank = (int)((dist_de[t] * R + dist_m[t]) & 31);
                worst = std::max(worst, ++cnt[bank]);
            }
            tot[r] += worst;
        }
    }
    for (double& t : tot) t /= samples;
    return tot;
}

// Connected sets of five spins of `pool` containing `root` (duplicates removed), at most `cap`.
void connected_sets(const std::vector<uint64_t>& adj, uint64_t pool, int root, size_t cap, std::set<uint64_t>& out) {
    // depth-first over connected partial sets containing root; `cap` bounds out's total size
    std::vector<uint64_t> stack{1ull << root};
    std::set<uint64_t> seen;
    while (!stack.empty() && out.size() < cap) {
        const uint64_t S = stack.back();
        stack.pop_back();
        if (!seen.insert(S).second) continue;
        if (popc(S) == 5) { out.insert(S); continue; }
        uint64_t front = 0;
        for (uint64_t t = S; t; t &= t - 1) front |= adj[__builtin_ctzll(t)];
        front &= pool & ~S;
        for (uint64_t t = front; t; t &= t - 1) stack.push_back(S | (1ull << __builtin_ctzll(t)));
    }
}

std::mutex g_lane_mu;
std::map<std::tuple<uint64_t, uint64_t, int, int, int64_t>, LaneChoice> g_lane_cache;

// Key of the cache: N, the bonds with the magnitudes of their couplings (not their signs), the
// energy stride and the number of histogram rows. Graphs that differ only in coupling signs (the
// disorder realisations of a batch) share one search: the chosen set is valid for every one of them
// (any five spins are), its stride keeps 8 R divisible by their common energy stride, and its
// modelled cost on another sign draw is close to that draw's own best (1.03-1.04 against 1.02 on
// EA 5x6 instances, index order 1.07-1.10).
uint64_t structure_hash(const isg_graph& g) {
    uint64_t h = 1469598103934665603ull;                      // FNV-1a
    auto mix = [&](uint64_t v) { for (int b = 0; b < 8; ++b) { h ^= (v >> (8 * b)) & 0xff; h *= 1099511628211ull; } };
    mix((uint64_t)g.n);
    mix((uint64_t)g.G);
    mix((uint64_t)g.n_e_c);
    for (size_t k = 0; k < g.bJ.size(); ++k) {
        mix((uint64_t)g.bi[k]);
        mix((uint64_t)g.bj[k]);
        mix((uint64_t)(g.bJ[k] < 0 ? -g.bJ[k] : g.bJ[k]));
    }
    return h;
}

}  // namespace

LaneChoice choose_lanes(const isg_graph& g, uint64_t pool, const int* baseline, int max_stride) {
    // strides keep 8 R a multiple of the energy stride (the program's address step per unit of field)
    return choose_lanes_in(g, pool, baseline, g.n + 1, std::min(max_stride, g.n + 32), g.G, true, false);
}

LaneChoice choose_lanes_in(const isg_graph& g, uint64_t pool, const int* baseline, int stride_lo, int stride_hi,
                           int64_t divisor, bool stride_times8_by_G, bool quick) {
    const int n = g.n;
    const std::tuple<uint64_t, uint64_t, int, int, int64_t> key(structure_hash(g), pool, stride_lo, stride_hi,
                                                                (divisor * 2 + (quick ? 1 : 0)) * (stride_times8_by_G ? 1 : -1));
    {
        std::lock_guard<std::mutex> lk(g_lane_mu);
        const auto it = g_lane_cache.find(key);
        if (it != g_lane_cache.end()) return it->second;
    }
    std::vector<int> strides;
    for (int R = stride_lo; R <= stride_hi; ++R)
        if (!stride_times8_by_G || (8 * (int64_t)R) % g.G == 0) strides.push_back(R);
    LaneChoice best;
    if (strides.empty() || popc(pool) < 5) { best.valid = false; return best; }
    std::vector<uint64_t> adj(n, 0);
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j)
            if (g.K[(size_t)i * n + j]) adj[i] |= 1ull << j;
    // candidates: dense greedy sets grown from every spin of the pool, and every connected set of
    // five around a few spins; the densest (most bonds inside the set) go on to the model
    std::set<uint64_t> cand;
    for (uint64_t t = pool; t; t &= t - 1) {
        const int v = __builtin_ctzll(t);
        uint64_t S = 1ull << v, clos = adj[v] | S;
        while (popc(S) < 5) {
            int bu = -1, bb = -1, bg = 1 << 30;
            for (uint64_t r = pool & ~S; r; r &= r - 1) {
                const int u = __builtin_ctzll(r);
                const int bonds = popc(adj[u] & S), grow = popc((adj[u] | (1ull << u)) & ~clos);
                if (bonds > bb || (bonds == bb && grow < bg)) { bu = u; bb = bonds; bg = grow; }
            }
            S |= 1ull << bu;
            clos |= adj[bu] | (1ull << bu);
        }
        cand.insert(S);
    }
    std::vector<int> seeds;                           // up to three, spread over the index range
    for (int part = 0; part < 3; ++part) {
        const uint64_t above = pool & ~((1ull << (part * n / 3)) - 1);
        if (!above) continue;
        const int v = __builtin_ctzll(above);
        if (std::find(seeds.begin(), seeds.end(), v) == seeds.end()) seeds.push_back(v);
    }
    if (!quick)
        for (int v : seeds) connected_sets(adj, pool, v, cand.size() + 2500, cand);
    auto inner_bonds = [&](uint64_t S) {
        int b = 0;
        for (uint64_t t = S; t; t &= t - 1) b += popc(adj[__builtin_ctzll(t)] & S);
        return b / 2;
    };
    int top = 0;
    for (uint64_t S : cand) top = std::max(top, inner_bonds(S));
    std::vector<std::pair<double, uint64_t>> screened;
    uint64_t base_mask = 0;
    for (int k = 0; k < 5; ++k) base_mask |= 1ull << baseline[k];
    auto spins_of = [](uint64_t S, int* L) { int k = 0; for (uint64_t t = S; t; t &= t - 1) L[k++] = __builtin_ctzll(t); };
    // screening: the same draws for every candidate, so the comparison is not left to chance
    for (uint64_t S : cand) {
        if (inner_bonds(S) + 1 < top) continue;
        int L[5];
        spins_of(S, L);
        const std::vector<double> c = lane_costs(g, L, strides, quick ? 24 : 48, 0x1a7e5, divisor);
        screened.push_back({*std::min_element(c.begin(), c.end()), S});
    }
    std::sort(screened.begin(), screened.end());
    if (screened.size() > (quick ? 3u : 12u)) screened.resize(quick ? 3 : 12);
    screened.push_back({0.0, base_mask});
    // refine the best few (and the index order's set) with many more samples
    best.valid = false;
    for (const auto& sc : screened) {
        int L[5];
        if (sc.second == base_mask) std::memcpy(L, baseline, sizeof L);
        else spins_of(sc.second, L);
        const std::vector<double> c = lane_costs(g, L, strides, quick ? 192 : 1024, 0x5eed, divisor);
        const size_t r = (size_t)(std::min_element(c.begin(), c.end()) - c.begin());
        if (sc.second == base_mask) best.cost_index_order = c[r];
        if (!best.valid || c[r] < best.cost) {
            best.valid = true;
            best.cost = c[r];
            best.stride = strides[r];
            std::memcpy(best.spins, L, sizeof L);
        }
    }
    std::lock_guard<std::mutex> lk(g_lane_mu);
    if (g_lane_cache.size() >= 4096) g_lane_cache.clear();   // a server plans graph after graph
    g_lane_cache[key] = best;
    return best;
}

}  // namespace isg
