// host.cpp -- graph model, options, planner, program blobs, errors and the host emulation of the
// enumeration kernels (no CUDA calls in this file).
#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <memory>
#include <mutex>
#include <numeric>
#include <string>
#include <vector>

#include "isg_internal.h"

namespace isg {

static thread_local std::string t_last_error;

void set_error(const std::string& msg) { t_last_error = msg; }
void clear_error() { t_last_error.clear(); }
[[noreturn]] void fail(isg_status s, const std::string& msg) { throw Error{s, msg}; }

void check_self_check_word(unsigned int word, const char* what) {
    if (!word) return;
    std::string msg = std::string(what) + " self-check failed (status " + std::to_string(word) + ":";
    if (word & kSelfCheckLostBin) msg += " a walk's tracked bin differed from its recomputation;";
    if (word & kSelfCheckOutOfRange) msg += " a walk's address left the histogram;";
    msg.back() = ')';
    fail(ISG_ERR_INTERNAL, msg);
}

isg_options resolve_options(const isg_options* opt) {
    isg_options o;
    isg_options_init(&o);
    if (opt) {
        if (opt->struct_size != (int32_t)sizeof(isg_options))
            fail(ISG_ERR_INVALID, "isg_options.struct_size mismatch (initialise with isg_options_init)");
        o = *opt;
    }
    if (o.max_spins <= 0) o.max_spins = 40;
    if (o.max_spins > 62) o.max_spins = 62;
    if (o.symmetry && (o.shard_bits || o.shard_lo || o.shard_hi))
        fail(ISG_ERR_INVALID, "symmetry cannot be combined with shards");
    return o;
}

static int64_t igcd(int64_t a, int64_t b) {
    a = a < 0 ? -a : a;
    b = b < 0 ? -b : b;
    while (b) { int64_t t = a % b; a = b; b = t; }
    return a;
}

// ---------------------------------------------------------------------------------------------
// Planner
// ---------------------------------------------------------------------------------------------
static int weight_classes(const isg_graph& g, std::vector<int32_t>& w) {
    std::vector<int64_t> vals;
    int64_t bits = 0;
    for (size_t b = 0; b < g.bJ.size(); ++b) {
        int64_t a = g.bJ[b] < 0 ? -g.bJ[b] : g.bJ[b];
        vals.push_back(a);
        bits |= a;
    }
    std::sort(vals.begin(), vals.end());
    vals.erase(std::unique(vals.begin(), vals.end()), vals.end());
    int nbits = 0;
    for (int t = 0; t < 63; ++t) if ((bits >> t) & 1) ++nbits;
    w.clear();
    if (vals.empty()) { w.push_back(1); return 0; }       // no bonds: one empty class
    if ((int)vals.size() <= nbits || (int)vals.size() <= 4) {
        for (int64_t v : vals) w.push_back((int32_t)v);
        return 0;                                          // distinct-value classes
    }
    for (int t = 0; t < 63; ++t) if ((bits >> t) & 1) w.push_back((int32_t)(1 << t));
    return 1;                                              // binary classes
}

int choose_stride(const isg_graph& g, int requested, int residue) {
    const int n_m = g.n + 1;
    if (requested == 0 && residue > 0) {
        if (residue >= 32) fail(ISG_ERR_INVALID, "stride_residue must lie in [1, 31]");
        for (int s = n_m; s < n_m + 64; ++s)
            if (s % 32 == residue && (8 * (int64_t)s) % g.G == 0) return s;
    }
    if (requested > 0) {
        if (requested < n_m || (8 * (int64_t)requested) % g.G)
            fail(ISG_ERR_INVALID, "bin_stride must be >= N + 1 and make 8 * stride a multiple of the energy stride");
        return requested;
    }
    // Residues of the stride mod 32, best first: lanes of a warp differ in five outer spins, so
    // their bins differ by a few columns (|dm| <= 5) and a few rows; these residues send the
    // common small offsets (de * stride + dm) to distinct banks (a residue of 31 or 1 collides
    // whenever de = dm or de = -dm).
    static const int pref[] = {6, 26, 7, 25, 13, 19, 9, 23, 5, 27, 11, 21};
    for (int r : pref)
        for (int s = n_m; s < n_m + 32; ++s)
            if (s % 32 == r && (8 * (int64_t)s) % g.G == 0) return s;
    return n_m;
}

static size_t blob_words(int n, int nc) {
    return kHeaderWords + (size_t)n * (sizeof(SiteRec) / 8) + (size_t)n * (nc - 1) + ((size_t)nc + 1) / 2;
}

// Minimum-residual-degree greedy independent set of at most bmax spins among the free spins
// 0 .. free-1 outside `excluded`: repeatedly take the candidate with the fewest neighbours among
// the remaining candidates (ties: lowest index), then drop it and its neighbours. Sorted.
static std::vector<int> low_block_spins(const isg_graph& g, int free, int bmax, uint64_t excluded) {
    const int n = g.n;
    std::vector<char> alive(free, 1);
    for (int c = 0; c < free; ++c) if ((excluded >> c) & 1) alive[c] = 0;
    std::vector<int> low;
    while ((int)low.size() < bmax) {
        int best = -1, best_deg = 1 << 30;
        for (int c = 0; c < free; ++c) {
            if (!alive[c]) continue;
            int d = 0;
            for (int o = 0; o < free; ++o) if (alive[o] && o != c && g.K[(size_t)c * n + o] != 0) ++d;
            if (d < best_deg) { best_deg = d; best = c; }
        }
        if (best < 0) break;
        low.push_back(best);
        alive[best] = 0;
        for (int o = 0; o < free; ++o) if (g.K[(size_t)best * n + o] != 0) alive[o] = 0;
    }
    std::sort(low.begin(), low.end());
    return low;
}

// Inner bits q for a low block of b spins (see make_plan).
static int inner_bits_for(const isg_options& o, int free, int b, int shards_log2) {
    if (o.inner_bits > 0) {
        const int q = o.inner_bits;
        if (q < b || q > free - 5 || q > 26)
            fail(ISG_ERR_INVALID, "inner_bits must satisfy low block <= q <= N - shard_bits - 5 and q <= 26");
        return q;
    }
    // about 2^15 warp tasks (several per resident warp, so the dynamic queue balances), but at
    // least 2^12 configurations per lane so the from-scratch start of a task stays negligible
    int q = free - 5 - std::max(0, 15 - shards_log2);
    int qmin = std::min(12, free - 5);
    // small problems are latency-bound: spread them over >= 256 warp tasks where they allow it
    if (free - 5 - qmin < 8) qmin = std::max(b, free - 5 - 8);
    q = std::max(q, qmin);
    q = std::min(q, 20);
    q = std::min(q, free - 5);
    return std::max(q, b);
}

// Internal order: the low block, the other inner spins, the five lane spins (positions q..q+4),
// the remaining free spins, then the shard spins in the caller's order at the top.
static void order_spins(Plan& p, int n, int free, const std::vector<int>& low, const int* lanes) {
    std::vector<char> used(n, 0);
    int pos = 0;
    for (int l : low) { p.perm[pos++] = l; used[l] = 1; }
    if (lanes) for (int k = 0; k < 5; ++k) used[lanes[k]] = 1;
    for (int s = 0; s < free && pos < p.q; ++s) if (!used[s]) { p.perm[pos++] = s; used[s] = 1; }
    if (lanes) for (int k = 0; k < 5; ++k) p.perm[pos++] = lanes[k];
    for (int s = 0; s < free; ++s) if (!used[s]) p.perm[pos++] = s;
    for (int s = free; s < n; ++s) p.perm[pos++] = s;
}

// Symmetric chain decomposition of the 5-bit lane values (de Bruijn, Tengbergen and Kruyswijk,
// 1951): read the bits of a value from bit 0 up, a 0 as an opening and a 1 as a closing bracket,
// and match brackets. Values with the same matched pairs (the same matched positions holding the
// same bits) form one chain: the unmatched bits read 1..1 0..0, with one more 1 for each step up
// the chain. Each chain holds consecutive popcounts: chain t holds [low[t], low[t] + len[t]).
static void lane_chains(int* chain_of, int* low, int* len) {
    std::vector<std::pair<uint32_t, uint32_t>> keys;    // (matched positions, their bits) per chain
    for (uint32_t l = 0; l < 32; ++l) {
        int open[5], sp = 0;
        uint32_t matched = 0;
        for (int b = 0; b < 5; ++b) {
            if (!((l >> b) & 1)) open[sp++] = b;
            else if (sp) matched |= (1u << b) | (1u << open[--sp]);
        }
        const std::pair<uint32_t, uint32_t> key(matched, l & matched);   // the pairs and their bits
        int t = 0;
        while (t < (int)keys.size() && keys[t] != key) ++t;
        if (t == (int)keys.size()) keys.push_back(key);
        chain_of[l] = t;
    }
    if ((int)keys.size() != kLaneTables) fail(ISG_ERR_INTERNAL, "lane values do not form ten chains");
    for (int t = 0; t < kLaneTables; ++t) { low[t] = 5; len[t] = 0; }
    for (int l = 0; l < 32; ++l) {
        low[chain_of[l]] = std::min(low[chain_of[l]], __builtin_popcount((unsigned)l));
        ++len[chain_of[l]];
    }
}

// Order of the packed layout. The chains' bank ranges tile the 32 banks in a circular order
// (slot k: banks [beta[k], beta[k] + len[k]), the length-6 chain at bank 0), and the row holds
// them in the order path[0..9] of slots. A chain spans len + N - 5 words of a row; the next one
// starts at the first word after it whose bank is its beta, c = (N - 5) mod 32 banks on, plus
// gap[k] words. For each circular arrangement of the lengths (126: which four of the other nine
// slots hold the length-4 chains) a dynamic programme over subsets finds the path of least total
// gap; the least over all arrangements is kept. Depends on N only through c, so it is computed
// once per residue.
struct PackedOrder {
    int len[kLaneTables], beta[kLaneTables], path[kLaneTables], gap[kLaneTables];
    int total_gap;
};

static PackedOrder packed_order_search(int c) {
    PackedOrder best{};
    best.total_gap = 1 << 30;
    constexpr int S = 1 << kLaneTables;
    std::vector<int> dp((size_t)S * kLaneTables), from((size_t)S * kLaneTables);
    for (int sel = 0; sel < (1 << (kLaneTables - 1)); ++sel) {
        if (__builtin_popcount((unsigned)sel) != 4) continue;
        int len[kLaneTables], beta[kLaneTables];
        len[0] = 6;
        for (int k = 1; k < kLaneTables; ++k) len[k] = ((sel >> (k - 1)) & 1) ? 4 : 2;
        beta[0] = 0;
        for (int k = 1; k < kLaneTables; ++k) beta[k] = beta[k - 1] + len[k - 1];
        auto gap = [&](int i, int j) { return (((beta[j] - beta[i] - len[i] - c) % 32) + 32) % 32; };
        std::fill(dp.begin(), dp.end(), 1 << 29);
        for (int j = 0; j < kLaneTables; ++j) dp[((size_t)1 << j) * kLaneTables + j] = 0;
        for (int m = 1; m < S; ++m)
            for (int i = 0; i < kLaneTables; ++i) {
                const int v = dp[(size_t)m * kLaneTables + i];
                if (!((m >> i) & 1) || v >= best.total_gap) continue;
                for (int j = 0; j < kLaneTables; ++j) {
                    if ((m >> j) & 1) continue;
                    const size_t to = (size_t)(m | (1 << j)) * kLaneTables + j;
                    if (v + gap(i, j) < dp[to]) { dp[to] = v + gap(i, j); from[to] = i; }
                }
            }
        for (int j = 0; j < kLaneTables; ++j) {
            const int v = dp[(size_t)(S - 1) * kLaneTables + j];
            if (v >= best.total_gap) continue;
            best.total_gap = v;
            std::copy(len, len + kLaneTables, best.len);
            std::copy(beta, beta + kLaneTables, best.beta);
            for (int m = S - 1, x = j, k = kLaneTables - 1; k >= 0; --k) {
                best.path[k] = x;
                const int px = from[(size_t)m * kLaneTables + x];
                m ^= 1 << x;
                x = px;
            }
            for (int k = 0; k + 1 < kLaneTables; ++k) best.gap[k] = gap(best.path[k], best.path[k + 1]);
            best.gap[kLaneTables - 1] = 0;
        }
    }
    return best;
}

static const PackedOrder& packed_order(int c) {
    static std::mutex mu;
    static std::unique_ptr<PackedOrder> cache[32];
    std::lock_guard<std::mutex> lk(mu);
    if (!cache[c]) cache[c].reset(new PackedOrder(packed_order_search(c)));
    return *cache[c];
}

void lane_table_layout(Plan& p, int n, int64_t rows, int64_t G, int fixed_stride) {
    int chain_of[32], low[kLaneTables], len[kLaneTables];
    lane_chains(chain_of, low, len);
    const int rest = n - 5;                        // spins outside the lane bits
    // strides R with R % 32 == 0 and (8 R) % G == 0: the multiples of `unit`
    const int64_t unit = 32 / igcd(32, G / igcd(G, 8)) * (G / igcd(G, 8));
    auto round_up = [&](int64_t x) { return (x + unit - 1) / unit * unit; };
    if (fixed_stride > 0 && (fixed_stride % 32 || (8 * (int64_t)fixed_stride) % G || fixed_stride < n + 1))
        fail(ISG_ERR_INVALID, "lane tables need a row stride that is a multiple of 32, at least N + 1, with "
                              "8 x stride a multiple of the energy stride " + std::to_string(G));
    for (int t = 0; t < kLaneTables; ++t) { p.sub_m_lo[t] = low[t]; p.sub_m_hi[t] = low[t] + len[t] - 1 + rest; }

    // separate: chains in order of their lowest popcount take consecutive banks
    const int64_t Rs = fixed_stride > 0 ? fixed_stride : round_up(n + 1);
    const int64_t sub_words = rows * Rs + 32;
    const int64_t sep_words = kLaneTables * sub_words;
    // packed: the searched order, its banks rotated so that the first chain's sub-table starts at word 0
    const PackedOrder& po = packed_order(rest % 32);
    int64_t A[kLaneTables];
    int slot_chain[kLaneTables];
    {
        bool taken[kLaneTables] = {};
        for (int k = 0; k < kLaneTables; ++k) {      // any chain of a slot's length takes the slot
            int t = 0;
            while (taken[t] || len[t] != po.len[k]) ++t;
            taken[t] = true;
            slot_chain[k] = t;
        }
    }
    int64_t span = 0;
    for (int k = 0; k < kLaneTables; ++k) {
        const int s = po.path[k];
        A[s] = span;
        span += po.len[s] + rest + po.gap[k];
    }
    const int64_t Rp = round_up(span);
    const int64_t packed_words = (rows - 1) * Rp + span;
    const bool packed = fixed_stride == 0 && packed_words < sep_words;

    int32_t off[kLaneTables];
    if (packed) {
        const int rot = ((low[slot_chain[po.path[0]]] - po.beta[po.path[0]]) % 32 + 32) % 32;
        for (int k = 0; k < kLaneTables; ++k) {
            const int t = slot_chain[k];
            // first word of chain t's range: A (bank beta + rot), minus its lowest column
            off[t] = (int32_t)(A[k] + low[slot_chain[po.path[0]]] - low[t]);
            if (((off[t] + low[t]) % 32 + 32) % 32 != (po.beta[k] + rot) % 32)
                fail(ISG_ERR_INTERNAL, "packed lane table lost its bank");
        }
        p.stride = (int)Rp;
        p.copy_words = (int)(packed_words + low[slot_chain[po.path[0]]]);
    } else {
        int order[kLaneTables];
        for (int t = 0; t < kLaneTables; ++t) order[t] = t;
        std::stable_sort(order, order + kLaneTables, [&](int x, int y) { return low[x] < low[y]; });
        int bank = 0;
        for (int i = 0; i < kLaneTables; ++i) {
            const int t = order[i];
            if (bank - low[t] < 0 || bank - low[t] >= 32) fail(ISG_ERR_INTERNAL, "lane sub-table offset out of range");
            off[t] = (int32_t)(t * sub_words + bank - low[t]);
            bank += len[t];
        }
        p.stride = (int)Rs;
        p.copy_words = (int)sep_words;
    }
    p.n_sub = kLaneTables;
    p.packed = packed;
    for (int t = 0; t < kLaneTables; ++t) p.sub_off[t] = off[t];
    for (int l = 0; l < 32; ++l) { p.lane_sub[l] = (int8_t)chain_of[l]; p.lane_word[l] = off[chain_of[l]]; }

    // every lane its own bank; every word of a sub-table its own and inside the copy
    uint32_t banks = 0;
    for (int l = 0; l < 32; ++l) banks |= 1u << ((p.lane_word[l] + __builtin_popcount((unsigned)l)) & 31);
    if (p.stride % 32 || (8 * (int64_t)p.stride) % G || banks != 0xffffffffu)
        fail(ISG_ERR_INTERNAL, "lane tables do not give every lane its own bank");
    std::vector<uint8_t> owner((size_t)p.copy_words, 0xff);
    for (int t = 0; t < kLaneTables; ++t)
        for (int64_t e = 0; e < rows; ++e)
            for (int m = p.sub_m_lo[t]; m <= p.sub_m_hi[t]; ++m) {
                const int64_t w = p.sub_off[t] + e * p.stride + m;
                if (w < 0 || w >= p.copy_words || owner[(size_t)w] != 0xff)
                    fail(ISG_ERR_INTERNAL, "lane sub-tables overlap or leave the copy");
                owner[(size_t)w] = (uint8_t)t;
            }
}

Plan make_plan(const isg_graph& g, const isg_options& o, const DeviceInfo& d, bool single_graph) {
    Plan p;
    const int n = g.n;
    if (n > o.max_spins)
        fail(ISG_ERR_TOO_LARGE, "graph has " + std::to_string(n) + " spins, more than max_spins = " +
                                    std::to_string(o.max_spins));
    if (o.lane_model < 0 || o.lane_model > 4) fail(ISG_ERR_INVALID, "lane_model must lie in [0, 4]");
    if (o.lane_model == 4 && o.bin_stride % 32 != 0) fail(ISG_ERR_INVALID, "lane tables need a row stride that is a multiple of 32");
    const int k = o.shard_bits;
    if (k < 0 || k > n) fail(ISG_ERR_INVALID, "shard_bits must lie in [0, N]");
    int64_t lo = o.shard_lo, hi = o.shard_hi;
    if (lo == 0 && hi == 0) hi = (int64_t)1 << k;
    if (lo < 0 || lo >= hi || hi > ((int64_t)1 << k)) fail(ISG_ERR_INVALID, "shard range must satisfy 0 <= lo < hi <= 2^shard_bits");
    const int free = n - k;
    p.perm.resize(n);
    std::iota(p.perm.begin(), p.perm.end(), 0);

    const bool forced = o.inner_bits > 0 || o.low_bits > 0;
    if (free < 6 || (free < 11 && !forced)) {
        p.small = true;
        p.stride = n + 1;
        p.s_lo = (uint64_t)lo << free;
        p.s_hi = (uint64_t)hi << free;
        p.q = 0;
        p.b = 0;
        p.threads = 256;
        const uint64_t states = p.s_hi - p.s_lo;
        p.grid = (int)std::max<uint64_t>(1, std::min<uint64_t>((states + p.threads - 1) / p.threads, (uint64_t)d.sms * 8));
        p.smem_bytes = blob_words(n, 21) * 8;
        return p;
    }

    // Low block: greedy independent set among the spins below the shard bits, lowest degree first.
    int bmax = o.low_bits > 0 ? o.low_bits : kMaxLow;
    if (bmax > kMaxLow) fail(ISG_ERR_INVALID, "low_bits must be <= 7");
    bmax = std::min(bmax, free - 5);
    std::vector<int> low = low_block_spins(g, free, bmax, 0);
    if (o.low_bits > 0 && (int)low.size() < o.low_bits)
        fail(ISG_ERR_INVALID, "no independent set of low_bits spins below the shard bits");
    p.b = (int)low.size();
    const int shards_log2 = [&] { int t = 0; while (((int64_t)1 << t) < (hi - lo)) ++t; return t; }();
    p.q = inner_bits_for(o, free, p.b, shards_log2);
    order_spins(p, n, free, low, nullptr);

    // Histogram geometry: the program's bytes and the widest row stride that fits shared memory.
    std::vector<int32_t> w;
    weight_classes(g, w);
    const size_t prog_bytes = blob_words(n, (int)w.size()) * 8;
    // Lane tables (lane_model 4) make every warp reduction conflict-free; single-graph plans take
    // them by default wherever one copy (or the caller's copies) fits shared memory and the caller
    // fixes no stride. Any layout takes at least n_e_c (10 (N - 5) + 32) words a copy: above that
    // bound no layout is computed.
    Plan lt;
    bool lane_tables = false;
    if (o.lane_model == 4 || (o.lane_model == 0 && single_graph && o.bin_stride == 0 && o.stride_residue == 0 &&
                              !o.warp_aggregate)) {
        const int64_t least_words = g.n_e_c * (int64_t)(10 * (n - 5) + 32);
        if (prog_bytes + (size_t)least_words * 4 > d.smem_optin) {
            if (o.lane_model == 4)
                fail(ISG_ERR_TOO_LARGE, "histogram of " + std::to_string(g.n_e_c * (n + 1)) +
                                            " bins in lane tables does not fit shared memory");
        } else {
            lane_table_layout(lt, n, g.n_e_c, g.G, o.lane_model == 4 ? o.bin_stride : 0);
            lane_tables = o.lane_model == 4 ||
                          prog_bytes + (size_t)std::max(1, o.copies) * (size_t)lt.copy_words * 4 <= d.smem_optin;
        }
    }
    int max_stride = n + 1;
    while (max_stride < n + 32 && prog_bytes + (size_t)g.n_e_c * (max_stride + 1) * 4 <= d.smem_optin) ++max_stride;

    // Lane spins by the bank-conflict model (lanes.cpp): the index order's five spins at q..q+4
    // are one candidate; another set moves to those positions, with the low block and the other
    // inner spins chosen among the rest.
    // lane_model 0: with autotune the thorough search (graphs of kLaneModelMinFree free spins or
    // more), else the quick one from kLaneQuickMinFree free spins (enumerations of several
    // milliseconds against a search of about three); batches and the server choose explicitly
    const bool plain_quick = o.lane_model == 0 && single_graph && !o.autotune && free >= kLaneQuickMinFree;
    const bool use_model = o.lane_model == 1 || o.lane_model == 3 || plain_quick ||
                           (o.lane_model == 0 && single_graph && o.autotune && free >= kLaneModelMinFree);
    LaneChoice lc;
    if (use_model && !lane_tables && prog_bytes + (size_t)g.n_e_c * (n + 1) * 4 <= d.smem_optin) {
        const uint64_t pool = free >= 64 ? ~0ull : ((1ull << free) - 1);
        if (o.lane_model == 3 || plain_quick)
            lc = choose_lanes_in(g, pool, &p.perm[p.q], n + 1, std::min(max_stride, n + 32), g.G, true, true);
        else
            lc = choose_lanes(g, pool, &p.perm[p.q], max_stride);
    }
    if (lc.valid) {
        p.lane_model = true;
        p.lane_cost = lc.cost;
        p.lane_cost_index_order = lc.cost_index_order;
        uint64_t lane_mask = 0;
        for (int t = 0; t < 5; ++t) lane_mask |= 1ull << lc.spins[t];
        bool same = true;
        for (int t = 0; t < 5; ++t) same = same && p.perm[p.q + t] == lc.spins[t];
        if (!same) {
            std::vector<int> low2 = low_block_spins(g, free, bmax, lane_mask);
            if (low2.size() < low.size()) {
                // the low block would shrink (more mid flips, each with its program loads), which
                // costs more than the conflicts save: keep the index order
                p.lane_model = false;
                p.lane_cost = p.lane_cost_index_order = 0;
            } else {
                p.b = (int)low2.size();
                p.q = inner_bits_for(o, free, p.b, shards_log2);
                order_spins(p, n, free, low2, lc.spins);
            }
        }
    }
    const int pk = free - p.q;               // outer bits below the shard bits
    p.prefix_base = (uint64_t)lo << pk;
    p.n_tasks = ((uint64_t)(hi - lo) << pk) / 32;

    // Launch shape and shared memory. Lane tables too large for two CTAs per SM take one CTA of
    // 1024 threads by default.
    p.threads = o.block_threads > 0 ? o.block_threads : 512;
    if (lane_tables && o.block_threads == 0 && o.ctas_per_sm == 0 &&
        2 * (prog_bytes + (size_t)lt.copy_words * 4 + 1024) > d.smem_per_sm)
        p.threads = 1024;
    if (p.threads % 32 || p.threads < 32 || p.threads > 1024) fail(ISG_ERR_INVALID, "block_threads must be a multiple of 32 in [32, 1024]");
    const int warps = p.threads / 32;
    // row stride: the model's pick for its lane spins, unless the caller fixes a stride or residue;
    // lane tables take their layout's (the caller's, if fixed)
    if (lane_tables) p.stride = lt.stride;
    else if (p.lane_model && o.bin_stride == 0 && o.stride_residue == 0) p.stride = lc.stride;
    else p.stride = choose_stride(g, o.bin_stride, o.stride_residue);
    if (!lane_tables && prog_bytes + (size_t)g.n_e_c * p.stride * 4 > d.smem_optin && o.bin_stride == 0) p.stride = n + 1;
    const int64_t nb = (int64_t)g.n_e_c * p.stride;
    if (lane_tables) {
        p.n_sub = lt.n_sub;
        p.packed = lt.packed;
        p.copy_words = lt.copy_words;
        std::copy(lt.sub_off, lt.sub_off + kLaneTables, p.sub_off);
        std::copy(lt.sub_m_lo, lt.sub_m_lo + kLaneTables, p.sub_m_lo);
        std::copy(lt.sub_m_hi, lt.sub_m_hi + kLaneTables, p.sub_m_hi);
        std::copy(lt.lane_word, lt.lane_word + 32, p.lane_word);
        std::copy(lt.lane_sub, lt.lane_sub + 32, p.lane_sub);
    } else {
        p.n_sub = 1;
        p.copy_words = (int)nb;
        p.sub_off[0] = 0;
        p.sub_m_lo[0] = 0;
        p.sub_m_hi[0] = n;
    }
    const size_t bin_bytes = (size_t)p.copy_words * 4;
    if (prog_bytes + bin_bytes > d.smem_optin)
        fail(ISG_ERR_TOO_LARGE, "histogram of " + std::to_string(g.n_e_c * (n + 1)) + " bins" +
                                    (lane_tables ? " in lane tables" : "") + " does not fit shared memory");
    p.ctas_per_sm = o.ctas_per_sm > 0 ? o.ctas_per_sm : 2;
    if (o.copies > 0) {
        p.copies = o.copies;
        if (p.copies > warps) fail(ISG_ERR_INVALID, "copies must not exceed warps per CTA");
        if (prog_bytes + p.copies * bin_bytes > d.smem_optin) fail(ISG_ERR_TOO_LARGE, "copies do not fit shared memory");
    } else if (lane_tables) {
        // no bank conflicts to spread: one copy a CTA (the least to clear and flush) ran as fast
        // as two or four on the 6x6 torus and saved 1.6 us of a 4x4 call
        p.copies = 1;
    } else {
        const size_t per_cta = std::min(d.smem_optin, d.smem_per_sm / p.ctas_per_sm - 1024);
        int c = 1;
        while (c * 2 <= warps && prog_bytes + (size_t)(c * 2) * bin_bytes <= per_cta) c *= 2;
        p.copies = c;
    }
    p.smem_bytes = prog_bytes + (size_t)p.copies * bin_bytes;
    while (p.ctas_per_sm > 1 && (p.smem_bytes + 1024) * p.ctas_per_sm > d.smem_per_sm) --p.ctas_per_sm;
    const uint64_t per_copy_warps = (uint64_t)((warps + p.copies - 1) / p.copies);
    const uint64_t per_round = per_copy_warps << (p.q + 5);      // max increments of a bin per round
    uint64_t F = 0xffffffffull / per_round;
    if (F < 1) fail(ISG_ERR_INVALID, "inner_bits too large for 32-bit bins with this many warps per copy");
    if (o.flush_tasks > 0) F = std::min<uint64_t>(F, (uint64_t)o.flush_tasks);
    p.flush_rounds = (int)std::min<uint64_t>(F, 1u << 30);
    p.grid = (int)std::max<uint64_t>(1, std::min<uint64_t>(p.n_tasks, (uint64_t)d.sms * p.ctas_per_sm));
    p.aggregate = o.warp_aggregate != 0;
    return p;
}

// ---------------------------------------------------------------------------------------------
// Program blob
// ---------------------------------------------------------------------------------------------
std::vector<uint64_t> build_program(const isg_graph& g, const Plan& p) {
    const int n = g.n;
    std::vector<int32_t> w;
    const int binary = weight_classes(g, w);
    const int nc = (int)w.size();
    const size_t words = blob_words(n, nc);
    std::vector<uint64_t> blob(words, 0);
    ProgHeader h{};
    h.n = n;
    h.q = p.q;
    h.b = p.b;
    h.nc = nc;
    h.n_m = n + 1;
    h.n_e_c = (int32_t)g.n_e_c;
    const int stride = p.stride > 0 ? p.stride : n + 1;
    h.stride = stride;
    h.nbins_c = (int32_t)(g.n_e_c * stride);
    h.G = (int32_t)g.G;
    h.sE = (int32_t)(8 * stride / g.G);
    h.words = (int32_t)words;
    h.e_lo = g.e_lo;
    h.S = g.S;
    h.off_site = kHeaderWords;
    h.off_maskx = kHeaderWords + n * (int)(sizeof(SiteRec) / 8);
    h.off_w = h.off_maskx + n * (nc - 1);
    h.w0 = w[0];
    std::memcpy(blob.data(), &h, sizeof h);
    SiteRec* site = reinterpret_cast<SiteRec*>(blob.data() + h.off_site);
    uint64_t* maskx = blob.data() + h.off_maskx;
    int32_t* wv = reinterpret_cast<int32_t*>(blob.data() + h.off_w);
    for (int c = 0; c < nc; ++c) wv[c] = w[c];
    for (int a = 0; a < n; ++a) {
        const int ca = p.perm[a];
        SiteRec& rec = site[a];
        int64_t dw = 0;
        for (int b = 0; b < n; ++b) {
            const int64_t J = g.K[(size_t)ca * n + p.perm[b]];
            if (!J) continue;
            const int64_t aJ = J < 0 ? -J : J;
            dw += aJ;
            if (J < 0) rec.sgn |= 1ull << b;
            for (int c = 0; c < nc; ++c) {
                const bool in = binary ? ((aJ & w[c]) != 0) : (aJ == w[c]);
                if (!in) continue;
                if (c == 0) rec.mask0 |= 1ull << b;
                else maskx[(size_t)a * (nc - 1) + c - 1] |= 1ull << b;
            }
        }
        rec.degw = (int32_t)dw;
        for (int k = 0; k < p.b; ++k)
            rec.A[k] = (a >= p.b) ? (int32_t)(-2 * g.K[(size_t)p.perm[k] * n + ca] * h.sE) : 0;
    }
    return blob;
}

void rank_shards(int n, int rank, int world, bool sym, int32_t& bits, int64_t& lo, int64_t& hi) {
    if (world < 1 || world > (1 << 20)) fail(ISG_ERR_INVALID, "world_size must lie in [1, 2^20]");
    if (rank < 0 || rank >= world) fail(ISG_ERR_INVALID, "rank must lie in [0, world_size)");
    // A power-of-two world splits the space evenly on log2(world) bits; any other world gets 64
    // times as many shards as ranks, so contiguous shares differ by at most one shard in 64.
    int L = 0;
    while ((1 << L) < world) ++L;
    int k = ((1 << L) == world) ? L : L + 6;
    k = std::min(k, sym ? n - 1 : n);
    const int64_t shards = (int64_t)1 << k;
    lo = (int64_t)rank * shards / world;
    hi = (int64_t)(rank + 1) * shards / world;
    bits = k;
    if (sym) {                                         // the top bit (spin N-1) up
        bits = k + 1;
        lo += shards;
        hi += shards;
    }
}

std::shared_ptr<const PlannedProgram> planned_program(const isg_graph& g, const isg_options& o, const DeviceInfo& d) {
    std::string key(reinterpret_cast<const char*>(&o), sizeof o);   // padding bytes can only cause misses
    key.append(reinterpret_cast<const char*>(&d), sizeof d);
    {
        std::lock_guard<std::mutex> lk(g.plan_mu);
        for (const auto& e : g.plan_cache)
            if (e.first == key) return e.second;
    }
    auto pp = std::make_shared<PlannedProgram>();
    pp->plan = make_plan(g, o, d, true);
    pp->blob = build_program(g, pp->plan);
    std::lock_guard<std::mutex> lk(g.plan_mu);
    if (g.plan_cache.size() >= 8) g.plan_cache.erase(g.plan_cache.begin());
    g.plan_cache.emplace_back(std::move(key), pp);
    return pp;
}

// ---------------------------------------------------------------------------------------------
// Host emulation of the kernels (same lane walk, bounds-checked counting)
// ---------------------------------------------------------------------------------------------
// Counts into one histogram copy; every address must be 4-byte aligned and lie among the bins of
// the counting lane's own sub-table: word first + e' stride + m with e' < rows and m in [m_lo, m_hi].
struct HostSink {
    std::vector<uint32_t>* hist;
    int64_t first, stride, rows, m_lo, m_hi;
    bool bad = false;
    void operator()(uint32_t& idx) {
        const int64_t w = (int64_t)(idx >> 2) - first;
        const int64_t e = w >= 0 ? w / stride : -1, m = w - e * stride;
        if ((idx & 3u) || w < 0 || e >= rows || m < m_lo || m > m_hi || (idx >> 2) >= hist->size()) { bad = true; return; }
        (*hist)[idx >> 2] += 1;
    }
};

template <int B>
static void emulate_tasks(const ProgView& v, const Plan& p, int64_t rows, std::vector<uint32_t>& hist, unsigned int& word) {
    for (uint64_t t = 0; t < p.n_tasks; ++t)
        for (int lane = 0; lane < 32; ++lane) {
            const uint32_t base = (uint32_t)p.lane_word[lane] * 4u;
            const int sub = p.lane_sub[lane];
            HostSink sink{&hist, p.lane_word[lane], p.stride, rows, p.sub_m_lo[sub], p.sub_m_hi[sub]};
            uint64_t last_state;
            uint32_t last_idx;
            lane_walk<B>(v, p.prefix_base + t * 32 + lane, base, sink, last_state, last_idx);
            if (last_idx != base + bin_offset(v, last_state)) word |= kSelfCheckLostBin;
            if (sink.bad) word |= kSelfCheckOutOfRange;
        }
}

// The kernels' walk on the host (see isg_debug_emulate). plant_site >= 0 plants a mistake in the
// program first: plant_delta is added to the field constant (sum |J|) in the site record at
// internal position plant_site, as a wrong program entry would. Returns the self-check word the
// walk produced.
static unsigned int emulate(const isg_graph& g, isg_options o, int plant_site, int32_t plant_delta, int64_t* g_out) {
    const bool sym = o.symmetry != 0;
    if (sym) { o.shard_bits = 1; o.shard_lo = 1; o.shard_hi = 2; }     // spin N-1 up only
    Plan p = make_plan(g, o, DeviceInfo{}, true);
    std::vector<uint64_t> blob = build_program(g, p);
    if (plant_site >= 0) {
        if (p.small || plant_site >= g.n) fail(ISG_ERR_INVALID, "no site record to plant a mistake in");
        SiteRec* site = reinterpret_cast<SiteRec*>(blob.data() + reinterpret_cast<const ProgHeader*>(blob.data())->off_site);
        site[plant_site].degw += plant_delta;
    }
    const ProgView v = make_view(blob.data());
    const int64_t stride = p.stride > 0 ? p.stride : g.n + 1;
    const int64_t nb = g.n_e_c * stride;
    std::vector<uint32_t> hist((size_t)std::max<int64_t>(nb, p.copy_words), 0);   // one copy
    unsigned int word = 0;
    if (p.small) {
        for (uint64_t s = p.s_lo; s < p.s_hi; ++s) {
            const uint32_t off = bin_offset(v, s);
            if ((off & 3u) || off >= nb * 4) { word |= kSelfCheckOutOfRange; continue; }
            hist[off >> 2] += 1;
        }
    } else {
        switch (p.b) {
            case 1: emulate_tasks<1>(v, p, g.n_e_c, hist, word); break;
            case 2: emulate_tasks<2>(v, p, g.n_e_c, hist, word); break;
            case 3: emulate_tasks<3>(v, p, g.n_e_c, hist, word); break;
            case 4: emulate_tasks<4>(v, p, g.n_e_c, hist, word); break;
            case 5: emulate_tasks<5>(v, p, g.n_e_c, hist, word); break;
            case 6: emulate_tasks<6>(v, p, g.n_e_c, hist, word); break;
            case 7: emulate_tasks<7>(v, p, g.n_e_c, hist, word); break;
            default: fail(ISG_ERR_INTERNAL, "bad low block size");
        }
    }
    if (word) return word;
    std::vector<int64_t> tab((size_t)public_bins(g), 0);
    if (p.small) {
        for (int64_t i = 0; i < nb; ++i) {
            if (!hist[(size_t)i]) continue;
            const int64_t pb = public_bin(g, i, stride);
            if (pb < 0) fail(ISG_ERR_INTERNAL, "emulated walk counted a padding column");
            tab[pb] += hist[(size_t)i];
        }
    } else {
        for (int t = 0; t < p.n_sub; ++t)              // the flush: each sub-table's own columns
            for (int64_t e = 0; e < g.n_e_c; ++e)
                for (int64_t m = p.sub_m_lo[t]; m <= p.sub_m_hi[t]; ++m)
                    tab[public_bin(g, e * stride + m, stride)] += hist[(size_t)(p.sub_off[t] + e * stride + m)];
    }
    if (!o.accumulate) std::memset(g_out, 0, sizeof(int64_t) * public_bins(g));
    const int64_t n_m = g.n + 1;
    for (int64_t e = 0; e <= g.S; ++e)
        for (int64_t m = 0; m < n_m; ++m)
            g_out[e * n_m + m] += tab[e * n_m + m] + (sym ? tab[e * n_m + (n_m - 1 - m)] : 0);
    return 0;
}

}  // namespace isg

using namespace isg;

extern "C" {

void isg_options_init(isg_options* opt) {
    if (!opt) return;
    std::memset(opt, 0, sizeof *opt);
    opt->struct_size = (int32_t)sizeof(isg_options);
    opt->max_spins = 40;
}

const char* isg_last_error(void) { return t_last_error.c_str(); }

const char* isg_version(void) { return "isg 0.1 (sm_103a)"; }

isg_status isg_graph_create(int32_t n_spins, int64_t n_edges, const int32_t* ei, const int32_t* ej,
                            const int32_t* J, isg_graph** out) {
    return guarded([&] {
        if (!out) fail(ISG_ERR_INVALID, "out is NULL");
        *out = nullptr;
        if (n_spins < 1 || n_spins > kMaxSpins) fail(ISG_ERR_INVALID, "n_spins must lie in [1, 64]");
        if (n_edges < 0) fail(ISG_ERR_INVALID, "n_edges must be >= 0");
        if (n_edges > 0 && (!ei || !ej || !J)) fail(ISG_ERR_INVALID, "edge arrays are NULL");
        isg_graph* g = new isg_graph();
        try {
            const int n = n_spins;
            g->n = n;
            g->K.assign((size_t)n * n, 0);
            for (int64_t b = 0; b < n_edges; ++b) {
                const int i = ei[b], j = ej[b];
                if (i < 0 || j < 0 || i >= n || j >= n) fail(ISG_ERR_INVALID, "edge " + std::to_string(b) + " has an endpoint out of range");
                if (i == j) fail(ISG_ERR_INVALID, "edge " + std::to_string(b) + " is a self loop");
                if (J[b] == 0 || J[b] > (1 << 20) || J[b] < -(1 << 20)) fail(ISG_ERR_INVALID, "edge " + std::to_string(b) + " has J = 0 or |J| > 2^20");
                g->K[(size_t)i * n + j] += J[b];
                g->K[(size_t)j * n + i] += J[b];
            }
            g->degree.assign(n, 0);
            int64_t gg = 0;
            for (int i = 0; i < n; ++i) {
                int64_t sum = 0, gi = 0;
                bool any = false;
                for (int j = 0; j < n; ++j) {
                    const int64_t v = g->K[(size_t)i * n + j];
                    if (!v) continue;
                    if (std::llabs(v) > (1 << 20)) fail(ISG_ERR_INVALID, "summed coupling exceeds 2^20 in magnitude");
                    any = true;
                    g->degree[i]++;
                    sum += v;
                    gi = igcd(gi, 2 * v);
                    if (j > i) { g->bi.push_back(i); g->bj.push_back(j); g->bJ.push_back(v); g->S += std::llabs(v); }
                }
                if (any) gg = igcd(gg, igcd(sum, gi));
            }
            g->e_ref = 0;
            for (size_t b = 0; b < g->bJ.size(); ++b) g->e_ref -= g->bJ[b];
            int64_t G = gg ? 2 * gg : 2;
            G = igcd(G, 8 * (int64_t)(n + 1));          // keep 8 (N + 1) / G integral
            g->G = G;
            g->e_lo = g->e_ref - G * ((g->e_ref + g->S) / G);
            g->n_e_c = (g->S - g->e_lo) / G + 1;
        } catch (...) {
            delete g;
            throw;
        }
        *out = g;
    });
}

void isg_graph_destroy(isg_graph* graph) { delete graph; }

isg_status isg_graph_bins(const isg_graph* g, int32_t* e_min, int32_t* e_step, int32_t* n_e, int32_t* m_min,
                          int32_t* n_m) {
    return guarded([&] {
        if (!g) fail(ISG_ERR_INVALID, "graph is NULL");
        if (g->S > (int64_t)1 << 30) fail(ISG_ERR_TOO_LARGE, "energy range exceeds int32");
        if (e_min) *e_min = (int32_t)(-g->S);
        if (e_step) *e_step = 2;
        if (n_e) *n_e = (int32_t)(g->S + 1);
        if (m_min) *m_min = -g->n;
        if (n_m) *n_m = g->n + 1;
    });
}

isg_status isg_graph_size(const isg_graph* g, int32_t* n_spins, int32_t* n_bonds) {
    return guarded([&] {
        if (!g) fail(ISG_ERR_INVALID, "graph is NULL");
        if (n_spins) *n_spins = g->n;
        if (n_bonds) *n_bonds = (int32_t)g->bJ.size();
    });
}

isg_status isg_debug_plan(const isg_graph* g, const isg_options* opt, int32_t sms, int64_t* out) {
    return guarded([&] {
        if (!g || !out) fail(ISG_ERR_INVALID, "NULL argument");
        isg_options o = resolve_options(opt);
        DeviceInfo d;
        if (sms > 0) d.sms = sms;
        Plan p = make_plan(*g, o, d, true);
        out[0] = p.small;
        out[1] = p.q;
        out[2] = p.b;
        out[3] = (int64_t)p.n_tasks;
        out[4] = p.threads;
        out[5] = p.copies;
        out[6] = p.ctas_per_sm;
        out[7] = p.flush_rounds;
        out[8] = p.grid;
        out[9] = (int64_t)p.smem_bytes;
        out[10] = g->G;
        out[11] = g->n_e_c;
        out[12] = (int64_t)build_program(*g, p).size() * 8;
        out[13] = p.stride;
        out[14] = p.lane_model;
        out[15] = (int64_t)std::llround(p.lane_cost * 1e6);
        out[16] = (int64_t)std::llround(p.lane_cost_index_order * 1e6);
        int64_t lanes = 0;
        if (!p.small) for (int t = 0; t < 5; ++t) lanes |= (int64_t)1 << p.perm[p.q + t];
        out[17] = lanes;
        out[18] = p.n_sub;
    });
}

isg_status isg_debug_lane_banks(const isg_graph* g, const isg_options* opt, int32_t samples, uint64_t seed,
                                double* mean_wavefronts, int32_t* max_wavefronts) {
    return guarded([&] {
        if (!g || !mean_wavefronts || !max_wavefronts || samples < 1) fail(ISG_ERR_INVALID, "bad argument");
        const isg_options o = resolve_options(opt);
        const Plan p = make_plan(*g, o, DeviceInfo{}, true);
        if (p.small) fail(ISG_ERR_INVALID, "a thread-per-configuration plan has no warp reductions");
        const std::vector<uint64_t> blob = build_program(*g, p);
        const ProgView v = make_view(blob.data());
        uint64_t x = seed;
        auto next = [&x] {                       // splitmix64
            uint64_t z = (x += 0x9E3779B97F4A7C15ull);
            z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
            z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
            return z ^ (z >> 31);
        };
        double total = 0;
        int worst = 0;
        for (int sample = 0; sample < samples; ++sample) {
            const uint64_t t = next() % p.n_tasks;
            const uint64_t inner = next() & ((1ull << p.q) - 1);
            uint32_t addr[32];
            for (int lane = 0; lane < 32; ++lane) {
                const uint64_t st = ((p.prefix_base + t * 32 + lane) << p.q) | inner;
                addr[lane] = (uint32_t)p.lane_word[lane] + bin_offset(v, st) / 4;
            }
            int per_bank[32] = {};
            for (int lane = 0; lane < 32; ++lane) {
                bool seen = false;
                for (int j = 0; j < lane; ++j) seen = seen || addr[j] == addr[lane];
                if (!seen) ++per_bank[addr[lane] & 31];
            }
            const int wf = *std::max_element(per_bank, per_bank + 32);
            total += wf;
            worst = std::max(worst, wf);
        }
        *mean_wavefronts = total / samples;
        *max_wavefronts = worst;
    });
}

isg_status isg_debug_lane_layout(const isg_graph* g, const isg_options* opt, int32_t* out) {
    return guarded([&] {
        if (!g || !out) fail(ISG_ERR_INVALID, "NULL argument");
        const Plan p = make_plan(*g, resolve_options(opt), DeviceInfo{}, true);
        if (p.small) fail(ISG_ERR_INVALID, "a thread-per-configuration plan has no histogram copies");
        std::fill(out, out + 99, 0);
        out[0] = p.stride;
        out[1] = p.copy_words;
        out[2] = p.n_sub;
        for (int t = 0; t < p.n_sub; ++t) {
            out[3 + t] = p.sub_off[t];
            out[13 + t] = p.sub_m_lo[t];
            out[23 + t] = p.sub_m_hi[t];
        }
        for (int l = 0; l < 32; ++l) {
            out[33 + l] = p.lane_word[l];
            out[65 + l] = p.lane_sub[l];
        }
        out[97] = p.packed;
    });
}

isg_status isg_debug_emulate(const isg_graph* g, const isg_options* opt, int64_t* g_out) {
    return guarded([&] {
        if (!g || !g_out) fail(ISG_ERR_INVALID, "NULL argument");
        check_self_check_word(emulate(*g, resolve_options(opt), -1, 0, g_out), "emulated enumeration");
    });
}

isg_status isg_rank_shards(int32_t n_spins, int32_t rank, int32_t world_size, int32_t symmetry, int32_t* shard_bits,
                           int64_t* shard_lo, int64_t* shard_hi) {
    return guarded([&] {
        if (n_spins < 1 || n_spins > kMaxSpins) fail(ISG_ERR_INVALID, "n_spins must lie in [1, 64]");
        int32_t bits = 0;
        int64_t lo = 0, hi = 0;
        rank_shards(n_spins, rank, world_size, symmetry != 0, bits, lo, hi);
        if (shard_bits) *shard_bits = bits;
        if (shard_lo) *shard_lo = lo;
        if (shard_hi) *shard_hi = hi;
    });
}

isg_status isg_debug_emulate_rank(const isg_graph* g, int32_t rank, int32_t world_size, const isg_options* opt,
                                  int64_t* g_out) {
    return guarded([&] {
        if (!g || !g_out) fail(ISG_ERR_INVALID, "NULL argument");
        isg_options o = resolve_options(opt);
        if (o.shard_bits || o.shard_lo || o.shard_hi) fail(ISG_ERR_INVALID, "the rank's shards come from rank and world_size");
        const bool sym = o.symmetry != 0;
        int32_t bits = 0;
        int64_t lo = 0, hi = 0;
        rank_shards(g->n, rank, world_size, sym, bits, lo, hi);
        if (lo == hi) {
            if (!o.accumulate) std::memset(g_out, 0, sizeof(int64_t) * public_bins(*g));
            return;
        }
        o.symmetry = 0;
        o.shard_bits = bits;
        o.shard_lo = lo;
        o.shard_hi = hi;
        std::vector<int64_t> part((size_t)public_bins(*g), 0);
        check_self_check_word(emulate(*g, o, -1, 0, part.data()), "emulated enumeration");
        if (!o.accumulate) std::memset(g_out, 0, sizeof(int64_t) * public_bins(*g));
        const int64_t n_m = g->n + 1;
        for (int64_t e = 0; e <= g->S; ++e)
            for (int64_t m = 0; m < n_m; ++m)
                g_out[e * n_m + m] += part[e * n_m + m] + (sym ? part[e * n_m + (n_m - 1 - m)] : 0);
    });
}

isg_status isg_debug_emulate_planted(const isg_graph* g, const isg_options* opt, int32_t site, int32_t delta,
                                     int64_t* g_out, uint32_t* word) {
    return guarded([&] {
        if (!g || !g_out) fail(ISG_ERR_INVALID, "NULL argument");
        if (site < 0) fail(ISG_ERR_INVALID, "site must be >= 0");
        const unsigned int w = emulate(*g, resolve_options(opt), site, delta, g_out);
        if (word) *word = w;
        check_self_check_word(w, "emulated enumeration");
    });
}

}  // extern "C"
