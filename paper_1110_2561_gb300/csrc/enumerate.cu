// enumerate.cu -- sm_103a kernels that enumerate all configurations of a graph into the exact
// degeneracy table g(E, M) (arXiv:1110.2561, Sec. 2-3), and the isg_enumerate entry point.
//
// Work decomposition (the paper splits the outer loops over MPI ranks, Sec. 3d; here the outer
// configuration bits are split over warps of one GPU): a task is 32 consecutive outer prefixes,
// one per lane; each lane walks the 2^q inner configurations of its prefix in Gray order
// (enum_core.cuh). Warps take tasks from a global counter, so uneven progress balances itself.
// Counts go into 32-bit shared-memory bins privatised per group of warps (red.shared.add), which
// a CTA-wide flush adds into the int64 table with 64-bit global atomics before any bin can wrap.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <map>
#include <memory>
#include <mutex>
#include <set>
#include <string>
#include <tuple>
#include <vector>

#include "enum_kernels.cuh"
#include "isg_internal.h"
#include "nvtx_range.h"

namespace isg {

// Self-check word of the device-output calls on this device: kernels OR a failed check into it
// (atomicOr, so calls on any stream may share it); isg_device_status reads and clears it.
static __device__ unsigned int g_device_status;

// ---------------------------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------------------------
unsigned int* device_status_word() {
    static std::mutex mu;
    static std::vector<unsigned int*> addr;
    int dev = 0;
    ISG_CUDA(cudaGetDevice(&dev));
    std::lock_guard<std::mutex> lk(mu);
    if ((int)addr.size() <= dev) addr.resize(dev + 1, nullptr);
    if (!addr[dev]) {
        void* p = nullptr;
        ISG_CUDA(cudaGetSymbolAddress(&p, g_device_status));
        addr[dev] = static_cast<unsigned int*>(p);
    }
    return addr[dev];
}

// The pool of pinned staging buffers (at most kStagePool kept; larger requests replace smaller
// buffers). Never freed at exit: pinned memory goes back to the system with the process.
static std::mutex g_stage_mu;
static std::vector<std::pair<char*, size_t>> g_stage_free;
constexpr size_t kStagePool = 8;

PinnedStage::PinnedStage(size_t bytes, void* stream) : stream_(stream) {
    bytes = std::max<size_t>(bytes, 1);
    {
        std::lock_guard<std::mutex> lk(g_stage_mu);
        size_t best = g_stage_free.size();
        for (size_t i = 0; i < g_stage_free.size(); ++i)
            if (g_stage_free[i].second >= bytes && (best == g_stage_free.size() || g_stage_free[i].second < g_stage_free[best].second))
                best = i;
        if (best < g_stage_free.size()) {
            p_ = g_stage_free[best].first;
            cap_ = g_stage_free[best].second;
            g_stage_free.erase(g_stage_free.begin() + (std::ptrdiff_t)best);
            return;
        }
    }
    cap_ = std::max<size_t>(64 << 10, (bytes + 4095) & ~(size_t)4095);
    void* p = nullptr;
    const cudaError_t e = cudaMallocHost(&p, cap_);
    if (e != cudaSuccess) fail(ISG_ERR_NOMEM, std::string("cudaMallocHost(staging): ") + cudaGetErrorString(e));
    p_ = static_cast<char*>(p);
}

PinnedStage::~PinnedStage() {
    if (!synced_) cudaStreamSynchronize(static_cast<cudaStream_t>(stream_));
    std::lock_guard<std::mutex> lk(g_stage_mu);
    if (g_stage_free.size() < kStagePool) {
        g_stage_free.emplace_back(p_, cap_);
        return;
    }
    size_t smallest = 0;                          // keep the larger buffers
    for (size_t i = 1; i < g_stage_free.size(); ++i)
        if (g_stage_free[i].second < g_stage_free[smallest].second) smallest = i;
    if (g_stage_free[smallest].second < cap_) {
        std::swap(g_stage_free[smallest].first, p_);
        std::swap(g_stage_free[smallest].second, cap_);
    }
    cudaFreeHost(p_);
}

void* scratch_alloc(size_t bytes, void* stream) {
    static std::mutex mu;
    static std::vector<cudaMemPool_t> pools;
    int dev = 0;
    ISG_CUDA(cudaGetDevice(&dev));
    cudaMemPool_t pool;
    {
        std::lock_guard<std::mutex> lk(mu);
        if ((int)pools.size() <= dev) pools.resize(dev + 1, nullptr);
        if (!pools[dev]) {
            cudaMemPoolProps props;
            std::memset(&props, 0, sizeof props);
            props.allocType = cudaMemAllocationTypePinned;
            props.location.type = cudaMemLocationTypeDevice;
            props.location.id = dev;
            ISG_CUDA(cudaMemPoolCreate(&pools[dev], &props));
            uint64_t keep = ~0ull;
            ISG_CUDA(cudaMemPoolSetAttribute(pools[dev], cudaMemPoolAttrReleaseThreshold, &keep));
        }
        pool = pools[dev];
    }
    void* p = nullptr;
    ISG_CUDA(cudaMallocFromPoolAsync(&p, bytes, pool, static_cast<cudaStream_t>(stream)));
    return p;
}

DeviceInfo device_info() {
    static std::mutex mu;
    static std::vector<DeviceInfo> cache;
    static std::vector<char> have;
    int dev = 0;
    ISG_CUDA(cudaGetDevice(&dev));
    std::lock_guard<std::mutex> lk(mu);
    if ((int)cache.size() <= dev) { cache.resize(dev + 1); have.resize(dev + 1, 0); }
    if (!have[dev]) {
        DeviceInfo d;
        int v = 0;
        ISG_CUDA(cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev));
        d.sms = v;
        ISG_CUDA(cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
        d.smem_optin = (size_t)v;
        ISG_CUDA(cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev));
        d.smem_per_sm = (size_t)v;
        cache[dev] = d;
        have[dev] = 1;
    }
    return cache[dev];
}

int kernel_occupancy(const void* kernel, int threads, size_t smem) {
    static std::mutex mu;
    static std::map<std::tuple<int, const void*, int, size_t>, int> occ_cache;
    static std::set<std::pair<int, const void*>> raised;
    int dev = 0;
    ISG_CUDA(cudaGetDevice(&dev));
    const size_t optin = device_info().smem_optin;
    std::lock_guard<std::mutex> lk(mu);
    const auto key = std::make_tuple(dev, kernel, threads, smem);
    const auto it = occ_cache.find(key);
    if (it != occ_cache.end()) return it->second;
    if (!raised.count({dev, kernel})) {
        // the dynamic limit may reach the device maximum less the kernel's static shared memory
        cudaFuncAttributes fa;
        ISG_CUDA(cudaFuncGetAttributes(&fa, kernel));
        ISG_CUDA(cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)(optin - std::min(optin, fa.sharedSizeBytes))));
        raised.insert({dev, kernel});
    }
    int occ = 0;
    ISG_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kernel, threads, smem));
    occ_cache[key] = occ;
    return occ;
}

// Grid: the planned CTAs per SM, capped by what the registers and shared memory of this
// instantiation allow (its occupancy), never more than tasks.
template <int B, class Sink>
static void launch_bs(const Plan& p, const EnumParams& a, cudaStream_t s) {
    const int smem = (int)(p.smem_bytes + 16);
    const int occ = kernel_occupancy(reinterpret_cast<const void*>(enumerate_kernel<B, Sink>), p.threads, (size_t)smem);
    if (occ < 1) fail(ISG_ERR_TOO_LARGE, "enumeration kernel does not fit an SM with this block size");
    const DeviceInfo d = device_info();
    const uint64_t want = (uint64_t)d.sms * (uint64_t)std::min(occ, p.ctas_per_sm);
    const int grid = (int)std::max<uint64_t>(1, std::min<uint64_t>(want, p.n_tasks));
    enumerate_kernel<B, Sink><<<grid, p.threads, smem, s>>>(a);
    ISG_CUDA(cudaGetLastError());
}

template <int B>
static void launch_b(const Plan& p, const EnumParams& a, cudaStream_t s) {
    if (p.aggregate) launch_bs<B, MatchSink>(p, a, s);
    else launch_bs<B, SmemSink>(p, a, s);
}

// Enqueue the kernels of one plan; `table` must be zeroed (or hold counts to add to). The program
// is read from d_blob (device), or, when d_blob is NULL, from host_blob, which must then fit the
// kernel parameters (program_fits_inline).
bool program_fits_inline(size_t words) { return words <= (size_t)kInlineProgramWords; }

void launch_enumeration(const Plan& p, const uint64_t* d_blob, int blob_words, int64_t* table,
                        unsigned long long* counter, unsigned int* status, cudaStream_t s,
                        const uint64_t* host_blob) {
    std::unique_ptr<EnumParams> P(new EnumParams());
    EnumArgs& a = P->a;
    if (!d_blob) {
        if (!host_blob || !program_fits_inline((size_t)blob_words)) fail(ISG_ERR_INTERNAL, "program does not fit inline");
        std::memcpy(P->program, host_blob, sizeof(uint64_t) * (size_t)blob_words);
    }
    if (p.small) {
        a.blob = d_blob;
        a.blob_words = blob_words;
        a.g = table;
        kernel_occupancy(reinterpret_cast<const void*>(enumerate_small_kernel), p.threads, (size_t)blob_words * 8);
        enumerate_small_kernel<<<p.grid, p.threads, blob_words * 8, s>>>(*P, p.s_lo, p.s_hi);
        ISG_CUDA(cudaGetLastError());
        return;
    }
    a.blob = d_blob;
    a.g = table;
    a.counter = counter;
    a.status = status;
    a.prefix_base = p.prefix_base;
    a.n_tasks = p.n_tasks;
    a.blob_words = blob_words;
    a.copies = p.copies;
    a.flush_rounds = p.flush_rounds;
    a.copy_words = p.copy_words;
    a.n_sub = p.n_sub;
    for (int t = 0; t < kLaneTables; ++t) {
        a.sub_off[t] = p.sub_off[t];
        a.sub_m_lo[t] = p.sub_m_lo[t];
        a.sub_m_hi[t] = p.sub_m_hi[t];
    }
    for (int l = 0; l < 32; ++l) a.lane_word[l] = p.lane_word[l];
    switch (p.b) {
        case 1: launch_b<1>(p, *P, s); break;
        case 2: launch_b<2>(p, *P, s); break;
        case 3: launch_b<3>(p, *P, s); break;
        case 4: launch_b<4>(p, *P, s); break;
        case 5: launch_b<5>(p, *P, s); break;
        case 6: launch_b<6>(p, *P, s); break;
        case 7: launch_b<7>(p, *P, s); break;
        default: fail(ISG_ERR_INTERNAL, "bad low block size");
    }
}

// ---------------------------------------------------------------------------------------------
// Autotuning: time candidate launch shapes on one shard and cache the winner per graph/device.
// ---------------------------------------------------------------------------------------------
static uint64_t graph_signature(const isg_graph& g) {
    uint64_t h = 1469598103934665603ull;                      // FNV-1a over N and the bond list
    auto mix = [&](uint64_t v) { for (int b = 0; b < 8; ++b) { h ^= (v >> (8 * b)) & 0xff; h *= 1099511628211ull; } };
    mix((uint64_t)g.n);
    for (size_t k = 0; k < g.bJ.size(); ++k) { mix((uint64_t)g.bi[k]); mix((uint64_t)g.bj[k]); mix((uint64_t)g.bJ[k]); }
    return h;
}

struct TunedShape {
    int stride_residue = 0, block_threads = 0, ctas_per_sm = 0, lane_model = 0;
};

static std::mutex g_tune_mu;
static std::map<std::pair<int, uint64_t>, TunedShape> g_tune_cache;

// Time one plan on its own scratch, its warp tasks capped at max_tasks: one warm-up and three
// timed launches, best of three (ms).
static float time_plan(const isg_graph& g, const isg_options& o, cudaStream_t s, int64_t* table, char* scratch,
                       uint64_t max_tasks) {
    const DeviceInfo d = device_info();
    Plan p = make_plan(g, o, d, true);
    p.n_tasks = std::min(p.n_tasks, max_tasks);
    const std::vector<uint64_t> blob = build_program(g, p);
    ISG_CUDA(cudaMemcpyAsync(scratch + 16, blob.data(), blob.size() * 8, cudaMemcpyHostToDevice, s));
    cudaEvent_t e0, e1;
    ISG_CUDA(cudaEventCreate(&e0));
    ISG_CUDA(cudaEventCreate(&e1));
    float best = 1e30f;
    for (int rep = 0; rep < 4; ++rep) {
        ISG_CUDA(cudaMemsetAsync(scratch, 0, 16, s));
        ISG_CUDA(cudaEventRecord(e0, s));
        launch_enumeration(p, reinterpret_cast<const uint64_t*>(scratch + 16), (int)blob.size(), table,
                           reinterpret_cast<unsigned long long*>(scratch), reinterpret_cast<unsigned int*>(scratch + 8), s,
                           nullptr);
        ISG_CUDA(cudaEventRecord(e1, s));
        ISG_CUDA(cudaEventSynchronize(e1));
        float ms = 0;
        ISG_CUDA(cudaEventElapsedTime(&ms, e0, e1));
        if (rep > 0) best = std::min(best, ms);
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return best;
}

// Candidates: the index order's lane spins at five row-stride residues, the bank-conflict
// model's lane spins at its own stride (graphs of at least 30 free spins) and lane tables (where
// ten padded copies of the histogram fit shared memory), each at three launch shapes. A trial runs the full plan with tasks 2^k times shorter (q - k inner bits), cut to the
// full launch's task count, so it keeps the launch's shape at 1/2^k of its work.
static TunedShape run_autotune(const isg_graph& g, const isg_options& base, cudaStream_t s) {
    TunedShape best;
    if (g.n < 30) return best;
    const DeviceInfo d = device_info();
    isg_options o0 = base;                          // the full launch at the planner's own split
    o0.autotune = 0;
    o0.shard_bits = 0; o0.shard_lo = 0; o0.shard_hi = 0; o0.accumulate = 0; o0.inner_bits = 0;
    if (!o0.lane_model) o0.lane_model = 2;
    const Plan p0 = make_plan(g, o0, d, true);
    if (p0.small) return best;
    const int k = std::min(4, p0.q - p0.b);
    if (k < 1) return best;
    const size_t table_bytes = sizeof(int64_t) * (size_t)public_bins(g);
    char* scratch = nullptr;
    scratch = static_cast<char*>(scratch_alloc(16 + 8 * (size_t)1700 + table_bytes + 256, s));
    struct Free {
        char* p; cudaStream_t s;
        ~Free() { if (p) { cudaFreeAsync(p, s); cudaStreamSynchronize(s); } }
    } guard{scratch, s};
    int64_t* table = reinterpret_cast<int64_t*>(scratch + ((16 + 8 * 1700 + 255) & ~(size_t)255));
    ISG_CUDA(cudaMemsetAsync(table, 0, table_bytes, s));
    static const int residues[] = {6, 13, 19, 5, 27};
    static const int shapes[][2] = {{512, 2}, {256, 4}, {1024, 1}};
    std::vector<int> lane_models;
    if (base.lane_model) lane_models.push_back(base.lane_model);
    else {
        lane_models.push_back(2);
        if (g.n >= kLaneModelMinFree) lane_models.push_back(1);
        lane_models.push_back(4);                   // lane tables, where they fit shared memory
    }
    float best_ms = 1e30f;
    for (int lm : lane_models) {
        std::vector<int> rs;
        if (base.stride_residue) rs.push_back(base.stride_residue);
        else if (lm == 1 || lm == 4) rs.push_back(0);   // the model's own stride; lane tables' multiple of 32
        else rs.assign(std::begin(residues), std::end(residues));
        for (int r : rs)
            for (auto& sh : shapes) {
                isg_options c = o0;
                c.lane_model = lm;
                c.stride_residue = r;
                c.block_threads = base.block_threads ? base.block_threads : sh[0];
                c.ctas_per_sm = base.ctas_per_sm ? base.ctas_per_sm : sh[1];
                c.inner_bits = p0.q - k;
                float ms;
                try {
                    ms = time_plan(g, c, s, table, scratch, p0.n_tasks);
                } catch (const Error&) {
                    continue;                       // a shape this graph cannot take
                }
                if (ms < best_ms) {
                    best_ms = ms;
                    best.stride_residue = c.stride_residue;
                    best.block_threads = c.block_threads;
                    best.ctas_per_sm = c.ctas_per_sm;
                    best.lane_model = lm;
                }
            }
    }
    return best;
}

static void fill_tuned(isg_options& o, const TunedShape& t) {
    if (!o.lane_model) o.lane_model = t.lane_model;
    if (!o.stride_residue && !o.bin_stride) o.stride_residue = t.stride_residue;
    if (!o.block_threads) o.block_threads = t.block_threads;
    if (!o.ctas_per_sm) o.ctas_per_sm = t.ctas_per_sm;
}

bool apply_cached_autotune(const isg_graph& g, isg_options& o) {
    int dev = 0;
    ISG_CUDA(cudaGetDevice(&dev));
    std::lock_guard<std::mutex> lk(g_tune_mu);
    const auto it = g_tune_cache.find(std::pair<int, uint64_t>(dev, graph_signature(g)));
    if (it == g_tune_cache.end()) return false;
    fill_tuned(o, it->second);
    return true;
}

// Fill the unset planning fields of o from the cache (tuning on a miss).
static void apply_autotune(const isg_graph& g, isg_options& o, cudaStream_t s) {
    int dev = 0;
    ISG_CUDA(cudaGetDevice(&dev));
    const std::pair<int, uint64_t> key(dev, graph_signature(g));
    TunedShape t;
    bool have = false;
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        auto it = g_tune_cache.find(key);
        if (it != g_tune_cache.end()) { t = it->second; have = true; }
    }
    if (!have) {
        t = run_autotune(g, o, s);
        std::lock_guard<std::mutex> lk(g_tune_mu);
        g_tune_cache[key] = t;
    }
    fill_tuned(o, t);
}

}  // namespace isg

using namespace isg;

extern "C" isg_status isg_autotune(const isg_graph* graph, void* stream, const isg_options* opt, isg_options* tuned) {
    return guarded([&] {
        NvtxRange nvtx("isg_autotune");
        if (!graph || !tuned) fail(ISG_ERR_INVALID, "graph or tuned is NULL");
        isg_options o = resolve_options(opt);
        o.autotune = 1;
        apply_autotune(*graph, o, static_cast<cudaStream_t>(stream));
        *tuned = o;
    });
}

namespace isg {

// Enumerate the shard range of o (planning fields resolved) into g_out; with `mirror` the range
// holds only configurations with spin N-1 up and the counts are completed by the M -> -M mirror
// (a global flip keeps E and negates M). Device output only enqueues; host output synchronises
// and checks the kernels' self-check word.
static void enumerate_range(const isg_graph& graph, cudaStream_t s, int64_t* g_out, bool g_out_on_device,
                            const isg_options& o, bool mirror) {
    const DeviceInfo d = device_info();
    const std::shared_ptr<const PlannedProgram> pp = planned_program(graph, o, d);
    const Plan& p = pp->plan;
    const std::vector<uint64_t>& blob = pp->blob;
    const size_t table_bytes = sizeof(int64_t) * (size_t)public_bins(graph);
    const size_t blob_bytes = blob.size() * 8;
    // scratch: [counter 8][status 8][blob][table: host mode or symmetry half]
    const size_t off_blob = 16, off_table = (off_blob + blob_bytes + 255) & ~(size_t)255;
    const bool own_table = !g_out_on_device || mirror;
    const size_t scratch_bytes = off_table + (own_table ? table_bytes : 0) + (mirror && !g_out_on_device ? table_bytes : 0);
    char* scratch = static_cast<char*>(scratch_alloc(scratch_bytes, s));
    struct Free {
        char* p; cudaStream_t s;
        ~Free() { if (p) cudaFreeAsync(p, s); }
    } guard{scratch, s};
    ISG_CUDA(cudaMemsetAsync(scratch, 0, 16, s));
    const bool inl = program_fits_inline(blob.size());
    if (!inl) ISG_CUDA(cudaMemcpyAsync(scratch + off_blob, blob.data(), blob_bytes, cudaMemcpyHostToDevice, s));
    int64_t* table = own_table ? reinterpret_cast<int64_t*>(scratch + off_table) : g_out;
    if (own_table || !o.accumulate) ISG_CUDA(cudaMemsetAsync(table, 0, table_bytes, s));
    // host output: the call's own status word, read below; device output: the device's word,
    // which isg_device_status reports
    unsigned int* status = g_out_on_device ? device_status_word() : reinterpret_cast<unsigned int*>(scratch + 8);
    launch_enumeration(p, inl ? nullptr : reinterpret_cast<const uint64_t*>(scratch + off_blob), (int)blob.size(),
                       table, reinterpret_cast<unsigned long long*>(scratch), status, s, blob.data());
    if (mirror) {
        const int n_m = graph.n + 1, n_e = (int)(graph.S + 1);
        int64_t* full = g_out_on_device ? g_out : reinterpret_cast<int64_t*>(scratch + off_table + table_bytes);
        const int acc = g_out_on_device ? o.accumulate : 0;
        mirror_kernel<<<std::min(1024, (n_e * n_m + 255) / 256), 256, 0, s>>>(table, full, n_e, n_m, acc);
        ISG_CUDA(cudaGetLastError());
        table = full;
    }
    if (!g_out_on_device) {
        // the table and the status word into pinned memory by asynchronous copies, one synchronisation
        PinnedStage stage(table_bytes + 16, s);
        const int64_t* host = reinterpret_cast<const int64_t*>(stage.data());
        unsigned int* word = reinterpret_cast<unsigned int*>(stage.data() + table_bytes);
        ISG_CUDA(cudaMemcpyAsync(stage.data(), table, table_bytes, cudaMemcpyDeviceToHost, s));
        ISG_CUDA(cudaMemcpyAsync(word, scratch + 8, sizeof *word, cudaMemcpyDeviceToHost, s));
        ISG_CUDA(cudaStreamSynchronize(s));
        stage.synced();
        check_self_check_word(*word, "enumeration");
        const size_t nb = (size_t)public_bins(graph);
        if (o.accumulate) for (size_t i = 0; i < nb; ++i) g_out[i] += host[i];
        else std::memcpy(g_out, host, table_bytes);
    }
}

}  // namespace isg

extern "C" isg_status isg_enumerate(const isg_graph* graph, void* stream, int64_t* g_out, int32_t g_out_on_device,
                                    const isg_options* opt) {
    return guarded([&] {
        NvtxRange nvtx("isg_enumerate");
        if (!graph || !g_out) fail(ISG_ERR_INVALID, "graph or g_out is NULL");
        isg_options o = resolve_options(opt);
        cudaStream_t s = static_cast<cudaStream_t>(stream);
        if (o.autotune) apply_autotune(*graph, o, s);
        const bool sym = o.symmetry != 0;
        if (sym) { o.shard_bits = 1; o.shard_lo = 1; o.shard_hi = 2; }      // spin N-1 up only
        enumerate_range(*graph, s, g_out, g_out_on_device != 0, o, sym);
    });
}

extern "C" isg_status isg_enumerate_rank(const isg_graph* graph, void* stream, int64_t* g_out, int32_t g_out_on_device,
                                         int32_t rank, int32_t world_size, const isg_options* opt) {
    return guarded([&] {
        NvtxRange nvtx("isg_enumerate_rank");
        if (!graph || !g_out) fail(ISG_ERR_INVALID, "graph or g_out is NULL");
        isg_options o = resolve_options(opt);
        if (o.shard_bits || o.shard_lo || o.shard_hi) fail(ISG_ERR_INVALID, "the rank's shards come from rank and world_size");
        const bool sym = o.symmetry != 0;
        int32_t bits = 0;
        int64_t lo = 0, hi = 0;
        rank_shards(graph->n, rank, world_size, sym, bits, lo, hi);
        cudaStream_t s = static_cast<cudaStream_t>(stream);
        if (lo == hi) {                                // no configurations for this rank
            const size_t table_bytes = sizeof(int64_t) * (size_t)public_bins(*graph);
            if (o.accumulate) return;
            if (g_out_on_device) ISG_CUDA(cudaMemsetAsync(g_out, 0, table_bytes, s));
            else std::memset(g_out, 0, table_bytes);
            return;
        }
        if (o.autotune) apply_autotune(*graph, o, s);
        o.symmetry = 0;
        o.shard_bits = bits;
        o.shard_lo = lo;
        o.shard_hi = hi;
        enumerate_range(*graph, s, g_out, g_out_on_device != 0, o, sym);
    });
}

extern "C" isg_status isg_device_status(void* stream, int32_t clear) {
    return guarded([&] {
        cudaStream_t s = static_cast<cudaStream_t>(stream);
        unsigned int* w = device_status_word();
        unsigned int word = 0;
        ISG_CUDA(cudaMemcpyAsync(&word, w, sizeof word, cudaMemcpyDeviceToHost, s));
        if (clear) ISG_CUDA(cudaMemsetAsync(w, 0, sizeof word, s));
        ISG_CUDA(cudaStreamSynchronize(s));
        check_self_check_word(word, "device-output call");
    });
}
