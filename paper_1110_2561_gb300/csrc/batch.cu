// batch.cu -- many independent graphs in one persistent launch (isg_enumerate_batch and the
// prepared-batch calls isg_batch_*).
//
// The paper splits one lattice's outer loops over MPI ranks (Sec. 3d). For thousands of small
// systems (disorder realisations) one launch per system leaves the GPU mostly idle, so here the
// unit of work is a tile = one warp task (32 outer prefixes x 2^q inner configurations) of one
// instance, and all tiles of all instances form one queue. Warps of a persistent grid pop tiles
// from a global counter; a tile maps to its instance by binary search over the instances'
// cumulative tile offsets (instances are ordered largest first, so the long tiles start early
// and the short ones fill the tail). Each warp owns a shared-memory slot holding the current
// instance's program and a private 32-bit histogram, flushed into that instance's int64 table
// after every tile.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <memory>
#include <mutex>
#include <numeric>
#include <string>
#include <vector>

#include "batch_internal.h"
#include "isg_internal.h"
#include "split_internal.h"
#include "nvtx_range.h"

namespace isg {

DeviceInfo device_info();

struct BatchArgs {
    const BatchInst* inst;
    const uint64_t* blobs;
    unsigned long long* counter;
    unsigned int* status;
    uint64_t n_tiles;
    int32_t n_inst;
    int32_t slot_words;      // per-warp shared slot: program words (even) + histogram words / 2
    int32_t prog_words;      // words reserved for the program in a slot (even)
    int32_t pad;
};

struct WarpSmemSink {
    __device__ __forceinline__ void operator()(uint32_t& addr) const {
        asm volatile("red.shared.add.u32 [%0], 1;" : "+r"(addr) : : "memory");
    }
};

__device__ __forceinline__ int find_instance(const BatchInst* inst, int n, uint64_t t) {
    int lo = 0, hi = n - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (inst[mid].tile_begin <= t) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

template <int B>
__global__ void __launch_bounds__(512) batch_kernel(BatchArgs a) {
    extern __shared__ __align__(16) uint64_t smem[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    uint64_t* slot = smem + (size_t)warp * a.slot_words;
    uint32_t* hist = reinterpret_cast<uint32_t*>(slot + a.prog_words);
    const uint32_t base = static_cast<uint32_t>(__cvta_generic_to_shared(hist));
    const ProgHeader* hd = reinterpret_cast<const ProgHeader*>(slot);
    WarpSmemSink sink;
    int cur = -1;
    for (;;) {
        unsigned long long t = 0;
        if (lane == 0) t = atomicAdd(a.counter, 1ull);
        t = __shfl_sync(0xffffffffu, t, 0);
        if (t >= a.n_tiles) break;
        const int i = find_instance(a.inst, a.n_inst, t);
        const BatchInst in = a.inst[i];
        if (i != cur) {                       // stage this instance's program into the slot
            __syncwarp();
            const uint64_t* src = a.blobs + in.blob_off;
            for (uint32_t w = lane; w < in.blob_words; w += 32) slot[w] = src[w];
            cur = i;
        }
        __syncwarp();
        const int nb = hd->nbins_c;
        for (int b = lane; b < nb; b += 32) hist[b] = 0;
        __syncwarp();
        const ProgView v = make_view(slot);
        const uint64_t task = in.task_lo + (t - in.tile_begin);
        uint64_t last_state;
        uint32_t last_idx;
        lane_walk<B>(v, in.prefix_base + task * 32 + lane, base, sink, last_state, last_idx);
        if (last_idx != base + bin_offset(v, last_state)) atomicOr(a.status, 1u);
        __syncwarp();
        const int n_m = hd->n_m, R = hd->stride;
        for (int b = lane; b < nb; b += 32) {
            const uint32_t c = hist[b];
            const int64_t ec = b / R, m = b - ec * R;
            if (c && m < n_m) {                  // padding columns m > N are never counted
                const int64_t e = (hd->e_lo + hd->G * ec + hd->S) / 2;
                atomicAdd(reinterpret_cast<unsigned long long*>(in.g + e * n_m + m), (unsigned long long)c);
            }
        }
    }
}

// Instances too small for the warp-task kernel (fewer than B + 5 spins): one CTA per instance,
// one thread per configuration, counted into the int64 table with global atomics.
__global__ void batch_small_kernel(const BatchInst* inst, const int* small_ids, const uint64_t* blobs) {
    extern __shared__ __align__(16) uint64_t smem[];
    const BatchInst in = inst[small_ids[blockIdx.x]];
    for (uint32_t w = threadIdx.x; w < in.blob_words; w += blockDim.x) smem[w] = blobs[in.blob_off + w];
    __syncthreads();
    const ProgHeader* hd = reinterpret_cast<const ProgHeader*>(smem);
    const ProgView v = make_view(smem);
    const uint64_t total = 1ull << hd->n;
    for (uint64_t s = threadIdx.x; s < total; s += blockDim.x) {
        const int64_t b = bin_offset(v, s) >> 2;
        const int64_t ec = b / hd->stride, m = b - ec * hd->stride;
        const int64_t e = (hd->e_lo + hd->G * ec + hd->S) / 2;
        atomicAdd(reinterpret_cast<unsigned long long*>(in.g + e * hd->n_m + m), 1ull);
    }
}

// Symmetry completion in place, one CTA per instance: the table holds the configurations with
// spin N-1 up; bins M and -M both become half(E, M) + half(E, -M).
__global__ void batch_mirror_kernel(const BatchInst* inst, const int* ids, const uint64_t* blobs) {
    const BatchInst in = inst[ids[blockIdx.x]];
    const ProgHeader* hd = reinterpret_cast<const ProgHeader*>(blobs + in.blob_off);
    const int n_m = hd->n_m, n_e = (int)(hd->S + 1), half = (n_m + 1) / 2;
    for (int i = threadIdx.x; i < n_e * half; i += blockDim.x) {
        const int e = i / half, m = i - e * half, m2 = n_m - 1 - m;
        int64_t* row = in.g + (size_t)e * n_m;
        if (m == m2) row[m] *= 2;
        else {
            const int64_t v = row[m] + row[m2];
            row[m] = v;
            row[m2] = v;
        }
    }
}

// ---------------------------------------------------------------------------------------------
// Host planning of a batch
// ---------------------------------------------------------------------------------------------
// Tasks of the whole configuration space of graph g under a plan with q inner bits.
static BatchPlan plan_batch(int n, const isg_graph* const* graphs, const isg_options& o, const DeviceInfo& d) {
    BatchPlan bp;
    if (o.shard_bits || o.shard_lo || o.shard_hi || o.accumulate)
        fail(ISG_ERR_INVALID, "batches take no shard or accumulate options");
    if (o.lane_model == 4)
        fail(ISG_ERR_INVALID, "lane tables (lane_model 4) are for single-graph enumerations; a batch keeps one histogram per warp");
    const bool sym = o.symmetry != 0;
    // common low block: the largest size every large-enough instance supports
    std::vector<int> b_of(n, 0);
    for (int k = 0; k < n; ++k) {
        const isg_graph& g = *graphs[k];
        if (g.n > o.max_spins) fail(ISG_ERR_TOO_LARGE, "graph " + std::to_string(k) + " has more than max_spins spins");
        isg_options ok = o;
        ok.inner_bits = 0;
        const Plan p = make_plan(g, ok, d);
        b_of[k] = p.small ? 0 : p.b;
    }
    int B = o.low_bits > 0 ? o.low_bits : kMaxLow;
    for (int k = 0; k < n; ++k) if (b_of[k] > 0) B = std::min(B, b_of[k]);
    bp.B = B;
    const int q_target = o.inner_bits > 0 ? o.inner_bits : 16;
    std::vector<int> idx(n);
    std::iota(idx.begin(), idx.end(), 0);
    std::stable_sort(idx.begin(), idx.end(), [&](int a, int b) { return graphs[a]->n > graphs[b]->n; });
    int max_words = 0, max_bins = 0;
    for (int k : idx) {
        const isg_graph& g = *graphs[k];
        BatchInst in{};
        Plan p;
        const bool small = g.n < B + 5 + (sym ? 1 : 0) || b_of[k] == 0;
        isg_options ok = o;
        if (small) {
            ok.inner_bits = 0;
            ok.low_bits = 0;
            p = make_plan(g, ok, d);
            p.small = true;
            p.q = 0;
            p.b = 0;
            std::iota(p.perm.begin(), p.perm.end(), 0);
        } else {
            ok.low_bits = B;
            if (sym) { ok.shard_bits = 1; ok.shard_lo = 1; ok.shard_hi = 2; }     // spin N-1 up only
            ok.inner_bits = std::max(B, std::min(q_target, g.n - (sym ? 6 : 5)));
            p = make_plan(g, ok, d);
        }
        const std::vector<uint64_t> blob = build_program(g, p);
        in.blob_off = (uint32_t)bp.blobs.size();
        in.blob_words = (uint32_t)blob.size();
        bp.blobs.insert(bp.blobs.end(), blob.begin(), blob.end());
        if (bp.blobs.size() & 1) bp.blobs.push_back(0);
        if (small) {
            bp.small_ids.push_back((int)bp.inst.size());
            bp.small_max_words = std::max(bp.small_max_words, (int)blob.size());
            in.n_tiles = 0;
        } else {
            in.prefix_base = p.prefix_base;
            in.task_lo = 0;
            in.n_tiles = p.n_tasks;
            if (sym) bp.mirror_ids.push_back((int)bp.inst.size());
            max_words = std::max(max_words, (int)blob.size());
            max_bins = std::max(max_bins, (int)(g.n_e_c * p.stride));
        }
        bp.inst.push_back(in);
        bp.order.push_back(k);
    }
    // tiles: cumulative over the instances in order
    uint64_t t = 0;
    for (auto& in : bp.inst) { in.tile_begin = t; t += in.n_tiles; }
    bp.n_tiles = t;
    bp.prog_words = (max_words + 1) & ~1;
    bp.slot_words = (bp.prog_words + (max_bins + 1) / 2 + 1) & ~1;   // even: slots stay 16-byte aligned
    bp.threads = o.block_threads > 0 ? o.block_threads : 512;
    if (bp.threads % 32 || bp.threads > 512) fail(ISG_ERR_INVALID, "batch block_threads must be a multiple of 32, at most 512");
    bp.warps_per_cta = bp.threads / 32;
    bp.smem = (size_t)bp.slot_words * 8 * bp.warps_per_cta;
    while (bp.smem > d.smem_optin && bp.warps_per_cta > 1) {
        bp.warps_per_cta /= 2;
        bp.threads = bp.warps_per_cta * 32;
        bp.smem = (size_t)bp.slot_words * 8 * bp.warps_per_cta;
    }
    if (bp.smem > d.smem_optin) fail(ISG_ERR_TOO_LARGE, "a batch instance's histogram does not fit shared memory");
    return bp;
}

template <int B>
static void launch_batch_b(const BatchPlan& bp, const BatchArgs& a, cudaStream_t s, int ctas_per_sm) {
    if (!bp.n_tiles) return;
    const int occ = kernel_occupancy(reinterpret_cast<const void*>(batch_kernel<B>), bp.threads, bp.smem);
    if (occ < 1) fail(ISG_ERR_TOO_LARGE, "batch kernel does not fit an SM");
    const DeviceInfo d = device_info();
    const uint64_t warps_needed = bp.n_tiles;
    const uint64_t want = (uint64_t)d.sms * (uint64_t)std::min(occ, ctas_per_sm);
    const int grid = (int)std::max<uint64_t>(1, std::min<uint64_t>(want, (warps_needed + bp.warps_per_cta - 1) / bp.warps_per_cta));
    batch_kernel<B><<<grid, bp.threads, bp.smem, s>>>(a);
    ISG_CUDA(cudaGetLastError());
}

// Enqueue the batch kernels. d_inst / d_blobs / d_small / counter / status on the device.
void launch_batch(const BatchPlan& bp, const BatchInst* d_inst, const uint64_t* d_blobs, const int* d_small,
                  unsigned long long* counter, unsigned int* status, cudaStream_t s, int ctas_per_sm) {
    BatchArgs a;
    std::memset(&a, 0, sizeof a);
    a.inst = d_inst;
    a.blobs = d_blobs;
    a.counter = counter;
    a.status = status;
    a.n_tiles = bp.n_tiles;
    a.n_inst = (int)bp.inst.size();
    a.slot_words = bp.slot_words;
    a.prog_words = bp.prog_words;
    switch (bp.B) {
        case 1: launch_batch_b<1>(bp, a, s, ctas_per_sm); break;
        case 2: launch_batch_b<2>(bp, a, s, ctas_per_sm); break;
        case 3: launch_batch_b<3>(bp, a, s, ctas_per_sm); break;
        case 4: launch_batch_b<4>(bp, a, s, ctas_per_sm); break;
        case 5: launch_batch_b<5>(bp, a, s, ctas_per_sm); break;
        case 6: launch_batch_b<6>(bp, a, s, ctas_per_sm); break;
        case 7: launch_batch_b<7>(bp, a, s, ctas_per_sm); break;
        default: fail(ISG_ERR_INTERNAL, "bad low block size");
    }
    if (!bp.small_ids.empty()) {
        const int smem = bp.small_max_words * 8;
        kernel_occupancy(reinterpret_cast<const void*>(batch_small_kernel), 256, (size_t)smem);
        batch_small_kernel<<<(int)bp.small_ids.size(), 256, smem, s>>>(d_inst, d_small, d_blobs);
        ISG_CUDA(cudaGetLastError());
    }
    if (!bp.mirror_ids.empty()) {
        batch_mirror_kernel<<<(int)bp.mirror_ids.size(), 256, 0, s>>>(d_inst, d_small + bp.small_ids.size(), d_blobs);
        ISG_CUDA(cudaGetLastError());
    }
}

void launch_mirror(const BatchInst* d_inst, const int* d_ids, int n, const uint64_t* d_blobs, cudaStream_t s) {
    if (n <= 0) return;
    batch_mirror_kernel<<<n, 256, 0, s>>>(d_inst, d_ids, d_blobs);
    ISG_CUDA(cudaGetLastError());
}

}  // namespace isg

using namespace isg;

// Parallel branches for a batch's split launches (concurrent kernels: enough to keep the GPU busy
// across the launches' ramps and tails).
constexpr size_t kSplitBranches = 8;

// A prepared batch: device-resident programs, descriptors and output tables, and the CUDA graph
// of one run (zero the tables and the counter, launch the kernels), captured on first use.
struct isg_batch {
    BatchPlan plan;
    int device = 0;
    int ctas_per_sm = 2;
    char* mem = nullptr;                 // one device allocation holding everything
    BatchInst* d_inst = nullptr;
    uint64_t* d_blobs = nullptr;
    int* d_small = nullptr;
    unsigned long long* d_counter = nullptr;
    unsigned int* d_status = nullptr;
    int64_t* d_tables = nullptr;
    size_t table_words = 0;
    std::vector<size_t> table_off;       // by caller index
    std::vector<size_t> table_len;
    cudaStream_t capture_stream = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    std::mutex mu;
    // graphs served by split-and-convolve (options.split): one launch each, before the tile kernel
    struct SplitJob {
        std::shared_ptr<const SplitPrepared> prep;
        const uint64_t* d_blob;
        int64_t* d_table;
    };
    std::vector<SplitJob> splits;
    bool has_tiles = true;
    // The split launches write disjoint tables (and the status word, by atomic OR), so they run as
    // parallel branches: round-robin over these streams, forked from and joined back into the
    // enqueuing stream (parallel nodes of the captured graph), beside the tile kernel.
    std::vector<cudaStream_t> branch;
    std::vector<cudaEvent_t> branch_done;
    cudaEvent_t fork = nullptr;
};

static void batch_enqueue(isg_batch* b, cudaStream_t s) {
    ISG_CUDA(cudaMemsetAsync(b->d_tables, 0, b->table_words * 8, s));
    ISG_CUDA(cudaMemsetAsync(b->d_counter, 0, 16, s));
    const size_t nb = b->branch.size();
    if (nb) {
        ISG_CUDA(cudaEventRecord(b->fork, s));
        for (cudaStream_t t : b->branch) ISG_CUDA(cudaStreamWaitEvent(t, b->fork, 0));
    }
    for (size_t k = 0; k < b->splits.size(); ++k) {
        const auto& j = b->splits[k];
        launch_split(*j.prep, j.d_blob, reinterpret_cast<unsigned long long*>(j.d_table), b->d_status,
                     nb ? b->branch[k % nb] : s, (int)std::max<size_t>(1, std::min(nb, b->splits.size())));
    }
    if (b->has_tiles)
        launch_batch(b->plan, b->d_inst, b->d_blobs, b->d_small, b->d_counter, b->d_status, s, b->ctas_per_sm);
    for (size_t i = 0; i < nb; ++i) {
        ISG_CUDA(cudaEventRecord(b->branch_done[i], b->branch[i]));
        ISG_CUDA(cudaStreamWaitEvent(s, b->branch_done[i], 0));
    }
}

// Time a batch plan on a subset of the graphs: its own device buffers, one warm-up and two timed
// runs, best of two (ms). Used by the batch autotuner; the tables are thrown away.
static float time_batch(int n, const isg_graph* const* graphs, const isg_options& o, cudaStream_t s, int ctas_per_sm) {
    const DeviceInfo d = device_info();
    BatchPlan bp = plan_batch(n, graphs, o, d);
    size_t words = 0;
    std::vector<size_t> off(bp.order.size());
    for (size_t k = 0; k < bp.order.size(); ++k) { off[k] = words; words += (size_t)public_bins(*graphs[bp.order[k]]); }
    size_t at = 0;
    auto take = [&](size_t bytes) { size_t o2 = at; at = (at + bytes + 255) & ~(size_t)255; return o2; };
    const size_t o_cnt = take(16), o_inst = take(sizeof(BatchInst) * bp.inst.size());
    std::vector<int> ids(bp.small_ids);
    ids.insert(ids.end(), bp.mirror_ids.begin(), bp.mirror_ids.end());
    const size_t o_small = take(sizeof(int) * std::max<size_t>(1, ids.size()));
    const size_t o_blobs = take(8 * bp.blobs.size()), o_tab = take(8 * words);
    char* mem = nullptr;
    mem = static_cast<char*>(scratch_alloc(at, s));
    struct Free {
        char* p; cudaStream_t s;
        ~Free() { if (p) { cudaFreeAsync(p, s); cudaStreamSynchronize(s); } }
    } guard{mem, s};
    int64_t* tables = reinterpret_cast<int64_t*>(mem + o_tab);
    for (size_t k = 0; k < bp.order.size(); ++k) bp.inst[k].g = tables + off[k];
    ISG_CUDA(cudaMemcpyAsync(mem + o_inst, bp.inst.data(), sizeof(BatchInst) * bp.inst.size(), cudaMemcpyHostToDevice, s));
    if (!ids.empty())
        ISG_CUDA(cudaMemcpyAsync(mem + o_small, ids.data(), sizeof(int) * ids.size(), cudaMemcpyHostToDevice, s));
    ISG_CUDA(cudaMemcpyAsync(mem + o_blobs, bp.blobs.data(), 8 * bp.blobs.size(), cudaMemcpyHostToDevice, s));
    cudaEvent_t e0, e1;
    ISG_CUDA(cudaEventCreate(&e0));
    ISG_CUDA(cudaEventCreate(&e1));
    float best = 1e30f;
    for (int rep = 0; rep < 3; ++rep) {
        ISG_CUDA(cudaMemsetAsync(tables, 0, 8 * words, s));
        ISG_CUDA(cudaMemsetAsync(mem + o_cnt, 0, 16, s));
        ISG_CUDA(cudaEventRecord(e0, s));
        launch_batch(bp, reinterpret_cast<BatchInst*>(mem + o_inst), reinterpret_cast<uint64_t*>(mem + o_blobs),
                     reinterpret_cast<int*>(mem + o_small), reinterpret_cast<unsigned long long*>(mem + o_cnt),
                     reinterpret_cast<unsigned int*>(mem + o_cnt + 8), s, ctas_per_sm);
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

// Batch autotuner: per-lane walk length, block size, and either the index order's lane spins at a
// histogram stride residue or the bank-conflict model's lane spins at their own stride (chosen once
// per graph structure, coupling signs aside), timed on every 8th graph (the subset keeps the
// batch's mix of sizes). Unset fields of o are filled in.
static void autotune_batch(int n, const isg_graph* const* graphs, isg_options& o, int& ctas_per_sm) {
    std::vector<const isg_graph*> sub;
    for (int k = 0; k < n; k += 8) sub.push_back(graphs[k]);
    cudaStream_t s = nullptr;
    ISG_CUDA(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
    struct Destroy {
        cudaStream_t s;
        ~Destroy() { cudaStreamDestroy(s); }
    } dguard{s};
    static const int qs[] = {16, 18, 14};
    static const int threads[] = {512, 256};
    // (lane_model, stride residue): the index order at two residues, the model at its own stride
    static const int lanes_residues[][2] = {{2, 6}, {2, 13}, {1, 0}};
    float best_ms = 1e30f;
    isg_options best = o;
    for (int q : qs)
        for (int t : threads)
            for (const auto& lr : lanes_residues) {
                if (o.lane_model && o.lane_model != lr[0]) continue;
                isg_options c = o;
                c.autotune = 0;
                if (!c.inner_bits) c.inner_bits = q;
                if (!c.block_threads) c.block_threads = t;
                c.lane_model = lr[0];
                if (!c.stride_residue && !c.bin_stride) c.stride_residue = lr[1];
                float ms;
                try {
                    ms = time_batch((int)sub.size(), sub.data(), c, s, ctas_per_sm);
                } catch (const Error&) {
                    continue;
                }
                if (ms < best_ms) { best_ms = ms; best = c; }
            }
    o = best;
    o.autotune = 0;
}

extern "C" {

isg_status isg_batch_create(int32_t n_graphs, const isg_graph* const* graphs, const isg_options* opt, isg_batch** out) {
    return guarded([&] {
        if (!out) fail(ISG_ERR_INVALID, "out is NULL");
        *out = nullptr;
        if (n_graphs < 1 || !graphs) fail(ISG_ERR_INVALID, "need at least one graph");
        NvtxRange nvtx("isg_batch_create");
        for (int k = 0; k < n_graphs; ++k) if (!graphs[k]) fail(ISG_ERR_INVALID, "graph " + std::to_string(k) + " is NULL");
        isg_options o = resolve_options(opt);
        const DeviceInfo d = device_info();
        std::unique_ptr<isg_batch> b(new isg_batch());
        ISG_CUDA(cudaGetDevice(&b->device));
        b->ctas_per_sm = o.ctas_per_sm > 0 ? o.ctas_per_sm : 2;
        // options.split: graphs whose split-and-convolve plan models less work than their full
        // enumeration (a launch's fixed cost included) are served by split launches; the others
        // (caller indices tile_of) by the tile queue
        std::vector<std::shared_ptr<const SplitPrepared>> sprep(n_graphs);
        std::vector<int> tile_of;
        std::vector<const isg_graph*> tile_graphs;
        for (int k = 0; k < n_graphs; ++k) {
            if (o.split) {
                try {
                    auto sp = prepare_split(*graphs[k], 0, false, true);
                    if (sp->plan.cost + kSplitLaunchWarpInstr < sp->plan.direct_cost) { sprep[k] = sp; continue; }
                } catch (const Error&) {
                    // no admissible boundary set: the tile queue
                }
            }
            tile_of.push_back(k);
            tile_graphs.push_back(graphs[k]);
        }
        b->has_tiles = !tile_of.empty();
        if (b->has_tiles) {
            if (o.autotune) autotune_batch((int)tile_graphs.size(), tile_graphs.data(), o, b->ctas_per_sm);
            b->plan = plan_batch((int)tile_graphs.size(), tile_graphs.data(), o, d);
            for (auto& c : b->plan.order) c = tile_of[c];          // plan order -> caller index
        }
        BatchPlan& bp = b->plan;
        b->table_off.assign(n_graphs, 0);
        b->table_len.assign(n_graphs, 0);
        size_t words = 0;
        for (size_t k = 0; k < bp.order.size(); ++k) {
            const int c = bp.order[k];
            b->table_off[c] = words;
            b->table_len[c] = (size_t)public_bins(*graphs[c]);
            words += b->table_len[c];
        }
        size_t split_words = 0;
        for (int k = 0; k < n_graphs; ++k)
            if (sprep[k]) {
                b->table_off[k] = words;
                b->table_len[k] = (size_t)public_bins(*graphs[k]);
                words += b->table_len[k];
                split_words += (sprep[k]->blob.size() + 31) & ~(size_t)31;       // 256-byte aligned programs
            }
        b->table_words = words;
        // layout: [counter 8][status 8][inst][small ids][blobs][split programs][tables], 256-byte
        // aligned pieces
        size_t off = 0;
        auto take = [&](size_t bytes) { size_t o2 = off; off = (off + bytes + 255) & ~(size_t)255; return o2; };
        std::vector<int> ids(bp.small_ids);
        ids.insert(ids.end(), bp.mirror_ids.begin(), bp.mirror_ids.end());
        const size_t o_cnt = take(16), o_inst = take(sizeof(BatchInst) * std::max<size_t>(1, bp.inst.size()));
        const size_t o_small = take(sizeof(int) * std::max<size_t>(1, ids.size()));
        const size_t o_blobs = take(8 * std::max<size_t>(1, bp.blobs.size())), o_split = take(8 * std::max<size_t>(1, split_words));
        const size_t o_tab = take(8 * std::max<size_t>(1, words));
        ISG_CUDA(cudaMalloc(reinterpret_cast<void**>(&b->mem), off));
        b->d_counter = reinterpret_cast<unsigned long long*>(b->mem + o_cnt);
        b->d_status = reinterpret_cast<unsigned int*>(b->mem + o_cnt + 8);
        b->d_inst = reinterpret_cast<BatchInst*>(b->mem + o_inst);
        b->d_small = reinterpret_cast<int*>(b->mem + o_small);
        b->d_blobs = reinterpret_cast<uint64_t*>(b->mem + o_blobs);
        b->d_tables = reinterpret_cast<int64_t*>(b->mem + o_tab);
        for (size_t k = 0; k < bp.order.size(); ++k) bp.inst[k].g = b->d_tables + b->table_off[bp.order[k]];
        if (b->has_tiles) {
            ISG_CUDA(cudaMemcpy(b->d_inst, bp.inst.data(), sizeof(BatchInst) * bp.inst.size(), cudaMemcpyHostToDevice));
            if (!ids.empty())
                ISG_CUDA(cudaMemcpy(b->d_small, ids.data(), sizeof(int) * ids.size(), cudaMemcpyHostToDevice));
            ISG_CUDA(cudaMemcpy(b->d_blobs, bp.blobs.data(), 8 * bp.blobs.size(), cudaMemcpyHostToDevice));
        }
        if (split_words) {
            std::vector<uint64_t> host(split_words, 0);
            size_t w = 0;
            for (int k = 0; k < n_graphs; ++k)
                if (sprep[k]) {
                    std::memcpy(host.data() + w, sprep[k]->blob.data(), 8 * sprep[k]->blob.size());
                    b->splits.push_back({sprep[k], reinterpret_cast<const uint64_t*>(b->mem + o_split) + w,
                                         b->d_tables + b->table_off[k]});
                    w += (sprep[k]->blob.size() + 31) & ~(size_t)31;
                }
            ISG_CUDA(cudaMemcpy(b->mem + o_split, host.data(), 8 * split_words, cudaMemcpyHostToDevice));
            split_prepare_launches();          // kernel attributes set now, not during graph capture
        }
        ISG_CUDA(cudaStreamCreateWithFlags(&b->capture_stream, cudaStreamNonBlocking));
        if (b->splits.size() > 1) {
            const size_t nb = std::min<size_t>(kSplitBranches, b->splits.size());
            ISG_CUDA(cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming));
            for (size_t i = 0; i < nb; ++i) {
                cudaStream_t t = nullptr;
                cudaEvent_t e = nullptr;
                ISG_CUDA(cudaStreamCreateWithFlags(&t, cudaStreamNonBlocking));
                b->branch.push_back(t);
                ISG_CUDA(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
                b->branch_done.push_back(e);
            }
        }
        *out = b.release();
    });
}

isg_status isg_batch_run(isg_batch* b, void* stream) {
    return guarded([&] {
        if (!b) fail(ISG_ERR_INVALID, "batch is NULL");
        NvtxRange nvtx("isg_batch_run");
        std::lock_guard<std::mutex> lk(b->mu);
        int dev = 0;
        ISG_CUDA(cudaGetDevice(&dev));
        if (dev != b->device) fail(ISG_ERR_INVALID, "batch belongs to another device");
        if (!b->exec) {
            ISG_CUDA(cudaStreamBeginCapture(b->capture_stream, cudaStreamCaptureModeThreadLocal));
            try {
                batch_enqueue(b, b->capture_stream);
            } catch (...) {
                cudaGraph_t g = nullptr;
                cudaStreamEndCapture(b->capture_stream, &g);
                if (g) cudaGraphDestroy(g);
                throw;
            }
            ISG_CUDA(cudaStreamEndCapture(b->capture_stream, &b->graph));
            ISG_CUDA(cudaGraphInstantiate(&b->exec, b->graph, 0));
        }
        ISG_CUDA(cudaGraphLaunch(b->exec, static_cast<cudaStream_t>(stream)));
    });
}

isg_status isg_batch_table(const isg_batch* b, int32_t k, int64_t** device_table) {
    return guarded([&] {
        if (!b || !device_table) fail(ISG_ERR_INVALID, "NULL argument");
        if (k < 0 || k >= (int)b->table_off.size()) fail(ISG_ERR_INVALID, "graph index out of range");
        *device_table = b->d_tables + b->table_off[k];
    });
}

isg_status isg_batch_status(isg_batch* b, void* stream) {
    return guarded([&] {
        if (!b) fail(ISG_ERR_INVALID, "batch is NULL");
        unsigned int st = 0;
        ISG_CUDA(cudaMemcpyAsync(&st, b->d_status, 4, cudaMemcpyDeviceToHost, static_cast<cudaStream_t>(stream)));
        ISG_CUDA(cudaStreamSynchronize(static_cast<cudaStream_t>(stream)));
        if (st) fail(ISG_ERR_INTERNAL, "batch self-check failed (status " + std::to_string(st) + ")");
    });
}

void isg_batch_destroy(isg_batch* b) {
    if (!b) return;
    int prev = 0;
    cudaGetDevice(&prev);
    cudaSetDevice(b->device);
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    if (b->capture_stream) cudaStreamDestroy(b->capture_stream);
    for (cudaStream_t t : b->branch) cudaStreamDestroy(t);
    for (cudaEvent_t e : b->branch_done) cudaEventDestroy(e);
    if (b->fork) cudaEventDestroy(b->fork);
    if (b->mem) cudaFree(b->mem);
    cudaSetDevice(prev);
    delete b;
}

isg_status isg_enumerate_batch(int32_t n_graphs, const isg_graph* const* graphs, void* stream, int64_t* const* g_out,
                               int32_t on_device, const isg_options* opt) {
    isg_batch* b = nullptr;
    isg_status st = isg_batch_create(n_graphs, graphs, opt, &b);
    if (st != ISG_OK) return st;
    st = guarded([&] {
        if (!g_out) fail(ISG_ERR_INVALID, "g_out is NULL");
        cudaStream_t s = static_cast<cudaStream_t>(stream);
        batch_enqueue(b, s);
        for (int k = 0; k < n_graphs; ++k) {
            if (!g_out[k]) fail(ISG_ERR_INVALID, "g_out[" + std::to_string(k) + "] is NULL");
            ISG_CUDA(cudaMemcpyAsync(g_out[k], b->d_tables + b->table_off[k], 8 * b->table_len[k],
                                     on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, s));
        }
        unsigned int status = 0;
        ISG_CUDA(cudaMemcpyAsync(&status, b->d_status, 4, cudaMemcpyDeviceToHost, s));
        ISG_CUDA(cudaStreamSynchronize(s));
        if (status) fail(ISG_ERR_INTERNAL, "batch self-check failed (status " + std::to_string(status) + ")");
    });
    isg_batch_destroy(b);
    return st;
}

}  // extern "C"
