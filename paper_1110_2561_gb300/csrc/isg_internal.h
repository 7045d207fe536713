// isg_internal.h -- host-side model shared by the library's translation units.
#pragma once
#include <cstdint>
#include <memory>
#include <mutex>
#include <new>
#include <string>
#include <utility>
#include <vector>

#include "../../include/isg.h"
#include "../../include/isg_debug.h"
#include "enum_core.cuh"

namespace isg {
struct PlannedProgram;
}

struct isg_graph {
    int n = 0;
    std::vector<int64_t> K;                 // n*n summed couplings, symmetric, zero diagonal
    std::vector<int32_t> bi, bj;            // distinct bonds (i < j)
    std::vector<int64_t> bJ;
    int64_t S = 0;                          // sum |J|
    int64_t G = 2;                          // energy stride of reachable energies
    int64_t e_ref = 0;                      // energy of the all-down configuration
    int64_t e_lo = 0;                       // smallest reachable-class energy >= -S
    int64_t n_e_c = 1;                      // compact energy bins
    std::vector<int> degree;                // distinct neighbours per spin
    // Plans and programs of recent isg_enumerate calls, keyed by the resolved options and the
    // device shape (planned_program): planning costs microseconds that latency-bound calls of one
    // graph would otherwise pay on every call.
    mutable std::mutex plan_mu;
    mutable std::vector<std::pair<std::string, std::shared_ptr<const isg::PlannedProgram>>> plan_cache;
};

namespace isg {

// Thread-local error message.
void set_error(const std::string& msg);
void clear_error();

// Exception type used inside the library; converted to a status at the ABI.
struct Error {
    isg_status status;
    std::string msg;
};
[[noreturn]] void fail(isg_status s, const std::string& msg);

// Run the body of a C entry point: clears the thread's error message, and turns what the body
// throws into the status the ABI returns (the message recorded for isg_last_error). No exception
// leaves the library.
template <class F>
isg_status guarded(F&& f) {
    try {
        clear_error();
        f();
        return ISG_OK;
    } catch (const Error& e) {
        set_error(e.msg);
        return e.status;
    } catch (const std::bad_alloc&) {
        set_error("host allocation failed");
        return ISG_ERR_NOMEM;
    } catch (...) {
        set_error("unexpected exception");
        return ISG_ERR_INTERNAL;
    }
}

// A CUDA runtime call that throws ISG_ERR_NOMEM / ISG_ERR_CUDA with the call's text on failure
// (for the .cu files; expands to CUDA runtime names only where it is used).
#define ISG_CUDA(call)                                                                              \
    do {                                                                                            \
        cudaError_t e_ = (call);                                                                    \
        if (e_ != cudaSuccess)                                                                      \
            ::isg::fail(e_ == cudaErrorMemoryAllocation ? ISG_ERR_NOMEM : ISG_ERR_CUDA,             \
                        std::string(#call) + ": " + cudaGetErrorString(e_));                        \
    } while (0)

// Resolved options with defaults applied.
isg_options resolve_options(const isg_options* opt);

// Execution plan of one enumeration.
struct Plan {
    bool small = false;        // thread-per-configuration kernel over [s_lo, s_hi)
    uint64_t s_lo = 0, s_hi = 0;
    int q = 0, b = 0;          // inner bits, low-block size
    std::vector<int> perm;     // internal position -> caller spin
    uint64_t prefix_base = 0;  // first lane prefix (multiple of 32)
    uint64_t n_tasks = 0;      // warp tasks: 32 lane prefixes each
    int stride = 0;            // histogram row stride (bins)
    bool aggregate = false;    // warp-aggregated counting (__match_any_sync)
    int threads = 512, copies = 1, ctas_per_sm = 2, flush_rounds = 1;
    int grid = 0;
    size_t smem_bytes = 0;
    bool lane_model = false;   // lane spins and stride chosen by the bank-conflict model
    double lane_cost = 0;      // the model's expected wavefronts per reduction (0 when not used)
    double lane_cost_index_order = 0;
    // Histogram layout of one copy (copy_words words): bin (e', m) of sub-table t is the word
    // sub_off[t] + e' stride + m, and sub-table t holds only the columns m in
    // [sub_m_lo[t], sub_m_hi[t]] (the words outside them may belong to another sub-table). Lane l
    // counts into sub-table lane_sub[l], whose first word is lane_word[l] = sub_off[lane_sub[l]].
    // One sub-table (the default): offset 0, columns [0, N], copy_words = n_e_c stride.
    int n_sub = 1, copy_words = 0;
    bool packed = false;       // lane tables side by side in each row (else a block each)
    int32_t sub_off[kLaneTables] = {};
    int32_t sub_m_lo[kLaneTables] = {};
    int32_t sub_m_hi[kLaneTables] = {};
    int32_t lane_word[32] = {};
    int8_t lane_sub[32] = {};
};

// Lane tables (options.lane_model = 4). With the row stride R a multiple of 32 words, a lane's
// bank is its up count plus its sub-table's offset (mod 32). The 32 lane values are split into
// the kLaneTables chains of a symmetric chain decomposition of the 5-bit cube (each chain holds
// consecutive popcounts), and the offsets make the banks of all 32 lanes distinct. A chain of
// popcounts [lo, lo + len) reaches the columns m in [lo, lo + len + N - 6]. Two layouts:
//   separate  sub-table t is a block of its own (n_e_c R + 32 words), R = `stride`;
//   packed    the ten sub-tables share each row, side by side in an order that keeps the row
//             short (R >= the row's span), so a copy takes about n_e_c (10 (N - 5) + 32) words.
// lane_table_layout fills p.stride, copy_words, n_sub, sub_off, sub_m_lo, sub_m_hi, lane_word
// and lane_sub for n spins, rows energy rows and energy stride G: with fixed_stride > 0 the
// separate layout at that stride (INVALID unless it is a multiple of 32 with 8 R / G whole and
// at least N + 1), else the smaller of the two at the least admissible strides. Every word of
// every sub-table is checked to be its sub-table's alone and every lane's bank its own.
void lane_table_layout(Plan& p, int n, int64_t rows, int64_t G, int fixed_stride);

// The lane spins of a plan chosen by the bank-conflict model (lanes.cpp).
struct LaneChoice {
    bool valid = false;
    int spins[5] = {0, 0, 0, 0, 0};  // caller spins for lane bits 0..4 (internal positions q..q+4)
    int stride = 0;                  // histogram row stride the model picks with them
    double cost = 0;                 // expected shared-memory wavefronts per warp reduction
    double cost_index_order = 0;     // the same for the index order's lane spins (at its best stride)
};

// Choose five lane spins among `pool` (a mask of free spins) and a row stride in [N + 1,
// max_stride] with the fewest expected wavefronts per warp reduction; `baseline` (the index
// order's lane spins) is always a candidate. Cached per graph structure (bonds and coupling
// magnitudes, energy stride, histogram rows; not the coupling signs), pool and stride limit.
LaneChoice choose_lanes(const isg_graph& g, uint64_t pool, const int* baseline, int max_stride);

// The same search over strides [stride_lo, stride_hi] (only those with 8 R divisible by the
// energy stride if stride_times8_by_G) for histograms whose rows are `divisor` units of energy
// apart (the split kernel's component histograms: divisor 2). quick: only the dense greedy sets,
// fewer draws (a few milliseconds; for planning per request).
LaneChoice choose_lanes_in(const isg_graph& g, uint64_t pool, const int* baseline, int stride_lo, int stride_hi,
                           int64_t divisor, bool stride_times8_by_G, bool quick = false);

struct DeviceInfo {
    int sms = 152;
    size_t smem_optin = 232448;
    size_t smem_per_sm = 233472;
};

// Free spins from which autotuning considers lane spins chosen by the conflict model (smaller
// enumerations take less time than the model's search).
constexpr int kLaneModelMinFree = 30;
// Free spins from which plain single-graph calls (no autotune) take the quick lane search.
constexpr int kLaneQuickMinFree = 36;

// Plan an enumeration of graph g under options o on a device with properties d. single_graph:
// the plan serves one graph's call (isg_enumerate and its relatives), where options.lane_model
// = 0 with autotune set may use the lane model; batches and the server plan thousands of graphs
// and keep the index order unless options.lane_model is 1.
Plan make_plan(const isg_graph& g, const isg_options& o, const DeviceInfo& d, bool single_graph = false);

// Build the program blob (64-bit words) of graph g for a plan: spins in internal order.
std::vector<uint64_t> build_program(const isg_graph& g, const Plan& p);

// A plan and its program.
struct PlannedProgram {
    Plan plan;
    std::vector<uint64_t> blob;
};

// make_plan and build_program for (g, o, d), from the graph's cache of recent calls when the same
// options and device shape were planned before. Thread-safe.
std::shared_ptr<const PlannedProgram> planned_program(const isg_graph& g, const isg_options& o, const DeviceInfo& d);

// Map bin i = e' * stride + m of the internal histogram to the public table index (-1 for the
// padding columns m > N, which are never counted).
inline int64_t public_bin(const isg_graph& g, int64_t compact, int64_t stride) {
    const int64_t n_m = g.n + 1;
    const int64_t ec = compact / stride, m = compact % stride;
    if (m >= n_m) return -1;
    const int64_t E = g.e_lo + g.G * ec;
    return ((E + g.S) / 2) * n_m + m;
}

// Stream-ordered scratch from the library's own memory pool on the current device (free it with
// cudaFreeAsync). The pool keeps freed memory for reuse instead of returning it at every
// synchronisation, so a call's few kilobytes of scratch cost no remapping. `stream` is a
// cudaStream_t.
void* scratch_alloc(size_t bytes, void* stream);

// Pinned host memory for the host-buffer forms of the calls: results are copied into it
// asynchronously and from it into the caller's arrays after one synchronisation (a pageable
// destination makes every copy a synchronous staged transfer), and host inputs go the other way.
// Buffers come from a small process-wide pool and return to it. The caller synchronises `stream`
// and then calls synced(); a stage destroyed without that (an error on the way) synchronises the
// stream first, so no copy in flight can touch a buffer that is back in the pool.
class PinnedStage {
   public:
    PinnedStage(size_t bytes, void* stream);
    ~PinnedStage();
    PinnedStage(const PinnedStage&) = delete;
    PinnedStage& operator=(const PinnedStage&) = delete;
    char* data() const { return p_; }
    void synced() { synced_ = true; }

   private:
    char* p_ = nullptr;
    size_t cap_ = 0;
    void* stream_ = nullptr;
    bool synced_ = false;
};

// Row stride of the shared histogram for a graph (>= N + 1), padded against bank conflicts.
int choose_stride(const isg_graph& g, int requested, int residue);

// CTAs of `threads` threads and `smem` bytes of dynamic shared memory that fit one SM for a
// kernel (a __global__ function's address) on the current device. The first call per device and
// kernel raises the kernel's dynamic shared-memory limit to the device maximum less its static
// shared memory. Results are cached per (device, kernel, threads, smem): both driver queries cost
// microseconds that a small call would otherwise pay on every launch. Thread-safe.
int kernel_occupancy(const void* kernel, int threads, size_t smem);

inline int64_t public_bins(const isg_graph& g) { return (g.S + 1) * (int64_t)(g.n + 1); }

// Bits of a kernel self-check word: a walk's incrementally tracked bin differed from the bin
// recomputed from scratch (set by the kernels); a walk's address left the histogram (set only by
// the host emulation, which checks every address).
constexpr unsigned int kSelfCheckLostBin = 1u;
constexpr unsigned int kSelfCheckOutOfRange = 2u;

// Throw ISG_ERR_INTERNAL naming the failed checks of a nonzero self-check word (no-op for 0).
// One function for every caller, so the kernels' word, the host emulation's and the device-wide
// word of isg_device_status are reported alike.
void check_self_check_word(unsigned int word, const char* what);

// The current device's self-check word of device-output calls (a file-scope __device__ word,
// looked up once per device; no allocation). Kernels OR their failures into it; isg_device_status
// reads and clears it.
unsigned int* device_status_word();

// The shards of rank `rank` of `world` ranks (isg_rank_shards): shard_bits `bits` and the range
// [lo, hi), empty (lo == hi) when there are more ranks than shards. With `sym` the range lies in
// the upper half of the space (spin N-1 up). Throws ISG_ERR_INVALID for a bad rank or world.
void rank_shards(int n, int rank, int world, bool sym, int32_t& bits, int64_t& lo, int64_t& hi);

// Fill the unset planning fields of o from the autotuner's cache for this graph on the current
// device, if isg_autotune (or isg_enumerate with autotune) tuned it before; no timing, no
// allocation. Returns whether the cache held an entry.
bool apply_cached_autotune(const isg_graph& g, isg_options& o);

}  // namespace isg
