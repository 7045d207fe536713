// server.cu -- a continuously batching request server over the tile-queue kernel (isg_server_*).
//
// Requests (graphs) arrive at any time from any thread. A worker thread owns one CUDA stream and
// runs engine steps: each step is one launch of the batch kernel over tiles (warp tasks) drawn
// from every admitted request, shortest remaining work first, up to a device-time budget, so
// requests that arrive while others are on the GPU join the next step and their tiles run next
// to the others'. A request is admitted when a slot (max_inflight) and room in the device table
// arena are free; its int64 table stays on the device, accumulating over the steps that carry
// its tiles, and is copied out (to a pinned mirror, then to the result buffer) by the step that
// carries its last tile. Two steps can be in flight, so planning the next step overlaps the
// current one. Requests of at least 28 spins whose lane tables fit one CTA's shared memory are
// the exception: a step gives each of them (up to kMaxLaneLaunches) one launch of the
// single-graph enumeration kernel over a range of its tasks, whose warp reductions are
// conflict-free, where the batch kernel's per-warp histograms are bound by bank conflicts. The paper distributes the outer loops of one lattice over processes with uniform
// shares (Sec. 3d); this is the same decomposition applied to a stream of lattices.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "batch_internal.h"
#include "isg_internal.h"
#include "nvtx_range.h"
#include "split_internal.h"

namespace isg {

DeviceInfo device_info();
void launch_enumeration(const Plan& p, const uint64_t* d_blob, int blob_words, int64_t* table,
                        unsigned long long* counter, unsigned int* status, cudaStream_t s,
                        const uint64_t* host_blob);

constexpr int kSplitMinSpins = 24;     // below this the tile path takes microseconds anyway
// requests given the quick lane search (lane_model option): their enumeration takes tens of
// milliseconds, against a few milliseconds of search
constexpr int kServerLaneModelMinSpins = 36;
// requests served with lane tables by the enumeration kernel: from this size on a request has
// enough warp tasks (at least 2^13, with inner bits min(16, N - 18)) to fill the GPU
constexpr int kServerLaneTableMinSpins = 28;
// enumeration-kernel launches per step for requests with lane tables (task counters in the step's
// counter block: words 2 .. 2 + kMaxLaneLaunches, inside its 256 bytes)
constexpr int kMaxLaneLaunches = 16;
static_assert(8 * (2 + kMaxLaneLaunches) <= 256, "lane-launch counters must fit the step's 256-byte counter block");

using Clock = std::chrono::steady_clock;

static double seconds_between(Clock::time_point a, Clock::time_point b) {
    return std::chrono::duration<double>(b - a).count();
}

enum class ReqState { Queued, Active, Finishing, Done, Failed, Cancelled };

struct Request {
    int64_t ticket = 0;
    int n = 0;
    int b = 0;                       // low-block size of its program (0: small kernel)
    int q = 0;
    int bins = 0;                    // compact histogram bins (stride included)
    std::vector<uint64_t> blob;      // tile program, or the split program when `split` is set
    std::shared_ptr<const SplitPrepared> split;   // served by split-and-convolve (one launch)
    std::shared_ptr<const Plan> lane;   // lane-table plan: served by the enumeration kernel, task ranges per step
    size_t table_words = 0;          // public table
    uint64_t total_tasks = 0, next_task = 0;
    uint64_t prefix_base = 0;        // lane prefix of task 0 (the upper half of the space with symmetry)
    bool sym = false;                // only spin N-1 up enumerated; the step with its last tile mirrors
    double configs = 0;
    size_t slot_off = 0, slot_bytes = 0;   // arena slot: [table][program]
    int64_t last_step = -1;          // last step that carries one of its tiles
    bool step_failed = false;        // a step carrying its tiles reported a failed self-check
    ReqState state = ReqState::Queued;
    isg_status status = ISG_OK;
    std::string message;
    Clock::time_point t_submit, t_admit, t_done;
    std::vector<int64_t> result;
};

struct Step {
    int64_t id = 0;
    int buf = 0;                     // descriptor buffer in use
    cudaEvent_t start = nullptr, done = nullptr;
    std::vector<int64_t> finishing;  // tickets whose last tile is in this step
    std::vector<int64_t> carried;    // tickets with tiles in this step
    double configs = 0;
};

// First-fit allocator over [0, size) with 256-byte granules.
class Arena {
   public:
    explicit Arena(size_t size) { free_[0] = size; }
    bool alloc(size_t bytes, size_t* off) {
        bytes = (bytes + 255) & ~(size_t)255;
        for (auto it = free_.begin(); it != free_.end(); ++it)
            if (it->second >= bytes) {
                *off = it->first;
                const size_t rest = it->second - bytes, o = it->first + bytes;
                free_.erase(it);
                if (rest) free_[o] = rest;
                return true;
            }
        return false;
    }
    void release(size_t off, size_t bytes) {
        bytes = (bytes + 255) & ~(size_t)255;
        auto it = free_.emplace(off, bytes).first;
        auto nx = std::next(it);
        if (nx != free_.end() && it->first + it->second == nx->first) { it->second += nx->second; free_.erase(nx); }
        if (it != free_.begin()) {
            auto pv = std::prev(it);
            if (pv->first + pv->second == it->first) { pv->second += it->second; free_.erase(it); }
        }
    }

   private:
    std::map<size_t, size_t> free_;
};

}  // namespace isg

using namespace isg;

struct isg_server {
    isg_server_options opt{};
    int device = 0;
    DeviceInfo dinfo;
    cudaStream_t stream = nullptr;
    char* arena_dev = nullptr;       // tables and programs
    char* arena_host = nullptr;      // pinned mirror of the tables for the copy-out
    std::unique_ptr<Arena> arena;
    // per descriptor buffer (two steps in flight): device and pinned host descriptors, small ids,
    // counter and status words
    BatchInst* desc_dev[2] = {nullptr, nullptr};
    BatchInst* desc_host[2] = {nullptr, nullptr};
    int* small_dev[2] = {nullptr, nullptr};
    int* small_host[2] = {nullptr, nullptr};
    unsigned long long* ctr_dev[2] = {nullptr, nullptr};
    unsigned int* status_host[2] = {nullptr, nullptr};
    cudaEvent_t ev_start[2] = {nullptr, nullptr}, ev_done[2] = {nullptr, nullptr};
    bool buf_busy[2] = {false, false};

    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<int64_t> queue;                         // waiting for admission (FIFO)
    std::unordered_map<int64_t, std::unique_ptr<Request>> reqs;
    std::vector<int64_t> active;                       // admitted, tiles left to issue
    std::deque<Step> inflight;
    int64_t next_ticket = 1, next_step = 0;
    size_t n_admitted = 0;                             // active + finishing
    int inject = 0;                                    // host-side failure injection (isg_debug_server_inject)
    bool stop = false;
    std::thread worker;
    // statistics
    double rate_est = 5e12;                            // configurations per second, running estimate
    int64_t steps_done = 0;
    double configs_done = 0, device_ms = 0;
    int64_t lane_requests = 0, lane_launches = 0;      // isg_debug_server_lane_counts
    Clock::time_point t_create;
};

namespace isg {

static void server_fail_cuda(cudaError_t e, const char* what) {
    if (e != cudaSuccess) fail(ISG_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

// Admit queued requests in arrival order while slots and arena space allow (caller holds mu).
static void admit_locked(isg_server* s) {
    while (!s->queue.empty() && (int)s->n_admitted < s->opt.max_inflight) {
        Request& r = *s->reqs[s->queue.front()];
        const size_t tbytes = ((r.table_words * 8) + 255) & ~(size_t)255;
        const size_t bytes = tbytes + r.blob.size() * 8;
        size_t off = 0;
        if (!s->arena->alloc(bytes, &off)) break;      // wait for memory to free up
        s->queue.pop_front();
        r.slot_off = off;
        r.slot_bytes = bytes;
        r.t_admit = Clock::now();
        r.state = ReqState::Active;
        s->active.push_back(r.ticket);                 // admitted first: a failing call below fails it too
        ++s->n_admitted;
        // zero the table and upload the program (ordered before any step that uses them)
        server_fail_cuda(cudaMemsetAsync(s->arena_dev + off, 0, r.table_words * 8, s->stream), "cudaMemsetAsync(table)");
        server_fail_cuda(cudaMemcpyAsync(s->arena_dev + off + tbytes, r.blob.data(), r.blob.size() * 8,
                                         cudaMemcpyHostToDevice, s->stream), "cudaMemcpyAsync(program)");
    }
}

// True while a step in flight carries one of the request's tiles (its slot is still written).
static bool carried_inflight(const isg_server* s, int64_t ticket) {
    for (const Step& st : s->inflight)
        if (std::find(st.carried.begin(), st.carried.end(), ticket) != st.carried.end()) return true;
    return false;
}

static void release_locked(isg_server* s, Request& r) {
    if (r.slot_bytes) {
        s->arena->release(r.slot_off, r.slot_bytes);
        r.slot_bytes = 0;
        --s->n_admitted;
    }
}

// Build and enqueue one engine step (caller holds mu; CUDA calls are asynchronous).
static bool issue_step_locked(isg_server* s) {
    NvtxRange nvtx("isg_server_step");
    int buf = -1;
    for (int k = 0; k < 2; ++k) if (!s->buf_busy[k]) { buf = k; break; }
    if (buf < 0 || s->active.empty()) return false;
    // shortest remaining work first
    std::vector<Request*> order;
    for (int64_t t : s->active) {
        Request* r = s->reqs[t].get();
        if (r->state == ReqState::Active) order.push_back(r);
    }
    if (order.empty()) return false;
    std::stable_sort(order.begin(), order.end(), [](const Request* a, const Request* b) {
        const double ra = a->b ? (double)(a->total_tasks - a->next_task) * (32.0 * (double)(1ull << a->q)) : a->configs;
        const double rb = b->b ? (double)(b->total_tasks - b->next_task) * (32.0 * (double)(1ull << b->q)) : b->configs;
        return ra < rb;
    });
    const double budget = std::max(1.0, s->opt.step_ms * 1e-3 * s->rate_est);
    BatchPlan bp;
    bp.B = kMaxLow;
    Step st;
    st.id = s->next_step++;
    st.buf = buf;
    std::vector<int64_t> finishing;
    int max_words = 0, max_bins = 0;
    uint64_t tiles = 0;
    double used = 0;
    std::vector<BatchInst> large, small, lane_mirror;
    std::vector<Request*> large_r, small_r, split_r, lane_r;
    std::vector<uint64_t> lane_lo, lane_n;             // task range of each lane-table launch
    std::vector<int> mirror;                           // descriptors of halved requests finishing here
    // a lane-table launch takes at least one full wave of warps (or the request's rest)
    const uint64_t lane_min_tasks = (uint64_t)std::max(1, s->dinfo.sms) * 32;
    for (Request* r : order) {
        if (used >= budget && (!large.empty() || !split_r.empty() || !lane_r.empty())) break;
        BatchInst in{};
        in.g = reinterpret_cast<int64_t*>(s->arena_dev + r->slot_off);
        const size_t tbytes = ((r->table_words * 8) + 255) & ~(size_t)255;
        in.blob_off = (uint32_t)((r->slot_off + tbytes) / 8);
        in.blob_words = (uint32_t)r->blob.size();
        if (r->split) {                                // whole request in one split launch
            split_r.push_back(r);
            used += r->configs;
            r->next_task = r->total_tasks;
        } else if (r->lane) {                          // a task range in one enumeration launch
            if ((int)lane_r.size() >= kMaxLaneLaunches) continue;
            const double per_tile = 32.0 * (double)(1ull << r->q);
            uint64_t take = (uint64_t)std::max(1.0, (budget - used) / per_tile);
            take = std::min<uint64_t>(std::max(take, lane_min_tasks), r->total_tasks - r->next_task);
            lane_r.push_back(r);
            lane_lo.push_back(r->next_task);
            lane_n.push_back(take);
            r->next_task += take;
            if (r->sym && r->next_task == r->total_tasks) lane_mirror.push_back(in);
            used += per_tile * (double)take;
        } else if (!r->b) {                            // whole request in the small kernel
            small.push_back(in);
            small_r.push_back(r);
            used += r->configs;
            r->next_task = r->total_tasks;
        } else {
            const double per_tile = 32.0 * (double)(1ull << r->q);
            uint64_t take = (uint64_t)std::max(1.0, (budget - used) / per_tile);
            take = std::min<uint64_t>(take, r->total_tasks - r->next_task);
            in.prefix_base = r->prefix_base;
            in.task_lo = r->next_task;
            in.n_tiles = take;
            r->next_task += take;
            if (r->sym && r->next_task == r->total_tasks) mirror.push_back((int)large.size());
            used += per_tile * (double)take;
            large.push_back(in);
            large_r.push_back(r);
            bp.B = std::min(bp.B, r->b);
            max_words = std::max(max_words, (int)r->blob.size());
            max_bins = std::max(max_bins, r->bins);
        }
    }
    // descriptors: large instances first (tile order), then the small ones
    for (auto& in : large) { in.tile_begin = tiles; tiles += in.n_tiles; }
    std::vector<BatchInst> desc = large;
    for (size_t k = 0; k < small.size(); ++k) {
        small[k].tile_begin = tiles;
        small[k].n_tiles = 0;
        bp.small_ids.push_back((int)(desc.size()));
        desc.push_back(small[k]);
        bp.small_max_words = std::max(bp.small_max_words, (int)small[k].blob_words);
    }
    bp.inst = desc;
    bp.n_tiles = tiles;
    // descriptors of the halved lane-table requests finishing here, for their mirror (not the batch's)
    const size_t lane_mirror_first = desc.size();
    desc.insert(desc.end(), lane_mirror.begin(), lane_mirror.end());
    bp.mirror_ids = mirror;                            // large descriptors come first: same indices
    bp.prog_words = (max_words + 1) & ~1;
    bp.slot_words = (bp.prog_words + (max_bins + 1) / 2 + 1) & ~1;   // even: slots stay 16-byte aligned
    bp.threads = s->opt.block_threads > 0 ? std::min(512, s->opt.block_threads) : 512;
    bp.warps_per_cta = bp.threads / 32;
    bp.smem = (size_t)bp.slot_words * 8 * bp.warps_per_cta;
    const DeviceInfo& d = s->dinfo;
    while (bp.smem > d.smem_optin && bp.warps_per_cta > 1) {
        bp.warps_per_cta /= 2;
        bp.threads = bp.warps_per_cta * 32;
        bp.smem = (size_t)bp.slot_words * 8 * bp.warps_per_cta;
    }
    std::memcpy(s->desc_host[buf], desc.data(), sizeof(BatchInst) * desc.size());
    // the kernels read the small kernel's ids, then the mirror's (at most one id per request)
    std::vector<int> ids(bp.small_ids);
    ids.insert(ids.end(), bp.mirror_ids.begin(), bp.mirror_ids.end());
    for (size_t k = 0; k < lane_mirror.size(); ++k) ids.push_back((int)(lane_mirror_first + k));
    if (!ids.empty()) std::memcpy(s->small_host[buf], ids.data(), sizeof(int) * ids.size());
    if (s->inject == 1) {
        s->inject = 0;
        fail(ISG_ERR_CUDA, "injected host-side failure before the step's first enqueue");
    }
    // From the first enqueue on, a failing call must not leave untracked work writing into the
    // arena: the stream is drained before the error propagates, so the slots of the requests it
    // fails can be released at once.
    struct DrainOnThrow {
        cudaStream_t st;
        bool armed = true;
        ~DrainOnThrow() { if (armed) cudaStreamSynchronize(st); }
    } drain{s->stream};
    server_fail_cuda(cudaEventRecord(s->ev_start[buf], s->stream), "cudaEventRecord");
    server_fail_cuda(cudaMemcpyAsync(s->desc_dev[buf], s->desc_host[buf], sizeof(BatchInst) * desc.size(),
                                     cudaMemcpyHostToDevice, s->stream), "cudaMemcpyAsync(descriptors)");
    if (!ids.empty())
        server_fail_cuda(cudaMemcpyAsync(s->small_dev[buf], s->small_host[buf], sizeof(int) * ids.size(),
                                         cudaMemcpyHostToDevice, s->stream), "cudaMemcpyAsync(small ids)");
    server_fail_cuda(cudaMemsetAsync(s->ctr_dev[buf], 0, 8 * (2 + kMaxLaneLaunches), s->stream), "cudaMemsetAsync(counters)");
    unsigned int* status = reinterpret_cast<unsigned int*>(s->ctr_dev[buf] + 1);
    for (Request* r : split_r) {                       // split requests first: each one launch, table in its slot
        const size_t tbytes = ((r->table_words * 8) + 255) & ~(size_t)255;
        launch_split(*r->split, reinterpret_cast<const uint64_t*>(s->arena_dev + r->slot_off + tbytes),
                     reinterpret_cast<unsigned long long*>(s->arena_dev + r->slot_off), status, s->stream);
    }
    if (!large.empty() || !small.empty())
        launch_batch(bp, s->desc_dev[buf], reinterpret_cast<const uint64_t*>(s->arena_dev), s->small_dev[buf], s->ctr_dev[buf],
                     status, s->stream, s->opt.ctas_per_sm > 0 ? s->opt.ctas_per_sm : 2);
    s->lane_launches += (int64_t)lane_r.size();
    for (size_t k = 0; k < lane_r.size(); ++k) {       // lane-table requests: their task ranges
        Request* r = lane_r[k];
        Plan lp = *r->lane;
        lp.prefix_base = r->prefix_base + lane_lo[k] * 32;
        lp.n_tasks = lane_n[k];
        const size_t tbytes = ((r->table_words * 8) + 255) & ~(size_t)255;
        launch_enumeration(lp, reinterpret_cast<const uint64_t*>(s->arena_dev + r->slot_off + tbytes), (int)r->blob.size(),
                           reinterpret_cast<int64_t*>(s->arena_dev + r->slot_off), s->ctr_dev[buf] + 2 + k, status,
                           s->stream, nullptr);
    }
    if (!lane_mirror.empty())
        launch_mirror(s->desc_dev[buf], s->small_dev[buf] + bp.small_ids.size() + bp.mirror_ids.size(),
                      (int)lane_mirror.size(), reinterpret_cast<const uint64_t*>(s->arena_dev), s->stream);
    if (s->inject == 2) {
        s->inject = 0;
        fail(ISG_ERR_CUDA, "injected host-side failure after the step's launch");
    }
    server_fail_cuda(cudaMemcpyAsync(s->status_host[buf], s->ctr_dev[buf] + 1, 4, cudaMemcpyDeviceToHost, s->stream),
                     "cudaMemcpyAsync(status)");
    // copy out the tables of requests whose last tile is in this step
    auto carried = [&](Request* r) {
        st.carried.push_back(r->ticket);
        r->last_step = st.id;
        if (r->next_task == r->total_tasks) {
            r->state = ReqState::Finishing;
            st.finishing.push_back(r->ticket);
            server_fail_cuda(cudaMemcpyAsync(s->arena_host + r->slot_off, s->arena_dev + r->slot_off, r->table_words * 8,
                                             cudaMemcpyDeviceToHost, s->stream), "cudaMemcpyAsync(table out)");
        }
    };
    for (Request* r : large_r) carried(r);
    for (Request* r : lane_r) carried(r);
    for (Request* r : small_r) carried(r);
    for (Request* r : split_r) carried(r);
    server_fail_cuda(cudaEventRecord(s->ev_done[buf], s->stream), "cudaEventRecord");
    drain.armed = false;
    st.configs = used;
    s->buf_busy[buf] = true;
    s->active.erase(std::remove_if(s->active.begin(), s->active.end(),
                                   [&](int64_t t) { return s->reqs[t]->state != ReqState::Active; }),
                    s->active.end());
    s->inflight.push_back(std::move(st));
    return true;
}

// The oldest in-flight step has completed: hand out results, free slots (caller holds mu).
static void complete_step_locked(isg_server* s, float ms) {
    Step st = std::move(s->inflight.front());
    s->inflight.pop_front();
    const unsigned int status = *s->status_host[st.buf];
    s->buf_busy[st.buf] = false;
    ++s->steps_done;
    s->device_ms += ms;
    s->configs_done += st.configs;
    if (ms > 0.05 && st.configs > 1e9) s->rate_est = 0.7 * s->rate_est + 0.3 * (st.configs / (ms * 1e-3));
    const Clock::time_point now = Clock::now();
    // a failed self-check taints every request with tiles in the step, finishing here or not
    if (status)
        for (int64_t t : st.carried) {
            auto it = s->reqs.find(t);
            if (it != s->reqs.end()) it->second->step_failed = true;
        }
    for (int64_t t : st.finishing) {
        auto it = s->reqs.find(t);
        if (it == s->reqs.end()) continue;
        Request& r = *it->second;
        if (r.state == ReqState::Cancelled) { release_locked(s, r); s->reqs.erase(it); continue; }
        if (r.state == ReqState::Failed) continue;     // failed on the host meanwhile: released below
        if (r.step_failed) {
            r.state = ReqState::Failed;
            r.status = ISG_ERR_INTERNAL;
            r.message = "enumeration self-check failed in a step carrying this request";
        } else {
            r.result.assign(reinterpret_cast<int64_t*>(s->arena_host + r.slot_off),
                            reinterpret_cast<int64_t*>(s->arena_host + r.slot_off) + r.table_words);
            r.state = ReqState::Done;
        }
        r.t_done = now;
        release_locked(s, r);
    }
    // cancelled requests whose last carrying step is now done, and requests failed on the host
    // while this step still wrote into their slots
    for (int64_t t : st.carried) {
        auto it = s->reqs.find(t);
        if (it == s->reqs.end()) continue;
        Request& r = *it->second;
        if (r.state == ReqState::Cancelled && r.last_step <= st.id) {
            release_locked(s, r);
            s->reqs.erase(it);
        } else if (r.state == ReqState::Failed && !carried_inflight(s, t)) {
            release_locked(s, r);
        }
    }
}

// Fail every admitted request that still has tiles to issue, after a host-side error while
// admitting or issuing (caller holds mu). A slot no in-flight step writes into is released now;
// the others when the last step carrying them completes.
static void fail_active_locked(isg_server* s, isg_status status, const std::string& msg) {
    const Clock::time_point now = Clock::now();
    for (int64_t t : s->active) {
        Request& r = *s->reqs[t];
        if (r.state == ReqState::Cancelled) {
            if (!carried_inflight(s, t)) { release_locked(s, r); s->reqs.erase(t); }
            continue;
        }
        r.state = ReqState::Failed;
        r.status = status;
        r.message = msg;
        r.t_done = now;
        if (!carried_inflight(s, t)) release_locked(s, r);
    }
    s->active.clear();
}

static void worker_main(isg_server* s) {
    cudaSetDevice(s->device);
    std::unique_lock<std::mutex> lk(s->mu);
    while (true) {
        if (s->stop && s->inflight.empty()) break;
        std::string err;
        try {
            if (!s->stop) admit_locked(s);
            if (!s->stop && s->inflight.size() < 2 && issue_step_locked(s)) continue;
        } catch (const Error& e) {
            err = e.msg;
        }
        if (!err.empty()) {                            // fail everything admitted; keep serving
            fail_active_locked(s, ISG_ERR_CUDA, err);
            s->cv_done.notify_all();
        }
        if (!s->inflight.empty()) {
            const int buf = s->inflight.front().buf;
            lk.unlock();
            const cudaError_t e = cudaEventSynchronize(s->ev_done[buf]);
            float ms = 0;
            if (e == cudaSuccess) cudaEventElapsedTime(&ms, s->ev_start[buf], s->ev_done[buf]);
            lk.lock();
            if (e != cudaSuccess) {
                Step st = std::move(s->inflight.front());
                s->inflight.pop_front();
                s->buf_busy[buf] = false;
                for (int64_t t : st.carried) {
                    auto it = s->reqs.find(t);
                    if (it == s->reqs.end()) continue;
                    Request& r = *it->second;
                    if (r.state == ReqState::Cancelled) {
                        if (!carried_inflight(s, t)) { release_locked(s, r); s->reqs.erase(it); }
                        continue;
                    }
                    r.state = ReqState::Failed;
                    r.status = ISG_ERR_CUDA;
                    r.message = std::string("step failed: ") + cudaGetErrorString(e);
                    r.t_done = Clock::now();
                    if (!carried_inflight(s, t)) release_locked(s, r);
                }
                s->active.erase(std::remove_if(s->active.begin(), s->active.end(),
                                               [&](int64_t t) { return s->reqs[t]->state == ReqState::Failed; }),
                                s->active.end());
            } else {
                complete_step_locked(s, ms);
            }
            s->cv_done.notify_all();
            continue;
        }
        if (s->stop) break;
        s->cv_work.wait_for(lk, std::chrono::milliseconds(50));
    }
}

}  // namespace isg

static void destroy_server(isg_server* s) {
    if (!s) return;
    if (s->worker.joinable()) {
        {
            std::lock_guard<std::mutex> lk(s->mu);
            s->stop = true;
        }
        s->cv_work.notify_all();
        s->worker.join();
    }
    int prev = 0;
    cudaGetDevice(&prev);
    cudaSetDevice(s->device);
    if (s->stream) cudaStreamSynchronize(s->stream);
    for (int k = 0; k < 2; ++k) {
        if (s->ev_start[k]) cudaEventDestroy(s->ev_start[k]);
        if (s->ev_done[k]) cudaEventDestroy(s->ev_done[k]);
        if (s->desc_dev[k]) cudaFree(s->desc_dev[k]);
        if (s->desc_host[k]) cudaFreeHost(s->desc_host[k]);
    }
    if (s->arena_dev) cudaFree(s->arena_dev);
    if (s->arena_host) cudaFreeHost(s->arena_host);
    if (s->stream) cudaStreamDestroy(s->stream);
    cudaSetDevice(prev);
    delete s;
}

extern "C" {

void isg_server_options_init(isg_server_options* o) {
    if (!o) return;
    std::memset(o, 0, sizeof *o);
    o->struct_size = (int32_t)sizeof(isg_server_options);
    o->max_spins = 40;
    o->max_inflight = 256;
    o->max_queued = 1 << 16;
    o->arena_bytes = (int64_t)64 << 20;
    o->step_ms = 20.0;
    o->split_work_ratio = 0.0;
    o->symmetry = 0;
    o->lane_model = 1;
}

isg_status isg_server_create(const isg_server_options* opt, isg_server** out) {
    return guarded([&] {
        if (!out) fail(ISG_ERR_INVALID, "out is NULL");
        *out = nullptr;
        isg_server_options o;
        isg_server_options_init(&o);
        if (opt) {
            if (opt->struct_size != (int32_t)sizeof(isg_server_options))
                fail(ISG_ERR_INVALID, "isg_server_options.struct_size mismatch (initialise with isg_server_options_init)");
            o = *opt;
        }
        if (o.max_spins < 1 || o.max_spins > 62) fail(ISG_ERR_INVALID, "max_spins must lie in [1, 62]");
        if (o.max_inflight < 1 || o.max_inflight > 65536) fail(ISG_ERR_INVALID, "max_inflight must lie in [1, 65536]");
        if (o.max_queued < 1) fail(ISG_ERR_INVALID, "max_queued must be >= 1");
        if (o.arena_bytes < (1 << 20)) fail(ISG_ERR_INVALID, "arena_bytes must be at least 1 MiB");
        if (!(o.step_ms > 0)) fail(ISG_ERR_INVALID, "step_ms must be > 0");
        if (!(o.split_work_ratio >= 0 && o.split_work_ratio <= 1)) fail(ISG_ERR_INVALID, "split_work_ratio must lie in [0, 1]");
        if (o.symmetry != 0 && o.symmetry != 1) fail(ISG_ERR_INVALID, "symmetry must be 0 or 1");
        if (o.lane_model != 0 && o.lane_model != 1) fail(ISG_ERR_INVALID, "lane_model must be 0 or 1");
        isg_server* s = new isg_server();
        s->opt = o;
        s->t_create = Clock::now();
        try {
            server_fail_cuda(cudaGetDevice(&s->device), "cudaGetDevice");
            s->dinfo = device_info();
            server_fail_cuda(cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking), "cudaStreamCreate");
            const size_t ab = (size_t)o.arena_bytes;
            cudaError_t e = cudaMalloc(reinterpret_cast<void**>(&s->arena_dev), ab);
            if (e != cudaSuccess) fail(ISG_ERR_NOMEM, std::string("cudaMalloc(arena): ") + cudaGetErrorString(e));
            e = cudaMallocHost(reinterpret_cast<void**>(&s->arena_host), ab);
            if (e != cudaSuccess) fail(ISG_ERR_NOMEM, std::string("cudaMallocHost(arena mirror): ") + cudaGetErrorString(e));
            s->arena.reset(new Arena(ab));
            const size_t n = (size_t)o.max_inflight;
            const size_t desc_bytes = (sizeof(BatchInst) * n + 255) & ~(size_t)255;
            const size_t small_bytes = (sizeof(int) * n + 255) & ~(size_t)255;
            for (int k = 0; k < 2; ++k) {
                char* d = nullptr;
                char* h = nullptr;
                e = cudaMalloc(reinterpret_cast<void**>(&d), desc_bytes + small_bytes + 256);
                if (e != cudaSuccess) fail(ISG_ERR_NOMEM, std::string("cudaMalloc(descriptors): ") + cudaGetErrorString(e));
                s->desc_dev[k] = reinterpret_cast<BatchInst*>(d);
                s->small_dev[k] = reinterpret_cast<int*>(d + desc_bytes);
                s->ctr_dev[k] = reinterpret_cast<unsigned long long*>(d + desc_bytes + small_bytes);
                e = cudaMallocHost(reinterpret_cast<void**>(&h), desc_bytes + small_bytes + 256);
                if (e != cudaSuccess) fail(ISG_ERR_NOMEM, std::string("cudaMallocHost(descriptors): ") + cudaGetErrorString(e));
                s->desc_host[k] = reinterpret_cast<BatchInst*>(h);
                s->small_host[k] = reinterpret_cast<int*>(h + desc_bytes);
                s->status_host[k] = reinterpret_cast<unsigned int*>(h + desc_bytes + small_bytes);
                server_fail_cuda(cudaEventCreate(&s->ev_start[k]), "cudaEventCreate");
                server_fail_cuda(cudaEventCreate(&s->ev_done[k]), "cudaEventCreate");
            }
            s->worker = std::thread(worker_main, s);
        } catch (...) {
            destroy_server(s);
            throw;
        }
        *out = s;
    });
}

isg_status isg_server_submit(isg_server* s, const isg_graph* g, int64_t* ticket) {
    return guarded([&] {
        if (!s || !g || !ticket) fail(ISG_ERR_INVALID, "NULL argument");
        if (g->n > s->opt.max_spins) fail(ISG_ERR_TOO_LARGE, "graph has more than max_spins spins");
        std::unique_ptr<Request> r(new Request());
        r->n = g->n;
        r->t_submit = Clock::now();
        r->table_words = (size_t)public_bins(*g);
        // plan outside the lock: split-and-convolve when enabled and its modelled work is below
        // split_work_ratio of the full enumeration's; else a warp-task program (q inner bits) or
        // the small kernel
        if (s->opt.split_work_ratio > 0 && g->n >= kSplitMinSpins) {
            try {
                auto sp = prepare_split(*g, 0, false, false);   // per request: no lane search at submit
                if (sp->plan.cost < s->opt.split_work_ratio * sp->plan.direct_cost) {
                    r->split = sp;
                    r->blob = sp->blob;
                    r->total_tasks = 1;
                    r->configs = sp->plan.cost / kDirectWarpInstrPerConfig;   // in full-enumeration configurations of work
                }
            } catch (const Error&) {
                // no admissible boundary set: served by tiles
            }
        }
        isg_options o;
        isg_options_init(&o);
        o.max_spins = s->opt.max_spins;
        const DeviceInfo d = s->dinfo;       // the server's device, not the caller's current one
        Plan p;
        if (r->split) {
            // planned above
        } else if (g->n >= kMaxLow + 5) {
            // with symmetry, from 13 spins: the shard with spin N-1 up (12 or more free spins)
            r->sym = s->opt.symmetry && g->n >= kMaxLow + 6;
            if (r->sym) {
                o.shard_bits = 1;
                o.shard_lo = 1;
                o.shard_hi = 2;
            }
            o.inner_bits = std::min(16, g->n - 5 - (r->sym ? 1 : 0));
            if (s->opt.lane_model && g->n >= kServerLaneTableMinSpins) {
                // lane tables where one copy fits a CTA (the enumeration kernel serves the
                // request), else, from kServerLaneModelMinSpins, the quick lane search for the
                // batch kernel's tiles
                isg_options lo = o;
                lo.lane_model = 4;
                lo.inner_bits = std::min(16, g->n - 18 - (r->sym ? 1 : 0));
                try {
                    Plan lp = make_plan(*g, lo, d, true);
                    if (!lp.small && lp.n_sub == kLaneTables) r->lane = std::make_shared<const Plan>(std::move(lp));
                } catch (const Error&) {
                    // too many energy rows for lane tables
                }
                if (!r->lane && g->n >= kServerLaneModelMinSpins) o.lane_model = 3;
            }
            p = r->lane ? *r->lane : make_plan(*g, o, d);
            if (p.small || p.q < p.b) fail(ISG_ERR_INTERNAL, "unexpected plan for a served graph");
            r->b = p.b;
            r->q = p.q;
            r->total_tasks = p.n_tasks;
            r->prefix_base = p.prefix_base;
        } else {
            p = make_plan(*g, o, d);
            p.small = true;
            p.q = 0;
            p.b = 0;
            p.stride = g->n + 1;
            for (int k = 0; k < g->n; ++k) p.perm[k] = k;
            r->b = 0;
            r->total_tasks = 1;
        }
        if (!r->split) {
            r->blob = build_program(*g, p);
            r->bins = (int)(g->n_e_c * (p.stride > 0 ? p.stride : g->n + 1));
            r->configs = std::ldexp(1.0, r->sym ? g->n - 1 : g->n);   // configurations enumerated
        }
        const size_t need = ((r->table_words * 8 + 255) & ~(size_t)255) + r->blob.size() * 8;
        if (need > (size_t)s->opt.arena_bytes) fail(ISG_ERR_TOO_LARGE, "request does not fit the server's table arena");
        std::lock_guard<std::mutex> lk(s->mu);
        if (s->stop) fail(ISG_ERR_INVALID, "server is shutting down");
        if ((int64_t)s->queue.size() >= s->opt.max_queued) fail(ISG_ERR_BUSY, "server queue is full");
        r->ticket = s->next_ticket++;
        if (r->lane) ++s->lane_requests;
        *ticket = r->ticket;
        s->queue.push_back(r->ticket);
        s->reqs.emplace(r->ticket, std::move(r));
        s->cv_work.notify_all();
    });
}

isg_status isg_server_poll(isg_server* s, int64_t ticket, int32_t* done) {
    return guarded([&] {
        if (!s || !done) fail(ISG_ERR_INVALID, "NULL argument");
        std::lock_guard<std::mutex> lk(s->mu);
        auto it = s->reqs.find(ticket);
        if (it == s->reqs.end() || it->second->state == ReqState::Cancelled) fail(ISG_ERR_INVALID, "unknown ticket");
        const ReqState st = it->second->state;
        *done = (st == ReqState::Done || st == ReqState::Failed) ? 1 : 0;
    });
}

isg_status isg_server_wait(isg_server* s, int64_t ticket, int64_t timeout_ms) {
    return guarded([&] {
        if (!s) fail(ISG_ERR_INVALID, "NULL argument");
        std::unique_lock<std::mutex> lk(s->mu);
        auto ready = [&] {
            auto it = s->reqs.find(ticket);
            return it == s->reqs.end() || it->second->state == ReqState::Done || it->second->state == ReqState::Failed ||
                   it->second->state == ReqState::Cancelled;
        };
        if (timeout_ms < 0) s->cv_done.wait(lk, ready);
        else if (!s->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), ready))
            fail(ISG_ERR_TIMEOUT, "request not finished within the timeout");
        auto it = s->reqs.find(ticket);
        if (it == s->reqs.end() || it->second->state == ReqState::Cancelled) fail(ISG_ERR_INVALID, "unknown ticket");
    });
}

isg_status isg_server_result(isg_server* s, int64_t ticket, int64_t* g_out, double* times) {
    return guarded([&] {
        if (!s || !g_out) fail(ISG_ERR_INVALID, "NULL argument");
        std::lock_guard<std::mutex> lk(s->mu);
        auto it = s->reqs.find(ticket);
        if (it == s->reqs.end() || it->second->state == ReqState::Cancelled) fail(ISG_ERR_INVALID, "unknown ticket");
        Request& r = *it->second;
        if (r.state == ReqState::Failed) {
            const isg_status st = r.status;
            const std::string msg = r.message;
            if (r.slot_bytes) r.state = ReqState::Cancelled;   // released once no in-flight step writes into it
            else s->reqs.erase(it);
            fail(st, msg);
        }
        if (r.state != ReqState::Done) fail(ISG_ERR_NOT_READY, "request not finished");
        std::memcpy(g_out, r.result.data(), sizeof(int64_t) * r.result.size());
        if (times) {
            times[0] = seconds_between(r.t_submit, r.t_admit);
            times[1] = seconds_between(r.t_admit, r.t_done);
            times[2] = seconds_between(r.t_submit, r.t_done);
            times[3] = seconds_between(s->t_create, r.t_submit);
        }
        s->reqs.erase(it);
    });
}

isg_status isg_server_cancel(isg_server* s, int64_t ticket) {
    return guarded([&] {
        if (!s) fail(ISG_ERR_INVALID, "NULL argument");
        std::lock_guard<std::mutex> lk(s->mu);
        auto it = s->reqs.find(ticket);
        if (it == s->reqs.end() || it->second->state == ReqState::Cancelled) fail(ISG_ERR_INVALID, "unknown ticket");
        Request& r = *it->second;
        switch (r.state) {
            case ReqState::Queued:
                s->queue.erase(std::remove(s->queue.begin(), s->queue.end(), ticket), s->queue.end());
                s->reqs.erase(it);
                break;
            case ReqState::Active:
            case ReqState::Finishing:
                r.state = ReqState::Cancelled;              // slot freed once no in-flight step carries it
                s->active.erase(std::remove(s->active.begin(), s->active.end(), ticket), s->active.end());
                if (r.last_step < 0 || s->inflight.empty() || r.last_step < s->inflight.front().id) {
                    release_locked(s, r);
                    s->reqs.erase(it);
                }
                break;
            default:                                          // finished: just drop the result
                if (r.slot_bytes) r.state = ReqState::Cancelled;   // failed, slot still written by a step
                else s->reqs.erase(it);
        }
        s->cv_done.notify_all();
    });
}

isg_status isg_server_stats(isg_server* s, double* stats) {
    return guarded([&] {
        if (!s || !stats) fail(ISG_ERR_INVALID, "NULL argument");
        std::lock_guard<std::mutex> lk(s->mu);
        stats[0] = (double)s->steps_done;
        stats[1] = s->configs_done;
        stats[2] = s->device_ms;
        stats[3] = (double)s->queue.size();
        stats[4] = (double)s->n_admitted;
        stats[5] = s->rate_est;
        stats[6] = seconds_between(s->t_create, Clock::now());
        stats[7] = (double)s->reqs.size();
    });
}

void isg_server_destroy(isg_server* s) { destroy_server(s); }

isg_status isg_debug_server_lane_counts(isg_server* s, int64_t* requests, int64_t* launches) {
    return guarded([&] {
        if (!s || !requests || !launches) fail(ISG_ERR_INVALID, "NULL argument");
        std::lock_guard<std::mutex> lk(s->mu);
        *requests = s->lane_requests;
        *launches = s->lane_launches;
    });
}

isg_status isg_debug_server_inject(isg_server* s, int32_t where) {
    return guarded([&] {
        if (!s) fail(ISG_ERR_INVALID, "NULL argument");
        if (where < 0 || where > 2) fail(ISG_ERR_INVALID, "where must be 0, 1 or 2");
        std::lock_guard<std::mutex> lk(s->mu);
        s->inject = where;
    });
}

}  // extern "C"
