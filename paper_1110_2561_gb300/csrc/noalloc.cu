// noalloc.cu -- isg_enumerate_noalloc: the enumeration entry point for callers that must not
// allocate device memory.
//
// isg_enumerate takes a few kilobytes of stream-ordered scratch per call (a pool allocation) for
// its task counter, its status word and the device copy of the graph program. Some callers
// cannot allow that: a process whose device memory is fully reserved by another allocator (for
// example a framework's caching allocator holding the whole GPU), a real-time or serving loop
// that must not enter an allocator on its hot path, or code that runs the enumeration inside a
// fixed memory budget. This entry point keeps that scratch in one statically sized array in
// device memory instead, so a call makes no cudaMalloc/cudaFree and no allocating library call.
//
// The array below is part of the library image: every GPU that loads libisg holds its 16 KiB
// until the process exits. Host code cannot use the array's name as a device address (on the
// host it names a stand-in object), so the device address is looked up once per device with
// cudaGetSymbolAddress and passed to the kernels.
#include <cuda_runtime.h>

#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "isg_internal.h"

namespace isg {

// Scratch of isg_enumerate_noalloc: [0, 8) task counter, program from byte 256 on. Shared by
// every call on a device. (The kernels' self-check goes to the device's status word, a file-scope
// __device__ word of its own that isg_device_status reads.)
constexpr size_t kNoallocScratchBytes = 16384;
constexpr size_t kNoallocProgramOffset = 256;
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoallocScratchBytes];

DeviceInfo device_info();
void launch_enumeration(const Plan& p, const uint64_t* d_blob, int blob_words, int64_t* table,
                        unsigned long long* counter, unsigned int* status, cudaStream_t s,
                        const uint64_t* host_blob);

// Device address of the scratch array on the current device, looked up on the first call that
// runs on that device (with that device current) and cached.
static unsigned char* noalloc_scratch_address() {
    static std::mutex mu;
    static std::vector<unsigned char*> addr;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) fail(ISG_ERR_CUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
    std::lock_guard<std::mutex> lk(mu);
    if ((int)addr.size() <= dev) addr.resize(dev + 1, nullptr);
    if (!addr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p)
            fail(ISG_ERR_CUDA, std::string("cudaGetSymbolAddress(no-alloc scratch): ") + cudaGetErrorString(e));
        addr[dev] = static_cast<unsigned char*>(p);
    }
    return addr[dev];
}

}  // namespace isg

using namespace isg;

extern "C" isg_status isg_enumerate_noalloc(const isg_graph* graph, void* stream, int64_t* g_out_device,
                                            const isg_options* opt) {
    return guarded([&] {
        if (!graph || !g_out_device) fail(ISG_ERR_INVALID, "graph or g_out_device is NULL");
        isg_options o = resolve_options(opt);
        // autotune: the cached choice for this graph, if it was tuned before (timing allocates)
        if (o.autotune) apply_cached_autotune(*graph, o);
        const DeviceInfo d = device_info();
        const Plan p = make_plan(*graph, o, d, true);
        const std::vector<uint64_t> blob = build_program(*graph, p);
        const size_t blob_bytes = blob.size() * 8;
        if (blob_bytes > kNoallocScratchBytes - kNoallocProgramOffset)
            fail(ISG_ERR_TOO_LARGE, "graph program of " + std::to_string(blob_bytes) + " bytes exceeds the " +
                                        std::to_string(kNoallocScratchBytes - kNoallocProgramOffset) +
                                        "-byte no-alloc scratch");
        unsigned char* scratch = noalloc_scratch_address();
        cudaStream_t s = static_cast<cudaStream_t>(stream);
        auto check = [](cudaError_t e, const char* what) {
            if (e != cudaSuccess) fail(ISG_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
        };
        // the counter must start at zero; the program is overwritten whole
        check(cudaMemsetAsync(scratch, 0, 8, s), "cudaMemsetAsync(counter)");
        check(cudaMemcpyAsync(scratch + kNoallocProgramOffset, blob.data(), blob_bytes, cudaMemcpyHostToDevice, s),
              "cudaMemcpyAsync(program)");
        if (!o.accumulate)
            check(cudaMemsetAsync(g_out_device, 0, sizeof(int64_t) * (size_t)public_bins(*graph), s),
                  "cudaMemsetAsync(g_out)");
        launch_enumeration(p, reinterpret_cast<const uint64_t*>(scratch + kNoallocProgramOffset), (int)blob.size(),
                           g_out_device, reinterpret_cast<unsigned long long*>(scratch), device_status_word(), s,
                           nullptr);
    });
}
