// batch_internal.h -- tile-queue descriptors shared by the batch and serving translation units.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>
#include <vector>

#include "isg_internal.h"

namespace isg {

struct BatchInst {
    int64_t* g;              // public table of this instance (device)
    uint64_t prefix_base;    // lane prefix of task 0
    uint64_t task_lo;        // first task of this instance in this launch
    uint64_t tile_begin;     // first tile of this instance in the launch's tile numbering
    uint64_t n_tiles;        // tiles (= tasks) of this instance in this launch
    uint32_t blob_off;       // word offset of the program in the blob array
    uint32_t blob_words;
};

struct BatchPlan {
    int B = kMaxLow;
    std::vector<BatchInst> inst;        // device descriptors (g filled by the caller), tile order
    std::vector<int> order;             // inst[k] describes graphs[order[k]]
    std::vector<uint64_t> blobs;
    std::vector<int> small_ids;         // descriptors of instances for the small kernel
    std::vector<int> mirror_ids;        // symmetry: instances whose half table is completed in place
    uint64_t n_tiles = 0;
    int prog_words = 0, slot_words = 0, threads = 512, warps_per_cta = 16, small_max_words = 0;
    size_t smem = 0;
    int grid = 0;
};

// Enqueue the batch kernels of a plan (device descriptors, programs and small-instance ids).
// d_small holds small_ids followed by mirror_ids.
void launch_batch(const BatchPlan& bp, const BatchInst* d_inst, const uint64_t* d_blobs, const int* d_small,
                  unsigned long long* counter, unsigned int* status, cudaStream_t s, int ctas_per_sm);

// The symmetry mirror alone (one CTA per instance): descriptors d_inst[d_ids[0 .. n)] hold the
// halves with spin N-1 up, completed in place.
void launch_mirror(const BatchInst* d_inst, const int* d_ids, int n, const uint64_t* d_blobs, cudaStream_t s);

}  // namespace isg
