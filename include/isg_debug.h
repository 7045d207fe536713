/*
 * isg_debug.h -- inspection calls of libisg for tests and tuning. They run on the host only and
 * make no CUDA call.
 */
#ifndef ISG_DEBUG_H
#define ISG_DEBUG_H

#include <stdint.h>

#include "isg.h"

#ifdef __cplusplus
extern "C" {
#endif

/*
 * The plan isg_enumerate would use for this graph and these options on a device with `sms`
 * multiprocessors (0 = 152). out[0..18] = small-kernel flag, inner bits q, low-block size b,
 * warp tasks, threads per CTA, histogram copies, CTAs per SM, tasks per flush round, grid,
 * shared-memory bytes per CTA, energy stride G, compact energy bins, bytes of the program that
 * isg_enumerate copies to the device, histogram row stride, whether the lane spins come from the
 * bank-conflict model (options.lane_model), the model's expected shared-memory wavefronts per warp
 * reduction of the plan and of the index order's lane spins (both x 10^6; 0 without the model),
 * the mask of the five lane spins (caller numbering), and the histogram sub-tables per copy
 * (1, or 10 with lane tables: options.lane_model = 4). Errors as isg_enumerate.
 */
ISG_API isg_status isg_debug_plan(const isg_graph* graph, const isg_options* opt, int32_t sms, int64_t* out);

/*
 * Shared-memory wavefronts of the enumeration kernel's warp reductions under the plan of *opt,
 * sampled on the host: for `samples` draws (splitmix64 from `seed`) of a warp task and an inner
 * configuration, the 32 lanes' word addresses (the lane's sub-table start plus its bin) at that
 * step, and the most distinct addresses that fall in one of the 32 banks (the wavefronts the
 * reduction takes; lanes at one address share one). Writes their mean and maximum. Errors:
 * INVALID (NULL pointers, samples < 1, or a plan without warp tasks), as isg_enumerate otherwise.
 */
ISG_API isg_status isg_debug_lane_banks(const isg_graph* graph, const isg_options* opt, int32_t samples, uint64_t seed,
                                        double* mean_wavefronts, int32_t* max_wavefronts);

/*
 * The histogram layout of one copy under the plan of *opt (host only), as 99 int32 in out:
 * [0] row stride R, [1] words of one copy, [2] sub-tables n_sub (1, or 10 with lane tables),
 * [3..13) sub_off, [13..23) m_lo, [23..33) m_hi, [33..65) lane_word, [65..97) lane_sub,
 * [97] packed (1: the lane tables share each row; 0: each is a block of its own), [98] 0.
 * Bin (e', m) of sub-table t is word sub_off[t] + e' R + m of the copy, for m in [m_lo[t], m_hi[t]];
 * lane l counts into sub-table lane_sub[l], starting at word lane_word[l]. Entries past n_sub
 * are 0. Errors: INVALID (NULL pointers, or a thread-per-configuration plan), as isg_enumerate
 * otherwise.
 */
ISG_API isg_status isg_debug_lane_layout(const isg_graph* graph, const isg_options* opt, int32_t* out);

/*
 * Run the enumeration kernels' per-thread walk on the host, with every counter address checked,
 * and write g (host buffer, isg_graph_bins geometry) as isg_enumerate would. The walk visits
 * 2^N configurations one by one (Sec. 3), so this is for small N. Returns ISG_ERR_INTERNAL if
 * an address leaves the histogram or the incrementally tracked bin of a thread's last
 * configuration differs from its recomputation.
 */
ISG_API isg_status isg_debug_emulate(const isg_graph* graph, const isg_options* opt, int64_t* g_out);

/*
 * isg_enumerate_rank's work for rank `rank` of `world_size` run on the host by the same walk as
 * isg_debug_emulate (shards, symmetry half and mirror as there), into a host table. For small N
 * only. Errors as isg_enumerate_rank and isg_debug_emulate.
 */
ISG_API isg_status isg_debug_emulate_rank(const isg_graph* graph, int32_t rank, int32_t world_size, const isg_options* opt,
                                          int64_t* g_out);

/*
 * isg_debug_emulate with a mistake planted in the program first: delta is added to the field
 * constant (the spin's sum of |J|) in the site record at internal position `site`, as a wrong
 * program entry would. *word (may be NULL) receives the self-check word the walk produced (bit 0:
 * a walk's tracked bin differed from its recomputation; bit 1: an address left the histogram);
 * the return value is the status the library reports for that word (ISG_ERR_INTERNAL when
 * nonzero, with the message that isg_device_status and the host-output calls give). The check
 * compares each walk's last bin only, so it sees a mistake whose effects do not cancel over the
 * walk: one in the spin at the top inner position (site = q - 1, flipped once per walk) always
 * shows; the reflected Gray order undoes most others in pairs. The graph must take the Gray-walk
 * kernel (at least 11 free spins, or forced inner_bits / low_bits); site < N.
 */
ISG_API isg_status isg_debug_emulate_planted(const isg_graph* graph, const isg_options* opt, int32_t site, int32_t delta,
                                             int64_t* g_out, uint32_t* word);

/*
 * Run the split kernel's per-warp work (isg_enumerate_split with the same boundary argument) on
 * the host, lane by lane, with every histogram, accumulator and table index checked, and write g
 * (host buffer, isg_graph_bins geometry). For small boundary sets and components only. Returns
 * ISG_ERR_INTERNAL if an index leaves its buffer or a parity or range check fails.
 */
ISG_API isg_status isg_debug_emulate_split(const isg_graph* graph, uint64_t boundary, int64_t* g_out);

/*
 * Measured peaks of the units that bound the enumeration kernel on the current device, in
 * lane-operations per second over the whole GPU: shared-memory 32-bit reductions with each lane
 * in its own bank (red_conflict_free) and with scattered addresses (red_scattered), integer ALU
 * operations (alu: independent xor/add chains), and the scattered reductions counted through
 * __match_any_sync warp aggregation (match_aggregated: lanes counted per second). Runs short
 * kernels on `stream` and synchronises it. Any output may be NULL (a NULL match_aggregated
 * skips that kernel). Errors: ISG_ERR_CUDA.
 */
ISG_API isg_status isg_probe_peaks(void* stream, double* red_conflict_free, double* red_scattered, double* alu,
                                   double* match_aggregated);

/*
 * Host-side failure injection for tests of the request server's error handling (no GPU fault is
 * made): where = 1 makes the server's next engine step fail on the host before its first enqueue,
 * where = 2 after its kernels were enqueued (the server then drains its stream before failing the
 * requests), 0 cancels a pending injection. The step fails like a failing CUDA call would: the
 * admitted requests with tiles left report ISG_ERR_CUDA, their arena slots are released once no
 * step in flight writes into them, and the server keeps serving. Errors: ISG_ERR_INVALID.
 */
ISG_API isg_status isg_debug_server_inject(isg_server* server, int32_t where);

/*
 * How the request server has served its lane-table requests so far: *requests = requests
 * submitted with lane tables (served by the single-graph enumeration kernel in task ranges),
 * *launches = enumeration-kernel launches issued for them. Errors: ISG_ERR_INVALID.
 */
ISG_API isg_status isg_debug_server_lane_counts(isg_server* server, int64_t* requests, int64_t* launches);

#ifdef __cplusplus
}
#endif

#endif /* ISG_DEBUG_H */
