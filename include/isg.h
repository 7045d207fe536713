/*
 * isg.h -- C ABI of libisg: exact degeneracy table g(E,M) of finite Ising systems on GB300.
 *
 * Method: Peretyatko, Bogatyrev, Kapitan, Kirienko, Nefedev, Belokon, "Rigorous Calculation of
 * the Partition Function for the Finite Number of Ising Spins" (arXiv:1110.2561).
 *
 * Conventions shared by every call (Sec. 2, Eq. 1 and Eq. 2 of the paper):
 *  - A graph has N spins (1 <= N <= 64) and bonds (i, j, J_ij) with integer J_ij of either sign
 *    (Sec. 2: J "could be sign-changing"). Bonds listed more than once are summed; a pair whose
 *    summed coupling is 0 carries no bond.
 *  - Configuration word s: spin i is up (S_i = +1) when bit i of s is 1, down otherwise (Sec. 3a).
 *  - E(s) = -sum over bonds of J_ij S_i S_j: Eq. (1) without the field term, each bond once.
 *  - M(s) = sum_i S_i, the spin excess (Sec. 2, Sec. 3a).
 *  - g(E, M) = number of configurations with that E and M (Sec. 2); the full table sums to 2^N
 *    and its column at fixed M sums to C(N, (N+M)/2) (Sec. 2, Sec. 4).
 *  - Table layout: int64, E-major, n_e x n_m. With S = sum over bonds of |J|:
 *    bin (e, m) holds E = e_min + 2e and M = -N + 2m, e_min = -S, n_e = S + 1, n_m = N + 1.
 *  - Thermodynamics: H = E - h M (Eq. 1), Z = sum over configurations of exp(-H/T) (Eq. 2),
 *    k_B = 1. Reported per system: ln Z, <E> := <H>, <M>, C = Var(H)/T^2, chi = Var(M)/T.
 *
 * General rules:
 *  - No call throws; every call returns an isg_status, and isg_last_error() returns a message
 *    for the last failing call on the calling thread.
 *  - The caller owns every buffer it passes; the library owns isg_graph and isg_server handles.
 *  - "stream" is a cudaStream_t passed as void* (NULL = the legacy default stream). Calls that
 *    read or write host buffers synchronise that stream before returning; calls whose buffers
 *    are all on the device only enqueue work on it.
 *  - Device pointers must belong to the current CUDA device; the library works on the device
 *    that is current when the call is made.
 */
#ifndef ISG_H
#define ISG_H

#include <stdint.h>

#if defined(__GNUC__)
#define ISG_API __attribute__((visibility("default")))
#else
#define ISG_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    ISG_OK = 0,
    ISG_ERR_INVALID = 1,    /* bad argument: graph, range, options or pointer */
    ISG_ERR_TOO_LARGE = 2,  /* N or the table exceeds a limit */
    ISG_ERR_NOMEM = 3,      /* host or device allocation failed */
    ISG_ERR_CUDA = 4,       /* a CUDA runtime call failed (message in isg_last_error) */
    ISG_ERR_TIMEOUT = 5,    /* a bounded device-side wait ran out */
    ISG_ERR_BUSY = 6,       /* server queue full */
    ISG_ERR_NOT_READY = 7,  /* server result not finished yet */
    ISG_ERR_INTERNAL = 8    /* a kernel self-check failed (bug): the result is not valid */
} isg_status;

typedef struct isg_graph isg_graph;

/* Thermodynamics precision (isg_thermo). */
#define ISG_FP64 0
#define ISG_FP32 1

/*
 * Enumeration options. Initialise with isg_options_init and change fields; every zero field
 * means "planner's choice". Results never depend on the planning fields (only on the graph and
 * the shard range); they exist for tuning and for tests that force every code path.
 */
typedef struct {
    int32_t struct_size;     /* sizeof(isg_options); set by isg_options_init */
    int32_t max_spins;       /* isg_enumerate refuses N > max_spins (default 40; at most 62) */
    int32_t inner_bits;      /* q: each thread walks 2^q configurations per task (0 = plan) */
    int32_t low_bits;        /* b <= 7: unrolled innermost Gray bits (0 = plan) */
    int32_t block_threads;   /* threads per CTA, multiple of 32, <= 1024 (0 = plan) */
    int32_t copies;          /* privatised 32-bit histogram copies per CTA (0 = plan) */
    int32_t ctas_per_sm;     /* resident CTAs per SM to launch (0 = plan) */
    int32_t flush_tasks;     /* flush the 32-bit bins after this many tasks per warp (0 = the
                                largest count that cannot overflow a 32-bit bin) */
    int32_t shard_bits;      /* k: the 2^N configurations form 2^k shards, shard j holding the
                                words whose top k bits (spins N-k .. N-1) equal j */
    int32_t bin_stride;      /* row stride (bins per energy row) of the shared histogram, >= N + 1
                                (0 = plan: padded against shared-memory bank conflicts) */
    int64_t shard_lo;        /* enumerate shards [shard_lo, shard_hi) only; 0,0 = all */
    int64_t shard_hi;
    int32_t accumulate;      /* 1: add the counts into g_out; 0: overwrite g_out */
    int32_t warp_aggregate;  /* 1: combine a warp's equal bins with __match_any_sync before the
                                shared-memory reduction (kept for comparison; 0 is faster on GB300) */
    int32_t stride_residue;  /* preferred residue mod 32 of the histogram row stride (0 = plan;
                                bin_stride, if set, wins) */
    int32_t autotune;        /* 1: pick the unset planning fields by timing candidates (see
                                isg_autotune); results are cached per graph and device */
    int32_t symmetry;        /* 1: enumerate only the configurations with spin N-1 up and add the
                                mirror image M -> -M (a global flip keeps E and negates M for any
                                couplings): the same exact table from half the visits. Not with
                                shards; isg_enumerate_noalloc ignores it */
    int32_t split;           /* batches (isg_batch_create, isg_enumerate_batch): 1 serves each graph whose
                                split-and-convolve plan (isg_enumerate_split) models less work than its
                                full enumeration, a launch's fixed cost included, by a split launch inside
                                the batch; the others go to the tile queue. Same tables either way. */
    int32_t lane_model;      /* which spins carry the lane index of a warp (the five spins at internal
                                positions q .. q+4, in which the 32 lanes of a warp task differ):
                                0 = plan: for isg_enumerate, isg_enumerate_rank and
                                isg_enumerate_noalloc, lane tables (as 4) where one copy of them fits
                                shared memory and no stride is fixed; else on graphs of at least 36
                                free spins the quick search under the model below (as 3); with autotune (isg_autotune,
                                autotune = 1, prepared batches with autotune) the timed faster of the
                                index order and the thorough search's set and histogram row stride
                                (graphs of at least 30 spins); otherwise the index order (as 2).
                                Searches are cached per graph structure, coupling signs aside.
                                1 = the set and stride with the fewest shared-memory bank conflicts
                                under a model of the warp reductions (thorough search), any graph.
                                2 = the five free spins after the inner ones in index order, stride
                                by a fixed preference. 3 = the model with a quick search (dense greedy
                                sets only, fewer draws: milliseconds instead of a tenth of a second).
                                4 = lane tables: the index order's lane spins, every histogram copy
                                split into ten sub-tables with a row stride R that is a multiple of
                                32 (and makes 8 R / G whole, G the graph's energy stride), so that
                                each lane's shared-memory bank is fixed by its up count and its
                                sub-table; no warp reduction has a bank conflict, on any graph. Each
                                sub-table holds only the columns its lanes reach, and the ten share
                                each row side by side where that is smaller than ten padded blocks:
                                about n_e (10 (N - 5) + 32) words a copy. A bin_stride set by the
                                caller selects the blocks at that stride (INVALID unless it meets
                                the rules above). One copy per CTA unless copies is set; TOO_LARGE if
                                one does not fit shared memory. Single-graph calls only: batches
                                (one histogram per warp) refuse 4 with INVALID. */
} isg_options;

/* Fill *opt with the defaults (all planner choices, full range, overwrite). */
ISG_API void isg_options_init(isg_options* opt);

/*
 * Build a graph from an edge list: n_edges bonds (i[b], j[b], J[b]), host arrays, copied.
 * Validation: 1 <= n_spins <= 64; 0 <= i, j < n_spins; i != j; J != 0; |J| <= 2^20.
 * Duplicate pairs are summed (a zero sum drops the bond). Sec. 2 / Eq. 1.
 * On success *out receives a handle to free with isg_graph_destroy.
 * Errors: ISG_ERR_INVALID (bad edge or count), ISG_ERR_NOMEM.
 */
ISG_API isg_status isg_graph_create(int32_t n_spins, int64_t n_edges, const int32_t* i, const int32_t* j,
                            const int32_t* J, isg_graph** out);

/* Free a graph handle (NULL is ignored). */
ISG_API void isg_graph_destroy(isg_graph* graph);

/*
 * Geometry of the table g for this graph (see the header comment): e_min = -S, e_step = 2,
 * n_e = S + 1, m_min = -N, n_m = N + 1. Any output pointer may be NULL.
 */
ISG_API isg_status isg_graph_bins(const isg_graph* graph, int32_t* e_min, int32_t* e_step, int32_t* n_e,
                          int32_t* m_min, int32_t* n_m);

/* Number of spins and of distinct bonds after summing duplicates. */
ISG_API isg_status isg_graph_size(const isg_graph* graph, int32_t* n_spins, int32_t* n_bonds);

/*
 * Enumerate all 2^N configurations (or the shard range of opt) and produce the exact table g
 * (Sec. 2: the degeneracy of M over E; Sec. 3: every configuration is visited).
 * g_out: n_e * n_m int64 (isg_graph_bins), on the device if g_out_on_device != 0 (the call then
 * only enqueues on stream) or on the host (the call synchronises stream). opt may be NULL.
 * Self-check: every walk recomputes its last bin from scratch and compares it with the bin it
 * tracked. A host-output call reports a mismatch as ISG_ERR_INTERNAL; a device-output call
 * records it in the device's self-check word, which isg_device_status reports.
 * Errors: ISG_ERR_INVALID, ISG_ERR_TOO_LARGE (N > max_spins, or the table does not fit the
 * shared-memory histogram), ISG_ERR_NOMEM, ISG_ERR_CUDA, ISG_ERR_INTERNAL (host output only).
 */
ISG_API isg_status isg_enumerate(const isg_graph* graph, void* stream, int64_t* g_out, int32_t g_out_on_device,
                         const isg_options* opt);

/*
 * One graph over several ranks (processes, one GPU each), as the paper splits the outer loops of
 * the enumeration over MPI processes and gathers the results at the root (Sec. 3d): the 2^N
 * configurations are cut into 2^k shards of consecutive words (the top k spins fixed, as
 * opt->shard_bits), and rank r of W takes the contiguous run [r 2^k / W, (r + 1) 2^k / W) (integer
 * division). k = log2 W when W is a power of two, else ceil(log2 W) + 6 (shares within one shard
 * in 64 of each other), at most N (at most N - 1 with symmetry; ranks beyond the shard count get
 * an empty share). With symmetry the shards are those of the half with spin N-1 up.
 * isg_rank_shards: the shard_bits and range [*shard_lo, *shard_hi) of rank `rank` (host only; any
 * output may be NULL). Errors: ISG_ERR_INVALID (N outside [1, 64], world_size outside [1, 2^20],
 * rank outside [0, world_size)).
 */
ISG_API isg_status isg_rank_shards(int32_t n_spins, int32_t rank, int32_t world_size, int32_t symmetry,
                                   int32_t* shard_bits, int64_t* shard_lo, int64_t* shard_hi);

/*
 * Rank `rank`'s share of g (see isg_rank_shards): the counts of its configurations, so the sum of
 * the W ranks' tables (one int64 all-reduce of n_e * n_m values) is the exact table. With
 * opt->symmetry each rank enumerates its shards of the spin-(N-1)-up half and adds their mirror
 * M -> -M (the mirror is linear, so the sum over ranks is again the whole table). A rank with an
 * empty share writes zeros (adds nothing with accumulate). g_out, placement, synchronisation,
 * self-check and errors as isg_enumerate; opt's shard fields must be 0.
 */
ISG_API isg_status isg_enumerate_rank(const isg_graph* graph, void* stream, int64_t* g_out, int32_t g_out_on_device,
                                      int32_t rank, int32_t world_size, const isg_options* opt);

/*
 * The kernels' self-check of the device-output calls (isg_enumerate, isg_enumerate_rank,
 * isg_enumerate_noalloc and isg_enumerate_split with their table on the device), which return before their kernels run:
 * each such kernel ORs a failed check into one self-check word per device, shared by all streams
 * and calls on that device. This call synchronises stream, reads the current device's word and,
 * if clear != 0, resets it to zero (ordered on stream after the read). It returns ISG_ERR_INTERNAL
 * (the message names the failed check) if the word was nonzero: some device-output call on this
 * device since the last clear produced a table that is not valid; the word does not say which.
 * Synchronise the streams of the calls to be covered before calling (or pass their stream).
 * Makes no allocation. Errors: ISG_ERR_INTERNAL, ISG_ERR_CUDA.
 */
ISG_API isg_status isg_device_status(void* stream, int32_t clear);

/*
 * Enumerate n_graphs independent graphs (for example disorder realisations) in one persistent
 * launch: every warp task (32 outer prefixes x 2^q configurations) of every graph is a tile of
 * one queue that the warps of one grid drain (Sec. 3d splits one lattice's outer loops over
 * processes; here the tiles of many lattices share one GPU). g_out[k] receives the table of
 * graphs[k] in its own geometry (isg_graph_bins), all on the device or all on the host
 * (on_device). opt: planning fields apply to every graph (inner_bits = per-lane walk length
 * target, low_bits, block_threads <= 512, ctas_per_sm, symmetry); shard and accumulate fields
 * must be 0.
 * The call synchronises stream. It plans, allocates and frees its own device memory; repeated
 * batches should use isg_batch_create / isg_batch_run. Errors as isg_enumerate.
 */
ISG_API isg_status isg_enumerate_batch(int32_t n_graphs, const isg_graph* const* graphs, void* stream,
                                       int64_t* const* g_out, int32_t on_device, const isg_options* opt);

typedef struct isg_batch isg_batch;

/*
 * Prepare a batch once: plan every graph, and place the programs, the tile descriptors and one
 * output table per graph in device memory owned by the batch (on the current device). Options as
 * isg_enumerate_batch; with opt->autotune the unset fields among inner_bits (per-lane walk
 * length), block_threads, lane_model and stride_residue are chosen by timing candidate plans on
 * every 8th graph first (synchronous; results never depend on them; the lane model's choice is
 * searched once per graph structure, coupling signs aside). The graphs may be destroyed
 * afterwards. Errors: ISG_ERR_INVALID, ISG_ERR_TOO_LARGE, ISG_ERR_NOMEM, ISG_ERR_CUDA.
 */
ISG_API isg_status isg_batch_create(int32_t n_graphs, const isg_graph* const* graphs, const isg_options* opt,
                                    isg_batch** out);

/*
 * Enqueue one run of a prepared batch on stream: zero its tables and task counter, then the
 * persistent launch. The first run captures these steps into a CUDA graph (on a stream of the
 * batch's own); every run launches that graph on `stream`. Runs of one batch share its tables:
 * a run overwrites the previous run's results. Errors: ISG_ERR_INVALID, ISG_ERR_CUDA.
 */
ISG_API isg_status isg_batch_run(isg_batch* batch, void* stream);

/* Device pointer of graph k's table inside the batch (isg_graph_bins geometry of graphs[k]),
 * valid until isg_batch_destroy. */
ISG_API isg_status isg_batch_table(const isg_batch* batch, int32_t k, int64_t** device_table);

/* Synchronise stream and report the kernels' self-check of the last run (ISG_ERR_INTERNAL if a
 * thread's tracked bin disagreed with its recomputation). */
ISG_API isg_status isg_batch_status(isg_batch* batch, void* stream);

/* Free a prepared batch (NULL is ignored). Synchronises the device's work on its memory. */
ISG_API void isg_batch_destroy(isg_batch* batch);

/*
 * Autotune the planning fields of isg_enumerate for this graph on the current device: candidate
 * launch shapes (histogram row-stride residue, threads per CTA, CTAs per SM) are timed with CUDA
 * events on one shard of the configuration space that holds as many warp tasks as the full
 * launch, and the fastest is written to *tuned (a copy of opt, or of the defaults, with the
 * fields filled in) and cached for the graph's program on this device, which isg_enumerate then
 * uses when opt->autotune is set. Results never depend on these fields. Synchronises stream;
 * allocates and frees scratch. Graphs with fewer than 30 spins are not worth timing: their
 * defaults are returned. Errors as isg_enumerate.
 */
ISG_API isg_status isg_autotune(const isg_graph* graph, void* stream, const isg_options* opt, isg_options* tuned);

/*
 * Split-and-convolve enumeration: the same exact table as isg_enumerate, computed with fewer
 * than 2^N configuration visits. This is a variant of the paper's full enumeration (Sec. 3), not
 * the paper's method. A boundary set S of spins is chosen whose removal leaves components with no
 * bond between them. For each of the 2^|S| configurations of S, each component's configurations
 * are enumerated under the field that S exerts on it (Eq. 1 restricted to the component and its
 * bonds to S), and the components' (E, M) histograms are convolved and shifted by the energy and
 * up count of S's own bonds and spins. The result is g(E, M) exactly (integer arithmetic
 * throughout). The global spin flip maps a configuration of S and its components' walks onto
 * the complement's with M negated and E kept, so only the configurations of S with its last spin
 * down are walked and each result is also added at -M. Visits: 2^(|S|-1) * sum over components
 * of 2^|C| (2^0 * sum 2^|C| when S is empty).
 * boundary: a mask of spins (bit i = spin i) to use as S, or 0 to let the library choose: the
 * cheapest, under a work model, among windows of consecutive indices, residue classes of the
 * index and the complement of an independent set. Each component must have at most 30 spins,
 * S at most 40, at most 16 distinct couplings, and the per-warp buffers (two (sum S_c + 2) x
 * (sum |C| + 1) accumulators) must fit in shared memory with the (S + 1)(N + 1) int64 table.
 * g_out: n_e * n_m int64 (isg_graph_bins), on the device if g_out_on_device (only enqueued) or on
 * the host (synchronises stream). The output is overwritten. A failed walk self-check is reported
 * as ISG_ERR_INTERNAL by a host-output call, and recorded for isg_device_status by a device-output
 * call.
 * Errors: ISG_ERR_INVALID (NULL, mask beyond N), ISG_ERR_TOO_LARGE (no admissible boundary, or
 * none cheaper than the full enumeration when boundary = 0), ISG_ERR_NOMEM, ISG_ERR_CUDA,
 * ISG_ERR_INTERNAL (host output only).
 */
ISG_API isg_status isg_enumerate_split(const isg_graph* graph, void* stream, int64_t* g_out, int32_t g_out_on_device,
                                       uint64_t boundary);

/*
 * Exact tables of n graphs (for example disorder realisations of lattices of a few sizes), each by
 * the cheaper method: split-and-convolve (library's boundary choice) where its plan models less
 * work than the full enumeration, else the batched full enumeration (isg_enumerate_batch, default
 * options). Planning is shared by graphs that differ only in coupling signs. The split programs go
 * to the device in one copy and their launches are enqueued back to back on stream.
 * g_out[k]: graph k's table (isg_graph_bins geometry), all on the device if g_out_on_device (only
 * enqueued) or all on the host (synchronises). Tables are overwritten. Errors as
 * isg_enumerate_split (TOO_LARGE when a graph admits no boundary set at all).
 */
ISG_API isg_status isg_enumerate_split_batch(int32_t n, const isg_graph* const* graphs, void* stream,
                                             int64_t* const* g_out, int32_t g_out_on_device);

/*
 * The boundary set isg_enumerate_split would use (boundary as there) and its cost: *chosen the
 * mask of S, *n_components and *largest_component the components left by removing it, *visits
 * = 2^(|S|-1) * sum 2^|C| (the walked configurations), *work_ratio the modelled work relative to the full enumeration (below 1:
 * cheaper). Host only; any output may be NULL. Errors as isg_enumerate_split's planning.
 */
ISG_API isg_status isg_split_plan(const isg_graph* graph, uint64_t boundary, uint64_t* chosen, int32_t* n_components,
                                  int32_t* largest_component, double* visits, double* work_ratio);

/*
 * isg_enumerate for callers that cannot allocate device memory: the paper has no counterpart
 * to this call. It is meant for a caller whose device memory is owned by another allocator, or
 * that runs the enumeration inside a fixed memory budget or a loop that must not enter an
 * allocator. It computes the same table as isg_enumerate with g_out on the device, but makes no
 * cudaMalloc, cudaFree or other allocating call: its task counter, status word and device copy
 * of the graph program live in one 16 KiB array of device memory inside the library, which
 * every GPU that loads the library keeps until the process exits.
 * g_out_device: n_e * n_m int64 on the current device (isg_graph_bins); the call only enqueues
 * work on stream. opt as for isg_enumerate (NULL = defaults), except that symmetry is ignored and
 * autotune only applies a choice already cached for this graph on this device by isg_autotune or
 * an isg_enumerate call with autotune (timing candidates would allocate); without one the
 * planner's defaults are used. The kernels' self-check goes to the device's self-check word:
 * read it with isg_device_status after the stream has run the call.
 * The first call on each device looks up that device's addresses of the array and of the
 * self-check word (with the device current); make that first call before any stream capture. All calls share the array and it
 * keeps the last call's contents (each call clears the counter and status words it needs), so
 * calls whose work overlaps on the GPU (different streams, or different host threads) race and
 * give wrong tables: issue them on one stream.
 * Errors: ISG_ERR_INVALID, ISG_ERR_TOO_LARGE (the graph program exceeds the 16128 bytes left for
 * it, or as isg_enumerate), ISG_ERR_CUDA.
 */
ISG_API isg_status isg_enumerate_noalloc(const isg_graph* graph, void* stream, int64_t* g_out_device,
                                         const isg_options* opt);

/*
 * Thermodynamics on the grid T[0..nT) x h[0..nh) from a table g of this graph's geometry
 * (Eq. 2 summed over the degeneracy table of Sec. 2). T > 0, host arrays. Outputs are
 * nT * nh doubles each, point (a, b) at index a * nh + b: logZ = ln Z, E = <H>, M = <M>,
 * C = Var(H)/T^2, chi = Var(M)/T; any output may be NULL. H = E_J - h M (Eq. 1), so the mean
 * exchange energy is <E_J> = E + h M from the same point's outputs. precision ISG_FP64 or ISG_FP32 (the
 * latter computes weights and sums in float, converting counts and finishing ln Z in double). A
 * grid whose fields are all zero (with at most 1024 energy bins) takes a per-energy path in double
 * in either precision: the sums over M are formed once per energy, then one exponential per
 * temperature and energy.
 * g on the device if g_on_device, outputs on the device if out_on_device; a call with any host
 * buffer synchronises stream. Any counts of this geometry are accepted; the graph's own tables,
 * whose counts lie only on the energies its configurations reach, take the faster path.
 * Errors: ISG_ERR_INVALID, ISG_ERR_NOMEM, ISG_ERR_CUDA.
 */
ISG_API isg_status isg_thermo(const int64_t* g, int32_t g_on_device, const isg_graph* graph, int32_t nT,
                      const double* T, int32_t nh, const double* h, int32_t precision, void* stream,
                      int32_t out_on_device, double* logZ, double* E, double* M, double* C, double* chi);

/*
 * Magnetisation statistics on the grid T[0..nT) x h[0..nh) from a table g of this graph's
 * geometry: the finite-system magnetisation curves that exact counting offers for comparison
 * with measured magnetisation, and Binder's cumulant, whose crossing between sizes locates the
 * ordering temperature of finite systems (Sec. 1, Sec. 5). With the weights of Eq. (2), per
 * point (a, b) at index a * nh + b: abs_M = <|M|>, M2 = <M^2>, M4 = <M^4>,
 * binder = 1 - <M^4> / (3 <M^2>^2) (0 when <M^2> = 0). At h = 0 the mean magnetisation <M> of a
 * finite system is exactly 0, so <|M|> and sqrt(<M^2>) are its magnetisation curves. Any output
 * may be NULL. Arguments, precision, placement, synchronisation and errors as for isg_thermo.
 */
ISG_API isg_status isg_magnetisation(const int64_t* g, int32_t g_on_device, const isg_graph* graph, int32_t nT,
                                     const double* T, int32_t nh, const double* h, int32_t precision, void* stream,
                                     int32_t out_on_device, double* abs_M, double* M2, double* M4, double* binder);

/*
 * Temperature of the specific-heat maximum at field h within [T_lo, T_hi] (the finite-system
 * transition temperature that motivates exact counting, Sec. 1): C(T) = Var(H)/T^2 from Eq. (2)
 * over the table g is evaluated by the thermodynamics kernels on a uniform grid of 257
 * temperatures; the bracket then shrinks to the two neighbours of the best grid point and the
 * grid is re-evaluated, until the bracket is below 1e-12 of the temperature (at most 12 rounds).
 * With several maxima the one that is highest on the first grid wins. g on the device or host
 * (g_on_device); synchronises stream. *T_peak receives the temperature, *C_peak (may be NULL)
 * the value of C there. Errors: ISG_ERR_INVALID, ISG_ERR_NOMEM, ISG_ERR_CUDA.
 */
ISG_API isg_status isg_specific_heat_peak(const int64_t* g, int32_t g_on_device, const isg_graph* graph, double h,
                                          double T_lo, double T_hi, int32_t precision, void* stream,
                                          double* T_peak, double* C_peak);

/*
 * Request server with continuous batching. A worker thread owns one stream on the device that is
 * current at isg_server_create and runs engine steps: each step is one launch of the batched
 * kernel over warp tasks drawn from every admitted request, shortest remaining work first, up to
 * step_ms of device time, so a request that arrives while others run joins the next step. A
 * request is admitted when one of max_inflight slots and room for its table in the device arena
 * are free; its table accumulates on the device and is copied out by the step carrying its last
 * task. Two steps are in flight at a time.
 */
typedef struct isg_server isg_server;

typedef struct {
    int32_t struct_size;     /* sizeof(isg_server_options); set by isg_server_options_init */
    int32_t max_spins;       /* largest N accepted (default 40) */
    int32_t max_inflight;    /* admitted requests at a time (default 256) */
    int32_t max_queued;      /* requests waiting for admission before submit returns BUSY (65536) */
    int64_t arena_bytes;     /* device memory for the admitted requests' tables and programs (64 MiB),
                                mirrored by as much pinned host memory */
    double step_ms;          /* device time per engine step (default 20 ms) */
    int32_t block_threads;   /* threads per CTA of the batched kernel, <= 512 (0 = 512) */
    int32_t ctas_per_sm;     /* 0 = 2 */
    double split_work_ratio; /* 0 (default): every request is enumerated configuration by configuration.
                                r in (0, 1]: a request of at least 24 spins whose split-and-convolve
                                plan (isg_enumerate_split) models less than r of that work is served
                                by one split launch instead; planned at submit, a few milliseconds
                                of host time. The table is the same either way. */
    int32_t symmetry;        /* 1: a request of at least 13 spins served by tile steps enumerates only
                                the configurations with spin N-1 up, and its table is completed by the
                                mirror M -> -M before it is copied out (the global spin flip maps
                                (E, M) to (E, -M) for any couplings): half the work, the same table.
                                0 (default): all 2^N configurations. */
    int32_t lane_model;      /* 1 (default): a tile-served request of at least 28 spins gets lane
                                tables (options.lane_model = 4) where one copy fits a CTA's shared
                                memory, and each step then serves a range of its tasks by a launch of
                                the single-graph enumeration kernel (conflict-free warp reductions;
                                at most 16 such launches a step); otherwise a request of at least 36
                                spins gets the lane spins and row stride of a quick search under the
                                bank-conflict model (options.lane_model = 3: a few milliseconds of
                                host time at submit) for the batch kernel's tiles. 0: the index order
                                in the batch kernel. The table is the same either way. */
} isg_server_options;

ISG_API void isg_server_options_init(isg_server_options* opt);

/* Start a server on the current device (allocates the arena, its pinned mirror and a stream).
 * Errors: ISG_ERR_INVALID, ISG_ERR_NOMEM, ISG_ERR_CUDA. */
ISG_API isg_status isg_server_create(const isg_server_options* opt, isg_server** out);

/* Queue the enumeration of all 2^N configurations of a graph (planned and copied at once; the
 * graph may be destroyed afterwards). *ticket identifies the request. Errors: ISG_ERR_TOO_LARGE
 * (N > max_spins, or its table exceeds the arena), ISG_ERR_BUSY (max_queued requests waiting). */
ISG_API isg_status isg_server_submit(isg_server* server, const isg_graph* graph, int64_t* ticket);

/* *done = 1 once the request has finished (successfully or not). */
ISG_API isg_status isg_server_poll(isg_server* server, int64_t ticket, int32_t* done);

/* Block until the request finishes, at most timeout_ms (< 0: no limit). ISG_ERR_TIMEOUT if the
 * wait ran out (the request continues). */
ISG_API isg_status isg_server_wait(isg_server* server, int64_t ticket, int64_t timeout_ms);

/* Copy a finished request's table into g_out (host, its graph's isg_graph_bins geometry) and
 * release the ticket. times (NULL or 4 doubles): seconds queued before admission, seconds from
 * admission to completion, seconds from submission to completion, submission time since the
 * server started. Errors: ISG_ERR_NOT_READY, ISG_ERR_INVALID (unknown ticket), or the request's
 * own failure status. */
ISG_API isg_status isg_server_result(isg_server* server, int64_t ticket, int64_t* g_out, double* times);

/* Drop a request: queued ones at once, running ones after the steps carrying them finish. */
ISG_API isg_status isg_server_cancel(isg_server* server, int64_t ticket);

/* stats[8]: steps completed, configurations enumerated, device milliseconds of the steps, queued
 * requests, admitted requests, current rate estimate (configurations per second), seconds since
 * creation, open tickets. */
ISG_API isg_status isg_server_stats(isg_server* server, double* stats);

/* Finish the in-flight steps, stop the worker and free everything (queued requests are dropped). */
ISG_API void isg_server_destroy(isg_server* server);

/* Message of the last failing call on this thread ("" if none). Valid until the next call. */
ISG_API const char* isg_last_error(void);

/* Library version string. */
ISG_API const char* isg_version(void);

#ifdef __cplusplus
}
#endif

#endif /* ISG_H */
