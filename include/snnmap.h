/*
 * snnmap.h - C ABI of the GB300 multilevel hypergraph partitioning pass for
 * mapping spiking neural networks onto neuromorphic cores.
 *
 * The operation is the partitioning problem of Ronzani & Silvano, "GPU-
 * Accelerated Hypergraph Partitioning and Placement to Map SNNs on
 * Neuromorphic Hardware", Sec. 3 (Partitioning Definition): given the SNN
 * hypergraph G = (N, E, omega) of Sec. 2 (one vertex per neuron, one
 * hyperedge per axon with one source and its destination synapses, omega(e)
 * the axon's spike frequency) and the per-core limits Omega (neurons),
 * Delta (distinct inbound axons) and Phi (inbound synapses), find rho : N -> P
 * that respects the three limits in every partition and keeps the
 * connectivity Conn = sum_e omega(e) * (lambda(e) - 1) low (Eq. connectivity),
 * with the multilevel method of Sec. 4.1 (coarsening by constrained matching,
 * then uncoarsening with prefix-validated refinement).
 *
 * Conventions shared by every call:
 *  - All arithmetic is integer and exact; results are deterministic and do
 *    not depend on thread scheduling.
 *  - Pointers named d_* are CUDA device pointers; h_* are host pointers.
 *    The caller owns every buffer it passes; the library never frees them.
 *  - stream is a cudaStream_t passed as void*; NULL means the legacy default
 *    stream. Every call enqueues its work on that stream and synchronizes the
 *    stream before returning, so outputs are ready on return.
 *  - Every call returns SNNMAP_OK or one of the SNNMAP_ERR_* codes, and never
 *    throws; snnmap_last_error() then describes the failure (per thread).
 *  - A handle is not thread safe: one call at a time per handle.
 */
#ifndef SNNMAP_H
#define SNNMAP_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define SNNMAP_OK 0
#define SNNMAP_ERR_INVALID 1        /* malformed input or arguments */
#define SNNMAP_ERR_INFEASIBLE 2     /* one neuron alone breaks Delta or Phi */
#define SNNMAP_ERR_OOM 3            /* device or host allocation failed */
#define SNNMAP_ERR_DEVICE_TIMEOUT 4 /* a bounded device wait ran out */
#define SNNMAP_ERR_CUDA 5           /* a CUDA runtime call failed */
#define SNNMAP_ERR_STATE 6          /* call not valid in the handle's state */

/* Per-core limits (Sec. 2, "SNN and Hardware Models"; Sec. 3 constraints)
 * and stopping rules. */
typedef struct {
    int32_t omega;             /* max neurons per core, >= 1 */
    int32_t delta;             /* max distinct inbound axons per core, >= 0 */
    int32_t phi;               /* max inbound synapses per core, >= 0 */
    int32_t max_levels;        /* cap on contractions; coarsening otherwise stops
                                  when no vertex has a candidate (Sec. 4.1) */
    int32_t max_refine_rounds; /* cap on refinement rounds per level */
    int32_t refine_nonpositive; /* 0 (default): a vertex proposes its best move only if
                                   its gain is positive; 1: every vertex with a feasible
                                   move to an adjacent partition proposes its best one
                                   (a variant of Sec. 4.1: moves that only pay after
                                   earlier moves of the sequence can join an enacted
                                   prefix, which still needs a positive total gain) */
} snnmap_params;

/* Summary of one snnmap_partition call. */
typedef struct {
    int32_t levels;          /* contractions performed */
    int32_t n_parts;         /* partition ids range over [0, n_parts): the
                                vertices of the coarsest level */
    int32_t nonempty_parts;  /* partitions holding at least one neuron */
    int32_t rounds;          /* refinement rounds that enacted moves */
    int64_t moves;           /* moves enacted in total */
    int64_t cost_initial;    /* Conn of the coarsest-level partition */
    int64_t cost;            /* final Conn (Eq. connectivity) */
    int64_t pins_total;      /* sum over levels of the pins processed */
} snnmap_stats;

/* One refinement round's outcome (Sec. 4.1, Uncoarsening and Refinement). */
typedef struct {
    int32_t level, round;
    int32_t n_props;  /* vertices that proposed a move */
    int32_t istar;    /* length of the enacted prefix (0: none) */
    int32_t n_active; /* vertices whose best move was evaluated: save > 0 and, after a
                         level's first round on the histogram path, affected by
                         the previous round's moves */
    int32_t rows;     /* 1: gains read from connection rows (snnmap_set_row_budget) */
    int64_t gain;     /* Conn removed by the enacted prefix */
} snnmap_round_log;

/* One coarsening level (Sec. 4.1, Coarsening). */
typedef struct {
    int32_t V, E;
    int64_t P;
    int32_t n_cand;      /* vertices with a valid candidate */
    int32_t n_pairs;     /* matched pairs */
    int64_t pair_terms;  /* sum over hyperedges of |e|(|e|-1): neighbour-histogram updates */
    int32_t n_block;     /* vertices whose histogram needed a block-wide table */
    int32_t n_global;    /* vertices whose histogram needed a table in global memory */
    int32_t carried;     /* 1: candidates carried from the level above (snnmap_set_coarsen_mode),
                            2: read from the score matrix, 0: full neighbour histogram */
    int32_t n_full;      /* vertices that took a full neighbour histogram */
    int64_t hist_work;   /* elements the level's neighbour histograms visited */
} snnmap_level_log;

/* Device time of one pipeline stage, summed over the calls since the last
 * snnmap_profile(h, 1) (CUDA events on the handle's stream). */
typedef struct {
    const char* name;  /* "build", "affinity", "match", "contract", "incidence",
                          "pincount", "gains", "sortmoves", "replay", "validity",
                          "apply" */
    int64_t calls;     /* times the stage ran */
    double ms;         /* summed device time */
} snnmap_stage_time;

typedef struct snnmap_hgraph snnmap_hgraph;

/* Defaults: max_levels 1024, max_refine_rounds 16; omega/delta/phi as given. */
snnmap_params snnmap_default_params(int32_t omega, int32_t delta, int32_t phi);

/*
 * Level 0 of the hierarchy from an SNN hypergraph (Sec. 2).
 *   n_vertices  neurons, ids 0..n_vertices-1.
 *   n_hedges    axons.
 *   d_offsets   int64[n_hedges+1], d_offsets[0] = 0, non-decreasing; axon a's
 *               pins are d_pins[d_offsets[a] .. d_offsets[a+1]).
 *   d_pins      int32[d_offsets[n_hedges]]: the first pin of each axon is its
 *               source neuron, the others its destination neurons, distinct
 *               and different from the source, in any order.
 *   d_w         int32[n_hedges], spike frequencies >= 0.
 * The library copies the input (the caller keeps its buffers) and drops axons
 * with no destination. Errors: SNNMAP_ERR_INVALID for an axon without pins,
 * a pin id out of range, a repeated destination, the source listed as a
 * destination, a negative weight or bad params; SNNMAP_ERR_INFEASIBLE if a
 * neuron alone has more than Delta inbound axons or Phi inbound synapses.
 * On success *out receives a new handle; release it with snnmap_free.
 */
int snnmap_build_hgraph(const snnmap_params* params, int32_t n_vertices, int32_t n_hedges,
                        const int64_t* d_offsets, const int32_t* d_pins, const int32_t* d_w,
                        void* stream, snnmap_hgraph** out);

/*
 * One coarsening step on the current coarsest level (Sec. 4.1, Coarsening):
 * the neighbour histogram and candidate of every vertex (Eq.
 * neigh_histogram: score = summed weight of shared hyperedges, candidates
 * filtered by Omega, Phi and Delta on the merged inbound set, ties to the
 * lower id) and the matching of Eq. matching over the candidate
 * pseudo-forest. *n_cand_out = vertices with a candidate, *n_pairs_out =
 * matched pairs (0 when no vertex has a candidate: coarsening is over).
 */
int snnmap_coarsen_level(snnmap_hgraph* h, void* stream, int32_t* n_cand_out,
                         int32_t* n_pairs_out);

/*
 * Materializes the next level from the last snnmap_coarsen_level matching
 * (Sec. 4.1: each super-node carries size, inbound-axon set size and
 * inbound pin count; pins are remapped, duplicate pins and duplicate
 * hyperedges removed, hyperedges inside one super-node dropped).
 * Outputs the new level's vertex, hyperedge and pin counts.
 * SNNMAP_ERR_STATE if the last coarsening found no pair.
 */
int snnmap_contract(snnmap_hgraph* h, void* stream, int32_t* V_out, int32_t* E_out,
                    int64_t* P_out);

/* Number of levels held (level 0 is the input) and the sizes of one. */
int snnmap_num_levels(const snnmap_hgraph* h, int32_t* n_levels);
int snnmap_level_dims(const snnmap_hgraph* h, int32_t level, int32_t* V, int32_t* E, int64_t* P);

/*
 * Projection (Sec. 4.1, Uncoarsening): d_rho_fine[n] = d_rho_coarse[cid(n)]
 * for the vertices n of `level`, cid mapping them to level+1.
 * d_rho_coarse: int32[V(level+1)], d_rho_fine: int32[V(level)], device.
 */
int snnmap_project(snnmap_hgraph* h, int32_t level, const int32_t* d_rho_coarse,
                   int32_t* d_rho_fine, void* stream);

/*
 * Refinement of one level (Sec. 4.1, Uncoarsening and Refinement), in place
 * on d_rho (int32[V(level)], device, values in [0, n_parts)). Each round
 * computes pins(p, e), every vertex's best feasible positive-gain move to an
 * adjacent partition (gain = save - loss), sorts the moves by decreasing
 * gain (ties: lower vertex id), recomputes each move's gain as if all earlier
 * moves were applied, checks Omega/Phi/Delta after every move with signed
 * events, and enacts the valid prefix of largest positive total gain; rounds
 * repeat until none enacts a move or max_refine_rounds is reached.
 * n_parts is the number of partition ids (vertices of the coarsest level).
 * *cost_out = Conn after refinement. The input must already respect the
 * limits (SNNMAP_ERR_INVALID otherwise).
 */
int snnmap_refine(snnmap_hgraph* h, int32_t level, int32_t n_parts, int32_t* d_rho,
                  void* stream, int64_t* cost_out);

/*
 * The whole pass (Sec. 4.1, Fig. partitioning_flow): coarsen and contract
 * until no candidate remains (or max_levels), one partition per coarsest
 * vertex, then project and refine level by level down to level 0.
 * d_rho_out: int32[n_vertices] device output, partition of every neuron.
 * *cost_out = Conn (Eq. connectivity). stats may be NULL.
 * The handle's levels beyond 0 are rebuilt by each call.
 */
int snnmap_partition(snnmap_hgraph* h, void* stream, int32_t* d_rho_out, int64_t* cost_out,
                     snnmap_stats* stats);

/*
 * Connectivity of a partition of the level-0 neurons (Sec. 3, Eq.
 * connectivity): sum over axons of omega(e) * (distinct partitions among its
 * pins - 1). d_rho: int32[n_vertices] device, values in [0, n_parts)
 * (SNNMAP_ERR_INVALID otherwise). Uses the same per-axon pin-count pass as
 * refinement; temporaries come from the handle's scratch memory.
 */
int snnmap_connectivity(snnmap_hgraph* h, int32_t n_parts, const int32_t* d_rho, void* stream,
                        int64_t* cost_out);

/*
 * Convenience for callers holding host arrays: copies the SNN hypergraph
 * (same layout as snnmap_build_hgraph, host memory) to the device, runs
 * snnmap_partition and copies the partition back into h_rho_out
 * (int32[n_vertices], host). Device memory is released before returning.
 */
int snnmap_partition_host(const snnmap_params* params, int32_t n_vertices, int32_t n_hedges,
                          const int64_t* h_offsets, const int32_t* h_pins, const int32_t* h_w,
                          int32_t* h_rho_out, int64_t* cost_out, snnmap_stats* stats,
                          void* stream);

/*
 * Inspection of a level for verification. Every pointer is a device buffer
 * of the stated size, or NULL to skip that array:
 *   d_off int64[E+1], d_pins int32[P] (source first, destinations
 *   ascending), d_w int64[E], d_k int32[E] (original axons merged),
 *   d_selfdst uint8[E] (some merged axon ends inside the source),
 *   d_size, d_inpins, d_in_count, d_in_internal int32[V] (super-node state).
 * Hyperedge order within a level is unspecified.
 */
int snnmap_level_copy(const snnmap_hgraph* h, int32_t level, int64_t* d_off, int32_t* d_pins,
                      int64_t* d_w, int32_t* d_k, uint8_t* d_selfdst, int32_t* d_size,
                      int32_t* d_inpins, int32_t* d_in_count, int32_t* d_in_internal,
                      void* stream);

/*
 * Results of the last snnmap_coarsen_level, device int32/int64[V] buffers or
 * NULL: candidate (-1: none), its score, the shared inbound count with it,
 * and the matched partner (-1: unmatched).
 */
int snnmap_last_matching(const snnmap_hgraph* h, int32_t* d_cand, int64_t* d_cscore,
                         int32_t* d_cov, int32_t* d_match, void* stream);

/* cid map of `level` (int32[V(level)] into level+1), device buffer. */
int snnmap_level_cid(const snnmap_hgraph* h, int32_t level, int32_t* d_cid, void* stream);

/* Logs of the last snnmap_partition (or refine) calls: copies up to cap
 * entries, *n receives the number available. */
int snnmap_round_logs(const snnmap_hgraph* h, snnmap_round_log* out, int32_t cap, int32_t* n);
int snnmap_level_logs(const snnmap_hgraph* h, snnmap_level_log* out, int32_t cap, int32_t* n);

/* Stage timing: on != 0 clears the counters and starts recording CUDA events
 * around every stage; on == 0 stops. Recording adds two event records per
 * stage call and no synchronization. */
int snnmap_profile(snnmap_hgraph* h, int32_t on);
/* Copies up to cap stage records; *n receives the number of stages. */
int snnmap_stage_times(snnmap_hgraph* h, snnmap_stage_time* out, int32_t cap, int32_t* n);

/*
 * Memory of the hierarchy. Level 0 and the coarsest level always stay in
 * memory; the others keep only their sizes and cid map once their arrays
 * would exceed `bytes` (0: 40% of the device's memory, the default), and are
 * rebuilt exactly from the nearest level below that is still in memory when
 * a later call needs them (refinement, inspection). Results do not depend on
 * the budget.
 */
int snnmap_set_level_budget(snnmap_hgraph* h, int64_t bytes);

/*
 * The partition hypergraph G_P = (P, A, eta) of Sec. 3 ("Partitioning
 * Definition") for a level-0 partition d_rho (device int32[V(0)], values in
 * [0, n_parts)): every axon e is mapped through rho, its source's partition
 * becoming the source and the other partitions of its pins the
 * destinations (a destination in the source's partition is discarded, which
 * breaks the self-cycle); axons with the same source partition and the same
 * destination set merge, eta being their summed omega. An axon whose pins
 * all lie in one partition keeps no destination and is left out of A; the
 * sum of their omega is *internal_out (so sum(eta) + internal = sum(omega)).
 * The result stays in the handle: *n_hedges_out = |A|, *n_pins_out = its
 * pins; snnmap_partition_graph_copy fetches it. Errors: SNNMAP_ERR_INVALID
 * (n_parts < 1, host d_rho, a value outside [0, n_parts)).
 */
int snnmap_partition_graph(snnmap_hgraph* h, int32_t n_parts, const int32_t* d_rho, void* stream,
                           int32_t* n_hedges_out, int64_t* n_pins_out, int64_t* internal_out);
/* Copies the last G_P into device buffers (any may be NULL): d_offsets
 * int64[|A|+1], d_pins int32[pins] (per hyperedge: source partition, then
 * destination partitions ascending), d_eta int64[|A|], d_axons int32[|A|]
 * (axons merged into each). Hyperedge order is deterministic but otherwise
 * unspecified. SNNMAP_ERR_STATE if no G_P was computed. */
int snnmap_partition_graph_copy(const snnmap_hgraph* h, int64_t* d_offsets, int32_t* d_pins,
                                int64_t* d_eta, int32_t* d_axons, void* stream);

/*
 * Memory for connection rows in the refinement of snnmap_partition, and for
 * the score matrix of small coarsening levels. On levels (from the coarsest
 * down) whose vertices times the partitions fit in `bytes` (8 bytes per
 * vertex and partition), each vertex can keep its connection weight and
 * inbound overlap to every partition, updated as moves are enacted and
 * carried to the next finer level, instead of a histogram per round; the
 * library uses them where the measured work of the level above says they
 * pay. Coarsening levels with V vertices use a V x V score matrix when
 * 16 V^2 fits. -1: the default, 1/4 of the device's memory; 0: none. Results
 * do not depend on it (used only when the summed omega stays below 2^31 and
 * every axon's weight is positive).
 */
int snnmap_set_row_budget(snnmap_hgraph* h, int64_t bytes);

/*
 * How a coarsening level's candidates (Sec. 4.1, Eq. neigh_histogram) are
 * found after the previous level's contraction. mode 0 (default): each level
 * chooses by its measured work between a full neighbour histogram and the
 * carried form, in which only the super-nodes just formed, and vertices whose
 * candidate merged into a super-node that no longer suits them, take a full
 * histogram, while every other vertex compares its previous candidate with
 * the super-nodes just formed among its neighbours (exact: the score, shared
 * count and validity of two vertices neither of which merged do not change).
 * 1: always full histograms. 2: the carried form wherever a previous level
 * exists. Results do not depend on the mode. SNNMAP_ERR_INVALID for another
 * value.
 */
int snnmap_set_coarsen_mode(snnmap_hgraph* h, int32_t mode);

/*
 * Work thresholds of the histogram tiers (neighbour and connection
 * histograms): a vertex whose histogram visits at most wwork elements takes
 * one warp with a shared-memory table, at most bwork one block, at most
 * gwork one large block per SM, and more the split tier (work items spread
 * over all SMs into a table in global memory); a vertex whose table
 * overflows a tier moves on to the next. Negative values keep the current
 * setting; defaults 8192, 65536 and 4194304. Results do not depend on them
 * (they place work, not decide it): tests use them to drive every tier.
 */
int snnmap_set_histogram_tiers(snnmap_hgraph* h, int64_t wwork, int64_t bwork, int64_t gwork);

/*
 * Process-wide defaults of the histogram tier thresholds by input size, as an
 * autotuning sweep picked them (paper_2609_07577_gb300/autotune.py writes the
 * table, the Python package loads it): a handle built from a hypergraph of P
 * pins takes the thresholds of the first row with P <= max_pins[i] (rows in
 * increasing max_pins), or the built-in defaults beyond the last row (sizes
 * the sweep did not time); snnmap_set_histogram_tiers
 * overrides them per handle. n = 0 restores the built-in defaults. Handles
 * already built keep theirs. Results do not depend on the table.
 * SNNMAP_ERR_INVALID for n < 0, NULL arrays, negative thresholds or max_pins
 * not increasing.
 */
int snnmap_set_tier_table(int32_t n, const int64_t* max_pins, const int64_t* wwork,
                          const int64_t* bwork, const int64_t* gwork);

/* Bytes of device memory the handle currently holds. */
int snnmap_device_bytes(const snnmap_hgraph* h, int64_t* bytes);

/* Largest figure snnmap_device_bytes would have reported at the library's
 * checkpoints (after each contraction, level rebuild and refinement) since
 * the handle was built. */
int snnmap_peak_bytes(const snnmap_hgraph* h, int64_t* bytes);

/*
 * Releases the handle and everything it owns (waits for its stream first).
 * Device memory of handles comes from one stream-ordered memory pool per
 * device that the library creates: memory a handle frees stays in the pool
 * for the next allocation of any handle, and the pool hands all of it back to
 * the CUDA driver when the last live handle is freed (and after
 * snnmap_partition_host, snnmap_batch_partition or snnmap_serve_destroy when
 * no handle is live). NULL is ignored.
 */
void snnmap_free(snnmap_hgraph* h);

/*
 * Connectivity (same value as snnmap_connectivity) for callers that cannot
 * allocate device memory. This entry point has no counterpart in the paper;
 * it exists for callers whose device memory is entirely reserved by another
 * allocator (a framework's caching pool, a fixed per-tenant budget) and for
 * latency-critical loops that may not call cudaMalloc/cudaFree, since a free
 * can synchronize the whole device. It allocates nothing: no handle, no
 * cudaMalloc or cudaFree, no allocating library routine. Its scratch (one
 * count per hyperedge, an error word, an accumulator) is a static device
 * array of 16 MiB + 256 bytes that every device loading this library holds
 * until the process exits; hence the limit n_hedges <= 4,194,304, larger
 * inputs being rejected with SNNMAP_ERR_INVALID before any work is queued.
 * The first call on a device looks up the array's device address (with that
 * device current). Every call copies its error word to the host and
 * synchronizes the stream, so no call may be issued on a stream under
 * capture. Each call clears the accumulator before use; calls whose work
 * overlaps on the GPU share the array and race, so callers must not overlap
 * them.
 * Inputs (device, caller-owned): the level-0 layout of snnmap_build_hgraph
 * (d_offsets int64[n_hedges+1], d_pins, d_w int32) and d_rho int32[n_vertices]
 * with values in [0, n_parts). The caller guarantees d_offsets[n_hedges] <=
 * the length of d_pins, as for snnmap_build_hgraph (the call takes no pin
 * count and cannot check it). Output: *d_cost_out (device int64) = Conn.
 * Axons with no destination count zero. Cost grows with the square of an
 * axon's pin count. Errors: SNNMAP_ERR_INVALID (negative sizes, n_parts < 1,
 * n_hedges above the limit, host pointers; d_offsets[0] != 0 or decreasing
 * offsets; a pin id outside [0, n_vertices); a negative weight; a partition
 * id outside [0, n_parts)), SNNMAP_ERR_CUDA. snnmap_last_error() describes
 * failures.
 */
int snnmap_connectivity_noalloc(int32_t n_vertices, int32_t n_hedges, const int64_t* d_offsets,
                                const int32_t* d_pins, const int32_t* d_w, const int32_t* d_rho,
                                int32_t n_parts, int64_t* d_cost_out, void* stream);

/*
 * Batched and served forms. The paper maps one network at a time; these calls
 * run many independent mapping jobs (each the whole pass of snnmap_partition,
 * with bit-identical results) on one GPU at once. A server owns `slots`
 * worker threads, each with its own CUDA stream, so the kernels of different
 * jobs overlap on the device. Jobs start in submission order (FIFO); the job
 * at the head of the queue starts when a slot is free and its predicted
 * footprint (snnmap_job_footprint) fits in mem_budget beside the footprints
 * already reserved, or at once when nothing is reserved. A footprint stays
 * reserved while the job runs and, for jobs with keep_hierarchy set, until
 * snnmap_serve_release. Each job keeps at most about its level-0 size of
 * intermediate levels in memory (snnmap_set_level_budget) and gets the
 * larger of 4 times its level-0 size plus 256 MiB and mem_budget / (4 x
 * slots) for connection rows and the score matrix (snnmap_set_row_budget);
 * both count in its footprint. None of this changes a result.
 */
typedef struct snnmap_server snnmap_server;

typedef struct {
    /* inputs: the layout of snnmap_build_hgraph */
    snnmap_params params;
    int32_t n_vertices, n_hedges;
    const int64_t* offsets;   /* [n_hedges + 1] */
    const int32_t* pins;      /* [offsets[n_hedges]]; pin 0 of a hyperedge is its source */
    const int32_t* w;         /* [n_hedges] */
    int32_t* rho_out;         /* [n_vertices] result */
    int32_t on_host;          /* 1: the four arrays are host memory (pinned memory lets
                                 copies overlap other jobs); 0: device memory */
    int32_t keep_hierarchy;   /* 1: the job's handle (level hierarchy) stays on the device
                                 until snnmap_serve_release; see snnmap_serve_hgraph */
    /* outputs, written before the job counts as done */
    int32_t status;           /* SNNMAP_OK or the job's error code */
    int32_t slot;             /* worker slot that ran the job */
    int64_t cost;             /* Conn of rho_out */
    snnmap_stats stats;
    int64_t footprint;        /* predicted device bytes reserved for the job */
    int64_t peak_bytes;       /* measured: handle peak plus the job's input copies */
    double t_submit_ms, t_start_ms, t_end_ms;  /* host clock, ms since the server's creation */
    char error[128];          /* snnmap_last_error text of a failed job */
} snnmap_job;

typedef struct {
    int32_t slots;            /* jobs in flight at once (one stream each); 0: 8 */
    int32_t dry_run_us;       /* > 0: host-only run for testing the scheduler: no GPU is
                                 touched, each job holds its slot this many microseconds
                                 per million pins (at least 1 ms) and ends with status OK */
    int64_t mem_budget;       /* bytes of footprint admitted at once; 0: 80% of the device
                                 memory free at creation (dry run: 2^36) */
} snnmap_serve_opts;

/* Predicted peak device bytes of one job with the given level-0 sizes and
 * the smallest row budget a server grants (host-only arithmetic; no GPU
 * needed; a server adds any larger grant). on_host adds the input copies.
 * Errors: SNNMAP_ERR_INVALID for negative sizes or a NULL output. */
int snnmap_job_footprint(int32_t n_vertices, int32_t n_hedges, int64_t n_pins, int32_t on_host,
                         int64_t* bytes);

int snnmap_serve_create(const snnmap_serve_opts* opts, snnmap_server** out);
/* Queues a job; the job struct and its buffers must stay valid (and
 * unmodified) until the job is done. *ticket identifies it (>= 1). Returns
 * at once. Errors: SNNMAP_ERR_INVALID (NULL or negative sizes),
 * SNNMAP_ERR_STATE (server shutting down). Input errors of the job itself are
 * reported in job->status. */
int snnmap_serve_submit(snnmap_server* s, snnmap_job* job, int64_t* ticket);
/* Blocks until the job is done or timeout_ms passes (< 0: no limit); *done
 * (may be NULL) receives 1 if it is done. Any number of threads may submit
 * and wait; a ticket must not be released while another thread waits on
 * it. */
int snnmap_serve_wait(snnmap_server* s, int64_t ticket, double timeout_ms, int32_t* done);
/* The resident hierarchy of a done job submitted with keep_hierarchy (owned
 * by the server; valid until snnmap_serve_release). SNNMAP_ERR_STATE if the
 * job is not done, failed, or kept nothing. */
int snnmap_serve_hgraph(snnmap_server* s, int64_t ticket, snnmap_hgraph** out);
/* Frees a done job's hierarchy and footprint and forgets the ticket. */
int snnmap_serve_release(snnmap_server* s, int64_t ticket);
/* Jobs waiting, jobs running, and bytes of footprint reserved now; any
 * output may be NULL. */
int snnmap_serve_info(snnmap_server* s, int32_t* queued, int32_t* running, int64_t* reserved);
/* Finishes running jobs, marks queued ones SNNMAP_ERR_STATE, frees every kept
 * hierarchy and the server. */
int snnmap_serve_destroy(snnmap_server* s);

/* Runs n_jobs jobs to completion on one server (largest pin count first) and
 * returns SNNMAP_OK when every job succeeded, else the first failed job's
 * status; every job's own status, cost, stats and times are filled in.
 * keep_hierarchy is ignored. */
int snnmap_batch_partition(snnmap_job* jobs, int32_t n_jobs, const snnmap_serve_opts* opts);

/*
 * Placement swap refinement (Sec. 4.2, "Swap Proposals" and "Placement
 * Refinement") of the partition hypergraph G_P = (P, A, eta) on a width x
 * height lattice of cores, core h = y * width + x, distances Manhattan.
 *
 * Per round, each node p on core h = gamma(p) has a force towards every
 * adjacent core k (Eq. force: the sum over its hyperedges a of eta(a) times
 * the sum over the other pins q of dist(h, gamma(q)) - max(dist(k,
 * gamma(q)), 1)); the tension of two adjacent cores is the sum of the forces
 * of their occupants towards each other (Eq. tension; an empty core adds
 * nothing). Each occupied core proposes the adjacent core of largest
 * tension (the lowest core id on ties) when that tension is positive; the
 * proposals are matched by Eq. matching with tension as the score (an empty
 * core proposes nothing but may take its best proposer); the matched swaps,
 * ordered by decreasing tension (ties: lower core id first), are each
 * re-evaluated with every earlier swap applied, and the prefix with the
 * largest positive sum (the shortest on ties) is applied. Rounds repeat
 * until one applies nothing, or max_rounds have run. A swap's re-evaluated
 * tension is exactly the drop of the total residual distance (see
 * snnmap_place_trd), so every round lowers it by its logged gain.
 *
 * Multi-start: n_starts placements are refined together (the paper refines
 * its Pi starts concurrently); each one's result equals its refinement
 * alone. d_gamma: device int32[n_starts * n_nodes], start-major, gamma of
 * start s at d_gamma[s * n_nodes ..], refined in place; every start's cores
 * must be distinct and in [0, width * height).
 *
 * G_P: d_offsets int64[n_hedges + 1] (from 0, non-decreasing), d_pins int32
 * (node ids in [0, n_nodes); a repeated pin counts as often as it appears),
 * d_eta int64[n_hedges]; all device memory, owned by the caller, read only.
 * Sums are int64 and exact while sum_a eta(a) |a|^2 (width + height) < 2^63.
 *
 * Outputs on the host: h_rounds_out[n_starts] (may be NULL) receives each
 * start's rounds, the last one applying nothing unless max_rounds stopped
 * it; h_log (may be NULL) receives round r of start s at h_log[s * log_cap
 * + r] for r < min(rounds, log_cap).
 *
 * Errors: SNNMAP_ERR_INVALID (negative sizes or max_rounds, width or height
 * < 1, n_starts < 1, n_starts * width * height >= 2^31, n_nodes > width *
 * height, host pointers, malformed offsets, a pin or core out of range, two
 * nodes of one start on one core; d_gamma is then unchanged),
 * SNNMAP_ERR_OOM, SNNMAP_ERR_CUDA.
 */
typedef struct {
    int32_t props;    /* occupied cores that proposed a swap */
    int32_t swaps;    /* swaps in the matching */
    int32_t applied;  /* length of the applied prefix (0: none) */
    int32_t reserved;
    int64_t gain;     /* summed re-evaluated tension of the applied prefix */
} snnmap_place_log;

int snnmap_place_refine(int32_t n_nodes, int32_t n_hedges, const int64_t* d_offsets,
                        const int32_t* d_pins, const int64_t* d_eta, int32_t width,
                        int32_t height, int32_t n_starts, int32_t* d_gamma, int32_t max_rounds,
                        void* stream, int32_t* h_rounds_out, snnmap_place_log* h_log,
                        int32_t log_cap);

/* Total residual distance of each start's placement (the measure by which
 * Sec. 4.2 picks the best of its multi-start results): sum over hyperedges
 * a of eta(a) times the Manhattan distances between the cores of every
 * unordered pair of its pins. Arguments as in snnmap_place_refine; d_gamma
 * is read only; h_trd_out: host int64[n_starts]. Same errors. */
int snnmap_place_trd(int32_t n_nodes, int32_t n_hedges, const int64_t* d_offsets,
                     const int32_t* d_pins, const int64_t* d_eta, int32_t width, int32_t height,
                     int32_t n_starts, const int32_t* d_gamma, void* stream, int64_t* h_trd_out);

/* The choice among multi-start results (Sec. 4.2, "Placement Refinement"):
 * the start whose placement has the smallest total residual distance
 * (snnmap_place_trd), the lowest start on ties. Arguments as in
 * snnmap_place_trd; outputs on the host: *best_out the start, *trd_out (may
 * be NULL) its total residual distance, h_trd_out (may be NULL) int64
 * [n_starts] every start's. Same errors, and SNNMAP_ERR_INVALID for a NULL
 * best_out. */
int snnmap_place_best(int32_t n_nodes, int32_t n_hedges, const int64_t* d_offsets,
                      const int32_t* d_pins, const int64_t* d_eta, int32_t width, int32_t height,
                      int32_t n_starts, const int32_t* d_gamma, void* stream, int32_t* best_out,
                      int64_t* trd_out, int64_t* h_trd_out);

/*
 * Initial placement of G_P (Sec. 4.2, "Initial Placement") for n_starts
 * starts at once. Each start's node sequence begins as its given order
 * (d_seq0: device int32[n_starts * n_nodes], start-major, each a
 * permutation of [0, n_nodes); the paper draws them at random). The
 * sequence is bisected recursively (a section of n nodes into its first
 * ceil(n/2) and its remaining ones, down to single nodes); between the two
 * halves of every section, label propagation applies, one at a time, the
 * swap of a node of each half that lowers their cut the most (the summed
 * eta of hyperedges with pins in both halves, pins elsewhere ignored; ties
 * to the lower node of the first half, then of the second) while one lowers
 * it, at most 4 * min(size of the halves) swaps. Folding, bottom-up,
 * reverses a section (with everything inside it) when its child more
 * strongly connected to the section's sibling does not face that sibling
 * (ties keep the order). The i-th node of the final sequence goes to the
 * i-th core in Hilbert order (snnmap_hilbert_order).
 *
 * G_P as in snnmap_place_refine; the pins of a hyperedge must be distinct.
 * Outputs (device, start-major): d_seq_out int32[n_starts * n_nodes] the
 * final sequences (may be NULL), d_gamma_out int32[n_starts * n_nodes] the
 * placements (node -> core), ready for snnmap_place_refine.
 *
 * Work: per label-propagation round of a pair of halves of sizes nL, nR, an
 * nL x nR matrix of int64 (device memory grows with n_starts * n_nodes^2 /
 * 4 for the top split).
 *
 * Errors: SNNMAP_ERR_INVALID (negative sizes, width or height < 1,
 * n_starts outside [1, 65535], width * height or n_starts * n_nodes >= 2^31,
 * n_nodes > width * height, host pointers, malformed offsets, a pin out of
 * range or repeated within its hyperedge, an initial order that is not a
 * permutation), SNNMAP_ERR_OOM, SNNMAP_ERR_CUDA.
 */
int snnmap_place_initial(int32_t n_nodes, int32_t n_hedges, const int64_t* d_offsets,
                         const int32_t* d_pins, const int64_t* d_eta, int32_t width,
                         int32_t height, int32_t n_starts, const int32_t* d_seq0,
                         int32_t* d_seq_out, int32_t* d_gamma_out, void* stream);

/* The cores of a width x height lattice (core = y * width + x) in Hilbert
 * order: ordered by their index along the Hilbert curve of the smallest
 * power-of-two square covering the lattice, cells outside the lattice
 * skipped. d_order_out: device int32[width * height]. Errors:
 * SNNMAP_ERR_INVALID (width or height < 1, width * height >= 2^31, a host
 * pointer), SNNMAP_ERR_OOM, SNNMAP_ERR_CUDA. */
int snnmap_hilbert_order(int32_t width, int32_t height, int32_t* d_order_out, void* stream);

/* Kernels launched by the library in this process so far. */
int64_t snnmap_launch_count(void);

/*
 * Measurement utility with no counterpart in the paper: the on-chip ceiling
 * of the neighbour histogram of Eq. neigh_histogram as this library builds
 * it. The block tier's shared-memory table insert (hash probe, key claim,
 * integer adds of score and shared count) runs on keys made in registers
 * (no global memory), `distinct_keys` distinct neighbours per table (1 to
 * 1536, the tier's load limit), the tier's block size and blocks per SM,
 * `rounds` tables per block, each followed by the scan that reads and
 * resets it. *updates_per_s: element updates per second of the timed launch
 * (after one untimed launch). Allocates 8 bytes of device memory; synchronizes
 * the stream. Errors: SNNMAP_ERR_INVALID, SNNMAP_ERR_CUDA.
 */
int snnmap_hist_ceiling(int32_t distinct_keys, int32_t rounds, void* stream,
                        double* updates_per_s);

/* Message of the last failed call on this thread ("" if none). */
const char* snnmap_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* SNNMAP_H */
