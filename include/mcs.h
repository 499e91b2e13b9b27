/*
 * mcs.h -- C ABI of the B300 (sm_103a) maximum common induced subgraph solver.
 *
 * The library computes, for graph pairs (G, H), a maximum common induced
 * subgraph (Section II-A: the largest graph isomorphic to an induced subgraph
 * of both G and H; mapped vertices keep their labels, and an arc x->y exists
 * in G exactly when f(x)->f(y) exists in H, self-loops included) with
 * McSplit's branch and bound (Section II-B, Algorithm 1, Eq. 1): label classes
 * are split by adjacency to each newly mapped pair (Table 1) and a branch is
 * pruned when |M| + sum over classes of min(|L|, |R|) <= |incumbent|.
 * All graph arithmetic is exact integer work; the size returned with status
 * MCS_OK is the proven optimum.
 *
 * Graph encoding (all entry points):
 *   n       number of vertices, 0 <= n <= MCS_MAX_N (256: the paper's solvers
 *           stop at 254, Section III-B).  Graphs of up to 64 vertices run on
 *           one-word bit sets; larger ones on two or four words per vertex
 *           set (mcs_solve and mcs_solve_batch choose per pair; the device
 *           entry point takes them with MCS_WIDE).  Serving, the ordering
 *           network, the strategies of Section IV-A and the allocation-free
 *           call take graphs of up to 64 vertices.
 *   adj     n*n bytes, row major, adj[i*n + j] == 1 iff arc i -> j, else 0.
 *           Without MCS_DIRECTED the matrix must be symmetric.  Diagonal
 *           entries are self-loops; they are allowed and must be matched.
 *   labels  n int32 vertex labels (>= 0), or NULL for unlabelled.  A vertex may
 *           only be mapped onto a vertex with the same label.
 *
 * Mapping encoding: for pair p, map[p*MCS_MAX_N + x] is the H vertex matched
 * to G vertex x (original numbering), or -1; entries x >= n_G are -1.
 *
 * Ownership: the caller owns every buffer passed in or out.  The library
 * copies what it needs before a call returns (synchronous calls) or before it
 * enqueues work (mcs_submit); it never keeps a caller pointer.  A context is
 * not thread safe: use one context per host thread.
 *
 * Errors: functions return MCS_OK (0) or a positive status on success and a
 * negative MCS_ERR_* code on failure; mcs_strerror() names every code.  Batch
 * calls also set a per-pair status and return the worst one.
 */
#ifndef MCS_H_
#define MCS_H_

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define MCS_MAX_N 256

/* status / return codes */
#define MCS_OK                 0   /* optimum found and proven                        */
#define MCS_TIMEOUT            1   /* time limit hit: size is a valid lower bound      */
#define MCS_PENDING            2   /* mcs_poll: request not finished yet               */
#define MCS_ERR_ARG           -1   /* NULL pointer, n out of range, entry not 0/1,     */
                                   /* asymmetric matrix without MCS_DIRECTED,          */
                                   /* negative label, unknown ticket                   */
#define MCS_ERR_NOMEM         -2   /* device or pinned allocation failed              */
#define MCS_ERR_CUDA          -3   /* a CUDA runtime call failed                      */
#define MCS_ERR_DEVICE_STALL  -4   /* a bounded device-side wait expired              */
#define MCS_ERR_UNSUPPORTED   -5   /* option not supported for these flags or inputs  */

/* flags */
#define MCS_DIRECTED          0x1u  /* arcs are ordered pairs (4-way class split)      */
#define MCS_ORDER_PLAIN       0x0u  /* degree order (Section IV-A); the default        */
#define MCS_ORDER_LEARNED     0x2u  /* candidate order from the ordering network      */
                                    /* (mcs_set_order_model); exact either way; falls  */
                                    /* back to the degree order without a model        */
#define MCS_NO_MAPPING        0x4u  /* do not return the mapping                       */
#define MCS_GRAPH_REPLAY      0x10u /* mcs_solve_batch_device only: capture this call's */
                                    /* launches in a CUDA graph and replay the graph   */
                                    /* when called again with identical arguments      */
#define MCS_NO_LEVEL_PRUNE    0x8u  /* diagnostic: do not re-test a level's bound      */
                                    /* before each sibling, so that with one searcher  */
                                    /* the node count equals the sequential recursion's */
#define MCS_WORD32            0x20u /* 32-bit node step: every graph of the call has at */
                                    /* most 32 vertices (others: MCS_ERR_ARG for that  */
                                    /* pair).  mcs_solve and mcs_solve_batch set it    */
                                    /* themselves when all graphs fit                  */
#define MCS_TOP_DOWN          0x40u /* top-down strategy (Section IV-A): goal-directed  */
                                    /* searches for min(n_G,n_H), one less, ... from  */
                                    /* the root until a goal is reached; the first    */
                                    /* goal reached is the optimum.  A time limit     */
                                    /* before that reports size 0 (MCS_TIMEOUT).      */
                                    /* mcs_solve and the batch calls; mcs_submit and  */
                                    /* MCS_ORDER_LEARNED: MCS_ERR_UNSUPPORTED.        */
#define MCS_ORDER_HR          0x100u /* static vertex order of Section IV-A instead of */
                                     /* the degree order: weakly connected components */
                                     /* (decreasing rows/columns ratio, then size),   */
                                     /* inside each a Hellerman-Rarick-style column   */
                                     /* order.  Exact either way.  Not with           */
                                     /* MCS_ORDER_LEARNED (MCS_ERR_ARG) or mcs_submit */
                                     /* (MCS_ERR_UNSUPPORTED).                        */
#define MCS_RESTART           0x200u /* randomized restarts (Section IV-A): once a    */
                                     /* pair's node count has doubled since its last  */
                                     /* new incumbent (and passed mcs_set_restart's   */
                                     /* minimum), one searcher puts every open branch */
                                     /* of its stack back in the work ring in a      */
                                     /* random order and starts afresh; the pending   */
                                     /* branches keep the record of what is left, so  */
                                     /* the result stays exact.  Not with             */
                                     /* MCS_TOP_DOWN / MCS_DEAD_END (MCS_ERR_ARG);    */
                                     /* with MCS_ORDER_LEARNED or in mcs_submit:      */
                                     /* MCS_ERR_UNSUPPORTED.                          */
#define MCS_WIDE              0x400u /* mcs_solve_batch_device: graphs of up to       */
                                     /* MCS_MAX_N vertices (four 64-bit words per     */
                                     /* vertex set); without it a graph of more than  */
                                     /* 64 vertices is MCS_ERR_ARG for its pair.      */
                                     /* Degree order only: with MCS_ORDER_LEARNED,     */
                                     /* MCS_ORDER_HR, MCS_TOP_DOWN, MCS_DEAD_END,      */
                                     /* MCS_RESTART or MCS_GRAPH_REPLAY the call is    */
                                     /* MCS_ERR_UNSUPPORTED (mcs_solve_batch reports   */
                                     /* it per pair for pairs over 64 vertices)        */
#define MCS_RACE              0x800u /* mcs_solve only: race the GPU search against a  */
                                     /* sequential CPU McSplit of the same pair on a   */
                                     /* host thread (the portfolio of Section IV with  */
                                     /* two contenders).  Each side publishes its best */
                                     /* size in host-mapped memory and prunes against  */
                                     /* the larger of the two; the first to finish its */
                                     /* proof stops the other, and the larger mapping  */
                                     /* is returned (exact).  Graphs of at most 64     */
                                     /* vertices, degree order; mcs_last_stats out[15] */
                                     /* tells which side finished first.  Other entry  */
                                     /* points, and other strategies: UNSUPPORTED.     */
#define MCS_DEAD_END          0x80u /* dead-end forecast (Section IV-A): after          */
                                    /* mcs_set_dead_end's threshold of nodes without  */
                                    /* a new incumbent, the pair's incumbent size is  */
                                    /* raised by one (or doubled); an unreachable     */
                                    /* raised value bounds the optimum, and a binary  */
                                    /* search of goal-directed searches from the root */
                                    /* closes the gap.  Exact.  Not with MCS_TOP_DOWN */
                                    /* (MCS_ERR_ARG); with MCS_ORDER_LEARNED or in    */
                                    /* mcs_submit: MCS_ERR_UNSUPPORTED.               */

typedef struct mcs_ctx mcs_ctx;

typedef struct {
    int32_t n;
    const uint8_t* adj;      /* n*n, row major, 0/1                               */
    const int32_t* labels;   /* n entries or NULL                                 */
} mcs_graph;

typedef struct {
    int32_t size;            /* |mapping|                                         */
    int32_t status;          /* MCS_OK, MCS_TIMEOUT or MCS_ERR_*                  */
    int32_t npairs;          /* entries written to g_idx/h_idx (== size)          */
    int32_t _pad;
    int16_t* g_idx;          /* caller-allocated, capacity >= min(nG, nH), or NULL */
    int16_t* h_idx;          /* same; pairs sorted by g_idx                        */
    uint64_t nodes;          /* search nodes expanded for this pair               */
    double seconds;          /* device time from the pair's start to its proof    */
} mcs_result;

/* Creates a context on CUDA device `device`: the state behind every solve
 * below (the paper's solver runs one search per process, Section III; a
 * context holds one CUDA stream and the device arenas of its searches).
 * flags: reserved, pass 0.  Returns NULL on failure (no device, allocation
 * failure). */
mcs_ctx* mcs_create(int device, uint32_t flags);
void mcs_destroy(mcs_ctx* ctx);

/* Solves one pair: a maximum common induced subgraph of G and H as defined
 * in Section II-A, found and proven by the branch and bound of Algorithm 1
 * (Section II-B) with the bound of Eq. 1.  out->size is its size and
 * out->g_idx / h_idx its vertex pairs (original numbering).  timeout_s <= 0
 * means no limit (an internal cap of one hour still bounds every device
 * wait).  Returns out->status. */
int mcs_solve(mcs_ctx* ctx, const mcs_graph* G, const mcs_graph* H,
              uint32_t flags, double timeout_s, mcs_result* out);

/* Solves npairs pairs (G[i], H[i]) -- each the problem of Section II-A by
 * Algorithm 1 and Eq. 1, as mcs_solve -- in one persistent launch.
 * timeout_s is per pair, counted from the moment the pair's search starts.
 * Returns the worst (lowest negative, else highest) per-pair status. */
int mcs_solve_batch(mcs_ctx* ctx, const mcs_graph* G, const mcs_graph* H,
                    int32_t npairs, uint32_t flags, double timeout_s,
                    mcs_result* out);

/* Device-resident batch (the problem of Section II-A by Algorithm 1 and
 * Eq. 1, as mcs_solve_batch): every pointer is a device pointer; nothing is
 * copied between host and device and the call does not synchronise.
 *   d_n[2p], d_n[2p+1]            vertex counts of G_p and H_p
 *   d_adj_off[2p], d_adj_off[2p+1] byte offsets of their matrices in d_adj
 *   d_lab_off[...]                 element offsets of their labels in d_labels
 *                                  (ignored when d_labels is NULL; an offset
 *                                  of -1 marks one graph as unlabelled)
 * Outputs (npairs entries each; d_map npairs*MCS_MAX_N, may be NULL):
 *   d_size, d_status, d_nodes, d_map, d_usec (device microseconds per pair,
 *   may be NULL).  `stream` is a cudaStream_t (NULL = the context's stream).
 * Invalid pairs get status MCS_ERR_ARG.  Returns 0 if the work was enqueued. */
int mcs_solve_batch_device(mcs_ctx* ctx, int32_t npairs,
                           const int32_t* d_n, const int64_t* d_adj_off,
                           const uint8_t* d_adj, const int64_t* d_lab_off,
                           const int32_t* d_labels, uint32_t flags, double timeout_s,
                           int32_t* d_size, int32_t* d_status, uint64_t* d_nodes,
                           int16_t* d_map, float* d_usec, void* stream);

/* Limits of mcs_solve_batch_noalloc's fixed scratch. */
#define MCS_NOALLOC_MAX_PAIRS     256
#define MCS_NOALLOC_MAX_WARPS     592
#define MCS_NOALLOC_SCRATCH_BYTES (26u << 20)   /* upper bound of the array, per device */

/* Device-resident batch solve that allocates nothing.  The paper has no
 * counterpart; this entry point exists for callers that cannot call
 * cudaMalloc -- for example code running while a stream is being captured
 * into a CUDA graph, a plug-in whose host framework owns all device memory,
 * or a latency-critical service that must not enter the allocator.
 *
 * Arguments, layouts and results are exactly those of
 * mcs_solve_batch_device, without the context; `stream` is a cudaStream_t
 * (NULL = the legacy default stream) and the call does not synchronise.  The
 * caller still owns every input and output buffer.  All scratch lives in one
 * file-scope device array of at most MCS_NOALLOC_SCRATCH_BYTES that every
 * GPU which loads the library holds until the process exits; the call makes
 * no cudaMalloc/cudaFree and uses no allocating library routine.
 *
 * Limits: at most MCS_NOALLOC_MAX_PAIRS pairs per call (more returns
 * MCS_ERR_ARG and enqueues nothing), at most MCS_NOALLOC_MAX_WARPS search
 * warps (one block of 4 warps per SM), and graphs of at most 64 vertices
 * (a larger one makes its pair MCS_ERR_ARG; MCS_WIDE: MCS_ERR_UNSUPPORTED).
 *
 * The first call on a device looks up the array's device address
 * (cudaGetSymbolAddress, with that device current) and caches it, and loads
 * every kernel variant the entry point can launch (any accepted flags) with
 * its shared-memory limit set; make that first call before any stream capture
 * begins.  MCS_ORDER_LEARNED is not available here (MCS_ERR_UNSUPPORTED).
 * Every call uses the same
 * array and overwrites what the previous call left there (the kernels
 * re-initialise all state they read), so calls whose executions overlap on
 * the GPU -- on different streams, or from different host threads on one
 * device -- race and must not be issued. */
int mcs_solve_batch_noalloc(int32_t npairs, const int32_t* d_n, const int64_t* d_adj_off,
                            const uint8_t* d_adj, const int64_t* d_lab_off,
                            const int32_t* d_labels, uint32_t flags, double timeout_s,
                            int32_t* d_size, int32_t* d_status, uint64_t* d_nodes,
                            int16_t* d_map, float* d_usec, void* stream);

/* ---- branching-order network (learned candidate order) ----------------
 * A small MLP scores candidate pairs (v, u) from vertex features (degree,
 * label, a 16-bin histogram of the neighbours' degrees) of v in G and u in H:
 * 36 inputs (zero-padded to 48) -> 128 -> 128 -> 1 logit, fp16 operands on
 * the tensor cores with fp32 accumulation.  With MCS_ORDER_LEARNED the solver
 * numbers vertices by their best score (most promising first) and tries the
 * candidates u of each chosen v in decreasing score.  This reorders McSplit's
 * choices only: every candidate is still tried and every bound (Eq. 1) is
 * still exact, so results stay optimal.  Without a loaded model the degree
 * order (Section IV-A) is used.
 * Parameter layout (float32): W1[48][128] (row = input), b1[128],
 * W2[128][128], b2[128], w3[128], b3[1]; inputs 36..47 of W1 must be 0. */
#define MCS_ORDER_NPARAMS 22913

/* Loads (copies) a model into the context; resets the optimiser state. */
int mcs_set_order_model(mcs_ctx* ctx, const float* params, int32_t nparams);
/* Copies the context's current model out (after training, for instance). */
int mcs_get_order_model(mcs_ctx* ctx, float* params, int32_t nparams);

/* Evaluates the model on a device-resident batch (layout of
 * mcs_solve_batch_device) and nrows device rows d_rows[r] = (pair, v, u) in
 * original vertex ids, labels d_y[r] in {0,1}, weights d_w[r] (or NULL = 1).
 * Host outputs, each optional: h_scores[nrows] logits; h_loss the mean
 * weighted binary cross-entropy with logits; h_grad[MCS_ORDER_NPARAMS] its
 * gradient; h_features[npairs][2][64][18] the vertex features.  Synchronous. */
int mcs_order_eval(mcs_ctx* ctx, int32_t npairs, const int32_t* d_n, const int64_t* d_adj_off,
                   const uint8_t* d_adj, const int64_t* d_lab_off, const int32_t* d_labels,
                   uint32_t flags, int32_t nrows, const int32_t* d_rows, const float* d_y,
                   const float* d_w, float* h_scores, float* h_loss, float* h_grad,
                   float* h_features);

/* Trains the loaded model on the device: `steps` Adam steps (lr, beta1 0.9,
 * beta2 0.999) on mini-batches of `batch` rows drawn with replacement by a
 * counter-based hash of (seed, step, i).  h_loss_per_step[steps] (optional)
 * receives each step's mean loss.  Synchronous. */
int mcs_order_train(mcs_ctx* ctx, int32_t npairs, const int32_t* d_n, const int64_t* d_adj_off,
                    const uint8_t* d_adj, const int64_t* d_lab_off, const int32_t* d_labels,
                    uint32_t flags, int32_t nrows, const int32_t* d_rows, const float* d_y,
                    const float* d_w, int32_t steps, int32_t batch, float lr, uint64_t seed,
                    float* h_loss_per_step);

/* Scores of every candidate pair of a device-resident batch (layout of
 * mcs_solve_batch_device) under the loaded model: d_scores[p][v][u]
 * (npairs x 64 x 64 floats, device memory owned by the caller) receives the
 * logit of (v, u) in original vertex ids for v < n_G(p), u < n_H(p); other
 * entries are not written.  This is the all-pairs pass that
 * MCS_ORDER_LEARNED runs before a search.  Asynchronous on `stream` (a
 * cudaStream_t; NULL = the context's stream).  MCS_ERR_ARG without a model. */
int mcs_order_score_grid(mcs_ctx* ctx, int32_t npairs, const int32_t* d_n, const int64_t* d_adj_off,
                         const uint8_t* d_adj, const int64_t* d_lab_off, const int32_t* d_labels,
                         uint32_t flags, float* d_scores, void* stream);

/* Serving: admit one request -- one pair, solved as in mcs_solve (Section
 * II-A, Algorithm 1, Eq. 1) -- and return its ticket.  The search starts on
 * the device as soon as a slot and device memory are free; requests
 * submitted while others run join them (continuous batching).  The paper
 * serves no request stream (its portfolio runs one instance at a time,
 * Section IV); this is the continuous-batching form of the same search.
 * Undirected requests with the degree order only (other flags:
 * MCS_ERR_UNSUPPORTED). */
int mcs_submit(mcs_ctx* ctx, const mcs_graph* G, const mcs_graph* H,
               uint32_t flags, double timeout_s, uint64_t* ticket);

/* Returns MCS_PENDING until the request finishes, then its status, and fills
 * `out` with its result (Section II-A: size and vertex pairs; mapping buffers
 * as in mcs_result).  A finished ticket is released by the first poll that
 * reports it.  A request lost by a failed server launch returns that
 * launch's error (MCS_ERR_DEVICE_STALL or MCS_ERR_CUDA) and is released. */
int mcs_poll(mcs_ctx* ctx, uint64_t ticket, mcs_result* out);

/* Launch shape used by every solve on this context: warps per block (1..8,
 * default 4), blocks per SM (default: as many as fit), class-stack entries
 * kept in shared memory per whole-warp searcher (default 256; narrower
 * searchers keep their class stacks in global memory and ignore it).  0
 * keeps the current value, -1 restores the default;
 * anything else out of range is MCS_ERR_ARG.  A shape whose shared memory
 * does not fit an SM makes the next solve return MCS_ERR_UNSUPPORTED. */
int mcs_set_launch(mcs_ctx* ctx, int warps_per_block, int blocks_per_sm,
                   int smem_stack_entries);

/* Restricts a solve to `warps` resident searchers in total (0 = the full
 * grid; a searcher is a group of mcs_set_search_group lanes, 8 by default).
 * With warps == 1 the search order is deterministic. */
int mcs_set_max_warps(mcs_ctx* ctx, int warps);

/* Work-sharing granularity of batch solves: a busy searcher checks every
 * poll_nodes search nodes (a power of two, 4..1024; default 16) whether a
 * searcher waits for work, and then hands over the upper part of the
 * candidates of its shallowest open level, keeping keep_quarters / 4 of them
 * (1..3; default 2, i.e. half; at least one).  0 keeps a value, -1 restores
 * its default; anything else is MCS_ERR_ARG.  Results do not depend on it. */
int mcs_set_steal(mcs_ctx* ctx, int poll_nodes, int keep_quarters);

/* Lanes per depth-first searcher of mcs_solve_batch[_device] (Section III's
 * data-parallel node step, Algorithm 1): 32 runs one search per warp with the
 * label classes of a node spread over the lanes; 16, 8, 4 or 2 run two to
 * sixteen independent searches per warp, each over its own lane group, for
 * instances whose nodes hold few classes (default 8).  Results are the same
 * for every value (the node counts of a multi-searcher solve vary as with any
 * work stealing).  Any other value: MCS_ERR_ARG.  Serving has its own
 * setting (mcs_set_serve_group). */
int mcs_set_search_group(mcs_ctx* ctx, int lanes);

/* How searchers narrower than a warp share it in plain batch solves
 * (mcs_solve_batch[_device], mcs_solve, without MCS_TOP_DOWN, MCS_DEAD_END or
 * MCS_RESTART):
 *   MCS_MODE_FREE (default): each searcher runs its own loop, and the warp
 *     serialises the searchers' diverging branches;
 *   MCS_MODE_LOCKSTEP: the searchers of a warp advance together, one node
 *     of each per pass (the "v unmatched" step and a child (v, u) are the
 *     same predicated split pass), so the warp issues one instruction
 *     stream for all of them.  Measured slower on the B300 (the searchers'
 *     memory waits add up instead of overlapping).
 * Results are the same either way (a lone searcher visits the same nodes).
 * Whole-warp searchers, goal-directed strategies and the server launch are
 * not affected.  MCS_ERR_ARG for other values. */
#define MCS_MODE_FREE      0
#define MCS_MODE_LOCKSTEP  1
int mcs_set_search_mode(mcs_ctx* ctx, int mode);

/* Lanes per searcher of the server launch behind mcs_submit / mcs_poll:
 * 32 (default; the best throughput and p50 latency measured on the
 * config-5 stream), 16 or 8.  The first warp of the server always admits
 * requests (it copies and packs each one).  Call before the first
 * mcs_submit on the context: MCS_ERR_UNSUPPORTED afterwards (unless the
 * value is unchanged); other values: MCS_ERR_ARG. */
int mcs_set_serve_group(mcs_ctx* ctx, int lanes);

/* MCS_DEAD_END parameters: threshold_nodes (>= 1; -1 restores the default
 * 2^22) is the number of search nodes of a pair, counted over all its
 * searchers at their polls, without a new incumbent before the incumbent size
 * is raised; doubling 1 doubles it, 0 (default) adds one, -1 restores the
 * default.  Applies to later calls.  MCS_ERR_ARG for other values. */
int mcs_set_dead_end(mcs_ctx* ctx, long long threshold_nodes, int doubling);

/* MCS_RESTART parameters: min_nodes (>= 1; -1 restores the default 2^20) is
 * the number of search nodes of a pair, counted over all its searchers at
 * their polls, before its first restart; seed selects the random order of the
 * spilled branches.  Applies to later calls.  MCS_ERR_ARG for other values. */
int mcs_set_restart(mcs_ctx* ctx, long long min_nodes, unsigned long long seed);

/* Statistics of the last solve on this context: out[0] search-kernel
 * microseconds (for mcs_solve_batch_device: once its stream has passed the
 * launch, else the previous value), out[1] total nodes (host API calls only),
 * out[2] donated tasks, out[3] donated tasks taken up, out[4] child levels
 * that spilled past the shared-memory class cache of whole-warp searchers (0
 * for searchers narrower than a warp, which keep the whole stack in global
 * memory),
 * out[5] searchers launched,
 * out[6] bytes copied host to device, out[7] bytes copied device to host
 * (out[6..7]: host API calls only), out[8] label classes read by node
 * expansions (the unit of algorithmic work), out[9] children cut by the bound
 * when created, out[10] / out[11] SM cycles summed over searchers while working /
 * waiting for work, out[12..14] index violations recorded by an
 * MCS_DEBUG_BOUNDS build (count, first code, first source line; 0 in
 * release builds), out[15] for an MCS_RACE solve the side that finished its
 * proof first (0 neither, 1 the CPU, 2 the GPU), out[16] the CPU side's
 * search nodes.  Returns the number of values written (<= n, <= 17). */
int mcs_last_stats(mcs_ctx* ctx, double* out, int n);

/* ---- failure injection (diagnostics; the paper has no counterpart) ------
 * Makes the library's failure paths run on demand in tests, without faulting
 * the GPU: every device-side wait of the search is bounded, and these hooks
 * make one of them run out, or make a host-side call fail as if the system
 * had refused it.  `value` applies to the context's later calls (a graph
 * captured by MCS_GRAPH_REPLAY keeps the values it was captured with); 0
 * turns a fault off.  Returns MCS_ERR_ARG for an unknown kind or a negative
 * value.
 *   MCS_FAULT_ALLOC          the value-th device or pinned-host allocation of a
 *                            batch solve from now fails once, as if out of
 *                            memory: that call returns MCS_ERR_NOMEM and the
 *                            next call allocates again
 *   MCS_FAULT_CUDA           the next `value` batch solves fail at their first
 *                            kernel launch with MCS_ERR_CUDA (nothing of that
 *                            call runs on the device; mcs_error_detail names it)
 *   MCS_FAULT_STALL_MS       limit, in milliseconds, of an idle searcher's wait
 *                            for work without progress anywhere in the launch
 *                            (default: the time limit + 2 s); also applies to
 *                            the server launch of mcs_submit
 *   MCS_FAULT_SPIN_LIMIT     iterations of a wait for a free work-ring slot
 *                            before it gives up (default 2^22)
 *   MCS_FAULT_WITHHOLD_EXIT  the searcher that ends a launch posts `value`
 *                            fewer exit tokens: as many searchers wait for work
 *                            that never comes until MCS_FAULT_STALL_MS expires
 *   MCS_FAULT_BLOCK_RING     1: work-ring slots other than the pair roots never
 *                            become free, so every hand-over of work waits
 *                            until MCS_FAULT_SPIN_LIMIT runs out
 * An expired wait makes the call (mcs_solve_batch, or mcs_poll for each
 * request of a failed server launch) return MCS_ERR_DEVICE_STALL; pairs that
 * finished before it keep their results, the others report MCS_PENDING; the
 * context stays usable. */
#define MCS_FAULT_ALLOC          1
#define MCS_FAULT_CUDA           2
#define MCS_FAULT_STALL_MS       3
#define MCS_FAULT_SPIN_LIMIT     4
#define MCS_FAULT_WITHHOLD_EXIT  5
#define MCS_FAULT_BLOCK_RING     6
int mcs_set_fault(mcs_ctx* ctx, int kind, long long value);

/* Micro-benchmark of the integer pipe the search is bound by: sustained
 * 32-bit population counts per second over the whole device (8 independent
 * chains per thread, 8 blocks of 256 threads per SM).  Not part of the
 * search; used as the measured roofline denominator. */
int mcs_bench_popc(mcs_ctx* ctx, double* popc_per_s);

const char* mcs_strerror(int code);

/* Detail of the last failing CUDA runtime call made by the library on the
 * calling host thread (error name, code, call), or "" if none failed. */
const char* mcs_error_detail(void);

#ifdef __cplusplus
}
#endif
#endif /* MCS_H_ */
