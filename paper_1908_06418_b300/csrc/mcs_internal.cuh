// Internal device-side layout of the B300 McSplit library (not installed;
// the public interface is include/mcs.h).
#pragma once
#include <cstdint>
#include <cuda_runtime.h>
#include <unordered_map>

namespace mcsk {

constexpr int kMaxN = 64;
constexpr int kLevels = kMaxN + 1;
// Classes on one warp's DFS stack: level d holds at most (64 - d) classes
// (they are disjoint and each keeps one unmatched G vertex), so the whole
// stack holds at most 64 + 63 + ... + 1 = 2080 entries.
constexpr int kStackMax = 2080 + 32;

typedef unsigned long long u64;

// Per-pair packed graph data, produced by the pack kernel (renumbered by the
// chosen vertex order; bit x of row v is vertex x in the new numbering).
// The out- and in-row of a vertex are adjacent (one 16-byte pair), so that the
// directed split reads one cache line per graph.
struct PairGraph {
    u64 rows[4 * kMaxN];   // G: rows[2v] bit x = arc v -> x, rows[2v + 1] bit x = arc x -> v
                           // (== the out-row when undirected); H: the same from 2 kMaxN
    ulonglong2 root[kMaxN];  // initial label classes (L mask, R mask)
    uint8_t permG[kMaxN];  // new number -> original number
    uint8_t permH[kMaxN];
    int32_t nG, nH, C0, valid;
    int32_t pad[4];
};

// Per-pair search state.
struct PairState {
    int32_t inc;           // incumbent size (atomicMax); starts at `floor`
    int32_t open;          // tasks of this pair that exist (queued or running)
    int32_t status;        // MCS_PENDING until finalised, or MCS_ERR_ARG
    int32_t abort;         // 0 running, 1 time limit hit, 2 goal reached (stop, optimal)
    u64 nodes;
    u64 t_start, deadline; // globaltimer ns
    u64 ticket;            // serve mode: the request's ticket
    u64 timeout_ns;        // serve mode: the request's limit (from its root's start)
    // Goal-directed search (top-down strategy, Section IV-A): only mappings
    // larger than `floor` are recorded, and the pair stops once the incumbent
    // reaches `cap`.  Plain search: floor 0, cap kNoCap.
    int32_t floor, cap;
    int32_t real;          // size of the largest recorded mapping (atomicMax)
    int32_t lo, hi;        // dead-end mode: bounds of the binary search over goals
    int32_t restarts;      // restart mode: restarts so far (part of the random order's counter)
    u64 dead;              // dead-end mode: nodes since the last new incumbent (approx.)
    u64 live, mark;        // restart mode: nodes so far and at the last new incumbent (approx.)
};
constexpr int32_t kNoCap = 1 << 30;

// A unit of work: one level of a pair's search tree (a node, its classes,
// the chosen left vertex v and the candidate set still to try).
constexpr int kTaskFresh = 1;      // node entry (bound + selection) still to do
constexpr int kTaskPending = 2;    // the "v stays unmatched" branch still to do
struct TaskHdr {
    int32_t pair, depth, C, v;
    u64 rrem;
    int32_t flags, bound;
    int32_t pad[2];
};
struct Task {
    TaskHdr h;                     // 40 -> padded to 48 below
    int32_t pad2[2];
    uint8_t Mg[kMaxN], Mh[kMaxN];  // the mapping prefix M (new numbering)
    ulonglong2 cls[kMaxN];
};
static_assert(sizeof(Task) % 16 == 0, "task slots must stay 16-byte aligned");

// Fields that different warps poll or update sit on separate 128-byte lines.
struct alignas(128) Control {
    u64 q_head, q_tail;            // ticket counters of the task ring
    u64 pad0[14];
    int32_t remaining;             // pairs not finalised
    int32_t error;                 // MCS_ERR_DEVICE_STALL if a bounded wait expired
    u64 last_progress;             // globaltimer ns of the last pair start/finish/donation
    u64 pad1[14];
    u64 donated, stolen, spilled;  // statistics (summed at warp exit)
    u64 class_visits;              // classes read by node expansions (algorithmic work units)
    u64 pruned;                    // children cut by the bound at creation
    u64 busy_cycles, idle_cycles;  // per-warp SM cycles with / waiting for work
    u64 pad2[9];
    // MCS_DEBUG_BOUNDS builds only: first index violation (code, value, source
    // line) and the number of violations; the offending access is skipped
    u64 dbg_code, dbg_val, dbg_line, dbg_count;
    u64 pad3[12];
};
static_assert(sizeof(Control) == 512, "one 128-byte line per group of fields");

// ---- serving (continuous batching) --------------------------------------
constexpr int kTaskPack = 4;       // root of a served request: copy + pack it first
constexpr int kSlotBytes = 2 * kMaxN * kMaxN + 2 * kMaxN * 4;   // adj G, adj H, labels G, H

// Request descriptor, written by the host into mapped pinned memory.
struct ServeReq {
    int32_t nG, nH;
    int32_t labelled;              // bit 0: G has labels, bit 1: H has labels
    int32_t flags;
    u64 ticket;
    u64 timeout_ns;
};
// Result record, written by the device into mapped pinned memory; `done`
// (the request's ticket) is written last, after a system-scope fence.
struct ServeRes {
    int32_t size, status;
    u64 nodes;
    float usec;
    int32_t pad;
    int16_t map[kMaxN];
    u64 done;
};
struct ServeDev {
    const u64* host_written;       // mapped: ring entries published by the host
    const int32_t* ring;           // mapped: slot of entry i % ring_cap
    int32_t ring_cap;
    int32_t nslots;
    const ServeReq* req;           // mapped [nslots]
    const uint8_t* hdata;          // mapped [nslots][kSlotBytes]
    uint8_t* ddata;                // device [nslots][kSlotBytes]
    ServeRes* res;                 // mapped [nslots]
    u64* dev_admitted;             // mapped: ring entries admitted by the device
    const int32_t* stop;           // mapped: host asks an idle server to exit
    int32_t* in_flight;            // device: admitted, unfinished requests
    u64 linger_ns;                 // idle time before the server exits
};

struct SearchParams {
    int32_t serving;               // 1: serve mode (requests arrive while the kernel runs)
    ServeDev sv;
    int32_t npairs;
    uint32_t flags;
    u64 timeout_ns;                // per pair
    u64 stall_ns;                  // idle-wait limit without any progress
    const PairGraph* graphs;
    PairState* state;
    uint16_t* best;                // [npairs][kLevels][kMaxN]: (g << 8) | h per size slot
    const int32_t* order;          // pair processing order (may be null)
    Control* ctl;
    Task* queue;
    u64* qseq;
    uint32_t qcap;                 // power of two
    int32_t stack_smem;            // class entries per warp kept in shared memory
    int32_t warp_smem_bytes;
    int32_t max_warps;             // searchers that take part (others exit at once)
    ulonglong2* gstack;            // per-warp overflow of the class stack
    const uint8_t* rank;           // learned order: [npairs][kMaxN][kMaxN] rank of u for v, or null
    uint32_t poll_mask;            // work sharing: poll every poll_mask + 1 nodes (power of two)
    int32_t steal_keep_q4;         // a donor keeps ceil(k * q / 4) of k candidates (1..3)
    u64 dead_nodes;                // MCS_DEAD_END: nodes without a new incumbent before a raise
    int32_t dead_double;           // MCS_DEAD_END: 1 doubles the incumbent size, 0 adds one
    u64 restart_min;               // MCS_RESTART: no restart before this many nodes of a pair
    u64 restart_seed;              // MCS_RESTART: seed of the random order of spilled branches
    int32_t lockstep;              // 1: searchers narrower than a warp advance in lockstep (plain batch mode)
    // GPU + CPU race (MCS_RACE; null otherwise): words in mapped host memory
    const volatile int32_t* race_cpu;   // best size found by the CPU search (read at polls)
    volatile int32_t* race_gpu;         // best size found here (written on each new incumbent)
    const volatile int32_t* race_stop;  // nonzero: the CPU search finished, stop
    // failure injection (mcs_set_fault; 0 in normal runs)
    uint32_t spin_limit;           // iterations of a ring-slot wait (0: kSpinLimit)
    int32_t withhold_exit;         // exit tokens not posted when a launch's last pair ends
    // outputs
    int32_t* out_size;
    int32_t* out_status;
    u64* out_nodes;
    int16_t* out_map;
    float* out_usec;
};

struct PackParams {
    int32_t npairs;
    uint32_t flags;
    const int32_t* n;
    const int64_t* adj_off;
    const uint8_t* adj;
    const int64_t* lab_off;
    const int32_t* labels;
    const float* vscore;           // optional per-vertex order key [npairs][2][kMaxN] (lower first)
    PairGraph* graphs;
    PairState* state;
    int32_t* out_size;
    int32_t* out_status;
    u64* out_nodes;
    int16_t* out_map;
    float* out_usec;
    Control* ctl;
    Task* queue;
    u64* qseq;
    uint32_t qcap;
    const int32_t* order;          // processing order of the pairs (may be null)
    int32_t block_ring;            // failure injection: non-root ring slots never become free
};

// Per-searcher shared memory layout (bytes from the searcher's base).  The
// pair's adjacency rows are copied into shared memory for whole-warp
// searchers; narrower searchers (several per warp) read them from global
// memory through the read-only cache, which leaves room for more of them.
constexpr int kSmAdjBytes = 4 * 64 * 8;          // gout, gin, hout, hin
__host__ __device__ constexpr bool adj_in_smem(int gs) { return gs == 32; }
__host__ __device__ constexpr int sm_adj_bytes(int gs) { return adj_in_smem(gs) ? kSmAdjBytes : 0; }
// Row indices in PairGraph::rows (and in a whole-warp searcher's shared copy).
__host__ __device__ constexpr int row_gout(int v) { return 2 * v; }
__host__ __device__ constexpr int row_gin(int v) { return 2 * v + 1; }
__host__ __device__ constexpr int row_hout(int u) { return 2 * kMaxN + 2 * u; }
__host__ __device__ constexpr int row_hin(int u) { return 2 * kMaxN + 2 * u + 1; }
// A searcher's levels: one 16-byte entry per depth d, {candidates still to
// try, info}, info = base | C << 16 | v << 24 | flags << 32 | bound << 40 |
// u << 48, where (v, u) is the pair matched at depth d once a deeper level
// exists (the mapping prefix M is read from these entries).
constexpr int kSmLvOff = 0;                      // 65 * 16 -> 1040 (offsets after the adjacency)
constexpr int kSmCycOff = 1040;                  // busy, idle cycles, clock mark, held ticket (4 x 8)
constexpr int kSmClsOff = 1072;                  // 16-byte aligned
static_assert(kSmClsOff % 16 == 0 && kSmAdjBytes % 16 == 0, "class cache must be 16-byte aligned");

// Searchers of at most 4 lanes (8 or more per warp, up to 256 per SM) keep
// their level arrays in their global region as well, after the class stack.
__host__ __device__ constexpr bool levels_in_smem(int gs) { return gs >= 8; }
constexpr int kLvEntries = 80;                   // 1,280 B >= kSmClsOff: level entries in global

inline int warp_smem_bytes(int stack_entries, int gs = 32) {
    return sm_adj_bytes(gs) + (levels_in_smem(gs) ? kSmClsOff : 0) + 16 * stack_entries;
}
// 16-byte entries of a searcher's global region: class-stack overflow, plus
// the level arrays of searchers that keep none in shared memory.
inline size_t gstack_entries(int stack_entries, int gs) {
    return (size_t)(kStackMax > stack_entries ? kStackMax - stack_entries : 0) +
           (levels_in_smem(gs) ? 0 : (size_t)kLvEntries);
}

}  // namespace mcsk

struct MlpState;
struct ServeState;

// Device arenas of the path for graphs of 65 to 256 vertices (mcs_wide.cu),
// one set per word count (2 or 4 words per vertex set).
struct WideArena {
    void* graphs = nullptr; size_t graphs_cap = 0;
    void* state = nullptr;  size_t state_cap = 0;
    void* best = nullptr;   size_t best_cap = 0;
    void* queue = nullptr;  size_t queue_cap = 0;
    void* qseq = nullptr;   size_t qseq_cap = 0;
    void* gstack = nullptr; size_t gstack_cap = 0;
    void* ctl = nullptr;    size_t ctl_cap = 0;
};

// Host-side context behind the opaque mcs_ctx handle of include/mcs.h.
struct mcs_ctx {
    typedef mcsk::u64 u64;
    typedef mcsk::PairGraph PairGraph;
    typedef mcsk::PairState PairState;
    typedef mcsk::Control Control;
    typedef mcsk::Task Task;
    int device = 0;
    cudaStream_t stream = nullptr;
    int sms = 0;
    int warps_per_block = 4;
    int blocks_per_sm = 0;        // 0: as many as fit
    int smem_stack = 0;           // class entries per searcher in shared memory (0: default)
    int max_warps = 0;            // 0: every launched searcher
    int group_lanes = 8;          // lanes per searcher of batch solves: 32, 16, 8, 4 or 2
    int serve_lanes = 32;         // lanes per searcher of the server launch: 32, 16 or 8
    int poll_nodes = 16;          // work-sharing poll interval (nodes, power of two)
    int steal_keep_q4 = 2;        // quarters of a donated level's candidates the donor keeps
    int lockstep = 0;             // 1: plain batch searchers narrower than a warp run in lockstep
    long long dead_nodes = 1LL << 22;   // MCS_DEAD_END: nodes without a new incumbent before a raise
    int dead_double = 0;          // MCS_DEAD_END: 1 doubles the incumbent size, 0 adds one
    long long restart_min = 1LL << 20;   // MCS_RESTART: nodes of a pair before its first restart
    unsigned long long restart_seed = 0; // MCS_RESTART: seed of the random branch order
    // resident blocks per SM of each launch configuration already asked of the
    // driver (key: warps per block, shared memory per block, kernel variant)
    std::unordered_map<uint64_t, int> occupancy;
    // device arenas
    int pairs_cap = 0;
    PairGraph* graphs = nullptr;
    PairState* state = nullptr;
    uint16_t* best = nullptr;
    int32_t* order = nullptr;
    Control* ctl = nullptr;
    Task* queue = nullptr;
    u64* qseq = nullptr;
    uint32_t qcap = 0;
    ulonglong2* gstack = nullptr;
    size_t gstack_entries = 0;
    // host-API staging
    uint8_t* d_in = nullptr;  size_t d_in_cap = 0;
    uint8_t* h_in = nullptr;  size_t h_in_cap = 0;
    uint8_t* d_out = nullptr; size_t d_out_cap = 0;
    uint8_t* h_out = nullptr; size_t h_out_cap = 0;
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    double stats[17] = {0};
    bool ev_pending = false;       // ev0/ev1 recorded by a device call, not yet read
    Control h_ctl;
    struct MlpState* mlp = nullptr;   // ordering network (mcs_mlp.cu), created on first use
    struct ServeState* serve = nullptr; // serving (mcs_serve.cu), created on first mcs_submit
    // MCS_GRAPH_REPLAY: one captured batch (its arguments and executable graph)
    cudaGraphExec_t graph_exec = nullptr;
    cudaGraph_t graph = nullptr;
    uint64_t graph_key[16] = {0};
    // graphs of 65 to 256 vertices (mcs_wide.cu)
    WideArena wide[2];
    void* wide_ctl = nullptr;      // control block of the last wide launch
    bool last_wide = false;        // the last device batch ran on the multi-word path
    // GPU + CPU race (MCS_RACE): three words of mapped host memory -- the CPU
    // side's best size, the GPU side's, and the stop flag -- and their device views
    int32_t* race_words = nullptr;
    int32_t* race_words_dev = nullptr;
    bool race_on = false;          // set while a racing solve is in flight
    // failure injection (mcs_set_fault): test hooks, all 0 in normal use
    long long fault_alloc_at = 0;  // the fault_alloc_at-th allocation from now fails (once)
    int fault_cuda = 0;            // solve calls still to fail at the API boundary
    long long fault_stall_ms = 0;  // idle-wait limit override
    long long fault_spin = 0;      // ring-slot wait limit override (iterations)
    int fault_withhold = 0;        // exit tokens withheld at the end of a launch
    int fault_block_ring = 0;      // ring slots other than the roots never free up
};

// Failure injection: true when the allocation about to be made must fail.
inline bool fault_alloc_now(mcs_ctx* c) {
    if (c->fault_alloc_at <= 0) return false;
    return --c->fault_alloc_at == 0;
}

// Work-sharing defaults for launches that do not take them from a context.
constexpr uint32_t kPollMaskDefault = 15;
constexpr int32_t kStealKeepDefault = 2;

// Class-stack entries per searcher kept in shared memory: for whole-warp
// searchers the value set by mcs_set_launch, else 256; narrower searchers
// keep their class stacks in global memory (0).
inline int stack_entries(const mcs_ctx* c, int gs) {
    if (gs != 32) return 0;
    return c->smem_stack > 0 ? c->smem_stack : 256;
}

// kernels.cu entry points used by the host library
namespace mcsk {
cudaError_t launch_pack(const PackParams& p, cudaStream_t s);
// gs: lanes per searcher (32: one search per warp; 16, 8, 4 or 2: two to sixteen)
cudaError_t launch_search(const SearchParams& p, int blocks, int warps_per_block,
                          bool directed, bool learned, cudaStream_t s, int gs = 32);
int search_max_blocks_per_sm(int warps_per_block, int smem_per_block, bool directed, bool learned,
                             int gs = 32, bool narrow = false);
int serve_max_blocks_per_sm(int warps_per_block, int smem_per_block, int gs);
// Loads the pack kernel and every whole-warp, degree-order batch
// instantiation of the search kernel (both word widths, directed or not,
// plain and goal-directed) on the current device and sets their dynamic
// shared-memory limit to smem, so that later launches make no loading or
// attribute call.
cudaError_t warm_batch_variants(int smem);
cudaError_t launch_popc_bench(unsigned long long* out, int blocks, int iters, cudaStream_t s);
cudaError_t launch_serve_init(Control* ctl, u64* qseq, uint32_t qcap, int32_t* in_flight, int block_ring,
                              cudaStream_t s);
}

// mcs_mlp.cu: learned candidate order
int mcs_order_prepare(mcs_ctx* c, int npairs, const int32_t* d_n, const int64_t* d_adj_off,
                      const uint8_t* d_adj, const int64_t* d_lab_off, const int32_t* d_labels,
                      uint32_t flags, cudaStream_t s, const float** vscore_out);
int mcs_order_ranks(mcs_ctx* c, int npairs, cudaStream_t s, const uint8_t** rank_out);
void mcs_order_free(mcs_ctx* c);
// mcs_serve.cu
void mcs_serve_free(mcs_ctx* c);
// mcs_wide.cu: pairs of up to 256 vertices per graph
int wide_run_device(mcs_ctx* c, int npairs, const int32_t* d_n, const int64_t* d_adj_off, const uint8_t* d_adj,
                    const int64_t* d_lab_off, const int32_t* d_labels, const int32_t* d_order, uint32_t flags,
                    double timeout_s, int max_n, int max_min_n, int32_t* d_size, int32_t* d_status,
                    uint64_t* d_nodes, int16_t* d_map, float* d_usec, cudaStream_t s, bool timed);
void wide_free(mcs_ctx* c);
