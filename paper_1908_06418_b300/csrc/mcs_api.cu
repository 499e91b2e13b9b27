// Host side of the C ABI declared in include/mcs.h.
//
// A context owns one CUDA stream, grow-only device arenas (packed graphs,
// per-pair state, incumbent mapping slots, the task ring, per-warp stack
// overflow) and pinned staging buffers.  A synchronous batch solve is:
//   one pinned H2D copy of the packed inputs -> pack_kernel -> search_kernel
//   -> one D2H copy of the results.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>
#include <numeric>
#include <vector>

#include <atomic>
#include <thread>

#include "mcs_cpu.h"
#include "mcs_internal.cuh"
#include "../../include/mcs.h"

using namespace mcsk;


namespace {

thread_local char g_detail[256] = "";

int cuda_fail(cudaError_t e, const char* what, int line) {
    snprintf(g_detail, sizeof(g_detail), "%s (%d) at mcs_api.cu:%d: %s", cudaGetErrorName(e), (int)e,
             line, what);
    if (e == cudaErrorMemoryAllocation) return MCS_ERR_NOMEM;
    return MCS_ERR_CUDA;
}
#define CK(x) do { cudaError_t _e = (x); if (_e != cudaSuccess) return cuda_fail(_e, #x, __LINE__); } while (0)

size_t align16(size_t x) { return (x + 15) & ~(size_t)15; }

// Every allocation of the batch path goes through these two, so that a test
// can make any one of them fail (mcs_set_fault, MCS_FAULT_ALLOC).
int dev_alloc(mcs_ctx* c, void** p, size_t n) {
    *p = nullptr;
    if (fault_alloc_now(c)) {
        snprintf(g_detail, sizeof(g_detail), "cudaMalloc(%zu): injected allocation failure", n);
        return MCS_ERR_NOMEM;
    }
    cudaError_t e = cudaMalloc(p, n);
    if (e != cudaSuccess) { *p = nullptr; cudaGetLastError(); return cuda_fail(e, "cudaMalloc", __LINE__); }
    return 0;
}
int host_alloc(mcs_ctx* c, void** p, size_t n) {
    *p = nullptr;
    if (fault_alloc_now(c)) {
        snprintf(g_detail, sizeof(g_detail), "cudaMallocHost(%zu): injected allocation failure", n);
        return MCS_ERR_NOMEM;
    }
    cudaError_t e = cudaMallocHost(p, n);
    if (e != cudaSuccess) { *p = nullptr; cudaGetLastError(); return cuda_fail(e, "cudaMallocHost", __LINE__); }
    return 0;
}

template <typename T>
int grow_dev(mcs_ctx* c, T*& p, size_t& cap, size_t need) {
    if (need <= cap && p) return 0;
    size_t n = std::max(need, cap * 3 / 2);
    if (p) cudaFree(p);
    p = nullptr;
    cap = 0;
    int rc = dev_alloc(c, (void**)&p, n);
    if (rc) return rc;
    cap = n;
    return 0;
}
template <typename T>
int grow_host(mcs_ctx* c, T*& p, size_t& cap, size_t need) {
    if (need <= cap && p) return 0;
    if (p) cudaFreeHost(p);
    p = nullptr;
    cap = 0;
    int rc = host_alloc(c, (void**)&p, need);
    if (rc) return rc;
    cap = need;
    return 0;
}

int launch_shape(mcs_ctx* c, bool directed, bool learned, bool narrow, int* blocks, int* warps_total,
                 int* wsmem) {
    // warps_total counts searchers: 32 / group_lanes of them share a warp
    const int spb = c->warps_per_block * (32 / c->group_lanes);
    *wsmem = warp_smem_bytes(stack_entries(c, c->group_lanes), c->group_lanes);
    int smem_block = spb * *wsmem;
    const uint64_t key = (uint64_t)c->warps_per_block | ((uint64_t)smem_block << 8) |
                         ((uint64_t)c->group_lanes << 40) | ((uint64_t)directed << 48) |
                         ((uint64_t)learned << 49) | ((uint64_t)narrow << 50);
    auto it = c->occupancy.find(key);
    int per_sm;
    if (it != c->occupancy.end()) {
        per_sm = it->second;
    } else {
        per_sm = search_max_blocks_per_sm(c->warps_per_block, smem_block, directed, learned, c->group_lanes,
                                          narrow);
        c->occupancy[key] = per_sm;
    }
    if (per_sm <= 0) return MCS_ERR_UNSUPPORTED;
    if (c->blocks_per_sm > 0) per_sm = std::min(per_sm, c->blocks_per_sm);
    *blocks = c->sms * per_sm;
    *warps_total = *blocks * spb;
    if (c->max_warps > 0) {
        int need_blocks = (c->max_warps + spb - 1) / spb;
        *blocks = std::min(*blocks, need_blocks);
        *warps_total = std::min(*warps_total, c->max_warps);
    }
    return 0;
}

int ensure_pairs(mcs_ctx* c, int npairs) {
    if (npairs <= c->pairs_cap) return 0;
    int n = std::max(npairs, c->pairs_cap * 3 / 2);
    cudaFree(c->graphs); cudaFree(c->state); cudaFree(c->best); cudaFree(c->order);
    c->graphs = nullptr; c->state = nullptr; c->best = nullptr; c->order = nullptr;
    c->pairs_cap = 0;
    int rc;
    if ((rc = dev_alloc(c, (void**)&c->graphs, sizeof(PairGraph) * (size_t)n)) ||
        (rc = dev_alloc(c, (void**)&c->state, sizeof(PairState) * (size_t)n)) ||
        (rc = dev_alloc(c, (void**)&c->best, sizeof(uint16_t) * (size_t)n * kLevels * kMaxN)) ||
        (rc = dev_alloc(c, (void**)&c->order, sizeof(int32_t) * (size_t)n)))
        return rc;
    c->pairs_cap = n;
    return 0;
}

int ensure_ring(mcs_ctx* c, int warps, int npairs) {
    // the roots of every pair + at most one outstanding ticket per warp, with slack
    uint32_t q = 1024;
    while (q < (uint32_t)(4 * warps + npairs)) q <<= 1;
    int rc;
    if (q > c->qcap) {
        cudaFree(c->queue); cudaFree(c->qseq);
        c->queue = nullptr; c->qseq = nullptr; c->qcap = 0;
        if ((rc = dev_alloc(c, (void**)&c->queue, sizeof(Task) * (size_t)q)) ||
            (rc = dev_alloc(c, (void**)&c->qseq, sizeof(u64) * (size_t)q)))
            return rc;
        c->qcap = q;
    }
    const size_t per = gstack_entries(stack_entries(c, c->group_lanes), c->group_lanes);
    size_t need = per * (size_t)warps;
    if (need > c->gstack_entries || !c->gstack) {
        cudaFree(c->gstack);
        c->gstack = nullptr;
        c->gstack_entries = 0;
        if ((rc = dev_alloc(c, (void**)&c->gstack, sizeof(ulonglong2) * std::max<size_t>(need, 1))))
            return rc;
        c->gstack_entries = std::max<size_t>(need, 1);
    }
    if (!c->ctl && (rc = dev_alloc(c, (void**)&c->ctl, sizeof(Control)))) return rc;
    return 0;
}

// Enqueues pack + search for a device-resident batch.
int run_device(mcs_ctx* c, int npairs, const int32_t* d_n, const int64_t* d_adj_off,
               const uint8_t* d_adj, const int64_t* d_lab_off, const int32_t* d_labels,
               const int32_t* d_order, uint32_t flags, double timeout_s, int32_t* d_size,
               int32_t* d_status, uint64_t* d_nodes, int16_t* d_map, float* d_usec,
               cudaStream_t s, bool timed) {
    if (npairs < 0) return MCS_ERR_ARG;
    // the two goal-directed strategies of Section IV-A are alternatives
    if ((flags & MCS_TOP_DOWN) && (flags & MCS_DEAD_END)) return MCS_ERR_ARG;
    if ((flags & MCS_RESTART) && (flags & (MCS_TOP_DOWN | MCS_DEAD_END))) return MCS_ERR_ARG;
    // one vertex order per call
    if ((flags & MCS_ORDER_HR) && (flags & MCS_ORDER_LEARNED)) return MCS_ERR_ARG;
    // goal-directed searches are compiled for the degree (or static) order only
    if ((flags & (MCS_TOP_DOWN | MCS_DEAD_END | MCS_RESTART)) && (flags & MCS_ORDER_LEARNED))
        return MCS_ERR_UNSUPPORTED;
    if (npairs == 0) return 0;
    const bool directed = (flags & MCS_DIRECTED) != 0;
    int rc = 0;
    // learned candidate order: scores of every (v, u), order keys for the
    // renumbering; without a loaded model the degree order is kept
    const float* vscore = nullptr;
    bool learned = false;
    if (flags & MCS_ORDER_LEARNED) {
        if ((rc = ensure_pairs(c, npairs))) return rc;
        rc = mcs_order_prepare(c, npairs, d_n, d_adj_off, d_adj, d_lab_off, d_labels, flags, s, &vscore);
        if (rc < 0) return rc;
        learned = (rc == 0);
        rc = 0;
    }
    int blocks = 0, warps = 0, wsmem = 0;
    rc = launch_shape(c, directed, learned, (flags & MCS_WORD32) != 0, &blocks, &warps, &wsmem);
    if (rc) return rc;
    if ((rc = ensure_pairs(c, npairs))) return rc;
    if ((rc = ensure_ring(c, warps, npairs))) return rc;

    PackParams pp;
    memset(&pp, 0, sizeof(pp));
    pp.npairs = npairs;
    pp.flags = flags;
    pp.n = d_n;
    pp.adj_off = d_adj_off;
    pp.adj = d_adj;
    pp.lab_off = d_lab_off;
    pp.labels = d_labels;
    pp.vscore = vscore;
    pp.graphs = c->graphs;
    pp.state = c->state;
    pp.out_size = d_size;
    pp.out_status = d_status;
    pp.out_nodes = reinterpret_cast<u64*>(d_nodes);
    pp.out_map = (flags & MCS_NO_MAPPING) ? nullptr : d_map;
    pp.out_usec = d_usec;
    pp.ctl = c->ctl;
    pp.queue = c->queue;
    pp.qseq = c->qseq;
    pp.qcap = c->qcap;
    pp.order = d_order;
    pp.block_ring = c->fault_block_ring;
    if (c->fault_cuda > 0) {
        // failure injection: this call's first launch fails at the API boundary
        --c->fault_cuda;
        return cuda_fail(cudaErrorLaunchFailure, "launch_pack (injected failure)", __LINE__);
    }
    CK(launch_pack(pp, s));
    const uint8_t* rank = nullptr;
    if (learned && (rc = mcs_order_ranks(c, npairs, s, &rank))) return rc;

    double tmo = timeout_s > 0 ? std::min(timeout_s, 3600.0) : 3600.0;
    SearchParams sp;
    memset(&sp, 0, sizeof(sp));
    sp.npairs = npairs;
    sp.flags = flags;
    sp.timeout_ns = (u64)(tmo * 1e9);
    sp.stall_ns = c->fault_stall_ms > 0 ? (u64)c->fault_stall_ms * 1000000ull : sp.timeout_ns + 2000000000ull;
    sp.spin_limit = (uint32_t)c->fault_spin;
    sp.withhold_exit = c->fault_withhold;
    sp.graphs = c->graphs;
    sp.state = c->state;
    sp.best = c->best;
    sp.order = d_order;
    sp.ctl = c->ctl;
    sp.queue = c->queue;
    sp.qseq = c->qseq;
    sp.qcap = c->qcap;
    sp.stack_smem = stack_entries(c, c->group_lanes);
    sp.warp_smem_bytes = wsmem;
    sp.max_warps = warps;
    sp.gstack = c->gstack;
    sp.rank = rank;
    sp.poll_mask = (uint32_t)c->poll_nodes - 1;
    sp.steal_keep_q4 = c->steal_keep_q4;
    sp.lockstep = c->race_on ? 0 : c->lockstep;
    if (c->race_on) {
        sp.race_cpu = c->race_words_dev;
        sp.race_gpu = c->race_words_dev + 1;
        sp.race_stop = c->race_words_dev + 2;
    }
    sp.dead_nodes = (u64)c->dead_nodes;
    sp.dead_double = c->dead_double;
    sp.restart_min = (u64)c->restart_min;
    sp.restart_seed = (u64)c->restart_seed;
    sp.out_size = d_size;
    sp.out_status = d_status;
    sp.out_nodes = reinterpret_cast<u64*>(d_nodes);
    sp.out_map = (flags & MCS_NO_MAPPING) ? nullptr : d_map;
    sp.out_usec = d_usec;
    if (timed) CK(cudaEventRecord(c->ev0, s));
    CK(launch_search(sp, blocks, c->warps_per_block, directed, learned, s, c->group_lanes));
    if (timed) CK(cudaEventRecord(c->ev1, s));
    c->stats[5] = warps;
    return 0;
}

struct HostLayout {
    size_t off_n, off_adjoff, off_laboff, off_order, off_labels, off_adj, total;
};

int check_graph(const mcs_graph* g) {
    if (!g) return MCS_ERR_ARG;
    if (g->n < 0 || g->n > MCS_MAX_N) return MCS_ERR_ARG;
    if (g->n > 0 && !g->adj) return MCS_ERR_ARG;
    return 0;
}

int worst(int a, int b) {
    if (a < 0 || b < 0) return std::min(a, b);
    return std::max(a, b);
}

// GPU + CPU race on one pair (MCS_RACE; the portfolio idea of Section IV):
// the GPU search runs as an ordinary one-pair batch while a host thread runs
// the CPU McSplit of mcs_cpu.cpp on the same pair.  The two share the
// incumbent through single-writer words of mapped host memory (each side
// prunes against the larger size), and the first to finish its proof stops
// the other.  The result is the larger of the two mappings; it is proven
// when either side finished (its proof covers every mapping larger than the
// sizes it pruned against, and those sizes were found by one of the two).
int solve_race(mcs_ctx* c, const mcs_graph* G, const mcs_graph* H, uint32_t flags, double timeout_s,
               mcs_result* out) {
    if (check_graph(G) || check_graph(H)) return MCS_ERR_ARG;
    if (G->n > kMaxN || H->n > kMaxN ||
        (flags & (MCS_ORDER_LEARNED | MCS_ORDER_HR | MCS_TOP_DOWN | MCS_DEAD_END | MCS_RESTART)))
        return MCS_ERR_UNSUPPORTED;
    if (cudaSetDevice(c->device) != cudaSuccess) return MCS_ERR_CUDA;
    if (!c->race_words) {
        void* h = nullptr;
        if (cudaHostAlloc(&h, 64, cudaHostAllocMapped | cudaHostAllocPortable) != cudaSuccess) {
            cudaGetLastError();
            return MCS_ERR_NOMEM;
        }
        void* d = nullptr;
        if (cudaHostGetDevicePointer(&d, h, 0) != cudaSuccess) {
            cudaGetLastError();
            cudaFreeHost(h);
            return MCS_ERR_CUDA;
        }
        c->race_words = (int32_t*)h;
        c->race_words_dev = (int32_t*)d;
    }
    volatile int32_t* w = c->race_words;
    w[0] = 0; w[1] = 0; w[2] = 0;
    std::atomic_thread_fence(std::memory_order_seq_cst);
    CpuRaceResult cres;
    memset(&cres, 0, sizeof(cres));
    std::chrono::steady_clock::time_point t_cpu{};
    std::thread cpu([&]() {
        cpu_mcs_race(G->n, G->adj, G->labels, H->n, H->adj, H->labels, (flags & MCS_DIRECTED) != 0, timeout_s,
                     w + 1, w + 0, w + 2, &cres);
        t_cpu = std::chrono::steady_clock::now();
        if (cres.complete) w[2] = 1;                   // proof done: stop the GPU side
    });
    int16_t gi[kMaxN], hi[kMaxN];
    mcs_result gres;
    memset(&gres, 0, sizeof(gres));
    gres.g_idx = gi;
    gres.h_idx = hi;
    c->race_on = true;
    const int rc = mcs_solve_batch(c, G, H, 1, flags, timeout_s, &gres);
    c->race_on = false;
    const auto t_gpu = std::chrono::steady_clock::now();
    w[2] = 1;                                          // stop the CPU side
    cpu.join();
    if (rc < 0 && rc != MCS_ERR_ARG) return rc;
    if (gres.status == MCS_ERR_ARG) { *out = gres; return MCS_ERR_ARG; }
    const bool gpu_done = gres.status == MCS_OK;
    const bool cpu_done = cres.complete;
    const bool cpu_larger = cres.size > gres.size;
    out->size = cpu_larger ? cres.size : gres.size;
    out->status = (gpu_done || cpu_done) ? MCS_OK : MCS_TIMEOUT;
    out->nodes = gres.nodes + cres.nodes;
    out->seconds = gres.seconds;
    // the mapping of the larger side, sorted by G vertex
    std::vector<std::pair<int, int>> m;
    if (cpu_larger) for (int i = 0; i < cres.size; ++i) m.push_back({cres.g[i], cres.h[i]});
    else for (int i = 0; i < gres.npairs; ++i) m.push_back({gi[i], hi[i]});
    std::sort(m.begin(), m.end());
    out->npairs = (flags & MCS_NO_MAPPING) ? 0 : (int)m.size();
    if (!(flags & MCS_NO_MAPPING))
        for (size_t i = 0; i < m.size(); ++i) {
            if (out->g_idx) out->g_idx[i] = (int16_t)m[i].first;
            if (out->h_idx) out->h_idx[i] = (int16_t)m[i].second;
        }
    // which side finished its proof first (0 neither, 1 the CPU, 2 the GPU)
    int winner = 0;
    if (cpu_done && (!gpu_done || t_cpu < t_gpu)) winner = 1;
    else if (gpu_done) winner = 2;
    c->stats[15] = winner;
    c->stats[16] = (double)cres.nodes;
    return out->status;
}

}  // namespace

extern "C" {

mcs_ctx* mcs_create(int device, uint32_t flags) {
    (void)flags;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) return nullptr;
    if (cudaSetDevice(device) != cudaSuccess) return nullptr;
    mcs_ctx* c = new (std::nothrow) mcs_ctx();
    if (!c) return nullptr;
    c->device = device;
    cudaDeviceProp prop;
    if (cudaGetDeviceProperties(&prop, device) != cudaSuccess) { delete c; return nullptr; }
    c->sms = prop.multiProcessorCount;
    if (cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreate(&c->ev0) != cudaSuccess || cudaEventCreate(&c->ev1) != cudaSuccess) {
        mcs_destroy(c);
        return nullptr;
    }
    return c;
}

void mcs_destroy(mcs_ctx* c) {
    if (!c) return;
    cudaSetDevice(c->device);
    if (c->stream) cudaStreamSynchronize(c->stream);
    mcs_serve_free(c);
    mcs_order_free(c);
    wide_free(c);
    if (c->graph_exec) cudaGraphExecDestroy(c->graph_exec);
    if (c->graph) cudaGraphDestroy(c->graph);
    cudaFree(c->graphs); cudaFree(c->state); cudaFree(c->best); cudaFree(c->order);
    cudaFree(c->ctl); cudaFree(c->queue); cudaFree(c->qseq); cudaFree(c->gstack);
    cudaFree(c->d_in); cudaFree(c->d_out);
    if (c->h_in) cudaFreeHost(c->h_in);
    if (c->race_words) cudaFreeHost(c->race_words);
    if (c->h_out) cudaFreeHost(c->h_out);
    if (c->ev0) cudaEventDestroy(c->ev0);
    if (c->ev1) cudaEventDestroy(c->ev1);
    if (c->stream) cudaStreamDestroy(c->stream);
    delete c;
}

int mcs_set_launch(mcs_ctx* c, int warps_per_block, int blocks_per_sm, int smem_stack_entries) {
    if (!c) return MCS_ERR_ARG;
    if (warps_per_block < -1 || warps_per_block > 8 || blocks_per_sm < -1 || smem_stack_entries < -1 ||
        smem_stack_entries > kStackMax)
        return MCS_ERR_ARG;
    // 0 keeps the current value, -1 restores the default
    if (warps_per_block) c->warps_per_block = warps_per_block > 0 ? warps_per_block : 4;
    if (blocks_per_sm) c->blocks_per_sm = blocks_per_sm > 0 ? blocks_per_sm : 0;
    if (smem_stack_entries) c->smem_stack = smem_stack_entries > 0 ? smem_stack_entries : 0;
    return 0;
}

int mcs_set_steal(mcs_ctx* c, int poll_nodes, int keep_quarters) {
    if (!c) return MCS_ERR_ARG;
    const bool pow2 = poll_nodes > 0 && (poll_nodes & (poll_nodes - 1)) == 0;
    if (!(poll_nodes == 0 || poll_nodes == -1 || (pow2 && poll_nodes >= 4 && poll_nodes <= 1024)))
        return MCS_ERR_ARG;
    if (keep_quarters < -1 || keep_quarters > 3) return MCS_ERR_ARG;
    if (poll_nodes) c->poll_nodes = poll_nodes > 0 ? poll_nodes : (int)kPollMaskDefault + 1;
    if (keep_quarters) c->steal_keep_q4 = keep_quarters > 0 ? keep_quarters : kStealKeepDefault;
    return 0;
}

int mcs_set_dead_end(mcs_ctx* c, long long threshold_nodes, int doubling) {
    if (!c || threshold_nodes == 0 || threshold_nodes < -1 || doubling < -1 || doubling > 1) return MCS_ERR_ARG;
    c->dead_nodes = threshold_nodes > 0 ? threshold_nodes : (1LL << 22);
    c->dead_double = doubling > 0 ? 1 : 0;
    return 0;
}

int mcs_set_restart(mcs_ctx* c, long long min_nodes, unsigned long long seed) {
    if (!c || min_nodes == 0 || min_nodes < -1) return MCS_ERR_ARG;
    c->restart_min = min_nodes > 0 ? min_nodes : (1LL << 20);
    c->restart_seed = seed;
    return 0;
}

int mcs_set_serve_group(mcs_ctx* c, int lanes) {
    if (!c || (lanes != 8 && lanes != 16 && lanes != 32)) return MCS_ERR_ARG;
    if (c->serve) return lanes == c->serve_lanes ? 0 : MCS_ERR_UNSUPPORTED;   // the server exists
    c->serve_lanes = lanes;
    return 0;
}

int mcs_set_search_group(mcs_ctx* c, int lanes) {
    if (!c || (lanes != 2 && lanes != 4 && lanes != 8 && lanes != 16 && lanes != 32)) return MCS_ERR_ARG;
    c->group_lanes = lanes;
    return 0;
}

int mcs_set_fault(mcs_ctx* c, int kind, long long value) {
    if (!c || value < 0) return MCS_ERR_ARG;
    switch (kind) {
        case MCS_FAULT_ALLOC: c->fault_alloc_at = value; return 0;
        case MCS_FAULT_CUDA: c->fault_cuda = (int)std::min<long long>(value, 1 << 30); return 0;
        case MCS_FAULT_STALL_MS: c->fault_stall_ms = value; return 0;
        case MCS_FAULT_SPIN_LIMIT:
            if (value > 0xffffffffLL) return MCS_ERR_ARG;
            c->fault_spin = value;
            return 0;
        case MCS_FAULT_WITHHOLD_EXIT: c->fault_withhold = (int)std::min<long long>(value, 1 << 30); return 0;
        case MCS_FAULT_BLOCK_RING: c->fault_block_ring = value ? 1 : 0; return 0;
        default: return MCS_ERR_ARG;
    }
}

int mcs_set_search_mode(mcs_ctx* c, int mode) {
    if (!c || (mode != MCS_MODE_FREE && mode != MCS_MODE_LOCKSTEP)) return MCS_ERR_ARG;
    c->lockstep = mode == MCS_MODE_LOCKSTEP;
    return 0;
}

int mcs_set_max_warps(mcs_ctx* c, int warps) {
    if (!c || warps < 0) return MCS_ERR_ARG;
    c->max_warps = warps;
    return 0;
}

int mcs_last_stats(mcs_ctx* c, double* out, int n) {
    if (!c || !out || n < 0) return MCS_ERR_ARG;
    if (c->ev_pending && cudaEventQuery(c->ev1) == cudaSuccess) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, c->ev0, c->ev1) == cudaSuccess) c->stats[0] = ms * 1e3;
        const Control* src = c->last_wide ? (const Control*)c->wide_ctl : c->ctl;
        if (src && cudaMemcpy(&c->h_ctl, src, sizeof(Control), cudaMemcpyDeviceToHost) == cudaSuccess) {
            c->stats[2] = (double)c->h_ctl.donated;
            c->stats[3] = (double)c->h_ctl.stolen;
            c->stats[4] = (double)c->h_ctl.spilled;
            c->stats[8] = (double)c->h_ctl.class_visits;
            c->stats[9] = (double)c->h_ctl.pruned;
            c->stats[10] = (double)c->h_ctl.busy_cycles;
            c->stats[11] = (double)c->h_ctl.idle_cycles;
            c->stats[12] = (double)c->h_ctl.dbg_count;
            c->stats[13] = (double)c->h_ctl.dbg_code;
            c->stats[14] = (double)c->h_ctl.dbg_line;
        }
        c->ev_pending = false;
    }
    int k = std::min(n, 17);
    for (int i = 0; i < k; ++i) out[i] = c->stats[i];
    return k;
}

int mcs_solve_batch_device(mcs_ctx* c, int32_t npairs, const int32_t* d_n,
                           const int64_t* d_adj_off, const uint8_t* d_adj,
                           const int64_t* d_lab_off, const int32_t* d_labels, uint32_t flags,
                           double timeout_s, int32_t* d_size, int32_t* d_status,
                           uint64_t* d_nodes, int16_t* d_map, float* d_usec, void* stream) {
    if (!c || npairs < 0) return MCS_ERR_ARG;
    if (npairs > 0 && (!d_n || !d_adj_off || !d_adj || !d_size || !d_status || !d_nodes))
        return MCS_ERR_ARG;
    if (flags & MCS_RACE) return MCS_ERR_UNSUPPORTED;          // mcs_solve only
    if (cudaSetDevice(c->device) != cudaSuccess) return MCS_ERR_CUDA;
    cudaStream_t s = stream ? (cudaStream_t)stream : c->stream;
    if ((flags & MCS_GRAPH_REPLAY) && (flags & MCS_WIDE)) return MCS_ERR_UNSUPPORTED;
    if ((flags & MCS_GRAPH_REPLAY) && npairs > 0) {
        // the call's identity: every argument that the launches capture
        double tmo = timeout_s;
        uint64_t key[16] = {(uint64_t)npairs, (uint64_t)d_n, (uint64_t)d_adj_off, (uint64_t)d_adj,
                            (uint64_t)d_lab_off, (uint64_t)d_labels, (uint64_t)flags, 0,
                            (uint64_t)d_size, (uint64_t)d_status, (uint64_t)d_nodes, (uint64_t)d_map,
                            (uint64_t)d_usec, (uint64_t)c->warps_per_block | ((uint64_t)c->group_lanes << 32),
                            (uint64_t)c->smem_stack | ((uint64_t)c->blocks_per_sm << 32),
                            (uint64_t)c->max_warps | ((uint64_t)c->poll_nodes << 32) |
                                ((uint64_t)c->steal_keep_q4 << 48) | ((uint64_t)c->lockstep << 56)};
        memcpy(&key[7], &tmo, sizeof(double));
        if (!c->graph_exec || memcmp(key, c->graph_key, sizeof(key)) != 0) {
            if (c->graph_exec) { cudaGraphExecDestroy(c->graph_exec); c->graph_exec = nullptr; }
            if (c->graph) { cudaGraphDestroy(c->graph); c->graph = nullptr; }
            // size every arena outside the capture: an uncaptured run on the
            // context's stream (its results are overwritten by the replay)
            int rc = run_device(c, npairs, d_n, d_adj_off, d_adj, d_lab_off, d_labels, nullptr,
                                flags & ~MCS_GRAPH_REPLAY, timeout_s, d_size, d_status, d_nodes,
                                d_map, d_usec, c->stream, false);
            if (rc) return rc;
            CK(cudaStreamSynchronize(c->stream));
            CK(cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeRelaxed));
            rc = run_device(c, npairs, d_n, d_adj_off, d_adj, d_lab_off, d_labels, nullptr,
                            flags & ~MCS_GRAPH_REPLAY, timeout_s, d_size, d_status, d_nodes, d_map,
                            d_usec, c->stream, true);
            cudaGraph_t g = nullptr;
            cudaError_t e = cudaStreamEndCapture(c->stream, &g);
            if (rc) { if (g) cudaGraphDestroy(g); return rc; }
            CK(e);
            c->graph = g;
            CK(cudaGraphInstantiate(&c->graph_exec, g, 0));
            memcpy(c->graph_key, key, sizeof(key));
        }
        CK(cudaGraphLaunch(c->graph_exec, s));
        c->ev_pending = true;
        c->stats[6] = c->stats[7] = 0;
        return 0;
    }
    int rc;
    if (flags & MCS_WIDE) {
        // graphs of up to MCS_MAX_N vertices: the multi-word path (n unknown
        // on the host, so its class stacks are sized for the largest graphs)
        if (flags & (MCS_ORDER_LEARNED | MCS_ORDER_HR | MCS_TOP_DOWN | MCS_DEAD_END | MCS_RESTART | MCS_GRAPH_REPLAY))
            return MCS_ERR_UNSUPPORTED;
        rc = wide_run_device(c, npairs, d_n, d_adj_off, d_adj, d_lab_off, d_labels, nullptr,
                             flags & ~(MCS_WIDE | MCS_WORD32), timeout_s, 0, 0, d_size, d_status, d_nodes, d_map,
                             d_usec, s, true);
        c->last_wide = true;
    } else {
        rc = run_device(c, npairs, d_n, d_adj_off, d_adj, d_lab_off, d_labels, nullptr, flags,
                        timeout_s, d_size, d_status, d_nodes, d_map, d_usec, s, true);
        c->last_wide = false;
    }
    c->ev_pending = (rc == 0 && npairs > 0);
    c->stats[6] = c->stats[7] = 0;
    return rc;
}

int mcs_solve_batch(mcs_ctx* c, const mcs_graph* G, const mcs_graph* H, int32_t npairs,
                    uint32_t flags, double timeout_s, mcs_result* out) {
    if (!c || npairs < 0 || (npairs > 0 && (!G || !H || !out))) return MCS_ERR_ARG;
    if (flags & MCS_RACE) return MCS_ERR_UNSUPPORTED;          // mcs_solve only
    if (cudaSetDevice(c->device) != cudaSuccess) return MCS_ERR_CUDA;
    if (!c->race_on) c->stats[15] = c->stats[16] = 0;
    // structural checks (content is validated on the device by the pack kernels);
    // pairs with a graph of more than 64 vertices go to the multi-word path
    const uint32_t kNotWide = MCS_ORDER_LEARNED | MCS_ORDER_HR | MCS_TOP_DOWN | MCS_DEAD_END | MCS_RESTART;
    std::vector<char> bad(npairs, 0), wide(npairs, 0);
    std::vector<int> dev(npairs, -1);
    size_t adj_bytes = 0, lab_count = 0;
    int n1 = 0, n2 = 0, wide_max_n = 0, wide_max_min_n = 0;
    for (int p = 0; p < npairs; ++p) {
        if (check_graph(&G[p]) || check_graph(&H[p])) { bad[p] = 1; continue; }
        wide[p] = std::max(G[p].n, H[p].n) > kMaxN;
        if (wide[p] && (flags & kNotWide)) { bad[p] = 2; continue; }
        adj_bytes += (size_t)G[p].n * G[p].n + (size_t)H[p].n * H[p].n;
        if (G[p].labels) lab_count += G[p].n;
        if (H[p].labels) lab_count += H[p].n;
        if (wide[p]) {
            ++n2;
            wide_max_n = std::max(wide_max_n, std::max(G[p].n, H[p].n));
            wide_max_min_n = std::max(wide_max_min_n, std::min(G[p].n, H[p].n));
        } else {
            ++n1;
        }
    }
    // device index: one-word pairs first, then the multi-word ones
    {
        int a = 0, b = n1;
        for (int p = 0; p < npairs; ++p)
            if (!bad[p]) dev[p] = wide[p] ? b++ : a++;
    }
    const int nd = n1 + n2;
    HostLayout L;
    size_t P2 = 2 * (size_t)nd;
    L.off_n = 0;
    L.off_adjoff = align16(L.off_n + 4 * P2);
    L.off_laboff = align16(L.off_adjoff + 8 * P2);
    L.off_order = align16(L.off_laboff + 8 * P2);
    L.off_labels = align16(L.off_order + 4 * (size_t)nd);
    L.off_adj = align16(L.off_labels + 4 * std::max<size_t>(lab_count, 1));
    L.total = align16(L.off_adj + std::max<size_t>(adj_bytes, 16));
    int rc;
    if ((rc = grow_host(c, c->h_in, c->h_in_cap, L.total))) return rc;
    if ((rc = grow_dev(c, c->d_in, c->d_in_cap, L.total))) return rc;
    int32_t* hn = (int32_t*)(c->h_in + L.off_n);
    int64_t* hao = (int64_t*)(c->h_in + L.off_adjoff);
    int64_t* hlo = (int64_t*)(c->h_in + L.off_laboff);
    int32_t* hord = (int32_t*)(c->h_in + L.off_order);
    int32_t* hlab = (int32_t*)(c->h_in + L.off_labels);
    uint8_t* hadj = c->h_in + L.off_adj;
    size_t ao = 0, lo = 0;
    for (int p = 0; p < npairs; ++p) {
        if (bad[p]) continue;
        const mcs_graph* gs[2] = {&G[p], &H[p]};
        for (int s = 0; s < 2; ++s) {
            size_t gi = 2 * (size_t)dev[p] + s;
            const mcs_graph* g = gs[s];
            hn[gi] = g->n;
            hao[gi] = (int64_t)ao;
            if (g->n) memcpy(hadj + ao, g->adj, (size_t)g->n * g->n);
            ao += (size_t)g->n * g->n;
            if (g->labels) {
                hlo[gi] = (int64_t)lo;
                memcpy(hlab + lo, g->labels, sizeof(int32_t) * g->n);
                lo += g->n;
            } else {
                hlo[gi] = -1;
            }
        }
    }
    // 32-bit node step when every one-word graph of the call has at most 32 vertices
    uint32_t flags1 = flags;
    {
        bool fit = true;
        for (int p = 0; p < npairs && fit; ++p)
            if (!bad[p] && !wide[p] && (G[p].n > 32 || H[p].n > 32)) fit = false;
        if (fit) flags1 |= MCS_WORD32;
    }
    // longest-processing-time-first within each launch: larger and denser pairs
    // start first (order entries are indices local to the launch's segment)
    {
        std::vector<double> cost(nd, 0.0);
        for (int p = 0; p < npairs; ++p) {
            if (bad[p]) continue;
            double nG = G[p].n, nH = H[p].n;
            cost[dev[p]] = std::min(nG, nH) * 1000.0 + std::max(nG, nH);
        }
        std::vector<int32_t> ord(nd);
        std::iota(ord.begin(), ord.begin() + n1, 0);
        std::iota(ord.begin() + n1, ord.end(), 0);
        std::stable_sort(ord.begin(), ord.begin() + n1, [&](int a, int b) { return cost[a] > cost[b]; });
        std::stable_sort(ord.begin() + n1, ord.end(),
                         [&](int a, int b) { return cost[n1 + a] > cost[n1 + b]; });
        memcpy(hord, ord.data(), sizeof(int32_t) * nd);
    }
    // outputs
    size_t o_size = 0, o_status = align16(4 * (size_t)nd), o_nodes = align16(o_status + 4 * (size_t)nd);
    size_t o_usec = align16(o_nodes + 8 * (size_t)nd), o_map = align16(o_usec + 4 * (size_t)nd);
    size_t o_total = align16(o_map + 2 * (size_t)nd * MCS_MAX_N);
    if ((rc = grow_host(c, c->h_out, c->h_out_cap, o_total))) return rc;
    if ((rc = grow_dev(c, c->d_out, c->d_out_cap, o_total))) return rc;
    cudaStream_t s = c->stream;
    Control wctl;
    memset(&wctl, 0, sizeof(wctl));
    if (nd > 0) {
        CK(cudaMemcpyAsync(c->d_in, c->h_in, L.total, cudaMemcpyHostToDevice, s));
        const int32_t* dn = (const int32_t*)(c->d_in + L.off_n);
        const int64_t* dao = (const int64_t*)(c->d_in + L.off_adjoff);
        const int64_t* dlo = (const int64_t*)(c->d_in + L.off_laboff);
        const int32_t* dord = (const int32_t*)(c->d_in + L.off_order);
        const int32_t* dlab = lab_count ? (const int32_t*)(c->d_in + L.off_labels) : nullptr;
        int32_t* dsize = (int32_t*)(c->d_out + o_size);
        int32_t* dstat = (int32_t*)(c->d_out + o_status);
        uint64_t* dnodes = (uint64_t*)(c->d_out + o_nodes);
        float* dusec = (float*)(c->d_out + o_usec);
        int16_t* dmap = (flags & MCS_NO_MAPPING) ? nullptr : (int16_t*)(c->d_out + o_map);
        if (n1 > 0) {
            rc = run_device(c, n1, dn, dao, c->d_in + L.off_adj, dlo, dlab, dord, flags1, timeout_s, dsize, dstat,
                            dnodes, dmap, dusec, s, true);
            if (rc) return rc;
        }
        if (n2 > 0) {
            rc = wide_run_device(c, n2, dn + 2 * n1, dao + 2 * n1, c->d_in + L.off_adj, dlo + 2 * n1, dlab,
                                 dord + n1, flags & ~MCS_WORD32, timeout_s, wide_max_n, wide_max_min_n,
                                 dsize + n1, dstat + n1, dnodes + n1, dmap ? dmap + (size_t)n1 * MCS_MAX_N : nullptr,
                                 dusec + n1, s, n1 == 0);
            if (rc) return rc;
        }
        size_t copy_bytes = (flags & MCS_NO_MAPPING) ? o_map : o_total;
        CK(cudaMemcpyAsync(c->h_out, c->d_out, copy_bytes, cudaMemcpyDeviceToHost, s));
        if (n1 > 0) CK(cudaMemcpyAsync(&c->h_ctl, c->ctl, sizeof(Control), cudaMemcpyDeviceToHost, s));
        else memset(&c->h_ctl, 0, sizeof(Control));
        if (n2 > 0) CK(cudaMemcpyAsync(&wctl, c->wide_ctl, sizeof(Control), cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
        float ms = 0.f;
        cudaEventElapsedTime(&ms, c->ev0, c->ev1);
        c->stats[0] = ms * 1e3;
        c->stats[2] = (double)c->h_ctl.donated + (double)wctl.donated;
        c->stats[3] = (double)c->h_ctl.stolen + (double)wctl.stolen;
        c->stats[4] = (double)c->h_ctl.spilled + (double)wctl.spilled;
        c->stats[8] = (double)c->h_ctl.class_visits + (double)wctl.class_visits;
        c->stats[9] = (double)c->h_ctl.pruned + (double)wctl.pruned;
        c->stats[10] = (double)c->h_ctl.busy_cycles;
        c->stats[11] = (double)c->h_ctl.idle_cycles;
        c->stats[12] = (double)c->h_ctl.dbg_count;
        c->stats[13] = (double)c->h_ctl.dbg_code;
        c->stats[14] = (double)c->h_ctl.dbg_line;
        c->stats[6] = (double)L.total;
        c->stats[7] = (double)(copy_bytes + sizeof(Control) * ((n1 > 0) + (n2 > 0)));
        c->ev_pending = false;
    }
    int32_t* rsize = (int32_t*)(c->h_out + o_size);
    int32_t* rstat = (int32_t*)(c->h_out + o_status);
    uint64_t* rnodes = (uint64_t*)(c->h_out + o_nodes);
    float* rusec = (float*)(c->h_out + o_usec);
    int16_t* rmap = (int16_t*)(c->h_out + o_map);
    int ret = MCS_OK;
    double tot_nodes = 0;
    for (int p = 0; p < npairs; ++p) {
        mcs_result& r = out[p];
        if (bad[p]) {
            const int st = bad[p] == 2 ? MCS_ERR_UNSUPPORTED : MCS_ERR_ARG;
            r.size = 0; r.status = st; r.npairs = 0; r.nodes = 0; r.seconds = 0;
            ret = worst(ret, st);
            continue;
        }
        const int d = dev[p];
        r.size = rsize[d];
        r.status = rstat[d];
        r.nodes = rnodes[d];
        r.seconds = rusec[d] * 1e-6;
        tot_nodes += (double)r.nodes;
        r.npairs = 0;
        if (!(flags & MCS_NO_MAPPING) && r.status >= 0) {
            int k = 0;
            for (int x = 0; x < G[p].n; ++x) {
                int16_t y = rmap[(size_t)d * MCS_MAX_N + x];
                if (y >= 0) {
                    if (r.g_idx) r.g_idx[k] = (int16_t)x;
                    if (r.h_idx) r.h_idx[k] = y;
                    ++k;
                }
            }
            r.npairs = k;
        }
        ret = worst(ret, r.status);
    }
    c->stats[1] = tot_nodes;
    if (nd > 0 && c->h_ctl.error) ret = worst(ret, c->h_ctl.error);
    if (nd > 0 && wctl.error) ret = worst(ret, wctl.error);
    return ret;
}

int mcs_solve(mcs_ctx* c, const mcs_graph* G, const mcs_graph* H, uint32_t flags,
              double timeout_s, mcs_result* out) {
    if (!c || !G || !H || !out) return MCS_ERR_ARG;
    if (flags & MCS_RACE) return solve_race(c, G, H, flags & ~MCS_RACE, timeout_s, out);
    int rc = mcs_solve_batch(c, G, H, 1, flags, timeout_s, out);
    return rc < 0 ? rc : out->status;
}

int mcs_bench_popc(mcs_ctx* c, double* popc_per_s) {
    if (!c || !popc_per_s) return MCS_ERR_ARG;
    if (cudaSetDevice(c->device) != cudaSuccess) return MCS_ERR_CUDA;
    unsigned long long* d = nullptr;
    CK(cudaMalloc((void**)&d, 16));
    const int blocks = c->sms * 8, iters = 1 << 16;
    int rc = 0;
    float ms = 0.f;
    for (int rep = 0; rep < 2 && rc == 0; ++rep) {      // the first pass warms up
        if (cudaEventRecord(c->ev0, c->stream) != cudaSuccess ||
            launch_popc_bench(d, blocks, iters, c->stream) != cudaSuccess ||
            cudaEventRecord(c->ev1, c->stream) != cudaSuccess ||
            cudaStreamSynchronize(c->stream) != cudaSuccess ||
            cudaEventElapsedTime(&ms, c->ev0, c->ev1) != cudaSuccess)
            rc = MCS_ERR_CUDA;
    }
    cudaFree(d);
    if (rc) return rc;
    *popc_per_s = (double)blocks * 256.0 * 8.0 * (double)iters / (ms * 1e-3);
    return 0;
}

const char* mcs_error_detail(void) { return g_detail; }

const char* mcs_strerror(int code) {
    switch (code) {
        case MCS_OK: return "ok: optimum found and proven";
        case MCS_TIMEOUT: return "timeout: size is a lower bound";
        case MCS_PENDING: return "pending";
        case MCS_ERR_ARG: return "invalid argument";
        case MCS_ERR_NOMEM: return "out of memory";
        case MCS_ERR_CUDA: return "CUDA error";
        case MCS_ERR_DEVICE_STALL: return "bounded device wait expired";
        case MCS_ERR_UNSUPPORTED: return "unsupported";
        default: return "unknown status";
    }
}

}  // extern "C"
