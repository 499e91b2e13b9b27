// Serving: mcs_submit / mcs_poll with continuous batching.
//
// Requests are written into mapped pinned host memory (a ring of slot
// numbers, per-slot descriptors and raw graphs).  A resident launch of the
// search kernel in serve mode admits them while it runs: its first warp polls
// the ring, copies and packs each request into its device slot and publishes
// it as a root task of the ticket ring; searchers of the context's width (8
// lanes by default) take it like a batch root, and the request's search then
// shares the GPU with every other in-flight request through the same work
// donation as a batch.  Results come back into
// mapped memory, marked done by the request's ticket after a system fence.
//
// Admission is bounded by device memory: a fixed pool of slots (packed
// graphs, search state, incumbent mappings) is allocated when serving starts;
// a request that finds no free slot waits in a host queue until a finished
// request's slot is released by mcs_poll.  The server launch exits after
// kLingerNs without work; mcs_submit / mcs_poll relaunch it when needed.
#include <algorithm>
#include <atomic>
#include <cstring>
#include <deque>
#include <new>
#include <unordered_map>
#include <vector>

#include "mcs_internal.cuh"
#include "../../include/mcs.h"

using namespace mcsk;

namespace {

constexpr int kSlots = 2048;
constexpr int kRing = 4096;                   // >= slots
constexpr u64 kLingerNs = 20ull * 1000000ull;   // 20 ms
constexpr double kMaxServeTimeout = 60.0;     // seconds

struct Pending {
    u64 ticket;
    int32_t nG, nH, labelled, flags;
    u64 timeout_ns;
    std::vector<uint8_t> data;                // kSlotBytes
};

struct Active {
    int slot;
    u64 ring_pos;
};

}  // namespace

struct ServeState {
    // mapped pinned host memory
    u64* h_written = nullptr;
    int32_t* h_ring = nullptr;
    ServeReq* h_req = nullptr;
    uint8_t* h_data = nullptr;
    ServeRes* h_res = nullptr;
    u64* h_admitted = nullptr;
    int32_t* h_stop = nullptr;
    // device memory
    uint8_t* d_data = nullptr;
    PairGraph* graphs = nullptr;
    PairState* state = nullptr;
    uint16_t* best = nullptr;
    Control* ctl = nullptr;
    Task* queue = nullptr;
    u64* qseq = nullptr;
    uint32_t qcap = 0;
    ulonglong2* gstack = nullptr;
    int32_t* in_flight = nullptr;
    int blocks = 0, warps = 0, wsmem = 0;   // warps: searchers of the server launch
    int gs = 32;                            // lanes per searcher of the server launch
    cudaStream_t stream = nullptr;
    cudaEvent_t done_ev = nullptr;
    bool running = false;
    int last_error = 0;                     // error of the last failed server launch
    u64 failed_upto = 0;                    // ring entries below this were lost by it
    u64 written = 0;
    u64 next_ticket = 0;
    std::vector<int> free_slots;
    std::unordered_map<u64, Active> active;
    std::deque<Pending> pending;
};

namespace {

int serve_fail(cudaError_t e) { return e == cudaErrorMemoryAllocation ? MCS_ERR_NOMEM : MCS_ERR_CUDA; }
#define CKS(x) do { cudaError_t _e = (x); if (_e != cudaSuccess) return serve_fail(_e); } while (0)

template <typename T>
int host_mapped(T*& p, size_t count) {
    CKS(cudaHostAlloc((void**)&p, sizeof(T) * count, cudaHostAllocMapped | cudaHostAllocPortable));
    memset((void*)p, 0, sizeof(T) * count);
    return 0;
}

template <typename T>
T* dev_view(T* host_ptr) {
    void* d = nullptr;
    if (cudaHostGetDevicePointer(&d, (void*)host_ptr, 0) != cudaSuccess) return nullptr;
    return (T*)d;
}

int serve_state(mcs_ctx* c, ServeState** out) {
    if (c->serve) { *out = c->serve; return 0; }
    ServeState* S = new (std::nothrow) ServeState();
    if (!S) return MCS_ERR_NOMEM;
    c->serve = S;
    int rc;
    if ((rc = host_mapped(S->h_written, 1)) || (rc = host_mapped(S->h_ring, kRing)) ||
        (rc = host_mapped(S->h_req, kSlots)) || (rc = host_mapped(S->h_data, (size_t)kSlots * kSlotBytes)) ||
        (rc = host_mapped(S->h_res, kSlots)) || (rc = host_mapped(S->h_admitted, 1)) ||
        (rc = host_mapped(S->h_stop, 1)))
        return rc;
    CKS(cudaMalloc((void**)&S->d_data, (size_t)kSlots * kSlotBytes));
    CKS(cudaMalloc((void**)&S->graphs, sizeof(PairGraph) * kSlots));
    CKS(cudaMalloc((void**)&S->state, sizeof(PairState) * kSlots));
    CKS(cudaMalloc((void**)&S->best, sizeof(uint16_t) * (size_t)kSlots * kLevels * kMaxN));
    CKS(cudaMalloc((void**)&S->ctl, sizeof(Control)));
    CKS(cudaMalloc((void**)&S->in_flight, sizeof(int32_t)));
    // launch shape: the context's warps per block and serving searcher width
    // (mcs_set_serve_group; at least 8 lanes: the level arrays and result
    // scratch stay in shared memory), undirected, plain order; warp 0 of the
    // grid admits requests
    S->gs = c->serve_lanes;
    S->wsmem = warp_smem_bytes(stack_entries(c, S->gs), S->gs);
    const int spw = 32 / S->gs;                     // searchers per warp
    int per_sm = serve_max_blocks_per_sm(c->warps_per_block, c->warps_per_block * spw * S->wsmem, S->gs);
    if (per_sm <= 0) return MCS_ERR_UNSUPPORTED;
    if (c->blocks_per_sm > 0 && c->blocks_per_sm < per_sm) per_sm = c->blocks_per_sm;
    S->blocks = c->sms * per_sm;
    S->warps = S->blocks * c->warps_per_block * spw;     // searchers (warp 0's are the admitter)
    uint32_t q = 1024;
    while (q < (uint32_t)(4 * S->warps + kSlots)) q <<= 1;
    S->qcap = q;
    CKS(cudaMalloc((void**)&S->queue, sizeof(Task) * q));
    CKS(cudaMalloc((void**)&S->qseq, sizeof(u64) * q));
    const size_t per = gstack_entries(stack_entries(c, S->gs), S->gs);
    CKS(cudaMalloc((void**)&S->gstack, sizeof(ulonglong2) * std::max<size_t>(per * S->warps, 1)));
    CKS(cudaStreamCreateWithFlags(&S->stream, cudaStreamNonBlocking));
    CKS(cudaEventCreateWithFlags(&S->done_ev, cudaEventDisableTiming));
    for (int i = kSlots - 1; i >= 0; --i) S->free_slots.push_back(i);
    *out = S;
    return 0;
}

// False once the server launch has ended.  A launch that ended with an
// error (a bounded device wait expired, or a CUDA error) loses the requests
// published while it ran and not finished: they are marked failed (their
// polls return the error) and are not admitted again; later requests start
// a fresh launch.
bool server_running(ServeState* S) {
    if (!S->running) return false;
    cudaError_t e = cudaEventQuery(S->done_ev);
    if (e == cudaErrorNotReady) return true;
    S->running = false;
    int err = 0;
    if (e != cudaSuccess) {
        err = MCS_ERR_CUDA;
    } else if (cudaMemcpy(&err, &S->ctl->error, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) {
        err = MCS_ERR_CUDA;
    }
    if (err) {
        S->last_error = err;
        S->failed_upto = S->written;
        *(volatile u64*)S->h_admitted = S->written;
    }
    return false;
}

int launch_server(mcs_ctx* c, ServeState* S) {
    CKS(launch_serve_init(S->ctl, S->qseq, S->qcap, S->in_flight, c->fault_block_ring, S->stream));
    SearchParams sp;
    memset(&sp, 0, sizeof(sp));
    sp.poll_mask = kPollMaskDefault;
    sp.steal_keep_q4 = kStealKeepDefault;
    sp.dead_nodes = 0;
    sp.dead_double = 0;
    sp.restart_min = 0;
    sp.restart_seed = 0;
    sp.serving = 1;
    sp.sv.host_written = dev_view(S->h_written);
    sp.sv.ring = dev_view(S->h_ring);
    sp.sv.ring_cap = kRing;
    sp.sv.nslots = kSlots;
    sp.sv.req = dev_view(S->h_req);
    sp.sv.hdata = dev_view(S->h_data);
    sp.sv.ddata = S->d_data;
    sp.sv.res = dev_view(S->h_res);
    sp.sv.dev_admitted = dev_view(S->h_admitted);
    sp.sv.stop = dev_view(S->h_stop);
    sp.sv.in_flight = S->in_flight;
    sp.sv.linger_ns = kLingerNs;
    if (!sp.sv.host_written || !sp.sv.ring || !sp.sv.req || !sp.sv.hdata || !sp.sv.res ||
        !sp.sv.dev_admitted || !sp.sv.stop)
        return MCS_ERR_CUDA;
    sp.npairs = kSlots;
    sp.flags = 0;
    sp.timeout_ns = (u64)(kMaxServeTimeout * 1e9);
    sp.stall_ns = c->fault_stall_ms > 0 ? (u64)c->fault_stall_ms * 1000000ull
                                        : sp.timeout_ns + kLingerNs + 2000000000ull;
    sp.spin_limit = (uint32_t)c->fault_spin;
    sp.withhold_exit = c->fault_withhold;
    sp.graphs = S->graphs;
    sp.state = S->state;
    sp.best = S->best;
    sp.ctl = S->ctl;
    sp.queue = S->queue;
    sp.qseq = S->qseq;
    sp.qcap = S->qcap;
    sp.stack_smem = stack_entries(c, S->gs);
    sp.warp_smem_bytes = S->wsmem;
    sp.max_warps = S->warps;
    sp.gstack = S->gstack;
    CKS(launch_search(sp, S->blocks, c->warps_per_block, false, false, S->stream, S->gs));
    CKS(cudaEventRecord(S->done_ev, S->stream));
    S->running = true;
    return 0;
}

// Places a request in a free slot and publishes it in the ring.
void place(ServeState* S, int slot, const Pending& p) {
    memcpy(S->h_data + (size_t)slot * kSlotBytes, p.data.data(), kSlotBytes);
    ServeReq& q = S->h_req[slot];
    q.nG = p.nG; q.nH = p.nH; q.labelled = p.labelled; q.flags = p.flags;
    q.ticket = p.ticket; q.timeout_ns = p.timeout_ns;
    *(volatile u64*)&S->h_res[slot].done = 0;
    std::atomic_thread_fence(std::memory_order_release);
    const u64 pos = S->written;
    *(volatile int32_t*)&S->h_ring[pos % kRing] = slot;
    std::atomic_thread_fence(std::memory_order_release);
    S->written = pos + 1;
    *(volatile u64*)S->h_written = S->written;
    S->active[p.ticket] = Active{slot, pos};
}

// Moves waiting requests into free slots and (re)launches the server when
// published requests are not admitted yet and no server launch is running.
int kick(mcs_ctx* c, ServeState* S) {
    // first: a launch that failed is recorded before new requests are published
    const bool running = server_running(S);
    while (!S->pending.empty() && !S->free_slots.empty()) {
        int slot = S->free_slots.back();
        S->free_slots.pop_back();
        place(S, slot, S->pending.front());
        S->pending.pop_front();
    }
    if (!running) {
        const u64 admitted = *(volatile u64*)S->h_admitted;
        if (S->written > admitted) {
            *(volatile int32_t*)S->h_stop = 0;
            return launch_server(c, S);
        }
    }
    return 0;
}

int check_graph_s(const mcs_graph* g) {
    if (!g || g->n < 0 || g->n > MCS_MAX_N || (g->n > 0 && !g->adj)) return MCS_ERR_ARG;
    if (g->n > kMaxN) return MCS_ERR_UNSUPPORTED;     // served requests: one-word bit sets
    return 0;
}

}  // namespace

void mcs_serve_free(mcs_ctx* c) {
    ServeState* S = c->serve;
    if (!S) return;
    if (S->h_stop) *(volatile int32_t*)S->h_stop = 1;
    if (S->stream) cudaStreamSynchronize(S->stream);
    if (S->done_ev) cudaEventDestroy(S->done_ev);
    if (S->stream) cudaStreamDestroy(S->stream);
    void* hs[] = {S->h_written, S->h_ring, S->h_req, S->h_data, S->h_res, S->h_admitted, S->h_stop};
    for (void* h : hs) if (h) cudaFreeHost(h);
    void* ds[] = {S->d_data, S->graphs, S->state, S->best, S->ctl, S->queue, S->qseq, S->gstack, S->in_flight};
    for (void* d : ds) cudaFree(d);
    delete S;
    c->serve = nullptr;
}

extern "C" {

int mcs_submit(mcs_ctx* c, const mcs_graph* G, const mcs_graph* H, uint32_t flags, double timeout_s,
               uint64_t* ticket) {
    if (!c || !ticket) return MCS_ERR_ARG;
    int chk = check_graph_s(G);
    if (!chk) chk = check_graph_s(H);
    if (chk) return chk;
    if (flags & (MCS_DIRECTED | MCS_ORDER_LEARNED | MCS_ORDER_HR | MCS_TOP_DOWN | MCS_DEAD_END | MCS_RESTART |
                 MCS_WIDE | MCS_RACE))
        return MCS_ERR_UNSUPPORTED;
    if (cudaSetDevice(c->device) != cudaSuccess) return MCS_ERR_CUDA;
    ServeState* S = nullptr;
    int rc = serve_state(c, &S);
    if (rc) return rc;
    Pending p;
    p.ticket = ++S->next_ticket;
    p.nG = G->n;
    p.nH = H->n;
    p.labelled = (G->labels ? 1 : 0) | (H->labels ? 2 : 0);
    p.flags = (int32_t)flags;
    const double t = timeout_s > 0 ? (timeout_s < kMaxServeTimeout ? timeout_s : kMaxServeTimeout) : kMaxServeTimeout;
    p.timeout_ns = (u64)(t * 1e9);
    p.data.assign(kSlotBytes, 0);
    if (G->n) memcpy(p.data.data(), G->adj, (size_t)G->n * G->n);
    if (H->n) memcpy(p.data.data() + kMaxN * kMaxN, H->adj, (size_t)H->n * H->n);
    if (G->labels) memcpy(p.data.data() + 2 * kMaxN * kMaxN, G->labels, sizeof(int32_t) * G->n);
    if (H->labels) memcpy(p.data.data() + 2 * kMaxN * kMaxN + 4 * kMaxN, H->labels, sizeof(int32_t) * H->n);
    S->pending.push_back(std::move(p));
    *ticket = S->next_ticket;
    return kick(c, S);
}

int mcs_poll(mcs_ctx* c, uint64_t ticket, mcs_result* out) {
    if (!c || !out) return MCS_ERR_ARG;
    ServeState* S = c->serve;
    if (!S) return MCS_ERR_ARG;
    if (cudaSetDevice(c->device) != cudaSuccess) return MCS_ERR_CUDA;
    int rc = kick(c, S);
    if (rc) return rc;
    auto it = S->active.find(ticket);
    if (it == S->active.end()) {
        for (const Pending& p : S->pending)
            if (p.ticket == ticket) return MCS_PENDING;
        return MCS_ERR_ARG;
    }
    const int slot = it->second.slot;
    ServeRes& r = S->h_res[slot];
    if (*(volatile u64*)&r.done != ticket) {
        // published while a server launch ran that then failed (a bounded
        // wait expired or a CUDA error), and not finished by it
        if (!server_running(S) && it->second.ring_pos < S->failed_upto && *(volatile u64*)&r.done != ticket) {
            S->active.erase(it);
            S->free_slots.push_back(slot);
            out->size = 0;
            out->status = S->last_error ? S->last_error : MCS_ERR_DEVICE_STALL;
            out->npairs = 0;
            out->nodes = 0;
            out->seconds = 0.0;
            return out->status;
        }
        return MCS_PENDING;
    }
    std::atomic_thread_fence(std::memory_order_acquire);
    out->size = r.size;
    out->status = r.status;
    out->nodes = r.nodes;
    out->seconds = r.usec * 1e-6;
    int k = 0;
    const int nG = S->h_req[slot].nG;
    for (int x = 0; x < nG && x < kMaxN; ++x) {
        const int16_t y = r.map[x];
        if (y >= 0) {
            if (out->g_idx) out->g_idx[k] = (int16_t)x;
            if (out->h_idx) out->h_idx[k] = y;
            ++k;
        }
    }
    out->npairs = k;
    const int status = r.status;
    S->active.erase(it);
    S->free_slots.push_back(slot);
    kick(c, S);
    return status;
}

}  // extern "C"
