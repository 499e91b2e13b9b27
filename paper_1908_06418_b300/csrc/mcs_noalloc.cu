// mcs_solve_batch_noalloc: the device-resident batch solve for callers that
// must not allocate device memory.
//
// Some callers cannot call cudaMalloc: code running while a CUDA graph is
// being captured on a stream that forbids allocation, plug-ins inside a host
// framework that owns every device allocation (a custom memory pool or a
// fixed memory budget), and real-time services that must not block in the
// allocator.  The regular entry points keep their scratch (packed graphs,
// per-pair state, incumbent slots, the task ring, per-warp stack overflow) in
// grow-only arenas that a context allocates on first use.  This entry point
// instead places all of that scratch in one file-scope device array of fixed
// size, created when the library is loaded on a device and kept until the
// process exits, and runs the same pack and search kernels on it.
#include <cstdio>
#include <cstring>
#include <mutex>

#include "mcs_internal.cuh"
#include "../../include/mcs.h"

using namespace mcsk;

namespace {

constexpr int kNaPairs = MCS_NOALLOC_MAX_PAIRS;
constexpr int kNaWarpsPerBlock = 4;
constexpr int kNaMaxWarps = MCS_NOALLOC_MAX_WARPS;
constexpr int kNaStackSmem = 256;                     // class entries per warp in shared memory
constexpr uint32_t kNaRing = 4096;                    // >= 4 * warps + pairs, a power of two
static_assert(kNaRing >= 4u * kNaMaxWarps + kNaPairs, "ring too small for the warp limit");

constexpr size_t al256(size_t x) { return (x + 255) & ~(size_t)255; }
constexpr size_t kOffGraphs = 0;
constexpr size_t kOffState = al256(kOffGraphs + sizeof(PairGraph) * kNaPairs);
constexpr size_t kOffBest = al256(kOffState + sizeof(PairState) * kNaPairs);
constexpr size_t kOffCtl = al256(kOffBest + sizeof(uint16_t) * kNaPairs * kLevels * kMaxN);
constexpr size_t kOffQueue = al256(kOffCtl + sizeof(Control));
constexpr size_t kOffSeq = al256(kOffQueue + sizeof(Task) * kNaRing);
constexpr size_t kOffStack = al256(kOffSeq + sizeof(u64) * kNaRing);
constexpr size_t kScratchBytes =
    al256(kOffStack + sizeof(ulonglong2) * (size_t)kNaMaxWarps * (kStackMax - kNaStackSmem));
static_assert(kScratchBytes <= MCS_NOALLOC_SCRATCH_BYTES, "header limit out of date");

// The scratch.  Each device that loads the library holds its own copy until
// the process exits.  In host code this name is only a stand-in for the
// device symbol: its device address comes from cudaGetSymbolAddress.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
unsigned char* g_ptr[kMaxDevices] = {};
int g_sms[kMaxDevices] = {};

// Once per device, with that device current: the device address of the
// scratch, the SM count, and every kernel variant this entry point can
// launch loaded with its shared-memory limit set (so that no later call, for
// any flags, makes a loading or attribute call).  Returns 0 or an MCS_ERR_*
// code.
int setup_current_device(int dev, unsigned char** ptr, int* sms) {
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_ptr[dev]) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) return MCS_ERR_CUDA;
        int n = 0;
        if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0)
            return MCS_ERR_CUDA;
        if (warm_batch_variants(kNaWarpsPerBlock * warp_smem_bytes(kNaStackSmem)) != cudaSuccess) {
            cudaGetLastError();
            return MCS_ERR_CUDA;
        }
        g_ptr[dev] = (unsigned char*)p;
        g_sms[dev] = n;
    }
    *ptr = g_ptr[dev];
    *sms = g_sms[dev];
    return 0;
}

}  // namespace

extern "C" int mcs_solve_batch_noalloc(int32_t npairs, const int32_t* d_n,
                                       const int64_t* d_adj_off, const uint8_t* d_adj,
                                       const int64_t* d_lab_off, const int32_t* d_labels,
                                       uint32_t flags, double timeout_s, int32_t* d_size,
                                       int32_t* d_status, uint64_t* d_nodes, int16_t* d_map,
                                       float* d_usec, void* stream) {
    if (npairs < 0 || npairs > kNaPairs) return MCS_ERR_ARG;     // beyond the fixed scratch
    if (npairs == 0) return 0;
    if (!d_n || !d_adj_off || !d_adj || !d_size || !d_status || !d_nodes) return MCS_ERR_ARG;
    if (flags & (MCS_ORDER_LEARNED | MCS_WIDE | MCS_RACE)) return MCS_ERR_UNSUPPORTED;
    if ((flags & MCS_TOP_DOWN) && (flags & MCS_DEAD_END)) return MCS_ERR_ARG;
    if ((flags & MCS_RESTART) && (flags & (MCS_TOP_DOWN | MCS_DEAD_END))) return MCS_ERR_ARG;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return MCS_ERR_CUDA;
    unsigned char* base = nullptr;
    int sms = 0;
    int rc = setup_current_device(dev, &base, &sms);
    if (rc) return rc;
    cudaStream_t s = (cudaStream_t)stream;
    const bool directed = (flags & MCS_DIRECTED) != 0;
    const int blocks = sms < kNaMaxWarps / kNaWarpsPerBlock ? sms : kNaMaxWarps / kNaWarpsPerBlock;
    const int warps = blocks * kNaWarpsPerBlock;

    PairGraph* graphs = (PairGraph*)(base + kOffGraphs);
    PairState* state = (PairState*)(base + kOffState);
    uint16_t* best = (uint16_t*)(base + kOffBest);
    Control* ctl = (Control*)(base + kOffCtl);
    Task* queue = (Task*)(base + kOffQueue);
    u64* qseq = (u64*)(base + kOffSeq);
    ulonglong2* gstack = (ulonglong2*)(base + kOffStack);
    int16_t* map = (flags & MCS_NO_MAPPING) ? nullptr : d_map;

    // The pack kernel re-initialises everything the search reads before it
    // writes it: the control block, every ring sequence word, the root
    // entries and each pair's state.  The incumbent slots and the stack
    // overflow are always written before they are read.
    PackParams pp;
    memset(&pp, 0, sizeof(pp));
    pp.npairs = npairs;
    pp.flags = flags;
    pp.n = d_n;
    pp.adj_off = d_adj_off;
    pp.adj = d_adj;
    pp.lab_off = d_lab_off;
    pp.labels = d_labels;
    pp.graphs = graphs;
    pp.state = state;
    pp.out_size = d_size;
    pp.out_status = d_status;
    pp.out_nodes = reinterpret_cast<u64*>(d_nodes);
    pp.out_map = map;
    pp.out_usec = d_usec;
    pp.ctl = ctl;
    pp.queue = queue;
    pp.qseq = qseq;
    pp.qcap = kNaRing;
    if (launch_pack(pp, s) != cudaSuccess) return MCS_ERR_CUDA;

    double tmo = timeout_s > 0 ? (timeout_s < 3600.0 ? timeout_s : 3600.0) : 3600.0;
    SearchParams sp;
    memset(&sp, 0, sizeof(sp));
    sp.poll_mask = kPollMaskDefault;
    sp.steal_keep_q4 = kStealKeepDefault;
    sp.dead_nodes = 1ull << 22;
    sp.dead_double = 0;
    sp.restart_min = 1ull << 20;
    sp.restart_seed = 0;
    sp.npairs = npairs;
    sp.flags = flags;
    sp.timeout_ns = (u64)(tmo * 1e9);
    sp.stall_ns = sp.timeout_ns + 2000000000ull;
    sp.graphs = graphs;
    sp.state = state;
    sp.best = best;
    sp.ctl = ctl;
    sp.queue = queue;
    sp.qseq = qseq;
    sp.qcap = kNaRing;
    sp.stack_smem = kNaStackSmem;
    sp.warp_smem_bytes = warp_smem_bytes(kNaStackSmem);
    sp.max_warps = warps;
    sp.gstack = gstack;
    sp.out_size = d_size;
    sp.out_status = d_status;
    sp.out_nodes = reinterpret_cast<u64*>(d_nodes);
    sp.out_map = map;
    sp.out_usec = d_usec;
    if (launch_search(sp, blocks, kNaWarpsPerBlock, directed, false, s) != cudaSuccess) return MCS_ERR_CUDA;
    return 0;
}
