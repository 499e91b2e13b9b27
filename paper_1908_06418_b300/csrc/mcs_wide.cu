// Graphs of 65 to 256 vertices: McSplit with multi-word bit sets.
//
// The paper's solvers keep their label classes in byte-sized frames, which
// caps a graph at 254 vertices (Section III-B); every workload it measures
// stays far below that, and the one-word kernels of mcs_kernels.cu hold a
// graph's vertex set in one 64-bit word.  This file carries the same branch
// and bound (Section II-B, Algorithm 1, the bound of Eq. 1, the label-class
// split of Table 1) on NW 64-bit words per vertex set: NW = 2 for graphs of
// up to 128 vertices, NW = 4 up to 256.
//
//   wide_pack_kernel    one warp per pair: validation, degree renumbering
//                       (total in+out degree when directed, ties to the lower
//                       index, Section IV-A), multi-word row bit sets, root
//                       label classes (label + self-loop).
//   wide_search_kernel  persistent depth-first searches, one per warp, the
//                       label classes of a node spread over the lanes; work
//                       moves between warps through the same ticket ring as
//                       the one-word kernels (donation of the upper half of
//                       the shallowest open level's candidates, exit tokens,
//                       per-pair atomicMax incumbents, bounded waits).
//
// The one-word kernels are untouched by this file: a launch holds pairs of
// one kind, and the host routes pairs with more than 64 vertices here.
#include <cstdint>
#include <cstring>
#include <type_traits>

#include "mcs_internal.cuh"
#include "../../include/mcs.h"

namespace mcsw {

using mcsk::u64;
using mcsk::Control;
using mcsk::PairState;
using mcsk::kNoCap;
using mcsk::kTaskFresh;
using mcsk::kTaskPending;

#define WFULL 0xffffffffu

constexpr unsigned kKeyNone = 0xFFFFFFFFu;
constexpr int kSpinLimit = 1 << 22;

__device__ __forceinline__ u64 gtimer() {
    u64 t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
__device__ __forceinline__ unsigned lanemask_lt() {
    unsigned m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}
template <typename T>
__device__ __forceinline__ T vload(const T* p) { return *(volatile const T*)p; }
__device__ __forceinline__ u64 shfl64(u64 x, int src) {
    unsigned lo = (unsigned)x, hi = (unsigned)(x >> 32);
    lo = __shfl_sync(WFULL, lo, src);
    hi = __shfl_sync(WFULL, hi, src);
    return ((u64)hi << 32) | lo;
}

// A vertex set of up to 64 * NW vertices.
template <int NW>
struct Bits {
    u64 w[NW];
    __host__ __device__ __forceinline__ static Bits zero() {
        Bits b;
#pragma unroll
        for (int k = 0; k < NW; ++k) b.w[k] = 0;
        return b;
    }
    __device__ __forceinline__ static Bits one(int i) {
        Bits b = zero();
#pragma unroll
        for (int k = 0; k < NW; ++k) b.w[k] = (k == (i >> 6)) ? (1ull << (i & 63)) : 0ull;
        return b;
    }
    __device__ __forceinline__ bool any() const {
        u64 x = 0;
#pragma unroll
        for (int k = 0; k < NW; ++k) x |= w[k];
        return x != 0;
    }
    __device__ __forceinline__ int popc() const {
        int s = 0;
#pragma unroll
        for (int k = 0; k < NW; ++k) s += __popcll(w[k]);
        return s;
    }
    // lowest member, or -1
    __device__ __forceinline__ int low() const {
        int r = -1;
#pragma unroll
        for (int k = NW - 1; k >= 0; --k)
            if (w[k]) r = k * 64 + __ffsll((long long)w[k]) - 1;
        return r;
    }
    __device__ __forceinline__ bool test(int i) const { return (w[i >> 6] >> (i & 63)) & 1ull; }
    __device__ __forceinline__ void clear(int i) {
#pragma unroll
        for (int k = 0; k < NW; ++k)
            if (k == (i >> 6)) w[k] &= ~(1ull << (i & 63));
    }
    __device__ __forceinline__ Bits operator&(const Bits& o) const {
        Bits r;
#pragma unroll
        for (int k = 0; k < NW; ++k) r.w[k] = w[k] & o.w[k];
        return r;
    }
    __device__ __forceinline__ Bits operator|(const Bits& o) const {
        Bits r;
#pragma unroll
        for (int k = 0; k < NW; ++k) r.w[k] = w[k] | o.w[k];
        return r;
    }
    __device__ __forceinline__ Bits operator^(const Bits& o) const {
        Bits r;
#pragma unroll
        for (int k = 0; k < NW; ++k) r.w[k] = w[k] ^ o.w[k];
        return r;
    }
    __device__ __forceinline__ Bits andnot(const Bits& o) const {   // this \ o
        Bits r;
#pragma unroll
        for (int k = 0; k < NW; ++k) r.w[k] = w[k] & ~o.w[k];
        return r;
    }
    __device__ __forceinline__ Bits shfl(int src) const {
        Bits r;
#pragma unroll
        for (int k = 0; k < NW; ++k) r.w[k] = shfl64(w[k], src);
        return r;
    }
};

template <int NW>
struct alignas(16) Cls {
    Bits<NW> L, R;
};

// Loads through L2 of what other warps (or an earlier kernel) wrote: a task
// slot is refilled by other SMs while the kernel runs, so L1 may hold old lines.
template <int NW>
__device__ __forceinline__ Bits<NW> ldcg(const Bits<NW>* p) {
    Bits<NW> b;
#pragma unroll
    for (int k = 0; k < NW; ++k) b.w[k] = __ldcg(&p->w[k]);
    return b;
}
template <int NW>
__device__ __forceinline__ Cls<NW> ldcg(const Cls<NW>* p) {
    Cls<NW> c;
    c.L = ldcg(&p->L);
    c.R = ldcg(&p->R);
    return c;
}

// Per-pair packed graph (renumbered; bit x of row v is vertex x in the new numbering).
template <int NW>
struct WGraph {
    Bits<NW> gout[64 * NW], gin[64 * NW], hout[64 * NW], hin[64 * NW];
    Cls<NW> root[64 * NW];
    uint8_t permG[64 * NW], permH[64 * NW];
    int32_t nG, nH, C0, valid;
};

struct WTaskHdr {
    int32_t pair, depth, C, v;
    int32_t flags, bound;
    int32_t pad[2];
};
template <int NW>
struct WTask {
    WTaskHdr h;
    Bits<NW> rrem;
    uint8_t Mg[64 * NW], Mh[64 * NW];
    Cls<NW> cls[64 * NW];
};

template <int NW>
struct WParams {
    int32_t npairs;
    uint32_t flags;
    // inputs (layout of mcs_solve_batch_device)
    const int32_t* n;
    const int64_t* adj_off;
    const uint8_t* adj;
    const int64_t* lab_off;
    const int32_t* labels;
    const int32_t* order;         // processing order of the pairs (may be null)
    // scratch
    WGraph<NW>* graphs;
    PairState* state;
    uint16_t* best;               // [npairs][64 NW + 1][64 NW]: (g << 8) | h per size slot
    Control* ctl;
    WTask<NW>* queue;
    u64* qseq;
    uint32_t qcap;                // power of two
    Cls<NW>* gstack;              // per-warp class stack
    size_t stack_entries;         // per warp
    int32_t max_warps;
    int32_t level_bytes;          // shared memory per warp
    u64 timeout_ns, stall_ns;
    uint32_t poll_mask;
    int32_t steal_keep_q4;
    uint32_t spin_limit;          // failure injection (0: kSpinLimit)
    int32_t withhold_exit;        // failure injection
    int32_t block_ring;           // failure injection
    // outputs
    int32_t* out_size;
    int32_t* out_status;
    u64* out_nodes;
    int16_t* out_map;             // [npairs][MCS_MAX_N] or null
    float* out_usec;
};

// ---------------------------------------------------------------------------
// pack: one warp per pair
// ---------------------------------------------------------------------------
// Lane l holds vertices l + 32 s, s < 2 NW.  Returns false (warp-uniform) if
// the graph is malformed.  skey: 64 NW long long of shared scratch.
template <int NW>
__device__ bool wide_pack_graph(int n, const uint8_t* a, const int32_t* lab, bool directed, Bits<NW>* out_rows,
                                Bits<NW>* in_rows, uint8_t* perm, long long* skey, int lane) {
    constexpr int S = 2 * NW;                  // vertices per lane
    bool ok = n >= 0 && n <= 64 * NW;
    for (int b0 = 0; ok && b0 < n * n; b0 += 32) {
        const int idx = b0 + lane;
        bool bad = false;
        if (idx < n * n) {
            const uint8_t x = a[idx];
            bad = x > 1;
            if (!directed) {
                const int i = idx / n, j = idx - i * n;
                bad |= x != a[j * n + i];
            }
        }
        if (__any_sync(WFULL, bad)) ok = false;
    }
    if (ok && lab) {
        bool bad = false;
        for (int i = lane; i < n; i += 32) bad |= lab[i] < 0;
        if (__any_sync(WFULL, bad)) ok = false;
    }
    if (!ok) return false;
    int deg[S];
#pragma unroll
    for (int s = 0; s < S; ++s) {
        const int i = lane + 32 * s;
        int d = 0;
        if (i < n)
            for (int j = 0; j < n; ++j) {
                if (j == i) continue;
                d += a[i * n + j];
                if (directed) d += a[j * n + i];
            }
        deg[s] = d;
    }
    // rank: earlier if higher degree, ties to the lower index
    int rank[S];
#pragma unroll
    for (int s = 0; s < S; ++s) rank[s] = 0;
    for (int j = 0; j < n; ++j) {
        int dj = 0;
#pragma unroll
        for (int s = 0; s < S; ++s) {
            const int v = __shfl_sync(WFULL, deg[s], j & 31);
            if (s == (j >> 5)) dj = v;
        }
#pragma unroll
        for (int s = 0; s < S; ++s) {
            const int i = lane + 32 * s;
            rank[s] += (dj > deg[s] || (dj == deg[s] && j < i)) ? 1 : 0;
        }
    }
    // new numbers of every vertex, in shared scratch (as the key array's first use)
    int* nr = reinterpret_cast<int*>(skey);
#pragma unroll
    for (int s = 0; s < S; ++s) {
        const int i = lane + 32 * s;
        if (i < n) { nr[i] = rank[s]; perm[rank[s]] = (uint8_t)i; }
    }
    __syncwarp();
#pragma unroll
    for (int s = 0; s < S; ++s) {
        const int i = lane + 32 * s;
        Bits<NW> o = Bits<NW>::zero(), in = Bits<NW>::zero();
        if (i < n)
            for (int j = 0; j < n; ++j) {
                if (j == i) continue;
                const int rj = nr[j];
                if (a[i * n + j]) o.w[rj >> 6] |= 1ull << (rj & 63);
                if (a[j * n + i]) in.w[rj >> 6] |= 1ull << (rj & 63);
            }
        if (i < n) {
            out_rows[rank[s]] = o;
            in_rows[rank[s]] = directed ? in : o;
        }
    }
    __syncwarp();
    // label + self-loop key of every new number
#pragma unroll
    for (int s = 0; s < S; ++s) {
        const int i = lane + 32 * s;
        if (i < n) {
            const long long lb = lab ? (long long)lab[i] : 0;
            skey[rank[s]] = lb * 2 + (a[i * n + i] ? 1 : 0);
        }
    }
    __syncwarp();
    return true;
}

template <int NW>
__global__ void wide_pack_kernel(WParams<NW> P) {
    constexpr int N = 64 * NW;
    __shared__ long long s_key[4][2][N];
    const int lane = threadIdx.x & 31;
    const int wib = threadIdx.x >> 5;
    const int p = blockIdx.x * (blockDim.x >> 5) + wib;
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < P.qcap; i += gridDim.x * blockDim.x) {
        if ((int)i < P.npairs) {
            WTask<NW>* t = P.queue + i;
            t->h.pair = P.order ? P.order[i] : (int)i;
            t->h.flags = kTaskFresh;
            t->h.depth = 0;
            t->h.C = 0;
            P.qseq[i] = (u64)i + 1;
        } else {
            P.qseq[i] = P.block_ring ? ~0ull : (u64)i;
        }
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        Control* c = P.ctl;
        c->q_head = 0;
        c->q_tail = (u64)P.npairs;
        c->remaining = P.npairs;
        c->error = 0;
        c->last_progress = gtimer();
        c->donated = c->stolen = c->spilled = c->class_visits = c->pruned = 0;
        c->busy_cycles = c->idle_cycles = 0;
        c->dbg_code = c->dbg_val = c->dbg_line = c->dbg_count = 0;
    }
    if (p >= P.npairs) return;
    const bool directed = (P.flags & MCS_DIRECTED) != 0;
    WGraph<NW>& pg = P.graphs[p];
    int nn[2];
    const uint8_t* aa[2];
    const int32_t* ll[2];
    for (int side = 0; side < 2; ++side) {
        const int gi = 2 * p + side;
        nn[side] = P.n[gi];
        aa[side] = P.adj + P.adj_off[gi];
        ll[side] = (P.labels && P.lab_off && P.lab_off[gi] >= 0) ? P.labels + P.lab_off[gi] : nullptr;
    }
    bool ok = true;
    for (int side = 0; side < 2 && ok; ++side)
        ok = wide_pack_graph<NW>(nn[side], aa[side], ll[side], directed, side ? pg.hout : pg.gout,
                                 side ? pg.hin : pg.gin, side ? pg.permH : pg.permG, s_key[wib][side], lane);
    __syncwarp();
    if (ok) {
        // one class per key present in both graphs; representative = lowest new G number
        const int nG = nn[0], nH = nn[1];
        const long long* kg = s_key[wib][0];
        const long long* kh = s_key[wib][1];
        int C = 0;
        for (int r0 = 0; r0 < N; r0 += 32) {
            const int r = r0 + lane;
            bool keep = false;
            Cls<NW> c;
            c.L = Bits<NW>::zero();
            c.R = Bits<NW>::zero();
            if (r < nG) {
                const long long k = kg[r];
                bool rep = true;
                for (int j = 0; j < nG; ++j)
                    if (kg[j] == k) {
                        c.L.w[j >> 6] |= 1ull << (j & 63);
                        if (j < r) rep = false;
                    }
                for (int j = 0; j < nH; ++j)
                    if (kh[j] == k) c.R.w[j >> 6] |= 1ull << (j & 63);
                keep = rep && c.R.any();
            }
            const unsigned m = __ballot_sync(WFULL, keep);
            if (keep) pg.root[C + __popc(m & lanemask_lt())] = c;
            C += __popc(m);
        }
        if (lane == 0) { pg.nG = nG; pg.nH = nH; pg.C0 = C; pg.valid = 1; }
    } else if (lane == 0) {
        pg.nG = 0; pg.nH = 0; pg.C0 = 0; pg.valid = 0;
    }
    if (lane == 0) {
        PairState& st = P.state[p];
        st.floor = 0; st.cap = kNoCap; st.inc = 0; st.real = 0; st.lo = st.hi = 0;
        st.dead = 0; st.live = st.mark = 0; st.restarts = 0;
        st.open = 1;
        st.status = ok ? MCS_PENDING : MCS_ERR_ARG;
        st.abort = 0;
        st.nodes = 0;
        st.t_start = st.deadline = 0;
        if (P.out_size) P.out_size[p] = 0;
        if (P.out_status) P.out_status[p] = ok ? MCS_PENDING : MCS_ERR_ARG;
        if (P.out_nodes) P.out_nodes[p] = 0;
        if (P.out_usec) P.out_usec[p] = 0.f;
    }
    if (P.out_map)
        for (int i = lane; i < MCS_MAX_N; i += 32) P.out_map[(size_t)p * MCS_MAX_N + i] = -1;
}

// ---------------------------------------------------------------------------
// search: one depth-first search per warp
// ---------------------------------------------------------------------------
__device__ __forceinline__ bool wait_seq(const u64* seq, u64 want, uint32_t limit) {
    const uint32_t lim = limit ? limit : (uint32_t)kSpinLimit;
    for (uint32_t it = 0; it < lim; ++it) {
        if (vload(seq) == want) return true;
        if (it > 64) __nanosleep(64);
    }
    return false;
}

// per level: base (20 bits) | C (9 bits) << 20 | v (8 bits) << 29 | flags (2 bits) << 37 | bound (9 bits) << 39
__device__ __forceinline__ u64 pack_info(int base, int C, int v, int flags, int bound) {
    return (u64)base | ((u64)C << 20) | ((u64)v << 29) | ((u64)flags << 37) | ((u64)bound << 39);
}

template <int NW>
struct Top {
    int d, base, C, v, flags, bound;
    Bits<NW> rrem;
};

template <int NW>
struct Lv {                                // a warp's level arrays in shared memory
    Bits<NW>* rrem;                        // [64 NW + 1]
    u64* info;                             // [64 NW + 1]
    uint8_t* Mg;                           // [64 NW]
    uint8_t* Mh;
};
template <int NW>
__host__ __device__ constexpr int level_bytes() {
    return (64 * NW + 1) * (8 * NW + 8) + 2 * 64 * NW + 16;
}

template <int NW>
__device__ __forceinline__ void load_level(const Lv<NW>& w, int d, Top<NW>& t) {
    const u64 inf = w.info[d];
    t.rrem = w.rrem[d];
    t.base = (int)(inf & 0xfffff);
    t.C = (int)((inf >> 20) & 0x1ff);
    t.v = (int)((inf >> 29) & 0xff);
    t.flags = (int)((inf >> 37) & 0x3);
    t.bound = (int)((inf >> 39) & 0x1ff);
}

// Result of scanning a level's classes: Eq. 1 sum and the class choice.
// Key = max(|L|, |R|) << 8 | lowest L vertex (unique per class).
template <int NW>
struct Scan {
    int sum;
    unsigned key;
    Bits<NW> R;
};

// Scans the classes of a level (removing v from its class first when
// remove_v >= 0: the "v stays unmatched" step) and chooses the next class.
template <int NW>
__device__ Scan<NW> scan_level(Cls<NW>* stk, int base, int C, int remove_v, int lane) {
    int sum = 0;
    unsigned best = kKeyNone;
    int bi = -1;
    for (int i0 = 0; i0 < C; i0 += 32) {
        const int i = i0 + lane;
        if (i < C) {
            Cls<NW>* ptr = stk + base + i;
            Bits<NW> L = ptr->L;
            const Bits<NW> R = ptr->R;
            if (remove_v >= 0 && L.test(remove_v)) {
                L.clear(remove_v);
                ptr->L = L;
            }
            if (L.any()) {
                const int a = L.popc(), b = R.popc();
                sum += min(a, b);
                const unsigned key = ((unsigned)max(a, b) << 8) | (unsigned)L.low();
                if (key < best) { best = key; bi = i; }
            }
        }
    }
    Scan<NW> r;
    r.sum = __reduce_add_sync(WFULL, sum);
    r.key = __reduce_min_sync(WFULL, best);
    const unsigned win = __ballot_sync(WFULL, best == r.key && r.key != kKeyNone);
    const int src = win ? __ffs(win) - 1 : 0;
    const int ci = __shfl_sync(WFULL, bi, src);
    __syncwarp();
    r.R = (win && ci >= 0) ? stk[base + ci].R : Bits<NW>::zero();
    return r;
}

template <int NW>
__device__ void write_best(const WParams<NW>& P, int pair, const Lv<NW>& w, int d, int v, int u, int lane) {
    constexpr int N = 64 * NW;
    uint16_t* slot = P.best + ((size_t)pair * (N + 1) + (d + 1)) * N;
    for (int i = lane; i < d; i += 32) slot[i] = (uint16_t)((w.Mg[i] << 8) | w.Mh[i]);
    if (lane == 0) slot[d] = (uint16_t)((v << 8) | u);
}

template <int NW>
__device__ void post_exit_tokens(const WParams<NW>& P, int count, int lane) {
    count = max(0, count - P.withhold_exit);
    u64 t0 = 0;
    if (lane == 0) t0 = atomicAdd(&P.ctl->q_tail, (u64)count);
    t0 = shfl64(t0, 0);
    bool ok = true;
    for (int i = lane; i < count; i += 32) {
        const u64 t = t0 + i;
        if (!wait_seq(P.qseq + (t & (P.qcap - 1)), t, P.spin_limit)) { ok = false; break; }
        P.queue[t & (P.qcap - 1)].h.pair = -1;
        __threadfence();
        P.qseq[t & (P.qcap - 1)] = t + 1;
    }
    if (!__all_sync(WFULL, ok) && lane == 0) atomicCAS(&P.ctl->error, 0, MCS_ERR_DEVICE_STALL);
}

template <int NW>
__device__ void finalize_pair(const WParams<NW>& P, int pair, int lane) {
    constexpr int N = 64 * NW;
    __threadfence();
    PairState& ps = P.state[pair];
    const WGraph<NW>& pg = P.graphs[pair];
    int status = 0, k = 0, ab = 0;
    if (lane == 0) { status = vload(&ps.status); ab = vload(&ps.abort); k = vload(&ps.inc); }
    status = __shfl_sync(WFULL, status, 0);
    k = __shfl_sync(WFULL, k, 0);
    ab = __shfl_sync(WFULL, ab, 0);
    if (status == MCS_PENDING) {
        if (k < 0 || k > N) k = 0;
        status = ab == 1 ? MCS_TIMEOUT : MCS_OK;
        if (P.out_map) {
            const uint16_t* slot = P.best + ((size_t)pair * (N + 1) + k) * N;
            for (int i = lane; i < k; i += 32) {
                const uint16_t e = vload(slot + i);
                const int gg = __ldcg(&pg.permG[e >> 8]), h = __ldcg(&pg.permH[e & 0xff]);
                P.out_map[(size_t)pair * MCS_MAX_N + gg] = (int16_t)h;
            }
        }
    } else {
        k = 0;
    }
    int last = 0;
    if (lane == 0) {
        const u64 now = gtimer();
        if (P.out_size) P.out_size[pair] = k;
        if (P.out_nodes) P.out_nodes[pair] = vload(&ps.nodes);
        const u64 t0 = vload(&ps.t_start);
        if (P.out_usec) P.out_usec[pair] = t0 ? (float)((now - t0) * 1e-3) : 0.f;
        __threadfence();
        if (P.out_status) P.out_status[pair] = status;
        ps.status = status;
        __threadfence();
        last = atomicSub(&P.ctl->remaining, 1) == 1;
        atomicMax(&P.ctl->last_progress, now);
    }
    last = __shfl_sync(WFULL, last, 0);
    if (last) post_exit_tokens<NW>(P, P.max_warps, lane);
    __syncwarp();
}

template <int NW>
__device__ __forceinline__ void end_task(const WParams<NW>& P, int pair, u64& nodes, int lane) {
    int last = 0;
    if (lane == 0) {
        if (nodes) atomicAdd(&P.state[pair].nodes, nodes);
        __threadfence();
        last = atomicSub(&P.state[pair].open, 1) == 1;
    }
    nodes = 0;
    last = __shfl_sync(WFULL, last, 0);
    if (last) finalize_pair<NW>(P, pair, lane);
}

// Work sharing: hands the upper part of the remaining candidates of the
// shallowest open level (or, with one left, the rest of the level with its
// "v unmatched" branch) to a waiting searcher.  False if the bounded wait
// for a ring slot expired.
template <int NW>
__device__ bool donate(const WParams<NW>& P, int pair, int d0, Top<NW>& t, int inc, const Lv<NW>& w,
                       Cls<NW>* stk, int lane, unsigned& donated) {
    Control* ctl = P.ctl;
    const uint32_t qmask = P.qcap - 1;
    if (lane == 0) {
        w.rrem[t.d] = t.rrem;
        w.info[t.d] = pack_info(t.base, t.C, t.v, t.flags, t.bound);
    }
    __syncwarp();
    int ds = -1;
    for (int off = d0; off <= t.d && ds < 0; off += 32) {
        const int d = off + lane;
        bool open = false;
        if (d <= t.d) {
            const u64 inf = w.info[d];
            const int fl = (int)((inf >> 37) & 3), bd = (int)((inf >> 39) & 0x1ff);
            open = (w.rrem[d].any() || (fl & kTaskPending)) && bd > inc;
        }
        const unsigned m = __ballot_sync(WFULL, open);
        if (m) ds = off + __ffs(m) - 1;
    }
    if (ds < 0) return true;
    const u64 inf = w.info[ds];
    const Bits<NW> rr = w.rrem[ds];
    const int fl = (int)((inf >> 37) & 3);
    const int k = rr.popc();
    Bits<NW> give = rr;
    int gflags = 0;
    if (k >= 2) {
        const int keep = min(k - 1, max(1, (k * P.steal_keep_q4 + 3) / 4));
        for (int j = 0; j < keep; ++j) give.clear(give.low());
    } else {
        gflags = fl & kTaskPending;
    }
    if (!(ds < t.d || k >= 2)) return true;
    u64 ticket = 0;
    int ok = 0;
    if (lane == 0) {
        ticket = atomicAdd(&ctl->q_tail, 1ull);
        atomicAdd(&P.state[pair].open, 1);
        ok = wait_seq(P.qseq + (ticket & qmask), ticket, P.spin_limit) ? 1 : -1;
    }
    ok = __shfl_sync(WFULL, ok, 0);
    if (ok < 0) {
        if (lane == 0) atomicCAS(&ctl->error, 0, MCS_ERR_DEVICE_STALL);
        return false;
    }
    ticket = shfl64(ticket, 0);
    WTask<NW>* dst = P.queue + (ticket & qmask);
    const int C = (int)((inf >> 20) & 0x1ff);
    const int bs = (int)(inf & 0xfffff);
    for (int i = lane; i < C; i += 32) dst->cls[i] = stk[bs + i];
    for (int i = lane; i < ds; i += 32) { dst->Mg[i] = w.Mg[i]; dst->Mh[i] = w.Mh[i]; }
    if (lane == 0) {
        dst->h.pair = pair;
        dst->h.depth = ds;
        dst->h.C = C;
        dst->h.v = (int)((inf >> 29) & 0xff);
        dst->rrem = give;
        dst->h.flags = gflags;
        dst->h.bound = (int)((inf >> 39) & 0x1ff);
        w.rrem[ds] = rr.andnot(give);
        w.info[ds] = (inf & ~(3ull << 37)) | ((u64)(fl & ~gflags) << 37);
    }
    __syncwarp();
    __threadfence();
    if (lane == 0) {
        P.qseq[ticket & qmask] = ticket + 1;
        atomicMax(&ctl->last_progress, gtimer());
    }
    __syncwarp();
    ++donated;
    if (ds == t.d) {
        t.rrem = rr.andnot(give);
        t.flags = fl & ~gflags;
    }
    return true;
}

template <bool DIR, int NW>
__global__ void __launch_bounds__(128) wide_search_kernel(WParams<NW> P) {
    constexpr int N = 64 * NW;
    extern __shared__ __align__(16) unsigned char smem[];
    const int lane = threadIdx.x & 31;
    const int wib = threadIdx.x >> 5;
    const int wid = blockIdx.x * (blockDim.x >> 5) + wib;
    if (wid >= P.max_warps) return;                    // the whole warp leaves
    unsigned char* base = smem + (size_t)wib * P.level_bytes;
    Lv<NW> w;
    w.rrem = reinterpret_cast<Bits<NW>*>(base);
    w.info = reinterpret_cast<u64*>(base + (N + 1) * 8 * NW);
    w.Mg = base + (N + 1) * (8 * NW + 8);
    w.Mh = w.Mg + N;
    Cls<NW>* stk = P.gstack + (size_t)wid * P.stack_entries;
    Control* ctl = P.ctl;
    const bool level_prune = (P.flags & MCS_NO_LEVEL_PRUNE) == 0;
    const uint32_t qmask = P.qcap - 1;
    u64 nodes = 0;
    unsigned tick = 0;
    unsigned cvisits = 0, pruned = 0, donated = 0, stolen = 0;
    while (true) {
        int got = 0;
        u64 qh = 0;
        if (lane == 0) {
            qh = atomicAdd(&ctl->q_head, 1ull);
            const u64* seq = P.qseq + (qh & qmask);
            for (int it = 0; got == 0; ++it) {
                if (vload(seq) == qh + 1) { got = 1; break; }
                if ((it & 63) == 63) {
                    if (vload(&ctl->error) != 0) { got = -1; break; }
                    const u64 now = gtimer(), lp = vload(&ctl->last_progress);
                    if (now > lp && now - lp > P.stall_ns) {
                        atomicCAS(&ctl->error, 0, MCS_ERR_DEVICE_STALL);
                        got = -1;
                        break;
                    }
                }
                __nanosleep(128u << min(it >> 2, 6));
            }
        }
        got = __shfl_sync(WFULL, got, 0);
        qh = shfl64(qh, 0);
        if (got < 0) break;
        __threadfence();
        const WTask<NW>* task = P.queue + (qh & qmask);
        int pair = 0, tflags = 0;
        if (lane == 0) { pair = vload(&task->h.pair); tflags = vload(&task->h.flags); }
        pair = __shfl_sync(WFULL, pair, 0);
        tflags = __shfl_sync(WFULL, tflags, 0);
        if (pair < 0 || pair >= P.npairs) {                // exit token
            __syncwarp();
            if (lane == 0) P.qseq[qh & qmask] = qh + P.qcap;
            break;
        }
        const bool fresh = (tflags & kTaskFresh) != 0;
        PairState& ps = P.state[pair];
        const WGraph<NW>& pg = P.graphs[pair];
        int pstat = 0;
        if (lane == 0) pstat = vload(&ps.status);
        pstat = __shfl_sync(WFULL, pstat, 0);
        if (fresh && pstat != MCS_PENDING) {               // malformed input
            __syncwarp();
            if (lane == 0) { P.qseq[qh & qmask] = qh + P.qcap; ps.open = 0; }
            finalize_pair<NW>(P, pair, lane);
            continue;
        }
        if (fresh && lane == 0) {
            const u64 now = gtimer();
            ps.t_start = now;
            ps.deadline = now + P.timeout_ns;
            atomicMax(&ctl->last_progress, now);
        }
        Top<NW> t;
        if (!fresh) {
            int hd4[4] = {0, 0, 0, 0};
            if (lane == 0) {
                hd4[0] = vload(&task->h.depth);
                hd4[1] = vload(&task->h.C);
                hd4[2] = vload(&task->h.v);
                hd4[3] = vload(&task->h.bound);
            }
            t.d = __shfl_sync(WFULL, hd4[0], 0);
            t.C = __shfl_sync(WFULL, hd4[1], 0);
            t.v = __shfl_sync(WFULL, hd4[2], 0);
            t.bound = __shfl_sync(WFULL, hd4[3], 0);
            t.d = min(max(t.d, 0), N - 1);
            t.C = min(max(t.C, 0), N);
            t.rrem = ldcg(&task->rrem);                    // written before the slot was published
            t.flags = tflags;
            for (int i = lane; i < t.d; i += 32) { w.Mg[i] = __ldcg(&task->Mg[i]); w.Mh[i] = __ldcg(&task->Mh[i]); }
            for (int i = lane; i < t.C; i += 32) stk[i] = ldcg(&task->cls[i]);
            ++stolen;
        } else {
            t.d = 0;
            t.C = __ldcg(&pg.C0);
            for (int i = lane; i < t.C; i += 32) stk[i] = ldcg(&pg.root[i]);
        }
        __syncwarp();
        if (lane == 0) {
            __threadfence();
            P.qseq[qh & qmask] = qh + P.qcap;              // release the slot
        }
        t.base = 0;
        const int d0 = t.d;
        int inc = 0, ab0 = 0;
        if (lane == 0) { inc = vload(&ps.inc); ab0 = vload(&ps.abort); }
        inc = __shfl_sync(WFULL, inc, 0);
        ab0 = __shfl_sync(WFULL, ab0, 0);
        if (ab0) {
            end_task<NW>(P, pair, nodes, lane);
            continue;
        }
        if (fresh) {
            ++nodes;
            cvisits += t.C;
            const Scan<NW> sc = scan_level<NW>(stk, 0, t.C, -1, lane);
            t.bound = sc.sum;
            if (t.bound <= inc) {
                end_task<NW>(P, pair, nodes, lane);
                continue;
            }
            t.v = sc.key & 0xff;
            t.rrem = sc.R;
            t.flags = kTaskPending;
        }
        int p_inc = 0, p_abort = 0, p_hungry = 0;
        while (t.d >= d0) {
            ++tick;
            if ((tick & P.poll_mask) == 0 && lane == 0) {
                p_inc = vload(&ps.inc);
                p_abort = vload(&ps.abort);
                p_hungry = vload(&ctl->q_head) > vload(&ctl->q_tail);
                if (!p_abort && (tick & 255) == 0 && gtimer() > vload(&ps.deadline)) {
                    ps.abort = 1;
                    p_abort = 1;
                }
                if (cvisits >= (1u << 31)) { atomicAdd(&ctl->class_visits, (u64)cvisits); cvisits = 0; }
                if (pruned >= (1u << 31)) { atomicAdd(&ctl->pruned, (u64)pruned); pruned = 0; }
            }
            if ((tick & P.poll_mask) == (P.poll_mask + 1) / 2) {
                inc = max(inc, __shfl_sync(WFULL, p_inc, 0));
                const int ab = __shfl_sync(WFULL, p_abort, 0);
                const int hungry = __shfl_sync(WFULL, p_hungry, 0);
                if (ab) break;
                if (hungry && !donate<NW>(P, pair, d0, t, inc, w, stk, lane, donated)) break;
            }
            if ((level_prune && t.bound <= inc) || (!t.rrem.any() && !(t.flags & kTaskPending))) {
                --t.d;
                if (t.d >= d0) load_level<NW>(w, t.d, t);
                continue;
            }
            if (!t.rrem.any()) {
                // "v stays unmatched": same M, v leaves its class
                ++nodes;
                cvisits += t.C;
                const Scan<NW> sc = scan_level<NW>(stk, t.base, t.C, t.v, lane);
                __syncwarp();
                t.bound = t.d + sc.sum;
                if (t.bound <= inc) {
                    t.flags = 0;
                } else {
                    t.v = sc.key & 0xff;
                    t.rrem = sc.R;
                    t.flags = kTaskPending;
                }
                continue;
            }
            // child (v, u): filterDomain (Table 1) + Eq. 1
            const int u = t.rrem.low();
            t.rrem.clear(u);
            ++nodes;
            cvisits += t.C;
            const int v = t.v;
            const Bits<NW> vb = Bits<NW>::one(v), ub = Bits<NW>::one(u);
            const Bits<NW> gB = pg.gout[v], hB = pg.hout[u];
            Bits<NW> gA = Bits<NW>::zero(), hA = Bits<NW>::zero();
            if (DIR) { gA = pg.gin[v]; hA = pg.hin[u]; }
            const int dm = t.d + 1;
            const int cbase = t.base + t.C;
            int sum = 0;
            unsigned best = kKeyNone;
            int bidx = -1;                                 // class * 4 + part of the best key
            for (int i0 = 0; i0 < t.C; i0 += 32) {
                const int i = i0 + lane;
                if (i < t.C) {
                    const Cls<NW> c = stk[t.base + i];
                    const Bits<NW> L = c.L.andnot(vb), R = c.R.andnot(ub);
                    if (DIR) {
                        const Bits<NW> la = L & gA, lb = L & gB, ra = R & hA, rb = R & hB;
                        const Bits<NW> lp[4] = {L.andnot(la | lb), la.andnot(lb), lb.andnot(la), la & lb};
                        const Bits<NW> rp[4] = {R.andnot(ra | rb), ra.andnot(rb), rb.andnot(ra), ra & rb};
#pragma unroll
                        for (int k = 0; k < 4; ++k) {
                            const int a = lp[k].popc(), b = rp[k].popc();
                            const int m = min(a, b);
                            sum += m;
                            const unsigned key = m ? (((unsigned)max(a, b) << 8) | (unsigned)lp[k].low()) : kKeyNone;
                            if (key < best) { best = key; bidx = i * 4 + k; }
                        }
                    } else {
                        const Bits<NW> l1 = L & gB, r1 = R & hB, l0 = L ^ l1, r0 = R ^ r1;
                        const int a1 = l1.popc(), b1 = r1.popc(), a0 = l0.popc(), b0 = r0.popc();
                        const int m1 = min(a1, b1), m0 = min(a0, b0);
                        sum += m1 + m0;
                        const unsigned k1 = m1 ? (((unsigned)max(a1, b1) << 8) | (unsigned)l1.low()) : kKeyNone;
                        const unsigned k0 = m0 ? (((unsigned)max(a0, b0) << 8) | (unsigned)l0.low()) : kKeyNone;
                        if (k1 < best) { best = k1; bidx = i * 4 + 1; }
                        if (k0 < best) { best = k0; bidx = i * 4 + 0; }
                    }
                }
            }
            sum = __reduce_add_sync(WFULL, sum);
            if (dm > inc) {
                int old = 0;
                if (lane == 0) old = atomicMax(&ps.inc, dm);
                old = __shfl_sync(WFULL, old, 0);
                if (old < dm) {
                    write_best<NW>(P, pair, w, t.d, v, u, lane);
                    inc = dm;
                } else {
                    inc = old;
                }
            }
            if (dm + sum <= inc) { ++pruned; continue; }
            const unsigned kmin = __reduce_min_sync(WFULL, best);
            const unsigned win = __ballot_sync(WFULL, best == kmin);
            const int bsel = __shfl_sync(WFULL, bidx, win ? __ffs(win) - 1 : 0);
            // descend: the child's classes, compacted onto the stack (the
            // chosen class's R side is the new level's candidate set)
            int pos = cbase;
            int cpos = -1;                                 // stack entry of the chosen class
            for (int i0 = 0; i0 < t.C; i0 += 32) {
                const int i = i0 + lane;
                Bits<NW> L = Bits<NW>::zero(), R = Bits<NW>::zero();
                if (i < t.C) {
                    const Cls<NW> c = stk[t.base + i];
                    L = c.L.andnot(vb);
                    R = c.R.andnot(ub);
                }
                auto emit = [&](const Bits<NW>& l, const Bits<NW>& r, int part) {
                    const bool keep = l.any() && r.any();
                    const unsigned mk = __ballot_sync(WFULL, keep);
                    const int q = pos + __popc(mk & lanemask_lt());
                    if (keep) {
                        Cls<NW> c;
                        c.L = l;
                        c.R = r;
                        stk[q] = c;
                        if (i * 4 + part == bsel) cpos = q;
                    }
                    pos += __popc(mk);
                };
                if (DIR) {
                    const Bits<NW> la = L & gA, lb = L & gB, ra = R & hA, rb = R & hB;
                    emit(L.andnot(la | lb), R.andnot(ra | rb), 0);
                    emit(la.andnot(lb), ra.andnot(rb), 1);
                    emit(lb.andnot(la), rb.andnot(ra), 2);
                    emit(la & lb, ra & rb, 3);
                } else {
                    const Bits<NW> l1 = L & gB, r1 = R & hB;
                    emit(l1, r1, 1);
                    emit(L ^ l1, R ^ r1, 0);
                }
            }
            const unsigned cw = __ballot_sync(WFULL, cpos >= 0);
            const int chosen = __shfl_sync(WFULL, cpos, cw ? __ffs(cw) - 1 : 0);
            if (lane == 0) {
                w.Mg[t.d] = (uint8_t)v;
                w.Mh[t.d] = (uint8_t)u;
                w.rrem[t.d] = t.rrem;
                w.info[t.d] = pack_info(t.base, t.C, t.v, t.flags, t.bound);
            }
            __syncwarp();
            t.d = dm;
            t.base = cbase;
            t.C = pos - cbase;
            t.v = kmin & 0xff;
            t.rrem = stk[chosen].R;
            t.flags = kTaskPending;
            t.bound = dm + sum;
        }
        end_task<NW>(P, pair, nodes, lane);
    }
    if (lane == 0) {
        if (cvisits) atomicAdd(&ctl->class_visits, (u64)cvisits);
        if (pruned) atomicAdd(&ctl->pruned, (u64)pruned);
        if (donated) atomicAdd(&ctl->donated, (u64)donated);
        if (stolen) atomicAdd(&ctl->stolen, (u64)stolen);
    }
}

}  // namespace mcsw

// ---------------------------------------------------------------------------
// host side (called by mcs_api.cu)
// ---------------------------------------------------------------------------
namespace {

template <int NW>
int wide_run(mcs_ctx* c, int npairs, const int32_t* d_n, const int64_t* d_adj_off, const uint8_t* d_adj,
             const int64_t* d_lab_off, const int32_t* d_labels, const int32_t* d_order, uint32_t flags,
             double timeout_s, int max_min_n, int32_t* d_size, int32_t* d_status, uint64_t* d_nodes,
             int16_t* d_map, float* d_usec, cudaStream_t s, bool timed) {
    using namespace mcsw;
    constexpr int N = 64 * NW;
    const bool directed = (flags & MCS_DIRECTED) != 0;
    constexpr int kWarpsPerBlock = 4;
    const int lb = level_bytes<NW>();
    const int smem = kWarpsPerBlock * lb;
    auto* k = directed ? wide_search_kernel<true, NW> : wide_search_kernel<false, NW>;
    if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, smem) != cudaSuccess) {
        cudaGetLastError();
        return MCS_ERR_UNSUPPORTED;
    }
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, kWarpsPerBlock * 32, smem) != cudaSuccess ||
        per_sm <= 0) {
        cudaGetLastError();
        return MCS_ERR_UNSUPPORTED;
    }
    if (c->blocks_per_sm > 0) per_sm = std::min(per_sm, c->blocks_per_sm);
    int blocks = c->sms * per_sm;
    int warps = blocks * kWarpsPerBlock;
    if (c->max_warps > 0) {
        warps = std::min(warps, c->max_warps);
        blocks = (warps + kWarpsPerBlock - 1) / kWarpsPerBlock;
    }
    // a level of a search over graphs of at most m vertices per pair side
    // holds at most m - d classes, so a warp's stack holds at most
    // m (m + 1) / 2 entries (m = the largest min(n_G, n_H) of the batch)
    const int m = std::min(std::max(max_min_n, 1), N);
    const size_t stack = (size_t)m * (m + 1) / 2 + 32;
    // arenas (grow-only, per word count)
    auto& A = c->wide[NW == 2 ? 0 : 1];
    auto grow = [&](void*& p, size_t& cap, size_t need) -> int {
        if (need <= cap && p) return 0;
        if (p) cudaFree(p);
        p = nullptr;
        cap = 0;
        if (fault_alloc_now(c) || cudaMalloc(&p, need) != cudaSuccess) {
            cudaGetLastError();
            p = nullptr;
            return MCS_ERR_NOMEM;
        }
        cap = need;
        return 0;
    };
    uint32_t q = 1024;
    while (q < (uint32_t)(4 * warps + npairs)) q <<= 1;
    int rc;
    if ((rc = grow(A.graphs, A.graphs_cap, sizeof(WGraph<NW>) * (size_t)npairs)) ||
        (rc = grow(A.state, A.state_cap, sizeof(PairState) * (size_t)npairs)) ||
        (rc = grow(A.best, A.best_cap, sizeof(uint16_t) * (size_t)npairs * (N + 1) * N)) ||
        (rc = grow(A.queue, A.queue_cap, sizeof(WTask<NW>) * (size_t)q)) ||
        (rc = grow(A.qseq, A.qseq_cap, sizeof(u64) * (size_t)q)) ||
        (rc = grow(A.gstack, A.gstack_cap, sizeof(Cls<NW>) * stack * (size_t)warps)) ||
        (rc = grow(A.ctl, A.ctl_cap, sizeof(Control))))
        return rc;
    WParams<NW> P;
    memset(&P, 0, sizeof(P));
    P.npairs = npairs;
    P.flags = flags;
    P.n = d_n;
    P.adj_off = d_adj_off;
    P.adj = d_adj;
    P.lab_off = d_lab_off;
    P.labels = d_labels;
    P.order = d_order;
    P.graphs = (WGraph<NW>*)A.graphs;
    P.state = (PairState*)A.state;
    P.best = (uint16_t*)A.best;
    P.ctl = (Control*)A.ctl;
    P.queue = (WTask<NW>*)A.queue;
    P.qseq = (u64*)A.qseq;
    P.qcap = q;
    P.gstack = (Cls<NW>*)A.gstack;
    P.stack_entries = stack;
    P.max_warps = warps;
    P.level_bytes = lb;
    const double tmo = timeout_s > 0 ? std::min(timeout_s, 3600.0) : 3600.0;
    P.timeout_ns = (u64)(tmo * 1e9);
    P.stall_ns = c->fault_stall_ms > 0 ? (u64)c->fault_stall_ms * 1000000ull : P.timeout_ns + 2000000000ull;
    P.poll_mask = (uint32_t)c->poll_nodes - 1;
    P.steal_keep_q4 = c->steal_keep_q4;
    P.spin_limit = (uint32_t)c->fault_spin;
    P.withhold_exit = c->fault_withhold;
    P.block_ring = c->fault_block_ring;
    P.out_size = d_size;
    P.out_status = d_status;
    P.out_nodes = reinterpret_cast<u64*>(d_nodes);
    P.out_map = (flags & MCS_NO_MAPPING) ? nullptr : d_map;
    P.out_usec = d_usec;
    const int pblocks = std::max(1, (npairs + 3) / 4);
    wide_pack_kernel<NW><<<pblocks, 128, 0, s>>>(P);
    if (cudaGetLastError() != cudaSuccess) return MCS_ERR_CUDA;
    if (timed && cudaEventRecord(c->ev0, s) != cudaSuccess) return MCS_ERR_CUDA;
    k<<<blocks, kWarpsPerBlock * 32, smem, s>>>(P);
    if (cudaGetLastError() != cudaSuccess) return MCS_ERR_CUDA;
    if (timed && cudaEventRecord(c->ev1, s) != cudaSuccess) return MCS_ERR_CUDA;
    c->stats[5] = warps;
    c->wide_ctl = A.ctl;
    return 0;
}

}  // namespace

// Enqueues pack + search of a batch of pairs with up to 256 vertices per
// graph.  max_min_n: the largest min(n_G, n_H) of the batch (it sizes the
// class stacks), or 0 when unknown (then the largest the word count allows).
int wide_run_device(mcs_ctx* c, int npairs, const int32_t* d_n, const int64_t* d_adj_off, const uint8_t* d_adj,
                    const int64_t* d_lab_off, const int32_t* d_labels, const int32_t* d_order, uint32_t flags,
                    double timeout_s, int max_n, int max_min_n, int32_t* d_size, int32_t* d_status,
                    uint64_t* d_nodes, int16_t* d_map, float* d_usec, cudaStream_t s, bool timed) {
    if (npairs <= 0) return npairs < 0 ? MCS_ERR_ARG : 0;
    if (max_n <= 0) max_n = 256;
    if (max_min_n <= 0) max_min_n = max_n;
    if (max_n <= 128)
        return wide_run<2>(c, npairs, d_n, d_adj_off, d_adj, d_lab_off, d_labels, d_order, flags, timeout_s,
                           max_min_n, d_size, d_status, d_nodes, d_map, d_usec, s, timed);
    return wide_run<4>(c, npairs, d_n, d_adj_off, d_adj, d_lab_off, d_labels, d_order, flags, timeout_s, max_min_n,
                       d_size, d_status, d_nodes, d_map, d_usec, s, timed);
}

void wide_free(mcs_ctx* c) {
    for (auto& A : c->wide) {
        void* ps[] = {A.graphs, A.state, A.best, A.queue, A.qseq, A.gstack, A.ctl};
        for (void* p : ps) cudaFree(p);
        A = WideArena();
    }
    c->wide_ctl = nullptr;
}
