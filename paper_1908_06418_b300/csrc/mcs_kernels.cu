// Device kernels of the B300 McSplit library.
//
//   pack_kernel    validates each input graph, renumbers its vertices (by
//                  descending degree, total in+out degree when directed,
//                  Section IV-A; or by a caller-supplied key), packs the
//                  adjacency into 64-bit row bitsets and builds the initial
//                  label classes (one per label + self-loop value present in
//                  both graphs).
//   search_kernel  persistent McSplit branch and bound (Section II-B,
//                  Algorithm 1, Eq. 1).  One warp runs one depth-first search;
//                  the label classes of a node are spread over the lanes (one
//                  or two per lane), so filterDomain (Table 1) is a warp-wide
//                  AND/popcount, the bound of Eq. 1 is one warp add-reduction
//                  and the class choice one warp min-reduction.  Work moves
//                  between warps through a task ring in HBM; incumbents are
//                  per-pair atomicMax counters.
//
// Every device-side wait is bounded (iteration count and globaltimer) and
// reports MCS_ERR_DEVICE_STALL through Control::error instead of trapping.
#include <atomic>
#include <type_traits>
#include "mcs_internal.cuh"
#include "../../include/mcs.h"

namespace mcsk {

#define FULL 0xffffffffu

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

// Index checks of the MCS_DEBUG_BOUNDS build: a violation is recorded in the
// Control block (first code / value / line, plus a count) and the caller
// skips or clamps the access, so a bad index never becomes a memory fault.
#ifdef MCS_DEBUG_BOUNDS
__device__ __noinline__ void dbg_fail(Control* c, int code, long long val, int line) {
    if (atomicAdd(&c->dbg_count, 1ull) == 0) {
        c->dbg_code = (u64)code;
        c->dbg_val = (u64)val;
        c->dbg_line = (u64)line;
    }
}
#define DBG_OK(ctl, cond, code, val) ((cond) ? true : (dbg_fail((ctl), (code), (long long)(val), __LINE__), false))
#else
#define DBG_OK(ctl, cond, code, val) (true)
#endif

// Loads that bypass L1: task slots are written by other SMs.
__device__ __forceinline__ ulonglong2 ld_cg(const ulonglong2* p) {
    ulonglong2 r;
    asm volatile("ld.global.cg.v2.u64 {%0, %1}, [%2];" : "=l"(r.x), "=l"(r.y) : "l"(p));
    return r;
}
__device__ __forceinline__ uint8_t ld_cg(const uint8_t* p) {
    unsigned short r;
    asm volatile("ld.global.cg.u8 %0, [%1];" : "=h"(r) : "l"(p));
    return (uint8_t)r;
}

__device__ __forceinline__ u64 shfl_xor64(u64 x, int m) {
    unsigned lo = (unsigned)x, hi = (unsigned)(x >> 32);
    lo = __shfl_xor_sync(FULL, lo, m);
    hi = __shfl_xor_sync(FULL, hi, m);
    return ((u64)hi << 32) | lo;
}
__device__ __forceinline__ u64 shfl64(u64 x, int src) {
    unsigned lo = (unsigned)x, hi = (unsigned)(x >> 32);
    lo = __shfl_sync(FULL, lo, src);
    hi = __shfl_sync(FULL, hi, src);
    return ((u64)hi << 32) | lo;
}

// ---------------------------------------------------------------------------
// pack kernel: one warp per pair
// ---------------------------------------------------------------------------
struct GraphIn {
    int n;
    const uint8_t* a;
    const int32_t* lab;
};

// Component ordering of the static order below: a before b when a's
// rows/columns ratio is larger (r/0 with r > 0 is infinite, 0/0 is 0), then
// when a is larger, then when its lowest vertex is lower.
struct CompKey { int rows, cols, size, low; };
__device__ __forceinline__ bool comp_ratio_gt(const CompKey& a, const CompKey& b) {
    const bool ia = a.cols == 0 && a.rows > 0, ib = b.cols == 0 && b.rows > 0;
    if (ia || ib) return ia && !ib;
    const int an = a.cols ? a.rows : 0, ad = a.cols ? a.cols : 1;
    const int bn = b.cols ? b.rows : 0, bd = b.cols ? b.cols : 1;
    return an * bd > bn * ad;
}
__device__ __forceinline__ bool comp_before(const CompKey& a, const CompKey& b) {
    if (comp_ratio_gt(a, b)) return true;
    if (comp_ratio_gt(b, a)) return false;
    if (a.size != b.size) return a.size > b.size;
    return a.low < b.low;
}

// The static vertex order of the portfolio modifications (Section IV-A), for
// MCS_ORDER_HR: weakly connected components in decreasing rows/columns ratio
// (rows: vertices with an out-arc, columns: with an in-arc), then size, then
// lowest vertex; inside a component, repeatedly the active column with a
// nonzero in the most of the shortest nonempty active rows (ties: lowest
// vertex) takes the next position; when no active row is left the remaining
// active columns follow in increasing order, then the component's vertices
// without an in-arc.  One warp; lane l holds vertices l and l + 32 (orow /
// icol: out- and in-neighbours without the vertex itself).  pos[s] receives
// the position of vertex lane + 32 s.  scratch: 64 words of shared memory.
// Every loop is bounded by the vertex count.
__device__ void hr_positions(int n, const u64 (&orow)[2], const u64 (&icol)[2], u64* scratch, int lane,
                             int (&pos)[2]) {
    u64 R[2];
    for (int s = 0; s < 2; ++s) {
        const int x = lane + 32 * s;
        R[s] = x < n ? (orow[s] | icol[s] | (1ull << x)) : 0ull;
        if (x < n) scratch[x] = R[s];
    }
    __syncwarp();
    // reach sets by repeated squaring: paths of up to 2^6 = 64 arcs
    for (int it = 0; it < 6; ++it) {
        u64 nr[2];
        for (int s = 0; s < 2; ++s) {
            u64 acc = R[s], m = R[s];
            while (m) { const int y = __ffsll((long long)m) - 1; m &= m - 1; acc |= scratch[y]; }
            nr[s] = acc;
        }
        __syncwarp();
        for (int s = 0; s < 2; ++s) {
            const int x = lane + 32 * s;
            R[s] = nr[s];
            if (x < n) scratch[x] = nr[s];
        }
        __syncwarp();
    }
    const u64 rownz = (u64)__ballot_sync(FULL, lane < n && orow[0] != 0) |
                      ((u64)__ballot_sync(FULL, lane + 32 < n && orow[1] != 0) << 32);
    const u64 colnz = (u64)__ballot_sync(FULL, lane < n && icol[0] != 0) |
                      ((u64)__ballot_sync(FULL, lane + 32 < n && icol[1] != 0) << 32);
    CompKey ck[2];
    for (int s = 0; s < 2; ++s) {
        ck[s].size = __popcll(R[s]);
        ck[s].rows = __popcll(R[s] & rownz);
        ck[s].cols = __popcll(R[s] & colnz);
        ck[s].low = R[s] ? __ffsll((long long)R[s]) - 1 : 64;
    }
    // offset of each vertex's component: sizes of the components ordered before it
    int off[2] = {0, 0};
    for (int j = 0; j < n; ++j) {
        CompKey cj;
        cj.size = __shfl_sync(FULL, ck[j >> 5].size, j & 31);
        cj.rows = __shfl_sync(FULL, ck[j >> 5].rows, j & 31);
        cj.cols = __shfl_sync(FULL, ck[j >> 5].cols, j & 31);
        cj.low = __shfl_sync(FULL, ck[j >> 5].low, j & 31);
        if (cj.low != j) continue;                      // warp-uniform: j represents its component
        for (int s = 0; s < 2; ++s)
            if (lane + 32 * s < n && comp_before(cj, ck[s])) off[s] += cj.size;
    }
    pos[0] = pos[1] = -1;
    int cur = 0;
    for (int comp = 0; cur < n && comp < kMaxN; ++comp) {
        // the component placed next: the one whose offset is cur
        const unsigned b0 = __ballot_sync(FULL, lane < n && off[0] == cur);
        const unsigned b1 = __ballot_sync(FULL, lane + 32 < n && off[1] == cur);
        if (!b0 && !b1) break;                          // (cannot happen: offsets are prefix sums)
        const int src = b0 ? __ffs(b0) - 1 : 32 + __ffs(b1) - 1;
        const u64 cm = shfl64(src < 32 ? R[0] : R[1], src & 31);
        u64 colact = cm & colnz, placed = 0;
        for (int step = 0; colact && step < kMaxN; ++step) {
            int len[2];
            bool act[2];
            for (int s = 0; s < 2; ++s) {
                const int x = lane + 32 * s;
                len[s] = (x < n && ((cm >> x) & 1)) ? __popcll(orow[s] & colact) : 0;
                act[s] = len[s] > 0;
            }
            const unsigned mn = __reduce_min_sync(FULL, (unsigned)min(act[0] ? len[0] : 255, act[1] ? len[1] : 255));
            if (mn == 255) {                            // no active row: the rest of the columns in order
                for (int s = 0; s < 2; ++s) {
                    const int x = lane + 32 * s;
                    if (x < n && ((colact >> x) & 1)) pos[s] = cur + __popcll(colact & ((1ull << x) - 1));
                }
                cur += __popcll(colact);
                placed |= colact;
                colact = 0;
                break;
            }
            const u64 S = (u64)__ballot_sync(FULL, act[0] && len[0] == (int)mn) |
                          ((u64)__ballot_sync(FULL, act[1] && len[1] == (int)mn) << 32);
            unsigned key = 0;
            for (int s = 0; s < 2; ++s) {
                const int x = lane + 32 * s;
                if (x < n && ((colact >> x) & 1))
                    key = max(key, ((unsigned)__popcll(icol[s] & S) << 7) | (unsigned)(127 - x));
            }
            const unsigned best = __reduce_max_sync(FULL, key);
            if (best == 0) break;                       // (cannot happen: colact is not empty)
            const int c = 127 - (int)(best & 127);
            if ((c & 31) == lane) pos[c >> 5] = cur;
            ++cur;
            colact &= ~(1ull << c);
            placed |= 1ull << c;
        }
        const u64 rest = cm & ~placed;                  // vertices without an in-arc, in order
        for (int s = 0; s < 2; ++s) {
            const int x = lane + 32 * s;
            if (x < n && ((rest >> x) & 1)) pos[s] = cur + __popcll(rest & ((1ull << x) - 1));
        }
        cur += __popcll(rest);
    }
    // every position 0..n-1 taken exactly once, else (never expected) the identity order
    u64 mine = 0;
    bool dup = false;
    for (int s = 0; s < 2; ++s) {
        const int x = lane + 32 * s;
        if (x < n) {
            if (pos[s] < 0 || pos[s] >= n) dup = true;
            else mine |= 1ull << pos[s];
        }
    }
    u64 all = mine;
    int total = __popcll(mine);
    for (int o = 16; o > 0; o >>= 1) {
        all |= shfl_xor64(all, o);
        total += __shfl_xor_sync(FULL, total, o);
    }
    const bool good = !__any_sync(FULL, dup) && total == n && all == (n == 64 ? ~0ull : ((1ull << n) - 1));
    if (!good) { pos[0] = lane; pos[1] = lane + 32; }
}

// Lane l handles vertices l and l + 32.  Returns false (warp-uniform) if the
// graph is malformed.  hr: the static order of hr_positions instead of the
// degree order (scratch: 64 words of shared memory).
__device__ bool pack_graph(const GraphIn& g, bool directed, const float* key,
                           u64* rows /* 2 per vertex: out, in */, uint8_t* perm,
                           long long* vkey /* per lane: 2 entries */, int lane, bool hr, u64* scratch) {
    const int n = g.n;
    bool ok = (n >= 0 && n <= kMaxN);
    // content checks: entries 0/1, symmetric when undirected, labels >= 0
    // (the loop trip count is warp-uniform so that every lane reaches the vote)
    for (int b0 = 0; ok && b0 < n * n; b0 += 32) {
        const int idx = b0 + lane;
        bool bad = false;
        if (idx < n * n) {
            uint8_t x = g.a[idx];
            bad = x > 1;
            if (!directed) {
                int i = idx / n, j = idx - i * n;
                bad |= (x != g.a[j * n + i]);
            }
        }
        if (__any_sync(FULL, bad)) ok = false;
    }
    if (g.lab) {
        bool bad = false;
        for (int i = lane; i < n; i += 32) bad |= g.lab[i] < 0;
        if (__any_sync(FULL, bad)) ok = false;
    }
    if (!ok) return false;
    // degree (total degree when directed), loops excluded
    int deg[2];
    float kv[2];
    for (int s = 0; s < 2; ++s) {
        int i = lane + 32 * s;
        int d = 0;
        if (i < n)
            for (int j = 0; j < n; ++j) {
                if (j == i) continue;
                d += g.a[i * n + j];
                if (directed) d += g.a[j * n + i];
            }
        deg[s] = d;
        kv[s] = (key && i < n) ? key[i] : 0.f;
    }
    // rank: earlier if higher degree (or lower caller key), ties to lower index
    int rank[2];
    if (hr) {
        u64 orow[2], icol[2];
        for (int s = 0; s < 2; ++s) {
            const int i = lane + 32 * s;
            u64 o = 0, in = 0;
            if (i < n)
                for (int j = 0; j < n; ++j) {
                    if (j == i) continue;
                    if (g.a[i * n + j]) o |= 1ull << j;
                    if (g.a[j * n + i]) in |= 1ull << j;
                }
            orow[s] = o;
            icol[s] = directed ? in : o;
        }
        hr_positions(n, orow, icol, scratch, lane, rank);
        __syncwarp();
    } else
    for (int s = 0; s < 2; ++s) {
        int i = lane + 32 * s;
        int r = 0;
        for (int j = 0; j < n; ++j) {
            int dj = __shfl_sync(FULL, deg[j >> 5], j & 31);
            float kj = __shfl_sync(FULL, kv[j >> 5], j & 31);
            bool before;
            if (key) before = (kj < kv[s]) || (kj == kv[s] && j < i);
            else before = (dj > deg[s]) || (dj == deg[s] && j < i);
            r += before ? 1 : 0;
        }
        rank[s] = r;
    }
    for (int s = 0; s < 2; ++s) {
        int i = lane + 32 * s;
        if (i < n) perm[rank[s]] = (uint8_t)i;
    }
    // rows in the new numbering
    for (int s = 0; s < 2; ++s) {
        int i = lane + 32 * s;
        u64 o = 0, in = 0;
        for (int j = 0; j < n; ++j) {
            int rj = __shfl_sync(FULL, rank[j >> 5], j & 31);
            if (i < n && j != i) {
                if (g.a[i * n + j]) o |= 1ull << rj;
                if (g.a[j * n + i]) in |= 1ull << rj;
            }
        }
        if (i < n) {
            rows[2 * rank[s]] = o;
            rows[2 * rank[s] + 1] = directed ? in : o;
            long long lab = g.lab ? (long long)g.lab[i] : 0;
            vkey[s] = lab * 2 + (g.a[i * n + i] ? 1 : 0);   // label + self-loop
        } else {
            vkey[s] = -1;
        }
    }
    return true;
}

// Packs one pair (one warp): validation, renumbering, row bitsets and the
// initial label classes into pg.  skey is 2 x 64 long long of shared scratch.
// Returns false (warp-uniform) when an input graph is malformed.
__device__ bool pack_pair_warp(const GraphIn (&g)[2], bool directed, const float* key0,
                               const float* key1, PairGraph& pg, long long* skey, int lane, bool hr = false) {
    bool ok = true;
    long long vk[2][2];
    for (int side = 0; side < 2 && ok; ++side) {
        if (g[side].n < 0 || g[side].n > kMaxN) { ok = false; break; }
        u64* rows = pg.rows + (side ? 2 * kMaxN : 0);
        uint8_t* perm = side ? pg.permH : pg.permG;
        ok = pack_graph(g[side], directed, side ? key1 : key0, rows, perm, vk[side], lane, hr,
                        reinterpret_cast<u64*>(skey));
    }
    __syncwarp();
    const int nG = g[0].n, nH = g[1].n;
    if (ok) {
        // label keys by new number
        for (int side = 0; side < 2; ++side) {
            const uint8_t* perm = side ? pg.permH : pg.permG;
            const int n = side ? nH : nG;
            // vk[side][s] belongs to original vertex lane + 32 s; place it at its new number
            __syncwarp();
            for (int r = lane; r < kMaxN; r += 32) skey[side * kMaxN + r] = -1;
            __syncwarp();
            for (int r = 0; r < n; ++r) {
                int orig = perm[r];
                long long k = __shfl_sync(FULL, (unsigned long long)vk[side][orig >> 5], orig & 31);
                if (lane == 0) skey[side * kMaxN + r] = k;
            }
            __syncwarp();
        }
        // one class per key present in both graphs; representative = lowest new G number
        int C = 0;
        for (int s = 0; s < 2; ++s) {
            int r = lane + 32 * s;
            long long k = r < nG ? skey[r] : -2;
            u64 L = 0, R = 0;
            bool rep = r < nG;
            for (int j = 0; j < kMaxN; ++j) {
                if (j < nG && skey[j] == k) { L |= 1ull << j; if (j < r) rep = false; }
                if (j < nH && skey[kMaxN + j] == k) R |= 1ull << j;
            }
            bool keep = rep && R != 0;
            unsigned m = __ballot_sync(FULL, keep);
            int pos = C + __popc(m & lanemask_lt());
            if (keep) pg.root[pos] = make_ulonglong2(L, R);
            C += __popc(m);
        }
        if (lane == 0) {
            pg.nG = nG; pg.nH = nH; pg.C0 = C; pg.valid = 1;
        }
    } else if (lane == 0) {
        pg.nG = 0; pg.nH = 0; pg.C0 = 0; pg.valid = 0;
    }
    __syncwarp();
    return ok;
}

__global__ void pack_kernel(PackParams P) {
    __shared__ long long s_key[4][2 * kMaxN];
    const int lane = threadIdx.x & 31;
    const int wib = threadIdx.x >> 5;
    const int p = blockIdx.x * (blockDim.x >> 5) + wib;
    // Ring: tickets 0 .. npairs-1 are the pair roots, published up front in
    // processing order; every other slot i is free for ticket i.
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < P.qcap; i += gridDim.x * blockDim.x) {
        if ((int)i < P.npairs) {
            Task* t = P.queue + i;
            t->h.pair = P.order ? P.order[i] : (int)i;
            t->h.flags = kTaskFresh;
            t->h.depth = 0;
            t->h.C = 0;
            P.qseq[i] = (u64)i + 1;
        } else {
            // failure injection: a slot that never frees up (no ticket matches)
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
    PairGraph& pg = P.graphs[p];
    GraphIn g[2];
    for (int side = 0; side < 2; ++side) {
        const int gi = 2 * p + side;
        g[side].n = P.n[gi];
        g[side].a = P.adj + P.adj_off[gi];
        g[side].lab = (P.labels && P.lab_off && P.lab_off[gi] >= 0) ? P.labels + P.lab_off[gi] : nullptr;
    }
    const float* k0 = P.vscore ? P.vscore + ((size_t)p * 2) * kMaxN : nullptr;
    const float* k1 = P.vscore ? P.vscore + ((size_t)p * 2 + 1) * kMaxN : nullptr;
    // the 32-bit node step holds graphs of at most 32 vertices
    const bool fits = !(P.flags & MCS_WORD32) || (g[0].n <= 32 && g[1].n <= 32);
    const bool ok = pack_pair_warp(g, directed, k0, k1, pg, s_key[wib], lane, (P.flags & MCS_ORDER_HR) != 0) && fits;
    if (lane == 0) {
        PairState& st = P.state[p];
        // top-down: the first goal is min(|V_G|, |V_H|) (Section IV)
        const int kmax = min(max(g[0].n, 0), max(g[1].n, 0));
        const bool td = (P.flags & MCS_TOP_DOWN) && ok && kmax > 0;
        st.floor = td ? kmax - 1 : 0;
        st.cap = td ? kmax : kNoCap;
        st.inc = st.floor;
        st.real = 0;
        st.lo = st.hi = 0;
        st.dead = 0;
        st.live = st.mark = 0;
        st.restarts = 0;
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

cudaError_t launch_pack(const PackParams& p, cudaStream_t s) {
    int blocks = (p.npairs + 3) / 4;
    if (blocks < 1) blocks = 1;
    pack_kernel<<<blocks, 128, 0, s>>>(p);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// search kernel
// ---------------------------------------------------------------------------
constexpr unsigned kKeyNone = 0xFFFFu;
constexpr int kSpinLimit = 1 << 22;   // iterations of a ring-slot wait

// A searcher is a group of GS lanes (GS = 32: one warp; 16 or 8: two or four
// independent depth-first searches per warp).  Every warp-level primitive of
// the search goes through this group: shuffles, votes and reductions carry
// the group's lane mask, so groups of one warp may take different branches.
template <int GS>
struct Grp {
    unsigned mask;      // the group's lanes
    int q;              // lane within the group
    int lane0;          // first lane of the group
    __device__ __forceinline__ explicit Grp(int lane) {
        q = lane & (GS - 1);
        lane0 = lane - q;
        mask = GS == 32 ? FULL : (((1u << GS) - 1u) << lane0);
    }
    __device__ __forceinline__ int shfl(int x, int src) const { return __shfl_sync(mask, x, src, GS); }
    __device__ __forceinline__ unsigned shflu(unsigned x, int src) const { return __shfl_sync(mask, x, src, GS); }
    __device__ __forceinline__ u64 shfl64(u64 x, int src) const {
        unsigned lo = (unsigned)x, hi = (unsigned)(x >> 32);
        lo = __shfl_sync(mask, lo, src, GS);
        hi = __shfl_sync(mask, hi, src, GS);
        return ((u64)hi << 32) | lo;
    }
    // group-relative vote: bit i = lane q == i
    __device__ __forceinline__ unsigned ballot(bool p) const {
        const unsigned b = __ballot_sync(mask, p);
        return GS == 32 ? b : (b >> lane0) & ((1u << GS) - 1u);
    }
    __device__ __forceinline__ bool all(bool p) const { return __all_sync(mask, p); }
    // redux.sync reduces over the lanes of its member mask only
    __device__ __forceinline__ int add(int x) const { return __reduce_add_sync(mask, x); }
    __device__ __forceinline__ unsigned umin(unsigned x) const { return __reduce_min_sync(mask, x); }
    __device__ __forceinline__ void sync() const { __syncwarp(mask); }
    __device__ __forceinline__ unsigned lt() const { return (1u << q) - 1u; }
};

struct WarpSmem {
    const u64* adj;      // PairGraph::rows layout, shared or global
    ulonglong2* lvl;     // per level: {candidates still to try, info} (kSmLvOff)
    ulonglong2* cls;
};
// The mapping prefix entry of depth i: (v << 8) | u of the pair matched there.
__device__ __forceinline__ uint16_t m_entry(u64 info) {
    return (uint16_t)((((info >> 24) & 0xff) << 8) | ((info >> 48) & 0xff));
}

// An adjacency row: shared-memory copy, or the packed pair in global memory
// (read-only for the kernel's lifetime, so through the non-coherent cache).
// In serve mode (COHERENT) slots are repacked while the kernel runs, so rows
// read in place go through L2.
template <bool SM, bool COHERENT = false>
__device__ __forceinline__ u64 adj_row(const u64* rows, int i) {
    if constexpr (SM) return rows[i];
    else if constexpr (COHERENT) return __ldcg(rows + i);
    else return __ldg(rows + i);
}
// Both rows {out, in} of a vertex in one 16-byte load (i = row_gout or row_hout).
template <bool SM, bool COHERENT = false>
__device__ __forceinline__ ulonglong2 adj_row_pair(const u64* rows, int i) {
    const ulonglong2* p = reinterpret_cast<const ulonglong2*>(rows + i);
    if constexpr (SM) return *p;
    else if constexpr (COHERENT) return __ldcg(p);
    else return __ldg(p);
}

__device__ __forceinline__ u64 pack_info(int base, int C, int v, int flags, int bound) {
    return (u64)base | ((u64)C << 16) | ((u64)v << 24) | ((u64)flags << 32) | ((u64)bound << 40);
}

struct Top {                // the cursor of the deepest level, kept in registers
    int d, base, C, v, flags, bound;
    u64 rrem;
};

// A searcher's class stack.  Whole-warp searchers keep its first S entries
// in shared memory and the rest in their global overflow; narrow searchers
// (many per SM, so little shared memory each) keep it all in global memory,
// where the L1 cache holds the top levels that are in use.
template <bool HAS_SM>
struct StackT {
    ulonglong2* sm;          // shared part (HAS_SM)
    ulonglong2* gm;          // global part
    int S;                   // entries in the shared part (0 without one)
#ifdef MCS_DEBUG_BOUNDS
    Control* ctl;
    __device__ __forceinline__ ulonglong2* at(int p) const {
        if (!DBG_OK(ctl, p >= 0 && p < kStackMax, 1, p)) p = 0;
        if constexpr (HAS_SM) return p < S ? sm + p : gm + (p - S);
        else return gm + p;
    }
#else
    __device__ __forceinline__ ulonglong2* at(int p) const {
        if constexpr (HAS_SM) return p < S ? sm + p : gm + (p - S);
        else return gm + p;
    }
#endif
};

// Result of scanning a level's classes (node entry): Eq. 1 sum and the class
// choice.  Key = max(|L|,|R|) << 6 | lowest L vertex (unique per class).
struct Scan {
    int sum;
    unsigned key;
    u64 R;
};

// Bit-set words of the node step.  Pairs whose graphs both have at most 32
// vertices run it on 32-bit words (one hardware popcount per set instead of
// two); the stored rows and classes stay 64-bit (their upper halves are 0).
template <typename W> struct Word;
template <> struct Word<u64> {
    static __device__ __forceinline__ int popc(u64 x) { return __popcll(x); }
    static __device__ __forceinline__ int low(u64 x) { return __ffsll(x) - 1; }   // lowest set bit
};
template <> struct Word<uint32_t> {
    static __device__ __forceinline__ int popc(uint32_t x) { return __popc(x); }
    static __device__ __forceinline__ int low(uint32_t x) { return __ffs(x) - 1; }
};

// Scan the classes of a level (optionally removing v from its class first,
// which is the "v stays unmatched" step) and choose the next branching class.
template <typename W, int GS, typename Stack>
__device__ __forceinline__ Scan scan_level(const Grp<GS>& g, const Stack& st, int base, int C,
                                           int remove_v) {
    int sum = 0;
    unsigned best = kKeyNone;
    W bestR = 0;
    const W vb = remove_v >= 0 ? ((W)1 << remove_v) : (W)0;
    auto one = [&](int i, bool have) {
        ulonglong2* ptr = st.at(base + (have ? i : 0));
        const ulonglong2 c = *ptr;
        W L = have ? (W)c.x : (W)0;
        const W R = have ? (W)c.y : (W)0;
        if (L & vb) {
            L &= ~vb;
            ptr->x = L;
        }
        if (L) {
            const int a = Word<W>::popc(L), b = Word<W>::popc(R);
            sum += min(a, b);
            const unsigned key = ((unsigned)max(a, b) << 6) | (unsigned)Word<W>::low(L);
            if (key < best) { best = key; bestR = R; }
        }
    };
    // slot 0 straight-line (lanes beyond the class count read entry 0 of the
    // level and contribute nothing), further slots when classes outnumber lanes
    one(g.q, g.q < C);
    for (int i0 = GS; i0 < C; i0 += GS) {
        const int i = i0 + g.q;
        if (i < C) one(i, true);
    }
    Scan r;
    r.sum = g.add(sum);
    r.key = g.umin(best);
    const unsigned win = g.ballot(best == r.key && r.key != kKeyNone);
    r.R = win ? g.shfl64((u64)bestR, __ffs(win) - 1) : 0ull;
    return r;
}

// Learned order: the candidate u of `rrem` with the lowest rank in the row
// rk[0..63] (ranks are distinct).  Each lane reads its contiguous 64/GS
// entries of the row with one or two vector loads (the row is 64-byte
// aligned), then the group takes the minimum of (rank << 6 | u).
template <int GS>
__device__ __forceinline__ int learned_pick(const uint8_t* rk, u64 rrem, const Grp<GS>& g) {
    constexpr int C = kMaxN / GS;                      // entries per lane
    const int u0 = g.q * C;
    const u64 bits = (rrem >> u0) & (C == 64 ? ~0ull : ((1ull << (C & 63)) - 1ull));
    unsigned kk = kKeyNone;
    if (bits) {
        uint32_t w[(C + 3) / 4];                       // the lane's ranks, 4 per word
        if constexpr (C == 2) {
            w[0] = __ldg(reinterpret_cast<const unsigned short*>(rk + u0));
        } else if constexpr (C == 4) {
            w[0] = __ldg(reinterpret_cast<const unsigned*>(rk + u0));
        } else if constexpr (C == 8) {
            const uint2 x = __ldg(reinterpret_cast<const uint2*>(rk + u0));
            w[0] = x.x; w[1] = x.y;
        } else {
#pragma unroll
            for (int h = 0; h < C / 16; ++h) {
                const uint4 x = __ldg(reinterpret_cast<const uint4*>(rk + u0) + h);
                w[4 * h] = x.x; w[4 * h + 1] = x.y; w[4 * h + 2] = x.z; w[4 * h + 3] = x.w;
            }
        }
#pragma unroll
        for (int b = 0; b < C; ++b)
            if ((bits >> b) & 1ull) kk = min(kk, (((w[b >> 2] >> (8 * (b & 3))) & 0xffu) << 6) | (unsigned)(u0 + b));
    }
    return (int)(g.umin(kk) & 63u);
}

// Bounded wait for a ring slot's sequence number: `limit` iterations (0:
// kSpinLimit; tests shorten it to make the wait expire).
__device__ __forceinline__ bool wait_seq(const u64* seq, u64 want, uint32_t limit) {
    const uint32_t lim = limit ? limit : (uint32_t)kSpinLimit;
    for (uint32_t it = 0; it < lim; ++it) {
        if (vload(seq) == want) return true;
        if (it > 64) __nanosleep(64);
    }
    return false;
}

template <int GS>
__device__ void write_best(const SearchParams& P, int pair, const WarpSmem& w, int d, int v, int u,
                           const Grp<GS>& g) {
    if (!DBG_OK(P.ctl, d + 1 < kLevels && pair >= 0 && pair < P.npairs, 6, d)) return;
    uint16_t* slot = P.best + ((size_t)pair * kLevels + (d + 1)) * kMaxN;
    for (int i = g.q; i < d; i += GS) slot[i] = m_entry(w.lvl[i].y);
    if (g.q == 0) slot[d] = (uint16_t)((v << 8) | u);
}

// Posts `count` exit tokens (pair = -1) at the tail of the ring: every
// searcher waiting on a ticket at or beyond the tail finds one and leaves.
// (Failure injection withholds P.withhold_exit of them: the searchers left
// without one give up at their idle-wait limit.)
template <int GS>
__device__ void post_exit_tokens(const SearchParams& P, int count, const Grp<GS>& g) {
    count = max(0, count - P.withhold_exit);
    u64 t0 = 0;
    if (g.q == 0) t0 = atomicAdd(&P.ctl->q_tail, (u64)count);
    t0 = g.shfl64(t0, 0);
    bool ok = true;
    for (int i = g.q; i < count; i += GS) {
        const u64 t = t0 + i;
        Task* dst = P.queue + (t & (P.qcap - 1));
        // a slot that never frees up ends this lane's posting (one expired wait
        // per lane at most; the error makes every waiting searcher leave)
        if (!wait_seq(P.qseq + (t & (P.qcap - 1)), t, P.spin_limit)) { ok = false; break; }
        dst->h.pair = -1;
        __threadfence();
        P.qseq[t & (P.qcap - 1)] = t + 1;
    }
    if (!g.all(ok) && g.q == 0) atomicCAS(&P.ctl->error, 0, MCS_ERR_DEVICE_STALL);
}

// Serve mode: the result record in mapped host memory, map built in the
// searcher's shared scratch (64 int16), then a system-scope fence and the
// done ticket.
template <int GS>
__device__ void finalize_served(const SearchParams& P, int pair, int status, int k, const Grp<GS>& g,
                                int16_t* smap) {
    PairState& ps = P.state[pair];
    const PairGraph& pg = P.graphs[pair];
    for (int i = g.q; i < kMaxN; i += GS) smap[i] = -1;
    g.sync();
    if (status == MCS_OK || status == MCS_TIMEOUT) {
        const uint16_t* slot = P.best + ((size_t)pair * kLevels + k) * kMaxN;
        for (int i = g.q; i < k; i += GS) {
            uint16_t e = vload(slot + i);
            if (!DBG_OK(P.ctl, (e >> 8) < kMaxN && (e & 0xff) < kMaxN, 8, e)) continue;
            smap[__ldcg(&pg.permG[e >> 8])] = (int16_t)__ldcg(&pg.permH[e & 0xff]);
        }
    }
    g.sync();
    ServeRes* r = P.sv.res + pair;
    for (int i = g.q; i < kMaxN; i += GS) r->map[i] = smap[i];
    u64 ticket = 0;
    if (g.q == 0) {
        const u64 now = gtimer(), t0 = vload(&ps.t_start);
        ticket = vload(&ps.ticket);
        r->size = k;
        r->status = status;
        r->nodes = vload(&ps.nodes);
        r->usec = t0 ? (float)((now - t0) * 1e-3) : 0.f;
    }
    g.sync();
    __threadfence_system();
    if (g.q == 0) {
        *(volatile u64*)&r->done = ticket;
        ps.status = status;
        __threadfence();
        atomicSub(P.sv.in_flight, 1);
        atomicMax(&P.ctl->last_progress, gtimer());
    }
    g.sync();
}

// Goal-directed search (Section IV), one lane: the pair searches again from
// its root for the goal `cap` (only mappings larger than `floor` = cap - 1 are
// recorded).  Out of line: it runs once per goal, and inlined it would cost
// the node loop registers.  False if the bounded wait for a ring slot expired.
__device__ __noinline__ bool requeue_goal(const SearchParams& P, int pair, int floor, int cap) {
    PairState& ps = P.state[pair];
    ps.floor = floor;
    ps.cap = cap;
    ps.inc = floor;
    ps.abort = 0;
    ps.open = 1;
    __threadfence();
    const uint32_t qmask = P.qcap - 1;
    const u64 t = atomicAdd(&P.ctl->q_tail, 1ull);
    if (!wait_seq(P.qseq + (t & qmask), t, P.spin_limit)) return false;
    Task* dst = P.queue + (t & qmask);
    dst->h.pair = pair;
    dst->h.flags = kTaskFresh;
    dst->h.depth = 0;
    dst->h.C = 0;
    __threadfence();
    P.qseq[t & qmask] = t + 1;
    atomicMax(&P.ctl->last_progress, gtimer());
    return true;
}

// Finish the pair: write size, status, nodes and the mapping (original numbers).
// GOAL (nonzero): a launch of a strategy of Section IV (MCS_TOP_DOWN,
// MCS_DEAD_END, MCS_RESTART): the size is the largest recorded mapping, and a
// pair may be searched again from its root with another goal instead of being
// finished.
template <bool SERVE, int GS, int GOAL>
__device__ void finalize_pair(const SearchParams& P, int pair, const Grp<GS>& g, int16_t* smap) {
    __threadfence();
    PairState& ps = P.state[pair];
    const PairGraph& pg = P.graphs[pair];
    // read by lane 0 and broadcast (see the note at task install)
    int status = 0, k = 0, ab = 0, fl = 0, cp = 0, lo = 0, hi = 0;
    if (g.q == 0) {
        status = vload(&ps.status);
        ab = vload(&ps.abort);
        if constexpr (GOAL) {
            k = vload(&ps.real);
            fl = vload(&ps.floor);
            cp = vload(&ps.cap);
            lo = vload(&ps.lo);
            hi = vload(&ps.hi);
        } else {
            k = vload(&ps.inc);
        }
    }
    status = g.shfl(status, 0);
    k = g.shfl(k, 0);
    ab = g.shfl(ab, 0);
    // Goal-directed strategies (Section IV): decide whether the pair is
    // settled, else the goal of its next search from the root (0: none).
    int next_goal = 0;
    if constexpr (GOAL) {
    fl = g.shfl(fl, 0);
    cp = g.shfl(cp, 0);
    lo = g.shfl(lo, 0);
    hi = g.shfl(hi, 0);
    if (status == MCS_PENDING && ab != 1) {
        if ((P.flags & MCS_TOP_DOWN) && cp < kNoCap && k < cp && fl > 0) {
            next_goal = fl;                       // top-down: goal fl + 1 unreachable, try fl
        } else if (P.flags & MCS_DEAD_END) {
            if (cp == kNoCap) {
                // the search with raised bounds ended: a mapping at least the last
                // raised value is optimal, else that value bounds the optimum
                lo = k;
                hi = k >= fl ? k : fl;
            } else if (k >= cp) {
                lo = cp;                          // the probed goal was reached
            } else {
                hi = cp - 1;                      // the probed goal is unreachable
            }
            if (lo < hi) next_goal = (lo + hi + 1) / 2;
        }
    }
    }
    if (next_goal > 0) {
        int ok = 1;
        if (g.q == 0) {
            ps.lo = lo;
            ps.hi = hi;
            ok = requeue_goal(P, pair, next_goal - 1, next_goal) ? 1 : 0;
        }
        ok = g.shfl(ok, 0);
        if (ok) { g.sync(); return; }
        // the ring slot never freed (recorded below): finish with what is known
        if (g.q == 0) atomicCAS(&P.ctl->error, 0, MCS_ERR_DEVICE_STALL);
    }
    if (status == MCS_PENDING) {
        if (!DBG_OK(P.ctl, k >= 0 && k < kLevels, 7, k)) k = 0;
        status = ab == 1 ? MCS_TIMEOUT : MCS_OK;
        if constexpr (SERVE) { finalize_served<GS>(P, pair, status, k, g, smap); return; }
        if (P.out_map) {
            const uint16_t* slot = P.best + ((size_t)pair * kLevels + k) * kMaxN;
            for (int i = g.q; i < k; i += GS) {
                uint16_t e = vload(slot + i);
                if (!DBG_OK(P.ctl, (e >> 8) < kMaxN && (e & 0xff) < kMaxN, 8, e)) continue;
                int gg = __ldcg(&pg.permG[e >> 8]), h = __ldcg(&pg.permH[e & 0xff]);
                P.out_map[(size_t)pair * MCS_MAX_N + gg] = (int16_t)h;
            }
        }
    } else {
        k = 0;
        if constexpr (SERVE) { finalize_served<GS>(P, pair, status, 0, g, smap); return; }
    }
    int last = 0;
    if (g.q == 0) {
        u64 now = gtimer();
        if (P.out_size) P.out_size[pair] = k;
        if (P.out_nodes) P.out_nodes[pair] = vload(&ps.nodes);
        u64 t0 = vload(&ps.t_start);
        if (P.out_usec) P.out_usec[pair] = t0 ? (float)((now - t0) * 1e-3) : 0.f;
        __threadfence();
        if (P.out_status) P.out_status[pair] = status;
        ps.status = status;
        __threadfence();
        last = atomicSub(&P.ctl->remaining, 1) == 1;
        atomicMax(&P.ctl->last_progress, now);
    }
    last = g.shfl(last, 0);
    if (last) post_exit_tokens<GS>(P, P.max_warps, g);
    g.sync();
}

// A task of `pair` ended: publish node count, drop the open count and finalise
// the pair if this was its last task.
template <bool SERVE, int GS, int GOAL, typename N>
__device__ __forceinline__ void end_task(const SearchParams& P, int pair, N& nodes, const Grp<GS>& g,
                                         int16_t* smap) {
    int last = 0;
    if (g.q == 0) {
        if (nodes) atomicAdd(&P.state[pair].nodes, (u64)nodes);
        __threadfence();
        last = atomicSub(&P.state[pair].open, 1) == 1;
    }
    nodes = 0;
    last = g.shfl(last, 0);
    if (last) finalize_pair<SERVE, GS, GOAL>(P, pair, g, smap);
}

// Serve mode: copies request `slot` out of mapped host memory into its device
// slot, packs it (validation, renumbering, rows, root classes; the whole
// warp) and sets up its search state.  skey: 2 x 64 long long of scratch.
__device__ void serve_pack(const SearchParams& P, int slot, int lane, long long* skey) {
    int rq[3] = {0, 0, 0};
    u64 rt = 0, rtk = 0;
    if (lane == 0) {
        const ServeReq* q = P.sv.req + slot;
        rq[0] = vload(&q->nG); rq[1] = vload(&q->nH); rq[2] = vload(&q->labelled);
        rt = vload(&q->timeout_ns); rtk = vload(&q->ticket);
    }
    for (int j = 0; j < 3; ++j) rq[j] = __shfl_sync(FULL, rq[j], 0);
    rt = shfl64(rt, 0);
    rtk = shfl64(rtk, 0);
    // copy the bytes the request uses (n*n per graph, labels when present) out
    // of mapped host memory: four 16-byte loads in flight per lane
    const uint4* src = reinterpret_cast<const uint4*>(P.sv.hdata + (size_t)slot * kSlotBytes);
    uint4* dst = reinterpret_cast<uint4*>(P.sv.ddata + (size_t)slot * kSlotBytes);
    const int nG = min(max(rq[0], 0), kMaxN), nH = min(max(rq[1], 0), kMaxN);
    const int seg_lo[4] = {0, kMaxN * kMaxN / 16, 2 * kMaxN * kMaxN / 16, (2 * kMaxN * kMaxN + 4 * kMaxN) / 16};
    const int seg_n[4] = {(nG * nG + 15) / 16, (nH * nH + 15) / 16, (rq[2] & 1) ? 4 * kMaxN / 16 : 0,
                          (rq[2] & 2) ? 4 * kMaxN / 16 : 0};
#pragma unroll
    for (int sg = 0; sg < 4; ++sg) {
        for (int i0 = lane; i0 < seg_n[sg]; i0 += 128) {
            uint4 v[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int i = i0 + 32 * u;
                if (i < seg_n[sg])
                    asm volatile("ld.volatile.global.v4.u32 {%0,%1,%2,%3}, [%4];"
                                 : "=r"(v[u].x), "=r"(v[u].y), "=r"(v[u].z), "=r"(v[u].w)
                                 : "l"(src + seg_lo[sg] + i));
            }
#pragma unroll
            for (int u = 0; u < 4; ++u)
                if (i0 + 32 * u < seg_n[sg]) dst[seg_lo[sg] + i0 + 32 * u] = v[u];
        }
    }
    __syncwarp();
    const uint8_t* d = P.sv.ddata + (size_t)slot * kSlotBytes;
    GraphIn gi[2];
    gi[0].n = rq[0]; gi[1].n = rq[1];
    gi[0].a = d; gi[1].a = d + kMaxN * kMaxN;
    gi[0].lab = (rq[2] & 1) ? reinterpret_cast<const int32_t*>(d + 2 * kMaxN * kMaxN) : nullptr;
    gi[1].lab = (rq[2] & 2) ? reinterpret_cast<const int32_t*>(d + 2 * kMaxN * kMaxN + 4 * kMaxN) : nullptr;
    const bool ok = pack_pair_warp(gi, false, nullptr, nullptr, const_cast<PairGraph&>(P.graphs[slot]), skey, lane);
    if (lane == 0) {
        PairState& ps = P.state[slot];
        ps.inc = 0; ps.open = 1; ps.abort = 0; ps.nodes = 0;
        ps.floor = 0; ps.cap = kNoCap; ps.real = 0; ps.lo = ps.hi = 0; ps.dead = 0;
        ps.live = ps.mark = 0; ps.restarts = 0;
        ps.t_start = 0; ps.deadline = 0; ps.ticket = rtk; ps.timeout_ns = rt;
        ps.status = ok ? MCS_PENDING : MCS_ERR_ARG;
    }
    // every lane's packed rows and classes are visible before the root is published
    __threadfence();
    __syncwarp();
}

// Serve mode, warp 0 of the grid: admits requests that the host published in
// the mapped ring.  Each is packed here (serve_pack) and published as a fresh
// root of the ticket ring, which searchers of any width take like a batch
// root.  Exits, posting one exit token per searcher (ntok), after linger_ns
// without admitted or unfinished requests.
__device__ void serve_admit(const SearchParams& P, int lane, long long* skey, int ntok) {
    Control* ctl = P.ctl;
    const ServeDev& S = P.sv;
    const uint32_t qmask = P.qcap - 1;
    u64 admitted = 0, idle0 = 0;
    if (lane == 0) { admitted = vload(S.dev_admitted); idle0 = gtimer(); }
    admitted = shfl64(admitted, 0);
    for (;;) {
        int act = 0;                   // 1: admit up to hw, -1: leave, 0: wait
        u64 hw = 0;
        if (lane == 0) {
            if (vload(&ctl->error) != 0) {
                act = -1;
            } else {
                hw = vload(S.host_written);
                if (hw > admitted) {
                    act = 1;
                } else {
                    const u64 now = gtimer();
                    if (vload(S.in_flight) > 0) {
                        idle0 = now;
                        const u64 lp = vload(&ctl->last_progress);
                        if (now > lp && now - lp > P.stall_ns) {      // requests stopped progressing
                            atomicCAS(&ctl->error, 0, MCS_ERR_DEVICE_STALL);
                            act = -1;
                        }
                    } else if (now - idle0 > S.linger_ns || vload(S.stop) != 0) {
                        act = -1;
                    }
                }
            }
        }
        act = __shfl_sync(FULL, act, 0);
        hw = shfl64(hw, 0);
        if (act < 0) break;
        if (act == 0) { __nanosleep(1000); continue; }
        int ok = 1;
        for (; admitted < hw; ++admitted) {
            int slot = 0;
            if (lane == 0) slot = vload(S.ring + (admitted % (u64)S.ring_cap));
            slot = __shfl_sync(FULL, slot, 0);
            if (slot < 0 || slot >= S.nslots) continue;
            serve_pack(P, slot, lane, skey);
            if (lane == 0) {
                const u64 t = atomicAdd(&ctl->q_tail, 1ull);
                if (wait_seq(P.qseq + (t & qmask), t, P.spin_limit)) {
                    Task* dst = P.queue + (t & qmask);
                    dst->h.pair = slot;
                    dst->h.flags = kTaskFresh;
                    dst->h.depth = 0;
                    dst->h.C = 0;
                    atomicAdd(S.in_flight, 1);
                    __threadfence();
                    P.qseq[t & qmask] = t + 1;
                } else {
                    ok = 0;
                }
            }
            ok = __shfl_sync(FULL, ok, 0);
            if (!ok) break;
        }
        if (!ok) {
            if (lane == 0) atomicCAS(&ctl->error, 0, MCS_ERR_DEVICE_STALL);
            break;
        }
        if (lane == 0) {
            *(volatile u64*)S.dev_admitted = admitted;
            __threadfence_system();
            idle0 = gtimer();
            atomicMax(&ctl->last_progress, idle0);
        }
        __syncwarp();
    }
    __syncwarp();
    post_exit_tokens<32>(P, ntok, Grp<32>(lane));
}

__device__ __forceinline__ void load_level(const WarpSmem& w, int d, Top& t) {
    if (d < 0 || d >= kLevels) d = 0;   // unreachable: callers test t.d >= d0 >= 0, depth <= 64
    const ulonglong2 e = w.lvl[d];
    const u64 inf = e.y;
    t.rrem = e.x;
    t.base = (int)(inf & 0xffff);
    t.C = (int)((inf >> 16) & 0xff);
    t.v = (int)((inf >> 24) & 0xff);
    t.flags = (int)((inf >> 32) & 0xff);
    t.bound = (int)((inf >> 40) & 0xff);
}

// Work sharing: hands part of the shallowest open level of this searcher's
// subtree to a waiting searcher through the ring -- the upper part of its
// remaining candidates u (the donor keeps the share P.steal_keep_q4 / 4, by
// default half), or, with one candidate left, the rest of the level
// including its "v unmatched" branch.  The level's classes and the mapping
// prefix M travel with the task.  Returns false if the bounded wait for the
// ring slot expired (the error is recorded in the control block).
template <int GS, typename Stack>
__device__ __forceinline__ bool donate(const SearchParams& P, int pair, int d0, Top& t, int inc,
                                       const WarpSmem& w, const Stack& st, const Grp<GS>& g,
                                       unsigned& donated) {
    Control* ctl = P.ctl;
    const uint32_t qmask = P.qcap - 1;
    // flush the top cursor so that every level is in shared memory
    if (g.q == 0) {
        w.lvl[t.d] = make_ulonglong2(t.rrem, pack_info(t.base, t.C, t.v, t.flags, t.bound));
    }
    g.sync();
    int ds = -1;
    for (int off = d0; off <= t.d && ds < 0; off += GS) {
        const int d = off + g.q;
        bool open = false;
        if (d <= t.d) {
            const ulonglong2 e = w.lvl[d];
            const int fl = (int)((e.y >> 32) & 0xff), bd = (int)((e.y >> 40) & 0xff);
            open = (e.x != 0 || (fl & kTaskPending)) && bd > inc;
        }
        const unsigned m = g.ballot(open);
        if (m) ds = off + __ffs(m) - 1;
    }
    if (ds < 0) return true;
    const u64 inf = w.lvl[ds].y;
    const u64 rr = w.lvl[ds].x;
    const int fl = (int)((inf >> 32) & 0xff);
    const int k = __popcll(rr);
    u64 give;
    int gflags;
    if (k >= 2) {
        // the upper candidates; the rest and the unmatched branch stay
        give = rr;
        // the donor keeps the lowest ceil(k q / 4) (at least 1, at most k - 1)
        const int keep = min(k - 1, max(1, (k * P.steal_keep_q4 + 3) / 4));
        for (int j = 0; j < keep; ++j) give &= give - 1;
        gflags = 0;
    } else {
        give = rr;
        gflags = fl & kTaskPending;
    }
    // keep work of our own: a level whose subtree we are inside (ds < t.d)
    // or the top with >= 2 candidates
    const bool worth = (ds < t.d) || k >= 2;
    u64 ticket = 0;
    int ok = 0;
    if (worth && g.q == 0) {
        // A searcher was waiting when we polled.  Donors that saw the same
        // waiter may all donate: the surplus (at most one task per busy
        // searcher per poll window, far below the ring capacity) waits in
        // the ring for the next idle searcher.
        ticket = atomicAdd(&ctl->q_tail, 1ull);
        atomicAdd(&P.state[pair].open, 1);
        ok = wait_seq(P.qseq + (ticket & qmask), ticket, P.spin_limit) ? 1 : -1;
    }
    ok = g.shfl(ok, 0);
    if (ok < 0) {
        if (g.q == 0) atomicCAS(&ctl->error, 0, MCS_ERR_DEVICE_STALL);
        return false;
    }
    if (ok == 0) return true;
    ticket = g.shfl64(ticket, 0);
    Task* dst = P.queue + (ticket & qmask);
    const int C = (int)((inf >> 16) & 0xff);
    const int bs = (int)(inf & 0xffff);
    for (int i = g.q; i < C; i += GS) dst->cls[i] = *st.at(bs + i);
    for (int i = g.q; i < ds; i += GS) {
        const uint16_t m = m_entry(w.lvl[i].y);
        dst->Mg[i] = (uint8_t)(m >> 8);
        dst->Mh[i] = (uint8_t)m;
    }
    if (g.q == 0) {
        dst->h.pair = pair;
        dst->h.depth = ds;
        dst->h.C = C;
        dst->h.v = (int)((inf >> 24) & 0xff);
        dst->h.rrem = give;
        dst->h.flags = gflags;
        dst->h.bound = (int)((inf >> 40) & 0xff);
        w.lvl[ds] = make_ulonglong2(rr & ~give, (inf & ~(0xffull << 32)) | ((u64)(fl & ~gflags) << 32));
    }
    g.sync();
    __threadfence();
    if (g.q == 0) {
        P.qseq[ticket & qmask] = ticket + 1;   // publish
        atomicMax(&ctl->last_progress, gtimer());
    }
    g.sync();
    ++donated;
    if (ds == t.d) {
        t.rrem = rr & ~give;
        t.flags = fl & ~gflags;
    }
    return true;
}

// SplitMix64 (Steele, Lea, Flood 2014), one output per counter value.
__device__ __forceinline__ u64 splitmix64(u64 x) {
    x += 0x9E3779B97F4A7C15ull;
    x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
    x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
    return x ^ (x >> 31);
}

// Randomized restart (Section IV-A, MCS_RESTART): this searcher gives up its
// position in the tree.  Every open level of its stack -- remaining
// candidates and, if still to do, the "v unmatched" branch -- goes to the
// ring as a task, so the pending branches are the record of what is left to
// visit and nothing is lost; the levels are spilled in a random order (an
// affine permutation x -> (a x + b) mod 2^k of the level span, a odd, from
// SplitMix64 of the seed, the pair and its restart count), and whoever takes
// them next continues from there.  The caller then ends its task.  Returns
// false if a bounded wait for a ring slot expired.
template <int GS, typename Stack>
__device__ __noinline__ bool spill_all(const SearchParams& P, int pair, int d0, const Top& t, int inc,
                                       const WarpSmem& w, const Stack& st, const Grp<GS>& g) {
    Control* ctl = P.ctl;
    const uint32_t qmask = P.qcap - 1;
    if (g.q == 0) {
        w.lvl[t.d] = make_ulonglong2(t.rrem, pack_info(t.base, t.C, t.v, t.flags, t.bound));
    }
    g.sync();
    int nr = 0;
    if (g.q == 0) nr = atomicAdd(&P.state[pair].restarts, 1);
    nr = g.shfl(nr, 0);
    const int span = t.d - d0 + 1;
    int m = 1;
    while (m < span) m <<= 1;
    const u64 r = splitmix64(P.restart_seed + ((u64)(unsigned)pair << 32) + (u64)(unsigned)nr);
    const unsigned a = (unsigned)(r >> 32) | 1u, b = (unsigned)r;
    for (int i = 0; i < m; ++i) {
        const int d = d0 + (int)((a * (unsigned)i + b) & (unsigned)(m - 1));
        if (d > t.d) continue;
        const u64 inf = w.lvl[d].y;
        const u64 rr = w.lvl[d].x;
        const int fl = (int)((inf >> 32) & 0xff), bd = (int)((inf >> 40) & 0xff);
        if (!((rr != 0 || (fl & kTaskPending)) && bd > inc)) continue;   // nothing left above the bound
        u64 ticket = 0;
        int ok = 0;
        if (g.q == 0) {
            ticket = atomicAdd(&ctl->q_tail, 1ull);
            atomicAdd(&P.state[pair].open, 1);
            ok = wait_seq(P.qseq + (ticket & qmask), ticket, P.spin_limit) ? 1 : -1;
        }
        ok = g.shfl(ok, 0);
        if (ok < 0) {
            if (g.q == 0) atomicCAS(&ctl->error, 0, MCS_ERR_DEVICE_STALL);
            return false;
        }
        ticket = g.shfl64(ticket, 0);
        Task* dst = P.queue + (ticket & qmask);
        const int C = (int)((inf >> 16) & 0xff);
        const int bs = (int)(inf & 0xffff);
        for (int i2 = g.q; i2 < C; i2 += GS) dst->cls[i2] = *st.at(bs + i2);
        for (int i2 = g.q; i2 < d; i2 += GS) {
            const uint16_t m = m_entry(w.lvl[i2].y);
            dst->Mg[i2] = (uint8_t)(m >> 8);
            dst->Mh[i2] = (uint8_t)m;
        }
        if (g.q == 0) {
            dst->h.pair = pair;
            dst->h.depth = d;
            dst->h.C = C;
            dst->h.v = (int)((inf >> 24) & 0xff);
            dst->h.rrem = rr;
            dst->h.flags = fl & kTaskPending;
            dst->h.bound = bd;
        }
        g.sync();
        __threadfence();
        if (g.q == 0) {
            P.qseq[ticket & qmask] = ticket + 1;   // publish
            atomicMax(&ctl->last_progress, gtimer());
        }
        g.sync();
    }
    return true;
}

// Minimum resident 256-thread blocks per SM the register allocation must allow
// (3 caps registers at 80 per thread, 4 at 64).  Narrow searchers take the
// tighter cap: more resident warps outweigh the few spilled registers.
#ifndef MCS_SEARCH_MINB
#define MCS_SEARCH_MINB 3
#endif
#ifndef MCS_GROUP_MINB
#define MCS_GROUP_MINB 4
#endif

// GOAL: the strategies of Section IV are compiled into instantiations of
// their own, so that the plain search (0) carries none of their bookkeeping:
// 1 top-down goal sizes (MCS_TOP_DOWN), 2 dead-end forecasting and
// randomized restarts (MCS_DEAD_END, MCS_RESTART).
template <bool DIR, bool LEARNED, bool SERVE, int GS, bool NARROW, int GOAL>
__global__ void __launch_bounds__(256, (GS == 32 ? MCS_SEARCH_MINB : MCS_GROUP_MINB)) search_kernel(SearchParams P) {
    static_assert(GS == 2 || GS == 4 || GS == 8 || GS == 16 || GS == 32, "searcher group size");
    static_assert(!SERVE || GS >= 8, "serve mode keeps the level arrays and result scratch in shared memory");
    static_assert(!GOAL || (!SERVE && !LEARNED), "goal-directed searches: batch launches, degree or static order");
    extern __shared__ __align__(16) unsigned char smem[];
    constexpr int GPW = 32 / GS;                       // searchers per warp
    const int lane = threadIdx.x & 31;
    const int wib = threadIdx.x >> 5;
    const Grp<GS> g(lane);
    const int sid = (blockIdx.x * (blockDim.x >> 5) + wib) * GPW + (lane / GS);
    if (sid >= P.max_warps) return;
    constexpr bool ADJ_SM = adj_in_smem(GS);
    // Choose a surviving child's branching class in the pass that writes its
    // classes (lazy) or while summing Eq. 1 for every child (eager).
#if defined(MCS_KEYS_MODE) && MCS_KEYS_MODE == 0
    constexpr bool LAZY_KEYS = true;
#elif defined(MCS_KEYS_MODE) && MCS_KEYS_MODE == 1
    constexpr bool LAZY_KEYS = false;
#else
    constexpr bool LAZY_KEYS = DIR;
#endif
    unsigned char* base = smem + (size_t)(wib * GPW + lane / GS) * P.warp_smem_bytes;
    unsigned char* lv = base + sm_adj_bytes(GS);       // level arrays and class cache
    WarpSmem w;
    u64* adj_sm = (u64*)base;                          // rows copied here when ADJ_SM
    w.adj = adj_sm;
    w.lvl = (ulonglong2*)(lv + kSmLvOff);
    w.cls = (ulonglong2*)(lv + kSmClsOff);
    constexpr bool STACK_SM = GS == 32;
    StackT<STACK_SM> st;
    st.sm = w.cls;
    st.S = STACK_SM ? P.stack_smem : 0;
    const size_t gper = (size_t)(kStackMax > st.S ? kStackMax - st.S : 0) + (levels_in_smem(GS) ? 0 : kLvEntries);
    st.gm = P.gstack + (size_t)sid * gper;
    if constexpr (!levels_in_smem(GS)) {
        // level arrays (and cycle counters) after the class stack, in global memory
        lv = reinterpret_cast<unsigned char*>(st.gm + kStackMax);
        w.lvl = (ulonglong2*)(lv + kSmLvOff);
    }
#ifdef MCS_DEBUG_BOUNDS
    st.ctl = P.ctl;
#endif

    Control* ctl = P.ctl;
    // finalize scratch (the level entries are unused then) and the busy / idle
    // / mark clock words, addressed from the level entries when needed
    // rather than held in registers through the search loop
    auto smap = [&]() { return reinterpret_cast<int16_t*>(w.lvl); };
    auto cyc = [&]() {
        return reinterpret_cast<u64*>(reinterpret_cast<unsigned char*>(w.lvl) + (kSmCycOff - kSmLvOff));
    };
    if constexpr (SERVE) {
        // warp 0 of the grid admits requests; its groups do not search
        if (blockIdx.x == 0 && wib == 0) {
            serve_admit(P, lane, reinterpret_cast<long long*>(smem), P.max_warps - GPW);
            return;
        }
    }
    const bool level_prune = (P.flags & MCS_NO_LEVEL_PRUNE) == 0;
    const uint32_t qmask = P.qcap - 1;
    int cur_pair = -1;
    unsigned nodes = 0;     // of the current task; flushed to the pair before it can wrap
    unsigned tick = 0;
    // statistics, meaningful in lane 0 of the group (32-bit: flushed to the
    // control block before they can wrap, and when the searcher leaves)
    unsigned spilled = 0, cvisits = 0, pruned = 0, donated = 0;
    if (g.q == 0) { cyc()[0] = 0; cyc()[1] = 0; }

    while (true) {
        // ------------------------------------------------------------------
        // acquire work: take the next ticket of the ring and sleep on that
        // slot until it is published (pair roots are published up front in
        // processing order; donations and exit tokens follow).
        // ------------------------------------------------------------------
        const long long c_idle = clock64();
        int got = 0;          // 1 task, -1 exit
        u64 qh = 0;
        if (g.q == 0) {
            qh = atomicAdd(&ctl->q_head, 1ull);
            const u64* seq = P.qseq + (qh & qmask);
            for (int it = 0; got == 0; ++it) {
                if (vload(seq) == qh + 1) { got = 1; break; }
                if ((it & 63) == 63) {
                    if (vload(&ctl->error) != 0) { got = -1; break; }
                    u64 now = gtimer(), lp = vload(&ctl->last_progress);
                    if (now > lp && now - lp > P.stall_ns) {
                        atomicCAS(&ctl->error, 0, MCS_ERR_DEVICE_STALL);
                        got = -1;
                        break;
                    }
                }
                __nanosleep(128u << min(it >> 2, 6));     // 0.13 .. 8 us
            }
        }
        got = g.shfl(got, 0);
        qh = g.shfl64(qh, 0);
        if (got < 0) break;
        __threadfence();
        const Task* task = P.queue + (qh & qmask);
        int pair = 0, tflags = 0;
        if (g.q == 0) { pair = vload(&task->h.pair); tflags = vload(&task->h.flags); }
        pair = g.shfl(pair, 0);
        tflags = g.shfl(tflags, 0);
        if (!DBG_OK(ctl, pair < P.npairs, 2, pair)) pair = -1;
        if (pair < 0) {                                   // exit token
            g.sync();
            if (g.q == 0) P.qseq[qh & qmask] = qh + P.qcap;
            break;
        }
        Top t;
        const bool fresh = (tflags & kTaskFresh) != 0;
        PairState& ps = P.state[pair];
        const PairGraph& pg = P.graphs[pair];
        int pstat = 0;
        if (g.q == 0) pstat = vload(&ps.status);
        pstat = g.shfl(pstat, 0);
        if (fresh) {
            if (pstat != MCS_PENDING) {                   // malformed input: report and skip
                g.sync();
                if (g.q == 0) { P.qseq[qh & qmask] = qh + P.qcap; ps.open = 0; }
                finalize_pair<SERVE, GS, GOAL>(P, pair, g, smap());
                continue;
            }
            if (g.q == 0) {
                u64 now = gtimer();
                if (!GOAL || vload(&ps.t_start) == 0) {   // the first root (goal searches re-enqueue it)
                    ps.t_start = now;
                    ps.deadline = now + (SERVE ? vload(&ps.timeout_ns) : P.timeout_ns);
                }
                atomicMax(&ctl->last_progress, now);
            }
        }
        // load the pair's rows into shared memory (through L2: in serve mode a
        // slot is repacked while the kernel runs, so L1 may hold old lines)
        if (!ADJ_SM) {
            // rows read in place: written by the pack kernel before this launch
            w.adj = pg.rows;
        } else if (pair != cur_pair || SERVE) {
            // every row pair {out, in} of both graphs, one 16-byte load each
            for (int i = g.q; i < 2 * kMaxN; i += GS)
                reinterpret_cast<ulonglong2*>(adj_sm)[i] = ld_cg(reinterpret_cast<const ulonglong2*>(pg.rows) + i);
            cur_pair = SERVE ? -1 : pair;
        }
        // NARROW: every pair has at most 32 vertices per graph (checked by the pack kernel)
        if (!fresh) {
            int hd4[4] = {0, 0, 0, 0};
            u64 rr = 0;
            if (g.q == 0) {
                hd4[0] = vload(&task->h.depth);
                hd4[1] = vload(&task->h.C);
                hd4[2] = vload(&task->h.v);
                hd4[3] = vload(&task->h.bound);
                rr = vload(&task->h.rrem);
            }
            t.d = g.shfl(hd4[0], 0);
            t.C = g.shfl(hd4[1], 0);
            t.v = g.shfl(hd4[2], 0);
            t.bound = g.shfl(hd4[3], 0);
            t.rrem = g.shfl64(rr, 0);
            t.flags = tflags;
            if (!DBG_OK(ctl, t.C >= 0 && t.C <= kMaxN, 3, t.C)) t.C = 0;
            if (!DBG_OK(ctl, t.d >= 0 && t.d < kMaxN, 4, t.d)) t.d = 0;
            // the mapping prefix: levels below the task's depth keep only their (v, u)
            for (int i = g.q; i < t.d; i += GS)
                w.lvl[i] = make_ulonglong2(0ull, ((u64)ld_cg(&task->Mg[i]) << 24) | ((u64)ld_cg(&task->Mh[i]) << 48));
            for (int i = g.q; i < t.C; i += GS) *st.at(i) = ld_cg(&task->cls[i]);
            if (g.q == 0) atomicAdd(&ctl->stolen, 1ull);   // rare: counted in place
        } else {
            t.d = 0;
            t.C = __ldcg(&pg.C0);
            for (int i = g.q; i < t.C; i += GS) *st.at(i) = __ldcg(&pg.root[i]);
        }
        g.sync();
        if (g.q == 0) {
            __threadfence();
            P.qseq[qh & qmask] = qh + P.qcap;              // release the slot
        }
        t.base = 0;
        const int d0 = t.d;
        // Values other searchers may be writing are read by lane 0 only and
        // broadcast: lanes are not guaranteed to execute a load at the same
        // time, and a lane-dependent copy would split the group at the next
        // branch (and make a later group-wide shuffle illegal).
        int inc = 0, ab0 = 0;
        if (g.q == 0) {
            inc = vload(&ps.inc);
            ab0 = vload(&ps.abort);
        }
        inc = g.shfl(inc, 0);
        ab0 = g.shfl(ab0, 0);
        // the start of the busy period is kept in memory (cyc()[2]), not in a
        // register that would stay live through the search loop
        if (g.q == 0) {
            const long long c_busy = clock64();
            cyc()[1] += (u64)(c_busy - c_idle);
            cyc()[2] = (u64)c_busy;
        }
        if (ab0) {
            end_task<SERVE, GS, GOAL>(P, pair, nodes, g, smap());
            if (g.q == 0) cyc()[0] += (u64)(clock64() - (long long)cyc()[2]);
            continue;
        }
        if (fresh) {
            // root node entry (Algorithm 1): bound of Eq. 1, then class choice
            ++nodes;
            cvisits += t.C;
            const Scan sc = scan_level<typename std::conditional<NARROW, uint32_t, u64>::type, GS>(g, st, 0, t.C, -1);
            t.bound = sc.sum;
            if (t.bound <= inc) {
                end_task<SERVE, GS, GOAL>(P, pair, nodes, g, smap());
                if (g.q == 0) cyc()[0] += (u64)(clock64() - (long long)cyc()[2]);
                continue;
            }
            t.v = sc.key & 63;
            t.rrem = sc.R;
            t.flags = kTaskPending;
        }

        // ------------------------------------------------------------------
        // depth-first search over this task's subtree
        // ------------------------------------------------------------------
        // polled values, loaded by lane 0 half a poll interval before they
        // are used so that the L2 round trip overlaps node work
        // One search node at the top of the stack: "v unmatched" when no
        // candidate u is left, else the child (v, u).  W is the bit-set word.
        auto node_step = [&](auto wtag) {
            using W = decltype(wtag);
                if (t.rrem == 0) {
                    // ---------------- "v stays unmatched": same M, v leaves its class ----------------
                    ++nodes;
                    cvisits += t.C;
                    const Scan sc = scan_level<W, GS>(g, st, t.base, t.C, t.v);
                    g.sync();
                    t.bound = t.d + sc.sum;
                    if (t.bound <= inc) {
                        t.flags = 0;            // pruned: the level is exhausted and pops next
                    } else {
                        t.v = sc.key & 63;
                        t.rrem = sc.R;
                        t.flags = kTaskPending;
                    }
                    return;
                }
                // ---------------- child (v, u): filterDomain + Eq. 1 ----------------
                int u;
                if (LEARNED) {
                    // the remaining candidate with the best learned rank for v
                    u = learned_pick<GS>(P.rank + ((size_t)pair * kMaxN + t.v) * kMaxN, t.rrem, g);
                } else {
                    u = __ffsll(t.rrem) - 1;
                }
                t.rrem &= ~(1ull << u);
                ++nodes;
                cvisits += t.C;
                const int v = t.v;
                const W vb = (W)1 << v, ub = (W)1 << u;
                W gB, hB, gA = 0, hA = 0;
                if constexpr (DIR) {
                    const ulonglong2 gv = adj_row_pair<ADJ_SM, SERVE>(w.adj, row_gout(v));
                    const ulonglong2 hu = adj_row_pair<ADJ_SM, SERVE>(w.adj, row_hout(u));
                    gB = (W)gv.x; gA = (W)gv.y; hB = (W)hu.x; hA = (W)hu.y;
                } else {
                    gB = (W)adj_row<ADJ_SM, SERVE>(w.adj, row_gout(v));
                    hB = (W)adj_row<ADJ_SM, SERVE>(w.adj, row_hout(u));
                }
                const int dm = t.d + 1;
                const int cbase = t.base + t.C;
                // parent and child both inside the shared-memory class cache:
                // shared-memory loads/stores instead of generic ones
                const bool in_sm = STACK_SM && cbase + kMaxN <= st.S;
                int sum = 0;
                unsigned best = kKeyNone;
                W bestR = 0;
                int pos = cbase;
                // Appends the part (l, r) to the child level when both sides are
                // non-empty (group-wide ballot compaction, order kept), and
                // offers it as the child's branching class: key max(|l|, |r|)
                // << 6 | lowest l vertex, the smallest key wins.
                auto emit = [&](W l, W r, bool keep) {
                    const unsigned mk = g.ballot(keep);
                    if (keep) {
                        const int q2 = pos + __popc(mk & g.lt());
                        if (in_sm) st.sm[q2] = make_ulonglong2((u64)l, (u64)r);
                        else *st.at(q2) = make_ulonglong2((u64)l, (u64)r);
                        if constexpr (LAZY_KEYS) {
                            const unsigned key = ((unsigned)max(Word<W>::popc(l), Word<W>::popc(r)) << 6) |
                                                 (unsigned)Word<W>::low(l);
                            if (key < best) { best = key; bestR = r; }
                        }
                    }
                    pos += __popc(mk);
                };
                // The child's classes are written, and its branching class chosen,
                // only once it survives Eq. 1 (55-60 % of children do not), in a
                // second pass over the classes kept in registers (both slots of a
                // whole warp, slot 0 of a narrow searcher; further slots of a
                // narrow searcher are re-read).  The first pass only sums Eq. 1.
                W Ls[2], Rs[2];
                // Eq. 1 terms of one class slot: min(|L'|, |R'|) over its parts
                // (with eager keys the branching class is chosen here as well;
                // with lazy keys only survivors choose it, in the second pass)
                auto part_sum = [&](W L, W R) -> int {
                    auto term = [&](W l, W r) -> int {
                        const int a = Word<W>::popc(l), b = Word<W>::popc(r), m = min(a, b);
                        if constexpr (!LAZY_KEYS) {
                            const unsigned key = m ? (((unsigned)max(a, b) << 6) | (unsigned)Word<W>::low(l)) : kKeyNone;
                            if (key < best) { best = key; bestR = r; }
                        }
                        return m;
                    };
                    if (DIR) {
                        const W la = L & gA, lb = L & gB, ra = R & hA, rb = R & hB;
                        const W lp[4] = {(W)(L & ~(la | lb)), (W)(la & ~lb), (W)(lb & ~la), (W)(la & lb)};
                        const W rp[4] = {(W)(R & ~(ra | rb)), (W)(ra & ~rb), (W)(rb & ~ra), (W)(ra & rb)};
                        int s4 = 0;
    #pragma unroll
                        for (int k = 0; k < 4; ++k) s4 += term(lp[k], rp[k]);
                        return s4;
                    } else {
                        const W l1 = L & gB, r1 = R & hB;
                        return term(l1, r1) + term((W)(L ^ l1), (W)(R ^ r1));
                    }
                };
                {
                    // slot 0, straight-line (a child's level holds at least the
                    // class of v and u, so t.C >= 1): lanes beyond the class count
                    // read the level's first class and contribute nothing
                    const bool have = g.q < t.C;
                    const int i = have ? g.q : 0;
                    const ulonglong2 c = in_sm ? st.sm[t.base + i] : *st.at(t.base + i);
                    const W L = have ? ((W)c.x & ~vb) : (W)0;
                    const W R = have ? ((W)c.y & ~ub) : (W)0;
                    Ls[0] = L;
                    Rs[0] = R;
                    sum += part_sum(L, R);
                }
                for (int sl = 1; sl * GS < t.C; ++sl) {      // further slots: more classes than lanes
                    const int i = sl * GS + g.q;
                    W L = 0, R = 0;
                    if (i < t.C) {
                        const ulonglong2 c = in_sm ? st.sm[t.base + i] : *st.at(t.base + i);
                        L = (W)c.x & ~vb;
                        R = (W)c.y & ~ub;
                    }
                    if constexpr (GS == 32) { Ls[1] = L; Rs[1] = R; }
                    sum += part_sum(L, R);
                }
                sum = g.add(sum);
                // incumbent (Algorithm 1): |M u {(v,u)}| beats the best so far
                if (dm > inc) {
                    int old = 0;
                    if (g.q == 0) old = atomicMax(&ps.inc, dm);
                    old = g.shfl(old, 0);
                    if (old < dm) {
                        write_best<GS>(P, pair, w, t.d, v, u, g);
                        inc = dm;
                        if (P.race_gpu && g.q == 0) {             // GPU + CPU race: publish the size
                            *P.race_gpu = dm;
                            __threadfence_system();
                        }
                        if constexpr (GOAL) {
                            if (g.q == 0) {
                                atomicMax(&ps.real, dm);        // a recorded mapping of size dm
                                if (GOAL == 2 && (P.flags & MCS_DEAD_END)) ps.dead = 0;
                                if (GOAL == 2 && (P.flags & MCS_RESTART)) ps.mark = vload(&ps.live);
                            }
                        }
                    } else {
                        inc = old;
                    }
                    // goal reached (Section IV; the cap is read only when the incumbent
                    // grows): the pair is solved -- every searcher on it stops at its
                    // next poll, this one now (depth -1 is below every task's)
                    if constexpr (GOAL) {
                        int cap = 0;
                        if (g.q == 0) cap = vload(&ps.cap);
                        cap = g.shfl(cap, 0);
                        if (inc >= cap) {
                            if (g.q == 0) atomicCAS(&ps.abort, 0, 2);
                            t.d = -1;
                            return;
                        }
                    }
                }
                if (dm + sum <= inc) { ++pruned; return; }    // child pruned by Eq. 1
                // descend: compact the child's classes onto the stack
                auto emit_parts = [&](W L, W R) {
                    if (DIR) {
                        const W la = L & gA, lb = L & gB, ra = R & hA, rb = R & hB;
                        const W lp[4] = {(W)(L & ~(la | lb)), (W)(la & ~lb), (W)(lb & ~la), (W)(la & lb)};
                        const W rp[4] = {(W)(R & ~(ra | rb)), (W)(ra & ~rb), (W)(rb & ~ra), (W)(ra & rb)};
#pragma unroll
                        for (int k = 0; k < 4; ++k) emit(lp[k], rp[k], lp[k] && rp[k]);
                    } else {
                        const W l1 = L & gB, r1 = R & hB, l0 = L ^ l1, r0 = R ^ r1;
                        emit(l1, r1, l1 && r1);
                        emit(l0, r0, l0 && r0);
                    }
                };
                emit_parts(Ls[0], Rs[0]);                  // slot 0 from registers
                for (int sl = 1; sl * GS < t.C; ++sl) {
                    W L = 0, R = 0;
                    if (GS == 32) {
                        L = Ls[1];
                        R = Rs[1];
                    } else {
                        const int i = sl * GS + g.q;
                        if (i < t.C) {
                            const ulonglong2 c = *st.at(t.base + i);
                            L = (W)c.x & ~vb;
                            R = (W)c.y & ~ub;
                        }
                    }
                    emit_parts(L, R);
                }
                const unsigned kmin = g.umin(best);
                const unsigned win = g.ballot(best == kmin);
                const u64 cR = g.shfl64((u64)bestR, __ffs(win) - 1);
                if (STACK_SM && pos > st.S) spilled += 1;   // narrow searchers have no shared part
                if (!DBG_OK(ctl, pos - cbase <= kMaxN && dm <= kMaxN, 5, (pos - cbase) * 1000 + dm)) pos = cbase;
                if (g.q == 0)
                    w.lvl[t.d] = make_ulonglong2(t.rrem, pack_info(t.base, t.C, t.v, t.flags, t.bound) | ((u64)u << 48));
                g.sync();
                t.d = dm;
                t.base = cbase;
                t.C = pos - cbase;
                t.v = kmin & 63;
                t.rrem = cR;
                t.flags = kTaskPending;
                t.bound = dm + sum;
        };

        // polled values of lane 0, packed in one word until their use:
        // incumbent << 2 | hungry << 1 | abort
        int p_word = 0, p_restart = 0;
        while (t.d >= d0) {
            ++tick;
            // twice per poll interval (one test per node): lane 0 loads the
            // polled values, and half an interval later the group uses them
            if ((tick & (P.poll_mask >> 1)) == 0) {
                if ((tick & P.poll_mask) == 0) {
                    if (g.q == 0) {
                        int p_inc = vload(&ps.inc);
                        int p_abort = vload(&ps.abort);
                        const int p_hungry = vload(&ctl->q_head) > vload(&ctl->q_tail);   // a searcher waits
                        if (!p_abort && (tick & 255) == 0 && gtimer() > vload(&ps.deadline)) {
                            if constexpr (GOAL) atomicCAS(&ps.abort, 0, 1);   // time limit (a reached goal stays)
                            else ps.abort = 1;                 // per-pair time limit
                            p_abort = 1;
                        }
                        if (!GOAL && P.race_cpu && (tick & 4095) == 0) {
                            // GPU + CPU race: prune against the CPU side's best size too,
                            // and stop once the CPU side has finished its proof (words in
                            // host memory: one bus round trip each, so every 4,096 nodes)
                            p_inc = max(p_inc, (int)*P.race_cpu);
                            if (!p_abort && *P.race_stop) {
                                ps.abort = 1;
                                p_abort = 1;
                            }
                        }
                        if (GOAL == 2 && (P.flags & MCS_RESTART) && p_abort == 0) {
                            // randomized restart (Section IV-A) once the pair's node count has
                            // doubled since its last new incumbent (and passed restart_min); the
                            // searcher whose poll wins the mark update restarts
                            const u64 step = (u64)P.poll_mask + 1;
                            const u64 now = atomicAdd((unsigned long long*)&ps.live, (unsigned long long)step) + step;
                            const u64 mk = vload(&ps.mark);
                            // room for a whole stack of spilled branches: unclaimed tasks stay
                            // under half the ring (else this restart waits for the next doubling)
                            const long long pend = (long long)vload(&ctl->q_tail) - (long long)vload(&ctl->q_head);
                            if (now >= P.restart_min && now >= 2 * mk && pend + 2 * kLevels < (long long)(P.qcap / 2) &&
                                atomicCAS((unsigned long long*)&ps.mark, (unsigned long long)mk, (unsigned long long)now) == mk)
                                p_restart = 1;
                        }
                        if (GOAL == 2 && (P.flags & MCS_DEAD_END) && p_abort == 0) {
                            // dead-end forecast (Section IV): the searcher whose poll takes the
                            // pair's count of nodes without a new incumbent past the threshold
                            // raises the incumbent size, as if a mapping of that size were known
                            const u64 step = (u64)P.poll_mask + 1;
                            const u64 before = atomicAdd((unsigned long long*)&ps.dead, (unsigned long long)step);
                            if (before < P.dead_nodes && before + step >= P.dead_nodes && vload(&ps.cap) == kNoCap) {
                                const int cur = vload(&ps.inc);
                                const int r = min(P.dead_double ? max(cur + 1, 2 * cur) : cur + 1, kMaxN);
                                atomicMax(&ps.floor, r);
                                atomicMax(&ps.inc, r);
                                atomicExch((unsigned long long*)&ps.dead, 0ull);
                                p_inc = max(p_inc, r);
                            }
                        }
                        if (cvisits >= (1u << 31)) { atomicAdd(&ctl->class_visits, (u64)cvisits); cvisits = 0; }
                        if (nodes >= (1u << 31)) { atomicAdd(&ps.nodes, (u64)nodes); nodes = 0; }
                        if (pruned >= (1u << 31)) { atomicAdd(&ctl->pruned, (u64)pruned); pruned = 0; }
                        p_word = (p_inc << 2) | (p_hungry << 1) | (p_abort != 0);
                    }
                } else {
                    const int pw = g.shfl(p_word, 0);
                    const int g_inc = pw >> 2;
                    const int ab = pw & 1;
                    const int hungry = (pw >> 1) & 1;
                    inc = max(inc, g_inc);
                    if (ab) break;
                    if constexpr (GOAL == 2) {
                        const int rst = g.shfl(p_restart, 0);
                        p_restart = 0;
                        if (rst) {                         // restart: every open level to the ring
                            spill_all<GS>(P, pair, d0, t, inc, w, st, g);
                            break;
                        }
                    }
                    // ---- donate the shallowest open level to a waiting searcher ----
                    if (hungry) {
                        const bool ok = donate<GS>(P, pair, d0, t, inc, w, st, g, donated);
                        if (g.q == 0 && donated) atomicAdd(&ctl->donated, (u64)donated);   // rare: counted in place
                        donated = 0;
                        if (!ok) break;
                    }
                }
            }
            // level prune: every node below this level has bound <= this one
            // pop every exhausted or bounded level in one go (without a trip
            // through the poll checks per level), then expand a node
            if ((level_prune && t.bound <= inc) || (t.rrem == 0 && !(t.flags & kTaskPending))) {
                do {
                    --t.d;
                    if (t.d < d0) break;
                    load_level(w, t.d, t);
                } while ((level_prune && t.bound <= inc) || (t.rrem == 0 && !(t.flags & kTaskPending)));
                if (t.d < d0) break;
            }
            if constexpr (NARROW) node_step(uint32_t{});
            else node_step(u64{});
        }
        end_task<SERVE, GS, GOAL>(P, pair, nodes, g, smap());
        if (g.q == 0) cyc()[0] += (u64)(clock64() - (long long)cyc()[2]);
    }
    if (g.q == 0) {
        if (spilled) atomicAdd(&ctl->spilled, (u64)spilled);
        if (cvisits) atomicAdd(&ctl->class_visits, (u64)cvisits);
        if (pruned) atomicAdd(&ctl->pruned, (u64)pruned);
        atomicAdd(&ctl->busy_cycles, cyc()[0]);
        atomicAdd(&ctl->idle_cycles, cyc()[1]);
    }
}

// ---------------------------------------------------------------------------
// lockstep searchers
// ---------------------------------------------------------------------------
// The same depth-first McSplit as search_kernel's plain batch mode (Algorithm
// 1, Eq. 1, filterDomain of Table 1), for searchers narrower than a warp, with
// the searchers of a warp advancing in lockstep: every pass of the warp's loop
// expands one node of every searcher that has work, as one predicated
// instruction stream.  The "v stays unmatched" step is the child step with
// empty adjacency rows and no u (each class keeps one part, L \ {v} and R,
// which is exactly the rescan of the level), so a node is one split pass, the
// Eq. 1 reductions, and a second pass that writes a surviving child's classes.
// Loops over class slots run to the warp's largest class count.  What is rare
// per node -- taking a task, ending one, a new incumbent, work donation --
// stays per searcher (divergent); the polls run on a tick shared by the warp.
// Searchers that wait for work poll their ring slot once per pass instead of
// sleeping on it.  Results, node counts of a lone searcher, and every bounded
// wait are those of search_kernel.
template <bool DIR, bool LEARNED, int GS, bool NARROW>
__global__ void __launch_bounds__(256, MCS_GROUP_MINB) lockstep_kernel(SearchParams P) {
    static_assert(GS == 2 || GS == 4 || GS == 8 || GS == 16, "lockstep searchers share a warp");
    using W = typename std::conditional<NARROW, uint32_t, u64>::type;
    extern __shared__ __align__(16) unsigned char smem[];
    constexpr int GPW = 32 / GS;
    constexpr int kNeed = 0, kRun = 1, kExit = 2;
    const int lane = threadIdx.x & 31;
    const int wib = threadIdx.x >> 5;
    const Grp<GS> g(lane);
    const int sid = (blockIdx.x * (blockDim.x >> 5) + wib) * GPW + (lane / GS);
    // searchers beyond the limit take no work, but stay in the loop for the
    // warp-wide votes until every searcher of the warp has left
    int state = sid < P.max_warps ? kNeed : kExit;
    unsigned char* lv = smem + (size_t)(wib * GPW + lane / GS) * P.warp_smem_bytes;
    WarpSmem w;
    w.adj = nullptr;
    w.lvl = (ulonglong2*)(lv + kSmLvOff);
    w.cls = nullptr;
    StackT<false> st;
    st.sm = nullptr;
    st.S = 0;
    const size_t gper = (size_t)kStackMax + (levels_in_smem(GS) ? 0 : kLvEntries);
    st.gm = P.gstack + (size_t)(state == kExit ? 0 : sid) * gper;
    if constexpr (!levels_in_smem(GS)) {
        lv = reinterpret_cast<unsigned char*>(st.gm + kStackMax);
        w.lvl = (ulonglong2*)(lv + kSmLvOff);
    }
#ifdef MCS_DEBUG_BOUNDS
    st.ctl = P.ctl;
#endif
    Control* ctl = P.ctl;
    // finalize scratch and the busy / idle / mark clock words, addressed from
    // the level entries rather than held in registers (as in search_kernel)
    auto smap = [&]() { return reinterpret_cast<int16_t*>(w.lvl); };
    auto cyc = [&]() {
        return reinterpret_cast<u64*>(reinterpret_cast<unsigned char*>(w.lvl) + (kSmCycOff - kSmLvOff));
    };
    const bool level_prune = (P.flags & MCS_NO_LEVEL_PRUNE) == 0;
    const uint32_t qmask = P.qcap - 1;
    unsigned nodes = 0;      // of the current task; flushed to the pair before it can wrap
    unsigned tick = 0;
    unsigned cvisits = 0, pruned = 0, donated = 0;
    if (state != kExit && g.q == 0) { cyc()[0] = 0; cyc()[1] = 0; cyc()[2] = (u64)clock64(); }
    bool holding = false;    // the ticket taken is kept in cyc()[3] while waiting for its slot
    unsigned wait_it = 0, idle_ns = 128;
    int pair = 0, d0 = 0, inc = 0;
    int p_word = 0;          // lane 0's polled values: incumbent << 2 | hungry << 1 | abort
    Top t;
    t.d = -1; t.base = 0; t.C = 0; t.v = 0; t.flags = 0; t.bound = 0; t.rrem = 0;

    while (__any_sync(FULL, state != kExit)) {
        // ---------------- searchers without work: take a ticket, check its slot ----------------
        if (state == kNeed) {
            u64 qh = 0;
            if (!holding) {
                if (g.q == 0) {
                    qh = atomicAdd(&ctl->q_head, 1ull);
                    cyc()[3] = qh;
                }
                holding = true;
                wait_it = 0;
            }
            int got = 0;
            if (g.q == 0) {
                qh = cyc()[3];
                if (vload(P.qseq + (qh & qmask)) == qh + 1) {
                    got = 1;
                } else if ((++wait_it & 63) == 0) {
                    if (vload(&ctl->error) != 0) {
                        got = -1;
                    } else {
                        const u64 now = gtimer(), lp = vload(&ctl->last_progress);
                        if (now > lp && now - lp > P.stall_ns) {
                            atomicCAS(&ctl->error, 0, MCS_ERR_DEVICE_STALL);
                            got = -1;
                        }
                    }
                }
            }
            got = g.shfl(got, 0);
            if (got < 0) state = kExit;
            if (got > 0) {
                qh = g.shfl64(qh, 0);
                holding = false;
                __threadfence();
                const Task* task = P.queue + (qh & qmask);
                int tpair = 0, tflags = 0;
                if (g.q == 0) { tpair = vload(&task->h.pair); tflags = vload(&task->h.flags); }
                tpair = g.shfl(tpair, 0);
                tflags = g.shfl(tflags, 0);
                if (!DBG_OK(ctl, tpair < P.npairs, 2, tpair)) tpair = -1;
                if (tpair < 0) {                                  // exit token
                    g.sync();
                    if (g.q == 0) P.qseq[qh & qmask] = qh + P.qcap;
                    state = kExit;
                } else {
                    pair = tpair;
                    // polled values belong to the task they were read for: a half
                    // tick right after this install must not apply the previous
                    // pair's incumbent or abort flag to this one
                    p_word = 0;
                    const bool fresh = (tflags & kTaskFresh) != 0;
                    PairState& ps = P.state[pair];
                    const PairGraph& pg = P.graphs[pair];
                    int pstat = 0;
                    if (g.q == 0) pstat = vload(&ps.status);
                    pstat = g.shfl(pstat, 0);
                    if (fresh && pstat != MCS_PENDING) {          // malformed input: report and skip
                        g.sync();
                        if (g.q == 0) { P.qseq[qh & qmask] = qh + P.qcap; ps.open = 0; }
                        finalize_pair<false, GS, 0>(P, pair, g, smap());
                    } else {
                        if (fresh && g.q == 0) {
                            const u64 now = gtimer();
                            ps.t_start = now;
                            ps.deadline = now + P.timeout_ns;
                            atomicMax(&ctl->last_progress, now);
                        }
                        if (!fresh) {
                            int hd4[4] = {0, 0, 0, 0};
                            u64 rr = 0;
                            if (g.q == 0) {
                                hd4[0] = vload(&task->h.depth);
                                hd4[1] = vload(&task->h.C);
                                hd4[2] = vload(&task->h.v);
                                hd4[3] = vload(&task->h.bound);
                                rr = vload(&task->h.rrem);
                            }
                            t.d = g.shfl(hd4[0], 0);
                            t.C = g.shfl(hd4[1], 0);
                            t.v = g.shfl(hd4[2], 0);
                            t.bound = g.shfl(hd4[3], 0);
                            t.rrem = g.shfl64(rr, 0);
                            t.flags = tflags;
                            if (!DBG_OK(ctl, t.C >= 0 && t.C <= kMaxN, 3, t.C)) t.C = 0;
                            if (!DBG_OK(ctl, t.d >= 0 && t.d < kMaxN, 4, t.d)) t.d = 0;
                            for (int i = g.q; i < t.d; i += GS)
                                w.lvl[i] = make_ulonglong2(0ull, ((u64)ld_cg(&task->Mg[i]) << 24) |
                                                                     ((u64)ld_cg(&task->Mh[i]) << 48));
                            for (int i = g.q; i < t.C; i += GS) *st.at(i) = ld_cg(&task->cls[i]);
                            if (g.q == 0) atomicAdd(&ctl->stolen, 1ull);   // rare: counted in place
                        } else {
                            t.d = 0;
                            t.C = __ldcg(&pg.C0);
                            for (int i = g.q; i < t.C; i += GS) *st.at(i) = __ldcg(&pg.root[i]);
                        }
                        g.sync();
                        if (g.q == 0) {
                            __threadfence();
                            P.qseq[qh & qmask] = qh + P.qcap;     // release the slot
                        }
                        t.base = 0;
                        d0 = t.d;
                        int ab0 = 0;
                        if (g.q == 0) { inc = vload(&ps.inc); ab0 = vload(&ps.abort); }
                        inc = g.shfl(inc, 0);
                        ab0 = g.shfl(ab0, 0);
                        if (g.q == 0) {
                            const long long now = clock64();
                            cyc()[1] += (u64)(now - (long long)cyc()[2]);
                            cyc()[2] = (u64)now;
                        }
                        state = kRun;
                        if (ab0) {
                            t.d = d0 - 1;                         // ends below
                        } else if (fresh) {
                            // root node entry (Algorithm 1): bound of Eq. 1, then class choice
                            ++nodes;
                            cvisits += t.C;
                            const Scan sc = scan_level<W, GS>(g, st, 0, t.C, -1);
                            t.bound = sc.sum;
                            if (t.bound <= inc) {
                                t.d = d0 - 1;
                            } else {
                                t.v = sc.key & 63;
                                t.rrem = sc.R;
                                t.flags = kTaskPending;
                            }
                        }
                    }
                }
            }
        }
        if (!__any_sync(FULL, state == kRun)) {
            __nanosleep(idle_ns);
            idle_ns = min(idle_ns * 2u, 8192u);
            continue;
        }
        idle_ns = 128;
        // ---------------- polls: one tick for the warp ----------------
        ++tick;
        if ((tick & P.poll_mask) == 0 && state == kRun && g.q == 0) {
            PairState& ps = P.state[pair];
            const int p_inc = vload(&ps.inc);
            int p_abort = vload(&ps.abort);
            const int p_hungry = vload(&ctl->q_head) > vload(&ctl->q_tail);     // a searcher waits
            if (!p_abort && (tick & 255) == 0 && gtimer() > vload(&ps.deadline)) {
                ps.abort = 1;                                   // per-pair time limit
                p_abort = 1;
            }
            if (cvisits >= (1u << 31)) { atomicAdd(&ctl->class_visits, (u64)cvisits); cvisits = 0; }
            if (pruned >= (1u << 31)) { atomicAdd(&ctl->pruned, (u64)pruned); pruned = 0; }
            if (nodes >= (1u << 31)) { atomicAdd(&ps.nodes, (u64)nodes); nodes = 0; }
            p_word = (p_inc << 2) | (p_hungry << 1) | (p_abort != 0);
        }
        if ((tick & P.poll_mask) == (P.poll_mask + 1) / 2 && state == kRun && t.d >= d0) {
            const int pw = g.shfl(p_word, 0);
            inc = max(inc, pw >> 2);
            if (pw & 1) {
                t.d = d0 - 1;                                   // time limit: leave the task
            } else if ((pw >> 1) & 1) {
                const bool ok = donate<GS>(P, pair, d0, t, inc, w, st, g, donated);
                if (g.q == 0 && donated) atomicAdd(&ctl->donated, (u64)donated);   // rare: counted in place
                donated = 0;
                if (!ok) t.d = d0 - 1;
            }
        }
        // ---------------- pop exhausted or bounded levels ----------------
        for (;;) {
            const bool pop = state == kRun && t.d >= d0 &&
                             ((level_prune && t.bound <= inc) || (t.rrem == 0 && !(t.flags & kTaskPending)));
            if (!__any_sync(FULL, pop)) break;
            if (pop) {
                --t.d;
                if (t.d >= d0) load_level(w, t.d, t);
            }
        }
        if (state == kRun && t.d < d0) {                        // the task is done
            end_task<false, GS, 0>(P, pair, nodes, g, smap());
            if (g.q == 0) {
                const long long now = clock64();
                cyc()[0] += (u64)(now - (long long)cyc()[2]);
                cyc()[2] = (u64)now;
            }
            state = kNeed;
        }
        // ---------------- one node of every searcher with work ----------------
        const bool act = state == kRun;
        const bool ch = act && t.rrem != 0;                     // child (v, u)
        const bool um = act && t.rrem == 0;                     // "v stays unmatched"
        int u = 0;
        if constexpr (LEARNED) {
            u = learned_pick<GS>(P.rank + ((size_t)pair * kMaxN + t.v) * kMaxN, ch ? t.rrem : 0ull, g);
        } else {
            u = ch ? __ffsll(t.rrem) - 1 : 0;
        }
        if (ch) t.rrem &= ~(1ull << u);
        if (act) {
            ++nodes;
            cvisits += t.C;
        }
        const int v = t.v;
        const W vb = act ? ((W)1 << v) : (W)0;
        const W ub = ch ? ((W)1 << u) : (W)0;
        W gB = 0, hB = 0, gA = 0, hA = 0;
        if (ch) {
            gB = (W)adj_row<false>(P.graphs[pair].rows, row_gout(v));
            hB = (W)adj_row<false>(P.graphs[pair].rows, row_hout(u));
            if (DIR) {
                gA = (W)adj_row<false>(P.graphs[pair].rows, row_gin(v));
                hA = (W)adj_row<false>(P.graphs[pair].rows, row_hin(u));
            }
        }
        const int nsl = ((int)__reduce_max_sync(FULL, act ? (unsigned)t.C : 0u) + GS - 1) / GS;
        int sum = 0;
        unsigned best = kKeyNone;
        W bestR = 0, L0 = 0, R0 = 0;
        for (int sl = 0; sl < nsl; ++sl) {
            const int i = sl * GS + g.q;
            const bool have = act && i < t.C;
            W L = 0, R = 0;
            if (have) {
                ulonglong2* ptr = st.at(t.base + i);
                const ulonglong2 c = *ptr;
                L = (W)c.x & ~vb;
                R = (W)c.y & ~ub;
                if (um && ((W)c.x & vb)) ptr->x = (u64)L;       // v leaves its class in place
            }
            if (sl == 0) { L0 = L; R0 = R; }
            if (DIR) {
                const W la = L & gA, lb = L & gB, ra = R & hA, rb = R & hB;
                const W lp[4] = {(W)(L & ~(la | lb)), (W)(la & ~lb), (W)(lb & ~la), (W)(la & lb)};
                const W rp[4] = {(W)(R & ~(ra | rb)), (W)(ra & ~rb), (W)(rb & ~ra), (W)(ra & rb)};
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    const int a = Word<W>::popc(lp[k]), b = Word<W>::popc(rp[k]);
                    const int m = min(a, b);
                    sum += m;
                    const unsigned key = m ? (((unsigned)max(a, b) << 6) | (unsigned)Word<W>::low(lp[k])) : kKeyNone;
                    if (key < best) { best = key; bestR = rp[k]; }
                }
            } else {
                const W l1 = L & gB, r1 = R & hB, l0 = L ^ l1, r0 = R ^ r1;
                const int a1 = Word<W>::popc(l1), b1 = Word<W>::popc(r1), a0 = Word<W>::popc(l0), b0 = Word<W>::popc(r0);
                const int m1 = min(a1, b1), m0 = min(a0, b0);
                sum += m1 + m0;
                const unsigned k1 = m1 ? (((unsigned)max(a1, b1) << 6) | (unsigned)Word<W>::low(l1)) : kKeyNone;
                const unsigned k0 = m0 ? (((unsigned)max(a0, b0) << 6) | (unsigned)Word<W>::low(l0)) : kKeyNone;
                if (k1 < best) { best = k1; bestR = r1; }
                if (k0 < best) { best = k0; bestR = r0; }
            }
        }
        sum = g.add(sum);
        const int dm = t.d + 1;
        // incumbent (Algorithm 1): |M u {(v,u)}| beats the best so far
        if (ch && dm > inc) {
            int old = 0;
            if (g.q == 0) old = atomicMax(&P.state[pair].inc, dm);
            old = g.shfl(old, 0);
            if (old < dm) {
                write_best<GS>(P, pair, w, t.d, v, u, g);
                inc = dm;
            } else {
                inc = old;
            }
        }
        const unsigned kmin = g.umin(best);
        const unsigned win = g.ballot(best == kmin);
        const u64 cR = g.shfl64((u64)bestR, win ? __ffs(win) - 1 : 0);
        if (um) {
            t.bound = t.d + sum;
            if (t.bound <= inc) {
                t.flags = 0;                                    // the level is exhausted and pops next
            } else {
                t.v = kmin & 63;
                t.rrem = cR;
                t.flags = kTaskPending;
            }
        }
        const bool surv = ch && dm + sum > inc;
        if (ch && !surv) ++pruned;                              // child pruned by Eq. 1
        // descend: the surviving child's classes, compacted onto the stack
        const int cbase = t.base + t.C;
        int pos = cbase;
        const int nsl2 = ((int)__reduce_max_sync(FULL, surv ? (unsigned)t.C : 0u) + GS - 1) / GS;
        for (int sl = 0; sl < nsl2; ++sl) {
            W L = 0, R = 0;
            if (sl == 0) {
                L = L0;
                R = R0;
            } else {
                const int i = sl * GS + g.q;
                if (surv && i < t.C) {
                    const ulonglong2 c = *st.at(t.base + i);
                    L = (W)c.x & ~vb;
                    R = (W)c.y & ~ub;
                }
            }
            if (!surv) { L = 0; R = 0; }
            auto emit = [&](W l, W r) {
                const bool keep = l && r;
                const unsigned mk = g.ballot(keep);
                if (keep) *st.at(pos + __popc(mk & g.lt())) = make_ulonglong2((u64)l, (u64)r);
                pos += __popc(mk);
            };
            if (DIR) {
                const W la = L & gA, lb = L & gB, ra = R & hA, rb = R & hB;
                emit((W)(L & ~(la | lb)), (W)(R & ~(ra | rb)));
                emit((W)(la & ~lb), (W)(ra & ~rb));
                emit((W)(lb & ~la), (W)(rb & ~ra));
                emit((W)(la & lb), (W)(ra & rb));
            } else {
                const W l1 = L & gB, r1 = R & hB;
                emit(l1, r1);
                emit((W)(L ^ l1), (W)(R ^ r1));
            }
        }
        if (surv) {
            if (!DBG_OK(ctl, pos - cbase <= kMaxN && dm <= kMaxN, 5, (pos - cbase) * 1000 + dm)) pos = cbase;
            if (g.q == 0)
                w.lvl[t.d] = make_ulonglong2(t.rrem, pack_info(t.base, t.C, t.v, t.flags, t.bound) | ((u64)u << 48));
            t.d = dm;
            t.base = cbase;
            t.C = pos - cbase;
            t.v = kmin & 63;
            t.rrem = cR;
            t.flags = kTaskPending;
            t.bound = dm + sum;
        }
        __syncwarp();
    }
    if (sid < P.max_warps && g.q == 0) {
        if (cvisits) atomicAdd(&ctl->class_visits, (u64)cvisits);
        if (pruned) atomicAdd(&ctl->pruned, (u64)pruned);
        atomicAdd(&ctl->busy_cycles, cyc()[0]);
        atomicAdd(&ctl->idle_cycles, cyc()[1]);
    }
}

// Raises a kernel's dynamic shared-memory limit on the current device when a
// launch needs more than was set before (one driver call per new maximum,
// not one per launch).  Per kernel instantiation: `Tag` is unique to it.
// Returns false (with the runtime's error state cleared) when the device
// cannot give the kernel that much shared memory.
template <typename Tag>
static bool ensure_smem_limit(void (*k)(SearchParams), int smem) {
    constexpr int kDevs = 64;
    static std::atomic<int> set_bytes[kDevs];
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev >= 0 && dev < kDevs && set_bytes[dev].load(std::memory_order_relaxed) >= smem) return true;
    if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, smem) != cudaSuccess) {
        cudaGetLastError();            // expected for a shape that does not fit: reported as unsupported
        return false;
    }
    if (dev >= 0 && dev < kDevs) {
        int cur = set_bytes[dev].load();
        while (cur < smem && !set_bytes[dev].compare_exchange_weak(cur, smem)) {
        }
    }
    return true;
}

template <bool DIR, bool LEARNED, bool SERVE, int GS, bool NARROW, int GOAL>
struct KernelTag {};

template <bool DIR, bool LEARNED, bool SERVE, int GS, bool NARROW, int GOAL = 0>
static cudaError_t launch_t(const SearchParams& p, int blocks, int wpb, cudaStream_t s) {
    size_t smem = (size_t)wpb * (32 / GS) * p.warp_smem_bytes;
    auto* k = search_kernel<DIR, LEARNED, SERVE, GS, NARROW, GOAL>;
    if (!ensure_smem_limit<KernelTag<DIR, LEARNED, SERVE, GS, NARROW, GOAL>>(k, (int)smem))
        return cudaErrorInvalidValue;
    k<<<blocks, wpb * 32, smem, s>>>(p);
    return cudaGetLastError();
}

template <bool DIR, bool LEARNED, int GS, bool NARROW>
static cudaError_t launch_l(const SearchParams& p, int blocks, int wpb, cudaStream_t s) {
    size_t smem = (size_t)wpb * (32 / GS) * p.warp_smem_bytes;
    auto* k = lockstep_kernel<DIR, LEARNED, GS, NARROW>;
    if (!ensure_smem_limit<KernelTag<DIR, LEARNED, true, GS, NARROW, 99>>(k, (int)smem))
        return cudaErrorInvalidValue;
    k<<<blocks, wpb * 32, smem, s>>>(p);
    return cudaGetLastError();
}

template <bool DIR, bool LEARNED, bool NARROW, int GOAL>
static cudaError_t launch_g(const SearchParams& p, int blocks, int wpb, int gs, cudaStream_t s) {
    if (GOAL == 0 && p.lockstep && gs < 32) {
        // plain batch searches narrower than a warp: lockstep searchers
        if (gs == 2) return launch_l<DIR, LEARNED, 2, NARROW>(p, blocks, wpb, s);
        if (gs == 4) return launch_l<DIR, LEARNED, 4, NARROW>(p, blocks, wpb, s);
        if (gs == 8) return launch_l<DIR, LEARNED, 8, NARROW>(p, blocks, wpb, s);
        return launch_l<DIR, LEARNED, 16, NARROW>(p, blocks, wpb, s);
    }
    if (gs == 2) return launch_t<DIR, LEARNED, false, 2, NARROW, GOAL>(p, blocks, wpb, s);
    if (gs == 4) return launch_t<DIR, LEARNED, false, 4, NARROW, GOAL>(p, blocks, wpb, s);
    if (gs == 8) return launch_t<DIR, LEARNED, false, 8, NARROW, GOAL>(p, blocks, wpb, s);
    if (gs == 16) return launch_t<DIR, LEARNED, false, 16, NARROW, GOAL>(p, blocks, wpb, s);
    return launch_t<DIR, LEARNED, false, 32, NARROW, GOAL>(p, blocks, wpb, s);
}

template <bool DIR, bool LEARNED, int GOAL = 0>
static cudaError_t launch_w(const SearchParams& p, int blocks, int wpb, int gs, bool narrow, cudaStream_t s) {
    return narrow ? launch_g<DIR, LEARNED, true, GOAL>(p, blocks, wpb, gs, s)
                  : launch_g<DIR, LEARNED, false, GOAL>(p, blocks, wpb, gs, s);
}

cudaError_t launch_search(const SearchParams& p, int blocks, int warps_per_block, bool directed,
                          bool learned, cudaStream_t s, int gs) {
    if (p.serving) {
        if (gs == 8) return launch_t<false, false, true, 8, false>(p, blocks, warps_per_block, s);
        if (gs == 16) return launch_t<false, false, true, 16, false>(p, blocks, warps_per_block, s);
        return launch_t<false, false, true, 32, false>(p, blocks, warps_per_block, s);
    }
    const bool narrow = (p.flags & MCS_WORD32) != 0;
    if (p.flags & (MCS_TOP_DOWN | MCS_DEAD_END | MCS_RESTART)) {
        // goal-directed strategies (the caller rejects them with the learned order)
        if (learned) return cudaErrorNotSupported;
        if (p.flags & MCS_TOP_DOWN)
            return directed ? launch_w<true, false, 1>(p, blocks, warps_per_block, gs, narrow, s)
                            : launch_w<false, false, 1>(p, blocks, warps_per_block, gs, narrow, s);
        return directed ? launch_w<true, false, 2>(p, blocks, warps_per_block, gs, narrow, s)
                        : launch_w<false, false, 2>(p, blocks, warps_per_block, gs, narrow, s);
    }
    if (directed) return learned ? launch_w<true, true>(p, blocks, warps_per_block, gs, narrow, s)
                                 : launch_w<true, false>(p, blocks, warps_per_block, gs, narrow, s);
    return learned ? launch_w<false, true>(p, blocks, warps_per_block, gs, narrow, s)
                   : launch_w<false, false>(p, blocks, warps_per_block, gs, narrow, s);
}

// Loads one whole-warp batch instantiation on the current device and sets its
// shared-memory limit (see warm_batch_variants).
template <bool DIR, bool NARROW, int GOAL>
static cudaError_t warm_t(int smem) {
    auto* k = search_kernel<DIR, false, false, 32, NARROW, GOAL>;
    if (!ensure_smem_limit<KernelTag<DIR, false, false, 32, NARROW, GOAL>>(k, smem)) return cudaErrorInvalidValue;
    cudaFuncAttributes a;
    return cudaFuncGetAttributes(&a, k);
}

cudaError_t warm_batch_variants(int smem) {
    cudaFuncAttributes a;
    cudaError_t e = cudaFuncGetAttributes(&a, pack_kernel);
    const cudaError_t r[] = {e,
        warm_t<false, false, 0>(smem), warm_t<false, true, 0>(smem), warm_t<true, false, 0>(smem),
        warm_t<true, true, 0>(smem), warm_t<false, false, 1>(smem), warm_t<false, true, 1>(smem),
        warm_t<true, false, 1>(smem), warm_t<true, true, 1>(smem), warm_t<false, false, 2>(smem),
        warm_t<false, true, 2>(smem), warm_t<true, false, 2>(smem), warm_t<true, true, 2>(smem)};
    for (cudaError_t x : r)
        if (x != cudaSuccess) return x;
    return cudaSuccess;
}

// Occupancy of the plain instantiation; the goal-directed one has the same
// launch bounds (register cap) and shared memory.
template <bool DIR, bool LEARNED, bool SERVE, int GS, bool NARROW>
static int occupancy_t(int wpb, int smem) {
    int nb = 0;
    auto* k = search_kernel<DIR, LEARNED, SERVE, GS, NARROW, false>;
    if (!ensure_smem_limit<KernelTag<DIR, LEARNED, SERVE, GS, NARROW, false>>(k, smem)) return 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k, wpb * 32, smem) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return nb;
}

template <bool DIR, bool LEARNED, bool NARROW>
static int occupancy_g(int wpb, int smem, int gs) {
    if (gs == 2) return occupancy_t<DIR, LEARNED, false, 2, NARROW>(wpb, smem);
    if (gs == 4) return occupancy_t<DIR, LEARNED, false, 4, NARROW>(wpb, smem);
    if (gs == 8) return occupancy_t<DIR, LEARNED, false, 8, NARROW>(wpb, smem);
    if (gs == 16) return occupancy_t<DIR, LEARNED, false, 16, NARROW>(wpb, smem);
    return occupancy_t<DIR, LEARNED, false, 32, NARROW>(wpb, smem);
}

template <bool DIR, bool LEARNED>
static int occupancy_w(int wpb, int smem, int gs, bool narrow) {
    return narrow ? occupancy_g<DIR, LEARNED, true>(wpb, smem, gs) : occupancy_g<DIR, LEARNED, false>(wpb, smem, gs);
}

int search_max_blocks_per_sm(int warps_per_block, int smem_per_block, bool directed, bool learned, int gs,
                             bool narrow) {
    if (directed) return learned ? occupancy_w<true, true>(warps_per_block, smem_per_block, gs, narrow)
                                 : occupancy_w<true, false>(warps_per_block, smem_per_block, gs, narrow);
    return learned ? occupancy_w<false, true>(warps_per_block, smem_per_block, gs, narrow)
                   : occupancy_w<false, false>(warps_per_block, smem_per_block, gs, narrow);
}

int serve_max_blocks_per_sm(int warps_per_block, int smem_per_block, int gs) {
    if (gs == 8) return occupancy_t<false, false, true, 8, false>(warps_per_block, smem_per_block);
    if (gs == 16) return occupancy_t<false, false, true, 16, false>(warps_per_block, smem_per_block);
    return occupancy_t<false, false, true, 32, false>(warps_per_block, smem_per_block);
}

// Serve mode: reset the control block and the ring before a server launch.
__global__ void serve_init_kernel(Control* c, u64* qseq, uint32_t qcap, int32_t* in_flight, int block_ring) {
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < qcap; i += gridDim.x * blockDim.x)
        qseq[i] = block_ring ? ~0ull : (u64)i;       // failure injection: no slot ever frees up
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        c->q_head = 0;
        c->q_tail = 0;
        c->remaining = 0x7fffffff;
        c->error = 0;
        c->last_progress = gtimer();
        c->donated = c->stolen = c->spilled = c->class_visits = c->pruned = 0;
        c->busy_cycles = c->idle_cycles = 0;
        c->dbg_code = c->dbg_val = c->dbg_line = c->dbg_count = 0;
        *in_flight = 0;
    }
}

cudaError_t launch_serve_init(Control* ctl, u64* qseq, uint32_t qcap, int32_t* in_flight, int block_ring,
                              cudaStream_t s) {
    serve_init_kernel<<<64, 256, 0, s>>>(ctl, qseq, qcap, in_flight, block_ring);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// integer-pipe micro-benchmark: sustained 32-bit population counts per second
// (the denominator of the search kernel's roofline)
// ---------------------------------------------------------------------------
__global__ void popc_bench_kernel(unsigned long long* out, int iters) {
    unsigned x0 = threadIdx.x * 0x9E3779B9u + blockIdx.x, x1 = x0 ^ 0x55555555u, x2 = x0 * 3u,
             x3 = x0 + 17u, x4 = ~x0, x5 = x0 >> 3, x6 = x0 << 5, x7 = x0 ^ 0xA5A5A5A5u;
    for (int i = 0; i < iters; ++i) {
        // 8 independent popc chains per thread; the xor keeps each chain live
        x0 ^= __popc(x0) + i; x1 ^= __popc(x1) + i; x2 ^= __popc(x2) + i; x3 ^= __popc(x3) + i;
        x4 ^= __popc(x4) + i; x5 ^= __popc(x5) + i; x6 ^= __popc(x6) + i; x7 ^= __popc(x7) + i;
    }
    unsigned acc = x0 ^ x1 ^ x2 ^ x3 ^ x4 ^ x5 ^ x6 ^ x7;
    if (acc == 0x12345678u) out[1] = acc;   // practically never; keeps the work observable
    if (threadIdx.x == 0 && blockIdx.x == 0) out[0] = (unsigned long long)iters;
}

cudaError_t launch_popc_bench(unsigned long long* out, int blocks, int iters, cudaStream_t s) {
    popc_bench_kernel<<<blocks, 256, 0, s>>>(out, iters);
    return cudaGetLastError();
}

}  // namespace mcsk
