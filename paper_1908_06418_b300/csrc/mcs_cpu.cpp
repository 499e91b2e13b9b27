// The CPU side of the GPU + CPU race (MCS_RACE): a sequential McSplit on the
// host that searches the same pair as the GPU and shares its incumbent.
//
// The paper's portfolio runs several solvers on one instance and keeps the
// first to finish (Section IV); here one contender is the GPU search and the
// other this CPU search.  It follows the same branch and bound (Section II-B,
// Algorithm 1: label classes split by adjacency to each new pair, Table 1;
// the bound of Eq. 1), on 64-bit bit sets: a class is a (G set, H set) pair.
// The incumbent is shared through two words of mapped host memory, each with
// one writer: the CPU publishes its best size in `cpu_best` and reads the
// GPU's in `gpu_best`, and prunes against the larger of the two (a size that
// either side has found as a mapping).  The search stops when it finishes,
// when `stop` is raised (the GPU finished first), or at its time limit.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <cstdint>
#include <cstring>
#include <vector>

#include "mcs_cpu.h"

namespace {

typedef unsigned long long u64;

struct Cls {
    u64 L, R;
};

struct Search {
    int nG = 0, nH = 0;
    bool directed = false;
    u64 gout[64], gin[64], hout[64], hin[64];     // rows in the new numbering
    int permG[64], permH[64];                     // new number -> original
    // shared incumbent
    const volatile int32_t* gpu_best = nullptr;
    volatile int32_t* cpu_best = nullptr;
    const volatile int32_t* stop = nullptr;
    std::chrono::steady_clock::time_point deadline;
    bool has_deadline = false;
    // state
    int best = 0;                                 // this side's best size
    int bestG[64], bestH[64];
    int curG[64], curH[64];
    uint64_t nodes = 0;
    bool aborted = false;
    std::vector<Cls> stack;                       // classes of every open level

    int shared_best() const {
        int g = gpu_best ? *gpu_best : 0;
        return std::max(best, g);
    }
    bool should_stop() {
        if (aborted) return true;
        if ((nodes & 1023) != 0) return false;
        if (stop && *stop) aborted = true;
        if (has_deadline && std::chrono::steady_clock::now() > deadline) aborted = true;
        return aborted;
    }
    // classes [b, e) of the stack; depth = |M|
    void solve(size_t b, size_t e, int depth) {
        ++nodes;
        if (should_stop()) return;
        if (depth > best) {
            best = depth;
            std::copy(curG, curG + depth, bestG);
            std::copy(curH, curH + depth, bestH);
            if (cpu_best) *cpu_best = best;
        }
        int bound = depth;
        size_t pick = e;
        unsigned key = ~0u;
        for (size_t i = b; i < e; ++i) {
            const int a = __builtin_popcountll(stack[i].L), c = __builtin_popcountll(stack[i].R);
            bound += std::min(a, c);
            if (stack[i].L == 0) continue;
            const unsigned k = ((unsigned)std::max(a, c) << 6) | (unsigned)__builtin_ctzll(stack[i].L);
            if (k < key) { key = k; pick = i; }
        }
        if (bound <= shared_best() || pick == e) return;
        const int v = __builtin_ctzll(stack[pick].L);
        u64 cand = stack[pick].R;
        while (cand) {
            const int u = __builtin_ctzll(cand);
            cand &= cand - 1;
            // split every class by adjacency to v in G and to u in H (Table 1)
            const size_t nb = stack.size();
            const u64 gB = gout[v], hB = hout[u], gA = directed ? gin[v] : 0, hA = directed ? hin[u] : 0;
            for (size_t i = b; i < e; ++i) {
                const u64 L = stack[i].L & ~(1ull << v), R = stack[i].R & ~(1ull << u);
                if (directed) {
                    const u64 lo = L & gB, li = L & gA, ro = R & hB, ri = R & hA;
                    const u64 lp[4] = {L & ~(lo | li), lo & ~li, li & ~lo, lo & li};
                    const u64 rp[4] = {R & ~(ro | ri), ro & ~ri, ri & ~ro, ro & ri};
                    for (int k = 0; k < 4; ++k)
                        if (lp[k] && rp[k]) stack.push_back(Cls{lp[k], rp[k]});
                } else {
                    const u64 l1 = L & gB, r1 = R & hB;
                    if (l1 && r1) stack.push_back(Cls{l1, r1});
                    if ((L ^ l1) && (R ^ r1)) stack.push_back(Cls{L ^ l1, R ^ r1});
                }
            }
            curG[depth] = v;
            curH[depth] = u;
            solve(nb, stack.size(), depth + 1);
            stack.resize(nb);
            if (aborted) return;
        }
        // "v stays unmatched": v leaves its class, M unchanged
        const u64 saved = stack[pick].L;
        stack[pick].L &= ~(1ull << v);
        solve(b, e, depth);
        stack[pick].L = saved;
    }
};

// Renumbers a graph by descending total degree (ties to the lower index) and
// packs its rows.  Returns false for a malformed matrix.
bool pack(int n, const uint8_t* a, bool directed, u64* out, u64* in, int* perm, int* newnum) {
    if (n < 0 || n > 64 || (n > 0 && !a)) return false;
    std::vector<int> deg(n, 0);
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) {
            const uint8_t x = a[i * n + j];
            if (x > 1) return false;
            if (!directed && x != a[j * n + i]) return false;
            if (i != j) { deg[i] += x; if (directed) deg[j] += x; }
        }
    std::vector<int> order(n);
    for (int i = 0; i < n; ++i) order[i] = i;
    std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return deg[x] > deg[y]; });
    for (int r = 0; r < n; ++r) { perm[r] = order[r]; newnum[order[r]] = r; }
    for (int r = 0; r < n; ++r) { out[r] = 0; in[r] = 0; }
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j)
            if (i != j && a[i * n + j]) {
                out[newnum[i]] |= 1ull << newnum[j];
                in[newnum[j]] |= 1ull << newnum[i];
            }
    if (!directed)
        for (int r = 0; r < n; ++r) in[r] = out[r];
    return true;
}

}  // namespace

int cpu_mcs_race(int nG, const uint8_t* adjG, const int32_t* labG, int nH, const uint8_t* adjH,
                 const int32_t* labH, bool directed, double timeout_s, const volatile int32_t* gpu_best,
                 volatile int32_t* cpu_best, const volatile int32_t* stop, CpuRaceResult* out) {
    Search S;
    S.nG = nG;
    S.nH = nH;
    S.directed = directed;
    S.gpu_best = gpu_best;
    S.cpu_best = cpu_best;
    S.stop = stop;
    if (timeout_s > 0) {
        S.has_deadline = true;
        S.deadline = std::chrono::steady_clock::now() +
                     std::chrono::microseconds((long long)(timeout_s * 1e6));
    }
    int newG[64], newH[64];
    out->size = 0;
    out->nodes = 0;
    out->complete = false;
    if (!pack(nG, adjG, directed, S.gout, S.gin, S.permG, newG) ||
        !pack(nH, adjH, directed, S.hout, S.hin, S.permH, newH))
        return -1;
    if (labG) for (int i = 0; i < nG; ++i) if (labG[i] < 0) return -1;
    if (labH) for (int i = 0; i < nH; ++i) if (labH[i] < 0) return -1;
    // root classes: one per (label, self-loop) value present in both graphs
    auto key = [](const int32_t* lab, const uint8_t* a, int n, int x) {
        return (long long)(lab ? lab[x] : 0) * 2 + (a[x * n + x] ? 1 : 0);
    };
    std::vector<long long> keys;
    for (int x = 0; x < nG; ++x) keys.push_back(key(labG, adjG, nG, x));
    std::sort(keys.begin(), keys.end());
    keys.erase(std::unique(keys.begin(), keys.end()), keys.end());
    for (long long k : keys) {
        Cls c{0, 0};
        for (int x = 0; x < nG; ++x) if (key(labG, adjG, nG, x) == k) c.L |= 1ull << newG[x];
        for (int y = 0; y < nH; ++y) if (key(labH, adjH, nH, y) == k) c.R |= 1ull << newH[y];
        if (c.L && c.R) S.stack.push_back(c);
    }
    S.stack.reserve(64 * 65);
    S.solve(0, S.stack.size(), 0);
    out->size = S.best;
    out->nodes = S.nodes;
    out->complete = !S.aborted;
    for (int i = 0; i < S.best; ++i) {
        out->g[i] = (int16_t)S.permG[S.bestG[i]];
        out->h[i] = (int16_t)S.permH[S.bestH[i]];
    }
    return 0;
}
