// Branching-order network: an FP16 MLP on the tensor cores that scores
// candidate pairs (v, u) so that McSplit tries likely candidates first.
//
// The order never changes the optimum -- every candidate is still tried and
// every bound is still exact -- it only changes how soon a good incumbent is
// found; with no model loaded the degree order is used (the fallback).
//
//   features_kernel  18 features per vertex: degree, label, histogram of the
//                    neighbours' degrees in 16 bins
//   mlp_fwd_kernel   x(v,u) = [f_G(v), f_H(u)] (36, padded to 48) -> 128 ->
//                    128 -> 1 logit; both hidden layers are tcgen05.mma
//                    (kind::f16: f16 operands in shared memory, f32
//                    accumulators in tensor memory), 128 rows per tile
//   bwd kernels      backward pass: a head kernel (logit gradient, w3, b2, b3,
//                    loss), then mlp_bwd_kernel -- dz1 and the W2, W1 and b1
//                    gradients as tcgen05.mma on 128-row tiles -- and an
//                    Adam update
//   keys / rank      per-pair vertex order keys (for the renumbering done by
//                    the pack kernel) and per-v candidate ranks (for the search)
#include <cmath>
#include <cstdio>
#include <cstring>
#include <vector>

#include <cuda_fp16.h>

#include "mcs_internal.cuh"
#include "../../include/mcs.h"

namespace mcsk {

constexpr int kF = 18;            // features per vertex
constexpr int kFP = 32;           // padded row of the fp16 feature table
constexpr int kIn = 48;           // padded network input (36 used)
constexpr int kH = 128;
constexpr int kNParams = kIn * kH + kH + kH * kH + kH + kH + 1;
static_assert(kNParams == MCS_ORDER_NPARAMS, "parameter layout out of date");
constexpr int kOffW1 = 0, kOffB1 = kIn * kH, kOffW2 = kOffB1 + kH, kOffB2 = kOffW2 + kH * kH,
              kOffW3 = kOffB2 + kH, kOffB3 = kOffW3 + kH;

__device__ __forceinline__ uint32_t pack2(float lo, float hi) {
    __half2 h = __floats2half2_rn(lo, hi);
    return *reinterpret_cast<uint32_t*>(&h);
}

// ---------------------------------------------------------------------------
// vertex features: one warp per graph (2 per pair)
// ---------------------------------------------------------------------------
struct FeatParams {
    int32_t npairs;
    uint32_t flags;
    const int32_t* n;
    const int64_t* adj_off;
    const uint8_t* adj;
    const int64_t* lab_off;
    const int32_t* labels;
    float* feat32;       // [npairs*2][64][kF] (may be null)
    __half* feat16;      // [npairs*2][64][kFP]
};

// One warp per graph, on bitsets: lane x (and x + 32) holds the out- and
// in-neighbour sets of its vertex (self-loops excluded), built from coalesced
// row reads and ballots.  degree = |out| (+ |in| if directed); the histogram
// bin b of x counts the neighbours (out or in) whose degree, capped at 15, is
// b: popc(nb(x) & bin_b), with bin_b a ballot over the warp.  All values are
// small multiples of 1/16 or 1/4, exact in fp32.
__global__ void features_kernel(FeatParams P) {
    const int lane = threadIdx.x & 31;
    const int gi = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (gi >= 2 * P.npairs) return;
    const bool directed = (P.flags & MCS_DIRECTED) != 0;
    int n = P.n[gi];
    if (n < 0 || n > kMaxN) n = 0;
    const uint8_t* a = P.adj + P.adj_off[gi];
    const int32_t* lab = (P.labels && P.lab_off && P.lab_off[gi] >= 0) ? P.labels + P.lab_off[gi] : nullptr;
    // out[s]: row of vertex lane + 32 s
    unsigned long long out[2] = {0ull, 0ull};
    for (int x0 = 0; x0 < n; x0 += 8) {
        // eight rows' loads in flight before the votes
        uint8_t blo[8], bhi[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            const int x = x0 + k;
            blo[k] = (x < n && lane < n) ? a[(size_t)x * n + lane] : 0;
            bhi[k] = (x < n && lane + 32 < n) ? a[(size_t)x * n + lane + 32] : 0;
        }
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            const int x = x0 + k;
            const unsigned lo = __ballot_sync(0xffffffffu, blo[k] != 0);
            const unsigned hi = __ballot_sync(0xffffffffu, bhi[k] != 0);
            const unsigned long long row = ((unsigned long long)hi << 32) | lo;
            if (x < n && (x & 31) == lane) { if (x < 32) out[0] = row; else out[1] = row; }
        }
    }
    unsigned long long in[2] = {0ull, 0ull};
    if (directed) {
        for (int y = 0; y < n; ++y) {
            const unsigned long long ry = __shfl_sync(0xffffffffu, y < 32 ? out[0] : out[1], y & 31);
            for (int s = 0; s < 2; ++s)
                if ((ry >> (lane + 32 * s)) & 1ull) in[s] |= 1ull << y;
        }
    }
    int deg[2];
    unsigned long long nb[2];
    for (int s = 0; s < 2; ++s) {
        const int x = lane + 32 * s;
        const unsigned long long self = 1ull << x;
        const unsigned long long o = x < n ? out[s] & ~self : 0ull, i = x < n ? in[s] & ~self : 0ull;
        deg[s] = __popcll(o) + (directed ? __popcll(i) : 0);
        nb[s] = o | i;
    }
    float f[2][kF];
    for (int s = 0; s < 2; ++s)
        for (int k = 0; k < kF; ++k) f[s][k] = 0.f;
    for (int b = 0; b < 16; ++b) {
        const unsigned lo = __ballot_sync(0xffffffffu, lane < n && min(deg[0], 15) == b);
        const unsigned hi = __ballot_sync(0xffffffffu, lane + 32 < n && min(deg[1], 15) == b);
        const unsigned long long bin = ((unsigned long long)hi << 32) | lo;
        for (int s = 0; s < 2; ++s) f[s][2 + b] = 0.25f * (float)__popcll(nb[s] & bin);
    }
    for (int s = 0; s < 2; ++s) {
        const int x = lane + 32 * s;
        if (x < n) {
            f[s][0] = deg[s] / 16.f;
            f[s][1] = lab ? (float)min(lab[x], 63) / 8.f : 0.f;
        } else {
            for (int k = 0; k < kF; ++k) f[s][k] = 0.f;
        }
        const size_t row = (size_t)gi * kMaxN + x;
        if (P.feat32)
            for (int k = 0; k < kF; ++k) P.feat32[row * kF + k] = f[s][k];
        uint32_t w[kFP / 2];
        for (int k = 0; k < kFP / 2; ++k)
            w[k] = 2 * k + 1 < kF ? pack2(f[s][2 * k], f[s][2 * k + 1]) : 0u;
        uint4* dst = reinterpret_cast<uint4*>(P.feat16 + row * kFP);
        for (int k = 0; k < kFP / 8; ++k) dst[k] = make_uint4(w[4 * k], w[4 * k + 1], w[4 * k + 2], w[4 * k + 3]);
    }
}

// ---------------------------------------------------------------------------
// forward pass (inference and training)
// ---------------------------------------------------------------------------
struct FwdParams {
    long long nrows;
    int32_t npairs;
    const int32_t* rows;     // [nrows][3] (pair, v, u) in original ids; null = all-pairs grid
    const int32_t* n;        // vertex counts (grid mode validity)
    const __half* feat16;
    const __half* W1t;       // [128][48]   (out, in)
    const __half* W2t;       // [128][128]  (out, in)
    const float* b1;
    const float* b2;
    const float* w3;
    const float* b3;
    float* s;                // [nrows] logits
    __half* h1;              // training: [nrows][128]
    float* h2;               // training: [nrows][128]
    int* err;                // set to 1 when a bounded wait gives up
};

__device__ __forceinline__ bool row_of(const FwdParams& P, long long r, int& p, int& v, int& u) {
    if (r >= P.nrows) return false;
    if (P.rows) {
        p = P.rows[3 * r]; v = P.rows[3 * r + 1]; u = P.rows[3 * r + 2];
        return v >= 0 && v < kMaxN && u >= 0 && u < kMaxN && p >= 0 && p < P.npairs;
    }
    p = (int)(r >> 12); v = (int)((r >> 6) & 63); u = (int)(r & 63);
    return v < P.n[2 * p] && u < P.n[2 * p + 1];
}

// ---- tcgen05 / TMEM / mbarrier primitives (inline PTX) -------------------
__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void tmem_alloc(uint32_t slot, uint32_t ncols) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" :: "r"(slot), "r"(ncols) : "memory");
}
__device__ __forceinline__ void tmem_relinquish() {
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" :: "r"(taddr), "r"(ncols) : "memory");
}
__device__ __forceinline__ void tc_before_sync() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_after_sync() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
// generic-proxy shared-memory writes -> visible to the tensor core (async proxy)
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void mbar_init(uint32_t a, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" :: "r"(a), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_init_fence() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ bool mbar_try(uint32_t a, uint32_t parity) {
    uint32_t ok;
    asm volatile("{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
                 "selp.u32 %0, 1, 0, p;\n}" : "=r"(ok) : "r"(a), "r"(parity) : "memory");
    return ok != 0;
}
__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
// bounded: gives up (false) after ~2 s (or 2^22 polls) instead of waiting forever
__device__ __forceinline__ bool mbar_wait(uint32_t a, uint32_t parity) {
    const unsigned long long t0 = global_ns();
    for (uint32_t i = 0; i < (1u << 22); ++i) {
        if (mbar_try(a, parity)) return true;
        if ((i & 255) == 255 && global_ns() - t0 > 2000000000ull) return false;
    }
    return false;
}
// D[tmem] (+)= A[smem] * B[smem]^T, one elected thread; acc = 0 overwrites D
__device__ __forceinline__ void umma_f16(uint32_t d, uint64_t adesc, uint64_t bdesc, uint32_t idesc, uint32_t acc) {
    asm volatile("{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                 "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}"
                 :: "r"(d), "l"(adesc), "l"(bdesc), "r"(idesc), "r"(acc) : "memory");
}
// arrives on the mbarrier once every MMA issued so far by this thread is done
__device__ __forceinline__ void umma_commit(uint32_t bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" :: "r"(bar) : "memory");
}
// 32 consecutive fp32 columns of this thread's TMEM lane; the wait carries the
// registers so that no use is scheduled before the load has landed
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&r)[32]) {
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31]) : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5]), "+r"(r[6]), "+r"(r[7]), "+r"(r[8]), "+r"(r[9]), "+r"(r[10]), "+r"(r[11]), "+r"(r[12]), "+r"(r[13]), "+r"(r[14]), "+r"(r[15]), "+r"(r[16]), "+r"(r[17]), "+r"(r[18]), "+r"(r[19]), "+r"(r[20]), "+r"(r[21]), "+r"(r[22]), "+r"(r[23]), "+r"(r[24]), "+r"(r[25]), "+r"(r[26]), "+r"(r[27]), "+r"(r[28]), "+r"(r[29]), "+r"(r[30]), "+r"(r[31]) :: "memory");
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&r)[16]) {
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]) : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5]), "+r"(r[6]), "+r"(r[7]), "+r"(r[8]), "+r"(r[9]), "+r"(r[10]), "+r"(r[11]), "+r"(r[12]), "+r"(r[13]), "+r"(r[14]), "+r"(r[15]) :: "memory");
}

// Shared-memory operand layout for the MMAs: no swizzle, K-major.  The tile is
// cut into 8-row x 16-byte core matrices (8 rows x 8 fp16); the cores of one
// 8-row group are consecutive along K (128 B apart: the leading byte offset)
// and consecutive 8-row groups are K/8 x 128 B apart (the stride byte offset).
__device__ __forceinline__ int kmaj_off(int row, int kchunk, int kchunks) {
    return (row >> 3) * (kchunks * 128) + kchunk * 128 + (row & 7) * 16;
}
// shared-memory matrix descriptor: start >> 4 | LBO >> 4 << 16 | SBO >> 4 << 32 |
// version 1 (bit 46) | no swizzle (bits 61-63 = 0)
__device__ __forceinline__ uint64_t kmaj_desc(uint32_t saddr, int kchunks) {
    const uint64_t lbo = 128, sbo = (uint64_t)kchunks * 128;
    return (uint64_t)((saddr >> 4) & 0x3FFFu) | ((lbo >> 4) << 16) | ((sbo >> 4) << 32) | (1ull << 46);
}

constexpr int kTile = 128;                            // rows per tile = MMA M = TMEM lanes
constexpr int kWorkers = 4;                           // independent 128-row pipelines per CTA
constexpr uint32_t kTmemCols = 512;                   // 128 per worker; layer 2 reuses layer 1's
constexpr int kK2 = kH + 16;                          // layer-2 K: h1 (128), then [1, 0 x 15] for b2
// instruction descriptor, kind::f16: D f32 (bits 4-5 = 1), A and B f16 (bits 7-12 = 0),
// both K-major (bits 15-16 = 0), N >> 3 at bit 17, M >> 4 at bit 24
constexpr uint32_t kIdesc = (1u << 4) | ((uint32_t)(kH >> 3) << 17) | ((uint32_t)(kTile >> 4) << 24);
constexpr int kSW1 = 0;                               // [W1t | b1 at input 36]  128 x 48 fp16
constexpr int kSW2 = kSW1 + kH * kIn * 2;             // [W2t | b2 at k = 128]   128 x 144
constexpr int kSWork = kSW2 + kH * kK2 * 2;           // per worker: A operand, 128 x 144 (x aliases it)
constexpr int kWBytes = kTile * kK2 * 2;
constexpr int kSW3 = kSWork + kWorkers * kWBytes;     // w3 (fp32)
constexpr int kSBar = kSW3 + kH * 4;                  // one mbarrier per worker, then the TMEM base
constexpr int kFwdSmem = kSBar + 8 * kWorkers + 16;
static_assert(kFwdSmem <= 227 * 1024, "shared memory per CTA");
// more than half of the SM's shared memory: one CTA per SM, so its 512 TMEM
// columns are the whole of the SM's tensor memory and the allocation never waits
static_assert(2 * (kFwdSmem + 1024) > 228 * 1024, "TMEM columns could be oversubscribed");

// barrier over the 128 threads of one worker (ids 1..kWorkers; 0 is __syncthreads)
__device__ __forceinline__ void worker_sync(int wk) {
    asm volatile("bar.sync %0, %1;" :: "r"(wk + 1), "r"(kTile) : "memory");
}
__device__ __forceinline__ bool worker_any(int wk, bool x) {
    uint32_t out;
    asm volatile("{\n\t.reg .pred p, q;\n\tsetp.ne.u32 p, %1, 0;\n\t"
                 "bar.red.or.pred q, %2, %3, p;\n\tselp.u32 %0, 1, 0, q;\n}"
                 : "=r"(out) : "r"((uint32_t)x), "r"(wk + 1), "r"(kTile) : "memory");
    return out != 0;
}
__device__ __forceinline__ void worker_fence_sync(int wk) {
    tc_before_sync();
    worker_sync(wk);
    tc_after_sync();
}
// (relu(lo), relu(hi)) rounded to fp16 and packed, lo in the low half
__device__ __forceinline__ uint32_t relu_pack2(float lo, float hi) {
    uint32_t d;
    asm("cvt.rn.relu.f16x2.f32 %0, %1, %2;" : "=r"(d) : "f"(hi), "f"(lo));
    return d;
}

// The next tile this worker computes after t (grid mode skips tiles whose
// two rows v are both >= n_G), or ntiles.
__device__ __forceinline__ long long next_tile(const FwdParams& P, long long t, long long stride, long long ntiles) {
    for (; t < ntiles; t += stride) {
        if (P.rows) return t;
        const int p = (int)(t >> 5), v0 = (int)(t & 31) * 2;
        if (v0 < P.n[2 * p] && P.n[2 * p + 1] > 0) return t;
    }
    return ntiles;
}

// The network input of one row as 5 core-matrix rows (the sixth is [1, 0..]):
// x = [f_G(v) (18), f_H(u) (18), 1 (the b1 input), 0 (11)].
struct XRow { uint4 c[5]; bool ok; };
__device__ __forceinline__ XRow gather_x(const FwdParams& P, long long r) {
    XRow x;
    int p = 0, v = 0, u = 0;
    x.ok = row_of(P, r, p, v, u);
    const uint4 z = make_uint4(0, 0, 0, 0);
    x.c[0] = x.c[1] = x.c[2] = x.c[3] = z;
    x.c[4] = make_uint4(0, 0, 0x3C00u, 0);                // fp16 1.0 at input 36 (b1)
    if (x.ok) {
        const __half* fg = P.feat16 + ((size_t)(2 * p) * kMaxN + v) * kFP;
        const __half* fh = P.feat16 + ((size_t)(2 * p + 1) * kMaxN + u) * kFP;
        const uint4 g0 = reinterpret_cast<const uint4*>(fg)[0], g1 = reinterpret_cast<const uint4*>(fg)[1];
        const uint4 h0 = reinterpret_cast<const uint4*>(fh)[0], h1 = reinterpret_cast<const uint4*>(fh)[1];
        const uint32_t g8 = reinterpret_cast<const uint32_t*>(fg)[8];
        const uint32_t h8 = reinterpret_cast<const uint32_t*>(fh)[8];
        x.c[0] = g0; x.c[1] = g1;
        x.c[2] = make_uint4(g8, h0.x, h0.y, h0.z);
        x.c[3] = make_uint4(h0.w, h1.x, h1.y, h1.z);
        x.c[4] = make_uint4(h1.w, h8, 0x3C00u, 0u);
    }
    return x;
}

// One CTA per SM, persistent: kWorkers groups of 4 warps each take 128-row
// tiles independently (their own operand buffer, mbarrier and 128 TMEM
// columns; the weights are shared).  Per tile: x into shared memory, layer 1
// = 3 MMAs (K = 48, the bias through a constant-1 input) into TMEM, ReLU +
// fp16 by the thread owning the row into shared memory, layer 2 = 9 MMAs
// (K = 144: h1 and a constant-1 column for the bias) into the same columns,
// ReLU + head dot product per thread (row t of the tile is TMEM lane t, read
// by thread t of the worker: warp j of a worker reads lanes 32j..32j+31).
// The next tile's inputs are loaded while the current one computes.  Biases
// b1 and b2 therefore enter as fp16, like the weights.
template <bool TRAIN>
__global__ void __launch_bounds__(kTile * kWorkers, 1) mlp_fwd_kernel(FwdParams P, long long ntiles) {
    extern __shared__ __align__(1024) unsigned char sm[];
    const int tid = threadIdx.x, warp = tid >> 5;
    const int wk = tid / kTile, rt = tid % kTile;
    const uint32_t sbase = smem_u32(sm);
    // weights with the biases as one more input: W1 column 36 = b1, W2 column 128 = b2
    for (int i = tid; i < kH * (kIn / 8); i += kTile * kWorkers) {
        const int n = i / (kIn / 8), kc = i % (kIn / 8);
        uint4 w = *reinterpret_cast<const uint4*>(P.W1t + n * kIn + kc * 8);
        if (kc == 4) w.z = (uint32_t)__half_as_ushort(__float2half_rn(P.b1[n]));   // inputs 36, 37
        *reinterpret_cast<uint4*>(sm + kSW1 + kmaj_off(n, kc, kIn / 8)) = w;
    }
    for (int i = tid; i < kH * (kK2 / 8); i += kTile * kWorkers) {
        const int n = i / (kK2 / 8), kc = i % (kK2 / 8);
        uint4 w = make_uint4(0, 0, 0, 0);
        if (kc < kH / 8) w = *reinterpret_cast<const uint4*>(P.W2t + n * kH + kc * 8);
        else if (kc == kH / 8) w.x = (uint32_t)__half_as_ushort(__float2half_rn(P.b2[n]));
        *reinterpret_cast<uint4*>(sm + kSW2 + kmaj_off(n, kc, kK2 / 8)) = w;
    }
    float* sw3 = reinterpret_cast<float*>(sm + kSW3);
    for (int i = tid; i < kH; i += kTile * kWorkers) sw3[i] = P.w3[i];
    uint32_t* tslot = reinterpret_cast<uint32_t*>(sm + kSBar + 8 * kWorkers);
    if (tid < kWorkers) { mbar_init(sbase + kSBar + 8 * tid, 1); mbar_init_fence(); }
    if (warp == 0) { tmem_alloc(smem_u32(tslot), kTmemCols); tmem_relinquish(); }
    fence_async_smem();
    tc_before_sync();
    __syncthreads();
    tc_after_sync();
    const uint32_t tmem = *tslot + (uint32_t)(wk * kH);            // this worker's columns
    const uint32_t tl = tmem + ((uint32_t)((warp & 3) * 32) << 16);  // this warp's lanes
    const uint32_t bar = sbase + kSBar + 8 * wk;
    const uint32_t sA = sbase + kSWork + wk * kWBytes;
    unsigned char* a = sm + kSWork + wk * kWBytes;
    const float b3 = *P.b3;
    const long long stride = (long long)gridDim.x * kWorkers;
    uint32_t phase = 0;
    long long t = next_tile(P, (long long)blockIdx.x * kWorkers + wk, stride, ntiles);
    XRow x = gather_x(P, t * kTile + rt);
    while (t < ntiles) {
        const long long r = t * kTile + rt;
        const bool ok = x.ok;
        // x (K = 48) in the first 128 x 48 of the buffer, as layer 1's A operand
#pragma unroll
        for (int j = 0; j < 5; ++j) *reinterpret_cast<uint4*>(a + kmaj_off(rt, j, kIn / 8)) = x.c[j];
        *reinterpret_cast<uint4*>(a + kmaj_off(rt, 5, kIn / 8)) = make_uint4(0, 0, 0, 0);
        fence_async_smem();
        worker_fence_sync(wk);
        if (rt == 0) {
#pragma unroll
            for (int k = 0; k < kIn / 16; ++k)
                umma_f16(tmem, kmaj_desc(sA + k * 256, kIn / 8), kmaj_desc(sbase + kSW1 + k * 256, kIn / 8),
                         kIdesc, k > 0);
            umma_commit(bar);
        }
        const long long tn = next_tile(P, t + stride, stride, ntiles);
        x = gather_x(P, tn * kTile + rt);                 // in flight during this tile
        if (worker_any(wk, !mbar_wait(bar, phase))) { if (rt == 0) atomicExch(P.err, 1); break; }
        phase ^= 1u;
        tc_after_sync();
        // ---- layer-1 epilogue: ReLU, fp16 -> A operand of layer 2 (overwrites x)
#pragma unroll
        for (int cb = 0; cb < kH / 16; ++cb) {
            uint32_t acc[16];
            tmem_ld16(tl + cb * 16, acc);
#pragma unroll
            for (int j = 0; j < 2; ++j) {
                const float* f = reinterpret_cast<const float*>(acc) + j * 8;
                const uint4 w = make_uint4(relu_pack2(f[0], f[1]), relu_pack2(f[2], f[3]),
                                           relu_pack2(f[4], f[5]), relu_pack2(f[6], f[7]));
                *reinterpret_cast<uint4*>(a + kmaj_off(rt, cb * 2 + j, kK2 / 8)) = w;
                if (TRAIN && ok) *reinterpret_cast<uint4*>(P.h1 + r * kH + cb * 16 + j * 8) = w;
            }
        }
        *reinterpret_cast<uint4*>(a + kmaj_off(rt, kH / 8, kK2 / 8)) = make_uint4(0x3C00u, 0, 0, 0);
        *reinterpret_cast<uint4*>(a + kmaj_off(rt, kH / 8 + 1, kK2 / 8)) = make_uint4(0, 0, 0, 0);
        // h1 is in shared memory and every warp's TMEM reads are done: layer 2
        // may overwrite the accumulator columns
        fence_async_smem();
        worker_fence_sync(wk);
        if (rt == 0) {
#pragma unroll
            for (int k = 0; k < kK2 / 16; ++k)
                umma_f16(tmem, kmaj_desc(sA + k * 256, kK2 / 8), kmaj_desc(sbase + kSW2 + k * 256, kK2 / 8),
                         kIdesc, k > 0);
            umma_commit(bar);
        }
        if (worker_any(wk, !mbar_wait(bar, phase))) { if (rt == 0) atomicExch(P.err, 1); break; }
        phase ^= 1u;
        tc_after_sync();
        // ---- layer-2 epilogue: ReLU, head
        float sacc = 0.f;
#pragma unroll
        for (int cb = 0; cb < kH / 16; ++cb) {
            uint32_t acc[16];
            tmem_ld16(tl + cb * 16, acc);
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const int c = cb * 16 + j * 4;
                const float4 w = *reinterpret_cast<const float4*>(sw3 + c);
                const float* f = reinterpret_cast<const float*>(acc) + j * 4;
                const float4 h = make_float4(fmaxf(f[0], 0.f), fmaxf(f[1], 0.f), fmaxf(f[2], 0.f), fmaxf(f[3], 0.f));
                sacc = fmaf(h.x, w.x, sacc);
                sacc = fmaf(h.y, w.y, sacc);
                sacc = fmaf(h.z, w.z, sacc);
                sacc = fmaf(h.w, w.w, sacc);
                if (TRAIN && ok) *reinterpret_cast<float4*>(P.h2 + r * kH + c) = h;
            }
        }
        if (ok) P.s[r] = sacc + b3;
        // the next tile overwrites the buffer and the columns just read
        worker_fence_sync(wk);
        t = tn;
    }
    tc_before_sync();
    __syncthreads();
    tc_after_sync();
    if (warp == 0) tmem_dealloc(*tslot, kTmemCols);
}

// ---------------------------------------------------------------------------
// backward pass
// ---------------------------------------------------------------------------
// Gradients are accumulated per row (not yet divided by the batch size B) so
// that fp16 copies of dz stay in the normal range; the Adam step divides by B.
struct HeadParams {
    int32_t nrows;
    const float* s;
    const float* y;
    const float* w;          // may be null
    const float* h2;         // [nrows][128]
    const float* w3;
    __half* dz2;             // out: [nrows][128]
    float* g_w3;             // [128]
    float* g_b2;             // [128]
    float* g_b3;             // [1]
    float* loss;             // [1] sum of w * BCE
};

// block = 128 threads (one per hidden unit), each block a chunk of rows
__global__ void bwd_head_kernel(HeadParams P, int rows_per_block) {
    const int c = threadIdx.x;
    const int r_begin = blockIdx.x * rows_per_block;
    const int r_end = min(P.nrows, r_begin + rows_per_block);
    float gw3 = 0.f, gb2 = 0.f, gb3 = 0.f, ls = 0.f;
    const float w3c = P.w3[c];
    for (int r = r_begin; r < r_end; ++r) {
        const float sr = P.s[r], yr = P.y[r], wr = P.w ? P.w[r] : 1.f;
        const float sig = 1.f / (1.f + expf(-sr));
        const float ds = wr * (sig - yr);
        const float h = P.h2[(size_t)r * kH + c];
        const float dz = h > 0.f ? ds * w3c : 0.f;
        P.dz2[(size_t)r * kH + c] = __float2half_rn(dz);
        gw3 += ds * h;
        gb2 += dz;
        if (c == 0) {
            gb3 += ds;
            ls += wr * (fmaxf(sr, 0.f) + log1pf(expf(-fabsf(sr))) - yr * sr);
        }
    }
    atomicAdd(&P.g_w3[c], gw3);
    atomicAdd(&P.g_b2[c], gb2);
    if (c == 0) { atomicAdd(P.g_b3, gb3); atomicAdd(P.loss, ls); }
}

// ---------------------------------------------------------------------------
// backward GEMMs on the 5th-generation tensor cores (one 128-row tile per CTA)
// ---------------------------------------------------------------------------
// For the rows r of a tile (dz2, h1 from the forward pass, x gathered again):
//   dz1[r][j]   = (sum_o dz2[r][o] W2[j][o]) * (h1[r][j] > 0)      MMA 1 (M r, N j, K o)
//   gW2[i][o]  += sum_r h1[r][i] dz2[r][o]                          MMA 2 (M i, N o, K r)
//   gW1[i][j]  += sum_r x[r][i] dz1[r][j]                           MMA 3 (M i, N j, K r)
// x[r][36] = 1 is the b1 input of the forward pass, so row 36 of MMA 3 is the
// b1 gradient (the sum of dz1 over the rows).  Every operand is K-major in
// shared memory (the layout of the forward pass); the transposed ones (h1,
// dz2, x, dz1 with the rows r as K) are written element by element by the
// thread that owns row r.  Accumulators in TMEM: MMA 1 columns 0-127, MMA 2
// 128-255, MMA 3 256-383; each CTA adds its tile's weight gradients to the
// global sums with atomics.
struct BwdParams {
    FwdParams fp;            // rows, feature table, pair count, row count (for gather_x)
    const __half* W2h;       // [in][out] (as stored in the parameters)
    const __half* h1;        // [nrows][128]
    const __half* dz2;       // [nrows][128]
    float* g_W1;             // [48][128] (rows 36.. not written)
    float* g_b1;             // [128]
    float* g_W2;             // [128][128]
    int* err;
};
constexpr int kBOpBytes = kTile * kH * 2;           // one 128 x 128 fp16 operand
constexpr int kBW2 = 0, kBDz2 = kBOpBytes, kBH1T = 2 * kBOpBytes, kBDz2T = 3 * kBOpBytes,
              kBXT = 4 * kBOpBytes, kBDz1T = 5 * kBOpBytes, kBBar = 6 * kBOpBytes;
constexpr int kBwdSmem = kBBar + 16;
static_assert(kBwdSmem <= 227 * 1024, "shared memory per CTA");
static_assert(2 * (kBwdSmem + 1024) > 228 * 1024, "one CTA per SM: its 512 TMEM columns never wait");

// element (m, k) of a 128-row K-major fp16 operand with K = 128
__device__ __forceinline__ void put_t(unsigned char* base, int m, int k, __half v) {
    *reinterpret_cast<__half*>(base + kmaj_off(m, k >> 3, kH / 8) + (k & 7) * 2) = v;
}

__global__ void __launch_bounds__(kTile, 1) mlp_bwd_kernel(BwdParams P) {
    extern __shared__ __align__(1024) unsigned char sm[];
    const int tid = threadIdx.x, warp = tid >> 5;
    const uint32_t sbase = smem_u32(sm);
    const long long r = (long long)blockIdx.x * kTile + tid;       // this thread's row
    const bool ok = r < P.fp.nrows;
    for (int i = tid; i < kH * (kH / 8); i += kTile) {               // W2h rows: n = in, k = out
        const int n = i / (kH / 8), kc = i % (kH / 8);
        *reinterpret_cast<uint4*>(sm + kBW2 + kmaj_off(n, kc, kH / 8)) =
            *reinterpret_cast<const uint4*>(P.W2h + n * kH + kc * 8);
    }
    // dz2: row r of MMA 1's A, and column r of MMA 2's B
    const __half hz = __ushort_as_half((unsigned short)0);
    for (int c = 0; c < kH / 8; ++c) {
        uint4 v = make_uint4(0, 0, 0, 0);
        if (ok) v = *reinterpret_cast<const uint4*>(P.dz2 + r * kH + c * 8);
        *reinterpret_cast<uint4*>(sm + kBDz2 + kmaj_off(tid, c, kH / 8)) = v;
        const __half* e = reinterpret_cast<const __half*>(&v);
        for (int q = 0; q < 8; ++q) put_t(sm + kBDz2T, c * 8 + q, tid, e[q]);
    }
    // h1: column r of MMA 2's A
    for (int c = 0; c < kH / 8; ++c) {
        uint4 v = make_uint4(0, 0, 0, 0);
        if (ok) v = *reinterpret_cast<const uint4*>(P.h1 + r * kH + c * 8);
        const __half* e = reinterpret_cast<const __half*>(&v);
        for (int q = 0; q < 8; ++q) put_t(sm + kBH1T, c * 8 + q, tid, e[q]);
    }
    // x (48 inputs, the rest of the 128 rows zero): column r of MMA 3's A
    {
        const XRow x = gather_x(P.fp, r);
        for (int c = 0; c < 5; ++c) {
            const __half* e = reinterpret_cast<const __half*>(&x.c[c]);
            for (int q = 0; q < 8; ++q) put_t(sm + kBXT, c * 8 + q, tid, x.ok ? e[q] : hz);
        }
        for (int i = 40; i < kH; ++i) put_t(sm + kBXT, i, tid, hz);
    }
    const uint32_t bar = sbase + kBBar;
    uint32_t* tslot = reinterpret_cast<uint32_t*>(sm + kBBar + 8);
    if (tid == 0) { mbar_init(bar, 1); mbar_init_fence(); }
    if (warp == 0) { tmem_alloc(smem_u32(tslot), 512); tmem_relinquish(); }
    fence_async_smem();
    tc_before_sync();
    __syncthreads();
    tc_after_sync();
    const uint32_t tmem = *tslot;
    const uint32_t lanes = (uint32_t)(warp * 32) << 16;
    bool stalled = false;
    if (tid == 0) {
#pragma unroll
        for (int k = 0; k < kH / 16; ++k) {
            umma_f16(tmem, kmaj_desc(sbase + kBDz2 + k * 256, kH / 8), kmaj_desc(sbase + kBW2 + k * 256, kH / 8),
                     kIdesc, k > 0);
            umma_f16(tmem + 128, kmaj_desc(sbase + kBH1T + k * 256, kH / 8),
                     kmaj_desc(sbase + kBDz2T + k * 256, kH / 8), kIdesc, k > 0);
        }
        umma_commit(bar);
    }
    if (__syncthreads_or(!mbar_wait(bar, 0))) stalled = true;
    tc_after_sync();
    if (!stalled) {
        // dz1 = MMA 1 * (h1 > 0): column r of MMA 3's B
        for (int cb = 0; cb < kH / 16; ++cb) {
            uint32_t acc[16];
            tmem_ld16(tmem + lanes + cb * 16, acc);
            uint4 hv[2] = {make_uint4(0, 0, 0, 0), make_uint4(0, 0, 0, 0)};
            if (ok) {
                hv[0] = *reinterpret_cast<const uint4*>(P.h1 + r * kH + cb * 16);
                hv[1] = *reinterpret_cast<const uint4*>(P.h1 + r * kH + cb * 16 + 8);
            }
            const __half* h = reinterpret_cast<const __half*>(hv);
            for (int q = 0; q < 16; ++q) {
                const float d = __uint_as_float(acc[q]);
                put_t(sm + kBDz1T, cb * 16 + q, tid, __float2half_rn(__half2float(h[q]) > 0.f ? d : 0.f));
            }
        }
        fence_async_smem();
        tc_before_sync();
        __syncthreads();
        tc_after_sync();
        if (tid == 0) {
#pragma unroll
            for (int k = 0; k < kH / 16; ++k)
                umma_f16(tmem + 256, kmaj_desc(sbase + kBXT + k * 256, kH / 8),
                         kmaj_desc(sbase + kBDz1T + k * 256, kH / 8), kIdesc, k > 0);
            umma_commit(bar);
        }
        // MMA 2 is done: row tid of gW2 (input tid) to the global sums
        for (int cb = 0; cb < kH / 16; ++cb) {
            uint32_t acc[16];
            tmem_ld16(tmem + 128 + lanes + cb * 16, acc);
            for (int q = 0; q < 16; ++q) atomicAdd(P.g_W2 + tid * kH + cb * 16 + q, __uint_as_float(acc[q]));
        }
        if (__syncthreads_or(!mbar_wait(bar, 1))) stalled = true;
        tc_after_sync();
        // inputs 0..35 and the b1 input (36) sit in TMEM lanes 0..36: warps 0 and 1
        // load (tcgen05.ld is a whole-warp instruction), rows 0..36 add
        if (!stalled && warp < 2) {
            float* dst = tid < 2 * kF ? P.g_W1 + tid * kH : P.g_b1;
            for (int cb = 0; cb < kH / 16; ++cb) {
                uint32_t acc[16];
                tmem_ld16(tmem + 256 + lanes + cb * 16, acc);
                if (tid <= 2 * kF)
                    for (int q = 0; q < 16; ++q) atomicAdd(dst + cb * 16 + q, __uint_as_float(acc[q]));
            }
        }
    }
    if (stalled && tid == 0) atomicExch(P.err, 1);
    tc_before_sync();
    __syncthreads();
    tc_after_sync();
    if (warp == 0) tmem_dealloc(tmem, 512);
}

// Adam (Kingma & Ba): per-row gradient sums are divided by the batch size
__global__ void adam_kernel(float* theta, float* m, float* v, const float* grad, int n, float inv_b,
                            float lr, float b1, float b2, float eps, float c1, float c2) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        if (i >= kOffW1 + kF * 2 * kH && i < kOffB1) continue;   // padded inputs stay zero
        const float gi = grad[i] * inv_b;
        const float mi = b1 * m[i] + (1.f - b1) * gi;
        const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
        m[i] = mi;
        v[i] = vi;
        theta[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    }
}

// fp32 master parameters -> fp16 tensor-core layouts
__global__ void sync_weights_kernel(const float* theta, __half* W1t, __half* W2t, __half* W2h) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < kH * kH; i += gridDim.x * blockDim.x) {
        const int in = i / kH, out = i % kH;
        W2t[out * kH + in] = __float2half_rn(theta[kOffW2 + i]);
        W2h[i] = __float2half_rn(theta[kOffW2 + i]);
        if (in < kIn) W1t[out * kIn + in] = __float2half_rn(theta[kOffW1 + in * kH + out]);
    }
}

// sample a mini-batch (with replacement) with a counter-based hash
__device__ __forceinline__ unsigned long long mix64(unsigned long long z) {
    z += 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}
__global__ void sample_kernel(const int32_t* rows, const float* y, const float* w, int nrows, int B,
                              unsigned long long seed, unsigned long long step, int32_t* brows,
                              float* by, float* bw) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < B; i += gridDim.x * blockDim.x) {
        const int r = (int)(mix64(seed ^ mix64(step * 0x100000001ull + i)) % (unsigned long long)nrows);
        brows[3 * i] = rows[3 * r];
        brows[3 * i + 1] = rows[3 * r + 1];
        brows[3 * i + 2] = rows[3 * r + 2];
        by[i] = y[r];
        bw[i] = w ? w[r] : 1.f;
    }
}

// ---------------------------------------------------------------------------
// order keys and candidate ranks
// ---------------------------------------------------------------------------
// vscore[p][0][v] = -max_u s(v,u), vscore[p][1][u] = -max_v s(v,u): the pack
// kernel numbers vertices by ascending key, i.e. most promising first.
__global__ void order_keys_kernel(const float* S, const int32_t* n, float* vscore) {
    const int p = blockIdx.x, t = threadIdx.x;      // 64 threads
    const int nG = n[2 * p], nH = n[2 * p + 1];
    const float* Sp = S + (size_t)p * 4096;
    float mg = -INFINITY, mh = -INFINITY;
    for (int j = 0; j < kMaxN; ++j) {
        if (t < nG && j < nH) mg = fmaxf(mg, Sp[t * 64 + j]);
        if (t < nH && j < nG) mh = fmaxf(mh, Sp[j * 64 + t]);
    }
    vscore[((size_t)p * 2) * kMaxN + t] = t < nG ? -mg : 0.f;
    vscore[((size_t)p * 2 + 1) * kMaxN + t] = t < nH ? -mh : 0.f;
}

// rank[p][v'][u'] (renumbered ids): position of u' in decreasing s(v', .)
__global__ void rank_kernel(const float* S, const PairGraph* graphs, uint8_t* rank) {
    const int p = blockIdx.x;
    const PairGraph& pg = graphs[p];
    const int nG = pg.nG, nH = pg.nH;
    const float* Sp = S + (size_t)p * 4096;
    for (int e = threadIdx.x; e < 4096; e += blockDim.x) {
        const int vn = e >> 6, un = e & 63;
        uint8_t r = 255;
        if (pg.valid && vn < nG && un < nH) {
            const int v = pg.permG[vn];
            const float su = Sp[v * 64 + pg.permH[un]];
            int c = 0;
            for (int w = 0; w < nH; ++w) {
                const float sw = Sp[v * 64 + pg.permH[w]];
                c += (sw > su) || (sw == su && w < un);
            }
            r = (uint8_t)c;
        }
        rank[(size_t)p * 4096 + e] = r;
    }
}

}  // namespace mcsk

using namespace mcsk;

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
struct MlpState {
    bool has_model = false;
    float* theta = nullptr;      // fp32 master parameters
    float* adam_m = nullptr;
    float* adam_v = nullptr;
    float* grad = nullptr;
    __half* W1t = nullptr;
    __half* W2t = nullptr;
    __half* W2h = nullptr;
    int* err = nullptr;          // device flag: a bounded wait of the forward kernel gave up
    long long adam_t = 0;
    // scratch
    size_t feat_pairs = 0;
    __half* feat16 = nullptr;
    float* feat32 = nullptr;
    size_t score_rows = 0;
    float* S = nullptr;
    size_t vs_pairs = 0;
    float* vscore = nullptr;
    size_t rank_pairs = 0;
    uint8_t* rank = nullptr;
    size_t train_rows = 0;
    __half* h1 = nullptr;
    float* h2 = nullptr;
    __half* dz2 = nullptr;
    float* s = nullptr;
    int32_t* brows = nullptr;
    float* by = nullptr;
    float* bw = nullptr;
    float* loss = nullptr;
};

namespace {

thread_local char g_mlp_detail[160] = "";

#define CKM(x) do { cudaError_t _e = (x); if (_e != cudaSuccess) { \
    snprintf(g_mlp_detail, sizeof(g_mlp_detail), "%s at mcs_mlp.cu:%d", cudaGetErrorName(_e), __LINE__); \
    return _e == cudaErrorMemoryAllocation ? MCS_ERR_NOMEM : MCS_ERR_CUDA; } } while (0)

template <typename T>
int grow(T*& p, size_t& cap, size_t need) {
    if (need <= cap && p) return 0;
    cudaFree(p);
    p = nullptr;
    cap = 0;
    CKM(cudaMalloc((void**)&p, sizeof(T) * need));
    cap = need;
    return 0;
}

int mlp_state(mcs_ctx* c, MlpState** out) {
    if (!c->mlp) {
        MlpState* m = new (std::nothrow) MlpState();
        if (!m) return MCS_ERR_NOMEM;
        c->mlp = m;
        CKM(cudaMalloc((void**)&m->theta, sizeof(float) * kNParams));
        CKM(cudaMalloc((void**)&m->adam_m, sizeof(float) * kNParams));
        CKM(cudaMalloc((void**)&m->adam_v, sizeof(float) * kNParams));
        CKM(cudaMalloc((void**)&m->grad, sizeof(float) * kNParams));
        CKM(cudaMalloc((void**)&m->W1t, sizeof(__half) * kH * kIn));
        CKM(cudaMalloc((void**)&m->W2t, sizeof(__half) * kH * kH));
        CKM(cudaMalloc((void**)&m->W2h, sizeof(__half) * kH * kH));
        CKM(cudaMalloc((void**)&m->loss, sizeof(float)));
        CKM(cudaMalloc((void**)&m->err, sizeof(int)));
        CKM(cudaMemset(m->err, 0, sizeof(int)));
    }
    *out = c->mlp;
    return 0;
}


int run_features(mcs_ctx* c, MlpState* m, int npairs, const int32_t* d_n, const int64_t* d_adj_off,
                 const uint8_t* d_adj, const int64_t* d_lab_off, const int32_t* d_labels,
                 uint32_t flags, bool want32, cudaStream_t s) {
    size_t cap16 = m->feat_pairs;
    int rc = grow(m->feat16, cap16, (size_t)npairs * 2 * kMaxN * kFP);
    if (rc) return rc;
    if (want32) {
        size_t cap32 = 0;
        cudaFree(m->feat32);
        m->feat32 = nullptr;
        if ((rc = grow(m->feat32, cap32, (size_t)npairs * 2 * kMaxN * kF))) return rc;
    }
    m->feat_pairs = cap16;
    FeatParams fp;
    fp.npairs = npairs; fp.flags = flags; fp.n = d_n; fp.adj_off = d_adj_off; fp.adj = d_adj;
    fp.lab_off = d_lab_off; fp.labels = d_labels;
    fp.feat32 = want32 ? m->feat32 : nullptr;
    fp.feat16 = m->feat16;
    int blocks = (2 * npairs + 3) / 4;
    features_kernel<<<blocks, 128, 0, s>>>(fp);
    CKM(cudaGetLastError());
    return 0;
}

template <bool TRAIN>
int run_forward(const mcs_ctx* c, MlpState* m, int npairs, long long nrows, const int32_t* rows,
                const int32_t* d_n, float* out_s, cudaStream_t s) {
    FwdParams P;
    P.nrows = nrows; P.npairs = npairs; P.rows = rows; P.n = d_n; P.feat16 = m->feat16;
    P.W1t = m->W1t; P.W2t = m->W2t;
    P.b1 = m->theta + kOffB1; P.b2 = m->theta + kOffB2; P.w3 = m->theta + kOffW3; P.b3 = m->theta + kOffB3;
    P.s = out_s; P.h1 = TRAIN ? m->h1 : nullptr; P.h2 = TRAIN ? m->h2 : nullptr;
    P.err = m->err;
    CKM(cudaFuncSetAttribute(mlp_fwd_kernel<TRAIN>, cudaFuncAttributeMaxDynamicSharedMemorySize, kFwdSmem));
    const long long ntiles = (nrows + kTile - 1) / kTile;
    // persistent: one CTA of kWorkers tile pipelines per SM
    const long long need = (ntiles + kWorkers - 1) / kWorkers;
    const long long grid = need < (long long)c->sms ? need : (long long)c->sms;
    if (grid > 0) mlp_fwd_kernel<TRAIN><<<(unsigned)grid, kTile * kWorkers, kFwdSmem, s>>>(P, ntiles);
    CKM(cudaGetLastError());
    return 0;
}

int ensure_train(MlpState* m, size_t B) {
    if (B <= m->train_rows && m->h1) return 0;
    size_t cap = 0;
    int rc;
    cudaFree(m->h1); cudaFree(m->h2); cudaFree(m->dz2); cudaFree(m->s);
    cudaFree(m->brows); cudaFree(m->by); cudaFree(m->bw);
    m->h1 = m->dz2 = nullptr; m->h2 = m->s = m->by = m->bw = nullptr; m->brows = nullptr;
    if ((rc = grow(m->h1, cap, B * kH))) return rc; cap = 0;
    if ((rc = grow(m->dz2, cap, B * kH))) return rc; cap = 0;
    if ((rc = grow(m->h2, cap, B * kH))) return rc; cap = 0;
    if ((rc = grow(m->s, cap, B))) return rc; cap = 0;
    if ((rc = grow(m->brows, cap, 3 * B))) return rc; cap = 0;
    if ((rc = grow(m->by, cap, B))) return rc; cap = 0;
    if ((rc = grow(m->bw, cap, B))) return rc;
    m->train_rows = B;
    return 0;
}

// loss (sum over rows) and per-row gradient sums for the B rows in brows/by/bw
int run_backward(const mcs_ctx* c, MlpState* m, int npairs, int B, const int32_t* rows, const float* y, const float* w,
                 cudaStream_t s) {
    CKM(cudaMemsetAsync(m->grad, 0, sizeof(float) * kNParams, s));
    CKM(cudaMemsetAsync(m->loss, 0, sizeof(float), s));
    int rc = run_forward<true>(c, m, npairs, B, rows, nullptr, m->s, s);
    if (rc) return rc;
    HeadParams hp;
    hp.nrows = B; hp.s = m->s; hp.y = y; hp.w = w; hp.h2 = m->h2; hp.w3 = m->theta + kOffW3;
    hp.dz2 = m->dz2; hp.g_w3 = m->grad + kOffW3; hp.g_b2 = m->grad + kOffB2; hp.g_b3 = m->grad + kOffB3;
    hp.loss = m->loss;
    const int rpb = 64;
    bwd_head_kernel<<<(B + rpb - 1) / rpb, kH, 0, s>>>(hp, rpb);
    CKM(cudaGetLastError());
    // dz1, the W2 and W1 gradients and the b1 gradient: one tensor-core kernel per 128-row tile
    BwdParams bp;
    bp.fp.nrows = B; bp.fp.npairs = npairs; bp.fp.rows = rows; bp.fp.n = nullptr; bp.fp.feat16 = m->feat16;
    bp.W2h = m->W2h; bp.h1 = m->h1; bp.dz2 = m->dz2;
    bp.g_W1 = m->grad + kOffW1; bp.g_b1 = m->grad + kOffB1; bp.g_W2 = m->grad + kOffW2; bp.err = m->err;
    CKM(cudaFuncSetAttribute(mlp_bwd_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kBwdSmem));
    if (B > 0) mlp_bwd_kernel<<<(B + kTile - 1) / kTile, kTile, kBwdSmem, s>>>(bp);
    CKM(cudaGetLastError());
    return 0;
}

int upload_model(mcs_ctx* c, MlpState* m, const float* params) {
    CKM(cudaMemcpyAsync(m->theta, params, sizeof(float) * kNParams, cudaMemcpyHostToDevice, c->stream));
    CKM(cudaMemsetAsync(m->adam_m, 0, sizeof(float) * kNParams, c->stream));
    CKM(cudaMemsetAsync(m->adam_v, 0, sizeof(float) * kNParams, c->stream));
    sync_weights_kernel<<<64, 256, 0, c->stream>>>(m->theta, m->W1t, m->W2t, m->W2h);
    CKM(cudaGetLastError());
    CKM(cudaStreamSynchronize(c->stream));
    m->adam_t = 0;
    m->has_model = true;
    return 0;
}

// reads and clears the forward kernel's stall flag (the stream is idle)
int check_stall(MlpState* m, cudaStream_t s) {
    int e = 0;
    CKM(cudaMemcpyAsync(&e, m->err, sizeof(int), cudaMemcpyDeviceToHost, s));
    CKM(cudaStreamSynchronize(s));
    if (!e) return 0;
    CKM(cudaMemsetAsync(m->err, 0, sizeof(int), s));
    snprintf(g_mlp_detail, sizeof(g_mlp_detail), "mlp_fwd_kernel: tensor-core completion wait gave up");
    return MCS_ERR_DEVICE_STALL;
}

}  // namespace

// Used by run_device (mcs_api.cu) for MCS_ORDER_LEARNED: features, scores of
// every (v, u), and the order keys consumed by the pack kernel.  Returns 1
// when no model is loaded (the caller keeps the degree order).
int mcs_order_prepare(mcs_ctx* c, int npairs, const int32_t* d_n, const int64_t* d_adj_off,
                      const uint8_t* d_adj, const int64_t* d_lab_off, const int32_t* d_labels,
                      uint32_t flags, cudaStream_t s, const float** vscore_out) {
    if (!c->mlp || !c->mlp->has_model) return 1;
    MlpState* m = c->mlp;
    int rc = run_features(c, m, npairs, d_n, d_adj_off, d_adj, d_lab_off, d_labels, flags, false, s);
    if (rc) return rc;
    size_t cap = m->score_rows;
    if ((rc = grow(m->S, cap, (size_t)npairs * 4096))) return rc;
    m->score_rows = cap;
    if ((rc = run_forward<false>(c, m, npairs, (long long)npairs * 4096, nullptr, d_n, m->S, s))) return rc;
    cap = m->vs_pairs;
    if ((rc = grow(m->vscore, cap, (size_t)npairs * 2 * kMaxN))) return rc;
    m->vs_pairs = cap;
    order_keys_kernel<<<npairs, 64, 0, s>>>(m->S, d_n, m->vscore);
    CKM(cudaGetLastError());
    *vscore_out = m->vscore;
    return 0;
}

// After the pack kernel: per-v candidate ranks in the renumbered ids.
int mcs_order_ranks(mcs_ctx* c, int npairs, cudaStream_t s, const uint8_t** rank_out) {
    MlpState* m = c->mlp;
    size_t cap = m->rank_pairs;
    int rc = grow(m->rank, cap, (size_t)npairs * 4096);
    if (rc) return rc;
    m->rank_pairs = cap;
    rank_kernel<<<npairs, 256, 0, s>>>(m->S, c->graphs, m->rank);
    CKM(cudaGetLastError());
    *rank_out = m->rank;
    return 0;
}

void mcs_order_free(mcs_ctx* c) {
    MlpState* m = c->mlp;
    if (!m) return;
    void* ps[] = {m->theta, m->adam_m, m->adam_v, m->grad, m->W1t, m->W2t, m->W2h, m->feat16,
                  m->feat32, m->S, m->vscore, m->rank, m->h1, m->h2, m->dz2, m->s,
                  m->brows, m->by, m->bw, m->loss};
    for (void* p : ps) cudaFree(p);
    delete m;
    c->mlp = nullptr;
}

extern "C" {

int mcs_set_order_model(mcs_ctx* c, const float* params, int32_t nparams) {
    if (!c || !params || nparams != kNParams) return MCS_ERR_ARG;
    if (cudaSetDevice(c->device) != cudaSuccess) return MCS_ERR_CUDA;
    MlpState* m = nullptr;
    int rc = mlp_state(c, &m);
    if (rc) return rc;
    return upload_model(c, m, params);
}

int mcs_get_order_model(mcs_ctx* c, float* params, int32_t nparams) {
    if (!c || !params || nparams != kNParams) return MCS_ERR_ARG;
    if (!c->mlp || !c->mlp->has_model) return MCS_ERR_ARG;
    if (cudaSetDevice(c->device) != cudaSuccess) return MCS_ERR_CUDA;
    CKM(cudaMemcpyAsync(params, c->mlp->theta, sizeof(float) * kNParams, cudaMemcpyDeviceToHost, c->stream));
    CKM(cudaStreamSynchronize(c->stream));
    return 0;
}

int mcs_order_eval(mcs_ctx* c, int32_t npairs, const int32_t* d_n, const int64_t* d_adj_off,
                   const uint8_t* d_adj, const int64_t* d_lab_off, const int32_t* d_labels,
                   uint32_t flags, int32_t nrows, const int32_t* d_rows, const float* d_y,
                   const float* d_w, float* h_scores, float* h_loss, float* h_grad,
                   float* h_features) {
    if (!c || npairs <= 0 || nrows < 0 || !d_n || !d_adj_off || !d_adj) return MCS_ERR_ARG;
    if ((h_loss || h_grad) && !d_y) return MCS_ERR_ARG;
    if ((h_scores || h_loss || h_grad) && (!d_rows || !c->mlp || !c->mlp->has_model)) return MCS_ERR_ARG;
    if (cudaSetDevice(c->device) != cudaSuccess) return MCS_ERR_CUDA;
    MlpState* m = nullptr;
    int rc = mlp_state(c, &m);
    if (rc) return rc;
    cudaStream_t s = c->stream;
    if ((rc = run_features(c, m, npairs, d_n, d_adj_off, d_adj, d_lab_off, d_labels, flags,
                           h_features != nullptr, s)))
        return rc;
    if (h_features)
        CKM(cudaMemcpyAsync(h_features, m->feat32, sizeof(float) * (size_t)npairs * 2 * kMaxN * kF,
                            cudaMemcpyDeviceToHost, s));
    if (nrows > 0 && (h_scores || h_loss || h_grad)) {
        if ((rc = ensure_train(m, (size_t)nrows))) return rc;
        if (h_loss || h_grad) {
            if ((rc = run_backward(c, m, npairs, nrows, d_rows, d_y, d_w, s))) return rc;
        } else {
            if ((rc = run_forward<false>(c, m, npairs, nrows, d_rows, d_n, m->s, s))) return rc;
        }
        if (h_scores) CKM(cudaMemcpyAsync(h_scores, m->s, sizeof(float) * nrows, cudaMemcpyDeviceToHost, s));
        if (h_grad) CKM(cudaMemcpyAsync(h_grad, m->grad, sizeof(float) * kNParams, cudaMemcpyDeviceToHost, s));
        if (h_loss) CKM(cudaMemcpyAsync(h_loss, m->loss, sizeof(float), cudaMemcpyDeviceToHost, s));
    }
    CKM(cudaStreamSynchronize(s));
    if ((rc = check_stall(m, s))) return rc;
    // the device sums over rows; report means
    if (nrows > 0) {
        if (h_loss) *h_loss /= (float)nrows;
        if (h_grad) for (int i = 0; i < kNParams; ++i) h_grad[i] /= (float)nrows;
    }
    return 0;
}

int mcs_order_train(mcs_ctx* c, int32_t npairs, const int32_t* d_n, const int64_t* d_adj_off,
                    const uint8_t* d_adj, const int64_t* d_lab_off, const int32_t* d_labels,
                    uint32_t flags, int32_t nrows, const int32_t* d_rows, const float* d_y,
                    const float* d_w, int32_t steps, int32_t batch, float lr, uint64_t seed,
                    float* h_loss_per_step) {
    if (!c || npairs <= 0 || nrows <= 0 || !d_n || !d_adj_off || !d_adj || !d_rows || !d_y ||
        steps < 0 || batch <= 0 || !(lr > 0.f))
        return MCS_ERR_ARG;
    if (!c->mlp || !c->mlp->has_model) return MCS_ERR_ARG;   // start from mcs_set_order_model
    if (cudaSetDevice(c->device) != cudaSuccess) return MCS_ERR_CUDA;
    MlpState* m = c->mlp;
    cudaStream_t s = c->stream;
    int rc = run_features(c, m, npairs, d_n, d_adj_off, d_adj, d_lab_off, d_labels, flags, false, s);
    if (rc) return rc;
    if ((rc = ensure_train(m, (size_t)batch))) return rc;
    std::vector<float> losses(steps > 0 ? steps : 1, 0.f);
    float* d_losses = nullptr;
    CKM(cudaMalloc((void**)&d_losses, sizeof(float) * (steps > 0 ? steps : 1)));
    const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
    for (int t = 0; t < steps && rc == 0; ++t) {
        sample_kernel<<<(batch + 255) / 256, 256, 0, s>>>(d_rows, d_y, d_w, nrows, batch, seed,
                                                          (unsigned long long)(m->adam_t + 1), m->brows,
                                                          m->by, m->bw);
        if (cudaGetLastError() != cudaSuccess) { rc = MCS_ERR_CUDA; break; }
        if ((rc = run_backward(c, m, npairs, batch, m->brows, m->by, m->bw, s))) break;
        cudaMemcpyAsync(d_losses + t, m->loss, sizeof(float), cudaMemcpyDeviceToDevice, s);
        m->adam_t += 1;
        const float c1 = 1.f - powf(b1, (float)m->adam_t), c2 = 1.f - powf(b2, (float)m->adam_t);
        adam_kernel<<<64, 256, 0, s>>>(m->theta, m->adam_m, m->adam_v, m->grad, kNParams,
                                       1.f / (float)batch, lr, b1, b2, eps, c1, c2);
        sync_weights_kernel<<<64, 256, 0, s>>>(m->theta, m->W1t, m->W2t, m->W2h);
        if (cudaGetLastError() != cudaSuccess) { rc = MCS_ERR_CUDA; break; }
    }
    if (rc == 0 && steps > 0) {
        if (cudaMemcpyAsync(losses.data(), d_losses, sizeof(float) * steps, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
            cudaStreamSynchronize(s) != cudaSuccess)
            rc = MCS_ERR_CUDA;
        if (h_loss_per_step)
            for (int t = 0; t < steps; ++t) h_loss_per_step[t] = losses[t] / (float)batch;
    }
    cudaFree(d_losses);
    if (rc == 0) rc = check_stall(m, s);
    return rc;
}

int mcs_order_score_grid(mcs_ctx* c, int32_t npairs, const int32_t* d_n, const int64_t* d_adj_off,
                         const uint8_t* d_adj, const int64_t* d_lab_off, const int32_t* d_labels,
                         uint32_t flags, float* d_scores, void* stream) {
    if (!c || npairs < 0 || (npairs > 0 && (!d_n || !d_adj_off || !d_adj || !d_scores))) return MCS_ERR_ARG;
    if (!c->mlp || !c->mlp->has_model) return MCS_ERR_ARG;
    if (npairs == 0) return 0;
    if (cudaSetDevice(c->device) != cudaSuccess) return MCS_ERR_CUDA;
    MlpState* m = c->mlp;
    cudaStream_t s = stream ? (cudaStream_t)stream : c->stream;
    int rc = run_features(c, m, npairs, d_n, d_adj_off, d_adj, d_lab_off, d_labels, flags, false, s);
    if (rc) return rc;
    return run_forward<false>(c, m, npairs, (long long)npairs * 4096, nullptr, d_n, d_scores, s);
}

}  // extern "C"
