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
//                    128 -> 1 logit; both hidden layers are mma.sync
//                    m16n8k16 (f16 in, f32 accumulate) with the layer-1 result
//                    converted to layer-2 A fragments in registers
//   bwd kernels      backward pass (head, two tensor-core GEMMs for dh1 and the
//                    weight gradients, column sums) and an Adam update
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

__device__ __forceinline__ void mma16816(float (&d)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.f16.f16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}
__device__ __forceinline__ uint32_t pack2(float lo, float hi) {
    __half2 h = __floats2half2_rn(lo, hi);
    return *reinterpret_cast<uint32_t*>(&h);
}
__device__ __forceinline__ uint32_t pack2h(__half lo, __half hi) {
    return (uint32_t)__half_as_ushort(lo) | ((uint32_t)__half_as_ushort(hi) << 16);
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

__global__ void features_kernel(FeatParams P) {
    const int lane = threadIdx.x & 31;
    const int gi = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (gi >= 2 * P.npairs) return;
    const bool directed = (P.flags & MCS_DIRECTED) != 0;
    int n = P.n[gi];
    if (n < 0 || n > kMaxN) n = 0;
    const uint8_t* a = P.adj + P.adj_off[gi];
    const int32_t* lab = (P.labels && P.lab_off && P.lab_off[gi] >= 0) ? P.labels + P.lab_off[gi] : nullptr;
    int deg[2];
    for (int s = 0; s < 2; ++s) {
        int x = lane + 32 * s, d = 0;
        if (x < n)
            for (int y = 0; y < n; ++y) {
                if (y == x) continue;
                d += a[x * n + y] != 0;
                if (directed) d += a[y * n + x] != 0;
            }
        deg[s] = d;
    }
    float hist[2][16];
    for (int s = 0; s < 2; ++s)
        for (int b = 0; b < 16; ++b) hist[s][b] = 0.f;
    for (int y = 0; y < n; ++y) {
        const int dy = __shfl_sync(0xffffffffu, deg[y >> 5], y & 31);
        const int by = dy < 15 ? dy : 15;
        for (int s = 0; s < 2; ++s) {
            int x = lane + 32 * s;
            if (x < n && y != x) {
                bool nb = a[x * n + y] != 0 || (directed && a[y * n + x] != 0);
                if (nb) {
#pragma unroll
                    for (int b = 0; b < 16; ++b) hist[s][b] += (b == by) ? 0.25f : 0.f;
                }
            }
        }
    }
    for (int s = 0; s < 2; ++s) {
        int x = lane + 32 * s;
        float f[kF];
        f[0] = x < n ? deg[s] / 16.f : 0.f;
        f[1] = (x < n && lab) ? (float)min(lab[x], 63) / 8.f : 0.f;
        for (int b = 0; b < 16; ++b) f[2 + b] = x < n ? hist[s][b] : 0.f;
        size_t row = (size_t)gi * kMaxN + x;
        if (P.feat32)
            for (int k = 0; k < kF; ++k) P.feat32[row * kF + k] = f[k];
        for (int k = 0; k < kFP; ++k) P.feat16[row * kFP + k] = __float2half_rn(k < kF ? f[k] : 0.f);
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

// x(row, k..k+1) for even k: G features, then H features, then zeros
__device__ __forceinline__ uint32_t xpair(const __half* fg, const __half* fh, int k) {
    if (k < kF) return *reinterpret_cast<const uint32_t*>(fg + k);
    if (k < 2 * kF) return *reinterpret_cast<const uint32_t*>(fh + (k - kF));
    return 0u;
}

template <bool TRAIN>
__global__ void __launch_bounds__(256) mlp_fwd_kernel(FwdParams P) {
    extern __shared__ __align__(16) unsigned char sm[];
    __half* sW1t = reinterpret_cast<__half*>(sm);           // 128 x 48
    __half* sW2t = sW1t + kH * kIn;                         // 128 x 128
    float* sb1 = reinterpret_cast<float*>(sW2t + kH * kH);
    float* sb2 = sb1 + kH;
    float* sw3 = sb2 + kH;
    for (int i = threadIdx.x; i < kH * kIn / 2; i += blockDim.x)
        reinterpret_cast<uint32_t*>(sW1t)[i] = reinterpret_cast<const uint32_t*>(P.W1t)[i];
    for (int i = threadIdx.x; i < kH * kH / 2; i += blockDim.x)
        reinterpret_cast<uint32_t*>(sW2t)[i] = reinterpret_cast<const uint32_t*>(P.W2t)[i];
    for (int i = threadIdx.x; i < kH; i += blockDim.x) { sb1[i] = P.b1[i]; sb2[i] = P.b2[i]; sw3[i] = P.w3[i]; }
    __syncthreads();
    const float b3 = *P.b3;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int g = lane >> 2, tq = lane & 3;
    const long long r0 = (long long)blockIdx.x * 128 + warp * 16;
    const __half* fg[2];
    const __half* fh[2];
    bool ok[2];
    long long rr[2];
    for (int h = 0; h < 2; ++h) {
        rr[h] = r0 + g + 8 * h;
        int p = 0, v = 0, u = 0;
        ok[h] = row_of(P, rr[h], p, v, u);
        if (!ok[h]) { p = 0; v = 0; u = 0; }
        fg[h] = P.feat16 + ((size_t)(2 * p) * kMaxN + v) * kFP;
        fh[h] = P.feat16 + ((size_t)(2 * p + 1) * kMaxN + u) * kFP;
    }
    // ---- layer 1: [16 x 48] x [48 x 128]
    float acc[16][4];
#pragma unroll
    for (int nt = 0; nt < 16; ++nt) acc[nt][0] = acc[nt][1] = acc[nt][2] = acc[nt][3] = 0.f;
#pragma unroll
    for (int kt = 0; kt < 3; ++kt) {
        const int k0 = kt * 16 + 2 * tq;
        uint32_t a[4];
        a[0] = ok[0] ? xpair(fg[0], fh[0], k0) : 0u;
        a[1] = ok[1] ? xpair(fg[1], fh[1], k0) : 0u;
        a[2] = ok[0] ? xpair(fg[0], fh[0], k0 + 8) : 0u;
        a[3] = ok[1] ? xpair(fg[1], fh[1], k0 + 8) : 0u;
#pragma unroll
        for (int nt = 0; nt < 16; ++nt) {
            const __half* wb = sW1t + (nt * 8 + g) * kIn + k0;
            mma16816(acc[nt], a, *reinterpret_cast<const uint32_t*>(wb),
                     *reinterpret_cast<const uint32_t*>(wb + 8));
        }
    }
    // ---- bias + ReLU, re-packed as layer-2 A fragments (k-tile = two n-tiles)
    uint32_t a2[8][4];
#pragma unroll
    for (int kt = 0; kt < 8; ++kt) {
        const int c0 = kt * 16 + 2 * tq;
        a2[kt][0] = pack2(fmaxf(acc[2 * kt][0] + sb1[c0], 0.f), fmaxf(acc[2 * kt][1] + sb1[c0 + 1], 0.f));
        a2[kt][1] = pack2(fmaxf(acc[2 * kt][2] + sb1[c0], 0.f), fmaxf(acc[2 * kt][3] + sb1[c0 + 1], 0.f));
        a2[kt][2] = pack2(fmaxf(acc[2 * kt + 1][0] + sb1[c0 + 8], 0.f), fmaxf(acc[2 * kt + 1][1] + sb1[c0 + 9], 0.f));
        a2[kt][3] = pack2(fmaxf(acc[2 * kt + 1][2] + sb1[c0 + 8], 0.f), fmaxf(acc[2 * kt + 1][3] + sb1[c0 + 9], 0.f));
        if (TRAIN) {
            if (ok[0]) {
                *reinterpret_cast<uint32_t*>(P.h1 + rr[0] * kH + c0) = a2[kt][0];
                *reinterpret_cast<uint32_t*>(P.h1 + rr[0] * kH + c0 + 8) = a2[kt][2];
            }
            if (ok[1]) {
                *reinterpret_cast<uint32_t*>(P.h1 + rr[1] * kH + c0) = a2[kt][1];
                *reinterpret_cast<uint32_t*>(P.h1 + rr[1] * kH + c0 + 8) = a2[kt][3];
            }
        }
    }
    // ---- layer 2: [16 x 128] x [128 x 128]
#pragma unroll
    for (int nt = 0; nt < 16; ++nt) acc[nt][0] = acc[nt][1] = acc[nt][2] = acc[nt][3] = 0.f;
#pragma unroll
    for (int kt = 0; kt < 8; ++kt) {
#pragma unroll
        for (int nt = 0; nt < 16; ++nt) {
            const __half* wb = sW2t + (nt * 8 + g) * kH + kt * 16 + 2 * tq;
            mma16816(acc[nt], a2[kt], *reinterpret_cast<const uint32_t*>(wb),
                     *reinterpret_cast<const uint32_t*>(wb + 8));
        }
    }
    // ---- bias + ReLU, head dot product (quad reduction over the 4 lanes of a row)
    float s0 = 0.f, s1 = 0.f;
#pragma unroll
    for (int nt = 0; nt < 16; ++nt) {
        const int c = nt * 8 + 2 * tq;
        const float h00 = fmaxf(acc[nt][0] + sb2[c], 0.f), h01 = fmaxf(acc[nt][1] + sb2[c + 1], 0.f);
        const float h10 = fmaxf(acc[nt][2] + sb2[c], 0.f), h11 = fmaxf(acc[nt][3] + sb2[c + 1], 0.f);
        s0 += h00 * sw3[c] + h01 * sw3[c + 1];
        s1 += h10 * sw3[c] + h11 * sw3[c + 1];
        if (TRAIN) {
            if (ok[0]) *reinterpret_cast<float2*>(P.h2 + rr[0] * kH + c) = make_float2(h00, h01);
            if (ok[1]) *reinterpret_cast<float2*>(P.h2 + rr[1] * kH + c) = make_float2(h10, h11);
        }
    }
    s0 += __shfl_xor_sync(0xffffffffu, s0, 1);
    s0 += __shfl_xor_sync(0xffffffffu, s0, 2);
    s1 += __shfl_xor_sync(0xffffffffu, s1, 1);
    s1 += __shfl_xor_sync(0xffffffffu, s1, 2);
    if (tq == 0) {
        if (ok[0]) P.s[rr[0]] = s0 + b3;
        if (ok[1]) P.s[rr[1]] = s1 + b3;
    }
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

// Generic tensor-core GEMM: C(m,n) (+)= sum_k A(m,k) B(k,n); one warp per
// 16 x 64 output tile and K chunk.  A.pair(m,k) packs A(m,k), A(m,k+1);
// B.pair(k,n) packs B(k,n), B(k+1,n) (k even, zero outside the matrix).
template <class AF, class BF, class CF>
__global__ void gemm_kernel(int M, int N, int K, int kchunk, AF A, BF B, CF C) {
    const int lane = threadIdx.x & 31, g = lane >> 2, tq = lane & 3;
    const int m0 = blockIdx.x * 16, n0 = blockIdx.y * 64;
    const int kb = blockIdx.z * kchunk, ke = min(K, kb + kchunk);
    float acc[8][4];
#pragma unroll
    for (int nt = 0; nt < 8; ++nt) acc[nt][0] = acc[nt][1] = acc[nt][2] = acc[nt][3] = 0.f;
    for (int k0 = kb; k0 < ke; k0 += 16) {
        uint32_t a[4];
        a[0] = A.pair(m0 + g, k0 + 2 * tq, M, ke);
        a[1] = A.pair(m0 + g + 8, k0 + 2 * tq, M, ke);
        a[2] = A.pair(m0 + g, k0 + 2 * tq + 8, M, ke);
        a[3] = A.pair(m0 + g + 8, k0 + 2 * tq + 8, M, ke);
#pragma unroll
        for (int nt = 0; nt < 8; ++nt) {
            const int n = n0 + nt * 8 + g;
            mma16816(acc[nt], a, B.pair(k0 + 2 * tq, n, N, ke), B.pair(k0 + 2 * tq + 8, n, N, ke));
        }
    }
#pragma unroll
    for (int nt = 0; nt < 8; ++nt) {
        const int n = n0 + nt * 8 + 2 * tq;
        C.put(m0 + g, n, acc[nt][0], M, N);
        C.put(m0 + g, n + 1, acc[nt][1], M, N);
        C.put(m0 + g + 8, n, acc[nt][2], M, N);
        C.put(m0 + g + 8, n + 1, acc[nt][3], M, N);
    }
}

__device__ __forceinline__ __half hz() { return __ushort_as_half((unsigned short)0); }

// row-major fp16 matrix, pairs along the second index (contiguous)
struct RowPairA {
    const __half* p; int ld;
    __device__ uint32_t pair(int m, int k, int M, int K) const {
        if (m >= M || k >= K) return 0u;
        if (k + 1 < K) return *reinterpret_cast<const uint32_t*>(p + (size_t)m * ld + k);
        return pack2h(p[(size_t)m * ld + k], hz());
    }
};
// B(k, n) = W[n][k]: fp16 matrix stored [n][k]; pairs along k contiguous
struct NKPairB {
    const __half* p; int ld;
    __device__ uint32_t pair(int k, int n, int N, int K) const {
        if (n >= N || k >= K) return 0u;
        if (k + 1 < K) return *reinterpret_cast<const uint32_t*>(p + (size_t)n * ld + k);
        return pack2h(p[(size_t)n * ld + k], hz());
    }
};
// A(m, k) = X[k][m] (X stored [k][m]); pairs along k are strided
struct TransA {
    const __half* p; int ld;
    __device__ uint32_t pair(int m, int k, int M, int K) const {
        if (m >= M || k >= K) return 0u;
        __half lo = p[(size_t)k * ld + m];
        __half hi = (k + 1 < K) ? p[(size_t)(k + 1) * ld + m] : hz();
        return pack2h(lo, hi);
    }
};
// B(k, n) = X[k][n] (X stored [k][n]); pairs along k are strided
struct KNPairB {
    const __half* p; int ld;
    __device__ uint32_t pair(int k, int n, int N, int K) const {
        if (n >= N || k >= K) return 0u;
        __half lo = p[(size_t)k * ld + n];
        __half hi = (k + 1 < K) ? p[(size_t)(k + 1) * ld + n] : hz();
        return pack2h(lo, hi);
    }
};
// A(i, r) = x(row r, input i): gathered from the feature table
struct InputTA {
    const int32_t* rows; const __half* feat; int npairs;
    __device__ __half at(int i, int r) const {
        const int p = rows[3 * r], v = rows[3 * r + 1], u = rows[3 * r + 2];
        if (p < 0 || p >= npairs || v < 0 || v >= kMaxN || u < 0 || u >= kMaxN) return hz();
        if (i < kF) return feat[((size_t)(2 * p) * kMaxN + v) * kFP + i];
        if (i < 2 * kF) return feat[((size_t)(2 * p + 1) * kMaxN + u) * kFP + (i - kF)];
        return hz();
    }
    __device__ uint32_t pair(int m, int k, int M, int K) const {
        if (m >= M || k >= K) return 0u;
        return pack2h(at(m, k), k + 1 < K ? at(m, k + 1) : hz());
    }
};
// dz1 = acc * (h1 > 0), stored fp16 [r][i]
struct StoreDz1 {
    __half* dz1; const __half* h1;
    __device__ void put(int m, int n, float v, int M, int N) const {
        if (m >= M || n >= N) return;
        const size_t o = (size_t)m * kH + n;
        dz1[o] = __float2half_rn(__half2float(h1[o]) > 0.f ? v : 0.f);
    }
};
struct AtomicAddC {
    float* g; int ld;
    __device__ void put(int m, int n, float v, int M, int N) const {
        if (m >= M || n >= N) return;
        atomicAdd(g + (size_t)m * ld + n, v);
    }
};

// column sums of dz1 -> g_b1
__global__ void colsum_kernel(const __half* x, int nrows, float* out) {
    const int c = threadIdx.x;
    float acc = 0.f;
    for (int r = blockIdx.x; r < nrows; r += gridDim.x) acc += __half2float(x[(size_t)r * kH + c]);
    atomicAdd(out + c, acc);
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
    __half* dz1 = nullptr;
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
    }
    *out = c->mlp;
    return 0;
}

size_t fwd_smem() { return sizeof(__half) * (kH * kIn + kH * kH) + sizeof(float) * 3 * kH; }

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
int run_forward(MlpState* m, int npairs, long long nrows, const int32_t* rows, const int32_t* d_n,
                float* out_s, cudaStream_t s) {
    FwdParams P;
    P.nrows = nrows; P.npairs = npairs; P.rows = rows; P.n = d_n; P.feat16 = m->feat16;
    P.W1t = m->W1t; P.W2t = m->W2t;
    P.b1 = m->theta + kOffB1; P.b2 = m->theta + kOffB2; P.w3 = m->theta + kOffW3; P.b3 = m->theta + kOffB3;
    P.s = out_s; P.h1 = TRAIN ? m->h1 : nullptr; P.h2 = TRAIN ? m->h2 : nullptr;
    const size_t sm = fwd_smem();
    CKM(cudaFuncSetAttribute(mlp_fwd_kernel<TRAIN>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
    const long long blocks = (nrows + 127) / 128;
    if (blocks > 0) mlp_fwd_kernel<TRAIN><<<(unsigned)blocks, 256, sm, s>>>(P);
    CKM(cudaGetLastError());
    return 0;
}

int ensure_train(MlpState* m, size_t B) {
    if (B <= m->train_rows && m->h1) return 0;
    size_t cap = 0;
    int rc;
    cudaFree(m->h1); cudaFree(m->h2); cudaFree(m->dz2); cudaFree(m->dz1); cudaFree(m->s);
    cudaFree(m->brows); cudaFree(m->by); cudaFree(m->bw);
    m->h1 = m->dz2 = m->dz1 = nullptr; m->h2 = m->s = m->by = m->bw = nullptr; m->brows = nullptr;
    if ((rc = grow(m->h1, cap, B * kH))) return rc; cap = 0;
    if ((rc = grow(m->dz2, cap, B * kH))) return rc; cap = 0;
    if ((rc = grow(m->dz1, cap, B * kH))) return rc; cap = 0;
    if ((rc = grow(m->h2, cap, B * kH))) return rc; cap = 0;
    if ((rc = grow(m->s, cap, B))) return rc; cap = 0;
    if ((rc = grow(m->brows, cap, 3 * B))) return rc; cap = 0;
    if ((rc = grow(m->by, cap, B))) return rc; cap = 0;
    if ((rc = grow(m->bw, cap, B))) return rc;
    m->train_rows = B;
    return 0;
}

// loss (sum over rows) and per-row gradient sums for the B rows in brows/by/bw
int run_backward(MlpState* m, int npairs, int B, const int32_t* rows, const float* y, const float* w,
                 cudaStream_t s) {
    CKM(cudaMemsetAsync(m->grad, 0, sizeof(float) * kNParams, s));
    CKM(cudaMemsetAsync(m->loss, 0, sizeof(float), s));
    int rc = run_forward<true>(m, npairs, B, rows, nullptr, m->s, s);
    if (rc) return rc;
    HeadParams hp;
    hp.nrows = B; hp.s = m->s; hp.y = y; hp.w = w; hp.h2 = m->h2; hp.w3 = m->theta + kOffW3;
    hp.dz2 = m->dz2; hp.g_w3 = m->grad + kOffW3; hp.g_b2 = m->grad + kOffB2; hp.g_b3 = m->grad + kOffB3;
    hp.loss = m->loss;
    const int rpb = 64;
    bwd_head_kernel<<<(B + rpb - 1) / rpb, kH, 0, s>>>(hp, rpb);
    CKM(cudaGetLastError());
    // dz1 = (dz2 W2^T) * relu'(z1):  M = B, N = 128 (in), K = 128 (out)
    {
        RowPairA A{m->dz2, kH};
        NKPairB Bm{m->W2h, kH};
        StoreDz1 C{m->dz1, m->h1};
        dim3 grid((B + 15) / 16, kH / 64, 1);
        gemm_kernel<<<grid, 32, 0, s>>>(B, kH, kH, kH, A, Bm, C);
        CKM(cudaGetLastError());
    }
    // g_W2[in][out] = h1^T dz2:  M = 128, N = 128, K = B (split over K)
    const int kchunk = 256;
    {
        TransA A{m->h1, kH};
        KNPairB Bm{m->dz2, kH};
        AtomicAddC C{m->grad + kOffW2, kH};
        dim3 grid(kH / 16, kH / 64, (B + kchunk - 1) / kchunk);
        gemm_kernel<<<grid, 32, 0, s>>>(kH, kH, B, kchunk, A, Bm, C);
        CKM(cudaGetLastError());
    }
    // g_W1[in][out] = x^T dz1:  M = 48, N = 128, K = B
    {
        InputTA A{rows, m->feat16, npairs};
        KNPairB Bm{m->dz1, kH};
        AtomicAddC C{m->grad + kOffW1, kH};
        dim3 grid(kIn / 16, kH / 64, (B + kchunk - 1) / kchunk);
        gemm_kernel<<<grid, 32, 0, s>>>(kIn, kH, B, kchunk, A, Bm, C);
        CKM(cudaGetLastError());
    }
    colsum_kernel<<<128, kH, 0, s>>>(m->dz1, B, m->grad + kOffB1);
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
    if ((rc = run_forward<false>(m, npairs, (long long)npairs * 4096, nullptr, d_n, m->S, s))) return rc;
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
                  m->feat32, m->S, m->vscore, m->rank, m->h1, m->h2, m->dz2, m->dz1, m->s,
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
            if ((rc = run_backward(m, npairs, nrows, d_rows, d_y, d_w, s))) return rc;
        } else {
            if ((rc = run_forward<false>(m, npairs, nrows, d_rows, d_n, m->s, s))) return rc;
        }
        if (h_scores) CKM(cudaMemcpyAsync(h_scores, m->s, sizeof(float) * nrows, cudaMemcpyDeviceToHost, s));
        if (h_grad) CKM(cudaMemcpyAsync(h_grad, m->grad, sizeof(float) * kNParams, cudaMemcpyDeviceToHost, s));
        if (h_loss) CKM(cudaMemcpyAsync(h_loss, m->loss, sizeof(float), cudaMemcpyDeviceToHost, s));
    }
    CKM(cudaStreamSynchronize(s));
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
        if ((rc = run_backward(m, npairs, batch, m->brows, m->by, m->bw, s))) break;
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
    return rc;
}

}  // extern "C"
