// jatam_mlp.cu -- the surrogate network 36 -> 256 -> 256 -> 8 (ReLU, softmax
// cross-entropy) on bfloat16 tensor cores with float32 accumulation: forward,
// backward and Adam for training, forward for inference.
//
// Every matrix product of the network -- forward and the three weight and two
// activation gradients of the backward pass -- is one call of a tile GEMM
// C[M x N] = A[M x K] B[K x N] whose operands are bfloat16 with arbitrary row
// and column strides (so transposes cost nothing) and whose epilogue is fused:
// bias + ReLU to bfloat16 (hidden layers), bias to float32 (logits), a ReLU
// derivative mask to bfloat16 (activation gradients), or plain float32
// (weight gradients).  The product itself is mma.sync.m16n8k16 (bf16 x bf16 ->
// f32) from shared-memory tiles, except the products with 256 output columns
// (both hidden layers and the first layer's activation gradient), which run on
// tcgen05 with the accumulator in tensor memory (jatam_tc.cu).  The weight gradients (K = the batch, only a
// few output tiles) split K over the grid's z dimension into float32 partial
// products that a second kernel sums in split order, so the bits do not
// depend on scheduling.
#include <cstdint>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "jatam_internal.cuh"

namespace jatam {
namespace {

constexpr int TM = 64, TN = 64, TK = 16;  // CTA tile; 4 warps of 32 x 32
constexpr int KP = TK + 8;                // padded row (halfs) of the shared tiles

enum Epi : int { EPI_F32 = 0, EPI_BIAS_F32 = 1, EPI_BIAS_RELU_BF16 = 2, EPI_MASK_BF16 = 3 };

struct GemmArgs {
    const __nv_bfloat16 *A;
    long long a_m, a_k;  // element (m, k) at A[m * a_m + k * a_k]
    const __nv_bfloat16 *B;
    long long b_k, b_n;  // element (k, n) at B[k * b_k + n * b_n]
    int M, N, K;
    int epi;
    const float *bias;             // [N] for the bias epilogues
    const __nv_bfloat16 *mask;     // [M x N] row-major: keep where mask > 0 (EPI_MASK_BF16)
    float *Cf;                     // [M x N] row-major float32 output
    __nv_bfloat16 *Cb;             // [M x N] row-major bfloat16 output
    int kchunk;                    // split-K: CTA z covers k in [z kchunk, (z + 1) kchunk); 0: all of K
    const __nv_bfloat16 *Bt;       // the same B with K contiguous (element (k, n) at Bt[n * K + k]), or null
    int bias_row;                  // weight gradients: also the column sums of B, as row M of C (the bias
                                   // gradient, stored right after the weights)
};

__device__ __forceinline__ void mma_bf16(float (&c)[4], const uint32_t (&a)[4], const uint32_t (&b)[2])
{
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0, %1, %2, %3}, {%4, %5, %6, %7}, {%8, %9}, "
        "{%0, %1, %2, %3};\n"
        : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

__global__ void __launch_bounds__(128) gemm_bf16_kernel(const GemmArgs g)
{
    __shared__ __align__(16) __nv_bfloat16 As[TM][KP];  // [m][k]
    __shared__ __align__(16) __nv_bfloat16 Bs[TN][KP];  // [n][k]
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int m0 = blockIdx.y * TM, n0 = blockIdx.x * TN;
    const int wm = (warp >> 1) * 32, wn = (warp & 1) * 32;  // warp's 32 x 32 sub-tile
    const int gq = lane >> 2, tq = lane & 3;
    float acc[2][4][4];
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j)
#pragma unroll
            for (int r = 0; r < 4; ++r) acc[i][j][r] = 0.f;
    const __nv_bfloat16 zero = __float2bfloat16(0.f);
    const int kbeg = g.kchunk ? (int)blockIdx.z * g.kchunk : 0;
    const int kend = g.kchunk ? min(g.K, kbeg + g.kchunk) : g.K;
    for (int k0 = kbeg; k0 < kend; k0 += TK) {
        // stage the A and B tiles (zero outside the matrices)
        for (int e = tid; e < TM * TK; e += blockDim.x) {
            const int m = e / TK, k = e % TK;
            const int gm = m0 + m, gk = k0 + k;
            As[m][k] = (gm < g.M && gk < kend) ? g.A[gm * g.a_m + gk * g.a_k] : zero;
        }
        for (int e = tid; e < TN * TK; e += blockDim.x) {
            const int n = e / TK, k = e % TK;
            const int gn = n0 + n, gk = k0 + k;
            Bs[n][k] = (gn < g.N && gk < kend) ? g.B[gk * g.b_k + gn * g.b_n] : zero;
        }
        __syncthreads();
        uint32_t af[2][4], bf[4][2];
#pragma unroll
        for (int i = 0; i < 2; ++i) {
            const int r = wm + 16 * i + gq;
            af[i][0] = *reinterpret_cast<const uint32_t *>(&As[r][2 * tq]);
            af[i][1] = *reinterpret_cast<const uint32_t *>(&As[r + 8][2 * tq]);
            af[i][2] = *reinterpret_cast<const uint32_t *>(&As[r][2 * tq + 8]);
            af[i][3] = *reinterpret_cast<const uint32_t *>(&As[r + 8][2 * tq + 8]);
        }
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int cidx = wn + 8 * j + gq;
            bf[j][0] = *reinterpret_cast<const uint32_t *>(&Bs[cidx][2 * tq]);
            bf[j][1] = *reinterpret_cast<const uint32_t *>(&Bs[cidx][2 * tq + 8]);
        }
#pragma unroll
        for (int i = 0; i < 2; ++i)
#pragma unroll
            for (int j = 0; j < 4; ++j) mma_bf16(acc[i][j], af[i], bf[j]);
        __syncthreads();
    }
    // epilogue: accumulator element r sits at row gq (+8 for r >= 2), column 2 tq + (r & 1)
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j)
#pragma unroll
            for (int r = 0; r < 4; ++r) {
                const int m = m0 + wm + 16 * i + gq + (r >= 2 ? 8 : 0);
                const int n = n0 + wn + 8 * j + 2 * tq + (r & 1);
                if (m >= g.M || n >= g.N) continue;
                float v = acc[i][j][r];
                const long long o = (long long)m * g.N + n;
                switch (g.epi) {
                case EPI_F32: g.Cf[(long long)blockIdx.z * g.M * g.N + o] = v; break;
                case EPI_BIAS_F32: g.Cf[o] = v + g.bias[n]; break;
                case EPI_BIAS_RELU_BF16: g.Cb[o] = __float2bfloat16_rn(fmaxf(v + g.bias[n], 0.f)); break;
                default: g.Cb[o] = __float2bfloat16_rn(__bfloat162float(g.mask[o]) > 0.f ? v : 0.f); break;
                }
            }
}

// Weight gradients C[M x N] = A^T B with A [K x M] and B [K x N] both stored row by row
// (K = the batch, M and N multiples of 8, rows 16-byte aligned): 64 x 64 output tiles of 4
// warps, K in steps of 32 through two shared-memory stages that cp.async fills as the rows
// lie in memory ([k][m] and [k][n]); ldmatrix.trans turns them into the m16n8k16 fragments.
// Split K over blockIdx.z as the general kernel does (float32 partial products, summed in
// split order afterwards).
constexpr int WG_KT = 32, WG_PAD = 72;  // k rows a stage; row length in halfs (64 + 8: 16-byte rows, no conflicts)

__device__ __forceinline__ void wg_cp16(uint32_t dst, const void *src, uint32_t bytes)
{
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(dst), "l"(src), "r"(bytes) : "memory");
}

__device__ __forceinline__ void ldsm_x4_trans(uint32_t (&r)[4], uint32_t addr)
{
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0, %1, %2, %3}, [%4];\n"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
                 : "r"(addr));
}

__global__ void __launch_bounds__(128) wgrad_kernel(const __nv_bfloat16 *A, long long lda, const __nv_bfloat16 *B,
                                                    long long ldb, int M, int N, int K, int kchunk, float *C,
                                                    int bias_row)
{
    __shared__ __align__(16) __nv_bfloat16 As[2][WG_KT][WG_PAD];  // [stage][k][m]
    __shared__ __align__(16) __nv_bfloat16 Bs[2][WG_KT][WG_PAD];  // [stage][k][n]
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int m0 = blockIdx.y * 64, n0 = blockIdx.x * 64;
    const int wm = (warp >> 1) * 32, wn = (warp & 1) * 32;
    const int kbeg = (int)blockIdx.z * kchunk, kend = min(K, kbeg + kchunk);
    const int nsteps = kend > kbeg ? (kend - kbeg + WG_KT - 1) / WG_KT : 0;
    auto fill = [&](int st, int step) {
        const int k0 = kbeg + step * WG_KT;
        // 32 rows x 8 pieces of 16 bytes for each operand: 2 + 2 pieces a thread
        for (int e = tid; e < WG_KT * 8; e += 128) {
            const int r = e >> 3, pc = (e & 7) * 8;
            const int gk = k0 + r;
            const bool ka = gk < kend;
            const bool ina = ka && m0 + pc < M, inb = ka && n0 + pc < N;
            wg_cp16((uint32_t)__cvta_generic_to_shared(&As[st][r][pc]), A + (ina ? (long long)gk * lda + m0 + pc : 0),
                    ina ? 16u : 0u);
            wg_cp16((uint32_t)__cvta_generic_to_shared(&Bs[st][r][pc]), B + (inb ? (long long)gk * ldb + n0 + pc : 0),
                    inb ? 16u : 0u);
        }
        asm volatile("cp.async.commit_group;\n" ::: "memory");
    };
    float acc[2][4][4];
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j)
#pragma unroll
            for (int r = 0; r < 4; ++r) acc[i][j][r] = 0.f;
    // bias_row: the CTAs of the first row of tiles also sum B's columns over their K range (in k order)
    const bool colsum = bias_row && blockIdx.y == 0 && tid < 64;
    float bsum = 0.f;
    if (nsteps > 0) fill(0, 0);
    for (int step = 0; step < nsteps; ++step) {
        const int st = step & 1;
        if (step + 1 < nsteps) {
            fill(st ^ 1, step + 1);
            asm volatile("cp.async.wait_group 1;\n" ::: "memory");
        } else {
            asm volatile("cp.async.wait_group 0;\n" ::: "memory");
        }
        __syncthreads();
        if (colsum) {
#pragma unroll 8
            for (int r = 0; r < WG_KT; ++r) bsum += __bfloat162float(Bs[st][r][tid]);
        }
#pragma unroll
        for (int kk = 0; kk < WG_KT; kk += 16) {
            // ldmatrix: lanes 8 j .. 8 j + 7 give the rows of 8 x 8 block j
            const int j = lane >> 3, rr = lane & 7;
            uint32_t af[2][4], bfr[2][4];
#pragma unroll
            for (int i = 0; i < 2; ++i) {
                // A fragment of rows m = wm + 16 i ..: blocks (k 0-7, m 0-7), (k 0-7, m 8-15), (k 8-15, m 0-7), (k 8-15, m 8-15)
                const int kr = kk + ((j >> 1) << 3) + rr, mc = wm + 16 * i + ((j & 1) << 3);
                ldsm_x4_trans(af[i], (uint32_t)__cvta_generic_to_shared(&As[st][kr][mc]));
            }
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                // B fragments of columns n = wn + 16 h ..: blocks (k 0-7, n 0-7), (k 8-15, n 0-7), (k 0-7, n 8-15), (k 8-15, n 8-15)
                const int kr = kk + ((j & 1) << 3) + rr, nc = wn + 16 * h + ((j >> 1) << 3);
                ldsm_x4_trans(bfr[h], (uint32_t)__cvta_generic_to_shared(&Bs[st][kr][nc]));
            }
#pragma unroll
            for (int i = 0; i < 2; ++i)
#pragma unroll
                for (int jn = 0; jn < 4; ++jn) {
                    const uint32_t b2[2] = {bfr[jn >> 1][2 * (jn & 1)], bfr[jn >> 1][2 * (jn & 1) + 1]};
                    mma_bf16(acc[i][jn], af[i], b2);
                }
        }
        __syncthreads();
    }
    const int gq = lane >> 2, tq = lane & 3;
    float *out = C + (long long)blockIdx.z * (M + bias_row) * N;
    if (colsum && n0 + tid < N) out[(long long)M * N + n0 + tid] = bsum;
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int jn = 0; jn < 4; ++jn)
#pragma unroll
            for (int r = 0; r < 4; ++r) {
                const int m = m0 + wm + 16 * i + gq + (r >= 2 ? 8 : 0);
                const int n = n0 + wn + 8 * jn + 2 * tq + (r & 1);
                if (m < M && n < N) out[(long long)m * N + n] = acc[i][jn][r];
            }
}

// features: bit (35 - j) of the genome for j < 36, zero for 36..47 (bfloat16 1.0 is 0x3F80); a
// thread per row, the row's 96 bytes in six 16-byte stores
__global__ void features_kernel(const unsigned long long *genomes, long long n, __nv_bfloat16 *x)
{
    for (long long r = blockIdx.x * (long long)blockDim.x + threadIdx.x; r < n; r += (long long)gridDim.x * blockDim.x) {
        const unsigned long long g = genomes[r];
        uint4 *dst = reinterpret_cast<uint4 *>(x + r * MLP_PAD);
#pragma unroll
        for (int q = 0; q < MLP_PAD / 8; ++q) {
            uint32_t w[4];
#pragma unroll
            for (int h = 0; h < 4; ++h) {
                const int j0 = 8 * q + 2 * h, j1 = j0 + 1;
                const uint32_t lo = (j0 < MLP_IN && ((g >> (MLP_IN - 1 - j0)) & 1ull)) ? 0x3F80u : 0u;
                const uint32_t hi = (j1 < MLP_IN && ((g >> (MLP_IN - 1 - j1)) & 1ull)) ? 0x3F80u : 0u;
                w[h] = lo | (hi << 16);
            }
            dst[q] = make_uint4(w[0], w[1], w[2], w[3]);
        }
    }
}

// softmax cross-entropy on float32 logits: d = (softmax - onehot) / B, as
// float32 and bfloat16 (for the products); per block of 256 rows, in a fixed
// order, the sum of the rows' losses (each divided by B) and of d's 8 columns
// (the output bias gradient) into part[9 block ..]
__global__ void __launch_bounds__(256) softmax_ce_kernel(const float *logits, const uint8_t *labels, long long B,
                                                         float *d, __nv_bfloat16 *dq, float *part)
{
    __shared__ float red[9][256];
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    float l = 0.f, dv[MLP_OUT];
#pragma unroll
    for (int c = 0; c < MLP_OUT; ++c) dv[c] = 0.f;
    if (i < B) {
        const float *z = logits + i * MLP_OUT;
        float mx = z[0];
        for (int c = 1; c < MLP_OUT; ++c) mx = fmaxf(mx, z[c]);
        float e[MLP_OUT], s = 0.f;
        for (int c = 0; c < MLP_OUT; ++c) {
            e[c] = expf(z[c] - mx);
            s += e[c];
        }
        const int y = labels[i];
#pragma unroll
        for (int c = 0; c < MLP_OUT; ++c) {
            const float v = (e[c] / s - (c == y ? 1.f : 0.f)) / (float)B;
            d[i * MLP_OUT + c] = v;
            dq[i * MLP_OUT + c] = __float2bfloat16_rn(v);
            dv[c] = v;
        }
        l = (logf(s) + mx - z[y]) / (float)B;
    }
    red[0][threadIdx.x] = l;
#pragma unroll
    for (int c = 0; c < MLP_OUT; ++c) red[1 + c][threadIdx.x] = dv[c];
    __syncthreads();
    for (int off = blockDim.x / 2; off > 0; off >>= 1) {
        if ((int)threadIdx.x < off) {
#pragma unroll
            for (int v = 0; v < 9; ++v) red[v][threadIdx.x] += red[v][threadIdx.x + off];
        }
        __syncthreads();
    }
    if (threadIdx.x < 9) part[9 * (long long)blockIdx.x + threadIdx.x] = red[threadIdx.x][0];
}

// the loss and the output bias gradient: the blocks' partial sums added in a fixed order
__global__ void __launch_bounds__(256) ce_sum_kernel(const float *part, long long blocks, float *loss, float *db3)
{
    __shared__ float red[9][256];
    float acc[9];
#pragma unroll
    for (int v = 0; v < 9; ++v) acc[v] = 0.f;
    for (long long b = threadIdx.x; b < blocks; b += blockDim.x) {
#pragma unroll
        for (int v = 0; v < 9; ++v) acc[v] += part[9 * b + v];
    }
#pragma unroll
    for (int v = 0; v < 9; ++v) red[v][threadIdx.x] = acc[v];
    __syncthreads();
    for (int off = blockDim.x / 2; off > 0; off >>= 1) {
        if ((int)threadIdx.x < off) {
#pragma unroll
            for (int v = 0; v < 9; ++v) red[v][threadIdx.x] += red[v][threadIdx.x + off];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) *loss = red[0][0];
    if (threadIdx.x >= 1 && threadIdx.x < 9) db3[threadIdx.x - 1] = red[threadIdx.x][0];
}

// dh2 = (dq W3^T) * [h2 > 0]: a warp per row, 8 columns a lane; each output the float32 sum of its
// 8 products in k order (products of two bfloat16 values are exact), then rounded to bfloat16
__global__ void __launch_bounds__(256) dh2_kernel(const __nv_bfloat16 *dq, const __nv_bfloat16 *w3,
                                                  const __nv_bfloat16 *h2, long long B, __nv_bfloat16 *dh2)
{
    __shared__ float w[MLP_H][MLP_OUT];  // W3[n][k]
    for (int i = threadIdx.x; i < MLP_H * MLP_OUT; i += blockDim.x) w[i / MLP_OUT][i % MLP_OUT] = __bfloat162float(w3[i]);
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (long long row = (long long)blockIdx.x * 8 + warp; row < B; row += (long long)gridDim.x * 8) {
        const uint4 qv = *reinterpret_cast<const uint4 *>(dq + row * MLP_OUT);
        const uint32_t qw[4] = {qv.x, qv.y, qv.z, qv.w};
        float q[MLP_OUT];
#pragma unroll
        for (int k = 0; k < MLP_OUT; ++k)
            q[k] = __uint_as_float(k & 1 ? (qw[k >> 1] & 0xFFFF0000u) : (qw[k >> 1] << 16));
        const uint4 mv = *reinterpret_cast<const uint4 *>(h2 + row * MLP_H + 8 * lane);
        const uint32_t mw[4] = {mv.x, mv.y, mv.z, mv.w};
        uint32_t ow[4];
#pragma unroll
        for (int h = 0; h < 4; ++h) {
            float v[2];
#pragma unroll
            for (int e = 0; e < 2; ++e) {
                const int n = 8 * lane + 2 * h + e;
                float acc = 0.f;
#pragma unroll
                for (int k = 0; k < MLP_OUT; ++k) acc = fmaf(q[k], w[n][k], acc);
                const float m = __uint_as_float(e ? (mw[h] & 0xFFFF0000u) : (mw[h] << 16));
                v[e] = m > 0.f ? acc : 0.f;
            }
            const __nv_bfloat162 hv = __floats2bfloat162_rn(v[0], v[1]);
            ow[h] = *reinterpret_cast<const uint32_t *>(&hv);
        }
        *reinterpret_cast<uint4 *>(dh2 + row * MLP_H + 8 * lane) = make_uint4(ow[0], ow[1], ow[2], ow[3]);
    }
}

// column sums of a [B x N] matrix (float32 or bfloat16) into out[N]
template <typename T>
__global__ void colsum_kernel(const T *a, long long B, int N, float *out)
{
    const int n = blockIdx.x;
    float s = 0.f;
    for (long long r = threadIdx.x; r < B; r += blockDim.x) s += (float)a[r * N + n];
    __shared__ float red[256];
    red[threadIdx.x] = s;
    __syncthreads();
    for (int off = blockDim.x / 2; off > 0; off >>= 1) {
        if ((int)threadIdx.x < off) red[threadIdx.x] += red[threadIdx.x + off];
        __syncthreads();
    }
    if (threadIdx.x == 0) out[n] = red[0];
}

template <>
__global__ void colsum_kernel<__nv_bfloat16>(const __nv_bfloat16 *a, long long B, int N, float *out)
{
    const int n = blockIdx.x;
    float s = 0.f;
    for (long long r = threadIdx.x; r < B; r += blockDim.x) s += __bfloat162float(a[r * N + n]);
    __shared__ float red[256];
    red[threadIdx.x] = s;
    __syncthreads();
    for (int off = blockDim.x / 2; off > 0; off >>= 1) {
        if ((int)threadIdx.x < off) red[threadIdx.x] += red[threadIdx.x + off];
        __syncthreads();
    }
    if (threadIdx.x == 0) out[n] = red[0];
}

// Adam on the float32 master parameters, then their bfloat16 copies
// the K-contiguous copies of W1 and W2 that the tcgen05 products read as their
// B operand: W1T [256 x 48] (W1T[n][k] = W1[k][n]) then W2T [256 x 256]
__device__ __forceinline__ void store_transposed(__nv_bfloat16 *pqt, long long i, __nv_bfloat16 v)
{
    if (i < MLP_PAD * MLP_H) {
        const long long k = i / MLP_H, n = i % MLP_H;
        pqt[n * MLP_PAD + k] = v;
    } else if (i >= MLP_PAD * MLP_H + MLP_H && i < MLP_PAD * MLP_H + MLP_H + MLP_H * MLP_H) {
        const long long j = i - (MLP_PAD * MLP_H + MLP_H);
        const long long k = j / MLP_H, n = j % MLP_H;
        pqt[MLP_PAD * MLP_H + n * MLP_H + k] = v;
    }
}

__global__ void adam_kernel(float *p, const float *g, float *m, float *v, long long n, float lr, float b1, float b2,
                            float eps, float c1, float c2, __nv_bfloat16 *pq, __nv_bfloat16 *pqt)
{
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const float gi = g[i];
        const float mi = b1 * m[i] + (1.f - b1) * gi;
        const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
        m[i] = mi;
        v[i] = vi;
        const float pi = p[i] - lr * (mi / c1) / (sqrtf(vi / c2) + eps);
        p[i] = pi;
        pq[i] = __float2bfloat16_rn(pi);
        if (pqt) store_transposed(pqt, i, pq[i]);
    }
}

__global__ void to_bf16_kernel(const float *p, long long n, __nv_bfloat16 *pq, __nv_bfloat16 *pqt)
{
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        pq[i] = __float2bfloat16_rn(p[i]);
        if (pqt) store_transposed(pqt, i, pq[i]);
    }
}

// out[i] = sum over z of part[z][i], z in increasing order
__global__ void splitk_sum_kernel(const float *part, int splits, long long n, float *out)
{
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        float s = 0.f;
        for (int z = 0; z < splits; ++z) s += part[(long long)z * n + i];
        out[i] = s;
    }
}

// the weight-gradient kernel's shapes: A^T B with both operands stored row by row over k
bool wgrad_ok(const GemmArgs &g, const float *splitk)
{
    return splitk && g.epi == EPI_F32 && g.a_m == 1 && g.b_n == 1 && g.M % 8 == 0 && g.N % 8 == 0 && g.a_k % 8 == 0 &&
           g.b_k % 8 == 0 && ((uintptr_t)g.A & 15) == 0 && ((uintptr_t)g.B & 15) == 0;
}

cudaError_t gemm(const GemmArgs &g, cudaStream_t st, float *splitk = nullptr, const MlpBuffers *tcb = nullptr)
{
    // the products with 256 output columns and K a multiple of 16 on tcgen05
    // (K-contiguous operands with 16-byte aligned rows, K <= 256)
    const bool bt = g.Bt != nullptr;
    const long long bn = bt ? g.K : g.b_n;
    const bool k_major = g.a_k == 1 && (bt || g.b_k == 1) && g.a_m % 8 == 0 && bn % 8 == 0 && g.K <= 256;
    if (tcb && tcb->tc && k_major && g.N == 256 && g.M >= 128 && g.K % 16 == 0 &&
        (g.epi == EPI_BIAS_RELU_BF16 || g.epi == EPI_MASK_BF16)) {
        return tc_gemm_n256(g.A, g.a_m, g.a_k, bt ? g.Bt : g.B, bt ? 1 : g.b_k, bt ? g.K : g.b_n, g.M, g.K,
                            g.epi == EPI_BIAS_RELU_BF16 ? 0 : 1, g.bias, g.mask, g.Cb, tcb->tc_err, st);
    }
    const dim3 tiles((g.N + TN - 1) / TN, (g.M + TM - 1) / TM);
    const int ntiles = (int)(tiles.x * tiles.y);
    // weight gradients (A^T B, both stored row by row over k): the cp.async / ldmatrix kernel
    if (wgrad_ok(g, splitk)) {
        int splits = (g.K + 8 * 32 - 1) / (8 * 32);  // at least 8 k-steps of 32 a split
        splits = min(splits, min(MLP_SPLITK_MAX, (304 + ntiles - 1) / ntiles));
        if (splits < 1) splits = 1;
        int kchunk = ((g.K + splits - 1) / splits + WG_KT - 1) / WG_KT * WG_KT;
        splits = (g.K + kchunk - 1) / kchunk;
        float *dst = splits > 1 ? splitk : g.Cf;
        wgrad_kernel<<<dim3(tiles.x, tiles.y, splits), 128, 0, st>>>(g.A, g.a_k, g.B, g.b_k, g.M, g.N, g.K, kchunk, dst,
                                                                   g.bias_row ? 1 : 0);
        if (splits > 1) {
            const long long n = (long long)(g.M + (g.bias_row ? 1 : 0)) * g.N;
            splitk_sum_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(splitk, splits, n, g.Cf);
        }
        return cudaGetLastError();
    }
    // a float32 product with few output tiles and a long K: split K over the grid
    int splits = 1;
    if (splitk && g.epi == EPI_F32 && ntiles < 64) {
        splits = (g.K + 8 * TK - 1) / (8 * TK);                        // at least 8 k-tiles a split
        splits = min(splits, min(MLP_SPLITK_MAX, (304 + ntiles - 1) / ntiles));  // about two CTAs per SM
    }
    if (splits <= 1) {
        GemmArgs h = g;
        h.kchunk = 0;
        gemm_bf16_kernel<<<tiles, 128, 0, st>>>(h);
        return cudaGetLastError();
    }
    GemmArgs h = g;
    h.kchunk = ((g.K + splits - 1) / splits + TK - 1) / TK * TK;
    splits = (g.K + h.kchunk - 1) / h.kchunk;
    h.Cf = splitk;
    gemm_bf16_kernel<<<dim3(tiles.x, tiles.y, splits), 128, 0, st>>>(h);
    const long long n = (long long)g.M * g.N;
    splitk_sum_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(splitk, splits, n, g.Cf);
    return cudaGetLastError();
}

unsigned grid_for(long long n) { return (unsigned)((n + 255) / 256 < 4096 ? (n + 255) / 256 : 4096); }

}  // namespace

// offsets of the six parameter tensors in the flat parameter vector
const long long MLP_OFF_W1 = 0;
const long long MLP_OFF_B1 = MLP_OFF_W1 + (long long)MLP_PAD * MLP_H;
const long long MLP_OFF_W2 = MLP_OFF_B1 + MLP_H;
const long long MLP_OFF_B2 = MLP_OFF_W2 + (long long)MLP_H * MLP_H;
const long long MLP_OFF_W3 = MLP_OFF_B2 + MLP_H;
const long long MLP_OFF_B3 = MLP_OFF_W3 + (long long)MLP_H * MLP_OUT;
const long long MLP_NPARAM = MLP_OFF_B3 + MLP_OUT;

cudaError_t mlp_forward(const MlpBuffers &b, const unsigned long long *genomes, long long B, cudaStream_t st,
                        bool logits_only)
{
    features_kernel<<<grid_for(B), 256, 0, st>>>(genomes, B, b.x);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const __nv_bfloat16 *Wq = b.wq;
    GemmArgs g{};
    // h1 = relu(x W1 + b1)
    g = GemmArgs{b.x, MLP_PAD, 1, Wq + MLP_OFF_W1, MLP_H, 1, (int)B, MLP_H, MLP_PAD, EPI_BIAS_RELU_BF16,
                 b.p + MLP_OFF_B1, nullptr, nullptr, b.h1, 0, b.wqt};
    if ((e = gemm(g, st, nullptr, &b)) != cudaSuccess) return e;
    if (logits_only && b.tc) {
        // logits = bf16(relu(h1 W2 + b2)) W3 + b3 in the epilogue of the second layer's product
        return tc_gemm_n256(b.h1, MLP_H, 1, b.wqt + MLP_PAD * MLP_H, 1, MLP_H, (int)B, MLP_H, 2, b.p + MLP_OFF_B2,
                            nullptr, nullptr, b.tc_err, st, Wq + MLP_OFF_W3, b.p + MLP_OFF_B3, b.logits);
    }
    if (b.tc) {
        // h2 = relu(h1 W2 + b2), stored, and logits = h2 W3 + b3 in the same epilogue
        return tc_gemm_n256(b.h1, MLP_H, 1, b.wqt + MLP_PAD * MLP_H, 1, MLP_H, (int)B, MLP_H, 3, b.p + MLP_OFF_B2,
                            nullptr, b.h2, b.tc_err, st, Wq + MLP_OFF_W3, b.p + MLP_OFF_B3, b.logits);
    }
    // h2 = relu(h1 W2 + b2)
    g = GemmArgs{b.h1, MLP_H, 1, Wq + MLP_OFF_W2, MLP_H, 1, (int)B, MLP_H, MLP_H, EPI_BIAS_RELU_BF16,
                 b.p + MLP_OFF_B2, nullptr, nullptr, b.h2, 0, b.wqt + MLP_PAD * MLP_H};
    if ((e = gemm(g, st, nullptr, &b)) != cudaSuccess) return e;
    // logits = h2 W3 + b3 (every product on mma.sync)
    g = GemmArgs{b.h2, MLP_H, 1, Wq + MLP_OFF_W3, MLP_OUT, 1, (int)B, MLP_OUT, MLP_H, EPI_BIAS_F32,
                 b.p + MLP_OFF_B3, nullptr, b.logits, nullptr};
    return gemm(g, st);
}

cudaError_t mlp_backward(const MlpBuffers &b, const uint8_t *labels, long long B, cudaStream_t st)
{
    cudaError_t e;
    float *G = b.grad;
    // the loss and db3 from per-block partial sums (in lrow: 9 values a block of 256 rows)
    const long long ceb = (B + 255) / 256;
    softmax_ce_kernel<<<(unsigned)ceb, 256, 0, st>>>(b.logits, labels, B, b.d, b.dq, b.lrow);
    ce_sum_kernel<<<1, 256, 0, st>>>(b.lrow, ceb, b.loss, G + MLP_OFF_B3);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    GemmArgs g{};
    // dW3 = h2^T dq  [256 x 8], K = B
    g = GemmArgs{b.h2, 1, MLP_H, b.dq, MLP_OUT, 1, MLP_H, MLP_OUT, (int)B, EPI_F32, nullptr, nullptr,
                 G + MLP_OFF_W3, nullptr};
    if ((e = gemm(g, st, b.splitk)) != cudaSuccess) return e;
    // dh2 = (dq W3^T) * [h2 > 0]  [B x 256], K = 8 (on mma.sync when every product is kept there)
    if (b.tc) {
        const long long rb = (B + 7) / 8;
        dh2_kernel<<<(unsigned)(rb < 4096 ? rb : 4096), 256, 0, st>>>(b.dq, b.wq + MLP_OFF_W3, b.h2, B, b.dh2);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    } else {
        g = GemmArgs{b.dq, MLP_OUT, 1, b.wq + MLP_OFF_W3, 1, MLP_OUT, (int)B, MLP_H, MLP_OUT, EPI_MASK_BF16, nullptr,
                     b.h2, nullptr, b.dh2};
        if ((e = gemm(g, st)) != cudaSuccess) return e;
    }
    // dW2 = h1^T dh2  [256 x 256]
    g = GemmArgs{b.h1, 1, MLP_H, b.dh2, MLP_H, 1, MLP_H, MLP_H, (int)B, EPI_F32, nullptr, nullptr, G + MLP_OFF_W2,
                 nullptr};
    // db2 = column sums of dh2: row 256 of the same product (b2 follows W2 in the parameters)
    g.bias_row = wgrad_ok(g, b.splitk) ? 1 : 0;
    if ((e = gemm(g, st, b.splitk)) != cudaSuccess) return e;
    if (!g.bias_row) colsum_kernel<__nv_bfloat16><<<MLP_H, 256, 0, st>>>(b.dh2, B, MLP_H, G + MLP_OFF_B2);
    // dh1 = (dh2 W2^T) * [h1 > 0]  [B x 256]
    g = GemmArgs{b.dh2, MLP_H, 1, b.wq + MLP_OFF_W2, 1, MLP_H, (int)B, MLP_H, MLP_H, EPI_MASK_BF16, nullptr, b.h1,
                 nullptr, b.dh1};
    if ((e = gemm(g, st, nullptr, &b)) != cudaSuccess) return e;
    // dW1 = x^T dh1  [48 x 256]
    g = GemmArgs{b.x, 1, MLP_PAD, b.dh1, MLP_H, 1, MLP_PAD, MLP_H, (int)B, EPI_F32, nullptr, nullptr, G + MLP_OFF_W1,
                 nullptr};
    // db1 = column sums of dh1: row 48 of the same product (b1 follows W1 in the parameters)
    g.bias_row = wgrad_ok(g, b.splitk) ? 1 : 0;
    if ((e = gemm(g, st, b.splitk)) != cudaSuccess) return e;
    if (!g.bias_row) colsum_kernel<__nv_bfloat16><<<MLP_H, 256, 0, st>>>(b.dh1, B, MLP_H, G + MLP_OFF_B1);
    return cudaGetLastError();
}

cudaError_t mlp_adam(const MlpBuffers &b, float lr, int t, cudaStream_t st)
{
    const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
    const float c1 = 1.f - powf(b1, (float)t), c2 = 1.f - powf(b2, (float)t);
    adam_kernel<<<grid_for(MLP_NPARAM), 256, 0, st>>>(b.p, b.grad, b.m, b.v, MLP_NPARAM, lr, b1, b2, eps, c1, c2,
                                                       b.wq, b.wqt);
    return cudaGetLastError();
}

cudaError_t mlp_refresh_bf16(const MlpBuffers &b, cudaStream_t st)
{
    to_bf16_kernel<<<grid_for(MLP_NPARAM), 256, 0, st>>>(b.p, MLP_NPARAM, b.wq, b.wqt);
    return cudaGetLastError();
}

}  // namespace jatam

namespace jatam {
namespace {

// class label of a classification result (the network's 8 outputs)
__global__ void labels_kernel(const jatam_result *res, long long n, uint8_t *labels)
{
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const jatam_result r = res[i];
        uint8_t y;
        if (r.cls == JATAM_UNBOUNDED) y = 0;
        else if (r.cls == JATAM_ND_LOCAL) y = 1;
        else if (r.cls == JATAM_ND_STERIC) y = 2;
        else y = r.size >= 16 ? 7 : r.size >= 8 ? 6 : r.size >= 4 ? 5 : r.size >= 2 ? 4 : 3;
        labels[i] = y;
    }
}

// packed genomes of S_{n,c} -> S_{3,8} (tiles beyond n all-zero, colours kept)
__global__ void embed_kernel(const unsigned long long *in, long long count, int n, int b, unsigned long long *out)
{
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < count;
         i += (long long)gridDim.x * blockDim.x) {
        const unsigned long long g = in[i];
        unsigned long long o = 0;
        for (int t = 0; t < n; ++t)
            for (int e = 0; e < 4; ++e) {
                const unsigned long long colour = (g >> (b * (4 * (n - 1 - t) + (3 - e)))) & ((1ull << b) - 1ull);
                o |= colour << (3 * (4 * (3 - 1 - t) + (3 - e)));
            }
        out[i] = o;
    }
}

// expected shape size under the predicted class probabilities
__global__ void score_kernel(const float *logits, long long n, float *score)
{
    // probability of a deterministic bounded shape of at least 8 tiles (classes 6, 7)
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const float *z = logits + i * MLP_OUT;
        float mx = z[0];
        for (int c = 1; c < MLP_OUT; ++c) mx = fmaxf(mx, z[c]);
        float s = 0.f, e = 0.f;
        for (int c = 0; c < MLP_OUT; ++c) {
            const float p = expf(z[c] - mx);
            s += p;
            if (c >= 6) e += p;
        }
        score[i] = e / s;
    }
}

// ---------------------------------------------------------------------------
// Indices of the `keep` largest non-negative scores among n (ties: lower index first), in
// increasing index order, by a radix select on the float bits (monotone for non-negative
// floats), over many CTAs with a scratch area (TOPN_SCRATCH_BYTES): three
// histogram launches find the threshold key 12, 12 and 8 bits at a time (the last CTA of each
// launch to finish -- a fence and an atomic ticket, no waiting -- picks the digit from the summed
// histogram and clears it for the next); a counting launch gives every CTA its keys above and
// equal to the threshold (its last CTA turns them into output positions and tie ranks), and a
// writing launch emits each CTA's chosen indices in order.  A warp whose keys share one digit
// adds them with one atomic.  Scratch: hist[4096] | ctrl[16] | counts[2][TOPN_MAX_CTAS] (u64).
// ---------------------------------------------------------------------------
constexpr int TN_THREADS = 256;
constexpr int TN_HIST = 4096;
constexpr int TOPN_MAX_CTAS = 1024;

__device__ __forceinline__ void tn_level(int lvl, int &shift, unsigned &dmask, unsigned &pmask)
{
    shift = lvl == 0 ? 20 : lvl == 1 ? 8 : 0;
    dmask = lvl < 2 ? 4095u : 255u;
    pmask = lvl == 0 ? 0u : lvl == 1 ? 0xFFF00000u : 0xFFFFFF00u;
}

__global__ void __launch_bounds__(TN_THREADS) topn_hist_kernel(const uint32_t *key, long long n, long long keep,
                                                               int lvl, unsigned *scratch)
{
    __shared__ unsigned local[TN_HIST];
    __shared__ int last_s;
    unsigned *hist = scratch, *ctrl = scratch + TN_HIST;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    int shift;
    unsigned dmask, pmask;
    tn_level(lvl, shift, dmask, pmask);
    const unsigned prefix = lvl == 0 ? 0u : __ldcg(&ctrl[0]);
    const unsigned long long want = lvl == 0 ? (unsigned long long)keep : __ldcg(&ctrl[1]);
    for (int i = tid; i <= (int)dmask; i += TN_THREADS) local[i] = 0u;
    __syncthreads();
    for (long long base = (long long)blockIdx.x * TN_THREADS; base < n; base += (long long)gridDim.x * TN_THREADS) {
        const long long i = base + tid;
        const uint32_t k = i < n ? key[i] : 0u;
        const bool in = i < n && (k & pmask) == prefix;
        const unsigned d = (k >> shift) & dmask;
        const unsigned act = __ballot_sync(0xffffffffu, in);
        if (act) {
            const int f = __ffs(act) - 1;
            const unsigned d0 = __shfl_sync(0xffffffffu, d, f);
            if (__all_sync(0xffffffffu, !in || d == d0)) {
                if (lane == f) atomicAdd(&local[d0], (unsigned)__popc(act));
            } else if (in) {
                atomicAdd(&local[d], 1u);
            }
        }
    }
    __syncthreads();
    for (int i = tid; i <= (int)dmask; i += TN_THREADS)
        if (local[i]) atomicAdd(&hist[i], local[i]);
    __threadfence();
    __syncthreads();
    if (tid == 0) last_s = atomicAdd(&ctrl[2], 1u) == gridDim.x - 1;
    __syncthreads();
    if (!last_s) return;
    __threadfence();
    // the last CTA: the summed histogram into shared memory (the global one starts at zero again for
    // the next launch)
    for (int i = tid; i <= (int)dmask; i += TN_THREADS) {
        local[i] = __ldcg(&hist[i]);
        hist[i] = 0u;
    }
    __syncthreads();
    if (warp == 0) {
        // lane l holds bins per l .. per l + per - 1; the crossing -- the highest digit d > 0 at which
        // the count from the top reaches `want`, else digit 0 -- lies in the lane whose bins take the
        // count from the top across `want`
        const int per = (int)(dmask + 1) / 32;
        unsigned sum = 0;
        for (int j = 0; j < per; ++j) sum += local[per * lane + j];
        unsigned incl = sum;  // keys in this lane's bins and above
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const unsigned v = __shfl_down_sync(0xffffffffu, incl, off);
            if (lane + off < 32) incl += v;
        }
        const unsigned above = incl - sum;
        const bool mine = (unsigned long long)above < want && (unsigned long long)incl >= want;
        if (mine) {
            unsigned long long acc = above;
            int dsel = 0;
            for (int j = per - 1; j >= 0; --j) {
                const int d = per * lane + j;
                if (d == 0) break;
                const unsigned h = local[d];
                if (acc + h >= want) {
                    dsel = d;
                    break;
                }
                acc += h;
            }
            ctrl[0] = prefix | ((unsigned)dsel << shift);
            ctrl[1] = (unsigned)(want - acc);
        }
    }
    if (tid == 0) ctrl[2] = 0u;  // the ticket, for the next launch
}

// a warp's keys in [lo, hi): counts above and equal to thr, eight chunks of 32 at a time
__device__ __forceinline__ void tn_warp_count(const uint32_t *key, long long lo, long long hi, uint32_t thr, int lane,
                                              unsigned long long &above, unsigned long long &equal)
{
    above = 0;
    equal = 0;
    for (long long c0 = lo; c0 < hi; c0 += 32 * 8) {
        uint32_t kk[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const long long i = c0 + 32 * u + lane;
            kk[u] = i < hi ? key[i] : 0u;
        }
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const long long i = c0 + 32 * u + lane;
            above += __popc(__ballot_sync(0xffffffffu, i < hi && kk[u] > thr));
            equal += __popc(__ballot_sync(0xffffffffu, i < hi && kk[u] == thr));
        }
    }
}

__global__ void __launch_bounds__(TN_THREADS) topn_count_kernel(const uint32_t *key, long long n, long long seg,
                                                                unsigned *scratch)
{
    __shared__ unsigned long long wa[TN_THREADS / 32], we[TN_THREADS / 32];
    __shared__ int last_s;
    unsigned *ctrl = scratch + TN_HIST;
    unsigned long long *counts = reinterpret_cast<unsigned long long *>(scratch + TN_HIST + 16);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const uint32_t thr = __ldcg(&ctrl[0]);
    const unsigned long long want = __ldcg(&ctrl[1]);
    const long long wseg = seg / (TN_THREADS / 32);
    const long long lo = (long long)blockIdx.x * seg + warp * wseg, hi = min(n, lo + wseg);
    unsigned long long above, equal;
    tn_warp_count(key, lo, hi, thr, lane, above, equal);
    if (lane == 0) {
        wa[warp] = above;
        we[warp] = equal;
    }
    __syncthreads();
    if (tid == 0) {
        unsigned long long a = 0, e = 0;
        for (int w = 0; w < TN_THREADS / 32; ++w) {
            a += wa[w];
            e += we[w];
        }
        counts[blockIdx.x] = a;
        counts[TOPN_MAX_CTAS + blockIdx.x] = e;
        __threadfence();
        last_s = atomicAdd(&ctrl[3], 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!last_s || warp != 0) return;
    __threadfence();
    // the last CTA: output position and equal keys before, per CTA, in CTA order -- exclusive scans
    // over 32 CTAs at a time (equal keys before, then above + the equal keys taken)
    unsigned long long eq = 0, pos = 0;
    for (unsigned b0 = 0; b0 < gridDim.x; b0 += 32) {
        const unsigned b = b0 + lane;
        const bool in = b < gridDim.x;
        const unsigned long long a = in ? __ldcg(&counts[b]) : 0ull, e = in ? __ldcg(&counts[TOPN_MAX_CTAS + b]) : 0ull;
        unsigned long long se = e;  // inclusive scan of e
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const unsigned long long v = __shfl_up_sync(0xffffffffu, se, off);
            if (lane >= off) se += v;
        }
        const unsigned long long eb = eq + se - e;  // equal keys before this CTA
        const unsigned long long take = eb >= want ? 0ull : min(e, want - eb);
        unsigned long long sp = a + take;  // inclusive scan of above + taken
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const unsigned long long v = __shfl_up_sync(0xffffffffu, sp, off);
            if (lane >= off) sp += v;
        }
        if (in) {
            counts[b] = pos + sp - (a + take);
            counts[TOPN_MAX_CTAS + b] = eb;
        }
        eq += __shfl_sync(0xffffffffu, se, 31);
        pos += __shfl_sync(0xffffffffu, sp, 31);
    }
    if (lane == 0) ctrl[3] = 0u;
}

__global__ void __launch_bounds__(TN_THREADS) topn_write_kernel(const uint32_t *key, long long n, long long seg,
                                                                const unsigned *scratch,
                                                                unsigned long long *idx_out)
{
    __shared__ unsigned long long wa[TN_THREADS / 32], we[TN_THREADS / 32];
    const unsigned *ctrl = scratch + TN_HIST;
    const unsigned long long *counts = reinterpret_cast<const unsigned long long *>(scratch + TN_HIST + 16);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const unsigned lt = (1u << lane) - 1u;
    const uint32_t thr = ctrl[0];
    const unsigned long long want = ctrl[1];
    const long long wseg = seg / (TN_THREADS / 32);
    const long long lo = (long long)blockIdx.x * seg + warp * wseg, hi = min(n, lo + wseg);
    unsigned long long above, equal;
    tn_warp_count(key, lo, hi, thr, lane, above, equal);
    if (lane == 0) {
        wa[warp] = above;
        we[warp] = equal;
    }
    __syncthreads();
    // this warp's output position and equal keys before it: the CTA's, then the warps before it
    unsigned long long pos = counts[blockIdx.x], r = counts[TOPN_MAX_CTAS + blockIdx.x];
    for (int w = 0; w < warp; ++w) {
        const unsigned long long take = r >= want ? 0ull : min(we[w], want - r);
        pos += wa[w] + take;
        r += we[w];
    }
    for (long long c0 = lo; c0 < hi; c0 += 32 * 8) {
        uint32_t kk[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const long long i = c0 + 32 * u + lane;
            kk[u] = i < hi ? key[i] : 0u;
        }
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const long long i = c0 + 32 * u + lane;
            const unsigned eqm = __ballot_sync(0xffffffffu, i < hi && kk[u] == thr);
            const bool take = (i < hi && kk[u] > thr) || ((eqm >> lane) & 1u && r + __popc(eqm & lt) < want);
            const unsigned selm = __ballot_sync(0xffffffffu, take);
            if (take) idx_out[pos + __popc(selm & lt)] = (unsigned long long)i;
            pos += __popc(selm);
            r += __popc(eqm);
        }
    }
}

__global__ void gather_kernel(const unsigned long long *src, const unsigned long long *idx, long long n,
                              unsigned long long *dst)
{
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        dst[i] = src[idx[i]];
}

unsigned grid_of(long long n) { return (unsigned)((n + 255) / 256 < 4096 ? (n + 255) / 256 : 4096); }

}  // namespace

cudaError_t launch_mlp_labels(const jatam_result *res, long long n, uint8_t *labels, cudaStream_t st)
{
    if (n) labels_kernel<<<grid_of(n), 256, 0, st>>>(res, n, labels);
    return cudaGetLastError();
}

cudaError_t launch_embed(const unsigned long long *in, long long n, int tiles, int bits_per_colour,
                         unsigned long long *out, cudaStream_t st)
{
    if (n) embed_kernel<<<grid_of(n), 256, 0, st>>>(in, n, tiles, bits_per_colour, out);
    return cudaGetLastError();
}

// Distinct candidates: an open-addressing table (capacity a power of two >= 2n,
// keys ~0 = empty) keeps the smallest index of each genome; slot[i] is the
// slot of candidate i.
__global__ void dedup_insert_kernel(const unsigned long long *cand, long long n, unsigned long long *keys,
                                    unsigned *first, unsigned cap_mask, unsigned *slot, unsigned *err)
{
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const unsigned long long g = cand[i];
        unsigned h = (unsigned)((g * 0x9E3779B97F4A7C15ull) >> 32) & cap_mask;
        bool done = false;
        for (unsigned p = 0; p <= cap_mask && !done; ++p) {
            const unsigned long long old = atomicCAS(&keys[h], ~0ull, g);
            if (old == ~0ull || old == g) {
                atomicMin(&first[h], (unsigned)i);
                slot[i] = h;
                done = true;
            } else {
                h = (h + 1) & cap_mask;
            }
        }
        if (!done) atomicOr(err, 1u);  // unreachable: the table holds at least 2n slots
    }
}

// the first occurrence of each genome scores one above every repeat
__global__ void dedup_mark_kernel(float *score, long long n, const unsigned *first, const unsigned *slot)
{
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        if (first[slot[i]] == (unsigned)i) score[i] += 1.f;
}

cudaError_t launch_topn_multi(const float *score, long long n, long long keep, unsigned long long *idx,
                              unsigned *scratch, cudaStream_t st)
{
    if (n <= 0 || keep <= 0) return cudaSuccess;
    const uint32_t *key = reinterpret_cast<const uint32_t *>(score);
    cudaError_t e = cudaMemsetAsync(scratch, 0, (TN_HIST + 16) * 4, st);
    if (e != cudaSuccess) return e;
    long long hb = (n + TN_THREADS * 2 - 1) / (TN_THREADS * 2);  // about 2 keys a thread
    if (hb > TOPN_MAX_CTAS) hb = TOPN_MAX_CTAS;
    for (int lvl = 0; lvl < 3; ++lvl)
        topn_hist_kernel<<<(unsigned)hb, TN_THREADS, 0, st>>>(key, n, keep, lvl, scratch);
    // segments of whole warp chunks: at least 512 keys a CTA, at most TOPN_MAX_CTAS CTAs
    long long cb = (n + 511) / 512;
    if (cb > TOPN_MAX_CTAS) cb = TOPN_MAX_CTAS;
    const long long unit = 32LL * (TN_THREADS / 32);
    const long long seg = ((n + cb - 1) / cb + unit - 1) / unit * unit;
    cb = (n + seg - 1) / seg;
    topn_count_kernel<<<(unsigned)cb, TN_THREADS, 0, st>>>(key, n, seg, scratch);
    topn_write_kernel<<<(unsigned)cb, TN_THREADS, 0, st>>>(key, n, seg, scratch, idx);
    return cudaGetLastError();
}


cudaError_t launch_screen(const float *logits, long long n, long long keep, float *score, unsigned long long *idx,
                          const unsigned long long *cand, unsigned long long *chosen, const ScreenTable &t,
                          cudaStream_t st)
{
    score_kernel<<<grid_of(n), 256, 0, st>>>(logits, n, score);
    cudaError_t e = cudaMemsetAsync(t.keys, 0xFF, (size_t)(t.cap_mask + 1) * 8, st);
    if (e != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(t.first, 0xFF, (size_t)(t.cap_mask + 1) * 4, st)) != cudaSuccess) return e;
    dedup_insert_kernel<<<grid_of(n), 256, 0, st>>>(cand, n, t.keys, t.first, t.cap_mask, t.slot, t.err);
    dedup_mark_kernel<<<grid_of(n), 256, 0, st>>>(score, n, t.first, t.slot);
    if ((e = launch_topn_multi(score, n, keep, idx, t.topn, st)) != cudaSuccess) return e;
    gather_kernel<<<grid_of(keep), 256, 0, st>>>(cand, idx, keep, chosen);
    return cudaGetLastError();
}

}  // namespace jatam
