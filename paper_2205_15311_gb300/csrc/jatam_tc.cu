// jatam_tc.cu -- the surrogate network's wide products on the 5th-generation
// tensor cores: D[M x 256] = A[M x K] B[K x 256] with bfloat16 operands and a
// float32 accumulator in tensor memory (TMEM), fused epilogue.
//
// A persistent CTA of 8 warps (one per SM) keeps the whole B operand resident
// in shared memory and works through 128-row tiles of D, i.e. 128 TMEM lanes x
// 256 float32 columns each.  K is consumed in chunks of 64.  Shared-memory
// operands use the canonical no-swizzle K-major layout -- 8-row x 16-byte core
// matrices, K-adjacent core matrices 128 B apart (leading byte offset),
// row-group-adjacent ones 1024 B apart (stride byte offset); B is a sequence of
// such 256-row chunks, A a ring of 128-row chunks filled by cp.async while the
// tensor core works on the chunks before them.  One thread issues the
// tcgen05.mma (K = 16 each) of a chunk and commits them to the chunk's ring-slot
// mbarrier, which frees the slot for the next fill.  After a tile's last chunk
// the 8 warps read the accumulator with tcgen05.ld (TMEM lanes 32w
// .. 32w + 31 for w = warp % 4, i.e. the tile's rows 32w .., and half warp / 4
// of the columns), add the bias and apply the ReLU
// (or keep the ReLU mask's entries), round to bfloat16 and store the rows
// through a per-warp staging buffer so that the lanes write whole 64-byte row
// pieces.  Every wait is bounded: a wait that runs out sets an error bit, and
// the CTA still releases its TMEM before it returns.
#include <cstdint>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "jatam_internal.cuh"

namespace jatam {
namespace {

constexpr int TC_M = 128, TC_N = 256, TC_KC = 64;  // tile rows, tile columns, K chunk
constexpr int TC_THREADS = 256;  // 8 warps: two per TMEM lane quarter in the epilogue
constexpr int TC_A_BYTES = TC_M * TC_KC * 2;       // 16 KB: one ring slot
constexpr int TC_B_BYTES = TC_N * TC_KC * 2;       // 32 KB: one K chunk of B
constexpr int TC_MAX_KCH = 4;                      // K <= 256
constexpr int TC_MAX_RING = 8;
constexpr int TC_STAGE_WORDS = 32 * 20;            // a warp's epilogue staging: 32 rows of 16 words, 16-byte padded
constexpr int TC_CTRL_BYTES = 2048;                // mbarriers (64 B), the TMEM address, the bias (1 KB)
constexpr int TC_OUT_BYTES = (TC_N * 8 + TC_M * 8) * 4;  // epi 2, 3: W3 as float32, the halves' partial logits
constexpr int TC_SMEM_BUDGET = 226 * 1024;
constexpr unsigned TC_WAIT_LIMIT = 1u << 20;       // mbarrier polls before giving up (about a second)
constexpr unsigned TC_ERR_TIMEOUT = 1u;

// byte offset of element (row, k) of a chunk in the core-matrix layout
__device__ __forceinline__ int cm_offset(int row, int k)
{
    return (((row >> 3) * (TC_KC / 8) + (k >> 3)) << 7) + ((row & 7) << 4) + ((k & 7) << 1);
}

// shared-memory matrix descriptor: start address, leading byte offset (between
// K-adjacent core matrices), stride byte offset (between row-adjacent groups of
// 8 rows), descriptor version 1, no swizzle
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo)
{
    uint64_t d = 0;
    d |= (uint64_t)((saddr >> 4) & 0x3FFFu);
    d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
    d |= (uint64_t)1 << 46;
    return d;
}

// instruction descriptor of kind::f16: float32 accumulator, bfloat16 A and B,
// both K-major, N = 256, M = 128
constexpr uint32_t TC_IDESC = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(TC_N >> 3) << 17) |
                              ((uint32_t)(TC_M >> 4) << 24);

__device__ __forceinline__ uint32_t smem_u32(const void *p)
{
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ bool mbar_wait(uint32_t mbar, uint32_t parity)
{
    for (unsigned it = 0; it < TC_WAIT_LIMIT; ++it) {
        uint32_t done;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(done)
            : "r"(mbar), "r"(parity)
            : "memory");
        if (done) return true;
    }
    return false;
}

struct TcArgs {
    const __nv_bfloat16 *A;
    long long a_m;       // element (m, k) at A[m * a_m + k]
    const __nv_bfloat16 *B;
    long long b_n;       // element (k, n) at B[n * b_n + k]
    int M, K;            // N = 256; K a multiple of 16, at most 256
    int ring;            // A ring slots
    int epi;             // 0: bias + ReLU -> bf16; 1: ReLU mask -> bf16; 2: bias + ReLU, rounded to bf16,
                         // then the 8 logits of the row (W3, b3) instead of the row itself; 3: both the
                         // row (as 0) and its logits (as 2)
    const float *bias;
    const __nv_bfloat16 *mask;
    __nv_bfloat16 *C;    // [M x 256] row-major (epi 0, 1)
    const __nv_bfloat16 *w3;  // epi 2: [256 x 8] row-major
    const float *b3;          // epi 2: [8]
    float *logits;            // epi 2: [M x 8] row-major
    unsigned *err;
};

__device__ __forceinline__ void cp_async16(uint32_t dst, const void *src, uint32_t bytes)
{
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(dst), "l"(src), "r"(bytes) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }

// wait until at most ring - 2 of this thread's copy groups are pending
__device__ __forceinline__ void cp_async_wait_ring(int ring)
{
    switch (ring) {
    case 2: cp_async_wait<0>(); break;
    case 3: cp_async_wait<1>(); break;
    case 4: cp_async_wait<2>(); break;
    case 5: cp_async_wait<3>(); break;
    case 6: cp_async_wait<4>(); break;
    case 7: cp_async_wait<5>(); break;
    default: cp_async_wait<6>(); break;
    }
}

__global__ void __launch_bounds__(TC_THREADS, 1) tc_gemm_kernel(const TcArgs g)
{
    extern __shared__ __align__(1024) unsigned char tc_smem[];
    const int nkc = (g.K + TC_KC - 1) / TC_KC;  // K chunks of a tile
    unsigned char *sb = tc_smem;                                      // B: nkc chunks of 32 KB
    unsigned char *sa = tc_smem + nkc * TC_B_BYTES;                   // A ring: g.ring slots of 16 KB
    uint32_t *stage = reinterpret_cast<uint32_t *>(sa + g.ring * TC_A_BYTES);  // 8 x 32 x 20 words
    float *outl = reinterpret_cast<float *>(stage + 8 * TC_STAGE_WORDS);  // epi 2, 3: W3, partial logits
    unsigned char *ctrl = reinterpret_cast<unsigned char *>(stage + 8 * TC_STAGE_WORDS) + TC_OUT_BYTES;
    uint64_t *mbar = reinterpret_cast<uint64_t *>(ctrl);             // [TC_MAX_RING]
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(ctrl + 8 * TC_MAX_RING);
    float *sbias = reinterpret_cast<float *>(ctrl + 8 * TC_MAX_RING + 16);  // [256]
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int ntiles = (g.M + TC_M - 1) / TC_M;
    const int mine = blockIdx.x < ntiles ? (ntiles - 1 - (int)blockIdx.x) / (int)gridDim.x + 1 : 0;
    const int total = mine * nkc;  // chunks this CTA consumes, tile by tile

    if (warp == 0) {
        // 256 TMEM columns for the 128 x 256 float32 accumulator
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 256;\n" ::"r"(smem_u32(tmem_slot))
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
    }
    if (tid == 0) {
        for (int i = 0; i < g.ring; ++i)
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_u32(mbar + i)) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    }
    for (int i = tid; i < TC_N; i += TC_THREADS) sbias[i] = g.epi != 1 ? g.bias[i] : 0.f;
    // epi 2, 3: W3 as float32, and after it the column halves' partial logits
    float *w3s = outl;               // [256][8]
    float *xch = outl + TC_N * 8;    // [128 rows][8]
    if (g.epi >= 2)
        for (int i = tid; i < TC_N * 8; i += TC_THREADS) w3s[i] = __bfloat162float(g.w3[i]);

    // B, resident: chunk c holds k in [64 c, 64 c + 64) of all 256 columns (zero past K)
    for (int e = tid; e < nkc * TC_N * (TC_KC / 8); e += TC_THREADS) {
        const int c = e / (TC_N * (TC_KC / 8)), rem = e % (TC_N * (TC_KC / 8));
        const int n = rem / (TC_KC / 8), k = (rem % (TC_KC / 8)) * 8;
        const int gk = c * TC_KC + k;
        const bool in = gk < g.K;  // K % 16 == 0: a piece is all in or all out
        cp_async16(smem_u32(sb + c * TC_B_BYTES + cm_offset(n, k)), g.B + (in ? n * g.b_n + gk : 0), in ? 16u : 0u);
    }
    // chunk q of this CTA: tile blockIdx.x + (q / nkc) gridDim.x, K chunk q % nkc, ring slot q % ring
    auto load_a = [&](int q) {
        const int m0 = ((int)blockIdx.x + (q / nkc) * (int)gridDim.x) * TC_M, k0 = (q % nkc) * TC_KC;
        unsigned char *dst = sa + (q % g.ring) * TC_A_BYTES;
        for (int e = tid; e < TC_M * (TC_KC / 8); e += TC_THREADS) {
            const int r = e / (TC_KC / 8), k = (e % (TC_KC / 8)) * 8;
            const int gm = m0 + r, gk = k0 + k;
            const bool in = gm < g.M && gk < g.K;
            cp_async16(smem_u32(dst + cm_offset(r, k)), g.A + (in ? (long long)gm * g.a_m + gk : 0), in ? 16u : 0u);
        }
    };
    // the first ring - 1 fills (the first group also carries B); empty groups keep the count uniform
    for (int q = 0; q < g.ring - 1; ++q) {
        if (q < total) load_a(q);
        cp_async_commit();
    }
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    const uint32_t tmem = *tmem_slot;
    bool ok = true;

    for (int q = 0; q < total && ok; ++q) {
        const int slot = q % g.ring;
        cp_async_wait_ring(g.ring);  // chunk q (and B) has landed in this thread's part
        // the copies must be visible to the tensor core's async proxy
        asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
        __syncthreads();
        const int kc = q % nkc;
        if (tid == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
            const int steps = min(TC_KC, g.K - kc * TC_KC) / 16;
            const uint32_t a0 = smem_u32(sa + slot * TC_A_BYTES), b0 = smem_u32(sb + kc * TC_B_BYTES);
            for (int s = 0; s < steps; ++s) {
                const uint64_t ad = smem_desc(a0 + s * 256, 128, 1024);
                const uint64_t bd = smem_desc(b0 + s * 256, 128, 1024);
                const uint32_t acc = (kc > 0 || s > 0) ? 1u : 0u;
                asm volatile(
                    "{\n\t.reg .pred p;\n\t"
                    "setp.ne.u32 p, %4, 0;\n\t"
                    "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}"
                    ::"r"(tmem), "l"(ad), "l"(bd), "r"(TC_IDESC), "r"(acc)
                    : "memory");
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(
                             smem_u32(mbar + slot))
                         : "memory");
        }
        // refill: chunk q + ring - 1 takes the slot of chunk q - 1, once its products have read it
        const int nq = q + g.ring - 1;
        if (nq < total) {
            if (q >= 1) {
                const int ps = (q - 1) % g.ring;
                ok = __syncthreads_and(mbar_wait(smem_u32(mbar + ps), (uint32_t)(((q - 1) / g.ring) & 1)) ? 1 : 0) != 0;
            }
            if (ok) load_a(nq);
        }
        cp_async_commit();
        if (ok && kc == nkc - 1) {
            // the tile's last products: wait for them, then the epilogue
            ok = __syncthreads_and(mbar_wait(smem_u32(mbar + slot), (uint32_t)((q / g.ring) & 1)) ? 1 : 0) != 0;
            if (!ok) break;
            asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
            // warp w reads TMEM lanes 32 (w % 4) .. (the rows of its quarter) and half w / 4 of the columns
            const int m0 = ((int)blockIdx.x + (q / nkc) * (int)gridDim.x) * TC_M;
            const int quarter = warp & 3, half = warp >> 2;
            const int wrow = m0 + quarter * 32;
            const uint32_t lane_base = tmem + ((uint32_t)(quarter * 32) << 16);
            uint32_t *st = stage + warp * TC_STAGE_WORDS;
            float part[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};  // epi 2: this half's logits of the row
            for (int cp = half * (TC_N / 2); cp < (half + 1) * (TC_N / 2); cp += 64) {
                // two 32-column reads, one wait
                uint32_t r[64];
                asm volatile(
                    "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, "
                    "%13, %14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, "
                    "[%32];\n"
                    : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
                      "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]),
                      "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]),
                      "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]),
                      "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
                    : "r"(lane_base + (uint32_t)cp));
                asm volatile(
                    "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, "
                    "%13, %14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, "
                    "[%32];\n"
                    : "=r"(r[32]), "=r"(r[33]), "=r"(r[34]), "=r"(r[35]), "=r"(r[36]), "=r"(r[37]), "=r"(r[38]),
                      "=r"(r[39]), "=r"(r[40]), "=r"(r[41]), "=r"(r[42]), "=r"(r[43]), "=r"(r[44]), "=r"(r[45]),
                      "=r"(r[46]), "=r"(r[47]), "=r"(r[48]), "=r"(r[49]), "=r"(r[50]), "=r"(r[51]), "=r"(r[52]),
                      "=r"(r[53]), "=r"(r[54]), "=r"(r[55]), "=r"(r[56]), "=r"(r[57]), "=r"(r[58]), "=r"(r[59]),
                      "=r"(r[60]), "=r"(r[61]), "=r"(r[62]), "=r"(r[63])
                    : "r"(lane_base + (uint32_t)cp + 32u));
                asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
#pragma unroll
                for (int b = 0; b < 2; ++b) {
                    const int c0 = cp + 32 * b;
                    // this lane's row, 32 columns, rounded to bfloat16 (bias + ReLU first for epi 0 and 2);
                    // the bias of the 32 columns, the same for every lane, read 16 bytes at a time
                    uint32_t w[16];
#pragma unroll
                    for (int q4 = 0; q4 < 8; ++q4) {
                        const float4 bb = g.epi != 1 ? *reinterpret_cast<const float4 *>(sbias + c0 + 4 * q4)
                                                     : make_float4(0.f, 0.f, 0.f, 0.f);
                        const float bv[4] = {bb.x, bb.y, bb.z, bb.w};
#pragma unroll
                        for (int h = 0; h < 4; h += 2) {
                            const int j = 4 * q4 + h;
                            float v0 = __uint_as_float(r[32 * b + j]), v1 = __uint_as_float(r[32 * b + j + 1]);
                            if (g.epi != 1) {
                                v0 = fmaxf(v0 + bv[h], 0.f);
                                v1 = fmaxf(v1 + bv[h + 1], 0.f);
                            }
                            const __nv_bfloat162 hv = __floats2bfloat162_rn(v0, v1);
                            w[j >> 1] = *reinterpret_cast<const uint32_t *>(&hv);
                        }
                    }
                    if (g.epi >= 2) {
                        // the row's partial logits over these 32 columns, in column order, from the
                        // rounded activations (the values the stored row holds)
#pragma unroll
                        for (int j = 0; j < 32; ++j) {
                            const float a = __uint_as_float(j & 1 ? (w[j >> 1] & 0xFFFF0000u) : (w[j >> 1] << 16));
                            const float4 wa = *reinterpret_cast<const float4 *>(w3s + (c0 + j) * 8);
                            const float4 wb = *reinterpret_cast<const float4 *>(w3s + (c0 + j) * 8 + 4);
                            part[0] = fmaf(a, wa.x, part[0]);
                            part[1] = fmaf(a, wa.y, part[1]);
                            part[2] = fmaf(a, wa.z, part[2]);
                            part[3] = fmaf(a, wa.w, part[3]);
                            part[4] = fmaf(a, wb.x, part[4]);
                            part[5] = fmaf(a, wb.y, part[5]);
                            part[6] = fmaf(a, wb.z, part[6]);
                            part[7] = fmaf(a, wb.w, part[7]);
                        }
                        if (g.epi == 2) continue;  // the row itself is not wanted
                    }
#pragma unroll
                    for (int q4 = 0; q4 < 4; ++q4)
                        *reinterpret_cast<uint4 *>(st + lane * 20 + 4 * q4) =
                            make_uint4(w[4 * q4], w[4 * q4 + 1], w[4 * q4 + 2], w[4 * q4 + 3]);
                    __syncwarp();
                    // 8 rows a pass, 4 lanes a row, 16 bytes a lane
#pragma unroll
                    for (int it = 0; it < 4; ++it) {
                        const int rr = it * 8 + (lane >> 2), pc = lane & 3;
                        const int grow = wrow + rr;
                        uint4 v = *reinterpret_cast<const uint4 *>(st + rr * 20 + 4 * pc);
                        if (grow < g.M) {
                            const long long o = (long long)grow * TC_N + c0 + 8 * pc;
                            if (g.epi == 1) {
                                // keep the entries where the mask is positive (rounding 0 gives 0, so
                                // masking after the rounding is the same as before it)
                                const uint4 mk = *reinterpret_cast<const uint4 *>(g.mask + o);
                                const uint32_t mw[4] = {mk.x, mk.y, mk.z, mk.w};
                                uint32_t vw[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
                                for (int h = 0; h < 4; ++h) {
                                    const float lo = __uint_as_float(mw[h] << 16);
                                    const float hi = __uint_as_float(mw[h] & 0xFFFF0000u);
                                    vw[h] = (lo > 0.f ? (vw[h] & 0xFFFFu) : 0u) | (hi > 0.f ? (vw[h] & 0xFFFF0000u) : 0u);
                                }
                                v = make_uint4(vw[0], vw[1], vw[2], vw[3]);
                            }
                            *reinterpret_cast<uint4 *>(g.C + o) = v;
                        }
                    }
                    __syncwarp();
                }
            }
            if (g.epi >= 2) {
                // the second column half hands its partial logits to the first, which adds them (first
                // half + second half, then the bias) and stores the row's 8 logits
                if (half == 1) {
#pragma unroll
                    for (int c = 0; c < 8; ++c) xch[(quarter * 32 + lane) * 8 + c] = part[c];
                }
                __syncthreads();
                const int grow = wrow + lane;
                if (half == 0 && grow < g.M) {
                    float o[8];
#pragma unroll
                    for (int c = 0; c < 8; ++c) o[c] = part[c] + xch[(quarter * 32 + lane) * 8 + c] + g.b3[c];
                    float4 *dst = reinterpret_cast<float4 *>(g.logits + (long long)grow * 8);
                    dst[0] = make_float4(o[0], o[1], o[2], o[3]);
                    dst[1] = make_float4(o[4], o[5], o[6], o[7]);
                }
            }
            // every warp has read the accumulator (and the exchanged logits) before the next tile's
            // products overwrite it
            asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
            __syncthreads();
            asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
        }
    }
    cp_async_wait<0>();
    if (!ok && tid == 0) atomicOr(g.err, TC_ERR_TIMEOUT);
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
    if (warp == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 256;\n" ::"r"(tmem) : "memory");
    }
}

}  // namespace

cudaError_t tc_gemm_n256(const __nv_bfloat16 *A, long long a_m, long long a_k, const __nv_bfloat16 *B, long long b_k,
                         long long b_n, int M, int K, int epi, const float *bias, const __nv_bfloat16 *mask,
                         __nv_bfloat16 *C, unsigned *err, cudaStream_t st, const __nv_bfloat16 *w3, const float *b3,
                         float *logits)
{
    static int sms[64] = {};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    if (!sms[dev]) {
        e = cudaFuncSetAttribute(tc_gemm_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, TC_SMEM_BUDGET);
        if (e != cudaSuccess) return e;
        int n = 0;
        e = cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
        if (e != cudaSuccess) return e;
        sms[dev] = n;
    }
    if (M <= 0) return cudaSuccess;
    // K-contiguous operands with 16-byte aligned rows only (the caller keeps the others on mma.sync)
    if (K <= 0 || K % 16 != 0 || K > TC_MAX_KCH * TC_KC || a_k != 1 || b_k != 1 || a_m % 8 != 0 || b_n % 8 != 0 ||
        ((uintptr_t)A & 15) != 0 || ((uintptr_t)B & 15) != 0 || ((uintptr_t)C & 15) != 0 ||
        (epi == 1 && ((uintptr_t)mask & 15) != 0) || (epi >= 2 && (!w3 || !b3 || ((uintptr_t)logits & 15) != 0)))
        return cudaErrorInvalidValue;
    const int nkc = (K + TC_KC - 1) / TC_KC;
    const int fixed = nkc * TC_B_BYTES + 8 * TC_STAGE_WORDS * 4 + TC_OUT_BYTES + TC_CTRL_BYTES;
    const int ring = min(TC_MAX_RING, (TC_SMEM_BUDGET - fixed) / TC_A_BYTES);
    const int bytes = fixed + ring * TC_A_BYTES;
    const int ntiles = (M + TC_M - 1) / TC_M;
    TcArgs g{A, a_m, B, b_n, M, K, ring, epi, bias, mask, C, w3, b3, logits, err};
    tc_gemm_kernel<<<(unsigned)min(ntiles, sms[dev]), TC_THREADS, bytes, st>>>(g);
    return cudaGetLastError();
}

}  // namespace jatam
