// jatam_tc.cu -- the surrogate network's wide products on the 5th-generation
// tensor cores: D[M x 256] = A[M x K] B[K x 256] with bfloat16 operands and a
// float32 accumulator in tensor memory (TMEM), fused epilogue.
//
// One CTA of 4 warps owns a 128-row tile of D, i.e. 128 TMEM lanes x 256
// float32 columns.  K is consumed in chunks of 64: all threads stage the A
// chunk (128 x 64) and the B chunk (256 x 64, transposed to K-major) into
// shared memory in the canonical no-swizzle K-major layout -- 8-row x 16-byte
// core matrices, K-adjacent core matrices 128 B apart (leading byte offset),
// row-group-adjacent ones 1024 B apart (stride byte offset) -- then one thread
// issues four tcgen05.mma (K = 16 each) and commits them to an mbarrier that
// every thread waits on before the buffers are reused.  The epilogue reads the
// accumulator with tcgen05.ld (warp w owns TMEM lanes 32w .. 32w + 31, i.e.
// the tile's rows 32w ..), adds the bias / applies the ReLU or the ReLU mask,
// and stores bfloat16 rows.  Every wait is bounded: a wait that runs out sets
// an error bit, and the CTA still releases its TMEM before it returns.
#include <cstdint>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "jatam_internal.cuh"

namespace jatam {
namespace {

constexpr int TC_M = 128, TC_N = 256, TC_KC = 64;  // tile rows, tile columns, K chunk
constexpr int TC_THREADS = 128;
constexpr int TC_A_BYTES = TC_M * TC_KC * 2;       // 16 KB
constexpr int TC_B_BYTES = TC_N * TC_KC * 2;       // 32 KB
// the operand buffers need 48 KB; asking for 100 KB keeps at most two CTAs on an
// SM, so their two 256-column TMEM allocations always fit the SM's 512 columns
// and tcgen05.alloc never has to wait for another CTA
constexpr int TC_SMEM = 100 * 1024;
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
    long long a_m, a_k;  // element (m, k) at A[m * a_m + k * a_k]
    const __nv_bfloat16 *B;
    long long b_k, b_n;  // element (k, n) at B[k * b_k + n * b_n]
    int M, K;            // N = 256; K a multiple of 16
    int epi;             // 0: bias + ReLU -> bf16; 1: ReLU mask -> bf16
    const float *bias;
    const __nv_bfloat16 *mask;
    __nv_bfloat16 *C;    // [M x 256] row-major
    unsigned *err;
};

__global__ void __launch_bounds__(TC_THREADS, 1) tc_gemm_kernel(const TcArgs g)
{
    extern __shared__ __align__(1024) unsigned char tc_smem[];
    unsigned char *sa = tc_smem;
    unsigned char *sb = tc_smem + TC_A_BYTES;
    uint64_t *mbar = reinterpret_cast<uint64_t *>(tc_smem + TC_A_BYTES + TC_B_BYTES);
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(tc_smem + TC_A_BYTES + TC_B_BYTES + 16);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int m0 = blockIdx.x * TC_M;

    if (warp == 0) {
        // 256 TMEM columns for the 128 x 256 float32 accumulator
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 256;\n" ::"r"(smem_u32(tmem_slot))
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
    }
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_u32(mbar)) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    const uint32_t tmem = *tmem_slot;
    const uint32_t mb = smem_u32(mbar);
    bool ok = true;
    uint32_t phase = 0;

    const __nv_bfloat16 zero = __float2bfloat16(0.f);
    // K % 16 == 0 (checked by the host), so a K-contiguous operand never has a partial 8-element piece
    const bool a_vec = g.a_k == 1 && g.a_m % 8 == 0 && ((uintptr_t)g.A & 15) == 0;
    const bool b_vec = g.b_k == 1 && g.b_n % 8 == 0 && ((uintptr_t)g.B & 15) == 0;
    for (int kc = 0; kc < g.K && ok; kc += TC_KC) {
        // stage the chunk: A rows m0 .., B columns 0 .. 255 (as rows of the K-major operand).
        // An operand whose K is contiguous (and rows 16-byte aligned) moves in
        // 16-byte pieces, one core-matrix row each; any other, element by element.
        if (a_vec) {
            for (int e = tid; e < TC_M * (TC_KC / 8); e += TC_THREADS) {
                const int r = e / (TC_KC / 8), k = (e % (TC_KC / 8)) * 8;
                const int gm = m0 + r, gk = kc + k;
                uint4 v = make_uint4(0u, 0u, 0u, 0u);
                if (gm < g.M && gk < g.K) v = *reinterpret_cast<const uint4 *>(g.A + gm * g.a_m + gk);
                *reinterpret_cast<uint4 *>(sa + cm_offset(r, k)) = v;
            }
        } else {
            for (int e = tid; e < TC_M * TC_KC; e += TC_THREADS) {
                const int r = e / TC_KC, k = e % TC_KC;
                const int gm = m0 + r, gk = kc + k;
                const __nv_bfloat16 v = (gm < g.M && gk < g.K) ? g.A[gm * g.a_m + gk * g.a_k] : zero;
                *reinterpret_cast<__nv_bfloat16 *>(sa + cm_offset(r, k)) = v;
            }
        }
        if (b_vec) {
            for (int e = tid; e < TC_N * (TC_KC / 8); e += TC_THREADS) {
                const int n = e / (TC_KC / 8), k = (e % (TC_KC / 8)) * 8;
                const int gk = kc + k;
                uint4 v = make_uint4(0u, 0u, 0u, 0u);
                if (gk < g.K) v = *reinterpret_cast<const uint4 *>(g.B + n * g.b_n + gk);
                *reinterpret_cast<uint4 *>(sb + cm_offset(n, k)) = v;
            }
        } else {
            for (int e = tid; e < TC_N * TC_KC; e += TC_THREADS) {
                const int n = e / TC_KC, k = e % TC_KC;
                const int gk = kc + k;
                const __nv_bfloat16 v = (gk < g.K) ? g.B[gk * g.b_k + n * g.b_n] : zero;
                *reinterpret_cast<__nv_bfloat16 *>(sb + cm_offset(n, k)) = v;
            }
        }
        // the generic-proxy stores must be visible to the tensor core's async proxy
        asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
        __syncthreads();
        if (tid == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
            const int steps = min(TC_KC, g.K - kc) / 16;
            for (int s = 0; s < steps; ++s) {
                const uint64_t ad = smem_desc(smem_u32(sa) + s * 256, 128, 1024);
                const uint64_t bd = smem_desc(smem_u32(sb) + s * 256, 128, 1024);
                const uint32_t acc = (kc > 0 || s > 0) ? 1u : 0u;
                asm volatile(
                    "{\n\t.reg .pred p;\n\t"
                    "setp.ne.u32 p, %4, 0;\n\t"
                    "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}"
                    ::"r"(tmem), "l"(ad), "l"(bd), "r"(TC_IDESC), "r"(acc)
                    : "memory");
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(mb)
                         : "memory");
        }
        // every thread waits for the products before the buffers are refilled;
        // the outcome is made uniform so that all threads leave the loop together
        ok = __syncthreads_and(mbar_wait(mb, phase) ? 1 : 0) != 0;
        phase ^= 1u;
    }
    if (!ok) {
        if (tid == 0) atomicOr(g.err, TC_ERR_TIMEOUT);
    } else {
        asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
        // epilogue: this warp's 32 rows, 32 columns at a time
        const int row = m0 + warp * 32 + lane;
        const uint32_t lane_base = tmem + ((uint32_t)(warp * 32) << 16);
        for (int c0 = 0; c0 < TC_N; c0 += 32) {
            uint32_t r[32];
            asm volatile(
                "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, "
                "%14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];\n"
                : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
                  "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]),
                  "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]),
                  "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]),
                  "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
                : "r"(lane_base + (uint32_t)c0));
            asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
            if (row < g.M) {
                __nv_bfloat16 *out = g.C + (long long)row * TC_N + c0;
#pragma unroll
                for (int j = 0; j < 32; j += 2) {
                    float v0 = __uint_as_float(r[j]), v1 = __uint_as_float(r[j + 1]);
                    if (g.epi == 0) {
                        v0 = fmaxf(v0 + g.bias[c0 + j], 0.f);
                        v1 = fmaxf(v1 + g.bias[c0 + j + 1], 0.f);
                    } else {
                        const __nv_bfloat162 mk =
                            *reinterpret_cast<const __nv_bfloat162 *>(g.mask + (long long)row * TC_N + c0 + j);
                        v0 = __bfloat162float(mk.x) > 0.f ? v0 : 0.f;
                        v1 = __bfloat162float(mk.y) > 0.f ? v1 : 0.f;
                    }
                    *reinterpret_cast<__nv_bfloat162 *>(out + j) = __floats2bfloat162_rn(v0, v1);
                }
            }
        }
    }
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
                         __nv_bfloat16 *C, unsigned *err, cudaStream_t st)
{
    static bool attr[64] = {};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    if (!attr[dev]) {
        e = cudaFuncSetAttribute(tc_gemm_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, TC_SMEM);
        if (e != cudaSuccess) return e;
        attr[dev] = true;
    }
    if (M <= 0) return cudaSuccess;
    if (K <= 0 || K % 16 != 0) return cudaErrorInvalidValue;
    TcArgs g{A, a_m, a_k, B, b_k, b_n, M, K, epi, bias, mask, C, err};
    tc_gemm_kernel<<<(unsigned)((M + TC_M - 1) / TC_M), TC_THREADS, TC_SMEM, st>>>(g);
    return cudaGetLastError();
}

}  // namespace jatam
