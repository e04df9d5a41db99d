// jatam_ga.cu -- genetic-algorithm kernels of libjatam.so (Section 2.2 of the
// paper: global roulette-wheel or tournament selection, single-point or
// uniform crossover, Poisson mutation of bit-encoded genomes; Section 3.2: the
// Fujiyama test-bed fitness, the Hamming weight of the genome).
//
// One thread breeds one child.  Its draws are fixed: word k of child i in
// generation g is word (k mod 4) of Philox4x32-10(ctr = (k >> 2, (2 << 24) | g,
// i_lo, i_hi), key = seed), in the order: selection of parent A (T tournament
// words, or one roulette dart), parent B, the crossover decision, two cut/mask
// words, one Poisson word per edge, then four bit-choice words per edge.
#include <cstdint>
#include <cuda_runtime.h>

#include "jatam_device.cuh"
#include "jatam_internal.cuh"

namespace jatam {
namespace {

// the draws of one child, one Philox block at a time
struct ChildDraws {
    uint32_t k0, k1, gen;
    unsigned long long child;
    uint32_t blk = 0xFFFFFFFFu;
    uint4 w;
    __device__ uint32_t word(int k)
    {
        const uint32_t b = (uint32_t)k >> 2;
        if (b != blk) {
            w = philox4x32_10(make_uint4(b, (2u << 24) | gen, (uint32_t)child, (uint32_t)(child >> 32)), k0, k1);
            blk = b;
        }
        const int s = k & 3;
        return s == 0 ? w.x : s == 1 ? w.y : s == 2 ? w.z : w.w;
    }
};

__device__ unsigned long long select_parent(const GaArgs &g, ChildDraws &d, int k0)
{
    if (g.selection == 0) {
        // tournament: the fittest of T uniformly drawn parents (the earliest on ties)
        unsigned long long best = 0;
        int32_t bf = 0;
        for (int j = 0; j < g.tournament; ++j) {
            const unsigned long long idx = ((unsigned long long)d.word(k0 + j) * g.N) >> 32;
            const int32_t f = g.fitness[idx];
            if (j == 0 || f > bf) {
                best = idx;
                bf = f;
            }
        }
        return best;
    }
    // roulette wheel: the parent in whose slice of the cumulative fitness the dart lands
    const unsigned long long total = g.cumsum[g.N - 1];
    const uint32_t u = d.word(k0);
    if (total == 0) return ((unsigned long long)u * g.N) >> 32;
    const unsigned long long dart = ((unsigned long long)u * total) >> 32;
    unsigned long long lo = 0, hi = g.N - 1;  // first i with cumsum[i] > dart
    while (lo < hi) {
        const unsigned long long mid = (lo + hi) >> 1;
        if (g.cumsum[mid] > dart) hi = mid;
        else lo = mid + 1;
    }
    return lo;
}

__global__ void __launch_bounds__(256) ga_breed_kernel(const GaArgs g)
{
    const unsigned long long i = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x;
    if (i >= g.Nc) return;
    ChildDraws d;
    d.k0 = g.key0;
    d.k1 = g.key1;
    d.gen = g.generation;
    d.child = i;
    const int T = g.selection == 0 ? g.tournament : 1;
    const unsigned long long a = g.parents[select_parent(g, d, 0)];
    const unsigned long long b = g.parents[select_parent(g, d, T)];
    unsigned long long child = a;
    const int k_cross = 2 * T, k_mask = 2 * T + 1, k_pois = 2 * T + 3, k_bit = 2 * T + 3 + 4 * g.n;
    if (g.crossover != 0 && d.word(k_cross) < g.crossover_threshold) {
        if (g.crossover == 1) {
            const int cut = 1 + (int)(((unsigned long long)d.word(k_mask) * (unsigned long long)(g.bits - 1)) >> 32);
            const unsigned long long low = (1ull << cut) - 1ull;
            child = (a & ~low) | (b & low);
        } else {
            const unsigned long long mask = ((unsigned long long)d.word(k_mask + 1) << 32) | d.word(k_mask);
            child = (a & ~mask) | (b & mask);
        }
    }
    if (g.b > 0) {
        for (int e = 0; e < 4 * g.n; ++e) {
            const uint32_t u = d.word(k_pois + e);
            int events = 0;
#pragma unroll
            for (int j = 0; j < 4; ++j) events += (u >= g.mutation_thresholds[j]) ? 1 : 0;
            const int t = e >> 2, side = e & 3;
            const int pos = g.b * (4 * (g.n - 1 - t) + (3 - side));
            for (int m = 0; m < events; ++m) {
                const int bit = (int)(((unsigned long long)d.word(k_bit + 4 * e + m) * (unsigned long long)g.b) >> 32);
                child ^= 1ull << (pos + bit);
            }
        }
    }
    g.children[i] = g.bits >= 64 ? child : (child & ((1ull << g.bits) - 1ull));
}

// inclusive prefix sum of the (non-negative parts of the) fitness values, one CTA
__global__ void __launch_bounds__(1024) ga_scan_kernel(const int32_t *fitness, unsigned long long n,
                                                       unsigned long long *cumsum)
{
    __shared__ unsigned long long part[1024];
    const unsigned long long per = (n + blockDim.x - 1) / blockDim.x;
    const unsigned long long lo = threadIdx.x * per, hi = min(n, lo + per);
    unsigned long long s = 0;
    for (unsigned long long i = lo; i < hi; ++i) s += fitness[i] > 0 ? (unsigned long long)fitness[i] : 0ull;
    part[threadIdx.x] = s;
    __syncthreads();
    for (int off = 1; off < (int)blockDim.x; off <<= 1) {
        const unsigned long long v = threadIdx.x >= (unsigned)off ? part[threadIdx.x - off] : 0ull;
        __syncthreads();
        part[threadIdx.x] += v;
        __syncthreads();
    }
    unsigned long long run = threadIdx.x ? part[threadIdx.x - 1] : 0ull;
    for (unsigned long long i = lo; i < hi; ++i) {
        run += fitness[i] > 0 ? (unsigned long long)fitness[i] : 0ull;
        cumsum[i] = run;
    }
}

__global__ void ga_hamming_kernel(const unsigned long long *genomes, unsigned long long n, int32_t *fitness)
{
    for (unsigned long long i = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; i < n;
         i += (unsigned long long)gridDim.x * blockDim.x)
        fitness[i] = __popcll(genomes[i]);
}

// best fitness and fitness total of a population: stats[0] = max, stats[1] = sum
__global__ void ga_stats_kernel(const int32_t *fitness, unsigned long long n, long long *stats)
{
    long long mx = -0x7FFFFFFFFFFFFFFFll, sm = 0;
    for (unsigned long long i = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; i < n;
         i += (unsigned long long)gridDim.x * blockDim.x) {
        mx = max(mx, (long long)fitness[i]);
        sm += fitness[i];
    }
    for (int off = 16; off > 0; off >>= 1) {
        mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, off));
        sm += __shfl_xor_sync(0xffffffffu, sm, off);
    }
    if ((threadIdx.x & 31) == 0) {
        atomicMax(reinterpret_cast<long long *>(&stats[0]), mx);
        atomicAdd(reinterpret_cast<unsigned long long *>(&stats[1]), (unsigned long long)sm);
    }
}

__global__ void ga_stats_reset_kernel(long long *stats)
{
    stats[0] = -0x7FFFFFFFFFFFFFFFll;
    stats[1] = 0;
}

}  // namespace

cudaError_t launch_ga_breed(const GaArgs &g, cudaStream_t st)
{
    if (g.N == 0 || g.Nc == 0) return cudaSuccess;
    if (g.selection == 1) {
        ga_scan_kernel<<<1, 1024, 0, st>>>(g.fitness, g.N, const_cast<unsigned long long *>(g.cumsum));
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    ga_breed_kernel<<<(unsigned)((g.Nc + 255) / 256), 256, 0, st>>>(g);
    return cudaGetLastError();
}

cudaError_t launch_ga_hamming(const unsigned long long *genomes, unsigned long long n, int32_t *fitness,
                              cudaStream_t st)
{
    if (n == 0) return cudaSuccess;
    const unsigned long long blocks = min((n + 255ull) / 256ull, 4096ull);
    ga_hamming_kernel<<<(unsigned)blocks, 256, 0, st>>>(genomes, n, fitness);
    return cudaGetLastError();
}

cudaError_t launch_ga_stats(const int32_t *fitness, unsigned long long n, long long *stats, cudaStream_t st)
{
    ga_stats_reset_kernel<<<1, 1, 0, st>>>(stats);
    if (n) {
        const unsigned long long blocks = min((n + 255ull) / 256ull, 1024ull);
        ga_stats_kernel<<<(unsigned)blocks, 256, 0, st>>>(fitness, n, stats);
    }
    return cudaGetLastError();
}

}  // namespace jatam
