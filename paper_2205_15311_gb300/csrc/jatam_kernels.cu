// jatam_kernels.cu -- sm_103a kernels of libjatam.so.
//
// One persistent warp serves 32 genotypes at a time, one per lane.  Each lane
// grows the replicate assemblies of its genotype one tile per loop iteration
// (Section 2.4: stochastic addition of bonding tiles until no tile fits or the
// grid edge is reached).  The lane's lattice lives in shared memory,
// interleaved so that word w of lane l sits at [w * 32 + l]: every lane always
// addresses its own bank, so the lane-private accesses never conflict (the
// bank-per-assembly idea of Section 2.4, kept because it still holds on
// sm_103a).  The per-genotype work that does not vectorise over lanes --
// building the binding tables and the canonical form of the final shape -- is
// done by the whole warp for one lane at a time, so it never serialises the
// warp behind a single lane.
//
// Per lane, for a lattice with rows of S bits (L <= S):
//   OCCA[NW]   occupancy of replicate 0 (kept for the comparison and the shape)
//   OCCB[NW]   occupancy of replicates 1..k-1
//   FRONT[NW]  frontier: empty in-grid sites with exactly one distinct candidate
//   NIB[S*S/8] 4-bit tuple id per cell: the placed tuple of an occupied cell or
//              the single candidate of a frontier cell
//   NBM[2 NT]  NBM[2 t + d/2] >> 16 (d & 1): the set of tuple ids that can
//              attach on side d of a placed tuple t (16 bits); NT = 8 tuple
//              ids for sets of at most two tiles, else 16
// A tuple id is the lowest (tile, rotation) index 4 t + r with that rotated
// colour tuple, so equal tuples (repeated tile types, symmetric tiles) share
// an id and never count as ambiguity (Section 2.4).

#include <cstdint>
#include <cuda_runtime.h>

#include <map>
#include <mutex>
#include <tuple>

#include "jatam_device.cuh"
#include "jatam_internal.cuh"

namespace jatam {

// Per-lane shared-memory layout of a lattice with rows of S bits.
template <int S, int NT = 16>
struct Geo {
    static constexpr int NW = (S * S) / 32;  // words per bitmap
    static constexpr int LOG2S = (S == 8) ? 3 : (S == 16) ? 4 : 5;
    static constexpr int OCCA = 0;
    static constexpr int OCCB = NW;
    static constexpr int FRONT = 2 * NW;
    static constexpr int NIB = 3 * NW;
    static constexpr int NBM = 3 * NW + (S * S) / 8;  // 2 words per tuple id: NT = 8 (<= 2 tiles) or 16
    static constexpr int CACHE = NBM + 2 * NT;  // per-warp shape cache: entry j in "lane" j's bank
    static constexpr int WORDS = CACHE + 3;      // 32-bit words per lane
};

namespace {

constexpr unsigned FULL = 0xffffffffu;
constexpr int HIST_SLOTS = 256;  // per-CTA phenotype aggregation table
constexpr int CHUNK = 32;        // items taken from the global counter at once
constexpr int CROP_PROBES = 4;   // slots of the crop table tried per lookup
constexpr int CROP_CELLS = 48;   // crops of at most this many cells are kept in the crop table

// key of a crop in the crop table: its h x w bits (row i at bits i * w ..) with h and w above
// them, so that crops of different dimensions never share a key (h * w <= CROP_CELLS)
__device__ __forceinline__ unsigned long long crop_key(unsigned long long bits, int h, int w)
{
    return bits | ((unsigned long long)h << 48) | ((unsigned long long)w << 56);
}

enum Phase : int { PH_NEED = 0, PH_INIT, PH_START, PH_GROW, PH_DOM, PH_SHAPE, PH_WRITE, PH_DONE };


// Jenkins one-at-a-time, one byte at a time (Section 2.5).
__device__ __forceinline__ uint32_t oaat_add(uint32_t h, uint32_t byte)
{
    h += byte;
    h += h << 10;
    h ^= h >> 6;
    return h;
}
__device__ __forceinline__ uint32_t oaat_finish(uint32_t h)
{
    h += h << 3;
    h ^= h >> 11;
    h += h << 15;
    return h;
}

// position of the i-th (0-based) set bit of v; requires i < popc(v)
__device__ __forceinline__ int nth_set(uint32_t v, uint32_t i)
{
    int pos = 0;
    uint32_t c = __popc(v & 0xFFFFu);
    if (i >= c) { i -= c; v >>= 16; pos += 16; }
    c = __popc(v & 0xFFu);
    if (i >= c) { i -= c; v >>= 8; pos += 8; }
    c = __popc(v & 0xFu);
    if (i >= c) { i -= c; v >>= 4; pos += 4; }
    c = __popc(v & 0x3u);
    if (i >= c) { i -= c; v >>= 2; pos += 2; }
    if (i >= (v & 1u)) pos += 1;
    return pos;
}

__device__ __forceinline__ unsigned lanemask_lt()
{
    unsigned m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

template <int S>
__device__ __forceinline__ int nib_get(const uint32_t *my, int b)
{
    return (my[(Geo<S>::NIB + (b >> 3)) * 32] >> ((b & 7) * 4)) & 15;
}
template <int S>
__device__ __forceinline__ void nib_set(uint32_t *my, int b, int v)
{
    uint32_t *p = &my[(Geo<S>::NIB + (b >> 3)) * 32];
    const int sh = (b & 7) * 4;
    *p = (*p & ~(15u << sh)) | ((uint32_t)v << sh);
}

// state of one lane's genotype
struct Lane {
    int phase;
    unsigned long long item;  // output position
    unsigned long long sid;   // stream id
    unsigned long long cols;  // colour of edge e of tile t at nibble 4 t + e
    int n, c, L, k;
    int rep, step, size, size0, nF;
    unsigned long long fc;       // lattices with at most 8 frontier words: byte w = sites in word w
    int sp;                      // movelist process: sites on this lane's stack
    int ymin, ymax, xmin, xmax;  // bounding box of the current replicate
    int x0, x1, y0, y1;          // bounding box of replicate 0
    int dlo, dhi;                // rows that may be dirty in any bitmap
    int blo, bhi;                // rows of OCCB written by the current replicate
    int diverged;                // replicate j > 0 can no longer end in replicate 0's configuration
    int forced;                  // replicate 0 so far never had more than one frontier site to choose from
    int cert;                    // replicate 0 so far: every occupied neighbour of a placed tile can only
                                 // receive, from that tile, the tuple it holds (or nothing)
    int cls, decided;
    uint32_t hash;
    uint32_t ka, kb;             // Philox blocks held: key = replicate * 512 + block (NO_BLOCK if none)
    uint4 pa, pb;                // pa: the block in use; pb: a block fetched ahead
};

constexpr uint32_t NO_BLOCK = 0xFFFFFFFFu;

// Philox block `key` (replicate key >> 9, block key & 511) of stream id sid
__device__ __forceinline__ uint4 philox_block(uint32_t key, unsigned long long sid, uint32_t k0, uint32_t k1)
{
    return philox4x32_10(make_uint4(key & 511u, key >> 9, (uint32_t)sid, (uint32_t)(sid >> 32)), k0, k1);
}

template <int S>
__device__ __forceinline__ void clear_rows(uint32_t *my, int base, int lo, int hi)
{
    const int wlo = (lo * S) >> 5, whi = (hi * S) >> 5;
    for (int w = wlo; w <= whi; ++w) my[(base + w) * 32] = 0u;
}

// ---------------------------------------------------------------------------
// binding tables of one lane's new genotype, built by the lane alone (all new
// lanes of a warp at once).  Tuple l = 4 t + r is tile t turned clockwise by r
// quarter turns: side d carries the colour of edge (d - r) mod 4.  l is the
// representative of its rotated tuple -- the lowest (tile, rotation) index with
// that tuple -- unless a lower rotation of the same tile gives the same tuple
// (r = 1: the tile is symmetric under a quarter turn; r = 2, 3: under a half
// turn, which a quarter-turn symmetry implies) or an earlier tile is a rotation
// of this one.  NBM[2 l + d / 2] >> 16 (d & 1) is the set of representatives
// whose side d + 2 carries the partner of l's colour on side d (Section 2.2:
// 1-2, 3-4, 5-6 bind; 0 and an odd top colour bind nothing).
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t rot16(uint32_t x, int k)
{
    return ((x << k) | (x >> (16 - k))) & 0xFFFFu;
}

// Bit planes over (tile, rotation): bit 4 t + r of plane(e, b) is bit b of the
// colour that tuple 4 t + r shows on side e, i.e. of edge (e - r) mod 4 of
// tile t.  x holds bit b of every edge of two tiles (bit 4 j + 16 u: edge j of
// tile u); one multiply moves edge (e - r) mod 4 of each tile to bit r of a
// nibble (at K_e and K_e + 16).  The constants put every partial product on
// its own bit, so no sum carries and no other product lands in the nibbles:
//   e = 0: edges 0,3,2,1 -> x * (2^11 + 2^10 + 2^5 + 1) >> 11
//   e = 1: edges 1,0,3,2 -> x * (2^11 + 2^6 + 2^5 + 1)  >> 10
//   e = 2: edges 2,1,0,3 -> x * (2^11 + 2^6 + 2 + 1)    >> 9
//   e = 3: edges 3,2,1,0 -> x * (2^15 + 2^10 + 2^5 + 1) >> 12
template <int E>
__device__ __forceinline__ uint32_t plane_spread(uint32_t x)  // tile 0 at bits 0..3, tile 1 at 16..19
{
    constexpr uint32_t MUL = E == 0 ? 0xC21u : E == 1 ? 0x861u : E == 2 ? 0x843u : 0x8421u;
    constexpr int K = E == 0 ? 11 : E == 1 ? 10 : E == 2 ? 9 : 12;
    return ((x * MUL) >> K) & 0x000F000Fu;
}
template <int E>
__device__ __forceinline__ uint32_t plane_byte(uint32_t x)  // tile 0 at bits 0..3, tile 1 at 4..7
{
    const uint32_t z = plane_spread<E>(x);
    return (z | (z >> 12)) & 0xFFu;
}

template <int S, int NT>
__device__ __forceinline__ void lane_tables(uint32_t *my, unsigned long long cols, int n, int c)
{
    using G = Geo<S>;
    constexpr int NTILE = NT / 4;
    const uint32_t lo = (uint32_t)cols, hi = (uint32_t)(cols >> 32);
    uint32_t tl[NTILE];
#pragma unroll
    for (int t = 0; t < NTILE; ++t) tl[t] = ((t < 2 ? lo : hi) >> (16 * (t & 1))) & 0xFFFFu;
    uint32_t reps = 0;
#pragma unroll
    for (int t = 0; t < NTILE; ++t) {
        const uint32_t tile = tl[t];
        uint32_t m = 1u | (rot16(tile, 4) != tile ? 2u : 0u) | (rot16(tile, 8) != tile ? 12u : 0u);
#pragma unroll
        for (int u = 0; u < t; ++u) {
            const uint32_t tu = tl[u];
            if (tile == tu || tile == rot16(tu, 4) || tile == rot16(tu, 8) || tile == rot16(tu, 12)) m = 0u;
        }
        if (t < n) reps |= m << (4 * t);
    }
    uint32_t P[4][3];
#pragma unroll
    for (int b = 0; b < 3; ++b) {
        const uint32_t xl = (lo >> b) & 0x11111111u;
        P[0][b] = plane_byte<0>(xl);
        P[1][b] = plane_byte<1>(xl);
        P[2][b] = plane_byte<2>(xl);
        P[3][b] = plane_byte<3>(xl);
        if constexpr (NTILE > 2) {
            const uint32_t xh = (hi >> b) & 0x11111111u;
            P[0][b] |= plane_byte<0>(xh) << 8;
            P[1][b] |= plane_byte<1>(xh) << 8;
            P[2][b] |= plane_byte<2>(xh) << 8;
            P[3][b] |= plane_byte<3>(xh) << 8;
        }
    }
    // not unrolled over tiles: the growth kernel is sensitive to its code size
    // (warps in different phases share the instruction cache)
#pragma unroll 1
    for (int t = 0; t < n; ++t) {
        const uint32_t tile_t = (uint32_t)(cols >> (16 * t)) & 0xFFFFu;
        uint32_t w[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) w[j] = 0u;
#pragma unroll
        for (int s = 0; s < 4; ++s) {
            const int a = (int)((tile_t >> (4 * s)) & 15u);
            const int pa = (a == 0) ? -1 : (a & 1) ? ((a + 1 < c) ? a + 1 : -1) : a - 1;
            const uint32_t rz = pa >= 0 ? reps : 0u;
            const uint32_t n0 = 0u - (uint32_t)(pa & 1), n1 = 0u - (uint32_t)((pa >> 1) & 1),
                           n2 = 0u - (uint32_t)((pa >> 2) & 1);
            uint32_t X[4];
#pragma unroll
            for (int e = 0; e < 4; ++e) X[e] = rz & ~(P[e][0] ^ n0) & ~(P[e][1] ^ n1) & ~(P[e][2] ^ n2);
            // edge s of tile t is side d = s + r of tuple 4 t + r; it binds side d + 2
#pragma unroll
            for (int r = 0; r < 4; ++r) {
                const int d = (s + r) & 3;
                w[2 * r + (d >> 1)] |= X[(d + 2) & 3] << (16 * (d & 1));
            }
        }
#pragma unroll
        for (int j = 0; j < 8; ++j) my[(G::NBM + 8 * t + j) * 32] = w[j];
    }
}

// one-at-a-time over (h, w) and (x, y) of every occupied cell of an image held
// as rows in lanes (row i in lane i, its first cell the most significant of wc bits)
__device__ __forceinline__ uint32_t image_hash(uint32_t v, int hc, int wc)
{
    uint32_t hsh = oaat_add(0u, (uint32_t)hc);
    hsh = oaat_add(hsh, (uint32_t)wc);
    for (int i = 0; i < hc; ++i) {
        uint32_t row = __shfl_sync(FULL, v, i);
        while (row) {
            const int p = 31 - __clz(row);
            hsh = oaat_add(hsh, (uint32_t)(wc - 1 - p));
            hsh = oaat_add(hsh, (uint32_t)i);
            row &= ~(1u << p);
        }
    }
    return oaat_finish(hsh);
}

// four image hashes sorted and hashed again, byte by byte (little endian)
__device__ __forceinline__ uint32_t c4_combine(uint32_t a, uint32_t b, uint32_t c, uint32_t d)
{
    uint32_t x[4] = {a, b, c, d};
#pragma unroll
    for (int i = 1; i < 4; ++i)
#pragma unroll
        for (int j = i; j > 0; --j)
            if (x[j - 1] > x[j]) {
                const uint32_t t = x[j];
                x[j] = x[j - 1];
                x[j - 1] = t;
            }
    uint32_t hsh = 0u;
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int byte = 0; byte < 4; ++byte) hsh = oaat_add(hsh, (x[i] >> (8 * byte)) & 255u);
    return oaat_finish(hsh);
}

// ---------------------------------------------------------------------------
// Exact side table of a call's shapes (Section 2.5 estimates the chance that
// two distinct shapes share a 32-bit hash; the table settles it exactly): the
// first warp that stores a hash keeps the canonical form under it, every later
// warp with the same hash compares its form with the stored one.  A form is a
// function of its crop, and every crop of a call is either in the call's crop
// table or in its spill list, so the pass over both (shape_scan_kernel) sees
// every distinct form.  All 32 lanes call it; lane i < h holds row i of the
// form.
// ---------------------------------------------------------------------------
constexpr int SHAPE_PROBES = 64;      // slots tried before a form is counted as not stored
constexpr int SHAPE_WAIT = 1 << 16;   // polls of a slot whose rows are still being written

__device__ __forceinline__ void shape_record(const ShapeTab &t, uint32_t hash, uint32_t row, int h, int w, int lane)
{
    const unsigned mask = (1u << t.log2) - 1u;
    const unsigned long long key = (1ull << 32) | hash;
    unsigned slot = (hash * 2654435761u) >> (32 - t.log2);
    int state = 0;  // 1: stored by this warp, 2: present, 3: table full
    if (lane == 0) {
        for (int p = 0; p < SHAPE_PROBES; ++p) {
            const unsigned long long old = atomicCAS(&t.key[slot], 0ull, key);
            if (old == 0ull) { state = 1; break; }
            if (old == key) { state = 2; break; }
            slot = (slot + 1) & mask;
        }
        if (!state) state = 3;
    }
    state = __shfl_sync(FULL, state, 0);
    slot = __shfl_sync(FULL, slot, 0);
    const uint32_t mine = lane < h ? row : 0u;
    const unsigned meta = 0x80000000u | ((unsigned)h << 8) | (unsigned)w;
    if (state == 1) {
        // the rows, then (after the warp barrier, which orders the lanes' stores before lane 0's
        // fence) the meta word that publishes them
        __stcg(&t.rows[(size_t)slot * 32 + lane], mine);
        __syncwarp();
        if (lane == 0) {
            __threadfence();
            atomicExch(&t.meta[slot], meta);
        }
    } else if (state == 2) {
        unsigned m = 0;
        if (lane == 0) {
            // the storing warp writes its rows and then the meta word; it waits on
            // nothing, so this bounded wait ends long before its limit
            for (int it = 0; it < SHAPE_WAIT && m == 0; ++it) {
                m = atomicOr(&t.meta[slot], 0u);
                if (m == 0) __nanosleep(64);
            }
        }
        if (lane == 0) __threadfence();  // the rows are read after the meta word was seen
        m = __shfl_sync(FULL, m, 0);
        if (m == 0) {
            if (lane == 0) atomicAdd(&t.stats[1], 1u);
        } else {
            const uint32_t have = __ldcg(&t.rows[(size_t)slot * 32 + lane]);
            if (__any_sync(FULL, m != meta || have != mine) && lane == 0) atomicAdd(&t.stats[0], 1u);
        }
    } else if (lane == 0) {
        atomicAdd(&t.stats[2], 1u);
    }
    __syncwarp();
}

// ---------------------------------------------------------------------------
// warp-cooperative canonical form + hash of owner o's replicate-0 shape
// ---------------------------------------------------------------------------
// canonical form + hash of a cropped shape held in lanes: lane i < h holds row
// i of the h x w crop (bit j = column j), the other lanes 0
__device__ __forceinline__ uint32_t crop_shape_hash(uint32_t r, int h, int w, int lane, bool c4, const ShapeTab &tab)
{
    uint32_t col = 0;  // lane j < w: column j, bit i = cell (x0 + j, y0 + i)
    for (int j = 0; j < w; ++j) {
        const uint32_t bj = __ballot_sync(FULL, (r >> j) & 1u);
        if (lane == j) col = bj;
    }
    const uint32_t rrev = __shfl_sync(FULL, r, (h - 1 - lane) & 31);
    const uint32_t crev = __shfl_sync(FULL, col, (w - 1 - lane) & 31);
    // the 8 images, each as rows whose first cell is the most significant bit
    uint32_t v[8];
    v[0] = __brev(r) >> (32 - w);     // identity
    v[1] = r;                         // mirror x
    v[2] = __brev(rrev) >> (32 - w);  // mirror y
    v[3] = rrev;                      // half turn
    v[4] = __brev(col) >> (32 - h);   // transpose
    v[5] = col;                       // quarter turn
    v[6] = __brev(crev) >> (32 - h);  // quarter turn the other way
    v[7] = crev;                      // anti-transpose
    // smallest (height, width) first: rows-images have (h, w), column-images (w, h)
    const int start = (h <= w) ? 0 : 4;
    const int stop = (h >= w) ? 8 : 4;
    const int hc = (start == 0) ? h : w;
    const int wc = (start == 0) ? w : h;
    uint32_t best = v[start];
#pragma unroll
    for (int t = 1; t < 8; ++t) {
        if (t > start && t < stop) {
            const uint32_t diff = __ballot_sync(FULL, lane < hc && v[t] != best);
            if (diff) {
                const int f = __ffs(diff) - 1;
                const uint32_t a = __shfl_sync(FULL, v[t], f);
                const uint32_t b = __shfl_sync(FULL, best, f);
                if (a < b) best = v[t];
            }
        }
    }
    if (c4) {
        // the rotation-only variant of Section 2.5: the images under the four
        // rotations (identity, half turn, and the two quarter turns), each
        // hashed, sorted, and hashed again
        const uint32_t h0 = image_hash(v[0], h, w), h3 = image_hash(v[3], h, w);
        const uint32_t h5 = image_hash(v[5], w, h), h6 = image_hash(v[6], w, h);
        return c4_combine(h0, h3, h5, h6);
    }
    const uint32_t hv = image_hash(best, hc, wc);
    if (tab.key) shape_record(tab, hv, best, hc, wc, lane);
    return hv;
}

// the crop of a form the crop table does not hold, appended to the call's spill list
__device__ __forceinline__ void spill_crop(const CropSpill &sp, uint32_t r, int h, int w, int lane)
{
    unsigned long long idx = 0;
    if (lane == 0) idx = atomicAdd(sp.count, 1ull);
    idx = __shfl_sync(FULL, idx, 0);
    if (idx < sp.cap) {
        sp.rows[idx * 32 + lane] = lane < h ? r : 0u;
        if (lane == 0) sp.meta[idx] = ((unsigned)h << 8) | (unsigned)w;
    }
}

template <int S>
__device__ __forceinline__ uint32_t coop_shape_hash(int o, const uint32_t *warp_lanes, const Lane &Ls, int lane,
                                                    bool c4, bool spill, const CropSpill &sp)
{
    using G = Geo<S>;
    const int x0 = __shfl_sync(FULL, Ls.x0, o), x1 = __shfl_sync(FULL, Ls.x1, o);
    const int y0 = __shfl_sync(FULL, Ls.y0, o), y1 = __shfl_sync(FULL, Ls.y1, o);
    const int h = y1 - y0 + 1, w = x1 - x0 + 1;
    const uint32_t wmask = (w >= 32) ? FULL : ((1u << w) - 1u);
    uint32_t r = 0;  // lane i < h: row i of the crop, bit j = cell (x0 + j, y0 + i)
    if (lane < h) {
        const int b = (y0 + lane) * S + x0;
        r = (warp_lanes[(G::OCCA + (b >> 5)) * 32 + o] >> (b & 31)) & wmask;
    }
    if (spill) spill_crop(sp, r, h, w, lane);
    return crop_shape_hash(r, h, w, lane, c4, ShapeTab{});
}

// W: the unsigned type that holds the colours (32 bits for at most two tiles).
template <typename W>
__device__ __forceinline__ int seed_outcome_w(W cols, int n, int c, int L)
{
    constexpr int BITS = 8 * (int)sizeof(W);
    const W ones = (W)0x1111111111111111ull;
    const W valid = (16 * n >= BITS) ? ~(W)0 : (W)(((W)1 << (16 * n)) - (W)1);
    const int cx = L >> 1;
    bool nd = false, unb = false;
    int sites = 0;
#pragma unroll
    for (int d = 0; d < 4; ++d) {
        const int a = (int)((cols >> (4 * d)) & 15u);
        const int pa = (a == 0) ? -1 : (a & 1) ? ((a + 1 < c) ? a + 1 : -1) : a - 1;
        if (pa < 0) continue;
        const W x = cols ^ ((W)pa * ones);
        const W nz = (x | (x >> 1) | (x >> 2) | (x >> 3)) & ones;
        W eq = ~nz & ones & valid;  // bit 4 m set: edge m carries colour pa
        if (!eq) continue;
        const int e = (d + 2) & 3;  // the candidate's side that faces the seed
        uint32_t first = 0xFFFFFFFFu;
        bool multi = false;
        while (eq) {
            const int m = ((BITS == 32 ? __ffs((int)eq) : __ffsll((long long)eq)) - 1) >> 2;
            eq &= eq - 1;
            const int t = m >> 2, i = m & 3;
            const uint32_t tile = (uint32_t)(cols >> (16 * t)) & 0xFFFFu;
            const int r = (e - i) & 3;  // turn that brings edge i to side e
            const uint32_t tup = ((tile << (4 * r)) | (tile >> (16 - 4 * r))) & 0xFFFFu;
            if (first == 0xFFFFFFFFu) first = tup;
            else if (tup != first) multi = true;
        }
        const int qx = cx + (d == 1) - (d == 3), qy = cx + (d == 2) - (d == 0);
        const bool inside = qx >= 0 && qy >= 0 && qx < L && qy < L;
        if (multi) nd = true;
        else if (!inside) unb = true;
        ++sites;
    }
    if (nd) return JATAM_ND_LOCAL;
    if (unb) return JATAM_UNBOUNDED;
    return -sites;
}

// The seed step of replicate 0 for sets of at most two tiles, branch-free: the
// candidates of side d of the seed are the representative tuples whose side
// d + 2 carries the partner of the seed's colour on side d, read from the bit
// planes of the binding tables (lane_tables), kept here with tile 1's rotations
// at bits 16..19; two or more is local ambiguity.  Same returns as seed_outcome_w.
__device__ __forceinline__ int seed_outcome_two(uint32_t cols, int n, int c, int L)
{
    const uint32_t t0 = cols & 0xFFFFu, t1 = cols >> 16;
    uint32_t reps = 1u | (rot16(t0, 4) != t0 ? 2u : 0u) | (rot16(t0, 8) != t0 ? 12u : 0u);
    if (n == 2) {
        uint32_t m = 1u | (rot16(t1, 4) != t1 ? 2u : 0u) | (rot16(t1, 8) != t1 ? 12u : 0u);
        if (t1 == t0 || t1 == rot16(t0, 4) || t1 == rot16(t0, 8) || t1 == rot16(t0, 12)) m = 0u;
        reps |= m << 16;
    }
    const int cx = L >> 1;
    bool nd = false, unb = false;
    int sites = 0;
#pragma unroll
    for (int d = 0; d < 4; ++d) {
        const int a = (int)((t0 >> (4 * d)) & 15u);
        const int pa = (a == 0) ? -1 : (a & 1) ? ((a + 1 < c) ? a + 1 : -1) : a - 1;
        const uint32_t n0 = 0u - (uint32_t)(pa & 1), n1 = 0u - (uint32_t)((pa >> 1) & 1),
                       n2 = 0u - (uint32_t)((pa >> 2) & 1);
        uint32_t X = pa >= 0 ? reps : 0u;
#pragma unroll
        for (int b = 0; b < 3; ++b) {
            const uint32_t x = (cols >> b) & 0x11111111u;
            const uint32_t P = (d == 0) ? plane_spread<2>(x) : (d == 1) ? plane_spread<3>(x)
                             : (d == 2) ? plane_spread<0>(x) : plane_spread<1>(x);  // side d + 2
            X &= ~(P ^ (b == 0 ? n0 : b == 1 ? n1 : n2));
        }
        if (X) {
            const int qx = cx + (d == 1) - (d == 3), qy = cx + (d == 2) - (d == 0);
            const bool inside = qx >= 0 && qy >= 0 && qx < L && qy < L;
            if (X & (X - 1)) nd = true;
            else if (!inside) unb = true;
            ++sites;
        }
    }
    if (nd) return JATAM_ND_LOCAL;
    if (unb) return JATAM_UNBOUNDED;
    return -sites;
}

// The seed step of replicate 0, evaluated straight from the colours: for each
// side d of the seed (tile 0, orientation 0) the candidates are the rotated
// tuples whose side facing the seed has the partner colour of the seed's side
// d.  Returns 1 (local ambiguity), 3 (unbounded), 0 (terminated: nothing can
// attach, every replicate ends as the lone seed) or minus the number of
// frontier sites after the seed (the assembly grows).
__device__ __forceinline__ int seed_outcome(unsigned long long cols, int n, int c, int L)
{
    if (n <= 2 && c <= 8) return seed_outcome_two((uint32_t)cols, n, c, L);
    return seed_outcome_w<unsigned long long>(cols, n, c, L);
}

// Seed-step table of every tile of 3-bit colours, indexed by its packed value t
// (12 bits, edge i at bits 3 (3 - i): the genotype's own encoding of one tile).
// Word k, nibble v (v = 1 .. 7): bit r is set when t turned by r shows colour v on
// side k, i.e. edge (k - r) mod 4 of t has colour v.  Colour 0 binds nothing and
// its nibbles hold two other fields: word 0 the turns that give distinct tuples
// (bit 0; bit 1 unless a quarter turn leaves t unchanged; bits 2 and 3 unless a
// half turn does, as in lane_tables), words 1 to 3 the smallest packed value of
// the four turns of t, 4 bits each, lowest first (two tiles are turns of each
// other exactly when these agree).  Built by the compiler.
constexpr uint32_t seed_tile_colour(uint32_t t, int i) { return (t >> (3 * (3 - i))) & 7u; }
constexpr uint32_t seed_tile_turn(uint32_t t, int r)
{
    uint32_t v = 0;
    for (int j = 0; j < 4; ++j) v |= seed_tile_colour(t, (j + 4 - r) & 3) << (3 * (3 - j));
    return v;
}
struct __align__(16) SeedTab {
    uint32_t w[4096][4];
};
constexpr SeedTab make_seed_tab()
{
    SeedTab T{};
    for (uint32_t t = 0; t < 4096; ++t) {
        for (int k = 0; k < 4; ++k) {
            uint32_t word = 0;
            for (int r = 0; r < 4; ++r) word |= 1u << (4 * seed_tile_colour(t, (k + 4 - r) & 3) + r);
            T.w[t][k] = word & ~15u;
        }
        uint32_t low = t;
        for (int r = 1; r < 4; ++r) low = seed_tile_turn(t, r) < low ? seed_tile_turn(t, r) : low;
        T.w[t][0] |= 1u | (seed_tile_turn(t, 1) != t ? 2u : 0u) | (seed_tile_turn(t, 2) != t ? 12u : 0u);
        T.w[t][1] |= low & 15u;
        T.w[t][2] |= (low >> 4) & 15u;
        T.w[t][3] |= low >> 8;
    }
    return T;
}
__device__ constexpr SeedTab g_seed_tab = make_seed_tab();

// nibble a: the colour that binds colour a (Section 2.2: 1-2, 3-4, 5-6; 0 and an
// odd top colour bind nothing, 0 here), the rule of seed_outcome_two for c <= 8
__device__ __forceinline__ uint32_t partner_nibbles(int c)
{
    uint32_t p = 0;
#pragma unroll
    for (int a = 1; a < 8; ++a) {
        const int pa = (a & 1) ? ((a + 1 < c) ? a + 1 : 0) : a - 1;
        p |= (uint32_t)pa << (4 * a);
    }
    return p;
}

// The seed step of replicate 0 for one or two tiles of 3-bit colours, from the
// packed genotype g and the seed table: the same outcome as seed_outcome_two.
// For side d of the seed the candidates are the distinct tuples whose side d + 2
// carries the partner pa of the seed's colour there: nibble pa of word d + 2 of
// each tile's entry, restricted to the tile's distinct turns (and to none of
// tile 1's when it is a turn of tile 0).
__device__ __forceinline__ int seed_outcome_tab(unsigned long long g, int n, uint32_t partner, int L)
{
    const uint4 *tab = reinterpret_cast<const uint4 *>(g_seed_tab.w);
    const uint32_t t0 = (uint32_t)(n == 2 ? g >> 12 : g) & 0xFFFu;
    const uint4 E0 = __ldg(tab + t0);
    uint4 E1 = make_uint4(0u, 0u, 0u, 0u);
    uint32_t reps1 = 0u;
    if (n == 2) {
        E1 = __ldg(tab + ((uint32_t)g & 0xFFFu));
        const bool turned = ((E0.y ^ E1.y) & 15u) == 0u && ((E0.z ^ E1.z) & 15u) == 0u && ((E0.w ^ E1.w) & 15u) == 0u;
        reps1 = turned ? 0u : (E1.x & 15u);
    }
    const uint32_t reps0 = E0.x & 15u;
    const int cx = L >> 1;
    bool nd = false, unb = false;
    int sites = 0;
#pragma unroll
    for (int d = 0; d < 4; ++d) {
        const uint32_t pa = (partner >> (4 * ((t0 >> (3 * (3 - d))) & 7u))) & 15u;
        const int k = (d + 2) & 3;
        const uint32_t w0 = k == 0 ? E0.x : k == 1 ? E0.y : k == 2 ? E0.z : E0.w;
        const uint32_t w1 = k == 0 ? E1.x : k == 1 ? E1.y : k == 2 ? E1.z : E1.w;
        const uint32_t X = pa ? (((w0 >> (4 * pa)) & reps0) | (((w1 >> (4 * pa)) & reps1) << 4)) : 0u;
        if (X) {
            const int qx = cx + (d == 1) - (d == 3), qy = cx + (d == 2) - (d == 0);
            const bool inside = qx >= 0 && qy >= 0 && qx < L && qy < L;
            if (X & (X - 1)) nd = true;
            else if (!inside) unb = true;
            ++sites;
        }
    }
    if (nd) return JATAM_ND_LOCAL;
    if (unb) return JATAM_UNBOUNDED;
    return -sites;
}

// The replicate just ended (local ambiguity, unbounded growth, or an empty
// frontier): apply the first-deciding-replicate rule.
// ---------------------------------------------------------------------------
// Dominance certificate of a final replicate-0 configuration A0 that is not
// closed (warp-wide job for lane o).  Attachment graph on the cells of A0:
// u -> v (adjacent) when u offers v's tuple of A0 to v.  A bad offer is one
// from u to an adjacent cell q of A0 (q not the seed's cell) that contains a
// tuple other than q's own.  If for every bad offer u -> q every path of the
// graph from the seed to u passes through q, all k replicates end in A0:
// before any deviation from A0 each placed cell v was attached through a
// neighbour u -> v placed earlier, so cells are placed in an order that
// respects the graph, u is placed after q, and no empty cell ever sees a
// tuple other than its own in A0 (cells outside A0 receive no offers: replicate
// 0 ended with an empty frontier); every cell of A0 is reachable, so each
// replicate fills A0 and stops.  Lane i holds row y0 + i of A0's bounding
// box (bit j: column x0 + j); once per distinct q, the cells with a path to
// q's bad offerers that avoids q are flood-filled against the edges, and the
// test fails if the seed is among them.
// ---------------------------------------------------------------------------
template <int S, int NT>
__device__ __forceinline__ bool coop_dominated(int o, const uint32_t *warp_lanes, const Lane &Ls, int lane)
{
    using G = Geo<S>;
    const uint32_t *ob = warp_lanes + o;
    const int x0 = __shfl_sync(FULL, Ls.x0, o), x1 = __shfl_sync(FULL, Ls.x1, o);
    const int y0 = __shfl_sync(FULL, Ls.y0, o), y1 = __shfl_sync(FULL, Ls.y1, o);
    const int Lo = __shfl_sync(FULL, Ls.L, o);
    const int h = y1 - y0 + 1, w = x1 - x0 + 1;
    const uint32_t wmask = (w >= 32) ? FULL : ((1u << w) - 1u);
    // the owner's binding table, word j in lane j
    const uint32_t nbm = (lane < 2 * NT) ? ob[(G::NBM + lane) * 32] : 0u;
    uint32_t occ = 0;
    if (lane < h) {
        const int b = (y0 + lane) * S + x0;
        occ = (ob[(G::OCCA + (b >> 5)) * 32] >> (b & 31)) & wmask;
    }
    uint32_t occN = __shfl_up_sync(FULL, occ, 1), occS = __shfl_down_sync(FULL, occ, 1);
    if (lane == 0) occN = 0u;
    if (lane == 31) occS = 0u;
    const int sx = (Lo >> 1) - x0, sy = (Lo >> 1) - y0;
    // tuple id of column j of this lane's row (0 outside the box)
    auto tuple_at = [&](int j) -> int {
        if (lane >= h || j >= w) return 0;
        const int b = (y0 + lane) * S + x0 + j;
        return (int)((ob[(G::NIB + (b >> 3)) * 32] >> ((b & 7) * 4)) & 15u);
    };
    uint32_t gN = 0, gE = 0, gS = 0, gW = 0;  // good edges: cell -> its neighbour on that side
    uint32_t bN = 0, bE = 0, bS = 0, bW = 0;  // bad offers: cell -> its neighbour on that side
    int tW = 0, tC = tuple_at(0);
    for (int j = 0; j < w; ++j) {
        const int tE = tuple_at(j + 1);
        const int tN = __shfl_up_sync(FULL, tC, 1), tS = __shfl_down_sync(FULL, tC, 1);
        const uint32_t m01 = __shfl_sync(FULL, nbm, (2 * tC) & 31);
        const uint32_t m23 = __shfl_sync(FULL, nbm, (2 * tC + 1) & 31);
        if ((occ >> j) & 1u) {
            const uint32_t bit = 1u << j;
            const uint32_t MN = m01 & 0xFFFFu, ME = m01 >> 16, MS = m23 & 0xFFFFu, MW = m23 >> 16;
            if ((occN >> j) & 1u) {
                if ((MN >> tN) & 1u) gN |= bit;
                if ((MN & ~(1u << tN)) && !(lane - 1 == sy && j == sx)) bN |= bit;
            }
            if (j + 1 < w && ((occ >> (j + 1)) & 1u)) {
                if ((ME >> tE) & 1u) gE |= bit;
                if ((ME & ~(1u << tE)) && !(lane == sy && j + 1 == sx)) bE |= bit;
            }
            if ((occS >> j) & 1u) {
                if ((MS >> tS) & 1u) gS |= bit;
                if ((MS & ~(1u << tS)) && !(lane + 1 == sy && j == sx)) bS |= bit;
            }
            if (j > 0 && ((occ >> (j - 1)) & 1u)) {
                if ((MW >> tW) & 1u) gW |= bit;
                if ((MW & ~(1u << tW)) && !(lane == sy && j - 1 == sx)) bW |= bit;
            }
        }
        tW = tC;
        tC = tE;
    }
    // cells that receive a bad offer
    const uint32_t fromAbove = __shfl_up_sync(FULL, bS, 1), fromBelow = __shfl_down_sync(FULL, bN, 1);
    uint32_t qs = (bE << 1) | (bW >> 1) | (lane > 0 ? fromAbove : 0u) | (lane < 31 ? fromBelow : 0u);
    qs &= occ;
    const bool seed_row = lane == sy;
    const uint32_t seed_bit = seed_row ? (1u << sx) : 0u;
    for (;;) {
        const unsigned hasq = __ballot_sync(FULL, qs != 0u);
        if (!hasq) return true;
        const int qy = __ffs(hasq) - 1;
        const int qx = __ffs(__shfl_sync(FULL, qs, qy)) - 1;
        if (lane == qy) qs &= ~(1u << qx);
        const uint32_t keep = occ & ((lane == qy) ? ~(1u << qx) : FULL);
        // the bad offerers of q: its north neighbour offering south, its south
        // neighbour offering north, its east one offering west, its west one east
        uint32_t X = 0u;
        if (lane == qy - 1) X = bS & (1u << qx);
        if (lane == qy + 1) X = bN & (1u << qx);
        if (lane == qy) X = (bW & ((qx + 1 < 32) ? (2u << qx) : 0u)) | (bE & ((qx > 0) ? (1u << (qx - 1)) : 0u));
        // every cell with a path to one of them that avoids q, one
        // breadth-first layer at a time against the edges: the seed among them
        // means an offerer can be placed before q
        for (;;) {
            if (__any_sync(FULL, (X & seed_bit) != 0u)) return false;
            const uint32_t below = __shfl_down_sync(FULL, X, 1);  // row below: this row's cells attach south
            const uint32_t above = __shfl_up_sync(FULL, X, 1);    // row above: this row's cells attach north
            uint32_t nX = X | (gE & (X >> 1)) | (gW & (X << 1)) | (lane < 31 ? (gS & below) : 0u) |
                          (lane > 0 ? (gN & above) : 0u);
            nX &= keep;
            if (!__any_sync(FULL, nX != X)) break;
            X = nX;
        }
    }
}

template <int S>
__device__ __forceinline__ void replicate_end(Lane &Ls, uint32_t *my, bool nd, bool unb)
{
    using G = Geo<S>;
    if (nd) {
        Ls.cls = JATAM_ND_LOCAL;
        Ls.decided = Ls.rep;
        Ls.phase = PH_WRITE;
        return;
    }
    if (unb) {
        Ls.cls = JATAM_UNBOUNDED;
        Ls.decided = Ls.rep;
        Ls.phase = PH_WRITE;
        return;
    }
    if (Ls.rep == 0) {
        Ls.size0 = Ls.size;
        Ls.x0 = Ls.xmin;
        Ls.x1 = Ls.xmax;
        Ls.y0 = Ls.ymin;
        Ls.y1 = Ls.ymax;
        if (Ls.forced || Ls.cert) {
            // The outcome of every later replicate is fixed: either every draw
            // of replicate 0 had a single frontier site, so every replicate
            // follows the same path; or the final configuration A0 is closed:
            // for every two adjacent tiles of A0, what either one offers the
            // other's cell is that cell's tuple or nothing (offers to the seed's
            // cell aside: the seed is always there first), and replicate 0
            // ended with no candidate outside A0.  Then, in any order, every
            // empty site a replicate can reach receives only A0's tuple there,
            // no site ever sees two distinct candidates, nothing attaches
            // outside A0, and the frontier empties only when all of A0
            // (connected through its bonds) is placed: all k replicates end in A0.
            Ls.cls = JATAM_DET_BOUNDED;
            Ls.decided = Ls.k;
            Ls.phase = PH_SHAPE;
            return;
        }
        if (Ls.k > 1) {
            // A0 is not closed: the warp tests whether every offending offer
            // comes too late in every order (coop_dominated)
            Ls.phase = PH_DOM;
            return;
        }
    } else if (Ls.diverged || Ls.size != Ls.size0) {
        Ls.cls = JATAM_ND_STERIC;
        Ls.decided = Ls.rep;
        Ls.phase = PH_SHAPE;
        return;
    }
    if (Ls.rep + 1 >= Ls.k) {
        Ls.cls = JATAM_DET_BOUNDED;
        Ls.decided = Ls.k;
        Ls.phase = PH_SHAPE;
    } else {
        // next replicate: its occupancy starts empty (the frontier of a
        // terminated replicate is already empty)
        if (Ls.blo <= Ls.bhi) clear_rows<S>(my, G::OCCB, Ls.blo, Ls.bhi);
        Ls.blo = S;
        Ls.bhi = -1;
        Ls.rep += 1;
        Ls.phase = PH_START;
    }
}

// a replicate lane's replicate has ended: local ambiguity, unbounded growth, or
// (recorded as DET_BOUNDED) an empty frontier in a configuration the warp then
// compares with replicate 0's
__device__ __forceinline__ void replicate_end_par(Lane &Ls, bool nd, bool unb)
{
    Ls.cls = nd ? JATAM_ND_LOCAL : unb ? JATAM_UNBOUNDED : JATAM_DET_BOUNDED;
    Ls.phase = PH_DONE;
}

// ---------------------------------------------------------------------------
// one growth step of one lane: seed placement or one drawn placement, then the
// evaluation of the new tile's empty neighbours and the replicate rule
// ---------------------------------------------------------------------------
// the Philox word of draw index s: the fetch-ahead has put its block in pa or pb
__device__ __forceinline__ bool current_word(Lane &Ls, uint32_t s, uint32_t &u)
{
    const uint32_t key = (uint32_t)Ls.rep * 512u + (s >> 2);
    if (Ls.ka != key) {
        if (Ls.kb != key) return false;
        Ls.pa = Ls.pb;
        Ls.kb = NO_BLOCK;
        Ls.ka = key;
    }
    const int sel = s & 3;
    u = sel == 0 ? Ls.pa.x : sel == 1 ? Ls.pa.y : sel == 2 ? Ls.pa.z : Ls.pa.w;
    return true;
}

// LIFO: the movelist process; stk: this lane's stack (S * S cells, global memory).
// PAR: replicate lanes -- the lane grows replicate Ls.rep alone on its own lattice
// (occupancy in OCCA, no comparison with replicate 0 while it grows, no
// certificates) and only records how it ended (replicate_end_par)
template <int S, bool LIFO, bool PAR = false>
__device__ __forceinline__ void lane_step(Lane &Ls, uint32_t *my, uint32_t k0, uint32_t k1, unsigned *err,
                                          uint16_t *stk)
{
    // Called by all 32 lanes; lanes that are not growing do the arithmetic on
    // harmless addresses of their own region and write nothing.  __syncwarp()
    // brings the warp back together after each data-dependent part.
    using G = Geo<S>;
    const bool active = Ls.phase == PH_START || Ls.phase == PH_GROW;
    const bool seed = Ls.phase == PH_START;
    const int occ = (PAR || Ls.rep == 0) ? G::OCCA : G::OCCB;
    int b = 0, tau = 0;
    bool placing = active;
    if (LIFO && active && !seed) {
        // the movelist process: the site on top of the stack
        if (Ls.sp < 1 || Ls.sp > S * S) {
            atomicOr(err, ERR_GUARD);  // unreachable: the stack holds the frontier, which is not empty here
            Ls.cls = 255;
            Ls.phase = PH_WRITE;
            placing = false;
        } else {
            Ls.sp -= 1;
            b = stk[Ls.sp];
            tau = nib_get<S>(my, b);
            my[(G::FRONT + (b >> 5)) * 32] &= ~(1u << (b & 31));
            Ls.nF -= 1;
            Ls.step += 1;
        }
    } else if (active && !seed) {
        // the growth loop's batched fetch-ahead has computed this block (in pa,
        // or in pb when it was fetched as the next replicate's first block)
        const uint32_t key = (uint32_t)Ls.rep * 512u + ((uint32_t)Ls.step >> 2);
        if (Ls.ka != key) {
            if (Ls.kb == key) {
                Ls.pa = Ls.pb;
                Ls.kb = NO_BLOCK;
                Ls.ka = key;
            } else {
                atomicOr(err, ERR_GUARD);  // unreachable: the fetch-ahead supplies every current block
                Ls.cls = 255;
                Ls.phase = PH_WRITE;
                placing = false;
            }
        }
        if (Ls.nF > 1) Ls.forced = 0;
        const int sel = Ls.step & 3;
        const uint32_t u = sel == 0 ? Ls.pa.x : sel == 1 ? Ls.pa.y : sel == 2 ? Ls.pa.z : Ls.pa.w;
        // rank i of the chosen site among the frontier sites in row-major order
        uint32_t i = placing ? __umulhi(u, (uint32_t)Ls.nF) : 0u;
        int w;
        uint32_t f;
        if constexpr (G::NW <= 8) {
            // the word holding it, from the packed per-word site counts: byte j
            // of P is the number of sites in words 0..j (at most L * L - 1 <=
            // 255, so the bytes never carry)
            const unsigned long long P = Ls.fc * 0x0101010101010101ull;
            const uint32_t ii = i * 0x01010101u;
            w = (__popc(__vcmpleu4((uint32_t)P, ii)) + __popc(__vcmpleu4((uint32_t)(P >> 32), ii))) >> 3;
            if (w > 0) i -= (uint32_t)(P >> (8 * (w - 1))) & 255u;
            f = my[(G::FRONT + min(w, G::NW - 1)) * 32];
        } else {
            w = (max(Ls.ymin - 1, 0) * S) >> 5;
            f = my[(G::FRONT + w) * 32];
            uint32_t cnt = placing ? __popc(f) : 1u;
            while (i >= cnt) {
                i -= cnt;
                if (++w >= G::NW) break;
                f = my[(G::FRONT + w) * 32];
                cnt = __popc(f);
            }
        }
        if (!placing) {
        } else if (w >= G::NW || i >= (uint32_t)__popc(f)) {
            atomicOr(err, ERR_GUARD);
            Ls.cls = 255;
            Ls.phase = PH_WRITE;
            placing = false;
        } else {
            const int bit = nth_set(f, i);
            b = w * 32 + bit;
            tau = nib_get<S>(my, b);
            my[(G::FRONT + w) * 32] = f & ~(1u << bit);
            if constexpr (G::NW <= 8) Ls.fc -= 1ull << (8 * w);
            Ls.nF -= 1;
            Ls.step += 1;
        }
    }
    if (seed) {
        // a new replicate: the seed, tile 0 in orientation 0, at the centre
        b = (Ls.L >> 1) * S + (Ls.L >> 1);
        tau = 0;
        Ls.size = 0;
        Ls.step = 0;
        Ls.nF = 0;
        Ls.fc = 0ull;
        Ls.sp = 0;
        Ls.diverged = 0;
        Ls.forced = 1;
        Ls.cert = 1;
        Ls.phase = PH_GROW;
    }
    __syncwarp();
    const int px = b & (S - 1), py = b >> G::LOG2S;

    // the placed cell's occupancy and frontier words: the east and west
    // neighbours of an in-grid cell always lie in the same words (a row never
    // straddles two), so their sides below read their own bits from these
    // instead of loading again (bits of other cells may be stale: no store
    // below is built from them)
    const uint32_t ow_b = my[(occ + (b >> 5)) * 32];
    const uint32_t fw_b = my[(G::FRONT + (b >> 5)) * 32];
    if (placing) {
        my[(occ + (b >> 5)) * 32] = ow_b | (1u << (b & 31));
        if (seed && (PAR || Ls.rep == 0)) nib_set<S>(my, b, 0);
        Ls.size += 1;
        Ls.ymin = seed ? py : min(Ls.ymin, py);
        Ls.ymax = seed ? py : max(Ls.ymax, py);
        Ls.xmin = seed ? px : min(Ls.xmin, px);
        Ls.xmax = seed ? px : max(Ls.xmax, px);
        Ls.dlo = min(Ls.dlo, py - 1);
        Ls.dhi = max(Ls.dhi, py + 1);
        if (!PAR && Ls.rep > 0) {
            Ls.blo = min(Ls.blo, py);
            Ls.bhi = max(Ls.bhi, py);
        }
    }

    // the empty neighbours of the new tile: only their candidate sets changed.
    // Straight-line code: every lane evaluates all four sides, whatever their
    // case, so the warp stays converged.
    const uint32_t m01 = my[(G::NBM + 2 * tau) * 32];
    const uint32_t m23 = my[(G::NBM + 2 * tau + 1) * 32];
    const int seed_cell = (Ls.L >> 1) * S + (Ls.L >> 1);
    bool nd = false, unb = false;
    unsigned long long newq = 0;  // movelist: the new frontier sites of this step, N, E, S, W, 16 bits each
    int nnew = 0;
#pragma unroll
    for (int d = 0; d < 4; ++d) {
        const uint32_t M = ((d == 0) ? m01 : (d == 1) ? (m01 >> 16) : (d == 2) ? m23 : (m23 >> 16)) & 0xFFFFu;
        const int qx = px + (d == 1) - (d == 3);
        const int qy = py + (d == 2) - (d == 0);
        const bool in = (unsigned)qx < (unsigned)Ls.L && (unsigned)qy < (unsigned)Ls.L;
        const int qb = in ? qy * S + qx : b;  // outside the grid: read the new tile's own cell, write nothing
        const int qw = qb >> 5;
        const uint32_t qbit = 1u << (qb & 31);
        const int sh = (qb & 7) * 4;
        const bool row = d == 1 || d == 3;  // east or west: the placed cell's words
        const uint32_t ow = row ? ow_b : my[(occ + qw) * 32];
        const uint32_t fw = row ? fw_b : my[(G::FRONT + qw) * 32];
        const uint32_t nw = my[(G::NIB + (qb >> 3)) * 32];
        const int tq = (nw >> sh) & 15;
        const bool empty = in && !(ow & qbit);
        const bool isf = (fw & qbit) != 0;
        const bool multi = (M & (M - 1)) != 0;
        // two distinct candidates at one site (inside or outside the grid), or a
        // frontier site whose single candidate is contradicted
        nd = nd || (!in && multi) || (empty && (isf ? (M & ~(1u << tq)) != 0 : multi));
        // one candidate outside the grid: growth past the cap
        unb = unb || (!in && M != 0 && !multi);
        // replicate 0: an occupied neighbour that could receive from the new
        // tile a tuple other than its own breaks the closure of the final
        // shape -- unless it is the seed, which every replicate places first
        if (!PAR && placing && Ls.rep == 0 && in && (ow & qbit) && (M & ~(1u << tq)) != 0 && qb != seed_cell) Ls.cert = 0;
        if (placing && empty && !isf && M != 0 && !multi) {
            const int tn = __ffs(M) - 1;
            // replicate 0 must hold the same tuple here, or this replicate can
            // no longer end in replicate 0's configuration
            if (!PAR && Ls.rep > 0 && !Ls.diverged && (!(my[(G::OCCA + qw) * 32] & qbit) || tq != tn)) Ls.diverged = 1;
            my[(G::NIB + (qb >> 3)) * 32] = (nw & ~(15u << sh)) | ((uint32_t)tn << sh);
            // a fresh read: an earlier side of this step may have set a bit of the same word
            my[(G::FRONT + qw) * 32] |= qbit;
            if constexpr (G::NW <= 8) Ls.fc += 1ull << (8 * qw);
            Ls.nF += 1;
            newq |= (unsigned long long)qb << (16 * nnew);
            ++nnew;
        }
    }
    if (LIFO && placing && !nd && !unb && nnew > 0) {
        // push the new sites in the drawn order: permutation floor(u m! / 2^32)
        // of the m sites in the factorial number system, the first pick first
        uint32_t u = 0;
        if (!current_word(Ls, (uint32_t)Ls.step, u)) {
            atomicOr(err, ERR_GUARD);  // unreachable: the fetch-ahead supplies the block of this push
            Ls.cls = 255;
            Ls.phase = PH_WRITE;
            placing = false;
        } else {
            if (nnew > 1) Ls.forced = 0;
            const uint32_t fact = nnew == 4 ? 24u : nnew == 3 ? 6u : nnew == 2 ? 2u : 1u;
            uint32_t idx = __umulhi(u, fact);
            uint32_t pool = 0x3210u;  // the sites not yet pushed, nibble j = site index
            for (int i = 0; i < nnew; ++i) {
                const int left = nnew - 1 - i;
                const uint32_t f = left == 3 ? 6u : left == 2 ? 2u : 1u;
                const uint32_t sel = idx / f;
                idx -= sel * f;
                const int item = (int)((pool >> (4 * sel)) & 15u);
                pool = (pool & ((1u << (4 * sel)) - 1u)) | ((pool >> (4 * sel + 4)) << (4 * sel));
                if (Ls.sp < S * S) stk[Ls.sp++] = (uint16_t)((newq >> (16 * item)) & 0xFFFFu);
                else atomicOr(err, ERR_GUARD);  // unreachable: at most S * S frontier sites
            }
        }
    }
    __syncwarp();
    if (placing && (nd || unb || Ls.nF == 0)) {
        if constexpr (PAR) replicate_end_par(Ls, nd, unb);
        else replicate_end<S>(Ls, my, nd, unb);
    }
    __syncwarp();
}

__device__ __forceinline__ unsigned table_slot(unsigned long long key, unsigned log2cap)
{
    return (unsigned)((key * 0x9E3779B97F4A7C15ull) >> (64 - log2cap));
}

__device__ void table_insert(const Table &T, unsigned long long key, unsigned long long cnt,
                             unsigned long long mid, unsigned smax, unsigned smin, unsigned *err)
{
    const unsigned cap = 1u << T.cap_log2;
    unsigned slot = table_slot(key, T.cap_log2);
    for (unsigned p = 0; p < cap; ++p) {
        const unsigned long long old = atomicCAS(&T.key[slot], EMPTY_KEY, key);
        if (old == EMPTY_KEY || old == key) {
            atomicAdd(&T.count[slot], cnt);
            atomicMin(&T.min_id[slot], mid);
            atomicMax(&T.size_max[slot], smax);
            atomicMin(&T.size_min[slot], smin);
            return;
        }
        slot = (slot + 1) & (cap - 1);
    }
    atomicOr(err, ERR_TABLE_FULL);
}

template <int SLOTS>
struct SmemHistT {
    static constexpr int slots = SLOTS;
    unsigned long long key[SLOTS];
    unsigned long long min_id[SLOTS];
    unsigned count[SLOTS];
    unsigned smax[SLOTS];
    unsigned smin[SLOTS];
};
using SmemHist = SmemHistT<HIST_SLOTS>;
// replicate lanes: small calls, few phenotypes, and a CTA's shared memory goes to more warps
using SmemHistSmall = SmemHistT<64>;

template <typename HT>
__device__ __forceinline__ void hist_insert(HT &H, const Table &T, unsigned long long key, unsigned cnt,
                                            unsigned long long id, unsigned smax, unsigned smin, unsigned *err)
{
    unsigned slot = table_slot(key, HT::slots == 256 ? 8 : HT::slots == 128 ? 7 : 6);
    for (int p = 0; p < 16; ++p) {
        const unsigned long long old = atomicCAS(&H.key[slot], EMPTY_KEY, key);
        if (old == EMPTY_KEY || old == key) {
            atomicAdd(&H.count[slot], cnt);
            atomicMin(&H.min_id[slot], id);
            atomicMax(&H.smax[slot], smax);
            atomicMin(&H.smin[slot], smin);
            return;
        }
        slot = (slot + 1) & (HT::slots - 1);
    }
    table_insert(T, key, cnt, id, smax, smin, err);
}

// decode a packed genotype into nibble-packed colours (tiles seed first,
// N, E, S, W, b bits per colour, the first tile's N edge most significant)
// UNROLLED: constant shifts for two tiles of 3-bit colours (the pre-filter,
// which unpacks every genotype of a call)
template <bool UNROLLED = false>
__device__ __forceinline__ unsigned long long unpack_genotype(unsigned long long g, int n, int b)
{
    if (UNROLLED && n == 2 && b == 3) {
        // two tiles of 3-bit colours: edge m = 4 t + e sits at bits 3 (7 - m)
        const uint32_t g32 = (uint32_t)g;
        uint32_t cols = 0;
#pragma unroll
        for (int m = 0; m < 8; ++m) cols |= ((g32 >> (3 * (7 - m))) & 7u) << (4 * m);
        return cols;
    }
    if (n <= 2) {
        // at most 8 colours of at most 4 bits: 32-bit arithmetic
        const uint32_t g32 = (uint32_t)g, cm = (1u << b) - 1u;
        uint32_t cols = 0;
        for (int m = 0; m < 4 * n; ++m) {
            const int pos = b * (4 * n - 1 - m);  // edge e of tile t is m = 4 t + e
            cols |= ((g32 >> pos) & cm) << (4 * m);
        }
        return cols;
    }
    unsigned long long cols = 0;
    const unsigned long long cm = (1ull << b) - 1ull;
    for (int t = 0; t < n; ++t)
        for (int e = 0; e < 4; ++e) {
            const int pos = b * (4 * (n - 1 - t) + (3 - e));
            cols |= ((g >> pos) & cm) << (4 * (4 * t + e));
        }
    return cols;
}

__device__ __forceinline__ int log2_colours(int c) { return c >= 8 ? 3 : c >= 4 ? 2 : c >= 2 ? 1 : 0; }

// The smallest packed genotype of g's orbit under the exact symmetries of the
// process: colour permutations that preserve the binding pairs (any pair to
// any pair, either order within a pair, the colours that bind nothing among
// themselves), turns of the non-seed tiles and permutations of them.  For each
// arrangement of the non-seed tiles the smallest relabelling is greedy: the
// colours, read in packed order (most significant first), get the smallest
// label still free in their class, a first-seen paired colour the odd label
// of the next free pair and its partner the even one.
__device__ __forceinline__ unsigned long long orbit_rep(unsigned long long g, int n, int c, int b)
{
    const unsigned long long cols = unpack_genotype(g, n, b);
    const int m = n - 1;
    const int nrot = 1 << (2 * m);
    const int nperm = (m <= 1) ? 1 : (m == 2) ? 2 : 6;
    const int top = (c % 2 == 0) ? c - 1 : -1;  // the top colour binds nothing when c is even
    unsigned long long best = g;
    for (int pk = 0; pk < nperm; ++pk) {
        // slot order of the non-seed tiles: permutation pk of 1 .. m
        int order[3] = {1, 2, 3};
        if (m == 2 && pk == 1) { order[0] = 2; order[1] = 1; }
        if (m == 3) {
            const int perms[6][3] = {{1, 2, 3}, {1, 3, 2}, {2, 1, 3}, {2, 3, 1}, {3, 1, 2}, {3, 2, 1}};
            order[0] = perms[pk][0]; order[1] = perms[pk][1]; order[2] = perms[pk][2];
        }
        for (int rk = 0; rk < nrot; ++rk) {
            uint32_t map = 0xFFFFFFFFu;  // nibble x: the label of colour x (15: none yet)
            int next_pair = 1, inert_seen = 0;
            unsigned long long v = 0;
            for (int pos = 0; pos < 4 * n; ++pos) {
                const int s = pos >> 2, e = pos & 3;
                int src;
                if (s == 0) {
                    src = e;
                } else {
                    const int r = (rk >> (2 * (s - 1))) & 3;
                    src = 4 * order[s - 1] + ((e - r) & 3);
                }
                const int x = (int)((cols >> (4 * src)) & 15u);
                int y = (int)((map >> (4 * x)) & 15u);
                if (y == 15) {
                    const bool inert = x == 0 || x == top;
                    if (inert) {
                        y = inert_seen == 0 ? 0 : top;
                        ++inert_seen;
                        map = (map & ~(15u << (4 * x))) | ((uint32_t)y << (4 * x));
                    } else {
                        const int partner = (x & 1) ? x + 1 : x - 1;
                        y = next_pair;
                        map = (map & ~(15u << (4 * x))) | ((uint32_t)next_pair << (4 * x));
                        map = (map & ~(15u << (4 * partner))) | ((uint32_t)(next_pair + 1) << (4 * partner));
                        next_pair += 2;
                    }
                }
                v = (v << b) | (unsigned long long)y;
            }
            best = v < best ? v : best;
        }
    }
    return best;
}

// One item of a launch: its colours (nibble-packed), size parameters and
// stream id.  ok is false for a record with a colour >= c or a parameter out
// of range (L must also fit the lattice template smax).
struct Item {
    unsigned long long sid, cols;
    int n, c, L, k;
    bool ok;
};

// COLS = false: the packed genotype only (it.cols is left 0; the pre-filter's table path)
template <bool UNROLLED = false, bool COLS = true>
__device__ __forceinline__ Item load_item(const LaunchArgs &a, unsigned long long idx, int b_uniform, int smax)
{
    Item it;
    it.n = a.n; it.c = a.c; it.L = a.L; it.k = a.k;
    it.ok = true;
    if (a.mode == MODE_RECORDS) {
        const uint4 raw = *reinterpret_cast<const uint4 *>(a.colours + 16ull * idx);
        if (a.shapes) {
            const uint32_t sh = *reinterpret_cast<const uint32_t *>(a.shapes + 4ull * idx);
            it.n = sh & 255; it.c = (sh >> 8) & 255; it.L = (sh >> 16) & 255; it.k = sh >> 24;
        }
        it.sid = a.ids ? a.ids[idx] : idx;
        unsigned long long cols = 0;
        bool ok = it.n >= 1 && it.n <= 4 && it.c >= 1 && it.c <= 8 && it.L >= 1 && it.L <= smax && it.k >= 1;
        const uint32_t wv[4] = {raw.x, raw.y, raw.z, raw.w};
#pragma unroll
        for (int e = 0; e < 16; ++e) {
            const int v = (wv[e >> 2] >> (8 * (e & 3))) & 255;
            if (e < 4 * it.n) {
                if (v >= it.c) ok = false;
                cols |= (unsigned long long)(v & 15) << (4 * e);
            }
        }
        it.cols = cols;
        it.ok = ok;
    } else {
        unsigned long long g;
        if (a.mode == MODE_RANGE) {
            g = a.first + idx;
        } else if (a.mode == MODE_GENOMES) {
            g = a.genomes[idx];
        } else {
            const unsigned long long i = a.first + idx;
            const uint4 w = philox4x32_10(make_uint4(0u, 1u << 24, (uint32_t)i, (uint32_t)(i >> 32)), a.key0, a.key1);
            g = ((unsigned long long)w.y << 32) | w.x;
        }
        const int bits = 4 * a.n * b_uniform;
        if (bits < 64) g &= (1ull << bits) - 1ull;
        it.sid = g;
        it.cols = COLS ? unpack_genotype<UNROLLED>(g, a.n, b_uniform) : 0ull;
    }
    return it;
}

__device__ __forceinline__ uint32_t monomer_shape_hash(bool c4)
{
    // the lone seed: a 1 x 1 crop with its cell at (0, 0), the same under every rotation
    const uint32_t h = oaat_finish(oaat_add(oaat_add(oaat_add(oaat_add(0u, 1u), 1u), 0u), 0u));
    return c4 ? c4_combine(h, h, h, h) : h;
}

__device__ __forceinline__ void write_result(const LaunchArgs &a, unsigned long long item, int cls, int decided,
                                             unsigned size, uint32_t hash)
{
    if (a.out) {
        const uint32_t w0 = (uint32_t)(cls & 255) | ((uint32_t)(decided & 255) << 8) | (size << 16);
        reinterpret_cast<uint2 *>(a.out)[item] = make_uint2(w0, hash);
    }
    if (a.fitness) a.fitness[item] = (cls == JATAM_DET_BOUNDED) ? (int32_t)size : 0;
}

// ---------------------------------------------------------------------------
// Pre-filter: one thread per item evaluates the seed step of replicate 0 (a
// lone seed, or local ambiguity / unboundedness right at the seed), writes the
// result of every item it decides, counts them into the histogram, and appends
// every other item to the list that the growth kernel consumes.
// ---------------------------------------------------------------------------
// genome deduplication: claim the genome's slot of the call's table (the claimer classifies it), or
// find it claimed and record the slot as a repeat's (the top bit set)
__device__ __forceinline__ bool genome_repeat(const LaunchArgs &a, unsigned long long g, unsigned long long idx)
{
    unsigned h = (unsigned)((g * 0x9E3779B97F4A7C15ull) >> 32) & a.dup_mask;
    for (unsigned p = 0; p <= a.dup_mask; ++p) {
        const unsigned long long old = atomicCAS(&a.dup_keys[h], ~0ull, g);
        if (old == ~0ull) {
            a.dup_owner[h] = (unsigned)idx;
            a.dup_slot[idx] = h;
            return false;
        }
        if (old == g) {
            a.dup_slot[idx] = h | 0x80000000u;
            return true;
        }
        h = (h + 1) & a.dup_mask;
    }
    atomicOr(a.err, ERR_GUARD);  // unreachable: the table holds at least 2 count slots
    return false;
}

constexpr int PF_ITEMS = 2;  // items per thread and iteration of the pre-filter (its barriers per item halve)

// TAB: genotypes (not records) of one or two tiles of 3-bit colours, whose seed
// step is read from the seed table (seed_outcome_tab); one lattice size class
template <bool TAB>
__global__ void __launch_bounds__(256, 5) prefilter_kernel(const LaunchArgs a, int smax)
{
    // keys decided here: 0 = (ND_LOCAL, 0), 1 = (UNBOUNDED, 0), 2 = (DET_BOUNDED, monomer)
    __shared__ unsigned s_cnt[3];
    __shared__ unsigned long long s_min[3];
    __shared__ unsigned s_fill[2][6];            // an iteration's items per list (two buffers, alternating)
    __shared__ unsigned long long s_base[6];     // where they go in the lists
    if (threadIdx.x < 3) {
        s_cnt[threadIdx.x] = 0u;
        s_min[threadIdx.x] = ~0ull;
    }
    if (threadIdx.x < 6) s_fill[0][threadIdx.x] = 0u;
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const int b_uniform = log2_colours(a.c);
    const uint32_t partner = TAB ? partner_nibbles(a.c) : 0u;
    const uint32_t mono = monomer_shape_hash(a.c4 != 0);
    const int nlists = 6;
    // this thread's decided items per key and their smallest stream ids (scalars: registers)
    unsigned hc0 = 0u, hc1 = 0u, hc2 = 0u;
    unsigned long long hm0 = ~0ull, hm1 = ~0ull, hm2 = ~0ull;
    const unsigned long long stride = (unsigned long long)gridDim.x * blockDim.x * PF_ITEMS;
    int buf = 0;
    for (unsigned long long base = (unsigned long long)blockIdx.x * blockDim.x * PF_ITEMS; base < a.count;
         base += stride, buf ^= 1) {
        int key[PF_ITEMS];
        bool grow[PF_ITEMS];
        int klass[PF_ITEMS];  // the list: size class (one class: 0) + 3 for a light item stored from the region's end
        unsigned long long sid[PF_ITEMS], idxs[PF_ITEMS];
#pragma unroll
        for (int u = 0; u < PF_ITEMS; ++u) {
            const unsigned long long idx = base + (unsigned long long)u * blockDim.x + threadIdx.x;
            idxs[u] = idx;
            key[u] = -1;
            grow[u] = false;
            klass[u] = 0;
            sid[u] = 0;
            if (idx < a.count) {
                const Item it = load_item<true, !TAB>(a, idx, b_uniform, smax);
                sid[u] = it.sid;
                if (a.bucket) klass[u] = (it.L <= 8) ? 0 : (it.L <= 16) ? 1 : 2;  // (+ 3 below for light items)
                if (!it.ok) {
                    atomicOr(a.err, ERR_INVALID_ITEM);
                    write_result(a, idx, 255, 0, 0u, 0u);
                } else if (a.orbits && orbit_rep(it.sid, it.n, it.c, b_uniform) != it.sid) {
                    // not its orbit's representative: the fill pass copies the representative's result
                } else if (a.dup_keys && genome_repeat(a, it.sid, idx)) {
                    // another item owns this genome (same genome, same stream id, same result): the fill
                    // pass copies its result
                } else {
                    const int so = TAB ? seed_outcome_tab(it.sid, it.n, partner, it.L)
                                       : seed_outcome(it.cols, it.n, it.c, it.L);
                    if (so < 0) {
                        grow[u] = true;
                        // two or more frontier sites after the seed: the genotypes that can
                        // run long (on uniform S_{2,8}, 57 % of those that grow, and every
                        // one of the slowest 1 % in a sample of 7,777); they are handed out
                        // first, so that the growth launch ends on genotypes with a single
                        // site, which finish soon (for calls large enough that every lane
                        // takes many genotypes: in a small call, warps given only heavy
                        // genotypes would set its length)
                        if (a.heavy_first && so > -2) klass[u] += 3;
                        else if (a.heavy_first == 2 && !a.bucket && so == -2) klass[u] = 1;  // the middle level
                    } else if (so == 0) {
                        write_result(a, idx, JATAM_DET_BOUNDED, it.k, 1u, mono);
                        key[u] = 2;
                    } else {
                        write_result(a, idx, so, 0, 0u, 0u);
                        key[u] = (so == JATAM_ND_LOCAL) ? 0 : 1;
                    }
                }
            }
        }
        // append to the list of the item's lattice size class (one class unless
        // the launch mixes sizes): warp offsets from shared counters, then one
        // global atomic per list and CTA iteration
        unsigned my_off[PF_ITEMS];
#pragma unroll
        for (int u = 0; u < PF_ITEMS; ++u) {
            my_off[u] = 0;
#pragma unroll
            for (int kc = 0; kc < nlists; ++kc) {
                // one size class: lists 0 and 3 (and 1, the middle level of a three-level order);
                // the table path has one class
                if (TAB ? (kc != 0 && kc != 3 && !(kc == 1 && a.heavy_first == 2))
                        : (!a.bucket && kc % 3 != 0 && !(kc == 1 && a.heavy_first == 2)))
                    continue;
                const unsigned gm = __ballot_sync(FULL, grow[u] && klass[u] == kc);
                unsigned woff = 0;
                if (gm && lane == 0) woff = atomicAdd(&s_fill[buf][kc], (unsigned)__popc(gm));
                woff = __shfl_sync(FULL, woff, 0);
                if (grow[u] && klass[u] == kc) my_off[u] = woff + __popc(gm & lanemask_lt());
            }
        }
        __syncthreads();
        if (threadIdx.x < nlists) {
            const unsigned f = s_fill[buf][threadIdx.x];
            if (f) s_base[threadIdx.x] = atomicAdd(&a.list_count[threadIdx.x], (unsigned long long)f);
            s_fill[buf ^ 1][threadIdx.x] = 0u;  // the next iteration's counters
        }
        __syncthreads();
#pragma unroll
        for (int u = 0; u < PF_ITEMS; ++u) {
            if (grow[u]) {
                // region klass % 3 of the list buffer: heavy items from its front, light ones from its end
                const unsigned long long pos = s_base[klass[u]] + my_off[u];
                const size_t region = (size_t)(klass[u] % 3) * a.list_stride;
                a.list[region + (klass[u] < 3 ? pos : a.list_stride - 1 - pos)] = idxs[u];
            }
        }
        if (a.use_hist) {
#pragma unroll
            for (int u = 0; u < PF_ITEMS; ++u) {
                const unsigned long long v = sid[u];
                if (key[u] == 0) {
                    hc0 += 1u;
                    hm0 = v < hm0 ? v : hm0;
                } else if (key[u] == 1) {
                    hc1 += 1u;
                    hm1 = v < hm1 ? v : hm1;
                } else if (key[u] == 2) {
                    hc2 += 1u;
                    hm2 = v < hm2 ? v : hm2;
                }
            }
        }
    }
    // the thread's counts and smallest stream ids, summed and reduced over the warp
    if (a.use_hist) {
        auto flush = [&](int q, unsigned hc, unsigned long long v) {
            const unsigned cnt = __reduce_add_sync(FULL, hc);
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) {
                const unsigned long long o = __shfl_xor_sync(FULL, v, off);
                v = o < v ? o : v;
            }
            if (lane == 0 && cnt) {
                atomicAdd(&s_cnt[q], cnt);
                atomicMin(&s_min[q], v);
            }
        };
        flush(0, hc0, hm0);
        flush(1, hc1, hm1);
        flush(2, hc2, hm2);
    }
    __syncthreads();
    if (a.use_hist && threadIdx.x < 3 && s_cnt[threadIdx.x]) {
        const int q = threadIdx.x;
        const unsigned long long key = (q == 0) ? ((unsigned long long)JATAM_ND_LOCAL << 32)
                                     : (q == 1) ? ((unsigned long long)JATAM_UNBOUNDED << 32)
                                                : (unsigned long long)mono;
        const unsigned sz = (q == 2) ? 1u : 0u;
        table_insert(a.table, key, s_cnt[q], s_min[q], sz, sz, a.err);
    }
}

// The work of one warp over one list of items (a pre-filter list): every
// lane takes items from the list through the shared counter `work_next` and
// the warp runs them to their class in batched phases.  `warp_lanes` is the
// warp's interleaved region of Geo<S, NT>::WORDS words per lane.
template <int S, int NT, bool LIFO>
__device__ __forceinline__ void warp_loop(const LaunchArgs &a, uint32_t *warp_lanes, SmemHist &H,
                                          const unsigned long long *list, unsigned long long front,
                                          unsigned long long back, unsigned long long *work_next,
                                          const unsigned long long *mid_list = nullptr,
                                          unsigned long long mid = 0)
{
    // items list[0 .. front) first, then mid_list[0 .. mid), then list[a.list_stride - 1],
    // list[a.list_stride - 2], ... (`back` of them): the pre-filter puts the longest-running
    // genotypes in front
    const unsigned long long total = front + mid + back;
    using G = Geo<S, NT>;
    const int lane = threadIdx.x & 31;
    uint32_t *my = warp_lanes + lane;
    for (int w = 0; w < 3 * G::NW; ++w) my[w * 32] = 0u;
    my[G::CACHE * 32] = 0u;  // key with h = 0: never matches a crop
    my[(G::CACHE + 1) * 32] = 0u;
    __syncwarp();

    Lane Ls;
    Ls.phase = PH_NEED;
    Ls.dlo = S;
    Ls.dhi = -1;
    Ls.blo = S;
    Ls.bhi = -1;
    Ls.n = a.n; Ls.c = a.c; Ls.L = a.L; Ls.k = a.k;
    Ls.cls = 0; Ls.decided = 0; Ls.hash = 0; Ls.size0 = 0;
    Ls.item = 0; Ls.sid = 0; Ls.cols = 0;
    Ls.rep = Ls.step = Ls.size = Ls.nF = 0;
    Ls.fc = 0ull;
    Ls.sp = 0;
    Ls.x0 = Ls.x1 = Ls.y0 = Ls.y1 = 0;
    // the movelist process: this lane's stack of S * S cells in the launch's scratch
    uint16_t *stk = LIFO ? a.lifo_stack + ((size_t)blockIdx.x * blockDim.x + threadIdx.x) * (S * S) : nullptr;
    constexpr bool lifo = LIFO;
    unsigned long long st_draw = 0, st_seed = 0, st_slots = 0, st_geno = 0;  // executed work (a.stats)
    Ls.ymin = Ls.ymax = Ls.xmin = Ls.xmax = 0;
    Ls.diverged = 0;
    Ls.forced = 0;
    Ls.cert = 0;
    Ls.ka = Ls.kb = NO_BLOCK;
    Ls.pa = Ls.pb = make_uint4(0, 0, 0, 0);
    unsigned long long q_next = 0, q_end = 0;  // this warp's slice of the work counter
    const int b_uniform = log2_colours(a.c);

    for (;;) {
        // ---- service: write finished genotypes and hand out new ones from the
        // pre-filter's list (all lanes together)
        for (;;) {
            if (a.esc_list) {
                // growth reached past the window: the item goes to the full-lattice launch unclassified
                // (a site outside the window with two candidates is local ambiguity there too, and an
                // ambiguity elsewhere in the same step comes first: those results stand)
                const bool esc = Ls.phase == PH_WRITE && Ls.cls == JATAM_UNBOUNDED;
                const unsigned em = __ballot_sync(FULL, esc);
                if (em) {
                    const int first_lane = __ffs(em) - 1;
                    unsigned long long base = 0;
                    if (lane == first_lane) base = atomicAdd(a.esc_count, (unsigned long long)__popc(em));
                    base = __shfl_sync(FULL, base, first_lane);
                    if (esc) {
                        a.esc_list[base + __popc(em & lanemask_lt())] = Ls.item;
                        Ls.phase = PH_NEED;
                    }
                }
            }
            if (Ls.phase == PH_WRITE) {
                const bool shaped = Ls.cls == JATAM_DET_BOUNDED || Ls.cls == JATAM_ND_STERIC;
                const unsigned size = shaped ? (unsigned)Ls.size0 : 0u;
                const uint32_t hash = shaped ? Ls.hash : 0u;
                write_result(a, Ls.item, Ls.cls, Ls.decided, size, hash);
                if (a.use_hist && Ls.cls != 255)
                    hist_insert(H, a.table, ((unsigned long long)Ls.cls << 32) | hash, 1u, Ls.sid, size, size, a.err);
                Ls.phase = PH_NEED;
            }
            const unsigned need = __ballot_sync(FULL, Ls.phase == PH_NEED);
            if (!need) break;
            const int cnt = __popc(need);
            const int rank = __popc(need & lanemask_lt());
            unsigned long long my_pos = ~0ull;
            int assigned = 0;
            while (assigned < cnt) {
                if (q_next >= q_end) {
                    unsigned long long nb = 0;
                    if (lane == 0) nb = atomicAdd(work_next, (unsigned long long)CHUNK);
                    nb = __shfl_sync(FULL, nb, 0);
                    if (nb >= total) break;
                    q_next = nb;
                    q_end = min(nb + (unsigned long long)CHUNK, total);
                }
                const int take = (int)min((unsigned long long)(cnt - assigned), q_end - q_next);
                if (Ls.phase == PH_NEED && rank >= assigned && rank < assigned + take)
                    my_pos = q_next + (unsigned long long)(rank - assigned);
                q_next += (unsigned long long)take;
                assigned += take;
            }
            if (Ls.phase == PH_NEED) {
                if (my_pos == ~0ull) {
                    Ls.phase = PH_DONE;
                } else {
                    const unsigned long long item =
                        my_pos < front ? list[my_pos]
                        : my_pos < front + mid ? mid_list[my_pos - front]
                                               : list[a.list_stride - 1 - (my_pos - front - mid)];
                    const Item it = load_item(a, item, b_uniform, a.esc_list ? JATAM_MAX_GRID : S);
                    Ls.item = item;
                    Ls.sid = it.sid;
                    Ls.cols = it.cols;
                    // in a window the lattice is the S x S window itself (its seed cell, S / 2, is the
                    // lattice's seed cell L / 2 shifted; row-major order is kept by the shift)
                    Ls.n = it.n; Ls.c = it.c; Ls.L = a.esc_list ? S : it.L; Ls.k = it.k;
                    Ls.phase = PH_INIT;
                }
            }
            break;  // every listed item grows: one round hands out work to all idle lanes
        }
        // ---- binding tables of the genotypes that grow: every new lane builds its own
        if (Ls.phase == PH_INIT) {
            lane_tables<S, NT>(my, Ls.cols, Ls.n, Ls.c);
            // a new genotype: clear whatever the previous one left in the bitmaps
            if (Ls.dlo <= Ls.dhi) {
                const int lo = max(Ls.dlo, 0), hi = min(Ls.dhi, S - 1);
                clear_rows<S>(my, G::OCCA, lo, hi);
                clear_rows<S>(my, G::OCCB, lo, hi);
                clear_rows<S>(my, G::FRONT, lo, hi);
            }
            Ls.dlo = S;
            Ls.dhi = -1;
            Ls.blo = S;
            Ls.bhi = -1;
            Ls.rep = 0;
            Ls.phase = PH_START;
            st_geno += 1;
            // the first Philox block comes from the growth rounds' batched fetch
            Ls.ka = NO_BLOCK;
            Ls.kb = NO_BLOCK;
        }
        if (__all_sync(FULL, Ls.phase == PH_DONE)) break;

        // ---- growth: one step per busy lane per round, until a.stop_at lanes
        // have finished their genotype or no lane is left growing
        for (;;) {
            // Philox blocks are computed for all lanes at once: when some lane
            // lacks the block of its current draw, every lane that will need a
            // block soon computes it in the same pass -- its current one, else
            // the one it needs after that: the next block of this replicate
            // while the replicate still draws past the current block (known
            // from replicate 0's size for a later replicate that has not
            // diverged from it; assumed in replicate 0), else block 0 of the
            // next replicate.  Keys grow along a genotype's draws, so a held
            // block below the current key is spent.
            {
                uint32_t want = NO_BLOCK;
                bool now = false;
                if (Ls.phase == PH_GROW) {
                    // the draw of this step: the rank (row-major process) or the push
                    // order after the pop (movelist process, one step later)
                    const uint32_t s = (uint32_t)Ls.step + (lifo ? 1u : 0u);
                    const uint32_t key = (uint32_t)Ls.rep * 512u + (s >> 2);
                    if (Ls.ka != key && Ls.kb == key) {
                        Ls.pa = Ls.pb;
                        Ls.ka = key;
                        Ls.kb = NO_BLOCK;
                    }
                    if (Ls.ka != key) {
                        want = key;
                        now = true;
                    } else if (Ls.kb == NO_BLOCK || Ls.kb < key) {
                        // the last draw of a replicate that ends in replicate 0's
                        // configuration: size0 - 1 placements after the seed
                        const int last = (Ls.size0 - 2 + (lifo ? 1 : 0)) >> 2;
                        const bool more = Ls.rep == 0 || Ls.diverged || (int)(s >> 2) < last;
                        if (more) want = key + 1u;
                        else if (Ls.rep + 1 < Ls.k) want = (uint32_t)(Ls.rep + 1) * 512u;
                    }
                } else if (Ls.phase == PH_START) {
                    // the movelist process draws the push order right after the seed
                    const uint32_t key = (uint32_t)Ls.rep * 512u;
                    if (Ls.ka != key && Ls.kb != key) {
                        want = key;
                        now = lifo;
                    }
                }
                if (__any_sync(FULL, now) && want != NO_BLOCK) {
                    const uint4 w = philox_block(want, Ls.sid, a.key0, a.key1);
                    if (now) {
                        Ls.pa = w;
                        Ls.ka = want;
                    } else {
                        Ls.pb = w;
                        Ls.kb = want;
                    }
                }
            }
            if (a.stats) {
                st_draw += __popc(__ballot_sync(FULL, Ls.phase == PH_GROW));
                st_seed += __popc(__ballot_sync(FULL, Ls.phase == PH_START));
                st_slots += 32;
            }
            lane_step<S, LIFO>(Ls, my, a.key0, a.key1, a.err, stk);
            const unsigned busy = __ballot_sync(FULL, Ls.phase == PH_START || Ls.phase == PH_GROW);
            if (!busy) break;
            const unsigned fin = __ballot_sync(FULL, Ls.phase == PH_DOM || Ls.phase == PH_SHAPE || Ls.phase == PH_WRITE);
            if (__popc(fin) >= a.stop_at) break;
        }

        // ---- dominance certificates of replicate-0 configurations that are not closed
        unsigned dom = __ballot_sync(FULL, Ls.phase == PH_DOM);
        while (dom) {
            const int o = __ffs(dom) - 1;
            dom &= dom - 1;
            const bool ok = coop_dominated<S, NT>(o, warp_lanes, Ls, lane);
            if (lane == o) {
                if (ok) {
                    Ls.cls = JATAM_DET_BOUNDED;
                    Ls.decided = Ls.k;
                    Ls.phase = PH_SHAPE;
                } else {
                    // replicate 1 (replicate 0 wrote nothing in OCCB)
                    Ls.rep = 1;
                    Ls.phase = PH_START;
                }
            }
            __syncwarp();
        }

        // ---- canonical shapes of finished genotypes: a per-warp cache keyed by
        // the exact crop (when it has at most 32 cells), then the launch's crop
        // table (at most CROP_CELLS cells), else one warp-wide job each
        unsigned long long ckey = 0ull, gbits = 0ull;
        int cslot = -1, gslot = -1;
        if (Ls.phase == PH_SHAPE) {
            const int h = Ls.y1 - Ls.y0 + 1, w = Ls.x1 - Ls.x0 + 1;
            if (h * w <= CROP_CELLS) {
                const uint32_t wmask = (w >= 32) ? FULL : ((1u << w) - 1u);
                unsigned long long bits = 0;  // row i of the crop at bits i * w ..
                for (int i = 0; i < h; ++i) {
                    const int b = (Ls.y0 + i) * S + Ls.x0;
                    bits |= (unsigned long long)((my[(G::OCCA + (b >> 5)) * 32] >> (b & 31)) & wmask) << (i * w);
                }
                const uint32_t hw = ((uint32_t)h << 8) | (uint32_t)w;
                if (h * w <= 32) {
                    ckey = ((unsigned long long)h << 40) | ((unsigned long long)w << 32) | bits;
                    cslot = (int)((uint32_t)((ckey * 0x9E3779B97F4A7C15ull) >> 32) >> 27);
                    const uint32_t *ce = warp_lanes + cslot;
                    const unsigned long long have =
                        ((unsigned long long)ce[(G::CACHE + 1) * 32] << 32) | ce[G::CACHE * 32];
                    if (have == ckey) {
                        Ls.hash = ce[(G::CACHE + 2) * 32];
                        Ls.phase = PH_WRITE;
                    }
                }
                if (Ls.phase == PH_SHAPE && a.crops) {
                    // open addressing, a few probes; a slot's key and meta word are each
                    // written once per launch (key by compare-and-swap, then the meta
                    // word), so a matching key with a valid meta word is always right
                    const unsigned mask = (1u << a.crops_log2) - 1u;
                    const unsigned long long key = crop_key(bits, h, w);
                    const unsigned s0 = (unsigned)((key * 0x9E3779B97F4A7C15ull) >> 40) & mask;
                    for (int p = 0; p < CROP_PROBES; ++p) {
                        const unsigned sl = (s0 + (unsigned)p) & mask;
                        const unsigned long long k = __ldcg(&a.crops[2 * sl]);
                        if (k == 0ull) {
                            gslot = (int)sl;
                            break;
                        }
                        if (k == key) {
                            const unsigned long long meta = __ldcg(&a.crops[2 * sl + 1]);
                            if ((meta >> 63) && (uint32_t)((meta >> 40) & 0xFFFFu) == hw) {
                                Ls.hash = (uint32_t)meta;
                                Ls.phase = PH_WRITE;
                                if (cslot >= 0) {
                                    uint32_t *ce = warp_lanes + cslot;
                                    ce[G::CACHE * 32] = (uint32_t)ckey;
                                    ce[(G::CACHE + 1) * 32] = (uint32_t)(ckey >> 32);
                                    ce[(G::CACHE + 2) * 32] = Ls.hash;
                                }
                            }
                            break;
                        }
                    }
                    if (Ls.phase == PH_SHAPE) gbits = key;
                    if (gslot < 0) gslot = (int)s0;  // the probes start there again on insertion
                }
            }
        }
        unsigned shp = __ballot_sync(FULL, Ls.phase == PH_SHAPE);
        while (shp) {
            const int o = __ffs(shp) - 1;
            shp &= shp - 1;
            // the owner claims its crop's slot of the call's crop table before the form is computed
            // (the key by compare-and-swap now, the meta word once the hash is known); a crop the
            // table cannot hold goes to the spill list, from which the side table of shapes takes it
            int claim = -1;
            int record = 0;
            if (lane == o) {
                record = 1;
                if (gbits) {
                    const unsigned mask = (1u << a.crops_log2) - 1u;
                    for (int p = 0; p < CROP_PROBES; ++p) {
                        const unsigned sl = ((unsigned)gslot + (unsigned)p) & mask;
                        const unsigned long long old = atomicCAS(&a.crops[2 * sl], 0ull, gbits);
                        if (old == 0ull) {
                            claim = (int)sl;
                            record = 0;  // the crop table holds it
                            break;
                        }
                        if (old == gbits) {
                            record = 0;  // another warp claimed this crop
                            break;
                        }
                    }
                }
            }
            record = __shfl_sync(FULL, record, o);
            const uint32_t hv = coop_shape_hash<S>(o, warp_lanes, Ls, lane, a.c4 != 0,
                                                   record != 0 && a.spill.rows != nullptr, a.spill);
            if (lane == o) {
                Ls.hash = hv;
                Ls.phase = PH_WRITE;
                if (cslot >= 0) {
                    uint32_t *ce = warp_lanes + cslot;
                    ce[G::CACHE * 32] = (uint32_t)ckey;
                    ce[(G::CACHE + 1) * 32] = (uint32_t)(ckey >> 32);
                    ce[(G::CACHE + 2) * 32] = hv;
                }
                if (claim >= 0) {
                    const unsigned long long meta = (1ull << 63) |
                        ((unsigned long long)(((Ls.y1 - Ls.y0 + 1) << 8) | (Ls.x1 - Ls.x0 + 1)) << 40) | hv;
                    __stcg(&a.crops[2 * claim + 1], meta);
                }
            }
            __syncwarp();
        }
    }
    if (a.stats) {
        st_geno = __reduce_add_sync(FULL, (unsigned)st_geno);
        if (lane == 0) {
            atomicAdd(&a.stats[0], st_draw);
            atomicAdd(&a.stats[1], st_seed);
            atomicAdd(&a.stats[2], st_slots);
            atomicAdd(&a.stats[3], st_geno);
        }
    }
}

template <typename HT>
__device__ __forceinline__ void hist_begin(HT &H)
{
    for (int i = threadIdx.x; i < HT::slots; i += blockDim.x) {
        H.key[i] = EMPTY_KEY;
        H.min_id[i] = ~0ull;
        H.count[i] = 0u;
        H.smax[i] = 0u;
        H.smin[i] = 0xFFFFFFFFu;
    }
    __syncthreads();
}

template <typename HT>
__device__ __forceinline__ void hist_end(HT &H, const LaunchArgs &a)
{
    __syncthreads();
    if (a.use_hist) {
        for (int i = threadIdx.x; i < HT::slots; i += blockDim.x)
            if (H.key[i] != EMPTY_KEY)
                table_insert(a.table, H.key[i], H.count[i], H.min_id[i], H.smax[i], H.smin[i], a.err);
    }
}

// One lattice template for every warp: the items of pre-filter list a.klass.
// CTAs of at most MAX_CTA_WARPS warps, three of which fit an SM's registers.
template <int S, int NT, bool LIFO>
__global__ void __launch_bounds__(MAX_CTA_WARPS * 32, 3) classify_kernel(const LaunchArgs a)
{
    extern __shared__ uint32_t smem_lanes[];
    __shared__ SmemHist H;
    hist_begin(H);
    const int warp = threadIdx.x >> 5;
    uint32_t *warp_lanes = smem_lanes + (size_t)warp * Geo<S, NT>::WORDS * 32;
    const bool three = a.heavy_first == 2 && !a.bucket && a.klass == 0;
    warp_loop<S, NT, LIFO>(a, warp_lanes, H, a.list + (size_t)a.klass * a.list_stride, a.list_count[a.klass],
                           a.list_count[3 + a.klass], a.work_next + a.klass, three ? a.list + a.list_stride : nullptr,
                           three ? a.list_count[1] : 0ull);
    hist_end(H, a);
}

// ---------------------------------------------------------------------------
// Replicate lanes, for calls too small to fill the GPU one genotype per lane: a
// warp takes one genotype at a time and lane r grows its replicate r (k <= 32)
// on the lane's own lattice, all k at once.  A replicate's process depends
// only on the genotype and on r (the draws are keyed by genotype, replicate and
// step), so each lane follows exactly the path replicate r takes in the
// sequential process.  Once every lane has ended, the first deciding replicate
// is the first r whose replicate ended in local ambiguity or unbounded growth,
// or (r > 0) in a configuration other than replicate 0's -- other cells or
// another tuple on a cell -- which is steric non-determinism; with none, the
// genotype is deterministic.  The shape is replicate 0's (lane 0's lattice).
// The latency of a genotype becomes that of its longest replicate instead of
// the sum over its replicates, at the cost of the exact shortcuts, which
// skip replicates that the lanes here run side by side anyway.
// ---------------------------------------------------------------------------
// 0xF in nibble i for every set bit i of a byte
__device__ __forceinline__ uint32_t nibble_mask(uint32_t byte)
{
    uint32_t m = byte & 255u;
    m = (m | (m << 12)) & 0x000F000Fu;
    m = (m | (m << 6)) & 0x03030303u;
    m = (m | (m << 3)) & 0x11111111u;
    return m * 0xFu;
}

template <int S, int NT>
__device__ __forceinline__ void reps_loop(const LaunchArgs &a, uint32_t *warp_lanes, SmemHistSmall &H,
                                          const unsigned long long *list, unsigned long long front,
                                          unsigned long long back, unsigned long long *work_next,
                                          const unsigned long long *mid_list, unsigned long long mid)
{
    const unsigned long long total = front + mid + back;
    using G = Geo<S, NT>;
    const int lane = threadIdx.x & 31;
    uint32_t *my = warp_lanes + lane;
    for (int w = 0; w < 3 * G::NW; ++w) my[w * 32] = 0u;
    __syncwarp();
    Lane Ls;
    Ls.phase = PH_DONE;
    Ls.dlo = S;
    Ls.dhi = -1;
    Ls.blo = S;
    Ls.bhi = -1;
    Ls.n = a.n; Ls.c = a.c; Ls.L = a.L; Ls.k = a.k;
    Ls.cls = 0; Ls.decided = 0; Ls.hash = 0; Ls.size0 = 0;
    Ls.item = 0; Ls.sid = 0; Ls.cols = 0;
    Ls.rep = Ls.step = Ls.size = Ls.nF = 0;
    Ls.fc = 0ull;
    Ls.sp = 0;
    Ls.x0 = Ls.x1 = Ls.y0 = Ls.y1 = 0;
    Ls.ymin = Ls.ymax = Ls.xmin = Ls.xmax = 0;
    Ls.diverged = 0;
    Ls.forced = 0;
    Ls.cert = 0;
    Ls.ka = Ls.kb = NO_BLOCK;
    Ls.pa = Ls.pb = make_uint4(0, 0, 0, 0);
    const int b_uniform = log2_colours(a.c);
    for (;;) {
        unsigned long long pos = 0;
        if (lane == 0) pos = atomicAdd(work_next, 1ull);
        pos = __shfl_sync(FULL, pos, 0);
        if (pos >= total) break;
        const unsigned long long item = pos < front ? list[pos]
                                        : pos < front + mid ? mid_list[pos - front]
                                                            : list[a.list_stride - 1 - (pos - front - mid)];
        const Item it = load_item(a, item, b_uniform, S);
        Ls.item = item;
        Ls.sid = it.sid;
        Ls.cols = it.cols;
        Ls.n = it.n; Ls.c = it.c; Ls.L = it.L; Ls.k = it.k;
        lane_tables<S, NT>(my, Ls.cols, Ls.n, Ls.c);
        if (Ls.dlo <= Ls.dhi) {
            const int lo = max(Ls.dlo, 0), hi = min(Ls.dhi, S - 1);
            clear_rows<S>(my, G::OCCA, lo, hi);
            clear_rows<S>(my, G::FRONT, lo, hi);
        }
        Ls.dlo = S;
        Ls.dhi = -1;
        Ls.rep = lane;
        Ls.ka = Ls.kb = NO_BLOCK;
        Ls.cls = JATAM_DET_BOUNDED;  // a lane without a replicate never deviates
        Ls.phase = lane < Ls.k ? PH_START : PH_DONE;
        __syncwarp();
        // every lane one step a round until all replicates have ended; the Philox block of a
        // lane's draw is computed in the round that first needs it (the lanes move in step,
        // so they need new blocks in the same rounds)
        for (int round = 1;; ++round) {
            const uint32_t key = (uint32_t)Ls.rep * 512u + ((uint32_t)Ls.step >> 2);
            if (Ls.phase == PH_GROW && Ls.ka != key) {
                Ls.pa = philox_block(key, Ls.sid, a.key0, a.key1);
                Ls.ka = key;
            }
            lane_step<S, false, true>(Ls, my, a.key0, a.key1, a.err, nullptr);
            // a replicate known to deviate -- ended in local ambiguity or unbounded growth, or
            // terminated at another size than replicate 0 -- makes every higher replicate
            // irrelevant (the first deviating one decides): those lanes stop, checked every
            // fourth round (a lane that runs on for a few rounds more changes no result)
            if ((round & 3) == 0) {
                const bool ended = lane < Ls.k && Ls.phase == PH_DONE;
                const int size0 = __shfl_sync(FULL, Ls.size, 0);
                const bool term0 = __shfl_sync(FULL, ended && Ls.cls == JATAM_DET_BOUNDED, 0);
                const bool known = ended && (Ls.cls != JATAM_DET_BOUNDED || (lane > 0 && term0 && Ls.size != size0));
                const unsigned km = __ballot_sync(FULL, known);
                if (km && lane > __ffs(km) - 1 && (Ls.phase == PH_START || Ls.phase == PH_GROW)) Ls.phase = PH_DONE;
            }
            if (!__any_sync(FULL, Ls.phase == PH_START || Ls.phase == PH_GROW)) break;
        }
        __syncwarp();
        // the first replicate that deviates from replicate 0
        const int size0 = __shfl_sync(FULL, Ls.size, 0);
        bool dev = false;
        if (lane < Ls.k) {
            if (Ls.cls != JATAM_DET_BOUNDED) {
                dev = true;
            } else if (lane > 0) {
                if (Ls.size != size0) dev = true;
                for (int w = 0; w < G::NW && !dev; ++w) {
                    const uint32_t o = my[(G::OCCA + w) * 32], o0 = warp_lanes[(G::OCCA + w) * 32];
                    if (o != o0) {
                        dev = true;
                    } else if (o) {
#pragma unroll
                        for (int q = 0; q < 4; ++q) {
                            const uint32_t m = nibble_mask(o >> (8 * q));
                            const int nw = G::NIB + 4 * w + q;
                            if ((my[nw * 32] ^ warp_lanes[nw * 32]) & m) dev = true;
                        }
                    }
                }
            }
        }
        const unsigned devm = __ballot_sync(FULL, dev);
        const int r = devm ? __ffs(devm) - 1 : 0;
        const int cr = __shfl_sync(FULL, Ls.cls, r);
        const int cls = !devm ? JATAM_DET_BOUNDED : (cr != JATAM_DET_BOUNDED ? cr : JATAM_ND_STERIC);
        const int decided = !devm ? Ls.k : r;
        // replicate 0's shape: the launch's crop table, else one warp-wide job
        uint32_t hash = 0;
        const bool shaped = cls == JATAM_DET_BOUNDED || cls == JATAM_ND_STERIC;
        if (shaped) {
            int have = 0, record = 0, claim = -1;
            uint32_t hv = 0;
            if (lane == 0) {
                Ls.x0 = Ls.xmin;
                Ls.x1 = Ls.xmax;
                Ls.y0 = Ls.ymin;
                Ls.y1 = Ls.ymax;
                const int h = Ls.y1 - Ls.y0 + 1, w = Ls.x1 - Ls.x0 + 1;
                record = 1;
                if (a.crops && h * w <= CROP_CELLS) {
                    const uint32_t wmask = (w >= 32) ? FULL : ((1u << w) - 1u);
                    unsigned long long bits = 0;
                    for (int i = 0; i < h; ++i) {
                        const int b = (Ls.y0 + i) * S + Ls.x0;
                        bits |= (unsigned long long)((my[(G::OCCA + (b >> 5)) * 32] >> (b & 31)) & wmask) << (i * w);
                    }
                    const uint32_t hw = ((uint32_t)h << 8) | (uint32_t)w;
                    const unsigned mask = (1u << a.crops_log2) - 1u;
                    const unsigned long long key = crop_key(bits, h, w);
                    const unsigned s0 = (unsigned)((key * 0x9E3779B97F4A7C15ull) >> 40) & mask;
                    // a few probes: the crop's meta word holds its hash once its claimer has written it;
                    // a free slot is claimed (key by compare-and-swap) before the form is computed
                    for (int p = 0; p < CROP_PROBES; ++p) {
                        const unsigned sl = (s0 + (unsigned)p) & mask;
                        unsigned long long k = __ldcg(&a.crops[2 * sl]);
                        if (k == 0ull) {
                            k = atomicCAS(&a.crops[2 * sl], 0ull, key);
                            if (k == 0ull) {
                                claim = (int)sl;
                                record = 0;
                                break;
                            }
                        }
                        if (k == key) {
                            record = 0;
                            const unsigned long long meta = __ldcg(&a.crops[2 * sl + 1]);
                            if ((meta >> 63) && (uint32_t)((meta >> 40) & 0xFFFFu) == hw) {
                                hv = (uint32_t)meta;
                                have = 1;
                            }
                            break;
                        }
                    }
                }
            }
            have = __shfl_sync(FULL, have, 0);
            record = __shfl_sync(FULL, record, 0);
            if (!have) {
                hv = coop_shape_hash<S>(0, warp_lanes, Ls, lane, a.c4 != 0, record != 0 && a.spill.rows != nullptr,
                                        a.spill);
                if (lane == 0 && claim >= 0) {
                    const unsigned long long meta = (1ull << 63) |
                        ((unsigned long long)(((Ls.y1 - Ls.y0 + 1) << 8) | (Ls.x1 - Ls.x0 + 1)) << 40) | hv;
                    __stcg(&a.crops[2 * claim + 1], meta);
                }
            }
            hash = hv;
        }
        if (lane == 0) {
            const unsigned size = shaped ? (unsigned)size0 : 0u;
            write_result(a, Ls.item, cls, decided, size, hash);
            if (a.use_hist) hist_insert(H, a.table, ((unsigned long long)cls << 32) | hash, 1u, Ls.sid, size, size, a.err);
        }
        __syncwarp();
    }
}

template <int S, int NT>
__global__ void __launch_bounds__(MAX_CTA_WARPS * 32, 3) classify_reps_kernel(const LaunchArgs a)
{
    extern __shared__ uint32_t smem_lanes[];
    __shared__ SmemHistSmall H;
    hist_begin(H);
    const int warp = threadIdx.x >> 5;
    uint32_t *warp_lanes = smem_lanes + (size_t)warp * Geo<S, NT>::WORDS * 32;
    const bool three = a.heavy_first == 2 && !a.bucket && a.klass == 0;
    reps_loop<S, NT>(a, warp_lanes, H, a.list + (size_t)a.klass * a.list_stride, a.list_count[a.klass],
                     a.list_count[3 + a.klass], a.work_next + a.klass, three ? a.list + a.list_stride : nullptr,
                     three ? a.list_count[1] : 0ull);
    hist_end(H, a);
}

// Mixed lattice sizes in one persistent launch: the first plan_w32 warps of a
// CTA own 32 x 32 regions, the next plan_w16 16 x 16 regions, the rest 8 x 8.
// A warp first works through the list of its own size class, then steals from
// the lists of the smaller classes (a larger region holds any smaller
// lattice).
__global__ void __launch_bounds__(256) classify_mixed_kernel(const LaunchArgs a)
{
    extern __shared__ uint32_t smem_lanes[];
    __shared__ SmemHist H;
    hist_begin(H);
    const int warp = threadIdx.x >> 5;
    const int w32 = a.plan_w32, w16 = a.plan_w16;
    constexpr size_t R32 = (size_t)Geo<32>::WORDS * 32, R16 = (size_t)Geo<16>::WORDS * 32,
                     R8 = (size_t)Geo<8>::WORDS * 32;
    if (warp < w32) {
        uint32_t *wl = smem_lanes + (size_t)warp * R32;
        for (int c = 2; c >= 0; --c)
            warp_loop<32, 16, false>(a, wl, H, a.list + (size_t)c * a.list_stride, a.list_count[c], a.list_count[3 + c],
                                     a.work_next + c);
    } else if (warp < w32 + w16) {
        uint32_t *wl = smem_lanes + (size_t)w32 * R32 + (size_t)(warp - w32) * R16;
        for (int c = 1; c >= 0; --c)
            warp_loop<16, 16, false>(a, wl, H, a.list + (size_t)c * a.list_stride, a.list_count[c], a.list_count[3 + c],
                                     a.work_next + c);
    } else {
        uint32_t *wl = smem_lanes + (size_t)w32 * R32 + (size_t)w16 * R16 + (size_t)(warp - w32 - w16) * R8;
        warp_loop<8, 16, false>(a, wl, H, a.list, a.list_count[0], a.list_count[3], a.work_next);
    }
    hist_end(H, a);
}


// ===========================================================================
// One genotype per warp, for lattices up to 32 x 32.  Lane y holds row y of
// the lattice in registers: the occupancy of the current replicate and of
// replicate 0, the frontier, and the 4-bit tuple ids (the placed tuple of an
// occupied cell, the single candidate of a frontier cell).  The warp runs one
// assembly step at a time (Section 2.4's stochastic addition of bonding tiles):
// the rank of the drawn frontier site is found by a prefix sum of the rows'
// site counts across the lanes, the row's lane places the tile, and the lanes
// of rows y - 1, y and y + 1 re-evaluate the new tile's four neighbours.  The
// binding table is spread over the lanes (word j in lane j, read by shuffle),
// and the lanes compute 32 Philox blocks of a replicate's stream at once (128
// draws).  Nothing but the CTA's histogram table lives in shared memory, and a
// new genotype or replicate clears its lattice by zeroing registers, so far
// more warps fit an SM than with one genotype per lane, whose 32 x 32 layout
// needs about 1 KB of shared memory per lane.  The draws, the replicate rule
// and the exact shortcuts (forced path, closed shape, dominated offers) are
// those of the lane-per-genotype kernel, so the results are identical.
// ===========================================================================
constexpr int WG_WARPS = 8;  // warps per CTA of the warp-per-genotype kernel
constexpr int WG_CHUNK = 4;  // items a warp takes from the list at once

// tuple id of cell x of a row: nibble x & 7 of word x >> 3 (selected without
// indexing, so the words stay in registers)
__device__ __forceinline__ int row_tuple(uint32_t n0, uint32_t n1, uint32_t n2, uint32_t n3, int x)
{
    const uint32_t w = x < 8 ? n0 : x < 16 ? n1 : x < 24 ? n2 : n3;
    return (int)((w >> ((x & 7) * 4)) & 15u);
}
__device__ __forceinline__ void row_tuple_set(uint32_t &n0, uint32_t &n1, uint32_t &n2, uint32_t &n3, int x, int t)
{
    const int sh = (x & 7) * 4;
    const uint32_t keep = ~(15u << sh), val = (uint32_t)t << sh;
    if (x < 8) n0 = (n0 & keep) | val;
    else if (x < 16) n1 = (n1 & keep) | val;
    else if (x < 24) n2 = (n2 & keep) | val;
    else n3 = (n3 & keep) | val;
}

// The binding table of one genotype, word j in lane j: word 2 t + h holds, at
// bits 16 q, the set of representative tuples u whose side (d + 2) mod 4
// carries the partner of tuple t's colour on side d = 2 h + q (Section 1.1's
// pairs 1-2, 3-4, 5-6; 0 and an odd top colour bind nothing).  Tuple a = 4 t +
// r is tile t turned clockwise by r quarter turns (side d shows edge (d - r)
// mod 4); a representative is the lowest a with its rotated colour tuple.
__device__ __forceinline__ uint32_t warp_binding_table(unsigned long long cols, int n, int c, int lane)
{
    const int na = 4 * n;
    uint32_t tup = 0xFFFFFFFFu;  // never equal to a 16-bit tuple
    if (lane < na) tup = rot16((uint32_t)(cols >> (16 * (lane >> 2))) & 0xFFFFu, 4 * (lane & 3));
    int rep = lane;
    for (int a = na - 1; a >= 0; --a) {
        const uint32_t ta = __shfl_sync(FULL, tup, a);
        if (a < lane && ta == tup) rep = a;
    }
    const unsigned isrep = __ballot_sync(FULL, lane < na && rep == lane);
    const int t = (lane >> 1) & 15, h = lane & 1;
    const uint32_t tt = __shfl_sync(FULL, tup, t);
    int p0, p1;  // partners of t's colours on sides 2h and 2h + 1
    {
        const int x0 = (int)((tt >> (8 * h)) & 15u), x1 = (int)((tt >> (8 * h + 4)) & 15u);
        p0 = (x0 == 0) ? -1 : (x0 & 1) ? ((x0 + 1 < c) ? x0 + 1 : -1) : x0 - 1;
        p1 = (x1 == 0) ? -1 : (x1 & 1) ? ((x1 + 1 < c) ? x1 + 1 : -1) : x1 - 1;
    }
    uint32_t word = 0;
    for (int u = 0; u < na; ++u) {
        const uint32_t tu = __shfl_sync(FULL, tup, u);
        if (!((isrep >> u) & 1u)) continue;
        // side 2h + q faces side (2h + q + 2) mod 4 of u
        const int f0 = (int)((tu >> (4 * ((2 * h + 2) & 3))) & 15u);
        const int f1 = (int)((tu >> (4 * ((2 * h + 3) & 3))) & 15u);
        if (p0 >= 0 && f0 == p0) word |= 1u << u;
        if (p1 >= 0 && f1 == p1) word |= 1u << (16 + u);
    }
    return (lane < 2 * na) ? word : 0u;
}

// Dominance certificate of replicate 0's final configuration A0 (rows in lanes,
// absolute coordinates): the attachment graph u -> v when u offers v's tuple,
// bad offers to cells of A0 (the seed's cell excepted), and for every cell q
// receiving a bad offer a flood fill from its bad offerers that avoids q --
// the certificate fails if it reaches the seed.  The argument is that of the
// lane-per-genotype kernel's coop_dominated.
__device__ __forceinline__ bool warp_dominated(uint32_t occ, uint32_t n0, uint32_t n1, uint32_t n2, uint32_t n3,
                                               uint32_t nbm, int x0, int x1, int L, int lane)
{
    uint32_t occN = __shfl_up_sync(FULL, occ, 1), occS = __shfl_down_sync(FULL, occ, 1);
    if (lane == 0) occN = 0u;
    if (lane == 31) occS = 0u;
    const int sx = L >> 1, sy = L >> 1;
    uint32_t gN = 0, gE = 0, gS = 0, gW = 0, bN = 0, bE = 0, bS = 0, bW = 0;
    int tW = 0, tC = row_tuple(n0, n1, n2, n3, x0);
    for (int x = x0; x <= x1; ++x) {
        const int tE = (x + 1 < 32) ? row_tuple(n0, n1, n2, n3, x + 1) : 0;
        const int tN = __shfl_up_sync(FULL, tC, 1), tS = __shfl_down_sync(FULL, tC, 1);
        const uint32_t m01 = __shfl_sync(FULL, nbm, (2 * tC) & 31);
        const uint32_t m23 = __shfl_sync(FULL, nbm, (2 * tC + 1) & 31);
        if ((occ >> x) & 1u) {
            const uint32_t bit = 1u << x;
            const uint32_t MN = m01 & 0xFFFFu, ME = m01 >> 16, MS = m23 & 0xFFFFu, MW = m23 >> 16;
            if ((occN >> x) & 1u) {
                if ((MN >> tN) & 1u) gN |= bit;
                if ((MN & ~(1u << tN)) && !(lane - 1 == sy && x == sx)) bN |= bit;
            }
            if (x + 1 < 32 && ((occ >> (x + 1)) & 1u)) {
                if ((ME >> tE) & 1u) gE |= bit;
                if ((ME & ~(1u << tE)) && !(lane == sy && x + 1 == sx)) bE |= bit;
            }
            if ((occS >> x) & 1u) {
                if ((MS >> tS) & 1u) gS |= bit;
                if ((MS & ~(1u << tS)) && !(lane + 1 == sy && x == sx)) bS |= bit;
            }
            if (x > 0 && ((occ >> (x - 1)) & 1u)) {
                if ((MW >> tW) & 1u) gW |= bit;
                if ((MW & ~(1u << tW)) && !(lane == sy && x - 1 == sx)) bW |= bit;
            }
        }
        tW = tC;
        tC = tE;
    }
    const uint32_t fromAbove = __shfl_up_sync(FULL, bS, 1), fromBelow = __shfl_down_sync(FULL, bN, 1);
    uint32_t qs = (bE << 1) | (bW >> 1) | (lane > 0 ? fromAbove : 0u) | (lane < 31 ? fromBelow : 0u);
    qs &= occ;
    const uint32_t seed_bit = (lane == sy) ? (1u << sx) : 0u;
    for (int guard = 0; guard < 1024; ++guard) {  // at most one pass per cell of A0
        const unsigned hasq = __ballot_sync(FULL, qs != 0u);
        if (!hasq) return true;
        const int qy = __ffs(hasq) - 1;
        const int qx = __ffs(__shfl_sync(FULL, qs, qy)) - 1;
        if (lane == qy) qs &= ~(1u << qx);
        const uint32_t keep = occ & ((lane == qy) ? ~(1u << qx) : FULL);
        uint32_t X = 0u;
        if (lane == qy - 1) X = bS & (1u << qx);
        if (lane == qy + 1) X = bN & (1u << qx);
        if (lane == qy) X = (bW & ((qx + 1 < 32) ? (2u << qx) : 0u)) | (bE & ((qx > 0) ? (1u << (qx - 1)) : 0u));
        for (int it = 0; it < 1024; ++it) {  // a layer per step: at most the cells of A0
            if (__any_sync(FULL, (X & seed_bit) != 0u)) return false;
            const uint32_t below = __shfl_down_sync(FULL, X, 1);
            const uint32_t above = __shfl_up_sync(FULL, X, 1);
            uint32_t nX = X | (gE & (X >> 1)) | (gW & (X << 1)) | (lane < 31 ? (gS & below) : 0u) |
                          (lane > 0 ? (gN & above) : 0u);
            nX &= keep;
            if (!__any_sync(FULL, nX != X)) break;
            X = nX;
        }
    }
    return false;  // unreachable: the passes are bounded by the cells of A0
}

struct WarpOutcome {
    int cls, decided, size;
    uint32_t hash;
};

// Classify one genotype with the whole warp (every value below is uniform
// across the warp except the row registers and `nbm`).
__device__ __forceinline__ WarpOutcome warp_classify(const LaunchArgs &a, const Item &it, int lane,
                                                     unsigned long long *st_draw, unsigned long long *st_seed)
{
    const int L = it.L, k = it.k, cx = it.L >> 1;
    const uint32_t nbm = warp_binding_table(it.cols, it.n, it.c, lane);
    uint32_t occ = 0, front = 0, occ0 = 0, n0 = 0, n1 = 0, n2 = 0, n3 = 0;
    int size0 = 0, x0 = cx, x1 = cx, y0 = cx, y1 = cx;
    WarpOutcome res{JATAM_DET_BOUNDED, k, 0, 0u};
    // Philox blocks of the current replicate: lane j holds block base + j
    uint4 blk = make_uint4(0, 0, 0, 0);
    int blk_base = -1, blk_rep = -1;
    for (int rep = 0; rep < k; ++rep) {
        // the seed: tile 0 in orientation 0 at the centre (tuple id 0)
        occ = (lane == cx) ? (1u << cx) : 0u;
        front = 0u;
        if (rep == 0 && lane == cx) row_tuple_set(n0, n1, n2, n3, cx, 0);
        int px = cx, py = cx, tau = 0;
        int size = 1, step = 0, nF = 0;
        int xmin = cx, xmax = cx, ymin = cx, ymax = cx;
        bool forced = true, cert = true, diverged = false;
        int outcome = 0;  // 1 local ambiguity, 2 unbounded, 3 terminated
        *st_seed += 1;
        for (int guard = 0; guard <= 32 * 32; ++guard) {
            // ---- re-evaluate the empty neighbours of the tile tau just placed at (px, py):
            // lane py - 1 its north side, lane py + 1 its south side, lane py its east and west
            // sides (indices wrap to a lane whose site lies outside the grid)
            const uint32_t m01 = __shfl_sync(FULL, nbm, 2 * tau), m23 = __shfl_sync(FULL, nbm, 2 * tau + 1);
            const bool isN = lane == ((py + 31) & 31), isS = lane == ((py + 1) & 31), isC = lane == py;
            bool nd = false, unb = false, bad = false, div = false;
            int added = 0;
            // up to two sites per lane: (sx1, sy1, M1) and, on lane py, the west side
            const int sx1 = isC ? px + 1 : px;
            const int sy1 = isN ? py - 1 : isS ? py + 1 : py;
            const uint32_t M1 = isN ? (m01 & 0xFFFFu) : isS ? (m23 & 0xFFFFu) : (m01 >> 16);
#pragma unroll
            for (int q = 0; q < 2; ++q) {
                const bool mine = q == 0 ? (isN || isS || isC) : isC;
                const int x = q == 0 ? sx1 : px - 1;
                const int y = q == 0 ? sy1 : py;
                const uint32_t M = q == 0 ? M1 : (m23 >> 16);
                const bool multi = (M & (M - 1u)) != 0u;
                const bool in = x >= 0 && x < L && y >= 0 && y < L;
                if (mine && !in) {
                    nd = nd || multi;
                    unb = unb || (M != 0u && !multi);
                } else if (mine) {
                    const uint32_t bit = 1u << x;
                    const bool empty = !(occ & bit);
                    const bool isf = (front & bit) != 0u;
                    const int tq = row_tuple(n0, n1, n2, n3, x);
                    nd = nd || (empty && (isf ? (M & ~(1u << tq)) != 0u : multi));
                    // replicate 0: an occupied neighbour that could receive another tuple from the new
                    // tile breaks the closure of the final shape (the seed's cell excepted)
                    if (rep == 0 && !empty && (M & ~(1u << tq)) != 0u && !(x == cx && y == cx)) bad = true;
                    if (empty && !isf && M != 0u && !multi) {
                        const int tn = __ffs(M) - 1;
                        // a later replicate must place replicate 0's tuple here to end in its configuration
                        if (rep > 0 && (!(occ0 & bit) || tq != tn)) div = true;
                        row_tuple_set(n0, n1, n2, n3, x, tn);
                        front |= bit;
                        ++added;
                    }
                }
            }
            const unsigned flags = __reduce_or_sync(FULL, (nd ? 1u : 0u) | (unb ? 2u : 0u) | (bad ? 4u : 0u) |
                                                              (div ? 8u : 0u));
            nF += (int)__reduce_add_sync(FULL, (unsigned)added);
            if (flags & 4u) cert = false;
            if (flags & 8u) diverged = true;
            if (flags & 1u) { outcome = 1; break; }
            if (flags & 2u) { outcome = 2; break; }
            if (nF == 0) { outcome = 3; break; }
            // ---- draw: word (step mod 4) of Philox block step >> 2 of this replicate's stream
            if (nF > 1) forced = false;
            const int b = step >> 2;
            if (blk_rep != rep || b < blk_base || b >= blk_base + 32) {
                blk_base = b;
                blk_rep = rep;
                blk = philox4x32_10(make_uint4((uint32_t)(b + lane), (uint32_t)rep, (uint32_t)it.sid,
                                               (uint32_t)(it.sid >> 32)), a.key0, a.key1);
            }
            const int sel = step & 3;
            const uint32_t word = sel == 0 ? blk.x : sel == 1 ? blk.y : sel == 2 ? blk.z : blk.w;
            const uint32_t u = __shfl_sync(FULL, word, b - blk_base);
            const uint32_t i = __umulhi(u, (uint32_t)nF);
            // the row holding frontier site number i (row-major order): a prefix sum of site counts
            const uint32_t cnt = (uint32_t)__popc(front);
            uint32_t incl = cnt;
#pragma unroll
            for (int off = 1; off < 32; off <<= 1) {
                const uint32_t v = __shfl_up_sync(FULL, incl, off);
                if (lane >= off) incl += v;
            }
            const uint32_t excl = incl - cnt;
            const unsigned hit = __ballot_sync(FULL, i >= excl && i < incl);
            if (hit == 0u) break;  // unreachable (i < nF = the sum of the counts): reported below as a guard error
            const int row = __ffs(hit) - 1;
            int bx = 0, bt = 0;
            if (lane == row) {
                bx = nth_set(front, i - excl);
                bt = row_tuple(n0, n1, n2, n3, bx);
                front &= ~(1u << bx);
                occ |= 1u << bx;
            }
            px = __shfl_sync(FULL, bx, row & 31);
            tau = __shfl_sync(FULL, bt, row & 31);
            py = row;
            nF -= 1;
            size += 1;
            step += 1;
            *st_draw += 1;
            xmin = min(xmin, px);
            xmax = max(xmax, px);
            ymin = min(ymin, py);
            ymax = max(ymax, py);
        }
        // ---- the first deciding replicate (reading R10) and the exact shortcuts
        if (outcome == 1 || outcome == 2 || outcome == 0) {
            res.cls = outcome == 2 ? JATAM_UNBOUNDED : JATAM_ND_LOCAL;
            res.decided = rep;
            if (outcome == 0) atomicOr(a.err, ERR_GUARD);  // unreachable: a replicate ends within L * L steps
            return res;
        }
        if (rep == 0) {
            size0 = size;
            occ0 = occ;
            x0 = xmin; x1 = xmax; y0 = ymin; y1 = ymax;
            if (forced || cert) break;  // every replicate ends in A0
            if (k > 1 && warp_dominated(occ0, n0, n1, n2, n3, nbm, x0, x1, L, lane)) break;
        } else if (diverged || size != size0) {
            res.cls = JATAM_ND_STERIC;
            res.decided = rep;
            break;
        }
    }
    // ---- replicate 0's shape: crop, canonical form under the 8 symmetries, hash
    res.size = size0;
    const int h = y1 - y0 + 1, w = x1 - x0 + 1;
    const uint32_t wmask = (w >= 32) ? FULL : ((1u << w) - 1u);
    const uint32_t r = (__shfl_sync(FULL, occ0, (y0 + lane) & 31) >> x0) & wmask;
    const uint32_t row = lane < h ? r : 0u;
    unsigned long long bits = 0ull;
    int gslot = -1;
    bool found = false;
    const uint32_t hw = ((uint32_t)h << 8) | (uint32_t)w;
    if (h * w <= CROP_CELLS && a.crops) {
        // the call's crop table (shared with the lane-per-genotype kernel's format)
        const unsigned long long mine = lane < h ? ((unsigned long long)row << (lane * w)) : 0ull;
        const uint32_t lo = __reduce_or_sync(FULL, (uint32_t)mine), hi = __reduce_or_sync(FULL, (uint32_t)(mine >> 32));
        bits = crop_key(((unsigned long long)hi << 32) | lo, h, w);
        const unsigned mask = (1u << a.crops_log2) - 1u;
        const unsigned s0 = (unsigned)((bits * 0x9E3779B97F4A7C15ull) >> 40) & mask;
        for (int p = 0; p < CROP_PROBES; ++p) {
            const unsigned sl = (s0 + (unsigned)p) & mask;
            const unsigned long long key = __ldcg(&a.crops[2 * sl]);
            if (key == 0ull) {
                gslot = (int)sl;
                break;
            }
            if (key == bits) {
                const unsigned long long meta = __ldcg(&a.crops[2 * sl + 1]);
                if ((meta >> 63) && (uint32_t)((meta >> 40) & 0xFFFFu) == hw) {
                    res.hash = (uint32_t)meta;
                    found = true;
                }
                break;
            }
        }
        if (gslot < 0) gslot = (int)s0;
    }
    if (!found) {
        // claim the crop's slot first; a crop the table cannot hold goes to the spill list, as in the
        // lane-per-genotype kernel
        int claim = -1, record = 1;
        if (lane == 0 && bits) {
            const unsigned mask = (1u << a.crops_log2) - 1u;
            for (int p = 0; p < CROP_PROBES; ++p) {
                const unsigned sl = ((unsigned)gslot + (unsigned)p) & mask;
                const unsigned long long old = atomicCAS(&a.crops[2 * sl], 0ull, bits);
                if (old == 0ull) {
                    claim = (int)sl;
                    record = 0;
                    break;
                }
                if (old == bits) {
                    record = 0;
                    break;
                }
            }
        }
        record = __shfl_sync(FULL, record, 0);
        if (record && a.spill.rows) spill_crop(a.spill, row, h, w, lane);
        res.hash = crop_shape_hash(row, h, w, lane, a.c4 != 0, ShapeTab{});
        if (lane == 0 && claim >= 0)
            __stcg(&a.crops[2 * claim + 1], (1ull << 63) | ((unsigned long long)hw << 40) | res.hash);
    }
    return res;
}

// the warps of a CTA work through one pre-filter list, a genotype at a time
__global__ void __launch_bounds__(WG_WARPS * 32, 3) classify_warp_kernel(const LaunchArgs a)
{
    __shared__ SmemHist H;
    hist_begin(H);
    const int lane = threadIdx.x & 31;
    const unsigned long long *list = a.list + (size_t)a.klass * a.list_stride;
    // a three-level heavy-first order keeps its middle level in region 1
    const bool three = a.heavy_first == 2 && !a.bucket && a.klass == 0;
    const unsigned long long *mid_list = a.list + a.list_stride;
    const unsigned long long front = a.list_count[a.klass], mid = three ? a.list_count[1] : 0ull;
    const unsigned long long total = front + mid + a.list_count[3 + a.klass];
    unsigned long long *work_next = a.work_next + a.klass;
    const int b_uniform = log2_colours(a.c);
    unsigned long long q_next = 0, q_end = 0, st_draw = 0, st_seed = 0, st_geno = 0;
    for (;;) {
        if (q_next >= q_end) {
            unsigned long long nb = 0;
            if (lane == 0) nb = atomicAdd(work_next, (unsigned long long)WG_CHUNK);
            nb = __shfl_sync(FULL, nb, 0);
            if (nb >= total) break;
            q_next = nb;
            q_end = min(nb + (unsigned long long)WG_CHUNK, total);
        }
        const unsigned long long pos = q_next++;
        const unsigned long long item = pos < front ? list[pos]
                                        : pos < front + mid ? mid_list[pos - front]
                                                            : list[a.list_stride - 1 - (pos - front - mid)];
        const Item it = load_item(a, item, b_uniform, 32);
        st_geno += 1;
        const WarpOutcome o = warp_classify(a, it, lane, &st_draw, &st_seed);
        if (lane == 0) {
            const bool shaped = o.cls == JATAM_DET_BOUNDED || o.cls == JATAM_ND_STERIC;
            const unsigned size = shaped ? (unsigned)o.size : 0u;
            const uint32_t hash = shaped ? o.hash : 0u;
            write_result(a, item, o.cls, o.decided, size, hash);
            if (a.use_hist)
                hist_insert(H, a.table, ((unsigned long long)o.cls << 32) | hash, 1u, it.sid, size, size, a.err);
        }
        __syncwarp();
    }
    if (a.stats && lane == 0) {
        atomicAdd(&a.stats[0], st_draw);
        atomicAdd(&a.stats[1], st_seed);
        atomicAdd(&a.stats[2], 32ull * (st_draw + st_seed));  // a warp step occupies all 32 lane slots
        atomicAdd(&a.stats[3], st_geno);
    }
    hist_end(H, a);
}


// Orbit mode, after the growth kernel: every genotype that is not its orbit's
// representative takes the representative's result (the representative is the
// smaller genotype, so it lies in the range, which starts at 0) and is counted
// in the histogram under the representative's stream id.
__global__ void __launch_bounds__(256) orbit_fill_kernel(const LaunchArgs a)
{
    __shared__ SmemHist H;
    hist_begin(H);
    const int b = log2_colours(a.c);
    const unsigned long long stride = (unsigned long long)gridDim.x * blockDim.x;
    for (unsigned long long idx = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; idx < a.count;
         idx += stride) {
        const unsigned long long g = a.first + idx;
        const unsigned long long r = orbit_rep(g, a.n, a.c, b);
        if (r == g) continue;
        const jatam_result res = a.out[r - a.first];
        a.out[idx] = res;
        if (a.use_hist && res.cls != 255)
            hist_insert(H, a.table, ((unsigned long long)res.cls << 32) | res.shape_hash, 1u, r, res.size, res.size,
                        a.err);
    }
    hist_end(H, a);
}

__global__ void reset_kernel(unsigned long long *work_next, unsigned *nkeys, unsigned long long *list_count,
                             unsigned long long *crops, unsigned crop_words, unsigned long long *extra,
                             int extra_words)
{
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        for (int c = 0; c < 3; ++c) work_next[c] = 0ull;
        for (int c = 0; c < 6; ++c) list_count[c] = 0ull;
        for (int c = 0; c < extra_words; ++c) extra[c] = 0ull;
        *nkeys = 0u;
    }
    for (unsigned i = blockIdx.x * blockDim.x + threadIdx.x; i < crop_words; i += gridDim.x * blockDim.x)
        crops[i] = 0ull;
}

__global__ void table_init_kernel(Table t)
{
    const unsigned cap = 1u << t.cap_log2;
    for (unsigned i = blockIdx.x * blockDim.x + threadIdx.x; i < cap; i += gridDim.x * blockDim.x) {
        t.key[i] = EMPTY_KEY;
        t.count[i] = 0ull;
        t.min_id[i] = ~0ull;
        t.size_max[i] = 0u;
        t.size_min[i] = 0xFFFFFFFFu;
    }
}

// the single-cell shape (h = w = 1) in the side table, by one thread: the
// pre-filter settles lone seeds without a warp computing their form
__device__ void shape_record_cell(const ShapeTab t, uint32_t hash)
{
    const unsigned mask = (1u << t.log2) - 1u;
    const unsigned long long key = (1ull << 32) | hash;
    const unsigned meta = 0x80000000u | (1u << 8) | 1u;
    unsigned slot = (hash * 2654435761u) >> (32 - t.log2);
    for (int p = 0; p < SHAPE_PROBES; ++p) {
        const unsigned long long old = atomicCAS(&t.key[slot], 0ull, key);
        if (old == 0ull) {
            for (int i = 0; i < 32; ++i) __stcg(&t.rows[(size_t)slot * 32 + i], i == 0 ? 1u : 0u);
            __threadfence();
            atomicExch(&t.meta[slot], meta);
            return;
        }
        if (old == key) {
            // the growth warps have finished (this is a later kernel); only a thread of
            // this kernel storing the same hash may still be writing: a bounded wait
            unsigned m = 0;
            for (int it = 0; it < SHAPE_WAIT && m == 0; ++it) {
                m = atomicOr(&t.meta[slot], 0u);
                if (m == 0) __nanosleep(64);
            }
            if (m == 0) {
                atomicAdd(&t.stats[1], 1u);
                return;
            }
            __threadfence();
            bool same = m == meta;
            for (int i = 0; i < 32 && same; ++i) same = __ldcg(&t.rows[(size_t)slot * 32 + i]) == (i == 0 ? 1u : 0u);
            if (!same) atomicAdd(&t.stats[0], 1u);
            return;
        }
        slot = (slot + 1) & mask;
    }
    atomicAdd(&t.stats[2], 1u);
}

// The side table of shapes of one call (or piece): a warp per crop of the crop
// table (key: bits, h, w; meta: valid bit and hash) and per spilled crop
// computes the crop's canonical form and stores or compares it under its hash.
// A crop-table hash that differs from the recomputed one is counted as a
// comparison given up (stats[1]): it cannot happen unless a kernel is wrong.
__global__ void __launch_bounds__(256) shape_scan_kernel(ShapeTab tab, const unsigned long long *crops,
                                                        unsigned crops_log2, CropSpill spill)
{
    const int lane = threadIdx.x & 31;
    const unsigned long long warp = (blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x) >> 5;
    const unsigned long long warps = (gridDim.x * (unsigned long long)blockDim.x) >> 5;
    const unsigned long long nslots = crops ? (1ull << crops_log2) : 0ull;
    unsigned long long nspill = spill.rows ? *spill.count : 0ull;
    if (nspill > spill.cap) nspill = spill.cap;
    for (unsigned long long i = warp; i < nslots + nspill; i += warps) {
        uint32_t row = 0;
        int h = 0, w = 0;
        uint32_t want = 0;
        bool check = false;
        if (i < nslots) {
            const unsigned long long key = crops[2 * i];
            const unsigned long long meta = crops[2 * i + 1];
            if (key == 0ull || !(meta >> 63)) continue;  // free slot, or a claim whose hash was never written
            h = (int)((key >> 48) & 255u);
            w = (int)(key >> 56);
            const unsigned long long bits = key & ((1ull << 48) - 1ull);
            const uint32_t wmask = (w >= 32) ? FULL : ((1u << w) - 1u);
            if (lane < h) row = (uint32_t)(bits >> (lane * w)) & wmask;
            want = (uint32_t)meta;
            check = true;
        } else {
            const unsigned long long j = i - nslots;
            const unsigned m = spill.meta[j];
            h = (int)(m >> 8);
            w = (int)(m & 255u);
            row = spill.rows[j * 32 + lane];
        }
        const uint32_t hv = crop_shape_hash(row, h, w, lane, false, tab);
        if (check && hv != want && lane == 0) atomicAdd(&tab.stats[1], 1u);
    }
    if (spill.rows && blockIdx.x == 0 && threadIdx.x == 0 && *spill.count > spill.cap) atomicAdd(&tab.stats[2], 1u);
}

// move the used slots into a dense list and leave the table empty again
__global__ void hist_compact_kernel(Table t, Compact c, unsigned *nkeys, ShapeTab shapes)
{
    const unsigned cap = 1u << t.cap_log2;
    for (unsigned i = blockIdx.x * blockDim.x + threadIdx.x; i < cap; i += gridDim.x * blockDim.x) {
        const unsigned long long k = t.key[i];
        if (k == EMPTY_KEY) continue;
        const unsigned cls = (unsigned)(k >> 32);
        if (shapes.key && (cls == JATAM_DET_BOUNDED || cls == JATAM_ND_STERIC) && t.size_min[i] == 1u)
            shape_record_cell(shapes, (uint32_t)k);
        const unsigned j = atomicAdd(nkeys, 1u);
        c.key[j] = k;
        c.count[j] = t.count[i];
        c.min_id[j] = t.min_id[i];
        c.size_max[j] = t.size_max[i];
        c.size_min[j] = t.size_min[i];
        t.key[i] = EMPTY_KEY;
        t.count[i] = 0ull;
        t.min_id[i] = ~0ull;
        t.size_max[i] = 0u;
        t.size_min[i] = 0xFFFFFFFFu;
    }
}

// rank every key among all keys (keys are distinct) and write the sorted histogram
__global__ void hist_emit_kernel(Compact c, const unsigned *nkeys, jatam_hist_entry *hist, unsigned cap,
                                 uint32_t *hist_len)
{
    constexpr int TILE = 1024;
    __shared__ unsigned long long tile[TILE];
    const unsigned nk = *nkeys;
    if (blockIdx.x == 0 && threadIdx.x == 0 && hist_len) *hist_len = nk;
    const unsigned per_block = blockDim.x;
    for (unsigned base = blockIdx.x * per_block; base < nk; base += gridDim.x * per_block) {
        const unsigned me = base + threadIdx.x;
        const unsigned long long mk = (me < nk) ? c.key[me] : EMPTY_KEY;
        unsigned rank = 0;
        for (unsigned t0 = 0; t0 < nk; t0 += TILE) {
            __syncthreads();
            for (unsigned j = threadIdx.x; j < TILE && t0 + j < nk; j += blockDim.x) tile[j] = c.key[t0 + j];
            __syncthreads();
            const unsigned lim = min((unsigned)TILE, nk - t0);
            for (unsigned j = 0; j < lim; ++j) rank += (tile[j] < mk) ? 1u : 0u;
        }
        if (me < nk && rank < cap) {
            jatam_hist_entry e;
            e.cls = (uint32_t)(mk >> 32);
            e.shape_hash = (uint32_t)mk;
            e.size = c.size_max[me];
            e.flags = (c.size_max[me] != c.size_min[me]) ? 1u : 0u;
            e.count = c.count[me];
            e.min_id = c.min_id[me];
            hist[rank] = e;
        }
    }
}

__global__ void philox_kernel(const uint32_t *in, unsigned long long n, uint32_t *out)
{
    for (unsigned long long i = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; i < n;
         i += (unsigned long long)gridDim.x * blockDim.x) {
        const uint32_t *r = in + 6 * i;
        const uint4 w = philox4x32_10(make_uint4(r[0], r[1], r[2], r[3]), r[4], r[5]);
        out[4 * i + 0] = w.x;
        out[4 * i + 1] = w.y;
        out[4 * i + 2] = w.z;
        out[4 * i + 3] = w.w;
    }
}

template <int S, int NT>
int smem_bytes_for(int warps) { return warps * Geo<S, NT>::WORDS * 32 * 4; }

// the instance for lattice template S, tuple-table size nt and process
template <int S, int NT, typename F>
auto with_process(bool lifo, F f)
{
    if (lifo) return f(classify_kernel<S, NT, true>, smem_bytes_for<S, NT>);
    return f(classify_kernel<S, NT, false>, smem_bytes_for<S, NT>);
}

template <typename F>
auto with_instance(int S, int nt, bool lifo, F f)
{
    if (nt == 8) {
        switch (S) {
        case 8: return with_process<8, 8>(lifo, f);
        case 16: return with_process<16, 8>(lifo, f);
        default: return with_process<32, 8>(lifo, f);
        }
    }
    switch (S) {
    case 8: return with_process<8, 16>(lifo, f);
    case 16: return with_process<16, 16>(lifo, f);
    default: return with_process<32, 16>(lifo, f);
    }
}

}  // namespace

int classify_smem_bytes(int S, int nt, int warps_per_cta)
{
    return with_instance(S, nt, false, [&](auto, auto bytes_for) { return bytes_for(warps_per_cta); });
}

cudaError_t classify_set_attributes(int S, int nt, int warps_per_cta, bool lifo)
{
    // The kernel's dynamic shared-memory limit is per device and shared by every
    // caller of the library, so it only ever grows: a caller that needs less
    // never lowers it under a launch that needs more.
    static std::mutex mu;
    static std::map<std::tuple<int, int, int, int>, int> limit;  // (device, S, nt, process) -> bytes set
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    const int bytes = classify_smem_bytes(S, nt, warps_per_cta);
    std::lock_guard<std::mutex> lock(mu);
    int &have = limit[std::make_tuple(dev, S, nt, lifo ? 1 : 0)];
    if (bytes <= have) return cudaSuccess;
    e = with_instance(S, nt, lifo, [&](auto kernel, auto) {
        return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    });
    if (e == cudaSuccess) have = bytes;
    return e;
}

cudaError_t classify_occupancy(int S, int nt, int warps_per_cta, int *blocks_per_sm, bool lifo)
{
    return with_instance(S, nt, lifo, [&](auto kernel, auto bytes_for) {
        return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, kernel, warps_per_cta * 32,
                                                             bytes_for(warps_per_cta));
    });
}

int default_warps_per_cta(int S, int nt)
{
    // the CTA size that keeps the most warps resident on an SM (ties: the larger CTA)
    static int cache[2][3] = {{0, 0, 0}, {0, 0, 0}};
    int &c = cache[nt == 8 ? 0 : 1][S == 8 ? 0 : S == 16 ? 1 : 2];
    if (c) return c;
    int best = 1, best_warps = 0;
    for (int w = MAX_CTA_WARPS; w >= 1; --w) {
        if (classify_smem_bytes(S, nt, w) > 200 * 1024) continue;
        if (classify_set_attributes(S, nt, w, false) != cudaSuccess) {  // the occupancy query needs the limit
            cudaGetLastError();
            continue;
        }
        int per_sm = 0;
        if (classify_occupancy(S, nt, w, &per_sm, false) != cudaSuccess) {
            cudaGetLastError();
            continue;
        }
        if (per_sm * w > best_warps) {
            best_warps = per_sm * w;
            best = w;
        }
    }
    c = best;
    return c;
}

namespace {
// the replicate-lanes instance for lattice template S (8 or 16) and tuple-table size nt
template <typename F>
auto with_reps_instance(int S, int nt, F f)
{
    if (nt == 8) {
        if (S == 8) return f(classify_reps_kernel<8, 8>, smem_bytes_for<8, 8>);
        return f(classify_reps_kernel<16, 8>, smem_bytes_for<16, 8>);
    }
    if (S == 8) return f(classify_reps_kernel<8, 16>, smem_bytes_for<8, 16>);
    return f(classify_reps_kernel<16, 16>, smem_bytes_for<16, 16>);
}
}  // namespace

cudaError_t classify_reps_prepare(int S, int nt, int warps_per_cta, int *blocks_per_sm)
{
    static std::mutex mu;
    static std::map<std::tuple<int, int, int>, int> limit;  // (device, S, nt) -> bytes set (grow-only)
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    {
        std::lock_guard<std::mutex> lock(mu);
        const int bytes = with_reps_instance(S, nt, [&](auto, auto bytes_for) { return bytes_for(warps_per_cta); });
        int &have = limit[std::make_tuple(dev, S, nt)];
        if (bytes > have) {
            e = with_reps_instance(S, nt, [&](auto kernel, auto) {
                return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
            });
            if (e != cudaSuccess) return e;
            have = bytes;
        }
    }
    return with_reps_instance(S, nt, [&](auto kernel, auto bytes_for) {
        return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, kernel, warps_per_cta * 32,
                                                             bytes_for(warps_per_cta));
    });
}

cudaError_t launch_classify_reps(const LaunchArgs &a, int S, int nt, int blocks, int warps_per_cta, cudaStream_t st)
{
    return with_reps_instance(S, nt, [&](auto kernel, auto bytes_for) {
        kernel<<<dim3(blocks), dim3(warps_per_cta * 32), bytes_for(warps_per_cta), st>>>(a);
        return cudaGetLastError();
    });
}

cudaError_t launch_classify(const LaunchArgs &a, int S, int nt, int blocks, int warps_per_cta, cudaStream_t st)
{
    return with_instance(S, nt, a.lifo_stack != nullptr, [&](auto kernel, auto bytes_for) {
        kernel<<<dim3(blocks), dim3(warps_per_cta * 32), bytes_for(warps_per_cta), st>>>(a);
        return cudaGetLastError();
    });
}

int classify_mixed_smem_bytes(int w32, int w16, int w8)
{
    return (w32 * Geo<32>::WORDS + w16 * Geo<16>::WORDS + w8 * Geo<8>::WORDS) * 32 * 4;
}

cudaError_t classify_mixed_prepare(int w32, int w16, int w8, int *blocks_per_sm)
{
    const int bytes = classify_mixed_smem_bytes(w32, w16, w8);
    {
        // grow-only, as for classify_kernel: a smaller plan never lowers the limit
        // under a captured launch of a larger one
        static std::mutex mu;
        static std::map<int, int> limit;  // device -> bytes set
        int dev = 0;
        cudaError_t e = cudaGetDevice(&dev);
        if (e != cudaSuccess) return e;
        std::lock_guard<std::mutex> lock(mu);
        int &have = limit[dev];
        if (bytes > have) {
            e = cudaFuncSetAttribute(classify_mixed_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
            if (e != cudaSuccess) return e;
            have = bytes;
        }
    }
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, classify_mixed_kernel, (w32 + w16 + w8) * 32,
                                                         bytes);
}

cudaError_t launch_classify_mixed(const LaunchArgs &a, int blocks, cudaStream_t st)
{
    const int warps = a.plan_w32 + a.plan_w16 + a.plan_w8;
    classify_mixed_kernel<<<blocks, warps * 32, classify_mixed_smem_bytes(a.plan_w32, a.plan_w16, a.plan_w8), st>>>(a);
    return cudaGetLastError();
}

cudaError_t classify_warp_occupancy(int *blocks_per_sm, int *warps_per_cta)
{
    *warps_per_cta = WG_WARPS;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, classify_warp_kernel, WG_WARPS * 32, 0);
}

cudaError_t launch_classify_warp(const LaunchArgs &a, int blocks, cudaStream_t st)
{
    classify_warp_kernel<<<blocks, WG_WARPS * 32, 0, st>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_reset(unsigned long long *work_next, unsigned *nkeys, unsigned long long *list_count,
                         cudaStream_t st, unsigned long long *crops, unsigned crops_log2, unsigned long long *extra,
                         int extra_words)
{
    const unsigned words = crops ? (2u << crops_log2) : 0u;
    reset_kernel<<<crops ? 16 : 1, 256, 0, st>>>(work_next, nkeys, list_count, crops, words, extra,
                                                  extra ? extra_words : 0);
    return cudaGetLastError();
}

cudaError_t load_index_range_kernels()
{
    // cudaFuncGetAttributes loads a kernel that lazy module loading has not yet loaded
    cudaFuncAttributes fa;
    cudaError_t e = cudaFuncGetAttributes(&fa, reset_kernel);
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, prefilter_kernel<false>);
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, prefilter_kernel<true>);
    return e;
}

cudaError_t launch_prefilter(const LaunchArgs &a, int smax, int blocks, cudaStream_t st)
{
    // the seed table covers genotypes (not records) of one or two tiles of 3-bit colours
    if (a.mode != MODE_RECORDS && !a.bucket && a.n >= 1 && a.n <= 2 && a.c == 8)
        prefilter_kernel<true><<<blocks, 256, 0, st>>>(a, smax);
    else
        prefilter_kernel<false><<<blocks, 256, 0, st>>>(a, smax);
    return cudaGetLastError();
}

cudaError_t launch_table_init(Table t, cudaStream_t st)
{
    table_init_kernel<<<256, 256, 0, st>>>(t);
    return cudaGetLastError();
}

cudaError_t launch_shape_scan(ShapeTab shapes, const unsigned long long *crops, unsigned crops_log2, CropSpill spill,
                              cudaStream_t st)
{
    shape_scan_kernel<<<128, 256, 0, st>>>(shapes, crops, crops_log2, spill);
    return cudaGetLastError();
}

cudaError_t launch_hist_compact(Table t, Compact c, unsigned *nkeys, int blocks, cudaStream_t st, ShapeTab shapes)
{
    hist_compact_kernel<<<blocks, 256, 0, st>>>(t, c, nkeys, shapes);
    return cudaGetLastError();
}

cudaError_t launch_hist_emit(Compact c, const unsigned *nkeys, jatam_hist_entry *hist, unsigned cap,
                             uint32_t *hist_len, int blocks, cudaStream_t st)
{
    hist_emit_kernel<<<blocks, 256, 0, st>>>(c, nkeys, hist, cap, hist_len);
    return cudaGetLastError();
}

// Genome deduplication: a result depends only on the genome (its stream id is the genome), so a
// repeat takes the result of the item that owns the genome's slot; every used slot is emptied again
__global__ void __launch_bounds__(256) dup_fill_kernel(const LaunchArgs a)
{
    __shared__ SmemHist H;
    hist_begin(H);
    for (unsigned long long idx = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; idx < a.count;
         idx += (unsigned long long)gridDim.x * blockDim.x) {
        const unsigned sl = a.dup_slot[idx], h = sl & 0x7FFFFFFFu;
        if (sl >> 31) {
            const unsigned f = a.dup_owner[h];
            if (a.fitness) a.fitness[idx] = a.fitness[f];
            if (a.out) {
                const jatam_result res = a.out[f];
                a.out[idx] = res;
                if (a.use_hist && res.cls != 255)
                    hist_insert(H, a.table, ((unsigned long long)res.cls << 32) | res.shape_hash, 1u, a.genomes[idx],
                                res.size, res.size, a.err);
            }
        }
        a.dup_keys[h] = ~0ull;
    }
    hist_end(H, a);
}

cudaError_t launch_dup_fill(const LaunchArgs &a, int blocks, cudaStream_t st)
{
    if (a.count == 0) return cudaSuccess;
    dup_fill_kernel<<<blocks, 256, 0, st>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_orbit_fill(const LaunchArgs &a, int blocks, cudaStream_t st)
{
    if (a.count == 0) return cudaSuccess;
    orbit_fill_kernel<<<blocks, 256, 0, st>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_philox(const uint32_t *in, unsigned long long n, uint32_t *out, cudaStream_t st)
{
    if (n == 0) return cudaSuccess;
    const unsigned long long blocks = min((n + 255ull) / 256ull, 4096ull);
    philox_kernel<<<(unsigned)blocks, 256, 0, st>>>(in, n, out);
    return cudaGetLastError();
}

}  // namespace jatam
