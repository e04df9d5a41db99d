// Internal interface between the host API (jatam_api.cu) and the device code
// (jatam_kernels.cu) of libjatam.so.  Not part of the public C ABI.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "jatam.h"

namespace jatam {

// where the genotypes of a launch come from
enum Mode : int {
    MODE_RANGE = 0,    // packed genotype = index (S_{n,c} in order)
    MODE_SAMPLED = 1,  // packed genotype = Philox sample of the index
    MODE_RECORDS = 2,  // explicit colour records, optional per-item shapes and stream ids
    MODE_GENOMES = 3,  // packed genomes given in an array (genetic algorithm)
};

// device error bits (sticky until the host reads them at a synchronising call)
enum ErrBits : unsigned {
    ERR_TABLE_FULL = 1u,    // the phenotype table ran out of slots
    ERR_INVALID_ITEM = 2u,  // a record had a colour >= c or a parameter out of range
    ERR_GUARD = 4u,         // a bounded loop found an inconsistent state
};

constexpr unsigned long long EMPTY_KEY = ~0ull;

// Global phenotype table: open addressing, linear probing, capacity 2^cap_log2.
struct Table {
    unsigned long long *key;     // (cls << 32) | hash, EMPTY_KEY when free
    unsigned long long *count;
    unsigned long long *min_id;
    unsigned *size_max;
    unsigned *size_min;
    unsigned cap_log2;
};

// Compacted copy of the used table slots, filled by the compaction kernel.
struct Compact {
    unsigned long long *key;
    unsigned long long *count;
    unsigned long long *min_id;
    unsigned *size_max;
    unsigned *size_min;
};

// Exact side table of one call's shapes: for every shape hash the call
// computed, the canonical form it was computed from (open addressing by hash,
// 2^log2 slots).  key: 0 free, else 2^32 | hash; meta: 0 until the inserting
// warp has written the rows, then 2^31 | h << 8 | w; rows[32 slot + i]: row i
// of the canonical form, its first cell in bit w - 1.  stats: [0] computed
// forms that differed from the one stored under their hash (collisions),
// [1] comparisons given up (a bounded wait for the rows ran out), [2] forms not
// stored (the table was full).  key == nullptr: no table.
struct ShapeTab {
    unsigned long long *key;
    unsigned *meta;
    uint32_t *rows;
    unsigned *stats;
    unsigned log2;
};

// Crops whose form a growth kernel computed but whose crop the call's crop
// table does not hold (more than 48 cells, or no free slot): rows[32 i + r] is
// row r of crop i (bit j = column j), meta[i] = h << 8 | w; *count entries
// (counted past cap when full).  The side table of shapes takes their forms,
// and those of every crop in the crop table, in a pass after the growth
// kernels, so that the growth kernels carry none of its code.
struct CropSpill {
    uint32_t *rows;
    unsigned *meta;
    unsigned long long *count;
    unsigned cap;
};

struct LaunchArgs {
    int mode;
    unsigned long long first;     // first index (MODE_RANGE / MODE_SAMPLED)
    unsigned long long count;     // items
    const uint8_t *colours;       // MODE_RECORDS: [count][16]
    const uint8_t *shapes;        // MODE_RECORDS: [count][4] or null
    const unsigned long long *ids;      // MODE_RECORDS: stream ids or null
    const unsigned long long *genomes;  // MODE_GENOMES: [count]
    int n, c, L, k;               // uniform parameters (records may override)
    uint32_t key0, key1;          // Philox key
    jatam_result *out;            // [count] or null
    int32_t *fitness;             // [count] or null
    Table table;
    int use_hist;
    int c4;                       // 1: the rotation-only hash variant instead of the canonical form
    int orbits;                   // 1: orbit mode (one classification per orbit of the exact symmetries)
    int lifo;                     // 1: the movelist process (the host sets lifo_stack)
    uint16_t *lifo_stack;         // movelist process: S * S cells of stack per thread of the growth launch; null:
                                  // the row-major process
    int stop_at;                    // finished lanes that end a growth round (1..32)
    unsigned long long *list;        // items left to grow, written by the pre-filter: 1 or 3 lists
    unsigned long long list_stride;  // capacity of one list (the call's item count)
    unsigned long long *list_count;  // [6]: items at the front of regions 0..2 of `list`, then items stored from their ends
    int bucket;                      // 1: lists by lattice size class (<= 8, <= 16, <= 32); 0: one list
    int klass;                       // classify_kernel: the list it works through
    int plan_w32, plan_w16, plan_w8; // classify_mixed_kernel: warps per CTA of each region size
    unsigned long long *work_next;  // [3] work counters (one per list), zeroed before the launch
    unsigned long long *stats;      // null, or [4] executed work: drawn placements, seed placements,
                                    // lane slots of the growth rounds, genotypes grown by warps
    unsigned *err;                  // sticky error bits
    int heavy_first;                // 1: the pre-filter lists the genotypes with two or more frontier
                                    // sites after the seed first (one size class only); 2: three levels --
                                    // three or four sites first, then two (region 1 of the list), then one
    unsigned long long *crops;      // null, or the crop table of the launch: 2^crops_log2 slots of
                                    // {crop bits, valid | h | w | hash}, cleared by the call's reset
    unsigned crops_log2;
    CropSpill spill;                // uncacheable crops of a call that keeps a side table of shapes (rows
                                    // null: none)
    unsigned long long *esc_list;   // non-null: window mode -- the items' lattice (L > S) is grown in the
                                    // S x S window around the seed; an item whose growth offers a tile
                                    // outside the window is not classified here but appended to esc_list
    unsigned long long *esc_count;  // (count in *esc_count) for a launch on the full lattice
    unsigned long long *dup_keys;   // non-null: genome deduplication -- an open-addressing table of the
    unsigned *dup_owner;            // call's genomes (keys ~0 = empty, 2^k >= 2 count slots, dup_mask =
    unsigned *dup_slot;             // 2^k - 1): the item that claims a genome's slot classifies it
    unsigned dup_mask;              // (dup_owner), a repeat records its slot with the top bit set
                                    // (dup_slot) and takes the owner's result in the fill pass
    int no_dedup;                   // JATAM_NO_DEDUP: every genome classified
};

// Lattice template: rows of S bits, S in {8, 16, 32}, L <= S; nt = 8 tuple ids
// (sets of at most two tiles, uniform launches only) or 16.
int classify_smem_bytes(int S, int nt, int warps_per_cta);
cudaError_t classify_set_attributes(int S, int nt, int warps_per_cta, bool lifo = false);
cudaError_t classify_occupancy(int S, int nt, int warps_per_cta, int *blocks_per_sm, bool lifo = false);
cudaError_t launch_classify(const LaunchArgs &a, int S, int nt, int blocks, int warps_per_cta, cudaStream_t st);
// replicate lanes (S = 8 or 16, k <= 32): one genotype per warp, lane r grows replicate r;
// prepare sets the shared-memory limit (grow-only) and returns the CTAs an SM holds
cudaError_t classify_reps_prepare(int S, int nt, int warps_per_cta, int *blocks_per_sm);
cudaError_t launch_classify_reps(const LaunchArgs &a, int S, int nt, int blocks, int warps_per_cta, cudaStream_t st);
// largest CTA of classify_kernel (its launch bounds hold it to 113 registers so
// that three such CTAs fit an SM)
constexpr int MAX_CTA_WARPS = 6;
// pre-filter grid: at most this many 256-thread CTAs per SM (five are resident at
// a time; many short CTAs end the launch with a short last wave)
constexpr long long PF_CTAS_PER_SM = 48;
// warps per CTA that keep the most warps resident on an SM
int default_warps_per_cta(int S, int nt);
// tuple-table size of a uniform launch of n-tile sets
inline int tuple_table_size(int n) { return (n >= 1 && n <= 2) ? 8 : 16; }
// finished lanes that end a growth round when nothing is tuned (measured on
// S_{2,8} at L = 16 and 19 and on S_{3,8} at L = 32; 18 for the 8 x 8 and
// 16 x 16 templates since the three-level heavy-first order: S_{2,8} growth
// kernel 2.11 ms at 14, 2.09 at 16, 2.085 at 18, 2.10 at 20, 2.15 at 22)
inline int default_stop_at(int S) { return S == 32 ? 12 : 18; }
// one genotype per warp (lattices up to 32 x 32, the row-major process): CTAs of
// *warps_per_cta warps, no dynamic shared memory
cudaError_t classify_warp_occupancy(int *blocks_per_sm, int *warps_per_cta);
cudaError_t launch_classify_warp(const LaunchArgs &a, int blocks, cudaStream_t st);
int classify_mixed_smem_bytes(int w32, int w16, int w8);
cudaError_t classify_mixed_prepare(int w32, int w16, int w8, int *blocks_per_sm);
cudaError_t launch_classify_mixed(const LaunchArgs &a, int blocks, cudaStream_t st);

// also zeroes extra[0 .. extra_words) when given
cudaError_t launch_reset(unsigned long long *work_next, unsigned *nkeys, unsigned long long *list_count,
                         cudaStream_t st, unsigned long long *crops = nullptr, unsigned crops_log2 = 0,
                         unsigned long long *extra = nullptr, int extra_words = 0);
cudaError_t launch_prefilter(const LaunchArgs &a, int smax, int blocks, cudaStream_t st);
// load the reset and pre-filter kernels on the current device now (not at their first launch)
cudaError_t load_index_range_kernels();
// jatam_shutdown: forget the per-device set-up of jatam_enumerate_noalloc
void noalloc_forget_devices();
cudaError_t launch_table_init(Table t, cudaStream_t st);
// the side table of shapes from the crop table (2^crops_log2 slots) and the spill list of one call or piece
cudaError_t launch_shape_scan(ShapeTab shapes, const unsigned long long *crops, unsigned crops_log2, CropSpill spill,
                              cudaStream_t st);
// also records the single-cell shape in `shapes` when a size-1 key is present
// (the pre-filter settles those genotypes without computing a canonical form)
cudaError_t launch_hist_compact(Table t, Compact c, unsigned *nkeys, int blocks, cudaStream_t st,
                                ShapeTab shapes = ShapeTab{});
cudaError_t launch_hist_emit(Compact c, const unsigned *nkeys, jatam_hist_entry *hist, unsigned cap,
                             uint32_t *hist_len, int blocks, cudaStream_t st);
cudaError_t launch_philox(const uint32_t *in, unsigned long long n, uint32_t *out, cudaStream_t st);
cudaError_t launch_orbit_fill(const LaunchArgs &a, int blocks, cudaStream_t st);
// genome deduplication (MODE_GENOMES): after the growth kernels, every repeat copies its owner's
// result, and every used slot of the table is emptied again (the table must be all empty before
// the first call that uses it)
cudaError_t launch_dup_fill(const LaunchArgs &a, int blocks, cudaStream_t st);

// genetic algorithm (jatam_ga.cu)
struct GaArgs {
    int n, c, b, bits;           // genome space: 4 n b bits, b = log2(c)
    int selection, tournament, crossover;
    uint32_t crossover_threshold;
    uint32_t mutation_thresholds[4];
    uint32_t key0, key1;
    const unsigned long long *parents;
    const int32_t *fitness;
    const unsigned long long *cumsum;  // roulette: workspace for the prefix sum of the fitness
    unsigned long long N;         // parents
    unsigned long long Nc;        // children to breed (child indices 0 .. Nc-1)
    uint32_t generation;
    unsigned long long *children;
};
cudaError_t launch_ga_breed(const GaArgs &g, cudaStream_t st);
cudaError_t launch_ga_hamming(const unsigned long long *genomes, unsigned long long n, int32_t *fitness,
                              cudaStream_t st);
cudaError_t launch_ga_stats(const int32_t *fitness, unsigned long long n, long long *stats, cudaStream_t st);

// surrogate network (jatam_mlp.cu): 36 -> 256 -> 256 -> 8, inputs padded to 48
constexpr int MLP_IN = 36, MLP_PAD = 48, MLP_H = 256, MLP_OUT = 8;
extern const long long MLP_OFF_W1, MLP_OFF_B1, MLP_OFF_W2, MLP_OFF_B2, MLP_OFF_W3, MLP_OFF_B3, MLP_NPARAM;

}  // namespace jatam
#include <cuda_bf16.h>
namespace jatam {

struct MlpBuffers {
    float *p, *grad, *m, *v;     // [MLP_NPARAM] master parameters, gradients, Adam moments
    __nv_bfloat16 *wq;           // [MLP_NPARAM] bfloat16 copy of the parameters (weights used by the products)
    __nv_bfloat16 *wqt;          // W1 and W2 transposed (K contiguous) for the tcgen05 products: [256 x 48 + 256 x 256]
    long long cap;               // batch capacity of the activation buffers
    __nv_bfloat16 *x, *h1, *h2, *dq, *dh1, *dh2;
    float *logits, *d, *lrow, *loss;  // lrow: the softmax blocks' partial sums (loss, output bias gradient)
    float *splitk;               // [MLP_SPLITK_MAX][256 x 256] partial weight gradients (split-K)
    unsigned *tc_err;            // error bits of the tcgen05 products (a bounded wait that ran out)
    int tc;                      // 1: products with 256 columns on tcgen05; 0: all on mma.sync
};
// D[M x 256] = A[M x K] B[K x 256] on tcgen05 (jatam_tc.cu); epi 0: bias + ReLU,
// 1: ReLU mask; 2: bias + ReLU, then logits[M x 8] = bf16(D) W3 + b3 instead of D; 3: both D (as 0)
// and the logits (as 2);
// K a multiple of 16, at most 256, both operands K-contiguous
cudaError_t tc_gemm_n256(const __nv_bfloat16 *A, long long a_m, long long a_k, const __nv_bfloat16 *B, long long b_k,
                         long long b_n, int M, int K, int epi, const float *bias, const __nv_bfloat16 *mask,
                         __nv_bfloat16 *C, unsigned *err, cudaStream_t st, const __nv_bfloat16 *w3 = nullptr,
                         const float *b3 = nullptr, float *logits = nullptr);
constexpr int MLP_SPLITK_MAX = 32;
// logits_only: the caller needs the logits alone (no backward pass follows), so the second hidden
// layer is not stored: its tensor-core epilogue computes the logits
cudaError_t mlp_forward(const MlpBuffers &b, const unsigned long long *genomes, long long B, cudaStream_t st,
                        bool logits_only = false);
cudaError_t mlp_backward(const MlpBuffers &b, const uint8_t *labels, long long B, cudaStream_t st);
cudaError_t mlp_adam(const MlpBuffers &b, float lr, int t, cudaStream_t st);
cudaError_t mlp_refresh_bf16(const MlpBuffers &b, cudaStream_t st);
cudaError_t launch_mlp_labels(const jatam_result *res, long long n, uint8_t *labels, cudaStream_t st);
cudaError_t launch_embed(const unsigned long long *in, long long n, int tiles, int bits_per_colour,
                         unsigned long long *out, cudaStream_t st);
// scratch of the screen's de-duplication: a table of cap_mask + 1 (a power of
// two >= 2n) slots and the slot of each of the n candidates
struct ScreenTable {
    unsigned long long *keys;
    unsigned *first, *slot, *err;
    unsigned cap_mask;
    unsigned *topn;  // TOPN_SCRATCH_BYTES of scratch for the selection
};
// scratch of the many-CTA selection: a 4096-bin histogram, 16 control words, two counts a CTA
constexpr size_t TOPN_SCRATCH_BYTES = (4096 + 16) * 4 + 2 * 1024 * 8;
// indices of the `keep` largest non-negative scores (ties: lower index first), in increasing order
// (scratch: TOPN_SCRATCH_BYTES, 16-byte aligned)
cudaError_t launch_topn_multi(const float *score, long long n, long long keep, unsigned long long *idx,
                              unsigned *scratch, cudaStream_t st);
// scores of n candidates from their logits: the network's probability of a
// deterministic bounded shape of >= 8 tiles, plus one for the first occurrence
// of each distinct genome (repeats rank below every distinct genome); idx = the
// `keep` best (ties: lower index), chosen = cand[idx]
cudaError_t launch_screen(const float *logits, long long n, long long keep, float *score, unsigned long long *idx,
                          const unsigned long long *cand, unsigned long long *chosen, const ScreenTable &t,
                          cudaStream_t st);

// the message returned by jatam_last_error() for the calling thread
void set_last_error(const char *msg);

}  // namespace jatam
