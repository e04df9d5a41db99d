/*
 * jatam.h -- C ABI of libjatam.so: batched stochastic tile self-assembly and
 * phenotype classification of JaTAM genotypes on one GB300 (sm_103a).
 *
 * The model is the one of the paper (arXiv 2205.15311, "Modifications to
 * Winfree's aTAM" and Section 1.1): square tiles with four coloured edges
 * (N, E, S, W), colours binding in adjacent pairs 1-2, 3-4, 5-6 (0 inert,
 * other pairs neutral), temperature 1, rotations allowed and mirror images
 * not, the first tile of the set as seed at the centre of an L x L grid, every
 * tile type unlimited.  For every genotype the library grows k replicate
 * assemblies, flags local non-determinism (two distinct tiles fit one site,
 * Section 2.4), unbounded growth (a tile fits outside the grid, appendix
 * "Modifications to Winfree's aTAM"), and steric non-determinism (a replicate
 * ends in a configuration different from replicate 0's, Section 2.4); a
 * genotype with none of these is deterministic and bounded.  The shape of
 * replicate 0 is put in canonical form under the 8 symmetries of the square
 * and hashed with Jenkins' one-at-a-time hash (Section 2.5), and the genotypes
 * are binned by (class, hash) into a phenotype histogram (Section 2.6).
 *
 * The random draws are fixed: step s of replicate j of the genotype with
 * stream id g uses word (s mod 4) of Philox4x32-10 with counter
 * (s >> 2, j, g_lo, g_hi) and key (seed_lo, seed_hi), and picks frontier site
 * floor(u * |F| / 2^32) of the frontier F in row-major order.  Results are
 * therefore bit-identical whatever the launch configuration.
 *
 * Conventions for every call
 *   - returns JATAM_OK (0) or a negative JATAM_E* code; jatam_last_error()
 *     gives a message for the calling thread's last failure;
 *   - buffers belong to the caller.  Each pointer may be device memory or host
 *     memory (pinned or pageable); the library detects which with
 *     cudaPointerGetAttributes and stages host buffers through device memory;
 *   - work is queued on the CUDA stream `stream` (NULL = legacy default
 *     stream).  The call returns before the work ends unless a host output
 *     buffer was given or cfg->flags has JATAM_SYNC; in those cases it waits
 *     for the stream and also reports errors found on the device;
 *   - a classification of at least 2^23 items whose results (or fitness
 *     values) go to page-locked host memory runs in pieces on two internal
 *     streams, each piece's results copied on a third while the next piece is
 *     classified; `stream` waits for all of it before the call returns, and the
 *     results equal the one-pass call's (not for records without stream ids,
 *     JATAM_ORBITS, JATAM_LIFO, JATAM_GRAPH or the profiling mode);
 *   - the library owns one workspace per device (the histogram table, counters
 *     and staging buffers); calls on one device are serialised through it, in
 *     the order they were made, whatever their streams.  jatam_shutdown()
 *     frees it.
 */
#ifndef JATAM_H
#define JATAM_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ---- */
#define JATAM_OK 0
#define JATAM_EINVAL (-1)       /* bad argument (size, range, null pointer, colour >= c, capacity) */
#define JATAM_ENOMEM (-2)       /* device allocation failed or the histogram table overflowed */
#define JATAM_ECUDA (-3)        /* a CUDA runtime call failed */
#define JATAM_ETIMEOUT (-4)     /* a bounded device-side loop gave up (internal invariant broken) */
#define JATAM_EUNSUPPORTED (-5) /* parameters outside the supported range (n > 4, c > 8, L > 32, k > 255) */

/* ---- phenotype classes ---- */
#define JATAM_DET_BOUNDED 0 /* every replicate ended in replicate 0's configuration */
#define JATAM_ND_LOCAL 1    /* two distinct rotated tiles fitted one empty site */
#define JATAM_ND_STERIC 2   /* a replicate ended in a configuration different from replicate 0's */
#define JATAM_UNBOUNDED 3   /* a tile fitted a site outside the L x L grid */

/* ---- jatam_config.flags ---- */
#define JATAM_SAMPLED 0x1u /* jatam_enumerate: index i names a uniformly sampled genotype (see below) */
#define JATAM_SYNC 0x2u    /* wait for the work to finish before returning */
#define JATAM_PER_SHAPE 0x4u /* jatam_classify_batch with mixed shapes: one fixed launch per lattice size
                                class instead of the single persistent launch */
#define JATAM_PERSISTENT 0x20u /* jatam_classify_batch with mixed shapes: the single persistent launch.
                                  Neither flag: the launch jatam_autotune_batch found faster
                                  (the persistent one until it has run) */
#define JATAM_C4_HASH 0x10u  /* the paper's rotation-only hash (Section 2.5): hash the 4 rotations of the
                                cropped shape, sort the 4 hashes, hash them again (16 bytes, little endian);
                                mirror images stay distinct.  Default: the canonical form under all 8
                                symmetries of the square */
#define JATAM_ORBITS 0x40u   /* jatam_enumerate over a range that starts at genotype 0: classify one
                                genotype per orbit of the exact symmetries of the process (colour
                                permutations that preserve the binding pairs, turns and permutations
                                of the non-seed tiles) and give every genotype its orbit
                                representative's result -- the smallest genotype of the orbit,
                                classified with itself as stream id.  With the draws fixed every
                                member assembles as the representative does, so this equals
                                classifying each genotype with the representative's stream id. */
#define JATAM_LIFO 0x80u     /* the movelist process of Section 2.4 instead of the uniform draw over the
                                row-major frontier: after each placement the sites that have just
                                become frontier sites, in the order N, E, S, W of the placed tile, are
                                pushed on a stack in a drawn order (permutation floor(u m! / 2^32) of
                                the m sites, factorial number system, first pick pushed first; u = word
                                s of the replicate's stream, s = placements after the seed so far) and
                                the next tile goes on the top site.  Items of one shape only (not the
                                mixed batches of jatam_classify_batch). */
#define JATAM_GRAPH 0x8u     /* capture the call's kernel sequence as a CUDA graph the first time a given
                                set of arguments is seen, and replay it on later calls with the same set */
#define JATAM_NO_DEDUP 0x100u /* ga_evaluate: classify every genome, also the repeats of a genome (by
                                default a batch's distinct genomes are classified once each and their
                                repeats copy the result, which is the same: a genome is its own stream
                                id); for batches known to hold no repeats, this saves the table pass */

/* Limits of the supported model sizes. */
#define JATAM_MAX_TILES 4
#define JATAM_MAX_COLOURS 8
#define JATAM_MAX_GRID 32
#define JATAM_MAX_REPLICATES 255

typedef struct {
    uint8_t n;      /* tile types, 1..4 (the seed is tile 0) */
    uint8_t c;      /* colours 0..c-1, 1..8 (a power of two for packed genotypes) */
    uint8_t L;      /* grid side, 1..32; the seed sits at (L/2, L/2) */
    uint8_t k;      /* replicate assemblies per genotype, 1..255 */
    uint32_t flags; /* JATAM_SAMPLED | JATAM_SYNC */
    uint64_t seed;  /* Philox key (low word, high word) */
} jatam_config;     /* 16 bytes */

typedef struct {
    uint8_t cls;         /* JATAM_DET_BOUNDED .. JATAM_UNBOUNDED */
    uint8_t decided_rep; /* replicate that decided a non-deterministic or unbounded class; k otherwise */
    uint16_t size;       /* tiles in replicate 0's final shape (classes 0 and 2), else 0 */
    uint32_t shape_hash; /* one-at-a-time hash of the canonical shape (classes 0 and 2), else 0 */
} jatam_result;          /* 8 bytes */

typedef struct {
    uint32_t cls;        /* class */
    uint32_t shape_hash; /* hash (0 for classes 1 and 3) */
    uint32_t size;       /* shape size; the largest seen if genotypes disagreed */
    uint32_t flags;      /* bit 0: genotypes with this key disagreed on the size (a hash collision) */
    uint64_t count;      /* genotypes with this (class, hash) */
    uint64_t min_id;     /* smallest stream id among them */
} jatam_hist_entry;      /* 32 bytes; a histogram is sorted by (cls, shape_hash) */

/*
 * jatam_enumerate -- classify genotypes first .. first+count-1 of the packed
 * space S_{n,c} (Section 2.1 "Binary encodings" and the appendix "Encoding
 * genome information": tiles seed first, each N, E, S, W, log2(c) bits per
 * colour, the first tile's N edge in the most significant bits).
 *   cfg      : n, c (power of two), L, k, seed, flags.  Without JATAM_SAMPLED
 *              index i is the genotype value itself.  With it, genotype i is
 *              words 0 and 1 of Philox4x32-10(ctr = (0, 1 << 24, i_lo, i_hi),
 *              key = seed) as (w1 << 32 | w0), masked to the 4 n log2(c) bits.
 *              The stream id of each genotype is its value.
 *   first, count : index range; first + count must not exceed 2^(4 n log2 c)
 *              for the in-order space.  count may be 0.
 *   out      : NULL or [count] results, out[i] for index first + i.
 *   hist     : NULL or [hist_cap] histogram entries of this call, sorted.
 *   hist_len : with hist, receives the number of distinct keys (which may
 *              exceed hist_cap: then only hist_cap entries are written and,
 *              when hist_len is host memory, JATAM_EINVAL is returned).
 *   stream   : cudaStream_t or NULL.
 */
int jatam_enumerate(const jatam_config *cfg, uint64_t first, uint64_t count, jatam_result *out,
                    jatam_hist_entry *hist, uint32_t hist_cap, uint32_t *hist_len, void *stream);

/*
 * jatam_last_shapes -- the exact side table of the phenotype histogram
 * (Section 2.5: shapes are binned by a 32-bit one-at-a-time hash, and the
 * paper estimates how likely two distinct shapes are to share one; this
 * table checks it exactly).  Every call on the current device that builds a
 * histogram with the canonical-form hash (not JATAM_C4_HASH) records, for
 * every shape hash of its histogram, the canonical form the hash was computed
 * from; every later computation of the same hash in that call compares its
 * own canonical form with the stored one and counts a collision when they
 * differ.  This call returns that table for the last such call on the device
 * (it waits for that call to finish).
 *   shapes : [cap] entries sorted by shape_hash (cap may be 0).
 *   len    : receives the number of distinct shape hashes.
 *   collisions : receives the number of canonical forms that differed from
 *            the form stored under their hash (0: every hash names one shape).
 * Returns JATAM_EINVAL if the last call on the device recorded no shapes or
 * cap < *len (the first cap entries are still written), JATAM_ENOMEM if the
 * table (16,384 hashes) overflowed.
 */
typedef struct {
    uint32_t shape_hash; /* hash of the histogram keys (class 0 or 2) with this shape */
    uint8_t h, w;        /* height and width of the canonical form */
    uint16_t size;       /* occupied cells */
    uint32_t rows[32];   /* row i < h of the canonical form: bit j set = cell (column j, row i) occupied */
} jatam_shape;           /* 136 bytes */
int jatam_last_shapes(jatam_shape *shapes, uint32_t cap, uint32_t *len, uint32_t *collisions);

/*
 * jatam_classify_batch -- classify N explicit tile sets (Section 2.6: a batch
 * of assemblies, hashed and binned).
 *   colours    : [N][16] uint8, colour of edge e of tile t at [i][4 t + e]
 *                (N, E, S, W); entries beyond 4 n are ignored.
 *   shapes     : NULL (every item uses cfg->n, c, L, k) or [N][4] uint8 giving
 *                each item's (n, c, L, k) -- batches may mix them.
 *   stream_ids : NULL (item i uses stream id i) or [N] uint64.
 *   out, hist, hist_cap, hist_len, stream : as for jatam_enumerate.
 * Items with a colour >= c or parameters out of range get cls = 255 and the
 * call reports JATAM_EINVAL once the work has finished.
 * Mixed shapes run as one persistent launch: the pre-filter sorts the items
 * that grow into three lists by lattice size (L <= 8, <= 16, <= 32); warps
 * with 32 x 32, 16 x 16 and 8 x 8 shared-memory regions (a per-CTA plan that
 * jatam_autotune picks) work through their own list and then steal from the
 * lists of smaller sizes.  With JATAM_PER_SHAPE the three lists run as three
 * fixed launches instead; without either flag, as the autotuner chose.
 * Results are identical either way.
 */
int jatam_classify_batch(const jatam_config *cfg, const uint8_t *colours, const uint8_t *shapes,
                         const uint64_t *stream_ids, uint64_t N, jatam_result *out, jatam_hist_entry *hist,
                         uint32_t hist_cap, uint32_t *hist_len, void *stream);

/*
 * ga_evaluate -- fitness of a population of packed genomes for the genetic
 * algorithm (Section 2.2 and Section 3.2): genome i is decoded as in
 * jatam_enumerate, classified with stream id = its value, and
 *   fitness[i] = size of its shape if it is deterministic and bounded, else 0.
 *   genomes : [N] uint64 packed genomes (4 n log2(c) bits used).
 *   fitness : [N] int32, required.   out : NULL or [N] results.
 */
int ga_evaluate(const jatam_config *cfg, const uint64_t *genomes, uint64_t N, int32_t *fitness,
                jatam_result *out, void *stream);

/* ---- genetic algorithm (Section 2.2; Section 3.2 for the Fujiyama test bed) ---- */
#define JATAM_GA_TOURNAMENT 0
#define JATAM_GA_ROULETTE 1
#define JATAM_GA_NO_CROSSOVER 0
#define JATAM_GA_ONE_POINT 1
#define JATAM_GA_UNIFORM 2
#define JATAM_GA_FITNESS_SHAPE 0   /* size of the deterministic bounded shape, else 0 (ga_evaluate) */
#define JATAM_GA_FITNESS_HAMMING 1 /* number of set bits: the paper's Fujiyama landscape */

typedef struct {
    uint8_t n, c;                    /* genome space S_{n,c}, c a power of two: 4 n log2(c) bits */
    uint8_t selection;               /* JATAM_GA_TOURNAMENT or JATAM_GA_ROULETTE (global roulette wheel) */
    uint8_t tournament;              /* tournament size, 1..16 */
    uint8_t crossover;               /* JATAM_GA_NO_CROSSOVER, JATAM_GA_ONE_POINT or JATAM_GA_UNIFORM */
    uint8_t reserved[3];
    uint32_t crossover_threshold;    /* a child is a crossover when its draw u < threshold (u uniform 32-bit) */
    uint32_t mutation_thresholds[4]; /* mutation events on one edge = #{j : u >= t_j}, t non-decreasing */
    uint64_t seed;                   /* Philox key */
} jatam_ga_config;                   /* 40 bytes */

/*
 * ga_breed -- one generation: children[i] from parents and their fitness.
 * Two parents are selected (tournament: the fittest of `tournament` uniform
 * draws, the earliest on ties; roulette: the parent in whose slice of the
 * cumulative non-negative fitness a uniform dart lands, uniform if all are 0),
 * crossed over (one point: the bits above a uniform cut in 1..bits-1 from the
 * first parent, the rest from the second; uniform: a random 64-bit mask picks
 * each bit), and mutated: every edge undergoes a Poisson number of events
 * (the thresholds), each flipping one uniformly chosen bit of the edge.  Word k
 * of child i in generation g is word (k mod 4) of Philox4x32-10(ctr =
 * (k >> 2, (2 << 24) | g, i_lo, i_hi), key = seed), in the order: selection
 * words of parent A (T or 1), of parent B, crossover decision, two cut/mask
 * words, one Poisson word per edge, four bit-choice words per edge.
 * parents, fitness, children: [N], host or device; children may not alias
 * parents.  Roulette needs the total fitness below 2^32.
 */
int ga_breed(const jatam_ga_config *ga, const uint64_t *parents, const int32_t *fitness, uint64_t N,
             uint32_t generation, uint64_t *children, void *stream);

/* ga_hamming -- fitness[i] = number of set bits of genomes[i] (Section 3.2). */
int ga_hamming(const uint64_t *genomes, uint64_t N, int32_t *fitness, void *stream);

/* ga_poisson_thresholds -- t_j = floor(2^32 P(K <= j)), j = 0..3, for
 * K ~ Poisson(rate): the per-edge mutation thresholds for a mean of `rate`
 * events per edge (host only). */
int ga_poisson_thresholds(double rate, uint32_t thresholds[4]);

/*
 * ga_run -- `generations` generations of the genetic algorithm on the device:
 * per generation the fitness (JATAM_GA_FITNESS_SHAPE: classification with
 * cls->L, cls->k, cls->seed, as ga_evaluate; JATAM_GA_FITNESS_HAMMING: ga_hamming),
 * its best value and total, then ga_breed with generation index g.
 *   population : [N] device memory; in: generation 0, out: the last generation
 *                (after `generations` breedings).
 *   best, total: NULL or [generations] (host or device): the best fitness and
 *                the sum of fitness of generation g's population.
 * Synchronises `stream` when best/total are host memory.
 */
int ga_run(const jatam_ga_config *ga, const jatam_config *cls, int fitness_kind, uint64_t N, uint32_t generations,
           uint64_t *population, int32_t *best, int64_t *total, void *stream);

/* ---- surrogate network (a learned pre-screen; the paper has no network) ----
 * A multilayer perceptron over the 36 bits of an S_{3,8} genome (feature j =
 * bit 35 - j): 36 -> 256 -> 256 -> 8, ReLU, softmax cross-entropy over the 8
 * phenotype classes {unbounded, local non-determinism, steric
 * non-determinism, deterministic bounded of size 1, 2-3, 4-7, 8-15, >= 16}.
 * Products run on bfloat16 tensor cores with float32 accumulation; the master
 * parameters and Adam (beta 0.9 / 0.999, eps 1e-8) are float32.  Parameters
 * form one float32 vector: W1 [48][256] (input rows 36..47 unused), b1 [256],
 * W2 [256][256], b2 [256], W3 [256][8], b3 [8] -- JATAM_MLP_NPARAM floats. */
#define JATAM_MLP_NPARAM 80392
typedef struct jatam_mlp jatam_mlp;

/* Create a network with capacity for batches of up to max_batch genomes;
 * its parameters start at zero (set them with jatam_mlp_set_params).  Its
 * products with 256 output columns run on tcgen05 (accumulator in tensor
 * memory), the 8-column output layer on the CUDA cores (float32 dot products
 * of a row), the others on mma.sync; the environment variable
 * JATAM_MLP_PRODUCTS=mma, read here, keeps all of them on mma.sync. */
int jatam_mlp_create(uint64_t max_batch, jatam_mlp **net);
void jatam_mlp_destroy(jatam_mlp *net);
/* params: [JATAM_MLP_NPARAM] float32, host or device; set also resets Adam. */
int jatam_mlp_set_params(jatam_mlp *net, const float *params, void *stream);
int jatam_mlp_get_params(jatam_mlp *net, float *params, void *stream);
/*
 * One training step on a batch: forward, loss, backward; then Adam with
 * learning rate lr unless lr == 0.  genomes [B] (36-bit, host or device),
 * labels [B] uint8 classes 0..7.  loss (host float, may be NULL) receives the
 * mean cross-entropy before the update; grads (NULL or [JATAM_MLP_NPARAM]
 * float32, host or device) receives the gradient of that loss.  Synchronises
 * when loss or grads is host memory.
 */
int jatam_mlp_train_step(jatam_mlp *net, const uint64_t *genomes, const uint8_t *labels, uint64_t B, float lr,
                         float *loss, float *grads, void *stream);
/* logits [N][8] float32 (host or device) for genomes [N] (N <= max_batch). */
int jatam_mlp_predict(jatam_mlp *net, const uint64_t *genomes, uint64_t N, float *logits, void *stream);

/* Training data for the network, on the device: labels[i] = class of
 * results[i] (the 8 classes above); out[i] = genomes[i] of S_{n,c} written as
 * an S_{3,8} genome (its tiles first, then all-zero tiles, each colour in 3
 * bits; an all-zero tile never binds, so the classification is unchanged). */
int jatam_mlp_labels(const jatam_result *results, uint64_t N, uint8_t *labels, void *stream);
int jatam_embed_genomes(const uint64_t *genomes, uint64_t N, int n, int c, uint64_t *out, void *stream);

/* The selection step of the pre-screen below, on its own: idx[0 .. keep) receives,
 * in increasing order, the indices of the keep largest of the n scores (all
 * non-negative float32; ties: lower index first).  scores and idx are device
 * memory; n <= 2^26, keep <= n.  Queued on `stream`; no synchronisation.  Its
 * 33 KB of scratch is part of the device's workspace, so it is ordered after
 * the device's previous call that uses the workspace. */
int jatam_select_top(const float *scores, uint64_t n, uint64_t keep, uint64_t *idx, void *stream);

/*
 * ga_run_screened -- ga_run with the network as a pre-screen (shape fitness):
 * each generation breeds ratio x N candidate children (child indices
 * 0 .. ratio N - 1 of ga_breed), scores each with the network's probability
 * of a deterministic bounded shape of at least 8 tiles (classes 6 and 7) and
 * keeps the N best (ties: lower index) as the next population -- distinct
 * genomes first: a repeat of an earlier candidate ranks below every first
 * occurrence, so the population does not collapse onto copies of the
 * network's favourite -- which the
 * plain classification then evaluates: every reported fitness is simulated,
 * the network only decides which candidates get simulated.  When online_lr >
 * 0, each generation's simulated population, labelled by its own results,
 * also trains the network for one Adam step at that learning rate (the
 * network follows the region the search moves into).  ratio x N must fit the
 * network's max_batch.
 */
int ga_run_screened(const jatam_ga_config *ga, const jatam_config *cls, uint64_t N, uint32_t generations,
                    uint32_t ratio, jatam_mlp *net, float online_lr, uint64_t *population, int32_t *best,
                    int64_t *total, void *stream);

/*
 * jatam_philox -- Philox4x32-10 (Salmon et al., SC'11) as computed by the
 * classification kernels, for checking the draws: for each of N records
 * in[6 i .. 6 i + 5] = (ctr0, ctr1, ctr2, ctr3, key0, key1) it writes the four
 * output words to out[4 i .. 4 i + 3].  Buffers may be host or device.
 */
int jatam_philox(const uint32_t *in, uint64_t N, uint32_t *out, void *stream);

/*
 * jatam_hist_merge -- host-only merge of two sorted histograms (the shards of
 * a range split across processes or devices): counts add, min_id takes the
 * minimum, size the maximum, flags OR.  a, b, out are host arrays; out may not
 * alias a or b.  Returns JATAM_EINVAL if the merged length exceeds cap
 * (*len still receives it).
 */
int jatam_hist_merge(const jatam_hist_entry *a, uint32_t na, const jatam_hist_entry *b, uint32_t nb,
                     jatam_hist_entry *out, uint32_t cap, uint32_t *len);

/*
 * jatam_autotune -- pick the launch shape of the classification kernel for
 * each of n_shapes configurations (Section 2.6 batches the space by device
 * capacity; the best batch shape depends on the grid size and tile count).
 * For every configuration it times the kernel on a sample of its space
 * (the first min(2^18, |space|) genotypes, or 2^18 sampled ones when
 * cfg.flags has JATAM_SAMPLED) for every candidate (warps per CTA in
 * {2, 4, 8}, growth-round threshold in {4, 8, 12, 16, 20, 24, 28}) and keeps
 * the fastest for the key (lattice template, n, c) of that configuration;
 * later calls with the same key use it.  The choice never changes results:
 * the draws depend only on the genotype, the replicate and the step.
 * Synchronises `stream`.
 */
int jatam_autotune(const jatam_config *shapes, uint32_t n_shapes, void *stream);

/*
 * jatam_set_tuning / jatam_get_tuning -- set or read the launch shape used for
 * cfg's key: warps_per_cta 1..6, stop_at 1..32 (lanes that must have finished
 * their genotype before a warp leaves a growth round); warps_per_cta 0 forgets
 * the key's setting.  A key never tuned or set uses the defaults: the CTA size
 * that keeps the most warps resident on an SM, and stop_at 18 (lattices up to
 * 16 x 16) or 12 (32 x 32).
 */
int jatam_set_tuning(const jatam_config *cfg, int warps_per_cta, int stop_at);
int jatam_get_tuning(const jatam_config *cfg, int *warps_per_cta, int *stop_at);

/*
 * jatam_set_genotypes_per_warp / jatam_get_genotypes_per_warp -- the layout of
 * the growth launch for cfg's key (lattice size class, n, c), for items of one
 * shape on the row-major process:
 *   32: one genotype per lane, its lattice in the lane's share of shared
 *       memory (every lattice size);
 *    1: one genotype per warp, lattice rows in lanes held in registers, the
 *       frontier rank found by a prefix sum across lanes (lattices of
 *       17 x 17 to 32 x 32 only, where the per-lane layout leaves few warps
 *       resident);
 *    0: forget the setting (the default: 32 until jatam_autotune has timed
 *       both on a 32 x 32 key).
 * jatam_autotune times both layouts for keys with L > 16.  The layout never
 * changes results.
 */
int jatam_set_genotypes_per_warp(const jatam_config *cfg, int genotypes_per_warp);
int jatam_get_genotypes_per_warp(const jatam_config *cfg, int *genotypes_per_warp);

/*
 * jatam_set_replicate_lanes / jatam_get_replicate_lanes -- replicate lanes for
 * small calls (Section 2.4's k independent assemblies of a genotype grown side
 * by side): a warp takes one genotype and its lane r grows replicate r, so a
 * genotype takes as long as its longest replicate instead of the sum of its
 * replicates.  Eligible: items of one shape, lattices up to 16 x 16, k <= 32,
 * the row-major process, no executed-work counters (jatam_profile(2)).
 *   0: for eligible calls whose item count times k is at most 2^21 (2^23
 *      for sets of three or more tiles) -- the default; the environment
 *      variable JATAM_REPLICATE_LANES, read once, sets the mode;
 *   1: never;   2: for every eligible call.
 * Results are the same either way.  The setting is per process.
 */
int jatam_set_replicate_lanes(int mode);
int jatam_get_replicate_lanes(void);

/*
 * jatam_set_mixed_plan / jatam_get_mixed_plan -- the CTA plan of the
 * persistent launch for mixed lattice sizes: warps with a 32 x 32, 16 x 16
 * and 8 x 8 region per CTA (at least one 32 x 32 warp, since only those can
 * run L > 16; at most 8 warps in total, shared memory permitting; default
 * 2, 4, 2).
 * jatam_autotune_batch -- time every candidate plan of the persistent launch
 * and the per-size fixed launches on the given mixed batch (colours[N][16],
 * shapes[N][4], host or device); keep the fastest plan, and make the faster
 * of the two launch forms the default of mixed batches.  Synchronises.
 */
int jatam_set_mixed_plan(int warps_32, int warps_16, int warps_8);
int jatam_get_mixed_plan(int *warps_32, int *warps_16, int *warps_8);
/* *per_shape = 1 if mixed batches without a launch-form flag use the per-size
 * fixed launches, 0 if the persistent launch. */
int jatam_get_mixed_launch(int *per_shape);
int jatam_autotune_batch(const uint8_t *colours, const uint8_t *shapes, uint64_t N, uint64_t seed, void *stream);

/*
 * jatam_profile -- enable is a bit set for every later call:
 *   bit 0 (1): record CUDA events around the classification kernels on the
 *              call's stream; jatam_kernel_ms() then waits for the last such
 *              pair and returns its elapsed milliseconds in *ms
 *              (JATAM_EINVAL if no call has been profiled);
 *   bit 1 (2): count the work the classification kernels executed;
 *              jatam_work_counters() waits for the last call and returns
 *              [0] drawn placements, [1] seed placements (replicates grown),
 *              [2] lane slots of the growth rounds (32 per warp round; the
 *              lanes not placing are the SIMT idle share), [3] genotypes grown
 *              by warps (those the seed-step pre-filter did not settle).
 *              JATAM_EINVAL if the last call on the device was not counted.
 * enable outside 0..3: JATAM_EINVAL.  The counters cost one ballot per round.
 */
int jatam_profile(int enable);
int jatam_kernel_ms(float *ms);
int jatam_work_counters(uint64_t counters[4]);

/*
 * jatam_enumerate_noalloc -- jatam_enumerate without any device allocation,
 * for callers that cannot allocate: code whose application owns every byte of
 * device memory through its own pool, code that runs where a cudaMalloc (or
 * the device-wide synchronisation a cudaFree implies) is not allowed, or code
 * that must not let a library grow a hidden workspace.  The paper has no
 * counterpart: it is an integration variant of the same classification.
 *   Its scratch (three counters and the list of genotypes left to grow after
 *   the seed-step pre-filter) lives in one fixed array of device memory that
 *   is part of the library (8 B per genotype for JATAM_NOALLOC_MAX_COUNT
 *   genotypes, about 8 MB); every GPU that loads the library holds it until
 *   the process exits.
 *   cfg   : as for jatam_enumerate (JATAM_SAMPLED and JATAM_C4_HASH honoured;
 *           with JATAM_SYNC the call waits for the stream and reports
 *           device-side errors; JATAM_ORBITS and JATAM_LIFO are rejected with
 *           JATAM_EINVAL).
 *   first, count : index range, count <= JATAM_NOALLOC_MAX_COUNT, else
 *           JATAM_EINVAL with a message naming the limit.
 *   out   : [count] results in device memory of the current device, or
 *           managed memory (required; host memory is rejected, as staging it
 *           would need an allocation, and so is another GPU's memory).  No
 *           histogram.
 *   stream: cudaStream_t or NULL.
 * The first call on each device looks up the scratch array's device address
 * and loads and configures every kernel instance the entry point may launch
 * (all lattice sizes and tile counts); make that first call before any stream
 * capture.  jatam_shutdown() forgets this set-up; call it before a
 * cudaDeviceReset, after which the array may sit at another address.  All
 * calls share the one array and start by clearing its counters: calls whose
 * work overlaps on the GPU (unordered streams) race on it.
 */
#define JATAM_NOALLOC_MAX_COUNT 1048576u
int jatam_enumerate_noalloc(const jatam_config *cfg, uint64_t first, uint64_t count, jatam_result *out, void *stream);

/*
 * jatam_workspace_bytes -- bytes of device memory the library's workspace
 * holds on the current device (0 if no call has created one there; the fixed
 * scratch array of jatam_enumerate_noalloc is not counted).  The paper has no
 * counterpart: it is a memory-accounting aid.
 */
int jatam_workspace_bytes(uint64_t *bytes);

/* Free every device workspace of the library (waits for queued work). */
void jatam_shutdown(void);

/* Message describing the calling thread's last failure ("" if none). */
const char *jatam_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* JATAM_H */
