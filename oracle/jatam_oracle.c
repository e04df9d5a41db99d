/*
 * jatam_oracle.c -- plain, slow, obviously-correct CPU oracle for the JaTAM
 * classification path.  TEST INFRASTRUCTURE ONLY: it is loaded by the test
 * suite, by the smoke check and by the CPU-baseline leg of the benchmark, and
 * by nothing in the product path.  It shares no code, header, table or
 * constant with the CUDA library: everything below is written out again from
 * the model's definitions.
 *
 * Model (Appendix "Modifications to Winfree's aTAM" and Section 2.1 of the
 * paper):
 *   - tiles are unit squares with four edge colours, ordered N, E, S, W;
 *   - temperature 1: a single bond suffices to attach a tile;
 *   - interaction matrix M_ij = (1 - i mod 2) d_{i,j+1} + (i mod 2) d_{i,j-1},
 *     i.e. colours bind in adjacent pairs 1-2, 3-4, 5-6, colour 0 is inert and
 *     all non-bonding pairs are neutral;
 *   - tiles may be rotated by multiples of 90 degrees but never mirrored;
 *   - the first tile of the set (the seed) starts at the centre of an empty
 *     grid; every tile type, the seed type included, is available without
 *     limit;
 *   - configurations are equal iff type and orientation agree everywhere;
 *     shapes are equal iff the occupied positions agree;
 *   - a configuration with a tile outside the origin-centred square of
 *     dimension d is unbounded by d.
 * Genome encoding (Appendix "Encoding genome information"): tiles seed first,
 * each tile N, E, S, W, log2(c) bits per colour.
 * Hash (Section 2.5 "Classifying self-assembled shapes" and the appendix
 * "One-at-a-time Hash"): Jenkins' 32-bit one-at-a-time hash over the
 * positions of the occupied sites relative to the cropped grid.
 *
 * Where the paper is silent the readings used here are:
 *   [R1]  the literal M: with c even the top odd colour has no partner;
 *   [R2]  a packed genotype is read MSB-first (first tile, N edge = top bits);
 *   [R4]  rotation r turns a tile clockwise: side d of (t, r) is colour
 *         col[t][(d - r) mod 4];
 *   [R5]  the seed is placed in orientation 0 at (L/2, L/2);
 *   [R7]  ambiguity counts distinct rotated colour tuples, so repeated tile
 *         types and symmetric tiles are not non-determinism (Section 2.4);
 *         a placed tile is recorded by the lowest (t, r) carrying its tuple;
 *   [R8]  after each placement (and after the seed) the empty neighbours of
 *         the new tile are (re)evaluated; >= 2 distinct candidates anywhere
 *         -> local non-determinism; else a candidate outside the grid ->
 *         unbounded; else an empty frontier -> terminated;
 *   [R9]  step s of replicate j draws word (s mod 4) of
 *         Philox4x32-10(ctr = (s >> 2, j, id_lo, id_hi), key = seed), and
 *         picks frontier site floor(u * |F| / 2^32) in row-major order;
 *   [R10] replicates run in order; the first one that is unbounded, locally
 *         non-deterministic, or terminates in a configuration different from
 *         replicate 0's decides the class; otherwise the genotype is
 *         deterministic and bounded;
 *   [R11] the shape of replicate 0 is canonicalised over the 8 symmetries of
 *         the square (minimum of (height, width, row-major bits)) and hashed
 *         as the bytes height, width, then x, y per occupied cell in
 *         row-major order.
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_MAXL 32
#define ORC_MAXN 4
#define ORC_MAXC 8

enum { ORC_DET_BOUNDED = 0, ORC_ND_LOCAL = 1, ORC_ND_STERIC = 2, ORC_UNBOUNDED = 3 };
enum { OUT_TERMINATED = 0, OUT_ND_LOCAL = 1, OUT_UNBOUNDED = 2 };

/* direction d: 0 = N, 1 = E, 2 = S, 3 = W; x grows to the east, y to the south */
static const int DX[4] = {0, 1, 0, -1};
static const int DY[4] = {-1, 0, 1, 0};

typedef struct {
    uint8_t cls;
    uint8_t decided_rep;
    uint16_t size;
    uint32_t shape_hash;
} orc_result;

/* ---------------------------------------------------------------------------
 * Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as easy
 * as 1, 2, 3", SC'11): ten rounds of the 4x32 Philox S-box with multipliers
 * 0xD2511F53 / 0xCD9E8D57 and Weyl key increments 0x9E3779B9 / 0xBB67AE85.
 * ------------------------------------------------------------------------- */
void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    uint32_t x0 = ctr[0], x1 = ctr[1], x2 = ctr[2], x3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; round++) {
        if (round > 0) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        uint64_t prod0 = (uint64_t)0xD2511F53u * (uint64_t)x0;
        uint64_t prod1 = (uint64_t)0xCD9E8D57u * (uint64_t)x2;
        uint32_t hi0 = (uint32_t)(prod0 >> 32), lo0 = (uint32_t)prod0;
        uint32_t hi1 = (uint32_t)(prod1 >> 32), lo1 = (uint32_t)prod1;
        uint32_t y0 = hi1 ^ x1 ^ k0;
        uint32_t y1 = lo1;
        uint32_t y2 = hi0 ^ x3 ^ k1;
        uint32_t y3 = lo0;
        x0 = y0; x1 = y1; x2 = y2; x3 = y3;
    }
    out[0] = x0; out[1] = x1; out[2] = x2; out[3] = x3;
}

/* ---------------------------------------------------------------------------
 * Jenkins one-at-a-time hash (Jenkins 1997; the paper's appendix "One-at-a-
 * time Hash"): start from 0; per byte add it, add the value shifted left by
 * 10, xor the value shifted right by 6; finish with add <<3, xor >>11,
 * add <<15.  All arithmetic modulo 2^32.  Bytes are taken unsigned; the
 * coordinates hashed here are < 32 so the paper's signed-char argument makes
 * no difference.
 * ------------------------------------------------------------------------- */
uint32_t orc_oaat(const uint8_t *bytes, uint64_t len)
{
    uint32_t h = 0;
    for (uint64_t i = 0; i < len; i++) {
        h += bytes[i];
        h += h << 10;
        h ^= h >> 6;
    }
    h += h << 3;
    h ^= h >> 11;
    h += h << 15;
    return h;
}

/* The interaction matrix M of the appendix: colours i and j bind iff
 * (i even and i = j + 1) or (i odd and i = j - 1). */
int orc_bind(int i, int j)
{
    if ((i % 2) == 0) return i == j + 1;
    return i == j - 1;
}

/* Decode a packed genotype: tiles seed first, each N, E, S, W, b = log2(c)
 * bits per colour, most significant bits first (reading [R2]). */
int orc_decode(uint64_t g, int n, int c, uint8_t col[16])
{
    int b = 0;
    while ((1 << b) < c) b++;
    if ((1 << b) != c || n < 1 || n > ORC_MAXN) return -1;
    memset(col, 0, 16);
    for (int t = 0; t < n; t++)
        for (int e = 0; e < 4; e++) {
            int pos = b * (4 * (n - 1 - t) + (3 - e));
            col[4 * t + e] = (uint8_t)((g >> pos) & (uint64_t)(c - 1));
        }
    return 0;
}

/* Genotype sampled uniformly from the packed space: words 0 and 1 of
 * Philox4x32-10(ctr = (0, 1 << 24, i_lo, i_hi), key = seed), masked to the
 * genome length. */
uint64_t orc_sample_genotype(uint64_t i, int n, int c, uint64_t seed)
{
    int b = 0;
    while ((1 << b) < c) b++;
    int bits = 4 * n * b;
    uint32_t ctr[4] = {0u, 1u << 24, (uint32_t)i, (uint32_t)(i >> 32)};
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    uint32_t w[4];
    orc_philox4x32_10(ctr, key, w);
    uint64_t v = ((uint64_t)w[1] << 32) | w[0];
    if (bits < 64) v &= (((uint64_t)1) << bits) - 1;
    return v;
}

/* The sampled genotypes of indices first .. first+count-1 (one call of
 * orc_sample_genotype per index). */
void orc_sample_genotypes(uint64_t first, uint64_t count, int n, int c, uint64_t seed, uint64_t *out)
{
    for (uint64_t i = 0; i < count; i++) out[i] = orc_sample_genotype(first + i, n, c, seed);
}

/* ---------------------------------------------------------------------------
 * Tile set with rotations
 * ------------------------------------------------------------------------- */
typedef struct {
    int n, c, L, k;
    uint64_t seed;
    int col[ORC_MAXN][4];
    int side[4 * ORC_MAXN][4]; /* side[4t + r][d] */
    int rep[4 * ORC_MAXN];     /* lowest (t, r) with the same rotated tuple */
} tileset;

static void make_tileset(tileset *T, int n, int c, int L, int k, uint64_t seed, const uint8_t col[16])
{
    T->n = n; T->c = c; T->L = L; T->k = k; T->seed = seed;
    for (int t = 0; t < n; t++)
        for (int e = 0; e < 4; e++) T->col[t][e] = col[4 * t + e];
    /* clockwise rotation by r quarter turns: the colour that was on side
       (d - r) mod 4 now faces direction d (reading [R4]) */
    for (int t = 0; t < n; t++)
        for (int r = 0; r < 4; r++)
            for (int d = 0; d < 4; d++) T->side[4 * t + r][d] = T->col[t][(d - r + 4) % 4];
    for (int a = 0; a < 4 * n; a++) {
        T->rep[a] = a;
        for (int b = 0; b < a; b++) {
            if (memcmp(T->side[a], T->side[b], sizeof T->side[a]) == 0) {
                T->rep[a] = b;
                break;
            }
        }
    }
}

/* ---------------------------------------------------------------------------
 * One assembly grid
 * ------------------------------------------------------------------------- */
typedef struct {
    int L;
    int cell[ORC_MAXL][ORC_MAXL];  /* -1 empty, else the recorded tuple id */
    int ncand[ORC_MAXL][ORC_MAXL]; /* |D(s)| of an empty site, as last evaluated */
    int cand[ORC_MAXL][ORC_MAXL];  /* the single candidate when ncand == 1 */
    int size;
    int nd_kind; /* local ambiguity found: 1 one neighbour offers two distinct tuples, 2 only different
                    neighbours disagree (two arms meeting: first-order steric, Section 2.4) */
} grid;

static int inside(const grid *G, int x, int y) { return x >= 0 && y >= 0 && x < G->L && y < G->L; }

/* D(q): the distinct rotated tuples that can attach at the empty site q,
 * i.e. those (t, r) for which some occupied neighbour offers a bond
 * (temperature 1, non-bonding faces neutral).  Returns |D(q)|; *only receives
 * the tuple when |D(q)| == 1. */
static int candidates(const tileset *T, const grid *G, int qx, int qy, int *only)
{
    int seen[4 * ORC_MAXN];
    int m = 0;
    memset(seen, 0, sizeof seen);
    for (int t = 0; t < T->n; t++) {
        for (int r = 0; r < 4; r++) {
            int a = 4 * t + r;
            int bonds = 0;
            for (int d = 0; d < 4; d++) {
                int nx = qx + DX[d], ny = qy + DY[d];
                if (!inside(G, nx, ny)) continue;
                int u = G->cell[ny][nx];
                if (u < 0) continue;
                /* the neighbour in direction d shows us its side (d + 2) mod 4 */
                if (orc_bind(T->side[a][d], T->side[u][(d + 2) % 4])) bonds = 1;
            }
            if (bonds && !seen[T->rep[a]]) {
                seen[T->rep[a]] = 1;
                m++;
                *only = T->rep[a];
            }
        }
    }
    return m;
}

/* Which kind of local ambiguity the empty site q (with |D(q)| >= 2) shows:
 * 1 if some single occupied neighbour alone offers two distinct tuples
 * (trivial non-determinism), 2 if every neighbour offers at most one and
 * different neighbours offer different tuples (two arms meeting at q: the
 * first-order steric non-determinism Section 2.4 detects together with the
 * trivial kind). */
static int ambiguity_kind(const tileset *T, const grid *G, int qx, int qy)
{
    for (int d = 0; d < 4; d++) {
        int nx = qx + DX[d], ny = qy + DY[d];
        if (!inside(G, nx, ny) || G->cell[ny][nx] < 0) continue;
        int u = G->cell[ny][nx];
        int seen[4 * ORC_MAXN], m = 0;
        memset(seen, 0, sizeof seen);
        for (int a = 0; a < 4 * T->n; a++)
            if (orc_bind(T->side[a][d], T->side[u][(d + 2) % 4]) && !seen[T->rep[a]]) {
                seen[T->rep[a]] = 1;
                m++;
            }
        if (m >= 2) return 1;
    }
    return 2;
}

static uint32_t draw(const tileset *T, uint64_t stream_id, int rep, int step)
{
    uint32_t ctr[4] = {(uint32_t)step >> 2, (uint32_t)rep, (uint32_t)stream_id, (uint32_t)(stream_id >> 32)};
    uint32_t key[2] = {(uint32_t)T->seed, (uint32_t)(T->seed >> 32)};
    uint32_t w[4];
    orc_philox4x32_10(ctr, key, w);
    return w[step & 3];
}

/* Optional per-step trace of a replicate, used by the tests to re-derive every
 * draw independently. */
typedef struct {
    int32_t nfront;  /* |F| before the draw */
    uint32_t u;      /* the Philox word */
    int32_t index;   /* chosen rank in F */
    int32_t x, y;    /* chosen site */
    int32_t tuple;   /* tuple placed */
} orc_trace_step;

/* Grow one replicate from the seed until it is decided. */
static int run_replicate(const tileset *T, uint64_t stream_id, int rep, grid *G, uint64_t *placements,
                         orc_trace_step *trace, int trace_cap, int *trace_len)
{
    int L = T->L;
    G->L = L;
    for (int y = 0; y < L; y++)
        for (int x = 0; x < L; x++) {
            G->cell[y][x] = -1;
            G->ncand[y][x] = 0;
            G->cand[y][x] = -1;
        }
    int px = L / 2, py = L / 2;
    G->cell[py][px] = T->rep[0];
    G->size = 1;
    G->nd_kind = 0;
    int step = 0;
    int fx[ORC_MAXL * ORC_MAXL], fy[ORC_MAXL * ORC_MAXL];
    for (;;) {
        int nd = 0, unb = 0;
        for (int d = 0; d < 4; d++) {
            int qx = px + DX[d], qy = py + DY[d];
            int in = inside(G, qx, qy);
            if (in && G->cell[qy][qx] >= 0) continue;
            int only = -1;
            int m = candidates(T, G, qx, qy, &only);
            if (in) {
                G->ncand[qy][qx] = m;
                G->cand[qy][qx] = (m == 1) ? only : -1;
            }
            if (m >= 2) {
                nd = 1;
                int kind = ambiguity_kind(T, G, qx, qy);
                if (G->nd_kind == 0 || kind < G->nd_kind) G->nd_kind = kind;
            }
            else if (!in && m >= 1) unb = 1;
        }
        if (nd) return OUT_ND_LOCAL;
        if (unb) return OUT_UNBOUNDED;
        int nf = 0;
        for (int y = 0; y < L; y++)
            for (int x = 0; x < L; x++)
                if (G->cell[y][x] < 0 && G->ncand[y][x] == 1) {
                    fx[nf] = x;
                    fy[nf] = y;
                    nf++;
                }
        if (nf == 0) return OUT_TERMINATED;
        uint32_t u = draw(T, stream_id, rep, step);
        int i = (int)(((uint64_t)u * (uint64_t)nf) >> 32);
        int sx = fx[i], sy = fy[i];
        if (trace && *trace_len < trace_cap) {
            orc_trace_step *ts = &trace[*trace_len];
            ts->nfront = nf; ts->u = u; ts->index = i; ts->x = sx; ts->y = sy; ts->tuple = G->cand[sy][sx];
            (*trace_len)++;
        }
        G->cell[sy][sx] = G->cand[sy][sx];
        G->size++;
        step++;
        (*placements)++;
        px = sx;
        py = sy;
    }
}

/* ---------------------------------------------------------------------------
 * The movelist process of Section 2.4 (reading L1), the alternative draw order:
 * the frontier is kept as a last-in-first-out stack.  After each placement
 * (and after the seed) the sites that have just become frontier sites, taken
 * in the order N, E, S, W of the placed tile, are pushed in a random order --
 * permutation number floor(u m! / 2^32) of the m sites, u the Philox word
 * whose index is the number of placements after the seed so far, decoded in
 * the factorial number system (digit i picks among the sites not yet taken,
 * the first pick is pushed first) -- and the next tile goes on the site at the
 * top.  Candidates, ambiguity and growth past the grid are judged as in the
 * row-major process.
 * ------------------------------------------------------------------------- */
static int g_lifo = 0; /* process of the classification calls below (0: row-major frontier, 1: movelist) */

void orc_set_process(int lifo) { g_lifo = lifo ? 1 : 0; }

/* the order in which permutation number idx of m items is pushed: out[i] = item pushed i-th */
void orc_lifo_permutation(uint32_t idx, int m, int out[4])
{
    int pool[4] = {0, 1, 2, 3};
    int left = m;
    for (int i = 0; i < m; i++) {
        int f = 1;
        for (int q = 2; q <= m - 1 - i; q++) f *= q;
        const int sel = (int)(idx / (uint32_t)f);
        idx %= (uint32_t)f;
        out[i] = pool[sel];
        for (int q = sel; q < left - 1; q++) pool[q] = pool[q + 1];
        left--;
    }
}

static int run_replicate_lifo(const tileset *T, uint64_t stream_id, int rep, grid *G, uint64_t *placements,
                              orc_trace_step *trace, int trace_cap, int *trace_len)
{
    int L = T->L;
    G->L = L;
    for (int y = 0; y < L; y++)
        for (int x = 0; x < L; x++) {
            G->cell[y][x] = -1;
            G->ncand[y][x] = 0;
            G->cand[y][x] = -1;
        }
    int px = L / 2, py = L / 2;
    G->cell[py][px] = T->rep[0];
    G->size = 1;
    G->nd_kind = 0; /* the ambiguity diagnostic covers the row-major process only */
    int placed = 0; /* placements after the seed */
    int sx_stack[ORC_MAXL * ORC_MAXL], sy_stack[ORC_MAXL * ORC_MAXL];
    int sp = 0;
    for (;;) {
        int nd = 0, unb = 0;
        int newx[4], newy[4], m = 0;
        for (int d = 0; d < 4; d++) {
            int qx = px + DX[d], qy = py + DY[d];
            int in = inside(G, qx, qy);
            if (in && G->cell[qy][qx] >= 0) continue;
            int only = -1;
            int mm = candidates(T, G, qx, qy, &only);
            if (in) {
                const int was_frontier = G->ncand[qy][qx] == 1;
                G->ncand[qy][qx] = mm;
                G->cand[qy][qx] = (mm == 1) ? only : -1;
                if (mm == 1 && !was_frontier) {
                    newx[m] = qx;
                    newy[m] = qy;
                    m++;
                }
            }
            if (mm >= 2) nd = 1;
            else if (!in && mm >= 1) unb = 1;
        }
        if (nd) return OUT_ND_LOCAL;
        if (unb) return OUT_UNBOUNDED;
        /* push the new sites in the drawn order */
        uint32_t u = draw(T, stream_id, rep, placed);
        int fact = 1;
        for (int q = 2; q <= m; q++) fact *= q;
        const uint32_t idx = (uint32_t)(((uint64_t)u * (uint64_t)fact) >> 32);
        int order[4];
        orc_lifo_permutation(idx, m, order);
        for (int i = 0; i < m; i++) {
            sx_stack[sp] = newx[order[i]];
            sy_stack[sp] = newy[order[i]];
            sp++;
        }
        if (sp == 0) return OUT_TERMINATED;
        sp--;
        const int sx = sx_stack[sp], sy = sy_stack[sp];
        if (trace && *trace_len < trace_cap) {
            orc_trace_step *ts = &trace[*trace_len];
            ts->nfront = m; ts->u = u; ts->index = (int32_t)idx; ts->x = sx; ts->y = sy; ts->tuple = G->cand[sy][sx];
            (*trace_len)++;
        }
        G->cell[sy][sx] = G->cand[sy][sx];
        G->size++;
        placed++;
        (*placements)++;
        px = sx;
        py = sy;
    }
}

static int same_configuration(const grid *A, const grid *B)
{
    for (int y = 0; y < A->L; y++)
        for (int x = 0; x < A->L; x++)
            if (A->cell[y][x] != B->cell[y][x]) return 0;
    return 1;
}

/* ---------------------------------------------------------------------------
 * Canonical form under the 8 symmetries of the square, and its hash
 * ------------------------------------------------------------------------- */

/* Image of (x, y) under symmetry s (4 rotations, then the 4 mirror images). */
static void symmetry(int s, int x, int y, int *ox, int *oy)
{
    switch (s) {
    case 0: *ox = x;  *oy = y;  break;
    case 1: *ox = -y; *oy = x;  break;
    case 2: *ox = -x; *oy = -y; break;
    case 3: *ox = y;  *oy = -x; break;
    case 4: *ox = -x; *oy = y;  break;
    case 5: *ox = x;  *oy = -y; break;
    case 6: *ox = y;  *oy = x;  break;
    default: *ox = -y; *oy = -x; break;
    }
}

/* Canonical form of a set of m cells: for every symmetry, translate the image
 * so that its minimum x and y are 0, giving an h x w bitmap; keep the image
 * with the smallest (h, w, row-major bit sequence), 0 before 1.  Writes the
 * bitmap (row-major, 1 byte per cell) to out[h * w]; returns 0. */
int orc_canonical(const int32_t *xs, const int32_t *ys, int m, uint8_t *out, int32_t *out_h, int32_t *out_w)
{
    static const int CAP = 2 * ORC_MAXL + 1;
    int best_h = 0, best_w = 0, have = 0;
    uint8_t best[(2 * ORC_MAXL + 1) * (2 * ORC_MAXL + 1)];
    uint8_t img[(2 * ORC_MAXL + 1) * (2 * ORC_MAXL + 1)];
    if (m <= 0) {
        *out_h = 0;
        *out_w = 0;
        return 0;
    }
    for (int s = 0; s < 8; s++) {
        int minx = 1 << 30, miny = 1 << 30, maxx = -(1 << 30), maxy = -(1 << 30);
        for (int i = 0; i < m; i++) {
            int tx, ty;
            symmetry(s, xs[i], ys[i], &tx, &ty);
            if (tx < minx) minx = tx;
            if (ty < miny) miny = ty;
            if (tx > maxx) maxx = tx;
            if (ty > maxy) maxy = ty;
        }
        int h = maxy - miny + 1, w = maxx - minx + 1;
        if (h > CAP || w > CAP) return -1;
        memset(img, 0, (size_t)h * (size_t)w);
        for (int i = 0; i < m; i++) {
            int tx, ty;
            symmetry(s, xs[i], ys[i], &tx, &ty);
            img[(ty - miny) * w + (tx - minx)] = 1;
        }
        int better = 0;
        if (!have) better = 1;
        else if (h != best_h) better = h < best_h;
        else if (w != best_w) better = w < best_w;
        else better = memcmp(img, best, (size_t)h * (size_t)w) < 0;
        if (better) {
            have = 1;
            best_h = h;
            best_w = w;
            memcpy(best, img, (size_t)h * (size_t)w);
        }
    }
    memcpy(out, best, (size_t)best_h * (size_t)best_w);
    *out_h = best_h;
    *out_w = best_w;
    return 0;
}

/* Hash of a canonical bitmap through one-at-a-time: first the height and the
 * width of the cropped grid, then bytes x, y of every occupied cell in
 * row-major order.  (Starting from state 0, a zero byte leaves the state at 0,
 * so without the non-zero dimension bytes a leading cell at (0, 0) would not
 * count and, e.g., the 2 x 2 square would hash like the L-tromino.) */
uint32_t orc_shape_hash(const uint8_t *bitmap, int h, int w)
{
    uint8_t bytes[2 + 2 * (2 * ORC_MAXL + 1) * (2 * ORC_MAXL + 1)];
    uint64_t nb = 0;
    bytes[nb++] = (uint8_t)h;
    bytes[nb++] = (uint8_t)w;
    for (int y = 0; y < h; y++)
        for (int x = 0; x < w; x++)
            if (bitmap[y * w + x]) {
                bytes[nb++] = (uint8_t)x;
                bytes[nb++] = (uint8_t)y;
            }
    return orc_oaat(bytes, nb);
}

/* The rotation-invariant variant of Section 2.5: hash each of the four
 * rotations of the shape (each cropped, hashed as orc_shape_hash hashes a
 * bitmap), sort the four hashes numerically, and hash the sorted hashes again
 * (their 16 bytes, little endian) with one-at-a-time.  Mirror images are not
 * identified. */
uint32_t orc_c4_hash(const int32_t *xs, const int32_t *ys, int m)
{
    uint32_t hs[4];
    uint8_t img[(2 * ORC_MAXL + 1) * (2 * ORC_MAXL + 1)];
    for (int s = 0; s < 4; s++) {
        int minx = 1 << 30, miny = 1 << 30, maxx = -(1 << 30), maxy = -(1 << 30);
        for (int i = 0; i < m; i++) {
            int tx, ty;
            symmetry(s, xs[i], ys[i], &tx, &ty);
            if (tx < minx) minx = tx;
            if (ty < miny) miny = ty;
            if (tx > maxx) maxx = tx;
            if (ty > maxy) maxy = ty;
        }
        int h = maxy - miny + 1, w = maxx - minx + 1;
        if (h < 1 || w < 1 || h > 2 * ORC_MAXL + 1 || w > 2 * ORC_MAXL + 1) return 0;
        memset(img, 0, (size_t)h * (size_t)w);
        for (int i = 0; i < m; i++) {
            int tx, ty;
            symmetry(s, xs[i], ys[i], &tx, &ty);
            img[(ty - miny) * w + (tx - minx)] = 1;
        }
        hs[s] = orc_shape_hash(img, h, w);
    }
    for (int i = 1; i < 4; i++)
        for (int j = i; j > 0 && hs[j - 1] > hs[j]; j--) {
            uint32_t t = hs[j];
            hs[j] = hs[j - 1];
            hs[j - 1] = t;
        }
    uint8_t bytes[16];
    for (int i = 0; i < 4; i++)
        for (int b = 0; b < 4; b++) bytes[4 * i + b] = (uint8_t)(hs[i] >> (8 * b));
    return orc_oaat(bytes, 16);
}

static int g_c4_hash = 0; /* hash mode of the classification calls below (0: D4 canonical form, 1: C4) */

void orc_set_hash_mode(int c4) { g_c4_hash = c4 ? 1 : 0; }

/* ---------------------------------------------------------------------------
 * Exact side table of the shapes (Section 2.5 estimates the chance that two
 * distinct shapes share a 32-bit hash; this table settles it): while it is
 * on, every canonical form hashed by the classification calls is stored under
 * its hash, and a form that differs from the one already stored under the
 * same hash counts as a collision.  Row i of a form: bit j = column j.
 * ------------------------------------------------------------------------- */
#define ORC_SHAPE_SLOTS (1 << 16)
typedef struct {
    int used;
    uint32_t hash;
    int h, w;
    uint32_t rows[ORC_MAXL];
} orc_shape_entry;
static orc_shape_entry *g_shape_tab = NULL;
static int g_shape_on = 0;
static uint64_t g_shape_collisions = 0, g_shape_overflow = 0;
static pthread_mutex_t g_shape_mu = PTHREAD_MUTEX_INITIALIZER;

int orc_shape_table_begin(void)
{
    if (!g_shape_tab) g_shape_tab = (orc_shape_entry *)malloc(sizeof(orc_shape_entry) * ORC_SHAPE_SLOTS);
    if (!g_shape_tab) return -2;
    memset(g_shape_tab, 0, sizeof(orc_shape_entry) * ORC_SHAPE_SLOTS);
    g_shape_collisions = 0;
    g_shape_overflow = 0;
    g_shape_on = 1;
    return 0;
}

void orc_shape_table_add(uint32_t hash, const uint8_t *bm, int h, int w)
{
    orc_shape_entry e;
    memset(&e, 0, sizeof e);
    e.used = 1;
    e.hash = hash;
    e.h = h;
    e.w = w;
    for (int y = 0; y < h && y < ORC_MAXL; y++)
        for (int x = 0; x < w && x < 32; x++)
            if (bm[y * w + x]) e.rows[y] |= (uint32_t)1 << x;
    pthread_mutex_lock(&g_shape_mu);
    uint32_t slot = hash & (ORC_SHAPE_SLOTS - 1);
    int placed = 0;
    for (int p = 0; p < ORC_SHAPE_SLOTS; p++) {
        orc_shape_entry *t = &g_shape_tab[slot];
        if (!t->used) {
            *t = e;
            placed = 1;
            break;
        }
        if (t->hash == hash) {
            if (t->h != h || t->w != w || memcmp(t->rows, e.rows, sizeof e.rows) != 0) g_shape_collisions++;
            placed = 1;
            break;
        }
        slot = (slot + 1) & (ORC_SHAPE_SLOTS - 1);
    }
    if (!placed) g_shape_overflow++;
    pthread_mutex_unlock(&g_shape_mu);
}

/* Stop recording; the stored forms, sorted by hash: hashes[i], hw[2 i] = h,
 * hw[2 i + 1] = w, rows[32 i .. 32 i + 31].  Returns -1 if more than cap. */
int orc_shape_table_end(uint32_t *hashes, int32_t *hw, uint32_t *rows, int cap, int *len, uint64_t *collisions,
                        uint64_t *overflow)
{
    g_shape_on = 0;
    int m = 0;
    if (g_shape_tab) {
        /* selection of the entries in increasing hash order (plain and slow) */
        uint64_t last = 0;
        int first = 1;
        for (;;) {
            int best = -1;
            for (int i = 0; i < ORC_SHAPE_SLOTS; i++) {
                const orc_shape_entry *t = &g_shape_tab[i];
                if (!t->used || (!first && (uint64_t)t->hash <= last)) continue;
                if (best < 0 || t->hash < g_shape_tab[best].hash) best = i;
            }
            if (best < 0) break;
            if (m < cap) {
                hashes[m] = g_shape_tab[best].hash;
                hw[2 * m] = g_shape_tab[best].h;
                hw[2 * m + 1] = g_shape_tab[best].w;
                for (int r = 0; r < 32; r++) rows[32 * m + r] = r < ORC_MAXL ? g_shape_tab[best].rows[r] : 0u;
            }
            m++;
            last = g_shape_tab[best].hash;
            first = 0;
        }
    }
    *len = m;
    *collisions = g_shape_collisions;
    *overflow = g_shape_overflow;
    return m > cap ? -1 : 0;
}

static uint32_t hash_of_grid(const grid *G)
{
    int32_t xs[ORC_MAXL * ORC_MAXL], ys[ORC_MAXL * ORC_MAXL];
    uint8_t bm[(2 * ORC_MAXL + 1) * (2 * ORC_MAXL + 1)];
    int m = 0;
    for (int y = 0; y < G->L; y++)
        for (int x = 0; x < G->L; x++)
            if (G->cell[y][x] >= 0) {
                xs[m] = x;
                ys[m] = y;
                m++;
            }
    if (g_c4_hash) return orc_c4_hash(xs, ys, m);
    int32_t h, w;
    orc_canonical(xs, ys, m, bm, &h, &w);
    uint32_t hash = orc_shape_hash(bm, h, w);
    if (g_shape_on) orc_shape_table_add(hash, bm, h, w);
    return hash;
}

/* ---------------------------------------------------------------------------
 * Classification of one genotype (reading [R10] / [R11])
 * ------------------------------------------------------------------------- */
static int valid_params(int n, int c, int L, int k)
{
    return n >= 1 && n <= ORC_MAXN && c >= 1 && c <= 8 && L >= 1 && L <= ORC_MAXL && k >= 1 && k <= 255;
}

/* Diagnostic mode of the classification calls below: ND_LOCAL results carry
 * the kind of ambiguity that decided them in `size` (1 trivial, 2 first-order
 * steric; see ambiguity_kind).  Classes and every other field are unchanged. */
static int g_nd_detail = 0;
void orc_set_nd_detail(int on) { g_nd_detail = on ? 1 : 0; }

/* Classify one genotype given its colours col[4t + e].  When rep0_cells is not
 * NULL it receives replicate 0's final grid (L*L ints, row-major, -1 empty).
 * When trace is not NULL it receives the steps of replicate trace_rep. */
int orc_classify_ex(int n, int c, int L, int k, uint64_t seed, const uint8_t col[16], uint64_t stream_id,
                    orc_result *res, uint64_t *placements, int32_t *rep0_cells, int trace_rep,
                    orc_trace_step *trace, int trace_cap, int *trace_len)
{
    if (!valid_params(n, c, L, k)) return -1;
    for (int i = 0; i < 4 * n; i++)
        if (col[i] >= c) return -1;
    tileset T;
    make_tileset(&T, n, c, L, k, seed, col);
    grid *A0 = (grid *)malloc(sizeof(grid));
    grid *Aj = (grid *)malloc(sizeof(grid));
    if (!A0 || !Aj) {
        free(A0);
        free(Aj);
        return -2;
    }
    uint64_t placed = 0;
    int cls = ORC_DET_BOUNDED, decided = k;
    int tl = 0;
    for (int j = 0; j < k; j++) {
        grid *G = (j == 0) ? A0 : Aj;
        int want = (trace && j == trace_rep);
        int out = (g_lifo ? run_replicate_lifo : run_replicate)(&T, stream_id, j, G, &placed, want ? trace : NULL, trace_cap, &tl);
        if (out == OUT_UNBOUNDED) { cls = ORC_UNBOUNDED; decided = j; break; }
        if (out == OUT_ND_LOCAL) { cls = ORC_ND_LOCAL; decided = j; break; }
        if (j > 0 && !same_configuration(A0, Aj)) { cls = ORC_ND_STERIC; decided = j; break; }
    }
    res->cls = (uint8_t)cls;
    res->decided_rep = (uint8_t)decided;
    res->size = 0;
    res->shape_hash = 0;
    if (cls == ORC_ND_LOCAL && g_nd_detail) res->size = (uint16_t)((decided == 0 ? A0 : Aj)->nd_kind);
    if (cls == ORC_DET_BOUNDED || cls == ORC_ND_STERIC) {
        res->size = (uint16_t)A0->size;
        res->shape_hash = hash_of_grid(A0);
    }
    if (rep0_cells) {
        for (int y = 0; y < L; y++)
            for (int x = 0; x < L; x++) rep0_cells[y * L + x] = A0->cell[y][x];
    }
    if (placements) *placements += placed;
    if (trace_len) *trace_len = tl;
    free(A0);
    free(Aj);
    return 0;
}

int orc_classify(int n, int c, int L, int k, uint64_t seed, const uint8_t col[16], uint64_t stream_id,
                 orc_result *res, uint64_t *placements)
{
    return orc_classify_ex(n, c, L, k, seed, col, stream_id, res, placements, NULL, -1, NULL, 0, NULL);
}

/* ---------------------------------------------------------------------------
 * Batch drivers (one POSIX thread per core over contiguous ranges)
 * ------------------------------------------------------------------------- */
typedef struct {
    int n, c, L, k, sampled;
    uint64_t seed, first, count;
    const uint8_t *cols;    /* explicit colours [count][16] or NULL */
    const uint8_t *shapes;  /* per-item (n, c, L, k) [count][4] or NULL */
    const uint64_t *ids;    /* stream ids or NULL */
    orc_result *out;
    uint64_t lo, hi;        /* this thread's range of items */
    uint64_t placements;
    int status;
} job;

static void *worker(void *arg)
{
    job *J = (job *)arg;
    for (uint64_t i = J->lo; i < J->hi; i++) {
        uint8_t col[16];
        int n = J->n, c = J->c, L = J->L, k = J->k;
        uint64_t sid;
        if (J->cols) {
            memcpy(col, J->cols + 16 * i, 16);
            if (J->shapes) {
                n = J->shapes[4 * i + 0];
                c = J->shapes[4 * i + 1];
                L = J->shapes[4 * i + 2];
                k = J->shapes[4 * i + 3];
            }
            sid = J->ids ? J->ids[i] : i;
        } else {
            uint64_t idx = J->first + i;
            uint64_t g = J->sampled ? orc_sample_genotype(idx, n, c, J->seed) : idx;
            if (orc_decode(g, n, c, col) != 0) {
                J->status = -1;
                return NULL;
            }
            sid = g;
        }
        int rc = orc_classify(n, c, L, k, J->seed, col, sid, &J->out[i], &J->placements);
        if (rc != 0) {
            J->status = rc;
            return NULL;
        }
    }
    return NULL;
}

static int run_jobs(job *proto, uint64_t count, int nthreads, uint64_t *placements)
{
    if (nthreads < 1) nthreads = 1;
    if (nthreads > 256) nthreads = 256;
    if ((uint64_t)nthreads > count && count > 0) nthreads = (int)count;
    job jobs[256];
    pthread_t th[256];
    for (int t = 0; t < nthreads; t++) {
        jobs[t] = *proto;
        jobs[t].lo = count * (uint64_t)t / (uint64_t)nthreads;
        jobs[t].hi = count * (uint64_t)(t + 1) / (uint64_t)nthreads;
        jobs[t].placements = 0;
        jobs[t].status = 0;
    }
    for (int t = 1; t < nthreads; t++) pthread_create(&th[t], NULL, worker, &jobs[t]);
    worker(&jobs[0]);
    for (int t = 1; t < nthreads; t++) pthread_join(th[t], NULL);
    uint64_t total = 0;
    int status = 0;
    for (int t = 0; t < nthreads; t++) {
        total += jobs[t].placements;
        if (jobs[t].status) status = jobs[t].status;
    }
    if (placements) *placements = total;
    return status;
}

/* Classify genotype indices first .. first+count-1 of the packed space
 * (in order, or sampled when sampled != 0).  The stream id of each genotype
 * is its packed value. */
int orc_enumerate(int n, int c, int L, int k, uint64_t seed, int sampled, uint64_t first, uint64_t count,
                  orc_result *out, int nthreads, uint64_t *placements)
{
    if (!valid_params(n, c, L, k)) return -1;
    job proto;
    memset(&proto, 0, sizeof proto);
    proto.n = n; proto.c = c; proto.L = L; proto.k = k; proto.sampled = sampled;
    proto.seed = seed; proto.first = first; proto.count = count; proto.out = out;
    return run_jobs(&proto, count, nthreads, placements);
}

/* Classify explicit colour records cols[count][16]; shapes[count][4] gives
 * per-item (n, c, L, k) or is NULL (then n, c, L, k apply to all); ids gives
 * stream ids or is NULL (then the item index is the stream id). */
int orc_classify_batch(const uint8_t *cols, const uint8_t *shapes, int n, int c, int L, int k, uint64_t seed,
                       const uint64_t *ids, uint64_t count, orc_result *out, int nthreads, uint64_t *placements)
{
    job proto;
    memset(&proto, 0, sizeof proto);
    proto.n = n; proto.c = c; proto.L = L; proto.k = k;
    proto.seed = seed; proto.count = count; proto.cols = cols; proto.shapes = shapes; proto.ids = ids;
    proto.out = out;
    return run_jobs(&proto, count, nthreads, placements);
}

/* ---------------------------------------------------------------------------
 * Genetic algorithm (Section 2.2 "Genetic Algorithms"; appendix "Efficient
 * bit-wise implementations of common evolutionary operators"): one generation
 * turns a parent population with its fitness values into a child population.
 *   selection  -- tournament (the best of T uniformly drawn parents, the
 *                 earliest drawn on ties) or global roulette wheel (the parent
 *                 in whose slice of the cumulative fitness a dart lands,
 *                 Section 2.2; uniform when all fitness values are 0);
 *   crossover  -- none, single point (the bits above a cut point from parent
 *                 A, the rest from B) or uniform (each bit from A or B);
 *   mutation   -- every edge (gene) undergoes a Poisson number of events with
 *                 mean rate mu; each event flips one uniformly chosen bit of
 *                 the edge's log2(c) bits (Section 2.2; appendix "Encoding
 *                 genome information": flips of single bits).
 * Draws: word k of child i in generation g is word (k mod 4) of
 * Philox4x32-10(ctr = (k >> 2, (2 << 24) | g, i_lo, i_hi), key = seed), laid
 * out as: tournament A (T words) or roulette dart A (1), tournament B / dart B,
 * crossover decision, two mask/cut words, one Poisson word per edge, and
 * four bit-choice words per edge.
 * ------------------------------------------------------------------------- */
typedef struct {
    int n, c;
    int selection;   /* 0 tournament, 1 roulette */
    int tournament;  /* T */
    int crossover;   /* 0 none, 1 single point, 2 uniform */
    uint32_t crossover_threshold;
    uint32_t mutation_thresholds[4];
    uint64_t seed;
} orc_ga;

static uint32_t ga_word(const orc_ga *G, uint32_t generation, uint64_t child, int k)
{
    uint32_t ctr[4] = {(uint32_t)k >> 2, (2u << 24) | generation, (uint32_t)child, (uint32_t)(child >> 32)};
    uint32_t key[2] = {(uint32_t)G->seed, (uint32_t)(G->seed >> 32)};
    uint32_t w[4];
    orc_philox4x32_10(ctr, key, w);
    return w[k & 3];
}

/* The roulette wheel's cumulative search: the first index whose running sum
 * of weights exceeds the dart (equivalently: reaches dart + 1). */
uint64_t orc_roulette_pick(const uint64_t *cumsum, uint64_t N, uint64_t dart)
{
    for (uint64_t i = 0; i < N; i++)
        if (cumsum[i] > dart) return i;
    return N - 1;
}

/* index of the parent chosen by selection from words starting at k0 */
static uint64_t ga_select(const orc_ga *G, const int32_t *fitness, const uint64_t *cumsum, uint64_t N,
                          uint32_t generation, uint64_t child, int k0)
{
    if (G->selection == 0) {
        uint64_t best = 0;
        int have = 0;
        for (int j = 0; j < G->tournament; j++) {
            uint64_t idx = ((uint64_t)ga_word(G, generation, child, k0 + j) * N) >> 32;
            if (!have || fitness[idx] > fitness[best]) {
                best = idx;
                have = 1;
            }
        }
        return best;
    }
    uint64_t total = cumsum[N - 1];
    uint32_t u = ga_word(G, generation, child, k0);
    if (total == 0) return ((uint64_t)u * N) >> 32;
    uint64_t dart = ((uint64_t)u * total) >> 32;  /* uniform in [0, total) */
    return orc_roulette_pick(cumsum, N, dart);
}

int orc_ga_breed(const orc_ga *G, const uint64_t *parents, const int32_t *fitness, uint64_t N, uint32_t generation,
                 uint64_t *children)
{
    int b = 0;
    while ((1 << b) < G->c) b++;
    const int bits = 4 * G->n * b;
    const uint64_t all = bits >= 64 ? ~0ull : (((uint64_t)1 << bits) - 1);
    const int T = G->selection == 0 ? G->tournament : 1;
    if (N == 0) return 0;
    uint64_t *cumsum = (uint64_t *)malloc(sizeof(uint64_t) * N);
    if (!cumsum) return -2;
    uint64_t run = 0;
    for (uint64_t i = 0; i < N; i++) {
        run += fitness[i] > 0 ? (uint64_t)fitness[i] : 0;
        cumsum[i] = run;
    }
    const int k_cross = 2 * T, k_mask = 2 * T + 1, k_pois = 2 * T + 3, k_bit = 2 * T + 3 + 4 * G->n;
    for (uint64_t i = 0; i < N; i++) {
        uint64_t a = parents[ga_select(G, fitness, cumsum, N, generation, i, 0)];
        uint64_t bb = parents[ga_select(G, fitness, cumsum, N, generation, i, T)];
        uint64_t child = a;
        if (G->crossover != 0 && ga_word(G, generation, i, k_cross) < G->crossover_threshold) {
            if (G->crossover == 1) {
                /* cut in 1 .. bits-1: the top bits - cut from A, the low cut bits from B */
                int cut = 1 + (int)(((uint64_t)ga_word(G, generation, i, k_mask) * (uint64_t)(bits - 1)) >> 32);
                uint64_t low = ((uint64_t)1 << cut) - 1;
                child = (a & ~low) | (bb & low);
            } else {
                uint64_t mask = ((uint64_t)ga_word(G, generation, i, k_mask + 1) << 32) | ga_word(G, generation, i, k_mask);
                child = (a & ~mask) | (bb & mask);
            }
        }
        for (int e = 0; e < 4 * G->n && b > 0; e++) {
            uint32_t u = ga_word(G, generation, i, k_pois + e);
            int events = 0;
            for (int j = 0; j < 4; j++)
                if (u >= G->mutation_thresholds[j]) events++;
            int t = e / 4, side = e % 4;
            int pos = b * (4 * (G->n - 1 - t) + (3 - side));
            for (int m = 0; m < events; m++) {
                int bit = (int)(((uint64_t)ga_word(G, generation, i, k_bit + 4 * e + m) * (uint64_t)b) >> 32);
                child ^= (uint64_t)1 << (pos + bit);
            }
        }
        children[i] = child & all;
    }
    free(cumsum);
    return 0;
}

/* floor(2^32 P(K <= j)) for K ~ Poisson(rate), j = 0..3, saturated at 2^32 - 1 */
int orc_poisson_thresholds(double rate, uint32_t out[4])
{
    if (!(rate >= 0.0)) return -1;
    double term = exp(-rate), cdf = 0.0;
    for (int j = 0; j < 4; j++) {
        cdf += term;
        term *= rate / (double)(j + 1);
        double t = floor(cdf * 4294967296.0);
        out[j] = t >= 4294967295.0 ? 4294967295u : (uint32_t)t;
    }
    return 0;
}

/* Fujiyama test-bed fitness (Section 3.2): the Hamming weight of the genome */
int orc_hamming(uint64_t g) { int h = 0; while (g) { h += (int)(g & 1); g >>= 1; } return h; }

/* ---------------------------------------------------------------------------
 * Orbits of the exact symmetries of the process (the orbit mode of the
 * enumeration): a permutation of the c colours that preserves M, turning any
 * non-seed tile, and permuting the non-seed tiles.  With the draws fixed every
 * genotype of an orbit assembles identically (the process sees only which
 * rotated tuples bind, never the labels, and the seed is untouched).  The
 * representative of an orbit is its smallest packed genotype, found here by
 * applying every element of the group.
 * ------------------------------------------------------------------------- */
static pthread_mutex_t g_aut_mutex = PTHREAD_MUTEX_INITIALIZER;
static int g_aut_ready[ORC_MAXC + 1];
static int g_aut_count[ORC_MAXC + 1];
static uint8_t g_aut[ORC_MAXC + 1][128][ORC_MAXC];

/* every permutation p of 0 .. c-1 with M(p[i], p[j]) == M(i, j), by brute force */
static void colour_automorphisms(int c)
{
    pthread_mutex_lock(&g_aut_mutex);
    if (!g_aut_ready[c]) {
        int p[ORC_MAXC];
        for (int i = 0; i < c; i++) p[i] = i;
        int count = 0;
        for (;;) {
            int ok = 1;
            for (int i = 0; i < c && ok; i++)
                for (int j = 0; j < c && ok; j++)
                    if (orc_bind(p[i], p[j]) != orc_bind(i, j)) ok = 0;
            if (ok && count < 128) {
                for (int i = 0; i < c; i++) g_aut[c][count][i] = (uint8_t)p[i];
                count++;
            }
            /* next permutation in lexicographic order */
            int i = c - 2;
            while (i >= 0 && p[i] >= p[i + 1]) i--;
            if (i < 0) break;
            int j = c - 1;
            while (p[j] <= p[i]) j--;
            int t = p[i]; p[i] = p[j]; p[j] = t;
            for (int a = i + 1, b2 = c - 1; a < b2; a++, b2--) { t = p[a]; p[a] = p[b2]; p[b2] = t; }
        }
        g_aut_count[c] = count;
        g_aut_ready[c] = 1;
    }
    pthread_mutex_unlock(&g_aut_mutex);
}

int orc_colour_automorphism_count(int c)
{
    if (c < 1 || c > ORC_MAXC) return -1;
    colour_automorphisms(c);
    return g_aut_count[c];
}

static uint64_t encode_genotype(const uint8_t col[16], int n, int c)
{
    int b = 0;
    while ((1 << b) < c) b++;
    uint64_t g = 0;
    for (int t = 0; t < n; t++)
        for (int e = 0; e < 4; e++) g |= (uint64_t)col[4 * t + e] << (b * (4 * (n - 1 - t) + (3 - e)));
    return g;
}

uint64_t orc_orbit_rep(uint64_t g, int n, int c)
{
    uint8_t col[16], img[16];
    if (orc_decode(g, n, c, col) != 0) return g;
    colour_automorphisms(c);
    const int m = n - 1;                        /* non-seed tiles */
    int nperm = 1, nrot = 1;
    for (int i = 2; i <= m; i++) nperm *= i;
    for (int i = 0; i < m; i++) nrot *= 4;
    uint64_t best = g;
    for (int a = 0; a < g_aut_count[c]; a++) {
        const uint8_t *pi = g_aut[c][a];
        for (int pk = 0; pk < nperm; pk++) {
            /* the pk-th permutation of the non-seed slots (factorial number system) */
            int perm[ORC_MAXN], pool[ORC_MAXN], np = m, code = pk;
            for (int i = 0; i < m; i++) pool[i] = i + 1;
            for (int i = 0; i < m; i++) {
                int f = 1;
                for (int q = 2; q <= m - 1 - i; q++) f *= q;
                int sel = code / f;
                code %= f;
                perm[i] = pool[sel];
                for (int q = sel; q < np - 1; q++) pool[q] = pool[q + 1];
                np--;
            }
            for (int rk = 0; rk < nrot; rk++) {
                for (int e = 0; e < 4; e++) img[e] = pi[col[e]];
                int code_r = rk;
                for (int s = 0; s < m; s++) {
                    const int r = code_r % 4;
                    code_r /= 4;
                    const int t = perm[s];
                    for (int e = 0; e < 4; e++) img[4 * (s + 1) + e] = pi[col[4 * t + ((e - r + 4) % 4)]];
                }
                const uint64_t v = encode_genotype(img, n, c);
                if (v < best) best = v;
            }
        }
    }
    return best;
}

/* representatives of genotypes first .. first + count - 1 */
int orc_orbit_reps(int n, int c, uint64_t first, uint64_t count, uint64_t *out)
{
    for (uint64_t i = 0; i < count; i++) out[i] = orc_orbit_rep(first + i, n, c);
    return 0;
}
