// jatam_api.cu -- host side of libjatam.so: argument checks, the per-device
// workspace, staging of host buffers, launches, and the error state.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <tuple>
#include <vector>
#include <mutex>
#include <string>

#include <cuda_runtime.h>

#include "jatam_internal.cuh"
#include "jatam_pipe.h"

using namespace jatam;

struct jatam_mlp {
    int device = -1;
    jatam::MlpBuffers b{};
    int t = 0;              // Adam steps taken
    void *stage = nullptr;  // host inputs: genomes then labels; host outputs
    size_t stage_bytes = 0;
};

namespace {

thread_local std::string g_last_error;
std::mutex g_mutex;
int g_profile = 0;  // bit 0: events around the growth kernels; bit 1: executed-work counters
int g_stop_override = 0;
bool g_mixed_per_shape = false;  // the default launch form of mixed batches (set by jatam_autotune_batch)
int g_warps_override = 0;
int g_per_warp_override = 0;  // JATAM_GENOTYPES_PER_WARP: 1 or 32 for every 32 x 32 launch
int g_window = 1;             // lattices of 17..32: grow in a 16 x 16 window first (JATAM_WINDOW=0: off)
int g_crop_table = 1;          // the call's crop table of hashes (JATAM_CROP_TABLE=0: every form is computed)
// levels of the heavy-first order of uniform launches (JATAM_HEAVY_LEVELS=2: two or more frontier
// sites after the seed, then one).  Three (three or four, then two, then one) measured 1.7 % faster
// on the S_{2,8} growth kernel (2.182 -> 2.145 ms)
int g_heavy_levels = 3;
// genotypes per warp of a 32 x 32 launch when nothing is tuned or set
int g_default_per_warp32 = 32;
// replicate lanes (one genotype per warp, its k replicates side by side): 0 for calls on lattices
// up to 16 x 16 with k <= 32 whose items x k is at most REPS_MAX_WORK (four times that for sets of
// three or more tiles, whose genotypes grow longer), 1 never, 2 whenever eligible
// (jatam_set_replicate_lanes; JATAM_REPLICATE_LANES).  Measured crossovers, L = 16: S_{2,8} slices
// (k = 20) 2^16 items 0.217 against 0.226 ms, 2^17 0.303 against 0.289; all of S_{2,4} (k = 10)
// 0.153 against 0.172; S_{3,8} samples (k = 20) 2^18 0.414 against 0.471, 2^19 0.735 against 0.664
int g_reps_mode = 0;
size_t REPS_MAX_WORK = size_t(1) << 21;
// genome batches classify each distinct genome once (JATAM_GENOME_DEDUP=0: every item)
int g_dedup = 1;

struct Tuning {
    int warps = 0;    // 0: the CTA size that keeps the most warps resident
    int stop_at = 0;  // 0: default_stop_at (14 for lattices up to 16 x 16, 12 for 32 x 32)
    int w32 = 2, w16 = 4, w8 = 2;  // warps per CTA of each region size in the mixed launch
    int per_warp = 0;  // genotypes a warp grows at once: 32 (one per lane) or 1 (one per warp, 32 x 32
                       // lattices only); 0: the default of the lattice template
};
// launch shape per key (lattice template, n, c); n = c = 0 for mixed batches
std::map<std::tuple<int, int, int>, Tuning> g_tuned;

// optional overrides of the launch shape (for tuning sweeps)
// host-buffer calls of at least 2 * PIPE_MIN_ITEMS items run in pieces (JATAM_PIPE_PIECE_LOG2 sets it,
// 2^20 .. 2^26)
size_t PIPE_MIN_ITEMS = size_t(1) << 22;
// The piece schedule of such calls (pipe_schedule).  Measured end to end (results to page-locked
// memory), S_{2,8} in full: staggered with 2 pieces 2.67 ms, 3 pieces 2.87, 4 pieces 2.85; paired
// geometric with 4 pieces 2.75; equal pieces side by side (the earlier schedule) 2.83; the
// device-output call 2.33.  S_{3,8} sample of 2^28 at L = 32 (window and escalation launches): paired
// geometric with 4 pieces 75.7 ms, 8 pieces 78.2; staggered with 2 or 4 pieces 80.4-80.7; the earlier
// schedule 79.8; the device-output call 73.9.  Records from page-locked memory (with stream ids) also
// copy their inputs piece by piece: on 10^7 mixed records (28 B in, 8 B out each) two equal pieces
// take 5.60-5.63 ms against 6.16 with the inputs copied at once; 3, 4 and 6 pieces 6.4, 7.1 and 8.7 ms
// (each piece runs a launch per lattice size, each with its tail); a first piece of 0.3, 0.4 or 0.6
// of the call 5.8-6.1 ms.  JATAM_PIPE_FORM (bit 0 staggered, bit 1 geometric sizes), JATAM_PIPE_PIECES
// and JATAM_PIPE_STAGE override it.
int g_pipe_form = -1;
int g_pipe_pieces = 0;
int g_pipe_stage = 1;  // JATAM_PIPE_STAGE=0: host record inputs copied at once even in pipelined calls

void read_env_overrides()
{
    static bool done = false;
    if (done) return;
    done = true;
    if (const char *v = getenv("JATAM_STOP_AT")) {
        int x = atoi(v);
        if (x >= 1 && x <= 32) g_stop_override = x;
    }
    if (const char *v = getenv("JATAM_WARPS_PER_CTA")) {
        int x = atoi(v);
        if (x >= 1 && x <= MAX_CTA_WARPS) g_warps_override = x;
    }
    if (const char *v = getenv("JATAM_WINDOW")) g_window = atoi(v) != 0;
    if (const char *v = getenv("JATAM_PIPE_PIECE_LOG2")) {
        const int x = atoi(v);
        if (x >= 20 && x <= 26) PIPE_MIN_ITEMS = size_t(1) << x;
    }
    if (const char *v = getenv("JATAM_PIPE_FORM")) g_pipe_form = atoi(v) & 3;
    if (const char *v = getenv("JATAM_PIPE_STAGE")) g_pipe_stage = atoi(v) != 0;
    if (const char *v = getenv("JATAM_PIPE_PIECES")) {
        const int x = atoi(v);
        if (x >= 2 && x <= 8) g_pipe_pieces = x;
    }
    if (const char *v = getenv("JATAM_CROP_TABLE")) g_crop_table = atoi(v) != 0;
    if (const char *v = getenv("JATAM_HEAVY_LEVELS")) g_heavy_levels = atoi(v) == 2 ? 2 : 3;
    if (const char *v = getenv("JATAM_GENOME_DEDUP")) g_dedup = atoi(v) != 0;
    if (const char *v = getenv("JATAM_REPLICATE_LANES")) {
        const int x = atoi(v);
        if (x >= 0 && x <= 2) g_reps_mode = x;
    }
    if (const char *v = getenv("JATAM_REPLICATE_LANES_MAX_LOG2")) {
        const int x = atoi(v);
        if (x >= 8 && x <= 30) REPS_MAX_WORK = size_t(1) << x;
    }
    if (const char *v = getenv("JATAM_GENOTYPES_PER_WARP")) {
        int x = atoi(v);
        if (x == 1 || x == 32) g_per_warp_override = x;
    }
}

int fail(int code, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_last_error = buf;
    return code;
}

#define CUDA_TRY(expr)                                                                        \
    do {                                                                                      \
        cudaError_t e_ = (expr);                                                              \
        if (e_ != cudaSuccess)                                                                \
            return fail(JATAM_ECUDA, "%s failed: %s", #expr, cudaGetErrorString(e_));         \
    } while (0)

constexpr unsigned TABLE_LOG2 = 18;  // 262,144 phenotype slots per device
constexpr unsigned CROPS_LOG2 = 12;  // 4,096 slots of the per-call crop table (64 KB)
constexpr unsigned SHAPES_LOG2 = 14;  // 16,384 slots of the call's shape side table (2.2 MB)
// per call or piece: counts [0..5] and work counters [6..8] of the window's escalation list, and
// [9] the number of spilled crops
constexpr int ESC_CTL_WORDS = 10;
constexpr unsigned SPILL_CAP = 1u << 16;  // crops the crop table cannot hold, per call or piece (8.3 MB)

struct Workspace {
    int device = -1;
    int num_sms = 0;
    Table table{};
    Compact compact{};
    unsigned long long *work_next = nullptr;
    unsigned long long *crops = nullptr;  // crop -> shape hash within one call (cleared by its reset)
    unsigned long long *stats = nullptr;  // [4] executed-work counters of the last counted call
    bool stats_valid = false;
    ShapeTab shapes{};           // canonical form per shape hash of the last call with a histogram
    bool shapes_valid = false;   // the last call filled `shapes` (a histogram, not the C4 hash)
    unsigned *err = nullptr;
    unsigned *nkeys = nullptr;
    unsigned long long *list_count = nullptr;
    void *list = nullptr;  // items left to grow after the pre-filter (8 B each)
    size_t list_bytes = 0;
    // window mode: the items whose growth leaves the window (8 B each), and its control words:
    // [0] their count, [3] 0 (the list format's count of light items), [6] the work counter
    void *esc = nullptr;
    size_t esc_bytes = 0;
    unsigned long long *esc_ctl = nullptr;
    uint32_t *spill_rows = nullptr;  // SPILL_CAP x 32 rows, then SPILL_CAP meta words
    size_t spill_bytes = 0;
    unsigned *host_words = nullptr;  // pinned: [0] err, [1] nkeys
    void *stage_in = nullptr;
    size_t stage_in_bytes = 0;
    void *stage_out = nullptr;
    size_t stage_out_bytes = 0;
    void *stage_aux = nullptr;
    size_t stage_aux_bytes = 0;
    jatam_hist_entry *stage_hist = nullptr;
    size_t stage_hist_cap = 0;
    cudaEvent_t last = nullptr;  // end of the previous call's work on this device
    cudaEvent_t k_start = nullptr, k_stop = nullptr;  // around the last profiled kernel
    bool k_valid = false;
    std::map<std::string, cudaGraphExec_t> graphs;  // captured calls, by argument set
    void *lifo_buf = nullptr;  // movelist process: one stack per thread of the growth launch
    size_t lifo_bytes = 0;
    void *ga_buf = nullptr;   // ga_run / ga_breed: fitness, children, cumsum, stats
    size_t ga_bytes = 0;
    void *topn_buf = nullptr;    // jatam_select_top: the selection's scratch
    size_t topn_bytes = 0;
    void *dedup_buf = nullptr;   // genome deduplication: table keys, first occurrences, item slots
    size_t dedup_bytes = 0;
    void *screen_buf = nullptr;  // ga_run_screened: candidates, chosen indices, scores
    size_t screen_bytes = 0;
    unsigned long long *screen_cand = nullptr, *screen_idx = nullptr;
    float *screen_score = nullptr;
    ScreenTable screen_table{};
    cudaStream_t capture = nullptr;                  // private stream used only for capturing
    // a pipelined call: pieces alternate between the caller's stream (scratch
    // above) and `aux` (scratch `alt`), so that a piece fills the SMs that the
    // previous piece's last genotypes leave idle; results go back on `copy`
    struct Scratch {
        unsigned long long *work_next = nullptr, *list_count = nullptr, *crops = nullptr;
        unsigned *nkeys = nullptr;  // cleared by the reset, read by nobody
        void *list = nullptr;
        size_t list_bytes = 0;
        void *esc = nullptr;
        size_t esc_bytes = 0;
        unsigned long long *esc_ctl = nullptr;
        uint32_t *spill_rows = nullptr;
        size_t spill_bytes = 0;
    } alt;
    cudaStream_t aux = nullptr, copy = nullptr;
    cudaStream_t h2d = nullptr;                  // per-piece input copies of pipelined record calls
    cudaEvent_t in_ev[PIPE_MAX_CHUNKS] = {};     // end of each piece's input copies
    cudaEvent_t pipe_ev[PIPE_MAX_CHUNKS] = {};  // end of each piece's classification
    cudaEvent_t pf_ev[PIPE_MAX_CHUNKS] = {};    // end of each piece's pre-filter
    cudaEvent_t pipe_start = nullptr, aux_done = nullptr, pipe_done = nullptr;
};

std::map<int, Workspace *> g_ws;

int grow(void **p, size_t *have, size_t want)
{
    if (*have >= want) return JATAM_OK;
    if (*p) cudaFree(*p);
    *p = nullptr;
    *have = 0;
    size_t sz = want < (1u << 20) ? (1u << 20) : want;
    cudaError_t e = cudaMalloc(p, sz);
    if (e != cudaSuccess) {
        cudaGetLastError();
        *p = nullptr;
        return fail(JATAM_ENOMEM, "cudaMalloc of %zu bytes failed: %s", sz, cudaGetErrorString(e));
    }
    *have = sz;
    return JATAM_OK;
}

int workspace(Workspace **out)
{
    read_env_overrides();
    int dev = 0;
    CUDA_TRY(cudaGetDevice(&dev));
    auto it = g_ws.find(dev);
    if (it != g_ws.end()) {
        *out = it->second;
        return JATAM_OK;
    }
    Workspace *w = new Workspace();
    w->device = dev;
    CUDA_TRY(cudaDeviceGetAttribute(&w->num_sms, cudaDevAttrMultiProcessorCount, dev));
    const size_t cap = size_t(1) << TABLE_LOG2;
    w->table.cap_log2 = TABLE_LOG2;
    CUDA_TRY(cudaMalloc(&w->table.key, cap * 8));
    CUDA_TRY(cudaMalloc(&w->table.count, cap * 8));
    CUDA_TRY(cudaMalloc(&w->table.min_id, cap * 8));
    CUDA_TRY(cudaMalloc(&w->table.size_max, cap * 4));
    CUDA_TRY(cudaMalloc(&w->table.size_min, cap * 4));
    CUDA_TRY(cudaMalloc(&w->compact.key, cap * 8));
    CUDA_TRY(cudaMalloc(&w->compact.count, cap * 8));
    CUDA_TRY(cudaMalloc(&w->compact.min_id, cap * 8));
    CUDA_TRY(cudaMalloc(&w->compact.size_max, cap * 4));
    CUDA_TRY(cudaMalloc(&w->compact.size_min, cap * 4));
    CUDA_TRY(cudaMalloc(&w->work_next, 3 * 8));
    CUDA_TRY(cudaMalloc(&w->crops, (size_t(2) << CROPS_LOG2) * 8));
    CUDA_TRY(cudaMalloc(&w->stats, 4 * 8));
    w->shapes.log2 = SHAPES_LOG2;
    CUDA_TRY(cudaMalloc(&w->shapes.key, (size_t(8) + 4 + 128) << SHAPES_LOG2));
    w->shapes.meta = reinterpret_cast<unsigned *>(w->shapes.key + (size_t(1) << SHAPES_LOG2));
    w->shapes.rows = reinterpret_cast<uint32_t *>(w->shapes.meta + (size_t(1) << SHAPES_LOG2));
    CUDA_TRY(cudaMalloc(&w->shapes.stats, 4 * 4));
    CUDA_TRY(cudaMalloc(&w->err, 4));
    CUDA_TRY(cudaMalloc(&w->nkeys, 4));
    CUDA_TRY(cudaMalloc(&w->list_count, 6 * 8));
    CUDA_TRY(cudaMalloc(&w->esc_ctl, ESC_CTL_WORDS * 8));
    CUDA_TRY(cudaMemset(w->esc_ctl, 0, ESC_CTL_WORDS * 8));
    CUDA_TRY(cudaMallocHost(&w->host_words, 16));
    CUDA_TRY(cudaEventCreateWithFlags(&w->last, cudaEventDisableTiming));
    CUDA_TRY(cudaEventCreate(&w->k_start));
    CUDA_TRY(cudaEventCreate(&w->k_stop));
    CUDA_TRY(launch_table_init(w->table, nullptr));
    CUDA_TRY(launch_reset(w->work_next, w->nkeys, w->list_count, nullptr, w->crops, CROPS_LOG2));
    CUDA_TRY(cudaMemsetAsync(w->err, 0, 4, nullptr));
    CUDA_TRY(cudaDeviceSynchronize());
    g_ws[dev] = w;
    *out = w;
    return JATAM_OK;
}

enum Kind { K_NULL, K_DEVICE, K_HOST };

Kind kind_of(const void *p, int device)
{
    if (!p) return K_NULL;
    cudaPointerAttributes at;
    cudaError_t e = cudaPointerGetAttributes(&at, p);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return K_HOST;
    }
    if ((at.type == cudaMemoryTypeDevice && at.device == device) || at.type == cudaMemoryTypeManaged)
        return K_DEVICE;
    if (at.type == cudaMemoryTypeDevice) return K_NULL;  // another device's memory: rejected by the caller
    return K_HOST;
}

// page-locked host memory (cudaMallocHost / cudaHostRegister): copies from the
// device to it run asynchronously
bool is_pinned(const void *p)
{
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeHost;
}

bool is_pow2(int c) { return c == 1 || c == 2 || c == 4 || c == 8; }
int log2c(int c) { return c >= 8 ? 3 : c >= 4 ? 2 : c >= 2 ? 1 : 0; }
int lattice_template(int L) { return L <= 8 ? 8 : L <= 16 ? 16 : 32; }

int check_params(int n, int c, int L, int k, bool packed)
{
    if (n < 1 || n > JATAM_MAX_TILES || c < 1 || c > JATAM_MAX_COLOURS || L < 1 || L > JATAM_MAX_GRID || k < 1 ||
        k > JATAM_MAX_REPLICATES)
        return fail(JATAM_EUNSUPPORTED, "unsupported parameters n=%d c=%d L=%d k=%d (n 1..4, c 1..8, L 1..32, k 1..255)",
                    n, c, L, k);
    if (packed && !is_pow2(c)) return fail(JATAM_EINVAL, "packed genotypes need c to be a power of two, got %d", c);
    return JATAM_OK;
}

int g_plan[3] = {2, 4, 2};  // mixed launch: warps with 32x32, 16x16, 8x8 regions per CTA

bool plan_fits(int w32, int w16, int w8)
{
    const int warps = w32 + w16 + w8;
    // at least one warp with a 32 x 32 region: a batch may hold any lattice size,
    // and only such a warp can run an item with L > 16
    return w32 >= 1 && w16 >= 0 && w8 >= 0 && w32 <= 8 && w16 <= 8 && w8 <= 8 && warps <= 8 &&
           classify_mixed_smem_bytes(w32, w16, w8) <= 200 * 1024;
}

Tuning tuning_for(int S, int n, int c)
{
    Tuning t;
    t.w32 = g_plan[0];
    t.w16 = g_plan[1];
    t.w8 = g_plan[2];
    const int nt = tuple_table_size(n);
    auto it = g_tuned.find(std::make_tuple(S, n, c));
    if (it != g_tuned.end()) {
        t.warps = it->second.warps;
        t.stop_at = it->second.stop_at;
        t.per_warp = it->second.per_warp;
    }
    if (t.warps == 0) t.warps = default_warps_per_cta(S, nt);
    if (t.stop_at == 0) t.stop_at = default_stop_at(S);
    if (g_warps_override) t.warps = g_warps_override;
    if (g_stop_override) t.stop_at = g_stop_override;
    if (t.per_warp == 0) t.per_warp = (S == 32) ? g_default_per_warp32 : 32;
    if (g_per_warp_override && S == 32) t.per_warp = g_per_warp_override;
    if (S != 32) t.per_warp = 32;
    while (t.warps > 1 && classify_smem_bytes(S, nt, t.warps) > 200 * 1024) --t.warps;  // what fits on one SM
    return t;
}

// Record inputs that live in host memory: run() copies them into the staging
// buffer the launch arguments already point at -- all at once before the
// classification, or, in a call that runs in pieces from page-locked memory, each
// piece's slice just before that piece (so that the copies overlap the
// classification of the pieces before it)
struct HostInputs {
    const uint8_t *colours = nullptr;            // [N][16], or null: not from the host
    const uint8_t *shapes = nullptr;             // [N][4]
    const unsigned long long *ids = nullptr;     // [N]
    uint8_t *colours_dev = nullptr, *shapes_dev = nullptr;  // their staging copies
    unsigned long long *ids_dev = nullptr;
    bool any() const { return colours || shapes || ids; }
};

struct Outputs {
    jatam_result *out_dev = nullptr;
    int32_t *fit_dev = nullptr;
    jatam_hist_entry *hist_dev = nullptr;
    uint32_t *hist_len_dev = nullptr;
    bool host_out = false, host_fit = false, host_hist = false, host_len = false;
};

// Run the classification of one launch description plus the histogram
// kernels, stage host outputs, and synchronise when needed.
int run(Workspace *w, LaunchArgs a, int S, jatam_result *out, int32_t *fitness, jatam_hist_entry *hist,
        uint32_t hist_cap, uint32_t *hist_len, bool sync_flag, cudaStream_t st, const Tuning *force = nullptr,
        float *kernel_ms = nullptr, bool per_shape = false, bool use_graph = false,
        const HostInputs *hin = nullptr)
{
    Outputs o;
    const Kind ko = kind_of(out, w->device), kf = kind_of(fitness, w->device), kh = kind_of(hist, w->device),
               kl = kind_of(hist_len, w->device);
    if ((out && ko == K_NULL) || (fitness && kf == K_NULL) || (hist && kh == K_NULL) || (hist_len && kl == K_NULL))
        return fail(JATAM_EINVAL, "an output buffer lives on another device");
    if (hist && !hist_len) return fail(JATAM_EINVAL, "hist needs hist_len");
    if (hist && hist_cap == 0) return fail(JATAM_EINVAL, "hist_cap must be positive when hist is given");
    const size_t n_items = (size_t)a.count;
    // staging: out and fitness share stage_out (out first, 16-byte aligned fitness after it)
    size_t out_bytes = (ko == K_HOST) ? n_items * sizeof(jatam_result) : 0;
    size_t fit_off = (out_bytes + 255) & ~size_t(255);
    size_t fit_bytes = (kf == K_HOST) ? n_items * sizeof(int32_t) : 0;
    if (out_bytes + fit_bytes) {
        int rc = grow(&w->stage_out, &w->stage_out_bytes, fit_off + fit_bytes + 256);
        if (rc) return rc;
    }
    o.host_out = ko == K_HOST;
    o.host_fit = kf == K_HOST;
    o.out_dev = o.host_out ? reinterpret_cast<jatam_result *>(w->stage_out) : out;
    o.fit_dev = o.host_fit ? reinterpret_cast<int32_t *>(static_cast<char *>(w->stage_out) + fit_off) : fitness;
    if (hist) {
        o.host_hist = kh == K_HOST;
        o.host_len = kl == K_HOST;
        if (o.host_hist) {
            if (w->stage_hist_cap < hist_cap) {
                if (w->stage_hist) cudaFree(w->stage_hist);
                w->stage_hist = nullptr;
                w->stage_hist_cap = 0;
                cudaError_t e = cudaMalloc(&w->stage_hist, (size_t)hist_cap * sizeof(jatam_hist_entry));
                if (e != cudaSuccess) {
                    cudaGetLastError();
                    return fail(JATAM_ENOMEM, "cannot stage %u histogram entries", hist_cap);
                }
                w->stage_hist_cap = hist_cap;
            }
            o.hist_dev = w->stage_hist;
        } else {
            o.hist_dev = hist;
        }
        o.hist_len_dev = o.host_len ? reinterpret_cast<uint32_t *>(w->nkeys) : hist_len;
    }
    a.out = o.out_dev;
    a.fitness = o.fit_dev;
    a.table = w->table;
    a.use_hist = hist ? 1 : 0;
    a.work_next = w->work_next;
    a.crops = g_crop_table ? w->crops : nullptr;
    a.crops_log2 = CROPS_LOG2;
    // the exact shape side table: calls with a histogram and the canonical-form hash
    const bool record_shapes = hist && !a.c4;
    const size_t spill_need = (size_t)SPILL_CAP * (32 * 4 + 4);
    if (record_shapes) {
        int rc = grow(reinterpret_cast<void **>(&w->spill_rows), &w->spill_bytes, spill_need);
        if (rc) return rc;
    }
    auto spill_of = [&](uint32_t *rows, unsigned long long *ctl) -> CropSpill {
        if (!record_shapes) return CropSpill{};
        return CropSpill{rows, reinterpret_cast<unsigned *>(rows + (size_t)SPILL_CAP * 32), ctl + 9, SPILL_CAP};
    };
    a.spill = spill_of(w->spill_rows, w->esc_ctl);
    a.stats = (g_profile & 2) ? w->stats : nullptr;
    // genome batches: every distinct genome is classified once, its repeats copy the result (a result
    // depends only on the genome: it is also the stream id).  Not with the executed-work counters, the
    // orbit mode, or a call large enough to run in pieces from host buffers
    const bool dedup = a.mode == MODE_GENOMES && g_dedup && !a.no_dedup && !a.stats && !a.orbits && n_items >= 2 &&
                       n_items < (size_t(1) << 30) && !(n_items >= 2 * PIPE_MIN_ITEMS && (o.host_out || o.host_fit));
    a.dup_keys = nullptr;
    a.dup_owner = nullptr;
    a.dup_slot = nullptr;
    a.dup_mask = 0;
    if (dedup) {
        // keys of 2^27 slots at most, at the front of the buffer (so that they outlive a regrowth of the
        // rest); a new buffer is emptied once, every call empties the slots it used
        size_t cap = 1;
        while (cap < 2 * n_items) cap <<= 1;
        const size_t kb = cap * 8, ob = (cap * 4 + 255) & ~size_t(255);
        const size_t need = kb + ob + n_items * 4 + 256;
        if (need > w->dedup_bytes) {
            int rc = grow(&w->dedup_buf, &w->dedup_bytes, need);
            if (rc) return rc;
            CUDA_TRY(cudaMemset(w->dedup_buf, 0xFF, w->dedup_bytes));
            CUDA_TRY(cudaDeviceSynchronize());  // empty before any stream of the call uses it
        }
        char *p = static_cast<char *>(w->dedup_buf);
        a.dup_keys = reinterpret_cast<unsigned long long *>(p);
        a.dup_owner = reinterpret_cast<unsigned *>(p + kb);
        a.dup_slot = reinterpret_cast<unsigned *>(p + kb + ob);
        a.dup_mask = (unsigned)(cap - 1);
    }
    a.err = w->err;
    const bool mixed = a.mode == MODE_RECORDS && a.shapes;
    const Tuning tune = force ? *force : tuning_for(S, mixed ? 0 : a.n, mixed ? 0 : a.c);
    a.stop_at = tune.stop_at;
    // lattices of 17 to 32: the items first grow in the 16 x 16 window around the seed, where four
    // times as many warps fit an SM; the few whose growth leaves the window run on the full lattice
    // (for calls of at least 2^23 items: smaller ones end in a thin escalation launch -- on S_{3,8},
    // 2^22 items 2.67 ms with the window, 2.41 without; 2^24 5.90 against 7.12; 2^26 19.8 against 26.5)
    const bool windowed = !mixed && !a.lifo && S == 32 && tune.per_warp != 1 && g_window &&
                          n_items >= (size_t(1) << 23);
    const int regions = mixed ? 3 : (g_heavy_levels == 3 ? 2 : 1);
    if (n_items) {
        int rc = grow(&w->list, &w->list_bytes, n_items * 8 * regions);
        if (rc) return rc;
        if (windowed) {
            rc = grow(&w->esc, &w->esc_bytes, n_items * 8);
            if (rc) return rc;
        }
    }
    a.list = static_cast<unsigned long long *>(w->list);
    a.list_stride = n_items;
    a.list_count = w->list_count;
    a.bucket = mixed ? 1 : 0;
    a.klass = 0;
    a.plan_w32 = tune.w32;
    a.plan_w16 = tune.w16;
    a.plan_w8 = tune.w8;

    // the single-template launch (not used for mixed sizes)
    const bool per_warp = !mixed && !a.lifo && S == 32 && tune.per_warp == 1;
    // replicate lanes for calls too small to fill the GPU one genotype per lane (the executed-work
    // counters model the one-genotype-per-lane kernel, so profiled calls keep it)
    const bool reps = !mixed && !a.lifo && !a.stats && S <= 16 && a.k >= 1 && a.k <= 32 &&
                      (g_reps_mode == 2 ||
                       (g_reps_mode == 0 && n_items * (size_t)a.k <= REPS_MAX_WORK * (a.n >= 3 ? 4 : 1)));
    const int rwarps = 3;  // with the small CTA histogram: 18 warps an SM (21 for sets of at most two tiles)
    long long rblocks = 0;
    if (reps && n_items) {
        int per_sm = 0;
        CUDA_TRY(classify_reps_prepare(S, tuple_table_size(a.n), rwarps, &per_sm));
        if (per_sm < 1) return fail(JATAM_ECUDA, "classification kernel does not fit on an SM");
        rblocks = (long long)per_sm * w->num_sms;
        const long long needed = (long long)((n_items + rwarps - 1) / rwarps);
        if (needed < rblocks) rblocks = needed < 1 ? 1 : needed;
    }
    int warps = tune.warps;
    const int nt = mixed ? 16 : tuple_table_size(a.n);
    long long blocks = 0;
    if (per_warp) {
        int per_sm = 0;
        CUDA_TRY(classify_warp_occupancy(&per_sm, &warps));
        if (per_sm < 1) return fail(JATAM_ECUDA, "classification kernel does not fit on an SM");
        blocks = (long long)per_sm * w->num_sms;
        const long long needed = (long long)((n_items + warps - 1) / warps);
        if (needed < blocks) blocks = needed < 1 ? 1 : needed;
    } else if (!mixed) {
        CUDA_TRY(classify_set_attributes(S, nt, warps, a.lifo != 0));
        int per_sm = 0;
        CUDA_TRY(classify_occupancy(S, nt, warps, &per_sm, a.lifo != 0));
        if (per_sm < 1) return fail(JATAM_ECUDA, "classification kernel does not fit on an SM");
        blocks = (long long)per_sm * w->num_sms;
        const long long lanes_per_cta = 32LL * warps;
        const long long needed = (long long)((n_items + lanes_per_cta - 1) / lanes_per_cta);
        if (needed < blocks) blocks = needed < 1 ? 1 : needed;
    }

    // the window launch (S = 16) and the full-lattice launch of the items that leave the window
    const Tuning tw = tuning_for(16, a.n, a.c);
    int wblocks = 0;
    if (windowed) {
        CUDA_TRY(classify_set_attributes(16, nt, tw.warps));
        int pw = 0;
        CUDA_TRY(classify_occupancy(16, nt, tw.warps, &pw));
        if (pw < 1) return fail(JATAM_ECUDA, "classification kernel does not fit on an SM");
        wblocks = pw * w->num_sms;
        const long long need = (long long)((n_items + 32LL * tw.warps - 1) / (32LL * tw.warps));
        if (need < wblocks) wblocks = need < 1 ? 1 : (int)need;
    }
    // the window launch of list `la.klass` on the 16 x 16 template, then the full 32 x 32 launch of
    // the items that left the window (their list in `esc`, its counters in `ctl`)
    auto launch_windowed = [&](const LaunchArgs &la, int ntw, int wwarps, int wstop, long long wb, int fwarps,
                               long long fb, int fstop, void *esc, unsigned long long *ctl,
                               cudaStream_t s) -> int {
        LaunchArgs aw = la;
        aw.esc_list = static_cast<unsigned long long *>(esc);
        aw.esc_count = ctl;
        aw.stop_at = wstop;
        CUDA_TRY(launch_classify(aw, 16, ntw, (int)(wb < 1 ? 1 : wb), wwarps, s));
        LaunchArgs af = la;
        af.esc_list = nullptr;
        af.esc_count = nullptr;
        af.list = static_cast<unsigned long long *>(esc);
        af.list_stride = la.list_stride;
        af.list_count = ctl;
        af.work_next = ctl + 6;
        af.klass = 0;
        af.bucket = 0;
        af.heavy_first = 0;  // the escalated items form one plain list
        af.stop_at = fstop;
        // (one genotype per warp here was measured 2x slower on the S_{3,8} sample: 143 against 75 ms)
        CUDA_TRY(launch_classify(af, 32, ntw, (int)(fb < 1 ? 1 : fb), fwarps, s));
        return JATAM_OK;
    };
    auto launch_growth = [&](const LaunchArgs &la, long long nb, cudaStream_t s, void *esc,
                             unsigned long long *ctl) -> int {
        if (reps) {
            CUDA_TRY(launch_classify_reps(la, S, nt, (int)rblocks, rwarps, s));
            return JATAM_OK;
        }
        if (windowed) {
            long long wb = (long long)((la.count + 32ull * tw.warps - 1) / (32ull * tw.warps));
            if (wb > wblocks) wb = wblocks;
            return launch_windowed(la, nt, tw.warps, tw.stop_at, wb, warps, nb, la.stop_at, esc, ctl, s);
        }
        CUDA_TRY(launch_classify(la, S, nt, (int)nb, warps, s));
        return JATAM_OK;
    };

    // heavy genotypes first when every lane of the growth launch takes at least
    // 8 genotypes on average (pieces of a pipelined call are at least 2^23)
    // (genotypes in progress at once: a lane's, or a warp's with one genotype per warp)
    const unsigned long long lanes = mixed ? 4ull * 160ull * (unsigned long long)w->num_sms  // about 4 CTAs of 5 warps an SM
                                   : reps ? (unsigned long long)rblocks * rwarps  // one genotype a warp
                                   : windowed ? (unsigned long long)wblocks * tw.warps * 32  // the window launch reads the list
                                           : (unsigned long long)blocks * warps * (per_warp ? 1 : 32);
    a.heavy_first = (n_items >= 8ull * lanes) ? ((!mixed && g_heavy_levels == 3) ? 2 : 1) : 0;

    a.lifo_stack = nullptr;
    if (a.lifo) {
        if (mixed) return fail(JATAM_EINVAL, "JATAM_LIFO needs items of one shape");
        const size_t bytes = (size_t)(blocks < 1 ? 1 : blocks) * warps * 32 * (size_t)S * S * 2;
        int rc = grow(&w->lifo_buf, &w->lifo_bytes, bytes);
        if (rc) return rc;
        a.lifo_stack = static_cast<uint16_t *>(w->lifo_buf);
    }

    // launch shapes of the growth kernels, fixed before anything is enqueued
    struct FixedLaunch {
        int S, blocks, warps, stop_at;
    } fixed[3] = {};
    if (n_items && mixed && per_shape) {
        for (int kc = 0; kc < 3; ++kc) {
            const int Sk = 8 << kc;
            const Tuning tk = tuning_for(Sk, 0, 0);
            CUDA_TRY(classify_set_attributes(Sk, 16, tk.warps));
            int pk = 0;
            CUDA_TRY(classify_occupancy(Sk, 16, tk.warps, &pk));
            if (pk < 1) return fail(JATAM_ECUDA, "classification kernel does not fit on an SM");
            fixed[kc] = {Sk, pk * w->num_sms, tk.warps, tk.stop_at};
        }
    }
    // mixed batches: one fixed launch per lattice size class, each over its own list (the window of
    // the uniform launches was measured slower here: 4.62 against 3.97 ms on the 10^7 batch, the extra
    // launch costing more than the class of lattices 17 to 32 gains)
    auto launch_per_size = [&](const LaunchArgs &la, cudaStream_t s) -> int {
        for (int kc = 0; kc < 3; ++kc) {
            LaunchArgs ak = la;
            ak.klass = kc;
            ak.stop_at = fixed[kc].stop_at;
            CUDA_TRY(launch_classify(ak, fixed[kc].S, 16, fixed[kc].blocks, fixed[kc].warps, s));
        }
        return JATAM_OK;
    };
    int mixed_blocks = 0;
    if (n_items && mixed && !per_shape) {
        int pm = 0;
        CUDA_TRY(classify_mixed_prepare(a.plan_w32, a.plan_w16, a.plan_w8, &pm));
        if (pm < 1) return fail(JATAM_ECUDA, "mixed classification kernel does not fit on an SM");
        mixed_blocks = pm * w->num_sms;
    }
    long long pblocks = (long long)(n_items + 255) / 256;
    if (pblocks > PF_CTAS_PER_SM * w->num_sms) pblocks = PF_CTAS_PER_SM * w->num_sms;
    const bool timed = (g_profile & 1) || kernel_ms;

    // the device work of the call; `events` brackets the growth kernels
    // the side table starts empty in every call that records shapes (keys and meta words; rows are
    // always written before their meta word)
    auto clear_shapes = [&](cudaStream_t s) -> int {
        if (!record_shapes) return JATAM_OK;
        CUDA_TRY(cudaMemsetAsync(w->shapes.key, 0, (size_t(8) + 4) << SHAPES_LOG2, s));
        CUDA_TRY(cudaMemsetAsync(w->shapes.stats, 0, 4 * 4, s));
        return JATAM_OK;
    };
    auto enqueue = [&](cudaStream_t s, bool events) -> int {
        if (int rc = clear_shapes(s)) return rc;
        CUDA_TRY(launch_reset(w->work_next, w->nkeys, w->list_count, s, w->crops, CROPS_LOG2, w->esc_ctl,
                              ESC_CTL_WORDS));
        if (a.stats) CUDA_TRY(cudaMemsetAsync(a.stats, 0, 4 * 8, s));
        if (n_items) CUDA_TRY(launch_prefilter(a, S, (int)pblocks, s));
        if (events) CUDA_TRY(cudaEventRecord(w->k_start, s));
        if (n_items && per_warp) CUDA_TRY(launch_classify_warp(a, (int)blocks, s));
        if (n_items && !mixed && !per_warp) {
            if (int rc = launch_growth(a, blocks, s, w->esc, w->esc_ctl)) return rc;
        }
        if (n_items && mixed && per_shape) {
            // one fixed launch per lattice size class, each over its own list
            if (int rc = launch_per_size(a, s)) return rc;
        }
        if (n_items && mixed && !per_shape) CUDA_TRY(launch_classify_mixed(a, mixed_blocks, s));
        if (n_items && dedup) CUDA_TRY(launch_dup_fill(a, (int)pblocks, s));
        if (events) CUDA_TRY(cudaEventRecord(w->k_stop, s));
        if (record_shapes) CUDA_TRY(launch_shape_scan(w->shapes, a.crops, CROPS_LOG2, a.spill, s));
        if (n_items && a.orbits) CUDA_TRY(launch_orbit_fill(a, (int)pblocks, s));
        if (hist) {
            CUDA_TRY(launch_hist_compact(w->table, w->compact, w->nkeys, 2 * w->num_sms, s,
                                         record_shapes ? w->shapes : ShapeTab{}));
            CUDA_TRY(launch_hist_emit(w->compact, w->nkeys, o.hist_dev, hist_cap,
                                      o.host_len ? nullptr : o.hist_len_dev, w->num_sms, s));
        }
        return JATAM_OK;
    };

    // results that go to page-locked host memory: classify the items in pieces
    // and copy each piece's results on a second stream while the next piece is
    // classified.  The phenotype table accumulates over the pieces and is
    // compacted once.  Not for records without stream ids (their stream id is
    // the item's index in the call), the orbit mode (members read their
    // representative's result anywhere in the range), graph replay or timed calls.
    // (device-output calls in pieces on two streams were measured too, with and without the window:
    // no faster on S_{3,8}, slower on S_{2,8})
    const bool pipelined = n_items >= 2 * PIPE_MIN_ITEMS && !use_graph && !timed && !a.orbits && !a.lifo &&
                           !(a.mode == MODE_RECORDS && !a.ids) && (o.host_out || o.host_fit) &&
                           (!o.host_out || is_pinned(out)) && (!o.host_fit || is_pinned(fitness));
    // record inputs in page-locked memory: copied piece by piece on a stream of their own
    const bool staged_pieces = pipelined && g_pipe_stage && hin && hin->any() &&
                               (!hin->colours || is_pinned(hin->colours)) && (!hin->shapes || is_pinned(hin->shapes)) &&
                               (!hin->ids || is_pinned(hin->ids));
    auto enqueue_pieces = [&](cudaStream_t s) -> int {
        PipeSchedule ps;
        if (!pipe_schedule(n_items, PIPE_MIN_ITEMS, windowed, staged_pieces, g_pipe_form, g_pipe_pieces, &ps))
            return fail(JATAM_EINVAL, "internal: piece schedule");
        const bool stagger = ps.stagger;
        const size_t *sizes = ps.sizes;
        const size_t per = ps.per;
        Workspace::Scratch &alt = w->alt;
        if (staged_pieces && !w->h2d) {
            CUDA_TRY(cudaStreamCreateWithFlags(&w->h2d, cudaStreamNonBlocking));
            for (int c = 0; c < PIPE_MAX_CHUNKS; ++c)
                CUDA_TRY(cudaEventCreateWithFlags(&w->in_ev[c], cudaEventDisableTiming));
        }
        if (!w->copy) {
            CUDA_TRY(cudaStreamCreateWithFlags(&w->aux, cudaStreamNonBlocking));
            CUDA_TRY(cudaStreamCreateWithFlags(&w->copy, cudaStreamNonBlocking));
            for (int c = 0; c < PIPE_MAX_CHUNKS; ++c) {
                CUDA_TRY(cudaEventCreateWithFlags(&w->pipe_ev[c], cudaEventDisableTiming));
                CUDA_TRY(cudaEventCreateWithFlags(&w->pf_ev[c], cudaEventDisableTiming));
            }
            CUDA_TRY(cudaEventCreateWithFlags(&w->pipe_start, cudaEventDisableTiming));
            CUDA_TRY(cudaEventCreateWithFlags(&w->aux_done, cudaEventDisableTiming));
            CUDA_TRY(cudaEventCreateWithFlags(&w->pipe_done, cudaEventDisableTiming));
            CUDA_TRY(cudaMalloc(&alt.work_next, 3 * 8));
            CUDA_TRY(cudaMalloc(&alt.list_count, 6 * 8));
            CUDA_TRY(cudaMalloc(&alt.nkeys, 4));
            CUDA_TRY(cudaMalloc(&alt.crops, (size_t(2) << CROPS_LOG2) * 8));
            CUDA_TRY(cudaMalloc(&alt.esc_ctl, ESC_CTL_WORDS * 8));
        }
        {
            int rc = grow(&alt.list, &alt.list_bytes, per * 8 * regions);
            if (rc) return rc;
            if (windowed) {
                rc = grow(&alt.esc, &alt.esc_bytes, per * 8);
                if (rc) return rc;
            }
            if (record_shapes) {
                rc = grow(reinterpret_cast<void **>(&alt.spill_rows), &alt.spill_bytes, spill_need);
                if (rc) return rc;
            }
        }
        if (a.stats) CUDA_TRY(cudaMemsetAsync(a.stats, 0, 4 * 8, s));
        if (int rc = clear_shapes(s)) return rc;
        CUDA_TRY(cudaEventRecord(w->pipe_start, s));
        CUDA_TRY(cudaStreamWaitEvent(w->aux, w->pipe_start, 0));
        int c = 0;
        for (size_t start = 0; start < n_items; start += sizes[c], ++c) {
            if (c >= PIPE_MAX_CHUNKS || sizes[c] == 0) return fail(JATAM_EINVAL, "internal: too many pieces");
            const size_t cnt = sizes[c];
            const bool odd = (c & 1) != 0;
            cudaStream_t cs = odd ? w->aux : s;
            unsigned long long *wn = odd ? alt.work_next : w->work_next;
            unsigned long long *lc = odd ? alt.list_count : w->list_count;
            unsigned long long *cr = odd ? alt.crops : w->crops;
            unsigned *nk = odd ? alt.nkeys : w->nkeys;
            void *esc = odd ? alt.esc : w->esc;
            unsigned long long *ectl = odd ? alt.esc_ctl : w->esc_ctl;
            LaunchArgs ac = a;
            ac.work_next = wn;
            ac.list_count = lc;
            ac.crops = g_crop_table ? cr : nullptr;
            ac.list = static_cast<unsigned long long *>(odd ? alt.list : w->list);
            ac.list_stride = per;
            ac.count = cnt;
            if (a.mode == MODE_RANGE || a.mode == MODE_SAMPLED) ac.first = a.first + start;
            if (a.mode == MODE_GENOMES) ac.genomes = a.genomes + start;
            if (a.mode == MODE_RECORDS) {
                ac.colours = a.colours + 16 * start;
                if (a.shapes) ac.shapes = a.shapes + 4 * start;
                ac.ids = a.ids + start;
            }
            if (a.out) ac.out = a.out + start;
            if (a.fitness) ac.fitness = a.fitness + start;
            ac.spill = spill_of(odd ? alt.spill_rows : w->spill_rows, ectl);
            if (staged_pieces) {
                // this piece's records, shapes and stream ids; the staging buffer is free once the
                // previous call has ended (pipe_start follows it on the caller's stream)
                if (c == 0) CUDA_TRY(cudaStreamWaitEvent(w->h2d, w->pipe_start, 0));
                if (hin->colours)
                    CUDA_TRY(cudaMemcpyAsync(hin->colours_dev + 16 * start, hin->colours + 16 * start, 16 * cnt,
                                             cudaMemcpyHostToDevice, w->h2d));
                if (hin->shapes)
                    CUDA_TRY(cudaMemcpyAsync(hin->shapes_dev + 4 * start, hin->shapes + 4 * start, 4 * cnt,
                                             cudaMemcpyHostToDevice, w->h2d));
                if (hin->ids)
                    CUDA_TRY(cudaMemcpyAsync(hin->ids_dev + start, hin->ids + start, 8 * cnt, cudaMemcpyHostToDevice,
                                             w->h2d));
                CUDA_TRY(cudaEventRecord(w->in_ev[c], w->h2d));
                CUDA_TRY(cudaStreamWaitEvent(cs, w->in_ev[c], 0));
            }
            if (stagger && c > 0) CUDA_TRY(cudaStreamWaitEvent(cs, w->pf_ev[c - 1], 0));
            CUDA_TRY(launch_reset(wn, nk, lc, cs, cr, CROPS_LOG2, ectl, ESC_CTL_WORDS));
            long long pb = (long long)(cnt + 255) / 256;
            if (pb > PF_CTAS_PER_SM * w->num_sms) pb = PF_CTAS_PER_SM * w->num_sms;
            CUDA_TRY(launch_prefilter(ac, S, (int)pb, cs));
            if (stagger) CUDA_TRY(cudaEventRecord(w->pf_ev[c], cs));
            if (per_warp) {
                long long bc = (long long)((cnt + warps - 1) / warps);
                if (bc > blocks) bc = blocks;
                CUDA_TRY(launch_classify_warp(ac, (int)(bc < 1 ? 1 : bc), cs));
            } else if (!mixed) {
                const long long lanes_per_cta = 32LL * warps;
                long long bc = (long long)((cnt + lanes_per_cta - 1) / lanes_per_cta);
                if (bc > blocks) bc = blocks;
                if (int rc = launch_growth(ac, bc < 1 ? 1 : bc, cs, esc, ectl)) return rc;
            } else if (per_shape) {
                if (int rc = launch_per_size(ac, cs)) return rc;
            } else {
                CUDA_TRY(launch_classify_mixed(ac, mixed_blocks, cs));
            }
            if (record_shapes) CUDA_TRY(launch_shape_scan(w->shapes, ac.crops, CROPS_LOG2, ac.spill, cs));
            CUDA_TRY(cudaEventRecord(w->pipe_ev[c], cs));
            CUDA_TRY(cudaStreamWaitEvent(w->copy, w->pipe_ev[c], 0));
            if (o.host_out)
                CUDA_TRY(cudaMemcpyAsync(out + start, o.out_dev + start, cnt * sizeof(jatam_result),
                                         cudaMemcpyDeviceToHost, w->copy));
            if (o.host_fit)
                CUDA_TRY(cudaMemcpyAsync(fitness + start, o.fit_dev + start, cnt * sizeof(int32_t),
                                         cudaMemcpyDeviceToHost, w->copy));
        }
        CUDA_TRY(cudaEventRecord(w->aux_done, w->aux));
        CUDA_TRY(cudaStreamWaitEvent(s, w->aux_done, 0));
        if (hist) {
            CUDA_TRY(launch_hist_compact(w->table, w->compact, w->nkeys, 2 * w->num_sms, s,
                                         record_shapes ? w->shapes : ShapeTab{}));
            CUDA_TRY(launch_hist_emit(w->compact, w->nkeys, o.hist_dev, hist_cap,
                                      o.host_len ? nullptr : o.hist_len_dev, w->num_sms, s));
        }
        CUDA_TRY(cudaEventRecord(w->pipe_done, w->copy));
        CUDA_TRY(cudaStreamWaitEvent(s, w->pipe_done, 0));
        return JATAM_OK;
    };

    CUDA_TRY(cudaStreamWaitEvent(st, w->last, 0));
    if (hin && hin->any() && !staged_pieces && n_items) {
        // host record inputs staged all at once, before the classification
        if (hin->colours)
            CUDA_TRY(cudaMemcpyAsync(hin->colours_dev, hin->colours, 16 * n_items, cudaMemcpyHostToDevice, st));
        if (hin->shapes)
            CUDA_TRY(cudaMemcpyAsync(hin->shapes_dev, hin->shapes, 4 * n_items, cudaMemcpyHostToDevice, st));
        if (hin->ids)
            CUDA_TRY(cudaMemcpyAsync(hin->ids_dev, hin->ids, 8 * n_items, cudaMemcpyHostToDevice, st));
    }
    if (pipelined) {
        int rc = enqueue_pieces(st);
        if (rc) return rc;
    } else if (!use_graph) {
        int rc = enqueue(st, timed);
        if (rc) return rc;
    } else {
        // one instantiated graph per distinct argument set, replayed on the caller's stream
        std::string key;
        auto put = [&key](const void *p, size_t n) { key.append(static_cast<const char *>(p), n); };
        const void *ptrs[] = {a.colours, a.shapes, a.ids, a.genomes, a.out, a.fitness, a.list, o.hist_dev,
                              o.host_len ? nullptr : o.hist_len_dev, a.lifo_stack, w->esc, a.dup_keys, a.dup_owner, a.dup_slot};
        put(ptrs, sizeof ptrs);
        const long long nums[] = {a.mode, (long long)a.first, (long long)a.count, a.n, a.c, a.L, a.k, a.key0, a.key1,
                                  a.use_hist, a.stop_at, (long long)a.list_stride, a.bucket, a.plan_w32, a.plan_w16,
                                  a.plan_w8, S, blocks, warps, per_shape, mixed_blocks, pblocks, hist_cap,
                                  fixed[0].blocks, fixed[0].warps, fixed[0].stop_at, fixed[1].blocks, fixed[1].warps,
                                  fixed[1].stop_at, fixed[2].blocks, fixed[2].warps, fixed[2].stop_at,
                                  a.stats ? 1 : 0, a.c4, a.orbits, per_warp ? 1 : 0, windowed ? 1 : 0,
                                  wblocks, tw.warps, tw.stop_at, g_heavy_levels, reps ? 1 : 0, rblocks,
                                  (long long)a.dup_mask};
        put(nums, sizeof nums);
        cudaGraphExec_t exec = nullptr;
        auto it = w->graphs.find(key);
        if (it != w->graphs.end()) {
            exec = it->second;
        } else {
            if (w->graphs.size() >= 64) {
                for (auto &kv : w->graphs) cudaGraphExecDestroy(kv.second);
                w->graphs.clear();
            }
            if (!w->capture) CUDA_TRY(cudaStreamCreateWithFlags(&w->capture, cudaStreamNonBlocking));
            cudaGraph_t graph = nullptr;
            CUDA_TRY(cudaStreamBeginCapture(w->capture, cudaStreamCaptureModeThreadLocal));
            const int rc = enqueue(w->capture, false);
            cudaError_t ec = cudaStreamEndCapture(w->capture, &graph);
            if (rc) {
                if (graph) cudaGraphDestroy(graph);
                return rc;
            }
            if (ec != cudaSuccess) return fail(JATAM_ECUDA, "stream capture failed: %s", cudaGetErrorString(ec));
            ec = cudaGraphInstantiate(&exec, graph, 0);
            cudaGraphDestroy(graph);
            if (ec != cudaSuccess) return fail(JATAM_ECUDA, "graph instantiation failed: %s", cudaGetErrorString(ec));
            w->graphs[key] = exec;
        }
        if (timed) CUDA_TRY(cudaEventRecord(w->k_start, st));
        CUDA_TRY(cudaGraphLaunch(exec, st));
        if (timed) CUDA_TRY(cudaEventRecord(w->k_stop, st));
    }
    if (timed) w->k_valid = true;
    w->stats_valid = a.stats != nullptr;
    w->shapes_valid = record_shapes;
    if (o.host_out && n_items && !pipelined)
        CUDA_TRY(cudaMemcpyAsync(out, o.out_dev, n_items * sizeof(jatam_result), cudaMemcpyDeviceToHost, st));
    if (o.host_fit && n_items && !pipelined)
        CUDA_TRY(cudaMemcpyAsync(fitness, o.fit_dev, n_items * sizeof(int32_t), cudaMemcpyDeviceToHost, st));
    const bool must_sync = sync_flag || o.host_out || o.host_fit || o.host_hist || o.host_len;
    if (must_sync) {
        CUDA_TRY(cudaMemcpyAsync(&w->host_words[0], w->err, 4, cudaMemcpyDeviceToHost, st));
        CUDA_TRY(cudaMemcpyAsync(&w->host_words[1], w->nkeys, 4, cudaMemcpyDeviceToHost, st));
    }
    CUDA_TRY(cudaEventRecord(w->last, st));
    if (kernel_ms) {
        CUDA_TRY(cudaEventSynchronize(w->k_stop));
        CUDA_TRY(cudaEventElapsedTime(kernel_ms, w->k_start, w->k_stop));
    }
    if (!must_sync) return JATAM_OK;
    CUDA_TRY(cudaStreamSynchronize(st));
    const unsigned err = w->host_words[0];
    const unsigned nk = w->host_words[1];
    if (hist) {
        if (o.host_len) *hist_len = nk;
        if (o.host_hist && nk) {
            const size_t nc = nk < hist_cap ? nk : hist_cap;
            CUDA_TRY(cudaMemcpy(hist, o.hist_dev, nc * sizeof(jatam_hist_entry), cudaMemcpyDeviceToHost));
        }
    }
    if (err) {
        CUDA_TRY(cudaMemsetAsync(w->err, 0, 4, st));
        CUDA_TRY(cudaStreamSynchronize(st));
        if (err & ERR_GUARD) return fail(JATAM_ETIMEOUT, "a bounded device loop found an inconsistent state");
        if (err & ERR_TABLE_FULL) return fail(JATAM_ENOMEM, "the phenotype table (%u slots) overflowed", 1u << TABLE_LOG2);
        if (err & ERR_INVALID_ITEM) return fail(JATAM_EINVAL, "an item had a colour >= c or parameters out of range");
    }
    if (hist && nk > hist_cap && (o.host_len))
        return fail(JATAM_EINVAL, "histogram has %u keys but hist_cap is %u", nk, hist_cap);
    return JATAM_OK;
}

// copy a host input to the staging buffer, or pass a device pointer through
int stage_input(Workspace *w, const void *p, size_t bytes, void **stage, size_t *have, const void **dev,
                cudaStream_t st)
{
    Kind k = kind_of(p, w->device);
    if (k == K_NULL && p) return fail(JATAM_EINVAL, "an input buffer lives on another device");
    if (k != K_HOST) {
        *dev = p;
        return JATAM_OK;
    }
    int rc = grow(stage, have, bytes);
    if (rc) return rc;
    CUDA_TRY(cudaMemcpyAsync(*stage, p, bytes, cudaMemcpyHostToDevice, st));
    *dev = *stage;
    return JATAM_OK;
}

}  // namespace

void jatam::set_last_error(const char *msg) { g_last_error = msg; }

extern "C" {

int jatam_enumerate(const jatam_config *cfg, uint64_t first, uint64_t count, jatam_result *out,
                    jatam_hist_entry *hist, uint32_t hist_cap, uint32_t *hist_len, void *stream)
{
    std::lock_guard<std::mutex> lock(g_mutex);
    g_last_error.clear();
    if (!cfg) return fail(JATAM_EINVAL, "cfg is NULL");
    int rc = check_params(cfg->n, cfg->c, cfg->L, cfg->k, true);
    if (rc) return rc;
    const int bits = 4 * cfg->n * log2c(cfg->c);
    const bool sampled = (cfg->flags & JATAM_SAMPLED) != 0;
    if (!sampled) {
        const uint64_t space = bits >= 64 ? ~0ull : (1ull << bits);
        if (first > space || count > space - first)
            return fail(JATAM_EINVAL, "index range [%llu, %llu + %llu) exceeds the %d-bit space", (unsigned long long)first,
                        (unsigned long long)first, (unsigned long long)count, bits);
    } else if (count > ~0ull - first) {
        return fail(JATAM_EINVAL, "index range overflows");
    }
    const bool orbits = (cfg->flags & JATAM_ORBITS) != 0;
    if (orbits && (sampled || first != 0))
        return fail(JATAM_EINVAL, "JATAM_ORBITS needs an index range that starts at genotype 0");
    Workspace *w = nullptr;
    rc = workspace(&w);
    if (rc) return rc;
    LaunchArgs a{};
    a.mode = sampled ? MODE_SAMPLED : MODE_RANGE;
    a.first = first;
    a.count = count;
    a.orbits = orbits ? 1 : 0;
    a.lifo = (cfg->flags & JATAM_LIFO) ? 1 : 0;
    a.c4 = (cfg->flags & JATAM_C4_HASH) ? 1 : 0;
    a.n = cfg->n; a.c = cfg->c; a.L = cfg->L; a.k = cfg->k;
    a.key0 = (uint32_t)cfg->seed;
    a.key1 = (uint32_t)(cfg->seed >> 32);
    return run(w, a, lattice_template(cfg->L), out, nullptr, hist, hist_cap, hist_len,
               (cfg->flags & JATAM_SYNC) != 0, static_cast<cudaStream_t>(stream), nullptr, nullptr, false,
               (cfg->flags & JATAM_GRAPH) != 0);
}

int jatam_classify_batch(const jatam_config *cfg, const uint8_t *colours, const uint8_t *shapes,
                         const uint64_t *stream_ids, uint64_t N, jatam_result *out, jatam_hist_entry *hist,
                         uint32_t hist_cap, uint32_t *hist_len, void *stream)
{
    std::lock_guard<std::mutex> lock(g_mutex);
    g_last_error.clear();
    if (!cfg) return fail(JATAM_EINVAL, "cfg is NULL");
    if (N && !colours) return fail(JATAM_EINVAL, "colours is NULL");
    if ((reinterpret_cast<uintptr_t>(colours) & 15) || (reinterpret_cast<uintptr_t>(shapes) & 3) ||
        (reinterpret_cast<uintptr_t>(stream_ids) & 7))
        return fail(JATAM_EINVAL, "colours must be 16-byte, shapes 4-byte and stream_ids 8-byte aligned");
    int S = 32;
    if (!shapes) {
        int rc = check_params(cfg->n, cfg->c, cfg->L, cfg->k, false);
        if (rc) return rc;
        S = lattice_template(cfg->L);
    }
    Workspace *w = nullptr;
    int rc = workspace(&w);
    if (rc) return rc;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    CUDA_TRY(cudaStreamWaitEvent(st, w->last, 0));
    LaunchArgs a{};
    a.mode = MODE_RECORDS;
    a.count = N;
    a.lifo = (cfg->flags & JATAM_LIFO) ? 1 : 0;
    a.c4 = (cfg->flags & JATAM_C4_HASH) ? 1 : 0;
    a.n = cfg->n; a.c = cfg->c; a.L = cfg->L; a.k = cfg->k;
    a.key0 = (uint32_t)cfg->seed;
    a.key1 = (uint32_t)(cfg->seed >> 32);
    // stage host inputs one after the other in stage_in (16-byte aligned pieces)
    const size_t cb = (size_t)N * 16, sb = shapes ? (size_t)N * 4 : 0, ib = stream_ids ? (size_t)N * 8 : 0;
    const size_t off_s = (cb + 255) & ~size_t(255), off_i = (off_s + sb + 255) & ~size_t(255);
    const Kind kc = kind_of(colours, w->device), ks = kind_of(shapes, w->device), ki = kind_of(stream_ids, w->device);
    if ((kc == K_NULL && colours) || (ks == K_NULL && shapes) || (ki == K_NULL && stream_ids))
        return fail(JATAM_EINVAL, "an input buffer lives on another device");
    if (kc == K_HOST || ks == K_HOST || ki == K_HOST) {
        rc = grow(&w->stage_in, &w->stage_in_bytes, off_i + ib + 256);
        if (rc) return rc;
    }
    // host inputs: run() copies them into stage_in, at once or piece by piece
    char *base = static_cast<char *>(w->stage_in);
    HostInputs hin;
    a.colours = colours;
    if (kc == K_HOST && N) {
        hin.colours = colours;
        hin.colours_dev = reinterpret_cast<uint8_t *>(base);
        a.colours = hin.colours_dev;
    }
    a.shapes = shapes;
    if (ks == K_HOST && N) {
        hin.shapes = shapes;
        hin.shapes_dev = reinterpret_cast<uint8_t *>(base + off_s);
        a.shapes = hin.shapes_dev;
    }
    a.ids = reinterpret_cast<const unsigned long long *>(stream_ids);
    if (ki == K_HOST && N) {
        hin.ids = reinterpret_cast<const unsigned long long *>(stream_ids);
        hin.ids_dev = reinterpret_cast<unsigned long long *>(base + off_i);
        a.ids = hin.ids_dev;
    }
    return run(w, a, S, out, nullptr, hist, hist_cap, hist_len, (cfg->flags & JATAM_SYNC) != 0, st, nullptr, nullptr,
               (cfg->flags & JATAM_PER_SHAPE) != 0 || (!(cfg->flags & JATAM_PERSISTENT) && g_mixed_per_shape),
               (cfg->flags & JATAM_GRAPH) != 0, &hin);
}

int ga_evaluate(const jatam_config *cfg, const uint64_t *genomes, uint64_t N, int32_t *fitness, jatam_result *out,
                void *stream)
{
    std::lock_guard<std::mutex> lock(g_mutex);
    g_last_error.clear();
    if (!cfg) return fail(JATAM_EINVAL, "cfg is NULL");
    if (!fitness) return fail(JATAM_EINVAL, "fitness is NULL");
    if (N && !genomes) return fail(JATAM_EINVAL, "genomes is NULL");
    if (reinterpret_cast<uintptr_t>(genomes) & 7) return fail(JATAM_EINVAL, "genomes must be 8-byte aligned");
    int rc = check_params(cfg->n, cfg->c, cfg->L, cfg->k, true);
    if (rc) return rc;
    Workspace *w = nullptr;
    rc = workspace(&w);
    if (rc) return rc;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    CUDA_TRY(cudaStreamWaitEvent(st, w->last, 0));
    const void *gdev = nullptr;
    rc = stage_input(w, genomes, (size_t)N * 8, &w->stage_in, &w->stage_in_bytes, &gdev, st);
    if (rc) return rc;
    LaunchArgs a{};
    a.mode = MODE_GENOMES;
    a.count = N;
    a.lifo = (cfg->flags & JATAM_LIFO) ? 1 : 0;
    a.c4 = (cfg->flags & JATAM_C4_HASH) ? 1 : 0;
    a.no_dedup = (cfg->flags & JATAM_NO_DEDUP) ? 1 : 0;
    a.genomes = static_cast<const unsigned long long *>(gdev);
    a.n = cfg->n; a.c = cfg->c; a.L = cfg->L; a.k = cfg->k;
    a.key0 = (uint32_t)cfg->seed;
    a.key1 = (uint32_t)(cfg->seed >> 32);
    return run(w, a, lattice_template(cfg->L), out, fitness, nullptr, 0, nullptr, (cfg->flags & JATAM_SYNC) != 0, st,
               nullptr, nullptr, false, (cfg->flags & JATAM_GRAPH) != 0);
}

namespace {

int check_ga(const jatam_ga_config *ga, GaArgs *g)
{
    if (!ga) return fail(JATAM_EINVAL, "ga is NULL");
    int rc = check_params(ga->n, ga->c, 1, 1, true);
    if (rc) return rc;
    if (ga->selection > 1 || ga->crossover > 2 || (ga->selection == 0 && (ga->tournament < 1 || ga->tournament > 16)))
        return fail(JATAM_EINVAL, "selection 0/1, tournament 1..16, crossover 0..2");
    for (int j = 1; j < 4; ++j)
        if (ga->mutation_thresholds[j] < ga->mutation_thresholds[j - 1])
            return fail(JATAM_EINVAL, "mutation thresholds must not decrease");
    *g = GaArgs{};
    g->n = ga->n;
    g->c = ga->c;
    g->b = log2c(ga->c);
    g->bits = 4 * ga->n * g->b;
    g->selection = ga->selection;
    g->tournament = ga->tournament;
    g->crossover = ga->crossover;
    g->crossover_threshold = ga->crossover_threshold;
    for (int j = 0; j < 4; ++j) g->mutation_thresholds[j] = ga->mutation_thresholds[j];
    g->key0 = (uint32_t)ga->seed;
    g->key1 = (uint32_t)(ga->seed >> 32);
    if (g->crossover == 1 && g->bits < 2) return fail(JATAM_EINVAL, "one-point crossover needs at least 2 bits");
    return JATAM_OK;
}

// GA scratch: [fitness N x 4][children N x 8][cumsum N x 8][stats 16], 256-byte aligned pieces
struct GaScratch {
    int32_t *fitness;
    unsigned long long *children, *cumsum;
    jatam_result *results;  // the population's classification (online training of a screening network)
    uint8_t *labels;
    long long *stats;
};

int ga_scratch(Workspace *w, uint64_t N, GaScratch *s)
{
    const size_t a = ((size_t)N * 4 + 255) & ~size_t(255), b = ((size_t)N * 8 + 255) & ~size_t(255);
    const size_t c = ((size_t)N + 255) & ~size_t(255);
    int rc = grow(&w->ga_buf, &w->ga_bytes, a + 3 * b + c + 256);
    if (rc) return rc;
    char *p = static_cast<char *>(w->ga_buf);
    s->fitness = reinterpret_cast<int32_t *>(p);
    s->children = reinterpret_cast<unsigned long long *>(p + a);
    s->cumsum = reinterpret_cast<unsigned long long *>(p + a + b);
    s->results = reinterpret_cast<jatam_result *>(p + a + 2 * b);
    s->labels = reinterpret_cast<uint8_t *>(p + a + 3 * b);
    s->stats = reinterpret_cast<long long *>(p + a + 3 * b + c);
    return JATAM_OK;
}

}  // namespace

int ga_breed(const jatam_ga_config *ga, const uint64_t *parents, const int32_t *fitness, uint64_t N,
             uint32_t generation, uint64_t *children, void *stream)
{
    std::lock_guard<std::mutex> lock(g_mutex);
    g_last_error.clear();
    GaArgs g;
    int rc = check_ga(ga, &g);
    if (rc) return rc;
    if (N && (!parents || !fitness || !children)) return fail(JATAM_EINVAL, "parents, fitness, children required");
    if (N == 0) return JATAM_OK;
    if (generation >= (1u << 24)) return fail(JATAM_EINVAL, "generation must be < 2^24");
    Workspace *w = nullptr;
    rc = workspace(&w);
    if (rc) return rc;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    CUDA_TRY(cudaStreamWaitEvent(st, w->last, 0));
    GaScratch sc;
    rc = ga_scratch(w, 2 * N, &sc);  // room to stage host parents next to the children
    if (rc) return rc;
    const Kind kp = kind_of(parents, w->device), kf = kind_of(fitness, w->device), kc = kind_of(children, w->device);
    if ((kp == K_NULL) || (kf == K_NULL) || (kc == K_NULL)) return fail(JATAM_EINVAL, "a buffer lives on another device");
    const unsigned long long *dp = reinterpret_cast<const unsigned long long *>(parents);
    const int32_t *df = fitness;
    if (kp == K_HOST) {
        CUDA_TRY(cudaMemcpyAsync(sc.cumsum + N, parents, (size_t)N * 8, cudaMemcpyHostToDevice, st));
        dp = sc.cumsum + N;
    }
    if (kf == K_HOST) {
        CUDA_TRY(cudaMemcpyAsync(sc.fitness, fitness, (size_t)N * 4, cudaMemcpyHostToDevice, st));
        df = sc.fitness;
    }
    unsigned long long *dc = kc == K_HOST ? sc.children : reinterpret_cast<unsigned long long *>(children);
    g.parents = dp;
    g.fitness = df;
    g.cumsum = sc.cumsum;
    g.N = N;
    g.Nc = N;
    g.generation = generation;
    g.children = dc;
    CUDA_TRY(launch_ga_breed(g, st));
    if (kc == K_HOST) CUDA_TRY(cudaMemcpyAsync(children, dc, (size_t)N * 8, cudaMemcpyDeviceToHost, st));
    CUDA_TRY(cudaEventRecord(w->last, st));
    if (kc == K_HOST || kp == K_HOST || kf == K_HOST) CUDA_TRY(cudaStreamSynchronize(st));
    return JATAM_OK;
}

int ga_hamming(const uint64_t *genomes, uint64_t N, int32_t *fitness, void *stream)
{
    std::lock_guard<std::mutex> lock(g_mutex);
    g_last_error.clear();
    if (N && (!genomes || !fitness)) return fail(JATAM_EINVAL, "genomes and fitness required");
    if (N == 0) return JATAM_OK;
    Workspace *w = nullptr;
    int rc = workspace(&w);
    if (rc) return rc;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    CUDA_TRY(cudaStreamWaitEvent(st, w->last, 0));
    GaScratch sc;
    rc = ga_scratch(w, N, &sc);
    if (rc) return rc;
    const Kind kg = kind_of(genomes, w->device), kf = kind_of(fitness, w->device);
    const unsigned long long *dg = reinterpret_cast<const unsigned long long *>(genomes);
    if (kg == K_HOST) {
        CUDA_TRY(cudaMemcpyAsync(sc.children, genomes, (size_t)N * 8, cudaMemcpyHostToDevice, st));
        dg = sc.children;
    }
    int32_t *df = kf == K_HOST ? sc.fitness : fitness;
    CUDA_TRY(launch_ga_hamming(dg, N, df, st));
    if (kf == K_HOST) CUDA_TRY(cudaMemcpyAsync(fitness, df, (size_t)N * 4, cudaMemcpyDeviceToHost, st));
    CUDA_TRY(cudaEventRecord(w->last, st));
    if (kf == K_HOST || kg == K_HOST) CUDA_TRY(cudaStreamSynchronize(st));
    return JATAM_OK;
}

int ga_poisson_thresholds(double rate, uint32_t thresholds[4])
{
    g_last_error.clear();
    if (!thresholds || !(rate >= 0.0)) return fail(JATAM_EINVAL, "rate must be >= 0 and thresholds non-NULL");
    double term = exp(-rate), cdf = 0.0;
    for (int j = 0; j < 4; ++j) {
        cdf += term;
        term *= rate / (double)(j + 1);
        const double t = floor(cdf * 4294967296.0);
        thresholds[j] = t >= 4294967295.0 ? 4294967295u : (uint32_t)t;
    }
    return JATAM_OK;
}

}  // extern "C"

namespace {
// The GA loop; with a network, each generation breeds ratio x N candidates,
// the network scores them and the best N (the only ones simulated) form the
// next population.
int ga_loop(const jatam_ga_config *ga, const jatam_config *cls, int fitness_kind, uint64_t N, uint32_t generations,
            uint64_t *population, int32_t *best, int64_t *total, void *stream, jatam_mlp *net, uint32_t ratio,
            float online_lr)
{
    GaArgs g;
    {
        std::lock_guard<std::mutex> lock(g_mutex);
        g_last_error.clear();
        int rc = check_ga(ga, &g);
        if (rc) return rc;
        if (fitness_kind != JATAM_GA_FITNESS_SHAPE && fitness_kind != JATAM_GA_FITNESS_HAMMING)
            return fail(JATAM_EINVAL, "fitness_kind must be JATAM_GA_FITNESS_SHAPE or _HAMMING");
        if (fitness_kind == JATAM_GA_FITNESS_SHAPE && !cls) return fail(JATAM_EINVAL, "cls is required for shape fitness");
        if (!population || N == 0) return fail(JATAM_EINVAL, "population and N > 0 are required");
        if (generations >= (1u << 24)) return fail(JATAM_EINVAL, "generations must be < 2^24");
    }
    Workspace *w = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_mutex);
        int rc = workspace(&w);
        if (rc) return rc;
        if (kind_of(population, w->device) != K_DEVICE) return fail(JATAM_EINVAL, "population must be device memory");
        if (net) {
            const unsigned long long M = (unsigned long long)N * ratio;
            if (ratio < 1 || (long long)M > net->b.cap || M > (1ull << 26))
                return fail(JATAM_EINVAL, "ratio x N must be at least N and fit the network's batch capacity");
            unsigned cap = 1;
            while (cap < 2 * M) cap <<= 1;
            const size_t a8 = ((size_t)M * 8 + 255) & ~size_t(255), a4 = ((size_t)M * 4 + 255) & ~size_t(255);
            const size_t need = 2 * a8 + a4 + (size_t)cap * 12 + a4 + 256 + 1024 + TOPN_SCRATCH_BYTES + 256;
            rc = grow(&w->screen_buf, &w->screen_bytes, need);
            if (rc) return rc;
            char *p = static_cast<char *>(w->screen_buf);
            w->screen_cand = reinterpret_cast<unsigned long long *>(p);
            w->screen_idx = reinterpret_cast<unsigned long long *>(p + a8);
            w->screen_score = reinterpret_cast<float *>(p + 2 * a8);
            w->screen_table.keys = reinterpret_cast<unsigned long long *>(p + 2 * a8 + a4);
            w->screen_table.first = reinterpret_cast<unsigned *>(p + 2 * a8 + a4 + (size_t)cap * 8);
            w->screen_table.slot = reinterpret_cast<unsigned *>(p + 2 * a8 + a4 + (size_t)cap * 12);
            w->screen_table.err = reinterpret_cast<unsigned *>(p + 2 * a8 + a4 + (size_t)cap * 12 + a4);
            w->screen_table.cap_mask = cap - 1;
            w->screen_table.topn = reinterpret_cast<unsigned *>(p + ((2 * a8 + a4 + (size_t)cap * 12 + a4 + 256 + 1024 +
                                                                      255) & ~size_t(255)));
        }
    }
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const Kind kb = kind_of(best, w->device), kt = kind_of(total, w->device);
    std::vector<long long> host_stats;
    if (kb == K_HOST || kt == K_HOST) host_stats.resize(2 * (size_t)generations);
    jatam_config cc{};
    if (cls) cc = *cls;
    cc.n = ga->n;
    cc.c = ga->c;
    // the fitness call is the same every generation: replay its graph; a screened population is chosen
    // distinct (repeats rank last), so it skips the repeat table
    cc.flags = JATAM_GRAPH | (net ? JATAM_NO_DEDUP : 0u);
    unsigned long long *pop = reinterpret_cast<unsigned long long *>(population);
    for (uint32_t gen = 0; gen < generations; ++gen) {
        GaScratch sc;
        {
            std::lock_guard<std::mutex> lock(g_mutex);
            int rc = ga_scratch(w, N, &sc);
            if (rc) return rc;
        }
        int rc = (fitness_kind == JATAM_GA_FITNESS_SHAPE)
                     ? ga_evaluate(&cc, reinterpret_cast<const uint64_t *>(pop), N, sc.fitness,
                                   net ? sc.results : nullptr, stream)
                     : ga_hamming(reinterpret_cast<const uint64_t *>(pop), N, sc.fitness, stream);
        if (rc) return rc;
        std::lock_guard<std::mutex> lock(g_mutex);
        CUDA_TRY(launch_ga_stats(sc.fitness, N, sc.stats, st));
        if (kb == K_DEVICE) CUDA_TRY(cudaMemcpyAsync(best + gen, sc.stats, 4, cudaMemcpyDeviceToDevice, st));
        if (kt == K_DEVICE) CUDA_TRY(cudaMemcpyAsync(total + gen, sc.stats + 1, 8, cudaMemcpyDeviceToDevice, st));
        if (!host_stats.empty())
            CUDA_TRY(cudaMemcpyAsync(&host_stats[2 * gen], sc.stats, 16, cudaMemcpyDeviceToHost, st));
        GaArgs gg = g;
        gg.parents = pop;
        gg.fitness = sc.fitness;
        gg.cumsum = sc.cumsum;
        gg.N = N;
        gg.Nc = N;
        gg.generation = gen;
        gg.children = sc.children;
        if (!net) {
            CUDA_TRY(launch_ga_breed(gg, st));
            CUDA_TRY(cudaMemcpyAsync(pop, sc.children, (size_t)N * 8, cudaMemcpyDeviceToDevice, st));
        } else {
            if (online_lr > 0.f) {
                // the simulated population, labelled by its own results, trains the network
                CUDA_TRY(launch_mlp_labels(sc.results, (long long)N, sc.labels, st));
                CUDA_TRY(mlp_forward(net->b, pop, (long long)N, st));
                CUDA_TRY(mlp_backward(net->b, sc.labels, (long long)N, st));
                net->t += 1;
                CUDA_TRY(mlp_adam(net->b, online_lr, net->t, st));
            }
            const unsigned long long M = (unsigned long long)N * ratio;
            gg.Nc = M;
            gg.children = w->screen_cand;
            CUDA_TRY(launch_ga_breed(gg, st));
            CUDA_TRY(mlp_forward(net->b, w->screen_cand, (long long)M, st, true));
            CUDA_TRY(launch_screen(net->b.logits, (long long)M, (long long)N, w->screen_score, w->screen_idx,
                                   w->screen_cand, pop, w->screen_table, st));
        }
        CUDA_TRY(cudaEventRecord(w->last, st));
        if (!host_stats.empty()) CUDA_TRY(cudaStreamSynchronize(st));  // host_stats must not be read early
    }
    if (!host_stats.empty()) {
        for (uint32_t gen = 0; gen < generations; ++gen) {
            if (kb == K_HOST) best[gen] = (int32_t)host_stats[2 * gen];
            if (kt == K_HOST) total[gen] = host_stats[2 * gen + 1];
        }
    }
    return JATAM_OK;
}

// after a synchronisation: a bounded wait of the tcgen05 products that ran out
int mlp_tc_status(jatam_mlp *m)
{
    if (!m->b.tc) return JATAM_OK;
    unsigned e = 0;
    CUDA_TRY(cudaMemcpy(&e, m->b.tc_err, 4, cudaMemcpyDeviceToHost));
    if (!e) return JATAM_OK;
    CUDA_TRY(cudaMemset(m->b.tc_err, 0, 4));
    return fail(JATAM_ETIMEOUT, "a tensor-core product gave up waiting for its result");
}

}  // namespace

extern "C" {

int ga_run(const jatam_ga_config *ga, const jatam_config *cls, int fitness_kind, uint64_t N, uint32_t generations,
           uint64_t *population, int32_t *best, int64_t *total, void *stream)
{
    return ga_loop(ga, cls, fitness_kind, N, generations, population, best, total, stream, nullptr, 1, 0.f);
}

int ga_run_screened(const jatam_ga_config *ga, const jatam_config *cls, uint64_t N, uint32_t generations,
                    uint32_t ratio, jatam_mlp *net, float online_lr, uint64_t *population, int32_t *best,
                    int64_t *total, void *stream)
{
    if (!net || !(online_lr >= 0.f) || online_lr > 1.f) {
        std::lock_guard<std::mutex> lock(g_mutex);
        return fail(JATAM_EINVAL, "net is required and 0 <= online_lr <= 1");
    }
    return ga_loop(ga, cls, JATAM_GA_FITNESS_SHAPE, N, generations, population, best, total, stream, net, ratio,
                   online_lr);
}

int jatam_mlp_create(uint64_t max_batch, jatam_mlp **net)
{
    std::lock_guard<std::mutex> lock(g_mutex);
    g_last_error.clear();
    if (!net || max_batch == 0 || max_batch > (1ull << 26)) return fail(JATAM_EINVAL, "net required, 1 <= max_batch <= 2^26");
    if (MLP_NPARAM != JATAM_MLP_NPARAM) return fail(JATAM_EINVAL, "parameter count mismatch");
    jatam_mlp *m = new jatam_mlp();
    CUDA_TRY(cudaGetDevice(&m->device));
    const long long P = MLP_NPARAM, Bc = (long long)max_batch;
    MlpBuffers &b = m->b;
    b.cap = Bc;
    auto alloc = [&](void **p, size_t bytes) -> int {
        cudaError_t e = cudaMalloc(p, bytes);
        if (e != cudaSuccess) {
            cudaGetLastError();
            return fail(JATAM_ENOMEM, "cudaMalloc of %zu bytes failed", bytes);
        }
        return JATAM_OK;
    };
    int rc = 0;
    rc |= alloc((void **)&b.p, P * 4); rc |= alloc((void **)&b.grad, P * 4);
    rc |= alloc((void **)&b.m, P * 4); rc |= alloc((void **)&b.v, P * 4);
    rc |= alloc((void **)&b.wq, P * 2);
    rc |= alloc((void **)&b.x, Bc * MLP_PAD * 2); rc |= alloc((void **)&b.h1, Bc * MLP_H * 2);
    rc |= alloc((void **)&b.h2, Bc * MLP_H * 2); rc |= alloc((void **)&b.dq, Bc * MLP_OUT * 2);
    rc |= alloc((void **)&b.dh1, Bc * MLP_H * 2); rc |= alloc((void **)&b.dh2, Bc * MLP_H * 2);
    rc |= alloc((void **)&b.logits, Bc * MLP_OUT * 4); rc |= alloc((void **)&b.d, Bc * MLP_OUT * 4);
    rc |= alloc((void **)&b.lrow, (Bc + 64) * 4);  // 9 partial sums a block of 256 rows
    rc |= alloc((void **)&b.splitk, (size_t)MLP_SPLITK_MAX * MLP_H * MLP_H * 4);
    rc |= alloc((void **)&b.tc_err, 4);
    rc |= alloc((void **)&b.wqt, (size_t)(MLP_PAD * MLP_H + MLP_H * MLP_H) * 2);
    rc |= alloc((void **)&b.loss, 16);
    if (rc) {
        jatam_mlp_destroy(m);
        return JATAM_ENOMEM;
    }
    CUDA_TRY(cudaMemset(b.p, 0, P * 4));
    CUDA_TRY(cudaMemset(b.m, 0, P * 4));
    CUDA_TRY(cudaMemset(b.v, 0, P * 4));
    CUDA_TRY(cudaMemset(b.wq, 0, P * 2));
    CUDA_TRY(cudaMemset(b.tc_err, 0, 4));
    CUDA_TRY(cudaMemset(b.wqt, 0, (size_t)(MLP_PAD * MLP_H + MLP_H * MLP_H) * 2));
    {
        // JATAM_MLP_PRODUCTS=mma keeps every product on mma.sync (for comparisons)
        const char *v = getenv("JATAM_MLP_PRODUCTS");
        b.tc = (v && strcmp(v, "mma") == 0) ? 0 : 1;
    }
    *net = m;
    return JATAM_OK;
}

void jatam_mlp_destroy(jatam_mlp *m)
{
    if (!m) return;
    MlpBuffers &b = m->b;
    void *ptrs[] = {b.p, b.grad, b.m, b.v, b.wq, b.x, b.h1, b.h2, b.dq, b.dh1, b.dh2, b.logits, b.d, b.lrow, b.loss,
                    b.splitk, b.tc_err, b.wqt, m->stage};
    cudaDeviceSynchronize();
    for (void *p : ptrs)
        if (p) cudaFree(p);
    delete m;
}

namespace {
int mlp_stage(jatam_mlp *m, size_t bytes) { return grow(&m->stage, &m->stage_bytes, bytes); }
}  // namespace

int jatam_mlp_set_params(jatam_mlp *m, const float *params, void *stream)
{
    std::lock_guard<std::mutex> lock(g_mutex);
    g_last_error.clear();
    if (!m || !params) return fail(JATAM_EINVAL, "net and params required");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const size_t bytes = (size_t)MLP_NPARAM * 4;
    CUDA_TRY(cudaMemcpyAsync(m->b.p, params, bytes, cudaMemcpyDefault, st));
    CUDA_TRY(cudaMemsetAsync(m->b.m, 0, bytes, st));
    CUDA_TRY(cudaMemsetAsync(m->b.v, 0, bytes, st));
    m->t = 0;
    CUDA_TRY(mlp_refresh_bf16(m->b, st));
    CUDA_TRY(cudaStreamSynchronize(st));
    return JATAM_OK;
}

int jatam_mlp_get_params(jatam_mlp *m, float *params, void *stream)
{
    std::lock_guard<std::mutex> lock(g_mutex);
    g_last_error.clear();
    if (!m || !params) return fail(JATAM_EINVAL, "net and params required");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    CUDA_TRY(cudaMemcpyAsync(params, m->b.p, (size_t)MLP_NPARAM * 4, cudaMemcpyDefault, st));
    CUDA_TRY(cudaStreamSynchronize(st));
    return JATAM_OK;
}

int jatam_mlp_train_step(jatam_mlp *m, const uint64_t *genomes, const uint8_t *labels, uint64_t B, float lr,
                         float *loss, float *grads, void *stream)
{
    std::lock_guard<std::mutex> lock(g_mutex);
    g_last_error.clear();
    if (!m || !genomes || !labels || B == 0 || (long long)B > m->b.cap)
        return fail(JATAM_EINVAL, "net, genomes, labels required and 1 <= B <= max_batch");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const Kind kg = kind_of(genomes, m->device), kl = kind_of(labels, m->device);
    const unsigned long long *dg = reinterpret_cast<const unsigned long long *>(genomes);
    const uint8_t *dl = labels;
    const size_t gb = ((size_t)B * 8 + 255) & ~size_t(255);
    if (kg == K_HOST || kl == K_HOST) {
        int rc = mlp_stage(m, gb + B + 256);
        if (rc) return rc;
        char *s8 = static_cast<char *>(m->stage);
        if (kg == K_HOST) {
            CUDA_TRY(cudaMemcpyAsync(s8, genomes, (size_t)B * 8, cudaMemcpyHostToDevice, st));
            dg = reinterpret_cast<const unsigned long long *>(s8);
        }
        if (kl == K_HOST) {
            CUDA_TRY(cudaMemcpyAsync(s8 + gb, labels, B, cudaMemcpyHostToDevice, st));
            dl = reinterpret_cast<const uint8_t *>(s8 + gb);
        }
    }
    CUDA_TRY(mlp_forward(m->b, dg, (long long)B, st));
    CUDA_TRY(mlp_backward(m->b, dl, (long long)B, st));
    if (grads) CUDA_TRY(cudaMemcpyAsync(grads, m->b.grad, (size_t)MLP_NPARAM * 4, cudaMemcpyDefault, st));
    float h_loss = 0.f;
    if (loss) CUDA_TRY(cudaMemcpyAsync(&h_loss, m->b.loss, 4, cudaMemcpyDeviceToHost, st));
    if (lr != 0.f) {
        m->t += 1;
        CUDA_TRY(mlp_adam(m->b, lr, m->t, st));
    }
    if (loss || (grads && kind_of(grads, m->device) == K_HOST) || kg == K_HOST || kl == K_HOST) {
        CUDA_TRY(cudaStreamSynchronize(st));
        if (loss) *loss = h_loss;
        return mlp_tc_status(m);
    }
    return JATAM_OK;
}

int jatam_mlp_predict(jatam_mlp *m, const uint64_t *genomes, uint64_t N, float *logits, void *stream)
{
    std::lock_guard<std::mutex> lock(g_mutex);
    g_last_error.clear();
    if (!m || !genomes || !logits || N == 0 || (long long)N > m->b.cap)
        return fail(JATAM_EINVAL, "net, genomes, logits required and 1 <= N <= max_batch");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const Kind kg = kind_of(genomes, m->device), ko = kind_of(logits, m->device);
    const unsigned long long *dg = reinterpret_cast<const unsigned long long *>(genomes);
    if (kg == K_HOST) {
        int rc = mlp_stage(m, (size_t)N * 8);
        if (rc) return rc;
        CUDA_TRY(cudaMemcpyAsync(m->stage, genomes, (size_t)N * 8, cudaMemcpyHostToDevice, st));
        dg = static_cast<const unsigned long long *>(m->stage);
    }
    CUDA_TRY(mlp_forward(m->b, dg, (long long)N, st, true));
    CUDA_TRY(cudaMemcpyAsync(logits, m->b.logits, (size_t)N * MLP_OUT * 4, cudaMemcpyDefault, st));
    if (kg == K_HOST || ko == K_HOST) {
        CUDA_TRY(cudaStreamSynchronize(st));
        return mlp_tc_status(m);
    }
    return JATAM_OK;
}

int jatam_mlp_labels(const jatam_result *results, uint64_t N, uint8_t *labels, void *stream)
{
    std::lock_guard<std::mutex> lock(g_mutex);
    g_last_error.clear();
    if (N && (!results || !labels)) return fail(JATAM_EINVAL, "results and labels required");
    int dev = 0;
    CUDA_TRY(cudaGetDevice(&dev));
    if (N && (kind_of(results, dev) != K_DEVICE || kind_of(labels, dev) != K_DEVICE))
        return fail(JATAM_EINVAL, "results and labels must be device memory");
    CUDA_TRY(launch_mlp_labels(results, (long long)N, labels, static_cast<cudaStream_t>(stream)));
    return JATAM_OK;
}

int jatam_select_top(const float *scores, uint64_t n, uint64_t keep, uint64_t *idx, void *stream)
{
    std::lock_guard<std::mutex> lock(g_mutex);
    g_last_error.clear();
    if (n && (!scores || (keep && !idx))) return fail(JATAM_EINVAL, "scores and idx required");
    if (n > (1ull << 26) || keep > n) return fail(JATAM_EINVAL, "n <= 2^26 and keep <= n required");
    int dev = 0;
    CUDA_TRY(cudaGetDevice(&dev));
    if (n && (kind_of(scores, dev) != K_DEVICE || (keep && kind_of(idx, dev) != K_DEVICE)))
        return fail(JATAM_EINVAL, "scores and idx must be device memory");
    if (!keep) return JATAM_OK;
    // the scratch of the selection lives in the device's workspace; like every call that uses the
    // workspace, this one is ordered after the previous such call on the device
    Workspace *w = nullptr;
    int rc = workspace(&w);
    if (rc) return rc;
    rc = grow(&w->topn_buf, &w->topn_bytes, TOPN_SCRATCH_BYTES);
    if (rc) return rc;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    CUDA_TRY(cudaStreamWaitEvent(st, w->last, 0));
    CUDA_TRY(launch_topn_multi(scores, (long long)n, (long long)keep, reinterpret_cast<unsigned long long *>(idx),
                               static_cast<unsigned *>(w->topn_buf), st));
    CUDA_TRY(cudaEventRecord(w->last, st));
    return JATAM_OK;
}

int jatam_embed_genomes(const uint64_t *genomes, uint64_t N, int n, int c, uint64_t *out, void *stream)
{
    std::lock_guard<std::mutex> lock(g_mutex);
    g_last_error.clear();
    if (N && (!genomes || !out)) return fail(JATAM_EINVAL, "genomes and out required");
    if (n < 1 || n > 3 || !(c == 2 || c == 4 || c == 8)) return fail(JATAM_EINVAL, "n 1..3 and c in {2, 4, 8}");
    int dev = 0;
    CUDA_TRY(cudaGetDevice(&dev));
    if (N && (kind_of(genomes, dev) != K_DEVICE || kind_of(out, dev) != K_DEVICE))
        return fail(JATAM_EINVAL, "genomes and out must be device memory");
    CUDA_TRY(launch_embed(reinterpret_cast<const unsigned long long *>(genomes), (long long)N, n, log2c(c),
                          reinterpret_cast<unsigned long long *>(out), static_cast<cudaStream_t>(stream)));
    return JATAM_OK;
}

int jatam_philox(const uint32_t *in, uint64_t N, uint32_t *out, void *stream)
{
    std::lock_guard<std::mutex> lock(g_mutex);
    g_last_error.clear();
    if (N && (!in || !out)) return fail(JATAM_EINVAL, "in/out is NULL");
    Workspace *w = nullptr;
    int rc = workspace(&w);
    if (rc) return rc;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    CUDA_TRY(cudaStreamWaitEvent(st, w->last, 0));
    const void *din = nullptr;
    rc = stage_input(w, in, (size_t)N * 24, &w->stage_in, &w->stage_in_bytes, &din, st);
    if (rc) return rc;
    const Kind ko = kind_of(out, w->device);
    if (ko == K_NULL && out) return fail(JATAM_EINVAL, "out lives on another device");
    uint32_t *dout = out;
    if (ko == K_HOST) {
        rc = grow(&w->stage_aux, &w->stage_aux_bytes, (size_t)N * 16);
        if (rc) return rc;
        dout = static_cast<uint32_t *>(w->stage_aux);
    }
    CUDA_TRY(launch_philox(static_cast<const uint32_t *>(din), N, dout, st));
    if (ko == K_HOST && N) CUDA_TRY(cudaMemcpyAsync(out, dout, (size_t)N * 16, cudaMemcpyDeviceToHost, st));
    CUDA_TRY(cudaEventRecord(w->last, st));
    if (ko == K_HOST || kind_of(in, w->device) == K_HOST) CUDA_TRY(cudaStreamSynchronize(st));
    return JATAM_OK;
}

int jatam_hist_merge(const jatam_hist_entry *a, uint32_t na, const jatam_hist_entry *b, uint32_t nb,
                     jatam_hist_entry *out, uint32_t cap, uint32_t *len)
{
    g_last_error.clear();
    if ((na && !a) || (nb && !b) || !len || (cap && !out)) return fail(JATAM_EINVAL, "NULL argument");
    uint32_t i = 0, j = 0, m = 0;
    auto key = [](const jatam_hist_entry &e) { return ((uint64_t)e.cls << 32) | e.shape_hash; };
    while (i < na || j < nb) {
        jatam_hist_entry e;
        if (j >= nb || (i < na && key(a[i]) < key(b[j]))) {
            e = a[i++];
        } else if (i >= na || key(b[j]) < key(a[i])) {
            e = b[j++];
        } else {
            e = a[i];
            const jatam_hist_entry &f = b[j];
            e.count += f.count;
            e.min_id = e.min_id < f.min_id ? e.min_id : f.min_id;
            e.flags |= f.flags | (e.size != f.size ? 1u : 0u);
            e.size = e.size > f.size ? e.size : f.size;
            ++i;
            ++j;
        }
        if (m < cap) out[m] = e;
        ++m;
    }
    *len = m;
    if (m > cap) return fail(JATAM_EINVAL, "merged histogram has %u keys but cap is %u", m, cap);
    return JATAM_OK;
}

int jatam_autotune(const jatam_config *shapes, uint32_t n_shapes, void *stream)
{
    std::lock_guard<std::mutex> lock(g_mutex);
    g_last_error.clear();
    if (n_shapes && !shapes) return fail(JATAM_EINVAL, "shapes is NULL");
    Workspace *w = nullptr;
    int rc = workspace(&w);
    if (rc) return rc;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    for (uint32_t i = 0; i < n_shapes; ++i) {
        const jatam_config &cfg = shapes[i];
        rc = check_params(cfg.n, cfg.c, cfg.L, cfg.k, true);
        if (rc) return rc;
        const int S = lattice_template(cfg.L);
        const int bits = 4 * cfg.n * log2c(cfg.c);
        const bool sampled = (cfg.flags & JATAM_SAMPLED) != 0;
        unsigned long long count = 1ull << 18;
        if (!sampled && bits < 18) count = 1ull << bits;
        LaunchArgs a{};
        a.mode = sampled ? MODE_SAMPLED : MODE_RANGE;
        a.first = 0;
        a.count = count;
        a.n = cfg.n; a.c = cfg.c; a.L = cfg.L; a.k = cfg.k;
        a.key0 = (uint32_t)cfg.seed;
        a.key1 = (uint32_t)(cfg.seed >> 32);
        Tuning best;
        float best_ms = 1e30f;
        for (int warps : {2, 3, 4, 5, 6}) {
            const int bytes = classify_smem_bytes(S, tuple_table_size(cfg.n), warps);
            if (bytes > 200 * 1024) continue;
            for (int stop : {4, 8, 12, 16, 20, 24, 28}) {
                Tuning t;
                t.warps = warps;
                t.stop_at = stop;
                float ms_min = 1e30f;
                for (int rep = 0; rep < 2; ++rep) {
                    float ms = 0.f;
                    rc = run(w, a, S, nullptr, nullptr, nullptr, 0, nullptr, true, st, &t, &ms);
                    if (rc) return rc;
                    ms_min = ms < ms_min ? ms : ms_min;
                }
                if (ms_min < best_ms) {
                    best_ms = ms_min;
                    best = t;
                }
            }
        }
        if (S == 32) {
            // one genotype per warp: a single launch shape
            Tuning t;
            t.per_warp = 1;
            float ms_min = 1e30f;
            for (int rep = 0; rep < 2; ++rep) {
                float ms = 0.f;
                rc = run(w, a, S, nullptr, nullptr, nullptr, 0, nullptr, true, st, &t, &ms);
                if (rc) return rc;
                ms_min = ms < ms_min ? ms : ms_min;
            }
            if (ms_min < best_ms) {
                best_ms = ms_min;
                best = t;
            }
            if (best.per_warp == 0) best.per_warp = 32;
        }
        g_tuned[std::make_tuple(S, (int)cfg.n, (int)cfg.c)] = best;
    }
    return JATAM_OK;
}

int jatam_set_replicate_lanes(int mode)
{
    std::lock_guard<std::mutex> lock(g_mutex);
    g_last_error.clear();
    read_env_overrides();
    if (mode < 0 || mode > 2) return fail(JATAM_EINVAL, "mode must be 0 (by call size), 1 (never) or 2 (whenever eligible)");
    g_reps_mode = mode;
    return JATAM_OK;
}

int jatam_get_replicate_lanes(void)
{
    std::lock_guard<std::mutex> lock(g_mutex);
    read_env_overrides();
    return g_reps_mode;
}

int jatam_set_genotypes_per_warp(const jatam_config *cfg, int genotypes_per_warp)
{
    std::lock_guard<std::mutex> lock(g_mutex);
    g_last_error.clear();
    if (!cfg) return fail(JATAM_EINVAL, "cfg is NULL");
    if (cfg->L < 1 || cfg->L > JATAM_MAX_GRID) return fail(JATAM_EUNSUPPORTED, "L must be 1..32");
    if (!(genotypes_per_warp == 0 || genotypes_per_warp == 1 || genotypes_per_warp == 32))
        return fail(JATAM_EINVAL, "genotypes_per_warp must be 0, 1 or 32");
    const int S = lattice_template(cfg->L);
    if (genotypes_per_warp == 1 && S != 32)
        return fail(JATAM_EINVAL, "one genotype per warp is built for lattices of 17 x 17 to 32 x 32");
    g_tuned[std::make_tuple(S, (int)cfg->n, (int)cfg->c)].per_warp = genotypes_per_warp;
    return JATAM_OK;
}

int jatam_get_genotypes_per_warp(const jatam_config *cfg, int *genotypes_per_warp)
{
    std::lock_guard<std::mutex> lock(g_mutex);
    g_last_error.clear();
    if (!cfg || !genotypes_per_warp) return fail(JATAM_EINVAL, "cfg and genotypes_per_warp are required");
    if (cfg->L < 1 || cfg->L > JATAM_MAX_GRID) return fail(JATAM_EUNSUPPORTED, "L must be 1..32");
    const int S = lattice_template(cfg->L);
    *genotypes_per_warp = tuning_for(S, cfg->n, cfg->c).per_warp;
    return JATAM_OK;
}

int jatam_set_tuning(const jatam_config *cfg, int warps_per_cta, int stop_at)
{
    std::lock_guard<std::mutex> lock(g_mutex);
    g_last_error.clear();
    if (!cfg) return fail(JATAM_EINVAL, "cfg is NULL");
    if (cfg->L < 1 || cfg->L > JATAM_MAX_GRID) return fail(JATAM_EUNSUPPORTED, "L must be 1..32");
    const int S = lattice_template(cfg->L);
    if (warps_per_cta == 0) {
        g_tuned.erase(std::make_tuple(S, (int)cfg->n, (int)cfg->c));
        return JATAM_OK;
    }
    if (warps_per_cta < 1 || warps_per_cta > MAX_CTA_WARPS || stop_at < 1 || stop_at > 32)
        return fail(JATAM_EINVAL, "warps_per_cta must be 0..%d and stop_at 1..32", MAX_CTA_WARPS);
    if (classify_smem_bytes(S, tuple_table_size(cfg->n), warps_per_cta) > 200 * 1024)
        return fail(JATAM_EINVAL, "%d warps of a %dx%d lattice do not fit in shared memory", warps_per_cta, S, S);
    Tuning &t = g_tuned[std::make_tuple(S, (int)cfg->n, (int)cfg->c)];  // keeps the layout setting
    t.warps = warps_per_cta;
    t.stop_at = stop_at;
    return JATAM_OK;
}

int jatam_get_tuning(const jatam_config *cfg, int *warps_per_cta, int *stop_at)
{
    std::lock_guard<std::mutex> lock(g_mutex);
    g_last_error.clear();
    if (!cfg || !warps_per_cta || !stop_at) return fail(JATAM_EINVAL, "NULL argument");
    const Tuning t = tuning_for(lattice_template(cfg->L), cfg->n, cfg->c);
    *warps_per_cta = t.warps;
    *stop_at = t.stop_at;
    return JATAM_OK;
}

int jatam_set_mixed_plan(int warps_32, int warps_16, int warps_8)
{
    std::lock_guard<std::mutex> lock(g_mutex);
    g_last_error.clear();
    if (!plan_fits(warps_32, warps_16, warps_8))
        return fail(JATAM_EINVAL, "plan %d/%d/%d: at least one 32 x 32 warp, at most 8 warps, regions that fit "
                                  "in shared memory", warps_32, warps_16, warps_8);
    g_plan[0] = warps_32;
    g_plan[1] = warps_16;
    g_plan[2] = warps_8;
    return JATAM_OK;
}

int jatam_get_mixed_plan(int *warps_32, int *warps_16, int *warps_8)
{
    std::lock_guard<std::mutex> lock(g_mutex);
    g_last_error.clear();
    if (!warps_32 || !warps_16 || !warps_8) return fail(JATAM_EINVAL, "NULL argument");
    *warps_32 = g_plan[0];
    *warps_16 = g_plan[1];
    *warps_8 = g_plan[2];
    return JATAM_OK;
}

int jatam_get_mixed_launch(int *per_shape)
{
    std::lock_guard<std::mutex> lock(g_mutex);
    g_last_error.clear();
    if (!per_shape) return fail(JATAM_EINVAL, "per_shape is NULL");
    *per_shape = g_mixed_per_shape ? 1 : 0;
    return JATAM_OK;
}

int jatam_autotune_batch(const uint8_t *colours, const uint8_t *shapes, uint64_t N, uint64_t seed, void *stream)
{
    std::lock_guard<std::mutex> lock(g_mutex);
    g_last_error.clear();
    if (!colours || !shapes || N == 0) return fail(JATAM_EINVAL, "colours, shapes and N > 0 are required");
    Workspace *w = nullptr;
    int rc = workspace(&w);
    if (rc) return rc;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    CUDA_TRY(cudaStreamWaitEvent(st, w->last, 0));
    // the batch as device memory in stage_in: colours, then shapes
    const Kind kc = kind_of(colours, w->device), ks = kind_of(shapes, w->device);
    const size_t cb = (size_t)N * 16, off_s = (cb + 255) & ~size_t(255);
    const uint8_t *dc = colours, *ds = shapes;
    if (kc == K_HOST || ks == K_HOST) {
        rc = grow(&w->stage_in, &w->stage_in_bytes, off_s + (size_t)N * 4 + 256);
        if (rc) return rc;
        char *base = static_cast<char *>(w->stage_in);
        if (kc == K_HOST) {
            CUDA_TRY(cudaMemcpyAsync(base, colours, cb, cudaMemcpyHostToDevice, st));
            dc = reinterpret_cast<const uint8_t *>(base);
        }
        if (ks == K_HOST) {
            CUDA_TRY(cudaMemcpyAsync(base + off_s, shapes, (size_t)N * 4, cudaMemcpyHostToDevice, st));
            ds = reinterpret_cast<const uint8_t *>(base + off_s);
        }
    }
    LaunchArgs a{};
    a.mode = MODE_RECORDS;
    a.count = N;
    a.colours = dc;
    a.shapes = ds;
    a.key0 = (uint32_t)seed;
    a.key1 = (uint32_t)(seed >> 32);
    static const int plans[][3] = {{1, 2, 1}, {2, 4, 2}, {1, 3, 2}, {2, 2, 2}, {1, 4, 3}, {2, 3, 3},
                                   {3, 3, 2}, {1, 5, 2}, {2, 5, 1}, {1, 6, 1}, {4, 2, 2}, {2, 6, 0}};
    int best[3] = {g_plan[0], g_plan[1], g_plan[2]};
    float best_ms = 1e30f;
    for (const auto &p : plans) {
        if (!plan_fits(p[0], p[1], p[2])) continue;
        for (int stop : {4, 8, 16}) {
            Tuning t;
            t.stop_at = stop;
            t.w32 = p[0];
            t.w16 = p[1];
            t.w8 = p[2];
            float ms = 0.f;
            rc = run(w, a, 32, nullptr, nullptr, nullptr, 0, nullptr, true, st, &t, &ms);
            if (rc) return rc;
            if (ms < best_ms) {
                best_ms = ms;
                best[0] = p[0];
                best[1] = p[1];
                best[2] = p[2];
                g_tuned[std::make_tuple(32, 0, 0)] = t;
            }
        }
    }
    g_plan[0] = best[0];
    g_plan[1] = best[1];
    g_plan[2] = best[2];
    // the per-size fixed launches on the same batch
    float fixed_ms = 1e30f;
    for (int rep = 0; rep < 2; ++rep) {
        float ms = 0.f;
        rc = run(w, a, 32, nullptr, nullptr, nullptr, 0, nullptr, true, st, nullptr, &ms, true);
        if (rc) return rc;
        fixed_ms = ms < fixed_ms ? ms : fixed_ms;
    }
    g_mixed_per_shape = fixed_ms < best_ms;
    return JATAM_OK;
}

int jatam_profile(int enable)
{
    std::lock_guard<std::mutex> lock(g_mutex);
    g_last_error.clear();
    if (enable < 0 || enable > 3) return fail(JATAM_EINVAL, "enable must be 0..3");
    g_profile = enable;
    return JATAM_OK;
}

int jatam_work_counters(uint64_t counters[4])
{
    std::lock_guard<std::mutex> lock(g_mutex);
    g_last_error.clear();
    if (!counters) return fail(JATAM_EINVAL, "counters is NULL");
    int dev = 0;
    CUDA_TRY(cudaGetDevice(&dev));
    auto it = g_ws.find(dev);
    if (it == g_ws.end() || !it->second->stats_valid) return fail(JATAM_EINVAL, "no counted call on this device");
    CUDA_TRY(cudaEventSynchronize(it->second->last));
    CUDA_TRY(cudaMemcpy(counters, it->second->stats, 4 * 8, cudaMemcpyDeviceToHost));
    return JATAM_OK;
}

int jatam_kernel_ms(float *ms)
{
    std::lock_guard<std::mutex> lock(g_mutex);
    g_last_error.clear();
    if (!ms) return fail(JATAM_EINVAL, "ms is NULL");
    int dev = 0;
    CUDA_TRY(cudaGetDevice(&dev));
    auto it = g_ws.find(dev);
    if (it == g_ws.end() || !it->second->k_valid) return fail(JATAM_EINVAL, "no profiled call on this device");
    CUDA_TRY(cudaEventSynchronize(it->second->k_stop));
    CUDA_TRY(cudaEventElapsedTime(ms, it->second->k_start, it->second->k_stop));
    return JATAM_OK;
}

void jatam_shutdown(void)
{
    std::lock_guard<std::mutex> lock(g_mutex);
    int cur = 0;
    cudaGetDevice(&cur);
    for (auto &kv : g_ws) {
        Workspace *w = kv.second;
        cudaSetDevice(w->device);
        cudaDeviceSynchronize();
        cudaFree(w->table.key); cudaFree(w->table.count); cudaFree(w->table.min_id);
        cudaFree(w->table.size_max); cudaFree(w->table.size_min);
        cudaFree(w->compact.key); cudaFree(w->compact.count); cudaFree(w->compact.min_id);
        cudaFree(w->compact.size_max); cudaFree(w->compact.size_min);
        cudaFree(w->work_next); cudaFree(w->crops); cudaFree(w->stats); cudaFree(w->err); cudaFree(w->nkeys); cudaFree(w->list_count);
        cudaFree(w->shapes.key); cudaFree(w->shapes.stats); cudaFree(w->esc_ctl);
        if (w->esc) cudaFree(w->esc);
        if (w->alt.esc) cudaFree(w->alt.esc);
        if (w->alt.esc_ctl) cudaFree(w->alt.esc_ctl);
        if (w->spill_rows) cudaFree(w->spill_rows);
        if (w->alt.spill_rows) cudaFree(w->alt.spill_rows);
        if (w->list) cudaFree(w->list);
        cudaFreeHost(w->host_words);
        if (w->stage_in) cudaFree(w->stage_in);
        if (w->stage_out) cudaFree(w->stage_out);
        if (w->stage_aux) cudaFree(w->stage_aux);
        if (w->stage_hist) cudaFree(w->stage_hist);
        if (w->ga_buf) cudaFree(w->ga_buf);
        if (w->screen_buf) cudaFree(w->screen_buf);
        if (w->topn_buf) cudaFree(w->topn_buf);
        if (w->dedup_buf) cudaFree(w->dedup_buf);
        if (w->lifo_buf) cudaFree(w->lifo_buf);
        cudaEventDestroy(w->last);
        cudaEventDestroy(w->k_start);
        cudaEventDestroy(w->k_stop);
        for (auto &kv : w->graphs) cudaGraphExecDestroy(kv.second);
        if (w->capture) cudaStreamDestroy(w->capture);
        if (w->h2d) {
            cudaStreamDestroy(w->h2d);
            for (int c = 0; c < PIPE_MAX_CHUNKS; ++c) cudaEventDestroy(w->in_ev[c]);
        }
        if (w->copy) {
            cudaStreamDestroy(w->copy);
            cudaStreamDestroy(w->aux);
            for (int c = 0; c < PIPE_MAX_CHUNKS; ++c) {
                cudaEventDestroy(w->pipe_ev[c]);
                cudaEventDestroy(w->pf_ev[c]);
            }
            cudaEventDestroy(w->pipe_start);
            cudaEventDestroy(w->aux_done);
            cudaEventDestroy(w->pipe_done);
            cudaFree(w->alt.work_next);
            cudaFree(w->alt.list_count);
            cudaFree(w->alt.nkeys);
            cudaFree(w->alt.crops);
        }
        if (w->alt.list) cudaFree(w->alt.list);
        delete w;
    }
    g_ws.clear();
    cudaSetDevice(cur);
    noalloc_forget_devices();
}

int jatam_last_shapes(jatam_shape *shapes, uint32_t cap, uint32_t *len, uint32_t *collisions)
{
    std::lock_guard<std::mutex> lock(g_mutex);
    if (!len || !collisions) return fail(JATAM_EINVAL, "len and collisions are required");
    if (cap && !shapes) return fail(JATAM_EINVAL, "shapes is NULL");
    int dev = 0;
    CUDA_TRY(cudaGetDevice(&dev));
    auto it = g_ws.find(dev);
    if (it == g_ws.end() || !it->second->shapes_valid)
        return fail(JATAM_EINVAL, "the last call on this device built no histogram with the canonical-form hash");
    Workspace *w = it->second;
    CUDA_TRY(cudaEventSynchronize(w->last));
    const size_t nslot = size_t(1) << SHAPES_LOG2;
    std::vector<unsigned long long> keys(nslot);
    std::vector<unsigned> meta(nslot);
    std::vector<uint32_t> rows(nslot * 32);
    unsigned st[4] = {0, 0, 0, 0};
    CUDA_TRY(cudaMemcpy(keys.data(), w->shapes.key, nslot * 8, cudaMemcpyDeviceToHost));
    CUDA_TRY(cudaMemcpy(meta.data(), w->shapes.meta, nslot * 4, cudaMemcpyDeviceToHost));
    CUDA_TRY(cudaMemcpy(rows.data(), w->shapes.rows, nslot * 128, cudaMemcpyDeviceToHost));
    CUDA_TRY(cudaMemcpy(st, w->shapes.stats, 16, cudaMemcpyDeviceToHost));
    std::vector<jatam_shape> all;
    for (size_t i = 0; i < nslot; ++i) {
        if (!keys[i]) continue;
        jatam_shape e{};
        e.shape_hash = (uint32_t)keys[i];
        const unsigned m = meta[i];
        e.h = (uint8_t)((m >> 8) & 0xFF);
        e.w = (uint8_t)(m & 0xFF);
        unsigned size = 0;
        for (int r = 0; r < 32; ++r) {
            // stored with the first cell in bit w - 1; returned with column j in bit j
            const uint32_t v = rows[i * 32 + r];
            uint32_t out = 0;
            for (int j = 0; j < e.w; ++j)
                if ((v >> (e.w - 1 - j)) & 1u) out |= 1u << j;
            e.rows[r] = r < e.h ? out : 0u;
            size += (unsigned)__builtin_popcount(e.rows[r]);
        }
        e.size = (uint16_t)size;
        all.push_back(e);
    }
    std::sort(all.begin(), all.end(), [](const jatam_shape &x, const jatam_shape &y) { return x.shape_hash < y.shape_hash; });
    *len = (uint32_t)all.size();
    *collisions = st[0];
    for (size_t i = 0; i < all.size() && i < cap; ++i) shapes[i] = all[i];
    if (st[1]) return fail(JATAM_ETIMEOUT, "%u shape comparisons gave up waiting for the stored rows", st[1]);
    if (st[2]) return fail(JATAM_ENOMEM, "the shape side table (%zu slots) overflowed %u times", nslot, st[2]);
    if (all.size() > cap) return fail(JATAM_EINVAL, "%zu shapes but cap is %u", all.size(), cap);
    return JATAM_OK;
}

int jatam_workspace_bytes(uint64_t *bytes)
{
    std::lock_guard<std::mutex> lock(g_mutex);
    if (!bytes) return fail(JATAM_EINVAL, "bytes is NULL");
    int dev = 0;
    CUDA_TRY(cudaGetDevice(&dev));
    auto it = g_ws.find(dev);
    if (it == g_ws.end()) {
        *bytes = 0;
        return JATAM_OK;
    }
    const Workspace *w = it->second;
    const size_t cap = size_t(1) << TABLE_LOG2;
    size_t b = 2 * cap * (8 + 8 + 8 + 4 + 4);                  // phenotype table and its compacted copy
    b += 3 * 8 + (size_t(2) << CROPS_LOG2) * 8 + 4 * 8 + 4 + 4 + 6 * 8;  // counters, crop table
    b += ((size_t(8) + 4 + 128) << SHAPES_LOG2) + 4 * 4;                 // shape side table
    b += w->list_bytes + w->stage_in_bytes + w->stage_out_bytes + w->stage_aux_bytes +
         w->stage_hist_cap * sizeof(jatam_hist_entry) + w->lifo_bytes + w->ga_bytes + w->screen_bytes + w->topn_bytes + w->dedup_bytes +
         w->alt.list_bytes + w->esc_bytes + w->alt.esc_bytes + ESC_CTL_WORDS * 8 + w->spill_bytes +
         w->alt.spill_bytes;
    if (w->copy) b += 3 * 8 + 6 * 8 + 4 + (size_t(2) << CROPS_LOG2) * 8;
    *bytes = b;
    return JATAM_OK;
}

const char *jatam_last_error(void) { return g_last_error.c_str(); }

}  // extern "C"
