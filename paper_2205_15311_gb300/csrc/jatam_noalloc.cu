// jatam_noalloc.cu -- jatam_enumerate_noalloc: classification of an index
// range without any device allocation by the library.
//
// Who needs this: code that runs where cudaMalloc is not an option -- for
// example a host callback or a library that must not touch the CUDA allocator
// because the application owns all device memory through its own pool, or
// code that must not trigger the implicit device synchronisation cudaFree
// performs.  jatam_enumerate allocates a per-device workspace on first use and
// grows it for larger calls; this entry point instead keeps its scratch in
// one fixed array in device memory that is part of the loaded library.
//
// The scratch array below (NOALLOC_BYTES) is reserved on every GPU where the
// library's module is loaded, for as long as the process lives.  It holds
// three counters and the list of genotypes left to grow after the seed-step
// pre-filter, so a call may classify at most JATAM_NOALLOC_MAX_COUNT
// genotypes.  Every call reuses the same array: two calls that overlap on the
// GPU (different streams, no ordering between them) race on it and give
// wrong results.
#include <cstdint>
#include <mutex>

#include <cuda_runtime.h>

#include "jatam_internal.cuh"

using namespace jatam;

namespace {

constexpr size_t NOALLOC_HEADER = 256;  // work counter, list length, error word
constexpr size_t NOALLOC_BYTES = NOALLOC_HEADER + (size_t)JATAM_NOALLOC_MAX_COUNT * 8;

// The scratch itself.  Host code must not use this name as an address: on the
// host it is only a stand-in, so the device address is looked up once per
// device with cudaGetSymbolAddress.
static __device__ __align__(256) unsigned char g_noalloc_scratch[NOALLOC_BYTES];

constexpr int MAX_DEVICES = 64;
struct DeviceState {
    bool ready = false;
    unsigned char *scratch = nullptr;  // device address of g_noalloc_scratch on this device
    int num_sms = 0;
    int warps[3][2] = {};   // [lattice template 8, 16, 32][tuple table 8, 16]: warps per CTA
    int per_sm[3][2] = {};  // resident CTAs of that launch shape per SM
};
DeviceState g_dev[MAX_DEVICES];
std::mutex g_noalloc_mutex;

int noalloc_fail(int code, const char *msg)
{
    jatam::set_last_error(msg);  // read back with jatam_last_error()
    return code;
}

int lattice_template_of(int L) { return L <= 8 ? 8 : L <= 16 ? 16 : 32; }
int template_slot(int S) { return S == 8 ? 0 : S == 16 ? 1 : 2; }
int colour_bits(int c) { return c >= 8 ? 3 : c >= 4 ? 2 : c >= 2 ? 1 : 0; }

// Set-up of device `dev` (the calling thread's current device), once: the
// scratch array's device address, the SM count, and for every lattice template
// and tuple-table size the launch limits and occupancy of the classification
// kernel -- so that every kernel a later call launches is already loaded and
// configured, whatever its L and n.
int device_setup(int dev, DeviceState **out)
{
    if (dev < 0 || dev >= MAX_DEVICES) return noalloc_fail(JATAM_EUNSUPPORTED, "device ordinal out of range");
    DeviceState &d = g_dev[dev];
    if (!d.ready) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || p == nullptr) {
            cudaGetLastError();
            return noalloc_fail(JATAM_ECUDA, "cudaGetSymbolAddress of the scratch array failed");
        }
        if (cudaDeviceGetAttribute(&d.num_sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
            return noalloc_fail(JATAM_ECUDA, "cudaDeviceGetAttribute failed");
        if (load_index_range_kernels() != cudaSuccess) {
            cudaGetLastError();
            return noalloc_fail(JATAM_ECUDA, "loading the pre-filter kernel failed");
        }
        const int Ss[3] = {8, 16, 32}, nts[2] = {8, 16};
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 2; ++j) {
                const int w = default_warps_per_cta(Ss[i], nts[j]);
                int per_sm = 0;
                if (classify_set_attributes(Ss[i], nts[j], w) != cudaSuccess ||
                    classify_occupancy(Ss[i], nts[j], w, &per_sm) != cudaSuccess || per_sm < 1) {
                    cudaGetLastError();
                    return noalloc_fail(JATAM_ECUDA, "classification kernel does not fit on an SM");
                }
                d.warps[i][j] = w;
                d.per_sm[i][j] = per_sm;
            }
        d.scratch = static_cast<unsigned char *>(p);
        d.ready = true;
    }
    *out = &d;
    return JATAM_OK;
}

}  // namespace

// jatam_shutdown: the next call on each device looks everything up again (a
// cudaDeviceReset reloads the module, and the array may then sit elsewhere)
void jatam::noalloc_forget_devices()
{
    std::lock_guard<std::mutex> lock(g_noalloc_mutex);
    for (auto &d : g_dev) d = DeviceState{};
}

extern "C" int jatam_enumerate_noalloc(const jatam_config *cfg, uint64_t first, uint64_t count, jatam_result *out,
                                       void *stream)
{
    std::lock_guard<std::mutex> lock(g_noalloc_mutex);
    jatam::set_last_error("");
    if (!cfg || !out) return noalloc_fail(JATAM_EINVAL, "cfg and out are required");
    const int n = cfg->n, c = cfg->c, L = cfg->L, k = cfg->k;
    if (n < 1 || n > JATAM_MAX_TILES || L < 1 || L > JATAM_MAX_GRID || k < 1 || k > JATAM_MAX_REPLICATES ||
        !(c == 1 || c == 2 || c == 4 || c == 8))
        return noalloc_fail(JATAM_EUNSUPPORTED, "n 1..4, c in {1, 2, 4, 8}, L 1..32, k 1..255");
    if (count > JATAM_NOALLOC_MAX_COUNT)
        return noalloc_fail(JATAM_EINVAL, "count exceeds JATAM_NOALLOC_MAX_COUNT (the fixed scratch holds "
                                          "1,048,576 genotypes per call)");
    const bool sampled = (cfg->flags & JATAM_SAMPLED) != 0;
    if (cfg->flags & (JATAM_ORBITS | JATAM_LIFO))
        return noalloc_fail(JATAM_EINVAL, "JATAM_ORBITS and JATAM_LIFO need jatam_enumerate");
    const int bits = 4 * n * colour_bits(c);
    if (!sampled) {
        const uint64_t space = bits >= 64 ? ~0ull : (1ull << bits);
        if (first > space || count > space - first) return noalloc_fail(JATAM_EINVAL, "index range exceeds the space");
    }
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return noalloc_fail(JATAM_ECUDA, "cudaGetDevice failed");
    // out must be memory the current device owns (or managed memory): another
    // GPU's buffer would be written through a peer pointer
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, out) != cudaSuccess ||
        !((at.type == cudaMemoryTypeDevice && at.device == dev) || at.type == cudaMemoryTypeManaged)) {
        cudaGetLastError();
        return noalloc_fail(JATAM_EINVAL, "out must be device memory of the current device");
    }
    DeviceState *d = nullptr;
    int rc = device_setup(dev, &d);
    if (rc) return rc;
    cudaStream_t st = static_cast<cudaStream_t>(stream);

    unsigned char *base = d->scratch;
    unsigned long long *work_next = reinterpret_cast<unsigned long long *>(base);        // [3]
    unsigned long long *list_count = reinterpret_cast<unsigned long long *>(base + 128);  // [6]
    unsigned *err = reinterpret_cast<unsigned *>(base + 64);
    unsigned *nkeys = reinterpret_cast<unsigned *>(base + 68);
    unsigned long long *list = reinterpret_cast<unsigned long long *>(base + NOALLOC_HEADER);

    LaunchArgs a{};
    a.mode = sampled ? MODE_SAMPLED : MODE_RANGE;
    a.first = first;
    a.count = count;
    a.n = n; a.c = c; a.L = L; a.k = k;
    a.c4 = (cfg->flags & JATAM_C4_HASH) ? 1 : 0;
    a.key0 = (uint32_t)cfg->seed;
    a.key1 = (uint32_t)(cfg->seed >> 32);
    a.out = out;
    a.fitness = nullptr;
    a.use_hist = 0;
    a.list = list;
    a.list_stride = count;
    a.list_count = list_count;
    a.bucket = 0;
    a.klass = 0;
    a.work_next = work_next;
    a.err = err;

    const int S = lattice_template_of(L);
    a.stop_at = default_stop_at(S);
    const int nt = tuple_table_size(cfg->n);
    const int warps = d->warps[template_slot(S)][nt == 8 ? 0 : 1];
    const int per_sm = d->per_sm[template_slot(S)][nt == 8 ? 0 : 1];
    long long blocks = (long long)per_sm * d->num_sms;
    const long long needed = (long long)((count + 32ull * warps - 1) / (32ull * warps));
    if (needed < blocks) blocks = needed < 1 ? 1 : needed;
    // heavy genotypes first when every lane takes at least 8 genotypes on average
    a.heavy_first = (count >= 8ull * (unsigned long long)blocks * warps * 32) ? 1 : 0;

    // the counters and the error word start at zero in every call
    if (launch_reset(work_next, nkeys, list_count, st) != cudaSuccess) return noalloc_fail(JATAM_ECUDA, "launch failed");
    if (cudaMemsetAsync(err, 0, 4, st) != cudaSuccess) return noalloc_fail(JATAM_ECUDA, "cudaMemsetAsync failed");
    if (count) {
        long long pblocks = (long long)((count + 255) / 256);
        if (pblocks > PF_CTAS_PER_SM * d->num_sms) pblocks = PF_CTAS_PER_SM * d->num_sms;
        if (launch_prefilter(a, S, (int)pblocks, st) != cudaSuccess) return noalloc_fail(JATAM_ECUDA, "launch failed");
        if (launch_classify(a, S, nt, (int)blocks, warps, st) != cudaSuccess)
            return noalloc_fail(JATAM_ECUDA, "launch failed");
    }
    if (cfg->flags & JATAM_SYNC) {
        unsigned h_err = 0;
        if (cudaMemcpyAsync(&h_err, err, 4, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
            cudaStreamSynchronize(st) != cudaSuccess)
            return noalloc_fail(JATAM_ECUDA, "synchronisation failed");
        if (h_err) return noalloc_fail(JATAM_ETIMEOUT, "a bounded device loop found an inconsistent state");
    }
    return JATAM_OK;
}
