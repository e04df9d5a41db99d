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
    int stop_at;                    // finished lanes that end a growth round (1..32)
    unsigned long long *list;        // items left to grow, written by the pre-filter
    unsigned long long *list_count;  // their number
    unsigned long long *work_next;  // work counter, zeroed before the launch
    unsigned *err;                  // sticky error bits
};

// Lattice template: rows of S bits, S in {8, 16, 32}, L <= S.
int classify_smem_bytes(int S, int warps_per_cta);
cudaError_t classify_set_attributes(int S, int warps_per_cta);
cudaError_t classify_occupancy(int S, int warps_per_cta, int *blocks_per_sm);
cudaError_t launch_classify(const LaunchArgs &a, int S, int blocks, int warps_per_cta, cudaStream_t st);

cudaError_t launch_reset(unsigned long long *work_next, unsigned *nkeys, unsigned long long *list_count,
                         cudaStream_t st);
cudaError_t launch_prefilter(const LaunchArgs &a, int smax, int blocks, cudaStream_t st);
cudaError_t launch_table_init(Table t, cudaStream_t st);
cudaError_t launch_hist_compact(Table t, Compact c, unsigned *nkeys, int blocks, cudaStream_t st);
cudaError_t launch_hist_emit(Compact c, const unsigned *nkeys, jatam_hist_entry *hist, unsigned cap,
                             uint32_t *hist_len, int blocks, cudaStream_t st);
cudaError_t launch_philox(const uint32_t *in, unsigned long long n, uint32_t *out, cudaStream_t st);

// the message returned by jatam_last_error() for the calling thread
void set_last_error(const char *msg);

}  // namespace jatam
