// Internal declarations of the search library (not part of the C ABI).
#pragma once

#include <cstdint>
#include <string>
#include <vector>

#include "hicops.h"

namespace hicops {

// Physical constants (monoisotopic, Da).
constexpr double kWaterDa = 18.010565;
constexpr double kProtonDa = 1.007276466812;

// Largest peptide length supported: modification state is a 64-bit mask.
constexpr uint32_t kMaxLen = 64;
constexpr uint32_t kHistBins = 256;
constexpr uint32_t kMaxTopK = 32;
constexpr uint32_t kMaxTopN = 1024;   // query bins per spectrum (after the tolerance widening)

// The search walks peptide ids in chunks of 2^kChunkShift; every bucket
// stores where each chunk starts (the skip table).
constexpr uint32_t kChunkShift = 14;
constexpr uint32_t kChunk = 1u << kChunkShift;
// A bucket holding at least P >> kHotShift entries (1/64 of the database)
// is also stored as a pid bitmap.
constexpr uint32_t kHotShift = 6;

// Counter packing for one (spectrum, peptide) pair, 32 bits:
//   bits 26..31 nb, bits 20..25 ny, bits 0..19 S (sum of quantised intensity).
constexpr uint32_t kNbShift = 26;
constexpr uint32_t kNyShift = 20;
constexpr uint32_t kSMask = (1u << 20) - 1;

// Query bins per spectrum: every retained peak widened to 2 t + 1 bins.
inline uint32_t query_bins_cap(const hicops_params& p) { return (2 * p.tol_bins + 1) * p.top_n_peaks; }

// Thread-local error message (host.cpp).
void set_error(const char* fmt, ...);

// Host peptide table plus the device index.
struct DeviceIndex {
    bool ready = false;
    int device = -1;
    double* mass = nullptr;        // [P] neutral mass, pid order
    uint64_t* off = nullptr;       // [n_bins + 1] bucket offsets (multiples of 4)
    uint32_t* entry = nullptr;     // [n_stored + 4] pid << 1 | isY, pid ascending in a bucket; each
                                   // bucket padded to a multiple of 4 with 0xffffffff (16-byte groups)
    uint64_t n_stored = 0;         // entries including the pads (off[n_bins])
    int64_t* lf = nullptr;         // [kMaxLen + 1] LF[n] = round(2^32 log10 n!)
    int64_t* ls = nullptr;         // [s_max + 1]   LS[s] = round(2^32 log10 s)
    // chunk skip table of every non-empty bucket: row[bin] (-1 empty) and
    // skip[row * skip_stride + j] = entries with pid < j << kChunkShift
    int32_t* skip_row = nullptr;   // [n_bins]
    uint32_t* skip = nullptr;      // [rows * skip_stride]
    uint32_t skip_stride = 0;      // chunks + 1
    // hot buckets (at least P >> kHotShift entries) as pid bitmaps
    int32_t* hot_id = nullptr;     // [n_bins] (-1 not hot)
    uint32_t* pid_map = nullptr;   // [P] global pids of a subset (else NULL)
    uint32_t* hot_b = nullptr;     // [n_hot * hot_words] b-ion bits
    uint32_t* hot_y = nullptr;     // [n_hot * hot_words] y-ion bits
    uint32_t* hot_flags = nullptr; // [n_hot] bit 0: has b entries, bit 1: has y entries
    uint32_t n_hot = 0;
    uint64_t hot_words = 0;
    uint64_t bytes = 0;
    // optional per-phase timing of the last search (events on the call's stream)
    bool timing = false;
    void* ev[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};
    // launch shape used by hicops_search
    hicops_search_config cfg = {0, 0, 0, 0};
};

// Counts every kernel launch of the library.
void count_launches(uint64_t n);

}  // namespace hicops

struct hicops_index {
    hicops_params p;
    // residue masses used for every ion: unmodified (with fixed mod) and with
    // the letter's variable modification, indexed by ASCII letter
    double mres[128];
    double mmod[128];
    int8_t var_type[128];          // variable-mod rule per letter (-1 none)
    uint32_t n_var = 0;
    std::vector<double> var_delta;
    std::vector<uint32_t> var_max;

    // base (unmodified, deduplicated) peptides, in sequence-byte order
    std::string residues;          // concatenated letters
    std::vector<uint64_t> base_off;   // [B + 1]
    // database entries in pid order
    std::vector<double> mass;
    std::vector<uint32_t> base;
    std::vector<uint64_t> mask;

    // a shard of a database holds its entries pid_base, pid_base + pid_stride, ...:
    // global pid = local pid * pid_stride + pid_base (1 and 0 for a whole database)
    uint32_t pid_stride = 1, pid_base = 0;
    // a subset of a database (hicops_index_subset): global pid of each local
    // pid, ascending; empty otherwise (then the stride rule holds)
    std::vector<uint32_t> pid_map;

    uint32_t n_bins = 0;           // bins 0 .. n_bins-1 (absolute bin numbers)
    uint64_t s_max = 0;            // largest possible S
    hicops_index_stats stats{};
    hicops::DeviceIndex dev;
};

namespace hicops {
hicops_status validate_params(const hicops_params* p);
hicops_status upload_index(hicops_index* idx);
void free_device_index(hicops_index* idx);
}  // namespace hicops
