/*
 * hicops.h — C ABI of the GB300 peptide-database search library.
 *
 * The library implements the data-parallel hot path of the paper's
 * superstep 3 ("Partial Database Peptide Search", Eq. 4, Supplementary
 * Algorithm 3): for each experimental spectrum, the precursor-mass filter
 * (filter_1), the shared-fragment-ion filter over a fragment-ion index
 * (filter_2), hyperscore scoring of the candidates, the per-spectrum top-k
 * heap and the score histogram (the "local null distribution" of the
 * Sampling section), plus the linear-tail-fit e-value of superstep 4
 * (Supplementary Algorithm 4).  The database it searches is built by
 * superstep 1 ("Partial Database Construction", Supplementary Algorithm 1):
 * in-silico tryptic digestion, modification variants (the 2^m variants of
 * the Notation section), b/y model spectra and the fragment-ion index.
 *
 * Conventions for every entry point:
 *   - Every call returns a hicops_status; no exception crosses the ABI.
 *     On failure hicops_last_error() returns a thread-local message.
 *   - The caller owns every input and output buffer.  The library copies
 *     what it keeps; an index owns the device memory it allocated.
 *   - Device work runs on the CUDA device that is current for the calling
 *     thread when the index is built; later calls must use the same device.
 *   - An index is immutable after it is built: concurrent hicops_search
 *     calls on different streams are safe.
 *
 * Numeric readings (the paper leaves these open; they are fixed here):
 *   - monoisotopic residue masses, H2O 18.010565 Da, proton 1.007276466812 Da;
 *   - M = (sum of residue masses, left to right) + H2O; b_i = prefix_i +
 *     proton; y_i = ((sum of residues i+1..L from the C terminus) + H2O) +
 *     proton; fragment charge 1; FP64 throughout, no fused multiply-add;
 *   - bin(mz) = floor(mz / bin_width_da) for frag_mz_min <= mz < frag_mz_max;
 *     a query peak and a peptide ion are shared iff their bins are equal
 *     (bin width = the fragment tolerance dF);
 *   - a peptide's ion set is its set of distinct bins; a bin holding both a
 *     b and a y ion of one peptide counts once, as b;
 *   - pid = rank of the peptide in (neutral mass, sequence bytes,
 *     modification state) ascending order;
 *   - hyperscore HS = log10(nb!) + log10(ny!) + log10(S), S = sum of the
 *     matched quantised intensities; the exact rank key is
 *     K = LF[nb] + LF[ny] + LS[S] (int64, 2^32 fixed point, each term
 *     rounded to nearest); top-k by (K desc, pid asc); histogram bin
 *     min(255, K >> 31) over every candidate.
 */
#ifndef HICOPS_H
#define HICOPS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    HICOPS_OK = 0,
    HICOPS_EINVAL = 1,      /* invalid argument or unsupported parameter combination */
    HICOPS_ENOMEM = 2,      /* host or device allocation failed */
    HICOPS_ECUDA = 3,       /* a CUDA runtime call failed (message in hicops_last_error) */
    HICOPS_ETIMEOUT = 4,    /* a bounded device or host wait ran out */
    HICOPS_EOVERFLOW = 5,   /* a size limit of the index or of a counter would be exceeded */
    HICOPS_EBUSY = 6,       /* resource temporarily unavailable (server admission) */
    HICOPS_ECANCELLED = 7   /* request cancelled */
} hicops_status;

/* One modification rule (Notation section: each peptide expands into its
 * modified forms).  residues: NUL-terminated residue letters.  fixed = 1
 * applies delta_da to every such residue; fixed = 0 makes it variable with at
 * most max_per_peptide modified positions per peptide.  A residue letter may
 * carry at most one fixed and one variable rule. */
typedef struct hicops_mod {
    const char* residues;
    double delta_da;
    uint32_t max_per_peptide;
    uint32_t fixed;
} hicops_mod;

/* Search parameters.  Digestion follows the paper's Experimental Setup
 * (trypsin: cut after K/R unless followed by P; missed cleavages; length and
 * neutral-mass limits).  Limits: 2 <= min_len <= max_len <= 64;
 * 1 <= top_k <= 32; hist_bins == 256; 1 <= top_n_peaks <= 1024;
 * 2*(max_len-1) * intensity_scale < 2^20 (per-peptide counters are packed
 * into 32 bits); bin_width_da > 0; 0 < frag_mz_min < frag_mz_max and
 * frag_mz_max / bin_width_da < 2^31. */
typedef struct hicops_params {
    uint32_t min_len, max_len, missed_cleavages, max_total_mods; /* max_total_mods 0 = no cap */
    double min_mass, max_mass;
    double frag_mz_min, frag_mz_max, bin_width_da;
    uint32_t top_n_peaks, min_shared, top_k, hist_bins;
    uint32_t intensity_scale;
    /* Fragment tolerance in bins (dF = tol_bins * bin_width_da on a finer
     * grid; Experimental Setup's dF): a retained peak in bin b covers bins
     * b - tol_bins .. b + tol_bins, and an ion bin is shared iff some
     * retained peak covers it; it counts once, with the largest quantised
     * intensity of the peaks covering it.  0 = equal bins.  Requires
     * (2 * tol_bins + 1) * top_n_peaks <= 1024 (HICOPS_EINVAL otherwise). */
    uint32_t tol_bins;
    /* E-value of the top-k rows from the spectrum's score histogram
     * (Superstep 4, Supplementary Algorithm 4): 0 = the linear tail fit;
     * HICOPS_EVALUE_LOG_WEIBULL = the log-Weibull (Gumbel) fit instead;
     * HICOPS_EVALUE_SMOOTH = either fit on the histogram smoothed by the
     * 5-point quadratic Savitzky-Golay filter.  Other bits: HICOPS_EINVAL.
     * Superstep 4's own order, smoothing then the tail fit, is
     * HICOPS_EVALUE_SMOOTH (the Python workloads' default). */
    uint32_t evalue_mode;
    uint32_t reserved;   /* 0 */
} hicops_params;

#define HICOPS_EVALUE_LOG_WEIBULL 1u
#define HICOPS_EVALUE_SMOOTH 2u

/* Protein database: n_proteins sequences, protein i = seq[off[i] .. off[i+1]). */
typedef struct hicops_proteins {
    uint64_t n_proteins;
    const char* seq;
    const uint64_t* off;     /* [n_proteins + 1] */
} hicops_proteins;

/* A batch of experimental spectra (superstep 2's batches; a batch is the
 * unit of one search call).  Peaks of spectrum q are
 * mz/intensity[peak_off[q] .. peak_off[q+1]).  on_device = 1: every pointer
 * of the batch AND every output pointer of the call are device pointers on
 * the index's device, and the call is asynchronous on cuda_stream (results
 * are ready when the stream reaches that point).  on_device = 0: host
 * pointers; the call copies inputs in and results out and returns after the
 * results are in the caller's buffers.  A spectrum may hold any number of
 * raw peaks.  mz and intensity hold at least peak_off[n] entries (device
 * batches: the entries [peak_off[0], peak_off[n]) are the batch's).
 * Invalid spectra (charge 0, non-finite precursor, negative tolerance, no
 * peak inside [frag_mz_min, frag_mz_max), peak offsets that decrease or leave
 * [peak_off[0], peak_off[n])) do not fail the batch: their rows are padding,
 * their histogram is empty, and none of their peaks is read. */
typedef struct hicops_batch {
    uint32_t n;
    uint32_t on_device;
    const uint64_t* peak_off;  /* [n + 1] */
    const float* mz;
    const float* intensity;
    const double* prec_mz;     /* [n] precursor m/z */
    const uint8_t* charge;     /* [n] precursor charge z */
    const double* prec_tol_da; /* [n] precursor mass tolerance dM (Da) */
    void* cuda_stream;         /* cudaStream_t; NULL = legacy default stream */
} hicops_batch;

/* One peptide-spectrum match.  Padding rows (fewer than top_k candidates or
 * an invalid spectrum): pid = UINT32_MAX, key = INT64_MIN, nb = ny = 0,
 * hyperscore = 0, evalue = +inf. */
typedef struct hicops_psm {
    uint32_t query;        /* spectrum index within the batch */
    uint32_t pid;          /* peptide id (rank in the sorted database) */
    uint8_t nb, ny;        /* shared b / y ion bins */
    uint16_t reserved;
    float hyperscore;      /* (float)(key * 2^-32) */
    int64_t key;           /* exact rank key K */
    double evalue;         /* survival-tail fit (FP64) */
} hicops_psm;

typedef struct hicops_index_stats {
    uint64_t n_peptides;       /* P (database entries: sequence x modification state) */
    uint64_t n_base_peptides;  /* distinct unmodified sequences */
    uint64_t n_entries;        /* E: fragment-index entries (distinct bins summed over peptides) */
    uint64_t n_bins;           /* number of m/z bins */
    uint64_t device_bytes;     /* HBM held by the index */
    uint64_t max_bucket;       /* largest bucket */
    double host_ms;            /* digestion + variants + sort */
    double device_ms;          /* fragment-index build on the GPU */
} hicops_index_stats;

typedef struct hicops_index hicops_index;

/* Superstep 1 on the host only: digest, enumerate modification variants and
 * sort into pid order.  Uses no GPU.  The result supports
 * hicops_index_get_stats / hicops_peptide; hicops_index_upload makes it
 * searchable.  Errors: HICOPS_EINVAL (parameters), HICOPS_EOVERFLOW (2^31
 * peptides or more), HICOPS_ENOMEM. */
hicops_status hicops_digest(const hicops_proteins* proteins, const hicops_mod* mods, uint32_t n_mods,
                            const hicops_params* params, hicops_index** out);

/* Builds the device fragment-ion index (model spectra -> integer bins ->
 * radix-sorted CSR, pid ascending inside each bucket) on the current
 * device.  Errors: HICOPS_ECUDA, HICOPS_ENOMEM, HICOPS_EOVERFLOW (2^32 or
 * more entries in one bucket). */
hicops_status hicops_index_upload(hicops_index* index);

/* hicops_digest followed by hicops_index_upload. */
hicops_status hicops_build_index(const hicops_proteins* proteins, const hicops_mod* mods, uint32_t n_mods,
                                 const hicops_params* params, hicops_index** out);

/* Searches one batch (superstep 3's filter_1, filter_2, score, heap; and the
 * superstep-4 e-value).  Outputs: out_psm [n * top_k] rows, spectrum q at
 * rows q*top_k .. q*top_k+top_k-1 in rank order; out_hist [n * 256] or NULL;
 * out_nscored [n] (number of candidates, = sum of the histogram) or NULL.
 * Errors: HICOPS_EINVAL (bad batch,
 * index not uploaded), HICOPS_ECUDA, HICOPS_ENOMEM. */
hicops_status hicops_search(hicops_index* index, const hicops_batch* batch, hicops_psm* out_psm,
                            uint32_t* out_hist, uint32_t* out_nscored);

/* Largest batch hicops_search_noalloc accepts. */
#define HICOPS_NOALLOC_MAX_SPECTRA 64u

/* hicops_search without any device or host allocation.  The paper has no
 * counterpart: it is an addition of this library for callers that must not
 * allocate while they search, e.g. a serving loop with hard latency bounds
 * (cudaFree synchronises the device and cudaMalloc can stall on it) or a
 * process whose device memory is already reserved by another allocator, so
 * that hicops_search's stream-ordered scratch would fail.
 *   Same search, results and output layout as hicops_search, for a batch of
 * at most HICOPS_NOALLOC_MAX_SPECTRA spectra whose buffers are all on the
 * device (batch->on_device = 1).  out_psm [n * top_k] is a device buffer;
 * out_hist [n * 256] and out_nscored [n] are device buffers or NULL.  Work is
 * enqueued on batch->cuda_stream and the call returns without waiting.
 *   Scratch: one fixed array of about 1.2 MB in the library's device memory
 * per device, shared by every call on that device; each call rewrites what it
 * uses, so nothing has to be cleared between calls.  Calls whose work
 * overlaps in time (other streams or threads) race on that array and give
 * wrong results: order them, e.g. on one stream.  The first call on each
 * device looks up the array's device address (which may load the library's
 * device code on that device); make that first call before any stream
 * capture begins.  The looked-up address belongs to the device's context:
 * after that context is replaced (cudaDeviceReset), the next call looks it up
 * again, so make that call before any stream capture too.
 * Errors: HICOPS_EINVAL (more than HICOPS_NOALLOC_MAX_SPECTRA spectra, host
 * pointers, the hicops_search cases), HICOPS_ECUDA. */
hicops_status hicops_search_noalloc(hicops_index* index, const hicops_batch* batch, hicops_psm* out_psm,
                                    uint32_t* out_hist, uint32_t* out_nscored);

/* hicops_search with its device scratch in caller memory.  No passage
 * defines it: a memory-management addition of this library for callers that
 * pool device memory themselves (the serving loop below admits its launches
 * this way, by the bytes each one needs).
 *   hicops_search_scratch_bytes: *out_bytes receives the scratch one search of
 * n spectra takes on this index with its current launch shape (n = 0 counts
 * as 1).  It depends on n alone, not on the spectra's peaks.
 *   hicops_search_scratch: same search, results and output layout as
 * hicops_search, for a batch whose buffers are all on the device
 * (on_device = 1), with scratch a device buffer of scratch_bytes bytes that
 * starts on a 256-byte boundary.  out_psm [n * top_k] is a device buffer;
 * out_hist [n * 256] and out_nscored [n] are device buffers or NULL.  Work is
 * enqueued on batch->cuda_stream and the call returns without waiting or
 * allocating; the scratch must stay untouched until the stream has passed the
 * search, and needs no clearing before it.  A change of the index's launch
 * shape (hicops_index_set_config, hicops_autotune) can change the bytes.
 * Errors: HICOPS_EINVAL (host pointers, NULL or misaligned scratch, the
 * hicops_search cases), HICOPS_ENOMEM (scratch_bytes below what
 * hicops_search_scratch_bytes gives for this n), HICOPS_ECUDA. */
hicops_status hicops_search_scratch_bytes(const hicops_index* index, uint32_t n, uint64_t* out_bytes);
hicops_status hicops_search_scratch(hicops_index* index, const hicops_batch* batch, void* scratch,
                                    uint64_t scratch_bytes, hicops_psm* out_psm, uint32_t* out_hist,
                                    uint32_t* out_nscored);

/* Measurement helper: per spectrum, the precursor window [lo, hi) (Eq. 4's
 * filter_1), the number of retained peaks and the number of index entries
 * inside the window over the retained peaks' buckets (H(q), the work of
 * filter_2, Eq. 4 terms k32'/k33).  Any output may be NULL.  Same pointer
 * rules and errors as hicops_search. */
hicops_status hicops_search_work(hicops_index* index, const hicops_batch* batch, uint32_t* out_lo,
                                 uint32_t* out_hi, uint32_t* out_npeaks, uint64_t* out_hits);

/* Sizes of the index: P and the unmodified sequences (Notation section: the
 * database of D = zeta * 2^m entries), the fragment-index entries and bins
 * (Superstep 1 items 2-3), device bytes and build times.  The name
 * hicops_index_stats is the struct's; the call carries get_ so the two do
 * not collide in C.  Errors: HICOPS_EINVAL (NULL). */
hicops_status hicops_index_get_stats(const hicops_index* index, hicops_index_stats* out);

/* The parameters the index was built with (the Experimental Setup's
 * digestion and tolerance settings as this library reads them).  No passage
 * defines the call itself: a library utility.  Errors: HICOPS_EINVAL (NULL). */
hicops_status hicops_index_get_params(const hicops_index* index, hicops_params* out);

/* Checkpoint of an index's host half (the digested database: peptide table,
 * masses, modification tables, and a part's pid mapping) in one file at
 * path, so a later process skips digestion (the paper writes its prepared
 * data back for reuse, Superstep 2); hicops_index_load reads it back as a
 * host-only index, and hicops_index_upload rebuilds the device half.  The
 * format is fixed-width little-endian, versioned, and checked on load.
 * Errors: HICOPS_EINVAL (NULL, unwritable / unreadable path, not a complete
 * index file of this format, inconsistent contents, invalid parameters),
 * HICOPS_ENOMEM. */
hicops_status hicops_index_save(const hicops_index* index, const char* path);
hicops_status hicops_index_load(const char* path, hicops_index** out);

/* ---- database sharding (paper: every process searches its own partition of
 * the database, Superstep 3 and the Load Balancing section; the partial
 * score distributions are added and the results assembled, Superstep 4). */

/* Most shards of one database. */
#define HICOPS_MAX_SHARDS 64u

/* Shard `shard` of n_shards of a digested database (hicops_digest; need not
 * be uploaded): the entries with pid = shard, shard + n_shards, ... (a
 * round-robin partition of the mass-sorted order, so every shard sees every
 * precursor window evenly).  The shard is a host-only index like
 * hicops_digest's; hicops_index_upload builds its device part.  Its search
 * results carry global pids, its histograms and candidate counts cover its own
 * candidates, and its e-values are fitted to its own histogram only: combine
 * the shards with hicops_merge_shards.  hicops_peptide on a shard takes global
 * pids of the shard; hicops_index_copy_csr reports shard-local pids.
 * Errors: HICOPS_EINVAL (shard >= n_shards, n_shards outside
 * [1, HICOPS_MAX_SHARDS], index already a shard), HICOPS_ENOMEM. */
hicops_status hicops_index_shard(const hicops_index* full, uint32_t n_shards, uint32_t shard,
                                 hicops_index** out);

/* The part of a whole database (hicops_digest; need not be uploaded) holding
 * the n entries pids[0] < pids[1] < ... (strictly ascending global pids, any
 * subset: e.g. one partition of hicops_partition_lbe).  Like a shard of
 * hicops_index_shard it is a host-only index, its rows carry global pids and
 * hicops_merge_shards combines it with the other parts; it cannot be split
 * again.  The caller keeps pids.  Errors: HICOPS_EINVAL (NULL, pids not
 * strictly ascending or not below the database size, index already a part),
 * HICOPS_ENOMEM. */
hicops_status hicops_index_subset(const hicops_index* full, const uint32_t* pids, uint64_t n,
                                  hicops_index** out);

/* The load-balancing partition of Superstep 1 (the improved LBE with the Mod
 * Distance, Supplementary Text 3 and Supplementary Fig. 3): part[pid] in
 * [0, n_parts) for every pid of a whole database.  The entries sharing one
 * unmodified sequence form a cluster, ordered inside by (edit distance to
 * the unmodified sequence, Mod Distance to it, pid); the clusters follow one
 * another by their smallest pid and position i of the sequence goes to part
 * i mod n_parts, so every part holds an equal share (within one entry) of
 * every cluster and of every mass range.  part [P] is caller-owned host
 * memory.  Host only.  Errors: HICOPS_EINVAL (NULL, n_parts outside
 * [1, HICOPS_MAX_SHARDS], index already a part). */
hicops_status hicops_partition_lbe(const hicops_index* full, uint32_t n_parts, uint32_t* part);

/* Combines the shards' searches of the same n spectra: per spectrum, sums the
 * histograms and candidate counts, merges the shard top-k lists by (key desc,
 * pid asc) and fits the e-value to the summed histogram (the same merge and
 * fit as hicops_search), so the result equals the unsharded search.
 *   shard_psm [n_shards * n * top_k]: shard s's rows of spectrum q at
 *   (s * n + q) * top_k; hist [hist_parts * n * 256] and nscored
 *   [hist_parts * n]: hist_parts = n_shards (per shard, summed here) or 1
 *   (already summed, e.g. by an all-reduce).  evalue_mode as in hicops_params
 *   (the shards' own; HICOPS_EINVAL for other bits).  Outputs as hicops_search
 *   (out_hist, out_nscored may be NULL).  on_device = 1: every buffer is a
 *   device buffer and the work is enqueued on cuda_stream; 0: host buffers,
 *   the call copies and waits.  Runs on the current device.
 * Errors: HICOPS_EINVAL (sizes, NULL inputs), HICOPS_ECUDA, HICOPS_ENOMEM. */
hicops_status hicops_merge_shards(uint32_t n_shards, uint32_t n, uint32_t top_k, const hicops_psm* shard_psm,
                                  const uint32_t* hist, const uint32_t* nscored, uint32_t hist_parts,
                                  uint32_t evalue_mode, int on_device, void* cuda_stream, hicops_psm* out_psm,
                                  uint32_t* out_hist, uint32_t* out_nscored);

/* ---- sampled partial score distributions (Sampling section and its
 * figure: a process's partial distribution of one spectrum is reduced to at
 * most s samples around its mean before it leaves the process; the tails,
 * which the fit recovers, are pruned first).  A sample is one histogram bin.
 * The mean is the integer average (rounded down) of the locations of the
 * three most intense bins (count descending, lower location first; fewer
 * when fewer bins are non-zero); of the non-zero bins' span, the end farther
 * from the mean is dropped (the upper end on a tie) while more than s bins
 * remain.  A record is s + 1 words: word 0 = lo | len << 16, words 1..len the
 * counts of bins lo .. lo+len-1 (exact), the rest 0; len = 0 for an empty
 * histogram.  Score histograms of 0.5 log10 units a bin span far fewer than
 * the paper's s = 120 bins, so at that s the record holds the whole
 * histogram. */
#define HICOPS_SAMPLE_S 120u

/* Samples n histograms hist [n * 256] into records out_rec [n * (s + 1)],
 * 1 <= s <= 256.  on_device = 1: device buffers, enqueued on cuda_stream;
 * 0: host buffers, the call copies and waits.  Errors: HICOPS_EINVAL (s out
 * of range, NULL), HICOPS_ECUDA, HICOPS_ENOMEM. */
hicops_status hicops_hist_sample(uint32_t n, const uint32_t* hist, uint32_t s, uint32_t* out_rec, int on_device,
                                 void* cuda_stream);

/* Assembles sampled partial distributions (Superstep 4's addition of the
 * partial distributions): out_hist [n * 256] = per spectrum the sum over the
 * n_parts parts of their records' counts, rec [n_parts * n * (s + 1)] (part
 * p's record of spectrum q at (p * n + q) * (s + 1)).  The result goes to
 * hicops_merge_shards with hist_parts = 1.  Buffers as hicops_hist_sample,
 * but the call always waits for cuda_stream (it reads back whether every
 * record was well formed).  Errors as hicops_hist_sample; also HICOPS_EINVAL
 * for n_parts outside [1, HICOPS_MAX_SHARDS] or a record whose bins leave
 * [0, 256) or exceed s (out_hist then holds the sums of the valid records). */
hicops_status hicops_hist_unsample(uint32_t n_parts, uint32_t n, uint32_t s, const uint32_t* rec, uint32_t* out_hist,
                                   int on_device, void* cuda_stream);

/* ---- host ingest pipeline (Superstep 3's R/I/K sub-tasks: Buffering and
 * Task Scheduling sections, Supplementary Algorithm 2).  MS2 text files
 * ("S <scan> <scan> <precursor m/z>", "Z <charge> <[M+H]+>" (the first Z
 * gives the charge; none = charge 0), optional "H"/"I"/"D" lines, and
 * "<m/z> <intensity>" peak lines) are parsed into batch buffers by R
 * workers, searched by I workers (hicops_search on a stream of their own)
 * and written by one K thread; buffers circulate through a recycle and a
 * forward queue.  Workers move between R and I by the paper's rules (see
 * hicops_sched_*), an I worker forecasting its next wait for the forward
 * queue by double exponential smoothing (hicops_des_step). */
typedef struct hicops_pipeline_config {
    uint32_t batch_spectra;   /* spectra per buffer (0 = 1024) */
    uint32_t n_buffers;       /* buffers in circulation (0 = 20; >= 2) */
    uint32_t n_workers;       /* R + I worker threads (0 = 4; >= 2); one starts as R */
    uint32_t reserved;        /* 0 */
    double prec_tol_da;       /* precursor tolerance dM of every spectrum (>= 0) */
    double alpha;             /* smoothing factor in (0, 1) (else 0.5) */
    double t_min_s, t_max_s;  /* wait thresholds t_min and t_max in seconds (<= 0: 1 ms, 50 ms) */
} hicops_pipeline_config;

typedef struct hicops_pipeline_stats {
    uint64_t spectra, batches;           /* searched */
    uint64_t moves_i_to_r, moves_r_to_i; /* scheduler decisions taken */
    double seconds;                      /* wall time of the run */
    double wait_seconds;                 /* time I workers waited for the forward queue */
} hicops_pipeline_stats;

/* Searches every spectrum of the files against an uploaded index and writes
 * out_path: a tab-separated header line, then one line per real top-k row
 * "file scan spectrum rank pid nb ny hyperscore evalue n_scored" (file = index
 * into paths, spectrum = index inside the file; hyperscore and evalue in
 * their shortest round-trip decimal form), rows of a spectrum consecutive and
 * in rank order, spectra in no set
 * order.  The rows are those hicops_search gives for the same spectra with
 * tolerance prec_tol_da.  stats may be NULL.  Errors: HICOPS_EINVAL (NULL,
 * bad config, unreadable file, malformed MS2 line (the message names file and
 * line), unwritable output), search errors as hicops_search. */
hicops_status hicops_pipeline_run(hicops_index* index, const char* const* paths, uint32_t n_paths,
                                  const char* out_path, const hicops_pipeline_config* cfg,
                                  hicops_pipeline_stats* stats);

/* Parses one MS2 file (format above) into caller-owned host arrays:
 * peak_off [n_spectra + 1], mz / intensity [n_peaks], prec_mz / charge /
 * scan [n_spectra].  *n_spectra and *n_peaks are always set; the arrays are
 * written only when they fit cap_spectra and cap_peaks (call once with caps
 * 0 to size them).  Any array pointer may be NULL.  Errors: HICOPS_EINVAL
 * (NULL, unreadable file, malformed line). */
hicops_status hicops_ms2_read(const char* path, uint32_t cap_spectra, uint64_t cap_peaks, uint32_t* n_spectra,
                              uint64_t* n_peaks, uint64_t* peak_off, float* mz, float* intensity,
                              double* prec_mz, uint8_t* charge, uint32_t* scan);

/* One step of double exponential smoothing (LaViola 2003, as the Task
 * Scheduling section forecasts t_wait): s1 = a x + (1 - a) s1, s2 = a s1 +
 * (1 - a) s2, both starting at the first sample (first != 0); returns the
 * forecast of the next sample, (2 + a/(1-a)) s1 - (1 + a/(1-a)) s2.
 * state [2] is the caller's. */
double hicops_des_step(double* state, double x, double alpha, int first);

/* The scheduling rules: an I worker turns to R when
 * (t_wait >= t_min and t_cum + t_fct > t_max) or (the forward queue holds
 * fewer than 5 buffers and no worker is in R); an R worker turns to I when
 * (the queue holds 15 or more and more than one worker is in R) or the queue
 * is full.  Return 1 for a move. */
int hicops_sched_i_to_r(double t_wait, double t_cum, double t_fct, double t_min, double t_max, uint32_t qf_len,
                        uint32_t n_r);
int hicops_sched_r_to_i(uint32_t qf_len, uint32_t qf_cap, uint32_t n_r);

/* Peptide pid: sequence (NUL-terminated, truncated to cap-1 letters), neutral
 * mass and the bitmask of positions carrying a variable modification (bit j =
 * residue j, 0-based): the database entry a PSM names (the results of
 * Supplementary Table 1 list peptide sequences with their modifications).
 * On a shard or part, pid is a global pid of that shard or part.  Host only.
 * seq, mass and modmask may be NULL (cap = 0 leaves seq untouched).  Errors:
 * HICOPS_EINVAL (NULL index, pid not in the index). */
hicops_status hicops_peptide(const hicops_index* index, uint32_t pid, char* seq, uint32_t cap,
                             double* mass, uint64_t* modmask);

/* Copies the fragment index (Superstep 1 items 2-3: the model spectra's ions
 * binned and indexed) to host buffers: off [n_bins + 1] bucket offsets and
 * entries [n_entries] = pid << 1 | isY, buckets back to back (the device
 * copy pads each bucket to a multiple of 4 entries; the pads are left out).
 * Either may be NULL.  Errors: HICOPS_EINVAL (not uploaded), HICOPS_ECUDA,
 * HICOPS_ENOMEM (host staging of the padded copy). */
hicops_status hicops_index_copy_csr(const hicops_index* index, uint64_t* off, uint32_t* entries);

/* Launch shape of the search kernel (the paper's R/I/K balancing of
 * superstep 3 becomes the choice of how spectra and peptide ranges map onto
 * persistent CTAs).  Zero fields take the default.  threads: CTA size, 256,
 * 384 or 512 (default 384 for top_k <= 16, else 256).  chunk_entries: index entries a CTA aims to accumulate per pass
 * over a range of peptide ids, in units of 1024, 1..16 (default 12); the range
 * is sized from the spectrum's entry density.  ctas_per_sm: resident CTAs per
 * SM (0 = as many as fit).  seg_pids: a spectrum's precursor window is split
 * into work units of at least this many peptide ids (0 = split only when the
 * batch is too small to fill the GPU).  Results do not depend on the shape. */
typedef struct hicops_search_config {
    uint32_t threads;
    uint32_t chunk_entries;
    uint32_t ctas_per_sm;
    uint32_t seg_pids;
} hicops_search_config;

/* Sets the launch shape hicops_search uses for this index (NULL = defaults).
 * Errors: HICOPS_EINVAL for an unsupported shape. */
hicops_status hicops_index_set_config(hicops_index* index, const hicops_search_config* cfg);

/* Times every candidate launch shape on a device-resident sample batch
 * (on_device = 1) and stores the fastest in the index (as
 * hicops_index_set_config would); *best and *best_ms receive it when not
 * NULL.  Synchronises the batch's stream. */
hicops_status hicops_autotune(hicops_index* index, const hicops_batch* sample, hicops_search_config* best,
                              double* best_ms);

/* A reusable search (the batched form): device scratch for up to
 * max_spectra spectra is allocated once at creation, and hicops_plan_search
 * enqueues the whole search (preprocessing to e-value) on the batch's stream
 * without allocating.  With use_graph = 1 and a non-NULL stream, the first
 * call for a given (batch, outputs) is captured into a CUDA graph and later
 * calls with the same pointers and sizes replay it.  The batch and outputs
 * must be device pointers (on_device = 1).  A plan serves one stream at a
 * time.  Errors: HICOPS_EINVAL (batch larger than max_spectra, host
 * pointers), HICOPS_ENOMEM, HICOPS_ECUDA. */
typedef struct hicops_plan hicops_plan;
hicops_status hicops_plan_create(hicops_index* index, uint32_t max_spectra, const hicops_search_config* cfg,
                                 hicops_plan** out);
hicops_status hicops_plan_search(hicops_plan* plan, const hicops_batch* batch, hicops_psm* out_psm,
                                 uint32_t* out_hist, uint32_t* out_nscored, int use_graph);
void hicops_plan_destroy(hicops_plan* plan);

/* Serving loop (the paper's buffering and R/I/K pipeline of superstep 3,
 * Buffering and Task Scheduling sections, as a request server).  The index
 * stays resident; requests (batches of spectra in host memory) are copied at
 * submission and queued.  The server's device memory is one pool of
 * memory_budget bytes, allocated at creation.  A scheduler thread packs the
 * oldest waiting requests into one launch while that launch's block (its
 * spectra, the search's scratch as hicops_search_scratch_bytes counts it,
 * its PSM rows, histograms and counts) fits the pool's largest free range,
 * and launches it on an idle stream; when the oldest request does not fit,
 * it waits until launches in flight return their blocks.  Requests that
 * arrive while others run are thus admitted as memory and streams free up,
 * and their work overlaps on the device.  n_slots: launches in flight at
 * most (one stream each, 1..64); slot_spectra: spectra one launch packs at most;
 * memory_budget: the pool's bytes.  A request of more than slot_spectra
 * spectra, or whose launch alone would not fit the pool, is rejected at
 * submission (HICOPS_EINVAL).  Results do not depend on how requests are
 * packed.  The launch shape is the index's at creation.  Zero fields take the
 * defaults (4 launches, 32768 spectra, 16 GiB).  Errors of create:
 * HICOPS_EINVAL (n_slots above 64, a budget below one launch of one
 * 512-peak spectrum),
 * HICOPS_ENOMEM (the pool cannot be allocated), HICOPS_ECUDA. */
typedef struct hicops_server_cfg {
    uint32_t n_slots;
    uint32_t slot_spectra;
    uint64_t memory_budget;
} hicops_server_cfg;

typedef struct hicops_server_stats {
    uint64_t submitted, completed, launches, spectra;
    uint32_t n_slots;          /* launches in flight at most */
    uint32_t reserved;
    uint64_t pool_bytes;       /* the device pool */
    uint64_t pool_peak;        /* most pool bytes held by launches at once */
    uint64_t memory_waits;     /* times the oldest request had to wait for pool memory */
} hicops_server_stats;

typedef struct hicops_server hicops_server;

hicops_status hicops_server_create(hicops_index* index, const hicops_server_cfg* cfg, hicops_server** out);

/* Queues a request (batch in host memory, on_device = 0; the arrays are
 * copied before the call returns).  *ticket identifies it for poll/cancel.
 * Errors: HICOPS_EINVAL (NULL pointers, device pointers, 0 or more than
 * slot_spectra spectra, peak offsets that decrease, a launch larger than
 * the pool). */
hicops_status hicops_server_submit(hicops_server* srv, const hicops_batch* batch, uint64_t* ticket);

/* Waits up to timeout_ms (0 = do not wait, < 0 = wait forever) for the
 * request; when it is done, copies its rows [n * top_k], histograms
 * [n * 256] and candidate counts [n] (either may be NULL) to host memory
 * and forgets the ticket.  HICOPS_ETIMEOUT: not done yet (the ticket stays
 * valid); HICOPS_ECANCELLED: cancelled; HICOPS_EINVAL: unknown ticket. */
hicops_status hicops_server_poll(hicops_server* srv, uint64_t ticket, int timeout_ms, hicops_psm* out_psm,
                                 uint32_t* out_hist, uint32_t* out_nscored);

/* Cancels a request that has not been launched yet (HICOPS_EBUSY if it
 * has). */
hicops_status hicops_server_cancel(hicops_server* srv, uint64_t ticket);

/* Counters of the server (requests submitted and completed, launches,
 * spectra, pool use): the buffering section's queues observed.  Errors:
 * HICOPS_EINVAL (NULL). */
hicops_status hicops_server_get_stats(hicops_server* srv, hicops_server_stats* out);

/* Waits for launched work, drops queued requests, frees the pool and the
 * streams. */
void hicops_server_destroy(hicops_server* srv);

/* Per-phase device time of the last hicops_search on this index, measured
 * with CUDA events recorded on the call's stream (the phases of Eq. 4:
 * preprocessing and filter_1, filter_2 with scoring, the merge).  No passage
 * defines the call: a measurement utility.  With timing enabled, concurrent
 * searches on one index overwrite each other's events.
 * hicops_index_last_timing waits for the last call's end event.  Errors:
 * HICOPS_EINVAL (not uploaded, timing not enabled), HICOPS_ECUDA. */
typedef struct hicops_timing {
    float prep_ms;      /* preprocessing + precursor window */
    float plan_ms;      /* work-unit planning (segments, scan) */
    float search_ms;    /* shared-peak accumulation, scoring, top-k, histogram */
    float merge_ms;     /* top-k merge + e-value */
    float total_ms;     /* first to last kernel of the call */
} hicops_timing;

hicops_status hicops_index_set_timing(hicops_index* index, int enable);
hicops_status hicops_index_last_timing(hicops_index* index, hicops_timing* out);

/* Number of CUDA kernels this library has launched in this process.  No
 * passage: a library utility (it shows that searches ran on the GPU). */
uint64_t hicops_kernel_launches(void);

/* Frees an index and its device half.  NULL is a no-op.  No passage: a
 * library utility. */
void hicops_index_free(hicops_index* index);

/* Thread-local description of the last failure on this thread (never NULL;
 * owned by the library, valid until the thread's next failing call).  No
 * passage: a library utility. */
const char* hicops_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* HICOPS_H */
