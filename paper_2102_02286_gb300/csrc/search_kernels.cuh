// Device kernels of the search path (included by search.cu only):
// preprocessing + precursor window, unit planning, the shared-peak search
// kernel (search_kernel.cuh), the top-k merge + e-value, and the work count.
#pragma once

#include <cfloat>
#include <cmath>

#include "dev_common.cuh"

namespace hicops {
namespace {

constexpr int kPrepThreads = 256;
constexpr int kPrepWarpPeaks = 256;        // spectra with at most this many raw peaks: one warp each
constexpr int kPrepWarps = 8;              // spectra per block of prep_warp_kernel
constexpr int kMinSegPids = (int)kChunk;  // smallest segment of a split window
constexpr int kMaxSegs = 64;              // most segments a window is split into
constexpr int kMergeWarps = 8;          // spectra per merge block

struct UnitTop {
    int64_t key;
    uint32_t pid;
    uint32_t packed;    // nb << 26 | ny << 20 | S
};

struct PrepArgs {
    const uint64_t* peak_off;
    const float* mz;
    const float* inten;
    const double* prec_mz;
    const uint8_t* charge;
    const double* tol;
    uint32_t n;
    uint32_t topn;      // peaks retained
    uint32_t stride;    // qbin / qiq words per spectrum (>= topn)
    double w, mz_lo, mz_hi, scale;
    const double* mass;
    uint64_t P;
    uint32_t* qbin;     // [n * stride]
    uint32_t* qiq;      // [n * stride]
    uint32_t* qn;       // [n]
    uint32_t* lo;       // [n]
    uint32_t* hi;       // [n]
};

__device__ __forceinline__ void bitonic_sort_u64(uint64_t* s, int npow) {
    for (int k = 2; k <= npow; k <<= 1) {
        for (int j = k >> 1; j > 0; j >>= 1) {
            for (int i = threadIdx.x; i < npow; i += blockDim.x) {
                const int ixj = i ^ j;
                if (ixj > i) {
                    const uint64_t a = s[i], b = s[ixj];
                    const bool up = (i & k) == 0;
                    if ((a > b) == up) { s[i] = b; s[ixj] = a; }
                }
            }
            __syncthreads();
        }
    }
}

__device__ __forceinline__ int next_pow2(int v) {
    int p = 1;
    while (p < v) p <<= 1;
    return p;
}

// first index in [0, n) with mass[i] >= x  (or > x when upper)
__device__ __forceinline__ uint64_t mass_bound(const double* mass, uint64_t n, double x, bool upper) {
    uint64_t a = 0, b = n;
    while (a < b) {
        const uint64_t m = (a + b) >> 1;
        const double v = mass[m];
        if (upper ? (v <= x) : (v < x)) a = m + 1; else b = m;
    }
    return a;
}

// Spectra of more than kPrepWarpPeaks raw peaks, one block each, any number
// of raw peaks: the raw peaks are taken in chunks of kPrepChunk, and each
// chunk is merged with the running list of the best top_n bins so far (in
// raw form again: bin << 32 | intensity bits), sorted by bin, reduced to one
// representative per bin (its largest intensity), re-keyed by (intensity
// desc, bin asc), sorted, and cut to top_n.  A bin's value in the list only
// grows, so a bin left out at some chunk has top_n better bins from then on:
// the final list is the top_n bins of the whole spectrum by their largest
// intensity (R8), whatever the chunking.
constexpr int kPrepSort = 4096;                // keys sorted per chunk
constexpr int kPrepChunk = kPrepSort - (int)kMaxTopN;   // raw peaks per chunk

__global__ void __launch_bounds__(kPrepThreads) prep_kernel(PrepArgs a) {
    __shared__ uint64_t keys[kPrepSort];
    __shared__ uint64_t best[kMaxTopN];          // the running list, raw form
    __shared__ int s_nrep;
    const uint32_t q = blockIdx.x;
    const uint64_t p0 = a.peak_off[q], p1 = a.peak_off[q + 1];
    // a spectrum's peaks lie inside the batch's [peak_off[0], peak_off[n]),
    // else it is invalid and nothing of it is read
    const bool inside = p0 <= p1 && p0 >= a.peak_off[0] && p1 <= a.peak_off[a.n];
    const uint64_t cnt = inside ? p1 - p0 : 0;
    if (cnt <= (uint64_t)kPrepWarpPeaks) return;   // prep_warp_kernel's spectra
    const double prec = a.prec_mz[q];
    const double tol = a.tol[q];
    const uint32_t z = a.charge[q];
    bool valid = inside && z > 0 && isfinite(prec) && isfinite(tol) && tol >= 0.0;
    int keep = 0;
    if (valid && cnt > 0) {
        for (uint64_t base = 0; base < cnt; base += kPrepChunk) {
            const int m = (int)min((uint64_t)kPrepChunk, cnt - base);
            const int total = m + keep;
            const int npow = next_pow2(total);
            // key = bin << 32 | intensity bits (positive finite floats order as integers)
            for (int i = threadIdx.x; i < npow; i += blockDim.x) {
                uint64_t k = ~0ull;
                if (i < m) {
                    const float mz = a.mz[p0 + base + i], I = a.inten[p0 + base + i];
                    const double md = (double)mz;
                    if (isfinite(mz) && isfinite(I) && I > 0.0f && md >= a.mz_lo && md < a.mz_hi) {
                        const uint32_t bin = (uint32_t)floor(md / a.w);
                        k = ((uint64_t)bin << 32) | __float_as_uint(I);
                    }
                } else if (i < total) {
                    k = best[i - m];
                }
                keys[i] = k;
            }
            if (threadIdx.x == 0) s_nrep = 0;
            __syncthreads();
            bitonic_sort_u64(keys, npow);
            // one representative per bin: the last (most intense) of each run
            uint64_t rep[kPrepSort / kPrepThreads];
            int nr = 0;
            for (int i = threadIdx.x; i < npow; i += blockDim.x) {
                const uint64_t k = keys[i];
                if (k == ~0ull) continue;
                const bool last = (i + 1 == npow) || ((keys[i + 1] >> 32) != (k >> 32));
                // re-key: intensity descending, then bin ascending
                if (last) rep[nr++] = ((uint64_t)(~(uint32_t)k) << 32) | (k >> 32);
            }
            __syncthreads();
            for (int r = 0; r < nr; ++r) keys[atomicAdd(&s_nrep, 1)] = rep[r];
            __syncthreads();
            const int nrep = s_nrep;
            const int npow2 = next_pow2(nrep > 0 ? nrep : 1);
            for (int i = nrep + threadIdx.x; i < npow2; i += blockDim.x) keys[i] = ~0ull;
            __syncthreads();
            bitonic_sort_u64(keys, npow2);
            keep = nrep < (int)a.topn ? nrep : (int)a.topn;
            // the running list back in raw form for the next chunk
            for (int t = threadIdx.x; t < keep; t += blockDim.x) {
                const uint64_t k = keys[t];
                best[t] = ((uint64_t)(uint32_t)k << 32) | (uint32_t)~(uint32_t)(k >> 32);
            }
            __syncthreads();
        }
        if (keep > 0) {
            const double Imax = (double)__uint_as_float(~(uint32_t)(keys[0] >> 32));
            for (int t = threadIdx.x; t < keep; t += blockDim.x) {
                const uint64_t k = keys[t];
                const double I = (double)__uint_as_float(~(uint32_t)(k >> 32));
                const double r = floor(__dmul_rn(I, a.scale) / Imax);
                a.qbin[(uint64_t)q * a.stride + t] = (uint32_t)k;
                a.qiq[(uint64_t)q * a.stride + t] = r < 1.0 ? 1u : (uint32_t)r;
            }
        }
    }
    valid = valid && keep > 0;
    if (threadIdx.x == 0) {
        a.qn[q] = valid ? (uint32_t)keep : 0u;
        uint32_t lo = 0, hi = 0;
        if (valid) {
            const double Mq = __dmul_rn(__dsub_rn(prec, kProtonDa), (double)z);
            lo = (uint32_t)mass_bound(a.mass, a.P, __dsub_rn(Mq, tol), false);
            hi = (uint32_t)mass_bound(a.mass, a.P, __dadd_rn(Mq, tol), true);
        }
        a.lo[q] = lo;
        a.hi[q] = hi;
    }
}

__device__ __forceinline__ void warp_bitonic_sort_u64(uint64_t* s, int npow, int lane) {
    for (int k = 2; k <= npow; k <<= 1) {
        for (int j = k >> 1; j > 0; j >>= 1) {
            for (int i = lane; i < npow; i += 32) {
                const int ixj = i ^ j;
                if (ixj > i) {
                    const uint64_t x = s[i], y = s[ixj];
                    const bool up = (i & k) == 0;
                    if ((x > y) == up) { s[i] = y; s[ixj] = x; }
                }
            }
            __syncwarp();
        }
    }
}

// prep_kernel's computation for spectra of at most kPrepWarpPeaks raw
// peaks, one warp each, in a 2 KB slice of shared memory: the same keys and
// sorts, so the same retained peaks, quantised intensities and window.
__global__ void __launch_bounds__(kPrepWarps * 32) prep_warp_kernel(PrepArgs a) {
    __shared__ uint64_t keys_all[kPrepWarps][kPrepWarpPeaks];
    const int lane = threadIdx.x & 31, wi = threadIdx.x >> 5;
    const uint32_t q = blockIdx.x * kPrepWarps + wi;
    if (q >= a.n) return;
    uint64_t* keys = keys_all[wi];
    const uint64_t p0 = a.peak_off[q], p1 = a.peak_off[q + 1];
    const bool inside = p0 <= p1 && p0 >= a.peak_off[0] && p1 <= a.peak_off[a.n];   // as in prep_kernel
    const uint64_t cnt = inside ? p1 - p0 : 0;
    if (cnt > (uint64_t)kPrepWarpPeaks) return;   // prep_kernel's spectra
    const double prec = a.prec_mz[q];
    const double tol = a.tol[q];
    const uint32_t z = a.charge[q];
    bool valid = inside && z > 0 && isfinite(prec) && isfinite(tol) && tol >= 0.0;
    int keep = 0;
    if (valid && cnt > 0) {
        const int npow = next_pow2((int)cnt);
        for (int i = lane; i < npow; i += 32) {
            uint64_t k = ~0ull;
            if (i < (int)cnt) {
                const float m = a.mz[p0 + i], I = a.inten[p0 + i];
                const double md = (double)m;
                if (isfinite(m) && isfinite(I) && I > 0.0f && md >= a.mz_lo && md < a.mz_hi) {
                    const uint32_t bin = (uint32_t)floor(md / a.w);
                    k = ((uint64_t)bin << 32) | __float_as_uint(I);
                }
            }
            keys[i] = k;
        }
        __syncwarp();
        warp_bitonic_sort_u64(keys, npow, lane);
        // one representative per bin (the most intense), re-keyed by
        // (intensity desc, bin asc) and compacted in place in index order
        int nrep = 0;
        for (int i0 = 0; i0 < npow; i0 += 32) {
            const int i = i0 + lane;
            uint64_t r = 0;
            bool is_rep = false;
            if (i < npow) {
                const uint64_t k = keys[i];
                if (k != ~0ull) {
                    is_rep = (i + 1 == npow) || ((keys[i + 1] >> 32) != (k >> 32));
                    r = ((uint64_t)(~(uint32_t)k) << 32) | (k >> 32);
                }
            }
            const unsigned msk = __ballot_sync(0xffffffffu, is_rep);
            __syncwarp();   // every read of this round before any write (writes land at indices <= i)
            if (is_rep) keys[nrep + __popc(msk & ((1u << lane) - 1u))] = r;
            nrep += __popc(msk);
            __syncwarp();
        }
        const int npow2 = next_pow2(nrep > 0 ? nrep : 1);
        for (int i = nrep + lane; i < npow2; i += 32) keys[i] = ~0ull;
        __syncwarp();
        warp_bitonic_sort_u64(keys, npow2, lane);
        keep = nrep < (int)a.topn ? nrep : (int)a.topn;
        if (keep > 0) {
            const double Imax = (double)__uint_as_float(~(uint32_t)(keys[0] >> 32));
            for (int t = lane; t < keep; t += 32) {
                const uint64_t k = keys[t];
                const double I = (double)__uint_as_float(~(uint32_t)(k >> 32));
                const double r = floor(__dmul_rn(I, a.scale) / Imax);
                a.qbin[(uint64_t)q * a.stride + t] = (uint32_t)k;
                a.qiq[(uint64_t)q * a.stride + t] = r < 1.0 ? 1u : (uint32_t)r;
            }
        }
    }
    valid = valid && keep > 0;
    if (lane == 0) {
        a.qn[q] = valid ? (uint32_t)keep : 0u;
        uint32_t lo = 0, hi = 0;
        if (valid) {
            const double Mq = __dmul_rn(__dsub_rn(prec, kProtonDa), (double)z);
            lo = (uint32_t)mass_bound(a.mass, a.P, __dsub_rn(Mq, tol), false);
            hi = (uint32_t)mass_bound(a.mass, a.P, __dadd_rn(Mq, tol), true);
        }
        a.lo[q] = lo;
        a.hi[q] = hi;
    }
}

// work units per spectrum: its window split into pieces of >= seg_pids ids
__global__ void plan_kernel(const uint32_t* __restrict__ qn, const uint32_t* __restrict__ lo,
                            const uint32_t* __restrict__ hi, uint32_t n, uint32_t max_seg, uint32_t seg_pids,
                            uint32_t* __restrict__ nseg) {
    const uint32_t q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= n) return;
    uint32_t s = 0;
    if (qn[q] > 0 && hi[q] > lo[q]) {
        const uint32_t W = hi[q] - lo[q];
        s = (uint32_t)(((uint64_t)W + seg_pids - 1) / seg_pids);
        if (s > max_seg) s = max_seg;
    }
    nseg[q] = s;
}

// ---- unit order: longest first (the persistent CTAs take units in this
// order, so the short ones fill the end of the launch).  A unit's cost is
// estimated as its peptide range times the spectrum's retained peaks; units
// are bucketed by the cost's binary magnitude (a counting sort over 64
// buckets, descending), block histograms first so that the global atomics
// stay few.
constexpr int kOrderBuckets = 64;
constexpr uint32_t kOrderMinSpectra = 2048;   // smaller batches take their units in spectrum order

__device__ __forceinline__ int order_bucket(const uint32_t* qn, const uint32_t* lo, const uint32_t* hi,
                                            const uint64_t* seg_off, uint32_t q, uint32_t* ns) {
    *ns = (uint32_t)(seg_off[q + 1] - seg_off[q]);
    if (*ns == 0) return 0;
    const uint64_t W = hi[q] - lo[q];
    const uint64_t cost = ((W + *ns - 1) / *ns) * (uint64_t)(qn[q] ? qn[q] : 1) + 1;
    return __clzll((long long)cost);   // 0 for the costliest magnitudes: descending order
}

__global__ void order_count_kernel(const uint32_t* __restrict__ qn, const uint32_t* __restrict__ lo,
                                   const uint32_t* __restrict__ hi, const uint64_t* __restrict__ seg_off,
                                   uint32_t n, uint32_t* __restrict__ cnt) {
    __shared__ uint32_t bc[kOrderBuckets];
    for (int i = threadIdx.x; i < kOrderBuckets; i += blockDim.x) bc[i] = 0;
    __syncthreads();
    const uint32_t q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q < n) {
        uint32_t ns;
        const int b = order_bucket(qn, lo, hi, seg_off, q, &ns);
        if (ns) atomicAdd(&bc[b], ns);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < kOrderBuckets; i += blockDim.x)
        if (bc[i]) atomicAdd(&cnt[i], bc[i]);
}

// cnt[0..63] counts -> cnt[64..127] exclusive starts (one warp)
__global__ void order_scan_kernel(uint32_t* __restrict__ cnt) {
    const int lane = threadIdx.x;
    const uint32_t a = cnt[lane], b = cnt[32 + lane];
    uint32_t ia = a, ib = b;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t xa = __shfl_up_sync(0xffffffffu, ia, o), xb = __shfl_up_sync(0xffffffffu, ib, o);
        if (lane >= o) { ia += xa; ib += xb; }
    }
    const uint32_t tot_a = __shfl_sync(0xffffffffu, ia, 31);
    cnt[kOrderBuckets + lane] = ia - a;
    cnt[kOrderBuckets + 32 + lane] = tot_a + ib - b;
}

__global__ void order_scatter_kernel(const uint32_t* __restrict__ qn, const uint32_t* __restrict__ lo,
                                     const uint32_t* __restrict__ hi, const uint64_t* __restrict__ seg_off,
                                     uint32_t n, uint32_t* __restrict__ cursor, uint32_t* __restrict__ order,
                                     uint32_t* __restrict__ order_q) {
    __shared__ uint32_t bc[kOrderBuckets], bb[kOrderBuckets];
    for (int i = threadIdx.x; i < kOrderBuckets; i += blockDim.x) bc[i] = 0;
    __syncthreads();
    const uint32_t q = blockIdx.x * blockDim.x + threadIdx.x;
    uint32_t ns = 0, local = 0;
    int b = 0;
    if (q < n) {
        b = order_bucket(qn, lo, hi, seg_off, q, &ns);
        if (ns) local = atomicAdd(&bc[b], ns);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < kOrderBuckets; i += blockDim.x)
        if (bc[i]) bb[i] = atomicAdd(&cursor[i], bc[i]);
    __syncthreads();
    if (ns) {
        const uint32_t pos = bb[b] + local;
        const uint64_t u0 = seg_off[q];
        for (uint32_t s = 0; s < ns; ++s) {
            order[pos + s] = (uint32_t)(u0 + s);
            order_q[pos + s] = q;
        }
    }
}

#include "search_kernel.cuh"

// lower bound of pid key (pid << 1) in entry[a, b)
__device__ __forceinline__ uint64_t entry_lower_bound(const uint32_t* __restrict__ entry, uint64_t a, uint64_t b,
                                                      uint32_t pid) {
    const uint32_t key = pid << 1;
    while (a < b) {
        const uint64_t m = (a + b) >> 1;
        if (__ldg(entry + m) < key) a = m + 1; else b = m;
    }
    return a;
}

struct MergeArgs {
    const uint64_t* seg_off;
    const UnitTop* utop;
    const uint32_t* hist;
    uint32_t n, k;
    uint32_t q_base;          // query index written into the rows
    hicops_psm* out;
    uint32_t pid_stride, pid_base;   // row pid = list pid * pid_stride + pid_base ...
    const uint32_t* pid_map;         // ... or pid_map[list pid] when not NULL
    uint32_t ev_mode;                // HICOPS_EVALUE_* bits
};

__device__ __forceinline__ double warp_sum_f64(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// One warp per spectrum (kMergeWarps spectra per block): the top-k merge of
// the spectrum's unit lists, then the e-value fit (Supplementary Algorithm
// 4) over its histogram.  Lane l owns unit lists l and l + 32 (at most 64
// units, each sorted by (key desc, pid asc)); k rounds of a warp argmax
// over the list heads give the rows in rank order.  Lane l holds histogram
// bins 8l .. 8l + 7.
__global__ void __launch_bounds__(kMergeWarps * 32) merge_kernel(MergeArgs a) {
    __shared__ int64_t gsurv[kMergeWarps][kHistBins + 1];   // the fit's survival function G[0..256]
    const int lane = threadIdx.x & 31;
    const uint32_t q = blockIdx.x * kMergeWarps + (threadIdx.x >> 5);
    if (q >= a.n) return;
    int64_t* const G = gsurv[threadIdx.x >> 5];
    const uint32_t k = a.k;
    const uint64_t u0 = a.seg_off[q];
    const int nseg = (int)(a.seg_off[q + 1] - u0);
    const UnitTop* lists = a.utop + u0 * k;
    uint32_t h0 = 0, h1 = 0;   // heads of lists lane and lane + 32
    UnitTop row;               // row `lane` of the result
    row.key = INT64_MIN;
    row.pid = 0xffffffffu;
    row.packed = 0u;
    for (uint32_t r = 0; r < k; ++r) {
        int64_t bk = INT64_MIN;
        uint32_t bp = 0xffffffffu, bpk = 0u;
        int which = -1;
        if (lane < nseg && h0 < k) {
            const UnitTop t = lists[(uint64_t)lane * k + h0];
            if (t.pid != 0xffffffffu) { bk = t.key; bp = t.pid; bpk = t.packed; which = 0; }
        }
        if (lane + 32 < nseg && h1 < k) {
            const UnitTop t = lists[(uint64_t)(lane + 32) * k + h1];
            if (t.pid != 0xffffffffu && better(t.key, t.pid, bk, bp)) { bk = t.key; bp = t.pid; bpk = t.packed; which = 1; }
        }
        int64_t wk = bk;
        uint32_t wp = bp, wpk = bpk;
        int wl = lane;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const int64_t ok = __shfl_xor_sync(0xffffffffu, wk, o);
            const uint32_t op = __shfl_xor_sync(0xffffffffu, wp, o);
            const uint32_t opk = __shfl_xor_sync(0xffffffffu, wpk, o);
            const int ol = __shfl_xor_sync(0xffffffffu, wl, o);
            if (better(ok, op, wk, wp) || (ok == wk && op == wp && ol < wl)) { wk = ok; wp = op; wpk = opk; wl = ol; }
        }
        if (wp != 0xffffffffu && lane == wl) { if (which == 0) ++h0; else ++h1; }
        if ((uint32_t)lane == r) { row.key = wk; row.pid = wp; row.packed = wpk; }
    }
    // the histogram, bins 8 lane .. 8 lane + 7 of this lane
    const uint32_t* hq = a.hist + (uint64_t)q * kHistBins + 8 * lane;   // caller's buffer: 4-byte aligned only
    uint32_t v[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) v[i] = hq[i];
    uint32_t nl = 0;
#pragma unroll
    for (int i = 0; i < 8; ++i) nl += v[i];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) nl += __shfl_xor_sync(0xffffffffu, nl, o);
    const double N = (double)nl;
    // the distribution the fit sees (R16): the histogram, or 35 times its
    // 5-point quadratic Savitzky-Golay smoothing (zero outside the bins);
    // integers, so every sum and comparison below is exact
    int64_t g[8];
    {
        const uint32_t l2 = __shfl_up_sync(0xffffffffu, v[6], 1), l1 = __shfl_up_sync(0xffffffffu, v[7], 1);
        const uint32_t r1 = __shfl_down_sync(0xffffffffu, v[0], 1), r2 = __shfl_down_sync(0xffffffffu, v[1], 1);
        int64_t e[12];
        e[0] = lane > 0 ? l2 : 0;
        e[1] = lane > 0 ? l1 : 0;
#pragma unroll
        for (int i = 0; i < 8; ++i) e[2 + i] = v[i];
        e[10] = lane < 31 ? r1 : 0;
        e[11] = lane < 31 ? r2 : 0;
        const bool smooth = (a.ev_mode & HICOPS_EVALUE_SMOOTH) != 0u;
#pragma unroll
        for (int i = 0; i < 8; ++i)
            g[i] = smooth ? -3 * e[i] + 12 * e[i + 1] + 17 * e[i + 2] + 12 * e[i + 3] - 3 * e[i + 4] : e[i + 2];
    }
    // survival G[j] = sum of g[i >= j]: within the lane, then over the lanes above
    int64_t loc[8];
    int64_t run = 0;
#pragma unroll
    for (int i = 7; i >= 0; --i) { run += g[i]; loc[i] = run; }
    int64_t above = run;   // inclusive suffix over lanes >= lane
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int64_t y = __shfl_down_sync(0xffffffffu, above, o);
        if (lane + o < 32) above += y;
    }
    const int64_t G0 = __shfl_sync(0xffffffffu, above, 0);
    above -= run;           // lanes > lane
    // G[j] in shared memory, so that the fit's points (a few bins next to
    // one another) are spread one a lane and its FP64 logarithms run once
    // for the warp rather than once per bin of a lane
#pragma unroll
    for (int i = 0; i < 8; ++i) G[8 * lane + i] = loc[i] + above;
    if (lane == 0) G[kHistBins] = 0;
    __syncwarp();
    const double dG0 = (double)G0;
    const int64_t key0 = __shfl_sync(0xffffffffu, row.key, 0);
    const uint32_t pid0 = __shfl_sync(0xffffffffu, row.pid, 0);
    const bool have_top = pid0 != 0xffffffffu;
    const bool weibull = (a.ev_mode & HICOPS_EVALUE_LOG_WEIBULL) != 0u;
    double cn = 0, sx = 0, sy = 0, sxx = 0, sxy = 0;
    if (weibull) {
        // R17: least squares of -ln(-ln F_j) on x = j + 1, F_j = 1 - G[j+1] / G[0],
        // over the bins with 0 < F_j < 1
        for (int j = lane; j < (int)kHistBins && have_top; j += 32) {
            const int64_t gn = G[j + 1];
            if (gn > 0 && gn < G0) {
                const double x = (double)(j + 1);
                const double y = -log(-log1p(-((double)gn / dG0)));
                cn += 1.0;
                sx += x;
                sy += y;
                sxx += x * x;
                sxy += x * y;
            }
        }
    } else {
        // R12 on g: the mode (largest g, lowest bin on ties), then the line
        // through (j, log10(G[j] / G[0])) for j in [mode + 1, jtop - 1], G[j] > 0
        int64_t bv = g[0];
        int bj = 8 * lane;
#pragma unroll
        for (int i = 1; i < 8; ++i)
            if (g[i] > bv) { bv = g[i]; bj = 8 * lane + i; }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const int64_t ov = __shfl_xor_sync(0xffffffffu, bv, o);
            const int oj = __shfl_xor_sync(0xffffffffu, bj, o);
            if (ov > bv || (ov == bv && oj < bj)) { bv = ov; bj = oj; }
        }
        const int mode = bj;
        int64_t jtop = 0;
        if (have_top) { jtop = key0 >> 31; if (jtop > 255) jtop = 255; }
        for (int j = mode + 1 + lane; j <= (int)jtop - 1 && have_top; j += 32) {
            const int64_t gj = G[j];
            if (gj > 0) {
                const double x = (double)j;
                const double y = log10((double)gj / dG0);
                cn += 1.0;
                sx += x;
                sy += y;
                sxx += x * x;
                sxy += x * y;
            }
        }
    }
    cn = warp_sum_f64(cn);
    sx = warp_sum_f64(sx);
    sy = warp_sum_f64(sy);
    sxx = warp_sum_f64(sxx);
    sxy = warp_sum_f64(sxy);
    bool fit = cn >= 3.0;
    double wfit = 0.0, bfit = 0.0;
    if (fit) {
        const double den = cn * sxx - sx * sx;
        wfit = (cn * sxy - sx * sy) / den;
        bfit = (sy - wfit * sx) / cn;
        if (weibull) fit = wfit > 0.0;
    }
    if ((uint32_t)lane < k) {
        hicops_psm o;
        o.query = a.q_base + q;
        o.reserved = 0;
        if (row.pid != 0xffffffffu) {
            o.pid = a.pid_map ? a.pid_map[row.pid] : row.pid * a.pid_stride + a.pid_base;
            o.nb = (uint8_t)(row.packed >> kNbShift);
            o.ny = (uint8_t)((row.packed >> kNyShift) & 63u);
            o.key = row.key;
            o.hyperscore = (float)((double)row.key * 0x1p-32);
            const double x = (double)row.key * 0x1p-31;
            if (!fit) o.evalue = N;
            else if (weibull) o.evalue = N * -expm1(-exp(-(wfit * x + bfit)));   // N * P(score >= x)
            else o.evalue = N * exp10(wfit * x + bfit);
        } else {
            o.pid = 0xffffffffu;
            o.nb = o.ny = 0;
            o.key = INT64_MIN;
            o.hyperscore = 0.0f;
            o.evalue = INFINITY;
        }
        a.out[(uint64_t)q * k + lane] = o;
    }
}

// Fragment tolerance of t bins (R15): replaces spectrum q's retained peaks
// (distinct bins in any order) by the union of their windows [b - t, b + t]
// cut to [0, n_bins), ascending, each bin with the largest iq of the peaks
// covering it.  One warp per spectrum, in place: the peaks are read into
// shared memory and sorted by bin first.  Peak i emits the bins of its
// window above the previous peak's window, so no bin is emitted twice, and
// only peaks j >= i can cover them.
constexpr int kExpWarps = 4;

struct ExpandArgs {
    uint32_t* qbin;
    uint32_t* qiq;
    uint32_t* qn;
    uint32_t n, stride, t, n_bins;
};

__global__ void __launch_bounds__(kExpWarps * 32) expand_kernel(ExpandArgs a) {
    __shared__ uint64_t keys_all[kExpWarps][kMaxTopN];
    const int lane = threadIdx.x & 31, wi = threadIdx.x >> 5;
    const uint32_t q = blockIdx.x * kExpWarps + wi;
    if (q >= a.n) return;   // warp-uniform
    const uint32_t cnt = a.qn[q];
    if (cnt == 0) return;
    uint64_t* keys = keys_all[wi];
    uint32_t* qb = a.qbin + (uint64_t)q * a.stride;
    uint32_t* qi = a.qiq + (uint64_t)q * a.stride;
    const int npow = next_pow2((int)cnt);
    for (int i = lane; i < npow; i += 32) keys[i] = i < (int)cnt ? ((uint64_t)qb[i] << 32) | qi[i] : ~0ull;
    __syncwarp();
    warp_bitonic_sort_u64(keys, npow, lane);
    const uint32_t t = a.t;
    uint32_t base = 0;
    for (uint32_t i0 = 0; i0 < cnt; i0 += 32) {   // warp-uniform trip count
        const uint32_t i = i0 + lane;
        uint32_t lo = 0, hi = 0;   // bins [lo, hi) emitted by peak i
        if (i < cnt) {
            const uint32_t b = (uint32_t)(keys[i] >> 32);
            lo = b > t ? b - t : 0u;
            if (i > 0) lo = max(lo, (uint32_t)(keys[i - 1] >> 32) + t + 1u);
            hi = min(b + t + 1u, a.n_bins);
            if (hi < lo) hi = lo;
        }
        const uint32_t len = hi - lo;
        uint32_t incl = len;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t x = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += x;
        }
        const uint32_t pos = base + incl - len;
        base += __shfl_sync(0xffffffffu, incl, 31);
        for (uint32_t x = lo; x < hi; ++x) {
            uint32_t best = 0;
            for (uint32_t j = i; j < cnt; ++j) {
                const uint64_t kj = keys[j];
                if ((uint32_t)(kj >> 32) > x + t) break;
                best = max(best, (uint32_t)kj);
            }
            qb[pos + (x - lo)] = x;
            qi[pos + (x - lo)] = best;
        }
    }
    if (lane == 0) a.qn[q] = base;
}

// per spectrum: sum over retained peaks of the bucket entries inside [lo, hi)
__global__ void work_kernel(const uint32_t* __restrict__ qbin, const uint32_t* __restrict__ qn,
                            const uint32_t* __restrict__ lo, const uint32_t* __restrict__ hi, uint32_t topn,
                            const uint64_t* __restrict__ off, const uint32_t* __restrict__ entry,
                            uint64_t* __restrict__ hits) {
    const uint32_t q = blockIdx.x;
    uint64_t h = 0;
    for (uint32_t t = threadIdx.x; t < qn[q]; t += blockDim.x) {
        const uint32_t bin = qbin[(uint64_t)q * topn + t];
        const uint64_t b0 = off[bin], b1 = off[bin + 1];
        const uint64_t c = entry_lower_bound(entry, b0, b1, lo[q]);
        const uint64_t e = entry_lower_bound(entry, c, b1, hi[q]);
        h += e - c;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) h += __shfl_xor_sync(0xffffffffu, h, o);
    __shared__ uint64_t red[8];
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = h;
    __syncthreads();
    if (threadIdx.x == 0) {
        uint64_t t = 0;
        for (int w = 0; w < (int)(blockDim.x / 32); ++w) t += red[w];
        hits[q] = t;
    }
}

}  // namespace
}  // namespace hicops
