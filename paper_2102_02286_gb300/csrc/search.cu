// Superstep 3 search on the GPU (paper: "Superstep 3: Partial Database
// Peptide Search", Eq. 4; Supplementary Algorithm 3) and the superstep-4
// e-value (Supplementary Algorithm 4).
//
//   prep_kernel    R sub-task's "minimal computations": filter, bin, merge,
//                  keep the B most intense peaks, quantise; precursor mass and
//                  filter_1 (binary search of the mass-sorted database).
//   search_kernel  filter_2 + score + heap: per (spectrum, peptide-id
//                  segment) work unit, stream every retained peak's bucket
//                  restricted to the segment, accumulate (nb, ny, S) per
//                  peptide in shared memory one chunk of peptide ids at a
//                  time, keep candidates with nb + ny >= min_shared, rank them
//                  by the exact hyperscore key, keep a top-k and the score
//                  histogram.  Persistent CTAs pull units from a device
//                  counter.
//   merge_kernel   merge the per-segment top-k lists of each spectrum, then
//                  the survival-tail e-value (FP64).
#include <atomic>
#include <cfloat>
#include <cmath>

#include "dev_common.cuh"

namespace hicops {
namespace {

constexpr int kPrepThreads = 256;
constexpr int kSearchThreads = 256;
constexpr int kChunk = 16384;             // peptide ids per shared-memory counter chunk
constexpr int kMinSegPids = kChunk;       // smallest segment of a split window
constexpr int kMaxSegs = 64;              // most segments a window is split into
constexpr int kMergeThreads = 256;
constexpr uint16_t kNoIdx = 0xffff;       // padding slot of the merge sort

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
    uint32_t topn;
    double w, mz_lo, mz_hi, scale;
    const double* mass;
    uint64_t P;
    uint32_t* qbin;     // [n * topn]
    uint32_t* qiq;      // [n * topn]
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

__global__ void __launch_bounds__(kPrepThreads) prep_kernel(PrepArgs a) {
    __shared__ uint64_t keys[HICOPS_MAX_PEAKS];
    __shared__ int s_nrep;
    const uint32_t q = blockIdx.x;
    const uint64_t p0 = a.peak_off[q], p1 = a.peak_off[q + 1];
    const uint64_t cnt = p1 >= p0 ? p1 - p0 : 0;
    const double prec = a.prec_mz[q];
    const double tol = a.tol[q];
    const uint32_t z = a.charge[q];
    bool valid = cnt <= HICOPS_MAX_PEAKS && p1 >= p0 && z > 0 && isfinite(prec) && isfinite(tol) && tol >= 0.0;
    int keep = 0;
    if (valid && cnt > 0) {
        const int npow = next_pow2((int)cnt);
        // key = bin << 32 | intensity bits (positive finite floats order as integers)
        for (int i = threadIdx.x; i < npow; i += blockDim.x) {
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
        if (threadIdx.x == 0) s_nrep = 0;
        __syncthreads();
        bitonic_sort_u64(keys, npow);
        // one representative per bin: the last (most intense) of each run
        uint64_t rep[HICOPS_MAX_PEAKS / kPrepThreads];
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
        if (keep > 0) {
            const double Imax = (double)__uint_as_float(~(uint32_t)(keys[0] >> 32));
            for (int t = threadIdx.x; t < keep; t += blockDim.x) {
                const uint64_t k = keys[t];
                const double I = (double)__uint_as_float(~(uint32_t)(k >> 32));
                const double r = floor(__dmul_rn(I, a.scale) / Imax);
                a.qbin[(uint64_t)q * a.topn + t] = (uint32_t)k;
                a.qiq[(uint64_t)q * a.topn + t] = r < 1.0 ? 1u : (uint32_t)r;
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

// segments per spectrum window
__global__ void plan_kernel(const uint32_t* __restrict__ qn, const uint32_t* __restrict__ lo,
                            const uint32_t* __restrict__ hi, uint32_t n, uint32_t max_seg,
                            uint32_t* __restrict__ nseg) {
    const uint32_t q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= n) return;
    uint32_t s = 0;
    if (qn[q] > 0 && hi[q] > lo[q]) {
        const uint32_t W = hi[q] - lo[q];
        s = (W + kMinSegPids - 1) / kMinSegPids;
        if (s > max_seg) s = max_seg;
    }
    nseg[q] = s;
}

struct SearchArgs {
    const uint32_t* qbin;
    const uint32_t* qiq;
    const uint32_t* qn;
    const uint32_t* lo;
    const uint32_t* hi;
    const uint64_t* seg_off;    // [n + 1] first unit of each spectrum
    uint32_t n;
    uint32_t topn;
    const uint64_t* off;        // bucket offsets
    const uint32_t* entry;      // pid << 1 | isY
    const int64_t* lf;
    const int64_t* ls;
    uint32_t min_shared;
    uint32_t k;
    UnitTop* utop;              // [units * k]
    uint32_t* hist;             // [n * 256]
    uint32_t* nscored;          // [n]
    unsigned long long* work;   // unit counter
};

template <int KMAX>
struct TopK {
    int64_t key[KMAX];
    uint32_t pid[KMAX];
    uint32_t pk[KMAX];
    int n;
    __device__ __forceinline__ void init() {
        n = 0;
#pragma unroll
        for (int i = 0; i < KMAX; ++i) { key[i] = INT64_MIN; pid[i] = 0xffffffffu; pk[i] = 0; }
    }
    // (key desc, pid asc); slot k-1 is the current worst of a full list
    __device__ __forceinline__ void insert(int64_t kk, uint32_t p, uint32_t packed, int k) {
        // position: first slot worse than (kk, p)
        int pos = 0;
#pragma unroll
        for (int i = 0; i < KMAX; ++i)
            if (i < n && (key[i] > kk || (key[i] == kk && pid[i] < p))) pos = i + 1;
        if (pos >= k) return;
#pragma unroll
        for (int i = KMAX - 1; i > 0; --i) {
            if (i > pos) { key[i] = key[i - 1]; pid[i] = pid[i - 1]; pk[i] = pk[i - 1]; }
        }
#pragma unroll
        for (int i = 0; i < KMAX; ++i)
            if (i == pos) { key[i] = kk; pid[i] = p; pk[i] = packed; }
        if (n < k) ++n;
    }
    __device__ __forceinline__ void pop() {
#pragma unroll
        for (int i = 0; i < KMAX - 1; ++i) { key[i] = key[i + 1]; pid[i] = pid[i + 1]; pk[i] = pk[i + 1]; }
        key[KMAX - 1] = INT64_MIN;
        pid[KMAX - 1] = 0xffffffffu;
        --n;
    }
};

__device__ __forceinline__ bool better(int64_t ka, uint32_t pa, int64_t kb, uint32_t pb) {
    return ka > kb || (ka == kb && pa < pb);
}

struct SearchShared {
    uint32_t pbin[kMaxTopN];
    uint32_t pinc[kMaxTopN];     // counter increment without the b/y count bits: iq
    uint32_t cur[kMaxTopN];
    uint32_t end[kMaxTopN];
    uint32_t longp[kMaxTopN];
    uint32_t hist[kHistBins];
    int64_t lf[kMaxLen + 1];
    int64_t wkey[kSearchThreads / 32];
    uint32_t wpid[kSearchThreads / 32];
    uint32_t wpk[kSearchThreads / 32];
    int nlong;
    uint64_t unit;
    uint32_t q, np;
    uint32_t seg_lo, seg_hi;
};

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

template <int KMAX>
__global__ void __launch_bounds__(kSearchThreads) search_kernel(SearchArgs a) {
    extern __shared__ __align__(16) uint32_t cnt[];   // kChunk counters
    __shared__ SearchShared sh;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    constexpr int nwarps = kSearchThreads / 32;
    for (int i = tid; i < kChunk; i += kSearchThreads) cnt[i] = 0;
    for (int i = tid; i < kHistBins; i += kSearchThreads) sh.hist[i] = 0;
    for (int i = tid; i <= (int)kMaxLen; i += kSearchThreads) sh.lf[i] = a.lf[i];
    const uint64_t total_units = a.seg_off[a.n];
    const int k = (int)a.k;
    __syncthreads();
    for (;;) {
        if (tid == 0) {
            const uint64_t u = atomicAdd(a.work, 1ull);
            sh.unit = u;
            if (u < total_units) {
                // spectrum owning unit u: last q with seg_off[q] <= u
                uint32_t lo_q = 0, hi_q = a.n;
                while (hi_q - lo_q > 1) {
                    const uint32_t m = (lo_q + hi_q) >> 1;
                    if (a.seg_off[m] <= u) lo_q = m; else hi_q = m;
                }
                const uint32_t q = lo_q;
                const uint32_t s = (uint32_t)(u - a.seg_off[q]);
                const uint32_t ns = (uint32_t)(a.seg_off[q + 1] - a.seg_off[q]);
                const uint32_t W = a.hi[q] - a.lo[q];
                const uint32_t len = (W + ns - 1) / ns;
                sh.q = q;
                sh.np = a.qn[q];
                sh.seg_lo = a.lo[q] + s * len;
                sh.seg_hi = min(a.hi[q], sh.seg_lo + len);
            }
        }
        __syncthreads();
        const uint64_t u = sh.unit;
        if (u >= total_units) break;
        const uint32_t q = sh.q, np = sh.np, seg_lo = sh.seg_lo, seg_hi = sh.seg_hi;
        // peaks of spectrum q and their bucket ranges inside the segment
        for (uint32_t t = tid; t < np; t += kSearchThreads) {
            const uint32_t bin = a.qbin[(uint64_t)q * a.topn + t];
            const uint64_t b0 = a.off[bin], b1 = a.off[bin + 1];
            const uint64_t c = entry_lower_bound(a.entry, b0, b1, seg_lo);
            const uint64_t e = entry_lower_bound(a.entry, c, b1, seg_hi);
            sh.pbin[t] = bin;
            sh.pinc[t] = a.qiq[(uint64_t)q * a.topn + t];
            // entries of one bucket fit in 32 bits relative to the bucket start
            sh.cur[t] = (uint32_t)(c - b0);
            sh.end[t] = (uint32_t)(e - b0);
        }
        TopK<KMAX> top;
        top.init();
        __syncthreads();
        for (uint32_t c0 = seg_lo; c0 < seg_hi; c0 += kChunk) {
            const uint32_t c1 = min(seg_hi, c0 + (uint32_t)kChunk);
            if (tid == 0) sh.nlong = 0;
            __syncthreads();
            // phase A: every peak takes up to 4 entries of its run
            for (uint32_t t = tid; t < np; t += kSearchThreads) {
                const uint64_t base = a.off[sh.pbin[t]];
                uint32_t idx = sh.cur[t];
                const uint32_t e = sh.end[t];
                uint32_t v[4];
#pragma unroll
                for (int i = 0; i < 4; ++i) v[i] = (idx + i < e) ? __ldg(a.entry + base + idx + i) : 0xffffffffu;
                const uint32_t inc = sh.pinc[t];
                int taken = 0;
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    if (taken == i && (v[i] >> 1) < c1) {
                        atomicAdd(&cnt[(v[i] >> 1) - c0], inc + ((v[i] & 1u) ? (1u << kNyShift) : (1u << kNbShift)));
                        ++taken;
                    }
                }
                idx += taken;
                sh.cur[t] = idx;
                if (taken == 4 && idx < e) sh.longp[atomicAdd(&sh.nlong, 1)] = t;
            }
            __syncthreads();
            // phase B: long runs, one warp per peak, 128 entries in flight per step
            const int nlong = sh.nlong;
            for (int li = warp; li < nlong; li += nwarps) {
                const uint32_t t = sh.longp[li];
                const uint64_t base = a.off[sh.pbin[t]];
                uint32_t idx = sh.cur[t];
                const uint32_t e = sh.end[t];
                const uint32_t inc = sh.pinc[t];
                for (;;) {
                    uint32_t v[4];
#pragma unroll
                    for (int r = 0; r < 4; ++r) {
                        const uint32_t j = idx + r * 32 + lane;
                        v[r] = j < e ? __ldg(a.entry + base + j) : 0xffffffffu;
                    }
                    uint32_t done = 0;
                    bool stop = false;
#pragma unroll
                    for (int r = 0; r < 4; ++r) {
                        if (stop) break;
                        const bool ok = (v[r] >> 1) < c1;
                        const unsigned bal = __ballot_sync(0xffffffffu, ok);
                        if (ok) atomicAdd(&cnt[(v[r] >> 1) - c0], inc + ((v[r] & 1u) ? (1u << kNyShift) : (1u << kNbShift)));
                        done += __popc(bal);
                        if (bal != 0xffffffffu) stop = true;
                    }
                    idx += done;
                    if (stop) break;
                }
                if (lane == 0) sh.cur[t] = idx;
            }
            __syncthreads();
            // epilogue: filter, score, histogram, top-k; clear the counters
            const uint32_t span = c1 - c0;
            for (uint32_t i4 = tid * 4; i4 < span; i4 += kSearchThreads * 4) {
                uint4 c4 = *reinterpret_cast<uint4*>(&cnt[i4]);
                if ((c4.x | c4.y | c4.z | c4.w) == 0) continue;
                *reinterpret_cast<uint4*>(&cnt[i4]) = make_uint4(0, 0, 0, 0);
                const uint32_t cv[4] = {c4.x, c4.y, c4.z, c4.w};
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    const uint32_t c = cv[j];
                    const uint32_t nb = c >> kNbShift, ny = (c >> kNyShift) & 63u;
                    if (c != 0 && nb + ny >= a.min_shared) {
                        const uint32_t S = c & kSMask;
                        const int64_t K = sh.lf[nb] + sh.lf[ny] + __ldg(a.ls + S);
                        const int64_t hb = K >> 31;
                        atomicAdd(&sh.hist[hb > 255 ? 255 : (hb < 0 ? 0 : hb)], 1u);
                        top.insert(K, c0 + i4 + j, c, k);
                    }
                }
            }
            __syncthreads();
        }
        // block top-k: k rounds of block-wide argmax over the thread heads
        for (int r = 0; r < k; ++r) {
            int64_t bk = top.n > 0 ? top.key[0] : INT64_MIN;
            uint32_t bp = top.n > 0 ? top.pid[0] : 0xffffffffu;
            uint32_t bpk = top.n > 0 ? top.pk[0] : 0u;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                const int64_t ok = __shfl_xor_sync(0xffffffffu, bk, o);
                const uint32_t op = __shfl_xor_sync(0xffffffffu, bp, o);
                const uint32_t opk = __shfl_xor_sync(0xffffffffu, bpk, o);
                if (better(ok, op, bk, bp)) { bk = ok; bp = op; bpk = opk; }
            }
            if (lane == 0) { sh.wkey[warp] = bk; sh.wpid[warp] = bp; sh.wpk[warp] = bpk; }
            __syncthreads();
            bk = sh.wkey[0]; bp = sh.wpid[0]; bpk = sh.wpk[0];
            for (int w = 1; w < nwarps; ++w)
                if (better(sh.wkey[w], sh.wpid[w], bk, bp)) { bk = sh.wkey[w]; bp = sh.wpid[w]; bpk = sh.wpk[w]; }
            if (top.n > 0 && top.pid[0] == bp && top.key[0] == bk && bp != 0xffffffffu) top.pop();
            if (tid == 0) {
                UnitTop o;
                o.key = bk;
                o.pid = bp;
                o.packed = bpk;
                a.utop[u * k + r] = o;
            }
            __syncthreads();
        }
        // histogram of this unit into the spectrum's histogram
        uint32_t mine = 0;
        for (int j = tid; j < (int)kHistBins; j += kSearchThreads) {
            const uint32_t h = sh.hist[j];
            if (h) { atomicAdd(&a.hist[(uint64_t)q * kHistBins + j], h); mine += h; sh.hist[j] = 0; }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) mine += __shfl_xor_sync(0xffffffffu, mine, o);
        if (lane == 0 && mine) atomicAdd(&a.nscored[q], mine);
        __syncthreads();
    }
}

struct MergeArgs {
    const uint64_t* seg_off;
    const UnitTop* utop;
    const uint32_t* hist;
    uint32_t n, k;
    uint32_t q_base;          // query index written into the rows
    hicops_psm* out;
};

__device__ __forceinline__ double block_sum(double v, double* red) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) red[w] = v;
    __syncthreads();
    double t = 0;
    for (int i = 0; i < (int)(blockDim.x / 32); ++i) t += red[i];
    return t;
}

// one block per spectrum: merge the segment lists, then the e-value fit
__global__ void __launch_bounds__(kMergeThreads) merge_kernel(MergeArgs a) {
    __shared__ UnitTop buf[kMaxSegs * kMaxTopK];
    __shared__ uint16_t sk[kMaxSegs * kMaxTopK];
    __shared__ uint32_t suf[kHistBins];
    __shared__ double red[kMergeThreads / 32];
    __shared__ uint32_t s_mode;
    const uint32_t q = blockIdx.x;
    const uint32_t k = a.k;
    const uint64_t u0 = a.seg_off[q], u1 = a.seg_off[q + 1];
    const int nseg = (int)(u1 - u0);
    const int m = nseg * (int)k;
    // sort (key desc, pid asc) by sorting an index-tagged 64-bit rank
    const int npow = next_pow2(m > 0 ? m : 1);
    for (int i = threadIdx.x; i < npow; i += blockDim.x) {
        if (i < m) {
            buf[i] = a.utop[u0 * k + i];
            sk[i] = (uint16_t)i;
        } else {
            sk[i] = kNoIdx;
        }
    }
    __syncthreads();
    // odd-even by comparator over buf via index sort (bitonic on indices)
    for (int kk = 2; kk <= npow; kk <<= 1) {
        for (int j = kk >> 1; j > 0; j >>= 1) {
            for (int i = threadIdx.x; i < npow; i += blockDim.x) {
                const int ixj = i ^ j;
                if (ixj > i) {
                    const uint16_t x = sk[i], y = sk[ixj];
                    // "x after y" in (key desc, pid asc) order; padding last
                    bool x_after;
                    if (x == kNoIdx) x_after = (y != kNoIdx);
                    else if (y == kNoIdx) x_after = false;
                    else x_after = better(buf[y].key, buf[y].pid, buf[x].key, buf[x].pid);
                    const bool up = (i & kk) == 0;
                    if (x_after == up) { sk[i] = y; sk[ixj] = x; }
                }
            }
            __syncthreads();
        }
    }
    // survival function and fit over the histogram
    const uint32_t* h = a.hist + (uint64_t)q * kHistBins;
    const int j = threadIdx.x;   // one bin per thread (256 threads)
    const uint32_t hv = h[j];
    // suffix sums
    suf[j] = hv;
    __syncthreads();
    for (int o = 1; o < (int)kHistBins; o <<= 1) {
        const uint32_t add = (j + o < (int)kHistBins) ? suf[j + o] : 0u;
        __syncthreads();
        suf[j] += add;
        __syncthreads();
    }
    // mode: highest count, lowest bin on ties
    if (j == 0) s_mode = 0;
    __syncthreads();
    {
        const uint64_t v = ((uint64_t)hv << 32) | (uint32_t)(255 - j);
        uint64_t best = v;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const uint64_t ov = __shfl_xor_sync(0xffffffffu, best, o);
            if (ov > best) best = ov;
        }
        __shared__ uint64_t wbest[kMergeThreads / 32];
        if ((j & 31) == 0) wbest[j >> 5] = best;
        __syncthreads();
        if (j == 0) {
            uint64_t b = wbest[0];
            for (int w = 1; w < kMergeThreads / 32; ++w) if (wbest[w] > b) b = wbest[w];
            s_mode = 255 - (uint32_t)(b & 0xffffffffu);
        }
        __syncthreads();
    }
    const double N = (double)suf[0];
    const bool have_top = m > 0 && sk[0] != kNoIdx && buf[sk[0]].pid != 0xffffffffu;
    int64_t jtop = 0;
    if (have_top) { jtop = buf[sk[0]].key >> 31; if (jtop > 255) jtop = 255; }
    const bool pt = have_top && j >= (int)s_mode + 1 && j <= jtop - 1 && suf[j] > 0;
    const double x = (double)j;
    const double y = pt ? log10((double)suf[j] / N) : 0.0;
    const double cn = block_sum(pt ? 1.0 : 0.0, red);
    const double sx = block_sum(pt ? x : 0.0, red);
    const double sy = block_sum(pt ? y : 0.0, red);
    const double sxx = block_sum(pt ? x * x : 0.0, red);
    const double sxy = block_sum(pt ? x * y : 0.0, red);
    const bool fit = cn >= 3.0;
    double wfit = 0.0, bfit = 0.0;
    if (fit) {
        const double den = cn * sxx - sx * sx;
        wfit = (cn * sxy - sx * sy) / den;
        bfit = (sy - wfit * sx) / cn;
    }
    for (uint32_t r = threadIdx.x; r < k; r += blockDim.x) {
        hicops_psm o;
        o.query = a.q_base + q;
        o.reserved = 0;
        const bool real = (int)r < m && sk[r] != kNoIdx && buf[sk[r]].pid != 0xffffffffu;
        if (real) {
            const UnitTop t = buf[sk[r]];
            o.pid = t.pid;
            o.nb = (uint8_t)(t.packed >> kNbShift);
            o.ny = (uint8_t)((t.packed >> kNyShift) & 63u);
            o.key = t.key;
            o.hyperscore = (float)((double)t.key * 0x1p-32);
            if (fit) o.evalue = N * exp10(wfit * ((double)t.key * 0x1p-31) + bfit);
            else o.evalue = N;
        } else {
            o.pid = 0xffffffffu;
            o.nb = o.ny = 0;
            o.key = INT64_MIN;
            o.hyperscore = 0.0f;
            o.evalue = INFINITY;
        }
        a.out[(uint64_t)q * k + r] = o;
    }
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

// ---------------------------------------------------------------- host side

struct DevBatch {
    const uint64_t* peak_off;
    const float* mz;
    const float* inten;
    const double* prec;
    const uint8_t* z;
    const double* tol;
};

// stream-ordered scratch; freed on every exit path
struct Scratch {
    cudaStream_t s;
    std::vector<void*> ptrs;
    explicit Scratch(cudaStream_t st) : s(st) {}
    template <class T>
    cudaError_t get(T** p, uint64_t n) {
        cudaError_t e = cudaMallocAsync((void**)p, sizeof(T) * (n ? n : 1), s);
        if (e == cudaSuccess) ptrs.push_back(*p);
        return e;
    }
    ~Scratch() { for (void* p : ptrs) cudaFreeAsync(p, s); }
};

hicops_status check_batch(const hicops_index* idx, const hicops_batch* b) {
    if (!idx || !b) { set_error("NULL argument"); return HICOPS_EINVAL; }
    if (!idx->dev.ready) { set_error("index has no device part (call hicops_index_upload)"); return HICOPS_EINVAL; }
    if (b->n && (!b->peak_off || !b->prec_mz || !b->charge || !b->prec_tol_da)) {
        set_error("batch pointers are NULL");
        return HICOPS_EINVAL;
    }
    int dev = -1;
    HC_CUDA(cudaGetDevice(&dev));
    if (dev != idx->dev.device) { set_error("current device %d is not the index's device %d", dev, idx->dev.device); return HICOPS_EINVAL; }
    return HICOPS_OK;
}

// Inputs on the device (copied from the host when on_device = 0).
hicops_status stage_inputs(const hicops_batch* b, Scratch& sc, DevBatch& d, uint64_t* npk_out) {
    const cudaStream_t s = sc.s;
    if (b->on_device) {
        d = DevBatch{b->peak_off, b->mz, b->intensity, b->prec_mz, b->charge, b->prec_tol_da};
        *npk_out = 0;
        return HICOPS_OK;
    }
    const uint64_t npk = b->peak_off[b->n];
    if (npk && (!b->mz || !b->intensity)) { set_error("peak arrays are NULL"); return HICOPS_EINVAL; }
    uint64_t* po; float *mz, *it; double *pr, *tl; uint8_t* z;
    HC_CUDA(sc.get(&po, b->n + 1));
    HC_CUDA(sc.get(&mz, npk));
    HC_CUDA(sc.get(&it, npk));
    HC_CUDA(sc.get(&pr, b->n));
    HC_CUDA(sc.get(&tl, b->n));
    HC_CUDA(sc.get(&z, b->n));
    HC_CUDA(cudaMemcpyAsync(po, b->peak_off, sizeof(uint64_t) * (b->n + 1), cudaMemcpyHostToDevice, s));
    if (npk) {
        HC_CUDA(cudaMemcpyAsync(mz, b->mz, sizeof(float) * npk, cudaMemcpyHostToDevice, s));
        HC_CUDA(cudaMemcpyAsync(it, b->intensity, sizeof(float) * npk, cudaMemcpyHostToDevice, s));
    }
    HC_CUDA(cudaMemcpyAsync(pr, b->prec_mz, sizeof(double) * b->n, cudaMemcpyHostToDevice, s));
    HC_CUDA(cudaMemcpyAsync(tl, b->prec_tol_da, sizeof(double) * b->n, cudaMemcpyHostToDevice, s));
    HC_CUDA(cudaMemcpyAsync(z, b->charge, sizeof(uint8_t) * b->n, cudaMemcpyHostToDevice, s));
    d = DevBatch{po, mz, it, pr, z, tl};
    *npk_out = npk;
    return HICOPS_OK;
}

hicops_status run_prep(hicops_index* idx, const DevBatch& d, uint32_t n, Scratch& sc, uint32_t** qbin,
                       uint32_t** qiq, uint32_t** qn, uint32_t** lo, uint32_t** hi) {
    const hicops_params& p = idx->p;
    HC_CUDA(sc.get(qbin, (uint64_t)n * p.top_n_peaks));
    HC_CUDA(sc.get(qiq, (uint64_t)n * p.top_n_peaks));
    HC_CUDA(sc.get(qn, n));
    HC_CUDA(sc.get(lo, n));
    HC_CUDA(sc.get(hi, n));
    PrepArgs pa{d.peak_off, d.mz, d.inten, d.prec, d.z, d.tol, n, p.top_n_peaks, p.bin_width_da,
                p.frag_mz_min, p.frag_mz_max, (double)p.intensity_scale, idx->dev.mass, idx->mass.size(),
                *qbin, *qiq, *qn, *lo, *hi};
    prep_kernel<<<n, kPrepThreads, 0, sc.s>>>(pa);
    count_launches(1);
    HC_CUDA(cudaGetLastError());
    return HICOPS_OK;
}

int g_sm_count = 0;

inline void mark(hicops_index* idx, int i, cudaStream_t s) {
    if (idx->dev.timing) cudaEventRecord((cudaEvent_t)idx->dev.ev[i], s);
}

template <int KMAX>
hicops_status launch_search(const SearchArgs& sa, cudaStream_t s) {
    static int blocks_per_sm = -1;
    const size_t smem = sizeof(uint32_t) * kChunk;
    if (blocks_per_sm < 0) {
        HC_CUDA(cudaFuncSetAttribute(search_kernel<KMAX>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        HC_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks_per_sm, search_kernel<KMAX>, kSearchThreads, smem));
        if (blocks_per_sm < 1) blocks_per_sm = 1;
    }
    search_kernel<KMAX><<<g_sm_count * blocks_per_sm, kSearchThreads, smem, s>>>(sa);
    count_launches(1);
    HC_CUDA(cudaGetLastError());
    return HICOPS_OK;
}

}  // namespace
}  // namespace hicops

using namespace hicops;

extern "C" hicops_status hicops_search(hicops_index* idx, const hicops_batch* b, hicops_psm* out_psm,
                                       uint32_t* out_hist, uint32_t* out_nscored) {
    hicops_status st = check_batch(idx, b);
    if (st != HICOPS_OK) return st;
    if (!out_psm) { set_error("out_psm is NULL"); return HICOPS_EINVAL; }
    const uint32_t n = b->n;
    if (n == 0) return HICOPS_OK;
    if (!g_sm_count) {
        int dev;
        HC_CUDA(cudaGetDevice(&dev));
        HC_CUDA(cudaDeviceGetAttribute(&g_sm_count, cudaDevAttrMultiProcessorCount, dev));
    }
    const hicops_params& p = idx->p;
    const uint32_t k = p.top_k;
    cudaStream_t s = (cudaStream_t)b->cuda_stream;
    hicops_psm* d_psm = nullptr;
    uint32_t *d_hist = nullptr, *d_ns = nullptr;
    {
        Scratch sc(s);
        DevBatch d;
        uint64_t npk = 0;
        st = stage_inputs(b, sc, d, &npk);
        if (st != HICOPS_OK) return st;
        uint32_t *qbin, *qiq, *qn, *lo, *hi;
        mark(idx, 0, s);
        st = run_prep(idx, d, n, sc, &qbin, &qiq, &qn, &lo, &hi);
        if (st != HICOPS_OK) return st;
        mark(idx, 1, s);
        // split windows across CTAs when the batch is small
        const uint32_t ctas = (uint32_t)g_sm_count * 2;
        uint32_t max_seg = (4 * ctas + n - 1) / n;
        if (max_seg < 1) max_seg = 1;
        if (max_seg > (uint32_t)kMaxSegs) max_seg = kMaxSegs;
        uint32_t* nseg;
        uint64_t *seg_off, *stmp;
        HC_CUDA(sc.get(&nseg, n));
        HC_CUDA(sc.get(&seg_off, n + 1));
        HC_CUDA(sc.get(&stmp, scan_tmp_words(n)));
        plan_kernel<<<(n + 255) / 256, 256, 0, s>>>(qn, lo, hi, n, max_seg, nseg);
        count_launches(1);
        HC_CUDA(cudaGetLastError());
        HC_CUDA(exclusive_scan<uint32_t>(nseg, n, seg_off, seg_off + n, stmp, s));
        UnitTop* utop;
        unsigned long long* work;
        HC_CUDA(sc.get(&utop, (uint64_t)n * max_seg * k));
        HC_CUDA(sc.get(&work, 1));
        if (b->on_device) {
            d_psm = out_psm;
            d_hist = out_hist;
            d_ns = out_nscored;
        }
        if (!d_psm) HC_CUDA(sc.get(&d_psm, (uint64_t)n * k));
        if (!d_hist) HC_CUDA(sc.get(&d_hist, (uint64_t)n * kHistBins));
        if (!d_ns) HC_CUDA(sc.get(&d_ns, n));
        HC_CUDA(cudaMemsetAsync(d_hist, 0, sizeof(uint32_t) * n * kHistBins, s));
        HC_CUDA(cudaMemsetAsync(d_ns, 0, sizeof(uint32_t) * n, s));
        HC_CUDA(cudaMemsetAsync(work, 0, sizeof(unsigned long long), s));
        SearchArgs sa{qbin, qiq, qn, lo, hi, seg_off, n, p.top_n_peaks, idx->dev.off, idx->dev.entry,
                      idx->dev.lf, idx->dev.ls, p.min_shared, k, utop, d_hist, d_ns, work};
        mark(idx, 2, s);
        if (k <= 8) st = launch_search<8>(sa, s);
        else if (k <= 16) st = launch_search<16>(sa, s);
        else st = launch_search<32>(sa, s);
        if (st != HICOPS_OK) return st;
        mark(idx, 3, s);
        MergeArgs ma{seg_off, utop, d_hist, n, k, 0, d_psm};
        merge_kernel<<<n, kMergeThreads, 0, s>>>(ma);
        count_launches(1);
        HC_CUDA(cudaGetLastError());
        mark(idx, 4, s);
        if (!b->on_device) {
            HC_CUDA(cudaMemcpyAsync(out_psm, d_psm, sizeof(hicops_psm) * n * k, cudaMemcpyDeviceToHost, s));
            if (out_hist)
                HC_CUDA(cudaMemcpyAsync(out_hist, d_hist, sizeof(uint32_t) * n * kHistBins, cudaMemcpyDeviceToHost, s));
            if (out_nscored)
                HC_CUDA(cudaMemcpyAsync(out_nscored, d_ns, sizeof(uint32_t) * n, cudaMemcpyDeviceToHost, s));
        }
    }
    if (!b->on_device) HC_CUDA(cudaStreamSynchronize(s));
    return HICOPS_OK;
}

extern "C" hicops_status hicops_search_work(hicops_index* idx, const hicops_batch* b, uint32_t* out_lo,
                                            uint32_t* out_hi, uint32_t* out_npeaks, uint64_t* out_hits) {
    hicops_status st = check_batch(idx, b);
    if (st != HICOPS_OK) return st;
    const uint32_t n = b->n;
    if (n == 0) return HICOPS_OK;
    cudaStream_t s = (cudaStream_t)b->cuda_stream;
    {
        Scratch sc(s);
        DevBatch d;
        uint64_t npk = 0;
        st = stage_inputs(b, sc, d, &npk);
        if (st != HICOPS_OK) return st;
        uint32_t *qbin, *qiq, *qn, *lo, *hi;
        st = run_prep(idx, d, n, sc, &qbin, &qiq, &qn, &lo, &hi);
        if (st != HICOPS_OK) return st;
        uint64_t* hits;
        HC_CUDA(sc.get(&hits, n));
        work_kernel<<<n, 256, 0, s>>>(qbin, qn, lo, hi, idx->p.top_n_peaks, idx->dev.off, idx->dev.entry, hits);
        count_launches(1);
        HC_CUDA(cudaGetLastError());
        const cudaMemcpyKind kind = b->on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
        if (out_lo) HC_CUDA(cudaMemcpyAsync(out_lo, lo, sizeof(uint32_t) * n, kind, s));
        if (out_hi) HC_CUDA(cudaMemcpyAsync(out_hi, hi, sizeof(uint32_t) * n, kind, s));
        if (out_npeaks) HC_CUDA(cudaMemcpyAsync(out_npeaks, qn, sizeof(uint32_t) * n, kind, s));
        if (out_hits) HC_CUDA(cudaMemcpyAsync(out_hits, hits, sizeof(uint64_t) * n, kind, s));
    }
    if (!b->on_device) HC_CUDA(cudaStreamSynchronize(s));
    return HICOPS_OK;
}

namespace hicops {
static std::atomic<uint64_t> g_launches{0};
void count_launches(uint64_t n) { g_launches.fetch_add(n, std::memory_order_relaxed); }
}  // namespace hicops

extern "C" uint64_t hicops_kernel_launches(void) { return hicops::g_launches.load(); }

extern "C" hicops_status hicops_index_set_timing(hicops_index* idx, int enable) {
    if (!idx || !idx->dev.ready) { set_error("index not uploaded"); return HICOPS_EINVAL; }
    if (enable && !idx->dev.ev[0]) {
        for (int i = 0; i < 5; ++i) {
            cudaEvent_t e;
            HC_CUDA(cudaEventCreate(&e));
            idx->dev.ev[i] = e;
        }
    }
    idx->dev.timing = enable != 0;
    return HICOPS_OK;
}

extern "C" hicops_status hicops_index_last_timing(hicops_index* idx, hicops_timing* out) {
    if (!idx || !out || !idx->dev.timing) { set_error("timing is not enabled"); return HICOPS_EINVAL; }
    cudaEvent_t* e = (cudaEvent_t*)idx->dev.ev;
    HC_CUDA(cudaEventSynchronize(e[4]));
    float t[4];
    for (int i = 0; i < 4; ++i) HC_CUDA(cudaEventElapsedTime(&t[i], e[i], e[i + 1]));
    out->prep_ms = t[0];
    out->plan_ms = t[1];
    out->search_ms = t[2];
    out->merge_ms = t[3];
    HC_CUDA(cudaEventElapsedTime(&out->total_ms, e[0], e[4]));
    return HICOPS_OK;
}
