// filter_2 + score + heap of superstep 3 (paper: Eq. 4 terms k32'..k34,
// Supplementary Algorithm 3), included by search_kernels.cuh.
//
// One persistent CTA pulls work units (spectrum q, peptide-id segment) from a
// device counter.  The segment is cut into super-chunks of whole skip-table
// columns (kChunk peptide ids each, at most kMaxCols); the columns per
// super-chunk are chosen per unit from the skip tables so that a super-chunk
// holds about target_entries index entries of the spectrum's ordinary peaks.
//
// Almost every peptide in a precursor window is hit by at most one ordinary
// peak, and with fewer than min_shared - 1 hot slices such a peptide cannot
// reach min_shared.  So a super-chunk is searched as:
//   pass A  every index entry (all ordinary peaks' runs, rounded out to
//           16-byte groups, laid end to end by a prefix sum; lane l of a warp
//           takes the 4-entry groups 4 l, 4 l + 128, ..., one 16-byte load
//           each) sets the peptide's bit in a "seen" bit-plane and, when it
//           was set, in a "twice" plane (shared-memory atomicOr), and is
//           logged in shared memory as (peptide offset << 1 | isY | peak <<
//           19); first bits set in the twice plane are counted;
//   mark    only when nslices >= min_shared - 1 (peptides seen once with
//           enough hot bits are candidates too) or when there are more than
//           kRound candidates: the planes are scanned with the bitmaps,
//           candidates counted and split into rounds of at most kRound
//           candidates by runs of whole plane words; when the hot peaks alone
//           can reach min_shared, the peptides of the segment no ordinary
//           peak hit but with enough hot bits are scored here; otherwise
//           there is one round of the twice plane;
//   replay  per round, the log is walked; a candidate's record goes to its
//           warp's queue, and full queues add (1 << 26 | iq) for a b ion or
//           (1 << 20 | iq) for a y ion to the peptide's 32-bit counter (nb |
//           ny | S) in an open-addressing table of kSlots 64-bit slots
//           (offset << 32 | counter); a round has fewer than kSlots keys, so
//           probing always ends;
//   epilogue the occupied slots get the hot peaks' contributions from the
//           bucket bitmaps; peptides with nb + ny >= min_shared are ranked
//           with the exact key K = LF[nb] + LF[ny] + LS[S] and counted in the
//           shared histogram; those better than their warp's k-th enter the
//           warp's top-k list in shared memory (lanes take turns at points
//           where the warp is converged), and the warps' lists are merged at
//           the end of the unit.  Keeping the lists out of registers leaves
//           80 registers a thread, so CTAs of 384 threads run two per SM.
// The planes take 2 x 512 words per column of the super-chunk and the log
// the words after them, so sparse spectra get wide super-chunks and dense
// ones long logs.  A super-chunk whose planes and log do not fit is searched
// column by column with 16384 directly indexed counters.

constexpr int kMaxHot = 6;                 // bitmap slices (b or y bitmap of a hot bucket) per spectrum
constexpr int kMaxWarps = 16;              // CTAs of up to 512 threads
constexpr int kTouchCap = 3584;            // touched list of a direct-counter column (more: full scan)
constexpr uint32_t kSlots = 1024;          // candidate counters per round
constexpr uint32_t kRound = 768;           // candidates per round (+31 at most)
constexpr uint32_t kListWords = 1152;      // compaction lists: up to 3 groups of 32 slots per warp
constexpr uint32_t kRoundsCap = 32;        // candidate rounds of a super-chunk at most
constexpr uint32_t kSmemPerCta = 233472 / 2 - 1024;   // shared memory of one of two CTAs on an SM


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
    const int32_t* skip_row;
    const uint32_t* skip;
    uint32_t skip_stride;
    const int32_t* hot_id;
    const uint32_t* hot_b;
    const uint32_t* hot_y;
    const uint32_t* hot_flags;
    uint64_t hot_words;
    const int64_t* lf;
    const int64_t* ls;
    uint32_t s_max;             // last valid index of ls
    uint32_t min_shared;
    uint32_t k;
    uint32_t target_entries;    // entries aimed for per super-chunk
    UnitTop* utop;              // [units * k]
    uint32_t* hist;             // [n * 256]
    uint32_t* nscored;          // [n]
    unsigned long long* work;   // unit counter
    const uint32_t* order;      // [units] the units in the order they are taken (longest first), or NULL
    const uint32_t* order_q;    // [units] the spectrum of each of them
};

__device__ __forceinline__ bool better(int64_t ka, uint32_t pa, int64_t kb, uint32_t pb) {
    return ka > kb || (ka == kb && pa < pb);
}

// A warp's best k candidates of the current unit, sorted by (key desc, pid
// asc), in shared memory; one lane at a time inserts (warp-synchronous).
template <int KMAX>
struct WarpTop {
    int64_t key[KMAX];
    uint32_t pid[KMAX];
    uint32_t pk[KMAX];
    int n;
    __device__ __forceinline__ bool passes(int64_t kk, uint32_t p, int k) const {
        return n < k || better(kk, p, key[k - 1], pid[k - 1]);
    }
    __device__ __forceinline__ void insert(int64_t kk, uint32_t p, uint32_t packed, int k) {
        if (!passes(kk, p, k)) return;
        int pos = n < k ? n : k - 1;
        while (pos > 0 && better(kk, p, key[pos - 1], pid[pos - 1])) {
            key[pos] = key[pos - 1];
            pid[pos] = pid[pos - 1];
            pk[pos] = pk[pos - 1];
            --pos;
        }
        key[pos] = kk;
        pid[pos] = p;
        pk[pos] = packed;
        if (n < k) ++n;
    }
};

template <int MAXP>
struct SearchShared {
    uint32_t pbase[MAXP];             // bucket start of each ordinary peak, in 4-entry groups
    uint32_t prow[MAXP];              // its skip-table row
    uint32_t pinc[MAXP];              // its quantised intensity
    uint32_t pre[2][MAXP + 1];        // exclusive prefix of the run lengths (parity)
    uint32_t rs[2][MAXP];             // run starts relative to the bucket (parity)
    union {
        uint16_t touched[MAXP <= 512 ? 1 : kTouchCap];   // counters that became non-zero (else dynamic)
        uint16_t hotc[MAXP];          // (classification) hot peaks: index into qbin
    };
    uint16_t wli[2][kMaxWarps];       // peak holding each warp's first entry (parity)
    uint16_t wb[kRoundsCap + 1];      // first plane word of each candidate round
    int ntouched;                     // > kTouchCap means the list overflowed
    int nrounds;
    uint32_t ncand[2];                // candidates counted by pass A (alternating super-chunks)
    const uint32_t* slice[kMaxHot];   // bitmap rows of the spectrum's hot slices
    uint32_t slice_inc[kMaxHot];      // counter increment of a set bit
    uint32_t hist[kHistBins];
    int64_t lf[kMaxLen + 1];
    uint32_t wsum[kMaxWarps];
    uint32_t wcand[kMaxWarps];
    int nnorm, nhotc, nslices, nhotpeaks;
    uint64_t unit;
    uint32_t q, np;
    uint32_t seg_lo, seg_hi;
};

// Dynamic shared memory of the kernel for top-k lists of KMAX, CTAs of
// THREADS and at most MAXP query bins, in 32-bit words: what two CTAs on an
// SM leave beside their static part.  A super-chunk of m columns (W = 512 m
// words per plane):
//   [0, W) seen plane | [W, 2W) twice plane | [2W, 2W + R) log |
//   [kListWord, kSlotWord) slot compaction lists | [kSlotWord, kDynWords) kSlots 64-bit slots;
// or [0, 16384) direct counters (lists and slots are zero then), with the
// direct columns' touched list right above them for MAXP = 512, where the
// smaller static part leaves the planes and log about 21 k words (about
// 15.5 k for MAXP = 1024).
template <int KMAX, int THREADS, int MAXP>
struct Layout {
    static constexpr uint32_t kStatic = sizeof(SearchShared<MAXP>) + (THREADS / 32) * sizeof(WarpTop<KMAX>) + 64;
    static constexpr uint32_t kDynWords = ((kSmemPerCta - kStatic) / 4) & ~31u;
    static constexpr uint32_t kSlotWord = kDynWords - 2 * kSlots;
    static constexpr uint32_t kListWord = kSlotWord - kListWords;
    static constexpr uint32_t kMaxRounds = kListWord / kRound + 2;
    // widest super-chunk (columns of kChunk ids): planes within the counters'
    // 16384 words (below the touched list) and 19-bit record offsets, and
    // room for a log of 2048 words beside the widest planes
    static constexpr uint32_t kMaxCols = (kListWord - 2048) / 1024 < 16 ? (kListWord - 2048) / 1024 : 16;
    static constexpr bool kTouchDyn = MAXP <= 512;
    static_assert(kMaxRounds <= kRoundsCap, "round starts fit");
    static_assert(kMaxCols >= 1 && 2 * kMaxCols * kChunk / 32 < kListWord, "planes leave room for a log");
    static_assert(2 * kMaxCols * kChunk / 32 <= kChunk, "planes never reach the touched list");
    static_assert(2 * kMaxCols * kChunk <= 0x80000u, "record offsets fit 19 bits below the peak index");
    static_assert(!kTouchDyn || kChunk + kTouchCap / 2 <= kListWord, "the touched list lies below the lists");
    static_assert(kDynWords >= kChunk, "the direct counters fit");
};

__device__ __forceinline__ uint32_t counter_inc_y(uint32_t isy, uint32_t iq) {
    return iq + (isy ? (1u << kNyShift) : (1u << kNbShift));
}

__device__ __forceinline__ uint32_t slot_of(uint32_t off) { return (off * 2654435761u) >> 22; }   // 10 bits

// A run [ra, rb) of a bucket (positions relative to its 16-byte aligned
// start) is read as whole groups of 4 entries: from ra rounded down to a
// multiple of 4 to rb rounded up.  The extra entries at either end lie in the
// same bucket outside the run's columns, or are the bucket's pad slots; both
// fall outside every peptide range the run is searched for.
__device__ __forceinline__ uint32_t group_start(uint32_t ra) { return ra & ~3u; }
__device__ __forceinline__ uint32_t group_len(uint32_t ra, uint32_t rb) {
    return ra == rb ? 0u : ((rb + 3u) & ~3u) - (ra & ~3u);
}

// Exclusive scan of the ordinary peaks' run lengths (in whole groups), in two
// halves around a barrier the caller provides.  Thread tid owns peaks
// tid*ppt .. +ppt-1.
template <int PPT, class SH>
__device__ __forceinline__ uint32_t scan_runs_1(SH& sh, int nnorm, int ppt, const uint32_t (&ra)[PPT],
                                                const uint32_t (&rb)[PPT]) {
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    uint32_t sum = 0;
#pragma unroll
    for (int i = 0; i < PPT; ++i) {
        const int t = tid * ppt + i;
        if (i < ppt && t < nnorm) sum += group_len(ra[i], rb[i]);
    }
    uint32_t incl = sum;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t x = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += x;
    }
    if (lane == 31) sh.wsum[warp] = incl;
    return incl - sum;
}

// Warp shares are multiples of 4 entries so that a lane's 4 consecutive
// entries never cross into the next warp's share.
template <int THREADS>
__device__ __forceinline__ uint32_t warp_share(uint32_t total) {
    constexpr int nwarps = THREADS / 32;
    return ((total + nwarps - 1) / nwarps + 3) & ~3u;
}

template <int THREADS, int PPT, class SH>
__device__ __forceinline__ void scan_runs_2(SH& sh, int buf, int nnorm, int ppt, uint32_t excl,
                                            const uint32_t (&ra)[PPT], const uint32_t (&rb)[PPT]) {
    const int tid = threadIdx.x, warp = tid >> 5;
    constexpr int nwarps = THREADS / 32;
    uint32_t wbase = 0, total = 0;
#pragma unroll
    for (int w = 0; w < nwarps; ++w) {
        const uint32_t s = sh.wsum[w];
        if (w < warp) wbase += s;
        total += s;
    }
    const uint32_t per = warp_share<THREADS>(total);
    uint32_t run = wbase + excl;
#pragma unroll
    for (int i = 0; i < PPT; ++i) {
        const int t = tid * ppt + i;
        if (i < ppt && t < nnorm) {
            const uint32_t len = group_len(ra[i], rb[i]);
            sh.pre[buf][t] = run;
            sh.rs[buf][t] = group_start(ra[i]);
            if (len)   // warps whose share starts inside this run
                for (uint32_t w = (run + per - 1) / per; w * per < run + len && w < (uint32_t)nwarps; ++w)
                    sh.wli[buf][w] = (uint16_t)t;
            run += len;
        }
    }
    if (tid == 0) sh.pre[buf][nnorm] = total;
}

template <int KMAX, int THREADS, int MAXP>
__global__ void __launch_bounds__(THREADS, THREADS <= 384 ? 2 : 1) search_kernel(SearchArgs a) {
    using L = Layout<KMAX, THREADS, MAXP>;
    constexpr uint32_t kDynWords = L::kDynWords, kSlotWord = L::kSlotWord, kListWord = L::kListWord;
    constexpr uint32_t kMaxRounds = L::kMaxRounds, kMaxCols = L::kMaxCols;
    extern __shared__ __align__(16) uint32_t smem32[];   // kDynWords words (layout above)
    uint32_t* const cnt = smem32;
    uint32_t* const seen = smem32;
    uint32_t* const lists = smem32 + kListWord;
    unsigned long long* const tab = reinterpret_cast<unsigned long long*>(smem32 + kSlotWord);
    __shared__ SearchShared<MAXP> sh;
    uint16_t* const touched = L::kTouchDyn ? reinterpret_cast<uint16_t*>(smem32 + kChunk) : sh.touched;
    constexpr int nwarps = THREADS / 32;
    constexpr int PPT = (MAXP + THREADS - 1) / THREADS;   // ordinary peaks per thread (at most)
    constexpr int kListStride = (32 / nwarps + (32 % nwarps ? 1 : 0)) * 32;   // list words per warp
    static_assert(kListStride * nwarps <= (int)kListWords, "compaction lists fit");
    __shared__ WarpTop<KMAX> wtop[nwarps];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const unsigned lt = (1u << lane) - 1u;
    const uint32_t last_col = a.skip_stride - 1;
    for (int i = tid; i < (int)kDynWords; i += THREADS) smem32[i] = 0u;
    for (int i = tid; i < (int)kHistBins; i += THREADS) sh.hist[i] = 0;
    for (int i = tid; i <= (int)kMaxLen; i += THREADS) sh.lf[i] = a.lf[i];
    if (tid == 0) { sh.ncand[0] = 0u; sh.ncand[1] = 0u; }
    if (tid < nwarps) wtop[tid].n = 0;
    const uint64_t total_units = a.seg_off[a.n];
    const int k = (int)a.k;
    const uint32_t min_shared = a.min_shared;
    int par = 0;                  // alternates per super-chunk: which ncand counts
    uint32_t log_lo = kListWord, log_dirty = 0;   // words [log_lo, log_dirty) may hold log records
    __syncthreads();
    for (;;) {
        if (tid == 0) {
            const uint64_t t = atomicAdd(a.work, 1ull);
            const bool listed = t < total_units && a.order;
            const uint64_t u = listed ? (uint64_t)a.order[t] : t;
            sh.unit = u;
            sh.nnorm = 0;
            sh.nhotc = 0;
            sh.nslices = 0;
            sh.nhotpeaks = 0;
            sh.ntouched = 0;
            if (u < total_units) {
                // spectrum owning unit u (without an order list: the last q
                // with seg_off[q] <= u)
                uint32_t lo_q = 0, hi_q = a.n;
                if (listed) lo_q = a.order_q[t];
                else
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
        // classify the retained peaks: hot (bitmap) candidates or ordinary (skip table)
        for (uint32_t t = tid; t < np; t += THREADS) {
            const uint32_t bin = a.qbin[(uint64_t)q * a.topn + t];
            if (a.hot_id[bin] >= 0) {
                sh.hotc[atomicAdd(&sh.nhotc, 1)] = (uint16_t)t;
                continue;
            }
            const int32_t row = a.skip_row[bin];
            if (row < 0) continue;   // empty bucket
            const int s = atomicAdd(&sh.nnorm, 1);
            sh.pbase[s] = (uint32_t)(a.off[bin] >> 2);
            sh.prow[s] = (uint32_t)row;
            sh.pinc[s] = a.qiq[(uint64_t)q * a.topn + t];
        }
        __syncthreads();
        if (warp == 0) {
            // bitmap slices for the hot peaks while they last (warp 0, 32
            // hot peaks at a time: lanes load their peaks' tables together,
            // a prefix of slices needed picks the takers); the rest are
            // streamed like ordinary peaks.  Which hot peaks get slices does
            // not change any result.
            int ns = 0, nh = 0;   // warp-uniform
            const int nhc = sh.nhotc;
            for (int c0 = 0; c0 < nhc; c0 += 32) {
                const int c = c0 + lane;
                const bool act = c < nhc;
                uint32_t bin = 0, iq = 0, fl = 0;
                int32_t hid = 0;
                if (act) {
                    const uint32_t t = sh.hotc[c];
                    bin = a.qbin[(uint64_t)q * a.topn + t];
                    iq = a.qiq[(uint64_t)q * a.topn + t];
                    hid = a.hot_id[bin];
                    fl = a.hot_flags[hid];
                }
                const int need = (fl & 1u ? 1 : 0) + (fl & 2u ? 1 : 0);
                int incl = need;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const int x = __shfl_up_sync(0xffffffffu, incl, o);
                    if (lane >= o) incl += x;
                }
                const bool take = act && ns + incl <= kMaxHot;   // a prefix of the lanes
                if (take) {
                    int p = ns + incl - need;
                    if (fl & 1u) { sh.slice[p] = a.hot_b + (uint64_t)hid * a.hot_words; sh.slice_inc[p++] = (1u << kNbShift) + iq; }
                    if (fl & 2u) { sh.slice[p] = a.hot_y + (uint64_t)hid * a.hot_words; sh.slice_inc[p] = (1u << kNyShift) + iq; }
                } else if (act) {
                    const int s = atomicAdd(&sh.nnorm, 1);
                    sh.pbase[s] = (uint32_t)(a.off[bin] >> 2);
                    sh.prow[s] = (uint32_t)a.skip_row[bin];
                    sh.pinc[s] = iq;
                }
                const unsigned tm = __ballot_sync(0xffffffffu, take);
                nh += __popc(tm);
                if (tm) ns += __shfl_sync(0xffffffffu, incl, 31 - __clz(tm));   // the last taker's prefix
            }
            if (lane == 0) {
                sh.nslices = ns;
                sh.nhotpeaks = nh;
            }
        }
        __syncthreads();
        const int nnorm = sh.nnorm, nslices = sh.nslices;
        const bool hot_alone = sh.nhotpeaks >= (int)min_shared;
        // peptides hit once are candidates too when the hot slices alone can
        // supply the other min_shared - 1 shared peaks
        const bool once_counts = (uint32_t)nslices + 1u >= min_shared;
        const int ppt = (nnorm + THREADS - 1) / THREADS;
        const uint32_t col_lo = seg_lo >> kChunkShift, col_end = ((seg_hi - 1) >> kChunkShift) + 1;
        uint32_t ra[PPT], rb[PPT];
        auto load_runs = [&](uint32_t c0l, uint32_t c1l) {
#pragma unroll
            for (int i = 0; i < PPT; ++i) {
                const int t = tid * ppt + i;
                ra[i] = rb[i] = 0;
                if (i < ppt && t < nnorm) {
                    const uint32_t* sk = a.skip + (uint64_t)sh.prow[t] * a.skip_stride;
                    ra[i] = __ldg(sk + c0l);
                    rb[i] = __ldg(sk + min(c1l, last_col));
                }
            }
        };
        // columns per super-chunk, from the segment's total entries
        uint32_t m = 1;
        {
            load_runs(col_lo, col_end);
            uint32_t s = 0;
#pragma unroll
            for (int i = 0; i < PPT; ++i) s += rb[i] - ra[i];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
            if (lane == 0) sh.wsum[warp] = s;
            __syncthreads();
            uint32_t total = 0;
#pragma unroll
            for (int w = 0; w < nwarps; ++w) total += sh.wsum[w];
            const uint32_t ncols = col_end - col_lo;
            {
                // about target_entries entries, and planes (1024 words a
                // column) plus 1.25 times the mean log within kListWord
                // words, so that denser-than-mean super-chunks still fit
                uint64_t want = total ? ((uint64_t)a.target_entries * ncols) / total : ncols;
                const uint64_t fit = (uint64_t)kListWord * ncols / ((uint64_t)1024 * ncols + total + total / 4);
                if (want > fit) want = fit;
                if (want < 1) want = 1;
                if (want > kMaxCols) want = kMaxCols;
                m = min((uint32_t)want, ncols);
            }
            __syncthreads();   // wsum is reused by the scans
        }
        // a lane's scored candidate waiting for its warp's list (flush)
        int64_t pK = 0;
        uint32_t pP = 0u, pC = 0u;
        bool pend = false;
        uint32_t* twice = smem32;   // the current super-chunk's twice plane and log
        uint32_t* logw = smem32;

        // Calls fn(f, entry, peak) for every entry f of parity buffer buf.
        // Warp w takes a contiguous share; lane l takes f0 + l + 32 j, kJ
        // loads in flight before any is used.  Each lane walks the runs
        // forward, keeping the current run's end and the entry-array base
        // gb (entry f of the run is entry[gb + f]) in registers.
        auto for_each_entry = [&](int buf, auto&& fn) {
            constexpr int kJ = 8;
            const uint32_t R = sh.pre[buf][nnorm];
            const uint32_t per = warp_share<THREADS>(R);
            const uint32_t f0 = (uint32_t)warp * per, f1 = min(R, f0 + per);
            if (f0 >= f1) return;
            int li = sh.wli[buf][warp];
            uint32_t nxt = sh.pre[buf][li + 1];
            uint64_t gb = ((uint64_t)sh.pbase[li] << 2) + sh.rs[buf][li] - sh.pre[buf][li];
            for (uint32_t fb = f0 + lane; fb < f1; fb += 32 * kJ) {
                uint32_t ev[kJ];
                uint32_t lp[kJ];
#pragma unroll
                for (int j = 0; j < kJ; ++j) {
                    const uint32_t f = fb + 32 * j;
                    ev[j] = 0xffffffffu;
                    lp[j] = 0;
                    if (f < f1) {
                        while (f >= nxt) {
                            ++li;
                            nxt = sh.pre[buf][li + 1];
                            gb = ((uint64_t)sh.pbase[li] << 2) + sh.rs[buf][li] - sh.pre[buf][li];
                        }
                        lp[j] = (uint32_t)li;
                        ev[j] = __ldg(a.entry + (gb + f));
                    }
                }
#pragma unroll
                for (int j = 0; j < kJ; ++j)
                    if (fb + 32 * j < f1) fn(fb + 32 * j, ev[j], (int)lp[j]);
            }
        };
        auto score = [&](uint32_t c, uint32_t pid) {
            const uint32_t nb = c >> kNbShift, ny = (c >> kNyShift) & 63u;
            if (nb + ny >= min_shared) {
                uint32_t S = c & kSMask;
                if (S > a.s_max) S = a.s_max;   // unreachable for a consistent index
                const int64_t K = sh.lf[nb] + sh.lf[ny] + __ldg(a.ls + S);
                const int64_t hb = K >> 31;
                atomicAdd(&sh.hist[hb > 255 ? 255 : (hb < 0 ? 0 : hb)], 1u);
                if (wtop[warp].passes(K, pid, k)) { pK = K; pP = pid; pC = c; pend = true; }
            }
        };
        // pending candidates into the warp's list, one lane at a time; every
        // lane of the warp calls it (convergent points only)
        auto flush = [&]() {
            unsigned pm = __ballot_sync(0xffffffffu, pend);
            while (pm) {
                const int l = __ffs(pm) - 1;
                pm &= pm - 1;
                if (lane == l) wtop[warp].insert(pK, pP, pC, k);
                __syncwarp();
            }
            pend = false;
        };
        // one counter (c, pid): filter, add the hot slices, score
        auto visit = [&](uint32_t c, uint32_t pid) {
            const uint32_t nn = (c >> kNbShift) + ((c >> kNyShift) & 63u);
            if (nn + (uint32_t)nslices < min_shared) return;
            uint32_t hw[kMaxHot];   // every slice's word in flight at once
#pragma unroll
            for (int s = 0; s < kMaxHot; ++s) hw[s] = s < nslices ? __ldg(sh.slice[s] + (pid >> 5)) : 0u;
#pragma unroll
            for (int s = 0; s < kMaxHot; ++s)
                if ((hw[s] >> (pid & 31)) & 1u) c += sh.slice_inc[s];
            score(c, pid);
        };

        // ---- one column with direct counters (the caller provides the
        // barriers before and after)
        auto column_pass = [&](int buf, uint32_t cb, uint32_t x0, uint32_t x1) {
            for_each_entry(buf, [&](uint32_t, uint32_t e, int li) {
                const uint32_t pid = e >> 1;
                bool first = false;
                uint32_t off = 0;
                if (pid >= x0 && pid < x1) {
                    off = pid - cb;
                    first = atomicAdd(&cnt[off], counter_inc_y(e & 1u, sh.pinc[li])) == 0u;
                }
                if (first) {
                    const int slot = atomicAdd(&sh.ntouched, 1);
                    if (slot < kTouchCap) touched[slot] = (uint16_t)off;
                }
            });
            __syncthreads();
            const int nt = sh.ntouched;
            if (nt <= kTouchCap && !hot_alone) {
                for (int i0 = warp * 32; i0 < nt; i0 += THREADS) {   // warp-uniform trip count
                    const int i = i0 + lane;
                    if (i < nt) {
                        const uint32_t w = touched[i];
                        const uint32_t c = cnt[w];
                        cnt[w] = 0u;
                        visit(c, cb + w);
                    }
                    flush();
                }
            } else {
                // every counter, 32 peptide ids per step; bitmaps alone can
                // qualify a peptide when hot_alone
                for (uint32_t gi = tid; gi < kChunk / 32; gi += THREADS) {   // warp-uniform trip count
                    const uint32_t gp = cb + (gi << 5);
                    const bool act = !(gp + 32 <= x0 || gp >= x1);
                    const uint32_t lo_b = x0 > gp ? x0 - gp : 0u;
                    const uint32_t hi_b = x1 - gp >= 32u ? 32u : x1 - gp;
                    const uint32_t valid = (hi_b >= 32u ? 0xffffffffu : ((1u << hi_b) - 1u)) & ~((1u << lo_b) - 1u);
                    uint32_t hw[kMaxHot];
#pragma unroll
                    for (int s = 0; s < kMaxHot; ++s) hw[s] = act && s < nslices ? __ldg(sh.slice[s] + (gp >> 5)) : 0u;
                    uint32_t cand = 0;
                    for (int j = 0; act && j < 32; ++j) {
                        const int jb = (j + lane) & 31;   // rotated: lanes hit different banks
                        const uint32_t c = cnt[(gi << 5) + jb];
                        uint32_t hc = 0;
#pragma unroll
                        for (int s = 0; s < kMaxHot; ++s) hc += (hw[s] >> jb) & 1u;
                        const uint32_t nn = (c >> kNbShift) + ((c >> kNyShift) & 63u);
                        if ((c != 0u || hc > 0u) && nn + hc >= min_shared) cand |= 1u << jb;
                    }
                    cand &= act ? valid : 0u;
                    while (__any_sync(0xffffffffu, cand != 0u)) {   // one candidate a lane per step
                        if (cand) {
                            const int jb = __ffs(cand) - 1;
                            cand &= cand - 1;
                            uint32_t c = cnt[(gi << 5) + jb];
#pragma unroll
                            for (int s = 0; s < kMaxHot; ++s)
                                if ((hw[s] >> jb) & 1u) c += sh.slice_inc[s];
                            score(c, gp + jb);
                        }
                        flush();
                    }
                    if (act) {
#pragma unroll 4
                        for (int j = 0; j < 32; ++j) cnt[(gi << 5) + ((j + lane) & 31)] = 0u;
                    }
                }
            }
            __syncthreads();
            if (tid == 0) sh.ntouched = 0;
        };

        // ---- a super-chunk in passes (see the header); entries of parity
        // buffer buf, peptide ids [x0, x1) of the span starting at cb
        // Pass A over the entries of parity buffer buf (the walk of
        // for_each_entry, specialised to groups): lane l of a warp takes the
        // 4-entry groups starting at f0 + 4 l + 128 j, each one 16-byte load,
        // kG groups in flight before any is used; then per entry the
        // seen-plane atomic, one 16-byte store of the group's 4 log records,
        // and the twice-plane atomics of second hits, so latencies overlap.
        // A log record is (entry - 2 cb) | peak << 19, i.e. offset << 1 |
        // isY in bits 0..18; entries outside [x0, x1) log 0xffffffff.
        auto pass_a = [&](int buf, uint32_t cb, uint32_t x0, uint32_t x1, int par) {
            constexpr int kG = 4;
            const uint32_t R = sh.pre[buf][nnorm];                 // a multiple of 4
            const uint32_t per = warp_share<THREADS>(R);           // a multiple of 4
            const uint32_t f0 = (uint32_t)warp * per, f1 = min(R, f0 + per);
            uint32_t fresh = 0;   // twice bits this lane set first
            if (f0 < f1) {
                int li = sh.wli[buf][warp];
                uint32_t nxt = sh.pre[buf][li + 1];
                const uint32_t* gp = a.entry + (((uint64_t)sh.pbase[li] << 2) + sh.rs[buf][li] - sh.pre[buf][li]);
                uint32_t lsh = (uint32_t)li << 19;
                // entries of pids in [x0, x1): e - e_lo < e_span (unsigned)
                const uint32_t e_lo = x0 << 1, e_span = (x1 - x0) << 1, e_cb = cb << 1;
                uint4* const log4 = reinterpret_cast<uint4*>(logw);
                for (uint32_t fb = f0 + 4u * lane; fb < f1; fb += 128u * kG) {
                    uint4 ev[kG];
                    uint32_t lr[kG];
#pragma unroll
                    for (int g = 0; g < kG; ++g) {
                        const uint32_t f = fb + 128u * g;
                        ev[g] = make_uint4(0xffffffffu, 0xffffffffu, 0xffffffffu, 0xffffffffu);
                        lr[g] = 0u;
                        if (f < f1) {
                            while (f >= nxt) {
                                ++li;
                                nxt = sh.pre[buf][li + 1];
                                gp = a.entry + (((uint64_t)sh.pbase[li] << 2) + sh.rs[buf][li] - sh.pre[buf][li]);
                                lsh = (uint32_t)li << 19;
                            }
                            lr[g] = lsh;
                            ev[g] = __ldg(reinterpret_cast<const uint4*>(gp + f));   // 16-byte aligned
                        }
                    }
#pragma unroll
                    for (int g = 0; g < kG; ++g) {
                        const uint32_t f = fb + 128u * g;
                        const uint32_t e4[4] = {ev[g].x, ev[g].y, ev[g].z, ev[g].w};
                        uint32_t rec[4], old[4], bitv[4], wd[4];
#pragma unroll
                        for (int i = 0; i < 4; ++i) {
                            const bool in = e4[i] - e_lo < e_span;
                            const uint32_t o2 = e4[i] - e_cb;
                            bitv[i] = in ? __funnelshift_l(0u, 1u, o2 >> 1) : 0u;   // 1 << (offset & 31)
                            wd[i] = o2 >> 6;
                            old[i] = in ? atomicOr(&seen[wd[i]], bitv[i]) : 0u;
                            rec[i] = in ? (o2 | lr[g]) : 0xffffffffu;
                        }
                        if (f < f1) log4[f >> 2] = make_uint4(rec[0], rec[1], rec[2], rec[3]);
#pragma unroll
                        for (int i = 0; i < 4; ++i)
                            if (old[i] & bitv[i]) fresh += (atomicOr(&twice[wd[i]], bitv[i]) & bitv[i]) ? 0u : 1u;
                    }
                }
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) fresh += __shfl_xor_sync(0xffffffffu, fresh, o);
            if (lane == 0 && fresh) atomicAdd(&sh.ncand[par], fresh);
        };
        // candidate plane (twice, plus peptides seen once with enough hot
        // bits when once_counts), its count and the rounds; clears the seen
        // plane.  Warp w owns words [w * wpw, (w + 1) * wpw), lane l every
        // 32nd of them (barriers inside).
        auto mark = [&](uint32_t cb, uint32_t words, uint32_t x0, uint32_t x1) {
            const uint32_t G = words >> 5;          // groups of 32 plane words, split evenly over the warps
            const uint32_t g0 = (uint32_t)warp * G / nwarps, g1 = (uint32_t)(warp + 1) * G / nwarps;
            const uint32_t wbeg = g0 << 5, wpw = (g1 - g0) << 5;
            uint32_t mine = 0;
            // lane l takes the 4 words wbeg + i0 + 4 l (i0 = 0, 128, ...:
            // warp-uniform trips): 16-byte plane reads, and one 16-byte
            // bitmap read per hot slice, all slices' reads in flight together
            const uint32_t need = min_shared - 1;   // <= nslices <= kMaxHot when once_counts
            for (uint32_t i0 = 0; i0 < wpw; i0 += 128u) {
                const uint32_t w = wbeg + i0 + 4u * lane;
                const bool act = i0 + 4u * lane < wpw;
                uint4 s4 = make_uint4(0u, 0u, 0u, 0u), c4 = s4;
                if (act) {
                    s4 = *reinterpret_cast<const uint4*>(seen + w);
                    c4 = *reinterpret_cast<const uint4*>(twice + w);
                }
                const bool any_s = (s4.x | s4.y | s4.z | s4.w) != 0u;
                if (any_s) *reinterpret_cast<uint4*>(seen + w) = make_uint4(0u, 0u, 0u, 0u);
                uint32_t ho[4] = {0u, 0u, 0u, 0u};   // hot_alone: peptides of no ordinary hit that qualify
                if (act && once_counts && (any_s || hot_alone)) {
                    uint4 h[kMaxHot];
#pragma unroll
                    for (int sl = 0; sl < kMaxHot; ++sl)
                        h[sl] = sl < nslices ? __ldg(reinterpret_cast<const uint4*>(sh.slice[sl] + (cb >> 5) + w))
                                             : make_uint4(0u, 0u, 0u, 0u);
                    // per peptide its hot-bit count (b1, b2: the two low bits,
                    // b3: 4 or more): seen once with at least need hot bits
                    // joins the candidates; seen never with at least
                    // min_shared is scored here (supersets for need or
                    // min_shared above 3: visit() is exact)
                    auto at_least = [](uint32_t b1, uint32_t b2, uint32_t b3, uint32_t t) {
                        if (t == 0) return 0xffffffffu;
                        if (t == 1) return b1 | b2 | b3;
                        if (t == 2) return b2 | b3;
                        if (t == 3) return (b2 & b1) | b3;
                        return b3;
                    };
                    auto word = [&](uint32_t s1, uint32_t& c2, uint32_t& hot_only, auto pick) {
                        uint32_t b1 = 0, b2 = 0, b3 = 0;
#pragma unroll
                        for (int sl = 0; sl < kMaxHot; ++sl) {
                            const uint32_t hh = pick(h[sl]);
                            const uint32_t k1 = b1 & hh;
                            b1 ^= hh;
                            const uint32_t k2 = b2 & k1;
                            b2 ^= k1;
                            b3 |= k2;
                        }
                        c2 |= s1 & at_least(b1, b2, b3, need);
                        if (hot_alone) hot_only = ~s1 & at_least(b1, b2, b3, min_shared);
                    };
                    word(s4.x, c4.x, ho[0], [](const uint4& v) { return v.x; });
                    word(s4.y, c4.y, ho[1], [](const uint4& v) { return v.y; });
                    word(s4.z, c4.z, ho[2], [](const uint4& v) { return v.z; });
                    word(s4.w, c4.w, ho[3], [](const uint4& v) { return v.w; });
                    if (any_s) *reinterpret_cast<uint4*>(twice + w) = c4;
                }
                mine += __popc(c4.x) + __popc(c4.y) + __popc(c4.z) + __popc(c4.w);
                if (hot_alone) {
                    // score them now (they are in no log), inside [x0, x1)
#pragma unroll
                    for (int kw = 0; kw < 4; ++kw) {
                        const uint32_t gp = cb + ((w + (uint32_t)kw) << 5);
                        const uint32_t lo_b = x0 > gp ? min(x0 - gp, 32u) : 0u;
                        const uint32_t hi_b = x1 > gp ? min(x1 - gp, 32u) : 0u;
                        const uint32_t valid = (hi_b >= 32u ? 0xffffffffu : ((1u << hi_b) - 1u)) &
                                               ~(lo_b >= 32u ? 0xffffffffu : ((1u << lo_b) - 1u));
                        uint32_t msk = ho[kw] & valid;
                        while (__any_sync(0xffffffffu, msk != 0u)) {
                            if (msk) {
                                const int b = __ffs(msk) - 1;
                                msk &= msk - 1;
                                visit(0u, gp + (uint32_t)b);
                            }
                            flush();
                        }
                    }
                }
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) mine += __shfl_xor_sync(0xffffffffu, mine, o);
            if (lane == 0) sh.wcand[warp] = mine;
            // a round whose first word is never found is empty: it starts at words
            for (int r = tid; r <= (int)kMaxRounds; r += THREADS) sh.wb[r] = r == 0 ? 0 : (uint16_t)words;
            __syncthreads();
            uint32_t run = 0, total = 0;
#pragma unroll
            for (int w = 0; w < nwarps; ++w) {
                if (w < warp) run += sh.wcand[w];
                total += sh.wcand[w];
            }
            // round r holds the words with r * kRound <= candidates-before < (r + 1) * kRound;
            // one round (the common case) starts at word 0 and needs no scan
            for (uint32_t i0 = 0; total > kRound && i0 < wpw; i0 += 32) {
                const uint32_t w = wbeg + i0 + lane;
                const uint32_t cw = __popc(twice[w]);
                uint32_t incl = cw;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const uint32_t x = __shfl_up_sync(0xffffffffu, incl, o);
                    if (lane >= o) incl += x;
                }
                const uint32_t before = run + incl - cw;
                const uint32_t r = before / kRound;
                if (r > 0 && (before - __popc(twice[w - 1])) / kRound < r) sh.wb[r] = (uint16_t)w;
                run += __shfl_sync(0xffffffffu, incl, 31);
            }
            if (tid == 0) sh.nrounds = (int)(total ? (total - 1) / kRound + 1 : 0);
            __syncthreads();
        };
        // Replay of the log: 4 records per thread in flight, then their
        // twice-plane words; a candidate's record goes to its warp's queue
        // (the warp's compaction-list words, free until the epilogue), and a
        // full queue is inserted into the table with every lane busy, so the
        // insert loop never runs for one or two lanes.  The loop is
        // warp-uniform (i0 - lane is the warp's first index).
        auto replay = [&](uint32_t R, uint32_t wlo, uint32_t whi) {
            constexpr int kU = 4;
            uint32_t* const queue = lists + (uint32_t)warp * kListStride;
            uint32_t qn = 0;
            auto flush = [&]() {
                __syncwarp();   // the other lanes' appends are visible
                for (uint32_t j = lane; j < qn; j += 32) {
                    const uint32_t r = queue[j];
                    const uint32_t off = (r & 0x7ffffu) >> 1;
                    const uint32_t v = counter_inc_y(r & 1u, sh.pinc[r >> 19]);
                    const unsigned long long item = ((unsigned long long)off << 32) | v;
                    uint32_t sl = slot_of(off);
                    for (uint32_t probe = 0; probe < kSlots; ++probe) {
                        const unsigned long long old = atomicCAS(&tab[sl], 0ull, item);
                        if (old == 0ull) break;
                        if ((uint32_t)(old >> 32) == off) { atomicAdd(&tab[sl], (unsigned long long)v); break; }
                        sl = (sl + 1) & (kSlots - 1);
                    }
                }
                __syncwarp();
                qn = 0;
            };
            for (uint32_t i0 = tid; i0 - lane < R; i0 += kU * THREADS) {
                uint32_t rec[kU], tw[kU];
#pragma unroll
                for (int u = 0; u < kU; ++u) {
                    const uint32_t i = i0 + u * THREADS;
                    rec[u] = i < R ? logw[i] : 0xffffffffu;
                }
#pragma unroll
                for (int u = 0; u < kU; ++u)
                    tw[u] = rec[u] != 0xffffffffu ? twice[(rec[u] & 0x7ffffu) >> 6] : 0u;
#pragma unroll
                for (int u = 0; u < kU; ++u) {
                    const uint32_t off = (rec[u] & 0x7ffffu) >> 1;
                    const uint32_t w = off >> 5;
                    const bool cand = rec[u] != 0xffffffffu && ((tw[u] >> (off & 31)) & 1u) && w >= wlo && w < whi;
                    const unsigned msk = __ballot_sync(0xffffffffu, cand);
                    if (qn + 32 > (uint32_t)kListStride) flush();
                    if (cand) queue[qn + __popc(msk & lt)] = rec[u];
                    qn += __popc(msk);
                }
            }
            flush();
        };
        // Visits the occupied slots.  Warp w compacts the occupied slot
        // indices of its share [w * spw, (w + 1) * spw) into its list words,
        // visits them with all lanes, and zeroes the slots and the list.
        auto slots_epilogue = [&](uint32_t cb) {
            const uint32_t base = (uint32_t)warp * kListStride;
            uint32_t cnt = 0;
            for (uint32_t g = warp; g < kSlots / 32; g += nwarps) {   // groups of 32 slots
                const uint32_t sl = (g << 5) + lane;
                const bool occ = tab[sl] != 0ull;
                const unsigned msk = __ballot_sync(0xffffffffu, occ);
                if (occ) lists[base + cnt + __popc(msk & lt)] = sl;
                cnt += __popc(msk);
            }
            __syncwarp();
            for (uint32_t i0 = 0; i0 < cnt; i0 += 32) {
                const uint32_t i = i0 + lane;
                if (i < cnt) {
                    const uint32_t sl = lists[base + i];
                    const unsigned long long v = tab[sl];
                    tab[sl] = 0ull;
                    visit((uint32_t)v, cb + (uint32_t)(v >> 32));
                }
                flush();
            }
            __syncwarp();
            for (uint32_t i0 = 0; i0 < (uint32_t)kListStride; i0 += 32) lists[base + i0 + lane] = 0u;
        };
        // zeroes plane words [w0, w1), both multiples of 4
        auto clear_words = [&](uint32_t* plane, uint32_t w0, uint32_t w1) {
            uint4* p4 = reinterpret_cast<uint4*>(plane);
            for (uint32_t i = w0 / 4 + tid; i < w1 / 4; i += THREADS) p4[i] = make_uint4(0u, 0u, 0u, 0u);
        };
        // prologue: bounds of the first super-chunk
        uint32_t c = col_lo;
        uint32_t e = min(col_lo + m, col_end);
        int buf = 0;
        load_runs(c, e);
        {
            const uint32_t excl = scan_runs_1<PPT>(sh, nnorm, ppt, ra, rb);
            __syncthreads();
            scan_runs_2<THREADS, PPT>(sh, buf, nnorm, ppt, excl, ra, rb);
        }
        __syncthreads();
        while (c < col_end) {
            const uint32_t R = sh.pre[buf][nnorm];
            const uint32_t words = ((e - c) << kChunkShift) >> 5;
            const bool direct = 2 * words + R > kListWord;
            // words [log_lo, log_dirty) may hold old log records: clear them
            // before they become counters or this super-chunk's planes
            if (log_dirty > log_lo && (direct || 2 * words > log_lo)) {
                for (uint32_t i = log_lo + tid; i < log_dirty; i += THREADS) smem32[i] = 0u;
                log_lo = kListWord;
                log_dirty = 0;
                __syncthreads();
            }
            if (direct) {
                // column by column with direct counters
                if (e - c == 1) {
                    const uint32_t cb = c << kChunkShift;
                    column_pass(buf, cb, max(seg_lo, cb), min(seg_hi, cb + kChunk));
                    __syncthreads();
                } else {
                    for (uint32_t cc = c; cc < e; ++cc) {
                        load_runs(cc, cc + 1);
                        const uint32_t excl = scan_runs_1<PPT>(sh, nnorm, ppt, ra, rb);
                        __syncthreads();
                        scan_runs_2<THREADS, PPT>(sh, buf ^ 1, nnorm, ppt, excl, ra, rb);
                        __syncthreads();
                        const uint32_t cb = cc << kChunkShift;
                        column_pass(buf ^ 1, cb, max(seg_lo, cb), min(seg_hi, cb + kChunk));
                        __syncthreads();
                    }
                }
                c = e;
                if (c < col_end) {
                    e = min(c + m, col_end);
                    load_runs(c, e);
                    const uint32_t excl = scan_runs_1<PPT>(sh, nnorm, ppt, ra, rb);
                    __syncthreads();
                    scan_runs_2<THREADS, PPT>(sh, buf, nnorm, ppt, excl, ra, rb);
                    __syncthreads();
                }
                continue;
            }
            const uint32_t cbase = c << kChunkShift;
            const uint32_t x0 = max(seg_lo, cbase), x1 = min(seg_hi, e << kChunkShift);
            twice = seen + words;
            logw = seen + 2 * words;
            const uint32_t nc = e, ne = min(e + m, col_end);
            const bool more = nc < col_end;
            if (more) load_runs(nc, ne);                 // next super-chunk's bounds: in flight during pass A
            pass_a(buf, cbase, x0, x1, par);
            uint32_t excl = 0;
            if (more) excl = scan_runs_1<PPT>(sh, nnorm, ppt, ra, rb);
            if (2 * words < log_lo) log_lo = 2 * words;
            if (2 * words + R > log_dirty) log_dirty = 2 * words + R;
            __syncthreads();
            const uint32_t ncand = sh.ncand[par];
            if (tid == 0) sh.ncand[par ^ 1] = 0u;         // the next super-chunk's count
            if (once_counts || ncand > kRound) {
                mark(cbase, words, x0, x1);               // two barriers inside
                const int nr = sh.nrounds;
                for (int r = 0; r < nr; ++r) {
                    const uint32_t wlo = sh.wb[r];
                    const uint32_t whi = r == nr - 1 ? words : sh.wb[r + 1];
                    replay(R, wlo, whi);
                    __syncthreads();
                    slots_epilogue(cbase);
                    __syncthreads();
                }
                clear_words(twice, 0u, words);
            } else if (ncand) {
                replay(R, 0u, words);
                __syncthreads();
                slots_epilogue(cbase);
                clear_words(seen, 0u, words);
                clear_words(twice, 0u, words);
            } else {
                clear_words(seen, 0u, words);             // the twice plane is empty
            }
            if (more) scan_runs_2<THREADS, PPT>(sh, buf ^ 1, nnorm, ppt, excl, ra, rb);
            buf ^= 1;
            par ^= 1;
            c = nc;
            e = ne;
            __syncthreads();
        }
        // the unit's top-k: thread 0 merges the warps' lists
        __syncthreads();
        if (tid == 0) {
            int hd[nwarps];
#pragma unroll
            for (int w = 0; w < nwarps; ++w) hd[w] = 0;
            for (int r = 0; r < k; ++r) {
                int bw = -1;
                int64_t bk = INT64_MIN;
                uint32_t bp = 0xffffffffu, bpk = 0u;
#pragma unroll
                for (int w = 0; w < nwarps; ++w) {
                    if (hd[w] < wtop[w].n) {
                        const int64_t kk = wtop[w].key[hd[w]];
                        const uint32_t pp = wtop[w].pid[hd[w]];
                        if (bw < 0 || better(kk, pp, bk, bp)) { bw = w; bk = kk; bp = pp; bpk = wtop[w].pk[hd[w]]; }
                    }
                }
#pragma unroll
                for (int w = 0; w < nwarps; ++w)
                    if (w == bw) ++hd[w];
                UnitTop o;
                o.key = bw >= 0 ? bk : INT64_MIN;
                o.pid = bw >= 0 ? bp : 0xffffffffu;
                o.packed = bw >= 0 ? bpk : 0u;
                a.utop[u * k + r] = o;
            }
#pragma unroll
            for (int w = 0; w < nwarps; ++w) wtop[w].n = 0;
        }
        // histogram of this unit into the spectrum's histogram
        uint32_t mine = 0;
        for (int jb = tid; jb < (int)kHistBins; jb += THREADS) {
            const uint32_t h = sh.hist[jb];
            if (h) { atomicAdd(&a.hist[(uint64_t)q * kHistBins + jb], h); mine += h; sh.hist[jb] = 0; }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) mine += __shfl_xor_sync(0xffffffffu, mine, o);
        if (lane == 0 && mine) atomicAdd(&a.nscored[q], mine);
        __syncthreads();
    }
}
