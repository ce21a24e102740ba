// filter_2 + score + heap of superstep 3 (paper: Eq. 4 terms k32'..k34,
// Supplementary Algorithm 3), included by search_kernels.cuh.
//
// One persistent CTA pulls work units (spectrum q, peptide-id segment) from a
// device counter.  The segment is cut into super-chunks of whole skip-table
// columns (kChunk peptide ids each); the number of columns per super-chunk is
// chosen per unit from the skip tables so that a super-chunk holds about
// target_entries index entries of the spectrum's ordinary peaks.  Per
// super-chunk:
//   1. the run bounds of the next super-chunk are loaded first (their
//      latency hides behind step 2);
//   2. every index entry of the super-chunk (all ordinary peaks' runs laid end
//      to end by a prefix sum) is read once and adds (1 << 26 | iq) for a b ion
//      or (1 << 20 | iq) for a y ion to the peptide's 32-bit counter
//      (nb | ny | S), kept in shared memory: directly indexed for a single
//      column (16384 counters), or in an open-addressing table of 8192
//      64-bit slots (pid offset << 32 | counter) for wider super-chunks;
//      slots or counters that become non-zero go to a touched list;
//   3. the epilogue visits the touched counters, adds the hot peaks'
//      contributions from the bucket bitmaps, keeps peptides with
//      nb + ny >= min_shared, ranks them with the exact key
//      K = LF[nb] + LF[ny] + LS[S], updates the thread's top-k and the shared
//      histogram, and clears what it visited.
// A super-chunk whose entries exceed kMaxEntries is redone column by column
// with direct counters, so the table never holds more than kMaxEntries keys
// (< kSlots: probing always ends).  Hot peaks (buckets holding >= 1/32 of
// the database) never touch the counters; when the spectrum has at least
// min_shared of them a peptide can qualify through bitmaps alone, and the unit
// then runs column by column with a dense epilogue that also tests the
// bitmaps.

constexpr int kMaxHot = 6;                 // bitmap slices (b or y bitmap of a hot bucket) per spectrum
constexpr int kMaxWarps = 16;              // CTAs of up to 512 threads
constexpr int kTouchCap = 4096;            // touched list of one super-chunk
constexpr uint32_t kSlots = 8192;          // hash slots: 64 KB, the same bytes as kChunk counters
constexpr uint32_t kMaxEntries = 6144;     // most entries a hashed super-chunk may hold
constexpr uint32_t kMaxCols = 64;          // widest super-chunk (columns of kChunk ids)

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
    uint32_t min_shared;
    uint32_t k;
    uint32_t target_entries;    // entries aimed for per super-chunk
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
    // sorted by (key desc, pid asc); keeps the best k
    __device__ __forceinline__ void insert(int64_t kk, uint32_t p, uint32_t packed, int k) {
        int pos = 0;
#pragma unroll
        for (int i = 0; i < KMAX; ++i)
            if (i < n && (key[i] > kk || (key[i] == kk && pid[i] < p))) pos = i + 1;
        if (pos >= k) return;
#pragma unroll
        for (int i = KMAX - 1; i > 0; --i)
            if (i > pos) { key[i] = key[i - 1]; pid[i] = pid[i - 1]; pk[i] = pk[i - 1]; }
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
    uint64_t pbase[kMaxTopN];         // bucket start of each ordinary peak
    uint32_t prow[kMaxTopN];          // its skip-table row
    uint32_t pinc[kMaxTopN];          // its quantised intensity
    uint32_t pre[2][kMaxTopN + 1];    // exclusive prefix of the run lengths (parity)
    uint32_t rs[2][kMaxTopN];         // run starts relative to the bucket (parity)
    union {
        uint16_t touched[kTouchCap];  // slots / counters that became non-zero
        uint16_t hotc[kMaxTopN];      // (classification) hot peaks: index into qbin
    };
    uint16_t wli[2][kMaxWarps];       // peak holding each warp's first entry (parity)
    int ntouched;                     // > kTouchCap means the list overflowed
    const uint32_t* slice[kMaxHot];   // bitmap rows of the spectrum's hot slices
    uint32_t slice_inc[kMaxHot];      // counter increment of a set bit
    uint32_t hist[kHistBins];
    int64_t lf[kMaxLen + 1];
    int64_t wkey[kMaxWarps];
    uint32_t wpid[kMaxWarps];
    uint32_t wpk[kMaxWarps];
    uint32_t wsum[kMaxWarps];
    int nnorm, nhotc, nslices, nhotpeaks;
    uint64_t unit;
    uint32_t q, np;
    uint32_t seg_lo, seg_hi;
};

__device__ __forceinline__ uint32_t counter_inc(uint32_t e, uint32_t iq) {
    return iq + ((e & 1u) ? (1u << kNyShift) : (1u << kNbShift));
}

__device__ __forceinline__ uint32_t slot_of(uint32_t off) { return (off * 2654435761u) >> 19; }   // 13 bits

// Exclusive scan of the ordinary peaks' run lengths, in two halves around a
// barrier the caller provides.  Thread tid owns peaks tid*ppt .. +ppt-1.
template <int PPT>
__device__ __forceinline__ uint32_t scan_runs_1(SearchShared& sh, int nnorm, int ppt, const uint32_t (&ra)[PPT],
                                                const uint32_t (&rb)[PPT]) {
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    uint32_t sum = 0;
#pragma unroll
    for (int i = 0; i < PPT; ++i) {
        const int t = tid * ppt + i;
        if (i < ppt && t < nnorm) sum += rb[i] - ra[i];
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

template <int THREADS, int PPT>
__device__ __forceinline__ void scan_runs_2(SearchShared& sh, int buf, int nnorm, int ppt, uint32_t excl,
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
    const uint32_t per = (total + nwarps - 1) / nwarps;
    uint32_t run = wbase + excl;
#pragma unroll
    for (int i = 0; i < PPT; ++i) {
        const int t = tid * ppt + i;
        if (i < ppt && t < nnorm) {
            const uint32_t len = rb[i] - ra[i];
            sh.pre[buf][t] = run;
            sh.rs[buf][t] = ra[i];
            if (len)   // warps whose share starts inside this run
                for (uint32_t w = (run + per - 1) / per; w * per < run + len && w < (uint32_t)nwarps; ++w)
                    sh.wli[buf][w] = (uint16_t)t;
            run += len;
        }
    }
    if (tid == 0) sh.pre[buf][nnorm] = total;
}

template <int KMAX, int THREADS>
__global__ void __launch_bounds__(THREADS, THREADS <= 256 ? 2 : 1) search_kernel(SearchArgs a) {
    extern __shared__ __align__(16) unsigned long long tab[];   // kSlots slots, or 2 * kSlots direct counters
    uint32_t* const cnt = reinterpret_cast<uint32_t*>(tab);
    __shared__ SearchShared sh;
    constexpr int nwarps = THREADS / 32;
    constexpr int PPT = kMaxTopN / THREADS;             // ordinary peaks per thread (at most)
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const unsigned lt = (1u << lane) - 1u;
    const uint32_t last_col = a.skip_stride - 1;
    for (int i = tid; i < (int)kSlots; i += THREADS) tab[i] = 0ull;
    for (int i = tid; i < (int)kHistBins; i += THREADS) sh.hist[i] = 0;
    for (int i = tid; i <= (int)kMaxLen; i += THREADS) sh.lf[i] = a.lf[i];
    const uint64_t total_units = a.seg_off[a.n];
    const int k = (int)a.k;
    const uint32_t min_shared = a.min_shared;
    __syncthreads();
    for (;;) {
        if (tid == 0) {
            const uint64_t u = atomicAdd(a.work, 1ull);
            sh.unit = u;
            sh.nnorm = 0;
            sh.nhotc = 0;
            sh.nslices = 0;
            sh.nhotpeaks = 0;
            sh.ntouched = 0;
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
            sh.pbase[s] = a.off[bin];
            sh.prow[s] = (uint32_t)row;
            sh.pinc[s] = a.qiq[(uint64_t)q * a.topn + t];
        }
        __syncthreads();
        if (tid == 0) {
            // bitmap slices in peak order while they last; the rest are ordinary
            int ns = 0, nh = 0;
            for (int c = 0; c < sh.nhotc; ++c) {
                const uint32_t t = sh.hotc[c];
                const uint32_t bin = a.qbin[(uint64_t)q * a.topn + t];
                const uint32_t iq = a.qiq[(uint64_t)q * a.topn + t];
                const int32_t hid = a.hot_id[bin];
                const uint32_t fl = a.hot_flags[hid];
                const int need = (fl & 1u ? 1 : 0) + (fl & 2u ? 1 : 0);
                if (ns + need <= kMaxHot) {
                    if (fl & 1u) { sh.slice[ns] = a.hot_b + (uint64_t)hid * a.hot_words; sh.slice_inc[ns++] = (1u << kNbShift) + iq; }
                    if (fl & 2u) { sh.slice[ns] = a.hot_y + (uint64_t)hid * a.hot_words; sh.slice_inc[ns++] = (1u << kNyShift) + iq; }
                    ++nh;
                } else {
                    const int s = sh.nnorm++;
                    sh.pbase[s] = a.off[bin];
                    sh.prow[s] = (uint32_t)a.skip_row[bin];
                    sh.pinc[s] = iq;
                }
            }
            sh.nslices = ns;
            sh.nhotpeaks = nh;
        }
        __syncthreads();
        const int nnorm = sh.nnorm, nslices = sh.nslices;
        const bool hot_alone = sh.nhotpeaks >= (int)min_shared;
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
            if (!hot_alone) {
                uint64_t want = total ? ((uint64_t)a.target_entries * ncols) / total : ncols;
                if (want < 1) want = 1;
                if (want > kMaxCols) want = kMaxCols;
                m = min((uint32_t)want, ncols);
            }
            __syncthreads();   // wsum is reused by the scans
        }
        TopK<KMAX> top;
        top.init();

        // entries of super-chunk [cbase, cbase + span) clipped to [x0, x1);
        // direct counters when dense, otherwise the hash table
        auto accumulate = [&](int buf, uint32_t cbase, uint32_t x0, uint32_t x1, bool dense) {
            const uint32_t R = sh.pre[buf][nnorm];
            const uint32_t per = (R + nwarps - 1) / nwarps;
            const uint32_t f0 = (uint32_t)warp * per, f1 = min(R, f0 + per);
            int li = 0;
            if (f0 < f1) {
                li = sh.wli[buf][warp];
                const uint32_t fs = f0 + lane;
                if (fs < f1)
                    while (sh.pre[buf][li + 1] <= fs) ++li;
            }
            for (uint32_t fb = f0; fb < f1; fb += 4 * 32) {   // uniform across the warp
                uint32_t e[4], inc[4];
#pragma unroll
                for (int r = 0; r < 4; ++r) {
                    const uint32_t ff = fb + r * 32 + lane;
                    e[r] = 0xffffffffu;
                    inc[r] = 0;
                    if (ff < f1) {
                        while (sh.pre[buf][li + 1] <= ff) ++li;
                        e[r] = __ldg(a.entry + sh.pbase[li] + sh.rs[buf][li] + (ff - sh.pre[buf][li]));
                        inc[r] = sh.pinc[li];
                    }
                }
#pragma unroll
                for (int r = 0; r < 4; ++r) {
                    const uint32_t pid = e[r] >> 1;
                    const bool act = pid >= x0 && pid < x1;
                    bool first = false;
                    uint32_t where = 0;
                    if (act) {
                        const uint32_t off = pid - cbase;
                        const uint32_t v = counter_inc(e[r], inc[r]);
                        if (dense) {
                            first = atomicAdd(&cnt[off], v) == 0u;
                            where = off;
                        } else {
                            const unsigned long long item = ((unsigned long long)off << 32) | v;
                            uint32_t sl = slot_of(off);
                            for (uint32_t probe = 0; probe < kSlots; ++probe) {
                                const unsigned long long old = atomicCAS(&tab[sl], 0ull, item);
                                if (old == 0ull) { first = true; break; }
                                if ((uint32_t)(old >> 32) == off) { atomicAdd(&tab[sl], (unsigned long long)v); break; }
                                sl = (sl + 1) & (kSlots - 1);
                            }
                            where = sl;
                        }
                    }
                    const unsigned bal = __ballot_sync(0xffffffffu, first);
                    if (bal) {
                        const int leader = __ffs(bal) - 1;
                        int base = 0;
                        if (lane == leader) base = atomicAdd(&sh.ntouched, __popc(bal));
                        base = __shfl_sync(0xffffffffu, base, leader);
                        const int slot = base + __popc(bal & lt);
                        if (first && slot < kTouchCap) sh.touched[slot] = (uint16_t)where;
                    }
                }
            }
        };
        auto score = [&](uint32_t c, uint32_t pid) {
            const uint32_t nb = c >> kNbShift, ny = (c >> kNyShift) & 63u;
            if (nb + ny >= min_shared) {
                const uint32_t S = c & kSMask;
                const int64_t K = sh.lf[nb] + sh.lf[ny] + __ldg(a.ls + S);
                const int64_t hb = K >> 31;
                atomicAdd(&sh.hist[hb > 255 ? 255 : (hb < 0 ? 0 : hb)], 1u);
                top.insert(K, pid, c, k);
            }
        };
        // one counter (c, pid): filter, add the hot slices, score
        auto visit = [&](uint32_t c, uint32_t pid) {
            const uint32_t nn = (c >> kNbShift) + ((c >> kNyShift) & 63u);
            if (nn + (uint32_t)nslices < min_shared) return;
            for (int s = 0; s < nslices; ++s)
                if ((__ldg(sh.slice[s] + (pid >> 5)) >> (pid & 31)) & 1u) c += sh.slice_inc[s];
            score(c, pid);
        };
        // epilogue of a super-chunk; clears what it visits
        auto epilogue = [&](uint32_t cbase, uint32_t x0, uint32_t x1, bool dense) {
            const int nt = sh.ntouched;
            if (nt <= kTouchCap && !hot_alone) {
                for (int i = tid; i < nt; i += THREADS) {
                    const uint32_t w = sh.touched[i];
                    if (dense) {
                        const uint32_t c = cnt[w];
                        cnt[w] = 0u;
                        visit(c, cbase + w);
                    } else {
                        const unsigned long long v = tab[w];
                        tab[w] = 0ull;
                        visit((uint32_t)v, cbase + (uint32_t)(v >> 32));
                    }
                }
            } else if (!dense) {
                for (uint32_t i = tid; i < kSlots; i += THREADS) {
                    const unsigned long long v = tab[i];
                    if (v == 0ull) continue;
                    tab[i] = 0ull;
                    visit((uint32_t)v, cbase + (uint32_t)(v >> 32));
                }
            } else {
                // every counter of the column, 32 peptide ids per step; with
                // >= min_shared hot peaks the bitmaps alone can qualify a peptide
                for (uint32_t gi = tid; gi < kChunk / 32; gi += THREADS) {
                    const uint32_t gp = cbase + (gi << 5);
                    if (gp + 32 <= x0 || gp >= x1) continue;
                    const uint32_t lo_b = x0 > gp ? x0 - gp : 0u;
                    const uint32_t hi_b = x1 - gp >= 32u ? 32u : x1 - gp;
                    const uint32_t valid = (hi_b >= 32u ? 0xffffffffu : ((1u << hi_b) - 1u)) & ~((1u << lo_b) - 1u);
                    uint32_t hw[kMaxHot];
#pragma unroll
                    for (int s = 0; s < kMaxHot; ++s) hw[s] = s < nslices ? __ldg(sh.slice[s] + (gp >> 5)) : 0u;
                    uint32_t cand = 0;
                    for (int j = 0; j < 32; ++j) {
                        const int jb = (j + lane) & 31;   // rotated: lanes hit different banks
                        const uint32_t c = cnt[(gi << 5) + jb];
                        uint32_t hc = 0;
#pragma unroll
                        for (int s = 0; s < kMaxHot; ++s) hc += (hw[s] >> jb) & 1u;
                        const uint32_t nn = (c >> kNbShift) + ((c >> kNyShift) & 63u);
                        if ((c != 0u || hc > 0u) && nn + hc >= min_shared) cand |= 1u << jb;
                    }
                    cand &= valid;
                    while (cand) {
                        const int jb = __ffs(cand) - 1;
                        cand &= cand - 1;
                        uint32_t c = cnt[(gi << 5) + jb];
#pragma unroll
                        for (int s = 0; s < kMaxHot; ++s)
                            if ((hw[s] >> jb) & 1u) c += sh.slice_inc[s];
                        score(c, gp + jb);
                    }
#pragma unroll 4
                    for (int j = 0; j < 32; ++j) cnt[(gi << 5) + ((j + lane) & 31)] = 0u;
                }
            }
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
            if (R > kMaxEntries && e - c > 1) {
                // too many entries for the table: this super-chunk column by column
                for (uint32_t cc = c; cc < e; ++cc) {
                    load_runs(cc, cc + 1);
                    const uint32_t excl = scan_runs_1<PPT>(sh, nnorm, ppt, ra, rb);
                    __syncthreads();
                    scan_runs_2<THREADS, PPT>(sh, buf ^ 1, nnorm, ppt, excl, ra, rb);
                    __syncthreads();
                    const uint32_t cb = cc << kChunkShift;
                    const uint32_t x0 = max(seg_lo, cb), x1 = min(seg_hi, cb + kChunk);
                    accumulate(buf ^ 1, cb, x0, x1, true);
                    __syncthreads();
                    epilogue(cb, x0, x1, true);
                    __syncthreads();
                    if (tid == 0) sh.ntouched = 0;
                    __syncthreads();
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
            const bool dense = (e - c) == 1;
            const uint32_t cbase = c << kChunkShift;
            const uint32_t x0 = max(seg_lo, cbase), x1 = min(seg_hi, e << kChunkShift);
            const uint32_t nc = e, ne = min(e + m, col_end);
            const bool more = nc < col_end;
            if (more) load_runs(nc, ne);                 // next super-chunk's bounds
            accumulate(buf, cbase, x0, x1, dense);
            uint32_t excl = 0;
            if (more) excl = scan_runs_1<PPT>(sh, nnorm, ppt, ra, rb);
            __syncthreads();
            epilogue(cbase, x0, x1, dense);
            if (more) scan_runs_2<THREADS, PPT>(sh, buf ^ 1, nnorm, ppt, excl, ra, rb);
            __syncthreads();
            if (tid == 0) sh.ntouched = 0;
            buf ^= 1;
            c = nc;
            e = ne;
            // the next accumulate appends to ntouched: make the reset visible
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
