// filter_2 + score + heap of superstep 3 (paper: Eq. 4 terms k32'..k34,
// Supplementary Algorithm 3), included by search.cu.
//
// One persistent CTA pulls work units (spectrum q, peptide-id segment) from a
// device counter.  A segment is walked in chunks of kChunk peptide ids
// aligned to multiples of kChunk; per chunk:
//   1. every ordinary peak reads its bucket's run for this chunk from the
//      chunk skip table (two adjacent words, no search); runs of up to
//      kShortRun entries are accumulated by the thread that owns the peak,
//      longer runs are listed and spread over all warps;
//   2. each entry adds (1 << 26 | iq) for a b ion or (1 << 20 | iq) for a y
//      ion to the peptide's 32-bit counter in shared memory (nb | ny | S);
//   3. the epilogue walks the chunk 32 peptides at a time, adds the hot
//      peaks' contributions from the bucket bitmaps, keeps peptides with
//      nb + ny >= min_shared, ranks them with the exact key
//      K = LF[nb] + LF[ny] + LS[S], updates the thread's top-k and the
//      shared histogram, and clears the counters.
// Hot peaks (buckets holding >= 1/32 of the database, up to kMaxHot per
// spectrum) never touch the counters: a peptide can only reach min_shared
// through them alone when the spectrum has >= min_shared hot peaks, which
// the epilogue checks with the bitmaps.

constexpr int kMaxHot = 8;
constexpr int kShortRun = 8;
constexpr int kMaxWarps = 16;           // CTAs of up to 512 threads

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
    uint32_t chunk_mult;        // counters per CTA = chunk_mult * kChunk
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
    uint64_t pbase[kMaxTopN];     // bucket start of each ordinary peak
    uint32_t prow[kMaxTopN];      // its skip-table row
    uint32_t pinc[kMaxTopN];      // its quantised intensity
    uint32_t rs[kMaxTopN];        // run start (relative to the bucket) in this chunk
    uint32_t longp[kMaxTopN];     // peaks with a long run in this chunk
    uint32_t lpre[kMaxTopN + 1];  // exclusive prefix of the long runs' lengths
    int32_t hot[kMaxHot];
    uint32_t hot_inc[kMaxHot];
    uint32_t hot_fl[kMaxHot];
    uint32_t hist[kHistBins];
    int64_t lf[kMaxLen + 1];
    int64_t wkey[kMaxWarps];
    uint32_t wpid[kMaxWarps];
    uint32_t wpk[kMaxWarps];
    int nnorm, nhot, nlong;
    uint64_t unit;
    uint32_t q, np;
    uint32_t seg_lo, seg_hi;
};

__device__ __forceinline__ uint32_t counter_inc(uint32_t e, uint32_t iq) {
    return iq + ((e & 1u) ? (1u << kNyShift) : (1u << kNbShift));
}

template <int KMAX, int THREADS>
__global__ void __launch_bounds__(THREADS) search_kernel(SearchArgs a) {
    extern __shared__ __align__(16) uint32_t cnt[];   // chunk_mult * kChunk counters
    __shared__ SearchShared sh;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    constexpr int nwarps = THREADS / 32;
    const uint32_t cm = a.chunk_mult;
    const uint32_t span = kChunk * cm;
    const uint32_t last_col = a.skip_stride - 1;
    for (int i = tid; i < (int)span; i += THREADS) cnt[i] = 0;
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
            sh.nhot = 0;
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
        // classify the retained peaks: hot (bitmap) or ordinary (skip table)
        for (uint32_t t = tid; t < np; t += THREADS) {
            const uint32_t bin = a.qbin[(uint64_t)q * a.topn + t];
            const uint32_t iq = a.qiq[(uint64_t)q * a.topn + t];
            const int32_t hid = a.hot_id[bin];
            if (hid >= 0) {
                const int s = atomicAdd(&sh.nhot, 1);
                if (s < kMaxHot) {
                    sh.hot[s] = hid;
                    sh.hot_inc[s] = iq;
                    sh.hot_fl[s] = a.hot_flags[hid];
                    continue;
                }
            }
            const int32_t row = a.skip_row[bin];
            if (row < 0) continue;   // empty bucket
            const int s = atomicAdd(&sh.nnorm, 1);
            sh.pbase[s] = a.off[bin];
            sh.prow[s] = (uint32_t)row;
            sh.pinc[s] = iq;
        }
        TopK<KMAX> top;
        top.init();
        __syncthreads();
        const int nhot = min(sh.nhot, kMaxHot);
        const int nnorm = sh.nnorm;
        const uint32_t j_first = (seg_lo >> kChunkShift) / cm, j_last = ((seg_hi - 1) >> kChunkShift) / cm;
        for (uint32_t j = j_first; j <= j_last; ++j) {
            const uint32_t cbase = (j * cm) << kChunkShift;
            const uint32_t c0 = max(seg_lo, cbase), c1 = min(seg_hi, cbase + span);
            const uint32_t col0 = j * cm, col1 = min(col0 + cm, last_col);
            if (tid == 0) sh.nlong = 0;
            __syncthreads();
            // 1. runs of this chunk; short runs accumulated here
            for (int t = tid; t < nnorm; t += THREADS) {
                const uint32_t* sk = a.skip + (uint64_t)sh.prow[t] * a.skip_stride;
                const uint32_t ra = __ldg(sk + col0), rb = __ldg(sk + col1);
                const uint32_t len = rb - ra;
                if (len <= (uint32_t)kShortRun) {
                    const uint32_t* ep = a.entry + sh.pbase[t] + ra;
                    uint32_t v[kShortRun];
#pragma unroll
                    for (int i = 0; i < kShortRun; ++i) v[i] = (uint32_t)i < len ? __ldg(ep + i) : 0xffffffffu;
                    const uint32_t iq = sh.pinc[t];
#pragma unroll
                    for (int i = 0; i < kShortRun; ++i) {
                        const uint32_t pid = v[i] >> 1;
                        if ((uint32_t)i < len && pid >= c0 && pid < c1) atomicAdd(&cnt[pid - cbase], counter_inc(v[i], iq));
                    }
                } else {
                    const int s = atomicAdd(&sh.nlong, 1);
                    sh.longp[s] = (uint32_t)t;
                    sh.rs[t] = ra;
                    sh.lpre[s + 1] = len;
                }
            }
            __syncthreads();
            // 2. long runs spread over the warps
            const int nl = sh.nlong;
            if (nl > 0) {
                if (warp == 0) {
                    uint32_t carry = 0;
                    for (int b = 0; b < nl; b += 32) {
                        const int i = b + lane;
                        uint32_t v = i < nl ? sh.lpre[i + 1] : 0u;
#pragma unroll
                        for (int o = 1; o < 32; o <<= 1) {
                            const uint32_t x = __shfl_up_sync(0xffffffffu, v, o);
                            if (lane >= o) v += x;
                        }
                        if (i < nl) sh.lpre[i + 1] = carry + v;
                        carry += __shfl_sync(0xffffffffu, v, 31);
                    }
                    if (lane == 0) sh.lpre[0] = 0;
                }
                __syncthreads();
                const uint32_t R = sh.lpre[nl];
                const uint32_t per = (R + nwarps - 1) / nwarps;
                const uint32_t f0 = (uint32_t)warp * per, f1 = min(R, f0 + per);
                if (f0 + lane < f1) {
                    // long run holding flat index f0 + lane
                    int li = 0, hi_i = nl;
                    const uint32_t fs = f0 + lane;
                    while (hi_i - li > 1) {
                        const int m = (li + hi_i) >> 1;
                        if (sh.lpre[m] <= fs) li = m; else hi_i = m;
                    }
                    for (uint32_t f = fs; f < f1; f += 32) {
                        while (sh.lpre[li + 1] <= f) ++li;
                        const uint32_t t = sh.longp[li];
                        const uint32_t e = __ldg(a.entry + sh.pbase[t] + sh.rs[t] + (f - sh.lpre[li]));
                        const uint32_t pid = e >> 1;
                        if (pid >= c0 && pid < c1) atomicAdd(&cnt[pid - cbase], counter_inc(e, sh.pinc[t]));
                    }
                }
            }
            __syncthreads();
            // 3. epilogue, 32 peptide ids per step
            const uint32_t g0 = (c0 - cbase) >> 5, g1 = (c1 - cbase + 31) >> 5;
            for (uint32_t g = g0 + tid; g < g1; g += THREADS) {
                const uint32_t gp = cbase + (g << 5);
                uint4* c4 = reinterpret_cast<uint4*>(&cnt[g << 5]);
                uint32_t nz = 0;
                uint32_t nzq = 0;   // which of the 8 uint4 words are non-zero
#pragma unroll
                for (int w4 = 0; w4 < 8; ++w4) {
                    const uint4 v = c4[w4];
                    const uint32_t m = (v.x ? 1u : 0u) | (v.y ? 2u : 0u) | (v.z ? 4u : 0u) | (v.w ? 8u : 0u);
                    nz |= m << (4 * w4);
                    nzq |= (m ? 1u : 0u) << w4;
                }
                const uint32_t lo_b = c0 > gp ? c0 - gp : 0u;
                const uint32_t hi_b = c1 - gp >= 32u ? 32u : c1 - gp;
                const uint32_t valid = (hi_b >= 32u ? 0xffffffffu : ((1u << hi_b) - 1u)) & ~((1u << lo_b) - 1u);
                uint32_t wb[kMaxHot], wy[kMaxHot];
                const uint64_t word = gp >> 5;
#pragma unroll
                for (int h = 0; h < kMaxHot; ++h) {
                    wb[h] = 0;
                    wy[h] = 0;
                    if (h < nhot) {
                        const uint64_t o = (uint64_t)sh.hot[h] * a.hot_words + word;
                        if (sh.hot_fl[h] & 1u) wb[h] = __ldg(a.hot_b + o) & valid;
                        if (sh.hot_fl[h] & 2u) wy[h] = __ldg(a.hot_y + o) & valid;
                    }
                }
                uint32_t cand = nz & valid;
                if (nhot >= (int)min_shared) {
                    // peptides reaching min_shared through hot peaks alone
                    for (int jb = 0; jb < 32; ++jb) {
                        uint32_t hc = 0;
#pragma unroll
                        for (int h = 0; h < kMaxHot; ++h) hc += ((wb[h] | wy[h]) >> jb) & 1u;
                        if (hc >= min_shared) cand |= 1u << jb;
                    }
                }
                while (cand) {
                    const int jb = __ffs(cand) - 1;
                    cand &= cand - 1;
                    uint32_t c = cnt[(g << 5) + jb];
#pragma unroll
                    for (int h = 0; h < kMaxHot; ++h) {
                        if ((wb[h] >> jb) & 1u) c += (1u << kNbShift) + sh.hot_inc[h];
                        if ((wy[h] >> jb) & 1u) c += (1u << kNyShift) + sh.hot_inc[h];
                    }
                    const uint32_t nb = c >> kNbShift, ny = (c >> kNyShift) & 63u;
                    if (nb + ny >= min_shared) {
                        const uint32_t S = c & kSMask;
                        const int64_t K = sh.lf[nb] + sh.lf[ny] + __ldg(a.ls + S);
                        const int64_t hb = K >> 31;
                        atomicAdd(&sh.hist[hb > 255 ? 255 : (hb < 0 ? 0 : hb)], 1u);
                        top.insert(K, gp + jb, c, k);
                    }
                }
#pragma unroll
                for (int w4 = 0; w4 < 8; ++w4)
                    if ((nzq >> w4) & 1u) c4[w4] = make_uint4(0, 0, 0, 0);
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
