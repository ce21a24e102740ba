// Device side of superstep 1 (paper: Supplementary Algorithm 1,
// model_spectrum + parallel_index): b/y model spectra for every database
// entry, integer m/z binning, and the fragment-ion index as a CSR whose
// buckets list peptide ids in ascending order.  The paper indexes with a
// CFIR-style inverted index built by a parallel sort; here the sort is a
// stable LSD radix sort by bin over (bin, pid, isY) keys emitted in pid
// order, so each bucket comes out pid-ascending without a comparison sort.
#include <algorithm>
#include <new>
#include <cmath>
#include <chrono>
#include <vector>

#include "dev_common.cuh"

namespace hicops {
namespace {

constexpr int kIonThreads = 256;

struct IonArgs {
    const uint32_t* base;        // [P] base peptide id
    const uint64_t* mask;        // [P] modified-position mask
    const uint64_t* base_off;    // [B+1]
    const char* residues;        // concatenated base sequences
    const double* mres;          // [128]
    const double* mmod;          // [128]
    double w, mz_lo, mz_hi;
    uint64_t P;
};

// Visits the distinct in-range ion bins of one peptide in ascending bin
// order; a bin reached by both a b and a y ion is reported once, as b.
// b_i = (m_1 + .. + m_i) + proton, summed left to right;
// y_i = ((m_L + m_{L-1} + .. + m_{i+1}) + H2O) + proton, summed from the C terminus.
template <class F>
__device__ __forceinline__ void for_each_ion_bin(const IonArgs& a, const double* mres, const double* mmod,
                                                 uint64_t pid, F&& emit) {
    const uint32_t b = a.base[pid];
    const uint64_t m = a.mask[pid];
    const char* s = a.residues + a.base_off[b];
    const int L = (int)(a.base_off[b + 1] - a.base_off[b]);
    auto rm = [&](int j) -> double {
        const unsigned char c = (unsigned char)s[j];
        return ((m >> j) & 1ull) ? mmod[c] : mres[c];
    };
    // b stream state: next ion index ib (1..L-1), running prefix
    int ib = 1;
    double pre = 0.0;
    // y stream state: next ion index iy (L-1 down to 1), running suffix
    int iy = L - 1;
    double suf = 0.0;
    uint32_t bb = 0, by = 0;
    bool hb = false, hy = false;
    auto next_b = [&]() -> bool {
        while (ib <= L - 1) {
            pre = pre + rm(ib - 1);
            const double mz = pre + kProtonDa;
            ++ib;
            if (mz < a.mz_lo) continue;
            if (mz >= a.mz_hi) { ib = L; return false; }
            bb = (uint32_t)floor(mz / a.w);
            return true;
        }
        return false;
    };
    auto next_y = [&]() -> bool {
        while (iy >= 1) {
            suf = suf + rm(iy);
            const double mz = (suf + kWaterDa) + kProtonDa;
            --iy;
            if (mz < a.mz_lo) continue;
            if (mz >= a.mz_hi) { iy = 0; return false; }
            by = (uint32_t)floor(mz / a.w);
            return true;
        }
        return false;
    };
    hb = next_b();
    hy = next_y();
    uint32_t last = 0xffffffffu;
    while (hb || hy) {
        if (hb && (!hy || bb <= by)) {
            if (bb != last) { emit(bb, 0u); last = bb; }
            hb = next_b();
        } else {
            if (by != last) { emit(by, 1u); last = by; }
            hy = next_y();
        }
    }
}

__global__ void ion_count_kernel(IonArgs a, uint32_t* __restrict__ count) {
    __shared__ double smres[128], smmod[128];
    for (int i = threadIdx.x; i < 128; i += blockDim.x) { smres[i] = a.mres[i]; smmod[i] = a.mmod[i]; }
    __syncthreads();
    const uint64_t pid = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (pid >= a.P) return;
    uint32_t n = 0;
    for_each_ion_bin(a, smres, smmod, pid, [&](uint32_t, uint32_t) { ++n; });
    count[pid] = n;
}

__global__ void ion_emit_kernel(IonArgs a, const uint64_t* __restrict__ off, uint64_t* __restrict__ keys) {
    __shared__ double smres[128], smmod[128];
    for (int i = threadIdx.x; i < 128; i += blockDim.x) { smres[i] = a.mres[i]; smmod[i] = a.mmod[i]; }
    __syncthreads();
    const uint64_t pid = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (pid >= a.P) return;
    uint64_t o = off[pid];
    for_each_ion_bin(a, smres, smmod, pid, [&](uint32_t bin, uint32_t isy) {
        keys[o++] = ((uint64_t)bin << 32) | (uint64_t)((uint32_t)(pid << 1) | isy);
    });
}

// ---- stable LSD radix sort on the bin field (bits 32..) of 64-bit keys

constexpr int kRsBits = 8;
constexpr int kRsRadix = 1 << kRsBits;
constexpr int kRsWarps = 8;
constexpr int kRsRounds = 16;
constexpr int kRsTile = kRsWarps * 32 * kRsRounds;

__device__ __forceinline__ uint32_t digit_of(uint64_t k, int shift) {
    return (uint32_t)(k >> shift) & (kRsRadix - 1);
}

// counts[d * ntiles + tile] = number of keys of tile with digit d
__global__ void __launch_bounds__(kRsWarps * 32) rs_count_kernel(const uint64_t* __restrict__ keys, uint64_t n,
                                                                 int shift, uint32_t* __restrict__ counts,
                                                                 uint64_t ntiles) {
    __shared__ uint32_t h[kRsRadix];
    for (int i = threadIdx.x; i < kRsRadix; i += blockDim.x) h[i] = 0;
    __syncthreads();
    const uint64_t base = (uint64_t)blockIdx.x * kRsTile;
    for (int i = threadIdx.x; i < kRsTile; i += blockDim.x) {
        const uint64_t g = base + i;
        if (g < n) atomicAdd(&h[digit_of(keys[g], shift)], 1u);
    }
    __syncthreads();
    for (int d = threadIdx.x; d < kRsRadix; d += blockDim.x) counts[(uint64_t)d * ntiles + blockIdx.x] = h[d];
}

// Stable scatter: warp w owns items [w*32*R, (w+1)*32*R) of the tile and
// walks them in order, 32 at a time; equal digits inside a round are ranked
// by lane.
__global__ void __launch_bounds__(kRsWarps * 32) rs_scatter_kernel(const uint64_t* __restrict__ in,
                                                                   uint64_t* __restrict__ out, uint64_t n,
                                                                   int shift, const uint64_t* __restrict__ offs,
                                                                   uint64_t ntiles) {
    __shared__ uint32_t wcount[kRsWarps][kRsRadix];
    __shared__ uint64_t tile_base[kRsRadix];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int i = threadIdx.x; i < kRsWarps * kRsRadix; i += blockDim.x) (&wcount[0][0])[i] = 0;
    for (int d = threadIdx.x; d < kRsRadix; d += blockDim.x) tile_base[d] = offs[(uint64_t)d * ntiles + blockIdx.x];
    __syncthreads();
    const uint64_t wbase = (uint64_t)blockIdx.x * kRsTile + (uint64_t)w * 32 * kRsRounds;
    const unsigned lt = (1u << lane) - 1u;
    // pass 1: per-warp digit counts
    for (int r = 0; r < kRsRounds; ++r) {
        const uint64_t g = wbase + (uint64_t)r * 32 + lane;
        const uint32_t d = g < n ? digit_of(in[g], shift) : 0xffffu;
        const unsigned peers = __match_any_sync(0xffffffffu, d);
        if (d != 0xffffu && (peers & lt) == 0) wcount[w][d] += __popc(peers);
        __syncwarp();
    }
    __syncthreads();
    // exclusive prefix over warps, per digit
    for (int d = threadIdx.x; d < kRsRadix; d += blockDim.x) {
        uint32_t run = 0;
        for (int ww = 0; ww < kRsWarps; ++ww) {
            uint32_t c = wcount[ww][d];
            wcount[ww][d] = run;
            run += c;
        }
    }
    __syncthreads();
    // pass 2: scatter
    for (int r = 0; r < kRsRounds; ++r) {
        const uint64_t g = wbase + (uint64_t)r * 32 + lane;
        uint64_t k = 0;
        uint32_t d = 0xffffu;
        if (g < n) { k = in[g]; d = digit_of(k, shift); }
        const unsigned peers = __match_any_sync(0xffffffffu, d);
        uint32_t before = 0;
        if (d != 0xffffu) before = wcount[w][d];
        __syncwarp();
        if (d != 0xffffu) {
            out[tile_base[d] + before + __popc(peers & lt)] = k;
            if ((peers & lt) == 0) wcount[w][d] = before + __popc(peers);
        }
        __syncwarp();
    }
}

// off[b] = first position whose bin is >= b (keys sorted by bin)
__global__ void bucket_off_kernel(const uint64_t* __restrict__ keys, uint64_t n, uint32_t nbins,
                                  uint64_t* __restrict__ off) {
    const uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i > n) return;
    const int64_t prev = i == 0 ? -1 : (int64_t)(keys[i - 1] >> 32);
    const int64_t cur = i == n ? (int64_t)nbins : (int64_t)(keys[i] >> 32);
    for (int64_t b = prev + 1; b <= cur; ++b) off[b] = i;
}

// Bucket sizes rounded up to whole groups of 4 entries (16 bytes), so that
// every bucket starts 16-byte aligned in the entry array.
__global__ void padded_size_kernel(const uint64_t* __restrict__ off, uint32_t nbins, uint32_t* __restrict__ psz) {
    const uint32_t b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b < nbins) psz[b] = (uint32_t)((off[b + 1] - off[b] + 3) & ~3ull);
}

// entry[poff[bin] + rank in bucket] = pid << 1 | isY; the up to 3 slots after
// a bucket's last entry keep the pad value 0xffffffff (pid 2^31 - 1, above
// every peptide id, so a bucket stays pid-sorted and no window contains it).
__global__ void take_low_kernel(const uint64_t* __restrict__ keys, uint64_t n, const uint64_t* __restrict__ off,
                                const uint64_t* __restrict__ poff, uint32_t* __restrict__ entry) {
    const uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const uint32_t bin = (uint32_t)(keys[i] >> 32);
    entry[poff[bin] + (i - off[bin])] = (uint32_t)keys[i];
}

__global__ void bucket_max_kernel(const uint64_t* __restrict__ off, uint32_t nbins, unsigned long long* mx) {
    const uint32_t b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b < nbins) atomicMax(mx, (unsigned long long)(off[b + 1] - off[b]));
}

// flag[b] = bucket b holds at least lo entries (and is hot when lo > 1)
__global__ void bucket_flag_kernel(const uint64_t* __restrict__ off, uint32_t nbins, uint64_t lo,
                                   uint32_t* __restrict__ flag) {
    const uint32_t b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b < nbins) flag[b] = (off[b + 1] - off[b]) >= lo ? 1u : 0u;
}

__global__ void row_of_kernel(const uint32_t* __restrict__ flag, const uint64_t* __restrict__ scan, uint32_t nbins,
                              int32_t* __restrict__ row) {
    const uint32_t b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b < nbins) row[b] = flag[b] ? (int32_t)scan[b] : -1;
}

// Chunk skip table: skip[row * stride + j] = number of entries of the bucket
// with pid < j * 2^kChunkShift, for j = 0 .. stride-1 (the last column is the
// bucket size).  Every cell is written by exactly one entry.
__global__ void skip_fill_kernel(const uint64_t* __restrict__ keys, uint64_t n, const uint64_t* __restrict__ off,
                                 const int32_t* __restrict__ row, uint32_t stride, uint32_t* __restrict__ skip) {
    const uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const uint32_t bin = (uint32_t)(keys[i] >> 32);
    const uint32_t ch = ((uint32_t)keys[i] >> 1) >> kChunkShift;
    const uint64_t b0 = off[bin], b1 = off[bin + 1];
    uint32_t* base = skip + (uint64_t)row[bin] * stride;
    const uint32_t rel = (uint32_t)(i - b0);
    const uint32_t jlo = (i == b0) ? 0u : (((uint32_t)keys[i - 1] >> 1) >> kChunkShift) + 1u;
    for (uint32_t j = jlo; j <= ch; ++j) base[j] = rel;
    if (i + 1 == b1)
        for (uint32_t j = ch + 1; j < stride; ++j) base[j] = (uint32_t)(b1 - b0);
}

// Hot buckets as pid bitmaps: bit pid of hb[h] (b ion) or hy[h] (y ion).
__global__ void hot_fill_kernel(const uint64_t* __restrict__ keys, uint64_t n, const int32_t* __restrict__ hot_id,
                                uint64_t words, uint32_t* __restrict__ hb, uint32_t* __restrict__ hy,
                                uint32_t* __restrict__ hflags) {
    const uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int32_t h = hot_id[(uint32_t)(keys[i] >> 32)];
    if (h < 0) return;
    const uint32_t e = (uint32_t)keys[i];
    const uint32_t pid = e >> 1;
    uint32_t* bm = (e & 1u) ? hy : hb;
    atomicOr(&bm[(uint64_t)h * words + (pid >> 5)], 1u << (pid & 31));
    atomicOr(&hflags[h], (e & 1u) ? 2u : 1u);
}

template <class T>
cudaError_t dalloc(T** p, uint64_t n, std::vector<void*>& tmp) {
    cudaError_t e = cudaMalloc((void**)p, sizeof(T) * (n ? n : 1));
    if (e == cudaSuccess) tmp.push_back(*p);
    return e;
}

struct TmpFree {
    std::vector<void*> ptrs;
    ~TmpFree() { for (void* p : ptrs) cudaFree(p); }
};

}  // namespace

void free_device_index(hicops_index* idx) {
    DeviceIndex& d = idx->dev;
    if (d.device >= 0) {
        int cur = -1;
        cudaGetDevice(&cur);
        if (cur != d.device) cudaSetDevice(d.device);
        cudaFree(d.mass);
        cudaFree(d.off);
        cudaFree(d.entry);
        cudaFree(d.lf);
        cudaFree(d.ls);
        cudaFree(d.skip_row);
        cudaFree(d.skip);
        cudaFree(d.hot_id);
        cudaFree(d.hot_b);
        cudaFree(d.hot_y);
        cudaFree(d.hot_flags);
        cudaFree(d.pid_map);
        for (void* e : d.ev) if (e) cudaEventDestroy((cudaEvent_t)e);
        if (cur >= 0 && cur != d.device) cudaSetDevice(cur);
    }
    d = DeviceIndex{};
}

hicops_status upload_index(hicops_index* idx) {
    if (idx->dev.ready) return HICOPS_OK;
    auto t0 = std::chrono::steady_clock::now();
    DeviceIndex& d = idx->dev;
    HC_CUDA(cudaGetDevice(&d.device));
    const hicops_params& p = idx->p;
    const uint64_t P = idx->mass.size();
    const uint64_t B = idx->base_off.size() - 1;
    TmpFree tf;   // destroyed after the stream guard has synchronised
    cudaStream_t s;
    HC_CUDA(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
    struct StreamGuard { cudaStream_t s; ~StreamGuard() { cudaStreamSynchronize(s); cudaStreamDestroy(s); } } sg{s};

    // persistent parts
    HC_CUDA(cudaMalloc(&d.mass, sizeof(double) * (P ? P : 1)));
    HC_CUDA(cudaMemcpyAsync(d.mass, idx->mass.data(), sizeof(double) * P, cudaMemcpyHostToDevice, s));
    if (!idx->pid_map.empty()) {   // a subset: its rows report global pids
        HC_CUDA(cudaMalloc(&d.pid_map, sizeof(uint32_t) * P));
        HC_CUDA(cudaMemcpyAsync(d.pid_map, idx->pid_map.data(), sizeof(uint32_t) * P, cudaMemcpyHostToDevice, s));
    }
    HC_CUDA(cudaMalloc(&d.off, sizeof(uint64_t) * (idx->n_bins + 1)));
    // score tables (host libm, FP64): LF[n] = round(2^32 sum_{i<=n} log10 i), LS[s] = round(2^32 log10 s)
    std::vector<int64_t> lf(kMaxLen + 1), ls(idx->s_max + 1);
    double acc = 0.0;
    lf[0] = 0;
    for (uint32_t n = 1; n <= kMaxLen; ++n) {
        if (n >= 2) acc = acc + std::log10((double)n);
        lf[n] = std::llround(std::ldexp(acc, 32));
    }
    ls[0] = 0;
    for (uint64_t v = 1; v <= idx->s_max; ++v) ls[v] = std::llround(std::ldexp(std::log10((double)v), 32));
    HC_CUDA(cudaMalloc(&d.lf, sizeof(int64_t) * lf.size()));
    HC_CUDA(cudaMalloc(&d.ls, sizeof(int64_t) * ls.size()));
    HC_CUDA(cudaMemcpyAsync(d.lf, lf.data(), sizeof(int64_t) * lf.size(), cudaMemcpyHostToDevice, s));
    HC_CUDA(cudaMemcpyAsync(d.ls, ls.data(), sizeof(int64_t) * ls.size(), cudaMemcpyHostToDevice, s));

    // temporaries: peptide table
    uint32_t* d_base;
    uint64_t *d_mask, *d_boff;
    char* d_res;
    double *d_mres, *d_mmod;
    HC_CUDA(dalloc(&d_base, P, tf.ptrs));
    HC_CUDA(dalloc(&d_mask, P, tf.ptrs));
    HC_CUDA(dalloc(&d_boff, B + 1, tf.ptrs));
    HC_CUDA(dalloc(&d_res, idx->residues.size() + 1, tf.ptrs));
    HC_CUDA(dalloc(&d_mres, 128, tf.ptrs));
    HC_CUDA(dalloc(&d_mmod, 128, tf.ptrs));
    HC_CUDA(cudaMemcpyAsync(d_base, idx->base.data(), sizeof(uint32_t) * P, cudaMemcpyHostToDevice, s));
    HC_CUDA(cudaMemcpyAsync(d_mask, idx->mask.data(), sizeof(uint64_t) * P, cudaMemcpyHostToDevice, s));
    HC_CUDA(cudaMemcpyAsync(d_boff, idx->base_off.data(), sizeof(uint64_t) * (B + 1), cudaMemcpyHostToDevice, s));
    HC_CUDA(cudaMemcpyAsync(d_res, idx->residues.data(), idx->residues.size(), cudaMemcpyHostToDevice, s));
    HC_CUDA(cudaMemcpyAsync(d_mres, idx->mres, sizeof(double) * 128, cudaMemcpyHostToDevice, s));
    HC_CUDA(cudaMemcpyAsync(d_mmod, idx->mmod, sizeof(double) * 128, cudaMemcpyHostToDevice, s));

    IonArgs a{d_base, d_mask, d_boff, d_res, d_mres, d_mmod, p.bin_width_da, p.frag_mz_min, p.frag_mz_max, P};
    uint32_t* d_cnt;
    uint64_t* d_ionoff;
    uint64_t* d_total;
    HC_CUDA(dalloc(&d_cnt, P, tf.ptrs));
    HC_CUDA(dalloc(&d_ionoff, P, tf.ptrs));
    HC_CUDA(dalloc(&d_total, 1, tf.ptrs));
    uint64_t* d_scan_tmp;
    HC_CUDA(dalloc(&d_scan_tmp, scan_tmp_words(P), tf.ptrs));
    const unsigned pgrid = (unsigned)((P + kIonThreads - 1) / kIonThreads);
    if (P) ion_count_kernel<<<pgrid, kIonThreads, 0, s>>>(a, d_cnt);
    HC_CUDA(cudaGetLastError());
    HC_CUDA(exclusive_scan<uint32_t>(d_cnt, P, d_ionoff, d_total, d_scan_tmp, s));
    uint64_t E = 0;
    HC_CUDA(cudaMemcpyAsync(&E, d_total, sizeof(uint64_t), cudaMemcpyDeviceToHost, s));
    HC_CUDA(cudaStreamSynchronize(s));

    uint64_t *keys, *keys2;
    HC_CUDA(dalloc(&keys, E, tf.ptrs));
    HC_CUDA(dalloc(&keys2, E, tf.ptrs));
    if (P) ion_emit_kernel<<<pgrid, kIonThreads, 0, s>>>(a, d_ionoff, keys);
    HC_CUDA(cudaGetLastError());

    // stable radix sort on the bin bits
    int bin_bits = 1;
    while ((1ull << bin_bits) < idx->n_bins) ++bin_bits;
    const uint64_t ntiles = (E + kRsTile - 1) / kRsTile;
    if (E) {
        uint32_t* counts;
        uint64_t* offs;
        HC_CUDA(dalloc(&counts, ntiles * kRsRadix, tf.ptrs));
        HC_CUDA(dalloc(&offs, ntiles * kRsRadix, tf.ptrs));
        uint64_t* stmp;
        HC_CUDA(dalloc(&stmp, scan_tmp_words(ntiles * kRsRadix), tf.ptrs));
        for (int shift = 32; shift < 32 + bin_bits; shift += kRsBits) {
            rs_count_kernel<<<(unsigned)ntiles, kRsWarps * 32, 0, s>>>(keys, E, shift, counts, ntiles);
            HC_CUDA(cudaGetLastError());
            HC_CUDA(exclusive_scan<uint32_t>(counts, ntiles * kRsRadix, offs, nullptr, stmp, s));
            rs_scatter_kernel<<<(unsigned)ntiles, kRsWarps * 32, 0, s>>>(keys, keys2, E, shift, offs, ntiles);
            HC_CUDA(cudaGetLastError());
            std::swap(keys, keys2);
        }
    }
    // bucket offsets of the sorted keys (uoff), then the stored layout: each
    // bucket padded to a multiple of 4 entries (d.off), so that the search
    // reads whole 16-byte groups
    const uint32_t nb = idx->n_bins;
    const unsigned bgrid = (nb + 255) / 256;
    const unsigned egrid = (unsigned)((E + 255) / 256);
    uint64_t* uoff;
    HC_CUDA(dalloc(&uoff, (uint64_t)nb + 1, tf.ptrs));
    bucket_off_kernel<<<(unsigned)((E + 1 + 255) / 256), 256, 0, s>>>(keys, E, nb, uoff);
    HC_CUDA(cudaGetLastError());
    unsigned long long* d_mx = (unsigned long long*)d_total;
    HC_CUDA(cudaMemsetAsync(d_mx, 0, sizeof(uint64_t), s));
    bucket_max_kernel<<<bgrid, 256, 0, s>>>(uoff, nb, d_mx);
    HC_CUDA(cudaGetLastError());
    uint64_t mx = 0;
    HC_CUDA(cudaMemcpyAsync(&mx, d_mx, sizeof(uint64_t), cudaMemcpyDeviceToHost, s));
    HC_CUDA(cudaStreamSynchronize(s));
    if (mx >= (1ull << 32) - 3) {
        set_error("a bucket holds %llu entries (limit 2^32 - 4)", (unsigned long long)mx);
        return HICOPS_EOVERFLOW;
    }
    uint32_t* flag;
    uint64_t *rscan, *rtotal, *btmp;
    HC_CUDA(dalloc(&flag, nb, tf.ptrs));
    HC_CUDA(dalloc(&rscan, nb, tf.ptrs));
    HC_CUDA(dalloc(&rtotal, 1, tf.ptrs));
    HC_CUDA(dalloc(&btmp, scan_tmp_words(nb), tf.ptrs));
    padded_size_kernel<<<bgrid, 256, 0, s>>>(uoff, nb, flag);
    HC_CUDA(cudaGetLastError());
    HC_CUDA(exclusive_scan<uint32_t>(flag, nb, d.off, d.off + nb, btmp, s));
    uint64_t Ep = 0;
    HC_CUDA(cudaMemcpyAsync(&Ep, d.off + nb, sizeof(uint64_t), cudaMemcpyDeviceToHost, s));
    HC_CUDA(cudaStreamSynchronize(s));
    // four spare words: the allocation is never empty and ends 16-byte aligned
    HC_CUDA(cudaMalloc(&d.entry, sizeof(uint32_t) * (Ep + 4)));
    HC_CUDA(cudaMemsetAsync(d.entry, 0xff, sizeof(uint32_t) * (Ep + 4), s));
    if (E) take_low_kernel<<<egrid, 256, 0, s>>>(keys, E, uoff, d.off, d.entry);
    HC_CUDA(cudaGetLastError());

    // chunk skip tables for every non-empty bucket (positions relative to
    // the bucket start, so the same in both layouts)
    bucket_flag_kernel<<<bgrid, 256, 0, s>>>(uoff, nb, 1, flag);
    HC_CUDA(cudaGetLastError());
    HC_CUDA(exclusive_scan<uint32_t>(flag, nb, rscan, rtotal, btmp, s));
    HC_CUDA(cudaMalloc(&d.skip_row, sizeof(int32_t) * nb));
    row_of_kernel<<<bgrid, 256, 0, s>>>(flag, rscan, nb, d.skip_row);
    HC_CUDA(cudaGetLastError());
    uint64_t rows = 0;
    HC_CUDA(cudaMemcpyAsync(&rows, rtotal, sizeof(uint64_t), cudaMemcpyDeviceToHost, s));
    HC_CUDA(cudaStreamSynchronize(s));
    d.skip_stride = (uint32_t)(((P + kChunk - 1) >> kChunkShift) + 1);
    HC_CUDA(cudaMalloc(&d.skip, sizeof(uint32_t) * (rows ? rows : 1) * d.skip_stride));
    if (E) skip_fill_kernel<<<egrid, 256, 0, s>>>(keys, E, uoff, d.skip_row, d.skip_stride, d.skip);
    HC_CUDA(cudaGetLastError());

    // hot buckets as bitmaps
    const uint64_t hot_lo = std::max<uint64_t>(2, P >> kHotShift);
    bucket_flag_kernel<<<bgrid, 256, 0, s>>>(uoff, nb, hot_lo, flag);
    HC_CUDA(cudaGetLastError());
    HC_CUDA(exclusive_scan<uint32_t>(flag, nb, rscan, rtotal, btmp, s));
    HC_CUDA(cudaMalloc(&d.hot_id, sizeof(int32_t) * nb));
    row_of_kernel<<<bgrid, 256, 0, s>>>(flag, rscan, nb, d.hot_id);
    HC_CUDA(cudaGetLastError());
    uint64_t nhot = 0;
    HC_CUDA(cudaMemcpyAsync(&nhot, rtotal, sizeof(uint64_t), cudaMemcpyDeviceToHost, s));
    HC_CUDA(cudaStreamSynchronize(s));
    d.n_hot = (uint32_t)nhot;
    // rows cover every pid of the last search chunk (up to 2 * kChunk past P)
    // and start 16-byte aligned
    d.hot_words = ((P + 2ull * kChunk + 31) / 32 + 3) & ~3ull;
    const uint64_t hbytes = sizeof(uint32_t) * (nhot ? nhot : 1) * d.hot_words;
    HC_CUDA(cudaMalloc(&d.hot_b, hbytes));
    HC_CUDA(cudaMalloc(&d.hot_y, hbytes));
    HC_CUDA(cudaMalloc(&d.hot_flags, sizeof(uint32_t) * (nhot ? nhot : 1)));
    HC_CUDA(cudaMemsetAsync(d.hot_b, 0, hbytes, s));
    HC_CUDA(cudaMemsetAsync(d.hot_y, 0, hbytes, s));
    HC_CUDA(cudaMemsetAsync(d.hot_flags, 0, sizeof(uint32_t) * (nhot ? nhot : 1), s));
    if (E && nhot) hot_fill_kernel<<<egrid, 256, 0, s>>>(keys, E, d.hot_id, d.hot_words, d.hot_b, d.hot_y, d.hot_flags);
    HC_CUDA(cudaGetLastError());
    HC_CUDA(cudaStreamSynchronize(s));

    d.n_stored = Ep;
    d.bytes = sizeof(double) * P + sizeof(uint64_t) * (idx->n_bins + 1) + sizeof(uint32_t) * (Ep + 4) +
              sizeof(int64_t) * (lf.size() + ls.size()) + sizeof(int32_t) * 2 * nb +
              sizeof(uint32_t) * rows * d.skip_stride + 2 * hbytes;
    idx->stats.n_entries = E;
    idx->stats.max_bucket = mx;
    idx->stats.device_bytes = d.bytes;
    idx->stats.device_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    d.ready = true;
    return HICOPS_OK;
}

}  // namespace hicops

extern "C" hicops_status hicops_index_upload(hicops_index* idx) {
    if (!idx) { hicops::set_error("index is NULL"); return HICOPS_EINVAL; }
    hicops_status st = hicops::upload_index(idx);
    if (st != HICOPS_OK) hicops::free_device_index(idx);
    return st;
}

// The device keeps every bucket padded to a multiple of 4 entries; the copy
// leaves the pad slots out, so buckets are back to back as documented.
extern "C" hicops_status hicops_index_copy_csr(const hicops_index* idx, uint64_t* off, uint32_t* entries) {
    if (!idx || !idx->dev.ready) { hicops::set_error("index not uploaded"); return HICOPS_EINVAL; }
    if (!off && !entries) return HICOPS_OK;
    const uint32_t nb = idx->n_bins;
    std::vector<uint64_t> poff(nb + 1);
    std::vector<uint32_t> pent;
    try {
        pent.resize(idx->dev.n_stored);
    } catch (const std::bad_alloc&) {
        hicops::set_error("out of host memory");
        return HICOPS_ENOMEM;
    }
    HC_CUDA(cudaMemcpy(poff.data(), idx->dev.off, sizeof(uint64_t) * (nb + 1), cudaMemcpyDeviceToHost));
    if (!pent.empty())
        HC_CUDA(cudaMemcpy(pent.data(), idx->dev.entry, sizeof(uint32_t) * pent.size(), cudaMemcpyDeviceToHost));
    uint64_t o = 0;
    for (uint32_t b = 0; b < nb; ++b) {
        if (off) off[b] = o;
        for (uint64_t i = poff[b]; i < poff[b + 1] && pent[i] != 0xffffffffu; ++i) {
            if (entries) entries[o] = pent[i];
            ++o;
        }
    }
    if (off) off[nb] = o;
    return HICOPS_OK;
}
