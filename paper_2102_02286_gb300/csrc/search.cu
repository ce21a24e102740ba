// Superstep 3 search on the GPU (paper: "Superstep 3: Partial Database
// Peptide Search", Eq. 4; Supplementary Algorithm 3) and the superstep-4
// e-value (Supplementary Algorithm 4): host orchestration.
//
// One search is a fixed sequence on one stream:
//   prep_kernel    R sub-task's "minimal computations": filter, bin, merge,
//                  keep the B most intense peaks, quantise; precursor mass and
//                  filter_1 (binary search of the mass-sorted database);
//   plan_kernel +  work units (spectrum, peptide-id segment);
//   exclusive scan
//   search_kernel  filter_2 + score + heap over persistent CTAs;
//   merge_kernel   per-spectrum top-k merge and the survival-tail e-value.
// hicops_search allocates its scratch stream-ordered per call; a plan
// (hicops_plan_*) allocates it once and can replay the sequence as a CUDA
// graph.
#include <atomic>
#include <mutex>
#include <cfloat>
#include <cmath>
#include <vector>

#include "search_kernels.cuh"
#include "search_scratch.h"

namespace hicops {

static std::atomic<uint64_t> g_launches{0};
void count_launches(uint64_t n) { g_launches.fetch_add(n, std::memory_order_relaxed); }

namespace {

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

// persistent scratch of a plan
struct Arena {
    std::vector<void*> ptrs;
    template <class T>
    cudaError_t get(T** p, uint64_t n) {
        cudaError_t e = cudaMalloc((void**)p, sizeof(T) * (n ? n : 1));
        if (e == cudaSuccess) ptrs.push_back(*p);
        return e;
    }
    ~Arena() { for (void* p : ptrs) cudaFree(p); }
};

// Device scratch of one search of up to cap_n spectra.
struct Workspace {
    uint32_t cap_n = 0, max_seg = 0;
    uint32_t *qbin = nullptr, *qiq = nullptr, *qn = nullptr, *lo = nullptr, *hi = nullptr, *nseg = nullptr;
    uint64_t *seg_off = nullptr, *stmp = nullptr;
    UnitTop* utop = nullptr;
    unsigned long long* work = nullptr;
    uint32_t* order = nullptr;   // [cap_n * max_seg] units, longest first
    uint32_t* order_q = nullptr; // [cap_n * max_seg] their spectra
    uint32_t* ocnt = nullptr;    // [2 * kOrderBuckets] bucket counts and starts
    hicops_psm* psm = nullptr;   // used when the caller gives no device output
    uint32_t* hist = nullptr;
    uint32_t* ns = nullptr;
};

template <class A>
hicops_status alloc_workspace(A& al, const hicops_params& p, uint32_t cap_n, uint32_t max_seg, bool outputs,
                              Workspace& w) {
    w.cap_n = cap_n;
    w.max_seg = max_seg;
    HC_CUDA(al.get(&w.qbin, (uint64_t)cap_n * query_bins_cap(p)));
    HC_CUDA(al.get(&w.qiq, (uint64_t)cap_n * query_bins_cap(p)));
    HC_CUDA(al.get(&w.qn, cap_n));
    HC_CUDA(al.get(&w.lo, cap_n));
    HC_CUDA(al.get(&w.hi, cap_n));
    HC_CUDA(al.get(&w.nseg, cap_n));
    HC_CUDA(al.get(&w.seg_off, (uint64_t)cap_n + 1));
    HC_CUDA(al.get(&w.stmp, scan_tmp_words(cap_n)));
    HC_CUDA(al.get(&w.utop, (uint64_t)cap_n * max_seg * p.top_k));
    HC_CUDA(al.get(&w.work, 1));
    HC_CUDA(al.get(&w.order, (uint64_t)cap_n * max_seg));
    HC_CUDA(al.get(&w.order_q, (uint64_t)cap_n * max_seg));
    HC_CUDA(al.get(&w.ocnt, 2 * kOrderBuckets));
    if (outputs) {
        HC_CUDA(al.get(&w.psm, (uint64_t)cap_n * p.top_k));
        HC_CUDA(al.get(&w.hist, (uint64_t)cap_n * kHistBins));
        HC_CUDA(al.get(&w.ns, cap_n));
    }
    return HICOPS_OK;
}

std::atomic<int> g_sm_count{0};   // set on first use; every thread computes the same value

hicops_status sm_count() {
    if (!g_sm_count.load(std::memory_order_relaxed)) {
        int dev, c = 0;
        HC_CUDA(cudaGetDevice(&dev));
        HC_CUDA(cudaDeviceGetAttribute(&c, cudaDevAttrMultiProcessorCount, dev));
        g_sm_count.store(c, std::memory_order_relaxed);
    }
    return HICOPS_OK;
}

hicops_status check_config(const hicops_search_config& c) {
    if (c.threads != 0 && c.threads != 256 && c.threads != 384 && c.threads != 512) {
        set_error("threads must be 256, 384 or 512");
        return HICOPS_EINVAL;
    }
    if (c.chunk_entries > 16) { set_error("chunk_entries must be in 1..16"); return HICOPS_EINVAL; }
    if (c.ctas_per_sm > 8) { set_error("ctas_per_sm must be <= 8"); return HICOPS_EINVAL; }
    return HICOPS_OK;
}

// Default shape: 384-thread CTAs (two fit an SM while the top-k lists are
// at most 16 long), else 256; super-chunks of up to about 12 k entries (the
// planes and the log's room cap sparse spectra's super-chunks earlier).
hicops_search_config resolved(const hicops_search_config& c, uint32_t k) {
    hicops_search_config r = c;
    if (!r.threads) r.threads = k <= 16 ? 384 : 256;
    if (!r.chunk_entries) r.chunk_entries = 12;
    return r;
}

// Units per spectrum cap: large when the batch cannot fill the GPU.
uint32_t max_segments(const hicops_search_config& c, uint32_t n) {
    if (c.seg_pids) return kMaxSegs;
    const uint32_t want = 8u * (uint32_t)g_sm_count.load(std::memory_order_relaxed);
    uint32_t m = (want + n - 1) / (n ? n : 1);
    if (m < 1) m = 1;
    if (m > (uint32_t)kMaxSegs) m = kMaxSegs;
    return m;
}

template <int KMAX, int THREADS, int MAXP>
hicops_status launch_search_t(const SearchArgs& sa, uint32_t ctas_per_sm, uint64_t max_units, cudaStream_t s) {
    static std::atomic<int> occ{-1};   // CTAs per SM; concurrent first calls compute the same value
    const size_t smem = sizeof(uint32_t) * Layout<KMAX, THREADS, MAXP>::kDynWords;   // planes, log, slots / counters
    if (occ.load(std::memory_order_acquire) < 0) {
        HC_CUDA(cudaFuncSetAttribute(search_kernel<KMAX, THREADS, MAXP>,
                                     cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        int b = 0;
        HC_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, search_kernel<KMAX, THREADS, MAXP>, THREADS,
                                                              smem));
        occ.store(b < 1 ? 1 : b, std::memory_order_release);
    }
    int per_sm = occ.load(std::memory_order_acquire);
    if (ctas_per_sm && (int)ctas_per_sm < per_sm) per_sm = (int)ctas_per_sm;
    // no more CTAs than work units can exist
    uint64_t grid = (uint64_t)g_sm_count.load(std::memory_order_relaxed) * per_sm;
    if (max_units < grid) grid = max_units ? max_units : 1;
    search_kernel<KMAX, THREADS, MAXP><<<(unsigned)grid, THREADS, smem, s>>>(sa);
    count_launches(1);
    HC_CUDA(cudaGetLastError());
    return HICOPS_OK;
}

// The kernel for at most 512 query bins a spectrum (no fragment tolerance, or
// a narrow one) has the smaller static shared memory and the larger planes.
template <int THREADS, int MAXP>
hicops_status launch_search_p(const SearchArgs& sa, uint32_t ctas_per_sm, uint64_t max_units, cudaStream_t s) {
    if (sa.k <= 8) return launch_search_t<8, THREADS, MAXP>(sa, ctas_per_sm, max_units, s);
    if (sa.k <= 16) return launch_search_t<16, THREADS, MAXP>(sa, ctas_per_sm, max_units, s);
    return launch_search_t<32, THREADS, MAXP>(sa, ctas_per_sm, max_units, s);
}

template <int THREADS>
hicops_status launch_search_k(const SearchArgs& sa, uint32_t ctas_per_sm, uint64_t max_units, cudaStream_t s) {
    if (sa.topn <= 512) return launch_search_p<THREADS, 512>(sa, ctas_per_sm, max_units, s);
    return launch_search_p<THREADS, kMaxTopN>(sa, ctas_per_sm, max_units, s);
}

hicops_status launch_search(const SearchArgs& sa, const hicops_search_config& c, uint64_t max_units,
                            cudaStream_t s) {
    if (c.threads == 512) return launch_search_k<512>(sa, c.ctas_per_sm, max_units, s);
    if (c.threads == 384) return launch_search_k<384>(sa, c.ctas_per_sm, max_units, s);
    return launch_search_k<256>(sa, c.ctas_per_sm, max_units, s);
}

inline void mark(hicops_index* idx, int i, cudaStream_t s, bool on) {
    if (on && idx->dev.timing) cudaEventRecord((cudaEvent_t)idx->dev.ev[i], s);
}

// Query preprocessing of n spectra (R8), then, with a fragment tolerance of
// t > 0 bins, the widening of every spectrum's bins (R15).  qbin / qiq hold
// query_bins_cap(p) words per spectrum.
hicops_status prepare_queries(hicops_index* idx, const DevBatch& d, uint32_t n, uint32_t* qbin, uint32_t* qiq,
                              uint32_t* qn, uint32_t* lo, uint32_t* hi, cudaStream_t s) {
    const hicops_params& p = idx->p;
    const uint32_t stride = query_bins_cap(p);
    PrepArgs pa{d.peak_off, d.mz, d.inten, d.prec, d.z, d.tol, n, p.top_n_peaks, stride, p.bin_width_da,
                p.frag_mz_min, p.frag_mz_max, (double)p.intensity_scale, idx->dev.mass, idx->mass.size(),
                qbin, qiq, qn, lo, hi};
    prep_warp_kernel<<<(n + kPrepWarps - 1) / kPrepWarps, kPrepWarps * 32, 0, s>>>(pa);
    prep_kernel<<<n, kPrepThreads, 0, s>>>(pa);   // spectra of more than kPrepWarpPeaks peaks
    count_launches(2);
    HC_CUDA(cudaGetLastError());
    if (p.tol_bins > 0) {
        ExpandArgs ea{qbin, qiq, qn, n, stride, p.tol_bins, idx->n_bins};
        expand_kernel<<<(n + kExpWarps - 1) / kExpWarps, kExpWarps * 32, 0, s>>>(ea);
        count_launches(1);
        HC_CUDA(cudaGetLastError());
    }
    return HICOPS_OK;
}

// The whole search of n spectra on stream s, writing PSM rows, histograms
// and candidate counts to device memory.  Allocates nothing.
hicops_status enqueue_search(hicops_index* idx, const DevBatch& d, uint32_t n, const Workspace& w,
                             const hicops_search_config& cfg_in, hicops_psm* d_psm, uint32_t* d_hist, uint32_t* d_ns,
                             cudaStream_t s, bool timing_marks) {
    const hicops_params& p = idx->p;
    const DeviceIndex& di = idx->dev;
    const hicops_search_config cfg = resolved(cfg_in, idx->p.top_k);
    const uint32_t k = p.top_k;
    mark(idx, 0, s, timing_marks);
    hicops_status st = prepare_queries(idx, d, n, w.qbin, w.qiq, w.qn, w.lo, w.hi, s);
    if (st != HICOPS_OK) return st;
    mark(idx, 1, s, timing_marks);
    const uint32_t max_seg = w.max_seg;
    const uint32_t seg_pids = cfg.seg_pids ? cfg.seg_pids : (uint32_t)kMinSegPids;
    plan_kernel<<<(n + 255) / 256, 256, 0, s>>>(w.qn, w.lo, w.hi, n, max_seg, seg_pids, w.nseg);
    count_launches(1);
    HC_CUDA(cudaGetLastError());
    HC_CUDA(exclusive_scan<uint32_t>(w.nseg, n, w.seg_off, w.seg_off + n, w.stmp, s));
    // longest units first; a small batch has too few units per CTA for the
    // order to matter, and its three kernels would be most of its launch cost
    const bool ordered = n >= kOrderMinSpectra;
    if (ordered) {
        HC_CUDA(cudaMemsetAsync(w.ocnt, 0, sizeof(uint32_t) * kOrderBuckets, s));
        order_count_kernel<<<(n + 255) / 256, 256, 0, s>>>(w.qn, w.lo, w.hi, w.seg_off, n, w.ocnt);
        order_scan_kernel<<<1, 32, 0, s>>>(w.ocnt);
        order_scatter_kernel<<<(n + 255) / 256, 256, 0, s>>>(w.qn, w.lo, w.hi, w.seg_off, n, w.ocnt + kOrderBuckets,
                                                             w.order, w.order_q);
        count_launches(3);
        HC_CUDA(cudaGetLastError());
    }
    HC_CUDA(cudaMemsetAsync(d_hist, 0, sizeof(uint32_t) * n * kHistBins, s));
    HC_CUDA(cudaMemsetAsync(d_ns, 0, sizeof(uint32_t) * n, s));
    HC_CUDA(cudaMemsetAsync(w.work, 0, sizeof(unsigned long long), s));
    SearchArgs sa{w.qbin, w.qiq, w.qn, w.lo, w.hi, w.seg_off, n, query_bins_cap(p), di.off, di.entry,
                  di.skip_row, di.skip, di.skip_stride, di.hot_id, di.hot_b, di.hot_y, di.hot_flags,
                  di.hot_words, di.lf, di.ls, (uint32_t)idx->s_max, p.min_shared, k, cfg.chunk_entries * 1024u, w.utop, d_hist, d_ns,
                  w.work, ordered ? w.order : nullptr, w.order_q};
    mark(idx, 2, s, timing_marks);
    st = launch_search(sa, cfg, (uint64_t)n * max_seg, s);
    if (st != HICOPS_OK) return st;
    mark(idx, 3, s, timing_marks);
    MergeArgs ma{w.seg_off, w.utop, d_hist, n, k, 0, d_psm, idx->pid_stride, idx->pid_base, di.pid_map,
                 p.evalue_mode};
    merge_kernel<<<(n + kMergeWarps - 1) / kMergeWarps, kMergeWarps * 32, 0, s>>>(ma);
    count_launches(1);
    HC_CUDA(cudaGetLastError());
    mark(idx, 4, s, timing_marks);
    return HICOPS_OK;
}

hicops_status check_batch(const hicops_index* idx, const hicops_batch* b) {
    if (!idx || !b) { set_error("NULL argument"); return HICOPS_EINVAL; }
    if (!idx->dev.ready) { set_error("index has no device part (call hicops_index_upload)"); return HICOPS_EINVAL; }
    if (b->n && (!b->peak_off || !b->prec_mz || !b->charge || !b->prec_tol_da)) {
        set_error("batch pointers are NULL");
        return HICOPS_EINVAL;
    }
    int dev = -1;
    HC_CUDA(cudaGetDevice(&dev));
    if (dev != idx->dev.device) {
        set_error("current device %d is not the index's device %d", dev, idx->dev.device);
        return HICOPS_EINVAL;
    }
    return sm_count();
}

// Inputs on the device (copied from the host when on_device = 0).
hicops_status stage_inputs(const hicops_batch* b, Scratch& sc, DevBatch& d) {
    const cudaStream_t s = sc.s;
    if (b->on_device) {
        d = DevBatch{b->peak_off, b->mz, b->intensity, b->prec_mz, b->charge, b->prec_tol_da};
        return HICOPS_OK;
    }
    const uint64_t npk = b->peak_off[b->n];
    if (npk && (!b->mz || !b->intensity)) { set_error("peak arrays are NULL"); return HICOPS_EINVAL; }
    uint64_t* po;
    float *mz, *it;
    double *pr, *tl;
    uint8_t* z;
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
    return HICOPS_OK;
}

constexpr uint64_t align256(uint64_t x) { return (x + 255) & ~uint64_t(255); }

// alloc_workspace's allocators over caller memory.  Carve hands out
// consecutive 256-byte aligned pieces of one buffer and fails when they would
// not fit; Tally only adds up the bytes Carve would hand out.
struct Carve {
    unsigned char* base;
    uint64_t cap, used;
    template <class T>
    cudaError_t get(T** p, uint64_t n) {
        const uint64_t bytes = align256(sizeof(T) * (n ? n : 1));
        if (used + bytes > cap) return cudaErrorMemoryAllocation;
        *p = reinterpret_cast<T*>(base + used);
        used += bytes;
        return cudaSuccess;
    }
};

struct Tally {
    uint64_t used = 0;
    template <class T>
    cudaError_t get(T** p, uint64_t n) {
        *p = nullptr;
        used += align256(sizeof(T) * (n ? n : 1));
        return cudaSuccess;
    }
};

// The workspace of a search in caller memory: alloc_workspace's pieces
// without the PSM rows (the caller always gives those), then a histogram and
// candidate-count block for callers that pass none.
template <class A>
hicops_status scratch_workspace(A& al, const hicops_params& p, uint32_t n, uint32_t max_seg, Workspace& w) {
    hicops_status st = alloc_workspace(al, p, n, max_seg, false, w);
    if (st != HICOPS_OK) return st;
    HC_CUDA(al.get(&w.hist, (uint64_t)n * kHistBins));
    HC_CUDA(al.get(&w.ns, n));
    return HICOPS_OK;
}

}  // namespace

uint64_t scratch_bytes(const hicops_index* idx, const hicops_search_config& cfg, uint32_t n) {
    if (!n) n = 1;
    Tally t;
    Workspace w;
    scratch_workspace(t, idx->p, n, max_segments(cfg, n), w);
    return t.used;
}

hicops_status search_in_scratch(hicops_index* idx, const hicops_batch* b, const hicops_search_config& cfg,
                                void* scratch, uint64_t bytes, hicops_psm* out_psm, uint32_t* out_hist,
                                uint32_t* out_nscored) {
    hicops_status st = check_batch(idx, b);
    if (st != HICOPS_OK) return st;
    if (!b->on_device || !out_psm) {
        set_error("a search in caller scratch takes device pointers (on_device = 1) and a device out_psm");
        return HICOPS_EINVAL;
    }
    if (!scratch || (reinterpret_cast<uintptr_t>(scratch) & 255u)) {
        set_error("scratch must be a 256-byte aligned device pointer");
        return HICOPS_EINVAL;
    }
    const uint32_t n = b->n;
    if (n == 0) return HICOPS_OK;
    const uint64_t need = scratch_bytes(idx, cfg, n);
    if (bytes < need) {
        set_error("scratch of %llu bytes; a search of %u spectra needs %llu", (unsigned long long)bytes, n,
                  (unsigned long long)need);
        return HICOPS_ENOMEM;
    }
    Carve cv{static_cast<unsigned char*>(scratch), bytes, 0};
    Workspace w;
    st = scratch_workspace(cv, idx->p, n, max_segments(cfg, n), w);
    if (st != HICOPS_OK) return st;
    const DevBatch d{b->peak_off, b->mz, b->intensity, b->prec_mz, b->charge, b->prec_tol_da};
    return enqueue_search(idx, d, n, w, cfg, out_psm, out_hist ? out_hist : w.hist, out_nscored ? out_nscored : w.ns,
                          (cudaStream_t)b->cuda_stream, false);
}

}  // namespace hicops

using namespace hicops;

extern "C" hicops_status hicops_search_scratch_bytes(const hicops_index* idx, uint32_t n, uint64_t* out_bytes) {
    if (!idx || !out_bytes) { set_error("NULL argument"); return HICOPS_EINVAL; }
    if (!idx->dev.ready) { set_error("index has no device part (call hicops_index_upload)"); return HICOPS_EINVAL; }
    hicops_status st = sm_count();
    if (st != HICOPS_OK) return st;
    *out_bytes = scratch_bytes(idx, idx->dev.cfg, n);
    return HICOPS_OK;
}

extern "C" hicops_status hicops_search_scratch(hicops_index* idx, const hicops_batch* b, void* scratch,
                                               uint64_t bytes, hicops_psm* out_psm, uint32_t* out_hist,
                                               uint32_t* out_nscored) {
    if (!idx) { set_error("NULL argument"); return HICOPS_EINVAL; }
    return search_in_scratch(idx, b, idx->dev.cfg, scratch, bytes, out_psm, out_hist, out_nscored);
}

struct hicops_plan {
    hicops_index* idx = nullptr;
    hicops_search_config cfg{};
    Arena arena;
    Workspace ws;
    // captured graph and the call it was captured for
    cudaGraphExec_t exec = nullptr;
    cudaGraph_t graph = nullptr;
    hicops_batch key_batch{};
    const void* key_out[3] = {nullptr, nullptr, nullptr};
    uint64_t graph_launches = 0;
    ~hicops_plan() {
        if (exec) cudaGraphExecDestroy(exec);
        if (graph) cudaGraphDestroy(graph);
    }
};

extern "C" hicops_status hicops_search(hicops_index* idx, const hicops_batch* b, hicops_psm* out_psm,
                                       uint32_t* out_hist, uint32_t* out_nscored) {
    hicops_status st = check_batch(idx, b);
    if (st != HICOPS_OK) return st;
    if (!out_psm) { set_error("out_psm is NULL"); return HICOPS_EINVAL; }
    const uint32_t n = b->n;
    if (n == 0) return HICOPS_OK;
    const hicops_params& p = idx->p;
    const uint32_t k = p.top_k;
    cudaStream_t s = (cudaStream_t)b->cuda_stream;
    {
        Scratch sc(s);
        DevBatch d;
        st = stage_inputs(b, sc, d);
        if (st != HICOPS_OK) return st;
        Workspace w;
        st = alloc_workspace(sc, p, n, max_segments(idx->dev.cfg, n), !b->on_device, w);
        if (st != HICOPS_OK) return st;
        hicops_psm* d_psm = b->on_device ? out_psm : w.psm;
        uint32_t* d_hist = b->on_device && out_hist ? out_hist : nullptr;
        uint32_t* d_ns = b->on_device && out_nscored ? out_nscored : nullptr;
        if (!d_hist) { if (!w.hist) HC_CUDA(sc.get(&w.hist, (uint64_t)n * kHistBins)); d_hist = w.hist; }
        if (!d_ns) { if (!w.ns) HC_CUDA(sc.get(&w.ns, n)); d_ns = w.ns; }
        st = enqueue_search(idx, d, n, w, idx->dev.cfg, d_psm, d_hist, d_ns, s, true);
        if (st != HICOPS_OK) return st;
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
    const hicops_params& p = idx->p;
    {
        Scratch sc(s);
        DevBatch d;
        st = stage_inputs(b, sc, d);
        if (st != HICOPS_OK) return st;
        uint32_t *qbin, *qiq, *qn, *lo, *hi;
        uint64_t* hits;
        HC_CUDA(sc.get(&qbin, (uint64_t)n * query_bins_cap(p)));
        HC_CUDA(sc.get(&qiq, (uint64_t)n * query_bins_cap(p)));
        HC_CUDA(sc.get(&qn, n));
        HC_CUDA(sc.get(&lo, n));
        HC_CUDA(sc.get(&hi, n));
        HC_CUDA(sc.get(&hits, n));
        st = prepare_queries(idx, d, n, qbin, qiq, qn, lo, hi, s);
        if (st != HICOPS_OK) return st;
        work_kernel<<<n, 256, 0, s>>>(qbin, qn, lo, hi, query_bins_cap(p), idx->dev.off, idx->dev.entry, hits);
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

extern "C" hicops_status hicops_index_set_config(hicops_index* idx, const hicops_search_config* cfg) {
    if (!idx) { set_error("index is NULL"); return HICOPS_EINVAL; }
    hicops_search_config c = cfg ? *cfg : hicops_search_config{0, 0, 0, 0};
    hicops_status st = check_config(c);
    if (st != HICOPS_OK) return st;
    idx->dev.cfg = c;
    return HICOPS_OK;
}

extern "C" hicops_status hicops_plan_create(hicops_index* idx, uint32_t max_spectra, const hicops_search_config* cfg,
                                            hicops_plan** out) {
    if (!idx || !out || !max_spectra) { set_error("invalid argument"); return HICOPS_EINVAL; }
    *out = nullptr;
    if (!idx->dev.ready) { set_error("index not uploaded"); return HICOPS_EINVAL; }
    HC_CUDA(cudaSetDevice(idx->dev.device));
    hicops_status st = sm_count();
    if (st != HICOPS_OK) return st;
    hicops_plan* pl = new (std::nothrow) hicops_plan();
    if (!pl) { set_error("out of host memory"); return HICOPS_ENOMEM; }
    pl->idx = idx;
    pl->cfg = cfg ? *cfg : idx->dev.cfg;
    st = check_config(pl->cfg);
    // per-unit top-k lists: up to kMaxSegs units per spectrum within 1 GiB
    const uint64_t per_seg = (uint64_t)max_spectra * idx->p.top_k * sizeof(UnitTop);
    uint64_t segs = (1ull << 30) / per_seg;
    if (segs > (uint64_t)kMaxSegs) segs = kMaxSegs;
    if (segs < 1) segs = 1;
    if (st == HICOPS_OK) st = alloc_workspace(pl->arena, idx->p, max_spectra, (uint32_t)segs, true, pl->ws);
    if (st != HICOPS_OK) { delete pl; return st; }
    *out = pl;
    return HICOPS_OK;
}

extern "C" hicops_status hicops_plan_search(hicops_plan* pl, const hicops_batch* b, hicops_psm* out_psm,
                                            uint32_t* out_hist, uint32_t* out_nscored, int use_graph) {
    if (!pl) { set_error("plan is NULL"); return HICOPS_EINVAL; }
    hicops_status st = check_batch(pl->idx, b);
    if (st != HICOPS_OK) return st;
    if (!b->on_device || !out_psm) { set_error("a plan takes device pointers (on_device = 1) and out_psm"); return HICOPS_EINVAL; }
    const uint32_t n = b->n;
    if (n > pl->ws.cap_n) { set_error("batch of %u spectra exceeds the plan's %u", n, pl->ws.cap_n); return HICOPS_EINVAL; }
    if (n == 0) return HICOPS_OK;
    cudaStream_t s = (cudaStream_t)b->cuda_stream;
    uint32_t* d_hist = out_hist ? out_hist : pl->ws.hist;
    uint32_t* d_ns = out_nscored ? out_nscored : pl->ws.ns;
    DevBatch d{b->peak_off, b->mz, b->intensity, b->prec_mz, b->charge, b->prec_tol_da};
    Workspace w = pl->ws;
    const uint32_t want = max_segments(pl->cfg, n);
    if (want < w.max_seg) w.max_seg = want;
    if (!use_graph || s == nullptr)
        return enqueue_search(pl->idx, d, n, w, pl->cfg, out_psm, d_hist, d_ns, s, true);
    const bool same = pl->exec && memcmp(&pl->key_batch, b, sizeof(hicops_batch)) == 0 &&
                      pl->key_out[0] == out_psm && pl->key_out[1] == out_hist && pl->key_out[2] == out_nscored;
    if (!same) {
        if (pl->exec) { cudaGraphExecDestroy(pl->exec); pl->exec = nullptr; }
        if (pl->graph) { cudaGraphDestroy(pl->graph); pl->graph = nullptr; }
        // first-use set-up of the kernel attributes happens outside capture
        st = enqueue_search(pl->idx, d, n, w, pl->cfg, out_psm, d_hist, d_ns, s, false);
        if (st != HICOPS_OK) return st;
        const uint64_t before = g_launches.load();
        HC_CUDA(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
        st = enqueue_search(pl->idx, d, n, w, pl->cfg, out_psm, d_hist, d_ns, s, false);
        cudaGraph_t g = nullptr;
        cudaError_t e = cudaStreamEndCapture(s, &g);
        if (st != HICOPS_OK) { if (g) cudaGraphDestroy(g); return st; }
        if (e != cudaSuccess) { set_error("graph capture failed: %s", cudaGetErrorString(e)); return HICOPS_ECUDA; }
        pl->graph = g;
        HC_CUDA(cudaGraphInstantiate(&pl->exec, g, 0));
        pl->graph_launches = g_launches.load() - before;
        g_launches.fetch_sub(pl->graph_launches);   // counted again at every replay
        pl->key_batch = *b;
        pl->key_out[0] = out_psm;
        pl->key_out[1] = out_hist;
        pl->key_out[2] = out_nscored;
        return HICOPS_OK;   // the direct run above produced this call's results
    }
    HC_CUDA(cudaGraphLaunch(pl->exec, s));
    count_launches(pl->graph_launches);
    return HICOPS_OK;
}

extern "C" void hicops_plan_destroy(hicops_plan* pl) { delete pl; }

extern "C" hicops_status hicops_autotune(hicops_index* idx, const hicops_batch* b, hicops_search_config* best,
                                         double* best_ms) {
    hicops_status st = check_batch(idx, b);
    if (st != HICOPS_OK) return st;
    if (!b->on_device || b->n == 0) { set_error("autotune needs a non-empty device batch"); return HICOPS_EINVAL; }
    const uint32_t cand_threads[2] = {256, 384};
    const uint32_t cand_cm[4] = {4, 8, 12, 16};   // chunk_entries
    const uint32_t cand_ctas[2] = {0, 1};
    const uint32_t cand_seg[3] = {0, 1u << 18, 1u << 16};
    cudaStream_t s = (cudaStream_t)b->cuda_stream;
    cudaEvent_t e0, e1;
    HC_CUDA(cudaEventCreate(&e0));
    HC_CUDA(cudaEventCreate(&e1));
    hicops_search_config bc{0, 0, 0, 0};
    double bms = 1e300;
    hicops_plan* pl = nullptr;
    hicops_psm* psm = nullptr;
    st = HICOPS_OK;
    for (uint32_t th : cand_threads)
        for (uint32_t cm : cand_cm)
            for (uint32_t ct : cand_ctas)
                for (uint32_t sp : cand_seg) {
                    if (st != HICOPS_OK) break;
                    hicops_search_config c{th, cm, ct, sp};
                    st = hicops_plan_create(idx, b->n, &c, &pl);
                    if (st != HICOPS_OK) break;
                    if (!psm && cudaMalloc(&psm, sizeof(hicops_psm) * b->n * idx->p.top_k) != cudaSuccess) {
                        set_error("out of device memory");
                        st = HICOPS_ENOMEM;
                        break;
                    }
                    // one warm run, then two timed runs
                    double ms = 0;
                    for (int r = 0; r < 3 && st == HICOPS_OK; ++r) {
                        cudaEventRecord(e0, s);
                        st = hicops_plan_search(pl, b, psm, nullptr, nullptr, 0);
                        cudaEventRecord(e1, s);
                        if (cudaEventSynchronize(e1) != cudaSuccess) { set_error("autotune run failed"); st = HICOPS_ECUDA; }
                        float t = 0;
                        cudaEventElapsedTime(&t, e0, e1);
                        if (r > 0) ms += t / 2.0;
                    }
                    hicops_plan_destroy(pl);
                    pl = nullptr;
                    if (st == HICOPS_OK && ms < bms) { bms = ms; bc = c; }
                }
    if (psm) cudaFree(psm);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (st != HICOPS_OK) return st;
    idx->dev.cfg = bc;
    if (best) *best = bc;
    if (best_ms) *best_ms = bms;
    return HICOPS_OK;
}

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

// ---- search without allocation (an addition of this library; the paper has
// no counterpart).  The scratch of one search of at most
// HICOPS_NOALLOC_MAX_SPECTRA spectra lives in one file-scope device array;
// the entry point carves the same Workspace out of it that hicops_search
// allocates, and runs the same kernel sequence.
namespace hicops {
namespace {

constexpr uint32_t kNoAllocSegs = 16;      // work units per spectrum at most
constexpr int kNoAllocDevices = 64;        // device ordinals served

// Workspace bytes for cap spectra at the largest top_n_peaks and top_k, in
// alloc_workspace's order (each piece 256-byte aligned), plus room for the
// scan's temporary words.
constexpr uint64_t noalloc_bytes(uint64_t cap) {
    return 2 * align256(4 * cap * kMaxTopN)                      // qbin, qiq
           + 4 * align256(4 * cap)                               // qn, lo, hi, nseg
           + align256(8 * (cap + 1))                             // seg_off
           + 4096                                                // scan temporaries
           + align256(sizeof(UnitTop) * cap * kNoAllocSegs * kMaxTopK)
           + 256                                                 // work counter
           + 2 * align256(4 * cap * kNoAllocSegs)                // unit order and its spectra
           + align256(4 * 2 * kOrderBuckets)                     // its bucket counts
           + align256(sizeof(hicops_psm) * cap * kMaxTopK)       // psm (unused here)
           + align256(4 * cap * kHistBins) + align256(4 * cap);  // hist, n_scored
}
constexpr uint64_t kNoAllocBytes = noalloc_bytes(HICOPS_NOALLOC_MAX_SPECTRA);
static_assert(kNoAllocBytes <= (2u << 20), "the no-allocation scratch is meant to stay small");

// Shared by every hicops_search_noalloc call on a device.  Nothing in it
// has to start at zero: each search writes its pieces before reading them
// and clears the histogram, counters and work counter itself.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

std::mutex g_noalloc_mu;
void* g_noalloc_base[kNoAllocDevices] = {};
unsigned long long g_noalloc_ctx[kNoAllocDevices] = {};   // context the address belongs to

// Unique id of the calling thread's current context (the driver's
// cuCtxGetId, reached through the runtime), or 0 when there is none or the
// driver cannot tell.  Ids are never reused within a process, unlike
// context handles.
unsigned long long current_context_id() {
    using GetCurrent = int (*)(void**);
    using GetId = int (*)(void*, unsigned long long*);
    static GetCurrent get_current = nullptr;
    static GetId get_id = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void* f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_current = reinterpret_cast<GetCurrent>(f);
        f = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_id = reinterpret_cast<GetId>(f);
    });
    void* ctx = nullptr;
    unsigned long long id = 0;
    if (get_current && get_id && get_current(&ctx) == 0 && ctx && get_id(ctx, &id) == 0) return id;
    return 0;
}

// Device address of the array on device dev, which must be current.  The
// first call on a device looks it up (this can load the module on that
// device), and so does the first call after the device's context was
// replaced (cudaDeviceReset), because the address belongs to the context.
hicops_status noalloc_scratch(int dev, unsigned char** out) {
    if (dev < 0 || dev >= kNoAllocDevices) {
        set_error("hicops_search_noalloc serves device ordinals below %d, not %d", kNoAllocDevices, dev);
        return HICOPS_EINVAL;
    }
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    const unsigned long long ctx = current_context_id();
    if (!g_noalloc_base[dev] || ctx == 0 || ctx != g_noalloc_ctx[dev]) {
        void* p = nullptr;
        HC_CUDA(cudaGetSymbolAddress(&p, g_noalloc_scratch));
        g_noalloc_base[dev] = p;
        g_noalloc_ctx[dev] = current_context_id();   // the lookup may have created the context
    }
    *out = static_cast<unsigned char*>(g_noalloc_base[dev]);
    return HICOPS_OK;
}

}  // namespace
}  // namespace hicops

extern "C" hicops_status hicops_search_noalloc(hicops_index* idx, const hicops_batch* b, hicops_psm* out_psm,
                                               uint32_t* out_hist, uint32_t* out_nscored) {
    hicops_status st = check_batch(idx, b);
    if (st != HICOPS_OK) return st;
    if (!b->on_device || !out_psm) {
        set_error("hicops_search_noalloc takes device pointers (on_device = 1) and a device out_psm");
        return HICOPS_EINVAL;
    }
    const uint32_t n = b->n;
    if (n > HICOPS_NOALLOC_MAX_SPECTRA) {
        set_error("batch of %u spectra exceeds hicops_search_noalloc's limit of %u (HICOPS_NOALLOC_MAX_SPECTRA)", n,
                  (unsigned)HICOPS_NOALLOC_MAX_SPECTRA);
        return HICOPS_EINVAL;
    }
    if (n == 0) return HICOPS_OK;
    unsigned char* base = nullptr;
    st = noalloc_scratch(idx->dev.device, &base);
    if (st != HICOPS_OK) return st;
    Carve cv{base, kNoAllocBytes, 0};
    Workspace w;
    uint32_t segs = max_segments(idx->dev.cfg, n);
    if (segs > kNoAllocSegs) segs = kNoAllocSegs;
    st = alloc_workspace(cv, idx->p, n, segs, true, w);
    if (st != HICOPS_OK) {
        set_error("hicops_search_noalloc: scratch of %llu bytes is too small", (unsigned long long)kNoAllocBytes);
        return HICOPS_ENOMEM;
    }
    const DevBatch d{b->peak_off, b->mz, b->intensity, b->prec_mz, b->charge, b->prec_tol_da};
    return enqueue_search(idx, d, n, w, idx->dev.cfg, out_psm, out_hist ? out_hist : w.hist,
                          out_nscored ? out_nscored : w.ns, (cudaStream_t)b->cuda_stream, false);
}

// ---- database sharding (paper: each process searches its partition of the
// database, Superstep 3; the partial score distributions are added and the
// results assembled, Superstep 4).  A shard's rows carry global pids; the
// merge sums the partial histograms and candidate counts, merges the shard
// top-k lists by (key desc, pid asc) with merge_kernel and fits the e-value
// to the summed histogram, so the result equals the unsharded search.
namespace hicops {
namespace {

// one block per spectrum: shard rows -> unit lists, summed histogram
__global__ void shard_gather_kernel(const hicops_psm* __restrict__ parts, uint32_t n_shards, uint32_t n,
                                    uint32_t k, const uint32_t* __restrict__ hist_in,
                                    const uint32_t* __restrict__ ns_in, uint32_t hist_parts,
                                    UnitTop* __restrict__ utop, uint64_t* __restrict__ seg_off,
                                    uint32_t* __restrict__ hist, uint32_t* __restrict__ ns) {
    const uint32_t q = blockIdx.x;
    for (uint32_t i = threadIdx.x; i < n_shards * k; i += blockDim.x) {
        const uint32_t s = i / k, r = i % k;
        const hicops_psm row = parts[((uint64_t)s * n + q) * k + r];
        UnitTop t;
        t.key = row.key;
        t.pid = row.pid;
        t.packed = ((uint32_t)row.nb << kNbShift) | ((uint32_t)row.ny << kNyShift);
        utop[((uint64_t)q * n_shards + s) * k + r] = t;
    }
    for (uint32_t j = threadIdx.x; j < kHistBins; j += blockDim.x) {
        uint32_t h = 0;
        for (uint32_t p = 0; p < hist_parts; ++p) h += hist_in[((uint64_t)p * n + q) * kHistBins + j];
        hist[(uint64_t)q * kHistBins + j] = h;
    }
    if (threadIdx.x == 0) {
        uint32_t c = 0;
        for (uint32_t p = 0; p < hist_parts; ++p) c += ns_in[(uint64_t)p * n + q];
        ns[q] = c;
        seg_off[q] = (uint64_t)q * n_shards;
        if (q == n - 1) seg_off[n] = (uint64_t)n * n_shards;
    }
}

}  // namespace
}  // namespace hicops

extern "C" hicops_status hicops_merge_shards(uint32_t n_shards, uint32_t n, uint32_t top_k,
                                             const hicops_psm* shard_psm, const uint32_t* hist,
                                             const uint32_t* nscored, uint32_t hist_parts,
                                             uint32_t evalue_mode, int on_device, void* cuda_stream,
                                             hicops_psm* out_psm, uint32_t* out_hist, uint32_t* out_nscored) {
    if (n_shards < 1 || n_shards > HICOPS_MAX_SHARDS) {
        set_error("n_shards must be in [1, %u]", (unsigned)HICOPS_MAX_SHARDS);
        return HICOPS_EINVAL;
    }
    if (top_k < 1 || top_k > kMaxTopK) { set_error("top_k must be in [1, %u]", kMaxTopK); return HICOPS_EINVAL; }
    if (hist_parts != 1 && hist_parts != n_shards) { set_error("hist_parts must be 1 or n_shards"); return HICOPS_EINVAL; }
    if (evalue_mode & ~(HICOPS_EVALUE_LOG_WEIBULL | HICOPS_EVALUE_SMOOTH)) {
        set_error("unknown evalue_mode bits");
        return HICOPS_EINVAL;
    }
    if (n == 0) return HICOPS_OK;
    if (!shard_psm || !hist || !nscored || !out_psm) { set_error("NULL argument"); return HICOPS_EINVAL; }
    cudaStream_t s = (cudaStream_t)cuda_stream;
    {
        Scratch sc(s);
        const hicops_psm* d_parts = shard_psm;
        const uint32_t *d_hin = hist, *d_nin = nscored;
        const uint64_t rows = (uint64_t)n_shards * n * top_k;
        if (!on_device) {
            hicops_psm* p;
            uint32_t *h, *c;
            HC_CUDA(sc.get(&p, rows));
            HC_CUDA(sc.get(&h, (uint64_t)hist_parts * n * kHistBins));
            HC_CUDA(sc.get(&c, (uint64_t)hist_parts * n));
            HC_CUDA(cudaMemcpyAsync(p, shard_psm, sizeof(hicops_psm) * rows, cudaMemcpyHostToDevice, s));
            HC_CUDA(cudaMemcpyAsync(h, hist, sizeof(uint32_t) * hist_parts * n * kHistBins, cudaMemcpyHostToDevice, s));
            HC_CUDA(cudaMemcpyAsync(c, nscored, sizeof(uint32_t) * hist_parts * n, cudaMemcpyHostToDevice, s));
            d_parts = p;
            d_hin = h;
            d_nin = c;
        }
        UnitTop* utop;
        uint64_t* seg_off;
        uint32_t *d_hist, *d_ns;
        hicops_psm* d_out = on_device ? out_psm : nullptr;
        HC_CUDA(sc.get(&utop, rows));
        HC_CUDA(sc.get(&seg_off, (uint64_t)n + 1));
        if (on_device && out_hist) d_hist = out_hist; else HC_CUDA(sc.get(&d_hist, (uint64_t)n * kHistBins));
        if (on_device && out_nscored) d_ns = out_nscored; else HC_CUDA(sc.get(&d_ns, n));
        if (!d_out) HC_CUDA(sc.get(&d_out, (uint64_t)n * top_k));
        shard_gather_kernel<<<n, 256, 0, s>>>(d_parts, n_shards, n, top_k, d_hin, d_nin, hist_parts, utop,
                                              seg_off, d_hist, d_ns);
        count_launches(1);
        HC_CUDA(cudaGetLastError());
        MergeArgs ma{seg_off, utop, d_hist, n, top_k, 0, d_out, 1u, 0u, nullptr, evalue_mode};
        merge_kernel<<<(n + kMergeWarps - 1) / kMergeWarps, kMergeWarps * 32, 0, s>>>(ma);
        count_launches(1);
        HC_CUDA(cudaGetLastError());
        if (!on_device) {
            HC_CUDA(cudaMemcpyAsync(out_psm, d_out, sizeof(hicops_psm) * n * top_k, cudaMemcpyDeviceToHost, s));
            if (out_hist)
                HC_CUDA(cudaMemcpyAsync(out_hist, d_hist, sizeof(uint32_t) * n * kHistBins, cudaMemcpyDeviceToHost, s));
            if (out_nscored)
                HC_CUDA(cudaMemcpyAsync(out_nscored, d_ns, sizeof(uint32_t) * n, cudaMemcpyDeviceToHost, s));
        }
    }
    if (!on_device) HC_CUDA(cudaStreamSynchronize(s));
    return HICOPS_OK;
}

// ---- sampled partial score distributions (paper: Sampling section and its
// figure).  One warp per spectrum; lane l holds bins 8 l .. 8 l + 7.
namespace hicops {
namespace {

constexpr uint32_t kBinsPerLane = kHistBins / 32;

// warp-wide best of (count, bin) pairs: higher count, then lower bin
__device__ __forceinline__ void warp_best(uint32_t& c, uint32_t& j) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const uint32_t oc = __shfl_xor_sync(0xffffffffu, c, o), oj = __shfl_xor_sync(0xffffffffu, j, o);
        if (oc > c || (oc == c && oj < j)) { c = oc; j = oj; }
    }
}

__global__ void hist_sample_kernel(const uint32_t* __restrict__ hist, uint32_t n, uint32_t s,
                                   uint32_t* __restrict__ rec) {
    const uint32_t lane = threadIdx.x & 31;
    const uint32_t q = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (q >= n) return;
    const uint32_t* h = hist + (uint64_t)q * kHistBins;
    uint32_t v[kBinsPerLane];
#pragma unroll
    for (uint32_t i = 0; i < kBinsPerLane; ++i) v[i] = h[lane * kBinsPerLane + i];
    // support [L, R] of the non-zero bins
    uint32_t L = kHistBins, R = 0;
#pragma unroll
    for (uint32_t i = 0; i < kBinsPerLane; ++i)
        if (v[i]) { L = min(L, lane * kBinsPerLane + i); R = max(R, lane * kBinsPerLane + i); }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        L = min(L, __shfl_xor_sync(0xffffffffu, L, o));
        R = max(R, __shfl_xor_sync(0xffffffffu, R, o));
    }
    uint32_t* out = rec + (uint64_t)q * (s + 1);
    uint32_t lo = 0, len = 0;
    if (L <= R) {
        // the three most intense bins: three rounds of a warp arg-max, each
        // winner taken out of the next round
        uint32_t taken = 0, sum = 0, k = 0;
        for (int r = 0; r < 3; ++r) {
            uint32_t c = 0, j = 0xffffffffu;
#pragma unroll
            for (uint32_t i = 0; i < kBinsPerLane; ++i) {
                const uint32_t b = lane * kBinsPerLane + i;
                if (!((taken >> i) & 1u) && (v[i] > c || (v[i] == c && v[i] && b < j))) { c = v[i]; j = b; }
            }
            warp_best(c, j);
            if (c == 0) break;
            sum += j;
            ++k;
            if (j / kBinsPerLane == lane) taken |= 1u << (j % kBinsPerLane);
        }
        const uint32_t m = sum / k;
        if (R - L + 1 <= s) {
            lo = L;
            len = R - L + 1;
        } else {
            // pruning the farther end first ends with s bins, the lower side
            // longer by at most one, unless an end of the support stops it
            const int dl = (int)(s / 2), dh = (int)((s - 1) / 2);
            int a = (int)m - dl, b = (int)m + dh;
            if (a < (int)L) { a = (int)L; b = (int)L + (int)s - 1; }
            else if (b > (int)R) { b = (int)R; a = (int)R - (int)s + 1; }
            lo = (uint32_t)a;
            len = s;
        }
    }
    if (lane == 0) out[0] = lo | (len << 16);
    for (uint32_t i = lane; i < s; i += 32) out[1 + i] = i < len ? h[lo + i] : 0u;
}

__global__ void hist_unsample_kernel(const uint32_t* __restrict__ rec, uint32_t n_parts, uint32_t n, uint32_t s,
                                     uint32_t* __restrict__ hist, uint32_t* __restrict__ bad) {
    const uint32_t lane = threadIdx.x & 31;
    const uint32_t q = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (q >= n) return;
    uint32_t acc[kBinsPerLane];
#pragma unroll
    for (uint32_t i = 0; i < kBinsPerLane; ++i) acc[i] = 0;
    for (uint32_t p = 0; p < n_parts; ++p) {
        const uint32_t* r = rec + ((uint64_t)p * n + q) * (s + 1);
        const uint32_t w0 = r[0], lo = w0 & 0xffffu, len = w0 >> 16;
        if (len > s || lo + len > kHistBins) {   // not a record of this s
            if (lane == 0) atomicOr(bad, 1u);
            continue;
        }
#pragma unroll
        for (uint32_t i = 0; i < kBinsPerLane; ++i) {
            const uint32_t b = lane * kBinsPerLane + i;
            if (b >= lo && b < lo + len) acc[i] += r[1 + (b - lo)];
        }
    }
#pragma unroll
    for (uint32_t i = 0; i < kBinsPerLane; ++i) hist[(uint64_t)q * kHistBins + lane * kBinsPerLane + i] = acc[i];
}

constexpr int kSampleWarps = 8;

}  // namespace
}  // namespace hicops

extern "C" hicops_status hicops_hist_sample(uint32_t n, const uint32_t* hist, uint32_t s, uint32_t* out_rec,
                                            int on_device, void* cuda_stream) {
    if (s < 1 || s > kHistBins) { set_error("s must be in [1, %u]", kHistBins); return HICOPS_EINVAL; }
    if (n == 0) return HICOPS_OK;
    if (!hist || !out_rec) { set_error("NULL argument"); return HICOPS_EINVAL; }
    cudaStream_t st = (cudaStream_t)cuda_stream;
    {
        Scratch sc(st);
        const uint32_t* d_h = hist;
        uint32_t* d_r = out_rec;
        if (!on_device) {
            uint32_t* h;
            HC_CUDA(sc.get(&h, (uint64_t)n * kHistBins));
            HC_CUDA(sc.get(&d_r, (uint64_t)n * (s + 1)));
            HC_CUDA(cudaMemcpyAsync(h, hist, sizeof(uint32_t) * n * kHistBins, cudaMemcpyHostToDevice, st));
            d_h = h;
        }
        hist_sample_kernel<<<(n + kSampleWarps - 1) / kSampleWarps, kSampleWarps * 32, 0, st>>>(d_h, n, s, d_r);
        count_launches(1);
        HC_CUDA(cudaGetLastError());
        if (!on_device)
            HC_CUDA(cudaMemcpyAsync(out_rec, d_r, sizeof(uint32_t) * n * (s + 1), cudaMemcpyDeviceToHost, st));
    }
    if (!on_device) HC_CUDA(cudaStreamSynchronize(st));
    return HICOPS_OK;
}

extern "C" hicops_status hicops_hist_unsample(uint32_t n_parts, uint32_t n, uint32_t s, const uint32_t* rec,
                                              uint32_t* out_hist, int on_device, void* cuda_stream) {
    if (s < 1 || s > kHistBins) { set_error("s must be in [1, %u]", kHistBins); return HICOPS_EINVAL; }
    if (n_parts < 1 || n_parts > HICOPS_MAX_SHARDS) {
        set_error("n_parts must be in [1, %u]", (unsigned)HICOPS_MAX_SHARDS);
        return HICOPS_EINVAL;
    }
    if (n == 0) return HICOPS_OK;
    if (!rec || !out_hist) { set_error("NULL argument"); return HICOPS_EINVAL; }
    cudaStream_t st = (cudaStream_t)cuda_stream;
    uint32_t bad = 0;
    {
        Scratch sc(st);
        const uint32_t* d_r = rec;
        uint32_t* d_h = out_hist;
        uint32_t* d_bad;
        HC_CUDA(sc.get(&d_bad, 1));
        HC_CUDA(cudaMemsetAsync(d_bad, 0, sizeof(uint32_t), st));
        if (!on_device) {
            uint32_t* r;
            HC_CUDA(sc.get(&r, (uint64_t)n_parts * n * (s + 1)));
            HC_CUDA(sc.get(&d_h, (uint64_t)n * kHistBins));
            HC_CUDA(cudaMemcpyAsync(r, rec, sizeof(uint32_t) * n_parts * n * (s + 1), cudaMemcpyHostToDevice, st));
            d_r = r;
        }
        hist_unsample_kernel<<<(n + kSampleWarps - 1) / kSampleWarps, kSampleWarps * 32, 0, st>>>(d_r, n_parts, n, s,
                                                                                                 d_h, d_bad);
        count_launches(1);
        HC_CUDA(cudaGetLastError());
        if (!on_device)
            HC_CUDA(cudaMemcpyAsync(out_hist, d_h, sizeof(uint32_t) * n * kHistBins, cudaMemcpyDeviceToHost, st));
        HC_CUDA(cudaMemcpyAsync(&bad, d_bad, sizeof(uint32_t), cudaMemcpyDeviceToHost, st));
        HC_CUDA(cudaStreamSynchronize(st));
    }
    if (bad) { set_error("a sampled record's bins leave [0, 256) or exceed s"); return HICOPS_EINVAL; }
    return HICOPS_OK;
}
