// Serving loop: continuous batching of search requests over several CUDA
// streams (the paper's superstep-3 buffering between the R, I and K
// sub-tasks, Buffering / Task Scheduling sections, recast as a request
// server on one GPU).
//
// submit() copies a request and queues it.  Device memory is one pool of
// memory_budget bytes, allocated at creation.  The scheduler thread packs the
// oldest waiting requests into one launch for as long as the launch's block
// (its spectra, the search's scratch and its outputs, sized exactly for
// them) fits the largest free range of the pool, takes that block, copies
// the spectra into it and enqueues the search on an idle stream.  When the
// oldest request does not fit, it waits until launches in flight give their
// blocks back: requests are admitted by device memory, and at most n_slots
// launches are in flight.  A completion thread per stream waits for its
// launch's event, hands each request its rows and returns the block.  Work
// of different streams overlaps on the device.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <iterator>
#include <map>
#include <memory>
#include <mutex>
#include <thread>
#include <vector>

#include "dev_common.cuh"
#include "pool_map.h"
#include "search_scratch.h"

namespace {

using hicops::set_error;

struct Request {
    uint64_t id = 0;
    uint32_t n = 0;
    uint64_t npk = 0;
    std::vector<uint64_t> peak_off;
    std::vector<float> mz, inten;
    std::vector<double> prec, tol;
    std::vector<uint8_t> z;
    std::vector<hicops_psm> psm;
    std::vector<uint32_t> hist, ns;
    enum State { kQueued, kLaunched, kDone, kCancelled, kFailed } state = kQueued;
    hicops_status err = HICOPS_OK;
};

template <class T>
struct Pinned {
    T* p = nullptr;
    size_t cap = 0;
    cudaError_t reserve(size_t n) {
        if (n <= cap) return cudaSuccess;
        if (p) cudaFreeHost(p);
        p = nullptr;
        cap = 0;
        cudaError_t e = cudaHostAlloc((void**)&p, sizeof(T) * (n ? n : 1), cudaHostAllocDefault);
        if (e == cudaSuccess) cap = n;
        return e;
    }
    ~Pinned() { if (p) cudaFreeHost(p); }
};

constexpr uint32_t kMaxLanes = 64;   // launches in flight at most (n_slots)

constexpr uint64_t piece(uint64_t bytes) { return (std::max<uint64_t>(bytes, 1) + 255) & ~uint64_t(255); }

// One launch in flight at a time: its stream, its event, the pinned staging
// of its spectra and results, and its block of the pool.
struct Lane {
    cudaStream_t stream = nullptr;
    cudaEvent_t done = nullptr;
    Pinned<uint64_t> h_off;
    Pinned<float> h_mz, h_in;
    Pinned<double> h_prec, h_tol;
    Pinned<uint8_t> h_z;
    Pinned<hicops_psm> h_psm;
    Pinned<uint32_t> h_hist, h_ns;
    std::vector<std::shared_ptr<Request>> batch;   // requests in flight, in packing order
    uint32_t n = 0;
    uint64_t npk = 0;
    uint64_t off = 0, bytes = 0;   // the launch's block of the pool
    bool busy = false;       // packed (scheduler) until results are handed out (waiter)
    bool launched = false;   // the lane's event has been recorded
    std::thread waiter;
};

}  // namespace

struct hicops_server {
    hicops_index* idx = nullptr;
    int device = 0;
    uint32_t cap = 0;                // spectra per launch at most
    uint32_t k = 0;
    hicops_search_config cfg{};      // launch shape, fixed at creation
    unsigned char* pool = nullptr;   // device pool of map.size bytes
    hicops::PoolMap map;
    std::vector<std::unique_ptr<Lane>> lanes;
    std::mutex mu;
    std::condition_variable cv_sched;   // queue, lanes or pool changed
    std::condition_variable cv_done;    // a request finished
    std::condition_variable cv_lane;    // a lane was launched (for its waiter)
    std::deque<std::shared_ptr<Request>> queue;
    std::map<uint64_t, std::shared_ptr<Request>> reqs;
    uint64_t next_id = 1;
    bool stop = false;
    std::thread scheduler;
    hicops_server_stats st{};
};

namespace {

// Device bytes of one launch of n spectra holding npk peaks, in the order
// launch() lays the block out: peak offsets, m/z, intensities, precursor
// m/z, tolerances, charges, PSM rows, histograms, candidate counts, then the
// search's scratch.
uint64_t launch_bytes(const hicops_server* srv, uint32_t n, uint64_t npk) {
    return piece(8ull * (n + 1)) + 2 * piece(4 * npk) + 2 * piece(8ull * n) + piece(n) +
           piece(sizeof(hicops_psm) * (uint64_t)n * srv->k) + piece(4ull * n * hicops::kHistBins) + piece(4ull * n) +
           hicops::scratch_bytes(srv->idx, srv->cfg, n);
}

hicops_status launch(hicops_server* srv, Lane& ln) {
    // pack the lane's requests into one batch in pinned memory
    const uint32_t n = ln.n;
    const uint64_t npk = ln.npk;
    HC_CUDA(ln.h_off.reserve(n + 1));
    HC_CUDA(ln.h_mz.reserve(npk));
    HC_CUDA(ln.h_in.reserve(npk));
    HC_CUDA(ln.h_prec.reserve(n));
    HC_CUDA(ln.h_tol.reserve(n));
    HC_CUDA(ln.h_z.reserve(n));
    HC_CUDA(ln.h_psm.reserve((size_t)n * srv->k));
    HC_CUDA(ln.h_hist.reserve((size_t)n * hicops::kHistBins));
    HC_CUDA(ln.h_ns.reserve(n));
    uint64_t po = 0;
    uint32_t q = 0;
    for (auto& r : ln.batch) {
        for (uint32_t i = 0; i < r->n; ++i) ln.h_off.p[q + i] = po + r->peak_off[i];
        memcpy(ln.h_mz.p + po, r->mz.data(), sizeof(float) * r->npk);
        memcpy(ln.h_in.p + po, r->inten.data(), sizeof(float) * r->npk);
        memcpy(ln.h_prec.p + q, r->prec.data(), sizeof(double) * r->n);
        memcpy(ln.h_tol.p + q, r->tol.data(), sizeof(double) * r->n);
        memcpy(ln.h_z.p + q, r->z.data(), r->n);
        po += r->npk;
        q += r->n;
    }
    ln.h_off.p[n] = po;
    // the block, laid out as launch_bytes counts it
    unsigned char* at = srv->pool + ln.off;
    auto take = [&](uint64_t bytes) {
        unsigned char* p = at;
        at += piece(bytes);
        return (void*)p;
    };
    auto* d_off = static_cast<uint64_t*>(take(8ull * (n + 1)));
    auto* d_mz = static_cast<float*>(take(4 * npk));
    auto* d_in = static_cast<float*>(take(4 * npk));
    auto* d_prec = static_cast<double*>(take(8ull * n));
    auto* d_tol = static_cast<double*>(take(8ull * n));
    auto* d_z = static_cast<uint8_t*>(take(n));
    auto* d_psm = static_cast<hicops_psm*>(take(sizeof(hicops_psm) * (uint64_t)n * srv->k));
    auto* d_hist = static_cast<uint32_t*>(take(4ull * n * hicops::kHistBins));
    auto* d_ns = static_cast<uint32_t*>(take(4ull * n));
    const uint64_t used = (uint64_t)(at - (srv->pool + ln.off));
    cudaStream_t s = ln.stream;
    HC_CUDA(cudaMemcpyAsync(d_off, ln.h_off.p, sizeof(uint64_t) * (n + 1), cudaMemcpyHostToDevice, s));
    if (npk) {
        HC_CUDA(cudaMemcpyAsync(d_mz, ln.h_mz.p, sizeof(float) * npk, cudaMemcpyHostToDevice, s));
        HC_CUDA(cudaMemcpyAsync(d_in, ln.h_in.p, sizeof(float) * npk, cudaMemcpyHostToDevice, s));
    }
    HC_CUDA(cudaMemcpyAsync(d_prec, ln.h_prec.p, sizeof(double) * n, cudaMemcpyHostToDevice, s));
    HC_CUDA(cudaMemcpyAsync(d_tol, ln.h_tol.p, sizeof(double) * n, cudaMemcpyHostToDevice, s));
    HC_CUDA(cudaMemcpyAsync(d_z, ln.h_z.p, n, cudaMemcpyHostToDevice, s));
    hicops_batch b{n, 1, d_off, d_mz, d_in, d_prec, d_z, d_tol, s};
    hicops_status st =
        hicops::search_in_scratch(srv->idx, &b, srv->cfg, at, ln.bytes - used, d_psm, d_hist, d_ns);
    if (st != HICOPS_OK) return st;
    HC_CUDA(cudaMemcpyAsync(ln.h_psm.p, d_psm, sizeof(hicops_psm) * n * srv->k, cudaMemcpyDeviceToHost, s));
    HC_CUDA(cudaMemcpyAsync(ln.h_hist.p, d_hist, sizeof(uint32_t) * n * hicops::kHistBins, cudaMemcpyDeviceToHost,
                            s));
    HC_CUDA(cudaMemcpyAsync(ln.h_ns.p, d_ns, sizeof(uint32_t) * n, cudaMemcpyDeviceToHost, s));
    HC_CUDA(cudaEventRecord(ln.done, s));
    return HICOPS_OK;
}

void scheduler_main(hicops_server* srv) {
    cudaSetDevice(srv->device);
    std::unique_lock<std::mutex> lk(srv->mu);
    bool short_of_memory = false;   // the oldest request is waiting for pool memory
    for (;;) {
        Lane* lane = nullptr;
        srv->cv_sched.wait(lk, [&] {
            if (srv->stop) return true;
            while (!srv->queue.empty() && srv->queue.front()->state == Request::kCancelled) srv->queue.pop_front();
            if (srv->queue.empty()) return false;
            for (auto& l : srv->lanes)
                if (!l->busy) { lane = l.get(); return true; }
            return false;
        });
        if (srv->stop) return;
        // the oldest waiting requests whose launch fits the largest free range
        const uint64_t room = srv->map.largest();
        std::vector<std::shared_ptr<Request>> pack;
        uint32_t n = 0;
        uint64_t npk = 0, bytes = 0;
        size_t taken = 0;   // queue entries packed or skipped as cancelled
        for (auto& r : srv->queue) {
            if (r->state == Request::kCancelled) { ++taken; continue; }
            if (n + r->n > srv->cap) break;
            const uint64_t b = launch_bytes(srv, n + r->n, npk + r->npk);
            if (b > room) break;
            pack.push_back(r);
            n += r->n;
            npk += r->npk;
            bytes = b;
            ++taken;
        }
        if (pack.empty()) {
            // a launch in flight gives its block back, a request arrives or
            // the server stops; submit() keeps every request within the pool
            if (!short_of_memory) srv->st.memory_waits++;
            short_of_memory = true;
            srv->cv_sched.wait(lk);
            continue;
        }
        short_of_memory = false;
        uint64_t off = 0;
        if (!srv->map.take(bytes, &off)) continue;   // cannot happen: bytes <= the largest free range
        srv->queue.erase(srv->queue.begin(), srv->queue.begin() + (std::ptrdiff_t)taken);
        for (auto& r : pack) r->state = Request::kLaunched;
        Lane& ln = *lane;
        ln.batch = std::move(pack);
        ln.n = n;
        ln.npk = npk;
        ln.off = off;
        ln.bytes = bytes;
        ln.busy = true;
        srv->st.pool_peak = srv->map.peak;
        lk.unlock();
        hicops_status st = launch(srv, ln);
        lk.lock();
        if (st != HICOPS_OK) {
            // nothing of the launch runs past a failed call: wait for what was
            // enqueued before the block goes back
            lk.unlock();
            cudaStreamSynchronize(ln.stream);
            lk.lock();
            for (auto& r : ln.batch) { r->state = Request::kFailed; r->err = st; }
            ln.batch.clear();
            srv->map.give(ln.off, ln.bytes);
            ln.busy = false;
            srv->cv_done.notify_all();
            continue;
        }
        ln.launched = true;
        srv->st.launches++;
        srv->st.spectra += n;
        srv->cv_lane.notify_all();
    }
}

void waiter_main(hicops_server* srv, Lane* ln) {
    cudaSetDevice(srv->device);
    std::unique_lock<std::mutex> lk(srv->mu);
    for (;;) {
        srv->cv_lane.wait(lk, [&] { return srv->stop || ln->launched; });
        if (ln->launched) {
            lk.unlock();
            const cudaError_t e = cudaEventSynchronize(ln->done);
            lk.lock();
            uint32_t q = 0;
            for (auto& r : ln->batch) {
                if (e != cudaSuccess) {
                    r->state = Request::kFailed;
                    r->err = HICOPS_ECUDA;
                } else {
                    r->psm.assign(ln->h_psm.p + (uint64_t)q * srv->k, ln->h_psm.p + (uint64_t)(q + r->n) * srv->k);
                    for (auto& row : r->psm) row.query -= q;
                    r->hist.assign(ln->h_hist.p + (uint64_t)q * hicops::kHistBins,
                                   ln->h_hist.p + (uint64_t)(q + r->n) * hicops::kHistBins);
                    r->ns.assign(ln->h_ns.p + q, ln->h_ns.p + q + r->n);
                    r->state = Request::kDone;
                }
                q += r->n;
                srv->st.completed++;
            }
            ln->batch.clear();
            if (e == cudaSuccess) srv->map.give(ln->off, ln->bytes);   // else the block stays out of use
            ln->launched = false;
            ln->busy = false;
            srv->cv_done.notify_all();
            srv->cv_sched.notify_all();
            continue;
        }
        if (srv->stop) return;
    }
}

void free_server(hicops_server* srv) {
    cudaSetDevice(srv->device);
    for (auto& ln : srv->lanes) {
        if (ln->stream) cudaStreamSynchronize(ln->stream);
        if (ln->done) cudaEventDestroy(ln->done);
        if (ln->stream) cudaStreamDestroy(ln->stream);
    }
    if (srv->pool) cudaFree(srv->pool);
    delete srv;
}

}  // namespace

extern "C" hicops_status hicops_server_create(hicops_index* idx, const hicops_server_cfg* cfg_in,
                                              hicops_server** out) {
    if (!idx || !out) { set_error("NULL argument"); return HICOPS_EINVAL; }
    *out = nullptr;
    if (!idx->dev.ready) { set_error("index not uploaded"); return HICOPS_EINVAL; }
    hicops_server_cfg cfg = cfg_in ? *cfg_in : hicops_server_cfg{0, 0, 0};
    if (!cfg.n_slots) cfg.n_slots = 4;
    if (!cfg.slot_spectra) cfg.slot_spectra = 32768;
    if (!cfg.memory_budget) cfg.memory_budget = 16ull << 30;
    if (cfg.n_slots > kMaxLanes) {   // each costs a stream, a thread and pinned staging
        set_error("n_slots must be at most %u", kMaxLanes);
        return HICOPS_EINVAL;
    }
    HC_CUDA(cudaSetDevice(idx->dev.device));
    uint64_t probe = 0;
    hicops_status st = hicops_search_scratch_bytes(idx, 1, &probe);   // also learns the SM count
    if (st != HICOPS_OK) return st;
    std::unique_ptr<hicops_server, void (*)(hicops_server*)> srv(new hicops_server(), free_server);
    srv->idx = idx;
    srv->device = idx->dev.device;
    srv->cap = cfg.slot_spectra;
    srv->k = idx->p.top_k;
    srv->cfg = idx->dev.cfg;
    const uint64_t pool_bytes = cfg.memory_budget & ~uint64_t(255);
    const uint64_t one = launch_bytes(srv.get(), 1, 512);
    if (pool_bytes < one) {
        set_error("memory budget of %llu bytes is below one launch of one 512-peak spectrum (%llu bytes)",
                  (unsigned long long)cfg.memory_budget, (unsigned long long)one);
        return HICOPS_EINVAL;
    }
    if (cudaMalloc((void**)&srv->pool, pool_bytes) != cudaSuccess) {
        cudaGetLastError();
        srv->pool = nullptr;
        set_error("cannot allocate the server's device pool of %llu bytes", (unsigned long long)pool_bytes);
        return HICOPS_ENOMEM;
    }
    srv->map.init(pool_bytes);
    srv->st.pool_bytes = pool_bytes;
    for (uint32_t i = 0; i < cfg.n_slots; ++i) {
        auto ln = std::make_unique<Lane>();
        HC_CUDA(cudaStreamCreateWithFlags(&ln->stream, cudaStreamNonBlocking));
        HC_CUDA(cudaEventCreateWithFlags(&ln->done, cudaEventDisableTiming));
        // result staging for a full launch now; spectra staging grows on use
        HC_CUDA(ln->h_psm.reserve((size_t)cfg.slot_spectra * srv->k));
        HC_CUDA(ln->h_hist.reserve((size_t)cfg.slot_spectra * hicops::kHistBins));
        HC_CUDA(ln->h_ns.reserve(cfg.slot_spectra));
        srv->lanes.push_back(std::move(ln));
    }
    srv->st.n_slots = cfg.n_slots;
    hicops_server* s = srv.release();
    for (auto& ln : s->lanes) ln->waiter = std::thread(waiter_main, s, ln.get());
    s->scheduler = std::thread(scheduler_main, s);
    *out = s;
    return HICOPS_OK;
}

extern "C" hicops_status hicops_server_submit(hicops_server* srv, const hicops_batch* b, uint64_t* ticket) {
    if (!srv || !b || !ticket) { set_error("NULL argument"); return HICOPS_EINVAL; }
    if (b->on_device) { set_error("server requests are host batches (on_device = 0)"); return HICOPS_EINVAL; }
    if (b->n == 0 || b->n > srv->cap) { set_error("request of %u spectra (1..%u)", b->n, srv->cap); return HICOPS_EINVAL; }
    if (!b->peak_off || !b->prec_mz || !b->charge || !b->prec_tol_da) { set_error("batch pointers are NULL"); return HICOPS_EINVAL; }
    const uint32_t n = b->n;
    for (uint32_t i = 0; i < n; ++i)
        if (b->peak_off[i + 1] < b->peak_off[i]) {
            set_error("peak offsets decrease at spectrum %u", i);
            return HICOPS_EINVAL;
        }
    auto r = std::make_shared<Request>();
    r->n = n;
    const uint64_t base = b->peak_off[0];
    r->peak_off.resize(n + 1);
    for (uint32_t i = 0; i <= n; ++i) r->peak_off[i] = b->peak_off[i] - base;
    const uint64_t m = r->peak_off[n];
    if (m && (!b->mz || !b->intensity)) { set_error("peak arrays are NULL"); return HICOPS_EINVAL; }
    const uint64_t need = launch_bytes(srv, n, m);
    if (need > srv->map.size) {
        set_error("a request of %u spectra and %llu peaks needs %llu bytes of device memory; the pool holds %llu", n,
                  (unsigned long long)m, (unsigned long long)need, (unsigned long long)srv->map.size);
        return HICOPS_EINVAL;
    }
    r->npk = m;
    r->mz.assign(b->mz + base, b->mz + base + m);
    r->inten.assign(b->intensity + base, b->intensity + base + m);
    r->prec.assign(b->prec_mz, b->prec_mz + n);
    r->tol.assign(b->prec_tol_da, b->prec_tol_da + n);
    r->z.assign(b->charge, b->charge + n);
    std::lock_guard<std::mutex> lk(srv->mu);
    r->id = srv->next_id++;
    srv->reqs[r->id] = r;
    srv->queue.push_back(r);
    srv->st.submitted++;
    *ticket = r->id;
    srv->cv_sched.notify_all();
    return HICOPS_OK;
}

extern "C" hicops_status hicops_server_poll(hicops_server* srv, uint64_t ticket, int timeout_ms, hicops_psm* out_psm,
                                            uint32_t* out_hist, uint32_t* out_nscored) {
    if (!srv) { set_error("server is NULL"); return HICOPS_EINVAL; }
    std::unique_lock<std::mutex> lk(srv->mu);
    auto it = srv->reqs.find(ticket);
    if (it == srv->reqs.end()) { set_error("unknown ticket %llu", (unsigned long long)ticket); return HICOPS_EINVAL; }
    std::shared_ptr<Request> r = it->second;
    auto finished = [&] {
        return r->state == Request::kDone || r->state == Request::kCancelled || r->state == Request::kFailed;
    };
    if (timeout_ms < 0) srv->cv_done.wait(lk, finished);
    else if (!srv->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), finished)) return HICOPS_ETIMEOUT;
    srv->reqs.erase(it);
    if (r->state == Request::kCancelled) { set_error("request cancelled"); return HICOPS_ECANCELLED; }
    if (r->state == Request::kFailed) { set_error("request failed"); return r->err; }
    if (out_psm) memcpy(out_psm, r->psm.data(), sizeof(hicops_psm) * r->psm.size());
    if (out_hist) memcpy(out_hist, r->hist.data(), sizeof(uint32_t) * r->hist.size());
    if (out_nscored) memcpy(out_nscored, r->ns.data(), sizeof(uint32_t) * r->ns.size());
    return HICOPS_OK;
}

extern "C" hicops_status hicops_server_cancel(hicops_server* srv, uint64_t ticket) {
    if (!srv) { set_error("server is NULL"); return HICOPS_EINVAL; }
    std::lock_guard<std::mutex> lk(srv->mu);
    auto it = srv->reqs.find(ticket);
    if (it == srv->reqs.end()) { set_error("unknown ticket"); return HICOPS_EINVAL; }
    if (it->second->state != Request::kQueued) { set_error("request already launched"); return HICOPS_EBUSY; }
    it->second->state = Request::kCancelled;
    srv->cv_done.notify_all();
    return HICOPS_OK;
}

extern "C" hicops_status hicops_server_get_stats(hicops_server* srv, hicops_server_stats* out) {
    if (!srv || !out) { set_error("NULL argument"); return HICOPS_EINVAL; }
    std::lock_guard<std::mutex> lk(srv->mu);
    *out = srv->st;
    return HICOPS_OK;
}

extern "C" void hicops_server_destroy(hicops_server* srv) {
    if (!srv) return;
    {
        std::lock_guard<std::mutex> lk(srv->mu);
        srv->stop = true;
        for (auto& r : srv->queue)
            if (r->state == Request::kQueued) r->state = Request::kCancelled;
        srv->queue.clear();
    }
    srv->cv_sched.notify_all();
    if (srv->scheduler.joinable()) srv->scheduler.join();
    // launched lanes finish: their waiters hand out results, then exit
    for (auto& ln : srv->lanes) {
        srv->cv_lane.notify_all();
        if (ln->waiter.joinable()) ln->waiter.join();
    }
    srv->cv_done.notify_all();
    free_server(srv);
}
