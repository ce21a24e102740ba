// Serving loop: continuous batching of search requests over several CUDA
// streams (the paper's superstep-3 buffering between the R, I and K
// sub-tasks, Buffering / Task Scheduling sections, recast as a request
// server on one GPU).
//
// submit() copies a request and queues it.  The scheduler thread packs the
// waiting requests, oldest first, into the next free slot (a stream with a
// reusable search plan and pinned staging buffers) and launches them as one
// batch; a completion thread per slot waits for the slot's event, hands each
// request its rows and frees the slot.  Requests that arrive while slots are
// busy are admitted as soon as one frees up; work of different slots
// overlaps on the device.  All waits are host waits with limits.
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <thread>
#include <vector>

#include "dev_common.cuh"

namespace {

using hicops::set_error;

struct Request {
    uint64_t id = 0;
    uint32_t n = 0;
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

template <class T>
struct DevBuf {
    T* p = nullptr;
    size_t cap = 0;
    cudaError_t reserve(size_t n) {
        if (n <= cap) return cudaSuccess;
        if (p) cudaFree(p);
        p = nullptr;
        cap = 0;
        cudaError_t e = cudaMalloc((void**)&p, sizeof(T) * (n ? n : 1));
        if (e == cudaSuccess) cap = n;
        return e;
    }
    ~DevBuf() { if (p) cudaFree(p); }
};

struct Slot {
    cudaStream_t stream = nullptr;
    cudaEvent_t done = nullptr;
    hicops_plan* plan = nullptr;
    Pinned<uint64_t> h_off;
    Pinned<float> h_mz, h_in;
    Pinned<double> h_prec, h_tol;
    Pinned<uint8_t> h_z;
    Pinned<hicops_psm> h_psm;
    Pinned<uint32_t> h_hist, h_ns;
    DevBuf<uint64_t> d_off;
    DevBuf<float> d_mz, d_in;
    DevBuf<double> d_prec, d_tol;
    DevBuf<uint8_t> d_z;
    DevBuf<hicops_psm> d_psm;
    DevBuf<uint32_t> d_hist, d_ns;
    std::vector<std::shared_ptr<Request>> batch;   // requests in flight, in packing order
    uint32_t n = 0;
    bool busy = false;       // packed (scheduler) until results are handed out (waiter)
    bool launched = false;   // the slot's event has been recorded
    std::thread waiter;
};

}  // namespace

struct hicops_server {
    hicops_index* idx = nullptr;
    int device = 0;
    uint32_t cap = 0;        // spectra per slot
    uint32_t k = 0;
    std::vector<std::unique_ptr<Slot>> slots;
    std::mutex mu;
    std::condition_variable cv_sched;   // queue or slot state changed
    std::condition_variable cv_done;    // a request finished
    std::condition_variable cv_slot;    // a slot was launched (for its waiter)
    std::deque<std::shared_ptr<Request>> queue;
    std::map<uint64_t, std::shared_ptr<Request>> reqs;
    uint64_t next_id = 1;
    bool stop = false;
    std::thread scheduler;
    hicops_server_stats st{};
};

namespace {

hicops_status launch_slot(hicops_server* srv, Slot& sl) {
    // pack the slot's requests into one batch in pinned memory
    uint64_t npk = 0;
    for (auto& r : sl.batch) npk += r->peak_off[r->n];
    const uint32_t n = sl.n;
    HC_CUDA(sl.h_off.reserve(n + 1));
    HC_CUDA(sl.h_mz.reserve(npk));
    HC_CUDA(sl.h_in.reserve(npk));
    HC_CUDA(sl.h_prec.reserve(n));
    HC_CUDA(sl.h_tol.reserve(n));
    HC_CUDA(sl.h_z.reserve(n));
    HC_CUDA(sl.d_off.reserve(n + 1));
    HC_CUDA(sl.d_mz.reserve(npk));
    HC_CUDA(sl.d_in.reserve(npk));
    HC_CUDA(sl.d_prec.reserve(n));
    HC_CUDA(sl.d_tol.reserve(n));
    HC_CUDA(sl.d_z.reserve(n));
    uint64_t po = 0;
    uint32_t q = 0;
    for (auto& r : sl.batch) {
        const uint64_t m = r->peak_off[r->n];
        for (uint32_t i = 0; i < r->n; ++i) sl.h_off.p[q + i] = po + r->peak_off[i];
        memcpy(sl.h_mz.p + po, r->mz.data(), sizeof(float) * m);
        memcpy(sl.h_in.p + po, r->inten.data(), sizeof(float) * m);
        memcpy(sl.h_prec.p + q, r->prec.data(), sizeof(double) * r->n);
        memcpy(sl.h_tol.p + q, r->tol.data(), sizeof(double) * r->n);
        memcpy(sl.h_z.p + q, r->z.data(), r->n);
        po += m;
        q += r->n;
    }
    sl.h_off.p[n] = po;
    cudaStream_t s = sl.stream;
    HC_CUDA(cudaMemcpyAsync(sl.d_off.p, sl.h_off.p, sizeof(uint64_t) * (n + 1), cudaMemcpyHostToDevice, s));
    if (npk) {
        HC_CUDA(cudaMemcpyAsync(sl.d_mz.p, sl.h_mz.p, sizeof(float) * npk, cudaMemcpyHostToDevice, s));
        HC_CUDA(cudaMemcpyAsync(sl.d_in.p, sl.h_in.p, sizeof(float) * npk, cudaMemcpyHostToDevice, s));
    }
    HC_CUDA(cudaMemcpyAsync(sl.d_prec.p, sl.h_prec.p, sizeof(double) * n, cudaMemcpyHostToDevice, s));
    HC_CUDA(cudaMemcpyAsync(sl.d_tol.p, sl.h_tol.p, sizeof(double) * n, cudaMemcpyHostToDevice, s));
    HC_CUDA(cudaMemcpyAsync(sl.d_z.p, sl.h_z.p, n, cudaMemcpyHostToDevice, s));
    hicops_batch b{n, 1, sl.d_off.p, sl.d_mz.p, sl.d_in.p, sl.d_prec.p, sl.d_z.p, sl.d_tol.p, s};
    hicops_status st = hicops_plan_search(sl.plan, &b, sl.d_psm.p, sl.d_hist.p, sl.d_ns.p, 0);
    if (st != HICOPS_OK) return st;
    HC_CUDA(cudaMemcpyAsync(sl.h_psm.p, sl.d_psm.p, sizeof(hicops_psm) * n * srv->k, cudaMemcpyDeviceToHost, s));
    HC_CUDA(cudaMemcpyAsync(sl.h_hist.p, sl.d_hist.p, sizeof(uint32_t) * n * hicops::kHistBins,
                            cudaMemcpyDeviceToHost, s));
    HC_CUDA(cudaMemcpyAsync(sl.h_ns.p, sl.d_ns.p, sizeof(uint32_t) * n, cudaMemcpyDeviceToHost, s));
    HC_CUDA(cudaEventRecord(sl.done, s));
    return HICOPS_OK;
}

void scheduler_main(hicops_server* srv) {
    cudaSetDevice(srv->device);
    std::unique_lock<std::mutex> lk(srv->mu);
    for (;;) {
        Slot* free_slot = nullptr;
        srv->cv_sched.wait(lk, [&] {
            if (srv->stop) return true;
            if (srv->queue.empty()) return false;
            for (auto& s : srv->slots) if (!s->busy) { free_slot = s.get(); return true; }
            return false;
        });
        if (srv->stop) return;
        // pack the oldest waiting requests that fit the slot
        Slot& sl = *free_slot;
        sl.batch.clear();
        sl.n = 0;
        while (!srv->queue.empty()) {
            auto r = srv->queue.front();
            if (r->state == Request::kCancelled) { srv->queue.pop_front(); continue; }
            if (sl.n + r->n > srv->cap) break;
            srv->queue.pop_front();
            r->state = Request::kLaunched;
            sl.batch.push_back(r);
            sl.n += r->n;
        }
        if (sl.batch.empty()) continue;
        sl.busy = true;
        lk.unlock();
        hicops_status st = launch_slot(srv, sl);
        lk.lock();
        if (st != HICOPS_OK) {
            for (auto& r : sl.batch) { r->state = Request::kFailed; r->err = st; }
            sl.batch.clear();
            sl.busy = false;
            srv->cv_done.notify_all();
            continue;
        }
        sl.launched = true;
        srv->st.launches++;
        srv->st.spectra += sl.n;
        srv->cv_slot.notify_all();
    }
}

void waiter_main(hicops_server* srv, Slot* sl) {
    cudaSetDevice(srv->device);
    std::unique_lock<std::mutex> lk(srv->mu);
    for (;;) {
        srv->cv_slot.wait(lk, [&] { return srv->stop || sl->launched; });
        if (sl->launched) {
            lk.unlock();
            const cudaError_t e = cudaEventSynchronize(sl->done);
            lk.lock();
            uint32_t q = 0;
            for (auto& r : sl->batch) {
                if (e != cudaSuccess) {
                    r->state = Request::kFailed;
                    r->err = HICOPS_ECUDA;
                } else {
                    r->psm.assign(sl->h_psm.p + (uint64_t)q * srv->k, sl->h_psm.p + (uint64_t)(q + r->n) * srv->k);
                    for (auto& row : r->psm) row.query -= q;
                    r->hist.assign(sl->h_hist.p + (uint64_t)q * hicops::kHistBins,
                                   sl->h_hist.p + (uint64_t)(q + r->n) * hicops::kHistBins);
                    r->ns.assign(sl->h_ns.p + q, sl->h_ns.p + q + r->n);
                    r->state = Request::kDone;
                }
                q += r->n;
                srv->st.completed++;
            }
            sl->batch.clear();
            sl->launched = false;
            sl->busy = false;
            srv->cv_done.notify_all();
            srv->cv_sched.notify_all();
            continue;
        }
        if (srv->stop) return;
    }
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
    auto srv = std::make_unique<hicops_server>();
    srv->idx = idx;
    srv->device = idx->dev.device;
    srv->cap = cfg.slot_spectra;
    srv->k = idx->p.top_k;
    HC_CUDA(cudaSetDevice(srv->device));
    // scratch of one slot: the plan (per spectrum: retained peaks, window,
    // units, per-unit top-k, rows, histogram) plus staged inputs (up to
    // 512 peaks per spectrum before it grows)
    const hicops_params& p = idx->p;
    const uint64_t per_spec = 8ull * hicops::query_bins_cap(p) + 48 + 64ull * p.top_k * 16 + p.top_k * 32ull * 2 +
                              2 * 4 * hicops::kHistBins + 8 + 512ull * 8 + 17;
    const uint64_t slot_bytes = per_spec * cfg.slot_spectra;
    uint64_t n_slots = cfg.memory_budget / (slot_bytes ? slot_bytes : 1);
    if (n_slots > cfg.n_slots) n_slots = cfg.n_slots;
    if (n_slots < 1) { set_error("memory budget below one slot (%llu bytes)", (unsigned long long)slot_bytes); return HICOPS_EINVAL; }
    srv->st.slot_bytes = slot_bytes;
    for (uint64_t i = 0; i < n_slots; ++i) {
        auto sl = std::make_unique<Slot>();
        HC_CUDA(cudaStreamCreateWithFlags(&sl->stream, cudaStreamNonBlocking));
        HC_CUDA(cudaEventCreateWithFlags(&sl->done, cudaEventDisableTiming));
        hicops_status st = hicops_plan_create(idx, cfg.slot_spectra, nullptr, &sl->plan);
        if (st != HICOPS_OK) return st;
        HC_CUDA(sl->d_psm.reserve((size_t)cfg.slot_spectra * srv->k));
        HC_CUDA(sl->d_hist.reserve((size_t)cfg.slot_spectra * hicops::kHistBins));
        HC_CUDA(sl->d_ns.reserve(cfg.slot_spectra));
        HC_CUDA(sl->h_psm.reserve((size_t)cfg.slot_spectra * srv->k));
        HC_CUDA(sl->h_hist.reserve((size_t)cfg.slot_spectra * hicops::kHistBins));
        HC_CUDA(sl->h_ns.reserve(cfg.slot_spectra));
        srv->slots.push_back(std::move(sl));
    }
    srv->st.n_slots = (uint32_t)n_slots;
    hicops_server* s = srv.release();
    for (auto& sl : s->slots) sl->waiter = std::thread(waiter_main, s, sl.get());
    s->scheduler = std::thread(scheduler_main, s);
    *out = s;
    return HICOPS_OK;
}

extern "C" hicops_status hicops_server_submit(hicops_server* srv, const hicops_batch* b, uint64_t* ticket) {
    if (!srv || !b || !ticket) { set_error("NULL argument"); return HICOPS_EINVAL; }
    if (b->on_device) { set_error("server requests are host batches (on_device = 0)"); return HICOPS_EINVAL; }
    if (b->n == 0 || b->n > srv->cap) { set_error("request of %u spectra (1..%u)", b->n, srv->cap); return HICOPS_EINVAL; }
    if (!b->peak_off || !b->prec_mz || !b->charge || !b->prec_tol_da) { set_error("batch pointers are NULL"); return HICOPS_EINVAL; }
    auto r = std::make_shared<Request>();
    const uint32_t n = b->n;
    r->n = n;
    const uint64_t base = b->peak_off[0];
    r->peak_off.resize(n + 1);
    for (uint32_t i = 0; i <= n; ++i) r->peak_off[i] = b->peak_off[i] - base;
    const uint64_t m = r->peak_off[n];
    if (m && (!b->mz || !b->intensity)) { set_error("peak arrays are NULL"); return HICOPS_EINVAL; }
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
    // launched slots finish: their waiters hand out results, then exit
    for (auto& sl : srv->slots) {
        srv->cv_slot.notify_all();
        if (sl->waiter.joinable()) sl->waiter.join();
    }
    cudaSetDevice(srv->device);
    for (auto& sl : srv->slots) {
        if (sl->stream) cudaStreamSynchronize(sl->stream);
        if (sl->plan) hicops_plan_destroy(sl->plan);
        if (sl->done) cudaEventDestroy(sl->done);
        if (sl->stream) cudaStreamDestroy(sl->stream);
    }
    srv->cv_done.notify_all();
    delete srv;
}
