// Host ingest pipeline of Superstep 3 (Buffering and Task Scheduling
// sections; Supplementary Algorithm 2): MS2 spectrum files are parsed into
// batch buffers by the R sub-task, searched on the GPU by the I sub-task and
// written out by the K sub-task, the buffers circulating through the recycle
// queue q_r and the forward queue q_f.  A pool of worker threads is split
// between R and I by the adaptive rule of the Task Scheduling section: an
// I worker that waited for q_f forecasts its next wait by double exponential
// smoothing and turns to R when the waits pile up (or q_f runs dry with no
// R left); an R worker turns to I when q_f holds many buffers or is full,
// and every R worker turns to I once the input is exhausted.  K is one
// thread.  Results equal one hicops_search of the same spectra: the pipeline
// only changes when and where a batch is searched.
#include <algorithm>
#include <atomic>
#include <cerrno>
#include <charconv>
#include <chrono>
#include <condition_variable>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <deque>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include <cuda_runtime.h>

#include "hicops_internal.h"

using hicops::set_error;

namespace {

// ------------------------------------------------------------------ MS2 text

// One spectrum of an MS2 file: "S <scan> <scan> <precursor m/z>", then
// optional "I"/"D" lines, "Z <charge> <[M+H]+>" lines (the first gives the
// charge; none = charge 0, an invalid spectrum) and "<m/z> <intensity>" peak
// lines.  "H" lines head the file.
struct Ms2Parsed {
    std::vector<uint64_t> off{0};
    std::vector<float> mz, inten;
    std::vector<double> prec;
    std::vector<uint8_t> z;
    std::vector<uint32_t> scan;
};

const char* skip_ws(const char* p, const char* e) {
    while (p < e && (*p == ' ' || *p == '\t' || *p == '\r')) ++p;
    return p;
}

// Parses lines [p, e) (whole lines, starting at an S line or at the file
// start); returns false with a message naming the line on malformed input.
bool parse_ms2(const char* p, const char* e, uint64_t first_line, Ms2Parsed& out, std::string& err) {
    uint64_t line = first_line;
    bool open = false, have_z = false;
    while (p < e) {
        const char* nl = (const char*)memchr(p, '\n', (size_t)(e - p));
        const char* le = nl ? nl : e;
        ++line;
        const char* q = skip_ws(p, le);
        if (q < le) {
            const char c = *q;
            if (c == 'H') {
                if (open) { err = "H line inside a spectrum at line " + std::to_string(line); return false; }
            } else if (c == 'S') {
                if (open) out.off.push_back(out.mz.size());
                std::string s(q + 1, le);
                unsigned long a = 0, b = 0;
                double pm = 0;
                if (sscanf(s.c_str(), "%lu %lu %lf", &a, &b, &pm) != 3) {
                    err = "malformed S line at line " + std::to_string(line);
                    return false;
                }
                out.scan.push_back((uint32_t)a);
                out.prec.push_back(pm);
                out.z.push_back(0);
                open = true;
                have_z = false;
            } else if (c == 'Z') {
                if (!open) { err = "Z line before any S line at line " + std::to_string(line); return false; }
                std::string s(q + 1, le);
                int zc = 0;
                double mh = 0;
                if (sscanf(s.c_str(), "%d %lf", &zc, &mh) != 2 || zc < 0 || zc > 255) {
                    err = "malformed Z line at line " + std::to_string(line);
                    return false;
                }
                if (!have_z) out.z.back() = (uint8_t)zc;
                have_z = true;
            } else if (c == 'I' || c == 'D') {
                // per-spectrum annotations: not used by the search
            } else {
                if (!open) { err = "peak before any S line at line " + std::to_string(line); return false; }
                // two numbers, each correctly rounded to float32
                float m = 0.0f, it = 0.0f;
                const auto r1 = std::from_chars(q, le, m);
                const char* q2 = r1.ec == std::errc() ? skip_ws(r1.ptr, le) : q;
                const auto r2 = std::from_chars(q2, le, it);
                if (r1.ec != std::errc() || q2 == r1.ptr || r2.ec != std::errc() || skip_ws(r2.ptr, le) != le) {
                    err = "malformed peak line at line " + std::to_string(line);
                    return false;
                }
                out.mz.push_back(m);
                out.inten.push_back(it);
            }
        }
        p = nl ? nl + 1 : e;
    }
    if (open) out.off.push_back(out.mz.size());
    return true;
}

bool read_file(const char* path, std::string& buf, std::string& err) {
    FILE* f = fopen(path, "rb");
    if (!f) { err = std::string("cannot open ") + path + ": " + strerror(errno); return false; }
    buf.clear();
    char tmp[1 << 16];
    size_t n;
    while ((n = fread(tmp, 1, sizeof(tmp), f)) > 0) buf.append(tmp, n);
    const bool bad = ferror(f) != 0;
    fclose(f);
    if (bad) { err = std::string("cannot read ") + path; return false; }
    return true;
}

// ------------------------------------------------------------------ buffers

struct Buffer {
    uint32_t file = 0;
    uint64_t first_spectrum = 0;   // index of the first spectrum inside its file
    Ms2Parsed sp;
    std::vector<double> tol;
    std::vector<hicops_psm> psm;
    std::vector<uint32_t> hist, ns;
    bool last = false;             // poison: K stops
};

template <class T>
struct Queue {
    std::mutex mu;
    std::condition_variable cv;
    std::deque<T> q;
    void push(T v) {
        { std::lock_guard<std::mutex> l(mu); q.push_back(std::move(v)); }
        cv.notify_all();
    }
    size_t size() { std::lock_guard<std::mutex> l(mu); return q.size(); }
};

// Cursor over the input: the next chunk of at most `batch` spectra.
struct Source {
    std::mutex mu;
    std::vector<std::string> paths;
    size_t file = 0;               // file being cut
    std::string text;              // its contents
    size_t pos = 0;                // next unread byte
    uint64_t line = 0, spectra = 0;
    bool loaded = false, done = false;
};

}  // namespace

// LaViola's double exponential smoothing: s1 = a x + (1 - a) s1, s2 = a s1 +
// (1 - a) s2 (both start at the first sample); the forecast one step ahead
// is (2 + a / (1 - a)) s1 - (1 + a / (1 - a)) s2.
extern "C" double hicops_des_step(double* state, double x, double alpha, int first) {
    if (first) { state[0] = x; state[1] = x; }
    state[0] = alpha * x + (1.0 - alpha) * state[0];
    state[1] = alpha * state[0] + (1.0 - alpha) * state[1];
    const double r = alpha / (1.0 - alpha);
    return (2.0 + r) * state[0] - (1.0 + r) * state[1];
}

// The Task Scheduling section's two rules (regions of q_f: w1 below 5
// buffers, w2 below 15, w3 from 15).
extern "C" int hicops_sched_i_to_r(double t_wait, double t_cum, double t_fct, double t_min, double t_max,
                                   uint32_t qf_len, uint32_t n_r) {
    return (t_wait >= t_min && t_cum + t_fct > t_max) || (qf_len < 5 && n_r == 0);
}

extern "C" int hicops_sched_r_to_i(uint32_t qf_len, uint32_t qf_cap, uint32_t n_r) {
    return (qf_len >= 15 && n_r > 1) || qf_len >= qf_cap;
}

extern "C" hicops_status hicops_ms2_read(const char* path, uint32_t cap_spectra, uint64_t cap_peaks,
                                         uint32_t* n_spectra, uint64_t* n_peaks, uint64_t* peak_off, float* mz,
                                         float* intensity, double* prec_mz, uint8_t* charge, uint32_t* scan) {
    if (!path || !n_spectra || !n_peaks) { set_error("NULL argument"); return HICOPS_EINVAL; }
    std::string buf, err;
    if (!read_file(path, buf, err)) { set_error("%s", err.c_str()); return HICOPS_EINVAL; }
    Ms2Parsed p;
    if (!parse_ms2(buf.data(), buf.data() + buf.size(), 0, p, err)) {
        set_error("%s: %s", path, err.c_str());
        return HICOPS_EINVAL;
    }
    *n_spectra = (uint32_t)p.prec.size();
    *n_peaks = p.mz.size();
    if (p.prec.size() > cap_spectra || p.mz.size() > cap_peaks) return HICOPS_OK;   // sizes only
    if (peak_off) memcpy(peak_off, p.off.data(), sizeof(uint64_t) * p.off.size());
    if (mz) memcpy(mz, p.mz.data(), sizeof(float) * p.mz.size());
    if (intensity) memcpy(intensity, p.inten.data(), sizeof(float) * p.inten.size());
    if (prec_mz) memcpy(prec_mz, p.prec.data(), sizeof(double) * p.prec.size());
    if (charge) memcpy(charge, p.z.data(), p.z.size());
    if (scan) memcpy(scan, p.scan.data(), sizeof(uint32_t) * p.scan.size());
    return HICOPS_OK;
}

extern "C" hicops_status hicops_pipeline_run(hicops_index* idx, const char* const* paths, uint32_t n_paths,
                                             const char* out_path, const hicops_pipeline_config* cfg_in,
                                             hicops_pipeline_stats* stats) {
    if (!idx || (n_paths && !paths) || !out_path) { set_error("NULL argument"); return HICOPS_EINVAL; }
    if (!idx->dev.ready) { set_error("index has no device part (call hicops_index_upload)"); return HICOPS_EINVAL; }
    hicops_pipeline_config cfg{};
    if (cfg_in) cfg = *cfg_in;
    if (!cfg.batch_spectra) cfg.batch_spectra = 1024;
    if (!cfg.n_buffers) cfg.n_buffers = 20;
    if (!cfg.n_workers) cfg.n_workers = 4;
    if (!(cfg.alpha > 0.0 && cfg.alpha < 1.0)) cfg.alpha = 0.5;
    if (!(cfg.t_min_s > 0.0)) cfg.t_min_s = 1e-3;
    if (!(cfg.t_max_s > 0.0)) cfg.t_max_s = 0.05;
    if (!(cfg.prec_tol_da >= 0.0)) { set_error("prec_tol_da must be >= 0"); return HICOPS_EINVAL; }
    if (cfg.n_buffers < 2 || cfg.n_workers < 2) { set_error("need n_buffers >= 2 and n_workers >= 2"); return HICOPS_EINVAL; }
    for (uint32_t i = 0; i < n_paths; ++i)
        if (!paths[i]) { set_error("paths[%u] is NULL", i); return HICOPS_EINVAL; }
    FILE* out = fopen(out_path, "wb");
    if (!out) { set_error("cannot create %s: %s", out_path, strerror(errno)); return HICOPS_EINVAL; }
    fprintf(out, "file\tscan\tspectrum\trank\tpid\tnb\tny\thyperscore\tevalue\tn_scored\n");

    const uint32_t k = idx->p.top_k;
    Source src;
    for (uint32_t i = 0; i < n_paths; ++i) src.paths.emplace_back(paths[i]);
    src.done = n_paths == 0;
    Queue<Buffer*> q_r, q_f, q_k;   // recycle, forward, result
    std::vector<Buffer> pool(cfg.n_buffers);
    for (auto& b : pool) q_r.push(&b);

    std::atomic<uint32_t> n_r{1}, n_i{cfg.n_workers - 1};   // first iteration: one R worker
    std::atomic<uint32_t> producing{0};     // R workers holding a buffer
    std::atomic<bool> failed{false};
    std::mutex err_mu;
    std::string first_err;
    hicops_status first_st = HICOPS_OK;
    auto fail = [&](hicops_status st, const std::string& msg) {
        std::lock_guard<std::mutex> l(err_mu);
        if (!failed.exchange(true)) { first_st = st; first_err = msg; }
        q_f.cv.notify_all();
        q_r.cv.notify_all();
        q_k.cv.notify_all();
    };
    std::atomic<uint64_t> n_spec{0}, n_batches{0}, moves_ir{0}, moves_ri{0};
    std::atomic<uint64_t> wait_ns{0};
    auto input_done = [&]() { std::lock_guard<std::mutex> l(src.mu); return src.done; };

    // R: cut the next chunk of whole spectra from the input and parse it
    auto produce = [&](Buffer* b) -> bool {   // false: no input left
        const char* beg = nullptr;
        const char* end = nullptr;
        uint64_t line0 = 0;
        std::string text_copy;
        {
            std::lock_guard<std::mutex> l(src.mu);
            for (;;) {
                if (src.done) return false;
                if (!src.loaded) {
                    std::string err;
                    if (!read_file(src.paths[src.file].c_str(), src.text, err)) {
                        src.done = true;
                        fail(HICOPS_EINVAL, err);
                        return false;
                    }
                    src.loaded = true;
                    src.pos = 0;
                    src.line = 0;
                    src.spectra = 0;
                }
                if (src.pos < src.text.size()) break;
                src.loaded = false;
                if (++src.file == src.paths.size()) { src.done = true; return false; }
            }
            // the chunk ends before the (batch + 1)-th S line from here
            const std::string& t = src.text;
            size_t p = src.pos, e = t.size();
            uint32_t seen = 0;
            uint64_t lines = 0;
            while (p < t.size()) {
                const size_t nl = t.find('\n', p);
                const size_t le = nl == std::string::npos ? t.size() : nl;
                size_t q = p;
                while (q < le && (t[q] == ' ' || t[q] == '\t')) ++q;
                if (q < le && t[q] == 'S' && seen++ == cfg.batch_spectra) { e = p; break; }
                ++lines;
                p = nl == std::string::npos ? t.size() : nl + 1;
            }
            text_copy.assign(t, src.pos, e - src.pos);
            line0 = src.line;
            b->file = (uint32_t)src.file;
            b->first_spectrum = src.spectra;
            src.line += lines;
            src.spectra += std::min<uint32_t>(seen, cfg.batch_spectra);
            src.pos = e;
        }
        beg = text_copy.data();
        end = beg + text_copy.size();
        b->sp = Ms2Parsed{};
        std::string err;
        if (!parse_ms2(beg, end, line0, b->sp, err)) {
            fail(HICOPS_EINVAL, src.paths[b->file] + ": " + err);
            return false;
        }
        const size_t n = b->sp.prec.size();
        b->tol.assign(n, cfg.prec_tol_da);
        b->last = false;
        return true;
    };

    auto worker = [&](bool start_as_r) {
        bool is_r = start_as_r;
        cudaStream_t stream = nullptr;
        if (cudaSetDevice(idx->dev.device) != cudaSuccess ||   // the current device is per thread
            cudaStreamCreateWithFlags(&stream, cudaStreamNonBlocking) != cudaSuccess) {
            fail(HICOPS_ECUDA, "cudaStreamCreateWithFlags failed");
            return;
        }
        double des[2] = {0, 0};
        bool des_first = true;
        double t_cum = 0.0;
        while (!failed.load()) {
            if (is_r) {
                Buffer* b = nullptr;
                {
                    std::unique_lock<std::mutex> l(q_r.mu);
                    q_r.cv.wait(l, [&] { return !q_r.q.empty() || failed.load(); });
                    if (failed.load()) break;
                    b = q_r.q.front();
                    q_r.q.pop_front();
                }
                ++producing;
                const bool got = produce(b);
                if (got) q_f.push(b);
                else q_r.push(b);
                --producing;
                q_f.cv.notify_all();
                // c_{R->I}, and every R worker turns to I once the input is exhausted
                const uint32_t len = (uint32_t)q_f.size();
                if (!got || input_done() || hicops_sched_r_to_i(len, cfg.n_buffers, n_r.load())) {
                    --n_r;
                    ++n_i;
                    if (got) ++moves_ri;
                    is_r = false;
                }
                continue;
            }
            // I: the next filled buffer; t_wait is the time q_f.pop() blocked
            Buffer* b = nullptr;
            const auto t0 = std::chrono::steady_clock::now();
            {
                std::unique_lock<std::mutex> l(q_f.mu);
                q_f.cv.wait(l, [&] {
                    return !q_f.q.empty() || failed.load() ||
                           (input_done() && producing.load() == 0) ||
                           (n_r.load() == 0 && !input_done());
                });
                if (!q_f.q.empty()) {
                    b = q_f.q.front();
                    q_f.q.pop_front();
                }
            }
            const double t_wait = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
            wait_ns += (uint64_t)(t_wait * 1e9);
            if (failed.load()) break;
            if (!b) {
                if (input_done() && producing.load() == 0) break;   // nothing left to search
                // q_f ran dry with no R worker: this worker turns to R
                --n_i;
                ++n_r;
                ++moves_ir;
                is_r = true;
                continue;
            }
            const double t_fct = hicops_des_step(des, t_wait, cfg.alpha, des_first);
            des_first = false;
            t_cum += t_wait;
            const uint32_t n = (uint32_t)b->sp.prec.size();
            b->psm.resize((size_t)n * k);
            b->hist.resize((size_t)n * hicops::kHistBins);
            b->ns.resize(n);
            hicops_batch hb{};
            hb.n = n;
            hb.on_device = 0;
            hb.peak_off = b->sp.off.data();
            hb.mz = b->sp.mz.data();
            hb.intensity = b->sp.inten.data();
            hb.prec_mz = b->sp.prec.data();
            hb.charge = b->sp.z.data();
            hb.prec_tol_da = b->tol.data();
            hb.cuda_stream = stream;
            const hicops_status st = n ? hicops_search(idx, &hb, b->psm.data(), b->hist.data(), b->ns.data())
                                       : HICOPS_OK;
            if (st != HICOPS_OK) {
                fail(st, std::string("search: ") + hicops_last_error());
                break;
            }
            n_spec += n;
            ++n_batches;
            q_k.push(b);
            // c_{I->R}
            if (!input_done() &&
                hicops_sched_i_to_r(t_wait, t_cum, t_fct, cfg.t_min_s, cfg.t_max_s, (uint32_t)q_f.size(), n_r.load()) &&
                n_i.load() > 1) {
                --n_i;
                ++n_r;
                ++moves_ir;
                t_cum = 0.0;
                is_r = true;
            }
        }
        cudaStreamDestroy(stream);
        q_f.cv.notify_all();
    };

    // K: rows of every searched buffer, then the buffer back to q_r; numbers
    // in their shortest round-trip decimal form
    std::thread writer([&] {
        std::string text;
        char num[64];
        auto put_u = [&](uint64_t v, char sep) {
            const auto r = std::to_chars(num, num + sizeof(num), v);
            text.append(num, r.ptr);
            text.push_back(sep);
        };
        for (;;) {
            Buffer* b = nullptr;
            {
                std::unique_lock<std::mutex> l(q_k.mu);
                q_k.cv.wait(l, [&] { return !q_k.q.empty() || failed.load(); });
                if (q_k.q.empty()) break;
                b = q_k.q.front();
                q_k.q.pop_front();
            }
            if (b->last) break;
            const uint32_t n = (uint32_t)b->sp.prec.size();
            text.clear();
            for (uint32_t s = 0; s < n; ++s) {
                for (uint32_t r = 0; r < k; ++r) {
                    const hicops_psm& o = b->psm[(size_t)s * k + r];
                    if (o.pid == 0xffffffffu) break;
                    put_u(b->file, '\t');
                    put_u(b->sp.scan[s], '\t');
                    put_u(b->first_spectrum + s, '\t');
                    put_u(r, '\t');
                    put_u(o.pid, '\t');
                    put_u(o.nb, '\t');
                    put_u(o.ny, '\t');
                    auto rh = std::to_chars(num, num + sizeof(num), o.hyperscore);
                    text.append(num, rh.ptr);
                    text.push_back('\t');
                    auto re = std::to_chars(num, num + sizeof(num), o.evalue);
                    text.append(num, re.ptr);
                    text.push_back('\t');
                    put_u(b->ns[s], '\n');
                }
            }
            if (!text.empty() && fwrite(text.data(), 1, text.size(), out) != text.size())
                fail(HICOPS_EINVAL, std::string("cannot write ") + out_path);
            q_r.push(b);
        }
    });

    const auto t_start = std::chrono::steady_clock::now();
    std::vector<std::thread> workers;
    for (uint32_t w = 0; w < cfg.n_workers; ++w) workers.emplace_back(worker, w == 0);
    for (auto& t : workers) t.join();
    Buffer poison;
    poison.last = true;
    q_k.push(&poison);
    writer.join();
    const double secs = std::chrono::duration<double>(std::chrono::steady_clock::now() - t_start).count();
    if (fclose(out) != 0 && !failed.load()) fail(HICOPS_EINVAL, std::string("cannot write ") + out_path);
    if (stats) {
        stats->spectra = n_spec.load();
        stats->batches = n_batches.load();
        stats->seconds = secs;
        stats->moves_i_to_r = moves_ir.load();
        stats->moves_r_to_i = moves_ri.load();
        stats->wait_seconds = (double)wait_ns.load() * 1e-9;
    }
    if (failed.load()) { set_error("%s", first_err.c_str()); return first_st; }
    return HICOPS_OK;
}
