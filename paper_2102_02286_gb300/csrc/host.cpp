// Host side of superstep 1 (paper: "Superstep 1: Partial Database
// Construction", Supplementary Algorithm 1): in-silico tryptic digestion,
// modification variants (the 2^m variants of the Notation section) and the
// sort that fixes peptide ids.  Multithreaded C++; the device fragment index
// is built from this table by index_build.cu.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <cstdarg>
#include <cerrno>
#include <cstdio>
#include <cstring>
#include <memory>
#include <functional>
#include <numeric>
#include <thread>

#include "hicops_internal.h"

namespace hicops {

static thread_local char g_err[512] = "";

void set_error(const char* fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
}

static double residue_da(char c) {
    // monoisotopic residue masses
    switch (c) {
        case 'A': return 71.037114;  case 'R': return 156.101111; case 'N': return 114.042927;
        case 'D': return 115.026943; case 'C': return 103.009185; case 'E': return 129.042593;
        case 'Q': return 128.058578; case 'G': return 57.021464;  case 'H': return 137.058912;
        case 'I': return 113.084064; case 'L': return 113.084064; case 'K': return 128.094963;
        case 'M': return 131.040485; case 'F': return 147.068414; case 'P': return 97.052764;
        case 'S': return 87.032028;  case 'T': return 101.047679; case 'W': return 186.079313;
        case 'Y': return 163.063329; case 'V': return 99.068414;
        default: return 0.0;
    }
}

hicops_status validate_params(const hicops_params* p) {
    if (!p) { set_error("params is NULL"); return HICOPS_EINVAL; }
    if (p->min_len < 2 || p->max_len < p->min_len || p->max_len > kMaxLen) {
        set_error("peptide length limits must satisfy 2 <= min_len <= max_len <= %u", kMaxLen);
        return HICOPS_EINVAL;
    }
    if (!(p->bin_width_da > 0) || !(p->frag_mz_min > 0) || !(p->frag_mz_max > p->frag_mz_min) ||
        !(p->frag_mz_max / p->bin_width_da < 2147483647.0)) {
        set_error("fragment range / bin width invalid");
        return HICOPS_EINVAL;
    }
    if (p->top_k < 1 || p->top_k > kMaxTopK) { set_error("top_k must be in [1, %u]", kMaxTopK); return HICOPS_EINVAL; }
    if (p->top_n_peaks < 1 || p->top_n_peaks > kMaxTopN) {
        set_error("top_n_peaks must be in [1, %u]", kMaxTopN);
        return HICOPS_EINVAL;
    }
    if (p->tol_bins >= kMaxTopN || (uint64_t)(2 * p->tol_bins + 1) * p->top_n_peaks > kMaxTopN) {
        set_error("(2 * tol_bins + 1) * top_n_peaks must be <= %u", kMaxTopN);
        return HICOPS_EINVAL;
    }
    if (p->hist_bins != kHistBins) { set_error("hist_bins must be %u", kHistBins); return HICOPS_EINVAL; }
    if (p->evalue_mode & ~(HICOPS_EVALUE_LOG_WEIBULL | HICOPS_EVALUE_SMOOTH)) {
        set_error("unknown evalue_mode bits");
        return HICOPS_EINVAL;
    }
    if (p->intensity_scale < 1) { set_error("intensity_scale must be >= 1"); return HICOPS_EINVAL; }
    if (p->min_shared < 1) { set_error("min_shared must be >= 1"); return HICOPS_EINVAL; }
    // a peptide shares at most one ion per query bin
    const uint64_t max_matched = std::min<uint64_t>(query_bins_cap(*p), 2ull * (p->max_len - 1));
    if (max_matched * p->intensity_scale > kSMask) {
        set_error("min((2*tol_bins+1)*top_n_peaks, 2*(max_len-1)) * intensity_scale must be < 2^20");
        return HICOPS_EOVERFLOW;
    }
    if (!(p->min_mass <= p->max_mass)) { set_error("min_mass > max_mass"); return HICOPS_EINVAL; }
    return HICOPS_OK;
}

namespace {

unsigned n_threads() {
    unsigned t = std::thread::hardware_concurrency();
    return t ? std::min(t, 64u) : 4u;
}

template <class F>
void parallel_for(size_t n, F&& f) {
    const unsigned T = n_threads();
    std::atomic<size_t> next{0};
    const size_t grain = std::max<size_t>(1, n / (T * 16));
    std::vector<std::thread> th;
    for (unsigned t = 0; t < T; ++t)
        th.emplace_back([&, t] {
            for (;;) {
                size_t a = next.fetch_add(grain);
                if (a >= n) break;
                size_t b = std::min(n, a + grain);
                for (size_t i = a; i < b; ++i) f(i, t);
            }
        });
    for (auto& x : th) x.join();
}

// parallel merge sort: sort T runs in parallel, then merge pairwise
template <class T, class Less>
void parallel_sort(std::vector<T>& v, Less less) {
    const size_t n = v.size();
    unsigned T_ = n_threads();
    if (n < 100000 || T_ == 1) { std::sort(v.begin(), v.end(), less); return; }
    unsigned runs = 1;
    while (runs < T_) runs <<= 1;
    std::vector<size_t> cut(runs + 1);
    for (unsigned r = 0; r <= runs; ++r) cut[r] = n * r / runs;
    {
        std::vector<std::thread> th;
        for (unsigned r = 0; r < runs; ++r)
            th.emplace_back([&, r] { std::sort(v.begin() + cut[r], v.begin() + cut[r + 1], less); });
        for (auto& x : th) x.join();
    }
    std::vector<T> tmp(n);
    std::vector<T>* src = &v;
    std::vector<T>* dst = &tmp;
    for (unsigned width = 1; width < runs; width <<= 1) {
        std::vector<std::thread> th;
        for (unsigned r = 0; r < runs; r += 2 * width) {
            size_t a = cut[r], m = cut[std::min(runs, r + width)], e = cut[std::min(runs, r + 2 * width)];
            th.emplace_back([=, &less] {
                std::merge(src->begin() + a, src->begin() + m, src->begin() + m, src->begin() + e,
                           dst->begin() + a, less);
            });
        }
        for (auto& x : th) x.join();
        std::swap(src, dst);
    }
    if (src != &v) v.swap(*src);
}

struct BaseRef {
    uint64_t pos;   // offset into the protein sequence buffer
    uint32_t len;
};

struct Entry {
    double mass;
    uint32_t base;
    uint64_t mask_rev;   // bit-reversed mask: position 0 is the most significant bit
};

inline uint64_t bitrev64(uint64_t x) {
    x = ((x >> 1) & 0x5555555555555555ull) | ((x & 0x5555555555555555ull) << 1);
    x = ((x >> 2) & 0x3333333333333333ull) | ((x & 0x3333333333333333ull) << 2);
    x = ((x >> 4) & 0x0F0F0F0F0F0F0F0Full) | ((x & 0x0F0F0F0F0F0F0F0Full) << 4);
    x = ((x >> 8) & 0x00FF00FF00FF00FFull) | ((x & 0x00FF00FF00FF00FFull) << 8);
    x = ((x >> 16) & 0x0000FFFF0000FFFFull) | ((x & 0x0000FFFF0000FFFFull) << 16);
    return (x >> 32) | (x << 32);
}

}  // namespace
}  // namespace hicops

using namespace hicops;

extern "C" const char* hicops_last_error(void) { return hicops::g_err; }

extern "C" hicops_status hicops_digest(const hicops_proteins* prot, const hicops_mod* mods, uint32_t n_mods,
                                       const hicops_params* params, hicops_index** out) {
    if (!out) { set_error("out is NULL"); return HICOPS_EINVAL; }
    *out = nullptr;
    if (!prot || (prot->n_proteins && (!prot->seq || !prot->off))) { set_error("proteins invalid"); return HICOPS_EINVAL; }
    if (n_mods && !mods) { set_error("mods is NULL"); return HICOPS_EINVAL; }
    hicops_status st = validate_params(params);
    if (st != HICOPS_OK) return st;
    auto t0 = std::chrono::steady_clock::now();

    hicops_index* idx = new (std::nothrow) hicops_index();
    if (!idx) { set_error("out of host memory"); return HICOPS_ENOMEM; }
    idx->p = *params;
    double fixed[128] = {0};
    bool has_fixed[128] = {false};
    for (int c = 0; c < 128; ++c) idx->var_type[c] = -1;
    for (uint32_t i = 0; i < n_mods; ++i) {
        const hicops_mod& m = mods[i];
        if (!m.residues || !std::isfinite(m.delta_da)) { delete idx; set_error("mod %u invalid", i); return HICOPS_EINVAL; }
        if (m.fixed) {
            for (const char* r = m.residues; *r; ++r) {
                unsigned char c = (unsigned char)*r;
                if (c >= 128 || has_fixed[c]) { delete idx; set_error("two fixed mods on '%c'", *r); return HICOPS_EINVAL; }
                has_fixed[c] = true;
                fixed[c] = m.delta_da;
            }
        } else {
            const int t = (int)idx->n_var++;
            idx->var_delta.push_back(m.delta_da);
            idx->var_max.push_back(m.max_per_peptide);
            for (const char* r = m.residues; *r; ++r) {
                unsigned char c = (unsigned char)*r;
                if (c >= 128 || idx->var_type[c] >= 0) {
                    delete idx;
                    set_error("residue '%c' carries two variable mods (unsupported)", *r);
                    return HICOPS_EINVAL;
                }
                idx->var_type[c] = (int8_t)t;
            }
        }
    }
    if (idx->n_var > 127) { delete idx; set_error("too many variable mods"); return HICOPS_EINVAL; }
    // m = residue (+ fixed) (+ variable), two FP64 adds in that order
    for (int c = 0; c < 128; ++c) {
        double m = residue_da((char)c);
        if (has_fixed[c]) m = m + fixed[c];
        idx->mres[c] = m;
        idx->mmod[c] = idx->var_type[c] >= 0 ? m + idx->var_delta[idx->var_type[c]] : m;
    }

    const hicops_params& p = idx->p;
    const char* seq = prot->seq;
    // 1. tryptic base peptides per protein
    const size_t NP = prot->n_proteins;
    const unsigned T = n_threads();
    std::vector<std::vector<BaseRef>> per_thread(T);
    parallel_for(NP, [&](size_t i, unsigned t) {
        const uint64_t a = prot->off[i], e = prot->off[i + 1];
        if (e <= a) return;
        // boundaries: protein start, after K/R not followed by P, protein end
        uint64_t bounds_buf[4096];
        std::vector<uint64_t> big;
        uint64_t* bnd = bounds_buf;
        size_t nb = 0;
        const uint64_t len = e - a;
        if (len + 2 > 4096) { big.resize(len + 2); bnd = big.data(); }
        bnd[nb++] = a;
        for (uint64_t k = a; k + 1 < e; ++k)
            if ((seq[k] == 'K' || seq[k] == 'R') && seq[k + 1] != 'P') bnd[nb++] = k + 1;
        bnd[nb++] = e;
        for (size_t x = 0; x + 1 < nb; ++x) {
            for (size_t y = x + 1; y < nb && y - x - 1 <= p.missed_cleavages; ++y) {
                const uint64_t L = bnd[y] - bnd[x];
                if (L < p.min_len) continue;
                if (L > p.max_len) break;
                bool ok = true;
                for (uint64_t k = bnd[x]; k < bnd[y]; ++k)
                    if (residue_da(seq[k]) == 0.0) { ok = false; break; }
                if (ok) per_thread[t].push_back(BaseRef{bnd[x], (uint32_t)L});
            }
        }
    });
    std::vector<BaseRef> bases;
    for (auto& v : per_thread) { bases.insert(bases.end(), v.begin(), v.end()); std::vector<BaseRef>().swap(v); }
    // 2. deduplicate base sequences; base id = rank in byte order
    auto seq_less = [seq](const BaseRef& x, const BaseRef& y) {
        int c = memcmp(seq + x.pos, seq + y.pos, std::min(x.len, y.len));
        return c != 0 ? c < 0 : x.len < y.len;
    };
    parallel_sort(bases, seq_less);
    {
        size_t w = 0;
        for (size_t i = 0; i < bases.size(); ++i) {
            if (w > 0 && bases[w - 1].len == bases[i].len &&
                memcmp(seq + bases[w - 1].pos, seq + bases[i].pos, bases[i].len) == 0)
                continue;
            bases[w++] = bases[i];
        }
        bases.resize(w);
    }
    const size_t NB = bases.size();
    idx->base_off.resize(NB + 1);
    idx->base_off[0] = 0;
    for (size_t i = 0; i < NB; ++i) idx->base_off[i + 1] = idx->base_off[i] + bases[i].len;
    idx->residues.resize(idx->base_off[NB]);
    parallel_for(NB, [&](size_t i, unsigned) {
        memcpy(&idx->residues[idx->base_off[i]], seq + bases[i].pos, bases[i].len);
    });

    // 3. variants: every subset of modifiable positions within the per-rule
    //    caps (and the global cap), masses summed left to right
    std::vector<std::vector<Entry>> ent(T);
    parallel_for(NB, [&](size_t bi, unsigned t) {
        const char* s = &idx->residues[idx->base_off[bi]];
        const uint32_t L = (uint32_t)(idx->base_off[bi + 1] - idx->base_off[bi]);
        // sites in position order, with their rule
        uint32_t site_pos[kMaxLen];
        int site_rule[kMaxLen];
        uint32_t ns = 0;
        for (uint32_t j = 0; j < L; ++j) {
            int r = idx->var_type[(unsigned char)s[j]];
            if (r >= 0) { site_pos[ns] = j; site_rule[ns] = r; ++ns; }
        }
        // depth-first over sites: choose modified / unmodified
        uint32_t used[128] = {0};
        std::function<void(uint32_t, uint64_t, uint32_t)> rec = [&](uint32_t i, uint64_t mask, uint32_t total) {
            if (i == ns) {
                double sum = 0.0;
                for (uint32_t j = 0; j < L; ++j)
                    sum = sum + (((mask >> j) & 1ull) ? idx->mmod[(unsigned char)s[j]] : idx->mres[(unsigned char)s[j]]);
                const double M = sum + kWaterDa;
                if (M >= p.min_mass && M <= p.max_mass) ent[t].push_back(Entry{M, (uint32_t)bi, bitrev64(mask)});
                return;
            }
            rec(i + 1, mask, total);
            const int r = site_rule[i];
            if (used[r] < idx->var_max[r] && (p.max_total_mods == 0 || total < p.max_total_mods)) {
                used[r]++;
                rec(i + 1, mask | (1ull << site_pos[i]), total + 1);
                used[r]--;
            }
        };
        rec(0, 0, 0);
    });
    size_t total = 0;
    for (auto& v : ent) total += v.size();
    if (total >= (1ull << 31)) {
        delete idx;
        set_error("database has %zu entries; pid must fit in 31 bits", total);
        return HICOPS_EOVERFLOW;
    }
    std::vector<Entry> all;
    all.reserve(total);
    for (auto& v : ent) { all.insert(all.end(), v.begin(), v.end()); std::vector<Entry>().swap(v); }
    // 4. pid order: (mass, sequence bytes, modification state)
    parallel_sort(all, [](const Entry& a, const Entry& b) {
        if (a.mass != b.mass) return a.mass < b.mass;
        if (a.base != b.base) return a.base < b.base;
        return a.mask_rev < b.mask_rev;
    });
    idx->mass.resize(total);
    idx->base.resize(total);
    idx->mask.resize(total);
    parallel_for(total, [&](size_t i, unsigned) {
        idx->mass[i] = all[i].mass;
        idx->base[i] = all[i].base;
        idx->mask[i] = bitrev64(all[i].mask_rev);
    });

    idx->n_bins = (uint32_t)std::floor(p.frag_mz_max / p.bin_width_da) + 1;
    idx->s_max = std::min<uint64_t>(query_bins_cap(p), 2ull * (p.max_len - 1)) * p.intensity_scale;
    idx->stats.n_peptides = total;
    idx->stats.n_base_peptides = NB;
    idx->stats.n_bins = idx->n_bins;
    idx->stats.host_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    *out = idx;
    return HICOPS_OK;
}

extern "C" hicops_status hicops_build_index(const hicops_proteins* prot, const hicops_mod* mods, uint32_t n_mods,
                                            const hicops_params* params, hicops_index** out) {
    hicops_status st = hicops_digest(prot, mods, n_mods, params, out);
    if (st != HICOPS_OK) return st;
    st = hicops_index_upload(*out);
    if (st != HICOPS_OK) { hicops_index_free(*out); *out = nullptr; }
    return st;
}

extern "C" hicops_status hicops_index_get_params(const hicops_index* idx, hicops_params* out) {
    if (!idx || !out) { set_error("NULL argument"); return HICOPS_EINVAL; }
    *out = idx->p;
    return HICOPS_OK;
}

extern "C" hicops_status hicops_index_get_stats(const hicops_index* idx, hicops_index_stats* out) {
    if (!idx || !out) { set_error("NULL argument"); return HICOPS_EINVAL; }
    *out = idx->stats;
    return HICOPS_OK;
}

namespace {

bool is_part(const hicops_index* idx) { return idx->pid_stride != 1 || !idx->pid_map.empty(); }

// The part of a whole database holding global pids g(0) < g(1) < ... < g(n-1),
// as a host-only index (hicops_index_upload builds its device part).
template <class Global>
hicops_index* make_part(const hicops_index* full, size_t n, Global g) {
    hicops_index* idx = new (std::nothrow) hicops_index();
    if (!idx) return nullptr;
    idx->p = full->p;
    memcpy(idx->mres, full->mres, sizeof(idx->mres));
    memcpy(idx->mmod, full->mmod, sizeof(idx->mmod));
    memcpy(idx->var_type, full->var_type, sizeof(idx->var_type));
    idx->n_var = full->n_var;
    idx->var_delta = full->var_delta;
    idx->var_max = full->var_max;
    idx->residues = full->residues;
    idx->base_off = full->base_off;
    idx->mass.resize(n);
    idx->base.resize(n);
    idx->mask.resize(n);
    for (size_t i = 0; i < n; ++i) {
        const size_t k = g(i);
        idx->mass[i] = full->mass[k];
        idx->base[i] = full->base[k];
        idx->mask[i] = full->mask[k];
    }
    idx->n_bins = full->n_bins;
    idx->s_max = full->s_max;
    idx->stats = hicops_index_stats{};
    idx->stats.n_peptides = n;
    idx->stats.n_base_peptides = full->stats.n_base_peptides;
    idx->stats.n_bins = full->n_bins;
    return idx;
}

}  // namespace

extern "C" hicops_status hicops_index_shard(const hicops_index* full, uint32_t n_shards, uint32_t shard,
                                            hicops_index** out) {
    if (!full || !out) { set_error("NULL argument"); return HICOPS_EINVAL; }
    *out = nullptr;
    if (is_part(full)) { set_error("the index is already a shard"); return HICOPS_EINVAL; }
    if (n_shards < 1 || n_shards > HICOPS_MAX_SHARDS || shard >= n_shards) {
        set_error("shard %u of %u: need 1 <= n_shards <= %u and shard < n_shards", shard, n_shards,
                  (unsigned)HICOPS_MAX_SHARDS);
        return HICOPS_EINVAL;
    }
    const size_t P = full->mass.size();
    const size_t n = P > shard ? (P - shard + n_shards - 1) / n_shards : 0;
    // round-robin over the mass-sorted order
    hicops_index* idx = make_part(full, n, [&](size_t i) { return i * n_shards + shard; });
    if (!idx) { set_error("out of host memory"); return HICOPS_ENOMEM; }
    idx->pid_stride = n_shards;
    idx->pid_base = shard;
    *out = idx;
    return HICOPS_OK;
}

extern "C" hicops_status hicops_index_subset(const hicops_index* full, const uint32_t* pids, uint64_t n,
                                             hicops_index** out) {
    if (!full || !out || (n && !pids)) { set_error("NULL argument"); return HICOPS_EINVAL; }
    *out = nullptr;
    if (is_part(full)) { set_error("the index is already a shard"); return HICOPS_EINVAL; }
    const size_t P = full->mass.size();
    for (uint64_t i = 0; i < n; ++i) {
        if (pids[i] >= P || (i > 0 && pids[i] <= pids[i - 1])) {
            set_error("pids must be strictly ascending and below %zu (pids[%llu] = %u)", P,
                      (unsigned long long)i, pids[i]);
            return HICOPS_EINVAL;
        }
    }
    hicops_index* idx = make_part(full, n, [&](size_t i) { return (size_t)pids[i]; });
    if (!idx) { set_error("out of host memory"); return HICOPS_ENOMEM; }
    idx->pid_map.assign(pids, pids + n);
    *out = idx;
    return HICOPS_OK;
}

// R18, the improved LBE of Superstep 1 (Supplementary Text 3, Supplementary
// Fig. 3).  Variants of one base peptide differ from it only by modified
// residues, each a symbol of its own, so their edit distance to it is the
// number of modified positions, and the letters equal from the termini are
// the unmodified runs at both ends (the whole peptide, twice, when none is
// modified); inside a base, a larger run means a smaller Mod Distance.
extern "C" hicops_status hicops_partition_lbe(const hicops_index* full, uint32_t n_parts, uint32_t* part) {
    if (!full || !part) { set_error("NULL argument"); return HICOPS_EINVAL; }
    if (is_part(full)) { set_error("the index is already a shard"); return HICOPS_EINVAL; }
    if (n_parts < 1 || n_parts > HICOPS_MAX_SHARDS) {
        set_error("n_parts must be in [1, %u]", (unsigned)HICOPS_MAX_SHARDS);
        return HICOPS_EINVAL;
    }
    const size_t P = full->mass.size();
    const size_t NB = full->base_off.size() - 1;
    std::vector<uint32_t> first(NB, UINT32_MAX);   // each cluster's smallest pid
    for (size_t pid = P; pid-- > 0;) first[full->base[pid]] = (uint32_t)pid;
    struct Key {
        uint32_t cluster, edits, ends_rev, pid;   // ends_rev = 2 L - a: ascending = Mod Distance ascending
    };
    std::vector<Key> keys(P);
    parallel_for(P, [&](size_t pid, unsigned) {
        const uint32_t b = full->base[pid];
        const uint32_t L = (uint32_t)(full->base_off[b + 1] - full->base_off[b]);
        const uint64_t m = full->mask[pid];
        uint32_t a = 2 * L;
        if (m) a = (uint32_t)__builtin_ctzll(m) + (L - 1 - (63 - (uint32_t)__builtin_clzll(m)));
        keys[pid] = Key{first[b], (uint32_t)__builtin_popcountll(m), 2 * L - a, (uint32_t)pid};
    });
    parallel_sort(keys, [](const Key& x, const Key& y) {
        if (x.cluster != y.cluster) return x.cluster < y.cluster;
        if (x.edits != y.edits) return x.edits < y.edits;
        if (x.ends_rev != y.ends_rev) return x.ends_rev < y.ends_rev;
        return x.pid < y.pid;
    });
    for (size_t i = 0; i < P; ++i) part[keys[i].pid] = (uint32_t)(i % n_parts);
    return HICOPS_OK;
}

extern "C" hicops_status hicops_peptide(const hicops_index* idx, uint32_t pid, char* seq, uint32_t cap,
                                        double* mass, uint64_t* modmask) {
    if (!idx) { set_error("index is NULL"); return HICOPS_EINVAL; }
    if (!idx->pid_map.empty()) {
        auto it = std::lower_bound(idx->pid_map.begin(), idx->pid_map.end(), pid);
        if (it == idx->pid_map.end() || *it != pid) {
            set_error("pid %u is not in this shard", pid);
            return HICOPS_EINVAL;
        }
        pid = (uint32_t)(it - idx->pid_map.begin());
    } else {
        if (pid < idx->pid_base || (pid - idx->pid_base) % idx->pid_stride != 0) {
            set_error("pid %u is not in this shard", pid);
            return HICOPS_EINVAL;
        }
        pid = (pid - idx->pid_base) / idx->pid_stride;
    }
    if (pid >= idx->mass.size()) { set_error("pid out of range"); return HICOPS_EINVAL; }
    const uint32_t b = idx->base[pid];
    const uint64_t a = idx->base_off[b], e = idx->base_off[b + 1];
    if (seq && cap) {
        const uint64_t n = std::min<uint64_t>(e - a, cap - 1);
        memcpy(seq, &idx->residues[a], n);
        seq[n] = 0;
    }
    if (mass) *mass = idx->mass[pid];
    if (modmask) *modmask = idx->mask[pid];
    return HICOPS_OK;
}

extern "C" void hicops_index_free(hicops_index* idx) {
    if (!idx) return;
    hicops::free_device_index(idx);
    delete idx;
}

// ---- checkpoint: the host half of an index in one file (the paper writes
// its preprocessed data back for reuse, Superstep 2); the device half is
// rebuilt from it by hicops_index_upload.  Little-endian, fixed-width fields.

namespace {

constexpr char kIndexMagic[8] = {'H', 'I', 'C', 'O', 'P', 'S', 'I', 'X'};
constexpr uint32_t kIndexFormat = 1;

struct FileOut {
    FILE* f;
    bool ok = true;
    void raw(const void* p, size_t n) {
        if (ok && n && fwrite(p, 1, n, f) != n) ok = false;
    }
    template <class T>
    void pod(const T& v) { raw(&v, sizeof(T)); }
    template <class T>
    void vec(const std::vector<T>& v) {
        pod<uint64_t>(v.size());
        raw(v.data(), v.size() * sizeof(T));
    }
};

struct FileIn {
    FILE* f;
    uint64_t left;   // bytes not yet read
    bool ok = true;
    void raw(void* p, size_t n) {
        if (!ok || n > left || (n && fread(p, 1, n, f) != n)) { ok = false; return; }
        left -= n;
    }
    template <class T>
    void pod(T& v) { raw(&v, sizeof(T)); }
    template <class T>
    void vec(std::vector<T>& v) {
        uint64_t n = 0;
        pod(n);
        if (!ok || n > left / sizeof(T)) { ok = false; return; }   // never allocate past the file
        v.resize(n);
        raw(v.data(), n * sizeof(T));
    }
};

}  // namespace

extern "C" hicops_status hicops_index_save(const hicops_index* idx, const char* path) {
    if (!idx || !path) { set_error("NULL argument"); return HICOPS_EINVAL; }
    FILE* f = fopen(path, "wb");
    if (!f) { set_error("cannot create %s: %s", path, strerror(errno)); return HICOPS_EINVAL; }
    FileOut o{f};
    o.raw(kIndexMagic, sizeof(kIndexMagic));
    o.pod(kIndexFormat);
    o.pod<uint32_t>(sizeof(hicops_params));
    o.pod(idx->p);
    o.raw(idx->mres, sizeof(idx->mres));
    o.raw(idx->mmod, sizeof(idx->mmod));
    o.raw(idx->var_type, sizeof(idx->var_type));
    o.pod(idx->n_var);
    o.vec(idx->var_delta);
    o.vec(idx->var_max);
    o.pod<uint64_t>(idx->residues.size());
    o.raw(idx->residues.data(), idx->residues.size());
    o.vec(idx->base_off);
    o.vec(idx->mass);
    o.vec(idx->base);
    o.vec(idx->mask);
    o.pod(idx->pid_stride);
    o.pod(idx->pid_base);
    o.vec(idx->pid_map);
    o.pod(idx->n_bins);
    o.pod(idx->s_max);
    o.pod(idx->stats);
    const bool closed = fclose(f) == 0;
    if (!o.ok || !closed) { set_error("cannot write %s", path); return HICOPS_EINVAL; }
    return HICOPS_OK;
}

extern "C" hicops_status hicops_index_load(const char* path, hicops_index** out) {
    if (!path || !out) { set_error("NULL argument"); return HICOPS_EINVAL; }
    *out = nullptr;
    FILE* f = fopen(path, "rb");
    if (!f) { set_error("cannot open %s: %s", path, strerror(errno)); return HICOPS_EINVAL; }
    uint64_t size = 0;
    if (fseek(f, 0, SEEK_END) == 0) {
        const long e = ftell(f);
        size = e > 0 ? (uint64_t)e : 0;
    }
    rewind(f);
    std::unique_ptr<hicops_index> idx(new (std::nothrow) hicops_index());
    if (!idx) { fclose(f); set_error("out of host memory"); return HICOPS_ENOMEM; }
    FileIn in{f, size};
    char magic[8] = {};
    uint32_t format = 0, psize = 0;
    in.raw(magic, sizeof(magic));
    in.pod(format);
    in.pod(psize);
    const bool header = in.ok && memcmp(magic, kIndexMagic, sizeof(magic)) == 0 && format == kIndexFormat &&
                        psize == sizeof(hicops_params);
    if (header) {
        in.pod(idx->p);
        in.raw(idx->mres, sizeof(idx->mres));
        in.raw(idx->mmod, sizeof(idx->mmod));
        in.raw(idx->var_type, sizeof(idx->var_type));
        in.pod(idx->n_var);
        in.vec(idx->var_delta);
        in.vec(idx->var_max);
        uint64_t nres = 0;
        in.pod(nres);
        if (in.ok && nres <= in.left) {
            idx->residues.resize(nres);
            in.raw(&idx->residues[0], nres);
        } else {
            in.ok = false;
        }
        in.vec(idx->base_off);
        in.vec(idx->mass);
        in.vec(idx->base);
        in.vec(idx->mask);
        in.pod(idx->pid_stride);
        in.pod(idx->pid_base);
        in.vec(idx->pid_map);
        in.pod(idx->n_bins);
        in.pod(idx->s_max);
        in.pod(idx->stats);
    }
    fclose(f);
    if (!header || !in.ok || in.left != 0) {
        set_error("%s is not a complete index file of this format", path);
        return HICOPS_EINVAL;
    }
    // consistency of what was read: sizes, ranges and orders
    hicops_index& x = *idx;
    const size_t P = x.mass.size();
    bool good = x.n_var == x.var_delta.size() && x.n_var == x.var_max.size() && !x.base_off.empty() &&
                x.base_off.front() == 0 && x.base_off.back() == x.residues.size() && x.base.size() == P &&
                x.mask.size() == P && x.pid_stride >= 1 && (x.pid_map.empty() || x.pid_map.size() == P) &&
                P < (1ull << 31);
    for (size_t i = 1; good && i < x.base_off.size(); ++i) good = x.base_off[i] >= x.base_off[i - 1];
    for (size_t i = 0; good && i < 128; ++i) good = x.var_type[i] < (int)x.n_var;
    for (size_t i = 0; good && i < P; ++i) {
        good = x.base[i] + 1 < x.base_off.size() &&
               x.base_off[x.base[i] + 1] - x.base_off[x.base[i]] <= kMaxLen && (i == 0 || x.mass[i] >= x.mass[i - 1]);
    }
    for (size_t i = 1; good && i < x.pid_map.size(); ++i) good = x.pid_map[i] > x.pid_map[i - 1];
    // every residue byte indexes the 128-entry mass tables on the device and
    // must be a letter with a mass (digestion keeps no other)
    for (size_t i = 0; good && i < x.residues.size(); ++i) {
        const unsigned char c = (unsigned char)x.residues[i];
        good = c < 128 && x.mres[c] > 0.0 && std::isfinite(x.mres[c]) && std::isfinite(x.mmod[c]);
    }
    if (!good) { set_error("%s: inconsistent index contents", path); return HICOPS_EINVAL; }
    hicops_status st = validate_params(&x.p);
    if (st != HICOPS_OK) return st;
    // the bin count and the largest S follow from the parameters, as in
    // hicops_digest; a file that disagrees would size the device tables wrongly
    const uint32_t n_bins = (uint32_t)std::floor(x.p.frag_mz_max / x.p.bin_width_da) + 1;
    const uint64_t s_max = std::min<uint64_t>(query_bins_cap(x.p), 2ull * (x.p.max_len - 1)) * x.p.intensity_scale;
    if (x.n_bins != n_bins || x.s_max != s_max) {
        set_error("%s: stored bin count %u / largest S %llu disagree with the parameters (%u / %llu)", path,
                  x.n_bins, (unsigned long long)x.s_max, n_bins, (unsigned long long)s_max);
        return HICOPS_EINVAL;
    }
    x.dev = hicops::DeviceIndex{};
    *out = idx.release();
    return HICOPS_OK;
}
