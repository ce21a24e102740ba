// Host-side memory and undefined-behaviour check (test infrastructure): the
// library's host half (digestion, LBE partition, shards and subsets, peptide
// lookup, MS2 parsing, the scheduling forecast and rules) and the oracle
// (database, partition, search, e-values, edit and Mod Distance), built with
// AddressSanitizer and UndefinedBehaviorSanitizer and driven through their
// C entry points.  Results are checked too: the library's and the oracle's
// LBE partitions agree, every part resolves its global pids, a checkpoint
// round-trips and every truncated checkpoint is rejected.  The device
// half is replaced by stubs: nothing here touches a GPU.
#include <cassert>
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <vector>

#include "hicops.h"

#define CHECK(c)                                                              \
    do {                                                                      \
        if (!(c)) {                                                           \
            fprintf(stderr, "check failed at line %d: %s\n", __LINE__, #c);   \
            exit(2);                                                          \
        }                                                                     \
    } while (0)

// ---- stubs for the device half of the library
struct hicops_index;
namespace hicops {
void free_device_index(hicops_index*) {}
}
extern "C" hicops_status hicops_index_upload(hicops_index*) { return HICOPS_ECUDA; }
extern "C" hicops_status hicops_search(hicops_index*, const hicops_batch*, hicops_psm*, uint32_t*, uint32_t*) {
    return HICOPS_ECUDA;
}

// ---- the oracle's C entry points (its own layout, declared here)
extern "C" {
struct OrMod {
    const char* residues;
    double delta;
    uint32_t max_per_peptide;
    uint32_t fixed;
};
struct OrParams {
    uint32_t min_len, max_len, missed_cleavages, pad0;
    double min_mass, max_mass;
    double frag_mz_min, frag_mz_max, bin_width;
    uint32_t top_n_peaks, min_shared, top_k, hist_bins;
    uint32_t intensity_scale, max_total_mods;
    uint32_t tol_bins, evalue_mode;
};
struct OrPsm {
    uint32_t pid;
    uint32_t nb, ny, S;
    int64_t key;
    double hyperscore;
    double evalue;
};
void* or_db_build(const char* seq, const uint64_t* prot_off, uint32_t n_prot, const OrMod* mods, uint32_t n_mods,
                  const OrParams* params);
void or_db_free(void* h);
uint64_t or_db_size(void* h);
void or_partition_lbe(void* h, uint32_t n_parts, uint32_t* part);
void or_search(void* h, const uint64_t* peak_off, const float* mz, const float* inten, const double* prec_mz,
               const uint8_t* charge, const double* tol, const uint32_t* sel, uint32_t n_sel, OrPsm* out_psm,
               uint32_t* out_hist, uint32_t* out_nscored, uint32_t* out_lo, uint32_t* out_hi);
void or_evalue(const uint32_t* hist, uint32_t nbins, const int64_t* keys, const uint32_t* pids, uint32_t k,
               uint32_t ev_mode, double* out);
uint32_t or_edit_distance(const char* x, const uint8_t* xc, const char* y, const uint8_t* yc);
double or_mod_distance(const char* x, const uint8_t* xc, const char* y, const uint8_t* yc);
}

namespace {

// a fixed pseudo-random proteome (64-bit LCG), residues over the 20 letters
std::string proteome(uint32_t n, std::vector<uint64_t>& off) {
    const char* aa = "ACDEFGHIKLMNPQRSTVWY";
    uint64_t s = 2102022860ull;
    std::string seq;
    off.assign(1, 0);
    for (uint32_t p = 0; p < n; ++p) {
        s = s * 6364136223846793005ull + 1442695040888963407ull;
        const uint32_t len = 60 + (uint32_t)((s >> 33) % 140);
        for (uint32_t i = 0; i < len; ++i) {
            s = s * 6364136223846793005ull + 1442695040888963407ull;
            seq.push_back(aa[(s >> 33) % 20]);
        }
        off.push_back(seq.size());
    }
    return seq;
}

void write_text(const char* path, const char* text) {
    FILE* f = fopen(path, "wb");
    CHECK(f != nullptr);
    fputs(text, f);
    fclose(f);
}

}  // namespace

int main(int argc, char** argv) {
    CHECK(argc == 3);   // golden MS2 file, a scratch directory
    std::vector<uint64_t> off;
    const std::string seq = proteome(30, off);
    const uint32_t n_prot = (uint32_t)(off.size() - 1);

    // ---- library host half
    hicops_mod mods[3] = {{"C", 57.021464, 0, 1}, {"M", 15.994915, 2, 0}, {"STY", 79.966331, 1, 0}};
    hicops_params p{};
    p.min_len = 7;
    p.max_len = 40;
    p.missed_cleavages = 2;
    p.min_mass = 500.0;
    p.max_mass = 5000.0;
    p.frag_mz_min = 100.0;
    p.frag_mz_max = 2000.0;
    p.bin_width_da = 0.01;
    p.top_n_peaks = 100;
    p.min_shared = 4;
    p.top_k = 5;
    p.hist_bins = 256;
    p.intensity_scale = 10000;
    hicops_proteins prot{n_prot, seq.data(), off.data()};
    hicops_index* idx = nullptr;
    CHECK(hicops_digest(&prot, mods, 3, &p, &idx) == HICOPS_OK);
    hicops_index_stats st{};
    CHECK(hicops_index_get_stats(idx, &st) == HICOPS_OK);
    const uint64_t P = st.n_peptides;
    CHECK(P > 1000);
    std::vector<uint32_t> part(P);
    CHECK(hicops_partition_lbe(idx, 4, part.data()) == HICOPS_OK);
    for (uint32_t s = 0; s < 4; ++s) {
        std::vector<uint32_t> pids;
        for (uint64_t i = 0; i < P; ++i)
            if (part[i] == s) pids.push_back((uint32_t)i);
        hicops_index* sub = nullptr;
        CHECK(hicops_index_subset(idx, pids.data(), pids.size(), &sub) == HICOPS_OK);
        char a[64], b[64];
        double ma = 0, mb = 0;
        uint64_t ka = 0, kb = 0;
        for (size_t i = 0; i < pids.size(); i += 17) {
            CHECK(hicops_peptide(sub, pids[i], a, sizeof(a), &ma, &ka) == HICOPS_OK);
            CHECK(hicops_peptide(idx, pids[i], b, sizeof(b), &mb, &kb) == HICOPS_OK);
            CHECK(strcmp(a, b) == 0 && ma == mb && ka == kb);
        }
        hicops_index* again = nullptr;
        CHECK(hicops_index_subset(sub, pids.data(), 1, &again) == HICOPS_EINVAL);
        hicops_index_free(sub);
    }
    uint32_t bad[3] = {5, 5, 9};
    hicops_index* none = nullptr;
    CHECK(hicops_index_subset(idx, bad, 3, &none) == HICOPS_EINVAL);
    hicops_index* sh = nullptr;
    CHECK(hicops_index_shard(idx, 3, 1, &sh) == HICOPS_OK);
    hicops_index_free(sh);

    // ---- checkpoint: round trip, then every truncation and a flipped byte of the file
    const std::string ck = std::string(argv[2]) + "/db.hix";
    CHECK(hicops_index_save(idx, ck.c_str()) == HICOPS_OK);
    hicops_index* back = nullptr;
    CHECK(hicops_index_load(ck.c_str(), &back) == HICOPS_OK);
    {
        char a[64], b[64];
        double ma = 0, mb = 0;
        uint64_t ka = 0, kb = 0;
        CHECK(hicops_peptide(back, 7, a, sizeof(a), &ma, &ka) == HICOPS_OK);
        CHECK(hicops_peptide(idx, 7, b, sizeof(b), &mb, &kb) == HICOPS_OK);
        CHECK(strcmp(a, b) == 0 && ma == mb && ka == kb);
    }
    hicops_index_free(back);
    std::string blob;
    {
        FILE* f = fopen(ck.c_str(), "rb");
        CHECK(f != nullptr);
        char buf[1 << 16];
        size_t n;
        while ((n = fread(buf, 1, sizeof(buf), f)) > 0) blob.append(buf, n);
        fclose(f);
    }
    const std::string cut = std::string(argv[2]) + "/cut.hix";
    for (size_t len = 0; len < blob.size(); len += 1 + len / 3) {
        FILE* f = fopen(cut.c_str(), "wb");
        CHECK(f != nullptr);
        fwrite(blob.data(), 1, len, f);
        fclose(f);
        hicops_index* x = nullptr;
        CHECK(hicops_index_load(cut.c_str(), &x) == HICOPS_EINVAL && x == nullptr);
    }
    for (size_t at : {size_t(20), size_t(200), blob.size() / 2, blob.size() - 5}) {
        std::string bad = blob;
        bad[at] = (char)(bad[at] ^ 0x5a);
        FILE* f = fopen(cut.c_str(), "wb");
        CHECK(f != nullptr);
        fwrite(bad.data(), 1, bad.size(), f);
        fclose(f);
        hicops_index* x = nullptr;
        const hicops_status s = hicops_index_load(cut.c_str(), &x);   // rejected, or a consistent index
        if (s == HICOPS_OK) hicops_index_free(x);
    }

    // ---- oracle: same database, same partition; a search; e-values
    OrMod omods[3] = {{"C", 57.021464, 0, 1}, {"M", 15.994915, 2, 0}, {"STY", 79.966331, 1, 0}};
    OrParams op{};
    op.min_len = 7;
    op.max_len = 40;
    op.missed_cleavages = 2;
    op.min_mass = 500.0;
    op.max_mass = 5000.0;
    op.frag_mz_min = 100.0;
    op.frag_mz_max = 2000.0;
    op.bin_width = 0.01;
    op.top_n_peaks = 100;
    op.min_shared = 4;
    op.top_k = 5;
    op.hist_bins = 256;
    op.intensity_scale = 10000;
    op.tol_bins = 1;
    op.evalue_mode = 3;
    void* db = or_db_build(seq.data(), off.data(), n_prot, omods, 3, &op);
    CHECK(or_db_size(db) == P);
    std::vector<uint32_t> opart(P);
    or_partition_lbe(db, 4, opart.data());
    CHECK(opart == part);
    const uint64_t peak_off[3] = {0, 4, 4};
    const float mz[4] = {175.119f, 300.2f, 450.25f, 1200.5f};
    const float it[4] = {10.0f, 20.0f, 5.0f, 40.0f};
    const double prec[2] = {700.0, 900.0};
    const uint8_t z[2] = {2, 2};
    const double tol[2] = {500.0, 500.0};
    const uint32_t sel[2] = {0, 1};
    std::vector<OrPsm> psm(2 * 5);
    std::vector<uint32_t> hist(2 * 256), ns(2), lo(2), hi(2);
    or_search(db, peak_off, mz, it, prec, z, tol, sel, 2, psm.data(), hist.data(), ns.data(), lo.data(), hi.data());
    CHECK(ns[1] == 0);   // the second spectrum has no peaks
    or_db_free(db);
    uint32_t h[256] = {};
    for (int j = 0; j < 256; ++j) h[j] = (uint32_t)(1e6 * std::exp(-std::abs(j - 30.0) / 4.0));
    const int64_t keys[2] = {int64_t(60) << 31, int64_t(45) << 31};
    const uint32_t pids[2] = {1, 2};
    double ev[2];
    for (uint32_t mode = 0; mode < 4; ++mode) {
        or_evalue(h, 256, keys, pids, 2, mode, ev);
        CHECK(std::isfinite(ev[0]) && std::isfinite(ev[1]) && ev[0] <= ev[1]);
    }
    const uint8_t c0[8] = {0, 0, 0, 0, 0, 0, 0, 0}, cq[8] = {0, 1, 0, 0, 0, 1, 0, 0};
    CHECK(or_edit_distance("MEGSYIRK", c0, "MEGSYIRK", cq) == 2);
    CHECK(or_mod_distance("MEGSYIRK", c0, "MEGSYIRK", cq) == 1.625);

    // ---- MS2 parsing, forecast and rules
    uint32_t nsp = 0;
    uint64_t npk = 0;
    CHECK(hicops_ms2_read(argv[1], 0, 0, &nsp, &npk, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr) ==
          HICOPS_OK);
    std::vector<uint64_t> po(nsp + 1);
    std::vector<float> pm(npk), pi(npk);
    std::vector<double> pp(nsp);
    std::vector<uint8_t> pz(nsp);
    std::vector<uint32_t> sc(nsp);
    CHECK(hicops_ms2_read(argv[1], nsp, npk, &nsp, &npk, po.data(), pm.data(), pi.data(), pp.data(), pz.data(),
                          sc.data()) == HICOPS_OK);
    CHECK(nsp == 3 && npk == 5 && pz[1] == 0);
    const std::string dir = argv[2];
    const char* bad_files[] = {"101.5 20\n", "S\t1\t1\t500\n100 1 2\n", "S\t1\t1\n", "S\t1\t1\t500\n100 abc",
                               "S\t1\t1\t500\nZ\t999\t1\n", ""};
    for (int i = 0; i < 6; ++i) {
        const std::string path = dir + "/bad" + std::to_string(i) + ".ms2";
        write_text(path.c_str(), bad_files[i]);
        const hicops_status s = hicops_ms2_read(path.c_str(), 0, 0, &nsp, &npk, nullptr, nullptr, nullptr, nullptr,
                                                nullptr, nullptr);
        CHECK(i == 5 ? (s == HICOPS_OK && nsp == 0) : s == HICOPS_EINVAL);
    }
    double state[2];
    double f = 0;
    for (int i = 0; i < 50; ++i) f = hicops_des_step(state, 1.0 + 0.5 * i, 0.5, i == 0);
    CHECK(std::fabs(f - (1.0 + 0.5 * 50)) < 1e-9);
    CHECK(hicops_sched_i_to_r(0.002, 0.04, 0.02, 0.001, 0.05, 10, 1) == 1);
    CHECK(hicops_sched_r_to_i(20, 20, 1) == 1);

    hicops_index_free(idx);
    printf("host sanitize ok: %llu peptides\n", (unsigned long long)P);
    return 0;
}
