// HiCOPS search oracle: a plain, slow, single-threaded FP64 CPU
// implementation of the superstep-3 search (paper: "Superstep 3: Partial
// Database Peptide Search", Eq. 4 and Supplementary Algorithm 3) and of the
// database construction it depends on (Superstep 1, Supplementary
// Algorithm 1), plus the superstep-4 linear-tail-fit e-value
// (Supplementary Algorithm 4).
//
// TEST INFRASTRUCTURE ONLY.  Only the tests, __graft_entry__.smoke() and the
// CPU-baseline leg of bench.py load this library.  It shares no code, header
// or table with the CUDA path; it is written from the paper's definitions:
//
//   * the fragment index is an accelerator for shared-peak counting, so the
//     oracle does NOT build an index: for every spectrum and every peptide
//     inside the precursor window it intersects the two bin sets directly
//     (filter_1 = precursor mass window, filter_2 = shared peaks >= k,
//     Supplementary Text 4's shp(f, g, k));
//   * scores are the hyperscore (Superstep 3, cost term k33/k34);
//   * each spectrum keeps its top hits and its score histogram (Sampling
//     section: M top hits plus the local score distribution);
//   * the e-value is a linear fit to the survival tail of that histogram
//     (Superstep 4, Supplementary Algorithm 4).
//
// Where the paper is silent the oracle takes these readings:
//   R1 monoisotopic residue masses, H2O 18.010565, proton 1.007276466812;
//   R2 trypsin: cut after K/R unless the next residue is P; peptides from
//      consecutive cut boundaries with <= missed_cleavages internal sites;
//   R3 variable modifications: every subset of modifiable positions with at
//      most max_per_peptide positions per rule (the 2^m variants of the
//      Notation section); a position carries at most one modification;
//   R4 peptide order: (neutral mass, sequence bytes, per-position mod codes)
//      ascending; pid = rank in that order;
//   R5 masses summed left to right in FP64:  M = sum(m_j) + H2O;
//      b_i = sum_{j<=i} m_j + proton;  y_i = (sum_{j=L..i+1} m_j + H2O) + proton;
//   R6 bin(mz) = floor(mz / w) for frag_mz_min <= mz < frag_mz_max; a peak
//      and an ion are shared iff their bins are equal (w = dF);
//   R15 (fragment tolerance of t bins, dF = t * w on a finer grid) an ion
//      bin x is shared iff some retained peak bin b has |x - b| <= t, i.e.
//      x lies in the union of the peaks' windows [b - t, b + t]; it counts
//      once and contributes the largest iq of the peaks covering it; t = 0
//      is R6;
//   R7 a peptide's ion set is its set of distinct bins; a bin holding both a
//      b and a y ion of the same peptide counts once, as b;
//   R8 preprocessing: drop non-finite / non-positive / out-of-range peaks,
//      bin, merge equal bins keeping the max intensity, keep the top_n most
//      intense (ties to the lower bin), iq = max(1, floor(I*scale/Imax));
//      precursor neutral mass Mq = (prec_mz - proton) * z;
//   R9 window: Mq - dM <= M_p <= Mq + dM;
//   R10 hyperscore HS = log10(nb!) + log10(ny!) + log10(S); rank key
//      K = LF[nb] + LF[ny] + LS[S] with LF[n] = llround(2^32 * sum log10 i)
//      and LS[s] = llround(2^32 * log10 s); top-k by (K desc, pid asc);
//   R11 histogram bin = min(255, K >> 31) over every candidate;
//   R12 e-value: survival s_j = sum_{i>=j} hist_i; least-squares line through
//      (j, log10(s_j / N)) for j in [mode+1, jtop-1] with s_j > 0; e = N *
//      10^(w * K*2^-31 + b); fewer than 3 points -> e = N;
//   R16 (optional) the fit sees the histogram smoothed by the 5-point
//      quadratic Savitzky-Golay filter (taps -3 12 17 12 -3 over 35, zero
//      outside the bins), kept as 35 times its value so it stays integer;
//   R18 LBE partition with the Mod Distance: a cluster is the set of entries
//      sharing one unmodified sequence; inside a cluster entries are ordered
//      by (edit distance to the unmodified sequence, Mod Distance to it,
//      pid); clusters follow one another in the order of their smallest
//      pid; position i of that sequence goes to partition i mod P.  Edit
//      distance: Levenshtein over residues, a modified residue being a
//      symbol of its own; Mod Distance 2 - a / max(len x, len y), a = the
//      letters equal from the N-terminus up to the first edit plus those
//      equal from the C-terminus up to the last edit (2 len when x = y);
//   R17 (optional, instead of R12) log-Weibull (Gumbel) fit: least squares
//      of -ln(-ln F_j) on x = j + 1, F_j = fraction scoring below j + 1, over
//      bins with 0 < F_j < 1; e = N * (1 - exp(-exp(-(a x + c)))), x =
//      K*2^-31; fewer than 3 points or a <= 0 -> e = N.
//   R19 sampling of a partial score distribution (Sampling section and its
//      figure): a sample is one histogram bin; the mean is the integer
//      average (rounded down) of the locations of the three most intense
//      bins (count descending, lower location first on equal counts; fewer
//      when fewer bins are non-zero); from the non-zero support [L, R] the
//      tail samples are pruned first: while more than s bins remain, the
//      end farther from the mean is dropped (the upper end on a tie); the
//      kept bins are one run [lo, lo + len) with their exact counts.
//
// Parity pins: see tests/test_oracle_pins.py (closed forms, elemental
// composition masses, brute force on tiny inputs, invariants, library
// routines, the Mod Distance worked example).  Parity unpinned: the absolute
// scale of the hyperscore, the histogram bin width and the e-value fit
// window (R10-R12), the smoothing window and order (R16), the log-Weibull
// fitting method (R17), the LBE cluster rule (R18) and the sampling's
// rounding of the mean and tie rule (R19) are readings with no printed
// value.  R19 is pinned by hand-worked distributions and by its result
// stated as an optimisation (tests/golden/sampling_hand.txt).

#include <cmath>
#include <cstdint>
#include <cstring>
#include <string>
#include <vector>
#include <algorithm>
#include <map>

namespace {

const double kWater = 18.010565;
const double kProton = 1.007276466812;

double residue_mass(char aa) {
    switch (aa) {
        case 'G': return 57.021464;  case 'A': return 71.037114;
        case 'S': return 87.032028;  case 'P': return 97.052764;
        case 'V': return 99.068414;  case 'T': return 101.047679;
        case 'C': return 103.009185; case 'L': return 113.084064;
        case 'I': return 113.084064; case 'N': return 114.042927;
        case 'D': return 115.026943; case 'Q': return 128.058578;
        case 'K': return 128.094963; case 'E': return 129.042593;
        case 'M': return 131.040485; case 'H': return 137.058912;
        case 'F': return 147.068414; case 'R': return 156.101111;
        case 'Y': return 163.063329; case 'W': return 186.079313;
        default:  return -1.0;
    }
}

}  // namespace

extern "C" {

// One modification rule.  residues: NUL-terminated letters it applies to.
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
    uint32_t tol_bins;         // R15 fragment tolerance in bins (0 = R6)
    uint32_t evalue_mode;      // bit 0: R17 log-Weibull fit (else R12), bit 1: R16 smoothing
};

// One PSM row of the oracle's output.
struct OrPsm {
    uint32_t pid;       // UINT32_MAX for padding rows
    uint32_t nb, ny, S;
    int64_t key;        // INT64_MIN for padding rows
    double hyperscore;  // FP64, computed directly
    double evalue;
};

}  // extern "C"

namespace {

struct Peptide {
    double mass;
    std::string seq;
    std::vector<uint8_t> code;   // per position: 0 or 1 + variable-mod index
};

struct Db {
    OrParams p;
    std::vector<double> fixed_delta;      // per ASCII letter
    std::vector<double> var_delta;        // per variable-mod index
    std::vector<std::string> var_res;
    std::vector<uint32_t> var_max;
    std::vector<Peptide> peps;
};

// mass of residue j of a peptide, R5 with fixed + variable modifications
double position_mass(const Db& db, char aa, uint8_t code) {
    double m = residue_mass(aa);
    if (db.fixed_delta[(unsigned char)aa] != 0.0) m = m + db.fixed_delta[(unsigned char)aa];
    if (code) m = m + db.var_delta[code - 1];
    return m;
}

double peptide_mass(const Db& db, const std::string& s, const std::vector<uint8_t>& code) {
    double sum = 0.0;
    for (size_t j = 0; j < s.size(); ++j) sum = sum + position_mass(db, s[j], code[j]);
    return sum + kWater;
}

// R5: b_i and y_i for i = 1..L-1 (b[i-1], y[i-1]); y_i covers residues i+1..L
void ions(const Db& db, const Peptide& pep, std::vector<double>& b, std::vector<double>& y) {
    const size_t L = pep.seq.size();
    b.assign(L - 1, 0.0);
    y.assign(L - 1, 0.0);
    double pre = 0.0;
    for (size_t i = 1; i < L; ++i) {
        pre = pre + position_mass(db, pep.seq[i - 1], pep.code[i - 1]);
        b[i - 1] = pre + kProton;
    }
    for (size_t i = 1; i < L; ++i) {
        double suf = 0.0;
        for (size_t j = L; j >= i + 1; --j) suf = suf + position_mass(db, pep.seq[j - 1], pep.code[j - 1]);
        y[i - 1] = (suf + kWater) + kProton;
    }
}

bool in_range(const OrParams& p, double mz) { return mz >= p.frag_mz_min && mz < p.frag_mz_max; }
uint32_t bin_of(const OrParams& p, double mz) { return (uint32_t)std::floor(mz / p.bin_width); }

// R7: distinct ion bins, b precedence.  Returns (bin, isY) sorted by bin.
std::vector<std::pair<uint32_t, int>> ion_bins(const Db& db, const Peptide& pep) {
    std::vector<double> b, y;
    ions(db, pep, b, y);
    std::map<uint32_t, int> m;
    for (double v : y) if (in_range(db.p, v)) m[bin_of(db.p, v)] = 1;
    for (double v : b) if (in_range(db.p, v)) m[bin_of(db.p, v)] = 0;   // b overrides y
    return std::vector<std::pair<uint32_t, int>>(m.begin(), m.end());
}

bool std_letters(const std::string& s) {
    for (char c : s) if (residue_mass(c) < 0) return false;
    return true;
}

// R3: recursive enumeration over the positions of the peptide.
void enumerate(const Db& db, const std::string& s, size_t pos, std::vector<uint8_t>& code,
               std::vector<uint32_t>& used, uint32_t total, std::vector<Peptide>& out) {
    if (pos == s.size()) {
        Peptide pep;
        pep.seq = s;
        pep.code = code;
        pep.mass = peptide_mass(db, s, code);
        if (pep.mass >= db.p.min_mass && pep.mass <= db.p.max_mass) out.push_back(pep);
        return;
    }
    code[pos] = 0;
    enumerate(db, s, pos + 1, code, used, total, out);
    for (size_t t = 0; t < db.var_res.size(); ++t) {
        if (db.var_res[t].find(s[pos]) == std::string::npos) continue;
        if (used[t] >= db.var_max[t]) continue;
        if (db.p.max_total_mods && total >= db.p.max_total_mods) continue;
        code[pos] = (uint8_t)(t + 1);
        used[t]++;
        enumerate(db, s, pos + 1, code, used, total + 1, out);
        used[t]--;
        code[pos] = 0;
    }
}

bool pep_less(const Peptide& a, const Peptide& b) {
    if (a.mass != b.mass) return a.mass < b.mass;
    if (a.seq != b.seq) return a.seq < b.seq;
    return a.code < b.code;
}

struct Query {
    bool valid;
    double Mq, tol;
    std::vector<uint32_t> bins;   // sorted ascending
    std::vector<uint32_t> iq;     // parallel to bins
};

// R8
Query preprocess(const OrParams& p, const float* mz, const float* inten, uint64_t n,
                 double prec_mz, uint8_t z, double tol) {
    Query q;
    std::map<uint32_t, double> merged;
    for (uint64_t i = 0; i < n; ++i) {
        double m = (double)mz[i], I = (double)inten[i];
        if (!std::isfinite(m) || !std::isfinite(I) || !(I > 0.0)) continue;
        if (!in_range(p, m)) continue;
        uint32_t b = bin_of(p, m);
        auto it = merged.find(b);
        if (it == merged.end() || I > it->second) merged[b] = I;
    }
    std::vector<std::pair<uint32_t, double>> v(merged.begin(), merged.end());
    std::sort(v.begin(), v.end(), [](const std::pair<uint32_t, double>& a, const std::pair<uint32_t, double>& b) {
        if (a.second != b.second) return a.second > b.second;
        return a.first < b.first;
    });
    if (v.size() > p.top_n_peaks) v.resize(p.top_n_peaks);
    q.valid = z > 0 && std::isfinite(prec_mz) && std::isfinite(tol) && tol >= 0.0 && !v.empty();
    q.Mq = (prec_mz - kProton) * (double)z;
    q.tol = tol;
    if (!q.valid) return q;
    const double Imax = v[0].second;
    std::sort(v.begin(), v.end());
    for (auto& e : v) {
        double r = std::floor((e.second * (double)p.intensity_scale) / Imax);
        uint32_t iq = r < 1.0 ? 1u : (uint32_t)r;
        q.bins.push_back(e.first);
        q.iq.push_back(iq);
    }
    return q;
}

// R15: is ion bin x inside some retained peak's window [b - t, b + t]?  If
// so, iq = the largest quantised intensity of the peaks whose window holds x.
bool covered(const Query& q, uint32_t x, uint32_t t, uint32_t& iq) {
    const uint32_t from = x > t ? x - t : 0u;
    auto it = std::lower_bound(q.bins.begin(), q.bins.end(), from);   // first peak with b >= x - t
    bool hit = false;
    iq = 0;
    for (; it != q.bins.end() && (uint64_t)*it <= (uint64_t)x + t; ++it) {
        hit = true;
        iq = std::max(iq, q.iq[it - q.bins.begin()]);
    }
    return hit;
}

double log10_factorial(uint32_t n) {
    double s = 0.0;
    for (uint32_t i = 2; i <= n; ++i) s = s + std::log10((double)i);
    return s;
}

// R10
int64_t rank_key(uint32_t nb, uint32_t ny, uint32_t S) {
    return std::llround(std::ldexp(log10_factorial(nb), 32)) +
           std::llround(std::ldexp(log10_factorial(ny), 32)) +
           std::llround(std::ldexp(std::log10((double)S), 32));
}

// R12 (linear tail fit), R16 (Savitzky-Golay smoothing first), R17
// (log-Weibull fit instead of the tail fit)
void evalues(const uint32_t* hist, uint32_t nbins, const std::vector<OrPsm>& top, uint32_t ev_mode,
             std::vector<double>& ev) {
    ev.assign(top.size(), INFINITY);
    if (top.empty() || top[0].pid == UINT32_MAX) return;
    double N = 0.0;
    for (uint32_t j = 0; j < nbins; ++j) N += (double)hist[j];
    // the distribution the fit sees: the histogram, or (R16) 35 times its
    // 5-point quadratic Savitzky-Golay smoothing, the histogram taken as 0
    // outside its bins; integers either way
    std::vector<int64_t> g(nbins, 0);
    for (int64_t j = 0; j < (int64_t)nbins; ++j) {
        if (!(ev_mode & 2u)) { g[j] = hist[j]; continue; }
        static const int64_t c[5] = {-3, 12, 17, 12, -3};
        for (int d = -2; d <= 2; ++d) {
            const int64_t i = j + d;
            if (i >= 0 && i < (int64_t)nbins) g[j] += c[d + 2] * (int64_t)hist[i];
        }
    }
    std::vector<int64_t> G(nbins + 1, 0);   // G[j] = sum of g[i >= j]
    for (int64_t j = (int64_t)nbins - 1; j >= 0; --j) G[j] = G[j + 1] + g[j];
    const double G0 = (double)G[0];
    double n = 0, sx = 0, sy = 0, sxx = 0, sxy = 0;
    if (ev_mode & 1u) {
        // R17: the log-Weibull (Gumbel) CDF F(x) = exp(-exp(-(a x + c)))
        // fitted by least squares of -ln(-ln F_j) on x = j + 1, where F_j =
        // 1 - G[j + 1] / G[0] is the fraction scoring below j + 1, over the
        // bins with 0 < F_j < 1
        for (uint32_t j = 0; j < nbins; ++j) {
            if (!(G[j + 1] > 0 && G[j + 1] < G[0])) continue;
            const double x = (double)(j + 1);
            const double yv = -std::log(-std::log1p(-((double)G[j + 1] / G0)));
            n += 1; sx += x; sy += yv; sxx += x * x; sxy += x * yv;
        }
        double a = 0, c = 0;
        bool fit = n >= 3;
        if (fit) {
            const double den = n * sxx - sx * sx;
            a = (n * sxy - sx * sy) / den;
            c = (sy - a * sx) / n;
            fit = a > 0;
        }
        for (size_t r = 0; r < top.size(); ++r) {
            if (top[r].pid == UINT32_MAX) continue;
            if (!fit) { ev[r] = N; continue; }
            const double x = std::ldexp((double)top[r].key, -31);
            ev[r] = N * -std::expm1(-std::exp(-(a * x + c)));   // N * P(score >= x)
        }
        return;
    }
    // R12 on g: survival G[j] / G[0]; line through (j, log10 of it) for j in
    // [mode + 1, jtop - 1] with G[j] > 0; mode = the largest g, lowest bin
    uint32_t mode = 0;
    for (uint32_t j = 1; j < nbins; ++j) if (g[j] > g[mode]) mode = j;
    const int64_t jtop = std::min<int64_t>(nbins - 1, top[0].key >> 31);
    for (int64_t j = mode + 1; j <= jtop - 1; ++j) {
        if (!(G[j] > 0)) continue;
        double x = (double)j, yv = std::log10((double)G[j] / G0);
        n += 1; sx += x; sy += yv; sxx += x * x; sxy += x * yv;
    }
    bool fit = n >= 3;
    double w = 0, b = 0;
    if (fit) {
        double den = n * sxx - sx * sx;
        w = (n * sxy - sx * sy) / den;
        b = (sy - w * sx) / n;
    }
    for (size_t r = 0; r < top.size(); ++r) {
        if (top[r].pid == UINT32_MAX) continue;
        if (!fit) { ev[r] = N; continue; }
        double x = std::ldexp((double)top[r].key, -31);
        ev[r] = N * std::pow(10.0, w * x + b);
    }
}

// R18: residue i of a peptide as one symbol (letter, modification code)
uint32_t symbol(const std::string& seq, const std::vector<uint8_t>& code, size_t i) {
    return (uint32_t)(unsigned char)seq[i] << 8 | code[i];
}

// R18: Levenshtein distance (unit insertions, deletions, substitutions)
uint32_t edit_distance(const std::string& xs, const std::vector<uint8_t>& xc, const std::string& ys,
                       const std::vector<uint8_t>& yc) {
    const size_t n = xs.size(), m = ys.size();
    std::vector<uint32_t> prev(m + 1), cur(m + 1);
    for (size_t j = 0; j <= m; ++j) prev[j] = (uint32_t)j;
    for (size_t i = 1; i <= n; ++i) {
        cur[0] = (uint32_t)i;
        for (size_t j = 1; j <= m; ++j) {
            const uint32_t sub = prev[j - 1] + (symbol(xs, xc, i - 1) == symbol(ys, yc, j - 1) ? 0u : 1u);
            cur[j] = std::min({prev[j] + 1u, cur[j - 1] + 1u, sub});
        }
        std::swap(prev, cur);
    }
    return prev[m];
}

// R18: Mod Distance 2 - a / max(len x, len y)
double mod_distance(const std::string& xs, const std::vector<uint8_t>& xc, const std::string& ys,
                    const std::vector<uint8_t>& yc) {
    const size_t n = xs.size(), m = ys.size();
    size_t a = 0;
    for (size_t i = 0; i < std::min(n, m) && symbol(xs, xc, i) == symbol(ys, yc, i); ++i) ++a;   // from the N-terminus
    for (size_t i = 0; i < std::min(n, m) && symbol(xs, xc, n - 1 - i) == symbol(ys, yc, m - 1 - i); ++i) ++a;   // C
    return 2.0 - (double)a / (double)std::max(n, m);
}

}  // namespace

extern "C" {

// R18 for two peptides given as letters and per-position modification codes
// (0 = none): edit distance and Mod Distance.
uint32_t or_edit_distance(const char* x, const uint8_t* xc, const char* y, const uint8_t* yc) {
    const std::string xs(x), ys(y);
    return edit_distance(xs, std::vector<uint8_t>(xc, xc + xs.size()), ys, std::vector<uint8_t>(yc, yc + ys.size()));
}

double or_mod_distance(const char* x, const uint8_t* xc, const char* y, const uint8_t* yc) {
    const std::string xs(x), ys(y);
    return mod_distance(xs, std::vector<uint8_t>(xc, xc + xs.size()), ys, std::vector<uint8_t>(yc, yc + ys.size()));
}

// R18: the LBE partition of the database over n_parts: part[pid].
void or_partition_lbe(void* h, uint32_t n_parts, uint32_t* part) {
    const Db* db = (Db*)h;
    const size_t P = db->peps.size();
    std::map<std::string, std::vector<uint32_t>> clusters;   // unmodified sequence -> pids (ascending)
    for (size_t pid = 0; pid < P; ++pid) clusters[db->peps[pid].seq].push_back((uint32_t)pid);
    std::vector<std::vector<uint32_t>> order;
    for (auto& kv : clusters) {
        const std::string& base = kv.first;
        const std::vector<uint8_t> none(base.size(), 0);
        std::vector<uint32_t> c = kv.second;
        std::stable_sort(c.begin(), c.end(), [&](uint32_t x, uint32_t y) {
            const Peptide& px = db->peps[x];
            const Peptide& py = db->peps[y];
            const uint32_t ex = edit_distance(px.seq, px.code, base, none);
            const uint32_t ey = edit_distance(py.seq, py.code, base, none);
            if (ex != ey) return ex < ey;
            const double mx = mod_distance(px.seq, px.code, base, none);
            const double my = mod_distance(py.seq, py.code, base, none);
            if (mx != my) return mx < my;
            return x < y;
        });
        order.push_back(c);
    }
    std::sort(order.begin(), order.end(), [&](const std::vector<uint32_t>& x, const std::vector<uint32_t>& y) {
        return *std::min_element(x.begin(), x.end()) < *std::min_element(y.begin(), y.end());
    });
    size_t i = 0;
    for (auto& c : order)
        for (uint32_t pid : c) part[pid] = (uint32_t)(i++ % n_parts);
}

// Builds the oracle's peptide database (Superstep 1 without an index).
void* or_db_build(const char* seq, const uint64_t* prot_off, uint32_t n_prot,
                  const OrMod* mods, uint32_t n_mods, const OrParams* params) {
    Db* db = new Db();
    db->p = *params;
    db->fixed_delta.assign(256, 0.0);
    for (uint32_t i = 0; i < n_mods; ++i) {
        if (mods[i].fixed) {
            for (const char* r = mods[i].residues; *r; ++r) db->fixed_delta[(unsigned char)*r] = mods[i].delta;
        } else {
            db->var_delta.push_back(mods[i].delta);
            db->var_res.push_back(mods[i].residues);
            db->var_max.push_back(mods[i].max_per_peptide);
        }
    }
    std::vector<Peptide> all;
    for (uint32_t pr = 0; pr < n_prot; ++pr) {
        const std::string prot(seq + prot_off[pr], seq + prot_off[pr + 1]);
        // R2: boundaries 0, after each K/R not followed by P, and the end
        std::vector<size_t> cuts{0};
        for (size_t i = 0; i + 1 < prot.size(); ++i)
            if ((prot[i] == 'K' || prot[i] == 'R') && prot[i + 1] != 'P') cuts.push_back(i + 1);
        cuts.push_back(prot.size());
        for (size_t a = 0; a + 1 < cuts.size(); ++a) {
            for (size_t b = a + 1; b < cuts.size() && b - a - 1 <= db->p.missed_cleavages; ++b) {
                size_t len = cuts[b] - cuts[a];
                if (len < db->p.min_len || len > db->p.max_len) continue;
                std::string s = prot.substr(cuts[a], len);
                if (!std_letters(s)) continue;
                std::vector<uint8_t> code(len, 0);
                std::vector<uint32_t> used(db->var_res.size(), 0);
                enumerate(*db, s, 0, code, used, 0, all);
            }
        }
    }
    std::sort(all.begin(), all.end(), pep_less);
    // identical (sequence, mod state) from several proteins: one entry
    for (auto& pep : all) {
        if (!db->peps.empty() && db->peps.back().seq == pep.seq && db->peps.back().code == pep.code) continue;
        db->peps.push_back(pep);
    }
    return db;
}

void or_db_free(void* h) { delete (Db*)h; }

uint64_t or_db_size(void* h) { return ((Db*)h)->peps.size(); }

// Peptide pid: sequence (NUL-terminated, up to cap-1 letters), neutral mass
// and per-position mod codes (0 = none, 1 + variable-mod index).
uint32_t or_db_peptide(void* h, uint64_t pid, char* seq, uint32_t cap, double* mass, uint8_t* codes) {
    const Db* db = (Db*)h;
    const Peptide& p = db->peps[pid];
    uint32_t L = (uint32_t)p.seq.size();
    if (seq) { uint32_t n = std::min(L, cap - 1); memcpy(seq, p.seq.data(), n); seq[n] = 0; }
    if (mass) *mass = p.mass;
    if (codes) memcpy(codes, p.code.data(), L);
    return L;
}

void or_db_masses(void* h, double* out) {
    const Db* db = (Db*)h;
    for (size_t i = 0; i < db->peps.size(); ++i) out[i] = db->peps[i].mass;
}

// b and y ion m/z (unbinned) of peptide pid, i = 1..L-1; returns L-1.
uint32_t or_db_ions(void* h, uint64_t pid, double* b, double* y) {
    const Db* db = (Db*)h;
    std::vector<double> vb, vy;
    ions(*db, db->peps[pid], vb, vy);
    for (size_t i = 0; i < vb.size(); ++i) { b[i] = vb[i]; y[i] = vy[i]; }
    return (uint32_t)vb.size();
}

// Distinct ion bins of peptide pid (R7), sorted by bin; returns the count.
uint32_t or_db_bins(void* h, uint64_t pid, uint32_t* bins, uint8_t* is_y) {
    const Db* db = (Db*)h;
    auto v = ion_bins(*db, db->peps[pid]);
    for (size_t i = 0; i < v.size(); ++i) { bins[i] = v[i].first; is_y[i] = (uint8_t)v[i].second; }
    return (uint32_t)v.size();
}

// Preprocessed query (R8): returns the number of retained peaks (0 when the
// spectrum is invalid) and writes bins (ascending), quantised intensities,
// neutral precursor mass and validity.
uint32_t or_preprocess(const OrParams* p, const float* mz, const float* inten, uint64_t n,
                       double prec_mz, uint8_t z, double tol, uint32_t* bins, uint32_t* iq,
                       double* Mq, int* valid) {
    Query q = preprocess(*p, mz, inten, n, prec_mz, z, tol);
    *Mq = q.Mq;
    *valid = q.valid;
    for (size_t i = 0; i < q.bins.size(); ++i) { bins[i] = q.bins[i]; iq[i] = q.iq[i]; }
    return (uint32_t)q.bins.size();
}

int64_t or_rank_key(uint32_t nb, uint32_t ny, uint32_t S) { return rank_key(nb, ny, S); }

double or_hyperscore(uint32_t nb, uint32_t ny, uint32_t S) {
    return log10_factorial(nb) + log10_factorial(ny) + std::log10((double)S);
}

// e-values for a given histogram and sorted top-k keys (R12; ev_mode bit 0
// R17, bit 1 R16).
void or_evalue(const uint32_t* hist, uint32_t nbins, const int64_t* keys, const uint32_t* pids,
               uint32_t k, uint32_t ev_mode, double* out) {
    std::vector<OrPsm> top(k);
    for (uint32_t i = 0; i < k; ++i) { top[i].key = keys[i]; top[i].pid = pids[i]; }
    std::vector<double> ev;
    evalues(hist, nbins, top, ev_mode, ev);
    for (uint32_t i = 0; i < k; ++i) out[i] = ev[i];
}

// R19: the bins [*lo, *lo + *len) of hist[0..nbins) kept when the
// distribution is sampled down to at most s bins around its mean; *len = 0
// for an empty histogram.  Returns the mean's location.
uint32_t or_hist_sample(const uint32_t* hist, uint32_t nbins, uint32_t s, uint32_t* lo, uint32_t* len) {
    *lo = 0;
    *len = 0;
    // the three most intense samples (count descending, location ascending)
    std::vector<uint32_t> order;
    for (uint32_t j = 0; j < nbins; ++j)
        if (hist[j] > 0) order.push_back(j);
    if (order.empty() || s == 0) return 0;
    std::stable_sort(order.begin(), order.end(), [&](uint32_t a, uint32_t b) { return hist[a] > hist[b]; });
    const size_t top = std::min<size_t>(3, order.size());
    uint64_t sum = 0;
    for (size_t i = 0; i < top; ++i) sum += order[i];
    const uint32_t mean = (uint32_t)(sum / top);
    // the support, then the tails pruned first
    uint32_t a = nbins, b = 0;
    for (uint32_t j = 0; j < nbins; ++j)
        if (hist[j] > 0) { a = std::min(a, j); b = std::max(b, j); }
    while (b - a + 1 > s) {
        if (b - mean >= mean - a) --b;
        else ++a;
    }
    *lo = a;
    *len = b - a + 1;
    return mean;
}

// Search the selected spectra (indices sel[0..n_sel-1] of the batch).
// Outputs per selected spectrum: psm[top_k], hist[hist_bins], n_scored,
// window [lo, hi).
// With n_shards > 1 only the database entries pid = shard (mod n_shards)
// are candidates: the partition one process searches (Superstep 3).
void or_search_shard(void* h, const uint64_t* peak_off, const float* mz, const float* inten,
                     const double* prec_mz, const uint8_t* charge, const double* tol,
                     const uint32_t* sel, uint32_t n_sel,
                     OrPsm* out_psm, uint32_t* out_hist, uint32_t* out_nscored,
                     uint32_t* out_lo, uint32_t* out_hi, uint32_t n_shards, uint32_t shard) {
    const Db* db = (Db*)h;
    const OrParams& p = db->p;
    const uint32_t K = p.top_k, H = p.hist_bins;
    std::vector<double> masses(db->peps.size());
    for (size_t i = 0; i < db->peps.size(); ++i) masses[i] = db->peps[i].mass;
    for (uint32_t si = 0; si < n_sel; ++si) {
        const uint32_t qi = sel[si];
        const uint64_t a = peak_off[qi], e = peak_off[qi + 1];
        Query q = preprocess(p, mz + a, inten + a, e - a, prec_mz[qi], charge[qi], tol[qi]);
        uint32_t* hist = out_hist + (uint64_t)si * H;
        for (uint32_t j = 0; j < H; ++j) hist[j] = 0;
        std::vector<OrPsm> cand;
        uint32_t lo = 0, hi = 0;
        if (q.valid) {
            // filter_1 (R9)
            lo = (uint32_t)(std::lower_bound(masses.begin(), masses.end(), q.Mq - q.tol) - masses.begin());
            hi = (uint32_t)(std::upper_bound(masses.begin(), masses.end(), q.Mq + q.tol) - masses.begin());
            for (uint32_t pid = lo; pid < hi; ++pid) {
                if (pid % n_shards != shard) continue;
                // filter_2: shared peaks between query bins and the peptide's ion bins
                auto ib = ion_bins(*db, db->peps[pid]);
                uint32_t nb = 0, ny = 0, S = 0;
                for (auto& bt : ib) {
                    uint32_t iq = 0;
                    if (p.tol_bins == 0) {   // R6: equal bins
                        auto it = std::lower_bound(q.bins.begin(), q.bins.end(), bt.first);
                        if (it == q.bins.end() || *it != bt.first) continue;
                        iq = q.iq[it - q.bins.begin()];
                    } else if (!covered(q, bt.first, p.tol_bins, iq)) {   // R15
                        continue;
                    }
                    if (bt.second) ny++; else nb++;
                    S += iq;
                }
                if (nb + ny < p.min_shared) continue;
                OrPsm c;
                c.pid = pid; c.nb = nb; c.ny = ny; c.S = S;
                c.key = rank_key(nb, ny, S);
                c.hyperscore = log10_factorial(nb) + log10_factorial(ny) + std::log10((double)S);
                c.evalue = 0;
                cand.push_back(c);
                int64_t hb = c.key >> 31;
                hist[hb > (int64_t)H - 1 ? H - 1 : hb]++;
            }
        }
        std::sort(cand.begin(), cand.end(), [](const OrPsm& x, const OrPsm& y) {
            if (x.key != y.key) return x.key > y.key;
            return x.pid < y.pid;
        });
        std::vector<OrPsm> top(K);
        for (uint32_t r = 0; r < K; ++r) {
            if (r < cand.size()) top[r] = cand[r];
            else { top[r].pid = UINT32_MAX; top[r].nb = top[r].ny = top[r].S = 0;
                   top[r].key = INT64_MIN; top[r].hyperscore = 0; top[r].evalue = INFINITY; }
        }
        std::vector<double> ev;
        evalues(hist, H, top, p.evalue_mode, ev);
        for (uint32_t r = 0; r < K; ++r) { top[r].evalue = ev[r]; out_psm[(uint64_t)si * K + r] = top[r]; }
        out_nscored[si] = (uint32_t)cand.size();
        if (out_lo) out_lo[si] = lo;
        if (out_hi) out_hi[si] = hi;
    }
}

void or_search(void* h, const uint64_t* peak_off, const float* mz, const float* inten,
               const double* prec_mz, const uint8_t* charge, const double* tol,
               const uint32_t* sel, uint32_t n_sel,
               OrPsm* out_psm, uint32_t* out_hist, uint32_t* out_nscored,
               uint32_t* out_lo, uint32_t* out_hi) {
    or_search_shard(h, peak_off, mz, inten, prec_mz, charge, tol, sel, n_sel, out_psm, out_hist, out_nscored,
                    out_lo, out_hi, 1, 0);
}

}  // extern "C"
