// Host-side parts of libwtheta: bin edges (Sec. 2.1), squared-chord edges
// (App. A geometry), the FP32 guard band and screening table used by the
// counting kernels, and the Landy-Szalay estimator (Eq. 2).
#include <cmath>
#include <limits>
#include <cstring>

#include "wtheta_internal.h"

namespace wtheta {

static const double kPi = 3.14159265358979323846;

int validate_edges(const double* e, int K) {
    if (!e || K < 1 || K > kMaxBins) return WTHETA_EINVAL;
    for (int k = 0; k <= K; ++k) {
        if (!std::isfinite(e[k]) || e[k] < 0.0 || e[k] > 180.0) return WTHETA_EINVAL;
        if (k > 0 && !(e[k] > e[k - 1])) return WTHETA_EINVAL;
    }
    return WTHETA_OK;
}

// c_k = (2 sin(theta_k / 2))^2, the squared chord between unit vectors at
// angle theta_k.  Evaluated as (4 h) h with h = sin(theta pi/360).
void chord2_edges(const double* e, int K, double* c) {
    for (int k = 0; k <= K; ++k) {
        const double h = std::sin(e[k] * (kPi / 360.0));
        c[k] = (4.0 * h) * h;
    }
}

// Half-width g(c) of the guard band around an FP32 edge.
//
// Let a, b be FP64 unit vectors, s = |a - b|^2 exactly, s64 its FP64
// evaluation (the truth predicate) and s32 the kernel's FP32 evaluation from
// a32 = fl32(a), b32 = fl32(b):  d_i = fl(a32_i - b32_i),
// s32 = fma(dz, dz, fma(dy, dy, dx * dx)).  With u = 2^-24:
//   |d_i - (a_i - b_i)| <= u(1+u)(|a_i| + |b_i|) + u |a_i - b_i|      (=: e_i)
//   sum 2|d_i| e_i      <= 4u(1+u) sqrt(s) + 2u s       (Cauchy-Schwarz,
//                                                        |a| = |b| = 1)
//   sum e_i^2           <= 12 u^2 (1+u)^2 + 3 u^2 s
//   so the exact sum of squares of the rounded d_i, S', has
//   |S' - s| <= E1(s) = 4u(1+u)sqrt(s) + 2us + 12u^2(1+u)^2 + 3u^2 s,
//   and three roundings of non-negative terms add gamma_3 (s + E1(s)),
//   gamma_3 = 3u / (1 - 3u).
// The truth s64 differs from s by at most 8 u64 s (u64 = 2^-53), and the FP32
// edge fl32(c) from c by u c.  If a pair's s32 is more than E + 8 u64 s + u c
// below (above) fl32(c), s64 is below (at or above) c.  Near an edge
// s <= s_b = 2c + 1e-12 (the bound holds for every c >= 0), so E, evaluated
// at s_b, is an upper bound there.  Absolute terms of 2^-146 cover subnormal
// rounding, and the total is doubled for margin.
double guard_half_width(double c) {
    const double u = 5.9604644775390625e-08;       // 2^-24
    const double u64 = 1.1102230246251565e-16;     // 2^-53
    const double tiny = 1.401298464324817e-45 * 8; // 2^-146
    const double sb = 2.0 * c + 1e-12;
    const double rs = std::sqrt(sb) * (1.0 + 1e-12);
    const double e1 = 4.0 * u * (1.0 + u) * rs + 2.0 * u * sb +
                      12.0 * u * u * (1.0 + u) * (1.0 + u) + 3.0 * u * u * sb;
    const double g3 = 3.0 * u / (1.0 - 3.0 * u);
    const double e32 = e1 + g3 * (sb + e1);
    const double e64 = 8.0 * u64 * sb;
    const double edge = u * c;
    return 2.0 * (e32 + e64 + edge + tiny);
}

static float round_down_f(double x) {
    float f = (float)x;
    if ((double)f > x) f = std::nextafter(f, -INFINITY);
    return f;
}

static float round_up_f(double x) {
    float f = (float)x;
    if ((double)f < x) f = std::nextafter(f, INFINITY);
    return f;
}

static uint32_t bits_of(float f) {
    uint32_t b;
    std::memcpy(&b, &f, 4);
    return b;
}

void guard_bounds(double c, uint32_t* lo_bits, uint32_t* hi_bits, double* g_out) {
    const double g = guard_half_width(c);
    const double c32 = (double)(float)c;
    const double lo = c32 - g, hi = c32 + g;
    *lo_bits = lo <= 0.0 ? 0u : bits_of(round_down_f(lo));
    *hi_bits = bits_of(round_up_f(hi));
    if (g_out) *g_out = g;
}

// Builds the screening table for an edge set.  Edges with c_k = 0 (only
// e_0 = 0 can give it) need no band: every s >= 0 is at or above them.
int build_table(const double* edges_deg, int K, BinTable* t) {
    int rc = validate_edges(edges_deg, K);
    if (rc) return rc;
    std::memset(t, 0, sizeof(*t));
    t->K = K;
    chord2_edges(edges_deg, K, t->c64);
    struct Band { uint32_t lo, hi; int k; };
    Band bands[kMaxBins + 1];
    size_t n_bands = 0;
    for (int k = 0; k <= K; ++k) {
        t->band[k][0] = t->band[k][1] = 0xFFFFFFFFu;
        if (t->c64[k] == 0.0) continue;
        Band b;
        guard_bounds(t->c64[k], &b.lo, &b.hi, nullptr);
        b.k = k;
        bands[n_bands++] = b;
        t->band[k][0] = b.lo;
        t->band[k][1] = b.hi;
    }
    // K >= 1 and the edges increase, so c_K > 0 and there is at least one band.
    t->h_top = bands[n_bands - 1].hi;
    const uint32_t lo_first = bands[0].lo;
    // the shift whose buckets holding several bands cover the least of the
    // range (their values go through a band search), the coarsest on ties
    int best_shift = -1;
    long long best_width = -1;
    for (int shift = 30; shift >= 0; --shift) {
        long long n = (long long)(t->h_top >> shift) - (long long)(lo_first >> shift) + 1;
        if (n > kMaxLut) break;
        // count buckets that meet more than one band
        int complex_buckets = 0;
        long long prev_bucket = -1;
        int prev_count = 0;
        for (size_t i = 0; i < n_bands; ++i) {
            const Band& b = bands[i];
            long long b0 = b.lo >> shift, b1 = b.hi >> shift;
            for (long long q = b0; q <= b1; ++q) {
                if (q == prev_bucket) {
                    if (++prev_count == 2) ++complex_buckets;
                } else {
                    prev_bucket = q;
                    prev_count = 1;
                }
            }
        }
        const long long width = (long long)complex_buckets << shift;
        if (best_width < 0 || width < best_width) {
            best_width = width;
            best_shift = shift;
        }
        if (complex_buckets == 0) break;
    }
    if (best_shift < 0) best_shift = 30;
    const int shift = best_shift;
    const long long base = lo_first >> shift;
    const long long top = t->h_top >> shift;
    t->shift = shift;
    t->base = (int32_t)base;
    t->n_lut = (int32_t)(top - base + 1);
    t->n_complex = 0;
    // slot below the first band: the number of edges with c = 0 (0 or 1)
    const int slot0 = bands[0].k;
    for (long long q = base; q <= top; ++q) {
        const uint32_t q_lo = (uint32_t)(q << shift);
        const uint32_t q_hi = (uint32_t)(((q + 1) << shift) - 1);
        int hits = 0, which = -1;
        int slot_before = slot0;
        for (size_t i = 0; i < n_bands; ++i) {
            if (bands[i].hi < q_lo) slot_before = bands[i].k + 1;
            if (bands[i].lo <= q_hi && bands[i].hi >= q_lo) {
                ++hits;
                if (which < 0) which = (int)i;
            }
        }
        uint32_t* e = t->lut[q - base];
        if (hits == 0) {
            e[0] = 0xFFFFFFFFu; e[1] = 0xFFFFFFFFu;
            e[2] = (uint32_t)slot_before; e[3] = (uint32_t)slot_before;
        } else if (hits == 1) {
            e[0] = bands[which].lo; e[1] = bands[which].hi;
            e[2] = (uint32_t)bands[which].k; e[3] = (uint32_t)(bands[which].k + 1);
        } else {
            // every in-range value of the bucket is placed by a search of the
            // bands (FP64 only inside one); one beyond the top edge (only the
            // top bucket can hold one) is overflow
            e[0] = 0u; e[1] = t->h_top;
            e[2] = (uint32_t)(K + 1); e[3] = (uint32_t)(K + 1);
            ++t->n_complex;
        }
    }
    return WTHETA_OK;
}

}  // namespace wtheta

using namespace wtheta;

extern "C" {

const char* wtheta_strerror(int status) {
    switch (status) {
        case WTHETA_OK: return "ok";
        case WTHETA_EINVAL: return "invalid argument";
        case WTHETA_ENOMEM: return "out of memory";
        case WTHETA_ECUDA: return "CUDA runtime error";
        case WTHETA_ETIMEOUT: return "bounded wait timed out";
        case WTHETA_EBUDGET: return "request exceeds the memory budget";
        case WTHETA_EDEVICE: return "device reported invalid input";
        case WTHETA_ESIZE: return "input larger than the entry point takes";
        case WTHETA_EBUSY: return "not in a state that allows the call";
        case WTHETA_ECANCELED: return "request cancelled";
        default: return "unknown status";
    }
}

int wtheta_edges(double lo, double hi, int32_t K, int32_t mode, double* e) {
    if (!e || K < 1 || K > kMaxBins) return WTHETA_EINVAL;
    if (!std::isfinite(lo) || !std::isfinite(hi) || !(lo >= 0.0) || !(hi > lo) || hi > 180.0)
        return WTHETA_EINVAL;
    if (mode != WTHETA_BINS_LINEAR && mode != WTHETA_BINS_LN && mode != WTHETA_BINS_LOG10)
        return WTHETA_EINVAL;
    if (mode != WTHETA_BINS_LINEAR && !(lo > 0.0)) return WTHETA_EINVAL;
    if (mode == WTHETA_BINS_LINEAR) {
        const double step = (hi - lo) / (double)K;
        for (int k = 0; k <= K; ++k) e[k] = lo + (double)k * step;
    } else if (mode == WTHETA_BINS_LN) {
        const double step = std::log(hi / lo) / (double)K;
        for (int k = 0; k <= K; ++k) e[k] = lo * std::exp((double)k * step);
    } else {
        const double step = std::log10(hi / lo) / (double)K;
        for (int k = 0; k <= K; ++k) e[k] = lo * std::pow(10.0, (double)k * step);
    }
    e[0] = lo;
    e[K] = hi;
    for (int k = 1; k <= K; ++k)
        if (!(e[k] > e[k - 1])) return WTHETA_EINVAL;
    return WTHETA_OK;
}

int wtheta_chord2_edges(const double* edges, int32_t K, double* c) {
    if (!c) return WTHETA_EINVAL;
    int rc = validate_edges(edges, K);
    if (rc) return rc;
    chord2_edges(edges, K, c);
    return WTHETA_OK;
}

int wtheta_guard_band(const double* edges, int32_t K, uint32_t* lo_bits, uint32_t* hi_bits,
                      double* half_width) {
    if (!lo_bits || !hi_bits) return WTHETA_EINVAL;
    int rc = validate_edges(edges, K);
    if (rc) return rc;
    double c[kMaxBins + 1];
    chord2_edges(edges, K, c);
    for (int k = 0; k <= K; ++k) {
        double g;
        guard_bounds(c[k], &lo_bits[k], &hi_bits[k], &g);
        if (half_width) half_width[k] = g;
    }
    return WTHETA_OK;
}

// Pairs (i, j) with first index i < r: cross r n_b; auto (i < j) r(n-1) - r(r-1)/2.
static unsigned long long pairs_before(long long r, long long n_a, long long n_b, int is_auto) {
    const unsigned long long R = (unsigned long long)r;
    if (!is_auto) return R * (unsigned long long)n_b;
    return R * (unsigned long long)(n_a - 1) - R * (R - 1) / 2;
}

int wtheta_shard_rows(int64_t n_a, int64_t n_b, int32_t is_auto, int32_t shard, int32_t n_shards,
                      int64_t* row_begin, int64_t* row_end) {
    if (!row_begin || !row_end || n_a < 0 || n_b < 0 || n_shards < 1 || shard < 0 ||
        shard >= n_shards || (is_auto != 0 && is_auto != 1))
        return WTHETA_EINVAL;
    const unsigned long long total = pairs_before(n_a, n_a, n_b, is_auto);
    // smallest row r with pairs_before(r) >= s * total / n_shards (exact integers)
    auto boundary = [&](int s) -> long long {
        if (s <= 0) return 0;
        if (s >= n_shards) return n_a;
        const unsigned long long target =
            (unsigned long long)((__int128)total * s / n_shards);
        long long lo = 0, hi = n_a;
        while (lo < hi) {
            const long long mid = lo + (hi - lo) / 2;
            if (pairs_before(mid, n_a, n_b, is_auto) >= target) hi = mid;
            else lo = mid + 1;
        }
        return lo;
    };
    *row_begin = boundary(shard);
    *row_end = boundary(shard + 1);
    return WTHETA_OK;
}

int wtheta_shard_weights(const uint64_t* weights, int64_t n_rows, int32_t shard,
                         int32_t n_shards, int64_t* row_begin, int64_t* row_end) {
    if (!row_begin || !row_end || n_rows < 0 || (n_rows > 0 && !weights) || n_shards < 1 ||
        shard < 0 || shard >= n_shards)
        return WTHETA_EINVAL;
    unsigned __int128 total = 0;
    for (int64_t r = 0; r < n_rows; ++r) total += weights[r];
    // boundary s: the smallest row r whose prefix weight reaches s / n_shards of
    // the total (rows split evenly by number when every weight is zero)
    auto boundary = [&](int s) -> long long {
        if (s <= 0) return 0;
        if (s >= n_shards) return n_rows;
        if (total == 0) return (long long)((__int128)n_rows * s / n_shards);
        const unsigned __int128 target = total * (unsigned)s;  // compared with prefix * n_shards
        unsigned __int128 prefix = 0;
        for (int64_t r = 0; r < n_rows; ++r) {
            if (prefix * (unsigned)n_shards >= target) return r;
            prefix += weights[r];
        }
        return n_rows;
    };
    *row_begin = boundary(shard);
    *row_end = boundary(shard + 1);
    return WTHETA_OK;
}

int wtheta_ls(const uint64_t* DD, const uint64_t* DR, const uint64_t* RR, int64_t nd,
              int64_t nr, int32_t K, double* w) {
    if (!DD || !DR || !RR || !w || K < 1 || K > kMaxBins || nd < 2 || nr < 2)
        return WTHETA_EINVAL;
    const double Ndd = (double)nd * (double)(nd - 1) / 2.0;
    const double Ndr = (double)nd * (double)nr;
    const double Nrr = (double)nr * (double)(nr - 1) / 2.0;
    for (int k = 1; k <= K; ++k) {
        const double dd = (double)DD[k] / Ndd;
        const double dr = (double)DR[k] / Ndr;
        const double rr = (double)RR[k] / Nrr;
        // Eq. 2 divides by the random pairs of the bin: none, no estimate
        w[k - 1] = RR[k] ? ((dd - 2.0 * dr) + rr) / rr : std::numeric_limits<double>::quiet_NaN();
    }
    return WTHETA_OK;
}

int wtheta_estimate(const uint64_t* DD, const uint64_t* DR, const uint64_t* RR, int64_t nd,
                    int64_t nr, int32_t K, int32_t est, double* w) {
    if (!DD || !DR || !RR || !w || K < 1 || K > kMaxBins || nd < 2 || nr < 2 || est < 0 ||
        est > WTHETA_EST_HAMILTON)
        return WTHETA_EINVAL;
    if (est == WTHETA_EST_LANDY_SZALAY) return wtheta_ls(DD, DR, RR, nd, nr, K, w);
    const double Ndd = (double)nd * (double)(nd - 1) / 2.0;
    const double Ndr = (double)nd * (double)nr;
    const double Nrr = (double)nr * (double)(nr - 1) / 2.0;
    const double nan = std::numeric_limits<double>::quiet_NaN();
    for (int k = 1; k <= K; ++k) {
        const double dd = (double)DD[k] / Ndd;
        const double dr = (double)DR[k] / Ndr;
        const double rr = (double)RR[k] / Nrr;
        double v;
        if (est == WTHETA_EST_NATURAL) v = RR[k] ? dd / rr - 1.0 : nan;
        else if (est == WTHETA_EST_DAVIS_PEEBLES) v = DR[k] ? dd / dr - 1.0 : nan;
        else v = DR[k] ? (dd * rr) / (dr * dr) - 1.0 : nan;
        w[k - 1] = v;
    }
    return WTHETA_OK;
}

int wtheta_ls_cross(const uint64_t* D1D2, const uint64_t* D1R2, const uint64_t* R1D2,
                    const uint64_t* R1R2, int64_t nd1, int64_t nd2, int64_t nr1, int64_t nr2,
                    int32_t K, double* w) {
    if (!D1D2 || !D1R2 || !R1D2 || !R1R2 || !w || K < 1 || K > kMaxBins || nd1 < 1 ||
        nd2 < 1 || nr1 < 1 || nr2 < 1)
        return WTHETA_EINVAL;
    for (int k = 1; k <= K; ++k) {
        const double a = (double)D1D2[k] / ((double)nd1 * (double)nd2);
        const double b = (double)D1R2[k] / ((double)nd1 * (double)nr2);
        const double c = (double)R1D2[k] / ((double)nr1 * (double)nd2);
        const double d = (double)R1R2[k] / ((double)nr1 * (double)nr2);
        w[k - 1] = R1R2[k] ? (((a - b) - c) + d) / d : std::numeric_limits<double>::quiet_NaN();
    }
    return WTHETA_OK;
}

}  // extern "C"
