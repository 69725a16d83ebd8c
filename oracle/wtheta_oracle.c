/*
 * CPU oracle for exact angular pair counts and the Landy-Szalay w(theta).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the CPU
 * baseline leg of the benchmark call this code.  The library under test never
 * links, loads or calls it, and this file shares no code with the library.
 *
 * It is the plain definition, evaluated pair by pair in IEEE FP64:
 *   - unit vectors from RA/Dec (App. A gives theta from alpha, delta; the unit
 *     vector is the same geometry without the arctan);
 *   - squared chord s = |a - b|^2, a monotone function of the angle theta on
 *     [0, 180] deg (s = 4 sin^2(theta/2)), so binning s against the squared
 *     chords of the degree edges bins theta;
 *   - bins half-open [e_{k-1}, e_k), with an underflow slot (theta < e_0) and
 *     an overflow slot (theta >= e_K) so that every pair lands somewhere;
 *   - auto counts take every unordered pair i < j once, no self pairs, giving
 *     n(n-1)/2 pairs; cross counts take all n_a * n_b ordered pairs (Sec. 2);
 *   - the estimator of Eq. 2 with each count divided by its pair total
 *     (Sec. 2 gives the totals n(n-1)/2 and n*n_r).
 *
 * Build with -ffp-contract=off: every multiply and add rounds separately, in
 * the order written.  Each count is one FP64 predicate per pair; there is no
 * blocking or reordering.  Threads own interleaved rows and private histograms
 * that are summed at the end (integer sums, order independent).
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <unistd.h>

#define ORC_PI 3.14159265358979323846

int orc_num_threads(void) {
    long n = sysconf(_SC_NPROCESSORS_ONLN);
    return n > 0 ? (int)n : 1;
}

/* Bin edges in degrees (Sec. 2.1: user-set low and high limits; evenly spaced,
 * natural-log or base-10-log bins).  Both logarithmic modes give geometric
 * edges e_k = lo * (hi/lo)^(k/K); the base only names the width. */
int orc_edges(double lo, double hi, int K, int mode, double* e) {
    if (K < 1 || !(lo >= 0.0) || !(hi > lo) || !(hi <= 180.0)) return -1;
    if (mode != 0 && !(lo > 0.0)) return -1;
    for (int k = 0; k <= K; ++k) {
        if (mode == 0) {
            e[k] = lo + (double)k * ((hi - lo) / (double)K);
        } else if (mode == 1) {
            e[k] = lo * exp((double)k * (log(hi / lo) / (double)K));
        } else if (mode == 2) {
            e[k] = lo * pow(10.0, (double)k * (log10(hi / lo) / (double)K));
        } else {
            return -1;
        }
    }
    e[0] = lo;
    e[K] = hi;
    return 0;
}

/* Squared chord of each degree edge: c = (2 sin(theta/2))^2 = 4 h h. */
void orc_chord2(const double* e, int K, double* c) {
    for (int k = 0; k <= K; ++k) {
        double h = sin(e[k] * (ORC_PI / 360.0));
        c[k] = 4.0 * h * h;
    }
}

/* RA/Dec (degrees, interleaved) -> unit vectors, SoA: x[0..n), y[0..n), z[0..n). */
void orc_radec_to_xyz(const double* ra_dec, int64_t n, double* xyz) {
    for (int64_t i = 0; i < n; ++i) {
        double a = ra_dec[2 * i] * (ORC_PI / 180.0);
        double d = ra_dec[2 * i + 1] * (ORC_PI / 180.0);
        xyz[i] = cos(d) * cos(a);
        xyz[n + i] = cos(d) * sin(a);
        xyz[2 * n + i] = sin(d);
    }
}

/* The pair predicate: squared chord, evaluated ((dx*dx + dy*dy) + dz*dz). */
static double pair_s(const double* A, int64_t na, int64_t i,
                     const double* B, int64_t nb, int64_t j) {
    double dx = A[i] - B[j];
    double dy = A[na + i] - B[nb + j];
    double dz = A[2 * na + i] - B[2 * nb + j];
    return ((dx * dx) + (dy * dy)) + (dz * dz);
}

/* Slot of s: the number of edges c_k with c_k <= s (0 = underflow, K+1 = overflow). */
static int slot_of(double s, const double* c, int K) {
    if (s >= c[K]) return K + 1;
    int k = 0;
    while (k <= K && c[k] <= s) ++k;
    return k;
}

typedef struct {
    const double *A, *B, *c, *tau;
    int64_t na, nb;
    int K, is_auto, tid, nthreads;
    uint64_t* hist;     /* K+2 slots (count) or 1 slot (ambiguous count) */
} job_t;

static void* count_rows(void* p) {
    job_t* J = (job_t*)p;
    for (int64_t i = J->tid; i < J->na; i += J->nthreads) {
        int64_t j0 = J->is_auto ? i + 1 : 0;
        for (int64_t j = j0; j < J->nb; ++j) {
            double s = pair_s(J->A, J->na, i, J->B, J->nb, j);
            J->hist[slot_of(s, J->c, J->K)] += 1;
        }
    }
    return NULL;
}

static void* ambiguous_rows(void* p) {
    job_t* J = (job_t*)p;
    for (int64_t i = J->tid; i < J->na; i += J->nthreads) {
        int64_t j0 = J->is_auto ? i + 1 : 0;
        for (int64_t j = j0; j < J->nb; ++j) {
            double s = pair_s(J->A, J->na, i, J->B, J->nb, j);
            for (int k = 0; k <= J->K; ++k) {
                if (fabs(s - J->c[k]) <= J->tau[k]) { J->hist[0] += 1; break; }
            }
        }
    }
    return NULL;
}

static int run_jobs(void* (*fn)(void*), const double* A, int64_t na,
                    const double* B, int64_t nb, const double* c, const double* tau,
                    int K, int is_auto, int nslots, uint64_t* out, int nthreads) {
    if (nthreads <= 0) nthreads = orc_num_threads();
    job_t* jobs = (job_t*)calloc((size_t)nthreads, sizeof(job_t));
    pthread_t* th = (pthread_t*)calloc((size_t)nthreads, sizeof(pthread_t));
    uint64_t* hist = (uint64_t*)calloc((size_t)nthreads * (size_t)nslots, sizeof(uint64_t));
    if (!jobs || !th || !hist) { free(jobs); free(th); free(hist); return -2; }
    for (int t = 0; t < nthreads; ++t) {
        job_t j = {A, B, c, tau, na, nb, K, is_auto, t, nthreads, hist + (size_t)t * nslots};
        jobs[t] = j;
        pthread_create(&th[t], NULL, fn, &jobs[t]);
    }
    for (int s = 0; s < nslots; ++s) out[s] = 0;
    for (int t = 0; t < nthreads; ++t) {
        pthread_join(th[t], NULL);
        for (int s = 0; s < nslots; ++s) out[s] += hist[(size_t)t * nslots + s];
    }
    free(jobs); free(th); free(hist);
    return 0;
}

/* Exact pair counts.  xyz_a, xyz_b: SoA unit vectors.  For is_auto, B must be
 * A (same array, nb == na) and the unordered pairs i < j are counted.
 * counts: K+2 slots. */
int orc_count(const double* xyz_a, int64_t na, const double* xyz_b, int64_t nb,
              const double* c, int K, int is_auto, uint64_t* counts, int nthreads) {
    if (is_auto) { xyz_b = xyz_a; nb = na; }
    return run_jobs(count_rows, xyz_a, na, xyz_b, nb, c, NULL, K, is_auto, K + 2,
                    counts, nthreads);
}

/* Number of pairs whose s lies within tau_k of some edge c_k: the pairs whose
 * slot could change if the unit vectors moved by a few FP64 ulps. */
int orc_count_ambiguous(const double* xyz_a, int64_t na, const double* xyz_b, int64_t nb,
                        const double* c, const double* tau, int K, int is_auto,
                        uint64_t* out, int nthreads) {
    if (is_auto) { xyz_b = xyz_a; nb = na; }
    return run_jobs(ambiguous_rows, xyz_a, na, xyz_b, nb, c, tau, K, is_auto, 1,
                    out, nthreads);
}

/* Landy-Szalay, Eq. 2, each count normalised by its pair total:
 *   dd = DD/(n_d(n_d-1)/2), dr = DR/(n_d n_r), rr = RR/(n_r(n_r-1)/2),
 *   w = (dd - 2 dr + rr) / rr  for bins 1..K (slots 0 and K+1 are not bins);
 * NaN where RR_k = 0 (the estimator divides by it). */
int orc_ls(const uint64_t* DD, const uint64_t* DR, const uint64_t* RR,
           int64_t nd, int64_t nr, int K, double* w) {
    if (nd < 2 || nr < 2 || K < 1) return -1;
    double Ndd = (double)nd * (double)(nd - 1) / 2.0;
    double Ndr = (double)nd * (double)nr;
    double Nrr = (double)nr * (double)(nr - 1) / 2.0;
    for (int k = 1; k <= K; ++k) {
        double dd = (double)DD[k] / Ndd;
        double dr = (double)DR[k] / Ndr;
        double rr = (double)RR[k] / Nrr;
        /* no random pairs in the bin: Eq. 2 has no value there */
        w[k - 1] = RR[k] ? ((dd - 2.0 * dr) + rr) / rr : NAN;
    }
    return 0;
}

/* Cross-correlation form of the same estimator between catalogues 1 and 2:
 *   w = (d1d2 - d1r2 - r1d2 + r1r2) / r1r2, each count over its n_a n_b;
 * NaN where R1R2_k = 0. */
int orc_ls_cross(const uint64_t* D1D2, const uint64_t* D1R2, const uint64_t* R1D2,
                 const uint64_t* R1R2, int64_t nd1, int64_t nd2, int64_t nr1,
                 int64_t nr2, int K, double* w) {
    if (nd1 < 1 || nd2 < 1 || nr1 < 1 || nr2 < 1 || K < 1) return -1;
    for (int k = 1; k <= K; ++k) {
        double a = (double)D1D2[k] / ((double)nd1 * (double)nd2);
        double b = (double)D1R2[k] / ((double)nd1 * (double)nr2);
        double c = (double)R1D2[k] / ((double)nr1 * (double)nd2);
        double d = (double)R1R2[k] / ((double)nr1 * (double)nr2);
        w[k - 1] = R1R2[k] ? (((a - b) - c) + d) / d : NAN;
    }
    return 0;
}
