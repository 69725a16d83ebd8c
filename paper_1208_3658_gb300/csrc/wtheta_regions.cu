// Region-pair counts and the jackknife of w(theta).
//
// Sec. 4 of the paper points at error estimates from many realisations of a
// survey.  The delete-one jackknife draws them from the survey itself: the
// footprint is cut into R regions, and sample k is the survey without region
// k.  Every pair that sample k keeps is a pair between two regions other
// than k, so the counts of all samples follow from the counts of every
// region pair:
//   DD_{-k} = DD - sum_b DD[k, b]              (both orders of the pair
//   RR_{-k} likewise,                           folded into a <= b)
//   DR_{-k} = DR - sum_b DR[k, b] - sum_a DR[a, k] + DR[k, k].
// The region-pair counts come from one persistent launch: each catalogue is
// sorted by (region, spatial key) and every region starts on a tile
// boundary, so a tile pair lies in one region pair, and a count of the
// launch is one region pair (its own range of tile pairs and its own K+2
// slots).  Tile pairs beyond the top edge are skipped as in a single count.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <limits>
#include <vector>

#include "wtheta_internal.h"

using namespace wtheta;

namespace {

struct RegionLayout {
    std::vector<long long> n;        // points per region
    std::vector<long long> src;      // R+1: sorted positions of each region
    std::vector<long long> dst;      // R+1: padded positions (tile-aligned)
};

RegionLayout layout_of(const std::vector<unsigned long long>& sizes, long long T) {
    RegionLayout L;
    const int R = (int)sizes.size();
    L.n.resize(R);
    L.src.assign(R + 1, 0);
    L.dst.assign(R + 1, 0);
    for (int r = 0; r < R; ++r) {
        L.n[r] = (long long)sizes[r];
        L.src[r + 1] = L.src[r] + L.n[r];
        L.dst[r + 1] = L.dst[r] + round_up(L.n[r], T);
    }
    return L;
}

int count_regions_impl(const double* cd, long long nd, const int* ld, const double* cr,
                       long long nr, const int* lr, int is_xyz, const double* edges, int K,
                       int R, unsigned long long* counts, long long* sizes_out,
                       cudaStream_t st) {
    TraceRange trace("wtheta_count_regions");
    if (!counts || !sizes_out || nd < 0 || nr < 0 || R < 1 || R > 256 ||
        (nd > 0 && (!cd || !ld)) || (nr > 0 && (!cr || !lr)))
        return WTHETA_EINVAL;
    BinTable tab;
    int rc = build_table(edges, K, &tab);
    if (rc) return rc;
    DeviceInfo di;
    if ((rc = device_info(&di))) return rc;
    const Variant* v = pick_variant(nullptr, K, tab.n_lut, di.max_smem_optin);
    if (!v) return WTHETA_EINVAL;
    const long long T = (long long)v->nt * v->r;
    const size_t K2 = (size_t)K + 2;
    const size_t out_bytes = (size_t)3 * R * R * K2 * 8;
    if ((rc = check_cuda(cudaMemsetAsync(counts, 0, out_bytes, st)))) return rc;

    // phase 1: FP64 unit vectors, order by (region, key), region sizes
    const long long n_of[2] = {nd, nr};
    const double* c_of[2] = {cd, cr};
    const int* l_of[2] = {ld, lr};
    size_t b1 = 256 + ((size_t)2 * R * 8 + 255) / 256 * 256;
    size_t off_x[2], off_sort[2];
    for (int c = 0; c < 2; ++c) {
        off_x[c] = b1;
        if (!is_xyz) b1 += ((size_t)n_of[c] * 24 + 255) / 256 * 256;
        off_sort[c] = b1;
        b1 += order_bytes(n_of[c], 1);
    }
    unsigned char* m1 = nullptr;
    if ((rc = dev_malloc_async((void**)&m1, b1, st))) return rc;
    unsigned long long* d_sizes = (unsigned long long*)(m1 + 256);
    const double* x64[2];
    const unsigned* order[2] = {nullptr, nullptr};
    const unsigned* slab[2] = {nullptr, nullptr};
    rc = check_cuda(cudaMemsetAsync(d_sizes, 0, (size_t)2 * R * 8, st));
    for (int c = 0; c < 2 && !rc; ++c) {
        x64[c] = c_of[c];
        if (!is_xyz) {
            double* x = (double*)(m1 + off_x[c]);
            rc = launch_radec_to_xyz(c_of[c], n_of[c], x, di.sm_count, st);
            x64[c] = x;
        }
        if (!rc)
            rc = spatial_order(x64[c], n_of[c], n_of[c], is_xyz, l_of[c], R, m1 + off_sort[c],
                               di.sm_count, st, &order[c], &slab[c]);
        if (!rc && n_of[c] > 0)
            rc = launch_count_labels(slab[c], n_of[c], R, d_sizes + (size_t)c * R, di.sm_count, st);
    }
    std::vector<unsigned long long> hs(2 * (size_t)R, 0);
    if (!rc) rc = check_cuda(cudaMemcpyAsync(hs.data(), d_sizes, hs.size() * 8,
                                             cudaMemcpyDeviceToHost, st));
    if (!rc) rc = check_cuda(cudaStreamSynchronize(st));
    if (rc) {
        cudaFreeAsync(m1, st);
        return rc;
    }
    RegionLayout L[2] = {layout_of(std::vector<unsigned long long>(hs.begin(), hs.begin() + R), T),
                         layout_of(std::vector<unsigned long long>(hs.begin() + R, hs.end()), T)};
    for (int r = 0; r < R; ++r) {
        sizes_out[r] = L[0].n[r];
        sizes_out[R + r] = L[1].n[r];
    }

    // the region pairs of the three counts, biggest first
    struct Cnt { int kind, a, b; long long items; };
    std::vector<Cnt> cnts;
    for (int kind = 0; kind < 3; ++kind) {
        const RegionLayout& A = L[kind == 2 ? 1 : 0];
        const RegionLayout& B = L[kind == 0 ? 0 : 1];
        for (int a = 0; a < R; ++a)
            for (int b = (kind == 1 ? 0 : a); b < R; ++b) {
                const long long ta = (A.dst[a + 1] - A.dst[a]) / T;
                const long long tb = (B.dst[b + 1] - B.dst[b]) / T;
                const bool aut = kind != 1 && a == b;
                const long long items = aut ? ta * (ta + 1) / 2 : ta * tb;
                if (items > 0) cnts.push_back({kind, a, b, items});
            }
    }
    std::stable_sort(cnts.begin(), cnts.end(),
                     [](const Cnt& x, const Cnt& y) { return x.items > y.items; });
    long long total_items = 0;
    for (const Cnt& q : cnts) total_items += q.items;
    const bool cull = edges[K] < 180.0 && total_items > 0;
    const int n_segs = (int)cnts.size();

    // phase 2: region-aligned FP32 copies, caps, tables
    size_t b2 = 256;  // cursor, kept total
    const size_t off_segs = b2;
    b2 += ((size_t)std::max(n_segs, 1) * sizeof(Segment) + 255) / 256 * 256;
    const size_t off_cull = b2;
    b2 += ((size_t)std::max(n_segs, 1) * sizeof(CullSeg) + 255) / 256 * 256;
    const size_t off_kept = b2;
    b2 += ((size_t)std::max(n_segs, 1) * 8 + 255) / 256 * 256;
    const size_t off_off = b2;
    b2 += ((size_t)4 * (R + 1) * 8 + 255) / 256 * 256;
    size_t off_p32[2], off_c32[2], off_tc[2];
    for (int c = 0; c < 2; ++c) {
        const long long np = L[c].dst[R];
        off_p32[c] = b2;
        b2 += ((size_t)np * 16 + 255) / 256 * 256;
        off_c32[c] = b2;
        b2 += ((size_t)np / 32 * 16 + 255) / 256 * 256;
        off_tc[c] = b2;
        b2 += ((size_t)(np / T) * sizeof(TileCap) + 255) / 256 * 256;
    }
    const size_t off_lists = b2;
    b2 += (size_t)total_items * 4;
    unsigned char* m2 = nullptr;
    if ((rc = dev_malloc_async((void**)&m2, b2, st))) {
        cudaFreeAsync(m1, st);
        return rc;
    }
    unsigned long long* cursor = (unsigned long long*)m2;
    unsigned long long* n_kept = cursor + 1;
    Segment* d_segs = (Segment*)(m2 + off_segs);
    CullSeg* d_cull = (CullSeg*)(m2 + off_cull);
    unsigned long long* d_kept = (unsigned long long*)(m2 + off_kept);
    long long* d_off = (long long*)(m2 + off_off);
    std::vector<long long> h_off;
    for (int c = 0; c < 2; ++c) {
        h_off.insert(h_off.end(), L[c].src.begin(), L[c].src.end());
        h_off.insert(h_off.end(), L[c].dst.begin(), L[c].dst.end());
    }
    rc = check_cuda(cudaMemcpyAsync(d_off, h_off.data(), h_off.size() * 8,
                                    cudaMemcpyHostToDevice, st));
    Prepared P[2];
    TileCap* tcaps[2];
    for (int c = 0; c < 2 && !rc; ++c) {
        const long long np = L[c].dst[R];
        float4* p32 = (float4*)(m2 + off_p32[c]);
        float4* c32 = (float4*)(m2 + off_c32[c]);
        tcaps[c] = (TileCap*)(m2 + off_tc[c]);
        rc = launch_gather_regions(x64[c], n_of[c], order[c], d_off + (size_t)c * 2 * (R + 1),
                                   d_off + (size_t)c * 2 * (R + 1) + (R + 1), R, np, p32, c,
                                   di.sm_count, st);
        if (!rc) rc = launch_chunk_caps(p32, np, c32, di.sm_count, st);
        if (!rc && cull) rc = launch_tile_caps(p32, np, (int)T, np / T, tcaps[c], st);
        P[c].p32 = p32;
        P[c].c32 = c32;
        P[c].x64 = x64[c];
        P[c].stride = n_of[c];
    }
    std::vector<Segment> segs;
    std::vector<CullSeg> cs;
    long long item = 0;
    for (const Cnt& q : cnts) {
        const int ca = q.kind == 2 ? 1 : 0, cb = q.kind == 0 ? 0 : 1;
        const long long ta0 = L[ca].dst[q.a] / T, tb0 = L[cb].dst[q.b] / T;
        const long long ta = (L[ca].dst[q.a + 1] - L[ca].dst[q.a]) / T;
        const long long tb = (L[cb].dst[q.b + 1] - L[cb].dst[q.b]) / T;
        const bool aut = q.kind != 1 && q.a == q.b;
        Prepared A = P[ca], B = P[cb];
        A.p32 += ta0 * T;
        A.c32 += ta0 * T / 32;
        B.p32 += tb0 * T;
        B.c32 += tb0 * T / 32;
        const unsigned long long na = (unsigned long long)L[ca].n[q.a];
        const unsigned long long nb = (unsigned long long)L[cb].n[q.b];
        unsigned long long* c = counts + (((size_t)q.kind * R + q.a) * R + q.b) * K2;
        Segment g = make_segment(A, B, ta, aut ? ta : tb, aut ? 1 : 0, item, c,
                                 aut ? na * (na - 1) / 2 : na * nb);
        segs.push_back(g);
        CullSeg x;
        std::memset(&x, 0, sizeof(x));
        x.begin = item;
        x.n = q.items;
        x.ta = ta;
        x.tb = aut ? ta : tb;
        x.is_auto = aut ? 1 : 0;
        if (cull) {
            x.ca = tcaps[ca] + ta0;
            x.cb = tcaps[cb] + tb0;
            x.list = (unsigned*)(m2 + off_lists) + item;
        }
        cs.push_back(x);
        item += q.items;
    }
    if (!rc && n_segs > 0) {
        rc = check_cuda(cudaMemcpyAsync(d_segs, segs.data(), sizeof(Segment) * segs.size(),
                                        cudaMemcpyHostToDevice, st));
        if (!rc && cull)
            rc = check_cuda(cudaMemcpyAsync(d_cull, cs.data(), sizeof(CullSeg) * cs.size(),
                                            cudaMemcpyHostToDevice, st));
        if (!rc) rc = check_cuda(cudaMemsetAsync(m2, 0, 16, st));
        if (!rc && cull) rc = check_cuda(cudaMemsetAsync(d_kept, 0, (size_t)n_segs * 8, st));
        if (!rc && cull)
            rc = launch_cull_batch(d_cull, n_segs, total_items, edges[K] * (3.14159265358979323846 / 180.0), d_kept,
                                   d_segs, n_kept, di.sm_count, st);
        const size_t smem = v->smem(K, tab.n_lut);
        int grid = 0;
        if (!rc) rc = grid_for(v, smem, total_items, di.sm_count, 0, &grid);
        if (!rc) {
            PairParams prm = make_params(v, tab, nullptr, d_segs, n_segs, 0, total_items, cursor,
                                         nullptr);
            if (cull) prm.n_items_dev = n_kept;
            rc = launch_pairs(v, prm, grid, smem, st);
        }
        if (!rc) rc = launch_finalize_segments(d_segs, n_segs, K, st);
    }
    const cudaError_t f2 = cudaFreeAsync(m2, st);
    const cudaError_t f1 = cudaFreeAsync(m1, st);
    if (!rc) rc = check_cuda(f2);
    if (!rc) rc = check_cuda(f1);
    return rc;
}

// Landy-Szalay with normalised counts for one sample (slots 1..K of K+2).
void ls_of(const double* DD, const double* DR, const double* RR, double nd, double nr, int K,
           double* w) {
    const double Ndd = nd * (nd - 1.0) / 2.0, Ndr = nd * nr, Nrr = nr * (nr - 1.0) / 2.0;
    for (int k = 1; k <= K; ++k) {
        const double dd = DD[k] / Ndd, dr = DR[k] / Ndr, rr = RR[k] / Nrr;
        w[k - 1] = ((dd - 2.0 * dr) + rr) / rr;
    }
}

}  // namespace

extern "C" {

int wtheta_count_regions(const double* coords_d, int64_t n_d, const int32_t* labels_d,
                         const double* coords_r, int64_t n_r, const int32_t* labels_r,
                         int32_t coords_are_xyz, const double* bin_edges_deg, int32_t n_bins,
                         int32_t n_regions, uint64_t* counts, int64_t* region_sizes,
                         void* stream) {
    if (coords_are_xyz != 0 && coords_are_xyz != 1) return WTHETA_EINVAL;
    return count_regions_impl(coords_d, n_d, labels_d, coords_r, n_r, labels_r, coords_are_xyz,
                              bin_edges_deg, n_bins, n_regions, (unsigned long long*)counts,
                              (long long*)region_sizes, (cudaStream_t)stream);
}

int wtheta_jackknife(const uint64_t* counts, const int64_t* sizes, int32_t R, int32_t K,
                     double* w, double* w_jk, double* cov) {
    if (!counts || !sizes || !w || !w_jk || !cov || R < 2 || R > 256 || K < 1 || K > kMaxBins)
        return WTHETA_EINVAL;
    const size_t K2 = (size_t)K + 2;
    auto at = [&](int kind, int a, int b) { return counts + (((size_t)kind * R + a) * R + b) * K2; };
    // totals and the pairs that touch each region, per slot
    std::vector<double> tot(3 * K2, 0.0), touch((size_t)3 * R * K2, 0.0);
    long long nd = 0, nr = 0;
    for (int r = 0; r < R; ++r) {
        if (sizes[r] < 0 || sizes[R + r] < 0) return WTHETA_EINVAL;
        nd += sizes[r];
        nr += sizes[R + r];
    }
    for (int kind = 0; kind < 3; ++kind)
        for (int a = 0; a < R; ++a)
            for (int b = 0; b < R; ++b) {
                if (kind != 1 && b < a) continue;
                const uint64_t* c = at(kind, a, b);
                for (size_t k = 0; k < K2; ++k) {
                    const double v = (double)c[k];
                    tot[kind * K2 + k] += v;
                    touch[((size_t)kind * R + a) * K2 + k] += v;
                    if (b != a) touch[((size_t)kind * R + b) * K2 + k] += v;
                }
            }
    ls_of(&tot[0], &tot[K2], &tot[2 * K2], (double)nd, (double)nr, K, w);
    std::vector<double> s(3 * K2);
    for (int r = 0; r < R; ++r) {
        for (int kind = 0; kind < 3; ++kind)
            for (size_t k = 0; k < K2; ++k)
                s[kind * K2 + k] = tot[kind * K2 + k] - touch[((size_t)kind * R + r) * K2 + k];
        ls_of(&s[0], &s[K2], &s[2 * K2], (double)(nd - sizes[r]), (double)(nr - sizes[R + r]), K,
              w_jk + (size_t)r * K);
    }
    // covariance: (R-1)/R sum_r (w_r - mean)(w_r - mean)^T
    std::vector<double> mean(K, 0.0);
    for (int r = 0; r < R; ++r)
        for (int k = 0; k < K; ++k) mean[k] += w_jk[(size_t)r * K + k];
    for (int k = 0; k < K; ++k) mean[k] /= (double)R;
    for (int i = 0; i < K; ++i)
        for (int j = 0; j < K; ++j) {
            double acc = 0.0;
            for (int r = 0; r < R; ++r)
                acc += (w_jk[(size_t)r * K + i] - mean[i]) * (w_jk[(size_t)r * K + j] - mean[j]);
            cov[(size_t)i * K + j] = acc * (double)(R - 1) / (double)R;
        }
    return WTHETA_OK;
}

}  // extern "C"
