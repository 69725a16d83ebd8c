// Pair-count kernels of libwtheta and the entry points that launch them.
//
// The computation is Sec. 2 of arXiv:1208.3658: every pair's angular
// separation (App. A) is binned (Sec. 2.1); auto counts take each unordered
// pair i < j once, cross counts every (i, j).  The paper splits the pair
// matrix into sub-matrices, one kernel launch each, with per-block shared
// histograms summed on the host.  Here one persistent launch walks the whole
// (triangular or rectangular) space of tile pairs from a device work cursor:
//   - RA/Dec -> FP64 unit vectors once per point (kept in the caller's order
//     for the rare FP64 recheck);
//   - the points are put in spatial order (cube-map face, then a Hilbert curve
//     on the face; a radix sort of 31-bit keys) so that a tile of consecutive
//     points is a compact patch of sky and a warp's pairs mostly share one
//     fate (all beyond the top edge, or all in range);
//   - tile pairs whose bounding caps lie wholly beyond the top edge are
//     skipped (their pairs are overflow); inside a tile pair, a thread's group
//     of R consecutive A points and a chunk of 32 B points are settled in one
//     slot, or by one FP32 comparison per pair against a single edge, when
//     their bounding spheres allow it;
//   - FP32 float4 copies (x, y, z, original index) padded to whole tiles with
//     far-away sentinel points that never land in a bin;
//   - a CTA stages the B tile in shared memory, negated and duplicated for
//     packed FP32x2 arithmetic, and keeps R A points per thread in registers;
//     the squared chord of two pairs costs 3 add.f32x2 + 1 mul.f32x2 +
//     2 fma.f32x2, i.e. the 6 FP32 operations per pair in half the issue slots;
//   - s is screened against the top edge: pairs beyond it are overflow and
//     cost nothing more (Sec. 2.2: separations outside the bin range can be
//     skipped); the overflow slot is filled at the end as total minus the rest;
//   - in-range pairs are binned by a table lookup on the bits of s, the FP32
//     comparison being final outside a rigorous guard band around each edge;
//     inside it the pair is recomputed in FP64 exactly as the definition says;
//   - counts go to private per-thread (or per-warp, warp-aggregated) uint32
//     shared histograms, flushed into uint64 global counts before any can wrap.
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstring>
#include <mutex>

#include "wtheta_internal.h"

namespace wtheta {

// ---------------------------------------------------------------------------
// device error word and helpers
// ---------------------------------------------------------------------------
__device__ unsigned int g_device_error;

static std::atomic<unsigned long long> g_launches{0};
static inline void count_launch(unsigned n = 1) { g_launches.fetch_add(n, std::memory_order_relaxed); }

static constexpr float kSentinel = 1.0e10f;  // sentinel offset; (1e10)^2 >> 4

__host__ __device__ constexpr int ilog2(int x) { return x <= 1 ? 0 : 1 + ilog2(x / 2); }

__device__ __forceinline__ float min3f(float a, float b, float c) {
    float d;
    asm("min.f32 %0, %1, %2, %3;" : "=f"(d) : "f"(a), "f"(b), "f"(c));
    return d;
}

// two FP32 values packed in one 64-bit register, for the sm_100-family
// packed FP32x2 instructions (each lane rounds exactly like its scalar op)
typedef unsigned long long f2_t;
__device__ __forceinline__ f2_t pack2(float lo, float hi) {
    f2_t r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
    return r;
}
__device__ __forceinline__ void unpack2(f2_t v, float& lo, float& hi) {
    asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(v));
}
__device__ __forceinline__ f2_t add2(f2_t a, f2_t b) {
    f2_t r;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}
__device__ __forceinline__ f2_t mul2(f2_t a, f2_t b) {
    f2_t r;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}
__device__ __forceinline__ f2_t fma2(f2_t a, f2_t b, f2_t c) {
    f2_t r;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r) : "l"(a), "l"(b), "l"(c));
    return r;
}

// Shared-memory accesses of the hot loops, through 32-bit shared-window
// addresses (so no generic 64-bit address arithmetic on the way).
__device__ __forceinline__ unsigned smem_addr(const void* p) {
    return (unsigned)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void lds_f2x2(unsigned a, f2_t& x, f2_t& y) {
    asm volatile("ld.shared.v2.b64 {%0, %1}, [%2];" : "=l"(x), "=l"(y) : "r"(a));
}
__device__ __forceinline__ f2_t lds_f2(unsigned a) {
    f2_t z;
    asm volatile("ld.shared.b64 %0, [%1];" : "=l"(z) : "r"(a));
    return z;
}
__device__ __forceinline__ uint4 lds_u4(unsigned a) {
    uint4 v;
    asm volatile("ld.shared.v4.b32 {%0, %1, %2, %3}, [%4];"
                 : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w) : "r"(a));
    return v;
}
__device__ __forceinline__ double lds_f64(unsigned a) {
    double v;
    asm volatile("ld.shared.f64 %0, [%1];" : "=d"(v) : "r"(a));
    return v;
}
__device__ __forceinline__ long long lds_s64(unsigned a) {
    long long v;
    asm volatile("ld.shared.b64 %0, [%1];" : "=l"(v) : "r"(a));
    return v;
}
__device__ __forceinline__ unsigned lds_u32(unsigned a) {
    unsigned v;
    asm volatile("ld.shared.b32 %0, [%1];" : "=r"(v) : "r"(a) : "memory");
    return v;
}
__device__ __forceinline__ void sts_u32(unsigned a, unsigned v) {
    asm volatile("st.shared.b32 [%0], %1;" :: "r"(a), "r"(v) : "memory");
}
__device__ __forceinline__ void red_add_shared(unsigned a, unsigned v) {
    asm volatile("red.shared.add.u32 [%0], %1;" :: "r"(a), "r"(v) : "memory");
}
__device__ __forceinline__ void inc_shared(unsigned a) {
    unsigned c;
    asm volatile("ld.shared.b32 %0, [%1];" : "=r"(c) : "r"(a) : "memory");
    asm volatile("st.shared.b32 [%0], %1;" :: "r"(a), "r"(c + 1u) : "memory");
}

// ---------------------------------------------------------------------------
// conversion kernels
// ---------------------------------------------------------------------------
__device__ __forceinline__ void radec_unit(double ra, double dec, double& x, double& y, double& z) {
    const double d2r = 3.14159265358979323846 / 180.0;
    if (!isfinite(ra) || !isfinite(dec)) atomicOr(&g_device_error, WTHETA_DERR_NONFINITE);
    else if (fabs(dec) > 90.0) atomicOr(&g_device_error, WTHETA_DERR_DEC_RANGE);
    const double a = ra * d2r, d = dec * d2r;
    const double cd = cos(d), sd = sin(d), ca = cos(a), sa = sin(a);
    x = __dmul_rn(cd, ca);
    y = __dmul_rn(cd, sa);
    z = sd;
}

__device__ __forceinline__ void check_unit(double x, double y, double z) {
    if (!isfinite(x) || !isfinite(y) || !isfinite(z)) {
        atomicOr(&g_device_error, WTHETA_DERR_NONFINITE);
    } else {
        const double r2 = x * x + y * y + z * z;
        if (fabs(r2 - 1.0) > 1e-6) atomicOr(&g_device_error, WTHETA_DERR_NOT_UNIT);
    }
}

__device__ __forceinline__ float4 point32(double x, double y, double z, long long idx) {
    return make_float4(__double2float_rn(x), __double2float_rn(y), __double2float_rn(z),
                       __int_as_float((int)idx));
}

// Padding point k of catalogue tag t: far from the unit sphere and from the
// padding of any other tag, (+-S (k+1), S t, 0) with the sign of t's parity;
// its squared chord with anything else is at least S^2 >> 4, so it never
// lands in a bin.
__device__ __forceinline__ float4 sentinel32(int tag, long long k) {
    const float sign = (tag & 1) ? -1.f : 1.f;
    return make_float4(sign * kSentinel * (float)(k + 1), kSentinel * (float)tag, 0.f, 0.f);
}

// RA/Dec degrees -> FP64 unit vectors (SoA with stride xyz_stride).
__global__ void k_radec_to_xyz(const double* __restrict__ rd, long long n,
                               double* __restrict__ xyz, long long xyz_stride) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        double x, y, z;
        radec_unit(rd[2 * i], rd[2 * i + 1], x, y, z);
        xyz[i] = x;
        xyz[xyz_stride + i] = y;
        xyz[2 * xyz_stride + i] = z;
    }
}

// Caller's FP64 SoA unit vectors -> FP32 float4 copies in the same order
// (w = index), then sentinels up to n_pad.
__global__ void k_xyz_to_f32(const double* __restrict__ xyz, long long n, long long n_pad,
                             float4* __restrict__ p32, int tag) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n_pad;
         i += (long long)gridDim.x * blockDim.x) {
        if (i < n) {
            const double x = xyz[i], y = xyz[n + i], z = xyz[2 * n + i];
            check_unit(x, y, z);
            p32[i] = point32(x, y, z, i);
        } else {
            p32[i] = sentinel32(tag, i - n);
        }
    }
}

// ---------------------------------------------------------------------------
// spatial order: cube-map face + Hilbert index of a 2^L x 2^L grid on it
// ---------------------------------------------------------------------------
// Position along the Hilbert curve of cell (x, y) in an S x S grid (S a power
// of two): descend the quadrants from the largest, adding each quadrant's
// offset along the curve and reflecting/transposing the remaining coordinates
// into that quadrant's orientation.
__device__ __forceinline__ unsigned hilbert_index(unsigned S, unsigned x, unsigned y) {
    unsigned d = 0;
    for (unsigned h = S >> 1; h > 0; h >>= 1) {
        const unsigned rx = (x & h) ? 1u : 0u, ry = (y & h) ? 1u : 0u;
        d += h * h * ((3u * rx) ^ ry);
        if (ry == 0) {
            if (rx == 1) {
                x = S - 1 - x;
                y = S - 1 - y;
            }
            const unsigned t = x;
            x = y;
            y = t;
        }
    }
    return d;
}

__device__ __forceinline__ unsigned cell_key(double x, double y, double z, int L) {
    const double ax = fabs(x), ay = fabs(y), az = fabs(z);
    unsigned face;
    double u, v, m;
    if (ax >= ay && ax >= az) { face = x >= 0 ? 0u : 1u; u = y; v = z; m = ax; }
    else if (ay >= az)        { face = y >= 0 ? 2u : 3u; u = x; v = z; m = ay; }
    else                      { face = z >= 0 ? 4u : 5u; u = x; v = y; m = az; }
    const unsigned S = 1u << L;
    if (!(m > 0.0)) return face * S * S;  // not a unit vector; any cell will do
    const double fu = (u / m + 1.0) * 0.5 * (double)S, fv = (v / m + 1.0) * 0.5 * (double)S;
    const unsigned iu = (unsigned)fmin(fmax(fu, 0.0), (double)(S - 1));
    const unsigned iv = (unsigned)fmin(fmax(fv, 0.0), (double)(S - 1));
    return face * S * S + hilbert_index(S, iu, iv);
}

// Spatial order of a catalogue: a 31-bit key per point (cube-map face, then
// the Hilbert index of its cell on a 2^14 x 2^14 grid of the face, cells of
// about 20 arcsec), sorted by a stable least-significant-digit radix sort
// (4 passes of 8 bits: per-block digit counts, a scan of each digit's counts
// across the blocks, a stable scatter).  Consecutive points of the order are then close on the sky down
// to the scale of a few points, which the per-tile culling and the
// per-chunk settling of pairs both rely on.
constexpr int kSortLevel = 14;
constexpr int kSortThreads = 256;
// Rounds of 256 keys per block of the sort: enough blocks for about two per
// SM of a large GPU (at most 16 rounds), so that a small catalogue's passes
// are short, one round each, instead of a few blocks looping over 16 rounds.
static inline int sort_rounds(long long n) {
    const long long r = (n + 256LL * 304 - 1) / (256LL * 304);
    return (int)std::min<long long>(std::max<long long>(r, 1), 16);
}

__global__ void k_sort_keys(const double* __restrict__ xyz, long long stride, long long n,
                            int check, unsigned* __restrict__ key, unsigned* __restrict__ idx) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const double x = xyz[i], y = xyz[stride + i], z = xyz[2 * stride + i];
        if (check) check_unit(x, y, z);
        key[i] = cell_key(x, y, z, kSortLevel);
        idx[i] = (unsigned)i;
    }
}

// hist[d * n_blocks + b] = keys of block b whose digit is d.
__global__ void __launch_bounds__(kSortThreads) k_digit_hist(const unsigned* __restrict__ key,
                                                             long long n, int shift, int rounds,
                                                             unsigned* __restrict__ hist) {
    __shared__ unsigned cnt[256];
    const int t = threadIdx.x;
    cnt[t] = 0;
    __syncthreads();
    const long long tile = (long long)kSortThreads * rounds;
    const long long lo = blockIdx.x * tile, hi = min(lo + tile, n);
    for (long long i = lo + t; i < hi; i += kSortThreads) atomicAdd(&cnt[(key[i] >> shift) & 255u], 1u);
    __syncthreads();
    hist[(long long)t * gridDim.x + blockIdx.x] = cnt[t];
}

// Per digit d, the keys of digit d in blocks before b: hist[d * n_blocks + b]
// becomes that count (an exclusive scan along the digit's row, which is
// contiguous: coalesced), and tot[d] the digit's total.  One warp per digit,
// 8 digits per block of 256 threads.
__global__ void __launch_bounds__(256) k_digit_rows(unsigned* __restrict__ hist, int n_blocks,
                                                    unsigned* __restrict__ tot) {
    const int lane = threadIdx.x & 31;
    const int d = blockIdx.x * 8 + (threadIdx.x >> 5);
    unsigned* row = hist + (long long)d * n_blocks;
    unsigned run = 0;
#pragma unroll 4
    for (int b0 = 0; b0 < n_blocks; b0 += 32) {
        const int b = b0 + lane;
        const unsigned v = b < n_blocks ? row[b] : 0u;
        unsigned incl = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned u = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += u;
        }
        if (b < n_blocks) row[b] = run + incl - v;
        run += __shfl_sync(0xffffffffu, incl, 31);
    }
    if (lane == 0) tot[d] = run;
}

// Stable scatter of one pass: block b writes its keys of digit d from the
// keys of smaller digits (the exclusive scan of tot, done here by every
// block) plus rows[d * n_blocks + b] (k_digit_rows) on, in index order
// (rounds of 256 keys; inside a round, warps in order and lanes in order).
__global__ void __launch_bounds__(kSortThreads) k_digit_scatter(
    const unsigned* __restrict__ key_in, const unsigned* __restrict__ idx_in, long long n,
    int shift, int rounds, const unsigned* __restrict__ rows, const unsigned* __restrict__ tot,
    unsigned* __restrict__ key_out, unsigned* __restrict__ idx_out) {
    static_assert(kSortThreads == 256, "one thread per digit");
    __shared__ unsigned base[256];
    __shared__ unsigned wcnt[kSortThreads / 32][256];
    __shared__ unsigned wsum[kSortThreads / 32];
    const int t = threadIdx.x, lane = t & 31, w = t >> 5;
    {
        const unsigned x = tot[t];
        unsigned incl = x;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned u = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += u;
        }
        if (lane == 31) wsum[w] = incl;
        __syncthreads();
        unsigned pre = incl - x;
        for (int q = 0; q < w; ++q) pre += wsum[q];
        base[t] = pre + rows[(long long)t * gridDim.x + blockIdx.x];
    }
    const long long lo = blockIdx.x * (long long)kSortThreads * rounds;
    for (int r = 0; r < rounds; ++r) {
#pragma unroll
        for (int q = 0; q < kSortThreads / 32; ++q) wcnt[q][t] = 0;
        __syncthreads();
        const long long i = lo + (long long)r * kSortThreads + t;
        const bool valid = i < n;
        const unsigned k = valid ? key_in[i] : 0u;
        const unsigned d = valid ? (k >> shift) & 255u : 256u;
        const unsigned peers = __match_any_sync(0xffffffffu, d);
        const unsigned rank = __popc(peers & ((1u << lane) - 1u));
        if (valid && rank == 0) wcnt[w][d] = __popc(peers);
        __syncthreads();
        {
            unsigned acc = base[t];
#pragma unroll
            for (int q = 0; q < kSortThreads / 32; ++q) {
                const unsigned c = wcnt[q][t];
                wcnt[q][t] = acc;
                acc += c;
            }
            base[t] = acc;
        }
        __syncthreads();
        if (valid) {
            const unsigned pos = wcnt[w][d] + rank;
            key_out[pos] = k;
            idx_out[pos] = idx_in[i];
        }
        __syncthreads();
    }
}

// The one or two catalogues of a count, prepared together: both into one
// FP64 SoA array x (stride N = na + nb), converted from RA/Dec or copied from
// unit vectors (then checked), each point with its sort key (the cell key,
// with the catalogue in bit 31 so that b's points sort after a's) and its
// position.  FP64 work: launched in blocks of 64 threads, so that a small
// catalogue still spreads over every SM.
__global__ void __launch_bounds__(64) k_joint_keys(const double* __restrict__ a, long long na,
                                                   const double* __restrict__ b, long long nb,
                                                   int is_xyz, double* __restrict__ x,
                                                   unsigned* __restrict__ key,
                                                   unsigned* __restrict__ idx) {
    const long long N = na + nb;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N;
         i += (long long)gridDim.x * blockDim.x) {
        const bool in_b = i >= na;
        const double* src = in_b ? b : a;
        const long long j = in_b ? i - na : i, n = in_b ? nb : na;
        double px, py, pz;
        if (is_xyz) {
            px = src[j];
            py = src[n + j];
            pz = src[2 * n + j];
            check_unit(px, py, pz);
        } else {
            radec_unit(src[2 * j], src[2 * j + 1], px, py, pz);
        }
        x[i] = px;
        x[N + i] = py;
        x[2 * N + i] = pz;
        key[i] = cell_key(px, py, pz, kSortLevel) | (in_b ? 0x80000000u : 0u);
        idx[i] = (unsigned)i;
    }
}

// FP32 and FP64 copies of both catalogues in the joint order (order: the
// sorted positions of x, a's points first): a's at [0, na) with sentinels up
// to pa, b's at [pa, pa + nb) with sentinels up to pa + pb (tags tag0 and
// tag0 + 1); the FP64 copy has stride pa + pb, and each FP32 point keeps in w
// its index within its own catalogue.
__global__ void k_gather_joint(const double* __restrict__ x, long long na, long long pa,
                               long long nb, long long pb, const unsigned* __restrict__ order,
                               int tag0, float4* __restrict__ p32, double* __restrict__ s64) {
    const long long N = na + nb, P = pa + pb;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < P;
         i += (long long)gridDim.x * blockDim.x) {
        const bool in_b = i >= pa;
        const long long j = in_b ? i - pa : i, n = in_b ? nb : na;
        double px, py, pz;
        float4 q;
        if (j < n) {
            const long long k = order[(in_b ? na : 0) + j];
            px = x[k];
            py = x[N + k];
            pz = x[2 * N + k];
            q = point32(px, py, pz, in_b ? k - na : k);
        } else {
            q = sentinel32(tag0 + (in_b ? 1 : 0), j - n);
            px = q.x;
            py = q.y;
            pz = q.z;
        }
        p32[i] = q;
        s64[i] = px;
        s64[P + i] = py;
        s64[2 * P + i] = pz;
    }
}

// FP32 copies in sorted order (w = original index); slots n..n_pad-1 get
// sentinels.
__global__ void k_gather_points(const double* __restrict__ xyz, long long stride, long long n,
                                long long n_pad, const unsigned* __restrict__ order,
                                float4* __restrict__ p32, double* __restrict__ s64, int tag) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n_pad;
         i += (long long)gridDim.x * blockDim.x) {
        double x, y, z;
        float4 q;
        if (i < n) {
            const long long j = order[i];
            x = xyz[j];
            y = xyz[stride + j];
            z = xyz[2 * stride + j];
            q = point32(x, y, z, j);
        } else {
            q = sentinel32(tag, i - n);
            x = q.x;
            y = q.y;
            z = q.z;
        }
        p32[i] = q;
        s64[i] = x;
        s64[n_pad + i] = y;
        s64[2 * n_pad + i] = z;
    }
}

// Labels in sorted order (the digit of one more radix pass); a label outside
// [0, n_labels) sets WTHETA_DERR_LABEL and counts as 0.
__global__ void k_sorted_labels(const unsigned* __restrict__ order, const int* __restrict__ labels,
                                long long n, int n_labels, unsigned* __restrict__ out) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        int l = labels[order[i]];
        if (l < 0 || l >= n_labels) {
            atomicOr(&g_device_error, WTHETA_DERR_LABEL);
            l = 0;
        }
        out[i] = (unsigned)l;
    }
}

// sizes[l] = number of points with label l (labels sorted or not).
__global__ void k_count_labels(const unsigned* __restrict__ lab, long long n, int n_labels,
                               unsigned long long* __restrict__ sizes) {
    __shared__ unsigned c[256];
    for (int q = threadIdx.x; q < 256; q += blockDim.x) c[q] = 0;
    __syncthreads();
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x)
        atomicAdd(&c[lab[i] & 255u], 1u);
    __syncthreads();
    for (int q = threadIdx.x; q < n_labels; q += blockDim.x)
        if (c[q]) atomicAdd(sizes + q, (unsigned long long)c[q]);
}

// FP32 copies with every region starting on a tile boundary: region r's
// points (sorted positions src[r] .. src[r+1]-1) go to dst[r] .., the rest of
// its last tile holds sentinels.  dst[R] = n_pad.  A sentinel is numbered
// within its region (below the tile size) and tagged by its region and
// array, so that no two sentinels a count can pair coincide in FP32 (numbered
// by their position in a long array, sentinels more than 2^24 points in would
// round onto one another).
__global__ void k_gather_regions(const double* __restrict__ xyz, long long stride,
                                 const unsigned* __restrict__ order,
                                 const long long* __restrict__ src,
                                 const long long* __restrict__ dst, int R, long long n_pad,
                                 float4* __restrict__ p32, int tag) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n_pad;
         i += (long long)gridDim.x * blockDim.x) {
        int lo = 0, hi = R - 1;  // last region with dst <= i
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (dst[mid] <= i) lo = mid; else hi = mid - 1;
        }
        const long long j = i - dst[lo], n_lo = src[lo + 1] - src[lo];
        if (j < n_lo) {
            const long long k = order[src[lo] + j];
            p32[i] = point32(xyz[k], xyz[stride + k], xyz[2 * stride + k], k);
        } else {
            p32[i] = sentinel32(2 * lo + tag, j - n_lo);
        }
    }
}

// The catalogues of a batch into one FP64 SoA array (stride N) with a label
// per point (its catalogue): catalogue c's points go to positions
// [off[c], off[c + 1]), converted from RA/Dec or copied from unit vectors.
struct BatchCat {
    const double* src;   // interleaved RA/Dec degrees, or SoA unit vectors (3 n)
    long long n;
};
__global__ void k_batch_gather(const BatchCat* __restrict__ cats, const long long* __restrict__ off,
                               int n_cats, int is_xyz, long long N, double* __restrict__ x,
                               int* __restrict__ lab) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N;
         i += (long long)gridDim.x * blockDim.x) {
        int lo = 0, hi = n_cats - 1;  // last catalogue with off <= i
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (off[mid] <= i) lo = mid; else hi = mid - 1;
        }
        const BatchCat c = cats[lo];
        const long long j = i - off[lo];
        double px, py, pz;
        if (is_xyz) {
            px = c.src[j];
            py = c.src[c.n + j];
            pz = c.src[2 * c.n + j];
        } else {
            radec_unit(c.src[2 * j], c.src[2 * j + 1], px, py, pz);
        }
        x[i] = px;
        x[N + i] = py;
        x[2 * N + i] = pz;
        lab[i] = lo;
    }
}

// acc[k] += add[k] for the K+2 slots (combining two counts of one shard).
__global__ void k_add_counts(unsigned long long* acc, const unsigned long long* add, int n) {
    for (int k = threadIdx.x; k < n; k += blockDim.x) acc[k] += add[k];
}

// counts[K+1] = total - sum(counts[0..K]): the overflow slot.
__global__ void k_finalize(unsigned long long* counts, int K, unsigned long long total) {
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        unsigned long long s = 0;
        for (int k = 0; k <= K; ++k) s += counts[k];
        counts[K + 1] = total - s;
    }
}

// ---------------------------------------------------------------------------
// the pair-count kernel
// ---------------------------------------------------------------------------
// kHistLane: one private uint32 column per thread, plain read-modify-write;
// kHistWarp: one column per warp, lanes with equal slots merged by
//            __match_any_sync and added by one shared atomic;
// kHistLaneAtomic: one private column per thread, updated by a shared atomic
//            add (one instruction instead of load, add, store).


// Tile-pair index -> (I, J).  Auto: upper triangle I <= J, row-major.
__device__ __forceinline__ void item_to_tiles(long long t, long long T_a, long long T_b,
                                              int is_auto, long long* I, long long* J) {
    if (!is_auto) {
        *I = t / T_b;
        *J = t - *I * T_b;
        return;
    }
    const long long T = T_a;
    // rows 0..I-1 hold off(I) = I T - I (I - 1) / 2 items
    const double b = 2.0 * (double)T + 1.0;
    long long i = (long long)floor((b - sqrt(fmax(b * b - 8.0 * (double)t, 0.0))) * 0.5);
    if (i < 0) i = 0;
    if (i > T - 1) i = T - 1;
    while (i > 0 && i * T - i * (i - 1) / 2 > t) --i;
    while (i + 1 < T && (i + 1) * T - (i + 1) * i / 2 <= t) ++i;
    *I = i;
    *J = i + (t - (i * T - i * (i - 1) / 2));
}

// Bounding cap of each tile of T spatially ordered FP32 points (positions
// [0, n); padding sentinels, far off the unit sphere, are left out):
// centre = normalised FP64 sum, radius = the largest angle from the centre,
// plus 1e-6 rad for the FP32 rounding of the points (a point moves by at most
// ~1.1e-7 rad from its FP64 position).
__device__ __forceinline__ bool is_sentinel(const float4& q) {
    return q.x * q.x + q.y * q.y + q.z * q.z > 4.f;
}

__global__ void __launch_bounds__(128) k_tile_caps(const float4* __restrict__ p32, long long n,
                                                   int T, TileCap* __restrict__ caps) {
    __shared__ double red[4][4];
    __shared__ int cnt[4];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const long long t0 = (long long)blockIdx.x * T;
    const long long t1 = min(t0 + (long long)T, n);
    double sx = 0, sy = 0, sz = 0;
    int c = 0;
    for (long long i = t0 + tid; i < t1; i += blockDim.x) {
        const float4 q = p32[i];
        if (is_sentinel(q)) continue;
        sx += q.x; sy += q.y; sz += q.z;
        ++c;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        sx += __shfl_xor_sync(0xffffffffu, sx, o);
        sy += __shfl_xor_sync(0xffffffffu, sy, o);
        sz += __shfl_xor_sync(0xffffffffu, sz, o);
        c += __shfl_xor_sync(0xffffffffu, c, o);
    }
    if (lane == 0) { red[warp][0] = sx; red[warp][1] = sy; red[warp][2] = sz; cnt[warp] = c; }
    __syncthreads();
    sx = red[0][0] + red[1][0] + red[2][0] + red[3][0];
    sy = red[0][1] + red[1][1] + red[2][1] + red[3][1];
    sz = red[0][2] + red[1][2] + red[2][2] + red[3][2];
    c = cnt[0] + cnt[1] + cnt[2] + cnt[3];
    const double nrm = sqrt(sx * sx + sy * sy + sz * sz);
    const bool empty = c == 0;
    const bool spread = !(nrm > 1e-3 * (double)c);  // centre ill-defined: no skipping
    const double cx = spread ? 1.0 : sx / nrm, cy = spread ? 0.0 : sy / nrm,
                 cz = spread ? 0.0 : sz / nrm;
    double m = 0;
    for (long long i = t0 + tid; i < t1; i += blockDim.x) {
        const float4 q = p32[i];
        if (is_sentinel(q)) continue;
        const double dx = cx - q.x, dy = cy - q.y, dz = cz - q.z;
        m = fmax(m, dx * dx + dy * dy + dz * dz);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
    __syncthreads();
    if (lane == 0) red[warp][3] = m;
    __syncthreads();
    if (tid == 0) {
        m = fmax(fmax(red[0][3], red[1][3]), fmax(red[2][3], red[3][3]));
        TileCap cap;
        cap.x = cx; cap.y = cy; cap.z = cz;
        cap.rho = empty ? -1.0
                        : (spread ? 4.0 : 2.0 * asin(fmin(1.0, 0.5 * sqrt(m))) + 1e-6);
        caps[blockIdx.x] = cap;
    }
}

// Bounding sphere of every chunk of 32 consecutive spatially ordered FP32
// points: centre = the FP32 mean of the chunk's points, radius = the largest
// FP32 distance of a point from it, enlarged by a relative 1e-6 for the few
// roundings of that arithmetic.  A chunk holding a padding sentinel gets
// radius -1, so that its pairs are never settled per chunk.  One warp per
// chunk.
__global__ void k_chunk_caps(const float4* __restrict__ p32, long long n, long long n_pad,
                             float4* __restrict__ caps) {
    const int lane = threadIdx.x & 31;
    const long long n_chunks = n_pad / 32;
    const long long wpb = blockDim.x / 32;
    for (long long c = blockIdx.x * wpb + (threadIdx.x >> 5); c < n_chunks;
         c += (long long)gridDim.x * wpb) {
        const long long i = c * 32 + lane;
        const float4 q = p32[i];
        float sx = q.x, sy = q.y, sz = q.z;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            sx += __shfl_xor_sync(0xffffffffu, sx, o);
            sy += __shfl_xor_sync(0xffffffffu, sy, o);
            sz += __shfl_xor_sync(0xffffffffu, sz, o);
        }
        const float cx = sx * (1.f / 32), cy = sy * (1.f / 32), cz = sz * (1.f / 32);
        const float dx = q.x - cx, dy = q.y - cy, dz = q.z - cz;
        float m = dx * dx + dy * dy + dz * dz;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
        const bool pad = __any_sync(0xffffffffu, i >= n || is_sentinel(q));
        if (lane == 0) caps[c] = make_float4(cx, cy, cz, pad ? -1.f : sqrtf(m) * (1.f + 1e-6f));
    }
}

// Whether two tiles may hold a pair below the top edge theta_top (radians):
// their caps' centres are closer than theta_top + both radii (+ 3e-6 rad of
// slack for the FP64 arithmetic here).  Empty tiles hold no pair.
__device__ __forceinline__ bool caps_may_meet(const TileCap& A, const TileCap& B,
                                              double theta_top) {
    if (!(A.rho >= 0.0 && B.rho >= 0.0)) return false;
    const double dx = A.x - B.x, dy = A.y - B.y, dz = A.z - B.z;
    const double chord = sqrt(dx * dx + dy * dy + dz * dz);
    const double theta_c = 2.0 * asin(fmin(1.0, 0.5 * chord));
    return theta_c - A.rho - B.rho - 3e-6 <= theta_top;
}

// Keeps the tile pairs that may hold a pair below the top edge: those whose
// caps are closer than theta_top + margin.  The skipped ones hold only
// overflow pairs (and empty tiles none), which the overflow slot (total minus
// the other slots) accounts for; counts stay exact.  Kept items are appended
// in any order (the counts do not depend on it).
__global__ void k_cull_items(const TileCap* __restrict__ ca, const TileCap* __restrict__ cb,
                             long long tiles_a, long long tiles_b, int is_auto, long long n_items,
                             double theta_top, unsigned* __restrict__ list,
                             unsigned long long* __restrict__ n_list,
                             unsigned long long* __restrict__ stats) {
    const long long stride = (long long)gridDim.x * blockDim.x;
    const long long n_round = (n_items + 31) / 32 * 32;
    const int lane = threadIdx.x & 31;
    unsigned long long skipped = 0;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n_round; t += stride) {
        bool keep = false;
        if (t < n_items) {
            long long I, J;
            item_to_tiles(t, tiles_a, tiles_b, is_auto, &I, &J);
            keep = caps_may_meet(ca[I], cb[J], theta_top);
            skipped += keep ? 0 : 1;
        }
        const unsigned m = __ballot_sync(0xffffffffu, keep);
        unsigned long long base = 0;
        if (lane == 0 && m) base = atomicAdd(n_list, (unsigned long long)__popc(m));
        base = __shfl_sync(0xffffffffu, base, 0);
        if (keep) list[base + __popc(m & ((1u << lane) - 1u))] = (unsigned)t;
    }
    if (stats) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) skipped += __shfl_xor_sync(0xffffffffu, skipped, o);
        if (lane == 0 && skipped) atomicAdd(stats + WTHETA_STAT_SKIPPED, skipped);
    }
}

// The same skipping for a batch's work table.  cs holds every count's items
// in the full table (begin, n), its tiles' caps and its list; each kept
// item's index within its count is appended to that count's list (in any
// order), kept[seg] counting them.
__global__ void k_cull_batch(const CullSeg* __restrict__ cs, int n_segs, long long total,
                             double theta_top, unsigned long long* __restrict__ kept,
                             unsigned long long* __restrict__ stats) {
    const long long stride = (long long)gridDim.x * blockDim.x;
    const long long n_round = (total + 31) / 32 * 32;
    const int lane = threadIdx.x & 31;
    unsigned long long skipped = 0;
    for (long long g = blockIdx.x * (long long)blockDim.x + threadIdx.x; g < n_round; g += stride) {
        bool keep = false;
        int seg = -1;
        long long local = 0;
        if (g < total) {
            int lo = 0, hi = n_segs - 1;  // last count with begin <= g
            while (lo < hi) {
                const int mid = (lo + hi + 1) >> 1;
                if (cs[mid].begin <= g) lo = mid; else hi = mid - 1;
            }
            seg = lo;
            local = g - cs[seg].begin + cs[seg].offset;
            long long I, J;
            item_to_tiles(local, cs[seg].ta, cs[seg].tb, cs[seg].is_auto, &I, &J);
            keep = caps_may_meet(cs[seg].ca[I], cs[seg].cb[J], theta_top);
            skipped += keep ? 0 : 1;
        }
        const unsigned peers = __match_any_sync(0xffffffffu, keep ? seg : -1);
        const int leader = __ffs(peers) - 1;
        unsigned long long base = 0;
        if (keep && lane == leader) base = atomicAdd(kept + seg, (unsigned long long)__popc(peers));
        base = __shfl_sync(0xffffffffu, base, leader);
        if (keep) cs[seg].list[base + __popc(peers & ((1u << lane) - 1u))] = (unsigned)local;
    }
    if (stats) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) skipped += __shfl_xor_sync(0xffffffffu, skipped, o);
        if (lane == 0 && skipped) atomicAdd(stats + WTHETA_STAT_SKIPPED, skipped);
    }
}

// Kept tile pairs per tile row of every count (rows[cs_row0[seg] + I]), for
// splitting the rows of each count among shards by their work.
__global__ void k_cull_rows(const CullSeg* __restrict__ cs, int n_segs, long long total,
                            double theta_top, const long long* __restrict__ row0,
                            unsigned long long* __restrict__ rows) {
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long g = blockIdx.x * (long long)blockDim.x + threadIdx.x; g < total; g += stride) {
        int lo = 0, hi = n_segs - 1;  // last count with begin <= g
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (cs[mid].begin <= g) lo = mid; else hi = mid - 1;
        }
        const long long local = g - cs[lo].begin + cs[lo].offset;
        long long I, J;
        item_to_tiles(local, cs[lo].ta, cs[lo].tb, cs[lo].is_auto, &I, &J);
        if (caps_may_meet(cs[lo].ca[I], cs[lo].cb[J], theta_top)) atomicAdd(rows + row0[lo] + I, 1ull);
    }
}

// After k_cull_batch: each count's kept items become a contiguous range of
// the launch's items, in the table's order; *total receives their number.
__global__ void k_cull_prefix(Segment* __restrict__ segs, const CullSeg* __restrict__ cs,
                              const unsigned long long* __restrict__ kept, int n_segs,
                              unsigned long long* __restrict__ total) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    unsigned long long acc = 0;
    for (int i = 0; i < n_segs; ++i) {
        segs[i].item_begin = (long long)acc;
        segs[i].item_offset = 0;
        segs[i].item_list = cs[i].list;
        acc += kept[i];
    }
    *total = acc;
}

// FP64 recheck: the definition's squared chord and slot for the pair of
// sorted positions (ia, jb), read from the FP64 copies in the spatial order,
// or from the caller's FP64 arrays through the original indices kept in the
// FP32 copies (S.sorted64 says which); c64 is the shared address of
// the FP64 edges.  hint >= 0: the slot just below the one edge whose guard
// band held the FP32 value (checked, else the edges are searched in order).
__device__ __forceinline__ unsigned recheck_slot(const Segment& S, long long ia, long long jb,
                                                 unsigned c64, int K, int hint = -1) {
    const long long i = (S.sorted64 & 1) ? ia : __float_as_int(S.a32[ia].w);
    const long long j = (S.sorted64 & 2) ? jb : __float_as_int(S.b32[jb].w);
    const double* a = S.a64;
    const double* b = S.b64;
    const long long as = S.a64_stride, bs = S.b64_stride;
    const double dx = __dsub_rn(a[i], b[j]);
    const double dy = __dsub_rn(a[as + i], b[bs + j]);
    const double dz = __dsub_rn(a[2 * as + i], b[2 * bs + j]);
    const double s = __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz));
    if (hint >= 0 && hint <= K) {
        // the FP32 value lay in the guard band of edge `hint` alone: the slot
        // is hint or hint + 1, confirmed against the neighbouring edges
        if (s < lds_f64(c64 + 8u * (unsigned)hint)) {
            if (hint == 0 || lds_f64(c64 + 8u * (unsigned)(hint - 1)) <= s) return (unsigned)hint;
        } else if (hint == K || s < lds_f64(c64 + 8u * (unsigned)(hint + 1))) {
            return (unsigned)hint + 1u;
        }
    }
    // the number of edges at or below s, by bisection (K+1 = overflow)
    unsigned lo = 0, hi = (unsigned)K + 1;
    while (lo < hi) {
        const unsigned mid = (lo + hi) >> 1;
        if (lds_f64(c64 + 8u * mid) <= s) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}

template <int NT, int R, int JU, int HM, int DEF>
struct PairKernel {
    static constexpr int TA = NT * R;   // A points per tile
    static constexpr int TB = NT * R;   // B points per tile (equal: auto needs square tiles)
    static constexpr int NW = NT / 32;
    // columns of the private histograms (one per thread or per warp) and the
    // words from one slot's row to the next: per-warp columns updated by
    // shared reductions (kHistWarpRed) take an odd stride, so that lanes adding
    // to different rows of their warp's column hit different banks
    static constexpr int HCOLS = (HM == kHistWarp || HM == kHistWarpRed) ? NW : NT;
    static constexpr int HSTRIDE = HM == kHistWarpRed ? (NW | 1) : HCOLS;
    static constexpr unsigned ROWB = 4u * HSTRIDE;

    static size_t smem_bytes(int K, int n_lut) {
        size_t b = (size_t)TB * 24;             // B tile: {-x,-x,-y,-y} + {-z,-z}
        b += (size_t)TB / 32 * 16;              // bounding spheres of its 32-point chunks
        b += (size_t)n_lut * 16;                // screening table
        b += (size_t)(K + 2) * 8;               // FP64 edges (+ pad)
        b += (size_t)(K + 2) * 8;               // guard band of every edge
        b += (size_t)(K + 2) * ROWB;            // histograms, row K+1 a trash row
        return b;
    }
};

template <int NT, int HCOLS, int HSTRIDE = HCOLS>
__device__ __forceinline__ void flush_hist(unsigned* hist, int K,
                                           unsigned long long* __restrict__ counts) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int b = warp; b <= K + 1; b += NT / 32) {
        unsigned long long sum = 0;
        for (int q = lane; q < HCOLS; q += 32) {
            sum += hist[b * HSTRIDE + q];
            hist[b * HSTRIDE + q] = 0;
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o);
        if (lane == 0 && sum && b <= K) atomicAdd(counts + b, sum);  // row K+1 is trash
    }
}

template <int HM>
__device__ __forceinline__ void hist_add(unsigned cell, unsigned v) {
    if (HM == kHistLane) {
        unsigned c;
        asm volatile("ld.shared.b32 %0, [%1];" : "=r"(c) : "r"(cell) : "memory");
        asm volatile("st.shared.b32 [%0], %1;" :: "r"(cell), "r"(c + v) : "memory");
    } else {
        red_add_shared(cell, v);
    }
}

// Table entry of an FP32 squared chord's bucket (bits >= 0: non-negative).
__device__ __forceinline__ uint4 lut_entry(unsigned bits, unsigned lut, int shift, int base,
                                           int top_idx) {
    const int idx = min(max((int)(bits >> shift) - base, 0), top_idx);
    return lds_u4(lut + 16u * (unsigned)idx);
}

// Bins NV screened values s[h R + r] (pairs of A point r and B point j + h)
// into the thread's private histogram column at shared address col.  The
// table gives the byte offset of the row below / above the guard band of the
// bucket's edge; a value beyond the top edge (or masked with +inf) lands in
// the trash row K+1.  A value inside a band is counted, for now, in the row
// above it; the function returns true if the step held any such value, and
// the caller then settles them (recount_band_values).  No branch.
template <int NV, int HM>
__device__ __forceinline__ bool bin_values(const float (&s)[NV], unsigned col, unsigned lut,
                                           int shift, int base, int top_idx) {
    bool any_band = false;
#pragma unroll
    for (int v = 0; v < NV; ++v) {
        const unsigned bits = __float_as_uint(s[v]);
        const uint4 e = lut_entry(bits, lut, shift, base, top_idx);
        const bool below = bits < e.x;
        any_band |= !below && bits <= e.y;
        hist_add<HM>(col + (below ? e.z : e.w), 1u);
    }
    return any_band;
}

// A step's NV squared chords, passed by value.
template <int NV>
struct StepValues {
    float v[NV];
};

// Rare: the step held values inside a guard band.  Given the step's values
// again, take back their provisional counts and add each to the row its FP64
// recheck gives (one copy of the recheck code, in a loop over a bitmask);
// returns the number of values rechecked.  Kept out of line: its FP64
// registers then do not weigh on the loops that call it.
template <int NT, int R, int NV, int HM>
__device__ __noinline__ unsigned recount_band_values(const StepValues<NV> sv, unsigned col,
                                                     unsigned lut, int shift, int base,
                                                     int top_idx, unsigned row_bytes, int K,
                                                     const Segment& S, long long a0, long long bj,
                                                     unsigned sC) {
    const float (&s)[NV] = sv.v;
    unsigned n_recheck = 0;
    unsigned mask = 0;
    int hint_v = -1, hint = -1;  // the first such value and its edge's lower slot
#pragma unroll
    for (int v = 0; v < NV; ++v) {
        const unsigned bits = __float_as_uint(s[v]);
        const uint4 e = lut_entry(bits, lut, shift, base, top_idx);
        if (bits >= e.x && bits <= e.y) {
            mask |= 1u << v;
            hist_add<HM>(col + e.w, 0xFFFFFFFFu);  // -1
            if (hint_v < 0) {
                hint_v = v;
                hint = e.w == e.z + row_bytes ? (int)(e.z / row_bytes) : -1;
            }
        }
    }
    while (mask) {
        const int v = __ffs(mask) - 1;
        mask &= mask - 1;
        const unsigned slot =
            recheck_slot(S, a0 + v % R, bj + v / R, sC, K, v == hint_v ? hint : -1);
        ++n_recheck;
        hist_add<HM>(col + slot * row_bytes, 1u);
    }
    return n_recheck;
}

// Squared chords of JU consecutive B points (from j) with the thread's R A
// points: s[h R + r].  On a diagonal tile, pairs with i >= j get +inf, i
// being a_first + r (the thread's first A point's position in the tile).
// The B tile sits at shared addresses bxy (16 B per point: -x,-x,-y,-y) and
// bz (8 B per point: -z,-z).
template <int NT, int R, int JU, bool DIAG>
__device__ __forceinline__ void chords(float (&s)[JU * R], unsigned bxy_base, unsigned bz_base,
                                       const f2_t (&ax)[R / 2], const f2_t (&ay)[R / 2],
                                       const f2_t (&az)[R / 2], int j, int a_first) {
#pragma unroll
    for (int h = 0; h < JU; ++h) {
        f2_t bx, by;
        lds_f2x2(bxy_base + 16u * (unsigned)(j + h), bx, by);
        const f2_t bz = lds_f2(bz_base + 8u * (unsigned)(j + h));
#pragma unroll
        for (int q = 0; q < R / 2; ++q) {
            const f2_t dx = add2(ax[q], bx);
            const f2_t dy = add2(ay[q], by);
            const f2_t dz = add2(az[q], bz);
            const f2_t t = fma2(dz, dz, fma2(dy, dy, mul2(dx, dx)));
            unpack2(t, s[h * R + 2 * q], s[h * R + 2 * q + 1]);
        }
    }
    if (DIAG) {
#pragma unroll
        for (int h = 0; h < JU; ++h)
#pragma unroll
            for (int r = 0; r < R; ++r)
                if (j + h <= a_first + r) s[h * R + r] = __int_as_float(0x7f800000);
    }
}

template <int NV>
__device__ __forceinline__ float min_of(const float (&s)[NV]) {
    float m = s[0];
#pragma unroll
    for (int v = 1; v + 1 < NV; v += 2) m = min3f(m, s[v], s[v + 1]);
    if (NV % 2 == 0) m = fminf(m, s[NV - 1]);
    return m;
}

// The FP32 steps [j0, j1) of a B tile for the thread's R A points, each pair
// binned through the table (values inside a guard band settled in FP64).
template <int NT, int R, int JU, int HM, bool DIAG>
__device__ __forceinline__ void exact_steps(int j0, int j1, unsigned bxy, unsigned bz,
                                            unsigned lut, unsigned sC,
                                            unsigned col, const f2_t (&ax)[R / 2],
                                            const f2_t (&ay)[R / 2], const f2_t (&az)[R / 2],
                                            float hf, int shift, int base, int top_idx,
                                            unsigned row_bytes, int K, const Segment& S,
                                            long long a0, long long b0, int a_first,
                                            unsigned long long& n_recheck) {
    constexpr int NV = JU * R;
#pragma unroll 1
    for (int j = j0; j < j1; j += JU) {
        float s[NV];
        chords<NT, R, JU, DIAG>(s, bxy, bz, ax, ay, az, j, a_first);
        const float m = min_of(s);
        if (!(m <= hf)) continue;
        if (bin_values<NV, HM>(s, col, lut, shift, base, top_idx)) {
            StepValues<NV> s2;
            chords<NT, R, JU, DIAG>(s2.v, bxy, bz, ax, ay, az, j, a_first);
            n_recheck += recount_band_values<NT, R, NV, HM>(s2, col, lut, shift, base, top_idx,
                                                            row_bytes, K, S, a0, b0 + j, sC);
        }
    }
}

// Bounding sphere of the thread's R A points (FP32): centre = their mean,
// radius = the largest distance from it, enlarged by a relative 1e-6 for the
// roundings of that arithmetic.  Padding sentinels give a radius far above 2.
template <int R>
__device__ __forceinline__ float4 group_cap(const f2_t (&ax)[R / 2], const f2_t (&ay)[R / 2],
                                            const f2_t (&az)[R / 2]) {
    float x[R], y[R], z[R];
#pragma unroll
    for (int q = 0; q < R / 2; ++q) {
        unpack2(ax[q], x[2 * q], x[2 * q + 1]);
        unpack2(ay[q], y[2 * q], y[2 * q + 1]);
        unpack2(az[q], z[2 * q], z[2 * q + 1]);
    }
    float cx = 0.f, cy = 0.f, cz = 0.f;
#pragma unroll
    for (int r = 0; r < R; ++r) { cx += x[r]; cy += y[r]; cz += z[r]; }
    cx *= 1.f / R; cy *= 1.f / R; cz *= 1.f / R;
    float m = 0.f;
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const float dx = x[r] - cx, dy = y[r] - cy, dz = z[r] - cz;
        m = fmaxf(m, dx * dx + dy * dy + dz * dz);
    }
    return make_float4(cx, cy, cz, sqrtf(m) * (1.f + 1e-6f));
}

// How the pairs of a group of A points (sphere ga) with a chunk of B points
// (sphere gb) can be settled.  By the triangle inequality every FP32 pair
// distance lies within |ca - cb| -/+ (ra + rb); the FP64 unit vectors are
// within 1.2e-7 of their FP32 copies and the FP32 arithmetic here errs by a
// few units in the last place, all covered by the 1e-6 absolute and relative
// slack, so every pair's FP64 squared chord lies in [slo, shi].  The table
// classifies both ends (values inside a guard band or a bucket with several
// edges are ambiguous):
//   0  both ends in one slot: every pair is in slot rlo;
//   1  adjacent slots k and k+1 (rlo = slot k), split by edge k alone: each
//      pair is in one or the other by one FP32 comparison outside the
//      edge's guard band;
//   3  slots k, k+1, k+2, split by edges k and k+1: two comparisons per pair;
//   2  anything else: bin pair by pair.
// rlo is a byte offset of a slot's row, slot * row_bytes; a span wholly
// above h_top (the top edge's band) is the overflow row trash at once.
__device__ __forceinline__ int span_class(float4 ga, float4 gb, unsigned lut, int shift, int base,
                                          int top_idx, unsigned row_bytes, unsigned& rlo,
                                          unsigned h_top, unsigned trash) {
    const float dx = ga.x - gb.x, dy = ga.y - gb.y, dz = ga.z - gb.z;
    const float dc = sqrtf(dx * dx + dy * dy + dz * dz);
    const float rr = (ga.w + gb.w) * (1.f + 1e-6f) + 1e-6f;
    const float lo = dc * (1.f - 1e-6f) - rr, hi = dc * (1.f + 1e-6f) + rr;
    const float slo = lo > 0.f ? lo * lo * (1.f - 1e-5f) : 0.f;
    const float shi = hi * hi * (1.f + 1e-5f);
    if (!(ga.w <= 2.f && gb.w >= 0.f && gb.w <= 2.f)) return 2;  // padding (or NaN)
    const unsigned bl = __float_as_uint(slo), bh = __float_as_uint(shi);
    if (bl > h_top) {  // every pair beyond the top edge's band: overflow (row trash)
        rlo = trash;
        return 0;
    }
    const uint4 el = lut_entry(bl, lut, shift, base, top_idx);
    const uint4 eh = lut_entry(bh, lut, shift, base, top_idx);
    if (!(bl < el.x || bl > el.y) || !(bh < eh.x || bh > eh.y)) return 2;
    rlo = bl < el.x ? el.z : el.w;
    const unsigned rhi = bh < eh.x ? eh.z : eh.w;
    if (rlo == rhi) return 0;
    if (rhi == rlo + row_bytes) return 1;
    if (rhi == rlo + 2u * row_bytes) return 3;
    return 2;
}

// One step of a three-slot chunk: as two_slot_step, against two edges (the
// middles of their guard bands mid1 < mid2), with one accumulator each.
template <int R, int JU>
__device__ __forceinline__ void three_slot_step(unsigned bxy_base, unsigned bz_base,
                                                const f2_t (&ax)[R / 2], const f2_t (&ay)[R / 2],
                                                const f2_t (&az)[R / 2], int j, f2_t nmid1,
                                                f2_t nmid2, unsigned& neg1, unsigned& neg2,
                                                float& mb1, float& mb2) {
#pragma unroll
    for (int h = 0; h < JU; ++h) {
        f2_t bx, by;
        lds_f2x2(bxy_base + 16u * (unsigned)(j + h), bx, by);
        const f2_t bz = lds_f2(bz_base + 8u * (unsigned)(j + h));
#pragma unroll
        for (int q = 0; q < R / 2; ++q) {
            const f2_t dx = add2(ax[q], bx);
            const f2_t dy = add2(ay[q], by);
            const f2_t dz = add2(az[q], bz);
            const f2_t t = fma2(dz, dz, fma2(dy, dy, mul2(dx, dx)));
            float d0, d1, e0, e1;
            unpack2(add2(t, nmid1), d0, d1);
            unpack2(add2(t, nmid2), e0, e1);
            mb1 = min3f(mb1, fabsf(d0), fabsf(d1));
            mb2 = min3f(mb2, fabsf(e0), fabsf(e1));
            neg1 += (__float_as_uint(d0) >> 31) + (__float_as_uint(d1) >> 31);
            neg2 += (__float_as_uint(e0) >> 31) + (__float_as_uint(e1) >> 31);
        }
    }
}

// One step of a two-slot chunk: for JU B points and the thread's R A points,
// d = s - mid evaluated as fma(dz, dz, fma(dy, dy, fma(dx, dx, -mid))) from the
// same FP32 differences as chords().  Each fma rounds once, on a magnitude of
// at most max(s, mid), so for s <= 2c + 1e-12 (the only values near the edge)
// |d - (s - mid)| stays within the three roundings the guard band already
// allows for s (gamma_3 (s + E1), evaluated at 2c + 1e-12), and |d| > G
// settles the side of the FP64 squared chord exactly as the band does; far
// above the edge d is large and positive.  neg[q] counts the values with
// d < 0 and mb[q] keeps the smallest |d|, one accumulator per A pair q so that
// the steps' dependency chains interleave.
template <int R, int JU>
__device__ __forceinline__ void two_slot_step(unsigned bxy_base, unsigned bz_base,
                                              const f2_t (&ax)[R / 2], const f2_t (&ay)[R / 2],
                                              const f2_t (&az)[R / 2], int j, f2_t nmid,
                                              unsigned (&neg)[R / 2], float (&mb)[R / 2]) {
#pragma unroll
    for (int h = 0; h < JU; ++h) {
        f2_t bx, by;
        lds_f2x2(bxy_base + 16u * (unsigned)(j + h), bx, by);
        const f2_t bz = lds_f2(bz_base + 8u * (unsigned)(j + h));
#pragma unroll
        for (int q = 0; q < R / 2; ++q) {
            const f2_t dx = add2(ax[q], bx);
            const f2_t dy = add2(ay[q], by);
            const f2_t dz = add2(az[q], bz);
            float d0, d1;
            unpack2(fma2(dz, dz, fma2(dy, dy, fma2(dx, dx, nmid))), d0, d1);
            mb[q] = min3f(mb[q], fabsf(d0), fabsf(d1));
            neg[q] += (__float_as_uint(d0) >> 31) + (__float_as_uint(d1) >> 31);
        }
    }
}

// The pairs of the thread's R A points (tile positions a_first ..) with the
// B points [j_begin, j_end) of the staged tile.
template <int NT, int R, int JU, int HM, int DEF, bool DIAG>
__device__ __forceinline__ void tile_pass(unsigned bxy, unsigned bz, unsigned lut,
                                          unsigned sC, unsigned hist,
                                          const f2_t (&ax)[R / 2], const f2_t (&ay)[R / 2],
                                          const f2_t (&az)[R / 2], const PairParams& p,
                                          const Segment& S, long long I, long long J, int a_first,
                                          int j_begin, int j_end,
                                          unsigned long long& n_recheck) {
    using PK = PairKernel<NT, R, JU, HM, DEF>;
    constexpr int TA = PK::TA, TB = PK::TB;
    constexpr int NV = JU * R;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const unsigned h_top = p.tab.h_top;
    const float hf = __uint_as_float(h_top);
    const int shift = p.tab.shift, base = p.tab.base, K = p.tab.K, top_idx = p.tab.n_lut - 1;
    constexpr unsigned row_bytes = PK::ROWB;
    const unsigned col =
        hist + 4u * (unsigned)((HM == kHistWarp || HM == kHistWarpRed) ? warp : tid);
    const long long a0 = I * TA + a_first, b0 = J * TB;

    if (DEF) {
        // Deferred binning: the screening loop only notes, one bit per step,
        // which of 32 consecutive steps hold an in-range value; those steps
        // are then recomputed and binned.  The screening loop stays small.
        static_assert(TB % (4 * 32 * JU) == 0, "units must hold whole 32-step blocks");
#pragma unroll 1
        for (int jb = j_begin; jb < j_end; jb += 32 * JU) {
            unsigned mask = 0;
#pragma unroll 1
            for (int st = 0; st < 32; ++st) {
                float s[NV];
                chords<NT, R, JU, DIAG>(s, bxy, bz, ax, ay, az, jb + st * JU, a_first);
                mask |= (min_of(s) <= hf ? 1u : 0u) << st;
            }
            while (mask) {
                const int st = __ffs(mask) - 1;
                mask &= mask - 1;
                const int j = jb + st * JU;
                StepValues<NV> s;
                chords<NT, R, JU, DIAG>(s.v, bxy, bz, ax, ay, az, j, a_first);
                if (bin_values<NV, HM>(s.v, col, lut, shift, base, top_idx))
                    n_recheck += recount_band_values<NT, R, NV, HM>(s, col, lut, shift, base,
                                                                    top_idx, row_bytes, K, S, a0,
                                                                    b0 + j, sC);
            }
        }
        return;
    } else if (HM == kHistWarp) {
#pragma unroll 1
        for (int j = j_begin; j < j_end; j += JU) {
            float s[NV];
            chords<NT, R, JU, DIAG>(s, bxy, bz, ax, ay, az, j, a_first);
            const float m = min_of(s);
            if (!__any_sync(0xffffffffu, m <= hf)) continue;
            const unsigned trash = (unsigned)(K + 1) * row_bytes;
            unsigned amb_mask = 0;
#pragma unroll
            for (int v = 0; v < NV; ++v) {
                const unsigned bits = __float_as_uint(s[v]);
                const uint4 e = lut_entry(bits, lut, shift, base, top_idx);
                const bool amb = bits >= e.x && bits <= e.y;
                amb_mask |= amb ? (1u << v) : 0u;
                const unsigned off = amb ? trash : (bits < e.x ? e.z : e.w);
                const unsigned peers = __match_any_sync(0xffffffffu, off);
                if (lane == __ffs(peers) - 1) red_add_shared(col + off, (unsigned)__popc(peers));
            }
            while (amb_mask) {
                const int v = __ffs(amb_mask) - 1;
                amb_mask &= amb_mask - 1;
                const unsigned slot = recheck_slot(S, a0 + v % R, b0 + j + v / R, sC, K);
                ++n_recheck;
                red_add_shared(col + slot * row_bytes, 1u);
            }
        }
        return;
    }
    // pair by pair (diagonal tiles, or span binning off; spans go through
    // span_item's jobs)
    exact_steps<NT, R, JU, HM, DIAG>(j_begin, j_end, bxy, bz, lut, sC, col, ax, ay, az, hf, shift,
                                     base, top_idx, row_bytes, K, S, a0, b0, a_first, n_recheck);
}

// The thread's R A points, R consecutive points of the spatial order (a
// compact group: see span_class), packed two by two for the FP32x2
// instructions.  Each value goes through an explicit add of +0 (exact; it
// only turns -0 into +0, which leaves every squared chord unchanged): the
// packed operands then get registers of their own instead of being formed in
// place from the vector-load destinations, a layout measured to cost about a
// quarter of the screening loop's throughput.
template <int R>
__device__ __forceinline__ void load_group(const float4* __restrict__ gA, f2_t (&ax)[R / 2],
                                           f2_t (&ay)[R / 2], f2_t (&az)[R / 2]) {
#pragma unroll
    for (int q = 0; q < R / 2; ++q) {
        const float4 a = gA[2 * q];
        const float4 b = gA[2 * q + 1];
        ax[q] = pack2(__fadd_rn(a.x, 0.f), __fadd_rn(b.x, 0.f));
        ay[q] = pack2(__fadd_rn(a.y, 0.f), __fadd_rn(b.y, 0.f));
        az[q] = pack2(__fadd_rn(a.z, 0.f), __fadd_rn(b.z, 0.f));
    }
}

// ---------------------------------------------------------------------------
// Span jobs.  A (group, chunk) pair whose span needs its pairs computed (two
// slots, three slots, or pair by pair) is a job: the lane whose R A points
// form the group, its sub-tile, the chunk's index in the staged B tile and
// the lowest slot of the span.  Each warp keeps one ring of 32 jobs per kind
// in shared memory and runs a full ring as one round, one job per lane: a
// lane computes only pairs whose slot is not known from the spheres, whatever
// its own group's spans, and the lanes of a round run the same loop.  A job's
// A points are read again from the FP32 copy of the catalogue (L2).
// ---------------------------------------------------------------------------
constexpr int kJobTwo = 0, kJobThree = 1, kJobExact = 2, kJobKinds = 3, kChunk = 32;

// Bits 0-4 lane, 5-7 sub-tile, 8-15 chunk, 16-29 slot; the ring loop keeps
// the job's kind + 1 in bits 30-31 of the word it carries.
__device__ __forceinline__ unsigned job_word(int lane, int sub, int chunk, unsigned slot) {
    return (unsigned)lane | ((unsigned)sub << 5) | ((unsigned)chunk << 8) | (slot << 16);
}

// Chunk c of the B tile starts its steps at point JU c (mod 32): lanes of a
// round on neighbouring chunks then read points in different banks.
template <int JU>
__device__ __forceinline__ int chunk_point(int c0, int t, int rot) {
    return c0 + ((t + rot) & (kChunk - 1));
}

__device__ __forceinline__ unsigned atom_add_shared(unsigned a, unsigned v) {
    unsigned old;
    asm volatile("atom.shared.add.u32 %0, [%1], %2;" : "=r"(old) : "r"(a), "r"(v) : "memory");
    return old;
}

// A chunk's pairs with the lane's R A points (tile positions a_first ..)
// binned pair by pair through the table, values inside a guard band settled
// in FP64: the chunk's points t0, t0 + ts, ... (in its rotated order).  The
// tile pair (I, J) is read from shared memory (sIJ) only for those values.
template <int NT, int R, int JU, int HM>
__device__ __forceinline__ void exact_chunk(int c0, int rot, int t0, int ts, int a_first,
                                            unsigned sIJ,
                                            unsigned bxy, unsigned bz, unsigned lut, unsigned sC,
                                            unsigned col, const f2_t (&ax)[R / 2],
                                            const f2_t (&ay)[R / 2], const f2_t (&az)[R / 2],
                                            const PairParams& p, const Segment& S,
                                            unsigned& n_recheck) {
    using PK = PairKernel<NT, R, JU, HM, 0>;
    constexpr int TA = PK::TA, TB = PK::TB;
    constexpr int NV = R;  // one B point per step: fewer live values
    const float hf = __uint_as_float(p.tab.h_top);
    const int shift = p.tab.shift, base = p.tab.base, top_idx = p.tab.n_lut - 1;
#pragma unroll 1
    for (int t = t0; t < kChunk; t += ts) {
        const int j = chunk_point<JU>(c0, t, rot);
        float s[NV];
        chords<NT, R, 1, false>(s, bxy, bz, ax, ay, az, j, 0);
        if (!(min_of(s) <= hf)) continue;
        if (bin_values<NV, HM>(s, col, lut, shift, base, top_idx)) {
            StepValues<NV> s2;
            chords<NT, R, 1, false>(s2.v, bxy, bz, ax, ay, az, j, 0);
            const long long a0 = lds_s64(sIJ) * TA + a_first;
            const long long b0 = lds_s64(sIJ + 8u) * TB;
            n_recheck += recount_band_values<NT, R, NV, HM>(s2, col, lut, shift, base, top_idx,
                                                            PK::ROWB, p.tab.K, S, a0, b0 + j, sC);
        }
    }
}

// A job's R A points (the owner lane's group) from the FP32 copy.
template <int NT, int R, int JU, int HM>
__device__ __forceinline__ int job_points(unsigned job, unsigned sIJ, const Segment& S,
                                          f2_t (&ax)[R / 2], f2_t (&ay)[R / 2],
                                          f2_t (&az)[R / 2]) {
    constexpr int TA = PairKernel<NT, R, JU, HM, 0>::TA, SA = 32 * R;
    const int a_first = (int)((job >> 5) & 7u) * SA + (int)(job & 31u) * R;
    load_group<R>(S.a32 + lds_s64(sIJ) * TA + a_first, ax, ay, az);
    return a_first;
}

// A job of the pair-by-pair kind (the chunk's points t0, t0 + ts, ...).
template <int NT, int R, int JU, int HM>
__device__ __forceinline__ void exact_job(unsigned job, int t0, int ts, unsigned sIJ,
                                          unsigned bxy, unsigned bz, unsigned lut, unsigned sC,
                                          unsigned col, const PairParams& p, const Segment& S,
                                          unsigned& n_recheck) {
    f2_t ax[R / 2], ay[R / 2], az[R / 2];
    const int a_first = job_points<NT, R, JU, HM>(job, sIJ, S, ax, ay, az);
    const int c = (int)((job >> 8) & 255u);
    exact_chunk<NT, R, JU, HM>(c * kChunk, (JU * c) & (kChunk - 1), t0, ts, a_first, sIJ, bxy,
                               bz, lut, sC, col, ax, ay, az, p, S, n_recheck);
}

// The middle of the guard band of edge k (band table at shared address band)
// and the band's half-width.
__device__ __forceinline__ float edge_mid(unsigned band, unsigned k, float& G) {
    unsigned lo, hi;
    asm volatile("ld.shared.v2.b32 {%0, %1}, [%2];" : "=r"(lo), "=r"(hi) : "r"(band + 8u * k));
    const float lo_f = __uint_as_float(lo), hi_f = __uint_as_float(hi);
    const float mid = 0.5f * (lo_f + hi_f);
    G = fmaxf(mid - lo_f, hi_f - mid);
    return mid;
}

// A job of kind T (two or three slots) over the chunk's steps t0, t0 + ts,
// ... (JU points each).  Two slots: d = s - mid per pair, mid the middle of
// the edge's guard band; three slots: the same against two edges.  neg1 and
// neg2 count the values with d < 0 for the first and second edge (neg2 = 0
// for two slots), mb1 and mb2 keep the smallest |d|.
template <int NT, int R, int JU, int HM>
__device__ __forceinline__ void span_part(int T, unsigned job, int t0, int ts, unsigned sIJ,
                                          unsigned bxy, unsigned bz, unsigned band,
                                          const Segment& S, unsigned& neg1, unsigned& neg2,
                                          float& mb1, float& mb2) {
    f2_t ax[R / 2], ay[R / 2], az[R / 2];
    job_points<NT, R, JU, HM>(job, sIJ, S, ax, ay, az);
    const int c = (int)((job >> 8) & 255u);
    const int c0 = c * kChunk, rot = (JU * c) & (kChunk - 1);
    const unsigned slot = (job >> 16) & 0x3FFFu;
    float G;
    const float mid = edge_mid(band, slot, G);
    const f2_t nmid = pack2(-mid, -mid);
    neg1 = neg2 = 0;
    mb1 = mb2 = __int_as_float(0x7f800000);
    if (T == kJobTwo) {
        unsigned negq[R / 2];
        float mbq[R / 2];
#pragma unroll
        for (int q = 0; q < R / 2; ++q) {
            negq[q] = 0;
            mbq[q] = __int_as_float(0x7f800000);
        }
#pragma unroll 1
        for (int t = t0; t < kChunk; t += ts)
            two_slot_step<R, JU>(bxy, bz, ax, ay, az, chunk_point<JU>(c0, t, rot), nmid, negq,
                                 mbq);
#pragma unroll
        for (int q = 0; q < R / 2; ++q) {
            neg1 += negq[q];
            mb1 = fminf(mb1, mbq[q]);
        }
        return;
    }
    const float mid2 = edge_mid(band, slot + 1u, G);
#pragma unroll 1
    for (int t = t0; t < kChunk; t += ts)
        three_slot_step<R, JU>(bxy, bz, ax, ay, az, chunk_point<JU>(c0, t, rot), nmid,
                               pack2(-mid2, -mid2), neg1, neg2, mb1, mb2);
}

// Settles a two- or three-slot job from its counts (summed over the lanes
// that shared it): |d| > G for every value puts each value outside its
// edge's guard band, and then d < 0 means below the edge.  Returns false if
// some value had |d| <= G (rare): nothing is counted, and the chunk has to go
// pair by pair.
template <int NT, int R, int JU, int HM>
__device__ __forceinline__ bool span_settle(int T, unsigned job, unsigned band, unsigned col,
                                            unsigned neg1, unsigned neg2, float mb1, float mb2) {
    constexpr unsigned NP = (unsigned)(R * kChunk);
    constexpr unsigned row_bytes = PairKernel<NT, R, JU, HM, 0>::ROWB;
    const unsigned slot = (job >> 16) & 0x3FFFu;
    const unsigned rlo = slot * row_bytes;
    float G, G2 = 0.f;
    edge_mid(band, slot, G);
    if (mb1 <= G) return false;
    if (T == kJobTwo) {
        hist_add<HM>(col + rlo, neg1);
        hist_add<HM>(col + rlo + row_bytes, NP - neg1);
        return true;
    }
    edge_mid(band, slot + 1u, G2);
    if (mb2 <= G2) return false;
    hist_add<HM>(col + rlo, neg1);
    hist_add<HM>(col + rlo + row_bytes, neg2 - neg1);
    hist_add<HM>(col + rlo + 2u * row_bytes, NP - neg2);
    return true;
}

// Adds a warp's count (lanes with flag set, times w) to a 64-bit shared
// counter at address a (statistics only).
__device__ __forceinline__ void warp_stat(unsigned a, bool flag, unsigned w) {
    const unsigned m = __ballot_sync(0xffffffffu, flag);
    if ((threadIdx.x & 31) == 0 && m)
        asm volatile("red.shared.add.u64 [%0], %1;" ::"r"(a),
                     "l"((unsigned long long)__popc(m) * w)
                     : "memory");
}

// One round of jobs of kind T: this lane's share of job `run` (active: the
// lane has one; steps t0, t0 + ts, ... of the job, its ts lanes adjacent and
// ts a power of two).  Span jobs are settled by the first lane of each job
// from the counts summed over its ts lanes; the return value is the job (bit
// 30 set) if it has to go pair by pair, else 0.
template <int NT, int R, int JU, int HM, bool ST>
__device__ __forceinline__ unsigned job_round(int T, unsigned run, bool active, int t0, int ts,
                                              unsigned sIJ, unsigned bxy, unsigned bz,
                                              unsigned lut, unsigned band, unsigned sC,
                                              unsigned col, const PairParams& p,
                                              const Segment& S, bool stats, unsigned stat) {
    constexpr unsigned NP = (unsigned)(R * kChunk);
    const int lane = threadIdx.x & 31;
    unsigned n_recheck = 0, fb = 0;
    bool settled = false;
    if (T == kJobExact) {
        if (active) exact_job<NT, R, JU, HM>(run, t0, ts, sIJ, bxy, bz, lut, sC, col, p, S, n_recheck);
    } else {
        unsigned neg1 = 0, neg2 = 0;
        float mb1 = __int_as_float(0x7f800000), mb2 = mb1;
        if (active)
            span_part<NT, R, JU, HM>(T, run, t0 * JU, ts * JU, sIJ, bxy, bz, band, S, neg1, neg2,
                                     mb1, mb2);
#pragma unroll 1
        for (int o = ts >> 1; o > 0; o >>= 1) {
            neg1 += __shfl_xor_sync(0xffffffffu, neg1, o);
            neg2 += __shfl_xor_sync(0xffffffffu, neg2, o);
            mb1 = fminf(mb1, __shfl_xor_sync(0xffffffffu, mb1, o));
            mb2 = fminf(mb2, __shfl_xor_sync(0xffffffffu, mb2, o));
        }
        if (active && t0 == 0) {
            settled = span_settle<NT, R, JU, HM>(T, run, band, col, neg1, neg2, mb1, mb2);
            if (!settled) fb = run | (1u << 30);
        }
    }
    if (ST && stats) {
        warp_stat(stat + 8u, settled, NP);
        if (__any_sync(0xffffffffu, n_recheck != 0)) {
            unsigned long long v = n_recheck;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
            if (lane == 0)
                asm volatile("red.shared.add.u64 [%0], %1;" ::"r"(stat), "l"(v) : "memory");
        }
    }
    return fb;
}

// Lanes per job for a round of m < 32 jobs: the largest power of two with
// m ts <= 32 (span jobs: at most the chunk's steps, kChunk / JU).
template <int JU>
__device__ __forceinline__ int round_share(int T, int m) {
    int ts = 1 << (31 - __clz(32 / m));
    if (T != kJobExact) ts = min(ts, kChunk / JU);
    return ts;
}

// A warp's share of one item with span binning: units of its own sub-tile
// first, then those left of the others (shared counters at address units, one
// per sub-tile).  Each lane classifies its group against every chunk of a
// unit; a chunk in one slot is counted at once, the others become jobs (the
// warp's rings in the block's ring array at shared address rings, 32 words
// per kind) and a ring that fills runs as one round.  When every unit is
// taken, the jobs left in all the warps' rings are pooled and shared out
// evenly (a warp would otherwise run its own leftovers in partial rounds
// while the others wait at the next item's barrier; a block of one warp
// flushes its own rings instead); then the diagonal units of an auto count
// that the warp took go pair by pair, with the i < j mask.
// The tile pair (I, J) stays in shared memory (sIJ) and the statistics go to
// the block's shared counters (stat: rechecks, span pairs, skipped pairs), so
// that the rounds run with few live registers.  Every thread of the block
// calls this once per item (it holds block barriers).
template <int NT, int R, int JU, int HM, bool ST>
__device__ __forceinline__ void span_item(unsigned units, unsigned rings, unsigned sIJ,
                                          unsigned bxy, unsigned bz, unsigned lut, unsigned caps,
                                          unsigned band, unsigned sC, unsigned hist,
                                          const PairParams& p, const Segment& S, bool diag,
                                          unsigned stat) {
    using PK = PairKernel<NT, R, JU, HM, 0>;
    constexpr int TA = PK::TA, TB = PK::TB;
    constexpr int NW = NT / 32, SA = 32 * R, UPS = 4, UB = TB / UPS, CPU = UB / kChunk;
    constexpr unsigned row_bytes = PK::ROWB;
    constexpr unsigned NP = (unsigned)(R * kChunk);
    constexpr unsigned RING_BYTES = 4u * kJobKinds * 32u;  // one warp's rings
    static_assert(NW <= 8 && TB / kChunk <= 256 && UB % kChunk == 0 && kChunk % JU == 0 &&
                      NW * UPS <= 32,
                  "job fields");
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const unsigned ring = rings + RING_BYTES * (unsigned)warp;
    const unsigned col = hist + 4u * (unsigned)(HM == kHistWarpRed ? warp : tid);
    const bool stats = ST && p.stats != nullptr;
    unsigned fills = 0;      // jobs waiting per kind, 8 bits each
    unsigned diag_units = 0;  // diagonal units taken (bit sub UPS + u)
    int k = 0, cap_sub = -1, cn = -1;  // cn: next chunk of the current unit, -1: none
    float4 ga = make_float4(0.f, 0.f, 0.f, 0.f);
    // A block of one warp has nobody to pool its leftovers with: when its
    // units are all taken it flushes its own rings in the ring steps below
    // (partial rounds, each job shared among lanes), so that the span jobs
    // redone pair by pair join the pair-by-pair ring's last round.
    bool done = false;
#pragma unroll 1
    for (;;) {
#pragma unroll 1
        while (k < NW && cn < 0) {
            const int sub = (warp + k) % NW;
            unsigned u = 0;
            if (lane == 0) u = atom_add_shared(units + 4u * (unsigned)sub, 1u);
            u = __shfl_sync(0xffffffffu, u, 0);
            if (u >= (unsigned)UPS) {
                ++k;
                continue;
            }
            const int ub = (int)u * UB;
            if (diag && ub + UB <= sub * SA) continue;  // every pair has i >= j
            if (diag && ub < (sub + 1) * SA) {
                diag_units |= 1u << (sub * UPS + (int)u);
                continue;
            }
            if (sub != cap_sub) {
                f2_t ax[R / 2], ay[R / 2], az[R / 2];
                load_group<R>(S.a32 + lds_s64(sIJ) * TA + sub * SA + lane * R, ax, ay, az);
                ga = group_cap<R>(ax, ay, az);
                cap_sub = sub;
            }
            cn = ub / kChunk;
        }
        if (k == NW) {
            if constexpr (NW > 1) break;  // every unit taken: the leftovers are pooled below
            done = true;
        }
        // the chunk's job word with its kind + 1 in bits 30-31 (0: none)
        unsigned kj = 0;
        if (!done) {
            const int c = cn;
            cn = (c + 1) % CPU == 0 ? -1 : c + 1;
            const uint4 gbu = lds_u4(caps + 16u * (unsigned)c);
            const float4 gb = make_float4(__uint_as_float(gbu.x), __uint_as_float(gbu.y),
                                          __uint_as_float(gbu.z), __uint_as_float(gbu.w));
            unsigned rlo = 0;
            const unsigned trash = (unsigned)(p.tab.K + 1) * row_bytes;
            const int mode = span_class(ga, gb, lut, p.tab.shift, p.tab.base, p.tab.n_lut - 1,
                                        row_bytes, rlo, p.tab.h_top, trash);
            if (mode == 0) {
                if (rlo != trash) hist_add<HM>(col + rlo, NP);  // the trash row is never read
            } else {
                kj = job_word(lane, (warp + k) % NW, c, rlo / row_bytes) |
                     ((unsigned)(mode == 1 ? kJobTwo + 1 : mode == 3 ? kJobThree + 1
                                                                     : kJobExact + 1) << 30);
            }
            if (stats) {
                warp_stat(stat + 8u, mode == 0, NP);
                warp_stat(stat + 16u, mode == 0, NP);
            }
        }
        // Most chunks fill no ring: their jobs are appended at once and the
        // warp takes the next chunk (fills stay below 64, so 8 bits each).
        if (!done) {
            const unsigned kind = kj >> 30;
            const unsigned m1 = __ballot_sync(0xffffffffu, kind == 1u);
            const unsigned m2 = __ballot_sync(0xffffffffu, kind == 2u);
            const unsigned m3 = __ballot_sync(0xffffffffu, kind == 3u);
            const unsigned nf = fills + (unsigned)__popc(m1) + ((unsigned)__popc(m2) << 8) +
                                ((unsigned)__popc(m3) << 16);
            if ((nf & 0x202020u) == 0u) {
                if (kind != 0u) {
                    const int T = (int)kind - 1;
                    const unsigned mk = T == 0 ? m1 : T == 1 ? m2 : m3;
                    const int pos = (int)((fills >> (8 * T)) & 255u) +
                                    __popc(mk & ((1u << lane) - 1u));
                    sts_u32(ring + 128u * (unsigned)T + 4u * (unsigned)pos, kj & 0x3FFFFFFFu);
                }
                fills = nf;
                continue;
            }
        }
        // A ring that fills runs as one round, one job per lane: the two-slot
        // ring, the pair-by-pair ring for the two-slot jobs that found a value
        // near their edge, the three-slot ring, the same for its jobs, then the
        // pair-by-pair ring for the chunk's own job.  One code path per kind.
        unsigned fb = 0;  // this lane's job that has to go pair by pair (bit 30: valid)
#pragma unroll 1
        for (int st = 0; st < 5; ++st) {
            const int T = (0x298 >> (2 * st)) & 3;  // rings 0, 2, 1, 2, 2
            const bool from_fb = (st & 1) != 0;
            const unsigned word = from_fb ? fb : kj;
            const bool push = from_fb ? fb != 0u : (kj >> 30) == (unsigned)(T + 1);
            if (from_fb) fb = 0u;
            // one-warp blocks, units all taken: every ring but the
            // pair-by-pair one flushes at its step, that one at the last
            const bool flush = done && (T != kJobExact || st == 4);
            const unsigned m = __ballot_sync(0xffffffffu, push);
            const int fill = (int)((fills >> (8 * T)) & 255u);
            const int n = __popc(m);
            if (n == 0 && !(flush && fill > 0)) continue;
            const unsigned rt = ring + 128u * (unsigned)T;
            const int pos = fill + __popc(m & ((1u << lane) - 1u));
            const unsigned job = word & 0x3FFFFFFFu;
            if (push && pos < 32) sts_u32(rt + 4u * (unsigned)pos, job);
            const int total = fill + n;
            if (total < 32 && !flush) {
                fills += (unsigned)n << (8 * T);
                continue;
            }
            // a full round gives each lane a job; a flushed partial round
            // shares each job among ts lanes (round_share)
            const int ts = total < 32 ? round_share<JU>(T, total) : 1;
            const int jl = lane / ts;
            __syncwarp();
            const unsigned run = lds_u32(rt + 4u * (unsigned)min(jl, 31));
            __syncwarp();
            if (push && pos >= 32) sts_u32(rt + 4u * (unsigned)(pos - 32), job);
            fills = (fills & ~(255u << (8 * T))) | ((unsigned)max(total - 32, 0) << (8 * T));
            fb = job_round<NT, R, JU, HM, ST>(T, run, jl < total, lane % ts, ts, sIJ, bxy, bz, lut,
                                              band, sC, col, p, S, stats, stat);
        }
        if (done) break;
    }
    // The leftovers of every warp, pooled (blocks of several warps).  Once
    // all warps are here the rings are quiescent; each warp publishes its
    // fills in its unit counter (no longer claimed), and the jobs of each
    // kind, the rings taken in warp order, are shared out in contiguous slices
    // of about n / NW jobs, each slice one round with the lanes of a job
    // adjacent.
    if constexpr (NW > 1) {
        __syncthreads();
        if (lane == 0) sts_u32(units + 4u * (unsigned)warp, fills);
        __syncthreads();
        unsigned fl[NW];
#pragma unroll
        for (int q = 0; q < NW; ++q) fl[q] = lds_u32(units + 4u * (unsigned)q);
        unsigned fb0 = 0, fb1 = 0;  // pooled two- and three-slot jobs to redo pair by pair
#pragma unroll 1
        for (int T = 0; T < kJobKinds; ++T) {
            int n = 0;
#pragma unroll
            for (int q = 0; q < NW; ++q) n += (int)((fl[q] >> (8 * T)) & 255u);
            const int lo = warp * n / NW, m = (warp + 1) * n / NW - lo;
            if (m == 0) continue;
            const int ts = round_share<JU>(T, m);
            const int jl = lane / ts;
            // job lo + jl of the pool: position i of warp q's ring
            int i = lo + min(jl, m - 1), q = 0;
#pragma unroll
            for (int w = 0; w < NW - 1; ++w) {
                const int f = (int)((fl[w] >> (8 * T)) & 255u);
                const bool past = q == w && i >= f;
                i -= past ? f : 0;
                q += past ? 1 : 0;
            }
            const unsigned run =
                lds_u32(rings + RING_BYTES * (unsigned)q + 128u * (unsigned)T + 4u * (unsigned)i);
            const unsigned fb = job_round<NT, R, JU, HM, ST>(T, run, jl < m, lane % ts, ts, sIJ,
                                                             bxy, bz, lut, band, sC, col, p, S,
                                                             stats, stat);
            if (T == kJobTwo) fb0 = fb;
            if (T == kJobThree) fb1 = fb;
        }
        __syncthreads();  // every pooled job read: the rings are free again
        // pooled span jobs that found a value near an edge (rare): pair by pair,
        // each warp its own, through its pair-by-pair ring
#pragma unroll 1
        for (int h = 0; h < 2; ++h) {
            const unsigned fb = h == 0 ? fb0 : fb1;
            const unsigned m = __ballot_sync(0xffffffffu, fb != 0u);
            if (m == 0u) continue;
            const int n = __popc(m);
            const unsigned rt = ring + 128u * (unsigned)kJobExact;
            if (fb) sts_u32(rt + 4u * (unsigned)__popc(m & ((1u << lane) - 1u)), fb & 0x3FFFFFFFu);
            __syncwarp();
            const int ts = round_share<JU>(kJobExact, n);
            const int jl = lane / ts;
            const unsigned run = lds_u32(rt + 4u * (unsigned)min(jl, n - 1));
            __syncwarp();
            job_round<NT, R, JU, HM, ST>(kJobExact, run, jl < n, lane % ts, ts, sIJ, bxy, bz, lut,
                                         band, sC, col, p, S, stats, stat);
        }
    }
    // the diagonal units taken: pair by pair, i < j
#pragma unroll 1
    while (diag_units) {
        const int b = __ffs(diag_units) - 1;
        diag_units &= diag_units - 1;
        const int sub = b / UPS, ub = (b % UPS) * UB, a_first = sub * SA + lane * R;
        const long long I = lds_s64(sIJ), J = lds_s64(sIJ + 8u);
        f2_t ax[R / 2], ay[R / 2], az[R / 2];
        load_group<R>(S.a32 + I * TA + a_first, ax, ay, az);
        unsigned long long nr = 0;
        tile_pass<NT, R, JU, HM, 0, true>(bxy, bz, lut, sC, hist, ax, ay, az, p, S, I, J, a_first,
                                          ub, ub + UB, nr);
        if (stats) {
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) nr += __shfl_xor_sync(0xffffffffu, nr, o);
            if (lane == 0 && nr)
                asm volatile("red.shared.add.u64 [%0], %1;" ::"r"(stat), "l"(nr) : "memory");
        }
    }
    __syncwarp();
}

// ST: with the span path's statistics code (a launch with p.stats set); the
// build without it is the one launched when no statistics are asked for.
template <int NT, int R, int JU, int HM, int DEF, bool ST>
__global__ void __launch_bounds__(NT, R == 8 ? 640 / NT : 1) k_pairs(const __grid_constant__ PairParams p) {
    using PK = PairKernel<NT, R, JU, HM, DEF>;
    constexpr int TA = PK::TA, TB = PK::TB, HCOLS = PK::HCOLS, HSTRIDE = PK::HSTRIDE;
    constexpr int NW = NT / 32, SA = 32 * R, UPS = 4, UB = TB / UPS;
    static_assert(TA == NW * SA && TB % UPS == 0, "units tile the item");
    __shared__ unsigned s_units[NW];
    // span job rings (one per kind and warp) for the shapes that bin spans
    __shared__ unsigned s_ring[(!DEF && HM != kHistWarp) ? NW * kJobKinds * 32 : 1];
    extern __shared__ __align__(16) unsigned char smem[];
    const int K = p.tab.K;
    ulonglong2* sBxy = reinterpret_cast<ulonglong2*>(smem);
    f2_t* sBz = reinterpret_cast<f2_t*>(sBxy + TB);
    float4* sCap = reinterpret_cast<float4*>(sBz + TB);
    uint4* sLut = reinterpret_cast<uint4*>(sCap + TB / 32);
    double* sC = reinterpret_cast<double*>(sLut + p.tab.n_lut);
    uint2* sBand = reinterpret_cast<uint2*>(sC + (K + 2));
    unsigned* hist = reinterpret_cast<unsigned*>(sBand + (K + 2));
    // the item and its tile pair (I, J), in two buffers by the parity of the
    // block's item count: thread 0 writes the next item's pair while other
    // warps may still read the current one
    __shared__ long long s_item, s_IJ[2][2];
    __shared__ unsigned long long s_stat[3];  // span-path rechecks, span pairs, skipped pairs

    const int tid = threadIdx.x;
    constexpr unsigned row_bytes = PK::ROWB;
    for (int q = tid; q < p.tab.n_lut; q += NT)
        sLut[q] = make_uint4(p.tab.lut[q][0], p.tab.lut[q][1], p.tab.lut[q][2] * row_bytes,
                             p.tab.lut[q][3] * row_bytes);
    for (int q = tid; q <= K; q += NT) {
        sC[q] = p.tab.c64[q];
        sBand[q] = make_uint2(p.tab.band[q][0], p.tab.band[q][1]);
    }
    for (int q = tid; q < (K + 2) * HSTRIDE; q += NT) hist[q] = 0u;
    if (tid < 3) s_stat[tid] = 0ull;

    // the current count lives in shared memory; thread 0 switches it when an
    // item of another count is claimed, after the block flushed its columns
    __shared__ Segment sSeg;
    __shared__ int s_seg;
    // items of this launch: p.n_items, or fewer when a device-side pass kept
    // only some of them (tile pairs wholly beyond the top edge are skipped)
    const long long n_launch =
        p.n_items_dev ? min(p.n_items, (long long)*p.n_items_dev) : p.n_items;
    unsigned long long n_recheck = 0, n_items = 0;
    int since_flush = 0, cur_seg = -2;
    for (;;) {
        if (tid == 0) {
            const long long t = (long long)atomicAdd(p.cursor, 1ull);
            s_item = t < n_launch ? t : p.n_items;
            int seg = -1;
            if (t < n_launch && p.n_segs > 0) {
                const long long g = p.item_begin + t;
                int lo = 0, hi = p.n_segs - 1;  // last segment with item_begin <= g
                while (lo < hi) {
                    const int mid = (lo + hi + 1) >> 1;
                    if (p.segs[mid].item_begin <= g) lo = mid; else hi = mid - 1;
                }
                seg = lo;
            }
            s_seg = seg;
            if (t < n_launch) {
                // tile pair of the item (one thread: FP64 and 64-bit divisions)
                const Segment* G = seg < 0 ? &p.seg0 : p.segs + seg;
                long long local = p.item_begin + t - G->item_begin + G->item_offset;
                if (G->item_list) local = G->item_list[local];
                long long I, J;
                item_to_tiles(local, G->tiles_a, G->tiles_b, G->is_auto, &I, &J);
                s_IJ[n_items & 1][0] = I;
                s_IJ[n_items & 1][1] = J;
            }
        }
        __syncthreads();  // s_item visible; previous item's shared reads finished
        const long long t = s_item;
        if (t >= p.n_items) break;
        const int seg = s_seg;
        if (seg != cur_seg) {
            if (cur_seg != -2 && since_flush > 0) {
                flush_hist<NT, HCOLS, HSTRIDE>(hist, K, sSeg.counts);
                since_flush = 0;
            }
            __syncthreads();  // flush done before the segment is replaced
            if (tid == 0) sSeg = seg < 0 ? p.seg0 : p.segs[seg];
            cur_seg = seg;
            __syncthreads();
        }
        const Segment& S = sSeg;
        const long long I = s_IJ[n_items & 1][0], J = s_IJ[n_items & 1][1];
        const float4* gB = S.b32 + J * TB;
#pragma unroll 4
        for (int q = 0; q < R; ++q) {
            const float4 b = gB[q * NT + tid];
            sBxy[q * NT + tid] = make_ulonglong2(pack2(-b.x, -b.x), pack2(-b.y, -b.y));
            sBz[q * NT + tid] = pack2(-b.z, -b.z);
        }
        if (S.b_caps)
            for (int q = tid; q < TB / 32; q += NT) sCap[q] = S.b_caps[J * (TB / 32) + q];
        if (tid < NW) s_units[tid] = 0;
        __syncthreads();  // B tile staged, unit counters reset
        const unsigned a_bxy = smem_addr(sBxy), a_bz = smem_addr(sBz), a_lut = smem_addr(sLut),
                       a_cap = smem_addr(sCap), a_band = smem_addr(sBand),
                       a_hist = smem_addr(hist), a_c = smem_addr(sC);
        // The item is split into units of one warp's worth of A points (SA =
        // 32 R consecutive points, a sub-tile) by a quarter of the B tile.  A
        // warp takes the units of its own sub-tile first, then those left of
        // the others, so the warps of the block finish the item together
        // whatever the mix of cheap and costly units.
        const int lane = tid & 31, warp = tid >> 5;
        const bool diag = S.is_auto && I == J;
        bool spans = false;
        if constexpr (!DEF && HM != kHistWarp) spans = p.span && S.b_caps;
        if constexpr (!DEF && HM != kHistWarp) {
            if (spans)
                span_item<NT, R, JU, HM, ST>(smem_addr(s_units), smem_addr(s_ring),
                                         smem_addr(s_IJ[n_items & 1]), a_bxy, a_bz, a_lut, a_cap, a_band, a_c,
                                         a_hist, p, S, diag, smem_addr(s_stat));
        }
        int cur = -1;
        f2_t ax[R / 2], ay[R / 2], az[R / 2];
#pragma unroll 1
        for (int k = 0; k < NW && !spans; ++k) {
            const int sub = (warp + k) % NW;
#pragma unroll 1
            for (;;) {
                unsigned u = 0;
                if (lane == 0) u = atomicAdd(&s_units[sub], 1u);
                u = __shfl_sync(0xffffffffu, u, 0);
                if (u >= (unsigned)UPS) break;
                const int a_first = sub * SA + lane * R;
                const int jb = (int)u * UB, je = jb + UB;
                if (diag && je <= sub * SA) continue;  // every pair has i >= j
                if (sub != cur) {
                    load_group<R>(S.a32 + I * TA + a_first, ax, ay, az);
                    cur = sub;
                }
                if (diag && jb < (sub + 1) * SA)
                    tile_pass<NT, R, JU, HM, DEF, true>(a_bxy, a_bz, a_lut, a_c, a_hist, ax, ay,
                                                        az, p, S, I, J, a_first, jb, je,
                                                        n_recheck);
                else
                    tile_pass<NT, R, JU, HM, DEF, false>(a_bxy, a_bz, a_lut, a_c, a_hist, ax, ay,
                                                         az, p, S, I, J, a_first, jb, je,
                                                         n_recheck);
            }
        }
        ++n_items;
        if (++since_flush == p.items_per_flush) {
            __syncthreads();
            flush_hist<NT, HCOLS, HSTRIDE>(hist, K, sSeg.counts);
            __syncthreads();
            since_flush = 0;
        }
    }
    // all threads left the loop after the same barrier
    if (cur_seg != -2) flush_hist<NT, HCOLS, HSTRIDE>(hist, K, sSeg.counts);
    if (p.stats) {
        unsigned long long v = n_recheck;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if ((tid & 31) == 0 && v) atomicAdd(p.stats + WTHETA_STAT_RECHECK, v);
        if (tid == 0) {
            // the span path's counts (the loop's last barrier ordered them)
            if (s_stat[0]) atomicAdd(p.stats + WTHETA_STAT_RECHECK, s_stat[0]);
            if (s_stat[1]) atomicAdd(p.stats + WTHETA_STAT_SPAN, s_stat[1]);
            // pairs of chunks settled in one slot were never computed
            if (s_stat[2]) atomicAdd(p.stats + WTHETA_STAT_PAIRS, 0ull - s_stat[2]);
        }
        if (tid == 0 && n_items) {
            atomicAdd(p.stats + WTHETA_STAT_TILES, n_items);
            atomicAdd(p.stats + WTHETA_STAT_PAIRS, n_items * (unsigned long long)TA * TB);
        }
    }
}

// The device tables of a w(theta) launch (its counts' segments and culling
// table), written by one small kernel from its parameters, which also zeroes
// n0 words at z0 and n1 at z1 (the launch cursor and the kept counters).
struct CountTables {
    Segment segs[3];
    CullSeg cs[3];
    int n_segs;
    int with_cull;
};
__global__ void k_set_tables(const CountTables t, Segment* __restrict__ segs,
                             CullSeg* __restrict__ cs, unsigned long long* __restrict__ z0, int n0,
                             unsigned long long* __restrict__ z1, int n1) {
    const int i = threadIdx.x;
    if (i < t.n_segs) {
        segs[i] = t.segs[i];
        if (t.with_cull) cs[i] = t.cs[i];
    }
    if (i < n0) z0[i] = 0ull;
    if (i < n1) z1[i] = 0ull;
}

// counts[K+1] = total - sum(counts[0..K]) for every count of a batch.
__global__ void k_finalize_segments(const Segment* __restrict__ segs, int n_segs, int K) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n_segs; i += gridDim.x * blockDim.x) {
        unsigned long long* c = segs[i].counts;
        unsigned long long s = 0;
        for (int k = 0; k <= K; ++k) s += c[k];
        c[K + 1] = segs[i].total - s;
    }
}

// ---------------------------------------------------------------------------
// launch plumbing
// ---------------------------------------------------------------------------
template <int NT, int R, int JU, int HM, int DEF>
static Variant make_variant() {
    constexpr bool spans = !DEF && HM != kHistWarp;  // only the span path has ST code
    return Variant{NT, R, JU, HM, DEF, &k_pairs<NT, R, JU, HM, DEF, true>,
                   spans ? &k_pairs<NT, R, JU, HM, DEF, false> : &k_pairs<NT, R, JU, HM, DEF, true>,
                   &PairKernel<NT, R, JU, HM, DEF>::smem_bytes};
}

// The build of v's kernel for a launch with these parameters.
static void (*pair_kernel(const Variant* v, const PairParams& prm))(PairParams) {
    return prm.stats ? v->kernel : v->kernel_fast;
}

// Instantiated shapes (tile = threads x points_per_thread).  Per-warp
// histograms (mode 2) need the whole warp in step, so they bin inline.
const Variant* variants(int* n) {
    static const Variant v[] = {
        make_variant<128, 8, 2, kHistLaneAtomic, 0>(), make_variant<128, 8, 2, kHistLaneAtomic, 1>(),
        make_variant<128, 8, 2, kHistLane, 1>(),       make_variant<128, 8, 2, kHistWarp, 0>(),
        make_variant<128, 8, 1, kHistLaneAtomic, 1>(), make_variant<64, 16, 2, kHistLaneAtomic, 1>(),
        make_variant<64, 16, 2, kHistWarp, 0>(),       make_variant<128, 16, 2, kHistLaneAtomic, 1>(),
        make_variant<256, 8, 2, kHistLaneAtomic, 1>(), make_variant<256, 8, 2, kHistWarp, 0>(),
        make_variant<64, 8, 2, kHistLaneAtomic, 0>(),  make_variant<128, 8, 2, kHistWarpRed, 0>(),
        make_variant<64, 8, 2, kHistWarpRed, 0>(),     make_variant<32, 8, 2, kHistLaneAtomic, 0>(),
    };
    *n = (int)(sizeof(v) / sizeof(v[0]));
    return v;
}

int device_info(DeviceInfo* out) {
    static std::mutex mu;
    static DeviceInfo cache[64];
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return WTHETA_ECUDA;
    std::lock_guard<std::mutex> g(mu);
    if (cache[dev].sm_count == 0) {
        if (cudaDeviceGetAttribute(&cache[dev].sm_count, cudaDevAttrMultiProcessorCount, dev) !=
                cudaSuccess ||
            cudaDeviceGetAttribute(&cache[dev].max_smem_optin,
                                   cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess)
            return WTHETA_ECUDA;
        // keep freed scratch in this process's stream-ordered pool between calls
        cudaMemPool_t pool;
        if (cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
            unsigned long long keep = ~0ull;
            cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
        }
    }
    *out = cache[dev];
    return WTHETA_OK;
}

// The default shape for one call: tiles of 256 points (one warp) when the
// larger catalogue has at most 16k points and of 512 points (64 threads) up
// to 64k, so that a small count still has tile pairs for every SM and each
// CTA's share stays short; the 1024-point shape otherwise.
const Variant* pick_for_size(const wtheta_tune* tune, long long n_max, int K, int n_lut,
                             int max_smem) {
    if (!tune && n_max <= 65536) {
        wtheta_tune small = {};
        small.threads = n_max <= 16384 ? 32 : 64;
        small.points_per_thread = 8;
        const Variant* v = pick_variant(&small, K, n_lut, max_smem);
        if (v) return v;
    }
    return pick_variant(tune, K, n_lut, max_smem);
}

const Variant* pick_variant(const wtheta_tune* tune, int K, int n_lut, int max_smem) {
    int nv = 0;
    const Variant* v = variants(&nv);
    const int want_nt = tune && tune->threads ? tune->threads : 128;
    const int want_r = tune && tune->points_per_thread ? tune->points_per_thread : 8;
    const int want_ju = tune && tune->j_per_screen ? tune->j_per_screen : 2;
    int want_hm = tune && tune->hist_mode ? tune->hist_mode : 0;
    int want_def = tune && tune->deferred ? (tune->deferred == 2 ? 1 : 0) : -1;
    auto fits = [&](const Variant& x) { return x.smem(K, n_lut) <= (size_t)max_smem; };
    auto shape = [&](const Variant& x) {
        return x.nt == want_nt && x.r == want_r && x.ju == want_ju;
    };
    if (want_hm == 0) {
        // private per-thread histograms while they fit comfortably (measured
        // 15% faster on the survey workload than per-warp columns, whose shared
        // reductions contend); per-warp columns updated by shared reductions
        // otherwise, which keep the span path at large bin counts
        want_hm = kHistWarp;
        for (int i = 0; i < nv; ++i)
            if (shape(v[i]) && v[i].hm == kHistWarpRed && v[i].def == 0 && fits(v[i]))
                want_hm = kHistWarpRed;
        for (int i = 0; i < nv; ++i)
            if (shape(v[i]) && v[i].hm == kHistLaneAtomic && v[i].smem(K, n_lut) <= 100 * 1024)
                want_hm = kHistLaneAtomic;
    }
    if (want_def < 0) want_def = 0;  // inline binning measured faster once in-range pairs matter
    for (int i = 0; i < nv; ++i)
        if (shape(v[i]) && v[i].hm == want_hm && v[i].def == want_def && fits(v[i])) return &v[i];
    // fall back: same tile size, per-warp histograms (with span jobs first)
    for (int hm : {(int)kHistWarpRed, (int)kHistWarp})
        for (int i = 0; i < nv; ++i)
            if (v[i].nt * v[i].r == want_nt * want_r && v[i].hm == hm && v[i].def == 0 &&
                fits(v[i]))
                return &v[i];
    return nullptr;
}

int grid_for(const Variant* v, size_t smem, long long n_items, int sm_count, int want_per_sm,
                    int* grid) {
    static std::mutex mu;
    {
        std::lock_guard<std::mutex> g(mu);
        if (cudaFuncSetAttribute((const void*)v->kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)smem) != cudaSuccess ||
            cudaFuncSetAttribute((const void*)v->kernel_fast,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)smem) != cudaSuccess)
            return WTHETA_ECUDA;
    }
    int per_sm = 0;
    int per_sm_fast = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, (const void*)v->kernel, v->nt,
                                                      smem) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm_fast, (const void*)v->kernel_fast,
                                                      v->nt, smem) != cudaSuccess)
        return WTHETA_ECUDA;
    per_sm = std::min(per_sm, per_sm_fast);  // one grid size for both builds
    per_sm = std::max(per_sm, 1);
    if (want_per_sm > 0) per_sm = std::min(per_sm, want_per_sm);
    long long g = (long long)per_sm * sm_count;
    if (g > n_items) g = n_items;
    *grid = (int)std::max(g, 1LL);
    return WTHETA_OK;
}

long long round_up(long long x, long long m) { return (x + m - 1) / m * m; }

int check_cuda(cudaError_t e) {
    if (e == cudaSuccess) return WTHETA_OK;
    if (e == cudaErrorMemoryAllocation) return WTHETA_ENOMEM;
    return WTHETA_ECUDA;
}

static int launch_grid(long long n, int sm_count) {
    const long long g = (n + 255) / 256;
    return (int)std::min<long long>(std::max<long long>(g, 1), (long long)sm_count * 16);
}

static long long sort_blocks(long long n) {
    const long long tile = (long long)kSortThreads * sort_rounds(n);
    return std::max<long long>(1, (n + tile - 1) / tile);
}

size_t order_bytes(long long n, int with_labels) {
    const size_t a4 = ((size_t)n * 4 + 255) / 256 * 256;
    return (4 + (with_labels ? 1 : 0)) * a4 +                   // keys, indices (x2), labels
           ((size_t)sort_blocks(n) * 256 * 4 + 255) / 256 * 256 +  // digit counts per block
           256 * 4;                                              // digit totals
}

// The buffers of a sort's scratch (order_bytes(n, with_labels) bytes): keys
// and indices twice (passes alternate), labels, per-block digit counts and
// the digit totals.
struct SortBufs {
    unsigned* key[2];
    unsigned* idx[2];
    unsigned* lab;
    unsigned* hist;
    unsigned* tot;
    long long G;
    int rounds;
};
static SortBufs sort_bufs(unsigned char* scratch, long long n, int with_labels) {
    const size_t a4 = ((size_t)n * 4 + 255) / 256 * 256;
    SortBufs B;
    B.G = sort_blocks(n);
    B.rounds = sort_rounds(n);
    B.key[0] = (unsigned*)scratch;
    B.key[1] = (unsigned*)(scratch + a4);
    B.idx[0] = (unsigned*)(scratch + 2 * a4);
    B.idx[1] = (unsigned*)(scratch + 3 * a4);
    B.lab = (unsigned*)(scratch + 4 * a4);
    B.hist = (unsigned*)(scratch + (4 + (with_labels ? 1 : 0)) * a4);
    B.tot = B.hist + ((size_t)B.G * 256 + 63) / 64 * 64;
    return B;
}

// One stable pass on the byte of key_in at shift.
static void digit_pass(const SortBufs& B, const unsigned* key_in, const unsigned* idx_in,
                       long long n, int shift, unsigned* key_out, unsigned* idx_out,
                       cudaStream_t st) {
    k_digit_hist<<<(unsigned)B.G, kSortThreads, 0, st>>>(key_in, n, shift, B.rounds, B.hist);
    k_digit_rows<<<256 / 8, 256, 0, st>>>(B.hist, (int)B.G, B.tot);
    k_digit_scatter<<<(unsigned)B.G, kSortThreads, 0, st>>>(key_in, idx_in, n, shift, B.rounds,
                                                            B.hist, B.tot, key_out, idx_out);
    count_launch(3);
}

// The four passes over 32-bit keys in B.key[0] (indices in B.idx[0]); the
// sorted keys and indices come back in the same buffers.
static void key_passes(const SortBufs& B, long long n, cudaStream_t st) {
    for (int pass = 0; pass < 4; ++pass) {
        const int in = pass & 1, o = in ^ 1;
        digit_pass(B, B.key[in], B.idx[in], n, 8 * pass, B.key[o], B.idx[o], st);
    }
}

int spatial_order(const double* x64, long long stride, long long n, int check,
                  const int* labels, int n_labels, unsigned char* scratch, int sm_count,
                  cudaStream_t st, const unsigned** order, const unsigned** sorted_labels) {
    const SortBufs B = sort_bufs(scratch, n, labels != nullptr);
    *order = B.idx[0];
    if (sorted_labels) *sorted_labels = nullptr;
    if (n <= 0) return WTHETA_OK;
    k_sort_keys<<<launch_grid(n, sm_count), 256, 0, st>>>(x64, stride, n, check, B.key[0],
                                                          B.idx[0]);
    count_launch();
    key_passes(B, n, st);
    if (labels) {
        // one more stable pass per byte of the label (two above 256 labels):
        // regions in label order, each in spatial order
        int cur = 0;
        for (int shift = 0; shift == 0 || (shift < 16 && (n_labels - 1) >> shift); shift += 8) {
            k_sorted_labels<<<launch_grid(n, sm_count), 256, 0, st>>>(B.idx[cur], labels, n,
                                                                      n_labels, B.lab);
            count_launch();
            digit_pass(B, B.lab, B.idx[cur], n, shift, B.key[cur ^ 1], B.idx[cur ^ 1], st);
            cur ^= 1;
        }
        *order = B.idx[cur];
        if (sorted_labels) *sorted_labels = B.key[cur];
    }
    return check_cuda(cudaGetLastError());
}

size_t prepare_bytes(long long n, long long n_pad, int is_xyz) {
    size_t b = (size_t)n_pad * 16 + 256;               // FP32 points
    b += ((size_t)n_pad / 32 * 16 + 255) / 256 * 256;  // chunk bounding spheres
    b += order_bytes(n, 0);                            // the sort
    if (!is_xyz) b += ((size_t)n * 24 + 255) / 256 * 256;  // FP64 SoA
    b += (size_t)n_pad * 24 + 256;                     // the same, in the spatial order
    return b;
}

int prepare(const double* coords, long long n, long long n_pad, int is_xyz, int tag,
                   unsigned char* scratch, int sm_count, cudaStream_t st, Prepared* out) {
    TraceRange trace("prepare");
    unsigned char* sp = scratch;
    float4* p32 = (float4*)sp;
    sp += ((size_t)n_pad * 16 + 255) / 256 * 256;
    float4* c32 = (float4*)sp;
    sp += ((size_t)n_pad / 32 * 16 + 255) / 256 * 256;
    unsigned char* sort_scratch = sp;
    sp += order_bytes(n, 0);
    const double* x64 = coords;
    long long stride = n;
    if (!is_xyz && n > 0) {
        double* x = (double*)sp;
        k_radec_to_xyz<<<launch_grid(n, sm_count), 256, 0, st>>>(coords, n, x, n);
        count_launch();
        x64 = x;
    }
    if (!is_xyz) sp += ((size_t)n * 24 + 255) / 256 * 256;
    double* s64 = (double*)sp;  // FP64 SoA in the spatial order (stride n_pad)
    const unsigned* order = nullptr;
    int rc = spatial_order(x64, stride, n, is_xyz, nullptr, 0, sort_scratch, sm_count, st, &order,
                           nullptr);
    if (rc) return rc;
    k_gather_points<<<launch_grid(n_pad, sm_count), 256, 0, st>>>(x64, stride, n, n_pad, order,
                                                                  p32, s64, tag);
    k_chunk_caps<<<launch_grid(n_pad, sm_count), 256, 0, st>>>(p32, n, n_pad, c32);
    count_launch(2);
    out->p32 = p32;
    out->c32 = c32;
    out->x64 = s64;
    out->stride = n_pad;
    out->sorted = 1;
    return check_cuda(cudaGetLastError());
}

size_t prepare_joint_bytes(long long na, long long pa, long long nb, long long pb) {
    const long long N = na + nb, P = pa + pb;
    size_t b = ((size_t)P * 16 + 255) / 256 * 256;       // FP32 points
    b += ((size_t)P / 32 * 16 + 255) / 256 * 256;        // chunk bounding spheres
    b += ((size_t)P * 24 + 255) / 256 * 256;             // FP64, spatial order
    b += ((size_t)N * 24 + 255) / 256 * 256;             // FP64, input order
    b += order_bytes(N, 0);                              // the sort
    return b;
}

int prepare_joint(const double* a, long long na, long long pa, const double* b, long long nb,
                  long long pb, int is_xyz, int tag0, unsigned char* scratch, int sm_count,
                  cudaStream_t st, Prepared* A, Prepared* B) {
    TraceRange trace("prepare");
    const long long N = na + nb, P = pa + pb;
    if (N >= (1LL << 32) - 1) return WTHETA_EINVAL;  // 32-bit positions in the sort
    unsigned char* sp = scratch;
    float4* p32 = (float4*)sp;
    sp += ((size_t)P * 16 + 255) / 256 * 256;
    float4* c32 = (float4*)sp;
    sp += ((size_t)P / 32 * 16 + 255) / 256 * 256;
    double* s64 = (double*)sp;
    sp += ((size_t)P * 24 + 255) / 256 * 256;
    double* x = (double*)sp;
    sp += ((size_t)N * 24 + 255) / 256 * 256;
    const SortBufs S = sort_bufs(sp, N, 0);
    if (N > 0) {
        const long long g = std::min<long long>((N + 63) / 64, (long long)sm_count * 32);
        k_joint_keys<<<(unsigned)g, 64, 0, st>>>(a, na, b, nb, is_xyz, x, S.key[0], S.idx[0]);
        count_launch();
        key_passes(S, N, st);
    }
    if (P > 0) {
        k_gather_joint<<<launch_grid(P, sm_count), 256, 0, st>>>(x, na, pa, nb, pb, S.idx[0], tag0,
                                                                 p32, s64);
        k_chunk_caps<<<launch_grid(P, sm_count), 256, 0, st>>>(p32, P, P, c32);
        count_launch(2);
    }
    A->p32 = p32;
    A->c32 = c32;
    A->x64 = s64;
    A->stride = P;
    A->sorted = 1;
    B->p32 = p32 + pa;
    B->c32 = c32 + pa / 32;
    B->x64 = s64 + pa;
    B->stride = P;
    B->sorted = 1;
    return check_cuda(cudaGetLastError());
}

int launch_radec_to_xyz(const double* coords, long long n, double* xyz, int sm_count,
                        cudaStream_t st) {
    if (n <= 0) return WTHETA_OK;
    k_radec_to_xyz<<<launch_grid(n, sm_count), 256, 0, st>>>(coords, n, xyz, n);
    count_launch();
    return check_cuda(cudaGetLastError());
}

int launch_count_labels(const unsigned* lab, long long n, int n_labels,
                        unsigned long long* sizes, int sm_count, cudaStream_t st) {
    if (n <= 0) return WTHETA_OK;
    k_count_labels<<<launch_grid(n, sm_count), 256, 0, st>>>(lab, n, n_labels, sizes);
    count_launch();
    return check_cuda(cudaGetLastError());
}

int launch_gather_regions(const double* x64, long long stride, const unsigned* order,
                          const long long* src, const long long* dst, int R, long long n_pad,
                          float4* p32, int tag, int sm_count, cudaStream_t st) {
    if (n_pad <= 0) return WTHETA_OK;
    k_gather_regions<<<launch_grid(n_pad, sm_count), 256, 0, st>>>(x64, stride, order, src, dst,
                                                                   R, n_pad, p32, tag);
    count_launch();
    return check_cuda(cudaGetLastError());
}

int launch_chunk_caps(const float4* p32, long long n_pad, float4* c32, int sm_count,
                      cudaStream_t st) {
    if (n_pad <= 0) return WTHETA_OK;
    k_chunk_caps<<<launch_grid(n_pad, sm_count), 256, 0, st>>>(p32, n_pad, n_pad, c32);
    count_launch();
    return check_cuda(cudaGetLastError());
}

int launch_cull_batch(const CullSeg* cs, int n_segs, long long total, double theta_top,
                      unsigned long long* kept, Segment* segs, unsigned long long* n_kept,
                      int sm_count, cudaStream_t st, unsigned long long* stats) {
    if (n_segs <= 0) return WTHETA_OK;
    k_cull_batch<<<launch_grid(std::max(total, 1LL), sm_count), 256, 0, st>>>(
        cs, n_segs, total, theta_top, kept, stats);
    k_cull_prefix<<<1, 32, 0, st>>>(segs, cs, kept, n_segs, n_kept);
    count_launch(2);
    return check_cuda(cudaGetLastError());
}

unsigned long long per_item_bound(const Variant* v) {
    // A thread bins (or settles by chunk) R x TB pairs per unit of its own
    // sub-tile and may take the units of every other sub-tile of the item
    // (NT/32 of them): own = NT/32 x R TB pairs of its own groups.  With span
    // jobs it also runs at most one job (R x 32 pairs) per round of its warp;
    // the warp's jobs are at most one per lane and chunk, plus one
    // pair-by-pair job for each span job that found a value near an edge, so
    // its full rounds add at most 2 own; after them come at most three pooled
    // rounds and two rounds of pooled jobs redone pair by pair.  A per-warp
    // column gains 32 times as much.
    const unsigned long long own = (unsigned long long)(v->nt / 32) * (unsigned long long)v->r *
                                   (unsigned long long)v->nt * (unsigned long long)v->r;
    return (v->hm == kHistWarp || v->hm == kHistWarpRed ? 32ull : 1ull) *
           (3ull * own + 5ull * 32ull * (unsigned)v->r);
}

Segment make_segment(const Prepared& A, const Prepared& B, long long ta, long long tb,
                            int is_auto, long long item_begin, unsigned long long* counts,
                            unsigned long long total) {
    Segment g;
    std::memset(&g, 0, sizeof(g));
    g.a32 = A.p32; g.b32 = B.p32; g.a64 = A.x64; g.b64 = B.x64;
    g.b_caps = B.c32;
    g.a64_stride = A.stride; g.b64_stride = B.stride;
    g.sorted64 = (A.sorted ? 1 : 0) | (B.sorted ? 2 : 0);
    g.tiles_a = ta; g.tiles_b = tb;
    g.item_begin = item_begin;
    g.n_items = is_auto ? ta * (ta + 1) / 2 : ta * tb;
    g.counts = counts;
    g.total = total;
    g.is_auto = is_auto;
    return g;
}

PairParams make_params(const Variant* v, const BinTable& tab, const Segment* seg0,
                              const Segment* segs, int n_segs, long long item_begin,
                              long long n_items, unsigned long long* cursor,
                              unsigned long long* stats) {
    PairParams prm;
    std::memset(&prm, 0, sizeof(prm));
    if (seg0) prm.seg0 = *seg0;
    prm.segs = segs;
    prm.n_segs = n_segs;
    prm.item_begin = item_begin;
    prm.n_items = n_items;
    prm.items_per_flush = (int)std::min<unsigned long long>(0xFFFFFFFFull / per_item_bound(v),
                                                            1ull << 30);
    prm.cursor = cursor;
    prm.stats = stats;
    prm.span = 1;
    std::memcpy(&prm.tab, &tab, sizeof(tab));
    return prm;
}

// Core of wtheta_count / wtheta_count_xyz / wtheta_count_ex.
static int count_impl(const double* ca, long long n_a, const double* cb, long long n_b,
                      int is_xyz, const double* edges, int K, int is_auto,
                      unsigned long long* counts, const wtheta_tune* tune,
                      unsigned long long* stats, cudaStream_t st) {
    TraceRange trace("wtheta_count");
    if (!counts || n_a < 0 || n_b < 0 || (is_auto != 0 && is_auto != 1) ||
        (is_xyz != 0 && is_xyz != 1))
        return WTHETA_EINVAL;
    if (n_a > 0 && !ca) return WTHETA_EINVAL;
    if (is_auto) {
        if (cb && cb != ca) return WTHETA_EINVAL;
        if (n_b != n_a && !(cb == nullptr && n_b == 0)) return WTHETA_EINVAL;
        cb = ca;
        n_b = n_a;
    } else if (n_b > 0 && !cb) {
        return WTHETA_EINVAL;
    }
    if (tune && (tune->threads < 0 || tune->points_per_thread < 0 || tune->hist_mode < 0 ||
                 tune->hist_mode > 4 || tune->j_per_screen < 0 || tune->j_per_screen > 2 ||
                 tune->deferred < 0 || tune->deferred > 2 || tune->blocks_per_sm < 0 ||
                 tune->skip_far < 0 || tune->skip_far > 2 || tune->span_bins < 0 ||
                 tune->span_bins > 2))
        return WTHETA_EINVAL;
    static thread_local BinTable tab;  // large; built per call on the host
    int rc = build_table(edges, K, &tab);
    if (rc) return rc;
    DeviceInfo di;
    if ((rc = device_info(&di))) return rc;

    if ((rc = check_cuda(cudaMemsetAsync(counts, 0, sizeof(unsigned long long) * (K + 2), st))))
        return rc;
    const unsigned long long total =
        is_auto ? (unsigned long long)n_a * (unsigned long long)(n_a > 0 ? n_a - 1 : 0) / 2ull
                : (unsigned long long)n_a * (unsigned long long)n_b;
    const bool empty = is_auto ? n_a < 2 : (n_a == 0 || n_b == 0);
    if (empty) {
        k_finalize<<<1, 1, 0, st>>>(counts, K, total);
        count_launch();
        return check_cuda(cudaGetLastError());
    }

    const Variant* v = pick_for_size(tune, std::max(n_a, n_b), K, tab.n_lut, di.max_smem_optin);
    if (!v) return WTHETA_EINVAL;  // no instantiated shape matches the tuning request
    const long long T = (long long)v->nt * v->r;  // TA == TB
    const long long pa = round_up(n_a, T), pb = is_auto ? pa : round_up(n_b, T);

    const long long ta = pa / T, tb = pb / T;
    const long long n_items = is_auto ? ta * (ta + 1) / 2 : ta * tb;
    const size_t smem = v->smem(K, tab.n_lut);
    const int want_per_sm = tune && tune->blocks_per_sm ? tune->blocks_per_sm : 0;
    int resident = 0;  // blocks resident at once
    if ((rc = grid_for(v, smem, 1LL << 40, di.sm_count, want_per_sm, &resident))) return rc;
    // skip tile pairs wholly beyond the top edge (their pairs are overflow),
    // unless the items fill at most two waves of the launch: the caps and the
    // culling launches then cost about what they could save
    const bool skip_far = (!tune || tune->skip_far != 2) && edges[K] < 180.0 && n_items > 0 &&
                          n_items < (1LL << 32) &&
                          (n_items > 2LL * resident || (tune && tune->skip_far == 1));

    // scratch: the cursor and the kept count, both catalogues prepared
    // together, then the tile caps and the kept list
    const size_t bp = prepare_joint_bytes(n_a, pa, is_auto ? 0 : n_b, is_auto ? 0 : pb);
    const size_t off_caps = 256 + (bp + 255) / 256 * 256;
    const size_t off_list = off_caps + (skip_far ? ((size_t)(ta + tb) * sizeof(TileCap) + 255) / 256 * 256 : 0);
    const size_t bytes = off_list + (skip_far ? (size_t)n_items * 4 : 0);
    void* scratch = nullptr;
    if ((rc = dev_malloc_async(&scratch, bytes, st))) return rc;
    unsigned char* sp = (unsigned char*)scratch;
    unsigned long long* cursor = (unsigned long long*)sp;
    Prepared A, B;
    rc = prepare_joint(ca, n_a, pa, is_auto ? nullptr : cb, is_auto ? 0 : n_b, is_auto ? 0 : pb,
                       is_xyz, 0, sp + 256, di.sm_count, st, &A, &B);
    if (is_auto) B = A;
    if (!rc) rc = check_cuda(cudaMemsetAsync(cursor, 0, 2 * sizeof(unsigned long long), st));

    unsigned* list = nullptr;
    unsigned long long* n_list = nullptr;
    if (!rc && skip_far) {
        n_list = cursor + 1;
        TileCap* caps_a = (TileCap*)(sp + off_caps);
        TileCap* caps_b = is_auto ? caps_a : caps_a + ta;
        list = (unsigned*)(sp + off_list);
        // one launch over both catalogues (b's tiles follow a's)
        k_tile_caps<<<(unsigned)(is_auto ? ta : ta + tb), 128, 0, st>>>(A.p32, is_auto ? pa : pa + pb,
                                                                     (int)T, caps_a);
        const double theta_top = edges[K] * (3.14159265358979323846 / 180.0);
        k_cull_items<<<launch_grid(n_items, di.sm_count), 256, 0, st>>>(
            caps_a, caps_b, ta, tb, is_auto, n_items, theta_top, list, n_list, stats);
        count_launch(2);
        rc = check_cuda(cudaGetLastError());
    }
    int grid = 0;
    if (!rc) rc = grid_for(v, smem, n_items, di.sm_count, want_per_sm, &grid);
    if (!rc) {
        Segment seg = make_segment(A, B, ta, tb, is_auto, 0, counts, total);
        seg.item_list = list;
        PairParams prm = make_params(v, tab, &seg, nullptr, 0, 0, n_items, cursor, stats);
        prm.n_items_dev = n_list;
        prm.span = !(tune && tune->span_bins == 2);
        pair_kernel(v, prm)<<<grid, v->nt, smem, st>>>(prm);
        count_launch();
        rc = check_cuda(cudaGetLastError());
        if (!rc) {
            k_finalize<<<1, 1, 0, st>>>(counts, K, total);
            count_launch();
            rc = check_cuda(cudaGetLastError());
        }
    }
    const cudaError_t fe = cudaFreeAsync(scratch, st);
    if (!rc) rc = check_cuda(fe);
    return rc;
}

// Pairs (i < j) of an auto count of n points whose first point i is in the
// sorted rows [r0, r1).
static unsigned long long auto_pairs_in_rows(long long n, long long r0, long long r1) {
    if (r1 <= r0) return 0ull;
    const unsigned long long a = (unsigned long long)r0, b = (unsigned long long)r1;
    return (b - a) * (unsigned long long)(n - 1) - (b * (b - 1) / 2 - (a ? a * (a - 1) / 2 : 0ull));
}

// First item (tile pair) of tile row I: auto counts enumerate the upper
// triangle row by row (row I holds t - I items), cross counts the rectangle.
static long long row_item(long long I, long long ta, long long tb, int is_auto) {
    return is_auto ? I * ta - I * (I - 1) / 2 : I * tb;
}

// The three counts of one w(theta) (DD, DR, RR) in one persistent launch:
// each catalogue is prepared once, far tile pairs of each count are skipped
// on the device, and the counts are three segments of one work table, so
// there is one launch tail instead of three.  counts: device, 3 x (K+2).
//
// With n_shards > 1 only shard `shard` of each count is counted: the tile
// rows of the count (points of its first catalogue in the spatial order) are
// split into n_shards contiguous ranges holding equal numbers of kept tile
// pairs (one synchronisation brings the kept tile pairs per row to the host),
// and the shard counts the pairs whose first point lies in its rows, overflow
// slot included; the shards' counts add up to the whole count.
static int count_wtheta_impl(const double* cd, long long nd, const double* cr, long long nr,
                             int is_xyz, const double* edges, int K,
                             unsigned long long* counts, const wtheta_tune* tune,
                             unsigned long long* stats, cudaStream_t st, int shard = 0,
                             int n_shards = 1) {
    TraceRange trace("wtheta_count_wtheta");
    if (!counts || nd < 0 || nr < 0 || (nd > 0 && !cd) || (nr > 0 && !cr) ||
        (is_xyz != 0 && is_xyz != 1) || n_shards < 1 || shard < 0 || shard >= n_shards)
        return WTHETA_EINVAL;
    if (tune && (tune->threads < 0 || tune->points_per_thread < 0 || tune->hist_mode < 0 ||
                 tune->hist_mode > 4 || tune->j_per_screen < 0 || tune->j_per_screen > 2 ||
                 tune->deferred < 0 || tune->deferred > 2 || tune->blocks_per_sm < 0 ||
                 tune->skip_far < 0 || tune->skip_far > 2 || tune->span_bins < 0 ||
                 tune->span_bins > 2))
        return WTHETA_EINVAL;
    static thread_local BinTable tab;
    int rc = build_table(edges, K, &tab);
    if (rc) return rc;
    DeviceInfo di;
    if ((rc = device_info(&di))) return rc;
    const size_t K2 = (size_t)K + 2;
    if ((rc = check_cuda(cudaMemsetAsync(counts, 0, 3 * K2 * 8, st)))) return rc;
    const Variant* v = pick_for_size(tune, std::max(nd, nr), K, tab.n_lut, di.max_smem_optin);
    if (!v) return WTHETA_EINVAL;
    const long long T = (long long)v->nt * v->r;
    const long long pd = round_up(nd, T), pr = round_up(nr, T);
    const long long td = pd / T, tr = pr / T;
    const unsigned long long ndd = (unsigned long long)nd * (unsigned long long)(nd > 0 ? nd - 1 : 0) / 2;
    const unsigned long long ndr = (unsigned long long)nd * (unsigned long long)nr;
    const unsigned long long nrr = (unsigned long long)nr * (unsigned long long)(nr > 0 ? nr - 1 : 0) / 2;
    // the counts with work, biggest first
    struct Cnt {
        int kind;
        long long items;            // tile pairs of the count (of the shard's rows)
        unsigned long long total;   // pairs of the count (of the shard's rows)
        long long offset;           // first item of the shard's rows
    };
    Cnt all[3] = {{0, td * (td + 1) / 2, ndd, 0}, {1, td * tr, ndr, 0}, {2, tr * (tr + 1) / 2, nrr, 0}};
    std::vector<Cnt> cnts;
    for (const Cnt& c : all)
        if (c.total > 0) cnts.push_back(c);
    std::stable_sort(cnts.begin(), cnts.end(),
                     [](const Cnt& a, const Cnt& b) { return a.items > b.items; });
    const int n_segs = (int)cnts.size();
    long long total_items = 0;
    for (const Cnt& c : cnts) total_items += c.items;
    const size_t smem = v->smem(K, tab.n_lut);
    const int want_per_sm = tune && tune->blocks_per_sm ? tune->blocks_per_sm : 0;
    int resident = 0;  // blocks resident at once
    if ((rc = grid_for(v, smem, 1LL << 40, di.sm_count, want_per_sm, &resident))) return rc;
    // skip far tile pairs unless the items fill at most two waves of the
    // launch (the caps and the culling launches then cost about what they
    // could save) or a shard split needs the kept items per row
    const bool cull = (!tune || tune->skip_far != 2) && edges[K] < 180.0 && td * td < (1LL << 32) &&
                      td * tr < (1LL << 32) && tr * tr < (1LL << 32) &&
                      (total_items > 2LL * resident || n_shards > 1 || (tune && tune->skip_far == 1));
    // scratch: cursor and kept total, segments, culling table, kept counts,
    // both catalogues prepared together, tile caps, kept lists (and kept
    // items per row)
    const size_t bp = prepare_joint_bytes(nd, pd, nr, pr);
    size_t bytes = 256 + 1024 + 1024 + 256;
    const size_t off_prep = bytes;
    bytes += (bp + 255) / 256 * 256;
    const size_t off_caps = bytes;
    if (cull) bytes += ((size_t)(td + tr) * sizeof(TileCap) + 255) / 256 * 256;
    const size_t off_rows = bytes;
    if (n_shards > 1) bytes += ((size_t)(2 * td + tr) * 8 + 255) / 256 * 256 + 256;
    const size_t off_lists = bytes;
    if (cull) bytes += (size_t)total_items * 4;
    unsigned char* m = nullptr;
    if ((rc = dev_malloc_async((void**)&m, bytes, st))) return rc;
    unsigned long long* cursor = (unsigned long long*)m;
    unsigned long long* n_kept = cursor + 1;
    Segment* d_segs = (Segment*)(m + 256);
    CullSeg* d_cull = (CullSeg*)(m + 256 + 1024);
    unsigned long long* d_kept = (unsigned long long*)(m + 256 + 2048);
    static_assert(3 * sizeof(Segment) <= 1024 && 3 * sizeof(CullSeg) <= 1024, "tables fit");
    Prepared D, R;
    rc = prepare_joint(cd, nd, pd, cr, nr, pr, is_xyz, 0, m + off_prep, di.sm_count, st, &D, &R);
    TileCap* caps_d = (TileCap*)(m + off_caps);
    TileCap* caps_r = caps_d + td;  // R's tiles follow D's in the joint copies
    if (!rc && (cull || n_shards > 1) && td + tr > 0)
        rc = launch_tile_caps(D.p32, pd + pr, (int)T, td + tr, caps_d, st);
    const double theta_top = edges[K] * (3.14159265358979323846 / 180.0);
    auto cull_seg = [&](int i, long long begin) {
        const int k = cnts[i].kind;
        CullSeg c;
        std::memset(&c, 0, sizeof(CullSeg));
        c.begin = begin;
        c.n = cnts[i].items;
        c.offset = cnts[i].offset;
        c.ta = k == 2 ? tr : td;
        c.tb = k == 0 ? td : tr;
        c.is_auto = k != 1;
        c.ca = k == 2 ? caps_r : caps_d;
        c.cb = k == 0 ? caps_d : caps_r;
        return c;
    };
    if (!rc && n_shards > 1 && n_segs > 0) {
        // kept tile pairs per tile row of every count (all tile pairs count when
        // nothing is skipped), then this shard's rows of each count
        long long row0[3], nrow[3], item = 0;
        CullSeg cs[3];
        for (int i = 0; i < n_segs; ++i) {
            cs[i] = cull_seg(i, item);
            item += cnts[i].items;
            row0[i] = i == 0 ? 0 : row0[i - 1] + nrow[i - 1];
            nrow[i] = cnts[i].kind == 2 ? tr : td;
        }
        unsigned long long* d_rows = (unsigned long long*)(m + off_rows);
        long long* d_row0 = (long long*)(m + off_rows + ((size_t)(2 * td + tr) * 8 + 255) / 256 * 256);
        const long long n_rows = row0[n_segs - 1] + nrow[n_segs - 1];
        std::vector<unsigned long long> rows(n_rows);
        rc = check_cuda(cudaMemsetAsync(d_rows, 0, (size_t)n_rows * 8, st));
        if (!rc) rc = check_cuda(cudaMemcpyAsync(d_cull, cs, sizeof(CullSeg) * n_segs,
                                                 cudaMemcpyHostToDevice, st));
        if (!rc) rc = check_cuda(cudaMemcpyAsync(d_row0, row0, sizeof(row0), cudaMemcpyHostToDevice, st));
        if (!rc) {
            k_cull_rows<<<launch_grid(total_items, di.sm_count), 256, 0, st>>>(
                d_cull, n_segs, total_items, cull ? theta_top : 4.0, d_row0, d_rows);
            count_launch();
            rc = check_cuda(cudaGetLastError());
        }
        if (!rc) rc = check_cuda(cudaMemcpyAsync(rows.data(), d_rows, (size_t)n_rows * 8,
                                                 cudaMemcpyDeviceToHost, st));
        if (!rc) rc = check_cuda(cudaStreamSynchronize(st));
        for (int i = 0; i < n_segs && !rc; ++i) {
            const int k = cnts[i].kind;
            const int aut = k != 1;
            long long I0 = 0, I1 = 0;
            rc = wtheta_shard_weights((const uint64_t*)rows.data() + row0[i], nrow[i], shard, n_shards,
                                      (int64_t*)&I0, (int64_t*)&I1);
            const long long ta = k == 2 ? tr : td, tb = k == 0 ? td : tr;
            const long long n_a = k == 2 ? nr : nd, n_b = k == 0 ? nd : nr;
            const long long r0 = std::min(I0 * T, n_a), r1 = std::min(I1 * T, n_a);
            cnts[i].offset = row_item(I0, ta, tb, aut);
            cnts[i].items = row_item(I1, ta, tb, aut) - cnts[i].offset;
            cnts[i].total = aut ? auto_pairs_in_rows(n_a, r0, r1)
                                : (unsigned long long)(r1 - r0) * (unsigned long long)n_b;
        }
        total_items = 0;
        for (const Cnt& c : cnts) total_items += c.items;
    }
    Segment segs[3];
    CullSeg cs[3];
    long long item = 0;
    for (int i = 0; i < n_segs; ++i) {
        const int k = cnts[i].kind;
        const Prepared& A = k == 2 ? R : D;
        const Prepared& B = k == 0 ? D : R;
        const long long ta = k == 2 ? tr : td, tb = k == 0 ? td : tr;
        segs[i] = make_segment(A, B, ta, tb, k != 1, item, counts + (size_t)k * K2, cnts[i].total);
        segs[i].n_items = cnts[i].items;
        segs[i].item_offset = cnts[i].offset;
        cs[i] = cull_seg(i, item);
        cs[i].list = (unsigned*)(m + off_lists) + item;
        item += cnts[i].items;
    }
    if (!rc && n_segs > 0) {
        // the segments and culling table, cursor and kept counters zeroed: one
        // small launch instead of copies from pageable memory and memsets
        CountTables tbl;
        std::memset(&tbl, 0, sizeof(tbl));
        for (int i = 0; i < n_segs; ++i) {
            tbl.segs[i] = segs[i];
            tbl.cs[i] = cs[i];
        }
        tbl.n_segs = n_segs;
        tbl.with_cull = cull ? 1 : 0;
        k_set_tables<<<1, 32, 0, st>>>(tbl, d_segs, d_cull, cursor, 2, d_kept, cull ? 3 : 0);
        count_launch();
        rc = check_cuda(cudaGetLastError());
        if (!rc && cull)
            rc = launch_cull_batch(d_cull, n_segs, total_items, theta_top, d_kept, d_segs, n_kept,
                                   di.sm_count, st, stats);
        int grid = 0;
        if (!rc) rc = grid_for(v, smem, std::max(total_items, 1LL), di.sm_count, want_per_sm, &grid);
        if (!rc && total_items > 0) {
            PairParams prm = make_params(v, tab, nullptr, d_segs, n_segs, 0, total_items, cursor,
                                         stats);
            if (cull) prm.n_items_dev = n_kept;
            prm.span = !(tune && tune->span_bins == 2);
            rc = launch_pairs(v, prm, grid, smem, st);
        }
        if (!rc) rc = launch_finalize_segments(d_segs, n_segs, K, st);
    }
    const cudaError_t fe = cudaFreeAsync(m, st);
    if (!rc) rc = check_cuda(fe);
    return rc;
}

int launch_pairs(const Variant* v, const PairParams& prm, int grid, size_t smem,
                 cudaStream_t st) {
    pair_kernel(v, prm)<<<grid, v->nt, smem, st>>>(prm);
    count_launch();
    return check_cuda(cudaGetLastError());
}

int launch_finalize_segments(const Segment* d_segs, int n_segs, int K, cudaStream_t st) {
    if (n_segs <= 0) return WTHETA_OK;
    k_finalize_segments<<<(n_segs + 127) / 128, 128, 0, st>>>(d_segs, n_segs, K);
    count_launch();
    return check_cuda(cudaGetLastError());
}

int launch_tile_caps(const float4* p32, long long n, int T, long long tiles, TileCap* caps,
                     cudaStream_t st) {
    if (tiles <= 0) return WTHETA_OK;
    k_tile_caps<<<(unsigned)tiles, 128, 0, st>>>(p32, n, T, caps);
    count_launch();
    return check_cuda(cudaGetLastError());
}

int launch_cull_items(const TileCap* ca, const TileCap* cb, long long ta, long long tb,
                      int is_auto, long long n_items, double theta_top, unsigned* list,
                      unsigned long long* n_list, int sm_count, cudaStream_t st) {
    if (n_items <= 0) return WTHETA_OK;
    k_cull_items<<<launch_grid(n_items, sm_count), 256, 0, st>>>(ca, cb, ta, tb, is_auto, n_items,
                                                                   theta_top, list, n_list, nullptr);
    count_launch();
    return check_cuda(cudaGetLastError());
}

void add_launches(long long n) { g_launches.fetch_add((unsigned long long)n); }

// -1: no injected failure; n >= 0: the allocation after n more succeed fails
static std::atomic<long long> g_fail_alloc{-1};

static bool injected_failure() {
    long long v = g_fail_alloc.load();
    while (v >= 0) {
        if (g_fail_alloc.compare_exchange_weak(v, v - 1)) return v == 0;
    }
    return false;
}

int dev_malloc(void** p, size_t bytes) {
    if (injected_failure()) return WTHETA_ENOMEM;
    const cudaError_t e = cudaMalloc(p, bytes);
    if (e == cudaErrorMemoryAllocation) {
        cudaGetLastError();
        return WTHETA_ENOMEM;
    }
    return check_cuda(e);
}

int dev_malloc_async(void** p, size_t bytes, cudaStream_t st) {
    if (injected_failure()) return WTHETA_ENOMEM;
    const cudaError_t e = cudaMallocAsync(p, bytes, st);
    if (e == cudaErrorMemoryAllocation) {
        cudaGetLastError();
        return WTHETA_ENOMEM;
    }
    return check_cuda(e);
}

TraceRange::TraceRange(const char* name) { nvtxRangePushA(name); }
TraceRange::~TraceRange() { nvtxRangePop(); }

// ---------------------------------------------------------------------------
// allocation-free variant of the xyz count
// ---------------------------------------------------------------------------
// The fixed scratch of wtheta_count_xyz_noalloc: a 256-byte head holding the
// work cursor, then FP32 float4 copies of catalogue a and (cross counts)
// catalogue b, each padded to whole tiles.  It is loaded with the library's
// module on every device that uses it and lives until the process exits.
static __device__ __align__(256) unsigned char
    g_noalloc_scratch[256 + 16 * (size_t)WTHETA_NOALLOC_MAX_POINTS];

// Device address of g_noalloc_scratch on the current device.  In host code
// the symbol names a host-side stand-in, not device memory, so the address is
// looked up once per device (with that device current) and cached.
static int noalloc_scratch(unsigned char** out) {
    static std::mutex mu;
    static void* addr[64] = {};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return WTHETA_ECUDA;
    std::lock_guard<std::mutex> g(mu);
    if (!addr[dev]) {
        void* p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || p == nullptr) return WTHETA_ECUDA;
        addr[dev] = p;
    }
    *out = (unsigned char*)addr[dev];
    return WTHETA_OK;
}

static int count_xyz_noalloc_impl(const double* ca, long long n_a, const double* cb,
                                  long long n_b, const double* edges, int K, int is_auto,
                                  unsigned long long* counts, cudaStream_t st) {
    if (!counts || n_a < 0 || n_b < 0 || (is_auto != 0 && is_auto != 1)) return WTHETA_EINVAL;
    if (n_a > 0 && !ca) return WTHETA_EINVAL;
    if (is_auto) {
        if (cb && cb != ca) return WTHETA_EINVAL;
        if (n_b != n_a && !(cb == nullptr && n_b == 0)) return WTHETA_EINVAL;
        cb = ca;
        n_b = n_a;
    } else if (n_b > 0 && !cb) {
        return WTHETA_EINVAL;
    }
    const long long T = WTHETA_NOALLOC_TILE;
    // each size alone first, so that the rounding below cannot overflow
    if (n_a > (long long)WTHETA_NOALLOC_MAX_POINTS || n_b > (long long)WTHETA_NOALLOC_MAX_POINTS)
        return WTHETA_ESIZE;
    const long long pa = round_up(n_a, T), pb = is_auto ? 0 : round_up(n_b, T);
    if (pa + pb > (long long)WTHETA_NOALLOC_MAX_POINTS) return WTHETA_ESIZE;
    static thread_local BinTable tab;
    int rc = build_table(edges, K, &tab);
    if (rc) return rc;
    DeviceInfo di;
    if ((rc = device_info(&di))) return rc;
    unsigned char* base = nullptr;
    if ((rc = noalloc_scratch(&base))) return rc;

    if ((rc = check_cuda(cudaMemsetAsync(counts, 0, sizeof(unsigned long long) * (K + 2), st))))
        return rc;
    const unsigned long long total =
        is_auto ? (unsigned long long)n_a * (unsigned long long)(n_a > 0 ? n_a - 1 : 0) / 2ull
                : (unsigned long long)n_a * (unsigned long long)n_b;
    const bool empty = is_auto ? n_a < 2 : (n_a == 0 || n_b == 0);
    if (empty) {
        k_finalize<<<1, 1, 0, st>>>(counts, K, total);
        count_launch();
        return check_cuda(cudaGetLastError());
    }
    wtheta_tune fixed = {128, 8, 0, 0, 0, 0, 2, 2};  // the tile of WTHETA_NOALLOC_TILE points
    const Variant* v = pick_variant(&fixed, K, tab.n_lut, di.max_smem_optin);
    if (!v || (long long)v->nt * v->r != T) return WTHETA_EINVAL;

    unsigned long long* cursor = (unsigned long long*)base;
    float4* a32 = (float4*)(base + 256);
    float4* b32 = is_auto ? a32 : a32 + pa;
    const int cvt_threads = 256;
    auto cvt_grid = [&](long long n) {
        long long g = (n + cvt_threads - 1) / cvt_threads;
        return (int)std::min<long long>(std::max<long long>(g, 1), (long long)di.sm_count * 16);
    };
    // every word the kernels read is rewritten here: both padded copies and the cursor
    k_xyz_to_f32<<<cvt_grid(pa), cvt_threads, 0, st>>>(ca, n_a, pa, a32, 0);
    count_launch();
    if (!is_auto) {
        k_xyz_to_f32<<<cvt_grid(pb), cvt_threads, 0, st>>>(cb, n_b, pb, b32, 1);
        count_launch();
    }
    if ((rc = check_cuda(cudaMemsetAsync(cursor, 0, sizeof(unsigned long long), st)))) return rc;
    const long long ta = pa / T, tb = is_auto ? ta : pb / T;
    const long long n_items = is_auto ? ta * (ta + 1) / 2 : ta * tb;
    const size_t smem = v->smem(K, tab.n_lut);
    int grid = 0;
    if ((rc = grid_for(v, smem, n_items, di.sm_count, 0, &grid))) return rc;
    Prepared A, B;
    A.p32 = a32; A.x64 = ca; A.stride = n_a;
    B.p32 = b32; B.x64 = cb; B.stride = n_b;
    const Segment seg = make_segment(A, B, ta, tb, is_auto, 0, counts, total);
    const PairParams prm = make_params(v, tab, &seg, nullptr, 0, 0, n_items, cursor, nullptr);
    pair_kernel(v, prm)<<<grid, v->nt, smem, st>>>(prm);
    count_launch();
    if ((rc = check_cuda(cudaGetLastError()))) return rc;
    k_finalize<<<1, 1, 0, st>>>(counts, K, total);
    count_launch();
    return check_cuda(cudaGetLastError());
}

}  // namespace wtheta

// ---------------------------------------------------------------------------
// batched counts: one work queue over many catalogue pairs, one graph
// ---------------------------------------------------------------------------

struct wtheta_plan {
    int dev = 0;
    int K = 0;
    int n_cats = 0;
    int is_xyz = 0;                        // catalogues are SoA unit vectors, not RA/Dec
    wtheta::BinTable tab;
    const wtheta::Variant* v = nullptr;
    wtheta_tune tune = {};
    int autotuned = 0;
    float autotune_ms = 0.f;
    std::vector<wtheta_catalog_pair> cats;
    void* scratch = nullptr;               // prepared copies of every catalogue
    std::vector<wtheta::Prepared> prep;    // 2 per catalogue pair
    std::vector<long long> n_pad;
    // all catalogues (data 2m, randoms 2m + 1) are prepared together: one FP64
    // array of every point, one sort by (catalogue, spatial key), FP32 copies
    // with every catalogue starting on a tile boundary
    std::vector<long long> src_off, dst_off;  // 2 n_cats + 1 each
    long long n_all = 0, n_all_pad = 0;
    wtheta::BatchCat* d_cats = nullptr;
    long long* d_src_off = nullptr;         // src_off, then dst_off (for the gather)
    double* x_all = nullptr;
    int* lab_all = nullptr;
    unsigned char* sort_scratch = nullptr;
    float4* p32_all = nullptr;
    float4* c32_all = nullptr;
    wtheta::TileCap* caps_all = nullptr;
    wtheta::Segment* d_segs = nullptr;
    int n_segs = 0;
    long long total_items = 0;
    long long pairs = 0;
    unsigned long long* d_counts = nullptr;  // internal: [cat][kind][K+2]
    unsigned long long* d_cursor = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    int graph_kernels = 0;
    int grid = 0;
    size_t smem = 0;
    long long runs = 0;
    // skipping of far tile pairs, done in the graph on every run
    int cull = 0;
    double theta_top = 0.0;
    void* cull_mem = nullptr;
    wtheta::CullSeg* d_cull = nullptr;        // per count, in the work table's order
    unsigned long long* d_kept = nullptr;     // per count
    unsigned long long* d_total = nullptr;    // kept items of the run
    unsigned long long* d_stats = nullptr;    // WTHETA_NSTATS of the last run
    std::vector<wtheta::TileCap*> caps;       // per catalogue
    int sm_count = 0;
};

namespace wtheta {

// Autotuner cache: the shape picked for batches of similar work on a device
// of this size, keyed by (SM count, K, log2 of the batch's pair count).
struct TuneKey {
    int sm, K, size_bucket;
};
static std::mutex g_tune_mu;
static std::vector<std::pair<TuneKey, int>> g_tune_cache;

static int lookup_tuned(const TuneKey& k) {
    std::lock_guard<std::mutex> g(g_tune_mu);
    for (auto& e : g_tune_cache)
        if (e.first.sm == k.sm && e.first.K == k.K && e.first.size_bucket == k.size_bucket)
            return e.second;
    return -1;
}

static void store_tuned(const TuneKey& k, int idx) {
    std::lock_guard<std::mutex> g(g_tune_mu);
    g_tune_cache.push_back({k, idx});
}

// Preparation of every catalogue of a plan, as one pipeline over all of them
// (a constant number of launches whatever the number of catalogues):
// conversion into one FP64 array with a catalogue label per point, one
// spatial sort by (catalogue, key), FP32 copies with every catalogue starting
// on a tile boundary (sentinels in the rest of its last tile), chunk spheres
// and, when far tile pairs are skipped, tile caps.  Reads the catalogues'
// current contents (the graph replays it on every run).
static int batch_prepare(wtheta_plan* P, int T, cudaStream_t st) {
    const int nc2 = 2 * P->n_cats;
    if (P->n_all <= 0) return WTHETA_OK;
    k_batch_gather<<<launch_grid(P->n_all, P->sm_count), 256, 0, st>>>(
        P->d_cats, P->d_src_off, nc2, P->is_xyz, P->n_all, P->x_all, P->lab_all);
    count_launch();
    const unsigned* order = nullptr;
    int rc = spatial_order(P->x_all, P->n_all, P->n_all, P->is_xyz, P->lab_all, nc2,
                           P->sort_scratch, P->sm_count, st, &order, nullptr);
    if (!rc)
        rc = launch_gather_regions(P->x_all, P->n_all, order, P->d_src_off, P->d_src_off + nc2 + 1,
                                   nc2, P->n_all_pad, P->p32_all, 0, P->sm_count, st);
    if (!rc) rc = launch_chunk_caps(P->p32_all, P->n_all_pad, P->c32_all, P->sm_count, st);
    if (!rc && P->cull)
        rc = launch_tile_caps(P->p32_all, P->n_all_pad, T, P->n_all_pad / T, P->caps_all, st);
    return rc;
}

// Lays out the plan's scratch and work table for one kernel shape (its tile
// T = threads x points_per_thread), prepares every catalogue on stream st.
static int plan_layout(wtheta_plan* P, const Variant* v, int sm_count, cudaStream_t st) {
    const long long T = (long long)v->nt * v->r;
    const int nc = P->n_cats, nc2 = 2 * nc;
    P->sm_count = sm_count;
    P->n_pad.assign(nc2, 0);
    P->src_off.assign(nc2 + 1, 0);
    P->dst_off.assign(nc2 + 1, 0);
    std::vector<BatchCat> hc(nc2);
    for (int c = 0; c < nc2; ++c) {
        const wtheta_catalog_pair& q = P->cats[c / 2];
        hc[c].src = c % 2 ? q.rand : q.data;
        hc[c].n = c % 2 ? q.n_rand : q.n_data;
        P->n_pad[c] = round_up(hc[c].n, T);
        P->src_off[c + 1] = P->src_off[c] + hc[c].n;
        P->dst_off[c + 1] = P->dst_off[c] + P->n_pad[c];
    }
    P->n_all = P->src_off[nc2];
    P->n_all_pad = P->dst_off[nc2];
    const long long N = P->n_all, NP = P->n_all_pad;
    auto a256 = [](size_t b) { return (b + 255) / 256 * 256; };
    // scratch: the cursor head, the catalogue table and offsets, the FP64
    // array and labels, the sort, the FP32 copies and chunk spheres
    size_t bytes = 256;
    const size_t off_cats = bytes;
    bytes += a256((size_t)nc2 * sizeof(BatchCat));
    const size_t off_offs = bytes;
    bytes += a256((size_t)2 * (nc2 + 1) * 8);
    const size_t off_x = bytes;
    bytes += a256((size_t)N * 24);
    const size_t off_lab = bytes;
    bytes += a256((size_t)N * 4);
    const size_t off_sort = bytes;
    bytes += a256(order_bytes(N, 1));
    const size_t off_p32 = bytes;
    bytes += a256((size_t)NP * 16);
    const size_t off_c32 = bytes;
    bytes += a256((size_t)NP / 32 * 16);
    if (P->scratch) cudaFree(P->scratch);
    P->scratch = nullptr;
    int rc = dev_malloc(&P->scratch, bytes);
    if (rc) return rc;
    unsigned char* base = (unsigned char*)P->scratch;
    P->d_cursor = (unsigned long long*)base;
    P->d_cats = (BatchCat*)(base + off_cats);
    P->d_src_off = (long long*)(base + off_offs);
    P->x_all = (double*)(base + off_x);
    P->lab_all = (int*)(base + off_lab);
    P->sort_scratch = base + off_sort;
    P->p32_all = (float4*)(base + off_p32);
    P->c32_all = (float4*)(base + off_c32);
    std::vector<long long> offs(P->src_off);
    offs.insert(offs.end(), P->dst_off.begin(), P->dst_off.end());
    rc = check_cuda(cudaMemcpyAsync(P->d_cats, hc.data(), sizeof(BatchCat) * nc2,
                                    cudaMemcpyHostToDevice, st));
    if (!rc) rc = check_cuda(cudaMemcpyAsync(P->d_src_off, offs.data(), offs.size() * 8,
                                             cudaMemcpyHostToDevice, st));
    if (rc) return rc;
    // every catalogue's view of the shared copies (FP64 in the caller's order:
    // the FP32 copies carry each point's position in the FP64 array)
    P->prep.assign(nc2, Prepared());
    for (int c = 0; c < nc2; ++c) {
        Prepared& q = P->prep[c];
        q.p32 = P->p32_all + P->dst_off[c];
        q.c32 = P->c32_all + P->dst_off[c] / 32;
        q.x64 = P->x_all;
        q.stride = N;
        q.sorted = 0;
    }
    // the work table: DD, DR, RR of every pair, biggest count first
    std::vector<Segment> segs;
    std::vector<int> seg_cat_a, seg_cat_b;  // prepared catalogue of each side
    P->pairs = 0;
    for (int m = 0; m < nc; ++m) {
        const long long nd = P->cats[m].n_data, nr = P->cats[m].n_rand;
        const long long td = P->n_pad[2 * m] / T, tr = P->n_pad[2 * m + 1] / T;
        unsigned long long* c = P->d_counts + (size_t)3 * m * (P->K + 2);
        const unsigned long long ndd = (unsigned long long)nd * (unsigned long long)(nd - 1) / 2;
        const unsigned long long ndr = (unsigned long long)nd * (unsigned long long)nr;
        const unsigned long long nrr = (unsigned long long)nr * (unsigned long long)(nr - 1) / 2;
        P->pairs += (long long)(ndd + ndr + nrr);
        segs.push_back(make_segment(P->prep[2 * m], P->prep[2 * m], td, td, 1, 0, c, ndd));
        segs.push_back(make_segment(P->prep[2 * m], P->prep[2 * m + 1], td, tr, 0, 0,
                                    c + (P->K + 2), ndr));
        segs.push_back(make_segment(P->prep[2 * m + 1], P->prep[2 * m + 1], tr, tr, 1, 0,
                                    c + 2 * (P->K + 2), nrr));
        seg_cat_a.insert(seg_cat_a.end(), {2 * m, 2 * m, 2 * m + 1});
        seg_cat_b.insert(seg_cat_b.end(), {2 * m, 2 * m + 1, 2 * m + 1});
    }
    std::vector<int> order(segs.size());
    for (size_t i = 0; i < order.size(); ++i) order[i] = (int)i;
    std::stable_sort(order.begin(), order.end(),
                     [&](int a, int b) { return segs[a].n_items > segs[b].n_items; });
    std::vector<Segment> sorted;
    std::vector<CullSeg> cull(segs.size());
    long long items = 0;
    for (size_t i = 0; i < order.size(); ++i) {
        Segment g = segs[order[i]];
        g.item_begin = items;
        CullSeg& q = cull[i];
        std::memset(&q, 0, sizeof(q));
        q.begin = items;
        q.n = g.n_items;
        q.ta = g.tiles_a;
        q.tb = g.tiles_b;
        q.is_auto = g.is_auto;
        items += g.n_items;
        sorted.push_back(g);
    }
    P->total_items = items;
    P->n_segs = (int)sorted.size();
    if (P->d_segs) cudaFree(P->d_segs);
    P->d_segs = nullptr;
    if (P->cull_mem) cudaFree(P->cull_mem);
    P->cull_mem = nullptr;
    P->caps.assign(2 * nc, nullptr);
    if ((rc = dev_malloc((void**)&P->d_segs, sizeof(Segment) * sorted.size()))) return rc;
    if (P->cull) {
        // kept counters, total, the count table, the tile caps of all the
        // catalogues' tiles, and one list of item indices per count
        size_t cb = ((size_t)P->n_segs * 8 + 8 + 255) / 256 * 256;
        const size_t off_cs = cb;
        cb += (sizeof(CullSeg) * P->n_segs + 255) / 256 * 256;
        const size_t off_caps = cb;
        cb += ((size_t)(NP / T) * sizeof(TileCap) + 255) / 256 * 256;
        const size_t off_lists = cb;
        cb += (size_t)items * 4;
        if ((rc = dev_malloc(&P->cull_mem, cb))) return rc;
        unsigned char* cm = (unsigned char*)P->cull_mem;
        P->d_kept = (unsigned long long*)cm;
        P->d_total = P->d_kept + P->n_segs;
        P->d_cull = (CullSeg*)(cm + off_cs);
        P->caps_all = (TileCap*)(cm + off_caps);
        for (int c = 0; c < nc2; ++c) P->caps[c] = P->caps_all + P->dst_off[c] / T;
        unsigned* lists = (unsigned*)(cm + off_lists);
        for (size_t i = 0; i < order.size(); ++i) {
            cull[i].ca = P->caps[seg_cat_a[order[i]]];
            cull[i].cb = P->caps[seg_cat_b[order[i]]];
            cull[i].list = lists + cull[i].begin;
        }
        rc = check_cuda(cudaMemcpyAsync(P->d_cull, cull.data(), sizeof(CullSeg) * cull.size(),
                                        cudaMemcpyHostToDevice, st));
        if (rc) return rc;
    }
    rc = check_cuda(cudaMemcpyAsync(P->d_segs, sorted.data(), sizeof(Segment) * sorted.size(),
                                    cudaMemcpyHostToDevice, st));
    // the catalogues, prepared once now (for the autotuner's timing); the
    // graph prepares them again on every run
    if (!rc) rc = batch_prepare(P, (int)T, st);
    return rc;
}

static int launch_batch_pairs(wtheta_plan* P, const Variant* v, long long item_begin,
                              long long n_items, int grid, size_t smem, cudaStream_t st,
                              const unsigned long long* n_items_dev = nullptr,
                              unsigned long long* stats = nullptr) {
    PairParams prm = make_params(v, P->tab, nullptr, P->d_segs, P->n_segs, item_begin,
                                 n_items, P->d_cursor, stats);
    prm.span = P->tune.span_bins != 2;
    prm.n_items_dev = n_items_dev;
    pair_kernel(v, prm)<<<grid, v->nt, smem, st>>>(prm);
    count_launch();
    return check_cuda(cudaGetLastError());
}

// Times each candidate shape on the first items of the queue (the biggest
// counts) and keeps the fastest per pair.  Candidates share a tile size per
// layout; a different tile size re-lays the plan out.
static int autotune(wtheta_plan* P, const DeviceInfo& di, cudaStream_t st, int* best_idx) {
    int nv = 0;
    const Variant* vs = variants(&nv);
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)
        return WTHETA_ECUDA;
    float best = 1e30f;
    int rc = WTHETA_OK;
    long long cur_T = -1;
    for (int i = 0; i < nv && !rc; ++i) {
        const Variant* v = &vs[i];
        const size_t smem = v->smem(P->K, P->tab.n_lut);
        if (smem > (size_t)di.max_smem_optin) continue;
        const long long T = (long long)v->nt * v->r;
        if (T != cur_T) {
            if ((rc = plan_layout(P, v, di.sm_count, st))) break;
            cur_T = T;
        }
        int grid = 0;
        if ((rc = grid_for(v, smem, P->total_items, di.sm_count, 0, &grid))) break;
        // a sample of several items per CTA, from the front of the queue
        const long long n_sample =
            std::min<long long>(P->total_items, std::max<long long>(8LL * grid, P->total_items / 64));
        float ms = 0.f;
        for (int rep = 0; rep < 2 && !rc; ++rep) {  // first pass warms up
            rc = check_cuda(cudaMemsetAsync(P->d_cursor, 0, 8, st));
            if (!rc) rc = check_cuda(cudaEventRecord(e0, st));
            if (!rc) rc = launch_batch_pairs(P, v, 0, n_sample, grid, smem, st);
            if (!rc) rc = check_cuda(cudaEventRecord(e1, st));
            if (!rc) rc = check_cuda(cudaEventSynchronize(e1));
            if (!rc) rc = check_cuda(cudaEventElapsedTime(&ms, e0, e1));
        }
        if (rc) break;
        const float per = ms / ((float)n_sample * (float)T * (float)T);  // per pair
        if (per < best) {
            best = per;
            *best_idx = i;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return rc;
}

static int plan_capture(wtheta_plan* P, const DeviceInfo& di) {
    cudaStream_t cs;
    int rc = check_cuda(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
    if (rc) return rc;
    const unsigned long long launches0 = g_launches.load();
    rc = check_cuda(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
    if (!rc) {
        // re-prepare every catalogue from its current coordinates (one
        // pipeline over all of them, tile caps included), then count
        const int T = P->v->nt * P->v->r;
        rc = batch_prepare(P, T, cs);
        if (!rc && P->cull) {
            // the kept tile pairs of every count, and the launch's item ranges
            if (!rc) rc = check_cuda(cudaMemsetAsync(P->d_kept, 0, (size_t)P->n_segs * 8, cs));
            if (!rc) {
                k_cull_batch<<<launch_grid(P->total_items, di.sm_count), 256, 0, cs>>>(
                    P->d_cull, P->n_segs, P->total_items, P->theta_top, P->d_kept, nullptr);
                k_cull_prefix<<<1, 32, 0, cs>>>(P->d_segs, P->d_cull, P->d_kept, P->n_segs,
                                                P->d_total);
                count_launch(2);
                rc = check_cuda(cudaGetLastError());
            }
        }
        const size_t nbytes = (size_t)P->n_cats * 3 * (P->K + 2) * sizeof(unsigned long long);
        if (!rc) rc = check_cuda(cudaMemsetAsync(P->d_counts, 0, nbytes, cs));
        if (!rc) rc = check_cuda(cudaMemsetAsync(P->d_cursor, 0, 8, cs));
        if (!rc) rc = check_cuda(cudaMemsetAsync(P->d_stats, 0, 8 * WTHETA_NSTATS, cs));
        if (!rc)
            rc = launch_batch_pairs(P, P->v, 0, P->total_items, P->grid, P->smem, cs,
                                    P->cull ? P->d_total : nullptr, P->d_stats);
        if (!rc) {
            k_finalize_segments<<<(P->n_segs + 127) / 128, 128, 0, cs>>>(P->d_segs, P->n_segs,
                                                                        P->K);
            count_launch();
            rc = check_cuda(cudaGetLastError());
        }
        cudaGraph_t g = nullptr;
        const cudaError_t ce = cudaStreamEndCapture(cs, &g);
        if (!rc) rc = check_cuda(ce);
        if (!rc) {
            P->graph = g;
            rc = check_cuda(cudaGraphInstantiate(&P->exec, g, 0));
        } else if (g) {
            cudaGraphDestroy(g);
        }
    }
    // launches recorded during capture are replayed, not launched: uncount them
    P->graph_kernels = (int)(g_launches.load() - launches0);
    g_launches.fetch_sub(P->graph_kernels);
    cudaStreamDestroy(cs);
    return rc;
}

static void plan_release(wtheta_plan* P) {
    if (P->exec) cudaGraphExecDestroy(P->exec);
    if (P->graph) cudaGraphDestroy(P->graph);
    if (P->scratch) cudaFree(P->scratch);
    if (P->d_segs) cudaFree(P->d_segs);
    if (P->d_counts) cudaFree(P->d_counts);
    if (P->cull_mem) cudaFree(P->cull_mem);
    if (P->d_stats) cudaFree(P->d_stats);
    delete P;
}

static int batch_plan_impl(const wtheta_catalog_pair* cats, int n_cats, int is_xyz,
                           const double* edges, int K, const wtheta_tune* tune, cudaStream_t st,
                           wtheta_plan** out) {
    // catalogues are labelled by 16-bit index in the shared sort
    if (!out || !cats || n_cats < 1 || n_cats > 32768 || (is_xyz != 0 && is_xyz != 1))
        return WTHETA_EINVAL;
    for (int m = 0; m < n_cats; ++m) {
        const wtheta_catalog_pair& c = cats[m];
        if (c.n_data < 2 || c.n_rand < 2 || !c.data || !c.rand) return WTHETA_EINVAL;
    }
    if (tune && (tune->threads < 0 || tune->points_per_thread < 0 || tune->hist_mode < 0 ||
                 tune->hist_mode > 4 || tune->j_per_screen < 0 || tune->j_per_screen > 2 ||
                 tune->deferred < 0 || tune->deferred > 2 || tune->blocks_per_sm < 0 ||
                 tune->skip_far < 0 || tune->skip_far > 2 || tune->span_bins < 0 ||
                 tune->span_bins > 2))
        return WTHETA_EINVAL;
    wtheta_plan* P = new wtheta_plan();
    P->K = K;
    P->n_cats = n_cats;
    P->is_xyz = is_xyz;
    P->cats.assign(cats, cats + n_cats);
    int rc = build_table(edges, K, &P->tab);
    if (!rc) {
        P->cull = (!tune || tune->skip_far != 2) && edges[K] < 180.0;
        P->theta_top = edges[K] * (3.14159265358979323846 / 180.0);
        // list entries are 32-bit item indices within a count
        for (int m = 0; m < n_cats; ++m) {
            const long long t = (std::max(cats[m].n_data, cats[m].n_rand) + 255) / 256;
            if (t * t >= (1LL << 32)) P->cull = 0;
        }
    }
    DeviceInfo di;
    if (!rc) rc = device_info(&di);
    if (!rc) rc = check_cuda(cudaGetDevice(&P->dev));
    if (!rc)
        rc = dev_malloc((void**)&P->d_counts, (size_t)n_cats * 3 * (K + 2) * sizeof(unsigned long long));
    if (!rc) rc = dev_malloc((void**)&P->d_stats, 8 * WTHETA_NSTATS);
    if (rc) {
        plan_release(P);
        return rc;
    }
    int nv = 0;
    const Variant* vs = variants(&nv);
    if (tune) {
        P->v = pick_variant(tune, K, P->tab.n_lut, di.max_smem_optin);
        if (!P->v) rc = WTHETA_EINVAL;
    } else {
        // size bucket: log2 of the batch's pairs
        long long pairs = 0;
        for (int m = 0; m < n_cats; ++m)
            pairs += cats[m].n_data * cats[m].n_data / 2 + cats[m].n_data * cats[m].n_rand +
                     cats[m].n_rand * cats[m].n_rand / 2;
        int bucket = 0;
        while ((1LL << (bucket + 1)) <= pairs && bucket < 62) ++bucket;
        const TuneKey key{di.sm_count, K, bucket};
        int idx = lookup_tuned(key);
        if (idx < 0) {
            cudaEvent_t t0, t1;
            cudaEventCreate(&t0);
            cudaEventCreate(&t1);
            cudaEventRecord(t0, st);
            rc = autotune(P, di, st, &idx);
            cudaEventRecord(t1, st);
            cudaEventSynchronize(t1);
            cudaEventElapsedTime(&P->autotune_ms, t0, t1);
            cudaEventDestroy(t0);
            cudaEventDestroy(t1);
            if (!rc && idx >= 0) store_tuned(key, idx);
        }
        if (!rc && idx < 0) rc = WTHETA_EINVAL;
        if (!rc) {
            P->v = &vs[idx];
            P->autotuned = 1;
        }
    }
    if (!rc) {
        P->tune.threads = P->v->nt;
        P->tune.points_per_thread = P->v->r;
        P->tune.j_per_screen = P->v->ju;
        P->tune.hist_mode = P->v->hm;
        P->tune.deferred = P->v->def + 1;
        P->tune.skip_far = P->cull ? 1 : 2;
        P->tune.span_bins = tune && tune->span_bins == 2 ? 2 : 1;
        P->smem = P->v->smem(K, P->tab.n_lut);
        rc = plan_layout(P, P->v, di.sm_count, st);
    }
    if (!rc) rc = grid_for(P->v, P->smem, P->total_items, di.sm_count,
                           tune && tune->blocks_per_sm ? tune->blocks_per_sm : 0, &P->grid);
    if (!rc) {
        P->tune.blocks_per_sm = (P->grid + di.sm_count - 1) / di.sm_count;
        rc = check_cuda(cudaStreamSynchronize(st));
    }
    if (!rc) rc = plan_capture(P, di);
    if (rc) {
        cudaStreamSynchronize(st);
        plan_release(P);
        return rc;
    }
    *out = P;
    return WTHETA_OK;
}

}  // namespace wtheta

using namespace wtheta;

extern "C" {

int wtheta_count(const double* a, int64_t n_a, const double* b, int64_t n_b, const double* edges,
                 int32_t K, int32_t is_auto, uint64_t* counts, void* stream) {
    return count_impl(a, n_a, b, n_b, 0, edges, K, is_auto, (unsigned long long*)counts, nullptr,
                      nullptr, (cudaStream_t)stream);
}

int wtheta_count_xyz(const double* a, int64_t n_a, const double* b, int64_t n_b,
                     const double* edges, int32_t K, int32_t is_auto, uint64_t* counts,
                     void* stream) {
    return count_impl(a, n_a, b, n_b, 1, edges, K, is_auto, (unsigned long long*)counts, nullptr,
                      nullptr, (cudaStream_t)stream);
}

int wtheta_count_ex(const double* a, int64_t n_a, const double* b, int64_t n_b, int32_t is_xyz,
                    const double* edges, int32_t K, int32_t is_auto, uint64_t* counts,
                    const wtheta_tune* tune, uint64_t* stats, void* stream) {
    return count_impl(a, n_a, b, n_b, is_xyz, edges, K, is_auto, (unsigned long long*)counts, tune,
                      (unsigned long long*)stats, (cudaStream_t)stream);
}

int wtheta_radec_to_xyz(const double* rd, int64_t n, double* xyz, void* stream) {
    if (n < 0 || (n > 0 && (!rd || !xyz))) return WTHETA_EINVAL;
    if (n == 0) return WTHETA_OK;
    const int threads = 256;
    const int grid = (int)std::min<long long>((n + threads - 1) / threads, 1 << 20);
    k_radec_to_xyz<<<grid, threads, 0, (cudaStream_t)stream>>>(rd, n, xyz, n);
    count_launch();
    return check_cuda(cudaGetLastError());
}

int wtheta_count_xyz_noalloc(const double* a, int64_t n_a, const double* b, int64_t n_b,
                             const double* edges, int32_t K, int32_t is_auto, uint64_t* counts,
                             void* stream) {
    return count_xyz_noalloc_impl(a, n_a, b, n_b, edges, K, is_auto, (unsigned long long*)counts,
                                  (cudaStream_t)stream);
}

int wtheta_batch_plan(const wtheta_catalog_pair* cats, int32_t n_cats, const double* edges,
                      int32_t K, const wtheta_tune* tune, void* stream, wtheta_plan** plan) {
    return batch_plan_impl(cats, n_cats, 0, edges, K, tune, (cudaStream_t)stream, plan);
}

int wtheta_batch_plan_ex(const wtheta_catalog_pair* cats, int32_t n_cats, int32_t coords_are_xyz,
                         const double* edges, int32_t K, const wtheta_tune* tune, void* stream,
                         wtheta_plan** plan) {
    return batch_plan_impl(cats, n_cats, coords_are_xyz, edges, K, tune, (cudaStream_t)stream,
                           plan);
}

int wtheta_batch_run(wtheta_plan* P, uint64_t* counts, void* stream) {
    if (!P || !counts) return WTHETA_EINVAL;
    TraceRange trace("wtheta_batch_run");
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) return WTHETA_ECUDA;
    if (dev != P->dev) return WTHETA_EINVAL;
    cudaStream_t st = (cudaStream_t)stream;
    int rc = check_cuda(cudaGraphLaunch(P->exec, st));
    if (rc) return rc;
    count_launch((unsigned)P->graph_kernels);
    ++P->runs;
    const size_t bytes = (size_t)P->n_cats * 3 * (P->K + 2) * sizeof(unsigned long long);
    return check_cuda(cudaMemcpyAsync(counts, P->d_counts, bytes, cudaMemcpyDeviceToDevice, st));
}

int wtheta_batch_info(const wtheta_plan* P, wtheta_batch_info_t* info) {
    if (!P || !info) return WTHETA_EINVAL;
    std::memset(info, 0, sizeof(*info));
    info->tune = P->tune;
    info->n_items = P->total_items;
    info->pairs = P->pairs;
    const long long T = (long long)P->v->nt * P->v->r;
    info->evaluated_pairs = P->total_items * T * T;
    if (P->runs > 0) {
        // pairs whose squared chord the last run computed (it must have finished)
        unsigned long long st[WTHETA_NSTATS];
        if (cudaDeviceSynchronize() != cudaSuccess ||
            cudaMemcpy(st, P->d_stats, sizeof(st), cudaMemcpyDeviceToHost) != cudaSuccess)
            return WTHETA_ECUDA;
        info->evaluated_pairs = (long long)st[WTHETA_STAT_PAIRS];
    }
    info->n_counts = 3 * P->n_cats;
    info->graph_kernels = P->graph_kernels;
    info->autotune_ms = P->autotune_ms;
    info->autotuned = P->autotuned;
    return WTHETA_OK;
}

int wtheta_batch_free(wtheta_plan* P) {
    if (!P) return WTHETA_EINVAL;
    cudaDeviceSynchronize();
    plan_release(P);
    return WTHETA_OK;
}

int wtheta_count_shard(const double* a, int64_t n_a, const double* b, int64_t n_b,
                       const double* edges, int32_t K, int32_t is_auto, int32_t shard,
                       int32_t n_shards, uint64_t* counts, void* stream) {
    int64_t r0 = 0, r1 = 0;
    if (is_auto) {
        if (b && b != a) return WTHETA_EINVAL;
        if (n_b != n_a && !(b == nullptr && n_b == 0)) return WTHETA_EINVAL;
    }
    int rc = wtheta_shard_rows(n_a, is_auto ? n_a : n_b, is_auto, shard, n_shards, &r0, &r1);
    if (rc) return rc;
    if (!counts || (n_a > 0 && !a) || (!is_auto && n_b > 0 && !b)) return WTHETA_EINVAL;
    cudaStream_t st = (cudaStream_t)stream;
    const double* rows = a ? a + 2 * r0 : nullptr;
    if (!is_auto)
        return count_impl(rows, r1 - r0, b, n_b, 0, edges, K, 0, (unsigned long long*)counts,
                          nullptr, nullptr, st);
    // rows [r0, r1) of an auto count: the pairs inside the rows, plus the rows
    // against every later point
    rc = count_impl(rows, r1 - r0, nullptr, 0, 0, edges, K, 1, (unsigned long long*)counts,
                    nullptr, nullptr, st);
    if (rc || r1 >= n_a || r1 == r0) return rc;
    unsigned long long* tmp = nullptr;
    if ((rc = dev_malloc_async((void**)&tmp, sizeof(unsigned long long) * (K + 2), st)))
        return rc;
    rc = count_impl(rows, r1 - r0, a + 2 * r1, n_a - r1, 0, edges, K, 0, tmp, nullptr, nullptr,
                    st);
    if (!rc) {
        k_add_counts<<<1, 64, 0, st>>>((unsigned long long*)counts, tmp, K + 2);
        count_launch();
        rc = check_cuda(cudaGetLastError());
    }
    const cudaError_t fe = cudaFreeAsync(tmp, st);
    return rc ? rc : check_cuda(fe);
}

uint64_t wtheta_kernel_launches(void) { return g_launches.load(std::memory_order_relaxed); }

int wtheta_get_error(void* stream, uint32_t* code) {
    if (!code) return WTHETA_EINVAL;
    cudaStream_t st = (cudaStream_t)stream;
    int rc = check_cuda(cudaStreamSynchronize(st));
    if (rc) return rc;
    unsigned int v = 0, zero = 0;
    if ((rc = check_cuda(cudaMemcpyFromSymbol(&v, g_device_error, sizeof(v))))) return rc;
    if ((rc = check_cuda(cudaMemcpyToSymbol(g_device_error, &zero, sizeof(zero))))) return rc;
    *code = v;
    return WTHETA_OK;
}

int wtheta_inject_alloc_failure(int32_t after) {
    if (after < -1) return WTHETA_EINVAL;
    g_fail_alloc.store(after);
    return WTHETA_OK;
}

int wtheta_count_wtheta(const double* coords_d, int64_t n_d, const double* coords_r,
                        int64_t n_r, int32_t coords_are_xyz, const double* bin_edges_deg,
                        int32_t n_bins, uint64_t* counts, const wtheta_tune* tune,
                        uint64_t* stats, void* stream) {
    return count_wtheta_impl(coords_d, n_d, coords_r, n_r, coords_are_xyz, bin_edges_deg, n_bins,
                             (unsigned long long*)counts, tune, (unsigned long long*)stats,
                             (cudaStream_t)stream);
}

int wtheta_count_wtheta_shard(const double* coords_d, int64_t n_d, const double* coords_r,
                              int64_t n_r, int32_t coords_are_xyz, const double* bin_edges_deg,
                              int32_t n_bins, int32_t shard, int32_t n_shards, uint64_t* counts,
                              const wtheta_tune* tune, uint64_t* stats, void* stream) {
    return count_wtheta_impl(coords_d, n_d, coords_r, n_r, coords_are_xyz, bin_edges_deg, n_bins,
                             (unsigned long long*)counts, tune, (unsigned long long*)stats,
                             (cudaStream_t)stream, shard, n_shards);
}

int wtheta_correlate(const double* data, int64_t n_d, const double* rand, int64_t n_r,
                     const double* edges, int32_t K, uint64_t* counts_out, double* w_out,
                     void* stream) {
    if (n_d < 0 || n_r < 0 || (n_d > 0 && !data) || (n_r > 0 && !rand)) return WTHETA_EINVAL;
    int rc = validate_edges(edges, K);
    if (rc) return rc;
    if (w_out && (n_d < 2 || n_r < 2)) return WTHETA_EINVAL;
    cudaStream_t st = (cudaStream_t)stream;
    const size_t nslot = (size_t)K + 2;
    void* buf = nullptr;
    const size_t bytes = 256 + (size_t)(n_d + n_r) * 16 + 3 * nslot * 8;
    if ((rc = dev_malloc_async(&buf, bytes, st))) return rc;
    unsigned long long* dc = (unsigned long long*)buf;  // 3 (K+2) counts
    double* dd = (double*)((unsigned char*)buf + ((3 * nslot * 8 + 255) / 256) * 256);
    double* dr = dd + 2 * n_d;
    rc = check_cuda(cudaMemcpyAsync(dd, data, (size_t)n_d * 16, cudaMemcpyHostToDevice, st));
    if (!rc) rc = check_cuda(cudaMemcpyAsync(dr, rand, (size_t)n_r * 16, cudaMemcpyHostToDevice, st));
    if (!rc) rc = count_wtheta_impl(dd, n_d, dr, n_r, 0, edges, K, dc, nullptr, nullptr, st);
    uint64_t host_counts[3 * (kMaxBins + 2)];
    if (!rc)
        rc = check_cuda(cudaMemcpyAsync(host_counts, dc, 3 * nslot * 8, cudaMemcpyDeviceToHost, st));
    cudaError_t fe = cudaFreeAsync(buf, st);
    cudaError_t se = cudaStreamSynchronize(st);
    if (!rc) rc = check_cuda(fe);
    if (!rc) rc = check_cuda(se);
    if (rc) return rc;
    if (counts_out) std::memcpy(counts_out, host_counts, 3 * nslot * 8);
    if (w_out)
        rc = wtheta_ls(host_counts, host_counts + nslot, host_counts + 2 * nslot, n_d, n_r, K, w_out);
    return rc;
}

}  // extern "C"
