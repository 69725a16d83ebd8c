// Pair-count kernels of libwtheta and the entry points that launch them.
//
// The computation is Sec. 2 of arXiv:1208.3658: every pair's angular
// separation (App. A) is binned (Sec. 2.1); auto counts take each unordered
// pair i < j once, cross counts every (i, j).  The paper splits the pair
// matrix into sub-matrices, one kernel launch each, with per-block shared
// histograms summed on the host.  Here one persistent launch walks the whole
// (triangular or rectangular) space of tile pairs from a device work cursor:
//   - RA/Dec -> FP64 unit vectors once per point (SoA, for the rare FP64
//     recheck) and FP32 float4 copies (x, y, z, 0) padded to whole tiles with
//     far-away sentinel points that never land in a bin;
//   - a CTA loads the B tile into shared memory and keeps R A points per
//     thread in registers; each pair costs 3 FADD + 1 FMUL + 2 FFMA for the
//     FP32 squared chord s;
//   - s is screened against the top edge: pairs beyond it are overflow and
//     cost nothing more (Sec. 2.2: separations outside the bin range can be
//     skipped); the overflow slot is filled at the end as total minus the rest;
//   - in-range pairs are binned by a table lookup on the bits of s, the FP32
//     comparison being final outside a rigorous guard band around each edge;
//     inside it the pair is recomputed in FP64 exactly as the definition says;
//   - counts go to private per-thread (or per-warp, warp-aggregated) uint32
//     shared histograms, flushed into uint64 global counts before any can wrap.
#include <cuda_runtime.h>

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

__device__ __forceinline__ float min3f(float a, float b, float c) {
    float d;
    asm("min.f32 %0, %1, %2, %3;" : "=f"(d) : "f"(a), "f"(b), "f"(c));
    return d;
}

// ---------------------------------------------------------------------------
// conversion kernels
// ---------------------------------------------------------------------------
// RA/Dec degrees -> FP64 unit vectors (SoA with stride xyz_stride) and, when
// p32 is not null, FP32 float4 copies for n <= i < n_pad set to sentinels
// (sign * kSentinel * (i - n + 1), 0, 0).
__global__ void k_radec_to_xyz(const double* __restrict__ rd, long long n, long long n_pad,
                               double* __restrict__ xyz, long long xyz_stride,
                               float4* __restrict__ p32, float sign) {
    const double d2r = 3.14159265358979323846 / 180.0;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n_pad;
         i += (long long)gridDim.x * blockDim.x) {
        if (i < n) {
            const double ra = rd[2 * i], dec = rd[2 * i + 1];
            if (!isfinite(ra) || !isfinite(dec)) atomicOr(&g_device_error, WTHETA_DERR_NONFINITE);
            else if (fabs(dec) > 90.0) atomicOr(&g_device_error, WTHETA_DERR_DEC_RANGE);
            const double a = ra * d2r, d = dec * d2r;
            const double cd = cos(d), sd = sin(d), ca = cos(a), sa = sin(a);
            const double x = __dmul_rn(cd, ca), y = __dmul_rn(cd, sa), z = sd;
            if (xyz) {
                xyz[i] = x;
                xyz[xyz_stride + i] = y;
                xyz[2 * xyz_stride + i] = z;
            }
            if (p32)
                p32[i] = make_float4(__double2float_rn(x), __double2float_rn(y),
                                     __double2float_rn(z), 0.f);
        } else if (p32) {
            p32[i] = make_float4(sign * kSentinel * (float)(i - n + 1), 0.f, 0.f, 0.f);
        }
    }
}

// Caller's FP64 SoA unit vectors -> FP32 float4 copies (+ sentinels).
__global__ void k_xyz_to_f32(const double* __restrict__ xyz, long long n, long long n_pad,
                             float4* __restrict__ p32, float sign) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n_pad;
         i += (long long)gridDim.x * blockDim.x) {
        if (i < n) {
            const double x = xyz[i], y = xyz[n + i], z = xyz[2 * n + i];
            if (!isfinite(x) || !isfinite(y) || !isfinite(z)) {
                atomicOr(&g_device_error, WTHETA_DERR_NONFINITE);
            } else {
                const double r2 = x * x + y * y + z * z;
                if (fabs(r2 - 1.0) > 1e-6) atomicOr(&g_device_error, WTHETA_DERR_NOT_UNIT);
            }
            p32[i] = make_float4(__double2float_rn(x), __double2float_rn(y),
                                 __double2float_rn(z), 0.f);
        } else {
            p32[i] = make_float4(sign * kSentinel * (float)(i - n + 1), 0.f, 0.f, 0.f);
        }
    }
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
struct PairParams {
    const float4* a32;
    const float4* b32;
    const double* a64;       // FP64 SoA of catalogue a, stride a64_stride
    const double* b64;
    long long a64_stride, b64_stride;
    long long tiles_a, tiles_b;
    long long n_items;       // tile pairs
    int is_auto;
    int items_per_flush;     // flush the uint32 histograms after this many items
    unsigned long long* cursor;
    unsigned long long* counts;   // K+2 slots (slot K+1 filled by k_finalize)
    unsigned long long* stats;    // WTHETA_NSTATS or null
    BinTable tab;
};

enum HistMode { kHistLane = 1, kHistWarp = 2 };

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

// FP64 recheck: the definition's squared chord and slot for pair (i, j).
__device__ __noinline__ unsigned recheck_slot(const double* __restrict__ a64, long long as,
                                              long long i, const double* __restrict__ b64,
                                              long long bs, long long j,
                                              const double* __restrict__ c64, int K) {
    const double dx = __dsub_rn(a64[i], b64[j]);
    const double dy = __dsub_rn(a64[as + i], b64[bs + j]);
    const double dz = __dsub_rn(a64[2 * as + i], b64[2 * bs + j]);
    const double s = __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz));
    unsigned k = 0;
    while (k <= (unsigned)K && c64[k] <= s) ++k;
    return k;  // K+1 = overflow
}

template <int NT, int R, int HM>
struct PairKernel {
    static constexpr int TA = NT * R;   // A points per tile
    static constexpr int TB = NT * R;   // B points per tile (equal: auto needs square tiles)
    static constexpr int NW = NT / 32;
    static constexpr int HCOLS = HM == kHistLane ? NT : NW;

    static size_t smem_bytes(int K, int n_lut) {
        size_t b = (size_t)TB * 16;             // B tile
        b += (size_t)n_lut * 16;                // screening table
        b += (size_t)(K + 2) * 8;               // FP64 edges (+ pad)
        b += (size_t)(K + 1) * HCOLS * 4;       // histograms
        return b;
    }
};

template <int NT, int R, int HM>
__device__ __forceinline__ void flush_hist(unsigned* hist, int K,
                                           unsigned long long* __restrict__ counts) {
    constexpr int HCOLS = PairKernel<NT, R, HM>::HCOLS;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int b = warp; b <= K; b += NT / 32) {
        unsigned long long sum = 0;
        for (int q = lane; q < HCOLS; q += 32) {
            sum += hist[b * HCOLS + q];
            hist[b * HCOLS + q] = 0;
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o);
        if (lane == 0 && sum) atomicAdd(counts + b, sum);
    }
}

// One tile pair: B tile in shared memory, R A points per thread in registers.
template <int NT, int R, int HM, bool DIAG>
__device__ __forceinline__ void tile_pass(const float4* __restrict__ sB, const uint4* __restrict__ sLut,
                                          const double* __restrict__ sC, unsigned* __restrict__ hist,
                                          const float (&ax)[R], const float (&ay)[R],
                                          const float (&az)[R], const PairParams& p,
                                          long long I, long long J, unsigned long long& n_binned,
                                          unsigned long long& n_recheck) {
    constexpr int TA = PairKernel<NT, R, HM>::TA;
    constexpr int TB = PairKernel<NT, R, HM>::TB;
    constexpr int HCOLS = PairKernel<NT, R, HM>::HCOLS;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const float hf = __uint_as_float(p.tab.h_top);
    const int shift = p.tab.shift, base = p.tab.base, K = p.tab.K;
    unsigned* myhist = HM == kHistLane ? hist + tid : hist + warp;

#pragma unroll 2
    for (int j = 0; j < TB; ++j) {
        const float4 b = sB[j];
        float s[R];
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const float dx = ax[r] - b.x, dy = ay[r] - b.y, dz = az[r] - b.z;
            s[r] = __fmaf_rn(dz, dz, __fmaf_rn(dy, dy, __fmul_rn(dx, dx)));
            if (DIAG) {
                if (j <= r * NT + tid) s[r] = __int_as_float(0x7f800000);  // i >= j: not a pair
            }
        }
        float m = s[0];
#pragma unroll
        for (int r = 1; r + 1 < R; r += 2) m = min3f(m, s[r], s[r + 1]);
        if (R % 2 == 0) m = fminf(m, s[R - 1]);

        const bool any_in = m <= hf;
        if (HM == kHistLane) {
            if (!any_in) continue;
#pragma unroll
            for (int r = 0; r < R; ++r) {
                if (s[r] <= hf) {
                    const unsigned bits = __float_as_uint(s[r]);
                    const int idx = max((int)(bits >> shift) - base, 0);
                    const uint4 e = sLut[idx];
                    unsigned slot;
                    if (bits < e.x) slot = e.z;
                    else if (bits > e.y) slot = e.w;
                    else {
                        slot = recheck_slot(p.a64, p.a64_stride, I * TA + r * NT + tid, p.b64,
                                            p.b64_stride, J * TB + j, sC, K);
                        ++n_recheck;
                    }
                    if (slot <= (unsigned)K) myhist[slot * HCOLS] += 1u;
                    ++n_binned;
                }
            }
        } else {
            if (!__any_sync(0xffffffffu, any_in)) continue;
#pragma unroll
            for (int r = 0; r < R; ++r) {
                const bool in = s[r] <= hf;
                unsigned slot = 0xffffffffu;
                if (in) {
                    const unsigned bits = __float_as_uint(s[r]);
                    const int idx = max((int)(bits >> shift) - base, 0);
                    const uint4 e = sLut[idx];
                    if (bits < e.x) slot = e.z;
                    else if (bits > e.y) slot = e.w;
                    else {
                        slot = recheck_slot(p.a64, p.a64_stride, I * TA + r * NT + tid, p.b64,
                                            p.b64_stride, J * TB + j, sC, K);
                        ++n_recheck;
                    }
                    ++n_binned;
                }
                const bool take = in && slot <= (unsigned)K;
                const unsigned act = __ballot_sync(0xffffffffu, take);
                if (take) {
                    const unsigned peers = __match_any_sync(act, slot);
                    if (lane == __ffs(peers) - 1)
                        atomicAdd(myhist + slot * HCOLS, (unsigned)__popc(peers));
                }
            }
        }
    }
    (void)lane;
}

template <int NT, int R, int HM>
__global__ void __launch_bounds__(NT) k_pairs(const __grid_constant__ PairParams p) {
    using PK = PairKernel<NT, R, HM>;
    constexpr int TA = PK::TA, TB = PK::TB, HCOLS = PK::HCOLS;
    extern __shared__ __align__(16) unsigned char smem[];
    const int K = p.tab.K;
    float4* sB = reinterpret_cast<float4*>(smem);
    uint4* sLut = reinterpret_cast<uint4*>(sB + TB);
    double* sC = reinterpret_cast<double*>(sLut + p.tab.n_lut);
    unsigned* hist = reinterpret_cast<unsigned*>(sC + (K + 2));
    __shared__ long long s_item;

    const int tid = threadIdx.x;
    for (int q = tid; q < p.tab.n_lut; q += NT)
        sLut[q] = make_uint4(p.tab.lut[q][0], p.tab.lut[q][1], p.tab.lut[q][2], p.tab.lut[q][3]);
    for (int q = tid; q <= K; q += NT) sC[q] = p.tab.c64[q];
    for (int q = tid; q < (K + 1) * HCOLS; q += NT) hist[q] = 0u;

    unsigned long long n_binned = 0, n_recheck = 0, n_items = 0;
    int since_flush = 0;
    for (;;) {
        if (tid == 0) s_item = (long long)atomicAdd(p.cursor, 1ull);
        __syncthreads();  // s_item visible; previous item's sB reads finished
        const long long t = s_item;
        if (t >= p.n_items) break;
        long long I, J;
        item_to_tiles(t, p.tiles_a, p.tiles_b, p.is_auto, &I, &J);
        const float4* gB = p.b32 + J * TB;
#pragma unroll
        for (int q = 0; q < R; ++q) sB[q * NT + tid] = gB[q * NT + tid];
        float ax[R], ay[R], az[R];
        const float4* gA = p.a32 + I * TA;
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const float4 a = gA[r * NT + tid];
            ax[r] = a.x; ay[r] = a.y; az[r] = a.z;
        }
        __syncthreads();  // B tile staged
        if (p.is_auto && I == J)
            tile_pass<NT, R, HM, true>(sB, sLut, sC, hist, ax, ay, az, p, I, J, n_binned, n_recheck);
        else
            tile_pass<NT, R, HM, false>(sB, sLut, sC, hist, ax, ay, az, p, I, J, n_binned, n_recheck);
        ++n_items;
        if (++since_flush == p.items_per_flush) {
            __syncthreads();
            flush_hist<NT, R, HM>(hist, K, p.counts);
            __syncthreads();
            since_flush = 0;
        }
    }
    // all threads left the loop after the same barrier
    flush_hist<NT, R, HM>(hist, K, p.counts);
    if (p.stats) {
        unsigned long long v1 = n_binned, v2 = n_recheck;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            v1 += __shfl_xor_sync(0xffffffffu, v1, o);
            v2 += __shfl_xor_sync(0xffffffffu, v2, o);
        }
        if ((tid & 31) == 0) {
            if (v1) atomicAdd(p.stats + WTHETA_STAT_BINNED, v1);
            if (v2) atomicAdd(p.stats + WTHETA_STAT_RECHECK, v2);
        }
        if (tid == 0 && n_items) {
            atomicAdd(p.stats + WTHETA_STAT_TILES, n_items);
            atomicAdd(p.stats + WTHETA_STAT_PAIRS, n_items * (unsigned long long)TA * TB);
        }
    }
}

// ---------------------------------------------------------------------------
// launch plumbing
// ---------------------------------------------------------------------------
struct Variant {
    int nt, r, hm;
    void (*kernel)(PairParams);
    size_t (*smem)(int, int);
};

template <int NT, int R, int HM>
static Variant make_variant() {
    return Variant{NT, R, HM, &k_pairs<NT, R, HM>, &PairKernel<NT, R, HM>::smem_bytes};
}

static const Variant* variants(int* n) {
    static const Variant v[] = {
        make_variant<128, 8, kHistLane>(), make_variant<256, 4, kHistLane>(),
        make_variant<128, 4, kHistLane>(), make_variant<256, 8, kHistLane>(),
        make_variant<128, 8, kHistWarp>(), make_variant<256, 4, kHistWarp>(),
        make_variant<128, 4, kHistWarp>(), make_variant<256, 8, kHistWarp>(),
    };
    *n = (int)(sizeof(v) / sizeof(v[0]));
    return v;
}

struct DeviceInfo {
    int sm_count = 0;
    int max_smem_optin = 0;
};

static int device_info(DeviceInfo* out) {
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

static const Variant* pick_variant(const wtheta_tune* tune, int K, int n_lut, int max_smem) {
    int nv = 0;
    const Variant* v = variants(&nv);
    const int want_nt = tune && tune->threads ? tune->threads : 128;
    const int want_r = tune && tune->points_per_thread ? tune->points_per_thread : 8;
    int want_hm = tune && tune->hist_mode ? tune->hist_mode : 0;
    if (want_hm == 0) {
        // private per-thread histograms while they fit comfortably
        want_hm = v[0].smem(K, n_lut) <= 100 * 1024 ? kHistLane : kHistWarp;
    }
    for (int i = 0; i < nv; ++i)
        if (v[i].nt == want_nt && v[i].r == want_r && v[i].hm == want_hm &&
            v[i].smem(K, n_lut) <= (size_t)max_smem)
            return &v[i];
    // fall back: anything that fits, per-warp first
    for (int i = 0; i < nv; ++i)
        if (v[i].hm == kHistWarp && v[i].smem(K, n_lut) <= (size_t)max_smem) return &v[i];
    return nullptr;
}

static int grid_for(const Variant* v, size_t smem, long long n_items, int sm_count, int* grid) {
    static std::mutex mu;
    {
        std::lock_guard<std::mutex> g(mu);
        if (cudaFuncSetAttribute((const void*)v->kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)smem) != cudaSuccess)
            return WTHETA_ECUDA;
    }
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, (const void*)v->kernel, v->nt,
                                                      smem) != cudaSuccess)
        return WTHETA_ECUDA;
    per_sm = std::max(per_sm, 1);
    long long g = (long long)per_sm * sm_count;
    if (g > n_items) g = n_items;
    *grid = (int)std::max(g, 1LL);
    return WTHETA_OK;
}

static inline long long round_up(long long x, long long m) { return (x + m - 1) / m * m; }

static int check_cuda(cudaError_t e) {
    if (e == cudaSuccess) return WTHETA_OK;
    if (e == cudaErrorMemoryAllocation) return WTHETA_ENOMEM;
    return WTHETA_ECUDA;
}

// Core of wtheta_count / wtheta_count_xyz / wtheta_count_ex.
static int count_impl(const double* ca, long long n_a, const double* cb, long long n_b,
                      int is_xyz, const double* edges, int K, int is_auto,
                      unsigned long long* counts, const wtheta_tune* tune,
                      unsigned long long* stats, cudaStream_t st) {
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
    if (tune && ((tune->threads && tune->threads != 128 && tune->threads != 256) ||
                 (tune->points_per_thread && tune->points_per_thread != 4 &&
                  tune->points_per_thread != 8) ||
                 (tune->hist_mode < 0 || tune->hist_mode > 2)))
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

    const Variant* v = pick_variant(tune, K, tab.n_lut, di.max_smem_optin);
    if (!v) return WTHETA_EINVAL;
    const long long T = (long long)v->nt * v->r;  // TA == TB
    const long long pa = round_up(n_a, T), pb = is_auto ? pa : round_up(n_b, T);

    // scratch: FP32 copies of both catalogues, FP64 SoA when converting from
    // RA/Dec, and the work cursor
    size_t bytes = (size_t)pa * 16 + (is_auto ? 0 : (size_t)pb * 16) + 256;
    if (!is_xyz) bytes += (size_t)pa * 24 + (is_auto ? 0 : (size_t)pb * 24);
    void* scratch = nullptr;
    if ((rc = check_cuda(cudaMallocAsync(&scratch, bytes, st)))) return rc;
    unsigned char* sp = (unsigned char*)scratch;
    unsigned long long* cursor = (unsigned long long*)sp;
    sp += 256;
    float4* a32 = (float4*)sp;
    sp += (size_t)pa * 16;
    float4* b32 = a32;
    if (!is_auto) { b32 = (float4*)sp; sp += (size_t)pb * 16; }
    const double* a64 = ca;
    const double* b64 = cb;
    long long as = n_a, bs = n_b;
    const int cvt_threads = 256;
    auto cvt_grid = [&](long long n) {
        long long g = (n + cvt_threads - 1) / cvt_threads;
        return (int)std::min<long long>(std::max<long long>(g, 1), (long long)di.sm_count * 16);
    };
    if (!is_xyz) {
        double* x64a = (double*)sp;
        sp += (size_t)pa * 24;
        k_radec_to_xyz<<<cvt_grid(pa), cvt_threads, 0, st>>>(ca, n_a, pa, x64a, pa, a32, 1.f);
        count_launch();
        a64 = x64a; as = pa;
        if (!is_auto) {
            double* x64b = (double*)sp;
            sp += (size_t)pb * 24;
            k_radec_to_xyz<<<cvt_grid(pb), cvt_threads, 0, st>>>(cb, n_b, pb, x64b, pb, b32, -1.f);
            count_launch();
            b64 = x64b; bs = pb;
        } else {
            b64 = a64; bs = as;
        }
    } else {
        k_xyz_to_f32<<<cvt_grid(pa), cvt_threads, 0, st>>>(ca, n_a, pa, a32, 1.f);
        count_launch();
        if (!is_auto) {
            k_xyz_to_f32<<<cvt_grid(pb), cvt_threads, 0, st>>>(cb, n_b, pb, b32, -1.f);
            count_launch();
        }
    }
    rc = check_cuda(cudaMemsetAsync(cursor, 0, sizeof(unsigned long long), st));

    const long long ta = pa / T, tb = pb / T;
    const long long n_items = is_auto ? ta * (ta + 1) / 2 : ta * tb;
    const size_t smem = v->smem(K, tab.n_lut);
    int grid = 0;
    if (!rc) rc = grid_for(v, smem, n_items, di.sm_count, &grid);
    if (!rc) {
        PairParams prm;
        std::memset(&prm, 0, sizeof(prm));
        prm.a32 = a32; prm.b32 = b32; prm.a64 = a64; prm.b64 = b64;
        prm.a64_stride = as; prm.b64_stride = bs;
        prm.tiles_a = ta; prm.tiles_b = tb; prm.n_items = n_items;
        prm.is_auto = is_auto;
        // a histogram cell gains at most T (per-thread) or 32 T (per-warp) per item
        const unsigned long long per_item = (v->hm == kHistLane ? 1ull : 32ull) * (unsigned long long)T;
        prm.items_per_flush = (int)std::min<unsigned long long>(0xFFFFFFFFull / per_item, 1ull << 30);
        prm.cursor = cursor; prm.counts = counts; prm.stats = stats;
        std::memcpy(&prm.tab, &tab, sizeof(tab));
        v->kernel<<<grid, v->nt, smem, st>>>(prm);
        count_launch();
        rc = check_cuda(cudaGetLastError());
        if (!rc) {
            k_finalize<<<1, 1, 0, st>>>(counts, K, total);
            count_launch();
            rc = check_cuda(cudaGetLastError());
        }
    }
    cudaError_t fe = cudaFreeAsync(scratch, st);
    if (!rc) rc = check_cuda(fe);
    return rc;
}

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
    wtheta_tune fixed = {128, 8, 0, 0};  // the tile of WTHETA_NOALLOC_TILE points
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
    k_xyz_to_f32<<<cvt_grid(pa), cvt_threads, 0, st>>>(ca, n_a, pa, a32, 1.f);
    count_launch();
    if (!is_auto) {
        k_xyz_to_f32<<<cvt_grid(pb), cvt_threads, 0, st>>>(cb, n_b, pb, b32, -1.f);
        count_launch();
    }
    if ((rc = check_cuda(cudaMemsetAsync(cursor, 0, sizeof(unsigned long long), st)))) return rc;
    const long long ta = pa / T, tb = is_auto ? ta : pb / T;
    const long long n_items = is_auto ? ta * (ta + 1) / 2 : ta * tb;
    const size_t smem = v->smem(K, tab.n_lut);
    int grid = 0;
    if ((rc = grid_for(v, smem, n_items, di.sm_count, &grid))) return rc;
    PairParams prm;
    std::memset(&prm, 0, sizeof(prm));
    prm.a32 = a32; prm.b32 = b32; prm.a64 = ca; prm.b64 = cb;
    prm.a64_stride = n_a; prm.b64_stride = n_b;
    prm.tiles_a = ta; prm.tiles_b = tb; prm.n_items = n_items;
    prm.is_auto = is_auto;
    const unsigned long long per_item = (v->hm == kHistLane ? 1ull : 32ull) * (unsigned long long)T;
    prm.items_per_flush = (int)std::min<unsigned long long>(0xFFFFFFFFull / per_item, 1ull << 30);
    prm.cursor = cursor; prm.counts = counts; prm.stats = nullptr;
    std::memcpy(&prm.tab, &tab, sizeof(tab));
    v->kernel<<<grid, v->nt, smem, st>>>(prm);
    count_launch();
    if ((rc = check_cuda(cudaGetLastError()))) return rc;
    k_finalize<<<1, 1, 0, st>>>(counts, K, total);
    count_launch();
    return check_cuda(cudaGetLastError());
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
    k_radec_to_xyz<<<grid, threads, 0, (cudaStream_t)stream>>>(rd, n, n, xyz, n, nullptr, 1.f);
    count_launch();
    return check_cuda(cudaGetLastError());
}

int wtheta_count_xyz_noalloc(const double* a, int64_t n_a, const double* b, int64_t n_b,
                             const double* edges, int32_t K, int32_t is_auto, uint64_t* counts,
                             void* stream) {
    return count_xyz_noalloc_impl(a, n_a, b, n_b, edges, K, is_auto, (unsigned long long*)counts,
                                  (cudaStream_t)stream);
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
    if ((rc = check_cuda(cudaMallocAsync(&buf, bytes, st)))) return rc;
    unsigned long long* dc = (unsigned long long*)buf;  // 3 (K+2) counts
    double* dd = (double*)((unsigned char*)buf + ((3 * nslot * 8 + 255) / 256) * 256);
    double* dr = dd + 2 * n_d;
    rc = check_cuda(cudaMemcpyAsync(dd, data, (size_t)n_d * 16, cudaMemcpyHostToDevice, st));
    if (!rc) rc = check_cuda(cudaMemcpyAsync(dr, rand, (size_t)n_r * 16, cudaMemcpyHostToDevice, st));
    if (!rc) rc = count_impl(dd, n_d, nullptr, 0, 0, edges, K, 1, dc, nullptr, nullptr, st);
    if (!rc) rc = count_impl(dd, n_d, dr, n_r, 0, edges, K, 0, dc + nslot, nullptr, nullptr, st);
    if (!rc) rc = count_impl(dr, n_r, nullptr, 0, 0, edges, K, 1, dc + 2 * nslot, nullptr, nullptr, st);
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
