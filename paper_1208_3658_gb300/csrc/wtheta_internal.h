// Internal declarations shared by the library's host and device sources.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>
#include <vector>

#include "wtheta.h"

namespace wtheta {

constexpr int kMaxBins = 256;      // K upper limit (slots 0..K+1)
constexpr int kMaxLut = 512;       // entries of the FP32 screening table

// Screening table for one edge set, built on the host, read by every counting
// kernel.  Non-negative FP32 values order like their bit patterns, so the
// kernel works on the bits of the FP32 squared chord s:
//   - bits > h_top: at or above the top edge for certain -> overflow slot,
//     which is never stored (it is the pair total minus the other slots);
//   - else idx = max((bits >> shift) - base, 0), e = lut[idx] and
//       bits < e.x -> slot e.z,  bits > e.y -> slot e.w,
//       otherwise the pair is inside an edge's guard band (or the bucket holds
//       more than one band) and is recomputed in FP64 against c64;
//   - slot K+1 (overflow) in the table, and any value beyond h_top, goes to a
//     trash row that is never added to the counts;
//   - a bucket holding several bands has {0, h_top, K+1, K+1}: all its
//     in-range values are rechecked, values beyond h_top are overflow;
//   - every band's upper bound is at most h_top, so a value beyond h_top is
//     never taken for a band value.
struct BinTable {
    int32_t K;
    uint32_t h_top;        // FP32 bits of the top edge's upper guard bound
    int32_t shift;         // bucket = bits >> shift
    int32_t base;          // bucket of the lowest guard bound
    int32_t n_lut;         // entries used
    int32_t n_complex;     // buckets holding more than one guard band
    double c64[kMaxBins + 1];            // FP64 squared-chord edges
    uint32_t band[kMaxBins + 1][2];      // {lo_bits, hi_bits}: guard band of edge k (c_k > 0)
    uint32_t lut[kMaxLut][4];            // {lo_bits, hi_bits, slot_below, slot_above}
};


// Private histogram columns of the pair kernel: per thread, plain
// read-modify-write (1); per warp, lanes merged by __match_any_sync (2); per
// thread, shared reduction (3); per warp, shared reduction (4: the shared
// atomic unit merges lanes that hit one word at full rate, and the rows of a
// warp's column sit an odd number of words apart so that different rows hit
// different banks).
enum HistMode { kHistLane = 1, kHistWarp = 2, kHistLaneAtomic = 3, kHistWarpRed = 4 };

// One count: catalogue a against catalogue b (auto: a = b, pairs i < j).
struct Segment {
    const float4* a32;       // FP32 points (x, y, z, original index bits), tile-padded
    const float4* b32;
    const double* a64;       // FP64 SoA, stride a64_stride (order: sorted64)
    const double* b64;
    long long a64_stride, b64_stride;
    long long tiles_a, tiles_b;
    long long item_begin;    // first global item (tile pair) of this count
    long long n_items;       // tile pairs of this count
    unsigned long long* counts;  // K+2 slots (slot K+1 filled by the finalize kernel)
    unsigned long long total;    // pairs of the count: n(n-1)/2 or n_a n_b
    long long item_offset;   // item of the count that global item item_begin is
    const unsigned* item_list;   // if set: the count's kept items (tile pairs not skipped)
    const float4* b_caps;    // bounding spheres of B's chunks of 32 sorted points, or null
    int is_auto;
    int sorted64;            // bit 0 (a64), bit 1 (b64): in the spatial order, else original
};

// Bounding cap of one tile of spatially ordered points: unit centre and an
// angular radius (radians) that bounds every point's angle from the centre.
struct TileCap {
    double x, y, z, rho;     // rho < 0: no real point in the tile
};

// One count of a batch, for skipping its far tile pairs on the device: its
// items in the full work table, its tiles' caps, and the list of kept items.
struct CullSeg {
    long long begin, n;
    long long offset;        // the count's item that index 0 of this range is (a shard's rows)
    const TileCap* ca;
    const TileCap* cb;
    long long ta, tb;
    unsigned* list;
    int is_auto;
    int sorted64;            // bit 0 (a64), bit 1 (b64): in the spatial order, else original
};

struct PairParams {
    Segment seg0;            // the count, when n_segs == 0
    const Segment* segs;     // device table sorted by item_begin, when n_segs > 0
    int n_segs;
    int items_per_flush;     // flush the uint32 histograms after this many items
    long long item_begin;    // this launch takes global items [item_begin, item_begin + n_items)
    long long n_items;
    const unsigned long long* n_items_dev;  // if set: at most this many items (device count)
    unsigned long long* cursor;
    unsigned long long* stats;    // WTHETA_NSTATS or null
    int span;                // settle (A group, B chunk) spans without a lookup per pair
    int pad_;
    BinTable tab;
};

struct Variant {
    int nt, r, ju, hm, def;
    void (*kernel)(PairParams);       // the build with statistics code
    void (*kernel_fast)(PairParams);  // the build launched without statistics
    size_t (*smem)(int, int);
};

struct DeviceInfo {
    int sm_count = 0;
    int max_smem_optin = 0;
};

// One catalogue made ready for the pair kernel: FP64 unit vectors (the
// caller's, or converted from RA/Dec into scratch) and spatially ordered FP32
// copies padded to whole tiles.
struct Prepared {
    const float4* p32 = nullptr;
    const float4* c32 = nullptr;   // bounding sphere of each chunk of 32 sorted points
    const double* x64 = nullptr;   // FP64 SoA (stride), in the spatial order if sorted
    long long stride = 0;
    int sorted = 0;
};

// Host-side launch plumbing (wtheta_count.cu), shared by the single-count,
// batched and serving paths.
int device_info(DeviceInfo* out);
const Variant* variants(int* n);
const Variant* pick_variant(const wtheta_tune* tune, int K, int n_lut, int max_smem);
const Variant* pick_for_size(const wtheta_tune* tune, long long n_max, int K, int n_lut,
                             int max_smem);
int grid_for(const Variant* v, size_t smem, long long n_items, int sm_count, int want_per_sm,
             int* grid);
long long round_up(long long x, long long m);
int check_cuda(cudaError_t e);
size_t prepare_bytes(long long n, long long n_pad, int is_xyz);
int prepare(const double* coords, long long n, long long n_pad, int is_xyz, int tag,
            unsigned char* scratch, int sm_count, cudaStream_t st, Prepared* out);
// The one or two catalogues of a count prepared together (b absent: nb = pb
// = 0): one conversion and key launch, one sort of the na + nb points, one
// gather into FP32 and FP64 copies with a's points at [0, pa) and b's at
// [pa, pa + pb) (each catalogue tile-padded with sentinels of tags tag0 and
// tag0 + 1: catalogues that a count may pair need different tags), one
// launch for the chunk spheres of both.  scratch: prepare_joint_bytes(na, pa,
// nb, pb); a and b may lie in its first 16 (na + nb) bytes (the FP32 copies,
// written after both are read).
size_t prepare_joint_bytes(long long na, long long pa, long long nb, long long pb);
int prepare_joint(const double* a, long long na, long long pa, const double* b, long long nb,
                  long long pb, int is_xyz, int tag0, unsigned char* scratch, int sm_count,
                  cudaStream_t st, Prepared* A, Prepared* B);
unsigned long long per_item_bound(const Variant* v);
Segment make_segment(const Prepared& A, const Prepared& B, long long ta, long long tb,
                     int is_auto, long long item_begin, unsigned long long* counts,
                     unsigned long long total);
PairParams make_params(const Variant* v, const BinTable& tab, const Segment* seg0,
                       const Segment* segs, int n_segs, long long item_begin, long long n_items,
                       unsigned long long* cursor, unsigned long long* stats);
int launch_pairs(const Variant* v, const PairParams& prm, int grid, size_t smem, cudaStream_t st);
int launch_finalize_segments(const Segment* d_segs, int n_segs, int K, cudaStream_t st);
// Spatial order of n FP64 points (SoA, stride): *order = original indices
// sorted by Hilbert key, or by (label, key) when labels (device, values in
// [0, n_labels), n_labels <= 65536) are given; *sorted_labels (optional) then
// receives the labels in that order.  scratch: order_bytes(n, labels != 0).
size_t order_bytes(long long n, int with_labels);
int spatial_order(const double* x64, long long stride, long long n, int check,
                  const int* labels, int n_labels, unsigned char* scratch, int sm_count,
                  cudaStream_t st, const unsigned** order, const unsigned** sorted_labels);
int launch_radec_to_xyz(const double* coords, long long n, double* xyz, int sm_count,
                        cudaStream_t st);
// sizes[l] += points with label l (sizes zeroed by the caller).
int launch_count_labels(const unsigned* lab, long long n, int n_labels,
                        unsigned long long* sizes, int sm_count, cudaStream_t st);
// FP32 copies with region r's sorted points (positions src[r]..src[r+1]-1 of
// order) from dst[r] on, sentinels up to dst[r+1]; dst[R] = n_pad.
int launch_gather_regions(const double* x64, long long stride, const unsigned* order,
                          const long long* src, const long long* dst, int R, long long n_pad,
                          float4* p32, int tag, int sm_count, cudaStream_t st);
// Bounding sphere of every chunk of 32 positions (sentinels mark padding).
int launch_chunk_caps(const float4* p32, long long n_pad, float4* c32, int sm_count,
                      cudaStream_t st);
// Skipping over a table of counts: kept items per count, then each count's
// kept range and list written into segs, their number into *n_kept.
int launch_cull_batch(const CullSeg* cs, int n_segs, long long total, double theta_top,
                      unsigned long long* kept, Segment* segs, unsigned long long* n_kept,
                      int sm_count, cudaStream_t st, unsigned long long* stats = nullptr);
// Bounding cap of every tile of T points (real points [0, n)).
int launch_tile_caps(const float4* p32, long long n, int T, long long tiles, TileCap* caps,
                     cudaStream_t st);
// Appends the items of one count that caps_may_meet keeps (indices < 2^32)
// to list, counting them in *n_list (which the caller zeroes).
int launch_cull_items(const TileCap* ca, const TileCap* cb, long long ta, long long tb,
                      int is_auto, long long n_items, double theta_top, unsigned* list,
                      unsigned long long* n_list, int sm_count, cudaStream_t st);
void add_launches(long long n);

// Device allocations of the library go through these, so that a test can make
// the n-th one fail on the host (wtheta_inject_alloc_failure) without
// touching the GPU.  Both return WTHETA_OK, WTHETA_ENOMEM or WTHETA_ECUDA.
int dev_malloc(void** p, size_t bytes);
int dev_malloc_async(void** p, size_t bytes, cudaStream_t st);

// A named range on the host timeline (NVTX), for profilers; costs nothing
// measurable when no tool is attached.
struct TraceRange {
    explicit TraceRange(const char* name);
    ~TraceRange();
    TraceRange(const TraceRange&) = delete;
    TraceRange& operator=(const TraceRange&) = delete;
};

// Host-side helpers (wtheta_host.cpp).
int validate_edges(const double* edges_deg, int K);
void chord2_edges(const double* edges_deg, int K, double* c);
double guard_half_width(double c);
void guard_bounds(double c, uint32_t* lo_bits, uint32_t* hi_bits, double* g);
int build_table(const double* edges_deg, int K, BinTable* t);

}  // namespace wtheta
