// Internal declarations shared by the library's host and device sources.
#pragma once
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
    uint32_t lut[kMaxLut][4];            // {lo_bits, hi_bits, slot_below, slot_above}
};

// Host-side helpers (wtheta_host.cpp).
int validate_edges(const double* edges_deg, int K);
void chord2_edges(const double* edges_deg, int K, double* c);
double guard_half_width(double c);
void guard_bounds(double c, uint32_t* lo_bits, uint32_t* hi_bits, double* g);
int build_table(const double* edges_deg, int K, BinTable* t);

}  // namespace wtheta
