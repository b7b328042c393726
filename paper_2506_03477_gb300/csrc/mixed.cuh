// Mixed-precision chi0 assembly on tcgen05 tensor cores (declarations).
#pragma once
#include "internal.cuh"

namespace qsgw {

// Device scratch owned by a context for the mixed path, grown on demand and reused by every
// accumulate call: digit planes of the row operand, FP32 copy of Z for the column operand,
// FP32 weights, per-chunk maxima / exponents, and the list of upper-triangle tiles.
struct MixedScratch {
  void* planes = nullptr;
  size_t planes_cap = 0;
  void* aux = nullptr;  // int2 tile list
  int n_tiles = 0;
  int tiles_key_n = -1;
  int tiles_key_tj = -1;
  bool attr_set = false;
  int n_sm = 0;
};

// acc: two double-float accumulators back to back, each float2 (hi, lo) planes
// [L][2 (re, im)][n_pad (J)][n_pad (I)]; chi0 is their sum.
qsgw_status mixed_accumulate(MixedScratch& s, const double2* Z, long long ldz, int n_pb, int n_pad, int n_occ,
                             int n_unocc, const double* eo, const double* eu, const OmegaGrid& g, float4* acc,
                             int* d_err, cudaStream_t stream);
void mixed_free(MixedScratch& s);

}  // namespace qsgw
