// Mixed-precision chi0 assembly on tcgen05 tensor cores (declarations).
#pragma once
#include "internal.cuh"

namespace qsgw {

struct MixedScratch {
  void* planes = nullptr;  // digit planes of the row operand
  size_t planes_cap = 0;
  void* aux = nullptr;  // per-column weights / scales
  size_t aux_cap = 0;
};

qsgw_status mixed_accumulate(MixedScratch& s, const double2* Z, long long ldz, int n_pb, int n_pad, int n_occ,
                             int n_unocc, const double* eo, const double* eu, const OmegaGrid& g, float4* acc,
                             int* d_err, cudaStream_t stream);
void mixed_free(MixedScratch& s);

}  // namespace qsgw
