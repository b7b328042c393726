// Mixed-precision chi0 assembly (tcgen05). Placeholder until the tensor-core path lands.
#include "mixed.cuh"

namespace qsgw {

qsgw_status mixed_accumulate(MixedScratch&, const double2*, long long, int, int, int, int, const double*,
                             const double*, const OmegaGrid&, float4*, int*, cudaStream_t) {
  return QSGW_ERR_STATE;
}

void mixed_free(MixedScratch& s) {
  if (s.planes) cudaFree(s.planes);
  if (s.aux) cudaFree(s.aux);
  s = MixedScratch{};
}

}  // namespace qsgw
