// Synthetic Z on the device (input generation, not part of the method): Philox4x32-10
// (Salmon et al., SC'11) with counter (k, n, m, I) and key (seed, (gen_q << 8) | 0), then a
// Box-Muller pair scaled so that Re and Im are each N(0, 1/2), times the row scale
// s_I = 1 / (1 + I / s_div). Written from the published definition; the host-side generator
// used by the tests is a separate implementation of the same definition.
#include "internal.cuh"

namespace qsgw {

struct Philox4 {
  uint32_t x, y, z, w;
};

__device__ __forceinline__ Philox4 philox4x32_10(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3, uint32_t k0,
                                                 uint32_t k1) {
#pragma unroll
  for (int rnd = 0; rnd < 10; ++rnd) {
    if (rnd) {
      k0 += 0x9E3779B9u;
      k1 += 0xBB67AE85u;
    }
    const uint32_t hi0 = __umulhi(0xD2511F53u, c0), lo0 = 0xD2511F53u * c0;
    const uint32_t hi1 = __umulhi(0xCD9E8D57u, c2), lo1 = 0xCD9E8D57u * c2;
    const uint32_t n0 = hi1 ^ c1 ^ k0, n2 = hi0 ^ c3 ^ k1;
    c0 = n0;
    c1 = lo1;
    c2 = n2;
    c3 = lo0;
  }
  return {c0, c1, c2, c3};
}

__device__ __forceinline__ double u53(uint32_t hi, uint32_t lo) {
  const unsigned long long bits = ((unsigned long long)hi << 21) | (lo >> 11);
  return (double)bits * 0x1.0p-53;
}

__global__ void synth_z_kernel(unsigned long long seed, int gen_q, int k, int n_pb, int n_unocc, long long K,
                               double s_div, double2* __restrict__ Z, long long ldz) {
  const uint32_t key0 = (uint32_t)seed, key1 = ((uint32_t)gen_q << 8) | 0u;
  const long long total = K * n_pb;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const long long r = e / n_pb;
    const int I = (int)(e % n_pb);
    const int n = (int)(r / n_unocc), m = (int)(r % n_unocc);
    const Philox4 o = philox4x32_10((uint32_t)k, (uint32_t)n, (uint32_t)m, (uint32_t)I, key0, key1);
    const double u1 = u53(o.x, o.y) + 0x1.0p-53;  // (0, 1]
    const double u2 = u53(o.z, o.w);
    const double rad = sqrt(-log(u1));
    const double ang = 2.0 * 3.14159265358979323846 * u2;
    double sn, cs;
    sincos(ang, &sn, &cs);
    const double sI = 1.0 / (1.0 + (double)I / s_div);
    Z[(size_t)r * ldz + I] = make_double2(rad * cs * sI, rad * sn * sI);
  }
}

void launch_synth_z(unsigned long long seed, int gen_q, int k, int n_pb, int n_occ, int n_unocc, double s_div,
                    double2* Z, long long ldz, cudaStream_t s) {
  const long long K = (long long)n_occ * n_unocc;
  const long long total = K * n_pb;
  long long blocks = (total + 255) / 256;
  if (blocks > 152 * 32) blocks = 152 * 32;
  if (blocks < 1) blocks = 1;
  synth_z_kernel<<<(int)blocks, 256, 0, s>>>(seed, gen_q, k, n_pb, n_unocc, K, s_div, Z, ldz);
}

}  // namespace qsgw
