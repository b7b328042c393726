// FP64 path: transition weights (step a1) and the FP64 complex HERK (step a4, plain form).
//
// chi0(l) = -s * sum_r |w_l(Delta_r)| conj(z_{I,r}) z_{J,r} with |w_l(Delta)| = 2 Delta/(Delta^2 + omega_l^2)
// (Sec. 2, Eq. (polfx) at w = i omega). The accumulator holds the positive-weight sum; the
// factor -s is applied when chi0 is read out.
//
// GB300 executes FP64 on CUDA cores at ~1 TFLOP/s (measured), so this kernel is DFMA-bound by
// a wide margin: operands are staged through shared memory once per 16-column K-step, each
// thread keeps a 4x4 block of complex accumulators in registers, and only tiles on or above
// the diagonal are computed.
#include "internal.cuh"

namespace qsgw {

__global__ void weights_fp64_kernel(const double* __restrict__ eo, const double* __restrict__ eu, int n_occ,
                                    int n_unocc, OmegaGrid g, double* __restrict__ w, long long ldw, int* d_err) {
  const long long K = (long long)n_occ * n_unocc;
  for (long long r = blockIdx.x * (long long)blockDim.x + threadIdx.x; r < K; r += (long long)gridDim.x * blockDim.x) {
    const int n = (int)(r / n_unocc), m = (int)(r % n_unocc);
    const double d = eu[m] - eo[n];  // Delta_knm
    const bool ok = (d > 0.0) && isfinite(d);
    if (!ok) atomicCAS(d_err, DEV_OK, DEV_DOMAIN);
    for (int l = 0; l < g.L; ++l) w[l * ldw + r] = ok ? 2.0 * d / (d * d + g.w2[l]) : 0.0;
  }
}

void launch_weights_fp64(const double* eps_occ, const double* eps_unocc, int n_occ, int n_unocc, const OmegaGrid& g,
                         double* w, long long ldw, int* d_err, cudaStream_t s) {
  const long long K = (long long)n_occ * n_unocc;
  int blocks = (int)((K + 255) / 256);
  if (blocks > 152 * 16) blocks = 152 * 16;
  if (blocks < 1) blocks = 1;
  weights_fp64_kernel<<<blocks, 256, 0, s>>>(eps_occ, eps_unocc, n_occ, n_unocc, g, w, ldw, d_err);
}

// Given column weights (one set, L = 1): w[r] = v[r mod period], checked v > 0 and finite. Used
// for Eq. (sigx), where column r = n' * n_pb + mu carries the Coulomb eigenvalue v_mu(k).
__global__ void weights_given_fp64_kernel(const double* __restrict__ v, int period, long long K,
                                          double* __restrict__ w, int* d_err) {
  for (long long r = blockIdx.x * (long long)blockDim.x + threadIdx.x; r < K; r += (long long)gridDim.x * blockDim.x) {
    const double x = v[r % period];
    const bool ok = (x > 0.0) && isfinite(x);
    if (!ok) atomicCAS(d_err, DEV_OK, DEV_DOMAIN);
    w[r] = ok ? x : 0.0;
  }
}

void launch_weights_given_fp64(const double* v, int period, long long K, double* w, int* d_err, cudaStream_t s) {
  int blocks = (int)((K + 255) / 256);
  if (blocks > 152 * 16) blocks = 152 * 16;
  if (blocks < 1) blocks = 1;
  weights_given_fp64_kernel<<<blocks, 256, 0, s>>>(v, period, K, w, d_err);
}

constexpr int kT = 64;   // output tile (I and J)
constexpr int kKS = 16;  // K-step (columns staged per iteration)

// One 64 x 64 output tile (I tile ti, J tile tj) of one frequency over columns [r_begin, r_end):
// sum_r w[r] conj(Z[I, r]) Z[J, r], added to out (add) or stored into it.
__device__ __forceinline__ void herk_fp64_tile(const double2* __restrict__ Z, long long ldz, int n_pb, int n_pad,
                                               long long r_begin, long long r_end, const double* __restrict__ wl,
                                               int ti, int tj, double2* __restrict__ out, bool add) {
  __shared__ double2 sA[kKS][kT];
  __shared__ double2 sB[kKS][kT];
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  const int i0 = ti * kT, j0 = tj * kT;

  double cr[4][4], ci[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) cr[a][b] = ci[a][b] = 0.0;

  for (long long r0 = r_begin; r0 < r_end; r0 += kKS) {
    __syncthreads();
#pragma unroll
    for (int e = tid; e < kKS * kT; e += 256) {
      const int rr = e / kT, ii = e % kT;
      const long long r = r0 + rr;
      double2 za = make_double2(0.0, 0.0), zb = make_double2(0.0, 0.0);
      if (r < r_end) {
        if (i0 + ii < n_pb) za = Z[(i0 + ii) + r * ldz];
        if (j0 + ii < n_pb) {
          const double wr = wl[r];
          zb = Z[(j0 + ii) + r * ldz];
          zb.x *= wr;
          zb.y *= wr;
        }
      }
      sA[rr][ii] = za;
      sB[rr][ii] = zb;
    }
    __syncthreads();
#pragma unroll 4
    for (int rr = 0; rr < kKS; ++rr) {
      double2 a[4], b[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        a[q] = sA[rr][ty + 16 * q];
        b[q] = sB[rr][tx + 16 * q];
      }
#pragma unroll
      for (int p = 0; p < 4; ++p)
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          // conj(a) * b
          cr[p][q] = fma(a[p].x, b[q].x, cr[p][q]);
          cr[p][q] = fma(a[p].y, b[q].y, cr[p][q]);
          ci[p][q] = fma(a[p].x, b[q].y, ci[p][q]);
          ci[p][q] = fma(-a[p].y, b[q].x, ci[p][q]);
        }
    }
  }
#pragma unroll
  for (int p = 0; p < 4; ++p)
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int I = i0 + ty + 16 * p, J = j0 + tx + 16 * q;
      double2* o = out + (size_t)J * n_pad + I;
      double2 v = add ? *o : make_double2(0.0, 0.0);
      v.x += cr[p][q];
      v.y += ci[p][q];
      *o = v;
    }
}

// grid: x = J tile - tj0, y = I tile, z = frequency + L * K-slice. Tiles strictly below the diagonal
// exit at once. With tj0 > 0 and fewer I tiles than J tiles the grid covers one off-diagonal block
// of the output: rows of I tiles [0, gridDim.y), columns of J tiles [tj0, n_pad / 64). With S = 1 the
// tile is added to acc; with S > 1 (few output tiles) slice sk covers columns [K sk / S, K (sk + 1) / S)
// and stores its tile into its own partial buffer part[sk], which herk_fp64_reduce_kernel then adds
// to acc in slice order (deterministic).
__global__ void __launch_bounds__(256) herk_fp64_kernel(const double2* __restrict__ Z, long long ldz, int n_pb,
                                                        int n_pad, long long K, const double* __restrict__ w,
                                                        long long ldw, int L, int S, int tj0,
                                                        double2* __restrict__ acc, double2* __restrict__ part) {
  const int tj = blockIdx.x + tj0, ti = blockIdx.y, l = blockIdx.z % L, sk = blockIdx.z / L;
  if (tj < ti) return;
  const size_t nn = (size_t)n_pad * n_pad;
  double2* out = S == 1 ? acc + (size_t)l * nn : part + ((size_t)sk * L + l) * nn;
  herk_fp64_tile(Z, ldz, n_pb, n_pad, K * sk / S, K * (sk + 1) / S, w + (long long)l * ldw, ti, tj, out, S == 1);
}

// Batch over blocks of distinct q-points in one launch: grid (items, frequency), item = (block,
// upper-triangle tile, K-slice), each block with the slice count the one-block path would pick, so
// the sums run in the same order and the result is bitwise that of one launch per block.
__global__ void __launch_bounds__(256) herk_fp64_batch_kernel(const __grid_constant__ Fp64Batch p) {
  const int l = blockIdx.y;
  int b = 0;
  while (b + 1 < p.nb && p.b[b + 1].item0 <= (int)blockIdx.x) ++b;
  const Fp64Blk& B = p.b[b];
  const int local = blockIdx.x - B.item0, sk = local % B.S, t = local / B.S;
  int tj = (int)((sqrt(8.0 * t + 1.0) - 1.0) * 0.5);  // upper tile (ti, tj), ti <= tj, by column
  while ((tj + 1) * (tj + 2) / 2 <= t) ++tj;
  while (tj * (tj + 1) / 2 > t) --tj;
  const int ti = t - tj * (tj + 1) / 2;
  const size_t nn = (size_t)B.n_pad * B.n_pad;
  double2* out = B.S == 1 ? B.acc + (size_t)l * nn : B.part + ((size_t)sk * p.L + l) * nn;
  herk_fp64_tile(B.Z, B.ldz, B.n_pb, B.n_pad, B.K * sk / B.S, B.K * (sk + 1) / B.S, B.w + (long long)l * B.ldw, ti,
                 tj, out, B.S == 1);
}

// acc += sum over slices sk = 0 .. S-1 of part[sk], on the upper-triangle tiles; grid as the HERK
// without the slice dimension.
__global__ void __launch_bounds__(256) herk_fp64_reduce_kernel(int n_pad, int L, int S, int tj0,
                                                               const double2* __restrict__ part,
                                                               double2* __restrict__ acc) {
  const int tj = blockIdx.x + tj0, ti = blockIdx.y, l = blockIdx.z;
  if (tj < ti) return;
  const size_t nn = (size_t)n_pad * n_pad;
  for (int e = threadIdx.x; e < kT * kT; e += 256) {
    const size_t o = (size_t)(tj * kT + e / kT) * n_pad + ti * kT + e % kT;
    double2 v = acc[l * nn + o];
    for (int sk = 0; sk < S; ++sk) {
      const double2 x = part[((size_t)sk * L + l) * nn + o];
      v.x += x.x;
      v.y += x.y;
    }
    acc[l * nn + o] = v;
  }
}

int herk_fp64_slices(int n_pad, int L, long long K, int ti_end, int tj0) {
  const int nt = n_pad / kT;
  const long long tiles =
      (ti_end > 0 ? (long long)ti_end * (nt - tj0) : (long long)nt * (nt + 1) / 2) * L;
  const long long want = 2 * 152;  // two CTAs per SM of a GB300
  long long S = tiles >= want ? 1 : (want + tiles - 1) / tiles;
  const long long steps = (K + kKS - 1) / kKS;
  if (S > 16) S = 16;
  if (S > steps) S = steps > 0 ? steps : 1;
  return (int)S;
}

void launch_herk_fp64_batch(const Fp64Batch& p, cudaStream_t s) {
  if (p.nb < 1 || p.items < 1) return;
  herk_fp64_batch_kernel<<<dim3(p.items, p.L), 256, 0, s>>>(p);
  for (int b = 0; b < p.nb; ++b) {
    const Fp64Blk& B = p.b[b];
    if (B.S > 1) {
      const int nt = B.n_pad / kT;
      herk_fp64_reduce_kernel<<<dim3(nt, nt, p.L), 256, 0, s>>>(B.n_pad, p.L, B.S, 0, B.part, B.acc);
    }
  }
}

void launch_herk_fp64(const double2* Z, long long ldz, int n_pb, int n_pad, long long K, const double* w,
                      long long ldw, int L, int S, double2* acc, double2* part, cudaStream_t s, int ti_end, int tj0) {
  const int nt = n_pad / kT, ny = ti_end > 0 ? ti_end : nt;
  dim3 grid(nt - tj0, ny, L * S);
  herk_fp64_kernel<<<grid, 256, 0, s>>>(Z, ldz, n_pb, n_pad, K, w, ldw, L, S, tj0, acc, part);
  if (S > 1) herk_fp64_reduce_kernel<<<dim3(nt - tj0, ny, L), 256, 0, s>>>(n_pad, L, S, tj0, part, acc);
}

}  // namespace qsgw
