// Real-axis route of chi0 (Eqs. (impolf) and (hilbert), Sec. 2): the transition columns are put
// in the histogram bins [edges[j], edges[j+1]) holding their energy Delta, gathered bin by bin
// (pair compaction) into per-bin staging that collects the columns of many accumulate calls, and
// each bin's spectral weight S_j = sum_{r in bin j} conj(z_I,r) z_J,r is a Hermitian update run by
// the chi0 kernels with weight 1 over the staged columns. The kernels here do the binning, a
// stable counting sort of the columns by bin, the gather, and the real-axis chi0 (the Hilbert
// transformation and the anti-Hermitian part). Every step is deterministic.
#include "internal.cuh"

namespace qsgw {

// Bin of every column r = n * n_unocc + m (Delta = eu[m] - eo[n]); -1 outside all bins. Delta <= 0
// or non-finite sets DEV_DOMAIN.
__global__ void hist_bin_kernel(const double* __restrict__ eo, const double* __restrict__ eu, int n_occ,
                                int n_unocc, const double* __restrict__ edges, int n_bins, int* __restrict__ bins,
                                int* d_err) {
  const long long K = (long long)n_occ * n_unocc;
  for (long long r = blockIdx.x * (long long)blockDim.x + threadIdx.x; r < K; r += (long long)gridDim.x * blockDim.x) {
    const double d = eu[r % n_unocc] - eo[r / n_unocc];
    if (!(d > 0.0) || !isfinite(d)) atomicCAS(d_err, DEV_OK, DEV_DOMAIN);
    int b = -1;
    if (d >= edges[0] && d < edges[n_bins]) {  // largest j with edges[j] <= d
      int lo = 0, hi = n_bins - 1;
      while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (edges[mid] <= d) lo = mid; else hi = mid - 1;
      }
      b = lo;
    }
    bins[r] = b;
  }
}

// One CTA (256 threads) per bin: number of columns in the bin.
__global__ void __launch_bounds__(256) hist_count_kernel(const int* __restrict__ bins, long long K,
                                                         int* __restrict__ counts) {
  __shared__ int part[8];
  const int j = blockIdx.x;
  int c = 0;
  for (long long r = threadIdx.x; r < K; r += 256) c += bins[r] == j;
  for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
  if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = c;
  __syncthreads();
  if (threadIdx.x == 0) {
    int t = 0;
    for (int w = 0; w < 8; ++w) t += part[w];
    counts[j] = t;
  }
}

// Exclusive scan of the bin counts (offsets[n_bins] = columns inside all bins); one thread.
__global__ void hist_scan_kernel(const int* __restrict__ counts, int n_bins, int* __restrict__ offsets) {
  if (blockIdx.x != 0 || threadIdx.x != 0) return;
  int s = 0;
  for (int j = 0; j < n_bins; ++j) {
    offsets[j] = s;
    s += counts[j];
  }
  offsets[n_bins] = s;
}

// One CTA (1024 threads) per bin: the bin's columns in increasing r, written to
// perm[offsets[j] ...] (a stable counting sort: ballot and popc within warps, warp totals in smem).
__global__ void __launch_bounds__(1024) hist_perm_kernel(const int* __restrict__ bins, long long K,
                                                         const int* __restrict__ offsets, int* __restrict__ perm) {
  __shared__ int wsum[32];
  const int j = blockIdx.x, t = threadIdx.x, lane = t & 31, w = t >> 5;
  int base = offsets[j];
  for (long long r0 = 0; r0 < K; r0 += 1024) {
    const long long r = r0 + t;
    const bool f = r < K && bins[r] == j;
    const unsigned m = __ballot_sync(0xffffffffu, f);
    if (lane == 0) wsum[w] = __popc(m);
    __syncthreads();
    int before = 0, total = 0;
    for (int q = 0; q < 32; ++q) {
      before += q < w ? wsum[q] : 0;
      total += wsum[q];
    }
    if (f) perm[base + before + __popc(m & ((1u << lane) - 1u))] = (int)r;
    base += total;
    __syncthreads();
  }
}

__device__ __forceinline__ void put(double2* d, double2 x) { *d = x; }
__device__ __forceinline__ void put(float2* d, double2 x) { *d = make_float2((float)x.x, (float)x.y); }

// Column p of the sorted order, Z[:, perm[p]] in bin j = bins[perm[p]], goes to column
// p - offsets[j] of that bin's destination dptr[j] (n_pb complex values per column; one CTA per
// column). complex64 destinations take Z rounded to nearest, the rounding the digit preparation
// applies to complex128 input, so staging in complex64 leaves the mixed-precision result unchanged.
template <typename T>
__global__ void __launch_bounds__(256) gather_bins_kernel(const double2* __restrict__ Z, long long ldz, int n_pb,
                                                          const int* __restrict__ perm, const int* __restrict__ bins,
                                                          const int* __restrict__ offsets, T* const* __restrict__ dptr) {
  const int p = blockIdx.x;
  const int r = perm[p];
  const int j = bins[r];
  const double2* src = Z + (long long)r * ldz;
  T* dst = dptr[j] + (long long)(p - offsets[j]) * n_pb;
  for (int i = threadIdx.x; i < n_pb; i += 256) put(dst + i, src[i]);
}

// Real-axis chi0 from the spectral weights (Eqs. (hilbert) and (impolf)), for NO outputs
// o0 .. o0 + NO - 1 (those below n_out):
//   out[o] = sum_j K[j][o] S_j + i coef[o] S_{bins_out[o]},
// the first sum being the Hilbert transformation of the histogram and the second term the
// anti-Hermitian part inside the output's own bin. S_j is exactly Hermitian (the readout writes
// the mirror of its upper triangle), so the Hermitian part H_o is too: each thread computes one
// element on or above the diagonal and writes its mirror, out_JI = conj(H_IJ) + i coef conj(S_IJ).
// The bins are summed in increasing j in FP64. Block (32, 8): 32 rows I by 8 columns J; grid
// (row tiles, column groups, output groups); blocks wholly below the diagonal leave at once.
constexpr int kHilbChunk = 128;  // bins of K staged in shared memory at a time

template <int NO>
__global__ void __launch_bounds__(256) hilbert_kernel(const double2* __restrict__ S, int n, int nb, int n_out,
                                                      const double* __restrict__ K, const int* __restrict__ bins_out,
                                                      const double* __restrict__ coef, double2* __restrict__ out) {
  __shared__ double sK[kHilbChunk][NO];
  if (blockIdx.x * 32 > blockIdx.y * 8 + 7) return;
  const int I = blockIdx.x * 32 + threadIdx.x, J = blockIdx.y * 8 + threadIdx.y;
  const int tid = threadIdx.y * 32 + threadIdx.x, o0 = blockIdx.z * NO;
  const bool act = I <= J && J < n;
  const long long nn = (long long)n * n, e = (long long)J * n + I;
  double hr[NO], hi[NO];
#pragma unroll
  for (int o = 0; o < NO; ++o) hr[o] = hi[o] = 0.0;
  for (int j0 = 0; j0 < nb; j0 += kHilbChunk) {
    const int cnt = min(kHilbChunk, nb - j0);
    __syncthreads();
    for (int t = tid; t < cnt * NO; t += 256) {
      const int jj = t / NO, oo = t % NO;
      sK[jj][oo] = o0 + oo < n_out ? K[(long long)(j0 + jj) * n_out + o0 + oo] : 0.0;
    }
    __syncthreads();
    if (act) {
      const double2* sp = S + (long long)j0 * nn + e;
      for (int jj = 0; jj < cnt; ++jj) {
        const double2 v = sp[jj * nn];
#pragma unroll
        for (int o = 0; o < NO; ++o) {
          hr[o] = fma(sK[jj][o], v.x, hr[o]);
          hi[o] = fma(sK[jj][o], v.y, hi[o]);
        }
      }
    }
  }
  if (!act) return;
#pragma unroll
  for (int o = 0; o < NO; ++o) {
    if (o0 + o >= n_out) break;
    const double c = coef[o0 + o];
    const double2 sb = S[(long long)bins_out[o0 + o] * nn + e];
    double2* dst = out + (long long)(o0 + o) * nn;
    dst[e] = make_double2(hr[o] - c * sb.y, hi[o] + c * sb.x);
    if (I != J) dst[(long long)I * n + J] = make_double2(hr[o] + c * sb.y, c * sb.x - hi[o]);
  }
}

void launch_hist_sort(const double* eo, const double* eu, int n_occ, int n_unocc, const double* edges, int n_bins,
                      int* bins, int* counts, int* offsets, int* perm, int* d_err, cudaStream_t s) {
  const long long K = (long long)n_occ * n_unocc;
  int blocks = (int)((K + 255) / 256);
  if (blocks > 152 * 16) blocks = 152 * 16;
  hist_bin_kernel<<<blocks, 256, 0, s>>>(eo, eu, n_occ, n_unocc, edges, n_bins, bins, d_err);
  hist_count_kernel<<<n_bins, 256, 0, s>>>(bins, K, counts);
  hist_scan_kernel<<<1, 1, 0, s>>>(counts, n_bins, offsets);
  hist_perm_kernel<<<n_bins, 1024, 0, s>>>(bins, K, offsets, perm);
}

void launch_gather_bins(const double2* Z, long long ldz, int n_pb, const int* perm, const int* bins,
                        const int* offsets, int n, void* const* dptr, bool z32, cudaStream_t s) {
  if (n <= 0) return;
  if (z32)
    gather_bins_kernel<float2><<<n, 256, 0, s>>>(Z, ldz, n_pb, perm, bins, offsets,
                                                 reinterpret_cast<float2* const*>(dptr));
  else
    gather_bins_kernel<double2><<<n, 256, 0, s>>>(Z, ldz, n_pb, perm, bins, offsets,
                                                  reinterpret_cast<double2* const*>(dptr));
}

void launch_hilbert(const double2* S, int n, int nb, int n_out, const double* K, const int* bins_out,
                    const double* coef, double2* out, cudaStream_t s) {
  // output groups of at most 12 (registers), sized evenly and rounded up to a multiple of 4
  const int groups = (n_out + 11) / 12;
  const int per = ((n_out + groups - 1) / groups + 3) / 4 * 4;
  const dim3 grid((n + 31) / 32, (n + 7) / 8, (n_out + per - 1) / per), block(32, 8);
  if (per == 4)
    hilbert_kernel<4><<<grid, block, 0, s>>>(S, n, nb, n_out, K, bins_out, coef, out);
  else if (per == 8)
    hilbert_kernel<8><<<grid, block, 0, s>>>(S, n, nb, n_out, K, bins_out, coef, out);
  else
    hilbert_kernel<12><<<grid, block, 0, s>>>(S, n, nb, n_out, K, bins_out, coef, out);
}

}  // namespace qsgw
