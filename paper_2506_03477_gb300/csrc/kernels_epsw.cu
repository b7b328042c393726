// Epilogue kernels (steps a6, a7, a9): read-out of the chi0 accumulator as a full Hermitian
// matrix, formation of eps, and W from the Cholesky inverse. All are HBM-bound streaming
// kernels; transposed reads go through a 32x33 shared-memory tile so every global access is
// coalesced.
//
//   chi0 = -s * acc, mirrored: chi0_IJ = conj(chi0_JI), diag imaginary part exactly 0
//   eps  = I - D chi0 D,  D = diag(sqrt v)                       Eq. (dielectricfunction)
//   W    = D eps^{-1} D, W^c = W - diag(v)                       Eq. (screenedcoulomb), Eq. (wc)
#include "internal.cuh"

namespace qsgw {

// Accumulator element (I, J) of frequency l, `loc` = J * n_pad + I.
// ACC_FP64: double2 [l][J][I]. ACC_DF32: float2 (hi, lo) planes [l][re|im][J][I], then an FP64
// buffer of the same layout (pieces of split tiles).
template <int KIND>
__device__ __forceinline__ double2 load_acc(const void* acc, int l, size_t loc, int n_pad) {
  const size_t nn = (size_t)n_pad * n_pad;
  if (KIND == ACC_FP64) return static_cast<const double2*>(acc)[(size_t)l * nn + loc];
  const float2* a = static_cast<const float2*>(acc) + (size_t)l * 2 * nn + loc;
  // FP64 buffer of the split tiles after the double-float one (gridDim.z = number of frequencies)
  const double* b = reinterpret_cast<const double*>(static_cast<const float2*>(acc) + (size_t)gridDim.z * 2 * nn) +
                    (size_t)l * 2 * nn + loc;
  const float2 re = a[0], im = a[nn];
  return make_double2(((double)re.x + (double)re.y) + b[0], ((double)im.x + (double)im.y) + b[nn]);
}

// MODE 0: out = chi0. MODE 1: out = eps. Grid (n/32 J-blocks, n/32 I-blocks, L), block (32, 8).
template <int KIND, int MODE>
__global__ void readout_kernel(const void* __restrict__ acc, int n, int n_pad, double spin,
                               const double* __restrict__ v, double2* __restrict__ out) {
  __shared__ double2 t[32][33];
  const int bj = blockIdx.x, bi = blockIdx.y, l = blockIdx.z;
  const int tx = threadIdx.x, ty = threadIdx.y;
  const bool upper = bi <= bj;
  // stage the source block: for an upper/diagonal output block it is acc block (bi, bj) with
  // t[jj][ii] = acc(I, J); for a lower block it is acc block (bj, bi) with t[ii][jj] = acc(J, I).
  for (int y = ty; y < 32; y += 8) {
    size_t loc;
    if (upper) loc = (size_t)(bj * 32 + y) * n_pad + (bi * 32 + tx);  // t[y=jj][tx=ii]
    else       loc = (size_t)(bi * 32 + y) * n_pad + (bj * 32 + tx);  // t[y=ii][tx=jj]
    t[y][tx] = load_acc<KIND>(acc, l, loc, n_pad);
  }
  __syncthreads();
  for (int y = ty; y < 32; y += 8) {
    const int ii = tx, jj = y;
    const int I = bi * 32 + ii, J = bj * 32 + jj;
    if (I >= n || J >= n) continue;
    double2 a;
    if (upper) a = (bi < bj || ii <= jj) ? t[jj][ii] : make_double2(t[ii][jj].x, -t[ii][jj].y);
    else a = make_double2(t[ii][jj].x, -t[ii][jj].y);
    double2 c = make_double2(-spin * a.x, I == J ? 0.0 : -spin * a.y);  // chi0
    if (MODE == 1) {
      const double d = sqrt(v[I]) * sqrt(v[J]);
      c = make_double2((I == J ? 1.0 : 0.0) - d * c.x, -d * c.y);
    }
    out[(size_t)l * n * n + (size_t)J * n + I] = c;
  }
}

template <int MODE>
static void launch_readout(const void* acc, AccKind kind, int n, int n_pad, int L, double spin, const double* v,
                           double2* out, cudaStream_t s) {
  const int nb = (n + 31) / 32;
  dim3 grid(nb, nb, L), block(32, 8);
  if (kind == ACC_FP64) readout_kernel<ACC_FP64, MODE><<<grid, block, 0, s>>>(acc, n, n_pad, spin, v, out);
  else readout_kernel<ACC_DF32, MODE><<<grid, block, 0, s>>>(acc, n, n_pad, spin, v, out);
}

void launch_finalize_chi(const void* acc, AccKind kind, int n, int n_pad, int L, double spin, double2* out,
                         cudaStream_t s) {
  launch_readout<0>(acc, kind, n, n_pad, L, spin, nullptr, out, s);
}

void launch_form_eps(const void* acc, AccKind kind, int n, int n_pad, int L, double spin, const double* v,
                     double2* eps, cudaStream_t s) {
  launch_readout<1>(acc, kind, n, n_pad, L, spin, v, eps, s);
}

// In place on w ([L][n][n], column-major): the lower triangle holds sg * eps^{-1} (sg = +-1); write
// the full W = D eps^{-1} D (minus diag(v) when wc != 0). One CTA per lower block pair (bi >= bj):
// it reads its lower block before writing it and its (never read) mirror block above the diagonal.
__global__ void w_from_inverse_kernel(double2* __restrict__ w, int n, const double* __restrict__ v, int wc,
                                      double sg) {
  const int bj = blockIdx.x, bi = blockIdx.y, l = blockIdx.z;
  if (bi < bj) return;
  __shared__ double2 t[32][33];
  double2* m = w + (size_t)l * n * n;
  const int tx = threadIdx.x, ty = threadIdx.y;
  for (int y = ty; y < 32; y += 8) {  // t[jj][ii] = X(I = bi*32+ii, J = bj*32+jj), lower part valid
    const int I = bi * 32 + tx, J = bj * 32 + y;
    t[y][tx] = (I < n && J < n) ? m[(size_t)J * n + I] : make_double2(0.0, 0.0);
  }
  __syncthreads();
  // block (bi, bj): elements with I >= J come from t directly, diagonal-block upper part mirrors.
  for (int y = ty; y < 32; y += 8) {
    const int ii = tx, jj = y, I = bi * 32 + ii, J = bj * 32 + jj;
    if (I >= n || J >= n) continue;
    double2 x = (bi > bj || ii >= jj) ? t[jj][ii] : make_double2(t[ii][jj].x, -t[ii][jj].y);
    const double d = sg * (sqrt(v[I]) * sqrt(v[J]));
    double2 o = make_double2(d * x.x, I == J ? 0.0 : d * x.y);
    if (wc && I == J) o.x -= v[I];
    m[(size_t)J * n + I] = o;
  }
  if (bi == bj) return;
  // mirror block (bj, bi): W(J', I') with J' = bj*32+jj (row), I' = bi*32+ii (col) = conj(W(I', J'))
  for (int y = ty; y < 32; y += 8) {
    const int jj = tx, ii = y;  // row index jj fastest for coalescing
    const int R = bj * 32 + jj, C = bi * 32 + ii;
    if (R >= n || C >= n) continue;
    const double2 x = t[jj][ii];  // X(C, R)
    const double d = sg * (sqrt(v[R]) * sqrt(v[C]));
    m[(size_t)C * n + R] = make_double2(d * x.x, -d * x.y);
  }
}

void launch_w_from_inverse(double2* w, int n, int L, const double* v, int wc, double sg, cudaStream_t s) {
  const int nb = (n + 31) / 32;
  dim3 grid(nb, nb, L), block(32, 8);
  w_from_inverse_kernel<<<grid, block, 0, s>>>(w, n, v, wc, sg);
}

}  // namespace qsgw
