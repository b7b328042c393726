// eps^{-1} in FP64 for every frequency at once (step a8): the Hermitian positive definite eps of
// Eq. (dielectricfunction) is inverted by a block sweep whose pivot blocks are factored by
// Cholesky. The paper keeps this inversion in double precision even in its mixed-precision mode.
//
// Sweep on pivot block k (rows and columns [k0, k0 + bk), bk <= 32), on the current matrix A:
//   S     = A_kk^{-1}                    Cholesky A_kk = L L^H, S = L^{-H} L^{-1}
//   A_ik <- A_ik S,  A_kj <- S A_kj      (i, j outside the block)
//   A_ij <- A_ij - A_ik S A_kj           (i, j outside the block)
//   A_kk <- -S
// After every block has been swept once, in order, A = -eps^{-1}. The pivot block of step k is
// the Schur complement of the leading k0 x k0 block, whose Cholesky factor is the diagonal block
// of eps's own Cholesky factor L. So a pivot that is not positive at local column m means that
// the leading minor of order k0 + m + 1 is not positive definite: the same index a Cholesky
// factorisation of eps reports first. The flop count, N^3 / 2 complex multiply-adds, equals that
// of a Cholesky factorisation plus the inverse from the factor. Every step except the tiny pivot
// is a rank-bk update of the whole lower triangle, so all SMs stay busy to the last step (the
// trailing matrix of a right-looking Cholesky shrinks, and its last steps leave most SMs idle).
//
// GB300 runs FP64 on the CUDA cores at ~1.2 TFLOP/s with DFMA (faster than its FP64 MMA, ~1.05
// TFLOP/s, both measured), so the update is a DFMA register-tile kernel: 64 x 64 output tiles,
// 4 x 4 complex accumulators per thread, operands staged in shared memory. Only the lower triangle
// of A is read or written (element (I, J), I >= J, at J * n + I of each frequency's matrix).
#include "internal.cuh"

namespace qsgw {

constexpr int SB = 32;  // pivot block width
constexpr int ST = 64;  // update tile (rows and columns)

__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
  return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ double2 conj2(double2 a) { return make_double2(a.x, -a.y); }

// One CTA per frequency: Cholesky of the pivot block, its inverse S (written whole to sbuf[l],
// column-major SB x SB), and A_kk <- -S on the lower triangle. info[l] keeps the first
// non-positive pivot (1-based global index); a failed pivot continues with 1 so the sweep runs to
// its end, and that frequency's result is unspecified.
__global__ void __launch_bounds__(256) sweep_pivot_kernel(double2* __restrict__ w, int n, int k0, int bk,
                                                          double2* __restrict__ sbuf, int* __restrict__ info) {
  const int l = blockIdx.x, t = threadIdx.x;
  double2* m = w + (size_t)l * n * n;
  __shared__ double2 a[SB][SB + 1];  // a[i][j] = A(k0 + i, k0 + j), lower triangle
  __shared__ double2 x[SB][SB + 1];  // x = L^{-1}, lower triangle
  __shared__ int fail;
  if (t == 0) fail = 0;
  for (int e = t; e < bk * bk; e += blockDim.x) {
    const int i = e % bk, j = e / bk;
    if (i >= j) a[i][j] = m[(size_t)(k0 + j) * n + k0 + i];
  }
  __syncthreads();
  for (int j = 0; j < bk; ++j) {  // right-looking Cholesky of the block
    double d = a[j][j].x;
    if (!(d > 0.0)) {
      if (t == 0 && fail == 0) fail = j + 1;
      d = 1.0;
    }
    const double r = sqrt(d), ri = 1.0 / r;
    __syncthreads();  // every thread has read the pivot
    if (t == 0) a[j][j] = make_double2(r, 0.0);
    for (int i = j + 1 + t; i < bk; i += blockDim.x) {
      a[i][j].x *= ri;
      a[i][j].y *= ri;
    }
    __syncthreads();
    const int mt = bk - j - 1;
    for (int e = t; e < mt * mt; e += blockDim.x) {
      const int i = j + 1 + e % mt, c = j + 1 + e / mt;
      if (i >= c) {
        const double2 p = cmul(a[i][j], conj2(a[c][j]));
        a[i][c].x -= p.x;
        a[i][c].y -= p.y;
      }
    }
    __syncthreads();
  }
  if (t < bk) {  // column t of L^{-1} by forward substitution
    const int j = t;
    for (int i = 0; i < j; ++i) x[i][j] = make_double2(0.0, 0.0);
    x[j][j] = make_double2(1.0 / a[j][j].x, 0.0);
    for (int i = j + 1; i < bk; ++i) {
      double sr = 0.0, si = 0.0;
      for (int c = j; c < i; ++c) {
        const double2 u = a[i][c], v = x[c][j];
        sr = fma(u.x, v.x, fma(-u.y, v.y, sr));
        si = fma(u.x, v.y, fma(u.y, v.x, si));
      }
      const double li = 1.0 / a[i][i].x;
      x[i][j] = make_double2(-sr * li, -si * li);
    }
  }
  __syncthreads();
  double2* s = sbuf + (size_t)l * SB * SB;
  for (int e = t; e < bk * bk; e += blockDim.x) {  // S = x^H x
    const int i = e % bk, j = e / bk;
    double sr = 0.0, si = 0.0;
    for (int c = max(i, j); c < bk; ++c) {  // conj(x[c][i]) x[c][j]
      const double2 u = x[c][i], v = x[c][j];
      sr = fma(u.x, v.x, fma(u.y, v.y, sr));
      si = fma(u.x, v.y, fma(-u.y, v.x, si));
    }
    if (i == j) si = 0.0;
    s[j * SB + i] = make_double2(sr, si);
    if (i >= j) m[(size_t)(k0 + j) * n + k0 + i] = make_double2(-sr, -si);
  }
  if (t == 0 && fail != 0 && info[l] == 0) info[l] = k0 + fail;
}

// Grid (row tiles of 32, frequency). C = column block k of A for rows outside the pivot block
// (A(i, k0 + c), read from the lower triangle, conjugated above the block), P = C S. Both go to
// column-major n x SB buffers: P for the update and the write-back, C as a copy, because the
// update overwrites column and row k of A with P.
constexpr int SP = 32;  // panel rows per CTA
__global__ void __launch_bounds__(256) sweep_panel_kernel(const double2* __restrict__ w, int n, int k0, int bk,
                                                          const double2* __restrict__ sbuf, double2* __restrict__ pbuf,
                                                          double2* __restrict__ cbuf) {
  const int l = blockIdx.y, i0 = blockIdx.x * SP, t = threadIdx.x;
  const double2* m = w + (size_t)l * n * n;
  __shared__ double2 cs[SP][SB + 1];
  __shared__ double2 ss[SB][SB + 1];
  for (int e = t; e < SB * SB; e += blockDim.x) {
    const int i = e % SB, j = e / SB;
    ss[i][j] = (i < bk && j < bk) ? sbuf[(size_t)l * SB * SB + j * SB + i] : make_double2(0.0, 0.0);
  }
  for (int e = t; e < SP * SB; e += blockDim.x) {  // rows at or below the block: lower triangle, i fastest
    const int r = e % SP, c = e / SP, i = i0 + r;
    if (i >= k0) cs[r][c] = (i >= k0 + bk && i < n && c < bk) ? m[(size_t)(k0 + c) * n + i] : make_double2(0.0, 0.0);
  }
  for (int e = t; e < SP * SB; e += blockDim.x) {  // rows above the block: A(i, k0 + c) = conj(A(k0 + c, i))
    const int c = e % SB, r = e / SB, i = i0 + r;
    if (i < k0) cs[r][c] = c < bk ? conj2(m[(size_t)i * n + k0 + c]) : make_double2(0.0, 0.0);
  }
  __syncthreads();
  const int r = t % SP;
  const int i = i0 + r;
  for (int c = t / SP; c < bk; c += 256 / SP) {
    double pr = 0.0, pi = 0.0;
#pragma unroll 8
    for (int d = 0; d < SB; ++d) {
      const double2 u = cs[r][d], v = ss[d][c];
      pr = fma(u.x, v.x, fma(-u.y, v.y, pr));
      pi = fma(u.x, v.y, fma(u.y, v.x, pi));
    }
    if (i < n) {
      pbuf[((size_t)l * SB + c) * n + i] = make_double2(pr, pi);
      cbuf[((size_t)l * SB + c) * n + i] = cs[r][c];
    }
  }
}

// Grid (lower 64 x 64 tiles, frequency). A(I, J) -= sum_c P(I, c) conj(C(J, c)) for I >= J outside
// the pivot block's rows and columns; column k (J in the block) becomes P(I, J - k0), row k (I in
// the block, J left of it) becomes conj(P(J, I - k0)); the pivot block itself was written by the
// pivot kernel. Each element belongs to one CTA, and the update reads only the P and C buffers.
__global__ void __launch_bounds__(256) sweep_update_kernel(double2* __restrict__ w, int n, int k0, int bk,
                                                           const double2* __restrict__ pbuf,
                                                           const double2* __restrict__ cbuf) {
  const int l = blockIdx.y, t = threadIdx.x;
  int ti = (int)((sqrt(8.0 * blockIdx.x + 1.0) - 1.0) * 0.5);  // lower tile (ti, tj), ti >= tj
  while ((ti + 1) * (ti + 2) / 2 <= (int)blockIdx.x) ++ti;
  while (ti * (ti + 1) / 2 > (int)blockIdx.x) --ti;
  const int tj = blockIdx.x - ti * (ti + 1) / 2;
  const int I0 = ti * ST, J0 = tj * ST;
  double2* m = w + (size_t)l * n * n;
  const double2* P = pbuf + (size_t)l * SB * n;
  const double2* C = cbuf + (size_t)l * SB * n;
  constexpr int KH = 16;  // columns of P and C staged per pass
  __shared__ double2 ps[KH][ST];
  __shared__ double2 cs[KH][ST];
  const int tx = t & 15, ty = t >> 4;
  double ar[4][4], ai[4][4];
#pragma unroll
  for (int p = 0; p < 4; ++p)
#pragma unroll
    for (int q = 0; q < 4; ++q) ar[p][q] = ai[p][q] = 0.0;
  for (int c0 = 0; c0 < bk; c0 += KH) {
    __syncthreads();
    for (int e = t; e < KH * ST; e += 256) {
      const int r = e % ST, c = c0 + e / ST;
      const bool ok = c < bk;
      ps[e / ST][r] = (ok && I0 + r < n) ? P[(size_t)c * n + I0 + r] : make_double2(0.0, 0.0);
      cs[e / ST][r] = (ok && J0 + r < n) ? C[(size_t)c * n + J0 + r] : make_double2(0.0, 0.0);
    }
    __syncthreads();
#pragma unroll 4
    for (int c = 0; c < KH; ++c) {
      double2 u[4], v[4];
#pragma unroll
      for (int p = 0; p < 4; ++p) {
        u[p] = ps[c][tx + 16 * p];
        v[p] = cs[c][ty + 16 * p];
      }
#pragma unroll
      for (int p = 0; p < 4; ++p)
#pragma unroll
        for (int q = 0; q < 4; ++q) {  // u conj(v)
          ar[p][q] = fma(u[p].x, v[q].x, fma(u[p].y, v[q].y, ar[p][q]));
          ai[p][q] = fma(u[p].y, v[q].x, fma(-u[p].x, v[q].y, ai[p][q]));
        }
    }
  }
#pragma unroll
  for (int q = 0; q < 4; ++q)
#pragma unroll
    for (int p = 0; p < 4; ++p) {
      const int I = I0 + tx + 16 * p, J = J0 + ty + 16 * q;
      if (I >= n || J >= n || I < J) continue;
      const bool inI = (unsigned)(I - k0) < (unsigned)bk, inJ = (unsigned)(J - k0) < (unsigned)bk;
      if (inI && inJ) continue;
      double2* o = m + (size_t)J * n + I;
      if (inJ) {
        *o = P[(size_t)(J - k0) * n + I];
      } else if (inI) {
        *o = conj2(P[(size_t)(I - k0) * n + J]);
      } else {
        double2 a = *o;
        a.x -= ar[p][q];
        a.y -= ai[p][q];
        *o = a;
      }
    }
}

void launch_eps_inverse(double2* w, int n, int L, double2* sbuf, double2* pbuf, double2* cbuf, int* d_info,
                        cudaStream_t s) {
  const int nt = (n + ST - 1) / ST;
  const int tiles = nt * (nt + 1) / 2;
  for (int k0 = 0; k0 < n; k0 += SB) {
    const int bk = n - k0 < SB ? n - k0 : SB;
    sweep_pivot_kernel<<<L, 256, 0, s>>>(w, n, k0, bk, sbuf, d_info);
    if (n <= bk) break;  // a single block: nothing outside it
    sweep_panel_kernel<<<dim3((n + SP - 1) / SP, L), 256, 0, s>>>(w, n, k0, bk, sbuf, pbuf, cbuf);
    sweep_update_kernel<<<dim3(tiles, L), 256, 0, s>>>(w, n, k0, bk, pbuf, cbuf);
  }
}

}  // namespace qsgw
