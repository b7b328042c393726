// eps^{-1} in FP64 for every frequency at once (step a8): the Hermitian positive definite eps of
// Eq. (dielectricfunction) is inverted by a block sweep whose pivot blocks are factored by
// Cholesky. The paper keeps this inversion in double precision even in its mixed-precision mode.
//
// Sweep on pivot block k (rows and columns [k0, k0 + bk), bk <= 32), on the current matrix A:
//   S     = A_kk^{-1}                    Cholesky A_kk = L L^H, X = L^{-1}, S = X^H X
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
// TFLOP/s, both measured). The update, 95 % of the flops, therefore runs on the tcgen05 tensor
// cores in exact integer arithmetic that reproduces FP64 accuracy:
//   every row of P and of C (32 complex values) is put on a power-of-two grid, x 2^e with
//   max |x 2^e| <= 127, and cut into 7 integer digits, x 2^e = sum_s d_s 2^(-8 s), |d_s| <= 128
//   (each an exact FP16 value), with a remainder below 2^-49 of the row maximum;
//   the product of level L = i + j (digits i of P, j of C, L <= 6) is a sum of 64 products of
//   integers below 2^14 per pair, at most 7 * 64 * 128^2 < 2^24 over the pairs of a level, so
//   each level accumulates exactly in its own FP32 TMEM accumulator whatever the rounding mode;
//   the levels are combined in FP64, sum_L acc_L 2^(-8 L), and scaled by 2^(-eP - eC).
// The dropped levels (i + j >= 7) and the digit remainders are below 2^-52 of |P|max |C|max per
// product, so the update carries FP64 accuracy (the error is relative to the sum of the terms'
// magnitudes, as for an FP64 product). 28 digit pairs x 4 K-steps = 112 MMAs (M = 128: 64 rows
// times (Re, Im); N = 64; K = 16) per 64 x 64 tile and frequency. The mixed-precision contexts use
// it; the plain FP64 contexts keep the DFMA update kernel. Only the lower triangle of A is read or
// written (element (I, J), I >= J, at J * n + I of each frequency's matrix).
#include <cuda_fp16.h>

#include "internal.cuh"
#include "tc_ptx.cuh"

namespace qsgw {

constexpr int SB = 32;  // pivot block width
constexpr int ST = 64;  // update tile (rows and columns)

__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
  return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ double2 conj2(double2 a) { return make_double2(a.x, -a.y); }

// (hi 2^32 + lo) 2^sh as the nearest double (ties to even), in integer arithmetic: the 128-bit
// value is exact, its leading 53 bits become the significand and the rest decides the rounding.
// |hi| < 2^42, |lo| < 2^49; the result's exponent must stay in the normal range (the caller
// bounds sh).
__device__ __forceinline__ double i128_to_double(long long hi, long long lo, int sh) {
  __int128 v = (__int128)hi * ((__int128)1 << 32) + lo;
  if (v == 0) return 0.0;
  const bool neg = v < 0;
  unsigned __int128 m = neg ? (unsigned __int128)(-v) : (unsigned __int128)v;
  const unsigned long long mh0 = (unsigned long long)(m >> 64);
  const int lz = mh0 ? __clzll((long long)mh0) : 64 + __clzll((long long)(unsigned long long)m);
  m <<= lz;  // leading bit at 127
  const unsigned long long mh = (unsigned long long)(m >> 64), ml = (unsigned long long)m;
  unsigned long long mant = mh >> 11;  // 53 bits
  const unsigned long long rem = mh & 0x7FFull;
  const bool up = rem > 0x400ull || (rem == 0x400ull && (ml != 0 || (mant & 1ull)));
  mant += up ? 1ull : 0ull;
  int ex = 127 - lz + sh;  // exponent of the leading bit
  if (mant >> 53) {
    mant >>= 1;
    ++ex;
  }
  const unsigned long long bits = ((unsigned long long)neg << 63) | ((unsigned long long)(ex + 1023) << 52) |
                                  (mant & 0xFFFFFFFFFFFFFull);
  return __longlong_as_double((long long)bits);
}

// One CTA per frequency: Cholesky of the pivot block A_kk = L L^H and X = L^{-1} (lower triangular,
// written whole to sbuf[l], column-major SB x SB, zeros above the diagonal). The panel kernel forms
// S = X^H X from it. info[l] keeps the first non-positive pivot (1-based global index); a failed
// pivot continues with 1 so the sweep runs to its end, and that frequency's result is unspecified.
// X is formed alongside the factorisation by forward elimination on [L | I]: once column j of L is
// final, row j of X is scaled by 1/L_jj and subtracted, times L_ij, from every row i > j. Each step
// is a rank-1 update over all threads, like the factorisation's own; FP64 issue is scarce on this
// GPU, so no thread runs a long serial chain.
__global__ void __launch_bounds__(256) sweep_pivot_kernel(double2* __restrict__ w, int n, int k0, int bk,
                                                          double2* __restrict__ sbuf, int* __restrict__ info) {
  const int l = blockIdx.x, t = threadIdx.x;
  double2* m = w + (size_t)l * n * n;
  __shared__ double2 a[SB][SB + 1];  // a[i][j] = A(k0 + i, k0 + j), lower triangle; becomes L
  __shared__ double2 x[SB][SB + 1];  // becomes X = L^{-1}; starts as the identity
  __shared__ double rdiag;           // 1 / L_jj of the current step
  __shared__ int fail;
  if (t == 0) fail = 0;
  for (int e = t; e < SB * SB; e += blockDim.x) {
    const int i = e % SB, j = e / SB;
    if (i < bk && j < bk && i >= j) a[i][j] = m[(size_t)(k0 + j) * n + k0 + i];
    x[i][j] = make_double2(i == j ? 1.0 : 0.0, 0.0);
  }
  __syncthreads();
  for (int j = 0; j < bk; ++j) {
    if (t == 0) {  // one thread: an FP64 square root and division cost dozens of FP64 operations
      double d = a[j][j].x;
      if (!(d > 0.0)) {
        if (fail == 0) fail = j + 1;
        d = 1.0;
      }
      const double r = sqrt(d);
      a[j][j] = make_double2(r, 0.0);
      rdiag = 1.0 / r;
    }
    __syncthreads();
    const double ri = rdiag;
    for (int i = j + 1 + t; i < bk; i += blockDim.x) {  // column j of L
      a[i][j].x *= ri;
      a[i][j].y *= ri;
    }
    for (int k = t; k <= j; k += blockDim.x) {  // row j of X is final
      x[j][k].x *= ri;
      x[j][k].y *= ri;
    }
    __syncthreads();
    const int mt = bk - j - 1;
    for (int e = t; e < mt * mt; e += blockDim.x) {  // trailing update of A
      const int i = j + 1 + e % mt, c = j + 1 + e / mt;
      if (i >= c) {
        const double2 p = cmul(a[i][j], conj2(a[c][j]));
        a[i][c].x -= p.x;
        a[i][c].y -= p.y;
      }
    }
    for (int e = t; e < mt * (j + 1); e += blockDim.x) {  // X rows below j: x_ik -= L_ij x_jk
      const int i = j + 1 + e % mt, k = e / mt;
      const double2 p = cmul(a[i][j], x[j][k]);
      x[i][k].x -= p.x;
      x[i][k].y -= p.y;
    }
    __syncthreads();
  }
  double2* xs = sbuf + (size_t)l * SB * SB;
  for (int e = t; e < SB * SB; e += blockDim.x) {
    const int i = e % SB, j = e / SB;
    xs[j * SB + i] = (i < bk && j < bk && i >= j) ? x[i][j] : make_double2(0.0, 0.0);
  }
  if (t == 0 && fail != 0 && info[l] == 0) info[l] = k0 + fail;
}

// Grid (row tiles of 32, frequency). C = column block k of A for rows outside the pivot block
// (A(i, k0 + c), read from the lower triangle, conjugated above the block) and P = C S with
// S = A_kk^{-1} = X^H X, formed as P = (C X^H) X: thread (row i, column c) computes Y_ic = sum_{d<=c}
// C_id conj(X_cd), then P_ic = sum_{d>=c} Y_id X_dc (c + 1 and bk - c terms: every thread does the
// same work). Both go to column-major n x SB buffers: P for the update and the write-back, C as a
// copy, because the update overwrites column and row k of A with P. The CTA over the pivot block's
// rows also writes A_kk <- -S (lower triangle).
constexpr int SP = 32;  // panel rows per CTA
static_assert(SP == SB, "one panel CTA covers exactly the pivot block's rows");
__global__ void __launch_bounds__(256) sweep_panel_kernel(double2* __restrict__ w, int n, int k0, int bk,
                                                          const double2* __restrict__ sbuf, double2* __restrict__ pbuf,
                                                          double2* __restrict__ cbuf) {
  const int l = blockIdx.y, i0 = blockIdx.x * SP, t = threadIdx.x;
  double2* m = w + (size_t)l * n * n;
  __shared__ double2 cs[SP][SB + 1];
  __shared__ double2 xs[SB][SB + 1];
  __shared__ double2 ys[SP][SB + 1];
  for (int e = t; e < SB * SB; e += blockDim.x) {
    const int i = e % SB, j = e / SB;
    xs[i][j] = sbuf[(size_t)l * SB * SB + j * SB + i];  // zeros outside the bk x bk lower triangle
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
  for (int c = t / SP; c < SB; c += 256 / SP) {  // Y = C X^H
    double yr = 0.0, yi = 0.0;
    for (int d = 0; d <= c; ++d) {  // C_rd conj(X_cd)
      const double2 u = cs[r][d], v = xs[c][d];
      yr = fma(u.x, v.x, fma(u.y, v.y, yr));
      yi = fma(u.y, v.x, fma(-u.x, v.y, yi));
    }
    ys[r][c] = make_double2(yr, yi);
  }
  __syncthreads();
  const int i = i0 + r;
  for (int c = t / SP; c < bk; c += 256 / SP) {  // P = Y X
    double pr = 0.0, pi = 0.0;
    for (int d = c; d < SB; ++d) {
      const double2 u = ys[r][d], v = xs[d][c];
      pr = fma(u.x, v.x, fma(-u.y, v.y, pr));
      pi = fma(u.x, v.y, fma(u.y, v.x, pi));
    }
    if (i < n) {
      pbuf[((size_t)l * SB + c) * n + i] = make_double2(pr, pi);
      cbuf[((size_t)l * SB + c) * n + i] = cs[r][c];
    }
  }
  if (i0 == k0) {  // A_kk <- -S, S = X^H X on the lower triangle
    for (int e = t; e < bk * bk; e += blockDim.x) {
      const int a = e % bk, b = e / bk;  // S(a, b), a >= b
      if (a < b) continue;
      double sr = 0.0, si = 0.0;
      for (int c = a; c < bk; ++c) {  // conj(X_ca) X_cb
        const double2 u = xs[c][a], v = xs[c][b];
        sr = fma(u.x, v.x, fma(u.y, v.y, sr));
        si = fma(u.x, v.y, fma(-u.y, v.x, si));
      }
      m[(size_t)(k0 + b) * n + k0 + a] = make_double2(-sr, a == b ? 0.0 : -si);
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

// ------------------------------------------------------------------ the update on the tensor cores
constexpr int DL = 7;                       // integer digits per value, and digit levels kept
constexpr int DIG_A = 128 * 2 * SB * 2;     // bytes of one level of a P row-tile image (M = 128, K' = 64): 16 KB
constexpr int DIG_B = ST * 2 * SB * 2;      // bytes of one level of a C column-tile image (N = 64): 8 KB
constexpr int IMG_A = DL * DIG_A;           // 112 KB
constexpr int IMG_B = DL * DIG_B;           // 56 KB
constexpr uint64_t kTcWaitNs = 1000000000ull;

size_t eps_inverse_digit_bytes(int n, int L) {
  const size_t ntr = (size_t)(n + ST - 1) / ST;
  return (size_t)L * ntr * (IMG_A + IMG_B) + 2 * sizeof(int) * (size_t)L * ntr * ST;
}

// Grid (64-row tiles, frequency, side): side 0 cuts the rows of P into the A-operand image of the
// tile ([level][k-group 8][row group 16][8 rows][8 K'] FP16: Re rows (Pr, Pi), Im rows (Pi, -Pr) along
// K' = 2 c + (0, 1)), side 1 the rows of C into the B-operand image ([level][k-group 8][row group 8]
// [8 rows][8 K']: (Cr, Ci)), each with the row's grid exponent (e with max |x 2^e| <= 127). Values of
// columns c >= bk, rows past n and the rows of the pivot block (zero in P and C) give zero digits.
__global__ void __launch_bounds__(256) sweep_digits_kernel(int n, int bk, const double2* __restrict__ pbuf,
                                                           const double2* __restrict__ cbuf,
                                                           uint8_t* __restrict__ imgA, uint8_t* __restrict__ imgB,
                                                           int* __restrict__ eP, int* __restrict__ eC) {
  const int tr = blockIdx.x, l = blockIdx.y, side = blockIdx.z, t = threadIdx.x;
  const int ntr = gridDim.x;
  const int r = t & (ST - 1), q = t >> 6;  // row of the tile, quarter of the columns (8 of 32)
  const int i = tr * ST + r;
  const double2* src = (side == 0 ? pbuf : cbuf) + (size_t)l * SB * n;
  __shared__ double red[4][ST];
  double2 v[8];
  double m = 0.0;
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    const int c = q * 8 + k;
    v[k] = (i < n && c < bk) ? src[(size_t)c * n + i] : make_double2(0.0, 0.0);
    m = fmax(m, fmax(fabs(v[k].x), fabs(v[k].y)));
  }
  red[q][r] = m;
  __syncthreads();
  m = fmax(fmax(red[0][r], red[1][r]), fmax(red[2][r], red[3][r]));
  int e = 0;
  if (m > 0.0 && isfinite(m)) {
    int E;
    frexp(m, &E);  // m = f 2^E, f in [0.5, 1): m 2^(7 - E) in [64, 128)
    e = 7 - E;
    if (ldexp(m, e) > 127.0) --e;
    e = max(-400, min(400, e));  // keeps 2^(-16 - eP - eC) and 2^(-48 - eP - eC) normal doubles
  }
  if (q == 0 && i < ntr * ST) (side == 0 ? eP : eC)[(size_t)l * ntr * ST + i] = e;
  // x 2^e on the grid of 2^-48, as an exact 56-bit integer (|x 2^e| <= 127; rint drops below 2^-49),
  // then 7 balanced base-256 digits from the bottom: d = the low byte as a signed value in
  // [-128, 127], T <- (T - d) / 256; the last (leading) digit is in [-128, 128].
  const double g = ldexp(1.0, e + 48);
  long long Tr[8], Ti[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    Tr[k] = __double2ll_rn(v[k].x * g);
    Ti[k] = __double2ll_rn(v[k].y * g);
  }
  uint8_t* img = side == 0 ? imgA + ((size_t)l * ntr + tr) * IMG_A : imgB + ((size_t)l * ntr + tr) * IMG_B;
  for (int lev = DL - 1; lev >= 0; --lev) {
    __half dr[8], di[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      long long a, b;
      if (lev > 0) {
        a = ((Tr[k] + 128) & 255) - 128;
        b = ((Ti[k] + 128) & 255) - 128;
        Tr[k] = (Tr[k] - a) >> 8;  // exact: T - a is a multiple of 256
        Ti[k] = (Ti[k] - b) >> 8;
      } else {
        a = Tr[k];
        b = Ti[k];
      }
      dr[k] = __int2half_rn((int)a);  // integers of magnitude <= 128: exact
      di[k] = __int2half_rn((int)b);
    }
    // this thread's 8 complex columns are k-groups 2q and 2q + 1 (4 columns, 8 K' values each)
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int kg = 2 * q + h;
      __half re[8], im[8];
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        re[2 * k] = dr[4 * h + k];
        re[2 * k + 1] = di[4 * h + k];
        im[2 * k] = di[4 * h + k];
        im[2 * k + 1] = __hneg(dr[4 * h + k]);
      }
      if (side == 0) {
        uint8_t* base = img + lev * DIG_A + kg * 2048;
        *reinterpret_cast<uint4*>(base + (r >> 3) * 128 + (r & 7) * 16) = *reinterpret_cast<const uint4*>(re);
        const int mi = ST + r;
        *reinterpret_cast<uint4*>(base + (mi >> 3) * 128 + (mi & 7) * 16) = *reinterpret_cast<const uint4*>(im);
      } else {
        uint8_t* base = img + lev * DIG_B + kg * 1024;
        *reinterpret_cast<uint4*>(base + (r >> 3) * 128 + (r & 7) * 16) = *reinterpret_cast<const uint4*>(re);
      }
    }
  }
}

// Persistent: one CTA per SM runs the (frequency, lower 64 x 64 tile) items item = blockIdx.x +
// k gridDim.x, one CTA per SM (168 KB of operand images, 448 TMEM columns). Warp 16, one thread:
// bulk copies of an item's two images, its 112 MMAs, and, as soon as those MMAs are done (the
// images are free), the copies of the next item, so they overlap this item's epilogue. Warps 0..15
// (epilogue): read TMEM (warp w: lane quarter w mod 4, i.e. lane m = row m mod 64 of the tile, Re
// part for m < 64 and Im part above; columns 16 (w / 4) .. + 16), combine the 7 levels and update
// their half of each element (the element rules of sweep_update_kernel), then free TMEM for the
// next item's MMAs. Every wait is bounded (1 s); one that gives up sets DEV_TIMEOUT and the CTA
// stops at the next item (tiles not reached are left unchanged).
constexpr int TC_EPI = 512;               // epilogue threads
constexpr int TC_THREADS = TC_EPI + 32;   // + the copy / MMA warp
__device__ __forceinline__ void tc_item(int item, int tiles, int& l, int& ti, int& tj) {
  l = item / tiles;
  const int tile = item - l * tiles;
  ti = (int)((sqrt(8.0 * tile + 1.0) - 1.0) * 0.5);  // lower tile (ti, tj), ti >= tj
  while ((ti + 1) * (ti + 2) / 2 <= tile) ++ti;
  while (ti * (ti + 1) / 2 > tile) --ti;
  tj = tile - ti * (ti + 1) / 2;
}
__global__ void __launch_bounds__(TC_THREADS, 1) sweep_update_tc_kernel(double2* __restrict__ w, int n, int k0, int bk,
                                                                        int L, const double2* __restrict__ pbuf,
                                                                        const uint8_t* __restrict__ imgA,
                                                                        const uint8_t* __restrict__ imgB,
                                                                        const int* __restrict__ eP,
                                                                        const int* __restrict__ eC, int* d_err) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint8_t* sA = smem;
  uint8_t* sB = sA + IMG_A;
  // [0] images landed, [1] MMAs done (images free, accumulators ready), [2] TMEM read out (16 warps)
  uint64_t* bars = reinterpret_cast<uint64_t*>(sB + IMG_B);
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 3);
  int* sabort = reinterpret_cast<int*>(tmem_slot + 1);  // set by the copy / MMA thread when it gives up
  int* sdec = sabort + 1;  // [2] the epilogue warps' common stop decision, by item parity
  int* sE = sdec + 2;      // [64] grid exponents of the item's rows (P), [64] of its columns (C)
  const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
  const int ntr = (n + ST - 1) / ST;
  const int tiles = ntr * (ntr + 1) / 2, items = tiles * L;
  if (t == 0) {
    mbar_init(&bars[0], 1);
    mbar_init(&bars[1], 1);
    mbar_init(&bars[2], TC_EPI / 32);
    *sabort = 0;
    sdec[0] = sdec[1] = 0;
    fence_mbar_init();
  }
  if (warp == 0) {
    tmem_alloc(tmem_slot, 512);
    tmem_relinquish();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;
  if (warp == TC_EPI / 32) {
    // ---------------- copies and MMAs (one thread)
    if (lane == 0) {
      auto load = [&](int item) {
        int l, ti, tj;
        tc_item(item, tiles, l, ti, tj);
        mbar_arrive_expect_tx(&bars[0], IMG_A + IMG_B);
        bulk_g2s(sA, imgA + ((size_t)l * ntr + ti) * IMG_A, IMG_A, &bars[0]);
        bulk_g2s(sB, imgB + ((size_t)l * ntr + tj) * IMG_B, IMG_B, &bars[0]);
      };
      const uint32_t idesc = make_idesc_f16_f32(128, ST);
      const uint32_t a0 = smem_u32(sA), b0 = smem_u32(sB);
      int k = 0;
      bool inflight = false;  // copies issued and not yet waited for
      if ((int)blockIdx.x < items) {
        load(blockIdx.x);
        inflight = true;
      }
      for (int item = blockIdx.x; item < items; item += gridDim.x, ++k) {
        bool ok = mbar_wait_bounded(&bars[0], k & 1, kTcWaitNs);
        inflight = !ok;
        if (ok && k > 0) ok = mbar_wait_bounded(&bars[2], (k - 1) & 1, kTcWaitNs);  // TMEM read out
        if (!ok) {
          atomicCAS(d_err, DEV_OK, DEV_TIMEOUT);
          *sabort = 1;
          mbar_arrive(&bars[1]);  // (release: after the flag) lets the epilogue warps see it and leave
          break;
        }
        tc_fence_after();
        for (int lev = 0; lev < DL; ++lev) {
          uint32_t acc = 0;
          for (int i = 0; i <= lev; ++i) {
            const int j = lev - i;
#pragma unroll
            for (int ks = 0; ks < 4; ++ks) {
              const uint64_t ad = make_smem_desc(a0 + i * DIG_A + ks * 4096, 2048, 128, 0);
              const uint64_t bd = make_smem_desc(b0 + j * DIG_B + ks * 2048, 16 * ST, 128, 0);
              mma_f16(tmem + lev * ST, ad, bd, idesc, acc);
              acc = 1;
            }
          }
        }
        mma_commit(&bars[1]);
        if (item + (int)gridDim.x < items) {  // the images are free once the MMAs are done
          if (!mbar_wait_bounded(&bars[1], k & 1, kTcWaitNs)) {
            atomicCAS(d_err, DEV_OK, DEV_TIMEOUT);
            *sabort = 1;
            break;
          }
          load(item + gridDim.x);
          inflight = true;
        }
      }
      if (inflight) mbar_wait_bounded(&bars[0], k & 1, kTcWaitNs);  // no copy left landing at exit
    }
  } else {
    // ---------------- epilogue warps
    const int quarter = warp & 3, cg = warp >> 2;
    const int lm = quarter * 32 + lane;  // TMEM lane: row of the tile, Re (< 64) or Im part
    const int row = lm & (ST - 1), part = lm >> 6;
    const uint32_t tl = tmem + ((uint32_t)(quarter * 32) << 16);
    int k = 0;
    for (int item = blockIdx.x; item < items; item += gridDim.x, ++k) {
      int l, ti, tj;
      tc_item(item, tiles, l, ti, tj);
      if (t < 2 * ST)
        sE[t] = t < ST ? eP[(size_t)l * ntr * ST + ti * ST + t] : eC[(size_t)l * ntr * ST + tj * ST + t - ST];
      const bool done = mbar_wait_bounded(&bars[1], k & 1, kTcWaitNs);
      if (!done && lane == 0) {
        atomicCAS(d_err, DEV_OK, DEV_TIMEOUT);
        sdec[k & 1] = 1;
      }
      if (t == 0 && *((volatile int*)sabort)) sdec[k & 1] = 1;
      tc_fence_after();
      named_bar_sync(1, TC_EPI);  // sE written; this item's decision final (every warp reads the same)
      if (sdec[k & 1]) break;
      if (t == 0) sdec[(k + 1) & 1] = 0;  // written again only after this item's closing barrier
      double2* m = w + (size_t)l * n * n;
      const double2* P = pbuf + (size_t)l * SB * n;
      const int I = ti * ST + row;
      const int e_i = sE[row];
      constexpr int CW = 4;  // columns per TMEM read round
      for (int c0 = cg * 16; c0 < cg * 16 + 16; c0 += CW) {
        uint32_t r[DL][CW];
#pragma unroll
        for (int lev = 0; lev < DL; ++lev) tmem_ld_x4(tl + lev * ST + c0, r[lev]);
        tmem_ld_wait();
        double val[CW], old[CW];
        bool upd[CW];
#pragma unroll
        for (int jj = 0; jj < CW; ++jj) {
          const int J = tj * ST + c0 + jj;
          const bool inI = (unsigned)(I - k0) < (unsigned)bk, inJ = (unsigned)(J - k0) < (unsigned)bk;
          upd[jj] = I < n && J < n && I >= J && !inI && !inJ;
          // the level sums are exact integers below 2^23: combine them exactly, hi = a0 2^16 + a1 2^8
          // + a2 and lo = a3 2^24 + a4 2^16 + a5 2^8 + a6, value = (hi 2^32 + lo) 2^(-48 - eP - eC),
          // rounded once to double in integer arithmetic (the FP64 pipe only does the subtraction)
          long long a[DL];
#pragma unroll
          for (int lev = 0; lev < DL; ++lev) a[lev] = __float2int_rn(__uint_as_float(r[lev][jj]));
          const long long hi = a[0] * 65536LL + a[1] * 256LL + a[2];
          const long long lo = a[3] * 16777216LL + a[4] * 65536LL + a[5] * 256LL + a[6];
          const int ee = e_i + sE[ST + c0 + jj];  // |ee| <= 800: the result stays a normal double
          val[jj] = i128_to_double(hi, lo, -48 - ee);
        }
        if (c0 + CW >= cg * 16 + 16) {  // the last TMEM read of this item: free it for the next MMAs
          tc_fence_before();
          __syncwarp();
          if (lane == 0) mbar_arrive(&bars[2]);
        }
#pragma unroll
        for (int jj = 0; jj < CW; ++jj)  // the loads first, all independent
          old[jj] = upd[jj] ? reinterpret_cast<const double*>(m + (size_t)(tj * ST + c0 + jj) * n + I)[part] : 0.0;
#pragma unroll
        for (int jj = 0; jj < CW; ++jj)
          if (upd[jj]) reinterpret_cast<double*>(m + (size_t)(tj * ST + c0 + jj) * n + I)[part] = old[jj] - val[jj];
        if (part == 0) {  // the pivot block's column and row take P (the Re thread writes both parts)
#pragma unroll
          for (int jj = 0; jj < CW; ++jj) {
            const int J = tj * ST + c0 + jj;
            if (I >= n || J >= n || I < J) continue;
            const bool inI = (unsigned)(I - k0) < (unsigned)bk, inJ = (unsigned)(J - k0) < (unsigned)bk;
            if (inI == inJ) continue;
            m[(size_t)J * n + I] = inJ ? P[(size_t)(J - k0) * n + I] : conj2(P[(size_t)(I - k0) * n + J]);
          }
        }
      }
      named_bar_sync(1, TC_EPI);  // every warp is done with sE before the next item writes it
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    tmem_dealloc(tmem, 512);
  }
}

static size_t tc_update_smem() { return 1024 + IMG_A + IMG_B + 64 + 2 * ST * sizeof(int); }
static_assert(3 * 8 + 4 + 4 + 2 * 4 <= 64, "barriers, TMEM slot and the stop flags fit their 64 bytes");

void launch_eps_inverse(double2* w, int n, int L, double2* sbuf, double2* pbuf, double2* cbuf, uint8_t* dig,
                        int* d_info, int* d_err, cudaStream_t s) {
  const int nt = (n + ST - 1) / ST;
  const int tiles = nt * (nt + 1) / 2;
  int n_sm = 1;
  if (dig) {  // the attribute belongs to the current context: set it on every call
    cudaFuncSetAttribute(sweep_update_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tc_update_smem());
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev) !=
                                                  cudaSuccess)
      n_sm = 1;
  }
  uint8_t* imgA = dig;
  uint8_t* imgB = imgA + (size_t)L * nt * IMG_A;
  int* eP = reinterpret_cast<int*>(imgB + (size_t)L * nt * IMG_B);
  int* eC = eP + (size_t)L * nt * ST;
  for (int k0 = 0; k0 < n; k0 += SB) {
    const int bk = n - k0 < SB ? n - k0 : SB;
    sweep_pivot_kernel<<<L, 256, 0, s>>>(w, n, k0, bk, sbuf, d_info);
    sweep_panel_kernel<<<dim3((n + SP - 1) / SP, L), 256, 0, s>>>(w, n, k0, bk, sbuf, pbuf, cbuf);
    if (n <= bk) break;  // a single block: nothing outside it to update
    if (dig) {
      sweep_digits_kernel<<<dim3(nt, L, 2), 256, 0, s>>>(n, bk, pbuf, cbuf, imgA, imgB, eP, eC);
      sweep_update_tc_kernel<<<std::min(n_sm, tiles * L), TC_THREADS, tc_update_smem(), s>>>(w, n, k0, bk, L, pbuf,
                                                                                             imgA, imgB, eP, eC, d_err);
    } else {
      sweep_update_kernel<<<dim3(tiles, L), 256, 0, s>>>(w, n, k0, bk, pbuf, cbuf);
    }
  }
}

}  // namespace qsgw
