// Mixed-precision chi0 assembly on tcgen05 tensor cores (steps a1-a5). The same kernels compute the
// exchange self-energy of Eq. (sigx), a Hermitian update of the same form with given column weights.
//
//   chi0_IJ(l) = -s * sum_r |w_l(Delta_r)| conj(z_{I,r}) z_{J,r},  |w_l| = 2 Delta/(Delta^2 + omega_l^2)
//   (Sec. 2, Eq. (polfx) at w = i omega; the accumulator holds the positive-weight sum).
//
// Real form: with z = a + i b, stack Re and Im along the MMA M dimension. For 64 rows I of
// a tile the 128 A-rows are (a_I, b_I) for the real part and (-b_I, a_I) for the imaginary
// part, paired along K with B-columns (w a_J, w b_J):
//   Re = sum a_I (w a_J) + b_I (w b_J),   Im = sum a_I (w b_J) - b_I (w a_J).
// Every frequency is stacked along N: B-column n = l * TJ + j holds w_l(Delta_r) z_{J0+j, r},
// so one MMA of N = TJ * L <= 256 updates all frequencies from a single A tile in shared memory.
//
// Exact leading digit. tcgen05 accumulates FP32 with truncation (round toward zero, measured),
// so a plain float split would drift. Every operand value x of a chunk of 1024 columns is scaled
// by a power of two 2^e chosen from the chunk maximum (|x 2^e| <= 90) and split as
//   x 2^e = d0 + d1 + d2 + rem,  d0 = rint(x 2^e) in [-90, 90],  d1 = fp16(x 2^e - d0),
//   d2 = fp16(x 2^e - d0 - d1),  |rem| <= 2^-24,
// all three exact FP16 values (11 significant bits each; d0 is an integer). Products d0_A d0_B are
// integers and a chunk sum of them stays below 2 * 1024 * 90^2 < 2^24, so the level-0 TMEM
// accumulator is exact. The five products d0 d1, d1 d0, d0 d2, d2 d0, d1 d1 share a second
// accumulator whose truncation error is relative to its own, ~2^-6 smaller, magnitude. That error
// is the largest one left and grows faster than linearly with the chunk length (more truncating
// adds into a larger sum), which is what bounds CHR: 2048-column chunks measured 1.8e-6 relative
// on a narrow block, above the 1e-6 bar, against ~0.4e-6 at 1024. With |d1| <= 1/2 and |d2| <=
// 2^-12 the dropped products d1 d2, d2 d1 and d2 d2 are below 2^-13 each, ~2^-26 of the largest
// product 90^2, under the FP32 rounding of the inputs; so 6 MMA products serve a flop pair (BF16
// digits, 8 significant bits, left d1 d2 at ~2^-20 and needed 8). After each chunk the sum of
// both accumulators, rounded once to FP32, is stashed, and two drainer warps scale it by
// 2^-(eA+eB) (exact) and add it into a double-float (2 x FP32) accumulator in global memory while
// the next chunk's MMAs run; GB300's FP64 rate (~1.2 TFLOP/s) would make an FP64 read-modify-write
// here the bottleneck.
//
// Both operands' digits are formed once per call by the row preparation, as the exact
// shared-memory image of each K-block: the Re rows (a, b) of every row (the row image), and the
// B planes (all frequencies, scaled) per J tile. Every output tile of a J tile column reads the same
// B image, so forming B in each CTA repeated the same digit arithmetic once per I tile; the
// tensor-core kernel moves the images with bulk copies, forms the Im rows (-b, a) of A in shared
// memory and issues the MMAs. At one frequency (L = 1) the row image is the B operand as well.
#include <algorithm>
#include <cstring>
#include <vector>

#include <cuda_fp16.h>

#include "mixed.cuh"
#include "tc_ptx.cuh"

namespace qsgw {

constexpr int KBR = 16;                   // transition columns per K-block
constexpr int KBK = 2 * KBR;              // K' per K-block (re/im pairs)
constexpr int CHR = 1024;                 // columns per exact FP32 chunk
constexpr float DMAX = 90.f;              // |leading digit| bound: 2 * CHR * DMAX^2 < 2^24
constexpr int KB_PER_CH = CHR / KBR;      // 64
constexpr int TI = 64;                    // rows I per tile (M = 128)
constexpr int A_PLANE = 128 * KBK * 2;    // bytes of one digit plane of one A K-block (8 KB)
constexpr int A_HALF = A_PLANE / 2;       // its 64 Re rows (4 KB); the 64 Im rows follow
constexpr int A_STAGE = 3 * A_PLANE;      // 24 KB
constexpr int NS = 3;                     // pipeline stages: the A and B digit planes of one K-block each
constexpr size_t kSmemMax = 227 * 1024;
constexpr int NBG = 256;                  // epilogue threads (warps 2..9): chunk scales, TMEM -> stash
constexpr int NDR = 64;                   // drainer threads (warps 10, 11): deferred accumulator updates
constexpr int NTHREADS = 64 + NBG + NDR;
constexpr uint32_t TMEM_L12 = 256;        // column of the level-1+2 accumulator
constexpr uint64_t kWaitNs = 1000000000ull;

// Largest e with m * 2^e <= DMAX (m > 0), so that the leading digit fits in [-DMAX, DMAX].
__device__ __forceinline__ int scale_exp(float m) {
  if (!(m > 0.f) || !isfinite(m)) return 0;
  int E;
  const float f = frexpf(m, &E);  // m = f 2^E, f in [0.5, 1)
  int e = 7 - E;                  // m 2^e = 128 f in [64, 128)
  float s = 128.f * f;
  while (s > DMAX) {              // two halvings at most for DMAX >= 32
    s *= 0.5f;
    --e;
  }
  return max(-120, min(120, e));
}
__device__ __forceinline__ float exp2i(int e) {
  e = max(-126, min(127, e));
  return __int_as_float((e + 127) << 23);
}

// Digit arithmetic. The leading digit is rounded on the FP32 pipe by the add-subtract of 1.5 * 2^23;
// the FP16 digits come from the FP32 -> FP16 conversion (round to nearest even, FP16 subnormals
// included) and back. The _rn intrinsics are never contracted into FMAs, which the rounding relies on.
// (t + 1.5*2^23) - 1.5*2^23 is t rounded to the nearest integer (ties to even) for |t| < 2^22.
__device__ __forceinline__ float rint_add(float t) {
  return __fsub_rn(__fadd_rn(t, 12582912.0f), 12582912.0f);
}

// The FP16 value nearest to x, as an FP32 value.
__device__ __forceinline__ float h16(float x) { return __half2float(__float2half_rn(x)); }

// Three FP16-exact digits of t (|t| <= DMAX + 1/2): d0 = rint(t) (integer), then the remainder
// split twice into FP16 parts. t - d0 and u - d1 are exact in FP32 (d1 is within a factor of two
// of u, or u is below the FP16 normal range and u - d1 is a multiple of u's own last bit).
__device__ __forceinline__ void digits3(float t, float& d0, float& d1, float& d2) {
  d0 = rint_add(t);
  const float u = __fsub_rn(t, d0);
  d1 = h16(u);
  d2 = h16(__fsub_rn(u, d1));
}

// Three FP16-exact digits of the exact product a * b (|a b| <= DMAX + 1/2), with the product fused
// into the rounding: fma(a, b, 1.5 * 2^23) rounds a b to the nearest integer in one step, and
// u = fma(a, b, -d0) is a b - d0 rounded once (|u| <= 1/2), so d0 + d1 + d2 follows the exact
// product rather than fl(a b).
__device__ __forceinline__ void digits3_mul(float a, float b, float& d0, float& d1, float& d2) {
  d0 = __fsub_rn(__fmaf_rn(a, b, 12582912.0f), 12582912.0f);
  const float u = __fmaf_rn(a, b, -d0);
  d1 = h16(u);
  d2 = h16(__fsub_rn(u, d1));
}

// Two FP16-exact FP32 values -> packed f16x2 (lo in the low half); the conversion is exact.
__device__ __forceinline__ uint32_t pack_h2(float lo, float hi) {
  const __half2 h = __floats2half2_rn(lo, hi);
  return *reinterpret_cast<const uint32_t*>(&h);
}

// ------------------------------------------------------------------ prep: columns
constexpr int kMaxBlocks = 32;  // blocks per launch (descriptors travel by value as kernel parameters)

// Column preparation of one block of a batch: the weights are computed from the levels (eo, eu:
// Delta, domain check, |w_l| for every frequency) or given (wv: w_r = wv[r mod n_unocc], one set;
// Eq. (sigx) column r = n' * n_pb + mu carries the Coulomb eigenvalue v_mu(k)).
struct PrepColsBlk {
  const double* eo;
  const double* eu;
  const double* wv;  // non-null: given weights
  float* wst;        // [r][l] FP32 weights
  float* wmax;       // [chunk][l] their chunk maxima (the B-operand scale bound)
  long long K;       // columns of this launch
  long long r0;      // block column of this launch's first column (the (n, m) index of column r0 + r)
  int n_unocc, n_ch;
};
struct PrepColsArgs {
  PrepColsBlk b[kMaxBlocks];
  OmegaGrid g;
  int* d_err;
};

// One CTA per (chunk of CHR columns, block); CTAs past a block's chunk count leave at once.
constexpr int PC_THREADS = 1024;  // prep_cols threads per chunk; each handles CHR / PC_THREADS columns
__global__ void __launch_bounds__(PC_THREADS) prep_cols_kernel(const __grid_constant__ PrepColsArgs p) {
  __shared__ float red[PC_THREADS / 32][kMaxOmega];
  const PrepColsBlk& B = p.b[blockIdx.y];
  const int c = blockIdx.x, t = threadIdx.x;
  if (c >= B.n_ch) return;
  const long long K = B.K;
  if (B.wv) {  // given weights, checked > 0 and finite
    float wm = 0.f;
    for (int sub = 0; sub < CHR / PC_THREADS; ++sub) {
      const long long r = (long long)c * CHR + sub * PC_THREADS + t;
      float w = 0.f;
      if (r < K) {
        const double x = B.wv[(B.r0 + r) % B.n_unocc];
        const bool ok = (x > 0.0) && isfinite(x);
        if (!ok) atomicCAS(p.d_err, DEV_OK, DEV_DOMAIN);
        w = ok ? (float)x : 0.f;
      }
      B.wst[r] = w;
      wm = fmaxf(wm, w);
    }
    for (int o = 16; o > 0; o >>= 1) wm = fmaxf(wm, __shfl_xor_sync(0xffffffffu, wm, o));
    if ((t & 31) == 0) red[t >> 5][0] = wm;
    __syncthreads();
    if (t == 0) {
      float m = 0.f;
      for (int w = 0; w < PC_THREADS / 32; ++w) m = fmaxf(m, red[w][0]);
      B.wmax[c] = m;
    }
    return;
  }
  const int L = p.g.L;
  float wm[kMaxOmega];  // loops over l run to the constant kMaxOmega so wm stays in registers
#pragma unroll
  for (int l = 0; l < kMaxOmega; ++l) wm[l] = 0.f;
  for (int sub = 0; sub < CHR / PC_THREADS; ++sub) {
    const long long r = (long long)c * CHR + sub * PC_THREADS + t;
    bool ok = false;
    float d = 0.f;
    if (r < K) {
      const int n = (int)((B.r0 + r) / B.n_unocc), m = (int)((B.r0 + r) % B.n_unocc);
      const double dd = B.eu[m] - B.eo[n];
      ok = (dd > 0.0) && isfinite(dd);
      if (!ok) atomicCAS(p.d_err, DEV_OK, DEV_DOMAIN);
      d = (float)dd;
    }
#pragma unroll
    for (int l = 0; l < kMaxOmega; ++l) {
      if (l >= L) break;
      const float w = ok ? 2.f * d / (d * d + p.g.w2f[l]) : 0.f;
      B.wst[r * L + l] = w;
      wm[l] = fmaxf(wm[l], w);
    }
  }
#pragma unroll
  for (int l = 0; l < kMaxOmega; ++l) {
    if (l >= L) break;
    float w = wm[l];
    for (int o = 16; o > 0; o >>= 1) w = fmaxf(w, __shfl_xor_sync(0xffffffffu, w, o));
    if ((t & 31) == 0) red[t >> 5][l] = w;
  }
  __syncthreads();
  if (t < L) {
    float m = 0.f;
    for (int w = 0; w < PC_THREADS / 32; ++w) m = fmaxf(m, red[w][t]);
    B.wmax[c * L + t] = m;
  }
}

// ------------------------------------------------------------------ prep: rows
// Shared-memory operand layout (both operands, canonical no-swizzle K-major): 8-row core matrices of
// 16-byte rows (8 K' values), the 4 core matrices of a row group along K' 128 bytes apart, row
// groups 512 bytes apart; one digit plane of R rows of a K-block is R * 64 bytes:
//   byte (row >> 3) * 512 + kgroup * 128 + (row & 7) * 16.
// Row image (A operand, and at L = 1 also the B operand): for every K-block and digit plane, the
// (a, b) digit pairs of all prep rows in that layout, [K-block][plane][n_rows * 64 bytes], so the 64
// rows of an I tile (or the TJ rows of a J tile) are one contiguous slice. The tensor-core kernel
// copies an I tile's slice into the 64 Re rows of its A stage and forms the 64 Im rows (-b, a) from
// them in shared memory, so the imaginary rows never travel through HBM.
// B image of J tile jt (L >= 2): [K-block][plane][n = l * TJ + j in the same layout], values
// 2^eB w_l(Delta_r) z_{J, r} (re, im pairs along K'), eB from max_r |w_l| * max_r |z_J| of the chunk.
// Every CTA of a J tile column, and every I tile, reads the same B image, so the scaled digits of a
// column are formed once per call rather than once per output tile.
// At L = 1 the weights are positive and the product conj(z_I) w z_J is the product of the rows
// y = sqrt(w) z of both sides, so one row image with per-row exponents serves both operands: its
// digits are those of the exact product (FP32 sqrt(w)) (FP32 z) scaled by 2^e_I, e_I from the chunk
// maximum of |y_I|, and the epilogue takes 2^-(e_I + e_J) off each element.
// Rows past n_pb get zero digits. TZ: double2 (complex128 input) or float2 (complex64): every
// element is rounded to FP32 on load. All blocks of one launch have the same TZ.
struct PrepRowsBlk {
  const void* Z;  // TZ [r][ldz], at the launch's first column
  long long ldz, K;
  uint8_t* rimg;      // row image [n_kb][3][n_rows * 64]
  uint8_t* bplanes;   // B image [n_jt][n_kb][3][N * 64] (L >= 2)
  const float* wst;   // [r][L] weights (prep_cols)
  const float* wmax;  // [chunk][L] their chunk maxima
  float* zmax;
  int* expA;
  int n_pb, n_pad, n_kb, n_jt, n_ch, n_it, n_itb;
  int a_rows;  // rows I < a_rows are A rows (all rows, or the first row set of a restricted block)
  int b_row0;  // rows I >= b_row0 are B rows (0, or the restricted block's col0)
};
struct PrepRowsArgs {
  PrepRowsBlk b[kMaxBlocks];
  int TJ, L, N;
};

// The row value that enters the digits: z itself, or sqrt(w_r) z at L = 1.
__device__ __forceinline__ float row_weight(const float* wst, long long r, int L) {
  return L == 1 ? sqrtf(wst[r]) : 1.f;
}

// Row maxima of every chunk, zmax[c][I] = max over the chunk's columns of max(|Re y|, |Im y|) (y the
// row value above, each |.| the FP32 product), and their exponents; grid (chunk, row tile < n_it,
// block).
template <typename TZ>
__global__ void __launch_bounds__(256) prep_max_kernel(const __grid_constant__ PrepRowsArgs p) {
  __shared__ float red[4][TI];
  const PrepRowsBlk& B = p.b[blockIdx.z];
  const int c = blockIdx.x, it = blockIdx.y;
  if (c >= B.n_ch || it >= B.n_it) return;
  const TZ* __restrict__ Z = static_cast<const TZ*>(B.Z);
  const long long ldz = B.ldz, K = B.K;
  const int il = threadIdx.x & (TI - 1), q = threadIdx.x >> 6;
  const int I = it * TI + il;
  const bool rowok = I < B.n_pb;
  float m = 0.f;
  constexpr int U = 8;  // loads in flight per thread
  for (int jc0 = q; jc0 < CHR; jc0 += 4 * U) {
    TZ z[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const long long r = (long long)c * CHR + jc0 + 4 * u;
      z[u] = TZ{};
      if (rowok && r < K) z[u] = Z[I + r * ldz];
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const long long r = (long long)c * CHR + jc0 + 4 * u;
      const float s = row_weight(B.wst, r, p.L);  // columns past K: z = 0
      m = fmaxf(m, s * fmaxf(fabsf((float)z[u].x), fabsf((float)z[u].y)));
    }
  }
  red[q][il] = m;
  __syncthreads();
  if (q == 0) {
    m = fmaxf(fmaxf(red[0][il], red[1][il]), fmaxf(red[2][il], red[3][il]));
    B.zmax[(size_t)c * B.n_pad + I] = m;
    B.expA[(size_t)c * B.n_pad + I] = scale_exp(m);
  }
}

// The digit planes: PR_SPLIT CTAs per (chunk, 64-row tile), each over KB_PER_CH / PR_SPLIT K-blocks,
// so the grid fills the SMs in several waves; the row maxima come from prep_max_kernel. Thread
// (row il, k-group q) forms the digits of 4 columns of its row per K-block.
constexpr int PR_SPLIT = 8;
template <typename TZ>
__global__ void __launch_bounds__(256, 3) prep_rows_kernel(const __grid_constant__ PrepRowsArgs p) {
  const PrepRowsBlk& B = p.b[blockIdx.z];
  const int c = blockIdx.x / PR_SPLIT, part = blockIdx.x % PR_SPLIT, it = blockIdx.y;
  if (c >= B.n_ch || it >= B.n_itb) return;
  const TZ* __restrict__ Z = static_cast<const TZ*>(B.Z);
  const long long ldz = B.ldz, K = B.K;
  const int n_pb = B.n_pb, n_pad = B.n_pad, n_kb = B.n_kb, n_jt = B.n_jt, TJ = p.TJ, L = p.L, N = p.N;
  const size_t RPLANE = (size_t)B.n_itb * TI * 64;  // bytes of one plane of the row image per K-block
  const int BPLANE = 64 * N, BSTAGE = 3 * BPLANE;
  const int il = threadIdx.x & (TI - 1), q = threadIdx.x >> 6;
  const int I = it * TI + il;
  const bool rowok = I < n_pb;
  const int jt = I / TJ, jj = I % TJ;
  const bool sym = L == 1;
  // CTA-uniform: b_row0 is a multiple of the tile rows, and tiles past n_it carry B rows only
  const bool need_a = it < B.n_it && it * TI < B.a_rows;
  if (!need_a && !(it * TI + TI > B.b_row0 && it * TI < n_jt * TJ)) return;
  const bool need_b = jt < n_jt && I >= B.b_row0;
  const bool need_row = need_a || (sym && need_b);  // this row's slice of the row image is read
  const float m = rowok ? B.zmax[(size_t)c * n_pad + I] : 0.f;  // rows past n_pb: zero
  const float sA = exp2i(scale_exp(m));
  float bsc[kMaxOmega];  // 2^eB of this column for every frequency (the kernel's epilogue uses 2^-eB)
#pragma unroll
  for (int l = 0; l < kMaxOmega; ++l)
    bsc[l] = l < L ? exp2i(scale_exp(B.wmax[(size_t)c * L + l] * m)) : 0.f;
  const int rofs = (I >> 3) * 512 + q * 128 + (I & 7) * 16;  // this thread's 16 bytes in a row-image plane
  const int kb_begin = c * KB_PER_CH + part * (KB_PER_CH / PR_SPLIT);
  float na[4], nb[4];  // the next K-block's values, loaded one step ahead
#pragma unroll
  for (int rr = 0; rr < 4; ++rr) {
    const long long r = (long long)kb_begin * KBR + q * 4 + rr;
    TZ z{};
    if (rowok && r < K) z = Z[I + r * ldz];
    na[rr] = (float)z.x;
    nb[rr] = (float)z.y;
  }
  for (int kbi = 0; kbi < KB_PER_CH / PR_SPLIT; ++kbi) {
    const int kb = kb_begin + kbi;
    float a[4], b[4];
#pragma unroll
    for (int rr = 0; rr < 4; ++rr) {
      a[rr] = na[rr];
      b[rr] = nb[rr];
    }
    if (kbi + 1 < KB_PER_CH / PR_SPLIT) {
#pragma unroll
      for (int rr = 0; rr < 4; ++rr) {
        const long long r = (long long)(kb + 1) * KBR + q * 4 + rr;
        TZ z{};
        if (rowok && r < K) z = Z[I + r * ldz];
        na[rr] = (float)z.x;
        nb[rr] = (float)z.y;
      }
    }
    if (need_row) {
      float da[3][4], db[3][4];
      if (sym) {  // digits of the exact products (sqrt(w_r) 2^e) a and (sqrt(w_r) 2^e) b
        const float* wr = B.wst + (size_t)kb * KBR + q * 4;
#pragma unroll
        for (int rr = 0; rr < 4; ++rr) {
          const float ws = sqrtf(wr[rr]) * sA;
          digits3_mul(ws, a[rr], da[0][rr], da[1][rr], da[2][rr]);
          digits3_mul(ws, b[rr], db[0][rr], db[1][rr], db[2][rr]);
        }
      } else {
#pragma unroll
        for (int rr = 0; rr < 4; ++rr) {
          digits3(a[rr] * sA, da[0][rr], da[1][rr], da[2][rr]);
          digits3(b[rr] * sA, db[0][rr], db[1][rr], db[2][rr]);
        }
      }
      uint8_t* base = B.rimg + (size_t)kb * 3 * RPLANE + rofs;
#pragma unroll
      for (int pl = 0; pl < 3; ++pl) {
        uint4 re;  // (a, b) pairs along K'
        re.x = pack_h2(da[pl][0], db[pl][0]);
        re.y = pack_h2(da[pl][1], db[pl][1]);
        re.z = pack_h2(da[pl][2], db[pl][2]);
        re.w = pack_h2(da[pl][3], db[pl][3]);
        *reinterpret_cast<uint4*>(base + pl * RPLANE) = re;
      }
    }
    if (need_b && !sym) {
      const float* wr = B.wst + ((size_t)kb * KBR + q * 4) * L;  // this thread's 4 columns, every frequency
      uint8_t* bb = B.bplanes + ((size_t)jt * n_kb + kb) * BSTAGE + q * 128;
#pragma unroll
      for (int l = 0; l < kMaxOmega; ++l) {  // to the constant bound, so bsc stays in registers
        if (l >= L) break;
        float d[3][8];
#pragma unroll
        for (int rr = 0; rr < 4; ++rr) {
          const float ww = wr[rr * L + l] * bsc[l];
          digits3_mul(ww, a[rr], d[0][2 * rr], d[1][2 * rr], d[2][2 * rr]);
          digits3_mul(ww, b[rr], d[0][2 * rr + 1], d[1][2 * rr + 1], d[2][2 * rr + 1]);
        }
        const int n = l * TJ + jj;
        uint8_t* dst = bb + (n >> 3) * 512 + (n & 7) * 16;
#pragma unroll
        for (int pl = 0; pl < 3; ++pl) {
          uint4 v;
          v.x = pack_h2(d[pl][0], d[pl][1]);
          v.y = pack_h2(d[pl][2], d[pl][3]);
          v.z = pack_h2(d[pl][4], d[pl][5]);
          v.w = pack_h2(d[pl][6], d[pl][7]);
          *reinterpret_cast<uint4*>(dst + pl * BPLANE) = v;
        }
      }
    }
  }
}

// L = 1 in one pass: the row maxima and the row image of one chunk of PS_ROWS rows (one 8-row
// group), with the chunk's FP32 values staged in shared memory, so Z is read from HBM once instead
// of once for the maxima and once for the digits. Grid (chunk, row group, block); 256 threads.
//   load:   thread (row t mod 8, column t / 8 + 32 k) reads z, keeps the running max of
//           sqrt(w_r) max(|Re z|, |Im z|) (each the FP32 product, as prep_max_kernel);
//   digits: thread (row t mod 8, k-group (t / 8) mod 4, K-block t / 32 + 8 k) as prep_rows_kernel.
constexpr int PS_ROWS = 8;
constexpr int PS_LD = PS_ROWS + 1;  // staged column stride in float2: keeps the digit reads conflict-free
constexpr size_t kPrepSymSmem = (size_t)CHR * PS_LD * sizeof(float2) + CHR * sizeof(float) + 8 * PS_ROWS * 4;
template <typename TZ>
__global__ void __launch_bounds__(256, 2) prep_sym_kernel(const __grid_constant__ PrepRowsArgs p) {
  extern __shared__ float4 sym_smem[];
  float2* sz = reinterpret_cast<float2*>(sym_smem);   // [CHR][PS_LD]
  float* ssw = reinterpret_cast<float*>(sz + CHR * PS_LD);  // [CHR] sqrt(w_r)
  float* red = ssw + CHR;                             // [8 warps][PS_ROWS]
  const PrepRowsBlk& B = p.b[blockIdx.z];
  const int c = blockIdx.x, g = blockIdx.y, t = threadIdx.x;
  if (c >= B.n_ch || g * PS_ROWS >= B.n_itb * TI) return;
  const int TJ = p.TJ;
  const int I0 = g * PS_ROWS, it = I0 / TI, jt = I0 / TJ;
  // CTA-uniform: tiles are 64 rows, J tiles a multiple of 16 rows, b_row0 a multiple of both
  const bool need_a = it < B.n_it && it * TI < B.a_rows;
  const bool need_b = jt < B.n_jt && I0 >= B.b_row0;
  if (!need_a && !need_b) return;
  const TZ* __restrict__ Z = static_cast<const TZ*>(B.Z);
  const long long ldz = B.ldz, K = B.K;
  const int row = t & (PS_ROWS - 1), I = I0 + row;
  const bool rowok = I < B.n_pb;
  for (int j = t; j < CHR; j += 256) ssw[j] = sqrtf(B.wst[(size_t)c * CHR + j]);  // 0 past K
  __syncthreads();
  float m = 0.f;
  constexpr int U = 16;  // loads in flight per thread
  for (int j0 = t / PS_ROWS; j0 < CHR; j0 += U * (256 / PS_ROWS)) {
    TZ z[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int j = j0 + u * (256 / PS_ROWS);
      const long long r = (long long)c * CHR + j;
      z[u] = TZ{};
      if (rowok && r < K) z[u] = Z[I + r * ldz];
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int j = j0 + u * (256 / PS_ROWS);
      const float a = (float)z[u].x, b = (float)z[u].y;
      sz[j * PS_LD + row] = make_float2(a, b);
      m = fmaxf(m, ssw[j] * fmaxf(fabsf(a), fabsf(b)));
    }
  }
  // max over the 32 threads of this row in the warp (lanes row, row + 8, row + 16, row + 24), then
  // over the 8 warps
  m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, 8));
  m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, 16));
  if ((t & 31) < PS_ROWS) red[(t >> 5) * PS_ROWS + row] = m;
  __syncthreads();
  m = 0.f;
#pragma unroll
  for (int w = 0; w < 8; ++w) m = fmaxf(m, red[w * PS_ROWS + row]);
  const int eA = scale_exp(m);
  if (t < PS_ROWS && I < B.n_pad) {
    B.zmax[(size_t)c * B.n_pad + I] = m;
    B.expA[(size_t)c * B.n_pad + I] = eA;
  }
  const float sA = exp2i(eA);
  const size_t RPLANE = (size_t)B.n_itb * TI * 64;
  const int q = (t >> 3) & 3, kbs = t >> 5;
  uint8_t* const rbase = B.rimg + (size_t)(I >> 3) * 512 + q * 128 + (I & 7) * 16;
  for (int kbl = kbs; kbl < KB_PER_CH; kbl += 8) {
    const int kb = c * KB_PER_CH + kbl;
    float da[3][4], db[3][4];
#pragma unroll
    for (int rr = 0; rr < 4; ++rr) {
      const int j = kbl * KBR + q * 4 + rr;
      const float2 v = sz[j * PS_LD + row];
      const float ws = ssw[j] * sA;  // digits of the exact products (sqrt(w_r) 2^e) a and (sqrt(w_r) 2^e) b
      digits3_mul(ws, v.x, da[0][rr], da[1][rr], da[2][rr]);
      digits3_mul(ws, v.y, db[0][rr], db[1][rr], db[2][rr]);
    }
    uint8_t* base = rbase + (size_t)kb * 3 * RPLANE;
#pragma unroll
    for (int pl = 0; pl < 3; ++pl) {
      uint4 re;  // (a, b) pairs along K'
      re.x = pack_h2(da[pl][0], db[pl][0]);
      re.y = pack_h2(da[pl][1], db[pl][1]);
      re.z = pack_h2(da[pl][2], db[pl][2]);
      re.w = pack_h2(da[pl][3], db[pl][3]);
      *reinterpret_cast<uint4*>(base + pl * RPLANE) = re;
    }
  }
}

// ------------------------------------------------------------------ main tensor-core kernel
// One block of transition columns (one accumulate request) for one q-point, as the kernel sees it.
struct BlockDesc {
  const uint8_t* rimg;     // row image [n_kb][3][n_rows * 64]
  const uint8_t* bplanes;  // B image (L >= 2)
  const float* zmax;
  const int* expA;
  const float* wmax;
  const int2* tiles;
  float2* acc;    // [l][part][J][I] (hi, lo): whole tiles, each owned by one CTA
  double* acc2;   // [l][part][J][I] FP64: the reduced pieces of split tiles (piece_reduce_kernel)
  int tile_off;   // first global tile index of this block
  int n_pb, n_pad, n_kb, n_tiles, n_ch;
  int n_kbr;      // K-blocks holding columns (ceil(K / KBR)); the rest of the last chunk is padding
  int n_rows;     // rows of the row image (a multiple of 64)
};
constexpr int kFscrPerCta = 256 * 128;  // flush scratch pairs per CTA: [column n < 256][accumulator lane < 128]

// Work schedule. The T tiles of all blocks (block-major, then tile-major, so consecutive tiles share
// their row operand) are handed out whole through a global counter, so the CTAs run through them in
// near lockstep and the row-operand planes of a K-block are read from HBM once and served to the
// other CTAs of that row tile from L2. The last R tiles (R = T mod #CTAs, or all tiles if T is
// smaller) are cut into P chunk ranges each, so the final wave keeps every SM busy. Each piece sums
// into a private double-float partial buffer; piece_reduce_kernel then adds a tile's P partials, in
// piece order, to the FP64 accumulator (deterministic, no atomics).
struct MainArgs {
  BlockDesc blk[kMaxBlocks];
  int nb;
  int T, T_whole, P, n_items;
  int* counter;
  int L, TJ, N;
  uint32_t idesc;
  int* d_err;
  float2* fscr;  // per-CTA flush scratch, kFscrPerCta pairs each (see the chunk epilogue)
  float2* pbuf;  // per-piece partial sums of split tiles, kFscrPerCta pairs each (double-float)
};

struct WorkItem {
  int gt;      // global tile index, -1 = none
  int c0, c1;  // chunk range
  int flags;   // bit 0: last item of this CTA; bit 1: piece of a split tile
  int pid;     // piece index (its partial buffer), -1 for a whole tile
};
// Items in flight, producer -> MMA issuer and builders. The producer publishes item i before its
// wait on `empty` for that item's first K-block; at that point the consumers have released every
// K-block up to NS before it, and with it read every item whose first K-block lies there. Since an
// item has at least one K-block, the slot of item i - kRing is free once kRing >= NS + 1 (with
// one-K-block items, kRing = NS overwrote an item not yet read).
constexpr int kRing = 2 * NS;
static_assert(kRing >= NS + 1, "item ring shorter than the load pipeline");

__device__ __forceinline__ int block_of_tile(const BlockDesc* blk, int nb, int gt) {
  int b = 0;
  while (b + 1 < nb && blk[b + 1].tile_off <= gt) ++b;
  return b;
}

// K-blocks of an item: its chunks [c0, c1), the last chunk of the block cut at n_kbr. At least one,
// since (n_ch - 1) * CHR < K. Every item ends on a chunk end, so its last K-block closes a chunk.
__device__ __forceinline__ int item_nkb(const WorkItem& w, const BlockDesc& bd) {
  return min(w.c1 * KB_PER_CH, bd.n_kbr) - w.c0 * KB_PER_CH;
}

__device__ WorkItem decode_item(const MainArgs& p, const BlockDesc* blk, int i) {
  WorkItem w;
  w.gt = -1;
  w.c0 = w.c1 = 0;
  w.flags = 0;
  w.pid = -1;
  if (i >= p.n_items) return w;
  if (i < p.T_whole) {
    w.gt = i;
    const BlockDesc& bd = blk[block_of_tile(blk, p.nb, i)];
    w.c0 = 0;
    w.c1 = bd.n_ch;
    return w;
  }
  const int j = i - p.T_whole;
  w.gt = p.T_whole + j / p.P;
  const int piece = j % p.P;
  const BlockDesc& bd = blk[block_of_tile(blk, p.nb, w.gt)];
  w.c0 = piece * bd.n_ch / p.P;
  w.c1 = (piece + 1) * bd.n_ch / p.P;
  w.flags = 2;
  w.pid = j;
  return w;
}

__device__ __forceinline__ void df_add(float2& v, float x) {
  const float s = v.x + x;
  const float bb = s - v.x;
  const float e = (v.x - (s - bb)) + (x - bb);
  v.x = s;
  v.y += e;
}

// Bytes of the B digit planes of one K-block of one J tile (3 planes of N rows x 32 K' FP16).
__host__ __device__ constexpr size_t b_stage_bytes(int N) { return (size_t)3 * 64 * N; }

__host__ __device__ constexpr size_t main_smem_bytes(int N) {
  return 1024 + (size_t)NS * (A_STAGE + b_stage_bytes(N)) + 256 * 4 * 2 + 32 * 8 + 64 +
         sizeof(BlockDesc) * kMaxBlocks + sizeof(WorkItem) * kRing;
}

// 168 registers at most: the register file is split over the 4 SM sub-partitions and 12 warps
// put 3 on each of them (3 * 32 * 168 <= 16384); __launch_bounds__ lets ptxas enforce it.
__global__ void __launch_bounds__(NTHREADS, 1) herk_mixed_kernel(MainArgs p) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  const int N = p.N, TJ = p.TJ, L = p.L;
  const int BPLANE = 64 * N;  // bytes of one B digit plane of one K-block
  const int BSTAGE = 3 * BPLANE;
  const int STAGE = A_STAGE + BSTAGE;  // a multiple of 1024 (N is a multiple of 16)
  uint8_t* sStage = smem;              // [NS][A planes | B planes]
  float* sScB = reinterpret_cast<float*>(sStage + NS * STAGE);  // [2][256] 2^-eB per B column, by chunk parity
  uint64_t* bars = reinterpret_cast<uint64_t*>(sScB + 512);
  uint64_t* full = bars;             // [NS]   producer -> MMA and epilogue warps (bulk copies landed)
  uint64_t* empty = full + NS;       // [NS]   MMA commit + 8 epilogue warps -> producer
  uint64_t* accfull = empty + NS;    // MMA commit at chunk end -> epilogue
  uint64_t* accempty = accfull + 1;  // 8 epilogue warps -> MMA
  uint64_t* finbar = accempty + 1;
  uint64_t* stashed = finbar + 1;    // 8 epilogue warps -> drainers: a chunk end (stash or heartbeat)
  uint64_t* drained = stashed + 1;   // 2 drainer warps -> epilogue: that stash is in the accumulator
  uint64_t* built = drained + 1;     // [NS]   8 epilogue warps -> MMA: the stage's Im rows are formed
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(built + NS);
  int* abortB = reinterpret_cast<int*>(tmem_slot + 1);  // [2] epilogue-warp failure flags, by chunk parity
  int* sdesc = abortB + 2;  // [8] stash: kind (1 whole-tile chunk, 3 piece chunk, 2 end), block, it, jt, chunk,
                            //     parity, piece, first chunk of the piece
  BlockDesc* sBlk = reinterpret_cast<BlockDesc*>(bars + 32);  // block table, copied from the parameters
  WorkItem* ring = reinterpret_cast<WorkItem*>(sBlk + kMaxBlocks);  // items in flight, producer -> others

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  for (int i = tid; i < p.nb; i += NTHREADS) sBlk[i] = p.blk[i];
  int next_i = 0;  // producer thread only: the next item index it grabbed
  if (tid == 0) {
    for (int s = 0; s < NS; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1 + NBG / 32);
      mbar_init(&built[s], NBG / 32);
    }
    mbar_init(accfull, 1);
    mbar_init(accempty, NBG / 32);
    mbar_init(finbar, 1);
    mbar_init(stashed, NBG / 32);
    mbar_init(drained, NDR / 32);
    abortB[0] = abortB[1] = 0;
    fence_mbar_init();
  }
  if (warp == 1) {
    tmem_alloc(tmem_slot, 512);
    tmem_relinquish();
  }
  __syncthreads();  // block table in shared memory
  if (tid == 0) {   // first item (and whether it is the last) before the roles split
    WorkItem w = decode_item(p, sBlk, atomicAdd(p.counter, 1));
    next_i = atomicAdd(p.counter, 1);
    if (w.gt >= 0 && next_i >= p.n_items) w.flags |= 1;
    ring[0] = w;
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  if (warp == 0) {
    // ---------------- producer: grabs items; bulk copies of the A and B digit planes of each K-block
    if (lane == 0) {
      int issued = 0, g = 0, pos = 0;
      WorkItem cur = ring[0];
      bool stop = cur.gt < 0;
      while (!stop) {
        const BlockDesc& bd = sBlk[block_of_tile(sBlk, p.nb, cur.gt)];
        const int2 tile = bd.tiles[cur.gt - bd.tile_off];
        const int nkb = item_nkb(cur, bd);
        for (int kbi = 0; kbi < nkb; ++kbi, ++g) {
          const int s = g % NS, round = g / NS;
          const int kb = cur.c0 * KB_PER_CH + kbi;
          if (g >= NS && !mbar_wait_bounded(&empty[s], (round - 1) & 1, kWaitNs)) {
            atomicCAS(p.d_err, DEV_OK, DEV_TIMEOUT);
            stop = true;
            break;
          }
          uint8_t* st = sStage + s * STAGE;
          const size_t rplane = (size_t)bd.n_rows * 64;
          const uint8_t* rk = bd.rimg + (size_t)kb * 3 * rplane;
          mbar_arrive_expect_tx(&full[s], 3 * A_HALF + BSTAGE);
          for (int pl = 0; pl < 3; ++pl)  // the I tile's 64 Re rows of each plane
            bulk_g2s(st + pl * A_PLANE, rk + pl * rplane + (size_t)tile.x * TI * 64, A_HALF, &full[s]);
          if (L == 1) {  // the J tile's TJ rows of the same row image
            for (int pl = 0; pl < 3; ++pl)
              bulk_g2s(st + A_STAGE + pl * BPLANE, rk + pl * rplane + (size_t)tile.y * TJ * 64, BPLANE, &full[s]);
          } else {
            bulk_g2s(st + A_STAGE, bd.bplanes + ((size_t)tile.y * bd.n_kb + kb) * BSTAGE, BSTAGE, &full[s]);
          }
          issued = g + 1;
        }
        if (stop || (cur.flags & 1)) break;
        // publish the next item before the arrive of its first K-block (release orders the store)
        WorkItem nx = decode_item(p, sBlk, next_i);
        next_i = atomicAdd(p.counter, 1);
        if (next_i >= p.n_items) nx.flags |= 1;
        ++pos;
        ring[pos % kRing] = nx;
        cur = nx;
      }
      // never leave a bulk copy in flight into shared memory at exit
      for (int k = (issued > NS ? issued - NS : 0); k < issued; ++k)
        mbar_wait_bounded(&full[k % NS], (k / NS) & 1, kWaitNs);
    }
  } else if (warp == 1) {
    // ---------------- MMA issuer (one thread)
    if (lane == 0) {
      const uint32_t idesc = p.idesc;
      int g = 0, pos = 0, lc = 0;  // lc: chunks started by this CTA
      WorkItem cur = ring[0];
      bool stop = cur.gt < 0;
      while (!stop) {
        int nkb = item_nkb(cur, sBlk[block_of_tile(sBlk, p.nb, cur.gt)]);
        for (int kbi = 0; kbi < nkb; ++kbi, ++g) {
          const int s = g % NS, kbl = kbi % KB_PER_CH;
          bool ok = mbar_wait_bounded(&built[s], (g / NS) & 1, kWaitNs);
          if (ok && kbi == 0 && pos > 0) {  // the item was published before this K-block's copies
            cur = ring[pos % kRing];
            nkb = item_nkb(cur, sBlk[block_of_tile(sBlk, p.nb, cur.gt)]);
          }
          if (ok && kbl == 0 && lc > 0) ok = mbar_wait_bounded(accempty, (lc - 1) & 1, kWaitNs);
          if (!ok) {
            atomicCAS(p.d_err, DEV_OK, DEV_TIMEOUT);
            stop = true;
            break;
          }
          if (kbl == 0) ++lc;
          tc_fence_after();
          const uint32_t a_base = smem_u32(sStage + s * STAGE), b_base = a_base + A_STAGE;
#pragma unroll
          for (int ks = 0; ks < 2; ++ks) {  // k-groups 2 ks, 2 ks + 1: 128 bytes apart, row groups 512
            const uint32_t ao = a_base + ks * 256, bo = b_base + ks * 256;
            const uint64_t a0 = make_smem_desc(ao, 128, 512, 0);
            const uint64_t a1 = make_smem_desc(ao + A_PLANE, 128, 512, 0);
            const uint64_t a2 = make_smem_desc(ao + 2 * A_PLANE, 128, 512, 0);
            const uint64_t b0 = make_smem_desc(bo, 128, 512, 0);
            const uint64_t b1 = make_smem_desc(bo + BPLANE, 128, 512, 0);
            const uint64_t b2 = make_smem_desc(bo + 2 * BPLANE, 128, 512, 0);
            const uint32_t acc_in = (kbl == 0 && ks == 0) ? 0u : 1u;
            // grouped by A digit, so each A plane is read from shared memory once per K-step and
            // kept in the collector buffer for the products that follow
            mma_f16_a_fill(tmem, a0, b0, idesc, acc_in);
            mma_f16_a_use(tmem + TMEM_L12, a0, b1, idesc, acc_in);
            mma_f16_a_lastuse(tmem + TMEM_L12, a0, b2, idesc, 1u);
            mma_f16_a_fill(tmem + TMEM_L12, a1, b0, idesc, 1u);
            mma_f16_a_lastuse(tmem + TMEM_L12, a1, b1, idesc, 1u);
            mma_f16(tmem + TMEM_L12, a2, b0, idesc, 1u);
          }
          mma_commit(&empty[s]);
          if (kbl == KB_PER_CH - 1 || kbi == nkb - 1) mma_commit(accfull);  // an item ends a chunk
        }
        if (stop || (cur.flags & 1)) break;
        ++pos;
      }
      // drain: all issued MMAs complete before TMEM is released
      mma_commit(finbar);
      mbar_wait_bounded(finbar, 0, kWaitNs);
    }
  } else if (warp < 2 + NBG / 32) {
    // ---------------- epilogue warps: the Im rows of each A stage, the chunk's B scales for the
    // drainers, and the chunk epilogue. Per K-block they wait for the copies, form the 64 Im rows
    // (-b, a) of every plane from the 64 Re rows (a, b) (swap the FP16 halves of each pair, flip the
    // sign of the new low half), hand the stage to the MMA issuer and release it to the producer.
    const int bt = tid - 64;
    const int quarter = warp & 3;             // TMEM lane quarter this warp may access
    const int wg = (warp - 2) >> 2;           // column half handled in the epilogue
    const int m_row = quarter * 32 + lane;    // accumulator lane = A row
    const bool has_col = bt < N;              // B column n = bt (frequency bl, tile column bj)
    const int bl = bt / TJ, bj = bt % TJ;
    int it = 0, jt = 0, b = 0;
    // Deferred flush. At a chunk end of a whole tile the epilogue stores the two scaled
    // accumulator levels to this CTA's scratch (plain stores, no loads), frees TMEM and hands the
    // stash to the drainer warps, which do the double-float read-modify-write of the accumulator
    // while the next chunk runs. Every chunk end is announced (pieces as an empty stash), so a
    // drainer never waits longer than one chunk. A warp whose wait on the drainers times out
    // ("ddead") stops stashing and waiting; the error flag is set.
    float* const fscr = reinterpret_cast<float*>(p.fscr + (size_t)blockIdx.x * kFscrPerCta);
    int ns = 0;  // chunk ends announced
    bool ddead = false;
    // A warp whose wait timed out ("dead", warp-uniform) skips waits and work for the rest of its
    // chunk and sets abortB[chunk parity]; at that chunk's epilogue barrier every epilogue warp reads
    // the flag and all leave together, so no named barrier is ever left short of a warp. (Items end
    // on chunk boundaries, so no warp reads the item ring after a failure.)
    bool dead = false;
    int g = 0, pos = 0, lc = 0;
    WorkItem cur = ring[0];
    bool more = cur.gt >= 0;
    while (more) {
      int nkb = item_nkb(cur, sBlk[block_of_tile(sBlk, p.nb, cur.gt)]);
      for (int kbi = 0; kbi < nkb; ++kbi, ++g) {
        const int s = g % NS, kbl = kbi % KB_PER_CH;
        bool ok = !dead && mbar_wait_bounded(&full[s], (g / NS) & 1, kWaitNs);
        if (!dead && __any_sync(0xffffffffu, !ok)) {
          dead = true;
          if (lane == 0) {
            abortB[lc & 1] = 1;
            atomicCAS(p.d_err, DEV_OK, DEV_TIMEOUT);
          }
        }
        if (kbi == 0) {  // new item: published before this K-block's copies (or before the roles split)
          if (pos > 0) cur = ring[pos % kRing];
          b = block_of_tile(sBlk, p.nb, cur.gt);
          nkb = item_nkb(cur, sBlk[b]);
          const int2 tile = sBlk[b].tiles[cur.gt - sBlk[b].tile_off];
          it = tile.x;
          jt = tile.y;
        }
        if (!dead) {
          uint4* st4 = reinterpret_cast<uint4*>(sStage + s * STAGE);
#pragma unroll
          for (int pl = 0; pl < 3; ++pl) {
            uint4 v = st4[pl * (A_PLANE / 16) + bt];
            v.x = __byte_perm(v.x, 0, 0x1032) ^ 0x8000u;
            v.y = __byte_perm(v.y, 0, 0x1032) ^ 0x8000u;
            v.z = __byte_perm(v.z, 0, 0x1032) ^ 0x8000u;
            v.w = __byte_perm(v.w, 0, 0x1032) ^ 0x8000u;
            st4[pl * (A_PLANE / 16) + A_HALF / 16 + bt] = v;
          }
          fence_proxy_async_smem();  // visible to the tensor core's reads
          __syncwarp();
          if (lane == 0) mbar_arrive(&built[s]);
        }
        const BlockDesc& bd = sBlk[b];
        const int c = cur.c0 + kbi / KB_PER_CH;
        if (kbl == 0 && has_col) {  // 2^-eB of this chunk, the inverse of the scale the prep applied
          const int J = jt * TJ + bj;
          if (L == 1) {
            sScB[(lc & 1) * 256 + bt] = J < bd.n_pb ? exp2i(-bd.expA[(size_t)c * bd.n_pad + J]) : 0.f;
          } else {
            const float zm = J < bd.n_pb ? bd.zmax[(size_t)c * bd.n_pad + J] : 0.f;
            sScB[(lc & 1) * 256 + bt] = exp2i(-scale_exp(bd.wmax[c * L + bl] * zm));
          }
        }
        __syncwarp();
        if (lane == 0 && !dead) mbar_arrive(&empty[s]);
        if (kbl == KB_PER_CH - 1 || kbi == nkb - 1) {
          // ------------- chunk epilogue: TMEM -> registers -> scaled -> global accumulator
          ok = !dead && mbar_wait_bounded(accfull, lc & 1, kWaitNs);
          if (!dead && __any_sync(0xffffffffu, !ok)) {
            dead = true;
            if (lane == 0) {
              abortB[lc & 1] = 1;
              atomicCAS(p.d_err, DEV_OK, DEV_TIMEOUT);
            }
          }
          named_bar_sync(1, NBG);  // the chunk's exponent table (written at chunk start) is complete
          if (abortB[lc & 1]) {    // some builder warp failed in this chunk: all leave together
            more = false;
            break;
          }
          ++lc;
          if (ns > 0 && !ddead) {  // the drainers are done with the previous stash: scratch and descriptor free
            const bool okd = mbar_wait_bounded(drained, (ns - 1) & 1, kWaitNs);
            if (__any_sync(0xffffffffu, !okd)) {
              ddead = true;
              if (lane == 0) atomicCAS(p.d_err, DEV_OK, DEV_TIMEOUT);
            }
          }
          tc_fence_after();
          const bool piece = (cur.flags & 2) != 0;
          const int half = N / 2;  // a multiple of 8
          const uint32_t tl = tmem + ((uint32_t)(quarter * 32) << 16);
          const int col_end = (wg + 1) * half;
          for (int col0 = wg * half; col0 < col_end; col0 += 16) {
            const int cnt = min(16, col_end - col0);  // 16 or 8
            uint32_t r0[16], r1[16];
            if (cnt == 16) {
              tmem_ld_x16(tl + col0, r0);
              tmem_ld_x16(tl + TMEM_L12 + col0, r1);
            } else {
              tmem_ld_x8(tl + col0, *reinterpret_cast<uint32_t(*)[8]>(&r0[0]));
              tmem_ld_x8(tl + TMEM_L12 + col0, *reinterpret_cast<uint32_t(*)[8]>(&r1[0]));
            }
            tmem_ld_wait();
            // stash the two levels' sum rounded once to FP32 (whole tile or piece); the drainers scale
            // and add it. Its rounding, 2^-24 of the chunk's value and unbiased, sits far below the
            // truncation error the level-1+2 accumulator already carries, and halves the stash.
            if (ddead) continue;
#pragma unroll
            for (int jj = 0; jj < 16; ++jj)
              if (jj < cnt) fscr[(col0 + jj) * 128 + m_row] = __fadd_rn(__uint_as_float(r0[jj]), __uint_as_float(r1[jj]));
          }
          tc_fence_before();
          __threadfence_block();  // the stash is visible before it is announced
          __syncwarp();
          if (lane == 0) mbar_arrive(accempty);
          if (bt == 0) {
            sdesc[0] = piece ? 3 : 1;
            sdesc[1] = b;
            sdesc[2] = it;
            sdesc[3] = jt;
            sdesc[4] = c;
            sdesc[5] = (lc - 1) & 1;
            sdesc[6] = cur.pid;
            sdesc[7] = c == cur.c0;  // first chunk of the piece: its partial buffer starts here
          }
          __syncwarp();
          if (lane == 0) mbar_arrive(stashed);
          ++ns;
          named_bar_sync(1, NBG);  // exponent table of this chunk no longer needed
        }
      }
      more = more && !(cur.flags & 1);
      ++pos;
    }
    // end of work: let the drainers finish the last stash, then tell them to stop
    if (ns > 0 && !ddead && !mbar_wait_bounded(drained, (ns - 1) & 1, kWaitNs) && lane == 0)
      atomicCAS(p.d_err, DEV_OK, DEV_TIMEOUT);
    __syncwarp();
    if (bt == 0) sdesc[0] = 2;
    __syncwarp();
    if (lane == 0) mbar_arrive(stashed);
  } else {
    // ---------------- drainers: double-float read-modify-write of each stashed chunk.
    // Thread (warp dw, lane) owns accumulator lanes m = dw * 32 + lane (Re rows) and m + 64 (Im
    // rows), i.e. row I = it * 64 + m of the tile, for all N columns; 8 columns (16 elements) per
    // round trip. Whole tiles go into the accumulator, each element of which only this CTA
    // writes; pieces of split tiles go into the piece's own partial buffer ([n][m], as the stash),
    // written rather than added on the piece's first chunk.
    const int mlo = (warp - 2 - NBG / 32) * 32 + lane;
    const float* const fscr = reinterpret_cast<const float*>(p.fscr + (size_t)blockIdx.x * kFscrPerCta);
    for (int nd = 0;; ++nd) {
      if (!mbar_wait_bounded(stashed, nd & 1, kWaitNs)) {
        if (lane == 0) atomicCAS(p.d_err, DEV_OK, DEV_TIMEOUT);
        break;
      }
      const int kind = sdesc[0];
      if (kind == 2) break;
      if (kind == 1 || kind == 3) {
        const BlockDesc& bd = sBlk[sdesc[1]];
        const int it = sdesc[2], jt = sdesc[3], c = sdesc[4];
        const float* scB = sScB + sdesc[5] * 256;
        const bool whole = kind == 1, first = !whole && sdesc[7];
        const int I = it * TI + mlo;
        const size_t nn = (size_t)bd.n_pad * bd.n_pad;
        // target of column n, Re row: dst + col_off(n); the Im row is hs further
        float2* const dst = whole ? bd.acc + I : p.pbuf + (size_t)sdesc[6] * kFscrPerCta + mlo;
        const size_t hs = whole ? nn : 64;
        const int jmax = whole ? bd.n_pb - jt * TJ : TJ;  // tile columns j < jmax lie inside the matrix
        if (!whole || I < bd.n_pb) {
          const float scA = exp2i(-bd.expA[(size_t)c * bd.n_pad + I]);  // the Re and Im rows of I share it
          for (int n0 = 0; n0 < N; n0 += 8) {
            float x[16];
            float2 v[16];
            float sc[8];
            size_t off[8];
            uint32_t okm = 0;
#pragma unroll
            for (int e = 0; e < 8; ++e) {
              const int n = n0 + e, l = n / TJ, j = n - l * TJ;
              if (n < N && j < jmax) {
                okm |= 1u << e;
                sc[e] = scA * scB[n];
                off[e] = whole ? (size_t)l * 2 * nn + (size_t)(jt * TJ + j) * bd.n_pad : (size_t)n * 128;
                x[2 * e] = fscr[n * 128 + mlo];
                x[2 * e + 1] = fscr[n * 128 + mlo + 64];
                v[2 * e] = first ? make_float2(0.f, 0.f) : dst[off[e]];
                v[2 * e + 1] = first ? make_float2(0.f, 0.f) : dst[off[e] + hs];
              }
            }
#pragma unroll
            for (int e = 0; e < 8; ++e)
              if (okm & (1u << e)) {
                df_add(v[2 * e], x[2 * e] * sc[e]);
                df_add(v[2 * e + 1], x[2 * e + 1] * sc[e]);
                dst[off[e]] = v[2 * e];
                dst[off[e] + hs] = v[2 * e + 1];
              }
          }
        }
      }
      __syncwarp();
      if (lane == 0) mbar_arrive(drained);
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    tmem_dealloc(tmem, 512);
  }
}

// After the tensor-core launch: the P piece partials of each split tile r (pieces r * P .. r * P +
// P - 1), summed in piece order in FP64 and added to the FP64 accumulator, which the readout adds
// to the double-float one. One CTA row per split tile; no atomics, so the result is deterministic.
__global__ void __launch_bounds__(256) piece_reduce_kernel(MainArgs p) {
  const int r = blockIdx.x, gt = p.T_whole + r;
  const BlockDesc& bd = p.blk[block_of_tile(p.blk, p.nb, gt)];
  const int2 tile = bd.tiles[gt - bd.tile_off];
  const int N = p.N, TJ = p.TJ;
  const size_t nn = (size_t)bd.n_pad * bd.n_pad;
  for (int e = blockIdx.y * blockDim.x + threadIdx.x; e < N * 128; e += gridDim.y * blockDim.x) {
    const int n = e >> 7, m = e & 127;
    const int I = tile.x * TI + (m % TI), part = m / TI, l = n / TJ, J = tile.y * TJ + (n - l * TJ);
    if (I >= bd.n_pb || J >= bd.n_pb) continue;
    double sum = 0.0;
    for (int q = 0; q < p.P; ++q) {
      const float2 v = p.pbuf[(size_t)(r * p.P + q) * kFscrPerCta + e];
      sum += (double)v.x + (double)v.y;
    }
    bd.acc2[(size_t)part * nn + I + (size_t)l * 2 * nn + (size_t)J * bd.n_pad] += sum;
  }
}

// ------------------------------------------------------------------ host side
// J columns per tile: the widest TJ with N = TJ * L <= 256 and N % 16 == 0 (MMA shape rule for
// M = 128), within the kernel's shared memory. L = 12: 20, L = 16: 16, L = 1: 256.
static bool tile_width_ok(int t, int L) {
  return t >= 1 && t * L >= 16 && t * L <= 256 && (t * L) % 16 == 0 && main_smem_bytes(t * L) <= kSmemMax;
}

static int tile_width(int L) {
  for (int t = 256 / L; t >= 1; --t)
    if (tile_width_ok(t, L)) return t;
  return 0;
}

int mixed_tile_cols(int L) { return L >= 1 && L <= kMaxOmega ? tile_width(L) : 0; }

// Default width for one block of n_pb rows: among the valid widths down to 3/4 of the widest, the one
// whose J tiles overhang n_pb least (the overhang is padding the MMAs compute), the wider on a tie.
// n_pb = 428 at L = 1: 224 (2 J tiles, 448 rows) rather than 256 (512 rows).
static int tile_width_for(int L, int n_pb) {
  const int t0 = tile_width(L);
  int best = t0;
  long long best_rows = (long long)(n_pb + t0 - 1) / t0 * t0;
  for (int t = t0 - 1; 4 * t >= 3 * t0; --t) {
    if (!tile_width_ok(t, L)) continue;
    const long long rows = (long long)(n_pb + t - 1) / t * t;
    if (rows < best_rows) {
      best = t;
      best_rows = rows;
    }
  }
  return best;
}

bool mixed_plan_valid(int L, const TilePlan& p) {
  return L >= 1 && L <= kMaxOmega && (p.tj == 0 || tile_width_ok(p.tj, L)) && p.pieces >= 0 && p.pieces <= 64;
}

int mixed_plan_candidates(int L, TilePlan* out, int max_out) {
  if (L < 1 || L > kMaxOmega) return 0;
  int n = 0, widths = 0;
  for (int t = 256 / L; t >= 1 && widths < 3; --t) {
    if (!tile_width_ok(t, L)) continue;
    ++widths;
    for (int pieces : {0, 1})
      if (n < max_out) out[n++] = TilePlan{t, pieces};
  }
  return n;
}

static int ilog2(long long x) {
  int e = 0;
  while (x > 1) {
    x >>= 1;
    ++e;
  }
  return e;
}

void mixed_plan_class(int nb, const MixedBlock* in, int* ca, int* cc) {
  long long area = 0;
  long long ch = 1;
  for (int b = 0; b < nb; ++b) {
    area += (long long)(in[b].n_pad / TI) * (in[b].n_pad / TI);
    const long long K = (long long)in[b].n_occ * in[b].n_unocc;
    ch = std::max(ch, (K + CHR - 1) / CHR);
  }
  *ca = ilog2(std::max(1LL, area));
  *cc = ilog2(ch);
}

static size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

static bool herk_set_attributes() {
  return cudaFuncSetAttribute(herk_mixed_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemMax) ==
             cudaSuccess &&
         cudaFuncSetAttribute(prep_sym_kernel<double2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)kPrepSymSmem) == cudaSuccess &&
         cudaFuncSetAttribute(prep_sym_kernel<float2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)kPrepSymSmem) == cudaSuccess;
}

// Device list of the tiles on or above the diagonal for one (n_pb, TJ), cached in the scratch. The
// order is column-major (J tile outer), so the CTAs that run at the same time share J tiles and
// read each B image from L2 rather than HBM.
static qsgw_status tile_list(MixedScratch& s, int n_pb, int n_pad, int TJ, int rows_i, int col0, const int2** out,
                             int* count) {
  for (auto& e : s.tile_lists)
    if (e.n_pb == n_pb && e.tj == TJ && e.rows_i == rows_i && e.col0 == col0) {
      *out = e.tiles;
      *count = e.count;
      return QSGW_OK;
    }
  std::vector<int2> tl;
  const int n_it = n_pad / TI, n_jt = (n_pb + TJ - 1) / TJ;
  if (rows_i > 0) {  // the off-diagonal block: I tiles covering rows [0, rows_i), J tiles from col0
    for (int jt = col0 / TJ; jt < n_jt; ++jt)
      for (int it = 0; it * TI < rows_i; ++it) tl.push_back(make_int2(it, jt));
  } else {
    for (int jt = 0; jt < n_jt; ++jt)
      for (int it = 0; it < n_it; ++it)
        if (jt * TJ + TJ - 1 >= it * TI && it * TI < n_pb) tl.push_back(make_int2(it, jt));
  }
  if (tl.empty()) return QSGW_ERR_ARG;
  int2* d = nullptr;
  if (cudaMalloc(&d, tl.size() * sizeof(int2)) != cudaSuccess) return QSGW_ERR_NOMEM;
  if (cudaMemcpy(d, tl.data(), tl.size() * sizeof(int2), cudaMemcpyHostToDevice) != cudaSuccess) {
    cudaFree(d);
    return QSGW_ERR_CUDA;
  }
  s.tile_lists.push_back({n_pb, TJ, rows_i, col0, (int)tl.size(), d});
  *out = d;
  *count = (int)tl.size();
  return QSGW_OK;
}

// One block's shape within one launch (K: the launch's columns of the block) and its scratch.
struct Geom {
  long long K;
  int n_ch, n_kb, n_it, n_jt, n_itb;
};
static Geom geom_of(int n_pb, int n_pad, long long K, int TJ) {
  Geom G;
  G.K = K;
  G.n_ch = (int)((K + CHR - 1) / CHR);
  G.n_kb = G.n_ch * KB_PER_CH;
  G.n_it = n_pad / TI;
  G.n_jt = (n_pb + TJ - 1) / TJ;
  G.n_itb = (std::max(n_pad, G.n_jt * TJ) + TI - 1) / TI;  // row tiles of the prep: A rows and B rows
  return G;
}
// Digit-plane bytes of one K-block: the row image, and the B image unless L = 1 (where the row
// image is the B operand too).
static size_t plane_bytes_per_kb(const Geom& G, int N, int L) {
  return (size_t)3 * G.n_itb * TI * 64 + (L == 1 ? 0 : (size_t)G.n_jt * b_stage_bytes(N));
}
static size_t geom_bytes(const Geom& G, int n_pad, int N, int L) {
  return align256((size_t)G.n_kb * 3 * G.n_itb * TI * 64) +
         align256(L == 1 ? 0 : (size_t)G.n_jt * G.n_kb * b_stage_bytes(N)) +
         align256((size_t)G.n_kb * KBR * L * sizeof(float)) + 2 * align256((size_t)G.n_ch * n_pad * sizeof(float)) +
         align256((size_t)G.n_ch * L * sizeof(float));
}
struct Carve {
  uint8_t* a;  // row image
  uint8_t* b;  // B image (null at L = 1)
  float* w;
  float* zmax;
  int* expA;
  float* wmax;
};
static Carve carve(uint8_t* base, const Geom& G, int n_pad, int N, int L) {
  Carve c;
  size_t o = 0;
  c.a = base + o;
  o += align256((size_t)G.n_kb * 3 * G.n_itb * TI * 64);
  c.b = L == 1 ? nullptr : base + o;
  o += align256(L == 1 ? 0 : (size_t)G.n_jt * G.n_kb * b_stage_bytes(N));
  c.w = reinterpret_cast<float*>(base + o);
  o += align256((size_t)G.n_kb * KBR * L * sizeof(float));
  c.zmax = reinterpret_cast<float*>(base + o);
  o += align256((size_t)G.n_ch * n_pad * sizeof(float));
  c.expA = reinterpret_cast<int*>(base + o);
  o += align256((size_t)G.n_ch * n_pad * sizeof(float));
  c.wmax = reinterpret_cast<float*>(base + o);
  return c;
}

// One launch sequence over nb blocks, each with Z at the launch's first column (block column r0[b])
// and its shape and scratch: prep_cols, prep_rows (A and B digit planes), the persistent
// tensor-core kernel over all (block, tile, chunk) items, and the ordered reduction of the pieces of
// split tiles. grid_cap: CTAs at most (and flush-scratch slots in fscr / pbuf).
static qsgw_status launch_blocks(int nb, const MixedBlock* in, const long long* r0, const Geom* G, const Carve* S,
                                 const int2* const* tiles, const int* n_tiles, const OmegaGrid& g, int TJ, int pieces,
                                 int grid_cap, float2* fscr, float2* pbuf, int* counter, int* d_err,
                                 cudaStream_t stream) {
  const int L = g.L, N = TJ * L;
  MainArgs a;
  std::memset(&a, 0, sizeof(a));
  a.nb = nb;
  a.L = L;
  a.TJ = TJ;
  a.N = N;
  a.idesc = make_idesc_f16_f32(128, (uint32_t)N);
  a.d_err = d_err;
  a.fscr = fscr;
  a.pbuf = pbuf;
  a.counter = counter;
  PrepColsArgs pc;
  std::memset(&pc, 0, sizeof(pc));
  pc.g = g;
  pc.d_err = d_err;
  PrepRowsArgs pr[2];  // [0]: complex128 Z, [1]: complex64
  std::memset(pr, 0, sizeof(pr));
  for (int t = 0; t < 2; ++t) {
    pr[t].TJ = TJ;
    pr[t].L = L;
    pr[t].N = N;
  }
  int T = 0, min_ch_tail = 1 << 30;
  int nr[2] = {0, 0}, max_it[2] = {0, 0}, max_ita[2] = {0, 0}, max_chr[2] = {0, 0}, max_ch = 0;
  for (int b = 0; b < nb; ++b) {
    const MixedBlock& B = in[b];
    BlockDesc& d = a.blk[b];
    d.rimg = S[b].a;
    d.bplanes = S[b].b;
    d.zmax = S[b].zmax;
    d.expA = S[b].expA;
    d.wmax = S[b].wmax;
    d.tiles = tiles[b];
    d.n_tiles = n_tiles[b];
    d.acc = reinterpret_cast<float2*>(B.acc);
    d.acc2 = reinterpret_cast<double*>(d.acc + (size_t)L * 2 * B.n_pad * B.n_pad);
    d.tile_off = T;
    d.n_pb = B.n_pb;
    d.n_pad = B.n_pad;
    d.n_kb = G[b].n_kb;
    d.n_kbr = (int)((G[b].K + KBR - 1) / KBR);
    d.n_ch = G[b].n_ch;
    d.n_rows = G[b].n_itb * TI;
    T += d.n_tiles;
    pc.b[b] = PrepColsBlk{B.eo, B.eu, B.wv, S[b].w, S[b].wmax, G[b].K, r0[b], B.n_unocc, G[b].n_ch};
    const int t = B.z32 ? 1 : 0;
    pr[t].b[nr[t]++] = PrepRowsBlk{B.Z, B.ldz, G[b].K, S[b].a, S[b].b, S[b].w, S[b].wmax, S[b].zmax, S[b].expA,
                                   B.n_pb, B.n_pad, G[b].n_kb, G[b].n_jt, G[b].n_ch, G[b].n_it, G[b].n_itb,
                                   B.rows_i > 0 ? B.rows_i : B.n_pad, B.rows_i > 0 ? B.col0 : 0};
    max_ch = std::max(max_ch, G[b].n_ch);
    max_chr[t] = std::max(max_chr[t], G[b].n_ch);
    max_it[t] = std::max(max_it[t], G[b].n_itb);
    max_ita[t] = std::max(max_ita[t], G[b].n_it);
  }
  prep_cols_kernel<<<dim3(max_ch, nb), PC_THREADS, 0, stream>>>(pc);
  if (L == 1) {  // one pass: maxima and the row image, Z read once
    const int rg = TI / PS_ROWS;
    if (nr[0] > 0)
      prep_sym_kernel<double2><<<dim3(max_chr[0], max_it[0] * rg, nr[0]), 256, kPrepSymSmem, stream>>>(pr[0]);
    if (nr[1] > 0)
      prep_sym_kernel<float2><<<dim3(max_chr[1], max_it[1] * rg, nr[1]), 256, kPrepSymSmem, stream>>>(pr[1]);
  } else {
    if (nr[0] > 0) {
      prep_max_kernel<double2><<<dim3(max_chr[0], max_ita[0], nr[0]), 256, 0, stream>>>(pr[0]);
      prep_rows_kernel<double2><<<dim3(max_chr[0] * PR_SPLIT, max_it[0], nr[0]), 256, 0, stream>>>(pr[0]);
    }
    if (nr[1] > 0) {
      prep_max_kernel<float2><<<dim3(max_chr[1], max_ita[1], nr[1]), 256, 0, stream>>>(pr[1]);
      prep_rows_kernel<float2><<<dim3(max_chr[1] * PR_SPLIT, max_it[1], nr[1]), 256, 0, stream>>>(pr[1]);
    }
  }
  // whole tiles first; the last R tiles (a partial last wave) are split into P chunk ranges
  const int Gc = grid_cap;
  const int R = T >= Gc ? T % Gc : T;
  a.T = T;
  a.T_whole = T - R;
  for (int b = 0; b < nb; ++b) {  // smallest chunk count among blocks that own tail tiles
    const BlockDesc& d = a.blk[b];
    if (d.tile_off + d.n_tiles > a.T_whole && d.n_ch < min_ch_tail) min_ch_tail = d.n_ch;
  }
  int P = R > 0 ? Gc / R : 1;
  if (P < 1) P = 1;
  if (pieces > 0) P = pieces;
  if (R > 0 && P > min_ch_tail) P = min_ch_tail;
  a.P = P;
  a.n_items = a.T_whole + R * P;
  if (cudaMemsetAsync(counter, 0, sizeof(int), stream) != cudaSuccess) return QSGW_ERR_CUDA;
  const int grid = a.n_items < Gc ? a.n_items : Gc;
  herk_mixed_kernel<<<grid, NTHREADS, main_smem_bytes(N), stream>>>(a);
  if (R > 0) piece_reduce_kernel<<<dim3(R, (N * 128 + 255) / 256), 256, 0, stream>>>(a);
  return cudaGetLastError() == cudaSuccess ? QSGW_OK : QSGW_ERR_CUDA;
}

// Digit planes (row image and B image) of one launch at most: a call whose planes would exceed it
// runs as launches over chunk ranges (every launch covers the same chunks of every block; each chunk is flushed into the
// accumulator anyway, so the cut changes nothing but the launch count).
constexpr size_t kBPlaneBudget = 8ull << 30;

static const void* advance_cols(const void* Z, bool z32, long long ldz, long long r0) {
  return static_cast<const uint8_t*>(Z) + (size_t)r0 * ldz * (z32 ? sizeof(float2) : sizeof(double2));
}

qsgw_status mixed_accumulate_batch(MixedScratch& s, int nb, const MixedBlock* in, const OmegaGrid& g, int* d_err,
                                   cudaStream_t stream) {
  if (nb < 1 || nb > kMaxBlocks) return QSGW_ERR_ARG;
  const int L = g.L;
  // the tile plan: forced, tuned for this size class, or the default; launches over a restricted
  // block (the I^c products, whose row offsets are multiples of the default width) keep the default
  TilePlan plan;
  bool restricted = false;
  for (int b = 0; b < nb; ++b) restricted = restricted || in[b].rows_i > 0;
  if (!restricted) {
    if (s.use_forced) {
      plan = s.forced;
    } else if (!s.plans.empty()) {
      int ca = 0, cc = 0;
      mixed_plan_class(nb, in, &ca, &cc);
      for (const PlanEntry& e : s.plans)
        if (e.L == L && e.ca == ca && e.cc == cc) plan = e.plan;
    }
  }
  const int TJ = plan.tj > 0 ? plan.tj : (nb == 1 && !restricted ? tile_width_for(L, in[0].n_pb) : tile_width(L));
  const int N = TJ * L;
  if (!tile_width_ok(TJ, L)) return QSGW_ERR_ARG;
  if (s.n_sm == 0) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&s.n_sm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
      return QSGW_ERR_CUDA;
  }
  if (!s.attr_set) {
    if (!herk_set_attributes()) return QSGW_ERR_CUDA;
    s.attr_set = true;
  }
  const int2* tiles[kMaxBlocks];
  int n_tiles[kMaxBlocks];
  long long Kb[kMaxBlocks];
  int max_ch = 0;
  size_t b_per_chunk = 0;  // digit-plane bytes of one chunk of every block
  for (int b = 0; b < nb; ++b) {
    const MixedBlock& B = in[b];
    if (B.rows_i > 0 && (B.col0 % TJ != 0 || B.col0 < B.rows_i || B.col0 >= B.n_pb)) return QSGW_ERR_ARG;
    qsgw_status st = tile_list(s, B.n_pb, B.n_pad, TJ, B.rows_i, B.col0, &tiles[b], &n_tiles[b]);
    if (st != QSGW_OK) return st;
    Kb[b] = (long long)B.n_occ * B.n_unocc;
    max_ch = std::max(max_ch, (int)((Kb[b] + CHR - 1) / CHR));
    b_per_chunk += KB_PER_CH * plane_bytes_per_kb(geom_of(B.n_pb, B.n_pad, CHR, TJ), N, L);
  }
  int cpl = max_ch;  // chunks per launch
  if ((size_t)cpl * b_per_chunk > kBPlaneBudget) cpl = std::max(1, (int)(kBPlaneBudget / b_per_chunk));
  // scratch: flush areas, then the blocks' planes for the first (largest) launch
  const size_t fscr_bytes = align256((size_t)s.n_sm * kFscrPerCta * sizeof(float2));
  size_t total = 2 * fscr_bytes;
  for (int b = 0; b < nb; ++b)
    total += geom_bytes(geom_of(in[b].n_pb, in[b].n_pad, std::min(Kb[b], (long long)cpl * CHR), TJ), in[b].n_pad, N,
                        L);
  if (s.planes_cap < total) {
    if (s.planes) cudaFree(s.planes);
    s.planes = nullptr;
    s.planes_cap = 0;
    if (cudaMalloc(&s.planes, total) != cudaSuccess) return QSGW_ERR_NOMEM;
    s.planes_cap = total;
  }
  if (!s.counter && cudaMalloc(&s.counter, sizeof(int)) != cudaSuccess) return QSGW_ERR_NOMEM;
  uint8_t* base = static_cast<uint8_t*>(s.planes);
  float2* fscr = reinterpret_cast<float2*>(base);
  float2* pbuf = reinterpret_cast<float2*>(base + fscr_bytes);
  for (int c0 = 0; c0 < max_ch; c0 += cpl) {
    MixedBlock sub[kMaxBlocks];
    long long r0[kMaxBlocks];
    Geom G[kMaxBlocks];
    Carve S[kMaxBlocks];
    const int2* st_tiles[kMaxBlocks];
    int st_n[kMaxBlocks];
    int ns = 0;
    size_t off = 2 * fscr_bytes;
    for (int b = 0; b < nb; ++b) {
      const long long c0r = (long long)c0 * CHR;
      if (Kb[b] <= c0r) continue;  // this block's columns ended in an earlier launch
      sub[ns] = in[b];
      sub[ns].Z = advance_cols(in[b].Z, in[b].z32, in[b].ldz, c0r);
      r0[ns] = c0r;
      G[ns] = geom_of(in[b].n_pb, in[b].n_pad, std::min(Kb[b] - c0r, (long long)cpl * CHR), TJ);
      S[ns] = carve(base + off, G[ns], in[b].n_pad, N, L);
      off += geom_bytes(G[ns], in[b].n_pad, N, L);
      st_tiles[ns] = tiles[b];
      st_n[ns] = n_tiles[b];
      ++ns;
    }
    qsgw_status st = launch_blocks(ns, sub, r0, G, S, st_tiles, st_n, g, TJ, plan.pieces, s.n_sm, fscr, pbuf,
                                   s.counter, d_err, stream);
    if (st != QSGW_OK) return st;
  }
  return QSGW_OK;
}

qsgw_status mixed_accumulate(MixedScratch& s, const void* Z, bool z32, long long ldz, int n_pb, int n_pad, int n_occ,
                             int n_unocc, const double* eo, const double* eu, const double* wv, const OmegaGrid& g,
                             float4* acc, int* d_err, cudaStream_t stream) {
  MixedBlock b{Z, ldz, n_pb, n_pad, n_occ, n_unocc, eo, eu, acc, z32, wv};
  return mixed_accumulate_batch(s, 1, &b, g, d_err, stream);
}

// ------------------------------------------------------------------ allocation-free variant
// One block of columns, chi0 written straight to the caller's buffer, every intermediate in a
// fixed file-scope device array instead of cudaMalloc'd scratch. See qsgw_chi0_block_noalloc.
// The columns go through the array one chunk of 1024 at a time, so the number of columns does not
// count against it.
constexpr size_t kNoAllocBytes = 128ull << 20;
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

// Upper-triangle tile list of one (n_pb, TJ), in the order tile_list() uses, built on the device.
__global__ void noalloc_tiles_kernel(int n_pb, int n_it, int n_jt, int TJ, int2* out) {
  if (blockIdx.x != 0 || threadIdx.x != 0) return;
  int k = 0;
  for (int jt = 0; jt < n_jt; ++jt)
    for (int it = 0; it < n_it; ++it)
      if (jt * TJ + TJ - 1 >= it * TI && it * TI < n_pb) out[k++] = make_int2(it, jt);
}

qsgw_status mixed_chi0_noalloc(const double2* Z, long long ldz, int n_pb, int n_occ, int n_unocc, const double* eo,
                               const double* eu, const OmegaGrid& g, double spin, double2* chi0, cudaStream_t stream) {
  const int L = g.L, TJ = tile_width(L), N = TJ * L;
  if (TJ < 1) return QSGW_ERR_ARG;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return QSGW_ERR_CUDA;
  // Set-up on every call, in the current context: the array's device address (a lookup, no
  // allocation) and the kernel's shared-memory limit. Neither is cached, because both belong to
  // the context: after cudaDeviceReset the module is loaded again and the array may move.
  void* scratch = nullptr;
  if (cudaGetSymbolAddress(&scratch, g_noalloc_scratch) != cudaSuccess || !scratch) return QSGW_ERR_CUDA;
  if (!herk_set_attributes()) return QSGW_ERR_CUDA;
  int n_sm = 0;
  if (cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return QSGW_ERR_CUDA;
  const int n_pad = pad_to(n_pb, kPad);
  const long long K = (long long)n_occ * n_unocc;
  const int n_ch = (int)((K + CHR - 1) / CHR);
  const int n_it = n_pad / TI, n_jt = (n_pb + TJ - 1) / TJ;
  int n_tiles = 0;
  for (int it = 0; it < n_it; ++it)
    for (int jt = 0; jt < n_jt; ++jt)
      if (jt * TJ + TJ - 1 >= it * TI && it * TI < n_pb) ++n_tiles;
  // layout inside the fixed array: error flag and work counter, accumulators, tile list, the planes
  // of one chunk, then per-CTA flush scratch and as many piece partial buffers; the grid is capped to
  // the CTAs there is room for
  size_t off = 256;
  const size_t o_acc = off;
  const size_t acc_bytes = (size_t)L * 2 * n_pad * n_pad * (sizeof(float2) + sizeof(double));
  off += align256(acc_bytes);
  const size_t o_tiles = off;
  off += align256((size_t)n_tiles * sizeof(int2));
  const size_t o_blk = off;
  off += geom_bytes(geom_of(n_pb, n_pad, std::min(K, (long long)CHR), TJ), n_pad, N, L);
  const size_t o_fscr = off, fscr_cta = (size_t)kFscrPerCta * sizeof(float2);
  if (off + 2 * fscr_cta > kNoAllocBytes) return QSGW_ERR_ARG;  // beyond the fixed array: use the context API
  const int cap_ctas = (int)((kNoAllocBytes - off) / (2 * fscr_cta));
  uint8_t* base = static_cast<uint8_t*>(scratch);
  int* d_err = reinterpret_cast<int*>(base);
  int* counter = d_err + 1;
  // the array keeps the previous call's contents: clear what must start at zero
  if (cudaMemsetAsync(base, 0, 256, stream) != cudaSuccess) return QSGW_ERR_CUDA;
  if (cudaMemsetAsync(base + o_acc, 0, acc_bytes, stream) != cudaSuccess) return QSGW_ERR_CUDA;
  int2* tiles = reinterpret_cast<int2*>(base + o_tiles);
  noalloc_tiles_kernel<<<1, 1, 0, stream>>>(n_pb, n_it, n_jt, TJ, tiles);
  float2* fscr = reinterpret_cast<float2*>(base + o_fscr);
  float2* pbuf = reinterpret_cast<float2*>(base + o_fscr + (size_t)cap_ctas * fscr_cta);
  const int grid_cap = n_sm < cap_ctas ? n_sm : cap_ctas;
  const int2* tl = tiles;
  for (int c = 0; c < n_ch; ++c) {
    const long long r0 = (long long)c * CHR;
    const Geom G = geom_of(n_pb, n_pad, std::min(K - r0, (long long)CHR), TJ);
    const Carve S = carve(base + o_blk, G, n_pad, N, L);
    MixedBlock B{advance_cols(Z, false, ldz, r0), ldz, n_pb, n_pad, n_occ, n_unocc, eo, eu,
                 reinterpret_cast<float4*>(base + o_acc), false, nullptr};
    const qsgw_status st =
        launch_blocks(1, &B, &r0, &G, &S, &tl, &n_tiles, g, TJ, 0, grid_cap, fscr, pbuf, counter, d_err, stream);
    if (st != QSGW_OK) return st;
  }
  launch_finalize_chi(base + o_acc, ACC_DF32, n_pb, n_pad, L, spin, chi0, stream);
  if (cudaGetLastError() != cudaSuccess) return QSGW_ERR_CUDA;
  int h_err = 0;
  if (cudaMemcpyAsync(&h_err, d_err, sizeof(int), cudaMemcpyDeviceToHost, stream) != cudaSuccess ||
      cudaStreamSynchronize(stream) != cudaSuccess)
    return QSGW_ERR_CUDA;
  if (h_err == DEV_DOMAIN) return QSGW_ERR_DOMAIN;
  if (h_err == DEV_TIMEOUT) return QSGW_ERR_TIMEOUT;
  return QSGW_OK;
}

qsgw_status mixed_autotune(MixedScratch& s, int nb, const MixedBlock* in, const OmegaGrid& g, int* d_err,
                           cudaStream_t stream, int reps, TilePlan* best, float* best_ms) {
  if (nb < 1 || nb > kMaxBlocks || reps < 1) return QSGW_ERR_ARG;
  for (int b = 0; b < nb; ++b)
    if (in[b].rows_i > 0) return QSGW_ERR_ARG;
  const int L = g.L;
  std::vector<MixedBlock> blk(in, in + nb);
  size_t total = 0;
  std::vector<size_t> off(nb);
  for (int b = 0; b < nb; ++b) {  // scratch accumulators of the blocks' own sizes
    off[b] = total;
    total += align256((size_t)blk[b].n_pad * blk[b].n_pad * L * 2 * sizeof(float4));
  }
  void* tmp = nullptr;
  if (cudaMalloc(&tmp, total) != cudaSuccess) {
    cudaGetLastError();
    return QSGW_ERR_NOMEM;
  }
  for (int b = 0; b < nb; ++b) blk[b].acc = reinterpret_cast<float4*>(static_cast<uint8_t*>(tmp) + off[b]);
  TilePlan cand[16];
  const int nc = mixed_plan_candidates(L, cand, 16);
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  qsgw_status st = QSGW_OK;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) st = QSGW_ERR_CUDA;
  const bool saved_use = s.use_forced;
  const TilePlan saved = s.forced;
  float bms = 0.f;
  TilePlan bp;
  for (int c = 0; c < nc && st == QSGW_OK; ++c) {
    s.use_forced = true;
    s.forced = cand[c];
    st = mixed_accumulate_batch(s, nb, blk.data(), g, d_err, stream);  // warm-up: scratch, tile lists
    if (st != QSGW_OK) break;
    if (cudaEventRecord(e0, stream) != cudaSuccess) st = QSGW_ERR_CUDA;
    for (int r = 0; r < reps && st == QSGW_OK; ++r) st = mixed_accumulate_batch(s, nb, blk.data(), g, d_err, stream);
    if (st != QSGW_OK) break;
    float ms = 0.f;
    if (cudaEventRecord(e1, stream) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
        cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) {
      st = QSGW_ERR_CUDA;
      break;
    }
    ms /= reps;
    if (c == 0 || ms < bms) {
      bms = ms;
      bp = cand[c];
    }
  }
  s.use_forced = saved_use;
  s.forced = saved;
  cudaStreamSynchronize(stream);
  cudaFree(tmp);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (st != QSGW_OK) return st;
  if (nc == 0) return QSGW_ERR_ARG;
  int ca = 0, cc = 0;
  mixed_plan_class(nb, in, &ca, &cc);
  bool found = false;
  for (PlanEntry& e : s.plans)
    if (e.L == L && e.ca == ca && e.cc == cc) {
      e.plan = bp;
      found = true;
    }
  if (!found) s.plans.push_back(PlanEntry{L, ca, cc, bp});
  if (best) *best = bp;
  if (best_ms) *best_ms = bms;
  return QSGW_OK;
}

void mixed_free(MixedScratch& s) {
  if (s.planes) cudaFree(s.planes);
  if (s.counter) cudaFree(s.counter);
  for (auto& e : s.tile_lists) cudaFree(e.tiles);
  s = MixedScratch{};
}

}  // namespace qsgw
