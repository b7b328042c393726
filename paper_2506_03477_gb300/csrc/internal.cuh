// Internal declarations shared by the library's translation units (not installed).
#pragma once
#include <cuda_runtime.h>
#include <cstddef>
#include <cstdint>

#include "../../include/qsgw.h"

namespace qsgw {

constexpr int kMaxOmega = 16;
constexpr int kMaxNpb = 16384;
constexpr int kPad = 64;  // accumulators are padded to a multiple of 64 rows / columns

// Sticky device-side error codes (stored in ctx->d_err, first error wins).
enum DevErr : int { DEV_OK = 0, DEV_DOMAIN = 1, DEV_TIMEOUT = 2 };

struct OmegaGrid {
  int L;
  double w2[kMaxOmega];  // omega_l^2 (FP64)
  float w2f[kMaxOmega];  // omega_l^2 (FP32, mixed path)
};

inline int pad_to(int n, int m) { return (n + m - 1) / m * m; }

// ---- FP64 path (kernels_fp64.cu)
// |w_l(Delta_r)| for one k-point into w[l*ldw + r] (FP64); flags Delta <= 0 / non-finite.
void launch_weights_fp64(const double* eps_occ, const double* eps_unocc, int n_occ, int n_unocc, const OmegaGrid& g,
                         double* w, long long ldw, int* d_err, cudaStream_t s);
// w[r] = v[r mod period] (one weight set), domain check v > 0.
void launch_weights_given_fp64(const double* v, int period, long long K, double* w, int* d_err, cudaStream_t s);
// acc[l][J][I] += sum_r w[l][r] conj(Z[I,r]) Z[J,r] on upper-triangle 64x64 tiles. With S > 1 the
// columns are cut into S slices that sum into part ([S][L][n_pad][n_pad], caller's scratch) and are
// then added to acc in slice order; herk_fp64_slices picks S (1 unless output tiles are scarce).
// ti_end > 0 restricts the output to the block of I tiles [0, ti_end) and J tiles [tj0, n_pad/64)
// (tj0 >= ti_end): an off-diagonal block, i.e. a general product of two row sets of Z.
int herk_fp64_slices(int n_pad, int L, long long K, int ti_end = 0, int tj0 = 0);
void launch_herk_fp64(const double2* Z, long long ldz, int n_pb, int n_pad, long long K, const double* w,
                      long long ldw, int L, int S, double2* acc, double2* part, cudaStream_t s, int ti_end = 0,
                      int tj0 = 0);
// Blocks of distinct q-points in one launch over all (block, upper tile, K-slice) items; block b
// uses S = herk_fp64_slices(n_pad, L, K) slices (partials in part, reduced per block after the
// launch), so each block's result is bitwise that of launch_herk_fp64 on it alone.
struct Fp64Blk {
  const double2* Z;
  long long ldz, K;
  const double* w;  // weights [l][r], leading dimension ldw
  long long ldw;
  double2* acc;
  double2* part;  // S > 1: [S][L][n_pad][n_pad]
  int n_pb, n_pad, S, item0;
};
struct Fp64Batch {
  Fp64Blk b[32];
  int nb, L, items;
};
void launch_herk_fp64_batch(const Fp64Batch& p, cudaStream_t s);

// ---- shared epilogues (kernels_epsw.cu)
// Accumulator formats: FP64 complex (double2 [l][J][I]) or double-float planes (float2 hi/lo [l][re|im][J][I]).
enum AccKind { ACC_FP64 = 0, ACC_DF32 = 1 };
// chi0 = -s * mirror(acc): full Hermitian, diag imag = 0 (out is [L][n][n]).
void launch_finalize_chi(const void* acc, AccKind kind, int n, int n_pad, int L, double spin, double2* out,
                         cudaStream_t s);
// eps = I - D chi0 D with chi0 = -s * mirror(acc), full matrix.
void launch_form_eps(const void* acc, AccKind kind, int n, int n_pad, int L, double spin, const double* v,
                     double2* eps, cudaStream_t s);
// In place: lower triangle of sg * eps^{-1} (sg = +-1) -> full W = D eps^{-1} D (minus diag(v) if wc).
void launch_w_from_inverse(double2* w, int n, int L, const double* v, int wc, double sg, cudaStream_t s);

// ---- eps^{-1} (epsinv.cu)
// In place on w ([L][n][n], column-major; the lower triangle of each Hermitian positive definite
// matrix is read): the lower triangle becomes -eps^{-1}. sbuf: [L][32][32], pbuf and cbuf:
// [L][32][n] complex128 scratch. dig: eps_inverse_digit_bytes(n, L) bytes of scratch for the
// update on the tensor cores (FP64 accuracy from exact integer digits), or null for the plain DFMA
// update. d_info[l] (zeroed by the caller) receives the 1-based index of the first non-positive
// pivot, as a Cholesky factorisation would report it; a bounded wait that gave up sets d_err.
size_t eps_inverse_digit_bytes(int n, int L);
void launch_eps_inverse(double2* w, int n, int L, double2* sbuf, double2* pbuf, double2* cbuf, uint8_t* dig,
                        int* d_info, int* d_err, cudaStream_t s);

// ---- real-axis route (spectral.cu)
// Bin every column by Delta (edges: device [n_bins + 1]), count per bin, exclusive offsets
// ([n_bins + 1]) and the stable permutation perm (columns in bin order; offsets[n_bins] of them).
void launch_hist_sort(const double* eo, const double* eu, int n_occ, int n_unocc, const double* edges, int n_bins,
                      int* bins, int* counts, int* offsets, int* perm, int* d_err, cudaStream_t s);
// Sorted column p (p < n) -> column p - offsets[j] of dptr[j] (device array of n_bins device
// pointers), j its bin; complex64 destinations (z32) or complex128.
void launch_gather_bins(const double2* Z, long long ldz, int n_pb, const int* perm, const int* bins,
                        const int* offsets, int n, void* const* dptr, bool z32, cudaStream_t s);
// out[o] = sum_j K[j * n_out + o] S_j + i coef[o] S_{bins_out[o]} for o < n_out (device arrays;
// S [nb][n][n] exactly Hermitian, out [n_out][n][n], column-major complex128).
void launch_hilbert(const double2* S, int n, int nb, int n_out, const double* K, const int* bins_out,
                    const double* coef, double2* out, cudaStream_t s);

// ---- imaginary-axis correlation self-energy, Eq. (sigci) (sigc.cu)
struct SigcMesh {
  double om[kMaxOmega];  // the imaginary frequencies of W^c, increasing, om[0] > 0
  int L;
};
// w[i * NT + n' * n_qp + n] = w_i(e_qp[n] - e_band[n']) for every band n' < n_band and target n,
// NT = n_band * n_qp; non-finite energies set DEV_DOMAIN and weight 0.
void launch_sigc_weights(const double* e_qp, const double* e_band, int n_qp, int n_band, const SigcMesh& m,
                         double* w, int* d_err, cudaStream_t s);
// Zt (column-major M x n_pb) = transpose of columns [c0, c0 + M) of Z (column-major n_pb x ..., ldz).
void launch_transpose_cols(const double2* Z, long long ldz, int n_pb, long long c0, int M, double2* Zt, cudaStream_t s);
// Stacked operand of the product D = sum_i w_i conj(Z) W^c_i (column (i, mu), S2 = Y0 + n_pb rows):
// rows [0, M) w[i * NT + row0 + row] Zt[row, mu]; rows [M, Y0) zero; rows Y0 + nu conj(Wc_i[nu, mu]).
void launch_sigc_stack_d(const double2* Zt, int M, int n_pb, const double* w, long long NT, long long row0, int L,
                         const double2* Wc, int Y0, void* Z2, bool z32, cudaStream_t s);
// Stacked operand of I -= D Z^T over the columns (band b, nu) of nb bands (S3 = Y3 + n_qp rows):
// rows [0, n_qp) conj(D(b n_qp + n, nu)) read from the step-2 accumulator (element (I, J = Y0 + nu));
// rows [n_qp, Y3) zero; rows Y3 + m Zt[b n_qp + m, nu].
void launch_sigc_stack_i(const void* accD, AccKind kind, int n_padD, int Y0, const double2* Zt, int n_qp, int nb,
                         int n_pb, int Y3, void* Z3, bool z32, cudaStream_t s);
// out[m * n_qp + n] = -(accumulator element (I = n, J = Y3 + m)).
void launch_sigc_readout(const void* accI, AccKind kind, int n_padI, int n_qp, int Y3, double2* out, cudaStream_t s);

// ---- synthetic Z (synth.cu)
void launch_synth_z(unsigned long long seed, int gen_q, int k, int n_pb, int n_occ, int n_unocc, double s_div,
                    double2* Z, long long ldz, cudaStream_t s);

}  // namespace qsgw
