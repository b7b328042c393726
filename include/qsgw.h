/*
 * qsgw.h — C ABI of the GB300 (sm_103a) library that assembles the RPA polarization
 * chi0(q, i omega) in the mixed product basis and forms eps and W from it
 * (Obata, Kotani, Oda, "Efficient implementation of the quasiparticle self-consistent GW
 * method on GPU", arXiv:2506.03477).
 *
 * What is computed (Sec. 2, Eq. (polfx) on the imaginary axis, delta -> 0):
 *
 *   chi0_IJ(q, i omega_l) = s * sum_{k, n occ, m unocc} w_l(Delta_knm) conj(z_{I,knm}) z_{J,knm}
 *   w_l(Delta) = 1/(i omega_l - Delta) - 1/(i omega_l + Delta) = -2 Delta / (Delta^2 + omega_l^2)
 *   Delta_knm  = eps_unocc[k, m] - eps_occ[k, n]  (must be > 0)
 *
 * i.e. chi0(l) = -s * Y_l^H Y_l with Y_l = diag(sqrt|w_l|) Z^T: a Hermitian rank-K update per
 * frequency. The conjugate sits on the row index I, so chi0 is the transpose (equivalently
 * the complex conjugate) of the paper's Pi_{mu nu} = sum Z_mu Z_nu^* for the same Z. There is no
 * 1/N_k factor; Brillouin-zone weights belong in Z or in s.
 *
 *   eps_IJ = delta_IJ - sqrt(v_I) chi0_IJ sqrt(v_J)       Eq. (dielectricfunction)
 *   W_IJ   = sqrt(v_I) [eps^{-1}]_IJ sqrt(v_J)            Eq. (screenedcoulomb)
 *   W^c_IJ = W_IJ - v_I delta_IJ                          Eq. (wc)
 *
 * The same kernels also give, each in its own section below:
 *   - the exchange self-energy Sigma^x, Eq. (sigx): a Hermitian update with given column
 *     weights v_mu(k);
 *   - the real-axis route, Eqs. (impolf) and (hilbert): the spectral weight of every histogram
 *     bin of transition energies, then chi0 on the real axis;
 *   - the imaginary-axis correlation self-energy I^c, Eq. (sigci): D = sum_i w_i conj(Z) W^c_i
 *     and D Z^T, each as a block of a Hermitian update of a stacked operand.
 *
 * Conventions shared by every call
 *   - Complex numbers are interleaved (re, im) pairs of double (C99 double complex layout).
 *   - Matrices are column-major: element (I, J) of an n_pb x n_pb matrix is at J*n_pb + I.
 *     A stack over frequencies is [n_omega][n_pb][n_pb], frequency slowest.
 *   - Device pointers are CUDA global-memory pointers on the context's current device.
 *     Where a call says "device or host", the library detects pageable/pinned host memory
 *     with cudaPointerGetAttributes and stages it through device memory it owns.
 *   - The caller owns all inputs and outputs; the library only borrows them until the stream
 *     work of the call has completed. The context owns its accumulators and scratch.
 *   - Every call is asynchronous and ordered on the stream given to qsgw_chi0_init, except
 *     where stated. Argument errors are returned synchronously and leave the context
 *     unchanged. Errors found on the device (Delta <= 0, a bounded wait that gave up) are
 *     sticky: they are returned by the next qsgw_chi0_finalize, qsgw_eps_inv, qsgw_chi0_sync
 *     or qsgw_chi0_destroy, which synchronise the stream.
 *   - Not thread-safe: one host thread per context at a time.
 */
#ifndef QSGW_H
#define QSGW_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct qsgw_ctx qsgw_ctx; /* opaque; created by qsgw_chi0_init, owned by the library */

typedef enum {
  QSGW_OK = 0,
  QSGW_ERR_ARG = -1,     /* invalid argument (returned synchronously) */
  QSGW_ERR_DOMAIN = -2,  /* some Delta <= 0 or non-finite (device-detected, sticky) */
  QSGW_ERR_NOMEM = -3,   /* device allocation failed */
  QSGW_ERR_CUDA = -4,    /* a CUDA runtime / library call failed */
  QSGW_ERR_NOT_PD = -5,  /* eps not positive definite at some frequency (see info) */
  QSGW_ERR_TIMEOUT = -6, /* a bounded device-side wait gave up (sticky) */
  QSGW_ERR_STATE = -7    /* call not valid in the context's current state */
} qsgw_status;

typedef enum {
  QSGW_FP64 = 0,        /* FP64 arithmetic end to end (CUDA-core DFMA) */
  QSGW_MIXED_F16X3 = 1, /* tcgen05 tensor cores on exact 3-digit slices (an integer leading digit
                           and two FP16 digits; 6 products per flop pair), FP32 per chunk of 1024
                           columns, double-float (2 x FP32) across chunks; eps and W stay FP64 */
  QSGW_MIXED_BF16X3 = 1, /* the same value under its earlier name (the slices were BF16 then) */
  QSGW_MIXED_TF32X3 = 2  /* reserved, rejected by qsgw_chi0_init with QSGW_ERR_ARG: TF32 hi/lo
                            splitting (3 products) has no exact leading level, and the tensor
                            cores' truncating FP32 accumulation leaves 4e-6..1.7e-5 relative error,
                            above the 1e-6 bar; an exact-digit TF32 form needs 6 products at half
                            the FP16 rate, slower than QSGW_MIXED_F16X3 */
} qsgw_prec;

/* Create a context for n_q independent q-points (Alg. 1 loops over q; each q has its own
 * n_pb[q] product-basis size and its own accumulator).
 *   ctx          out: new context (NULL on error)
 *   n_q          number of q-points, >= 1
 *   n_pb         host [n_q], each in [1, 16384]
 *   n_omega      number of imaginary frequencies, in [1, 16]
 *   omega        host [n_omega], omega_l in Ry, finite and >= 0 (sign is irrelevant: Pi(w) = Pi(-w))
 *   spin_factor  s in the formula above (2 for a spin-degenerate system), finite
 *   prec         arithmetic of the chi0 assembly
 *   cuda_stream  cudaStream_t all work is ordered on (NULL = legacy default stream)
 * Allocates the accumulators (zeroed); returns QSGW_ERR_NOMEM if they do not fit. */
qsgw_status qsgw_chi0_init(qsgw_ctx **ctx, int n_q, const int *n_pb, int n_omega, const double *omega,
                           double spin_factor, qsgw_prec prec, void *cuda_stream);

/* Add one block of transition columns, normally one k-point, to chi0(q) (the k / n / n'
 * sums of Eq. (polfx); Alg. 1 accumulates Im Pi per k-point and batch of n').
 *   Z          device or host, complex128, column-major n_pb[q] x (n_occ*n_unocc) with leading
 *              dimension ldz >= n_pb[q]; column r = n*n_unocc + m holds z_{I, k n m}
 *              (unoccupied index fastest, as the paper's Z(1:n_pb, n', n))
 *   eps_occ    device or host [n_occ], eps_unocc device or host [n_unocc], Ry
 *   n_omega, omega  must equal the grid given to qsgw_chi0_init (host), else QSGW_ERR_ARG
 * Columns with Delta <= 0 or non-finite contribute nothing and set QSGW_ERR_DOMAIN (sticky).
 * The result does not depend on how columns are split across calls, up to rounding.
 * Host arrays are copied into one of two device staging slots the context owns (allocated on
 * first use, grown when a larger block arrives). Outside stream capture the copies run on an
 * internal copy stream, so they overlap the kernels of the previous call; they are NOT
 * ordered after earlier work queued on cuda_stream, so host arrays must hold their data when
 * the call is made. Host eps arrays are read during the call (through a pinned buffer of the
 * context); a host Z in pinned memory must stay unchanged until qsgw_chi0_sync or
 * qsgw_chi0_finalize, one in pageable memory is read before the call returns. */
qsgw_status qsgw_chi0_accumulate(qsgw_ctx *ctx, int q, const void *Z, long long ldz, int n_occ, int n_unocc,
                                 const double *eps_occ, const double *eps_unocc, int n_omega, const double *omega);

/* Same as qsgw_chi0_accumulate with Z in complex64 (interleaved FP32 re, im; same layout, ldz
 * in elements), for QSGW_MIXED_F16X3 contexts only (QSGW_ERR_ARG otherwise). The mixed path
 * rounds every element of Z to FP32 before it forms digits, so the result is bit-identical to
 * qsgw_chi0_accumulate on the complex128 data that rounds to this Z. It moves half the bytes
 * (host staging and HBM reads). The paper's mixed precision likewise holds Z in single
 * precision; eps and W stay FP64. */
qsgw_status qsgw_chi0_accumulate_c64(qsgw_ctx *ctx, int q, const void *Z, long long ldz, int n_occ, int n_unocc,
                                     const double *eps_occ, const double *eps_unocc, int n_omega,
                                     const double *omega);

/* One block of transition columns (normally one k-point) for one q-point; see
 * qsgw_chi0_accumulate for the meaning and layout of every field. All pointers device. */
typedef struct {
  int q;
  const void *Z;
  long long ldz;
  int n_occ, n_unocc;
  const double *eps_occ;
  const double *eps_unocc;
} qsgw_block;

/* Batched form of qsgw_chi0_accumulate over independent q-points (Alg. 1 loops over q). The
 * blocks must name distinct q (QSGW_ERR_ARG otherwise), at most 32 per call, all pointers on the
 * device. In QSGW_MIXED_F16X3 every block's operands are prepared and then ONE persistent
 * tensor-core launch works through all (block, tile, chunk) items, balanced over the SMs, so
 * uneven n_pb and column counts share the GPU; in QSGW_FP64 ONE launch of the FP64 kernel covers
 * all (block, tile, K-slice) items, each block cut into the slices the one-block call would use,
 * so its result is bitwise that of qsgw_chi0_accumulate on the block alone.
 * The first call with a new set of shapes allocates scratch and tile lists; after such a warm-up
 * call the sequence contains only kernel launches and can be captured in a CUDA graph. */
qsgw_status qsgw_chi0_accumulate_batch(qsgw_ctx *ctx, int n_blocks, const qsgw_block *blocks);

/* ---- tile plans and the autotuner (Alg. 1 QKM blocks; the batching pattern of the mixed path) ----
 * A tile plan of the tensor-core launch: J columns per output tile (0 = the widest one allowed,
 * with N = tile_cols * n_omega <= 256 and a multiple of 16) and the number of chunk-range pieces
 * each tile of a partial last wave is cut into (0 = enough pieces to fill the SMs, capped by the
 * block's chunk count; 1 = not cut). Every plan gives the same result up to the order of the
 * double-float additions (chunks are exact FP32 sums in every plan). */
typedef struct {
  int tile_cols;
  int tail_pieces;
} qsgw_tile_plan;

/* The tuner's candidates for n_omega frequencies: the three widest valid tile widths, each with
 * the default tail cut and with none. Writes at most max_out plans; returns how many. */
int qsgw_tile_plan_candidates(int n_omega, qsgw_tile_plan *out, int max_out);

/* Time every candidate plan on these blocks (as for qsgw_chi0_accumulate_batch: distinct q, device
 * pointers) with CUDA events, reps launches each after one warm-up launch, into scratch
 * accumulators of the blocks' sizes that are allocated for the call and freed after it, so the
 * context's chi0 is untouched. The fastest plan is kept for the blocks' size class (n_omega, log2
 * of the blocks' total 64 x 64 output-tile area, log2 of their largest chunk count of 1024
 * columns), and later mixed accumulate calls of that class use it. When the environment variable
 * QSGW_TUNE_CACHE names a file, the choice is appended to it, and qsgw_chi0_init of a mixed
 * context reads the plans back from it. chosen and ms_chosen (nullable) receive the plan and its
 * time per launch. QSGW_MIXED_F16X3 chi0 contexts only (QSGW_ERR_STATE otherwise); QSGW_ERR_NOMEM
 * if the scratch accumulators do not fit. Synchronises the stream. */
qsgw_status qsgw_chi0_autotune(qsgw_ctx *ctx, int n_blocks, const qsgw_block *blocks, int reps,
                               qsgw_tile_plan *chosen, float *ms_chosen);

/* Use this plan for every later mixed accumulate call of the context (NULL: back to the tuned or
 * default plan). QSGW_ERR_ARG for a tile width the frequency count does not allow. The I^c
 * products keep the default width whatever is set. */
qsgw_status qsgw_chi0_set_tile_plan(qsgw_ctx *ctx, const qsgw_tile_plan *plan);

/* Write chi0(q) (the scaled, mirrored accumulator: full Hermitian, imaginary part of the
 * diagonal exactly zero) into chi0, device complex128 [n_omega][n_pb][n_pb]. Synchronises
 * the stream and returns any sticky device error. The accumulator is kept. */
qsgw_status qsgw_chi0_finalize(qsgw_ctx *ctx, int q, void *chi0);

/* From the current accumulator of q: eps (Eq. dielectricfunction), its inverse in FP64, and W
 * (Eq. screenedcoulomb), or W^c (Eq. wc) when correlation_only != 0, for every frequency. The
 * inverse is a block sweep over 32 x 32 pivot blocks, each factored by Cholesky: the pivot blocks
 * are the Schur complements of the leading blocks, so their Cholesky factors are the diagonal
 * blocks of eps = L L^H, and the cost is that of a Cholesky factorisation plus the inverse from
 * it. All frequencies go through each launch; the context keeps 3 x 32 x n_pb x n_omega complex
 * values of scratch for it.
 *   v         device [n_pb], Coulomb eigenvalues v_I > 0 (diagonal MPB basis, Eq. (eqvcoue))
 *   W         device complex128 [n_omega][n_pb][n_pb], full Hermitian
 *   eps_out   NULL or device complex128, same layout: eps before factorisation
 *   info      host [n_omega]: 0, or j+1 if the j-th Cholesky pivot was not positive; the W of
 *             such a frequency is left unspecified and QSGW_ERR_NOT_PD is returned
 * Synchronises the stream. */
qsgw_status qsgw_eps_inv(qsgw_ctx *ctx, int q, const double *v, void *W, void *eps_out, int correlation_only,
                         int *info);

/* Zero the accumulator of q (start a new chi0(q)). Asynchronous. */
qsgw_status qsgw_chi0_reset(qsgw_ctx *ctx, int q);

/* Wait for all queued work; return and clear any sticky device error. */
qsgw_status qsgw_chi0_sync(qsgw_ctx *ctx);

/* Free everything the context owns. Synchronises first; returns any sticky device error. */
qsgw_status qsgw_chi0_destroy(qsgw_ctx *ctx);

/* Static, human-readable name of a status code. */
const char *qsgw_status_string(qsgw_status s);

/* ---- exchange self-energy, Eq. (sigx) (Sec. 2) --------------------------------------------
 *   Sigma^x_{nm}(q) = - sum_k sum_{n' occ} sum_mu conj(Z^{(q-k)n', qn}_{k mu}) v_mu(k) Z^{(q-k)n', qm}_{k mu}
 * A Hermitian update of the same form as chi0, with the Coulomb eigenvalues v_mu(k) as column
 * weights: the rows/columns are the n_qp states n, m at q, the contraction runs over (k, n', mu).
 * The same tensor-core (or FP64) kernels compute it.
 *
 * Create a context for n_q independent q-points with n_qp[q] states each (1 <= n_qp <= 16384);
 * prec as for qsgw_chi0_init (QSGW_MIXED_F16X3: <= 1e-6 relative error). qsgw_chi0_finalize
 * then writes Sigma^x (device complex128 [n_qp][n_qp], column-major, full Hermitian, negative
 * semidefinite); qsgw_chi0_reset / sync / destroy apply. The chi0-only calls
 * (qsgw_chi0_accumulate*, qsgw_eps_inv, qsgw_chi0_accumulate_batch / _synthetic) return
 * QSGW_ERR_STATE on such a context, and qsgw_sigx_accumulate* does on a chi0 context. */
qsgw_status qsgw_sigx_init(qsgw_ctx **ctx, int n_q, const int *n_qp, qsgw_prec prec, void *cuda_stream);

/* Add one k-point (or any block of occupied states n') to Sigma^x(q).
 *   Z      device or host, complex128, column-major n_qp[q] x (n_occ * n_pb) with leading
 *          dimension ldz >= n_qp[q]; column r = n' * n_pb + mu holds Z^{(q-k)n', qn}_{k mu} for
 *          n = 0 .. n_qp-1 (mu fastest)
 *   v      device or host [n_pb], v_mu(k) > 0 and finite, else QSGW_ERR_DOMAIN (sticky; those
 *          columns contribute nothing)
 * Host arrays follow the same rules as in qsgw_chi0_accumulate. */
qsgw_status qsgw_sigx_accumulate(qsgw_ctx *ctx, int q, const void *Z, long long ldz, int n_occ, int n_pb,
                                 const double *v);
/* Same with Z in complex64 (QSGW_MIXED_F16X3 contexts only; bit-identical to complex128 input
 * that rounds to this Z, as for qsgw_chi0_accumulate_c64). */
qsgw_status qsgw_sigx_accumulate_c64(qsgw_ctx *ctx, int q, const void *Z, long long ldz, int n_occ, int n_pb,
                                     const double *v);

/* ---- real-axis route, Eqs. (impolf) and (hilbert) (Sec. 2) ------------------------------------
 * The paper's own route to chi0: the spectral weight of every histogram bin [edges[j], edges[j+1])
 * of transition energies,
 *   S_j(I, J) = sum over columns r = (k, n, m) with Delta_r in bin j of conj(z_{I,r}) z_{J,r},
 * so that on the real axis Im chi0(w) = -pi s S_j / (edges[j+1] - edges[j]) inside bin j, and the
 * Hermitian part follows by the Hilbert transformation, Eq. (hilbert). Each column carries weight
 * 1 into the bin holding its Delta (the paper spreads it with tetrahedron weights, which need a
 * k-mesh), and the density is taken uniform inside a bin, so the Hilbert weight of bin j at w is
 * (1/(R-L)) ln(|w-L| (w+L) / (|w-R| (w+R))) with L, R its edges. The spin factor s is left to
 * the caller.
 *
 * Create a context for one q-point: n_pb in [1, 16384]; n_bins in [1, 4096]; edges host
 * [n_bins + 1], finite, strictly increasing, edges[0] > 0; prec as for qsgw_chi0_init. It holds
 * one accumulator per bin and a staging area per bin for the columns of many accumulate calls:
 * 4096 columns of n_pb values per bin (complex64 in the mixed precision, complex128 in FP64), fewer
 * (a multiple of 16, at least 16) where that would exceed 16 GiB in all. QSGW_ERR_NOMEM if the
 * device cannot hold them. qsgw_chi0_reset(ctx, j) clears bin j, its staged columns included;
 * sync / destroy apply; the other chi0 calls return QSGW_ERR_STATE. */
qsgw_status qsgw_spectral_init(qsgw_ctx **ctx, int n_pb, int n_bins, const double *edges, qsgw_prec prec,
                               void *cuda_stream);

/* Add one block of transition columns (normally one k-point): Z, ldz, n_occ, n_unocc, eps_occ,
 * eps_unocc as in qsgw_chi0_accumulate, all on the device. The columns are put in bins by Delta
 * and gathered bin by bin (a stable counting sort) into the bins' staging. A bin whose staging
 * cannot take its new columns is first accumulated over the staged ones by the chi0 kernels with
 * weight 1 (a bin with more new columns than its staging holds is accumulated over them at once),
 * so the tensor-core kernel sees whole 1024-column chunks rather than the few columns one call
 * puts in a bin. Columns outside every bin contribute
 * nothing; Delta <= 0 or non-finite sets QSGW_ERR_DOMAIN (sticky). Synchronises once (bin
 * counts). */
qsgw_status qsgw_spectral_accumulate(qsgw_ctx *ctx, const void *Z, long long ldz, int n_occ, int n_unocc,
                                     const double *eps_occ, const double *eps_unocc);

/* Accumulate every bin over its staged columns, then write S_j for every bin: device complex128
 * [n_bins][n_pb][n_pb], column-major, full Hermitian, positive semidefinite. Accumulation may go
 * on afterwards. Synchronises and returns any sticky device error. */
qsgw_status qsgw_spectral_finalize(qsgw_ctx *ctx, void *S);

/* chi0 on the real axis (without s) at the centres w_o of the bins bins_out[o] (host [n_out],
 * each in [0, n_bins)), from S as written by qsgw_spectral_finalize (device):
 *   out[o] = sum_j K_j(w_o) S_j + i (-pi / (R - L)) S_{bins_out[o]},
 * device complex128 [n_out][n_pb][n_pb]. One FP64 kernel sums the bins in increasing j for every
 * element on or above the diagonal, adds the anti-Hermitian part and writes the mirror (S_j must
 * be exactly Hermitian, as qsgw_spectral_finalize writes it). Synchronises. */
qsgw_status qsgw_spectral_real_axis(qsgw_ctx *ctx, const void *S, int n_out, const int *bins_out, void *out);

/* ---- imaginary-axis correlation self-energy, Eq. (sigci) (Sec. 2) -------------------------------
 * The part of the correlation self-energy from the imaginary-axis contour:
 *   I_nm = - sum_k sum_{n'} sum_i w_i(e_qn - e_{q-k n'})
 *            sum_{mu, nu} conj(Z_{k, n' n, mu}) W^c_{mu nu}(k, i omega_i) Z_{k, n' m, nu}.
 * The paper takes the weights w_i from the cited method of Aryasetiawan and Gunnarsson without
 * stating it. Here dE/(dE^2 + w^2) is integrated exactly against W^c interpolated on the mesh:
 * constant below omega_0, linear between mesh points, decaying as 1/w^2 beyond the last. The
 * weights are odd in dE and 0 at dE = 0. Both contractions run on the chi0 kernels as blocks of
 * Hermitian updates: first D = sum_i w_i conj(Z) W^c_i, then D Z^T. In the mixed precision they
 * run on the tensor cores; the error is bounded relative to the sum of the terms' magnitudes, as
 * for chi0.
 *
 * Create a context for one q-point:
 *   n_qp target states, in [1, 4096];
 *   n_pb in [1, 8192];
 *   omega: host [n_omega], n_omega <= 16, finite, strictly increasing, omega[0] > 0 (the
 *     frequencies W^c is given at);
 *   prec as for qsgw_chi0_init.
 * qsgw_chi0_reset(ctx, 0) clears the sum; sync / destroy apply; the other chi0 calls return
 * QSGW_ERR_STATE. */
qsgw_status qsgw_sigc_init(qsgw_ctx **ctx, int n_qp, int n_pb, int n_omega, const double *omega, qsgw_prec prec,
                           void *cuda_stream);

/* Add one k-point. All arrays are on the device:
 *   Z: complex128, column-major n_pb x (n_band * n_qp), leading dimension ldz >= n_pb; column
 *     r = n' * n_qp + n holds Z^{(q-k) n', q n}_{k mu};
 *   e_qp: [n_qp], the energies e_qn of the target states (the same in every call);
 *   e_band: [n_band], the energies e_{q-k n'} of the bands n';
 *   Wc: complex128 [n_omega][n_pb][n_pb], column-major per frequency, Hermitian, as
 *     qsgw_eps_inv writes W^c (column mu is read, and W^c_{mu nu} taken as conj(W^c_{nu mu})).
 * Bands go in batches of 4096 / n_qp. The work is queued on the context's stream, and the inputs
 * must stay valid until it has run. Non-finite energies set QSGW_ERR_DOMAIN (sticky). */
qsgw_status qsgw_sigc_accumulate(qsgw_ctx *ctx, const void *Z, long long ldz, int n_band, const double *e_qp,
                                 const double *e_band, const void *Wc);

/* Write I^c to I: device complex128 n_qp x n_qp, column-major, element (n, m) at m * n_qp + n.
 * It is not Hermitian in general: the weights depend on the row's energy e_qn. Synchronises and
 * returns any sticky device error. */
qsgw_status qsgw_sigc_finalize(qsgw_ctx *ctx, void *I);

/* ---- diagnostics (no counterpart in the paper) ---------------------------------------------
 * Exercises the bounded device-side wait that every pipeline barrier of the tensor-core kernel
 * uses: one thread waits on an mbarrier phase that nothing completes and gives up after
 * limit_seconds (1e-3 .. 2, else QSGW_ERR_ARG). The expected result is QSGW_ERR_TIMEOUT; QSGW_OK
 * would mean the wait returned without timing out. Synchronises cuda_stream (NULL = legacy
 * default stream); no GPU fault or hang is involved, and the device stays usable afterwards. */
qsgw_status qsgw_selftest_wait_timeout(double limit_seconds, void *cuda_stream);

/* ---- allocation-free form (no counterpart in the paper) --------------------------------
 * chi0 of ONE block of transition columns, computed in mixed precision exactly as
 * qsgw_chi0_accumulate + qsgw_chi0_finalize would on a fresh context, but without allocating
 * any device memory: every intermediate (digit planes, weights, tile list, accumulators, error
 * flag) lives in one fixed 128 MiB array in the library's device image. It is for callers that
 * cannot call cudaMalloc: code whose device memory is entirely reserved by another allocator
 * (a framework's caching pool or a fixed arena), code that must not risk the implicit device
 * synchronisation cudaMalloc/cudaFree may cause, and code paths that are not allowed to fail on
 * an allocation at run time. Every GPU that loads the library holds the array until exit.
 *   Z, eps_occ, eps_unocc  device; same meaning and layout as in qsgw_chi0_accumulate
 *   n_omega, omega         host, as in qsgw_chi0_init (1..16 frequencies, omega_l >= 0)
 *   spin_factor            s of the formula at the top of this file
 *   chi0                   device complex128 [n_omega][n_pb][n_pb], overwritten with the full
 *                          Hermitian chi0 of this block
 *   cuda_stream            stream the work is ordered on; the call synchronises it at the end to
 *                          return device-detected errors (QSGW_ERR_DOMAIN, QSGW_ERR_TIMEOUT)
 * Sizes whose intermediates do not fit the fixed array return QSGW_ERR_ARG (use the context
 * API instead). The columns go through the array one chunk of 1024 at a time, so their number
 * does not count: n_pb <= 256 always fits, with any n_occ * n_unocc. The space left after the
 * accumulators and one chunk's digit planes holds one flush area per CTA, and the tensor-core grid
 * is capped at the CTAs it has room for (about 90 at n_pb = 256 with 16 frequencies, the SM count for
 * smaller blocks). Every call looks
 * up the array's device address in the current context (and sets the kernel's shared-memory
 * limit there), so the call stays valid after the context is reset. All calls share the one
 * array: calls whose GPU work overlaps (other streams, other host threads) race and must not be
 * issued. */
qsgw_status qsgw_chi0_block_noalloc(const void *Z, long long ldz, int n_pb, int n_occ, int n_unocc,
                                    const double *eps_occ, const double *eps_unocc, int n_omega,
                                    const double *omega, double spin_factor, void *chi0, void *cuda_stream);

/* ---- synthetic inputs (not part of the paper's method) --------------------------------
 * The paper's Z comes from PMT eigenfunctions (Eq. (defz)), which are not available. These
 * entry points draw Z on the device from Philox4x32-10 with the same counter layout as the
 * host-side generator used by the tests:
 *   key = (seed, (gen_q << 8) | 0), counter = (k, n, m, I);
 *   u1 = ((w0 << 21 | w1 >> 11) + 1) * 2^-53, u2 = (w2 << 21 | w3 >> 11) * 2^-53;
 *   z = sqrt(-ln u1) (cos 2 pi u2 + i sin 2 pi u2) / (1 + I / s_div). */

/* Fill Z (device complex128, column-major n_pb x (n_occ*n_unocc), leading dimension ldz)
 * with the synthetic Z of k-point k. Asynchronous on `cuda_stream`. */
qsgw_status qsgw_synth_z(unsigned long long seed, int gen_q, int k, int n_pb, int n_occ, int n_unocc, double s_div,
                         void *Z, long long ldz, void *cuda_stream);

/* Accumulate k-points k_begin..k_end-1 of the synthetic Z into chi0(q) without ever storing
 * the whole Z: each k-point is drawn into context-owned device scratch, then accumulated.
 *   eps_occ    device [k_end-k_begin][n_occ]
 *   eps_unocc  device, the per-k blocks concatenated; block i has n_unocc_per_k[i] entries
 *   n_unocc_per_k  host [k_end-k_begin] */
qsgw_status qsgw_chi0_accumulate_synthetic(qsgw_ctx *ctx, int q, unsigned long long seed, int gen_q, int k_begin,
                                           int k_end, int n_occ, const int *n_unocc_per_k, const double *eps_occ,
                                           const double *eps_unocc, double s_div);

#ifdef __cplusplus
}
#endif
#endif /* QSGW_H */
