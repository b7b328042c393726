// C ABI (include/qsgw.h): context, argument validation, host staging, stream ordering, and the
// eps -> eps^{-1} -> W sequence (FP64 block sweep with Cholesky pivots, all frequencies per launch).
// Also the host side of Sigma^x (given column weights), of the real-axis route (binning,
// per-bin staging and flushes, the Hilbert weights) and of I^c (band batches of the two
// stacked products).
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>
#include <vector>

#include "internal.cuh"
#include "mixed.cuh"

using namespace qsgw;

struct QAcc {
  int n_pb = 0;
  int n_pad = 0;
  void* acc = nullptr;  // FP64: double2 [L][n_pad][n_pad]; mixed: 2 copies of float2 (hi, lo) [L][re|im][n_pad][n_pad]
  size_t bytes = 0;
};

struct qsgw_ctx {
  int device = 0;
  int n_q = 0;
  OmegaGrid g{};
  double omega[kMaxOmega] = {};
  double spin = 2.0;
  qsgw_prec prec = QSGW_FP64;
  bool sigx = false;  // exchange self-energy context (qsgw_sigx_init): given weights, one weight set
  // real-axis route (qsgw_spectral_init): one accumulator ("q") per histogram bin of Delta
  bool spectral = false;
  int n_bins = 0;
  std::vector<double> edges;  // host [n_bins + 1]
  double* d_edges = nullptr;
  double* d_one = nullptr;  // the weight 1 of every column
  int* d_offsets = nullptr;  // [n_bins + 1] (counts first, then exclusive offsets)
  int* d_counts = nullptr;
  void* d_bins = nullptr;
  size_t bins_cap = 0;
  void* d_perm = nullptr;
  size_t perm_cap = 0;
  void* d_zsort = nullptr;  // the columns of bins that overflow their staging in one call
  size_t zsort_cap = 0;
  // per-bin staging: stage_cols columns of n_pb values per bin (complex64 in the mixed precision,
  // complex128 in FP64), filled over accumulate calls and flushed as one update per bin
  void* d_stage = nullptr;
  int stage_cols = 0;
  std::vector<int> fill;       // columns staged per bin
  void** d_dptr = nullptr;     // [n_bins] gather destinations of one call
  std::vector<void*> h_dptr;
  // imaginary-axis correlation self-energy (qsgw_sigc_init): q[0] accumulates the product
  // D Z^T of the stacked operand [conj(D); Z] (rows 0..n_qp and Y3..Y3+n_qp), q[1] the product
  // D of [w conj(Z); W^c] for one batch of bands (rows 0..M and Y0..Y0+n_pb)
  bool sigc = false;
  SigcMesh smesh{};
  int sc_nqp = 0, sc_npb = 0, sc_nbb = 0, sc_Y3 = 0;
  void* d_wsc = nullptr;  // integration weights of one call
  size_t wsc_cap = 0;
  void* d_zt = nullptr;  // a batch of Z, transposed
  size_t zt_cap = 0;
  void* d_z2 = nullptr;  // stacked operand of D
  size_t z2_cap = 0;
  void* d_z3 = nullptr;  // stacked operand of I
  size_t z3_cap = 0;
  cudaStream_t stream = nullptr;
  std::vector<QAcc> q;
  int* d_err = nullptr;
  // scratch, grown on demand
  double* d_w = nullptr;
  size_t w_cap = 0;  // doubles
  void* d_part = nullptr;  // FP64 HERK split-K partials
  size_t part_cap = 0;     // bytes
  void* d_zstage = nullptr;
  size_t zstage_cap = 0;  // bytes
  // host operands: two staging slots filled on a copy stream, so the copies of one block
  // overlap the kernels of the previous one
  void* d_hstage[2] = {};     // Z
  size_t hstage_cap[2] = {};  // bytes
  double* d_es[2] = {};       // eps_occ, eps_unocc
  size_t es_cap[2] = {};      // bytes
  double* h_eb[2] = {};       // pinned bounce buffers for host eps
  size_t eb_cap[2] = {};      // bytes
  cudaStream_t cstream = nullptr;
  cudaEvent_t hcopied[2] = {};  // slot filled (recorded on cstream)
  cudaEvent_t hfree[2] = {};    // last reader of the slot done (recorded on stream)
  int hslot = 0;
  MixedScratch mixed;
  // eps^{-1} scratch: the pivot inverses [L][32][32] and the panel buffers P, C [L][32][n_pb]
  void* d_sbuf = nullptr;
  size_t sbuf_cap = 0;
  void* d_pbuf = nullptr;
  size_t pbuf_cap = 0;
  void* d_cbuf = nullptr;
  size_t cbuf_cap = 0;
  void* d_dig = nullptr;  // digit images of the update on the tensor cores (mixed contexts)
  size_t dig_cap = 0;
  int* d_info = nullptr;
};

namespace {

qsgw_status cuda_status(cudaError_t e) {
  if (e == cudaSuccess) return QSGW_OK;
  if (e == cudaErrorMemoryAllocation) return QSGW_ERR_NOMEM;
  return QSGW_ERR_CUDA;
}

#define QSGW_CK(expr)                                   \
  do {                                                  \
    cudaError_t e_ = (expr);                            \
    if (e_ != cudaSuccess) return cuda_status(e_);      \
  } while (0)

bool is_device_ptr(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

qsgw_status grow(void** p, size_t* cap, size_t need_bytes) {
  if (*cap >= need_bytes) return QSGW_OK;
  if (*p) cudaFree(*p);
  *p = nullptr;
  *cap = 0;
  QSGW_CK(cudaMalloc(p, need_bytes));
  *cap = need_bytes;
  return QSGW_OK;
}

// Pinned host buffer of at least need_bytes (the caller has made sure no copy still reads it).
qsgw_status grow_pinned(void** p, size_t* cap, size_t need_bytes) {
  if (*cap >= need_bytes) return QSGW_OK;
  if (*p) cudaFreeHost(*p);
  *p = nullptr;
  *cap = 0;
  if (cudaMallocHost(p, need_bytes) != cudaSuccess) {
    cudaGetLastError();
    *p = nullptr;
    return QSGW_ERR_NOMEM;
  }
  *cap = need_bytes;
  return QSGW_OK;
}

// Read and clear the sticky device error (synchronises the stream).
qsgw_status take_device_error(qsgw_ctx* c) {
  QSGW_CK(cudaStreamSynchronize(c->stream));
  int h = 0;
  QSGW_CK(cudaMemcpy(&h, c->d_err, sizeof(int), cudaMemcpyDeviceToHost));
  if (h != DEV_OK) {
    QSGW_CK(cudaMemset(c->d_err, 0, sizeof(int)));
    return h == DEV_DOMAIN ? QSGW_ERR_DOMAIN : QSGW_ERR_TIMEOUT;
  }
  return QSGW_OK;
}

void load_plans(qsgw_ctx* c);  // tuned tile plans from the plan file (defined with the autotuner calls)

qsgw_status check_grid(const qsgw_ctx* c, int n_omega, const double* omega) {
  if (n_omega != c->g.L || !omega) return QSGW_ERR_ARG;
  for (int l = 0; l < n_omega; ++l)
    if (std::memcmp(&omega[l], &c->omega[l], sizeof(double)) != 0) return QSGW_ERR_ARG;
  return QSGW_OK;
}

// Core of accumulate once every pointer is on the device. z32: Z holds complex64 (mixed only).
// wv: given weights w_r = wv[r mod n_unocc] (exchange self-energy contexts) instead of Delta.
qsgw_status accumulate_device(qsgw_ctx* c, int q, const void* Z, bool z32, long long ldz, int n_occ, int n_unocc,
                              const double* eo, const double* eu, const double* wv = nullptr) {
  QAcc& a = c->q[q];
  const long long K = (long long)n_occ * n_unocc;
  if (c->prec == QSGW_FP64) {
    if (z32) return QSGW_ERR_ARG;
    qsgw_status st = grow(reinterpret_cast<void**>(&c->d_w), &c->w_cap, sizeof(double) * (size_t)K * c->g.L);
    if (st != QSGW_OK) return st;
    if (wv)
      launch_weights_given_fp64(wv, n_unocc, K, c->d_w, c->d_err, c->stream);
    else
      launch_weights_fp64(eo, eu, n_occ, n_unocc, c->g, c->d_w, K, c->d_err, c->stream);
    const int S = herk_fp64_slices(a.n_pad, c->g.L, K);
    if (S > 1) {
      st = grow(&c->d_part, &c->part_cap, sizeof(double2) * (size_t)S * c->g.L * a.n_pad * a.n_pad);
      if (st != QSGW_OK) return st;
    }
    launch_herk_fp64(static_cast<const double2*>(Z), ldz, a.n_pb, a.n_pad, K, c->d_w, K, c->g.L, S,
                     static_cast<double2*>(a.acc), static_cast<double2*>(c->d_part), c->stream);
  } else {
    qsgw_status st = mixed_accumulate(c->mixed, Z, z32, ldz, a.n_pb, a.n_pad, n_occ, n_unocc, eo, eu, wv, c->g,
                                      static_cast<float4*>(a.acc), c->d_err, c->stream);
    if (st != QSGW_OK) return st;
  }
  return cuda_status(cudaGetLastError());
}

}  // namespace

extern "C" {

const char* qsgw_status_string(qsgw_status s) {
  switch (s) {
    case QSGW_OK: return "QSGW_OK";
    case QSGW_ERR_ARG: return "QSGW_ERR_ARG: invalid argument";
    case QSGW_ERR_DOMAIN: return "QSGW_ERR_DOMAIN: a transition energy Delta <= 0 or non-finite";
    case QSGW_ERR_NOMEM: return "QSGW_ERR_NOMEM: device allocation failed";
    case QSGW_ERR_CUDA: return "QSGW_ERR_CUDA: CUDA runtime or library error";
    case QSGW_ERR_NOT_PD: return "QSGW_ERR_NOT_PD: eps not positive definite at some frequency";
    case QSGW_ERR_TIMEOUT: return "QSGW_ERR_TIMEOUT: a bounded device wait gave up";
    case QSGW_ERR_STATE: return "QSGW_ERR_STATE: call not valid in this state";
  }
  return "QSGW: unknown status";
}

qsgw_status qsgw_chi0_init(qsgw_ctx** out, int n_q, const int* n_pb, int n_omega, const double* omega,
                           double spin_factor, qsgw_prec prec, void* cuda_stream) {
  if (!out) return QSGW_ERR_ARG;
  *out = nullptr;
  if (n_q < 1 || !n_pb || n_omega < 1 || n_omega > kMaxOmega || !omega || !std::isfinite(spin_factor))
    return QSGW_ERR_ARG;
  if (prec != QSGW_FP64 && prec != QSGW_MIXED_F16X3) return QSGW_ERR_ARG;
  for (int i = 0; i < n_q; ++i)
    if (n_pb[i] < 1 || n_pb[i] > kMaxNpb) return QSGW_ERR_ARG;
  for (int l = 0; l < n_omega; ++l)
    if (!std::isfinite(omega[l]) || omega[l] < 0.0) return QSGW_ERR_ARG;

  qsgw_ctx* c = new (std::nothrow) qsgw_ctx();
  if (!c) return QSGW_ERR_NOMEM;
  c->n_q = n_q;
  c->spin = spin_factor;
  c->prec = prec;
  c->stream = static_cast<cudaStream_t>(cuda_stream);
  c->g.L = n_omega;
  for (int l = 0; l < n_omega; ++l) {
    c->omega[l] = omega[l];
    c->g.w2[l] = omega[l] * omega[l];
    c->g.w2f[l] = (float)(omega[l] * omega[l]);
  }
  qsgw_status st = QSGW_OK;
  cudaError_t e = cudaGetDevice(&c->device);
  if (e == cudaSuccess) e = cudaMalloc(&c->d_err, sizeof(int));
  if (e == cudaSuccess) e = cudaMemsetAsync(c->d_err, 0, sizeof(int), c->stream);
  if (e != cudaSuccess) st = cuda_status(e);
  c->q.resize(n_q);
  for (int i = 0; i < n_q && st == QSGW_OK; ++i) {
    QAcc& a = c->q[i];
    a.n_pb = n_pb[i];
    a.n_pad = pad_to(n_pb[i], kPad);
    // mixed: two double-float copies (see herk_mixed_kernel's persistent schedule)
    a.bytes = (size_t)a.n_pad * a.n_pad * n_omega * (prec == QSGW_FP64 ? sizeof(double2) : 2 * sizeof(float4));
    e = cudaMalloc(&a.acc, a.bytes);
    if (e == cudaSuccess) e = cudaMemsetAsync(a.acc, 0, a.bytes, c->stream);
    if (e != cudaSuccess) st = cuda_status(e);
  }
  if (st == QSGW_OK) st = cuda_status(cudaStreamSynchronize(c->stream));
  if (st != QSGW_OK) {
    qsgw_chi0_destroy(c);
    return st;
  }
  if (prec == QSGW_MIXED_F16X3) load_plans(c);
  *out = c;
  return QSGW_OK;
}

}  // extern "C"

namespace {
// qsgw_chi0_accumulate(_c64) and qsgw_sigx_accumulate(_c64): z32 selects complex64 Z. For an
// exchange self-energy context (c->sigx) the columns are (n', mu) with given weights
// eps_unocc[mu] = v_mu (n_unocc = n_pb of the k-point) and eps_occ is unused.
qsgw_status accumulate_any(qsgw_ctx* c, int q, const void* Z, bool z32, long long ldz, int n_occ, int n_unocc,
                           const double* eps_occ, const double* eps_unocc, int n_omega, const double* omega) {
  const bool sx = c && c->sigx;
  if (!c || q < 0 || q >= c->n_q || !Z || (!sx && !eps_occ) || !eps_unocc) return QSGW_ERR_ARG;
  if (z32 && c->prec != QSGW_MIXED_F16X3) return QSGW_ERR_ARG;
  const QAcc& a = c->q[q];
  if (ldz < a.n_pb || n_occ < 1 || n_unocc < 1) return QSGW_ERR_ARG;
  if ((long long)n_occ * n_unocc > (1LL << 31)) return QSGW_ERR_ARG;
  qsgw_status st = sx ? QSGW_OK : check_grid(c, n_omega, omega);
  if (st != QSGW_OK) return st;
  const long long K = (long long)n_occ * n_unocc;
  const double* wv = sx ? eps_unocc : nullptr;
  if (sx) eps_occ = nullptr;

  const bool z_dev = is_device_ptr(Z);
  const bool e_dev = (sx || is_device_ptr(eps_occ)) && is_device_ptr(eps_unocc);
  if (z_dev && e_dev)
    return sx ? accumulate_device(c, q, Z, z32, ldz, n_occ, n_unocc, nullptr, nullptr, wv)
              : accumulate_device(c, q, Z, z32, ldz, n_occ, n_unocc, eps_occ, eps_unocc);

  // Host operands go through the next of two staging slots. Outside stream capture their copies
  // run on the context's copy stream, after the kernels that last read that slot but not after
  // the rest of the queued work, so they overlap the previous call's kernels. Host eps pass
  // through a pinned bounce buffer, so no copy from pageable memory is queued (such a copy may
  // hold the caller until the stream reaches it, which would serialise the calls). Under stream
  // capture the copies stay on the captured stream and read the caller's arrays directly.
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  QSGW_CK(cudaStreamIsCapturing(c->stream, &cap));
  const bool capturing = cap != cudaStreamCaptureStatusNone;
  if (!c->cstream) {
    QSGW_CK(cudaStreamCreateWithFlags(&c->cstream, cudaStreamNonBlocking));
    for (int i = 0; i < 2; ++i) {
      QSGW_CK(cudaEventCreateWithFlags(&c->hcopied[i], cudaEventDisableTiming));
      QSGW_CK(cudaEventCreateWithFlags(&c->hfree[i], cudaEventDisableTiming));
    }
  }
  const int s = c->hslot;
  c->hslot ^= 1;
  const size_t zbytes = z_dev ? 0 : (z32 ? sizeof(float2) : sizeof(double2)) * (size_t)ldz * (size_t)K;
  const int n_eo = sx ? 0 : n_occ;  // host eps_occ values staged (none for Sigma^x)
  const size_t ebytes = e_dev ? 0 : sizeof(double) * (size_t)(n_eo + n_unocc);
  if (c->hstage_cap[s] < zbytes || c->es_cap[s] < ebytes || c->eb_cap[s] < ebytes) {
    // the slot is about to be reallocated: nothing may still fill or read it
    QSGW_CK(cudaStreamSynchronize(c->cstream));
    QSGW_CK(cudaStreamSynchronize(c->stream));
  }
  st = grow(&c->d_hstage[s], &c->hstage_cap[s], zbytes);
  if (st == QSGW_OK) st = grow(reinterpret_cast<void**>(&c->d_es[s]), &c->es_cap[s], ebytes);
  if (st == QSGW_OK) st = grow_pinned(reinterpret_cast<void**>(&c->h_eb[s]), &c->eb_cap[s], ebytes);
  if (st != QSGW_OK) return st;

  cudaStream_t cs = capturing ? c->stream : c->cstream;
  if (!capturing) QSGW_CK(cudaStreamWaitEvent(cs, c->hfree[s], 0));
  const double* eo = eps_occ;
  const double* eu = eps_unocc;
  if (!e_dev) {
    const size_t bo = sizeof(double) * (size_t)n_eo, bu = sizeof(double) * (size_t)n_unocc;
    if (!capturing) {
      QSGW_CK(cudaEventSynchronize(c->hcopied[s]));  // the bounce buffer's previous copy is done
      if (bo) std::memcpy(c->h_eb[s], eps_occ, bo);
      std::memcpy(c->h_eb[s] + n_eo, eps_unocc, bu);
      QSGW_CK(cudaMemcpyAsync(c->d_es[s], c->h_eb[s], ebytes, cudaMemcpyHostToDevice, cs));
    } else {
      if (bo) QSGW_CK(cudaMemcpyAsync(c->d_es[s], eps_occ, bo, cudaMemcpyDefault, cs));
      QSGW_CK(cudaMemcpyAsync(c->d_es[s] + n_eo, eps_unocc, bu, cudaMemcpyDefault, cs));
    }
    eo = sx ? nullptr : c->d_es[s];
    eu = c->d_es[s] + n_eo;
  }
  const void* Zd = Z;
  if (!z_dev) {
    QSGW_CK(cudaMemcpyAsync(c->d_hstage[s], Z, zbytes, cudaMemcpyDefault, cs));
    Zd = c->d_hstage[s];
  }
  if (!capturing) {
    QSGW_CK(cudaEventRecord(c->hcopied[s], cs));
    QSGW_CK(cudaStreamWaitEvent(c->stream, c->hcopied[s], 0));
  }
  st = sx ? accumulate_device(c, q, Zd, z32, ldz, n_occ, n_unocc, nullptr, nullptr, eu)
          : accumulate_device(c, q, Zd, z32, ldz, n_occ, n_unocc, eo, eu);
  if (st != QSGW_OK) return st;
  if (!capturing) QSGW_CK(cudaEventRecord(c->hfree[s], c->stream));
  return QSGW_OK;
}

// ---- real-axis route: per-bin staging
constexpr int kStageCols = 4096;              // staged columns per bin (four exact FP32 chunks)
constexpr size_t kStageBudget = 16ull << 30;  // bytes of staging at most; fewer columns per bin beyond

size_t spectral_col_bytes(const qsgw_ctx* c) {
  return (c->prec == QSGW_FP64 ? sizeof(double2) : sizeof(float2)) * (size_t)c->q[0].n_pb;
}

struct BinCols {
  int j;          // bin
  const void* Z;  // its columns, n_pb values each, consecutive
  int cnt;
};

// S_j += sum over the given columns of conj(z_I) z_J (weight 1), for every listed bin: up to 32
// bins per launch of the tensor-core kernel, or one FP64 update per bin.
qsgw_status spectral_update(qsgw_ctx* c, const std::vector<BinCols>& v) {
  const int n_pb = c->q[0].n_pb;
  MixedBlock mb[32];
  int nb = 0;
  for (size_t i = 0; i < v.size(); ++i) {
    const BinCols& x = v[i];
    const QAcc& a = c->q[x.j];
    if (c->prec == QSGW_FP64) {
      qsgw_status st = accumulate_device(c, x.j, x.Z, false, n_pb, x.cnt, 1, nullptr, nullptr, c->d_one);
      if (st != QSGW_OK) return st;
      continue;
    }
    mb[nb++] = MixedBlock{x.Z, n_pb, a.n_pb, a.n_pad, x.cnt, 1, nullptr, nullptr, static_cast<float4*>(a.acc), true,
                          c->d_one};
    if (nb == 32 || i + 1 == v.size()) {
      qsgw_status st = mixed_accumulate_batch(c->mixed, nb, mb, c->g, c->d_err, c->stream);
      if (st != QSGW_OK) return st;
      nb = 0;
    }
  }
  return cuda_status(cudaGetLastError());
}

// Runs the update of every listed bin over its staged columns and empties its staging.
qsgw_status spectral_flush(qsgw_ctx* c, const std::vector<int>& js) {
  const size_t cb = spectral_col_bytes(c);
  std::vector<BinCols> v;
  for (int j : js)
    if (c->fill[j] > 0)
      v.push_back({j, static_cast<uint8_t*>(c->d_stage) + (size_t)j * c->stage_cols * cb, c->fill[j]});
  qsgw_status st = spectral_update(c, v);
  if (st != QSGW_OK) return st;
  for (int j : js) c->fill[j] = 0;
  return QSGW_OK;
}

// ---- imaginary-axis correlation self-energy
constexpr int kSigcRows = 4096;  // rows (band, target) of one batch of the product D
constexpr int kSigcAlign = 256;  // row offset of the second row set: a multiple of the tile width at L = 1

// The product of two row sets of a stacked operand Z (column-major, S rows, K columns): rows I <
// rows_i against rows J >= col0, with weight 1, into accumulator q.
qsgw_status sigc_product(qsgw_ctx* c, int q, const void* Z, int S, long long K, int rows_i, int col0) {
  QAcc& a = c->q[q];
  if (c->prec == QSGW_FP64) {
    qsgw_status st = grow(reinterpret_cast<void**>(&c->d_w), &c->w_cap, sizeof(double) * (size_t)K);
    if (st != QSGW_OK) return st;
    launch_weights_given_fp64(c->d_one, 1, K, c->d_w, c->d_err, c->stream);
    const int ti_end = (rows_i + 63) / 64, tj0 = col0 / 64;
    const int Sl = herk_fp64_slices(a.n_pad, 1, K, ti_end, tj0);
    if (Sl > 1) {
      st = grow(&c->d_part, &c->part_cap, sizeof(double2) * (size_t)Sl * a.n_pad * a.n_pad);
      if (st != QSGW_OK) return st;
    }
    launch_herk_fp64(static_cast<const double2*>(Z), S, S, a.n_pad, K, c->d_w, K, 1, Sl, static_cast<double2*>(a.acc),
                     static_cast<double2*>(c->d_part), c->stream, ti_end, tj0);
    return cuda_status(cudaGetLastError());
  }
  MixedBlock b{Z, S, S, a.n_pad, (int)K, 1, nullptr, nullptr, static_cast<float4*>(a.acc), true, c->d_one};
  b.rows_i = rows_i;
  b.col0 = col0;
  return mixed_accumulate_batch(c->mixed, 1, &b, c->g, c->d_err, c->stream);
}
}  // namespace

extern "C" {

qsgw_status qsgw_chi0_accumulate(qsgw_ctx* c, int q, const void* Z, long long ldz, int n_occ, int n_unocc,
                                 const double* eps_occ, const double* eps_unocc, int n_omega, const double* omega) {
  if (c && (c->sigx || c->spectral || c->sigc)) return QSGW_ERR_STATE;
  return accumulate_any(c, q, Z, false, ldz, n_occ, n_unocc, eps_occ, eps_unocc, n_omega, omega);
}

qsgw_status qsgw_chi0_accumulate_c64(qsgw_ctx* c, int q, const void* Z, long long ldz, int n_occ, int n_unocc,
                                     const double* eps_occ, const double* eps_unocc, int n_omega,
                                     const double* omega) {
  if (c && (c->sigx || c->spectral || c->sigc)) return QSGW_ERR_STATE;
  return accumulate_any(c, q, Z, true, ldz, n_occ, n_unocc, eps_occ, eps_unocc, n_omega, omega);
}

qsgw_status qsgw_sigx_init(qsgw_ctx** ctx, int n_q, const int* n_qp, qsgw_prec prec, void* cuda_stream) {
  const double omega0 = 0.0;  // one weight set; the frequency grid is not used
  qsgw_status st = qsgw_chi0_init(ctx, n_q, n_qp, 1, &omega0, 1.0, prec, cuda_stream);
  if (st == QSGW_OK) (*ctx)->sigx = true;
  return st;
}

qsgw_status qsgw_sigx_accumulate(qsgw_ctx* c, int q, const void* Z, long long ldz, int n_occ, int n_pb,
                                 const double* v) {
  if (!c || !c->sigx) return c ? QSGW_ERR_STATE : QSGW_ERR_ARG;
  return accumulate_any(c, q, Z, false, ldz, n_occ, n_pb, nullptr, v, 0, nullptr);
}

qsgw_status qsgw_sigx_accumulate_c64(qsgw_ctx* c, int q, const void* Z, long long ldz, int n_occ, int n_pb,
                                     const double* v) {
  if (!c || !c->sigx) return c ? QSGW_ERR_STATE : QSGW_ERR_ARG;
  return accumulate_any(c, q, Z, true, ldz, n_occ, n_pb, nullptr, v, 0, nullptr);
}

}  // extern "C"

namespace {
// Checks a batch of blocks (distinct q, device pointers) and describes them for the mixed kernels.
qsgw_status batch_blocks(qsgw_ctx* c, int n_blocks, const qsgw_block* blocks, MixedBlock* mb) {
  if (!c || n_blocks < 1 || n_blocks > 32 || !blocks) return QSGW_ERR_ARG;
  if (c->sigx || c->spectral || c->sigc) return QSGW_ERR_STATE;
  for (int i = 0; i < n_blocks; ++i) {
    const qsgw_block& b = blocks[i];
    if (b.q < 0 || b.q >= c->n_q || !b.Z || !b.eps_occ || !b.eps_unocc || b.n_occ < 1 || b.n_unocc < 1)
      return QSGW_ERR_ARG;
    const QAcc& a = c->q[b.q];
    if (b.ldz < a.n_pb || (long long)b.n_occ * b.n_unocc > (1LL << 31)) return QSGW_ERR_ARG;
    for (int j = 0; j < i; ++j)
      if (blocks[j].q == b.q) return QSGW_ERR_ARG;
    if (!is_device_ptr(b.Z) || !is_device_ptr(b.eps_occ) || !is_device_ptr(b.eps_unocc)) return QSGW_ERR_ARG;
    mb[i] = MixedBlock{b.Z, b.ldz, a.n_pb, a.n_pad, b.n_occ, b.n_unocc, b.eps_occ,
                       b.eps_unocc, static_cast<float4*>(a.acc), /*z32*/ false, /*wv*/ nullptr};
  }
  return QSGW_OK;
}

// Tuned plans persist in a text file named by QSGW_TUNE_CACHE, one line per size class:
// "qsgw-plan <n_omega> <area class> <chunk class> <tile columns> <tail pieces>".
void load_plans(qsgw_ctx* c) {
  const char* path = std::getenv("QSGW_TUNE_CACHE");
  if (!path || !*path) return;
  FILE* f = std::fopen(path, "r");
  if (!f) return;
  char line[256];
  while (std::fgets(line, sizeof(line), f)) {
    PlanEntry e{};
    if (std::sscanf(line, "qsgw-plan %d %d %d %d %d", &e.L, &e.ca, &e.cc, &e.plan.tj, &e.plan.pieces) != 5) continue;
    if (e.L != c->g.L || !mixed_plan_valid(e.L, e.plan)) continue;
    bool found = false;
    for (PlanEntry& x : c->mixed.plans)
      if (x.L == e.L && x.ca == e.ca && x.cc == e.cc) {
        x.plan = e.plan;  // the last line of a class wins
        found = true;
      }
    if (!found) c->mixed.plans.push_back(e);
  }
  std::fclose(f);
}

void save_plan(int L, int ca, int cc, const TilePlan& p) {
  const char* path = std::getenv("QSGW_TUNE_CACHE");
  if (!path || !*path) return;
  FILE* f = std::fopen(path, "a");
  if (!f) return;
  std::fprintf(f, "qsgw-plan %d %d %d %d %d\n", L, ca, cc, p.tj, p.pieces);
  std::fclose(f);
}
}  // namespace

extern "C" {

qsgw_status qsgw_chi0_accumulate_batch(qsgw_ctx* c, int n_blocks, const qsgw_block* blocks) {
  MixedBlock mb[32];
  qsgw_status bst = batch_blocks(c, n_blocks, blocks, mb);
  if (bst != QSGW_OK) return bst;
  if (c->prec == QSGW_FP64) {
    // weights of every block, then ONE launch of the FP64 HERK over all (block, tile, slice) items
    const int L = c->g.L;
    size_t w_total = 0, part_total = 0;
    int S[32];
    for (int i = 0; i < n_blocks; ++i) {
      const QAcc& a = c->q[blocks[i].q];
      const long long K = (long long)blocks[i].n_occ * blocks[i].n_unocc;
      S[i] = herk_fp64_slices(a.n_pad, L, K);
      w_total += (size_t)K * L;
      if (S[i] > 1) part_total += (size_t)S[i] * L * a.n_pad * a.n_pad;
    }
    qsgw_status st = grow(reinterpret_cast<void**>(&c->d_w), &c->w_cap, sizeof(double) * w_total);
    if (st == QSGW_OK && part_total) st = grow(&c->d_part, &c->part_cap, sizeof(double2) * part_total);
    if (st != QSGW_OK) return st;
    Fp64Batch fb;
    std::memset(&fb, 0, sizeof(fb));
    fb.nb = n_blocks;
    fb.L = L;
    size_t w_off = 0, p_off = 0;
    for (int i = 0; i < n_blocks; ++i) {
      const qsgw_block& b = blocks[i];
      const QAcc& a = c->q[b.q];
      const long long K = (long long)b.n_occ * b.n_unocc;
      double* w = c->d_w + w_off;
      launch_weights_fp64(b.eps_occ, b.eps_unocc, b.n_occ, b.n_unocc, c->g, w, K, c->d_err, c->stream);
      const int nt = a.n_pad / 64;
      double2* part = S[i] > 1 ? static_cast<double2*>(c->d_part) + p_off : nullptr;
      fb.b[i] = Fp64Blk{static_cast<const double2*>(b.Z), b.ldz, K, w, K, static_cast<double2*>(a.acc), part,
                        a.n_pb, a.n_pad, S[i], fb.items};
      fb.items += nt * (nt + 1) / 2 * S[i];
      w_off += (size_t)K * L;
      if (S[i] > 1) p_off += (size_t)S[i] * L * a.n_pad * a.n_pad;
    }
    launch_herk_fp64_batch(fb, c->stream);
    return cuda_status(cudaGetLastError());
  }
  qsgw_status st = mixed_accumulate_batch(c->mixed, n_blocks, mb, c->g, c->d_err, c->stream);
  if (st != QSGW_OK) return st;
  return cuda_status(cudaGetLastError());
}

int qsgw_tile_plan_candidates(int n_omega, qsgw_tile_plan* out, int max_out) {
  if (!out || max_out < 1) return 0;
  TilePlan cand[16];
  const int n = std::min(mixed_plan_candidates(n_omega, cand, 16), max_out);
  for (int i = 0; i < n; ++i) out[i] = qsgw_tile_plan{cand[i].tj, cand[i].pieces};
  return n;
}

qsgw_status qsgw_chi0_set_tile_plan(qsgw_ctx* c, const qsgw_tile_plan* plan) {
  if (!c) return QSGW_ERR_ARG;
  if (c->prec != QSGW_MIXED_F16X3) return QSGW_ERR_STATE;
  if (!plan) {
    c->mixed.use_forced = false;
    return QSGW_OK;
  }
  const TilePlan p{plan->tile_cols, plan->tail_pieces};
  if (!mixed_plan_valid(c->g.L, p)) return QSGW_ERR_ARG;
  c->mixed.forced = p;
  c->mixed.use_forced = true;
  return QSGW_OK;
}

qsgw_status qsgw_chi0_autotune(qsgw_ctx* c, int n_blocks, const qsgw_block* blocks, int reps,
                               qsgw_tile_plan* chosen, float* ms_chosen) {
  MixedBlock mb[32];
  qsgw_status st = batch_blocks(c, n_blocks, blocks, mb);
  if (st != QSGW_OK) return st;
  if (c->prec != QSGW_MIXED_F16X3) return QSGW_ERR_STATE;
  if (reps < 1 || reps > 100) return QSGW_ERR_ARG;
  TilePlan best;
  float ms = 0.f;
  st = mixed_autotune(c->mixed, n_blocks, mb, c->g, c->d_err, c->stream, reps, &best, &ms);
  if (st != QSGW_OK) return st;
  int ca = 0, cc = 0;
  mixed_plan_class(n_blocks, mb, &ca, &cc);
  save_plan(c->g.L, ca, cc, best);
  if (chosen) *chosen = qsgw_tile_plan{best.tj, best.pieces};
  if (ms_chosen) *ms_chosen = ms;
  return QSGW_OK;
}

qsgw_status qsgw_chi0_finalize(qsgw_ctx* c, int q, void* chi0) {
  if (!c || q < 0 || q >= c->n_q || !chi0) return QSGW_ERR_ARG;
  if (c->spectral || c->sigc) return QSGW_ERR_STATE;  // their own finalize calls read them out
  const QAcc& a = c->q[q];
  launch_finalize_chi(a.acc, c->prec == QSGW_FP64 ? ACC_FP64 : ACC_DF32, a.n_pb, a.n_pad, c->g.L, c->spin,
                      static_cast<double2*>(chi0), c->stream);
  QSGW_CK(cudaGetLastError());
  return take_device_error(c);
}

qsgw_status qsgw_eps_inv(qsgw_ctx* c, int q, const double* v, void* W, void* eps_out, int correlation_only,
                         int* info) {
  if (!c || q < 0 || q >= c->n_q || !v || !W || !info) return QSGW_ERR_ARG;
  if (c->sigx || c->spectral || c->sigc) return QSGW_ERR_STATE;
  const QAcc& a = c->q[q];
  const int n = a.n_pb, L = c->g.L;
  const size_t nn = (size_t)n * n;
  double2* w = static_cast<double2*>(W);
  if (!c->d_info) QSGW_CK(cudaMalloc(&c->d_info, sizeof(int) * kMaxOmega));
  qsgw_status st = grow(&c->d_sbuf, &c->sbuf_cap, sizeof(double2) * 32 * 32 * L);
  if (st == QSGW_OK) st = grow(&c->d_pbuf, &c->pbuf_cap, sizeof(double2) * 32 * (size_t)n * L);
  if (st == QSGW_OK) st = grow(&c->d_cbuf, &c->cbuf_cap, sizeof(double2) * 32 * (size_t)n * L);
  const bool tc = c->prec == QSGW_MIXED_F16X3;  // the update on the tensor cores, at FP64 accuracy
  if (st == QSGW_OK && tc) st = grow(&c->d_dig, &c->dig_cap, eps_inverse_digit_bytes(n, L));
  if (st != QSGW_OK) return st;

  launch_form_eps(a.acc, c->prec == QSGW_FP64 ? ACC_FP64 : ACC_DF32, n, a.n_pad, L, c->spin, v, w, c->stream);
  QSGW_CK(cudaGetLastError());
  if (eps_out) QSGW_CK(cudaMemcpyAsync(eps_out, w, sizeof(double2) * nn * L, cudaMemcpyDeviceToDevice, c->stream));
  QSGW_CK(cudaMemsetAsync(c->d_info, 0, sizeof(int) * kMaxOmega, c->stream));
  launch_eps_inverse(w, n, L, static_cast<double2*>(c->d_sbuf), static_cast<double2*>(c->d_pbuf),
                     static_cast<double2*>(c->d_cbuf), tc ? static_cast<uint8_t*>(c->d_dig) : nullptr, c->d_info,
                     c->d_err, c->stream);
  QSGW_CK(cudaGetLastError());
  launch_w_from_inverse(w, n, L, v, correlation_only, -1.0, c->stream);  // the sweep leaves -eps^{-1}
  QSGW_CK(cudaGetLastError());
  int hinfo[kMaxOmega];
  QSGW_CK(cudaMemcpyAsync(hinfo, c->d_info, sizeof(int) * kMaxOmega, cudaMemcpyDeviceToHost, c->stream));
  st = take_device_error(c);
  if (st != QSGW_OK) return st;
  qsgw_status res = QSGW_OK;
  for (int l = 0; l < L; ++l) {
    info[l] = hinfo[l];  // first non-positive pivot (1-based), as a Cholesky factorisation reports it
    if (info[l] != 0) res = QSGW_ERR_NOT_PD;
  }
  return res;
}

qsgw_status qsgw_chi0_reset(qsgw_ctx* c, int q) {
  if (!c || q < 0 || q >= c->n_q) return QSGW_ERR_ARG;
  if (c->spectral) c->fill[q] = 0;  // columns staged for the bin belong to the sum being cleared
  QSGW_CK(cudaMemsetAsync(c->q[q].acc, 0, c->q[q].bytes, c->stream));
  return QSGW_OK;
}

qsgw_status qsgw_chi0_sync(qsgw_ctx* c) {
  if (!c) return QSGW_ERR_ARG;
  return take_device_error(c);
}

qsgw_status qsgw_chi0_destroy(qsgw_ctx* c) {
  if (!c) return QSGW_ERR_ARG;
  qsgw_status st = QSGW_OK;
  if (c->d_err) st = take_device_error(c);
  for (auto& a : c->q)
    if (a.acc) cudaFree(a.acc);
  if (c->d_w) cudaFree(c->d_w);
  if (c->d_part) cudaFree(c->d_part);
  if (c->d_zstage) cudaFree(c->d_zstage);
  for (void* p : {(void*)c->d_edges, (void*)c->d_one, (void*)c->d_offsets, (void*)c->d_counts, c->d_bins, c->d_perm,
                  c->d_zsort, c->d_stage, (void*)c->d_dptr, c->d_wsc, c->d_zt, c->d_z2, c->d_z3})
    if (p) cudaFree(p);
  if (c->cstream) cudaStreamSynchronize(c->cstream);
  for (int i = 0; i < 2; ++i) {
    if (c->d_hstage[i]) cudaFree(c->d_hstage[i]);
    if (c->d_es[i]) cudaFree(c->d_es[i]);
    if (c->h_eb[i]) cudaFreeHost(c->h_eb[i]);
    if (c->hcopied[i]) cudaEventDestroy(c->hcopied[i]);
    if (c->hfree[i]) cudaEventDestroy(c->hfree[i]);
  }
  if (c->cstream) cudaStreamDestroy(c->cstream);
  mixed_free(c->mixed);
  for (void* p : {c->d_sbuf, c->d_pbuf, c->d_cbuf, c->d_dig})
    if (p) cudaFree(p);
  if (c->d_info) cudaFree(c->d_info);
  if (c->d_err) cudaFree(c->d_err);
  delete c;
  return st;
}

// ---- real-axis route: Eqs. (impolf) and (hilbert) --------------------------------------------
qsgw_status qsgw_spectral_init(qsgw_ctx** ctx, int n_pb, int n_bins, const double* edges, qsgw_prec prec,
                               void* cuda_stream) {
  if (!ctx) return QSGW_ERR_ARG;
  *ctx = nullptr;
  if (n_bins < 1 || n_bins > 4096 || !edges || !(edges[0] > 0.0)) return QSGW_ERR_ARG;
  for (int j = 0; j <= n_bins; ++j)
    if (!std::isfinite(edges[j]) || (j > 0 && !(edges[j] > edges[j - 1]))) return QSGW_ERR_ARG;
  const std::vector<int> npb(n_bins, n_pb);
  const double omega0 = 0.0;
  // spin -1: the readout's -s * acc then gives S_j = +acc (the weights are +1)
  qsgw_status st = qsgw_chi0_init(ctx, n_bins, npb.data(), 1, &omega0, -1.0, prec, cuda_stream);
  if (st != QSGW_OK) return st;
  qsgw_ctx* c = *ctx;
  c->spectral = true;
  c->n_bins = n_bins;
  c->edges.assign(edges, edges + n_bins + 1);
  const double one = 1.0;
  cudaError_t e = cudaMalloc(&c->d_edges, sizeof(double) * (n_bins + 1));
  if (e == cudaSuccess) e = cudaMalloc(&c->d_one, sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc(&c->d_offsets, sizeof(int) * (n_bins + 1));
  if (e == cudaSuccess) e = cudaMalloc(&c->d_counts, sizeof(int) * n_bins);
  if (e == cudaSuccess) e = cudaMalloc(&c->d_dptr, sizeof(void*) * n_bins);
  const size_t cb = spectral_col_bytes(c);
  long long cols = (long long)(kStageBudget / (cb * n_bins));
  cols = std::min<long long>(kStageCols, cols / 16 * 16);
  c->stage_cols = (int)std::max<long long>(16, cols);
  c->fill.assign(n_bins, 0);
  c->h_dptr.assign(n_bins, nullptr);
  if (e == cudaSuccess) e = cudaMalloc(&c->d_stage, cb * n_bins * c->stage_cols);
  if (e == cudaSuccess)
    e = cudaMemcpy(c->d_edges, edges, sizeof(double) * (n_bins + 1), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(c->d_one, &one, sizeof(double), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) {
    cudaGetLastError();
    qsgw_chi0_destroy(c);
    *ctx = nullptr;
    return e == cudaErrorMemoryAllocation ? QSGW_ERR_NOMEM : cuda_status(e);
  }
  return QSGW_OK;
}

qsgw_status qsgw_spectral_accumulate(qsgw_ctx* c, const void* Z, long long ldz, int n_occ, int n_unocc,
                                     const double* eps_occ, const double* eps_unocc) {
  if (!c || !Z || !eps_occ || !eps_unocc || n_occ < 1 || n_unocc < 1) return QSGW_ERR_ARG;
  if (!c->spectral) return QSGW_ERR_STATE;
  const int n_pb = c->q[0].n_pb;
  if (ldz < n_pb || (long long)n_occ * n_unocc > (1LL << 31)) return QSGW_ERR_ARG;
  if (!is_device_ptr(Z) || !is_device_ptr(eps_occ) || !is_device_ptr(eps_unocc)) return QSGW_ERR_ARG;
  const long long K = (long long)n_occ * n_unocc;
  qsgw_status st = grow(&c->d_bins, &c->bins_cap, sizeof(int) * (size_t)K);
  if (st == QSGW_OK) st = grow(&c->d_perm, &c->perm_cap, sizeof(int) * (size_t)K);
  if (st != QSGW_OK) return st;
  launch_hist_sort(eps_occ, eps_unocc, n_occ, n_unocc, c->d_edges, c->n_bins, static_cast<int*>(c->d_bins),
                   c->d_counts, c->d_offsets, static_cast<int*>(c->d_perm), c->d_err, c->stream);
  std::vector<int> off(c->n_bins + 1);
  QSGW_CK(cudaMemcpyAsync(off.data(), c->d_offsets, sizeof(int) * (c->n_bins + 1), cudaMemcpyDeviceToHost,
                          c->stream));
  QSGW_CK(cudaStreamSynchronize(c->stream));
  const int n_in = off[c->n_bins];
  if (n_in == 0) return QSGW_OK;
  // bins whose staging cannot take this call's columns are flushed first (stream order puts the
  // flush's reads of the staging before the gather's writes); a bin with more columns than the
  // staging holds takes them through the overflow buffer and is updated at once
  const int cap = c->stage_cols;
  std::vector<int> fl;
  bool over = false;
  for (int j = 0; j < c->n_bins; ++j) {
    const int cnt = off[j + 1] - off[j];
    if (cnt > 0 && c->fill[j] > 0 && c->fill[j] + cnt > cap) fl.push_back(j);
    over = over || cnt > cap;
  }
  st = spectral_flush(c, fl);
  if (st != QSGW_OK) return st;
  const size_t cb = spectral_col_bytes(c);
  if (over && (st = grow(&c->d_zsort, &c->zsort_cap, cb * (size_t)n_in)) != QSGW_OK) return st;
  std::vector<BinCols> direct;
  for (int j = 0; j < c->n_bins; ++j) {
    const int cnt = off[j + 1] - off[j];
    if (cnt > cap) {
      c->h_dptr[j] = static_cast<uint8_t*>(c->d_zsort) + (size_t)off[j] * cb;
      direct.push_back({j, c->h_dptr[j], cnt});
    } else {
      c->h_dptr[j] = static_cast<uint8_t*>(c->d_stage) + ((size_t)j * cap + c->fill[j]) * cb;
    }
  }
  QSGW_CK(cudaMemcpyAsync(c->d_dptr, c->h_dptr.data(), sizeof(void*) * c->n_bins, cudaMemcpyHostToDevice, c->stream));
  launch_gather_bins(static_cast<const double2*>(Z), ldz, n_pb, static_cast<const int*>(c->d_perm),
                     static_cast<const int*>(c->d_bins), c->d_offsets, n_in, c->d_dptr, c->prec != QSGW_FP64,
                     c->stream);
  for (int j = 0; j < c->n_bins; ++j) {
    const int cnt = off[j + 1] - off[j];
    if (cnt <= cap) c->fill[j] += cnt;
  }
  st = spectral_update(c, direct);
  if (st != QSGW_OK) return st;
  return cuda_status(cudaGetLastError());
}

qsgw_status qsgw_spectral_finalize(qsgw_ctx* c, void* S) {
  if (!c || !S) return QSGW_ERR_ARG;
  if (!c->spectral) return QSGW_ERR_STATE;
  std::vector<int> all(c->n_bins);
  for (int j = 0; j < c->n_bins; ++j) all[j] = j;
  qsgw_status st = spectral_flush(c, all);  // the staged columns enter S_j
  if (st != QSGW_OK) return st;
  const size_t nn = (size_t)c->q[0].n_pb * c->q[0].n_pb;
  for (int j = 0; j < c->n_bins; ++j) {
    const QAcc& a = c->q[j];
    launch_finalize_chi(a.acc, c->prec == QSGW_FP64 ? ACC_FP64 : ACC_DF32, a.n_pb, a.n_pad, 1, c->spin,
                        static_cast<double2*>(S) + (size_t)j * nn, c->stream);
  }
  QSGW_CK(cudaGetLastError());
  return take_device_error(c);
}

qsgw_status qsgw_spectral_real_axis(qsgw_ctx* c, const void* S, int n_out, const int* bins_out, void* out) {
  if (!c || !S || !out || n_out < 1 || !bins_out) return QSGW_ERR_ARG;
  if (!c->spectral) return QSGW_ERR_STATE;
  const int nb = c->n_bins;
  for (int o = 0; o < n_out; ++o)
    if (bins_out[o] < 0 || bins_out[o] >= nb) return QSGW_ERR_ARG;
  const int n_pb = c->q[0].n_pb;
  // Hilbert weights of every bin at the output frequencies (bin centres), FP64 on the host:
  // (1/(R-L)) P.V. int_L^R [1/(w-D) - 1/(w+D)] dD for a density uniform in the bin
  std::vector<double> Kw((size_t)n_out * nb), coef(n_out);
  for (int o = 0; o < n_out; ++o) {
    const int i = bins_out[o];
    const double w = 0.5 * (c->edges[i] + c->edges[i + 1]);
    coef[o] = -M_PI / (c->edges[i + 1] - c->edges[i]);
    for (int j = 0; j < nb; ++j) {
      const double L = c->edges[j], R = c->edges[j + 1];
      Kw[(size_t)j * n_out + o] = std::log(std::fabs(w - L) * (w + L) / (std::fabs(w - R) * (w + R))) / (R - L);
    }
  }
  double *dK = nullptr, *dcoef = nullptr;
  int* dbins = nullptr;
  cudaError_t e = cudaMalloc(&dK, sizeof(double) * Kw.size());
  if (e == cudaSuccess) e = cudaMalloc(&dcoef, sizeof(double) * n_out);
  if (e == cudaSuccess) e = cudaMalloc(&dbins, sizeof(int) * n_out);
  if (e == cudaSuccess) e = cudaMemcpyAsync(dK, Kw.data(), sizeof(double) * Kw.size(), cudaMemcpyHostToDevice, c->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(dcoef, coef.data(), sizeof(double) * n_out, cudaMemcpyHostToDevice, c->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(dbins, bins_out, sizeof(int) * n_out, cudaMemcpyHostToDevice, c->stream);
  qsgw_status st = cuda_status(e);
  if (st == QSGW_OK) {  // Hilbert sum and anti-Hermitian part in one kernel
    launch_hilbert(static_cast<const double2*>(S), n_pb, nb, n_out, dK, dbins, dcoef, static_cast<double2*>(out),
                   c->stream);
    st = cuda_status(cudaGetLastError());
  }
  if (st == QSGW_OK) st = cuda_status(cudaStreamSynchronize(c->stream));
  else cudaStreamSynchronize(c->stream);
  cudaFree(dK);
  cudaFree(dcoef);
  cudaFree(dbins);
  return st;
}

// ---- imaginary-axis correlation self-energy: Eq. (sigci) -----------------------------------------
qsgw_status qsgw_sigc_init(qsgw_ctx** ctx, int n_qp, int n_pb, int n_omega, const double* omega, qsgw_prec prec,
                           void* cuda_stream) {
  if (!ctx) return QSGW_ERR_ARG;
  *ctx = nullptr;
  if (n_qp < 1 || n_qp > kSigcRows || n_pb < 1 || n_pb > 8192 || n_omega < 1 || n_omega > kMaxOmega || !omega)
    return QSGW_ERR_ARG;
  for (int i = 0; i < n_omega; ++i)
    if (!std::isfinite(omega[i]) || !(omega[i] > 0.0) || (i > 0 && !(omega[i] > omega[i - 1]))) return QSGW_ERR_ARG;
  if (prec == QSGW_MIXED_F16X3 && mixed_tile_cols(1) != kSigcAlign) return QSGW_ERR_ARG;
  const int nbb = std::max(1, kSigcRows / n_qp);
  const int Y3 = pad_to(n_qp, kSigcAlign);
  const int npb[2] = {Y3 + n_qp, pad_to(nbb * n_qp, kSigcAlign) + n_pb};
  const double omega0 = 0.0;
  qsgw_status st = qsgw_chi0_init(ctx, 2, npb, 1, &omega0, 1.0, prec, cuda_stream);
  if (st != QSGW_OK) return st;
  qsgw_ctx* c = *ctx;
  c->sigc = true;
  c->sc_nqp = n_qp;
  c->sc_npb = n_pb;
  c->sc_nbb = nbb;
  c->sc_Y3 = Y3;
  c->smesh.L = n_omega;
  for (int i = 0; i < n_omega; ++i) c->smesh.om[i] = omega[i];
  const double one = 1.0;
  cudaError_t e = cudaMalloc(&c->d_one, sizeof(double));
  if (e == cudaSuccess) e = cudaMemcpy(c->d_one, &one, sizeof(double), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) {
    cudaGetLastError();
    qsgw_chi0_destroy(c);
    *ctx = nullptr;
    return cuda_status(e);
  }
  return QSGW_OK;
}

qsgw_status qsgw_sigc_accumulate(qsgw_ctx* c, const void* Z, long long ldz, int n_band, const double* e_qp,
                                 const double* e_band, const void* Wc) {
  if (!c || !Z || !e_qp || !e_band || !Wc || n_band < 1) return QSGW_ERR_ARG;
  if (!c->sigc) return QSGW_ERR_STATE;
  const int n_qp = c->sc_nqp, n_pb = c->sc_npb, L = c->smesh.L, Y3 = c->sc_Y3;
  if (ldz < n_pb || (long long)n_band * n_qp > (1LL << 30)) return QSGW_ERR_ARG;
  if (!is_device_ptr(Z) || !is_device_ptr(e_qp) || !is_device_ptr(e_band) || !is_device_ptr(Wc)) return QSGW_ERR_ARG;
  const bool z32 = c->prec != QSGW_FP64;
  const size_t elt = z32 ? sizeof(float2) : sizeof(double2);
  const long long NT = (long long)n_band * n_qp;
  const int nbb = std::min(c->sc_nbb, n_band);
  const int Mmax = nbb * n_qp, S2max = pad_to(Mmax, kSigcAlign) + n_pb, S3 = Y3 + n_qp;
  qsgw_status st = grow(&c->d_wsc, &c->wsc_cap, sizeof(double) * (size_t)NT * L);
  if (st == QSGW_OK) st = grow(&c->d_zt, &c->zt_cap, sizeof(double2) * (size_t)Mmax * n_pb);
  if (st == QSGW_OK) st = grow(&c->d_z2, &c->z2_cap, elt * (size_t)S2max * L * n_pb);
  if (st == QSGW_OK) st = grow(&c->d_z3, &c->z3_cap, elt * (size_t)S3 * nbb * n_pb);
  if (st != QSGW_OK) return st;
  double* w = static_cast<double*>(c->d_wsc);
  launch_sigc_weights(e_qp, e_band, n_qp, n_band, c->smesh, w, c->d_err, c->stream);
  const AccKind kind = z32 ? ACC_DF32 : ACC_FP64;
  for (int b0 = 0; b0 < n_band; b0 += nbb) {
    const int nb = std::min(nbb, n_band - b0), M = nb * n_qp, Y0 = pad_to(M, kSigcAlign), S2 = Y0 + n_pb;
    double2* Zt = static_cast<double2*>(c->d_zt);
    launch_transpose_cols(static_cast<const double2*>(Z), ldz, n_pb, (long long)b0 * n_qp, M, Zt, c->stream);
    launch_sigc_stack_d(Zt, M, n_pb, w, NT, (long long)b0 * n_qp, L, static_cast<const double2*>(Wc), Y0, c->d_z2,
                        z32, c->stream);
    QSGW_CK(cudaMemsetAsync(c->q[1].acc, 0, c->q[1].bytes, c->stream));
    st = sigc_product(c, 1, c->d_z2, S2, (long long)L * n_pb, M, Y0);
    if (st != QSGW_OK) return st;
    launch_sigc_stack_i(c->q[1].acc, kind, c->q[1].n_pad, Y0, Zt, n_qp, nb, n_pb, Y3, c->d_z3, z32, c->stream);
    st = sigc_product(c, 0, c->d_z3, S3, (long long)nb * n_pb, n_qp, Y3);
    if (st != QSGW_OK) return st;
  }
  return cuda_status(cudaGetLastError());
}

qsgw_status qsgw_sigc_finalize(qsgw_ctx* c, void* I) {
  if (!c || !I) return QSGW_ERR_ARG;
  if (!c->sigc) return QSGW_ERR_STATE;
  if (!is_device_ptr(I)) return QSGW_ERR_ARG;
  launch_sigc_readout(c->q[0].acc, c->prec == QSGW_FP64 ? ACC_FP64 : ACC_DF32, c->q[0].n_pad, c->sc_nqp, c->sc_Y3,
                      static_cast<double2*>(I), c->stream);
  QSGW_CK(cudaGetLastError());
  return take_device_error(c);
}

qsgw_status qsgw_chi0_block_noalloc(const void* Z, long long ldz, int n_pb, int n_occ, int n_unocc,
                                    const double* eps_occ, const double* eps_unocc, int n_omega, const double* omega,
                                    double spin_factor, void* chi0, void* cuda_stream) {
  if (!Z || !eps_occ || !eps_unocc || !omega || !chi0 || n_pb < 1 || n_pb > kMaxNpb || ldz < n_pb || n_occ < 1 ||
      n_unocc < 1 || n_omega < 1 || n_omega > kMaxOmega || !std::isfinite(spin_factor))
    return QSGW_ERR_ARG;
  if ((long long)n_occ * n_unocc > (1LL << 31)) return QSGW_ERR_ARG;
  OmegaGrid g{};
  g.L = n_omega;
  for (int l = 0; l < n_omega; ++l) {
    if (!std::isfinite(omega[l]) || omega[l] < 0.0) return QSGW_ERR_ARG;
    g.w2[l] = omega[l] * omega[l];
    g.w2f[l] = (float)(omega[l] * omega[l]);
  }
  if (!is_device_ptr(Z) || !is_device_ptr(eps_occ) || !is_device_ptr(eps_unocc) || !is_device_ptr(chi0))
    return QSGW_ERR_ARG;
  return mixed_chi0_noalloc(static_cast<const double2*>(Z), ldz, n_pb, n_occ, n_unocc, eps_occ, eps_unocc, g,
                            spin_factor, static_cast<double2*>(chi0), static_cast<cudaStream_t>(cuda_stream));
}

qsgw_status qsgw_synth_z(unsigned long long seed, int gen_q, int k, int n_pb, int n_occ, int n_unocc, double s_div,
                         void* Z, long long ldz, void* cuda_stream) {
  if (!Z || n_pb < 1 || n_occ < 1 || n_unocc < 1 || ldz < n_pb || k < 0 || gen_q < 0 || gen_q > 0xFFFFFF ||
      !(s_div > 0.0))
    return QSGW_ERR_ARG;
  if (!is_device_ptr(Z)) return QSGW_ERR_ARG;
  launch_synth_z(seed, gen_q, k, n_pb, n_occ, n_unocc, s_div, static_cast<double2*>(Z), ldz,
                 static_cast<cudaStream_t>(cuda_stream));
  return cuda_status(cudaGetLastError());
}

qsgw_status qsgw_chi0_accumulate_synthetic(qsgw_ctx* c, int q, unsigned long long seed, int gen_q, int k_begin,
                                           int k_end, int n_occ, const int* n_unocc_per_k, const double* eps_occ,
                                           const double* eps_unocc, double s_div) {
  if (c && (c->sigx || c->spectral || c->sigc)) return QSGW_ERR_STATE;
  if (!c || q < 0 || q >= c->n_q || k_begin < 0 || k_end <= k_begin || n_occ < 1 || !n_unocc_per_k || !eps_occ ||
      !eps_unocc || !(s_div > 0.0) || gen_q < 0 || gen_q > 0xFFFFFF)
    return QSGW_ERR_ARG;
  if (!is_device_ptr(eps_occ) || !is_device_ptr(eps_unocc)) return QSGW_ERR_ARG;
  const QAcc& a = c->q[q];
  size_t max_cols = 0;
  for (int i = 0; i < k_end - k_begin; ++i) {
    if (n_unocc_per_k[i] < 1) return QSGW_ERR_ARG;
    const size_t cols = (size_t)n_occ * n_unocc_per_k[i];
    if (cols > max_cols) max_cols = cols;
  }
  qsgw_status st = grow(&c->d_zstage, &c->zstage_cap, sizeof(double2) * (size_t)a.n_pb * max_cols);
  if (st != QSGW_OK) return st;
  size_t eu_off = 0;
  for (int i = 0; i < k_end - k_begin; ++i) {
    const int nu = n_unocc_per_k[i];
    auto* Zs = static_cast<double2*>(c->d_zstage);
    launch_synth_z(seed, gen_q, k_begin + i, a.n_pb, n_occ, nu, s_div, Zs, a.n_pb, c->stream);
    st = accumulate_device(c, q, Zs, false, a.n_pb, n_occ, nu, eps_occ + (size_t)i * n_occ, eps_unocc + eu_off);
    if (st != QSGW_OK) return st;
    eu_off += nu;
  }
  return QSGW_OK;
}

}  // extern "C"
