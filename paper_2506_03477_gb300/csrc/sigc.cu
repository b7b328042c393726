// Imaginary-axis correlation self-energy, Eq. (sigci) (Sec. 2):
//
//   I_nm = - sum_k sum_{n'} sum_i w_i(e_qn - e_{q-k n'}) sum_{mu, nu} conj(Z_{n' n, mu}) W^c_{mu nu}(k, i omega_i) Z_{n' m, nu}
//
// evaluated as two products, each the off-diagonal block of a Hermitian update of a stacked
// operand, so that the tensor-core (or FP64) HERK kernels run them unchanged over a restricted
// tile list:
//   D[(n', n), nu] = sum_{i, mu} w_i conj(Z_{n' n, mu}) W^c_i[mu, nu]
//       rows (n', n) scaled by w_i and rows nu = conj(W^c_i[nu, mu]) (= W^c_i[mu, nu], W^c Hermitian)
//       over the columns (i, mu);
//   I_nm -= sum_{n', nu} D[(n', n), nu] Z_{n' m, nu}
//       rows n = conj(D[(n', n), nu]) and rows m = Z_{n' m, nu} over the columns (n', nu).
// The kernels here compute the integration weights, transpose a batch of Z, build both stacked
// operands and read the result out.
#include "internal.cuh"

namespace qsgw {
namespace {

constexpr double kPi = 3.14159265358979323846;

// T(x) = (1 - atan(x)/x) / x^2, the tail factor; for x < 1/2 its alternating series
// sum_k (-1)^k x^(2k) / (2k + 3), which avoids the cancellation of the closed form.
__device__ double tail_factor(double x) {
  if (x < 0.5) {
    double t = 0.0, p = 1.0;
    for (int k = 0; k < 30; ++k) {
      t += p / (2 * k + 3);
      p *= -x * x;
    }
    return t;
  }
  return (1.0 - atan(x) / x) / (x * x);
}

// Integration weights of Eq. (sigci): sum_i w_i X(i omega_i) ~= (1/pi) int_0^inf dE/(dE^2+w^2) X(iw) dw
// with dE/(dE^2+w^2) integrated exactly and X interpolated on the mesh: constant on [0, omega_0],
// linear between mesh points, X_{L-1} (omega_{L-1}/w)^2 beyond the last (W^c decays as 1/w^2).
// Segment [a, b] (h = b - a) adds (b A - B)/h to w(a) and (B - a A)/h to w(b), with
// A = atan(h dE / (dE^2 + a b)) and B = (dE/2) log1p((b^2 - a^2) / (dE^2 + a^2)) the increments of
// the antiderivatives atan(w/dE) and (dE/2) ln(dE^2 + w^2); the tail adds (dE/W) T(|dE|/W).
// dE = 0 gives 0 (principal value). Weights are stored frequency-major: w[i * NT + t].
__global__ void sigc_weights_kernel(const double* __restrict__ e_qp, const double* __restrict__ e_band, int n_qp,
                                    int n_band, SigcMesh m, double* __restrict__ w, int* d_err) {
  const long long NT = (long long)n_band * n_qp;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < NT; t += (long long)gridDim.x * blockDim.x) {
    const int b = (int)(t / n_qp), n = (int)(t % n_qp);
    const double dE = e_qp[n] - e_band[b];
    if (!isfinite(dE)) atomicCAS(d_err, DEV_OK, DEV_DOMAIN);
    if (dE == 0.0 || !isfinite(dE)) {
      for (int i = 0; i < m.L; ++i) w[i * NT + t] = 0.0;
      continue;
    }
    double carry = atan(m.om[0] / dE);  // [0, omega_0], X = X_0
    for (int i = 0; i + 1 < m.L; ++i) {
      const double a = m.om[i], bb = m.om[i + 1], h = bb - a;
      const double A = atan(h * dE / (dE * dE + a * bb));
      const double B = 0.5 * dE * log1p((bb - a) * (bb + a) / (dE * dE + a * a));
      w[i * NT + t] = (carry + (bb * A - B) / h) / kPi;
      carry = (B - a * A) / h;
    }
    const double W = m.om[m.L - 1];
    w[(m.L - 1) * NT + t] = (carry + dE / W * tail_factor(fabs(dE) / W)) / kPi;
  }
}

// 32 x 32 tiles through shared memory: reads along mu, writes along the rows of Zt.
__global__ void __launch_bounds__(256) transpose_cols_kernel(const double2* __restrict__ Z, long long ldz, int n_pb,
                                                             long long c0, int M, double2* __restrict__ Zt) {
  __shared__ double2 t[32][33];
  const int r0 = blockIdx.x * 32, mu0 = blockIdx.y * 32;
  for (int y = threadIdx.y; y < 32; y += 8) {
    const int r = r0 + y, mu = mu0 + threadIdx.x;
    if (r < M && mu < n_pb) t[y][threadIdx.x] = Z[(c0 + r) * ldz + mu];
  }
  __syncthreads();
  for (int y = threadIdx.y; y < 32; y += 8) {
    const int mu = mu0 + y, r = r0 + threadIdx.x;
    if (r < M && mu < n_pb) Zt[(size_t)mu * M + r] = t[threadIdx.x][y];
  }
}

__device__ __forceinline__ void put(double2* d, double2 x) { *d = x; }
__device__ __forceinline__ void put(float2* d, double2 x) { *d = make_float2((float)x.x, (float)x.y); }

// Grid (256-row blocks of the S2 = Y0 + n_pb stacked rows, frequency i, groups of SD_MU columns
// mu); column-major output, column (i, mu). Thread r writes row r of the group's columns: the
// weight w_i of a D row is loaded once for them all, and the group's loads are independent.
constexpr int SD_MU = 16;
template <typename T>
__global__ void __launch_bounds__(256) stack_d_kernel(const double2* __restrict__ Zt, int M, int n_pb,
                                                      const double* __restrict__ w, long long NT, long long row0,
                                                      const double2* __restrict__ Wc, int Y0, T* __restrict__ Z2) {
  const int r = blockIdx.x * 256 + threadIdx.x, i = blockIdx.y, mu0 = blockIdx.z * SD_MU;
  const int S2 = Y0 + n_pb;
  if (r >= S2) return;
  const int nmu = min(SD_MU, n_pb - mu0);
  double2 v[SD_MU];
  if (r < M) {
    const double x = w[i * NT + row0 + r];
#pragma unroll
    for (int u = 0; u < SD_MU; ++u)
      if (u < nmu) {
        const double2 z = Zt[(size_t)(mu0 + u) * M + r];
        v[u] = make_double2(x * z.x, x * z.y);
      }
  } else if (r >= Y0) {
#pragma unroll
    for (int u = 0; u < SD_MU; ++u)
      if (u < nmu) {  // column mu of W^c_i: element (nu, mu), nu = r - Y0
        const double2 q = Wc[((size_t)i * n_pb + mu0 + u) * n_pb + (r - Y0)];
        v[u] = make_double2(q.x, -q.y);
      }
  } else {
#pragma unroll
    for (int u = 0; u < SD_MU; ++u) v[u] = make_double2(0.0, 0.0);
  }
#pragma unroll
  for (int u = 0; u < SD_MU; ++u)
    if (u < nmu) put(Z2 + ((size_t)i * n_pb + mu0 + u) * S2 + r, v[u]);
}

// Element (I, J) of an accumulator (loc = J * n_pad + I), one frequency: FP64 complex, or the
// double-float planes (hi, lo) of Re and Im followed by the FP64 sums of split tiles.
__device__ __forceinline__ double2 acc_at(const void* acc, AccKind kind, int n_pad, size_t loc) {
  if (kind == ACC_FP64) return static_cast<const double2*>(acc)[loc];
  const size_t nn = (size_t)n_pad * n_pad;
  const float2* a = static_cast<const float2*>(acc);
  const double* b = reinterpret_cast<const double*>(a + 2 * nn);
  const float2 re = a[loc], im = a[nn + loc];
  return make_double2(((double)re.x + (double)re.y) + b[loc], ((double)im.x + (double)im.y) + b[nn + loc]);
}

// One CTA per stacked column (band b, nu); column-major, S3 = Y3 + n_qp rows.
template <typename T>
__global__ void __launch_bounds__(256) stack_i_kernel(const void* __restrict__ accD, AccKind kind, int n_padD, int Y0,
                                                      const double2* __restrict__ Zt, int n_qp, int nb, int n_pb,
                                                      int Y3, T* __restrict__ Z3) {
  const int col = blockIdx.x, b = col / n_pb, nu = col % n_pb;
  const int S3 = Y3 + n_qp, M = nb * n_qp;
  T* dst = Z3 + (size_t)col * S3;
  const size_t dloc = (size_t)(Y0 + nu) * n_padD + (size_t)b * n_qp;
  const double2* zt = Zt + (size_t)nu * M + (size_t)b * n_qp;
  for (int r = threadIdx.x; r < S3; r += 256) {
    double2 v = make_double2(0.0, 0.0);
    if (r < n_qp) {
      const double2 d = acc_at(accD, kind, n_padD, dloc + r);
      v = make_double2(d.x, -d.y);
    } else if (r >= Y3) {
      v = zt[r - Y3];
    }
    put(dst + r, v);
  }
}

__global__ void sigc_readout_kernel(const void* __restrict__ accI, AccKind kind, int n_padI, int n_qp, int Y3,
                                    double2* __restrict__ out) {
  const int n = blockIdx.x * blockDim.x + threadIdx.x, m = blockIdx.y;
  if (n >= n_qp) return;
  const double2 v = acc_at(accI, kind, n_padI, (size_t)(Y3 + m) * n_padI + n);
  out[(size_t)m * n_qp + n] = make_double2(-v.x, -v.y);
}

}  // namespace

void launch_sigc_weights(const double* e_qp, const double* e_band, int n_qp, int n_band, const SigcMesh& m,
                         double* w, int* d_err, cudaStream_t s) {
  const long long NT = (long long)n_band * n_qp;
  int blocks = (int)((NT + 255) / 256);
  if (blocks > 152 * 8) blocks = 152 * 8;
  sigc_weights_kernel<<<blocks, 256, 0, s>>>(e_qp, e_band, n_qp, n_band, m, w, d_err);
}

void launch_transpose_cols(const double2* Z, long long ldz, int n_pb, long long c0, int M, double2* Zt, cudaStream_t s) {
  transpose_cols_kernel<<<dim3((M + 31) / 32, (n_pb + 31) / 32), dim3(32, 8), 0, s>>>(Z, ldz, n_pb, c0, M, Zt);
}

void launch_sigc_stack_d(const double2* Zt, int M, int n_pb, const double* w, long long NT, long long row0, int L,
                         const double2* Wc, int Y0, void* Z2, bool z32, cudaStream_t s) {
  const dim3 grid((Y0 + n_pb + 255) / 256, L, (n_pb + SD_MU - 1) / SD_MU);
  if (z32)
    stack_d_kernel<float2><<<grid, 256, 0, s>>>(Zt, M, n_pb, w, NT, row0, Wc, Y0, static_cast<float2*>(Z2));
  else
    stack_d_kernel<double2><<<grid, 256, 0, s>>>(Zt, M, n_pb, w, NT, row0, Wc, Y0, static_cast<double2*>(Z2));
}

void launch_sigc_stack_i(const void* accD, AccKind kind, int n_padD, int Y0, const double2* Zt, int n_qp, int nb,
                         int n_pb, int Y3, void* Z3, bool z32, cudaStream_t s) {
  const int cols = nb * n_pb;
  if (z32)
    stack_i_kernel<float2><<<cols, 256, 0, s>>>(accD, kind, n_padD, Y0, Zt, n_qp, nb, n_pb, Y3,
                                                static_cast<float2*>(Z3));
  else
    stack_i_kernel<double2><<<cols, 256, 0, s>>>(accD, kind, n_padD, Y0, Zt, n_qp, nb, n_pb, Y3,
                                                 static_cast<double2*>(Z3));
}

void launch_sigc_readout(const void* accI, AccKind kind, int n_padI, int n_qp, int Y3, double2* out, cudaStream_t s) {
  sigc_readout_kernel<<<dim3((n_qp + 127) / 128, n_qp), 128, 0, s>>>(accI, kind, n_padI, n_qp, Y3, out);
}

}  // namespace qsgw
