/*
 * Plain FP64 CPU oracle for the RPA polarization chi0(q, i omega_l) in the mixed product
 * basis, the dielectric matrix eps and the screened Coulomb interaction W.
 *
 * TEST INFRASTRUCTURE ONLY. This file is the reference the CUDA library is checked against.
 * Only the tests, the smoke check and the benchmark's CPU-baseline leg may load it; the
 * library never calls it, and it shares no code, header or table with the library.
 *
 * Everything is a direct transcription of the definitions, in double precision, with plain
 * loops (OpenMP over independent output entries only; every sum runs in a fixed order):
 *
 *   Eq. (polfx), Sec. 2: Pi_{mu nu}(q, w) = sum_k sum_{n occ} sum_{n' unocc} Z_mu Z_nu^*
 *        [ 1/(w - Delta + i delta) - 1/(w + Delta - i delta) ],  Delta = e_{q+k n'} - e_{k n}.
 *   On the imaginary axis w = i omega_l with delta -> 0 the bracket is
 *        1/(i omega - Delta) - 1/(i omega + Delta) = -2 Delta / (Delta^2 + omega^2).
 *   Index convention (the conjugate sits on the row index):
 *        chi0_IJ(l) = s * sum_r w_l(Delta_r) conj(z_{I,r}) z_{J,r},
 *   which is the transpose (= complex conjugate) of the paper's Pi_{mu nu} for the same Z.
 *   No 1/N_k factor: any Brillouin-zone weight is carried by Z or by the spin factor s.
 *
 *   Eq. (dielectricfunction): eps_{mu nu} = delta_{mu nu} - sqrt(v_mu) Pi_{mu nu} sqrt(v_nu)
 *   Eq. (screenedcoulomb):    W_{mu nu}   = sqrt(v_mu) eps^{-1}_{mu nu} sqrt(v_nu)
 *   Eq. (wc):                 W^c_{mu nu} = sqrt(v_mu) (eps^{-1}_{mu nu} - delta_{mu nu}) sqrt(v_nu)
 *   eps is Hermitian positive definite (eps >= I because chi0(i omega) is negative
 *   semidefinite, Sec. 2), so eps^{-1} is formed by a textbook Cholesky factorisation
 *   eps = L L^H followed by forward and backward substitution against the identity.
 *
 * Matrices are column-major per frequency: element (i, j) of frequency l is at
 * l*N*N + j*N + i.
 *
 * Also Eq. (sigx) (exchange self-energy), a Hermitian update of the same form with the
 * Coulomb eigenvalues as column weights: see oracle_sigx; the real-axis route of Eqs.
 * (impolf) and (hilbert): oracle_hist_spectral, oracle_hilbert_weight; and the imaginary-axis
 * correlation self-energy of Eq. (sigci): oracle_sigc_weights, oracle_sigc.
 */
#include <complex.h>
#include <math.h>
#include <stddef.h>
#include <stdlib.h>

typedef double complex zdouble;

/* Sec. 2, Eq. (polfx) at w = i omega, delta -> 0. */
double oracle_weight(double delta, double omega) { return -2.0 * delta / (delta * delta + omega * omega); }

/* Transition energies of one k-point, r = n * n_unocc + m: Delta_r = e_unocc[m] - e_occ[n].
 * Returns the number of columns with Delta <= 0 or non-finite (the method needs Delta > 0). */
int oracle_delta(int n_occ, int n_unocc, const double *eps_occ, const double *eps_unocc, double *delta) {
  int bad = 0;
  for (int n = 0; n < n_occ; ++n)
    for (int m = 0; m < n_unocc; ++m) {
      double d = eps_unocc[m] - eps_occ[n];
      delta[(size_t)n * n_unocc + m] = d;
      if (!(d > 0.0) || !isfinite(d)) ++bad;
    }
  return bad;
}

/* chi0 restricted to rows I in a set and columns J in a set, every frequency:
 *   out[(l * nJ + j) * nI + i] = s * sum_{r<K} w_l(Delta_r) conj(ZI[i*K + r]) ZJ[j*K + r]
 * ZI is (nI x K) row-major (row i holds z_{I_i, r} for all r), ZJ likewise.
 * With ZI = ZJ = all rows this is the full matrix in the column-major layout above. */
void oracle_chi0_rows(long long K, int nI, const zdouble *ZI, int nJ, const zdouble *ZJ, const double *delta, int L,
                      const double *omega, double spin, zdouble *out) {
  double *wl = (double *)malloc((size_t)(K > 0 ? K : 1) * sizeof(double));
  for (int l = 0; l < L; ++l) {
    for (long long r = 0; r < K; ++r) wl[r] = oracle_weight(delta[r], omega[l]);
#pragma omp parallel for schedule(dynamic, 1)
    for (int j = 0; j < nJ; ++j) {
      const zdouble *zj = ZJ + (size_t)j * K;
      for (int i = 0; i < nI; ++i) {
        const zdouble *zi = ZI + (size_t)i * K;
        zdouble acc = 0.0;
        for (long long r = 0; r < K; ++r) acc += wl[r] * (conj(zi[r]) * zj[r]);
        out[((size_t)l * nJ + j) * nI + i] = spin * acc;
      }
    }
  }
  free(wl);
}

/* Eq. (sigx), Sec. 2: the exchange self-energy in the basis of the states at q,
 *   Sigma^x_{nm}(q) = - sum_k sum_{n' occ} sum_mu conj(Z^{(q-k)n', qn}_{k mu}) v_mu(k) Z^{(q-k)n', qm}_{k mu}.
 * Z is row-major (n_qp x Ktot): row n holds, for k = 0..n_k-1, n' = 0..n_occ[k]-1 and mu =
 * 0..n_pb-1 (mu fastest), the value Z^{(q-k)n', qn}_{k mu}; Ktot = n_pb * sum_k n_occ[k].
 * v is [n_k][n_pb] (the Coulomb eigenvalues v_mu(k) of Eq. (eqvcoue)).
 * out is column-major n_qp x n_qp: element (n, m) at m * n_qp + n. */
void oracle_sigx(int n_k, const int *n_occ, int n_pb, int n_qp, long long Ktot, const zdouble *Z, const double *v,
                 zdouble *out) {
#pragma omp parallel for schedule(dynamic, 1)
  for (int m = 0; m < n_qp; ++m) {
    for (int n = 0; n < n_qp; ++n) {
      zdouble acc = 0.0;
      long long r = 0;
      for (int k = 0; k < n_k; ++k)
        for (int np = 0; np < n_occ[k]; ++np)
          for (int mu = 0; mu < n_pb; ++mu, ++r)
            acc += v[(size_t)k * n_pb + mu] * (conj(Z[(size_t)n * Ktot + r]) * Z[(size_t)m * Ktot + r]);
      out[(size_t)m * n_qp + n] = -acc;
    }
  }
}

/* Eq. (impolf), Sec. 2, real-axis route: the spectral weight of every histogram bin
 * [edges[j], edges[j+1]) of transition energies,
 *   S_j(I, J) = sum over columns r with edges[j] <= Delta_r < edges[j+1] of conj(ZI[i, r]) ZJ[j, r],
 * so that Im chi0(w) on the real axis is -pi S_j / (edges[j+1] - edges[j]) inside bin j (each
 * column carries weight 1 into the bin holding its Delta; the paper spreads it with tetrahedron
 * weights, which need a k-mesh). Columns outside every bin contribute nothing; the count of
 * such columns is returned. out[(j * nJ + jj) * nI + i], ZI / ZJ row-major as in oracle_chi0_rows. */
long long oracle_hist_spectral(long long K, int nI, const zdouble *ZI, int nJ, const zdouble *ZJ, const double *delta,
                               int n_bins, const double *edges, zdouble *out) {
  int *bin = (int *)malloc((size_t)(K > 0 ? K : 1) * sizeof(int));
  long long outside = 0;
  for (long long r = 0; r < K; ++r) {
    bin[r] = -1;
    for (int j = 0; j < n_bins; ++j)
      if (edges[j] <= delta[r] && delta[r] < edges[j + 1]) bin[r] = j;
    if (bin[r] < 0) ++outside;
  }
  for (size_t t = 0; t < (size_t)n_bins * nJ * nI; ++t) out[t] = 0.0;
#pragma omp parallel for schedule(dynamic, 1)
  for (int jj = 0; jj < nJ; ++jj)
    for (int i = 0; i < nI; ++i)
      for (long long r = 0; r < K; ++r)
        if (bin[r] >= 0)
          out[((size_t)bin[r] * nJ + jj) * nI + i] += conj(ZI[(size_t)i * K + r]) * ZJ[(size_t)jj * K + r];
  free(bin);
  return outside;
}

/* Eq. (hilbert): the Hilbert-transformation weight of bin [L, R) at real frequency w > 0, for a
 * density uniform inside the bin: (1/(R-L)) P.V. int_L^R [1/(w - D) - 1/(w + D)] dD
 *   = (1/(R-L)) ln( |w - L| (w + L) / (|w - R| (w + R)) ). */
double oracle_hilbert_weight(double w, double L, double R) {
  return log(fabs(w - L) * (w + L) / (fabs(w - R) * (w + R))) / (R - L);
}

/* Eq. (dielectricfunction): eps = I - D chi D with D = diag(sqrt(v)), one frequency. */
void oracle_eps(int N, const zdouble *chi, const double *v, zdouble *eps) {
  for (int j = 0; j < N; ++j)
    for (int i = 0; i < N; ++i)
      eps[(size_t)j * N + i] = (i == j ? 1.0 : 0.0) - sqrt(v[i]) * chi[(size_t)j * N + i] * sqrt(v[j]);
}

/* Textbook Cholesky eps = L L^H on the lower triangle (column-major, L overwrites a copy).
 * Returns 0 on success, or j+1 if the j-th pivot is not positive (eps not HPD). */
int oracle_cholesky(int N, const zdouble *A, zdouble *Lf) {
  for (size_t t = 0; t < (size_t)N * N; ++t) Lf[t] = 0.0;
  for (int j = 0; j < N; ++j) {
    double d = creal(A[(size_t)j * N + j]);
    for (int k = 0; k < j; ++k) {
      zdouble ljk = Lf[(size_t)k * N + j];
      d -= creal(ljk * conj(ljk));
    }
    if (!(d > 0.0)) return j + 1;
    double ljj = sqrt(d);
    Lf[(size_t)j * N + j] = ljj;
#pragma omp parallel for schedule(static)
    for (int i = j + 1; i < N; ++i) {
      zdouble s = A[(size_t)j * N + i];
      for (int k = 0; k < j; ++k) s -= Lf[(size_t)k * N + i] * conj(Lf[(size_t)k * N + j]);
      Lf[(size_t)j * N + i] = s / ljj;
    }
  }
  return 0;
}

/* eps^{-1} from the Cholesky factor: solve L Y = I, then L^H X = Y, column by column. */
void oracle_cholesky_inverse(int N, const zdouble *Lf, zdouble *X) {
#pragma omp parallel for schedule(dynamic, 4)
  for (int c = 0; c < N; ++c) {
    zdouble *x = X + (size_t)c * N;
    for (int i = 0; i < N; ++i) {           /* forward: L y = e_c */
      zdouble s = (i == c) ? 1.0 : 0.0;
      for (int k = 0; k < i; ++k) s -= Lf[(size_t)k * N + i] * x[k];
      x[i] = s / Lf[(size_t)i * N + i];
    }
    for (int i = N - 1; i >= 0; --i) {      /* backward: L^H x = y, (L^H)_{ik} = conj(L_{ki}) */
      zdouble s = x[i];
      for (int k = i + 1; k < N; ++k) s -= conj(Lf[(size_t)i * N + k]) * x[k];
      x[i] = s / conj(Lf[(size_t)i * N + i]);
    }
  }
}

/* eps, W = D eps^{-1} D and W^c = W - diag(v) for every frequency (Eqs. dielectricfunction,
 * screenedcoulomb, wc). `work` holds N*N complex values. info[l] = 0 or the failed pivot+1;
 * W and W^c of a failed frequency are left as zero. eps_out / Wc_out may be NULL. */
void oracle_eps_w(int N, int L, const zdouble *chi, const double *v, zdouble *eps_out, zdouble *W_out, zdouble *Wc_out,
                  int *info, zdouble *work_eps, zdouble *work_l) {
  size_t NN = (size_t)N * N;
  for (int l = 0; l < L; ++l) {
    oracle_eps(N, chi + l * NN, v, work_eps);
    if (eps_out)
      for (size_t t = 0; t < NN; ++t) eps_out[l * NN + t] = work_eps[t];
    zdouble *W = W_out + l * NN;
    info[l] = oracle_cholesky(N, work_eps, work_l);
    if (info[l] != 0) {
      for (size_t t = 0; t < NN; ++t) W[t] = 0.0;
      if (Wc_out)
        for (size_t t = 0; t < NN; ++t) Wc_out[l * NN + t] = 0.0;
      continue;
    }
    oracle_cholesky_inverse(N, work_l, W); /* W <- eps^{-1} */
    for (int j = 0; j < N; ++j)
      for (int i = 0; i < N; ++i) W[(size_t)j * N + i] *= sqrt(v[i]) * sqrt(v[j]);
    if (Wc_out)
      for (int j = 0; j < N; ++j)
        for (int i = 0; i < N; ++i) Wc_out[l * NN + (size_t)j * N + i] = W[(size_t)j * N + i] - (i == j ? v[i] : 0.0);
  }
}

/* Integration weights of Eq. (sigci), Sec. 2: w[i] such that
 *   int_{-inf}^{inf} dw/(2 pi) X(i w) / (dE - i w)  ~=  sum_i w[i] X(i omega_i)
 * for X even in w (W^c(i w) = W^c(-i w)), i.e. (1/pi) int_0^inf dE/(dE^2 + w^2) X(i w) dw.
 * The paper takes the weights from the method of Aryasetiawan and Gunnarsson, which it cites
 * but does not give. Reading used here: the sharply peaked factor dE/(dE^2 + w^2) is integrated
 * exactly and only X is interpolated on the mesh 0 < omega_0 < ... < omega_{L-1}:
 *   X = X_0 on [0, omega_0];
 *   X linear between neighbouring mesh points;
 *   X = X_{L-1} (omega_{L-1} / w)^2 beyond omega_{L-1} (the large-w decay of W^c).
 * With F(w) = atan(w / dE) and G(w) = (dE / 2) ln(dE^2 + w^2) the antiderivatives of
 * dE/(dE^2+w^2) and w dE/(dE^2+w^2), segment [a, b] of length h adds (b A - B)/h to the weight of
 * a and (B - a A)/h to that of b, A = F(b) - F(a), B = G(b) - G(a) (evaluated without
 * cancellation, see below). The tail adds
 * (dE / W) T(|dE| / W), W = omega_{L-1}, T(x) = (1 - atan(x)/x) / x^2 (its series for small x).
 * dE = 0 gives 0 (the principal value of the limits dE -> 0+ and 0-). */
static double sigc_tail(double x) {
  if (x < 0.5) {  /* T(x) = sum_k (-1)^k x^(2k) / (2k + 3) */
    double t = 0.0, p = 1.0;
    for (int k = 0; k < 40; ++k, p *= -x * x) t += p / (2 * k + 3);
    return t;
  }
  return (1.0 - atan(x) / x) / (x * x);
}

void oracle_sigc_weights(double dE, int L, const double *omega, double *w) {
  for (int i = 0; i < L; ++i) w[i] = 0.0;
  if (dE == 0.0) return;
  w[0] += atan(omega[0] / dE);
  for (int i = 0; i + 1 < L; ++i) {
    const double a = omega[i], b = omega[i + 1], h = b - a;
    /* A and B as differences of the antiderivatives, in forms without cancellation:
     * atan(b/dE) - atan(a/dE) = atan(h dE / (dE^2 + a b)) (0 <= a < b), and
     * ln((dE^2 + b^2) / (dE^2 + a^2)) = log1p((b^2 - a^2) / (dE^2 + a^2)). */
    const double A = atan(h * dE / (dE * dE + a * b));
    const double B = 0.5 * dE * log1p((b - a) * (b + a) / (dE * dE + a * a));
    w[i] += (b * A - B) / h;
    w[i + 1] += (B - a * A) / h;
  }
  const double W = omega[L - 1];
  w[L - 1] += dE / W * sigc_tail(fabs(dE) / W);
  const double pi = 3.14159265358979323846;
  for (int i = 0; i < L; ++i) w[i] /= pi;
}

/* Eq. (sigci), Sec. 2: the imaginary-axis part of the correlation self-energy,
 *   I_nm = - sum_k sum_{n'} sum_i w_i(e_qp[n] - e_band[k][n'])
 *            sum_{mu, nu} conj(Z_k[n' n, mu]) Wc_k(i omega_i)[mu, nu] Z_k[n' m, nu].
 * Z_k is column-major n_pb x (n_band[k] * n_qp): column r = n' * n_qp + n holds
 * Z^{(q-k) n', q n}_{k mu} for mu = 0 .. n_pb - 1; the blocks of all k follow one another.
 * e_band is the concatenation of the n_band[k] band energies e_{q-k, n'}. Wc_k is [L][n_pb][n_pb]
 * column-major (element (mu, nu) of frequency i at i*n_pb*n_pb + nu*n_pb + mu), blocks of all k
 * one after another. out is column-major n_qp x n_qp: element (n, m) at m * n_qp + n.
 * For every (k, n', i) the product y_m = Wc_i Z[n' m, :] is formed first, then its inner
 * products with conj(Z[n' n, :]). */
void oracle_sigc(int n_k, const int *n_band, int n_pb, int n_qp, const zdouble *Z, const double *e_qp,
                 const double *e_band, int L, const double *omega, const zdouble *Wc, zdouble *out) {
  const size_t nn = (size_t)n_pb * n_pb;
  for (size_t t = 0; t < (size_t)n_qp * n_qp; ++t) out[t] = 0.0;
  double *w = (double *)malloc((size_t)n_qp * L * sizeof(double));
  zdouble *y = (zdouble *)malloc((size_t)n_qp * n_pb * sizeof(zdouble));
  size_t zoff = 0, eoff = 0;
  for (int k = 0; k < n_k; ++k) {
    const zdouble *Wk = Wc + (size_t)k * L * nn;
    for (int np = 0; np < n_band[k]; ++np) {
      const zdouble *Zb = Z + zoff + (size_t)np * n_qp * n_pb;  /* column n of this band at Zb + n*n_pb */
      for (int n = 0; n < n_qp; ++n) oracle_sigc_weights(e_qp[n] - e_band[eoff + np], L, omega, w + (size_t)n * L);
      for (int i = 0; i < L; ++i) {
        const zdouble *Wi = Wk + (size_t)i * nn;
#pragma omp parallel for schedule(static)
        for (int m = 0; m < n_qp; ++m)
          for (int mu = 0; mu < n_pb; ++mu) {
            zdouble t = 0.0;
            for (int nu = 0; nu < n_pb; ++nu) t += Wi[(size_t)nu * n_pb + mu] * Zb[(size_t)m * n_pb + nu];
            y[(size_t)m * n_pb + mu] = t;
          }
#pragma omp parallel for schedule(static)
        for (int m = 0; m < n_qp; ++m)
          for (int n = 0; n < n_qp; ++n) {
            zdouble t = 0.0;
            for (int mu = 0; mu < n_pb; ++mu) t += conj(Zb[(size_t)n * n_pb + mu]) * y[(size_t)m * n_pb + mu];
            out[(size_t)m * n_qp + n] -= w[(size_t)n * L + i] * t;
          }
      }
    }
    zoff += (size_t)n_band[k] * n_qp * n_pb;
    eoff += (size_t)n_band[k];
  }
  free(w);
  free(y);
}
