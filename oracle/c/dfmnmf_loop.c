/* dfmnmf_loop.c -- second FP64 CPU oracle of distributed FastMNMF, in plain C loops.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the library links or calls this file;
 * the tests compare it with the NumPy oracle (oracle/dfmnmf_oracle.py) so that
 * each of the two checks the other.  It shares no code with either the NumPy
 * oracle or the CUDA path: every step is written out as loops from the
 * paper's update rules, in double precision and double complex.
 *
 *   Eq. (2)          lambda[n][f][t] = sum_b W[n][f][b] H[n][b][t]
 *   Sec. IV-A        yhat[f][t][m]   = max(sum_n lambda[n][f][t] g[f][n][m], eps)
 *   Eq. (13)         V[f][k][mu][a][b] = (1/T) sum_t x_a conj(x_b) / yhat[f][t][o_k + mu]
 *   Eqs. (14)-(15)   for mu ascending: q = (Q_fk V_fk,mu)^{-1} e_mu (pseudo-inverse when the
 *                    smallest partial pivot is <= rtol max|entry|), q <- q / sqrt(max(Re q^H V q, eps)),
 *                    row mu of Q_fk <- q^H
 *   Sec. III-B       P[f][t][o_k + u] = |sum_v Q_fk[u][v] x[f][t][o_k + v]|^2
 *   Eqs. (8)-(10)    the multiplicative updates of W, H and g (yhat rebuilt before each)
 *   Eq. (12)         sum_{f,t,m} (P / yhat + ln yhat) - T sum_{f,k} ln |det Q_fk|^2
 *   Sec. II-A/III-B  Wiener filter c_n = Q_fk^{-1} diag(lambda_n g_n / yhat) Q_fk x_ftk
 *
 * Arrays (all C-contiguous, row-major): x [F][T][M] complex; Q [F][sum_k M_k^2]
 * complex, block k at offset sum_{k'<k} M_k'^2, row-major; V [F][sum_k M_k^3]
 * complex, block k at offset sum_{k'<k} M_k'^3 as [mu][a][b]; W [N][F][B];
 * H [N][B][T]; g [F][N][M]; P and yhat [F][T][M]; the Wiener output
 * [N][F][T][M] complex.  mics[k] = M_k, M = sum_k M_k.
 */
#include <complex.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>

typedef double complex cplx;

typedef struct {
  int F, T, K, N, B, M;
  const int* mics;
} dims_t;

static dims_t make_dims(int F, int T, int K, const int* mics, int N, int B) {
  dims_t d;
  d.F = F; d.T = T; d.K = K; d.N = N; d.B = B; d.mics = mics;
  d.M = 0;
  for (int k = 0; k < K; ++k) d.M += mics[k];
  return d;
}

static int mic_offset(const dims_t* d, int k) {
  int o = 0;
  for (int j = 0; j < k; ++j) o += d->mics[j];
  return o;
}

static int q_offset(const dims_t* d, int k) {
  int o = 0;
  for (int j = 0; j < k; ++j) o += d->mics[j] * d->mics[j];
  return o;
}

static int q_size(const dims_t* d) { return q_offset(d, d->K); }

static int v_offset(const dims_t* d, int k) {
  int o = 0;
  for (int j = 0; j < k; ++j) o += d->mics[j] * d->mics[j] * d->mics[j];
  return o;
}

static int v_size(const dims_t* d) { return v_offset(d, d->K); }

/* ------------------------------------------------------------------ model */

/* Eq. (2) */
static void source_psd(const dims_t* d, const double* W, const double* H, double* lam) {
  for (int n = 0; n < d->N; ++n)
    for (int f = 0; f < d->F; ++f)
      for (int t = 0; t < d->T; ++t) {
        double s = 0.0;
        for (int b = 0; b < d->B; ++b) s += W[((size_t)n * d->F + f) * d->B + b] * H[((size_t)n * d->B + b) * d->T + t];
        lam[((size_t)n * d->F + f) * d->T + t] = s;
      }
}

/* yhat with the Sec. IV-A floor */
static void model_variance(const dims_t* d, const double* lam, const double* g, double eps, double* y) {
  for (int f = 0; f < d->F; ++f)
    for (int t = 0; t < d->T; ++t)
      for (int m = 0; m < d->M; ++m) {
        double s = 0.0;
        for (int n = 0; n < d->N; ++n) s += lam[((size_t)n * d->F + f) * d->T + t] * g[((size_t)f * d->N + n) * d->M + m];
        y[((size_t)f * d->T + t) * d->M + m] = s > eps ? s : eps;
      }
}

/* ------------------------------------------------------- Eq. (13) */
static void covariances(const dims_t* d, const cplx* x, const double* y, cplx* V) {
  const int vs = v_size(d);
  for (int f = 0; f < d->F; ++f)
    for (int k = 0; k < d->K; ++k) {
      const int mk = d->mics[k], o = mic_offset(d, k);
      cplx* Vk = V + (size_t)f * vs + v_offset(d, k);
      for (int mu = 0; mu < mk; ++mu)
        for (int a = 0; a < mk; ++a)
          for (int b = 0; b < mk; ++b) {
            cplx s = 0.0;
            for (int t = 0; t < d->T; ++t) {
              const cplx* xt = x + ((size_t)f * d->T + t) * d->M + o;
              s += xt[a] * conj(xt[b]) / y[((size_t)f * d->T + t) * d->M + o + mu];
            }
            Vk[(mu * mk + a) * mk + b] = s / (double)d->T;
          }
    }
}

/* ------------------------------------------------ linear algebra (n <= 64) */

/* Solves A z = rhs by Gaussian elimination with partial pivoting (the first
 * largest |entry| of the column wins).  A (n x n) and rhs are overwritten.
 * Returns the smallest |pivot| in *minpiv and the largest |A_ij| of the input
 * in *maxabs. */
static void ge_solve(int n, cplx* A, cplx* rhs, cplx* z, double* minpiv, double* maxabs) {
  double mx = 0.0;
  for (int i = 0; i < n * n; ++i)
    if (cabs(A[i]) > mx) mx = cabs(A[i]);
  double mp = INFINITY;
  for (int c = 0; c < n; ++c) {
    int p = c;
    double best = cabs(A[c * n + c]);
    for (int r = c + 1; r < n; ++r)
      if (cabs(A[r * n + c]) > best) {
        best = cabs(A[r * n + c]);
        p = r;
      }
    if (p != c) {
      for (int j = 0; j < n; ++j) {
        const cplx tmp = A[c * n + j];
        A[c * n + j] = A[p * n + j];
        A[p * n + j] = tmp;
      }
      const cplx tmp = rhs[c];
      rhs[c] = rhs[p];
      rhs[p] = tmp;
    }
    const cplx piv = A[c * n + c];
    if (cabs(piv) < mp) mp = cabs(piv);
    if (piv == 0.0) continue;
    for (int r = c + 1; r < n; ++r) {
      const cplx l = A[r * n + c] / piv;
      for (int j = c; j < n; ++j) A[r * n + j] -= l * A[c * n + j];
      rhs[r] -= l * rhs[c];
    }
  }
  for (int i = n - 1; i >= 0; --i) {
    cplx s = rhs[i];
    for (int j = i + 1; j < n; ++j) s -= A[i * n + j] * z[j];
    z[i] = A[i * n + i] != 0.0 ? s / A[i * n + i] : s;
  }
  *minpiv = mp;
  *maxabs = mx;
}

/* z = pinv(A) e_mu through the singular value decomposition by one-sided
 * (Hestenes) Jacobi rotations: the columns of A are rotated pairwise until
 * orthogonal, G = A J with J unitary; then sigma_c = ||G[:, c]||, and
 * pinv(A) e_mu = sum_c J[:, c] conj(G[mu][c]) / sigma_c^2 over the sigma_c
 * above rtol * sigma_max. */
static void pinv_column(int n, const cplx* A, int mu, double rtol, cplx* z) {
  cplx* G = malloc(sizeof(cplx) * n * n);
  cplx* J = malloc(sizeof(cplx) * n * n);
  memcpy(G, A, sizeof(cplx) * n * n);
  for (int i = 0; i < n * n; ++i) J[i] = (i / n == i % n) ? 1.0 : 0.0;
  for (int sweep = 0; sweep < 100; ++sweep) {
    double worst = 0.0;
    for (int p = 0; p < n - 1; ++p)
      for (int q = p + 1; q < n; ++q) {
        double alpha = 0.0, beta = 0.0;
        cplx gamma = 0.0; /* G[:,p]^H G[:,q] */
        for (int r = 0; r < n; ++r) {
          alpha += creal(G[r * n + p] * conj(G[r * n + p]));
          beta += creal(G[r * n + q] * conj(G[r * n + q]));
          gamma += conj(G[r * n + p]) * G[r * n + q];
        }
        const double ag = cabs(gamma);
        if (!(ag > 1e-300) || !(ag > 1e-15 * sqrt(alpha * beta))) continue;
        if (ag / sqrt(alpha * beta) > worst) worst = ag / sqrt(alpha * beta);
        const cplx phase = gamma / ag;                  /* column q is first turned by conj(phase) */
        const double zeta = (beta - alpha) / (2.0 * ag);
        const double tn = (zeta >= 0.0 ? 1.0 : -1.0) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
        const double cs = 1.0 / sqrt(1.0 + tn * tn), sn = cs * tn;
        for (int r = 0; r < n; ++r) {
          const cplx gp = G[r * n + p], gq = G[r * n + q] * conj(phase);
          G[r * n + p] = cs * gp - sn * gq;
          G[r * n + q] = sn * gp + cs * gq;
          const cplx jp = J[r * n + p], jq = J[r * n + q] * conj(phase);
          J[r * n + p] = cs * jp - sn * jq;
          J[r * n + q] = sn * jp + cs * jq;
        }
      }
    if (worst < 1e-15) break;
  }
  double smax2 = 0.0;
  double* s2 = malloc(sizeof(double) * n);
  for (int c = 0; c < n; ++c) {
    double s = 0.0;
    for (int r = 0; r < n; ++r) s += creal(G[r * n + c] * conj(G[r * n + c]));
    s2[c] = s;
    if (s > smax2) smax2 = s;
  }
  for (int r = 0; r < n; ++r) z[r] = 0.0;
  for (int c = 0; c < n; ++c) {
    if (!(s2[c] > 0.0) || !(sqrt(s2[c]) > rtol * sqrt(smax2))) continue;
    const cplx coef = conj(G[mu * n + c]) / s2[c];
    for (int r = 0; r < n; ++r) z[r] += J[r * n + c] * coef;
  }
  free(s2);
  free(G);
  free(J);
}

/* ------------------------------------------------- Eqs. (14)-(15) */
static int ip_update(const dims_t* d, const cplx* V, cplx* Q, double eps, double rtol) {
  const int qs = q_size(d), vs = v_size(d);
  int singular_count = 0;
  for (int f = 0; f < d->F; ++f)
    for (int k = 0; k < d->K; ++k) {
      const int mk = d->mics[k];
      cplx* Qk = Q + (size_t)f * qs + q_offset(d, k);
      const cplx* Vk = V + (size_t)f * vs + v_offset(d, k);
      cplx* A = malloc(sizeof(cplx) * mk * mk);
      cplx* A0 = malloc(sizeof(cplx) * mk * mk);
      cplx* e = malloc(sizeof(cplx) * mk);
      cplx* q = malloc(sizeof(cplx) * mk);
      for (int mu = 0; mu < mk; ++mu) {
        const cplx* Vm = Vk + (size_t)mu * mk * mk;
        for (int i = 0; i < mk; ++i)
          for (int j = 0; j < mk; ++j) {
            cplx s = 0.0;
            for (int l = 0; l < mk; ++l) s += Qk[i * mk + l] * Vm[l * mk + j];
            A[i * mk + j] = s;
            A0[i * mk + j] = s;
          }
        for (int i = 0; i < mk; ++i) e[i] = (i == mu) ? 1.0 : 0.0;
        double minpiv, maxabs;
        ge_solve(mk, A, e, q, &minpiv, &maxabs);
        if (!(minpiv > rtol * maxabs)) {
          pinv_column(mk, A0, mu, rtol, q);
          ++singular_count;
        }
        double s = 0.0; /* Re q^H V_mu q */
        for (int a = 0; a < mk; ++a)
          for (int b = 0; b < mk; ++b) s += creal(conj(q[a]) * Vm[a * mk + b] * q[b]);
        const double r = 1.0 / sqrt(s > eps ? s : eps);
        for (int j = 0; j < mk; ++j) Qk[mu * mk + j] = conj(q[j]) * r;
      }
      free(A);
      free(A0);
      free(e);
      free(q);
    }
  return singular_count;
}

/* ------------------------------------------------- projected power */
static void projected_power(const dims_t* d, const cplx* x, const cplx* Q, double* P) {
  const int qs = q_size(d);
  for (int f = 0; f < d->F; ++f)
    for (int k = 0; k < d->K; ++k) {
      const int mk = d->mics[k], o = mic_offset(d, k);
      const cplx* Qk = Q + (size_t)f * qs + q_offset(d, k);
      for (int t = 0; t < d->T; ++t) {
        const cplx* xt = x + ((size_t)f * d->T + t) * d->M + o;
        for (int u = 0; u < mk; ++u) {
          cplx yv = 0.0;
          for (int v = 0; v < mk; ++v) yv += Qk[u * mk + v] * xt[v];
          P[((size_t)f * d->T + t) * d->M + o + u] = creal(yv * conj(yv));
        }
      }
    }
}

/* ------------------------------------------------- Eqs. (8)-(10) */

/* The two sums over m that Eqs. (8) and (9) share:
 *   num_part[n][f][t] = sum_m g[f][n][m] P[f][t][m] / yhat^2,
 *   den_part[n][f][t] = sum_m g[f][n][m] / yhat,
 * with yhat rebuilt from the current W, H and g. */
static void nmf_parts(const dims_t* d, const double* W, const double* H, const double* g, const double* P,
                      double eps, double* num_part, double* den_part) {
  const size_t nft = (size_t)d->N * d->F * d->T, ftm = (size_t)d->F * d->T * d->M;
  double* lam = malloc(sizeof(double) * nft);
  double* y = malloc(sizeof(double) * ftm);
  source_psd(d, W, H, lam);
  model_variance(d, lam, g, eps, y);
  for (int n = 0; n < d->N; ++n)
    for (int f = 0; f < d->F; ++f)
      for (int t = 0; t < d->T; ++t) {
        double a = 0.0, b = 0.0;
        for (int m = 0; m < d->M; ++m) {
          const double gv = g[((size_t)f * d->N + n) * d->M + m];
          const double yv = y[((size_t)f * d->T + t) * d->M + m];
          a += gv * P[((size_t)f * d->T + t) * d->M + m] / (yv * yv);
          b += gv / yv;
        }
        num_part[((size_t)n * d->F + f) * d->T + t] = a;
        den_part[((size_t)n * d->F + f) * d->T + t] = b;
      }
  free(lam);
  free(y);
}

/* Eq. (8): W[n][f][b] *= sqrt(sum_t H num_part / max(sum_t H den_part, eps)) */
static void update_W(const dims_t* d, double* W, const double* H, const double* g, const double* P, double eps) {
  const size_t nft = (size_t)d->N * d->F * d->T;
  double* a = malloc(sizeof(double) * nft);
  double* b = malloc(sizeof(double) * nft);
  nmf_parts(d, W, H, g, P, eps, a, b);
  for (int n = 0; n < d->N; ++n)
    for (int f = 0; f < d->F; ++f)
      for (int k = 0; k < d->B; ++k) {
        double num = 0.0, den = 0.0;
        for (int t = 0; t < d->T; ++t) {
          const double h = H[((size_t)n * d->B + k) * d->T + t];
          num += h * a[((size_t)n * d->F + f) * d->T + t];
          den += h * b[((size_t)n * d->F + f) * d->T + t];
        }
        W[((size_t)n * d->F + f) * d->B + k] *= sqrt(num / (den > eps ? den : eps));
      }
  free(a);
  free(b);
}

/* Eq. (9): H[n][b][t] *= sqrt(sum_f W num_part / max(sum_f W den_part, eps)) */
static void update_H(const dims_t* d, const double* W, double* H, const double* g, const double* P, double eps) {
  const size_t nft = (size_t)d->N * d->F * d->T;
  double* a = malloc(sizeof(double) * nft);
  double* b = malloc(sizeof(double) * nft);
  nmf_parts(d, W, H, g, P, eps, a, b);
  for (int n = 0; n < d->N; ++n)
    for (int k = 0; k < d->B; ++k)
      for (int t = 0; t < d->T; ++t) {
        double num = 0.0, den = 0.0;
        for (int f = 0; f < d->F; ++f) {
          const double w = W[((size_t)n * d->F + f) * d->B + k];
          num += w * a[((size_t)n * d->F + f) * d->T + t];
          den += w * b[((size_t)n * d->F + f) * d->T + t];
        }
        H[((size_t)n * d->B + k) * d->T + t] *= sqrt(num / (den > eps ? den : eps));
      }
  free(a);
  free(b);
}

/* Eq. (10): g[f][n][m] *= sqrt(sum_t lambda P / yhat^2 / max(sum_t lambda / yhat, eps)) */
static void update_g(const dims_t* d, const double* W, const double* H, double* g, const double* P, double eps) {
  const size_t nft = (size_t)d->N * d->F * d->T, ftm = (size_t)d->F * d->T * d->M;
  double* lam = malloc(sizeof(double) * nft);
  double* y = malloc(sizeof(double) * ftm);
  double* gn = malloc(sizeof(double) * (size_t)d->F * d->N * d->M);
  source_psd(d, W, H, lam);
  model_variance(d, lam, g, eps, y);
  for (int f = 0; f < d->F; ++f)
    for (int n = 0; n < d->N; ++n)
      for (int m = 0; m < d->M; ++m) {
        double num = 0.0, den = 0.0;
        for (int t = 0; t < d->T; ++t) {
          const double l = lam[((size_t)n * d->F + f) * d->T + t];
          const double yv = y[((size_t)f * d->T + t) * d->M + m];
          num += l * P[((size_t)f * d->T + t) * d->M + m] / (yv * yv);
          den += l / yv;
        }
        gn[((size_t)f * d->N + n) * d->M + m] = g[((size_t)f * d->N + n) * d->M + m] * sqrt(num / (den > eps ? den : eps));
      }
  memcpy(g, gn, sizeof(double) * (size_t)d->F * d->N * d->M);
  free(lam);
  free(y);
  free(gn);
}

/* ln |det A|^2 from the pivots of Gaussian elimination with partial pivoting */
static double log_abs_det_sq(int n, const cplx* A_in) {
  cplx* A = malloc(sizeof(cplx) * n * n);
  memcpy(A, A_in, sizeof(cplx) * n * n);
  double acc = 0.0;
  for (int c = 0; c < n; ++c) {
    int p = c;
    double best = cabs(A[c * n + c]);
    for (int r = c + 1; r < n; ++r)
      if (cabs(A[r * n + c]) > best) {
        best = cabs(A[r * n + c]);
        p = r;
      }
    if (p != c)
      for (int j = 0; j < n; ++j) {
        const cplx tmp = A[c * n + j];
        A[c * n + j] = A[p * n + j];
        A[p * n + j] = tmp;
      }
    const cplx piv = A[c * n + c];
    acc += log(creal(piv * conj(piv)));
    if (piv == 0.0) continue;
    for (int r = c + 1; r < n; ++r) {
      const cplx l = A[r * n + c] / piv;
      for (int j = c; j < n; ++j) A[r * n + j] -= l * A[c * n + j];
    }
  }
  free(A);
  return acc;
}

/* inverse of A (n x n) by Gauss-Jordan elimination with partial pivoting */
static void invert(int n, const cplx* A_in, cplx* inv) {
  cplx* A = malloc(sizeof(cplx) * n * n);
  memcpy(A, A_in, sizeof(cplx) * n * n);
  for (int i = 0; i < n * n; ++i) inv[i] = (i / n == i % n) ? 1.0 : 0.0;
  for (int c = 0; c < n; ++c) {
    int p = c;
    double best = cabs(A[c * n + c]);
    for (int r = c + 1; r < n; ++r)
      if (cabs(A[r * n + c]) > best) {
        best = cabs(A[r * n + c]);
        p = r;
      }
    for (int j = 0; j < n && p != c; ++j) {
      cplx tmp = A[c * n + j]; A[c * n + j] = A[p * n + j]; A[p * n + j] = tmp;
      tmp = inv[c * n + j]; inv[c * n + j] = inv[p * n + j]; inv[p * n + j] = tmp;
    }
    const cplx piv = A[c * n + c];
    for (int j = 0; j < n; ++j) {
      A[c * n + j] /= piv;
      inv[c * n + j] /= piv;
    }
    for (int r = 0; r < n; ++r) {
      if (r == c) continue;
      const cplx l = A[r * n + c];
      for (int j = 0; j < n; ++j) {
        A[r * n + j] -= l * A[c * n + j];
        inv[r * n + j] -= l * inv[c * n + j];
      }
    }
  }
  free(A);
}

/* ================================================== entry points (ctypes) */

void oracle_loop_source_psd(int F, int T, int K, const int* mics, int N, int B, const double* W, const double* H,
                            double* lam) {
  const dims_t d = make_dims(F, T, K, mics, N, B);
  source_psd(&d, W, H, lam);
}

void oracle_loop_covariances(int F, int T, int K, const int* mics, int N, int B, const cplx* x, const double* W,
                             const double* H, const double* g, double eps, cplx* V) {
  const dims_t d = make_dims(F, T, K, mics, N, B);
  double* lam = malloc(sizeof(double) * (size_t)N * F * T);
  double* y = malloc(sizeof(double) * (size_t)F * T * d.M);
  source_psd(&d, W, H, lam);
  model_variance(&d, lam, g, eps, y);
  covariances(&d, x, y, V);
  free(lam);
  free(y);
}

int oracle_loop_ip_update(int F, int T, int K, const int* mics, const cplx* V, cplx* Q, double eps, double rtol) {
  const dims_t d = make_dims(F, T, K, mics, 1, 1);
  return ip_update(&d, V, Q, eps, rtol);
}

void oracle_loop_projected_power(int F, int T, int K, const int* mics, const cplx* x, const cplx* Q, double* P) {
  const dims_t d = make_dims(F, T, K, mics, 1, 1);
  projected_power(&d, x, Q, P);
}

void oracle_loop_update_W(int F, int T, int K, const int* mics, int N, int B, double* W, const double* H,
                          const double* g, const double* P, double eps) {
  const dims_t d = make_dims(F, T, K, mics, N, B);
  update_W(&d, W, H, g, P, eps);
}

void oracle_loop_update_H(int F, int T, int K, const int* mics, int N, int B, const double* W, double* H,
                          const double* g, const double* P, double eps) {
  const dims_t d = make_dims(F, T, K, mics, N, B);
  update_H(&d, W, H, g, P, eps);
}

void oracle_loop_update_g(int F, int T, int K, const int* mics, int N, int B, const double* W, const double* H,
                          double* g, const double* P, double eps) {
  const dims_t d = make_dims(F, T, K, mics, N, B);
  update_g(&d, W, H, g, P, eps);
}

/* n_iter MM iterations in place (Sec. III-B order: IP of every block, then
 * W, H, g).  Returns the number of pseudo-inverse solves taken. */
int oracle_loop_iterate(int F, int T, int K, const int* mics, int N, int B, const cplx* x, cplx* Q, double* W,
                        double* H, double* g, int n_iter, double eps, double rtol) {
  const dims_t d = make_dims(F, T, K, mics, N, B);
  cplx* V = malloc(sizeof(cplx) * (size_t)F * v_size(&d));
  double* P = malloc(sizeof(double) * (size_t)F * T * d.M);
  double* lam = malloc(sizeof(double) * (size_t)N * F * T);
  double* y = malloc(sizeof(double) * (size_t)F * T * d.M);
  int singular = 0;
  for (int it = 0; it < n_iter; ++it) {
    source_psd(&d, W, H, lam);
    model_variance(&d, lam, g, eps, y);
    covariances(&d, x, y, V);
    singular += ip_update(&d, V, Q, eps, rtol);
    projected_power(&d, x, Q, P);
    update_W(&d, W, H, g, P, eps);
    update_H(&d, W, H, g, P, eps);
    update_g(&d, W, H, g, P, eps);
  }
  free(V);
  free(P);
  free(lam);
  free(y);
  return singular;
}

/* Eq. (12) */
double oracle_loop_neg_loglik(int F, int T, int K, const int* mics, int N, int B, const cplx* x, const cplx* Q,
                              const double* W, const double* H, const double* g, double eps) {
  const dims_t d = make_dims(F, T, K, mics, N, B);
  double* P = malloc(sizeof(double) * (size_t)F * T * d.M);
  double* lam = malloc(sizeof(double) * (size_t)N * F * T);
  double* y = malloc(sizeof(double) * (size_t)F * T * d.M);
  projected_power(&d, x, Q, P);
  source_psd(&d, W, H, lam);
  model_variance(&d, lam, g, eps, y);
  double data = 0.0;
  for (size_t i = 0; i < (size_t)F * T * d.M; ++i) data += P[i] / y[i] + log(y[i]);
  double ld = 0.0;
  const int qs = q_size(&d);
  for (int f = 0; f < F; ++f)
    for (int k = 0; k < K; ++k) ld += log_abs_det_sq(mics[k], Q + (size_t)f * qs + q_offset(&d, k));
  free(P);
  free(lam);
  free(y);
  return data - (double)T * ld;
}

/* Wiener filter: out[n][f][t][o_k + u] = (Q_fk^{-1} diag(lambda_n g_n / yhat) Q_fk x_ftk)_u */
void oracle_loop_wiener(int F, int T, int K, const int* mics, int N, int B, const cplx* x, const cplx* Q,
                        const double* W, const double* H, const double* g, double eps, cplx* out) {
  const dims_t d = make_dims(F, T, K, mics, N, B);
  double* lam = malloc(sizeof(double) * (size_t)N * F * T);
  double* y = malloc(sizeof(double) * (size_t)F * T * d.M);
  source_psd(&d, W, H, lam);
  model_variance(&d, lam, g, eps, y);
  const int qs = q_size(&d);
  for (int f = 0; f < F; ++f)
    for (int k = 0; k < K; ++k) {
      const int mk = mics[k], o = mic_offset(&d, k);
      const cplx* Qk = Q + (size_t)f * qs + q_offset(&d, k);
      cplx* Qi = malloc(sizeof(cplx) * mk * mk);
      cplx* z = malloc(sizeof(cplx) * mk);
      cplx* u = malloc(sizeof(cplx) * mk);
      invert(mk, Qk, Qi);
      for (int t = 0; t < T; ++t) {
        const cplx* xt = x + ((size_t)f * T + t) * d.M + o;
        for (int a = 0; a < mk; ++a) {
          z[a] = 0.0;
          for (int b = 0; b < mk; ++b) z[a] += Qk[a * mk + b] * xt[b];
        }
        for (int n = 0; n < N; ++n) {
          for (int a = 0; a < mk; ++a) {
            const double gain = lam[((size_t)n * F + f) * T + t] * g[((size_t)f * N + n) * d.M + o + a] /
                                y[((size_t)f * T + t) * d.M + o + a];
            u[a] = gain * z[a];
          }
          for (int a = 0; a < mk; ++a) {
            cplx s = 0.0;
            for (int b = 0; b < mk; ++b) s += Qi[a * mk + b] * u[b];
            out[(((size_t)n * F + f) * T + t) * d.M + o + a] = s;
          }
        }
      }
      free(Qi);
      free(z);
      free(u);
    }
  free(lam);
  free(y);
}
