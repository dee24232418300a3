// adjoint.cu -- reverse-mode gradient of unrolled MM iterations.
//
// The loss is a function of the state reached after n_iter iterations of
// the FP32 form (Sec. III-B schedule): Eq. (12), or the mean squared error
// of the multichannel Wiener filter output against given source images.
// The gradient with respect to the initial state (Q0, W0, H0, g0) is the
// reverse pass of the iteration written out by hand:
//
//   forward of one iteration (recomputed in FP64 from the stored state)
//     lambda0 = W H, y0 = sum_n lambda0 g                      (Eq. 2)
//     V_k,mu  = (1/T) sum_t x x^H / yhat0_mu                   (Eq. 13)
//     rows mu of every block: A = Q V_mu, q = A^-1 e_mu,
//       q <- q / sqrt(max(Re q^H V_mu q, eps)), row mu <- q^H  (Eqs. 14, 15)
//     P = |Q' x|^2
//     W' = W sqrt(num/den)  num = A0 H^T, den = D0 H^T        (Eq. 8)
//     H' = H sqrt(num/den)  num = W'^T A1, den = W'^T D1      (Eq. 9)
//     g' = g sqrt(num/den)  num = sum_t lambda2 P / yhat2^2,
//                           den = sum_t lambda2 / yhat2        (Eq. 10)
//     with A = sum_m g P / yhat^2, D = sum_m g / yhat at the current model;
//   reverse: the adjoints of (g', H', W', P, Q', V, yhat, lambda) in the
//   opposite order, each the transpose of the step's linearisation
//   (conjugate transpose for complex quantities, the floors of Sec. IV-A
//   passing no gradient where they hold).
//
// The forward iterations themselves are the context's own (the captured
// FP32 iteration graph); the state is stored every `every` iterations and
// each segment is recomputed from its checkpoint during the reverse sweep.
// The loss and its adjoint are FP64.  Inside the unrolled iterations the IP
// side (V, the IP rows, P = |Q x|^2 and their adjoints) is FP64 and the NMF
// side (model, statistics, multiplicative updates and their adjoints) is
// single precision, as in the forward iterations it differentiates: GB300
// issues FP64 at about 1/64 of its FP32 rate.  Complex adjoints are
// dL/dRe + i dL/dIm.
#include "../../include/dfmnmf.h"
#include "common.cuh"
#include "internal.h"

#include <algorithm>
#include <type_traits>
#include <cstdarg>
#include <cstdio>
#include <utility>

// The NMF side of the reverse pass (the recomputed model, statistics and multiplicative
// updates, and their adjoints) in one real type: single precision through the unrolled
// iterations, double precision for the loss and its adjoint.
template <class R>
struct AdjSide {
  R *Wd, *Hd, *gd;  // the state being differentiated: [N][F][B], [N][B][T], [F][N][M]
  R *lam0, *lam1, *lam2, *y0, *y1, *y2, *r0, *r1, *r2, *P, *A0, *D0, *A1, *D1;
  R *numW, *denW, *W1, *numH, *denH, *H1, *numG, *denG;
  R *Wb, *Wb1, *Hb, *Hb1, *gb, *gb1, *lamb, *yb, *Pb, *Ab, *Db, *nb, *db;
};

struct dfmnmf_adj {
  dfmnmf_ctx* c;
  int n_iter, every, n_ckpt, device;
  // stored states (context layouts: Q complex128 [F][K][MK][MK], W [N][F][B], H [N][B][Tp], g [F][N][M])
  double2* ckQ;
  float *ckW, *ckH, *ckg;
  double2* sgQ;  // the states of one segment
  float *sgW, *sgH, *sgg;
  double2* fnQ;  // the final state
  float *fnW, *fnH, *fng;
  // FP64 copies of the state being differentiated and the recomputed forward
  double *Wd, *Hd, *gd;  // [N][F][B], [N][B][T], [F][N][M]
  double2* Qd;           // [F][K][MK][MK]
  double *lam0, *lam1, *lam2, *y0, *y1, *y2, *P, *A0, *D0, *A1, *D1;
  double *r0, *r1, *r2;  // 1 / max(y, eps) of y0, y1, y2: every division by the model becomes a product
  double *numW, *denW, *W1, *numH, *denH, *H1, *numG, *denG;
  double2 *V, *Qs;  // V [F][K][MK][MK][MK]; Qs [F][K][MK+1][MK][MK] (rows before each IP row update)
  // adjoints
  double2 *Qb, *Qb1;
  double *Wb, *Wb1, *Hb, *Hb1, *gb, *gb1;
  double *lamb, *yb, *Pb, *Ab, *Db, *nb, *db;
  double2* Vb;
  double* Vh;  // packed Hermitian parts of Vb (k_a_Vh)
  // Wiener-filter loss
  double2 *Binv, *ubar, *cvec, *zbar;
  double* G4;
  double* red;      // loss accumulator
  unsigned* flags;  // [0] a system below the singular threshold
  AdjSide<float> sf;  // single-precision NMF side of the unrolled iterations
  double2* x64;       // the observation in FP64 [F][T][M]
  double* r0d;        // FP64 copy of sf.r0 for the covariances of Eq. 13
};

namespace dfm {
namespace {

int afail(int code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  set_last_error(buf);
  return code;
}

#define ACK(call)                                                                                     \
  do {                                                                                                \
    cudaError_t e_ = (call);                                                                          \
    if (e_ != cudaSuccess)                                                                            \
      return afail(DFMNMF_ECUDA, "%s failed: %s (%s:%d)", #call, cudaGetErrorString(e_), __FILE__, __LINE__); \
  } while (0)

#define ACKE(call)                       \
  do {                                   \
    cudaError_t e_ = (call);             \
    if (e_ != cudaSuccess) return e_;    \
  } while (0)

template <class R> __device__ __forceinline__ R flo(R y, R eps) { return y > eps ? y : eps; }
__device__ __forceinline__ double2 cadd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ double2 csub(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
  return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ double2 cmulc(double2 a, double2 b) {  // a conj(b)
  return make_double2(a.x * b.x + a.y * b.y, a.y * b.x - a.x * b.y);
}
__device__ __forceinline__ double2 cconj(double2 a) { return make_double2(a.x, -a.y); }
__device__ __forceinline__ double2 cscale(double2 a, double s) { return make_double2(a.x * s, a.y * s); }
__device__ __forceinline__ double cabs2(double2 a) { return a.x * a.x + a.y * a.y; }
__device__ __forceinline__ double2 crecip(double2 a) {  // 1 / a = conj(a) / |a|^2
  const double d = cabs2(a);
  return make_double2(a.x / d, -a.y / d);
}
__device__ __forceinline__ double2 ld(const float2* p) {
  const float2 v = __ldg(p);
  return make_double2((double)v.x, (double)v.y);
}
// the observation converted once to FP64 (conversions run on the FP64 pipe too)
__device__ __forceinline__ double2 ld(const double2* p) { return __ldg(p); }
// Sum over the 32 lanes of a warp in a fixed butterfly order (deterministic).
template <class R> __device__ __forceinline__ R warp_sum(R v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Inverse by Gauss-Jordan elimination with partial pivoting (n <= 4, fully unrolled: the
// pivot row is brought up by compare-and-swap so every index stays static; the columns of the
// identity are the right-hand sides).  Returns ln |det A|^2 (sum of ln |pivot|^2).
template <int n>
__device__ double gj_inverse(double2 (&A)[n][n], double2 (&X)[n][n]) {
#pragma unroll
  for (int i = 0; i < n; ++i)
#pragma unroll
    for (int j = 0; j < n; ++j) X[i][j] = make_double2(i == j ? 1.0 : 0.0, 0.0);
  double ld2 = 0.0;
#pragma unroll
  for (int c = 0; c < n; ++c) {
#pragma unroll
    for (int rr = c + 1; rr < n; ++rr)
      if (cabs2(A[rr][c]) > cabs2(A[c][c])) {
#pragma unroll
        for (int j = 0; j < n; ++j) {
          double2 t = A[c][j];
          A[c][j] = A[rr][j];
          A[rr][j] = t;
          t = X[c][j];
          X[c][j] = X[rr][j];
          X[rr][j] = t;
        }
      }
    const double2 piv = A[c][c];
    ld2 += log(cabs2(piv));
    const double2 inv = cabs2(piv) > 0.0 ? crecip(piv) : make_double2(0.0, 0.0);
#pragma unroll
    for (int j = 0; j < n; ++j) {
      A[c][j] = cmul(A[c][j], inv);
      X[c][j] = cmul(X[c][j], inv);
    }
#pragma unroll
    for (int rr = 0; rr < n; ++rr) {
      if (rr == c) continue;
      const double2 m = A[rr][c];
#pragma unroll
      for (int j = 0; j < n; ++j) {
        A[rr][j] = csub(A[rr][j], cmul(m, A[c][j]));
        X[rr][j] = csub(X[rr][j], cmul(m, X[c][j]));
      }
    }
  }
  return ld2;
}

// ---------------------------------------------------------------- conversions and products
// the state (context layouts, FP32) to arrays of type R; H loses its row padding
template <class R>
__global__ void k_a_tod(const float* __restrict__ W, const float* __restrict__ H, const float* __restrict__ g,
                        R* __restrict__ Wd, R* __restrict__ Hd, R* __restrict__ gd, size_t nW,
                        size_t nH, size_t ng, int T, int Tp) {
  const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < nW) {
    Wd[i] = (R)W[i];
  } else if (i < nW + nH) {
    const size_t j = i - nW;
    Hd[j] = (R)H[(j / T) * Tp + j % T];
  } else if (i < nW + nH + ng) {
    const size_t j = i - nW - nH;
    gd[j] = (R)g[j];
  }
}

// out[n][f][t] = sum_b X[n][f][b] Y[n][b][t]
template <class R>
__global__ void k_a_nmf_b(const R* __restrict__ X, const R* __restrict__ Y, R* __restrict__ out, int N,
                          int F, int B, int T) {
  const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (size_t)N * F * T) return;
  const int t = (int)(i % T), f = (int)((i / T) % F), n = (int)(i / ((size_t)F * T));
  const R* x = X + ((size_t)n * F + f) * B;
  const R* y = Y + (size_t)n * B * T + t;
  R s = R(0);
  for (int b = 0; b < B; ++b) s += x[b] * y[(size_t)b * T];
  out[i] = s;
}

// out[n][f][b] (+)= sum_t X[n][f][t] Y[n][b][t]; one warp per output, lanes over t
template <class R>
__global__ void k_a_nmf_t(const R* __restrict__ X, const R* __restrict__ Y, R* __restrict__ out, int N,
                          int F, int B, int T, int acc) {
  const size_t w = ((size_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (w >= (size_t)N * F * B) return;
  const int b = (int)(w % B), f = (int)((w / B) % F), n = (int)(w / ((size_t)F * B));
  const R* x = X + ((size_t)n * F + f) * T;
  const R* y = Y + ((size_t)n * B + b) * T;
  R s = R(0);
  for (int t = lane; t < T; t += 32) s += x[t] * y[t];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if (lane == 0) out[w] = (acc ? out[w] : R(0)) + s;
}

// out[n][b][t] (+)= sum_f X[n][f][b] Y[n][f][t].  CTA = (32 frames, one (n, b)); its 8 warps
// take every 8th frequency and their partial sums are added in warp order through shared
// memory (a fixed order: the result does not depend on scheduling).
constexpr int NMF_F_WARPS = 8;
template <class R>
__global__ void __launch_bounds__(32 * NMF_F_WARPS) k_a_nmf_f(const R* __restrict__ X,
                                                             const R* __restrict__ Y,
                                                             R* __restrict__ out, int N, int F, int B, int T,
                                                             int acc) {
  __shared__ R part[NMF_F_WARPS][32];
  const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5;
  const int t = blockIdx.x * 32 + lane;
  const int b = (int)(blockIdx.y % B), n = (int)(blockIdx.y / B);
  R s = R(0);
  if (t < T)
    for (int f = wp; f < F; f += NMF_F_WARPS)
      s += X[((size_t)n * F + f) * B + b] * Y[((size_t)n * F + f) * T + t];
  part[wp][lane] = s;
  __syncthreads();
  if (wp == 0 && t < T) {
    R v = R(0);
#pragma unroll
    for (int w = 0; w < NMF_F_WARPS; ++w) v += part[w][lane];
    const size_t i = ((size_t)n * B + b) * T + t;
    out[i] = (acc ? out[i] : R(0)) + v;
  }
}

// y[f][t][m] = sum_n lam[n][f][t] g[f][n][m] (before the floor) and ry = 1 / max(y, eps).
// GB300 issues FP64 at a small fraction of its FP32 rate and a division costs
// about ten FP64 instructions, so the reverse kernels multiply by ry instead
// of dividing by the model.
template <class R>
__global__ void k_a_y(const R* __restrict__ lam, const R* __restrict__ g, R* __restrict__ y,
                      R* __restrict__ ry, int N, int F, int T, int M, R eps) {
  const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (size_t)F * T * M) return;
  const int m = (int)(i % M), t = (int)((i / M) % T), f = (int)(i / ((size_t)T * M));
  R s = R(0);
  for (int n = 0; n < N; ++n) s += lam[((size_t)n * F + f) * T + t] * g[((size_t)f * N + n) * M + m];
  y[i] = s;
  ry[i] = R(1) / flo(s, eps);
}

// V[f][k][mu][a][b] = (1/T) sum_t x_a conj(x_b) / yhat0[f][t][o_k + mu]   (Eq. 13)
// One warp per (f, k) and pair a <= b (V[b][a] = conj V[a][b]), lanes over t: the product
// x_a conj(x_b) is formed once per frame and weighted by the reciprocals r0 of all MK
// microphones.
template <int MK>
__global__ void k_a_V(const double2* __restrict__ x, const double* __restrict__ r0, double2* __restrict__ V, int F,
                      int T, int K) {
  constexpr int NP = MK * (MK + 1) / 2;
  const size_t w = ((size_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (w >= (size_t)F * K * NP) return;
  int pidx = (int)(w % NP), a = 0;
  while (pidx >= MK - a) {  // pair index -> (a, b), a <= b, row by row
    pidx -= MK - a;
    ++a;
  }
  const int b = a + pidx;
  const int k = (int)((w / NP) % K), f = (int)(w / ((size_t)NP * K));
  const int M = K * MK, o = k * MK;
  double sr[MK], si[MK];
#pragma unroll
  for (int mu = 0; mu < MK; ++mu) sr[mu] = si[mu] = 0.0;
  for (int t = lane; t < T; t += 32) {
    const size_t r = ((size_t)f * T + t) * M + o;
    const double2 p = cmulc(ld(x + r + a), ld(x + r + b));
#pragma unroll
    for (int mu = 0; mu < MK; ++mu) {
      const double wv = r0[r + mu];
      sr[mu] += wv * p.x;
      si[mu] += wv * p.y;
    }
  }
#pragma unroll
  for (int mu = 0; mu < MK; ++mu) {
    sr[mu] = warp_sum(sr[mu]);
    si[mu] = warp_sum(si[mu]);
  }
  if (lane == 0) {
#pragma unroll
    for (int mu = 0; mu < MK; ++mu) {
      double2* Vm = V + (((size_t)f * K + k) * MK + mu) * MK * MK;
      const double vr = sr[mu] / T, vi = si[mu] / T;
      Vm[a * MK + b] = make_double2(vr, vi);
      if (a != b) Vm[b * MK + a] = make_double2(vr, -vi);
    }
  }
}

// P[f][t][o_k + a] = |(Q_fk x_ftk)_a|^2 (formed in FP64, stored as RR); block (f, k) of Q at
// Q + (f K + k) * bstride
template <class RR>
__global__ void k_a_P(const double2* __restrict__ x, const double2* __restrict__ Q, size_t bstride,
                      RR* __restrict__ P, int F, int T, int K, int MK) {
  const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (size_t)F * T * K) return;
  const int k = (int)(i % K), t = (int)((i / K) % T), f = (int)(i / ((size_t)K * T));
  const int M = K * MK, o = k * MK;
  const double2* q = Q + ((size_t)f * K + k) * bstride;
  const double2* xr = x + ((size_t)f * T + t) * M + o;
  for (int a = 0; a < MK; ++a) {
    double2 z = make_double2(0.0, 0.0);
    for (int c2 = 0; c2 < MK; ++c2) z = cadd(z, cmul(q[a * MK + c2], ld(xr + c2)));
    P[((size_t)f * T + t) * M + o + a] = (RR)cabs2(z);
  }
}

// A[n][f][t] = sum_m g P / yhat^2, D[n][f][t] = sum_m g / yhat; one thread per (f, t) for all
// sources, P / yhat^2 and 1 / yhat formed once per microphone
template <class R>
__global__ void k_a_AD(const R* __restrict__ P, const R* __restrict__ ry, const R* __restrict__ g,
                       R* __restrict__ A, R* __restrict__ D, int N, int F, int T, int M) {
  const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (size_t)F * T) return;
  const int t = (int)(i % T), f = (int)(i / T);
  const size_t r = i * M;
  R a[16], d[16];
#pragma unroll
  for (int n = 0; n < 16; ++n) a[n] = d[n] = R(0);
  for (int m = 0; m < M; ++m) {
    const R rv = ry[r + m], u = P[r + m] * (rv * rv);
#pragma unroll
    for (int n = 0; n < 16; ++n)
      if (n < N) {
        const R gg = g[((size_t)f * N + n) * M + m];
        a[n] += gg * u;
        d[n] += gg * rv;
      }
  }
#pragma unroll
  for (int n = 0; n < 16; ++n)
    if (n < N) {
      A[((size_t)n * F + f) * T + t] = a[n];
      D[((size_t)n * F + f) * T + t] = d[n];
    }
}

// out = theta sqrt(num / max(den, eps))   (Eqs. 8-10)
template <class R>
__global__ void k_a_mu(const R* __restrict__ th, const R* __restrict__ num, const R* __restrict__ den,
                       R* __restrict__ out, size_t n, R eps) {
  const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = th[i] * sqrt(num[i] / flo(den[i], eps));
}

// num[f][n][m] = sum_t lam P / yhat^2, den = sum_t lam / yhat   (Eq. 10); one warp per
// output, lanes over t
template <class R>
__global__ void k_a_gnum(const R* __restrict__ lam, const R* __restrict__ P, const R* __restrict__ ry,
                         R* __restrict__ num, R* __restrict__ den, int N, int F, int T, int M) {
  const size_t i = ((size_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (i >= (size_t)F * N * M) return;
  const int m = (int)(i % M), n = (int)((i / M) % N), f = (int)(i / ((size_t)M * N));
  const R* l = lam + ((size_t)n * F + f) * T;
  R a = R(0), d = R(0);
  for (int t = lane; t < T; t += 32) {
    const size_t r = ((size_t)f * T + t) * M + m;
    const R rv = ry[r];
    a += l[t] * P[r] * (rv * rv);
    d += l[t] * rv;
  }
  a = warp_sum(a);
  d = warp_sum(d);
  if (lane == 0) {
    num[i] = a;
    den[i] = d;
  }
}

// ---------------------------------------------------------------- lane-parallel block algebra
// One MK x MK block (MK <= 4) per 16-lane half warp: lane sb + e holds entry (i, j) = (e / MK,
// e % MK) of a matrix for e < MK^2 (the other lanes carry don't-care values and contribute zeros
// to sums); a vector v is held in "row layout" (lane (i, j) holds v_i) or "column layout" (lane
// (i, j) holds v_j).  GB300 issues an FP64 warp instruction at a small fraction of the FP32
// rate, so a block per thread leaves each thread a long serial FP64 chain; a block per half warp
// divides the chain by the block size.
__device__ __forceinline__ double2 shfl2(double2 v, int src) {
  return make_double2(__shfl_sync(0xffffffffu, v.x, src), __shfl_sync(0xffffffffu, v.y, src));
}
// sum over the 16 lanes of a half warp (xor butterfly, fixed order)
__device__ __forceinline__ double half_sum(double v) {
#pragma unroll
  for (int o = 8; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ double half_max(double v) {
#pragma unroll
  for (int o = 8; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}
// sum_l v(l, j) (to every lane of column j) and sum_l v(i, l) (to every lane of row i)
template <int MK>
__device__ __forceinline__ double2 col_sum(double2 v, int j, int sb) {
  double2 s = make_double2(0.0, 0.0);
#pragma unroll
  for (int l = 0; l < MK; ++l) s = cadd(s, shfl2(v, sb + l * MK + j));
  return s;
}
template <int MK>
__device__ __forceinline__ double2 row_sum(double2 v, int i, int sb) {
  double2 s = make_double2(0.0, 0.0);
#pragma unroll
  for (int l = 0; l < MK; ++l) s = cadd(s, shfl2(v, sb + i * MK + l));
  return s;
}

// Gauss-Jordan elimination with partial pivoting on A q = b, lane-parallel: lane (i, j) holds
// A_ij and b_i (row layout); the pivot of column c is the largest |A_rc| for r >= c, the lowest
// row on ties.  b ends as the solution (row layout); A is destroyed.  Returns the smallest
// |pivot| (the same in every lane of the block).
template <int MK>
__device__ double gj_lanes(double2& a, double2& b, int i, int j, bool act, int sb) {
  double minpiv = 1e300;
#pragma unroll
  for (int c = 0; c < MK; ++c) {
    double key = (act && j == c && i >= c) ? cabs2(a) : -1.0;
    int prow = i;
#pragma unroll
    for (int o = 8; o > 0; o >>= 1) {
      const double ok = __shfl_xor_sync(0xffffffffu, key, o);
      const int orow = __shfl_xor_sync(0xffffffffu, prow, o);
      if (ok > key || (ok == key && orow < prow)) {
        key = ok;
        prow = orow;
      }
    }
    int src = threadIdx.x & 31;
    if (act && i == c) src = sb + prow * MK + j;
    else if (act && i == prow) src = sb + c * MK + j;
    a = shfl2(a, src);
    b = shfl2(b, src);
    const double2 piv = shfl2(a, sb + c * MK + c);
    minpiv = fmin(minpiv, sqrt(cabs2(piv)));
    const double2 inv = cabs2(piv) > 0.0 ? crecip(piv) : make_double2(0.0, 0.0);
    const double2 rowc = cmul(shfl2(a, sb + c * MK + j), inv);
    const double2 bc = cmul(shfl2(b, sb + c * MK), inv);
    const double2 m = shfl2(a, sb + i * MK + c);
    if (i == c) {
      a = rowc;
      b = bc;
    } else {
      a = csub(a, cmul(m, rowc));
      b = csub(b, cmul(m, bc));
    }
  }
  return minpiv;
}

// Forward IP of every block (Eqs. 14, 15), keeping the rows before each row update: one block
// per half warp (lane layout above), four warps per CTA.
template <int MK>
__global__ void __launch_bounds__(128) k_a_ipfwd(const double2* __restrict__ Q, const double2* __restrict__ V,
                                                 double2* __restrict__ Qs, int nb, double eps, double rtol,
                                                 unsigned* __restrict__ flags) {
  constexpr int E = MK * MK;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int seg = lane >> 4, e = lane & 15, sb = seg << 4;
  const bool act = e < E;
  const int i = act ? e / MK : 0, j = act ? e % MK : 0;
  const int blk = (blockIdx.x * (blockDim.x >> 5) + warp) * 2 + seg;
  const bool valid = blk < nb;
  const size_t id = valid ? (size_t)blk : 0;  // a spare half warp repeats block 0 and writes nothing
  double2 qc = act ? Q[id * E + e] : make_double2(0.0, 0.0);
  bool sing = false;
#pragma unroll
  for (int mu = 0; mu < MK; ++mu) {
    if (act && valid) Qs[(id * (MK + 1) + mu) * E + e] = qc;
    const double2* Vm = V + (id * MK + mu) * E;
    double2 a = make_double2(0.0, 0.0);  // A = Qc V_mu
#pragma unroll
    for (int l = 0; l < MK; ++l) {
      const double2 ql = shfl2(qc, sb + i * MK + l);
      if (act) a = cadd(a, cmul(ql, Vm[l * MK + j]));
    }
    const double scale = half_max(act ? sqrt(cabs2(a)) : 0.0);
    double2 b = make_double2((act && i == mu) ? 1.0 : 0.0, 0.0);
    const double mp = gj_lanes<MK>(a, b, i, j, act, sb);
    sing |= !(mp > rtol * scale);
    const double2 qj = shfl2(b, sb + j * MK);
    double term = 0.0;  // Re(conj(q_i) V_ij q_j)
    if (act) {
      const double2 vq = cmul(Vm[i * MK + j], qj);
      term = b.x * vq.x + b.y * vq.y;
    }
    const double s = half_sum(term);
    const double inv = 1.0 / sqrt(flo(s, eps));
    if (i == mu) qc = cconj(cscale(qj, inv));
  }
  if (act && valid) Qs[(id * (MK + 1) + MK) * E + e] = qc;
  if (sing && valid && e == 0) atomicOr(flags, 1u);
}

// ---------------------------------------------------------------- reverse kernels
// out = theta rho, rho = sqrt(num / max(den, eps)): bar_theta (=/+=) bar_out rho,
// bar_num = r / max(den, eps), bar_den = -r num / den^2 (0 under the floor),
// r = bar_out theta / (2 rho)
template <class R>
__global__ void k_a_mub(const R* __restrict__ th, const R* __restrict__ num, const R* __restrict__ den,
                        const R* __restrict__ bar_out, R* __restrict__ bar_th, R* __restrict__ numb,
                        R* __restrict__ denb, size_t n, R eps) {
  const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const R dn = flo(den[i], eps);
  const R rho = sqrt(num[i] / dn);
  bar_th[i] = bar_out[i] * rho;
  const R r = rho > R(0) ? bar_out[i] * th[i] / (R(2) * rho) : R(0);
  numb[i] = r / dn;
  denb[i] = den[i] > eps ? -r * num[i] / (dn * dn) : R(0);
}

// Reverse of the g update's sums (Eq. 10) and of the model at lambda2, per (f, t):
//   ybar[m] = sum_n lam2 (-2 numb P / yhat^3 - denb / yhat^2)  (0 under the floor)
//   Pbar[m] += sum_n numb lam2 / yhat^2
//   lamb[n] = sum_m (numb P / yhat^2 + denb / yhat + ybar[m] g)
template <class R>
__global__ void k_a_gstat_b(const R* __restrict__ numb, const R* __restrict__ denb,
                            const R* __restrict__ lam, const R* __restrict__ P,
                            const R* __restrict__ y, const R* __restrict__ ry, const R* __restrict__ g,
                            R* __restrict__ lamb, R* __restrict__ Pb, R* __restrict__ yb, int N, int F,
                            int T, int M, R eps) {
  const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (size_t)F * T) return;
  const int t = (int)(i % T), f = (int)(i / T);
  const size_t r = i * M;
  for (int m = 0; m < M; ++m) {
    // sum_n lam numb and sum_n lam denb first, then the per-microphone factors
    const R rv = ry[r + m], r2 = rv * rv, pm = P[r + m];
    R u = R(0), v = R(0);
    for (int n = 0; n < N; ++n) {
      const R l = lam[((size_t)n * F + f) * T + t];
      const size_t q = ((size_t)f * N + n) * M + m;
      u += l * numb[q];
      v += l * denb[q];
    }
    const R a = R(-2) * pm * (r2 * rv) * u - r2 * v;
    yb[r + m] = y[r + m] > eps ? a : R(0);
    Pb[r + m] += r2 * u;
  }
  for (int n = 0; n < N; ++n) {
    R s = R(0);
    for (int m = 0; m < M; ++m) {
      const R rv = ry[r + m];
      const size_t q = ((size_t)f * N + n) * M + m;
      s += numb[q] * P[r + m] * (rv * rv) + denb[q] * rv + yb[r + m] * g[q];
    }
    lamb[((size_t)n * F + f) * T + t] = s;
  }
}

// Reverse of A = sum_m g P / yhat^2, D = sum_m g / yhat, per (f, t, m):
//   ybar (=/+=) sum_n (-2 Ab g P / yhat^3 - Db g / yhat^2)  (0 under the floor),
//   Pbar += sum_n Ab g / yhat^2
template <class R>
__global__ void k_a_stat_b(const R* __restrict__ Ab, const R* __restrict__ Db,
                           const R* __restrict__ g, const R* __restrict__ P, const R* __restrict__ y,
                           const R* __restrict__ ry, R* __restrict__ yb, R* __restrict__ Pb, int N,
                           int F, int T, int M, R eps, int acc) {
  const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (size_t)F * T * M) return;
  const int m = (int)(i % M), t = (int)((i / M) % T), f = (int)(i / ((size_t)T * M));
  // the source sums first: sum_n Ab g and sum_n Db g, then the per-microphone factors
  const R rv = ry[i], r2 = rv * rv, pi = P[i];
  R sa = R(0), sd = R(0);
  for (int n = 0; n < N; ++n) {
    const size_t nf = ((size_t)n * F + f) * T + t;
    const R gg = g[((size_t)f * N + n) * M + m];
    sa += Ab[nf] * gg;
    sd += Db[nf] * gg;
  }
  const R a = R(-2) * pi * (r2 * rv) * sa - r2 * sd;
  const R pb = r2 * sa;
  const R v = y[i] > eps ? a : R(0);
  yb[i] = (acc ? yb[i] : R(0)) + v;
  Pb[i] += pb;
}

// lamb[n][f][t] (=/+=) sum_m ybar[f][t][m] g[f][n][m]   (reverse of y = sum_n lambda g)
template <class R>
__global__ void k_a_y_b(const R* __restrict__ yb, const R* __restrict__ g, R* __restrict__ lamb,
                        int N, int F, int T, int M, int acc) {
  const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (size_t)N * F * T) return;
  const int t = (int)(i % T), f = (int)((i / T) % F), n = (int)(i / ((size_t)F * T));
  const R* gr = g + ((size_t)f * N + n) * M;
  const R* yr = yb + ((size_t)f * T + t) * M;
  R s = R(0);
  for (int m = 0; m < M; ++m) s += yr[m] * gr[m];
  lamb[i] = (acc ? lamb[i] : R(0)) + s;
}

// gbar[f][n][m] += sum_t (Ab P / yhat^2 + Db / yhat + ybar lam); NULL terms are skipped.
// One warp per output, lanes over t.
template <class R>
__global__ void k_a_gbar(const R* __restrict__ Ab, const R* __restrict__ Db, const R* __restrict__ yb,
                         const R* __restrict__ lam, const R* __restrict__ P, const R* __restrict__ ry,
                         R* __restrict__ gb, int N, int F, int T, int M) {
  const size_t i = ((size_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (i >= (size_t)F * N * M) return;
  const int m = (int)(i % M), n = (int)((i / M) % N), f = (int)(i / ((size_t)M * N));
  const size_t nf = ((size_t)n * F + f) * T;
  R s = R(0);
  for (int t = lane; t < T; t += 32) {
    const size_t r = ((size_t)f * T + t) * M + m;
    const R rv = ry[r];
    if (Ab) s += Ab[nf + t] * P[r] * (rv * rv);
    if (Db) s += Db[nf + t] * rv;
    if (yb) s += yb[r] * lam[nf + t];
  }
  s = warp_sum(s);
  if (lane == 0) gb[i] += s;
}

// gbar[f][n][m] += sum_t G4[n][f][t][m]; one warp per output, lanes over t
__global__ void k_a_red_t4(const double* __restrict__ G4, double* __restrict__ gb, int N, int F, int T, int M) {
  const size_t i = ((size_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (i >= (size_t)F * N * M) return;
  const int m = (int)(i % M), n = (int)((i / M) % N), f = (int)(i / ((size_t)M * N));
  double s = 0.0;
  for (int t = lane; t < T; t += 32) s += G4[(((size_t)n * F + f) * T + t) * M + m];
  s = warp_sum(s);
  if (lane == 0) gb[i] += s;
}

// Reverse of P = |Q x|^2: Qbar[f][k][a][b] += sum_t 2 Pbar_a z_a conj(x_b), z = Q_fk x_ftk.
// One warp per (f, k, a), lanes over t: z_a is formed once per frame for all b.
template <int MK, class RR>
__global__ void k_a_Pb(const double2* __restrict__ x, const double2* __restrict__ Q, size_t bstride,
                       const RR* __restrict__ Pb, double2* __restrict__ Qb, int F, int T, int K) {
  const size_t w = ((size_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (w >= (size_t)F * K * MK) return;
  const int a = (int)(w % MK), k = (int)((w / MK) % K), f = (int)(w / ((size_t)MK * K));
  const int M = K * MK, o = k * MK;
  const double2* q = Q + ((size_t)f * K + k) * bstride + a * MK;
  double2 qa[MK], acc[MK];
#pragma unroll
  for (int c2 = 0; c2 < MK; ++c2) {
    qa[c2] = q[c2];
    acc[c2] = make_double2(0.0, 0.0);
  }
  for (int t = lane; t < T; t += 32) {
    const size_t r = ((size_t)f * T + t) * M + o;
    double2 xv[MK];
    double2 z = make_double2(0.0, 0.0);
#pragma unroll
    for (int c2 = 0; c2 < MK; ++c2) {
      xv[c2] = ld(x + r + c2);
      z = cadd(z, cmul(qa[c2], xv[c2]));
    }
    const double s2 = 2.0 * (double)Pb[r + a];
#pragma unroll
    for (int b = 0; b < MK; ++b) acc[b] = cadd(acc[b], cscale(cmulc(z, xv[b]), s2));
  }
#pragma unroll
  for (int b = 0; b < MK; ++b) acc[b] = make_double2(warp_sum(acc[b].x), warp_sum(acc[b].y));
  if (lane == 0) {
#pragma unroll
    for (int b = 0; b < MK; ++b) {
      double2* p = Qb + (((size_t)f * K + k) * MK + a) * MK + b;
      *p = cadd(*p, acc[b]);
    }
  }
}

// Reverse of the IP rows of one block, mu = MK-1 .. 0.  For row mu with
// A = Qc V_mu, q = A^-1 e_mu, s = Re q^H V_mu q, sigma = sqrt(max(s, eps)):
//   qbar_n = conj(row mu of Qbar); Qbar row mu <- 0
//   qbar = qbar_n / sigma;  if s > eps: sbar = -Re(qbar_n^H q) / (2 sigma^3),
//   qbar += 2 sbar V q
//   y = A^-H qbar;  Qbar += -y (q^H V_mu);  Vbar_mu = (sbar q - Qc^H y) q^H
// One block per half warp (lane layout above), four warps per CTA.
template <int MK>
__global__ void __launch_bounds__(128) k_a_ipb(const double2* __restrict__ Qs, const double2* __restrict__ V,
                                               const double2* __restrict__ Qbin, double2* __restrict__ Qbout,
                                               double2* __restrict__ Vb, int nb, double eps) {
  constexpr int E = MK * MK;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int seg = lane >> 4, e = lane & 15, sb = seg << 4;
  const bool act = e < E;
  const int i = act ? e / MK : 0, j = act ? e % MK : 0;
  const int blk = (blockIdx.x * (blockDim.x >> 5) + warp) * 2 + seg;
  const bool valid = blk < nb;
  const size_t id = valid ? (size_t)blk : 0;  // a spare half warp repeats block 0 and writes nothing
  const double2 z = make_double2(0.0, 0.0);
  double2 qbe = act ? Qbin[id * E + e] : z;  // Qbar_ij
#pragma unroll
  for (int mu = MK - 1; mu >= 0; --mu) {
    const double2* Qc = Qs + (id * (MK + 1) + mu) * E;
    const double2* Vm = V + (id * MK + mu) * E;
    double2 a = z;  // A = Qc V_mu
    if (act)
#pragma unroll
      for (int l = 0; l < MK; ++l) a = cadd(a, cmul(Qc[i * MK + l], Vm[l * MK + j]));
    double2 ah = cconj(shfl2(a, sb + j * MK + i));  // (A^H)_ij for the adjoint solve
    double2 q = make_double2((act && i == mu) ? 1.0 : 0.0, 0.0);
    gj_lanes<MK>(a, q, i, j, act, sb);  // q = A^-1 e_mu (row layout)
    const double2 qj = shfl2(q, sb + j * MK);
    const double2 vij = act ? Vm[i * MK + j] : z;
    const double2 vq = row_sum<MK>(cmul(vij, qj), i, sb);  // (V q)_i, row layout
    const double s = half_sum((act && j == 0) ? q.x * vq.x + q.y * vq.y : 0.0);
    const double sig = sqrt(flo(s, eps));
    const double2 qn = cconj(shfl2(qbe, sb + mu * MK + i));  // conj(Qbar_mu,i), row layout
    const double dotr = half_sum((act && j == 0) ? qn.x * q.x + qn.y * q.y : 0.0);
    double2 y = cscale(qn, 1.0 / sig);
    if (i == mu) qbe = z;
    double sbar = 0.0;
    if (s > eps) {
      sbar = -dotr / (2.0 * sig * sig * sig);
      y = cadd(y, cscale(vq, 2.0 * sbar));
    }
    gj_lanes<MK>(ah, y, i, j, act, sb);  // y = A^-H qbar (row layout)
    const double2 w = col_sum<MK>(cmul(cconj(q), vij), j, sb);  // (q^H V_mu)_j, column layout
    qbe = csub(qbe, cmul(y, w));
    // u_i = sbar q_i - sum_l conj(Qc_li) y_l: column sums of conj(Qc_ij) y_i, taken from column i
    const double2 cs = col_sum<MK>(act ? cmul(cconj(Qc[i * MK + j]), y) : z, j, sb);
    const double2 u = csub(cscale(q, sbar), shfl2(cs, sb + i));
    if (act && valid) Vb[(id * MK + mu) * E + e] = cmulc(u, qj);  // Vbar_ij = u_i conj(q_j)
  }
  if (act && valid) Qbout[id * E + e] = qbe;
}

// Reverse of Eq. 13 and of 1/yhat0: ybar0[f][t][o_k+mu] += -Re(x^H Vbar_mu x) / (T yhat0^2).
// Re(x^H Vb x) = sum_a Re Vb_aa |x_a|^2 + sum_{a<b} [(Re Vb_ab + Re Vb_ba) Re p_ab
// - (Im Vb_ab - Im Vb_ba) Im p_ab] with p_ab = conj(x_a) x_b: k_a_Vh packs these MK^2 reals per
// (f, k, mu) (diagonal at [a][a], the sums at [a][b], the differences at [b][a] for a < b), and
// k_a_Vb forms the products p_ab of one (f, t, k) once for all mu.
template <int MK>
__global__ void k_a_Vh(const double2* __restrict__ Vb, double* __restrict__ Vh, size_t n) {
  const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;  // i = (f K + k) MK + mu
  const double2* v = Vb + i * MK * MK;
  double* h = Vh + i * MK * MK;
#pragma unroll
  for (int a = 0; a < MK; ++a) {
    h[a * MK + a] = v[a * MK + a].x;
#pragma unroll
    for (int b = a + 1; b < MK; ++b) {
      h[a * MK + b] = v[a * MK + b].x + v[b * MK + a].x;
      h[b * MK + a] = v[a * MK + b].y - v[b * MK + a].y;
    }
  }
}

template <int MK, class RR>
__global__ void k_a_Vb(const double2* __restrict__ x, const double* __restrict__ Vh, const RR* __restrict__ y0,
                       const RR* __restrict__ r0, RR* __restrict__ yb, int F, int T, int K, double eps) {
  const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (size_t)F * T * K) return;
  const int k = (int)(i % K), t = (int)((i / K) % T), f = (int)(i / ((size_t)K * T));
  const int M = K * MK, o = k * MK;
  const double2* xr = x + ((size_t)f * T + t) * M + o;
  double2 xv[MK];
#pragma unroll
  for (int a = 0; a < MK; ++a) xv[a] = ld(xr + a);
  double pr[MK][MK], pi[MK][MK];  // pr[a][a] = |x_a|^2; pr/pi[a][b] = Re/Im conj(x_a) x_b for a < b
#pragma unroll
  for (int a = 0; a < MK; ++a) {
    pr[a][a] = xv[a].x * xv[a].x + xv[a].y * xv[a].y;
#pragma unroll
    for (int b = a + 1; b < MK; ++b) {
      pr[a][b] = xv[a].x * xv[b].x + xv[a].y * xv[b].y;
      pi[a][b] = xv[a].x * xv[b].y - xv[a].y * xv[b].x;
    }
  }
  const double invT = 1.0 / (double)T;
#pragma unroll
  for (int mu = 0; mu < MK; ++mu) {
    const size_t e = ((size_t)f * T + t) * M + o + mu;
    if (!((double)y0[e] > eps)) continue;
    const double* h = Vh + (((size_t)f * K + k) * MK + mu) * MK * MK;
    double s = 0.0;
#pragma unroll
    for (int a = 0; a < MK; ++a) {
      s += h[a * MK + a] * pr[a][a];
#pragma unroll
      for (int b = a + 1; b < MK; ++b) s += h[a * MK + b] * pr[a][b] - h[b * MK + a] * pi[a][b];
    }
    const double r = (double)r0[e];
    yb[e] += (RR)(-s * (r * r) * invT);
  }
}

// ---------------------------------------------------------------- losses
__device__ void block_add(double v, double* red) {
  __shared__ double sm[32];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0) sm[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x < 32) {
    v = threadIdx.x < (blockDim.x >> 5) ? sm[threadIdx.x] : 0.0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (threadIdx.x == 0) atomicAdd(red, v);
  }
}

// data term of Eq. 12 and its adjoints: Pbar = 1/yhat, ybar = 1/yhat - P/yhat^2 (0 under the floor)
__global__ void k_a_nll_data(const double* __restrict__ P, const double* __restrict__ y,
                             const double* __restrict__ ry, double* __restrict__ Pb, double* __restrict__ yb,
                             double* __restrict__ red, size_t n, double eps) {
  const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  double v = 0.0;
  if (i < n) {
    const double yy = flo(y[i], eps), rv = ry[i];
    v = P[i] * rv + log(yy);
    Pb[i] = rv;
    yb[i] = y[i] > eps ? rv - P[i] * (rv * rv) : 0.0;
  }
  block_add(v, red);
}

// -T ln|det Q_fk|^2 and its adjoint -2 T Q^-H, added to Qbar
template <int MK>
__global__ void k_a_logdet_b(const double2* __restrict__ Q, double2* __restrict__ Qb, double* __restrict__ red, int nb,
                             int T) {
  const int id = blockIdx.x * blockDim.x + threadIdx.x;
  double v = 0.0;
  if (id < nb) {
    double2 A[MK][MK], X[MK][MK];
#pragma unroll
    for (int i = 0; i < MK; ++i)
#pragma unroll
      for (int j = 0; j < MK; ++j) A[i][j] = Q[(size_t)id * MK * MK + i * MK + j];
    v = -(double)T * gj_inverse<MK>(A, X);
#pragma unroll
    for (int i = 0; i < MK; ++i)
#pragma unroll
      for (int j = 0; j < MK; ++j) {
        double2* p = Qb + (size_t)id * MK * MK + i * MK + j;
        *p = csub(*p, cscale(cconj(X[j][i]), 2.0 * T));
      }
  }
  block_add(v, red);
}

template <int MK>
__global__ void k_a_inv(const double2* __restrict__ Q, double2* __restrict__ Binv, int nb) {
  const int id = blockIdx.x * blockDim.x + threadIdx.x;
  if (id >= nb) return;
  double2 A[MK][MK], X[MK][MK];
#pragma unroll
  for (int i = 0; i < MK; ++i)
#pragma unroll
    for (int j = 0; j < MK; ++j) A[i][j] = Q[(size_t)id * MK * MK + i * MK + j];
  gj_inverse<MK>(A, X);
#pragma unroll
  for (int i = 0; i < MK; ++i)
#pragma unroll
    for (int j = 0; j < MK; ++j) Binv[(size_t)id * MK * MK + i * MK + j] = X[i][j];
}

// Wiener filter MSE, per (f, t): for each block and source, z = Q x, gamma = lam g / yhat,
// u = gamma z, c = B u (B = Q^-1), d = c - c_true, loss += |d|^2 / S, cbar = 2 d / S,
// ubar = B^H cbar, gammabar = Re(conj(ubar) z), zbar += gamma ubar;
// lamb[n] = sum_m gammabar g / yhat, ybar[m] = -sum_n gammabar lam g / yhat^2 (0 under the floor),
// G4[n][f][t][m] = gammabar lam / yhat (summed over t into gbar); ubar, c and zbar are kept
// for the Q adjoint
template <int MK>
__global__ void k_a_wiener_ft(const float2* __restrict__ x, const double2* __restrict__ Q,
                              const double2* __restrict__ Binv, const float2* __restrict__ ct,
                              const double* __restrict__ lam, const double* __restrict__ g,
                              const double* __restrict__ y, double* __restrict__ lamb, double* __restrict__ yb,
                              double* __restrict__ G4, double2* __restrict__ ubar, double2* __restrict__ cvec,
                              double2* __restrict__ zbar, double* __restrict__ red, int N, int F, int T, int K,
                              double eps, double invS) {
  const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int M = K * MK;
  double loss = 0.0;
  if (i < (size_t)F * T) {
    const int t = (int)(i % T), f = (int)(i / T);
    for (int n = 0; n < N; ++n) lamb[((size_t)n * F + f) * T + t] = 0.0;
    for (int k = 0; k < K; ++k) {
      const int o = k * MK;
      const double2* q = Q + ((size_t)f * K + k) * MK * MK;
      const double2* B = Binv + ((size_t)f * K + k) * MK * MK;
      const size_t r = ((size_t)f * T + t) * M + o;
      double2 z[MK], zb[MK];
      double yh[MK], ybm[MK];
#pragma unroll
      for (int a = 0; a < MK; ++a) {
        double2 s = make_double2(0.0, 0.0);
#pragma unroll
        for (int c2 = 0; c2 < MK; ++c2) s = cadd(s, cmul(q[a * MK + c2], ld(x + r + c2)));
        z[a] = s;
        zb[a] = make_double2(0.0, 0.0);
        yh[a] = flo(y[r + a], eps);
        ybm[a] = 0.0;
      }
      for (int n = 0; n < N; ++n) {
        const double l = lam[((size_t)n * F + f) * T + t];
        const double* gr = g + ((size_t)f * N + n) * M + o;
        const size_t rn = (((size_t)n * F + f) * T + t) * M + o;
        double2 u[MK], cb[MK];
        double gam[MK];
#pragma unroll
        for (int a = 0; a < MK; ++a) {
          gam[a] = l * gr[a] / yh[a];
          u[a] = cscale(z[a], gam[a]);
        }
#pragma unroll
        for (int a = 0; a < MK; ++a) {
          double2 c = make_double2(0.0, 0.0);
#pragma unroll
          for (int b = 0; b < MK; ++b) c = cadd(c, cmul(B[a * MK + b], u[b]));
          cvec[rn + a] = c;
          const double2 d = csub(c, ld(ct + rn + a));
          loss += cabs2(d) * invS;
          cb[a] = cscale(d, 2.0 * invS);
        }
        double lb = 0.0;
#pragma unroll
        for (int a = 0; a < MK; ++a) {
          double2 ub = make_double2(0.0, 0.0);  // (B^H cbar)_a
#pragma unroll
          for (int j = 0; j < MK; ++j) ub = cadd(ub, cmul(cconj(B[j * MK + a]), cb[j]));
          ubar[rn + a] = ub;
          const double gb = ub.x * z[a].x + ub.y * z[a].y;  // Re(conj(ubar) z)
          zb[a] = cadd(zb[a], cscale(ub, gam[a]));
          lb += gb * gr[a] / yh[a];
          ybm[a] += -gb * l * gr[a] / (yh[a] * yh[a]);
          G4[rn + a] = gb * l / yh[a];
        }
        lamb[((size_t)n * F + f) * T + t] += lb;
      }
#pragma unroll
      for (int a = 0; a < MK; ++a) {
        zbar[r + a] = zb[a];
        yb[r + a] = y[r + a] > eps ? ybm[a] : 0.0;
      }
    }
  }
  block_add(loss, red);
}

// Qbar[f][k][a][b] = sum_t (zbar_a conj(x_b) - sum_n ubar_n,a conj(c_n,b))
// (the second sum is -B^H (sum cbar u^H) B^H, the adjoint through B = Q^-1)
__global__ void k_a_wiener_q(const float2* __restrict__ x, const double2* __restrict__ zbar,
                             const double2* __restrict__ ubar, const double2* __restrict__ cvec,
                             double2* __restrict__ Qb, int N, int F, int T, int K, int MK) {
  const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (size_t)F * K * MK * MK) return;
  const int b = (int)(i % MK), a = (int)((i / MK) % MK), k = (int)((i / ((size_t)MK * MK)) % K);
  const int f = (int)(i / ((size_t)MK * MK * K));
  const int M = K * MK, o = k * MK;
  double2 acc = make_double2(0.0, 0.0);
  for (int t = 0; t < T; ++t) {
    const size_t r = ((size_t)f * T + t) * M + o;
    acc = cadd(acc, cmulc(zbar[r + a], ld(x + r + b)));
    for (int n = 0; n < N; ++n) {
      const size_t rn = (((size_t)n * F + f) * T + t) * M + o;
      acc = csub(acc, cmulc(ubar[rn + a], cvec[rn + b]));
    }
  }
  Qb[i] = acc;
}

inline unsigned nblk(size_t n, int t = 256) { return (unsigned)((n + t - 1) / t); }

#define AL(...)                                   \
  do {                                            \
    __VA_ARGS__;                                  \
    cudaError_t e_ = cudaGetLastError();          \
    if (e_ != cudaSuccess) return e_;             \
  } while (0)

#define MK_DISPATCH(MK, KERNEL, GRID, BLOCK, SMEM, STREAM, ...)                        \
  switch (MK) {                                                                        \
    case 1: KERNEL<1><<<GRID, BLOCK, SMEM, STREAM>>>(__VA_ARGS__); break;              \
    case 2: KERNEL<2><<<GRID, BLOCK, SMEM, STREAM>>>(__VA_ARGS__); break;              \
    case 3: KERNEL<3><<<GRID, BLOCK, SMEM, STREAM>>>(__VA_ARGS__); break;              \
    case 4: KERNEL<4><<<GRID, BLOCK, SMEM, STREAM>>>(__VA_ARGS__); break;              \
    default: return cudaErrorInvalidValue;                                             \
  }

#define MK_DISPATCH2(MK, KERNEL, RT, GRID, BLOCK, SMEM, STREAM, ...)                \
  switch (MK) {                                                                        \
    case 1: KERNEL<1, RT><<<GRID, BLOCK, SMEM, STREAM>>>(__VA_ARGS__); break;          \
    case 2: KERNEL<2, RT><<<GRID, BLOCK, SMEM, STREAM>>>(__VA_ARGS__); break;          \
    case 3: KERNEL<3, RT><<<GRID, BLOCK, SMEM, STREAM>>>(__VA_ARGS__); break;          \
    case 4: KERNEL<4, RT><<<GRID, BLOCK, SMEM, STREAM>>>(__VA_ARGS__); break;          \
    default: return cudaErrorInvalidValue;                                             \
  }

struct Dims {
  int N, F, T, B, K, MK, M, Tp;
  size_t nft, ftm, nfb, nbt, fnm, nq, nv, nqs, nftm;
  double eps;
};

Dims dims_of(const dfmnmf_ctx* c) {
  Dims d;
  d.N = c->N; d.F = c->F; d.T = c->T; d.B = c->B; d.K = c->K; d.MK = c->MK; d.M = c->M; d.Tp = c->Tp;
  d.nft = (size_t)d.N * d.F * d.T;
  d.ftm = (size_t)d.F * d.T * d.M;
  d.nfb = (size_t)d.N * d.F * d.B;
  d.nbt = (size_t)d.N * d.B * d.T;
  d.fnm = (size_t)d.F * d.N * d.M;
  d.nq = (size_t)d.F * d.K * d.MK * d.MK;
  d.nv = d.nq * d.MK;
  d.nqs = d.nq * (d.MK + 1);
  d.nftm = d.nft * d.M;
  d.eps = (double)c->eps;
  return d;
}

// The double-precision NMF side: the FP64 arrays of the workspace.
AdjSide<double> dside(dfmnmf_adj* a) {
  AdjSide<double> v;
  v.Wd = a->Wd; v.Hd = a->Hd; v.gd = a->gd;
  v.lam0 = a->lam0; v.lam1 = a->lam1; v.lam2 = a->lam2; v.y0 = a->y0; v.y1 = a->y1; v.y2 = a->y2;
  v.r0 = a->r0; v.r1 = a->r1; v.r2 = a->r2; v.P = a->P; v.A0 = a->A0; v.D0 = a->D0; v.A1 = a->A1; v.D1 = a->D1;
  v.numW = a->numW; v.denW = a->denW; v.W1 = a->W1; v.numH = a->numH; v.denH = a->denH; v.H1 = a->H1;
  v.numG = a->numG; v.denG = a->denG;
  v.Wb = a->Wb; v.Wb1 = a->Wb1; v.Hb = a->Hb; v.Hb1 = a->Hb1; v.gb = a->gb; v.gb1 = a->gb1;
  v.lamb = a->lamb; v.yb = a->yb; v.Pb = a->Pb; v.Ab = a->Ab; v.Db = a->Db; v.nb = a->nb; v.db = a->db;
  return v;
}

template <class S, class D>
__global__ void k_a_cvt(const S* __restrict__ in, D* __restrict__ out, size_t n) {
  const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = (D)in[i];
}
template <class S, class D>
cudaError_t convert(const S* in, D* out, size_t n, cudaStream_t s) {
  AL(k_a_cvt<S, D><<<nblk(n), 256, 0, s>>>(in, out, n));
  return cudaSuccess;
}

// A stored state (context layouts) into the side's Wd, Hd, gd (type R) and Qd (FP64)
template <class R>
cudaError_t load_state(dfmnmf_adj* a, const AdjSide<R>& v, const Dims& d, const double2* Q, const float* W,
                       const float* H, const float* g, cudaStream_t s) {
  AL(k_a_tod<R><<<nblk(d.nfb + d.nbt + d.fnm), 256, 0, s>>>(W, H, g, v.Wd, v.Hd, v.gd, d.nfb, d.nbt, d.fnm, d.T,
                                                             d.Tp));
  return cudaMemcpyAsync(a->Qd, Q, d.nq * sizeof(double2), cudaMemcpyDeviceToDevice, s);
}

// lam = W H, yraw = sum_n lam g and ry = 1 / max(yraw, eps)
template <class R>
cudaError_t model(const Dims& d, const R* W, const R* H, const R* g, R* lam, R* y, R* ry, cudaStream_t s) {
  AL(k_a_nmf_b<R><<<nblk(d.nft), 256, 0, s>>>(W, H, lam, d.N, d.F, d.B, d.T));
  AL(k_a_y<R><<<nblk(d.ftm), 256, 0, s>>>(lam, g, y, ry, d.N, d.F, d.T, d.M, (R)d.eps));
  return cudaSuccess;
}

template <class R>
cudaError_t nmf_t(const Dims& d, const R* X, const R* Y, R* out, int acc, cudaStream_t s) {
  AL(k_a_nmf_t<R><<<nblk(d.nfb * 32), 256, 0, s>>>(X, Y, out, d.N, d.F, d.B, d.T, acc));
  return cudaSuccess;
}
template <class R>
cudaError_t nmf_f(const Dims& d, const R* X, const R* Y, R* out, int acc, cudaStream_t s) {
  AL(k_a_nmf_f<R><<<dim3((unsigned)((d.T + 31) / 32), (unsigned)(d.N * d.B)), 32 * NMF_F_WARPS, 0, s>>>(
      X, Y, out, d.N, d.F, d.B, d.T, acc));
  return cudaSuccess;
}

// Reverse of one iteration whose input state is in (v.Wd, v.Hd, v.gd, Qd); the adjoint of its
// output state is in (Qb1, v.Wb1, v.Hb1, v.gb1) (consumed); the adjoint of its input state is
// written to (Qb, v.Wb, v.Hb, v.gb).  The IP side (V, the IP rows, P = |Q x|^2 and their
// adjoints) is FP64; the NMF side runs in R.
template <class R>
cudaError_t reverse_iteration(dfmnmf_adj* a, const AdjSide<R>& v, const Dims& d, cudaStream_t s) {
  const dfmnmf_ctx* c = a->c;
  const double eps = d.eps;
  const R epsr = (R)d.eps;
  const int nb = d.F * d.K;
  // forward, recomputed
  cudaError_t e = model<R>(d, v.Wd, v.Hd, v.gd, v.lam0, v.y0, v.r0, s);
  if (e != cudaSuccess) return e;
  const double* r0d = reinterpret_cast<const double*>(v.r0);
  if constexpr (!std::is_same<R, double>::value) {  // the weights of Eq. 13 in FP64, converted once
    if ((e = convert(v.r0, a->r0d, d.ftm, s))) return e;
    r0d = a->r0d;
  }
  MK_DISPATCH(d.MK, k_a_V, nblk((size_t)d.F * d.K * (d.MK * (d.MK + 1) / 2) * 32), 256, 0, s, a->x64, r0d, a->V,
              d.F, d.T, d.K);
  AL((void)0);
  MK_DISPATCH(d.MK, k_a_ipfwd, nblk(nb, 8), 128, 0, s, a->Qd, a->V, a->Qs, nb, eps, (double)c->singular_rtol, a->flags);
  AL((void)0);
  const double2* Qn = a->Qs + (size_t)d.MK * d.MK * d.MK;  // rows after the last update, stride (MK+1) MK^2
  const size_t qstr = (size_t)(d.MK + 1) * d.MK * d.MK;
  AL(k_a_P<R><<<nblk((size_t)d.F * d.T * d.K), 256, 0, s>>>(a->x64, Qn, qstr, v.P, d.F, d.T, d.K, d.MK));
  AL(k_a_AD<R><<<nblk((size_t)d.F * d.T), 256, 0, s>>>(v.P, v.r0, v.gd, v.A0, v.D0, d.N, d.F, d.T, d.M));
  if ((e = nmf_t<R>(d, v.A0, v.Hd, v.numW, 0, s)) || (e = nmf_t<R>(d, v.D0, v.Hd, v.denW, 0, s))) return e;
  AL(k_a_mu<R><<<nblk(d.nfb), 256, 0, s>>>(v.Wd, v.numW, v.denW, v.W1, d.nfb, epsr));
  if ((e = model<R>(d, v.W1, v.Hd, v.gd, v.lam1, v.y1, v.r1, s))) return e;
  AL(k_a_AD<R><<<nblk((size_t)d.F * d.T), 256, 0, s>>>(v.P, v.r1, v.gd, v.A1, v.D1, d.N, d.F, d.T, d.M));
  if ((e = nmf_f<R>(d, v.W1, v.A1, v.numH, 0, s)) || (e = nmf_f<R>(d, v.W1, v.D1, v.denH, 0, s))) return e;
  AL(k_a_mu<R><<<nblk(d.nbt), 256, 0, s>>>(v.Hd, v.numH, v.denH, v.H1, d.nbt, epsr));
  if ((e = model<R>(d, v.W1, v.H1, v.gd, v.lam2, v.y2, v.r2, s))) return e;
  AL(k_a_gnum<R><<<nblk(d.fnm * 32), 256, 0, s>>>(v.lam2, v.P, v.r2, v.numG, v.denG, d.N, d.F, d.T, d.M));

  // reverse of the g update (Eq. 10)
  AL(k_a_mub<R><<<nblk(d.fnm), 256, 0, s>>>(v.gd, v.numG, v.denG, v.gb1, v.gb, v.nb, v.db, d.fnm, epsr));
  ACKE(cudaMemsetAsync(v.Pb, 0, d.ftm * sizeof(R), s));
  AL(k_a_gstat_b<R><<<nblk((size_t)d.F * d.T), 256, 0, s>>>(v.nb, v.db, v.lam2, v.P, v.y2, v.r2, v.gd, v.lamb,
                                                          v.Pb, v.yb, d.N, d.F, d.T, d.M, epsr));
  AL(k_a_gbar<R><<<nblk(d.fnm * 32), 256, 0, s>>>(nullptr, nullptr, v.yb, v.lam2, v.P, v.r2, v.gb, d.N, d.F, d.T,
                                                d.M));
  if ((e = nmf_t<R>(d, v.lamb, v.H1, v.Wb1, 1, s)) || (e = nmf_f<R>(d, v.W1, v.lamb, v.Hb1, 1, s))) return e;
  // reverse of the H update (Eq. 9)
  AL(k_a_mub<R><<<nblk(d.nbt), 256, 0, s>>>(v.Hd, v.numH, v.denH, v.Hb1, v.Hb, v.nb, v.db, d.nbt, epsr));
  if ((e = nmf_t<R>(d, v.A1, v.nb, v.Wb1, 1, s)) || (e = nmf_t<R>(d, v.D1, v.db, v.Wb1, 1, s))) return e;
  AL(k_a_nmf_b<R><<<nblk(d.nft), 256, 0, s>>>(v.W1, v.nb, v.Ab, d.N, d.F, d.B, d.T));
  AL(k_a_nmf_b<R><<<nblk(d.nft), 256, 0, s>>>(v.W1, v.db, v.Db, d.N, d.F, d.B, d.T));
  AL(k_a_stat_b<R><<<nblk(d.ftm), 256, 0, s>>>(v.Ab, v.Db, v.gd, v.P, v.y1, v.r1, v.yb, v.Pb, d.N, d.F, d.T,
                                             d.M, epsr, 0));
  AL(k_a_gbar<R><<<nblk(d.fnm * 32), 256, 0, s>>>(v.Ab, v.Db, v.yb, v.lam1, v.P, v.r1, v.gb, d.N, d.F, d.T,
                                                d.M));
  AL(k_a_y_b<R><<<nblk(d.nft), 256, 0, s>>>(v.yb, v.gd, v.lamb, d.N, d.F, d.T, d.M, 0));
  if ((e = nmf_t<R>(d, v.lamb, v.Hd, v.Wb1, 1, s)) || (e = nmf_f<R>(d, v.W1, v.lamb, v.Hb, 1, s))) return e;
  // reverse of the W update (Eq. 8)
  AL(k_a_mub<R><<<nblk(d.nfb), 256, 0, s>>>(v.Wd, v.numW, v.denW, v.Wb1, v.Wb, v.nb, v.db, d.nfb, epsr));
  if ((e = nmf_f<R>(d, v.nb, v.A0, v.Hb, 1, s)) || (e = nmf_f<R>(d, v.db, v.D0, v.Hb, 1, s))) return e;
  AL(k_a_nmf_b<R><<<nblk(d.nft), 256, 0, s>>>(v.nb, v.Hd, v.Ab, d.N, d.F, d.B, d.T));
  AL(k_a_nmf_b<R><<<nblk(d.nft), 256, 0, s>>>(v.db, v.Hd, v.Db, d.N, d.F, d.B, d.T));
  AL(k_a_stat_b<R><<<nblk(d.ftm), 256, 0, s>>>(v.Ab, v.Db, v.gd, v.P, v.y0, v.r0, v.yb, v.Pb, d.N, d.F, d.T,
                                             d.M, epsr, 0));
  // reverse of the projections and of the IP rows (Eqs. 13-15)
  MK_DISPATCH2(d.MK, k_a_Pb, R, nblk((size_t)d.F * d.K * d.MK * 32), 256, 0, s, a->x64, Qn, qstr, v.Pb, a->Qb1, d.F,
               d.T, d.K);
  AL((void)0);
  MK_DISPATCH(d.MK, k_a_ipb, nblk(nb, 8), 128, 0, s, a->Qs, a->V, a->Qb1, a->Qb, a->Vb, nb, eps);
  AL((void)0);
  MK_DISPATCH(d.MK, k_a_Vh, nblk(d.nq / d.MK), 256, 0, s, a->Vb, a->Vh, d.nq / d.MK);  // one thread per (f, k, mu)
  AL((void)0);
  MK_DISPATCH2(d.MK, k_a_Vb, R, nblk((size_t)d.F * d.T * d.K), 256, 0, s, a->x64, a->Vh, v.y0, v.r0, v.yb, d.F,
               d.T, d.K, eps);
  AL((void)0);
  // reverse of the model at the input state
  AL(k_a_gbar<R><<<nblk(d.fnm * 32), 256, 0, s>>>(v.Ab, v.Db, v.yb, v.lam0, v.P, v.r0, v.gb, d.N, d.F, d.T,
                                                d.M));
  AL(k_a_y_b<R><<<nblk(d.nft), 256, 0, s>>>(v.yb, v.gd, v.lamb, d.N, d.F, d.T, d.M, 0));
  if ((e = nmf_t<R>(d, v.lamb, v.Hd, v.Wb, 1, s)) || (e = nmf_f<R>(d, v.Wd, v.lamb, v.Hb, 1, s))) return e;
  return cudaSuccess;
}

// Loss of the state in (Wd, Hd, gd, Qd) into red and its adjoint into (Qb, Wb, Hb, gb).
cudaError_t loss_and_adjoint(dfmnmf_adj* a, const Dims& d, int loss, const float2* ct, cudaStream_t s) {
  const dfmnmf_ctx* c = a->c;
  const double eps = d.eps;
  const int nb = d.F * d.K;
  cudaError_t e = model<double>(d, a->Wd, a->Hd, a->gd, a->lam0, a->y0, a->r0, s);
  if (e != cudaSuccess) return e;
  ACKE(cudaMemsetAsync(a->red, 0, sizeof(double), s));
  ACKE(cudaMemsetAsync(a->gb, 0, d.fnm * sizeof(double), s));
  const size_t qstr = (size_t)d.MK * d.MK;
  if (loss == DFMNMF_LOSS_NLL) {
    AL(k_a_P<double><<<nblk((size_t)d.F * d.T * d.K), 256, 0, s>>>(a->x64, a->Qd, qstr, a->P, d.F, d.T, d.K, d.MK));
    AL(k_a_nll_data<<<nblk(d.ftm), 256, 0, s>>>(a->P, a->y0, a->r0, a->Pb, a->yb, a->red, d.ftm, eps));
    ACKE(cudaMemsetAsync(a->Qb, 0, d.nq * sizeof(double2), s));
    MK_DISPATCH2(d.MK, k_a_Pb, double, nblk((size_t)d.F * d.K * d.MK * 32), 256, 0, s, a->x64, a->Qd, qstr, a->Pb, a->Qb, d.F,
                d.T, d.K);
    AL((void)0);
    MK_DISPATCH(d.MK, k_a_logdet_b, nblk(nb, 64), 64, 0, s, a->Qd, a->Qb, a->red, nb, d.T);
    AL((void)0);
    AL(k_a_y_b<double><<<nblk(d.nft), 256, 0, s>>>(a->yb, a->gd, a->lamb, d.N, d.F, d.T, d.M, 0));
  } else {
    MK_DISPATCH(d.MK, k_a_inv, nblk(nb, 64), 64, 0, s, a->Qd, a->Binv, nb);
    AL((void)0);
    const double invS = 1.0 / (double)d.nftm;
    MK_DISPATCH(d.MK, k_a_wiener_ft, nblk((size_t)d.F * d.T), 256, 0, s, c->x, a->Qd, a->Binv, ct, a->lam0, a->gd,
                a->y0, a->lamb, a->yb, a->G4, a->ubar, a->cvec, a->zbar, a->red, d.N, d.F, d.T, d.K, eps, invS);
    AL((void)0);
    AL(k_a_wiener_q<<<nblk(d.nq), 256, 0, s>>>(c->x, a->zbar, a->ubar, a->cvec, a->Qb, d.N, d.F, d.T, d.K, d.MK));
    AL(k_a_red_t4<<<nblk(d.fnm * 32), 256, 0, s>>>(a->G4, a->gb, d.N, d.F, d.T, d.M));
    AL(k_a_y_b<double><<<nblk(d.nft), 256, 0, s>>>(a->yb, a->gd, a->lamb, d.N, d.F, d.T, d.M, 1));
  }
  AL(k_a_gbar<double><<<nblk(d.fnm * 32), 256, 0, s>>>(nullptr, nullptr, a->yb, a->lam0, a->P, a->r0, a->gb, d.N, d.F, d.T,
                                                d.M));
  if ((e = nmf_t<double>(d, a->lamb, a->Hd, a->Wb, 0, s)) || (e = nmf_f<double>(d, a->Wd, a->lamb, a->Hb, 0, s))) return e;
  return cudaSuccess;
}

}  // namespace
}  // namespace dfm

using dfm::afail;

namespace {

size_t q_n(const dfmnmf_ctx* c) { return (size_t)c->F * c->K * c->MK * c->MK; }
size_t w_n(const dfmnmf_ctx* c) { return (size_t)c->N * c->F * c->B; }
size_t h_n(const dfmnmf_ctx* c) { return (size_t)c->N * c->B * c->Tp; }
size_t g_n(const dfmnmf_ctx* c) { return (size_t)c->F * c->N * c->M; }

cudaError_t save_state(const dfmnmf_ctx* c, double2* Q, float* W, float* H, float* g, cudaStream_t s) {
  cudaError_t e;
  if ((e = cudaMemcpyAsync(Q, c->Q64, q_n(c) * sizeof(double2), cudaMemcpyDeviceToDevice, s))) return e;
  if ((e = cudaMemcpyAsync(W, c->W, w_n(c) * sizeof(float), cudaMemcpyDeviceToDevice, s))) return e;
  if ((e = cudaMemcpyAsync(H, c->H, h_n(c) * sizeof(float), cudaMemcpyDeviceToDevice, s))) return e;
  return cudaMemcpyAsync(g, c->g, g_n(c) * sizeof(float), cudaMemcpyDeviceToDevice, s);
}

cudaError_t restore_state(dfmnmf_ctx* c, const double2* Q, const float* W, const float* H, const float* g,
                          cudaStream_t s) {
  cudaError_t e;
  if ((e = cudaMemcpyAsync(c->Q64, Q, q_n(c) * sizeof(double2), cudaMemcpyDeviceToDevice, s))) return e;
  if ((e = cudaMemcpyAsync(c->W, W, w_n(c) * sizeof(float), cudaMemcpyDeviceToDevice, s))) return e;
  if ((e = cudaMemcpyAsync(c->H, H, h_n(c) * sizeof(float), cudaMemcpyDeviceToDevice, s))) return e;
  if ((e = cudaMemcpyAsync(c->g, g, g_n(c) * sizeof(float), cudaMemcpyDeviceToDevice, s))) return e;
  if ((e = dfm::launch_lambda(c, s))) return e;
  return dfm::launch_q_convert(c, s);
}

void free_adj(dfmnmf_adj* a) {
  if (!a) return;
  void* p[] = {a->ckQ, a->ckW, a->ckH, a->ckg, a->sgQ, a->sgW, a->sgH, a->sgg, a->fnQ, a->fnW, a->fnH, a->fng,
               a->Wd, a->Hd, a->gd, a->Qd, a->lam0, a->lam1, a->lam2, a->y0, a->y1, a->y2, a->r0, a->r1, a->r2,
               a->P, a->A0, a->D0,
               a->A1, a->D1, a->numW, a->denW, a->W1, a->numH, a->denH, a->H1, a->numG, a->denG, a->V, a->Qs,
               a->Qb, a->Qb1, a->Wb, a->Wb1, a->Hb, a->Hb1, a->gb, a->gb1, a->lamb, a->yb, a->Pb, a->Ab, a->Db,
               a->nb, a->db, a->Vb, a->Vh, a->Binv, a->ubar, a->cvec, a->zbar, a->G4, a->red, a->flags};
  for (void* q : p)
    if (q) cudaFree(q);
  const AdjSide<float>& f = a->sf;
  void* ps[] = {f.Wd, f.Hd, f.gd, f.lam0, f.lam1, f.lam2, f.y0, f.y1, f.y2, f.r0, f.r1, f.r2, f.P, f.A0, f.D0,
                f.A1, f.D1, f.numW, f.denW, f.W1, f.numH, f.denH, f.H1, f.numG, f.denG, f.Wb, f.Wb1, f.Hb, f.Hb1,
                f.gb, f.gb1, f.lamb, f.yb, f.Pb, f.Ab, f.Db, f.nb, f.db};
  for (void* q : ps)
    if (q) cudaFree(q);
  if (a->x64) cudaFree(a->x64);
  if (a->r0d) cudaFree(a->r0d);
  delete a;
}

template <class T>
bool aalloc(T** p, size_t n) {
  if (cudaMalloc(reinterpret_cast<void**>(p), (n ? n : 1) * sizeof(T)) != cudaSuccess) {
    cudaGetLastError();
    *p = nullptr;
    return false;
  }
  return true;
}

}  // namespace

extern "C" {

int dfmnmf_adjoint_create(dfmnmf_adj** out, dfmnmf_ctx* c, int n_iter, int every) {
  if (!out || !c) return afail(DFMNMF_EINVAL, "null argument");
  *out = nullptr;
  if (n_iter < 0 || every < 1) return afail(DFMNMF_EINVAL, "n_iter >= 0 and every >= 1 required");
  if (c->precision != DFMNMF_FP32) return afail(DFMNMF_EINVAL, "the adjoint differentiates the FP32 form");
  if (c->MK < 1 || c->MK > 4) return afail(DFMNMF_EINVAL, "the adjoint supports subarrays of 1 to 4 microphones");
  if (cudaSetDevice(c->device) != cudaSuccess) return afail(DFMNMF_ECUDA, "cudaSetDevice failed");
  dfmnmf_adj* a = new dfmnmf_adj();
  a->c = c;
  a->n_iter = n_iter;
  a->every = every;
  a->device = c->device;
  a->n_ckpt = n_iter > 0 ? (n_iter + every - 1) / every : 0;
  const dfm::Dims d = dfm::dims_of(c);
  const size_t nck = (size_t)(a->n_ckpt > 0 ? a->n_ckpt : 1), nsg = (size_t)every;
  const size_t nmax = std::max(std::max(d.nfb, d.nbt), d.fnm);
  const bool wien = true;
  bool ok = aalloc(&a->ckQ, nck * q_n(c)) && aalloc(&a->ckW, nck * w_n(c)) && aalloc(&a->ckH, nck * h_n(c)) &&
            aalloc(&a->ckg, nck * g_n(c)) && aalloc(&a->sgQ, nsg * q_n(c)) && aalloc(&a->sgW, nsg * w_n(c)) &&
            aalloc(&a->sgH, nsg * h_n(c)) && aalloc(&a->sgg, nsg * g_n(c)) && aalloc(&a->fnQ, q_n(c)) &&
            aalloc(&a->fnW, w_n(c)) && aalloc(&a->fnH, h_n(c)) && aalloc(&a->fng, g_n(c)) &&
            aalloc(&a->Wd, d.nfb) && aalloc(&a->Hd, d.nbt) && aalloc(&a->gd, d.fnm) && aalloc(&a->Qd, d.nq) &&
            aalloc(&a->lam0, d.nft) && aalloc(&a->lam1, d.nft) && aalloc(&a->lam2, d.nft) &&
            aalloc(&a->y0, d.ftm) && aalloc(&a->y1, d.ftm) && aalloc(&a->y2, d.ftm) && aalloc(&a->P, d.ftm) &&
            aalloc(&a->r0, d.ftm) && aalloc(&a->r1, d.ftm) && aalloc(&a->r2, d.ftm) &&
            aalloc(&a->A0, d.nft) && aalloc(&a->D0, d.nft) && aalloc(&a->A1, d.nft) && aalloc(&a->D1, d.nft) &&
            aalloc(&a->numW, d.nfb) && aalloc(&a->denW, d.nfb) && aalloc(&a->W1, d.nfb) &&
            aalloc(&a->numH, d.nbt) && aalloc(&a->denH, d.nbt) && aalloc(&a->H1, d.nbt) &&
            aalloc(&a->numG, d.fnm) && aalloc(&a->denG, d.fnm) && aalloc(&a->V, d.nv) && aalloc(&a->Qs, d.nqs) &&
            aalloc(&a->Qb, d.nq) && aalloc(&a->Qb1, d.nq) && aalloc(&a->Wb, d.nfb) && aalloc(&a->Wb1, d.nfb) &&
            aalloc(&a->Hb, d.nbt) && aalloc(&a->Hb1, d.nbt) && aalloc(&a->gb, d.fnm) && aalloc(&a->gb1, d.fnm) &&
            aalloc(&a->lamb, d.nft) && aalloc(&a->yb, d.ftm) && aalloc(&a->Pb, d.ftm) && aalloc(&a->Ab, d.nft) &&
            aalloc(&a->Db, d.nft) && aalloc(&a->nb, nmax) && aalloc(&a->db, nmax) && aalloc(&a->Vb, d.nv) && aalloc(&a->Vh, d.nv) &&
            aalloc(&a->Binv, d.nq) && (!wien || (aalloc(&a->ubar, d.nftm) && aalloc(&a->cvec, d.nftm) &&
                                                 aalloc(&a->zbar, d.ftm) && aalloc(&a->G4, d.nftm))) &&
            aalloc(&a->red, 1) && aalloc(&a->flags, 4);
  AdjSide<float>& f = a->sf;
  ok = ok && aalloc(&f.Wd, d.nfb) && aalloc(&f.Hd, d.nbt) && aalloc(&f.gd, d.fnm) && aalloc(&f.lam0, d.nft) &&
       aalloc(&f.lam1, d.nft) && aalloc(&f.lam2, d.nft) && aalloc(&f.y0, d.ftm) && aalloc(&f.y1, d.ftm) &&
       aalloc(&f.y2, d.ftm) && aalloc(&f.r0, d.ftm) && aalloc(&f.r1, d.ftm) && aalloc(&f.r2, d.ftm) &&
       aalloc(&f.P, d.ftm) && aalloc(&f.A0, d.nft) && aalloc(&f.D0, d.nft) && aalloc(&f.A1, d.nft) &&
       aalloc(&f.D1, d.nft) && aalloc(&f.numW, d.nfb) && aalloc(&f.denW, d.nfb) && aalloc(&f.W1, d.nfb) &&
       aalloc(&f.numH, d.nbt) && aalloc(&f.denH, d.nbt) && aalloc(&f.H1, d.nbt) && aalloc(&f.numG, d.fnm) &&
       aalloc(&f.denG, d.fnm) && aalloc(&f.Wb, d.nfb) && aalloc(&f.Wb1, d.nfb) && aalloc(&f.Hb, d.nbt) &&
       aalloc(&f.Hb1, d.nbt) && aalloc(&f.gb, d.fnm) && aalloc(&f.gb1, d.fnm) && aalloc(&f.lamb, d.nft) &&
       aalloc(&f.yb, d.ftm) && aalloc(&f.Pb, d.ftm) && aalloc(&f.Ab, d.nft) && aalloc(&f.Db, d.nft) &&
       aalloc(&f.nb, nmax) && aalloc(&f.db, nmax) && aalloc(&a->x64, d.ftm) && aalloc(&a->r0d, d.ftm);
  if (!ok) {
    free_adj(a);
    return afail(DFMNMF_ENOMEM, "device allocation of the adjoint workspace failed");
  }
  *out = a;
  return DFMNMF_OK;
}

int dfmnmf_adjoint_run(dfmnmf_adj* a, int loss, const void* c_true, double* loss_host, void* dQ0, double* dW0,
                       double* dH0, double* dg0, void* stream) {
  if (!a) return afail(DFMNMF_EINVAL, "null adjoint");
  if (loss != DFMNMF_LOSS_NLL && loss != DFMNMF_LOSS_WIENER_MSE) return afail(DFMNMF_EINVAL, "unknown loss %d", loss);
  if (loss == DFMNMF_LOSS_WIENER_MSE && !c_true) return afail(DFMNMF_EINVAL, "the Wiener loss needs c_true");
  dfmnmf_ctx* c = a->c;
  ACK(cudaSetDevice(a->device));
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  const dfm::Dims d = dfm::dims_of(c);
  ACK(cudaMemsetAsync(a->flags, 0, 4 * sizeof(unsigned), s));
  ACK(dfm::convert(reinterpret_cast<const float*>(c->x), reinterpret_cast<double*>(a->x64), 2 * d.ftm, s));
  // forward: the context's own iterations, the state stored every `every` iterations
  for (int i = 0; i < a->n_iter; ++i) {
    if (i % a->every == 0) {
      const size_t j = (size_t)(i / a->every);
      ACK(save_state(c, a->ckQ + j * q_n(c), a->ckW + j * w_n(c), a->ckH + j * h_n(c), a->ckg + j * g_n(c), s));
    }
    int r = dfmnmf_iterate(c, 1, stream);
    if (r) return r;
  }
  ACK(save_state(c, a->fnQ, a->fnW, a->fnH, a->fng, s));
  // loss of the final state and its adjoint
  ACK(dfm::load_state<double>(a, dfm::dside(a), d, a->fnQ, a->fnW, a->fnH, a->fng, s));
  ACK(dfm::loss_and_adjoint(a, d, loss, reinterpret_cast<const float2*>(c_true), s));
  // the unrolled iterations are reversed with the NMF side in single precision (the forward
  // iterations they differentiate run it in single precision too); the loss and its adjoint
  // above, and the IP side throughout, are FP64
  if (a->n_ckpt > 0) {
    ACK(dfm::convert(a->Wb, a->sf.Wb, d.nfb, s));
    ACK(dfm::convert(a->Hb, a->sf.Hb, d.nbt, s));
    ACK(dfm::convert(a->gb, a->sf.gb, d.fnm, s));
  }
  // reverse sweep, one segment per checkpoint, recomputing the segment's states
  for (int j = a->n_ckpt - 1; j >= 0; --j) {
    const int i0 = j * a->every, len = std::min(a->every, a->n_iter - i0);
    ACK(cudaMemcpyAsync(a->sgQ, a->ckQ + (size_t)j * q_n(c), q_n(c) * sizeof(double2), cudaMemcpyDeviceToDevice, s));
    ACK(cudaMemcpyAsync(a->sgW, a->ckW + (size_t)j * w_n(c), w_n(c) * sizeof(float), cudaMemcpyDeviceToDevice, s));
    ACK(cudaMemcpyAsync(a->sgH, a->ckH + (size_t)j * h_n(c), h_n(c) * sizeof(float), cudaMemcpyDeviceToDevice, s));
    ACK(cudaMemcpyAsync(a->sgg, a->ckg + (size_t)j * g_n(c), g_n(c) * sizeof(float), cudaMemcpyDeviceToDevice, s));
    if (len > 1) {
      ACK(restore_state(c, a->sgQ, a->sgW, a->sgH, a->sgg, s));
      for (int i = 1; i < len; ++i) {
        int r = dfmnmf_iterate(c, 1, stream);
        if (r) return r;
        ACK(save_state(c, a->sgQ + (size_t)i * q_n(c), a->sgW + (size_t)i * w_n(c), a->sgH + (size_t)i * h_n(c),
                       a->sgg + (size_t)i * g_n(c), s));
      }
    }
    for (int i = len - 1; i >= 0; --i) {
      std::swap(a->Qb, a->Qb1);
      std::swap(a->sf.Wb, a->sf.Wb1);
      std::swap(a->sf.Hb, a->sf.Hb1);
      std::swap(a->sf.gb, a->sf.gb1);
      ACK(dfm::load_state<float>(a, a->sf, d, a->sgQ + (size_t)i * q_n(c), a->sgW + (size_t)i * w_n(c),
                                 a->sgH + (size_t)i * h_n(c), a->sgg + (size_t)i * g_n(c), s));
      ACK(dfm::reverse_iteration<float>(a, a->sf, d, s));
    }
  }
  if (a->n_ckpt > 0) {
    ACK(dfm::convert(a->sf.Wb, a->Wb, d.nfb, s));
    ACK(dfm::convert(a->sf.Hb, a->Hb, d.nbt, s));
    ACK(dfm::convert(a->sf.gb, a->gb, d.fnm, s));
  }
  // the context ends at the final state, as after dfmnmf_iterate(n_iter)
  ACK(restore_state(c, a->fnQ, a->fnW, a->fnH, a->fng, s));
  if (dQ0) ACK(cudaMemcpyAsync(dQ0, a->Qb, d.nq * sizeof(double2), cudaMemcpyDefault, s));
  if (dW0) ACK(cudaMemcpyAsync(dW0, a->Wb, d.nfb * sizeof(double), cudaMemcpyDefault, s));
  if (dH0) ACK(cudaMemcpyAsync(dH0, a->Hb, d.nbt * sizeof(double), cudaMemcpyDefault, s));
  if (dg0) ACK(cudaMemcpyAsync(dg0, a->gb, d.fnm * sizeof(double), cudaMemcpyDefault, s));
  double L = 0.0;
  unsigned fl[4], cf[dfm::FLAG_COUNT];
  ACK(cudaMemcpyAsync(&L, a->red, sizeof(double), cudaMemcpyDeviceToHost, s));
  ACK(cudaMemcpyAsync(fl, a->flags, sizeof fl, cudaMemcpyDeviceToHost, s));
  ACK(cudaMemcpyAsync(cf, c->flags, sizeof cf, cudaMemcpyDeviceToHost, s));
  ACK(cudaStreamSynchronize(s));
  if (loss_host) *loss_host = L;
  if (fl[0]) return afail(DFMNMF_ENUMERIC, "a system of the IP update was singular: the gradient is not defined");
  if (cf[dfm::FLAG_NONFINITE] || !(L == L) || L > 1e308 || L < -1e308)
    return afail(DFMNMF_ENUMERIC, "a non-finite value was produced");
  return DFMNMF_OK;
}

void dfmnmf_adjoint_destroy(dfmnmf_adj* a) {
  if (!a) return;
  cudaSetDevice(a->device);
  cudaDeviceSynchronize();
  free_adj(a);
}

}  // extern "C"
