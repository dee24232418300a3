// kernels_init.cu -- initialisation from given source images (Sec. IV-A,
// steps 3, 5 and 6; the soft masks that produce the images and the IS-NMF of
// step 4 are outside this library).
//
//   k_init_R     R_fn = sum_t c_nft c_nft^H / T (M x M): exact products summed
//                in float pairs, FP64 out; one CTA per (f, n)
//   k_init_linv  R_fn = L L^H (FP64 Cholesky) and L^{-1}, kept in single
//                precision; one warp per (f, n)
//   k_init_h     h[n][f][t] = c^H R_fn^{-1} c / M = |L^{-1} c|^2 / M
//   k_init_Q     per block (f, k): the generalised eigenvectors w of the pair
//                (R_f,N-2^(k), R_f,N-1^(k)) by Cholesky of the second and cyclic
//                complex Jacobi rotations on L^{-1} R_a L^{-H} (FP64, one warp
//                per block), ascending eigenvalues, w^H R_b w = 1; Q rows w^H;
//                g[f][n][o_k + mu] = w_mu^H R_fn^(k) w_mu
//
// The small dense factorisations run one warp per matrix with the matrix in
// shared memory (lane = row or column), so that no thread needs a large
// local-memory frame.
#include "common.cuh"
#include "internal.h"

namespace dfm {

namespace {

constexpr int IT = 32;    // frames per staged chunk of k_init_R
constexpr int IMAX = 32;  // largest matrix order of the warp factorisations

__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
  return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ double2 cmulc(double2 a, double2 b) {  // a conj(b)
  return make_double2(a.x * b.x + a.y * b.y, a.y * b.x - a.x * b.y);
}

// In-place lower Cholesky factor of the n x n Hermitian matrix A (row-major,
// lower triangle used) by the warp; lane i owns row i.  Returns false (on
// every lane) if a pivot is not positive; that pivot is replaced by a tiny
// value so that the rest stays finite.
__device__ bool warp_cholesky(double2* A, int n, int lane) {
  bool ok = true;
  for (int j = 0; j < n; ++j) {
    __syncwarp();
    double d = A[j * n + j].x;
    if (!(d > 0.0)) {
      ok = false;
      d = 1e-300;
    }
    const double ljj = sqrt(d);
    __syncwarp();
    if (lane > j && lane < n) {
      const double2 v = A[lane * n + j];
      A[lane * n + j] = make_double2(v.x / ljj, v.y / ljj);
    }
    if (lane == j) A[j * n + j] = make_double2(ljj, 0.0);
    __syncwarp();
    if (lane > j && lane < n) {
      const double2 lij = A[lane * n + j];
      for (int c = j + 1; c <= lane; ++c) {  // A[i][c] -= L[i][j] conj(L[c][j])
        const double2 p = cmulc(lij, A[c * n + j]);
        A[lane * n + c].x -= p.x;
        A[lane * n + c].y -= p.y;
      }
    }
  }
  __syncwarp();
  return ok;
}

// X = L^{-1} (lower triangular, zero above the diagonal) by forward
// substitution; lane c owns column c.
__device__ void warp_lower_inverse(const double2* L, double2* X, int n, int lane) {
  if (lane < n) {
    const int c = lane;
    for (int i = 0; i < n; ++i) {
      if (i < c) {
        X[i * n + c] = make_double2(0.0, 0.0);
        continue;
      }
      double sr = (i == c) ? 1.0 : 0.0, si = 0.0;
      for (int q = c; q < i; ++q) {
        const double2 p = cmul(L[i * n + q], X[q * n + c]);
        sr -= p.x;
        si -= p.y;
      }
      const double lii = L[i * n + i].x;
      X[i * n + c] = make_double2(sr / lii, si / lii);
    }
  }
  __syncwarp();
}

}  // namespace

// Thread r of the CTA owns packed entry r = a M + b of c c^H for source
// n = blockIdx.y at frequency f = blockIdx.x: a == b |c_a|^2, a < b
// Re(c_a conj c_b), a > b Im(c_b conj c_a).
__global__ void k_init_R(const float2* __restrict__ c, double2* __restrict__ R, int F, int T, int M) {
  extern __shared__ float2 cs[];  // [IT][M]
  const int f = blockIdx.x, n = blockIdx.y, tid = threadIdx.x;
  const int a = tid / M, b = tid % M;
  const bool act = tid < M * M;
  const int lo = a < b ? a : b, hi = a < b ? b : a;
  float ah = 0.f, al = 0.f;
  for (int t0 = 0; t0 < T; t0 += IT) {
    const int nt = min(IT, T - t0);
    __syncthreads();
    for (int i = tid; i < nt * M; i += blockDim.x) cs[i] = c[(((size_t)n * F + f) * T + t0) * M + i];
    __syncthreads();
    if (act)
      for (int tt = 0; tt < nt; ++tt) {
        const float2 xa = cs[tt * M + lo], xb = cs[tt * M + hi];
        dd p1, p2, sum;
        if (a <= b) {  // Re(x_lo conj x_hi) = xa.x xb.x + xa.y xb.y
          p1 = two_prod(xa.x, xb.x);
          p2 = two_prod(xa.y, xb.y);
          sum = two_sum(p1.hi, p2.hi);
          sum.lo = __fadd_rn(sum.lo, __fadd_rn(p1.lo, p2.lo));
        } else {  // Im(x_lo conj x_hi) = xa.y xb.x - xa.x xb.y
          p1 = two_prod(xa.y, xb.x);
          p2 = two_prod(xa.x, xb.y);
          sum = two_sum(p1.hi, -p2.hi);
          sum.lo = __fadd_rn(sum.lo, __fsub_rn(p1.lo, p2.lo));
        }
        const dd s2 = two_sum(ah, sum.hi);
        ah = s2.hi;
        al = __fadd_rn(al, __fadd_rn(s2.lo, sum.lo));
      }
  }
  if (!act) return;
  const double v = ((double)ah + (double)al) / (double)T;
  double* Rd = reinterpret_cast<double*>(R + ((size_t)n * F + f) * M * M);
  if (a == b) {
    Rd[2 * (a * M + a)] = v;
    Rd[2 * (a * M + a) + 1] = 0.0;
  } else if (a < b) {
    Rd[2 * (a * M + b)] = v;
    Rd[2 * (b * M + a)] = v;
  } else {  // v = Im(c_b conj c_a) = Im R[b][a] = -Im R[a][b]
    Rd[2 * (b * M + a) + 1] = v;
    Rd[2 * (a * M + b) + 1] = -v;
  }
}

// L^{-1} of the Cholesky factor of R_fn, one warp (= CTA) per (f, n), stored
// in single precision [N][F][M][M].  A non-positive pivot sets the
// non-finite flag.
__global__ void __launch_bounds__(32) k_init_linv(const double2* __restrict__ R, float2* __restrict__ Linv, int M,
                                                  unsigned* __restrict__ flags) {
  extern __shared__ double2 sm[];  // L, X: M*M each
  const int id = blockIdx.x, lane = threadIdx.x;
  double2 *L = sm, *X = sm + M * M;
  const double2* Rm = R + (size_t)id * M * M;
  for (int i = lane; i < M * M; i += 32) L[i] = Rm[i];
  const bool ok = warp_cholesky(L, M, lane);
  warp_lower_inverse(L, X, M, lane);
  float2* out = Linv + (size_t)id * M * M;
  for (int i = lane; i < M * M; i += 32) out[i] = make_float2((float)X[i].x, (float)X[i].y);
  if (!ok && lane == 0) atomicOr(flags + FLAG_NONFINITE, 1u);
}

// h[n][f][t] = |L^{-1} c|^2 / M, one thread per frame of a (f, n).
__global__ void k_init_h(const float2* __restrict__ c, const float2* __restrict__ Linv, float* __restrict__ h, int F,
                         int T, int M) {
  const int f = blockIdx.y, n = blockIdx.z;
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= T) return;
  const float2* L = Linv + ((size_t)n * F + f) * M * M;
  const float2* cv = c + (((size_t)n * F + f) * T + t) * M;
  float acc = 0.f;
  for (int i = 0; i < M; ++i) {
    float zr = 0.f, zi = 0.f;
    for (int k = 0; k <= i; ++k) {
      const float2 l = __ldg(L + i * M + k), x = __ldg(cv + k);
      zr = fmaf(l.x, x.x, fmaf(-l.y, x.y, zr));
      zi = fmaf(l.x, x.y, fmaf(l.y, x.x, zi));
    }
    acc = fmaf(zr, zr, fmaf(zi, zi, acc));
  }
  h[((size_t)n * F + f) * T + t] = acc / (float)M;
}

// One warp (= CTA) per block id = f K + k: generalised eigenvectors of
// (R_a, R_b), the k-th diagonal blocks of the covariances of sources N-2 and
// N-1.  Shared memory, MK*MK entries each: L (Cholesky factor of R_b, later
// X R_a), X = L^{-1}, C = X R_a X^H (rotated to diagonal, later the
// eigenvectors), U (accumulated rotations).
__global__ void __launch_bounds__(32) k_init_Q(const double2* __restrict__ R, double2* __restrict__ Q64,
                                               float* __restrict__ g, int F, int K, int MK, int N,
                                               unsigned* __restrict__ flags) {
  extern __shared__ double2 sm[];
  const int id = blockIdx.x, lane = threadIdx.x;
  const int f = id / K, k = id % K, M = K * MK, o = k * MK, n2 = MK * MK;
  double2 *L = sm, *X = sm + n2, *C = X + n2, *U = C + n2;
  auto Rblk = [&](int n, int a, int b) { return R[((size_t)n * F + f) * M * M + (size_t)(o + a) * M + o + b]; };
  for (int i = lane; i < n2; i += 32) {
    L[i] = Rblk(N - 1, i / MK, i % MK);
    U[i] = make_double2(i / MK == i % MK ? 1.0 : 0.0, 0.0);
  }
  const bool ok = warp_cholesky(L, MK, lane);
  warp_lower_inverse(L, X, MK, lane);
  // C = X R_a X^H; lane i forms row i of X R_a (in L's storage), then row i of C
  double2* Tm = L;
  if (lane < MK) {
    const int i = lane;
    for (int j = 0; j < MK; ++j) {
      double sr = 0.0, si = 0.0;
      for (int q = 0; q < MK; ++q) {
        const double2 p = cmul(X[i * MK + q], Rblk(N - 2, q, j));
        sr += p.x;
        si += p.y;
      }
      Tm[i * MK + j] = make_double2(sr, si);
    }
    for (int j = 0; j < MK; ++j) {
      double sr = 0.0, si = 0.0;
      for (int q = 0; q < MK; ++q) {  // T[i][q] conj(X[j][q])
        const double2 p = cmulc(Tm[i * MK + q], X[j * MK + q]);
        sr += p.x;
        si += p.y;
      }
      C[i * MK + j] = make_double2(sr, si);
    }
  }
  __syncwarp();
  // cyclic complex Jacobi: with e = C_pq / |C_pq| and the real rotation
  // (cs, sn) that zeroes the off-diagonal entry of the 2 x 2 symmetric
  // [[a, |z|], [|z|, b]], the unitary acting on columns (p, q) is
  // p' = cs p - sn conj(e) q, q' = sn p + cs conj(e) q; C <- U^H C U (columns,
  // then rows with e in place of conj(e)) and U accumulates the columns.
  for (int sweep = 0; sweep < 60; ++sweep) {
    double off = 0.0;
    for (int p = 0; p < MK; ++p)
      for (int q = p + 1; q < MK; ++q) {
        const double2 z = C[p * MK + q];
        const double ca = C[p * MK + p].x, cb = C[q * MK + q].x;
        const double az = sqrt(z.x * z.x + z.y * z.y);
        const double scale = fabs(ca) + fabs(cb);
        __syncwarp();
        if (!(az > 1e-300) || !(az > 1e-17 * scale)) continue;
        off = fmax(off, az / fmax(scale, 1e-300));
        const double er = z.x / az, ei = z.y / az;
        const double tau = (cb - ca) / (2.0 * az);
        const double t = (tau >= 0.0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
        const double cs = 1.0 / sqrt(1.0 + t * t), sn = t * cs;
        if (lane < MK) {
          const int r = lane;
          const double2 up = C[r * MK + p], uq = C[r * MK + q];
          const double cqr = er * uq.x + ei * uq.y, cqi = er * uq.y - ei * uq.x;  // conj(e) uq
          C[r * MK + p] = make_double2(cs * up.x - sn * cqr, cs * up.y - sn * cqi);
          C[r * MK + q] = make_double2(sn * up.x + cs * cqr, sn * up.y + cs * cqi);
          const double2 vp = U[r * MK + p], vq = U[r * MK + q];
          const double cvr = er * vq.x + ei * vq.y, cvi = er * vq.y - ei * vq.x;
          U[r * MK + p] = make_double2(cs * vp.x - sn * cvr, cs * vp.y - sn * cvi);
          U[r * MK + q] = make_double2(sn * vp.x + cs * cvr, sn * vp.y + cs * cvi);
        }
        __syncwarp();
        if (lane < MK) {
          const int cc = lane;
          const double2 rp = C[p * MK + cc], rq = C[q * MK + cc];
          const double eqr = er * rq.x - ei * rq.y, eqi = er * rq.y + ei * rq.x;  // e rq
          C[p * MK + cc] = make_double2(cs * rp.x - sn * eqr, cs * rp.y - sn * eqi);
          C[q * MK + cc] = make_double2(sn * rp.x + cs * eqr, sn * rp.y + cs * eqi);
        }
        __syncwarp();
      }
    if (off < 1e-16) break;
  }
  // lane s: rank of the eigenvalue C_ss among all (ascending, ties by index)
  int rank = 0;
  if (lane < MK) {
    const double ds = C[lane * MK + lane].x;
    for (int j = 0; j < MK; ++j) {
      const double dj = C[j * MK + j].x;
      rank += (dj < ds || (dj == ds && j < lane)) ? 1 : 0;
    }
  }
  __syncwarp();
  // w_s = X^H u_s into column s of C; row `rank` of Q is w_s^H
  double2* Wm = C;
  if (lane < MK) {
    const int s = lane;
    for (int j = 0; j < MK; ++j) {  // w_j = sum_q conj(X[q][j]) U[q][s]
      double sr = 0.0, si = 0.0;
      for (int q = 0; q < MK; ++q) {
        const double2 p = cmulc(U[q * MK + s], X[q * MK + j]);
        sr += p.x;
        si += p.y;
      }
      Wm[j * MK + s] = make_double2(sr, si);
    }
    double2* qrow = Q64 + (size_t)id * n2 + (size_t)rank * MK;
    for (int j = 0; j < MK; ++j) qrow[j] = make_double2(Wm[j * MK + s].x, -Wm[j * MK + s].y);
    for (int n = 0; n < N; ++n) {  // w^H R_n w
      double acc = 0.0;
      for (int a = 0; a < MK; ++a) {
        double tr = 0.0, ti = 0.0;
        for (int b = 0; b < MK; ++b) {
          const double2 p = cmul(Rblk(n, a, b), Wm[b * MK + s]);
          tr += p.x;
          ti += p.y;
        }
        const double2 wa = Wm[a * MK + s];
        acc += wa.x * tr + wa.y * ti;  // Re(conj(w_a) (R w)_a)
      }
      g[((size_t)f * N + n) * M + o + rank] = (float)acc;
    }
  }
  if (!ok && lane == 0) atomicOr(flags + FLAG_NONFINITE, 1u);
}

bool init_supported(int M, int MK) { return M <= IMAX && MK <= IMAX; }

cudaError_t launch_init_from_images(dfmnmf_ctx* c, const float2* cimg, double2* R, float2* Linv, float* h,
                                    cudaStream_t s) {
  const int M = c->M, MK = c->MK;
  if (!init_supported(M, MK)) return cudaErrorInvalidValue;
  k_init_R<<<dim3(c->F, c->N), ((M * M + 31) / 32) * 32, (size_t)IT * M * sizeof(float2), s>>>(cimg, R, c->F, c->T,
                                                                                               M);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_init_Q<<<c->F * c->K, 32, (size_t)4 * MK * MK * sizeof(double2), s>>>(R, c->Q64, c->g, c->F, c->K, MK, c->N,
                                                                           c->flags);
  e = cudaGetLastError();
  if (e != cudaSuccess || !h) return e;
  k_init_linv<<<c->N * c->F, 32, (size_t)2 * M * M * sizeof(double2), s>>>(R, Linv, M, c->flags);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_init_h<<<dim3((c->T + 127) / 128, c->F, c->N), 128, 0, s>>>(cimg, Linv, h, c->F, c->T, M);
  return cudaGetLastError();
}

}  // namespace dfm
