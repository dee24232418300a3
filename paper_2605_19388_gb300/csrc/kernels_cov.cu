// kernels_cov.cu -- weighted covariances of Eq. (13) in float-float.
//
//   V[f][k][mu] = (1/T) sum_t x_ftk x_ftk^H / yhat_ft(o_k + mu)
//
// With fewer sources than microphones per subarray (the paper's determined
// case, N = 3 on 4-microphone subarrays) V is the covariance of a rank-N
// signal plus a weak noise floor, with condition numbers of 1e6..1e8.  The
// IP update of Eq. (14) is dominated by the noise-floor eigenvector, so
// single-precision rounding of the entries of x x^H (error u |x_a||x_b|,
// i.e. u * lambda_max in the quadratic form) would move its result by
// O(1).  The kernel therefore forms every product x_a conj(x_b) exactly as an
// unevaluated float pair (Dekker's product), multiplies it by the FP32 weight
// 1/yhat exactly, and accumulates hi/lo pairs with Knuth's two-sum; the sum
// is returned in FP64.  The weight itself may carry FP32 rounding: that is a
// relative perturbation of each positive semidefinite term and moves the
// eigenvalues of V only relatively.
#include "common.cuh"
#include "internal.h"

namespace dfm {

constexpr int NMAXC = 16;

// Exact real/imag parts of x_a conj(x_b) as (hi, lo) float pairs.
__device__ __forceinline__ void exact_re(float2 a, float2 b, float& hi, float& lo) {
  const dd p1 = two_prod(a.x, b.x), p2 = two_prod(a.y, b.y);
  const dd s = two_sum(p1.hi, p2.hi);
  hi = s.hi;
  lo = __fadd_rn(__fadd_rn(p1.lo, p2.lo), s.lo);
}
__device__ __forceinline__ void exact_im(float2 a, float2 b, float& hi, float& lo) {
  // Im(a conj b) = a.y b.x - a.x b.y
  const dd p1 = two_prod(a.y, b.x), p2 = two_prod(a.x, b.y);
  const dd s = two_sum(p1.hi, -p2.hi);
  hi = s.hi;
  lo = __fsub_rn(__fadd_rn(p1.lo, s.lo), p2.lo);
}

// Reduce-scatter of C float pairs across a warp (see warp_reduce_scatter);
// pairs are added with two-sum on the high parts.
template <int C>
__device__ __forceinline__ void warp_reduce_scatter_dd(float (&hi)[C], float (&lo)[C], int lane) {
  static_assert(C % 32 == 0, "needs a multiple of 32 entries");
#pragma unroll
  for (int half = C / 2, bit = 16; bit >= 1; half >>= 1, bit >>= 1) {
    const bool upper = (lane & bit) != 0;
#pragma unroll
    for (int i = 0; i < half; ++i) {
      const float kh = upper ? hi[half + i] : hi[i], kl = upper ? lo[half + i] : lo[i];
      const float sh = upper ? hi[i] : hi[half + i], sl = upper ? lo[i] : lo[half + i];
      const float oh = __shfl_xor_sync(DFM_FULL_MASK, sh, bit);
      const float ol = __shfl_xor_sync(DFM_FULL_MASK, sl, bit);
      const dd s = two_sum(kh, oh);
      hi[i] = s.hi;
      lo[i] = __fadd_rn(__fadd_rn(kl, ol), s.lo);
    }
  }
}

// One warp per (subarray k, group of G rows mu, slice of frames); every lane
// keeps G x MK^2 float-pair partial sums.  x x^H is stored packed as MK^2
// reals R[a*MK+b]: a == b |x_a|^2, a < b Re(x_a conj x_b), a > b Im(x_b conj x_a).
template <int MK>
__global__ void __launch_bounds__(256, 2) k_cov(const float2* __restrict__ x, const float* __restrict__ lam,
                                                const float* __restrict__ g, double2* __restrict__ V, int F,
                                                int T, int K, int N, float eps) {
  constexpr int G = (MK == 4) ? 2 : MK;
  constexpr int NG = MK / G;
  constexpr int E = MK * MK;
  constexpr int C = G * E;
  constexpr int CP = (C + 31) / 32 * 32;
  constexpr int NW = 8;
  const int f = blockIdx.x;
  const int M = K * MK;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int items = K * NG;
  const int WPI = (items <= NW) ? NW / items : 1;
  const int nslots = items * WPI;
  extern __shared__ double smd[];
  double* part = smd;                                                   // [nslots][CP]
  float* gs = reinterpret_cast<float*>(smd + (size_t)(items <= NW ? NW : items) * CP);  // [N][M]
  for (int i = threadIdx.x; i < N * M; i += blockDim.x) gs[i] = g[(size_t)f * N * M + i];
  __syncthreads();
  for (int slot = warp; slot < nslots; slot += NW) {
    const int item = slot / WPI, pid = slot % WPI;
    const int k = item / NG, mu0 = (item % NG) * G;
    float ah[CP], al[CP];
#pragma unroll
    for (int i = 0; i < CP; ++i) { ah[i] = 0.f; al[i] = 0.f; }
    const float* gsk = gs + k * MK + mu0;
    for (int t = pid * 32 + lane; t < T; t += WPI * 32) {
      float2 xv[MK];
      load_block<MK>(x + ((size_t)f * T + t) * M + k * MK, xv);
      float ys[G];
#pragma unroll
      for (int q = 0; q < G; ++q) ys[q] = 0.f;
#pragma unroll
      for (int n = 0; n < NMAXC; ++n) {
        if (n < N) {
          const float l = __ldg(lam + ((size_t)n * F + f) * T + t);
#pragma unroll
          for (int q = 0; q < G; ++q) ys[q] = fmaf(l, gsk[n * M + q], ys[q]);
        }
      }
      float w[G];
#pragma unroll
      for (int q = 0; q < G; ++q) w[q] = __frcp_rn(fmaxf(ys[q], eps));
      float rh[E], rl[E];
#pragma unroll
      for (int a = 0; a < MK; ++a) {
        exact_re(xv[a], xv[a], rh[a * MK + a], rl[a * MK + a]);
#pragma unroll
        for (int b = a + 1; b < MK; ++b) {
          exact_re(xv[a], xv[b], rh[a * MK + b], rl[a * MK + b]);
          exact_im(xv[a], xv[b], rh[b * MK + a], rl[b * MK + a]);
        }
      }
#pragma unroll
      for (int q = 0; q < G; ++q)
#pragma unroll
        for (int r = 0; r < E; ++r) {
          const dd p = two_prod(w[q], rh[r]);
          const float e = __fmaf_rn(w[q], rl[r], p.lo);
          const dd s = two_sum(ah[q * E + r], p.hi);
          ah[q * E + r] = s.hi;
          al[q * E + r] = __fadd_rn(al[q * E + r], __fadd_rn(s.lo, e));
        }
    }
    warp_reduce_scatter_dd<CP>(ah, al, lane);
#pragma unroll
    for (int i = 0; i < CP / 32; ++i)
      part[slot * CP + lane * (CP / 32) + i] = (double)ah[i] + (double)al[i];
  }
  __syncthreads();
  const double invT = 1.0 / (double)T;
  const int total = K * MK * E;
  for (int idx = threadIdx.x; idx < total; idx += blockDim.x) {
    const int b = idx % MK, a = (idx / MK) % MK, mu = (idx / E) % MK, k = idx / (MK * E);
    const int lo = a < b ? a : b, hi = a < b ? b : a;
    const int item = k * NG + mu / G, q = mu % G;
    double re = 0.0, im = 0.0;
    for (int pid = 0; pid < WPI; ++pid) {
      const double* pp = part + (item * WPI + pid) * CP + q * E;
      re += pp[lo * MK + hi];
      if (lo != hi) im += pp[hi * MK + lo];
    }
    if (a > b) im = -im;
    V[(size_t)f * total + idx] = make_double2(re * invT, im * invT);
  }
}

cudaError_t launch_cov(const dfmnmf_ctx* c, cudaStream_t s) {
  DFM_MK_DISPATCH(c->MK, {
    constexpr int G = (MK_ == 4) ? 2 : MK_;
    constexpr int CP = (G * MK_ * MK_ + 31) / 32 * 32;
    const int items = c->K * (MK_ / G);
    const size_t sm = (size_t)(items <= 8 ? 8 : items) * CP * sizeof(double) + (size_t)c->N * c->M * sizeof(float);
    if (sm > 48 * 1024) cudaFuncSetAttribute(k_cov<MK_>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    k_cov<MK_><<<c->F, 256, sm, s>>>(c->x, c->lam, c->g, c->V, c->F, c->T, c->K, c->N, c->eps);
  });
  return cudaGetLastError();
}

}  // namespace dfm
