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

// One warp per (subarray k, part of the MK^2 packed entries, slice of frames):
// each lane forms only its part of the exact products x_a conj(x_b) and
// accumulates them against all MK weights 1/yhat, so no product is formed
// twice.  x x^H is packed as MK^2 reals R[a*MK+b]: a == b |x_a|^2,
// a < b Re(x_a conj x_b), a > b Im(x_b conj x_a).  Every entry, the diagonal
// ones included, is accumulated with the full two-sum: a new term may exceed
// the running sum (a loud frame after quiet ones), and the fast two-sum then
// drops up to half an ulp of the partial sum, which breaks the rank structure
// of V at the 1e-8 level when T is small.
template <int MK>
struct CovCfg {
  static constexpr int E = MK * MK;
  static constexpr int PARTS = (MK == 4) ? 2 : 1;  // entry parts per subarray
  static constexpr int EP = E / PARTS;              // entries per lane
  static constexpr int C = MK * EP;                 // float-pair accumulators per lane
  static constexpr int CP = (C + 31) / 32 * 32;
};

template <int MK>
__device__ __forceinline__ void exact_entry(const float2 (&xv)[MK], int r, float& hi, float& lo) {
  const int a = r / MK, b = r % MK;
  if (a == b) exact_re(xv[a], xv[a], hi, lo);
  else if (a < b) exact_re(xv[a], xv[b], hi, lo);
  else exact_im(xv[b], xv[a], hi, lo);
}

// Accumulate w_q * R[E0 + j] (exact products) for q < MK, j < EP into the pairs.
template <int MK, int E0, int EP, int CP>
__device__ __forceinline__ void cov_accumulate_impl(const float2 (&xv)[MK], const float (&w)[MK], float (&ah)[CP],
                                                    float (&al)[CP]) {
#pragma unroll
  for (int j = 0; j < EP; ++j) {
    const int r = E0 + j;
    float rh, rl;
    exact_entry<MK>(xv, r, rh, rl);
#pragma unroll
    for (int q = 0; q < MK; ++q) {
      const dd p = two_prod(w[q], rh);
      const float e = __fmaf_rn(w[q], rl, p.lo);
      const dd s = two_sum(ah[q * EP + j], p.hi);
      ah[q * EP + j] = s.hi;
      al[q * EP + j] = __fadd_rn(al[q * EP + j], __fadd_rn(s.lo, e));
    }
  }
}
template <int MK, int E0>
__device__ __forceinline__ void cov_accumulate(const float2 (&xv)[MK], const float (&w)[MK],
                                               float (&ah)[CovCfg<MK>::CP], float (&al)[CovCfg<MK>::CP]) {
  cov_accumulate_impl<MK, E0, CovCfg<MK>::EP, CovCfg<MK>::CP>(xv, w, ah, al);
}

// Frames are staged through shared memory in chunks of CT (x rows and the
// lambda rows of the frequency), double-buffered with cp.async so that the
// float-float arithmetic never waits on global memory.
constexpr int CT = 64;

template <int MK>
__global__ void __launch_bounds__(256, 2) k_cov(const float2* __restrict__ x, const float* __restrict__ lam,
                                                const float* __restrict__ g, double2* __restrict__ V, float4* __restrict__ Vdd,
                                                int F, int T, int Tp, int K, int N, float eps, int fb) {
  using Cfg = CovCfg<MK>;
  constexpr int E = Cfg::E, EP = Cfg::EP, CP = Cfg::CP, PARTS = Cfg::PARTS;
  constexpr int NW = 8;
  const int f = fb + blockIdx.x, tid = threadIdx.x;
  const int M = K * MK;
  const int warp = tid >> 5, lane = tid & 31;
  const int items = K * PARTS;
  const int WPI = (items <= NW) ? NW / items : 1;
  const int nslots = items * WPI;
  const int maxslots = items <= NW ? NW : items;
  extern __shared__ double smd[];
  double* part = smd;                                                      // [maxslots][CP]
  float2* xs = reinterpret_cast<float2*>(smd + (size_t)maxslots * CP);     // [2][CT][M]
  float* ls = reinterpret_cast<float*>(xs + 2 * CT * M);                   // [2][N][CT]
  float* gs = ls + 2 * N * CT;                                             // [N][M]
  for (int i = tid; i < N * M; i += blockDim.x) gs[i] = g[(size_t)f * N * M + i];
  const bool vec = (M % 2) == 0;
  auto issue = [&](int c) {
    const int t0 = c * CT, nt = min(CT, T - t0), buf = c & 1;
    const float2* src = x + ((size_t)f * T + t0) * M;
    float2* dst = xs + (size_t)buf * CT * M;
    if (vec)
      for (int i = tid; i < nt * M / 2; i += blockDim.x) cp_async16(dst + 2 * i, src + 2 * i);
    else
      for (int i = tid; i < nt * M; i += blockDim.x) {
        cp_async4(reinterpret_cast<float*>(dst + i), reinterpret_cast<const float*>(src + i));
        cp_async4(reinterpret_cast<float*>(dst + i) + 1, reinterpret_cast<const float*>(src + i) + 1);
      }
    for (int i = tid; i < N * nt; i += blockDim.x) {
      const int n = i / nt, tt = i % nt;
      cp_async4(ls + (buf * N + n) * CT + tt, lam + ((size_t)n * F + f) * Tp + t0 + tt);
    }
    cp_async_commit();
  };
  // every warp owns slots warp, warp + NW, ...; with K <= NW/PARTS a warp owns one slot
  float ah[CP], al[CP];
  const int nchunk = (T + CT - 1) / CT;
  for (int slot0 = 0; slot0 < nslots; slot0 += NW) {
    const int slot = slot0 + warp;
    const bool mine = slot < nslots;
    const int item = mine ? slot / WPI : 0, pid = mine ? slot % WPI : 0;
    const int k = item / PARTS, e0 = (item % PARTS) * EP;
#pragma unroll
    for (int i = 0; i < CP; ++i) { ah[i] = 0.f; al[i] = 0.f; }
    const float* gsk = gs + k * MK;
    __syncthreads();
    issue(0);
    for (int c = 0; c < nchunk; ++c) {
      if (c + 1 < nchunk) {
        issue(c + 1);
        cp_async_wait<1>();
      } else {
        cp_async_wait<0>();
      }
      __syncthreads();
      const int nt = min(CT, T - c * CT), buf = c & 1;
      const float2* xb = xs + (size_t)buf * CT * M;
      const float* lb = ls + buf * N * CT;
      if (mine) {
        for (int tt = pid * 32 + lane; tt < nt; tt += WPI * 32) {
          float2 xv[MK];
#pragma unroll
          for (int q = 0; q < MK; ++q) xv[q] = xb[tt * M + k * MK + q];
          float ys[MK];
#pragma unroll
          for (int q = 0; q < MK; ++q) ys[q] = 0.f;
          for (int n = 0; n < N; ++n) {
            const float l = lb[n * CT + tt];
#pragma unroll
            for (int q = 0; q < MK; ++q) ys[q] = fmaf(l, gsk[n * M + q], ys[q]);
          }
          float w[MK];
#pragma unroll
          for (int q = 0; q < MK; ++q) w[q] = fast_rcp(fmaxf(ys[q], eps));
          if (e0 == 0) cov_accumulate<MK, 0>(xv, w, ah, al);
          else cov_accumulate<MK, EP>(xv, w, ah, al);
        }
      }
      __syncthreads();
    }
    warp_reduce_scatter_dd<CP>(ah, al, lane);
    if (mine)
#pragma unroll
      for (int i = 0; i < CP / 32; ++i)
        part[slot * CP + lane * (CP / 32) + i] = (double)ah[i] + (double)al[i];
  }
  __syncthreads();
  const double invT = 1.0 / (double)T;
  const int total = K * MK * E;
  for (int idx = tid; idx < total; idx += blockDim.x) {
    const int b = idx % MK, a = (idx / MK) % MK, mu = (idx / E) % MK, k = idx / (MK * E);
    const int lo = a < b ? a : b, hi = a < b ? b : a;
    const int rre = lo * MK + hi, rim = hi * MK + lo;
    double re = 0.0, im = 0.0;
    for (int pid = 0; pid < WPI; ++pid) {
      re += part[((k * PARTS + rre / EP) * WPI + pid) * CP + (rre % EP) + mu * EP];
      if (lo != hi) im += part[((k * PARTS + rim / EP) * WPI + pid) * CP + (rim % EP) + mu * EP];
    }
    if (a > b) im = -im;
    re *= invT;
    im *= invT;
    V[(size_t)f * total + idx] = make_double2(re, im);
    const float rh = (float)re, ih = (float)im;
    Vdd[(size_t)f * total + idx] = make_float4(rh, (float)(re - (double)rh), ih, (float)(im - (double)ih));
  }
}

// ------------------------------------------------------------------------
// One all-microphone block per frequency (conventional FastMNMF, K = 1,
// M_k = MK = 16 or 32: the comparator of the distributed form).  Thread r of
// the CTA owns packed entry r of x x^H (r = a * MK + b: a == b |x_a|^2,
// a < b Re(x_a conj x_b), a > b Im(x_b conj x_a)) and keeps the float-float
// sums of that entry against MUG of the MK weights 1/yhat_mu in registers;
// blockIdx.y selects which MUG (all 16 for MK = 16, a quarter of the 32 for
// MK = 32, so that a thread's accumulators stay within the 64 registers a
// 1024-thread CTA allows).  Frames arrive in chunks of CT through a
// double-buffered cp.async ring (x rows and lambda rows); the weights of a
// chunk are formed once into shared memory and read as broadcasts.
template <int MK, int MUG, int NM>
__global__ void __launch_bounds__(MK * MK) k_cov_all(const float2* __restrict__ x, const float* __restrict__ lam,
                                                      const float* __restrict__ g, double2* __restrict__ V,
                                                      float4* __restrict__ Vdd, int F, int T, int Tp, int N,
                                                      float eps, int fb) {
  constexpr int E = MK * MK, NT = MK * MK;
  const int f = fb + blockIdx.x, tid = threadIdx.x, mu0 = blockIdx.y * MUG;
  extern __shared__ __align__(16) float smc[];
  float2* xs = reinterpret_cast<float2*>(smc);     // [2][CT][MK]
  float* ls = smc + 2 * 2 * CT * MK;               // [2][NM][CT]
  float* ws = ls + 2 * NM * CT;                    // [CT][MUG] weights of the current chunk
  float* gs = ws + CT * MUG;                       // [N][MK]
  for (int i = tid; i < N * MK; i += NT) gs[i] = g[(size_t)f * N * MK + i];
  const int nchunk = (T + CT - 1) / CT;
  auto issue = [&](int c) {
    const int t0 = c * CT, nt = min(CT, T - t0), buf = c & 1;
    const float2* src = x + ((size_t)f * T + t0) * MK;
    float2* dst = xs + (size_t)buf * CT * MK;
    for (int i = tid; i < nt * MK / 2; i += NT) cp_async16(dst + 2 * i, src + 2 * i);
    // lambda rows: warp w copies rows w, w + NT/32, ... in 16-byte pieces (rows are zero up to Tp)
    const int nq = (nt + 3) / 4, q = tid & 31;
    if (q < nq && q < CT / 4)
      for (int n = tid >> 5; n < N; n += NT / 32)
        cp_async16(ls + (buf * NM + n) * CT + 4 * q, lam + ((size_t)n * F + f) * Tp + t0 + 4 * q);
    cp_async_commit();
  };
  const int a = tid / MK, b = tid % MK;
  const bool diag = a == b;
  float ah[MUG], al[MUG];
#pragma unroll
  for (int q = 0; q < MUG; ++q) { ah[q] = 0.f; al[q] = 0.f; }
  __syncthreads();
  issue(0);
  for (int c = 0; c < nchunk; ++c) {
    if (c + 1 < nchunk) {
      issue(c + 1);
      cp_async_wait<1>();
    } else {
      cp_async_wait<0>();
    }
    __syncthreads();
    const int nt = min(CT, T - c * CT), buf = c & 1;
    const float2* xb = xs + (size_t)buf * CT * MK;
    const float* lb = ls + buf * NM * CT;
    // weights w[tt][q] = 1 / max(sum_n lambda g_(mu0 + q), eps) of the chunk's frames
    for (int i = tid; i < CT * MUG; i += NT) {
      const int tt = i / MUG, mu = mu0 + i % MUG;
      float y = 0.f;
#pragma unroll
      for (int n = 0; n < NM; ++n)  // NM is a register bound (8 or 16), not N itself
        if (n < N) y = fmaf(lb[n * CT + tt], gs[n * MK + mu], y);
      ws[i] = tt < nt ? fast_rcp(fmaxf(y, eps)) : 0.f;
    }
    __syncthreads();
    for (int tt = 0; tt < nt; ++tt) {
      const float2 xa = xb[tt * MK + (a < b ? a : b)], xo = xb[tt * MK + (a < b ? b : a)];
      float rh, rl;
      if (a <= b) exact_re(xa, xo, rh, rl);
      else exact_im(xa, xo, rh, rl);
      const float4* wr = reinterpret_cast<const float4*>(ws + tt * MUG);
#pragma unroll
      for (int q4 = 0; q4 < MUG / 4; ++q4) {
        const float4 w4 = wr[q4];
        const float wv[4] = {w4.x, w4.y, w4.z, w4.w};
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int q = q4 * 4 + u;
          const dd p = two_prod(wv[u], rh);
          const float e = __fmaf_rn(wv[u], rl, p.lo);
          const dd s = two_sum(ah[q], p.hi);
          ah[q] = s.hi;
          al[q] = __fadd_rn(al[q], __fadd_rn(s.lo, e));
        }
      }
    }
    __syncthreads();
  }
  // V[f][mu][a][b] (this thread's real or imaginary part, both halves of the Hermitian pair)
  const double invT = 1.0 / (double)T;
#pragma unroll
  for (int q = 0; q < MUG; ++q) {
    const double v = ((double)ah[q] + (double)al[q]) * invT;
    const float vh = (float)v, vl = (float)(v - (double)vh);
    double* Vd = reinterpret_cast<double*>(V + ((size_t)f * MK + mu0 + q) * E);
    float* Vf = reinterpret_cast<float*>(Vdd + ((size_t)f * MK + mu0 + q) * E);
    if (diag) {
      Vd[2 * (a * MK + a)] = v;
      Vd[2 * (a * MK + a) + 1] = 0.0;
      Vf[4 * (a * MK + a)] = vh; Vf[4 * (a * MK + a) + 1] = vl; Vf[4 * (a * MK + a) + 2] = 0.f; Vf[4 * (a * MK + a) + 3] = 0.f;
    } else if (a < b) {  // Re V[a][b] = Re V[b][a]
      Vd[2 * (a * MK + b)] = v;
      Vd[2 * (b * MK + a)] = v;
      Vf[4 * (a * MK + b)] = vh; Vf[4 * (a * MK + b) + 1] = vl;
      Vf[4 * (b * MK + a)] = vh; Vf[4 * (b * MK + a) + 1] = vl;
    } else {  // a > b: Im(x_b conj x_a) = Im V[b][a] = -Im V[a][b]
      Vd[2 * (b * MK + a) + 1] = v;
      Vd[2 * (a * MK + b) + 1] = -v;
      Vf[4 * (b * MK + a) + 2] = vh; Vf[4 * (b * MK + a) + 3] = vl;
      Vf[4 * (a * MK + b) + 2] = -vh; Vf[4 * (a * MK + b) + 3] = -vl;
    }
  }
}

template <int MK, int MUG, int NM>
static cudaError_t launch_cov_all_k(const dfmnmf_ctx* c, cudaStream_t s, int fb, int fc) {
  const size_t sm = ((size_t)2 * 2 * CT * MK + 2 * (size_t)NM * CT + (size_t)CT * MUG + (size_t)c->N * MK) * sizeof(float);
  auto kern = k_cov_all<MK, MUG, NM>;
  if (sm > 48 * 1024) cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  kern<<<dim3(fc, MK / MUG), MK * MK, sm, s>>>(c->x, c->lam, c->g, c->V, c->Vdd, c->F, c->T, c->Tp, c->N, c->eps, fb);
  return cudaGetLastError();
}

template <int MK, int MUG>
static cudaError_t launch_cov_all(const dfmnmf_ctx* c, cudaStream_t s, int fb, int fc) {
  return c->N <= 8 ? launch_cov_all_k<MK, MUG, 8>(c, s, fb, fc) : launch_cov_all_k<MK, MUG, 16>(c, s, fb, fc);
}

cudaError_t launch_cov(const dfmnmf_ctx* c, cudaStream_t s, int fb, int fc) {
  if (c->MK == 16) return launch_cov_all<16, 16>(c, s, fb, fc);
  if (c->MK == 32) return launch_cov_all<32, 8>(c, s, fb, fc);
  DFM_MK_DISPATCH(c->MK, {
    constexpr int CP = CovCfg<MK_>::CP;
    const int items = c->K * CovCfg<MK_>::PARTS;
    const size_t sm = (size_t)(items <= 8 ? 8 : items) * CP * sizeof(double) + 2 * (size_t)CT * c->M * sizeof(float2) +
                      (2 * (size_t)c->N * CT + (size_t)c->N * c->M) * sizeof(float);
    if (sm > 48 * 1024) cudaFuncSetAttribute(k_cov<MK_>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    k_cov<MK_><<<fc, 256, sm, s>>>(c->x, c->lam, c->g, c->V, c->Vdd, c->F, c->T, c->Tp, c->K, c->N, c->eps, fb);
  });
  return cudaGetLastError();
}

}  // namespace dfm
