// kernels_model.cu -- per-frequency streaming kernels of one MM iteration.
//
//   k_lambda     lambda[n][f][t] = sum_b W[n][f][b] H[n][b][t]            (Eq. 2)
//   k_pstats     P = |Q_fk x_ftk|^2 (Sec. III-B, y = W^H x) and the MU
//                statistics A = sum_m g P yhat^-2, D = sum_m g yhat^-1 that
//                Eqs. (8) and (9) contract with H and W
//   k_gupd       g <- g sqrt(sum_t lambda P yhat^-2 / max(sum_t lambda yhat^-1, eps)) (Eq. 10)
//
// yhat[f][t][m] = max(sum_n lambda[n][f][t] g[f][n][m], eps) is never stored:
// every kernel rebuilds it in registers from lambda and g (the factorised sum
// stated with Table I), which costs N FMAs per value and saves a [F][T][M]
// round trip through memory.
#include "common.cuh"
#include "internal.h"

namespace dfm {

constexpr int NMAXR = 16;  // register bound on N in the per-frame kernels

// ------------------------------------------------------------------ lambda
__global__ void __launch_bounds__(256) k_lambda(const float* __restrict__ W, const float* __restrict__ H,
                                                float* __restrict__ lam, int F, int T, int B) {
  extern __shared__ float ws[];
  const int n = blockIdx.z, f = blockIdx.y;
  const int t = blockIdx.x * 256 + threadIdx.x;
  for (int b = threadIdx.x; b < B; b += 256) ws[b] = W[((size_t)n * F + f) * B + b];
  __syncthreads();
  if (t >= T) return;
  const float* Hn = H + (size_t)n * B * T + t;
  float s = 0.f;
  for (int b = 0; b < B; ++b) s = fmaf(ws[b], Hn[(size_t)b * T], s);
  lam[((size_t)n * F + f) * T + t] = s;
}

cudaError_t launch_lambda(const dfmnmf_ctx* c, cudaStream_t s) {
  dim3 grid((c->T + 255) / 256, c->F, c->N);
  k_lambda<<<grid, 256, c->B * sizeof(float), s>>>(c->W, c->H, c->lam, c->F, c->T, c->B);
  return cudaGetLastError();
}

// --------------------------------------------------- projected power + stats
// Thread per frame t: P for all M microphones (when COMPUTE_P) or read back,
// then A[n][f][t] = sum_m g P yhat^-2 and D[n][f][t] = sum_m g yhat^-1.
template <int MK, bool COMPUTE_P>
__global__ void __launch_bounds__(128) k_pstats(const float2* __restrict__ x, const double2* __restrict__ Q64,
                                                const float* __restrict__ lam, const float* __restrict__ g,
                                                float* __restrict__ P, float* __restrict__ A,
                                                float* __restrict__ D, int F, int T, int K, int N, float eps) {
  extern __shared__ float sm[];
  const int M = K * MK;
  const int f = blockIdx.x;
  float* gs = sm;                                            // [N][M]
  float2* Qh = reinterpret_cast<float2*>(sm + ((N * M + 1) & ~1));  // [K][MK][MK] high parts
  float2* Ql = Qh + K * MK * MK;                                      // low parts
  for (int i = threadIdx.x; i < N * M; i += blockDim.x) gs[i] = g[(size_t)f * N * M + i];
  if (COMPUTE_P)
    for (int i = threadIdx.x; i < K * MK * MK; i += blockDim.x) split_c(Q64[(size_t)f * K * MK * MK + i], Qh[i], Ql[i]);
  __syncthreads();
  const int t = blockIdx.y * blockDim.x + threadIdx.x;
  if (t >= T) return;
  float lr[NMAXR], accA[NMAXR], accD[NMAXR];
#pragma unroll
  for (int n = 0; n < NMAXR; ++n) {
    lr[n] = (n < N) ? __ldg(lam + ((size_t)n * F + f) * T + t) : 0.f;
    accA[n] = 0.f;
    accD[n] = 0.f;
  }
  float* Pt = P + ((size_t)f * T + t) * M;
  for (int k = 0; k < K; ++k) {
    float pv[MK];
    if (COMPUTE_P) {
      float2 xv[MK];
      load_block<MK>(x + ((size_t)f * T + t) * M + k * MK, xv);
#pragma unroll
      for (int mu = 0; mu < MK; ++mu) {
        const float2 y = cdot2<MK>(Qh + (k * MK + mu) * MK, Ql + (k * MK + mu) * MK, xv);
        pv[mu] = fmaf(y.x, y.x, y.y * y.y);
      }
      if constexpr (MK == 4) {
        *reinterpret_cast<float4*>(Pt + k * MK) = make_float4(pv[0], pv[1], pv[2], pv[3]);
      } else {
#pragma unroll
        for (int mu = 0; mu < MK; ++mu) Pt[k * MK + mu] = pv[mu];
      }
    } else {
      if constexpr (MK == 4) {
        const float4 q = *reinterpret_cast<const float4*>(Pt + k * MK);
        pv[0] = q.x; pv[1] = q.y; pv[2] = q.z; pv[3] = q.w;
      } else {
#pragma unroll
        for (int mu = 0; mu < MK; ++mu) pv[mu] = Pt[k * MK + mu];
      }
    }
#pragma unroll
    for (int mu = 0; mu < MK; ++mu) {
      const int m = k * MK + mu;
      float ys = 0.f;
#pragma unroll
      for (int n = 0; n < NMAXR; ++n)
        if (n < N) ys = fmaf(lr[n], gs[n * M + m], ys);
      const float w = __frcp_rn(fmaxf(ys, eps));
      const float u = pv[mu] * w * w;
#pragma unroll
      for (int n = 0; n < NMAXR; ++n) {
        if (n < N) {
          const float gn = gs[n * M + m];
          accA[n] = fmaf(gn, u, accA[n]);
          accD[n] = fmaf(gn, w, accD[n]);
        }
      }
    }
  }
#pragma unroll
  for (int n = 0; n < NMAXR; ++n) {
    if (n < N) {
      A[((size_t)n * F + f) * T + t] = accA[n];
      D[((size_t)n * F + f) * T + t] = accD[n];
    }
  }
}

// ------------------------------------------------------------------ g update
// One warp per (subarray k, n-chunk of NC sources, t slice); registers hold
// the 2 x NC x MK partial numerators / denominators of Eq. (10).
template <int MK>
__global__ void __launch_bounds__(256) k_gupd(const float* __restrict__ lam, const float* __restrict__ P,
                                              float* __restrict__ g, int F, int T, int K, int N, float eps,
                                              unsigned* __restrict__ flags) {
  constexpr int NC = 8;
  constexpr int C = 2 * NC * MK;
  constexpr int CP = (C + 31) / 32 * 32;
  constexpr int NW = 8;
  const int f = blockIdx.x;
  const int M = K * MK;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  extern __shared__ float sm[];
  float* gs = sm;            // [N][M]
  float* part = sm + N * M;  // [slots][CP]
  for (int i = threadIdx.x; i < N * M; i += blockDim.x) gs[i] = g[(size_t)f * N * M + i];
  __syncthreads();
  const int nchunks = (N + NC - 1) / NC;
  const int items = K * nchunks;
  const int WPI = (items <= NW) ? NW / items : 1;
  const int nslots = items * WPI;
  for (int slot = warp; slot < nslots; slot += NW) {
    const int item = slot / WPI, pid = slot % WPI;
    const int k = item / nchunks;
    const bool upper = (item % nchunks) != 0;
    float acc[CP];
#pragma unroll
    for (int i = 0; i < CP; ++i) acc[i] = 0.f;
    for (int t = pid * 32 + lane; t < T; t += WPI * 32) {
      float lr[NMAXR];
#pragma unroll
      for (int n = 0; n < NMAXR; ++n) lr[n] = (n < N) ? __ldg(lam + ((size_t)n * F + f) * T + t) : 0.f;
      const float* Pt = P + ((size_t)f * T + t) * M + k * MK;
#pragma unroll
      for (int mu = 0; mu < MK; ++mu) {
        const int m = k * MK + mu;
        float ys = 0.f;
#pragma unroll
        for (int n = 0; n < NMAXR; ++n)
          if (n < N) ys = fmaf(lr[n], gs[n * M + m], ys);
        const float w = __frcp_rn(fmaxf(ys, eps));
        const float u = __ldg(Pt + mu) * w * w;
#pragma unroll
        for (int j = 0; j < NC; ++j) {
          // n0 is 0 or NC (N <= 2 NC): both branches index registers statically
          const float l = upper ? lr[NC + j] : lr[j];
          acc[(j * MK + mu) * 2 + 0] = fmaf(l, u, acc[(j * MK + mu) * 2 + 0]);
          acc[(j * MK + mu) * 2 + 1] = fmaf(l, w, acc[(j * MK + mu) * 2 + 1]);
        }
      }
    }
    warp_reduce_scatter<CP>(acc, lane);
#pragma unroll
    for (int i = 0; i < CP / 32; ++i) part[slot * CP + lane * (CP / 32) + i] = acc[i];
  }
  __syncthreads();
  for (int idx = threadIdx.x; idx < N * M; idx += blockDim.x) {
    const int n = idx / M, m = idx % M;
    const int k = m / MK, mu = m % MK;
    const int item = k * nchunks + n / NC, j = n % NC;
    float num = 0.f, den = 0.f;
    for (int pid = 0; pid < WPI; ++pid) {
      const float* pp = part + (item * WPI + pid) * CP;
      num += pp[(j * MK + mu) * 2 + 0];
      den += pp[(j * MK + mu) * 2 + 1];
    }
    const float gnew = gs[idx] * sqrtf(num / fmaxf(den, eps));
    if (!finitef(gnew)) atomicOr(flags + FLAG_NONFINITE, 1u);
    g[(size_t)f * N * M + idx] = gnew;
  }
}

// ----------------------------------------------------------------- launchers

static size_t pstats_smem(const dfmnmf_ctx* c) {
  return (size_t)((c->N * c->M + 1) & ~1) * sizeof(float) + 2 * (size_t)c->K * c->MK * c->MK * sizeof(float2);
}

cudaError_t launch_power_stats(const dfmnmf_ctx* c, cudaStream_t s) {
  dim3 grid(c->F, (c->T + 127) / 128);
  DFM_MK_DISPATCH(c->MK, {
    k_pstats<MK_, true><<<grid, 128, pstats_smem(c), s>>>(c->x, c->Q64, c->lam, c->g, c->P, c->A, c->D, c->F,
                                                         c->T, c->K, c->N, c->eps);
  });
  return cudaGetLastError();
}

cudaError_t launch_stats(const dfmnmf_ctx* c, cudaStream_t s) {
  dim3 grid(c->F, (c->T + 127) / 128);
  DFM_MK_DISPATCH(c->MK, {
    k_pstats<MK_, false><<<grid, 128, pstats_smem(c), s>>>(c->x, c->Q64, c->lam, c->g, c->P, c->A, c->D, c->F,
                                                          c->T, c->K, c->N, c->eps);
  });
  return cudaGetLastError();
}

cudaError_t launch_gupd(const dfmnmf_ctx* c, cudaStream_t s) {
  DFM_MK_DISPATCH(c->MK, {
    constexpr int CP = (2 * 8 * MK_ + 31) / 32 * 32;
    const int nchunks = (c->N + 7) / 8;
    const int items = c->K * nchunks;
    const int slots = items <= 8 ? 8 : items;
    const size_t sm = (size_t)(c->N * c->M + slots * CP) * sizeof(float);
    if (sm > 48 * 1024) cudaFuncSetAttribute(k_gupd<MK_>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    k_gupd<MK_><<<c->F, 256, sm, s>>>(c->lam, c->P, c->g, c->F, c->T, c->K, c->N, c->eps, c->flags);
  });
  return cudaGetLastError();
}

}  // namespace dfm
