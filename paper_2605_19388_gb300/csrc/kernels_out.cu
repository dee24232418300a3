// kernels_out.cu -- on-demand outputs: the negative log-likelihood of
// Eq. (12) and the per-subarray multichannel Wiener filter.
#include "common.cuh"
#include "internal.h"

namespace dfm {

constexpr int NMAXO = 16;

// Data term of Eq. (12): sum_{t,m} (P/yhat + ln yhat) for one (f, 128-frame
// chunk), P recomputed from x and Q.  Per-thread FP32 sums over the M terms
// of a frame, FP64 across frames; one partial per CTA, reduced in a fixed
// order by k_nll_final.
template <int MK>
__global__ void __launch_bounds__(128) k_nll_data(const float2* __restrict__ x, const double2* __restrict__ Q64,
                                                  const float* __restrict__ lam, const float* __restrict__ g,
                                                  double* __restrict__ part, int F, int T, int Tp, int K, int N,
                                                  float eps) {
  extern __shared__ float sm[];
  const int M = K * MK;
  const int f = blockIdx.x;
  float* gs = sm;
  float2* Qh = reinterpret_cast<float2*>(sm + ((N * M + 1) & ~1));
  float2* Ql = Qh + K * MK * MK;
  __shared__ double wsum[4];
  for (int i = threadIdx.x; i < N * M; i += blockDim.x) gs[i] = g[(size_t)f * N * M + i];
  for (int i = threadIdx.x; i < K * MK * MK; i += blockDim.x) split_c(Q64[(size_t)f * K * MK * MK + i], Qh[i], Ql[i]);
  __syncthreads();
  const int t = blockIdx.y * blockDim.x + threadIdx.x;
  double acc = 0.0;
  if (t < T) {
    float lr[NMAXO];
#pragma unroll
    for (int n = 0; n < NMAXO; ++n) lr[n] = (n < N) ? lam[((size_t)n * F + f) * Tp + t] : 0.f;
    for (int k = 0; k < K; ++k) {
      float2 xv[MK];
#pragma unroll
      for (int nu = 0; nu < MK; ++nu) xv[nu] = x[((size_t)f * T + t) * M + k * MK + nu];
      float s = 0.f;
#pragma unroll
      for (int mu = 0; mu < MK; ++mu) {
        const float2 yv = cdot2<MK>(Qh + (k * MK + mu) * MK, Ql + (k * MK + mu) * MK, xv);
        const float p = fmaf(yv.x, yv.x, yv.y * yv.y);
        float ys = 0.f;
#pragma unroll
        for (int n = 0; n < NMAXO; ++n)
          if (n < N) ys = fmaf(lr[n], gs[n * M + k * MK + mu], ys);
        ys = fmaxf(ys, eps);
        s += p / ys + logf(ys);
      }
      acc += (double)s;
    }
  }
  acc = warp_sum_d(acc);
  if ((threadIdx.x & 31) == 0) wsum[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) part[(size_t)f * gridDim.y + blockIdx.y] = ((wsum[0] + wsum[1]) + (wsum[2] + wsum[3]));
}

// nll = sum(data partials) - T * sum(log-dets), both summed in a fixed order.
__global__ void __launch_bounds__(256) k_nll_final(const double* __restrict__ part, size_t npart,
                                                   const double* __restrict__ logdet, size_t nld, int T,
                                                   double* __restrict__ out, unsigned* __restrict__ flags) {
  __shared__ double sd[256], sl[256];
  double a = 0.0, b = 0.0;
  for (size_t i = threadIdx.x; i < npart; i += 256) a += part[i];
  for (size_t i = threadIdx.x; i < nld; i += 256) b += logdet[i];
  sd[threadIdx.x] = a;
  sl[threadIdx.x] = b;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (threadIdx.x < o) {
      sd[threadIdx.x] += sd[threadIdx.x + o];
      sl[threadIdx.x] += sl[threadIdx.x + o];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    const double v = sd[0] - (double)T * sl[0];
    if (!isfinite(v)) atomicOr(flags + FLAG_NONFINITE, 2u);
    *out = v;
  }
}


static size_t gq_smem(const dfmnmf_ctx* c) {
  return (size_t)((c->N * c->M + 1) & ~1) * sizeof(float) + 2 * (size_t)c->K * c->MK * c->MK * sizeof(float2);
}

cudaError_t launch_loglik(const dfmnmf_ctx* c, cudaStream_t s) {
  const int ty = (c->T + 127) / 128;
  const size_t npart = (size_t)c->F * ty;
  double* ld = c->red + npart;
  const size_t nld = (size_t)c->F * c->K;
  if (c->MK == 16) {
    k_nll_data<16><<<dim3(c->F, ty), 128, gq_smem(c), s>>>(c->x, c->Q64, c->lam, c->g, c->red, c->F, c->T, c->Tp,
                                                            c->K, c->N, c->eps);
  } else if (c->MK == 32) {
    k_nll_data<32><<<dim3(c->F, ty), 128, gq_smem(c), s>>>(c->x, c->Q64, c->lam, c->g, c->red, c->F, c->T, c->Tp,
                                                            c->K, c->N, c->eps);
  } else {
    DFM_MK_DISPATCH(c->MK, {
      k_nll_data<MK_><<<dim3(c->F, ty), 128, gq_smem(c), s>>>(c->x, c->Q64, c->lam, c->g, c->red, c->F, c->T,
                                                               c->Tp, c->K, c->N, c->eps);
    });
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  e = launch_logdet(c, ld, s);
  if (e != cudaSuccess) return e;
  k_nll_final<<<1, 256, 0, s>>>(c->red, npart, ld, nld, c->T, c->nll_dev, c->flags);
  return cudaGetLastError();
}

// Wiener filter: c_n = Q^{-1} diag(lambda_n g_n / yhat) Q x per subarray block.
template <int MK>
__global__ void __launch_bounds__(128) k_separate(const float2* __restrict__ x, const double2* __restrict__ Q64,
                                                  const float2* __restrict__ Qinv, const float* __restrict__ lam,
                                                  const float* __restrict__ g, float2* __restrict__ out, int F,
                                                  int T, int Tp, int K, int N, float eps) {
  extern __shared__ float sm[];
  const int M = K * MK;
  const int f = blockIdx.x;
  float* gs = sm;
  float2* Qh = reinterpret_cast<float2*>(sm + ((N * M + 1) & ~1));
  float2* Ql = Qh + K * MK * MK;
  float2* Qi = Ql + K * MK * MK;
  for (int i = threadIdx.x; i < N * M; i += blockDim.x) gs[i] = g[(size_t)f * N * M + i];
  for (int i = threadIdx.x; i < K * MK * MK; i += blockDim.x) {
    split_c(Q64[(size_t)f * K * MK * MK + i], Qh[i], Ql[i]);
    Qi[i] = Qinv[(size_t)f * K * MK * MK + i];
  }
  __syncthreads();
  const int t = blockIdx.y * blockDim.x + threadIdx.x;
  if (t >= T) return;
  float lr[NMAXO];
#pragma unroll
  for (int n = 0; n < NMAXO; ++n) lr[n] = (n < N) ? lam[((size_t)n * F + f) * Tp + t] : 0.f;
  for (int k = 0; k < K; ++k) {
    float2 xv[MK], y[MK];
    float iy[MK];
#pragma unroll
    for (int nu = 0; nu < MK; ++nu) xv[nu] = x[((size_t)f * T + t) * M + k * MK + nu];
#pragma unroll
    for (int mu = 0; mu < MK; ++mu) {
      y[mu] = cdot2<MK>(Qh + (k * MK + mu) * MK, Ql + (k * MK + mu) * MK, xv);
      float ys = 0.f;
#pragma unroll
      for (int n = 0; n < NMAXO; ++n)
        if (n < N) ys = fmaf(lr[n], gs[n * M + k * MK + mu], ys);
      iy[mu] = 1.f / fmaxf(ys, eps);
    }
    for (int n = 0; n < N; ++n) {
      float ln = 0.f;
#pragma unroll
      for (int q = 0; q < NMAXO; ++q) ln = (q == n) ? lr[q] : ln;
      float2 z[MK];
#pragma unroll
      for (int mu = 0; mu < MK; ++mu) {
        const float gain = ln * gs[n * M + k * MK + mu] * iy[mu];
        z[mu] = make_float2(gain * y[mu].x, gain * y[mu].y);
      }
      float2* op = out + (((size_t)n * F + f) * T + t) * M + k * MK;
#pragma unroll
      for (int a = 0; a < MK; ++a) {
        float cr = 0.f, ci = 0.f;
#pragma unroll
        for (int mu = 0; mu < MK; ++mu) {
          const float2 q = Qi[(k * MK + a) * MK + mu];
          cr = fmaf(q.x, z[mu].x, fmaf(-q.y, z[mu].y, cr));
          ci = fmaf(q.x, z[mu].y, fmaf(q.y, z[mu].x, ci));
        }
        op[a] = make_float2(cr, ci);
      }
    }
  }
}

cudaError_t launch_separate(const dfmnmf_ctx* c, float2* out, cudaStream_t s) {
  const int ty = (c->T + 127) / 128;
  const size_t sm = gq_smem(c) + (size_t)c->K * c->MK * c->MK * sizeof(float2);
  if (c->MK == 16) {
    k_separate<16><<<dim3(c->F, ty), 128, sm, s>>>(c->x, c->Q64, c->Qinv32, c->lam, c->g, out, c->F, c->T, c->Tp,
                                                    c->K, c->N, c->eps);
  } else if (c->MK == 32) {
    k_separate<32><<<dim3(c->F, ty), 128, sm, s>>>(c->x, c->Q64, c->Qinv32, c->lam, c->g, out, c->F, c->T, c->Tp,
                                                    c->K, c->N, c->eps);
  } else {
    DFM_MK_DISPATCH(c->MK, {
      k_separate<MK_><<<dim3(c->F, ty), 128, sm, s>>>(c->x, c->Q64, c->Qinv32, c->lam, c->g, out, c->F, c->T,
                                                       c->Tp, c->K, c->N, c->eps);
    });
  }
  return cudaGetLastError();
}

}  // namespace dfm
