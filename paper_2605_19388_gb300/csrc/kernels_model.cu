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
#include "../../include/dfmnmf.h"

namespace dfm {


// ------------------------------------------------------------------ lambda
// lambda[n][f][t] = sum_b W[n][f][b] H[n][b][t] (Eq. 2) for a tile of
// LAM_F frequencies x 256 frames of one source.  The W rows of the tile sit
// in shared memory; each thread keeps H of four adjacent frames for 16 bases
// at a time in registers (float4 loads; the row stride Tp is a multiple of 4)
// and writes four frames of each frequency as one float4, so every W value
// read from shared memory serves four FMAs.  Frames T .. Tp-1 are written
// too: H is zero there, so the zero tail of lambda is kept.
constexpr int LAM_F = 8;
constexpr int LAM_THREADS = 64;

__global__ void __launch_bounds__(LAM_THREADS) k_lambda(const float* __restrict__ W, const float* __restrict__ H,
                                                        float* __restrict__ lam, int F, int Tp, int B) {
  extern __shared__ __align__(16) float ws[];  // [LAM_F][Bq], Bq = B rounded up to 16, zero padded
  const int n = blockIdx.z, f0 = blockIdx.y * LAM_F;
  const int Bq = (B + 15) & ~15;
  const int t = 4 * (blockIdx.x * LAM_THREADS + threadIdx.x);
  {
    // W tile: all loads issued before any store (B <= 64: at most 8 per thread)
    float v[LAM_F * 64 / LAM_THREADS];
#pragma unroll
    for (int k = 0; k < LAM_F * 64 / LAM_THREADS; ++k) {
      const int i = threadIdx.x + k * LAM_THREADS, fi = i / Bq, b = i % Bq;
      v[k] = (i < LAM_F * Bq && f0 + fi < F && b < B) ? __ldg(W + ((size_t)n * F + f0 + fi) * B + b) : 0.f;
    }
#pragma unroll
    for (int k = 0; k < LAM_F * 64 / LAM_THREADS; ++k) {
      const int i = threadIdx.x + k * LAM_THREADS;
      if (i < LAM_F * Bq) ws[i] = v[k];
    }
  }
  __syncthreads();
  if (t >= Tp) return;
  const float* Hn = H + (size_t)n * B * Tp + t;
  const int nf = min(LAM_F, F - f0);
  float4 acc[LAM_F];
#pragma unroll
  for (int fi = 0; fi < LAM_F; ++fi) acc[fi] = make_float4(0.f, 0.f, 0.f, 0.f);
  for (int b0 = 0; b0 < Bq; b0 += 16) {
    float4 h[16];
#pragma unroll
    for (int j = 0; j < 16; ++j)
      h[j] = (b0 + j < B) ? __ldg(reinterpret_cast<const float4*>(Hn + (size_t)(b0 + j) * Tp))
                          : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
    for (int fi = 0; fi < LAM_F; ++fi) {
#pragma unroll
      for (int j = 0; j < 16; ++j) {
        const float wv = ws[fi * Bq + b0 + j];
        acc[fi].x = fmaf(wv, h[j].x, acc[fi].x);
        acc[fi].y = fmaf(wv, h[j].y, acc[fi].y);
        acc[fi].z = fmaf(wv, h[j].z, acc[fi].z);
        acc[fi].w = fmaf(wv, h[j].w, acc[fi].w);
      }
    }
  }
#pragma unroll
  for (int fi = 0; fi < LAM_F; ++fi)
    if (fi < nf) *reinterpret_cast<float4*>(lam + ((size_t)n * F + f0 + fi) * Tp + t) = acc[fi];
}

cudaError_t launch_lambda(const dfmnmf_ctx* c, cudaStream_t s) {
  dim3 grid((c->Tp / 4 + LAM_THREADS - 1) / LAM_THREADS, (c->F + LAM_F - 1) / LAM_F, c->N);
  const size_t sm = (size_t)LAM_F * ((c->B + 15) & ~15) * sizeof(float);
  k_lambda<<<grid, LAM_THREADS, sm, s>>>(c->W, c->H, c->lam, c->F, c->Tp, c->B);
  return cudaGetLastError();
}

// --------------------------------------------------- projected power + stats
// Thread per (frame t, subarray k).  The thread projects x_ftk (when
// COMPUTE_P: compensated dot products when COMP, plain FP32 otherwise) or
// reads P back, rebuilds yhat for its M_k microphones, and forms its
// subarray's share of A[n][f][t] = sum_m g P yhat^-2 and
// D[n][f][t] = sum_m g yhat^-1 one source at a time (g rows as vector loads
// from shared memory), so nothing is padded to a maximum source count.  The
// K shares of a frame sit in adjacent lanes and are added by xor shuffles
// (K a power of two) or through shared memory.
// Row of MK floats from shared memory, 16 bytes per load when MK is a
// multiple of 4 (callers pass rows that start at multiples of MK floats of a
// 16-byte aligned array).
template <int MK>
__device__ __forceinline__ void load_row(const float* __restrict__ p, float (&v)[MK]) {
  if constexpr (MK % 4 == 0) {
#pragma unroll
    for (int i = 0; i < MK; i += 4) {
      const float4 q = *reinterpret_cast<const float4*>(p + i);
      v[i] = q.x; v[i + 1] = q.y; v[i + 2] = q.z; v[i + 3] = q.w;
    }
  } else {
#pragma unroll
    for (int i = 0; i < MK; ++i) v[i] = p[i];
  }
}

template <int MK, bool COMPUTE_P, bool COMP>
__global__ void __launch_bounds__(256) k_pstats(const float2* __restrict__ x, const double2* __restrict__ Q64,
                                                const float* __restrict__ lam, const float* __restrict__ g,
                                                float* __restrict__ P, float* __restrict__ A,
                                                float* __restrict__ D, int F, int T, int Tp, int K, int N, float eps,
                                                int fb) {
  extern __shared__ __align__(16) float sm[];
  const int f = fb + blockIdx.x, tid = threadIdx.x;
  const int M = K * MK;
  const int TB = blockDim.x / K;
  const int k = tid % K, tl = tid / K;
  const int t = blockIdx.y * TB + tl;
  const bool valid = tl < TB && t < T;
  const bool pow2 = (K & (K - 1)) == 0;
  float* gs = sm;                                                  // [N][M]
  const int qoff = (N * M + 3) & ~3;
  float2* Qh = reinterpret_cast<float2*>(sm + qoff);               // [K][MK][MK] high parts
  float2* Ql = Qh + K * MK * MK;                                   // low parts
  float* red = sm + qoff + (COMPUTE_P ? 4 * K * MK * MK : 0);      // [TB][K][2] when K is not a power of two
  for (int i = tid; i < N * M; i += blockDim.x) gs[i] = g[(size_t)f * N * M + i];
  if (COMPUTE_P)
    for (int i = tid; i < K * MK * MK; i += blockDim.x) split_c(Q64[(size_t)f * K * MK * MK + i], Qh[i], Ql[i]);
  __syncthreads();
  const int tc = valid ? t : 0;
  float pv[MK];
  float* Pt = P + ((size_t)f * T + tc) * M + k * MK;
  if (COMPUTE_P) {
    float2 xv[MK];
    load_block<MK>(x + ((size_t)f * T + tc) * M + k * MK, xv);
#pragma unroll
    for (int mu = 0; mu < MK; ++mu) {
      const float2* qh = Qh + (k * MK + mu) * MK;
      float2 y;
      if (COMP) {
        y = cdot2<MK>(qh, Ql + (k * MK + mu) * MK, xv);
      } else {
        float yr = 0.f, yi = 0.f;
#pragma unroll
        for (int nu = 0; nu < MK; ++nu) {
          yr = fmaf(qh[nu].x, xv[nu].x, fmaf(-qh[nu].y, xv[nu].y, yr));
          yi = fmaf(qh[nu].x, xv[nu].y, fmaf(qh[nu].y, xv[nu].x, yi));
        }
        y = make_float2(yr, yi);
      }
      pv[mu] = fmaf(y.x, y.x, y.y * y.y);
    }
    if (valid) {
      if constexpr (MK == 4) {
        *reinterpret_cast<float4*>(Pt) = make_float4(pv[0], pv[1], pv[2], pv[3]);
      } else {
#pragma unroll
        for (int mu = 0; mu < MK; ++mu) Pt[mu] = pv[mu];
      }
    }
  } else {
    load_row<MK>(Pt, pv);
  }
  // yhat for the subarray's microphones
  float ys[MK];
#pragma unroll
  for (int mu = 0; mu < MK; ++mu) ys[mu] = 0.f;
  const float* lt = lam + (size_t)f * Tp + tc;
  for (int n = 0; n < N; ++n) {
    const float l = __ldg(lt + (size_t)n * F * Tp);
    float gv[MK];
    load_row<MK>(gs + n * M + k * MK, gv);
#pragma unroll
    for (int mu = 0; mu < MK; ++mu) ys[mu] = fmaf(l, gv[mu], ys[mu]);
  }
  float w[MK], u[MK];
#pragma unroll
  for (int mu = 0; mu < MK; ++mu) {
    w[mu] = fast_rcp(fmaxf(ys[mu], eps));
    u[mu] = pv[mu] * w[mu] * w[mu];
  }
  for (int n = 0; n < N; ++n) {
    float gv[MK];
    load_row<MK>(gs + n * M + k * MK, gv);
    float a = 0.f, d = 0.f;
#pragma unroll
    for (int mu = 0; mu < MK; ++mu) {
      a = fmaf(gv[mu], u[mu], a);
      d = fmaf(gv[mu], w[mu], d);
    }
    const size_t o = ((size_t)n * F + f) * Tp + tc;
    if (pow2) {
      for (int s = 1; s < K; s <<= 1) {
        a += __shfl_xor_sync(DFM_FULL_MASK, a, s);
        d += __shfl_xor_sync(DFM_FULL_MASK, d, s);
      }
      if (valid && k == 0) {
        A[o] = a;
        D[o] = d;
      }
    } else {
      __syncthreads();
      if (tl < TB) {
        red[(tl * K + k) * 2] = a;
        red[(tl * K + k) * 2 + 1] = d;
      }
      __syncthreads();
      if (valid && k == 0) {
        float sa = 0.f, sd = 0.f;
        for (int kk = 0; kk < K; ++kk) {
          sa += red[(tl * K + kk) * 2];
          sd += red[(tl * K + kk) * 2 + 1];
        }
        A[o] = sa;
        D[o] = sd;
      }
    }
  }
}

// Frame-per-thread variant for the common layouts (compile-time K and M_k):
// every thread owns whole frames of one frequency, keeps P, yhat, w and u of
// all M microphones in registers, reads g[f] rows from shared memory as
// broadcast vector loads and writes A, D for every source -- no shuffles and
// no per-subarray redundancy.  Q (split in two floats) is read from shared
// memory when P is formed here.
template <int K, int MK, bool COMPUTE_P, bool COMP>
__global__ void __launch_bounds__(128) k_pstats_ft(const float2* __restrict__ x, const double2* __restrict__ Q64,
                                                   const float* __restrict__ lam, const float* __restrict__ g,
                                                   float* __restrict__ P, float* __restrict__ A,
                                                   float* __restrict__ D, int F, int T, int Tp, int N, float eps,
                                                   int fb, int tpc) {
  constexpr int M = K * MK;
  extern __shared__ __align__(16) float sm[];
  const int f = fb + blockIdx.x, tid = threadIdx.x;
  float* gs = sm;                                                       // [N][M]
  float2* Qh = reinterpret_cast<float2*>(sm + ((N * M + 3) & ~3));      // [K][MK][MK] high parts
  float2* Ql = Qh + K * MK * MK;                                        // low parts
  for (int i = tid; i < N * M; i += blockDim.x) gs[i] = g[(size_t)f * N * M + i];
  if (COMPUTE_P)
    for (int i = tid; i < K * MK * MK; i += blockDim.x) split_c(Q64[(size_t)f * K * MK * MK + i], Qh[i], Ql[i]);
  __syncthreads();
  const int t0 = blockIdx.y * tpc, t1 = min(T, t0 + tpc);
  const float* lt = lam + (size_t)f * Tp;
#pragma unroll 2
  for (int t = t0 + tid; t < t1; t += blockDim.x) {
    float pv[M];
    float* Pt = P + ((size_t)f * T + t) * M;
    if (COMPUTE_P) {
#pragma unroll
      for (int k = 0; k < K; ++k) {
        float2 xv[MK];
        load_block<MK>(x + ((size_t)f * T + t) * M + k * MK, xv);
#pragma unroll
        for (int mu = 0; mu < MK; ++mu) {
          const float2* qh = Qh + (k * MK + mu) * MK;
          float2 y;
          if (COMP) {
            y = cdot2<MK>(qh, Ql + (k * MK + mu) * MK, xv);
          } else {
            float yr = 0.f, yi = 0.f;
#pragma unroll
            for (int nu = 0; nu < MK; ++nu) {
              yr = fmaf(qh[nu].x, xv[nu].x, fmaf(-qh[nu].y, xv[nu].y, yr));
              yi = fmaf(qh[nu].x, xv[nu].y, fmaf(qh[nu].y, xv[nu].x, yi));
            }
            y = make_float2(yr, yi);
          }
          pv[k * MK + mu] = fmaf(y.x, y.x, y.y * y.y);
        }
      }
      if constexpr (M % 4 == 0) {
#pragma unroll
        for (int m = 0; m < M; m += 4)
          *reinterpret_cast<float4*>(Pt + m) = make_float4(pv[m], pv[m + 1], pv[m + 2], pv[m + 3]);
      } else {
#pragma unroll
        for (int m = 0; m < M; ++m) Pt[m] = pv[m];
      }
    } else {
      if constexpr (M % 4 == 0) {
#pragma unroll
        for (int m = 0; m < M; m += 4) {
          const float4 q = *reinterpret_cast<const float4*>(Pt + m);
          pv[m] = q.x; pv[m + 1] = q.y; pv[m + 2] = q.z; pv[m + 3] = q.w;
        }
      } else {
#pragma unroll
        for (int m = 0; m < M; ++m) pv[m] = Pt[m];
      }
    }
    // the lambda of up to LAM_R sources are requested together (one memory
    // latency instead of one per source); more sources follow in a loop
    constexpr int LAM_R = 8;
    float lv[LAM_R];
#pragma unroll
    for (int n = 0; n < LAM_R; ++n) lv[n] = n < N ? __ldg(lt + (size_t)n * F * Tp + t) : 0.f;
    float ys[M];
#pragma unroll
    for (int m = 0; m < M; ++m) ys[m] = 0.f;
#pragma unroll
    for (int n = 0; n < LAM_R; ++n) {
      if (n < N) {
        float gr[M];
        load_row<M>(gs + n * M, gr);
#pragma unroll
        for (int m = 0; m < M; ++m) ys[m] = fmaf(lv[n], gr[m], ys[m]);
      }
    }
    for (int n = LAM_R; n < N; ++n) {
      const float l = __ldg(lt + (size_t)n * F * Tp + t);
      float gr[M];
      load_row<M>(gs + n * M, gr);
#pragma unroll
      for (int m = 0; m < M; ++m) ys[m] = fmaf(l, gr[m], ys[m]);
    }
    float w[M], u[M];
#pragma unroll
    for (int m = 0; m < M; ++m) {
      w[m] = fast_rcp(fmaxf(ys[m], eps));
      u[m] = pv[m] * w[m] * w[m];
    }
    for (int n = 0; n < N; ++n) {
      float gr[M];
      load_row<M>(gs + n * M, gr);
      float a = 0.f, d = 0.f;
#pragma unroll
      for (int m = 0; m < M; ++m) {
        a = fmaf(gr[m], u[m], a);
        d = fmaf(gr[m], w[m], d);
      }
      const size_t o = ((size_t)n * F + f) * Tp + t;
      A[o] = a;
      D[o] = d;
    }
  }
}

// ------------------------------------------------------------------ g update
// One CTA per frequency.  Frames arrive in chunks of GT through an NST-stage
// cp.async ring (lambda rows and the [t][m] block of P), NST - 1 chunks
// ahead of the one being used; thread (slice s, microphone m) keeps
// g[f][:][m] and the 2 N partial sums of Eq. (10) in registers, and the
// slices are added in a fixed order at the end.
constexpr int GT = 128;

// NM is N itself for N <= 8 (no padded work) and 16 (guarded) above.
template <int NM, int NST>
__global__ void __launch_bounds__(256) k_gupd(const float* __restrict__ lam, const float* __restrict__ P,
                                              float* __restrict__ g, int F, int T, int Tp, int M, int N, float eps,
                                              unsigned* __restrict__ flags, float* __restrict__ grad) {
  extern __shared__ __align__(16) float smg[];
  const int f = blockIdx.x, tid = threadIdx.x;
  const int S = blockDim.x / M;            // frame slices
  const int m = tid % M, s = tid / M;
  const bool active = s < S;
  float* ls = smg;                         // [NST][N][GT]
  float* ps = ls + NST * N * GT;           // [NST][GT][M]
  float* red = ps + NST * GT * M;          // [S][M][2N]
  const bool vec = (M % 4) == 0;
  const int nchunk = (T + GT - 1) / GT;
  auto issue = [&](int c) {
    if (c < nchunk) {
      const int t0 = c * GT, nt = min(GT, T - t0), buf = c % NST;
      // lambda rows: warp w copies rows w, w + 8, ... as 16-byte pieces (rows are
      // 16-byte aligned and zero up to Tp, so the last piece may run past T)
      const int nq = (nt + 3) / 4, q = tid & 31;
      if (q < nq)
        for (int n = tid >> 5; n < N; n += 8)
          cp_async16(ls + (buf * N + n) * GT + 4 * q, lam + ((size_t)n * F + f) * Tp + t0 + 4 * q);
      const float* src = P + ((size_t)f * T + t0) * M;
      float* dst = ps + (size_t)buf * GT * M;
      if (vec)
        for (int i = tid; i < nt * M / 4; i += blockDim.x) cp_async16(dst + 4 * i, src + 4 * i);
      else
        for (int i = tid; i < nt * M; i += blockDim.x) cp_async4(dst + i, src + i);
    }
    cp_async_commit();  // an empty group past the end keeps the group count uniform
  };
  float gr[NM], num[NM], den[NM];
#pragma unroll
  for (int n = 0; n < NM; ++n) {
    gr[n] = (active && n < N) ? g[((size_t)f * N + n) * M + m] : 0.f;
    num[n] = 0.f;
    den[n] = 0.f;
  }
#pragma unroll
  for (int c = 0; c < NST - 1; ++c) issue(c);
  for (int c = 0; c < nchunk; ++c) {
    issue(c + NST - 1);
    cp_async_wait<NST - 1>();
    __syncthreads();
    const int nt = min(GT, T - c * GT), buf = c % NST;
    const float* lb = ls + buf * N * GT;
    const float* pb = ps + (size_t)buf * GT * M;
    if (active) {
      for (int tt = s; tt < nt; tt += S) {
        float l[NM];
        float ys = 0.f;
#pragma unroll
        for (int n = 0; n < NM; ++n) {
          l[n] = (NM <= 8 || n < N) ? lb[n * GT + tt] : 0.f;
          ys = fmaf(l[n], gr[n], ys);
        }
        const float w = fast_rcp(fmaxf(ys, eps));
        const float u = pb[tt * M + m] * w * w;
#pragma unroll
        for (int n = 0; n < NM; ++n) {
          num[n] = fmaf(l[n], u, num[n]);
          den[n] = fmaf(l[n], w, den[n]);
        }
      }
    }
    __syncthreads();
  }
  if (active)
#pragma unroll
    for (int n = 0; n < NM; ++n)
      if (n < N) {
        red[(s * M + m) * 2 * N + 2 * n] = num[n];
        red[(s * M + m) * 2 * N + 2 * n + 1] = den[n];
      }
  __syncthreads();
  for (int i = tid; i < N * M; i += blockDim.x) {
    const int n = i / M, mm = i % M;
    float a = 0.f, d = 0.f;
    for (int q = 0; q < S; ++q) {
      a += red[(q * M + mm) * 2 * N + 2 * n];
      d += red[(q * M + mm) * 2 * N + 2 * n + 1];
    }
    const size_t gi = ((size_t)f * N + n) * M + mm;
    if (grad) {  // gradient of Eq. (12): sum_t lambda (1/yhat - P/yhat^2)
      grad[gi] = d - a;
      continue;
    }
    const float gnew = g[gi] * sqrtf(a / fmaxf(d, eps));
    if (!finitef(gnew)) atomicOr(flags + FLAG_NONFINITE, 1u);
    g[gi] = gnew;
  }
}

// Quad variant (M = 4, 8, 16, 32 or 64, N <= 8; 128 threads): thread (slot s,
// quad q) owns microphones 4q .. 4q+3, so a frame's lambda values serve four
// microphones per load and P arrives as one 16-byte read; the slots of a warp
// are added by xor shuffles and the warps through shared memory, in a fixed
// order.
template <int NM, int NST>
__global__ void __launch_bounds__(128) k_gupd4(const float* __restrict__ lam, const float* __restrict__ P,
                                               float* __restrict__ g, int F, int T, int Tp, int M, int N, float eps,
                                               unsigned* __restrict__ flags, float* __restrict__ grad) {
  extern __shared__ __align__(16) float smq[];
  const int f = blockIdx.x, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int Q = M / 4, S = 128 / Q;  // quads per frame, frame slots (128 threads)
  const int q = tid % Q, s = tid / Q;
  float* ls = smq;                          // [NST][N][GT]
  float* ps = ls + NST * NM * GT;           // [NST][GT][M]
  float* red = ps + NST * GT * M;           // [4 warps][M][2N]
  const int nchunk = (T + GT - 1) / GT;
  auto issue = [&](int c) {
    if (c < nchunk) {
      const int t0 = c * GT, nt = min(GT, T - t0), buf = c % NST;
      const int nq = (nt + 3) / 4, qq = tid & 31;
      if (qq < nq)
        for (int n = tid >> 5; n < NM; n += 4)
          cp_async16(ls + (buf * NM + n) * GT + 4 * qq, lam + ((size_t)n * F + f) * Tp + t0 + 4 * qq);
      const float* src = P + ((size_t)f * T + t0) * M;
      float* dst = ps + (size_t)buf * GT * M;
      for (int i = tid; i < nt * M / 4; i += 128) cp_async16(dst + 4 * i, src + 4 * i);
    }
    cp_async_commit();
  };
  float gr[NM][4], num[NM][4], den[NM][4];
#pragma unroll
  for (int n = 0; n < NM; ++n)
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      gr[n][j] = g[((size_t)f * NM + n) * M + 4 * q + j];
      num[n][j] = 0.f;
      den[n][j] = 0.f;
    }
#pragma unroll
  for (int c = 0; c < NST - 1; ++c) issue(c);
  for (int c = 0; c < nchunk; ++c) {
    issue(c + NST - 1);
    cp_async_wait<NST - 1>();
    __syncthreads();
    const int nt = min(GT, T - c * GT), buf = c % NST;
    const float* lb = ls + buf * NM * GT;
    const float* pb = ps + (size_t)buf * GT * M;
    for (int tt = s; tt < nt; tt += S) {
      float l[NM];
#pragma unroll
      for (int n = 0; n < NM; ++n) l[n] = lb[n * GT + tt];
      const float4 p4 = *reinterpret_cast<const float4*>(pb + tt * M + 4 * q);
      const float pv[4] = {p4.x, p4.y, p4.z, p4.w};
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        float ys = 0.f;
#pragma unroll
        for (int n = 0; n < NM; ++n) ys = fmaf(l[n], gr[n][j], ys);
        const float w = fast_rcp(fmaxf(ys, eps));
        const float u = pv[j] * w * w;
#pragma unroll
        for (int n = 0; n < NM; ++n) {
          num[n][j] = fmaf(l[n], u, num[n][j]);
          den[n][j] = fmaf(l[n], w, den[n][j]);
        }
      }
    }
    __syncthreads();
  }
  // slots of the warp (lanes differing in the bits above the quad index), then the warps
#pragma unroll
  for (int o = 16; o >= 1; o >>= 1)
    if (o >= Q)
#pragma unroll
      for (int n = 0; n < NM; ++n)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          num[n][j] += __shfl_xor_sync(DFM_FULL_MASK, num[n][j], o);
          den[n][j] += __shfl_xor_sync(DFM_FULL_MASK, den[n][j], o);
        }
  if (lane < Q)
#pragma unroll
    for (int n = 0; n < NM; ++n)
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        red[(warp * M + 4 * q + j) * 2 * NM + 2 * n] = num[n][j];
        red[(warp * M + 4 * q + j) * 2 * NM + 2 * n + 1] = den[n][j];
      }
  __syncthreads();
  for (int i = tid; i < NM * M; i += 128) {
    const int n = i / M, mm = i % M;
    float a = 0.f, d = 0.f;
    for (int w = 0; w < 4; ++w) {
      a += red[(w * M + mm) * 2 * NM + 2 * n];
      d += red[(w * M + mm) * 2 * NM + 2 * n + 1];
    }
    const size_t gi = ((size_t)f * NM + n) * M + mm;
    if (grad) {  // gradient of Eq. (12)
      grad[gi] = d - a;
      continue;
    }
    const float gnew = g[gi] * sqrtf(a / fmaxf(d, eps));
    if (!finitef(gnew)) atomicOr(flags + FLAG_NONFINITE, 1u);
    g[gi] = gnew;
  }
}

// ----------------------------------------------------------------- launchers

template <int K, int MK, bool COMPUTE_P, bool COMP>
static cudaError_t launch_pstats_ft(const dfmnmf_ctx* c, cudaStream_t s, int fb, int fc) {
  // one frame per thread where P is formed here; two for the statistics alone, whose loads of both frames
  // the unrolled loop issues together
  const int tpc = COMPUTE_P ? 128 : 256;
  dim3 grid(fc, (c->T + tpc - 1) / tpc);
  const size_t sm = ((size_t)((c->N * c->M + 3) & ~3) + (COMPUTE_P ? 4 * (size_t)K * MK * MK : 0)) * sizeof(float);
  auto kern = k_pstats_ft<K, MK, COMPUTE_P, COMP>;
  if (sm > 48 * 1024) cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  kern<<<grid, 128, sm, s>>>(c->x, c->Q64, c->lam, c->g, c->P, c->A, c->D, c->F, c->T, c->Tp, c->N, c->eps, fb, tpc);
  return cudaGetLastError();
}

template <bool COMPUTE_P, bool COMP>
static cudaError_t launch_pstats_impl(const dfmnmf_ctx* c, cudaStream_t s, int fb, int fc) {
  if (COMPUTE_P && pstats_tma_supported(c->K, c->MK, c->N)) return launch_pstats_tma(c, s, fb, fc, COMP);
  if (c->MK == 4 && c->K == 4) return launch_pstats_ft<4, 4, COMPUTE_P, COMP>(c, s, fb, fc);
  if (c->MK == 4 && c->K == 2) return launch_pstats_ft<2, 4, COMPUTE_P, COMP>(c, s, fb, fc);
  if (c->MK == 4 && c->K == 1) return launch_pstats_ft<1, 4, COMPUTE_P, COMP>(c, s, fb, fc);
  if (c->MK == 4 && c->K == 3) return launch_pstats_ft<3, 4, COMPUTE_P, COMP>(c, s, fb, fc);
  if (c->MK == 16 && c->K == 1) return launch_pstats_ft<1, 16, COMPUTE_P, COMP>(c, s, fb, fc);
  if (c->MK == 32 && c->K == 1) return launch_pstats_ft<1, 32, COMPUTE_P, COMP>(c, s, fb, fc);
  if (c->MK == 4 && c->K == 8) return launch_pstats_ft<8, 4, COMPUTE_P, COMP>(c, s, fb, fc);
  const int TB = 256 / c->K;
  dim3 grid(fc, (c->T + TB - 1) / TB);
  const bool pow2 = (c->K & (c->K - 1)) == 0;
  const size_t sm = (size_t)((c->N * c->M + 3) & ~3) * sizeof(float) +
                    (COMPUTE_P ? 4 * (size_t)c->K * c->MK * c->MK * sizeof(float) : 0) +
                    (pow2 ? 0 : (size_t)TB * c->K * 2 * sizeof(float));
  DFM_MK_DISPATCH(c->MK, {
    auto kern = k_pstats<MK_, COMPUTE_P, COMP>;
    if (sm > 48 * 1024) cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    kern<<<grid, 256, sm, s>>>(c->x, c->Q64, c->lam, c->g, c->P, c->A, c->D, c->F, c->T, c->Tp, c->K, c->N, c->eps,
                               fb);
  });
  return cudaGetLastError();
}

cudaError_t launch_power_stats(const dfmnmf_ctx* c, cudaStream_t s, int fb, int fc) {
  return c->precision == DFMNMF_FP32 ? launch_pstats_impl<true, true>(c, s, fb, fc)
                                     : launch_pstats_impl<true, false>(c, s, fb, fc);
}

cudaError_t launch_power_stats_comp(const dfmnmf_ctx* c, cudaStream_t s) {
  return launch_pstats_impl<true, true>(c, s, 0, c->F);
}

cudaError_t launch_stats(const dfmnmf_ctx* c, cudaStream_t s) { return launch_pstats_impl<false, false>(c, s, 0, c->F); }


// Four stages while they fit in 64 KB of shared memory (several CTAs per SM),
// else two.
template <int NM>
static cudaError_t launch_gupd4(const dfmnmf_ctx* c, cudaStream_t s, float* grad) {
  const int M = c->M;
  const size_t stage = (size_t)(NM * GT + GT * M) * sizeof(float);
  const size_t red = (size_t)4 * M * 2 * NM * sizeof(float);
  const bool deep = 4 * stage + red <= 64 * 1024;
  const size_t sm = (deep ? 4 : 2) * stage + red;
  auto k4 = deep ? k_gupd4<NM, 4> : k_gupd4<NM, 2>;
  if (sm > 48 * 1024) cudaFuncSetAttribute(k4, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  k4<<<c->F, 128, sm, s>>>(c->lam, c->P, c->g, c->F, c->T, c->Tp, M, c->N, c->eps, c->flags, grad);
  return cudaGetLastError();
}

cudaError_t launch_gupd(const dfmnmf_ctx* c, cudaStream_t s, float* grad) {
  const int M = c->M, N = c->N;
  if (M >= 4 && M <= 64 && (M & (M - 1)) == 0 && N <= 8) {  // quads per frame a power of two (warp shuffles)
    switch (N) {
      case 1: return launch_gupd4<1>(c, s, grad);
      case 2: return launch_gupd4<2>(c, s, grad);
      case 3: return launch_gupd4<3>(c, s, grad);
      case 4: return launch_gupd4<4>(c, s, grad);
      case 5: return launch_gupd4<5>(c, s, grad);
      case 6: return launch_gupd4<6>(c, s, grad);
      case 7: return launch_gupd4<7>(c, s, grad);
      default: return launch_gupd4<8>(c, s, grad);
    }
  }
  const int S = 256 / M;
  const size_t stage = (size_t)(N * GT + GT * M) * sizeof(float);
  const size_t red = (size_t)S * M * 2 * N * sizeof(float);
  const bool deep = 4 * stage + red <= 64 * 1024;
  const size_t sm = (deep ? 4 : 2) * stage + red;
#define DFM_GUPD_K(NMV, NSTV)                                                                                    \
  {                                                                                                              \
    if (sm > 48 * 1024)                                                                                          \
      cudaFuncSetAttribute(k_gupd<NMV, NSTV>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);             \
    k_gupd<NMV, NSTV><<<c->F, 256, sm, s>>>(c->lam, c->P, c->g, c->F, c->T, c->Tp, M, N, c->eps, c->flags, grad); \
  }
#define DFM_GUPD(NMV)           \
  if (deep) DFM_GUPD_K(NMV, 4)  \
  else DFM_GUPD_K(NMV, 2)
  switch (N) {
    case 1: DFM_GUPD(1) break;
    case 2: DFM_GUPD(2) break;
    case 3: DFM_GUPD(3) break;
    case 4: DFM_GUPD(4) break;
    case 5: DFM_GUPD(5) break;
    case 6: DFM_GUPD(6) break;
    case 7: DFM_GUPD(7) break;
    case 8: DFM_GUPD(8) break;
    default: DFM_GUPD(16) break;
  }
#undef DFM_GUPD
#undef DFM_GUPD_K
  return cudaGetLastError();
}

}  // namespace dfm
