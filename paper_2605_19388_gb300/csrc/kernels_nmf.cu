// kernels_nmf.cu -- the NMF multiplicative updates as register-tiled products.
//
// With the MU statistics A[n][f][t] = sum_m g P yhat^-2 and
// D[n][f][t] = sum_m g yhat^-1 already formed (k_pstats), Eqs. (8) and (9)
// are plain products per source n:
//   Eq. (8)  num_W[f][b] = sum_t A[f][t] H[b][t]   (F x T)(T x B)
//   Eq. (9)  num_H[b][t] = sum_f W[f][b] A[f][t]   (B x F)(F x T)
// (same with D for the denominators), followed by the square-root ratio.  The
// updated factor is then multiplied back into lambda = W H for the rows (or
// columns) the CTA owns, so the refresh of the model that the paper asks for
// after every rule costs no extra pass over W or H.
#include "common.cuh"
#include "internal.h"

namespace dfm {

constexpr int TILE = 16;  // f (Eq. 8) or t (Eq. 9) per CTA, and b per CTA
constexpr int NWARP = 8;
constexpr int KCH = 64;   // reduction chunk staged in shared memory

// ------------------------------------------------------------------ Eq. (8)
// grid (ceil(F/16), N, ceil(B/16)); 8 warps split T; lane = (f pair, b quad).
__global__ void __launch_bounds__(256) k_wupd(const float* __restrict__ A, const float* __restrict__ D,
                                              const float* __restrict__ H, float* __restrict__ W,
                                              float* __restrict__ lam, int F, int T, int B, float eps,
                                              int refresh, unsigned* __restrict__ flags) {
  constexpr int AS = 18;  // padded row (floats) of the [t][f] staging tiles: 8-byte aligned pairs
  constexpr int HS = 20;  // padded row of the [t][b] tile: 16-byte aligned quads
  __shared__ __align__(16) float As[KCH * AS];
  __shared__ __align__(16) float Ds[KCH * AS];
  __shared__ __align__(16) float Hs[KCH * HS];
  __shared__ float red[NWARP * 32 * 16];
  __shared__ float Wn[TILE * TILE];
  const int f0 = blockIdx.x * TILE, n = blockIdx.y, b0 = blockIdx.z * TILE;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int fp = lane >> 2, bq = lane & 3;
  const float* An = A + (size_t)n * F * T;
  const float* Dn = D + (size_t)n * F * T;
  const float* Hn = H + (size_t)n * B * T;
  float acc[16];
#pragma unroll
  for (int i = 0; i < 16; ++i) acc[i] = 0.f;
  for (int t0 = 0; t0 < T; t0 += KCH) {
    for (int idx = tid; idx < TILE * KCH; idx += 256) {
      const int tt = idx % KCH, r = idx / KCH;
      const int t = t0 + tt;
      const int f = f0 + r, b = b0 + r;
      As[tt * AS + r] = (t < T && f < F) ? An[(size_t)f * T + t] : 0.f;
      Ds[tt * AS + r] = (t < T && f < F) ? Dn[(size_t)f * T + t] : 0.f;
      Hs[tt * HS + r] = (t < T && b < B) ? Hn[(size_t)b * T + t] : 0.f;
    }
    __syncthreads();
#pragma unroll
    for (int s = 0; s < KCH / NWARP; ++s) {
      const int tt = warp * (KCH / NWARP) + s;
      const float2 a2 = *reinterpret_cast<const float2*>(As + tt * AS + 2 * fp);
      const float2 d2 = *reinterpret_cast<const float2*>(Ds + tt * AS + 2 * fp);
      const float4 h4 = *reinterpret_cast<const float4*>(Hs + tt * HS + 4 * bq);
      const float av[2] = {a2.x, a2.y}, dv[2] = {d2.x, d2.y}, hv[4] = {h4.x, h4.y, h4.z, h4.w};
#pragma unroll
      for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          acc[(i * 4 + j) * 2 + 0] = fmaf(av[i], hv[j], acc[(i * 4 + j) * 2 + 0]);
          acc[(i * 4 + j) * 2 + 1] = fmaf(dv[i], hv[j], acc[(i * 4 + j) * 2 + 1]);
        }
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 16; ++i) red[(warp * 32 + lane) * 16 + i] = acc[i];
  __syncthreads();
  {
    const int fi = tid / TILE, bi = tid % TILE;  // 256 threads = 16 x 16 outputs
    const int l = (fi >> 1) * 4 + (bi >> 2);
    const int slot = ((fi & 1) * 4 + (bi & 3)) * 2;
    float num = 0.f, den = 0.f;
#pragma unroll
    for (int w = 0; w < NWARP; ++w) {
      num += red[(w * 32 + l) * 16 + slot + 0];
      den += red[(w * 32 + l) * 16 + slot + 1];
    }
    const int f = f0 + fi, b = b0 + bi;
    float wn = 0.f;
    if (f < F && b < B) {
      float* wp = W + ((size_t)n * F + f) * B + b;
      wn = *wp * sqrtf(num / fmaxf(den, eps));
      if (!finitef(wn)) atomicOr(flags + FLAG_NONFINITE, 1u);
      *wp = wn;
    }
    Wn[fi * TILE + bi] = wn;
  }
  if (!refresh) return;
  __syncthreads();
  // lambda[n][f][t] = sum_b Wn[f][b] H[b][t] for the 16 rows of this CTA (B <= 16 here)
  for (int t = tid; t < T; t += 256) {
    float hv[TILE];
#pragma unroll
    for (int b = 0; b < TILE; ++b) hv[b] = (b < B) ? __ldg(Hn + (size_t)b * T + t) : 0.f;
#pragma unroll 4
    for (int fi = 0; fi < TILE; ++fi) {
      const int f = f0 + fi;
      if (f >= F) break;
      float s = 0.f;
#pragma unroll
      for (int b = 0; b < TILE; ++b) s = fmaf(Wn[fi * TILE + b], hv[b], s);
      lam[((size_t)n * F + f) * T + t] = s;
    }
  }
}

// ------------------------------------------------------------------ Eq. (9)
// grid (ceil(T/16), N, ceil(B/16)); 8 warps split F; lane = (t pair, b quad).
__global__ void __launch_bounds__(256) k_hupd(const float* __restrict__ A, const float* __restrict__ D,
                                              const float* __restrict__ W, float* __restrict__ H,
                                              float* __restrict__ lam, int F, int T, int B, float eps,
                                              int refresh, unsigned* __restrict__ flags) {
  __shared__ __align__(16) float As[KCH * TILE];
  __shared__ __align__(16) float Ds[KCH * TILE];
  __shared__ __align__(16) float Ws[KCH * TILE];
  __shared__ float red[NWARP * 32 * 16];
  __shared__ float Hn_s[TILE * TILE];  // [b][t]
  const int t0 = blockIdx.x * TILE, n = blockIdx.y, b0 = blockIdx.z * TILE;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int tp = lane >> 2, bq = lane & 3;
  const float* An = A + (size_t)n * F * T;
  const float* Dn = D + (size_t)n * F * T;
  const float* Wg = W + (size_t)n * F * B;
  float acc[16];
#pragma unroll
  for (int i = 0; i < 16; ++i) acc[i] = 0.f;
  for (int fc = 0; fc < F; fc += KCH) {
    for (int idx = tid; idx < KCH * TILE; idx += 256) {
      const int c = idx % TILE, fi = idx / TILE;
      const int f = fc + fi, t = t0 + c, b = b0 + c;
      As[fi * TILE + c] = (f < F && t < T) ? An[(size_t)f * T + t] : 0.f;
      Ds[fi * TILE + c] = (f < F && t < T) ? Dn[(size_t)f * T + t] : 0.f;
      Ws[fi * TILE + c] = (f < F && b < B) ? Wg[(size_t)f * B + b] : 0.f;
    }
    __syncthreads();
#pragma unroll
    for (int s = 0; s < KCH / NWARP; ++s) {
      const int fi = warp * (KCH / NWARP) + s;
      const float2 a2 = *reinterpret_cast<const float2*>(As + fi * TILE + 2 * tp);
      const float2 d2 = *reinterpret_cast<const float2*>(Ds + fi * TILE + 2 * tp);
      const float4 w4 = *reinterpret_cast<const float4*>(Ws + fi * TILE + 4 * bq);
      const float av[2] = {a2.x, a2.y}, dv[2] = {d2.x, d2.y}, wv[4] = {w4.x, w4.y, w4.z, w4.w};
#pragma unroll
      for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          acc[(i * 4 + j) * 2 + 0] = fmaf(wv[j], av[i], acc[(i * 4 + j) * 2 + 0]);
          acc[(i * 4 + j) * 2 + 1] = fmaf(wv[j], dv[i], acc[(i * 4 + j) * 2 + 1]);
        }
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 16; ++i) red[(warp * 32 + lane) * 16 + i] = acc[i];
  __syncthreads();
  {
    const int bi = tid / TILE, ti = tid % TILE;
    const int l = (ti >> 1) * 4 + (bi >> 2);
    const int slot = ((ti & 1) * 4 + (bi & 3)) * 2;
    float num = 0.f, den = 0.f;
#pragma unroll
    for (int w = 0; w < NWARP; ++w) {
      num += red[(w * 32 + l) * 16 + slot + 0];
      den += red[(w * 32 + l) * 16 + slot + 1];
    }
    const int b = b0 + bi, t = t0 + ti;
    float hn = 0.f;
    if (b < B && t < T) {
      float* hp = H + ((size_t)n * B + b) * T + t;
      hn = *hp * sqrtf(num / fmaxf(den, eps));
      if (!finitef(hn)) atomicOr(flags + FLAG_NONFINITE, 1u);
      *hp = hn;
    }
    Hn_s[bi * TILE + ti] = hn;
  }
  if (!refresh) return;
  __syncthreads();
  // lambda[n][f][t0..t0+16) = sum_b W[n][f][b] Hn[b][t] for every f (B <= 16 here)
  const int ti = tid % TILE, fl = tid / TILE;
  const int t = t0 + ti;
  float hcol[TILE];
#pragma unroll
  for (int b = 0; b < TILE; ++b) hcol[b] = Hn_s[b * TILE + ti];
  for (int f = fl; f < F; f += 256 / TILE) {
    const float* wr = Wg + (size_t)f * B;
    float s = 0.f;
#pragma unroll
    for (int b = 0; b < TILE; ++b)
      if (b < B) s = fmaf(__ldg(wr + b), hcol[b], s);
    if (t < T) lam[((size_t)n * F + f) * T + t] = s;
  }
}

bool nmf_fused_lambda(const dfmnmf_ctx* c) { return c->B <= TILE; }

cudaError_t launch_wupd(const dfmnmf_ctx* c, cudaStream_t s) {
  const int nb = (c->B + TILE - 1) / TILE;
  dim3 grid((c->F + TILE - 1) / TILE, c->N, nb);
  k_wupd<<<grid, 256, 0, s>>>(c->A, c->D, c->H, c->W, c->lam, c->F, c->T, c->B, c->eps, nb == 1, c->flags);
  return cudaGetLastError();
}

cudaError_t launch_hupd(const dfmnmf_ctx* c, cudaStream_t s) {
  const int nb = (c->B + TILE - 1) / TILE;
  dim3 grid((c->T + TILE - 1) / TILE, c->N, nb);
  k_hupd<<<grid, 256, 0, s>>>(c->A, c->D, c->W, c->H, c->lam, c->F, c->T, c->B, c->eps, nb == 1, c->flags);
  return cudaGetLastError();
}

}  // namespace dfm
