// kernels_nmf.cu -- the NMF multiplicative updates as register-tiled products.
//
// With the MU statistics A[n][f][t] = sum_m g P yhat^-2 and
// D[n][f][t] = sum_m g yhat^-1 already formed (k_pstats), Eqs. (8) and (9)
// are plain products per source n:
//   Eq. (8)  num_W[f][b] = sum_t A[f][t] H[b][t]   (F x T)(T x B)
//   Eq. (9)  num_H[b][t] = sum_f W[f][b] A[f][t]   (B x F)(F x T)
// (same with D for the denominators), followed by the square-root ratio.  The
// refresh of the model lambda = W H that the paper asks for after every rule
// is the separate tiled k_lambda launch: done here, by the CTA that finishes
// a tile, it serialised an O(F) (Eq. 9) or register-heavy (Eq. 8) tail
// behind the split reduction.
#include "common.cuh"
#include "internal.h"

namespace dfm {

constexpr int TILE = 16;  // f (Eq. 8) or t (Eq. 9) per CTA, and b per CTA
constexpr int NWARP = 8;
constexpr int KCH = 64;   // reduction chunk staged in shared memory
constexpr int NMF_MAX_SPLIT = 8;
constexpr int RS = 17;    // row stride of the cross-warp reduction array (odd: no bank conflicts)

// Split-reduction epilogue shared by k_wupd / k_hupd.  Thread tid holds the
// CTA's partial (num, den) of one output.  With S > 1 the partial is written
// to part[tile][split][tid], and the CTA that takes the last ticket of the
// tile returns true with the S partials summed in split order; the others
// return false.  The ticket is reset for the next launch.
__device__ __forceinline__ bool split_fixup(float& num, float& den, int S, int split, int tile,
                                            float* __restrict__ part, unsigned* __restrict__ ticket) {
  if (S == 1) return true;
  __shared__ unsigned last;
  float2* p = reinterpret_cast<float2*>(part) + ((size_t)tile * S) * 256;
  p[(size_t)split * 256 + threadIdx.x] = make_float2(num, den);
  __syncthreads();  // the CTA's partials are written ...
  if (threadIdx.x == 0) {
    __threadfence();  // ... and released at device scope before the ticket is taken
    last = (atomicAdd(ticket + tile, 1u) == (unsigned)(S - 1));
    if (last) __threadfence();  // acquire the other CTAs' partials
  }
  __syncthreads();
  if (!last) return false;
  num = 0.f;
  den = 0.f;
  for (int q = 0; q < S; ++q) {
    const float2 v = __ldcg(p + (size_t)q * 256 + threadIdx.x);
    num += v.x;
    den += v.y;
  }
  if (threadIdx.x == 0) ticket[tile] = 0u;
  return true;
}

// ------------------------------------------------------------------ Eq. (8)
// grid (ceil(F/16), N, ceil(B/16) * S); the S CTAs of a tile split the frames
// (chunks of 64), 8 warps split each chunk; lane = (f pair, b quad).  A, D
// and H tiles are read one chunk ahead into registers as float4 rows (the
// padded row stride Tp is a multiple of 4) and stored transposed ([t][f],
// [t][b]) after the current chunk is consumed.  Every CTA writes its partial
// sums; the last CTA of a tile (counted with an atomic ticket) adds the S
// partials in a fixed order and updates W.  Nothing waits
// on another CTA.
__global__ void __launch_bounds__(256) k_wupd(const float* __restrict__ A, const float* __restrict__ D,
                                              const float* __restrict__ H, float* __restrict__ W,
                                              int F, int T, int Tp, int B, float eps,
                                              unsigned* __restrict__ flags, int S, int cps,
                                              float* __restrict__ part, unsigned* __restrict__ ticket,
                                              float* __restrict__ grad) {
  constexpr int TS = 20;  // padded row of the transposed tiles: conflict-free stores, 16-byte rows
  constexpr int STAGE = 3 * KCH * TS;
  __shared__ __align__(16) float stg[STAGE];
  __shared__ float red[NWARP * 32 * RS];
  const int nb = (B + TILE - 1) / TILE;
  const int bt = blockIdx.z % nb, split = blockIdx.z / nb;
  const int f0 = blockIdx.x * TILE, n = blockIdx.y, b0 = bt * TILE;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int fp = lane >> 2, bq = lane & 3;
  const float* An = A + (size_t)n * F * Tp;
  const float* Dn = D + (size_t)n * F * Tp;
  const float* Hn = H + (size_t)n * B * Tp;
  float* As = stg;
  float* Ds = As + KCH * TS;
  float* Hs = Ds + KCH * TS;
  const int r = tid % TILE, q = tid / TILE;  // row of the tile, float4 column of the chunk
  const float4 z4 = make_float4(0.f, 0.f, 0.f, 0.f);
  auto fetch = [&](int c, float4& a4, float4& d4, float4& h4) {
    const int t = c * KCH + 4 * q;
    const int f = f0 + r, b = b0 + r;
    const bool tin = t < Tp;
    a4 = (tin && f < F) ? __ldg(reinterpret_cast<const float4*>(An + (size_t)f * Tp + t)) : z4;
    d4 = (tin && f < F) ? __ldg(reinterpret_cast<const float4*>(Dn + (size_t)f * Tp + t)) : z4;
    h4 = (tin && b < B) ? __ldg(reinterpret_cast<const float4*>(Hn + (size_t)b * Tp + t)) : z4;
  };
  auto store = [&](const float4& a4, const float4& d4, const float4& h4) {
    const float av[4] = {a4.x, a4.y, a4.z, a4.w}, dv[4] = {d4.x, d4.y, d4.z, d4.w}, hv[4] = {h4.x, h4.y, h4.z, h4.w};
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      As[(4 * q + j) * TS + r] = av[j];
      Ds[(4 * q + j) * TS + r] = dv[j];
      Hs[(4 * q + j) * TS + r] = hv[j];
    }
  };
  float acc[16];
#pragma unroll
  for (int i = 0; i < 16; ++i) acc[i] = 0.f;
  const int c0 = split * cps, c1 = min((T + KCH - 1) / KCH, c0 + cps);
  float4 pa, pd, ph;
  if (c0 < c1) fetch(c0, pa, pd, ph);
  for (int c = c0; c < c1; ++c) {
    store(pa, pd, ph);
    __syncthreads();
    if (c + 1 < c1) fetch(c + 1, pa, pd, ph);
#pragma unroll
    for (int s = 0; s < KCH / NWARP; ++s) {
      const int tt = warp * (KCH / NWARP) + s;
      const float2 a2 = *reinterpret_cast<const float2*>(As + tt * TS + 2 * fp);
      const float2 d2 = *reinterpret_cast<const float2*>(Ds + tt * TS + 2 * fp);
      const float4 h4 = *reinterpret_cast<const float4*>(Hs + tt * TS + 4 * bq);
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
  for (int i = 0; i < 16; ++i) red[(warp * 32 + lane) * RS + i] = acc[i];
  __syncthreads();
  {
    const int fi = tid / TILE, bi = tid % TILE;  // 256 threads = 16 x 16 outputs
    const int l = (fi >> 1) * 4 + (bi >> 2);
    const int slot = ((fi & 1) * 4 + (bi & 3)) * 2;
    float num = 0.f, den = 0.f;
#pragma unroll
    for (int w = 0; w < NWARP; ++w) {
      num += red[(w * 32 + l) * RS + slot + 0];
      den += red[(w * 32 + l) * RS + slot + 1];
    }
    if (!split_fixup(num, den, S, split, (n * gridDim.x + blockIdx.x) * nb + bt, part, ticket)) return;
    const int f = f0 + fi, b = b0 + bi;
    if (grad) {  // gradient of Eq. (12): sum_t H (D - A)
      if (f < F && b < B) grad[((size_t)n * F + f) * B + b] = den - num;
    } else if (f < F && b < B) {
      float* wp = W + ((size_t)n * F + f) * B + b;
      const float wn = *wp * sqrtf(num / fmaxf(den, eps));
      if (!finitef(wn)) atomicOr(flags + FLAG_NONFINITE, 1u);
      *wp = wn;
    }
  }
}

// ------------------------------------------- Eq. (8) with the Eq. (2) refresh
// One CTA per (source n, WL_F = 10 consecutive frequencies): 52 x 5 CTAs on
// the paper's 513 bins, two per SM, one wave.  H[n] ([B][Tp]) and the CTA's
// A and D rows ([10][Tp] each) are staged in shared memory by 16-byte
// cp.async (all contiguous; the row stride Tp is a multiple of 4).  Warp w
// takes frequency pair w % 5 and the 128-frame blocks k = w / 5 (mod 2);
// each lane owns four consecutive frames of a block (16-byte shared-memory
// reads of A, D and H), accumulates num[b] = sum_t A H[b] and
// den[b] = sum_t D H[b] for 16 bases of both frequencies, one reduce-scatter
// gives lane l the warp totals of frequency l / 16, basis l % 16, the second
// warp's totals are added to the first's through shared memory (fixed
// order), and that lane updates the W entry.  Then warp w refreshes
// lambda[n][f][t] = sum_b W[n][f][b] H[n][b][t] (Eq. 2) for frequency w of
// the CTA, four frames per lane, in the basis order of k_lambda (bit for bit
// the same refresh).  No partial sums leave the CTA, no second launch.  More
// than 16 bases are taken 16 at a time.
constexpr int WL_F = 10;
constexpr int WL_PAIRS = WL_F / 2;
constexpr int WL_THREADS = 2 * WL_PAIRS * 32;

size_t wlam_smem_bytes(const dfmnmf_ctx* c) {
  const int Bq = (c->B + 15) & ~15;
  return ((size_t)c->B * c->Tp + 2 * (size_t)WL_F * c->Tp + WL_PAIRS * 32 * 2 + (size_t)WL_F * Bq) * sizeof(float);
}

__global__ void __launch_bounds__(WL_THREADS, 2) k_wlam(const float* __restrict__ A, const float* __restrict__ D,
                                                        const float* __restrict__ H, float* __restrict__ W,
                                                        float* __restrict__ lam, int F, int T, int Tp, int B,
                                                        float eps, unsigned* __restrict__ flags) {
  extern __shared__ __align__(16) float smw[];
  const int Bq = (B + 15) & ~15;
  float* Hs = smw;                          // [B][Tp]
  float* As = Hs + (size_t)B * Tp;          // [WL_F][Tp]
  float* Ds = As + (size_t)WL_F * Tp;       // [WL_F][Tp]
  float* red = Ds + (size_t)WL_F * Tp;      // [WL_PAIRS][32 lanes][2]: the second warp's totals
  float* wrow = red + WL_PAIRS * 32 * 2;    // [WL_F][Bq]: the new W rows
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int n = blockIdx.y, f0 = blockIdx.x * WL_F, nf = min(WL_F, F - f0);
  {
    const float* srcH = H + (size_t)n * B * Tp;
    const float* srcA = A + ((size_t)n * F + f0) * Tp;
    const float* srcD = D + ((size_t)n * F + f0) * Tp;
    const int nh = B * Tp / 4, na = nf * Tp / 4;
    for (int i = tid; i < nh; i += WL_THREADS) cp_async16(Hs + 4 * i, srcH + 4 * i);
    for (int i = tid; i < na; i += WL_THREADS) {
      cp_async16(As + 4 * i, srcA + 4 * i);
      cp_async16(Ds + 4 * i, srcD + 4 * i);
    }
    cp_async_commit();
    cp_async_wait<0>();
  }
  __syncthreads();
  const int p = warp % WL_PAIRS, second = warp / WL_PAIRS;
  const int fa = 2 * p, fb = 2 * p + 1;
  const bool vb = fb < nf;
  const float* Aa = As + (size_t)fa * Tp;
  const float* Da = Ds + (size_t)fa * Tp;
  const float* Ab = As + (size_t)(vb ? fb : fa) * Tp;
  const float* Db = Ds + (size_t)(vb ? fb : fa) * Tp;
  const bool va = fa < nf;
  for (int b0 = 0; b0 < B; b0 += 16) {
    float acc[64];  // entry 2 (fi 16 + j) + {0: num, 1: den}
#pragma unroll
    for (int i = 0; i < 64; ++i) acc[i] = 0.f;
    if (va) {
      for (int t = 128 * second + 4 * lane; t < T; t += 256) {
        // frames t .. t+3; A and D beyond T are read as zero, H is zero there
        float4 a0 = *reinterpret_cast<const float4*>(Aa + t), d0 = *reinterpret_cast<const float4*>(Da + t);
        float4 a1 = *reinterpret_cast<const float4*>(Ab + t), d1 = *reinterpret_cast<const float4*>(Db + t);
        if (t + 3 >= T) {
          const float4 z = make_float4(0.f, 0.f, 0.f, 0.f);
          if (t + 1 >= T) { a0.y = z.y; d0.y = z.y; a1.y = z.y; d1.y = z.y; }
          if (t + 2 >= T) { a0.z = z.z; d0.z = z.z; a1.z = z.z; d1.z = z.z; }
          a0.w = z.w; d0.w = z.w; a1.w = z.w; d1.w = z.w;
        }
#pragma unroll
        for (int j = 0; j < 16; ++j) {
          const float4 h = (b0 + j < B) ? *reinterpret_cast<const float4*>(Hs + (size_t)(b0 + j) * Tp + t)
                                        : make_float4(0.f, 0.f, 0.f, 0.f);
          acc[2 * j] = fmaf(a0.x, h.x, fmaf(a0.y, h.y, fmaf(a0.z, h.z, fmaf(a0.w, h.w, acc[2 * j]))));
          acc[2 * j + 1] = fmaf(d0.x, h.x, fmaf(d0.y, h.y, fmaf(d0.z, h.z, fmaf(d0.w, h.w, acc[2 * j + 1]))));
          acc[32 + 2 * j] = fmaf(a1.x, h.x, fmaf(a1.y, h.y, fmaf(a1.z, h.z, fmaf(a1.w, h.w, acc[32 + 2 * j]))));
          acc[33 + 2 * j] = fmaf(d1.x, h.x, fmaf(d1.y, h.y, fmaf(d1.z, h.z, fmaf(d1.w, h.w, acc[33 + 2 * j]))));
        }
      }
    }
    warp_reduce_scatter<64>(acc, lane);
    if (second) {
      red[(p * 32 + lane) * 2] = acc[0];
      red[(p * 32 + lane) * 2 + 1] = acc[1];
    }
    __syncthreads();
    if (!second) {
      const float num = acc[0] + red[(p * 32 + lane) * 2];
      const float den = acc[1] + red[(p * 32 + lane) * 2 + 1];
      const int fl = (lane >> 4) ? fb : fa, b = b0 + (lane & 15);
      if (fl < nf && b < B) {
        float* wp = W + ((size_t)n * F + f0 + fl) * B + b;
        const float wn = *wp * sqrtf(num / fmaxf(den, eps));
        if (!finitef(wn)) atomicOr(flags + FLAG_NONFINITE, 1u);
        *wp = wn;
        wrow[fl * Bq + b] = wn;
      }
    }
    __syncthreads();  // wrow complete; red free for the next 16 bases
  }
  // warp w: frequency w of the CTA, four consecutive frames per lane (H is zero on T .. Tp-1, so is lambda)
  for (int fl = warp; fl < nf; fl += WL_THREADS / 32) {
    float* L = lam + ((size_t)n * F + f0 + fl) * Tp;
    const float* wr = wrow + fl * Bq;
    for (int t = 4 * lane; t < Tp; t += 128) {
      float4 l = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll 4
      for (int b = 0; b < B; ++b) {
        const float w = wr[b];
        const float4 h = *reinterpret_cast<const float4*>(Hs + (size_t)b * Tp + t);
        l.x = fmaf(w, h.x, l.x);
        l.y = fmaf(w, h.y, l.y);
        l.z = fmaf(w, h.z, l.z);
        l.w = fmaf(w, h.w, l.w);
      }
      *reinterpret_cast<float4*>(L + t) = l;
    }
  }
}
bool wlam_supported(const dfmnmf_ctx* c) {
  return c->smem_optin > 0 && wlam_smem_bytes(c) <= (size_t)c->smem_optin;
}

cudaError_t launch_wlam(const dfmnmf_ctx* c, cudaStream_t s) {
  const size_t sm = wlam_smem_bytes(c);
  cudaFuncSetAttribute(k_wlam, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  dim3 grid((c->F + WL_F - 1) / WL_F, c->N);
  k_wlam<<<grid, WL_THREADS, sm, s>>>(c->A, c->D, c->H, c->W, c->lam, c->F, c->T, c->Tp, c->B, c->eps, c->flags);
  return cudaGetLastError();
}

// ------------------------------------------------------------------ Eq. (9)
// grid (ceil(T/16), N, ceil(B/16) * S); the S CTAs of a tile split the
// frequencies (chunks of 64) and finish as in k_wupd; lane = (t pair, b quad).
// A, D (row stride Tp) and W (rows of B) tiles arrive by 16-byte cp.async in
// their natural [f][t] / [f][b] layouts, double-buffered.
__global__ void __launch_bounds__(256) k_hupd(const float* __restrict__ A, const float* __restrict__ D,
                                              const float* __restrict__ W, float* __restrict__ H,
                                              int F, int T, int Tp, int B, float eps,
                                              unsigned* __restrict__ flags, int S, int cps,
                                              float* __restrict__ part, unsigned* __restrict__ ticket,
                                              float* __restrict__ grad) {
  constexpr int STAGE = 3 * KCH * TILE;
  __shared__ __align__(16) float stg[2 * STAGE];
  __shared__ float red[NWARP * 32 * RS];
  const int nb = (B + TILE - 1) / TILE;
  const int bt = blockIdx.z % nb, split = blockIdx.z / nb;
  const int t0 = blockIdx.x * TILE, n = blockIdx.y, b0 = bt * TILE;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int tp = lane >> 2, bq = lane & 3;
  const float* An = A + (size_t)n * F * Tp;
  const float* Dn = D + (size_t)n * F * Tp;
  const float* Wg = W + (size_t)n * F * B;
  const bool wvec = (B % 4) == 0;
  auto issue = [&](int ch) {
    float* As = stg + (ch & 1) * STAGE;
    float* Ds = As + KCH * TILE;
    float* Ws = Ds + KCH * TILE;
    const int fc = ch * KCH;
    const int fi = tid / 4, q = tid % 4;  // 64 rows x 4 float4
    const int f = fc + fi, t = t0 + 4 * q, b = b0 + 4 * q;
    if (f < F && t < Tp) {
      cp_async16(As + fi * TILE + 4 * q, An + (size_t)f * Tp + t);
      cp_async16(Ds + fi * TILE + 4 * q, Dn + (size_t)f * Tp + t);
    } else {
      *reinterpret_cast<float4*>(As + fi * TILE + 4 * q) = make_float4(0.f, 0.f, 0.f, 0.f);
      *reinterpret_cast<float4*>(Ds + fi * TILE + 4 * q) = make_float4(0.f, 0.f, 0.f, 0.f);
    }
    if (wvec && f < F && b + 3 < B) {
      cp_async16(Ws + fi * TILE + 4 * q, Wg + (size_t)f * B + b);
    } else {
#pragma unroll
      for (int j = 0; j < 4; ++j)
        Ws[fi * TILE + 4 * q + j] = (f < F && b + j < B) ? Wg[(size_t)f * B + b + j] : 0.f;
    }
    cp_async_commit();
  };
  float acc[16];
#pragma unroll
  for (int i = 0; i < 16; ++i) acc[i] = 0.f;
  const int c0 = split * cps, c1 = min((F + KCH - 1) / KCH, c0 + cps);
  if (c0 < c1) issue(c0);
  for (int ch = c0; ch < c1; ++ch) {
    if (ch + 1 < c1) {
      issue(ch + 1);
      cp_async_wait<1>();
    } else {
      cp_async_wait<0>();
    }
    __syncthreads();
    const float* As = stg + (ch & 1) * STAGE;
    const float* Ds = As + KCH * TILE;
    const float* Ws = Ds + KCH * TILE;
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
  for (int i = 0; i < 16; ++i) red[(warp * 32 + lane) * RS + i] = acc[i];
  __syncthreads();
  {
    const int bi = tid / TILE, ti = tid % TILE;
    const int l = (ti >> 1) * 4 + (bi >> 2);
    const int slot = ((ti & 1) * 4 + (bi & 3)) * 2;
    float num = 0.f, den = 0.f;
#pragma unroll
    for (int w = 0; w < NWARP; ++w) {
      num += red[(w * 32 + l) * RS + slot + 0];
      den += red[(w * 32 + l) * RS + slot + 1];
    }
    if (!split_fixup(num, den, S, split, (n * gridDim.x + blockIdx.x) * nb + bt, part, ticket)) return;
    const int b = b0 + bi, t = t0 + ti;
    if (grad) {  // gradient of Eq. (12): sum_f W (D - A)
      if (b < B && t < T) grad[((size_t)n * B + b) * Tp + t] = den - num;
    } else if (b < B && t < T) {
      float* hp = H + ((size_t)n * B + b) * Tp + t;
      const float hn = *hp * sqrtf(num / fmaxf(den, eps));
      if (!finitef(hn)) atomicOr(flags + FLAG_NONFINITE, 1u);
      *hp = hn;
    }
  }
}

// Number of splits of the reduction: enough CTAs for cfg_nmf_ctas per SM
// (4 unless tuned), at most NMF_MAX_SPLIT, never more than the number of
// 64-wide chunks.
static void split_plan(const dfmnmf_ctx* c, int tiles, int nch, int* S, int* cps) {
  const int target = (c->cfg_nmf_ctas > 0 ? c->cfg_nmf_ctas : 4) * (c->num_sms > 0 ? c->num_sms : 152);
  int s = (target + tiles - 1) / tiles;
  s = s < 1 ? 1 : (s > NMF_MAX_SPLIT ? NMF_MAX_SPLIT : s);
  s = s > nch ? nch : s;
  *cps = (nch + s - 1) / s;
  *S = (nch + *cps - 1) / *cps;
}

size_t nmf_scratch_floats(const dfmnmf_ctx* c) {
  const int nb = (c->B + TILE - 1) / TILE;
  const size_t tw = (size_t)c->N * ((c->F + TILE - 1) / TILE) * nb;
  const size_t th = (size_t)c->N * ((c->T + TILE - 1) / TILE) * nb;
  return (tw > th ? tw : th) * NMF_MAX_SPLIT * 512;
}
size_t nmf_ticket_count(const dfmnmf_ctx* c) { return nmf_scratch_floats(c) / (NMF_MAX_SPLIT * 512); }

cudaError_t launch_wupd(const dfmnmf_ctx* c, cudaStream_t s, float* grad) {
  const int nb = (c->B + TILE - 1) / TILE;
  const int tiles = ((c->F + TILE - 1) / TILE) * c->N * nb;
  int S, cps;
  split_plan(c, tiles, (c->T + KCH - 1) / KCH, &S, &cps);
  dim3 grid((c->F + TILE - 1) / TILE, c->N, nb * S);
  k_wupd<<<grid, 256, 0, s>>>(c->A, c->D, c->H, c->W, c->F, c->T, c->Tp, c->B, c->eps, c->flags, S, cps,
                              c->nmf_part, c->nmf_ticket, grad);
  return cudaGetLastError();
}

cudaError_t launch_hupd(const dfmnmf_ctx* c, cudaStream_t s, float* grad) {
  const int nb = (c->B + TILE - 1) / TILE;
  const int tiles = ((c->T + TILE - 1) / TILE) * c->N * nb;
  int S, cps;
  split_plan(c, tiles, (c->F + KCH - 1) / KCH, &S, &cps);
  dim3 grid((c->T + TILE - 1) / TILE, c->N, nb * S);
  k_hupd<<<grid, 256, 0, s>>>(c->A, c->D, c->W, c->H, c->F, c->T, c->Tp, c->B, c->eps, c->flags, S, cps,
                              c->nmf_part, c->nmf_ticket, grad);
  return cudaGetLastError();
}

}  // namespace dfm
