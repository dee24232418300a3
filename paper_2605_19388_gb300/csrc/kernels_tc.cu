// kernels_tc.cu -- tensor-core form of the weighted covariances (Eq. 13).
//
//   V[f][k][mu][a][b] = (1/T) sum_t R[f][k][a,b](t) * w[f][t][k,mu],
//   R = x_ftk x_ftk^H packed as M_k^2 = 16 reals, w = 1/yhat.
//
// For every frequency this is an (16 K x T) by (T x 4 K) product.  The
// operands are split into two bfloat16 parts, R = R_hi + R_lo and
// w = w_hi + w_lo, and three products R_hi w_hi + R_hi w_lo + R_lo w_hi are
// accumulated in FP32 (the dropped R_lo w_lo term is below 2^-16 relative).
// A plain bfloat16 contraction loses too much: on the paper-sized workload
// it moves the IP update by 6e-2 relative, the split form by 1.5e-4.
//
// R depends only on the observation, so it is formed once (k_rprep) into
// two bfloat16 arrays; the weights change every iteration: k_wprep forms
// w_hi / w_lo from lambda and g in one streaming pass.  Both are stored in
// the order k_vtc reads them: a tile of FPC = 8 / K frequencies (128 rows of
// R, 32 rows of w) is cut into chunks of 64 frames, and each (tile, chunk)
// block of 128 x 64 (R) or 32 x 64 (w) values is contiguous in memory
// ([tiles][Tr / 64][rows][64], Tr = T rounded up to 64, zero tail), so every
// tensor copy reads one contiguous 16 KB or 4 KB block instead of 128-byte
// pieces of rows 2 Tr bytes apart.  k_vtc then only moves and multiplies:
// one thread streams the four operand tiles of each 64-frame chunk with TMA
// (128-byte swizzled, with an evict-first L2 policy: R and w are read once
// per iteration, and R, 84 MB on the paper-sized workload, would otherwise
// push the streaming kernels' operands out of L2) into a
// 2-stage shared-memory ring (two CTAs per SM), one thread issues
// tcgen05.mma (M = 128 rows = 128 / (16 K) frequencies, N = 32 weights,
// K = 16 frames per instruction, FP32 accumulators in tensor memory) and the
// four warps read the accumulators back with tcgen05.ld.  (Forming w inside
// k_vtc, by warps beside the TMA and MMA threads, left the tensor pipe
// waiting on them for most of every chunk.)
//
// Supported layouts: M_k = 4 and K in {1, 2, 4, 8} (M = 128 / (16 K) * 16 K
// rows per tile, N = 32 columns).  Every mbarrier wait is bounded; a wait
// that gives up sets FLAG_TIMEOUT and the CTA skips the rest of its work.
#include <cuda.h>
#include <cuda_bf16.h>

#include "../../include/dfmnmf.h"
#include "common.cuh"
#include "internal.h"

namespace dfm {

constexpr int TC_KC = 64;       // frames per chunk (128 bytes of bfloat16 per row)
constexpr int TC_ROWS = 128;    // MMA M
constexpr int TC_COLS = 32;     // MMA N
constexpr int TC_STAGES = 2;
constexpr int TC_A_BYTES = TC_ROWS * TC_KC * 2;   // 16 KB per operand part
constexpr int TC_B_BYTES = TC_COLS * TC_KC * 2;   // 4 KB per operand part
constexpr int TC_STAGE_BYTES = 2 * TC_A_BYTES + 2 * TC_B_BYTES;
constexpr unsigned long long TC_WAIT_CYCLES = 2000000000ull;  // ~1 s at 2 GHz

// ------------------------------------------------------------ PTX helpers
__device__ __forceinline__ unsigned smem_u32(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(unsigned long long* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_arrive(unsigned long long* bar) {
  asm volatile("{\n .reg .b64 st;\n mbarrier.arrive.shared::cta.b64 st, [%0];\n}" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(unsigned long long* bar, unsigned bytes) {
  asm volatile("{\n .reg .b64 st;\n mbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1;\n}" ::"r"(smem_u32(bar)),
               "r"(bytes)
               : "memory");
}
// Wait for the phase with the given parity to complete; false on timeout.
__device__ __forceinline__ bool mbar_wait(unsigned long long* bar, unsigned parity) {
  const unsigned addr = smem_u32(bar);
  const unsigned long long start = clock64();
  while (true) {
    unsigned ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
        : "=r"(ok)
        : "r"(addr), "r"(parity)
        : "memory");
    if (ok) return true;
    if (clock64() - start > TC_WAIT_CYCLES) return false;
  }
}

__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, int c0, int c1,
                                            unsigned long long* bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
          smem_u32(dst)),
      "l"(reinterpret_cast<unsigned long long>(map)), "r"(c0), "r"(c1), "r"(smem_u32(bar))
      : "memory");
}
// The same copy with an L2 cache policy (createpolicy).
__device__ __forceinline__ void tma_load_2d_hint(void* dst, const CUtensorMap* map, int c0, int c1,
                                                 unsigned long long* bar, unsigned long long policy) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint [%0], [%1, {%2, "
      "%3}], [%4], %5;" ::"r"(smem_u32(dst)),
      "l"(reinterpret_cast<unsigned long long>(map)), "r"(c0), "r"(c1), "r"(smem_u32(bar)), "l"(policy)
      : "memory");
}
__device__ __forceinline__ unsigned long long l2_evict_first_policy() {
  unsigned long long p;
  asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
  return p;
}

// Position of element (row, t) of a tensor-core operand in the tiled layout:
// rows of tile `tile` (rows_per_tile of them), chunk t / 64 of nch, frame t % 64.
__host__ __device__ __forceinline__ size_t tc_index(int tile, int row, int t, int nch, int rows_per_tile) {
  return (((size_t)tile * nch + (t >> 6)) * rows_per_tile + row) * TC_KC + (t & (TC_KC - 1));
}

// Shared-memory matrix descriptor: K-major operand tile with 128-byte
// swizzle, 8-row groups 1024 bytes apart (stride byte offset), descriptor
// version 1, base offset 0.
__device__ __forceinline__ unsigned long long smem_desc_sw128(unsigned addr) {
  unsigned long long d = 0;
  d |= (unsigned long long)((addr >> 4) & 0x3FFF);
  d |= (unsigned long long)(1) << 16;              // leading byte offset (unused by swizzled K-major)
  d |= (unsigned long long)((1024 >> 4) & 0x3FFF) << 32;
  d |= 1ull << 46;                                 // version
  d |= 2ull << 61;                                 // 128-byte swizzle
  return d;
}

// Instruction descriptor, kind::f16: D FP32, A and B bfloat16, both K-major,
// N = 32, M = 128.
constexpr unsigned TC_IDESC = (1u << 4) | (1u << 7) | (1u << 10) | ((TC_COLS >> 3) << 17) | ((TC_ROWS >> 4) << 24);

__device__ __forceinline__ void umma_bf16(unsigned tmem_d, unsigned long long a, unsigned long long b, unsigned acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(
          tmem_d),
      "l"(a), "l"(b), "r"(TC_IDESC), "r"(acc)
      : "memory");
}
__device__ __forceinline__ void umma_commit(unsigned long long* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}

// ------------------------------------------------------------- R prepare
// Packed entry r of block k of frequency f at frame t, for t < Tr (zero beyond
// T), in the tiled layout: row (f % FPC) * 16K + 16 k + r of tile f / FPC.
__global__ void __launch_bounds__(128) k_rprep(const float2* __restrict__ x, __nv_bfloat16* __restrict__ Rhi,
                                               __nv_bfloat16* __restrict__ Rlo, int F, int T, int Tr, int K) {
  const int f = blockIdx.y;
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= Tr) return;
  const int M = K * 4;
  const int FPC = TC_ROWS / (16 * K), nch = Tr / TC_KC;
  const int tile = f / FPC, frow = (f % FPC) * 16 * K;
  for (int k = 0; k < K; ++k) {
    float R[16];
    if (t < T) {
      float2 xv[4];
      load_block<4>(x + ((size_t)f * T + t) * M + k * 4, xv);
#pragma unroll
      for (int a = 0; a < 4; ++a) {
        R[a * 4 + a] = fmaf(xv[a].x, xv[a].x, xv[a].y * xv[a].y);
#pragma unroll
        for (int b = a + 1; b < 4; ++b) {
          R[a * 4 + b] = fmaf(xv[a].x, xv[b].x, xv[a].y * xv[b].y);
          R[b * 4 + a] = fmaf(xv[a].y, xv[b].x, -xv[a].x * xv[b].y);
        }
      }
    } else {
#pragma unroll
      for (int r = 0; r < 16; ++r) R[r] = 0.f;
    }
#pragma unroll
    for (int r = 0; r < 16; ++r) {
      const __nv_bfloat16 h = __float2bfloat16_rn(R[r]);
      const __nv_bfloat16 l = __float2bfloat16_rn(R[r] - __bfloat162float(h));
      const size_t o = tc_index(tile, frow + k * 16 + r, t, nch, TC_ROWS);
      Rhi[o] = h;
      Rlo[o] = l;
    }
  }
}

// ------------------------------------------------------------- weights
// w = 1 / max(yhat, eps), yhat[f][t][m] = sum_n lambda[n][f][t] g[f][n][m]
// (Eq. 2 with the floor of Sec. IV-A), split into two bfloat16 parts and
// stored as rows (f % FPC) * M + m of tile f / FPC, Tr frames, zero beyond T:
// the B operand of the contraction, read by TMA in the same 128-byte swizzled
// tiles as R.  Each thread forms two adjacent frames of one frequency for
// every microphone (float2 lambda loads, g[f] from shared memory four
// microphones per load, 4-byte stores coalesced along t; row m + 1 of a tile
// block sits 64 frames after row m).  NM is N itself for N <= 8 and 16
// (guarded) above; MV is M (4, 8, 16 or 32).
template <int NM, int MV>
__global__ void __launch_bounds__(128) k_wprep(const float* __restrict__ lam, const float* __restrict__ g,
                                               __nv_bfloat16* __restrict__ whi, __nv_bfloat16* __restrict__ wlo,
                                               int F, int T, int Tp, int Tr, int N, float eps, int fb) {
  extern __shared__ __align__(16) float gw[];  // [N][MV]
  const int f = fb + blockIdx.y;
  for (int i = threadIdx.x; i < N * MV; i += blockDim.x) gw[i] = g[(size_t)f * N * MV + i];
  __syncthreads();
  const int t = 2 * (blockIdx.x * blockDim.x + threadIdx.x);
  if (t >= Tr) return;
  constexpr int FPC = TC_COLS / MV;
  const int nch = Tr / TC_KC;
  const int tile = f / FPC, frow = (f % FPC) * MV;
  float2 lv[NM];
#pragma unroll
  for (int n = 0; n < NM; ++n) {
    lv[n] = make_float2(0.f, 0.f);
    if ((NM <= 8 || n < N) && t < Tp) lv[n] = *reinterpret_cast<const float2*>(lam + ((size_t)n * F + f) * Tp + t);
  }
  const bool v0 = t < T, v1 = t + 1 < T;
  const size_t o0 = tc_index(tile, frow, t, nch, TC_COLS);
  __nv_bfloat162* ph = reinterpret_cast<__nv_bfloat162*>(whi + o0);
  __nv_bfloat162* pl = reinterpret_cast<__nv_bfloat162*>(wlo + o0);
#pragma unroll
  for (int m4 = 0; m4 < MV; m4 += 4) {
    float2 y[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) y[j] = make_float2(0.f, 0.f);
#pragma unroll
    for (int n = 0; n < NM; ++n)
      if (NM <= 8 || n < N) {
        const float4 gv4 = *reinterpret_cast<const float4*>(gw + n * MV + m4);
        const float gv[4] = {gv4.x, gv4.y, gv4.z, gv4.w};
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          y[j].x = fmaf(lv[n].x, gv[j], y[j].x);
          y[j].y = fmaf(lv[n].y, gv[j], y[j].y);
        }
      }
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const float w0 = v0 ? fast_rcp(fmaxf(y[j].x, eps)) : 0.f;
      const float w1 = v1 ? fast_rcp(fmaxf(y[j].y, eps)) : 0.f;
      const __nv_bfloat162 h = __floats2bfloat162_rn(w0, w1);
      const float2 hf = __bfloat1622float2(h);
      const __nv_bfloat162 l = __floats2bfloat162_rn(w0 - hf.x, w1 - hf.y);
      ph[(m4 + j) * (TC_KC / 2)] = h;
      pl[(m4 + j) * (TC_KC / 2)] = l;
    }
  }
}

// ------------------------------------------------------------ contraction
struct TcSmem {
  unsigned long long full[TC_STAGES];
  unsigned long long empty[TC_STAGES];
  unsigned long long done;
  unsigned tmem_base;
  unsigned abort;
};

__host__ __device__ constexpr size_t tc_ring_bytes() { return (size_t)TC_STAGES * TC_STAGE_BYTES; }

// One CTA per tile of TC_ROWS / (16 K) frequencies, four warps: lane 0 of
// warp 0 streams the four operand tiles of every 64-frame chunk (R_hi, R_lo,
// w_hi, w_lo) into the shared-memory ring, lane 0 of warp 1 issues the three
// split products per 16 frames, and all four warps read the accumulators back.
__global__ void __launch_bounds__(128, 2) k_vtc(const __grid_constant__ CUtensorMap map_rhi,
                                                const __grid_constant__ CUtensorMap map_rlo,
                                                const __grid_constant__ CUtensorMap map_whi,
                                                const __grid_constant__ CUtensorMap map_wlo,
                                                double2* __restrict__ V, float4* __restrict__ Vdd, int T, int Tr,
                                                int K, unsigned* __restrict__ flags, int fb, int fe) {
  extern __shared__ __align__(1024) unsigned char tc_raw[];
  unsigned char* ring = reinterpret_cast<unsigned char*>(((unsigned long long)tc_raw + 1023) & ~1023ull);
  TcSmem* ctl = reinterpret_cast<TcSmem*>(ring + tc_ring_bytes());
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int FPC = TC_ROWS / (16 * K);    // frequencies per CTA
  const int f0 = fb + blockIdx.x * FPC;  // frequencies f0 .. min(f0 + FPC, fe) - 1 are this CTA's
  const int M = 4 * K;
  const int nch = Tr / TC_KC;

  if (tid == 0) {
    for (int s = 0; s < TC_STAGES; ++s) {
      mbar_init(&ctl->full[s], 1);
      mbar_init(&ctl->empty[s], 1);
    }
    mbar_init(&ctl->done, 1);
    ctl->abort = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 32;" ::"r"(smem_u32(&ctl->tmem_base))
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  }
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const unsigned tmem = ctl->tmem_base;

  if (warp == 0 && lane == 0) {
    // ---- TMA producer: block (tile, chunk) of R and of w, one contiguous copy each
    const unsigned long long evict_first = l2_evict_first_policy();
    const int tile = f0 / FPC;
    for (int c = 0; c < nch; ++c) {
      const int s = c % TC_STAGES;
      if (c >= TC_STAGES && !mbar_wait(&ctl->empty[s], ((c / TC_STAGES) + 1) & 1)) {
        atomicOr(&ctl->abort, 1u);
        break;
      }
      if (ctl->abort) break;
      unsigned char* st = ring + s * TC_STAGE_BYTES;
      mbar_arrive_expect_tx(&ctl->full[s], TC_STAGE_BYTES);
      const int blk = tile * nch + c;
      tma_load_2d_hint(st, &map_rhi, 0, blk * TC_ROWS, &ctl->full[s], evict_first);
      tma_load_2d_hint(st + TC_A_BYTES, &map_rlo, 0, blk * TC_ROWS, &ctl->full[s], evict_first);
      tma_load_2d_hint(st + 2 * TC_A_BYTES, &map_whi, 0, blk * TC_COLS, &ctl->full[s], evict_first);
      tma_load_2d_hint(st + 2 * TC_A_BYTES + TC_B_BYTES, &map_wlo, 0, blk * TC_COLS, &ctl->full[s], evict_first);
    }
  } else if (warp == 1 && lane == 0) {
    // ---- MMA issuer
    for (int c = 0; c < nch; ++c) {
      const int s = c % TC_STAGES;
      if (!mbar_wait(&ctl->full[s], (c / TC_STAGES) & 1)) {
        atomicOr(&ctl->abort, 1u);
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const unsigned base = smem_u32(ring + s * TC_STAGE_BYTES);
      const unsigned a_hi = base, a_lo = base + TC_A_BYTES;
      const unsigned b_hi = base + 2 * TC_A_BYTES, b_lo = b_hi + TC_B_BYTES;
#pragma unroll
      for (int kk = 0; kk < TC_KC / 16; ++kk) {
        const unsigned off = kk * 32;  // 16 bfloat16 along K inside the 128-byte swizzle atom
        umma_bf16(tmem, smem_desc_sw128(a_hi + off), smem_desc_sw128(b_hi + off), (c > 0 || kk > 0) ? 1u : 0u);
        umma_bf16(tmem, smem_desc_sw128(a_hi + off), smem_desc_sw128(b_lo + off), 1u);
        umma_bf16(tmem, smem_desc_sw128(a_lo + off), smem_desc_sw128(b_hi + off), 1u);
      }
      umma_commit(&ctl->empty[s]);
    }
    umma_commit(&ctl->done);
  }

  // ---- epilogue: the four warps read the accumulators (lane = row)
  __syncwarp();
  const bool ok = mbar_wait(&ctl->done, 0);
  if (!ok) atomicOr(&ctl->abort, 1u);
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  unsigned r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
      "%15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]),
        "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
        "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(tmem + ((unsigned)(warp * 32) << 16)));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
  {
    const int row = tid;                      // 0..127
    const int fj = row / (16 * K), rk = row % (16 * K);
    const int k = rk / 16, e = rk % 16;       // packed entry e = a * 4 + b
    const int f = f0 + fj;
    if (ok && !ctl->abort && f < fe) {
      const int a = e / 4, b = e % 4;
      const double invT = 1.0 / (double)T;
      const size_t blk = (size_t)f * K + k;
#pragma unroll
      for (int mu = 0; mu < 4; ++mu) {
        const float v = __uint_as_float(r[fj * M + k * 4 + mu]);
        const double dv = (double)v * invT;
        double2* Vb = V + (blk * 4 + mu) * 16;
        float4* Vd = Vdd + (blk * 4 + mu) * 16;
        double* vdbl = reinterpret_cast<double*>(Vb);
        float* vflt = reinterpret_cast<float*>(Vd);
        const float fv = (float)dv;
        if (a == b) {
          Vb[a * 4 + a] = make_double2(dv, 0.0);
          Vd[a * 4 + a] = make_float4(fv, 0.f, 0.f, 0.f);
        } else if (a < b) {  // real part of V[a][b] and V[b][a]
          vdbl[2 * (a * 4 + b)] = dv;
          vdbl[2 * (b * 4 + a)] = dv;
          vflt[4 * (a * 4 + b)] = fv; vflt[4 * (a * 4 + b) + 1] = 0.f;
          vflt[4 * (b * 4 + a)] = fv; vflt[4 * (b * 4 + a) + 1] = 0.f;
        } else {  // e = a*4+b with a > b holds Im(x_b conj x_a) = Im V[b][a]
          vdbl[2 * (b * 4 + a) + 1] = dv;
          vdbl[2 * (a * 4 + b) + 1] = -dv;
          vflt[4 * (b * 4 + a) + 2] = fv; vflt[4 * (b * 4 + a) + 3] = 0.f;
          vflt[4 * (a * 4 + b) + 2] = -fv; vflt[4 * (a * 4 + b) + 3] = 0.f;
        }
      }
    }
  }
  __syncthreads();
  if (ctl->abort && tid == 0) atomicOr(flags + FLAG_TIMEOUT, 1u);
  if (warp == 0) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 32;" ::"r"(tmem) : "memory");
  }
}

// ------------------------------------------------- projections and MU statistics through TMA
// P = |Q x|^2 and the MU statistics A = sum_m g P / yhat^2, D = sum_m g / yhat
// for 4 subarrays of 4 microphones, one CTA per (frequency, 128 frames).
// Thread 0 brings the x tile (128 frames x 16 complex, 16 KB, 128-byte
// swizzle) and the lambda rows of every source (N x 512 B) into shared memory
// with two tensor copies on one mbarrier; every thread reads its frame's row
// with the swizzle undone (16-byte chunk c of row i sits at chunk c ^ (i % 8),
// so the eight rows of a quarter-warp hit eight different bank groups); P is
// staged in shared memory with a 64-byte swizzle (chunk c of row i at
// c ^ ((i / 2) % 4)) and written back by one tensor store, which clips the
// frames past T; A and D are stored directly (consecutive frames per warp).
constexpr int PT_ROWS = 128;
constexpr int PT_X_BYTES = PT_ROWS * 128;  // 16 complex64 per frame
constexpr int PT_P_BYTES = PT_ROWS * 64;   // 16 float per frame

__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* map, int c0, int c1, int c2,
                                            unsigned long long* bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], "
      "[%5];" ::"r"(smem_u32(dst)),
      "l"(reinterpret_cast<unsigned long long>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(smem_u32(bar))
      : "memory");
}
__device__ __forceinline__ void tma_store_3d(const CUtensorMap* map, int c0, int c1, int c2, const void* src) {
  asm volatile("cp.async.bulk.tensor.3d.global.shared::cta.bulk_group [%0, {%1, %2, %3}], [%4];" ::"l"(
                   reinterpret_cast<unsigned long long>(map)),
               "r"(c0), "r"(c1), "r"(c2), "r"(smem_u32(src))
               : "memory");
}

template <bool COMP>
__global__ void __launch_bounds__(128) k_pstats_tma(const __grid_constant__ CUtensorMap map_x,
                                                    const __grid_constant__ CUtensorMap map_l,
                                                    const __grid_constant__ CUtensorMap map_p,
                                                    const double2* __restrict__ Q64,
                                                    const float2* __restrict__ Q32, const float* __restrict__ g,
                                                    float* __restrict__ A, float* __restrict__ D, int F, int T,
                                                    int Tp, int N, float eps, int fb, unsigned* __restrict__ flags) {
  constexpr int K = 4, MK = 4, M = 16;
  extern __shared__ __align__(16) unsigned char pt_raw[];
  unsigned char* base = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(pt_raw) + 1023) & ~uintptr_t(1023));
  unsigned char* xs = base;                                    // [128][128 B], 128-byte swizzle
  unsigned char* ps = base + PT_X_BYTES;                       // [128][64 B], 64-byte swizzle
  float* ls = reinterpret_cast<float*>(ps + PT_P_BYTES);       // [N][128]
  float* gs = ls + N * PT_ROWS;                                // [N][M]
  float2* Qh = reinterpret_cast<float2*>(gs + ((N * M + 3) & ~3));  // [K][MK][MK]
  float2* Ql = Qh + K * MK * MK;
  unsigned long long* bar = reinterpret_cast<unsigned long long*>(Ql + K * MK * MK);
  const int f = fb + blockIdx.x, tid = threadIdx.x, t0 = blockIdx.y * PT_ROWS;
  if (tid == 0) {
    mbar_init(bar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    mbar_arrive_expect_tx(bar, (unsigned)(PT_X_BYTES + N * PT_ROWS * 4));
    tma_load_3d(xs, &map_x, 0, t0, f, bar);
    tma_load_3d(ls, &map_l, t0, f, 0, bar);
  }
  for (int i = tid; i < N * M; i += blockDim.x) gs[i] = g[(size_t)f * N * M + i];
  // plain projections take the single-precision copy of Q (the rounded FP64
  // master, written beside it), compensated ones split the master in two floats
  for (int i = tid; i < K * MK * MK; i += blockDim.x) {
    if (COMP) split_c(Q64[(size_t)f * K * MK * MK + i], Qh[i], Ql[i]);
    else Qh[i] = Q32[(size_t)f * K * MK * MK + i];
  }
  __syncthreads();
  if (!mbar_wait(bar, 0)) {  // the copies did not arrive within the budget: report, skip the tile
    if (tid == 0) atomicOr(flags + FLAG_TIMEOUT, 1u);
    return;
  }
  const int i = tid, t = t0 + i;
  float pv[M];
#pragma unroll
  for (int k = 0; k < K; ++k) {
    float2 xv[MK];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int c = 2 * k + h;
      const float4 q = *reinterpret_cast<const float4*>(xs + i * 128 + ((c ^ (i & 7)) << 4));
      xv[2 * h] = make_float2(q.x, q.y);
      xv[2 * h + 1] = make_float2(q.z, q.w);
    }
#pragma unroll
    for (int mu = 0; mu < MK; ++mu) {
      const float2* qh = Qh + (k * MK + mu) * MK;
      float2 y;
      if (COMP) {
        y = cdot2<MK>(qh, Ql + (k * MK + mu) * MK, xv);
      } else {
        // the row of Q as two 16-byte shared-memory loads (rows are 32 bytes, 16-byte aligned)
        const float4 q01 = reinterpret_cast<const float4*>(qh)[0], q23 = reinterpret_cast<const float4*>(qh)[1];
        const float2 qv[4] = {make_float2(q01.x, q01.y), make_float2(q01.z, q01.w), make_float2(q23.x, q23.y),
                              make_float2(q23.z, q23.w)};
        float yr = 0.f, yi = 0.f;
#pragma unroll
        for (int nu = 0; nu < MK; ++nu) {
          yr = fmaf(qv[nu].x, xv[nu].x, fmaf(-qv[nu].y, xv[nu].y, yr));
          yi = fmaf(qv[nu].x, xv[nu].y, fmaf(qv[nu].y, xv[nu].x, yi));
        }
        y = make_float2(yr, yi);
      }
      pv[k * MK + mu] = fmaf(y.x, y.x, y.y * y.y);
    }
  }
#pragma unroll
  for (int c = 0; c < 4; ++c)
    *reinterpret_cast<float4*>(ps + i * 64 + ((c ^ ((i >> 1) & 3)) << 4)) =
        make_float4(pv[4 * c], pv[4 * c + 1], pv[4 * c + 2], pv[4 * c + 3]);
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  __syncthreads();
  if (tid == 0) {
    tma_store_3d(&map_p, 0, t0, f, ps);
    asm volatile("cp.async.bulk.commit_group;" ::: "memory");
  }
  float ys[M];
#pragma unroll
  for (int m = 0; m < M; ++m) ys[m] = 0.f;
  for (int n = 0; n < N; ++n) {
    const float l = ls[n * PT_ROWS + i];
    const float4* gr4 = reinterpret_cast<const float4*>(gs + n * M);  // 16-byte aligned: M = 16
#pragma unroll
    for (int m4 = 0; m4 < M / 4; ++m4) {
      const float4 gv = gr4[m4];
      ys[4 * m4] = fmaf(l, gv.x, ys[4 * m4]);
      ys[4 * m4 + 1] = fmaf(l, gv.y, ys[4 * m4 + 1]);
      ys[4 * m4 + 2] = fmaf(l, gv.z, ys[4 * m4 + 2]);
      ys[4 * m4 + 3] = fmaf(l, gv.w, ys[4 * m4 + 3]);
    }
  }
  float w[M], u[M];
#pragma unroll
  for (int m = 0; m < M; ++m) {
    w[m] = fast_rcp(fmaxf(ys[m], eps));
    u[m] = pv[m] * w[m] * w[m];
  }
  if (t < T)
    for (int n = 0; n < N; ++n) {
      const float4* gr4 = reinterpret_cast<const float4*>(gs + n * M);
      float a = 0.f, d = 0.f;
#pragma unroll
      for (int m4 = 0; m4 < M / 4; ++m4) {
        const float4 gv4 = gr4[m4];
        const float gv[4] = {gv4.x, gv4.y, gv4.z, gv4.w};
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          a = fmaf(gv[j], u[4 * m4 + j], a);
          d = fmaf(gv[j], w[4 * m4 + j], d);
        }
      }
      const size_t o = ((size_t)n * F + f) * Tp + t;
      A[o] = a;
      D[o] = d;
    }
  if (tid == 0) asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");  // ps is read before the CTA exits
}

bool pstats_tma_supported(int K, int MK, int N) { return K == 4 && MK == 4 && N >= 1 && N <= 16; }

static size_t pstats_tma_smem(int N) {
  return 1024 + PT_X_BYTES + PT_P_BYTES + (size_t)N * PT_ROWS * 4 + (size_t)((N * 16 + 3) & ~3) * 4 +
         2 * 4 * 16 * sizeof(float2) + 16;
}

// ------------------------------------------------------------- host side
typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

static EncodeTiledFn encode_fn() {
  static EncodeTiledFn fn = nullptr;
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiledFn>(p);
  }
  return fn;
}

bool tc_supported(int MK, int K) { return MK == 4 && (K == 1 || K == 2 || K == 4 || K == 8); }

size_t tc_smem_bytes(const dfmnmf_ctx*) { return 1024 + tc_ring_bytes() + sizeof(TcSmem); }

// Tiles of FPC = 8 / K frequencies of the tiled operand layout (the last one
// padded with zero rows), and the elements of R (each part) and w (each part).
int tc_tiles(const dfmnmf_ctx* c) {
  const int FPC = TC_ROWS / (16 * c->K);
  return (c->F + FPC - 1) / FPC;
}
void tc_operand_elems(const dfmnmf_ctx* c, size_t* nr, size_t* nw) {
  *nr = (size_t)tc_tiles(c) * TC_ROWS * c->Tr;
  *nw = (size_t)tc_tiles(c) * TC_COLS * c->Tr;
}

// Four 2-D bfloat16 maps with 128-byte swizzle over the tiled layout viewed as
// rows of 64 frames: R_hi / R_lo (boxes of 128 rows, one (tile, chunk) block)
// and w_hi / w_lo (boxes of 32 rows).  The x coordinate of every copy is 0.
cudaError_t tc_make_maps(dfmnmf_ctx* c) {
  EncodeTiledFn fn = encode_fn();
  if (!fn) return cudaErrorNotSupported;
  const cuuint64_t strides[1] = {(cuuint64_t)TC_KC * 2};
  const cuuint32_t estr[2] = {1, 1};
  const cuuint64_t blocks = (cuuint64_t)tc_tiles(c) * (c->Tr / TC_KC);
  struct { unsigned char* map; void* base; cuuint64_t rows; cuuint32_t box_rows; } m[4] = {
      {c->tmap_hi, c->Rhi, blocks * TC_ROWS, TC_ROWS},
      {c->tmap_lo, c->Rlo, blocks * TC_ROWS, TC_ROWS},
      {c->tmap_whi, c->wy_hi, blocks * TC_COLS, TC_COLS},
      {c->tmap_wlo, c->wy_lo, blocks * TC_COLS, TC_COLS}};
  for (int i = 0; i < 4; ++i) {
    const cuuint64_t dims[2] = {(cuuint64_t)TC_KC, m[i].rows};
    const cuuint32_t box[2] = {TC_KC, m[i].box_rows};
    const CUresult r = fn(reinterpret_cast<CUtensorMap*>(m[i].map), CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, m[i].base,
                          dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                          CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return cudaErrorInvalidValue;
  }
  return cudaSuccess;
}

cudaError_t launch_rprep(const dfmnmf_ctx* c, cudaStream_t s) {
  dim3 grid((c->Tr + 127) / 128, c->F);
  k_rprep<<<grid, 128, 0, s>>>(c->x, reinterpret_cast<__nv_bfloat16*>(c->Rhi),
                               reinterpret_cast<__nv_bfloat16*>(c->Rlo), c->F, c->T, c->Tr, c->K);
  return cudaGetLastError();
}

cudaError_t launch_wprep(const dfmnmf_ctx* c, cudaStream_t s, int fb, int fc) {
  dim3 grid((c->Tr / 2 + 127) / 128, fc);
  const size_t sm = (size_t)c->N * c->M * sizeof(float);
  auto whi = reinterpret_cast<__nv_bfloat16*>(c->wy_hi);
  auto wlo = reinterpret_cast<__nv_bfloat16*>(c->wy_lo);
#define DFM_WPREP(NMV, MV) \
  k_wprep<NMV, MV><<<grid, 128, sm, s>>>(c->lam, c->g, whi, wlo, c->F, c->T, c->Tp, c->Tr, c->N, c->eps, fb)
#define DFM_WPREP_N(MV)               \
  switch (c->N) {                     \
    case 1: DFM_WPREP(1, MV); break;  \
    case 2: DFM_WPREP(2, MV); break;  \
    case 3: DFM_WPREP(3, MV); break;  \
    case 4: DFM_WPREP(4, MV); break;  \
    case 5: DFM_WPREP(5, MV); break;  \
    case 6: DFM_WPREP(6, MV); break;  \
    case 7: DFM_WPREP(7, MV); break;  \
    case 8: DFM_WPREP(8, MV); break;  \
    default: DFM_WPREP(16, MV); break; \
  }
  switch (c->M) {
    case 4: DFM_WPREP_N(4); break;
    case 8: DFM_WPREP_N(8); break;
    case 16: DFM_WPREP_N(16); break;
    case 32: DFM_WPREP_N(32); break;
    default: return cudaErrorInvalidValue;
  }
#undef DFM_WPREP_N
#undef DFM_WPREP
  return cudaGetLastError();
}

// x as floats [F][T][2M] (boxes of 128 frames x 32 floats, 128-byte swizzle),
// lambda [N][F][Tp] (boxes of 128 frames x 1 frequency x N sources), P
// [F][T][M] (boxes of 128 frames x 16 floats, 64-byte swizzle).  Frames past
// T (or Tp) read as zeros and are not written.  The maps are encoded at
// launch and passed by value, so a captured graph keeps them.
cudaError_t launch_pstats_tma(const dfmnmf_ctx* c, cudaStream_t s, int fb, int fc, bool comp) {
  EncodeTiledFn fn = encode_fn();
  if (!fn || !pstats_tma_supported(c->K, c->MK, c->N)) return cudaErrorNotSupported;
  CUtensorMap mx, ml, mp;
  const cuuint32_t e3[3] = {1, 1, 1};
  {
    const cuuint64_t dims[3] = {32, (cuuint64_t)c->T, (cuuint64_t)c->F};
    const cuuint64_t str[2] = {128, (cuuint64_t)c->T * 128};
    const cuuint32_t box[3] = {32, PT_ROWS, 1};
    if (fn(&mx, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, c->x, dims, str, box, e3, CU_TENSOR_MAP_INTERLEAVE_NONE,
           CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) !=
        CUDA_SUCCESS)
      return cudaErrorInvalidValue;
  }
  {
    const cuuint64_t dims[3] = {(cuuint64_t)c->Tp, (cuuint64_t)c->F, (cuuint64_t)c->N};
    const cuuint64_t str[2] = {(cuuint64_t)c->Tp * 4, (cuuint64_t)c->F * c->Tp * 4};
    const cuuint32_t box[3] = {PT_ROWS, 1, (cuuint32_t)c->N};
    if (fn(&ml, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, c->lam, dims, str, box, e3, CU_TENSOR_MAP_INTERLEAVE_NONE,
           CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) !=
        CUDA_SUCCESS)
      return cudaErrorInvalidValue;
  }
  {
    const cuuint64_t dims[3] = {16, (cuuint64_t)c->T, (cuuint64_t)c->F};
    const cuuint64_t str[2] = {64, (cuuint64_t)c->T * 64};
    const cuuint32_t box[3] = {16, PT_ROWS, 1};
    if (fn(&mp, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, c->P, dims, str, box, e3, CU_TENSOR_MAP_INTERLEAVE_NONE,
           CU_TENSOR_MAP_SWIZZLE_64B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) !=
        CUDA_SUCCESS)
      return cudaErrorInvalidValue;
  }
  const size_t sm = pstats_tma_smem(c->N);
  auto kern = comp ? k_pstats_tma<true> : k_pstats_tma<false>;
  cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  dim3 grid(fc, (c->T + PT_ROWS - 1) / PT_ROWS);
  kern<<<grid, 128, sm, s>>>(mx, ml, mp, c->Q64, c->Q32, c->g, c->A, c->D, c->F, c->T, c->Tp, c->N, c->eps, fb,
                             c->flags);
  return cudaGetLastError();
}

cudaError_t launch_vtc(const dfmnmf_ctx* c, cudaStream_t s, int fb, int fc) {
  const size_t sm = tc_smem_bytes(c);
  cudaFuncSetAttribute(k_vtc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  const int FPC = TC_ROWS / (16 * c->K);
  const int grid = (fc + FPC - 1) / FPC;
  auto map = [](const unsigned char* p) { return *reinterpret_cast<const CUtensorMap*>(p); };
  k_vtc<<<grid, 128, sm, s>>>(map(c->tmap_hi), map(c->tmap_lo), map(c->tmap_whi), map(c->tmap_wlo), c->V, c->Vdd,
                              c->T, c->Tr, c->K, c->flags, fb, fb + fc);
  return cudaGetLastError();
}

}  // namespace dfm
