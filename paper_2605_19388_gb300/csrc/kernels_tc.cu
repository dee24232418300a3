// kernels_tc.cu -- tensor-core form of the weighted covariances (Eq. 13).
//
//   V[f][k][mu][a][b] = (1/T) sum_t R[f][k][a,b](t) * w[f][t][k,mu],
//   R = x_ftk x_ftk^H packed as M_k^2 = 16 reals, w = 1/yhat (Eq. 2, floored).
//
// For every frequency this is an (16 K x T) by (T x 4 K) product.  Its
// operands are split into two bfloat16 parts, R = R_hi + R_lo and
// w = w_hi + w_lo, and R_hi w_hi + R_hi w_lo + R_lo w_hi (+ R_lo w_lo) are
// accumulated in FP32 (the R_lo w_lo term is below 2^-16 relative; a plain
// bfloat16 contraction moves the IP update by 6e-2 relative on the
// paper-sized workload, the split form by 1.5e-4).
//
// k_vtc reads the observation x and lambda, g -- the method's own operands,
// each once -- and forms the split R and w on chip:
//   * one persistent CTA per SM walks a contiguous range of the flattened
//     (tile, 64-frame chunk) work list, so every SM gets the same number of
//     chunks; a tile is 8 / K frequencies (128 rows (f, k, entry) of R, 32
//     rows (f, m) of w);
//   * warp 0 streams each chunk's x tile (16 KB, swizzled), lambda rows and
//     g rows by TMA into a ring of raw stages;
//   * converter warps (one (frequency, subarray) pair per warp, lanes over
//     frame pairs) form R = x x^H and w = 1/max(sum_n lambda g, eps) in
//     registers, split them into bfloat16 pairs and write the K-major,
//     128-byte-swizzled operand tiles of the MMA (frames are laid out along
//     the contraction axis in the order (lane, j) -> 2 lane + j for frame
//     lane + 32 j; the contraction does not depend on the order, A and B use
//     the same one);
//   * one thread issues tcgen05.mma (M = 128, N = 64: w_hi and w_lo side by
//     side, K = 16 frames per instruction, FP32 accumulators in tensor memory,
//     two accumulator buffers so the epilogue of one tile overlaps the next);
//   * four epilogue warps read the accumulators with tcgen05.ld and write V.
//     A tile whose chunks are split between two CTAs is finished by the CTA
//     that arrives last: each part is stored in FP32, and the last one adds
//     the parts in CTA order (deterministic), in FP64.
//
// Supported layouts: M_k = 4 and K in {1, 2, 4, 8}.  Every mbarrier wait is
// bounded; a wait that gives up sets FLAG_TIMEOUT, the CTA drains its copies
// in flight and its tensor-core work, frees its tensor memory and returns.
// The pipeline waits use the context's budget (`budget` cycles, ~1 s unless
// set otherwise); the waits that drain copies and tensor-core work before the
// CTA exits always use the full ~1 s budget, so no copy or MMA can outlive it.
#include <cuda.h>
#include <cuda_bf16.h>

#include "../../include/dfmnmf.h"
#include "common.cuh"
#include "internal.h"
#include "tc_ptx.cuh"

namespace dfm {

// ------------------------------------------------------ fused contraction
constexpr int VX_ROWS = 128;                      // MMA M: rows (frequency, subarray, packed entry)
constexpr int VX_WROWS = 32;                      // rows (frequency, microphone) of one weight part
constexpr int VX_N = 2 * VX_WROWS;                // MMA N: w_hi rows, then w_lo rows
constexpr int VX_A_BYTES = VX_ROWS * 128;         // 16 KB: one 128-row region of 128-byte rows
// Per operand type.  bfloat16 (TF = false): chunks of 64 frames, R_hi and R_lo in two A regions, the
// B tile 64 rows of 64 frames.  TF32 (TF = true): chunks of 32 frames, the split kept along the
// contraction axis -- position 2 t holds the high part of frame t, 2 t + 1 its low part, and both
// positions of B hold w(t) -- so a row of A is 64 values in two 128-byte regions (frames 0..15,
// 16..31), and B is two 64-row regions.
template <bool TF> struct VxCfg {
  static constexpr int KC = TF ? 32 : 64;                         // frames per chunk
  static constexpr int X_BYTES = TF ? 8192 : 16384;               // raw x tile: 8/K frequencies x KC frames x 4K complex64
  static constexpr int B_BYTES = TF ? 2 * VX_N * 128 : VX_N * 128;
  static constexpr int OP_BYTES = 2 * VX_A_BYTES + B_BYTES;       // 40 KB (bfloat16), 48 KB (TF32)
};
constexpr int VX_OS = 3;                          // operand stages (unit i uses i % 3)
constexpr int VX_MAX_RS = 6;                      // raw stages at most
constexpr int VX_CW = 8;                          // converter warps per group: the 8 (frequency, subarray) pairs
constexpr int VX_PROD_WARP = 0;                   // TMA producer
constexpr int VX_MMA_WARP = 1;                    // MMA issuer
constexpr int VX_EPI_WARP = 2;                    // warps 2..5: epilogue (four consecutive warps: every lane quadrant)
constexpr int VX_CONV_WARP = 6;                   // warps 6..: converters
constexpr int VX_ACC_COLS = 64;                   // tensor-memory columns per accumulator buffer

// Instruction descriptors: D FP32 (bits 4-5 = 1), A and B of one type (bits 7-9, 10-12: bfloat16 = 1 under
// kind::f16, TF32 = 2 under kind::tf32), both K-major, N = 64 (bits 17-22: N / 8), M = 128 (bits 24-28: M / 16).
constexpr unsigned VX_IDESC = (1u << 4) | (1u << 7) | (1u << 10) | ((VX_N >> 3) << 17) | ((VX_ROWS >> 4) << 24);
constexpr unsigned VX_IDESC_TF32 = (1u << 4) | (2u << 7) | (2u << 10) | ((VX_N >> 3) << 17) | ((VX_ROWS >> 4) << 24);

__device__ __forceinline__ void umma_bf16(unsigned tmem_d, unsigned long long a, unsigned long long b, unsigned acc) {
  umma_f16_id(tmem_d, a, b, VX_IDESC, acc);
}
__device__ __forceinline__ void umma_tf32(unsigned tmem_d, unsigned long long a, unsigned long long b, unsigned acc) {
  umma_tf32_id(tmem_d, a, b, VX_IDESC_TF32, acc);
}

struct VxCtl {
  unsigned long long raw_full[VX_MAX_RS];
  unsigned long long raw_empty[VX_MAX_RS];
  unsigned long long op_full[VX_OS];
  unsigned long long op_empty[VX_OS];
  unsigned long long acc_full[2];
  unsigned long long acc_empty[2];
  unsigned long long done;
  unsigned tmem_base;
  unsigned abort;
  unsigned last;
};

// CTA b of a G-CTA grid owns units [b U / G, (b + 1) U / G); the CTA owning unit u.
__host__ __device__ __forceinline__ int vx_cta_of(long long u, int G, long long U) {
  return (int)(((u + 1) * G - 1) / U);
}

// Barrier 1 among the 128 epilogue threads, returning the OR of `pred` over them.
__device__ __forceinline__ bool epi_bar_or(bool pred) {
  unsigned r;
  asm volatile(
      "{\n .reg .pred p, q;\n setp.ne.u32 p, %1, 0;\n barrier.red.or.pred q, 1, 128, p;\n selp.u32 %0, 1, 0, q;\n}"
      : "=r"(r)
      : "r"((unsigned)pred)
      : "memory");
  return r != 0;
}
__device__ __forceinline__ void epi_bar() { asm volatile("bar.sync 1, 128;" ::: "memory"); }

// Entry e = 4a + b of the packed x x^H of block blk (sums over t already
// scaled by 1/T) into V (FP64) and Vdd (float pairs), all four mu at once:
// e with a == b is V[a][a]; a < b is Re V[a][b] = Re V[b][a]; a > b is
// Im(x_b conj x_a) = Im V[b][a] = -Im V[a][b].
__device__ __forceinline__ void vx_write_v(double2* __restrict__ V, float4* __restrict__ Vdd, size_t blk, int a,
                                           int b, const double (&dv)[4]) {
#pragma unroll
  for (int mu = 0; mu < 4; ++mu) {
    double2* Vb = V + (blk * 4 + mu) * 16;
    float4* Vd = Vdd + (blk * 4 + mu) * 16;
    double* vdbl = reinterpret_cast<double*>(Vb);
    float* vflt = reinterpret_cast<float*>(Vd);
    const float fv = (float)dv[mu];
    if (a == b) {
      Vb[a * 4 + a] = make_double2(dv[mu], 0.0);
      Vd[a * 4 + a] = make_float4(fv, 0.f, 0.f, 0.f);
    } else if (a < b) {
      vdbl[2 * (a * 4 + b)] = dv[mu];
      vdbl[2 * (b * 4 + a)] = dv[mu];
      vflt[4 * (a * 4 + b)] = fv; vflt[4 * (a * 4 + b) + 1] = 0.f;
      vflt[4 * (b * 4 + a)] = fv; vflt[4 * (b * 4 + a) + 1] = 0.f;
    } else {
      vdbl[2 * (b * 4 + a) + 1] = dv[mu];
      vdbl[2 * (a * 4 + b) + 1] = -dv[mu];
      vflt[4 * (b * 4 + a) + 2] = fv; vflt[4 * (b * 4 + a) + 3] = 0.f;
      vflt[4 * (a * 4 + b) + 2] = -fv; vflt[4 * (a * 4 + b) + 3] = 0.f;
    }
  }
}

// Nearest TF32 value of x (round half away from zero), as an FP32 number with the low 13 bits zero.
__device__ __forceinline__ float tf32_rna(float x) {
  unsigned r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}

// r = hi + lo with hi = bfloat16(r) (round to nearest) and lo = bfloat16(r - hi), for two frames at once.
__device__ __forceinline__ void vx_split_store(unsigned char* hi, unsigned char* lo, float r0, float r1) {
  const __nv_bfloat162 h = __floats2bfloat162_rn(r0, r1);
  const float h0 = __uint_as_float((unsigned)__bfloat16_as_ushort(h.x) << 16);
  const float h1 = __uint_as_float((unsigned)__bfloat16_as_ushort(h.y) << 16);
  *reinterpret_cast<__nv_bfloat162*>(hi) = h;
  *reinterpret_cast<__nv_bfloat162*>(lo) = __floats2bfloat162_rn(r0 - h0, r1 - h1);
}

// The fused contraction; see the head of this file.  K subarrays of 4
// microphones, CG groups of 8 converter warps (each group converts every
// CG-th chunk of the CTA).  Dynamic shared memory, 1024-byte aligned:
// VX_OS operand stages (R_hi, R_lo, w_hi | w_lo), RS raw stages of
// stage_bytes (x tile, lambda [N][8/K][64], g [8/K][N][M]), control block.
// `part` holds one 128-row block of FP32 partial sums per (tile, CTA) pair
// that shares a tile (slot tile - tb + CTA), `tickets` one counter per tile,
// zero between launches (the CTA that completes a tile resets it).
template <int K, int CG, bool TF>
__global__ void __launch_bounds__((VX_CONV_WARP + VX_CW * CG) * 32, 1)
    k_vtc(const __grid_constant__ CUtensorMap map_x, const __grid_constant__ CUtensorMap map_l,
          const __grid_constant__ CUtensorMap map_g, double2* __restrict__ V, float4* __restrict__ Vdd,
          float4* __restrict__ part, unsigned* __restrict__ tickets, int F, int T, int N, float eps, int tb,
          int ntile, int nch, int RS, int stage_bytes, unsigned budget, unsigned* __restrict__ flags) {
  constexpr int FPC = 8 / K, M = 4 * K;
  constexpr unsigned SWZ = (K == 1) ? 0x10u : (K == 2) ? 0x30u : 0x70u;  // 32-, 64-, 128-byte swizzle of x
  extern __shared__ __align__(1024) unsigned char vx_raw[];
  // 1024-byte alignment by an offset from the shared array (not by integer casts of the pointer), so that
  // the compiler keeps every derived pointer in the shared window (32-bit shared loads and stores)
  unsigned char* ops = vx_raw + ((1024u - (smem_u32(vx_raw) & 1023u)) & 1023u);
  using Cfg = VxCfg<TF>;
  constexpr int KC = Cfg::KC, X_BYTES = Cfg::X_BYTES, OP_BYTES = Cfg::OP_BYTES;
  unsigned char* raw = ops + VX_OS * OP_BYTES;
  VxCtl* ctl = reinterpret_cast<VxCtl*>(raw + (size_t)RS * stage_bytes);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const long long U = (long long)ntile * nch;  // below 2^31 (checked at launch)
  const int G = gridDim.x;
  const int u_begin = (int)((long long)blockIdx.x * U / G);
  const int nloc = (int)((long long)(blockIdx.x + 1) * U / G) - u_begin;
  const int c_begin = u_begin % nch;  // chunk of the CTA's first unit
  const int lbytes = FPC * N * KC * 4;  // lambda rows of one stage
  volatile unsigned* abort_flag = &ctl->abort;

  if (tid == 0) {
    for (int s = 0; s < RS; ++s) {
      mbar_init(&ctl->raw_full[s], 1);
      mbar_init(&ctl->raw_empty[s], VX_CW);
    }
    for (int s = 0; s < VX_OS; ++s) {
      mbar_init(&ctl->op_full[s], VX_CW);
      mbar_init(&ctl->op_empty[s], 1);
    }
    for (int s = 0; s < 2; ++s) {
      mbar_init(&ctl->acc_full[s], 1);
      mbar_init(&ctl->acc_empty[s], 4);
    }
    mbar_init(&ctl->done, 1);
    ctl->abort = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&ctl->tmem_base)),
                 "r"(2 * VX_ACC_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  }
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const unsigned tmem = ctl->tmem_base;

  if (warp == VX_PROD_WARP) {
    // ---- TMA producer: the whole warp walks the units (warp-uniform control flow), one elected lane
    // issues the copies
    const unsigned tx = (unsigned)(X_BYTES + lbytes + FPC * N * M * 4);
    int issued = 0, tile = tb + u_begin / nch, c = c_begin;
    for (int i = 0; i < nloc; ++i, c = (c + 1 == nch) ? (++tile, 0) : c + 1) {
      const int s = i % RS;
      if (i >= RS && !mbar_wait_warp(&ctl->raw_empty[s], ((i / RS) - 1) & 1, 128, budget)) {
        if (lane == 0) atomicOr(&ctl->abort, 1u);
        break;
      }
      if (__any_sync(DFM_FULL_MASK, *abort_flag != 0)) break;
      unsigned char* st = raw + (size_t)s * stage_bytes;
      if (elect_one()) {
        mbar_arrive_expect_tx(&ctl->raw_full[s], tx);
        if (K == 8) tma_load_4d(st, &map_x, 0, 0, c * KC, tile, &ctl->raw_full[s]);
        else tma_load_3d(st, &map_x, 0, c * KC, tile * FPC, &ctl->raw_full[s]);
        tma_load_3d(st + X_BYTES, &map_l, c * KC, tile * FPC, 0, &ctl->raw_full[s]);
        tma_load_3d(st + X_BYTES + lbytes, &map_g, 0, 0, tile * FPC, &ctl->raw_full[s]);
      }
      __syncwarp();
      issued = i + 1;
    }
    // every copy issued has landed before the CTA moves on (bounded wait)
    for (int i = issued > RS ? issued - RS : 0; i < issued; ++i)
      if (!mbar_wait_warp(&ctl->raw_full[i % RS], (i / RS) & 1, 128) && lane == 0) atomicOr(&ctl->abort, 1u);
  } else if (warp == VX_MMA_WARP) {
    // ---- MMA issuer: the whole warp walks the units, one elected lane issues per chunk R_hi (w_hi | w_lo)
    // then R_lo (w_hi | w_lo), 16 frames per instruction
    const unsigned long long dstage0 = smem_desc_sw128(smem_u32(ops));
    int sg = -1;
    for (int i = 0, c = c_begin; i < nloc; ++i, c = (c + 1 == nch) ? 0 : c + 1) {
      const bool first = (i == 0 || c == 0), last = (i == nloc - 1 || c == nch - 1);
      if (first) {
        ++sg;
        if (sg >= 2 && !mbar_wait_warp(&ctl->acc_empty[sg & 1], ((sg >> 1) - 1) & 1, 32, budget)) {
          if (lane == 0) atomicOr(&ctl->abort, 1u);
          break;
        }
      }
      const int os = i % VX_OS;
      if (!mbar_wait_warp(&ctl->op_full[os], (i / VX_OS) & 1, 32, budget)) {
        if (lane == 0) atomicOr(&ctl->abort, 1u);
        break;
      }
      if (__any_sync(DFM_FULL_MASK, *abort_flag != 0)) break;
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      // descriptors of the stage: the start-address field (address / 16, 14 bits, no carry below 256 KB)
      // advances by the byte offset / 16 of each tile and of each 16-frame step (32 bytes)
      const unsigned long long da = dstage0 + (unsigned long long)((os * OP_BYTES) >> 4);
      const unsigned d = tmem + (unsigned)((sg & 1) * VX_ACC_COLS);
      if (elect_one()) {
        if constexpr (TF) {
          // 8 steps of 8 positions (4 frames, high and low parts): region s / 4, 32 bytes per step in it
#pragma unroll
          for (int st8 = 0; st8 < 8; ++st8) {
            const unsigned long long a = da + (unsigned long long)(((st8 >> 2) * VX_A_BYTES) >> 4) + 2 * (st8 & 3);
            const unsigned long long b =
                da + (unsigned long long)((2 * VX_A_BYTES + (st8 >> 2) * VX_N * 128) >> 4) + 2 * (st8 & 3);
            umma_tf32(d, a, b, (first && st8 == 0) ? 0u : 1u);
          }
        } else {
#pragma unroll
          for (int kk = 0; kk < KC / 16; ++kk) {
            const unsigned long long b = da + (unsigned long long)(((2 * VX_A_BYTES) >> 4) + 2 * kk);
            umma_bf16(d, da + (unsigned long long)(2 * kk), b, (first && kk == 0) ? 0u : 1u);
            umma_bf16(d, da + (unsigned long long)((VX_A_BYTES >> 4) + 2 * kk), b, 1u);
          }
        }
        umma_commit(&ctl->op_empty[os]);
        if (last) umma_commit(&ctl->acc_full[sg & 1]);
      }
      __syncwarp();
    }
    if (elect_one()) umma_commit(&ctl->done);
    __syncwarp();
  } else if (warp >= VX_EPI_WARP && warp < VX_EPI_WARP + 4) {
    // ---- epilogue: warp w reads tensor-memory lanes 32 (w % 4) .. + 31 (row = lane)
    const int q = warp & 3, row = q * 32 + lane;
    const int pair = row >> 4, e = row & 15;
    const int fj = pair / K, k = pair % K, a = e >> 2, b = e & 3;
    const bool up = lane >= 16;  // the second (frequency, subarray) pair of the warp
    const double invT = 1.0 / (double)T;
    int sg = -1;
    for (int i0 = 0; i0 < nloc;) {
      const int u0 = u_begin + i0;
      const int tl = u0 / nch, c0 = u0 % nch;
      const int len = min(nch - c0, nloc - i0);
      const bool full = (c0 == 0 && len == nch);
      ++sg;
      // polls are rare while the converters run (they would take their issue slots); the CTA's last tile is
      // awaited closely, since nothing else is left to run and the launch ends with it
      const bool okw = mbar_wait(&ctl->acc_full[sg & 1], (sg >> 1) & 1, (i0 + len == nloc) ? 32u : 512u, budget);
      if (!okw) atomicOr(&ctl->abort, 1u);
      if (epi_bar_or(!okw || *abort_flag)) break;
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      unsigned h[8], l[8];
      const unsigned ta = tmem + ((unsigned)(q * 32) << 16) + (unsigned)((sg & 1) * VX_ACC_COLS + 8 * q);
      asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
                   : "=r"(h[0]), "=r"(h[1]), "=r"(h[2]), "=r"(h[3]), "=r"(h[4]), "=r"(h[5]), "=r"(h[6]), "=r"(h[7])
                   : "r"(ta));
      asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
                   : "=r"(l[0]), "=r"(l[1]), "=r"(l[2]), "=r"(l[3]), "=r"(l[4]), "=r"(l[5]), "=r"(l[6]), "=r"(l[7])
                   : "r"(ta + VX_WROWS));
      asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      __syncwarp();
      if (lane == 0) mbar_arrive(&ctl->acc_empty[sg & 1]);
      float v[4];
#pragma unroll
      for (int mu = 0; mu < 4; ++mu)
        v[mu] = __uint_as_float(up ? h[4 + mu] : h[mu]) + __uint_as_float(up ? l[4 + mu] : l[mu]);
      const int tile = tb + tl, f = tile * FPC + fj;
      const size_t blk = (size_t)f * K + k;
      if (full) {
        if (f < F) {
          double dv[4];
#pragma unroll
          for (int mu = 0; mu < 4; ++mu) dv[mu] = (double)v[mu] * invT;
          vx_write_v(V, Vdd, blk, a, b, dv);
        }
      } else {
        // tile shared with other CTAs: publish this part, the last CTA to arrive adds them in CTA order
        const int bfirst = vx_cta_of((long long)tl * nch, G, U);
        const int blast = vx_cta_of((long long)tl * nch + nch - 1, G, U);
        part[((size_t)tl + blockIdx.x) * VX_ROWS + row] = make_float4(v[0], v[1], v[2], v[3]);
        __threadfence();
        epi_bar();
        if (tid == VX_EPI_WARP * 32) ctl->last = (atomicAdd(&tickets[tile], 1u) == (unsigned)(blast - bfirst));
        epi_bar();
        if (ctl->last) {
          __threadfence();
          double dv[4] = {0.0, 0.0, 0.0, 0.0};
          for (int bb = bfirst; bb <= blast; ++bb) {
            const float4 p = __ldcg(part + ((size_t)tl + bb) * VX_ROWS + row);
            dv[0] += (double)p.x;
            dv[1] += (double)p.y;
            dv[2] += (double)p.z;
            dv[3] += (double)p.w;
          }
          if (f < F) {
#pragma unroll
            for (int mu = 0; mu < 4; ++mu) dv[mu] *= invT;
            vx_write_v(V, Vdd, blk, a, b, dv);
          }
          if (tid == VX_EPI_WARP * 32) tickets[tile] = 0u;
        }
        epi_bar();
      }
      i0 += len;
    }
  } else if (warp >= VX_CONV_WARP) {
    // ---- converters: warp cw of group grp forms rows 16 cw .. 16 cw + 15 of R (pair cw) and the w rows of
    // its four microphones for frames lane and lane + 32 of every CG-th chunk
    const int cw = (warp - VX_CONV_WARP) % VX_CW, grp = (warp - VX_CONV_WARP) / VX_CW;
    const int fj = cw / K, k = cw % K;
    const unsigned lo4 = (unsigned)(lane & 3) * 4, c8 = (unsigned)(lane >> 2);
    const int wrow = fj * M + 4 * k;  // first w row of this pair
    int c = (u_begin + grp) % nch;  // chunk of unit i, advanced by CG per step
    for (int i = grp; i < nloc; i += CG) {
      const int s = i % RS, os = i % VX_OS;
      bool ok = mbar_wait_warp(&ctl->raw_full[s], (i / RS) & 1, 32, budget);
      if (ok && i >= VX_OS) ok = mbar_wait_warp(&ctl->op_empty[os], ((i / VX_OS) - 1) & 1, 32, budget);
      if (!ok) {
        if (lane == 0) atomicOr(&ctl->abort, 1u);
        break;
      }
      if (__any_sync(DFM_FULL_MASK, *abort_flag != 0)) break;
      const unsigned char* st = raw + (size_t)s * stage_bytes;
      const float* ls = reinterpret_cast<const float*>(st + X_BYTES);
      const float* gs = reinterpret_cast<const float*>(st + X_BYTES + lbytes);
      unsigned char* op = ops + os * OP_BYTES;
      if constexpr (TF) {
        // TF32: frame `lane` of the chunk.  R and w each split as hi = the value rounded to TF32 (cvt.rna)
        // and lo = value - hi (exact); hi and lo of a frame are adjacent on the contraction axis, so each
        // entry is one 8-byte store: region lane / 16, 16-byte chunk (lane % 16) / 2 of the row (swizzled
        // with the row), half lane % 2.
        float2 xv[4];
#pragma unroll
        for (int hh = 0; hh < 2; ++hh) {
          const unsigned lin = (unsigned)((fj * KC + lane) * (8 * M) + k * 32 + hh * 16);
          const float4 qv = *reinterpret_cast<const float4*>(st + (lin ^ ((lin >> 3) & SWZ)));
          xv[2 * hh] = make_float2(qv.x, qv.y);
          xv[2 * hh + 1] = make_float2(qv.z, qv.w);
        }
        const unsigned kq = (unsigned)(lane & 15);
        const unsigned tfoff = (unsigned)(lane >> 4) * VX_A_BYTES + (kq & 1u) * 8u;
        unsigned char* arow = op + cw * 16 * 128 + tfoff;
#pragma unroll
        for (int aa = 0; aa < 4; ++aa)
#pragma unroll
          for (int bb = 0; bb < 4; ++bb) {
            const float2 xa = xv[aa], xb = xv[bb];
            const float r = (aa == bb) ? fmaf(xa.x, xa.x, xa.y * xa.y)
                            : (aa < bb) ? fmaf(xa.x, xb.x, xa.y * xb.y)
                                        : fmaf(xb.y, xa.x, -xb.x * xa.y);
            const int e = aa * 4 + bb;
            const unsigned off = (unsigned)(e * 128) + (((kq >> 1) ^ (unsigned)(e & 7)) << 4);
            const float h = tf32_rna(r);
            *reinterpret_cast<float2*>(arow + off) = make_float2(h, r - h);
          }
        float y[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll 4
        for (int n = 0; n < N; ++n) {
          const float l0 = ls[(n * FPC + fj) * KC + lane];
          const float4 gv = *reinterpret_cast<const float4*>(gs + (fj * N + n) * M + 4 * k);
          y[0] = fmaf(l0, gv.x, y[0]); y[1] = fmaf(l0, gv.y, y[1]);
          y[2] = fmaf(l0, gv.z, y[2]); y[3] = fmaf(l0, gv.w, y[3]);
        }
        const bool v0 = c * KC + lane < T;
        unsigned char* bt = op + 2 * VX_A_BYTES + (unsigned)(lane >> 4) * (VX_N * 128) + (kq & 1u) * 8u;
#pragma unroll
        for (int mu = 0; mu < 4; ++mu) {
          const int rw = wrow + mu;
          const unsigned off = (unsigned)(rw * 128) + (((kq >> 1) ^ (unsigned)(rw & 7)) << 4);
          const float w = v0 ? fast_rcp(fmaxf(y[mu], eps)) : 0.f;
          const float h = tf32_rna(w), l = w - h;
          *reinterpret_cast<float2*>(bt + off) = make_float2(h, h);
          *reinterpret_cast<float2*>(bt + VX_WROWS * 128 + off) = make_float2(l, l);
        }
      } else {
        // x of frames lane and lane + 32, microphones 0..3 of the pair
        float2 xv[2][4];
  #pragma unroll
        for (int j = 0; j < 2; ++j)
  #pragma unroll
          for (int hh = 0; hh < 2; ++hh) {
            const unsigned lin = (unsigned)((fj * KC + lane + 32 * j) * (8 * M) + k * 32 + hh * 16);
            const float4 qv = *reinterpret_cast<const float4*>(st + (lin ^ ((lin >> 3) & SWZ)));
            xv[j][2 * hh] = make_float2(qv.x, qv.y);
            xv[j][2 * hh + 1] = make_float2(qv.z, qv.w);
          }
        // R = x x^H, entry 4a + b: |x_a|^2 (a == b), Re x_a conj x_b (a < b), Im x_b conj x_a (a > b)
        // (scalar single precision: packed pairs cost more register moves than they save)
        unsigned char* arow = op + cw * 16 * 128 + lo4;
  #pragma unroll
        for (int aa = 0; aa < 4; ++aa)
  #pragma unroll
          for (int bb = 0; bb < 4; ++bb) {
            float r[2];
  #pragma unroll
            for (int j = 0; j < 2; ++j) {
              const float2 xa = xv[j][aa], xb = xv[j][bb];
              if (aa == bb) r[j] = fmaf(xa.x, xa.x, xa.y * xa.y);
              else if (aa < bb) r[j] = fmaf(xa.x, xb.x, xa.y * xb.y);
              else r[j] = fmaf(xb.y, xa.x, -xb.x * xa.y);
            }
            const int e = aa * 4 + bb;
            const unsigned off = (unsigned)(e * 128) + ((c8 ^ (unsigned)(e & 7)) << 4);
            vx_split_store(arow + off, arow + VX_A_BYTES + off, r[0], r[1]);
          }
        // w = 1 / max(yhat, eps) for the pair's four microphones, zero past T
        float y[2][4];
  #pragma unroll
        for (int j = 0; j < 2; ++j)
  #pragma unroll
          for (int mu = 0; mu < 4; ++mu) y[j][mu] = 0.f;
#pragma unroll 4
        for (int n = 0; n < N; ++n) {
          const float l0 = ls[(n * FPC + fj) * KC + lane], l1 = ls[(n * FPC + fj) * KC + lane + 32];
          const float4 gv = *reinterpret_cast<const float4*>(gs + (fj * N + n) * M + 4 * k);
          y[0][0] = fmaf(l0, gv.x, y[0][0]); y[0][1] = fmaf(l0, gv.y, y[0][1]);
          y[0][2] = fmaf(l0, gv.z, y[0][2]); y[0][3] = fmaf(l0, gv.w, y[0][3]);
          y[1][0] = fmaf(l1, gv.x, y[1][0]); y[1][1] = fmaf(l1, gv.y, y[1][1]);
          y[1][2] = fmaf(l1, gv.z, y[1][2]); y[1][3] = fmaf(l1, gv.w, y[1][3]);
        }
        const bool v0 = c * KC + lane < T, v1 = c * KC + lane + 32 < T;
        unsigned char* bt = op + 2 * VX_A_BYTES + lo4;
  #pragma unroll
        for (int mu = 0; mu < 4; ++mu) {
          const int rw = wrow + mu;
          const unsigned off = (unsigned)(rw * 128) + ((c8 ^ (unsigned)(rw & 7)) << 4);
          vx_split_store(bt + off, bt + VX_WROWS * 128 + off, v0 ? fast_rcp(fmaxf(y[0][mu], eps)) : 0.f,
                         v1 ? fast_rcp(fmaxf(y[1][mu], eps)) : 0.f);
        }
      }
      // generic-proxy writes of the operand tiles, then hand the stages over
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      __syncwarp();
      if (lane == 0) {
        mbar_arrive(&ctl->raw_empty[s]);
        mbar_arrive(&ctl->op_full[os]);
      }
      for (c += CG; c >= nch;) c -= nch;
    }
  }

  __syncthreads();
  if (warp == 0) {
    // all tensor-core work of the CTA has completed before its tensor memory is freed (bounded wait)
    if (!mbar_wait_warp(&ctl->done, 0, 32) && lane == 0) atomicOr(&ctl->abort, 1u);
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(2 * VX_ACC_COLS) : "memory");
  }
  if (tid == 0 && *abort_flag) atomicOr(flags + FLAG_TIMEOUT, 1u);
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
  unsigned char* base = pt_raw + ((1024u - (smem_u32(pt_raw) & 1023u)) & 1023u);  // stays in the shared window
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

// Tiles of 8 / K frequencies; slots of partial sums (one per (tile, CTA) pair
// that can share a tile: tiles + CTAs) and tickets (one per tile).
int tc_tiles(const dfmnmf_ctx* c) {
  const int FPC = 8 / c->K;
  return (c->F + FPC - 1) / FPC;
}
size_t tc_part_float4s(const dfmnmf_ctx* c) { return ((size_t)tc_tiles(c) + (size_t)c->num_sms) * VX_ROWS; }
size_t tc_ticket_count(const dfmnmf_ctx* c) { return (size_t)tc_tiles(c); }

// Raw stage of the fused contraction: x tile, lambda rows, g rows, rounded to 1 KB.
static bool vx_tf32(const dfmnmf_ctx* c) { return c->precision == DFMNMF_TF32_TC; }
static int vx_kc(bool tf) { return tf ? VxCfg<true>::KC : VxCfg<false>::KC; }
static int vx_op_bytes(bool tf) { return tf ? VxCfg<true>::OP_BYTES : VxCfg<false>::OP_BYTES; }
static int vx_stage_bytes(int K, int N, bool tf) {
  const int FPC = 8 / K;
  const int b = (tf ? VxCfg<true>::X_BYTES : VxCfg<false>::X_BYTES) + FPC * N * vx_kc(tf) * 4 + FPC * N * 4 * K * 4;
  return (b + 1023) & ~1023;
}

// Raw stages that fit beside the operand stages (at most VX_MAX_RS, at least 2; 0 if none fit).
int tc_raw_stages(const dfmnmf_ctx* c) {
  const bool tf = vx_tf32(c);
  const long avail = (long)c->smem_optin - 1024 - (long)VX_OS * vx_op_bytes(tf) - (long)sizeof(VxCtl);
  const long rs = avail / vx_stage_bytes(c->K, c->N, tf);
  return rs < 2 ? 0 : (int)(rs > VX_MAX_RS ? VX_MAX_RS : rs);
}

template <int K, int CG, bool TF>
static cudaError_t launch_vtc_k(const dfmnmf_ctx* c, cudaStream_t s, const CUtensorMap& mx, const CUtensorMap& ml,
                                const CUtensorMap& mg, int tb, int ntile, int nch, int G, int RS, int stage,
                                size_t smem) {
  auto kern = k_vtc<K, CG, TF>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  kern<<<G, (VX_CONV_WARP + VX_CW * CG) * 32, smem, s>>>(mx, ml, mg, c->V, c->Vdd, c->tc_part, c->tc_ticket, c->F,
                                                          c->T, c->N, c->eps, tb, ntile, nch, RS, stage,
                                                          c->wait_cycles, c->flags);
  return cudaGetLastError();
}

// The fused contraction for frequencies [fb, fb + fc), fb a multiple of 8 / K.
// x as floats [F][T][2M] (boxes of KC frames x 8/K frequencies, KC = 64 for
// bfloat16 operands and 32 for TF32; for K = 8 the 256-byte frame rows as two
// 128-byte halves), lambda [N][F][Tp] (KC frames x 8/K frequencies x N),
// g [F][N][M] (8/K frequencies); frames past T and
// frequencies past F read as zeros.  The maps are encoded at launch and
// passed by value, so a captured graph keeps them.
cudaError_t launch_vtc(const dfmnmf_ctx* c, cudaStream_t s, int fb, int fc) {
  EncodeTiledFn fn = encode_fn();
  if (!fn || !tc_supported(c->MK, c->K) || !c->tc_part) return cudaErrorNotSupported;
  const int K = c->K, FPC = 8 / K, M = c->M;
  if (fc <= 0) return cudaSuccess;
  if (fb % FPC) return cudaErrorInvalidValue;
  const int tb = fb / FPC, ntile = (fb + fc + FPC - 1) / FPC - tb;
  const bool tf = vx_tf32(c);
  const int KC = vx_kc(tf);
  const int nch = (c->T + KC - 1) / KC;
  const long long U = (long long)ntile * nch;
  const int G = (int)(U < c->num_sms ? U : c->num_sms);
  const int RS = tc_raw_stages(c), stage = vx_stage_bytes(K, c->N, tf);
  if (RS == 0 || U >= (1ll << 31) / (c->num_sms + 1)) return cudaErrorInvalidValue;  // unit indices stay 32-bit
  const size_t smem = 1024 + (size_t)VX_OS * vx_op_bytes(tf) + (size_t)RS * stage + sizeof(VxCtl);
  CUtensorMap mx, ml, mg;
  const cuuint32_t e4[4] = {1, 1, 1, 1};
  CUresult r;
  if (K == 8) {
    const cuuint64_t dims[4] = {32, 2, (cuuint64_t)c->T, (cuuint64_t)c->F};
    const cuuint64_t str[3] = {128, 256, (cuuint64_t)c->T * 256};
    const cuuint32_t box[4] = {32, 2, (cuuint32_t)KC, 1};
    r = fn(&mx, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, c->x, dims, str, box, e4, CU_TENSOR_MAP_INTERLEAVE_NONE,
           CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  } else {
    const cuuint64_t dims[3] = {(cuuint64_t)(2 * M), (cuuint64_t)c->T, (cuuint64_t)c->F};
    const cuuint64_t str[2] = {(cuuint64_t)(8 * M), (cuuint64_t)c->T * 8 * M};
    const cuuint32_t box[3] = {(cuuint32_t)(2 * M), (cuuint32_t)KC, (cuuint32_t)FPC};
    const CUtensorMapSwizzle sw =
        K == 1 ? CU_TENSOR_MAP_SWIZZLE_32B : K == 2 ? CU_TENSOR_MAP_SWIZZLE_64B : CU_TENSOR_MAP_SWIZZLE_128B;
    r = fn(&mx, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, c->x, dims, str, box, e4, CU_TENSOR_MAP_INTERLEAVE_NONE, sw,
           CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  }
  if (r != CUDA_SUCCESS) return cudaErrorInvalidValue;
  {
    const cuuint64_t dims[3] = {(cuuint64_t)c->Tp, (cuuint64_t)c->F, (cuuint64_t)c->N};
    const cuuint64_t str[2] = {(cuuint64_t)c->Tp * 4, (cuuint64_t)c->F * c->Tp * 4};
    const cuuint32_t box[3] = {(cuuint32_t)KC, (cuuint32_t)FPC, (cuuint32_t)c->N};
    if (fn(&ml, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, c->lam, dims, str, box, e4, CU_TENSOR_MAP_INTERLEAVE_NONE,
           CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) !=
        CUDA_SUCCESS)
      return cudaErrorInvalidValue;
  }
  {
    const cuuint64_t dims[3] = {(cuuint64_t)M, (cuuint64_t)c->N, (cuuint64_t)c->F};
    const cuuint64_t str[2] = {(cuuint64_t)M * 4, (cuuint64_t)c->N * M * 4};
    const cuuint32_t box[3] = {(cuuint32_t)M, (cuuint32_t)c->N, (cuuint32_t)FPC};
    if (fn(&mg, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, c->g, dims, str, box, e4, CU_TENSOR_MAP_INTERLEAVE_NONE,
           CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) !=
        CUDA_SUCCESS)
      return cudaErrorInvalidValue;
  }
#define DFM_VTC_TF(KK, TFV)                                                                                      \
  return c->cfg_vx_groups == 1 ? launch_vtc_k<KK, 1, TFV>(c, s, mx, ml, mg, tb, ntile, nch, G, RS, stage, smem) \
                               : launch_vtc_k<KK, 2, TFV>(c, s, mx, ml, mg, tb, ntile, nch, G, RS, stage, smem)
#define DFM_VTC(KK)                \
  if (tf) DFM_VTC_TF(KK, true);    \
  else DFM_VTC_TF(KK, false)
  switch (K) {
    case 1: DFM_VTC(1);
    case 2: DFM_VTC(2);
    case 4: DFM_VTC(4);
    default: DFM_VTC(8);
  }
#undef DFM_VTC
#undef DFM_VTC_TF
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

}  // namespace dfm
