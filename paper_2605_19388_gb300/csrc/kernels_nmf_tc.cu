// kernels_nmf_tc.cu -- the products of the W update (Eq. 8) on the tensor cores, used by the
// tensor-core forms:
//   num[n][f][b] = sum_t A[n][f][t] H[n][b][t],   den[n][f][b] = sum_t D[n][f][t] H[n][b][t]
// as tcgen05.mma of kind::tf32: A, D and H are read by TMA straight from their FP32 arrays (the
// tensor cores use the TF32 part of each value) into 128-byte-swizzled K-major tiles, M = 128 bins,
// N = B rounded up to 16, K = 8 frames per instruction, FP32 accumulation in tensor memory (num in
// columns 0 .. NB - 1, den in NB .. 2 NB - 1).  The frames of each (source, 128-bin tile) are
// split over S CTAs; every CTA stores its FP32 part and the last to arrive adds the S parts in split
// order and applies W <- W sqrt(num / max(den, eps)) (Eq. 8 with the floor of Sec. IV-A), or writes
// den - num in gradient mode.  Nothing waits on another CTA.
//
// The H update (Eq. 9) contracts over the bins, the leading axis of A and D in memory: its TF32
// operands would have to be transposed on chip first, so it stays on the CUDA cores (k_hupd).
#include <cuda.h>

#include "../../include/dfmnmf.h"
#include "common.cuh"
#include "internal.h"
#include "tc_ptx.cuh"

namespace dfm {

constexpr int WT_ROWS = 128;                  // MMA M: bins per tile
constexpr int WT_KC = 32;                     // frames per chunk (one 128-byte row of FP32)
constexpr int WT_STAGES = 4;
constexpr int WT_AD_BYTES = WT_ROWS * 128;    // one A or D chunk: 16 KB
constexpr int WT_MAX_SPLIT = 8;

struct WtCtl {
  unsigned long long full[WT_STAGES];
  unsigned long long empty[WT_STAGES];
  unsigned long long done;
  unsigned tmem_base;
  unsigned abort;
  unsigned last;
};

// grid (ceil(F / 128), N, S); 128 threads.  Dynamic shared memory: WT_STAGES stages of
// (A chunk, D chunk, H chunk of NB rows), 1024-byte aligned, then the control block.
__global__ void __launch_bounds__(128, 1) k_wupd_tc(const __grid_constant__ CUtensorMap map_a,
                                                    const __grid_constant__ CUtensorMap map_d,
                                                    const __grid_constant__ CUtensorMap map_h, float* __restrict__ W,
                                                    int F, int B, int NB, float eps, unsigned* __restrict__ flags,
                                                    int S, int cps, int nch, float2* __restrict__ part,
                                                    unsigned* __restrict__ ticket, float* __restrict__ grad) {
  extern __shared__ __align__(1024) unsigned char wt_raw[];
  unsigned char* base = wt_raw + ((1024u - (smem_u32(wt_raw) & 1023u)) & 1023u);
  const int stage_bytes = 2 * WT_AD_BYTES + NB * 128;
  WtCtl* ctl = reinterpret_cast<WtCtl*>(base + (size_t)WT_STAGES * stage_bytes);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int ft = blockIdx.x, n = blockIdx.y, split = blockIdx.z;
  const int tile = n * gridDim.x + ft;
  const int c0 = split * cps, c1 = min(nch, c0 + cps), nloc = max(0, c1 - c0);
  const unsigned cols = NB <= 16 ? 32u : NB <= 32 ? 64u : 128u;  // tensor-memory columns: num and den
  const unsigned idesc = (1u << 4) | (2u << 7) | (2u << 10) | ((unsigned)(NB >> 3) << 17) | ((WT_ROWS >> 4) << 24);
  volatile unsigned* abort_flag = &ctl->abort;

  if (tid == 0) {
    for (int s = 0; s < WT_STAGES; ++s) {
      mbar_init(&ctl->full[s], 1);
      mbar_init(&ctl->empty[s], 1);
    }
    mbar_init(&ctl->done, 1);
    ctl->abort = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&ctl->tmem_base)),
                 "r"(cols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  }
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const unsigned tmem = ctl->tmem_base;

  if (warp == 0) {
    // ---- TMA producer: chunk i of this CTA's frames into stage i % WT_STAGES
    const unsigned tx = (unsigned)stage_bytes;
    int issued = 0;
    for (int i = 0; i < nloc; ++i) {
      const int s = i % WT_STAGES;
      if (i >= WT_STAGES && !mbar_wait_warp(&ctl->empty[s], ((i / WT_STAGES) - 1) & 1, 64)) {
        if (lane == 0) atomicOr(&ctl->abort, 1u);
        break;
      }
      unsigned char* st = base + (size_t)s * stage_bytes;
      const int t0 = (c0 + i) * WT_KC;
      if (elect_one()) {
        mbar_arrive_expect_tx(&ctl->full[s], tx);
        tma_load_3d(st, &map_a, t0, ft * WT_ROWS, n, &ctl->full[s]);
        tma_load_3d(st + WT_AD_BYTES, &map_d, t0, ft * WT_ROWS, n, &ctl->full[s]);
        tma_load_3d(st + 2 * WT_AD_BYTES, &map_h, t0, 0, n, &ctl->full[s]);
      }
      __syncwarp();
      issued = i + 1;
    }
    for (int i = issued > WT_STAGES ? issued - WT_STAGES : 0; i < issued; ++i)
      if (!mbar_wait_warp(&ctl->full[i % WT_STAGES], (i / WT_STAGES) & 1, 64) && lane == 0) atomicOr(&ctl->abort, 1u);
  } else if (warp == 1) {
    // ---- MMA issuer: 4 steps of 8 frames per chunk, A -> num, D -> den
    const unsigned long long d0 = smem_desc_sw128(smem_u32(base));
    for (int i = 0; i < nloc; ++i) {
      const int s = i % WT_STAGES;
      if (!mbar_wait_warp(&ctl->full[s], (i / WT_STAGES) & 1)) {
        if (lane == 0) atomicOr(&ctl->abort, 1u);
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const unsigned long long da = d0 + (unsigned long long)((s * stage_bytes) >> 4);
      if (elect_one()) {
#pragma unroll
        for (int k = 0; k < WT_KC / 8; ++k) {
          const unsigned long long h = da + (unsigned long long)((2 * WT_AD_BYTES) >> 4) + 2 * k;
          const unsigned acc = (i == 0 && k == 0) ? 0u : 1u;
          umma_tf32_id(tmem, da + 2 * k, h, idesc, acc);
          umma_tf32_id(tmem + (unsigned)NB, da + (unsigned long long)(WT_AD_BYTES >> 4) + 2 * k, h, idesc, acc);
        }
        umma_commit(&ctl->empty[s]);
      }
      __syncwarp();
    }
    if (elect_one()) umma_commit(&ctl->done);
    __syncwarp();
  }
  __syncthreads();

  // ---- epilogue: all four warps; thread (warp, lane) owns bin row 32 warp + lane of the tile
  const bool ok = mbar_wait_warp(&ctl->done, 0, 64) && !*abort_flag;
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const int row = warp * 32 + lane, f = ft * WT_ROWS + row;
  float2* pp = part + (((size_t)tile * S + split) * WT_ROWS + row) * NB;
  for (int b0 = 0; b0 < NB; b0 += 16) {
    unsigned hn[16], hd[16];
    const unsigned ta = tmem + ((unsigned)(warp * 32) << 16) + (unsigned)b0;
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15}, [%16];"
        : "=r"(hn[0]), "=r"(hn[1]), "=r"(hn[2]), "=r"(hn[3]), "=r"(hn[4]), "=r"(hn[5]), "=r"(hn[6]), "=r"(hn[7]),
          "=r"(hn[8]), "=r"(hn[9]), "=r"(hn[10]), "=r"(hn[11]), "=r"(hn[12]), "=r"(hn[13]), "=r"(hn[14]),
          "=r"(hn[15])
        : "r"(ta));
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15}, [%16];"
        : "=r"(hd[0]), "=r"(hd[1]), "=r"(hd[2]), "=r"(hd[3]), "=r"(hd[4]), "=r"(hd[5]), "=r"(hd[6]), "=r"(hd[7]),
          "=r"(hd[8]), "=r"(hd[9]), "=r"(hd[10]), "=r"(hd[11]), "=r"(hd[12]), "=r"(hd[13]), "=r"(hd[14]),
          "=r"(hd[15])
        : "r"(ta + (unsigned)NB));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int j = 0; j < 16; ++j)  // an empty split (no frames) contributes zeros
      pp[b0 + j] = (ok && nloc > 0) ? make_float2(__uint_as_float(hn[j]), __uint_as_float(hd[j])) : make_float2(0.f, 0.f);
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(cols) : "memory");
  if (tid == 0) {
    if (!ok) atomicOr(flags + FLAG_TIMEOUT, 1u);
    __threadfence();  // this CTA's parts are released at device scope before its ticket
    ctl->last = (atomicAdd(ticket + tile, 1u) == (unsigned)(S - 1));
    if (ctl->last) __threadfence();
  }
  __syncthreads();
  if (!ctl->last) return;
  if (f < F) {
    const float2* pt = part + ((size_t)tile * S * WT_ROWS + row) * NB;
    for (int b = 0; b < B; ++b) {
      float num = 0.f, den = 0.f;
      for (int q = 0; q < S; ++q) {
        const float2 v = __ldcg(pt + (size_t)q * WT_ROWS * NB + b);
        num += v.x;
        den += v.y;
      }
      if (grad) {
        grad[((size_t)n * F + f) * B + b] = den - num;
      } else {
        float* wp = W + ((size_t)n * F + f) * B + b;
        const float wn = *wp * sqrtf(num / fmaxf(den, eps));
        if (!finitef(wn)) atomicOr(flags + FLAG_NONFINITE, 1u);
        *wp = wn;
      }
    }
  }
  if (tid == 0) ticket[tile] = 0u;
}

// -------------------------------------------------------------- host side
typedef CUresult (*EncodeTiledFnW)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                   const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                   CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

static EncodeTiledFnW encode_fn_w() {
  static EncodeTiledFnW fn = nullptr;
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiledFnW>(p);
  }
  return fn;
}

static void wtc_plan(const dfmnmf_ctx* c, int* S, int* cps, int* nch) {
  const int tiles = ((c->F + WT_ROWS - 1) / WT_ROWS) * c->N;
  *nch = (c->T + WT_KC - 1) / WT_KC;
  int s = (c->num_sms + tiles - 1) / tiles;  // about one CTA per SM
  s = s < 1 ? 1 : (s > WT_MAX_SPLIT ? WT_MAX_SPLIT : s);
  s = s > *nch ? *nch : s;
  *cps = (*nch + s - 1) / s;
  *S = (*nch + *cps - 1) / *cps;
}

size_t wupd_tc_scratch_float2s(const dfmnmf_ctx* c) {
  const int NB = (c->B + 15) & ~15;
  return (size_t)((c->F + WT_ROWS - 1) / WT_ROWS) * c->N * WT_MAX_SPLIT * WT_ROWS * NB;
}
size_t wupd_tc_ticket_count(const dfmnmf_ctx* c) { return (size_t)((c->F + WT_ROWS - 1) / WT_ROWS) * c->N; }

cudaError_t launch_wupd_tc(const dfmnmf_ctx* c, cudaStream_t s, float* grad) {
  EncodeTiledFnW fn = encode_fn_w();
  if (!fn || !c->wtc_part) return cudaErrorNotSupported;
  const int NB = (c->B + 15) & ~15;
  int S, cps, nch;
  wtc_plan(c, &S, &cps, &nch);
  CUtensorMap ma, md, mh;
  const cuuint32_t e3[3] = {1, 1, 1};
  const cuuint64_t dad[3] = {(cuuint64_t)c->Tp, (cuuint64_t)c->F, (cuuint64_t)c->N};
  const cuuint64_t sad[2] = {(cuuint64_t)c->Tp * 4, (cuuint64_t)c->F * c->Tp * 4};
  const cuuint32_t bad[3] = {WT_KC, WT_ROWS, 1};
  const cuuint64_t dh[3] = {(cuuint64_t)c->Tp, (cuuint64_t)c->B, (cuuint64_t)c->N};
  const cuuint64_t sh[2] = {(cuuint64_t)c->Tp * 4, (cuuint64_t)c->B * c->Tp * 4};
  const cuuint32_t bh[3] = {WT_KC, (cuuint32_t)NB, 1};
  if (fn(&ma, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, c->A, dad, sad, bad, e3, CU_TENSOR_MAP_INTERLEAVE_NONE,
         CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS ||
      fn(&md, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, c->D, dad, sad, bad, e3, CU_TENSOR_MAP_INTERLEAVE_NONE,
         CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS ||
      fn(&mh, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, c->H, dh, sh, bh, e3, CU_TENSOR_MAP_INTERLEAVE_NONE,
         CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
    return cudaErrorInvalidValue;
  const size_t smem = 1024 + (size_t)WT_STAGES * (2 * WT_AD_BYTES + NB * 128) + sizeof(WtCtl);
  cudaError_t e = cudaFuncSetAttribute(k_wupd_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  dim3 grid((c->F + WT_ROWS - 1) / WT_ROWS, c->N, S);
  k_wupd_tc<<<grid, 128, smem, s>>>(ma, md, mh, c->W, c->F, c->B, NB, c->eps, c->flags, S, cps, nch,
                                    reinterpret_cast<float2*>(c->wtc_part), c->wtc_ticket, grad);
  return cudaGetLastError();
}

}  // namespace dfm
