// noalloc.cu -- the negative log-likelihood of Eq. (12) without any device
// allocation (dfmnmf_loglik_noalloc).
//
// Who needs this: callers that are not allowed to allocate device memory at
// the point where they want the cost, for example an audio engine's
// real-time thread (cudaMalloc may block and implicitly synchronise the whole
// device, which breaks its deadline) or a plug-in whose host application owns
// the GPU memory budget and forbids allocations by guests.  They already hold
// x, Q, W, H and g in device memory and only want one number back.
//
// The regular path keeps its partial sums in buffers that dfmnmf_init
// allocates.  Here the same partial sums (one per CTA of the data term, one
// per diagonaliser block for the log-determinants, and the result) live in a
// file-scope __device__ array of DFMNMF_NOALLOC_SCRATCH_DOUBLES doubles that
// every GPU loading this library holds until the process exits.  Host code
// must not use the array's name as a device address (on the host it is only a
// stand-in symbol): the device address is asked of the runtime with
// cudaGetSymbolAddress, with the device current, and cached per CUDA context.
// The cache key is the context's unique id (cuCtxGetId), not the device
// number: after a device reset, or with another context current on the same
// device, the module is loaded anew and the array may sit elsewhere, so a new
// id means a new lookup.  The first call in a context does that set-up (under
// lazy module loading it is also where the module is loaded and the array
// backed); later calls find the address without taking a lock.  All calls
// share the one array: every entry a call reads is written earlier by the
// same call, so nothing has to be cleared, but two calls whose work overlaps
// on the GPU (different streams, no ordering between them) race on it.
#include <cuda.h>
#include <float.h>
#include <math.h>

#include <atomic>
#include <mutex>

#include "../../include/dfmnmf.h"
#include "common.cuh"
#include "internal.h"
#include "noalloc_cache.h"
#include <stdio.h>

namespace {

constexpr int kScratch = DFMNMF_NOALLOC_SCRATCH_DOUBLES;
constexpr int kNMax = 16;

static __device__ __align__(256) double g_nll_scratch[kScratch];

std::mutex g_scratch_mu;                          // serialises set-ups (inserts), never lookups
dfm::ScratchCache<double*, 64> g_scratch_cache;   // context id -> device address of g_nll_scratch

// Data term of Eq. (12) for one (f, 128-frame chunk): lambda is formed from W
// and H on the fly, P from the compensated projection Q x.
template <int MK>
__global__ void __launch_bounds__(128) k_na_data(const float2* __restrict__ x, const double2* __restrict__ Q64,
                                                 const float* __restrict__ W, const float* __restrict__ H,
                                                 const float* __restrict__ g, double* __restrict__ part, int F,
                                                 int T, int K, int N, int B, float eps) {
  extern __shared__ float sm[];
  const int M = K * MK;
  const int f = blockIdx.x;
  float* gs = sm;                                                    // [N][M]
  float* ws = gs + N * M;                                            // [N][B]
  float2* Qh = reinterpret_cast<float2*>(sm + ((N * M + N * B + 1) & ~1));  // [K][MK][MK] high parts
  float2* Ql = Qh + K * MK * MK;                                     // low parts
  __shared__ double wsum[4];
  for (int i = threadIdx.x; i < N * M; i += blockDim.x) gs[i] = g[(size_t)f * N * M + i];
  for (int i = threadIdx.x; i < N * B; i += blockDim.x) {
    const int n = i / B, b = i % B;
    ws[i] = W[((size_t)n * F + f) * B + b];
  }
  for (int i = threadIdx.x; i < K * MK * MK; i += blockDim.x)
    dfm::split_c(Q64[(size_t)f * K * MK * MK + i], Qh[i], Ql[i]);
  __syncthreads();
  const int t = blockIdx.y * blockDim.x + threadIdx.x;
  double acc = 0.0;
  if (t < T) {
    float lr[kNMax];
#pragma unroll
    for (int n = 0; n < kNMax; ++n) {
      float s = 0.f;
      if (n < N)
        for (int b = 0; b < B; ++b) s = fmaf(ws[n * B + b], H[((size_t)n * B + b) * T + t], s);
      lr[n] = s;
    }
    for (int k = 0; k < K; ++k) {
      float2 xv[MK];
#pragma unroll
      for (int nu = 0; nu < MK; ++nu) xv[nu] = x[((size_t)f * T + t) * M + k * MK + nu];
      float s = 0.f;
#pragma unroll
      for (int mu = 0; mu < MK; ++mu) {
        const float2 yv = dfm::cdot2<MK>(Qh + (k * MK + mu) * MK, Ql + (k * MK + mu) * MK, xv);
        const float p = fmaf(yv.x, yv.x, yv.y * yv.y);
        float ys = 0.f;
#pragma unroll
        for (int n = 0; n < kNMax; ++n)
          if (n < N) ys = fmaf(lr[n], gs[n * M + k * MK + mu], ys);
        ys = fmaxf(ys, eps);
        s += p / ys + logf(ys);
      }
      acc += (double)s;
    }
  }
  acc = dfm::warp_sum_d(acc);
  if ((threadIdx.x & 31) == 0) wsum[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) part[(size_t)f * gridDim.y + blockIdx.y] = (wsum[0] + wsum[1]) + (wsum[2] + wsum[3]);
}

// ln |det Q_fk|^2 by FP64 Gaussian elimination with partial pivoting.
template <int MK>
__global__ void k_na_logdet(const double2* __restrict__ Q64, double* __restrict__ out, int nblocks) {
  const int blk = blockIdx.x * blockDim.x + threadIdx.x;
  if (blk >= nblocks) return;
  double ar[MK][MK], ai[MK][MK];
  for (int r = 0; r < MK; ++r)
    for (int c = 0; c < MK; ++c) {
      const double2 v = Q64[(size_t)blk * MK * MK + r * MK + c];
      ar[r][c] = v.x;
      ai[r][c] = v.y;
    }
  double acc = 0.0;
  for (int c = 0; c < MK; ++c) {
    int p = c;
    double best = ar[c][c] * ar[c][c] + ai[c][c] * ai[c][c];
    for (int r = c + 1; r < MK; ++r) {
      const double m = ar[r][c] * ar[r][c] + ai[r][c] * ai[r][c];
      if (m > best) { best = m; p = r; }
    }
    for (int q = 0; q < MK && p != c; ++q) {
      double tr = ar[c][q]; ar[c][q] = ar[p][q]; ar[p][q] = tr;
      tr = ai[c][q]; ai[c][q] = ai[p][q]; ai[p][q] = tr;
    }
    acc += log(best);
    if (!(best > 0.0)) continue;
    for (int r = c + 1; r < MK; ++r) {
      const double mr = (ar[r][c] * ar[c][c] + ai[r][c] * ai[c][c]) / best;
      const double mi = (ai[r][c] * ar[c][c] - ar[r][c] * ai[c][c]) / best;
      for (int q = c; q < MK; ++q) {
        ar[r][q] -= mr * ar[c][q] - mi * ai[c][q];
        ai[r][q] -= mr * ai[c][q] + mi * ar[c][q];
      }
    }
  }
  out[blk] = acc;
}

// result = sum(data partials) - T * sum(log-dets), fixed summation order.
__global__ void __launch_bounds__(256) k_na_final(const double* __restrict__ part, int npart,
                                                  const double* __restrict__ logdet, int nld, int T,
                                                  double* __restrict__ out) {
  __shared__ double sd[256], sl[256];
  double a = 0.0, b = 0.0;
  for (int i = threadIdx.x; i < npart; i += 256) a += part[i];
  for (int i = threadIdx.x; i < nld; i += 256) b += logdet[i];
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
  if (threadIdx.x == 0) *out = sd[0] - (double)T * sl[0];
}

int fail(int code, const char* msg) {
  dfm::set_last_error(msg);
  return code;
}

typedef CUresult (*CtxGetCurrentFn)(CUcontext*);
typedef CUresult (*CtxGetIdFn)(CUcontext, unsigned long long*);

// Unique id of the CUDA context current on this thread; 0 if none is current
// yet (the runtime makes the device's primary context current on first use)
// or the driver cannot tell.
unsigned long long current_context_id() {
  static std::atomic<CtxGetCurrentFn> get_cur{nullptr};
  static std::atomic<CtxGetIdFn> get_id{nullptr};
  CtxGetCurrentFn gc = get_cur.load(std::memory_order_acquire);
  CtxGetIdFn gi = get_id.load(std::memory_order_acquire);
  if (!gc || !gi) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &p, 12000, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess || !p)
      return 0;
    gc = reinterpret_cast<CtxGetCurrentFn>(p);
    if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &p, 12000, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess || !p)
      return 0;
    gi = reinterpret_cast<CtxGetIdFn>(p);
    get_cur.store(gc, std::memory_order_release);
    get_id.store(gi, std::memory_order_release);
  }
  CUcontext ctx = nullptr;
  unsigned long long id = 0;
  if (gc(&ctx) != CUDA_SUCCESS || !ctx || gi(ctx, &id) != CUDA_SUCCESS) return 0;
  return id;
}

// Device address of g_nll_scratch in the current context: a lock-free cache
// hit, or the set-up (cudaGetSymbolAddress with the device current) whose
// result is cached under the context's id.
int scratch_address(double** out) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    return fail(DFMNMF_ECUDA, "dfmnmf_loglik_noalloc: no CUDA device");
  }
  unsigned long long id = current_context_id();
  if (id != 0 && g_scratch_cache.find(id, out)) return DFMNMF_OK;
  std::lock_guard<std::mutex> lock(g_scratch_mu);
  if (id != 0 && g_scratch_cache.find(id, out)) return DFMNMF_OK;
  void* p = nullptr;
  const cudaError_t e = cudaGetSymbolAddress(&p, g_nll_scratch);
  if (e != cudaSuccess || !p) {
    cudaGetLastError();
    char msg[256];
    snprintf(msg, sizeof msg, "dfmnmf_loglik_noalloc: cudaGetSymbolAddress failed: %s", cudaGetErrorString(e));
    return fail(DFMNMF_ECUDA, msg);
  }
  if (id == 0) id = current_context_id();  // the lookup made the primary context current
  if (id != 0) g_scratch_cache.insert(id, static_cast<double*>(p));  // a full table only stops caching
  *out = static_cast<double*>(p);
  return DFMNMF_OK;
}

}  // namespace

extern "C" int dfmnmf_loglik_noalloc(const dfmnmf_desc* d, const void* x_dev, const void* Q_dev,
                                     const float* W_dev, const float* H_dev, const float* g_dev,
                                     double* nll_host, void* stream) {
  if (!d || !x_dev || !Q_dev || !W_dev || !H_dev || !g_dev || !nll_host)
    return fail(DFMNMF_EINVAL, "dfmnmf_loglik_noalloc: null argument");
  if (d->F < 1 || d->T < 1 || d->K < 1 || d->N < 1 || d->B < 1 || !d->mics)
    return fail(DFMNMF_EINVAL, "dfmnmf_loglik_noalloc: sizes must be positive");
  if (d->F > 65535 || d->K > 16 || d->N > kNMax || d->B > 64)
    return fail(DFMNMF_EINVAL, "dfmnmf_loglik_noalloc: limits F <= 65535, K <= 16, N <= 16, B <= 64");
  const int MK = d->mics[0];
  for (int k = 0; k < d->K; ++k)
    if (d->mics[k] != MK || MK < 1 || MK > 4)
      return fail(DFMNMF_EINVAL, "dfmnmf_loglik_noalloc: subarrays must all have the same size M_k in 1..4");
  const int ty = (d->T + 127) / 128;
  const long long need = (long long)d->F * ty + (long long)d->F * d->K + 1;
  if (need > kScratch) {
    char msg[256];
    snprintf(msg, sizeof msg,
             "dfmnmf_loglik_noalloc: F*ceil(T/128) + F*K + 1 = %lld scratch doubles exceeds the maximum %d",
             need, kScratch);
    return fail(DFMNMF_EINVAL, msg);
  }
  double* scratch = nullptr;
  int r = scratch_address(&scratch);
  if (r) return r;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  const float eps = fmaxf((float)(d->floor_eps > 0 ? d->floor_eps : 1e-6), FLT_MIN);  // as dfmnmf_init
  const int F = d->F, T = d->T, K = d->K, N = d->N, B = d->B, M = K * MK;
  double* part = scratch;
  double* logdet = scratch + (size_t)F * ty;
  double* result = logdet + (size_t)F * K;
  const size_t smem = (size_t)((N * B + N * M + 1) & ~1) * sizeof(float) + 2 * (size_t)K * MK * MK * sizeof(float2);
  const float2* x = static_cast<const float2*>(x_dev);
  const double2* Q = static_cast<const double2*>(Q_dev);
  auto launch = [&]() -> cudaError_t {
    DFM_MK_DISPATCH(MK, {
      k_na_data<MK_><<<dim3(F, ty), 128, smem, s>>>(x, Q, W_dev, H_dev, g_dev, part, F, T, K, N, B, eps);
      k_na_logdet<MK_><<<(F * K + 127) / 128, 128, 0, s>>>(Q, logdet, F * K);
    });
    k_na_final<<<1, 256, 0, s>>>(part, F * ty, logdet, F * K, T, result);
    return cudaGetLastError();
  };
  cudaError_t e = launch();
  double v = 0.0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&v, result, sizeof(double), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) {
    char msg[256];
    snprintf(msg, sizeof msg, "dfmnmf_loglik_noalloc: %s", cudaGetErrorString(e));
    return fail(DFMNMF_ECUDA, msg);
  }
  *nll_host = v;
  if (!isfinite(v)) return fail(DFMNMF_ENUMERIC, "dfmnmf_loglik_noalloc: the cost is not finite");
  return DFMNMF_OK;
}
