// internal.h -- library context and kernel launchers (not part of the ABI).
#pragma once
#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

struct dfmnmf_ctx {
  // sizes
  int F, T, K, MK, M, N, B;
  int precision, ip_arith;
  float eps;            // floor of Sec. IV-A
  float singular_rtol;  // relative pivot / singular-value cut-off of the IP solve
  int device;
  // state and buffers (device)
  float2* x;       // [F][T][M]
  double2* Q64;    // [F][K*MK*MK]   master copy
  float2* Q32;     // [F][K*MK*MK]   single-precision copy used by the streaming kernels
  float2* Qinv32;  // [F][K*MK*MK]   inverse blocks (Wiener filter)
  double2* V;      // [F][K][MK][MK][MK]  (FP64: float-float accumulated)
  float* W;        // [N][F][B]
  float* H;        // [N][B][T]
  float* g;        // [F][N][M]
  float* lam;      // [N][F][T]
  float* P;        // [F][T][M]
  float* A;        // [N][F][T]
  float* D;        // [N][F][T]
  double* red;     // loglik partial sums
  double* nll_dev; // 1 double
  unsigned* flags; // dfm::FLAG_COUNT words
  size_t red_len;
  // CUDA graph of one iteration, captured on first use
  cudaStream_t cap_stream;
  cudaGraph_t graph;
  cudaGraphExec_t gexec;
  int launches_per_iter;
};

namespace dfm {

// All launchers return cudaGetLastError() after enqueueing.
cudaError_t launch_lambda(const dfmnmf_ctx* c, cudaStream_t s);
cudaError_t launch_cov(const dfmnmf_ctx* c, cudaStream_t s);
cudaError_t launch_ip(const dfmnmf_ctx* c, cudaStream_t s);
cudaError_t launch_power_stats(const dfmnmf_ctx* c, cudaStream_t s);  // P + A/D (current lambda)
cudaError_t launch_wupd(const dfmnmf_ctx* c, cudaStream_t s);         // Eq. 8 + lambda
cudaError_t launch_stats(const dfmnmf_ctx* c, cudaStream_t s);        // A/D from stored P
cudaError_t launch_hupd(const dfmnmf_ctx* c, cudaStream_t s);         // Eq. 9 + lambda
cudaError_t launch_gupd(const dfmnmf_ctx* c, cudaStream_t s);         // Eq. 10
cudaError_t launch_loglik(const dfmnmf_ctx* c, cudaStream_t s);       // Eq. 12 -> c->nll_dev
cudaError_t launch_qinv(const dfmnmf_ctx* c, cudaStream_t s);
cudaError_t launch_separate(const dfmnmf_ctx* c, float2* out, cudaStream_t s);
cudaError_t launch_q_convert(const dfmnmf_ctx* c, cudaStream_t s);    // Q64 -> Q32

// Record the message returned by dfmnmf_last_error() on this thread.
void set_last_error(const char* msg);

// Whether the NMF update kernels refresh lambda themselves (else a separate
// lambda launch follows them).
bool nmf_fused_lambda(const dfmnmf_ctx* c);

}  // namespace dfm
