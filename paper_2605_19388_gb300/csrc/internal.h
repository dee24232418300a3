// internal.h -- library context and kernel launchers (not part of the ABI).
#pragma once
#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

struct dfmnmf_ctx {
  // sizes
  int F, T, K, MK, M, N, B;
  int Tp;               // row stride of lambda, A and D: T rounded up to a multiple of 4 (zero tail)
  int Tr;               // row length of the tensor-core operands: T rounded up to 64 (zero tail)
  int precision, ip_arith;
  float eps;            // floor of Sec. IV-A
  float singular_rtol;  // relative pivot / singular-value cut-off of the IP solve
  int device;
  int num_sms;          // multiprocessors of the device
  // launch shapes (dfmnmf_autotune): per-frequency kernels on 1 or 2 graph
  // branches, and the CTAs per SM the split NMF products aim for
  int cfg_branches;
  int cfg_nmf_ctas;
  // state and buffers (device)
  float2* x;       // [F][T][M]
  double2* Q64;    // [F][K*MK*MK]   master copy
  float2* Q32;     // [F][K*MK*MK]   single-precision copy used by the streaming kernels
  float2* Qinv32;  // [F][K*MK*MK]   inverse blocks (Wiener filter)
  double2* V;      // [F][K][MK][MK][MK]  (FP64: float-float accumulated)
  float4* Vdd;     // same entries as float pairs (re hi, re lo, im hi, im lo) for the IP kernel
  float* W;        // [N][F][B]
  float* H;        // [N][B][Tp]  (zero tail; the ABI layout [N][B][T] is converted on copy)
  float* g;        // [F][N][M]
  float* lam;      // [N][F][Tp]
  float* P;        // [F][T][M]
  float* A;        // [N][F][Tp]
  float* D;        // [N][F][Tp]
  double* red;     // loglik partial sums
  float* nmf_part;       // split-reduction partials of the NMF updates
  unsigned* nmf_ticket;  // per-tile tickets of the split reductions (self-resetting)
  double* nll_dev; // 1 double
  // gradient of Eq. (12) (dfmnmf_cost_gradient), allocated on first use
  double2* gQ;
  float *gW, *gH, *gg;
  unsigned* flags; // dfm::FLAG_COUNT words
  // tensor-core form (k_vtc): FP32 partial sums of tiles shared by two CTAs and one ticket per tile
  float4* tc_part;
  unsigned* tc_ticket;
  float2* wtc_part;    // tensor-core forms: FP32 parts of the W-update products (k_wupd_tc) ...
  unsigned* wtc_ticket;  // ... and one ticket per (source, 128-bin tile)
  int smem_optin;      // opt-in shared memory per block of the device
  int cfg_vx_groups;   // converter warp groups of k_vtc (1 or 2)
  int cfg_wupd_tc;     // tensor-core forms: W-update products on the tensor cores (k_wupd_tc) when 1
  unsigned wait_cycles;  // budget of the pipeline waits of the tensor-core covariance kernel
  size_t red_len;
  // CUDA graph of one iteration, captured on first use
  cudaStream_t cap_stream;
  cudaGraph_t graph;
  cudaGraphExec_t gexec;
  int launches_per_iter;
  cudaStream_t side_stream;   // second branch of the captured iteration
  cudaEvent_t fork_ev, join_ev;
};

namespace dfm {

// The tensor-core forms (bfloat16 or TF32 split operands of the covariance contraction).
inline bool is_tc(int precision) { return precision == 1 || precision == 2; }

// All launchers return cudaGetLastError() after enqueueing.
cudaError_t launch_lambda(const dfmnmf_ctx* c, cudaStream_t s);
// Launchers of the per-frequency kernels take a frequency range [fb, fb + fc).
cudaError_t launch_cov(const dfmnmf_ctx* c, cudaStream_t s, int fb, int fc);
cudaError_t launch_vtc(const dfmnmf_ctx* c, cudaStream_t s, int fb, int fc);  // tensor-core covariances (BF16_TC form)
bool tc_supported(int MK, int K);
size_t tc_part_float4s(const dfmnmf_ctx* c);   // partial-sum slots of launch_vtc (float4 each)
size_t tc_ticket_count(const dfmnmf_ctx* c);   // tickets of launch_vtc
int tc_raw_stages(const dfmnmf_ctx* c);        // raw stages of k_vtc that fit in shared memory (0: none)
cudaError_t launch_ip(const dfmnmf_ctx* c, cudaStream_t s, int fb, int fc);
cudaError_t launch_power_stats(const dfmnmf_ctx* c, cudaStream_t s, int fb, int fc);  // P + A/D (current lambda)
// The NMF updates take `grad`: NULL updates the factor (Eq. 8, 9 or 10);
// otherwise the gradient of Eq. (12) with respect to it (den - num of the
// rule) is written there and the factor is left unchanged.
cudaError_t launch_wupd(const dfmnmf_ctx* c, cudaStream_t s, float* grad = nullptr);  // Eq. 8
cudaError_t launch_wlam(const dfmnmf_ctx* c, cudaStream_t s);  // Eq. 8 and the Eq. 2 refresh, one launch
bool wlam_supported(const dfmnmf_ctx* c);  // its shared-memory tile fits (B Tp + 16 Tp floats)
cudaError_t launch_wupd_tc(const dfmnmf_ctx* c, cudaStream_t s, float* grad = nullptr);  // Eq. 8, tcgen05 TF32
size_t wupd_tc_scratch_float2s(const dfmnmf_ctx* c);
size_t wupd_tc_ticket_count(const dfmnmf_ctx* c);
cudaError_t launch_stats(const dfmnmf_ctx* c, cudaStream_t s);        // A/D from stored P
cudaError_t launch_hupd(const dfmnmf_ctx* c, cudaStream_t s, float* grad = nullptr);  // Eq. 9
cudaError_t launch_gupd(const dfmnmf_ctx* c, cudaStream_t s, float* grad = nullptr);  // Eq. 10
cudaError_t launch_power_stats_comp(const dfmnmf_ctx* c, cudaStream_t s);  // P (compensated) + A/D, band-wide
// P + A/D with TMA tiles (4 subarrays of 4 microphones, N <= 16); comp: compensated projections
bool pstats_tma_supported(int K, int MK, int N);
cudaError_t launch_pstats_tma(const dfmnmf_ctx* c, cudaStream_t s, int fb, int fc, bool comp);
cudaError_t launch_qgrad(const dfmnmf_ctx* c, double2* dQ, cudaStream_t s);  // d Eq. 12 / d Q from V and Q
cudaError_t launch_loglik(const dfmnmf_ctx* c, cudaStream_t s);       // Eq. 12 -> c->nll_dev
cudaError_t launch_logdet(const dfmnmf_ctx* c, double* out, cudaStream_t s);  // ln|det Q_fk|^2 per block
cudaError_t launch_qinv(const dfmnmf_ctx* c, cudaStream_t s);
cudaError_t launch_separate(const dfmnmf_ctx* c, float2* out, cudaStream_t s);
cudaError_t launch_q_convert(const dfmnmf_ctx* c, cudaStream_t s);    // Q64 -> Q32
// initialisation from source images (Sec. IV-A, steps 3, 5, 6): R scratch
// [N][F][M][M] FP64, Linv scratch [N][F][M][M]; h may be NULL
bool init_supported(int M, int MK);
cudaError_t launch_init_from_images(dfmnmf_ctx* c, const float2* cimg, double2* R, float2* Linv, float* h,
                                    cudaStream_t s);

// Record the message returned by dfmnmf_last_error() on this thread.
void set_last_error(const char* msg);

size_t nmf_scratch_floats(const dfmnmf_ctx* c);
size_t nmf_ticket_count(const dfmnmf_ctx* c);

}  // namespace dfm
