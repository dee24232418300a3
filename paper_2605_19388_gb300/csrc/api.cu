// api.cu -- the C ABI of include/dfmnmf.h: argument checks, device state,
// the iteration schedule and its CUDA graph.
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <string>

#include <float.h>

#include "../../include/dfmnmf.h"
#include "common.cuh"
#include "internal.h"

struct dfmnmf_batch {
  int count, device;
  cudaGraph_t graph;       // one child graph (a context's iteration) per mixture, no edges
  cudaGraphExec_t gexec;
};

namespace {

thread_local std::string g_last_error;

int fail(int code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  g_last_error = buf;
  return code;
}

#define CK(call)                                                                          \
  do {                                                                                    \
    cudaError_t e_ = (call);                                                              \
    if (e_ != cudaSuccess)                                                                \
      return fail(DFMNMF_ECUDA, "%s failed: %s (%s:%d)", #call, cudaGetErrorString(e_), __FILE__, __LINE__); \
  } while (0)

cudaStream_t as_stream(void* s) { return reinterpret_cast<cudaStream_t>(s); }

__global__ void k_identity_blocks(double2* Q, int F, int K, int MK) {
  const size_t n = (size_t)F * K * MK * MK;
  const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int e = (int)(i % (size_t)(MK * MK));
  Q[i] = make_double2((e / MK == e % MK) ? 1.0 : 0.0, 0.0);
}

void free_ctx(dfmnmf_ctx* c) {
  if (!c) return;
  if (c->gexec) cudaGraphExecDestroy(c->gexec);
  if (c->graph) cudaGraphDestroy(c->graph);
  if (c->cap_stream) cudaStreamDestroy(c->cap_stream);
  if (c->side_stream) cudaStreamDestroy(c->side_stream);
  if (c->fork_ev) cudaEventDestroy(c->fork_ev);
  if (c->join_ev) cudaEventDestroy(c->join_ev);
  void* ptrs[] = {c->x, c->Q64, c->Q32, c->Qinv32, c->V, c->Vdd, c->W, c->H, c->g, c->lam,
                  c->P, c->A, c->D, c->red, c->nll_dev, c->flags, c->nmf_part, c->nmf_ticket, c->tc_part, c->tc_ticket, c->wtc_part, c->wtc_ticket, c->gQ, c->gW, c->gH, c->gg};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  delete c;
}

template <class T>
int dalloc(T** p, size_t count, const char* what) {
  cudaError_t e = cudaMalloc(reinterpret_cast<void**>(p), count * sizeof(T) + 16);
  if (e != cudaSuccess) {
    *p = nullptr;
    cudaGetLastError();
    return fail(DFMNMF_ENOMEM, "cudaMalloc of %s (%zu bytes) failed: %s", what, count * sizeof(T),
                cudaGetErrorString(e));
  }
  return DFMNMF_OK;
}

bool is_host_ptr(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return true;
  }
  return a.type == cudaMemoryTypeHost || a.type == cudaMemoryTypeUnregistered;
}

size_t nQ(const dfmnmf_ctx* c) { return (size_t)c->F * c->K * c->MK * c->MK; }
size_t nW(const dfmnmf_ctx* c) { return (size_t)c->N * c->F * c->B; }
size_t nH(const dfmnmf_ctx* c) { return (size_t)c->N * c->B * c->Tp; }
// copy H between the ABI layout [N][B][T] and the padded internal one
cudaError_t copy_H(dfmnmf_ctx* c, void* dst, const void* src, bool to_internal, cudaStream_t s) {
  const size_t w = (size_t)c->T * sizeof(float), pitch = (size_t)c->Tp * sizeof(float);
  return to_internal ? cudaMemcpy2DAsync(dst, pitch, src, w, w, (size_t)c->N * c->B, cudaMemcpyDefault, s)
                     : cudaMemcpy2DAsync(dst, w, src, pitch, w, (size_t)c->N * c->B, cudaMemcpyDefault, s);
}
size_t ng(const dfmnmf_ctx* c) { return (size_t)c->F * c->N * c->M; }
size_t nx(const dfmnmf_ctx* c) { return (size_t)c->F * c->T * c->M; }

// The launches of one iteration in order; stage s is the range of entries
// with stage == s.  `ranged` launches are per frequency and take a frequency
// range; the captured iteration runs them for two halves of the band on two
// branches so that the latency-bound IP of one half overlaps the streaming
// kernels of the other.
typedef cudaError_t (*LaunchFn)(const dfmnmf_ctx*, cudaStream_t, int, int);
struct Launch {
  int stage;
  const char* name;
  LaunchFn fn;
  bool ranged;
};

int iteration_launches(const dfmnmf_ctx* c, Launch* out) {
  int n = 0;
  if (dfm::is_tc(c->precision)) out[n++] = {DFMNMF_STAGE_COV, "k_vtc", dfm::launch_vtc, true};
  else out[n++] = {DFMNMF_STAGE_COV, "k_cov", dfm::launch_cov, true};
  out[n++] = {DFMNMF_STAGE_IP, "k_ip", dfm::launch_ip, true};
  out[n++] = {DFMNMF_STAGE_W, "k_pstats", dfm::launch_power_stats, true};
  if ((dfm::is_tc(c->precision) && c->cfg_wupd_tc) || !dfm::wlam_supported(c)) {
    if (dfm::is_tc(c->precision) && c->cfg_wupd_tc)
      out[n++] = {DFMNMF_STAGE_W, "k_wupd_tc", [](const dfmnmf_ctx* c, cudaStream_t s, int, int) { return dfm::launch_wupd_tc(c, s); }, false};
    else
      out[n++] = {DFMNMF_STAGE_W, "k_wupd", [](const dfmnmf_ctx* c, cudaStream_t s, int, int) { return dfm::launch_wupd(c, s); }, false};
    out[n++] = {DFMNMF_STAGE_W, "k_lambda", [](const dfmnmf_ctx* c, cudaStream_t s, int, int) { return dfm::launch_lambda(c, s); }, false};
  } else {
    out[n++] = {DFMNMF_STAGE_W, "k_wlam", [](const dfmnmf_ctx* c, cudaStream_t s, int, int) { return dfm::launch_wlam(c, s); }, false};
  }
  out[n++] = {DFMNMF_STAGE_H, "k_stats", [](const dfmnmf_ctx* c, cudaStream_t s, int, int) { return dfm::launch_stats(c, s); }, false};
  out[n++] = {DFMNMF_STAGE_H, "k_hupd", [](const dfmnmf_ctx* c, cudaStream_t s, int, int) { return dfm::launch_hupd(c, s); }, false};
  out[n++] = {DFMNMF_STAGE_H, "k_lambda", [](const dfmnmf_ctx* c, cudaStream_t s, int, int) { return dfm::launch_lambda(c, s); }, false};
  out[n++] = {DFMNMF_STAGE_G, "k_gupd", [](const dfmnmf_ctx* c, cudaStream_t s, int, int) { return dfm::launch_gupd(c, s); }, false};
  return n;
}
constexpr int kMaxLaunches = 16;

int enqueue_stage(dfmnmf_ctx* c, int stage, cudaStream_t s) {
  if (stage < DFMNMF_STAGE_COV || stage > DFMNMF_STAGE_G) return fail(DFMNMF_EINVAL, "unknown stage %d", stage);
  Launch L[kMaxLaunches];
  const int n = iteration_launches(c, L);
  for (int i = 0; i < n; ++i)
    if (L[i].stage == stage) {
      cudaError_t e = L[i].fn(c, s, 0, c->F);
      if (e != cudaSuccess) return fail(DFMNMF_ECUDA, "launch of %s failed: %s", L[i].name, cudaGetErrorString(e));
    }
  return DFMNMF_OK;
}

// Split point of the band: a multiple of 8 frequencies.  The tensor-core
// form is not split: its covariance kernel is persistent over the whole band
// and its partial-sum slots serve one launch at a time.
int band_split(const dfmnmf_ctx* c) {
  if (c->cfg_branches == 1 || dfm::is_tc(c->precision)) return 0;
  const int h = ((c->F / 2) + 7) & ~7;
  return (h > 0 && h < c->F) ? h : 0;
}

// One iteration for capture: ranged launches for both halves on two branches,
// joined before the first band-wide launch.
int enqueue_iteration(dfmnmf_ctx* c, cudaStream_t s) {
  Launch L[kMaxLaunches];
  const int n = iteration_launches(c, L);
  const int h = band_split(c);
  int i = 0;
  if (h > 0) {
    CK(cudaEventRecord(c->fork_ev, s));
    CK(cudaStreamWaitEvent(c->side_stream, c->fork_ev, 0));
    for (; i < n && L[i].ranged; ++i) {
      cudaError_t e = L[i].fn(c, s, 0, h);
      if (e == cudaSuccess) e = L[i].fn(c, c->side_stream, h, c->F - h);
      if (e != cudaSuccess) return fail(DFMNMF_ECUDA, "launch of %s failed: %s", L[i].name, cudaGetErrorString(e));
    }
    CK(cudaEventRecord(c->join_ev, c->side_stream));
    CK(cudaStreamWaitEvent(s, c->join_ev, 0));
  }
  for (; i < n; ++i) {
    cudaError_t e = L[i].fn(c, s, 0, c->F);
    if (e != cudaSuccess) return fail(DFMNMF_ECUDA, "launch of %s failed: %s", L[i].name, cudaGetErrorString(e));
  }
  return DFMNMF_OK;
}

int ensure_graph(dfmnmf_ctx* c) {
  if (c->gexec) return DFMNMF_OK;
  CK(cudaStreamBeginCapture(c->cap_stream, cudaStreamCaptureModeThreadLocal));
  int r = enqueue_iteration(c, c->cap_stream);
  cudaGraph_t graph = nullptr;
  cudaError_t e = cudaStreamEndCapture(c->cap_stream, &graph);
  if (r) {
    if (graph) cudaGraphDestroy(graph);
    return r;
  }
  if (e != cudaSuccess) return fail(DFMNMF_ECUDA, "graph capture failed: %s", cudaGetErrorString(e));
  c->graph = graph;
  CK(cudaGraphInstantiate(&c->gexec, c->graph, 0));
  size_t nodes = 0;
  CK(cudaGraphGetNodes(c->graph, nullptr, &nodes));
  c->launches_per_iter = (int)nodes;
  return DFMNMF_OK;
}

void drop_graph(dfmnmf_ctx* c) {
  if (c->gexec) cudaGraphExecDestroy(c->gexec);
  if (c->graph) cudaGraphDestroy(c->graph);
  c->gexec = nullptr;
  c->graph = nullptr;
}

int refresh_derived(dfmnmf_ctx* c, cudaStream_t s) {
  CK(dfm::launch_lambda(c, s));
  CK(dfm::launch_q_convert(c, s));
  return DFMNMF_OK;
}

}  // namespace

void dfm::set_last_error(const char* msg) { g_last_error = msg ? msg : ""; }

extern "C" {

int dfmnmf_version(void) { return DFMNMF_VERSION; }

const char* dfmnmf_last_error(void) { return g_last_error.c_str(); }

int dfmnmf_init(dfmnmf_ctx** out, const dfmnmf_desc* d, const void* x, const float* W0, const float* H0,
                const float* g0, const void* Q0, void* stream) {
  g_last_error.clear();
  if (!out || !d) return fail(DFMNMF_EINVAL, "null context or descriptor");
  *out = nullptr;
  if (!x || !W0 || !H0 || !g0) return fail(DFMNMF_EINVAL, "x, W0, H0 and g0 are required");
  if (d->F < 1 || d->T < 1 || d->K < 1 || d->N < 1 || d->B < 1)
    return fail(DFMNMF_EINVAL, "sizes must be positive (F=%d T=%d K=%d N=%d B=%d)", d->F, d->T, d->K, d->N, d->B);
  if (d->F > 65535) return fail(DFMNMF_EINVAL, "F=%d exceeds 65535", d->F);
  if (d->K > 16 || d->N > 16 || d->B > 64)
    return fail(DFMNMF_EINVAL, "limits: K <= 16, N <= 16, B <= 64 (K=%d N=%d B=%d)", d->K, d->N, d->B);
  if (!d->mics) return fail(DFMNMF_EINVAL, "mics is NULL");
  const int MK = d->mics[0];
  for (int k = 0; k < d->K; ++k) {
    if (d->mics[k] < 1) return fail(DFMNMF_EINVAL, "mics[%d]=%d must be positive", k, d->mics[k]);
    if (d->mics[k] != MK)
      return fail(DFMNMF_EINVAL, "this release needs equal subarray sizes (mics[0]=%d, mics[%d]=%d)", MK, k,
                  d->mics[k]);
  }
  if (MK > 4 && !((MK == 16 || MK == 32) && d->K == 1))
    return fail(DFMNMF_EINVAL,
                "subarray size M_k=%d: this release supports 1..4, or 16 or 32 with K = 1 (all-microphone form)", MK);
  if (d->precision != DFMNMF_FP32 && !dfm::is_tc(d->precision))
    return fail(DFMNMF_EINVAL, "precision %d is not built in this release", d->precision);
  if (dfm::is_tc(d->precision) && !dfm::tc_supported(MK, d->K))
    return fail(DFMNMF_EINVAL, "the tensor-core form needs M_k = 4 and K in {1, 2, 4, 8} (M_k=%d K=%d)", MK, d->K);
  if (d->ip_arith < 0 || d->ip_arith > 2) return fail(DFMNMF_EINVAL, "unknown ip_arith %d", d->ip_arith);

  dfmnmf_ctx* c = new dfmnmf_ctx;
  memset(c, 0, sizeof *c);
  c->F = d->F; c->T = d->T; c->Tp = (d->T + 3) & ~3; c->Tr = (d->T + 63) & ~63; c->K = d->K; c->MK = MK; c->M = d->K * MK; c->N = d->N; c->B = d->B;
  c->precision = d->precision;
  c->ip_arith = d->ip_arith;
  c->eps = (float)(d->floor_eps > 0 ? d->floor_eps : 1e-6);
  if (c->eps < FLT_MIN) c->eps = FLT_MIN;  // the floored quantities stay normal floats
  c->singular_rtol = (d->ip_arith == DFMNMF_IP_F32) ? 1e-6f : 1e-12f;
  if (cudaGetDevice(&c->device) != cudaSuccess) {
    cudaGetLastError();
    delete c;
    return fail(DFMNMF_ECUDA, "no CUDA device");
  }
  if (cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, c->device) != cudaSuccess) c->num_sms = 152;
  if (cudaDeviceGetAttribute(&c->smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, c->device) != cudaSuccess)
    c->smem_optin = 232448;
  c->cfg_vx_groups = 2;
  c->wait_cycles = 2000000000u;  // ~1 s at 2 GHz
  c->cfg_branches = 2;
  c->cfg_nmf_ctas = 4;
  int r = 0;
  const int ty = (c->T + 127) / 128;
  c->red_len = (size_t)c->F * ty + (size_t)c->F * c->K;
  if ((r = dalloc(&c->x, nx(c), "x")) || (r = dalloc(&c->Q64, nQ(c), "Q64")) ||
      (r = dalloc(&c->Q32, nQ(c), "Q32")) || (r = dalloc(&c->Qinv32, nQ(c), "Qinv")) ||
      (r = dalloc(&c->V, nQ(c) * MK, "V")) || (r = dalloc(&c->Vdd, nQ(c) * MK, "Vdd")) || (r = dalloc(&c->W, nW(c), "W")) ||
      (r = dalloc(&c->H, nH(c), "H")) || (r = dalloc(&c->g, ng(c), "g")) ||
      (r = dalloc(&c->lam, (size_t)c->N * c->F * c->Tp, "lambda")) || (r = dalloc(&c->P, nx(c), "P")) ||
      (r = dalloc(&c->A, (size_t)c->N * c->F * c->Tp, "A")) ||
      (r = dalloc(&c->D, (size_t)c->N * c->F * c->Tp, "D")) || (r = dalloc(&c->red, c->red_len, "red")) ||
      (r = dalloc(&c->nll_dev, 1, "nll")) || (r = dalloc(&c->flags, dfm::FLAG_COUNT, "flags")) ||
      (r = dalloc(&c->nmf_part, dfm::nmf_scratch_floats(c), "nmf partials")) ||
      (r = dalloc(&c->nmf_ticket, dfm::nmf_ticket_count(c), "nmf tickets"))) {
    free_ctx(c);
    return r;
  }
  if (dfm::is_tc(c->precision)) {
    if ((r = dalloc(&c->tc_part, dfm::tc_part_float4s(c), "tensor-core partial sums")) ||
        (r = dalloc(&c->tc_ticket, dfm::tc_ticket_count(c), "tensor-core tickets")) ||
        (r = dalloc(&c->wtc_part, dfm::wupd_tc_scratch_float2s(c), "tensor-core W-update parts")) ||
        (r = dalloc(&c->wtc_ticket, dfm::wupd_tc_ticket_count(c), "tensor-core W-update tickets"))) {
      free_ctx(c);
      return r;
    }
    if (dfm::tc_raw_stages(c) == 0) {
      free_ctx(c);
      return fail(DFMNMF_EINVAL, "the tensor-core form needs more shared memory than the device offers (N=%d K=%d)",
                  c->N, c->K);
    }
  }
  cudaStream_t s = as_stream(stream);
  auto bail = [&](int code) { free_ctx(c); return code; };
  if (cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking) != cudaSuccess ||
      cudaStreamCreateWithFlags(&c->side_stream, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreateWithFlags(&c->fork_ev, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&c->join_ev, cudaEventDisableTiming) != cudaSuccess)
    return bail(fail(DFMNMF_ECUDA, "stream or event creation failed"));
#define CKI(call)                                                                                        \
  do {                                                                                                   \
    cudaError_t e_ = (call);                                                                             \
    if (e_ != cudaSuccess) return bail(fail(DFMNMF_ECUDA, "%s failed: %s", #call, cudaGetErrorString(e_))); \
  } while (0)
  CKI(cudaMemcpyAsync(c->x, x, nx(c) * sizeof(float2), cudaMemcpyDefault, s));
  CKI(cudaMemcpyAsync(c->W, W0, nW(c) * sizeof(float), cudaMemcpyDefault, s));
  CKI(cudaMemsetAsync(c->H, 0, nH(c) * sizeof(float), s));
  CKI(copy_H(c, c->H, H0, true, s));
  CKI(cudaMemcpyAsync(c->g, g0, ng(c) * sizeof(float), cudaMemcpyDefault, s));
  if (Q0) {
    CKI(cudaMemcpyAsync(c->Q64, Q0, nQ(c) * sizeof(double2), cudaMemcpyDefault, s));
  } else {
    k_identity_blocks<<<(unsigned)((nQ(c) + 255) / 256), 256, 0, s>>>(c->Q64, c->F, c->K, MK);
    CKI(cudaGetLastError());
  }
  CKI(cudaMemsetAsync(c->flags, 0, dfm::FLAG_COUNT * sizeof(unsigned), s));
  CKI(cudaMemsetAsync(c->nmf_ticket, 0, dfm::nmf_ticket_count(c) * sizeof(unsigned), s));
  CKI(cudaMemsetAsync(c->P, 0, nx(c) * sizeof(float), s));
  CKI(cudaMemsetAsync(c->lam, 0, (size_t)c->N * c->F * c->Tp * sizeof(float), s));
  CKI(cudaMemsetAsync(c->A, 0, (size_t)c->N * c->F * c->Tp * sizeof(float), s));
  CKI(cudaMemsetAsync(c->D, 0, (size_t)c->N * c->F * c->Tp * sizeof(float), s));
  if (c->tc_ticket) CKI(cudaMemsetAsync(c->tc_ticket, 0, dfm::tc_ticket_count(c) * sizeof(unsigned), s));
  if (c->wtc_ticket) CKI(cudaMemsetAsync(c->wtc_ticket, 0, dfm::wupd_tc_ticket_count(c) * sizeof(unsigned), s));
  if ((r = refresh_derived(c, s))) return bail(r);
#undef CKI
  *out = c;
  return DFMNMF_OK;
}

int dfmnmf_set_observation(dfmnmf_ctx* c, const void* x, void* stream) {
  if (!c || !x) return fail(DFMNMF_EINVAL, "null argument");
  CK(cudaSetDevice(c->device));
  CK(cudaMemcpyAsync(c->x, x, nx(c) * sizeof(float2), cudaMemcpyDefault, as_stream(stream)));
  return DFMNMF_OK;
}

int dfmnmf_iterate(dfmnmf_ctx* c, int n_iter, void* stream) {
  if (!c) return fail(DFMNMF_EINVAL, "null context");
  if (n_iter < 0) return fail(DFMNMF_EINVAL, "n_iter=%d is negative", n_iter);
  if (n_iter == 0) return DFMNMF_OK;
  CK(cudaSetDevice(c->device));
  int r = ensure_graph(c);
  if (r) return r;
  for (int i = 0; i < n_iter; ++i) CK(cudaGraphLaunch(c->gexec, as_stream(stream)));
  return DFMNMF_OK;
}

int dfmnmf_run_stage(dfmnmf_ctx* c, int stage, void* stream) {
  if (!c) return fail(DFMNMF_EINVAL, "null context");
  if (stage < DFMNMF_STAGE_COV || stage > DFMNMF_STAGE_G) return fail(DFMNMF_EINVAL, "unknown stage %d", stage);
  CK(cudaSetDevice(c->device));
  return enqueue_stage(c, stage, as_stream(stream));
}

int dfmnmf_set_option(dfmnmf_ctx* c, int option, int value) {
  if (!c) return fail(DFMNMF_EINVAL, "null context");
  switch (option) {
    case DFMNMF_OPT_BRANCHES:
      if (value != 1 && value != 2) return fail(DFMNMF_EINVAL, "branches must be 1 or 2 (got %d)", value);
      c->cfg_branches = value;
      break;
    case DFMNMF_OPT_NMF_CTAS:
      if (value != 2 && value != 4 && value != 8) return fail(DFMNMF_EINVAL, "nmf_ctas must be 2, 4 or 8 (got %d)", value);
      c->cfg_nmf_ctas = value;
      break;
    case DFMNMF_OPT_VX_GROUPS:
      if (value != 1 && value != 2) return fail(DFMNMF_EINVAL, "vx_groups must be 1 or 2 (got %d)", value);
      c->cfg_vx_groups = value;
      break;
    case DFMNMF_OPT_WUPD_TC:
      if (value != 0 && value != 1) return fail(DFMNMF_EINVAL, "wupd_tc must be 0 or 1 (got %d)", value);
      if (value == 1 && !dfm::is_tc(c->precision))
        return fail(DFMNMF_EINVAL, "the tensor-core W update belongs to the tensor-core forms");
      c->cfg_wupd_tc = value;
      break;
    case DFMNMF_OPT_WAIT_CYCLES:
      if (value < 1) return fail(DFMNMF_EINVAL, "wait_cycles must be positive (got %d)", value);
      c->wait_cycles = (unsigned)value;
      break;
    default:
      return fail(DFMNMF_EINVAL, "unknown option %d", option);
  }
  drop_graph(c);
  return DFMNMF_OK;
}

int dfmnmf_get_option(const dfmnmf_ctx* c, int option) {
  if (!c) return -1;
  switch (option) {
    case DFMNMF_OPT_BRANCHES: return c->cfg_branches;
    case DFMNMF_OPT_NMF_CTAS: return c->cfg_nmf_ctas;
    case DFMNMF_OPT_VX_GROUPS: return c->cfg_vx_groups;
    case DFMNMF_OPT_WUPD_TC: return c->cfg_wupd_tc;
    case DFMNMF_OPT_WAIT_CYCLES: return c->wait_cycles > 0x7fffffffu ? 0x7fffffff : (int)c->wait_cycles;
    default: return -1;
  }
}

int dfmnmf_launches_per_iteration(const dfmnmf_ctx* c) {
  if (!c) return -1;
  Launch L[kMaxLaunches];
  const int n = iteration_launches(c, L);
  int ranged = 0;
  for (int i = 0; i < n; ++i) ranged += L[i].ranged ? 1 : 0;
  return band_split(c) > 0 ? n + ranged : n;
}

int dfmnmf_kernel_times(dfmnmf_ctx* c, int n_iter, double* avg_ms, const char** names, int cap, int* count,
                        void* stream) {
  if (!c || !avg_ms || !count || n_iter < 1) return fail(DFMNMF_EINVAL, "bad argument");
  CK(cudaSetDevice(c->device));
  Launch L[kMaxLaunches];
  const int n = iteration_launches(c, L);
  *count = n;
  if (cap < n) return fail(DFMNMF_EINVAL, "capacity %d < %d kernels", cap, n);
  cudaStream_t s = as_stream(stream);
  // One iteration, band-wide launches in order, captured into a graph with a
  // timing event after every launch: replays run back to back on the device,
  // so host launch latency does not enter the per-kernel times.
  cudaEvent_t ev[kMaxLaunches + 1] = {};
  int nev = 0;
  for (; nev <= n; ++nev)
    if (cudaEventCreate(&ev[nev]) != cudaSuccess) break;
  int rc = nev <= n ? fail(DFMNMF_ECUDA, "event creation failed") : DFMNMF_OK;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t gexec = nullptr;
  if (!rc && cudaStreamBeginCapture(c->cap_stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess)
    rc = fail(DFMNMF_ECUDA, "capture failed");
  if (!rc) {
    cudaError_t e = cudaEventRecordWithFlags(ev[0], c->cap_stream, cudaEventRecordExternal);
    for (int i = 0; i < n && e == cudaSuccess; ++i) {
      e = L[i].fn(c, c->cap_stream, 0, c->F);
      if (e == cudaSuccess) e = cudaEventRecordWithFlags(ev[i + 1], c->cap_stream, cudaEventRecordExternal);
    }
    const cudaError_t e2 = cudaStreamEndCapture(c->cap_stream, &graph);
    if (e != cudaSuccess || e2 != cudaSuccess) rc = fail(DFMNMF_ECUDA, "capture of the timed iteration failed: %s",
                                                         cudaGetErrorString(e != cudaSuccess ? e : e2));
  }
  if (!rc && cudaGraphInstantiate(&gexec, graph, 0) != cudaSuccess) rc = fail(DFMNMF_ECUDA, "graph instantiation failed");
  for (int i = 0; i < n; ++i) avg_ms[i] = 0.0;
  for (int it = 0; it < n_iter && !rc; ++it) {
    if (cudaGraphLaunch(gexec, s) != cudaSuccess || cudaStreamSynchronize(s) != cudaSuccess) {
      rc = fail(DFMNMF_ECUDA, "timed iteration failed");
      break;
    }
    for (int i = 0; i < n; ++i) {
      float ms = 0.f;
      cudaEventElapsedTime(&ms, ev[i], ev[i + 1]);
      avg_ms[i] += ms / n_iter;
    }
  }
  if (gexec) cudaGraphExecDestroy(gexec);
  if (graph) cudaGraphDestroy(graph);
  for (int i = 0; i < nev; ++i) cudaEventDestroy(ev[i]);
  if (names)
    for (int i = 0; i < n; ++i) names[i] = L[i].name;
  return rc;
}

int dfmnmf_kernel_times_isolated(dfmnmf_ctx* c, int reps, double* avg_ms, const char** names, int cap, int* count,
                                 void* stream) {
  if (!c || !avg_ms || !count || reps < 1) return fail(DFMNMF_EINVAL, "bad argument");
  CK(cudaSetDevice(c->device));
  Launch L[kMaxLaunches];
  const int n = iteration_launches(c, L);
  *count = n;
  if (cap < n) return fail(DFMNMF_EINVAL, "capacity %d < %d kernels", cap, n);
  cudaStream_t s = as_stream(stream);
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  int rc = (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)
               ? fail(DFMNMF_ECUDA, "event creation failed")
               : DFMNMF_OK;
  // Each kernel of the iteration alone: `reps` band-wide launches back to back in one graph, timed by
  // two events around the graph (so neither host latency nor per-launch events enter the time).
  for (int i = 0; i < n && !rc; ++i) {
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t gexec = nullptr;
    cudaError_t e = cudaStreamBeginCapture(c->cap_stream, cudaStreamCaptureModeThreadLocal);
    for (int r = 0; r < reps && e == cudaSuccess; ++r) e = L[i].fn(c, c->cap_stream, 0, c->F);
    const cudaError_t e2 = cudaStreamEndCapture(c->cap_stream, &graph);
    if (e == cudaSuccess) e = e2;
    if (e == cudaSuccess) e = cudaGraphInstantiate(&gexec, graph, 0);
    if (e == cudaSuccess) e = cudaGraphLaunch(gexec, s);  // warm-up
    if (e == cudaSuccess) e = cudaEventRecord(e0, s);
    if (e == cudaSuccess) e = cudaGraphLaunch(gexec, s);
    if (e == cudaSuccess) e = cudaEventRecord(e1, s);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    avg_ms[i] = ms / reps;
    if (gexec) cudaGraphExecDestroy(gexec);
    if (graph) cudaGraphDestroy(graph);
    if (e != cudaSuccess) rc = fail(DFMNMF_ECUDA, "isolated timing of %s failed: %s", L[i].name, cudaGetErrorString(e));
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (names)
    for (int i = 0; i < n; ++i) names[i] = L[i].name;
  return rc;
}

int dfmnmf_cost_gradient(dfmnmf_ctx* c, void* dQ, float* dW, float* dH, float* dg, double* nll_host, void* stream) {
  if (!c) return fail(DFMNMF_EINVAL, "null context");
  if (c->MK > 16) return fail(DFMNMF_EINVAL, "the cost gradient supports blocks of up to 16 microphones (M_k=%d)", c->MK);
  CK(cudaSetDevice(c->device));
  cudaStream_t s = as_stream(stream);
  int r = 0;
  if (!c->gQ && ((r = dalloc(&c->gQ, nQ(c), "dQ")) || (r = dalloc(&c->gW, nW(c), "dW")) ||
                 (r = dalloc(&c->gH, nH(c), "dH")) || (r = dalloc(&c->gg, ng(c), "dg")))) {
    cudaFree(c->gQ); cudaFree(c->gW); cudaFree(c->gH); cudaFree(c->gg);
    c->gQ = nullptr; c->gW = c->gH = c->gg = nullptr;
    return r;
  }
  // every statistic from the current state: lambda, float-float V, compensated P with A and D
  CK(dfm::launch_lambda(c, s));
  CK(dfm::launch_cov(c, s, 0, c->F));
  CK(dfm::launch_power_stats_comp(c, s));
  CK(dfm::launch_wupd(c, s, c->gW));
  CK(dfm::launch_hupd(c, s, c->gH));
  CK(dfm::launch_gupd(c, s, c->gg));
  CK(dfm::launch_qgrad(c, c->gQ, s));
  bool host = false;
  if (dQ) { CK(cudaMemcpyAsync(dQ, c->gQ, nQ(c) * sizeof(double2), cudaMemcpyDefault, s)); host |= is_host_ptr(dQ); }
  if (dW) { CK(cudaMemcpyAsync(dW, c->gW, nW(c) * sizeof(float), cudaMemcpyDefault, s)); host |= is_host_ptr(dW); }
  if (dH) { CK(copy_H(c, dH, c->gH, false, s)); host |= is_host_ptr(dH); }
  if (dg) { CK(cudaMemcpyAsync(dg, c->gg, ng(c) * sizeof(float), cudaMemcpyDefault, s)); host |= is_host_ptr(dg); }
  if (nll_host) return dfmnmf_loglik(c, nll_host, stream);  // synchronises
  if (host) CK(cudaStreamSynchronize(s));
  return DFMNMF_OK;
}

int dfmnmf_autotune(dfmnmf_ctx* c, int iters_per_trial, int* branches, int* nmf_ctas, void* stream) {
  if (!c || iters_per_trial < 1) return fail(DFMNMF_EINVAL, "bad argument");
  CK(cudaSetDevice(c->device));
  cudaStream_t s = as_stream(stream);
  // the trials advance the state: keep a copy and put it back after every trial
  double2* Qb = nullptr;
  float *Wb = nullptr, *Hb = nullptr, *gb = nullptr;
  unsigned* fb = nullptr;
  int r = 0;
  if ((r = dalloc(&Qb, nQ(c), "Q backup")) || (r = dalloc(&Wb, nW(c), "W backup")) ||
      (r = dalloc(&Hb, nH(c), "H backup")) || (r = dalloc(&gb, ng(c), "g backup")) ||
      (r = dalloc(&fb, dfm::FLAG_COUNT, "flags backup"))) {
    cudaFree(Qb); cudaFree(Wb); cudaFree(Hb); cudaFree(gb); cudaFree(fb);
    return r;
  }
  auto copy_state = [&](bool save) -> cudaError_t {
    cudaError_t e = cudaSuccess;
    const cudaMemcpyKind k = cudaMemcpyDeviceToDevice;
    if (save) {
      if (e == cudaSuccess) e = cudaMemcpyAsync(Qb, c->Q64, nQ(c) * sizeof(double2), k, s);
      if (e == cudaSuccess) e = cudaMemcpyAsync(Wb, c->W, nW(c) * sizeof(float), k, s);
      if (e == cudaSuccess) e = cudaMemcpyAsync(Hb, c->H, nH(c) * sizeof(float), k, s);
      if (e == cudaSuccess) e = cudaMemcpyAsync(gb, c->g, ng(c) * sizeof(float), k, s);
      if (e == cudaSuccess) e = cudaMemcpyAsync(fb, c->flags, dfm::FLAG_COUNT * sizeof(unsigned), k, s);
    } else {
      if (e == cudaSuccess) e = cudaMemcpyAsync(c->Q64, Qb, nQ(c) * sizeof(double2), k, s);
      if (e == cudaSuccess) e = cudaMemcpyAsync(c->W, Wb, nW(c) * sizeof(float), k, s);
      if (e == cudaSuccess) e = cudaMemcpyAsync(c->H, Hb, nH(c) * sizeof(float), k, s);
      if (e == cudaSuccess) e = cudaMemcpyAsync(c->g, gb, ng(c) * sizeof(float), k, s);
      if (e == cudaSuccess) e = cudaMemcpyAsync(c->flags, fb, dfm::FLAG_COUNT * sizeof(unsigned), k, s);
      if (e == cudaSuccess) e = dfm::launch_lambda(c, s);
      if (e == cudaSuccess) e = dfm::launch_q_convert(c, s);
    }
    return e;
  };
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  // first option: graph branches of the per-frequency kernels (FP32 form) or converter warp groups of the
  // persistent covariance kernel (tensor-core form, one branch); second: CTAs per SM of the NMF products
  const bool tc = dfm::is_tc(c->precision);
  const int old_br = c->cfg_branches, old_ct = c->cfg_nmf_ctas, old_vx = c->cfg_vx_groups;
  int best_br = old_br, best_ct = old_ct, best_vx = old_vx;
  float best = INFINITY;
  cudaError_t e = copy_state(true);
  if (e == cudaSuccess) e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  const int br_opts[2] = {1, 2}, ct_opts[3] = {2, 4, 8};
  for (int ib = 0; ib < 2 && e == cudaSuccess && !r; ++ib)
    for (int ic = 0; ic < 3 && e == cudaSuccess && !r; ++ic) {
      c->cfg_branches = tc ? 1 : br_opts[ib];
      c->cfg_vx_groups = tc ? br_opts[ib] : old_vx;
      c->cfg_nmf_ctas = ct_opts[ic];
      if (!tc && c->cfg_branches == 2 && band_split(c) == 0) continue;  // band too small to split
      drop_graph(c);
      if ((r = ensure_graph(c))) break;
      e = cudaGraphLaunch(c->gexec, s);  // warm-up
      if (e == cudaSuccess) e = cudaEventRecord(e0, s);
      for (int i = 0; i < iters_per_trial && e == cudaSuccess; ++i) e = cudaGraphLaunch(c->gexec, s);
      if (e == cudaSuccess) e = cudaEventRecord(e1, s);
      if (e == cudaSuccess) e = cudaEventSynchronize(e1);
      float ms = 0.f;
      if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
      if (e == cudaSuccess && ms < best) {
        best = ms;
        best_br = c->cfg_branches;
        best_ct = c->cfg_nmf_ctas;
        best_vx = c->cfg_vx_groups;
      }
      if (e == cudaSuccess) e = copy_state(false);
    }
  c->cfg_branches = (e == cudaSuccess && !r) ? best_br : old_br;
  c->cfg_nmf_ctas = (e == cudaSuccess && !r) ? best_ct : old_ct;
  c->cfg_vx_groups = (e == cudaSuccess && !r) ? best_vx : old_vx;
  drop_graph(c);
  if (e == cudaSuccess) e = copy_state(false);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaFree(Qb); cudaFree(Wb); cudaFree(Hb); cudaFree(gb); cudaFree(fb);
  if (r) return r;
  if (e != cudaSuccess) return fail(DFMNMF_ECUDA, "autotune: %s", cudaGetErrorString(e));
  if (branches) *branches = c->cfg_branches;
  if (nmf_ctas) *nmf_ctas = c->cfg_nmf_ctas;
  return DFMNMF_OK;
}

int dfmnmf_batch_create(dfmnmf_batch** out, dfmnmf_ctx* const* ctxs, int count) {
  if (!out || !ctxs || count < 1) return fail(DFMNMF_EINVAL, "bad argument");
  *out = nullptr;
  for (int i = 0; i < count; ++i) {
    if (!ctxs[i]) return fail(DFMNMF_EINVAL, "context %d is NULL", i);
    if (ctxs[i]->device != ctxs[0]->device) return fail(DFMNMF_EINVAL, "contexts on different devices");
  }
  CK(cudaSetDevice(ctxs[0]->device));
  for (int i = 0; i < count; ++i) {
    const int r = ensure_graph(ctxs[i]);
    if (r) return r;
  }
  cudaGraph_t g = nullptr;
  cudaGraphExec_t ge = nullptr;
  CK(cudaGraphCreate(&g, 0));
  cudaError_t e = cudaSuccess;
  for (int i = 0; i < count && e == cudaSuccess; ++i) {
    cudaGraphNode_t node;
    e = cudaGraphAddChildGraphNode(&node, g, nullptr, 0, ctxs[i]->graph);  // independent branches
  }
  if (e == cudaSuccess) e = cudaGraphInstantiate(&ge, g, 0);
  if (e != cudaSuccess) {
    cudaGraphDestroy(g);
    return fail(DFMNMF_ECUDA, "batch graph: %s", cudaGetErrorString(e));
  }
  dfmnmf_batch* b = new dfmnmf_batch;
  b->count = count;
  b->device = ctxs[0]->device;
  b->graph = g;
  b->gexec = ge;
  *out = b;
  return DFMNMF_OK;
}

int dfmnmf_batch_iterate(dfmnmf_batch* b, int n_iter, void* stream) {
  if (!b) return fail(DFMNMF_EINVAL, "null batch");
  if (n_iter < 0) return fail(DFMNMF_EINVAL, "n_iter=%d is negative", n_iter);
  CK(cudaSetDevice(b->device));
  for (int i = 0; i < n_iter; ++i) CK(cudaGraphLaunch(b->gexec, as_stream(stream)));
  return DFMNMF_OK;
}

void dfmnmf_batch_destroy(dfmnmf_batch* b) {
  if (!b) return;
  cudaSetDevice(b->device);
  if (b->gexec) cudaGraphExecDestroy(b->gexec);
  if (b->graph) cudaGraphDestroy(b->graph);
  delete b;
}

int dfmnmf_init_from_images(dfmnmf_ctx* c, const void* c_img, float* h_out, void* stream) {
  if (!c || !c_img) return fail(DFMNMF_EINVAL, "null argument");
  if (c->N < 2) return fail(DFMNMF_EINVAL, "the initialisation needs N >= 2 sources (N = %d)", c->N);
  if (!dfm::init_supported(c->M, c->MK)) return fail(DFMNMF_EINVAL, "the initialisation supports M <= 32 (M = %d)", c->M);
  if (is_host_ptr(c_img) || (h_out && is_host_ptr(h_out)))
    return fail(DFMNMF_EINVAL, "c_img and h_out must be device memory");
  CK(cudaSetDevice(c->device));
  cudaStream_t s = as_stream(stream);
  const size_t nR = (size_t)c->N * c->F * c->M * c->M;
  double2* R = nullptr;
  float2* Linv = nullptr;
  CK(cudaMallocAsync(reinterpret_cast<void**>(&R), nR * sizeof(double2), s));
  cudaError_t e = cudaMallocAsync(reinterpret_cast<void**>(&Linv), nR * sizeof(float2), s);
  if (e == cudaSuccess)
    e = dfm::launch_init_from_images(c, reinterpret_cast<const float2*>(c_img), R, Linv, h_out, s);
  if (e == cudaSuccess) e = dfm::launch_q_convert(c, s);
  if (Linv) cudaFreeAsync(Linv, s);
  cudaFreeAsync(R, s);
  if (e != cudaSuccess) return fail(DFMNMF_ECUDA, "initialisation failed: %s", cudaGetErrorString(e));
  unsigned flags[dfm::FLAG_COUNT];
  CK(cudaMemcpyAsync(flags, c->flags, sizeof flags, cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  if (flags[dfm::FLAG_NONFINITE])
    return fail(DFMNMF_ENUMERIC, "a covariance of the initial images is not positive definite");
  return DFMNMF_OK;
}

int dfmnmf_loglik(dfmnmf_ctx* c, double* nll_host, void* stream) {
  if (!c || !nll_host) return fail(DFMNMF_EINVAL, "null argument");
  CK(cudaSetDevice(c->device));
  cudaStream_t s = as_stream(stream);
  CK(dfm::launch_lambda(c, s));  // lambda = W H of the current state (stages may leave it behind)
  CK(dfm::launch_loglik(c, s));
  unsigned flags[dfm::FLAG_COUNT];
  double v = 0.0;
  CK(cudaMemcpyAsync(&v, c->nll_dev, sizeof(double), cudaMemcpyDeviceToHost, s));
  CK(cudaMemcpyAsync(flags, c->flags, sizeof flags, cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  *nll_host = v;
  if (flags[dfm::FLAG_TIMEOUT]) return fail(DFMNMF_ETIMEOUT, "a bounded device wait gave up");
  if (flags[dfm::FLAG_NONFINITE]) return fail(DFMNMF_ENUMERIC, "a non-finite value was produced (flags=%u)",
                                              flags[dfm::FLAG_NONFINITE]);
  return DFMNMF_OK;
}

int dfmnmf_separate(dfmnmf_ctx* c, void* c_out, void* stream) {
  if (!c || !c_out) return fail(DFMNMF_EINVAL, "null argument");
  if (is_host_ptr(c_out)) return fail(DFMNMF_EINVAL, "c_out must be device memory");
  CK(cudaSetDevice(c->device));
  cudaStream_t s = as_stream(stream);
  CK(dfm::launch_lambda(c, s));
  CK(dfm::launch_qinv(c, s));
  CK(dfm::launch_separate(c, reinterpret_cast<float2*>(c_out), s));
  return DFMNMF_OK;
}

int dfmnmf_get_params(dfmnmf_ctx* c, void* Q, float* W, float* H, float* g, void* stream) {
  if (!c) return fail(DFMNMF_EINVAL, "null context");
  CK(cudaSetDevice(c->device));
  cudaStream_t s = as_stream(stream);
  bool host = false;
  if (Q) { CK(cudaMemcpyAsync(Q, c->Q64, nQ(c) * sizeof(double2), cudaMemcpyDefault, s)); host |= is_host_ptr(Q); }
  if (W) { CK(cudaMemcpyAsync(W, c->W, nW(c) * sizeof(float), cudaMemcpyDefault, s)); host |= is_host_ptr(W); }
  if (H) { CK(copy_H(c, H, c->H, false, s)); host |= is_host_ptr(H); }
  if (g) { CK(cudaMemcpyAsync(g, c->g, ng(c) * sizeof(float), cudaMemcpyDefault, s)); host |= is_host_ptr(g); }
  if (host) CK(cudaStreamSynchronize(s));
  return DFMNMF_OK;
}

int dfmnmf_set_params(dfmnmf_ctx* c, const void* Q, const float* W, const float* H, const float* g,
                      void* stream) {
  if (!c) return fail(DFMNMF_EINVAL, "null context");
  CK(cudaSetDevice(c->device));
  cudaStream_t s = as_stream(stream);
  if (Q) CK(cudaMemcpyAsync(c->Q64, Q, nQ(c) * sizeof(double2), cudaMemcpyDefault, s));
  if (W) CK(cudaMemcpyAsync(c->W, W, nW(c) * sizeof(float), cudaMemcpyDefault, s));
  if (H) CK(copy_H(c, c->H, H, true, s));
  if (g) CK(cudaMemcpyAsync(c->g, g, ng(c) * sizeof(float), cudaMemcpyDefault, s));
  return refresh_derived(c, s);
}

int dfmnmf_get_buffer(dfmnmf_ctx* c, int which, void* dst, size_t dst_bytes, void* stream) {
  if (!c || !dst) return fail(DFMNMF_EINVAL, "null argument");
  const void* src = nullptr;
  size_t bytes = 0;
  switch (which) {
    case DFMNMF_BUF_V: src = c->V; bytes = nQ(c) * c->MK * sizeof(double2); break;
    case DFMNMF_BUF_P: src = c->P; bytes = nx(c) * sizeof(float); break;
    case DFMNMF_BUF_LAMBDA: src = c->lam; bytes = (size_t)c->N * c->F * c->T * sizeof(float); break;
    default: return fail(DFMNMF_EINVAL, "unknown buffer %d", which);
  }
  if (dst_bytes < bytes) return fail(DFMNMF_EINVAL, "buffer %d needs %zu bytes, got %zu", which, bytes, dst_bytes);
  CK(cudaSetDevice(c->device));
  cudaStream_t s = as_stream(stream);
  if (which == DFMNMF_BUF_LAMBDA) CK(dfm::launch_lambda(c, s));  // W H of the current state
  if (which == DFMNMF_BUF_LAMBDA)  // drop the padding of the row stride
    CK(cudaMemcpy2DAsync(dst, (size_t)c->T * sizeof(float), src, (size_t)c->Tp * sizeof(float),
                         (size_t)c->T * sizeof(float), (size_t)c->N * c->F, cudaMemcpyDefault, s));
  else
    CK(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDefault, s));
  if (is_host_ptr(dst)) CK(cudaStreamSynchronize(s));
  return DFMNMF_OK;
}

void dfmnmf_destroy(dfmnmf_ctx* c) {
  if (!c) return;
  cudaSetDevice(c->device);
  cudaDeviceSynchronize();
  free_ctx(c);
}

}  // extern "C"
