// common.cuh -- device helpers shared by the distributed-FastMNMF kernels.
//
// Complex arithmetic over a templated real type, a float-float ("double
// float") real type built from Dekker's exact product and Knuth's exact sum,
// and warp reductions.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#define DFM_FULL_MASK 0xffffffffu

namespace dfm {

// ---------------------------------------------------------------- float-float
// A value is hi + lo with |lo| <= ulp(hi)/2.  Exact transformations:
//   two_sum  (Knuth, TAOCP vol. 2, 4.2.2):  a + b = s + e exactly.
//   two_prod (Dekker 1971 via a fused multiply-add): a * b = p + e exactly.
// Arithmetic below follows the standard double-word algorithms
// (accurate addition, product with cross terms, long division, one Newton
// step for the square root); relative error about 2^-46.
struct dd {
  float hi, lo;
};

__device__ __forceinline__ dd dd_make(float h, float l) { dd r; r.hi = h; r.lo = l; return r; }
__device__ __forceinline__ dd two_sum(float a, float b) {
  float s = __fadd_rn(a, b);
  float bb = __fsub_rn(s, a);
  float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  return dd_make(s, e);
}
__device__ __forceinline__ dd quick_two_sum(float a, float b) {
  float s = __fadd_rn(a, b);
  float e = __fsub_rn(b, __fsub_rn(s, a));
  return dd_make(s, e);
}
__device__ __forceinline__ dd two_prod(float a, float b) {
  float p = __fmul_rn(a, b);
  float e = __fmaf_rn(a, b, -p);
  return dd_make(p, e);
}
__device__ __forceinline__ dd operator+(dd a, dd b) {
  dd s = two_sum(a.hi, b.hi);
  dd t = two_sum(a.lo, b.lo);
  s.lo = __fadd_rn(s.lo, t.hi);
  s = quick_two_sum(s.hi, s.lo);
  s.lo = __fadd_rn(s.lo, t.lo);
  return quick_two_sum(s.hi, s.lo);
}
__device__ __forceinline__ dd operator-(dd a) { return dd_make(-a.hi, -a.lo); }
__device__ __forceinline__ dd operator-(dd a, dd b) { return a + (-b); }
__device__ __forceinline__ dd operator*(dd a, dd b) {
  dd p = two_prod(a.hi, b.hi);
  p.lo = __fmaf_rn(a.hi, b.lo, __fmaf_rn(a.lo, b.hi, p.lo));
  return quick_two_sum(p.hi, p.lo);
}
__device__ __forceinline__ dd mul_f(dd a, float b) {
  dd p = two_prod(a.hi, b);
  p.lo = __fmaf_rn(a.lo, b, p.lo);
  return quick_two_sum(p.hi, p.lo);
}
__device__ __forceinline__ dd operator/(dd a, dd b) {
  float q1 = __fdiv_rn(a.hi, b.hi);
  dd r = a - mul_f(b, q1);
  float q2 = __fdiv_rn(r.hi, b.hi);
  r = r - mul_f(b, q2);
  float q3 = __fdiv_rn(r.hi, b.hi);
  dd q = quick_two_sum(q1, q2);
  return q + dd_make(q3, 0.f);
}

// ------------------------------------------------------------- real traits
template <class R> struct RealOps;

template <> struct RealOps<double> {
  static __device__ __forceinline__ double from_f(float a) { return (double)a; }
  static __device__ __forceinline__ double from_d(double a) { return a; }
  static __device__ __forceinline__ double to_d(double a) { return a; }
  static __device__ __forceinline__ float to_f(double a) { return (float)a; }
  static __device__ __forceinline__ double zero() { return 0.0; }
  static __device__ __forceinline__ double one() { return 1.0; }
  static __device__ __forceinline__ double add(double a, double b) { return a + b; }
  static __device__ __forceinline__ double sub(double a, double b) { return a - b; }
  static __device__ __forceinline__ double mul(double a, double b) { return a * b; }
  static __device__ __forceinline__ double div(double a, double b) { return a / b; }
  static __device__ __forceinline__ double sqrt_(double a) { return sqrt(a); }
  static __device__ __forceinline__ double shfl(double a, int src) { return __shfl_sync(DFM_FULL_MASK, a, src); }
  static __device__ __forceinline__ double shfl_xor(double a, int m) { return __shfl_xor_sync(DFM_FULL_MASK, a, m); }
};

template <> struct RealOps<float> {
  static __device__ __forceinline__ float from_f(float a) { return a; }
  static __device__ __forceinline__ float from_d(double a) { return (float)a; }
  static __device__ __forceinline__ double to_d(float a) { return (double)a; }
  static __device__ __forceinline__ float to_f(float a) { return a; }
  static __device__ __forceinline__ float zero() { return 0.f; }
  static __device__ __forceinline__ float one() { return 1.f; }
  static __device__ __forceinline__ float add(float a, float b) { return a + b; }
  static __device__ __forceinline__ float sub(float a, float b) { return a - b; }
  static __device__ __forceinline__ float mul(float a, float b) { return a * b; }
  static __device__ __forceinline__ float div(float a, float b) { return a / b; }
  static __device__ __forceinline__ float sqrt_(float a) { return sqrtf(a); }
  static __device__ __forceinline__ float shfl(float a, int src) { return __shfl_sync(DFM_FULL_MASK, a, src); }
  static __device__ __forceinline__ float shfl_xor(float a, int m) { return __shfl_xor_sync(DFM_FULL_MASK, a, m); }
};

template <> struct RealOps<dd> {
  static __device__ __forceinline__ dd from_f(float a) { return dd_make(a, 0.f); }
  static __device__ __forceinline__ dd from_d(double a) {
    float h = (float)a;
    return dd_make(h, (float)(a - (double)h));
  }
  static __device__ __forceinline__ double to_d(dd a) { return (double)a.hi + (double)a.lo; }
  static __device__ __forceinline__ float to_f(dd a) { return a.hi; }
  static __device__ __forceinline__ dd zero() { return dd_make(0.f, 0.f); }
  static __device__ __forceinline__ dd one() { return dd_make(1.f, 0.f); }
  static __device__ __forceinline__ dd add(dd a, dd b) { return a + b; }
  static __device__ __forceinline__ dd sub(dd a, dd b) { return a - b; }
  static __device__ __forceinline__ dd mul(dd a, dd b) { return a * b; }
  static __device__ __forceinline__ dd div(dd a, dd b) { return a / b; }
  // One Newton step from the single-precision root: y = x + (a - x^2) / (2x).
  static __device__ __forceinline__ dd sqrt_(dd a) {
    if (!(a.hi > 0.f)) return dd_make(0.f, 0.f);
    float x = sqrtf(a.hi);
    dd r = a - two_prod(x, x);
    float corr = __fdiv_rn(r.hi, 2.f * x);
    return quick_two_sum(x, corr);
  }
  static __device__ __forceinline__ dd shfl(dd a, int src) {
    return dd_make(__shfl_sync(DFM_FULL_MASK, a.hi, src), __shfl_sync(DFM_FULL_MASK, a.lo, src));
  }
  static __device__ __forceinline__ dd shfl_xor(dd a, int m) {
    return dd_make(__shfl_xor_sync(DFM_FULL_MASK, a.hi, m), __shfl_xor_sync(DFM_FULL_MASK, a.lo, m));
  }
};

// ------------------------------------------------------------------ complex
template <class R> struct cx {
  R re, im;
};
template <class R> __device__ __forceinline__ cx<R> cmake(R a, R b) { cx<R> c; c.re = a; c.im = b; return c; }
template <class R> __device__ __forceinline__ cx<R> czero() { return cmake(RealOps<R>::zero(), RealOps<R>::zero()); }
template <class R> __device__ __forceinline__ cx<R> cadd(cx<R> a, cx<R> b) {
  using O = RealOps<R>;
  return cmake(O::add(a.re, b.re), O::add(a.im, b.im));
}
template <class R> __device__ __forceinline__ cx<R> csub(cx<R> a, cx<R> b) {
  using O = RealOps<R>;
  return cmake(O::sub(a.re, b.re), O::sub(a.im, b.im));
}
template <class R> __device__ __forceinline__ cx<R> cmul(cx<R> a, cx<R> b) {
  using O = RealOps<R>;
  return cmake(O::sub(O::mul(a.re, b.re), O::mul(a.im, b.im)),
               O::add(O::mul(a.re, b.im), O::mul(a.im, b.re)));
}
template <class R> __device__ __forceinline__ cx<R> cconj(cx<R> a) {
  using O = RealOps<R>;
  return cmake(a.re, O::sub(O::zero(), a.im));
}
template <class R> __device__ __forceinline__ cx<R> cscale(cx<R> a, R s) {
  using O = RealOps<R>;
  return cmake(O::mul(a.re, s), O::mul(a.im, s));
}
// 1 / a = conj(a) / |a|^2  (a == 0 gives 0; callers flag singularity separately)
template <class R> __device__ __forceinline__ cx<R> crecip(cx<R> a) {
  using O = RealOps<R>;
  R n = O::add(O::mul(a.re, a.re), O::mul(a.im, a.im));
  if (!(O::to_f(n) > 0.f)) return czero<R>();
  R inv = O::div(O::one(), n);
  return cmake(O::mul(a.re, inv), O::sub(O::zero(), O::mul(a.im, inv)));
}
template <class R> __device__ __forceinline__ float cabs2_f(cx<R> a) {
  float r = RealOps<R>::to_f(a.re), i = RealOps<R>::to_f(a.im);
  return r * r + i * i;
}
template <class R> __device__ __forceinline__ cx<R> cshfl(cx<R> a, int src) {
  return cmake(RealOps<R>::shfl(a.re, src), RealOps<R>::shfl(a.im, src));
}
template <class R> __device__ __forceinline__ cx<R> cfrom_f2(float2 v) {
  return cmake(RealOps<R>::from_f(v.x), RealOps<R>::from_f(v.y));
}
template <class R> __device__ __forceinline__ cx<R> cfrom_d2(double2 v) {
  return cmake(RealOps<R>::from_d(v.x), RealOps<R>::from_d(v.y));
}

// --------------------------------------------------------------- reductions
__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(DFM_FULL_MASK, v, o);
  return v;
}
__device__ __forceinline__ double warp_sum_d(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(DFM_FULL_MASK, v, o);
  return v;
}

// Reduce-scatter of C partial sums held by every lane of a warp (C a multiple
// of 32): afterwards lane l holds the warp totals of entries
// [l*C/32, (l+1)*C/32) in v[0 .. C/32).  Halving exchange, C - C/32 shuffles.
template <int C>
__device__ __forceinline__ void warp_reduce_scatter(float (&v)[C], int lane) {
  static_assert(C % 32 == 0, "reduce-scatter needs a multiple of 32 entries");
#pragma unroll
  for (int half = C / 2, bit = 16; bit >= 1; half >>= 1, bit >>= 1) {
    const bool upper = (lane & bit) != 0;
#pragma unroll
    for (int i = 0; i < half; ++i) {
      float keep = upper ? v[half + i] : v[i];
      float send = upper ? v[i] : v[half + i];
      v[i] = keep + __shfl_xor_sync(DFM_FULL_MASK, send, bit);
    }
  }
}

__device__ __forceinline__ bool finitef(float v) { return isfinite(v); }

// Hardware reciprocal (rcp.approx.ftz.f32, relative error <= 2^-23): the
// weights 1/yhat only ever enter as relative perturbations of positive terms.
// Every argument is max(yhat, eps) with eps at least the smallest normal float
// (dfmnmf_init raises a smaller floor to it), so flushing subnormal inputs
// changes nothing; the flush variant needs no subnormal handling around the
// hardware instruction.
__device__ __forceinline__ float fast_rcp(float a) {
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(a));
  return r;
}

// Compensated complex dot product y = sum_nu q_nu x_nu with q = qh + ql a
// float pair (the FP64 diagonaliser row split in two floats) and x single
// precision: every product qh * x is exact (Dekker), the running sum is kept
// error-free with Knuth's two-sum, and the rounding terms plus the ql * x
// products are added in single precision ("Dot2" of Ogita, Rump and Oishi).
// The result is as accurate as if computed in twice the working precision
// and then rounded, which matters when the row has large entries and y is
// small (cancellation by a factor |q| |x| / |y| of 1e2..1e4 on the outputs
// that track the noise floor).
template <int MK>
__device__ __forceinline__ float2 cdot2(const float2* __restrict__ qh, const float2* __restrict__ ql,
                                        const float2 (&x)[MK]) {
  float sr = 0.f, cr = 0.f, si = 0.f, ci = 0.f;
#pragma unroll
  for (int nu = 0; nu < MK; ++nu) {
    const float2 a = qh[nu], b = ql[nu], v = x[nu];
    // real part: a.x v.x - a.y v.y ; imag: a.x v.y + a.y v.x
    dd p = two_prod(a.x, v.x);
    dd s = two_sum(sr, p.hi);
    sr = s.hi; cr = __fadd_rn(cr, __fadd_rn(s.lo, p.lo));
    p = two_prod(-a.y, v.y);
    s = two_sum(sr, p.hi);
    sr = s.hi; cr = __fadd_rn(cr, __fadd_rn(s.lo, p.lo));
    cr = __fmaf_rn(b.x, v.x, __fmaf_rn(-b.y, v.y, cr));
    p = two_prod(a.x, v.y);
    s = two_sum(si, p.hi);
    si = s.hi; ci = __fadd_rn(ci, __fadd_rn(s.lo, p.lo));
    p = two_prod(a.y, v.x);
    s = two_sum(si, p.hi);
    si = s.hi; ci = __fadd_rn(ci, __fadd_rn(s.lo, p.lo));
    ci = __fmaf_rn(b.x, v.y, __fmaf_rn(b.y, v.x, ci));
  }
  return make_float2(__fadd_rn(sr, cr), __fadd_rn(si, ci));
}

// Split an FP64 complex into a float pair (hi = rounded, lo = remainder).
__device__ __forceinline__ void split_c(double2 q, float2& hi, float2& lo) {
  hi = make_float2((float)q.x, (float)q.y);
  lo = make_float2((float)(q.x - (double)hi.x), (float)(q.y - (double)hi.y));
}

// MK consecutive complex64 values (vector loads when MK is even: the caller
// guarantees 16-byte alignment then).
template <int MK>
__device__ __forceinline__ void load_block(const float2* __restrict__ p, float2 (&v)[MK]) {
  if constexpr (MK % 2 == 0) {
#pragma unroll
    for (int i = 0; i < MK; i += 2) {
      float4 q = __ldg(reinterpret_cast<const float4*>(p + i));
      v[i] = make_float2(q.x, q.y);
      v[i + 1] = make_float2(q.z, q.w);
    }
  } else {
#pragma unroll
    for (int i = 0; i < MK; ++i) v[i] = __ldg(p + i);
  }
}

// flags[0]: non-finite value produced; flags[1]: IP blocks that took the
// pseudo-inverse path (counter); flags[2]: a bounded device wait gave up.
enum { FLAG_NONFINITE = 0, FLAG_PINV = 1, FLAG_TIMEOUT = 2, FLAG_COUNT = 4 };

// ------------------------------------------------------------ async copies
// cp.async (global -> shared, bypassing registers); groups are committed and
// waited on explicitly.
__device__ __forceinline__ void cp_async4(void* smem, const void* gmem) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

// Dispatch on the subarray size M_k (1..4) as the compile-time constant MK_.
#define DFM_MK_DISPATCH(MKV, ...)                          \
  switch (MKV) {                                           \
    case 1: { constexpr int MK_ = 1; __VA_ARGS__; } break; \
    case 2: { constexpr int MK_ = 2; __VA_ARGS__; } break; \
    case 3: { constexpr int MK_ = 3; __VA_ARGS__; } break; \
    case 4: { constexpr int MK_ = 4; __VA_ARGS__; } break; \
    default: return cudaErrorInvalidValue;                 \
  }

}  // namespace dfm
