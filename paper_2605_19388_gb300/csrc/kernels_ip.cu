// kernels_ip.cu -- iterative projection of the diagonaliser blocks
// (Eqs. 14-15) and the small dense FP64 block kernels (log-determinant,
// inverse, precision conversion).
//
// Layout of the IP kernel: one diagonaliser block Q_fk (M_k <= 4) per
// 16-lane half warp, one matrix element per lane (lane e -> row e / M_k,
// column e % M_k).  For each mu in ascending order the half warp
//   1. forms A = Q_fk V_fk,mu (each lane one entry, M_k complex FMAs),
//   2. solves A q = e_mu by Gauss-Jordan elimination with partial pivoting,
//      exchanging rows and pivots through warp shuffles,
//   3. normalises q <- q / sqrt(max(Re q^H V q, eps)) (Eq. 15) and writes
//      row mu of Q_fk = q^H.
// Gauss-Jordan with partial pivoting selects the same pivots as Gaussian
// elimination with partial pivoting, so the singularity test (smallest
// |pivot| <= rtol * max|A_ij|) is the one of Sec. IV-A's pseudo-inverse rule;
// a singular system is solved with the SVD pseudo-inverse (one-sided Jacobi,
// FP64, one lane), which is the rare path.
//
// The arithmetic type R is a template parameter: IEEE double, float-float
// pairs (dfm::dd) or float.
#include <type_traits>

#include "../../include/dfmnmf.h"
#include "common.cuh"
#include "internal.h"

namespace dfm {

// q = pinv(A) e_mu by one-sided (Hestenes) Jacobi on the columns of A.
// Singular values <= rtol * s_max are dropped.  One thread, FP64.
template <int MK>
__device__ void pinv_column(cx<double> (&U)[MK][MK], int mu, double rtol, cx<double> (&q)[MK]) {
  cx<double> Vm[MK][MK];
#pragma unroll
  for (int r = 0; r < MK; ++r)
#pragma unroll
    for (int c = 0; c < MK; ++c) Vm[r][c] = cmake(r == c ? 1.0 : 0.0, 0.0);
  for (int sweep = 0; sweep < 60; ++sweep) {
    double off = 0.0;
    for (int p = 0; p < MK; ++p)
      for (int qq = p + 1; qq < MK; ++qq) {
        double al = 0.0, be = 0.0, gr = 0.0, gi = 0.0;
        for (int r = 0; r < MK; ++r) {
          al += U[r][p].re * U[r][p].re + U[r][p].im * U[r][p].im;
          be += U[r][qq].re * U[r][qq].re + U[r][qq].im * U[r][qq].im;
          gr += U[r][p].re * U[r][qq].re + U[r][p].im * U[r][qq].im;  // conj(u_p) u_q
          gi += U[r][p].re * U[r][qq].im - U[r][p].im * U[r][qq].re;
        }
        const double gm = sqrt(gr * gr + gi * gi);
        const double nrm = sqrt(al * be);
        if (!(gm > 1e-300) || !(gm > 1e-15 * nrm)) continue;
        off = fmax(off, gm / nrm);
        const double pr = gr / gm, pi = -gi / gm;  // conj(gamma / |gamma|)
        const double zeta = (be - al) / (2.0 * gm);
        const double tt = (zeta >= 0.0 ? 1.0 : -1.0) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
        const double cs = 1.0 / sqrt(1.0 + tt * tt), sn = cs * tt;
        for (int r = 0; r < MK; ++r) {
          cx<double> up = U[r][p], uq = U[r][qq];
          cx<double> uq2 = cmake(uq.re * pr - uq.im * pi, uq.re * pi + uq.im * pr);
          U[r][p] = cmake(cs * up.re - sn * uq2.re, cs * up.im - sn * uq2.im);
          U[r][qq] = cmake(sn * up.re + cs * uq2.re, sn * up.im + cs * uq2.im);
          cx<double> vp = Vm[r][p], vq = Vm[r][qq];
          cx<double> vq2 = cmake(vq.re * pr - vq.im * pi, vq.re * pi + vq.im * pr);
          Vm[r][p] = cmake(cs * vp.re - sn * vq2.re, cs * vp.im - sn * vq2.im);
          Vm[r][qq] = cmake(sn * vp.re + cs * vq2.re, sn * vp.im + cs * vq2.im);
        }
      }
    if (off < 1e-15) break;
  }
  double sig2[MK], smax2 = 0.0;
  for (int c = 0; c < MK; ++c) {
    double s = 0.0;
    for (int r = 0; r < MK; ++r) s += U[r][c].re * U[r][c].re + U[r][c].im * U[r][c].im;
    sig2[c] = s;
    smax2 = fmax(smax2, s);
  }
  for (int r = 0; r < MK; ++r) q[r] = cmake(0.0, 0.0);
  for (int c = 0; c < MK; ++c) {
    if (!(sig2[c] > rtol * rtol * smax2) || !(sig2[c] > 0.0)) continue;
    // coefficient conj(U[mu][c]) / sigma_c^2
    const double cr = U[mu][c].re / sig2[c], ci = -U[mu][c].im / sig2[c];
    for (int r = 0; r < MK; ++r) {
      q[r].re += Vm[r][c].re * cr - Vm[r][c].im * ci;
      q[r].im += Vm[r][c].re * ci + Vm[r][c].im * cr;
    }
  }
}

// V entry as the working type: float pairs come straight from the float-float
// copy (no FP64 instructions), doubles from the FP64 copy.
template <class R> struct VLoad;
template <> struct VLoad<dd> {
  static __device__ __forceinline__ cx<dd> get(const double2*, const float4* vd, size_t i) {
    const float4 v = vd[i];
    return cmake(dd_make(v.x, v.y), dd_make(v.z, v.w));
  }
};
template <> struct VLoad<double> {
  static __device__ __forceinline__ cx<double> get(const double2* v, const float4*, size_t i) {
    return cfrom_d2<double>(v[i]);
  }
};
template <> struct VLoad<float> {
  static __device__ __forceinline__ cx<float> get(const double2*, const float4* vd, size_t i) {
    const float4 v = vd[i];
    return cmake(v.x, v.z);
  }
};

// Eqs. (14)-(15), step 2, in the working precision R: A q = e_mu by Gauss-Jordan elimination with partial
// pivoting on the 16 lanes of a half warp (lane (i, j) holds A_ij; rows exchanged and pivots broadcast by
// shuffles, the first maximum taken on ties), then the singularity test of Sec. IV-A; a singular system is
// solved by lane 0 with the FP64 pseudo-inverse of Q V_mu (Vmu: the FP64 V_mu of the block, qrow: the
// half warp's shared slot for q).  Returns this lane's q_i.
template <int MK, class R>
__device__ __forceinline__ cx<R> ip_gj_solve(cx<R> a, int mu, int i, int j, int e, int sb, bool act, bool valid,
                                             float maxabs, float rtol, const cx<R>* Qb,
                                             const double2* __restrict__ Vmu, cx<double>* qrow, unsigned segmask,
                                             unsigned* __restrict__ flags) {
  using O = RealOps<R>;
  const int lane = threadIdx.x & 31;
  auto L = [&](int r, int c) { return sb + r * MK + c; };
  cx<R> b = (act && i == mu) ? cmake(O::one(), O::zero()) : czero<R>();
  float minpiv = INFINITY;
#pragma unroll
  for (int c = 0; c < MK; ++c) {
    float key = (act && j == c && i >= c) ? cabs2_f(a) : -1.f;
    int prow = i;
#pragma unroll
    for (int o = 8; o > 0; o >>= 1) {
      const float ok = __shfl_xor_sync(DFM_FULL_MASK, key, o);
      const int orow = __shfl_xor_sync(DFM_FULL_MASK, prow, o);
      if (ok > key || (ok == key && orow < prow)) {
        key = ok;
        prow = orow;
      }
    }
    int src = lane;
    if (act && i == c) src = L(prow, j);
    else if (act && i == prow) src = L(c, j);
    a = cshfl(a, src);
    b = cshfl(b, src);
    const cx<R> piv = cshfl(a, L(c, c));
    minpiv = fminf(minpiv, sqrtf(cabs2_f(piv)));
    const cx<R> inv = crecip(piv);
    const cx<R> rowc = cmul(cshfl(a, L(c, j)), inv);
    const cx<R> bc = cmul(cshfl(b, L(c, 0)), inv);
    const cx<R> m = cshfl(a, L(i, c));
    if (i == c) {
      a = rowc;
      b = bc;
    } else {
      a = csub(a, cmul(m, rowc));
      b = csub(b, cmul(m, bc));
    }
  }
  if (minpiv > rtol * maxabs) return b;
  if (e == 0 && valid) {
    cx<double> U[MK][MK], q[MK];
    for (int r = 0; r < MK; ++r)
      for (int c = 0; c < MK; ++c) {
        double sr = 0.0, si = 0.0;
        for (int l = 0; l < MK; ++l) {
          const cx<R> qrl = Qb[r * MK + l];
          const double qr = O::to_d(qrl.re), qim = O::to_d(qrl.im);
          const double2 v = Vmu[l * MK + c];
          sr += qr * v.x - qim * v.y;
          si += qr * v.y + qim * v.x;
        }
        U[r][c] = cmake(sr, si);
      }
    pinv_column<MK>(U, mu, (double)rtol, q);
    for (int r = 0; r < MK; ++r) qrow[r] = q[r];
    atomicAdd(flags + FLAG_PINV, 1u);
  }
  __syncwarp(segmask);
  return cfrom_d2<R>(make_double2(qrow[i].re, qrow[i].im));
}
template <int MK, class R>
__device__ __noinline__ cx<R> ip_gj_solve_outline(cx<R> a, int mu, int i, int j, int e, int sb, bool act,
                                                  bool valid, float maxabs, float rtol, const cx<R>* Qb,
                                                  const double2* __restrict__ Vmu, cx<double>* qrow,
                                                  unsigned segmask, unsigned* __restrict__ flags) {
  return ip_gj_solve<MK, R>(a, mu, i, j, e, sb, act, valid, maxabs, rtol, Qb, Vmu, qrow, segmask, flags);
}

// NREF is the number of float-pair refinement steps of the mixed-precision
// solve (three for the FP32 form; one for the tensor-core form, whose
// covariances already carry a relative error near 2^-16).
template <int MK, class R, int NREF = 3>
__global__ void __launch_bounds__(128) k_ip(const double2* __restrict__ V, const float4* __restrict__ Vdd,
                                            double2* __restrict__ Q64,
                                            float2* __restrict__ Q32, int nblocks, float eps, float rtol,
                                            unsigned* __restrict__ flags) {
  using O = RealOps<R>;
  constexpr bool MIXED = std::is_same<R, dd>::value && (MK == 2 || MK == 4);
  constexpr int E = MK * MK;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int seg = lane >> 4, e = lane & 15, sb = seg << 4;
  const bool act = e < E;
  const int i = act ? e / MK : 0, j = act ? e % MK : 0;
  const int blk = (blockIdx.x * 4 + warp) * 2 + seg;
  const bool valid = blk < nblocks;
  const unsigned segmask = 0xffffu << sb;
  __shared__ cx<R> Qs[4][2][E];
  __shared__ cx<double> qfb[4][2][MK];
  cx<R>* Qb = Qs[warp][seg];
  if (act) {
    if (valid) Qb[e] = cfrom_d2<R>(Q64[(size_t)blk * E + e]);
    else Qb[e] = cmake(i == j ? O::one() : O::zero(), O::zero());
  }
  __syncwarp();
  const size_t vbase = (size_t)(valid ? blk : 0) * E * MK;
  const double2* Vb = V + vbase;
  auto L = [&](int r, int c) { return sb + r * MK + c; };
  // column j of V_mu for the next mu, requested one row update ahead so that its memory latency is not
  // on the chain of dependent steps
  cx<R> vnext[MK];
#pragma unroll
  for (int l = 0; l < MK; ++l) vnext[l] = VLoad<R>::get(V, Vdd, vbase + l * MK + j);

  for (int mu = 0; mu < MK; ++mu) {
    // 1. A = Q V_mu (lane (i, j)) and V_mu[i][j]
    cx<R> vcol[MK];
#pragma unroll
    for (int l = 0; l < MK; ++l) vcol[l] = vnext[l];
    if (mu + 1 < MK) {
#pragma unroll
      for (int l = 0; l < MK; ++l) vnext[l] = VLoad<R>::get(V, Vdd, vbase + (mu + 1) * E + l * MK + j);
    }
    cx<R> a = czero<R>(), vij = czero<R>();
#pragma unroll
    for (int l = 0; l < MK; ++l) {
      const cx<R> vlj = vcol[l];
      a = cadd(a, cmul(Qb[i * MK + l], vlj));
      if (l == i) vij = vlj;
    }
    float maxabs = act ? sqrtf(cabs2_f(a)) : 0.f;
#pragma unroll
    for (int o = 8; o > 0; o >>= 1) maxabs = fmaxf(maxabs, __shfl_xor_sync(DFM_FULL_MASK, maxabs, o));
    cx<R> qi;
    bool solved = false;
    if constexpr (MIXED) {
      // 2a. Mixed precision: Gauss-Jordan in single precision on [A | I] gives an
      // approximate inverse X (lane (i, j) ends with X_ij); NREF refinement
      // steps q <- q + X (e_mu - A q), the residual formed in float pairs from
      // the float-pair A, converge to the float-pair solution when cond(A) u is
      // small.  Taken only when every block of the warp has its smallest single
      // precision pivot above 1e-5 max|A_ij| (far from the singular threshold,
      // so the pseudo-inverse decision cannot differ) and its last correction
      // below 1e-9 |q| (three steps) or 1e-3 |q| (one step: the error left is
      // about the correction times the contraction factor, below 1e-6 |q| at
      // the conditioning of the paper-shaped workload); otherwise the warp
      // redoes the solve in float pairs.
      cx<float> af = cmake(O::to_f(a.re), O::to_f(a.im));
      cx<float> xf = cmake((act && i == j) ? 1.f : 0.f, 0.f);
      float mpf = INFINITY;
#pragma unroll
      for (int c = 0; c < MK; ++c) {
        // pivot row: the largest |a_ic|, i >= c, among the M_k lanes of column c (xor steps of M_k lanes),
        // magnitude and row packed in one word (low three bits 7 - i: the lower row wins a tie), then
        // broadcast from lane (0, c); the singularity decision of this path does not depend on near ties
        unsigned key = (act && j == c && i >= c) ? ((__float_as_uint(cabs2_f(af)) & ~7u) | (unsigned)(7 - i)) : 0u;
#pragma unroll
        for (int o = MK; o < MK * MK; o <<= 1) key = max(key, __shfl_xor_sync(DFM_FULL_MASK, key, o));
        key = __shfl_sync(DFM_FULL_MASK, key, L(0, c));
        const int prow = 7 - (int)(key & 7u);
        int src = lane;
        if (act && i == c) src = L(prow, j);
        else if (act && i == prow) src = L(c, j);
        af = cshfl(af, src);
        xf = cshfl(xf, src);
        const cx<float> piv = cshfl(af, L(c, c));
        mpf = fminf(mpf, sqrtf(cabs2_f(piv)));
        const cx<float> inv = crecip(piv);
        const cx<float> rowc = cmul(cshfl(af, L(c, j)), inv);
        const cx<float> xc = cmul(cshfl(xf, L(c, j)), inv);
        const cx<float> m = cshfl(af, L(i, c));
        if (i == c) {
          af = rowc;
          xf = xc;
        } else {
          af = csub(af, cmul(m, rowc));
          xf = csub(xf, cmul(m, xc));
        }
      }
      if (__all_sync(DFM_FULL_MASK, mpf > 1e-5f * maxabs)) {
        const cx<float> x0 = cshfl(xf, L(i, mu));
        cx<R> q = cmake(O::from_f(x0.re), O::from_f(x0.im));
        float dlast = 0.f;
#pragma unroll
        for (int it = 0; it < NREF; ++it) {
          const cx<R> qj = cshfl(q, L(j, 0));
          cx<R> t = cmul(a, qj);
#pragma unroll
          for (int o = 1; o < MK; o <<= 1) t = cadd(t, cmake(O::shfl_xor(t.re, o), O::shfl_xor(t.im, o)));
          const cx<R> r = csub((i == mu) ? cmake(O::one(), O::zero()) : czero<R>(), t);
          const cx<float> rj = cshfl(cmake(O::to_f(r.re), O::to_f(r.im)), L(j, 0));
          cx<float> d = cmul(xf, rj);
#pragma unroll
          for (int o = 1; o < MK; o <<= 1)
            d = cadd(d, cmake(__shfl_xor_sync(DFM_FULL_MASK, d.re, o), __shfl_xor_sync(DFM_FULL_MASK, d.im, o)));
          q = cadd(q, cmake(O::from_f(d.re), O::from_f(d.im)));
          dlast = act ? sqrtf(cabs2_f(d)) : 0.f;
        }
        float qmax = act ? sqrtf(cabs2_f(q)) : 0.f;
#pragma unroll
        for (int o = 8; o > 0; o >>= 1) {
          dlast = fmaxf(dlast, __shfl_xor_sync(DFM_FULL_MASK, dlast, o));
          qmax = fmaxf(qmax, __shfl_xor_sync(DFM_FULL_MASK, qmax, o));
        }
        constexpr float kAccept = NREF >= 3 ? 1e-9f : 1e-3f;
        if (__all_sync(DFM_FULL_MASK, dlast <= kAccept * qmax)) {
          qi = q;
          solved = true;
        }
      }
    }
    if (!solved) {
      // Gauss-Jordan in the working precision (and the pseudo-inverse when singular); out of line where it
      // is the fallback of the mixed-precision solve, so that the hot path keeps a small code footprint
      if constexpr (MIXED)
        qi = ip_gj_solve_outline<MK, R>(a, mu, i, j, e, sb, act, valid, maxabs, rtol, Qb, Vb + mu * E,
                                        qfb[warp][seg], segmask, flags);
      else
        qi = ip_gj_solve<MK, R>(a, mu, i, j, e, sb, act, valid, maxabs, rtol, Qb, Vb + mu * E, qfb[warp][seg],
                                segmask, flags);
    }
    // 3. normalisation (Eq. 15) and row update
    const cx<R> qj = cshfl(qi, L(j, 0));
    R term = O::zero();
    if (act) {
      const cx<R> vq = cmul(vij, qj);
      term = O::add(O::mul(qi.re, vq.re), O::mul(qi.im, vq.im));  // Re(conj(q_i) V_ij q_j)
    }
#pragma unroll
    for (int o = 8; o > 0; o >>= 1) term = O::add(term, O::shfl_xor(term, o));
    R s = term;
    if (!(O::to_f(s) > eps)) s = O::from_f(eps);
    const R rs = O::div(O::one(), O::sqrt_(s));
    __syncwarp();
    if (act && i == mu) Qb[mu * MK + j] = cscale(cconj(qj), rs);
    __syncwarp();
  }
  if (act && valid) {
    const cx<R> v = Qb[e];
    const double re = O::to_d(v.re), im = O::to_d(v.im);
    if (!isfinite(re) || !isfinite(im)) atomicOr(flags + FLAG_NONFINITE, 1u);
    Q64[(size_t)blk * E + e] = make_double2(re, im);
    Q32[(size_t)blk * E + e] = make_float2((float)re, (float)im);
  }
}

// Pseudo-inverse path of k_ip_all at M_k = 16 (rare): q = pinv(Q V_mu) e_mu
// in FP64 by one thread, kept out of line so that its local arrays do not
// weigh on the registers of the main path.
template <class R>
__device__ __noinline__ void ip16_pinv(const cx<R>* Qs, const double2* Vmu, int mu, float rtol, cx<double>* qout) {
  using O = RealOps<R>;
  constexpr int MK = 16;
  cx<double> U[MK][MK], q[MK];
  for (int r = 0; r < MK; ++r)
    for (int cc = 0; cc < MK; ++cc) {
      double sr = 0.0, si = 0.0;
      for (int l = 0; l < MK; ++l) {
        const cx<R> qrl = Qs[r * MK + l];
        const double qr = O::to_d(qrl.re), qim = O::to_d(qrl.im);
        const double2 v = Vmu[l * MK + cc];
        sr += qr * v.x - qim * v.y;
        si += qr * v.y + qim * v.x;
      }
      U[r][cc] = cmake(sr, si);
    }
  pinv_column<MK>(U, mu, (double)rtol, q);
  for (int r = 0; r < MK; ++r) qout[r] = q[r];
}

__device__ __forceinline__ double warp_sum_all(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(DFM_FULL_MASK, v, o);
  return v;  // every lane holds the same sum (each step adds the same two operands in every lane)
}

// Pseudo-inverse path at M_k = 32 (rare): q = pinv(Q V_mu) e_mu in FP64 by
// one warp, lane r owning row r of U = Q V_mu and of the rotation J, both in
// shared memory (a thread-private 32 x 32 FP64 array would need 16 KB of
// local memory per thread).  One-sided Jacobi rotations on the column pairs
// (p, q) -- the same rotation as pinv_column -- with the column sums of
// |U|^2 and U^H U formed by warp butterflies, so every lane sees the same
// values and the control flow stays uniform.
template <class R, int MK>
__device__ __noinline__ void ip_pinv_warp(const cx<R>* Qs, const double2* Vmu, int mu, float rtol,
                                          cx<double>* qout, cx<double>* U, cx<double>* Jm) {
  using O = RealOps<R>;
  const int lane = threadIdx.x & 31;
  const bool act = lane < MK;
  for (int cc = 0; cc < MK; ++cc) {
    if (act) {
      double sr = 0.0, si = 0.0;
      for (int l = 0; l < MK; ++l) {
        const cx<R> qrl = Qs[lane * MK + l];
        const double qr = O::to_d(qrl.re), qim = O::to_d(qrl.im);
        const double2 v = Vmu[l * MK + cc];
        sr += qr * v.x - qim * v.y;
        si += qr * v.y + qim * v.x;
      }
      U[lane * MK + cc] = cmake(sr, si);
      Jm[lane * MK + cc] = cmake(lane == cc ? 1.0 : 0.0, 0.0);
    }
  }
  __syncwarp();
  for (int sweep = 0; sweep < 60; ++sweep) {
    double off = 0.0;
    for (int p = 0; p < MK; ++p)
      for (int qq = p + 1; qq < MK; ++qq) {
        const cx<double> up = act ? U[lane * MK + p] : cmake(0.0, 0.0);
        const cx<double> uq = act ? U[lane * MK + qq] : cmake(0.0, 0.0);
        const double al = warp_sum_all(up.re * up.re + up.im * up.im);
        const double be = warp_sum_all(uq.re * uq.re + uq.im * uq.im);
        const double gr = warp_sum_all(up.re * uq.re + up.im * uq.im);  // conj(u_p) u_q
        const double gi = warp_sum_all(up.re * uq.im - up.im * uq.re);
        const double gm = sqrt(gr * gr + gi * gi);
        const double nrm = sqrt(al * be);
        if (!(gm > 1e-300) || !(gm > 1e-15 * nrm)) continue;
        off = fmax(off, gm / nrm);
        const double pr = gr / gm, pi = -gi / gm;  // conj(gamma / |gamma|)
        const double zeta = (be - al) / (2.0 * gm);
        const double tt = (zeta >= 0.0 ? 1.0 : -1.0) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
        const double cs = 1.0 / sqrt(1.0 + tt * tt), sn = cs * tt;
        if (act) {
          const cx<double> uq2 = cmake(uq.re * pr - uq.im * pi, uq.re * pi + uq.im * pr);
          U[lane * MK + p] = cmake(cs * up.re - sn * uq2.re, cs * up.im - sn * uq2.im);
          U[lane * MK + qq] = cmake(sn * up.re + cs * uq2.re, sn * up.im + cs * uq2.im);
          const cx<double> vp = Jm[lane * MK + p], vq = Jm[lane * MK + qq];
          const cx<double> vq2 = cmake(vq.re * pr - vq.im * pi, vq.re * pi + vq.im * pr);
          Jm[lane * MK + p] = cmake(cs * vp.re - sn * vq2.re, cs * vp.im - sn * vq2.im);
          Jm[lane * MK + qq] = cmake(sn * vp.re + cs * vq2.re, sn * vp.im + cs * vq2.im);
        }
        __syncwarp();
      }
    if (off < 1e-15) break;
  }
  double smax2 = 0.0;
  for (int cc = 0; cc < MK; ++cc) {
    const cx<double> u = act ? U[lane * MK + cc] : cmake(0.0, 0.0);
    smax2 = fmax(smax2, warp_sum_all(u.re * u.re + u.im * u.im));
  }
  cx<double> q = cmake(0.0, 0.0);
  for (int cc = 0; cc < MK; ++cc) {
    const cx<double> u = act ? U[lane * MK + cc] : cmake(0.0, 0.0);
    const double s2 = warp_sum_all(u.re * u.re + u.im * u.im);
    if (!(s2 > (double)rtol * (double)rtol * smax2) || !(s2 > 0.0)) continue;
    const cx<double> um = U[mu * MK + cc];
    const double cr = um.re / s2, ci = -um.im / s2;  // conj(U[mu][c]) / sigma_c^2
    if (act) {
      const cx<double> v = Jm[lane * MK + cc];
      q.re += v.re * cr - v.im * ci;
      q.im += v.re * ci + v.im * cr;
    }
  }
  if (act) qout[lane] = q;
  __syncwarp();
}

// One all-microphone block per CTA of MK^2 threads (conventional
// FastMNMF, M_k = MK = 16 or 32): thread e owns entry (i, j) = (e / MK,
// e % MK).  For mu ascending: V_mu is staged in shared memory, A = Q V_mu
// formed entry by entry, A q = e_mu solved by Gauss-Jordan elimination with
// partial pivoting (each warp finds the pivot row by a butterfly over the
// column's magnitudes, first maximum on ties; rows are exchanged through
// shared memory), then Eq. (15) with a block reduction of Re q^H V q.  The
// singularity test and the pseudo-inverse fallback are those of k_ip.
template <int MK, class R>
__global__ void __launch_bounds__(MK * MK, MK <= 16 ? 2 : 1) k_ip_all(const double2* __restrict__ V, const float4* __restrict__ Vdd,
                                                     double2* __restrict__ Q64, float2* __restrict__ Q32, float eps,
                                                     float rtol, unsigned* __restrict__ flags) {
  using O = RealOps<R>;
  constexpr int E = MK * MK, NW = E / 32;
  const int blk = blockIdx.x;
  const int e = threadIdx.x, i = e / MK, j = e % MK, lane = e & 31, warp = e >> 5;
  extern __shared__ __align__(16) unsigned char smip[];
  cx<R>* Qs = reinterpret_cast<cx<R>*>(smip);
  cx<R>* As = Qs + E;
  cx<R>* Vs = As + E;
  cx<double>* Ub = reinterpret_cast<cx<double>*>(Vs + E);  // [MK][MK] pinv workspace (MK = 32 only)
  cx<double>* Jb = Ub + E;
  __shared__ cx<R> bs[MK];
  __shared__ float keys[MK], wmax[NW];
  __shared__ R wred[NW];
  __shared__ cx<double> qfb[MK];
  Qs[e] = cfrom_d2<R>(Q64[(size_t)blk * E + e]);
  const size_t vbase = (size_t)blk * E * MK;
  const double2* Vb = V + vbase;
  for (int mu = 0; mu < MK; ++mu) {
    Vs[e] = VLoad<R>::get(V, Vdd, vbase + (size_t)mu * E + e);
    __syncthreads();
    // 1. A = Q V_mu
    cx<R> a = czero<R>();
    for (int l = 0; l < MK; ++l) a = cadd(a, cmul(Qs[i * MK + l], Vs[l * MK + j]));
    float m = sqrtf(cabs2_f(a));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(DFM_FULL_MASK, m, o));
    if (lane == 0) wmax[warp] = m;
    cx<R> bv = (i == mu) ? cmake(O::one(), O::zero()) : czero<R>();
    float minpiv = INFINITY;
    // 2. Gauss-Jordan with partial pivoting (b held by the threads of column 0)
    for (int c = 0; c < MK; ++c) {
      As[e] = a;
      if (j == 0) bs[i] = bv;
      if (j == c) {
        const float kv = cabs2_f(a);
        keys[i] = (i >= c) ? (kv == kv ? kv : -1.5f) : -1.f;  // rows above c never pivot; NaN never wins
      }
      __syncthreads();
      float best = lane < MK ? keys[lane] : -2.f;
      int prow = lane;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        const float ob = __shfl_xor_sync(DFM_FULL_MASK, best, o);
        const int op = __shfl_xor_sync(DFM_FULL_MASK, prow, o);
        if (ob > best || (ob == best && op < prow)) {
          best = ob;
          prow = op;
        }
      }
      const int ri = (i == c) ? prow : (i == prow ? c : i);  // this thread's row after the exchange
      const cx<R> piv = As[prow * MK + c];
      minpiv = fminf(minpiv, sqrtf(cabs2_f(piv)));
      const cx<R> inv = crecip(piv);
      const cx<R> rowc = cmul(As[prow * MK + j], inv);
      const cx<R> bc = cmul(bs[prow], inv);
      if (i == c) {
        a = rowc;
        bv = bc;
      } else {
        const cx<R> mi = As[ri * MK + c];
        a = csub(As[ri * MK + j], cmul(mi, rowc));
        bv = csub(bs[ri], cmul(mi, bc));
      }
      __syncthreads();
    }
    float maxabs = 0.f;
#pragma unroll
    for (int w = 0; w < NW; ++w) maxabs = fmaxf(maxabs, wmax[w]);
    const bool singular = !(minpiv > rtol * maxabs);
    if (singular) {
      if constexpr (MK <= 16) {
        if (e == 0) ip16_pinv<R>(Qs, Vb + (size_t)mu * E, mu, rtol, qfb);
      } else {
        if (warp == 0) ip_pinv_warp<R, MK>(Qs, Vb + (size_t)mu * E, mu, rtol, qfb, Ub, Jb);
      }
      if (e == 0) atomicAdd(flags + FLAG_PINV, 1u);
    } else if (j == 0) {
      qfb[i] = cmake(O::to_d(bv.re), O::to_d(bv.im));  // float pairs are exact in FP64
    }
    __syncthreads();
    // 3. normalisation (Eq. 15): s = Re q^H V q over the block
    const cx<R> qi = cfrom_d2<R>(make_double2(qfb[i].re, qfb[i].im));
    const cx<R> qj = cfrom_d2<R>(make_double2(qfb[j].re, qfb[j].im));
    const cx<R> vq = cmul(Vs[e], qj);
    R term = O::add(O::mul(qi.re, vq.re), O::mul(qi.im, vq.im));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) term = O::add(term, O::shfl_xor(term, o));
    if (lane == 0) wred[warp] = term;
    __syncthreads();
    R sum = O::zero();
#pragma unroll
    for (int w = 0; w < NW; ++w) sum = O::add(sum, wred[w]);
    if (!(O::to_f(sum) > eps)) sum = O::from_f(eps);
    const R rs = O::div(O::one(), O::sqrt_(sum));
    if (i == mu) Qs[mu * MK + j] = cscale(cconj(qj), rs);
    __syncthreads();
  }
  const cx<R> v = Qs[e];
  const double re = O::to_d(v.re), im = O::to_d(v.im);
  if (!isfinite(re) || !isfinite(im)) atomicOr(flags + FLAG_NONFINITE, 1u);
  Q64[(size_t)blk * E + e] = make_double2(re, im);
  Q32[(size_t)blk * E + e] = make_float2((float)re, (float)im);
}

template <int MK, class R>
static void launch_ip_all_k(const dfmnmf_ctx* c, cudaStream_t s, int nblocks, size_t o) {
  constexpr int E = MK * MK;
  const size_t sm = 3 * (size_t)E * sizeof(cx<R>) + (MK > 16 ? 2 * (size_t)E * sizeof(cx<double>) : 0);
  auto kern = k_ip_all<MK, R>;
  if (sm > 48 * 1024) cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  const size_t ov = o * E * MK, oq = o * E;
  kern<<<nblocks, E, sm, s>>>(c->V + ov, c->Vdd + ov, c->Q64 + oq, c->Q32 + oq, c->eps, c->singular_rtol, c->flags);
}

template <int MK>
static cudaError_t launch_ip_all(const dfmnmf_ctx* c, cudaStream_t s, int nblocks, size_t o) {
  switch (c->ip_arith) {
    case 0: launch_ip_all_k<MK, double>(c, s, nblocks, o); break;
    case 1: launch_ip_all_k<MK, dd>(c, s, nblocks, o); break;
    default: launch_ip_all_k<MK, float>(c, s, nblocks, o); break;
  }
  return cudaGetLastError();
}

// ln |det Q_fk|^2 by FP64 Gaussian elimination with partial pivoting, one
// thread per block.
template <int MK>
__global__ void k_logdet(const double2* __restrict__ Q64, double* __restrict__ out, int nblocks) {
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
    if (p != c)
      for (int q = 0; q < MK; ++q) {
        double t = ar[c][q]; ar[c][q] = ar[p][q]; ar[p][q] = t;
        t = ai[c][q]; ai[c][q] = ai[p][q]; ai[p][q] = t;
      }
    acc += log(best);
    if (!(best > 0.0)) continue;
    for (int r = c + 1; r < MK; ++r) {
      // m = a[r][c] / a[c][c]
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

// Q_fk^{-1} by FP64 Gauss-Jordan with partial pivoting, one thread per block.
template <int MK>
__global__ void k_qinv(const double2* __restrict__ Q64, float2* __restrict__ Qinv, int nblocks,
                       unsigned* __restrict__ flags) {
  const int blk = blockIdx.x * blockDim.x + threadIdx.x;
  if (blk >= nblocks) return;
  double ar[MK][2 * MK], ai[MK][2 * MK];
  for (int r = 0; r < MK; ++r)
    for (int c = 0; c < MK; ++c) {
      const double2 v = Q64[(size_t)blk * MK * MK + r * MK + c];
      ar[r][c] = v.x;
      ai[r][c] = v.y;
      ar[r][MK + c] = (r == c) ? 1.0 : 0.0;
      ai[r][MK + c] = 0.0;
    }
  for (int c = 0; c < MK; ++c) {
    int p = c;
    double best = ar[c][c] * ar[c][c] + ai[c][c] * ai[c][c];
    for (int r = c + 1; r < MK; ++r) {
      const double m = ar[r][c] * ar[r][c] + ai[r][c] * ai[r][c];
      if (m > best) { best = m; p = r; }
    }
    if (!(best > 0.0)) { atomicOr(flags + FLAG_NONFINITE, 1u); best = 1.0; }
    if (p != c)
      for (int q = 0; q < 2 * MK; ++q) {
        double t = ar[c][q]; ar[c][q] = ar[p][q]; ar[p][q] = t;
        t = ai[c][q]; ai[c][q] = ai[p][q]; ai[p][q] = t;
      }
    const double ir = ar[c][c] / best, ii = -ai[c][c] / best;  // 1 / pivot
    for (int q = 0; q < 2 * MK; ++q) {
      const double xr = ar[c][q], xi = ai[c][q];
      ar[c][q] = xr * ir - xi * ii;
      ai[c][q] = xr * ii + xi * ir;
    }
    for (int r = 0; r < MK; ++r) {
      if (r == c) continue;
      const double mr = ar[r][c], mi = ai[r][c];
      for (int q = 0; q < 2 * MK; ++q) {
        ar[r][q] -= mr * ar[c][q] - mi * ai[c][q];
        ai[r][q] -= mr * ai[c][q] + mi * ar[c][q];
      }
    }
  }
  for (int r = 0; r < MK; ++r)
    for (int c = 0; c < MK; ++c)
      Qinv[(size_t)blk * MK * MK + r * MK + c] = make_float2((float)ar[r][MK + c], (float)ai[r][MK + c]);
}

// Warp-per-block forms of k_logdet and k_qinv for the 32 x 32 all-microphone
// blocks: the matrix (and the identity it is reduced against) sits in shared
// memory, lane q owning columns q and q + 32; the pivot row is found by a
// butterfly over the lanes (lane r reads row r), first maximum on ties, as
// in the one-thread forms.
__device__ __forceinline__ void warp_argmax_first(double& best, int& row) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const double ob = __shfl_xor_sync(DFM_FULL_MASK, best, o);
    const int orow = __shfl_xor_sync(DFM_FULL_MASK, row, o);
    if (ob > best || (ob == best && orow < row)) {
      best = ob;
      row = orow;
    }
  }
}

template <int MK>
__global__ void __launch_bounds__(32) k_logdet_w(const double2* __restrict__ Q64, double* __restrict__ out,
                                                 int nblocks) {
  extern __shared__ __align__(16) double2 sld[];  // [MK][MK]
  const int blk = blockIdx.x, lane = threadIdx.x;
  for (int i = lane; i < MK * MK; i += 32) sld[i] = Q64[(size_t)blk * MK * MK + i];
  __syncwarp();
  double acc = 0.0;
  for (int c = 0; c < MK; ++c) {
    double best = -1.0;
    int p = lane;
    if (lane >= c && lane < MK) {
      const double2 v = sld[lane * MK + c];
      best = v.x * v.x + v.y * v.y;
      if (!(best == best)) best = -0.5;
    }
    warp_argmax_first(best, p);
    if (p != c)
      for (int q = lane; q < MK; q += 32) {
        const double2 t = sld[c * MK + q];
        sld[c * MK + q] = sld[p * MK + q];
        sld[p * MK + q] = t;
      }
    __syncwarp();
    const double2 pv = sld[c * MK + c];
    const double b2 = pv.x * pv.x + pv.y * pv.y;
    acc += log(b2);
    if (!(b2 > 0.0)) continue;
    for (int r = c + 1; r < MK; ++r) {
      const double2 arc = sld[r * MK + c];
      const double mr = (arc.x * pv.x + arc.y * pv.y) / b2;  // a[r][c] / a[c][c]
      const double mi = (arc.y * pv.x - arc.x * pv.y) / b2;
      __syncwarp();
      for (int q = c + lane; q < MK; q += 32) {
        const double2 cq = sld[c * MK + q];
        double2 v = sld[r * MK + q];
        v.x -= mr * cq.x - mi * cq.y;
        v.y -= mr * cq.y + mi * cq.x;
        sld[r * MK + q] = v;
      }
      __syncwarp();
    }
  }
  if (lane == 0) out[blk] = acc;
}

template <int MK>
__global__ void __launch_bounds__(32) k_qinv_w(const double2* __restrict__ Q64, float2* __restrict__ Qinv,
                                               int nblocks, unsigned* __restrict__ flags) {
  extern __shared__ __align__(16) double2 sqi[];  // [MK][2 MK]: [Q | I] reduced to [I | Q^-1]
  constexpr int W2 = 2 * MK;
  const int blk = blockIdx.x, lane = threadIdx.x;
  for (int i = lane; i < MK * W2; i += 32) {
    const int r = i / W2, q = i % W2;
    sqi[i] = q < MK ? Q64[(size_t)blk * MK * MK + r * MK + q] : make_double2(q - MK == r ? 1.0 : 0.0, 0.0);
  }
  __syncwarp();
  for (int c = 0; c < MK; ++c) {
    double best = -1.0;
    int p = lane;
    if (lane >= c && lane < MK) {
      const double2 v = sqi[lane * W2 + c];
      best = v.x * v.x + v.y * v.y;
      if (!(best == best)) best = -0.5;
    }
    warp_argmax_first(best, p);
    if (p != c)
      for (int q = lane; q < W2; q += 32) {
        const double2 t = sqi[c * W2 + q];
        sqi[c * W2 + q] = sqi[p * W2 + q];
        sqi[p * W2 + q] = t;
      }
    __syncwarp();
    const double2 pv = sqi[c * W2 + c];
    double b2 = pv.x * pv.x + pv.y * pv.y;
    if (!(b2 > 0.0)) {
      if (lane == 0) atomicOr(flags + FLAG_NONFINITE, 1u);
      b2 = 1.0;
    }
    const double ir = pv.x / b2, ii = -pv.y / b2;  // 1 / pivot
    __syncwarp();
    for (int q = lane; q < W2; q += 32) {
      const double2 x = sqi[c * W2 + q];
      sqi[c * W2 + q] = make_double2(x.x * ir - x.y * ii, x.x * ii + x.y * ir);
    }
    __syncwarp();
    for (int r = 0; r < MK; ++r) {
      if (r == c) continue;
      const double2 m = sqi[r * W2 + c];
      __syncwarp();
      for (int q = lane; q < W2; q += 32) {
        const double2 cq = sqi[c * W2 + q];
        double2 v = sqi[r * W2 + q];
        v.x -= m.x * cq.x - m.y * cq.y;
        v.y -= m.x * cq.y + m.y * cq.x;
        sqi[r * W2 + q] = v;
      }
      __syncwarp();
    }
  }
  for (int i = lane; i < MK * MK; i += 32) {
    const double2 v = sqi[(i / MK) * W2 + MK + i % MK];
    Qinv[(size_t)blk * MK * MK + i] = make_float2((float)v.x, (float)v.y);
  }
}

// Gradient of Eq. (12) with respect to one block Q_fk, packed as
// dL/dRe + i dL/dIm:  dQ[mu][j] = 2 T ((Q V_mu)[mu][j] - conj(Q^{-1})[j][mu]),
// where (Q V_mu)[mu][:] = (1/T) sum_t z_mu conj(x) / yhat_mu is the data term
// of the cost (Eq. 13's V) and -T ln|det Q|^2 contributes -conj(Q^{-1})^T.
// FP64, one thread per block (Gauss-Jordan inverse with partial pivoting).
template <int MK>
__global__ void k_qgrad(const double2* __restrict__ Q64, const double2* __restrict__ V, double2* __restrict__ dQ,
                        int nblocks, int T, unsigned* __restrict__ flags) {
  const int blk = blockIdx.x * blockDim.x + threadIdx.x;
  if (blk >= nblocks) return;
  constexpr int E = MK * MK;
  double ar[MK][2 * MK], ai[MK][2 * MK];
  for (int r = 0; r < MK; ++r)
    for (int c = 0; c < MK; ++c) {
      const double2 v = Q64[(size_t)blk * E + r * MK + c];
      ar[r][c] = v.x;
      ai[r][c] = v.y;
      ar[r][MK + c] = (r == c) ? 1.0 : 0.0;
      ai[r][MK + c] = 0.0;
    }
  bool ok = true;
  for (int c = 0; c < MK; ++c) {
    int p = c;
    double best = ar[c][c] * ar[c][c] + ai[c][c] * ai[c][c];
    for (int r = c + 1; r < MK; ++r) {
      const double m = ar[r][c] * ar[r][c] + ai[r][c] * ai[r][c];
      if (m > best) { best = m; p = r; }
    }
    if (!(best > 0.0)) { ok = false; best = 1.0; }
    if (p != c)
      for (int q = 0; q < 2 * MK; ++q) {
        double t = ar[c][q]; ar[c][q] = ar[p][q]; ar[p][q] = t;
        t = ai[c][q]; ai[c][q] = ai[p][q]; ai[p][q] = t;
      }
    const double ir = ar[c][c] / best, ii = -ai[c][c] / best;
    for (int q = 0; q < 2 * MK; ++q) {
      const double xr = ar[c][q], xi = ai[c][q];
      ar[c][q] = xr * ir - xi * ii;
      ai[c][q] = xr * ii + xi * ir;
    }
    for (int r = 0; r < MK; ++r) {
      if (r == c) continue;
      const double mr = ar[r][c], mi = ai[r][c];
      for (int q = 0; q < 2 * MK; ++q) {
        ar[r][q] -= mr * ar[c][q] - mi * ai[c][q];
        ai[r][q] -= mr * ai[c][q] + mi * ar[c][q];
      }
    }
  }
  if (!ok) atomicOr(flags + FLAG_NONFINITE, 1u);
  const double t2 = 2.0 * (double)T;
  for (int mu = 0; mu < MK; ++mu) {
    const double2* Vm = V + ((size_t)blk * MK + mu) * E;
    for (int j = 0; j < MK; ++j) {
      double sr = 0.0, si = 0.0;
      for (int l = 0; l < MK; ++l) {
        const double2 q = Q64[(size_t)blk * E + mu * MK + l], v = Vm[l * MK + j];
        sr += q.x * v.x - q.y * v.y;
        si += q.x * v.y + q.y * v.x;
      }
      // conj(Q^{-1})[j][mu]
      const double gr = t2 * (sr - ar[j][MK + mu]), gi = t2 * (si + ai[j][MK + mu]);
      dQ[(size_t)blk * E + mu * MK + j] = make_double2(gr, gi);
    }
  }
}

cudaError_t launch_qgrad(const dfmnmf_ctx* c, double2* dQ, cudaStream_t s) {
  const int nblocks = c->F * c->K;
  if (c->MK == 16) {
    k_qgrad<16><<<(nblocks + 63) / 64, 64, 0, s>>>(c->Q64, c->V, dQ, nblocks, c->T, c->flags);
    return cudaGetLastError();
  }
  DFM_MK_DISPATCH(c->MK, {
    k_qgrad<MK_><<<(nblocks + 127) / 128, 128, 0, s>>>(c->Q64, c->V, dQ, nblocks, c->T, c->flags);
  });
  return cudaGetLastError();
}

__global__ void k_q32(const double2* __restrict__ Q64, float2* __restrict__ Q32, size_t n) {
  const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) Q32[i] = make_float2((float)Q64[i].x, (float)Q64[i].y);
}


cudaError_t launch_ip(const dfmnmf_ctx* c, cudaStream_t s, int fb, int fc) {
  const int nblocks = fc * c->K;
  const size_t o = (size_t)fb * c->K;  // first block of the range
  if (c->MK == 16) return launch_ip_all<16>(c, s, nblocks, o);
  if (c->MK == 32) return launch_ip_all<32>(c, s, nblocks, o);
  const int grid = (nblocks + 7) / 8;  // 4 warps x 2 blocks per CTA
  DFM_MK_DISPATCH(c->MK, {
    switch (c->ip_arith) {
      case 0: k_ip<MK_, double><<<grid, 128, 0, s>>>(c->V + o * MK_ * MK_ * MK_, c->Vdd + o * MK_ * MK_ * MK_, c->Q64 + o * MK_ * MK_, c->Q32 + o * MK_ * MK_, nblocks, c->eps, c->singular_rtol, c->flags); break;
      case 1:
        if (is_tc(c->precision))
          k_ip<MK_, dd, 1><<<grid, 128, 0, s>>>(c->V + o * MK_ * MK_ * MK_, c->Vdd + o * MK_ * MK_ * MK_, c->Q64 + o * MK_ * MK_, c->Q32 + o * MK_ * MK_, nblocks, c->eps, c->singular_rtol, c->flags);
        else
          k_ip<MK_, dd><<<grid, 128, 0, s>>>(c->V + o * MK_ * MK_ * MK_, c->Vdd + o * MK_ * MK_ * MK_, c->Q64 + o * MK_ * MK_, c->Q32 + o * MK_ * MK_, nblocks, c->eps, c->singular_rtol, c->flags);
        break;
      default: k_ip<MK_, float><<<grid, 128, 0, s>>>(c->V + o * MK_ * MK_ * MK_, c->Vdd + o * MK_ * MK_ * MK_, c->Q64 + o * MK_ * MK_, c->Q32 + o * MK_ * MK_, nblocks, c->eps, c->singular_rtol, c->flags); break;
    }
  });
  return cudaGetLastError();
}

cudaError_t launch_logdet(const dfmnmf_ctx* c, double* out, cudaStream_t s) {
  const int nblocks = c->F * c->K;
  if (c->MK == 16) {
    k_logdet<16><<<(nblocks + 127) / 128, 128, 0, s>>>(c->Q64, out, nblocks);
    return cudaGetLastError();
  }
  if (c->MK == 32) {
    k_logdet_w<32><<<nblocks, 32, 32 * 32 * sizeof(double2), s>>>(c->Q64, out, nblocks);
    return cudaGetLastError();
  }
  DFM_MK_DISPATCH(c->MK, { k_logdet<MK_><<<(nblocks + 127) / 128, 128, 0, s>>>(c->Q64, out, nblocks); });
  return cudaGetLastError();
}

cudaError_t launch_qinv(const dfmnmf_ctx* c, cudaStream_t s) {
  const int nblocks = c->F * c->K;
  if (c->MK == 16) {
    k_qinv<16><<<(nblocks + 127) / 128, 128, 0, s>>>(c->Q64, c->Qinv32, nblocks, c->flags);
    return cudaGetLastError();
  }
  if (c->MK == 32) {
    k_qinv_w<32><<<nblocks, 32, 32 * 64 * sizeof(double2), s>>>(c->Q64, c->Qinv32, nblocks, c->flags);
    return cudaGetLastError();
  }
  DFM_MK_DISPATCH(c->MK, { k_qinv<MK_><<<(nblocks + 127) / 128, 128, 0, s>>>(c->Q64, c->Qinv32, nblocks, c->flags); });
  return cudaGetLastError();
}

cudaError_t launch_q_convert(const dfmnmf_ctx* c, cudaStream_t s) {
  const size_t n = (size_t)c->F * c->K * c->MK * c->MK;
  k_q32<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(c->Q64, c->Q32, n);
  return cudaGetLastError();
}

}  // namespace dfm
