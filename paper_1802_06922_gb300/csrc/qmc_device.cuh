// Device building blocks: counter-based draws, periodic geometry, B-spline weights,
// Jastrow functors and block reductions.
#pragma once
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "qmc_internal.h"

namespace qmcgb {

// ------------------------------------------------------------------ Philox4x32-10
// Counter-based generator of Salmon et al. (SC'11): ten rounds of two 32x32->64-bit
// multiplications whose halves are XOR-mixed with the other two words and the key; the
// key is bumped by the two Weyl constants between rounds.
struct U32x4 { uint32_t v[4]; };

__device__ __forceinline__ U32x4 philox4x32_10(uint32_t c0, uint32_t c1, uint32_t c2,
                                               uint32_t c3, uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    if (r) { k0 += 0x9E3779B9u; k1 += 0xBB67AE85u; }
    const uint32_t lo0 = 0xD2511F53u * c0, hi0 = __umulhi(0xD2511F53u, c0);
    const uint32_t lo1 = 0xCD9E8D57u * c2, hi1 = __umulhi(0xCD9E8D57u, c2);
    const uint32_t n0 = hi1 ^ c1 ^ k0, n2 = hi0 ^ c3 ^ k1;
    c0 = n0; c1 = lo1; c2 = n2; c3 = lo0;
  }
  U32x4 o; o.v[0] = c0; o.v[1] = c1; o.v[2] = c2; o.v[3] = c3;
  return o;
}

// Word -> open interval (0, 1): (w + 0.5) 2^-32, exact in double.
__device__ __forceinline__ double unit_open(uint32_t w) { return ((double)w + 0.5) * 0x1p-32; }

// Acceptance variate of the move of electron e of walker `wid` in sweep t (counter
// (t, e, wid, 1), first word).
__device__ __forceinline__ double move_u(const SysParams& S, uint32_t t, uint32_t e, uint32_t wid) {
  return unit_open(philox4x32_10(t, e, wid, 1u, S.seed_lo, S.seed_hi).v[0]);
}

// Gaussian displacement (Box-Muller on word pairs (0,1) and (2,3)) and acceptance
// variate of the move of electron e of walker `wid` in sweep t (trial move of
// Sec. "Trial Moves"; counter layout (t, e, wid, 0|1)).
__device__ __forceinline__ void move_draws(const SysParams& S, uint32_t t, uint32_t e,
                                           uint32_t wid, double xi[3], double& u) {
  const U32x4 a = philox4x32_10(t, e, wid, 0u, S.seed_lo, S.seed_hi);
  const double r1 = sqrt(-2.0 * log(unit_open(a.v[0])));
  const double g1 = 2.0 * M_PI * unit_open(a.v[1]);
  xi[0] = r1 * cos(g1);
  xi[1] = r1 * sin(g1);
  const double r2 = sqrt(-2.0 * log(unit_open(a.v[2])));
  xi[2] = r2 * cos(2.0 * M_PI * unit_open(a.v[3]));
  u = move_u(S, t, e, wid);
}

// Drift part of a drift-diffusion step for drift velocity v = grad_e ln|Psi|: tau v, or with
// a > 0 the nodal rescaling of Umrigar, Nightingale and Runge (J. Chem. Phys. 99, 2865 (1993);
// Sec. "Projector Monte Carlo"): tau v (-1 + sqrt(1 + 2 a |v|^2 tau)) / (a |v|^2 tau), written
// as tau v 2 / (1 + sqrt(1 + 2 a |v|^2 tau)), which stays below sqrt(2 tau / a) next to a node.
__device__ __forceinline__ void drift_disp(const double v[3], double tau, double a, double out[3]) {
  double f = tau;
  if (a > 0.0) {
    const double x = 2.0 * a * (v[0] * v[0] + v[1] * v[1] + v[2] * v[2]) * tau;
    if (!(x < 1e-12)) f = tau * 2.0 / (1.0 + sqrt(1.0 + x));
  }
  out[0] = f * v[0];
  out[1] = f * v[1];
  out[2] = f * v[2];
}

// ------------------------------------------------------------------ geometry
// Wrap into [0, L): the sign-corrected remainder.
__device__ __forceinline__ double wrap_box(double x, double L) {
  double m = fmod(x, L);
  if (m != 0.0 && m < 0.0) m += L;
  return m;
}
__device__ __forceinline__ double tfloor(double x) { return floor(x); }
__device__ __forceinline__ float tfloor(float x) { return floorf(x); }
__device__ __forceinline__ double trint(double x) { return rint(x); }
__device__ __forceinline__ float trint(float x) { return rintf(x); }
template <class T>
__device__ __forceinline__ T min_image(T d, T L) { return d - L * trint(d / L); }
// The same with the reciprocal of L precomputed (no division in the pair loops).
template <class T>
__device__ __forceinline__ T min_image(T d, T L, T invL) { return d - L * trint(d * invL); }

// ------------------------------------------------------------------ B-spline weights
// Uniform cubic B-spline weights of the nodes i-1..i+2 at fractional position t, and
// their first and second derivatives (Sec. "B-spline basis sets").
template <class T>
__device__ __forceinline__ void bspline_w(T t, T b[4], T db[4], T d2b[4]) {
  const T t2 = t * t, t3 = t2 * t, omt = T(1) - t;
  b[0] = omt * omt * omt * T(1.0 / 6.0);
  b[1] = (T(3) * t3 - T(6) * t2 + T(4)) * T(1.0 / 6.0);
  b[2] = (T(-3) * t3 + T(3) * t2 + T(3) * t + T(1)) * T(1.0 / 6.0);
  b[3] = t3 * T(1.0 / 6.0);
  db[0] = T(-0.5) * omt * omt;
  db[1] = T(1.5) * t2 - T(2) * t;
  db[2] = T(-1.5) * t2 + t + T(0.5);
  db[3] = T(0.5) * t2;
  d2b[0] = omt;
  d2b[1] = T(3) * t - T(2);
  d2b[2] = T(1) - T(3) * t;
  d2b[3] = t;
}

// One radial Jastrow functor u(r), u'(r), u''(r): the four control points p_i..p_{i+3}
// with i = floor(r M / rc) weighted by the cubic B-spline basis at t = r M / rc - i
// (p_m = 0 for m > M; u = 0 for r >= rc). Sec. "Jastrow factor".
// Precision-matched views of the system constants (no double<->float conversion in the
// single-precision kernels: on this GPU those run on the slow FP64 pipe).
template <class T> struct Cst;
template <> struct Cst<double> {
  __device__ static __forceinline__ double knot(const SysParams& S, int f, int m) { return S.jp[f][m]; }
  __device__ static __forceinline__ double rc(const SysParams& S, int f) { return S.jrc[f]; }
  __device__ static __forceinline__ double L(const SysParams& S) { return S.L; }
  __device__ static __forceinline__ double invL(const SysParams& S) { return S.invL; }
  __device__ static __forceinline__ const double* ions(const SysParams& S) { return S.ions; }
  __device__ static __forceinline__ double invd(const SysParams& S, int d) { return S.inv_delta[d]; }
  __device__ static __forceinline__ double Z(const SysParams& S) { return S.ion_Z; }
  __device__ static __forceinline__ double kappa(const SysParams& S) { return S.kappa; }
  __device__ static __forceinline__ double alpha(const SysParams& S) { return S.ew_alpha; }
};
template <> struct Cst<float> {
  __device__ static __forceinline__ float knot(const SysParams& S, int f, int m) { return S.jpf[f][m]; }
  __device__ static __forceinline__ float rc(const SysParams& S, int f) { return S.jrcf[f]; }
  __device__ static __forceinline__ float L(const SysParams& S) { return S.Lf; }
  __device__ static __forceinline__ float invL(const SysParams& S) { return S.invLf; }
  __device__ static __forceinline__ const float* ions(const SysParams& S) { return S.ionsf; }
  __device__ static __forceinline__ float invd(const SysParams& S, int d) { return S.inv_deltaf[d]; }
  __device__ static __forceinline__ float Z(const SysParams& S) { return S.ion_Zf; }
  __device__ static __forceinline__ float kappa(const SysParams& S) { return S.kappaf; }
  __device__ static __forceinline__ float alpha(const SysParams& S) { return S.ew_alphaf; }
};

template <class T>
__device__ __forceinline__ void jastrow_u(const SysParams& S, int f, T r, T& u, T& du, T& d2u) {
  u = du = d2u = T(0);
  const int M = S.jM[f];
  const T rc = Cst<T>::rc(S, f);
  if (M == 0 || !(r < rc)) return;
  const T scale = T(M) / rc;
  const T s = r * scale;
  int i = (int)tfloor(s);
  if (i < 0) i = 0;
  const T t = s - T(i);
  T b[4], db[4], d2b[4];
  bspline_w<T>(t, b, db, d2b);
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int m = i + q;
    const T p = (m <= M) ? Cst<T>::knot(S, f, m) : T(0);
    u += p * b[q];
    du += p * db[q];
    d2u += p * d2b[q];
  }
  du *= scale;
  d2u *= scale * scale;
}

// The three radial functors staged in shared memory: reading knots through a per-thread
// index from kernel parameters would serialise the constant-bank accesses of a warp.
// p is zero-padded beyond M so the four-point stencil needs no bounds test.
// pw holds the same spline in power form per knot interval, u = a0 + a1 t + a2 t^2 + a3 t^3
// (the cubic B-spline basis expanded and summed with the interval's four knots, in FP64),
// so that a value costs one 16-byte load and three FMAs.
// plo and scale_lo hold the rounding residues of the knots and of the scale M / r_c (zero
// in double precision): the J value of ln|Psi| sums ~10^5 pair terms, and a constant
// rounded once would shift every term the same way, moving J by ~2^-24 |J| (see
// jastrow_value6).
template <class T>
struct JastrowTab {
  int M[3];
  T rc[3], rc2[3], scale[3], scale_lo[3];
  T p[3][kMaxKnots + 4];
  T plo[3][kMaxKnots + 4];
  alignas(16) T pw[3][kMaxKnots + 1][4];
};

template <class T>
__device__ __forceinline__ void jastrow_tab_fill(const SysParams& S, JastrowTab<T>& J) {
  for (int i = threadIdx.x; i < 3 * (kMaxKnots + 4); i += blockDim.x) {
    const int f = i / (kMaxKnots + 4), m = i % (kMaxKnots + 4);
    J.p[f][m] = (m <= S.jM[f]) ? Cst<T>::knot(S, f, m) : T(0);
    J.plo[f][m] = (m <= S.jM[f]) ? T(S.jp[f][m] - (double)Cst<T>::knot(S, f, m)) : T(0);
  }
  for (int i = threadIdx.x; i < 3 * (kMaxKnots + 1); i += blockDim.x) {
    const int f = i / (kMaxKnots + 1), m = i % (kMaxKnots + 1);
    double q[4];
#pragma unroll
    for (int c = 0; c < 4; ++c) q[c] = (m + c <= S.jM[f]) ? S.jp[f][m + c] : 0.0;
    J.pw[f][m][0] = T((q[0] + 4.0 * q[1] + q[2]) / 6.0);
    J.pw[f][m][1] = T(0.5 * (q[2] - q[0]));
    J.pw[f][m][2] = T(0.5 * (q[0] - 2.0 * q[1] + q[2]));
    J.pw[f][m][3] = T((q[3] - q[0] + 3.0 * (q[1] - q[2])) / 6.0);
  }
  if (threadIdx.x < 3) {
    const int f = threadIdx.x;
    J.M[f] = S.jM[f];
    J.rc[f] = Cst<T>::rc(S, f);
    J.rc2[f] = S.jM[f] ? Cst<T>::rc(S, f) * Cst<T>::rc(S, f) : T(0);   // a term switched off: no pair inside
    J.scale[f] = S.jM[f] ? T(S.jM[f]) / Cst<T>::rc(S, f) : T(0);
    const double sd = S.jM[f] ? (double)S.jM[f] / S.jrc[f] : 0.0;
    J.scale_lo[f] = T(sd - (double)J.scale[f]);
  }
}

// 6 u(r) as a pair (hi, lo) whose sum carries no rounding common to all pairs: the knot
// interval coordinate uses the split scale (hi + lo), the basis is used without its
// factor 1/6 (integer coefficients), and the knots' residues enter lo. J summed from these
// and divided by 6 once is free of the systematic shifts a rounded M / r_c or 1/6 gives.
template <class T>
__device__ __forceinline__ void jastrow_value6(const JastrowTab<T>& J, int f, T r, T& hi, T& lo) {
  hi = lo = T(0);
  if (!(r < J.rc[f])) return;
  const T s = fma(r, J.scale[f], r * J.scale_lo[f]);
  int i = (int)tfloor(s);
  if (i < 0) i = 0;
  const T t = s - T(i);
  const T t2 = t * t, t3 = t2 * t, omt = T(1) - t;
  const T b[4] = {omt * omt * omt, T(3) * t3 - T(6) * t2 + T(4),
                  T(-3) * t3 + T(3) * t2 + T(3) * t + T(1), t3};
  const T* p = J.p[f] + i;
  const T* pl = J.plo[f] + i;
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    hi += p[q] * b[q];
    lo += pl[q] * b[q];
  }
}

template <class T>
__device__ __forceinline__ void jastrow_eval(const JastrowTab<T>& J, int f, T r, T& u, T& du,
                                             T& d2u) {
  u = du = d2u = T(0);
  if (!(r < J.rc[f])) return;
  const T scale = J.scale[f];
  const T s = r * scale;
  int i = (int)tfloor(s);
  if (i < 0) i = 0;
  const T t = s - T(i);
  T b[4], db[4], d2b[4];
  bspline_w<T>(t, b, db, d2b);
  const T* p = J.p[f] + i;
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    u += p[q] * b[q];
    du += p[q] * db[q];
    d2u += p[q] * d2b[q];
  }
  du *= scale;
  d2u *= scale * scale;
}

// r from r^2 in the value-only pair loop: in single precision x * rsqrt(x) (a few ulp, the
// hardware reciprocal root), in double precision the correctly rounded root.
__device__ __forceinline__ float sqrt_pair(float x) { return x > 0.f ? x * rsqrtf(x) : 0.f; }
__device__ __forceinline__ double sqrt_pair(double x) { return sqrt(x); }
__device__ __forceinline__ void load_pw(const float* c, float (&a)[4]) {
  const float4 v = *reinterpret_cast<const float4*>(c);
  a[0] = v.x; a[1] = v.y; a[2] = v.z; a[3] = v.w;
}
__device__ __forceinline__ void load_pw(const double* c, double (&a)[4]) {
  const double2 v0 = reinterpret_cast<const double2*>(c)[0], v1 = reinterpret_cast<const double2*>(c)[1];
  a[0] = v0.x; a[1] = v0.y; a[2] = v1.x; a[3] = v1.y;
}

// u(r) alone, from the squared distance (a Metropolis ratio needs no derivatives): 0 at
// and beyond the cutoff. Without a branch, so that the pair loop's iterations overlap;
// beyond the cutoff the spline is evaluated at r = 0 and discarded.
template <class T>
__device__ __forceinline__ T jastrow_value_r2(const JastrowTab<T>& J, int f, T r2) {
  const bool in = r2 < J.rc2[f];
  const T s = sqrt_pair(in ? r2 : T(0)) * J.scale[f];
  const T fl = tfloor(s);
  const int i = min(max((int)fl, 0), kMaxKnots);
  const T t = s - fl;
  T a[4];
  load_pw(&J.pw[f][i][0], a);
  const T u = ((a[3] * t + a[2]) * t + a[1]) * t + a[0];
  return in ? u : T(0);
}

// 1/sqrt(x) and e^x in the pair loops of the local energy: the hardware approximations
// (a few ulp) in single precision, the correctly rounded functions in double.
__device__ __forceinline__ float rsqrt_w(float x) { return rsqrtf(x); }
__device__ __forceinline__ double rsqrt_w(double x) { return 1.0 / sqrt(x); }
__device__ __forceinline__ float exp_w(float x) { return __expf(x); }
__device__ __forceinline__ double exp_w(double x) { return exp(x); }
__device__ __forceinline__ float erfc_w(float x) { return erfcf(x); }
__device__ __forceinline__ double erfc_w(double x) { return erfc(x); }

// Yukawa pair potential exp(-kappa r)/r for r < L/2 (stand-in for v_ee, v_eI).
template <class T>
__device__ __forceinline__ T yukawa(T r, T kappa, T L) {
  return (r < T(0.5) * L) ? exp(-kappa * r) / r : T(0);
}

// Barrier over `count` threads (a multiple of 32) of the block, id 1..15 (0 is the block).
__device__ __forceinline__ void named_barrier(int id, int count) {
  asm volatile("bar.sync %0, %1;\n" ::"r"(id), "r"(count) : "memory");
}

// ------------------------------------------------------------------ reductions
template <int N, class T>
__device__ __forceinline__ void warp_sum(T (&v)[N]) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1)
#pragma unroll
    for (int k = 0; k < N; ++k) v[k] += __shfl_xor_sync(0xffffffffu, v[k], o);
}

// Sum N values over the block: warp sums in T, then thread 0 adds the warp partials in
// double and stores the totals in out[0..N) (shared memory). Ends with a barrier, so
// every thread may read out[] afterwards. red: shared [32 * N] of T.
template <int N, class T>
__device__ __forceinline__ void block_sum(T (&v)[N], T* red, double* out) {
  warp_sum<N, T>(v);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  if (lane == 0)
#pragma unroll
    for (int k = 0; k < N; ++k) red[warp * N + k] = v[k];
  __syncthreads();
  if (threadIdx.x == 0) {
#pragma unroll
    for (int k = 0; k < N; ++k) {
      double s = 0.0;
      for (int w = 0; w < nw; ++w) s += (double)red[w * N + k];
      out[k] = s;
    }
  }
  __syncthreads();
}

// ------------------------------------------------------------------ compensated sums
// A pair (s, c) carries a sum whose value is s + c to about twice the working precision
// (TwoProduct by FMA and TwoSum: the error-free transformations of Ogita, Rump and Oishi,
// "Accurate sum and dot product", SIAM J. Sci. Comput. 26, 2005). Used for the dot
// products that decide a move, where cancellation can amplify single-precision rounding
// by the ratio sum|phi_j x_j| / |R|. In double precision the pair degenerates to a sum.
__device__ __forceinline__ void comp_fma(float& s, float& c, float a, float b) {
  const float p = __fmul_rn(a, b);
  const float e = __fmaf_rn(a, b, -p);
  const float t = __fadd_rn(s, p);
  const float z = __fsub_rn(t, s);
  const float q = __fadd_rn(__fsub_rn(s, __fsub_rn(t, z)), __fsub_rn(p, z));
  s = t;
  c = __fadd_rn(c, __fadd_rn(q, e));
}
__device__ __forceinline__ void comp_fma(double& s, double& c, double a, double b) { s += a * b; }
__device__ __forceinline__ void comp_merge(float& s, float& c, float s2, float c2) {
  const float t = __fadd_rn(s, s2);
  const float z = __fsub_rn(t, s);
  const float q = __fadd_rn(__fsub_rn(s, __fsub_rn(t, z)), __fsub_rn(s2, z));
  s = t;
  c = __fadd_rn(__fadd_rn(c, c2), q);
}
__device__ __forceinline__ void comp_merge(double& s, double& c, double s2, double c2) {
  s += s2;
  c += c2;
}
template <class T>
__device__ __forceinline__ void warp_sum_comp(T& s, T& c) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const T s2 = __shfl_xor_sync(0xffffffffu, s, o);
    const T c2 = __shfl_xor_sync(0xffffffffu, c, o);
    comp_merge(s, c, s2, c2);
  }
}

// ------------------------------------------------------------------ table loads
template <class TT> struct TabVec;
template <> struct TabVec<double> {
  static constexpr int V = 2;
  __device__ static __forceinline__ void load(const double* p, float (&)[2], double (&o)[2]) {
    const double2 q = __ldg(reinterpret_cast<const double2*>(p));
    o[0] = q.x; o[1] = q.y;
  }
};
template <> struct TabVec<float> {
  static constexpr int V = 4;
  __device__ static __forceinline__ void load(const float* p, float (&o)[4], double (&)[4]) {
    const float4 q = __ldg(reinterpret_cast<const float4*>(p));
    o[0] = q.x; o[1] = q.y; o[2] = q.z; o[3] = q.w;
  }
};
template <> struct TabVec<__nv_bfloat16> {
  static constexpr int V = 8;
  __device__ static __forceinline__ void load(const __nv_bfloat16* p, float (&o)[8], double (&)[8]) {
    const uint4 q = __ldg(reinterpret_cast<const uint4*>(p));
    const uint32_t w[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      o[2 * k] = __uint_as_float(w[k] << 16);
      o[2 * k + 1] = __uint_as_float(w[k] & 0xFFFF0000u);
    }
  }
};

// One table element (the V = 1 form of TabVec::load): into f, or into d for a double table.
__device__ __forceinline__ void tab_load1(const double* p, float&, double& d) { d = __ldg(p); }
__device__ __forceinline__ void tab_load1(const float* p, float& f, double&) { f = __ldg(p); }
__device__ __forceinline__ void tab_load1(const __nv_bfloat16* p, float& f, double&) {
  f = __uint_as_float((uint32_t)__ldg(reinterpret_cast<const unsigned short*>(p)) << 16);
}

// Working-precision accumulator type of a table type.
template <class TT> struct AccOf { using type = float; };
template <> struct AccOf<double> { using type = double; };

}  // namespace qmcgb
