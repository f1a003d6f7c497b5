// Three-body electron-electron-ion Jastrow factor (Sec. "Jastrow factor": the polynomial of
// Drummond et al. in the two electron-ion distances a = r_iI, b = r_jI and the pair distance
// c = r_ij, cut off at h = r_c / 2 in both electron-ion distances):
//   u(a, b, c) = sum_{l,m <= M_eI} sum_{n <= M_ee} gamma_lmn a^l b^m c^n (a - h)^3 (b - h)^3,
//   a < h and b < h (zero otherwise), J3 = sum_I sum_{i<j} u_{s(i) s(j)}(r_iI, r_jI, r_ij),
// one coefficient set for same-spin and one for opposite-spin pairs, gamma_lmn = gamma_mln.
// For electron i: grad_i u = u_a a^ + u_c c^ and
// lap_i u = u_aa + 2 u_a / a + u_cc + 2 u_c / c + 2 u_ac (a^ . c^), a^ = (r_i - R_I) / a,
// c^ = (r_i - r_j) / c.
#pragma once
#include "qmc_device.cuh"
#include "qmc_internal.h"

namespace qmcgb {

// The coefficient sets staged in shared memory (indices read through per-thread values would
// serialise the constant bank), the orders and the cutoff.
template <class T>
struct J3Tab {
  int on, meI, mee;
  T h, h2;
  T g[2][kJ3MaxCoef];   // [set][(l (M_eI + 1) + m) (M_ee + 1) + n]
};

template <class T>
__device__ __forceinline__ void j3_tab_fill(const SysParams& S, J3Tab<T>& J) {
  if (threadIdx.x == 0) {
    J.on = S.j3_on;
    J.meI = S.j3_meI;
    J.mee = S.j3_mee;
    J.h = (T)S.j3_h;
    J.h2 = (T)(S.j3_h * S.j3_h);
  }
  if (!S.j3_on) return;
  const int nc = (S.j3_meI + 1) * (S.j3_meI + 1) * (S.j3_mee + 1);
  for (int i = threadIdx.x; i < 2 * nc; i += blockDim.x)
    J.g[i / nc][i % nc] = (T)S.j3_g[(i / nc) * nc + i % nc];
}

// u(a, b, c) of set f; the caller has checked a < h and b < h. Horner in c, then b, then a.
template <class T>
__device__ __forceinline__ T j3_value(const J3Tab<T>& J, int f, T a, T b, T c) {
  const int me = J.meI, mc = J.mee;
  const T* g = J.g[f];
  T P = T(0);
  for (int l = me; l >= 0; --l) {
    T sl = T(0);
    for (int m = me; m >= 0; --m) {
      const T* gq = g + (l * (me + 1) + m) * (mc + 1);
      T q = T(0);
      for (int n = mc; n >= 0; --n) q = fma(q, c, gq[n]);
      sl = fma(sl, b, q);
    }
    P = fma(P, a, sl);
  }
  const T fa = a - J.h, fb = b - J.h;
  return P * (fa * fa * fa) * (fb * fb * fb);
}

// u and the partial derivatives d = (u, u_a, u_c, u_aa, u_cc, u_ac) of set f at (a, b, c),
// a < h and b < h. Horner with derivatives: a polynomial's value p, p' and p''/2 advance
// together (d2 <- d2 x + d1, d1 <- d1 x + p, p <- p x + coefficient).
template <class T>
__device__ __forceinline__ void j3_derivs(const J3Tab<T>& J, int f, T a, T b, T c, T (&d)[6]) {
  const int me = J.meI, mc = J.mee;
  const T* g = J.g[f];
  // P = sum_l a^l S_l, S_l = sum_m b^m q_lm(c); also S'_l and S''_l (c derivatives)
  T p0 = 0, p1 = 0, p2 = 0;       // P, P_a, P_aa / 2 (over S_l)
  T c0 = 0, c1 = 0;               // P_c, P_ac (over S'_l)
  T e0 = 0;                       // P_cc (over S''_l)
  for (int l = me; l >= 0; --l) {
    T s0 = 0, s1 = 0, s2 = 0;     // S_l, S'_l, S''_l
    for (int m = me; m >= 0; --m) {
      const T* gq = g + (l * (me + 1) + m) * (mc + 1);
      T q0 = 0, q1 = 0, q2 = 0;   // q, q', q''/2
      for (int n = mc; n >= 0; --n) {
        q2 = fma(q2, c, q1);
        q1 = fma(q1, c, q0);
        q0 = fma(q0, c, gq[n]);
      }
      s0 = fma(s0, b, q0);
      s1 = fma(s1, b, q1);
      s2 = fma(s2, b, T(2) * q2);
    }
    p2 = fma(p2, a, p1);
    p1 = fma(p1, a, p0);
    p0 = fma(p0, a, s0);
    c1 = fma(c1, a, c0);
    c0 = fma(c0, a, s1);
    e0 = fma(e0, a, s2);
  }
  const T P = p0, Pa = p1, Paa = T(2) * p2, Pc = c0, Pac = c1, Pcc = e0;
  const T fa = a - J.h, fb = b - J.h;
  const T F = fa * fa * fa, dF = T(3) * fa * fa, d2F = T(6) * fa, G = fb * fb * fb;
  d[0] = P * F * G;
  d[1] = (Pa * F + P * dF) * G;
  d[2] = Pc * F * G;
  d[3] = (Paa * F + T(2) * Pa * dF + P * d2F) * G;
  d[4] = Pcc * F * G;
  d[5] = (Pac * F + Pc * dF) * G;
}

// |x - q|^2 (minimum image) with the displacement in dv; q[k * stride] is coordinate k of
// a point stored in working precision or in double.
template <class T, class Q>
__device__ __forceinline__ T j3_dist2(const T (&x)[3], const Q* q, int stride, T L, T iL, T (&dv)[3]) {
#pragma unroll
  for (int k = 0; k < 3; ++k) dv[k] = min_image<T>(x[k] - (T)q[k * stride], L, iL);
  return dv[0] * dv[0] + dv[1] * dv[1] + dv[2] * dv[2];
}

// Group description of the J3 sums: the ions near a point are found by a ballot over a
// sub-warp of `ssize` lanes (lane slane, lanes sshift.. of the warp, mask smask; every lane
// of smask calls together), and the electrons j are split as j = jtid, jtid + jnt, ...
struct J3Group {
  int slane, ssize, sshift;
  unsigned smask;
  int jtid, jnt;
};

__device__ __forceinline__ J3Group j3_group_warps(int jtid, int jnt) {
  return J3Group{(int)(threadIdx.x & 31), 32, 0, 0xffffffffu, jtid, jnt};
}
__device__ __forceinline__ J3Group j3_group_sub(int ssize, int jtid, int jnt) {
  const int lane = threadIdx.x & 31, sh = lane & ~(ssize - 1);
  const unsigned m = ssize == 32 ? 0xffffffffu : (((1u << ssize) - 1u) << sh);
  return J3Group{lane - sh, ssize, sh, m, jtid, jnt};
}

// Bits of the ions I0 + (0..ssize) of this 32-aligned chunk that lie within h of x or y.
template <class T>
__device__ __forceinline__ unsigned j3_near_bits(const SysParams& S, const J3Tab<T>& J,
                                                 const T* ionw, const J3Group& G, int I0,
                                                 const T (&x)[3], const T (&y)[3], T L, T iL) {
  const int I = I0 + G.slane;
  bool near = false;
  if (I < S.n_ion) {
    T dv[3];
    near = j3_dist2<T>(x, ionw + I, S.n_ion, L, iL, dv) < J.h2 ||
           j3_dist2<T>(y, ionw + I, S.n_ion, L, iL, dv) < J.h2;
  }
  const unsigned b = __ballot_sync(G.smask, near) >> G.sshift;
  return G.ssize == 32 ? b : (b & ((1u << G.ssize) - 1u));
}

// J3(r') - J3(r) of a move of electron e from ro to rn (this thread's share) and, with
// kGrad, this thread's share of grad_e J3 at rn in g. pos: [3][n_e] electron positions
// (working precision or double). With near != nullptr the ions within h of ro or rn are also
// listed there (up to cap, by the group's lane 0), and n_near receives their count (every
// lane; it may exceed cap).
template <class T, bool kGrad, class PT>
__device__ __forceinline__ T j3_delta(const SysParams& S, const J3Tab<T>& J, const PT* pos,
                                      const T* ionw, int e, const T (&ro)[3], const T (&rn)[3],
                                      T L, T iL, const J3Group& G, T (&g)[3],
                                      int* near = nullptr, int cap = 0, int* n_near = nullptr) {
  const int n_e = S.n_e;
  const bool e_up = e < S.n_up;
  T dj = T(0);
  g[0] = g[1] = g[2] = T(0);
  int cnt = 0;
  for (int I0 = 0; I0 < S.n_ion; I0 += G.ssize) {
    unsigned bits = j3_near_bits<T>(S, J, ionw, G, I0, rn, ro, L, iL);
    while (bits) {
      const int I = I0 + __ffs(bits) - 1;
      bits &= bits - 1;
      if (near && G.slane == 0 && cnt < cap) near[cnt] = I;
      ++cnt;
      T dn[3], dq[3];
      const T an2 = j3_dist2<T>(rn, ionw + I, S.n_ion, L, iL, dn);
      const T ao2 = j3_dist2<T>(ro, ionw + I, S.n_ion, L, iL, dq);
      const bool in_n = an2 < J.h2, in_o = ao2 < J.h2;
      const T an = sqrt(an2), ao = sqrt(ao2);
      for (int j = G.jtid; j < n_e; j += G.jnt) {
        if (j == e) continue;
        const T rj[3] = {(T)pos[j], (T)pos[n_e + j], (T)pos[2 * n_e + j]};
        T db[3];
        const T b2 = j3_dist2<T>(rj, ionw + I, S.n_ion, L, iL, db);
        if (!(b2 < J.h2)) continue;
        const T b = sqrt(b2);
        const int f = ((j < S.n_up) == e_up) ? 0 : 1;
        T dc[3];
        if (in_n) {
          const T cn = sqrt(j3_dist2<T>(rn, rj, 1, L, iL, dc));
          if constexpr (kGrad) {
            T d[6];
            j3_derivs<T>(J, f, an, b, cn, d);
            dj += d[0];
            const T ga = an > T(0) ? d[1] / an : T(0), gc = cn > T(0) ? d[2] / cn : T(0);
#pragma unroll
            for (int k = 0; k < 3; ++k) g[k] += ga * dn[k] + gc * dc[k];
          } else {
            dj += j3_value<T>(J, f, an, b, cn);
          }
        }
        if (in_o) {
          const T co = sqrt(j3_dist2<T>(ro, rj, 1, L, iL, dc));
          dj -= j3_value<T>(J, f, ao, b, co);
        }
      }
    }
  }
  if (n_near) *n_near = cnt;
  return dj;
}

// Correction of the difference of move b when move a (same spin block) has been accepted
// before it within a window: sum_I [U(r'_a, r'_b) - U(r'_a, r_b) - U(r_a, r'_b) + U(r_a, r_b)],
// U(x, y) = u(|x - R_I|, |y - R_I|, |x - y|) of the same-spin set, over the ions listed near
// move a (nl ions in near[]).
template <class T>
__device__ __forceinline__ T j3_pair_correction(const SysParams& S, const J3Tab<T>& J,
                                                const T* ionw, const int* near, int nl,
                                                const T (&pa)[3], const T (&oa)[3],
                                                const T (&pb)[3], const T (&ob)[3], T L, T iL) {
  T q = T(0);
  T dv[3];
  const T c00 = sqrt(j3_dist2<T>(pa, pb, 1, L, iL, dv));
  const T c01 = sqrt(j3_dist2<T>(pa, ob, 1, L, iL, dv));
  const T c10 = sqrt(j3_dist2<T>(oa, pb, 1, L, iL, dv));
  const T c11 = sqrt(j3_dist2<T>(oa, ob, 1, L, iL, dv));
  for (int k = 0; k < nl; ++k) {
    const int I = near[k];
    const T a0 = j3_dist2<T>(pa, ionw + I, S.n_ion, L, iL, dv);
    const T a1 = j3_dist2<T>(oa, ionw + I, S.n_ion, L, iL, dv);
    const T b0 = j3_dist2<T>(pb, ionw + I, S.n_ion, L, iL, dv);
    const T b1 = j3_dist2<T>(ob, ionw + I, S.n_ion, L, iL, dv);
    const bool ia0 = a0 < J.h2, ia1 = a1 < J.h2, ib0 = b0 < J.h2, ib1 = b1 < J.h2;
    if (!((ia0 || ia1) && (ib0 || ib1))) continue;
    const T ra0 = sqrt(a0), ra1 = sqrt(a1), rb0 = sqrt(b0), rb1 = sqrt(b1);
    if (ia0 && ib0) q += j3_value<T>(J, 0, ra0, rb0, c00);
    if (ia0 && ib1) q -= j3_value<T>(J, 0, ra0, rb1, c01);
    if (ia1 && ib0) q -= j3_value<T>(J, 0, ra1, rb0, c10);
    if (ia1 && ib1) q += j3_value<T>(J, 0, ra1, rb1, c11);
  }
  return q;
}

constexpr int kJ3Threads = 256;

// Per electron i of every walker: grad_i J3 (3), lap_i J3 and the electron's share of J3,
// sum_I sum_{j > i} u, written to Wk.j3vgl [w][i][5] for the local-energy kernel. One block
// per walker, one warp per electron: the ions within h of r_i by a ballot, then the other
// electrons within h of each such ion, split over the lanes.
template <class TW>
__global__ void __launch_bounds__(kJ3Threads) k_j3_vgl(SysParams S, WalkParams Wk) {
  extern __shared__ __align__(16) char smem_j3[];
  __shared__ J3Tab<TW> j3t;
  j3_tab_fill<TW>(S, j3t);
  const int w = blockIdx.x;
  if (Wk.n_live && w >= *Wk.n_live) return;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int n_e = S.n_e;
  TW* posw = reinterpret_cast<TW*>(smem_j3);              // [3][n_e]
  const double* P = Wk.pos + (size_t)w * 3 * n_e;
  for (int i = threadIdx.x; i < 3 * n_e; i += blockDim.x) posw[i] = (TW)P[i];
  __syncthreads();
  const TW Lw = Cst<TW>::L(S), iLw = Cst<TW>::invL(S);
  const TW* ionw = Cst<TW>::ions(S);
  TW* out = static_cast<TW*>(Wk.j3vgl) + (size_t)w * n_e * 5;
  const J3Group G = j3_group_warps(lane, 32);
  for (int i = warp; i < n_e; i += nw) {
    const TW ri[3] = {posw[i], posw[n_e + i], posw[2 * n_e + i]};
    TW v[5] = {0, 0, 0, 0, 0};
    for (int I0 = 0; I0 < S.n_ion; I0 += 32) {
      unsigned bits = j3_near_bits<TW>(S, j3t, ionw, G, I0, ri, ri, Lw, iLw);
      while (bits) {
        const int I = I0 + __ffs(bits) - 1;
        bits &= bits - 1;
        TW da[3];
        const TW a = sqrt(j3_dist2<TW>(ri, ionw + I, S.n_ion, Lw, iLw, da));
        for (int j = lane; j < n_e; j += 32) {
          if (j == i) continue;
          const TW rj[3] = {posw[j], posw[n_e + j], posw[2 * n_e + j]};
          TW db[3], dc[3];
          const TW b2 = j3_dist2<TW>(rj, ionw + I, S.n_ion, Lw, iLw, db);
          if (!(b2 < j3t.h2)) continue;
          const TW c = sqrt(j3_dist2<TW>(ri, rj, 1, Lw, iLw, dc));
          const int f = ((j >= S.n_up) == (i >= S.n_up)) ? 0 : 1;
          TW d[6];
          j3_derivs<TW>(j3t, f, a, sqrt(b2), c, d);
          if (j > i) v[4] += d[0];
          if (!(a > TW(0)) || !(c > TW(0))) continue;
          const TW ia = TW(1) / a, ic = TW(1) / c;
          TW dot = 0;
#pragma unroll
          for (int k = 0; k < 3; ++k) {
            v[k] += d[1] * ia * da[k] + d[2] * ic * dc[k];
            dot += da[k] * dc[k];
          }
          v[3] += d[3] + TW(2) * d[1] * ia + d[4] + TW(2) * d[2] * ic + TW(2) * d[5] * dot * ia * ic;
        }
      }
    }
    warp_sum<5, TW>(v);
    if (lane == 0)
#pragma unroll
      for (int k = 0; k < 5; ++k) out[(size_t)i * 5 + k] = v[k];
  }
}

inline size_t j3_smem_bytes(int n_e, size_t tw) { return 3 * (size_t)n_e * tw; }

}  // namespace qmcgb
