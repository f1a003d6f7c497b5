// Non-local pseudopotential energy by 12-point angular quadrature (Sec. "Hamiltonian":
// semi-local channels sum_lm |Y_lm> dv_l(r) <Y_lm| within a cutoff, evaluated following
// Mitas, Shirley and Ceperley with a 12-point angular integration). For electron i at
// distance r < r_c from ion I (nearest image) the addition theorem gives
//   V_NL(i, I) = sum_l (2l+1) dv_l(r) (1/12) sum_q P_l(u . O n_q) Psi(r_i -> R_I + r O n_q) / Psi,
// n_q the icosahedron's vertices (exact to degree 5), O a random rotation per walker and
// measurement. Each quadrature point is a virtual move of electron i alone: its ratio is
// the determinant ratio phi(r') . Binv[i] (value-only tricubic gather of the spin block's
// orbitals dotted with the inverse row) times exp(dJ), with no update of anything.
//
// Three kernels: k_nlpp_pairs lists the (walker, electron, ion) pairs inside the cutoff;
// k_nlpp_eval gives one warp to each pair, which evaluates its 12 points; k_nlpp_sum adds
// each walker's pair energies in list order to E_L and to the walker's V_NL.
#pragma once
#include "qmc_kernels.cuh"

namespace qmcgb {

// Value of orbitals [o0, o0 + V) of lane `lane` at r, dotted with the inverse row brow
// (compensated); returns the lane's partial sum of phi_j(r) Binv[e][j].
template <class TT, class TW>
__device__ __forceinline__ void val_dot_lane(const SysParams& S, const int (&idx)[3][4],
                                             const typename AccOf<TT>::type (&w)[3][4], int o0,
                                             int n_eval, const TW* __restrict__ brow, TW& s,
                                             TW& c) {
  using A = typename AccOf<TT>::type;
  constexpr int V = TabVec<TT>::V;
  if (o0 >= n_eval) return;
  A acc[V];
#pragma unroll
  for (int v = 0; v < V; ++v) acc[v] = A(0);
  const TT* __restrict__ tab = static_cast<const TT*>(S.table);
  // 16 rows in flight per step of the outer loop (fully unrolled, a single accumulator per
  // orbital would put all 64 row loads in flight and exceed the register file)
#pragma unroll 1
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      const A wxy = w[0][a] * w[1][b];
      const size_t base = ((size_t)idx[0][a] * S.ny + idx[1][b]) * S.nz;
#pragma unroll
      for (int cc = 0; cc < 4; ++cc) {
        float cf[V];
        double cd[V];
        TabVec<TT>::load(tab + (base + idx[2][cc]) * S.ld + o0, cf, cd);
        const A wv = wxy * w[2][cc];
#pragma unroll
        for (int v = 0; v < V; ++v) {
          A cv;
          if constexpr (sizeof(A) == 8) cv = cd[v]; else cv = cf[v];
          acc[v] += wv * cv;
        }
      }
    }
#pragma unroll
  for (int v = 0; v < V; ++v)
    if (o0 + v < n_eval) comp_fma(s, c, (TW)acc[v], brow[o0 + v]);
}

// Pairs (electron, ion) of each walker within the cutoff: pairs[w][k] = e * n_ion + I in
// electron-major, ion-minor order, count[w] = k. One block per walker: each thread counts
// the pairs of one electron per pass, a block scan gives the offsets, then the thread writes
// them, so the list (and every sum over it) is the same from run to run.
static __global__ void __launch_bounds__(256) k_nlpp_pairs(SysParams S, WalkParams Wk,
                                                           int* __restrict__ pairs,
                                                           int* __restrict__ count, int cap) {
  __shared__ int part[256 / 32];
  const int w = blockIdx.x, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  if (Wk.n_live && w >= *Wk.n_live) return;
  const double* P = Wk.pos + (size_t)w * 3 * S.n_e;
  const double rc2 = S.nl_rcut * S.nl_rcut;
  // The test in single precision decides every pair whose r^2 is farther than a margin from
  // rc^2 (the single-precision distance is off by far less: a few ulp of L per component);
  // the few within it are decided in FP64, so the list is the FP64 one.
  const float rc2f = (float)rc2, marg = 1e-4f * rc2f + 64.f * 1.2e-7f * S.Lf * S.Lf;
  auto inside = [&](const double (&x)[3], const float (&xf)[3], int I) {
    float r2f = 0.f;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const float d = min_image<float>(xf[c] - S.ionsf[c * S.n_ion + I], S.Lf, S.invLf);
      r2f += d * d;
    }
    if (r2f > rc2f + marg) return false;
    if (r2f < rc2f - marg && r2f > marg) return true;
    double r2 = 0.0;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const double d = min_image<double>(x[c] - S.ions[c * S.n_ion + I], S.L);
      r2 += d * d;
    }
    return r2 < rc2 && r2 > 0.0;
  };
  int base = 0;
  for (int e0 = 0; e0 < S.n_e; e0 += blockDim.x) {
    const int e = e0 + tid;
    double x[3] = {0.0, 0.0, 0.0};
    float xf[3] = {0.f, 0.f, 0.f};
    int c = 0;
    if (e < S.n_e) {
      x[0] = P[e]; x[1] = P[S.n_e + e]; x[2] = P[2 * S.n_e + e];
      xf[0] = (float)x[0]; xf[1] = (float)x[1]; xf[2] = (float)x[2];
      for (int I = 0; I < S.n_ion; ++I) c += inside(x, xf, I);
    }
    // exclusive block scan of the counts
    int incl = c;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int v = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += v;
    }
    if (lane == 31) part[warp] = incl;
    __syncthreads();
    int before = 0, total = 0;
    for (int q = 0; q < (int)(blockDim.x >> 5); ++q) {
      before += q < warp ? part[q] : 0;
      total += part[q];
    }
    __syncthreads();
    if (c > 0) {
      int k = base + before + incl - c;
      for (int I = 0; I < S.n_ion; ++I)
        if (inside(x, xf, I)) {
          if (k < cap) pairs[(size_t)w * cap + k] = e * S.n_ion + I;
          ++k;
        }
    }
    base += total;
  }
  if (tid == 0) {
    count[w] = base;
    if (base > cap) atomicOr(Wk.err, kErrOverflow);
  }
}

// The 12 vertices of an icosahedron (0, +-1, +-phi), (+-1, +-phi, 0), (+-phi, 0, +-1),
// normalised, in the order of the oracle's table.
__device__ __forceinline__ void ico_vertex(int q, double v[3]) {
  const double ph = 1.6180339887498949, nrm = 1.0 / sqrt(1.0 + ph * ph);
  const double a = (q / 6) ? -1.0 : 1.0, b = ((q / 3) & 1) ? -ph : ph;
  const int k = q % 3;
  if (k == 0) { v[0] = 0.0; v[1] = a; v[2] = b; }
  else if (k == 1) { v[0] = a; v[1] = b; v[2] = 0.0; }
  else { v[0] = b; v[1] = 0.0; v[2] = a; }
  v[0] *= nrm; v[1] *= nrm; v[2] *= nrm;
}

// Uniform random rotation of walker `wid` at measurement t from Philox block
// (t, 0xD, wid, 3): Shoemake's unit quaternion from words 0..2.
__device__ __forceinline__ void nlpp_rotation(const SysParams& S, uint32_t t, uint32_t wid,
                                              double O[3][3]) {
  const U32x4 r = philox4x32_10(t, 0xDu, wid, 3u, S.seed_lo, S.seed_hi);
  const double u1 = unit_open(r.v[0]), u2 = unit_open(r.v[1]), u3 = unit_open(r.v[2]);
  const double a = sqrt(1.0 - u1), b = sqrt(u1);
  double s2, c2, s3, c3;
  sincos(2.0 * M_PI * u2, &s2, &c2);
  sincos(2.0 * M_PI * u3, &s3, &c3);
  const double x = a * s2, y = a * c2, z = b * s3, ww = b * c3;
  O[0][0] = 1 - 2 * (y * y + z * z); O[0][1] = 2 * (x * y - z * ww); O[0][2] = 2 * (x * z + y * ww);
  O[1][0] = 2 * (x * y + z * ww); O[1][1] = 1 - 2 * (x * x + z * z); O[1][2] = 2 * (y * z - x * ww);
  O[2][0] = 2 * (x * z - y * ww); O[2][1] = 2 * (y * z + x * ww); O[2][2] = 1 - 2 * (x * x + y * y);
}

// One warp per listed pair: the 12 virtual moves of electron e about ion I; the pair's
// V_NL (FP64) goes to vals[w][k].
template <class TT, class TW>
__global__ void __launch_bounds__(256, 2) k_nlpp_eval(SysParams S, WalkParams Wk, const int* __restrict__ pairs,
                                                   const int* __restrict__ count, int cap,
                                                   uint32_t t, double* __restrict__ vals) {
  using A = typename AccOf<TT>::type;
  constexpr int V = TabVec<TT>::V;
  __shared__ JastrowTab<TW> jt;
  __shared__ J3Tab<TW> j3t;
  jastrow_tab_fill<TW>(S, jt);
  j3_tab_fill<TW>(S, j3t);
  __syncthreads();
  const long long gw = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (gw >= (long long)Wk.n_w * cap) return;
  const int w = (int)(gw / cap), k = (int)(gw % cap);
  if (Wk.n_live && w >= *Wk.n_live) return;
  if (k >= min(count[w], cap)) return;
  const int pr = pairs[(size_t)w * cap + k];
  const int e = pr / S.n_ion, I = pr % S.n_ion;
  const int n_e = S.n_e;
  const double* P = Wk.pos + (size_t)w * 3 * n_e;
  const double x[3] = {P[e], P[n_e + e], P[2 * n_e + e]};
  double d[3], r2 = 0.0;
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    d[c] = min_image<double>(x[c] - S.ions[c * S.n_ion + I], S.L);
    r2 += d[c] * d[c];
  }
  // lane q < 12 prepares quadrature point q: its position r' and its channel weight
  // sum_l (2l+1) dv_l(r) P_l(u . O n_q) / 12
  double pq[3] = {0.0, 0.0, 0.0}, wq = 0.0;
  if (lane < 12) {
    const double r = sqrt(r2);
    double O[3][3], v[3], p[3];
    nlpp_rotation(S, sweep_index(Wk, t), Wk.wid[w], O);
    ico_vertex(lane, v);
    double ct = 0.0;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      p[a] = O[a][0] * v[0] + O[a][1] * v[1] + O[a][2] * v[2];
      ct += d[a] / r * p[a];
      pq[a] = wrap_box((x[a] - d[a]) + r * p[a], S.L);     // nearest image of ion I + r O n_q
    }
    double pl0 = 1.0, pl1 = ct;                             // P_0, P_1; then the recurrence
#pragma unroll
    for (int l = 0; l < kMaxNlChannels; ++l) {
      if (l < S.nl_nch) {
        const double dvl = S.nl_amp[l] * exp(-(r / S.nl_width[l]) * (r / S.nl_width[l]));
        wq += (2 * l + 1) * dvl * (l == 0 ? 1.0 : pl1);
      }
      if (l >= 1) {
        const double pn = ((2 * l + 1) * ct * pl1 - l * pl0) / (l + 1);
        pl0 = pl1;
        pl1 = pn;
      }
    }
    wq /= 12.0;
  }
  const int spin = e >= S.n_up;
  const int ns = spin ? S.n_dn : S.n_up, row = e - (spin ? S.n_up : 0);
  const TW* brow = binv_block<const TW>(S, Wk, w, spin) + (size_t)row * ns;
  const TW Lw = Cst<TW>::L(S), iLw = Cst<TW>::invL(S);
  const TW* ionw = Cst<TW>::ions(S);
  const int nn[3] = {S.nx, S.ny, S.nz};
  double total = 0.0;
#pragma unroll 1
  for (int q = 0; q < 12; ++q) {
    const double rn[3] = {__shfl_sync(0xffffffffu, pq[0], q), __shfl_sync(0xffffffffu, pq[1], q),
                          __shfl_sync(0xffffffffu, pq[2], q)};
    // determinant ratio: phi(r') . Binv[e] over the spin block's orbitals
    A wts[3][4];
    int idx[3][4];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      const double sg = rn[a] * S.inv_delta[a];
      const double fi = floor(sg);
      A db[4], d2b[4];
      bspline_w<A>((A)(sg - fi), wts[a], db, d2b);
#pragma unroll
      for (int qq = 0; qq < 4; ++qq) idx[a][qq] = ((((int)fi - 1 + qq) % nn[a]) + nn[a]) % nn[a];
    }
    TW s = TW(0), sc = TW(0);
#pragma unroll 1
    for (int o0 = lane * V; o0 < ns; o0 += 32 * V) val_dot_lane<TT, TW>(S, idx, wts, o0, ns, brow, s, sc);
    warp_sum_comp(s, sc);
    // Jastrow difference of moving e from x to r'
    const TW xo[3] = {(TW)x[0], (TW)x[1], (TW)x[2]}, xn[3] = {(TW)rn[0], (TW)rn[1], (TW)rn[2]};
    TW dj = TW(0);
#pragma unroll 2
    for (int j = lane; j < n_e + S.n_ion; j += 32) {
      if (j == e) continue;
      TW qp[3];
      int f;
      if (j < n_e) {
        qp[0] = (TW)P[j]; qp[1] = (TW)P[n_e + j]; qp[2] = (TW)P[2 * n_e + j];
        f = ((j >= S.n_up) == (e >= S.n_up)) ? 1 : 2;
      } else {
        const int J = j - n_e;
        qp[0] = ionw[J]; qp[1] = ionw[S.n_ion + J]; qp[2] = ionw[2 * S.n_ion + J];
        f = 0;
      }
      if (jt.M[f] == 0) continue;
      TW dn2 = TW(0), do2 = TW(0);
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        const TW an = min_image<TW>(xn[c] - qp[c], Lw, iLw), ao = min_image<TW>(xo[c] - qp[c], Lw, iLw);
        dn2 += an * an;
        do2 += ao * ao;
      }
      dj += jastrow_value_r2<TW>(jt, f, dn2) - jastrow_value_r2<TW>(jt, f, do2);
    }
    if (j3t.on) {
      TW g3[3];
      dj += j3_delta<TW, false>(S, j3t, P, ionw, e, xo, xn, Lw, iLw, j3_group_warps(lane, 32), g3);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) dj += __shfl_xor_sync(0xffffffffu, dj, o);
    const double wqq = __shfl_sync(0xffffffffu, wq, q);
    total += wqq * ((double)s + (double)sc) * exp((double)dj);
  }
  if (lane == 0) vals[(size_t)w * cap + k] = total;
}

// V_NL of each walker: the sum of its pairs' values in list order (one warp per walker, a
// fixed reduction tree), stored to vnl[w] and added to E_L.
static __global__ void k_nlpp_sum(WalkParams Wk, const double* __restrict__ vals,
                                  const int* __restrict__ count, int cap, double* __restrict__ vnl) {
  const long long gw = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (gw >= Wk.n_w) return;
  const int w = (int)gw;
  if (Wk.n_live && w >= *Wk.n_live) return;
  const int n = min(count[w], cap);
  double v = 0.0;
  for (int k = lane; k < n; k += 32) v += vals[(size_t)w * cap + k];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if (lane == 0) {
    vnl[w] = v;
    Wk.e_loc[w] += v;
  }
}

}  // namespace qmcgb
