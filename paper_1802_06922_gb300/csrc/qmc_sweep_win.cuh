// Metropolis sweep of one launch of the batched delayed update (Sec. "Multi-Determinant
// Slater-Jastrow Form", delayed updates; Sec. "Trial Moves", Eq. accept_reject).
//
// A launch covers the moves t = 0 .. kk-1 (electrons e_t = e0 + t, kk <= k) of one spin
// block. The inverse Binv0 is fixed during the launch (the window is flushed and the
// inverse refined by the batched kernels between launches), and the proposals r'_t with
// their orbital rows phi'_t were evaluated before it. Every dot product a move needs is
// then an entry of one kk x kk matrix formed at the start of the launch,
//   D[a][b] = phi'_a . Binv0[e_b],
// because an accepted move's new row Phi_l is its proposal row and U_l = Binv0[e_l]:
//   d_l  = Phi_l . Binv0[e_t]   = D[t_l][t]        (the window's d for move t)
//   crow = phi'_t . U_l         = D[t][t_l]        (the row that borders C)
//   a    = phi'_t . Binv0[e_t]  = D[t][t]
// and the ratio is the Schur complement a - crow . C^-1 d = a - y . d of the bordered C,
// y = C^-T crow. Per move the determinant costs O(m^2) for the window fill m instead of
// O(m N_s), and the product that forms D runs at full parallelism before the sequential
// part starts. All dots are compensated (TwoProduct and TwoSum); the diagonal keeps its pair.
//
// The Jastrow difference is regrouped the same way (Sec. "Jastrow factor"). Positions change
// within the launch only through its accepted moves, so
//   Delta J(t) = base[t] + sum over accepted t' < t of Q[t][t'],
// base[t] = sum_j u(|r'_t - r_j|) - u(|r_e_t - r_j|) with the positions at the launch start,
// Q[t][t'] = u(|r'_t - r'_t'|) - u(|r'_t - r_e_t'|) - u(|r_e_t - r'_t'|) + u(|r_e_t - r_e_t'|)
// (the pair of the two moved electrons, same spin). Both are formed before the moves.
//
// Roles within a move: the determinant warps form z = C^-1 d (one warp) and y with the
// ratio (the other) while the remaining warps evaluate the Jastrow difference; warp 0
// decides while the other warps border C^-1 into a second buffer (kept on acceptance). One thread moves each accepted move's rows with the bulk-copy unit, one move
// behind: its VGL row to the current set, its value and inverse rows to the window that
// the batched flush kernel receives.
#pragma once
#include "qmc_kernels.cuh"

namespace qmcgb {

constexpr int kWinMaxK = 32;          // moves per launch covered by the pair matrix D
constexpr int kWinP = kWinMaxK + 1;   // padded row length of D, WD, WC and C^-1
constexpr int kWinKc = 64;            // orbital chunk of the product that forms D
constexpr int kWinKs = kWinKc + 4;    // staged row length (16-byte rows, conflict-free reads)
constexpr int kWinDetWarps = 2;       // warps on z, y and the ratio
constexpr int kWinThreads = 256;      // the product's thread map assumes 256 threads
constexpr long long kWinWaitPolls = 20000000;   // bounded wait for a bulk copy (polls)

// u rounded down to working precision: for TW-valued A, u < A exactly when RD(u) < A.
__device__ __forceinline__ float round_down_w(double u, float) { return __double2float_rd(u); }
__device__ __forceinline__ double round_down_w(double u, double) { return u; }

template <class TW>
struct WinSmem {
  double* prop;   // [kWinMaxK][4] the launch's proposals (x, y, z, u)
  TW* propw;      // [kWinMaxK][4] the same in working precision, u rounded down
  double* posd;   // [3][n_e] exact positions
  TW* stg;        // [2][6 ld_v] bulk-copy staging: an accepted move's VGL row and inverse row
  TW* posw;       // [3][n_e] positions in working precision
  TW* D;          // [kWinMaxK][kWinP]
  TW* cinv;       // [2][kWinMaxK][kWinP] C^-1 of the window and its bordered successor
  TW* WD;         // [kWinMaxK][kWinP] WD[l][t] = D[t_l][t]: d_l of move t
  TW* WC;         // [kWinMaxK][kWinP] WC[t][l] = D[t][t_l]: crow_l of move t
  TW* dlo;        // [kWinMaxK] compensation of D's diagonal
  TW* jb;         // [kWinMaxK] Jastrow difference of each move at the launch-start positions
  TW* Q;          // [kWinMaxK][kWinP] pair corrections of the Jastrow difference
  TW* zvec;       // [kWinMaxK]
  TW* yvec;       // [kWinMaxK]
  TW* stA;        // [2][kWinMaxK][kWinKs] staged proposal value rows
  TW* stB;        // [2][kWinMaxK][kWinKs] staged inverse rows
  TW* red;        // [32][8] warp partials
  TW* sc;         // [8] sc[5]: the decided ratio; sc[6], sc[7]: the ratio as a pair
  int* wt;        // [kWinMaxK] move index t_l of window row l
  int* flag;      // [4]
};

template <class TW>
__host__ __device__ inline size_t sweep_win_smem_bytes(int n_e, int ld_v) {
  size_t b = sizeof(double) * (4 * (size_t)kWinMaxK + 3 * (size_t)n_e);
  b = (b + 15) & ~size_t(15);
  b += sizeof(TW) * (12 * (size_t)ld_v + 3 * (size_t)n_e + 6 * (size_t)kWinMaxK * kWinP + 4 * kWinMaxK +
                     4 * kWinMaxK + 4 * (size_t)kWinMaxK * kWinKs + 32 * 8 + 8);
  b += sizeof(int) * (kWinMaxK + 4);
  return b + 32;
}

template <class TW>
__device__ __forceinline__ WinSmem<TW> carve_win(char* base, int n_e, int ld_v) {
  WinSmem<TW> s;
  double* d = reinterpret_cast<double*>(base);
  s.prop = d; d += 4 * kWinMaxK;
  s.posd = d; d += 3 * n_e;
  char* c = reinterpret_cast<char*>(d);
  c = base + ((c - base + 15) & ~size_t(15));
  TW* t = reinterpret_cast<TW*>(c);
  s.stg = t; t += 12 * ld_v;                       // 16-byte aligned (ld_v is a multiple of 8)
  s.stA = t; t += 2 * kWinMaxK * kWinKs;           // 16-byte aligned rows
  s.stB = t; t += 2 * kWinMaxK * kWinKs;
  s.posw = t; t += 3 * n_e;
  s.propw = t; t += 4 * kWinMaxK;
  s.D = t; t += kWinMaxK * kWinP;
  s.cinv = t; t += 2 * kWinMaxK * kWinP;
  s.WD = t; t += kWinMaxK * kWinP;
  s.WC = t; t += kWinMaxK * kWinP;
  s.dlo = t; t += kWinMaxK;
  s.jb = t; t += kWinMaxK;
  s.Q = t; t += kWinMaxK * kWinP;
  s.zvec = t; t += kWinMaxK;
  s.yvec = t; t += kWinMaxK;
  s.red = t; t += 32 * 8;
  s.sc = t; t += 8;
  int* ip = reinterpret_cast<int*>(t);
  s.wt = ip; ip += kWinMaxK;
  s.flag = ip;
  return s;
}

// One block of kWinThreads threads per walker; moves e0 .. e1-1 (at most kWinMaxK and at
// most the window capacity Wk.kc <= kWinMaxK); Pv and prop hold the proposals of the
// electrons p_e0 .. p_e0 + p_n - 1 of every walker.
template <class TW, bool kFixedNode>
__global__ void __launch_bounds__(kWinThreads, 2)
    k_sweep_win(SysParams S, WalkParams Wk, int e0, int e1, const TW* __restrict__ Pv,
                const Prop* __restrict__ prop, int p_e0, int p_n) {
  extern __shared__ __align__(16) char smem_w[];
  __shared__ JastrowTab<TW> jt;
  __shared__ J3Tab<TW> j3t;
  __shared__ int j3_near[kWinMaxK][kJ3MaxNear];   // three-body Jastrow: ions near each move
  __shared__ int j3_nn[kWinMaxK];
  __shared__ __align__(8) uint64_t cp_bar[2];
  const int w = blockIdx.x;
  if (Wk.n_live && w >= *Wk.n_live) return;            // empty DMC slot
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  constexpr int nt = kWinThreads, nw = kWinThreads / 32;
  constexpr int nJ = nw - kWinDetWarps, dnt = 32 * kWinDetWarps, jn = 32 * nJ;
  constexpr int kBook = 32 * (nJ - 1);                 // keeps ln|det|, the sign, the count
  constexpr int kCopier = 32 * (nJ - 1) + 1;           // issues the bulk copies
  const int n_e = S.n_e, ld_v = Wk.ld_v, kc = Wk.kc, kk = e1 - e0;
  WinSmem<TW> sm = carve_win<TW>(smem_w, n_e, ld_v);
  const int spin = e0 >= S.n_up ? 1 : 0;
  const int first = spin ? S.n_up : 0;
  const int ns = spin ? S.n_dn : S.n_up;
  const TW Lw = Cst<TW>::L(S), iLw = Cst<TW>::invL(S);
  const TW* ionw = Cst<TW>::ions(S);
  const TW* B = binv_block<const TW>(S, Wk, w, spin);
  const TW* B0 = B + (size_t)(e0 - first) * ns;                        // row of move t: B0 + t ns
  const TW* P0 = Pv + ((size_t)w * p_n + (e0 - p_e0)) * 5 * ld_v;      // rows of move t: P0 + 5 t ld_v
  double* gpos = Wk.pos + (size_t)w * 3 * n_e;
  // positions and proposals arrive asynchronously while D is formed
  for (int i = tid; i < 3 * n_e; i += nt) cp_async_elem(sm.posd + i, gpos + i);
  {
    const double* pr = reinterpret_cast<const double*>(prop + (size_t)w * p_n + (e0 - p_e0));
    for (int i = tid; i < 4 * kk; i += nt) cp_async_elem(sm.prop + i, pr + i);
  }
  cp_async_commit();
  jastrow_tab_fill<TW>(S, jt);
  j3_tab_fill<TW>(S, j3t);
  if (tid == kCopier) {
    tc::mbar_init(&cp_bar[0], 1);
    tc::mbar_init(&cp_bar[1], 1);
    tc::fence_mbar_init();
  }

  // ---- D[a][b] = phi'_a . Binv0[e_b]; thread (a, b0) owns the outputs (a, b0 + 8q), q < 4.
  // Orbital chunks of kWinKc staged by cp.async, the next chunk in flight during the current.
  {
    const int a = tid >> 3, b0 = tid & 7;
    TW s[4] = {0, 0, 0, 0}, c[4] = {0, 0, 0, 0};
    const int nch = (ns + kWinKc - 1) / kWinKc;
    const auto stage = [&](int ch) {
      const int k0 = ch * kWinKc, kw = min(kWinKc, ns - k0);
      TW* A = sm.stA + (ch & 1) * kWinMaxK * kWinKs;
      TW* Bs = sm.stB + (ch & 1) * kWinMaxK * kWinKs;
      for (int i = tid; i < kk * kWinKc; i += nt) {
        const int r = i / kWinKc, k = i - r * kWinKc;
        if (k < kw) {
          cp_async_elem(A + r * kWinKs + k, P0 + (size_t)r * 5 * ld_v + k0 + k);
          cp_async_elem(Bs + r * kWinKs + k, B0 + (size_t)r * ns + k0 + k);
        }
      }
      cp_async_commit();
    };
    stage(0);
    for (int ch = 0; ch < nch; ++ch) {
      if (ch + 1 < nch) {
        stage(ch + 1);
        cp_async_wait_1();
      } else {
        cp_async_wait_all();
      }
      __syncthreads();
      const int kw = min(kWinKc, ns - ch * kWinKc);
      const TW* pa = sm.stA + (ch & 1) * kWinMaxK * kWinKs + a * kWinKs;
      const TW* pb = sm.stB + (ch & 1) * kWinMaxK * kWinKs + b0 * kWinKs;
      if (a < kk)
        for (int k = 0; k < kw; ++k) {
          const TW x = pa[k];
#pragma unroll
          for (int q = 0; q < 4; ++q) comp_fma(s[q], c[q], x, pb[8 * q * kWinKs + k]);
        }
      __syncthreads();                                 // this buffer is refilled two chunks on
    }
    if (a < kk) {
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int b = b0 + 8 * q;
        if (b == a) {
          sm.D[a * kWinP + a] = s[q];
          sm.dlo[a] = c[q];
        } else if (b < kk) {
          sm.D[a * kWinP + b] = s[q] + c[q];
        }
      }
    }
  }
  for (int i = tid; i < 3 * n_e; i += nt) sm.posw[i] = (TW)sm.posd[i];   // positions landed
  for (int i = tid; i < 4 * kk; i += nt)
    sm.propw[i] = (i & 3) == 3 ? round_down_w(sm.prop[i], TW(0)) : (TW)sm.prop[i];
  __syncthreads();

  // ---- the Jastrow difference of every move at the launch-start positions (8 threads per
  // move) and the pair corrections Q
  {
    static_assert(kWinThreads / 8 >= kWinMaxK, "one group of 8 threads per move");
    const int t = tid >> 3, gl = tid & 7;      // every lane takes part in the group sums
    TW v = TW(0);
    if (t < kk) {
      const TW rn[3] = {sm.propw[4 * t], sm.propw[4 * t + 1], sm.propw[4 * t + 2]};
      v = jastrow_delta_value<TW>(S, jt, sm.posw, ionw, e0 + t, rn, Lw, iLw, gl, 8);
      if (j3t.on) {
        // the three-body term, with the list of ions near the move for the pair corrections
        const int e = e0 + t;
        const TW ro[3] = {sm.posw[e], sm.posw[n_e + e], sm.posw[2 * n_e + e]};
        TW g3[3];
        int nn = 0;
        v += j3_delta<TW, false>(S, j3t, sm.posw, ionw, e, ro, rn, Lw, iLw,
                                 j3_group_sub(8, gl, 8), g3, j3_near[t], kJ3MaxNear, &nn);
        if (gl == 0) {
          j3_nn[t] = min(nn, kJ3MaxNear);
          if (nn > kJ3MaxNear) atomicOr(Wk.err, kErrJ3Near);
        }
      }
    }
#pragma unroll
    for (int o = 4; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (t < kk && gl == 0) sm.jb[t] = v;
    if (j3t.on) __syncthreads();                // the near-ion lists are complete
    for (int i = tid; i < kk * kk; i += nt) {
      const int ta = i / kk, tb = i - ta * kk;
      TW q = TW(0);
      if (ta != tb) {
        TW d2[4] = {0, 0, 0, 0};   // (r'_a, r'_b), (r'_a, r_b), (r_a, r'_b), (r_a, r_b)
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          const TW pa = sm.propw[4 * ta + c], pb = sm.propw[4 * tb + c];
          const TW oa = sm.posw[c * n_e + e0 + ta], ob = sm.posw[c * n_e + e0 + tb];
          const TW x0 = min_image<TW>(pa - pb, Lw, iLw), x1 = min_image<TW>(pa - ob, Lw, iLw);
          const TW x2 = min_image<TW>(oa - pb, Lw, iLw), x3 = min_image<TW>(oa - ob, Lw, iLw);
          d2[0] += x0 * x0; d2[1] += x1 * x1; d2[2] += x2 * x2; d2[3] += x3 * x3;
        }
        q = (jastrow_value_r2<TW>(jt, 1, d2[0]) - jastrow_value_r2<TW>(jt, 1, d2[1])) -
            (jastrow_value_r2<TW>(jt, 1, d2[2]) - jastrow_value_r2<TW>(jt, 1, d2[3]));
        if (j3t.on) {
          const TW pa[3] = {sm.propw[4 * ta], sm.propw[4 * ta + 1], sm.propw[4 * ta + 2]};
          const TW pb[3] = {sm.propw[4 * tb], sm.propw[4 * tb + 1], sm.propw[4 * tb + 2]};
          const TW oa[3] = {sm.posw[e0 + ta], sm.posw[n_e + e0 + ta], sm.posw[2 * n_e + e0 + ta]};
          const TW ob[3] = {sm.posw[e0 + tb], sm.posw[n_e + e0 + tb], sm.posw[2 * n_e + e0 + tb]};
          q += j3_pair_correction<TW>(S, j3t, ionw, j3_near[ta], j3_nn[ta], pa, oa, pb, ob, Lw, iLw);
        }
      }
      sm.Q[ta * kWinP + tb] = q;
    }
  }

  // ---- the moves
  double logdet = 0.0, sgn = 1.0, lprod = 1.0;   // ln|det| = logdet + ln lprod + lexp ln 2
  int lexp = 0;
  long long nacc = 0;
  if (tid == kBook) {
    logdet = Wk.logdet[2 * w + spin];
    sgn = Wk.sgn[2 * w + spin];
  }
  const bool det = warp >= nJ;
  const int dw = warp - nJ, dt = tid - jn;
  const bool trace = Wk.trace != nullptr;
  TW* VG = static_cast<TW*>(Wk.vgl) + (size_t)w * n_e * 5 * ld_v;
  TW* gphi = static_cast<TW*>(Wk.win_phi) + (size_t)w * kc * ld_v;
  TW* gu = static_cast<TW*>(Wk.win_u) + (size_t)w * kc * ld_v;
  // an accepted move's rows: the VGL row (5 ld_v) and, when its rows are 16-byte aligned, the
  // inverse row through the staging buffer; otherwise the inverse row by plain copies
  const bool row_vec = (ns * sizeof(TW)) % 16 == 0 && (reinterpret_cast<uintptr_t>(B) & 15) == 0;
  const uint32_t nb_vgl = 5u * ld_v * sizeof(TW), nb_val = ld_v * sizeof(TW);
  const uint32_t nb_row = row_vec ? ns * sizeof(TW) : 0u;
  int ncp = 0;                  // copier: bulk loads issued (staging buffer ncp & 1)
  int cp_t = -1, cp_l = -1;     // copier: move and window row of the load in flight
  bool cp_ok = true;
  // copier: the staged rows of (cp_t, cp_l) go out, the rows of move tp (window row lp) come in
  const auto copy_step = [&](int tp, int lp) {
    if (cp_t >= 0) {
      const int sb = (ncp - 1) & 1;
      TW* st = sm.stg + (size_t)sb * 6 * ld_v;
      cp_ok = tc::mbar_wait(&cp_bar[sb], (uint32_t)(((ncp - 1) >> 1) & 1), kWinWaitPolls) && cp_ok;
      tc::bulk_s2g(VG + (size_t)(e0 + cp_t) * 5 * ld_v, st, nb_vgl);
      tc::bulk_s2g(gphi + (size_t)cp_l * ld_v, st, nb_val);
      if (nb_row) tc::bulk_s2g(gu + (size_t)cp_l * ld_v, st + 5 * ld_v, nb_row);
      tc::bulk_commit();
      cp_t = -1;
    }
    if (tp >= 0) {
      const int sb = ncp & 1;
      TW* st = sm.stg + (size_t)sb * 6 * ld_v;
      tc::bulk_wait_read<1>();          // the stores that read this buffer two loads ago are done
      tc::mbar_arrive_expect_tx(&cp_bar[sb], nb_vgl + nb_row);
      tc::bulk_g2s(st, P0 + (size_t)tp * 5 * ld_v, nb_vgl, &cp_bar[sb]);
      if (nb_row) tc::bulk_g2s(st + 5 * ld_v, B0 + (size_t)tp * ns, nb_row, &cp_bar[sb]);
      ++ncp;
      cp_t = tp;
      cp_l = lp;
    }
  };
  int m = 0, cb = 0, pend = -1;   // window fill, current C^-1 buffer, move accepted last
  __syncthreads();                // D, positions, proposals and the copy barriers in place
  for (int t = 0; t < kk; ++t) {
    const int e = e0 + t;
    const TW* ci = sm.cinv + cb * kWinMaxK * kWinP;
    // v: Delta J, grad J at r' (3), grad phi' . x (3); the last six only for a trace
    TW v[7] = {0, 0, 0, 0, 0, 0, 0};
    if (!det) {
      if (tid == kCopier) copy_step(pend, m - 1);
      if (trace) {
        // the gradient of J at r' for the trace (Delta J itself comes from jb and Q)
        const TW rn[3] = {sm.propw[4 * t], sm.propw[4 * t + 1], sm.propw[4 * t + 2]};
        TW g[3];
        (void)jastrow_delta_grad<TW>(S, jt, sm.posw, ionw, e, rn, Lw, iLw, tid, jn, g);
        if (j3t.on) {
          const TW ro[3] = {sm.posw[e], sm.posw[n_e + e], sm.posw[2 * n_e + e]};
          TW g3[3];
          (void)j3_delta<TW, true>(S, j3t, sm.posw, ionw, e, ro, rn, Lw, iLw,
                                   j3_group_warps(tid, jn), g3);
          g[0] += g3[0]; g[1] += g3[1]; g[2] += g3[2];
        }
        v[1] = g[0]; v[2] = g[1]; v[3] = g[2];
      }
    } else {
      if (pend >= 0 && !row_vec)
        for (int j = dt; j < ns; j += dnt) gu[(size_t)(m - 1) * ld_v + j] = B0[(size_t)pend * ns + j];
      TW z0 = TW(0), c0 = TW(0), z1 = TW(0), c1 = TW(0);
      if (lane < m) {
        int l = 0;
        if (dw == 0) {
          // z = C^-1 d, d_l = WD[l][t]: row `lane` of C^-1
          const TW* cr = ci + lane * kWinP;
          for (; l + 1 < m; l += 2) {
            comp_fma(z0, c0, cr[l], sm.WD[l * kWinP + t]);
            comp_fma(z1, c1, cr[l + 1], sm.WD[(l + 1) * kWinP + t]);
          }
          if (l < m) comp_fma(z0, c0, cr[l], sm.WD[l * kWinP + t]);
        } else {
          // y = C^-T crow, crow_l = WC[t][l]: column `lane` of C^-1
          const TW* cw = sm.WC + t * kWinP;
          for (; l + 1 < m; l += 2) {
            comp_fma(z0, c0, cw[l], ci[l * kWinP + lane]);
            comp_fma(z1, c1, cw[l + 1], ci[(l + 1) * kWinP + lane]);
          }
          if (l < m) comp_fma(z0, c0, cw[l], ci[l * kWinP + lane]);
        }
        comp_merge(z0, c0, z1, c1);
        (dw == 0 ? sm.zvec : sm.yvec)[lane] = z0 + c0;
      }
      if (dw == 1) {
        // the ratio a - y . d = a - crow . C^-1 d, also the corner of the bordered C
        TW sv = TW(0), sc2 = TW(0);
        if (lane < m) comp_fma(sv, sc2, -(z0 + c0), sm.WD[lane * kWinP + t]);
        warp_sum_comp(sv, sc2);
        if (lane == 0) {
          TW a = sm.D[t * kWinP + t], ac = sm.dlo[t];
          comp_merge(a, ac, sv, sc2);
          sm.sc[6] = a;
          sm.sc[7] = ac;
        }
      }
      if (trace) {
        // x = Binv0[e] - sum_l z_l U_l (compensated) and grad phi' . x
        named_barrier(2, dnt);
        const TW* pg = P0 + (size_t)t * 5 * ld_v;
        for (int j = dt; j < ns; j += dnt) {
          TW xv = B0[(size_t)t * ns + j], xc = TW(0);
          for (int l = 0; l < m; ++l) comp_fma(xv, xc, -sm.zvec[l], B0[(size_t)sm.wt[l] * ns + j]);
          xv += xc;
          v[4] += pg[ld_v + j] * xv;
          v[5] += pg[2 * ld_v + j] * xv;
          v[6] += pg[3 * ld_v + j] * xv;
        }
      }
    }
    if (trace) {
      warp_sum<7, TW>(v);
      if (lane == 0)
#pragma unroll
        for (int k = 0; k < 7; ++k) sm.red[warp * 8 + k] = v[k];
    }
    __syncthreads();
    if (warp == 0) {
      TW tot[7] = {0, 0, 0, 0, 0, 0, 0};
      if (trace) {
        TW tv = TW(0);
        if (lane < 7)
#pragma unroll
          for (int q = 0; q < nw; ++q) tv += sm.red[q * 8 + lane];
#pragma unroll
        for (int k = 0; k < 7; ++k) tot[k] = __shfl_sync(0xffffffffu, tv, k);
      }
      {
        // Delta J = jb[t] + sum over the window's moves of Q[t][t_l]
        TW dj = lane < m ? sm.Q[t * kWinP + sm.wt[lane]] : TW(0);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) dj += __shfl_xor_sync(0xffffffffu, dj, o);
        tot[0] = sm.jb[t] + dj;
      }
      if (lane == 0) {
        const TW R = sm.sc[6] + sm.sc[7], dJ = tot[0];
        const bool ok = (R != TW(0)) && isfinite(R);
        const TW A = ok ? fmin(TW(1), R * R * texp<TW>(TW(2) * dJ)) : TW(0);
        bool accept = sm.propw[4 * t + 3] < A;          // u < A with u in FP64
        if (kFixedNode && R < TW(0)) accept = false;
        if (Wk.forced) accept = Wk.forced[(size_t)w * n_e + e] != 0;
        sm.flag[0] = accept;
        sm.sc[5] = R;
        if (accept) {
#pragma unroll
          for (int c = 0; c < 3; ++c) sm.posw[c * n_e + e] = sm.propw[4 * t + c];
          sm.wt[m] = t;
        }
        if (trace) {
          const double u = sm.prop[4 * t + 3];
          double* tr = Wk.trace + ((size_t)w * n_e + e) * 8;
          tr[0] = (double)R;
          tr[1] = (double)dJ;
#pragma unroll
          for (int c = 0; c < 3; ++c) tr[2 + c] = (ok ? (double)(tot[4 + c] / R) : 0.0) + (double)tot[1 + c];
          tr[5] = u;
          tr[6] = (double)A;
          tr[7] = accept ? 1.0 : 0.0;
        }
      }
    } else {
      // border C^-1 through its Schur complement R into the other buffer, kept only if the
      // move is accepted: [[C^-1 + z y^T / R, -z / R], [-y^T / R, 1 / R]], a row per warp
      const TW sinv = TW(1) / (sm.sc[6] + sm.sc[7]);
      TW* cn = sm.cinv + (cb ^ 1) * kWinMaxK * kWinP;
      const int m1 = m + 1;
      for (int a = warp - 1; a < m1; a += nw - 1) {
        if (lane < m1) {
          const int b = lane;
          TW cv;
          if (a < m)
            cv = b < m ? ci[a * kWinP + b] + sm.zvec[a] * sm.yvec[b] * sinv : -sm.zvec[a] * sinv;
          else
            cv = b < m ? -sm.yvec[b] * sinv : sinv;
          cn[a * kWinP + b] = cv;
        }
      }
      // the would-be window row's d and crow entries of the later moves
      if (warp == nw - 1)
        for (int t2 = lane; t2 < kk; t2 += 32) sm.WD[m * kWinP + t2] = sm.D[t * kWinP + t2];
      if (warp == nw - 2)
        for (int t2 = lane; t2 < kk; t2 += 32) sm.WC[t2 * kWinP + m] = sm.D[t2 * kWinP + t];
    }
    __syncthreads();
    pend = -1;
    if (sm.flag[0]) {
      if (tid == kBook) {
        const TW R = sm.sc[5];
        ++nacc;
        int ex;
        lprod = frexp(lprod * fabs((double)R), &ex);
        lexp += ex;
        if (R < TW(0)) sgn = -sgn;
#pragma unroll
        for (int c = 0; c < 3; ++c) sm.posd[c * n_e + e] = sm.prop[4 * t + c];
      }
      cb ^= 1;
      pend = t;
      ++m;
    }
  }
  // the last accepted rows; every bulk copy completes before the block exits
  if (tid == kCopier) {
    copy_step(pend, m - 1);
    copy_step(-1, -1);
    tc::bulk_wait_all<0>();
    if (!cp_ok) atomicOr(Wk.err, kErrTimeout);
  }
  if (pend >= 0 && !row_vec)
    for (int j = tid; j < ns; j += nt) gu[(size_t)(m - 1) * ld_v + j] = B0[(size_t)pend * ns + j];
  __syncthreads();

  // ---- hand C^-1 of the window to the batched flush kernel
  const TW* ci = sm.cinv + cb * kWinMaxK * kWinP;
  TW* gc = static_cast<TW*>(Wk.win_cinv) + (size_t)w * kc * kc;
  for (int i = tid; i < kc * kc; i += nt) {
    const int a = i / kc, b = i - a * kc;
    gc[i] = (a < m && b < m) ? ci[a * kWinP + b] : TW(0);
  }
  for (int i = tid; i < m; i += nt) Wk.win_row[(size_t)w * kc + i] = e0 + sm.wt[i] - first;
  // positions of this launch's electrons (the only ones it can move)
  for (int i = tid; i < 3 * (e1 - e0); i += nt) {
    const int c = i / (e1 - e0), j = c * n_e + e0 + (i - c * (e1 - e0));
    gpos[j] = sm.posd[j];
  }
  if (tid == 0) Wk.win_m[w] = m;
  if (tid == kBook) {
    Wk.logdet[2 * w + spin] = logdet + log(lprod) + (double)lexp * 0.69314718055994530942;
    Wk.sgn[2 * w + spin] = sgn;
    Wk.n_acc[w] += nacc;
  }
}

}  // namespace qmcgb
