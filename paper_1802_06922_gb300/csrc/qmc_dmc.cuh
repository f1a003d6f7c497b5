// Branching DMC with a variable population (Sec. "Diffusion Monte Carlo"): weights from
// the branching Green's function, stochastic copies, compaction and trial-energy feedback.
// Walker slots are padded to a capacity; the live count stays on the device, so a step
// never waits for the host.
#pragma once
#include "qmc_kernels.cuh"

namespace qmcgb {

// Copies M = floor(w + xi) of a walker, clamped to [0, cap] in double before the integer
// conversion: a weight of 2^31 or more (a walker next to a node) or a non-finite one must
// not overflow the prefix sums. Copies beyond the capacity are dropped in any case, so the
// clamp leaves every kept slot unchanged.
__device__ __forceinline__ int dmc_copies(double wgt, double xi, int cap) {
  const double mf = floor(wgt + xi);
  if (!(mf > 0.0)) return 0;
  return mf >= (double)cap ? cap : (int)mf;
}

// Teeth of the reconfiguration comb (k + xi) W / N, k = 0..N-1, below the cumulative weight c.
__device__ __forceinline__ int comb_teeth_below(double c, double W, int n, double xi) {
  const double t = ceil(c * (double)n / W - xi);
  return t <= 0.0 ? 0 : (t >= (double)n ? n : (int)t);
}

// One block. Weights w = exp(-tau_w/2 (E_old + E_new - 2 E_T)) (Eq. pmc:g_growth, Eq.
// pmc:walker_weight), tau_w = tau, or with D.tau_eff the walker's effective time step
// tau * (accepted |dr|^2) / (proposed |dr|^2) of this step's sweep (Umrigar, Nightingale and
// Runge). Copies: M = floor(w + xi) with xi from Philox block (step, 0xB, ID, 2); or, with
// D.reconfigure, a stochastic reconfiguration at a fixed count (Assaraf, Caffarel and
// Khelif): one comb of N teeth at (k + xi) W / N over the cumulative weights, xi from
// block (step, 0xC, 0, 2), walker i taking the teeth of [C_{i-1}, C_i) (the last walker
// the rest, so the counts add up to N). Destinations by prefix sums in walker order (the
// first copy keeps the ID, further copies take consecutive new IDs), population capped at
// `cap`, and E_T <- E_w - ln(N / N_target) / (10 tau) with E_w the weighted mean E_L of
// this step.
__global__ void __launch_bounds__(1024) k_dmc_branch(SysParams S, WalkParams Wk, DmcParams D,
                                                    int parity, uint32_t step0) {
  const uint32_t step = sweep_index(Wk, step0);
  __shared__ int scan[1024];
  __shared__ int scan2[1024];
  __shared__ double red[2 * 32];
  __shared__ double cscan[1024];
  const int n = D.n_live[parity];
  const int tid = threadIdx.x, nt = blockDim.x, lane = tid & 31, warp = tid >> 5;
  const double et = *D.e_trial;
  // each thread owns a contiguous range of walkers
  const int per = (n + nt - 1) / nt;
  const int i0 = min(n, tid * per), i1 = min(n, i0 + per);
  double sw = 0.0, swe = 0.0;
  for (int i = i0; i < i1; ++i) {
    double te = D.tau;
    if (D.tau_eff) {
      const double p = Wk.r2[2 * i], a = Wk.r2[2 * i + 1];
      te = p > 0.0 ? D.tau * a / p : 0.0;
    }
    const double wgt = exp(-0.5 * (D.e_old[i] + Wk.e_loc[i] - 2.0 * et) * te);
    Wk.weight[i] = wgt;
    sw += wgt;
    swe += wgt * Wk.e_loc[i];
  }
  // inclusive scan of the thread sums of the weights (the comb's cumulative weights)
  cscan[tid] = sw;
  __syncthreads();
  for (int o = 1; o < nt; o <<= 1) {
    const double a = tid >= o ? cscan[tid - o] : 0.0;
    __syncthreads();
    cscan[tid] += a;
    __syncthreads();
  }
  const double wtot = cscan[nt - 1];
  double cum = tid > 0 ? cscan[tid - 1] : 0.0;   // weight of the walkers before this range
  double xi_comb = 0.0;
  if (D.reconfigure) {
    const U32x4 r = philox4x32_10(step, 0xCu, 0u, 2u, S.seed_lo, S.seed_hi);
    xi_comb = unit_open(r.v[0]);
  }
  // copy counts of this thread's walkers
  auto copies = [&](int i, double c_before, double c_after) {
    if (D.reconfigure) {
      const int a = comb_teeth_below(c_before, wtot, n, xi_comb);
      const int b = i == n - 1 ? n : comb_teeth_below(c_after, wtot, n, xi_comb);
      return max(b - a, 0);
    }
    const U32x4 r = philox4x32_10(step, 0xBu, Wk.wid[i], 2u, S.seed_lo, S.seed_hi);
    return dmc_copies(Wk.weight[i], unit_open(r.v[0]), D.cap);
  };
  int mloc = 0, xloc = 0;
  {
    double c = cum;
    for (int i = i0; i < i1; ++i) {
      const double c1 = c + Wk.weight[i];
      const int M = copies(i, c, c1);
      c = c1;
      mloc = min(mloc + M, D.cap);               // sums bounded by cap: no overflow
      xloc = min(xloc + (M > 0 ? M - 1 : 0), D.cap);
    }
  }
  // block sums of the weights
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    sw += __shfl_xor_sync(0xffffffffu, sw, o);
    swe += __shfl_xor_sync(0xffffffffu, swe, o);
  }
  if (lane == 0) { red[warp] = sw; red[32 + warp] = swe; }
  // exclusive scans of copies and extra copies over the thread ranges
  scan[tid] = mloc;
  scan2[tid] = xloc;
  __syncthreads();
  for (int o = 1; o < nt; o <<= 1) {
    const int a = tid >= o ? scan[tid - o] : 0, b = tid >= o ? scan2[tid - o] : 0;
    __syncthreads();
    scan[tid] += a;
    scan2[tid] += b;
    __syncthreads();
  }
  const int total = scan[nt - 1];
  int dest = scan[tid] - mloc;
  int xr = scan2[tid] - xloc;
  const uint32_t nid = *D.next_id;
  for (int i = i0; i < i1; ++i) {
    const double c1 = cum + Wk.weight[i];
    const int M = copies(i, cum, c1);
    cum = c1;
    for (int c = 0; c < M && dest + c < D.cap; ++c) {
      const int d = dest + c;
      D.src_of[d] = i;
      D.wid_next[d] = c == 0 ? Wk.wid[i] : nid + (uint32_t)(xr + c - 1);
    }
    dest = min(dest + M, D.cap);
    xr = min(xr + (M > 0 ? M - 1 : 0), D.cap);
  }
  __syncthreads();
  if (tid == 0) {
    double tw = 0.0, twe = 0.0;
    for (int q = 0; q < (nt >> 5); ++q) { tw += red[q]; twe += red[32 + q]; }
    const int kept = min(total, D.cap);
    // kept extra copies: all copies in slots [0, kept) that are not first copies
    int kept_extra = 0;
    for (int d = 0; d < kept; ++d)
      if (D.wid_next[d] >= nid) ++kept_extra;
    const double emean = twe / tw;
    const double et_new = emean - log((double)max(kept, 1) / (double)D.n_target) / (10.0 * D.tau);
    D.stats[0] = tw;
    D.stats[1] = twe;
    D.stats[2] = emean;
    D.stats[3] = et;
    D.stats[4] = (double)n;
    D.stats[5] = (double)kept;
    *D.e_trial = et_new;
    *D.next_id = nid + (uint32_t)kept_extra;
    D.n_live[parity ^ 1] = kept;
  }
}

// Copy of the state of parent src_of[d] into destination slot d of the other buffer.
template <class TW>
__global__ void __launch_bounds__(256) k_dmc_copy(SysParams S, WalkParams src, WalkParams dst,
                                                 DmcParams D, int parity) {
  const int d = blockIdx.x;
  if (d >= D.n_live[parity ^ 1]) return;
  const int i = D.src_of[d];
  const int n_e = S.n_e;
  const size_t nv = (size_t)n_e * 5 * src.ld_v;
  const int tid = threadIdx.x, nt = blockDim.x;
  for (int k = tid; k < 3 * n_e; k += nt) dst.pos[(size_t)d * 3 * n_e + k] = src.pos[(size_t)i * 3 * n_e + k];
  for (int spin = 0; spin < 2; ++spin) {
    const size_t nb = spin ? (size_t)S.n_dn * S.n_dn : (size_t)S.n_up * S.n_up;
    const TW* bs = binv_block<const TW>(S, src, i, spin);
    TW* bd = binv_block<TW>(S, dst, d, spin);
    for (size_t k = tid; k < nb; k += nt) bd[k] = bs[k];
  }
  const float4* vs = reinterpret_cast<const float4*>(static_cast<const TW*>(src.vgl) + (size_t)i * nv);
  float4* vd = reinterpret_cast<float4*>(static_cast<TW*>(dst.vgl) + (size_t)d * nv);
  const size_t nv4 = nv * sizeof(TW) / 16;
  for (size_t k = tid; k < nv4; k += nt) vd[k] = vs[k];
  if (tid < 2) {
    dst.logdet[2 * d + tid] = src.logdet[2 * i + tid];
    dst.sgn[2 * d + tid] = src.sgn[2 * i + tid];
    dst.acc_since[2 * d + tid] = src.acc_since[2 * i + tid];
  }
  if (tid == 0) {
    dst.wid[d] = D.wid_next[d];
    dst.weight[d] = 1.0;
    dst.e_loc[d] = src.e_loc[i];
    dst.log_psi[d] = src.log_psi[i];
    dst.n_acc[d] = src.n_acc[i];
    D.e_old_next[d] = src.e_loc[i];
  }
}

}  // namespace qmcgb
