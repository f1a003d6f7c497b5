// Coulomb interactions of the periodic cell by Ewald summation (Sec. "Hamiltonian": v_ee =
// 1/r, v_eI = -Z/r and v_II = Z^2/r summed over every image of the cell, evaluated with the
// Ewald technique; Sec. "Long-Range Interactions": a short-ranged part summed in real space
// and a long-ranged part summed in reciprocal space). With splitting parameter alpha, point
// charges q (electrons -1, ions +Z) in a cube of side L and volume Omega, a neutralising
// background when the cell is charged, and the half set H of k = 2 pi n / L, |k| <= k_cut
// (one vector of each +-k pair):
//   V = sum_{a<b} q_a q_b erfc(alpha r_ab) / r_ab                          (nearest image)
//     + (4 pi / Omega) sum_{k in H} exp(-k^2 / (4 alpha^2)) / k^2 |rho_k|^2
//     - alpha / sqrt(pi) sum_a q_a^2 - pi Q^2 / (2 Omega alpha^2),   rho_k = sum_a q_a e^{i k.r_a}.
// The real-space pairs involving an electron are summed by the local-energy kernel; this
// file holds the reciprocal-space sum of every walker and the setup of the parts that do not
// depend on the electrons (the ions' rho_k, the coefficients c_k and the constant terms).
#pragma once
#include "qmc_device.cuh"
#include "qmc_internal.h"

namespace qmcgb {

constexpr int kEwThreads = 256;

// Phases e^{i k.r} = e^{2 pi i n.s} with s = r / L taken as a B-bit fixed-point fraction
// (s = round(2^B (x/L - rint(x/L))) mod 2^B): n.s mod 2^B is then the phase in turns, exact in
// wrapping integer arithmetic, with no argument reduction however large n.s grows; the
// signed phase p / 2^B in [-1/2, 1/2) turns into sin and cos by sincospi(2 p / 2^B).
// B = 32 in single precision (phase quantum 2^-32 turn), 64 in double.
template <class TW> struct EwFixed;
template <> struct EwFixed<float> {
  using U = uint32_t;
  __device__ static __forceinline__ U frac(double x, double invL) {
    const double f = x * invL - rint(x * invL);
    return (U)(long long)llrint(f * 4294967296.0);
  }
  __device__ static __forceinline__ void sincos_turn(U p, float& s, float& c) {
    sincospif((float)(int32_t)p * 0x1p-31f, &s, &c);
  }
};
template <> struct EwFixed<double> {
  using U = unsigned long long;
  __device__ static __forceinline__ U frac(double x, double invL) {
    const double f = x * invL - rint(x * invL);
    return (U)llrint(f * 0x1p63) << 1;
  }
  __device__ static __forceinline__ void sincos_turn(U p, double& s, double& c) {
    sincospi((double)(long long)p * 0x1p-63, &s, &c);
  }
};

// c_k = (4 pi / Omega) exp(-k^2 / (4 alpha^2)) / k^2 and the ions' share of rho_k,
// Z sum_I e^{i k.R_I} (re at rho[k], im at rho[n_k + k]); FP64. One thread per k.
static __global__ void k_ewald_kspace_setup(SysParams S, double* ck, double* rho) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= S.ew_nk) return;
  const int4 n = S.ew_n[k];
  const double tl = 2.0 * M_PI / S.L;
  const double kx = tl * n.x, ky = tl * n.y, kz = tl * n.z;
  const double k2 = kx * kx + ky * ky + kz * kz;
  ck[k] = 4.0 * M_PI / (S.L * S.L * S.L) * exp(-k2 / (4.0 * S.ew_alpha * S.ew_alpha)) / k2;
  using F = EwFixed<double>;
  const F::U ax = (F::U)(long long)n.x, ay = (F::U)(long long)n.y, az = (F::U)(long long)n.z;
  double re = 0.0, im = 0.0;
  for (int I = 0; I < S.n_ion; ++I) {
    const F::U p = ax * F::frac(S.ions[I], S.invL) + ay * F::frac(S.ions[S.n_ion + I], S.invL) +
                   az * F::frac(S.ions[2 * S.n_ion + I], S.invL);
    double s, c;
    F::sincos_turn(p, s, c);
    re += c;
    im += s;
  }
  rho[k] = S.ion_Z * re;
  rho[S.ew_nk + k] = S.ion_Z * im;
}

// The terms that do not depend on the electrons, into out[0]: the ion-ion real-space pairs
// Z^2 erfc(alpha R_IJ) / R_IJ (nearest image), the self terms -alpha / sqrt(pi) (N_e + N_ion Z^2)
// and the background -pi Q^2 / (2 Omega alpha^2), Q = N_ion Z - N_e. FP64, one block.
static __global__ void k_ewald_constant(SysParams S, double* out) {
  __shared__ double red[32];
  __shared__ double tot[1];
  const int nI = S.n_ion;
  double v = 0.0;
  for (long long p = threadIdx.x; p < (long long)nI * nI; p += blockDim.x) {
    const int a = (int)(p / nI), b = (int)(p % nI);
    if (b <= a) continue;
    double r2 = 0.0;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const double d = min_image<double>(S.ions[c * nI + a] - S.ions[c * nI + b], S.L, S.invL);
      r2 += d * d;
    }
    const double r = sqrt(r2);
    v += erfc(S.ew_alpha * r) / r;
  }
  double vv[1] = {v};
  block_sum<1, double>(vv, red, tot);
  if (threadIdx.x == 0) {
    const double Z = S.ion_Z, omega = S.L * S.L * S.L, q = nI * Z - S.n_e;
    out[0] = Z * Z * tot[0] - S.ew_alpha / sqrt(M_PI) * (S.n_e + nI * Z * Z) -
             M_PI * q * q / (2.0 * omega * S.ew_alpha * S.ew_alpha);
  }
}

// Reciprocal-space energy of every walker, added to its E_L: one block per walker, each
// thread a k vector at a time, rho_k = (ions' share) - sum_i e^{i k.r_i} summed over the
// electrons (fixed-point fractional coordinates staged in shared memory, read as broadcasts).
// Single precision sums runs of 32 electrons in float and the runs in double.
template <class TW>
__global__ void __launch_bounds__(kEwThreads) k_ewald_recip(SysParams S, WalkParams Wk) {
  using F = EwFixed<TW>;
  using U = typename F::U;
  extern __shared__ __align__(16) char smem_ew[];
  __shared__ double red[32];
  __shared__ double tot[1];
  const int w = blockIdx.x;
  if (Wk.n_live && w >= *Wk.n_live) return;
  const int n_e = S.n_e, nk = S.ew_nk;
  U* fs = reinterpret_cast<U*>(smem_ew);   // [3][n_e]
  const double* P = Wk.pos + (size_t)w * 3 * n_e;
  for (int i = threadIdx.x; i < 3 * n_e; i += blockDim.x) fs[i] = F::frac(P[i], S.invL);
  __syncthreads();
  double e = 0.0;
  for (int k = threadIdx.x; k < nk; k += blockDim.x) {
    const int4 n = S.ew_n[k];
    const U ax = (U)(long long)n.x, ay = (U)(long long)n.y, az = (U)(long long)n.z;
    double re = 0.0, im = 0.0;
    for (int i0 = 0; i0 < n_e; i0 += 32) {
      const int i1 = min(i0 + 32, n_e);
      TW cr = TW(0), ci = TW(0);
#pragma unroll 4
      for (int i = i0; i < i1; ++i) {
        const U p = ax * fs[i] + ay * fs[n_e + i] + az * fs[2 * n_e + i];
        TW s, c;
        F::sincos_turn(p, s, c);
        cr += c;
        ci += s;
      }
      re += (double)cr;
      im += (double)ci;
    }
    const double dr = S.ew_rho_ion[k] - re, di = S.ew_rho_ion[nk + k] - im;
    e += S.ew_ck[k] * (dr * dr + di * di);
  }
  double ev[1] = {e};
  block_sum<1, double>(ev, red, tot);
  if (threadIdx.x == 0) Wk.e_loc[w] += tot[0];
}

inline size_t ewald_smem_bytes(int n_e, size_t tw) { return 3 * (size_t)n_e * (tw == 4 ? 4 : 8); }

}  // namespace qmcgb
