// Instantiations of the kernels that depend on the working precision.
#include "qmc_kernels.cuh"
#include "qmc_launch.h"
#include "qmc_tc_kernels.cuh"
#include "qmc_dmc.cuh"
#include "qmc_sweep_win.cuh"
#include "qmc_logdet.cuh"
#include "qmc_ewald.cuh"

namespace qmcgb {
namespace {

template <class TW>
cudaError_t reinvert(const SysParams& S, const WalkParams& W, cudaStream_t st) {
  const size_t smem = reinvert_smem_bytes(W.ld_v);
  cudaError_t e = cudaFuncSetAttribute(k_reinvert<TW>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  k_reinvert<TW><<<2 * W.n_w, kThreads, smem, st>>>(S, W);
  return cudaGetLastError();
}

template <class TW>
size_t sweep_smem(int n_e, int ld_v, int k) {
  return sweep_smem_bytes<TW>(n_e, ld_v, k, kThreads / 32);
}

template <class TW>
cudaError_t sweep(const SysParams& S, const WalkParams& W, uint32_t t, int e0, int e1, int k,
                  const void* P, const void* prop, int p_e0, int p_n, int reinv_period,
                  int reinv_on_acc, int ext_flush, bool fixed_node, cudaStream_t st) {
  const size_t smem_win = sweep_win_smem_bytes<TW>(S.n_e, W.ld_v);
  if (ext_flush && reinv_period == 0 && k <= kWinMaxK && W.kc <= kWinMaxK && e1 - e0 <= k &&
      smem_win <= kMaxDynSmem) {
    // a launch of the batched delayed update: the pair-matrix form of the sweep
    const size_t smem = smem_win;
    auto kern = fixed_node ? k_sweep_win<TW, true> : k_sweep_win<TW, false>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    kern<<<W.n_w, kWinThreads, smem, st>>>(S, W, e0, e1, static_cast<const TW*>(P),
                                           static_cast<const Prop*>(prop), p_e0, p_n);
    return cudaGetLastError();
  }
  const size_t smem = sweep_smem_bytes<TW>(S.n_e, W.ld_v, k, kThreads / 32, !ext_flush);
  auto kern = fixed_node ? k_sweep<TW, TW, true, false> : k_sweep<TW, TW, false, false>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  kern<<<W.n_w, kThreads, smem, st>>>(S, W, t, e0, e1, k, static_cast<const TW*>(P),
                                      static_cast<const Prop*>(prop), p_e0, p_n, reinv_period,
                                      reinv_on_acc, ext_flush);
  return cudaGetLastError();
}

template <class TW>
cudaError_t flush(const SysParams& S, const WalkParams& W, int spin, cudaStream_t st) {
  const int ns = spin ? S.n_dn : S.n_up;
  if constexpr (sizeof(TW) == 4) {
    // single precision: both products of the flush on the tensor cores (3xTF32)
    const size_t smem = flush_tc_smem_bytes(W.kc);
    const int mx = flush_tc_mpad(W.kc);
    auto kern = mx <= 16 ? k_flush_tc<16> : mx <= 32 ? k_flush_tc<32> : k_flush_tc<64>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const dim3 grid(W.n_w, (ns + kTcRows - 1) / kTcRows);
    kern<<<grid, kThreads, smem, st>>>(S, W, spin);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_window_reset<<<(W.n_w + 255) / 256, 256, 0, st>>>(W);
    return cudaGetLastError();
  }
  const size_t smem = flush_smem_bytes<TW>(W.ld_v, W.kc);
  cudaError_t e = cudaFuncSetAttribute(k_flush<TW>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const dim3 grid(W.n_w, (ns + kFlushRows - 1) / kFlushRows);
  k_flush<TW><<<grid, kThreads, smem, st>>>(S, W, spin);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_window_reset<<<(W.n_w + 255) / 256, 256, 0, st>>>(W);
  return cudaGetLastError();
}

template <class TW>
cudaError_t refine(const SysParams& S, const WalkParams& W, int spin, int part, cudaStream_t st) {
  const int ns = spin ? S.n_dn : S.n_up;
  if (ns == 0) return cudaSuccess;
  if constexpr (sizeof(TW) == 4) {
    if (part == 1) {
      // X <- X + X R on the tensor cores (3xTF32) into the second buffer of the spin block
      const size_t smem = refine_update_tc_smem_bytes();
      cudaError_t e = cudaFuncSetAttribute(k_refine_update_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      if (e != cudaSuccess) return e;
      const int nt = (ns + kTcRows - 1) / kTcRows;
      k_refine_update_tc<<<dim3(W.n_w, nt * nt), kThreads, smem, st>>>(S, W, spin);
      return cudaGetLastError();
    }
    if (part == 2) {
      // after the buffer swap: a second Newton step or the FP64 re-inversion of the walkers
      // whose residual was too large for one step
      const size_t smem = std::max(reinvert_smem_bytes(W.ld_v), sizeof(float) * (kTileElems + 32));
      cudaError_t e = cudaFuncSetAttribute(k_refine_fallback<TW>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      if (e != cudaSuccess) return e;
      k_refine_fallback<TW><<<W.n_w, kThreads, smem, st>>>(S, W, spin);
      return cudaGetLastError();
    }
    if (ns > kRsMaxK) {
      // beyond the exactness bound of the slice products: every walker of this spin block
      // takes the FP64 re-inversion (refine_max set to NaN makes the update skip them and
      // the fallback re-invert them)
      return cudaMemset2DAsync(W.refine_max + spin, 2 * sizeof(float), 0xFF, sizeof(float), W.n_w, st);
    }
    // error-free residual on the tensor cores (power-of-two row scales first)
    k_refine_scales<TW><<<dim3(W.n_w, 2), kThreads, 0, st>>>(S, W, spin);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    // 8-bit slices where K = N_s allows them (15 slice pairs), 7-bit ones up to K = 512
    const bool b8 = ns <= RsSlicing<8>::kMaxK;
    const size_t smem = refine_tc_smem_bytes(b8 ? RsSlicing<8>::kSlices : RsSlicing<7>::kSlices);
    auto kern = b8 ? k_refine_residual_tc<8> : k_refine_residual_tc<7>;
    e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const int nt = (ns + kRsRows - 1) / kRsRows;
    kern<<<dim3(W.n_w, nt * nt), kThreads, smem, st>>>(S, W, spin);
    return cudaGetLastError();
  } else {
    // double precision needs no refinement: FP64 Gauss-Jordan of that spin block
    return cudaErrorNotSupported;
  }
}

template <class TW>
cudaError_t logdet_anchor(const SysParams& S, const WalkParams& W, int spin, cudaStream_t st) {
  if constexpr (sizeof(TW) == 4) {
    const int ns = spin ? S.n_dn : S.n_up;
    if (ns == 0 || ns > kLdMaxN) return cudaSuccess;   // larger blocks re-invert in FP64
    const size_t smem = logdet_smem_bytes(ns);
    cudaError_t e = cudaFuncSetAttribute(k_logdet_anchor, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k_logdet_anchor<<<W.n_w, kLdThreads, smem, st>>>(S, W, spin);
    return cudaGetLastError();
  } else {
    return cudaErrorNotSupported;                       // the FP64 form needs no anchor
  }
}

template <class TW>
cudaError_t local_energy(const SysParams& S, const WalkParams& W, cudaStream_t st) {
  const size_t smem = energy_smem_bytes(S.n_e, sizeof(TW));
  cudaError_t e = cudaFuncSetAttribute(k_local_energy<TW>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  k_local_energy<TW><<<W.n_w, kEnergyThreads, smem, st>>>(S, W);
  return cudaGetLastError();
}

template <class TW>
cudaError_t invert_batch(const void* A, void* Binv, double* logdet, double* sign, int n,
                         int batch, double* work, cudaStream_t st) {
  const size_t smem = invert_batch_smem_bytes(n);
  cudaError_t e = cudaFuncSetAttribute(k_invert_batch<TW>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  k_invert_batch<TW><<<batch, kThreads, smem, st>>>(
      static_cast<const TW*>(A), static_cast<TW*>(Binv), logdet, sign, n, work);
  return cudaGetLastError();
}

cudaError_t dmc_branch(const SysParams& S, const WalkParams& W, const DmcParams& D, int parity,
                       uint32_t step, cudaStream_t st) {
  k_dmc_branch<<<1, 1024, 0, st>>>(S, W, D, parity, step);
  return cudaGetLastError();
}

template <class TW>
cudaError_t dmc_copy(const SysParams& S, const WalkParams& src, const WalkParams& dst,
                     const DmcParams& D, int parity, cudaStream_t st) {
  k_dmc_copy<TW><<<D.cap, kThreads, 0, st>>>(S, src, dst, D, parity);
  return cudaGetLastError();
}

template <class TW>
cudaError_t ewald_recip(const SysParams& S, const WalkParams& W, cudaStream_t st) {
  if (!S.ew_on || S.ew_nk == 0) return cudaSuccess;
  const size_t smem = ewald_smem_bytes(S.n_e, sizeof(TW));
  cudaError_t e = cudaFuncSetAttribute(k_ewald_recip<TW>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  k_ewald_recip<TW><<<W.n_w, kEwThreads, smem, st>>>(S, W);
  return cudaGetLastError();
}

template <class TW>
cudaError_t j3_vgl(const SysParams& S, const WalkParams& W, cudaStream_t st) {
  const size_t smem = j3_smem_bytes(S.n_e, sizeof(TW));
  cudaError_t e = cudaFuncSetAttribute(k_j3_vgl<TW>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  k_j3_vgl<TW><<<W.n_w, kJ3Threads, smem, st>>>(S, W);
  return cudaGetLastError();
}

}  // namespace

const TwLaunch& tw_launch_f64() {
  static const TwLaunch L{sizeof(double), reinvert<double>, sweep<double>, local_energy<double>,
                          sweep_smem<double>, invert_batch<double>, flush<double>,
                          refine<double>, logdet_anchor<double>, dmc_branch, dmc_copy<double>,
                          ewald_recip<double>, j3_vgl<double>};
  return L;
}
const TwLaunch& tw_launch_f32() {
  static const TwLaunch L{sizeof(float), reinvert<float>, sweep<float>, local_energy<float>,
                          sweep_smem<float>, invert_batch<float>, flush<float>, refine<float>,
                          logdet_anchor<float>, dmc_branch, dmc_copy<float>, ewald_recip<float>,
                          j3_vgl<float>};
  return L;
}

cudaError_t launch_proposals(const SysParams& S, const WalkParams& W, uint32_t t, int e0, int e1,
                             void* prop, cudaStream_t st) {
  const long long n = (long long)W.n_w * (e1 - e0);
  const int blocks = (int)((n + 255) / 256);
  k_proposals<<<blocks, 256, 0, st>>>(S, W, t, e0, e1, static_cast<Prop*>(prop));
  return cudaGetLastError();
}

cudaError_t launch_drift_draws(const SysParams& S, const WalkParams& W, uint32_t t, void* draw,
                               cudaStream_t st) {
  const long long n = (long long)W.n_w * S.n_e;
  if (n == 0) return cudaSuccess;
  k_drift_draws<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(S, W, t, static_cast<Prop*>(draw));
  return cudaGetLastError();
}

static __global__ void k_set_word(uint32_t* p, uint32_t v) { *p = v; }

cudaError_t launch_set_word(uint32_t* p, uint32_t v, cudaStream_t st) {
  k_set_word<<<1, 1, 0, st>>>(p, v);
  return cudaGetLastError();
}

cudaError_t launch_accumulate(const WalkParams& W, double* out, long long* nacc, cudaStream_t st) {
  k_accumulate<<<1, 256, 0, st>>>(W, out, nacc);
  return cudaGetLastError();
}

cudaError_t launch_ewald_setup(const SysParams& S, double* ck, double* rho, double* cst, cudaStream_t st) {
  if (S.ew_nk > 0) {
    k_ewald_kspace_setup<<<(S.ew_nk + 255) / 256, 256, 0, st>>>(S, ck, rho);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  k_ewald_constant<<<1, 256, 0, st>>>(S, cst);
  return cudaGetLastError();
}

}  // namespace qmcgb
