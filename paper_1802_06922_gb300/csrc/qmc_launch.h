// Launchers of the kernels, one set per working precision (TW) and table type (TT).
#pragma once
#include <cuda_runtime.h>

#include "qmc_internal.h"

namespace qmcgb {

// Kernels that depend on the working precision only (TW = double or float).
struct TwLaunch {
  size_t tw_size;
  cudaError_t (*reinvert)(const SysParams&, const WalkParams&, cudaStream_t);
  cudaError_t (*sweep)(const SysParams&, const WalkParams&, uint32_t t, int e0, int e1, int k,
                       const void* P, const void* prop, int p_e0, int p_n, int reinv_period,
                       int reinv_on_acc, int ext_flush, bool fixed_node, cudaStream_t);
  cudaError_t (*local_energy)(const SysParams&, const WalkParams&, cudaStream_t);
  size_t (*sweep_smem)(int n_e, int ld_v, int k);
  cudaError_t (*invert_batch)(const void* A, void* Binv, double* logdet, double* sign, int n,
                              int batch, double* work, cudaStream_t);
  cudaError_t (*flush)(const SysParams&, const WalkParams&, int spin, cudaStream_t);
  // part 0: row scales + error-free residual; part 1: X <- X + X R into binv_alt[spin];
  // part 2 (after the caller has swapped binv and binv_alt of the spin block): FP64
  // fallback of the walkers whose residual was too large
  cudaError_t (*refine)(const SysParams&, const WalkParams&, int spin, int part, cudaStream_t);
  // ln|det A| of the spin block by the error-free FP32 LU (single precision only)
  cudaError_t (*logdet_anchor)(const SysParams&, const WalkParams&, int spin, cudaStream_t);
  cudaError_t (*dmc_branch)(const SysParams&, const WalkParams&, const DmcParams&, int parity,
                            uint32_t step, cudaStream_t);
  cudaError_t (*dmc_copy)(const SysParams&, const WalkParams& src, const WalkParams& dst,
                          const DmcParams&, int parity, cudaStream_t);
  // Ewald reciprocal-space energy of every walker, added to E_L
  cudaError_t (*ewald_recip)(const SysParams&, const WalkParams&, cudaStream_t);
  // three-body Jastrow gradient, Laplacian and value of every electron into W.j3vgl
  cudaError_t (*j3_vgl)(const SysParams&, const WalkParams&, cudaStream_t);
};
const TwLaunch& tw_launch_f64();
const TwLaunch& tw_launch_f32();

// Kernels that depend on the coefficient-table type.
struct TtLaunch {
  int vec;   // orbitals per 16-byte load
  cudaError_t (*vgl_current)(const SysParams&, const WalkParams&, cudaStream_t);
  cudaError_t (*vgl_proposals)(const SysParams&, const WalkParams&, int e0, int e1,
                               const void* prop, void* out, cudaStream_t);
  // drift-diffusion sweep of electrons [e0, e1) with in-kernel orbital evaluation; draw: the
  // sweep's draws from launch_drift_draws
  cudaError_t (*sweep_drift)(const SysParams&, const WalkParams&, uint32_t t, int e0, int e1,
                             int k, const void* draw, int reinv_period, int reinv_on_acc,
                             int ext_flush, bool fixed_node, cudaStream_t);
  // non-local pseudopotential energy of every walker (added to E_L), quadrature rotation t
  cudaError_t (*nlpp)(const SysParams&, const WalkParams&, uint32_t t, cudaStream_t);
};
const TtLaunch& tt_launch_f64();
const TtLaunch& tt_launch_f32();
const TtLaunch& tt_launch_bf16();

// Precision-independent kernels.
cudaError_t launch_proposals(const SysParams&, const WalkParams&, uint32_t t, int e0, int e1,
                             void* prop, cudaStream_t);
// Draws (xi, u) of every drift-diffusion move of sweep t: draw[w][e], W.n_w x S.n_e entries.
cudaError_t launch_drift_draws(const SysParams&, const WalkParams&, uint32_t t, void* draw,
                               cudaStream_t);
cudaError_t launch_accumulate(const WalkParams&, double* out, long long* nacc, cudaStream_t);
// *p = v on the stream (the sweep index of a replayed graph).
cudaError_t launch_set_word(uint32_t* p, uint32_t v, cudaStream_t);
// Ewald setup from the ions: c_k, the ions' rho_k and the constant terms (FP64).
cudaError_t launch_ewald_setup(const SysParams&, double* ck, double* rho, double* cst, cudaStream_t);

// Records the message returned by qmc_last_error on this thread; returns s.
int set_last_error(int s, const char* msg);

}  // namespace qmcgb
