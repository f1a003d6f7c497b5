// Instantiations of the orbital-evaluation kernels per coefficient-table type.
#include "qmc_kernels.cuh"
#include "qmc_launch.h"
#include "qmc_nlpp.cuh"

namespace qmcgb {
namespace {

template <class TT, class TW>
cudaError_t vgl_current(const SysParams& S, const WalkParams& W, cudaStream_t st) {
  constexpr int V = TabVec<TT>::V;
  const long long chunks = (W.ld_v + 32 * V - 1) / (32 * V);
  const long long warps = (long long)W.n_w * S.n_e * chunks;
  const long long blocks = (warps * 32 + 255) / 256;
  k_vgl_current<TT, TW><<<(unsigned)blocks, 256, 0, st>>>(S, W);
  return cudaGetLastError();
}

template <class TT, class TW>
cudaError_t vgl_proposals(const SysParams& S, const WalkParams& W, int e0, int e1,
                          const void* prop, void* out, cudaStream_t st) {
  constexpr int V = TabVec<TT>::V;
  const int ns = e0 < S.n_up ? S.n_up : S.n_dn;
  const long long chunks = (ns + 32 * V - 1) / (32 * V);
  const long long warps = (long long)W.n_w * (e1 - e0) * chunks;
  const long long blocks = (warps * 32 + 255) / 256;
  k_vgl_proposals<TT, TW><<<(unsigned)blocks, 256, 0, st>>>(
      S, W, e0, e1, static_cast<const Prop*>(prop), static_cast<TW*>(out));
  return cudaGetLastError();
}

template <class TT, class TW>
cudaError_t sweep_drift(const SysParams& S, const WalkParams& W, uint32_t t, int e0, int e1,
                        int k, const void* draw, int reinv_period, int reinv_on_acc,
                        int ext_flush, bool fixed_node, cudaStream_t st) {
  const size_t smem = sweep_smem_bytes<TW>(S.n_e, W.ld_v, k, kThreads / 32, !ext_flush);
  auto kern = fixed_node ? k_sweep<TW, TT, true, true> : k_sweep<TW, TT, false, true>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  kern<<<W.n_w, kThreads, smem, st>>>(S, W, t, e0, e1, k, nullptr, static_cast<const Prop*>(draw),
                                      0, S.n_e, reinv_period, reinv_on_acc, ext_flush);
  return cudaGetLastError();
}

template <class TT, class TW>
cudaError_t nlpp(const SysParams& S, const WalkParams& W, uint32_t t, cudaStream_t st) {
  if (S.nl_nch == 0 || S.n_ion == 0) return cudaSuccess;
  cudaError_t e = cudaMemsetAsync(W.nl_count, 0, sizeof(int) * W.n_w, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(W.vnl, 0, sizeof(double) * W.n_w, st);
  if (e != cudaSuccess) return e;
  k_nlpp_pairs<<<W.n_w, 256, 0, st>>>(S, W, W.nl_pairs, W.nl_count, W.nl_cap);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const long long warps = (long long)W.n_w * W.nl_cap;
  k_nlpp_eval<TT, TW><<<(unsigned)((warps * 32 + 255) / 256), 256, 0, st>>>(
      S, W, W.nl_pairs, W.nl_count, W.nl_cap, t, W.nl_val);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_nlpp_sum<<<(unsigned)(((long long)W.n_w * 32 + 255) / 256), 256, 0, st>>>(
      W, W.nl_val, W.nl_count, W.nl_cap, W.vnl);
  return cudaGetLastError();
}

}  // namespace

const TtLaunch& tt_launch_f64() {
  static const TtLaunch L{TabVec<double>::V, vgl_current<double, double>,
                          vgl_proposals<double, double>, sweep_drift<double, double>,
                          nlpp<double, double>};
  return L;
}
const TtLaunch& tt_launch_f32() {
  static const TtLaunch L{TabVec<float>::V, vgl_current<float, float>, vgl_proposals<float, float>,
                          sweep_drift<float, float>, nlpp<float, float>};
  return L;
}
const TtLaunch& tt_launch_bf16() {
  static const TtLaunch L{TabVec<__nv_bfloat16>::V, vgl_current<__nv_bfloat16, float>,
                          vgl_proposals<__nv_bfloat16, float>, sweep_drift<__nv_bfloat16, float>,
                          nlpp<__nv_bfloat16, float>};
  return L;
}

}  // namespace qmcgb
