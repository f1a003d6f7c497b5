// qmc_measure_rates: the arithmetic and L2 rates that bound the kernels the tensor cores and
// HBM do not (the roofline denominators of the FP32 pipe work, the FP64 steps and the
// L2-resident spline tables), measured on the device in use with CUDA events. Clocks are
// left as they are.
#include <cuda_runtime.h>

#include <cstdio>

#include "../../include/qmcgb.h"
#include "qmc_launch.h"

namespace {

constexpr int kChains = 8;           // independent FMA chains per thread
constexpr int kIters = 4096;         // FMA steps per chain

template <class T>
__global__ void __launch_bounds__(256) k_fma_rate(T a, T b, T* out) {
  T x[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) x[c] = T(threadIdx.x + c) * T(1e-3);
#pragma unroll 4
  for (int i = 0; i < kIters; ++i) {
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = fma(x[c], a, b);
  }
  T s = T(0);
#pragma unroll
  for (int c = 0; c < kChains; ++c) s += x[c];
  if (s == T(12345.678)) out[blockIdx.x] = s;   // keeps the chains alive; never true here
}

__global__ void __launch_bounds__(256) k_l2_read(const float4* __restrict__ buf, size_t n4, int reps,
                                                 float* out) {
  float acc = 0.f;
  const size_t stride = (size_t)gridDim.x * blockDim.x;
  for (int r = 0; r < reps; ++r)
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n4; i += stride) {
      const float4 v = __ldcg(buf + i);              // L2, not L1
      acc += v.x + v.y + v.z + v.w;
    }
  if (acc == 12345.678f) out[blockIdx.x] = acc;
}

qmc_status bad(const char* msg) { return static_cast<qmc_status>(qmcgb::set_last_error(QMC_ECUDA, msg)); }

#define QMC_TRY(x)                                  \
  do {                                              \
    cudaError_t e_ = (x);                           \
    if (e_ != cudaSuccess) { ok = false; err = e_; } \
  } while (0)

}  // namespace

extern "C" qmc_status qmc_measure_rates(double* out) {
  if (!out) return static_cast<qmc_status>(qmcgb::set_last_error(QMC_EINVAL, "qmc_measure_rates: NULL argument"));
  int dev = 0, sms = 0;
  cudaError_t err = cudaGetDevice(&dev);
  if (err == cudaSuccess) err = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (err != cudaSuccess) return bad(cudaGetErrorString(err));
  bool ok = true;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  float* sink = nullptr;
  float4* buf = nullptr;
  const size_t l2_bytes = size_t(48) << 20;          // well inside the 129 MB L2
  QMC_TRY(cudaEventCreate(&e0));
  QMC_TRY(cudaEventCreate(&e1));
  QMC_TRY(cudaMalloc(&sink, 64 * 1024 * sizeof(double)));
  QMC_TRY(cudaMalloc(&buf, l2_bytes));
  if (ok) QMC_TRY(cudaMemset(buf, 0, l2_bytes));
  const int blocks = sms * 8;
  auto timed = [&](auto launch, int repeat) -> double {   // best of `repeat`, ms
    double best = 1e30;
    for (int r = 0; r < repeat && ok; ++r) {
      launch();
      QMC_TRY(cudaEventRecord(e0));
      launch();
      QMC_TRY(cudaEventRecord(e1));
      QMC_TRY(cudaEventSynchronize(e1));
      float ms = 0.f;
      QMC_TRY(cudaEventElapsedTime(&ms, e0, e1));
      if (ms > 0.f && ms < best) best = ms;
    }
    return best;
  };
  const double fmas = (double)blocks * 256 * kChains * kIters;
  const double t32 = timed([&] { k_fma_rate<float><<<blocks, 256>>>(0.999f, 1e-3f, sink); }, 5);
  const double t64 = timed([&] { k_fma_rate<double><<<blocks, 256>>>(0.999, 1e-3, reinterpret_cast<double*>(sink)); }, 3);
  const size_t n4 = l2_bytes / sizeof(float4);
  const int reps = 100;
  const double tl2 = timed([&] { k_l2_read<<<sms * 4, 256>>>(buf, n4, reps, sink); }, 5);
  QMC_TRY(cudaGetLastError());
  if (ok) {
    out[0] = 2.0 * fmas / (t32 * 1e-3) / 1e12;       // FP32 TFLOP/s (an FMA = 2 flops)
    out[1] = 2.0 * fmas / (t64 * 1e-3) / 1e12;       // FP64 TFLOP/s
    out[2] = (double)l2_bytes * reps / (tl2 * 1e-3) / 1e9;   // L2 read GB/s
  }
  cudaFree(buf);
  cudaFree(sink);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (!ok) return bad(cudaGetErrorString(err));
  return QMC_OK;
}
