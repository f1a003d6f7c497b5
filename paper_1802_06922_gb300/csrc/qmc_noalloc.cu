// qmc_slater_invert_noalloc: the batched FP64 re-inversion of qmc_slater_invert with its
// FP64 work matrices taken from a fixed array compiled into the library, so the call
// itself never allocates device memory.
#include <cuda_runtime.h>

#include <cstdio>
#include <mutex>

#include "../../include/qmcgb.h"
#include "qmc_internal.h"
#include "qmc_launch.h"

namespace {

// Fixed FP64 work area: 2^21 doubles = 16 MiB. Every GPU on which the library is used
// holds it until the process exits. One n x n matrix per entry of the batch is needed.
constexpr size_t kWorkDoubles = size_t(1) << 21;
static __device__ __align__(256) double g_noalloc_work[kWorkDoubles];

// Device address of the work area per device (host code must not use the symbol itself:
// on the host it names a stand-in, not device memory). It is looked up again on every call
// whose stream is not being captured, so a context re-created after cudaDeviceReset gets
// its own address; a call under stream capture uses the address of the last uncaptured
// call on that device.
constexpr int kMaxDevices = 256;
double* g_work_addr[kMaxDevices] = {nullptr};
std::mutex g_work_mu;

qmc_status bad(qmc_status s, const char* msg) {
  return static_cast<qmc_status>(qmcgb::set_last_error(s, msg));
}

bool on_device(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

}  // namespace

extern "C" qmc_status qmc_slater_invert_noalloc(qmc_precision prec, const void* A, void* Binv,
                                                double* logdet, double* sign, int n, int batch,
                                                void* stream) {
  if (!A || !Binv) return bad(QMC_EINVAL, "qmc_slater_invert_noalloc: NULL matrix pointer");
  if (prec < QMC_FP64 || prec > QMC_FP32_BF16TAB)
    return bad(QMC_EINVAL, "qmc_slater_invert_noalloc: unknown precision");
  if (n < 1 || n > 1024) return bad(QMC_EINVAL, "qmc_slater_invert_noalloc: n must be in [1, 1024]");
  if (batch < 1) return bad(QMC_EINVAL, "qmc_slater_invert_noalloc: batch must be >= 1");
  const size_t need = (size_t)batch * (size_t)n * (size_t)n;
  if (need > kWorkDoubles) {
    char msg[256];
    snprintf(msg, sizeof msg,
             "qmc_slater_invert_noalloc: batch * n * n = %zu doubles exceeds the fixed work "
             "area of %zu doubles (16 MiB); split the batch",
             need, kWorkDoubles);
    return bad(QMC_EINVAL, msg);
  }
  if (!on_device(A) || !on_device(Binv) || (logdet && !on_device(logdet)) ||
      (sign && !on_device(sign)))
    return bad(QMC_EINVAL, "qmc_slater_invert_noalloc: every array must be device memory");
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return bad(QMC_ECUDA, cudaGetErrorString(e));
  if (dev < 0 || dev >= kMaxDevices) return bad(QMC_EINVAL, "qmc_slater_invert_noalloc: device index too large");
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  e = cudaStreamIsCapturing(static_cast<cudaStream_t>(stream), &cap);
  if (e != cudaSuccess) return bad(QMC_ECUDA, cudaGetErrorString(e));
  double* work = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_work_mu);
    if (cap == cudaStreamCaptureStatusNone || !g_work_addr[dev]) {
      if (cap != cudaStreamCaptureStatusNone)
        return bad(QMC_EINVAL, "qmc_slater_invert_noalloc: the first call on a device must "
                               "not be under stream capture");
      void* p = nullptr;
      e = cudaGetSymbolAddress(&p, g_noalloc_work);
      if (e != cudaSuccess) return bad(QMC_ECUDA, cudaGetErrorString(e));
      g_work_addr[dev] = static_cast<double*>(p);
    }
    work = g_work_addr[dev];
  }
  const qmcgb::TwLaunch& tw = prec == QMC_FP64 ? qmcgb::tw_launch_f64() : qmcgb::tw_launch_f32();
  e = tw.invert_batch(A, Binv, logdet, sign, n, batch, work, static_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) return bad(QMC_ECUDA, cudaGetErrorString(e));
  return QMC_OK;
}
