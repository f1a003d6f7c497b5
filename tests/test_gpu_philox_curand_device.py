"""GPU pin of the oracle's Philox4x32-10 on the counter word that cuRAND's host generator
leaves at zero: cuRAND's device API keys a Philox4_32_10 state with the 64-bit seed and
places the 64-bit subsequence number in counter words 2 and 3 and offset / 4 in words 0
and 1; the first curand4() of a fresh state returns the four words of that counter. A
small kernel (compiled here with nvcc against the toolkit's curand_kernel.h) draws them for
counters with word 3 in {0, 1, 2, 0xFFFFFFFF} (the move draws use 0 and 1, the branching
draw uses 2), and the oracle must give the same words.
"""
import ctypes
import os
import shutil
import subprocess
import tempfile

import numpy as np
import pytest

from oracle.philox import philox4x32_10, seed_key

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

SRC = r"""
#include <cuda_runtime.h>
#include <curand_kernel.h>

__global__ void draw(unsigned long long seed, const unsigned long long* subseq,
                     const unsigned long long* offs, uint4* out, int n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  curandStatePhilox4_32_10_t st;
  curand_init(seed, subseq[i], offs[i], &st);
  out[i] = curand4(&st);
}

extern "C" int curand_first_blocks(unsigned long long seed, const unsigned long long* subseq,
                                   const unsigned long long* offs, unsigned int* out, int n) {
  unsigned long long *ds = nullptr, *doff = nullptr;
  uint4* dout = nullptr;
  cudaError_t e = cudaMalloc(&ds, n * sizeof(unsigned long long));
  if (e == cudaSuccess) e = cudaMalloc(&doff, n * sizeof(unsigned long long));
  if (e == cudaSuccess) e = cudaMalloc(&dout, n * sizeof(uint4));
  if (e == cudaSuccess) e = cudaMemcpy(ds, subseq, n * sizeof(unsigned long long), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(doff, offs, n * sizeof(unsigned long long), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) {
    draw<<<(n + 127) / 128, 128>>>(seed, ds, doff, dout, n);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemcpy(out, dout, n * sizeof(uint4), cudaMemcpyDeviceToHost);
  cudaFree(ds);
  cudaFree(doff);
  cudaFree(dout);
  return (int)e;
}
"""


@pytest.fixture(scope="module")
def curand_dev():
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not found")
    d = tempfile.mkdtemp(prefix="curand_pin_")
    src = os.path.join(d, "pin.cu")
    lib = os.path.join(d, "libcurand_pin.so")
    with open(src, "w") as f:
        f.write(SRC)
    r = subprocess.run([nvcc, "-O2", "-shared", "-Xcompiler", "-fPIC", "-gencode",
                        "arch=compute_103a,code=sm_103a", src, "-o", lib],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    L = ctypes.CDLL(lib)
    L.curand_first_blocks.argtypes = [ctypes.c_ulonglong, ctypes.c_void_p, ctypes.c_void_p,
                                      ctypes.c_void_p, ctypes.c_int]
    L.curand_first_blocks.restype = ctypes.c_int
    yield L
    shutil.rmtree(d, ignore_errors=True)


@pytest.mark.parametrize("seed", [0, 0xA4093822299F31D0, 0xFFFFFFFFFFFFFFFF])
def test_oracle_equals_curand_device_philox(curand_dev, seed):
    rng = np.random.default_rng(seed & 0xFFFF)
    w3 = np.array([0, 1, 2, 0xFFFFFFFF], dtype=np.uint64)
    n = 256
    c3 = w3[np.arange(n) % 4]
    c2 = rng.integers(0, 2 ** 32, size=n, dtype=np.uint64)
    c01 = rng.integers(0, 2 ** 62, size=n, dtype=np.uint64)
    c01[:4] = [0, 1, 0xFFFFFFFF, 0x100000000]
    sub = np.ascontiguousarray((c3 << np.uint64(32)) | c2, dtype=np.uint64)
    off = np.ascontiguousarray(c01 * np.uint64(4), dtype=np.uint64)
    out = np.zeros((n, 4), dtype=np.uint32)
    rc = curand_dev.curand_first_blocks(seed, sub.ctypes.data, off.ctypes.data, out.ctypes.data, n)
    assert rc == 0, f"CUDA error {rc}"
    ref = np.stack(philox4x32_10((c01 & np.uint64(0xFFFFFFFF), c01 >> np.uint64(32), c2, c3),
                                 seed_key(seed)), -1)
    bad = np.argwhere(out != ref)
    assert bad.size == 0, f"first mismatch at {bad[0]}: counter word 3 = {c3[bad[0][0]]:#x}"
