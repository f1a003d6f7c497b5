// Tensor-core (tcgen05) kernels of the single-precision forms.
#pragma once
#include "qmc_kernels.cuh"
#include "tc_sm100.cuh"

namespace qmcgb {

// Split a float into its nearest TF32 value and the remainder (|lo| <= 2^-12 |x|, exact in
// FP32); the tensor core reads both as TF32, losing at most one bit of lo. The three
// products hi*hi + hi*lo + lo*hi then reproduce a single-precision product to about
// 2^-23 relative ("3xTF32").
__device__ __forceinline__ void split_tf32(float x, float& hi, float& lo) {
  uint32_t h;
  asm("cvt.rna.tf32.f32 %0, %1;\n" : "=r"(h) : "f"(x));
  hi = __uint_as_float(h);
  lo = x - hi;
}

constexpr long long kTcWaitPolls = 20000000;   // bounded mbarrier wait (polls)
constexpr int kTcRows = 128;                    // M of every MMA: one TMEM lane per row
constexpr int kTcKChunk = 32;                   // K elements staged per pass (tf32)
constexpr int kTcNChunk = 128;                  // columns of the update per pass

// Padded window width (a multiple of 16) for a window capacity kc.
__host__ __device__ inline int flush_tc_mpad(int kc) { return (kc + 15) & ~15; }

// Dynamic shared memory of k_flush_tc for a window capacity kc.
__host__ __device__ inline size_t flush_tc_smem_bytes(int kc) {
  const size_t mx = flush_tc_mpad(kc);
  size_t b = 0;
  b += 2 * (size_t)kTcRows * kTcKChunk * 4;     // Binv0 rows chunk, hi + lo
  b += 2 * mx * kTcKChunk * 4;                  // Phi chunk, hi + lo
  b += 2 * (size_t)kTcRows * mx * 4;            // Z, hi + lo
  b += 2 * (size_t)kTcNChunk * mx * 4;          // U^T chunk, hi + lo
  b += (size_t)kc * kc * 4 + (size_t)kc * 4 + 64;
  return b;
}

// Flush of the delayed-update windows on the tensor cores (see k_flush for the
// mathematics). Block (w, y) owns rows [128 y, 128 y + 128) of walker w's inverse:
//   D  = Binv0[rows] Phi^T          (tcgen05 kind::tf32, 3 passes: 3xTF32), TMEM cols [0, mp)
//   Z  = (D - delta) C^-T            (CUDA cores, one thread per row, from TMEM)
//   P  = Z U                         (tcgen05, 3xTF32) in chunks of 128 columns, TMEM [128, 256)
//   Binv0[rows] -= P                 (epilogue from TMEM)
// Every MMA is issued by thread 0 and completes on an mbarrier that the block waits for
// with a bounded poll; a timeout sets kErrTimeout and skips the rest of the block.
__global__ void __launch_bounds__(256) k_flush_tc(SysParams S, WalkParams Wk, int spin) {
  extern __shared__ __align__(1024) char smem_t[];
  __shared__ uint64_t bar;
  __shared__ uint32_t tbase;
  const int w = blockIdx.x;
  const int m = Wk.win_m[w];
  if (m == 0) return;
  const int ns = spin ? S.n_dn : S.n_up;
  const int r0 = blockIdx.y * kTcRows;
  if (r0 >= ns) return;
  const int nr = min(kTcRows, ns - r0);
  const int kc = Wk.kc, ld_v = Wk.ld_v;
  const int mp = (m + 15) & ~15;                // N of the first product, K of the second
  const int mx = flush_tc_mpad(kc);             // staged width of the Z and U^T tiles
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  float* A1h = reinterpret_cast<float*>(smem_t);
  float* A1l = A1h + kTcRows * kTcKChunk;
  float* B1h = A1l + kTcRows * kTcKChunk;
  float* B1l = B1h + mx * kTcKChunk;
  float* Zh = B1l + mx * kTcKChunk;
  float* Zl = Zh + kTcRows * mx;
  float* Uh = Zl + kTcRows * mx;
  float* Ul = Uh + kTcNChunk * mx;
  float* ci = Ul + kTcNChunk * mx;
  int* wrow = reinterpret_cast<int*>(ci + kc * kc);
  const float* gphi = static_cast<const float*>(Wk.win_phi) + (size_t)w * kc * ld_v;
  const float* gu = static_cast<const float*>(Wk.win_u) + (size_t)w * kc * ld_v;
  const float* gc = static_cast<const float*>(Wk.win_cinv) + (size_t)w * kc * kc;
  float* B = static_cast<float*>(Wk.binv) + (size_t)w * (S.n_up * S.n_up + S.n_dn * S.n_dn) +
             (spin ? S.n_up * S.n_up : 0);
  for (int i = tid; i < kc * kc; i += blockDim.x) ci[i] = gc[i];
  for (int i = tid; i < m; i += blockDim.x) wrow[i] = Wk.win_row[(size_t)w * kc + i];
  if (warp == 0) {
    tc::tmem_alloc(&tbase, 256);
    tc::tmem_relinquish();
  }
  if (tid == 0) {
    tc::mbar_init(&bar, 1);
    tc::fence_mbar_init();
  }
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  const uint32_t tmem = tbase;
  uint32_t phase = 0;
  bool ok = true;
  // ---------------------------------------------------------------- D = Binv0 Phi^T
  const int kc1 = kTcKChunk * 4 / 16;                      // 16-byte K columns per chunk
  const uint32_t id1 = tc::instr_desc(tc::kFmtTF32, kTcRows, mp);
  for (int k0 = 0; k0 < ns && ok; k0 += kTcKChunk) {
    for (int i = tid; i < kTcRows * kTcKChunk; i += blockDim.x) {
      const int r = i / kTcKChunk, k = i % kTcKChunk, j = k0 + k;
      const float x = (r < nr && j < ns) ? B[(size_t)(r0 + r) * ns + j] : 0.f;
      float hi, lo;
      split_tf32(x, hi, lo);
      const uint32_t off = tc::tile_offset(r, k, kc1, 4) >> 2;
      A1h[off] = hi;
      A1l[off] = lo;
    }
    for (int i = tid; i < mp * kTcKChunk; i += blockDim.x) {
      const int l = i / kTcKChunk, k = i % kTcKChunk, j = k0 + k;
      const float x = (l < m && j < ns) ? gphi[(size_t)l * ld_v + j] : 0.f;
      float hi, lo;
      split_tf32(x, hi, lo);
      const uint32_t off = tc::tile_offset(l, k, kc1, 4) >> 2;
      B1h[off] = hi;
      B1l[off] = lo;
    }
    tc::fence_async_smem();
    __syncthreads();
    if (tid == 0) {
      tc::fence_after();
      for (int s = 0; s < kTcKChunk / 8; ++s) {
        const uint64_t ah = tc::smem_desc(A1h + s * 64, 128, kc1 * 128);
        const uint64_t al = tc::smem_desc(A1l + s * 64, 128, kc1 * 128);
        const uint64_t bh = tc::smem_desc(B1h + s * 64, 128, kc1 * 128);
        const uint64_t bl = tc::smem_desc(B1l + s * 64, 128, kc1 * 128);
        const uint32_t first = (k0 == 0 && s == 0) ? 0u : 1u;
        tc::mma_tf32(tmem, ah, bh, id1, first);
        tc::mma_tf32(tmem, ah, bl, id1, 1u);
        tc::mma_tf32(tmem, al, bh, id1, 1u);
      }
      tc::mma_commit(&bar);
    }
    ok = tc::mbar_wait(&bar, phase, kTcWaitPolls);
    phase ^= 1u;
    ok = __syncthreads_and(ok);
    tc::fence_after();
  }
  // ---------------------------------------------------------------- Z = (D - delta) C^-T
  if (ok && warp < 4) {
    const int n = warp * 32 + lane;                         // TMEM lane = row in the tile
    float d[64];
#pragma unroll
    for (int c = 0; c < 64; c += 16) {
      if (c < mp) {
        float v[16];
        tc::tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + c, v);
#pragma unroll
        for (int q = 0; q < 16; ++q) d[c + q] = v[q];
      }
    }
#pragma unroll
    for (int l = 0; l < 64; ++l)
      if (l < m && wrow[l] == r0 + n) d[l] -= 1.f;
    const int kz = mx * 4 / 16;                             // K columns of the Z tile
    for (int l = 0; l < mp; ++l) {
      float z = 0.f;
      if (l < m) {
#pragma unroll
        for (int lp = 0; lp < 64; ++lp)
          if (lp < m) z += ci[l * kc + lp] * d[lp];
      }
      if (n >= nr) z = 0.f;
      float hi, lo;
      split_tf32(z, hi, lo);
      const uint32_t off = tc::tile_offset(n, l, kz, 4) >> 2;
      Zh[off] = hi;
      Zl[off] = lo;
    }
  }
  tc::fence_async_smem();
  tc::fence_before();
  ok = __syncthreads_and(ok);
  tc::fence_after();
  // ---------------------------------------------------------------- Binv0 -= Z U
  const int kz = mx * 4 / 16;
  const uint32_t id2 = tc::instr_desc(tc::kFmtTF32, kTcRows, kTcNChunk);
  for (int j0 = 0; j0 < ns && ok; j0 += kTcNChunk) {
    for (int i = tid; i < kTcNChunk * mp; i += blockDim.x) {
      const int jj = i / mp, l = i % mp, j = j0 + jj;
      const float x = (l < m && j < ns) ? gu[(size_t)l * ld_v + j] : 0.f;
      float hi, lo;
      split_tf32(x, hi, lo);
      const uint32_t off = tc::tile_offset(jj, l, kz, 4) >> 2;
      Uh[off] = hi;
      Ul[off] = lo;
    }
    tc::fence_async_smem();
    __syncthreads();
    if (tid == 0) {
      tc::fence_after();
      for (int s = 0; s < mp / 8; ++s) {
        const uint64_t ah = tc::smem_desc(Zh + s * 64, 128, kz * 128);
        const uint64_t al = tc::smem_desc(Zl + s * 64, 128, kz * 128);
        const uint64_t bh = tc::smem_desc(Uh + s * 64, 128, kz * 128);
        const uint64_t bl = tc::smem_desc(Ul + s * 64, 128, kz * 128);
        const uint32_t first = (s == 0) ? 0u : 1u;
        tc::mma_tf32(tmem + 128, ah, bh, id2, first);
        tc::mma_tf32(tmem + 128, ah, bl, id2, 1u);
        tc::mma_tf32(tmem + 128, al, bh, id2, 1u);
      }
      tc::mma_commit(&bar);
    }
    ok = tc::mbar_wait(&bar, phase, kTcWaitPolls);
    phase ^= 1u;
    ok = __syncthreads_and(ok);
    tc::fence_after();
    if (ok) {
      const int q = warp & 3, h = warp >> 2;               // lane quarter, column half
      const int n = q * 32 + lane;
#pragma unroll
      for (int c = 0; c < kTcNChunk / 2; c += 16) {
        float v[16];
        tc::tmem_ld16(tmem + ((uint32_t)(q * 32) << 16) + 128 + h * (kTcNChunk / 2) + c, v);
        if (n < nr) {
          const int jb = j0 + h * (kTcNChunk / 2) + c;
          float* row = B + (size_t)(r0 + n) * ns;
          if ((ns & 3) == 0 && jb + 16 <= ns) {
            float4* p4 = reinterpret_cast<float4*>(row + jb);
#pragma unroll
            for (int t = 0; t < 4; ++t) {
              float4 b4 = p4[t];
              b4.x -= v[4 * t]; b4.y -= v[4 * t + 1]; b4.z -= v[4 * t + 2]; b4.w -= v[4 * t + 3];
              p4[t] = b4;
            }
          } else {
#pragma unroll
            for (int t = 0; t < 16; ++t)
              if (jb + t < ns) row[jb + t] -= v[t];
          }
        }
      }
    }
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
  }
  if (!ok && tid == 0) atomicOr(Wk.err, kErrTimeout);
  tc::fence_before();
  __syncthreads();
  if (warp == 0) tc::tmem_dealloc(tmem, 256);
}

}  // namespace qmcgb
