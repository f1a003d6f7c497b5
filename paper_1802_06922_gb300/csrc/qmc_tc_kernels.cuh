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
constexpr int kTcKChunk = 32;                   // K elements of Binv0 staged per pass (tf32)
constexpr int kTcNChunk = 64;                   // columns of the update per accumulator
constexpr int kTcCols = 128;                    // TMEM columns per block: two accumulators

// Padded window width (a multiple of 16) for a window capacity kc.
__host__ __device__ inline int flush_tc_mpad(int kc) { return (kc + 15) & ~15; }

constexpr int kTcStageLd = kTcNChunk + 4;       // row stride (floats) of the epilogue tile

// Dynamic shared memory of k_flush_tc for a window capacity kc. The first region holds
// the Binv0 chunk during the first product and, once that is complete, the Z tile and the
// two U^T buffers of the second; the last region is the epilogue's staging tile (-P of one
// 64-column chunk, rows padded to kTcStageLd floats).
__host__ __device__ inline size_t flush_tc_smem_bytes(int kc) {
  const size_t mx = flush_tc_mpad(kc);
  const size_t a1 = 2 * (size_t)kTcRows * kTcKChunk * 4;                       // hi + lo
  const size_t zu = 2 * (size_t)kTcRows * mx * 4 + 2 * 2 * (size_t)kTcNChunk * mx * 4;
  size_t b = a1 > zu ? a1 : zu;
  b += 2 * mx * kTcKChunk * 4;                  // Phi chunk, hi + lo
  b += (size_t)kc * kc * 4 + (size_t)kc * 4 + 64;
  b = (b + 15) & ~(size_t)15;
  b += (size_t)kTcRows * kTcStageLd * 4;        // epilogue staging tile
  return b;
}

// Stages one 16-float slice of a Binv0 row into the hi/lo TF32 tiles.
__device__ __forceinline__ void stage_split16(const float (&x)[16], float* hi, float* lo, int r,
                                              int k, int kcols) {
#pragma unroll
  for (int t = 0; t < 4; ++t) {
    float4 h, l;
    split_tf32(x[4 * t], h.x, l.x);
    split_tf32(x[4 * t + 1], h.y, l.y);
    split_tf32(x[4 * t + 2], h.z, l.z);
    split_tf32(x[4 * t + 3], h.w, l.w);
    const uint32_t off = tc::tile_offset(r, k + 4 * t, kcols, 4) >> 2;
    *reinterpret_cast<float4*>(hi + off) = h;
    *reinterpret_cast<float4*>(lo + off) = l;
  }
}

// Flush of the delayed-update windows on the tensor cores (see k_flush for the
// mathematics). Block (w, y) owns rows [128 y, 128 y + 128) of walker w's inverse:
//   D  = Binv0[rows] Phi^T          (tcgen05 kind::tf32, 3 passes: 3xTF32), TMEM cols [0, mp)
//   Z  = (D - delta) C^-T            (CUDA cores, one thread per row, from TMEM)
//   P  = Z U                         (tcgen05, 3xTF32) in chunks of 64 columns, alternating
//                                    between TMEM cols [0, 64) and [64, 128)
//   Binv0[rows] -= P                 (epilogue from TMEM)
// The loads of the next Binv0 chunk are in flight while the tensor core works on the
// current one, and the epilogue's Binv0 values are loaded before its accumulator is ready,
// so each pass costs about one memory latency. KP is the padded window capacity (16, 32
// or 64). Every MMA is issued by thread 0 and completes on an mbarrier that the block
// waits for with a bounded poll; a timeout sets kErrTimeout and skips the rest of the block.
template <int KP>
__global__ void __launch_bounds__(256) k_flush_tc(SysParams S, WalkParams Wk, int spin) {
  extern __shared__ __align__(1024) char smem_t[];
  __shared__ uint64_t bar[3];                    // first product; second product, 2 buffers
  __shared__ uint32_t tbase;
  const int w = blockIdx.x;
  if (Wk.n_live && w >= *Wk.n_live) return;            // empty DMC slot
  const int m = Wk.win_m[w];
  if (m == 0) return;
  const int ns = spin ? S.n_dn : S.n_up;
  const int r0 = blockIdx.y * kTcRows;
  if (r0 >= ns) return;
  const int nr = min(kTcRows, ns - r0);
  const int kc = Wk.kc, ld_v = Wk.ld_v;
  const int mp = (m + 15) & ~15;                // N of the first product, K of the second
  const int mx = flush_tc_mpad(kc);             // staged width of the Z and U^T tiles (<= KP)
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  // shared memory: region 1 (A1 during the first product; Z and U^T after it), Phi, C^-1
  const size_t a1 = 2 * (size_t)kTcRows * kTcKChunk;
  const size_t zu = 2 * (size_t)kTcRows * mx + 4 * (size_t)kTcNChunk * mx;
  float* A1h = reinterpret_cast<float*>(smem_t);
  float* A1l = A1h + kTcRows * kTcKChunk;
  float* Zh = A1h;
  float* Zl = Zh + kTcRows * mx;
  float* Ub = Zl + kTcRows * mx;                // [buffer][hi, lo][64 x mx]
  float* B1h = A1h + (a1 > zu ? a1 : zu);
  float* B1l = B1h + mx * kTcKChunk;
  float* ci = B1l + mx * kTcKChunk;
  int* wrow = reinterpret_cast<int*>(ci + kc * kc);
  float* stage = reinterpret_cast<float*>(
      (reinterpret_cast<uintptr_t>(wrow + kc) + 64 + 15) & ~uintptr_t(15));   // [128][kTcStageLd]
  const float* gphi = static_cast<const float*>(Wk.win_phi) + (size_t)w * kc * ld_v;
  const float* gu = static_cast<const float*>(Wk.win_u) + (size_t)w * kc * ld_v;
  const float* gc = static_cast<const float*>(Wk.win_cinv) + (size_t)w * kc * kc;
  float* B = binv_block<float>(S, Wk, w, spin);
  const bool vec = (ns & 3) == 0 && (reinterpret_cast<uintptr_t>(B) & 15) == 0;
  // epilogue by bulk reduce-add: every row segment of a chunk is a whole number of 16-byte
  // pieces starting on a 16-byte boundary
  const bool bulk = vec;
  for (int i = tid; i < kc * kc; i += blockDim.x) ci[i] = gc[i];
  for (int i = tid; i < m; i += blockDim.x) wrow[i] = Wk.win_row[(size_t)w * kc + i];
  if (warp == 0) {
    tc::tmem_alloc(&tbase, kTcCols);
    tc::tmem_relinquish();
  }
  if (tid == 0) {
    for (int b = 0; b < 3; ++b) tc::mbar_init(&bar[b], 1);
    tc::fence_mbar_init();
  }
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  const uint32_t tmem = tbase;
  bool ok = true;
  // ---------------------------------------------------------------- D = Binv0 Phi^T
  // thread -> row lr of the tile, 16 consecutive columns lc.. of each 32-wide K chunk
  const int lr = tid >> 1, lc = (tid & 1) * 16;
  const int kc1 = kTcKChunk * 4 / 16;           // 16-byte K columns per chunk
  const float* brow = B + (size_t)(r0 + lr) * ns;
  float xa[16];
  constexpr int kPhiPer = KP * kTcKChunk / 256;  // Phi elements per thread and chunk
  float xp[kPhiPer];
  auto load_chunk = [&](int k0) {
    const int j = k0 + lc;
    if (vec) {
#pragma unroll
      for (int t = 0; t < 4; ++t) {
        float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
        if (lr < nr && j + 4 * t < ns) v = *reinterpret_cast<const float4*>(brow + j + 4 * t);
        xa[4 * t] = v.x; xa[4 * t + 1] = v.y; xa[4 * t + 2] = v.z; xa[4 * t + 3] = v.w;
      }
    } else {
#pragma unroll
      for (int t = 0; t < 16; ++t) xa[t] = (lr < nr && j + t < ns) ? brow[j + t] : 0.f;
    }
#pragma unroll
    for (int q = 0; q < kPhiPer; ++q) {
      const int i = tid + 256 * q, l = i / kTcKChunk, jj = k0 + i % kTcKChunk;
      xp[q] = (l < m && jj < ns) ? gphi[(size_t)l * ld_v + jj] : 0.f;
    }
  };
  const uint32_t id1 = tc::instr_desc(tc::kFmtTF32, kTcRows, mp);
  load_chunk(0);
  uint32_t ph1 = 0;
  for (int k0 = 0; k0 < ns; k0 += kTcKChunk) {
    if (k0 > 0) {                               // the previous chunk's MMAs read A1 and B1
      ok = tc::mbar_wait(&bar[0], ph1, kTcWaitPolls) && ok;
      ph1 ^= 1u;
    }
    stage_split16(xa, A1h, A1l, lr, lc, kc1);
#pragma unroll
    for (int q = 0; q < kPhiPer; ++q) {
      const int i = tid + 256 * q, l = i / kTcKChunk, k = i % kTcKChunk;
      if (l < mx) {
        float hi, lo;
        split_tf32(xp[q], hi, lo);
        const uint32_t off = tc::tile_offset(l, k, kc1, 4) >> 2;
        B1h[off] = hi;
        B1l[off] = lo;
      }
    }
    tc::fence_async_smem();
    ok = __syncthreads_and(ok);
    if (!ok) break;
    if (k0 + kTcKChunk < ns) load_chunk(k0 + kTcKChunk);
    if (tid == 0) {
      tc::fence_after();
#pragma unroll
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
      tc::mma_commit(&bar[0]);
    }
  }
  if (ok) ok = tc::mbar_wait(&bar[0], ph1, kTcWaitPolls);
  ok = __syncthreads_and(ok);
  tc::fence_after();
  // ---------------------------------------------------------------- Z = (D - delta) C^-T
  const int kz = mx * 4 / 16;                   // 16-byte K columns of the Z and U^T tiles
  const int n_chunks = (ns + kTcNChunk - 1) / kTcNChunk;
  auto stage_u = [&](int c, int t0, int nt) {   // U^T chunk c into buffer c & 1
    float* uh = Ub + (size_t)(c & 1) * 2 * kTcNChunk * mx;
    float* ul = uh + kTcNChunk * mx;
    const int j0 = c * kTcNChunk;
    for (int i = t0; i < kTcNChunk * mx; i += nt) {
      const int l = i / kTcNChunk, jj = i % kTcNChunk, j = j0 + jj;
      const float x = (l < m && j < ns) ? gu[(size_t)l * ld_v + j] : 0.f;
      float hi, lo;
      split_tf32(x, hi, lo);
      const uint32_t off = tc::tile_offset(jj, l, kz, 4) >> 2;
      uh[off] = hi;
      ul[off] = lo;
    }
  };
  // U^T element i of chunk c (tile row jj = i mod 64, window row l = i / 64): its global value,
  // and its hi/lo store into buffer c & 1. Loads are issued as a batch into registers one
  // phase ahead of the stores, so their latency overlaps the MMA waits.
  auto u_elem = [&](int c, int i) -> float {
    const int l = i / kTcNChunk, j = c * kTcNChunk + i % kTcNChunk;
    return (i < kTcNChunk * mx && l < m && j < ns) ? gu[(size_t)l * ld_v + j] : 0.f;
  };
  auto u_store = [&](int c, int i, float x) {
    if (i >= kTcNChunk * mx) return;
    float* uh = Ub + (size_t)(c & 1) * 2 * kTcNChunk * mx;
    float hi, lo;
    split_tf32(x, hi, lo);
    const uint32_t off = tc::tile_offset(i % kTcNChunk, i / kTcNChunk, kz, 4) >> 2;
    uh[off] = hi;
    uh[kTcNChunk * mx + off] = lo;
  };
  constexpr int kUPer = KP * kTcNChunk / 256;   // U^T elements per thread when 256 threads stage
  if (ok) {
    if (warp < 4) {
      const int n = warp * 32 + lane;           // TMEM lane = row in the tile
      float d[KP];
#pragma unroll
      for (int c = 0; c < KP; c += 16) {
        if (c < mp) {
          float v[16];
          tc::tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + c, v);
#pragma unroll
          for (int q = 0; q < 16; ++q) d[c + q] = v[q];
        } else {
#pragma unroll
          for (int q = 0; q < 16; ++q) d[c + q] = 0.f;
        }
      }
#pragma unroll
      for (int l = 0; l < KP; ++l)
        if (l < m && wrow[l] == r0 + n) d[l] -= 1.f;
      for (int l = 0; l < mx; ++l) {
        float z = 0.f;
        if (l < m) {
#pragma unroll
          for (int lp = 0; lp < KP; ++lp)
            if (lp < m) z = fmaf(ci[l * kc + lp], d[lp], z);
        }
        if (n >= nr) z = 0.f;
        float hi, lo;
        split_tf32(z, hi, lo);
        const uint32_t off = tc::tile_offset(n, l, kz, 4) >> 2;
        Zh[off] = hi;
        Zl[off] = lo;
      }
    } else {
      // chunks 0 and 1 by the upper four warps: all loads first, then the stores
      const int t0 = tid - 128;
      float ux0[2 * kUPer], ux1[2 * kUPer];
#pragma unroll
      for (int q = 0; q < 2 * kUPer; ++q) {
        ux0[q] = u_elem(0, t0 + 128 * q);
        ux1[q] = n_chunks > 1 ? u_elem(1, t0 + 128 * q) : 0.f;
      }
#pragma unroll
      for (int q = 0; q < 2 * kUPer; ++q) {
        u_store(0, t0 + 128 * q, ux0[q]);
        if (n_chunks > 1) u_store(1, t0 + 128 * q, ux1[q]);
      }
    }
  }
  tc::fence_async_smem();
  tc::fence_before();
  ok = __syncthreads_and(ok);
  tc::fence_after();
  // ---------------------------------------------------------------- Binv0 -= Z U
  const uint32_t id2 = tc::instr_desc(tc::kFmtTF32, kTcRows, kTcNChunk);
  auto issue2 = [&](int c) {                    // thread 0: P_c into TMEM cols (c & 1) * 64
    const float* uh = Ub + (size_t)(c & 1) * 2 * kTcNChunk * mx;
    const float* ul = uh + kTcNChunk * mx;
    const uint32_t dst = tmem + (uint32_t)((c & 1) * kTcNChunk);
    for (int s = 0; s < mp / 8; ++s) {
      const uint64_t ah = tc::smem_desc(Zh + s * 64, 128, kz * 128);
      const uint64_t al = tc::smem_desc(Zl + s * 64, 128, kz * 128);
      const uint64_t bh = tc::smem_desc(uh + s * 64, 128, kz * 128);
      const uint64_t bl = tc::smem_desc(ul + s * 64, 128, kz * 128);
      const uint32_t first = (s == 0) ? 0u : 1u;
      tc::mma_tf32(dst, ah, bh, id2, first);
      tc::mma_tf32(dst, ah, bl, id2, 1u);
      tc::mma_tf32(dst, al, bh, id2, 1u);
    }
    tc::mma_commit(&bar[1 + (c & 1)]);
  };
  if (ok && tid == 0) {
    tc::fence_after();
    issue2(0);
  }
  const int q4 = warp & 3, h2 = warp >> 2;      // lane quarter, column half of a chunk
  const int n = q4 * 32 + lane;
  float* erow = B + (size_t)(r0 + n) * ns;
  if (bulk) {
    // Binv0 += (-P): -P of each 64-column chunk is written to the staging tile (thread = row,
    // conflict-free with the padded stride) and added to global memory by one bulk
    // reduce-add per row, so the epilogue reads no Binv0 and the LSU pipe only stores the
    // tile once. The reduce-add rounds B + (-P) to nearest, exactly as B - P would be.
    for (int c = 0; c < n_chunks && ok; ++c) {
      // the U^T values of chunk c + 2, in flight while chunk c's MMAs finish
      const bool su = c + 2 < n_chunks;
      float ux[kUPer];
#pragma unroll
      for (int q = 0; q < kUPer; ++q) ux[q] = su ? u_elem(c + 2, tid + 256 * q) : 0.f;
      if (tid == 0 && c + 1 < n_chunks) {
        tc::fence_after();
        issue2(c + 1);
      }
      ok = tc::mbar_wait(&bar[1 + (c & 1)], (uint32_t)((c >> 1) & 1), kTcWaitPolls);
      // the previous chunk's reduce-adds have read the staging tile
      if (tid < kTcRows && c > 0) tc::bulk_wait_read<0>();
      ok = __syncthreads_and(ok);
      if (!ok) break;
      tc::fence_after();
#pragma unroll
      for (int g = 0; g < 2; ++g) {
        float v[16];
        tc::tmem_ld16(tmem + ((uint32_t)(q4 * 32) << 16) + (c & 1) * kTcNChunk + h2 * 32 + g * 16, v);
        float* srow = stage + (size_t)n * kTcStageLd + h2 * 32 + g * 16;
#pragma unroll
        for (int t = 0; t < 16; t += 4)
          *reinterpret_cast<float4*>(srow + t) = make_float4(-v[t], -v[t + 1], -v[t + 2], -v[t + 3]);
      }
      // U^T buffer c & 1 is free (its MMAs completed): chunk c + 2 goes there
      if (su)
#pragma unroll
        for (int q = 0; q < kUPer; ++q) u_store(c + 2, tid + 256 * q, ux[q]);
      tc::fence_async_smem();
      tc::fence_before();
      __syncthreads();
      if (tid < nr) {                            // one reduce-add per row of the tile
        const int j0 = c * kTcNChunk;
        const int cols = min(kTcNChunk, ns - j0);
        tc::bulk_s2g_add_f32(B + (size_t)(r0 + tid) * ns + j0, stage + (size_t)tid * kTcStageLd,
                             (uint32_t)cols * 4u);
        tc::bulk_commit();
      }
    }
    if (tid < kTcRows) tc::bulk_wait_all<0>();   // done before the block's shared memory goes
  }
  for (int c = 0; c < n_chunks && ok && !bulk; ++c) {
    // the other accumulator and U^T buffer were released by the previous iteration
    if (tid == 0 && c + 1 < n_chunks) {
      tc::fence_after();
      issue2(c + 1);
    }
    const int jb = c * kTcNChunk + h2 * 32;
    float bv[32];
    if (vec) {
#pragma unroll
      for (int t = 0; t < 8; ++t) {
        float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
        if (n < nr && jb + 4 * t < ns) v = *reinterpret_cast<const float4*>(erow + jb + 4 * t);
        bv[4 * t] = v.x; bv[4 * t + 1] = v.y; bv[4 * t + 2] = v.z; bv[4 * t + 3] = v.w;
      }
    } else {
#pragma unroll
      for (int t = 0; t < 32; ++t) bv[t] = (n < nr && jb + t < ns) ? erow[jb + t] : 0.f;
    }
    ok = tc::mbar_wait(&bar[1 + (c & 1)], (uint32_t)((c >> 1) & 1), kTcWaitPolls);
    ok = __syncthreads_and(ok);
    if (!ok) break;
    tc::fence_after();
#pragma unroll
    for (int g = 0; g < 2; ++g) {
      float v[16];
      tc::tmem_ld16(tmem + ((uint32_t)(q4 * 32) << 16) + (c & 1) * kTcNChunk + h2 * 32 + g * 16, v);
#pragma unroll
      for (int t = 0; t < 16; ++t) bv[16 * g + t] -= v[t];
    }
    if (n < nr) {
      if (vec) {
#pragma unroll
        for (int t = 0; t < 8; ++t)
          if (jb + 4 * t < ns)
            *reinterpret_cast<float4*>(erow + jb + 4 * t) =
                make_float4(bv[4 * t], bv[4 * t + 1], bv[4 * t + 2], bv[4 * t + 3]);
      } else {
#pragma unroll
        for (int t = 0; t < 32; ++t)
          if (jb + t < ns) erow[jb + t] = bv[t];
      }
    }
    // U^T buffer c & 1 is free (its MMAs completed): stage chunk c + 2 there
    if (c + 2 < n_chunks) stage_u(c + 2, tid, blockDim.x);
    tc::fence_async_smem();
    tc::fence_before();
    __syncthreads();
  }
  if (!ok && tid == 0) atomicOr(Wk.err, kErrTimeout);
  tc::fence_before();
  __syncthreads();
  if (warp == 0) tc::tmem_dealloc(tmem, kTcCols);
}

// =============================================================================
// Error-free residual R = I - A X of the single-precision inverse on the tensor cores.
//
// The re-inversion of the single-precision forms is one Newton step X <- X + X R (see
// refine_inverse). R must be accurate to about 2^-24 although the sums sum_j A_ej X_jf
// run through terms up to ~10^4 times larger than their result (random plane-wave
// Slater matrices have condition numbers 10^3..10^5), so FP32 or 3xTF32 products are not
// enough. Here each row of A (electron e) and each row of Binv (f; Binv[f][j] = X[j][f])
// is scaled by a power of two 2^E so that |x| < 1 and cut into S slices of b bits (RN
// splitting; slice i holds an integer times 2^(-b i), |integer| <= 2^b for the first slice
// and 2^(b-1) for the others, exact in BF16). The product of slice i of A with slice j of X
// is a sum of K products that are integers in units of 2^(-b (i+j)); the level-2 sum and
// the two level-3 sums together are bounded by K 2^(2b), and K 2^(2b) <= 2^24 lets an FP32
// accumulator sum them without rounding. Two slicings meet that bound: b = 8 with five
// slices and levels up to 6 (15 slice pairs) for K <= 256, and b = 7 with six slices and
// levels up to 7 (21 pairs) for K <= 512; both represent each scaled element to 2^-41 or
// better and drop only pairs below 2^-48. The pairs of level i+j = 2 and 3 carry the
// cancellation and get one exact accumulator each; the pairs of the higher levels
// (magnitude below 2^-2b of the first) share a third, ordinary FP32 accumulator. The
// epilogue forms R = delta - 2^(E_e+F_f) (L2 + L3 + L4+) with error-free (TwoSum) steps.
// This is an Ozaki-type splitting (Ozaki, Ogita, Oishi, Rump, "Error-free transformations
// of matrix multiplication by using fast routines of matrix multiplication"), restated
// for BF16 tcgen05 MMAs with FP32 accumulation.
// =============================================================================
constexpr int kRsRows = 128;      // M and N of the output tile
constexpr int kRsK = 32;          // BF16 K elements staged per chunk
// slices of kBits bits: their count, the highest level of the pairs taken, the largest K
template <int kBits> struct RsSlicing;
template <> struct RsSlicing<8> { static constexpr int kSlices = 5, kMaxLevel = 6, kMaxK = 256; };
template <> struct RsSlicing<7> { static constexpr int kSlices = 6, kMaxLevel = 7, kMaxK = 512; };
constexpr int kRsTile = kRsRows * kRsK;            // BF16 elements of one slice tile
constexpr int kRsMaxK = RsSlicing<7>::kMaxK;       // beyond it the FP64 re-inversion serves

__host__ __device__ inline size_t refine_tc_smem_bytes(int slices) {
  return (size_t)2 * 2 * slices * kRsTile * 2 + 2 * kRsRows * sizeof(int) + 64;
}

// Power-of-two exponent E of every row of A (operand 0: orbital values of the spin
// block's electrons) and of Binv (operand 1) with max_j |x_j| < 2^E; 0 for a zero row.
// One warp per row. rscale[(2 w + spin) * 2 ld_v + operand * ld_v + row].
template <class TW>
__global__ void __launch_bounds__(256) k_refine_scales(SysParams S, WalkParams Wk, int spin) {
  const int w = blockIdx.x, op = blockIdx.y;
  if (Wk.n_live && w >= *Wk.n_live) return;
  const int ns = spin ? S.n_dn : S.n_up;
  const int first = spin ? S.n_up : 0;
  const int ld5 = 5 * Wk.ld_v;
  const float* VG = static_cast<const float*>(Wk.vgl) + ((size_t)w * S.n_e + first) * ld5;
  const float* B = binv_block<const float>(S, Wk, w, spin);
  int* out = Wk.rscale + (size_t)(2 * w + spin) * 2 * Wk.ld_v + op * Wk.ld_v;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
  for (int r = warp; r < ns; r += nwarp) {
    const float* row = op == 0 ? VG + (size_t)r * ld5 : B + (size_t)r * ns;
    float mx = 0.f;
    for (int j = lane; j < ns; j += 32) mx = fmaxf(mx, fabsf(row[j]));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if (lane == 0) {
      int ex = 0;
      if (mx > 0.f && isfinite(mx)) frexpf(mx, &ex);   // mx = m 2^ex, m in [0.5, 1)
      out[r] = max(-60, min(60, ex));               // 2^(E_e + F_f) stays a normal float
    }
  }
}

__device__ __forceinline__ float pow2f(int e) { return __int_as_float((127 + e) << 23); }

__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  const float z = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, z)), __fsub_rn(b, z));
}

// Splits 16 consecutive K elements of one row into the BF16 slice tiles of kBits bits.
template <int kBits>
__device__ __forceinline__ void stage_slices16(const float (&x)[16], float inv_scale,
                                               __nv_bfloat16* tiles, int r, int k) {
  constexpr int kRsSlices = RsSlicing<kBits>::kSlices, kRsBits = kBits;
#pragma unroll
  for (int g = 0; g < 2; ++g) {
    float rem[8];
#pragma unroll
    for (int t = 0; t < 8; ++t) rem[t] = x[8 * g + t] * inv_scale;   // exact: power of two
    const uint32_t off = tc::tile_offset(r, k + 8 * g, kRsK * 2 / 16, 2) >> 1;
#pragma unroll
    for (int i = 1; i <= kRsSlices; ++i) {
      uint32_t pk[4];
#pragma unroll
      for (int t = 0; t < 8; t += 2) {
        float q2[2];
#pragma unroll
        for (int u = 0; u < 2; ++u) {
          const float tt = rem[t + u] * float(1 << kRsBits);
          const float q = rintf(tt);
          rem[t + u] = tt - q;                                        // exact, |rem| <= 1/2
          q2[u] = q * pow2f(-kRsBits * i);                            // exact
        }
        const __nv_bfloat162 h = __floats2bfloat162_rn(q2[0], q2[1]); // exact: <= 8 bits
        pk[t / 2] = *reinterpret_cast<const uint32_t*>(&h);
      }
      *reinterpret_cast<uint4*>(tiles + (size_t)(i - 1) * kRsTile + off) =
          make_uint4(pk[0], pk[1], pk[2], pk[3]);
    }
  }
}

// R[e][f] = delta_ef - sum_j A[e][j] X[j][f] for the 128 x 128 tile (blockIdx.y) of walker
// w's spin block, stored transposed (Rg[f][e]) in the first N_s^2 floats of the walker's
// FP64 work area (read by k_refine_update_tc), with max |R| into refine_max[w]. Chunks of 32 K elements are loaded into registers one chunk ahead,
// split into BF16 slices in one of two shared-memory stages, and multiplied (one thread
// issues the 15 or 21 slice-pair products per 16-wide K step) while the next chunk is split.
template <int kBits>
__global__ void __launch_bounds__(256, 1) k_refine_residual_tc(SysParams S, WalkParams Wk, int spin) {
  constexpr int kRsSlices = RsSlicing<kBits>::kSlices, kRsMaxLevel = RsSlicing<kBits>::kMaxLevel;
  extern __shared__ __align__(1024) char smem_rt[];
  __shared__ uint64_t bar[2];
  __shared__ uint32_t tbase;
  const int w = blockIdx.x;
  if (Wk.n_live && w >= *Wk.n_live) return;
  const int ns = spin ? S.n_dn : S.n_up;
  const int first = spin ? S.n_up : 0;
  const int nt = (ns + kRsRows - 1) / kRsRows;
  const int e0 = (blockIdx.y / nt) * kRsRows, f0 = (blockIdx.y % nt) * kRsRows;
  const int ld5 = 5 * Wk.ld_v;
  const float* VG = static_cast<const float*>(Wk.vgl) + ((size_t)w * S.n_e + first) * ld5;
  const float* B = binv_block<const float>(S, Wk, w, spin);
  float* Rg = reinterpret_cast<float*>(Wk.scratch64 + (size_t)(2 * w + spin) * Wk.ld_v * Wk.ld_v);
  const int* sc = Wk.rscale + (size_t)(2 * w + spin) * 2 * Wk.ld_v;
  __nv_bfloat16* tiles = reinterpret_cast<__nv_bfloat16*>(smem_rt);   // [stage][operand][slice]
  int* escA = reinterpret_cast<int*>(tiles + (size_t)2 * 2 * kRsSlices * kRsTile);
  int* escB = escA + kRsRows;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  for (int i = tid; i < kRsRows; i += blockDim.x) {
    escA[i] = (e0 + i < ns) ? sc[e0 + i] : 0;
    escB[i] = (f0 + i < ns) ? sc[Wk.ld_v + f0 + i] : 0;
  }
  if (warp == 0) {
    tc::tmem_alloc(&tbase, 512);
    tc::tmem_relinquish();
  }
  if (tid == 0) {
    tc::mbar_init(&bar[0], 1);
    tc::mbar_init(&bar[1], 1);
    tc::fence_mbar_init();
  }
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  const uint32_t tmem = tbase;
  // thread -> row lr of both operand tiles, 16 consecutive K elements lk..
  const int lr = tid >> 1, lk = (tid & 1) * 16;
  const float* arow = VG + (size_t)(e0 + lr) * ld5;
  const float* brow = B + (size_t)(f0 + lr) * ns;
  const bool a_ok = e0 + lr < ns, b_ok = f0 + lr < ns;
  const bool bvec = (ns & 3) == 0 && (reinterpret_cast<uintptr_t>(B) & 15) == 0;
  const bool avec = (ns & 3) == 0 && (reinterpret_cast<uintptr_t>(VG) & 15) == 0 && (ld5 & 3) == 0;
  const float inv_a = pow2f(-escA[lr]), inv_b = pow2f(-escB[lr]);
  float xa[16], xb[16];
  auto load_row = [&](const float* row, bool ok, bool vec, int j, float (&x)[16]) {
    if (vec) {
#pragma unroll
      for (int t = 0; t < 4; ++t) {
        float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
        if (ok && j + 4 * t < ns) v = *reinterpret_cast<const float4*>(row + j + 4 * t);
        x[4 * t] = v.x; x[4 * t + 1] = v.y; x[4 * t + 2] = v.z; x[4 * t + 3] = v.w;
      }
    } else {
#pragma unroll
      for (int t = 0; t < 16; ++t) x[t] = (ok && j + t < ns) ? row[j + t] : 0.f;
    }
  };
  const int nch = (ns + kRsK - 1) / kRsK;
  const uint32_t idesc = tc::instr_desc(tc::kFmtBF16, kRsRows, kRsRows);
  const int kcols = kRsK * 2 / 16;                   // 16-byte K columns per slice tile
  bool ok = true;
  load_row(arow, a_ok, avec, lk, xa);
  load_row(brow, b_ok, bvec, lk, xb);
  for (int c = 0; c < nch; ++c) {
    const int st = c & 1;
    if (c >= 2) {                                    // stage st was read by chunk c - 2
      ok = tc::mbar_wait(&bar[st], (uint32_t)(((c - 2) >> 1) & 1), kTcWaitPolls) && ok;
    }
    __nv_bfloat16* ta = tiles + (size_t)(st * 2 + 0) * kRsSlices * kRsTile;
    __nv_bfloat16* tb = tiles + (size_t)(st * 2 + 1) * kRsSlices * kRsTile;
    stage_slices16<kBits>(xa, inv_a, ta, lr, lk);
    stage_slices16<kBits>(xb, inv_b, tb, lr, lk);
    tc::fence_async_smem();
    ok = __syncthreads_and(ok);
    if (!ok) break;
    if (c + 1 < nch) {
      load_row(arow, a_ok, avec, (c + 1) * kRsK + lk, xa);
      load_row(brow, b_ok, bvec, (c + 1) * kRsK + lk, xb);
    }
    if (tid == 0) {
      tc::fence_after();
#pragma unroll 1
      for (int i = 1; i <= kRsSlices; ++i)
#pragma unroll 1
        for (int j = 1; i + j <= kRsMaxLevel; ++j) {
          const int lev = i + j;
          const int acc = lev == 2 ? 0 : (lev == 3 ? 1 : 2);
          // the first product into each accumulator, pairs (1,1), (1,2), (1,3), overwrites it
          const bool first_pair = (i == 1) && (j == acc + 1);
#pragma unroll
          for (int ks = 0; ks < kRsK / 16; ++ks) {
            // a 16-wide BF16 K step spans two 16-byte core-matrix columns (256 bytes)
            const uint64_t da = tc::smem_desc(ta + (size_t)(i - 1) * kRsTile + ks * 128, 128, kcols * 128);
            const uint64_t db = tc::smem_desc(tb + (size_t)(j - 1) * kRsTile + ks * 128, 128, kcols * 128);
            const uint32_t accum = (c == 0 && ks == 0 && first_pair) ? 0u : 1u;
            tc::mma_f16(tmem + (uint32_t)(acc * kRsRows), da, db, idesc, accum);
          }
        }
      tc::mma_commit(&bar[st]);
    }
  }
  if (ok) {
    const int cl = nch - 1;                          // the last commit covers every MMA
    ok = tc::mbar_wait(&bar[cl & 1], (uint32_t)((cl >> 1) & 1), kTcWaitPolls);
  }
  ok = __syncthreads_and(ok);
  tc::fence_after();
  float rmax = 0.f;
  if (ok) {
    const int q4 = warp & 3, h2 = warp >> 2;
    const int r = q4 * 32 + lane, e = e0 + r;
    const int ea = escA[r];
#pragma unroll 1
    for (int g = 0; g < kRsRows / 2; g += 16) {
      const int cb = h2 * (kRsRows / 2) + g;        // first column of this group in the tile
      float v0[16], v1[16], v2[16];
      const uint32_t ta = tmem + ((uint32_t)(q4 * 32) << 16) + cb;
      tc::tmem_ld16(ta, v0);
      tc::tmem_ld16(ta + kRsRows, v1);
      tc::tmem_ld16(ta + 2 * kRsRows, v2);
      float out[16];
#pragma unroll
      for (int t = 0; t < 16; ++t) {
        const int f = f0 + cb + t;
        const float sc2 = pow2f(ea + escB[cb + t]);
        float hi, lo, er;
        two_sum(e == f ? 1.f : 0.f, -(sc2 * v0[t]), hi, lo);
        two_sum(hi, -(sc2 * v1[t]), hi, er);
        lo = __fadd_rn(lo, er);
        two_sum(hi, -(sc2 * v2[t]), hi, er);
        lo = __fadd_rn(lo, er);
        out[t] = __fadd_rn(hi, lo);
      }
      if (e < ns) {
        // stored transposed, Rg[f][e] = R[e][f]: lanes hold consecutive e (coalesced), and
        // row e of R^T is contiguous for the update X <- X + X R
#pragma unroll
        for (int t = 0; t < 16; ++t)
          if (f0 + cb + t < ns) {
            rmax = fmaxf(rmax, isfinite(out[t]) ? fabsf(out[t]) : INFINITY);
            Rg[(size_t)(f0 + cb + t) * ns + e] = out[t];
          }
      }
    }
  }
  if (!ok) {
    rmax = INFINITY;                                 // falls back to the FP64 re-inversion
    if (tid == 0) atomicOr(Wk.err, kErrTimeout);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) rmax = fmaxf(rmax, __shfl_xor_sync(0xffffffffu, rmax, o));
  if (lane == 0) atomicMax(reinterpret_cast<int*>(Wk.refine_max + 2 * w + spin), __float_as_int(rmax));
  tc::fence_before();
  __syncthreads();
  if (warp == 0) tc::tmem_dealloc(tmem, 512);
}

// =============================================================================
// X <- X + X R of the Newton step on the tensor cores: with Binv = X^T the update reads
// Bn[e][j] = Binv[e][j] + sum_f R^T[e][f] Binv[f][j], a product of two N_s x N_s matrices per
// walker and spin. |R| <= 10^-2 (walkers above take the FP64 re-inversion), so 3xTF32
// operands (error ~2^-22 |R| |X|) keep the result at FP32 storage accuracy. Block
// (w, y) computes the 128 x 128 tile (e0, j0) into the spin block's second inverse buffer
// (binv_alt), which the host then makes the current one. A operand: rows e of R^T (K = f contiguous, as the residual kernel stores R).
// B operand: Binv[f][j0..j0+127], staged transposed into K-major tiles (thread = column j,
// 16 consecutive f packed into float4 stores). Two shared-memory stages, loads one
// chunk ahead in registers, MMAs issued by one thread with bounded mbarrier waits.
// =============================================================================
constexpr int kUpK = 32;                         // K (f) elements per chunk
__host__ __device__ inline size_t refine_update_tc_smem_bytes() {
  return (size_t)2 * 4 * kTcRows * kUpK * 4 + 64;   // 2 stages x {A, B} x {hi, lo}
}

__global__ void __launch_bounds__(256, 1) k_refine_update_tc(SysParams S, WalkParams Wk, int spin) {
  extern __shared__ __align__(1024) char smem_u[];
  __shared__ uint64_t bar[2];
  __shared__ uint32_t tbase;
  const int w = blockIdx.x;
  if (Wk.n_live && w >= *Wk.n_live) return;
  if (!(Wk.refine_max[2 * w + spin] <= kRefineSteps)) return;   // FP64 re-inversion instead
  const int ns = spin ? S.n_dn : S.n_up;
  const int nt = (ns + kTcRows - 1) / kTcRows;
  const int e0 = (blockIdx.y / nt) * kTcRows, j0 = (blockIdx.y % nt) * kTcRows;
  const float* B = binv_block<const float>(S, Wk, w, spin);
  const float* Rt = reinterpret_cast<const float*>(Wk.scratch64 + (size_t)(2 * w + spin) * Wk.ld_v * Wk.ld_v);
  float* Bn = static_cast<float*>(Wk.binv_alt[spin]) + (size_t)w * ns * ns;
  float* tiles = reinterpret_cast<float*>(smem_u);  // [stage][Ah, Al, Bh, Bl][128 x 32]
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  if (warp == 0) {
    tc::tmem_alloc(&tbase, kTcRows);
    tc::tmem_relinquish();
  }
  if (tid == 0) {
    tc::mbar_init(&bar[0], 1);
    tc::mbar_init(&bar[1], 1);
    tc::fence_mbar_init();
  }
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  const uint32_t tmem = tbase;
  const bool vec = (ns & 3) == 0 && (reinterpret_cast<uintptr_t>(B) & 15) == 0 &&
                   (reinterpret_cast<uintptr_t>(Rt) & 15) == 0;
  // A staging: thread -> row lr (= e0 + lr), 16 consecutive f
  const int lr = tid >> 1, lk = (tid & 1) * 16;
  const float* arow = Rt + (size_t)(e0 + lr) * ns;
  const bool a_ok = e0 + lr < ns;
  // B staging: thread -> column bj (= j0 + bj), 16 consecutive f starting at bk
  const int bj = tid & 127, bk = (tid >> 7) * 16;
  const bool b_ok = j0 + bj < ns;
  float xa[16], xb[16];
  auto load = [&](int k0) {
    const int f = k0 + lk;
    if (vec) {
#pragma unroll
      for (int t = 0; t < 4; ++t) {
        float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
        if (a_ok && f + 4 * t < ns) v = *reinterpret_cast<const float4*>(arow + f + 4 * t);
        xa[4 * t] = v.x; xa[4 * t + 1] = v.y; xa[4 * t + 2] = v.z; xa[4 * t + 3] = v.w;
      }
    } else {
#pragma unroll
      for (int t = 0; t < 16; ++t) xa[t] = (a_ok && f + t < ns) ? arow[f + t] : 0.f;
    }
#pragma unroll
    for (int t = 0; t < 16; ++t) {
      const int fb = k0 + bk + t;
      xb[t] = (b_ok && fb < ns) ? B[(size_t)fb * ns + j0 + bj] : 0.f;
    }
  };
  const int nch = (ns + kUpK - 1) / kUpK;
  const int kc1 = kUpK * 4 / 16;
  const uint32_t idesc = tc::instr_desc(tc::kFmtTF32, kTcRows, kTcRows);
  bool ok = true;
  load(0);
  for (int c = 0; c < nch; ++c) {
    const int st = c & 1;
    if (c >= 2) ok = tc::mbar_wait(&bar[st], (uint32_t)(((c - 2) >> 1) & 1), kTcWaitPolls) && ok;
    float* ah = tiles + (size_t)st * 4 * kTcRows * kUpK;
    float* al = ah + kTcRows * kUpK;
    float* bh = al + kTcRows * kUpK;
    float* bl = bh + kTcRows * kUpK;
    stage_split16(xa, ah, al, lr, lk, kc1);
    stage_split16(xb, bh, bl, bj, bk, kc1);
    tc::fence_async_smem();
    ok = __syncthreads_and(ok);
    if (!ok) break;
    if (c + 1 < nch) load((c + 1) * kUpK);
    if (tid == 0) {
      tc::fence_after();
#pragma unroll
      for (int s = 0; s < kUpK / 8; ++s) {
        const uint64_t dah = tc::smem_desc(ah + s * 64, 128, kc1 * 128);
        const uint64_t dal = tc::smem_desc(al + s * 64, 128, kc1 * 128);
        const uint64_t dbh = tc::smem_desc(bh + s * 64, 128, kc1 * 128);
        const uint64_t dbl = tc::smem_desc(bl + s * 64, 128, kc1 * 128);
        tc::mma_tf32(tmem, dah, dbh, idesc, (c == 0 && s == 0) ? 0u : 1u);
        tc::mma_tf32(tmem, dah, dbl, idesc, 1u);
        tc::mma_tf32(tmem, dal, dbh, idesc, 1u);
      }
      tc::mma_commit(&bar[st]);
    }
  }
  if (ok) {
    const int cl = nch - 1;
    ok = tc::mbar_wait(&bar[cl & 1], (uint32_t)((cl >> 1) & 1), kTcWaitPolls);
  }
  ok = __syncthreads_and(ok);
  tc::fence_after();
  if (ok) {
    const int q4 = warp & 3, h2 = warp >> 2;
    const int e = e0 + q4 * 32 + lane;
#pragma unroll 1
    for (int g = 0; g < kTcRows / 2; g += 16) {
      const int jb = j0 + h2 * (kTcRows / 2) + g;
      float v[16];
      tc::tmem_ld16(tmem + ((uint32_t)(q4 * 32) << 16) + h2 * (kTcRows / 2) + g, v);
      if (e < ns) {
        const float* src = B + (size_t)e * ns + jb;
        float* dst = Bn + (size_t)e * ns + jb;
        if (vec && jb + 16 <= ns) {
#pragma unroll
          for (int t = 0; t < 16; t += 4) {
            const float4 b4 = *reinterpret_cast<const float4*>(src + t);
            *reinterpret_cast<float4*>(dst + t) =
                make_float4(b4.x + v[t], b4.y + v[t + 1], b4.z + v[t + 2], b4.w + v[t + 3]);
          }
        } else {
#pragma unroll
          for (int t = 0; t < 16; ++t)
            if (jb + t < ns) dst[t] = src[t] + v[t];
        }
      }
    }
  } else if (tid == 0) {
    atomicOr(Wk.err, kErrTimeout);
  }
  tc::fence_before();
  __syncthreads();
  if (warp == 0) tc::tmem_dealloc(tmem, kTcRows);
}

}  // namespace qmcgb
