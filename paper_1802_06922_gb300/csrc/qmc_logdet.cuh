// Log-determinant anchor of the single-precision forms: ln|det A| of a walker's Slater
// matrix to FP64-class accuracy without FP64 arithmetic in the O(N^3) part.
//
// The single-precision forms carry ln|det A| as the FP64 running sum of the ln|R| of the
// accepted moves (Sec. "Multi-Determinant Slater-Jastrow Form": det A' = R det A). Each R is
// computed from single-precision orbital rows and inverse, so the sum drifts by about
// cond(A) 2^-24 per move. The anchor replaces it periodically by
//
//   ln|det A| = sum_k ln|U_kk| + ln|det(I + (P^T L U)^-1 P^T Delta)|
//             ~ sum_k ln|U_kk| + tr(X P^T Delta),          Delta = P A - L U,
//
// where P A = L U + Delta is an LU factorisation with partial pivoting computed in FP32 on
// the CUDA cores and X ~ A^-1 is the walker's inverse, accurate to FP32 storage right
// after the Newton re-inversion. det L = 1 and det(L U) = prod_k U_kk exactly, so the FP32
// rounding enters only through Delta, whose norm is about cond(A) 2^-24: the first-order
// term tr(X P^T Delta) carries it and the neglected second-order terms are about
// (cond(A) 2^-24)^2. Delta is known exactly: every update a <- a - l u of the elimination
// is done with error-free transformations (TwoProduct by FMA, TwoSum; Ogita, Rump and
// Oishi, "Accurate sum and dot product"), the part lost to rounding is added into a
// per-element FP32 companion, and the division l = a / u leaves the exact remainder
// fma(-l, u, a). With Binv[e][j] = X[j][e] and the rows of A never moved (logical row i of
// the factorisation lives in physical row pos[i] = electron pos[i]),
//   tr(X P^T Delta) = sum_{e,j} Binv[e][j] Lo[e][j],
// Lo[e][j] being the companion of element (e, j) when it leaves the active matrix.
//
// Blocked right-looking elimination, one 256-thread block per (walker, spin block):
//   panel   kLdNb columns of the active rows in shared memory; partial pivoting without row
//           exchanges (the pivot is the largest unused row of the column; each thread owns
//           whole panel rows, so one block barrier per column suffices);
//   U12     the pivot rows' remaining columns, forward substitution with the panel's
//           unit-lower L11, one thread per column;
//   update  the remaining rows: a <- a - L21 U12 in 4 x 4 register tiles, each a
//           compensated dot product of length kLdNb.
// The active matrix and its companions sit in the walker's FP64 work area (2 N^2 floats);
// the first panel reads the orbital values directly.
#pragma once
#include "qmc_kernels.cuh"

namespace qmcgb {

constexpr int kLdNb = 32;          // panel width
constexpr int kLdMaxN = 512;       // spin blocks up to this size (larger ones re-invert in FP64)
constexpr int kLdThreads = 256;

__host__ __device__ inline int logdet_panel_ld() { return kLdNb + 1; }
__host__ __device__ inline int logdet_u12_ld(int n) { return ((n + 3) & ~3) + 4; }

__host__ __device__ inline size_t logdet_smem_bytes(int n) {
  return sizeof(float) * ((size_t)kLdNb * logdet_u12_ld(n) + 2 * (size_t)n * logdet_panel_ld()) +
         sizeof(int) * (5 * (size_t)n + kLdNb + 32) + sizeof(float) * (size_t)(n + 16) +
         sizeof(double) * 16 + 16;
}

// a - l*u with the part lost to rounding added into lo (exact up to the rounding of lo).
__device__ __forceinline__ void ld_update(float& a, float& lo, float l, float u) {
  const float p = __fmul_rn(l, u);
  const float pe = __fmaf_rn(l, u, -p);        // l u = p + pe exactly
  const float s = __fsub_rn(a, p);             // TwoSum(a, -p) = s + e exactly
  const float z = __fsub_rn(s, a);
  const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, z)), __fsub_rn(-p, z));
  lo = __fadd_rn(lo, __fsub_rn(e, pe));        // a - l u = s + (e - pe)
  a = s;
}

// Accumulates t + tl += l*u with t + tl exact up to the rounding of tl.
__device__ __forceinline__ void ld_dot(float& t, float& tl, float l, float u) {
  const float p = __fmul_rn(l, u);
  const float pe = __fmaf_rn(l, u, -p);
  const float s = __fadd_rn(t, p);
  const float z = __fsub_rn(s, t);
  const float e = __fadd_rn(__fsub_rn(t, __fsub_rn(s, z)), __fsub_rn(p, z));
  tl = __fadd_rn(tl, __fadd_rn(e, pe));
  t = s;
}

__global__ void __launch_bounds__(kLdThreads, 2) k_logdet_anchor(SysParams S, WalkParams Wk, int spin) {
  extern __shared__ __align__(16) char smem_ld[];
  const int w = blockIdx.x;
  if (Wk.n_live && w >= *Wk.n_live) return;                    // empty DMC slot
  if (Wk.refine_fb[2 * w + spin]) return;                   // re-inverted in FP64: exact
  const int n = spin ? S.n_dn : S.n_up;
  if (n == 0 || n > kLdMaxN) return;
  const int first = spin ? S.n_up : 0;
  const int ld5 = 5 * Wk.ld_v;
  const float* VG = static_cast<const float*>(Wk.vgl) + ((size_t)w * S.n_e + first) * ld5;
  const float* B = binv_block<const float>(S, Wk, w, spin);
  float* Hi = reinterpret_cast<float*>(Wk.scratch64 + (size_t)(2 * w + spin) * Wk.ld_v * Wk.ld_v);
  float* Lo = Hi + (size_t)n * n;
  const int PL = logdet_panel_ld();
  const int ldu = logdet_u12_ld(n);
  float* U12 = reinterpret_cast<float*>(smem_ld);              // [kLdNb][ldu]
  float* Ph = U12 + (size_t)kLdNb * ldu;                       // [n][PL] panel values
  float* Pl = Ph + (size_t)n * PL;                             // [n][PL] their companions
  int* pos = reinterpret_cast<int*>(Pl + (size_t)n * PL);      // logical row -> electron
  int* npos = pos + n;                                         // next order of the rows
  int* rest = npos + n;                                        // update row i -> panel row
  int* usedf = rest + n;                                       // panel row used as pivot
  int* pivrow = usedf + n;                                     // [kLdNb] panel row of pivot j
  int* redi = pivrow + kLdNb;                                  // [2][8] warp arg-maxima
  float* pivv = reinterpret_cast<float*>(redi + 32);           // [n] U_kk
  float* redv = pivv + n;                                      // [2][8]
  double* redd = reinterpret_cast<double*>(((uintptr_t)(redv + 16) + 7) & ~(uintptr_t)7);
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  constexpr int kWarps = kLdThreads / 32;
  for (int i = tid; i < n; i += kLdThreads) pos[i] = i;
  float corr = 0.f;                                            // this thread's share of tr(X P^T Delta)
  bool singular = false;
  __syncthreads();
  for (int k0 = 0; k0 < n && !singular; k0 += kLdNb) {
    const int kb = min(kLdNb, n - k0);
    const int R = n - k0;                                      // active rows
    const bool from_a = k0 == 0;                               // the first panel reads A
    // ------------------------------------------------------------ load the panel
    for (int i = tid; i < R * kb; i += kLdThreads) {
      const int r = i / kb, c = i % kb;
      const int e = pos[k0 + r];
      const size_t g = (size_t)e * n + k0 + c;
      Ph[r * PL + c] = from_a ? VG[(size_t)e * ld5 + k0 + c] : Hi[g];
      Pl[r * PL + c] = from_a ? 0.f : Lo[g];
    }
    for (int r = tid; r < R; r += kLdThreads) usedf[r] = 0;
    __syncthreads();
    // ------------------------------------------------------------ panel factorisation
    // thread tid owns panel rows tid and tid + 256
    for (int j = 0; j < kb; ++j) {
      float best = -1.f;
      int bi = 0x7fffffff;
      for (int r = tid; r < R; r += kLdThreads) {
        if (usedf[r]) continue;
        const float v = fabsf(Ph[r * PL + j]);
        if (v > best || (v == best && r < bi)) { best = v; bi = r; }
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        const float ob = __shfl_xor_sync(0xffffffffu, best, o);
        const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
        if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
      }
      const int buf = (j & 1) * kWarps;
      if (lane == 0) { redv[buf + warp] = best; redi[buf + warp] = bi; }
      __syncthreads();
      best = redv[buf];
      bi = redi[buf];
#pragma unroll
      for (int q = 1; q < kWarps; ++q) {
        const float ob = redv[buf + q];
        const int oi = redi[buf + q];
        if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
      }
      const int piv = bi;
      const float pv = (piv < R) ? Ph[piv * PL + j] : 0.f;
      if (!(pv != 0.f) || !isfinite(pv)) { singular = true; break; }   // uniform
      if (tid == 0) { pivrow[j] = piv; pivv[k0 + j] = pv; }
      for (int r = tid; r < R; r += kLdThreads) {
        if (r == piv) { usedf[r] = 1; continue; }
        if (usedf[r]) continue;
        float* ph = Ph + r * PL;
        float* pl = Pl + r * PL;
        const float a = ph[j];
        const float l = __fdiv_rn(a, pv);
        pl[j] = __fadd_rn(pl[j], __fmaf_rn(-l, pv, a));     // exact remainder of the division
        ph[j] = l;
        const float* pr = Ph + piv * PL;
        int c = j + 1;
        for (; c + 4 <= kb; c += 4) {     // loads of a group before its stores (no aliasing stalls)
          float a[4], al[4], u[4];
#pragma unroll
          for (int q = 0; q < 4; ++q) { a[q] = ph[c + q]; al[q] = pl[c + q]; u[q] = pr[c + q]; }
#pragma unroll
          for (int q = 0; q < 4; ++q) ld_update(a[q], al[q], l, u[q]);
#pragma unroll
          for (int q = 0; q < 4; ++q) { ph[c + q] = a[q]; pl[c + q] = al[q]; }
        }
        for (; c < kb; ++c) ld_update(ph[c], pl[c], l, pr[c]);
      }
    }
    if (singular) break;
    __syncthreads();
    // every panel element is now final (L below the pivots, U in the pivot rows): its
    // companion enters the trace correction
    for (int i = tid; i < R * kb; i += kLdThreads) {
      const int r = i / kb, c = i % kb;
      corr = fmaf(B[(size_t)pos[k0 + r] * n + k0 + c], Pl[r * PL + c], corr);
    }
    // next order of the active rows: the pivots in pivot order, then the unused rows
    if (warp == 0) {
      int base = 0;
      for (int r0 = 0; r0 < R; r0 += 32) {
        const int r = r0 + lane;
        const bool un = r < R && !usedf[r];
        const unsigned m = __ballot_sync(0xffffffffu, un);
        if (un) {
          const int idx = base + __popc(m & ((1u << lane) - 1u));
          rest[idx] = r;
          npos[k0 + kb + idx] = pos[k0 + r];
        }
        base += __popc(m);
      }
      if (lane < kb) npos[k0 + lane] = pos[k0 + pivrow[lane]];
    }
    __syncthreads();
    const int nc = n - k0 - kb;                                // remaining columns
    if (nc > 0) {
      // ---------------------------------------------------------- U12 (forward substitution)
      // row j of U12 = a_j - sum_{m<j} L11[j][m] U12[m] (the updates of the unblocked
      // elimination, in the same order), one thread per column; the final rows are kept in
      // shared memory for the trailing update
      for (int c = tid; c < nc; c += kLdThreads) {
        const int col = k0 + kb + c;
        for (int j = 0; j < kb; ++j) {
          const int e = npos[k0 + j];
          float x = from_a ? VG[(size_t)e * ld5 + col] : Hi[(size_t)e * n + col];
          float xl = from_a ? 0.f : Lo[(size_t)e * n + col];
          const float* lj = Ph + pivrow[j] * PL;
#pragma unroll 4
          for (int m = 0; m < j; ++m) ld_update(x, xl, lj[m], U12[m * ldu + c]);
          U12[j * ldu + c] = x;
          corr = fmaf(B[(size_t)e * n + col], xl, corr);
        }
      }
      __syncthreads();
      // ---------------------------------------------------------- trailing update
      const int nr = R - kb;                                   // remaining rows
      // a warp covers 4 rows x 128 columns (lane: columns ct + lane + 32 b, so that every
      // global access of the warp is one contiguous 128-byte row segment); 8 warps stacked
      for (int rt = warp * 4; rt < nr; rt += kWarps * 4) {
        for (int ct = 0; ct < nc; ct += 128) {
          float t[4][4], tl[4][4];
#pragma unroll
          for (int a = 0; a < 4; ++a)
#pragma unroll
            for (int b = 0; b < 4; ++b) { t[a][b] = 0.f; tl[a][b] = 0.f; }
          int prw[4];
#pragma unroll
          for (int a = 0; a < 4; ++a) prw[a] = (rt + a < nr) ? rest[rt + a] : rest[rt];
#pragma unroll 4
          for (int m = 0; m < kb; ++m) {
            float uu[4];
#pragma unroll
            for (int b = 0; b < 4; ++b) {
              const int cc = ct + lane + 32 * b;
              uu[b] = cc < nc ? U12[m * ldu + cc] : 0.f;
            }
#pragma unroll
            for (int a = 0; a < 4; ++a) {
              const float l = Ph[prw[a] * PL + m];
#pragma unroll
              for (int b = 0; b < 4; ++b) ld_dot(t[a][b], tl[a][b], l, uu[b]);
            }
          }
#pragma unroll
          for (int a = 0; a < 4; ++a) {
            if (rt + a >= nr) continue;
            const int e = npos[k0 + kb + rt + a];
#pragma unroll
            for (int b = 0; b < 4; ++b) {
              const int cc = ct + lane + 32 * b;
              const int col = k0 + kb + cc;
              if (cc >= nc) continue;
              const size_t g = (size_t)e * n + col;
              float hi = from_a ? VG[(size_t)e * ld5 + col] : Hi[g];
              float lo = from_a ? 0.f : Lo[g];
              // hi - (t + tl): TwoSum(hi, -t) = s + es, lost part es - tl
              const float s = __fsub_rn(hi, t[a][b]);
              const float z = __fsub_rn(s, hi);
              const float es = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, z)), __fsub_rn(-t[a][b], z));
              lo = __fadd_rn(lo, __fsub_rn(es, tl[a][b]));
              Hi[g] = s;
              Lo[g] = lo;
            }
          }
        }
      }
    }
    __syncthreads();
    for (int i = tid; i < R; i += kLdThreads) pos[k0 + i] = npos[k0 + i];
    __syncthreads();
  }
  // ------------------------------------------------------------ ln|det A| and its sign
  double lsum = 0.0;
  int nneg = 0;
  if (!singular)
    for (int k = tid; k < n; k += kLdThreads) {
      const float u = pivv[k];
      lsum += log(fabs((double)u));
      nneg += u < 0.f;
    }
  double v[2] = {lsum, (double)corr};
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    v[0] += __shfl_xor_sync(0xffffffffu, v[0], o);
    v[1] += __shfl_xor_sync(0xffffffffu, v[1], o);
    nneg += __shfl_xor_sync(0xffffffffu, nneg, o);
  }
  if (lane == 0) { redd[2 * warp] = v[0]; redd[2 * warp + 1] = v[1]; redi[warp] = nneg; }
  __syncthreads();
  if (tid == 0 && !singular) {
    double ls = 0.0, cs = 0.0;
    int neg = 0;
    for (int q = 0; q < kWarps; ++q) { ls += redd[2 * q]; cs += redd[2 * q + 1]; neg += redi[q]; }
    // sign of the row order pos (logical -> electron): parity from its cycles
    int cycles = 0;
    for (int i = 0; i < n; ++i) usedf[i] = 0;
    for (int i = 0; i < n; ++i) {
      if (usedf[i]) continue;
      ++cycles;
      for (int j = i; !usedf[j]; j = pos[j]) usedf[j] = 1;
    }
    const int parity = (n - cycles + neg) & 1;
    const double ld_new = ls + cs;
    const int slot = 2 * w + spin;
    Wk.logdet_shift[slot] = (float)(ld_new - Wk.logdet[slot]);
    Wk.logdet[slot] = ld_new;
    Wk.sgn[slot] = parity ? -1.0 : 1.0;
  }
}

}  // namespace qmcgb
