// Kernels of the particle-by-particle sweep. Templated on the coefficient-table type TT
// (double, float, bf16) and the working type TW (double, or float for the mixed forms).
//
// Precision discipline of the mixed forms (TW = float): on this GPU FP64 arithmetic and
// double<->float conversions run at a small fraction of the FP32 rate, so per-element
// work stays in single precision; double is used by one thread per move (the proposal,
// ln|det| accumulation, the final sum of warp partials) and in the periodic FP64
// re-inversion.
#pragma once
#include "qmc_device.cuh"
#include "qmc_jastrow3.cuh"
#include "tc_sm100.cuh"

namespace qmcgb {

// =============================================================================
// Orbital evaluation: value, gradient and Laplacian of orbitals [o_begin, o_begin+32V)
// at point r, by one warp (Sec. "B-spline basis sets": 64 coefficient rows per point,
// each a contiguous run of orbital coefficients). Lane l owns V consecutive orbitals and
// reads them with one 16-byte load per row (V = 1: one orbital per lane, which spreads a
// small orbital set over more warps). r must be the same in every lane.
// =============================================================================
template <class TT, class TW, int V = TabVec<TT>::V>
__device__ __forceinline__ void vgl_warp(const SysParams& S, const double r[3], int o_begin,
                                         int n_eval, TW* __restrict__ out, int ld_out) {
  using A = typename AccOf<TT>::type;
  static_assert(V == TabVec<TT>::V || V == 1, "vector width: the table's or 1");
  const int lane = threadIdx.x & 31;
  // grid cell and fractional offset per axis, computed in double by lanes 0..2
  A tl = A(0);
  int il = 0;
  if (lane < 3) {
    const double s = r[lane] * S.inv_delta[lane];
    const double fi = floor(s);
    tl = (A)(s - fi);
    il = (int)fi;
  }
  const int o0 = o_begin + lane * V;
  const int nn[3] = {S.nx, S.ny, S.nz};
  A w[3][3][4];
  int idx[3][4];
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    const A t = __shfl_sync(0xffffffffu, tl, d);
    const int i = __shfl_sync(0xffffffffu, il, d);
    bspline_w<A>(t, w[d][0], w[d][1], w[d][2]);
    const A inv = Cst<A>::invd(S, d), inv2 = inv * inv;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      w[d][1][q] *= inv;
      w[d][2][q] *= inv2;
      idx[d][q] = (((i - 1 + q) % nn[d]) + nn[d]) % nn[d];   // always in [0, n)
    }
  }
  if (o0 >= n_eval) return;
  A acc[5][V];
#pragma unroll
  for (int k = 0; k < 5; ++k)
#pragma unroll
    for (int v = 0; v < V; ++v) acc[k][v] = A(0);
  const TT* __restrict__ tab = static_cast<const TT*>(S.table);
#pragma unroll
  for (int a = 0; a < 4; ++a) {
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      const A wxy = w[0][0][a] * w[1][0][b];
      const A dxy = w[0][1][a] * w[1][0][b];
      const A xdy = w[0][0][a] * w[1][1][b];
      const A lxy = w[0][2][a] * w[1][0][b] + w[0][0][a] * w[1][2][b];
      const size_t base = ((size_t)idx[0][a] * S.ny + idx[1][b]) * S.nz;
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        float cf[TabVec<TT>::V];
        double cd[TabVec<TT>::V];
        if constexpr (V == 1)
          tab_load1(tab + (base + idx[2][c]) * S.ld + o0, cf[0], cd[0]);
        else
          TabVec<TT>::load(tab + (base + idx[2][c]) * S.ld + o0, cf, cd);
        const A wv = wxy * w[2][0][c], wgx = dxy * w[2][0][c], wgy = xdy * w[2][0][c];
        const A wgz = wxy * w[2][1][c], wl = lxy * w[2][0][c] + wxy * w[2][2][c];
#pragma unroll
        for (int v = 0; v < V; ++v) {
          A cv;
          if constexpr (sizeof(A) == 8) cv = cd[v]; else cv = cf[v];
          acc[0][v] += wv * cv;
          acc[1][v] += wgx * cv;
          acc[2][v] += wgy * cv;
          acc[3][v] += wgz * cv;
          acc[4][v] += wl * cv;
        }
      }
    }
  }
  if constexpr (V == 1) {
    if (o0 < n_eval)
#pragma unroll
      for (int k = 0; k < 5; ++k) out[k * ld_out + o0] = (TW)acc[k][0];
    return;
  } else {
  if (o0 + V <= n_eval) {
#pragma unroll
    for (int k = 0; k < 5; ++k) {
      TW* p = out + k * ld_out + o0;
      if constexpr (sizeof(A) == 8) {
        *reinterpret_cast<double2*>(p) = make_double2(acc[k][0], acc[k][1]);
      } else {
#pragma unroll
        for (int v = 0; v < V; v += 4)
          *reinterpret_cast<float4*>(p + v) =
              make_float4(acc[k][v], acc[k][v + 1], acc[k][v + 2], acc[k][v + 3]);
      }
    }
  } else {
#pragma unroll
    for (int k = 0; k < 5; ++k)
#pragma unroll
      for (int v = 0; v < V; ++v)
        if (o0 + v < n_eval) out[k * ld_out + o0 + v] = (TW)acc[k][v];
  }
  }
}

// VGL of every electron of every walker at its current position (walker set-up and
// re-inversion): one warp per (walker, electron, 32V-orbital chunk).
template <class TT, class TW>
__global__ void __launch_bounds__(256, sizeof(TT) == 8 ? 1 : 2) k_vgl_current(SysParams S, WalkParams Wk) {
  constexpr int V = TabVec<TT>::V;
  const int chunks = (Wk.ld_v + 32 * V - 1) / (32 * V);
  const long long gw = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const long long total = (long long)Wk.n_w * S.n_e * chunks;
  if (gw >= total) return;
  const int ch = (int)(gw % chunks);
  const long long pe = gw / chunks;
  const int e = (int)(pe % S.n_e);
  const int w = (int)(pe / S.n_e);
  const double* P = Wk.pos + (size_t)w * 3 * S.n_e;
  const double r[3] = {P[e], P[S.n_e + e], P[2 * S.n_e + e]};
  const int ns = e < S.n_up ? S.n_up : S.n_dn;
  TW* out = static_cast<TW*>(Wk.vgl) + ((size_t)w * S.n_e + e) * 5 * Wk.ld_v;
  vgl_warp<TT, TW>(S, r, ch * 32 * V, ns, out, Wk.ld_v);
}

// Metropolis proposals of electrons [e0, e1) of every walker in sweep t:
// r' = wrap(r + step xi); prop[w][e-e0] = (x', y', z', u). One thread per move.
static __global__ void k_proposals(SysParams S, WalkParams Wk, uint32_t t, int e0, int e1,
                            Prop* __restrict__ prop) {
  const int ne = e1 - e0;
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (long long)Wk.n_w * ne) return;
  const int w = (int)(i / ne), e = e0 + (int)(i % ne);
  double xi[3], u;
  move_draws(S, sweep_index(Wk, t), (uint32_t)e, Wk.wid[w], xi, u);
  const double* P = Wk.pos + (size_t)w * 3 * S.n_e;
  Prop o;
  o.x = wrap_box(P[e] + S.step * xi[0], S.L);
  o.y = wrap_box(P[S.n_e + e] + S.step * xi[1], S.L);
  o.z = wrap_box(P[2 * S.n_e + e] + S.step * xi[2], S.L);
  o.u = u;
  prop[i] = o;
}

// Draws of the drift-diffusion moves of every electron of every walker in sweep t:
// draw[w][e] = (xi_x, xi_y, xi_z, ln u). They depend on the Philox counter alone, not on
// the chain, so they are formed ahead of the sequential moves, one thread per move, and the
// sweep reads them with its prefetch instead of evaluating Box-Muller in FP64 inside a move;
// the acceptance u < A is taken as ln u < ln A.
static __global__ void k_drift_draws(SysParams S, WalkParams Wk, uint32_t t,
                                     Prop* __restrict__ draw) {
  const int ne = S.n_e;
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (long long)Wk.n_w * ne) return;
  const int w = (int)(i / ne), e = (int)(i % ne);
  if (Wk.n_live && w >= *Wk.n_live) return;
  double xi[3], u;
  move_draws(S, sweep_index(Wk, t), (uint32_t)e, Wk.wid[w], xi, u);
  Prop o;
  o.x = xi[0];
  o.y = xi[1];
  o.z = xi[2];
  o.u = log(u);
  draw[i] = o;
}

// VGL at every proposed position of a chunk: out[w][e-e0][5][ld_v].
template <class TT, class TW>
__global__ void __launch_bounds__(256, sizeof(TT) == 8 ? 1 : 2) k_vgl_proposals(SysParams S, WalkParams Wk, int e0, int e1,
                                                      const Prop* __restrict__ prop,
                                                      TW* __restrict__ out) {
  constexpr int V = TabVec<TT>::V;
  const int ns = e0 < S.n_up ? S.n_up : S.n_dn;
  const int chunks = (ns + 32 * V - 1) / (32 * V);
  const long long gw = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const long long nmov = (long long)Wk.n_w * (e1 - e0);
  if (gw >= nmov * chunks) return;
  const int ch = (int)(gw % chunks);
  const long long mv = gw / chunks;
  const Prop p = prop[mv];
  const double r[3] = {p.x, p.y, p.z};
  TW* o = out + (size_t)mv * 5 * Wk.ld_v;
  vgl_warp<TT, TW>(S, r, ch * 32 * V, ns, o, Wk.ld_v);
  // the padding columns N_s..ld_v-1 of the five rows are zero, as in the current rows that an
  // accepted move's rows replace whole (the buffer also serves the other spin block's moves)
  if (ch == chunks - 1) {
    const int lane = threadIdx.x & 31;
    for (int j = ns + lane; j < Wk.ld_v; j += 32)
#pragma unroll
      for (int q = 0; q < 5; ++q) o[(size_t)q * Wk.ld_v + j] = TW(0);
  }
}

// =============================================================================
// FP64 Gauss-Jordan inversion with partial pivoting of M (n x n, row-major, global),
// in place, by one thread block. Returns false on an exactly zero or non-finite pivot.
// ln|det M| and its sign are accumulated from the pivots and row interchanges.
//
// The pivots are taken b at a time. Within a panel of b pivot columns, those columns are kept
// current in shared memory (Cur) and updated by every step as in plain Gauss-Jordan; each
// other element is left in M and represented as M[i][j] - sum_s F[i][s] H[s][j], with F[i][s]
// the multiplier of row i at step s (its panel column value then) and H[s] the pivot row of
// step s divided by its pivot. A pivot row's stored values become its H row and its earlier
// multipliers zero, so the one formula holds for every row. One pass per panel then applies
// the rank-b update, instead of one pass over the whole matrix per pivot: the matrix crosses
// L2 n/b times instead of n times, and the FP64 arithmetic becomes the bound.
// =============================================================================
// One pivot per pass, with O(n) shared memory: the form the sweep kernel's in-kernel
// re-inversion uses inside its own shared-memory budget.
static __device__ bool gj_invert_fp64_plain(double* __restrict__ M, int n, double* colk, int* perm,
                               double* redv, int* redi, double& logdet, double& sign) {
  const int tid = threadIdx.x, nt = blockDim.x;
  const int lane = tid & 31, warp = tid >> 5, nw = nt >> 5;
  double ld = 0.0, sg = 1.0;
  bool ok = true;
  for (int k = 0; k < n; ++k) {
    double best = -1.0;
    int bi = k;
    for (int i = k + tid; i < n; i += nt) {
      const double a = fabs(M[(size_t)i * n + k]);
      if (a > best) { best = a; bi = i; }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const double ob = __shfl_xor_sync(0xffffffffu, best, o);
      const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
      if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
    }
    if (lane == 0) { redv[warp] = best; redi[warp] = bi; }
    __syncthreads();
    best = redv[0];
    bi = redi[0];
    for (int w = 1; w < nw; ++w)
      if (redv[w] > best || (redv[w] == best && redi[w] < bi)) { best = redv[w]; bi = redi[w]; }
    const double pv = M[(size_t)bi * n + k];
    __syncthreads();
    if (!(pv != 0.0) || !isfinite(pv)) { ok = false; break; }   // uniform across the block
    if (bi != k) {
      for (int j = tid; j < n; j += nt) {
        const double a = M[(size_t)k * n + j];
        M[(size_t)k * n + j] = M[(size_t)bi * n + j];
        M[(size_t)bi * n + j] = a;
      }
      sg = -sg;
    }
    if (tid == 0) perm[k] = bi;
    if (tid == 0) ld += log(fabs(pv));
    if (pv < 0) sg = -sg;
    __syncthreads();
    for (int i = tid; i < n; i += nt) colk[i] = M[(size_t)i * n + k];
    __syncthreads();
    const double pinv = 1.0 / pv;
    for (int j = tid; j < n; j += nt) {
      const double pr = (j == k) ? pinv : M[(size_t)k * n + j] * pinv;
      M[(size_t)k * n + j] = pr;
      if (j == k) {
        for (int i = 0; i < n; ++i)
          if (i != k) M[(size_t)i * n + j] = -colk[i] * pinv;
      } else {
        for (int i = 0; i < n; ++i)
          if (i != k) M[(size_t)i * n + j] -= colk[i] * pr;
      }
    }
    __syncthreads();
  }
  if (ok) {
    for (int k = n - 1; k >= 0; --k) {
      const int p = perm[k];
      if (p != k)
        for (int i = tid; i < n; i += nt) {
          const double a = M[(size_t)i * n + k];
          M[(size_t)i * n + k] = M[(size_t)i * n + p];
          M[(size_t)i * n + p] = a;
        }
      __syncthreads();
    }
  }
  logdet = ld;   // valid in thread 0
  sign = sg;
  return ok;
}

__host__ __device__ inline int gj_panel_width(int n) { return n <= 512 ? 8 : 4; }
__host__ __device__ inline size_t gj_smem_bytes(int n) {
  const size_t b = gj_panel_width(n);
  return sizeof(double) * (32 + 3 * (size_t)n * b) + sizeof(int) * ((size_t)n + 32);
}

static __device__ bool gj_invert_fp64(double* __restrict__ M, int n, char* smem, double& logdet,
                                      double& sign) {
  const int b = gj_panel_width(n);
  double* redv = reinterpret_cast<double*>(smem);    // [32] pivot search, one per warp
  double* Cur = redv + 32;                            // [n][b] the panel's columns, current
  double* F = Cur + (size_t)n * b;                    // [n][b] multipliers of the panel's steps
  double* H = F + (size_t)n * b;                      // [b][n] scaled pivot rows
  int* perm = reinterpret_cast<int*>(H + (size_t)b * n);   // [n] pivot row of each step
  int* redi = perm + n;                               // [32]
  const int tid = threadIdx.x, nt = blockDim.x;
  const int lane = tid & 31, warp = tid >> 5, nw = nt >> 5;
  double ld = 0.0, sg = 1.0;
  bool ok = true;
  for (int k0 = 0; k0 < n && ok; k0 += b) {
    const int bb = min(b, n - k0);
    for (int i = tid; i < n * bb; i += nt) {
      const int r = i / bb, t = i - r * bb;
      Cur[r * b + t] = M[(size_t)r * n + k0 + t];
      F[r * b + t] = 0.0;
    }
    __syncthreads();
    for (int s = 0; s < bb; ++s) {
      const int k = k0 + s;
      double best = -1.0;
      int bi = k;
      for (int i = k + tid; i < n; i += nt) {
        const double a = fabs(Cur[i * b + s]);
        if (a > best) { best = a; bi = i; }
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        const double ob = __shfl_xor_sync(0xffffffffu, best, o);
        const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
        if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
      }
      if (lane == 0) { redv[warp] = best; redi[warp] = bi; }
      __syncthreads();
      best = redv[0];
      bi = redi[0];
      for (int w = 1; w < nw; ++w)
        if (redv[w] > best || (redv[w] == best && redi[w] < bi)) { best = redv[w]; bi = redi[w]; }
      const double pv = Cur[bi * b + s];
      __syncthreads();
      if (!(pv != 0.0) || !isfinite(pv)) { ok = false; break; }   // uniform across the block
      if (bi != k) {
        for (int j = tid; j < n; j += nt) {
          const double a = M[(size_t)k * n + j];
          M[(size_t)k * n + j] = M[(size_t)bi * n + j];
          M[(size_t)bi * n + j] = a;
        }
        if (tid < bb) {
          double a = Cur[k * b + tid];
          Cur[k * b + tid] = Cur[bi * b + tid];
          Cur[bi * b + tid] = a;
          a = F[k * b + tid];
          F[k * b + tid] = F[bi * b + tid];
          F[bi * b + tid] = a;
        }
        sg = -sg;
      }
      if (tid == 0) {
        perm[k] = bi;
        ld += log(fabs(pv));
      }
      if (pv < 0) sg = -sg;
      __syncthreads();
      // the pivot row, current and divided by the pivot
      const double pinv = 1.0 / pv;
      for (int j = tid; j < n; j += nt) {
        double v;
        if (j >= k0 && j < k0 + bb) {
          v = Cur[k * b + (j - k0)];
        } else {
          v = M[(size_t)k * n + j];
          for (int u = 0; u < s; ++u) v -= F[k * b + u] * H[(size_t)u * n + j];
        }
        H[(size_t)s * n + j] = v * pinv;
      }
      __syncthreads();
      // the panel's columns: one plain Gauss-Jordan step; the multipliers of this step
      for (int i = tid; i < n; i += nt) {
        if (i == k) continue;
        const double f = Cur[i * b + s];
        for (int t = 0; t < bb; ++t)
          Cur[i * b + t] = (t == s) ? -f * pinv : Cur[i * b + t] - f * H[(size_t)s * n + k0 + t];
        F[i * b + s] = f;
      }
      if (tid < bb) Cur[k * b + tid] = (tid == s) ? pinv : H[(size_t)s * n + k0 + tid];
      if (tid <= s) F[k * b + tid] = 0.0;
      for (int j = tid; j < n; j += nt)
        if (j < k0 || j >= k0 + bb) M[(size_t)k * n + j] = H[(size_t)s * n + j];
      __syncthreads();
    }
    if (!ok) break;
    // the rank-bb update of every other column, and the panel's columns written back
    for (int i = warp; i < n; i += nw) {
      double f[8];
#pragma unroll
      for (int t = 0; t < 8; ++t) f[t] = t < bb ? F[i * b + t] : 0.0;
      double* row = M + (size_t)i * n;
      for (int j = lane; j < n; j += 32) {
        if (j >= k0 && j < k0 + bb) {
          row[j] = Cur[i * b + (j - k0)];
        } else {
          double v = row[j];
#pragma unroll
          for (int t = 0; t < 8; ++t)
            if (t < bb) v -= f[t] * H[(size_t)t * n + j];
          row[j] = v;
        }
      }
    }
    __syncthreads();
  }
  if (ok) {
    for (int k = n - 1; k >= 0; --k) {
      const int p = perm[k];
      if (p != k)
        for (int i = tid; i < n; i += nt) {
          const double a = M[(size_t)i * n + k];
          M[(size_t)i * n + k] = M[(size_t)i * n + p];
          M[(size_t)i * n + p] = a;
        }
      __syncthreads();
    }
  }
  logdet = ld;   // valid in thread 0
  sign = sg;
  return ok;
}

// Re-inversion of one spin block of walker w from the orbital values at the current
// positions: M = A^T (M[j][e] = phi_j(r_e)), so M^-1 = (A^-1)^T = Binv. Writes Binv in
// working precision, ln|det A| and its sign. Called by one whole block.
template <class TW>
__device__ void reinvert_block(const SysParams& S, const WalkParams& Wk, int w, int spin,
                               char* smem) {
  const int ns = spin ? S.n_dn : S.n_up;
  if (ns == 0) return;
  const int first = spin ? S.n_up : 0;
  const size_t msz = (size_t)Wk.ld_v * Wk.ld_v;
  double* M = Wk.scratch64 + (size_t)(2 * w + spin) * msz;   // one work matrix per (walker, spin)
  const TW* VG = static_cast<const TW*>(Wk.vgl) + (size_t)w * S.n_e * 5 * Wk.ld_v;
  for (int i = threadIdx.x; i < ns * ns; i += blockDim.x) {
    const int j = i / ns, e = i % ns;
    M[i] = (double)VG[(size_t)(first + e) * 5 * Wk.ld_v + j];
  }
  __syncthreads();
  double ld, sg;
  const bool ok = gj_invert_fp64(M, ns, smem, ld, sg);
  TW* B = binv_block<TW>(S, Wk, w, spin);
  if (ok)
    for (int i = threadIdx.x; i < ns * ns; i += blockDim.x) B[i] = (TW)M[i];
  if (threadIdx.x == 0) {
    if (ok) {
      Wk.logdet[2 * w + spin] = ld;
      Wk.sgn[2 * w + spin] = sg;
    } else {
      atomicOr(Wk.err, kErrSingular);
    }
  }
  __syncthreads();
}

// The same with the one-pivot-per-pass inversion in the caller's small work arrays (the sweep
// kernel's in-kernel re-inversion).
template <class TW>
__device__ void reinvert_block_plain(const SysParams& S, const WalkParams& Wk, int w, int spin,
                                     double* colk, int* perm, double* redv, int* redi) {
  const int ns = spin ? S.n_dn : S.n_up;
  if (ns == 0) return;
  const int first = spin ? S.n_up : 0;
  const size_t msz = (size_t)Wk.ld_v * Wk.ld_v;
  double* M = Wk.scratch64 + (size_t)(2 * w + spin) * msz;   // one work matrix per (walker, spin)
  const TW* VG = static_cast<const TW*>(Wk.vgl) + (size_t)w * S.n_e * 5 * Wk.ld_v;
  for (int i = threadIdx.x; i < ns * ns; i += blockDim.x) {
    const int j = i / ns, e = i % ns;
    M[i] = (double)VG[(size_t)(first + e) * 5 * Wk.ld_v + j];
  }
  __syncthreads();
  double ld, sg;
  const bool ok = gj_invert_fp64_plain(M, ns, colk, perm, redv, redi, ld, sg);
  TW* B = binv_block<TW>(S, Wk, w, spin);
  if (ok)
    for (int i = threadIdx.x; i < ns * ns; i += blockDim.x) B[i] = (TW)M[i];
  if (threadIdx.x == 0) {
    if (ok) {
      Wk.logdet[2 * w + spin] = ld;
      Wk.sgn[2 * w + spin] = sg;
    } else {
      atomicOr(Wk.err, kErrSingular);
    }
  }
  __syncthreads();
}

__host__ __device__ inline size_t reinvert_smem_bytes(int ld_v) { return gj_smem_bytes(ld_v); }

template <class TW>
__global__ void __launch_bounds__(256) k_reinvert(SysParams S, WalkParams Wk) {
  extern __shared__ __align__(16) char smem_r[];
  const int w = blockIdx.x >> 1, spin = blockIdx.x & 1;
  reinvert_block<TW>(S, Wk, w, spin, smem_r);
}

// Batched FP64 re-inversion of caller-supplied Slater matrices (one block per matrix):
// A[b][e][j] = phi_j(r_e) in T, Binv[b][e][j] = (A^-1)[j][e] in T, ln|det A| and sign in
// double (-inf and 0 for an exactly singular matrix). `work` holds one FP64 n x n matrix
// per block.
template <class T>
__global__ void __launch_bounds__(256) k_invert_batch(const T* __restrict__ A, T* __restrict__ Binv,
                                                     double* __restrict__ logdet,
                                                     double* __restrict__ sign, int n,
                                                     double* __restrict__ work) {
  extern __shared__ __align__(16) char smem_i[];
  const size_t nn = (size_t)n * n;
  const int b = blockIdx.x;
  double* M = work + (size_t)b * nn;
  const T* Ab = A + (size_t)b * nn;
  for (size_t i = threadIdx.x; i < nn; i += blockDim.x) {
    const size_t j = i / n, e = i % n;
    M[i] = (double)Ab[e * n + j];
  }
  __syncthreads();
  double ld, sg;
  const bool ok = gj_invert_fp64(M, n, smem_i, ld, sg);
  T* Bb = Binv + (size_t)b * nn;
  for (size_t i = threadIdx.x; i < nn; i += blockDim.x) Bb[i] = ok ? (T)M[i] : T(0);
  if (threadIdx.x == 0) {
    if (logdet) logdet[b] = ok ? ld : -INFINITY;
    if (sign) sign[b] = ok ? sg : 0.0;
  }
}

__host__ __device__ inline size_t invert_batch_smem_bytes(int n) { return gj_smem_bytes(n); }

// =============================================================================
// Re-inversion of the single-precision forms by one Newton step with an accurate residual.
// GB300 runs FP64 at 1/71 of the FP32 rate, so an O(N^3) FP64 inversion per period would
// dominate the sweep. Instead, with X = A^-1 the current (drifted) inverse:
//   R = I - A X   summed with the error-free transformations of Dot2 (Ogita, Rump and
//                 Oishi, "Accurate sum and dot product", SIAM J. Sci. Comput. 26 (2005)):
//                 TwoProduct by FMA and TwoSum, as accurate as a double-length product of
//                 the single-precision A and X, on the FP32 pipe;
//   X <- X + X R  in single precision (R is small, so this product needs no extra care).
// One step takes an inverse that has drifted by |R| to one limited by the FP32 storage of
// X (error ~ |R|^2 + 2^-24). Binv = X^T, so the update reads Binv[e] += sum_f R[f][e] Binv[f].
// A residual above kRefineMax (or not finite) means the inverse is too far off for one
// step; the caller then falls back to the FP64 Gauss-Jordan re-inversion.
// =============================================================================
constexpr float kRefineMax = 1e-2f;
// The batched refinement takes the Newton step up to kRefineSteps; above kRefineMax the
// re-inversion's FP64 stage adds compensated steps in the walker's block until the residual
// is within kRefineMax (0.2 -> 0.04 -> 1.6e-3 -> 2.6e-6), and only a residual beyond
// kRefineSteps, or one that does not contract, takes the FP64 Gauss-Jordan re-inversion.
constexpr float kRefineSteps = 0.2f;
constexpr int kTileElems = 2 * 32 * 64;      // two 32 x 64 single-precision tiles

__device__ __forceinline__ void dot2_step(float a, float b, float& P, float& E) {
  const float h = __fmul_rn(a, b);
  const float r = __fmaf_rn(a, b, -h);         // a*b = h + r exactly
  const float x = __fadd_rn(P, h);             // TwoSum(P, h) = x + q exactly
  const float z = __fsub_rn(x, P);
  const float q = __fadd_rn(__fsub_rn(P, __fsub_rn(x, z)), __fsub_rn(h, z));
  P = x;
  E = __fadd_rn(E, __fadd_rn(q, r));
}

// Returns max |R| over the matrix (identical in every thread).
// One Newton step X <- X + X R when max |R| <= max_r; returns max |R| (before the step).
static __device__ float refine_inverse(const SysParams& S, const WalkParams& Wk, int w, int spin,
                                float* tile, float* redf, float max_r = kRefineMax) {
  const int ns = spin ? S.n_dn : S.n_up;
  const int first = spin ? S.n_up : 0;
  const int ld5 = 5 * Wk.ld_v;
  const float* VG = static_cast<const float*>(Wk.vgl) + ((size_t)w * S.n_e + first) * ld5;
  float* B = binv_block<float>(S, Wk, w, spin);
  float* Rg = reinterpret_cast<float*>(Wk.scratch64 + (size_t)(2 * w + spin) * Wk.ld_v * Wk.ld_v);
  float* Bn = Rg + (size_t)ns * ns;
  float* As = tile;
  float* Bs = tile + 32 * 64;
  const int tid = threadIdx.x, ty = tid >> 4, tx = tid & 15;
  float rmax = 0.f;
  // R = I - A Binv^T, 64 x 64 output tiles, 4 x 4 outputs per thread
  for (int te = 0; te < ns; te += 64)
    for (int tf = 0; tf < ns; tf += 64) {
      float P[4][4], E[4][4];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) P[i][j] = E[i][j] = 0.f;
      for (int k0 = 0; k0 < ns; k0 += 32) {
        __syncthreads();
        for (int i = tid; i < 64 * 32; i += blockDim.x) {
          const int r = i & 63, kk = i >> 6, j = k0 + kk;
          const int e = te + r, f = tf + r;
          As[kk * 64 + r] = (e < ns && j < ns) ? VG[(size_t)e * ld5 + j] : 0.f;
          Bs[kk * 64 + r] = (f < ns && j < ns) ? B[(size_t)f * ns + j] : 0.f;
        }
        __syncthreads();
#pragma unroll 4
        for (int kk = 0; kk < 32; ++kk) {
          float a[4], b[4];
#pragma unroll
          for (int i = 0; i < 4; ++i) {
            a[i] = As[kk * 64 + ty + 16 * i];
            b[i] = Bs[kk * 64 + tx + 16 * i];
          }
#pragma unroll
          for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int j = 0; j < 4; ++j) dot2_step(a[i], b[j], P[i][j], E[i][j]);
        }
      }
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const int e = te + ty + 16 * i, f = tf + tx + 16 * j;
          if (e < ns && f < ns) {
            const float r = __fsub_rn(__fsub_rn(e == f ? 1.f : 0.f, P[i][j]), E[i][j]);
            Rg[(size_t)e * ns + f] = r;
            rmax = fmaxf(rmax, isfinite(r) ? fabsf(r) : INFINITY);
          }
        }
    }
  // max |R| over the block
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) rmax = fmaxf(rmax, __shfl_xor_sync(0xffffffffu, rmax, o));
  __syncthreads();
  if ((tid & 31) == 0) redf[tid >> 5] = rmax;
  __syncthreads();
  rmax = 0.f;
  for (int q = 0; q < (int)(blockDim.x >> 5); ++q) rmax = fmaxf(rmax, redf[q]);
  if (!(rmax <= max_r)) return rmax;
  // Bn[e][j] = Binv[e][j] + sum_f R[f][e] Binv[f][j]
  for (int te = 0; te < ns; te += 64)
    for (int tj = 0; tj < ns; tj += 64) {
      float acc[4][4];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = 0.f;
      for (int f0 = 0; f0 < ns; f0 += 32) {
        __syncthreads();
        for (int i = tid; i < 64 * 32; i += blockDim.x) {
          const int c = i & 63, kk = i >> 6, f = f0 + kk;
          As[kk * 64 + c] = (f < ns && te + c < ns) ? Rg[(size_t)f * ns + te + c] : 0.f;
          Bs[kk * 64 + c] = (f < ns && tj + c < ns) ? B[(size_t)f * ns + tj + c] : 0.f;
        }
        __syncthreads();
#pragma unroll 4
        for (int kk = 0; kk < 32; ++kk) {
          float a[4], b[4];
#pragma unroll
          for (int i = 0; i < 4; ++i) {
            a[i] = As[kk * 64 + ty + 16 * i];
            b[i] = Bs[kk * 64 + tx + 16 * i];
          }
#pragma unroll
          for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
        }
      }
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const int e = te + ty + 16 * i, c = tj + tx + 16 * j;
          if (e < ns && c < ns) Bn[(size_t)e * ns + c] = B[(size_t)e * ns + c] + acc[i][j];
        }
    }
  __syncthreads();
  for (int i = tid; i < ns * ns; i += blockDim.x) B[i] = Bn[i];
  __syncthreads();
  return rmax;
}

// =============================================================================
// The sequential sweep of electrons [e0, e1) (one spin block) of every walker: one
// thread block per walker. Per move (Sec. "Trial Moves", Eq. accept_reject):
//   x  = column e of the current inverse = Binv0[e] - sum_l z_l U_l   (delayed window)
//   R  = phi(r') . x,   G = grad phi(r') . x / R
//   dJ = sum over electrons and ions of u(|r' - r_j|) - u(|r_e - r_j|), grad J at r'
//   A  = min(1, R^2 exp(2 dJ)), accept iff u < A.
// Accepted moves enter a delayed-update window (rank-k, Sec. "Multi-Determinant
// Slater-Jastrow Form"; k = 1 is Sherman-Morrison). With U_l = Binv0[e_l] (rows of the
// inverse at the window's electrons), Phi_l their new orbital rows and
// C[l][l'] = Phi_l . U_l', the current inverse is Binv[n] = Binv0[n] - sum_l (C^-1 d_n)_l U_l
// with d_n[l] = Phi_l . Binv0[n] - delta(n, e_l); a full window is applied to every row
// of Binv0 (the flush) and emptied.
// =============================================================================
constexpr long long kSweepWaitPolls = 20000000;   // bounded wait for a prefetch (polls)

template <class TW>
struct SweepSmem {
  double* posd;  // [3][n_e] exact positions
  double* outd;  // [16] block sums
  double* colk;  // [ld_v]  re-inversion
  double* redv;  // [32]
  double* propb; // [2][4] double-buffered proposal (x, y, z, u)
  TW* posw;      // [3][n_e] positions in working precision
  TW* phib;      // [2][5 * ld_v] double-buffered proposal orbitals (value, grad, lap)
  TW* rowb;      // [2][ld_v]     double-buffered Binv0[e]
  TW* xs;        // [ld_v]        current column e of the inverse (window applied)
  TW* wphi;      // [k][ld_v]   window: new orbital rows
  TW* wu;        // [k][ld_v]   window: Binv0 rows of the moved electrons
  TW* rowbuf;    // [nwarps][2][ld_v]  flush: double-buffered rows
  TW* cinv;      // [k][k + 1]  rows padded by one: both row and column walks are conflict-free
  TW* dvec;      // [k]
  TW* zvec;      // [k]
  TW* crow;      // [k]
  TW* yvec;      // [k]
  TW* dz;        // [nwarps][2k]  flush: per-warp d and z
  TW* red;       // [32][12]
  TW* sc;        // [8] per-move scalars: r' (3), R
  int* wrow;     // [k]
  int* perm;     // [ld_v]
  int* redi;     // [32]
  int* flag;     // [4]
  float* tile;   // [kTileElems] refinement tiles (single-precision forms only)
};

// `internal`: the kernel flushes windows and re-inverts itself (row buffers, flush
// scratch and refinement tiles are needed); otherwise both happen in batched kernels.
template <class TW>
__host__ __device__ inline size_t sweep_smem_bytes(int n_e, int ld_v, int k, int nwarps,
                                                   bool internal = true) {
  const int nrb = internal ? nwarps : 0;
  size_t b = sizeof(double) * (3 * (size_t)n_e + 16 + ld_v + 32 + 8);
  b += sizeof(TW) * (3 * (size_t)n_e + (size_t)ld_v * (10 + 3 + 2 * k + 2 * nrb) + (size_t)k * (k + 1) +
                     4 * k + 2 * k * nrb + 32 * 12 + 8);
  b += sizeof(int) * (k + ld_v + 32 + 4);
  b = (b + 15) & ~size_t(15);
  if (sizeof(TW) == 4 && internal) b += sizeof(float) * kTileElems;
  return b + 16;
}

template <class TW>
__device__ __forceinline__ SweepSmem<TW> carve(char* base, int n_e, int ld_v, int k, int nwarps,
                                               bool internal) {
  if (!internal) nwarps = 0;
  SweepSmem<TW> s;
  double* d = reinterpret_cast<double*>(base);
  s.propb = d; d += 8;                 // first: 16-byte aligned for cp.async
  s.posd = d; d += 3 * n_e;
  s.outd = d; d += 16;
  s.colk = d; d += ld_v;
  s.redv = d; d += 32;
  // working-precision arrays start 16-byte aligned (cp.async targets)
  char* c = reinterpret_cast<char*>(d);
  c = base + ((c - base + 15) & ~size_t(15));
  TW* t = reinterpret_cast<TW*>(c);
  s.phib = t; t += 10 * ld_v;
  s.rowb = t; t += 2 * ld_v;
  s.xs = t; t += ld_v;
  s.posw = t; t += 3 * n_e;
  s.wphi = t; t += (size_t)k * ld_v;
  s.wu = t; t += (size_t)k * ld_v;
  s.rowbuf = t; t += (size_t)nwarps * 2 * ld_v;
  s.cinv = t; t += k * (k + 1);
  s.dvec = t; t += k;
  s.zvec = t; t += k;
  s.crow = t; t += k;
  s.yvec = t; t += k;
  s.dz = t; t += 2 * k * nwarps;
  s.red = t; t += 32 * 12;
  s.sc = t; t += 8;
  int* ip = reinterpret_cast<int*>(t);
  s.wrow = ip; ip += k;
  s.perm = ip; ip += ld_v;
  s.redi = ip; ip += 32;
  s.flag = ip; ip += 4;
  const size_t off = (reinterpret_cast<char*>(ip) - base + 15) & ~size_t(15);
  s.tile = reinterpret_cast<float*>(base + off);
  return s;
}

// ---------------------------------------------------------------- async copies
__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(gmem));
}
__device__ __forceinline__ void cp_async_elem(float* smem, const float* gmem) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(sa), "l"(gmem));
}
__device__ __forceinline__ void cp_async_elem(double* smem, const double* gmem) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(sa), "l"(gmem));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
__device__ __forceinline__ void cp_async_wait_all() {
  asm volatile("cp.async.wait_group 0;\n" ::: "memory");
}
__device__ __forceinline__ void cp_async_wait_1() {
  asm volatile("cp.async.wait_group 1;\n" ::: "memory");
}

// Apply the window (m rows) to every row of Binv0 (B, ns x ns) and empty it:
// Binv0[n] -= sum_l z_l U_l with z = C^-1 d_n, d_n[l] = Phi_l . Binv0[n] - delta(n, e_l).
template <class TW>
__device__ void flush_window(TW* __restrict__ B, int ns, int m, int kc,
                             const SweepSmem<TW>& sm, int ld_v) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  TW* rbuf = sm.rowbuf + (size_t)warp * 2 * ld_v;     // two row buffers per warp
  TW* dw = sm.dz + (size_t)warp * 2 * kc;
  TW* zw = dw + kc;
  if (warp < ns) {
    for (int j = lane; j < ns; j += 32) cp_async_elem(rbuf + j, B + (size_t)warp * ns + j);
    cp_async_commit();
  }
  int it = 0;
  for (int n = warp; n < ns; n += nw, ++it) {
    TW* rb = rbuf + (size_t)(it & 1) * ld_v;
    const int nn = n + nw;
    if (nn < ns) {          // the next row of this warp is fetched while this one is used
      TW* nb = rbuf + (size_t)((it + 1) & 1) * ld_v;
      for (int j = lane; j < ns; j += 32) cp_async_elem(nb + j, B + (size_t)nn * ns + j);
      cp_async_commit();
      asm volatile("cp.async.wait_group 1;\n" ::: "memory");
    } else {
      cp_async_wait_all();
    }
    __syncwarp();
    for (int l = 0; l < m; ++l) {
      TW s = TW(0);
      const TW* ph = sm.wphi + (size_t)l * ld_v;
      for (int j = lane; j < ns; j += 32) s += ph[j] * rb[j];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
      if (lane == 0) dw[l] = s - (sm.wrow[l] == n ? TW(1) : TW(0));
    }
    __syncwarp();
    for (int l = lane; l < m; l += 32) {
      TW z = TW(0);
      for (int lp = 0; lp < m; ++lp) z += sm.cinv[l * (kc + 1) + lp] * dw[lp];
      zw[l] = z;
    }
    __syncwarp();
    for (int j = lane; j < ns; j += 32) {
      TW v = rb[j];
      for (int l = 0; l < m; ++l) v -= zw[l] * sm.wu[(size_t)l * ld_v + j];
      B[(size_t)n * ns + j] = v;
    }
    __syncwarp();
  }
}

// Jastrow difference of a move of electron e to r' (Sec. "Jastrow factor"): the sum over the
// other electrons j and the ions I of u(|r' - r_j|) - u(|r_e - r_j|), minimum image. Each
// returns the share of thread jtid of a group of jnt threads; posw is [3][n_e].
// Value only (a Metropolis ratio): electron pairs two per iteration, the pair j = e
// evaluated and dropped, no branches.
template <class TW>
__device__ __forceinline__ TW jastrow_delta_value(const SysParams& S, const JastrowTab<TW>& jt,
                                                  const TW* posw, const TW* ionw, int e,
                                                  const TW (&rn)[3], TW Lw, TW iLw, int jtid,
                                                  int jnt) {
  const int n_e = S.n_e;
  const TW ro[3] = {posw[e], posw[n_e + e], posw[2 * n_e + e]};
  TW dj = 0, dj2 = 0;
  const bool e_up = e < S.n_up;
  const auto pair_e = [&](int j) -> TW {
    const int f = ((j < S.n_up) == e_up) ? 1 : 2;
    TW rn2 = 0, ro2 = 0;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const TW q = posw[c * n_e + j];
      const TW dn = min_image<TW>(rn[c] - q, Lw, iLw);
      const TW dq = min_image<TW>(ro[c] - q, Lw, iLw);
      rn2 += dn * dn;
      ro2 += dq * dq;
    }
    const TW v = jastrow_value_r2<TW>(jt, f, rn2) - jastrow_value_r2<TW>(jt, f, ro2);
    return j != e ? v : TW(0);
  };
  int j = jtid;
  for (; j + jnt < n_e; j += 2 * jnt) {
    dj += pair_e(j);
    dj2 += pair_e(j + jnt);
  }
  if (j < n_e) dj += pair_e(j);
  for (int I = jtid; I < S.n_ion; I += jnt) {
    TW rn2 = 0, ro2 = 0;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const TW q = ionw[c * S.n_ion + I];
      const TW dn = min_image<TW>(rn[c] - q, Lw, iLw);
      const TW dq = min_image<TW>(ro[c] - q, Lw, iLw);
      rn2 += dn * dn;
      ro2 += dq * dq;
    }
    dj2 += jastrow_value_r2<TW>(jt, 0, rn2) - jastrow_value_r2<TW>(jt, 0, ro2);
  }
  return dj + dj2;
}

// The same difference with the gradient of J at r' in g (drift moves and traces).
template <class TW>
__device__ __forceinline__ TW jastrow_delta_grad(const SysParams& S, const JastrowTab<TW>& jt,
                                                 const TW* posw, const TW* ionw, int e,
                                                 const TW (&rn)[3], TW Lw, TW iLw, int jtid,
                                                 int jnt, TW (&g)[3]) {
  const int n_e = S.n_e;
  const TW ro[3] = {posw[e], posw[n_e + e], posw[2 * n_e + e]};
  TW dj = 0, gx = 0, gy = 0, gz = 0;
  const int ntot = n_e + S.n_ion;
  for (int j = jtid; j < ntot; j += jnt) {
    if (j == e) continue;
    TW q[3];
    int f;
    if (j < n_e) {
      q[0] = posw[j]; q[1] = posw[n_e + j]; q[2] = posw[2 * n_e + j];
      f = ((j >= S.n_up) == (e >= S.n_up)) ? 1 : 2;
    } else {
      const int I = j - n_e;
      q[0] = ionw[I]; q[1] = ionw[S.n_ion + I]; q[2] = ionw[2 * S.n_ion + I];
      f = 0;
    }
    if (jt.M[f] == 0) continue;
    TW dn[3], dq[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      dn[c] = min_image<TW>(rn[c] - q[c], Lw, iLw);
      dq[c] = min_image<TW>(ro[c] - q[c], Lw, iLw);
    }
    const TW rnn = sqrt(dn[0] * dn[0] + dn[1] * dn[1] + dn[2] * dn[2]);
    const TW roo = sqrt(dq[0] * dq[0] + dq[1] * dq[1] + dq[2] * dq[2]);
    TW un, dun, d2n, uo, duo, d2o;
    jastrow_eval<TW>(jt, f, rnn, un, dun, d2n);
    jastrow_eval<TW>(jt, f, roo, uo, duo, d2o);
    dj += un - uo;
    if (rnn > TW(0)) {
      const TW gg = dun / rnn;
      gx += gg * dn[0]; gy += gg * dn[1]; gz += gg * dn[2];
    }
  }
  g[0] = gx; g[1] = gy; g[2] = gz;
  return dj;
}

// ln|x| in the working precision, widened to FP64
__device__ __forceinline__ double log_abs_w(double x) { return log(fabs(x)); }
__device__ __forceinline__ double log_abs_w(float x) { return (double)logf(fabsf(x)); }

template <class TW>
__device__ __forceinline__ TW texp(TW x);
template <> __device__ __forceinline__ double texp<double>(double x) { return exp(x); }
template <> __device__ __forceinline__ float texp<float>(float x) { return expf(x); }

// kDrift: drift-diffusion proposals r' = r + tau grad ln|Psi| + sqrt(tau) xi (Eq.
// pmc:driftdiffusion_step with the adopted lambda = 1/2), whose orbital values are gathered
// in the kernel (table type TT) because the proposal depends on the current inverse; the
// acceptance includes the Green's-function ratio of Eq. pmc:g_driftdiffusion. The draws
// (xi, ln u) come from k_drift_draws through `prop` ([W][N_e], p_e0 = 0, p_n = N_e).
template <class TW, class TT, bool kFixedNode, bool kDrift>
__global__ void __launch_bounds__(256, 2) k_sweep(SysParams S, WalkParams Wk, uint32_t t, int e0,
                                              int e1, int kc, const TW* __restrict__ Pv,
                                              const Prop* __restrict__ prop, int p_e0, int p_n,
                                              int reinv_period, int reinv_on_acc, int ext_flush) {
  extern __shared__ __align__(16) char smem_s[];
  __shared__ JastrowTab<TW> jt;
  const int w = blockIdx.x;
  if (Wk.n_live && w >= *Wk.n_live) return;
  const int tid = threadIdx.x, nt = blockDim.x, lane = tid & 31, warp = tid >> 5;
  const int nw = nt >> 5;
  const int n_e = S.n_e, ld_v = Wk.ld_v, kcp = kc + 1;
  SweepSmem<TW> sm = carve<TW>(smem_s, n_e, ld_v, kc, nw, !ext_flush);
  jastrow_tab_fill<TW>(S, jt);
  __shared__ J3Tab<TW> j3t;
  j3_tab_fill<TW>(S, j3t);
  const int spin = e0 >= S.n_up ? 1 : 0;
  const int first = spin ? S.n_up : 0;
  const int ns = spin ? S.n_dn : S.n_up;
  const TW Lw = Cst<TW>::L(S), iLw = Cst<TW>::invL(S);
  const TW* ionw = Cst<TW>::ions(S);
  TW* B = binv_block<TW>(S, Wk, w, spin);
  TW* VG = static_cast<TW*>(Wk.vgl) + (size_t)w * n_e * 5 * ld_v;
  double* gpos = Wk.pos + (size_t)w * 3 * n_e;
  // Prefetch of move index e (orbital rows, proposal or drift draws, inverse row) into
  // buffer b: one thread hands the contiguous pieces to the bulk-copy unit, which completes
  // them on the buffer's mbarrier. An inverse row that is not 16-byte aligned (N_s *
  // sizeof(TW) not a multiple of 16) is fetched element-wise by every thread instead.
  __shared__ __align__(8) uint64_t pf_bar[2];
  const bool row_bulk = (ns * sizeof(TW)) % 16 == 0 && (reinterpret_cast<uintptr_t>(B) & 15) == 0;
  auto prefetch = [&](int e, int b) {
    const size_t mvi = (size_t)w * p_n + (e - p_e0);
    const TW* rs = B + (size_t)(e - first) * ns;
    TW* rd = sm.rowb + (size_t)b * ld_v;
    if (tid == 0) {
      // the block's reads of this buffer (ordered by the barrier before) precede the copies
      tc::fence_async_smem();
      const uint32_t nphi = 5u * ld_v * sizeof(TW), nrow = row_bulk ? ns * sizeof(TW) : 0u;
      tc::mbar_arrive_expect_tx(&pf_bar[b], nphi + (uint32_t)sizeof(Prop) + nrow);
      tc::bulk_g2s(sm.phib + (size_t)b * 5 * ld_v, kDrift ? VG + (size_t)e * 5 * ld_v : Pv + mvi * 5 * ld_v,
                   nphi, &pf_bar[b]);
      tc::bulk_g2s(sm.propb + 4 * b, prop + mvi, sizeof(Prop), &pf_bar[b]);
      if (row_bulk && nrow) tc::bulk_g2s(rd, rs, nrow, &pf_bar[b]);
    }
    if (!row_bulk) {
      for (int j = tid; j < ns; j += nt) cp_async_elem(rd + j, rs + j);
      cp_async_commit();
    }
  };
  // bounded wait for the prefetch of move index it (buffer it & 1, its (it >> 1)-th use)
  auto prefetch_wait = [&](int it) {
    if (!row_bulk) cp_async_wait_all();
    if (!tc::mbar_wait(&pf_bar[it & 1], (uint32_t)((it >> 1) & 1), kSweepWaitPolls) && lane == 0)
      atomicOr(Wk.err, kErrTimeout);
  };
  if (tid == 0) {
    tc::mbar_init(&pf_bar[0], 1);
    tc::mbar_init(&pf_bar[1], 1);
    tc::fence_mbar_init();
  }
  __syncthreads();
  for (int i = tid; i < 3 * n_e; i += nt) {
    const double p = gpos[i];
    sm.posd[i] = p;
    sm.posw[i] = (TW)p;
  }
  // thread 0: ln|det| = logdet + ln lprod + lexp ln 2, the accepted ratios multiplied in FP64
  // with their binary exponents split off (no logarithm inside a move)
  double logdet = 0.0, sgn = 1.0, lprod = 1.0;
  int lexp = 0;
  long long nacc = 0;
  double r2p = 0.0, r2a = 0.0;           // thread 0: squared proposed / accepted displacements
  if (tid == 0) {
    logdet = Wk.logdet[2 * w + spin];
    sgn = Wk.sgn[2 * w + spin];
  }
  int since = Wk.acc_since[2 * w + spin];
  int m = 0;
  const double sq_tau = kDrift ? sqrt(S.step) : 0.0, inv_2tau = kDrift ? 0.5 / S.step : 0.0;
  if (e0 < e1) prefetch(e0, 0);      // every prefetch issued is waited for inside the loop
  for (int e = e0; e < e1; ++e) {
    const int row = e - first;
    const int cur = (e - e0) & 1;
    prefetch_wait(e - e0);
    __syncthreads();
    if (e + 1 < e1) prefetch(e + 1, cur ^ 1);
    TW* phi = sm.phib + (size_t)cur * 5 * ld_v;
    const TW* row0 = sm.rowb + (size_t)cur * ld_v;
    if (!kDrift && tid == 0) {
      sm.sc[0] = (TW)sm.propb[4 * cur];
      sm.sc[1] = (TW)sm.propb[4 * cur + 1];
      sm.sc[2] = (TW)sm.propb[4 * cur + 2];
    }
    // Metropolis moves split the block: the determinant chain (d, z, x, ratio) runs on the
    // upper half of the warps while the lower half evaluates the Jastrow terms, which
    // depend on the positions only. Drift moves need x for the proposal and keep every
    // warp on each step.
    constexpr bool kSplit = !kDrift;
    const int nJ = kSplit ? nw / 2 : 0;              // Jastrow warps
    const bool det_grp = warp >= nJ;
    const int dt = tid - 32 * nJ, dnt = nt - 32 * nJ, dw = warp - nJ, dnw = nw - nJ;
    auto det_sync = [&]() {
      if constexpr (kSplit) named_barrier(2, dnt); else __syncthreads();
    };
    // With the block split, the bordering of C for an acceptance (crow_l = phi' . U_l,
    // a = phi' . Binv0[e], y = C^-T crow and a - crow . z, all compensated) rides along with
    // d and z: r' and its orbital row are known before the move starts. The Schur
    // complement a - crow . C^-1 d of the bordered C is the ratio itself (det of the
    // bordered C over det C), so x is formed only where the gradient is wanted. Drift
    // moves border C during the decision.
    const int nzy = kSplit ? 2 * m : m, nb = kSplit ? 2 * m + 1 : m;
    const bool need_x = !kSplit || Wk.trace;
    if (det_grp) {
      // d_l = Phi_l . Binv0[e] (compensated); with the split also crow_l and a.
      // A warp keeps four dots in flight so that their reductions overlap.
      constexpr int G = 4;
      for (int l0 = dw; l0 < nb; l0 += G * dnw) {
        const TW* a[G];
        const TW* b[G];
        TW s[G], c[G];
#pragma unroll
        for (int g = 0; g < G; ++g) {
          const int l = min(l0 + g * dnw, nb - 1);     // a slot past the end repeats a dot
          a[g] = l < m ? sm.wphi + (size_t)l * ld_v : phi;
          b[g] = (l < m || l == 2 * m) ? row0 : sm.wu + (size_t)(l - m) * ld_v;
          s[g] = TW(0);
          c[g] = TW(0);
        }
        for (int j = lane; j < ns; j += 32)
#pragma unroll
          for (int g = 0; g < G; ++g) comp_fma(s[g], c[g], a[g][j], b[g][j]);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1)
#pragma unroll
          for (int g = 0; g < G; ++g) {
            const TW s2 = __shfl_xor_sync(0xffffffffu, s[g], o);
            const TW c2 = __shfl_xor_sync(0xffffffffu, c[g], o);
            comp_merge(s[g], c[g], s2, c2);
          }
        if (lane == 0)
#pragma unroll
          for (int g = 0; g < G; ++g) {
            const int l = l0 + g * dnw;
            if (l < m) sm.dvec[l] = s[g] + c[g];
            else if (l < 2 * m) sm.crow[l - m] = s[g] + c[g];
            else if (l < nb) { sm.sc[4] = s[g]; sm.sc[5] = c[g]; }   // a, kept as a pair
          }
      }
      det_sync();
      // z = C^-1 d (row i of C^-1) and y = C^-T crow (column i - m), two partial sums each
      for (int i = dt; i < nzy; i += dnt) {
        const bool zi = i < m;
        const TW* ca = zi ? sm.cinv + i * kcp : sm.cinv + (i - m);
        const int cs = zi ? 1 : kcp;
        const TW* v = zi ? sm.dvec : sm.crow;
        TW z0 = TW(0), c0 = TW(0), z1 = TW(0), c1 = TW(0);
        int l = 0;
        for (; l + 1 < m; l += 2) {
          comp_fma(z0, c0, ca[l * cs], v[l]);
          comp_fma(z1, c1, ca[(l + 1) * cs], v[l + 1]);
        }
        if (l < m) comp_fma(z0, c0, ca[l * cs], v[l]);
        comp_merge(z0, c0, z1, c1);
        (zi ? sm.zvec[i] : sm.yvec[i - m]) = z0 + c0;
      }
      det_sync();
      if (kSplit && dw == dnw - 1) {
        // the ratio a - crow . z, also the corner of the bordered C
        TW sv = TW(0), sc2 = TW(0);
        for (int l = lane; l < m; l += 32) comp_fma(sv, sc2, -sm.crow[l], sm.zvec[l]);
        warp_sum_comp(sv, sc2);
        if (lane == 0) {
          TW a = sm.sc[4], ac2 = sm.sc[5];
          comp_merge(a, ac2, sv, sc2);
          sm.sc[6] = a;
          sm.sc[7] = ac2;
        }
      }
      // x = Binv0[e] - sum_l z_l U_l (column e of the current inverse), compensated
      for (int j = dt; need_x && j < ns; j += dnt) {
        TW xv = row0[j], xc = TW(0);
        for (int l = 0; l < m; ++l) comp_fma(xv, xc, -sm.zvec[l], sm.wu[(size_t)l * ld_v + j]);
        sm.xs[j] = xv + xc;
      }
    }
    if constexpr (kDrift) {
      // grad ln|Psi| at the current position: grad phi(r_e) . x + grad J(r_e)
      __syncthreads();
      TW g[6] = {0, 0, 0, 0, 0, 0};
      for (int j = tid; j < ns; j += nt) {
        const TW xv = sm.xs[j];
        g[0] += phi[ld_v + j] * xv;
        g[1] += phi[2 * ld_v + j] * xv;
        g[2] += phi[3 * ld_v + j] * xv;
      }
      const TW ro[3] = {sm.posw[e], sm.posw[n_e + e], sm.posw[2 * n_e + e]};
      for (int j = tid; j < n_e + S.n_ion; j += nt) {
        if (j == e) continue;
        TW q[3];
        int f;
        if (j < n_e) {
          q[0] = sm.posw[j]; q[1] = sm.posw[n_e + j]; q[2] = sm.posw[2 * n_e + j];
          f = ((j >= S.n_up) == (e >= S.n_up)) ? 1 : 2;
        } else {
          const int I = j - n_e;
          q[0] = ionw[I]; q[1] = ionw[S.n_ion + I]; q[2] = ionw[2 * S.n_ion + I];
          f = 0;
        }
        if (jt.M[f] == 0) continue;
        TW dq[3];
#pragma unroll
        for (int c = 0; c < 3; ++c) dq[c] = min_image<TW>(ro[c] - q[c], Lw, iLw);
        const TW r = sqrt(dq[0] * dq[0] + dq[1] * dq[1] + dq[2] * dq[2]);
        TW u, du, d2u;
        jastrow_eval<TW>(jt, f, r, u, du, d2u);
        if (r > TW(0)) {
          const TW gg = du / r;
          g[3] += gg * dq[0]; g[4] += gg * dq[1]; g[5] += gg * dq[2];
        }
      }
      if (j3t.on) {   // the three-body term's gradient at r_e (its difference is zero here)
        TW g3[3];
        (void)j3_delta<TW, true>(S, j3t, sm.posw, ionw, e, ro, ro, Lw, iLw,
                                 j3_group_warps(tid, nt), g3);
        g[3] += g3[0]; g[4] += g3[1]; g[5] += g3[2];
      }
      warp_sum<6, TW>(g);
      if (lane == 0)
#pragma unroll
        for (int k = 0; k < 6; ++k) sm.red[warp * 6 + k] = g[k];
      __syncthreads();
      if (tid == 0) {
        double go[3];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          TW v = TW(0);
          for (int q = 0; q < nw; ++q) v += sm.red[q * 6 + c] + sm.red[q * 6 + 3 + c];
          go[c] = (double)v;
        }
        // the move's draws, formed ahead of the sweep (k_drift_draws) and prefetched
        // (u stays in its slot for the decision)
        const double xi[3] = {sm.propb[4 * cur], sm.propb[4 * cur + 1], sm.propb[4 * cur + 2]};
        double dd[3];
        drift_disp(go, S.step, S.drift_a, dd);
        for (int c = 0; c < 3; ++c) {
          const double rn = wrap_box(sm.posd[c * n_e + e] + dd[c] + sq_tau * xi[c], S.L);
          sm.propb[4 * cur + c] = rn;
          sm.outd[10 + c] = dd[c];               // drift displacement of the forward move
          sm.sc[c] = (TW)rn;
        }
      }
      __syncthreads();
      // orbital values, gradients and Laplacians at r' (one warp per 32V-orbital chunk; one
      // orbital per lane while the block's warps cover the spin block that way)
      {
        constexpr int V = TabVec<TT>::V;
        const double rr[3] = {sm.propb[4 * cur], sm.propb[4 * cur + 1], sm.propb[4 * cur + 2]};
        if (ns <= 32 * nw) {
          if (warp < (ns + 31) / 32) vgl_warp<TT, TW, 1>(S, rr, warp * 32, ns, phi, ld_v);
        } else {
          const int chunks = (ns + 32 * V - 1) / (32 * V);
          for (int ch = warp; ch < chunks; ch += nw) vgl_warp<TT, TW>(S, rr, ch * 32 * V, ns, phi, ld_v);
        }
      }
      __syncthreads();
    }
    // drift moves: the ratio phi' . x (compensated) and its companion phi' . Binv0[e]
    // (compensated); the gradient wherever x is formed
    TW acc[9];
    TW rc = TW(0), ac = TW(0);     // compensation parts of acc[0] and acc[4]
    {
      TW a0 = 0, a1 = 0, a2 = 0, a3 = 0, a4 = 0;
      for (int j = dt; det_grp && need_x && j < ns; j += dnt) {   // the thread that wrote xs[j]
        const TW xv = sm.xs[j];
        if (!kSplit) {
          comp_fma(a0, rc, phi[j], xv);
          comp_fma(a4, ac, phi[j], row0[j]);
        }
        a1 += phi[ld_v + j] * xv;
        a2 += phi[2 * ld_v + j] * xv;
        a3 += phi[3 * ld_v + j] * xv;
      }
      acc[0] = a0; acc[1] = a1; acc[2] = a2; acc[3] = a3; acc[4] = a4;
    }
    // Jastrow difference and gradient at r' (the lower warps when the block is split)
    const int jtid = tid, jnt = kSplit ? 32 * nJ : nt;
    const bool jas_grp = !kSplit || !det_grp;
    if (!jas_grp) {
      acc[5] = 0; acc[6] = 0; acc[7] = 0; acc[8] = 0;
    } else if (!kDrift && !Wk.trace) {
      // Metropolis: the ratio needs Delta J only (no derivatives, no root beyond r_c)
      const TW rn[3] = {(TW)sm.propb[4 * cur], (TW)sm.propb[4 * cur + 1],
                        (TW)sm.propb[4 * cur + 2]};
      acc[5] = jastrow_delta_value<TW>(S, jt, sm.posw, ionw, e, rn, Lw, iLw, jtid, jnt);
      acc[6] = 0; acc[7] = 0; acc[8] = 0;
      if (j3t.on) {
        const TW ro[3] = {sm.posw[e], sm.posw[n_e + e], sm.posw[2 * n_e + e]};
        TW g3[3];
        acc[5] += j3_delta<TW, false>(S, j3t, sm.posw, ionw, e, ro, rn, Lw, iLw,
                                      j3_group_warps(jtid, jnt), g3);
      }
    } else {
      const TW rn[3] = {(TW)sm.propb[4 * cur], (TW)sm.propb[4 * cur + 1],
                        (TW)sm.propb[4 * cur + 2]};
      TW g[3];
      acc[5] = jastrow_delta_grad<TW>(S, jt, sm.posw, ionw, e, rn, Lw, iLw, jtid, jnt, g);
      if (j3t.on) {
        const TW ro[3] = {sm.posw[e], sm.posw[n_e + e], sm.posw[2 * n_e + e]};
        TW g3[3];
        acc[5] += j3_delta<TW, true>(S, j3t, sm.posw, ionw, e, ro, rn, Lw, iLw,
                                     j3_group_warps(jtid, jnt), g3);
        g[0] += g3[0]; g[1] += g3[1]; g[2] += g3[2];
      }
      acc[6] = g[0]; acc[7] = g[1]; acc[8] = g[2];
    }
    // block sums; warp partials added by thread 0 in working precision, R and a compensated
    warp_sum_comp(acc[0], rc);
    warp_sum_comp(acc[4], ac);
    {
      TW rest[7] = {acc[1], acc[2], acc[3], acc[5], acc[6], acc[7], acc[8]};
      warp_sum<7, TW>(rest);
      acc[1] = rest[0]; acc[2] = rest[1]; acc[3] = rest[2];
      acc[5] = rest[3]; acc[6] = rest[4]; acc[7] = rest[5]; acc[8] = rest[6];
    }
    if (lane == 0) {
#pragma unroll
      for (int k = 0; k < 9; ++k) sm.red[warp * 11 + k] = acc[k];
      sm.red[warp * 11 + 9] = rc;
      sm.red[warp * 11 + 10] = ac;
    }
    __syncthreads();
    if (warp == 0) {
      // lane k < 9 adds slot k of the warp partials (lanes 0 and 4 with their compensation)
      constexpr int kNW = kThreads / 32;
      TW v = TW(0);
      if (lane == 0 || lane == 4) {
        const int kq = lane == 0 ? 9 : 10;
        TW sv = sm.red[lane], cv = sm.red[kq];
#pragma unroll
        for (int q = 1; q < kNW; ++q) comp_merge(sv, cv, sm.red[q * 11 + lane], sm.red[q * 11 + kq]);
        v = sv + cv;
      } else if (lane < 9) {
#pragma unroll
        for (int q = 0; q < kNW; ++q) v += sm.red[q * 11 + lane];
      }
      TW tot[9];
#pragma unroll
      for (int k = 0; k < 9; ++k) tot[k] = __shfl_sync(0xffffffffu, v, k);
      if (lane == 0) {
      const TW R = kSplit ? sm.sc[6] + sm.sc[7] : tot[0], dJ = tot[5];
      const double u = sm.propb[4 * cur + 3];   // ln u for a drift move
      const bool ok = (R != TW(0)) && isfinite(R);
      TW A = TW(0);
      bool accept = false;
      double dr2 = 0.0;                          // |r' - r|^2 of a drift move
      if constexpr (kDrift) {
        // T(R'->R) / T(R->R') with displacement d = r' - r (minimum image) and the drift
        // displacements of both ends
        const double tau = S.step;
        double d[3], gn[3], db[3];
        for (int c = 0; c < 3; ++c) {
          d[c] = min_image<double>(sm.propb[4 * cur + c] - sm.posd[c * n_e + e], S.L);
          dr2 += d[c] * d[c];
          gn[c] = (double)(tot[1 + c] / R) + (double)tot[6 + c];
        }
        if (ok) {
          drift_disp(gn, tau, S.drift_a, db);
          double f2 = 0.0, b2 = 0.0;
          for (int c = 0; c < 3; ++c) {
            const double fw = d[c] - sm.outd[10 + c];
            const double bw = -d[c] - db[c];
            f2 += fw * fw;
            b2 += bw * bw;
          }
          // u < min(1, e^lr) decided as ln u < lr: the draws carry ln u, so a move takes no
          // exponential (A itself is formed for a trace only); ln|R| in working precision
          const double lr = 2.0 * log_abs_w(R) + 2.0 * (double)dJ + (f2 - b2) * inv_2tau;
          accept = u < lr;
          if (Wk.trace) A = (TW)fmin(1.0, exp(lr));
        }
      } else {
        A = ok ? fmin(TW(1), R * R * texp<TW>(TW(2) * dJ)) : TW(0);
        accept = u < (double)A;
      }
      if (kFixedNode && R < TW(0)) accept = false;
      if (Wk.forced) accept = Wk.forced[(size_t)w * n_e + e] != 0;
      if (kDrift) {
        r2p += dr2;
        if (accept) r2a += dr2;
      }
      if (Wk.trace) {
        double* tr = Wk.trace + ((size_t)w * n_e + e) * 8;
        tr[0] = (double)R;
        tr[1] = (double)dJ;
        tr[2] = (ok ? (double)(tot[1] / R) : 0.0) + (double)tot[6];
        tr[3] = (ok ? (double)(tot[2] / R) : 0.0) + (double)tot[7];
        tr[4] = (ok ? (double)(tot[3] / R) : 0.0) + (double)tot[8];
        tr[5] = kDrift ? move_u(S, sweep_index(Wk, t), (uint32_t)e, Wk.wid[w]) : u;
        tr[6] = (double)A;
        tr[7] = accept ? 1.0 : 0.0;
      }
      sm.flag[0] = accept;
      if (accept) {
        ++nacc;
        int ex;
        lprod = frexp(lprod * fabs((double)R), &ex);
        lexp += ex;
        if (R < TW(0)) sgn = -sgn;
        sm.posd[e] = sm.propb[4 * cur];
        sm.posd[n_e + e] = sm.propb[4 * cur + 1];
        sm.posd[2 * n_e + e] = sm.propb[4 * cur + 2];
        sm.posw[e] = sm.sc[0]; sm.posw[n_e + e] = sm.sc[1]; sm.posw[2 * n_e + e] = sm.sc[2];
        sm.wrow[m] = row;
        sm.sc[3] = R;
        if (kDrift) sm.sc[4] = tot[4];   // phi' . Binv0[e]: corner of the bordered C
      }
      }
    } else if (kDrift) {
      // While warp 0 decides, the other warps border C for an acceptance (wasted on a
      // rejection, but in time they would spend waiting): crow[l'] = phi' . U_l', then
      // y = C^-T crow and crow . z for the Schur complement (all compensated).
      for (int l = warp - 1; l < m; l += nw - 1) {
        TW s = TW(0), c = TW(0);
        for (int j = lane; j < ns; j += 32) comp_fma(s, c, phi[j], sm.wu[(size_t)l * ld_v + j]);
        warp_sum_comp(s, c);
        if (lane == 0) sm.crow[l] = s + c;
      }
      named_barrier(1, nt - 32);
      const int t1 = tid - 32;
      if (t1 < m) {
        TW y = TW(0), yc = TW(0);
        for (int l = 0; l < m; ++l) comp_fma(y, yc, sm.crow[l], sm.cinv[l * kcp + t1]);
        sm.yvec[t1] = y + yc;
      }
      if (warp == nw - 1) {
        TW sv = TW(0), sc2 = TW(0);
        for (int l = lane; l < m; l += 32) comp_fma(sv, sc2, -sm.crow[l], sm.zvec[l]);
        warp_sum_comp(sv, sc2);
        if (lane == 0) { sm.sc[6] = sv; sm.sc[7] = sc2; }
      }
    }
    __syncthreads();
    const bool accept = sm.flag[0] != 0;
    bool changed = false;     // Binv0 rewritten during this move (prefetched row is stale)
    if (accept) {
      TW* dst = VG + (size_t)e * 5 * ld_v;
      for (int i = tid; i < 5 * ld_v; i += nt) dst[i] = phi[i];
      for (int j = tid; j < ns; j += nt) {
        sm.wphi[(size_t)m * ld_v + j] = phi[j];
        sm.wu[(size_t)m * ld_v + j] = row0[j];
      }
      // Schur complement of the bordered C from its own entries, a - crow . C^-1 d, formed
      // by every thread from the values bordered before or during the decision
      TW a, ac2;
      if constexpr (kSplit) {
        a = sm.sc[6];
        ac2 = sm.sc[7];
      } else {
        a = sm.sc[4];
        ac2 = TW(0);
        comp_merge(a, ac2, sm.sc[6], sm.sc[7]);
      }
      // C^-1 of the bordered matrix
      const TW sinv = TW(1) / (a + ac2);
      for (int i = tid; i < (m + 1) * (m + 1); i += nt) {
        const int a = i / (m + 1), b = i % (m + 1);
        TW v;
        if (a < m && b < m)
          v = sm.cinv[a * kcp + b] + sm.zvec[a] * sm.yvec[b] * sinv;
        else if (a < m)
          v = -sm.zvec[a] * sinv;
        else if (b < m)
          v = -sm.yvec[b] * sinv;
        else
          v = sinv;
        sm.cinv[a * kcp + b] = v;
      }
      ++m;
      if (!ext_flush) {
        __syncthreads();       // the in-kernel flush and re-inversion read the new window
        if (m == kc) {
          flush_window<TW>(B, ns, m, kc, sm, ld_v);
          m = 0;
          changed = true;
        }
      }
    }
    if (reinv_period > 0) {
      if (accept || !reinv_on_acc) ++since;
      if (since >= reinv_period) {
        if (m > 0) {
          flush_window<TW>(B, ns, m, kc, sm, ld_v);
          m = 0;
        }
        cp_async_wait_all();   // the prefetch must land before the tiles reuse nothing it targets
        __syncthreads();
        bool full = true;
        if constexpr (sizeof(TW) == 4) {
          // FP64-accurate refinement; ln|det| keeps its FP64 accumulation of the ratios
          full = !(refine_inverse(S, Wk, w, spin, sm.tile, reinterpret_cast<float*>(sm.red)) <= kRefineMax);
        }
        if (full) {
          reinvert_block_plain<TW>(S, Wk, w, spin, sm.colk, sm.perm, sm.redv, sm.redi);
          if (tid == 0) {
            logdet = Wk.logdet[2 * w + spin];
            sgn = Wk.sgn[2 * w + spin];
            lprod = 1.0;
            lexp = 0;
          }
        }
        since = 0;
        changed = true;
      }
    }
    if (changed && e + 1 < e1) {
      // the inverse changed after the next row was prefetched: fetch it again
      prefetch_wait(e + 1 - e0);
      __syncthreads();
      const int nrow = e + 1 - first;
      TW* rd = sm.rowb + (size_t)(cur ^ 1) * ld_v;
      for (int j = tid; j < ns; j += nt) rd[j] = B[(size_t)nrow * ns + j];
      tc::fence_async_smem();   // ordered before the bulk copy that refills this buffer later
    }
  }
  cp_async_wait_all();
  __syncthreads();
  if (ext_flush) {
    // hand the window to the batched flush kernel
    TW* gphi = static_cast<TW*>(Wk.win_phi) + (size_t)w * kc * ld_v;
    TW* gu = static_cast<TW*>(Wk.win_u) + (size_t)w * kc * ld_v;
    TW* gc = static_cast<TW*>(Wk.win_cinv) + (size_t)w * kc * kc;
    for (int i = tid; i < m * ld_v; i += nt) {
      gphi[i] = sm.wphi[i];
      gu[i] = sm.wu[i];
    }
    for (int i = tid; i < kc * kc; i += nt) gc[i] = sm.cinv[(i / kc) * (kc + 1) + i % kc];
    for (int i = tid; i < m; i += nt) Wk.win_row[(size_t)w * kc + i] = sm.wrow[i];
    if (tid == 0) Wk.win_m[w] = m;
  } else if (m > 0) {
    flush_window<TW>(B, ns, m, kc, sm, ld_v);
  }
  __syncthreads();
  for (int i = tid; i < 3 * n_e; i += nt) gpos[i] = sm.posd[i];
  if (tid == 0) {
    Wk.logdet[2 * w + spin] = logdet + log(lprod) + (double)lexp * 0.69314718055994530942;
    Wk.sgn[2 * w + spin] = sgn;
    Wk.n_acc[w] += nacc;
    Wk.acc_since[2 * w + spin] = since;
    if (kDrift) {
      Wk.r2[2 * w] += r2p;
      Wk.r2[2 * w + 1] += r2a;
    }
  }
}

// =============================================================================
// Batched flush of the delayed-update windows (Sec. "Multi-Determinant Slater-Jastrow
// Form", delayed updates): for every walker, with the window's new orbital rows Phi_l,
// the inverse rows U_l = Binv0[e_l] and C^-1,
//   D[n][l] = Binv0[n] . Phi_l - delta(n, e_l),   Z[n] = C^-1 D[n],   Binv0[n] -= Z[n] U,
// i.e. two N_s x N_s x m products. Block (w, tile) owns kFlushRows rows of walker w's
// inverse. Register blocking: a thread owns one row of D (m outputs) in phase A and
// 8 threads share one row of the update in phase C.
// =============================================================================
constexpr int kFlushRows = 32;

template <class TW>
__host__ __device__ inline size_t flush_smem_bytes(int ld_v, int kc) {
  return sizeof(TW) * ((size_t)2 * kc * ld_v + (size_t)kFlushRows * (ld_v + 1) +
                       (size_t)kc * kc + (size_t)kFlushRows * (2 * kc + 1)) + sizeof(int) * kc + 16;
}

template <class TW>
__global__ void __launch_bounds__(256) k_flush(SysParams S, WalkParams Wk, int spin) {
  extern __shared__ __align__(16) char smem_f[];
  const int w = blockIdx.x;
  if (Wk.n_live && w >= *Wk.n_live) return;            // empty DMC slot
  const int m = Wk.win_m[w];
  if (m == 0) return;
  const int kc = Wk.kc, ld_v = Wk.ld_v, ldb = ld_v + 1;
  const int ns = spin ? S.n_dn : S.n_up;
  const int r0 = blockIdx.y * kFlushRows;
  if (r0 >= ns) return;
  const int nr = min(kFlushRows, ns - r0);
  TW* phi = reinterpret_cast<TW*>(smem_f);
  TW* U = phi + (size_t)kc * ld_v;
  TW* Bt = U + (size_t)kc * ld_v;
  TW* ci = Bt + (size_t)kFlushRows * ldb;
  TW* D = ci + kc * kc;
  TW* Z = D + kFlushRows * kc;                 // row stride kc + 1 (bank spread)
  int* wrow = reinterpret_cast<int*>(Z + kFlushRows * (kc + 1));
  const int tid = threadIdx.x, nt = blockDim.x;
  const TW* gphi = static_cast<const TW*>(Wk.win_phi) + (size_t)w * kc * ld_v;
  const TW* gu = static_cast<const TW*>(Wk.win_u) + (size_t)w * kc * ld_v;
  const TW* gc = static_cast<const TW*>(Wk.win_cinv) + (size_t)w * kc * kc;
  TW* B = binv_block<TW>(S, Wk, w, spin);
  for (int i = tid; i < m * ld_v; i += nt) { phi[i] = gphi[i]; U[i] = gu[i]; }
  for (int i = tid; i < kc * kc; i += nt) ci[i] = gc[i];
  for (int i = tid; i < m; i += nt) wrow[i] = Wk.win_row[(size_t)w * kc + i];
  for (int i = tid; i < nr * ns; i += nt) {
    const int r = i / ns, j = i % ns;
    Bt[r * ldb + j] = B[(size_t)(r0 + r) * ns + j];
  }
  __syncthreads();
  // phase A: D[r][l] = Bt[r] . Phi_l - delta
  {
    const int r = tid & 31, lg = tid >> 5, ng = nt >> 5;
    if (r < nr) {
      TW acc[8];
#pragma unroll
      for (int q = 0; q < 8; ++q) acc[q] = TW(0);
      const TW* br = Bt + r * ldb;
      for (int j = 0; j < ns; ++j) {
        const TW b = br[j];
#pragma unroll
        for (int q = 0; q < 8; ++q) {
          const int l = lg + q * ng;
          if (l < m) acc[q] += b * phi[(size_t)l * ld_v + j];
        }
      }
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        const int l = lg + q * ng;
        if (l < m) D[r * kc + l] = acc[q] - (wrow[l] == r0 + r ? TW(1) : TW(0));
      }
    }
  }
  __syncthreads();
  // phase B: Z[r] = C^-1 D[r]
  for (int i = tid; i < nr * m; i += nt) {
    const int r = i / m, l = i % m;
    TW z = TW(0);
    for (int lp = 0; lp < m; ++lp) z += ci[l * kc + lp] * D[r * kc + lp];
    Z[r * (kc + 1) + l] = z;
  }
  __syncthreads();
  // phase C: Binv0[r0 + r] -= Z[r] U
  {
    const int r = tid >> 3, c0 = tid & 7;
    if (r < nr) {
      const TW* zr = Z + r * (kc + 1);
      for (int j = c0; j < ns; j += 8) {
        TW v = Bt[r * ldb + j];
        for (int l = 0; l < m; ++l) v -= zr[l] * U[(size_t)l * ld_v + j];
        B[(size_t)(r0 + r) * ns + j] = v;
      }
    }
  }
}

// Empty every window after a flush round.
static __global__ void k_window_reset(WalkParams Wk) {
  const int w = blockIdx.x * blockDim.x + threadIdx.x;
  if (w < Wk.n_w) Wk.win_m[w] = 0;
}

// =============================================================================
// Batched single-precision re-inversion (the refinement of refine_inverse as separate
// kernels over all walkers): the error-free residual R = I - A X comes from the tensor
// cores (k_refine_residual_tc), then X <- X + X R into the second buffer of the spin block
// (k_refine_update_tc) and the FP64 fallback below.
// =============================================================================
// After the Newton update has written the refined inverses into the spin block's second
// buffer and the host has swapped the two buffers: walkers whose residual was too large
// (or not finite) are re-inverted in FP64 into the now current buffer, and the measured
// residual is recorded in refine_last.
template <class TW>
__global__ void __launch_bounds__(256) k_refine_fallback(SysParams S, WalkParams Wk, int spin) {
  extern __shared__ __align__(16) char smem_c[];
  const int w = blockIdx.x;
  if (Wk.n_live && w >= *Wk.n_live) return;          // empty DMC slot
  const float rm = Wk.refine_max[2 * w + spin];
  bool fp64 = !(rm <= kRefineSteps);
  if constexpr (sizeof(TW) == 4) {
    if (!fp64 && rm > kRefineMax) {
      // the batched step left about rm^2: up to two more steps here, each taken only if the
      // residual contracted (to at most a quarter of the last one), each leaving about the
      // square of the residual it started from; FP64 if that does not reach kRefineMax
      float* tile = reinterpret_cast<float*>(smem_c);
      float r = rm;
      for (int it = 0; it < 2 && r > kRefineMax; ++it) {
        const float rn = refine_inverse(S, Wk, w, spin, tile, tile + kTileElems, 0.25f * r);
        if (!(rn <= 0.25f * r)) { r = INFINITY; break; }   // no contraction: no step taken
        r = rn * rn;
      }
      fp64 = !(r <= kRefineMax);
    }
  }
  if (fp64) reinvert_block<TW>(S, Wk, w, spin, smem_c);
  if (threadIdx.x == 0) {
    Wk.refine_last[2 * w + spin] = rm;
    Wk.refine_max[2 * w + spin] = 0.f;
    Wk.refine_fb[2 * w + spin] = fp64 ? 1 : 0;
  }
}

// =============================================================================
// Local energy (Sec. "Hamiltonian", E_L = Psi^-1 H Psi) and ln|Psi| of every walker.
// Per electron i, with g_D = grad phi(r_i) . Binv[i] and l_D = lap phi(r_i) . Binv[i]:
//   T_i = -1/2 [ l_D - |g_D|^2 + lap_i J + |g_D + grad_i J|^2 ],
//   V = sum_{i<j} v(r_ij) - Z sum_{i,I} v(r_iI) + Z^2 sum_{I<J} v(R_IJ),
// v the Yukawa form, or with Ewald summation the real-space part erfc(alpha r) / r over the
// nearest image of every pair (the reciprocal-space part is a kernel of its own).
// One block per walker, one warp per electron; per-electron terms summed in FP64.
// =============================================================================
template <class TW>
__global__ void __launch_bounds__(kEnergyThreads) k_local_energy(SysParams S, WalkParams Wk) {
  extern __shared__ __align__(16) char smem_e[];
  __shared__ JastrowTab<TW> jt;
  jastrow_tab_fill<TW>(S, jt);
  TW* posw = reinterpret_cast<TW*>(smem_e);                  // [3][n_e]
  const int w = blockIdx.x;
  if (Wk.n_live && w >= *Wk.n_live) return;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int n_e = S.n_e, ld_v = Wk.ld_v;
  const double* P = Wk.pos + (size_t)w * 3 * n_e;
  for (int i = threadIdx.x; i < 3 * n_e; i += blockDim.x) posw[i] = (TW)P[i];
  __syncthreads();
  const TW Lw = Cst<TW>::L(S), iLw = Cst<TW>::invL(S), kap = Cst<TW>::kappa(S), Zw = Cst<TW>::Z(S);
  const TW alw = Cst<TW>::alpha(S);
  const bool ewald = S.ew_on != 0;
  const TW hL2 = TW(0.25) * Lw * Lw;
  const TW* ionw = Cst<TW>::ions(S);
  const TW* VG = static_cast<const TW*>(Wk.vgl) + (size_t)w * n_e * 5 * ld_v;

  double kin = 0.0, pot = 0.0, jas = 0.0;   // lane 0 of each warp
  for (int i = warp; i < n_e; i += nw) {
    const int spin = i >= S.n_up;
    const int ns = spin ? S.n_dn : S.n_up;
    const int row = i - (spin ? S.n_up : 0);
    const TW* Bi = binv_block<const TW>(S, Wk, w, spin) + (size_t)row * ns;
    const TW* v = VG + (size_t)i * 5 * ld_v;
    TW s[9];
    {
      TW g0 = 0, g1 = 0, g2 = 0, l0 = 0;
      for (int j = lane; j < ns; j += 32) {
        const TW b = Bi[j];
        g0 += v[ld_v + j] * b;
        g1 += v[2 * ld_v + j] * b;
        g2 += v[3 * ld_v + j] * b;
        l0 += v[4 * ld_v + j] * b;
      }
      s[0] = g0; s[1] = g1; s[2] = g2; s[3] = l0;
    }
    const TW ri[3] = {posw[i], posw[n_e + i], posw[2 * n_e + i]};
    double jsum;   // this electron's share of J, summed without loss (ln|Psi| needs J to
                   // about 1e-7 relative while its ~10^5 pair terms add up to ~10^4)
    {
      TW gx = 0, gy = 0, gz = 0, lj = 0, jj = 0, jc = 0, pv = 0;
      const int ntot = n_e + S.n_ion;
      for (int j = lane; j < ntot; j += 32) {
        if (j == i) continue;
        TW q[3];
        int f;
        if (j < n_e) {
          q[0] = posw[j]; q[1] = posw[n_e + j]; q[2] = posw[2 * n_e + j];
          f = ((j >= S.n_up) == (i >= S.n_up)) ? 1 : 2;
        } else {
          const int I = j - n_e;
          q[0] = ionw[I]; q[1] = ionw[S.n_ion + I]; q[2] = ionw[2 * S.n_ion + I];
          f = 0;
        }
        TW dd[3];
#pragma unroll
        for (int c = 0; c < 3; ++c) dd[c] = min_image<TW>(ri[c] - q[c], Lw, iLw);
        const TW r2 = dd[0] * dd[0] + dd[1] * dd[1] + dd[2] * dd[2];
        const bool once = (j >= n_e) || (j > i);
        // pairs beyond both cutoffs (Jastrow r_c, Yukawa L/2) contribute nothing; the Ewald
        // real-space part takes every pair
        const bool in_v = S.with_potential && once && (ewald || r2 < hL2);
        const bool in_j = jt.M[f] != 0 && r2 < jt.rc2[f];
        if (!(in_v || in_j) || !(r2 > TW(0))) continue;
        const TW rinv = rsqrt_w(r2), r0 = r2 * rinv;
        // one Newton correction: r2 * rsqrt(r2) in single precision carries a bias of a few
        // ulp that the J value (a sum of ~10^5 pair terms) would accumulate
        const TW r = fma(TW(0.5) * fma(-r0, r0, r2), rinv, r0);
        if (in_v) {
          // Yukawa e^{-kappa r} / r, or the Ewald real-space term erfc(alpha r) / r
          const TW y = (ewald ? erfc_w(alw * r) : exp_w(-kap * r)) * rinv;
          pv += (j < n_e) ? y : -Zw * y;
        }
        if (!in_j) continue;
        TW u, du, d2u;
        jastrow_eval<TW>(jt, f, r, u, du, d2u);
        if (once) {   // TwoSum: jj + jc carries the exact running sum of the 6 u terms
          TW u6, u6lo;
          jastrow_value6<TW>(jt, f, r, u6, u6lo);
          const TW t = jj + u6, z = t - jj;
          jc += ((jj - (t - z)) + (u6 - z)) + u6lo;
          jj = t;
        }
        const TW g = du * rinv;
        gx += g * dd[0]; gy += g * dd[1]; gz += g * dd[2];
        lj += d2u + TW(2) * g;
      }
      s[4] = gx; s[5] = gy; s[6] = gz; s[7] = lj; s[8] = pv;
      jsum = ((double)jj + (double)jc) / 6.0;
    }
    warp_sum<9, TW>(s);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) jsum += __shfl_xor_sync(0xffffffffu, jsum, o);
    if (lane == 0) {
      double j3[5] = {0.0, 0.0, 0.0, 0.0, 0.0};   // three-body Jastrow terms of electron i
      if (Wk.j3vgl) {
        const TW* q3 = static_cast<const TW*>(Wk.j3vgl) + ((size_t)w * n_e + i) * 5;
#pragma unroll
        for (int k = 0; k < 5; ++k) j3[k] = (double)q3[k];
      }
      const double g0 = s[0], g1 = s[1], g2 = s[2];
      const double lapD = (double)s[3] - (g0 * g0 + g1 * g1 + g2 * g2);
      const double gx = g0 + (double)s[4] + j3[0], gy = g1 + (double)s[5] + j3[1],
                   gz = g2 + (double)s[6] + j3[2];
      kin += -0.5 * (lapD + (double)s[7] + j3[3] + gx * gx + gy * gy + gz * gz);
      jsum += j3[4];
      pot += (double)s[8];
      jas += jsum;
    }
  }
  // sum the warp totals (lane 0 of each warp) in double
  double* part = reinterpret_cast<double*>(posw);   // reuse after the barrier
  __syncthreads();
  if (lane == 0) { part[3 * warp] = kin; part[3 * warp + 1] = pot; part[3 * warp + 2] = jas; }
  __syncthreads();
  if (threadIdx.x == 0) {
    double k = 0, p = 0, j = 0;
    for (int q = 0; q < nw; ++q) { k += part[3 * q]; p += part[3 * q + 1]; j += part[3 * q + 2]; }
    const double vii = !S.with_potential ? 0.0 : ewald ? *S.ew_const : S.v_ion_ion;
    Wk.e_loc[w] = k + p + vii;
    Wk.log_psi[w] = Wk.logdet[2 * w] + Wk.logdet[2 * w + 1] + j;
  }
}

inline size_t energy_smem_bytes(int n_e, size_t tw) {
  const size_t b = tw * 3 * (size_t)n_e;
  const size_t need = sizeof(double) * 3 * 32;   // warp partials, after the positions
  return b > need ? b : need;
}

// FP64 sums over walkers: (sum w, sum w E, sum w E^2, accepted) and reset of n_acc.
static __global__ void k_accumulate(WalkParams Wk, double* out, long long* nacc_total) {
  __shared__ double red[32 * 3];
  __shared__ long long redl[32];
  double a[3] = {0, 0, 0};
  long long acc = 0;
  for (int w = threadIdx.x; w < Wk.n_w; w += blockDim.x) {
    const double wt = Wk.weight[w], e = Wk.e_loc[w];
    a[0] += wt; a[1] += wt * e; a[2] += wt * e * e;
    acc += Wk.n_acc[w];
    Wk.n_acc[w] = 0;
  }
  warp_sum<3, double>(a);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) { red[3 * warp] = a[0]; red[3 * warp + 1] = a[1]; red[3 * warp + 2] = a[2]; redl[warp] = acc; }
  __syncthreads();
  if (threadIdx.x == 0) {
    double s[3] = {0, 0, 0};
    long long t = 0;
    for (int q = 0; q < (int)(blockDim.x >> 5); ++q) {
      s[0] += red[3 * q]; s[1] += red[3 * q + 1]; s[2] += red[3 * q + 2]; t += redl[q];
    }
    out[0] = s[0]; out[1] = s[1]; out[2] = s[2];
    *nacc_total = t;
  }
}

}  // namespace qmcgb
