// Internal structures shared by the C-ABI runtime and the kernel launchers.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <type_traits>

namespace qmcgb {

constexpr int kMaxKnots = 32;       // largest Jastrow M
constexpr int kMaxNlChannels = 4;   // non-local pseudopotential channels l = 0..3
constexpr int kEwMaxK = 65536;      // largest half set of Ewald k vectors
constexpr int kJ3MaxOrder = 4;      // largest polynomial order of the three-body Jastrow
constexpr int kJ3MaxCoef = (kJ3MaxOrder + 1) * (kJ3MaxOrder + 1) * (kJ3MaxOrder + 1);
constexpr int kJ3MaxNear = 8;       // ions within r_c / 2 of a move's two positions
constexpr size_t kMaxDynSmem = 227 * 1024;   // largest dynamic shared memory of one block (sm_103a)
constexpr int kMaxDelay = 64;       // largest delay rank k
constexpr int kThreads = 256;
constexpr int kEnergyThreads = 512;   // local energy: 16 warps per walker       // threads of the per-walker kernels

// One proposed move: new position and acceptance variate.
struct alignas(32) Prop {
  double x, y, z, u;
};

// Device error flags (bitwise OR into WalkParams::err).
enum : int { kErrSingular = 1, kErrNonFinite = 2, kErrTimeout = 4, kErrOverflow = 8, kErrJ3Near = 16 };

// Read-only description of a system, passed to kernels by value.
struct SysParams {
  int n_up, n_dn, n_e, n_ion;
  double L;
  // tricubic B-spline table [nx][ny][nz][ld] (table precision)
  const void* table;
  int nx, ny, nz, ld, n_orb;
  // Jastrow functors: 0 electron-ion, 1 same-spin pair, 2 opposite-spin pair
  int jM[3];
  double jrc[3];
  double jp[3][kMaxKnots + 1];
  float jpf[3][kMaxKnots + 1];   // single-precision copies for the mixed forms
  float jrcf[3];
  const double* ions;  // device [3][n_ion] (x block, y block, z block)
  const float* ionsf;  // the same in single precision
  double inv_delta[3]; // grid points per bohr along x, y, z (n / L)
  float inv_deltaf[3];
  float Lf, ion_Zf, kappaf;
  double invL;         // 1 / L
  float invLf;
  double ion_Z, kappa;
  int with_potential;
  double v_ion_ion;    // Z^2 sum_{I<J} v(R_IJ), a constant
  int move;            // 0 Metropolis, 1 drift
  double step;
  double drift_a;      // > 0: nodal drift rescaling parameter (0: the plain drift)
  // non-local pseudopotential: channels dv_l(r) = nl_amp[l] exp(-(r / nl_width[l])^2), r < nl_rcut
  int nl_nch;          // 0: none
  double nl_amp[kMaxNlChannels], nl_width[kMaxNlChannels], nl_rcut;
  // three-body e-e-I Jastrow (j3_on = 1): orders M_eI, M_ee, h = r_c / 2, coefficients
  // [2][M_eI + 1][M_eI + 1][M_ee + 1] (same-spin set, opposite-spin set)
  int j3_on, j3_meI, j3_mee;
  double j3_h;
  const double* j3_g;      // device
  // Coulomb interactions by Ewald summation in place of the Yukawa form (ew_on = 1)
  int ew_on;
  int ew_nk;               // k vectors in the half set
  double ew_alpha;         // splitting parameter (1/bohr)
  float ew_alphaf;
  const int4* ew_n;        // device [ew_nk] integer vectors n, k = 2 pi n / L (w unused)
  const double* ew_ck;     // device [ew_nk] (4 pi / Omega) exp(-k^2 / (4 alpha^2)) / k^2
  const double* ew_rho_ion;// device [2][ew_nk] Z sum_I cos(k.R_I), Z sum_I sin(k.R_I)
  const double* ew_const;  // device [1] ion-ion real-space, self and background terms
  uint32_t seed_lo, seed_hi;
};

// Mutable walker arrays, passed to kernels by value (pointers to device memory).
struct WalkParams {
  int n_w;
  int ld_v;            // row length of per-electron orbital vectors (>= max N_s, multiple of 8)
  double* pos;         // [W][3][n_e]
  void* binv[2];       // per spin block, working precision [W][N_s][N_s]; Binv[e][j] = (A^-1)[j][e]
  void* binv_alt[2];   // second buffer of each spin block: the single-precision re-inversion
                       // writes the refined inverse there and the two buffers swap roles
  void* vgl;           // working precision [W][n_e][5][ld_v]: value, gx, gy, gz, lap at r_e
  double* logdet;      // [W][2]
  double* sgn;         // [W][2]
  uint32_t* wid;       // [W]
  double* weight;      // [W]
  double* e_loc;       // [W]
  double* log_psi;     // [W]
  long long* n_acc;    // [W] accepted moves since the last accumulate
  int* acc_since;      // [W][2] accepted (or proposed) moves since the last re-inversion
  double* trace;       // optional [W][n_e][8] for the current sweep
  const uint8_t* forced;  // optional [W][n_e] decisions
  double* scratch64;   // [W][2][ld_v][ld_v] FP64 work matrices for re-inversion
  int* err;            // device error flags
  // delayed-update window handed from the sweep kernel to the batched flush kernel
  int kc;              // window capacity (delay rank k)
  void* win_phi;       // [W][kc][ld_v] new orbital rows of the accepted moves
  void* win_u;         // [W][kc][ld_v] Binv0 rows of the moved electrons
  void* win_cinv;      // [W][kc][kc]   C^-1
  int* win_row;        // [W][kc]       row (electron index within the spin block)
  int* win_m;          // [W]           fill
  float* refine_max;   // [W][2]        max |I - A X| of the refinement in progress of each
                       //               spin block (the two blocks' refinements may overlap)
  float* refine_last;  // [W][2]        max |I - A X| measured by the last refinement of each
                       //               spin block (before its Newton step); NaN if none yet
  int* refine_fb;      // [W][2]        1 if the last refinement re-inverted in FP64
  float* logdet_shift; // [W][2]        change of ln|det A| made by the last log-det anchor
                       //               (anchor value minus the accumulated one); NaN if none
  int* rscale;         // [W][2][2][ld_v] power-of-two exponents of the rows of A and X
  const int* n_live;   // optional device count: blocks of walkers >= *n_live return at once
  double* r2;          // [W][2] sums of the squared proposed and accepted displacements of
                       //        drift moves since the last reset (effective time step)
  double* vnl;         // [W]    non-local pseudopotential energy of the last measurement
  int* nl_pairs;       // [W][nl_cap] electron * n_ion + ion of the pairs inside the cutoff
  int* nl_count;       // [W]
  double* nl_val;      // [W][nl_cap] V_NL of each listed pair
  int nl_cap;
  void* j3vgl;         // working precision [W][n_e][5]: grad_i J3, lap_i J3 and electron i's
                       // share of J3 for the next local energy; nullptr without that term
  const uint32_t* t_base;  // optional device sweep index added to the kernels' sweep argument
                           // (a replayed graph passes offsets and reads the index here)
};

// Sweep index of the Philox counters: the launch argument, plus the device word when the
// launch belongs to a replayed graph.
__device__ __forceinline__ uint32_t sweep_index(const WalkParams& W, uint32_t t) {
  return W.t_base ? t + *W.t_base : t;
}

// Inverse of walker w's spin block: Binv[e][j] = (A^-1)[j][e], N_s x N_s, row-major.
template <class T>
__host__ __device__ inline T* binv_block(const SysParams& S, const WalkParams& W, int w, int spin) {
  const size_t ns = spin ? S.n_dn : S.n_up;
  using V = typename std::remove_const<T>::type;
  return static_cast<V*>(W.binv[spin]) + (size_t)w * ns * ns;
}

// Device state of the branching DMC of one system.
struct DmcParams {
  double* e_old;        // [cap] E_L before this step's sweep (per slot of the current buffer)
  double* e_old_next;   // [cap] the same for the other buffer
  int* src_of;          // [cap] parent slot of each destination slot
  uint32_t* wid_next;   // [cap] walker ID of each destination slot
  int* n_live;          // [2] population of buffer 0 and 1
  uint32_t* next_id;    // [1] next free walker ID
  double* e_trial;      // [1] E_T
  double* stats;        // [8] sum W, sum W E, weighted mean E, E_T used, population before, after
  int n_target, cap;
  double tau;
  int tau_eff;          // 1: branching factor with tau_eff = tau * accepted / proposed |dr|^2
  int reconfigure;      // 1: stochastic reconfiguration at a fixed walker count
};

}  // namespace qmcgb
