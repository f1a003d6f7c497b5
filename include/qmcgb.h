/*
 * qmcgb.h - C ABI of the GB300 particle-by-particle QMC library (libqmcgb.so).
 *
 * What the library computes (citations are to the QMCPACK paper, arXiv 1802.06922):
 *   Many independent walkers (Markov chains, Sec. "Variational Monte Carlo") move their
 *   electrons one at a time (Sec. "Trial Moves", particle-by-particle transition density)
 *   through a trial wavefunction Psi = D_up D_dn e^J (Eq. msdj with one determinant):
 *     - orbitals phi_j are periodic tricubic B-splines; one evaluation of value, gradient
 *       and Laplacian gathers the 64 coefficient rows around the point
 *       (Sec. "B-spline basis sets");
 *     - the determinant ratio of a move of electron e is phi(r') . column e of A^-1, and an
 *       accepted move updates A^-1 by Sherman-Morrison or by the delayed rank-k scheme
 *       (Sec. "Multi-Determinant Slater-Jastrow Form");
 *     - J holds one- and two-body terms built from 1D cubic B-spline radial functors
 *       with minimum-image distances, and optionally the three-body e-e-I polynomial
 *       term (Sec. "Jastrow factor");
 *     - a move is accepted with min(1, |Psi'/Psi|^2 T'/T) (Eq. accept_reject); DMC steps
 *       use drift-diffusion proposals (Eq. pmc:driftdiffusion_step), the fixed-node
 *       rule, weights (Eq. pmc:walker_weight) and branching (Sec. "Diffusion Monte Carlo");
 *     - the local energy E_L = Psi^-1 H Psi (Sec. "Hamiltonian") is kinetic plus a
 *       short-range Yukawa potential standing in for the Coulomb terms, or the Coulomb
 *       terms themselves by Ewald summation, plus optionally the non-local
 *       pseudopotential's quadrature of virtual moves.
 *
 * Conventions for every call:
 *   - Units are Hartree atomic units; the cell is the cube [0, L)^3, periodic.
 *   - Electrons 0..n_up-1 are spin up, n_up..n_up+n_dn-1 spin down.
 *   - Every function returns a qmc_status; nothing throws across the ABI. On failure the
 *     message of the calling thread is available from qmc_last_error().
 *   - Host arrays passed in are copied before the call returns; the caller keeps them.
 *   - Device buffers created by the library are owned by it and released by the
 *     matching destroy call. Device pointers passed in by the caller (trace buffers,
 *     outputs) are borrowed: the library never frees them, and they must stay valid
 *     until the work queued on the given stream has finished.
 *   - Calls that take a `stream` (a cudaStream_t, NULL = the legacy default stream)
 *     only enqueue work and return; device-side failures (a singular matrix, a bounded
 *     wait that timed out) are recorded in a device flag and reported by the next
 *     synchronising call (qmc_measure, qmc_accumulate_energy, qmc_get_state,
 *     qmc_check_errors).
 *   - Output pointers of qmc_measure and qmc_accumulate_energy may be host or device
 *     memory; the library looks at the pointer and copies accordingly.
 *   - destroy functions accept NULL.
 */
#ifndef QMCGB_H
#define QMCGB_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct qmc_system_s* qmc_system_t;
typedef struct qmc_walkers_s* qmc_walkers_t;
typedef struct qmc_dmc_s* qmc_dmc_t;

typedef enum {
  QMC_OK = 0,
  QMC_EINVAL = -1,     /* a bad argument: NULL handle, size out of range, wrong order of calls */
  QMC_ENOMEM = -2,     /* a device or host allocation failed */
  QMC_ECUDA = -3,      /* a CUDA runtime call failed */
  QMC_ESINGULAR = -4,  /* a Slater matrix had an exactly zero pivot at (re-)inversion */
  QMC_ETIMEOUT = -5,   /* a bounded device-side wait ran out */
  QMC_ESTATE = -6      /* a serialized state does not match the walker set */
} qmc_status;

typedef enum {
  QMC_FP64 = 0,          /* table, orbital values, inverse and ratios in double */
  QMC_FP32 = 1,          /* FP32 table, orbital values, inverse and ratios; re-inversion by a
                            Newton step with an error-free residual (see reinv_period);
                            FP64 ln|det| accumulation, energy sums and reductions */
  QMC_FP32_BF16TAB = 2   /* BF16 coefficient table, FP32 accumulation, else as QMC_FP32 */
} qmc_precision;

typedef enum {
  QMC_MOVE_METROPOLIS = 0,  /* r' = r + step * xi (Gaussian xi) */
  QMC_MOVE_DRIFT = 1        /* r' = r + step * grad ln|Psi| + sqrt(step) * xi */
} qmc_move;

/* Description of one system (Sec. "Hamiltonian", Sec. "Trial Moves"). */
typedef struct {
  int n_up, n_dn;          /* electrons per spin; each determinant is N_s x N_s */
  double L;                /* side of the periodic cubic cell (bohr) */
  int n_ion;               /* number of ions (may be 0) */
  const double* ion_pos;   /* host [n_ion][3], copied */
  double ion_Z;            /* ion charge in the potential */
  double kappa;            /* Yukawa screening (1/bohr); v(r) = exp(-kappa r)/r, r < L/2 */
  int with_potential;      /* 0: E_L is the kinetic energy only */
  qmc_precision prec;
  qmc_move move;
  double step;             /* sigma (Metropolis) or tau (drift), bohr or 1/Ha */
  int delay_k;             /* 1 = Sherman-Morrison rank-1; 2..64 = delayed rank-k */
  int reinv_period;        /* re-invert each Slater matrix every this many moves (0 = never):
                              QMC_FP64 by FP64 Gauss-Jordan; the single-precision forms by one
                              Newton step X <- X + X R whose residual R = I - A X is computed
                              error-free on the tensor cores; a walker whose |R| is above 1e-2
                              gets up to two more, compensated Newton steps while its residual
                              contracts, and above 0.2 (or without contraction) FP64
                              Gauss-Jordan, as do spin blocks above 512 electrons (the in-sweep
                              variant used with reinv_on_accepted sums R with compensated
                              arithmetic) */
  int reinv_on_accepted;   /* 1: count accepted moves of the determinant; 0: proposed moves */
  uint64_t seed;           /* Philox4x32-10 key of every draw */
  int logdet_period;       /* single-precision forms with batched re-inversion (delay_k >= 4,
                              reinv_on_accepted = 0): every this many moves of a spin block,
                              right after its re-inversion, ln|det A| is recomputed to FP64-class
                              accuracy by an LU factorisation in FP32 whose rounding errors are
                              captured exactly and folded back through the refined inverse;
                              between anchors ln|det| is the FP64 sum of the moves' ln|R|.
                              A positive multiple of reinv_period, or 0 = never. Ignored by
                              QMC_FP64, whose accumulated ln|det| needs no anchor. */
  double drift_a;          /* QMC_MOVE_DRIFT: > 0 rescales the drift near nodes of Psi
                              (Umrigar, Nightingale and Runge; Sec. "Projector Monte Carlo"):
                              the drift displacement tau v becomes
                              tau v 2 / (1 + sqrt(1 + 2 a |v|^2 tau)), below sqrt(2 tau / a)
                              for any v, in the proposal and in the Green's-function ratio of
                              the acceptance; 0 = the plain drift. */
  int prop_chunk;          /* Metropolis moves whose proposals and orbital rows are formed by
                              one launch pair, per spin block (0 = the whole block); smaller
                              batches keep the rows in L2 until the sweep reads them. A
                              launch parameter only: the chain does not depend on it. */
} qmc_system_desc;

/* Creates a system. Fails with QMC_EINVAL for n_up or n_dn outside [0, 1024], n_up+n_dn
 * = 0, L <= 0, step < 0, delay_k outside [1, 64], an unknown precision/move, a
 * logdet_period that is negative or not a multiple of a positive reinv_period, or a negative
 * prop_chunk. */
qmc_status qmc_system_create(const qmc_system_desc* desc, qmc_system_t* out);

/* Sets the B-spline orbital table (Sec. "B-spline basis sets"). coef is host memory
 * [nx][ny][nz][n_orb] in double, row (ix,iy,iz) holding the n_orb orbital coefficients of
 * node (ix,iy,iz) at position (ix*L/nx, iy*L/ny, iz*L/nz). It is copied to the device and
 * cast to the system's table precision. Requires n_orb >= max(n_up, n_dn) and each of
 * nx, ny, nz >= 4. Both spins use orbitals 0..N_s-1. */
qmc_status qmc_system_set_spline(qmc_system_t sys, int nx, int ny, int nz, int n_orb,
                                 const double* coef);

/* Sets one radial Jastrow functor u(r) = sum_{m=0}^{M} p_m B3(r M / rcut - m), u = 0 for
 * r >= rcut (Sec. "Jastrow factor"). which: 0 = electron-ion, 1 = same-spin pair,
 * 2 = opposite-spin pair. p: host [M+1]. If cusp_set, p[0] is replaced by
 * p[2] - (2 rcut / M) cusp so that u'(0) = cusp. 1 <= M <= 32, 0 < rcut <= L/2.
 * A functor that is never set is zero. */
qmc_status qmc_system_set_jastrow(qmc_system_t sys, int which, int M, double rcut,
                                  const double* p, int cusp_set, double cusp);

/* Semi-local (non-local) pseudopotential channels of every ion (Sec. "Hamiltonian": the
 * electron-ion term gains sum_lm |Y_lm> [v_l(r) - v_loc(r)] <Y_lm| within a cutoff, evaluated
 * following Mitas et al. with a 12-point angular integration). Channels l = 0 .. n_channels-1
 * with v_l - v_loc = amp[l] exp(-(r / width[l])^2) for r < rcut (host arrays, copied; a smooth
 * synthetic form, as no tabulated pseudopotential is used). Every measurement then adds, for
 * each electron within rcut of an ion (nearest image), the 12-point quadrature
 *   sum_l (2l+1) dv_l(r) (1/12) sum_q P_l(u . O n_q) Psi(r_i -> R_I + r O n_q) / Psi
 * to E_L: n_q the vertices of an icosahedron (exact to degree 5), O a uniform random rotation
 * from Philox block (t, 0xD, walker ID, 3) with t the walker set's count of completed sweeps,
 * and each ratio a virtual move (determinant ratio times exp(dJ)) with no update. At most
 * 2 N_e pairs per walker (else the next synchronising call fails with QMC_ECUDA).
 * n_channels = 0 removes the channels. QMC_EINVAL for n_channels outside [0, 4], a width
 * <= 0 or rcut outside (0, L/2]. Takes effect at the next measurement. */
qmc_status qmc_system_set_nonlocal(qmc_system_t sys, int n_channels, const double* amp,
                                   const double* width, double rcut);

/* Three-body electron-electron-ion Jastrow factor added to J (Sec. "Jastrow factor": the
 * correlation function of Drummond et al.). For electrons i < j and every ion I, with
 * a = r_iI, b = r_jI, c = r_ij (minimum image) and h = rcut / 2:
 *   u(a, b, c) = sum_{l,m=0}^{m_ei} sum_{n=0}^{m_ee} gamma_lmn a^l b^m c^n (a - h)^3 (b - h)^3
 * when a < h and b < h, else 0; J3 = sum_I sum_{i<j} u. gamma_same applies to same-spin
 * pairs, gamma_opp to opposite-spin pairs; each is host [m_ei+1][m_ei+1][m_ee+1] (index
 * (l (m_ei+1) + m) (m_ee+1) + n), copied, and must satisfy gamma_lmn = gamma_mln. Moves
 * (Metropolis, drift, the windowed delayed update), E_L, ln|Psi| and the pseudopotential's
 * virtual moves all include the term. At most 8 ions may lie within h of the two positions
 * of one move of the windowed delayed update (else the next synchronising call fails with
 * QMC_ECUDA). m_ei < 0 removes the term. Synchronous; no other call may use the system
 * meanwhile. QMC_EINVAL for orders above 4, rcut outside (0, L/2], a coefficient that is
 * not finite or a set that is not symmetric in l and m. */
qmc_status qmc_system_set_jastrow3(qmc_system_t sys, int m_ei, int m_ee, double rcut,
                                   const double* gamma_same, const double* gamma_opp);

/* Coulomb interactions by Ewald summation in place of the Yukawa form (Sec. "Hamiltonian":
 * v_ee = 1/r, v_eI = -Z/r and v_II = Z^2/r summed over every periodic image of the cell,
 * evaluated with the Ewald technique; Sec. "Long-Range Interactions": short-ranged terms
 * summed in real space, long-ranged ones in reciprocal space). With splitting parameter
 * alpha (1/bohr) and reciprocal cutoff kcut, electrons of charge -1, ions of charge +Z,
 * Q = N_ion Z - N_e and Omega = L^3, every measurement's potential becomes
 *   V = sum_{a<b} q_a q_b erfc(alpha r_ab) / r_ab          (nearest image of every pair)
 *     + (4 pi / Omega) sum_{k in H} exp(-k^2 / (4 alpha^2)) / k^2 |rho_k|^2
 *     - alpha / sqrt(pi) (N_e + N_ion Z^2) - pi Q^2 / (2 Omega alpha^2),
 * rho_k = Z sum_I e^{i k.R_I} - sum_i e^{i k.r_i}, H the vectors k = 2 pi n / L (n integer)
 * with 0 < |k| <= kcut, one of each +-k pair. The nearest-image real-space sum equals the
 * periodic one only when erfc(alpha L / 2) is negligible (alpha L / 2 >= 4: below 2e-8).
 * rho_k of every walker is evaluated from its positions at each measurement, O(N_e |H|).
 * alpha = 0 restores the Yukawa form. Synchronous (builds the ions' rho_k and the constant
 * terms on the device); no other call may use the system meanwhile. QMC_EINVAL for a system
 * without a potential, alpha < 0 or not finite, kcut not finite or <= 0 with alpha > 0,
 * kcut L / (2 pi) > 64, or more than 65536 vectors in H. */
qmc_status qmc_system_set_ewald(qmc_system_t sys, double alpha, double kcut);

/* Number of k vectors in the Ewald half set H of the system, or -1 when the Yukawa form is
 * in use. */
int qmc_system_ewald_count(qmc_system_t sys);

/* Creates n_walkers walkers (the ensemble of independent Markov chains of Sec.
 * "Variational Monte Carlo", each a configuration R of all electrons) with IDs
 * 0..n_walkers-1 at positions pos (host or device [n_walkers][n_up+n_dn][3], wrapped into
 * the cell). Evaluates the orbitals at every electron, inverts each Slater matrix in FP64
 * (A[e][j] = phi_j(r_e), Sec. "Multi-Determinant Slater-Jastrow Form") and records ln|det|
 * and its sign. Synchronous. QMC_ESINGULAR if a Slater matrix is singular. */
qmc_status qmc_walkers_create(qmc_system_t sys, int n_walkers, const double* pos,
                              qmc_walkers_t* out);

/* Advances every walker by n_sweeps sweeps of particle-by-particle moves (Sec. "Trial
 * Moves": one electron at a time, a Gaussian or drift-diffusion proposal accepted with
 * Eq. accept_reject); a sweep proposes one move for each electron in index order, then
 * measures the local energy. Uses (and then advances) the walker set's sweep counter,
 * which is part of every Philox counter, so the result depends only on the seed, the walker
 * IDs, the positions and the counter. Asynchronous on `stream`. */
qmc_status qmc_sweep(qmc_walkers_t w, int n_sweeps, void* stream);

/* Local energy and ln|Psi| of every walker's current configuration
 * (E_L = Psi^-1 H Psi, Sec. "Hamiltonian"). e_local and log_psi: [n_walkers] doubles,
 * host or device (either may be NULL). The values measured at the end of the last sweep are
 * returned unless a qmc_system_set_jastrow, qmc_system_set_jastrow3, qmc_system_set_nonlocal
 * or qmc_system_set_ewald call changed the system since, in which case the walkers are
 * measured again. Synchronises
 * `stream` when an output is host memory; reports deferred device errors. */
qmc_status qmc_measure(qmc_walkers_t w, double* e_local, double* log_psi, void* stream);

/* FP64 sums over walkers of the last measurement (Sec. "Variational Monte Carlo" and
 * Eq. pmc:weighted_average): out[0] = sum W, out[1] = sum W E_L, out[2] = sum W E_L^2,
 * out[3] = accepted / proposed moves since the previous call. W = 1 in VMC. out: host or
 * device [4]. Measures first if the walkers moved since the last measurement. */
qmc_status qmc_accumulate_energy(qmc_walkers_t w, double* out, void* stream);

/* Enables a per-move trace of the next sweeps: dev_buf (device, borrowed) receives, for
 * each traced sweep, [n_walkers][n_up+n_dn][8] doubles = (ratio R_det, dJ,
 * grad_e ln|Psi(R')| x,y,z, u, A, accepted). bytes bounds how many sweeps are traced;
 * NULL / 0 disables. */
qmc_status qmc_trace_enable(qmc_walkers_t w, void* dev_buf, size_t bytes);

/* Lockstep replay: the next qmc_sweep call of n sweeps takes its accept decisions from
 * accept_bits (host or device, [n][n_walkers][n_up+n_dn] bytes, 0 or 1) instead of
 * u < A. Used to compare reduced-precision runs move by move with a reference run.
 * The array is copied; NULL clears a pending replay. */
qmc_status qmc_replay_decisions(qmc_walkers_t w, const uint8_t* accept_bits, int n_sweeps);

/* Positions [n_walkers][n_e][3] of every walker, copied to host or device memory. */
qmc_status qmc_get_positions(qmc_walkers_t w, double* pos, void* stream);

/* Serialised walker state (positions, walker IDs, weights, sweep counter, seed) for
 * checkpoint/resume: a walker of Sec. "Diffusion Monte Carlo" is its configuration and
 * weight, and the Philox counters make the continuation reproducible. qmc_get_state with
 * buf = NULL stores the needed size in *len.
 * qmc_set_state rebuilds the inverses by FP64 re-inversion; QMC_ESTATE if the buffer does
 * not match this walker set's sizes. Synchronous. */
qmc_status qmc_get_state(qmc_walkers_t w, void* buf, size_t* len);
qmc_status qmc_set_state(qmc_walkers_t w, const void* buf, size_t len);

/* Inspection of one walker's state (synchronous; host or device output):
 *   qmc_get_inverse:  Binv[e][j] = (A^-1)[j][e] of spin block `spin` (0 up, 1 down) as
 *                     doubles [N_s][N_s] (row e is the column of A^-1 that a move of the
 *                     block's e-th electron dots with phi(r'));
 *   qmc_get_orbitals: value, gradient x, y, z and Laplacian of orbitals 0..N_s-1 at every
 *                     electron's current position, doubles [n_e][5][max(n_up, n_dn)].
 * QMC_EINVAL for a walker index outside [0, n_walkers) or spin outside {0, 1}. */
qmc_status qmc_get_inverse(qmc_walkers_t w, int walker, int spin, double* out);
qmc_status qmc_get_orbitals(qmc_walkers_t w, int walker, double* out);

/* The non-local pseudopotential part of the last measurement's E_L, [n_walkers] doubles
 * (host or device); zeros without channels. Synchronous. */
qmc_status qmc_get_nonlocal(qmc_walkers_t w, double* out);

/* ln|det A| and the sign of det A of every walker's two Slater matrices (Sec.
 * "Multi-Determinant Slater-Jastrow Form"), as the walker set carries them: logdet and sign
 * are [n_walkers][2] doubles (spin up, spin down), host or device, either may be NULL (not
 * both). In the single-precision forms ln|det A| is the FP64 running sum of the ln|R| of
 * the accepted moves since the last FP64 value (walker creation, an FP64 re-inversion or a
 * log-determinant anchor). Synchronous; reports deferred device errors. */
qmc_status qmc_get_logdet(qmc_walkers_t w, double* logdet, double* sign);

/* Numerical health of the single-precision forms, per walker and spin block ([n_walkers][2]
 * doubles each, host or device, either may be NULL):
 *   residual      max |I - A X| measured by the block's last batched re-inversion before
 *                 its Newton step (X the inverse it corrected); above 1e-2 means further
 *                 Newton steps followed, above 0.2 (or infinite) an FP64 Gauss-Jordan;
 *   logdet_shift  the change the last log-determinant anchor made to ln|det A| (anchored
 *                 value minus the accumulated one): the drift of the accumulated sum since
 *                 the previous FP64-class value.
 * NaN where nothing has run yet. Synchronous. */
qmc_status qmc_get_precision_report(qmc_walkers_t w, double* residual, double* logdet_shift);

/* Waits for the walkers' queued work on `stream` and reports deferred device errors. */
qmc_status qmc_check_errors(qmc_walkers_t w, void* stream);

/* Standalone FP64 re-inversion of a batch of Slater matrices (the periodic re-inversion
 * of the sweep, exposed on its own; the determinant-ratio convention of Sec.
 * "Multi-Determinant Slater-Jastrow Form").
 *   prec   QMC_FP64: A and Binv are doubles; QMC_FP32 or QMC_FP32_BF16TAB: floats.
 *   A      device [batch][n][n], A[b][e][j] = phi_j(r_e) (row e = orbitals of electron e).
 *   Binv   device [batch][n][n], Binv[b][e][j] = (A^-1)[j][e].
 *   logdet, sign  device [batch] doubles or NULL: ln|det A| and its sign; an exactly
 *          singular matrix gets -inf, sign 0 and Binv = 0.
 * Gauss-Jordan elimination with partial pivoting in FP64 on a work copy; the FP64 work
 * matrices (batch * n * n doubles) are allocated on `stream` (stream-ordered) and released
 * after the kernel. Asynchronous. QMC_EINVAL for n outside [1, 1024], batch outside
 * [1, 2^20] or a host pointer; QMC_ENOMEM if the work area cannot be allocated. */
qmc_status qmc_slater_invert(qmc_precision prec, const void* A, void* Binv, double* logdet,
                             double* sign, int n, int batch, void* stream);

/* The same computation as qmc_slater_invert, for callers that must not allocate device
 * memory: applications whose device memory is owned by their own pool allocator (a
 * cudaMalloc from inside this library could fail, or fragment a pool that has reserved
 * nearly all of HBM), and latency-sensitive loops that cannot accept the device-wide
 * synchronisation and unpredictable latency an allocation or free may bring. The paper
 * has no counterpart; this is a property of the library, not of the method.
 *   Arguments, layouts and results are exactly those of qmc_slater_invert.
 *   Work area: a fixed FP64 array compiled into libqmcgb, 2^21 doubles (16 MiB); every GPU
 *   on which the library is used holds it until the process exits. batch * n * n must not
 *   exceed 2^21 (for example 32 matrices of 256 x 256, or 8 of 512 x 512); a larger request
 *   fails with QMC_EINVAL before anything is enqueued. No cudaMalloc, cudaFree or other
 *   allocating routine is called.
 *   Each call whose stream is not being captured looks up the work area's device address
 *   on the current device (so a context re-created by cudaDeviceReset is served too); a
 *   call under stream capture reuses the address of the last uncaptured call on the device,
 *   and fails with QMC_EINVAL if there was none: make the first call before any capture.
 *   Every call uses the same work area, which keeps the last call's contents. A call
 *   overwrites each work element before reading it, so nothing needs clearing, but calls
 *   whose kernels overlap on the GPU (different streams or host threads) race on the work
 *   area and corrupt each other's results: serialise them. Asynchronous on `stream`. */
qmc_status qmc_slater_invert_noalloc(qmc_precision prec, const void* A, void* Binv,
                                     double* logdet, double* sign, int n, int batch,
                                     void* stream);

/* Branching DMC over one or more systems (Sec. "Diffusion Monte Carlo"), each advancing
 * on its own stream so that systems of uneven size share the GPU. Every system must use
 * QMC_MOVE_DRIFT (tau = step). One step of a system: a sweep of drift-diffusion moves with
 * the fixed-node rule (a move that changes the sign of Psi is rejected), the local energy,
 * the weights w = exp(-tau/2 (E_L(old) + E_L(new) - 2 E_T)) (Eq. pmc:g_growth and
 * Eq. pmc:walker_weight), M = floor(w + xi) copies of each walker (xi from Philox block
 * (step, 0xB, walker ID, 2)), children renormalised to weight 1 and appended in parent
 * order (the first copy keeps the parent's ID, further copies take new consecutive IDs),
 * the population capped at capacity_factor times the initial count, and the trial energy
 * fed back as E_T <- E_w - ln(N / N_0) / (10 tau) with E_w the weighted mean E_L.
 *   qmc_dmc_create: n_walkers[i] initial walkers of systems[i] at host positions[i]
 *                   ([n][n_e][3]), initial trial energies e_trial[i]; walker IDs 0..n-1.
 *                   The driver owns its walker storage; the systems must outlive it.
 *   qmc_dmc_step:   n_steps steps of every system, ordered after prior work on `stream`
 *                   and before later work on it. Asynchronous; populations stay on the GPU.
 *   qmc_dmc_read:   out[8] = population, sum of weights, sum of weight * E_L, weighted mean
 *                   E_L, E_T used, E_T for the next step, next free walker ID, population
 *                   before the last branching (host or device). Synchronous.
 *   qmc_dmc_walkers: positions [n][n_e][3], IDs [n] and E_L [n] of the current population
 *                   (any may be NULL); *n_out = population; QMC_EINVAL if n > max_walkers. */
qmc_status qmc_dmc_create(qmc_system_t const* systems, const int* n_walkers,
                          const double* const* positions, const double* e_trial, int n_systems,
                          int capacity_factor, qmc_dmc_t* out);
qmc_status qmc_dmc_step(qmc_dmc_t d, int n_steps, void* stream);
/* Refinements of the DMC step (Sec. "Diffusion Monte Carlo"), both off after create:
 *   effective_tau  1: a walker's branching factor uses tau_eff = tau * (sum of |r' - r|^2 of
 *                  its accepted moves) / (sum over all its proposed moves) of the step's
 *                  sweep instead of tau (Umrigar, Nightingale and Runge);
 *   reconfigure    1: population control by stochastic reconfiguration at a fixed walker
 *                  count (Assaraf, Caffarel and Khelif) instead of M = floor(w + xi)
 *                  branching: one comb of N teeth at (k + xi) W / N, k = 0..N-1, over the
 *                  cumulative weights in walker order (W the total weight, xi from Philox
 *                  block (step, 0xC, 0, 2) word 0); walker i gets the teeth falling in its
 *                  interval, the last walker the remainder, so the count stays N; copies are
 *                  placed and numbered as in branching and carry weight one. With N at its
 *                  target the E_T feedback reduces to E_T = E_w.
 * Applies to every system of d from the next step on. QMC_EINVAL for a NULL driver. */
qmc_status qmc_dmc_set_mode(qmc_dmc_t d, int effective_tau, int reconfigure);
qmc_status qmc_dmc_read(qmc_dmc_t d, int system, double* out);
qmc_status qmc_dmc_walkers(qmc_dmc_t d, int system, int max_walkers, double* pos, uint32_t* ids,
                           double* e_local, int* n_out);
int64_t qmc_dmc_launch_count(qmc_dmc_t d);
/* Per-kernel device time of the driver's steps, as qmc_profile_enable / qmc_profile_read of a
 * walker set (kernel classes of qmc_kernel), for one system (both of its slot buffers). The
 * systems run on concurrent streams, so the classes of different systems overlap in time.
 * Read synchronises with the recorded events and resets the sums. QMC_EINVAL for a NULL
 * driver or a bad system index. */
qmc_status qmc_dmc_profile_enable(qmc_dmc_t d, int enable);
qmc_status qmc_dmc_profile_read(qmc_dmc_t d, int system, double* ms, int64_t* launches);
void qmc_dmc_destroy(qmc_dmc_t d);

/* Rates of the current device that bound the kernels neither the tensor cores nor HBM
 * do (roofline denominators; no counterpart in the paper): out[0] = FP32 FMA throughput
 * (TFLOP/s, an FMA counted as 2 flops), out[1] = FP64 FMA throughput (TFLOP/s), out[2] =
 * read bandwidth of a 48 MiB L2-resident buffer (GB/s). Best of a few runs of dedicated
 * kernels timed with CUDA events; clocks are not touched. Synchronous; allocates and frees
 * 48 MiB of device memory. */
qmc_status qmc_measure_rates(double* out);

/* Kernel classes reported by qmc_profile_read. */
typedef enum {
  QMC_K_PROPOSE = 0,      /* Metropolis proposals (Philox + Box-Muller) */
  QMC_K_VGL = 1,          /* tricubic B-spline value/gradient/Laplacian at the proposals */
  QMC_K_SWEEP = 2,        /* sequential ratio / accept / inverse-update sweep */
  QMC_K_ENERGY = 3,       /* local energy and ln|Psi| */
  QMC_K_REINVERT = 4,     /* standalone FP64 re-inversion */
  QMC_K_VGL_CURRENT = 5,  /* orbitals at the current positions (set-up) */
  QMC_K_ACCUMULATE = 6,   /* FP64 reductions over walkers */
  QMC_K_FLUSH = 7,        /* batched application of the delayed-update windows */
  QMC_K_REFINE = 8,       /* single-precision re-inversion: error-free residual R = I - A X */
  QMC_K_REFINE_UPDATE = 9,/* single-precision re-inversion: X <- X + X R, FP64 fallback */
  QMC_K_LOGDET = 10,      /* log-determinant anchor (error-free FP32 LU) */
  QMC_K_NLPP = 11,        /* non-local pseudopotential quadrature (pairs and virtual moves) */
  QMC_K_EWALD = 12,       /* Ewald reciprocal-space energy (structure factors) */
  QMC_K_JASTROW3 = 13,    /* three-body Jastrow gradient, Laplacian and value per electron */
  QMC_K_BRANCH = 14,      /* DMC branching or reconfiguration, and the walker copies */
  QMC_NKERNELS = 15
} qmc_kernel;

/* Per-kernel timing: when enabled, every launch of the walker set is bracketed by CUDA
 * events on its stream. qmc_profile_read synchronises, stores the summed device time (ms)
 * and the launch count of each qmc_kernel class (arrays of QMC_NKERNELS, either may be
 * NULL) and resets the sums. */
qmc_status qmc_profile_enable(qmc_walkers_t w, int enable);
qmc_status qmc_profile_read(qmc_walkers_t w, double* ms, int64_t* launches);

/* Number of kernel launches the library enqueued since the walker set was created. */
int64_t qmc_launch_count(qmc_walkers_t w);

/* CUDA-graph replay of sweeps (no counterpart in the paper, which launches per move or per
 * batch; the persistent-launch batching of many walkers it motivates). On by default. With
 * it on, each sweep of qmc_sweep (and each step of qmc_dmc_step, over all of the driver's
 * systems) that is neither traced, replayed from decisions nor profiled runs as one CUDA
 * graph launched on the caller's stream, after one kernel that writes the sweep index to a
 * device word the graph's kernels read. A graph is captured, without running, the first time
 * a sweep starts from a given host state (system parameters, launch configuration, the walker
 * set's buffer assignment and its move counts since the last re-inversion and log-det
 * anchor) and is kept, up to 16 per walker set or driver, least recently used replaced;
 * a change of the Hamiltonian or of the launch configuration changes that state. The results
 * are identical bit for bit to those of direct launches. qmc_launch_count counts the graphs'
 * kernels and the index-setting kernel.
 *   qmc_graph_enable / qmc_dmc_graph_enable: enable != 0 turns replay on, 0 off (the kept
 *       graphs stay until destroy).
 *   qmc_graph_stats / qmc_dmc_graph_stats: captures and replays so far (either may be NULL).
 * QMC_EINVAL for a NULL handle. */
qmc_status qmc_graph_enable(qmc_walkers_t w, int enable);
qmc_status qmc_graph_stats(qmc_walkers_t w, int64_t* captures, int64_t* replays);
qmc_status qmc_dmc_graph_enable(qmc_dmc_t d, int enable);
qmc_status qmc_dmc_graph_stats(qmc_dmc_t d, int64_t* captures, int64_t* replays);

void qmc_walkers_destroy(qmc_walkers_t w);
void qmc_system_destroy(qmc_system_t sys);

/* Message of the last failed call on this thread ("" if none). */
const char* qmc_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* QMCGB_H */
