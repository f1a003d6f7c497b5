// C-ABI runtime of libqmcgb: object lifetimes, argument checks, host<->device copies and
// the order of kernel launches of a sweep.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/qmcgb.h"
#include "qmc_internal.h"
#include "qmc_launch.h"

using namespace qmcgb;

namespace {
thread_local std::string g_err;

qmc_status fail(qmc_status s, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  g_err = buf;
  return s;
}

#define QMC_CUDA(call)                                                                   \
  do {                                                                                   \
    cudaError_t e_ = (call);                                                             \
    if (e_ != cudaSuccess)                                                               \
      return fail(e_ == cudaErrorMemoryAllocation ? QMC_ENOMEM : QMC_ECUDA, "%s: %s (%s:%d)", \
                  #call, cudaGetErrorString(e_), __FILE__, __LINE__);                    \
  } while (0)

bool is_device_ptr(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

double host_min_image(double d, double L) { return d - L * std::nearbyint(d / L); }

double host_wrap(double x, double L) {
  double m = std::fmod(x, L);
  if (m != 0.0 && m < 0.0) m += L;
  return m;
}

int round_up(int x, int m) { return (x + m - 1) / m * m; }

// IEEE round-to-nearest-even of a float to bfloat16 (stored as the upper 16 bits).
uint16_t f32_to_bf16(float f) {
  uint32_t u;
  std::memcpy(&u, &f, 4);
  if ((u & 0x7fffffffu) > 0x7f800000u) return (uint16_t)((u >> 16) | 0x40);   // NaN
  const uint32_t lsb = (u >> 16) & 1u;
  u += 0x7fffu + lsb;
  return (uint16_t)(u >> 16);
}
}  // namespace

struct qmc_system_s {
  qmc_system_desc d{};
  SysParams P{};
  void* d_table = nullptr;
  double* d_ions = nullptr;
  float* d_ionsf = nullptr;
  uint64_t ham_version = 0;    // bumped by every change of the Hamiltonian's terms
  double* d_j3 = nullptr;      // three-body Jastrow coefficients [2][n_coef]
  int4* d_ew_n = nullptr;      // Ewald half set of integer k vectors
  double* d_ew = nullptr;      // c_k [n_k], the ions' rho_k [2][n_k], constant [1]
  bool has_spline = false;
  const TwLaunch* tw = nullptr;
  const TtLaunch* tt = nullptr;
};

namespace {
// Sweeps (and DMC steps) replayed as CUDA graphs. The launches of a sweep follow from host
// state alone: the system's parameters, the launch configuration, the walker set's device
// pointers (which the refinements' buffer swaps permute) and its counts of moves since the
// last re-inversion and log-det anchor. That state, byte for byte, keys a captured graph;
// `post` holds the state the captured sweep leaves, which a replay installs. The sweep index
// of the Philox counters reaches the graph's kernels through a device word set before each
// replay, so one graph serves every sweep that starts from the same state.
using Bytes = std::vector<unsigned char>;

template <class T>
void put(Bytes& b, const T& v) {
  const auto* p = reinterpret_cast<const unsigned char*>(&v);
  b.insert(b.end(), p, p + sizeof(T));
}

template <class T>
void take(const unsigned char*& p, T& v) {
  std::memcpy(&v, p, sizeof(T));
  p += sizeof(T);
}

struct GraphEntry {
  Bytes key, post;
  cudaGraphExec_t exec = nullptr;
  std::vector<int64_t> launches;   // kernels of the graph, per walker set
  uint64_t used = 0;
};

struct GraphCache {
  static constexpr size_t kMaxEntries = 16;
  std::vector<GraphEntry> entries;
  uint64_t clock = 0;
  int64_t captures = 0, replays = 0;
  bool enabled = true;

  GraphEntry* find(const Bytes& key) {
    for (auto& g : entries)
      if (g.key == key) return &g;
    return nullptr;
  }
  // a free entry, or the least recently used one with its graph destroyed
  GraphEntry& slot() {
    if (entries.size() < kMaxEntries) return entries.emplace_back();
    GraphEntry* lru = &entries[0];
    for (auto& g : entries)
      if (g.used < lru->used) lru = &g;
    if (lru->exec) cudaGraphExecDestroy(lru->exec);
    *lru = GraphEntry{};
    return *lru;
  }
  void clear() {
    for (auto& g : entries)
      if (g.exec) cudaGraphExecDestroy(g.exec);
    entries.clear();
  }
};
}  // namespace

struct qmc_walkers_s {
  qmc_system_s* sys = nullptr;
  WalkParams W{};
  uint32_t sweep = 0;
  int chunk = 0;               // moves per launch of a spin block
  void* d_P = nullptr;         // proposal orbital values [W][chunk][5][ld_v]
  Prop* d_prop = nullptr;      // [W][chunk]
  double* d_out = nullptr;     // [8] accumulate output
  long long* d_nacc = nullptr;
  long long proposed = 0;      // since the last accumulate
  double* trace = nullptr;     // borrowed
  size_t trace_sweeps = 0;     // capacity in sweeps
  size_t traced = 0;
  uint8_t* d_forced = nullptr;
  int forced_sweeps = 0;
  int64_t launches = 0;
  bool energy_valid = false;   // e_loc / log_psi hold the current configuration's values
  uint64_t energy_version = 0; // the system's Hamiltonian version they were measured with
  void* d_j3vgl = nullptr;     // three-body Jastrow terms per electron [W][n_e][5] (working precision)
  cudaStream_t side = nullptr; // the up block's last refinement of a sweep runs here, beside
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;   // the down block's moves
  int since_moves[2] = {0, 0}; // proposed moves per spin since the last re-inversion
  int since_anchor[2] = {0, 0};// proposed moves per spin since the last log-det anchor
  GraphCache graphs;
  cudaStream_t cap = nullptr;  // capture stream of the graphs
  uint32_t* d_t = nullptr;     // device sweep index read by replayed graphs
  bool profiling = false;
  struct Ev { int kind; cudaEvent_t a, b; };
  std::vector<Ev> events;
  double prof_ms[QMC_NKERNELS] = {0};
  int64_t prof_n[QMC_NKERNELS] = {0};
};

namespace {
// Launch bracket: counts one launch and, when profiling is on, records events around it.
struct Bracket {
  qmc_walkers_s* w;
  cudaStream_t st;
  int kind;
  cudaEvent_t a = nullptr, b = nullptr;
  Bracket(qmc_walkers_s* w_, cudaStream_t st_, int kind_) : w(w_), st(st_), kind(kind_) {
    w->launches += 1;
    if (!w->profiling) return;
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    cudaEventRecord(a, st);
  }
  ~Bracket() {
    if (!a) return;
    cudaEventRecord(b, st);
    w->events.push_back({kind, a, b});
  }
};

void drain_events(qmc_walkers_s* w) {
  for (auto& e : w->events) {
    float ms = 0.f;
    if (cudaEventSynchronize(e.b) == cudaSuccess && cudaEventElapsedTime(&ms, e.a, e.b) == cudaSuccess) {
      w->prof_ms[e.kind] += ms;
      w->prof_n[e.kind] += 1;
    }
    cudaEventDestroy(e.a);
    cudaEventDestroy(e.b);
  }
  w->events.clear();
}
}  // namespace

// ------------------------------------------------------------------------ errors
extern "C" const char* qmc_last_error(void) { return g_err.c_str(); }

int qmcgb::set_last_error(int s, const char* msg) {
  g_err = msg;
  return s;
}

// ------------------------------------------------------------------------ system
extern "C" qmc_status qmc_system_create(const qmc_system_desc* desc, qmc_system_t* out) {
  if (!desc || !out) return fail(QMC_EINVAL, "qmc_system_create: NULL argument");
  *out = nullptr;
  const qmc_system_desc& d = *desc;
  if (d.n_up < 0 || d.n_dn < 0 || d.n_up > 1024 || d.n_dn > 1024 || d.n_up + d.n_dn == 0)
    return fail(QMC_EINVAL, "electron counts must be in [0, 1024] with at least one electron");
  if (!(d.L > 0.0) || !std::isfinite(d.L)) return fail(QMC_EINVAL, "L must be positive");
  if (d.n_ion < 0 || (d.n_ion > 0 && !d.ion_pos)) return fail(QMC_EINVAL, "bad ion list");
  if (!(d.step >= 0.0)) return fail(QMC_EINVAL, "step must be >= 0");
  if (!(d.drift_a >= 0.0) || !std::isfinite(d.drift_a)) return fail(QMC_EINVAL, "drift_a must be >= 0");
  if (d.prop_chunk < 0) return fail(QMC_EINVAL, "prop_chunk must be >= 0");
  if (d.delay_k < 1 || d.delay_k > kMaxDelay) return fail(QMC_EINVAL, "delay_k must be in [1, %d]", kMaxDelay);
  if (d.prec < QMC_FP64 || d.prec > QMC_FP32_BF16TAB) return fail(QMC_EINVAL, "unknown precision");
  if (d.move != QMC_MOVE_METROPOLIS && d.move != QMC_MOVE_DRIFT) return fail(QMC_EINVAL, "unknown move");
  if (d.reinv_period < 0) return fail(QMC_EINVAL, "reinv_period must be >= 0");
  if (d.logdet_period < 0 || (d.logdet_period > 0 && (d.reinv_period <= 0 || d.logdet_period % d.reinv_period)))
    return fail(QMC_EINVAL, "logdet_period must be 0 or a positive multiple of reinv_period");
  qmc_system_s* s = new qmc_system_s;
  s->d = d;
  s->d.ion_pos = nullptr;
  SysParams& P = s->P;
  P.n_up = d.n_up;
  P.n_dn = d.n_dn;
  P.n_e = d.n_up + d.n_dn;
  P.n_ion = d.n_ion;
  P.L = d.L;
  P.Lf = (float)d.L;
  P.invL = 1.0 / d.L;
  P.invLf = (float)(1.0 / d.L);
  P.ion_Z = d.ion_Z;
  P.ion_Zf = (float)d.ion_Z;
  P.kappa = d.kappa;
  P.kappaf = (float)d.kappa;
  P.with_potential = d.with_potential;
  P.move = d.move;
  P.step = d.step;
  P.drift_a = d.drift_a > 0.0 ? d.drift_a : 0.0;
  P.seed_lo = (uint32_t)(d.seed & 0xffffffffu);
  P.seed_hi = (uint32_t)(d.seed >> 32);
  // ions: wrapped, device copies in [3][n_ion] layout; ion-ion constant on the host
  std::vector<double> ion((size_t)3 * std::max(d.n_ion, 1));
  std::vector<float> ionf(ion.size());
  for (int I = 0; I < d.n_ion; ++I)
    for (int c = 0; c < 3; ++c) {
      ion[(size_t)c * d.n_ion + I] = host_wrap(d.ion_pos[3 * I + c], d.L);
      ionf[(size_t)c * d.n_ion + I] = (float)ion[(size_t)c * d.n_ion + I];
    }
  double vii = 0.0;
  for (int I = 0; I < d.n_ion; ++I)
    for (int J = I + 1; J < d.n_ion; ++J) {
      double r2 = 0.0;
      for (int c = 0; c < 3; ++c) {
        const double dd = host_min_image(ion[(size_t)c * d.n_ion + I] - ion[(size_t)c * d.n_ion + J], d.L);
        r2 += dd * dd;
      }
      const double r = std::sqrt(r2);
      if (r < 0.5 * d.L) vii += d.ion_Z * d.ion_Z * std::exp(-d.kappa * r) / r;
    }
  P.v_ion_ion = vii;
  cudaError_t e = cudaMalloc(&s->d_ions, ion.size() * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc(&s->d_ionsf, ionf.size() * sizeof(float));
  if (e == cudaSuccess)
    e = cudaMemcpy(s->d_ions, ion.data(), ion.size() * sizeof(double), cudaMemcpyHostToDevice);
  if (e == cudaSuccess)
    e = cudaMemcpy(s->d_ionsf, ionf.data(), ionf.size() * sizeof(float), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) {
    qmc_system_destroy(s);
    return fail(QMC_ECUDA, "qmc_system_create: %s", cudaGetErrorString(e));
  }
  P.ions = s->d_ions;
  P.ionsf = s->d_ionsf;
  s->tw = d.prec == QMC_FP64 ? &tw_launch_f64() : &tw_launch_f32();
  s->tt = d.prec == QMC_FP64 ? &tt_launch_f64()
                             : (d.prec == QMC_FP32 ? &tt_launch_f32() : &tt_launch_bf16());
  *out = s;
  return QMC_OK;
}

extern "C" qmc_status qmc_system_set_spline(qmc_system_t s, int nx, int ny, int nz, int n_orb,
                                            const double* coef) {
  if (!s || !coef) return fail(QMC_EINVAL, "qmc_system_set_spline: NULL argument");
  if (nx < 4 || ny < 4 || nz < 4 || nx > 4096 || ny > 4096 || nz > 4096)
    return fail(QMC_EINVAL, "grid sizes must be in [4, 4096]");
  if (n_orb < std::max(s->P.n_up, s->P.n_dn) || n_orb > 4096)
    return fail(QMC_EINVAL, "n_orb must be >= max(n_up, n_dn) and <= 4096");
  const int ld = round_up(n_orb, 8);
  const size_t rows = (size_t)nx * ny * nz;
  const size_t esz = s->d.prec == QMC_FP64 ? 8 : (s->d.prec == QMC_FP32 ? 4 : 2);
  void* dt = nullptr;
  QMC_CUDA(cudaMalloc(&dt, rows * ld * esz));
  // convert and upload in slabs of rows
  const size_t slab = std::max<size_t>(1, (64u << 20) / (ld * esz));
  std::vector<unsigned char> host(std::min(rows, slab) * ld * esz);
  for (size_t r0 = 0; r0 < rows; r0 += slab) {
    const size_t nr = std::min(slab, rows - r0);
    std::memset(host.data(), 0, nr * ld * esz);
    for (size_t r = 0; r < nr; ++r) {
      const double* src = coef + (r0 + r) * n_orb;
      if (esz == 8) {
        std::memcpy(host.data() + r * ld * 8, src, sizeof(double) * n_orb);
      } else if (esz == 4) {
        float* dst = reinterpret_cast<float*>(host.data()) + r * ld;
        for (int o = 0; o < n_orb; ++o) dst[o] = (float)src[o];
      } else {
        uint16_t* dst = reinterpret_cast<uint16_t*>(host.data()) + r * ld;
        for (int o = 0; o < n_orb; ++o) dst[o] = f32_to_bf16((float)src[o]);
      }
    }
    cudaError_t e = cudaMemcpy(static_cast<unsigned char*>(dt) + r0 * ld * esz, host.data(),
                               nr * ld * esz, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
      cudaFree(dt);
      return fail(QMC_ECUDA, "qmc_system_set_spline: %s", cudaGetErrorString(e));
    }
  }
  if (s->d_table) cudaFree(s->d_table);
  s->d_table = dt;
  SysParams& P = s->P;
  P.table = dt;
  P.nx = nx; P.ny = ny; P.nz = nz; P.ld = ld; P.n_orb = n_orb;
  const int nn[3] = {nx, ny, nz};
  for (int c = 0; c < 3; ++c) {
    P.inv_delta[c] = (double)nn[c] / s->d.L;
    P.inv_deltaf[c] = (float)P.inv_delta[c];
  }
  s->has_spline = true;
  return QMC_OK;
}

extern "C" qmc_status qmc_system_set_jastrow(qmc_system_t s, int which, int M, double rcut,
                                             const double* p, int cusp_set, double cusp) {
  if (!s || !p) return fail(QMC_EINVAL, "qmc_system_set_jastrow: NULL argument");
  if (which < 0 || which > 2) return fail(QMC_EINVAL, "which must be 0, 1 or 2");
  if (M < 1 || M > kMaxKnots) return fail(QMC_EINVAL, "M must be in [1, %d]", kMaxKnots);
  if (!(rcut > 0.0) || rcut > 0.5 * s->d.L * (1 + 1e-12))
    return fail(QMC_EINVAL, "rcut must be in (0, L/2]");
  if (cusp_set && M < 2) return fail(QMC_EINVAL, "a cusp needs M >= 2");
  SysParams& P = s->P;
  ++s->ham_version;
  P.jM[which] = M;
  P.jrc[which] = rcut;
  P.jrcf[which] = (float)rcut;
  for (int m = 0; m <= kMaxKnots; ++m) P.jp[which][m] = m <= M ? p[m] : 0.0;
  if (cusp_set) P.jp[which][0] = P.jp[which][2] - (2.0 * rcut / M) * cusp;
  for (int m = 0; m <= kMaxKnots; ++m) P.jpf[which][m] = (float)P.jp[which][m];
  return QMC_OK;
}

extern "C" qmc_status qmc_system_set_nonlocal(qmc_system_t s, int n_channels, const double* amp,
                                               const double* width, double rcut) {
  if (!s) return fail(QMC_EINVAL, "qmc_system_set_nonlocal: NULL system");
  if (n_channels < 0 || n_channels > kMaxNlChannels)
    return fail(QMC_EINVAL, "n_channels must be in [0, %d]", kMaxNlChannels);
  SysParams& P = s->P;
  ++s->ham_version;
  if (n_channels == 0) {
    P.nl_nch = 0;
    return QMC_OK;
  }
  if (!amp || !width) return fail(QMC_EINVAL, "qmc_system_set_nonlocal: NULL channel arrays");
  if (!(rcut > 0.0) || rcut > 0.5 * s->d.L * (1 + 1e-12)) return fail(QMC_EINVAL, "rcut must be in (0, L/2]");
  for (int l = 0; l < n_channels; ++l)
    if (!(width[l] > 0.0) || !std::isfinite(amp[l])) return fail(QMC_EINVAL, "bad channel %d", l);
  for (int l = 0; l < kMaxNlChannels; ++l) {
    P.nl_amp[l] = l < n_channels ? amp[l] : 0.0;
    P.nl_width[l] = l < n_channels ? width[l] : 1.0;
  }
  P.nl_rcut = rcut;
  P.nl_nch = n_channels;
  return QMC_OK;
}

extern "C" qmc_status qmc_system_set_jastrow3(qmc_system_t s, int m_ei, int m_ee, double rcut,
                                              const double* gamma_same, const double* gamma_opp) {
  if (!s) return fail(QMC_EINVAL, "qmc_system_set_jastrow3: NULL system");
  SysParams& P = s->P;
  if (m_ei < 0) {
    ++s->ham_version;
    P.j3_on = 0;
    return QMC_OK;
  }
  if (m_ei > kJ3MaxOrder || m_ee < 0 || m_ee > kJ3MaxOrder)
    return fail(QMC_EINVAL, "the orders must lie in [0, %d]", kJ3MaxOrder);
  if (!gamma_same || !gamma_opp) return fail(QMC_EINVAL, "qmc_system_set_jastrow3: NULL coefficients");
  if (!(rcut > 0.0) || rcut > 0.5 * s->d.L * (1 + 1e-12)) return fail(QMC_EINVAL, "rcut must be in (0, L/2]");
  const int n1 = m_ei + 1, n3 = m_ee + 1, nc = n1 * n1 * n3;
  const double* g[2] = {gamma_same, gamma_opp};
  for (int f = 0; f < 2; ++f)
    for (int l = 0; l < n1; ++l)
      for (int m = 0; m < n1; ++m)
        for (int n = 0; n < n3; ++n) {
          const double a = g[f][(l * n1 + m) * n3 + n], b = g[f][(m * n1 + l) * n3 + n];
          if (!std::isfinite(a)) return fail(QMC_EINVAL, "a coefficient is not finite");
          if (a != b) return fail(QMC_EINVAL, "gamma_lmn must equal gamma_mln");
        }
  std::vector<double> h(2 * (size_t)nc);
  std::copy(gamma_same, gamma_same + nc, h.begin());
  std::copy(gamma_opp, gamma_opp + nc, h.begin() + nc);
  QMC_CUDA(cudaDeviceSynchronize());     // no kernel may still read the previous coefficients
  ++s->ham_version;
  P.j3_on = 0;
  cudaFree(s->d_j3);
  s->d_j3 = nullptr;
  QMC_CUDA(cudaMalloc(&s->d_j3, sizeof(double) * h.size()));
  QMC_CUDA(cudaMemcpy(s->d_j3, h.data(), sizeof(double) * h.size(), cudaMemcpyHostToDevice));
  P.j3_g = s->d_j3;
  P.j3_meI = m_ei;
  P.j3_mee = m_ee;
  P.j3_h = 0.5 * rcut;
  P.j3_on = 1;
  return QMC_OK;
}

extern "C" qmc_status qmc_system_set_ewald(qmc_system_t s, double alpha, double kcut) {
  if (!s) return fail(QMC_EINVAL, "qmc_system_set_ewald: NULL system");
  if (!std::isfinite(alpha) || alpha < 0.0) return fail(QMC_EINVAL, "alpha must be finite and >= 0");
  SysParams& P = s->P;
  ++s->ham_version;
  if (alpha == 0.0) {
    P.ew_on = 0;
    return QMC_OK;
  }
  if (!s->d.with_potential) return fail(QMC_EINVAL, "qmc_system_set_ewald: the system has no potential");
  if (!(kcut > 0.0) || !std::isfinite(kcut)) return fail(QMC_EINVAL, "kcut must be finite and > 0");
  const double L = s->d.L, tl = 2.0 * M_PI / L;
  const double nm = std::floor(kcut / tl);
  if (nm > 64.0) return fail(QMC_EINVAL, "kcut L / (2 pi) must not exceed 64");
  const int nmax = (int)nm;
  // the half set: one of each +-n pair (the first nonzero component of n positive)
  std::vector<int4> ns;
  for (int x = 0; x <= nmax; ++x)
    for (int y = -nmax; y <= nmax; ++y)
      for (int z = -nmax; z <= nmax; ++z) {
        if (!(x > 0 || (x == 0 && (y > 0 || (y == 0 && z > 0))))) continue;
        const double k2 = tl * tl * (double)(x * x + y * y + z * z);
        if (k2 > kcut * kcut) continue;
        if ((int)ns.size() == kEwMaxK)
          return fail(QMC_EINVAL, "more than %d k vectors in the half set", kEwMaxK);
        ns.push_back(make_int4(x, y, z, 0));
      }
  const int nk = (int)ns.size();
  QMC_CUDA(cudaDeviceSynchronize());     // no kernel may still read the previous tables
  cudaFree(s->d_ew_n);
  cudaFree(s->d_ew);
  s->d_ew_n = nullptr;
  s->d_ew = nullptr;
  P.ew_on = 0;
  QMC_CUDA(cudaMalloc(&s->d_ew_n, sizeof(int4) * (nk > 0 ? nk : 1)));
  QMC_CUDA(cudaMalloc(&s->d_ew, sizeof(double) * (3 * (size_t)nk + 1)));
  if (nk > 0) QMC_CUDA(cudaMemcpy(s->d_ew_n, ns.data(), sizeof(int4) * nk, cudaMemcpyHostToDevice));
  P.ew_nk = nk;
  P.ew_alpha = alpha;
  P.ew_alphaf = (float)alpha;
  P.ew_n = s->d_ew_n;
  P.ew_ck = s->d_ew;
  P.ew_rho_ion = s->d_ew + nk;
  P.ew_const = s->d_ew + 3 * (size_t)nk;
  QMC_CUDA(launch_ewald_setup(P, s->d_ew, s->d_ew + nk, s->d_ew + 3 * (size_t)nk, 0));
  QMC_CUDA(cudaDeviceSynchronize());
  P.ew_on = 1;
  return QMC_OK;
}

extern "C" int qmc_system_ewald_count(qmc_system_t s) { return (s && s->P.ew_on) ? s->P.ew_nk : -1; }

extern "C" void qmc_system_destroy(qmc_system_t s) {
  if (!s) return;
  cudaFree(s->d_j3);
  cudaFree(s->d_ew_n);
  cudaFree(s->d_ew);
  cudaFree(s->d_table);
  cudaFree(s->d_ions);
  cudaFree(s->d_ionsf);
  delete s;
}

// ------------------------------------------------------------------------ walkers
namespace {

qmc_status check_err(qmc_walkers_s* w, cudaStream_t st) {
  QMC_CUDA(cudaStreamSynchronize(st));
  int err = 0;
  QMC_CUDA(cudaMemcpy(&err, w->W.err, sizeof(int), cudaMemcpyDeviceToHost));
  if (err) {
    QMC_CUDA(cudaMemset(w->W.err, 0, sizeof(int)));
    if (err & kErrSingular) return fail(QMC_ESINGULAR, "a Slater matrix was singular at (re-)inversion");
    if (err & kErrTimeout) return fail(QMC_ETIMEOUT, "a bounded device wait timed out");
    if (err & kErrJ3Near)
      return fail(QMC_ECUDA, "more than %d ions within r_c / 2 of a move of the three-body Jastrow "
                             "factor", kJ3MaxNear);
    if (err & kErrOverflow)
      return fail(QMC_ECUDA, "more electron-ion pairs inside the pseudopotential cutoff than the "
                             "per-walker list holds (2 per electron)");
    return fail(QMC_ECUDA, "device error flag 0x%x", err);
  }
  return QMC_OK;
}

// Local energy (and ln|Psi|) of every walker: kinetic + local potential, then the non-local
// pseudopotential part when the system has one; t seeds the quadrature's rotation.
qmc_status measure_energy(qmc_walkers_s* w, const WalkParams& W0, uint32_t t, cudaStream_t st) {
  qmc_system_s* s = w->sys;
  WalkParams W = W0;
  W.j3vgl = nullptr;
  if (s->P.j3_on && s->P.n_ion > 0) {
    W.j3vgl = w->d_j3vgl;
    Bracket b(w, st, QMC_K_JASTROW3);
    QMC_CUDA(s->tw->j3_vgl(s->P, W, st));
  }
  { Bracket b(w, st, QMC_K_ENERGY); QMC_CUDA(s->tw->local_energy(s->P, W, st)); }
  if (s->P.ew_on && s->P.ew_nk > 0) {
    Bracket b(w, st, QMC_K_EWALD);
    QMC_CUDA(s->tw->ewald_recip(s->P, W, st));
  }
  if (s->P.nl_nch > 0 && s->P.n_ion > 0) {
    Bracket b(w, st, QMC_K_NLPP);
    QMC_CUDA(s->tt->nlpp(s->P, W, t, st));
    w->launches += 2;   // pair list, virtual moves, per-walker sums
  }
  return QMC_OK;
}

qmc_status setup_state(qmc_walkers_s* w, cudaStream_t st) {
  qmc_system_s* s = w->sys;
  { Bracket b(w, st, QMC_K_VGL_CURRENT); QMC_CUDA(s->tt->vgl_current(s->P, w->W, st)); }
  { Bracket b(w, st, QMC_K_REINVERT); QMC_CUDA(s->tw->reinvert(s->P, w->W, st)); }
  { qmc_status r = measure_energy(w, w->W, w->sweep, st); if (r != QMC_OK) return r; }
  QMC_CUDA(cudaMemsetAsync(w->W.acc_since, 0, sizeof(int) * 2 * w->W.n_w, st));
  w->since_moves[0] = w->since_moves[1] = 0;
  w->since_anchor[0] = w->since_anchor[1] = 0;
  w->energy_valid = true;
  w->energy_version = s->ham_version;
  return check_err(w, st);
}

void free_walkers(qmc_walkers_s* w) {
  WalkParams& W = w->W;
  void* ptrs[] = {W.pos, W.binv[0], W.binv[1], W.binv_alt[0], W.binv_alt[1], W.vgl, W.logdet,
                  W.sgn, W.wid, W.weight, W.e_loc, W.log_psi, W.n_acc, W.acc_since, W.scratch64,
                  W.err, w->d_P, w->d_prop, w->d_out, w->d_nacc, w->d_forced, W.win_phi,
                  W.win_u, W.win_cinv, W.win_row, W.win_m, W.refine_max, W.refine_last,
                  W.logdet_shift, W.refine_fb, W.rscale, W.r2, W.vnl, W.nl_pairs, W.nl_count,
                  W.nl_val,
                  w->d_j3vgl};
  for (void* p : ptrs) cudaFree(p);
  w->graphs.clear();
  cudaFree(w->d_t);
  if (w->cap) cudaStreamDestroy(w->cap);
  if (w->ev_fork) cudaEventDestroy(w->ev_fork);
  if (w->ev_join) cudaEventDestroy(w->ev_join);
  if (w->side) cudaStreamDestroy(w->side);
}

qmc_status upload_positions(qmc_walkers_s* w, const double* pos, bool pos_on_device) {
  const SysParams& P = w->sys->P;
  const int nw = w->W.n_w, ne = P.n_e;
  std::vector<double> h((size_t)nw * ne * 3);
  std::vector<double> src;
  if (pos_on_device) {
    src.resize(h.size());
    QMC_CUDA(cudaMemcpy(src.data(), pos, h.size() * sizeof(double), cudaMemcpyDeviceToHost));
    pos = src.data();
  }
  for (int a = 0; a < nw; ++a)
    for (int e = 0; e < ne; ++e)
      for (int c = 0; c < 3; ++c) {
        const double v = pos[((size_t)a * ne + e) * 3 + c];
        if (!std::isfinite(v)) return fail(QMC_EINVAL, "non-finite electron position");
        h[((size_t)a * 3 + c) * ne + e] = host_wrap(v, P.L);
      }
  QMC_CUDA(cudaMemcpy(w->W.pos, h.data(), h.size() * sizeof(double), cudaMemcpyHostToDevice));
  return QMC_OK;
}
}  // namespace

namespace {
// Allocates the device arrays of a walker set with `cap` slots (all zeroed where it
// matters); `proposals` adds the buffers of the batched Metropolis proposals.
qmc_status alloc_walkers(qmc_system_s* s, int cap, bool proposals, qmc_walkers_s** out) {
  const SysParams& P = s->P;
  qmc_walkers_s* w = new qmc_walkers_s;
  w->sys = s;
  WalkParams& W = w->W;
  W.n_w = cap;
  const int ns_max = std::max(P.n_up, P.n_dn);
  W.ld_v = round_up(std::max(ns_max, 1), 8);
  const size_t tw = s->tw->tw_size;
  const size_t nw = cap, ne = P.n_e;
  w->chunk = s->d.prop_chunk > 0 ? std::min(ns_max, s->d.prop_chunk) : ns_max;
  // keep the proposal buffer below 2 GiB by splitting spin blocks into chunks
  while (w->chunk > 32 && nw * w->chunk * 5 * W.ld_v * tw > (size_t(2) << 30)) w->chunk = (w->chunk + 1) / 2;
  const size_t np = proposals ? nw * (size_t)w->chunk : 1;
  // Metropolis proposals of a chunk, or the draws of every move of a drift sweep
  const size_t nprop = proposals ? np : s->d.move == QMC_MOVE_DRIFT ? nw * ne : 1;
  const size_t nb_up = (size_t)std::max(P.n_up, 1) * std::max(P.n_up, 1);
  const size_t nb_dn = (size_t)std::max(P.n_dn, 1) * std::max(P.n_dn, 1);
  // the second inverse buffers serve the batched single-precision re-inversion
  const bool alt = tw == sizeof(float);
  struct A { void** p; size_t bytes; } allocs[] = {
      {(void**)&W.pos, nw * 3 * ne * sizeof(double)},
      {(void**)&W.binv[0], nw * nb_up * tw},
      {(void**)&W.binv[1], nw * nb_dn * tw},
      {(void**)&W.binv_alt[0], alt ? nw * nb_up * tw : 0},
      {(void**)&W.binv_alt[1], alt ? nw * nb_dn * tw : 0},
      {(void**)&W.vgl, nw * ne * 5 * W.ld_v * tw},
      {(void**)&W.logdet, nw * 2 * sizeof(double)},
      {(void**)&W.sgn, nw * 2 * sizeof(double)},
      {(void**)&W.wid, nw * sizeof(uint32_t)},
      {(void**)&W.weight, nw * sizeof(double)},
      {(void**)&W.e_loc, nw * sizeof(double)},
      {(void**)&W.log_psi, nw * sizeof(double)},
      {(void**)&W.n_acc, nw * sizeof(long long)},
      {(void**)&W.acc_since, nw * 2 * sizeof(int)},
      {(void**)&W.scratch64, 2 * nw * (size_t)W.ld_v * W.ld_v * sizeof(double)},
      {(void**)&W.err, sizeof(int)},
      {(void**)&w->d_P, np * 5 * W.ld_v * tw},
      {(void**)&w->d_prop, nprop * sizeof(Prop)},
      {(void**)&w->d_out, 8 * sizeof(double)},
      {(void**)&w->d_nacc, sizeof(long long)},
      {(void**)&W.win_phi, nw * (size_t)s->d.delay_k * W.ld_v * tw},
      {(void**)&W.win_u, nw * (size_t)s->d.delay_k * W.ld_v * tw},
      {(void**)&W.win_cinv, nw * (size_t)s->d.delay_k * s->d.delay_k * tw},
      {(void**)&W.win_row, nw * (size_t)s->d.delay_k * sizeof(int)},
      {(void**)&W.win_m, nw * sizeof(int)},
      {(void**)&W.refine_max, nw * 2 * sizeof(float)},
      {(void**)&W.refine_last, nw * 2 * sizeof(float)},
      {(void**)&W.logdet_shift, nw * 2 * sizeof(float)},
      {(void**)&W.refine_fb, nw * 2 * sizeof(int)},
      {(void**)&W.r2, nw * 2 * sizeof(double)},
      {(void**)&W.vnl, nw * sizeof(double)},
      {(void**)&W.nl_pairs, nw * (size_t)std::max(64, 2 * (int)ne) * sizeof(int)},
      {(void**)&W.nl_count, nw * sizeof(int)},
      {(void**)&W.nl_val, nw * (size_t)std::max(64, 2 * (int)ne) * sizeof(double)},
      {(void**)&W.rscale, nw * 4 * (size_t)W.ld_v * sizeof(int)},
      {(void**)&w->d_j3vgl, nw * (size_t)ne * 5 * tw},
  };
  for (auto& a : allocs) {
    *a.p = nullptr;
    if (a.bytes == 0) continue;
    cudaError_t e = cudaMalloc(a.p, a.bytes);
    if (e != cudaSuccess) {
      free_walkers(w);
      delete w;
      return fail(QMC_ENOMEM, "cannot allocate %zu bytes of walker state: %s", a.bytes,
                  cudaGetErrorString(e));
    }
  }
  if (cudaMalloc(&w->d_t, sizeof(uint32_t)) != cudaSuccess) {
    w->d_t = nullptr;
    free_walkers(w);
    delete w;
    return fail(QMC_ENOMEM, "cannot allocate the walker set's sweep index");
  }
  if (cudaStreamCreateWithFlags(&w->side, cudaStreamNonBlocking) != cudaSuccess ||
      cudaStreamCreateWithFlags(&w->cap, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreateWithFlags(&w->ev_fork, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&w->ev_join, cudaEventDisableTiming) != cudaSuccess) {
    free_walkers(w);
    delete w;
    return fail(QMC_ECUDA, "cannot create the walker set's side stream");
  }
  // zero the orbital rows so padded columns never hold garbage
  cudaMemset(W.vgl, 0, nw * ne * 5 * W.ld_v * tw);
  cudaMemset(W.err, 0, sizeof(int));
  cudaMemset(W.n_acc, 0, nw * sizeof(long long));
  cudaMemset(W.acc_since, 0, nw * 2 * sizeof(int));
  cudaMemset(W.win_m, 0, nw * sizeof(int));
  cudaMemset(W.refine_max, 0, nw * 2 * sizeof(float));
  cudaMemset(W.refine_last, 0xFF, nw * 2 * sizeof(float));   // NaN: no refinement yet
  cudaMemset(W.logdet_shift, 0xFF, nw * 2 * sizeof(float));  // NaN: no anchor yet
  cudaMemset(W.refine_fb, 0, nw * 2 * sizeof(int));
  cudaMemset(W.r2, 0, nw * 2 * sizeof(double));
  cudaMemset(W.vnl, 0, nw * sizeof(double));
  W.nl_cap = std::max(64, 2 * (int)ne);
  W.kc = s->d.delay_k;
  *out = w;
  return QMC_OK;
}

// IDs 0..n-1, weights 1, positions from the caller, orbitals, FP64 inverses and E_L.
qmc_status init_walkers(qmc_walkers_s* w, int n, const double* pos) {
  const int saved = w->W.n_w;
  w->W.n_w = n;
  std::vector<uint32_t> ids(n);
  std::vector<double> ones(n, 1.0);
  for (int i = 0; i < n; ++i) ids[i] = (uint32_t)i;
  QMC_CUDA(cudaMemcpy(w->W.wid, ids.data(), n * sizeof(uint32_t), cudaMemcpyHostToDevice));
  QMC_CUDA(cudaMemcpy(w->W.weight, ones.data(), n * sizeof(double), cudaMemcpyHostToDevice));
  qmc_status st = upload_positions(w, pos, is_device_ptr(pos));
  if (st == QMC_OK) st = setup_state(w, 0);
  if (saved != n) w->W.n_w = saved;
  return st;
}
}  // namespace

extern "C" qmc_status qmc_walkers_create(qmc_system_t s, int n_walkers, const double* pos,
                                         qmc_walkers_t* out) {
  if (!s || !out || !pos) return fail(QMC_EINVAL, "qmc_walkers_create: NULL argument");
  *out = nullptr;
  if (!s->has_spline) return fail(QMC_EINVAL, "qmc_walkers_create: set the spline table first");
  if (n_walkers < 1 || n_walkers > (1 << 20)) return fail(QMC_EINVAL, "n_walkers must be in [1, 2^20]");
  qmc_walkers_s* w = nullptr;
  qmc_status st = alloc_walkers(s, n_walkers, s->d.move == QMC_MOVE_METROPOLIS, &w);
  if (st != QMC_OK) return st;
  st = init_walkers(w, n_walkers, pos);
  if (st != QMC_OK) {
    const std::string msg = g_err;
    free_walkers(w);
    delete w;
    g_err = msg;
    return st;
  }
  *out = w;
  return QMC_OK;
}

namespace {
// The sweeps of one walker set: Metropolis moves from batched proposals, or drift moves
// with in-kernel orbital evaluation; windows flushed in batches every k moves unless the
// re-inversion cadence counts accepted moves. t: the sweep index of the Philox counters (an
// offset from *W.t_base when that is set).
qmc_status sweep_once(qmc_walkers_s* w, WalkParams& W, uint32_t t, bool fixed_node, cudaStream_t st) {
  qmc_system_s* s = w->sys;
  const SysParams& P = s->P;
  const int kc = s->d.delay_k, period = s->d.reinv_period;
  const bool drift = s->d.move == QMC_MOVE_DRIFT;
  const bool ext = kc >= 4 && !(period > 0 && s->d.reinv_on_accepted) &&
                   !(period > 0 && s->d.prec == QMC_FP64);
  bool joined = true;             // the side stream's work has been joined back into st
  if (drift) {
    Bracket b(w, st, QMC_K_PROPOSE);
    QMC_CUDA(launch_drift_draws(P, W, t, w->d_prop, st));
  }
  for (int spin = 0; spin < 2; ++spin) {
    const int b0 = spin ? P.n_up : 0, b1 = spin ? P.n_e : P.n_up;
    const int pchunk = drift ? std::max(b1 - b0, 1) : w->chunk;
    for (int pc0 = b0; pc0 < b1; pc0 += pchunk) {
      const int pc1 = std::min(b1, pc0 + pchunk);
      if (!drift) {
        { Bracket b(w, st, QMC_K_PROPOSE); QMC_CUDA(launch_proposals(P, W, t, pc0, pc1, w->d_prop, st)); }
        { Bracket b(w, st, QMC_K_VGL); QMC_CUDA(s->tt->vgl_proposals(P, W, pc0, pc1, w->d_prop, w->d_P, st)); }
      }
      if (!ext) {
        Bracket b(w, st, QMC_K_SWEEP);
        if (drift)
          QMC_CUDA(s->tt->sweep_drift(P, W, t, pc0, pc1, kc, w->d_prop, period,
                                      s->d.reinv_on_accepted, 0, fixed_node, st));
        else
          QMC_CUDA(s->tw->sweep(P, W, t, pc0, pc1, kc, w->d_P, w->d_prop, pc0, pc1 - pc0,
                                period, s->d.reinv_on_accepted, 0, fixed_node, st));
        continue;
      }
      for (int e0 = pc0; e0 < pc1;) {
        int e1 = std::min(pc1, e0 + kc);
        if (period > 0) e1 = std::min(e1, e0 + (period - w->since_moves[spin]));
        {
          Bracket b(w, st, QMC_K_SWEEP);
          if (drift)
            QMC_CUDA(s->tt->sweep_drift(P, W, t, e0, e1, kc, w->d_prop, 0, 0, 1, fixed_node, st));
          else
            QMC_CUDA(s->tw->sweep(P, W, t, e0, e1, kc, w->d_P, w->d_prop, pc0, pc1 - pc0,
                                  0, 0, 1, fixed_node, st));
        }
        { Bracket b(w, st, QMC_K_FLUSH); QMC_CUDA(s->tw->flush(P, W, spin, st)); }
        w->launches += 1;   // the window reset that follows each flush
        if (period > 0) {
          w->since_moves[spin] += e1 - e0;
          if (w->since_moves[spin] >= period) {
            // The up block's last refinement of the sweep (and its log-det anchor) runs on the
            // side stream beside the down block's moves, which read the positions and the
            // down block's own arrays only; the sweep joins it back before it returns.
            const bool fork = spin == 0 && e1 == b1 && P.n_dn > 0;
            cudaStream_t rs = st;
            if (fork) {
              QMC_CUDA(cudaEventRecord(w->ev_fork, st));
              QMC_CUDA(cudaStreamWaitEvent(w->side, w->ev_fork, 0));
              rs = w->side;
            }
            { Bracket b(w, rs, QMC_K_REFINE); QMC_CUDA(s->tw->refine(P, W, spin, 0, rs)); }
            {
              Bracket b(w, rs, QMC_K_REFINE_UPDATE);
              QMC_CUDA(s->tw->refine(P, W, spin, 1, rs));
              // the refined inverse is in the second buffer: it becomes the current one
              std::swap(W.binv[spin], W.binv_alt[spin]);
              std::swap(w->W.binv[spin], w->W.binv_alt[spin]);
              QMC_CUDA(s->tw->refine(P, W, spin, 2, rs));
            }
            w->launches += 2;   // row scales + residual, update + fallback
            w->since_anchor[spin] += w->since_moves[spin];
            w->since_moves[spin] = 0;
            if (s->d.logdet_period > 0 && w->since_anchor[spin] >= s->d.logdet_period) {
              Bracket b(w, rs, QMC_K_LOGDET);
              QMC_CUDA(s->tw->logdet_anchor(P, W, spin, rs));
              w->since_anchor[spin] = 0;
            }
            if (fork) {
              QMC_CUDA(cudaEventRecord(w->ev_join, w->side));
              joined = false;
            }
          }
        }
        e0 = e1;
      }
    }
  }
  if (!joined) QMC_CUDA(cudaStreamWaitEvent(st, w->ev_join, 0));
  return QMC_OK;
}

// The host state a sweep of walker set w changes: its device pointers (the refinements swap
// the two inverse buffers of a spin block) and its move counts.
void put_state(Bytes& b, const qmc_walkers_s* w) {
  put(b, w->W);
  put(b, w->since_moves);
  put(b, w->since_anchor);
}

void take_state(const unsigned char*& p, qmc_walkers_s* w) {
  take(p, w->W);
  take(p, w->since_moves);
  take(p, w->since_anchor);
}

// Everything the launches of walker set w's sweep depend on besides the sweep index.
void put_walker_key(Bytes& b, const qmc_walkers_s* w) {
  put(b, w->sys->P);
  put(b, w->sys->d);
  put(b, w->chunk);
  put(b, w->d_P);
  put(b, w->d_prop);
  put(b, w->d_j3vgl);
  put_state(b, w);
}

// Ends a capture begun on `cap` and instantiates it; on any failure (of the capture's own
// launches, r, or of the capture) no graph is kept.
qmc_status end_capture(cudaStream_t cap, qmc_status r, cudaGraphExec_t* exec) {
  cudaGraph_t graph = nullptr;
  const cudaError_t e = cudaStreamEndCapture(cap, &graph);
  cudaError_t ei = cudaSuccess;
  if (r == QMC_OK && e == cudaSuccess) ei = cudaGraphInstantiate(exec, graph, 0);
  if (graph) cudaGraphDestroy(graph);
  if (r != QMC_OK) return r;
  if (e != cudaSuccess || ei != cudaSuccess) {
    cudaGetLastError();
    return fail(QMC_ECUDA, "graph capture: %s", cudaGetErrorString(e != cudaSuccess ? e : ei));
  }
  return QMC_OK;
}

// One Metropolis or drift sweep of w and its measurement, as a graph on stream st: captured
// (on w's capture stream; nothing runs) the first time its starting state is met, then
// replayed behind one launch that sets the device sweep index to w->sweep.
qmc_status sweep_graph(qmc_walkers_s* w, cudaStream_t st) {
  Bytes key;
  put_walker_key(key, w);
  GraphEntry* g = w->graphs.find(key);
  if (!g) {
    Bytes pre;
    put_state(pre, w);
    const int64_t l0 = w->launches;
    QMC_CUDA(cudaStreamBeginCapture(w->cap, cudaStreamCaptureModeRelaxed));
    WalkParams W = w->W;
    W.trace = nullptr;
    W.forced = nullptr;
    W.t_base = w->d_t;
    qmc_status r = sweep_once(w, W, 0u, false, w->cap);
    if (r == QMC_OK) r = measure_energy(w, W, 1u, w->cap);
    cudaGraphExec_t exec = nullptr;
    r = end_capture(w->cap, r, &exec);
    const int64_t n = w->launches - l0;
    Bytes post;
    put_state(post, w);
    const unsigned char* p = pre.data();
    take_state(p, w);
    w->launches = l0;
    if (r != QMC_OK) return r;
    g = &w->graphs.slot();
    g->key = std::move(key);
    g->post = std::move(post);
    g->exec = exec;
    g->launches = {n};
    ++w->graphs.captures;
  }
  QMC_CUDA(launch_set_word(w->d_t, w->sweep, st));
  QMC_CUDA(cudaGraphLaunch(g->exec, st));
  const unsigned char* p = g->post.data();
  take_state(p, w);
  w->launches += g->launches[0] + 1;
  g->used = ++w->graphs.clock;
  ++w->graphs.replays;
  return QMC_OK;
}
}  // namespace

extern "C" qmc_status qmc_sweep(qmc_walkers_t w, int n_sweeps, void* stream) {
  if (!w) return fail(QMC_EINVAL, "qmc_sweep: NULL walkers");
  if (n_sweeps < 0) return fail(QMC_EINVAL, "qmc_sweep: n_sweeps < 0");
  qmc_system_s* s = w->sys;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const SysParams& P = s->P;
  for (int sw = 0; sw < n_sweeps; ++sw) {
    WalkParams W = w->W;
    W.trace = nullptr;
    W.forced = nullptr;
    if (w->trace && w->traced < w->trace_sweeps)
      W.trace = w->trace + w->traced * (size_t)W.n_w * P.n_e * 8;
    if (w->d_forced && sw < w->forced_sweeps)
      W.forced = w->d_forced + (size_t)sw * W.n_w * P.n_e;
    if (w->graphs.enabled && !w->profiling && !W.trace && !W.forced) {
      qmc_status r = sweep_graph(w, st);
      if (r != QMC_OK) return r;
    } else {
      qmc_status r = sweep_once(w, W, w->sweep, false, st);
      if (r != QMC_OK) return r;
      r = measure_energy(w, W, w->sweep + 1, st);
      if (r != QMC_OK) return r;
    }
    if (W.trace) ++w->traced;
    ++w->sweep;
    w->proposed += (long long)W.n_w * P.n_e;
  }
  if (w->d_forced) {
    QMC_CUDA(cudaStreamSynchronize(st));
    cudaFree(w->d_forced);
    w->d_forced = nullptr;
    w->forced_sweeps = 0;
  }
  w->energy_valid = true;
  w->energy_version = w->sys->ham_version;
  return QMC_OK;
}

extern "C" qmc_status qmc_measure(qmc_walkers_t w, double* e_local, double* log_psi, void* stream) {
  if (!w) return fail(QMC_EINVAL, "qmc_measure: NULL walkers");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (!w->energy_valid || w->energy_version != w->sys->ham_version) {
    qmc_status r = measure_energy(w, w->W, w->sweep, st);
    if (r != QMC_OK) return r;
    w->energy_valid = true;
    w->energy_version = w->sys->ham_version;
  }
  const size_t b = sizeof(double) * w->W.n_w;
  if (e_local) QMC_CUDA(cudaMemcpyAsync(e_local, w->W.e_loc, b, cudaMemcpyDefault, st));
  if (log_psi) QMC_CUDA(cudaMemcpyAsync(log_psi, w->W.log_psi, b, cudaMemcpyDefault, st));
  const bool host = (e_local && !is_device_ptr(e_local)) || (log_psi && !is_device_ptr(log_psi));
  if (host) return check_err(w, st);
  return QMC_OK;
}

extern "C" qmc_status qmc_accumulate_energy(qmc_walkers_t w, double* out, void* stream) {
  if (!w || !out) return fail(QMC_EINVAL, "qmc_accumulate_energy: NULL argument");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  { Bracket b(w, st, QMC_K_ACCUMULATE); QMC_CUDA(launch_accumulate(w->W, w->d_out, w->d_nacc, st)); }
  double h[4];
  long long nacc = 0;
  QMC_CUDA(cudaMemcpyAsync(h, w->d_out, 3 * sizeof(double), cudaMemcpyDeviceToHost, st));
  QMC_CUDA(cudaMemcpyAsync(&nacc, w->d_nacc, sizeof(long long), cudaMemcpyDeviceToHost, st));
  qmc_status r = check_err(w, st);
  if (r != QMC_OK) return r;
  h[3] = w->proposed > 0 ? (double)nacc / (double)w->proposed : 0.0;
  w->proposed = 0;
  QMC_CUDA(cudaMemcpy(out, h, sizeof h, cudaMemcpyDefault));
  return QMC_OK;
}

extern "C" qmc_status qmc_trace_enable(qmc_walkers_t w, void* dev_buf, size_t bytes) {
  if (!w) return fail(QMC_EINVAL, "qmc_trace_enable: NULL walkers");
  if (!dev_buf || bytes == 0) {
    w->trace = nullptr;
    w->trace_sweeps = 0;
    w->traced = 0;
    return QMC_OK;
  }
  if (!is_device_ptr(dev_buf)) return fail(QMC_EINVAL, "qmc_trace_enable: the buffer must be device memory");
  const size_t per = (size_t)w->W.n_w * w->sys->P.n_e * 8 * sizeof(double);
  if (bytes < per) return fail(QMC_EINVAL, "qmc_trace_enable: buffer smaller than one sweep (%zu bytes)", per);
  w->trace = static_cast<double*>(dev_buf);
  w->trace_sweeps = bytes / per;
  w->traced = 0;
  return QMC_OK;
}

extern "C" qmc_status qmc_replay_decisions(qmc_walkers_t w, const uint8_t* bits, int n_sweeps) {
  if (!w) return fail(QMC_EINVAL, "qmc_replay_decisions: NULL walkers");
  if (w->d_forced) {
    cudaFree(w->d_forced);
    w->d_forced = nullptr;
    w->forced_sweeps = 0;
  }
  if (!bits || n_sweeps <= 0) return QMC_OK;
  const size_t n = (size_t)n_sweeps * w->W.n_w * w->sys->P.n_e;
  QMC_CUDA(cudaMalloc(&w->d_forced, n));
  QMC_CUDA(cudaMemcpy(w->d_forced, bits, n, cudaMemcpyDefault));
  w->forced_sweeps = n_sweeps;
  return QMC_OK;
}

extern "C" qmc_status qmc_get_positions(qmc_walkers_t w, double* pos, void* stream) {
  if (!w || !pos) return fail(QMC_EINVAL, "qmc_get_positions: NULL argument");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  qmc_status r = check_err(w, st);
  if (r != QMC_OK) return r;
  const int nw = w->W.n_w, ne = w->sys->P.n_e;
  std::vector<double> h((size_t)nw * ne * 3), o(h.size());
  QMC_CUDA(cudaMemcpy(h.data(), w->W.pos, h.size() * sizeof(double), cudaMemcpyDeviceToHost));
  for (int a = 0; a < nw; ++a)
    for (int c = 0; c < 3; ++c)
      for (int e = 0; e < ne; ++e) o[((size_t)a * ne + e) * 3 + c] = h[((size_t)a * 3 + c) * ne + e];
  QMC_CUDA(cudaMemcpy(pos, o.data(), o.size() * sizeof(double), cudaMemcpyDefault));
  return QMC_OK;
}

namespace {
struct StateHeader {
  uint64_t magic, seed;
  int32_t n_w, n_e, n_up, pad;
  uint32_t sweep, pad2;
};
constexpr uint64_t kMagic = 0x31305f4354415453ull;   // "STATE_01"
}  // namespace

extern "C" qmc_status qmc_get_state(qmc_walkers_t w, void* buf, size_t* len) {
  if (!w || !len) return fail(QMC_EINVAL, "qmc_get_state: NULL argument");
  const int nw = w->W.n_w, ne = w->sys->P.n_e;
  const size_t need = sizeof(StateHeader) + (size_t)nw * ne * 3 * sizeof(double) +
                      (size_t)nw * (sizeof(uint32_t) + sizeof(double));
  if (!buf) {
    *len = need;
    return QMC_OK;
  }
  if (*len < need) return fail(QMC_EINVAL, "qmc_get_state: buffer too small (%zu < %zu)", *len, need);
  qmc_status r = check_err(w, 0);
  if (r != QMC_OK) return r;
  StateHeader h{kMagic, w->sys->d.seed, nw, ne, w->sys->P.n_up, 0, w->sweep, 0};
  char* p = static_cast<char*>(buf);
  std::memcpy(p, &h, sizeof h);
  p += sizeof h;
  r = qmc_get_positions(w, reinterpret_cast<double*>(p), nullptr);
  if (r != QMC_OK) return r;
  p += (size_t)nw * ne * 3 * sizeof(double);
  QMC_CUDA(cudaMemcpy(p, w->W.wid, nw * sizeof(uint32_t), cudaMemcpyDeviceToHost));
  p += nw * sizeof(uint32_t);
  QMC_CUDA(cudaMemcpy(p, w->W.weight, nw * sizeof(double), cudaMemcpyDeviceToHost));
  *len = need;
  return QMC_OK;
}

extern "C" qmc_status qmc_set_state(qmc_walkers_t w, const void* buf, size_t len) {
  if (!w || !buf) return fail(QMC_EINVAL, "qmc_set_state: NULL argument");
  StateHeader h;
  if (len < sizeof h) return fail(QMC_ESTATE, "qmc_set_state: truncated state");
  std::memcpy(&h, buf, sizeof h);
  const int nw = w->W.n_w, ne = w->sys->P.n_e;
  const size_t need = sizeof(StateHeader) + (size_t)nw * ne * 3 * sizeof(double) +
                      (size_t)nw * (sizeof(uint32_t) + sizeof(double));
  if (h.magic != kMagic || h.n_w != nw || h.n_e != ne || h.n_up != w->sys->P.n_up ||
      h.seed != w->sys->d.seed || len != need)
    return fail(QMC_ESTATE, "qmc_set_state: state does not match this walker set");
  const char* p = static_cast<const char*>(buf) + sizeof h;
  qmc_status r = upload_positions(w, reinterpret_cast<const double*>(p), false);
  if (r != QMC_OK) return r;
  p += (size_t)nw * ne * 3 * sizeof(double);
  QMC_CUDA(cudaMemcpy(w->W.wid, p, nw * sizeof(uint32_t), cudaMemcpyHostToDevice));
  p += nw * sizeof(uint32_t);
  QMC_CUDA(cudaMemcpy(w->W.weight, p, nw * sizeof(double), cudaMemcpyHostToDevice));
  w->sweep = h.sweep;
  return setup_state(w, 0);
}

namespace {
// Copies n elements of working precision at dev to host doubles.
qmc_status fetch_tw(const qmc_walkers_s* w, const void* dev, size_t n, std::vector<double>& out) {
  out.resize(n);
  if (w->sys->tw->tw_size == sizeof(double)) {
    QMC_CUDA(cudaMemcpy(out.data(), dev, n * sizeof(double), cudaMemcpyDeviceToHost));
  } else {
    std::vector<float> f(n);
    QMC_CUDA(cudaMemcpy(f.data(), dev, n * sizeof(float), cudaMemcpyDeviceToHost));
    for (size_t i = 0; i < n; ++i) out[i] = f[i];
  }
  return QMC_OK;
}
}  // namespace

extern "C" qmc_status qmc_get_inverse(qmc_walkers_t w, int walker, int spin, double* out) {
  if (!w || !out) return fail(QMC_EINVAL, "qmc_get_inverse: NULL argument");
  const SysParams& P = w->sys->P;
  if (walker < 0 || walker >= w->W.n_w || spin < 0 || spin > 1)
    return fail(QMC_EINVAL, "qmc_get_inverse: walker or spin out of range");
  qmc_status r = check_err(w, 0);
  if (r != QMC_OK) return r;
  const size_t ns = spin ? P.n_dn : P.n_up;
  std::vector<double> h;
  r = fetch_tw(w, static_cast<const char*>(w->W.binv[spin]) + (size_t)walker * ns * ns * w->sys->tw->tw_size,
               ns * ns, h);
  if (r != QMC_OK) return r;
  QMC_CUDA(cudaMemcpy(out, h.data(), h.size() * sizeof(double), cudaMemcpyDefault));
  return QMC_OK;
}

extern "C" qmc_status qmc_get_orbitals(qmc_walkers_t w, int walker, double* out) {
  if (!w || !out) return fail(QMC_EINVAL, "qmc_get_orbitals: NULL argument");
  const SysParams& P = w->sys->P;
  if (walker < 0 || walker >= w->W.n_w) return fail(QMC_EINVAL, "qmc_get_orbitals: walker out of range");
  qmc_status r = check_err(w, 0);
  if (r != QMC_OK) return r;
  const int ld = w->W.ld_v, nsm = std::max(P.n_up, P.n_dn);
  std::vector<double> h;
  r = fetch_tw(w, static_cast<const char*>(w->W.vgl) + (size_t)walker * P.n_e * 5 * ld * w->sys->tw->tw_size,
               (size_t)P.n_e * 5 * ld, h);
  if (r != QMC_OK) return r;
  std::vector<double> o((size_t)P.n_e * 5 * nsm, 0.0);
  for (int e = 0; e < P.n_e; ++e)
    for (int c = 0; c < 5; ++c)
      for (int j = 0; j < nsm; ++j) o[((size_t)e * 5 + c) * nsm + j] = h[((size_t)e * 5 + c) * ld + j];
  QMC_CUDA(cudaMemcpy(out, o.data(), o.size() * sizeof(double), cudaMemcpyDefault));
  return QMC_OK;
}

extern "C" qmc_status qmc_get_nonlocal(qmc_walkers_t w, double* out) {
  if (!w || !out) return fail(QMC_EINVAL, "qmc_get_nonlocal: NULL argument");
  qmc_status r = check_err(w, 0);
  if (r != QMC_OK) return r;
  if (w->sys->P.nl_nch == 0 || w->sys->P.n_ion == 0) {
    std::vector<double> z(w->W.n_w, 0.0);
    QMC_CUDA(cudaMemcpy(out, z.data(), z.size() * sizeof(double), cudaMemcpyDefault));
    return QMC_OK;
  }
  QMC_CUDA(cudaMemcpy(out, w->W.vnl, sizeof(double) * w->W.n_w, cudaMemcpyDefault));
  return QMC_OK;
}

extern "C" qmc_status qmc_get_logdet(qmc_walkers_t w, double* logdet, double* sign) {
  if (!w || (!logdet && !sign)) return fail(QMC_EINVAL, "qmc_get_logdet: NULL argument");
  qmc_status r = check_err(w, 0);
  if (r != QMC_OK) return r;
  const size_t b = sizeof(double) * 2 * (size_t)w->W.n_w;
  if (logdet) QMC_CUDA(cudaMemcpy(logdet, w->W.logdet, b, cudaMemcpyDefault));
  if (sign) QMC_CUDA(cudaMemcpy(sign, w->W.sgn, b, cudaMemcpyDefault));
  return QMC_OK;
}

extern "C" qmc_status qmc_get_precision_report(qmc_walkers_t w, double* residual,
                                               double* logdet_shift) {
  if (!w || (!residual && !logdet_shift))
    return fail(QMC_EINVAL, "qmc_get_precision_report: NULL argument");
  qmc_status r = check_err(w, 0);
  if (r != QMC_OK) return r;
  const size_t n = 2 * (size_t)w->W.n_w;
  std::vector<float> f(n);
  std::vector<double> h(n);
  const float* src[2] = {w->W.refine_last, w->W.logdet_shift};
  double* dst[2] = {residual, logdet_shift};
  for (int k = 0; k < 2; ++k) {
    if (!dst[k]) continue;
    QMC_CUDA(cudaMemcpy(f.data(), src[k], n * sizeof(float), cudaMemcpyDeviceToHost));
    for (size_t i = 0; i < n; ++i) h[i] = f[i];
    QMC_CUDA(cudaMemcpy(dst[k], h.data(), n * sizeof(double), cudaMemcpyDefault));
  }
  return QMC_OK;
}

extern "C" qmc_status qmc_check_errors(qmc_walkers_t w, void* stream) {
  if (!w) return fail(QMC_EINVAL, "qmc_check_errors: NULL walkers");
  return check_err(w, static_cast<cudaStream_t>(stream));
}

extern "C" int64_t qmc_launch_count(qmc_walkers_t w) { return w ? w->launches : 0; }

extern "C" qmc_status qmc_graph_enable(qmc_walkers_t w, int enable) {
  if (!w) return fail(QMC_EINVAL, "qmc_graph_enable: NULL walkers");
  w->graphs.enabled = enable != 0;
  return QMC_OK;
}

extern "C" qmc_status qmc_graph_stats(qmc_walkers_t w, int64_t* captures, int64_t* replays) {
  if (!w) return fail(QMC_EINVAL, "qmc_graph_stats: NULL walkers");
  if (captures) *captures = w->graphs.captures;
  if (replays) *replays = w->graphs.replays;
  return QMC_OK;
}

extern "C" qmc_status qmc_profile_enable(qmc_walkers_t w, int enable) {
  if (!w) return fail(QMC_EINVAL, "qmc_profile_enable: NULL walkers");
  w->profiling = enable != 0;
  return QMC_OK;
}

extern "C" qmc_status qmc_profile_read(qmc_walkers_t w, double* ms, int64_t* launches) {
  if (!w) return fail(QMC_EINVAL, "qmc_profile_read: NULL walkers");
  drain_events(w);
  for (int k = 0; k < QMC_NKERNELS; ++k) {
    if (ms) ms[k] = w->prof_ms[k];
    if (launches) launches[k] = w->prof_n[k];
    w->prof_ms[k] = 0.0;
    w->prof_n[k] = 0;
  }
  return QMC_OK;
}

extern "C" void qmc_walkers_destroy(qmc_walkers_t w) {
  if (!w) return;
  cudaDeviceSynchronize();
  drain_events(w);
  free_walkers(w);
  delete w;
}

// ------------------------------------------------------------------------ standalone S8
extern "C" qmc_status qmc_slater_invert(qmc_precision prec, const void* A, void* Binv,
                                        double* logdet, double* sign, int n, int batch,
                                        void* stream) {
  if (!A || !Binv) return fail(QMC_EINVAL, "qmc_slater_invert: NULL matrix pointer");
  if (prec < QMC_FP64 || prec > QMC_FP32_BF16TAB) return fail(QMC_EINVAL, "qmc_slater_invert: unknown precision");
  if (n < 1 || n > 1024) return fail(QMC_EINVAL, "qmc_slater_invert: n must be in [1, 1024]");
  if (batch < 1 || batch > (1 << 20)) return fail(QMC_EINVAL, "qmc_slater_invert: batch must be in [1, 2^20]");
  if (!is_device_ptr(A) || !is_device_ptr(Binv) || (logdet && !is_device_ptr(logdet)) ||
      (sign && !is_device_ptr(sign)))
    return fail(QMC_EINVAL, "qmc_slater_invert: every array must be device memory");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const TwLaunch& tw = prec == QMC_FP64 ? tw_launch_f64() : tw_launch_f32();
  double* work = nullptr;
  QMC_CUDA(cudaMallocAsync(reinterpret_cast<void**>(&work), (size_t)batch * n * n * sizeof(double), st));
  const cudaError_t e = tw.invert_batch(A, Binv, logdet, sign, n, batch, work, st);
  const cudaError_t f = cudaFreeAsync(work, st);
  QMC_CUDA(e);
  QMC_CUDA(f);
  return QMC_OK;
}

// ------------------------------------------------------------------------ DMC
struct qmc_dmc_s {
  struct Sys {
    qmc_system_s* sys = nullptr;
    qmc_walkers_s* w[2] = {nullptr, nullptr};   // two slot buffers; walkers move on branching
    DmcParams D{};
    double* e_old[2] = {nullptr, nullptr};
    int parity = 0;
    cudaStream_t st = nullptr;
  };
  std::vector<Sys> sys;
  uint32_t step = 0;
  cudaEvent_t ev_in = nullptr, ev_done = nullptr;
  std::vector<cudaEvent_t> ev_out;
  GraphCache graphs;
  cudaStream_t cap = nullptr;  // capture stream of the step graphs
  uint32_t* d_t = nullptr;     // device step index read by replayed graphs
};

namespace {
void free_dmc(qmc_dmc_s* d) {
  for (auto& y : d->sys) {
    for (auto* w : y.w)
      if (w) { free_walkers(w); delete w; }
    cudaFree(y.e_old[0]);
    cudaFree(y.e_old[1]);
    cudaFree(y.D.src_of);
    cudaFree(y.D.wid_next);
    cudaFree(y.D.n_live);
    cudaFree(y.D.next_id);
    cudaFree(y.D.e_trial);
    cudaFree(y.D.stats);
    if (y.st) cudaStreamDestroy(y.st);
  }
  if (d->ev_in) cudaEventDestroy(d->ev_in);
  if (d->ev_done) cudaEventDestroy(d->ev_done);
  for (auto e : d->ev_out) cudaEventDestroy(e);
  d->graphs.clear();
  cudaFree(d->d_t);
  if (d->cap) cudaStreamDestroy(d->cap);
  delete d;
}
}  // namespace

extern "C" qmc_status qmc_dmc_create(qmc_system_t const* systems, const int* n_walkers,
                                     const double* const* positions, const double* e_trial,
                                     int n_systems, int capacity_factor, qmc_dmc_t* out) {
  if (!systems || !n_walkers || !positions || !e_trial || !out)
    return fail(QMC_EINVAL, "qmc_dmc_create: NULL argument");
  *out = nullptr;
  if (n_systems < 1 || n_systems > 64) return fail(QMC_EINVAL, "qmc_dmc_create: n_systems must be in [1, 64]");
  if (capacity_factor < 1 || capacity_factor > 8)
    return fail(QMC_EINVAL, "qmc_dmc_create: capacity_factor must be in [1, 8]");
  qmc_dmc_s* d = new qmc_dmc_s;
  d->sys.resize(n_systems);
  for (int i = 0; i < n_systems; ++i) {
    qmc_system_s* s = systems[i];
    auto& y = d->sys[i];
    y.sys = s;
    if (!s || !s->has_spline || !positions[i]) { free_dmc(d); return fail(QMC_EINVAL, "qmc_dmc_create: system %d incomplete", i); }
    if (s->d.move != QMC_MOVE_DRIFT) { free_dmc(d); return fail(QMC_EINVAL, "qmc_dmc_create: system %d must use drift moves", i); }
    const int n0 = n_walkers[i];
    const int cap = n0 * capacity_factor;
    if (n0 < 1 || cap > 1024 * 1024) { free_dmc(d); return fail(QMC_EINVAL, "qmc_dmc_create: bad walker count for system %d", i); }
    qmc_status st = alloc_walkers(s, cap, false, &y.w[0]);
    if (st == QMC_OK) st = alloc_walkers(s, cap, false, &y.w[1]);
    if (st == QMC_OK) st = init_walkers(y.w[0], n0, positions[i]);
    if (st != QMC_OK) { const std::string m = g_err; free_dmc(d); g_err = m; return st; }
    DmcParams& D = y.D;
    cudaError_t e = cudaSuccess;
    e = e ? e : cudaMalloc(&y.e_old[0], cap * sizeof(double));
    e = e ? e : cudaMalloc(&y.e_old[1], cap * sizeof(double));
    e = e ? e : cudaMalloc(&D.src_of, cap * sizeof(int));
    e = e ? e : cudaMalloc(&D.wid_next, cap * sizeof(uint32_t));
    e = e ? e : cudaMalloc(&D.n_live, 2 * sizeof(int));
    e = e ? e : cudaMalloc(&D.next_id, sizeof(uint32_t));
    e = e ? e : cudaMalloc(&D.e_trial, sizeof(double));
    e = e ? e : cudaMalloc(&D.stats, 8 * sizeof(double));
    e = e ? e : cudaStreamCreateWithFlags(&y.st, cudaStreamNonBlocking);
    if (e != cudaSuccess) { free_dmc(d); return fail(QMC_ENOMEM, "qmc_dmc_create: %s", cudaGetErrorString(e)); }
    const int live[2] = {n0, 0};
    const uint32_t nid = (uint32_t)n0;
    cudaMemcpy(D.n_live, live, sizeof live, cudaMemcpyHostToDevice);
    cudaMemcpy(D.next_id, &nid, sizeof nid, cudaMemcpyHostToDevice);
    cudaMemcpy(D.e_trial, &e_trial[i], sizeof(double), cudaMemcpyHostToDevice);
    cudaMemset(D.stats, 0, 8 * sizeof(double));
    cudaMemcpy(y.e_old[0], y.w[0]->W.e_loc, n0 * sizeof(double), cudaMemcpyDeviceToDevice);
    D.n_target = n0;
    D.cap = cap;
    D.tau = s->d.step;
    for (int b = 0; b < 2; ++b) {
      y.w[b]->W.n_w = cap;
      y.w[b]->W.n_live = D.n_live + b;
    }
  }
  d->ev_out.resize(n_systems);
  cudaError_t e = cudaEventCreateWithFlags(&d->ev_in, cudaEventDisableTiming);
  e = e ? e : cudaEventCreateWithFlags(&d->ev_done, cudaEventDisableTiming);
  for (auto& v : d->ev_out) e = e ? e : cudaEventCreateWithFlags(&v, cudaEventDisableTiming);
  e = e ? e : cudaStreamCreateWithFlags(&d->cap, cudaStreamNonBlocking);
  e = e ? e : cudaMalloc(&d->d_t, sizeof(uint32_t));
  if (e != cudaSuccess) { free_dmc(d); return fail(QMC_ECUDA, "qmc_dmc_create: %s", cudaGetErrorString(e)); }
  *out = d;
  return QMC_OK;
}

namespace {
// One DMC step of every system, each on its own stream: drift-diffusion sweep, local energy,
// branching weights and copy counts, copies into the other slot buffer. t: the step index of
// the Philox counters (an offset from *t_base when that is set).
qmc_status dmc_step_once(qmc_dmc_s* d, uint32_t t, const uint32_t* t_base) {
  for (auto& y : d->sys) {
    qmc_walkers_s* w = y.w[y.parity];
    qmc_walkers_s* w2 = y.w[y.parity ^ 1];
    WalkParams W = w->W;
    W.trace = nullptr;
    W.forced = nullptr;
    W.t_base = t_base;
    QMC_CUDA(cudaMemsetAsync(W.r2, 0, sizeof(double) * 2 * (size_t)W.n_w, y.st));
    qmc_status r = sweep_once(w, W, t, true, y.st);
    if (r != QMC_OK) return r;
    r = measure_energy(w, W, t + 1, y.st);
    if (r != QMC_OK) return r;
    DmcParams D = y.D;
    D.e_old = y.e_old[y.parity];
    D.e_old_next = y.e_old[y.parity ^ 1];
    {
      Bracket b(w, y.st, QMC_K_BRANCH);
      QMC_CUDA(y.sys->tw->dmc_branch(y.sys->P, W, D, y.parity, t, y.st));
      QMC_CUDA(y.sys->tw->dmc_copy(y.sys->P, W, w2->W, D, y.parity, y.st));
    }
    w->launches += 1;   // the copy kernel after the branching kernel
    y.parity ^= 1;
  }
  return QMC_OK;
}

// The host state a DMC step changes, and the key of its graph.
void put_dmc_state(Bytes& b, const qmc_dmc_s* d) {
  for (auto& y : d->sys) {
    put(b, y.parity);
    put_state(b, y.w[0]);
    put_state(b, y.w[1]);
  }
}

void take_dmc_state(const unsigned char*& p, qmc_dmc_s* d) {
  for (auto& y : d->sys) {
    take(p, y.parity);
    take_state(p, y.w[0]);
    take_state(p, y.w[1]);
  }
}

void put_dmc_key(Bytes& b, const qmc_dmc_s* d) {
  for (auto& y : d->sys) {
    put(b, y.D);
    put(b, y.e_old);
    put_walker_key(b, y.w[0]);
    put_walker_key(b, y.w[1]);
  }
  put_dmc_state(b, d);
}

// One step of every system as a graph on stream cs (captured on the driver's capture
// stream the first time its starting state is met, then replayed), its systems' streams
// made to wait for it so that the per-system reads see its results.
qmc_status dmc_step_graph(qmc_dmc_s* d, cudaStream_t cs) {
  Bytes key;
  put_dmc_key(key, d);
  GraphEntry* g = d->graphs.find(key);
  if (!g) {
    Bytes pre;
    put_dmc_state(pre, d);
    std::vector<int64_t> l0;
    for (auto& y : d->sys) {
      l0.push_back(y.w[0]->launches);
      l0.push_back(y.w[1]->launches);
    }
    QMC_CUDA(cudaStreamBeginCapture(d->cap, cudaStreamCaptureModeRelaxed));
    qmc_status r = QMC_OK;
    if (cudaEventRecord(d->ev_in, d->cap) != cudaSuccess) r = fail(QMC_ECUDA, "qmc_dmc_step: capture fork");
    for (auto& y : d->sys)
      if (r == QMC_OK && cudaStreamWaitEvent(y.st, d->ev_in, 0) != cudaSuccess)
        r = fail(QMC_ECUDA, "qmc_dmc_step: capture fork");
    if (r == QMC_OK) r = dmc_step_once(d, 0u, d->d_t);
    for (size_t i = 0; r == QMC_OK && i < d->sys.size(); ++i)
      if (cudaEventRecord(d->ev_out[i], d->sys[i].st) != cudaSuccess ||
          cudaStreamWaitEvent(d->cap, d->ev_out[i], 0) != cudaSuccess)
        r = fail(QMC_ECUDA, "qmc_dmc_step: capture join");
    cudaGraphExec_t exec = nullptr;
    r = end_capture(d->cap, r, &exec);
    std::vector<int64_t> n;
    size_t k = 0;
    for (auto& y : d->sys)
      for (auto* w : y.w) {
        n.push_back(w->launches - l0[k]);
        w->launches = l0[k++];
      }
    Bytes post;
    put_dmc_state(post, d);
    const unsigned char* p = pre.data();
    take_dmc_state(p, d);
    if (r != QMC_OK) return r;
    g = &d->graphs.slot();
    g->key = std::move(key);
    g->post = std::move(post);
    g->exec = exec;
    g->launches = std::move(n);
    ++d->graphs.captures;
  }
  for (auto& y : d->sys) y.w[y.parity]->sweep = d->step;
  QMC_CUDA(launch_set_word(d->d_t, d->step, cs));
  QMC_CUDA(cudaGraphLaunch(g->exec, cs));
  QMC_CUDA(cudaEventRecord(d->ev_done, cs));
  for (auto& y : d->sys) QMC_CUDA(cudaStreamWaitEvent(y.st, d->ev_done, 0));
  const unsigned char* p = g->post.data();
  take_dmc_state(p, d);
  size_t k = 0;
  for (auto& y : d->sys)
    for (auto* w : y.w) w->launches += g->launches[k++];
  d->sys[0].w[0]->launches += 1;   // the sweep-index launch
  g->used = ++d->graphs.clock;
  ++d->graphs.replays;
  return QMC_OK;
}
}  // namespace

extern "C" qmc_status qmc_dmc_step(qmc_dmc_t d, int n_steps, void* stream) {
  if (!d) return fail(QMC_EINVAL, "qmc_dmc_step: NULL driver");
  if (n_steps < 0) return fail(QMC_EINVAL, "qmc_dmc_step: n_steps < 0");
  cudaStream_t cs = static_cast<cudaStream_t>(stream);
  bool graphs = d->graphs.enabled;
  for (auto& y : d->sys)
    for (auto* w : y.w) graphs = graphs && !w->profiling;
  if (graphs) {
    for (int k = 0; k < n_steps; ++k) {
      qmc_status r = dmc_step_graph(d, cs);
      if (r != QMC_OK) return r;
      ++d->step;
    }
    return QMC_OK;
  }
  QMC_CUDA(cudaEventRecord(d->ev_in, cs));
  for (auto& y : d->sys) QMC_CUDA(cudaStreamWaitEvent(y.st, d->ev_in, 0));
  for (int k = 0; k < n_steps; ++k) {
    // the systems advance concurrently, one stream each
    for (auto& y : d->sys) y.w[y.parity]->sweep = d->step;
    qmc_status r = dmc_step_once(d, d->step, nullptr);
    if (r != QMC_OK) return r;
    ++d->step;
  }
  for (size_t i = 0; i < d->sys.size(); ++i) {
    QMC_CUDA(cudaEventRecord(d->ev_out[i], d->sys[i].st));
    QMC_CUDA(cudaStreamWaitEvent(cs, d->ev_out[i], 0));
  }
  return QMC_OK;
}

extern "C" qmc_status qmc_dmc_profile_enable(qmc_dmc_t d, int enable) {
  if (!d) return fail(QMC_EINVAL, "qmc_dmc_profile_enable: NULL driver");
  for (auto& y : d->sys)
    for (auto* w : y.w) w->profiling = enable != 0;
  return QMC_OK;
}

extern "C" qmc_status qmc_dmc_profile_read(qmc_dmc_t d, int system, double* ms, int64_t* launches) {
  if (!d) return fail(QMC_EINVAL, "qmc_dmc_profile_read: NULL driver");
  if (system < 0 || system >= (int)d->sys.size()) return fail(QMC_EINVAL, "qmc_dmc_profile_read: bad system");
  double acc_ms[QMC_NKERNELS] = {0};
  int64_t acc_n[QMC_NKERNELS] = {0};
  for (auto* w : d->sys[system].w) {
    drain_events(w);
    for (int k = 0; k < QMC_NKERNELS; ++k) {
      acc_ms[k] += w->prof_ms[k];
      acc_n[k] += w->prof_n[k];
      w->prof_ms[k] = 0.0;
      w->prof_n[k] = 0;
    }
  }
  for (int k = 0; k < QMC_NKERNELS; ++k) {
    if (ms) ms[k] = acc_ms[k];
    if (launches) launches[k] = acc_n[k];
  }
  return QMC_OK;
}

extern "C" qmc_status qmc_dmc_set_mode(qmc_dmc_t d, int effective_tau, int reconfigure) {
  if (!d) return fail(QMC_EINVAL, "qmc_dmc_set_mode: NULL driver");
  for (auto& y : d->sys) {
    y.D.tau_eff = effective_tau != 0;
    y.D.reconfigure = reconfigure != 0;
  }
  return QMC_OK;
}

extern "C" qmc_status qmc_dmc_read(qmc_dmc_t d, int system, double* out) {
  if (!d || !out) return fail(QMC_EINVAL, "qmc_dmc_read: NULL argument");
  if (system < 0 || system >= (int)d->sys.size()) return fail(QMC_EINVAL, "qmc_dmc_read: bad system");
  auto& y = d->sys[system];
  QMC_CUDA(cudaStreamSynchronize(y.st));
  qmc_status r = check_err(y.w[0], y.st);
  if (r == QMC_OK) r = check_err(y.w[1], y.st);
  if (r != QMC_OK) return r;
  double st[8];
  int live[2];
  uint32_t nid;
  double et;
  QMC_CUDA(cudaMemcpy(st, y.D.stats, sizeof st, cudaMemcpyDeviceToHost));
  QMC_CUDA(cudaMemcpy(live, y.D.n_live, sizeof live, cudaMemcpyDeviceToHost));
  QMC_CUDA(cudaMemcpy(&nid, y.D.next_id, sizeof nid, cudaMemcpyDeviceToHost));
  QMC_CUDA(cudaMemcpy(&et, y.D.e_trial, sizeof et, cudaMemcpyDeviceToHost));
  const double o[8] = {(double)live[y.parity], st[0], st[1], st[2], st[3], et, (double)nid, st[4]};
  QMC_CUDA(cudaMemcpy(out, o, sizeof o, cudaMemcpyDefault));
  return QMC_OK;
}

extern "C" qmc_status qmc_dmc_walkers(qmc_dmc_t d, int system, int max_walkers, double* pos,
                                      uint32_t* ids, double* e_local, int* n_out) {
  if (!d || !n_out) return fail(QMC_EINVAL, "qmc_dmc_walkers: NULL argument");
  if (system < 0 || system >= (int)d->sys.size()) return fail(QMC_EINVAL, "qmc_dmc_walkers: bad system");
  auto& y = d->sys[system];
  QMC_CUDA(cudaStreamSynchronize(y.st));
  int live[2];
  QMC_CUDA(cudaMemcpy(live, y.D.n_live, sizeof live, cudaMemcpyDeviceToHost));
  const int n = live[y.parity];
  *n_out = n;
  if (n > max_walkers) return fail(QMC_EINVAL, "qmc_dmc_walkers: %d walkers do not fit in %d", n, max_walkers);
  qmc_walkers_s* w = y.w[y.parity];
  const int ne = y.sys->P.n_e;
  if (pos) {
    std::vector<double> h((size_t)n * ne * 3), o(h.size());
    QMC_CUDA(cudaMemcpy(h.data(), w->W.pos, h.size() * sizeof(double), cudaMemcpyDeviceToHost));
    for (int a = 0; a < n; ++a)
      for (int c = 0; c < 3; ++c)
        for (int e = 0; e < ne; ++e) o[((size_t)a * ne + e) * 3 + c] = h[((size_t)a * 3 + c) * ne + e];
    QMC_CUDA(cudaMemcpy(pos, o.data(), o.size() * sizeof(double), cudaMemcpyDefault));
  }
  if (ids) QMC_CUDA(cudaMemcpy(ids, w->W.wid, n * sizeof(uint32_t), cudaMemcpyDefault));
  if (e_local) QMC_CUDA(cudaMemcpy(e_local, w->W.e_loc, n * sizeof(double), cudaMemcpyDefault));
  return QMC_OK;
}

extern "C" qmc_status qmc_dmc_graph_enable(qmc_dmc_t d, int enable) {
  if (!d) return fail(QMC_EINVAL, "qmc_dmc_graph_enable: NULL driver");
  d->graphs.enabled = enable != 0;
  return QMC_OK;
}

extern "C" qmc_status qmc_dmc_graph_stats(qmc_dmc_t d, int64_t* captures, int64_t* replays) {
  if (!d) return fail(QMC_EINVAL, "qmc_dmc_graph_stats: NULL driver");
  if (captures) *captures = d->graphs.captures;
  if (replays) *replays = d->graphs.replays;
  return QMC_OK;
}

extern "C" int64_t qmc_dmc_launch_count(qmc_dmc_t d) {
  if (!d) return 0;
  int64_t n = 0;
  for (auto& y : d->sys) n += y.w[0]->launches + y.w[1]->launches;
  return n;
}

extern "C" void qmc_dmc_destroy(qmc_dmc_t d) {
  if (!d) return;
  cudaDeviceSynchronize();
  for (auto& y : d->sys)
    for (auto* w : y.w) drain_events(w);
  free_dmc(d);
}
