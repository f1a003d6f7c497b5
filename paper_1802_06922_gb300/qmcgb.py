"""ctypes binding of libqmcgb (include/qmcgb.h): argument marshalling only.

Every step of the particle-by-particle path runs in the library's CUDA kernels. Loading
fails loudly (``RuntimeError``) when the library is missing or cannot be loaded; there is
no CPU fallback. Arrays may be numpy arrays (host memory) or torch tensors (host or CUDA
memory); they are passed to the library as plain pointers.
"""
from __future__ import annotations

import ctypes as C
import os
from dataclasses import dataclass
from typing import Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libqmcgb.so")

QMC_OK, QMC_EINVAL, QMC_ENOMEM, QMC_ECUDA, QMC_ESINGULAR, QMC_ETIMEOUT, QMC_ESTATE = 0, -1, -2, -3, -4, -5, -6
STATUS_NAMES = {0: "QMC_OK", -1: "QMC_EINVAL", -2: "QMC_ENOMEM", -3: "QMC_ECUDA",
                -4: "QMC_ESINGULAR", -5: "QMC_ETIMEOUT", -6: "QMC_ESTATE"}
PRECISIONS = {"fp64": 0, "fp32": 1, "bf16": 2}
KERNEL_CLASSES = ("propose", "vgl", "sweep", "energy", "reinvert", "vgl_current",
                  "accumulate", "flush", "refine", "refine_update", "logdet", "nlpp", "ewald",
                  "jastrow3", "branch")
MOVES = {"metropolis": 0, "drift": 1}

# Exported symbols and their ctypes signatures (argtypes, restype), as declared in
# include/qmcgb.h.
class SystemDesc(C.Structure):
    _fields_ = [("n_up", C.c_int), ("n_dn", C.c_int), ("L", C.c_double), ("n_ion", C.c_int),
                ("ion_pos", C.POINTER(C.c_double)), ("ion_Z", C.c_double),
                ("kappa", C.c_double), ("with_potential", C.c_int), ("prec", C.c_int),
                ("move", C.c_int), ("step", C.c_double), ("delay_k", C.c_int),
                ("reinv_period", C.c_int), ("reinv_on_accepted", C.c_int),
                ("seed", C.c_uint64), ("logdet_period", C.c_int), ("drift_a", C.c_double),
                ("prop_chunk", C.c_int)]


_vp, _i, _d, _sz = C.c_void_p, C.c_int, C.c_double, C.c_size_t
SIGNATURES = {
    "qmc_system_create": ([C.POINTER(SystemDesc), C.POINTER(_vp)], _i),
    "qmc_system_set_spline": ([_vp, _i, _i, _i, _i, _vp], _i),
    "qmc_system_set_jastrow": ([_vp, _i, _i, _d, _vp, _i, _d], _i),
    "qmc_system_set_nonlocal": ([_vp, _i, _vp, _vp, _d], _i),
    "qmc_system_set_ewald": ([_vp, _d, _d], _i),
    "qmc_system_set_jastrow3": ([_vp, _i, _i, _d, _vp, _vp], _i),
    "qmc_dmc_profile_enable": ([_vp, _i], _i),
    "qmc_dmc_profile_read": ([_vp, _i, _vp, _vp], _i),
    "qmc_system_ewald_count": ([_vp], _i),
    "qmc_get_nonlocal": ([_vp, _vp], _i),
    "qmc_walkers_create": ([_vp, _i, _vp, C.POINTER(_vp)], _i),
    "qmc_sweep": ([_vp, _i, _vp], _i),
    "qmc_measure": ([_vp, _vp, _vp, _vp], _i),
    "qmc_accumulate_energy": ([_vp, _vp, _vp], _i),
    "qmc_trace_enable": ([_vp, _vp, _sz], _i),
    "qmc_replay_decisions": ([_vp, _vp, _i], _i),
    "qmc_get_positions": ([_vp, _vp, _vp], _i),
    "qmc_get_state": ([_vp, _vp, C.POINTER(_sz)], _i),
    "qmc_set_state": ([_vp, _vp, _sz], _i),
    "qmc_get_inverse": ([_vp, _i, _i, _vp], _i),
    "qmc_get_orbitals": ([_vp, _i, _vp], _i),
    "qmc_check_errors": ([_vp, _vp], _i),
    "qmc_get_logdet": ([_vp, _vp, _vp], _i),
    "qmc_get_precision_report": ([_vp, _vp, _vp], _i),
    "qmc_launch_count": ([_vp], C.c_int64),
    "qmc_graph_enable": ([_vp, _i], _i),
    "qmc_graph_stats": ([_vp, _vp, _vp], _i),
    "qmc_dmc_graph_enable": ([_vp, _i], _i),
    "qmc_dmc_graph_stats": ([_vp, _vp, _vp], _i),
    "qmc_profile_enable": ([_vp, _i], _i),
    "qmc_profile_read": ([_vp, _vp, _vp], _i),
    "qmc_walkers_destroy": ([_vp], None),
    "qmc_system_destroy": ([_vp], None),
    "qmc_last_error": ([], C.c_char_p),
    "qmc_slater_invert": ([_i, _vp, _vp, _vp, _vp, _i, _i, _vp], _i),
    "qmc_slater_invert_noalloc": ([_i, _vp, _vp, _vp, _vp, _i, _i, _vp], _i),
    "qmc_dmc_create": ([_vp, _vp, _vp, _vp, _i, _i, C.POINTER(_vp)], _i),
    "qmc_dmc_step": ([_vp, _i, _vp], _i),
    "qmc_dmc_set_mode": ([_vp, _i, _i], _i),
    "qmc_dmc_read": ([_vp, _i, _vp], _i),
    "qmc_dmc_walkers": ([_vp, _i, _i, _vp, _vp, _vp, C.POINTER(_i)], _i),
    "qmc_dmc_launch_count": ([_vp], C.c_int64),
    "qmc_dmc_destroy": ([_vp], None),
    "qmc_measure_rates": ([_vp], _i),
}

_lib: Optional[C.CDLL] = None


def load(path: str = LIB_PATH) -> C.CDLL:
    """Load libqmcgb (building it first if it is missing or stale)."""
    global _lib
    if _lib is not None:
        return _lib
    from . import build as _build
    if not _build.up_to_date():
        _build.build()
    if not os.path.exists(path):
        raise RuntimeError(f"libqmcgb not found at {path}; run paper_1802_06922_gb300.build")
    lib = C.CDLL(path)
    for name, (args, res) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = res
    _lib = lib
    return lib


class QMCError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


def _check(status: int):
    if status != QMC_OK:
        raise QMCError(status, load().qmc_last_error().decode())


def _ptr(a) -> int:
    """Address of a contiguous numpy array or torch tensor."""
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        if not a.flags["C_CONTIGUOUS"]:
            raise ValueError("arrays must be C-contiguous")
        return a.ctypes.data
    if not a.is_contiguous():
        raise ValueError("tensors must be contiguous")
    return a.data_ptr()


def _stream_ptr(stream) -> int:
    if stream is None:
        return None
    return stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)


class System:
    """One system: cell, ions, orbital table, Jastrow functors, move parameters."""

    def __init__(self, n_up, n_dn, L, ions, precision="fp64", move="metropolis", step=0.3,
                 delay_k=1, reinv_period=0, reinv_on_accepted=False, seed=0, ion_Z=4.0,
                 kappa=1.0, with_potential=True, logdet_period=0, drift_a=0.0, prop_chunk=0):
        lib = load()
        ions = np.ascontiguousarray(np.asarray(ions, dtype=np.float64).reshape(-1, 3))
        self._ions = ions
        d = SystemDesc(int(n_up), int(n_dn), float(L), int(ions.shape[0]),
                       ions.ctypes.data_as(C.POINTER(C.c_double)), float(ion_Z), float(kappa),
                       int(bool(with_potential)), PRECISIONS[precision], MOVES[move],
                       float(step), int(delay_k), int(reinv_period), int(bool(reinv_on_accepted)),
                       int(seed) & 0xFFFFFFFFFFFFFFFF, int(logdet_period), float(drift_a),
                       int(prop_chunk))
        h = C.c_void_p()
        _check(lib.qmc_system_create(C.byref(d), C.byref(h)))
        self.h = h
        self.n_up, self.n_dn, self.L, self.precision = int(n_up), int(n_dn), float(L), precision

    def set_spline(self, coef: np.ndarray):
        coef = np.ascontiguousarray(coef, dtype=np.float64)
        nx, ny, nz, n_orb = coef.shape
        _check(load().qmc_system_set_spline(self.h, nx, ny, nz, n_orb, coef.ctypes.data))

    def set_jastrow(self, which: int, p, rcut: float, cusp: Optional[float] = None):
        p = np.ascontiguousarray(p, dtype=np.float64)
        _check(load().qmc_system_set_jastrow(self.h, int(which), p.shape[0] - 1, float(rcut),
                                             p.ctypes.data, int(cusp is not None),
                                             float(cusp or 0.0)))

    def set_nonlocal(self, amp, width, rcut: float):
        """Non-local pseudopotential channels dv_l(r) = amp[l] exp(-(r/width[l])^2), r < rcut
        (empty amp removes them)."""
        a = np.ascontiguousarray(amp, dtype=np.float64)
        b = np.ascontiguousarray(width, dtype=np.float64)
        _check(load().qmc_system_set_nonlocal(self.h, int(a.size), a.ctypes.data if a.size else None,
                                              b.ctypes.data if b.size else None, float(rcut)))

    def set_jastrow3(self, gamma_same, gamma_opp=None, rcut: float = 0.0):
        """Three-body e-e-I Jastrow term with coefficient arrays [M_eI+1][M_eI+1][M_ee+1]
        (gamma_opp defaults to gamma_same); None removes the term."""
        if gamma_same is None:
            _check(load().qmc_system_set_jastrow3(self.h, -1, 0, 0.0, None, None))
            return
        a = np.ascontiguousarray(gamma_same, dtype=np.float64)
        b = np.ascontiguousarray(a if gamma_opp is None else gamma_opp, dtype=np.float64)
        if a.ndim != 3 or a.shape[0] != a.shape[1] or b.shape != a.shape:
            raise ValueError("gamma arrays must have shape (M_eI + 1, M_eI + 1, M_ee + 1)")
        _check(load().qmc_system_set_jastrow3(self.h, a.shape[0] - 1, a.shape[2] - 1,
                                              float(rcut), a.ctypes.data, b.ctypes.data))

    def set_ewald(self, alpha: float, kcut: float = 0.0):
        """Coulomb interactions by Ewald summation with splitting parameter alpha and
        reciprocal cutoff kcut (alpha = 0 restores the Yukawa form)."""
        _check(load().qmc_system_set_ewald(self.h, float(alpha), float(kcut)))

    @property
    def ewald_count(self) -> int:
        """k vectors in the Ewald half set, -1 with the Yukawa form."""
        return int(load().qmc_system_ewald_count(self.h))

    def close(self):
        if getattr(self, "h", None):
            load().qmc_system_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Walkers:
    """A set of walkers of one system, resident on the GPU."""

    def __init__(self, system: System, positions):
        lib = load()
        self.system = system
        pos = positions
        if isinstance(pos, np.ndarray):
            pos = np.ascontiguousarray(pos, dtype=np.float64)
        self.n_w = int(pos.shape[0])
        self.n_e = system.n_up + system.n_dn
        h = C.c_void_p()
        _check(lib.qmc_walkers_create(system.h, self.n_w, _ptr(pos), C.byref(h)))
        self.h = h

    def sweep(self, n: int = 1, stream=None):
        _check(load().qmc_sweep(self.h, int(n), _stream_ptr(stream)))

    def measure(self, e_local=None, log_psi=None, stream=None):
        """Fill e_local / log_psi (numpy or torch, [n_w] float64); returns numpy copies
        when both are None."""
        if e_local is None and log_psi is None:
            e = np.zeros(self.n_w)
            l = np.zeros(self.n_w)
            _check(load().qmc_measure(self.h, e.ctypes.data, l.ctypes.data, _stream_ptr(stream)))
            return e, l
        _check(load().qmc_measure(self.h, _ptr(e_local), _ptr(log_psi), _stream_ptr(stream)))
        return e_local, log_psi

    def accumulate(self, out=None, stream=None):
        o = np.zeros(4) if out is None else out
        _check(load().qmc_accumulate_energy(self.h, _ptr(o), _stream_ptr(stream)))
        return o

    def trace_enable(self, buf, nbytes: Optional[int] = None):
        if buf is None:
            _check(load().qmc_trace_enable(self.h, None, 0))
            return
        nb = buf.numel() * buf.element_size() if nbytes is None else nbytes
        _check(load().qmc_trace_enable(self.h, _ptr(buf), nb))

    def replay(self, bits, n_sweeps: int):
        if bits is None:
            _check(load().qmc_replay_decisions(self.h, None, 0))
            return
        if isinstance(bits, np.ndarray):
            bits = np.ascontiguousarray(bits, dtype=np.uint8)
        _check(load().qmc_replay_decisions(self.h, _ptr(bits), int(n_sweeps)))

    def positions(self, out=None, stream=None):
        o = np.zeros((self.n_w, self.n_e, 3)) if out is None else out
        _check(load().qmc_get_positions(self.h, _ptr(o), _stream_ptr(stream)))
        return o

    def get_state(self) -> bytes:
        n = C.c_size_t(0)
        _check(load().qmc_get_state(self.h, None, C.byref(n)))
        buf = C.create_string_buffer(n.value)
        _check(load().qmc_get_state(self.h, buf, C.byref(n)))
        return buf.raw[: n.value]

    def set_state(self, state: bytes):
        buf = C.create_string_buffer(state, len(state))
        _check(load().qmc_set_state(self.h, buf, len(state)))

    def inverse(self, walker: int, spin: int) -> np.ndarray:
        ns = self.system.n_dn if spin else self.system.n_up
        o = np.zeros((ns, ns))
        _check(load().qmc_get_inverse(self.h, int(walker), int(spin), o.ctypes.data))
        return o

    def orbitals(self, walker: int) -> np.ndarray:
        o = np.zeros((self.n_e, 5, max(self.system.n_up, self.system.n_dn)))
        _check(load().qmc_get_orbitals(self.h, int(walker), o.ctypes.data))
        return o

    def nonlocal_energy(self) -> np.ndarray:
        """V_NL of every walker at the last measurement."""
        o = np.zeros(self.n_w)
        _check(load().qmc_get_nonlocal(self.h, o.ctypes.data))
        return o

    def logdet(self):
        """(ln|det A|, sign) of both spin blocks of every walker: two [n_w][2] arrays."""
        ld = np.zeros((self.n_w, 2))
        sg = np.zeros((self.n_w, 2))
        _check(load().qmc_get_logdet(self.h, ld.ctypes.data, sg.ctypes.data))
        return ld, sg

    def precision_report(self):
        """(residual, logdet_shift), each [n_w][2]: max |I - A X| measured by the last
        batched re-inversion of each walker and spin block, and the change the last
        log-determinant anchor made to ln|det A| (NaN before the first of each)."""
        r = np.zeros((self.n_w, 2))
        d = np.zeros((self.n_w, 2))
        _check(load().qmc_get_precision_report(self.h, r.ctypes.data, d.ctypes.data))
        return r, d

    def check(self, stream=None):
        _check(load().qmc_check_errors(self.h, _stream_ptr(stream)))

    def profile(self, enable: bool = True):
        _check(load().qmc_profile_enable(self.h, int(bool(enable))))

    def profile_read(self):
        """(ms, launches) per kernel class since the last read; indices as KERNEL_CLASSES."""
        ms = np.zeros(len(KERNEL_CLASSES))
        n = np.zeros(len(KERNEL_CLASSES), dtype=np.int64)
        _check(load().qmc_profile_read(self.h, ms.ctypes.data, n.ctypes.data))
        return ms, n

    def launch_count(self) -> int:
        return int(load().qmc_launch_count(self.h))

    def graphs(self, enable: bool = True):
        """Sweeps replayed as CUDA graphs (on by default)."""
        _check(load().qmc_graph_enable(self.h, int(bool(enable))))

    def graph_stats(self):
        """(captures, replays) of sweep graphs so far."""
        c, r = C.c_int64(0), C.c_int64(0)
        _check(load().qmc_graph_stats(self.h, C.byref(c), C.byref(r)))
        return c.value, r.value

    def close(self):
        if getattr(self, "h", None):
            load().qmc_walkers_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class DMC:
    """Branching DMC over one or more systems (each a System with move="drift")."""

    def __init__(self, systems, positions, e_trial, capacity_factor=2):
        lib = load()
        n = len(systems)
        self.systems = list(systems)
        self._pos = [np.ascontiguousarray(p, dtype=np.float64) for p in positions]
        hs = (C.c_void_p * n)(*[s.h.value for s in systems])
        nw = (C.c_int * n)(*[p.shape[0] for p in self._pos])
        pp = (C.c_void_p * n)(*[p.ctypes.data for p in self._pos])
        et = (C.c_double * n)(*[float(x) for x in e_trial])
        h = C.c_void_p()
        _check(lib.qmc_dmc_create(hs, nw, pp, et, n, int(capacity_factor), C.byref(h)))
        self.h = h
        self.cap = [int(p.shape[0]) * int(capacity_factor) for p in self._pos]

    def step(self, n=1, stream=None):
        _check(load().qmc_dmc_step(self.h, int(n), _stream_ptr(stream)))

    def profile(self, enable=True):
        _check(load().qmc_dmc_profile_enable(self.h, int(bool(enable))))

    def profile_read(self, system):
        """(ms, launches) per kernel class of one system since the last read."""
        ms = np.zeros(len(KERNEL_CLASSES))
        n = np.zeros(len(KERNEL_CLASSES), dtype=np.int64)
        _check(load().qmc_dmc_profile_read(self.h, int(system), ms.ctypes.data, n.ctypes.data))
        return ms, n

    def set_mode(self, effective_tau=False, reconfigure=False):
        """Effective time step in the branching factor; stochastic reconfiguration at a
        fixed walker count instead of branching."""
        _check(load().qmc_dmc_set_mode(self.h, int(bool(effective_tau)), int(bool(reconfigure))))

    def read(self, system):
        """dict: population, sum_w, sum_we, e_mean, e_trial_used, e_trial_next, next_id,
        population_before."""
        o = np.zeros(8)
        _check(load().qmc_dmc_read(self.h, int(system), o.ctypes.data))
        keys = ("population", "sum_w", "sum_we", "e_mean", "e_trial_used", "e_trial_next",
                "next_id", "population_before")
        return dict(zip(keys, o))

    def walkers(self, system):
        cap = self.cap[system]
        ne = self.systems[system].n_up + self.systems[system].n_dn
        pos = np.zeros((cap, ne, 3))
        ids = np.zeros(cap, dtype=np.uint32)
        el = np.zeros(cap)
        n = C.c_int(0)
        _check(load().qmc_dmc_walkers(self.h, int(system), cap, pos.ctypes.data, ids.ctypes.data,
                                      el.ctypes.data, C.byref(n)))
        k = n.value
        return pos[:k], ids[:k], el[:k]

    def launch_count(self) -> int:
        return int(load().qmc_dmc_launch_count(self.h))

    def graphs(self, enable: bool = True):
        """Steps (all systems) replayed as CUDA graphs (on by default)."""
        _check(load().qmc_dmc_graph_enable(self.h, int(bool(enable))))

    def graph_stats(self):
        """(captures, replays) of step graphs so far."""
        c, r = C.c_int64(0), C.c_int64(0)
        _check(load().qmc_dmc_graph_stats(self.h, C.byref(c), C.byref(r)))
        return c.value, r.value

    def close(self):
        if getattr(self, "h", None):
            load().qmc_dmc_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _invert_args(A, Binv, logdet, sign):
    """(precision, batch, n) of a batched re-inversion after checking every array: the
    library trusts these sizes, so a short or mistyped buffer must be refused here."""
    for name, t in (("A", A), ("Binv", Binv)):
        if not (hasattr(t, "is_cuda") and t.is_cuda):
            raise ValueError(f"{name} must be a CUDA tensor")
    if A.dim() != 3 or A.shape[1] != A.shape[2]:
        raise ValueError(f"A must be [batch][n][n], got {tuple(A.shape)}")
    if tuple(Binv.shape) != tuple(A.shape) or Binv.dtype != A.dtype:
        raise ValueError("Binv must have the shape and dtype of A")
    if A.element_size() not in (4, 8) or not A.is_floating_point():
        raise ValueError("A must be float32 or float64")
    batch = int(A.shape[0])
    for name, t in (("logdet", logdet), ("sign", sign)):
        if t is None:
            continue
        if not (hasattr(t, "is_cuda") and t.is_cuda) or t.element_size() != 8 or not t.is_floating_point():
            raise ValueError(f"{name} must be a CUDA float64 tensor")
        if t.numel() < batch:
            raise ValueError(f"{name} holds {t.numel()} values for a batch of {batch}")
    devs = {t.device for t in (A, Binv, logdet, sign) if t is not None}
    if len(devs) != 1:
        raise ValueError("all arrays must be on the same device")
    prec = PRECISIONS["fp64"] if A.element_size() == 8 else PRECISIONS["fp32"]
    return prec, batch, int(A.shape[1])


def measure_rates() -> dict:
    """FP32 and FP64 FMA throughput (TFLOP/s) and L2 read bandwidth (GB/s) of the current
    device, measured by the library's own kernels."""
    o = np.zeros(3)
    _check(load().qmc_measure_rates(o.ctypes.data))
    return {"fp32_tflops": float(o[0]), "fp64_tflops": float(o[1]), "l2_read_gbs": float(o[2])}


def slater_invert(A, Binv, logdet=None, sign=None, stream=None):
    """FP64 re-inversion of a batch of Slater matrices: A and Binv are CUDA tensors
    [batch][n][n] (float64 or float32), logdet/sign CUDA float64 [batch] or None."""
    prec, batch, n = _invert_args(A, Binv, logdet, sign)
    _check(load().qmc_slater_invert(prec, _ptr(A), _ptr(Binv), _ptr(logdet), _ptr(sign), n,
                                    batch, _stream_ptr(stream)))


def slater_invert_noalloc(A, Binv, logdet=None, sign=None, stream=None):
    """As slater_invert, for callers that cannot allocate device memory: uses the
    library's fixed 16 MiB work area (batch * n * n <= 2**21); concurrent calls race."""
    prec, batch, n = _invert_args(A, Binv, logdet, sign)
    _check(load().qmc_slater_invert_noalloc(prec, _ptr(A), _ptr(Binv), _ptr(logdet), _ptr(sign),
                                            n, batch, _stream_ptr(stream)))


def system_from_inputs(inputs: dict, precision="fp64", delay_k=1, reinv_period=0,
                       reinv_on_accepted=False, step=None, move=None,
                       logdet_period=0, drift_a=0.0, prop_chunk=0) -> System:
    """System (with spline table and Jastrow functors) from a ``synthetic.build_inputs``
    dictionary, or any dictionary with the same keys."""
    spec = inputs["spec"]
    s = System(spec.n_up, spec.n_dn, spec.L, inputs["ions"], precision=precision,
               move=move or spec.move, step=spec.step if step is None else step,
               delay_k=delay_k, reinv_period=reinv_period,
               reinv_on_accepted=reinv_on_accepted, seed=inputs["seed"], ion_Z=spec.ion_Z,
               kappa=spec.kappa, with_potential=spec.with_potential,
               logdet_period=logdet_period, drift_a=drift_a, prop_chunk=prop_chunk)
    s.set_spline(inputs["coef"])
    j = inputs["jastrow"]
    for which, key in enumerate(("eI", "same", "opp")):
        p = j.get(key, np.zeros(0))
        if p.size:
            s.set_jastrow(which, p, inputs["rcut"])
    return s
