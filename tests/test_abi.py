"""The C-ABI library loads, exports every symbol include/qmcgb.h declares, and rejects
bad arguments on the host before touching the GPU (CPU test)."""
import ctypes as C
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    text = open(os.path.join(ROOT, "include", "qmcgb.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return set(re.findall(r"\b(qmc_[a-z0-9_]+)\s*\(", text))


def test_every_declared_symbol_is_exported_and_bound():
    from paper_1802_06922_gb300 import qmcgb
    lib = qmcgb.load()
    declared = _declared()
    assert len(declared) >= 17
    for name in declared:
        assert hasattr(lib, name), name
    assert declared == set(qmcgb.SIGNATURES), declared ^ set(qmcgb.SIGNATURES)


def test_bad_arguments_are_rejected_on_the_host():
    from paper_1802_06922_gb300 import qmcgb
    lib = qmcgb.load()
    h = C.c_void_p()
    assert lib.qmc_system_create(None, C.byref(h)) == qmcgb.QMC_EINVAL
    assert b"NULL" in lib.qmc_last_error()
    base = dict(n_up=4, n_dn=4, L=10.0, n_ion=0, ion_pos=None, ion_Z=4.0, kappa=1.0,
                with_potential=1, prec=0, move=0, step=0.3, delay_k=1, reinv_period=0,
                reinv_on_accepted=0, seed=0)
    for bad in (dict(n_up=-1), dict(n_up=0, n_dn=0), dict(L=0.0), dict(delay_k=0),
                dict(delay_k=65), dict(prec=7), dict(move=3), dict(step=-1.0),
                dict(n_ion=2), dict(reinv_period=-1), dict(n_dn=5000)):
        d = qmcgb.SystemDesc(**{**base, **bad})
        assert lib.qmc_system_create(C.byref(d), C.byref(h)) == qmcgb.QMC_EINVAL, bad
        assert lib.qmc_last_error()
    # NULL handles everywhere
    assert lib.qmc_sweep(None, 1, None) == qmcgb.QMC_EINVAL
    assert lib.qmc_measure(None, None, None, None) == qmcgb.QMC_EINVAL
    assert lib.qmc_system_set_spline(None, 4, 4, 4, 1, None) == qmcgb.QMC_EINVAL
    assert lib.qmc_system_set_jastrow(None, 0, 8, 1.0, None, 0, 0.0) == qmcgb.QMC_EINVAL
    assert lib.qmc_walkers_create(None, 1, None, C.byref(h)) == qmcgb.QMC_EINVAL
    assert lib.qmc_launch_count(None) == 0
    lib.qmc_walkers_destroy(None)
    lib.qmc_system_destroy(None)


def test_python_binding_raises_instead_of_falling_back():
    from paper_1802_06922_gb300 import qmcgb
    with pytest.raises(qmcgb.QMCError):
        qmcgb.System(4, 4, -1.0, [])


def test_invert_wrappers_refuse_host_tensors():
    """The re-inversion wrappers check their arrays before calling the library."""
    torch = pytest.importorskip("torch")
    from paper_1802_06922_gb300 import qmcgb as q
    A = torch.zeros(2, 4, 4, dtype=torch.float64)
    for fn in (q.slater_invert, q.slater_invert_noalloc):
        with pytest.raises(ValueError):
            fn(A, torch.zeros_like(A))
