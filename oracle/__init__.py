"""Plain FP64 CPU oracle for particle-by-particle VMC/DMC through a Slater-Jastrow
wavefunction with B-spline orbitals and B-spline Jastrow functors.

TEST INFRASTRUCTURE ONLY. Nothing in the product path may import this package: only
``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` use it.
It shares no code with the CUDA library; the two meet only through the seeded inputs of
the ``synthetic`` package and through the published definition of the Philox4x32-10
counter-based generator, which each side implements on its own.

The oracle is deliberately slow and direct: every proposed move rebuilds the Slater
matrix with the moved electron's row replaced and takes its determinant by LU from
scratch, and the Jastrow factor is recomputed over all pairs. Each module cites the
section or equation of the paper it follows.

Parity status of every function is listed in the module docstrings; the pins are the
``-m "not gpu"`` tests in ``tests/test_oracle_*.py``. The DMC trial-energy feedback
constant and the walker-ID assignment of branched walkers are adopted readings the paper
gives no values for; they are pinned by the invariants any population control keeps (an
exact fixed point at the target, a negative feedback, unique IDs), not by values.
"""
