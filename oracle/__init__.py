"""FP64 CPU oracle of the quasi-cylindrical arbitrary-order PSATD PIC cycle.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this
package.  The library (``paper_1611_05712_gb300``) never imports it and shares
no code, table or constant generator with it; both sides receive the same
seeded inputs from ``paper_1611_05712_gb300.workloads``.

Paper: S. Jalas et al., "Accurate modeling of plasma acceleration with
arbitrary order pseudo-spectral particle-in-cell methods", arXiv:1611.05712.

Every function in ``psatd_rz`` cites the passage (section / equation) it
follows.  Where the paper is silent the reading taken is stated in the
docstring.  Pins that tie this oracle to the paper and to mathematics (not to
itself) live in ``tests/test_oracle_*.py``.

Parity status: all functions are pinned (closed forms, invariants, brute force
or an independent ODE solution); none is "parity unpinned".
"""
from . import psatd_rz  # noqa: F401
