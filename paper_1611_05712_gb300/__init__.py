"""GB300 (sm_103a) quasi-cylindrical arbitrary-order PSATD particle-in-cell cycle.

The compute path is the C-ABI library ``libpsatd_rz.so`` built from ``csrc/``
(declared in ``include/psatd_rz.h``); ``binding`` marshals arguments to it.
There is no CPU fallback: using the binding without the built library raises.
"""
__all__ = ["binding", "workloads"]
