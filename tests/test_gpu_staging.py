"""GPU tests of the staged particle input (pic_stage_particles / pic_take_particles): the
host-to-device copy of a particle set runs on the library's copy stream while queued
cycles compute, and taking the set is the same as writing it.

* A staged set taken in equals the same set written with pic_write_particles (particles
  read back bit-identical, FP64 and mixed forms), and the cycles that follow match the
  oracle (FP64 within 1e-12).
* Pipelined use: the next set is staged while a cycle runs; every take replaces the
  particles by its own set, and the host arrays may change once take has returned.
* Errors: take without a staged set, two stages without a take, staging buffers that are
  too small or misaligned, n beyond the capacity; an empty set; the moving window is
  switched off by a take, as by a write.
"""
import ctypes

import numpy as np
import pytest
import torch

from oracle import psatd_rz as O
from paper_1611_05712_gb300 import binding as bd
from paper_1611_05712_gb300 import workloads as W
from gpu_helpers import by_id, rel_err

pytestmark = pytest.mark.gpu

PRECISIONS = [bd.PIC_FP64, bd.PIC_MIXED_TF32X3, bd.PIC_MIXED_BF16X6]


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1611_05712_gb300.build import build
    build()


def _pinned(P):
    out = {k: torch.from_numpy(np.ascontiguousarray(P[k], dtype=np.float64)).pin_memory() for k in bd.SOA}
    out["id"] = torch.from_numpy(np.ascontiguousarray(P["id"], dtype=np.int32)).pin_memory()
    return out


def _same(a, b):
    for k in bd.SOA + ("id",):
        assert np.array_equal(a[k], b[k]), k


@pytest.mark.parametrize("precision", PRECISIONS)
def test_take_equals_write(precision):
    w = W.tiny(order_p=16, Nz=64, Nr=16, Nm=2, n_beam=256)
    P, npl, beams = W.particles(w)
    a = bd.Sim.from_workload(w, P, npl, beams, precision=precision)
    b = bd.Sim.from_workload(w, P, npl, beams, precision=precision)
    # a different set, staged from pinned memory into b and written into a
    rng = np.random.default_rng(5)
    Q = {k: v.copy() for k, v in P.items()}
    Q["uz"] = Q["uz"] + rng.normal(scale=0.01 * O.C_LIGHT, size=len(Q["uz"]))
    perm = rng.permutation(len(Q["x"]))
    Q = {k: v[perm] for k, v in Q.items()}
    a.write_particles(Q)
    b.stage_particles(_pinned(Q))
    b.take_particles()
    _same(a.read_particles(), b.read_particles())
    if precision == bd.PIC_FP64:
        _same(b.read_particles(), Q)


def test_take_then_cycles_match_oracle():
    w = W.tiny(order_p=16, Nz=64, Nr=16, Nm=2, n_beam=256)
    P, npl, beams = W.particles(w)
    s = bd.Sim.from_workload(w, P, npl, beams, precision=bd.PIC_FP64)
    g = O.Grid(w.Nz, w.Nr, w.Nm, w.dz, w.dr, w.dt)
    st = O.make_state(g, w.order_p, True, P, npl, beams)
    s.step(1)
    O.pic_step(st, 1)
    # replace the particles by the oracle's own state after that cycle: a no-op in value
    cur = {k: np.array(st.p[k]) for k in bd.SOA + ("id",)}
    s.stage_particles(_pinned(cur))
    s.take_particles()
    s.step(2)
    O.pic_step(st, 2)
    for name, ref in (("E", st.E), ("B", st.B)):
        assert rel_err(s.get(name), np.stack(ref)) < 1e-12, name
    got, ref = by_id(s.read_particles()), by_id(st.p)
    for k in bd.SOA:
        assert rel_err(got[k], ref[k]) < 1e-12, k


@pytest.mark.parametrize("precision", [bd.PIC_FP64, bd.PIC_MIXED_TF32X3])
def test_pipelined_stage_take(precision):
    w = W.tiny(order_p=16, Nz=64, Nr=16, Nm=2, n_beam=256)
    P, npl, beams = W.particles(w)
    s = bd.Sim.from_workload(w, P, npl, beams, precision=precision)
    ref = bd.Sim.from_workload(w, P, npl, beams, precision=precision)
    rng = np.random.default_rng(11)
    sets = []
    for _ in range(4):
        Q = {k: v.copy() for k, v in P.items()}
        Q["ux"] = Q["ux"] + rng.normal(scale=1e-3 * O.C_LIGHT, size=len(Q["ux"]))
        sets.append(_pinned(Q))
    s.stage_particles(sets[0])
    for k in range(len(sets)):
        s.take_particles()
        expect = {key: v.numpy().copy() for key, v in sets[k].items()}
        sets[k]["ux"].fill_(0.0)   # the host arrays are free once take has returned
        ref.write_particles(expect)
        _same(s.read_particles(), ref.read_particles())
        if k + 1 < len(sets):
            s.stage_particles(sets[k + 1])   # copies while the cycle below runs
        s.step(1)
        s.diagnostics(beams[-1][0], beams[-1][1])
    assert s.num_particles() == len(P["x"])


def test_stage_errors_and_empty_set():
    w = W.tiny(order_p=16, Nz=32, Nr=8, Nm=1, n_beam=16)
    P, npl, beams = W.particles(w)
    n = len(P["x"])
    s = bd.Sim.from_workload(w, P, npl, beams, capacity=n + 8, precision=bd.PIC_MIXED_TF32X3)
    lib = s.lib
    with pytest.raises(bd.PicError) as e:
        s.take_particles()
    assert e.value.status == 6
    pin = _pinned(P)
    s.stage_particles(pin)
    with pytest.raises(bd.PicError) as e:
        s.stage_particles(pin)
    assert e.value.status == 6
    s.take_particles()
    assert np.array_equal(s.read_particles()["id"], P["id"])
    nb = ctypes.c_size_t()
    assert lib.pic_stage_bytes(n, ctypes.byref(nb)) == 0
    buf = torch.empty(nb.value + 512, dtype=torch.uint8, device="cuda:0")
    base = (buf.data_ptr() + 255) // 256 * 256
    ptrs = (ctypes.c_void_p * 7)(*[pin[k].data_ptr() for k in bd.SOA])
    idp = ctypes.c_void_p(pin["id"].data_ptr())
    assert lib.pic_stage_particles(s.h, ptrs, idp, n, ctypes.c_void_p(base), nb.value - 1) == 1   # too small
    assert lib.pic_stage_particles(s.h, ptrs, idp, n, ctypes.c_void_p(base + 16), nb.value) == 1   # misaligned
    assert lib.pic_stage_particles(s.h, ptrs, idp, n + 9, ctypes.c_void_p(base), nb.value + 512) == 1
    assert lib.pic_stage_particles(s.h, ptrs, idp, -1, ctypes.c_void_p(base), nb.value) == 1
    # an empty set empties the simulation
    empty = {k: np.zeros(0) for k in bd.SOA}
    empty["id"] = np.zeros(0, np.int32)
    s.stage_particles(empty)
    s.take_particles()
    assert s.num_particles() == 0


def test_take_switches_the_window_off():
    w = W.tiny(order_p=16, Nz=32, Nr=8, Nm=1, n_beam=16)
    P, npl, beams = W.particles(w)
    n = len(P["x"])
    s = bd.Sim.from_workload(w, P, npl, beams, capacity=n + 8)
    s.window_setup(npl, 1, 8)
    s.step(2)
    s.stage_particles(_pinned(P))
    s.take_particles()
    with pytest.raises(bd.PicError) as e:
        s.window_state()
    assert e.value.status == 6
    s.step(1)
