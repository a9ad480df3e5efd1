"""GPU parity of the moving window (R-window; co-moving frame zeta = z - c t of section
"Accurate modeling of plasma accelerators in finite order PSATD", Fig. ez) against the
oracle, through the C ABI.

* FP64 form: plasma + beam cycles with the window moving every cycle and every other
  cycle; fields, spectral state and every particle (by id, including removed and
  re-injected ones) within 1e-12, identical ids, shift and drop counts.
* Mixed form: the same run at the mixed form's tolerances.
* A cold neutral plasma is a fixed point (positions and weights bit-identical by id).
* A forward-streaming plasma exhausts the reserve: the dropped count equals the oracle's.
* Diagnostics measure z from the window's back edge.
* Argument errors and the refusal of window handles by pic_batch_create.
"""
import dataclasses

import numpy as np
import pytest

from oracle import psatd_rz as O
from paper_1611_05712_gb300 import binding as bd
from paper_1611_05712_gb300 import workloads as W
from gpu_helpers import by_id, rel_err

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1611_05712_gb300.build import build
    build()


def _pair(w, precision, period, n_reserve, P=None, npl=None, beams=None):
    if P is None:
        P, npl, beams = W.particles(w)
    n = len(P["x"])
    s = bd.Sim.from_workload(w, P, npl, beams, precision=precision, capacity=n + n_reserve)
    Pg = s.read_particles() if precision != bd.PIC_FP64 else P   # the state the GPU holds
    s.window_setup(npl, period, n_reserve)
    g = O.Grid(w.Nz, w.Nr, w.Nm, w.dz, w.dr, w.dt)
    st = O.make_state(g, w.order_p, True, Pg, npl, beams)
    win = O.window_setup(st, npl, period, n_reserve)
    return s, st, win, g


def _compare(s, st, win, tol_f, tol_x, tol_u):
    for name, ref in (("E", st.E), ("B", st.B), ("EH", st.Eh), ("BH", st.Bh)):
        assert rel_err(s.get(name), np.stack(ref)) < tol_f, name
    assert rel_err(s.get("RHO_PREV_H"), st.rho_prev_h) < tol_f
    got, ref = by_id(s.read_particles()), by_id(st.p)
    assert np.array_equal(got["id"], ref["id"])
    assert np.array_equal(got["w"] == 0, ref["w"] == 0), "active sets differ"
    assert rel_err(got["w"], ref["w"]) < max(tol_x, 1e-12)
    for k in ("x", "y", "z"):
        assert rel_err(got[k], ref[k]) < tol_x, k
    for k in ("ux", "uy", "uz"):
        assert rel_err(got[k], ref[k]) < tol_u, k
    info = s.window_state()
    assert info["shifts"] == win.shifts and info["cycles"] == win.cycles
    assert info["back_column"] == win.shifts % st.g.Nz


@pytest.mark.parametrize("period", [1, 2])
def test_fp64_window_matches_oracle(period):
    w = W.plasma_beam_small(order_p=16)
    s, st, win, g = _pair(w, bd.PIC_FP64, period, 512)
    n_cycles = 12
    s.step(n_cycles)
    dropped = O.pic_step_window(st, win, n_cycles)
    _compare(s, st, win, 1e-12, 1e-12, 1e-12)
    assert s.window_state()["dropped"] == dropped == 0
    # the column that departed in the last cycle was re-injected at rest; the plasma
    # further in has felt the fields
    got = by_id(s.read_particles())
    fresh = win.col_ids[win.shifts - 1]
    assert fresh.size > 0 and not np.any(got["uz"][fresh])
    assert np.all(got["w"][fresh] > 0)
    assert np.any(got["uz"][win.col_ids[w.Nz // 2]])


def test_fp64_window_many_shifts_tiny():
    w = W.tiny(order_p=16, Nz=64, Nr=16, Nm=2, n_beam=256)
    s, st, win, g = _pair(w, bd.PIC_FP64, 1, 128)
    n_cycles = 70   # more than one turn of the ring
    s.step(n_cycles)
    dropped = O.pic_step_window(st, win, n_cycles)
    _compare(s, st, win, 1e-12, 1e-12, 1e-12)
    assert s.window_state()["dropped"] == dropped


@pytest.mark.parametrize("precision", [bd.PIC_MIXED_TF32X3, bd.PIC_MIXED_BF16X6])
def test_mixed_window_matches_oracle(precision):
    w = W.plasma_beam_small(order_p=16)
    s, st, win, g = _pair(w, precision, 1, 512)
    s.step(6)
    O.pic_step_window(st, win, 6)
    _compare(s, st, win, 1e-4, 1e-5, 1e-4)


def test_cold_plasma_fixed_point_gpu():
    w = dataclasses.replace(W.tiny(order_p=8, Nz=32, Nr=16, Nm=2), beams=[], ppc=(1, 1, 2))
    P, npl, beams = W.particles(w)
    s = bd.Sim.from_workload(w, P, npl, beams, capacity=len(P["x"]) + 16)
    s.window_setup(npl, 1, 16)
    s.step(w.Nz + 5)
    got = by_id(s.read_particles())
    for k in ("x", "y", "z", "w"):
        assert np.array_equal(got[k][:npl], P[k]), k
    assert not np.any(got["w"][npl:])
    c = O.C_LIGHT
    for k in ("ux", "uy", "uz"):
        assert np.abs(got[k]).max() < 1e-9 * c
    assert s.window_state()["dropped"] == 0


def test_reserve_exhaustion_counts_drops():
    w = dataclasses.replace(W.tiny(order_p=8, Nz=32, Nr=8, Nm=1), beams=[], ppc=(1, 1, 1))
    P, npl, beams = W.particles(w)
    # plasma streaming forward at 0.9 c: only the particles within 0.1 cell of the back
    # edge leave each cycle, while a whole column's template arrives
    u = 0.9 * O.C_LIGHT / np.sqrt(1 - 0.81)
    P["uz"] = np.full(npl, u)
    s, st, win, g = _pair(w, bd.PIC_FP64, 1, 4, P, npl, beams)
    s.step(10)
    dropped = O.pic_step_window(st, win, 10)
    assert dropped > 0
    assert s.window_state()["dropped"] == dropped
    _compare(s, st, win, 1e-12, 1e-12, 1e-12)


def test_diagnostics_use_window_coordinates():
    w = W.tiny(order_p=16, Nz=64, Nr=16, Nm=2, n_beam=256)
    P, npl, beams = W.particles(w)
    s = bd.Sim.from_workload(w, P, npl, beams, capacity=len(P["x"]) + 64)
    lo, hi, _ = beams[0]
    d0 = s.diagnostics(lo, hi)
    s.window_setup(npl, 1, 64)
    s.step(20)
    d1 = s.diagnostics(lo, hi)
    # gamma = 50 moves at c (1 - 2e-4): 20 cycles shift the window coordinate by 4e-3 dz
    assert abs(d1["z_mean"] - d0["z_mean"]) < 0.05 * w.dz
    got = s.read_particles()
    sel = (got["id"] >= lo) & (got["id"] < hi)
    zw = (got["z"][sel] - 20 * w.dz) % w.L
    ref = O.beam_diagnostics(got["x"][sel], got["y"][sel], zw, got["ux"][sel], got["uy"][sel],
                             got["uz"][sel], got["w"][sel])
    assert d1["z_mean"] == pytest.approx(ref["z_mean"], rel=1e-12)


def test_window_argument_errors():
    w = W.tiny(order_p=16, Nz=32, Nr=8, Nm=1, n_beam=16)
    P, npl, beams = W.particles(w)
    n = len(P["x"])
    s = bd.Sim.from_workload(w, P, npl, beams, capacity=n + 8)
    with pytest.raises(bd.PicError) as e:
        s.window_state()
    assert e.value.status == 6   # PIC_ERR_STATE
    for args in ((npl, 0, 0), (n + 1, 1, 0), (npl, 1, 9), (-1, 1, 0)):
        with pytest.raises(bd.PicError) as e:
            s.window_setup(*args)
        assert e.value.status == 1
    bad = dict(P)
    bad["id"] = P["id"].copy()
    bad["id"][0] = bad["id"][1]   # duplicate id
    s.write_particles(bad)
    with pytest.raises(bd.PicError):
        s.window_setup(npl, 1, 0)
    s.write_particles(P)
    s.window_setup(npl, 1, 8)
    with pytest.raises(bd.PicError):
        s.window_setup(npl, 1, 0)   # already on
    assert s.num_particles() == n + 8


def test_batch_refuses_window_handles():
    import torch
    w = W.tiny(order_p=16, Nz=32, Nr=8, Nm=1, n_beam=16)
    P, npl, beams = W.particles(w)
    sim_stream = torch.cuda.Stream()
    s = bd.Sim.from_workload(w, P, npl, beams, capacity=len(P["x"]) + 8, stream=sim_stream)
    s.window_setup(npl, 1, 8)
    with pytest.raises(bd.PicError):
        bd.Batch([s], cycles=2, origin=torch.cuda.Stream())


def test_window_with_sort_interval_mixed():
    # the window's records survive cycles without a sort (slots then stay where they are)
    w = W.plasma_beam_small(order_p=16)
    s, st, win, g = _pair(w, bd.PIC_MIXED_TF32X3, 1, 512)
    s.set_sort_interval(3)
    s.step(7)
    O.pic_step_window(st, win, 7)
    _compare(s, st, win, 1e-4, 1e-5, 1e-4)


def test_stage_calls_apply_the_pending_column_removal():
    # after a moving cycle the spectral subtraction is pending; a stage-wise field step
    # (forward transform, PSATD, inverse transform) must see it applied
    w = W.plasma_beam_small(order_p=16)
    s, st, win, g = _pair(w, bd.PIC_FP64, 1, 512)
    s.step(3)
    O.pic_step_window(st, win, 3)
    s.forward_transform()
    s.psatd()
    s.inverse_transform()
    # the stage calls reuse the deposit grids of the last cycle: compare with the oracle's
    # field step from the same sources
    dep = s.get("DEP")
    O.field_step(st, dep[0], (dep[1], dep[2], dep[3]))
    for name, ref in (("E", st.E), ("B", st.B), ("EH", st.Eh), ("BH", st.Bh)):
        assert rel_err(s.get(name), np.stack(ref)) < 1e-11, name
