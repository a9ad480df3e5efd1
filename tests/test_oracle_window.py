"""Pins of the oracle's moving window (R-window: the co-moving frame zeta = z - c t of
section "Accurate modeling of plasma accelerators in finite order PSATD", Fig. ez).

* Column removal: for a field state in the range of the transforms (a forward transform
  of arbitrary fields, transformed back), subtracting the forward transform of one
  column must leave exactly that column zero in real space and every other column
  untouched.  A wrong phase, column, Hankel order or sign fails at O(1).
* Removal rule: hand-computed window coordinates of ballistic particles (zero fields).
* Injection: explicit small cases for the choice of slots (smallest inactive ids).
* Fixed point: a cold neutral plasma with no fields is unchanged, particle by particle
  and id by id, by any number of window cycles; a template of the wrong column, a wrong
  removal sign or a wrong slot order breaks it.
* A beam at gamma = 1000 keeps its window coordinate while its array coordinate moves
  one cell per cycle.
"""
import dataclasses

import numpy as np
import pytest

from oracle import psatd_rz as O
from paper_1611_05712_gb300 import workloads as W


def _grid(Nz=16, Nr=8, Nm=2):
    w = W.tiny(order_p=8, Nz=Nz, Nr=Nr, Nm=Nm)
    return w, O.Grid(w.Nz, w.Nr, w.Nm, w.dz, w.dr, w.dt)


def _empty_state(w, g, parts=None):
    if parts is None:
        z = np.zeros(0)
        parts = {k: z.copy() for k in W.KEYS}
        parts["id"] = np.zeros(0, dtype=np.int32)
    return O.make_state(g, w.order_p, True, parts, 0)


@pytest.mark.parametrize("column", [0, 5, 15])
def test_clear_column_zeroes_exactly_that_column(column):
    w, g = _grid()
    st = _empty_state(w, g)
    rng = np.random.default_rng(7 + column)

    def rnd():
        return rng.normal(size=(g.Nm, g.Nr, g.Nz)) + 1j * rng.normal(size=(g.Nm, g.Nr, g.Nz))

    st.Eh = O.forward_vector(g, st.h, rnd(), rnd(), rnd())
    st.Bh = O.forward_vector(g, st.h, rnd(), rnd(), rnd())
    st.E = O.inverse_vector(g, st.h, *st.Eh)
    st.B = O.inverse_vector(g, st.h, *st.Bh)
    E0, B0 = [a.copy() for a in st.E], [a.copy() for a in st.B]
    O.window_clear_column(st, column)
    for F0, F, Fh in ((E0, st.E, st.Eh), (B0, st.B, st.Bh)):
        back = O.inverse_vector(g, st.h, *Fh)
        scale = max(np.abs(a).max() for a in F0)
        for c in range(3):
            assert np.abs(back[c][:, :, column]).max() < 1e-12 * scale
            keep = np.ones(g.Nz, dtype=bool)
            keep[column] = False
            assert np.abs(back[c][:, :, keep] - F0[c][:, :, keep]).max() < 1e-12 * scale
            assert np.array_equal(F[c][:, :, keep], F0[c][:, :, keep])
            assert not np.any(F[c][:, :, column])


def test_removal_rule_hand_cases():
    w, g = _grid()
    dz, L = g.dz, g.L
    back = 5 * dz
    h = 0.5 * g.dt * O.C_LIGHT   # half move at v = c: half a cell (c dt = dz)
    assert h == pytest.approx(0.5 * dz, rel=1e-12)
    # (z_old, half move, window moves?, removed?)
    cases = [
        (5.3 * dz, 0.0, True, True),          # at rest in the departing column
        (5.3 * dz, 0.0, False, False),        # the window does not move this cycle
        (5.3 * dz, h, True, False),           # keeps pace with the window at c
        (5.9 * dz, -0.25 * dz, True, True),   # zeta = 0.9 - 0.5 - 1 < 0
        (6.2 * dz, 0.0, True, False),         # next column: stays
        (5.2 * dz, -0.25 * dz, False, True),  # through the back edge without a shift
        (4.9 * dz, h, True, False),           # front column, forward at c
        (4.9 * dz, -h, True, False),          # front column: zeta = L - 0.1 dz - 2 dz
        (0.0, 0.0, True, False),              # far from the edge (zeta = L - 5 dz)
    ]
    for z, hm, sh, want in cases:
        got = O.window_removed(g, np.array([z]), np.array([hm]), back, sh)[0]
        assert bool(got) == want, (z / dz, hm / dz, sh)


def test_removal_through_gather_push_zero_fields():
    w, g = _grid()
    dz = g.dz
    st = _empty_state(w, g)
    c = O.C_LIGHT
    # u = gamma v for v = -0.5 c, 0, +c*0.999, -0.2 c
    def u_of(beta):
        return beta * c / np.sqrt(1.0 - beta * beta)
    z = np.array([5.6, 5.1, 5.05, 9.5]) * dz
    uz = np.array([u_of(-0.5), 0.0, u_of(0.999), u_of(-0.2)])
    n = z.size
    st.p = {"x": np.full(n, 2.0 * g.dr), "y": np.zeros(n), "z": z.copy(), "ux": np.zeros(n),
            "uy": np.zeros(n), "uz": uz.copy(), "w": np.ones(n), "id": np.arange(n, dtype=np.int32)}
    O.gather_push(st, window=(5 * dz, True))
    # zeta = 0.6 - 0.5 - 1, 0.1 - 1, 0.05 + 0.999 - 1, 4.5 - 0.2 - 1 (cells)
    assert list(st.p["w"]) == [0.0, 0.0, 1.0, 1.0]
    assert st.p["uz"][0] == 0.0 and st.p["uz"][2] > 0.0
    # removed particles keep their pushed position
    assert st.p["z"][0] == pytest.approx(5.1 * dz, rel=1e-12)
    # inactive particles stay where they are
    z_before = st.p["z"].copy()
    O.gather_push(st)
    assert st.p["z"][0] == z_before[0] and st.p["z"][1] == z_before[1]


def test_injection_takes_smallest_inactive_ids():
    w, g = _grid()
    st = _empty_state(w, g)
    n = 10
    ids = np.array([4, 0, 7, 3, 9, 1, 2, 8, 5, 6], dtype=np.int32)
    wts = np.ones(n)
    wts[[2, 3, 4]] = 0.0        # ids 7, 3, 9 inactive
    st.p = {"x": np.zeros(n), "y": np.zeros(n), "z": np.zeros(n), "ux": np.ones(n), "uy": np.ones(n),
            "uz": np.ones(n), "w": wts, "id": ids}
    tpl = {"x": np.array([1.0, 2.0]), "y": np.array([3.0, 4.0]), "z": np.array([5.0, 6.0]),
           "w": np.array([7.0, 8.0])}
    win = O.Window(1, 0, 0, tpl, [np.array([0, 1])])
    assert O.window_inject(st, win, 0) == 0
    by_id = {int(i): k for k, i in enumerate(st.p["id"])}
    for tid, pid in ((0, 3), (1, 7)):
        k = by_id[pid]
        assert (st.p["x"][k], st.p["y"][k], st.p["z"][k], st.p["w"][k]) == (
            tpl["x"][tid], tpl["y"][tid], tpl["z"][tid], tpl["w"][tid])
        assert st.p["ux"][k] == st.p["uy"][k] == st.p["uz"][k] == 0.0
    assert st.p["w"][by_id[9]] == 0.0
    # a template larger than the pool is cut to the pool
    win2 = O.Window(1, 0, 0, tpl, [np.array([0, 1])])
    assert O.window_inject(st, win2, 0) == 1
    assert st.p["w"][by_id[9]] == 7.0


def _plasma_state(Nz=16, Nr=8, Nm=2, ppc=(1, 1, 2)):
    w = dataclasses.replace(W.tiny(order_p=8, Nz=Nz, Nr=Nr, Nm=Nm), beams=[], ppc=ppc)
    g = O.Grid(w.Nz, w.Nr, w.Nm, w.dz, w.dr, w.dt)
    P, npl, _ = W.particles(w)
    return w, g, O.make_state(g, w.order_p, True, P, npl), P, npl


def test_cold_plasma_is_a_fixed_point():
    w, g, st, P, npl = _plasma_state()
    win = O.window_setup(st, npl, 1, 8)
    assert st.p["x"].size == npl + 8
    n_cycles = g.Nz + 3
    dropped = O.pic_step_window(st, win, n_cycles)
    assert dropped == 0 and win.shifts == n_cycles and win.cycles == n_cycles
    got = {k: v[np.argsort(st.p["id"])] for k, v in st.p.items()}
    for k in ("x", "y", "z", "w"):
        assert np.array_equal(got[k][:npl], P[k]), k
    assert not np.any(got["w"][npl:])
    for k in ("ux", "uy", "uz"):
        assert not np.any(got[k])
    e_scale = O.Q_E * w.plasma_density * g.dz / O.EPS0   # field of one cell's electron layer
    for F in st.E + st.B:
        assert np.abs(F).max() < 1e-9 * e_scale


def test_cold_plasma_period_two_moves_every_other_cycle():
    w, g, st, P, npl = _plasma_state()
    win = O.window_setup(st, npl, 2, 4)
    O.pic_step_window(st, win, 7)
    assert win.shifts == 3 and win.cycles == 7
    got = {k: v[np.argsort(st.p["id"])] for k, v in st.p.items()}
    for k in ("x", "y", "z", "w"):
        assert np.array_equal(got[k][:npl], P[k]), k


def test_beam_keeps_its_window_coordinate():
    w = dataclasses.replace(W.tiny(order_p=8, Nz=32, Nr=8, Nm=1, n_beam=64), plasma_density=0.0)
    g = O.Grid(w.Nz, w.Nr, w.Nm, w.dz, w.dr, w.dt)
    P, npl, beams = W.particles(w)
    P["w"] = P["w"] * 1e-6   # weak beam: nearly ballistic at gamma ~ 50
    P["uz"] = np.full(P["uz"].size, 1000.0 * O.C_LIGHT)
    st = O.make_state(g, w.order_p, True, P, npl)
    win = O.window_setup(st, npl, 1, 0)
    o0 = np.argsort(st.p["id"])
    z0 = O.window_z(g, win, st.p["z"])[o0]
    a0 = st.p["z"][o0]
    O.pic_step_window(st, win, 10)
    o1 = np.argsort(st.p["id"])
    zw = O.window_z(g, win, st.p["z"])[o1]
    # array coordinates move by 10 cells (mod L); window coordinates by 10 dz (beta - 1)
    da = (st.p["z"][o1] - a0) % g.L
    assert np.allclose(da, 10 * g.dz, rtol=0, atol=1e-5 * g.dz)
    assert np.abs(zw - z0).max() < 1e-5 * g.dz
    assert np.all(st.p["w"] > 0)
