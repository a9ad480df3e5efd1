"""Whole-cycle pins of the oracle (PIC loop of the introduction, PSATD of section
"Finite order pseudo-spectral solvers", workload of section "Accurate modeling of
plasma accelerators in finite order PSATD")."""
import numpy as np
import pytest

from oracle import psatd_rz as O
from paper_1611_05712_gb300 import workloads as W


@pytest.fixture(scope="module")
def small():
    w = W.plasma_beam_small()
    P, npl, beams = W.particles(w)
    g = O.Grid(w.Nz, w.Nr, w.Nm, w.dz, w.dr, w.dt)
    return w, g, P, npl, beams


def _gauss_residual(st):
    Kp, Kz = st.coef["Kp"], st.coef["Kz"]
    d = O.op_div(Kp, Kz, *st.Eh) - st.rho_prev_h / O.EPS0
    return np.abs(d).max() / np.abs(st.rho_prev_h / O.EPS0).max()


def test_gauss_law_and_charge_through_the_cycle(small):
    """Initial beam fields obey div E = rho/eps0 (relativistic Poisson, R-init); the
    corrected PSATD update keeps it; total charge (ions included) is conserved."""
    w, g, P, npl, beams = small
    st = O.make_state(g, 0, True, P, npl, beams)
    assert _gauss_residual(st) < 1e-13
    V = g.cell_volume()[:, None]
    q_beam = st.q * P["w"][npl:].sum()
    for _ in range(3):
        O.pic_step(st, 1)
        assert _gauss_residual(st) < 1e-13
        Pn = st.p
        rho = O.deposit_rho(g, Pn["x"], Pn["y"], Pn["z"], Pn["w"], st.q) + st.rho_ion
        assert (rho[0] * V).sum().real == pytest.approx(q_beam, rel=1e-10)
    # the sort keeps every particle exactly once
    assert np.array_equal(np.sort(st.p["id"]), np.arange(len(P["id"])))


def test_rigid_relativistic_beam_fields_co_move(small):
    """A gamma=1000 beam alone in vacuum with infinite order: its space-charge fields
    translate with the beam at ~c (no numerical dispersion), instead of staying put."""
    w, g, _, _, _ = small
    P, _, beams = W.particles(w, with_plasma=False)
    st = O.make_state(g, 0, True, P, 0, beams)
    E0 = st.E[0][0].copy()
    n = 8
    O.pic_step(st, n)
    shift = int(round(O.C_LIGHT * g.dt * n / g.dz))
    E1 = st.E[0][0]
    moved = np.abs(E1 - np.roll(E0, shift, axis=-1)).max() / np.abs(E0).max()
    static = np.abs(E1 - E0).max() / np.abs(E0).max()
    assert moved < 0.02 and static > 0.1


@pytest.mark.parametrize("order_p", [0, 32])
def test_initial_beam_fields_are_boosted_coulomb_fields(small, order_p):
    """A rigid beam moving along +z at beta carries B = (beta/c) z_hat x E (the Lorentz
    transform of its rest-frame field): B_r = -beta E_theta / c, B_theta = beta E_r / c,
    B_z = 0, mode by mode in real space (R-init; the plasma is neutral at t = 0)."""
    w, g, P, npl, beams = small
    st = O.make_state(g, order_p, True, P, npl, beams)
    (_, _, gam), = beams
    beta = np.sqrt(1.0 - 1.0 / gam ** 2)
    Er, Et, Ez = st.E
    Br, Bt, Bz = st.B
    scale = beta * np.abs(Er).max() / O.C_LIGHT
    assert scale > 0
    assert np.abs(Bt - beta * Er / O.C_LIGHT).max() < 1e-12 * scale
    assert np.abs(Br + beta * Et / O.C_LIGHT).max() < 1e-12 * scale
    assert np.abs(Bz).max() < 1e-12 * scale
    assert np.abs(Ez).max() > 1e-3 * np.abs(Er).max() / gam ** 2   # the longitudinal field exists
