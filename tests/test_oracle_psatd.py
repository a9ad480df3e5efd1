"""Pins of the oracle's PSATD field update.

Eq. psatd-eqE / psatd-eqB with the operators of Eq. qcyl-ops and [k_z]
(section "Finite order pseudo-spectral solvers"); Eq. omega_mod (section
"Numerical Cherenkov radiation"); Fig. stencil_reach (unit pulse).
"""
import json
import math
import os

import numpy as np
import pytest
from scipy.linalg import expm

from oracle import psatd_rz as O

HERE = os.path.dirname(__file__)
C = O.C_LIGHT


def _setup(Nz=16, Nr=8, Nm=2, cfl=0.7, p=0, dz=0.05e-6):
    g = O.Grid(Nz, Nr, Nm, dz, dz, cfl * dz / C)
    h = O.hankel_setup(g)
    return g, h, O.psatd_coefficients(g, h, p)


def _rand(rng, sh):
    return rng.normal(size=sh) + 1j * rng.normal(size=sh)


def _curl_matrix(kp, kz):
    return np.array([[kz, 0, -0.5j * kp], [0, -kz, -0.5j * kp], [1j * kp, 1j * kp, 0]])


@pytest.mark.parametrize("p,cfl", [(0, 0.7), (16, 0.7), (0, 4.0), (32, 1.0)])
def test_update_is_exact_solution_of_maxwell_with_constant_J(p, cfl):
    """With E^n obeying Gauss's law for rho^n and J obeying continuity, the update equals
    the exact solution of dE/dt = c^2 curl B - J/eps0, dB/dt = -curl E over dt
    (matrix exponential of the affine ODE in one spectral cell).  This pins every
    coefficient and sign of Eq. psatd-eqE/eqB in SI (R-units), independently of them."""
    g, h, coef = _setup(cfl=cfl, p=p)
    rng = np.random.default_rng(p + int(cfl * 10))
    sh = (g.Nm, g.Nr, g.Nz)
    Kp, Kz = coef["Kp"], coef["Kz"]
    rho_prev = _rand(rng, sh) * 1e-8
    J = tuple(_rand(rng, sh) for _ in range(3))
    Et = O.op_curl(Kp, Kz, *(_rand(rng, sh) for _ in range(3)))
    gl = O.op_grad(Kp, Kz, -rho_prev / (O.EPS0 * (Kp ** 2 + Kz ** 2)))
    E = tuple(1e5 * a + b for a, b in zip(Et, gl))
    B = tuple(1e-3 * b for b in O.op_curl(Kp, Kz, *(_rand(rng, sh) for _ in range(3))))
    rho_next = rho_prev - g.dt * O.op_div(Kp, Kz, *J)
    En, Bn, _, Jc = O.psatd_update(g, coef, None, E, B, J, rho_next, rho_prev,
                                   filt=False, correct=True)
    for i in range(3):   # continuity already held: the correction changes nothing
        assert np.abs(Jc[i] - J[i]).max() < 1e-12 * np.abs(J[i]).max()
    worst = 0.0
    for (m, n, k) in [(0, 0, 0), (1, 3, 5), (1, 7, 8), (0, 2, 15), (1, 0, 1)]:
        Cm = _curl_matrix(Kp[m, n, k], Kz[m, n, k])
        A = np.zeros((7, 7), complex)
        A[0:3, 3:6] = C * C * Cm
        A[3:6, 0:3] = -Cm
        A[0:3, 6] = -np.array([J[i][m, n, k] for i in range(3)]) / O.EPS0
        y0 = np.array([E[i][m, n, k] for i in range(3)] + [B[i][m, n, k] for i in range(3)] + [1])
        y1 = expm(A * g.dt) @ y0
        e = np.abs(y1[:3] - [En[i][m, n, k] for i in range(3)]).max() / np.abs(y1[:3]).max()
        b = np.abs(y1[3:6] - [Bn[i][m, n, k] for i in range(3)]).max() / np.abs(y1[3:6]).max()
        worst = max(worst, e, b)
    assert worst < 1e-12


def _vacuum_mode(g, coef, rng):
    """Divergence-free E and B in every spectral cell."""
    sh = (g.Nm, g.Nr, g.Nz)
    Kp, Kz = coef["Kp"], coef["Kz"]
    K = np.sqrt(Kp ** 2 + Kz ** 2)
    E = tuple(a / K for a in O.op_curl(Kp, Kz, *(_rand(rng, sh) for _ in range(3))))
    B = tuple(a / (K * C) for a in O.op_curl(Kp, Kz, *(_rand(rng, sh) for _ in range(3))))
    return E, B


def _vacuum_steps(g, coef, E, B, nsteps):
    zero = np.zeros_like(E[0])
    for _ in range(nsteps):
        E, B, _, _ = O.psatd_update(g, coef, None, E, B, (zero, zero, zero), zero, zero,
                                    filt=False, correct=False)
    return E, B


@pytest.mark.parametrize("p,cfl,nsteps", [(0, 0.5, 200), (0, 5.0, 50), (16, 1.0, 100),
                                          (4, 2.0, 50)])
def test_vacuum_dispersion(p, cfl, nsteps):
    """Vacuum modes rotate with omega^2 = c^2 (k_perp^2 + [k_z]^2) (Eq. omega_mod); with
    infinite order this is the exact omega = c k for any dt (no Courant limit, no
    numerical dispersion; FOPS).  Closed form after t = N dt:
    E(t) = cos(wt) E0 + (c/K) sin(wt) curl B0,  B(t) = cos(wt) B0 - sin(wt)/(cK) curl E0."""
    g, h, coef = _setup(cfl=cfl, p=p)
    rng = np.random.default_rng(7)
    E0, B0 = _vacuum_mode(g, coef, rng)
    E, B = _vacuum_steps(g, coef, E0, B0, nsteps)
    Kp, Kz = coef["Kp"], coef["Kz"]
    kz_exact = np.ones((g.Nr, 1)) * g.kz[None, :]
    Kz_law = kz_exact if p == 0 else O.modified_kz(kz_exact, g.dz, p)
    K = np.sqrt(Kp ** 2 + Kz_law ** 2)
    wt = C * K * nsteps * g.dt
    cB, cE = O.op_curl(Kp, Kz, *B0), O.op_curl(Kp, Kz, *E0)
    for i in range(3):
        Eref = np.cos(wt) * E0[i] + C * np.sin(wt) / K * cB[i]
        Bref = np.cos(wt) * B0[i] - np.sin(wt) / (C * K) * cE[i]
        assert np.abs(E[i] - Eref).max() < 1e-11 * np.abs(Eref).max()
        assert np.abs(B[i] - Bref).max() < 1e-11 * np.abs(Bref).max()


@pytest.mark.parametrize("p", [0, 8])
def test_vacuum_energy_conserved(p):
    """Sum of 2|E+|^2 + 2|E-|^2 + |Ez|^2 + c^2(...B) over spectral cells is invariant for
    divergence-free vacuum fields (the update is a rotation in that norm)."""
    g, h, coef = _setup(cfl=1.0, p=p)
    E, B = _vacuum_mode(g, coef, np.random.default_rng(11))

    def energy(E, B):
        w = (2.0, 2.0, 1.0)
        return sum(w[i] * (np.abs(E[i]) ** 2 + C * C * np.abs(B[i]) ** 2).sum() for i in range(3))

    e0 = energy(E, B)
    E, B = _vacuum_steps(g, coef, E, B, 300)
    assert energy(E, B) == pytest.approx(e0, rel=1e-12)


@pytest.mark.parametrize("filt", [False, True])
def test_gauss_and_continuity_maintained(filt):
    """Global spectral current correction (R-corr) makes (rho^{n+1}-rho^n)/dt + div J = 0
    exactly, and Gauss's law div E = rho/eps0 then holds after every step when it held
    initially, for arbitrary (non-conserving) sources."""
    g, h, coef = _setup(cfl=1.0, p=16)
    T = O.source_filter(g, h)
    rng = np.random.default_rng(13)
    sh = (g.Nm, g.Nr, g.Nz)
    Kp, Kz = coef["Kp"], coef["Kz"]
    rho = _rand(rng, sh) * 1e-6
    E = O.op_grad(Kp, Kz, -rho / (O.EPS0 * (Kp ** 2 + Kz ** 2)))
    B = tuple(np.zeros(sh, complex) for _ in range(3))
    for step in range(20):
        J = tuple(_rand(rng, sh) * 1e2 for _ in range(3))
        rho_next = _rand(rng, sh) * 1e-6
        E, B, rho_f, Jc = O.psatd_update(g, coef, T, E, B, J, rho_next, rho, filt=filt,
                                         correct=True)
        cont = (rho_f - rho) / g.dt + O.op_div(Kp, Kz, *Jc)
        assert np.abs(cont).max() < 1e-12 * np.abs(O.op_div(Kp, Kz, *Jc)).max()
        gauss = O.op_div(Kp, Kz, *E) - rho_f / O.EPS0
        assert np.abs(gauss).max() < 1e-11 * np.abs(rho_f / O.EPS0).max()
        divB = O.op_div(Kp, Kz, *B)
        assert np.abs(divB).max() < 1e-10 * max(np.abs(b).max() * Kp.max() for b in B)
        rho = rho_f


def test_small_x_series_match_direct_forms():
    """The power series used below omega dt = 0.25 agree with the direct forms where both
    are accurate (continuity of the coefficient tables across the switch)."""
    for x in (0.2, 0.25, 0.3):
        x2 = np.array([x * x])
        s0 = O._series_terms(x2, 0)[0] * x * x
        s1 = O._series_terms(x2, 1)[0] * x * x
        assert s0 == pytest.approx(math.sin(x) / x - 1.0, rel=1e-12)
        assert s1 == pytest.approx(math.cos(x) - math.sin(x) / x, rel=1e-12)


def _unit_pulse(p, Nz=512, Nr=64):
    gold = json.load(open(os.path.join(HERE, "golden", "stencil_reach.json")))
    dz = gold["dz_m"]
    g = O.Grid(Nz, Nr, 1, dz, gold["dr_m"], gold["cdt_over_dz"] * dz / C)
    h = O.hankel_setup(g)
    coef = O.psatd_coefficients(g, h, p)
    sh = (1, Nr, Nz)
    d = np.zeros(sh, complex)
    d[0, 0, Nz // 2] = 1.0
    z = np.zeros(sh, complex)
    Eh = O.forward_vector(g, h, z, z, d)
    Bh = O.forward_vector(g, h, d, z, z)
    En, Bn, _, _ = O.psatd_update(g, coef, None, Eh, Bh, (z, z, z), z, z, filt=False,
                                  correct=False)
    Ez = np.abs(O.inverse_vector(g, h, *En)[2][0, 0])
    dist = np.abs(np.arange(Nz) - Nz // 2)
    return Ez / Ez.max(), dist, gold


def _reach(prof, dist, thresh):
    beyond = [D for D in range(1, dist.max()) if prof[dist >= D].max() < thresh]
    return beyond[0] if beyond else dist.max()


def test_unit_pulse_order32_reaches_machine_precision_within_guard_cells():
    """Fig. stencil_reach: order 32 decays by ~16 orders of magnitude within ~60 cells;
    PSATD_inf keeps contributions along the whole axis."""
    prof, dist, gold = _unit_pulse(gold_order := 32)
    assert gold_order == json.load(open(os.path.join(HERE, "golden", "stencil_reach.json")))["order"]
    g_cells = gold["guard_cells_order_32"]
    assert prof[dist >= g_cells + 4].max() < 10.0 ** -(gold["decay_orders_of_magnitude"] - 1)
    prof_inf, _, _ = _unit_pulse(0)
    assert prof_inf[dist >= g_cells + 4].min() > 1e-9


def test_unit_pulse_reach_vs_order():
    """Delta N_z grows with the order; it exceeds the order at low order and is close to
    it at high order (Fig. stencil_reach, bottom)."""
    reach = {}
    for p in (4, 8, 16, 32, 64):
        prof, dist, _ = _unit_pulse(p)
        reach[p] = _reach(prof, dist, 1e-14)
    orders = sorted(reach)
    assert all(reach[a] < reach[b] for a, b in zip(orders, orders[1:]))
    assert reach[4] > 4 and reach[8] > 8
    assert reach[4] / 4 > reach[64] / 64
    assert 0.5 * 64 < reach[64] < 3 * 64


def test_source_filter_z_factor_is_the_binomial_stencil():
    # multiplying by cos^2(k_z dz/2) in Fourier space is the periodic (1/4, 1/2, 1/4) stencil
    # along z; the filter separates into a radial factor per (m, n) times this z factor
    g, h, _ = _setup(Nz=32, Nr=8, Nm=2)
    T = O.source_filter(g, h)
    rng = np.random.default_rng(12)
    f = _rand(rng, 32)
    want = 0.25 * np.roll(f, 1) + 0.5 * f + 0.25 * np.roll(f, -1)
    for m in range(2):
        for n in (0, 3, 7):
            tz = T[m][n] / T[m][n][0]
            assert np.allclose(O.ifft_z(tz * O.fft_z(f)), want, rtol=0, atol=1e-13)
    # the radial factor is cos^2(k_perp dr / 2): 1 in the long-wavelength limit, falling
    # with k_perp, within (0, 1]
    tr = T[:, :, 0]
    assert np.all(tr > 0) and np.all(tr <= 1)
    assert np.all(np.diff(tr, axis=1) < 0)
    assert tr[0][0] == pytest.approx(1.0, abs=0.05)
