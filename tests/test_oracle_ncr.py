"""Numerical Cherenkov radiation in the oracle (section "Numerical Cherenkov radiation":
Eq. omega_mod, Eq. resonance, Eq. resonance_k and the Fourier-space figure of E_z).

The plasma + relativistic beam case (256 x 64, 2 modes, gamma = 1000) advanced 200 cycles
at stencil order 4 and at infinite order from one initial state: the spectral amplitude
that the finite-order run adds to E_z of mode 0 (the spatial Fourier transform of the
axisymmetric part) peaks on the curve k_perp = sqrt(beta^2 k_z^2 - [k_z]_4^2) where the
modified dispersion relation meets the beam mode, and the infinite-order run, which has no
such curve, carries almost nothing there.  CPU only (about 40 s)."""
import numpy as np
import pytest

from oracle import psatd_rz as O
from paper_1611_05712_gb300 import workloads as W

CYCLES = 200


@pytest.fixture(scope="module")
def runs():
    w = W.plasma_beam_small()
    P, npl, beams = W.particles(w)
    g = O.Grid(w.Nz, w.Nr, w.Nm, w.dz, w.dr, w.dt)
    h = O.hankel_setup(g)
    maps = {}
    for p in (4, 0):
        st = O.make_state(g, p, True, P, npl, beams, h=h)
        O.pic_step(st, CYCLES)
        maps[p] = np.abs(st.Eh[2][0])
    gamma = beams[0][2]
    return g, h, maps, np.sqrt(1.0 - 1.0 / gamma ** 2)


def test_resonance_curve_is_where_the_modified_dispersion_meets_the_beam_mode():
    g = O.Grid(256, 64, 1, 0.05e-6, 0.05e-6, 0.05e-6 / O.C_LIGHT)
    beta = np.sqrt(1.0 - 1.0 / 1000.0 ** 2)
    for p in (4, 16, 64):
        kp = O.ncr_resonance_kperp(g.kz, g.dz, p, beta)
        ok = np.isfinite(kp)
        assert ok.any()
        # on the curve the phase velocity along z equals the beam velocity (Eq. resonance)
        omega = O.C_LIGHT * np.sqrt(kp[ok] ** 2 + O.modified_kz(g.kz[ok], g.dz, p) ** 2)
        assert np.allclose(omega / np.abs(g.kz[ok]), beta * O.C_LIGHT, rtol=1e-12)
    # higher order moves the resonance to larger |k_z| (the stencil is exact further out)
    first = [np.abs(g.kz)[np.isfinite(O.ncr_resonance_kperp(g.kz, g.dz, p, beta))].min() for p in (4, 16, 64)]
    assert first[0] < first[1] < first[2]
    assert not np.isfinite(O.ncr_resonance_kperp(g.kz, g.dz, 0, beta)).any()


def test_finite_order_excess_lies_on_the_resonance_curve(runs):
    g, h, maps, beta = runs
    kperp = h.kperp[0]
    kres = O.ncr_resonance_kperp(g.kz, g.dz, 4, beta)
    excess = maps[4] - maps[0]
    top = np.argsort(excess.ravel())[::-1][:10]
    dk = np.pi / g.R                              # spacing of the zeros of J_0 / R
    for k in top:
        n, f = divmod(int(k), g.Nz)
        assert np.isfinite(kres[f]), (n, f)
        assert abs(kperp[n] - kres[f]) < 1.5 * dk, (n, f, kperp[n], kres[f])
        # the infinite-order run has (almost) nothing there
        assert maps[0][n, f] < 0.1 * maps[4][n, f]
    # and the excess is a large part of the field at those modes
    assert excess.ravel()[top[0]] > 0.01 * maps[0].max()
