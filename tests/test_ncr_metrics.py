"""Pins of the error measures of the order study (section "Accurate modeling of plasma
accelerators in finite order PSATD", Eq. err-metrics) in the oracle, and agreement of the
package's host-side copies (paper_1611_05712_gb300/ncr.py, written separately) with them.
CPU only."""
import numpy as np
import pytest

from oracle import psatd_rz as O
from paper_1611_05712_gb300 import ncr


def test_err_ez_closed_form_from_a_chosen_spectrum():
    """E_inf and E_f built from chosen 2-D spectra S and S + D (both Hermitian so the
    fields are real): Err_Ez = sqrt(mean |D / S|^2) exactly."""
    rng = np.random.default_rng(3)
    nz, nr = 16, 8
    # transforms of real arrays plus a real constant: Hermitian, so the fields are real
    S = np.fft.fft2(rng.normal(size=(nr, nz))) + 5.0
    D = np.fft.fft2(rng.normal(size=(nr, nz))) * 1e-3
    e_inf = np.fft.ifft2(S).real
    e_f = np.fft.ifft2(S + D).real
    want = np.sqrt(np.mean(np.abs(D / S) ** 2))
    assert O.err_ez(e_f, e_inf) == pytest.approx(want, rel=1e-9)
    assert O.err_ez(e_inf, e_inf) == 0.0
    # a uniform scaling (1 + eps) gives |eps| in every Fourier cell
    assert O.err_ez(1.001 * e_inf, e_inf) == pytest.approx(1e-3, rel=1e-9)


def test_err_emittance_and_sigma_gamma_definitions():
    assert O.err_emittance(1.1, 1.0) == pytest.approx(0.1)
    assert O.err_sigma_gamma([1.0, 2.0], [1.0, 2.0]) == 0.0
    # two slices off by +10 % and -10 %: rms 0.1
    assert O.err_sigma_gamma([1.1, 1.8], [1.0, 2.0]) == pytest.approx(0.1)


def test_field_on_plane_mode_sum():
    F = [np.full((2, 3), 1.0 + 0j), np.full((2, 3), 0.5 + 0.25j)]
    # Re[1 + 2 (0.5 + 0.25 i)] at theta = 0
    assert np.allclose(O.field_on_plane(F), 2.0)
    # at theta = pi/2: e^{-i pi/2} = -i -> Re[1 + 2 (0.25 - 0.5 i)] = 1.5
    assert np.allclose(O.field_on_plane(F, np.pi / 2), 1.5)


def test_package_measures_agree_with_the_oracle():
    rng = np.random.default_rng(11)
    E = rng.normal(size=(3, 3, 8, 16)) + 1j * rng.normal(size=(3, 3, 8, 16))
    assert np.allclose(ncr.ez_plane(E), O.field_on_plane(list(E[2])), rtol=1e-14, atol=0)
    a, b = rng.normal(size=(8, 16)) + 3.0, rng.normal(size=(8, 16)) + 3.0
    assert ncr.err_ez(a, b) == pytest.approx(O.err_ez(a, b), rel=1e-13)
    s1, s2 = rng.uniform(1, 2, 12), rng.uniform(1, 2, 10)
    assert ncr.err_sigma_gamma(s1, s2) == pytest.approx(O.err_sigma_gamma(s1[:10], s2), rel=1e-14)
    assert ncr.err_emittance(2.5, 2.0) == pytest.approx(O.err_emittance(2.5, 2.0))
