"""Pins of the oracle's stencil coefficients and modified wavenumber.

Eq. finite_difference and the [k_z] equation (section "Finite order pseudo-spectral
solvers"); Eq. omega_mod and the statement that finite stencils lower the phase
velocity (section "Numerical Cherenkov radiation").
"""
import json
import math
import os
from fractions import Fraction

import numpy as np
import pytest

from oracle import psatd_rz as O

HERE = os.path.dirname(__file__)


def exact_alpha(n, j):
    """Eq. finite_difference with exact integers: (-1)^{j+1} 2 (n!)^2 / ((n-j)! (n+j)!)."""
    f = math.factorial
    return Fraction((-1) ** (j + 1) * 2 * f(n) ** 2, f(n - j) * f(n + j))


@pytest.mark.parametrize("n", [1, 2, 3, 5, 8, 16, 32, 64])
def test_alpha_matches_factorial_definition(n):
    a = O.fd_coefficients(n)
    for j in range(1, n + 1):
        assert a[j - 1] == pytest.approx(float(exact_alpha(n, j)), rel=1e-14, abs=0)


def test_alpha_matches_fornberg_table():
    gold = json.load(open(os.path.join(HERE, "golden", "fornberg_centered_weights.json")))
    for order, cs in gold["weights"].items():
        n = int(order) // 2
        a = O.fd_coefficients(n)
        for j, c in enumerate(cs, start=1):
            assert a[j - 1] == pytest.approx(2 * j * float(Fraction(c)), rel=1e-15)


@pytest.mark.parametrize("n", [1, 2, 4, 16, 128])
def test_alpha_moment_conditions(n):
    """A stencil of order 2n differentiates polynomials of degree <= 2n exactly:
    sum_j alpha_j = 1 and sum_j alpha_j j^{2k} = 0 for k = 1..n-1 (exact rationals)."""
    al = [exact_alpha(n, j) for j in range(1, n + 1)]
    assert sum(al) == 1
    for k in range(1, n):
        assert sum(a * j ** (2 * k) for j, a in enumerate(al, start=1)) == 0
    a = O.fd_coefficients(n)
    assert a.sum() == pytest.approx(1.0, abs=1e-13)


def test_alpha_large_n_limit():
    a = O.fd_coefficients(512)
    assert a[0] == pytest.approx(2.0, rel=2e-3)
    assert a[1] == pytest.approx(-2.0, rel=1e-2)


def test_order2_is_sine():
    kz = np.linspace(-np.pi, np.pi, 101) / 0.1
    assert np.allclose(O.modified_kz(kz, 0.1, 2), np.sin(kz * 0.1) / 0.1, rtol=0, atol=1e-13)


def test_infinite_order_is_exact():
    kz = np.linspace(-3, 3, 7)
    assert np.array_equal(O.modified_kz(kz, 0.1, 0), kz)


@pytest.mark.parametrize("p", [2, 4, 8, 16, 32])
def test_modified_kz_equals_real_space_stencil(p):
    """The spectral [k_z] must reproduce the real-space centred stencil of Eq.
    finite_difference applied to a periodic signal (derivative via ifft(i[k] fft))."""
    N, dz = 64, 0.37
    rng = np.random.default_rng(p)
    f = rng.normal(size=N)
    n = p // 2
    d_real = np.zeros(N)
    for j in range(1, n + 1):
        d_real += float(exact_alpha(n, j)) * (np.roll(f, -j) - np.roll(f, j)) / (2 * j * dz)
    kz = 2 * np.pi * np.fft.fftfreq(N, d=dz)
    d_spec = np.fft.ifft(1j * O.modified_kz(kz, dz, p) * np.fft.fft(f)).real
    assert np.allclose(d_spec, d_real, atol=1e-11 * np.abs(d_real).max())


@pytest.mark.parametrize("p", [4, 8, 16])
def test_modified_kz_truncation_order(p):
    """|[k]_p - k| = O(k^{p+1} dz^p): halving k divides the error by ~2^{p+1}."""
    dz = 1.0
    k1, k2 = 0.6, 0.3
    e1 = abs(O.modified_kz(np.array([k1]), dz, p)[0] - k1)
    e2 = abs(O.modified_kz(np.array([k2]), dz, p)[0] - k2)
    assert math.log2(e1 / e2) == pytest.approx(p + 1, abs=0.5)


@pytest.mark.parametrize("p", [2, 4, 8, 16, 32, 64, 256])
def test_phase_velocity_below_c_and_nyquist_zero(p):
    """Finite stencils give [k_z] <= k_z on [0, pi/dz] (reduced phase velocity, section NCR)
    and [k_z] = 0 at the Nyquist wavenumber (sin(j pi) = 0)."""
    dz = 0.05e-6
    k = np.linspace(0, np.pi / dz, 2001)
    km = O.modified_kz(k, dz, p)
    assert np.all(km <= k * (1 + 1e-14))
    assert abs(km[-1]) < 1e-9 * np.pi / dz


def test_higher_order_closer_to_exact():
    dz = 1.0
    k = np.linspace(0.01, 0.9 * np.pi, 50)
    errs = [np.abs(O.modified_kz(k, dz, p) - k).max() for p in (4, 8, 16, 32, 64)]
    assert all(a > b for a, b in zip(errs, errs[1:]))


def test_modified_dispersion_resonance_exists_only_for_finite_order():
    """Eq. resonance_k: a beam with gamma=3 meets modes with v_phi,z = v_beam only when
    [k_z] < k_z; PSATD_inf has v_phi > v_beam everywhere (section NCR)."""
    dz = 1.0
    vb = math.sqrt(1 - 1 / 9.0)
    kz = np.linspace(0.01, np.pi, 4000)
    for kr in (0.0, 0.05):
        vinf = np.sqrt(kr ** 2 + kz ** 2) / kz
        assert np.all(vinf >= 1.0 - 1e-15) and np.all(vinf > vb)
        v4 = np.sqrt(kr ** 2 + O.modified_kz(kz, dz, 4) ** 2) / kz
        assert np.any(v4 < vb)
