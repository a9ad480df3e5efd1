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
    s1, s2 = rng.uniform(1, 2, 12), rng.uniform(1, 2, 12)
    assert ncr.err_sigma_gamma(s1, s2) == pytest.approx(O.err_sigma_gamma(s1, s2), rel=1e-14)
    with pytest.raises(ValueError):
        ncr.err_sigma_gamma(s1, s2[:10])    # unpaired slices are refused, not truncated
    assert ncr.err_emittance(2.5, 2.0) == pytest.approx(O.err_emittance(2.5, 2.0))


def test_slice_spreads_on_a_common_grid_agree_with_the_oracle():
    """Both runs are sliced on the reference run's grid (z_start = zbar - 3 sigma_z of the
    reference), so slice i is the same interval of z in both; a run whose beam moved by a
    fraction of a slice still pairs slice by slice.  The package's binned version agrees
    with the oracle's loop version, and a beam compared with itself gives 0."""
    rng = np.random.default_rng(12)
    n = 4000
    z_ref = rng.normal(30e-6, 2e-6, n)
    g_ref = rng.normal(400.0, 0.4, n)
    w = rng.uniform(0.5, 1.5, n)
    z_f = z_ref + 0.3e-6                         # shifted by 0.6 of a slice
    g_f = g_ref * (1.0 + 1e-3 * rng.normal(size=n))
    z0, ns = ncr.slice_grid(z_ref, w)
    W = w.sum()
    zbar = (w * z_ref).sum() / W
    sz = np.sqrt((w * (z_ref - zbar) ** 2).sum() / W)
    assert z0 == pytest.approx(zbar - 3 * sz, rel=1e-12) and ns == int(np.ceil(6 * sz / O.SLICE_LEN))
    for zz, gg in ((z_ref, g_ref), (z_f, g_f)):
        a = ncr.slice_sigma_gamma(zz, gg, w, z0, ns)
        b = O.slice_sigma_gamma_on_grid(zz, gg, w, z0, ns)
        assert np.array_equal(np.isnan(a), np.isnan(b))
        assert np.allclose(a[~np.isnan(a)], b[~np.isnan(b)], rtol=1e-10, atol=0)
    ref = {"z": z_ref, "gamma": g_ref, "w": w}
    assert ncr.err_sigma_gamma_runs(ref, ref) == 0.0
    e = ncr.err_sigma_gamma_runs({"z": z_f, "gamma": g_f, "w": w}, ref)
    a = O.slice_sigma_gamma_on_grid(z_f, g_f, w, z0, ns)
    b = O.slice_sigma_gamma_on_grid(z_ref, g_ref, w, z0, ns)
    ok = ~np.isnan(a) & ~np.isnan(b) & (b > 0)
    assert e == pytest.approx(O.err_sigma_gamma(a[ok], b[ok]), rel=1e-9)


def test_resonance_curve_of_the_package_agrees_with_the_oracle():
    g = O.Grid(128, 32, 1, 0.05e-6, 0.05e-6, 0.05e-6 / O.C_LIGHT)
    beta = 0.9999
    for p in (4, 8, 32):
        want = O.ncr_resonance_kperp(g.kz, g.dz, p, beta)
        got = ncr.resonance_kperp(g.kz, O.modified_kz(g.kz, g.dz, p), beta)
        assert np.array_equal(np.isnan(got), np.isnan(want))
        assert np.allclose(got[~np.isnan(got)], want[~np.isnan(want)], rtol=1e-9)   # cancellation near threshold
