"""GPU parity of the beam diagnostics (emittance and slice energy spread of section
"Accurate modeling of plasma accelerators in finite order PSATD") against the oracle on
identical particle data, through the C ABI.

* FP64 form: a plasma plus a correlated Gaussian beam stored in shuffled array order; the
  whole beam and half of its ids; every reported quantity and slice value within 1e-11.
* Mixed form: the diagnostics of the FP32 particle state equal the oracle's on the same
  state read back in float64 (within 1e-11).
* Degenerate cases: no particle selected, sigma_z = 0 (no slices), more slices than the
  library's limit (PIC_ERR_ARG), and a slice buffer shorter than the number of slices.
"""
import numpy as np
import pytest

from oracle import psatd_rz as O
from paper_1611_05712_gb300 import binding as bd

pytestmark = pytest.mark.gpu

KEYS = ("W", "z_mean", "sigma_z", "gamma_mean", "emit_nx", "emit_ny", "sigma_gamma_mean")
DZ = 0.05e-6


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1611_05712_gb300.build import build
    build()


def particle_set(seed, Nz=512, Nr=64, n_plasma=20000, n_beam=30000, sig_z=1.0e-6, sig_r=0.5e-6, gamma=500.0,
                 same_z=False, dz=DZ):
    """Uniform plasma (ids 0..n_plasma-1) and a Gaussian beam with an x-ux correlation and
    a gamma chirp along z (ids n_plasma..), all in shuffled array order."""
    rng = np.random.default_rng(seed)
    L, R = Nz * dz, Nr * DZ
    zp = rng.uniform(0, L, n_plasma)
    rp = R * np.sqrt(rng.uniform(0, 0.98, n_plasma))
    tp = rng.uniform(0, 2 * np.pi, n_plasma)
    zc = 0.5 * L
    # same_z: a dyadic z and equal weights, so that every weighted sum is exact and the
    # centred z vanishes exactly on both sides
    zb = np.full(n_beam, 2.0 ** -20) if same_z else np.clip(rng.normal(zc, sig_z, n_beam), 0.0, L * (1 - 1e-12))
    xb = rng.normal(0, sig_r, n_beam)
    yb = rng.normal(0, sig_r, n_beam)
    c = O.C_LIGHT
    uxb = c * (rng.normal(0, 0.05, n_beam) + 0.3 * xb / sig_r * 0.05)
    uyb = c * rng.normal(0, 0.05, n_beam)
    uzb = c * gamma * (1 + 1e-3 * rng.normal(size=n_beam) + 2e-3 * (zb - zc) / max(sig_z, 1e-12))
    P = {"x": np.concatenate([rp * np.cos(tp), xb]), "y": np.concatenate([rp * np.sin(tp), yb]),
         "z": np.concatenate([zp, zb]),
         "ux": np.concatenate([c * 1e-3 * rng.normal(size=n_plasma), uxb]),
         "uy": np.concatenate([c * 1e-3 * rng.normal(size=n_plasma), uyb]),
         "uz": np.concatenate([c * 1e-3 * rng.normal(size=n_plasma), uzb]),
         "w": np.concatenate([np.full(n_plasma, 1e5),
                              np.full(n_beam, 1e4) if same_z else rng.uniform(0.5e4, 1.5e4, n_beam)]),
         "id": np.arange(n_plasma + n_beam, dtype=np.int32)}
    perm = rng.permutation(n_plasma + n_beam)
    return {k: v[perm] for k, v in P.items()}, n_plasma, n_plasma + n_beam


def make_sim(P, precision=bd.PIC_FP64, Nz=512, Nr=64, dz=DZ):
    cfg = bd.make_config(Nz, Nr, 1, dz, DZ, DZ / O.C_LIGHT, 16, True, precision, len(P["x"]))
    s = bd.Sim(cfg)
    s.write_particles(P)
    return s


def oracle_diag(P, lo, hi):
    sel = (P["id"] >= lo) & (P["id"] < hi)
    return O.beam_diagnostics(*(P[k][sel] for k in bd.SOA)), int(sel.sum())


def check(d, od, n, rel=1e-11):
    assert d["n_particles"] == n
    for k in KEYS:
        assert d[k] == pytest.approx(od[k], rel=rel, abs=1e-300), k
    assert d["n_slices"] == len(od["slice_sigma_gamma"])
    assert np.allclose(d["slice_sigma_gamma"], od["slice_sigma_gamma"], rtol=rel, atol=0)


def test_fp64_diagnostics_on_identical_data():
    P, lo, hi = particle_set(1)
    s = make_sim(P)
    for a, b in ((lo, hi), (lo, (lo + hi) // 2), ((lo + hi) // 2, hi)):
        od, n = oracle_diag(P, a, b)
        check(s.diagnostics(a, b), od, n)


@pytest.mark.parametrize("precision", [bd.PIC_MIXED_TF32X3, bd.PIC_MIXED_BF16X6])
def test_mixed_diagnostics_on_their_own_state(precision):
    P, lo, hi = particle_set(2)
    s = make_sim(P, precision)
    Q = s.read_particles()   # the FP32 cell-relative state in float64
    od, n = oracle_diag(Q, lo, hi)
    check(s.diagnostics(lo, hi), od, n)


def test_no_particle_selected():
    P, lo, hi = particle_set(3, n_plasma=1000, n_beam=1000)
    s = make_sim(P)
    d = s.diagnostics(hi + 10, hi + 20)
    assert d["n_particles"] == 0 and d["W"] == 0.0 and d["n_slices"] == 0


def test_zero_sigma_z_has_no_slices():
    P, lo, hi = particle_set(4, n_plasma=1000, n_beam=2000, same_z=True)
    s = make_sim(P)
    d = s.diagnostics(lo, hi)
    od, n = oracle_diag(P, lo, hi)
    assert d["sigma_z"] == 0.0 and od["sigma_z"] == 0.0
    assert d["n_slices"] == 0 and d["sigma_gamma_mean"] == 0.0
    for k in ("W", "gamma_mean", "emit_nx", "emit_ny"):
        assert d[k] == pytest.approx(od[k], rel=1e-11), k


def test_too_many_slices_is_an_argument_error():
    # a beam spread over 8 cm of z: 6 sigma_z / 0.5 um is far above the 65536-slice limit
    P, lo, hi = particle_set(5, Nz=4096, Nr=64, n_plasma=100, n_beam=5000, sig_z=3e-2, dz=20e-6)
    s = make_sim(P, Nz=4096, Nr=64, dz=20e-6)
    with pytest.raises(bd.PicError) as e:
        s.diagnostics(lo, hi)
    assert e.value.status == 1


def test_short_slice_buffer():
    P, lo, hi = particle_set(6)
    s = make_sim(P)
    od, n = oracle_diag(P, lo, hi)
    d = s.diagnostics(lo, hi, max_slices=3)
    assert d["n_slices"] == len(od["slice_sigma_gamma"]) > 3
    assert np.allclose(d["slice_sigma_gamma"], od["slice_sigma_gamma"][:3], rtol=1e-11, atol=0)
    assert d["sigma_gamma_mean"] == pytest.approx(od["sigma_gamma_mean"], rel=1e-11)
