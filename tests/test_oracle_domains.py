"""Pins of the oracle's guard-cell decomposition of the field step along z (section
"Finite order pseudo-spectral solvers": a finite-order stencil reaches a finite number of
cells, unit-pulse figure; "Conclusion": about 60 guard cells at p = 32, while the infinite
order solver is global).  CPU only."""
import numpy as np
import pytest

from oracle import psatd_rz as O

DZ = 0.05e-6
NZ, NR, NM = 256, 16, 2


@pytest.fixture(scope="module")
def setup():
    g = O.Grid(NZ, NR, NM, DZ, DZ, DZ / O.C_LIGHT)
    h = O.hankel_setup(g)
    rng = np.random.default_rng(7)
    sh = (NM, NR, NZ)
    E = tuple(rng.normal(size=sh) + 1j * rng.normal(size=sh) for _ in range(3))
    B = tuple((rng.normal(size=sh) + 1j * rng.normal(size=sh)) / O.C_LIGHT for _ in range(3))
    return g, h, E, B


def _err(a, b):
    return max(max(np.abs(x - y).max() for x, y in zip(a[0], b[0])) / max(np.abs(y).max() for y in b[0]),
               max(np.abs(x - y).max() for x, y in zip(a[1], b[1])) / max(np.abs(y).max() for y in b[1]))


def test_one_domain_without_guards_is_the_global_step(setup):
    g, h, E, B = setup
    glob = O.field_step_source_free(g, h, 32, E, B)
    assert _err(O.field_step_guarded(g, 32, E, B, 1, 0), glob) == 0.0


def test_source_free_step_of_an_eigenmode_is_a_rotation(setup):
    """The source-free step alone (no decomposition) is pinned independently: a unit
    spectral '+' mode of E with B chosen so that the pair is a vacuum eigenmode turns
    by exactly omega dt = c dt sqrt(K_perp^2 + [k_z]_p^2) (Eq. omega_mod)."""
    g, h, _, _ = setup
    p, m, n, f = 16, 0, 3, 5
    coef = O.psatd_coefficients(g, h, p)
    Kp, Kz = coef["Kp"][m, n, f], coef["Kz"][m, n, f]
    K = np.hypot(Kp, Kz)
    sh = (NM, NR, NZ)
    # divergence-free E direction: curl of a z-potential, normalised
    V = O.op_curl(Kp, Kz, 0.0, 0.0, 1.0)
    Eh = [np.zeros(sh, complex) for _ in range(3)]
    Bh = [np.zeros(sh, complex) for _ in range(3)]
    for i in range(3):
        Eh[i][m, n, f] = V[i]
    # eigenmode with E ~ e^{-i omega t}: B = -i curl E / (omega) ... take B = curl(E)/(i c K)
    cE = O.op_curl(Kp, Kz, *V)
    for i in range(3):
        Bh[i][m, n, f] = cE[i] / (1j * O.C_LIGHT * K)
    E = O.inverse_vector(g, h, *Eh)
    B = O.inverse_vector(g, h, *Bh)
    En, Bn = O.field_step_source_free(g, h, p, E, B)
    Ehn = O.forward_vector(g, h, *En)
    a = np.array([Eh[i][m, n, f] for i in range(3)])
    b = np.array([Ehn[i][m, n, f] for i in range(3)])
    phase = np.vdot(a, b) / np.vdot(a, a)
    assert np.abs(b - phase * a).max() < 1e-12 * np.abs(a).max()
    assert abs(abs(phase) - 1.0) < 1e-12
    assert abs(np.angle(phase) + O.C_LIGHT * g.dt * K) < 1e-12


def test_order_32_matches_the_global_step_with_64_guard_cells(setup):
    """About 60 guard cells at p = 32 (Conclusion): at 64 the interiors equal the global
    step to FP64 rounding."""
    g, h, E, B = setup
    glob = O.field_step_source_free(g, h, 32, E, B)
    assert _err(O.field_step_guarded(g, 32, E, B, 4, 64), glob) < 1e-13


def test_error_falls_with_guard_width_and_grows_with_order(setup):
    g, h, E, B = setup
    glob = O.field_step_source_free(g, h, 32, E, B)
    errs = [_err(O.field_step_guarded(g, 32, E, B, 4, gd), glob) for gd in (4, 8, 16, 32)]
    assert all(b < a for a, b in zip(errs, errs[1:])), errs
    assert errs[0] > 1e-3            # too few guard cells: spurious fields
    # at a fixed guard width a lower order (shorter stencil) is more local
    e_by_p = []
    for p in (8, 16, 32, 64):
        gl = O.field_step_source_free(g, h, p, E, B)
        e_by_p.append(_err(O.field_step_guarded(g, p, E, B, 4, 24), gl))
    assert all(b > a for a, b in zip(e_by_p, e_by_p[1:])), e_by_p


def test_infinite_order_is_not_local(setup):
    g, h, E, B = setup
    glob = O.field_step_source_free(g, h, 0, E, B)
    assert _err(O.field_step_guarded(g, 0, E, B, 4, 64), glob) > 1e-3
