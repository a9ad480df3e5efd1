"""Pins of the oracle's spectral transforms and quasi-cylindrical operators.

Section "Finite order pseudo-spectral solvers": Hankel transform along r, Fourier
transform along z, operator table Eq. qcyl-ops.  The DHT discretisation is not in the
paper; the pins below tie the oracle's reading to Bessel-function mathematics.
"""
import math

import numpy as np
import pytest
from scipy.special import jv

from oracle import psatd_rz as O


def test_dft_matches_explicit_sum_long_double():
    rng = np.random.default_rng(0)
    N = 12
    f = rng.normal(size=(3, N)) + 1j * rng.normal(size=(3, N))
    F = O.fft_z(f)
    i = np.arange(N, dtype=np.longdouble)
    for k in range(N):
        ang = -2 * np.pi * np.longdouble(k) * i / N
        ref = (f * (np.cos(ang) + 1j * np.sin(ang)).astype(np.complex128)).sum(axis=1)
        assert np.allclose(F[:, k], ref, atol=1e-13)
    assert np.allclose(O.ifft_z(F), f, atol=1e-14)


def test_kz_grid_order_and_nyquist_sign():
    g = O.Grid(8, 4, 1, 0.5, 1.0, 1.0)
    f = np.array([0, 1, 2, 3, -4, -3, -2, -1])
    assert np.allclose(g.kz, 2 * np.pi * f / (8 * 0.5))


@pytest.mark.parametrize("m", [0, 1, 2, 3])
def test_bessel_zeros(m):
    """alpha_{m,n}: J_m(alpha) = 0, interlacing with J_{m+1}, McMahon asymptotics."""
    N = 400
    g = O.Grid(4, N, m + 2, 1.0, 1.0, 1.0)
    h = O.hankel_setup(g)
    a = h.kperp[m] * g.R
    assert np.abs(jv(m, a)).max() < 1e-13
    b = h.kperp[m + 1] * g.R
    assert np.all(a < b) and np.all(b[:-1] < a[1:])
    n = np.arange(1, N + 1)
    beta = (n + 0.5 * m - 0.25) * np.pi
    mu = 4.0 * m * m
    mc = beta - (mu - 1) / (8 * beta) - 4 * (mu - 1) * (7 * mu - 31) / (3 * (8 * beta) ** 3)
    assert np.abs(a[100:] - mc[100:]).max() < 1e-9


@pytest.mark.parametrize("Nr,m", [(16, 0), (64, 1), (64, 2), (256, 1)])
def test_hankel_forward_is_fourier_bessel_quadrature(Nr, m):
    """For smooth low-order modes the forward DHT of order m approaches the
    Fourier-Bessel coefficient integral  2/(R^2 J_{m+1}(alpha_n)^2) int f(r) J_m(k_n r) r dr
    evaluated with the midpoint rule on the r nodes (independent formula)."""
    g = O.Grid(4, Nr, m + 1, 1.0, 1.0, 1.0)
    h = O.hankel_setup(g)
    a = h.kperp[m] * g.R
    r = g.r
    Mq = (2.0 / (g.R ** 2 * jv(m + 1, a) ** 2))[:, None] * (r * g.dr)[None, :] * jv(m, np.outer(h.kperp[m], r))
    nmax = Nr // 8
    M = h.M[m][1]
    assert np.abs(M[:nmax] - Mq[:nmax]).max() < 2e-2 * np.abs(M[:nmax]).max()


@pytest.mark.parametrize("Nr", [8, 64, 200])
def test_hankel_pseudo_inverse(Nr):
    """Moore-Penrose conditions of the truncated pseudo-inverse; order-m slot is a true inverse:
    the DHT of the sampled basis function J_m(k_{m,n} r) is the unit vector e_n."""
    g = O.Grid(4, Nr, 3, 1.0, 1.0, 1.0)
    h = O.hankel_setup(g)
    for m in range(3):
        for s in range(3):
            B, M = h.Binv[m][s], h.M[m][s]
            smax = np.linalg.norm(B, 2)
            # truncated Moore-Penrose: M B M = M, B M and M B symmetric, and B M B
            # differs from B by at most the dropped singular values (<= rcond sigma_max)
            assert np.abs(M @ B @ M - M).max() < 1e-11 * np.abs(M).max()
            assert np.abs(B @ M - (B @ M).T).max() < 1e-11
            assert np.abs(M @ B - (M @ B).T).max() < 1e-11
            assert np.linalg.norm(B @ M @ B - B, 2) <= O.PINV_RCOND * smax * (1 + 1e-9)
        Bz = h.Binv[m][1]
        assert np.abs(h.M[m][1] @ Bz - np.eye(Nr)).max() < 1e-11


def test_hankel_dropped_direction_is_the_dini_k0_function():
    """R-dht: for m >= 1 the order m-1 basis on the zeros of J_m lacks the k = 0 Dini
    function, giving exactly one near-null singular value that pinv drops; the order
    m and m+1 slots of m <= 1 keep full rank at Nr = 256."""
    g = O.Grid(4, 256, 3, 1.0, 1.0, 1.0)
    h = O.hankel_setup(g)
    for m in range(3):
        ranks = [np.linalg.matrix_rank(h.M[m][s], tol=1e-6 * np.abs(h.M[m][s]).max())
                 for s in range(3)]
        if m == 0:
            assert ranks == [256, 256, 256]
        else:
            assert ranks[0] == 255
    assert np.linalg.matrix_rank(h.M[1][1]) == 256 and np.linalg.matrix_rank(h.M[1][2]) == 256


def test_hankel_round_trip_on_representable_fields():
    g = O.Grid(8, 32, 2, 1.0, 1.0, 1.0)
    h = O.hankel_setup(g)
    rng = np.random.default_rng(3)
    sh = (g.Nm, g.Nr, g.Nz)
    Vh = tuple(rng.normal(size=sh) + 1j * rng.normal(size=sh) for _ in range(3))
    # project onto the kept subspace of each slot (M B) so the round trip is exact
    Vh = (np.stack([h.M[m][2] @ h.Binv[m][2] @ Vh[0][m] for m in range(2)]),
          np.stack([h.M[m][0] @ h.Binv[m][0] @ Vh[1][m] for m in range(2)]),
          Vh[2])
    Vr = O.inverse_vector(g, h, *Vh)
    back = O.forward_vector(g, h, *Vr)
    for a, b in zip(Vh, back):
        assert np.abs(a - b).max() < 1e-12 * np.abs(a).max()


# ---------------------------------------------------------------------------
# Convention pin (Eq. qcyl-ops with R-modes): spectral rules vs cylindrical finite
# differences of an analytic mode, on a fine sample around a point.
# ---------------------------------------------------------------------------
M_TEST, K_PERP, K_Z = 1, 1.3, 0.7


def _real_vector(coeffs, r, th, z, m=M_TEST):
    """Real-space (F_r, F_theta, F_z) of spectral (+, -, z) coefficients of mode m>=1:
    F = Re[2 F_m(r) e^{-i m theta} e^{i k_z z}] with F_pm of orders m+-1."""
    a, b, c = coeffs
    Fp = a * jv(m + 1, K_PERP * r)
    Fm = b * jv(m - 1, K_PERP * r)
    Fz = c * jv(m, K_PERP * r)
    ph = 2.0 * np.exp(-1j * m * th + 1j * K_Z * z)
    return np.real((Fp + Fm) * ph), np.real(1j * (Fp - Fm) * ph), np.real(Fz * ph)


def _real_scalar(s, r, th, z, m=M_TEST):
    return np.real(2.0 * s * jv(m, K_PERP * r) * np.exp(-1j * m * th + 1j * K_Z * z))


H = 1e-4
PTS = [(0.8, 0.3, 0.2), (2.1, -1.2, 1.5)]


def _d(f, r, th, z, axis):
    dr = [(H, 0, 0), (0, H, 0), (0, 0, H)][axis]
    return (f(r + dr[0], th + dr[1], z + dr[2]) - f(r - dr[0], th - dr[1], z - dr[2])) / (2 * H)


@pytest.mark.parametrize("pt", PTS)
def test_convention_grad(pt):
    r, th, z = pt
    s = 0.4 - 0.9j
    f = lambda r_, t_, z_: _real_scalar(s, r_, t_, z_)  # noqa: E731
    num = (_d(f, r, th, z, 0), _d(f, r, th, z, 1) / r, _d(f, r, th, z, 2))
    spec = O.op_grad(K_PERP, K_Z, s)
    ref = _real_vector(spec, r, th, z)
    assert np.allclose(num, ref, atol=1e-6)


@pytest.mark.parametrize("pt", PTS)
def test_convention_div_and_curl(pt):
    r, th, z = pt
    V = (0.3 + 0.2j, -0.5 + 0.1j, 0.7 - 0.4j)
    comp = lambda i: (lambda r_, t_, z_: _real_vector(V, r_, t_, z_)[i])  # noqa: E731
    Vr, Vt, Vz = comp(0), comp(1), comp(2)
    rVr = lambda r_, t_, z_: r_ * Vr(r_, t_, z_)  # noqa: E731
    rVt = lambda r_, t_, z_: r_ * Vt(r_, t_, z_)  # noqa: E731
    div = _d(rVr, r, th, z, 0) / r + _d(Vt, r, th, z, 1) / r + _d(Vz, r, th, z, 2)
    assert div == pytest.approx(_real_scalar(O.op_div(K_PERP, K_Z, *V), r, th, z), abs=1e-6)
    curl = (_d(Vz, r, th, z, 1) / r - _d(Vt, r, th, z, 2),
            _d(Vr, r, th, z, 2) - _d(Vz, r, th, z, 0),
            (_d(rVt, r, th, z, 0) - _d(Vr, r, th, z, 1)) / r)
    ref = _real_vector(O.op_curl(K_PERP, K_Z, *V), r, th, z)
    assert np.allclose(curl, ref, atol=1e-6)


def test_operator_identities():
    rng = np.random.default_rng(5)
    Kp, Kz = rng.uniform(0.1, 3, 20), rng.uniform(-3, 3, 20)
    X = rng.normal(size=20) + 1j * rng.normal(size=20)
    V = tuple(rng.normal(size=20) + 1j * rng.normal(size=20) for _ in range(3))
    K2 = Kp ** 2 + Kz ** 2
    assert np.allclose(O.op_div(Kp, Kz, *O.op_grad(Kp, Kz, X)), -K2 * X)
    assert np.allclose(O.op_div(Kp, Kz, *O.op_curl(Kp, Kz, *V)), 0, atol=1e-12)
    assert np.allclose(O.op_curl(Kp, Kz, *O.op_grad(Kp, Kz, X)), 0, atol=1e-12)
    cc = O.op_curl(Kp, Kz, *O.op_curl(Kp, Kz, *V))
    gd = O.op_grad(Kp, Kz, O.op_div(Kp, Kz, *V))
    for a, v, b in zip(cc, V, gd):
        assert np.allclose(a, K2 * v + b)
