"""Pins of the oracle's particle side: cell keys and sort, deposit, gather, push,
and the beam diagnostics (section "Accurate modeling of plasma accelerators in
finite order PSATD": emittance and slice energy spread, Eq. err-metrics)."""
import cmath
import math

import numpy as np
import pytest

from oracle import psatd_rz as O

DZ = 0.05e-6


def _grid(Nz=16, Nr=8, Nm=3):
    return O.Grid(Nz, Nr, Nm, DZ, DZ, DZ / O.C_LIGHT)


def _random_particles(g, n, rng, r_max=None):
    r_max = g.R * 0.999 if r_max is None else r_max
    r = r_max * np.sqrt(rng.uniform(0, 1, n))
    th = rng.uniform(0, 2 * np.pi, n)
    return r * np.cos(th), r * np.sin(th), rng.uniform(0, g.L, n)


# -------------------------------------------------------------------- keys and sort
def test_keys_and_stable_sort_brute_force():
    g = _grid()
    rng = np.random.default_rng(0)
    x, y, z = _random_particles(g, 500, rng)
    x[:40] = x[40:80]          # duplicate positions -> equal keys, stability matters
    y[:40] = y[40:80]
    z[:40] = z[40:80]
    keys = O.cell_keys(g, x, y, z)
    for i in range(len(x)):
        iz = min(max(math.floor(z[i] / g.dz), 0), g.Nz - 1)
        ir = min(max(math.floor(math.sqrt(x[i] * x[i] + y[i] * y[i]) / g.dr), 0), g.Nr - 1)
        assert keys[i] == iz * g.Nr + ir
    perm = O.sort_permutation(keys)
    assert list(perm) == sorted(range(len(x)), key=lambda i: (keys[i], i))


# -------------------------------------------------------------------- deposit
def _brute_rho(g, xs, ys, zs, ws, q):
    """Single-particle loops with atan2 and complex exponentials (independent path)."""
    out = np.zeros((g.Nm, g.Nr, g.Nz), complex)
    for x, y, z, w in zip(xs, ys, zs, ws):
        r = math.hypot(x, y)
        th = math.atan2(y, x) if r > 0 else 0.0
        i = math.floor(z / g.dz)
        s = z / g.dz - i
        u = r / g.dr - 0.5
        j = math.floor(u)
        t = u - j
        for di, wz in ((0, 1 - s), (1, s)):
            for dj, wr in ((0, 1 - t), (1, t)):
                jj, ii = j + dj, (i + di) % g.Nz
                for m in range(g.Nm):
                    sign = 1.0
                    jn = jj
                    if jj < 0:
                        jn, sign = 0, (-1.0) ** m
                    if jn >= g.Nr:
                        continue
                    V = 2 * math.pi * (jn + 0.5) * g.dr * g.dr * g.dz
                    out[m, jn, ii] += sign * q * w * wz * wr * cmath.exp(1j * m * th) / V
    return out


def test_deposit_rho_brute_force_including_axis_and_edge():
    g = _grid()
    rng = np.random.default_rng(1)
    x, y, z = _random_particles(g, 60, rng)
    # particles inside the first half cell (axis fold) and in the last cell (dropped node)
    x[:5], y[:5] = 0.2 * g.dr * np.cos(np.arange(5)), 0.2 * g.dr * np.sin(np.arange(5))
    x[5:10], y[5:10] = (g.R - 0.2 * g.dr) * np.cos(np.arange(5)), (g.R - 0.2 * g.dr) * np.sin(np.arange(5))
    x[10], y[10] = 0.0, 0.0
    w = rng.uniform(0.5, 2.0, 60)
    got = O.deposit_rho(g, x, y, z, w, -O.Q_E)
    ref = _brute_rho(g, x, y, z, w, -O.Q_E)
    assert np.abs(got - ref).max() < 1e-12 * np.abs(ref).max()


def test_deposit_total_charge_and_ring_modes():
    g = _grid()
    rng = np.random.default_rng(2)
    x, y, z = _random_particles(g, 1000, rng, r_max=g.R - g.dr)   # no dropped node
    w = rng.uniform(0.5, 2.0, 1000)
    rho = O.deposit_rho(g, x, y, z, w, 1.0)
    V = g.cell_volume()[:, None]
    assert (rho[0] * V).sum().real == pytest.approx(w.sum(), rel=1e-13)
    # ring of identical particles at one (r, z): rho_m = rho_0 e^{i m theta0}
    th0 = 0.7
    n = 7
    rr, zz = 2.3 * g.dr, 3.3 * g.dz
    xs, ys = np.full(n, rr * math.cos(th0)), np.full(n, rr * math.sin(th0))
    rho = O.deposit_rho(g, xs, ys, np.full(n, zz), np.ones(n), 1.0)
    for m in range(1, g.Nm):
        assert np.allclose(rho[m], rho[0] * cmath.exp(1j * m * th0), atol=1e-12 * np.abs(rho[0]).max())
    # evenly spaced ring: modes m = 1..n-1 cancel
    ths = 2 * np.pi * np.arange(n) / n + 0.1
    rho = O.deposit_rho(g, rr * np.cos(ths), rr * np.sin(ths), np.full(n, zz), np.ones(n), 1.0)
    assert np.abs(rho[1:]).max() < 1e-12 * np.abs(rho[0]).max()


def test_deposit_current_is_velocity_times_density():
    """J_z of particles all moving with v_z = V is V rho; a purely azimuthal velocity of
    a ring gives J_theta = v_theta rho and J_r = 0 (R-deposit)."""
    g = _grid()
    rng = np.random.default_rng(3)
    x, y, z = _random_particles(g, 200, rng)
    w = rng.uniform(1, 2, 200)
    rho = O.deposit_rho(g, x, y, z, w, 1.0)
    Jr, Jt, Jz = O.deposit_current(g, x, y, z, 0 * x, 0 * x, np.full(200, 3.0e7), w, 1.0)
    assert np.allclose(Jz, 3.0e7 * rho, atol=1e-12 * 3.0e7 * np.abs(rho).max())
    assert np.abs(Jr).max() == 0 and np.abs(Jt).max() == 0
    r = np.hypot(x, y)
    vth = 1.0e6
    vx, vy = -vth * y / r, vth * x / r
    Jr, Jt, Jz = O.deposit_current(g, x, y, z, vx, vy, 0 * x, w, 1.0)
    # r/theta fold sign differs from the scalar one, so compare away from the axis cell
    assert np.allclose(Jt[:, 1:], vth * rho[:, 1:], atol=1e-9 * vth * np.abs(rho).max())
    assert np.abs(Jr[:, 1:]).max() < 1e-9 * vth * np.abs(rho).max()


# -------------------------------------------------------------------- gather
def test_gather_linear_field_exact_and_mode_phase():
    g = _grid(Nz=32, Nr=16)
    rng = np.random.default_rng(4)
    n = 300
    r = rng.uniform(0.5 * g.dr, g.R - 1.5 * g.dr, n)     # interior: no fold, no drop
    th = rng.uniform(0, 2 * np.pi, n)
    z = rng.uniform(0, g.L - 1.01 * g.dz, n)             # no periodic wrap
    x, y = r * np.cos(th), r * np.sin(th)
    zn = np.arange(g.Nz) * g.dz
    rn = g.r
    sh = (g.Nm, g.Nr, g.Nz)
    Ez = np.zeros(sh, complex)
    Ez[0] = 1.5 + 2e6 * zn[None, :] - 3e6 * rn[:, None]
    A = 0.3 - 0.8j
    Ez[1] = A
    zero = np.zeros(sh, complex)
    F = O.gather(g, (zero, zero, Ez), (zero, zero, zero), x, y, z)
    ref = 1.5 + 2e6 * z - 3e6 * r + 2 * np.real(A * np.exp(-1j * th))
    assert np.allclose(F[2], ref, atol=1e-12 * np.abs(ref).max())
    # E_r of mode 0 rotates into E_x, E_y
    Er = np.zeros(sh, complex)
    Er[0] = 2.0
    F = O.gather(g, (Er, zero, zero), (zero, zero, zero), x, y, z)
    assert np.allclose(F[0], 2 * np.cos(th)) and np.allclose(F[1], 2 * np.sin(th))


def test_gather_is_adjoint_of_deposit():
    """sum_p q w_p F(x_p) = sum_nodes rho_0 F V for an m=0 scalar field: gather uses the
    same weights, fold and drop as deposit (momentum-conserving pairing)."""
    g = _grid(Nm=1)
    rng = np.random.default_rng(5)
    x, y, z = _random_particles(g, 400, rng)
    w = rng.uniform(0.5, 2, 400)
    F = np.zeros((1, g.Nr, g.Nz), complex)
    F[0] = rng.normal(size=(g.Nr, g.Nz))
    zero = np.zeros_like(F)
    Fp = O.gather(g, (zero, zero, F), (zero, zero, zero), x, y, z)[2]
    rho = O.deposit_rho(g, x, y, z, w, 1.0)
    lhs = (w * Fp).sum()
    rhs = (rho[0].real * F[0].real * g.cell_volume()[:, None]).sum()
    assert lhs == pytest.approx(rhs, rel=1e-12)


# -------------------------------------------------------------------- push
def test_boris_pure_electric_field():
    q, m, dt = -O.Q_E, O.M_E, 1e-16
    u = np.array([1e6, -2e7, 3e8])
    E = np.array([1e11, 2e10, -5e11])
    out = O.boris_push(*u, *E, 0.0, 0.0, 0.0, q, m, dt)
    assert np.allclose(out, u + q * E * dt / m, rtol=1e-15, atol=1e-15 * np.abs(u).max())


def test_boris_pure_magnetic_field_rotation():
    q, m, dt = -O.Q_E, O.M_E, 3e-14
    u = np.array([2e8, -1e8, 5e7])
    Bv = np.array([300.0, -100.0, 800.0])
    out = np.array(O.boris_push(*u, 0.0, 0.0, 0.0, *Bv, q, m, dt))
    assert np.linalg.norm(out) == pytest.approx(np.linalg.norm(u), rel=1e-14)
    gam = math.sqrt(1 + (u @ u) / O.C_LIGHT ** 2)
    t = q * dt / (2 * m * gam) * Bv
    bh = Bv / np.linalg.norm(Bv)
    up, op_ = u - (u @ bh) * bh, out - (out @ bh) * bh
    ang = math.atan2(np.linalg.norm(np.cross(up, op_)), up @ op_)
    assert ang == pytest.approx(2 * math.atan(np.linalg.norm(t)), rel=1e-12)
    assert out @ bh == pytest.approx(u @ bh, rel=1e-13)


def test_free_streaming_and_reflection():
    g = _grid()
    sh = (g.Nm, g.Nr, g.Nz)
    zero = np.zeros(sh, complex)
    x = np.array([0.5 * g.R, 0.999 * g.R])
    y = np.array([0.1 * g.R, 0.0])
    z = np.array([0.3 * g.L, 0.5 * g.L])
    ux = np.array([1e6, 2.9e8 * 50])
    uz = np.array([3e8, 0.0])
    P = dict(x=x, y=y, z=z, ux=ux, uy=0 * x, uz=uz, w=np.ones(2), id=np.arange(2, dtype=np.int32))
    st = O.State(g, 0, False, -O.Q_E, O.M_E, None, None, None, (zero,) * 3, (zero,) * 3,
                 None, None, None, None, {k: v.copy() for k, v in P.items()})
    O.gather_push(st)
    ig = O.inv_gamma(ux, 0 * x, uz)
    assert st.p["x"][0] == pytest.approx(x[0] + g.dt * ux[0] * ig[0], rel=1e-15)
    assert st.p["z"][0] == pytest.approx(z[0] + g.dt * uz[0] * ig[0], rel=1e-15)
    r_free = x[1] + g.dt * ux[1] * ig[1]
    assert r_free > g.R
    assert st.p["x"][1] == pytest.approx(2 * g.R - r_free, rel=1e-14)
    assert st.p["ux"][1] == pytest.approx(-ux[1], rel=1e-15)


# -------------------------------------------------------------------- diagnostics
def test_emittance_of_uncorrelated_gaussian():
    rng = np.random.default_rng(6)
    n = 200000
    sx, sux = 1e-6, 3e5
    x, y = rng.normal(0, sx, n), rng.normal(0, sx, n)
    ux, uy = rng.normal(0, sux, n), rng.normal(0, sux, n)
    z = rng.normal(0, 2e-6, n)
    uz = np.full(n, 3e11)
    d = O.beam_diagnostics(x, y, z, ux, uy, uz, np.ones(n))
    assert d["emit_nx"] == pytest.approx(sx * sux / O.C_LIGHT, rel=5 * math.sqrt(2.0 / n) * 3)
    assert d["emit_ny"] == pytest.approx(sx * sux / O.C_LIGHT, rel=5 * math.sqrt(2.0 / n) * 3)
    assert d["sigma_gamma_mean"] == pytest.approx(0.0, abs=1e-6)     # monoenergetic


def test_diagnostics_brute_force_small_beam():
    rng = np.random.default_rng(7)
    n = 40
    x, y = rng.normal(0, 1e-6, n), rng.normal(0, 2e-6, n)
    z = rng.normal(5e-6, 1e-6, n)
    ux, uy = 0.3e6 * x / 1e-6 + rng.normal(0, 1e5, n), rng.normal(0, 2e5, n)
    uz = rng.normal(1e11, 1e8, n)
    w = rng.uniform(0.5, 1.5, n)
    d = O.beam_diagnostics(x, y, z, ux, uy, uz, w)
    W = sum(w)
    mx = sum(wi * xi for wi, xi in zip(w, x)) / W
    mu = sum(wi * ui for wi, ui in zip(w, ux)) / W
    xx = sum(wi * (xi - mx) ** 2 for wi, xi in zip(w, x)) / W
    uu = sum(wi * (ui - mu) ** 2 for wi, ui in zip(w, ux)) / W
    xu = sum(wi * (xi - mx) * (ui - mu) for wi, xi, ui in zip(w, x, ux)) / W
    assert d["emit_nx"] == pytest.approx(math.sqrt(xx * uu - xu * xu) / O.C_LIGHT, rel=1e-12)
    mz = sum(wi * zi for wi, zi in zip(w, z)) / W
    sz = math.sqrt(sum(wi * (zi - mz) ** 2 for wi, zi in zip(w, z)) / W)
    slices = {}
    for wi, zi, uxi, uyi, uzi in zip(w, z, ux, uy, uz):
        dd = zi - mz + 3 * sz
        if 0 <= dd < 6 * sz:
            gam = math.sqrt(1 + (uxi ** 2 + uyi ** 2 + uzi ** 2) / O.C_LIGHT ** 2)
            slices.setdefault(math.floor(dd / O.SLICE_LEN), []).append((wi, gam))
    sig = []
    for k in sorted(slices):
        ws = sum(a for a, _ in slices[k])
        gm = sum(a * b for a, b in slices[k]) / ws
        sig.append(math.sqrt(sum(a * (b - gm) ** 2 for a, b in slices[k]) / ws))
    assert np.allclose(d["slice_sigma_gamma"], sig, rtol=1e-10, atol=1e-12)
    assert d["sigma_gamma_mean"] == pytest.approx(np.mean(sig), rel=1e-10)


def test_error_metrics():
    assert O.err_emittance(1.05, 1.0) == pytest.approx(0.05)
    assert O.err_sigma_gamma([1.1, 0.9], [1.0, 1.0]) == pytest.approx(0.1)
