"""Pins of the oracle's source path: the spectral transform of (rho, J), the vector axis
fold of the current deposit, and the time centring of J.

Section "Finite order pseudo-spectral solvers": Hankel transform along r of order m+1
for the '+' component, m-1 for the '-' component and m for z and scalars (the operator
table Eq. qcyl-ops only holds with these orders, see the convention tests of
``test_oracle_transforms.py``); Eq. psatd-eqE/eqB: J constant over the step and centred
at t^{n+1/2}, rho at t^n and t^{n+1}.  Each test here is chosen so that a plausible
slip in the oracle (swapped Hankel orders of J_+ and J_-, a sign of i J_theta, the
scalar fold sign used for r/theta components, J taken at x^n) fails it.
"""
import cmath
import math

import numpy as np
import pytest
from scipy.special import jv

from oracle import psatd_rz as O

DZ = 0.05e-6


def _grid(Nz=16, Nr=12, Nm=3):
    return O.Grid(Nz, Nr, Nm, DZ, DZ, DZ / O.C_LIGHT)


# ----------------------------------------------------------------- transforms of (rho, J)
def _analytic_mode(g, kp, f, m, coeffs):
    """Real-space mode-m amplitudes of the spectral basis function with (+, -, z, rho)
    coefficients ``coeffs`` at radial wavenumber kp and FFT bin f, built from Bessel
    functions directly: V_+ = a J_{m+1}(kp r) e^{i k_z z}, V_- = b J_{m-1}(kp r) e^{i k_z z},
    V_z = c J_m(kp r) e^{i k_z z}, rho = d J_m(kp r) e^{i k_z z};
    V_r = V_+ + V_-, V_theta = i (V_+ - V_-)."""
    a, b, c, d = coeffs
    r = g.r[:, None]
    ph = np.exp(1j * g.kz[f] * (np.arange(g.Nz) * g.dz))[None, :]
    Vp = a * jv(m + 1, kp * r) * ph
    Vm = b * jv(m - 1, kp * r) * ph
    return Vp + Vm, 1j * (Vp - Vm), c * jv(m, kp * r) * ph, d * jv(m, kp * r) * ph


@pytest.mark.parametrize("m,n,f", [(0, 2, 3), (1, 4, 5), (2, 1, 13), (1, 0, 0)])
def test_forward_sources_of_analytic_basis_modes(m, n, f):
    """A real-space source built from J_{m+1}, J_{m-1}, J_m at k_{m,n} transforms to the
    unit coefficient at (n, f) in the slot of its Hankel order; the '-' slot, whose
    order m-1 basis misses the Dini k=0 function for m >= 1, is checked by
    reconstruction in real space."""
    g = _grid()
    h = O.hankel_setup(g)
    coeffs = (0.7 - 0.2j, -0.4 + 0.9j, 0.3 + 0.5j, 1.1 - 0.6j)
    sh = (g.Nm, g.Nr, g.Nz)
    rho = np.zeros(sh, complex)
    Jr, Jt, Jz = (np.zeros(sh, complex) for _ in range(3))
    Vr, Vt, Vz, S = _analytic_mode(g, h.kperp[m][n], f, m, coeffs)
    Jr[m], Jt[m], Jz[m], rho[m] = Vr, Vt, Vz, S
    rho_h, Jp_h, Jm_h, Jz_h = O.forward_sources(g, h, rho, Jr, Jt, Jz)
    unit = np.zeros((g.Nr, g.Nz), complex)
    unit[n, f] = g.Nz                       # forward DFT is unnormalised
    a, b, c, d = coeffs
    tol = 1e-10 * g.Nz
    assert np.abs(rho_h[m] - d * unit).max() < tol
    assert np.abs(Jz_h[m] - c * unit).max() < tol
    assert np.abs(Jp_h[m] - a * unit).max() < tol
    if m == 0:
        # order -1 = -J_1 on the zeros of J_0: full rank, exact unit coefficient
        assert np.abs(Jm_h[m] - b * unit).max() < tol
    else:
        # B_{m-1} M_{m-1} B_{m-1} differs from B_{m-1} by at most the dropped singular
        # value (R-dht), so the reconstruction is the sampled J_{m-1} to that level
        B = h.Binv[m][0]
        ph = np.exp(1j * g.kz[f] * np.arange(g.Nz) * g.dz)[None, :]
        want = np.fft.fft(b * jv(m - 1, h.kperp[m][n] * g.r)[:, None] * ph, axis=-1)
        bound = 2 * O.PINV_RCOND * np.linalg.norm(B, 2) * abs(b) * g.Nz
        assert np.abs(B @ Jm_h[m] - want).max() < bound
        assert bound < 0.05 * np.abs(want).max()
    for other in range(g.Nm):
        if other != m:
            for arr in (rho_h, Jp_h, Jm_h, Jz_h):
                assert np.abs(arr[other]).max() == 0.0


@pytest.mark.parametrize("m,n,f", [(0, 3, 2), (1, 2, 7), (2, 5, 12)])
def test_inverse_vector_of_unit_modes_is_the_bessel_field(m, n, f):
    """The inverse transform of a unit spectral coefficient in the '+', '-' or z slot is
    the sampled Bessel function of that slot's order (R-modes), independently of the
    forward matrices."""
    g = _grid()
    h = O.hankel_setup(g)
    coeffs = (0.6 + 0.3j, -0.2 - 0.8j, 0.9 - 0.1j, 0.0)
    sh = (g.Nm, g.Nr, g.Nz)
    Vh = [np.zeros(sh, complex) for _ in range(3)]
    for slot, cf in enumerate(coeffs[:3]):
        Vh[slot][m, n, f] = cf * g.Nz         # inverse DFT divides by Nz
    Vr, Vt, Vz = O.inverse_vector(g, h, *Vh)
    Ar, At, Az, _ = _analytic_mode(g, h.kperp[m][n], f, m, coeffs)
    for got, ref in ((Vr[m], Ar), (Vt[m], At), (Vz[m], Az)):
        assert np.abs(got - ref).max() < 1e-12


def test_forward_sources_agrees_with_the_vector_transform_on_random_data():
    """(J_+, J_-, J_z) of forward_sources equal forward_vector's transform of the same
    (J_r, J_theta, J_z), and rho equals forward_scalar's (both routes state the same
    transform; the one of forward_vector is pinned by the tests above and the round
    trip)."""
    g = _grid(Nz=8, Nr=10, Nm=3)
    h = O.hankel_setup(g)
    rng = np.random.default_rng(11)
    sh = (g.Nm, g.Nr, g.Nz)
    rho, Jr, Jt, Jz = (rng.normal(size=sh) + 1j * rng.normal(size=sh) for _ in range(4))
    rho_h, Jp_h, Jm_h, Jz_h = O.forward_sources(g, h, rho, Jr, Jt, Jz)
    Vp, Vm, Vz = O.forward_vector(g, h, Jr, Jt, Jz)
    assert np.abs(Jp_h - Vp).max() == 0 and np.abs(Jm_h - Vm).max() == 0
    assert np.abs(Jz_h - Vz).max() == 0
    assert np.abs(rho_h - O.forward_scalar(g, h, rho)).max() == 0


# ----------------------------------------------------------------- vector axis fold
def _random_particles(g, n, rng, r_max):
    r = r_max * np.sqrt(rng.uniform(0, 1, n))
    th = rng.uniform(0, 2 * np.pi, n)
    return r * np.cos(th), r * np.sin(th), rng.uniform(0, g.L, n)


@pytest.mark.parametrize("axis", ["x", "y"])
def test_current_of_a_uniform_cartesian_drift_matches_shifted_density_modes(axis):
    """J = v rho for particles sharing one Cartesian velocity v along x (or y).  In modes,
    v_r = v cos(theta), v_theta = -v sin(theta) (or v sin, v cos), so
      J_r,m = (v/2)(rho_{m+1} + rho_{m-1}),  J_theta,m = (i v/2)(rho_{m+1} - rho_{m-1})
    (x drift; for y: J_r,m = (v/2i)(rho_{m+1} - rho_{m-1}), J_theta,m = (v/2)(...+...)),
    with rho_{-1} = conj(rho_1).  The identity holds node by node, the axis cell
    included, only when the r/theta components fold across the axis with the sign of
    the modes m +- 1, i.e. (-1)^{m+1}."""
    g = _grid(Nz=8, Nr=6, Nm=3)
    g_rho = O.Grid(g.Nz, g.Nr, g.Nm + 1, g.dz, g.dr, g.dt)   # modes 0..Nm for rho_{m+1}
    rng = np.random.default_rng(21)
    n = 400
    x, y, z = _random_particles(g, n, rng, r_max=2.5 * g.dr)   # many inside the axis cell
    w = rng.uniform(0.5, 2.0, n)
    v = 2.3e7
    zero = np.zeros(n)
    vx, vy = (np.full(n, v), zero) if axis == "x" else (zero, np.full(n, v))
    Jr, Jt, _ = O.deposit_current(g, x, y, z, vx, vy, zero, w, 1.0)
    rho = O.deposit_rho(g_rho, x, y, z, w, 1.0)

    def rho_m(k):
        return np.conj(rho[1]) if k == -1 else rho[k]

    for m in range(g.Nm):
        plus, minus = rho_m(m + 1), rho_m(m - 1)
        if axis == "x":
            er, et = 0.5 * v * (plus + minus), 0.5j * v * (plus - minus)
        else:
            er, et = v / 2j * (plus - minus), 0.5 * v * (plus + minus)
        scale = v * np.abs(rho).max()
        assert np.abs(Jr[m] - er).max() < 1e-12 * scale
        assert np.abs(Jt[m] - et).max() < 1e-12 * scale
    # the axis cell carries folded contributions: the test is not vacuous there
    assert np.abs(Jr[1:, 0, :]).max() > 0.1 * np.abs(Jr[1:]).max()


def _brute_current(g, xs, ys, zs, vxs, vys, vzs, ws, q):
    """Single-particle loops: atan2, complex exponentials, and the ghost node r = -dr/2
    treated geometrically as the point (dr/2, theta + pi), where the velocity is
    re-projected on the radial and azimuthal directions of that angle."""
    Jr = np.zeros((g.Nm, g.Nr, g.Nz), complex)
    Jt = np.zeros_like(Jr)
    Jz = np.zeros_like(Jr)
    for x, y, z, vx, vy, vz, w in zip(xs, ys, zs, vxs, vys, vzs, ws):
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
                ang = th
                if jj < 0:                       # ghost node: node 0 seen at theta + pi
                    jj, ang = 0, th + math.pi
                if jj >= g.Nr:
                    continue
                vr = vx * math.cos(ang) + vy * math.sin(ang)
                vt = -vx * math.sin(ang) + vy * math.cos(ang)
                V = 2 * math.pi * (jj + 0.5) * g.dr * g.dr * g.dz
                for m in range(g.Nm):
                    base = q * w * wz * wr * cmath.exp(1j * m * ang) / V
                    Jr[m, jj, ii] += base * vr
                    Jt[m, jj, ii] += base * vt
                    Jz[m, jj, ii] += base * vz
    return Jr, Jt, Jz


def test_current_deposit_brute_force_including_the_axis_cell():
    g = _grid(Nz=8, Nr=5, Nm=3)
    rng = np.random.default_rng(22)
    n = 80
    x, y, z = _random_particles(g, n, rng, r_max=g.R * 0.999)
    x[:20], y[:20] = (0.45 * g.dr * np.sqrt(rng.uniform(0, 1, 20)) * np.cos(np.arange(20)),
                      0.45 * g.dr * np.sqrt(rng.uniform(0, 1, 20)) * np.sin(np.arange(20)))
    vx, vy, vz = (rng.normal(0, 1e7, n) for _ in range(3))
    w = rng.uniform(0.5, 2.0, n)
    got = O.deposit_current(g, x, y, z, vx, vy, vz, w, -O.Q_E)
    ref = _brute_current(g, x, y, z, vx, vy, vz, w, -O.Q_E)
    for a, b in zip(got, ref):
        assert np.abs(a - b).max() < 1e-12 * np.abs(b).max()
    assert np.abs(ref[0][:, 0, :]).max() > 0      # axis-cell contributions exist


# ----------------------------------------------------------------- time centring of J
def _drifting_ring(g, nz_lattice, v):
    """Particles on a fine z lattice (spacing dz/nz_lattice) forming a smooth Gaussian
    density along z, on one evenly spaced ring in r (so only mode 0 is non-zero away
    from rounding), all with the same velocity v along z and no field."""
    zs = (np.arange(g.Nz * nz_lattice) + 0.5) * (g.dz / nz_lattice)
    zc, sig = 0.5 * g.L, 2.5 * g.dz
    dens = np.exp(-0.5 * ((zs - zc) / sig) ** 2)
    nth = 4
    th = 2 * np.pi * np.arange(nth) / nth + 0.3
    r0 = 2.4 * g.dr
    X = np.repeat(r0 * np.cos(th)[None, :], len(zs), 0).ravel()
    Y = np.repeat(r0 * np.sin(th)[None, :], len(zs), 0).ravel()
    Z = np.repeat(zs[:, None], nth, 1).ravel()
    Wt = np.repeat(dens[:, None], nth, 1).ravel()
    gam = 1.0 / math.sqrt(1.0 - (v / O.C_LIGHT) ** 2)
    n = len(Z)
    return dict(x=X, y=Y, z=Z, ux=np.zeros(n), uy=np.zeros(n), uz=np.full(n, gam * v),
                w=Wt, id=np.arange(n, dtype=np.int32))


def _continuity_residual(dt_factor):
    """Relative residual of (rho^{n+1} - rho^n)/dt + d_z J_z^{n+1/2} (spectral d_z,
    per r row) after one field-free gather_push."""
    Nz = 64
    g = O.Grid(Nz, 6, 1, DZ, DZ, dt_factor * DZ / O.C_LIGHT)
    v = 0.6 * O.C_LIGHT
    P = _drifting_ring(g, 40, v)
    zero = np.zeros((g.Nm, g.Nr, g.Nz), complex)
    st = O.State(g, 0, False, 1.0, O.M_E, None, None, None, (zero,) * 3, (zero,) * 3,
                 None, None, None, None, {k: a.copy() for k, a in P.items()})
    rho0 = O.deposit_rho(g, P["x"], P["y"], P["z"], P["w"], 1.0)
    _, _, Jz = O.gather_push(st)
    rho1 = O.deposit_rho(g, st.p["x"], st.p["y"], st.p["z"], st.p["w"], 1.0)
    drho = np.fft.fft((rho1 - rho0)[0], axis=-1) / g.dt
    divJ = 1j * g.kz[None, :] * np.fft.fft(Jz[0], axis=-1)
    return np.abs(drho + divJ).max() / np.abs(divJ).max()


def test_current_is_centred_between_the_two_densities():
    """Continuity (rho^{n+1} - rho^n)/dt + div J = 0 is met to second order in dt only
    when J is deposited at the mid-step position x^{n+1/2} (Eq. psatd-eqE/eqB: J at
    n+1/2, rho at n and n+1): the residual is small and falls by ~4 when dt halves.
    A J taken at x^n or x^{n+1} leaves a first-order residual (falls by ~2)."""
    r1 = _continuity_residual(1.0)
    r2 = _continuity_residual(0.5)
    assert r1 < 5e-3
    assert r1 / r2 > 3.2


def test_gather_push_current_equals_deposit_at_the_half_step_position():
    g = _grid(Nz=16, Nr=8, Nm=2)
    rng = np.random.default_rng(23)
    n = 50
    x, y, z = _random_particles(g, n, rng, r_max=0.8 * g.R)
    u = rng.normal(0, 0.5 * O.C_LIGHT, (3, n))
    P = dict(x=x, y=y, z=z, ux=u[0], uy=u[1], uz=u[2], w=rng.uniform(0.5, 2, n),
             id=np.arange(n, dtype=np.int32))
    zero = np.zeros((g.Nm, g.Nr, g.Nz), complex)
    st = O.State(g, 0, False, -O.Q_E, O.M_E, None, None, None, (zero,) * 3, (zero,) * 3,
                 None, None, None, None, {k: a.copy() for k, a in P.items()})
    J = O.gather_push(st)
    ig = O.inv_gamma(*u)
    v = u * ig
    hdt = 0.5 * g.dt
    zh = O.wrap_z(g, z + hdt * v[2])
    ref = O.deposit_current(g, x + hdt * v[0], y + hdt * v[1], zh, *v, P["w"], -O.Q_E)
    for a, b in zip(J, ref):
        assert np.abs(a - b).max() <= 1e-13 * np.abs(b).max()


# ----------------------------------------------------------------- vector axis fold, gather
def test_gather_reproduces_uniform_and_linear_cartesian_fields_across_the_axis():
    """Fields whose mode amplitudes are constant or linear in r are gathered exactly
    by linear interpolation anywhere inside r < R - dr, the axis cell included, only if
    the ghost node r = -dr/2 takes the value the field has there:
      * E = E0 x_hat (uniform): mode 1 with E_r,1 = E0/2, E_theta,1 = -i E0/2 at every
        node; the r/theta fold sign of m = 1 must be +1;
      * E = a (x, y) (radial, linear): mode 0 with E_r,0 = a r; fold sign -1 at m = 0;
      * S = b x (scalar, linear): mode 1 with S_1 = b r/2; fold sign -1 at m = 1."""
    g = _grid(Nz=8, Nr=6, Nm=2)
    rng = np.random.default_rng(24)
    n = 300
    x, y, z = _random_particles(g, n, rng, r_max=g.R - 1.01 * g.dr)
    x[:100], y[:100] = x[:100] * 0.04, y[:100] * 0.04         # inside the axis cell
    sh = (g.Nm, g.Nr, g.Nz)
    zero = np.zeros(sh, complex)
    E0, a, b = 3.0e9, 2.0e15, -5.0e14
    Er, Et = zero.copy(), zero.copy()
    Er[1], Et[1] = 0.5 * E0, -0.5j * E0
    Er[0] = a * g.r[:, None]
    Sz = zero.copy()
    Sz[1] = 0.5 * b * g.r[:, None]
    Ex, Ey, Ez, Bx, By, Bz = O.gather(g, (Er, Et, Sz), (zero, zero, zero), x, y, z)
    scale = E0 + a * g.R + abs(b) * g.R
    assert np.abs(Ex - (E0 + a * x)).max() < 1e-12 * scale
    assert np.abs(Ey - a * y).max() < 1e-12 * scale
    assert np.abs(Ez - b * x).max() < 1e-12 * scale
