"""Plain FP64 numpy oracle of one quasi-cylindrical arbitrary-order PSATD PIC cycle.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

Paper: Jalas et al., arXiv:1611.05712.  Sections are cited by their titles:
"Finite order pseudo-spectral solvers" (FOPS), "Numerical Cherenkov radiation"
(NCR) and "Accurate modeling of plasma accelerators in finite order PSATD"
(AMPA).  Equations by their labels: Eq. psatd-eqE / psatd-eqB (Cartesian
PSATD), the quasi-cylindrical operator table that follows them (Eq. qcyl-ops),
Eq. finite_difference (stencil coefficients), the modified wavenumber [k_z]
(Eq. kz-mod), Eq. omega_mod, and the error metrics of AMPA (Eq. err-metrics).

Everything is SI and float64 / complex128.  Library primitives used as single
steps: ``numpy.fft`` (the DFT along z), ``@`` (dense matrix products),
``numpy.linalg.pinv`` (Moore-Penrose inverse), ``scipy.special.jv`` and
``jn_zeros`` (Bessel functions and their zeros), ``numpy.argsort`` (stable).

Readings where the paper is silent (each repeated where it is used):
  R-units   SI form of Eq. psatd-eqE/eqB, re-derived from Maxwell with J constant
            over dt and rho linear in time; mu0 is defined as 1/(eps0 c^2).
  R-grid    z nodes i*dz (periodic), r nodes (j+1/2)*dr, R = Nr*dr; k_z in FFT
            order with the Nyquist bin negative.
  R-modes   F = Re[F_0 + 2 sum_{m>=1} F_m e^{-i m theta}], F_pm = (F_r -/+ i F_theta)/2,
            F_+ carries Hankel order m+1, F_- order m-1, F_z and scalars order m;
            d/dz -> +i k_z.  Projection onto mode m uses e^{+i m theta}.
  R-dht     k_{m,n} = (n-th zero of J_m)/R shared by the three orders; inverse
            matrix B_p[j,n] = J_p(k_{m,n} r_j); forward matrix = pinv(B_p) with
            singular values <= 1e-3 * sigma_max discarded (B_{m-1} has one
            near-null direction, the Dini k=0 function r^{m-1}).
  R-deposit linear weights in z and r, ghost node j=-1 folded into node 0 with
            sign (-1)^m (scalars, z) or (-1)^{m+1} (r, theta); node Nr dropped;
            cell volume 2 pi r_j dr dz; J at x^{n+1/2}, rho at x^{n+1}.
  R-filter  sources multiplied by cos^2(k_z dz/2) cos^2(k_perp dr/2).
  R-corr    global spectral current correction with grad/div of Eq. qcyl-ops.
  R-push    relativistic Boris push; positions advanced in two half steps;
            specular reflection at r >= R; periodic z.
  R-init    beam fields from a relativistic spectral Poisson solve.
  R-diag    normalised rms emittance; slice energy spread over 0.5 um slices in
            [zbar - 3 sigma_z, zbar + 3 sigma_z).
  R-window  moving window on a ring of z columns: removal behind the back edge,
            re-injection of each column's initial plasma at the front, departing
            column of E, B zeroed (section "Moving window" below).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np
from scipy.special import jn_zeros, jv

# CODATA 2018 (R-units).  mu0 is tied to eps0 and c so that mu0 eps0 c^2 = 1.
C_LIGHT = 299792458.0
EPS0 = 8.8541878128e-12
MU0 = 1.0 / (EPS0 * C_LIGHT * C_LIGHT)
Q_E = 1.602176634e-19
M_E = 9.1093837015e-31

PINV_RCOND = 1e-3          # R-dht singular-value cutoff, relative to sigma_max
SMALL_X = 0.25             # below this omega*dt the PSATD coefficients use series
SLICE_LEN = 0.5e-6         # AMPA: slices of 0.5 um for the slice energy spread


# --------------------------------------------------------------------------
# Grid (R-grid)
# --------------------------------------------------------------------------
@dataclass
class Grid:
    """The (z, r) grid of one azimuthal-mode set (FOPS: modes on separate 2D grids)."""

    Nz: int
    Nr: int
    Nm: int
    dz: float
    dr: float
    dt: float

    @property
    def L(self) -> float:
        return self.Nz * self.dz

    @property
    def R(self) -> float:
        return self.Nr * self.dr

    @property
    def r(self) -> np.ndarray:
        return (np.arange(self.Nr) + 0.5) * self.dr

    @property
    def kz(self) -> np.ndarray:
        """k_z = 2 pi f / (Nz dz), f in FFT order (R-grid)."""
        return 2.0 * np.pi * np.fft.fftfreq(self.Nz, d=self.dz)

    def cell_volume(self) -> np.ndarray:
        """Volume of the ring around node j: 2 pi r_j dr dz (R-deposit)."""
        return 2.0 * np.pi * self.r * self.dr * self.dz


# --------------------------------------------------------------------------
# Arbitrary-order stencil (FOPS, Eq. finite_difference and Eq. kz-mod)
# --------------------------------------------------------------------------
def fd_coefficients(n: int) -> np.ndarray:
    """alpha_{n,j}, j = 1..n, of the centred derivative of stencil order 2n.

    Eq. finite_difference: alpha_{n,j} = (-1)^{j+1} 2 (n!)^2 / ((n-j)! (n+j)!).
    The ratio of factorials is evaluated as the product
    prod_{i=1..j} (n-i+1)/(n+i), which is the same number and does not overflow.
    """
    if n < 1:
        raise ValueError("stencil half-width n must be >= 1")
    out = np.empty(n)
    prod = 1.0
    for j in range(1, n + 1):
        prod *= (n - j + 1) / (n + j)
        out[j - 1] = (2.0 if j % 2 == 1 else -2.0) * prod
    return out


def modified_kz(kz: np.ndarray, dz: float, order_p: int) -> np.ndarray:
    """[k_z] of a stencil of order p = 2n (Eq. kz-mod); order_p = 0 means infinite order.

    [k_z] = sum_{j=1}^{n} alpha_{n,j} sin(k_z j dz) / (j dz).  With infinite
    order the exact k_z is used (PSATD_inf).
    """
    kz = np.asarray(kz, dtype=np.float64)
    if order_p == 0:
        return kz.copy()
    if order_p < 2 or order_p % 2:
        raise ValueError("stencil order must be an even number >= 2 (or 0 for infinite)")
    n = order_p // 2
    alpha = fd_coefficients(n)
    out = np.zeros_like(kz)
    for j in range(1, n + 1):
        out += alpha[j - 1] * np.sin(kz * (j * dz)) / (j * dz)
    return out


# --------------------------------------------------------------------------
# Discrete Hankel transform (FOPS: Hankel along r, Fourier along z; R-dht)
# --------------------------------------------------------------------------
@dataclass
class Hankel:
    """Per-mode spectral radial grid and the six transform matrices.

    ``kperp[m]`` has Nr entries.  Slot order of ``Binv[m]`` / ``M[m]``:
    0 = '-' component (Bessel order m-1), 1 = 'z' and scalars (order m),
    2 = '+' component (order m+1).
    """

    kperp: list = field(default_factory=list)
    Binv: list = field(default_factory=list)
    M: list = field(default_factory=list)


def hankel_setup(g: Grid, rcond: float = PINV_RCOND) -> Hankel:
    """Build the DHT matrices of every mode (FOPS quasi-cylindrical transform; R-dht).

    k_{m,n} = alpha_{m,n} / R with alpha_{m,n} the n-th positive zero of J_m.
    Inverse transform  F(r_j) = sum_n Fhat_n J_p(k_{m,n} r_j)  (matrix Binv_p).
    Forward transform  Fhat = pinv(Binv_p) F, singular values below
    rcond * sigma_max dropped.  J_{-1} = -J_1 (scipy's jv follows it).
    """
    h = Hankel()
    r = g.r
    for m in range(g.Nm):
        kp = jn_zeros(m, g.Nr) / g.R
        h.kperp.append(kp)
        bs, ms = [], []
        for p in (m - 1, m, m + 1):
            B = jv(p, np.outer(r, kp))
            bs.append(B)
            ms.append(np.linalg.pinv(B, rtol=rcond))
        h.Binv.append(bs)
        h.M.append(ms)
    return h


def fft_z(F: np.ndarray) -> np.ndarray:
    """Forward DFT along z: Fhat(k_z) = sum_i F(z_i) e^{-i k_z z_i} (R-modes)."""
    return np.fft.fft(F, axis=-1)


def ifft_z(Fh: np.ndarray) -> np.ndarray:
    """Inverse DFT along z with the 1/Nz normalisation."""
    return np.fft.ifft(Fh, axis=-1)


def forward_sources(g: Grid, h: Hankel, rho, Jr, Jt, Jz):
    """Real-space (rho, J_r, J_theta, J_z)[m] -> spectral (rho, J_+, J_-, J_z)[m].

    FOPS: Fourier along z, then Hankel along r of order m (rho, J_z),
    m+1 (J_+) and m-1 (J_-), with J_pm = (J_r -/+ i J_theta)/2 (R-modes).
    Arrays are [Nm, Nr, Nz] complex.
    """
    rho_h = np.empty_like(rho)
    Jp_h = np.empty_like(Jr)
    Jm_h = np.empty_like(Jr)
    Jz_h = np.empty_like(Jz)
    for m in range(g.Nm):
        Jp = 0.5 * (Jr[m] - 1j * Jt[m])
        Jm = 0.5 * (Jr[m] + 1j * Jt[m])
        rho_h[m] = h.M[m][1] @ fft_z(rho[m])
        Jp_h[m] = h.M[m][2] @ fft_z(Jp)
        Jm_h[m] = h.M[m][0] @ fft_z(Jm)
        Jz_h[m] = h.M[m][1] @ fft_z(Jz[m])
    return rho_h, Jp_h, Jm_h, Jz_h


def forward_scalar(g: Grid, h: Hankel, S):
    """Spectral transform of a scalar grid [Nm, Nr, Nz] (order m)."""
    return np.stack([h.M[m][1] @ fft_z(S[m]) for m in range(g.Nm)])


def forward_vector(g: Grid, h: Hankel, Vr, Vt, Vz):
    """Real (r, theta, z) -> spectral (+, -, z) of a vector grid (FOPS; R-modes)."""
    Vp = np.empty_like(Vr)
    Vm = np.empty_like(Vr)
    Vzh = np.empty_like(Vz)
    for m in range(g.Nm):
        Vp[m] = h.M[m][2] @ fft_z(0.5 * (Vr[m] - 1j * Vt[m]))
        Vm[m] = h.M[m][0] @ fft_z(0.5 * (Vr[m] + 1j * Vt[m]))
        Vzh[m] = h.M[m][1] @ fft_z(Vz[m])
    return Vp, Vm, Vzh


def inverse_vector(g: Grid, h: Hankel, Vp, Vm, Vz):
    """Spectral (+, -, z)[m] -> real-space (r, theta, z)[m] (FOPS; R-modes).

    V_pm(r_j) = sum_n Binv_{m pm 1}[j, n] Vhat_pm[n], V_r = V_+ + V_-,
    V_theta = i (V_+ - V_-), then the inverse DFT along z.
    """
    Vr = np.empty_like(Vp)
    Vt = np.empty_like(Vp)
    Vzr = np.empty_like(Vz)
    for m in range(g.Nm):
        a = ifft_z(h.Binv[m][2] @ Vp[m])
        b = ifft_z(h.Binv[m][0] @ Vm[m])
        Vr[m] = a + b
        Vt[m] = 1j * (a - b)
        Vzr[m] = ifft_z(h.Binv[m][1] @ Vz[m])
    return Vr, Vt, Vzr


# --------------------------------------------------------------------------
# Spectral operators (FOPS Eq. qcyl-ops) and PSATD coefficients
# --------------------------------------------------------------------------
def op_grad(Kp, Kz, X):
    """i k X in the (+, -, z) basis: (-K_perp X/2, +K_perp X/2, i K_z X) (Eq. qcyl-ops, first row)."""
    return (-0.5 * Kp * X, 0.5 * Kp * X, 1j * Kz * X)


def op_curl(Kp, Kz, Vp, Vm, Vz):
    """i k x V in the (+, -, z) basis (Eq. qcyl-ops, second row)."""
    return (Kz * Vp - 0.5j * Kp * Vz,
            -Kz * Vm - 0.5j * Kp * Vz,
            1j * Kp * (Vp + Vm))


def op_div(Kp, Kz, Vp, Vm, Vz):
    """i k . V in the (+, -, z) basis.

    Not printed in the paper: the unique linear rule with div(grad X) = -K^2 X
    and div(curl V) = 0 for the operators of Eq. qcyl-ops (R-corr).
    """
    return Kp * (Vp - Vm) + 1j * Kz * Vz


def _series_terms(x2, kind):
    """Power series of (sin x - x)/x (kind 0) or (x cos x - sin x)/x (kind 1) divided by x^2.

    (sin x - x)/x   = sum_{k>=1} (-1)^k x^{2k} / (2k+1)!
    (x cos x - sin x)/x = sum_{k>=1} (-1)^k x^{2k} 2k / (2k+1)!
    Returned: the sum with x^{2k} replaced by x^{2k-2} (nine terms).
    """
    out = np.zeros_like(x2)
    pw = np.ones_like(x2)
    for k in range(1, 10):
        num = 1.0 if kind == 0 else 2.0 * k
        out += (-1) ** k * num / math.factorial(2 * k + 1) * pw
        pw = pw * x2
    return out


def psatd_coefficients(g: Grid, h: Hankel, order_p: int):
    """Per-cell coefficients of the SI PSATD update (Eq. psatd-eqE/eqB with [k_z], R-units).

    K_perp = k_{m,n}; K_z = [k_z]_p (Eq. kz-mod; only k_z is modified, FOPS);
    K = sqrt(K_perp^2 + K_z^2); x = c K dt; C = cos x; S = sin x.
    Returned arrays [Nm, Nr, Nz]:
      C, S_K = S/K, omc_K2 = (1-C)/K^2,
      a_next = (S/x - 1)/K^2, a_prev = (C - S/x)/K^2, inv_K2 = 1/K^2,
      Kp, Kz.  For x < SMALL_X the last two combinations use their power series
    (the direct forms cancel catastrophically there).
    """
    Kz1 = modified_kz(g.kz, g.dz, order_p)
    out = {k: np.empty((g.Nm, g.Nr, g.Nz)) for k in
           ("C", "S_K", "omc_K2", "a_next", "a_prev", "inv_K2", "Kp", "Kz")}
    cdt = C_LIGHT * g.dt
    for m in range(g.Nm):
        Kp = h.kperp[m][:, None] * np.ones((1, g.Nz))
        Kz = np.ones((g.Nr, 1)) * Kz1[None, :]
        K2 = Kp * Kp + Kz * Kz
        K = np.sqrt(K2)
        x = cdt * K
        C = np.cos(x)
        S = np.sin(x)
        small = x < SMALL_X
        a_next = np.where(small, cdt * cdt * _series_terms(x * x, 0), (S / x - 1.0) / K2)
        a_prev = np.where(small, cdt * cdt * _series_terms(x * x, 1), (C - S / x) / K2)
        sh = np.sin(0.5 * x)
        out["C"][m] = C
        out["S_K"][m] = S / K
        out["omc_K2"][m] = 2.0 * sh * sh / K2
        out["a_next"][m] = a_next
        out["a_prev"][m] = a_prev
        out["inv_K2"][m] = 1.0 / K2
        out["Kp"][m] = Kp
        out["Kz"][m] = Kz
    return out


def source_filter(g: Grid, h: Hankel):
    """Binomial source filter in spectral space (R-filter): cos^2(k_z dz/2) cos^2(k_perp dr/2)."""
    tz = np.cos(0.5 * g.kz * g.dz) ** 2
    return np.stack([np.outer(np.cos(0.5 * h.kperp[m] * g.dr) ** 2, tz) for m in range(g.Nm)])


def psatd_update(g: Grid, coef, T, E, B, J, rho_next, rho_prev, filt=True, correct=True):
    """One PSATD field push in spectral space (Eq. psatd-eqE/eqB + Eq. qcyl-ops + [k_z]).

    E, B, J: tuples (+, -, z) of [Nm, Nr, Nz] complex arrays (not modified).
    rho_next = rho^{n+1}, rho_prev = rho^n.  Steps:
      1. (R-filter) rho^{n+1}, J *= T  when filt.
      2. (R-corr) G = [(rho^{n+1}-rho^n)/dt + div J]/K^2 ; J += grad G  when correct.
      3. E^{n+1} = C E + c (S/K) curl B - (S/K)/(eps0 c) J
                   + grad(a_next rho^{n+1} + a_prev rho^n)/eps0
         B^{n+1} = C B - (S/K)/c curl E + mu0 (1-C)/K^2 curl J
    Returns (E_new, B_new, rho_next_filtered, J_used).
    """
    Kp, Kz = coef["Kp"], coef["Kz"]
    if filt:
        rho_next = rho_next * T
        J = tuple(Ji * T for Ji in J)
    if correct:
        G = ((rho_next - rho_prev) / g.dt + op_div(Kp, Kz, *J)) * coef["inv_K2"]
        gG = op_grad(Kp, Kz, G)
        J = tuple(Ji + gi for Ji, gi in zip(J, gG))
    C, S_K = coef["C"], coef["S_K"]
    cB = op_curl(Kp, Kz, *B)
    cE = op_curl(Kp, Kz, *E)
    cJ = op_curl(Kp, Kz, *J)
    gX = op_grad(Kp, Kz, (coef["a_next"] * rho_next + coef["a_prev"] * rho_prev) / EPS0)
    E_new = tuple(C * E[i] + C_LIGHT * S_K * cB[i] - S_K / (EPS0 * C_LIGHT) * J[i] + gX[i]
                  for i in range(3))
    B_new = tuple(C * B[i] - S_K / C_LIGHT * cE[i] + MU0 * coef["omc_K2"] * cJ[i]
                  for i in range(3))
    return E_new, B_new, rho_next, J


def beam_fields(g: Grid, coef, rho_h, gamma):
    """Space-charge fields of a beam moving along +z with Lorentz factor gamma (R-init).

    Relativistic Poisson solve phi = rho / (eps0 (K_perp^2 + K_z^2/gamma^2)),
    E = (+K_perp phi/2, -K_perp phi/2, -i K_z phi/gamma^2),  B = curl(0, 0, beta phi / c).
    Returns spectral (E, B) tuples (+, -, z).
    """
    Kp, Kz = coef["Kp"], coef["Kz"]
    beta = math.sqrt(1.0 - 1.0 / (gamma * gamma))
    phi = rho_h / (EPS0 * (Kp * Kp + Kz * Kz / (gamma * gamma)))
    E = (0.5 * Kp * phi, -0.5 * Kp * phi, -1j * Kz * phi / (gamma * gamma))
    zero = np.zeros_like(phi)
    B = op_curl(Kp, Kz, zero, zero, beta * phi / C_LIGHT)
    return E, B


# --------------------------------------------------------------------------
# Particles: cell keys and sort (PIC, particles per cell in AMPA)
# --------------------------------------------------------------------------
def cell_keys(g: Grid, x, y, z):
    """Integer cell key iz*Nr + ir with iz = floor(z/dz), ir = floor(r/dr), clamped.

    r = sqrt(x*x + y*y) evaluated as two rounded products and one rounded sum.
    """
    r = np.sqrt(x * x + y * y)
    iz = np.clip(np.floor(z / g.dz), 0, g.Nz - 1).astype(np.int64)
    ir = np.clip(np.floor(r / g.dr), 0, g.Nr - 1).astype(np.int64)
    return (iz * g.Nr + ir).astype(np.int32)


def sort_permutation(keys):
    """Stable counting-sort order: ascending key, ties by original index."""
    return np.argsort(keys, kind="stable").astype(np.int32)


# --------------------------------------------------------------------------
# Shape factors, deposit and gather (R-deposit, R-modes)
# --------------------------------------------------------------------------
def _polar(x, y):
    r = np.sqrt(x * x + y * y)
    safe = np.where(r > 0.0, r, 1.0)
    c = np.where(r > 0.0, x / safe, 1.0)
    s = np.where(r > 0.0, y / safe, 0.0)
    return r, c, s


def _weights(g: Grid, z, r):
    """Linear weights: z = (i+s) dz -> nodes i, i+1 (periodic); r = (j+1/2+t) dr -> nodes j, j+1."""
    u = z / g.dz
    fi = np.floor(u)
    s = u - fi
    i0 = np.mod(fi.astype(np.int64), g.Nz)
    i1 = np.mod(i0 + 1, g.Nz)
    v = r / g.dr - 0.5
    fj = np.floor(v)
    t = v - fj
    j0 = fj.astype(np.int64)
    return (i0, i1, 1.0 - s, s), (j0, j0 + 1, 1.0 - t, t)


def _scatter(g: Grid, zw, rw, val, vector_rt: bool, m: int):
    """Accumulate complex ``val`` with linear weights into an [Nr, Nz] grid with the axis fold."""
    i0, i1, wz0, wz1 = zw
    j0, j1, wr0, wr1 = rw
    fold = (-1.0) ** (m + 1) if vector_rt else (-1.0) ** m
    out = np.zeros(g.Nr * g.Nz, dtype=np.complex128)
    for (ii, wz) in ((i0, wz0), (i1, wz1)):
        for (jj, wr) in ((j0, wr0), (j1, wr1)):
            w = wz * wr
            jn = jj.copy()
            neg = jn < 0
            w = np.where(neg, w * fold, w)
            jn[neg] = -1 - jn[neg]          # node -1 -> node 0
            keep = jn < g.Nr                 # node >= Nr dropped
            idx = jn[keep] * g.Nz + ii[keep]
            contrib = (val * w)[keep]
            out += np.bincount(idx, weights=contrib.real, minlength=g.Nr * g.Nz)
            out += 1j * np.bincount(idx, weights=contrib.imag, minlength=g.Nr * g.Nz)
    return out.reshape(g.Nr, g.Nz)


def deposit_rho(g: Grid, x, y, z, w, q):
    """rho_m[i, j] = sum_p q w_p S_i S_j e^{+i m theta_p} / (2 pi r_j dr dz) (R-deposit)."""
    r, c, s = _polar(x, y)
    zw, rw = _weights(g, z, r)
    V = g.cell_volume()[:, None]
    e1 = c + 1j * s
    out = np.empty((g.Nm, g.Nr, g.Nz), dtype=np.complex128)
    ph = np.ones_like(e1)
    for m in range(g.Nm):
        out[m] = _scatter(g, zw, rw, q * w * ph, False, m) / V
        ph = ph * e1
    return out


def deposit_current(g: Grid, x, y, z, vx, vy, vz, w, q):
    """J_{r,theta,z;m} with the weights of ``deposit_rho`` times (v_r, v_theta, v_z) (R-deposit).

    v_r = (x v_x + y v_y)/r, v_theta = (x v_y - y v_x)/r (theta = 0 on the axis).
    """
    r, c, s = _polar(x, y)
    vr = c * vx + s * vy
    vt = c * vy - s * vx
    zw, rw = _weights(g, z, r)
    V = g.cell_volume()[:, None]
    e1 = c + 1j * s
    Jr = np.empty((g.Nm, g.Nr, g.Nz), dtype=np.complex128)
    Jt = np.empty_like(Jr)
    Jz = np.empty_like(Jr)
    ph = np.ones_like(e1)
    for m in range(g.Nm):
        base = q * w * ph
        Jr[m] = _scatter(g, zw, rw, base * vr, True, m) / V
        Jt[m] = _scatter(g, zw, rw, base * vt, True, m) / V
        Jz[m] = _scatter(g, zw, rw, base * vz, False, m) / V
        ph = ph * e1
    return Jr, Jt, Jz


def _interp(g: Grid, zw, rw, F, vector_rt: bool, m: int):
    i0, i1, wz0, wz1 = zw
    j0, j1, wr0, wr1 = rw
    fold = (-1.0) ** (m + 1) if vector_rt else (-1.0) ** m
    acc = np.zeros(len(i0), dtype=np.complex128)
    for (ii, wz) in ((i0, wz0), (i1, wz1)):
        for (jj, wr) in ((j0, wr0), (j1, wr1)):
            w = wz * wr
            neg = jj < 0
            jn = np.where(neg, -1 - jj, jj)
            w = np.where(neg, w * fold, w)
            keep = jn < g.Nr
            val = np.where(keep, F[np.minimum(jn, g.Nr - 1), ii], 0.0)
            acc += w * val
    return acc


def gather(g: Grid, E, B, x, y, z):
    """Fields at the particles (R-modes, R-deposit weights).

    E, B: tuples (r, theta, z) of real-space [Nm, Nr, Nz] complex grids.
    F = Re[F_0 + 2 sum_{m>=1} F_m e^{-i m theta}], then rotated to Cartesian:
    F_x = F_r cos - F_theta sin, F_y = F_r sin + F_theta cos.
    Returns (Ex, Ey, Ez, Bx, By, Bz).
    """
    r, c, s = _polar(x, y)
    zw, rw = _weights(g, z, r)
    e1 = c - 1j * s
    res = []
    for Fset in (E, B):
        comps = []
        for ci, F in enumerate(Fset):
            tot = np.zeros(len(x))
            ph = np.ones(len(x), dtype=np.complex128)
            for m in range(g.Nm):
                v = _interp(g, zw, rw, F[m], ci < 2, m)
                tot += (1.0 if m == 0 else 2.0) * (v * ph).real
                ph = ph * e1
            comps.append(tot)
        Fr, Ft, Fz = comps
        res += [Fr * c - Ft * s, Fr * s + Ft * c, Fz]
    return tuple(res)


def boris_push(ux, uy, uz, Ex, Ey, Ez, Bx, By, Bz, q, m, dt):
    """Relativistic Boris push of u = gamma v from n-1/2 to n+1/2 (R-push).

    u- = u + (q dt/2m) E; t = (q dt/(2 m gamma-)) B; u' = u- + u- x t;
    s = 2t/(1+|t|^2); u+ = u- + u' x s; u_new = u+ + (q dt/2m) E.
    """
    k = q * dt / (2.0 * m)
    umx, umy, umz = ux + k * Ex, uy + k * Ey, uz + k * Ez
    gm = np.sqrt(1.0 + (umx * umx + umy * umy + umz * umz) / (C_LIGHT * C_LIGHT))
    tx, ty, tz = k * Bx / gm, k * By / gm, k * Bz / gm
    upx = umx + (umy * tz - umz * ty)
    upy = umy + (umz * tx - umx * tz)
    upz = umz + (umx * ty - umy * tx)
    f = 2.0 / (1.0 + tx * tx + ty * ty + tz * tz)
    sx, sy, sz = f * tx, f * ty, f * tz
    ux2 = umx + (upy * sz - upz * sy) + k * Ex
    uy2 = umy + (upz * sx - upx * sz) + k * Ey
    uz2 = umz + (upx * sy - upy * sx) + k * Ez
    return ux2, uy2, uz2


def inv_gamma(ux, uy, uz):
    return 1.0 / np.sqrt(1.0 + (ux * ux + uy * uy + uz * uz) / (C_LIGHT * C_LIGHT))


def wrap_z(g: Grid, z):
    """Periodic z (R-grid): one wrap, particles move less than a box length per step."""
    z = np.where(z >= g.L, z - g.L, z)
    return np.where(z < 0.0, z + g.L, z)


def reflect_r(g: Grid, x, y, ux, uy):
    """Specular reflection at r >= R: r -> 2R - r, u_r -> -u_r (R-push)."""
    r = np.sqrt(x * x + y * y)
    out = r >= g.R
    if not np.any(out):
        return x, y, ux, uy
    rs = np.where(out, r, 1.0)
    cx, cy = x / rs, y / rs
    f = np.where(out, (2.0 * g.R - r) / rs, 1.0)
    ur = ux * cx + uy * cy
    ux2 = np.where(out, ux - 2.0 * ur * cx, ux)
    uy2 = np.where(out, uy - 2.0 * ur * cy, uy)
    return x * f, y * f, ux2, uy2


# --------------------------------------------------------------------------
# The PIC cycle
# --------------------------------------------------------------------------
@dataclass
class State:
    """Everything one PIC cycle reads and writes.

    Real-space fields E, B: tuples (r, theta, z) of [Nm, Nr, Nz] complex.
    Spectral fields Eh, Bh: tuples (+, -, z).  rho_prev_h: filtered rho^n.
    Particles: dict of float64 arrays x y z ux uy uz w and int32 id.
    rho_ion: real-space background added to every rho deposit.
    """

    g: Grid
    order_p: int
    filt: bool
    q: float
    m: float
    h: Hankel
    coef: dict
    T: np.ndarray
    E: tuple
    B: tuple
    Eh: tuple
    Bh: tuple
    rho_prev_h: np.ndarray
    rho_ion: np.ndarray
    p: dict


def make_state(g: Grid, order_p: int, filt: bool, particles: dict, n_neutral: int,
               beams=(), q: float = -Q_E, mass: float = M_E, h: Hankel | None = None) -> State:
    """Initial state (R-init).

    Ions: rho_ion = -rho of the first ``n_neutral`` particles (immobile background).
    Fields: zero, plus for each (id_lo, id_hi, gamma) in ``beams`` the space-charge
    field of the particles with id in [id_lo, id_hi).  rho^0 = rho(all) + rho_ion,
    transformed and filtered.
    """
    h = h if h is not None else hankel_setup(g)
    coef = psatd_coefficients(g, h, order_p)
    T = source_filter(g, h)
    P = {k: np.array(v, copy=True) for k, v in particles.items()}
    sel = P["id"] < n_neutral
    rho_ion = -deposit_rho(g, P["x"][sel], P["y"][sel], P["z"][sel], P["w"][sel], q)
    zero = np.zeros((g.Nm, g.Nr, g.Nz), dtype=np.complex128)
    Eh = [zero.copy(), zero.copy(), zero.copy()]
    Bh = [zero.copy(), zero.copy(), zero.copy()]
    for (lo, hi, gam) in beams:
        sel = (P["id"] >= lo) & (P["id"] < hi)
        rb = deposit_rho(g, P["x"][sel], P["y"][sel], P["z"][sel], P["w"][sel], q)
        rbh = forward_scalar(g, h, rb)
        if filt:
            rbh = rbh * T
        Eb, Bb = beam_fields(g, coef, rbh, gam)
        for i in range(3):
            Eh[i] = Eh[i] + Eb[i]
            Bh[i] = Bh[i] + Bb[i]
    rho0 = deposit_rho(g, P["x"], P["y"], P["z"], P["w"], q) + rho_ion
    rho0h = forward_scalar(g, h, rho0)
    if filt:
        rho0h = rho0h * T
    E = inverse_vector(g, h, *Eh)
    B = inverse_vector(g, h, *Bh)
    return State(g, order_p, filt, q, mass, h, coef, T, E, B, tuple(Eh), tuple(Bh),
                 rho0h, rho_ion, P)


def gather_push(st: State, window=None):
    """Gather E^n, B^n at x^n, push u^{n-1/2} -> u^{n+1/2}, move x^n -> x^{n+1/2} -> x^{n+1}.

    Returns the real-space current J^{n+1/2} deposited at x^{n+1/2} (R-deposit, R-push).
    Inactive particles (w = 0, R-window) keep their position and momentum.  With
    ``window = (back_z, shift)`` an active particle that ends behind the window's back
    edge is removed after its push and current deposit (``window_removed``, R-window).
    """
    g, P = st.g, st.p
    act = P["w"] != 0.0
    z0 = P["z"]
    F = gather(g, st.E, st.B, P["x"], P["y"], P["z"])
    ux, uy, uz = boris_push(P["ux"], P["uy"], P["uz"], *F, st.q, st.m, g.dt)
    ig = inv_gamma(ux, uy, uz)
    vx, vy, vz = ux * ig, uy * ig, uz * ig
    hdt = 0.5 * g.dt
    xh, yh, zh = P["x"] + hdt * vx, P["y"] + hdt * vy, wrap_z(g, P["z"] + hdt * vz)
    J = deposit_current(g, xh, yh, zh, vx, vy, vz, P["w"], st.q)
    x1, y1, z1 = xh + hdt * vx, yh + hdt * vy, wrap_z(g, zh + hdt * vz)
    x1, y1, ux, uy = reflect_r(g, x1, y1, ux, uy)
    new = {"x": x1, "y": y1, "z": z1, "ux": ux, "uy": uy, "uz": uz}
    for k, v in new.items():
        P[k] = np.where(act, v, P[k])
    if window is not None:
        back_z, shift = window
        gone = act & window_removed(g, z0, hdt * vz, back_z, shift)
        for k in ("w", "ux", "uy", "uz"):
            P[k] = np.where(gone, 0.0, P[k])
    return J


def sort_particles(st: State):
    """Stable sort of every particle array by cell key (a1)."""
    P = st.p
    perm = sort_permutation(cell_keys(st.g, P["x"], P["y"], P["z"]))
    for k in list(P.keys()):
        P[k] = P[k][perm]
    return perm


def field_step(st: State, rho_next, J):
    """Forward transforms, PSATD update, inverse transforms (a5..a9)."""
    g, h = st.g, st.h
    rho_h, Jp, Jm, Jz = forward_sources(g, h, rho_next, *J)
    E_new, B_new, rho_f, _ = psatd_update(g, st.coef, st.T, st.Eh, st.Bh, (Jp, Jm, Jz),
                                          rho_h, st.rho_prev_h, filt=st.filt, correct=True)
    st.Eh, st.Bh, st.rho_prev_h = E_new, B_new, rho_f
    st.E = inverse_vector(g, h, *E_new)
    st.B = inverse_vector(g, h, *B_new)


def pic_step(st: State, n_steps: int = 1):
    """n PIC cycles: gather+push (+J deposit), sort, rho deposit, field step."""
    for _ in range(n_steps):
        J = gather_push(st)
        sort_particles(st)
        P = st.p
        rho = deposit_rho(st.g, P["x"], P["y"], P["z"], P["w"], st.q) + st.rho_ion
        field_step(st, rho, J)
    return st


# --------------------------------------------------------------------------
# Guard-cell domain decomposition along z (FOPS: locality of the finite stencil,
# unit-pulse figure; Conclusion: about 60 guard cells at p = 32)
# --------------------------------------------------------------------------
def field_step_source_free(g: Grid, h: Hankel, order_p: int, E, B):
    """One source-free field step of real-space fields (a5..a9 with rho = J = 0).

    E, B: tuples (r, theta, z) of [Nm, Nr, Nz] complex grids.  Forward transform
    of E and B, the PSATD update of Eq. psatd-eqE/eqB with [k_z]_p and no sources,
    inverse transform.  Returns the new real-space (E, B).
    """
    coef = psatd_coefficients(g, h, order_p)
    T = source_filter(g, h)
    Eh = forward_vector(g, h, *E)
    Bh = forward_vector(g, h, *B)
    zero = np.zeros((g.Nm, g.Nr, g.Nz), dtype=np.complex128)
    E_new, B_new, _, _ = psatd_update(g, coef, T, Eh, Bh, (zero, zero, zero), zero, zero,
                                      filt=False, correct=False)
    return inverse_vector(g, h, *E_new), inverse_vector(g, h, *B_new)


def field_step_guarded(g: Grid, order_p: int, E, B, n_domains: int, guard: int):
    """The same source-free field step, advanced on n_domains equal z subdomains.

    Each subdomain d covers columns [d L, (d+1) L), L = Nz / n_domains; it is
    extended by ``guard`` columns of its neighbours on both sides (periodic z),
    advanced on its own grid of length L + 2 guard (its own DFT along z, so its own
    k_z and [k_z]_p; the same radial grid), and its interior columns are written back.
    With a finite-order stencil, whose real-space reach is finite, the interiors
    match the global step once ``guard`` covers that reach; with too few guard
    cells the periodic wrap of each local transform leaves spurious fields.
    """
    if n_domains < 1 or g.Nz % n_domains:
        raise ValueError("Nz must be a multiple of n_domains")
    L = g.Nz // n_domains
    gl = Grid(L + 2 * guard, g.Nr, g.Nm, g.dz, g.dr, g.dt)
    hl = hankel_setup(gl)
    E_out = tuple(np.empty_like(F) for F in E)
    B_out = tuple(np.empty_like(F) for F in B)
    for d in range(n_domains):
        cols = (np.arange(gl.Nz) + d * L - guard) % g.Nz
        El = tuple(F[:, :, cols] for F in E)
        Bl = tuple(F[:, :, cols] for F in B)
        En, Bn = field_step_source_free(gl, hl, order_p, El, Bl)
        for dst, src in zip(E_out + B_out, En + Bn):
            dst[:, :, d * L:(d + 1) * L] = src[:, :, guard:guard + L]
    return E_out, B_out


# --------------------------------------------------------------------------
# Moving window (R-window)
# --------------------------------------------------------------------------
# The paper follows the beams in co-moving coordinates zeta = z - c t (AMPA, Fig. ez:
# 35 mm of propagation) without stating the mechanics; R-window is the reading taken.
#   * The z grid is a ring: after k shifts the window's back column is k mod Nz and its
#     back edge lies at (k mod Nz) dz; arrays and particle positions never move.
#   * The window moves one cell at the end of every `period`-th cycle (period 1 when
#     c dt = dz, a window moving at c).
#   * Removal: in the push of every cycle, an active particle whose window coordinate
#     zeta = ((z^n - back) mod L) + (displacement of the step) - (dz if the window moves)
#     is negative has left through the back edge; its weight and momentum become 0
#     (inactive).  Its current of that step is still deposited.
#   * Injection: when the window moves, the departing column c becomes the front column;
#     the plasma loaded there at set-up (the template: ids of column c in increasing
#     order) is placed, at rest, into the inactive particles of smallest id.  A template
#     larger than the inactive pool is cut to the pool's size.
#   * Fields: after the field step of a moving cycle the departing column's E and B are
#     zeroed in real space and their transform is subtracted from the spectral state:
#     F^ <- F^ - forward(F 1_c), F <- F (1 - 1_c).  rho^ and the ion background stay.
#   * The ion background is fixed per array column; the template reloads each column's
#     initial plasma, so the fresh front is neutral.
@dataclass
class Window:
    """Moving-window state (R-window)."""

    period: int      # the window moves one cell every `period` cycles
    cycles: int      # cycles advanced since set-up
    shifts: int      # cells moved; the back column is shifts mod Nz
    tpl: dict        # x, y, z, w of the plasma at set-up, indexed by id (ids < n_plasma)
    col_ids: list    # per column, the template ids loaded there, increasing


def window_setup(st: State, n_plasma: int, period: int, n_reserve: int) -> Window:
    """Append ``n_reserve`` inactive particles (w = u = 0, ids np ..) and take the
    particles with id < n_plasma as the plasma template (R-window).  The ids held must be
    0 .. np-1.  Reserve particle k sits at the centre of cell (k mod Nz, (k div Nz) mod Nr)
    on the x axis: where an inactive particle sits changes no result, and spreading them
    keeps the cells of the sort small."""
    g, P = st.g, st.p
    n = P["x"].size
    if not np.array_equal(np.sort(P["id"]), np.arange(n)):
        raise ValueError("window: particle ids must be 0 .. np-1")
    if period < 1 or not 0 <= n_plasma <= n or n_reserve < 0:
        raise ValueError("window: bad period, n_plasma or n_reserve")
    k = np.arange(n_reserve)
    park = {"x": ((k // g.Nz) % g.Nr + 0.5) * g.dr, "z": (k % g.Nz + 0.5) * g.dz}
    for key in ("x", "y", "z", "ux", "uy", "uz", "w"):
        P[key] = np.concatenate([P[key], park.get(key, np.zeros(n_reserve))])
    P["id"] = np.concatenate([P["id"], np.arange(n, n + n_reserve, dtype=P["id"].dtype)])
    where = np.empty(n, dtype=np.int64)
    where[P["id"][:n]] = np.arange(n)
    at = where[:n_plasma]
    tpl = {k: P[k][at].copy() for k in ("x", "y", "z", "w")}
    col = np.clip(np.floor(tpl["z"] / g.dz).astype(np.int64), 0, g.Nz - 1)
    col_ids = [np.flatnonzero(col == c) for c in range(g.Nz)]
    return Window(period, 0, 0, tpl, col_ids)


def window_removed(g: Grid, z_old, half_move, back_z: float, shift: bool):
    """Particles whose window coordinate after this step is negative (R-window):
    zeta = ((z_old - back) mod L) + half_move + half_move - (dz if the window moves)."""
    zo = z_old - back_z
    zo = np.where(zo < 0.0, zo + g.L, zo)
    zn = (zo + half_move) + half_move - (g.dz if shift else 0.0)
    return zn < 0.0


def window_inject(st: State, win: Window, column: int) -> int:
    """Load the template of ``column`` into the inactive particles of smallest id, at rest
    (R-window).  Returns the number of template particles that found no slot."""
    P = st.p
    fresh = win.col_ids[column]
    free = np.sort(P["id"][P["w"] == 0.0])
    k = min(fresh.size, free.size)
    where = np.empty(P["id"].size, dtype=np.int64)
    where[P["id"]] = np.arange(P["id"].size)
    slots = where[free[:k]]
    for key in ("x", "y", "z", "w"):
        P[key][slots] = win.tpl[key][fresh[:k]]
    for key in ("ux", "uy", "uz"):
        P[key][slots] = 0.0
    return int(fresh.size - k)


def window_clear_column(st: State, column: int):
    """Remove the departing column's E and B: real space zeroed there, spectral state
    minus the forward transform of the column (R-window)."""
    g, h = st.g, st.h
    for name, hname in (("E", "Eh"), ("B", "Bh")):
        F = getattr(st, name)
        col = []
        for c in range(3):
            Fc = np.zeros_like(F[c])
            Fc[:, :, column] = F[c][:, :, column]
            col.append(Fc)
        D = forward_vector(g, h, *col)
        setattr(st, hname, tuple(getattr(st, hname)[c] - D[c] for c in range(3)))
        keep = []
        for c in range(3):
            Fn = F[c].copy()
            Fn[:, :, column] = 0.0
            keep.append(Fn)
        setattr(st, name, tuple(keep))


def pic_step_window(st: State, win: Window, n_steps: int = 1):
    """n PIC cycles in the moving window (R-window): push with removal, injection when the
    window moves, sort, rho deposit, field step, column removal.  Returns the number of
    template particles dropped for want of inactive slots."""
    g = st.g
    dropped = 0
    for _ in range(n_steps):
        shift = (win.cycles + 1) % win.period == 0
        column = win.shifts % g.Nz
        J = gather_push(st, window=(column * g.dz, shift))
        if shift:
            dropped += window_inject(st, win, column)
        sort_particles(st)
        P = st.p
        rho = deposit_rho(g, P["x"], P["y"], P["z"], P["w"], st.q) + st.rho_ion
        field_step(st, rho, J)
        if shift:
            window_clear_column(st, column)
            win.shifts += 1
        win.cycles += 1
    return dropped


def window_z(g: Grid, win: Window, z):
    """Window coordinate (z - back edge) mod L of array positions z (R-window)."""
    zw = z - (win.shifts % g.Nz) * g.dz
    return np.where(zw < 0.0, zw + g.L, zw)


# --------------------------------------------------------------------------
# Diagnostics (AMPA; R-diag)
# --------------------------------------------------------------------------
def beam_diagnostics(x, y, z, ux, uy, uz, w, slice_len: float = SLICE_LEN):
    """Beam quality of one beam (AMPA: emittance, slice energy spread).

    Normalised rms emittance (centred, weighted):
      eps_n,x = sqrt(<dx^2><dux^2> - <dx dux>^2)/c, same for y.
    Slice energy spread: slices of ``slice_len`` starting at zbar - 3 sigma_z,
    particles with 0 <= z - zbar + 3 sigma_z < 6 sigma_z, slice index
    floor((z - zbar + 3 sigma_z)/slice_len); per non-empty slice the weighted
    std of gamma; reported: the per-slice values and their mean.
    """
    W = w.sum()
    mean = lambda a: (w * a).sum() / W  # noqa: E731
    xm, ym, zm = mean(x), mean(y), mean(z)
    uxm, uym = mean(ux), mean(uy)
    dx, dy, dux, duy = x - xm, y - ym, ux - uxm, uy - uym
    ex = math.sqrt(max(mean(dx * dx) * mean(dux * dux) - mean(dx * dux) ** 2, 0.0)) / C_LIGHT
    ey = math.sqrt(max(mean(dy * dy) * mean(duy * duy) - mean(dy * duy) ** 2, 0.0)) / C_LIGHT
    sz = math.sqrt(mean((z - zm) ** 2))
    gam = np.sqrt(1.0 + (ux * ux + uy * uy + uz * uz) / (C_LIGHT * C_LIGHT))
    gm = mean(gam)
    d = z - zm + 3.0 * sz
    ns = int(math.ceil(6.0 * sz / slice_len)) if sz > 0 else 0
    inside = (d >= 0.0) & (d < 6.0 * sz)
    idx = np.floor(d[inside] / slice_len).astype(np.int64)
    idx = np.minimum(idx, max(ns - 1, 0))
    ww, gg = w[inside], gam[inside]
    sw = np.bincount(idx, weights=ww, minlength=ns)
    sg = np.bincount(idx, weights=ww * gg, minlength=ns)
    nonempty = sw > 0
    gbar = np.where(nonempty, sg / np.where(nonempty, sw, 1.0), 0.0)
    dg = gg - gbar[idx]
    sv = np.bincount(idx, weights=ww * dg * dg, minlength=ns)
    sig = np.where(nonempty, np.sqrt(sv / np.where(nonempty, sw, 1.0)), 0.0)
    return {
        "W": W, "x_mean": xm, "y_mean": ym, "z_mean": zm, "sigma_z": sz,
        "gamma_mean": gm, "emit_nx": ex, "emit_ny": ey,
        "slice_sigma_gamma": sig[nonempty], "slice_weight": sw[nonempty],
        "sigma_gamma_mean": float(sig[nonempty].mean()) if nonempty.any() else 0.0,
    }


def err_sigma_gamma(sig_f, sig_inf):
    """Err_sigma_gamma of AMPA Eq. err-metrics (rms of relative slice differences)."""
    sig_f, sig_inf = np.asarray(sig_f), np.asarray(sig_inf)
    return float(np.sqrt(np.mean(((sig_f - sig_inf) / sig_inf) ** 2)))


def err_emittance(eps_f, eps_inf):
    """Err_eps of AMPA Eq. err-metrics."""
    return (eps_f - eps_inf) / eps_inf


def field_on_plane(F_modes, theta=0.0):
    """F(r, z) at azimuth theta from mode grids F_m[r][z] (R-modes):
    Re[F_0 + 2 sum_{m>=1} F_m e^{-i m theta}]."""
    out = np.real(np.asarray(F_modes[0], dtype=np.complex128)).copy()
    for m in range(1, len(F_modes)):
        out = out + 2.0 * np.real(np.asarray(F_modes[m], dtype=np.complex128) * np.exp(-1j * m * theta))
    return out


def err_ez(ez_f, ez_inf):
    """Err_Ez of AMPA Eq. err-metrics: root mean square over all cells of the spatial
    (z, r) discrete Fourier transform of the relative difference of FFT_2(E_z)."""
    Ff = np.fft.fft2(np.asarray(ez_f, dtype=np.float64))
    Fi = np.fft.fft2(np.asarray(ez_inf, dtype=np.float64))
    return float(np.sqrt(np.mean(np.abs((Ff - Fi) / Fi) ** 2)))


def slice_sigma_gamma_on_grid(z, gamma, w, z_start, n_slices, slice_len: float = SLICE_LEN):
    """Per-slice weighted std of gamma on a given grid of n_slices slices of slice_len from
    z_start (AMPA: slices of 0.5 um; R-diag); NaN where a slice is empty.  Used to pair the
    slices of two runs on one grid (the reference run's) for Err_sigma_gamma."""
    out = np.full(n_slices, np.nan)
    members = [[] for _ in range(n_slices)]
    for zi, gi, wi in zip(z, gamma, w):
        k = math.floor((zi - z_start) / slice_len)
        if 0 <= k < n_slices:
            members[k].append((wi, gi))
    for k, mem in enumerate(members):
        if not mem:
            continue
        ws = sum(a for a, _ in mem)
        gm = sum(a * b for a, b in mem) / ws
        out[k] = math.sqrt(sum(a * (b - gm) ** 2 for a, b in mem) / ws)
    return out


def ncr_resonance_kperp(kz, dz: float, order_p: int, beta: float):
    """k_perp of the modes that numerical Cherenkov radiation excites for a beam at beta c
    (NCR, Eq. resonance_k rearranged): beta^2 k_z^2 = k_perp^2 + [k_z]_p^2, so
    k_perp = sqrt(beta^2 k_z^2 - [k_z]_p^2) where that is real, NaN elsewhere."""
    kz = np.asarray(kz, dtype=np.float64)
    d = beta * beta * kz * kz - modified_kz(kz, dz, order_p) ** 2
    return np.where(d > 0.0, np.sqrt(np.maximum(d, 0.0)), np.nan)
