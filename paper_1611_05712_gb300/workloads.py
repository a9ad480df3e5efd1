"""Seeded synthetic workloads: grids, plasma and Gaussian electron beams.

This module holds no arithmetic of the PIC method itself.  It only places
macroparticles (positions, momenta u = gamma*v, weights = physical electrons per
macroparticle) from a seeded numpy ``Philox`` generator, so that the CUDA path
and the CPU oracle start from identical arrays.  The workloads stand in for the
paper's beam-driven plasma-wakefield setup (section "Accurate modeling of
plasma accelerators in finite order PSATD": 1e17 cm^-3 plasma, 180 pC drive
beam of 8.4 um x 5 um, 50 pC witness beam, particles per cell laid out in
(z, r, theta), two azimuthal modes); the paper's own input scripts are not
available, so the sizes below are stated readings.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

C_LIGHT = 299792458.0
Q_E = 1.602176634e-19


@dataclass
class Beam:
    n: int                 # macroparticles
    gamma: float           # mean Lorentz factor
    charge: float          # total charge magnitude [C]
    sigma_z: float         # rms length [m]
    sigma_r: float         # rms width per transverse axis [m]
    z_center: float        # [m]
    rel_energy_spread: float = 0.0


@dataclass
class Workload:
    name: str
    Nz: int
    Nr: int
    Nm: int
    dz: float
    dr: float
    dt: float
    order_p: int                      # 0 = infinite order
    plasma_density: float             # electrons per m^3
    ppc: tuple                        # macroparticles per cell in (z, r, theta)
    beams: list = field(default_factory=list)
    steps: int = 1
    seed: int = 0

    @property
    def L(self):
        return self.Nz * self.dz

    @property
    def R(self):
        return self.Nr * self.dr


def _cfg(name, Nz, Nr, Nm, order_p, density_cm3, ppc, beams, steps, seed, cdt_over_dz=1.0,
         dz=0.05e-6, dr=0.05e-6):
    return Workload(name, Nz, Nr, Nm, dz, dr, cdt_over_dz * dz / C_LIGHT, order_p,
                    density_cm3 * 1e6, ppc, beams, steps, seed)


def plasma_beam_small(order_p: int = 0, seed: int = 1) -> Workload:
    """256 x 64 grid, 2 modes, 1e18 cm^-3 plasma at 1 macroparticle per cell plus a
    20k-particle gamma=1000 beam (sigma_z 1 um, sigma_r 0.5 um, 0.1 % energy spread);
    beam charge 6.3 pC puts its peak density near 1e19 cm^-3."""
    beam = Beam(20000, 1000.0, 6.3e-12, 1.0e-6, 0.5e-6, 6.4e-6, 1e-3)
    return _cfg("plasma_beam_256x64_m2", 256, 64, 2, order_p, 1e18, (1, 1, 1), [beam], 100, seed)


def wake_2048x256(order_p: int = 32, seed: int = 2) -> Workload:
    """2048 x 256 grid, 2 modes, 1e17 cm^-3 plasma at 2 macroparticles per cell
    (1 z x 1 r x 2 theta); 200k-particle 180 pC gamma=2000 drive beam
    (sigma_z 8.4 um, sigma_r 5 um) and a 100k-particle 50 pC gamma=400 witness
    beam (sigma_z 2 um, sigma_r 0.3 um)."""
    drive = Beam(200000, 2000.0, 180e-12, 8.4e-6, 5.0e-6, 80e-6, 0.0)
    witness = Beam(100000, 400.0, 50e-12, 2.0e-6, 0.3e-6, 30e-6, 0.0)
    return _cfg("wake_2048x256_m2", 2048, 256, 2, order_p, 1e17, (1, 1, 2), [drive, witness],
                2000, seed)


def large_8192x1024(order_p: int = 32, seed: int = 5, ppc=(2, 2, 3)) -> Workload:
    """8192 x 1024 grid, 3 modes, order 32, 1e17 cm^-3 plasma at 12 macroparticles
    per cell (~100M) plus 1M-particle drive and witness beams."""
    drive = Beam(1000000, 2000.0, 180e-12, 8.4e-6, 5.0e-6, 300e-6, 0.0)
    witness = Beam(1000000, 400.0, 50e-12, 2.0e-6, 0.3e-6, 250e-6, 0.0)
    return _cfg("large_8192x1024_m3", 8192, 1024, 3, order_p, 1e17, ppc, [drive, witness],
                5000, seed)


def large_crop_1024x128(order_p: int = 32, seed: int = 6) -> Workload:
    """A crop of the large run that the oracle finishes in seconds: 1024 x 128 grid, 3 modes,
    order 32, 1e17 cm^-3 plasma at 12 macroparticles per cell (2 z x 2 r x 3 theta), and
    drive and witness beams scaled into the 51.2 um x 6.4 um box (15,625 macroparticles each,
    1/64 of the large run's, the charge per macroparticle of the large run)."""
    drive = Beam(15625, 2000.0, 180e-12 / 64, 2.0e-6, 1.0e-6, 38e-6, 0.0)
    witness = Beam(15625, 400.0, 50e-12 / 64, 0.5e-6, 0.3e-6, 20e-6, 0.0)
    return _cfg("large_crop_1024x128_m3", 1024, 128, 3, order_p, 1e17, (2, 2, 3), [drive, witness], 1, seed)


def tiny(order_p: int = 0, seed: int = 3, Nz=16, Nr=8, Nm=2, n_beam=64) -> Workload:
    """A grid the oracle finishes instantly, for brute-force and stage tests."""
    beam = Beam(n_beam, 50.0, 1e-15, 2 * 0.05e-6, 2 * 0.05e-6, Nz * 0.05e-6 / 2, 1e-2)
    return _cfg(f"tiny_{Nz}x{Nr}_m{Nm}", Nz, Nr, Nm, order_p, 1e18, (1, 1, 1), [beam], 2, seed)


def scan_member(s: int, base_seed: int = 4000) -> Workload:
    """One simulation of the order/resolution scan: Nz from the 7-smooth integers in
    [512, 4096], Nr a multiple of 16 in [64, 512], Nm in {1,2,3},
    p in {8,16,24,32,48,64,inf}, c dt/dz in {0.5, 1.0}."""
    rng = np.random.Generator(np.random.Philox(base_seed + s))
    smooth = [n for n in range(512, 4097) if _is_7_smooth(n)]
    Nz = int(rng.choice(smooth))
    Nr = int(rng.choice(np.arange(64, 513, 16)))
    Nm = int(rng.choice([1, 2, 3]))
    p = int(rng.choice([8, 16, 24, 32, 48, 64, 0]))
    cf = float(rng.choice([0.5, 1.0]))
    L = Nz * 0.05e-6
    beam = Beam(20000, 1000.0, 6.3e-12, 1.0e-6, 0.5e-6, L / 2, 1e-3)
    return _cfg(f"scan_{s}", Nz, Nr, Nm, p, 1e18, (1, 1, 1), [beam], 100, base_seed + s,
                cdt_over_dz=cf)


def _is_7_smooth(n):
    for f in (2, 3, 5, 7):
        while n % f == 0:
            n //= f
    return n == 1


# --------------------------------------------------------------------------
def _plasma(w: Workload, rng):
    nz, nr, nth = w.ppc
    iz = (np.arange(w.Nz * nz) + 0.5) / nz
    jr = (np.arange(w.Nr * nr) + 0.5) / nr
    Z, Rr = np.meshgrid(iz * w.dz, jr * w.dr, indexing="ij")
    Z, Rr = Z.ravel(), Rr.ravel()
    th0 = rng.uniform(0.0, 2.0 * math.pi, size=Z.size)
    th = (th0[:, None] + 2.0 * math.pi * np.arange(nth)[None, :] / nth).ravel()
    Z = np.repeat(Z, nth)
    Rr = np.repeat(Rr, nth)
    # physical electrons in the ring element represented by one macroparticle
    wt = w.plasma_density * 2.0 * math.pi * Rr * (w.dr / nr) * (w.dz / nz) / nth
    n = Z.size
    zero = np.zeros(n)
    return dict(x=Rr * np.cos(th), y=Rr * np.sin(th), z=Z, ux=zero.copy(), uy=zero.copy(),
                uz=zero.copy(), w=wt)


def _beam(w: Workload, b: Beam, rng):
    n = b.n
    x = rng.normal(0.0, b.sigma_r, n)
    y = rng.normal(0.0, b.sigma_r, n)
    z = rng.normal(b.z_center, b.sigma_z, n)
    # keep the beam inside the box: redraw what falls outside r < 0.95 R, 0 <= z < L
    for _ in range(100):
        bad = (x * x + y * y >= (0.95 * w.R) ** 2) | (z < 0) | (z >= w.L)
        if not bad.any():
            break
        k = int(bad.sum())
        x[bad] = rng.normal(0.0, b.sigma_r, k)
        y[bad] = rng.normal(0.0, b.sigma_r, k)
        z[bad] = rng.normal(b.z_center, b.sigma_z, k)
    gam = b.gamma * (1.0 + b.rel_energy_spread * rng.normal(0.0, 1.0, n))
    uz = C_LIGHT * np.sqrt(gam * gam - 1.0)
    zero = np.zeros(n)
    wt = np.full(n, b.charge / Q_E / n)
    return dict(x=x, y=y, z=z, ux=zero.copy(), uy=zero.copy(), uz=uz, w=wt)


KEYS = ("x", "y", "z", "ux", "uy", "uz", "w")


def particles(w: Workload, with_plasma: bool = True):
    """All macroparticles of a workload as float64 SoA plus int32 ids.

    Returns (dict of arrays, n_plasma, beams) where beams is a list of
    (id_lo, id_hi, gamma).  Plasma particles come first (ids 0..n_plasma-1).
    """
    rng = np.random.Generator(np.random.Philox(w.seed))
    parts = []
    if with_plasma and w.plasma_density > 0:
        parts.append(_plasma(w, rng))
    n_plasma = parts[0]["x"].size if parts else 0
    beams = []
    lo = n_plasma
    for b in w.beams:
        parts.append(_beam(w, b, rng))
        beams.append((lo, lo + b.n, b.gamma))
        lo += b.n
    out = {k: np.ascontiguousarray(np.concatenate([p[k] for p in parts])) for k in KEYS}
    out["id"] = np.arange(out["x"].size, dtype=np.int32)
    return out, n_plasma, beams
