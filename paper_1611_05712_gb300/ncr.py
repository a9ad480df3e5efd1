"""Beam-quality and field errors of a finite-order run against an infinite-order run
(section "Accurate modeling of plasma accelerators in finite order PSATD", Eq. err-metrics),
the measures of numerical Cherenkov radiation (NCR) used in the paper's order study.

Host-side post-processing of arrays read back from the library; nothing here is part of
the PIC cycle.
  Err_sigma_gamma = sqrt(mean_i ((s_f,i - s_inf,i) / s_inf,i)^2) over the beam's slices;
  Err_eps         = (eps_f - eps_inf) / eps_inf;
  Err_Ez          = sqrt(mean over the (z, r) cells of |(F_f - F_inf) / F_inf|^2) with
                    F = 2-D discrete Fourier transform of E_z on the theta = 0 plane.
Err_Ez as printed divides cell by cell, so Fourier cells where F_inf nearly vanishes
dominate it; err_ez_l2 is the normalised L2 reading, ||F_f - F_inf|| / ||F_inf||.
"""
from __future__ import annotations

import numpy as np


def ez_plane(E: np.ndarray) -> np.ndarray:
    """E_z(r, z) at theta = 0 from the mode grids E[comp][m][r][z] (comp 2 = z):
    Re[E_z,0 + 2 sum_{m>=1} E_z,m]."""
    ez = np.array(E[2, 0].real, dtype=np.float64)
    for m in range(1, E.shape[1]):
        ez += 2.0 * E[2, m].real
    return ez


def err_sigma_gamma(slices_f, slices_inf) -> float:
    a = np.asarray(slices_f, dtype=np.float64)
    b = np.asarray(slices_inf, dtype=np.float64)
    n = min(a.size, b.size)
    a, b = a[:n], b[:n]
    return float(np.sqrt(np.mean(((a - b) / b) ** 2)))


def err_emittance(eps_f: float, eps_inf: float) -> float:
    return float((eps_f - eps_inf) / eps_inf)


def err_ez(ez_f: np.ndarray, ez_inf: np.ndarray) -> float:
    ff, fi = np.fft.fft2(ez_f), np.fft.fft2(ez_inf)
    return float(np.sqrt(np.mean(np.abs((ff - fi) / fi) ** 2)))


def err_ez_l2(ez_f: np.ndarray, ez_inf: np.ndarray) -> float:
    ff, fi = np.fft.fft2(ez_f), np.fft.fft2(ez_inf)
    return float(np.linalg.norm(ff - fi) / np.linalg.norm(fi))
