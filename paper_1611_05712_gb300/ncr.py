"""Beam-quality and field errors of a finite-order run against an infinite-order run
(section "Accurate modeling of plasma accelerators in finite order PSATD", Eq. err-metrics),
and the spectral signature of numerical Cherenkov radiation (section "Numerical Cherenkov
radiation", Eq. resonance and Eq. resonance_k), the measures of the paper's order study.

Host-side post-processing of arrays read back from the library; nothing here is part of
the PIC cycle.
  Err_sigma_gamma = sqrt(mean_i ((s_f,i - s_inf,i) / s_inf,i)^2) over the witness beam's
                    slices of 0.5 um within +-3 sigma_z: both runs are sliced on one grid,
                    the infinite-order run's (its mean z - 3 sigma_z onwards), so that slice
                    i is the same interval of z in both;
  Err_eps         = (eps_f - eps_inf) / eps_inf;
  Err_Ez          = sqrt(mean over the (z, r) cells of |(F_f - F_inf) / F_inf|^2) with
                    F = 2-D discrete Fourier transform of E_z on the theta = 0 plane.
Err_Ez as printed divides cell by cell, so Fourier cells where F_inf nearly vanishes
dominate it; err_ez_l2 is the normalised L2 reading, ||F_f - F_inf|| / ||F_inf||.

Spectral map: for mode 0 the quasi-cylindrical spectral state is the spatial Fourier
transform of an axisymmetric field (the order-0 Hankel transform is the transverse 2-D
Fourier transform of a radially symmetric function, with k_perp = |(k_x, k_y)|), so
|E_z^|(k_perp, k_z) of mode 0, read from the library's spectral fields, is the map of the
paper's Fourier-space figure.  Numerical Cherenkov radiation appears where the modified
dispersion relation omega = c sqrt(k_perp^2 + [k_z]^2) meets the beam mode omega = v k_z
(Eq. resonance_k): k_perp = sqrt(beta^2 k_z^2 - [k_z]^2), which exists only where
[k_z] < beta |k_z|, i.e. never at infinite order for beta < 1.
"""
from __future__ import annotations

import math

import numpy as np

SLICE_LEN = 0.5e-6


def ez_plane(E: np.ndarray) -> np.ndarray:
    """E_z(r, z) at theta = 0 from the mode grids E[comp][m][r][z] (comp 2 = z):
    Re[E_z,0 + 2 sum_{m>=1} E_z,m]."""
    ez = np.array(E[2, 0].real, dtype=np.float64)
    for m in range(1, E.shape[1]):
        ez += 2.0 * E[2, m].real
    return ez


def ez_spectral_map(Eh: np.ndarray, m: int = 0) -> np.ndarray:
    """|E_z^|[n, k_z] of mode m from the spectral fields Eh[comp][m][n][k_z] (comp 2 = z)."""
    return np.abs(np.asarray(Eh)[2, m])


def resonance_kperp(kz: np.ndarray, kz_mod: np.ndarray, beta: float) -> np.ndarray:
    """k_perp on Eq. resonance_k for each k_z: sqrt(beta^2 k_z^2 - [k_z]^2) where the root is
    real, NaN where the modified dispersion relation does not meet the beam mode."""
    d = (beta * np.asarray(kz, dtype=np.float64)) ** 2 - np.asarray(kz_mod, dtype=np.float64) ** 2
    out = np.full(d.shape, np.nan)
    ok = d > 0.0
    out[ok] = np.sqrt(d[ok])
    return out


def slice_grid(z, w, slice_len: float = SLICE_LEN):
    """(z_start, n_slices) of a beam: slices of slice_len from zbar - 3 sigma_z, covering
    +-3 sigma_z (weighted mean and rms)."""
    z = np.asarray(z, dtype=np.float64)
    w = np.asarray(w, dtype=np.float64)
    W = w.sum()
    zbar = float((w * z).sum() / W)
    sz = float(np.sqrt((w * (z - zbar) ** 2).sum() / W))
    return zbar - 3.0 * sz, int(math.ceil(6.0 * sz / slice_len)) if sz > 0 else 0


def slice_sigma_gamma(z, gamma, w, z_start: float, n_slices: int, slice_len: float = SLICE_LEN) -> np.ndarray:
    """Weighted standard deviation of gamma in the slices [z_start + i L, z_start + (i+1) L),
    i < n_slices; NaN for empty slices."""
    z, gamma, w = (np.asarray(a, dtype=np.float64) for a in (z, gamma, w))
    idx = np.floor((z - z_start) / slice_len)
    keep = (idx >= 0) & (idx < n_slices)
    idx = idx[keep].astype(np.int64)
    ww, gg = w[keep], gamma[keep]
    W = np.bincount(idx, weights=ww, minlength=n_slices)
    G1 = np.bincount(idx, weights=ww * gg, minlength=n_slices)
    out = np.full(n_slices, np.nan)
    ok = W > 0
    mean = np.zeros(n_slices)
    mean[ok] = G1[ok] / W[ok]
    G2 = np.bincount(idx, weights=ww * (gg - mean[idx]) ** 2, minlength=n_slices)
    out[ok] = np.sqrt(G2[ok] / W[ok])
    return out


def err_sigma_gamma(slices_f, slices_inf) -> float:
    """Eq. err-metrics over slices already paired (same grid): slices empty in either run,
    or with zero spread in the reference, are left out."""
    a = np.asarray(slices_f, dtype=np.float64)
    b = np.asarray(slices_inf, dtype=np.float64)
    if a.shape != b.shape:
        raise ValueError(f"slice arrays differ in length ({a.size} vs {b.size}): slice both runs on one grid")
    ok = np.isfinite(a) & np.isfinite(b) & (b > 0)
    if not ok.any():
        return float("nan")
    return float(np.sqrt(np.mean(((a[ok] - b[ok]) / b[ok]) ** 2)))


def err_sigma_gamma_runs(beam_f: dict, beam_inf: dict, slice_len: float = SLICE_LEN) -> float:
    """Err_sigma_gamma of two runs' beams (dicts of float64 z, gamma, w), both sliced on the
    infinite-order run's grid."""
    z0, n = slice_grid(beam_inf["z"], beam_inf["w"], slice_len)
    return err_sigma_gamma(slice_sigma_gamma(beam_f["z"], beam_f["gamma"], beam_f["w"], z0, n, slice_len),
                           slice_sigma_gamma(beam_inf["z"], beam_inf["gamma"], beam_inf["w"], z0, n, slice_len))


def beam_of(particles: dict, id_lo: int, id_hi: int, c_light: float = 299792458.0) -> dict:
    """z, gamma, w of the particles with id in [id_lo, id_hi) from a float64 particle set."""
    sel = (particles["id"] >= id_lo) & (particles["id"] < id_hi)
    ux, uy, uz = (np.asarray(particles[k], dtype=np.float64)[sel] for k in ("ux", "uy", "uz"))
    return {"z": np.asarray(particles["z"], dtype=np.float64)[sel],
            "gamma": np.sqrt(1.0 + (ux * ux + uy * uy + uz * uz) / (c_light * c_light)),
            "w": np.asarray(particles["w"], dtype=np.float64)[sel]}


def err_emittance(eps_f: float, eps_inf: float) -> float:
    return float((eps_f - eps_inf) / eps_inf)


def err_ez(ez_f: np.ndarray, ez_inf: np.ndarray) -> float:
    ff, fi = np.fft.fft2(ez_f), np.fft.fft2(ez_inf)
    return float(np.sqrt(np.mean(np.abs((ff - fi) / fi) ** 2)))


def err_ez_l2(ez_f: np.ndarray, ez_inf: np.ndarray) -> float:
    ff, fi = np.fft.fft2(ez_f), np.fft.fft2(ez_inf)
    return float(np.linalg.norm(ff - fi) / np.linalg.norm(fi))
