"""Numerical Cherenkov radiation and the order study on the GPU (section "Numerical Cherenkov
radiation": Eq. resonance_k and the Fourier-space figure of E_z; section "Accurate modeling
of plasma accelerators in finite order PSATD": Eq. err-metrics).

The plasma + relativistic beam case (256 x 64, 2 modes, gamma = 1000) advanced 200 cycles
in the FP64 form at several stencil orders from one initial state:
  * the spectral amplitude that order 4 adds to E_z of mode 0 (read from the library's
    spectral fields, which the library's own FFT and Hankel kernels produce) peaks on the
    resonance curve k_perp = sqrt(beta^2 k_z^2 - [k_z]_4^2), with [k_z] and k_perp from the
    library's tables; the infinite-order run carries almost nothing there;
  * Err_eps, Err_sigma_gamma (both runs sliced on one grid) and Err_Ez of orders 4 and 16
    against infinite order equal the oracle's values from the same runs on the host, and
    fall with the order.
"""
import numpy as np
import pytest

from oracle import psatd_rz as O
from paper_1611_05712_gb300 import binding as bd
from paper_1611_05712_gb300 import ncr
from paper_1611_05712_gb300 import workloads as W

pytestmark = pytest.mark.gpu

CYCLES = 200


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1611_05712_gb300.build import build
    build()


@pytest.fixture(scope="module")
def gpu_runs():
    w = W.plasma_beam_small()
    P, npl, beams = W.particles(w)
    lo, hi = beams[0][0], beams[0][1]
    out = {}
    for p in (0, 4, 16):
        s = bd.Sim.from_workload(w, P, npl, beams, order_p=p)
        s.step(CYCLES)
        out[p] = {"diag": s.diagnostics(lo, hi), "E": s.get("E"), "EH": s.get("EH"),
                  "kperp": s.get("KPERP"), "kz_mod": s.get("KZ_MOD"), "particles": s.read_particles()}
        s.close()
    return w, P, npl, beams, out


def test_ncr_peaks_lie_on_the_resonance_curve(gpu_runs):
    w, _, _, beams, runs = gpu_runs
    beta = np.sqrt(1.0 - 1.0 / beams[0][2] ** 2)
    kz = 2.0 * np.pi * np.fft.fftfreq(w.Nz, d=w.dz)
    m4, m0 = ncr.ez_spectral_map(runs[4]["EH"]), ncr.ez_spectral_map(runs[0]["EH"])
    kres = ncr.resonance_kperp(kz, runs[4]["kz_mod"], beta)
    assert not np.isfinite(ncr.resonance_kperp(kz, runs[0]["kz_mod"], beta)).any()   # none at p = inf
    kperp = runs[4]["kperp"][0]
    excess = m4 - m0
    top = np.argsort(excess.ravel())[::-1][:10]
    dk = np.pi / (w.Nr * w.dr)
    for k in top:
        n, f = divmod(int(k), w.Nz)
        assert np.isfinite(kres[f]), (n, f)
        assert abs(kperp[n] - kres[f]) < 1.5 * dk, (n, f, kperp[n], kres[f])
        assert m0[n, f] < 0.1 * m4[n, f]
    assert excess.ravel()[top[0]] > 0.01 * m0.max()


def test_order_sweep_errors_match_the_oracle(gpu_runs):
    w, P, npl, beams, runs = gpu_runs
    lo, hi = beams[0][0], beams[0][1]
    g = O.Grid(w.Nz, w.Nr, w.Nm, w.dz, w.dr, w.dt)
    h = O.hankel_setup(g)
    ref = {}
    for p in (0, 4, 16):
        st = O.make_state(g, p, True, P, npl, beams, h=h)
        O.pic_step(st, CYCLES)
        Q = st.p
        sel = (Q["id"] >= lo) & (Q["id"] < hi)
        gam = np.sqrt(1.0 + (Q["ux"] ** 2 + Q["uy"] ** 2 + Q["uz"] ** 2) / O.C_LIGHT ** 2)
        d = O.beam_diagnostics(Q["x"][sel], Q["y"][sel], Q["z"][sel], Q["ux"][sel], Q["uy"][sel],
                               Q["uz"][sel], Q["w"][sel])
        ref[p] = {"emit": d["emit_nx"], "ez": O.field_on_plane(list(st.E[2])),
                  "z": Q["z"][sel], "gamma": gam[sel], "w": Q["w"][sel]}
    z0, ns = ncr.slice_grid(ref[0]["z"], ref[0]["w"])
    s_inf = O.slice_sigma_gamma_on_grid(ref[0]["z"], ref[0]["gamma"], ref[0]["w"], z0, ns)
    errs = {}
    for p in (4, 16):
        gb, gi = ncr.beam_of(runs[p]["particles"], lo, hi), ncr.beam_of(runs[0]["particles"], lo, hi)
        got = {"eps": ncr.err_emittance(runs[p]["diag"]["emit_nx"], runs[0]["diag"]["emit_nx"]),
               "sg": ncr.err_sigma_gamma_runs(gb, gi),
               "ez": ncr.err_ez(ncr.ez_plane(runs[p]["E"]), ncr.ez_plane(runs[0]["E"])),
               "ez_l2": ncr.err_ez_l2(ncr.ez_plane(runs[p]["E"]), ncr.ez_plane(runs[0]["E"]))}
        s_f = O.slice_sigma_gamma_on_grid(ref[p]["z"], ref[p]["gamma"], ref[p]["w"], z0, ns)
        ok = ~np.isnan(s_f) & ~np.isnan(s_inf) & (s_inf > 0)
        want = {"eps": O.err_emittance(ref[p]["emit"], ref[0]["emit"]),
                "sg": O.err_sigma_gamma(s_f[ok], s_inf[ok]),
                "ez": O.err_ez(ref[p]["ez"], ref[0]["ez"]),
                "ez_l2": float(np.linalg.norm(np.fft.fft2(ref[p]["ez"]) - np.fft.fft2(ref[0]["ez"]))
                               / np.linalg.norm(np.fft.fft2(ref[0]["ez"])))}
        # Err_Ez as printed is the rms over Fourier cells of |dF / F_inf|, so the cells where
        # F_inf nearly vanishes (its value there is rounding noise of the infinite-order run)
        # dominate it, and two FP64 runs that differ only in rounding order (atomic order,
        # fused multiply-adds) give values a few 1e-3 apart while the other measures agree
        # to 1e-9: 1e-2 there, 1e-6 for the other measures
        for k in got:
            assert got[k] == pytest.approx(want[k], rel=1e-2 if k == "ez" else 1e-6), (p, k, got[k], want[k])
        errs[p] = got
    # the measures fall as the order grows (the paper's order study)
    assert errs[4]["ez_l2"] > errs[16]["ez_l2"]
    assert errs[4]["sg"] > errs[16]["sg"]
