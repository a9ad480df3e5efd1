"""GPU checks of the mixed form at the benchmarked full sizes, in the bench's launch
configuration (autotuned tiles).

* 2048 x 256, 2 modes, p = 32, 1.35M particles: one cycle against the FP64 oracle run on
  the same initial state (per-field and per-particle-array tolerances of the mixed form).
* 8192 x 1024, 3 modes, p = 32, 102.7M particles: what the oracle cannot run whole is
  checked by sampled outputs and by properties that hold at any size: the FP64 setup
  tables against the oracle's (Bessel zeros and pseudo-inverses), the cell sort as a
  stable sort of its keys, total charge, and Gauss's law div E = rho/eps0 in spectral
  space after a cycle (the corrected PSATD update keeps it, section "Finite order
  pseudo-spectral solvers"; the initial fields satisfy it by construction, R-init).
"""
import numpy as np
import pytest

from oracle import psatd_rz as O
from paper_1611_05712_gb300 import binding as bd
from paper_1611_05712_gb300 import workloads as W
from gpu_helpers import by_id, rel_err

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1611_05712_gb300.build import build
    build()


def test_mixed_full_cycle_wake_2048x256():
    w = W.wake_2048x256(order_p=32)
    P, npl, beams = W.particles(w)
    g = O.Grid(w.Nz, w.Nr, w.Nm, w.dz, w.dr, w.dt)
    s = bd.Sim.from_workload(w, P, npl, beams, precision=bd.PIC_MIXED_TF32X3)
    s.autotune()
    # the oracle starts from the particle state the float form holds
    Pf = s.read_particles()
    st = O.make_state(g, w.order_p, True, Pf, npl, beams)
    s.step(1)
    O.pic_step(st, 1)
    for name, ref in (("E", st.E), ("B", st.B), ("EH", st.Eh), ("BH", st.Bh)):
        assert rel_err(s.get(name), np.stack(ref)) < 1e-4, name
    got, ref = by_id(s.read_particles()), by_id(st.p)
    assert np.array_equal(got["id"], ref["id"])
    for k in ("x", "y", "z"):
        assert rel_err(got[k], ref[k]) < 1e-5, k
    for k in ("ux", "uy", "uz"):
        assert rel_err(got[k], ref[k]) < 1e-4, k


@pytest.fixture(scope="module")
def large():
    w = W.large_8192x1024(order_p=32)
    P, npl, beams = W.particles(w)
    s = bd.Sim.from_workload(w, P, npl, beams, precision=bd.PIC_MIXED_TF32X3)
    s.autotune()
    q_beams = -O.Q_E * float(P["w"][npl:].sum())
    n = len(P["x"])
    del P
    return w, s, npl, q_beams, n


def test_large_setup_tables_match_oracle(large):
    w, s, _, _, _ = large
    g = O.Grid(w.Nz, w.Nr, w.Nm, w.dz, w.dr, w.dt)
    h = O.hankel_setup(g)
    assert rel_err(s.get("KPERP"), np.stack(h.kperp)) < 1e-14
    assert rel_err(s.get("KZ_MOD"), O.modified_kz(g.kz, g.dz, w.order_p)) < 1e-13
    binv, mf = s.get("HANKEL_INV"), s.get("HANKEL_FWD")
    for m in range(w.Nm):
        for sl in range(3):
            assert np.abs(binv[m, sl] - h.Binv[m][sl]).max() < 1e-13
            assert rel_err(mf[m, sl], h.M[m][sl]) < 1e-12, (m, sl)


def test_large_cycle_properties(large):
    w, s, npl, q_beams, n = large
    s.step(1)
    s.sync()
    # the cell sort of this cycle: a permutation that orders the keys stably
    keys, perm = s.get("KEYS")[:n], s.get("PERM")[:n]
    assert np.array_equal(np.bincount(perm, minlength=n), np.ones(n, dtype=np.int64))
    ks = keys[perm]
    assert np.all(np.diff(ks) >= 0)
    same = np.diff(ks) == 0
    assert np.all(np.diff(perm)[same] > 0)
    # total charge: ions cancel the plasma, what remains is the beams' charge (the plasma's
    # share on the dropped node r = R changes as it moves: -3.9e-6 of the beams' charge
    # after one cycle)
    dep = s.get("DEP")
    g = O.Grid(w.Nz, w.Nr, w.Nm, w.dz, w.dr, w.dt)
    V = g.cell_volume()[:, None]
    q = float((dep[0, 0].astype(np.complex128) * V).sum().real)
    assert q == pytest.approx(q_beams, rel=1e-4)
    del dep
    # Gauss's law in spectral space with the modified k_z of order p
    kp = s.get("KPERP")[:, :, None]
    kz = s.get("KZ_MOD")[None, None, :]
    Eh = s.get("EH").astype(np.complex128)
    rho = s.get("RHO_PREV_H").astype(np.complex128) / O.EPS0
    res = O.op_div(kp, kz, Eh[0], Eh[1], Eh[2]) - rho
    # float32 beam-field set-up and update arithmetic: 6.6e-6 measured, constant over cycles
    assert np.abs(res).max() < 5e-5 * np.abs(rho).max()
