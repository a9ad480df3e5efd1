"""GPU checks of the tile tuning of the mixed form (pic_autotune / pic_set_tuning).

Every DHT tile height runs the same K order per output element, so the transforms agree
across tiles to rounding (asserted at 1e-6 relative, against 3e-5 for the stage itself);
every deposit chunk size meets the deposit tolerance against the FP64 oracle; the
autotuner's choice is one of the candidates and a cycle stepped with it matches the
untuned cycle.
"""
import numpy as np
import pytest

from oracle import psatd_rz as O
from paper_1611_05712_gb300 import binding as bd
from paper_1611_05712_gb300 import workloads as W
from gpu_helpers import per_slice_err, rel_err

pytestmark = pytest.mark.gpu

DZ = 0.05e-6


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1611_05712_gb300.build import build
    build()


def make(Nz, Nr, Nm, cap=0):
    cfg = bd.make_config(Nz, Nr, Nm, DZ, DZ, DZ / O.C_LIGHT, 0, True, bd.PIC_MIXED_TF32X3, cap)
    return bd.Sim(cfg), O.Grid(Nz, Nr, Nm, DZ, DZ, DZ / O.C_LIGHT)


def crand(rng, shape, scale=1.0):
    return scale * (rng.normal(size=shape) + 1j * rng.normal(size=shape))


@pytest.mark.parametrize("Nz,Nr,Nm", [(256, 200, 2), (128, 64, 3), (512, 256, 1)])
def test_dht_tiles_agree(Nz, Nr, Nm):
    s, g = make(Nz, Nr, Nm)
    h = O.hankel_setup(g)
    rng = np.random.default_rng(Nr)
    dep = crand(rng, (4, Nm, Nr, Nz))
    Eh, Bh = crand(rng, (3, Nm, Nr, Nz)), crand(rng, (3, Nm, Nr, Nz), 1e-8)
    ref_src = np.stack(O.forward_sources(g, h, dep[0], dep[1], dep[2], dep[3]))
    outs = []
    for nt in (0, 256, 128, 64, 48, 16):
        s.set_tuning(dht_n_tile=nt)
        assert s.get_tuning()["dht_n_tile"] == nt
        s.set("DEP", dep)
        s.forward_transform()
        s.set("EH", Eh)
        s.set("BH", Bh)
        s.inverse_transform()
        src, E, B = s.get("SRC_H"), s.get("E"), s.get("B")
        assert per_slice_err(src, ref_src) < 3e-5, nt
        outs.append((nt, src, E, B))
    for nt, src, E, B in outs[1:]:
        for a, b in ((src, outs[0][1]), (E, outs[0][2]), (B, outs[0][3])):
            assert rel_err(a, b) < 1e-6, nt


@pytest.mark.parametrize("chunk", [512, 1024, 2048])
def test_deposit_chunks_meet_tolerance(chunk):
    Nz, Nr, Nm = 256, 64, 2
    w = W.plasma_beam_small()
    P, _, _ = W.particles(w)
    n = len(P["x"])
    s, g = make(Nz, Nr, Nm, cap=n)
    s.set_tuning(band_chunk=chunk)
    s.write_particles(P)
    s.sort()
    P = s.read_particles()
    s.deposit(bd.PIC_DEP_RHO | bd.PIC_DEP_J)
    dep = s.get("DEP")
    rho = O.deposit_rho(g, P["x"], P["y"], P["z"], P["w"], -O.Q_E)
    ig = O.inv_gamma(P["ux"], P["uy"], P["uz"])
    J = O.deposit_current(g, P["x"], P["y"], P["z"], P["ux"] * ig, P["uy"] * ig, P["uz"] * ig, P["w"], -O.Q_E)
    assert rel_err(dep[0:1], rho[None]) < 1e-5
    assert rel_err(dep[1:], np.stack(J)) < 1e-5
    s.deposit(bd.PIC_DEP_J)   # J alone runs the banded kernel
    assert rel_err(s.get("DEP")[1:], np.stack(J)) < 1e-5


def test_autotune_choice_and_cycle():
    w = W.plasma_beam_small()
    P, npl, beams = W.particles(w)
    a = bd.Sim.from_workload(w, P, npl, beams, precision=bd.PIC_MIXED_TF32X3)
    b = bd.Sim.from_workload(w, P, npl, beams, precision=bd.PIC_MIXED_TF32X3)
    t = b.autotune()
    assert t["dht_n_tile"] in (256, 128, 64)
    assert t["band_chunk"] in (512, 1024, 2048)
    assert t["dht_ms"] > 0 and t["deposit_ms"] > 0
    assert b.get_tuning() == {"dht_n_tile": t["dht_n_tile"], "band_chunk": t["band_chunk"]}
    a.step(2)
    b.step(2)
    for name in ("E", "B"):
        assert rel_err(b.get(name), a.get(name)) < 1e-5, name


def test_set_tuning_rejects_bad_values():
    s, _ = make(64, 16, 1)
    for nt, ch in ((8, 1024), (24, 1024), (272, 1024), (0, 1000), (0, 4096)):
        with pytest.raises(bd.PicError):
            s.set_tuning(dht_n_tile=nt, band_chunk=ch)


@pytest.mark.parametrize("precision,tol_f,tol_x,tol_u", [(bd.PIC_FP64, 1e-11, 1e-11, 1e-11),
                                                          (bd.PIC_MIXED_TF32X3, 1e-4, 1e-5, 1e-4)])
def test_sort_interval_keeps_parity(precision, tol_f, tol_x, tol_u):
    # sorting every third cycle changes the order of the deposit additions only
    from gpu_helpers import by_id
    w = W.plasma_beam_small(order_p=16)
    P, npl, beams = W.particles(w)
    g = O.Grid(w.Nz, w.Nr, w.Nm, w.dz, w.dr, w.dt)
    s = bd.Sim.from_workload(w, P, npl, beams, precision=precision)
    s.set_sort_interval(3)
    assert s.get_sort_interval() == 3
    Pg = s.read_particles() if precision != bd.PIC_FP64 else P
    st = O.make_state(g, w.order_p, True, Pg, npl, beams)
    s.step(5)
    O.pic_step(st, 5)
    for name, ref in (("E", st.E), ("B", st.B)):
        assert rel_err(s.get(name), np.stack(ref)) < tol_f, name
    got, ref = by_id(s.read_particles()), by_id(st.p)
    for k in ("x", "y", "z"):
        assert rel_err(got[k], ref[k]) < tol_x, k
    for k in ("ux", "uy", "uz"):
        assert rel_err(got[k], ref[k]) < tol_u, k


def test_sort_interval_rejects_bad_values():
    w = W.tiny(order_p=16, Nz=32, Nr=8, Nm=1, n_beam=16)
    P, npl, beams = W.particles(w)
    s = bd.Sim.from_workload(w, P, npl, beams)
    for k in (0, -1, 17):
        with pytest.raises(bd.PicError):
            s.set_sort_interval(k)
    assert s.get_sort_interval() == 1
