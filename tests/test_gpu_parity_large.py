"""GPU parity against the FP64 oracle at the sizes the benchmarked configurations run.

* Transforms (a5/a6 forward, a8/a9 inverse) at Nr = 512 and 1024 and at the large run's
  8192 x 1024: the FP64 form within 1e-12 per (component, mode), both mixed forms within
  their stage tolerance (3e-5).  At Nr = 1024 the tensor-core DHT walks 32 K chunks and
  4 N tiles of 256 (TF32) or 8 of 128 (BF16).
* One full cycle of a crop of the large run (1024 x 128, 3 modes, p = 32, 12 plasma
  macroparticles per cell, drive and witness beams) in the FP64 and TF32x3 forms.
* A batch of three members of the order / resolution scan as the scan draws them
  (7-smooth Nz up to 3780, Nr up to 512, 3 modes, orders 8, 16 and infinite, c dt/dz 0.5
  and 1), advanced by one captured graph, each member against the oracle.
"""
import numpy as np
import pytest

from oracle import psatd_rz as O
from paper_1611_05712_gb300 import binding as bd
from paper_1611_05712_gb300 import workloads as W
from gpu_helpers import by_id, per_slice_err, rel_err

pytestmark = pytest.mark.gpu

DZ = 0.05e-6
TOL_FP64 = 1e-12
TOL_MIXED = 3e-5
SIZES = [(2048, 512, 2), (1024, 1024, 3), (8192, 1024, 1)]


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1611_05712_gb300.build import build
    build()


_hankel = {}


def _oracle_grid(Nz, Nr, Nm):
    g = O.Grid(Nz, Nr, Nm, DZ, DZ, DZ / O.C_LIGHT)
    key = (Nr, Nm)
    if key not in _hankel:
        _hankel[key] = O.hankel_setup(O.Grid(8, Nr, Nm, DZ, DZ, DZ / O.C_LIGHT))
    return g, _hankel[key]


def crand(rng, shape, scale=1.0):
    return scale * (rng.normal(size=shape) + 1j * rng.normal(size=shape))


@pytest.mark.parametrize("Nz,Nr,Nm", SIZES)
@pytest.mark.parametrize("precision,tol", [(bd.PIC_FP64, TOL_FP64), (bd.PIC_MIXED_TF32X3, TOL_MIXED),
                                           (bd.PIC_MIXED_BF16X6, TOL_MIXED)])
def test_transforms_at_configuration_sizes(Nz, Nr, Nm, precision, tol):
    cfg = bd.make_config(Nz, Nr, Nm, DZ, DZ, DZ / O.C_LIGHT, 32, True, precision, 0)
    s = bd.Sim(cfg)
    g, h = _oracle_grid(Nz, Nr, Nm)
    rng = np.random.default_rng(Nz + 7 * Nr + Nm)
    dep = crand(rng, (4, Nm, Nr, Nz))
    s.set("DEP", dep)
    s.forward_transform()
    ref = np.stack(O.forward_sources(g, h, dep[0], dep[1], dep[2], dep[3]))
    assert per_slice_err(s.get("SRC_H"), ref) < tol
    del dep, ref
    Eh, Bh = crand(rng, (3, Nm, Nr, Nz)), crand(rng, (3, Nm, Nr, Nz), 1e-8)
    s.set("EH", Eh)
    s.set("BH", Bh)
    s.inverse_transform()
    assert per_slice_err(s.get("E"), np.stack(O.inverse_vector(g, h, *Eh))) < tol
    assert per_slice_err(s.get("B"), np.stack(O.inverse_vector(g, h, *Bh))) < tol
    s.close()


@pytest.fixture(scope="module")
def crop():
    w = W.large_crop_1024x128(order_p=32)
    P, npl, beams = W.particles(w)
    g = O.Grid(w.Nz, w.Nr, w.Nm, w.dz, w.dr, w.dt)
    return w, P, npl, beams, g, O.hankel_setup(g)


@pytest.mark.parametrize("precision", [bd.PIC_FP64, bd.PIC_MIXED_TF32X3])
def test_full_cycle_on_a_crop_of_the_large_run(crop, precision):
    w, P, npl, beams, g, h = crop
    s = bd.Sim.from_workload(w, P, npl, beams, precision=precision)
    if precision != bd.PIC_FP64:
        s.autotune()
    # the oracle starts from the particle state the handle holds (the float form rounds it)
    st = O.make_state(g, w.order_p, True, s.read_particles(), npl, beams, h=h)
    s.step(1)
    O.pic_step(st, 1)
    tol_f, tol_x, tol_u = (TOL_FP64, TOL_FP64, TOL_FP64) if precision == bd.PIC_FP64 else (1e-4, 1e-5, 1e-4)
    for name, ref in (("E", st.E), ("B", st.B), ("EH", st.Eh), ("BH", st.Bh)):
        assert rel_err(s.get(name), np.stack(ref)) < tol_f, name
    got, ref = by_id(s.read_particles()), by_id(st.p)
    assert np.array_equal(got["id"], ref["id"])
    for k in ("x", "y", "z"):
        assert rel_err(got[k], ref[k]) < tol_x, k
    for k in ("ux", "uy", "uz"):
        assert rel_err(got[k], ref[k]) < tol_u, k
    s.close()


SCAN_MEMBERS = (13, 20, 45)   # (3780, 400, 3, p 8, cfl 1), (2100, 512, 3, p 16, cfl 0.5), (2187, 288, 3, inf, 0.5)


@pytest.mark.parametrize("precision,tol", [(bd.PIC_FP64, 1e-11), (bd.PIC_MIXED_TF32X3, 1e-4)])
def test_batch_of_scan_members_matches_the_oracle(precision, tol):
    import torch
    ws = [W.scan_member(k) for k in SCAN_MEMBERS]
    assert [w.Nm for w in ws] == [3, 3, 3] and 0 in [w.order_p for w in ws]
    streams = [torch.cuda.Stream() for _ in ws]
    sims, inputs = [], []
    for w, stream in zip(ws, streams):
        P, npl, beams = W.particles(w)
        sims.append(bd.Sim.from_workload(w, P, npl, beams, precision=precision, stream=stream))
        inputs.append((npl, beams))
    starts = [s.read_particles() for s in sims]
    batch = bd.Batch(sims, cycles=2)
    batch.launch(1)
    batch.origin.synchronize()
    for w, s, P0, (npl, beams) in zip(ws, sims, starts, inputs):
        g = O.Grid(w.Nz, w.Nr, w.Nm, w.dz, w.dr, w.dt)
        st = O.make_state(g, w.order_p, True, P0, npl, beams)
        O.pic_step(st, 2)
        s.sync()
        for name, ref in (("E", st.E), ("B", st.B)):
            assert rel_err(s.get(name), np.stack(ref)) < tol, (w.name, name)
        got, ref = by_id(s.read_particles()), by_id(st.p)
        for k in ("x", "y", "z"):
            assert rel_err(got[k], ref[k]) < (tol if precision == bd.PIC_FP64 else 1e-5), (w.name, k)
        for k in ("ux", "uy", "uz"):
            assert rel_err(got[k], ref[k]) < tol, (w.name, k)
    batch.close()
