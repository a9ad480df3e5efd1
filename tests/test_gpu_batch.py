"""Batched scan: several uneven simulations advanced by one captured CUDA graph per launch
give the same fields and particles as the same simulations stepped one by one (FP64:
1e-12 per field, differences come only from the order of atomic additions), and one of
them matches the FP64 oracle."""
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


def _members():
    """Three small members of an order / resolution scan with uneven sizes."""
    out = []
    for (Nz, Nr, Nm, p, cfl, seed) in ((120, 24, 1, 8, 0.5, 11), (256, 40, 2, 0, 1.0, 12),
                                       (96, 16, 3, 32, 1.0, 13)):
        w = W.tiny(order_p=p, seed=seed, Nz=Nz, Nr=Nr, Nm=Nm, n_beam=400)
        w.dt = cfl * w.dz / O.C_LIGHT
        out.append(w)
    return out


def _make(w, precision, stream):
    P, npl, beams = W.particles(w)
    return bd.Sim.from_workload(w, P, npl, beams, precision=precision, stream=stream), (P, npl, beams)


@pytest.mark.parametrize("precision,tol", [(bd.PIC_FP64, 1e-12), (bd.PIC_MIXED_TF32X3, 1e-5),
                                           (bd.PIC_MIXED_BF16X6, 1e-5)])
def test_batch_graph_matches_individual_stepping(precision, tol):
    import torch
    ws = _members()
    streams = [torch.cuda.Stream() for _ in ws]
    batched = [_make(w, precision, st)[0] for w, st in zip(ws, streams)]
    single = [_make(w, precision, None)[0] for w in ws]
    batch = bd.Batch(batched, cycles=2)
    assert batch.kernels_per_launch > 0
    batch.launch(2)
    batch.origin.synchronize()
    for s in single:
        s.step(4)
    for a, b in zip(batched, single):
        a.sync()
        for name in ("E", "B", "EH", "BH", "RHO_PREV_H"):
            assert rel_err(a.get(name), b.get(name)) < tol, name
        pa, pb = by_id(a.read_particles()), by_id(b.read_particles())
        for k in bd.SOA:
            assert rel_err(pa[k], pb[k]) < tol, k
    batch.close()


def test_batched_member_matches_oracle():
    import torch
    w = _members()[1]
    s, (P, npl, beams) = _make(w, bd.PIC_FP64, torch.cuda.Stream())
    batch = bd.Batch([s], cycles=2)
    batch.launch(1)
    batch.origin.synchronize()
    g = O.Grid(w.Nz, w.Nr, w.Nm, w.dz, w.dr, w.dt)
    st = O.make_state(g, w.order_p, True, P, npl, beams)
    O.pic_step(st, 2)
    for name, ref in (("E", st.E), ("B", st.B)):
        assert rel_err(s.get(name), np.stack(ref)) < 1e-11, name
    got, ref = by_id(s.read_particles()), by_id(st.p)
    for k in bd.SOA:
        assert rel_err(got[k], ref[k]) < 1e-11, k


def test_batch_rejects_odd_cycles_and_default_stream():
    w = _members()[0]
    s, _ = _make(w, bd.PIC_FP64, None)
    with pytest.raises(bd.PicError):
        bd.Batch([s], cycles=2)          # default stream
    import torch
    s2, _ = _make(w, bd.PIC_FP64, torch.cuda.Stream())
    with pytest.raises(bd.PicError):
        bd.Batch([s2], cycles=3)
