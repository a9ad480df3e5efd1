"""The two DHT paths of the FP64 form against the oracle (section "Finite order pseudo-spectral
solvers": Hankel transform along r).

The sliced path scales every matrix row and panel column by a power of two, cuts the values
into seven 7-bit slices (exact BF16 numbers), accumulates the slice products exactly in FP32
on the tensor cores and combines them in FP64; it must meet the FP64 bar (1e-12 per
(component, mode) against the oracle) like the FP64 SIMT GEMM, on random panels whose
columns span many orders of magnitude, on both directions, and inside full cycles.
"""
import numpy as np
import pytest

from oracle import psatd_rz as O
from paper_1611_05712_gb300 import binding as bd
from paper_1611_05712_gb300 import workloads as W
from gpu_helpers import by_id, per_slice_err, rel_err

pytestmark = pytest.mark.gpu

DZ = 0.05e-6
TOL = 1e-12


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1611_05712_gb300.build import build
    build()


def make(Nz, Nr, Nm, path):
    cfg = bd.make_config(Nz, Nr, Nm, DZ, DZ, DZ / O.C_LIGHT, 32, True, bd.PIC_FP64, 0)
    s = bd.Sim(cfg)
    s.set_dht_path(path)
    return s, O.Grid(Nz, Nr, Nm, DZ, DZ, DZ / O.C_LIGHT)


def panel(rng, shape, scale=1.0):
    """Complex random data whose z columns span ~12 orders of magnitude."""
    col = 10.0 ** rng.uniform(-6, 6, size=shape[-1])
    return scale * (rng.normal(size=shape) + 1j * rng.normal(size=shape)) * col


@pytest.mark.parametrize("Nz,Nr,Nm", [(16, 8, 2), (60, 33, 3), (256, 64, 2), (2048, 256, 2), (128, 200, 1),
                                      (96, 256, 4)])
@pytest.mark.parametrize("path", [bd.PIC_DHT_F64_SLICED, bd.PIC_DHT_F64_GEMM])
def test_fp64_dht_paths_match_the_oracle(Nz, Nr, Nm, path):
    s, g = make(Nz, Nr, Nm, path)
    assert s.get_dht_path() == path
    h = O.hankel_setup(g)
    rng = np.random.default_rng(Nz + 11 * Nr + path)
    dep = panel(rng, (4, Nm, Nr, Nz))
    s.set("DEP", dep)
    s.forward_transform()
    ref = np.stack(O.forward_sources(g, h, dep[0], dep[1], dep[2], dep[3]))
    assert per_slice_err(s.get("SRC_H"), ref) < TOL
    Eh, Bh = panel(rng, (3, Nm, Nr, Nz)), panel(rng, (3, Nm, Nr, Nz), 1e-8)
    s.set("EH", Eh)
    s.set("BH", Bh)
    s.inverse_transform()
    assert per_slice_err(s.get("E"), np.stack(O.inverse_vector(g, h, *Eh))) < TOL
    assert per_slice_err(s.get("B"), np.stack(O.inverse_vector(g, h, *Bh))) < TOL
    s.close()


def test_sliced_path_full_cycles_match_the_oracle():
    w = W.plasma_beam_small()
    P, npl, beams = W.particles(w)
    s = bd.Sim.from_workload(w, P, npl, beams)
    assert s.get_dht_path() == bd.PIC_DHT_AUTO      # Nr = 64: the sliced path
    g = O.Grid(w.Nz, w.Nr, w.Nm, w.dz, w.dr, w.dt)
    st = O.make_state(g, w.order_p, True, P, npl, beams)
    s.step(5)
    O.pic_step(st, 5)
    for name, ref in (("E", st.E), ("B", st.B), ("EH", st.Eh), ("BH", st.Bh)):
        assert rel_err(s.get(name), np.stack(ref)) < 1e-10, name
    got, ref = by_id(s.read_particles()), by_id(st.p)
    for k in bd.SOA:
        assert rel_err(got[k], ref[k]) < 1e-10, k
    s.close()


def test_dht_path_arguments():
    s, _ = make(64, 300, 1, bd.PIC_DHT_AUTO)             # Nr > 256: no sliced path
    with pytest.raises(bd.PicError):
        s.set_dht_path(bd.PIC_DHT_F64_SLICED)
    with pytest.raises(bd.PicError):
        s.set_dht_path(7)
    s.close()
    cfg = bd.make_config(64, 32, 1, DZ, DZ, DZ / O.C_LIGHT, 32, True, bd.PIC_MIXED_TF32X3, 0)
    m = bd.Sim(cfg)
    with pytest.raises(bd.PicError):
        m.set_dht_path(bd.PIC_DHT_F64_SLICED)
    m.close()
