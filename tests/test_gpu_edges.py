"""Edge cases of the newer entry points and forms on the GPU: empty particle sets in both
mixed forms, tuned tiles with autotuning on an empty set, and argument errors of the
window copy and tuning calls (returned as PIC_ERR_ARG, nothing launched)."""
import numpy as np
import pytest

from oracle import psatd_rz as O
from paper_1611_05712_gb300 import binding as bd

pytestmark = pytest.mark.gpu

DZ = 0.05e-6


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1611_05712_gb300.build import build
    build()


def make(Nz, Nr, Nm, precision, cap=16):
    cfg = bd.make_config(Nz, Nr, Nm, DZ, DZ, DZ / O.C_LIGHT, 16, True, precision, cap)
    return bd.Sim(cfg)


@pytest.mark.parametrize("precision", [bd.PIC_MIXED_TF32X3, bd.PIC_MIXED_BF16X6])
def test_mixed_forms_step_an_empty_particle_set(precision):
    s = make(48, 20, 2, precision)
    s.write_particles({k: np.zeros(0) for k in bd.SOA} | {"id": np.zeros(0, np.int32)})
    s.init_background(0)
    s.init_fields()
    t = s.autotune()   # no particles: the deposit chunk is left as it is
    assert t["band_chunk"] == 1024
    s.step(3)
    s.sync()
    assert np.abs(s.get("E")).max() == 0.0
    assert np.abs(s.get("B")).max() == 0.0


def test_copy_window_rejects_bad_arguments():
    a = make(64, 16, 2, bd.PIC_FP64)
    b = make(32, 16, 2, bd.PIC_FP64)
    c = make(32, 8, 2, bd.PIC_FP64)
    m = make(32, 16, 2, bd.PIC_MIXED_TF32X3)
    with pytest.raises(bd.PicError):
        a.copy_window_to(b, "EH", 0, 16, 0)       # spectral buffers are not windows in z
    with pytest.raises(bd.PicError):
        a.copy_window_to(b, "E", 0, 40, 0)        # longer than the destination
    with pytest.raises(bd.PicError):
        a.copy_window_to(c, "E", 0, 16, 0)        # another Nr
    with pytest.raises(bd.PicError):
        a.copy_window_to(m, "E", 0, 16, 0)        # another precision
    # a periodic window across the end of the source lands in order
    rng = np.random.default_rng(5)
    E = rng.normal(size=(3, 2, 16, 64)) + 1j * rng.normal(size=(3, 2, 16, 64))
    a.set("E", E)
    b.set("E", b.zeros("E"))
    a.copy_window_to(b, "E", 56, 16, 8)
    got = b.get("E")
    assert np.array_equal(got[..., 8:24], np.concatenate([E[..., 56:], E[..., :8]], axis=-1))
    assert np.abs(got[..., :8]).max() == 0.0 and np.abs(got[..., 24:]).max() == 0.0


def test_sort_of_one_cell_holding_every_particle_is_bounded():
    """pic_sort with 300,000 particles in one cell (FP64 handle): the cell's entries are
    ordered by an O(n log n) CTA sort, the permutation is the identity (stable order of
    equal keys, as the oracle's stable sort gives) and the sort stays in milliseconds."""
    import torch
    n, Nz, Nr = 300000, 64, 32
    cfg = bd.make_config(Nz, Nr, 1, DZ, DZ, DZ / O.C_LIGHT, 0, True, bd.PIC_FP64, n)
    s = bd.Sim(cfg)
    P = {k: np.zeros(n) for k in bd.SOA} | {"id": np.arange(n, dtype=np.int32)}
    P["x"][:], P["y"][:], P["z"][:], P["w"][:] = 3.3 * DZ, 1.1 * DZ, 7.5 * DZ, 1.0
    s.write_particles(P)
    s.sort()
    s.sync()
    g = O.Grid(Nz, Nr, 1, DZ, DZ, DZ / O.C_LIGHT)
    okeys = O.cell_keys(g, P["x"], P["y"], P["z"])
    assert np.array_equal(s.get("KEYS"), okeys)
    assert np.array_equal(s.get("PERM"), O.sort_permutation(okeys))
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(s.stream)
    s.sort()
    e1.record(s.stream)
    s.sync()
    torch.cuda.synchronize()
    assert e0.elapsed_time(e1) < 200.0
    s.close()
