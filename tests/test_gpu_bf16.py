"""GPU parity of the BF16-split form (PIC_MIXED_BF16X6) against the FP64 oracle.

Same mixed form as PIC_MIXED_TF32X3 (float grids, FP32 cell-relative particles, FP64 setup
and diagnostics) except the DHT: each float is split into three BF16 pieces and the six
products of order <= 2 are summed on the tensor cores with float accumulation.  Stated
tolerances are those of the TF32 form: transforms and PSATD 3e-5 per (component, mode) on
random inputs, one full cycle 1e-4 per field, and beam emittance and slice energy spread
within 1e-4 of the FP64 form after 100 cycles.
"""
import numpy as np
import pytest

from oracle import psatd_rz as O
from paper_1611_05712_gb300 import binding as bd
from paper_1611_05712_gb300 import workloads as W
from gpu_helpers import by_id, per_slice_err, rel_err

pytestmark = pytest.mark.gpu

DZ = 0.05e-6
TOL_STAGE = 3e-5


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1611_05712_gb300.build import build
    build()


def make(Nz, Nr, Nm):
    cfg = bd.make_config(Nz, Nr, Nm, DZ, DZ, DZ / O.C_LIGHT, 0, True, bd.PIC_MIXED_BF16X6, 0)
    return bd.Sim(cfg), O.Grid(Nz, Nr, Nm, DZ, DZ, DZ / O.C_LIGHT)


def crand(rng, shape, scale=1.0):
    return scale * (rng.normal(size=shape) + 1j * rng.normal(size=shape))


# Nr below, at and across the 64-element K chunk and the 128-row tile; Nz across the
# 128-column M tile
@pytest.mark.parametrize("Nz,Nr,Nm", [(16, 8, 2), (60, 33, 3), (256, 64, 2), (128, 200, 1), (2048, 256, 2)])
@pytest.mark.parametrize("n_tile", [0, 64, 16])
def test_bf16_forward_inverse_transform(Nz, Nr, Nm, n_tile):
    s, g = make(Nz, Nr, Nm)
    s.set_tuning(dht_n_tile=n_tile)
    h = O.hankel_setup(g)
    rng = np.random.default_rng(Nz + 5 * Nr)
    dep = crand(rng, (4, Nm, Nr, Nz))
    s.set("DEP", dep)
    s.forward_transform()
    ref = np.stack(O.forward_sources(g, h, dep[0], dep[1], dep[2], dep[3]))
    assert per_slice_err(s.get("SRC_H"), ref) < TOL_STAGE
    Eh, Bh = crand(rng, (3, Nm, Nr, Nz)), crand(rng, (3, Nm, Nr, Nz), 1e-8)
    s.set("EH", Eh)
    s.set("BH", Bh)
    s.inverse_transform()
    assert per_slice_err(s.get("E"), np.stack(O.inverse_vector(g, h, *Eh))) < TOL_STAGE
    assert per_slice_err(s.get("B"), np.stack(O.inverse_vector(g, h, *Bh))) < TOL_STAGE


def test_bf16_n_tile_is_capped_at_128():
    s, _ = make(64, 256, 1)
    s.set_tuning(dht_n_tile=256)   # accepted, applied as 128 (three planes fill shared memory)
    rng = np.random.default_rng(1)
    g = O.Grid(64, 256, 1, DZ, DZ, DZ / O.C_LIGHT)
    h = O.hankel_setup(g)
    dep = crand(rng, (4, 1, 256, 64))
    s.set("DEP", dep)
    s.forward_transform()
    ref = np.stack(O.forward_sources(g, h, dep[0], dep[1], dep[2], dep[3]))
    assert per_slice_err(s.get("SRC_H"), ref) < TOL_STAGE


def test_bf16_full_cycle_plasma_beam_256x64():
    w = W.plasma_beam_small()
    P, npl, beams = W.particles(w)
    g = O.Grid(w.Nz, w.Nr, w.Nm, w.dz, w.dr, w.dt)
    s = bd.Sim.from_workload(w, P, npl, beams, precision=bd.PIC_MIXED_BF16X6)
    st = O.make_state(g, w.order_p, True, P, npl, beams)
    s.step(1)
    O.pic_step(st, 1)
    for name, ref in (("E", st.E), ("B", st.B), ("EH", st.Eh), ("BH", st.Bh)):
        assert rel_err(s.get(name), np.stack(ref)) < 1e-4, name
    got, ref = by_id(s.read_particles()), by_id(st.p)
    for k in ("x", "y", "z"):
        assert rel_err(got[k], ref[k]) < 1e-5, k
    for k in ("ux", "uy", "uz"):
        assert rel_err(got[k], ref[k]) < 1e-4, k


def test_bf16_beam_quality_within_1e4_of_fp64_after_many_cycles():
    w = W.plasma_beam_small()
    P, npl, beams = W.particles(w)
    lo, hi = beams[0][0], beams[0][1]
    s64 = bd.Sim.from_workload(w, P, npl, beams, precision=bd.PIC_FP64)
    s16 = bd.Sim.from_workload(w, P, npl, beams, precision=bd.PIC_MIXED_BF16X6)
    s64.step(100)
    s16.step(100)
    d64, d16 = s64.diagnostics(lo, hi), s16.diagnostics(lo, hi)
    for k in ("emit_nx", "emit_ny"):
        assert abs(d16[k] - d64[k]) <= max(1e-4 * abs(d64[k]), 1e-12), (k, d16[k], d64[k])
    assert d16["sigma_gamma_mean"] == pytest.approx(d64["sigma_gamma_mean"], rel=1e-4)
    assert d16["gamma_mean"] == pytest.approx(d64["gamma_mean"], rel=1e-6)
