"""GPU parity of the mixed-precision form (PIC_MIXED_TF32X3) against the FP64 oracle.

Mixed form: float grids, FFT and PSATD in float, the DHT as 3-term TF32 products with
float accumulation, FP32 particles with z relative to its cell, FP64 setup and
diagnostics.  Stated per-field tolerances (max |gpu - oracle| / max |oracle|):
transforms and PSATD 3e-5 per (component, mode) on random inputs; one full cycle from an
identical state 1e-4 per field, particle positions 1e-5 (momenta 1e-4) per array.  The
beam-quality criterion of the mixed form -- beam emittance and slice energy spread within
1e-4 relative of the FP64 path after many cycles -- is checked against the FP64 GPU path.
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


def make(Nz, Nr, Nm, p=0, filt=True, cap=0, cfl=1.0):
    cfg = bd.make_config(Nz, Nr, Nm, DZ, DZ, cfl * DZ / O.C_LIGHT, p, filt, bd.PIC_MIXED_TF32X3, cap)
    g = O.Grid(Nz, Nr, Nm, DZ, DZ, cfl * DZ / O.C_LIGHT)
    return bd.Sim(cfg), g


def crand(rng, shape, scale=1.0):
    return scale * (rng.normal(size=shape) + 1j * rng.normal(size=shape))


SHAPES = [(16, 8, 2), (60, 33, 3), (256, 64, 2), (2048, 256, 2), (32, 4, 1), (128, 8, 1), (1024, 8, 1),
          (4096, 8, 1), (8192, 8, 2), (24, 4, 2), (343, 4, 1), (1000, 8, 2), (3456, 4, 3)]


@pytest.mark.parametrize("Nz,Nr,Nm", SHAPES)
def test_mixed_forward_inverse_transform(Nz, Nr, Nm):
    s, g = make(Nz, Nr, Nm)
    h = O.hankel_setup(g)
    rng = np.random.default_rng(Nz + 3 * Nr)
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


@pytest.mark.parametrize("p,filt,cfl", [(0, True, 1.0), (32, False, 0.5)])
def test_mixed_psatd_stage(p, filt, cfl):
    Nz, Nr, Nm = 60, 33, 3
    s, g = make(Nz, Nr, Nm, p, filt, cfl=cfl)
    h = O.hankel_setup(g)
    coef = O.psatd_coefficients(g, h, p)
    T = O.source_filter(g, h)
    rng = np.random.default_rng(5 + p)
    sh = (Nm, Nr, Nz)
    E = crand(rng, (3,) + sh, 1e9)
    B = crand(rng, (3,) + sh, 1e9 / O.C_LIGHT)
    src = np.stack([crand(rng, sh, 1e3)] + [crand(rng, sh, 1e3 * O.C_LIGHT) for _ in range(3)])
    rho_prev = crand(rng, sh, 1e3)
    for name, val in (("EH", E), ("BH", B), ("SRC_H", src), ("RHO_PREV_H", rho_prev)):
        s.set(name, val)
    s.psatd()
    En, Bn, rf, _ = O.psatd_update(g, coef, T, tuple(E), tuple(B), tuple(src[1:]), src[0], rho_prev,
                                   filt=filt, correct=True)
    assert per_slice_err(s.get("EH"), np.stack(En)) < TOL_STAGE
    assert per_slice_err(s.get("BH"), np.stack(Bn)) < TOL_STAGE
    assert rel_err(s.get("RHO_PREV_H"), rf) < TOL_STAGE


def test_mixed_sort_is_a_stable_sort_of_its_keys():
    """FP32 positions: keys are compared with the oracle's key rule applied to the
    positions the GPU holds (they may differ only for particles within float rounding
    of a cell edge); the permutation must be exactly the stable order of the GPU's keys."""
    Nz, Nr, n = 256, 64, 36384
    s, g = make(Nz, Nr, 1, cap=n)
    w = W.plasma_beam_small()
    P, _, _ = W.particles(w)
    s.write_particles(P)
    held = s.read_particles()
    s.sort()
    keys, perm = s.get("KEYS"), s.get("PERM")
    ref = O.cell_keys(g, held["x"], held["y"], held["z"])
    assert np.mean(keys == ref) > 0.999
    assert np.array_equal(perm, O.sort_permutation(keys))
    got = s.read_particles()
    assert np.array_equal(got["id"], held["id"][perm])


def test_mixed_deposit_and_gather_push():
    Nz, Nr, Nm, n = 64, 16, 2, 3000
    s, g = make(Nz, Nr, Nm, cap=n)
    rng = np.random.default_rng(9)
    r = g.R * 0.98 * np.sqrt(rng.uniform(0, 1, n))
    th = rng.uniform(0, 2 * np.pi, n)
    P = dict(x=r * np.cos(th), y=r * np.sin(th), z=rng.uniform(0, g.L, n),
             ux=rng.normal(0, 3e7, n), uy=rng.normal(0, 3e7, n), uz=rng.normal(1e8, 3e8, n),
             w=rng.uniform(0.5, 2.0, n) * 1e4, id=np.arange(n, dtype=np.int32))
    s.write_particles(P)
    P = s.read_particles()      # the float-held state is the common starting point
    s.deposit(bd.PIC_DEP_RHO | bd.PIC_DEP_J)
    dep = s.get("DEP")
    rho = O.deposit_rho(g, P["x"], P["y"], P["z"], P["w"], -O.Q_E)
    ig = O.inv_gamma(P["ux"], P["uy"], P["uz"])
    J = O.deposit_current(g, P["x"], P["y"], P["z"], P["ux"] * ig, P["uy"] * ig, P["uz"] * ig, P["w"], -O.Q_E)
    assert per_slice_err(dep[0:1], rho[None]) < 1e-5
    assert per_slice_err(dep[1:], np.stack(J)) < 1e-5
    E = crand(rng, (3, Nm, Nr, Nz), 1e10)
    B = crand(rng, (3, Nm, Nr, Nz), 1e10 / O.C_LIGHT)
    s.set("E", E)
    s.set("B", B)
    s.gather_push(fuse_current=True)
    zero = np.zeros((Nm, Nr, Nz), complex)
    st = O.State(g, 0, False, -O.Q_E, O.M_E, None, None, None, tuple(E.astype(np.complex64).astype(complex)),
                 tuple(B.astype(np.complex64).astype(complex)), None, None, zero, zero,
                 {k: v.copy() for k, v in P.items()})
    Jo = O.gather_push(st)
    got = s.read_particles()
    for k in ("x", "y", "z"):
        assert rel_err(got[k], st.p[k]) < 1e-5, k
    for k in ("ux", "uy", "uz"):
        assert rel_err(got[k], st.p[k]) < 1e-4, k
    assert rel_err(s.get("DEP")[1:], np.stack(Jo)) < 1e-4


def test_mixed_full_cycle_plasma_beam_256x64():
    w = W.plasma_beam_small()
    P, npl, beams = W.particles(w)
    g = O.Grid(w.Nz, w.Nr, w.Nm, w.dz, w.dr, w.dt)
    s = bd.Sim.from_workload(w, P, npl, beams, precision=bd.PIC_MIXED_TF32X3)
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


def test_mixed_beam_quality_within_1e4_of_fp64_after_many_cycles():
    """Beam-quality criterion: emittance and slice energy spread of the beam in the mixed form
    within 1e-4 relative of the FP64 form after 100 cycles of the 256 x 64 plasma + beam case
    (absolute emittance difference below 1e-12 m rad where the FP64 value is tiny)."""
    w = W.plasma_beam_small()
    P, npl, beams = W.particles(w)
    lo, hi = beams[0][0], beams[0][1]
    s64 = bd.Sim.from_workload(w, P, npl, beams, precision=bd.PIC_FP64)
    s32 = bd.Sim.from_workload(w, P, npl, beams, precision=bd.PIC_MIXED_TF32X3)
    s64.step(100)
    s32.step(100)
    d64, d32 = s64.diagnostics(lo, hi), s32.diagnostics(lo, hi)
    for k in ("emit_nx", "emit_ny"):
        assert abs(d32[k] - d64[k]) <= max(1e-4 * abs(d64[k]), 1e-12), (k, d32[k], d64[k])
    assert d32["sigma_gamma_mean"] == pytest.approx(d64["sigma_gamma_mean"], rel=1e-4)
    assert d32["gamma_mean"] == pytest.approx(d64["gamma_mean"], rel=1e-6)
