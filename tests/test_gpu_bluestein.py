"""GPU parity of the z transforms for lengths that are not 7-smooth (Bluestein's chirp-z
algorithm on power-of-two rows; Fourier transform along z of section "Finite order
pseudo-spectral solvers") against the oracle, whose DFT is numpy's at any length.

* Forward and inverse field transforms (z-DFT plus Hankel) at prime lengths (61, 127,
  1021, 2039, the largest FP64 Bluestein rows, M = 4096) and composite non-smooth ones
  (22 = 2 x 11, 143 = 11 x 13): FP64 within 1e-12 per (component, mode); both mixed forms
  within their stage tolerance 3e-5, up to Nz = 4093 (M = 8192).
* Two full PIC cycles of a plasma + beam case at a prime Nz = 61 in the FP64 and TF32x3
  forms.
(The length limits are checked on the CPU in test_library_abi.py.)
"""
import numpy as np
import pytest

from oracle import psatd_rz as O
from paper_1611_05712_gb300 import binding as bd
from paper_1611_05712_gb300 import workloads as W
from gpu_helpers import by_id, per_slice_err, rel_err

pytestmark = pytest.mark.gpu

DZ = 0.05e-6


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1611_05712_gb300.build import build
    build()


def make(Nz, Nr, Nm, precision, p=0):
    cfg = bd.make_config(Nz, Nr, Nm, DZ, DZ, DZ / O.C_LIGHT, p, True, precision, 0)
    return bd.Sim(cfg), O.Grid(Nz, Nr, Nm, DZ, DZ, DZ / O.C_LIGHT)


def crand(rng, shape, scale=1.0):
    return scale * (rng.normal(size=shape) + 1j * rng.normal(size=shape))


def transforms(Nz, Nr, Nm, precision, tol):
    s, g = make(Nz, Nr, Nm, precision)
    h = O.hankel_setup(g)
    rng = np.random.default_rng(Nz + 7 * Nr)
    dep = crand(rng, (4, Nm, Nr, Nz))
    s.set("DEP", dep)
    s.forward_transform()
    ref = np.stack(O.forward_sources(g, h, dep[0], dep[1], dep[2], dep[3]))
    assert per_slice_err(s.get("SRC_H"), ref) < tol
    Eh, Bh = crand(rng, (3, Nm, Nr, Nz)), crand(rng, (3, Nm, Nr, Nz), 1e-8)
    s.set("EH", Eh)
    s.set("BH", Bh)
    s.inverse_transform()
    assert per_slice_err(s.get("E"), np.stack(O.inverse_vector(g, h, *Eh))) < tol
    assert per_slice_err(s.get("B"), np.stack(O.inverse_vector(g, h, *Bh))) < tol


@pytest.mark.parametrize("Nz,Nr,Nm", [(61, 8, 2), (127, 4, 1), (22, 8, 1), (143, 8, 3), (1021, 4, 1),
                                      (2039, 4, 2)])
def test_fp64_transforms_non_smooth_lengths(Nz, Nr, Nm):
    transforms(Nz, Nr, Nm, bd.PIC_FP64, 1e-12)


@pytest.mark.parametrize("precision", [bd.PIC_MIXED_TF32X3, bd.PIC_MIXED_BF16X6])
@pytest.mark.parametrize("Nz,Nr,Nm", [(61, 8, 2), (143, 8, 1), (2039, 4, 1), (4093, 4, 1)])
def test_mixed_transforms_non_smooth_lengths(Nz, Nr, Nm, precision):
    transforms(Nz, Nr, Nm, precision, 3e-5)


@pytest.mark.parametrize("precision,tol_f,tol_x,tol_u", [(bd.PIC_FP64, 1e-12, 1e-12, 1e-12),
                                                          (bd.PIC_MIXED_TF32X3, 1e-4, 1e-5, 1e-4)])
def test_full_cycle_prime_length(precision, tol_f, tol_x, tol_u):
    w = W.tiny(order_p=16, Nz=61, Nr=16, Nm=2, n_beam=256)
    P, npl, beams = W.particles(w)
    g = O.Grid(w.Nz, w.Nr, w.Nm, w.dz, w.dr, w.dt)
    s = bd.Sim.from_workload(w, P, npl, beams, precision=precision)
    Pg = s.read_particles() if precision != bd.PIC_FP64 else P
    st = O.make_state(g, w.order_p, True, Pg, npl, beams)
    s.step(2)
    O.pic_step(st, 2)
    for name, ref in (("E", st.E), ("B", st.B), ("EH", st.Eh), ("BH", st.Bh)):
        assert rel_err(s.get(name), np.stack(ref)) < tol_f, name
    got, ref = by_id(s.read_particles()), by_id(st.p)
    for k in ("x", "y", "z"):
        assert rel_err(got[k], ref[k]) < tol_x, k
    for k in ("ux", "uy", "uz"):
        assert rel_err(got[k], ref[k]) < tol_u, k
