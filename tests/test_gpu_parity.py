"""GPU (sm_103a) parity of every stage of the PIC cycle against the FP64 oracle.

All calls go through the C ABI (libpsatd_rz.so via the ctypes binding).  FP64 bar:
max |gpu - oracle| / max |oracle| <= 1e-12 per (field, component, mode) and per particle
array after one step from an identical state; integer work (cell keys, sort
permutation) bit-exact.  Setup tables: the forward Hankel matrices are pseudo-inverses
refined by one Newton-Schulz step, agree to 1e-12.
"""
import math

import numpy as np
import pytest

from oracle import psatd_rz as O
from paper_1611_05712_gb300 import binding as bd
from paper_1611_05712_gb300 import workloads as W
from gpu_helpers import by_id, per_slice_err, rel_err

pytestmark = pytest.mark.gpu

TOL = 1e-12
DZ = 0.05e-6


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1611_05712_gb300.build import build
    build()
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"


def make(Nz, Nr, Nm, p=0, filt=True, cap=0, cfl=1.0):
    cfg = bd.make_config(Nz, Nr, Nm, DZ, DZ, cfl * DZ / O.C_LIGHT, p, filt, bd.PIC_FP64, cap)
    g = O.Grid(Nz, Nr, Nm, DZ, DZ, cfl * DZ / O.C_LIGHT)
    return bd.Sim(cfg), g


def crand(rng, shape, scale=1.0):
    return scale * (rng.normal(size=shape) + 1j * rng.normal(size=shape))


SHAPES = [(8, 4, 1), (16, 8, 2), (60, 33, 3), (256, 64, 2), (525, 48, 2), (2048, 256, 2)]
# every power-of-two pass structure of the radix-8 row transform (last pass radix 2, 4 or
# 8; 8, 16 values per thread) plus the mixed-radix rows of other 7-smooth lengths: two
# passes (24 = 8 x 3: the first from and the last to global memory only), radix 8 before
# odd radices (72, 1000, 3456), odd radices only (343, 2835)
FFT_SHAPES = SHAPES + [(32, 4, 1), (128, 8, 2), (512, 4, 1), (1024, 8, 1), (4096, 8, 2), (8192, 8, 2),
                       (24, 4, 2), (72, 4, 1), (343, 4, 1), (1000, 8, 2), (2835, 4, 1), (3456, 4, 3)]


# ---------------------------------------------------------------------------- setup (a0)
@pytest.mark.parametrize("Nz,Nr,Nm", SHAPES)
@pytest.mark.parametrize("p", [0, 2, 32])
def test_setup_tables(Nz, Nr, Nm, p):
    s, g = make(Nz, Nr, Nm, p)
    h = O.hankel_setup(g)
    assert rel_err(s.get("KPERP"), np.stack(h.kperp)) < 1e-14
    assert rel_err(s.get("KZ_MOD"), O.modified_kz(g.kz, g.dz, p)) < 1e-13
    binv = s.get("HANKEL_INV")
    mf = s.get("HANKEL_FWD")
    for m in range(Nm):
        for sl in range(3):
            assert np.abs(binv[m, sl] - h.Binv[m][sl]).max() < 1e-13
            assert rel_err(mf[m, sl], h.M[m][sl]) < 1e-12, (m, sl)


# ---------------------------------------------------------------------------- transforms
@pytest.mark.parametrize("Nz,Nr,Nm", FFT_SHAPES)
def test_forward_transform(Nz, Nr, Nm):
    s, g = make(Nz, Nr, Nm)
    h = O.hankel_setup(g)
    rng = np.random.default_rng(Nz + Nr)
    dep = crand(rng, (4, Nm, Nr, Nz))
    s.set("DEP", dep)
    s.forward_transform()
    got = s.get("SRC_H")
    ref = O.forward_sources(g, h, dep[0], dep[1], dep[2], dep[3])
    assert per_slice_err(got, np.stack(ref)) < TOL


@pytest.mark.parametrize("Nz,Nr,Nm", FFT_SHAPES)
def test_inverse_transform(Nz, Nr, Nm):
    s, g = make(Nz, Nr, Nm)
    h = O.hankel_setup(g)
    rng = np.random.default_rng(Nz * Nr)
    Eh, Bh = crand(rng, (3, Nm, Nr, Nz)), crand(rng, (3, Nm, Nr, Nz), 1e-8)
    s.set("EH", Eh)
    s.set("BH", Bh)
    s.inverse_transform()
    E, B = s.get("E"), s.get("B")
    assert per_slice_err(E, np.stack(O.inverse_vector(g, h, *Eh))) < TOL
    assert per_slice_err(B, np.stack(O.inverse_vector(g, h, *Bh))) < TOL


@pytest.mark.parametrize("scale", [1e-30, 1e-20, 1e25])
def test_forward_transform_over_the_double_word_range(scale):
    """The FP64 form's power-of-two z-FFT runs in double words (hi + lo floats): rows whose
    largest value lies between about 2^-100 and 2^127 keep ~48 bits relative to it (the low
    parts reach down to float subnormals), so source grids scaled by 1e-30, 1e-20 and 1e25
    (SI grids of plasma runs lie between) still meet the FP64 parity bar."""
    Nz, Nr, Nm = 256, 16, 2
    s, g = make(Nz, Nr, Nm)
    h = O.hankel_setup(g)
    rng = np.random.default_rng(11)
    dep = crand(rng, (4, Nm, Nr, Nz), scale)
    s.set("DEP", dep)
    s.forward_transform()
    ref = O.forward_sources(g, h, dep[0], dep[1], dep[2], dep[3])
    assert per_slice_err(s.get("SRC_H"), np.stack(ref)) < TOL


def test_ieee_transform_path_matches_the_oracle():
    """pic_set_dht_path(PIC_DHT_F64_GEMM) keeps the FP64 rows and the DHT in IEEE float64
    (the reference arithmetic for rounding-floor studies): same transforms, same bar."""
    Nz, Nr, Nm = 2048, 64, 2
    s, g = make(Nz, Nr, Nm)
    s.set_dht_path(bd.PIC_DHT_F64_GEMM)
    h = O.hankel_setup(g)
    rng = np.random.default_rng(12)
    dep = crand(rng, (4, Nm, Nr, Nz))
    s.set("DEP", dep)
    s.forward_transform()
    ref = O.forward_sources(g, h, dep[0], dep[1], dep[2], dep[3])
    assert per_slice_err(s.get("SRC_H"), np.stack(ref)) < TOL
    Eh = crand(rng, (3, Nm, Nr, Nz))
    s.set("EH", Eh)
    s.inverse_transform()
    assert per_slice_err(s.get("E"), np.stack(O.inverse_vector(g, h, *Eh))) < TOL


# ---------------------------------------------------------------------------- PSATD (a7)
@pytest.mark.parametrize("Nz,Nr,Nm", [(16, 8, 2), (60, 33, 3), (2048, 256, 2)])
@pytest.mark.parametrize("p,filt,cfl", [(0, True, 1.0), (16, False, 0.5), (32, True, 3.0)])
def test_psatd_stage(Nz, Nr, Nm, p, filt, cfl):
    s, g = make(Nz, Nr, Nm, p, filt, cfl=cfl)
    h = O.hankel_setup(g)
    coef = O.psatd_coefficients(g, h, p)
    T = O.source_filter(g, h)
    rng = np.random.default_rng(7 + p)
    sh = (Nm, Nr, Nz)
    E = crand(rng, (3,) + sh, 1e9)
    B = crand(rng, (3,) + sh, 1e9 / O.C_LIGHT)
    src = np.stack([crand(rng, sh, 1e3)] + [crand(rng, sh, 1e3 * O.C_LIGHT) for _ in range(3)])
    rho_prev = crand(rng, sh, 1e3)
    s.set("EH", E)
    s.set("BH", B)
    s.set("SRC_H", src)
    s.set("RHO_PREV_H", rho_prev)
    s.psatd()
    En, Bn, rf, _ = O.psatd_update(g, coef, T, tuple(E), tuple(B), tuple(src[1:]), src[0], rho_prev,
                                   filt=filt, correct=True)
    assert per_slice_err(s.get("EH"), np.stack(En)) < TOL
    assert per_slice_err(s.get("BH"), np.stack(Bn)) < TOL
    assert per_slice_err(s.get("RHO_PREV_H")[None], rf[None]) < TOL


# ---------------------------------------------------------------------------- particles
def _particles(g, n, rng, extra_axis=True):
    r = g.R * 0.999 * np.sqrt(rng.uniform(0, 1, n))
    th = rng.uniform(0, 2 * np.pi, n)
    P = dict(x=r * np.cos(th), y=r * np.sin(th), z=rng.uniform(0, g.L, n),
             ux=rng.normal(0, 3e7, n), uy=rng.normal(0, 3e7, n), uz=rng.normal(1e8, 3e8, n),
             w=rng.uniform(0.5, 2.0, n) * 1e4, id=np.arange(n, dtype=np.int32))
    if extra_axis and n > 10:
        P["x"][:3] = 0.0
        P["y"][:3] = 0.0                      # exactly on the axis
        P["x"][3] = 0.3 * g.dr
        P["y"][3] = -0.1 * g.dr               # inside the first half cell (fold)
        P["z"][4] = np.nextafter(g.L, 0)      # last representable z
        P["z"][5] = 0.0
        P["x"][6], P["y"][6] = (g.R - 1e-3 * g.dr), 0.0
    return P


@pytest.mark.parametrize("Nz,Nr,n", [(16, 8, 1), (16, 8, 1000), (60, 33, 4097), (256, 64, 36384),
                                     (2048, 256, 300000)])
def test_sort_bit_exact(Nz, Nr, n):
    s, g = make(Nz, Nr, 1, cap=n)
    rng = np.random.default_rng(n)
    P = _particles(g, n, rng)
    if n >= 1000:   # a crowded cell (> 16 particles) exercises the warp path
        k = min(400, n // 3)
        P["x"][-k:] = 0.5 * g.dr
        P["y"][-k:] = 0.5 * g.dr
        P["z"][-k:] = 2.5 * g.dz
    s.write_particles(P)
    s.sort()
    keys = O.cell_keys(g, P["x"], P["y"], P["z"])
    perm = O.sort_permutation(keys)
    assert np.array_equal(s.get("KEYS"), keys)
    assert np.array_equal(s.get("PERM"), perm)
    got = s.read_particles()
    for k in bd.SOA + ("id",):
        assert np.array_equal(got[k], P[k][perm]), k


@pytest.mark.parametrize("Nz,Nr,Nm,n", [(16, 8, 3, 500), (60, 33, 2, 3000), (256, 64, 2, 36384)])
def test_deposit(Nz, Nr, Nm, n):
    s, g = make(Nz, Nr, Nm, cap=n)
    rng = np.random.default_rng(11)
    P = _particles(g, n, rng)
    s.write_particles(P)
    s.deposit(bd.PIC_DEP_RHO | bd.PIC_DEP_J)
    dep = s.get("DEP")
    q = O.Q_E * -1
    rho = O.deposit_rho(g, P["x"], P["y"], P["z"], P["w"], q)
    ig = O.inv_gamma(P["ux"], P["uy"], P["uz"])
    J = O.deposit_current(g, P["x"], P["y"], P["z"], P["ux"] * ig, P["uy"] * ig, P["uz"] * ig, P["w"], q)
    assert per_slice_err(dep[0:1], rho[None]) < TOL
    assert per_slice_err(dep[1:], np.stack(J)) < TOL


@pytest.mark.parametrize("Nz,Nr,Nm,n", [(16, 8, 3, 700), (256, 64, 2, 36384)])
def test_gather_push(Nz, Nr, Nm, n):
    s, g = make(Nz, Nr, Nm, cap=n)
    rng = np.random.default_rng(13)
    P = _particles(g, n, rng)
    E = crand(rng, (3, Nm, Nr, Nz), 1e10)
    B = crand(rng, (3, Nm, Nr, Nz), 1e10 / O.C_LIGHT)
    s.write_particles(P)
    s.set("E", E)
    s.set("B", B)
    s.gather_push(fuse_current=True)
    zero = np.zeros((Nm, Nr, Nz), complex)
    st = O.State(g, 0, False, -O.Q_E, O.M_E, None, None, None, tuple(E), tuple(B), None, None,
                 zero, zero, {k: v.copy() for k, v in P.items()})
    J = O.gather_push(st)
    got = s.read_particles()
    for k in bd.SOA:
        assert rel_err(got[k], st.p[k]) < TOL, k
    assert per_slice_err(s.get("DEP")[1:], np.stack(J)) < TOL


@pytest.mark.parametrize("Nz,Nr,Nm,n", [(64, 33, 2, 6000), (256, 64, 3, 36384)])
def test_gather_push_from_rest(Nz, Nr, Nm, n):
    """Particles at rest: the momentum after one push is the gathered field itself (2 k E to
    first order), so the gather's arithmetic is measured at full scale, not against the
    momentum a particle already has.  A third of the particles sit in the axis cell (ghost
    node fold).  The FP64 form gathers from the double-word copy of E, B (products and sums
    on the float32 units, error a few 2^-48 of the summed terms); the IEEE path
    (PIC_DHT_F64_GEMM) gathers from the float64 grids: both against the oracle, and against
    each other."""
    rng = np.random.default_rng(29)
    g = O.Grid(Nz, Nr, Nm, DZ, DZ, DZ / O.C_LIGHT)
    P = _particles(g, n, rng)
    k0 = n // 3
    r = g.dr * rng.uniform(0, 1, k0)
    th = rng.uniform(0, 2 * np.pi, k0)
    P["x"][10:10 + k0] = r * np.cos(th)
    P["y"][10:10 + k0] = r * np.sin(th)
    for k in ("ux", "uy", "uz"):
        P[k][:] = 0.0
    E = crand(rng, (3, Nm, Nr, Nz), 1e12)
    B = crand(rng, (3, Nm, Nr, Nz), 1e12 / O.C_LIGHT)
    zero = np.zeros((Nm, Nr, Nz), complex)
    st = O.State(g, 0, False, -O.Q_E, O.M_E, None, None, None, tuple(E), tuple(B), None, None,
                 zero, zero, {k: v.copy() for k, v in P.items()})
    O.gather_push(st)
    got = {}
    for path in (bd.PIC_DHT_AUTO, bd.PIC_DHT_F64_GEMM):
        s, _ = make(Nz, Nr, Nm, cap=n)
        s.set_dht_path(path)
        s.write_particles(P)
        s.set("E", E)
        s.set("B", B)
        s.gather_push(fuse_current=True)
        got[path] = s.read_particles()
        for k in ("ux", "uy", "uz", "x", "y", "z"):
            assert rel_err(got[path][k], st.p[k]) < TOL, (path, k)
    for k in ("ux", "uy", "uz"):
        assert rel_err(got[bd.PIC_DHT_AUTO][k], got[bd.PIC_DHT_F64_GEMM][k]) < 1e-13, k


# ---------------------------------------------------------------------------- full cycle
def _compare_state(s, st, tol):
    """Physical states are compared per field (all components and modes share one scale):
    components that vanish physically (E_theta of mode 0 for a cold symmetric beam) hold
    only rounding noise from E_theta = i(E_+ - E_-), and higher modes of a nearly
    symmetric beam are residuals of cancelling sums taken in a different order (atomics
    vs bincount), so a per-component scale would measure noise, not the arithmetic."""
    assert rel_err(s.get("E"), np.stack(st.E)) < tol
    assert rel_err(s.get("B"), np.stack(st.B)) < tol
    assert rel_err(s.get("EH"), np.stack(st.Eh)) < tol
    assert rel_err(s.get("BH"), np.stack(st.Bh)) < tol
    assert rel_err(s.get("RHO_PREV_H"), st.rho_prev_h) < tol
    got, ref = by_id(s.read_particles()), by_id(st.p)
    assert np.array_equal(got["id"], ref["id"])
    for k in bd.SOA:
        assert rel_err(got[k], ref[k]) < tol, k


def test_full_cycle_plasma_beam_256x64():
    w = W.plasma_beam_small()
    P, npl, beams = W.particles(w)
    g = O.Grid(w.Nz, w.Nr, w.Nm, w.dz, w.dr, w.dt)
    s = bd.Sim.from_workload(w, P, npl, beams)
    st = O.make_state(g, w.order_p, True, P, npl, beams)
    assert rel_err(s.get("RHO_ION"), st.rho_ion) < TOL
    _compare_state(s, st, TOL)
    s.step(1)
    O.pic_step(st, 1)
    _compare_state(s, st, TOL)
    s.step(4)
    O.pic_step(st, 4)
    _compare_state(s, st, 1e-10)
    d = s.diagnostics(npl, npl + beams[0][1] - beams[0][0])
    sel = (st.p["id"] >= npl)
    od = O.beam_diagnostics(*(st.p[k][sel] for k in bd.SOA))
    for k in ("W", "z_mean", "sigma_z", "gamma_mean", "emit_nx", "emit_ny", "sigma_gamma_mean"):
        assert d[k] == pytest.approx(od[k], rel=1e-9, abs=1e-300), k
    assert np.allclose(d["slice_sigma_gamma"], od["slice_sigma_gamma"], rtol=1e-9)


@pytest.mark.parametrize("order_p", [32, 0])
def test_full_cycle_wake_2048x256(order_p):
    """The 2048 x 256, 2-mode wakefield workload (1.35M particles), one step, both orders."""
    w = W.wake_2048x256(order_p=order_p)
    P, npl, beams = W.particles(w)
    g = O.Grid(w.Nz, w.Nr, w.Nm, w.dz, w.dr, w.dt)
    s = bd.Sim.from_workload(w, P, npl, beams)
    st = O.make_state(g, order_p, True, P, npl, beams)
    s.step(1)
    O.pic_step(st, 1)
    _compare_state(s, st, TOL)


def test_order_switch_rebuilds_tables():
    s, g = make(64, 16, 2, p=0)
    h = O.hankel_setup(g)
    rng = np.random.default_rng(3)
    sh = (2, 16, 64)
    E, B = crand(rng, (3,) + sh), crand(rng, (3,) + sh, 1e-8)
    for p in (8, 0, 64):
        s.set("EH", E)
        s.set("BH", B)
        s.set("DEP", np.zeros((4,) + sh))
        s.set("RHO_PREV_H", np.zeros(sh))
        s.field_step(p)
        coef = O.psatd_coefficients(g, h, p)
        z = np.zeros(sh, complex)
        En, Bn, _, _ = O.psatd_update(g, coef, O.source_filter(g, h), tuple(E), tuple(B), (z, z, z), z, z)
        assert per_slice_err(s.get("EH"), np.stack(En)) < TOL
        assert rel_err(s.get("KZ_MOD"), O.modified_kz(g.kz, g.dz, p)) < 1e-13


def test_empty_particle_set_steps():
    s, g = make(32, 8, 2, cap=16)
    s.write_particles({k: np.zeros(0) for k in bd.SOA} | {"id": np.zeros(0, np.int32)})
    s.init_background(0)
    s.init_fields()
    s.step(2)
    s.sync()
    assert np.abs(s.get("E")).max() == 0.0


def test_invalid_state_and_arguments():
    s, g = make(32, 8, 2, cap=4)
    with pytest.raises(bd.PicError) as e:
        s.step(1)
    assert e.value.status == 6
    with pytest.raises(bd.PicError):
        s.write_particles({k: np.zeros(5) for k in bd.SOA} | {"id": np.zeros(5, np.int32)})
    with pytest.raises(bd.PicError):
        s.field_step(3)
