"""Guard-cell domain decomposition along z on one GPU (section "Finite order
pseudo-spectral solvers", unit-pulse figure; "Conclusion": about 60 guard cells at p = 32).

Four z subdomains, each advanced with its own Fourier transform over its interior plus g
guard cells per side: element by element against the oracle's decomposed step
(``field_step_guarded``) for several orders and guard widths, the small widths with their
spurious fields included; and against the global field step of the same fields (FP64, no
sources).  At p = 32 the interiors agree with the global update to rounding once g
reaches the stencil's extent and differ by spurious fields when g is small; at infinite
order (PSATD) no number of guard cells reaches rounding level.
"""
import numpy as np
import pytest

from oracle import psatd_rz as O
from paper_1611_05712_gb300 import binding as bd
from paper_1611_05712_gb300.domains import GuardedDomains
from gpu_helpers import rel_err

pytestmark = pytest.mark.gpu

DZ = 0.05e-6
NZ, NR, NM = 512, 32, 2


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1611_05712_gb300.build import build
    build()


def _fields(seed):
    rng = np.random.default_rng(seed)
    shape = (3, NM, NR, NZ)
    E = rng.normal(size=shape) + 1j * rng.normal(size=shape)
    B = (rng.normal(size=shape) + 1j * rng.normal(size=shape)) / O.C_LIGHT
    return E, B


@pytest.mark.parametrize("p,guard", [(8, 4), (8, 32), (16, 8), (16, 48), (32, 8), (32, 24), (32, 64),
                                     (64, 16), (64, 96), (0, 64)])
def test_decomposed_step_matches_the_oracle_decomposition(p, guard):
    cfg = bd.make_config(NZ, NR, NM, DZ, DZ, DZ / O.C_LIGHT, p, True, bd.PIC_FP64, 0)
    src, out = bd.Sim(cfg), bd.Sim(cfg)
    E, B = _fields(11)
    src.set("E", E)
    src.set("B", B)
    for h in (src, out):
        h.set("DEP", h.zeros("DEP"))
        h.set("RHO_PREV_H", h.zeros("RHO_PREV_H"))
    dom = GuardedDomains(cfg, 4, guard)
    dom.field_step(src, out)
    g = O.Grid(NZ, NR, NM, DZ, DZ, DZ / O.C_LIGHT)
    Eo, Bo = O.field_step_guarded(g, p, tuple(E), tuple(B), 4, guard)
    assert rel_err(out.get("E"), np.stack(Eo)) < 1e-12
    assert rel_err(out.get("B"), np.stack(Bo)) < 1e-12
    dom.close()
    src.close()
    out.close()


def decomposition_error(p, guard, n_domains=4, seed=7):
    """Decomposed against global step on the GPU.  All handles use the FP64 SIMT DHT, whose
    rounding floor (~1e-15) lets the locality of the stencil show down to FP64 rounding; the
    sliced tensor-core DHT agrees with the FP64 product to ~1e-13 only."""
    cfg = bd.make_config(NZ, NR, NM, DZ, DZ, DZ / O.C_LIGHT, p, True, bd.PIC_FP64, 0)
    glob, out = bd.Sim(cfg), bd.Sim(cfg)
    for h in (glob, out):
        h.set_dht_path(bd.PIC_DHT_F64_GEMM)
    rng = np.random.default_rng(seed)
    shape = (3, NM, NR, NZ)
    glob.set("E", rng.normal(size=shape) + 1j * rng.normal(size=shape))
    glob.set("B", (rng.normal(size=shape) + 1j * rng.normal(size=shape)) / O.C_LIGHT)
    for h in (glob, out):
        h.set("DEP", h.zeros("DEP"))
        h.set("RHO_PREV_H", h.zeros("RHO_PREV_H"))
    dom = GuardedDomains(cfg, n_domains, guard, dht_path=bd.PIC_DHT_F64_GEMM)
    dom.field_step(glob, out)
    glob.fields_to_spectral()
    glob.field_step()
    err = max(rel_err(out.get("E"), glob.get("E")), rel_err(out.get("B"), glob.get("B")))
    dom.close()
    glob.close()
    out.close()
    return err


def test_one_domain_without_guards_is_the_global_step():
    assert decomposition_error(32, 0, n_domains=1) < 1e-14


def test_order_32_reaches_rounding_with_enough_guard_cells():
    # 64 guard cells (the paper: about 60 at p = 32): FP64 rounding of one field step
    assert decomposition_error(32, 64) < 1e-14


def test_order_32_with_few_guard_cells_has_spurious_fields():
    assert decomposition_error(32, 8) > 1e-6


def test_error_falls_with_guard_width_at_order_32():
    errs = [decomposition_error(32, g) for g in (8, 16, 32, 64)]
    assert all(b < a for a, b in zip(errs, errs[1:])), errs


def test_infinite_order_is_not_local():
    assert decomposition_error(0, 96) > 1e-8
