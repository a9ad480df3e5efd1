"""The order study on the GPU (section "Accurate modeling of plasma accelerators in
finite order PSATD"): the plasma + beam case advanced 200 cycles at several stencil orders
from one initial state; the numerical-Cherenkov measures against the infinite-order run
(Eq. err-metrics) fall as the order grows (FP64 form)."""
import pytest

from paper_1611_05712_gb300 import binding as bd
from paper_1611_05712_gb300 import ncr
from paper_1611_05712_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1611_05712_gb300.build import build
    build()


def test_ncr_errors_fall_with_stencil_order():
    w = W.plasma_beam_small()
    P, npl, beams = W.particles(w)
    lo, hi = beams[0][0], beams[0][1]
    runs = {}
    for p in (0, 4, 16, 64):
        s = bd.Sim.from_workload(w, P, npl, beams, order_p=p)
        s.step(200)
        runs[p] = (s.diagnostics(lo, hi), ncr.ez_plane(s.get("E")))
        s.close()
    ref_d, ref_ez = runs[0]
    e_ez = [ncr.err_ez_l2(runs[p][1], ref_ez) for p in (4, 16, 64)]
    e_sg = [ncr.err_sigma_gamma(runs[p][0]["slice_sigma_gamma"], ref_d["slice_sigma_gamma"]) for p in (4, 16, 64)]
    assert e_ez[0] > e_ez[1] > e_ez[2], e_ez
    assert e_sg[0] > e_sg[2], e_sg
