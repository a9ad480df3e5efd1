"""Failure detection on the GPU without a GPU fault: a bounded mbarrier wait that nothing
completes (the same wait the tensor-core kernels use) runs out, raises the timeout bit of
the device error word and returns; the host reads PIC_ERR_TIMEOUT, the word stays set
until cleared, and the handle then steps normally."""
import numpy as np
import pytest

from paper_1611_05712_gb300 import binding as bd
from paper_1611_05712_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1611_05712_gb300.build import build
    build()


@pytest.mark.parametrize("precision", [bd.PIC_FP64, bd.PIC_MIXED_TF32X3])
def test_bounded_wait_times_out_and_the_handle_recovers(precision):
    w = W.tiny(order_p=8, Nz=32, Nr=8, Nm=2, n_beam=64)
    P, npl, beams = W.particles(w)
    s = bd.Sim.from_workload(w, P, npl, beams, precision=precision)
    s.selftest_wait_timeout(4096)
    with pytest.raises(bd.PicError) as e:
        s.sync()
    assert e.value.status == 4   # PIC_ERR_TIMEOUT
    with pytest.raises(bd.PicError):
        s.sync()                 # sticky until cleared
    s.clear_error()
    s.sync()
    s.step(2)
    s.sync()
    assert np.isfinite(s.get("E")).all()


def test_selftest_rejects_bad_poll_counts():
    w = W.tiny(order_p=8, Nz=16, Nr=8, Nm=1, n_beam=8)
    P, npl, beams = W.particles(w)
    s = bd.Sim.from_workload(w, P, npl, beams)
    for n in (0, -1, (1 << 24) + 1):
        with pytest.raises(bd.PicError):
            s.selftest_wait_timeout(n)
