"""CPU-side checks of the C-ABI library: it builds for sm_103a, loads, exports every
function include/psatd_rz.h declares, and rejects invalid configurations (host-only
validation, no kernel runs)."""
import ctypes
import shutil

import pytest

from paper_1611_05712_gb300 import binding as bd


@pytest.fixture(scope="module")
def lib():
    if shutil.which("nvcc") is None and not __import__("os").path.exists("/usr/local/cuda/bin/nvcc"):
        pytest.skip("nvcc not available")
    from paper_1611_05712_gb300.build import build
    build()
    return bd.load()


def test_exports_every_declared_function(lib):
    names = bd.declared_functions()
    assert len(names) >= 20
    for n in names:
        assert hasattr(lib, n), n


def test_required_bytes_and_validation(lib):
    cfg = bd.make_config(256, 64, 2, 5e-8, 5e-8, 1e-16, 0, True, bd.PIC_FP64, 1000)
    n = bd.required_bytes(cfg)
    assert n > 256 * 64 * 2 * 16 * 30
    bad = [
        dict(Nz=11), dict(Nz=4), dict(Nz=8192), dict(Nr=2), dict(Nr=2048), dict(Nm=0), dict(Nm=5),
        dict(order_p=3), dict(order_p=-2), dict(order_p=1024), dict(dt=0.0), dict(np_capacity=-1),
        dict(precision=7),
    ]
    for b in bad:
        c = bd.make_config(256, 64, 2, 5e-8, 5e-8, 1e-16, 0, True, bd.PIC_FP64, 1000)
        for k, v in b.items():
            setattr(c, k, v)
        out = ctypes.c_size_t()
        st = lib.pic_required_bytes(ctypes.byref(c), ctypes.byref(out))
        assert st == 1, b
        assert lib.pic_last_error().decode() != ""


def test_seven_smooth_lengths_accepted(lib):
    for nz in (8, 12, 60, 210, 343, 525, 2048, 4096, 3000):
        c = bd.make_config(nz, 16, 1, 5e-8, 5e-8, 1e-16, 0, True, bd.PIC_FP64, 10)
        out = ctypes.c_size_t()
        assert lib.pic_required_bytes(ctypes.byref(c), ctypes.byref(out)) == 0, nz


def test_null_handles_rejected(lib):
    assert lib.pic_sort(None) == 1
    assert lib.pic_step(None, 1) == 1
    assert lib.pic_init(None, None, 0, None, None) == 1
