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
        dict(Nz=2053), dict(Nz=4), dict(Nz=16384), dict(Nz=6000), dict(Nr=2), dict(Nr=2048), dict(Nm=0), dict(Nm=5),
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
    # float64 rows: powers of two up to 8192, other 7-smooth lengths up to 4096
    for nz in (8, 12, 60, 210, 343, 525, 2048, 4096, 3000, 8192):
        c = bd.make_config(nz, 16, 1, 5e-8, 5e-8, 1e-16, 0, True, bd.PIC_FP64, 10)
        out = ctypes.c_size_t()
        assert lib.pic_required_bytes(ctypes.byref(c), ctypes.byref(out)) == 0, nz


def test_non_smooth_lengths_within_the_bluestein_limit(lib):
    # lengths that are not 7-smooth use power-of-two Bluestein rows of M >= 2 Nz - 1, at most
    # 4096 (FP64) or 8192 (mixed forms)
    cases = [(11, bd.PIC_FP64, 0), (61, bd.PIC_FP64, 0), (2039, bd.PIC_FP64, 0), (2053, bd.PIC_FP64, 1),
             (4093, bd.PIC_FP64, 1), (4093, bd.PIC_MIXED_TF32X3, 0), (4093, bd.PIC_MIXED_BF16X6, 0),
             (4111, bd.PIC_MIXED_TF32X3, 1), (22, bd.PIC_MIXED_TF32X3, 0)]
    for nz, prec, want in cases:
        c = bd.make_config(nz, 16, 1, 5e-8, 5e-8, 1e-16, 0, True, prec, 10)
        out = ctypes.c_size_t()
        assert lib.pic_required_bytes(ctypes.byref(c), ctypes.byref(out)) == want, (nz, prec)


def test_null_handles_rejected(lib):
    assert lib.pic_sort(None) == 1
    assert lib.pic_step(None, 1) == 1
    assert lib.pic_init(None, None, 0, None, None) == 1


def test_stage_bytes_host_only(lib):
    # 7 float64 arrays and the int32 ids, each padded to a multiple of 32 elements
    out = ctypes.c_size_t()
    for n, padded in ((0, 0), (1, 32), (32, 32), (33, 64), (1348576, 1348576)):
        assert lib.pic_stage_bytes(n, ctypes.byref(out)) == 0
        assert out.value == padded * (7 * 8 + 4), n
    assert lib.pic_stage_bytes(-1, ctypes.byref(out)) == 1
    assert lib.pic_stage_bytes(4, None) == 1
    assert lib.pic_stage_particles(None, None, None, 0, None, 0) == 1
    assert lib.pic_take_particles(None) == 1
