"""The allocation-free sort entry point against the workspace-based one.

pic_sort_keys_noalloc serves callers that cannot allocate device memory when they need
the sort (inside a step being captured into a CUDA graph, or under a fixed memory budget):
its scratch is a fixed array inside the library.  Here it must give the same cell keys
and the same stable permutation, bit for bit, as pic_sort through a pic_sim handle, on
two calls in a row (the second on a different grid and particle set, so stale scratch
contents from the first call would show), and reject sizes beyond its limits.
"""
import ctypes

import numpy as np
import pytest

from paper_1611_05712_gb300 import binding as bd

pytestmark = pytest.mark.gpu

DZ = 0.05e-6


def _lib():
    from paper_1611_05712_gb300.build import build
    build()
    lib = bd.load()
    P = ctypes.c_void_p
    f = lib.pic_sort_keys_noalloc
    f.argtypes = [P, P, P, ctypes.c_int64, ctypes.c_int32, ctypes.c_int32, ctypes.c_double,
                  ctypes.c_double, P, P, P]
    f.restype = ctypes.c_int
    return lib


def _particles(Nz, Nr, n, seed):
    rng = np.random.default_rng(seed)
    R, L = Nr * DZ, Nz * DZ
    r = 0.999 * R * np.sqrt(rng.uniform(0, 1, n))
    th = rng.uniform(0, 2 * np.pi, n)
    P = dict(x=r * np.cos(th), y=r * np.sin(th), z=rng.uniform(0, L, n),
             ux=np.zeros(n), uy=np.zeros(n), uz=np.zeros(n), w=np.ones(n),
             id=np.arange(n, dtype=np.int32))
    k = n // 5                                   # one crowded cell
    P["x"][:k], P["y"][:k], P["z"][:k] = 0.5 * DZ, 0.2 * DZ, 1.5 * DZ
    P["x"][k:k + 3], P["y"][k:k + 3] = 0.0, 0.0  # on the axis
    return P


@pytest.mark.parametrize("case", [((128, 64, 20000, 1), (48, 24, 5003, 2))])
def test_noalloc_sort_matches_workspace_sort_twice(case):
    import torch
    lib = _lib()
    dev = torch.device("cuda:0")
    stream = torch.cuda.current_stream(dev)
    for Nz, Nr, n, seed in case:
        P = _particles(Nz, Nr, n, seed)
        cfg = bd.make_config(Nz, Nr, 1, DZ, DZ, DZ / 3e8, 0, True, bd.PIC_FP64, n)
        s = bd.Sim(cfg)
        s.write_particles(P)
        s.sort()
        keys_ref, perm_ref = s.get("KEYS"), s.get("PERM")
        x, y, z = (torch.from_numpy(P[k]).to(dev) for k in ("x", "y", "z"))
        keys = torch.full((n,), -7, dtype=torch.int32, device=dev)
        perm = torch.full((n,), -7, dtype=torch.int32, device=dev)
        st = lib.pic_sort_keys_noalloc(x.data_ptr(), y.data_ptr(), z.data_ptr(), n, Nz, Nr, DZ, DZ,
                                       keys.data_ptr(), perm.data_ptr(), stream.cuda_stream)
        assert st == 0, lib.pic_last_error().decode()
        torch.cuda.synchronize(dev)
        assert np.array_equal(keys.cpu().numpy(), keys_ref)
        assert np.array_equal(perm.cpu().numpy(), perm_ref)
        s.close()


def test_noalloc_sort_rejects_sizes_beyond_its_limits():
    lib = _lib()
    dummy = ctypes.c_void_p(16)
    st = lib.pic_sort_keys_noalloc(dummy, dummy, dummy, 262145, 16, 16, DZ, DZ, dummy, dummy, None)
    assert st == 1 and "262144" in lib.pic_last_error().decode()
    st = lib.pic_sort_keys_noalloc(dummy, dummy, dummy, 10, 512, 256, DZ, DZ, dummy, dummy, None)
    assert st == 1 and "65536" in lib.pic_last_error().decode()
