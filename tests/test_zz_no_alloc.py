"""The allocation-free sort entry point against the workspace-based one and the oracle.

pic_sort_keys_noalloc serves callers that cannot allocate device memory when they need
the sort (a fixed memory budget handed over at start-up, or a host allocator that owns
the device): its scratch is a fixed array inside the library.  Here it must give the
same cell keys and the same stable permutation, bit for bit, as pic_sort through a
pic_sim handle and as the oracle's cell keys and stable sort, on two calls in a row (the
second on a different grid and particle set, so stale scratch contents from the first
call would show); order a cell that holds every particle in bounded time; replay from a
captured CUDA graph; and reject sizes beyond its limits.
"""
import ctypes

import numpy as np
import pytest

from oracle import psatd_rz as O
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


def _particles(Nz, Nr, n, seed, crowded=5):
    rng = np.random.default_rng(seed)
    R, L = Nr * DZ, Nz * DZ
    r = 0.999 * R * np.sqrt(rng.uniform(0, 1, n))
    th = rng.uniform(0, 2 * np.pi, n)
    P = dict(x=r * np.cos(th), y=r * np.sin(th), z=rng.uniform(0, L, n),
             ux=np.zeros(n), uy=np.zeros(n), uz=np.zeros(n), w=np.ones(n),
             id=np.arange(n, dtype=np.int32))
    k = n // crowded                             # one crowded cell, scattered over the indices
    sel = rng.permutation(n)[:k]
    P["x"][sel], P["y"][sel], P["z"][sel] = 0.5 * DZ, 0.2 * DZ, 1.5 * DZ
    P["x"][sel[:3]], P["y"][sel[:3]] = 0.0, 0.0  # on the axis
    return P


def _noalloc(lib, P, Nz, Nr, stream):
    import torch
    dev = torch.device("cuda:0")
    n = len(P["x"])
    x, y, z = (torch.from_numpy(P[k]).to(dev) for k in ("x", "y", "z"))
    keys = torch.full((n,), -7, dtype=torch.int32, device=dev)
    perm = torch.full((n,), -7, dtype=torch.int32, device=dev)
    st = lib.pic_sort_keys_noalloc(x.data_ptr(), y.data_ptr(), z.data_ptr(), n, Nz, Nr, DZ, DZ,
                                   keys.data_ptr(), perm.data_ptr(), stream.cuda_stream)
    assert st == 0, lib.pic_last_error().decode()
    torch.cuda.synchronize(dev)
    return keys.cpu().numpy(), perm.cpu().numpy()


@pytest.mark.parametrize("case", [((128, 64, 20000, 1), (48, 24, 5003, 2))])
def test_noalloc_sort_matches_workspace_sort_twice(case):
    import torch
    lib = _lib()
    stream = torch.cuda.current_stream(torch.device("cuda:0"))
    for Nz, Nr, n, seed in case:
        P = _particles(Nz, Nr, n, seed)
        cfg = bd.make_config(Nz, Nr, 1, DZ, DZ, DZ / 3e8, 0, True, bd.PIC_FP64, n)
        s = bd.Sim(cfg)
        s.write_particles(P)
        s.sort()
        keys_ref, perm_ref = s.get("KEYS"), s.get("PERM")
        s.close()
        keys, perm = _noalloc(lib, P, Nz, Nr, stream)
        assert np.array_equal(keys, keys_ref)
        assert np.array_equal(perm, perm_ref)
        g = O.Grid(Nz, Nr, 1, DZ, DZ, DZ / O.C_LIGHT)
        okeys = O.cell_keys(g, P["x"], P["y"], P["z"])
        assert np.array_equal(keys, okeys)
        assert np.array_equal(perm, O.sort_permutation(okeys))


def test_noalloc_sort_of_one_cell_holding_every_particle_is_bounded():
    """All n = 262144 particles (the limit) in one cell: the ordering of that cell is an
    O(n log n) CTA sort, so the call stays in milliseconds; the permutation is the
    identity (stable order of equal keys)."""
    import torch
    lib = _lib()
    dev = torch.device("cuda:0")
    stream = torch.cuda.current_stream(dev)
    n, Nz, Nr = 262144, 64, 32
    P = dict(x=np.full(n, 3.3 * DZ), y=np.full(n, 1.1 * DZ), z=np.full(n, 7.5 * DZ))
    keys, perm = _noalloc(lib, P, Nz, Nr, stream)       # warm-up (and first-call set-up)
    assert np.array_equal(perm, np.arange(n, dtype=np.int32))
    g = O.Grid(Nz, Nr, 1, DZ, DZ, DZ / O.C_LIGHT)
    assert np.array_equal(keys, O.cell_keys(g, P["x"][:1], P["y"][:1], P["z"][:1]).repeat(n))
    # reversed arrival order in the scatter is likely; time the call on the device
    x, y, z = (torch.from_numpy(P[k]).to(dev) for k in ("x", "y", "z"))
    kt = torch.empty(n, dtype=torch.int32, device=dev)
    pt = torch.empty(n, dtype=torch.int32, device=dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    st = lib.pic_sort_keys_noalloc(x.data_ptr(), y.data_ptr(), z.data_ptr(), n, Nz, Nr, DZ, DZ,
                                   kt.data_ptr(), pt.data_ptr(), stream.cuda_stream)
    e1.record(stream)
    torch.cuda.synchronize(dev)
    assert st == 0
    ms = e0.elapsed_time(e1)
    assert ms < 200.0, ms
    assert np.array_equal(pt.cpu().numpy(), np.arange(n, dtype=np.int32))


def test_noalloc_sort_replays_from_a_captured_graph():
    """The call only enqueues kernels on its stream once the first call has looked up its
    scratch array, so it can be captured into a CUDA graph: captured on one particle set,
    then replayed after a second set is written into the same input buffers, the graph
    gives the keys and permutation that pic_sort gives for the second set, bit for bit."""
    import torch
    lib = _lib()
    dev = torch.device("cuda:0")
    Nz, Nr, n = 128, 64, 20000
    P0, P1 = _particles(Nz, Nr, n, 3), _particles(Nz, Nr, n, 4)
    bufs = {k: torch.from_numpy(P0[k]).to(dev) for k in ("x", "y", "z")}
    keys = torch.full((n,), -7, dtype=torch.int32, device=dev)
    perm = torch.full((n,), -7, dtype=torch.int32, device=dev)
    side = torch.cuda.Stream(dev)

    def call(stream):
        return lib.pic_sort_keys_noalloc(bufs["x"].data_ptr(), bufs["y"].data_ptr(), bufs["z"].data_ptr(), n,
                                         Nz, Nr, DZ, DZ, keys.data_ptr(), perm.data_ptr(), stream.cuda_stream)

    side.wait_stream(torch.cuda.current_stream(dev))
    with torch.cuda.stream(side):
        assert call(side) == 0   # outside the capture: the scratch address lookup
    torch.cuda.synchronize(dev)
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=side):
        st = call(torch.cuda.current_stream(dev))
    assert st == 0, lib.pic_last_error().decode()
    for k in ("x", "y", "z"):
        bufs[k].copy_(torch.from_numpy(P1[k]))
    torch.cuda.synchronize(dev)
    graph.replay()
    torch.cuda.synchronize(dev)
    cfg = bd.make_config(Nz, Nr, 1, DZ, DZ, DZ / 3e8, 0, True, bd.PIC_FP64, n)
    s = bd.Sim(cfg)
    s.write_particles(P1)
    s.sort()
    keys_ref, perm_ref = s.get("KEYS"), s.get("PERM")
    s.close()
    assert np.array_equal(keys.cpu().numpy(), keys_ref)
    assert np.array_equal(perm.cpu().numpy(), perm_ref)


def test_noalloc_sort_rejects_sizes_beyond_its_limits():
    """Oversized calls are refused before any launch; the buffers are real and sized
    for each call, so a regression in the checks would write memory the test owns."""
    import torch
    lib = _lib()
    dev = torch.device("cuda:0")
    for n, Nz, Nr, what in ((262145, 16, 16, "262144"), (10, 512, 256, "65536")):
        x, y, z = (torch.zeros(n, dtype=torch.float64, device=dev) for _ in range(3))
        keys = torch.zeros(n, dtype=torch.int32, device=dev)
        perm = torch.zeros(n, dtype=torch.int32, device=dev)
        st = lib.pic_sort_keys_noalloc(x.data_ptr(), y.data_ptr(), z.data_ptr(), n, Nz, Nr, DZ, DZ,
                                       keys.data_ptr(), perm.data_ptr(), None)
        assert st == 1 and what in lib.pic_last_error().decode()
        torch.cuda.synchronize(dev)
        assert int(keys.abs().sum()) == 0 and int(perm.abs().sum()) == 0
