"""ctypes binding of libpsatd_rz.so (include/psatd_rz.h).

Argument marshalling only: every stage of the PIC cycle runs in the library's CUDA
kernels.  PyTorch provides the device workspace and the stream.  There is no CPU
fallback; a missing library raises ``RuntimeError``.
"""
from __future__ import annotations

import ctypes
import os
import re

import numpy as np

PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(PKG, "lib", "libpsatd_rz.so")
HEADER = os.path.join(os.path.dirname(PKG), "include", "psatd_rz.h")

PIC_FP64, PIC_MIXED_TF32X3, PIC_MIXED_BF16X6 = 0, 1, 2
PIC_DEP_RHO, PIC_DEP_J = 1, 2
PIC_DHT_AUTO, PIC_DHT_F64_GEMM, PIC_DHT_F64_SLICED = 0, 1, 2
BUF = dict(E=0, B=1, EH=2, BH=3, DEP=4, SRC_H=5, RHO_PREV_H=6, RHO_ION=7, KPERP=8,
           HANKEL_INV=9, HANKEL_FWD=10, KZ_MOD=11, KEYS=12, PERM=13)
STATUS = {0: "PIC_OK", 1: "PIC_ERR_ARG", 2: "PIC_ERR_CUDA", 3: "PIC_ERR_OOM",
          4: "PIC_ERR_TIMEOUT", 5: "PIC_ERR_NUMERIC", 6: "PIC_ERR_STATE"}
SOA = ("x", "y", "z", "ux", "uy", "uz", "w")
STAGES = ("gather_layout", "gather_push", "sort", "deposit", "fft_fwd", "dht_fwd", "psatd", "dht_inv", "fft_inv")


class PicConfig(ctypes.Structure):
    _fields_ = [("Nz", ctypes.c_int32), ("Nr", ctypes.c_int32), ("Nm", ctypes.c_int32),
                ("order_p", ctypes.c_int32), ("dz", ctypes.c_double), ("dr", ctypes.c_double),
                ("dt", ctypes.c_double), ("filter", ctypes.c_int32), ("precision", ctypes.c_int32),
                ("np_capacity", ctypes.c_int64), ("q", ctypes.c_double), ("mass", ctypes.c_double)]


class PicDiag(ctypes.Structure):
    _fields_ = [("W", ctypes.c_double), ("x_mean", ctypes.c_double), ("y_mean", ctypes.c_double),
                ("z_mean", ctypes.c_double), ("sigma_z", ctypes.c_double),
                ("gamma_mean", ctypes.c_double), ("emit_nx", ctypes.c_double),
                ("emit_ny", ctypes.c_double), ("sigma_gamma_mean", ctypes.c_double),
                ("n_slices", ctypes.c_int32), ("n_particles", ctypes.c_int32)]


class PicTuning(ctypes.Structure):
    _fields_ = [("dht_n_tile", ctypes.c_int32), ("band_chunk", ctypes.c_int32),
                ("dht_ms", ctypes.c_double), ("deposit_ms", ctypes.c_double)]


class PicWindowInfo(ctypes.Structure):
    _fields_ = [("cycles", ctypes.c_int64), ("shifts", ctypes.c_int64), ("back_column", ctypes.c_int32),
                ("period", ctypes.c_int32), ("dropped", ctypes.c_int64), ("n_template", ctypes.c_int64)]


class PicError(RuntimeError):
    def __init__(self, status, where, text):
        super().__init__(f"{where}: {STATUS.get(status, status)}: {text}")
        self.status = status


_lib = None


def declared_functions():
    """Names of the functions declared in include/psatd_rz.h."""
    txt = open(HEADER).read()
    return sorted(set(re.findall(r"^\s*(?:pic_status|const char\*)\s+(pic_\w+)\s*\(", txt, re.M)))


def load():
    """Load libpsatd_rz.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} is missing: build it with "
                           "`python -m paper_1611_05712_gb300.build` (no CPU fallback exists)")
    lib = ctypes.CDLL(LIB_PATH)
    P, I32, I64, D, SZ = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_double, ctypes.c_size_t
    PP = ctypes.POINTER(ctypes.c_void_p)
    sig = {
        "pic_required_bytes": [ctypes.POINTER(PicConfig), ctypes.POINTER(SZ)],
        "pic_init": [ctypes.POINTER(PicConfig), P, SZ, P, ctypes.POINTER(P)],
        "pic_destroy": [P],
        "pic_write_particles": [P, PP, P, I64, I32],
        "pic_read_particles": [P, PP, P, I64, I32],
        "pic_num_particles": [P, ctypes.POINTER(I64)],
        "pic_stage_bytes": [I64, ctypes.POINTER(SZ)],
        "pic_stage_particles": [P, PP, P, I64, P, SZ],
        "pic_take_particles": [P],
        "pic_init_background": [P, I32],
        "pic_add_beam_fields": [P, I32, I32, D],
        "pic_init_fields": [P],
        "pic_sort": [P],
        "pic_deposit": [P, I32],
        "pic_gather_push": [P, I32],
        "pic_field_step": [P, I32],
        "pic_forward_transform": [P],
        "pic_psatd": [P],
        "pic_inverse_transform": [P],
        "pic_step": [P, I32],
        "pic_step_timed": [P, I32, P],
        "pic_diagnostics": [P, I32, I32, ctypes.POINTER(PicDiag), P, I32],
        "pic_buffer_bytes": [P, I32, ctypes.POINTER(SZ)],
        "pic_copy_buffer": [P, I32, P, SZ, I32],
        "pic_load_buffer": [P, I32, P, SZ, I32],
        "pic_sync": [P],
        "pic_launch_count": [P, ctypes.POINTER(I64)],
        "pic_batch_create": [PP, I32, I32, P, ctypes.POINTER(P)],
        "pic_batch_launch": [P, I32],
        "pic_batch_info": [P, ctypes.POINTER(I32), ctypes.POINTER(I64)],
        "pic_batch_destroy": [P],
        "pic_autotune": [P, ctypes.POINTER(PicTuning)],
        "pic_set_tuning": [P, ctypes.POINTER(PicTuning)],
        "pic_get_tuning": [P, ctypes.POINTER(PicTuning)],
        "pic_fields_to_spectral": [P],
        "pic_copy_window": [P, I32, I32, I32, P, I32],
        "pic_clear_error": [P],
        "pic_selftest_wait_timeout": [P, I32],
        "pic_window_required_bytes": [P, I64, ctypes.POINTER(SZ)],
        "pic_window_setup": [P, I64, I32, I64, P, SZ],
        "pic_window_state": [P, ctypes.POINTER(PicWindowInfo)],
        "pic_set_sort_interval": [P, I32],
        "pic_get_sort_interval": [P, ctypes.POINTER(I32)],
        "pic_set_dht_path": [P, I32],
        "pic_get_dht_path": [P, ctypes.POINTER(I32)],
    }
    for name, args in sig.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = ctypes.c_int
    lib.pic_last_error.argtypes = []
    lib.pic_last_error.restype = ctypes.c_char_p
    _lib = lib
    return lib


def _check(st, where):
    if st != 0:
        raise PicError(st, where, load().pic_last_error().decode())


def make_config(Nz, Nr, Nm, dz, dr, dt, order_p=0, filter=True, precision=PIC_FP64,
                np_capacity=0, q=-1.602176634e-19, mass=9.1093837015e-31):
    return PicConfig(Nz, Nr, Nm, order_p, dz, dr, dt, int(bool(filter)), precision,
                     np_capacity, q, mass)


def required_bytes(cfg: PicConfig) -> int:
    n = ctypes.c_size_t()
    _check(load().pic_required_bytes(ctypes.byref(cfg), ctypes.byref(n)), "pic_required_bytes")
    return n.value


class Sim:
    """One simulation handle: a device workspace (torch uint8 tensor) plus the C handle."""

    def __init__(self, cfg: PicConfig, device="cuda:0", stream=None):
        import torch
        self.lib = load()
        self.cfg = cfg
        self.device = torch.device(device)
        nbytes = required_bytes(cfg)
        self.workspace = torch.empty(nbytes + 256, dtype=torch.uint8, device=self.device)
        base = self.workspace.data_ptr()
        self._ws_ptr = (base + 255) // 256 * 256
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        h = ctypes.c_void_p()
        _check(self.lib.pic_init(ctypes.byref(cfg), ctypes.c_void_p(self._ws_ptr), nbytes,
                                 ctypes.c_void_p(self.stream.cuda_stream), ctypes.byref(h)),
               "pic_init")
        self.h = h
        self.cplx = np.complex128 if cfg.precision == PIC_FP64 else np.complex64

    def close(self):
        if getattr(self, "h", None):
            self.lib.pic_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- particles ------------------------------------------------------------------
    def write_particles(self, p: dict):
        """p: dict of float64 arrays x..w and int32 id (numpy: host copy; torch cuda: device)."""
        n = len(p["x"])
        on_host = isinstance(p["x"], np.ndarray)
        if on_host:
            keep = [np.ascontiguousarray(p[k], dtype=np.float64) for k in SOA]
            ids = np.ascontiguousarray(p["id"], dtype=np.int32)
            ptrs = (ctypes.c_void_p * 7)(*[a.ctypes.data for a in keep])
            idp = ids.ctypes.data
        else:
            keep = [p[k].contiguous() for k in SOA]
            ids = p["id"].contiguous()
            ptrs = (ctypes.c_void_p * 7)(*[a.data_ptr() for a in keep])
            idp = ids.data_ptr()
        _check(self.lib.pic_write_particles(self.h, ptrs, ctypes.c_void_p(idp), n, int(on_host)),
               "pic_write_particles")

    def num_particles(self):
        n = ctypes.c_int64()
        _check(self.lib.pic_num_particles(self.h, ctypes.byref(n)), "pic_num_particles")
        return n.value

    def read_particles(self):
        n = self.num_particles()
        out = {k: np.empty(n, np.float64) for k in SOA}
        out["id"] = np.empty(n, np.int32)
        ptrs = (ctypes.c_void_p * 7)(*[out[k].ctypes.data for k in SOA])
        _check(self.lib.pic_read_particles(self.h, ptrs, ctypes.c_void_p(out["id"].ctypes.data), n, 1),
               "pic_read_particles")
        return out

    # -- staged particle input ---------------------------------------------------------
    def stage_particles(self, p: dict):
        """Start the host-to-device copy of particle set p (host float64 arrays x..w and
        int32 id: numpy arrays or CPU torch tensors, page-locked for an asynchronous copy)
        into a device staging buffer on the handle's copy stream (pic_stage_particles).
        The arrays are kept alive here until take_particles."""
        import torch

        def host(a, dt):
            if isinstance(a, torch.Tensor):
                if a.device.type != "cpu" or a.dtype != dt[1]:
                    raise TypeError("stage_particles wants CPU tensors of the particle dtypes")
                a = a.contiguous()
                return a, a.data_ptr()
            a = np.ascontiguousarray(a, dtype=dt[0])
            return a, a.ctypes.data

        n = len(p["x"])
        arrs = [host(p[k], (np.float64, torch.float64)) for k in SOA]
        ids = host(p["id"], (np.int32, torch.int32))
        nb = ctypes.c_size_t()
        _check(self.lib.pic_stage_bytes(n, ctypes.byref(nb)), "pic_stage_bytes")
        buf = getattr(self, "_stage_buf", None)
        if buf is None or buf.numel() < nb.value + 256:
            buf = self._stage_buf = torch.empty(nb.value + 256, dtype=torch.uint8, device=self.device)
        ptr = (buf.data_ptr() + 255) // 256 * 256
        ptrs = (ctypes.c_void_p * 7)(*[a[1] for a in arrs])
        _check(self.lib.pic_stage_particles(self.h, ptrs, ctypes.c_void_p(ids[1]), n, ctypes.c_void_p(ptr),
                                            nb.value), "pic_stage_particles")
        self._staged = (arrs, ids)

    def take_particles(self):
        """Replace all particles by the staged set (pic_take_particles)."""
        _check(self.lib.pic_take_particles(self.h), "pic_take_particles")
        self._staged = None

    # -- initial state ----------------------------------------------------------------
    # -- moving window ---------------------------------------------------------------
    def window_setup(self, n_plasma, period=1, n_reserve=0):
        """Switch the moving window on: particles with id < n_plasma become the plasma
        template, n_reserve inactive particles are appended (pic_window_setup)."""
        import torch
        n = ctypes.c_size_t()
        _check(self.lib.pic_window_required_bytes(self.h, int(n_plasma), ctypes.byref(n)),
               "pic_window_required_bytes")
        self.window_ws = torch.empty(n.value + 256, dtype=torch.uint8, device=self.device)
        ptr = (self.window_ws.data_ptr() + 255) // 256 * 256
        _check(self.lib.pic_window_setup(self.h, int(n_plasma), int(period), int(n_reserve),
                                         ctypes.c_void_p(ptr), n.value), "pic_window_setup")

    def window_state(self):
        info = PicWindowInfo()
        _check(self.lib.pic_window_state(self.h, ctypes.byref(info)), "pic_window_state")
        return {k: getattr(info, k) for k, _ in PicWindowInfo._fields_}

    def init_background(self, n_neutral):
        _check(self.lib.pic_init_background(self.h, int(n_neutral)), "pic_init_background")

    def add_beam_fields(self, id_lo, id_hi, gamma):
        _check(self.lib.pic_add_beam_fields(self.h, int(id_lo), int(id_hi), float(gamma)),
               "pic_add_beam_fields")

    def init_fields(self):
        _check(self.lib.pic_init_fields(self.h), "pic_init_fields")

    # -- cycle ------------------------------------------------------------------------
    def sort(self):
        _check(self.lib.pic_sort(self.h), "pic_sort")

    def deposit(self, what=PIC_DEP_RHO | PIC_DEP_J):
        _check(self.lib.pic_deposit(self.h, int(what)), "pic_deposit")

    def gather_push(self, fuse_current=True):
        _check(self.lib.pic_gather_push(self.h, int(bool(fuse_current))), "pic_gather_push")

    def field_step(self, order_p=-1):
        _check(self.lib.pic_field_step(self.h, int(order_p)), "pic_field_step")

    def clear_error(self):
        _check(self.lib.pic_clear_error(self.h), "pic_clear_error")

    def selftest_wait_timeout(self, max_polls=4096):
        _check(self.lib.pic_selftest_wait_timeout(self.h, int(max_polls)), "pic_selftest_wait_timeout")

    def fields_to_spectral(self):
        _check(self.lib.pic_fields_to_spectral(self.h), "pic_fields_to_spectral")

    def copy_window_to(self, dst, name, src_z0, nz, dst_z0):
        """Periodic z window of buffer ``name`` of this handle into handle ``dst``."""
        _check(self.lib.pic_copy_window(self.h, BUF[name], int(src_z0), int(nz), dst.h, int(dst_z0)),
               "pic_copy_window")

    def forward_transform(self):
        _check(self.lib.pic_forward_transform(self.h), "pic_forward_transform")

    def psatd(self):
        _check(self.lib.pic_psatd(self.h), "pic_psatd")

    def inverse_transform(self):
        _check(self.lib.pic_inverse_transform(self.h), "pic_inverse_transform")

    def step(self, n=1):
        _check(self.lib.pic_step(self.h, int(n)), "pic_step")

    def step_timed(self, n):
        """n cycles with per-stage CUDA-event timing; returns (stage_ms dict, total_ms)."""
        out = np.zeros(len(STAGES) + 1)
        _check(self.lib.pic_step_timed(self.h, int(n), ctypes.c_void_p(out.ctypes.data)),
               "pic_step_timed")
        return dict(zip(STAGES, out[:-1].tolist())), float(out[-1])

    def sync(self):
        _check(self.lib.pic_sync(self.h), "pic_sync")

    def launch_count(self):
        n = ctypes.c_int64()
        _check(self.lib.pic_launch_count(self.h, ctypes.byref(n)), "pic_launch_count")
        return n.value

    def autotune(self):
        """Time the tile candidates on this simulation's data and keep the fastest."""
        t = PicTuning()
        _check(self.lib.pic_autotune(self.h, ctypes.byref(t)), "pic_autotune")
        return {f: getattr(t, f) for f, _ in PicTuning._fields_}

    def set_tuning(self, dht_n_tile=0, band_chunk=1024):
        t = PicTuning(dht_n_tile, band_chunk, 0.0, 0.0)
        _check(self.lib.pic_set_tuning(self.h, ctypes.byref(t)), "pic_set_tuning")

    def set_dht_path(self, path):
        """FP64 form: PIC_DHT_AUTO, PIC_DHT_F64_GEMM or PIC_DHT_F64_SLICED."""
        _check(self.lib.pic_set_dht_path(self.h, int(path)), "pic_set_dht_path")

    def get_dht_path(self):
        k = ctypes.c_int32()
        _check(self.lib.pic_get_dht_path(self.h, ctypes.byref(k)), "pic_get_dht_path")
        return k.value

    def set_sort_interval(self, k):
        _check(self.lib.pic_set_sort_interval(self.h, int(k)), "pic_set_sort_interval")

    def get_sort_interval(self):
        k = ctypes.c_int32()
        _check(self.lib.pic_get_sort_interval(self.h, ctypes.byref(k)), "pic_get_sort_interval")
        return k.value

    def get_tuning(self):
        t = PicTuning()
        _check(self.lib.pic_get_tuning(self.h, ctypes.byref(t)), "pic_get_tuning")
        return {"dht_n_tile": t.dht_n_tile, "band_chunk": t.band_chunk}

    def diagnostics(self, id_lo, id_hi, max_slices=4096):
        """Beam diagnostics of the particles with id in [id_lo, id_hi) (pic_diagnostics):
        the pic_diag fields as a dict, plus "slice_sigma_gamma", the first
        min(n_slices, max_slices) per-slice spreads of gamma."""
        d = PicDiag()
        sl = np.zeros(max_slices)
        _check(self.lib.pic_diagnostics(self.h, int(id_lo), int(id_hi), ctypes.byref(d),
                                        ctypes.c_void_p(sl.ctypes.data), max_slices),
               "pic_diagnostics")
        out = {f: getattr(d, f) for f, _ in PicDiag._fields_}
        out["slice_sigma_gamma"] = sl[:min(d.n_slices, max_slices)].copy()
        return out

    # -- buffers ----------------------------------------------------------------------
    def buffer_bytes(self, name):
        n = ctypes.c_size_t()
        _check(self.lib.pic_buffer_bytes(self.h, BUF[name], ctypes.byref(n)), "pic_buffer_bytes")
        return n.value

    def _shape(self, name):
        c = self.cfg
        g = (c.Nm, c.Nr, c.Nz)
        return {"E": (3,) + g, "B": (3,) + g, "EH": (3,) + g, "BH": (3,) + g, "DEP": (4,) + g,
                "SRC_H": (4,) + g, "RHO_PREV_H": g, "RHO_ION": g, "KPERP": (c.Nm, c.Nr),
                "HANKEL_INV": (c.Nm, 3, c.Nr, c.Nr), "HANKEL_FWD": (c.Nm, 3, c.Nr, c.Nr),
                "KZ_MOD": (c.Nz,), "KEYS": (-1,), "PERM": (-1,)}[name]

    def _dtype(self, name):
        if name in ("KEYS", "PERM"):
            return np.int32
        if name in ("KPERP", "HANKEL_INV", "HANKEL_FWD", "KZ_MOD"):
            return np.float64
        return self.cplx

    def get(self, name):
        """Copy an internal buffer to a host numpy array."""
        nb = self.buffer_bytes(name)
        out = np.empty(nb // np.dtype(self._dtype(name)).itemsize, self._dtype(name))
        _check(self.lib.pic_copy_buffer(self.h, BUF[name], ctypes.c_void_p(out.ctypes.data), nb, 1),
               "pic_copy_buffer")
        return out.reshape(self._shape(name))

    def zeros(self, name):
        """A host array of zeros with the shape and element type of buffer ``name``."""
        nb = self.buffer_bytes(name)
        return np.zeros(nb // np.dtype(self._dtype(name)).itemsize, self._dtype(name)).reshape(self._shape(name))

    def set(self, name, arr):
        """Copy a host numpy array into an internal buffer."""
        a = np.ascontiguousarray(arr, dtype=self._dtype(name))
        nb = self.buffer_bytes(name)
        if a.nbytes != nb:
            raise ValueError(f"{name}: {a.nbytes} bytes given, {nb} expected")
        _check(self.lib.pic_load_buffer(self.h, BUF[name], ctypes.c_void_p(a.ctypes.data), nb, 1),
               "pic_load_buffer")

    # -- convenience ------------------------------------------------------------------
    @classmethod
    def from_workload(cls, w, particles, n_plasma, beams, precision=PIC_FP64, filter=True,
                      order_p=None, capacity=None, device="cuda:0", stream=None):
        """Create a handle for a workload and bring it to its initial state: particles,
        neutralising ions for the plasma, beam space-charge fields, rho^0 and E^0, B^0."""
        n = len(particles["x"])
        cfg = make_config(w.Nz, w.Nr, w.Nm, w.dz, w.dr, w.dt,
                          w.order_p if order_p is None else order_p, filter, precision,
                          capacity if capacity is not None else n)
        s = cls(cfg, device=device, stream=stream)
        s.write_particles(particles)
        s.init_background(n_plasma)
        for lo, hi, gam in beams:
            s.add_beam_fields(lo, hi, gam)
        s.init_fields()
        return s


class Batch:
    """Many simulations advanced together by one captured CUDA graph per launch.

    Each simulation must have been created on its own (non-default) torch stream and brought
    to its initial state; ``cycles`` (even) full cycles of every simulation run per launch.
    """

    def __init__(self, sims, cycles=2, origin=None):
        import torch
        self.lib = load()
        self.sims = list(sims)
        self.origin = origin if origin is not None else torch.cuda.Stream(self.sims[0].device)
        arr = (ctypes.c_void_p * len(self.sims))(*[s.h.value for s in self.sims])
        h = ctypes.c_void_p()
        _check(self.lib.pic_batch_create(arr, len(self.sims), int(cycles),
                                         ctypes.c_void_p(self.origin.cuda_stream), ctypes.byref(h)),
               "pic_batch_create")
        self.h = h
        c, k = ctypes.c_int32(), ctypes.c_int64()
        _check(self.lib.pic_batch_info(self.h, ctypes.byref(c), ctypes.byref(k)), "pic_batch_info")
        self.cycles, self.kernels_per_launch = c.value, k.value

    def launch(self, n=1):
        _check(self.lib.pic_batch_launch(self.h, int(n)), "pic_batch_launch")

    def close(self):
        if getattr(self, "h", None):
            self.lib.pic_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
