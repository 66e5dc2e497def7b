"""Python binding of the lattice C ABI (include/lattice.h).

Argument marshalling only: every step of the evolution, the initial conditions
and the diagnostics run in the CUDA library. PyTorch supplies device memory
(the eight state buffers can be torch tensors) and the CUDA stream. There is no
CPU fallback: if the compiled library cannot be loaded, construction raises.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

import numpy as np

from . import build as _build

LAT_OK = 0
STATUS_NAMES = {0: "LAT_OK", 1: "LAT_EINVAL", 2: "LAT_ECFL", 3: "LAT_ENOMEM", 4: "LAT_ECUDA",
                5: "LAT_ENONFINITE", 6: "LAT_ETIMEOUT", 7: "LAT_EUNSUPPORTED", 8: "LAT_ESTATE"}

EXPORTED = ("lat_create", "lat_create_with_buffers", "lat_init_fields", "lat_evolve", "lat_energies",
            "lat_spectrum", "lat_get_state", "lat_set_state", "lat_get_scalars", "lat_set_scalars",
            "lat_sync", "lat_set_kernel", "lat_kernel_info", "lat_destroy", "lat_status_string",
            "lat_checkpoint_bytes", "lat_save_checkpoint", "lat_load_checkpoint", "lat_field_sums_static",
            "lat_set_g2", "lat_vjp", "lat_adjoint", "lat_batch_create", "lat_batch_init_fields",
            "lat_batch_evolve", "lat_batch_sync", "lat_batch_tune", "lat_batch_member", "lat_batch_info",
            "lat_batch_destroy", "lat_batch_check_barrier", "lat_slab_create", "lat_slab_sums", "lat_slab_step",
            "lat_slab_advance", "lat_energy_field", "lat_upload_state", "lat_get_hubble_length",
            "lat_set_hubble_length", "lat_download_state", "lat_get_background", "lat_set_background",
            "lat_recenter", "lat_tune", "lat_batch_tile_heights", "lat_slab_step_range", "lat_batch_shape",
            "lat_batch_set_shape", "lat_slab_advance_local", "lat_copy_regions",
            "lat_evolve_host", "lat_buffer_layout", "lat_slab_step_ranges")


class LatParams(C.Structure):
    _fields_ = [
        ("n", C.c_int32), ("precision", C.c_int32), ("model", C.c_int32), ("expansion", C.c_int32),
        ("L", C.c_double), ("dt", C.c_double),
        ("lam", C.c_double), ("m", C.c_double), ("g2", C.c_double),
        ("phi0", C.c_double * 2), ("dphi0", C.c_double * 2),
        ("eight_pi_G", C.c_double),
        ("A", C.c_double), ("B", C.c_double), ("r", C.c_double), ("s", C.c_double),
        ("kcut", C.c_double), ("fluct", C.c_double),
        ("seed", C.c_uint64),
        ("stencil", C.c_int32), ("split", C.c_int32),
    ]


class LatEnergyReport(C.Structure):
    _fields_ = [(k, C.c_double) for k in ("t", "a", "ad", "H", "rho", "p", "w", "curv_resid")] + [
        ("kin", C.c_double * 2), ("grad", C.c_double * 2), ("pot", C.c_double),
        ("mean", C.c_double * 2), ("var", C.c_double * 2)]


class LatticeError(RuntimeError):
    def __init__(self, status: int, what: str):
        super().__init__(f"{what}: {STATUS_NAMES.get(status, status)}")
        self.status = status


_lock = threading.Lock()
_lib = None


def library_path() -> str:
    return _build.LIB


def load_library(build_if_missing: bool = True):
    """Load liblattice.so (building it with nvcc if it is missing or stale)."""
    global _lib
    with _lock:
        if _lib is None:
            path = _build.build() if build_if_missing else _build.LIB
            if not os.path.exists(path):
                raise RuntimeError(f"lattice library not built: {path}")
            L = C.CDLL(path)
            P, dp = C.c_void_p, C.POINTER(C.c_double)
            i64p = C.POINTER(C.c_int64)
            L.lat_create.argtypes = [C.POINTER(LatParams), P, C.POINTER(P)]
            L.lat_create_with_buffers.argtypes = [C.POINTER(LatParams), P, C.POINTER(P), C.POINTER(P)]
            L.lat_init_fields.argtypes = [P]
            L.lat_evolve.argtypes = [P, C.c_int64]
            L.lat_energies.argtypes = [P, C.POINTER(LatEnergyReport)]
            L.lat_energy_field.argtypes = [P, P, P]
            L.lat_upload_state.argtypes = [P, C.POINTER(C.c_void_p), C.c_int]
            L.lat_download_state.argtypes = [P, C.POINTER(C.c_void_p), C.c_int]
            L.lat_get_background.argtypes = [P, dp]
            L.lat_set_background.argtypes = [P, dp]
            L.lat_recenter.argtypes = [P]
            L.lat_spectrum.argtypes = [P, C.c_int, C.c_int, dp, dp, i64p]
            L.lat_get_state.argtypes = [P, C.c_int, C.c_int, P, C.c_int]
            L.lat_set_state.argtypes = [P, C.c_int, C.c_int, P, C.c_int]
            L.lat_get_scalars.argtypes = [P, dp]
            L.lat_set_scalars.argtypes = [P, dp]
            L.lat_get_hubble_length.argtypes = [P, dp]
            L.lat_set_hubble_length.argtypes = [P, C.c_double]
            L.lat_sync.argtypes = [P]
            L.lat_set_kernel.argtypes = [P, C.c_int, C.c_int, C.c_int, C.c_int]
            L.lat_kernel_info.argtypes = [P, i64p]
            L.lat_tune.argtypes = [P, C.c_int, i64p]
            L.lat_batch_tile_heights.argtypes = [P, C.POINTER(C.c_int32)]
            L.lat_batch_shape.argtypes = [P, i64p]
            L.lat_batch_set_shape.argtypes = [P, C.c_int, C.c_int, C.c_int]
            L.lat_slab_advance_local.argtypes = [C.POINTER(P), C.c_int, C.POINTER(P), C.c_int, C.c_int]
            L.lat_copy_regions.argtypes = [C.POINTER(P), C.POINTER(P), C.c_int, C.c_uint64, P]
            L.lat_evolve_host.argtypes = [P, C.POINTER(P), C.c_int64, C.c_int, dp]
            L.lat_buffer_layout.argtypes = [C.c_uint64, C.POINTER(C.c_uint64), C.POINTER(C.c_uint64)]
            L.lat_slab_step_ranges.argtypes = [C.POINTER(P), C.c_int, C.POINTER(C.c_int32), C.c_int, P]
            L.lat_checkpoint_bytes.argtypes = [P, C.POINTER(C.c_uint64)]
            L.lat_save_checkpoint.argtypes = [P, P, C.c_uint64]
            L.lat_load_checkpoint.argtypes = [P, P, C.c_uint64]
            L.lat_field_sums_static.argtypes = [P, P, C.c_int, C.c_int, C.c_int, C.c_double, P, P]
            L.lat_set_g2.argtypes = [P, C.c_double]
            L.lat_vjp.argtypes = [P, C.c_int64, C.c_int64, P, P, dp]
            L.lat_adjoint.argtypes = [P, C.c_int64, C.c_int, C.c_int64, dp, dp, P, P]
            L.lat_batch_create.argtypes = [C.POINTER(LatParams), C.c_int, P, C.POINTER(P)]
            L.lat_batch_init_fields.argtypes = [P]
            L.lat_batch_evolve.argtypes = [P, C.c_int64]
            L.lat_batch_sync.argtypes = [P]
            L.lat_batch_tune.argtypes = [P, C.c_int]
            L.lat_batch_member.argtypes = [P, C.c_int, C.POINTER(P)]
            L.lat_batch_info.argtypes = [P, i64p]
            L.lat_batch_check_barrier.argtypes = [P, C.c_int64]
            L.lat_slab_create.argtypes = [C.POINTER(LatParams), C.c_int, C.c_int, P, C.POINTER(P), C.POINTER(P)]
            L.lat_slab_sums.argtypes = [P, P]
            L.lat_slab_step.argtypes = [P, P]
            L.lat_slab_step_range.argtypes = [P, C.c_int, C.c_int, P]
            L.lat_slab_advance.argtypes = [P, P, C.c_int]
            L.lat_batch_destroy.argtypes = [P]
            L.lat_batch_destroy.restype = None
            L.lat_destroy.argtypes = [P]
            L.lat_destroy.restype = None
            L.lat_status_string.argtypes = [C.c_int]
            L.lat_status_string.restype = C.c_char_p
            for name in EXPORTED:
                if name not in ("lat_destroy", "lat_status_string", "lat_batch_destroy"):
                    getattr(L, name).restype = C.c_int
            _lib = L
    return _lib


def field_sums_static(f_phi, f_chi, n: int, precision: int, model: int, L: float, out, stream=None):
    """Marshal lat_field_sums_static: torch CUDA tensors in, a CUDA float64 tensor
    of 4 elements out (written asynchronously on ``stream``, a torch.cuda.Stream
    or None for the current stream). The call allocates no device memory; see
    include/lattice.h for its scratch rules."""
    import torch
    L_ = load_library()
    s = stream if stream is not None else torch.cuda.current_stream()
    st = L_.lat_field_sums_static(C.c_void_p(f_phi.data_ptr()), C.c_void_p(f_chi.data_ptr()), int(n),
                                  int(precision), int(model), float(L), C.c_void_p(out.data_ptr()),
                                  C.c_void_p(s.cuda_stream))
    _check(st, "lat_field_sums_static")


def make_params(d: dict) -> LatParams:
    p = LatParams()
    p.n = int(d["n"]); p.precision = int(d.get("precision", 32))
    p.model = int(d.get("model", 0)); p.expansion = int(d.get("expansion", 1))
    p.L = float(d.get("L", 10.0)); p.dt = float(d["dt"])
    p.lam = float(d.get("lam", 0.0)); p.m = float(d.get("m", 0.0)); p.g2 = float(d.get("g2", 0.0))
    phi0 = d.get("phi0", (1.0, 0.0)); dphi0 = d.get("dphi0", (0.0, 0.0))
    p.phi0[0], p.phi0[1] = float(phi0[0]), float(phi0[1])
    p.dphi0[0], p.dphi0[1] = float(dphi0[0]), float(dphi0[1])
    p.eight_pi_G = float(d.get("eight_pi_G", 1.0))
    p.A = float(d.get("A", 0.0)); p.B = float(d.get("B", 0.0))
    p.r = float(d.get("r", 0.0)); p.s = float(d.get("s", 0.0))
    p.kcut = float(d.get("kcut", 0.0)); p.fluct = float(d.get("fluct", 1.0))
    p.seed = int(d.get("seed", 0))
    p.stencil = int(d.get("stencil", 7))
    p.split = int(d.get("split", 0))
    return p


def staggered_buffers(lib, elems: int, dtype, device):
    """Eight zeroed arrays of `elems` elements cut from one torch allocation at
    the offsets lat_buffer_layout gives (starts distinct modulo 2 KB, so that
    same-index accesses to the eight arrays spread over the memory partitions).
    The views keep the allocation alive."""
    import torch
    esize = torch.empty((), dtype=dtype).element_size()
    off = (C.c_uint64 * 8)()
    total = C.c_uint64()
    _check(lib.lat_buffer_layout(elems * esize, off, C.byref(total)), "lat_buffer_layout")
    arena = torch.zeros((total.value + esize - 1) // esize, dtype=dtype, device=device)
    return [arena[o // esize:o // esize + elems] for o in off]


def _check(st: int, what: str):
    if st != LAT_OK:
        raise LatticeError(st, what)


class Lattice:
    """One N^3 lattice of (phi, chi) on the GPU, driven through the C ABI.

    ``params`` is a dict with the keys of ``lat_params`` (see workloads.py for
    presets). State buffers are torch tensors on ``device`` (owned by this
    object) unless ``torch_buffers`` is False, in which case the library
    allocates them. Work is issued on ``stream`` (a torch.cuda.Stream; default
    a new non-default stream so evolution can be graph-captured).
    """

    def __init__(self, params: dict, device: int = 0, stream=None, torch_buffers: bool = True):
        import torch
        self._torch = torch
        if not torch.cuda.is_available():
            raise RuntimeError("Lattice needs a CUDA device; the library has no CPU path")
        self._L = load_library()
        self.params = dict(params)
        self.n = int(params["n"])
        self.precision = int(params.get("precision", 32))
        self.dtype = torch.float32 if self.precision == 32 else torch.float64
        self.np_dtype = np.float32 if self.precision == 32 else np.float64
        self.device = torch.device("cuda", device)
        torch.cuda.set_device(self.device)
        self.stream = stream if stream is not None else torch.cuda.Stream(device=self.device)
        self._p = make_params(params)
        h = C.c_void_p()
        sptr = C.c_void_p(self.stream.cuda_stream)
        self.buffers = None
        if torch_buffers:
            self.buffers = staggered_buffers(self._L, self.n ** 3, self.dtype, self.device)
            torch.cuda.synchronize(self.device)
            arr = (C.c_void_p * 8)(*[b.data_ptr() for b in self.buffers])
            _check(self._L.lat_create_with_buffers(C.byref(self._p), sptr, arr, C.byref(h)), "lat_create_with_buffers")
        else:
            _check(self._L.lat_create(C.byref(self._p), sptr, C.byref(h)), "lat_create")
        self._h = h

    @classmethod
    def _borrow(cls, lib, handle, params: dict, device, stream, owner):
        """A view of a handle owned elsewhere (an ensemble member); closing it
        does not destroy the handle."""
        import torch
        self = cls.__new__(cls)
        self._torch = torch
        self._L = lib
        self.params = dict(params)
        self.n = int(params["n"])
        self.precision = int(params.get("precision", 32))
        self.dtype = torch.float32 if self.precision == 32 else torch.float64
        self.np_dtype = np.float32 if self.precision == 32 else np.float64
        self.device = device
        self.stream = stream
        self.buffers = None
        self._p = make_params(params)
        self._h = handle
        self._owner = owner   # keeps the ensemble alive while the view exists
        return self

    # -- lifecycle
    def close(self):
        if getattr(self, "_owner", None) is not None:
            self._h = None
            return
        if getattr(self, "_h", None):
            self._L.lat_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    # -- evolution
    def init_fields(self):
        _check(self._L.lat_init_fields(self._h), "lat_init_fields")

    def evolve(self, n_steps: int):
        _check(self._L.lat_evolve(self._h, int(n_steps)), "lat_evolve")

    def sync(self):
        _check(self._L.lat_sync(self._h), "lat_sync")

    def set_kernel(self, variant: int = 0, ty: int = 0, zr: int = 0, depth: int = 0):
        _check(self._L.lat_set_kernel(self._h, int(variant), int(ty), int(zr), int(depth)), "lat_set_kernel")

    def tune(self, steps: int = 64) -> dict:
        """Autotune the step kernel on this lattice (lat_tune); the state is kept.
        Returns the chosen shape and the timings of the sweep."""
        out = (C.c_int64 * 8)()
        _check(self._L.lat_tune(self._h, int(steps), out), "lat_tune")
        return {"variant": int(out[0]), "ty": int(out[1]), "zr": int(out[2]), "depth": int(out[3]),
                "candidates": int(out[4]), "best_ms": out[5] * 1e-6, "slowest_ms": out[6] * 1e-6,
                "blocks": int(out[7])}

    def kernel_info(self) -> dict:
        out = (C.c_int64 * 8)()
        _check(self._L.lat_kernel_info(self._h, out), "lat_kernel_info")
        keys = ("variant", "blocks", "threads", "smem", "launches_per_step", "ty", "zr", "depth")
        return dict(zip(keys, [int(v) for v in out]))

    # -- state
    def get_state_host(self, field: int, what: int) -> np.ndarray:
        """One array on the host in the lattice dtype: what 0 = f, 1 = f' whole;
        2, 3 as stored (for phi of a split lattice: the fluctuation about the
        homogeneous mode)."""
        out = np.empty((self.n, self.n, self.n), dtype=self.np_dtype)
        _check(self._L.lat_get_state(self._h, field, what, out.ctypes.data_as(C.c_void_p), 0), "lat_get_state")
        return out

    def get_state(self):
        """(f_phi, f_chi, pi_phi, pi_chi) whole, as float64 numpy arrays [z][y][x]
        (rounded to the lattice precision)."""
        return tuple(self.get_state_host(i, w).astype(np.float64) for w in (0, 1) for i in (0, 1))

    def get_state_stored(self):
        """The four arrays as stored, float64 [z][y][x] (for a split lattice phi and
        its momentum are the fluctuations about background())."""
        return tuple(self.get_state_host(i, w).astype(np.float64) for w in (2, 3) for i in (0, 1))

    def get_state_exact(self):
        """(f_phi, f_chi, pi_phi, pi_chi) as the lattice holds them, in float64
        without rounding: the stored arrays plus the homogeneous mode of a split
        lattice."""
        f0, f1, p0, p1 = self.get_state_stored()
        P, Pi = self.background()
        return f0 + P, f1, p0 + Pi, p1

    def set_state_host(self, field: int, what: int, arr: np.ndarray):
        a = np.ascontiguousarray(arr, dtype=self.np_dtype).reshape(self.n, self.n, self.n)
        _check(self._L.lat_set_state(self._h, field, what, a.ctypes.data_as(C.c_void_p), 0), "lat_set_state")

    def set_state(self, f0, f1, pi0, pi1, t=0.0, a=1.0, ad=0.0, step=0):
        """Whole fields and momenta in (rounded to the lattice precision); on a
        split lattice the homogeneous mode then moves to their means."""
        # scalars first: the step count selects which ping-pong set is current
        self.set_scalars(t, a, ad, step)
        for i, arr in enumerate((f0, f1)):
            self.set_state_host(i, 0, arr)
        for i, arr in enumerate((pi0, pi1)):
            self.set_state_host(i, 1, arr)
        if self.params.get("split", 0):
            self.recenter()

    def background(self):
        """(P, Pi): the homogeneous inflaton mode of split storage at the field
        and momentum times (zero when phi is stored whole)."""
        out = (C.c_double * 2)()
        _check(self._L.lat_get_background(self._h, out), "lat_get_background")
        return out[0], out[1]

    def set_background(self, P: float, Pi: float):
        v = (C.c_double * 2)(float(P), float(Pi))
        _check(self._L.lat_set_background(self._h, v), "lat_set_background")

    def recenter(self):
        _check(self._L.lat_recenter(self._h), "lat_recenter")

    def upload_state(self, f0, f1, pi0, pi1):
        """Queue the upload of the whole state as stored (lat_upload_state) from
        four contiguous tensors of N^3 lattice-dtype elements: CUDA tensors, or host
        tensors (page-locked for asynchronous copies). Returns without waiting for
        the copies; the sources must stay unchanged until the lattice's stream has
        passed them (e.g. sync())."""
        ptrs = self._four(f0, f1, pi0, pi1, "upload_state")
        _check(self._L.lat_upload_state(self._h, ptrs, 1 if f0.is_cuda else 0), "lat_upload_state")

    def download_state(self, f0, f1, pi0, pi1):
        """Copy the state as stored into four tensors (lat_download_state; the
        counterpart of upload_state) and wait for the copies."""
        ptrs = self._four(f0, f1, pi0, pi1, "download_state")
        _check(self._L.lat_download_state(self._h, ptrs, 1 if f0.is_cuda else 0), "lat_download_state")

    def evolve_host(self, f0, f1, pi0, pi1, n_steps: int, chunks: int = 0):
        """Evolve a state held in four page-locked host tensors (the stored
        arrays) by n_steps, the state crossing the host link every step
        (lat_evolve_host: upload, step, download, the copies in z-chunks on one
        stream per direction). The tensors hold the evolved state on return.
        Returns the scalars after each step as a float64 array [n_steps, 8]
        (t, a, a', step, four sums)."""
        import numpy as np
        if any(t.is_cuda for t in (f0, f1, pi0, pi1)):
            raise ValueError("evolve_host takes four host tensors")
        ptrs = self._four(f0, f1, pi0, pi1, "evolve_host")
        out = np.zeros((max(0, int(n_steps)), 8), dtype=np.float64)
        _check(self._L.lat_evolve_host(self._h, ptrs, int(n_steps), int(chunks),
                                       out.ctypes.data_as(C.POINTER(C.c_double))), "lat_evolve_host")
        return out

    def _four(self, f0, f1, pi0, pi1, what):
        ts = (f0, f1, pi0, pi1)
        dev = all(t.is_cuda for t in ts)
        if not dev and any(t.is_cuda for t in ts):
            raise ValueError(f"{what} takes four CUDA tensors or four host tensors")
        for t in ts:
            if t.dtype != self.dtype or not t.is_contiguous() or t.numel() != self.n ** 3:
                raise ValueError(f"{what} arrays must be contiguous with N^3 lattice-dtype elements")
        return (C.c_void_p * 4)(*[t.data_ptr() for t in ts])

    def set_state_device(self, field: int, what: int, tensor):
        t = tensor.contiguous()
        assert t.dtype == self.dtype and t.numel() == self.n ** 3 and t.is_cuda
        _check(self._L.lat_set_state(self._h, field, what, C.c_void_p(t.data_ptr()), 1), "lat_set_state")

    def get_state_device(self, field: int, what: int, out=None):
        torch = self._torch
        if out is None:
            out = torch.empty(self.n ** 3, dtype=self.dtype, device=self.device)
        _check(self._L.lat_get_state(self._h, field, what, C.c_void_p(out.data_ptr()), 1), "lat_get_state")
        return out

    def scalars(self) -> dict:
        out = (C.c_double * 8)()
        _check(self._L.lat_get_scalars(self._h, out), "lat_get_scalars")
        return {"t": out[0], "a": out[1], "ad": out[2], "step": int(out[3]), "S": list(out[4:8])}

    def set_scalars(self, t=0.0, a=1.0, ad=0.0, step=0):
        v = (C.c_double * 4)(float(t), float(a), float(ad), float(step))
        _check(self._L.lat_set_scalars(self._h, v), "lat_set_scalars")

    def hubble_length(self) -> float:
        """The L = 1/H form's l = a/a' of program time at the momentum time
        (lat_get_hubble_length; expansion = 2 only)."""
        v = C.c_double()
        _check(self._L.lat_get_hubble_length(self._h, C.byref(v)), "lat_get_hubble_length")
        return v.value

    def set_hubble_length(self, ell: float):
        _check(self._L.lat_set_hubble_length(self._h, float(ell)), "lat_set_hubble_length")

    # -- checkpoints
    def save_checkpoint(self) -> bytes:
        """Exact checkpoint (parameters, FP64 scalar block, state arrays) as bytes."""
        nb = C.c_uint64()
        _check(self._L.lat_checkpoint_bytes(self._h, C.byref(nb)), "lat_checkpoint_bytes")
        buf = (C.c_ubyte * nb.value)()
        _check(self._L.lat_save_checkpoint(self._h, buf, nb.value), "lat_save_checkpoint")
        return bytes(buf)

    def load_checkpoint(self, blob: bytes):
        buf = (C.c_ubyte * len(blob)).from_buffer_copy(blob)
        _check(self._L.lat_load_checkpoint(self._h, buf, len(blob)), "lat_load_checkpoint")

    # -- diagnostics
    ENERGY_KEYS = ("t", "a", "ad", "H", "rho", "p", "w", "curv_resid", "kin0", "kin1",
                   "grad0", "grad1", "pot", "mean0", "mean1", "var0", "var1")

    def energies(self) -> dict:
        r = LatEnergyReport()
        _check(self._L.lat_energies(self._h, C.byref(r)), "lat_energies")
        vals = [r.t, r.a, r.ad, r.H, r.rho, r.p, r.w, r.curv_resid, r.kin[0], r.kin[1], r.grad[0], r.grad[1],
                r.pot, r.mean[0], r.mean[1], r.var[0], r.var[1]]
        return dict(zip(self.ENERGY_KEYS, vals))

    def energy_field(self, rho=None, p=None):
        """Energy density and pressure at every site (lat_energy_field) as (N, N, N)
        CUDA tensors [z][y][x] of the lattice dtype, written on the lattice's
        stream without a host synchronisation. ``rho``/``p``: optional
        preallocated contiguous tensors to fill."""
        torch = self._torch
        n = self.n
        if rho is None:
            rho = torch.empty((n, n, n), dtype=self.dtype, device=self.device)
        if p is None:
            p = torch.empty((n, n, n), dtype=self.dtype, device=self.device)
        for t in (rho, p):
            if t.dtype != self.dtype or not t.is_cuda or not t.is_contiguous() or t.numel() != n ** 3:
                raise ValueError("energy_field buffers must be contiguous CUDA tensors of N^3 lattice-dtype elements")
        _check(self._L.lat_energy_field(self._h, C.c_void_p(rho.data_ptr()), C.c_void_p(p.data_ptr())),
               "lat_energy_field")
        return rho, p

    def spectrum(self, field: int, nbins: int):
        k = np.zeros(nbins); p = np.zeros(nbins); c = np.zeros(nbins, dtype=np.int64)
        _check(self._L.lat_spectrum(self._h, field, nbins, k.ctypes.data_as(C.POINTER(C.c_double)),
                                    p.ctypes.data_as(C.POINTER(C.c_double)),
                                    c.ctypes.data_as(C.POINTER(C.c_int64))), "lat_spectrum")
        return k, p, c

    # -- derivatives
    def set_g2(self, g2: float):
        """Change the coupling g^2 (the state is kept)."""
        _check(self._L.lat_set_g2(self._h, float(g2)), "lat_set_g2")
        self.params["g2"] = float(g2)

    def vjp(self, n_steps: int, fbar, pibar, abar: float = 0.0, adbar: float = 0.0, ckpt_every: int = 0):
        """Reverse-mode product of n_steps steps from the current state (lat_vjp).
        fbar, pibar: CUDA tensors of 2*n^3 elements of the lattice dtype (phi then
        chi), the adjoint of the final f and pi; overwritten in place with the
        adjoint of the starting f and pi. Returns (abar0, adbar0, dkappa0, dg2).
        The lattice ends advanced by n_steps."""
        for t in (fbar, pibar):
            assert t.is_cuda and t.dtype == self.dtype and t.numel() == 2 * self.n ** 3 and t.is_contiguous()
        sb = (C.c_double * 4)(float(abar), float(adbar), 0.0, 0.0)
        self._torch.cuda.current_stream(self.device).synchronize()
        _check(self._L.lat_vjp(self._h, int(n_steps), int(ckpt_every), C.c_void_p(fbar.data_ptr()),
                               C.c_void_p(pibar.data_ptr()), sb), "lat_vjp")
        return sb[0], sb[1], sb[2], sb[3]

    def adjoint(self, n_steps: int, observable: int = 0, ckpt_every: int = 0):
        """An observable of the state after n_steps and its gradient with respect
        to the current state and g^2 (lat_adjoint): observable 0, J = <chi^2>;
        1, the fraction of the energy density in chi. Returns (J, dJ/df, dJ/dpi,
        dJ/dg2) with the gradients as CUDA tensors of shape (2, n, n, n). The
        lattice ends advanced by n_steps."""
        torch = self._torch
        n3 = self.n ** 3
        df = torch.empty(2 * n3, dtype=self.dtype, device=self.device)
        dp = torch.empty(2 * n3, dtype=self.dtype, device=self.device)
        J, dg2 = C.c_double(), C.c_double()
        torch.cuda.current_stream(self.device).synchronize()
        _check(self._L.lat_adjoint(self._h, int(n_steps), int(observable), int(ckpt_every), C.byref(J),
                                   C.byref(dg2), C.c_void_p(df.data_ptr()), C.c_void_p(dp.data_ptr())),
               "lat_adjoint")
        shp = (2, self.n, self.n, self.n)
        return J.value, df.view(shp), dp.view(shp), dg2.value


class Ensemble:
    """Independent lattices of uneven size and coupling stepped together by one
    persistent launch per evolve call (lat_batch_*). ``params_list`` holds one
    parameter dict per member (one precision for all)."""

    def __init__(self, params_list, device: int = 0, stream=None):
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("Ensemble needs a CUDA device; the library has no CPU path")
        self._torch = torch
        self._L = load_library()
        self.params = [dict(p) for p in params_list]
        self.device = torch.device("cuda", device)
        torch.cuda.set_device(self.device)
        self.stream = stream if stream is not None else torch.cuda.Stream(device=self.device)
        arr = (LatParams * len(self.params))(*[make_params(p) for p in self.params])
        h = C.c_void_p()
        _check(self._L.lat_batch_create(arr, len(self.params), C.c_void_p(self.stream.cuda_stream), C.byref(h)),
               "lat_batch_create")
        self._h = h

    def close(self):
        if getattr(self, "_h", None):
            self._L.lat_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __len__(self):
        return len(self.params)

    def init_fields(self):
        _check(self._L.lat_batch_init_fields(self._h), "lat_batch_init_fields")

    def evolve(self, n_steps: int):
        _check(self._L.lat_batch_evolve(self._h, int(n_steps)), "lat_batch_evolve")

    def sync(self):
        _check(self._L.lat_batch_sync(self._h), "lat_batch_sync")

    def tune(self, steps: int = 10):
        _check(self._L.lat_batch_tune(self._h, int(steps)), "lat_batch_tune")

    def set_shape(self, threads: int, tile_cap: int, depth: int = 1):
        """Step with this launch shape (threads per block, tile-height cap,
        prefetch depth) from now on."""
        _check(self._L.lat_batch_set_shape(self._h, int(threads), int(tile_cap), int(depth)), "lat_batch_set_shape")

    def check_barrier(self, timeout_ns: int = 200_000_000) -> int:
        """Run the bounded-barrier self-test; returns the lat_status it ends with
        (LAT_ETIMEOUT = 6 when the timeout works)."""
        return int(self._L.lat_batch_check_barrier(self._h, int(timeout_ns)))

    def info(self) -> dict:
        out = (C.c_int64 * 8)()
        _check(self._L.lat_batch_info(self._h, out), "lat_batch_info")
        keys = ("blocks", "threads", "smem", "ranges", "graph", "sites", "members", "launches")
        info = dict(zip(keys, [int(v) for v in out]))
        ty = (C.c_int32 * len(self.params))()
        _check(self._L.lat_batch_tile_heights(self._h, ty), "lat_batch_tile_heights")
        info["ty"] = [int(v) for v in ty]
        shape = (C.c_int64 * 4)()
        _check(self._L.lat_batch_shape(self._h, shape), "lat_batch_shape")
        info["tile_cap"], info["depth"] = int(shape[1]), int(shape[2])
        return info

    def member(self, i: int) -> Lattice:
        """Borrowed Lattice view of member i (state access, energies, spectra)."""
        h = C.c_void_p()
        _check(self._L.lat_batch_member(self._h, int(i), C.byref(h)), "lat_batch_member")
        return Lattice._borrow(self._L, h, self.params[i], self.device, self.stream, self)
