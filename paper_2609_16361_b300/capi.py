"""ctypes binding of libgrlb (include/grlb.h): argument marshalling only.

Every function here has the name of the C entry point it wraps and does nothing but convert
arguments; all work runs in the CUDA library.  The product path has no CPU fallback: if the
library is missing or cannot be loaded, `lib()` raises.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

import numpy as np

from . import inputs as _inputs

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.environ.get("GRLB_LIB") or os.path.join(HERE, "libgrlb.so")

GRLB_OK = 0
STATUS = {0: "OK", -1: "EINVAL", -2: "ENOMEM", -3: "ECUDA", -4: "ENUMERIC", -5: "ETIMEOUT",
          -6: "ESTATE"}


class GrlbError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"grlb {STATUS.get(status, status)}: {msg}")
        self.status = status


class grlb_params(C.Structure):
    _fields_ = [("nx", C.c_int32), ("ny", C.c_int32), ("nz", C.c_int32), ("bc", C.c_int32),
                ("collision", C.c_int32), ("storage", C.c_int32), ("dx", C.c_double),
                ("dt", C.c_double), ("gamma", C.c_double), ("mu_ref", C.c_double),
                ("prandtl", C.c_double), ("T_ref", C.c_double), ("sutherland", C.c_int32),
                ("streaming", C.c_int32), ("T_S", C.c_double), ("omega_rho", C.c_double),
                ("omega_mom", C.c_double), ("omega_E", C.c_double), ("omega_min", C.c_double),
                ("sensor_gain", C.c_double), ("J_min", C.c_double), ("rho_min", C.c_double),
                ("p_min", C.c_double), ("ref_rho", C.c_double), ("ref_p", C.c_double),
                ("left_prim", C.c_double * 5), ("right_prim", C.c_double * 5)]


class grlb_diag(C.Structure):
    _fields_ = [("totals", C.c_double * 5), ("ke", C.c_double), ("eps_s", C.c_double),
                ("eps_d", C.c_double), ("rho_min", C.c_double), ("p_min", C.c_double),
                ("n_floor", C.c_int64), ("n_nan", C.c_int64), ("n_sensor", C.c_int64),
                ("step", C.c_int64), ("s", C.c_double), ("ncells", C.c_int64)]

    def as_dict(self):
        return dict(totals=np.array(self.totals[:]), ke=self.ke, eps_s=self.eps_s,
                    eps_d=self.eps_d, rho_min=self.rho_min, p_min=self.p_min,
                    n_floor=self.n_floor, n_nan=self.n_nan, n_sensor=self.n_sensor,
                    step=self.step, s=self.s, ncells=self.ncells)


class grlb_check_counts(C.Structure):
    _fields_ = [("violations", C.c_int64), ("first_addr", C.c_uint64), ("live_regions", C.c_int64),
                ("unmatched", C.c_int64), ("overflow", C.c_int64)]

    def as_dict(self):
        return {name: int(getattr(self, name)) for name, _ in self._fields_}


class grlb_batch_config(C.Structure):
    _fields_ = [("block_x", C.c_int32), ("solo_min_cells", C.c_int32), ("use_graph", C.c_int32),
                ("schedule", C.c_int32), ("max_lanes", C.c_int32)]


_lock = threading.Lock()
_lib = None


def lib():
    """Load libgrlb.so (building it first if the sources are newer).  Raises if it cannot."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        from . import build as _build
        if LIB_PATH == _build.LIB and _build.needs_build():
            _build.build()
        elif LIB_PATH == _build.LIB_CHECKED and _build.needs_build(checked=True):
            _build.build(checked=True)
        if not os.path.exists(LIB_PATH):
            raise GrlbError(-3, f"CUDA library missing: {LIB_PATH}")
        L = C.CDLL(LIB_PATH)
        vp, dp, i32, i64, sz = C.c_void_p, C.POINTER(C.c_double), C.c_int, C.c_int64, C.c_size_t
        sig = {
            "grlb_last_error": ([], C.c_char_p),
            "grlb_version": ([], C.c_char_p),
            "grlb_create": ([C.POINTER(grlb_params), vp, C.POINTER(vp)], i32),
            "grlb_destroy": ([vp], None),
            "grlb_set_stream": ([vp, vp], i32),
            "grlb_device_bytes": ([vp], sz),
            "grlb_bytes_for": ([C.POINTER(grlb_params)], sz),
            "grlb_init_primitive": ([vp, dp, dp, dp], i32),
            "grlb_init_primitive_device": ([vp, vp, vp, vp], i32),
            "grlb_stage_primitive": ([vp, dp, dp, dp], i32),
            "grlb_init_from_stage": ([vp], i32),
            "grlb_step": ([vp, i32], i32),
            "grlb_set_source_device": ([vp, vp], i32),
            "grlb_step_diag": ([vp], i32),
            "grlb_diag_read": ([vp, C.POINTER(grlb_diag)], i32),
            "grlb_check_finite": ([vp, vp], i32),
            "grlb_read_conserved": ([vp, dp], i32),
            "grlb_read_primitive": ([vp, dp, dp, dp, dp], i32),
            "grlb_read_cells": ([vp, C.POINTER(C.c_int64), i64, dp], i32),
            "grlb_save": ([vp, vp, C.POINTER(sz)], i32),
            "grlb_load": ([vp, vp, sz], i32),
            "grlb_steps_done": ([vp], i64),
            "grlb_batch_create": ([C.POINTER(vp), i32, C.POINTER(grlb_batch_config),
                                   C.POINTER(vp)], i32),
            "grlb_batch_destroy": ([vp], None),
            "grlb_batch_set_stream": ([vp, vp], i32),
            "grlb_batch_set_active": ([vp, C.POINTER(C.c_int)], i32),
            "grlb_batch_step": ([vp, i32], i32),
            "grlb_batch_set_tile_x": ([vp, C.POINTER(C.c_int)], i32),
            "grlb_step_diag_noalloc": ([C.POINTER(grlb_params), vp, vp, vp, vp], i32),
            "grlb_spectrum_shells": ([C.POINTER(grlb_params)], C.c_int32),
            "grlb_spectral_diag": ([vp, C.c_int32, dp, dp], i32),
            "grlb_ffma_probe": ([C.c_int32, C.c_int32, vp, vp, dp], i32),
            "grlb_set_init_mode": ([vp, C.c_int32], i32),
            "grlb_halo_exchange_z": ([vp, vp], i32),
            "grlb_halo_pack_z": ([vp, vp, vp], i32),
            "grlb_halo_unpack_z": ([vp, vp, vp], i32),
            "grlb_trim_pool": ([], i32),
            "grlb_checked_build": ([], C.c_int32),
            "grlb_check_read": ([C.POINTER(grlb_check_counts), C.c_int32], i32),
            "grlb_check_probe": ([vp, C.c_uint64, C.c_int64, C.c_uint64, vp], i32),
        }
        for name, (args, res) in sig.items():
            fn = getattr(L, name)
            fn.argtypes = args
            fn.restype = res
        _lib = L
        return L


def exported_symbols():
    return ["grlb_last_error", "grlb_version", "grlb_create", "grlb_destroy", "grlb_set_stream",
            "grlb_device_bytes", "grlb_bytes_for", "grlb_init_primitive",
            "grlb_init_primitive_device", "grlb_stage_primitive", "grlb_init_from_stage",
            "grlb_set_source_device", "grlb_step",
            "grlb_step_diag", "grlb_diag_read", "grlb_check_finite", "grlb_read_conserved",
            "grlb_read_primitive", "grlb_read_cells",
            "grlb_save", "grlb_load", "grlb_steps_done", "grlb_batch_create",
            "grlb_batch_destroy", "grlb_batch_set_stream", "grlb_batch_set_active",
            "grlb_batch_step", "grlb_batch_set_tile_x", "grlb_step_diag_noalloc",
            "grlb_spectrum_shells", "grlb_spectral_diag", "grlb_ffma_probe",
            "grlb_set_init_mode", "grlb_halo_exchange_z", "grlb_halo_pack_z", "grlb_halo_unpack_z",
            "grlb_trim_pool", "grlb_checked_build", "grlb_check_read", "grlb_check_probe"]


def check(status):
    if status != GRLB_OK:
        raise GrlbError(status, lib().grlb_last_error().decode())


def _dp(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def to_params(prm: "_inputs.CaseParams") -> grlb_params:
    P = grlb_params()
    for name, _ in grlb_params._fields_:
        if name in ("pad0",):
            continue
        v = getattr(prm, name)
        if name in ("left_prim", "right_prim"):
            arr = getattr(P, name)
            for k in range(5):
                arr[k] = float(v[k])
        else:
            setattr(P, name, v)
    return P


# ---- thin wrappers with the C names -------------------------------------------------------
def grlb_create(prm, stream=None):
    h = C.c_void_p()
    P = to_params(prm)
    check(lib().grlb_create(C.byref(P), stream, C.byref(h)))
    return h


def grlb_destroy(h):
    lib().grlb_destroy(h)


def grlb_set_stream(h, stream):
    """Move the domain's later work to another cudaStream_t (int handle, or None)."""
    check(lib().grlb_set_stream(h, stream))


def grlb_bytes_for(prm) -> int:
    P = to_params(prm)
    return int(lib().grlb_bytes_for(C.byref(P)))


def grlb_init_primitive(h, rho, u, p):
    rho = np.ascontiguousarray(rho, np.float64)
    u = np.ascontiguousarray(u, np.float64)
    p = np.ascontiguousarray(p, np.float64)
    check(lib().grlb_init_primitive(h, _dp(rho), _dp(u), _dp(p)))


def grlb_stage_primitive(h, rho, u, p):
    """Enqueue the upload of host FP64 fields into a staging slot (arrays must be contiguous
    float64 and stay alive and unchanged until grlb_init_from_stage has run)."""
    for a in (rho, u, p):
        if not (a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]):
            raise GrlbError(-1, "staged arrays must be contiguous float64")
    check(lib().grlb_stage_primitive(h, _dp(rho), _dp(u), _dp(p)))


def grlb_init_from_stage(h):
    check(lib().grlb_init_from_stage(h))


def grlb_init_primitive_device(h, rho_ptr, u_ptr, p_ptr):
    """Device pointers (ints, e.g. torch tensor .data_ptr()) of FP64 fields on the device."""
    check(lib().grlb_init_primitive_device(h, rho_ptr, u_ptr, p_ptr))


def grlb_set_source_device(h, ptr):
    """Device pointer (int, e.g. a float32 torch tensor's data_ptr()) of 5 x N source rates in
    physical units, or None."""
    check(lib().grlb_set_source_device(h, ptr))


def grlb_step(h, n):
    check(lib().grlb_step(h, int(n)))


def grlb_step_diag(h):
    check(lib().grlb_step_diag(h))


GRLB_ENUMERIC = -4


def grlb_diag_read(h, allow_nonfinite: bool = False) -> dict:
    """Diagnostics of the last diagnostic sweep.  A non-finite state (n_nan > 0) makes the C
    call return GRLB_ENUMERIC: raised as GrlbError, or, with allow_nonfinite, the filled-in
    record is returned."""
    d = grlb_diag()
    st = lib().grlb_diag_read(h, C.byref(d))
    if st == GRLB_ENUMERIC and allow_nonfinite:
        return d.as_dict()
    check(st)
    return d.as_dict()


def grlb_check_finite(h, flag_ptr):
    """Enqueue the finiteness scan of the current state: sets the int32 at flag_ptr (device or
    page-locked host memory, as an int) to 1 if a stored population is non-finite."""
    check(lib().grlb_check_finite(h, flag_ptr))


def grlb_read_conserved(h, N, out=None):
    if out is None:
        out = np.empty((5, N), np.float64)
    check(lib().grlb_read_conserved(h, _dp(out)))
    return out


def grlb_read_primitive(h, N):
    rho, u, p, T = np.empty(N), np.empty((3, N)), np.empty(N), np.empty(N)
    check(lib().grlb_read_primitive(h, _dp(rho), _dp(u), _dp(p), _dp(T)))
    return rho, u, p, T


def grlb_read_cells(h, cells) -> np.ndarray:
    """Populations f*_q (lattice units) of the listed cells: array (35, len(cells))."""
    cells = np.ascontiguousarray(cells, np.int64).ravel()
    out = np.empty((35, cells.size))
    check(lib().grlb_read_cells(h, cells.ctypes.data_as(C.POINTER(C.c_int64)), cells.size, _dp(out)))
    return out


def grlb_save(h) -> np.ndarray:
    """Checkpoint as a uint8 array (header + stored populations)."""
    n = C.c_size_t(0)
    check(lib().grlb_save(h, None, C.byref(n)))
    buf = np.empty(n.value, np.uint8)
    check(lib().grlb_save(h, buf.ctypes.data_as(C.c_void_p), C.byref(n)))
    return buf


def grlb_load(h, data):
    buf = np.ascontiguousarray(np.frombuffer(data, np.uint8) if isinstance(data, bytes) else data)
    check(lib().grlb_load(h, buf.ctypes.data_as(C.c_void_p), buf.nbytes))


def grlb_steps_done(h) -> int:
    return int(lib().grlb_steps_done(h))


SCHED_CONCURRENT, SCHED_TABLE_CONST, SCHED_TABLE = 0, 1, 2


def grlb_batch_create(handles, block_x=0, use_graph=1, solo_min_cells=0, schedule=SCHED_CONCURRENT,
                      max_lanes=0):
    arr = (C.c_void_p * len(handles))(*[h.value for h in handles])
    cfg = grlb_batch_config(block_x, solo_min_cells, use_graph, schedule, max_lanes)
    b = C.c_void_p()
    check(lib().grlb_batch_create(arr, len(handles), C.byref(cfg), C.byref(b)))
    return b


def grlb_batch_destroy(b):
    lib().grlb_batch_destroy(b)


def grlb_batch_set_stream(b, stream):
    check(lib().grlb_batch_set_stream(b, stream))


def grlb_batch_set_active(b, active):
    if active is None:
        check(lib().grlb_batch_set_active(b, None))
    else:
        arr = (C.c_int * len(active))(*[int(bool(a)) for a in active])
        check(lib().grlb_batch_set_active(b, arr))


def grlb_batch_set_tile_x(b, tile_x):
    if tile_x is None:
        check(lib().grlb_batch_set_tile_x(b, None))
    else:
        arr = (C.c_int * len(tile_x))(*[int(t) for t in tile_x])
        check(lib().grlb_batch_set_tile_x(b, arr))


def grlb_batch_step(b, n):
    check(lib().grlb_batch_step(b, int(n)))


def grlb_step_diag_noalloc(prm, f_in_ptr, f_out_ptr, diag_out_ptr, stream=None):
    """One diagnostic sweep on caller-owned device buffers (device pointers as ints); the
    library allocates no device memory for it."""
    P = to_params(prm)
    check(lib().grlb_step_diag_noalloc(C.byref(P), f_in_ptr, f_out_ptr, diag_out_ptr, stream))


def grlb_set_init_mode(h, ce_init):
    check(lib().grlb_set_init_mode(h, int(ce_init)))


def grlb_halo_exchange_z(lower, upper):
    check(lib().grlb_halo_exchange_z(lower, upper))


def grlb_halo_pack_z(h, to_upper_ptr, to_lower_ptr):
    """Enqueue the packing of a slab's outgoing ghost slices into device buffers (ints)."""
    check(lib().grlb_halo_pack_z(h, to_upper_ptr, to_lower_ptr))


def grlb_halo_unpack_z(h, from_lower_ptr, from_upper_ptr):
    """Enqueue the unpacking of received ghost slices (device buffers, ints) into the slab."""
    check(lib().grlb_halo_unpack_z(h, from_lower_ptr, from_upper_ptr))


def grlb_spectrum_shells(prm) -> int:
    P = to_params(prm)
    return int(lib().grlb_spectrum_shells(C.byref(P)))


def grlb_spectral_diag(h, nbins):
    """Shell spectrum (nbins,) and dict(eps_s, eps_d, ke_u) of the domain's current state
    (lattice units; spectral derivatives)."""
    spec = np.zeros(max(int(nbins), 1))
    sums = np.zeros(3)
    check(lib().grlb_spectral_diag(h, int(nbins), _dp(spec), _dp(sums)))
    return spec[:int(nbins)], dict(eps_s=float(sums[0]), eps_d=float(sums[1]), ke_u=float(sums[2]))


def grlb_ffma_probe(ctas, iters, sink_ptr, stream=None) -> float:
    """Enqueue the FFMA issue-rate probe; returns its FFMA warp-instruction count."""
    n = C.c_double(0.0)
    check(lib().grlb_ffma_probe(int(ctas), int(iters), sink_ptr, stream, C.byref(n)))
    return n.value


# ---- convenience object --------------------------------------------------------------------
class Domain:
    """One domain on the current CUDA device (owns its C handle)."""

    def __init__(self, prm, stream=None):
        self.prm = prm
        self.N = prm.nx * prm.ny * prm.nz
        self.h = grlb_create(prm, stream)

    def close(self):
        if self.h is not None:
            grlb_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def init(self, rho, u, p, ce_init=None):
        """Initialise from host FP64 primitive fields; ce_init = True / False sets the domain's
        init mode first (None keeps it)."""
        if ce_init is not None:
            grlb_set_init_mode(self.h, 1 if ce_init else 0)
        grlb_init_primitive(self.h, rho, u, p)

    def step(self, n=1):
        grlb_step(self.h, n)

    def step_diag(self):
        grlb_step_diag(self.h)

    def diag(self, allow_nonfinite=False):
        return grlb_diag_read(self.h, allow_nonfinite)

    def conserved(self, out=None):
        return grlb_read_conserved(self.h, self.N, out)

    def primitive(self):
        return grlb_read_primitive(self.h, self.N)

    def spectral(self, nbins=None):
        nb = grlb_spectrum_shells(self.prm) if nbins is None else nbins
        return grlb_spectral_diag(self.h, nb)

    @property
    def steps(self):
        return grlb_steps_done(self.h)


def grlb_trim_pool():
    """Return the device memory the library's pool keeps for reuse to the system (synchronises)."""
    check(lib().grlb_trim_pool())


# ---- bounds-checked build (libgrlb_checked.so, selected with GRLB_LIB) -----------------------
def grlb_checked_build() -> bool:
    return bool(lib().grlb_checked_build())


def grlb_check_read(reset=False) -> dict:
    """Counts of the checked build's access tests (synchronises the device)."""
    c = grlb_check_counts()
    check(lib().grlb_check_read(C.byref(c), 1 if reset else 0))
    return c.as_dict()


def grlb_check_probe(base, nbytes, offset, access_bytes, stream=None):
    """Test [base + offset, + access_bytes) against a region [base, base + nbytes) made live for
    the probe alone; nothing at either address is accessed."""
    check(lib().grlb_check_probe(base, nbytes, offset, access_bytes, stream))
