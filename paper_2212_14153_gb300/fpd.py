"""ctypes binding of the C ABI in ``include/fpd.h`` (names kept identical).

Argument marshalling only: every step of the method runs in the CUDA
library ``libfpd.so``.  There is no CPU fallback; importing the binding on a
machine without the built library, or calling it without a GPU, raises.
PyTorch is used only to obtain the current CUDA stream.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libfpd.so")

FPD_OK, FPD_EINVAL, FPD_ENOMEM, FPD_ECUDA, FPD_ETIMEOUT, FPD_ENAN, FPD_EBUSY = 0, -1, -2, -3, -4, -5, -6
FPD_F64, FPD_F32, FPD_F32_F16STORE = 0, 1, 2
FPD_MRT_MAGIC, FPD_MRT_LL, FPD_BGK = 0, 1, 2
FPD_FLAG_FAST_BEAD, FPD_FLAG_NONFINITE, FPD_FLAG_COPY_TIMEOUT = 1, 2, 4
SLOT_FREE, SLOT_RUNNING, SLOT_FINISHED, SLOT_FAILED = 0, 1, 2, 3

_DP = ctypes.POINTER(ctypes.c_double)


class fpd_params(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_int32), ("ny", ctypes.c_int32),
        ("u_bottom", ctypes.c_double), ("u_top", ctypes.c_double),
        ("nu_f", ctypes.c_double), ("re", ctypes.c_double),
        ("visc_ratio", ctypes.c_double), ("xi", ctypes.c_double),
        ("bead_radius", ctypes.c_double),
        ("n_beads", ctypes.c_int32), ("n_fibers", ctypes.c_int32),
        ("k_s", ctypes.c_double), ("k_b", ctypes.c_double),
        ("stiffness_K", ctypes.c_double), ("k_ev", ctypes.c_double),
        ("phi_cut", ctypes.c_double),
        ("body_force_x", ctypes.c_double), ("body_force_y", ctypes.c_double),
        ("precision", ctypes.c_int32), ("collision", ctypes.c_int32),
        ("init_couette", ctypes.c_int32),
        ("s_e", ctypes.c_double), ("s_eps", ctypes.c_double), ("s_q", ctypes.c_double),
        ("centre_xy", _DP), ("theta0", _DP), ("bead_xy", _DP),
        ("sandwich_zl", ctypes.c_double), ("sandwich_zr", ctypes.c_double),
        ("periodic_y", ctypes.c_int32), ("bead_force_x", ctypes.c_double),
        ("bead_force_y", ctypes.c_double),
    ]


class FpdError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"fpd error {code}: {msg}")
        self.code = code


_lib = None
_lock = threading.Lock()

# name -> (restype, argtypes); every symbol include/fpd.h declares
SIGNATURES = {
    "fpd_version": (ctypes.c_int, []),
    "fpd_default_params": (None, [ctypes.POINTER(fpd_params)]),
    "fpd_create": (ctypes.c_int, [ctypes.POINTER(fpd_params), ctypes.c_void_p, ctypes.POINTER(ctypes.c_void_p)]),
    "fpd_step": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int64]),
    "fpd_prepare": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int64]),
    "fpd_sync": (ctypes.c_int, [ctypes.c_void_p]),
    "fpd_flags": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_uint32)]),
    "fpd_batch_slot_flags": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32, ctypes.POINTER(ctypes.c_uint32)]),
    "fpd_read_fields": (ctypes.c_int, [ctypes.c_void_p, _DP, _DP, _DP]),
    "fpd_internal_flow": (ctypes.c_int, [ctypes.c_void_p, _DP]),
    "fpd_workspace_bytes": (ctypes.c_int, [ctypes.POINTER(fpd_params), ctypes.POINTER(ctypes.c_uint64)]),
    "fpd_create_ex": (ctypes.c_int, [ctypes.POINTER(fpd_params), ctypes.c_void_p, ctypes.c_void_p, ctypes.c_uint64,
                                     ctypes.POINTER(ctypes.c_void_p)]),
    "fpd_save": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_char_p]),
    "fpd_load": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_char_p]),
    "fpd_batch_internal_flow": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32, _DP]),
    "fpd_read_beads": (ctypes.c_int, [ctypes.c_void_p, _DP, _DP, _DP, _DP]),
    "fpd_read_beads_async": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.POINTER(ctypes.c_uint64)]),
    "fpd_wait_read": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_uint64]),
    "fpd_export_beads": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32]),
    "fpd_take_beads": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int64, _DP]),
    "fpd_read_populations": (ctypes.c_int, [ctypes.c_void_p, _DP]),
    "fpd_write_populations": (ctypes.c_int, [ctypes.c_void_p, _DP]),
    "fpd_diag": (ctypes.c_int, [ctypes.c_void_p, _DP]),
    "fpd_diag_noalloc": (ctypes.c_int, [ctypes.c_void_p, _DP]),
    "fpd_derived": (ctypes.c_int, [ctypes.c_void_p, _DP]),
    "fpd_set_tuning": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32]),
    "fpd_sweep_variants": (ctypes.c_int32, []),
    "fpd_get_tuning": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_int32),
                                      ctypes.POINTER(ctypes.c_int32)]),
    "fpd_batch_set_tuning": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32]),
    "fpd_set_profiling": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int]),
    "fpd_kernel_times": (ctypes.c_int, [ctypes.c_void_p, _DP]),
    "fpd_last_error": (ctypes.c_char_p, [ctypes.c_void_p]),
    "fpd_destroy": (ctypes.c_int, [ctypes.c_void_p]),
    "fpd_batch_create": (ctypes.c_int, [ctypes.c_int32, ctypes.c_int32, ctypes.c_int64, ctypes.c_int32,
                                        ctypes.c_void_p, ctypes.POINTER(ctypes.c_void_p)]),
    "fpd_batch_add": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(fpd_params), ctypes.c_int64,
                                     ctypes.POINTER(ctypes.c_int32)]),
    "fpd_batch_run": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int64, ctypes.POINTER(ctypes.c_int64)]),
    "fpd_batch_sync": (ctypes.c_int, [ctypes.c_void_p]),
    "fpd_batch_poll": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_int32), ctypes.c_int32,
                                      ctypes.POINTER(ctypes.c_int32)]),
    "fpd_batch_slot_info": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32, ctypes.POINTER(ctypes.c_int64)]),
    "fpd_batch_read_fields": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32, _DP, _DP, _DP]),
    "fpd_batch_read_beads": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32, _DP, _DP, _DP, _DP]),
    "fpd_batch_step": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int64]),
    "fpd_batch_read": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32, _DP, _DP, _DP]),
    "fpd_batch_read_populations": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32, _DP]),
    "fpd_batch_remove": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32]),
    "fpd_batch_stats": (ctypes.c_int, [ctypes.c_void_p, _DP]),
    "fpd_batch_last_error": (ctypes.c_char_p, [ctypes.c_void_p]),
    "fpd_batch_destroy": (ctypes.c_int, [ctypes.c_void_p]),
}


def load_library(path: str = LIB_PATH):
    """Load ``libfpd.so`` (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(path):
                raise RuntimeError(f"CUDA library {path} is missing: run __graft_entry__.build() first")
            lib = ctypes.CDLL(path)
            for name, (res, args) in SIGNATURES.items():
                fn = getattr(lib, name)
                fn.restype = res
                fn.argtypes = args
            _lib = lib
    return _lib


def _ptr(a):
    if a is None:
        return None
    assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(_DP)


def _check(rc: int, handle=None):
    if rc != FPD_OK:
        msg = load_library().fpd_last_error(handle)
        raise FpdError(rc, msg.decode() if msg else "")


# ------------------------------------------------------------ thin wrappers
def fpd_version() -> int:
    return load_library().fpd_version()


def fpd_default_params() -> fpd_params:
    p = fpd_params()
    load_library().fpd_default_params(ctypes.byref(p))
    return p


def fpd_create(params: fpd_params, stream=None) -> ctypes.c_void_p:
    h = ctypes.c_void_p()
    rc = load_library().fpd_create(ctypes.byref(params), stream, ctypes.byref(h))
    _check(rc, None)
    return h


def fpd_workspace_bytes(params: fpd_params) -> int:
    n = ctypes.c_uint64()
    _check(load_library().fpd_workspace_bytes(ctypes.byref(params), ctypes.byref(n)), None)
    return int(n.value)


def fpd_create_ex(params: fpd_params, stream, workspace_ptr: int, workspace_bytes: int) -> ctypes.c_void_p:
    h = ctypes.c_void_p()
    rc = load_library().fpd_create_ex(ctypes.byref(params), stream, ctypes.c_void_p(workspace_ptr),
                                      int(workspace_bytes), ctypes.byref(h))
    _check(rc, None)
    return h


def fpd_step(h, n_steps: int) -> None:
    _check(load_library().fpd_step(h, int(n_steps)), h)


def fpd_prepare(h, n_steps: int) -> None:
    _check(load_library().fpd_prepare(h, n_steps), h)


def fpd_sync(h) -> None:
    _check(load_library().fpd_sync(h), h)


def fpd_flags(h) -> int:
    v = ctypes.c_uint32()
    _check(load_library().fpd_flags(h, ctypes.byref(v)), h)
    return int(v.value)


def fpd_batch_slot_flags(b, slot: int) -> int:
    v = ctypes.c_uint32()
    _bcheck(load_library().fpd_batch_slot_flags(b, slot, ctypes.byref(v)), b)
    return int(v.value)


def fpd_read_fields(h, ux, uy, rho) -> None:
    _check(load_library().fpd_read_fields(h, _ptr(ux), _ptr(uy), _ptr(rho)), h)


def fpd_save(h, path: str) -> None:
    _check(load_library().fpd_save(h, os.fsencode(path)), h)


def fpd_load(h, path: str) -> None:
    _check(load_library().fpd_load(h, os.fsencode(path)), h)


def fpd_internal_flow(h, eps) -> None:
    _check(load_library().fpd_internal_flow(h, _ptr(eps)), h)


def fpd_batch_internal_flow(b, slot: int, eps) -> None:
    _bcheck(load_library().fpd_batch_internal_flow(b, int(slot), _ptr(eps)), b)


def fpd_read_beads(h, pos, vel, force, support=None) -> None:
    _check(load_library().fpd_read_beads(h, _ptr(pos), _ptr(vel), _ptr(force), _ptr(support)), h)


def fpd_read_beads_async(h, dst_ptr: int) -> int:
    """dst_ptr: address of a host buffer of 7 * nb doubles (pinned for an
    asynchronous copy); returns the read's ticket."""
    t = ctypes.c_uint64(0)
    _check(load_library().fpd_read_beads_async(h, ctypes.c_void_p(dst_ptr), ctypes.byref(t)), h)
    return t.value


def fpd_wait_read(h, ticket: int) -> None:
    _check(load_library().fpd_wait_read(h, ctypes.c_uint64(ticket)), h)


def fpd_export_beads(h, slots: int) -> None:
    _check(load_library().fpd_export_beads(h, slots), h)


def fpd_take_beads(h, n: int, dst) -> None:
    _check(load_library().fpd_take_beads(h, n, _ptr(dst)), h)


def fpd_read_populations(h, f) -> None:
    _check(load_library().fpd_read_populations(h, _ptr(f)), h)


def fpd_write_populations(h, f) -> None:
    _check(load_library().fpd_write_populations(h, _ptr(f)), h)


def fpd_diag(h, out) -> None:
    _check(load_library().fpd_diag(h, _ptr(out)), h)


def fpd_diag_noalloc(h, out) -> None:
    """fpd_diag without device allocation (static scratch; see include/fpd.h)."""
    _check(load_library().fpd_diag_noalloc(h, _ptr(out)), h)


def fpd_set_tuning(h, variant: int) -> None:
    _check(load_library().fpd_set_tuning(h, int(variant)), h)


def fpd_sweep_variants() -> int:
    return int(load_library().fpd_sweep_variants())


def fpd_get_tuning(h) -> tuple[int, int]:
    v, n = ctypes.c_int32(0), ctypes.c_int32(0)
    _check(load_library().fpd_get_tuning(h, ctypes.byref(v), ctypes.byref(n)), h)
    return v.value, n.value


def fpd_batch_set_tuning(b, variant: int) -> None:
    _bcheck(load_library().fpd_batch_set_tuning(b, int(variant)), b)


def fpd_derived(h, out) -> None:
    _check(load_library().fpd_derived(h, _ptr(out)), h)


def fpd_set_profiling(h, on: bool) -> None:
    _check(load_library().fpd_set_profiling(h, 1 if on else 0), h)


def fpd_kernel_times(h, out) -> None:
    _check(load_library().fpd_kernel_times(h, _ptr(out)), h)


def fpd_last_error(h=None) -> str:
    msg = load_library().fpd_last_error(h)
    return msg.decode() if msg else ""


def fpd_destroy(h) -> None:
    if h is not None and h.value:
        load_library().fpd_destroy(h)


# ------------------------------------------------------------ convenience
def params_from_config(cfg: dict) -> tuple[fpd_params, list]:
    """Fill fpd_params from a workload dict; returns the struct and the numpy
    arrays it points to (keep them alive until fpd_create returns)."""
    p = fpd_default_params()
    simple = dict(nx="nx", ny="ny", u_bottom="u_bottom", u_top="u_top", nu_f="nu_f", re="re",
                  visc_ratio="visc_ratio", xi="xi", a="bead_radius", n_beads="n_beads",
                  n_fibers="n_fibers", k_s="k_s", k_b="k_b", stiffness_K="stiffness_K",
                  k_ev="k_ev", phi_cut="phi_cut", gx="body_force_x", gy="body_force_y",
                  precision="precision", collision="collision", init_couette="init_couette",
                  s_e="s_e", s_eps="s_eps", s_q="s_q", sandwich_zl="sandwich_zl",
                  sandwich_zr="sandwich_zr", periodic_y="periodic_y", bead_fx="bead_force_x",
                  bead_fy="bead_force_y")
    for k, field in simple.items():
        if k in cfg:
            setattr(p, field, cfg[k])
    keep = []
    nf = max(int(cfg.get("n_fibers", 0)), 1)
    cen = np.ascontiguousarray(cfg.get("centres", np.zeros((nf, 2))), dtype=np.float64).reshape(-1)
    th = np.ascontiguousarray(cfg.get("theta0", np.zeros(nf)), dtype=np.float64).reshape(-1)
    keep += [cen, th]
    p.centre_xy = _ptr(cen)
    p.theta0 = _ptr(th)
    if cfg.get("bead_xy") is not None:
        bx = np.ascontiguousarray(cfg["bead_xy"], dtype=np.float64).reshape(-1)
        keep.append(bx)
        p.bead_xy = _ptr(bx)
    return p, keep


def workspace_bytes(cfg: dict) -> int:
    """Device bytes a Simulation of cfg needs when given a workspace."""
    p, keep = params_from_config(cfg)
    return fpd_workspace_bytes(p)


class Simulation:
    """One FPD instance on the GPU, driven through the C ABI."""

    def __init__(self, cfg: dict, stream=None, workspace=None, tuning=None):
        """workspace: optional CUDA tensor (any dtype, contiguous, at least
        workspace_bytes(cfg) bytes, 256-byte aligned) that holds the state;
        it is kept referenced for the handle's lifetime.

        tuning: sweep launch shape.  None keeps variant 0, the shape a
        Batch also starts with, so a lone run and the same instance in a
        batch agree bit for bit; an int sets that variant; "auto" takes
        the fastest variant the autotuner measured for this workload
        (timed once on a scratch instance, then cached)."""
        if stream is None:
            import torch
            if not torch.cuda.is_available():
                raise RuntimeError("no CUDA device: the FPD library runs on the GPU only")
            stream = torch.cuda.current_stream().cuda_stream
        self.cfg = dict(cfg)
        p, keep = params_from_config(cfg)
        self._ws = workspace
        if workspace is not None:
            self.h = fpd_create_ex(p, stream, workspace.data_ptr(), workspace.numel() * workspace.element_size())
        else:
            self.h = fpd_create(p, stream)
        self.nx, self.ny = p.nx, p.ny
        self.nb = p.n_beads * p.n_fibers
        if tuning == "auto":
            from . import autotune
            tuning = autotune.tune(self.cfg)
        if tuning is not None:
            self.set_tuning(int(tuning))

    def close(self):
        if getattr(self, "h", None) is not None:
            fpd_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def step(self, n: int = 1):
        fpd_step(self.h, n)

    def prepare(self, n: int):
        """Capture the step graphs the next step(n) will replay."""
        fpd_prepare(self.h, n)

    def sync(self):
        fpd_sync(self.h)

    def flags(self) -> int:
        """Sticky FPD_FLAG_* bits of the instance (synchronises)."""
        return fpd_flags(self.h)

    def fields(self, out=None):
        """(u_x, u_y, rho), each ny x nx float64.  out: three such C-contiguous
        arrays to fill instead of new ones (e.g. views of page-locked host
        memory, which the device copies into several times faster)."""
        if out is None:
            out = tuple(np.zeros((self.ny, self.nx)) for _ in range(3))
        for a in out:
            if a.shape != (self.ny, self.nx) or a.dtype != np.float64 or not a.flags.c_contiguous:
                raise ValueError("fields(out=...) needs three C-contiguous float64 arrays of ny x nx")
        ux, uy, rho = out
        fpd_read_fields(self.h, ux, uy, rho)
        return ux, uy, rho

    def beads(self):
        n = max(self.nb, 1)
        R = np.zeros((n, 2)); V = np.zeros((n, 2)); F = np.zeros((n, 2)); S = np.zeros(n)
        fpd_read_beads(self.h, R, V, F, S)
        k = self.nb
        return R[:k], V[:k], F[:k], S[:k]

    def read_beads_async(self, buf) -> int:
        """Queue a copy of the current bead table into buf (a C-contiguous
        float64 host array or tensor of 7 * nb values: R_x, R_y, V_x, V_y,
        F_x, F_y, S, each nb long) and return a ticket for wait_read; buf
        must stay alive until then."""
        if isinstance(buf, np.ndarray):
            assert buf.dtype == np.float64 and buf.flags["C_CONTIGUOUS"] and buf.size >= 7 * self.nb
            ptr = buf.ctypes.data
        else:  # a torch tensor (pinned host memory keeps the copy asynchronous)
            assert buf.dtype.is_floating_point and buf.element_size() == 8 and buf.is_contiguous()
            assert not buf.is_cuda and buf.numel() >= 7 * self.nb
            ptr = buf.data_ptr()
        return fpd_read_beads_async(self.h, ptr)

    def wait_read(self, ticket: int) -> None:
        fpd_wait_read(self.h, ticket)

    def export_beads(self, slots: int) -> None:
        """Have every following step's bead phase write its table into a
        host ring of `slots` entries (0: off); take it with take_beads."""
        fpd_export_beads(self.h, slots)

    def take_beads(self, n: int, dst: np.ndarray | None = None) -> np.ndarray:
        """The bead table after n completed steps from the export ring
        (7 * nb doubles: R_x, R_y, V_x, V_y, F_x, F_y, S)."""
        if dst is None:
            dst = np.empty(7 * self.nb)
        fpd_take_beads(self.h, n, dst)
        return dst

    def save(self, path: str):
        """Checkpoint the whole device state to a file."""
        fpd_save(self.h, path)

    def load(self, path: str):
        """Resume from a checkpoint written with the same parameters."""
        fpd_load(self.h, path)

    def internal_flow(self) -> np.ndarray:
        """eps_v of every bead (Sec. 3.2)."""
        out = np.zeros(max(self.nb, 1))
        fpd_internal_flow(self.h, out)
        return out[:self.nb]

    def populations(self):
        f = np.zeros((9, self.ny, self.nx))
        fpd_read_populations(self.h, f)
        return f

    def set_populations(self, f):
        f = np.ascontiguousarray(f, dtype=np.float64)
        assert f.shape == (9, self.ny, self.nx)
        fpd_write_populations(self.h, f)

    def diag(self):
        out = np.zeros(4)
        fpd_diag(self.h, out)
        return out

    def derived(self) -> dict:
        out = np.zeros(8)
        fpd_derived(self.h, out)
        keys = ["nu_f", "k_s", "k_b", "k_ev", "l0", "rcut", "gamma_dot", "bytes_per_cell"]
        return dict(zip(keys, out.tolist()))

    def set_tuning(self, variant: int):
        fpd_set_tuning(self.h, variant)

    def tuning(self) -> tuple[int, int]:
        return fpd_get_tuning(self.h)

    def set_profiling(self, on: bool):
        fpd_set_profiling(self.h, on)

    def kernel_times(self) -> dict:
        out = np.zeros(4)
        fpd_kernel_times(self.h, out)
        return dict(lattice_ms=out[0], lattice_launches=int(out[1]), bead_ms=out[2], bead_launches=int(out[3]))


# ------------------------------------------------------------ batches
def _bcheck(rc: int, b):
    if rc != FPD_OK:
        msg = load_library().fpd_batch_last_error(b)
        raise FpdError(rc, msg.decode() if msg else "")


def fpd_batch_create(precision: int, max_slots: int, pool_bytes: int, max_beads: int, stream=None):
    h = ctypes.c_void_p()
    rc = load_library().fpd_batch_create(int(precision), int(max_slots), int(pool_bytes), int(max_beads), stream,
                                         ctypes.byref(h))
    if rc != FPD_OK:
        raise FpdError(rc, "fpd_batch_create failed")
    return h


def fpd_batch_add(b, params: fpd_params, n_steps: int) -> int:
    slot = ctypes.c_int32(-1)
    _bcheck(load_library().fpd_batch_add(b, ctypes.byref(params), int(n_steps), ctypes.byref(slot)), b)
    return slot.value


def fpd_batch_run(b, max_steps: int) -> int:
    done = ctypes.c_int64(0)
    _bcheck(load_library().fpd_batch_run(b, int(max_steps), ctypes.byref(done)), b)
    return done.value


def fpd_batch_sync(b) -> None:
    _bcheck(load_library().fpd_batch_sync(b), b)


def fpd_batch_poll(b, capacity: int = 4096) -> list:
    arr = (ctypes.c_int32 * capacity)()
    n = ctypes.c_int32(0)
    _bcheck(load_library().fpd_batch_poll(b, arr, capacity, ctypes.byref(n)), b)
    return [arr[i] for i in range(n.value)]


def fpd_batch_slot_info(b, slot: int) -> dict:
    out = (ctypes.c_int64 * 6)()
    _bcheck(load_library().fpd_batch_slot_info(b, int(slot), out), b)
    return dict(nx=out[0], ny=out[1], beads=out[2], steps_done=out[3], steps_req=out[4], state=out[5])


def fpd_batch_read_fields(b, slot: int, ux, uy, rho) -> None:
    _bcheck(load_library().fpd_batch_read_fields(b, int(slot), _ptr(ux), _ptr(uy), _ptr(rho)), b)


def fpd_batch_read_beads(b, slot: int, pos, vel, force, support=None) -> None:
    _bcheck(load_library().fpd_batch_read_beads(b, int(slot), _ptr(pos), _ptr(vel), _ptr(force), _ptr(support)), b)


def fpd_batch_step(b, n: int) -> None:
    _bcheck(load_library().fpd_batch_step(b, int(n)), b)


def fpd_batch_read(b, slot: int, ux, uy, pos) -> None:
    _bcheck(load_library().fpd_batch_read(b, int(slot), _ptr(ux), _ptr(uy), _ptr(pos)), b)


def fpd_batch_read_populations(b, slot: int, f) -> None:
    _bcheck(load_library().fpd_batch_read_populations(b, int(slot), _ptr(f)), b)


def fpd_batch_remove(b, slot: int) -> None:
    _bcheck(load_library().fpd_batch_remove(b, int(slot)), b)


def fpd_batch_stats(b) -> dict:
    out = np.zeros(8)
    _bcheck(load_library().fpd_batch_stats(b, _ptr(out)), b)
    keys = ["running", "cells", "finished", "pool_used", "pool_bytes", "global_steps", "cell_updates", "beads"]
    return dict(zip(keys, out.tolist()))


def fpd_batch_last_error(b) -> str:
    msg = load_library().fpd_batch_last_error(b)
    return msg.decode() if msg else ""


def fpd_batch_destroy(b) -> None:
    if b is not None and b.value:
        load_library().fpd_batch_destroy(b)


class Batch:
    """Many FPD instances advanced together on the GPU (C ABI fpd_batch_*)."""

    def __init__(self, precision: int, max_slots: int, pool_bytes: int, max_beads: int, stream=None):
        if stream is None:
            import torch
            if not torch.cuda.is_available():
                raise RuntimeError("no CUDA device: the FPD library runs on the GPU only")
            stream = torch.cuda.current_stream().cuda_stream
        self.h = fpd_batch_create(precision, max_slots, pool_bytes, max_beads, stream)
        self.precision = precision

    def close(self):
        if getattr(self, "h", None) is not None:
            fpd_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def add(self, cfg: dict, n_steps: int) -> int:
        p, keep = params_from_config(cfg)
        return fpd_batch_add(self.h, p, n_steps)

    def run(self, max_steps: int) -> int:
        return fpd_batch_run(self.h, max_steps)

    def step(self, n: int):
        """Up to n steps of every active instance (fpd_batch_step)."""
        fpd_batch_step(self.h, n)

    def read(self, slot: int):
        """Velocity field and bead positions of a slot (fpd_batch_read)."""
        i = self.info(slot)
        ux = np.zeros((i["ny"], i["nx"])); uy = np.zeros_like(ux)
        R = np.zeros((max(i["beads"], 1), 2))
        fpd_batch_read(self.h, slot, ux, uy, R)
        return ux, uy, R[:i["beads"]]

    def sync(self):
        fpd_batch_sync(self.h)

    def poll(self) -> list:
        return fpd_batch_poll(self.h)

    def info(self, slot: int) -> dict:
        return fpd_batch_slot_info(self.h, slot)

    def flags(self, slot: int) -> int:
        """Sticky FPD_FLAG_* bits of a slot (synchronises)."""
        return fpd_batch_slot_flags(self.h, slot)

    def fields(self, slot: int):
        i = self.info(slot)
        ux = np.zeros((i["ny"], i["nx"])); uy = np.zeros_like(ux); rho = np.zeros_like(ux)
        fpd_batch_read_fields(self.h, slot, ux, uy, rho)
        return ux, uy, rho

    def beads(self, slot: int):
        i = self.info(slot)
        n = max(i["beads"], 1)
        R = np.zeros((n, 2)); V = np.zeros((n, 2)); F = np.zeros((n, 2)); S = np.zeros(n)
        fpd_batch_read_beads(self.h, slot, R, V, F, S)
        k = i["beads"]
        return R[:k], V[:k], F[:k], S[:k]

    def populations(self, slot: int):
        i = self.info(slot)
        f = np.zeros((9, i["ny"], i["nx"]))
        fpd_batch_read_populations(self.h, slot, f)
        return f

    def internal_flow(self, slot: int) -> np.ndarray:
        """eps_v of every bead of a slot (Sec. 3.2)."""
        n = self.info(slot)["beads"]
        out = np.zeros(max(n, 1))
        fpd_batch_internal_flow(self.h, slot, out)
        return out[:n]

    def remove(self, slot: int):
        fpd_batch_remove(self.h, slot)

    def stats(self) -> dict:
        return fpd_batch_stats(self.h)

    def set_tuning(self, variant: int):
        fpd_batch_set_tuning(self.h, variant)
