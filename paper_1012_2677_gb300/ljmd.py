"""Thin Python binding of libljmd (declared in include/ljmd.h).

Argument marshalling only: every step of the computation runs in the CUDA
kernels of libljmd.so.  Functions carry the C names (ljmd_create, ...);
``System`` wraps a handle.  Arrays may be numpy (host) or torch CUDA tensors
(device, passed by pointer); torch streams are passed as cudaStream_t.
There is no CPU fallback: if the library cannot be loaded, calls raise.
"""
from __future__ import annotations

import ctypes
import os
import re

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "lib", "libljmd.so")
HEADER = os.path.join(os.path.dirname(HERE), "include", "ljmd.h")

LJ_OK, LJ_EINVAL, LJ_ENOMEM, LJ_EDEVICE, LJ_ESTATE, LJ_ERANGE = 0, -1, -2, -3, -4, -5
LJ_FP64, LJ_MIXED = 0, 1
LJ_LIST_FULL, LJ_LIST_HALF, LJ_LIST_AUTO = 0, 1, 2
LJ_TRUNC_QUADRATIC, LJ_TRUNC_SHIFT, LJ_TRUNC_CUT = 0, 1, 2
LJ_VALID_HALF_MARGIN, LJ_VALID_DUTC, LJ_VALID_DUTC_LDC, LJ_VALID_HALF_MARGIN_LDC = 0, 1, 2, 3
LJ_PAIRS_STATIC_MAX_ENTRIES = 524288  # static scratch of ljmd_get_pairs_static, in list entries
LJ_ST_NONFINITE, LJ_ST_LIST_OVERFLOW, LJ_ST_TIMEOUT, LJ_ST_CELL_RANGE = 1, 2, 4, 8


class LjmdError(RuntimeError):
    def __init__(self, code: int, what: str):
        self.code = code
        super().__init__("%s failed: %s (%d)" % (what, ljmd_strerror(code) if _LIB else "?", code))


class ljmd_params(ctypes.Structure):
    _fields_ = [("eps", ctypes.c_double), ("sigma", ctypes.c_double), ("cutoff", ctypes.c_double),
                ("margin", ctypes.c_double), ("truncation", ctypes.c_int32), ("list_form", ctypes.c_int32),
                ("energy_every", ctypes.c_int32), ("lanes", ctypes.c_int32)]


class ljmd_stats(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("steps", ctypes.c_int64), ("rebuilds", ctypes.c_int64),
                ("list_entries", ctypes.c_int64), ("cells_per_side", ctypes.c_int64), ("box", ctypes.c_double),
                ("mean_lifetime", ctypes.c_double), ("max_displacement", ctypes.c_double),
                ("status_word", ctypes.c_int32), ("precision", ctypes.c_int32),
                ("kernel_launches", ctypes.c_int64), ("ldc_checks", ctypes.c_int64), ("ldc_kept", ctypes.c_int64),
                ("validity", ctypes.c_int32), ("list_form", ctypes.c_int32)]


class ljmd_profile(ctypes.Structure):
    _fields_ = [("force_ms", ctypes.c_double), ("force_launches", ctypes.c_int64),
                ("integrate_ms", ctypes.c_double), ("integrate_launches", ctypes.c_int64),
                ("rebuild_ms", ctypes.c_double), ("rebuilds", ctypes.c_int64),
                ("energy_ms", ctypes.c_double), ("energy_launches", ctypes.c_int64),
                ("adjoint_ms", ctypes.c_double), ("adjoint_launches", ctypes.c_int64)]


class ljmd_batch_stats(ctypes.Structure):
    _fields_ = [("replicas", ctypes.c_int64), ("n", ctypes.c_int64), ("steps", ctypes.c_int64),
                ("rebuilds", ctypes.c_int64), ("list_entries", ctypes.c_int64), ("tiles", ctypes.c_int64),
                ("cells", ctypes.c_int64), ("kernel_launches", ctypes.c_int64), ("status_word", ctypes.c_int32),
                ("tile_cells", ctypes.c_int32), ("lanes", ctypes.c_int32), ("pad", ctypes.c_int32)]


_LIB = None
_P = ctypes.c_void_p
_I32, _I64, _U64, _D = ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64, ctypes.c_double
_SIGS = {
    "ljmd_version": (ctypes.c_int, []),
    "ljmd_strerror": (ctypes.c_char_p, [ctypes.c_int]),
    "ljmd_create": (ctypes.c_int, [ctypes.POINTER(_P), ctypes.POINTER(ljmd_params), _I32, _P]),
    "ljmd_destroy": (None, [_P]),
    "ljmd_init_lattice": (ctypes.c_int, [_P, _I64, _D, _D, _U64]),
    "ljmd_set_state": (ctypes.c_int, [_P, _I64, _D, _P, _P, _I32]),
    "ljmd_get_state": (ctypes.c_int, [_P, _P, _P, _P, _P, _I32]),
    "ljmd_build_pairlist": (ctypes.c_int, [_P, _D, _D]),
    "ljmd_compute_forces": (ctypes.c_int, [_P]),
    "ljmd_step": (ctypes.c_int, [_P, _D, _I64]),
    "ljmd_energies": (ctypes.c_int, [_P, _P, _P, _P]),
    "ljmd_set_energy_log": (ctypes.c_int, [_P, _P, _I64]),
    "ljmd_get_pairs": (ctypes.c_int, [_P, _P, _I64, _P]),
    "ljmd_set_wait_budget": (ctypes.c_int, [_I64]),
    "ljmd_get_pairs_static": (ctypes.c_int, [_P, _P, _I64, _P]),
    "ljmd_hvp": (ctypes.c_int, [_P, _P, _P, _P, _I32]),
    "ljmd_set_validity": (ctypes.c_int, [_P, _I32, _I32]),
    "ljmd_batch_create": (ctypes.c_int, [ctypes.POINTER(_P), ctypes.POINTER(ljmd_params), _I32, _P, _P, _P]),
    "ljmd_batch_destroy": (None, [_P]),
    "ljmd_batch_set_state": (ctypes.c_int, [_P, _P, _P, _I32]),
    "ljmd_batch_step": (ctypes.c_int, [_P, _D, _I64, _I32]),
    "ljmd_batch_energies": (ctypes.c_int, [_P, _P, _P, _P]),
    "ljmd_batch_get_state": (ctypes.c_int, [_P, _P, _P, _P, _I32]),
    "ljmd_batch_get_pairs": (ctypes.c_int, [_P, _I32, _P, _I64, _P]),
    "ljmd_batch_get_stats": (ctypes.c_int, [_P, ctypes.POINTER(ljmd_batch_stats)]),
    "ljmd_batch_set_tuning": (ctypes.c_int, [_P, _I32, _I32]),
    "ljmd_batch_autotune": (ctypes.c_int, [_P, _I32, _P, _P, _P]),
    "ljmd_batch_time_force": (ctypes.c_int, [_P, _I32, _P]),
    "ljmd_traj_loss_grad": (ctypes.c_int, [_P, _I64, _D, _P, _P, _D, _I64, _I64, _I64, _P, _P, _P, _P, _I32]),
    "ljmd_get_stats": (ctypes.c_int, [_P, ctypes.POINTER(ljmd_stats)]),
    "ljmd_get_grid": (ctypes.c_int, [_P, _P, _I64, _P, _I64, _P]),
    "ljmd_set_profiling": (ctypes.c_int, [_P, _I32]),
    "ljmd_set_tuning": (ctypes.c_int, [_P, _I32, _I32, _I32, _I32]),
    "ljmd_get_profile": (ctypes.c_int, [_P, ctypes.POINTER(ljmd_profile)]),
}


def load(build_if_missing: bool = True):
    """Load libljmd.so (building it with nvcc first if it is missing or stale)."""
    global _LIB
    if _LIB is not None:
        return _LIB
    if build_if_missing:
        from .build import build
        build()  # compiles only if the library is missing or older than a source
    if not os.path.exists(LIB_PATH):
        raise OSError("libljmd.so is not built (%s); run paper_1012_2677_gb300/build.py" % LIB_PATH)
    lib = ctypes.CDLL(LIB_PATH)
    for name, (res, args) in _SIGS.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _LIB = lib
    return lib


def declared_symbols(header: str = HEADER):
    """Names of the functions declared in an include/*.h header."""
    txt = open(header).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(ljmd_\w+)\s*\(", txt)))


def _chk(code: int, what: str):
    if code != LJ_OK:
        raise LjmdError(code, what)


def _is_torch(a) -> bool:
    return type(a).__module__.startswith("torch")


def _arr_ptr(a, dtype, n_expected=None):
    """(pointer, on_device, keepalive) for a numpy array or torch tensor of the given dtype."""
    if a is None:
        return None, 0, None
    if _is_torch(a):
        import torch
        tdt = {np.float64: torch.float64, np.int32: torch.int32, np.int64: torch.int64}[dtype]
        if a.dtype != tdt or not a.is_contiguous():
            raise TypeError("tensor must be contiguous %s" % tdt)
        if n_expected is not None and a.numel() != n_expected:
            raise ValueError("tensor has %d elements, expected %d" % (a.numel(), n_expected))
        return ctypes.c_void_p(a.data_ptr()), 1 if a.is_cuda else 0, a
    arr = np.ascontiguousarray(a, dtype=dtype)
    if n_expected is not None and arr.size != n_expected:
        raise ValueError("array has %d elements, expected %d" % (arr.size, n_expected))
    return arr.ctypes.data_as(ctypes.c_void_p), 0, arr


# ---- C names -------------------------------------------------------------------------------------

def ljmd_version() -> int:
    return load().ljmd_version()


def ljmd_strerror(code: int) -> str:
    return load().ljmd_strerror(int(code)).decode()


def ljmd_create(params: ljmd_params, precision: int, stream=None):
    h = _P()
    s = _stream_handle(stream)
    _chk(load().ljmd_create(ctypes.byref(h), ctypes.byref(params), int(precision), s), "ljmd_create")
    return h


def ljmd_destroy(h) -> None:
    if h:
        load().ljmd_destroy(h)


def ljmd_init_lattice(h, cells_per_side: int, density: float, T: float, seed: int) -> None:
    _chk(load().ljmd_init_lattice(h, int(cells_per_side), float(density), float(T), int(seed) & (2 ** 64 - 1)),
         "ljmd_init_lattice")


def ljmd_set_state(h, n: int, box: float, x, v=None) -> None:
    px, dx, kx = _arr_ptr(x, np.float64, 3 * n)
    pv, dv, kv = _arr_ptr(v, np.float64, 3 * n)
    if v is not None and dv != dx:
        raise ValueError("x and v must both be host or both be device arrays")
    _chk(load().ljmd_set_state(h, int(n), float(box), px, pv, dx), "ljmd_set_state")


def ljmd_get_state(h, x=None, v=None, f=None, img=None, on_device: int = 0) -> None:
    ptrs = [_arr_ptr(a, dt)[0] for a, dt in ((x, np.float64), (v, np.float64), (f, np.float64), (img, np.int32))]
    _chk(load().ljmd_get_state(h, *ptrs, int(on_device)), "ljmd_get_state")


def ljmd_build_pairlist(h, cutoff: float, margin: float) -> None:
    _chk(load().ljmd_build_pairlist(h, float(cutoff), float(margin)), "ljmd_build_pairlist")


def ljmd_compute_forces(h) -> None:
    _chk(load().ljmd_compute_forces(h), "ljmd_compute_forces")


def ljmd_step(h, dt: float, nsteps: int) -> None:
    _chk(load().ljmd_step(h, float(dt), int(nsteps)), "ljmd_step")


def ljmd_energies(h):
    pe, ke, vir = _D(), _D(), _D()
    _chk(load().ljmd_energies(h, ctypes.byref(pe), ctypes.byref(ke), ctypes.byref(vir)), "ljmd_energies")
    return pe.value, ke.value, vir.value


def ljmd_set_energy_log(h, device_log_ptr, capacity: int) -> None:
    _chk(load().ljmd_set_energy_log(h, device_log_ptr, int(capacity)), "ljmd_set_energy_log")


def ljmd_get_pairs(h):
    n = _I64()
    _chk(load().ljmd_get_pairs(h, None, 0, ctypes.byref(n)), "ljmd_get_pairs")
    out = np.empty((max(n.value, 1), 2), dtype=np.int64)
    _chk(load().ljmd_get_pairs(h, out.ctypes.data_as(_P), n.value, ctypes.byref(n)), "ljmd_get_pairs")
    return out[:n.value]


def ljmd_get_pairs_static(h, cap=None):
    """Unique pairs of the current list through the allocation-free export (one call)."""
    if cap is None:
        cap = max(ljmd_get_stats(h)["list_entries"], 1)
    n = _I64()
    out = np.empty((max(cap, 1), 2), dtype=np.int64)
    _chk(load().ljmd_get_pairs_static(h, out.ctypes.data_as(_P), cap, ctypes.byref(n)), "ljmd_get_pairs_static")
    return out[:min(n.value, cap)], n.value


def ljmd_hvp(h, w, hw, dtheta=None) -> None:
    """hw = H(x) w (Hessian of the potential energy); dtheta (4 doubles, optional) =
    (w.dF/deps, w.dF/dsigma, dPE/deps, dPE/dsigma).  w, hw: both host or both device, 3N FP64."""
    pw, dw, kw = _arr_ptr(w, np.float64)
    ph, dh, kh = _arr_ptr(hw, np.float64)
    if dw != dh:
        raise ValueError("w and hw must both be host or both be device arrays")
    dth = np.zeros(4) if dtheta is None else dtheta
    _chk(load().ljmd_hvp(h, pw, ph, dth.ctypes.data_as(_P), dw), "ljmd_hvp")
    return dth


def ljmd_traj_loss_grad(h, n: int, box: float, x0, v0, dt: float, nsteps: int, n_pe: int, ckpt_every: int,
                        gx0=None, gv0=None):
    """Loss of the differentiable trajectory (mean PE/N over the last n_pe steps + MSD) and its
    gradients by the reverse-time pass with checkpoints every ckpt_every steps.  x0, v0 (and gx0,
    gv0 when given) are all host or all device arrays of 3n FP64.  Returns (loss, (deps, dsigma))."""
    px, dx, kx = _arr_ptr(x0, np.float64, 3 * n)
    pv, dv, kv = _arr_ptr(v0, np.float64, 3 * n)
    pgx, dgx, kgx = _arr_ptr(gx0, np.float64, 3 * n)
    pgv, dgv, kgv = _arr_ptr(gv0, np.float64, 3 * n)
    for d, a in ((dv, v0), (dgx, gx0), (dgv, gv0)):
        if a is not None and d != dx:
            raise ValueError("all arrays must be host or all device")
    loss = _D()
    gth = np.zeros(2)
    _chk(load().ljmd_traj_loss_grad(h, int(n), float(box), px, pv, float(dt), int(nsteps), int(n_pe),
                                    int(ckpt_every), ctypes.byref(loss), pgx, pgv, gth.ctypes.data_as(_P), dx),
         "ljmd_traj_loss_grad")
    return loss.value, (float(gth[0]), float(gth[1]))


def ljmd_get_grid(h, n: int):
    """(GridPointer[n_cells + 1], GridList[n]) of the last list construction, int64 numpy arrays."""
    nc = _I64()
    _chk(load().ljmd_get_grid(h, None, 0, None, 0, ctypes.byref(nc)), "ljmd_get_grid")
    ptr = np.empty(nc.value + 1, dtype=np.int64)
    lst = np.empty(max(n, 1), dtype=np.int64)
    _chk(load().ljmd_get_grid(h, ptr.ctypes.data_as(_P), ptr.size, lst.ctypes.data_as(_P), n, ctypes.byref(nc)),
         "ljmd_get_grid")
    return ptr, lst[:n]


def ljmd_get_stats(h) -> dict:
    st = ljmd_stats()
    _chk(load().ljmd_get_stats(h, ctypes.byref(st)), "ljmd_get_stats")
    return {name: getattr(st, name) for name, _ in ljmd_stats._fields_}


def ljmd_set_wait_budget(cycles: int) -> None:
    """Budget of the bounded device waits in SM clock cycles (0: the default); a test knob."""
    _chk(load().ljmd_set_wait_budget(int(cycles)), "ljmd_set_wait_budget")


def ljmd_set_tuning(h, tile_cells: int = 0, lanes: int = 0, force_ctas_per_sm: int = 0, force_buffers: int = 0) -> None:
    _chk(load().ljmd_set_tuning(h, int(tile_cells), int(lanes), int(force_ctas_per_sm), int(force_buffers)),
         "ljmd_set_tuning")


def ljmd_set_profiling(h, enable: bool) -> None:
    _chk(load().ljmd_set_profiling(h, 1 if enable else 0), "ljmd_set_profiling")


def ljmd_get_profile(h) -> dict:
    pr = ljmd_profile()
    _chk(load().ljmd_get_profile(h, ctypes.byref(pr)), "ljmd_get_profile")
    return {name: getattr(pr, name) for name, _ in ljmd_profile._fields_}


def _stream_handle(stream):
    if stream is None:
        return None
    if isinstance(stream, int):
        return ctypes.c_void_p(stream)
    return ctypes.c_void_p(int(stream.cuda_stream))  # torch.cuda.Stream


# ---- object wrapper ------------------------------------------------------------------------------

class System:
    """One LJ system on the current CUDA device (a handle of libljmd)."""

    def __init__(self, eps=1.0, sigma=1.0, cutoff=2.5, margin=0.5, truncation=LJ_TRUNC_QUADRATIC,
                 list_form=LJ_LIST_FULL, energy_every=1, lanes=0, precision=LJ_MIXED, stream=None):
        self.params = ljmd_params(eps, sigma, cutoff, margin, truncation, list_form, energy_every, lanes)
        self.precision = precision
        self._keep = []
        self.h = ljmd_create(self.params, precision, stream)
        self.n = 0
        self.box = 0.0

    def close(self):
        if getattr(self, "h", None):
            ljmd_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def init_lattice(self, cells_per_side, density, T, seed):
        ljmd_init_lattice(self.h, cells_per_side, density, T, seed)
        st = self.stats()
        self.n, self.box = st["n"], st["box"]

    def set_state(self, x, v=None, box=None):
        n = (x.numel() if _is_torch(x) else np.asarray(x).size) // 3
        ljmd_set_state(self.h, n, float(box), x, v)
        self.n, self.box = n, float(box)

    def get_state(self):
        """(x, v, f, img) as numpy arrays in id order."""
        x = np.empty((self.n, 3))
        v = np.empty((self.n, 3))
        f = np.empty((self.n, 3))
        img = np.empty((self.n, 3), dtype=np.int32)
        ljmd_get_state(self.h, x, v, f, img, 0)
        return x, v, f, img

    def build_pairlist(self, cutoff=None, margin=None):
        ljmd_build_pairlist(self.h, self.params.cutoff if cutoff is None else cutoff,
                            self.params.margin if margin is None else margin)

    def compute_forces(self):
        ljmd_compute_forces(self.h)

    def step(self, dt, nsteps=1):
        ljmd_step(self.h, dt, nsteps)

    def energies(self):
        return ljmd_energies(self.h)

    def pairs(self):
        return ljmd_get_pairs(self.h)

    def pairs_static(self, cap=None):
        """(pairs, npairs) from the allocation-free export; pairs holds the first min(cap, npairs)."""
        return ljmd_get_pairs_static(self.h, cap)

    def set_validity(self, mode, max_ld=0):
        """List-validity rule (LJ_VALID_*) and N_l of the large displacement check."""
        _chk(load().ljmd_set_validity(self.h, int(mode), int(max_ld)), "ljmd_set_validity")

    def hvp(self, w):
        """(H w, (w.dF/deps, w.dF/dsigma, dPE/deps, dPE/dsigma)) at the current positions, id order."""
        w = np.ascontiguousarray(w, dtype=np.float64)
        hw = np.empty_like(w)
        dth = ljmd_hvp(self.h, w, hw)
        return hw, tuple(float(t) for t in dth)

    def traj_loss_grad(self, x0, v0, box, dt, nsteps, n_pe, ckpt_every):
        """(loss, g_x0, g_v0, (dloss/deps, dloss/dsigma)) of the differentiable trajectory (host arrays)."""
        x0 = np.ascontiguousarray(x0, dtype=np.float64)
        v0 = np.ascontiguousarray(v0, dtype=np.float64)
        n = x0.size // 3
        gx = np.empty_like(x0)
        gv = np.empty_like(v0)
        loss, gth = ljmd_traj_loss_grad(self.h, n, box, x0, v0, dt, nsteps, n_pe, ckpt_every, gx, gv)
        self.n, self.box = n, float(box)
        return loss, gx, gv, gth

    def stats(self):
        return ljmd_get_stats(self.h)

    def grid(self):
        """(GridPointer, GridList) of the cell grid of the last list construction."""
        return ljmd_get_grid(self.h, self.n)

    def set_tuning(self, tile_cells=0, lanes=0, force_ctas_per_sm=0, force_buffers=0):
        ljmd_set_tuning(self.h, tile_cells, lanes, force_ctas_per_sm, force_buffers)

    def set_profiling(self, enable=True):
        ljmd_set_profiling(self.h, enable)

    def profile(self):
        return ljmd_get_profile(self.h)

    def set_energy_log(self, tensor):
        """Register a float64 CUDA tensor of shape (cap, 4) for (step, pe, ke, virial) records."""
        if tensor is None:
            ljmd_set_energy_log(self.h, None, 0)
            return
        self._keep = [tensor]
        ljmd_set_energy_log(self.h, ctypes.c_void_p(tensor.data_ptr()), tensor.shape[0])


# ---- batched replicas ----------------------------------------------------------------------------

class Batch:
    """Independent LJ systems of uneven size advanced together (ljmd_batch_*).  Replica r owns the
    particles [base_r, base_r + n[r]) of the concatenated arrays."""

    def __init__(self, n, box, eps=1.0, sigma=1.0, cutoff=2.5, margin=0.3, truncation=LJ_TRUNC_QUADRATIC, lanes=0,
                 stream=None):
        self.n = np.ascontiguousarray(n, dtype=np.int64)
        self.box = np.ascontiguousarray(box, dtype=np.float64)
        self.R = len(self.n)
        self.N = int(self.n.sum())
        self.base = np.concatenate([[0], np.cumsum(self.n)[:-1]]).astype(np.int64)
        self.params = ljmd_params(eps, sigma, cutoff, margin, truncation, LJ_LIST_FULL, 0, lanes)
        h = _P()
        _chk(load().ljmd_batch_create(ctypes.byref(h), ctypes.byref(self.params), self.R,
                                      self.n.ctypes.data_as(_P), self.box.ctypes.data_as(_P), _stream_handle(stream)),
             "ljmd_batch_create")
        self.h = h

    def close(self):
        if getattr(self, "h", None):
            load().ljmd_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def set_state(self, x, v=None):
        px, dx, kx = _arr_ptr(x, np.float64, 3 * self.N)
        pv, dv, kv = _arr_ptr(v, np.float64, 3 * self.N)
        if v is not None and dv != dx:
            raise ValueError("x and v must both be host or both be device arrays")
        _chk(load().ljmd_batch_set_state(self.h, px, pv, dx), "ljmd_batch_set_state")

    def step(self, dt, nsteps=1, graph_steps=0):
        _chk(load().ljmd_batch_step(self.h, float(dt), int(nsteps), int(graph_steps)), "ljmd_batch_step")

    def energies(self):
        pe, ke, vir = (np.empty(self.R) for _ in range(3))
        _chk(load().ljmd_batch_energies(self.h, pe.ctypes.data_as(_P), ke.ctypes.data_as(_P), vir.ctypes.data_as(_P)),
             "ljmd_batch_energies")
        return pe, ke, vir

    def get_state(self):
        x, v, f = (np.empty((self.N, 3)) for _ in range(3))
        _chk(load().ljmd_batch_get_state(self.h, x.ctypes.data_as(_P), v.ctypes.data_as(_P), f.ctypes.data_as(_P), 0),
             "ljmd_batch_get_state")
        return x, v, f

    def pairs(self, r):
        n = _I64()
        _chk(load().ljmd_batch_get_pairs(self.h, int(r), None, 0, ctypes.byref(n)), "ljmd_batch_get_pairs")
        out = np.empty((max(n.value, 1), 2), dtype=np.int64)
        _chk(load().ljmd_batch_get_pairs(self.h, int(r), out.ctypes.data_as(_P), n.value, ctypes.byref(n)),
             "ljmd_batch_get_pairs")
        return out[:n.value]

    def stats(self):
        st = ljmd_batch_stats()
        _chk(load().ljmd_batch_get_stats(self.h, ctypes.byref(st)), "ljmd_batch_get_stats")
        return {name: getattr(st, name) for name, _ in ljmd_batch_stats._fields_}

    def set_tuning(self, tile_cells=0, lanes=0):
        _chk(load().ljmd_batch_set_tuning(self.h, int(tile_cells), int(lanes)), "ljmd_batch_set_tuning")

    def time_force(self, trials=5):
        """Mean device time (ms) of one force launch over all replicas."""
        ms = _D()
        _chk(load().ljmd_batch_time_force(self.h, int(trials), ctypes.byref(ms)), "ljmd_batch_time_force")
        return ms.value

    def autotune(self, trials=5):
        t, l, ms = _I32(), _I32(), _D()
        _chk(load().ljmd_batch_autotune(self.h, int(trials), ctypes.byref(t), ctypes.byref(l), ctypes.byref(ms)),
             "ljmd_batch_autotune")
        return t.value, l.value, ms.value
