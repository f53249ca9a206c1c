"""ctypes binding of the C oracle plus the grid-method structures in numpy.

Test infrastructure only (see the package docstring).  Every function follows
a passage of Watanabe, Suzuki and Ito, "Efficient Implementations of Molecular
Dynamics Simulations for Lennard-Jones Systems", cited in its docstring.
Arrays are float64 (N, 3) for positions/velocities/forces.
"""
from __future__ import annotations

import ctypes
import math
from dataclasses import dataclass

import numpy as np

from .build import build as _build

_LIB = None
_D = ctypes.c_double
_I64 = ctypes.c_int64
_U64 = ctypes.c_uint64
_P = ctypes.c_void_p

TRUNC_QUADRATIC = 0  # Eq. 2
TRUNC_SHIFT = 1      # constant shift only (Sec. 2.1, c2 = 0)
TRUNC_CUT = 2        # plain cut of Eq. 1


def lib():
    """Load (building first if needed) the oracle shared library."""
    global _LIB
    if _LIB is None:
        L = ctypes.CDLL(_build())
        sig = {
            "or_num_threads": (ctypes.c_int, []),
            "or_set_threads": (None, [ctypes.c_int]),
            "or_trunc_coeffs": (None, [_D, ctypes.c_int, _P, _P]),
            "or_v_raw": (_D, [_D, _D, _D]),
            "or_f_raw": (_D, [_D, _D, _D]),
            "or_pair_v": (_D, [_D, _D, _D, _D, _D, _D]),
            "or_pair_f": (_D, [_D, _D, _D, _D, _D]),
            "or_fcc_lattice": (_D, [_I64, _D, _P]),
            "or_splitmix_at": (_U64, [_U64, _U64]),
            "or_gaussian_raw": (None, [_I64, _U64, _P]),
            "or_init_velocities": (None, [_I64, _D, _U64, _P]),
            "or_forces": (None, [_I64, _P, _D, _D, _D, _D, _D, _D, _P, _P, _P]),
            "or_forces_sample": (None, [_I64, _P, _D, _D, _D, _D, _D, _P, _I64, _P]),
            "or_kinetic": (_D, [_I64, _P]),
            "or_vv_run": (None, [_I64, _P, _P, _P, _D, _D, _D, _D, _D, _D, _D, _I64, _P, _P, _P]),
            "or_pairs_within": (_I64, [_I64, _P, _D, _D, _P, _I64]),
            "or_neighbor_counts": (None, [_I64, _P, _D, _D, _P]),
            "or_hvp": (None, [_I64, _P, _D, _D, _D, _D, _D, _D, _P, _P]),
            "or_hessian": (None, [_I64, _P, _D, _D, _D, _D, _D, _D, _P]),
            "or_param_derivs": (None, [_I64, _P, _D, _D, _D, _D, _D, _D, _P, _P, _P]),
            "or_traj_loss_grad": (None, [_I64, _P, _P, _D, _D, _D, _D, _D, _D, _D, _I64, _I64,
                                         _P, _P, _P, _P]),
            "or_traj_loss": (_D, [_I64, _P, _P, _D, _D, _D, _D, _D, _D, _D, _I64, _I64]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _LIB = L
    return _LIB


def _ptr(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _f64(a, shape=None):
    a = np.ascontiguousarray(a, dtype=np.float64)
    if shape is not None:
        a = a.reshape(shape)
    return a


def num_threads() -> int:
    return lib().or_num_threads()


def set_threads(n: int) -> None:
    lib().or_set_threads(int(n))


@dataclass(frozen=True)
class LJParams:
    """Potential parameters: eps, sigma, rc = rc_over_sigma * sigma, truncation mode."""
    eps: float = 1.0
    sigma: float = 1.0
    rc_over_sigma: float = 2.5
    mode: int = TRUNC_QUADRATIC

    @property
    def rc(self) -> float:
        return self.rc_over_sigma * self.sigma

    @property
    def coeffs(self):
        return trunc_coeffs(self.rc_over_sigma, self.mode)

    def args(self):
        c2, c0 = self.coeffs
        return self.eps, self.sigma, self.rc, c2, c0


def trunc_coeffs(rc_over_sigma: float, mode: int = TRUNC_QUADRATIC):
    """c2, c0 of Eq. 2 from V(rc) = V'(rc) = 0 (Sec. 2.1); shift-only / cut variants."""
    c2, c0 = _D(), _D()
    lib().or_trunc_coeffs(float(rc_over_sigma), int(mode), ctypes.byref(c2), ctypes.byref(c0))
    return c2.value, c0.value


def v_raw(r, eps=1.0, sigma=1.0):
    """Eq. 1, untruncated LJ potential."""
    return lib().or_v_raw(float(r), float(eps), float(sigma))


def f_raw(r, eps=1.0, sigma=1.0):
    """-dV/dr of Eq. 1."""
    return lib().or_f_raw(float(r), float(eps), float(sigma))


def pair_v(r2, p: LJParams = LJParams()):
    """Eq. 2 truncated potential at squared distance r2 (0 beyond rc)."""
    eps, sigma, rc, c2, c0 = p.args()
    return lib().or_pair_v(float(r2), eps, sigma, rc, c2, c0)


def pair_f(r2, p: LJParams = LJParams()):
    """Alg. 6 force coefficient f: force on i from j is f (q_j - q_i)."""
    eps, sigma, rc, c2, _ = p.args()
    return lib().or_pair_f(float(r2), eps, sigma, rc, c2)


def fcc_lattice(M: int, rho: float):
    """FCC start (Sec. 4.5): M^3 cells x 4 sites at density rho. Returns (x[N,3], L)."""
    N = 4 * M ** 3
    x = np.empty((N, 3), dtype=np.float64)
    L = lib().or_fcc_lattice(int(M), float(rho), _ptr(x))
    return x, L


def splitmix_at(seed: int, k: int) -> int:
    """Draw k of the counter-based SplitMix64 stream `seed`."""
    return int(lib().or_splitmix_at(ctypes.c_uint64(seed & (2 ** 64 - 1)), ctypes.c_uint64(k)))


def gaussian_raw(N: int, seed: int):
    v = np.empty((N, 3), dtype=np.float64)
    lib().or_gaussian_raw(int(N), ctypes.c_uint64(seed & (2 ** 64 - 1)), _ptr(v))
    return v


def init_velocities(N: int, T: float, seed: int):
    """Gaussian velocities at T with zero total momentum, sum v^2 = 3(N-1)T."""
    v = np.empty((N, 3), dtype=np.float64)
    lib().or_init_velocities(int(N), float(T), ctypes.c_uint64(seed & (2 ** 64 - 1)), _ptr(v))
    return v


def forces(x, L: float, p: LJParams = LJParams()):
    """All-pairs forces, PE and virial W = sum_{i<j} r_ij . F_ij. Returns (F, pe, vir)."""
    x = _f64(x, (-1, 3))
    N = x.shape[0]
    F = np.empty_like(x)
    pe, vir = _D(), _D()
    eps, sigma, rc, c2, c0 = p.args()
    lib().or_forces(N, _ptr(x), float(L), eps, sigma, rc, c2, c0, _ptr(F), ctypes.byref(pe), ctypes.byref(vir))
    return F, pe.value, vir.value


def forces_sample(x, L: float, idx, p: LJParams = LJParams()):
    """Forces on the particles idx only (same all-pairs sum)."""
    x = _f64(x, (-1, 3))
    idx = np.ascontiguousarray(idx, dtype=np.int64)
    F = np.empty((idx.shape[0], 3), dtype=np.float64)
    eps, sigma, rc, c2, _ = p.args()
    lib().or_forces_sample(x.shape[0], _ptr(x), float(L), eps, sigma, rc, c2, _ptr(idx), idx.shape[0], _ptr(F))
    return F


def kinetic(v) -> float:
    v = _f64(v, (-1, 3))
    return lib().or_kinetic(v.shape[0], _ptr(v))


def vv_run(x, v, L: float, dt: float, nsteps: int, p: LJParams = LJParams()):
    """nsteps of velocity-Verlet (unwrapped positions). Returns (x, v, F, pe_t, ke_t, vir_t)."""
    x = _f64(x, (-1, 3)).copy()
    v = _f64(v, (-1, 3)).copy()
    F, _, _ = forces(x, L, p)
    pe_t = np.zeros(nsteps)
    ke_t = np.zeros(nsteps)
    vir_t = np.zeros(nsteps)
    eps, sigma, rc, c2, c0 = p.args()
    lib().or_vv_run(x.shape[0], _ptr(x), _ptr(v), _ptr(F), float(L), eps, sigma, rc, c2, c0, float(dt),
                    int(nsteps), _ptr(pe_t), _ptr(ke_t), _ptr(vir_t))
    return x, v, F, pe_t, ke_t, vir_t


def pairs_within(x, L: float, rs: float):
    """Brute-force pair set {(i, j): i < j, r_ij < rs}, lexicographic, int64 (P, 2)."""
    x = _f64(x, (-1, 3))
    N = x.shape[0]
    n = lib().or_pairs_within(N, _ptr(x), float(L), float(rs), None, 0)
    ij = np.empty((max(n, 1), 2), dtype=np.int64)
    lib().or_pairs_within(N, _ptr(x), float(L), float(rs), _ptr(ij), n)
    return ij[:n]


def neighbor_counts(x, L: float, rs: float):
    """Number of partners within rs of each particle (both directions)."""
    x = _f64(x, (-1, 3))
    cnt = np.empty(x.shape[0], dtype=np.int64)
    lib().or_neighbor_counts(x.shape[0], _ptr(x), float(L), float(rs), _ptr(cnt))
    return cnt


def hvp(x, L: float, w, p: LJParams = LJParams()):
    """Hessian of the potential energy times w (pairs within rc)."""
    x = _f64(x, (-1, 3))
    w = _f64(w, (-1, 3))
    out = np.empty_like(x)
    eps, sigma, rc, c2, c0 = p.args()
    lib().or_hvp(x.shape[0], _ptr(x), float(L), eps, sigma, rc, c2, c0, _ptr(w), _ptr(out))
    return out


def hessian(x, L: float, p: LJParams = LJParams()):
    """Dense (3N, 3N) Hessian of the potential energy (small N only)."""
    x = _f64(x, (-1, 3))
    N = x.shape[0]
    H = np.empty((3 * N, 3 * N), dtype=np.float64)
    eps, sigma, rc, c2, c0 = p.args()
    lib().or_hessian(N, _ptr(x), float(L), eps, sigma, rc, c2, c0, _ptr(H))
    return H


def param_derivs(x, L: float, p: LJParams = LJParams(), lam=None):
    """(dPE/deps, dPE/dsigma) and, if lam is given, (lam.dF/deps, lam.dF/dsigma)."""
    x = _f64(x, (-1, 3))
    lam_a = None if lam is None else _f64(lam, (-1, 3))
    dpe = np.zeros(2)
    vjp = np.zeros(2)
    eps, sigma, rc, c2, c0 = p.args()
    lib().or_param_derivs(x.shape[0], _ptr(x), float(L), eps, sigma, rc, c2, c0, _ptr(lam_a), _ptr(dpe),
                          _ptr(vjp))
    return dpe, (None if lam is None else vjp)


def traj_loss_grad(x0, v0, L: float, dt: float, nsteps: int, n_pe: int, p: LJParams = LJParams()):
    """Loss = mean over the last n_pe steps of PE/N + MSD at the end; exact FP64 adjoint.

    Returns (loss, g_x0[N,3], g_v0[N,3], (dloss/deps, dloss/dsigma)).
    """
    x0 = _f64(x0, (-1, 3))
    v0 = _f64(v0, (-1, 3))
    gx = np.empty_like(x0)
    gv = np.empty_like(x0)
    gth = np.zeros(2)
    loss = _D()
    eps, sigma, rc, c2, c0 = p.args()
    lib().or_traj_loss_grad(x0.shape[0], _ptr(x0), _ptr(v0), float(L), eps, sigma, rc, c2, c0, float(dt),
                            int(nsteps), int(n_pe), ctypes.byref(loss), _ptr(gx), _ptr(gv), _ptr(gth))
    return loss.value, gx, gv, (gth[0], gth[1])


def traj_loss(x0, v0, L: float, dt: float, nsteps: int, n_pe: int, p: LJParams = LJParams()) -> float:
    """Forward-only loss of traj_loss_grad (for finite differences)."""
    x0 = _f64(x0, (-1, 3))
    v0 = _f64(v0, (-1, 3))
    eps, sigma, rc, c2, c0 = p.args()
    return lib().or_traj_loss(x0.shape[0], _ptr(x0), _ptr(v0), float(L), eps, sigma, rc, c2, c0, float(dt),
                              int(nsteps), int(n_pe))


# --------------------------------------------------------------------------
# Grid method (Sec. 2.2) and sorted pair list (Sec. 2.4) as plain definitions.
# --------------------------------------------------------------------------

def wrap(x, L: float):
    """Fold positions into [0, L) with one correction per component."""
    x = _f64(x, (-1, 3)).copy()
    x = np.where(x >= L, x - L, x)
    x = np.where(x < 0.0, x + L, x)
    return x


def cells_per_side(L: float, rs: float) -> int:
    """Largest n with cell side L/n >= rs (Sec. 2.2: cells no smaller than the search length)."""
    return int(math.floor(L / rs))


def cell_labels(x, L: float, n: int):
    """Serial cell label of each (wrapped) particle: c = (cx n + cy) n + cz, cx = floor(x n/L)."""
    x = _f64(x, (-1, 3))
    inv_h = n / L
    c = np.floor(x * inv_h).astype(np.int64)
    c = np.clip(c, 0, n - 1)
    return (c[:, 0] * n + c[:, 1]) * n + c[:, 2]


def grid_list(labels, ncells: int):
    """Counting sort of particles by cell label (Sec. 2.2, Fig. 3).

    Returns (GridParticleNumber[ncells], GridPointer[ncells+1], GridList[N]) with
    GridList the particle indices ordered by label, ties kept in index order.
    """
    labels = np.asarray(labels, dtype=np.int64)
    count = np.bincount(labels, minlength=ncells).astype(np.int64)
    pointer = np.zeros(ncells + 1, dtype=np.int64)
    np.cumsum(count, out=pointer[1:])
    order = np.argsort(labels, kind="stable")
    return count, pointer, order


def sorted_pair_list(pairs, N: int):
    """KeyPointer / SortedList of Sec. 2.4 (Fig. 6): partners grouped by key = lower index."""
    pairs = np.asarray(pairs, dtype=np.int64).reshape(-1, 2)
    key = np.minimum(pairs[:, 0], pairs[:, 1])
    partner = np.maximum(pairs[:, 0], pairs[:, 1])
    order = np.lexsort((partner, key))
    key, partner = key[order], partner[order]
    kp = np.zeros(N + 1, dtype=np.int64)
    np.cumsum(np.bincount(key, minlength=N), out=kp[1:])
    return kp, partner
