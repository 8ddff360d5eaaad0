"""Python access to the FP64 CPU oracle (``sph_oracle.cpp``).

TEST INFRASTRUCTURE ONLY: the tests, the package smoke check and the CPU-baseline arm
of ``bench.py`` are the only users.  The product path (the CUDA library and its
binding) never imports this module, and this module imports nothing from it.

The shared library is compiled on first use with g++ (-O2 -ffp-contract=off) into
``oracle/_build/``; ``build()`` does the same explicitly.
"""

from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "sph_oracle.cpp")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "libsphoracle.so")
_lock = threading.Lock()
_lib = None

CXXFLAGS = ["-O2", "-std=c++17", "-ffp-contract=off", "-fPIC", "-shared", "-pthread"]


def build(force: bool = False) -> str:
    os.makedirs(_OUT_DIR, exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(["g++", *CXXFLAGS, "-o", tmp, _SRC])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = ctypes.CDLL(build())
            i64, i32, dbl = ctypes.c_int64, ctypes.c_int, ctypes.c_double
            P = ctypes.c_void_p
            L.orc_hilbert_cells.argtypes = [i64, P, P, P, i32, P]
            L.orc_hilbert_keys.argtypes = [i64, P, P, P, P]
            L.orc_stable_order.argtypes = [i64, P, P]
            L.orc_kernel.argtypes = [i64, P, P, P, P, P]
            L.orc_kernel.restype = None
            L.orc_pair_r2.argtypes = [i64, P, P, P, i64, P, P, P]
            L.orc_pair_r2.restype = None
            L.orc_ngb_sets.argtypes = [i64, P, P, P, P, i32, i64, P, i32, P, P]
            L.orc_density.argtypes = [i64, P, P, P, P, P, i64, P, i32, P, P, P, P, P]
            L.orc_density_iterate.argtypes = [i64, P, P, P, P, P, i64, P, dbl, dbl, i32, i32,
                                              P, P, P, P, P, P]
            L.orc_density_iterate.restype = i64
            L.orc_hydro.argtypes = [i64, P, P, P, P, P, P, P, P, P, P, P, i64, P, dbl, dbl, dbl,
                                    dbl, i32, P, P, P, P, P, P]
            L.orc_balsara.argtypes = [i64, P, P, P, P, dbl, P]
            L.orc_threads.argtypes = []
            L.orc_density_grouped.argtypes = [i64, P, P, P, P, P, i64, P, i32, P, P, P, P, P, P]
            L.orc_hydro_grouped.argtypes = [i64, P, P, P, P, P, P, P, P, P, P, P, i64, P, i32, dbl, dbl,
                                            dbl, dbl, P, P, P, P, P, P]
            L.orc_velocity_derivs.argtypes = [i64, P, P, P, P, P, P, P, i64, P, i32, P, P]
            L.orc_h_exact.argtypes = [i64, P, P, P, P, P, dbl, i32]
            L.orc_loss_grad.argtypes = [i64, P, P, P, P, P, P, P, P, P, dbl, dbl, dbl, dbl, dbl, i32,
                                        P, P, P, P]
            L.orc_grad_dual.argtypes = [i64, P, P, P, P, P, P, P, P, P, dbl, dbl, dbl, dbl, dbl, P, P, P]
            _lib = L
    return _lib


def _p(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _xyz(pos):
    pos = np.asarray(pos, dtype=np.float64)
    return _f64(pos[:, 0]), _f64(pos[:, 1]), _f64(pos[:, 2])


def threads() -> int:
    return int(lib().orc_threads())


def hilbert_cells(cells: np.ndarray, bits: int) -> np.ndarray:
    c = np.ascontiguousarray(cells, dtype=np.uint32)
    cx, cy, cz = (np.ascontiguousarray(c[:, a]) for a in range(3))
    out = np.empty(len(c), dtype=np.uint64)
    rc = lib().orc_hilbert_cells(len(c), _p(cx), _p(cy), _p(cz), bits, _p(out))
    if rc != 0:
        raise ValueError("bits out of range")
    return out


def hilbert_keys(pos: np.ndarray) -> np.ndarray:
    x, y, z = _xyz(pos)
    out = np.empty(len(x), dtype=np.uint64)
    if lib().orc_hilbert_keys(len(x), _p(x), _p(y), _p(z), _p(out)) != 0:
        raise ValueError("positions must lie in [0, 1)")
    return out


def stable_order(keys: np.ndarray) -> np.ndarray:
    k = np.ascontiguousarray(keys, dtype=np.uint64)
    perm = np.empty(len(k), dtype=np.int32)
    lib().orc_stable_order(len(k), _p(k), _p(perm))
    return perm


def kernel(r, h):
    r = _f64(np.atleast_1d(r))
    h = _f64(np.broadcast_to(h, r.shape))
    w, dwdr, dwdh = (np.empty_like(r) for _ in range(3))
    lib().orc_kernel(len(r), _p(r), _p(h), _p(w), _p(dwdr), _p(dwdh))
    return w, dwdr, dwdh


def pair_r2(pos, pi, pj):
    x, y, z = _xyz(pos)
    pi = np.ascontiguousarray(pi, dtype=np.int32)
    pj = np.ascontiguousarray(pj, dtype=np.int32)
    out = np.empty(len(pi))
    lib().orc_pair_r2(len(x), _p(x), _p(y), _p(z), len(pi), _p(pi), _p(pj), _p(out))
    return out


DENSITY, HYDRO = 0, 1


def ngb_sets(pos, h, targets=None, kind=DENSITY, use_tree=True):
    """CSR (offsets, idx) of neighbour sets; idx ascending particle indices per target."""
    x, y, z = _xyz(pos)
    n = len(x)
    h = _f64(h)
    t = np.arange(n, dtype=np.int32) if targets is None else np.ascontiguousarray(targets, dtype=np.int32)
    off = np.zeros(len(t) + 1, dtype=np.int64)
    L = lib()
    L.orc_ngb_sets(n, _p(x), _p(y), _p(z), _p(h), kind, len(t), _p(t), int(use_tree), _p(off), None)
    idx = np.empty(int(off[-1]), dtype=np.int32)
    L.orc_ngb_sets(n, _p(x), _p(y), _p(z), _p(h), kind, len(t), _p(t), int(use_tree), _p(off), _p(idx))
    return off, idx


def density(pos, m, h, targets=None, use_tree=True):
    x, y, z = _xyz(pos)
    n = len(x)
    m, h = _f64(m), _f64(h)
    t = np.arange(n, dtype=np.int32) if targets is None else np.ascontiguousarray(targets, dtype=np.int32)
    nt = len(t)
    rho, drhodh, f, neff = (np.empty(nt) for _ in range(4))
    nngb = np.empty(nt, dtype=np.int32)
    lib().orc_density(n, _p(x), _p(y), _p(z), _p(m), _p(h), nt, _p(t), int(use_tree), _p(rho),
                      _p(drhodh), _p(f), _p(neff), _p(nngb))
    return {"rho": rho, "drhodh": drhodh, "f": f, "neff": neff, "nngb": nngb}


def density_iterate(pos, m, h_init, targets=None, nngb=64.0, dn=2.0, max_iter=100, use_tree=True):
    """Iterates h of the targets; returns (h (all particles), dict of per-target outputs)."""
    x, y, z = _xyz(pos)
    n = len(x)
    m = _f64(m)
    h = _f64(np.array(h_init, dtype=np.float64, copy=True))
    t = np.arange(n, dtype=np.int32) if targets is None else np.ascontiguousarray(targets, dtype=np.int32)
    nt = len(t)
    rho, drhodh, f, neff = (np.empty(nt) for _ in range(4))
    nn = np.empty(nt, dtype=np.int32)
    iters = np.empty(nt, dtype=np.int32)
    failed = lib().orc_density_iterate(n, _p(x), _p(y), _p(z), _p(m), _p(h), nt, _p(t), nngb, dn,
                                       max_iter, int(use_tree), _p(rho), _p(drhodh), _p(f),
                                       _p(neff), _p(nn), _p(iters))
    return h, {"rho": rho, "drhodh": drhodh, "f": f, "neff": neff, "nngb": nn, "iters": iters,
               "failed": int(failed)}


def hydro(pos, vel, m, h, rho, f, u, targets=None, gamma=5.0 / 3.0, alpha=1.0, beta=2.0,
          eps=0.01, use_tree=True, fbal=None):
    """Accelerations and du/dt of the targets; fbal (n,) scales every pair's viscosity by
    the pair mean of the limiter (Balsara's switch, see balsara), None for the plain form."""
    x, y, z = _xyz(pos)
    vx, vy, vz = _xyz(vel)
    n = len(x)
    m, h, rho, f, u = (_f64(a) for a in (m, h, rho, f, u))
    fb = None if fbal is None else _f64(fbal)
    t = np.arange(n, dtype=np.int32) if targets is None else np.ascontiguousarray(targets, dtype=np.int32)
    nt = len(t)
    ax, ay, az, dudt = (np.empty(nt) for _ in range(4))
    nn = np.empty(nt, dtype=np.int32)
    lib().orc_hydro(n, _p(x), _p(y), _p(z), _p(vx), _p(vy), _p(vz), _p(m), _p(h), _p(rho), _p(f),
                    _p(u), nt, _p(t), gamma, alpha, beta, eps, int(use_tree), _p(ax), _p(ay),
                    _p(az), _p(dudt), _p(nn), None if fb is None else _p(fb))
    return {"acc": np.stack([ax, ay, az], axis=1), "dudt": dudt, "nngb": nn}


def balsara(divv, curl, u, h, gamma=5.0 / 3.0):
    """Balsara's limiter |div v| / (|div v| + |curl v| + 1e-4 c / h) of every particle."""
    divv, u, h = _f64(divv), _f64(u), _f64(h)
    curl = _f64(np.asarray(curl).reshape(-1, 3))
    out = np.empty(len(divv))
    lib().orc_balsara(len(divv), _p(divv), _p(curl), _p(u), _p(h), gamma, _p(out))
    return out


def curve_order(pos, targets=None):
    """The targets (all particles by default) in the order of the curve (stable)."""
    order = stable_order(hilbert_keys(pos))
    if targets is None:
        return order.astype(np.int32)
    keep = np.zeros(len(order), dtype=bool)
    keep[np.asarray(targets)] = True
    return order[keep[order]].astype(np.int32)


def density_grouped(pos, m, h, g, targets=None):
    """Grouped density (Sec. 2.1): the targets in curve order, g consecutive per group,
    one superset walk per group.  Returns the per-target outputs of ``density`` in the
    order of ``targets`` (ascending indices when None) and the walk statistics."""
    x, y, z = _xyz(pos)
    n = len(x)
    m, h = _f64(m), _f64(h)
    ordered = curve_order(pos, targets)
    nt = len(ordered)
    rho, drhodh, f, neff = (np.empty(nt) for _ in range(4))
    nngb = np.empty(nt, dtype=np.int32)
    stats = np.zeros(3, dtype=np.int64)
    rc = lib().orc_density_grouped(n, _p(x), _p(y), _p(z), _p(m), _p(h), nt, _p(ordered), int(g), _p(rho),
                                   _p(drhodh), _p(f), _p(neff), _p(nngb), _p(stats))
    if rc != 0:
        raise ValueError("group size must be >= 1")
    back = _back_to_targets(ordered, targets, n)
    out = {"rho": rho, "drhodh": drhodh, "f": f, "neff": neff, "nngb": nngb}
    out = {k: v[back] for k, v in out.items()}
    out.update(walks=int(stats[0]), candidates=int(stats[1]), pair_tests=int(stats[2]))
    return out


def hydro_grouped(pos, vel, m, h, rho, f, u, g, targets=None, gamma=5.0 / 3.0, alpha=1.0, beta=2.0, eps=0.01):
    """Grouped hydro (Sec. 2.1, symmetric criterion); outputs as ``hydro``, in the order of
    ``targets``, plus the walk statistics."""
    x, y, z = _xyz(pos)
    vx, vy, vz = _xyz(vel)
    n = len(x)
    m, h, rho, f, u = (_f64(a) for a in (m, h, rho, f, u))
    ordered = curve_order(pos, targets)
    nt = len(ordered)
    ax, ay, az, dudt = (np.empty(nt) for _ in range(4))
    nn = np.empty(nt, dtype=np.int32)
    stats = np.zeros(3, dtype=np.int64)
    rc = lib().orc_hydro_grouped(n, _p(x), _p(y), _p(z), _p(vx), _p(vy), _p(vz), _p(m), _p(h), _p(rho), _p(f),
                                 _p(u), nt, _p(ordered), int(g), gamma, alpha, beta, eps, _p(ax), _p(ay), _p(az),
                                 _p(dudt), _p(nn), _p(stats))
    if rc != 0:
        raise ValueError("group size must be >= 1")
    back = _back_to_targets(ordered, targets, n)
    return {"acc": np.stack([ax, ay, az], axis=1)[back], "dudt": dudt[back], "nngb": nn[back],
            "walks": int(stats[0]), "candidates": int(stats[1]), "pair_tests": int(stats[2])}


def _back_to_targets(ordered, targets, n):
    """Positions in ``ordered`` of every entry of ``targets`` (or of 0 .. n-1)."""
    where = np.full(n, -1, dtype=np.int64)
    where[ordered] = np.arange(len(ordered))
    t = np.arange(n) if targets is None else np.asarray(targets)
    return where[t]


def velocity_derivs(pos, vel, m, h, rho, targets=None, use_tree=True):
    """Divergence (nt,) and curl (nt, 3) of the velocity at the targets (density sets)."""
    x, y, z = _xyz(pos)
    n = len(x)
    v = _f64(np.asarray(vel).reshape(n, 3))
    t = np.arange(n, dtype=np.int32) if targets is None else np.ascontiguousarray(targets, dtype=np.int32)
    divv = np.empty(len(t))
    curl = np.empty((len(t), 3))
    lib().orc_velocity_derivs(n, _p(x), _p(y), _p(z), _p(v), _p(_f64(m)), _p(_f64(h)), _p(_f64(rho)), len(t),
                              _p(t), int(use_tree), _p(divv), _p(curl))
    return divv, curl


# ----------------------------------------------------------------------------- backward

def h_exact(pos, m, h, nngb=64.0, use_tree=True):
    """Smoothing lengths satisfying (4 pi/3) h^3 rho = nngb m exactly (from the given h)."""
    x, y, z = _xyz(pos)
    hh = _f64(np.array(h, dtype=np.float64, copy=True))
    lib().orc_h_exact(len(x), _p(x), _p(y), _p(z), _p(_f64(m)), _p(hh), nngb, int(use_tree))
    return hh


def loss_grad(pos, vel, m, u, h, w, s, nngb=64.0, gamma=5.0 / 3.0, alpha=1.0, beta=2.0, eps=0.01,
              use_tree=True):
    """L = sum w.a + sum s rho and dL/d(pos, vel, m) by the hand-written FP64 adjoint
    (h must satisfy the exact constraint, see h_exact)."""
    x, y, z = _xyz(pos)
    n = len(x)
    v = _f64(np.asarray(vel).reshape(n, 3))
    w = _f64(np.asarray(w).reshape(n, 3))
    loss = np.zeros(1)
    gx, gv = np.zeros((n, 3)), np.zeros((n, 3))
    gm = np.zeros(n)
    lib().orc_loss_grad(n, _p(x), _p(y), _p(z), _p(v), _p(_f64(m)), _p(_f64(u)), _p(_f64(h)), _p(w),
                        _p(_f64(s)), nngb, gamma, alpha, beta, eps, int(use_tree), _p(loss), _p(gx),
                        _p(gv), _p(gm))
    return float(loss[0]), gx, gv, gm


def grad_dual(pos, vel, m, u, h, w, s, nngb=64.0, gamma=5.0 / 3.0, alpha=1.0, beta=2.0, eps=0.01):
    """The same gradient by forward-mode dual numbers (small n: one pass per input)."""
    x, y, z = _xyz(pos)
    n = len(x)
    v = _f64(np.asarray(vel).reshape(n, 3))
    w = _f64(np.asarray(w).reshape(n, 3))
    gx, gv = np.zeros((n, 3)), np.zeros((n, 3))
    gm = np.zeros(n)
    lib().orc_grad_dual(n, _p(x), _p(y), _p(z), _p(v), _p(_f64(m)), _p(_f64(u)), _p(_f64(h)), _p(w),
                        _p(_f64(s)), nngb, gamma, alpha, beta, eps, _p(gx), _p(gv), _p(gm))
    return gx, gv, gm
