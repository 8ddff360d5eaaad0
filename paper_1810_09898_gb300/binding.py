"""ctypes binding of the C ABI in include/sphgrp.h (argument marshalling only).

Every function of the C ABI is exposed under its own name on the loaded library;
``Context`` wraps a ``sphgrp_ctx*`` and passes torch CUDA tensors as device pointers
on the current torch stream.
"""

from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
_LIB_PATH = os.path.join(HERE, "_build", "libsphgrp.so")

INDIVIDUAL, GROUPED = 0, 1
CENTRE_FIRST, CENTRE_BOX = 0, 1
ITER_PASSES, ITER_IN_GROUP, ITER_RECYCLE = 0, 1, 2
GROUP_COUNT, GROUP_RADIUS, GROUP_TREE = 0, 1, 2
DENSITY, HYDRO = 0, 1

EXPORTED = [
    "sphgrp_default_params",
    "sphgrp_last_error",
    "sphgrp_ctx_create",
    "sphgrp_ctx_destroy",
    "sphgrp_sfc_keys_sort",
    "sphgrp_tree_build",
    "sphgrp_ngb_search",
    "sphgrp_group_supersets",
    "sphgrp_density",
    "sphgrp_hydro_force",
    "sphgrp_velocity_derivs",
    "sphgrp_density_derivs",
    "sphgrp_key_split",
    "sphgrp_domain_boxes",
    "sphgrp_halo_select",
    "sphgrp_mask_compact",
    "sphgrp_hydro_force_balsara",
    "sphgrp_backward",
    "sphgrp_get_stats",
    "sphgrp_kernel_launches",
    "sphgrp_get_launch_log",
    "sphgrp_sfc_keys_sort_static",
    "sphgrp_batch_create",
    "sphgrp_batch_destroy",
    "sphgrp_batch_run",
    "sphgrp_batch_tune",
    "sphgrp_batch_get_config",
    "sphgrp_batch_set_config",
    "sphgrp_batch_stats",
]

BATCH_BACKWARD, BATCH_GRAPH = 1, 2
BATCH_CLASSES = 8
_IO_FIELDS = ("pos", "m", "vel", "u", "h", "active", "rho", "drhodh", "fgrad", "nngb", "acc", "dudt",
              "g_acc", "g_rho", "g_pos", "g_vel", "g_m")

# element type and elements per particle of every batch io array
_IO_LAYOUT = {"pos": ("float64", 3), "m": ("float32", 1), "vel": ("float32", 3), "u": ("float32", 1),
              "h": ("float64", 1), "active": ("uint8", 1), "rho": ("float32", 1), "drhodh": ("float32", 1),
              "fgrad": ("float32", 1), "nngb": ("int32", 1), "acc": ("float32", 3), "dudt": ("float32", 1),
              "g_acc": ("float32", 3), "g_rho": ("float32", 1), "g_pos": ("float32", 3), "g_vel": ("float32", 3),
              "g_m": ("float32", 1)}

_ERRORS = {
    -1: "SPHGRP_EINVAL",
    -2: "SPHGRP_ENOMEM",
    -3: "SPHGRP_ENOCONV",
    -4: "SPHGRP_ETIMEOUT",
    -5: "SPHGRP_EOVERFLOW",
    -6: "SPHGRP_ECUDA",
    -7: "SPHGRP_ESTATE",
}


class SphgrpError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{_ERRORS.get(code, code)}: {msg}")
        self.code = code


class Params(ctypes.Structure):
    _fields_ = [
        ("nngb", ctypes.c_double),
        ("nngb_tol", ctypes.c_double),
        ("max_iter", ctypes.c_int),
        ("leaf_size", ctypes.c_int),
        ("gamma", ctypes.c_double),
        ("alpha", ctypes.c_double),
        ("beta", ctypes.c_double),
        ("eps", ctypes.c_double),
        ("group_centre", ctypes.c_int),
        ("group_split", ctypes.c_double),
        ("iteration", ctypes.c_int),
        ("group_mode", ctypes.c_int),
        ("group_f", ctypes.c_double),
        ("group_level", ctypes.c_int),
        ("stack_shared", ctypes.c_int),
        ("iter_widen", ctypes.c_double),
    ]


class BatchIO(ctypes.Structure):
    _fields_ = [(f, ctypes.c_void_p) for f in _IO_FIELDS]


class Stats(ctypes.Structure):
    _fields_ = [(n, ctypes.c_int64) for n in (
        "walks", "nodes_tested", "candidates", "pair_tests", "pairs", "fp64_retests",
        "iterations", "max_stack", "members", "search_launches")] + [("search_ms", ctypes.c_double)]

    def as_dict(self) -> dict:
        return {n: getattr(self, n) for n, _ in self._fields_}


_lib = None


def sfc_keys_sort_static(pos, keys_out, perm_out):
    """sphgrp_sfc_keys_sort_static: keys and stable order without any device allocation
    (scratch in the library's fixed device array; n <= 2^19).  pos: n x 3 float64,
    keys_out: n int64 (the unsigned keys' bits), perm_out: n int32, all on the current
    device.  Synchronises the current stream."""
    n = pos.shape[0]
    L = load_library()
    _check(L.sphgrp_sfc_keys_sort_static(n, _arg(pos, "pos", _F64, 3 * n), _arg(keys_out, "keys_out", _I64, n),
                                         _arg(perm_out, "perm_out", _I32, n), _stream()))


def library_path() -> str:
    return _LIB_PATH


def load_library():
    """Loads libsphgrp.so; raises if it has not been built (no fallback exists)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(_LIB_PATH):
        raise ImportError(f"CUDA library not built: {_LIB_PATH} (run __graft_entry__.build())")
    L = ctypes.CDLL(_LIB_PATH)
    P, I64, I32 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int
    L.sphgrp_default_params.argtypes = [ctypes.POINTER(Params)]
    L.sphgrp_default_params.restype = None
    L.sphgrp_last_error.restype = ctypes.c_char_p
    L.sphgrp_ctx_create.argtypes = [ctypes.POINTER(P), ctypes.POINTER(Params), I64]
    L.sphgrp_ctx_destroy.argtypes = [P]
    L.sphgrp_sfc_keys_sort.argtypes = [P, I64, P, P, P, P]
    L.sphgrp_tree_build.argtypes = [P, I64, P, P, P]
    L.sphgrp_ngb_search.argtypes = [P, I64, P, P, I32, I32, I32, I64, P, P,
                                    ctypes.POINTER(I64), P]
    L.sphgrp_group_supersets.argtypes = [P, I64, P, P, I32, I32, I64, P, P, P, P,
                                         ctypes.POINTER(I64), ctypes.POINTER(I64), P]
    L.sphgrp_density.argtypes = [P, I64, P, P, I32, I32, I32, P, P, P, P, P, P]
    L.sphgrp_hydro_force.argtypes = [P, I64, P, P, P, P, P, P, I32, I32, P, P, P, P]
    L.sphgrp_hydro_force_balsara.argtypes = [P, I64, P, P, P, P, P, P, P, P, I32, I32, P, P, P, P]
    L.sphgrp_density_derivs.argtypes = [P, I64, P, P, I32, I32, P, P, P, P, P, P, P, P, P]
    L.sphgrp_key_split.argtypes = [P, I32, P, P, P]
    L.sphgrp_domain_boxes.argtypes = [P, P, I32, I32, P, ctypes.POINTER(I32), P]
    L.sphgrp_halo_select.argtypes = [P, P, I32, ctypes.c_double, I32, P, P, I32, I32, P, P, P]
    L.sphgrp_mask_compact.argtypes = [P, I64, P, I32, P, ctypes.POINTER(I64), P]
    L.sphgrp_velocity_derivs.argtypes = [P, I64, P, P, P, P, I32, P, P, P]
    L.sphgrp_backward.argtypes = [P, P, P, P, P, P, I32, P, P, P, P]
    L.sphgrp_get_stats.argtypes = [P, ctypes.POINTER(Stats)]
    L.sphgrp_kernel_launches.argtypes = [ctypes.POINTER(I64)]
    L.sphgrp_get_launch_log.argtypes = [P, I32, P, P, P, P, P, ctypes.POINTER(I32)]
    L.sphgrp_sfc_keys_sort_static.argtypes = [I64, P, P, P, P]
    L.sphgrp_batch_create.argtypes = [ctypes.POINTER(P), ctypes.POINTER(Params), I32, P, P]
    L.sphgrp_batch_destroy.argtypes = [P]
    L.sphgrp_batch_run.argtypes = [P, ctypes.POINTER(BatchIO), I32, P]
    L.sphgrp_batch_tune.argtypes = [P, ctypes.POINTER(BatchIO), P]
    L.sphgrp_batch_get_config.argtypes = [P, I32, ctypes.POINTER(I32), ctypes.POINTER(I32),
                                          ctypes.POINTER(ctypes.c_double), ctypes.POINTER(I32),
                                          ctypes.POINTER(ctypes.c_double), ctypes.POINTER(I64)]
    L.sphgrp_batch_set_config.argtypes = [P, I32, I32, I32, ctypes.c_double, I32]
    L.sphgrp_batch_stats.argtypes = [P, ctypes.POINTER(Stats)]
    for name in EXPORTED:
        if name not in ("sphgrp_default_params", "sphgrp_last_error"):
            getattr(L, name).restype = I32
    _lib = L
    return L


def _ptr(t):
    if t is None:
        return None
    return ctypes.c_void_p(t.data_ptr())


_F32, _F64, _I32, _I64, _U8 = "float32", "float64", "int32", "int64", "uint8"


def _arg(t, name: str, dtype: str, numel: int, optional: bool = False, cuda: bool = True):
    """Device pointer of tensor t after checking what the C ABI assumes of it: a dense
    array of the given element type holding at least numel elements, on the current
    CUDA device.  A wrong type or a short array would otherwise be read or written out
    of bounds by the kernels."""
    if t is None:
        if optional:
            return None
        raise ValueError(f"{name} is required")
    import torch

    if str(t.dtype) != f"torch.{dtype}":
        raise TypeError(f"{name} must be {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if t.numel() < numel:
        raise ValueError(f"{name} holds {t.numel()} elements, needs {numel}")
    if cuda and (not t.is_cuda or t.device.index != torch.cuda.current_device()):
        raise ValueError(f"{name} must be on the current CUDA device, got {t.device}")
    return ctypes.c_void_p(t.data_ptr())


def _stream():
    import torch

    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def _check(rc: int):
    if rc != 0:
        raise SphgrpError(rc, load_library().sphgrp_last_error().decode())


def kernel_launches() -> int:
    """Kernels launched by the library so far in this process."""
    n = ctypes.c_int64()
    _check(load_library().sphgrp_kernel_launches(ctypes.byref(n)))
    return int(n.value)


def default_params(**over) -> Params:
    p = Params()
    load_library().sphgrp_default_params(ctypes.byref(p))
    for k, v in over.items():
        setattr(p, k, v)
    return p


class Context:
    """One sphgrp_ctx: device workspace for up to n_max particles."""

    def __init__(self, n_max: int, **params):
        import torch

        if not torch.cuda.is_available():
            raise RuntimeError("sphgrp needs a CUDA device")
        self._L = load_library()
        self.params = default_params(**params)
        self._h = ctypes.c_void_p()
        _check(self._L.sphgrp_ctx_create(ctypes.byref(self._h), ctypes.byref(self.params), int(n_max)))
        self.n_max = int(n_max)
        self.n = 0   # particles of the last sfc_keys_sort

    def close(self):
        if self._h:
            self._L.sphgrp_ctx_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- a1 + a2
    def sfc_keys_sort(self, pos, keys_out=None, perm_out=None):
        n = pos.shape[0]
        _check(self._L.sphgrp_sfc_keys_sort(self._h, n, _arg(pos, "pos", _F64, 3 * n),
                                            _arg(keys_out, "keys_out", _I64, n, True),
                                            _arg(perm_out, "perm_out", _I32, n, True), _stream()))
        self.n = n

    # -- a3
    def tree_build(self, pos, m):
        n = pos.shape[0]
        _check(self._L.sphgrp_tree_build(self._h, n, _arg(pos, "pos", _F64, 3 * n), _arg(m, "m", _F32, n),
                                         _stream()))

    # -- a4 + a5 export
    def ngb_search(self, active, h, kind, mode, group_size, offsets, idx=None, cap=0) -> int:
        n_pairs = ctypes.c_int64()
        na = active.shape[0]
        _check(self._L.sphgrp_ngb_search(self._h, na, _arg(active, "active", _I32, na), _arg(h, "h", _F64, self.n),
                                         kind, mode, group_size, int(cap), _arg(offsets, "offsets", _I64, na + 1),
                                         _arg(idx, "idx", _I32, int(cap), True), ctypes.byref(n_pairs),
                                         _stream()))
        return int(n_pairs.value)

    def group_supersets(self, active, h, kind, group_size, group_offsets, group_first=None, members=None,
                        cand=None, cap=0):
        """Returns (n_groups, n_candidates)."""
        ng = ctypes.c_int64()
        n = ctypes.c_int64()
        na = active.shape[0]
        _check(self._L.sphgrp_group_supersets(self._h, na, _arg(active, "active", _I32, na),
                                              _arg(h, "h", _F64, self.n), kind, group_size, int(cap),
                                              _arg(group_offsets, "group_offsets", _I64, na + 1),
                                              _arg(group_first, "group_first", _I32, na + 1, True),
                                              _arg(members, "members", _I32, na, True),
                                              _arg(cand, "cand", _I32, int(cap), True), ctypes.byref(ng),
                                              ctypes.byref(n), _stream()))
        return int(ng.value), int(n.value)

    # -- a6 + a7
    def density(self, active, h, iterate, mode, group_size, rho, drhodh, fgrad, nngb, iters=None):
        na, n = active.shape[0], self.n
        _check(self._L.sphgrp_density(self._h, na, _arg(active, "active", _I32, na), _arg(h, "h", _F64, n),
                                      int(iterate), mode, group_size, _arg(rho, "rho", _F32, n),
                                      _arg(drhodh, "drhodh", _F32, n), _arg(fgrad, "fgrad", _F32, n),
                                      _arg(nngb, "nngb", _I32, n), _arg(iters, "iters", _I32, n, True), _stream()))

    def density_derivs(self, active, h, iterate, group_size, vel, rho, drhodh, fgrad, nngb, divv, curlv,
                       iters=None):
        """The density (as density, grouped form) with div v (n,) and curl v (n, 3) summed in
        the same loop, at every active particle's final h."""
        na, n = active.shape[0], self.n
        _check(self._L.sphgrp_density_derivs(self._h, na, _arg(active, "active", _I32, na), _arg(h, "h", _F64, n),
                                             int(iterate), group_size, _arg(vel, "vel", _F32, 3 * n),
                                             _arg(rho, "rho", _F32, n), _arg(drhodh, "drhodh", _F32, n),
                                             _arg(fgrad, "fgrad", _F32, n), _arg(nngb, "nngb", _I32, n),
                                             _arg(iters, "iters", _I32, n, True), _arg(divv, "divv", _F32, n),
                                             _arg(curlv, "curlv", _F32, 3 * n), _stream()))

    # -- f3: domain decomposition (paper_1810_09898_gb300.domain drives these)
    def key_split(self, splitters, dest):
        """dest (n int64, caller order) = 1 << owner rank of every particle's key, from the
        ascending splitters (int64 bit patterns of the 63-bit keys); after sfc_keys_sort."""
        ns = splitters.shape[0]
        _check(self._L.sphgrp_key_split(self._h, ns, _arg(splitters, "splitters", _I64, ns, ns == 0),
                                        _arg(dest, "dest", _I64, self.n), _stream()))

    def domain_boxes(self, h, level, boxes):
        """Tight boxes {lo, hi, hmax, count} of the particles per octree cell of `level`
        into boxes (cap x 8 float64); returns their number.  After tree_build."""
        nb = ctypes.c_int()
        _check(self._L.sphgrp_domain_boxes(self._h, _arg(h, "h", _F64, self.n), int(level), boxes.shape[0],
                                           _arg(boxes, "boxes", _F64, 8 * boxes.shape[0]), ctypes.byref(nb),
                                           _stream()))
        return nb.value

    def halo_select(self, h, kind, widen, boxes, box_rank, self_rank, world, mask, counts):
        """mask (n int64): bit r set for the particles rank r must import; counts per rank."""
        nb = box_rank.shape[0]
        _check(self._L.sphgrp_halo_select(self._h, _arg(h, "h", _F64, self.n), int(kind), float(widen), nb,
                                          _arg(boxes, "boxes", _F64, 8 * nb, nb == 0),
                                          _arg(box_rank, "box_rank", _I32, nb, nb == 0), int(self_rank),
                                          int(world), _arg(mask, "mask", _I64, self.n),
                                          _arg(counts, "counts", _I64, world), _stream()))

    def mask_compact(self, mask, bit, idx):
        """The particles with bit `bit` of mask, ascending, into idx (n int32); returns how many."""
        k = ctypes.c_int64()
        n = mask.shape[0]
        if n == 0:
            return 0
        _check(self._L.sphgrp_mask_compact(self._h, n, _arg(mask, "mask", _I64, n), int(bit),
                                           _arg(idx, "idx", _I32, n), ctypes.byref(k), _stream()))
        return k.value

    # -- a8
    def hydro_force(self, active, h, rho, fgrad, vel, u, mode, group_size, acc, dudt, nngb=None, divv=None,
                    curlv=None):
        """Accelerations and du/dt; with divv and curlv (all particles) the viscosity is
        limited by Balsara's switch (sphgrp_hydro_force_balsara)."""
        na, n = active.shape[0], self.n
        common = (_arg(active, "active", _I32, na), _arg(h, "h", _F64, n), _arg(rho, "rho", _F32, n),
                  _arg(fgrad, "fgrad", _F32, n), _arg(vel, "vel", _F32, 3 * n), _arg(u, "u", _F32, n))
        out = (_arg(acc, "acc", _F32, 3 * n), _arg(dudt, "dudt", _F32, n), _arg(nngb, "nngb", _I32, n, True),
               _stream())
        if divv is None and curlv is None:
            _check(self._L.sphgrp_hydro_force(self._h, na, *common, mode, group_size, *out))
        else:
            _check(self._L.sphgrp_hydro_force_balsara(self._h, na, *common, _arg(divv, "divv", _F32, n),
                                                      _arg(curlv, "curlv", _F32, 3 * n), mode, group_size, *out))

    def velocity_derivs(self, active, h, rho, vel, group_size, divv, curlv):
        """Velocity divergence (n,) and curl (n, 3) over the density sets (grouped walk)."""
        na, n = active.shape[0], self.n
        _check(self._L.sphgrp_velocity_derivs(self._h, na, _arg(active, "active", _I32, na),
                                              _arg(h, "h", _F64, n), _arg(rho, "rho", _F32, n),
                                              _arg(vel, "vel", _F32, 3 * n), int(group_size),
                                              _arg(divv, "divv", _F32, n), _arg(curlv, "curlv", _F32, 3 * n),
                                              _stream()))

    # -- a9
    def backward(self, h, vel, u, g_acc, g_rho, group_size, g_pos=None, g_vel=None, g_m=None):
        n = self.n
        no_acc = g_acc is None
        _check(self._L.sphgrp_backward(self._h, _arg(h, "h", _F64, n), _arg(vel, "vel", _F32, 3 * n, no_acc),
                                       _arg(u, "u", _F32, n, no_acc), _arg(g_acc, "g_acc", _F32, 3 * n, True),
                                       _arg(g_rho, "g_rho", _F32, n, True), int(group_size),
                                       _arg(g_pos, "g_pos", _F32, 3 * n, True),
                                       _arg(g_vel, "g_vel", _F32, 3 * n, True), _arg(g_m, "g_m", _F32, n, True),
                                       _stream()))

    def launch_log(self) -> list:
        import numpy as np

        cap = 128
        arrs = [np.zeros(cap, np.int64) for _ in range(4)]
        ms = np.zeros(cap, np.float64)
        cnt = ctypes.c_int()
        _check(self._L.sphgrp_get_launch_log(self._h, cap, *[a.ctypes.data_as(ctypes.c_void_p) for a in arrs],
                                             ms.ctypes.data_as(ctypes.c_void_p), ctypes.byref(cnt)))
        k = cnt.value
        return [{"members": int(arrs[0][i]), "candidates": int(arrs[1][i]), "pair_tests": int(arrs[2][i]),
                 "nodes": int(arrs[3][i]), "ms": float(ms[i])} for i in range(k)]

    def stats(self) -> dict:
        s = Stats()
        _check(self._L.sphgrp_get_stats(self._h, ctypes.byref(s)))
        return s.as_dict()


class Batch:
    """One sphgrp_batch: many independent periodic boxes solved together (a10).

    box_off: nbox + 1 offsets of the boxes' rows in the concatenated particle arrays;
    box_class: nbox class indices (autotuned configuration per class)."""

    def __init__(self, box_off, box_class=None, **params):
        import numpy as np
        import torch

        if not torch.cuda.is_available():
            raise RuntimeError("sphgrp needs a CUDA device")
        self._L = load_library()
        self.params = default_params(**params)
        self.box_off = np.ascontiguousarray(box_off, dtype=np.int64)
        self.nbox = len(self.box_off) - 1
        cls = None if box_class is None else np.ascontiguousarray(box_class, dtype=np.int32)
        self._cls = cls
        self._h = ctypes.c_void_p()
        _check(self._L.sphgrp_batch_create(ctypes.byref(self._h), ctypes.byref(self.params), self.nbox,
                                           self.box_off.ctypes.data_as(ctypes.c_void_p),
                                           None if cls is None else cls.ctypes.data_as(ctypes.c_void_p)))
        self.n = int(self.box_off[-1])

    def close(self):
        if self._h:
            self._L.sphgrp_batch_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @staticmethod
    def _io(arrays: dict, n: int, cuda: bool = True) -> BatchIO:
        """The io struct of n particles' arrays, each checked for type and length."""
        unknown = set(arrays) - set(_IO_FIELDS)
        if unknown:
            raise KeyError(f"unknown io arrays: {sorted(unknown)}")
        io = BatchIO()
        for f in _IO_FIELDS:
            t = arrays.get(f)
            dtype, per = _IO_LAYOUT[f]
            p = _arg(t, f, dtype, per * n, optional=True, cuda=cuda)
            setattr(io, f, None if p is None else p.value)
        return io

    def run(self, arrays: dict, backward: bool = False, graph: bool = False):
        flags = (BATCH_BACKWARD if backward else 0) | (BATCH_GRAPH if graph else 0)
        io = self._io(arrays, self.n)
        _check(self._L.sphgrp_batch_run(self._h, ctypes.byref(io), flags, _stream()))

    def tune(self, arrays: dict):
        io = self._io(arrays, self.n)
        _check(self._L.sphgrp_batch_tune(self._h, ctypes.byref(io), _stream()))

    def get_config(self, cls: int) -> dict:
        g, sm, lf = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        sp, ms = ctypes.c_double(), ctypes.c_double()
        nm = ctypes.c_int64()
        _check(self._L.sphgrp_batch_get_config(self._h, cls, ctypes.byref(g), ctypes.byref(sm), ctypes.byref(sp),
                                               ctypes.byref(lf), ctypes.byref(ms), ctypes.byref(nm)))
        return {"group_size": g.value, "max_slices": sm.value, "group_split": sp.value, "leaf_size": lf.value,
                "tuned_pass_ms": ms.value, "tuned_members": nm.value}

    def set_config(self, cls: int, group_size: int, max_slices: int, group_split: float, leaf_size: int = 0):
        _check(self._L.sphgrp_batch_set_config(self._h, cls, group_size, max_slices, float(group_split),
                                               int(leaf_size)))

    def stats(self) -> dict:
        st = Stats()
        _check(self._L.sphgrp_batch_stats(self._h, ctypes.byref(st)))
        return st.as_dict()
