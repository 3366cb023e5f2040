"""Thin ctypes binding of libmase (argument marshalling only).

Every compute step runs in the CUDA library; this module converts NumPy
arrays or CUDA tensors to pointers and back.  Loading fails loudly when the
library has not been built: there is no fallback path.
"""
from __future__ import annotations

import ctypes as C
import os
from dataclasses import dataclass

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libmase.so")

MASE_OK, MASE_NOT_CONVERGED = 0, 1
MASE_EINVAL, MASE_EUNOBSERVABLE, MASE_ENONFINITE, MASE_EDEVICE, MASE_ENOTREADY = -1, -2, -3, -4, -5
SNAP_CONVERGED, SNAP_MAX_ITER, SNAP_NOT_SPD, SNAP_NONFINITE, SNAP_DEVICE = 0, 1, 2, 3, 4
FP64, MIXED = 0, 1
START_FLAT, START_X0, START_LEARNED = 0, 1, 2
PER_AREA, BATCHED = 0, 1

_i32p = C.POINTER(C.c_int32)
_f64p = C.POINTER(C.c_double)
_u8p = C.POINTER(C.c_uint8)


class Network(C.Structure):
    _fields_ = [("n_bus", C.c_int32), ("n_branch", C.c_int32), ("slack_bus", C.c_int32),
                ("from_bus", _i32p), ("to_bus", _i32p), ("r", _f64p), ("x", _f64p),
                ("b_charge", _f64p)]


class Partition(C.Structure):
    _fields_ = [("n_area", C.c_int32), ("area_of_bus", _i32p)]


class Measurements(C.Structure):
    _fields_ = [("n_snap", C.c_int32), ("z", C.c_void_p), ("sigma", _f64p), ("mask", C.c_void_p)]


class Options(C.Structure):
    _fields_ = [("precision", C.c_int32), ("schedule", C.c_int32), ("use_graph", C.c_int32),
                ("refine", C.c_int32), ("threads", C.c_int32), ("device", C.c_int32),
                ("stream", C.c_void_p), ("profile", C.c_int32), ("wait_polls", C.c_int32),
                ("inner_iters", C.c_int32), ("autotune", C.c_int32), ("tensor_units", C.c_int32)]


class Stats(C.Structure):
    _fields_ = [("iters", _i32p), ("status", _i32p), ("J", _f64p), ("max_step", _f64p),
                ("stage_ms", C.c_double * 7), ("solve_ms", C.c_double), ("total_launches", C.c_int32),
                ("steps", C.c_int32), ("restarted", C.c_int32)]


class WarmstartOptions(C.Structure):
    _fields_ = [("hidden", C.c_int32), ("epochs", C.c_int32), ("batch", C.c_int32),
                ("lr", C.c_float), ("weight_decay", C.c_float), ("seed", C.c_uint64)]


class Info(C.Structure):
    _fields_ = [("n_bus", C.c_int32), ("n_branch", C.c_int32), ("n_area", C.c_int32),
                ("n_snap", C.c_int32), ("n_meas", C.c_int32), ("n_state", C.c_int32),
                ("n_boundary_bus", C.c_int32), ("n_gamma", C.c_int32),
                ("max_area_vars", C.c_int32), ("max_area_nb", C.c_int32),
                ("factor_nnz", C.c_int64), ("local_flops", C.c_int64),
                ("boundary_flops", C.c_int64), ("g_updates", C.c_int64),
                ("smem_bytes_max", C.c_int32), ("areas_in_smem", C.c_int32),
                ("n_supernodes", C.c_int64), ("n_units", C.c_int64), ("max_levels", C.c_int32),
                ("max_area_store", C.c_int32), ("boundary_store", C.c_int32),
                ("boundary_levels", C.c_int32), ("coord_S_elems", C.c_int64),
                ("coord_b_elems", C.c_int64), ("tuned", C.c_int32), ("local_classes", C.c_int32),
                ("class_areas", C.c_int32 * 4), ("class_threads", C.c_int32 * 4),
                ("class_smem", C.c_int32 * 4), ("back_threads", C.c_int32),
                ("coord_cluster", C.c_int32), ("tune_local_ms", C.c_float * 2)]

    def as_dict(self):
        out = {}
        for k, _ in self._fields_:
            v = getattr(self, k)
            out[k] = list(v) if hasattr(v, "_length_") else v
        return out


_lib = None


class MaseError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{code} ({status_str(code)}): {msg}")
        self.code = code


def load() -> C.CDLL:
    """Load libmase.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"libmase.so not built ({LIB_PATH}); run __graft_entry__.build()")
    lib = C.CDLL(LIB_PATH)
    H = C.c_void_p
    sig = {
        "mase_default_options": (None, [C.POINTER(Options)]),
        "mase_create": (C.c_int, [C.POINTER(Network), C.POINTER(Partition), C.POINTER(Measurements),
                                  C.POINTER(Options), C.POINTER(H)]),
        "mase_set_measurements": (C.c_int, [H, C.POINTER(Measurements)]),
        "mase_solve": (C.c_int, [H, C.c_void_p, C.c_double, C.c_int32, C.c_void_p, C.POINTER(Stats)]),
        "mase_measure": (C.c_int, [H, C.c_void_p, C.c_int32, C.c_void_p]),
        "mase_get_info": (C.c_int, [H, C.POINTER(Info)]),
        "mase_set_start_mode": (C.c_int, [H, C.c_int32]),
        "mase_destroy": (None, [H]),
        "mase_status_str": (C.c_char_p, [C.c_int]),
        "mase_last_error": (C.c_char_p, []),
        "mase_analyze": (C.c_int, [C.POINTER(Network), C.POINTER(Partition), C.POINTER(Info)]),
        "mase_selfcheck": (C.c_int, [C.POINTER(Network), C.POINTER(Partition), C.c_uint64, _f64p]),
        "mase_analyze_error": (C.c_char_p, []),
        "mase_abi_sizes": (None, [C.POINTER(C.c_int64)]),
        "mase_coordinator_noalloc": (C.c_int, [H, C.c_void_p, C.c_int64, C.c_void_p, C.c_int64,
                                               C.c_void_p, C.c_int64]),
        "mase_warmstart_default_options": (None, [C.POINTER(WarmstartOptions)]),
        "mase_warmstart_train": (C.c_int, [H, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int32,
                                           C.POINTER(WarmstartOptions), C.POINTER(C.c_double)]),
        "mase_warmstart_predict": (C.c_int, [H, C.c_void_p]),
        "mase_warmstart_save": (C.c_int, [H, C.c_char_p]),
        "mase_warmstart_load": (C.c_int, [H, C.c_char_p]),
        "mase_adamw_check": (C.c_int, [C.c_int64, C.c_int32, C.POINTER(C.c_float), C.c_float,
                                       C.POINTER(C.c_float), C.POINTER(C.c_float),
                                       C.POINTER(C.c_float), C.POINTER(C.c_float),
                                       C.POINTER(C.c_uint16)]),
        "mase_mlp_check": (C.c_int, [_i32p, C.c_int32, C.c_int32, C.POINTER(C.c_float),
                                     C.POINTER(C.c_float), C.POINTER(C.c_float),
                                     C.POINTER(C.c_float), C.POINTER(C.c_float)]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib


def abi_sizes() -> dict:
    """sizeof of the C structs in the library against this binding's copies."""
    out = (C.c_int64 * 4)()
    load().mase_abi_sizes(out)
    return {"options": (out[0], C.sizeof(Options)), "stats": (out[1], C.sizeof(Stats)),
            "info": (out[2], C.sizeof(Info)), "warmstart_options": (out[3], C.sizeof(WarmstartOptions))}


def status_str(code: int) -> str:
    return load().mase_status_str(code).decode()


def _last_error() -> str:
    return load().mase_last_error().decode()


def _ptr(a, ctype=None):
    """Pointer of a NumPy array or a torch CUDA/CPU tensor (contiguous)."""
    if a is None:
        return None
    if hasattr(a, "data_ptr"):
        if not a.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return C.c_void_p(a.data_ptr())
    if not a.flags["C_CONTIGUOUS"]:
        raise ValueError("array must be C-contiguous")
    return a.ctypes.data_as(C.c_void_p)


@dataclass
class _Keep:
    """Host arrays referenced by ctypes structs (kept alive by the caller)."""
    arrays: list


def _network(grid):
    fr = np.ascontiguousarray(grid.from_bus, dtype=np.int32)
    to = np.ascontiguousarray(grid.to_bus, dtype=np.int32)
    r = np.ascontiguousarray(grid.r, dtype=np.float64)
    x = np.ascontiguousarray(grid.x, dtype=np.float64)
    b = np.ascontiguousarray(grid.b_charge, dtype=np.float64)
    ar = np.ascontiguousarray(grid.area_of_bus, dtype=np.int32)
    net = Network(int(grid.n_bus), int(len(fr)), int(grid.slack),
                  fr.ctypes.data_as(_i32p), to.ctypes.data_as(_i32p), r.ctypes.data_as(_f64p),
                  x.ctypes.data_as(_f64p), b.ctypes.data_as(_f64p))
    part = Partition(int(grid.n_area), ar.ctypes.data_as(_i32p))
    return net, part, _Keep([fr, to, r, x, b, ar])


def analyze(grid) -> dict:
    """Host-only structural analysis of the setup (no GPU needed)."""
    lib = load()
    net, part, keep = _network(grid)
    info = Info()
    rc = lib.mase_analyze(C.byref(net), C.byref(part), C.byref(info))
    if rc != MASE_OK:
        raise MaseError(rc, lib.mase_analyze_error().decode())
    del keep
    return info.as_dict()


def selfcheck(grid, seed: int = 1) -> np.ndarray:
    """Host-only check of the symbolic setup against dense Cholesky (no GPU)."""
    lib = load()
    net, part, keep = _network(grid)
    out = np.zeros(4)
    rc = lib.mase_selfcheck(C.byref(net), C.byref(part), seed, out.ctypes.data_as(_f64p))
    if rc != MASE_OK:
        raise MaseError(rc, lib.mase_analyze_error().decode())
    del keep
    return out


def default_options() -> Options:
    o = Options()
    load().mase_default_options(C.byref(o))
    return o


def _numel(a) -> int:
    return int(a.numel()) if hasattr(a, "numel") else int(a.size)


def noalloc_sizes(info: dict, n_snap: int) -> tuple:
    """Element counts (S_blocks, b_blocks, dx_gamma) the no-alloc coordinator
    step expects for a handle with this structure and batch size."""
    return (n_snap * int(info["coord_S_elems"]), n_snap * int(info["coord_b_elems"]),
            n_snap * int(info["n_gamma"]))


def check_noalloc_args(need: tuple, S_blocks, b_blocks, dx_gamma) -> None:
    """Rejects (ValueError) tensors whose dtype is not float64 or whose size
    differs from ``need`` before anything is launched."""
    for name, t, n in (("S_blocks", S_blocks, need[0]), ("b_blocks", b_blocks, need[1]),
                       ("dx_gamma", dx_gamma, need[2])):
        dt = str(getattr(t, "dtype", ""))
        if dt not in ("torch.float64", "float64"):
            raise ValueError(f"{name} must be float64, got {dt or type(t).__name__}")
        if _numel(t) != n:
            raise ValueError(f"{name} has {_numel(t)} elements, the handle needs {n}")


_DTYPES = {"float64": ("torch.float64", "float64"), "uint8": ("torch.uint8", "uint8")}


def check_array(name: str, a, n: int, dtype: str) -> None:
    """Rejects (ValueError) an array or tensor whose element type is not
    ``dtype`` ("float64" or "uint8") or whose element count is not ``n``,
    before anything is passed to the library, which reads and writes these
    buffers at the sizes the handle implies.  None passes."""
    if a is None:
        return
    dt = str(getattr(a, "dtype", ""))
    if dt not in _DTYPES[dtype]:
        raise ValueError(f"{name} must be {dtype}, got {dt or type(a).__name__}")
    if _numel(a) != n:
        raise ValueError(f"{name} has {_numel(a)} elements, {n} expected")


@dataclass
class SolveResult:
    rc: int
    iters: np.ndarray
    status: np.ndarray
    J: np.ndarray
    max_step: np.ndarray
    launches: int
    steps: int
    stage_ms: tuple     # area, coordinator, back, bookkeeping, learned start, start/finish, loop gaps
    solve_ms: float
    restarted: int = 0  # learned-start snapshots solved again from the flat start


class Estimator:
    """One handle: a network, its partition and a batch of n_snap snapshots."""

    def __init__(self, grid, sigma, n_snap: int, z=None, mask=None, precision=MIXED,
                 schedule=BATCHED, use_graph=True, refine=1, threads=0, device=0, stream=None,
                 profile=False, wait_polls=0, inner_iters=0, autotune=True, tensor_units=-1):
        self.lib = load()
        m = int(grid.n_meas)
        check_array("z", z, int(n_snap) * m, "float64")
        check_array("mask", mask, int(n_snap) * m, "uint8")
        net, part, keep = _network(grid)
        sig = np.ascontiguousarray(sigma, dtype=np.float64)
        if sig.size != m:
            raise ValueError(f"sigma has {sig.size} elements, {m} expected")
        opt = default_options()
        opt.precision, opt.schedule, opt.use_graph = precision, schedule, int(bool(use_graph))
        opt.refine, opt.threads, opt.device = refine, threads, device
        opt.stream = C.c_void_p(stream) if stream else None
        opt.profile = int(bool(profile))
        opt.wait_polls = int(wait_polls)
        opt.inner_iters = int(inner_iters)
        opt.autotune = int(bool(autotune))
        opt.tensor_units = int(tensor_units)
        meas = Measurements(int(n_snap), _ptr(z), sig.ctypes.data_as(_f64p), _ptr(mask))
        h = C.c_void_p()
        rc = self.lib.mase_create(C.byref(net), C.byref(part), C.byref(meas), C.byref(opt), C.byref(h))
        if rc != MASE_OK:
            raise MaseError(rc, _last_error())
        self.h = h
        self.n_snap = int(n_snap)
        self.n_bus = int(grid.n_bus)
        self.n_meas = int(grid.n_meas)
        del keep

    def close(self):
        if getattr(self, "h", None):
            self.lib.mase_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_measurements(self, z, mask=None):
        check_array("z", z, self.n_snap * self.n_meas, "float64")
        check_array("mask", mask, self.n_snap * self.n_meas, "uint8")
        meas = Measurements(self.n_snap, _ptr(z), None, _ptr(mask))
        rc = self.lib.mase_set_measurements(self.h, C.byref(meas))
        if rc != MASE_OK:
            raise MaseError(rc, _last_error())

    def set_start_mode(self, mode: int):
        rc = self.lib.mase_set_start_mode(self.h, mode)
        if rc != MASE_OK:
            raise MaseError(rc, _last_error())

    def solve(self, x0=None, tol=1e-8, max_iter=10, x_out=None, check=True) -> SolveResult:
        """Solve the batch.  x_out: host array or CUDA tensor [n_snap, 2N]."""
        S = self.n_snap
        check_array("x0", x0, S * 2 * self.n_bus, "float64")
        check_array("x_out", x_out, S * 2 * self.n_bus, "float64")
        iters = np.zeros(S, dtype=np.int32)
        status = np.zeros(S, dtype=np.int32)
        J = np.zeros(S)
        ms = np.zeros(S)
        st = Stats(iters.ctypes.data_as(_i32p), status.ctypes.data_as(_i32p),
                   J.ctypes.data_as(_f64p), ms.ctypes.data_as(_f64p))
        rc = self.lib.mase_solve(self.h, _ptr(x0), float(tol), int(max_iter), _ptr(x_out), C.byref(st))
        if check and rc < 0:
            raise MaseError(rc, _last_error())
        return SolveResult(rc, iters, status, J, ms, int(st.total_launches), int(st.steps),
                           tuple(st.stage_ms), float(st.solve_ms), int(st.restarted))

    def measure(self, x, z_out, n_snap=None):
        n = self.n_snap if n_snap is None else n_snap
        check_array("x", x, int(n) * 2 * self.n_bus, "float64")
        check_array("z_out", z_out, int(n) * self.n_meas, "float64")
        rc = self.lib.mase_measure(self.h, _ptr(x), int(n), _ptr(z_out))
        if rc != MASE_OK:
            raise MaseError(rc, _last_error())

    def coordinator_noalloc(self, S_blocks, b_blocks, dx_gamma):
        """Coordinator step on caller-held condensed blocks, without device
        allocation (FP64 device tensors in, FP64 device tensor out).  Sizes and
        dtypes are checked here first; the C entry point checks the counts
        again."""
        need = noalloc_sizes(self.info(), self.n_snap)
        check_noalloc_args(need, S_blocks, b_blocks, dx_gamma)
        rc = self.lib.mase_coordinator_noalloc(self.h, _ptr(S_blocks), _numel(S_blocks), _ptr(b_blocks),
                                               _numel(b_blocks), _ptr(dx_gamma), _numel(dx_gamma))
        if rc != MASE_OK:
            raise MaseError(rc, _last_error())

    # ---- learned warm start
    def warmstart_train(self, z, x, epochs=20, batch=256, lr=1e-3, weight_decay=1e-4, hidden=512,
                        seed=1, mask=None) -> float:
        """Train the per-area networks on (z, x) pairs, with an optional
        presence mask [n][m] (uint8, 1 = present) per sample; returns the
        last-epoch loss."""
        if mask is not None:
            if tuple(mask.shape) != tuple(z.shape) or "uint8" not in str(mask.dtype):
                raise ValueError("mask must be uint8 with the shape of z")
        check_array("z", z, int(z.shape[0]) * self.n_meas, "float64")
        check_array("x", x, int(z.shape[0]) * 2 * self.n_bus, "float64")
        o = WarmstartOptions()
        self.lib.mase_warmstart_default_options(C.byref(o))
        o.hidden, o.epochs, o.batch, o.lr, o.weight_decay, o.seed = hidden, epochs, batch, lr, weight_decay, seed
        loss = C.c_double()
        n = int(z.shape[0])
        rc = self.lib.mase_warmstart_train(self.h, _ptr(z), _ptr(mask), _ptr(x), n, C.byref(o),
                                           C.byref(loss))
        if rc != MASE_OK:
            raise MaseError(rc, _last_error())
        return loss.value

    def warmstart_predict(self, x_out):
        check_array("x_out", x_out, self.n_snap * 2 * self.n_bus, "float64")
        rc = self.lib.mase_warmstart_predict(self.h, _ptr(x_out))
        if rc != MASE_OK:
            raise MaseError(rc, _last_error())

    def warmstart_save(self, path: str):
        rc = self.lib.mase_warmstart_save(self.h, path.encode())
        if rc != MASE_OK:
            raise MaseError(rc, _last_error())

    def warmstart_load(self, path: str):
        rc = self.lib.mase_warmstart_load(self.h, path.encode())
        if rc != MASE_OK:
            raise MaseError(rc, _last_error())

    def info(self) -> dict:
        inf = Info()
        rc = self.lib.mase_get_info(self.h, C.byref(inf))
        if rc != MASE_OK:
            raise MaseError(rc, _last_error())
        return inf.as_dict()


def mlp_check(dims, params, X, T):
    """One forward/backward pass of a single warm-start network with the
    library's training kernels: returns (loss, grads) (FP32)."""
    lib = load()
    d = np.ascontiguousarray(dims, dtype=np.int32)
    p = np.ascontiguousarray(params, dtype=np.float32)
    Xa = np.ascontiguousarray(X, dtype=np.float32)
    Ta = np.ascontiguousarray(T, dtype=np.float32)
    g = np.zeros_like(p)
    loss = C.c_float()
    fp = C.POINTER(C.c_float)
    rc = lib.mase_mlp_check(d.ctypes.data_as(_i32p), len(d) - 1, int(Xa.shape[0]), p.ctypes.data_as(fp),
                            Xa.ctypes.data_as(fp), Ta.ctypes.data_as(fp), C.byref(loss), g.ctypes.data_as(fp))
    if rc != MASE_OK:
        raise MaseError(rc, _last_error())
    return loss.value, g


def adamw_check(w, grads, lr, weight_decay):
    """Runs the library's AdamW kernel len(lr) times on FP32 parameters w with
    the given gradients [steps, n]; returns (w, m, v, w_bf16_bits)."""
    lib = load()
    wa = np.array(w, dtype=np.float32, copy=True)
    ga = np.ascontiguousarray(grads, dtype=np.float32)
    la = np.ascontiguousarray(lr, dtype=np.float32)
    n, steps = wa.size, la.size
    if ga.shape != (steps, n):
        raise ValueError("grads must be [steps, n]")
    m = np.zeros(n, dtype=np.float32)
    v = np.zeros(n, dtype=np.float32)
    w16 = np.zeros(n, dtype=np.uint16)
    fp = C.POINTER(C.c_float)
    rc = lib.mase_adamw_check(n, steps, la.ctypes.data_as(fp), float(weight_decay), ga.ctypes.data_as(fp),
                              wa.ctypes.data_as(fp), m.ctypes.data_as(fp), v.ctypes.data_as(fp),
                              w16.ctypes.data_as(C.POINTER(C.c_uint16)))
    if rc != MASE_OK:
        raise MaseError(rc, _last_error())
    return wa, m, v, w16
