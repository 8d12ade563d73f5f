"""GB300-native CTR-IBIM for the linearized Poisson-Boltzmann equation.

Thin Python binding (argument marshalling only) over the C ABI of
libctr_ibim.so (include/ctr_ibim.h); every step of the method runs in the
library's CUDA kernels.  Importing this package loads the library and fails
loudly when it has not been built (python -m paper_2210_03699_gb300.build).

Arrays may be numpy (host) or torch CUDA tensors (device, float64,
contiguous); outputs follow the input kind unless stated otherwise.
"""
from __future__ import annotations

import ctypes
import dataclasses
import os

import numpy as np

from . import build as _build

__all__ = ["Options", "SolveInfo", "CtrIbim", "CtrError", "weight_tables", "kernel_launches", "batch_solve",
           "Server", "RequestResult", "set_wait_limit",
           "library_path", "lib",
           "FP64", "FP32_REFINE", "DF64", "METHOD_HYB", "METHOD_KREG"]

FP64 = 0
FP32_REFINE = 1
DF64 = 2
METHOD_HYB = 0
METHOD_KREG = 1
FARFIELD_DIRECT = 0
FARFIELD_TREECODE = 1
RESIDUAL_UPDATE = 0
RESIDUAL_FULL = 1
ERR_DEVICE_WAIT = -7
ERR_CANCELLED = -9

_D = ctypes.POINTER(ctypes.c_double)
_I64 = ctypes.POINTER(ctypes.c_int64)


class CtrError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{msg} (status {status})")
        self.status = status


class _Grid(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64 * 3), ("origin", ctypes.c_double * 3), ("h", ctypes.c_double)]


class _Options(ctypes.Structure):
    _fields_ = [("tube_halfwidth", ctypes.c_double), ("precision", ctypes.c_int), ("tol", ctypes.c_double),
                ("restart", ctypes.c_int), ("max_iter", ctypes.c_int), ("max_refine", ctypes.c_int),
                ("inner_tol", ctypes.c_double), ("tile_targets", ctypes.c_int), ("residual", ctypes.c_int),
                ("method", ctypes.c_int), ("farfield", ctypes.c_int), ("tree_degree", ctypes.c_int),
                ("tree_theta", ctypes.c_double), ("tree_leaf", ctypes.c_int), ("tree_degree_fp32", ctypes.c_int),
                ("tree_theta_fp32", ctypes.c_double), ("residual_mode", ctypes.c_int), ("fp32_block", ctypes.c_int),
                ("fp32_tile", ctypes.c_int)]


class _Info(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_int64), ("refinements", ctypes.c_int64),
                ("matvecs_fp32", ctypes.c_int64), ("matvecs_fp64", ctypes.c_int64),
                ("residual", ctypes.c_double), ("converged", ctypes.c_int)]


class _ServerOptions(ctypes.Structure):
    _fields_ = [("max_slots", ctypes.c_int), ("hbm_budget_bytes", ctypes.c_int64), ("step_quantum_ms", ctypes.c_double)]


class _RequestResult(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int), ("M", ctypes.c_int64), ("G_pol", ctypes.c_double), ("info", _Info),
                ("t_submit", ctypes.c_double), ("t_admit", ctypes.c_double), ("t_done", ctypes.c_double)]


class _ServerStats(ctypes.Structure):
    _fields_ = [("budget_bytes", ctypes.c_int64), ("used_bytes", ctypes.c_int64),
                ("peak_used_bytes", ctypes.c_int64), ("peak_slots", ctypes.c_int), ("running", ctypes.c_int),
                ("waiting", ctypes.c_int), ("steps", ctypes.c_int64)]


@dataclasses.dataclass
class Options:
    tube_halfwidth: float = 0.0
    precision: int = FP64
    tol: float = 1e-10
    restart: int = 64
    max_iter: int = 400
    max_refine: int = 10
    inner_tol: float = 1e-5
    tile_targets: int = 0
    residual: int = DF64
    method: int = METHOD_HYB
    farfield: int = FARFIELD_DIRECT
    tree_degree: int = 10
    tree_theta: float = 0.8
    tree_leaf: int = 128
    tree_degree_fp32: int = 6
    tree_theta_fp32: float = 0.9
    residual_mode: int = RESIDUAL_UPDATE
    fp32_block: int = 0
    fp32_tile: int = 0

    def _c(self) -> _Options:
        return _Options(self.tube_halfwidth, self.precision, self.tol, self.restart, self.max_iter,
                        self.max_refine, self.inner_tol, self.tile_targets, self.residual, self.method,
                        self.farfield, self.tree_degree, self.tree_theta, self.tree_leaf, self.tree_degree_fp32,
                        self.tree_theta_fp32, self.residual_mode, self.fp32_block, self.fp32_tile)


@dataclasses.dataclass
class SolveInfo:
    iterations: int
    refinements: int
    matvecs_fp32: int
    matvecs_fp64: int
    residual: float
    converged: bool
    status: int


def library_path() -> str:
    return _build.LIB


def _load():
    path = library_path()
    if not os.path.exists(path):
        raise ImportError(f"libctr_ibim.so is not built ({path}); run python -m paper_2210_03699_gb300.build")
    L = ctypes.CDLL(path)
    P = ctypes.c_void_p
    sig = {
        "ctr_default_options": (None, [ctypes.POINTER(_Options)]),
        "ctr_ibim_setup": (ctypes.c_int, [ctypes.POINTER(_Grid), P, ctypes.c_int, ctypes.c_double, ctypes.c_double,
                                          ctypes.c_double, ctypes.c_int64, P, P, ctypes.POINTER(_Options), P,
                                          ctypes.POINTER(P)]),
        "ctr_ibim_destroy": (None, [P]),
        "ctr_ibim_num_nodes": (ctypes.c_int, [P, _I64]),
        "ctr_ibim_nodes": (ctypes.c_int, [P, P]),
        "ctr_ibim_geometry": (ctypes.c_int, [P, P, P, P]),
        "ctr_ibim_num_corrections": (ctypes.c_int, [P, _I64]),
        "ctr_ibim_corrections": (ctypes.c_int, [P, P, P, P, P, P, P]),
        "ctr_ibim_bad_nodes": (ctypes.c_int, [P, P]),
        "ctr_ibim_rhs": (ctypes.c_int, [P, P, ctypes.c_int]),
        "ctr_ibim_area": (ctypes.c_int, [P, _D]),
        "ctr_ibim_matvec": (ctypes.c_int, [P, P, P, ctypes.c_int, ctypes.c_int]),
        "ctr_ibim_solve": (ctypes.c_int, [P, P, P, ctypes.c_int, ctypes.POINTER(_Info)]),
        "ctr_ibim_batch_solve": (ctypes.c_int, [ctypes.POINTER(P), ctypes.c_int64, ctypes.POINTER(P),
                                                ctypes.POINTER(P), ctypes.c_int, ctypes.POINTER(_Info)]),
        "ctr_ibim_energy": (ctypes.c_int, [P, P, P, ctypes.c_int, _D, P]),
        "ctr_ibim_reaction_potential": (ctypes.c_int, [P, P, P, ctypes.c_int, ctypes.c_int64, P, P]),
        "ctr_ibim_potential_map": (ctypes.c_int, [P, P, P, ctypes.c_int64, P, P, ctypes.c_int, ctypes.c_int]),
        "ctr_weight_tables": (ctypes.c_int, [P]),
        "ctr_default_server_options": (None, [ctypes.POINTER(_ServerOptions)]),
        "ctr_server_create": (ctypes.c_int, [ctypes.POINTER(_ServerOptions), ctypes.POINTER(P)]),
        "ctr_server_submit": (ctypes.c_int, [P, ctypes.POINTER(_Grid), P, ctypes.c_double, ctypes.c_double,
                                             ctypes.c_double, ctypes.c_int64, P, P, ctypes.POINTER(_Options),
                                             ctypes.POINTER(ctypes.c_uint64)]),
        "ctr_server_poll": (ctypes.c_int, [P, ctypes.c_uint64, ctypes.POINTER(ctypes.c_int),
                                           ctypes.POINTER(_RequestResult)]),
        "ctr_server_wait": (ctypes.c_int, [P, ctypes.c_uint64, ctypes.c_double, ctypes.POINTER(_RequestResult)]),
        "ctr_server_fetch": (ctypes.c_int, [P, ctypes.c_uint64, P, P, ctypes.c_int64]),
        "ctr_server_release": (ctypes.c_int, [P, ctypes.c_uint64]),
        "ctr_server_stats": (ctypes.c_int, [P, ctypes.POINTER(_ServerStats)]),
        "ctr_server_destroy": (None, [P]),
        "ctr_server_cancel": (ctypes.c_int, [P, ctypes.c_uint64]),
        "ctr_set_wait_limit": (ctypes.c_int, [ctypes.c_int64]),
        "ctr_status_string": (ctypes.c_char_p, [ctypes.c_int]),
        "ctr_last_error": (ctypes.c_char_p, []),
        "ctr_kernel_launches": (ctypes.c_int64, []),
        "ctr_ibim_pair_schedule": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int] + [ctypes.POINTER(ctypes.c_int64)] * 4),
        "ctr_tuning_info": (ctypes.c_int, [ctypes.POINTER(ctypes.c_int)] * 3),
        "ctr_ibim_pair_tuning": (ctypes.c_int, [P, ctypes.c_int] + [ctypes.POINTER(ctypes.c_int)] * 4),
        "ctr_ibim_farfield_info": (ctypes.c_int, [P, ctypes.c_int, P] + [_I64] * 4),
        "ctr_ibim_time_operator": (ctypes.c_int, [P, ctypes.c_int, ctypes.c_int] + [_D] * 4),
        "ctr_farfield_plan": (ctypes.c_int, [ctypes.c_int64, P, P, P, ctypes.c_int, ctypes.c_int, ctypes.c_double,
                                             ctypes.c_int, ctypes.c_int, ctypes.c_int64, P, _I64, _I64, P, P, P,
                                             P, P]),
    }
    for name, (res, args) in sig.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    return L


lib = _load()


def _check(status: int, allow=(0,)):
    if status in allow:
        return status
    msg = lib.ctr_last_error().decode() or lib.ctr_status_string(status).decode()
    raise CtrError(status, msg)


def _is_torch(x) -> bool:
    return type(x).__module__.startswith("torch")


def _dptr(x, n=None):
    """(pointer, on_device) for a float64 contiguous numpy array or torch CUDA tensor."""
    if _is_torch(x):
        import torch
        if x.dtype != torch.float64 or not x.is_contiguous() or not x.is_cuda:
            raise TypeError("device arrays must be contiguous float64 CUDA tensors")
        if n is not None and x.numel() != n:
            raise ValueError(f"expected {n} elements, got {x.numel()}")
        return ctypes.c_void_p(x.data_ptr()), 1
    a = np.ascontiguousarray(x, dtype=np.float64)
    if n is not None and a.size != n:
        raise ValueError(f"expected {n} elements, got {a.size}")
    return a, 0


def _current_stream():
    try:
        import torch
        if torch.cuda.is_available():
            return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    except Exception:  # noqa: BLE001 - torch is optional for the binding
        pass
    return ctypes.c_void_p(None)


class CtrIbim:
    """One discretized CTR-IBIM system (surface + charges) resident on the GPU."""

    def __init__(self, grid_n, origin, h, sdist, eps_in, eps_out, kappa, charge_xyz, charge_q,
                 options: Options | None = None, stream=None):
        g = _Grid((ctypes.c_int64 * 3)(*[int(v) for v in grid_n]), (ctypes.c_double * 3)(*[float(v) for v in origin]),
                  float(h))
        n_total = int(grid_n[0]) * int(grid_n[1]) * int(grid_n[2])
        sd, sd_dev = _dptr(sdist, n_total)
        xyz = np.ascontiguousarray(charge_xyz, dtype=np.float64).reshape(-1, 3)
        q = np.ascontiguousarray(charge_q, dtype=np.float64).ravel()
        if xyz.shape[0] != q.size:
            raise ValueError("charge_xyz and charge_q disagree")
        self.options = options or Options()
        opt = self.options._c()
        self._stream = stream if stream is not None else _current_stream()
        handle = ctypes.c_void_p()
        sd_p = sd.ctypes.data_as(ctypes.c_void_p) if not sd_dev else sd
        st = lib.ctr_ibim_setup(ctypes.byref(g), sd_p, sd_dev, float(eps_in), float(eps_out), float(kappa), q.size,
                                xyz.ctypes.data_as(ctypes.c_void_p), q.ctypes.data_as(ctypes.c_void_p),
                                ctypes.byref(opt), self._stream, ctypes.byref(handle))
        _check(st)
        self._h = handle
        self.n_charges = q.size
        Mv = ctypes.c_int64()
        _check(lib.ctr_ibim_num_nodes(self._h, ctypes.byref(Mv)))
        self.M = int(Mv.value)
        Ev = ctypes.c_int64()
        _check(lib.ctr_ibim_num_corrections(self._h, ctypes.byref(Ev)))
        self.E = int(Ev.value)

    @classmethod
    def from_problem(cls, prob, options: Options | None = None, stream=None, sdist=None):
        """System for a synthetic.Problem (its tube half-width unless options say otherwise)."""
        g = prob.grid
        return cls(g.n, g.origin, g.h, prob.sdist if sdist is None else sdist, prob.eps_in, prob.eps_out,
                   prob.kappa, prob.charge_xyz, prob.charge_q,
                   options=options or Options(tube_halfwidth=prob.tube), stream=stream)

    def close(self):
        if getattr(self, "_h", None):
            lib.ctr_ibim_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:  # noqa: BLE001
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    # ------------------------------------------------------------ inspection
    def nodes(self) -> np.ndarray:
        out = np.empty(self.M, dtype=np.int64)
        _check(lib.ctr_ibim_nodes(self._h, out.ctypes.data_as(ctypes.c_void_p)))
        return out

    def geometry(self):
        P = np.empty((self.M, 3))
        n = np.empty((self.M, 3))
        W = np.empty(self.M)
        _check(lib.ctr_ibim_geometry(self._h, P.ctypes.data_as(ctypes.c_void_p), n.ctypes.data_as(ctypes.c_void_p),
                                     W.ctypes.data_as(ctypes.c_void_p)))
        return P, n, W

    def corrections(self):
        """(ptr, node, w) with w rows omega11, omega21, omega22, omega12."""
        ptr = np.empty(self.M + 1, dtype=np.int64)
        node = np.empty(self.E, dtype=np.int64)
        w = np.empty((4, self.E))
        vp = lambda a: a.ctypes.data_as(ctypes.c_void_p)  # noqa: E731
        _check(lib.ctr_ibim_corrections(self._h, vp(ptr), vp(node), vp(w[0]), vp(w[3]), vp(w[1]), vp(w[2])))
        return ptr, node, w

    def bad_nodes(self) -> np.ndarray:
        f = np.empty(self.M, dtype=np.uint8)
        _check(lib.ctr_ibim_bad_nodes(self._h, f.ctypes.data_as(ctypes.c_void_p)))
        return f.astype(bool)

    def rhs(self) -> np.ndarray:
        g = np.empty(2 * self.M)
        _check(lib.ctr_ibim_rhs(self._h, g.ctypes.data_as(ctypes.c_void_p), 0))
        return g

    def pair_schedule(self, precision: int = FP32_REFINE) -> dict:
        """Pair counts of the dense-sum schedule of one arithmetic (see ctr_ibim_pair_schedule)."""
        v = [ctypes.c_int64() for _ in range(4)]
        _check(lib.ctr_ibim_pair_schedule(self._h, int(precision), *[ctypes.byref(x) for x in v]))
        return {"one_sided_pairs": v[0].value, "symmetric_pairs": v[1].value, "items": v[2].value,
                "partial_bytes": v[3].value}

    def pair_tuning(self, precision: int = FP32_REFINE) -> dict:
        """Pair-kernel shape of one arithmetic's schedule (see ctr_ibim_pair_tuning)."""
        v = [ctypes.c_int() for _ in range(4)]
        _check(lib.ctr_ibim_pair_tuning(self._h, int(precision), *[ctypes.byref(x) for x in v]))
        return {"block_targets": v[0].value, "tile": v[1].value, "chunk": v[2].value, "unroll": v[3].value}

    def farfield_info(self, precision: int = FP32_REFINE) -> dict:
        """The treecode of this handle for one arithmetic (see ctr_ibim_farfield_info)."""
        perm = np.empty(self.M, dtype=np.int64)
        v = [ctypes.c_int64() for _ in range(4)]
        _check(lib.ctr_ibim_farfield_info(self._h, int(precision), perm.ctypes.data_as(ctypes.c_void_p),
                                          *[ctypes.byref(x) for x in v]))
        return {"perm": perm, "near_pairs": v[0].value, "far_evaluations": v[1].value,
                "far_interactions": v[2].value, "far_clusters": v[3].value}

    def time_operator(self, precision: int = FP32_REFINE, reps: int = 3) -> dict:
        """Mean milliseconds of the operator's phases over `reps` applications (see ctr_ibim_time_operator)."""
        v = [ctypes.c_double() for _ in range(4)]
        _check(lib.ctr_ibim_time_operator(self._h, int(precision), int(reps), *[ctypes.byref(x) for x in v]))
        return {"pack_ms": v[0].value, "pairs_ms": v[1].value, "far_ms": v[2].value, "finish_ms": v[3].value}

    def area(self) -> float:
        a = ctypes.c_double()
        _check(lib.ctr_ibim_area(self._h, ctypes.byref(a)))
        return float(a.value)

    # ------------------------------------------------------------ operator / solve / energy
    def matvec(self, x, precision: int = FP64, out=None):
        n = 2 * self.M
        xp, dev = _dptr(x, n)
        if dev:
            import torch
            y = out if out is not None else torch.empty_like(x)
            yp, _ = _dptr(y, n)
            _check(lib.ctr_ibim_matvec(self._h, xp, yp, int(precision), 1))
            return y
        y = np.empty(n)
        _check(lib.ctr_ibim_matvec(self._h, xp.ctypes.data_as(ctypes.c_void_p), y.ctypes.data_as(ctypes.c_void_p),
                                   int(precision), 0))
        return y

    def solve(self, device: bool = False):
        info = _Info()
        if device:
            import torch
            psi = torch.empty(self.M, dtype=torch.float64, device="cuda")
            dpsi = torch.empty(self.M, dtype=torch.float64, device="cuda")
            st = lib.ctr_ibim_solve(self._h, ctypes.c_void_p(psi.data_ptr()), ctypes.c_void_p(dpsi.data_ptr()), 1,
                                    ctypes.byref(info))
        else:
            psi = np.empty(self.M)
            dpsi = np.empty(self.M)
            st = lib.ctr_ibim_solve(self._h, psi.ctypes.data_as(ctypes.c_void_p), dpsi.ctypes.data_as(ctypes.c_void_p),
                                    0, ctypes.byref(info))
        _check(st, allow=(0, 1))
        return psi, dpsi, SolveInfo(info.iterations, info.refinements, info.matvecs_fp32, info.matvecs_fp64,
                                    info.residual, bool(info.converged), st)

    def energy(self, psi, dpsi):
        p, dev = _dptr(psi, self.M)
        d, dev2 = _dptr(dpsi, self.M)
        if dev != dev2:
            raise ValueError("psi and dpsi must both be host or both device arrays")
        G = ctypes.c_double()
        prx = np.empty(self.n_charges)
        pp = p if dev else p.ctypes.data_as(ctypes.c_void_p)
        dd = d if dev else d.ctypes.data_as(ctypes.c_void_p)
        _check(lib.ctr_ibim_energy(self._h, pp, dd, dev, ctypes.byref(G), prx.ctypes.data_as(ctypes.c_void_p)))
        return float(G.value), prx

    def reaction_potential(self, psi, dpsi, points):
        p, dev = _dptr(psi, self.M)
        d, _ = _dptr(dpsi, self.M)
        z = np.ascontiguousarray(points, dtype=np.float64).reshape(-1, 3)
        out = np.empty(z.shape[0])
        pp = p if dev else p.ctypes.data_as(ctypes.c_void_p)
        dd = d if dev else d.ctypes.data_as(ctypes.c_void_p)
        _check(lib.ctr_ibim_reaction_potential(self._h, pp, dd, dev, z.shape[0], z.ctypes.data_as(ctypes.c_void_p),
                                               out.ctypes.data_as(ctypes.c_void_p)))
        return out

    def potential_map(self, psi, dpsi, points, precision: int = FP32_REFINE):
        """psi_rxn (Eq. 2.31) at many points (see ctr_ibim_potential_map).  Host arrays in, host array out;
        with psi, dpsi and points all CUDA tensors the work stays on the device and a tensor is returned."""
        if _is_torch(points):
            import torch
            n = points.numel() // 3
            pts, _ = _dptr(points, 3 * n)
            p, d1 = _dptr(psi, self.M)
            d, d2 = _dptr(dpsi, self.M)
            if not (d1 and d2):
                raise ValueError("with device points, psi and dpsi must be device tensors too")
            out = torch.empty(n, dtype=torch.float64, device=points.device)
            _check(lib.ctr_ibim_potential_map(self._h, p, d, n, pts, ctypes.c_void_p(out.data_ptr()),
                                              int(precision), 1))
            return out
        p = np.ascontiguousarray(psi, dtype=np.float64)
        d = np.ascontiguousarray(dpsi, dtype=np.float64)
        z = np.ascontiguousarray(points, dtype=np.float64).reshape(-1, 3)
        out = np.empty(z.shape[0])
        vp = lambda a: a.ctypes.data_as(ctypes.c_void_p)  # noqa: E731
        _check(lib.ctr_ibim_potential_map(self._h, vp(p), vp(d), z.shape[0], vp(z), vp(out), int(precision), 0))
        return out


@dataclasses.dataclass
class RequestResult:
    status: int
    M: int
    G_pol: float
    info: SolveInfo
    t_submit: float
    t_admit: float
    t_done: float

    @property
    def latency(self) -> float:
        return self.t_done - self.t_submit


class Server:
    """Continuous-batching request server (ctr_server_*): submit problems, poll or wait for results."""

    def __init__(self, max_slots: int = 16, hbm_budget_bytes: int = 0, step_quantum_ms: float = 20.0):
        """step_quantum_ms: pair work of one system per engine step; a longer operator application runs
        in parts over consecutive steps (0: never split).  Results do not depend on it."""
        o = _ServerOptions(int(max_slots), int(hbm_budget_bytes), float(step_quantum_ms))
        h = ctypes.c_void_p()
        _check(lib.ctr_server_create(ctypes.byref(o), ctypes.byref(h)))
        self._h = h

    def submit(self, grid_n, origin, h, sdist, eps_in, eps_out, kappa, charge_xyz, charge_q,
               options: Options | None = None) -> int:
        g = _Grid((ctypes.c_int64 * 3)(*[int(v) for v in grid_n]),
                  (ctypes.c_double * 3)(*[float(v) for v in origin]), float(h))
        sd = np.ascontiguousarray(sdist, dtype=np.float64)
        xyz = np.ascontiguousarray(charge_xyz, dtype=np.float64).reshape(-1, 3)
        q = np.ascontiguousarray(charge_q, dtype=np.float64).ravel()
        opt = (options or Options())._c()
        t = ctypes.c_uint64()
        _check(lib.ctr_server_submit(self._h, ctypes.byref(g), sd.ctypes.data_as(ctypes.c_void_p), float(eps_in),
                                     float(eps_out), float(kappa), q.size, xyz.ctypes.data_as(ctypes.c_void_p),
                                     q.ctypes.data_as(ctypes.c_void_p), ctypes.byref(opt), ctypes.byref(t)))
        return int(t.value)

    def submit_problem(self, prob, options: Options | None = None) -> int:
        g = prob.grid
        return self.submit(g.n, g.origin, g.h, prob.sdist, prob.eps_in, prob.eps_out, prob.kappa,
                           prob.charge_xyz, prob.charge_q, options or Options(tube_halfwidth=prob.tube))

    @staticmethod
    def _result(r: _RequestResult) -> RequestResult:
        i = r.info
        return RequestResult(r.status, int(r.M), float(r.G_pol),
                             SolveInfo(i.iterations, i.refinements, i.matvecs_fp32, i.matvecs_fp64, i.residual,
                                       bool(i.converged), r.status), r.t_submit, r.t_admit, r.t_done)

    def poll(self, ticket: int):
        done = ctypes.c_int()
        r = _RequestResult()
        _check(lib.ctr_server_poll(self._h, ticket, ctypes.byref(done), ctypes.byref(r)))
        return self._result(r) if done.value else None

    def wait(self, ticket: int, timeout: float = 0.0) -> RequestResult:
        r = _RequestResult()
        _check(lib.ctr_server_wait(self._h, ticket, float(timeout), ctypes.byref(r)))
        return self._result(r)

    def fetch(self, ticket: int, M: int):
        psi = np.empty(M)
        dpsi = np.empty(M)
        _check(lib.ctr_server_fetch(self._h, ticket, psi.ctypes.data_as(ctypes.c_void_p),
                                    dpsi.ctypes.data_as(ctypes.c_void_p), M))
        return psi, dpsi

    def release(self, ticket: int):
        _check(lib.ctr_server_release(self._h, ticket))

    def cancel(self, ticket: int):
        """Cancel a request that has not finished (see ctr_server_cancel)."""
        _check(lib.ctr_server_cancel(self._h, ticket))

    def stats(self) -> dict:
        st = _ServerStats()
        _check(lib.ctr_server_stats(self._h, ctypes.byref(st)))
        return {f: getattr(st, f) for f, _ in _ServerStats._fields_}

    def close(self):
        if getattr(self, "_h", None):
            lib.ctr_server_destroy(self._h)
            self._h = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:  # noqa: BLE001
            pass


def batch_solve(systems, device: bool = False):
    """Solve several CtrIbim systems together in one multi-slot engine (see ctr_ibim_batch_solve).

    Returns a list of (psi, dpsi, SolveInfo), one per system.
    """
    n = len(systems)
    if n == 0:
        return []
    handles = (ctypes.c_void_p * n)(*[s._h for s in systems])
    outs = []
    if device:
        import torch
        for s in systems:
            outs.append((torch.empty(s.M, dtype=torch.float64, device="cuda"),
                         torch.empty(s.M, dtype=torch.float64, device="cuda")))
        pp = (ctypes.c_void_p * n)(*[ctypes.c_void_p(o[0].data_ptr()) for o in outs])
        dp = (ctypes.c_void_p * n)(*[ctypes.c_void_p(o[1].data_ptr()) for o in outs])
    else:
        for s in systems:
            outs.append((np.empty(s.M), np.empty(s.M)))
        pp = (ctypes.c_void_p * n)(*[o[0].ctypes.data_as(ctypes.c_void_p) for o in outs])
        dp = (ctypes.c_void_p * n)(*[o[1].ctypes.data_as(ctypes.c_void_p) for o in outs])
    infos = (_Info * n)()
    st = lib.ctr_ibim_batch_solve(handles, n, pp, dp, 1 if device else 0, infos)
    _check(st, allow=(0, 1))
    return [(o[0], o[1], SolveInfo(i.iterations, i.refinements, i.matvecs_fp32, i.matvecs_fp64, i.residual,
                                   bool(i.converged), st)) for o, i in zip(outs, infos)]


def tuning_info():
    """(targets per thread, sources per chunk, unroll) the autotuner last chose for the FP32 pair kernel."""
    R, V, U = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    _check(lib.ctr_tuning_info(ctypes.byref(R), ctypes.byref(V), ctypes.byref(U)))
    return int(R.value), int(V.value), int(U.value)


def farfield_plan(ijk, excl_ptr, excl, margin: int, degree: int = 10, theta: float = 0.8, leaf: int = 128,
                  block: int = 256, min_far: int = 0) -> dict:
    """Host-only tree and interaction lists of the treecode (see ctr_farfield_plan); no GPU needed.

    ijk: (M, 3) integer grid indices of the nodes; excl_ptr / excl: their correction sets (CSR);
    min_far <= 0 selects (degree + 1)^3.  Besides the lists, returns the work of one application:
    near_pairs (targets x directly summed sources) and far_evaluations (targets x proxy points)."""
    ijk = np.ascontiguousarray(ijk, dtype=np.int32).reshape(-1, 3)
    ep = np.ascontiguousarray(excl_ptr, dtype=np.int32)
    ex = np.ascontiguousarray(excl, dtype=np.int32)
    M = ijk.shape[0]
    if ex.size == 0:
        ex = np.zeros(1, dtype=np.int32)
    c = lambda a: a.ctypes.data_as(ctypes.c_void_p)
    n_near, n_far = ctypes.c_int64(), ctypes.c_int64()
    args = (M, c(ijk), c(ep), c(ex), int(margin), int(degree), float(theta), int(leaf), int(block), int(min_far))
    _check(lib.ctr_farfield_plan(*args, None, ctypes.byref(n_near), ctypes.byref(n_far), None, None, None, None,
                                 None))
    nb = (M + block - 1) // block
    perm = np.empty(M, dtype=np.int64)
    near_ptr = np.empty(nb + 1, dtype=np.int64)
    near_rng = np.empty(2 * max(1, n_near.value), dtype=np.int64)
    far_ptr = np.empty(nb + 1, dtype=np.int64)
    fb = np.empty(max(1, n_far.value), dtype=np.int64)
    fe = np.empty(max(1, n_far.value), dtype=np.int64)
    _check(lib.ctr_farfield_plan(*args, c(perm), ctypes.byref(n_near), ctypes.byref(n_far), c(near_ptr),
                                 c(near_rng), c(far_ptr), c(fb), c(fe)))
    rng = near_rng[:2 * n_near.value].reshape(-1, 2)
    # work of one application: targets per block x (direct sources, proxies of the far clusters)
    nt = np.minimum(block, M - block * np.arange(nb)).astype(np.int64)
    cs = np.concatenate([[0], np.cumsum(rng[:, 1] - rng[:, 0])])
    near_per_block = cs[near_ptr[1:]] - cs[near_ptr[:-1]]
    far_per_block = np.diff(far_ptr)
    return {"perm": perm, "near_ptr": near_ptr, "near_rng": rng, "far_ptr": far_ptr, "far_begin": fb[:n_far.value],
            "far_end": fe[:n_far.value], "near_pairs": int(np.sum(nt * near_per_block)),
            "far_evaluations": int(np.sum(nt * far_per_block)) * (degree + 1) ** 3}


def set_wait_limit(polls: int):
    """Polls of the pair kernels' bounded waits (< 0: the default); see ctr_set_wait_limit."""
    _check(lib.ctr_set_wait_limit(int(polls)))


def kernel_launches() -> int:
    """Kernels the library has launched in this process so far."""
    return int(lib.ctr_kernel_launches())


def weight_tables() -> np.ndarray:
    """The library's correction-weight tables, shape (2, 9, 39, 39) (see ctr_weight_tables)."""
    out = np.empty((2, 9, 39, 39))
    _check(lib.ctr_weight_tables(out.ctypes.data_as(ctypes.c_void_p)))
    return out
