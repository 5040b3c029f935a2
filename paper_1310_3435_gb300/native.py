"""ctypes binding of libsdd.so (include/sdd.h).

Argument marshalling only: every step of the Monte Carlo and the subdomain
solves runs in the library's CUDA kernels.  Functions keep the C names.
Arrays may be torch tensors (CUDA or CPU) or numpy arrays (host); CUDA tensors
are passed as device pointers, everything else as host pointers, and the
library copies and synchronises for host outputs.  Streams are
``torch.cuda.Stream`` objects, raw ``cudaStream_t`` integers or None (legacy
default stream).

The library must be built (``paper_1310_3435_gb300.build.build()``); there is
no fallback: loading fails loudly when it is missing.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

SDD_OK = 0
SDD_ERR_INVALID_ARG = -1
SDD_ERR_OOM = -2
SDD_ERR_CUDA = -3
SDD_ERR_NOT_CONVERGED = -4
SDD_ERR_NO_DEVICE = -5

SDD_FAMILY_BUMPS, SDD_FAMILY_RING, SDD_FAMILY_RIDGE, SDD_FAMILY_TABLE = 0, 1, 2, 3
SDD_MAX_TABLE = 4097
SDD_MAX_BUMPS, SDD_MAX_PARAMS = 6, 32
SDD_COEF_W, SDD_COEF_INV_W = 0, 1
SDD_BMAP_IDENTITY, SDD_BMAP_PAPER_1D, SDD_BMAP_TABLE = 0, 1, 2
SDD_FP64, SDD_FP32_STEP = 0, 1
SDD_SOLVER_SOR, SDD_SOLVER_CG_FP32_REFINE, SDD_SOLVER_CG_JACOBI_FP32_REFINE = 0, 1, 2
SDD_EXIT_END_OF_STEP, SDD_EXIT_BRIDGE = 0, 1
SDD_STEP_EULER, SDD_STEP_EXPONENTIAL = 0, 1
SDD_PLACE_ALL, SDD_PLACE_EQUISPACED, SDD_PLACE_EXTREMA = 0, 1, 2


class SddError(RuntimeError):
    def __init__(self, code: int, where: str, msg: str):
        super().__init__("%s failed (%d): %s" % (where, code, msg))
        self.code = code


class sdd_density(ctypes.Structure):
    _fields_ = [("family", ctypes.c_int32), ("coef_mode", ctypes.c_int32),
                ("n_params", ctypes.c_int32), ("tn", ctypes.c_int32),
                ("params", ctypes.c_double * SDD_MAX_PARAMS),
                ("table", ctypes.POINTER(ctypes.c_double))]


class sdd_bmap(ctypes.Structure):
    _fields_ = [("mode", ctypes.c_int32), ("reserved", ctypes.c_int32),
                ("edges", ctypes.POINTER(ctypes.c_double))]


class sdd_mc_params(ctypes.Structure):
    _fields_ = [("paths_per_node", ctypes.c_uint64), ("dt", ctypes.c_double),
                ("seed", ctypes.c_uint64), ("precision", ctypes.c_int32),
                ("chunk", ctypes.c_int32), ("max_steps", ctypes.c_uint64),
                ("tie_delta", ctypes.c_double), ("exit_test", ctypes.c_int32),
                ("stepper", ctypes.c_int32), ("reserved", ctypes.c_int32),
                ("path_begin", ctypes.c_uint64)]


class sdd_mc_stats(ctypes.Structure):
    _fields_ = [("paths", ctypes.c_uint64), ("path_steps", ctypes.c_uint64),
                ("ties", ctypes.c_uint64), ("non_exits", ctypes.c_uint64),
                ("max_stderr", ctypes.c_double)]


class sdd_node_sums(ctypes.Structure):
    _fields_ = [("sum", ctypes.c_double * 2), ("sumsq", ctypes.c_double * 2),
                ("sum_nt", ctypes.c_double * 2), ("sumsq_nt", ctypes.c_double * 2),
                ("paths", ctypes.c_uint64), ("ties", ctypes.c_uint64),
                ("non_exits", ctypes.c_uint64), ("steps", ctypes.c_uint64)]


NODE_SUMS_DTYPE = np.dtype([("sum", "<f8", (2,)), ("sumsq", "<f8", (2,)),
                            ("sum_nt", "<f8", (2,)), ("sumsq_nt", "<f8", (2,)),
                            ("paths", "<u8"), ("ties", "<u8"), ("non_exits", "<u8"),
                            ("steps", "<u8")])
assert NODE_SUMS_DTYPE.itemsize == ctypes.sizeof(sdd_node_sums)


class sdd_solve_params(ctypes.Structure):
    _fields_ = [("solver", ctypes.c_int32), ("max_iter", ctypes.c_int32),
                ("tol", ctypes.c_double), ("omega", ctypes.c_double),
                ("block_threads", ctypes.c_int32), ("reserved", ctypes.c_int32)]


class sdd_quality(ctypes.Structure):
    _fields_ = [("q_max", ctypes.c_double), ("q_mean", ctypes.c_double),
                ("folds", ctypes.c_int64), ("ref_q_max", ctypes.c_double),
                ("ref_q_mean", ctypes.c_double), ("ref_folds", ctypes.c_int64),
                ("r_max", ctypes.c_double), ("r_mean", ctypes.c_double),
                ("l_inf", ctypes.c_double)]


class sdd_solve_stats(ctypes.Structure):
    _fields_ = [("converged", ctypes.c_int32), ("subdomains", ctypes.c_int32),
                ("max_iterations", ctypes.c_int32), ("reserved", ctypes.c_int32),
                ("max_rel_residual", ctypes.c_double), ("node_iterations", ctypes.c_double)]


_lib = None


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Loads libsdd.so, building it first when it is missing or stale and
    nvcc is available.  Raises if the library cannot be had."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.LIB
    override = os.environ.get("SDD_LIBRARY")
    if override:                        # a specific build of libsdd.so (tuning variants)
        if not os.path.exists(override):
            raise ImportError("SDD_LIBRARY=%s does not exist" % override)
        path = override
    elif build_if_missing and not _build.up_to_date():
        try:
            path = _build.build()
        except Exception as e:          # no toolchain: fail loudly, no fallback
            if not os.path.exists(path):
                raise ImportError("libsdd.so is not built and cannot be built: %s" % e)
    if not os.path.exists(path):
        raise ImportError("libsdd.so not found at %s; run paper_1310_3435_gb300.build.build()"
                          % path)
    L = ctypes.CDLL(path)
    vp = ctypes.c_void_p
    P = ctypes.POINTER
    L.sdd_mesh_plan.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, P(sdd_density),
                                P(sdd_bmap), P(vp)]
    L.sdd_plan_num_nodes.argtypes = [vp, P(ctypes.c_int64)]
    L.sdd_plan_nodes.argtypes = [vp, vp]
    L.sdd_plan_edges.argtypes = [vp, vp]
    L.sdd_interface_mc.argtypes = [vp, P(sdd_mc_params), vp, vp, P(sdd_mc_stats), vp]
    L.sdd_interface_mc_sums.argtypes = [vp, P(sdd_mc_params), vp, vp]
    L.sdd_plan_last_mc_stats.argtypes = [vp, P(sdd_mc_stats)]
    L.sdd_subdomain_solve.argtypes = [vp, vp, P(sdd_solve_params), vp, P(sdd_solve_stats), vp]
    L.sdd_mesh_generate.argtypes = [vp, P(sdd_mc_params), P(sdd_solve_params), vp, vp, vp,
                                    P(sdd_mc_stats), P(sdd_solve_stats), vp]
    L.sdd_plan_destroy.argtypes = [vp]
    L.sdd_plan_destroy.restype = None
    L.sdd_last_error.argtypes = []
    L.sdd_last_error.restype = ctypes.c_char_p
    L.sdd_kernel_launches.argtypes = [P(ctypes.c_uint64)]
    L.sdd_plan_results.argtypes = [vp, vp, vp, vp, vp]
    L.sdd_batch_create.argtypes = [P(vp), ctypes.c_int, P(sdd_mc_params), P(sdd_solve_params),
                                   P(vp)]
    L.sdd_batch_run.argtypes = [vp, ctypes.c_int, vp]
    L.sdd_batch_run_phases.argtypes = [vp, ctypes.c_int, vp]
    L.sdd_batch_plan_stats.argtypes = [vp, ctypes.c_int, P(sdd_mc_stats), P(sdd_solve_stats)]
    L.sdd_batch_destroy.argtypes = [vp]
    L.sdd_batch_destroy.restype = None
    L.sdd_interface_mc_static.argtypes = [ctypes.c_int, vp, ctypes.c_int64, vp, P(sdd_density),
                                          P(sdd_mc_params), vp, vp, vp]
    L.sdd_interface_mc_static_stats.argtypes = [P(sdd_mc_stats), vp]
    L.sdd_plan_set_placement.argtypes = [vp, ctypes.c_int, ctypes.c_int]
    L.sdd_plan_placement.argtypes = [vp, vp, P(ctypes.c_int64)]
    L.sdd_mesh_quality.argtypes = [vp, vp, vp, P(sdd_quality), vp]
    L.sdd_mesh_smooth.argtypes = [vp, vp, ctypes.c_int, ctypes.c_double, ctypes.c_double, vp]
    L.sdd_mesh_smooth_subdomains.argtypes = [vp, vp, ctypes.c_int, ctypes.c_double,
                                             ctypes.c_double, ctypes.c_int, vp]
    u64p = P(ctypes.c_uint64)
    L.sdd_interface_mc_advance.argtypes = [vp, P(sdd_mc_params), ctypes.c_uint64, u64p, u64p, vp]
    L.sdd_interface_mc_finish.argtypes = [vp, P(sdd_mc_params), vp, vp, P(sdd_mc_stats), vp]
    L.sdd_mc_checkpoint_bytes.argtypes = [vp, u64p]
    L.sdd_mc_checkpoint_save.argtypes = [vp, vp, ctypes.c_uint64, vp]
    L.sdd_mc_checkpoint_load.argtypes = [vp, vp, ctypes.c_uint64, vp]
    for name in ("sdd_mesh_plan", "sdd_plan_num_nodes", "sdd_plan_nodes", "sdd_plan_edges",
                 "sdd_interface_mc", "sdd_interface_mc_sums", "sdd_plan_last_mc_stats",
                 "sdd_subdomain_solve", "sdd_mesh_generate", "sdd_kernel_launches",
                 "sdd_plan_results", "sdd_batch_create", "sdd_batch_run", "sdd_batch_run_phases",
                 "sdd_batch_plan_stats", "sdd_interface_mc_static",
                 "sdd_interface_mc_static_stats", "sdd_plan_set_placement",
                 "sdd_plan_placement", "sdd_mesh_quality", "sdd_mesh_smooth",
                 "sdd_mesh_smooth_subdomains", "sdd_interface_mc_advance", "sdd_interface_mc_finish", "sdd_mc_checkpoint_bytes",
                 "sdd_mc_checkpoint_save", "sdd_mc_checkpoint_load"):
        getattr(L, name).restype = ctypes.c_int
    _lib = L
    return L


def _check(rc: int, where: str, allow=()):
    if rc != SDD_OK and rc not in allow:
        msg = load().sdd_last_error()
        raise SddError(rc, where, msg.decode() if msg else "")
    return rc


def _ptr(a):
    """Raw pointer of a torch tensor or numpy array (None -> NULL)."""
    if a is None:
        return None
    if hasattr(a, "data_ptr"):
        if not a.is_contiguous():
            raise ValueError("arrays passed to libsdd must be contiguous")
        return ctypes.c_void_p(a.data_ptr())
    if isinstance(a, np.ndarray):
        if not a.flags["C_CONTIGUOUS"]:
            raise ValueError("arrays passed to libsdd must be contiguous")
        return ctypes.c_void_p(a.ctypes.data)
    raise TypeError("expected a torch tensor or numpy array, got %r" % type(a))


def _stream(s):
    if s is None:
        return None
    if hasattr(s, "cuda_stream"):
        return ctypes.c_void_p(s.cuda_stream)
    return ctypes.c_void_p(int(s))


# ---------------------------------------------------------- C-named calls --
def make_density(family: int, params, coef_mode: int = SDD_COEF_W) -> sdd_density:
    """Density record.  SDD_FAMILY_TABLE takes params = (tn, tn*tn values of
    ln w, row by row in t); the record then points at a numpy copy of the
    table, kept alive as the record's `_table` (the plan copies it)."""
    d = sdd_density()
    d.family = int(family)
    d.coef_mode = int(coef_mode)
    if d.family == SDD_FAMILY_TABLE:
        q = np.asarray(params, dtype=np.float64).ravel()
        tn = int(q[0])
        if q.size != 1 + tn * tn:
            raise ValueError("TABLE params must be (tn, tn*tn values of ln w)")
        d._table = np.ascontiguousarray(q[1:])
        d.tn = tn
        d.n_params = 0
        d.table = d._table.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
        return d
    p = [float(x) for x in params]
    if len(p) > SDD_MAX_PARAMS:
        raise ValueError("at most %d density parameters" % SDD_MAX_PARAMS)
    d.n_params = len(p)
    for q, v in enumerate(p):
        d.params[q] = v
    return d


def sdd_mesh_plan(n: int, sx: int, sy: int, density: sdd_density, bmap_mode: int = SDD_BMAP_IDENTITY,
                  edges=None):
    """Returns an opaque plan handle (ctypes.c_void_p)."""
    L = load()
    b = sdd_bmap()
    b.mode = int(bmap_mode)
    keep = None
    if edges is not None:
        keep = np.ascontiguousarray(edges, dtype=np.float64).ravel()
        if keep.size != 8 * n:
            raise ValueError("edges must hold [2][4][n] values")
        b.edges = keep.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    h = ctypes.c_void_p()
    _check(L.sdd_mesh_plan(int(n), int(sx), int(sy), ctypes.byref(density), ctypes.byref(b),
                           ctypes.byref(h)), "sdd_mesh_plan")
    return h


def sdd_plan_num_nodes(plan) -> int:
    v = ctypes.c_int64()
    _check(load().sdd_plan_num_nodes(plan, ctypes.byref(v)), "sdd_plan_num_nodes")
    return int(v.value)


def sdd_plan_nodes(plan) -> np.ndarray:
    m = sdd_plan_num_nodes(plan)
    out = np.zeros((m, 2), dtype=np.int32)
    _check(load().sdd_plan_nodes(plan, _ptr(out)), "sdd_plan_nodes")
    return out


def sdd_plan_edges(plan, n: int) -> np.ndarray:
    out = np.zeros((2, 4, n), dtype=np.float64)
    _check(load().sdd_plan_edges(plan, _ptr(out)), "sdd_plan_edges")
    return out


def mc_params(paths: int, dt: float, seed: int = 0, precision: int = SDD_FP64, chunk: int = 0,
              max_steps: int = 0, tie_delta: float = -1.0,
              exit_test: int = SDD_EXIT_END_OF_STEP,
              stepper: int = SDD_STEP_EULER, path_begin: int = 0) -> sdd_mc_params:
    m = sdd_mc_params()
    m.paths_per_node = int(paths)
    m.dt = float(dt)
    m.seed = int(seed) & 0xFFFFFFFFFFFFFFFF
    m.precision = int(precision)
    m.chunk = int(chunk)
    m.max_steps = int(max_steps)
    m.tie_delta = float(tie_delta)
    m.exit_test = int(exit_test)
    m.stepper = int(stepper)
    m.path_begin = int(path_begin)
    return m


def solve_params(solver: int = SDD_SOLVER_SOR, tol: float = 1e-10, max_iter: int = 0,
                 omega: float = 0.0, block_threads: int = 0) -> sdd_solve_params:
    s = sdd_solve_params()
    s.solver = int(solver)
    s.tol = float(tol)
    s.max_iter = int(max_iter)
    s.omega = float(omega)
    s.block_threads = int(block_threads)
    return s


def sdd_interface_mc(plan, mc: sdd_mc_params, mean=None, stderr=None, want_stats: bool = True,
                     stream=None):
    st = sdd_mc_stats()
    _check(load().sdd_interface_mc(plan, ctypes.byref(mc), _ptr(mean), _ptr(stderr),
                                   ctypes.byref(st) if want_stats else None, _stream(stream)),
           "sdd_interface_mc")
    return st if want_stats else None


def sdd_interface_mc_sums(plan, mc: sdd_mc_params, sums=None, stream=None):
    """Per-node sums; returns a numpy structured array when `sums` is None."""
    out = sums
    if out is None:
        out = np.zeros(sdd_plan_num_nodes(plan), dtype=NODE_SUMS_DTYPE)
    _check(load().sdd_interface_mc_sums(plan, ctypes.byref(mc), _ptr(out), _stream(stream)),
           "sdd_interface_mc_sums")
    return out


def sdd_plan_last_mc_stats(plan) -> sdd_mc_stats:
    st = sdd_mc_stats()
    _check(load().sdd_plan_last_mc_stats(plan, ctypes.byref(st)), "sdd_plan_last_mc_stats")
    return st


def sdd_subdomain_solve(plan, iface, sp: sdd_solve_params, mesh, want_stats: bool = True,
                        stream=None, allow_not_converged: bool = False):
    st = sdd_solve_stats()
    allow = (SDD_ERR_NOT_CONVERGED,) if allow_not_converged else ()
    _check(load().sdd_subdomain_solve(plan, _ptr(iface), ctypes.byref(sp), _ptr(mesh),
                                      ctypes.byref(st) if want_stats else None, _stream(stream)),
           "sdd_subdomain_solve", allow)
    return st if want_stats else None


def sdd_mesh_generate(plan, mc: sdd_mc_params, sp: sdd_solve_params, mesh, iface_mean=None,
                      iface_stderr=None, want_stats: bool = True, stream=None,
                      allow_not_converged: bool = False):
    ms, ss = sdd_mc_stats(), sdd_solve_stats()
    allow = (SDD_ERR_NOT_CONVERGED,) if allow_not_converged else ()
    _check(load().sdd_mesh_generate(plan, ctypes.byref(mc), ctypes.byref(sp), _ptr(mesh),
                                    _ptr(iface_mean), _ptr(iface_stderr),
                                    ctypes.byref(ms) if want_stats else None,
                                    ctypes.byref(ss) if want_stats else None, _stream(stream)),
           "sdd_mesh_generate", allow)
    return (ms, ss) if want_stats else None


def sdd_plan_results(plan, mesh=None, mean=None, stderr=None, stream=None) -> None:
    _check(load().sdd_plan_results(plan, _ptr(mesh), _ptr(mean), _ptr(stderr), _stream(stream)),
           "sdd_plan_results")


def sdd_batch_create(plans, mcs, sps):
    """plans: sequence of plan handles; mcs / sps: one parameter record each."""
    n = len(plans)
    if not (len(mcs) == len(sps) == n):
        raise ValueError("one mc and one solve record per plan")
    ph = (ctypes.c_void_p * n)(*[p.value if isinstance(p, ctypes.c_void_p) else p for p in plans])
    ma = (sdd_mc_params * n)(*mcs)
    sa = (sdd_solve_params * n)(*sps)
    h = ctypes.c_void_p()
    _check(load().sdd_batch_create(ph, n, ma, sa, ctypes.byref(h)), "sdd_batch_create")
    return h


def sdd_batch_run(batch, use_graph: bool = False, stream=None) -> None:
    _check(load().sdd_batch_run(batch, 1 if use_graph else 0, _stream(stream)), "sdd_batch_run")


def sdd_batch_run_phases(batch, phases: int, stream=None) -> None:
    _check(load().sdd_batch_run_phases(batch, int(phases), _stream(stream)), "sdd_batch_run_phases")


def sdd_batch_plan_stats(batch, index: int, allow_not_converged: bool = False):
    ms, ss = sdd_mc_stats(), sdd_solve_stats()
    allow = (SDD_ERR_NOT_CONVERGED,) if allow_not_converged else ()
    _check(load().sdd_batch_plan_stats(batch, int(index), ctypes.byref(ms), ctypes.byref(ss)),
           "sdd_batch_plan_stats", allow)
    return ms, ss


def sdd_batch_destroy(batch) -> None:
    if batch:
        load().sdd_batch_destroy(batch)


def sdd_interface_mc_static(n: int, nodes, edges, density: sdd_density, mc: sdd_mc_params,
                            mean, stderr=None, stream=None) -> None:
    """Allocation-free interface Monte Carlo (see include/sdd.h): device
    arrays nodes int32 [n_nodes][2], edges [2][4][n], mean/stderr [n_nodes][2]."""
    n_nodes = int(nodes.shape[0]) if hasattr(nodes, "shape") else 0
    _check(load().sdd_interface_mc_static(int(n), _ptr(nodes), n_nodes, _ptr(edges),
                                          ctypes.byref(density), ctypes.byref(mc), _ptr(mean),
                                          _ptr(stderr), _stream(stream)),
           "sdd_interface_mc_static")


def sdd_interface_mc_static_stats(stream=None) -> sdd_mc_stats:
    """Statistics of the last allocation-free call on the current device
    (synchronises `stream`)."""
    st = sdd_mc_stats()
    _check(load().sdd_interface_mc_static_stats(ctypes.byref(st), _stream(stream)),
           "sdd_interface_mc_static_stats")
    return st


def sdd_plan_set_placement(plan, mode: int, k: int = 7) -> None:
    _check(load().sdd_plan_set_placement(plan, int(mode), int(k)), "sdd_plan_set_placement")


def sdd_plan_placement(plan):
    """(mask [n_nodes] bool, number of Monte Carlo nodes)."""
    m = np.zeros(sdd_plan_num_nodes(plan), dtype=np.uint8)
    c = ctypes.c_int64()
    _check(load().sdd_plan_placement(plan, _ptr(m), ctypes.byref(c)), "sdd_plan_placement")
    return m.astype(bool), int(c.value)


def sdd_mesh_quality(plan, mesh, ref=None, stream=None) -> dict:
    q = sdd_quality()
    _check(load().sdd_mesh_quality(plan, _ptr(mesh), _ptr(ref), ctypes.byref(q), _stream(stream)),
           "sdd_mesh_quality")
    return {name: getattr(q, name) for name, _ in sdd_quality._fields_}


def sdd_mesh_smooth(plan, mesh, steps: int, dt: float, k: float, stream=None) -> None:
    """Perona-Malik smoothing of `mesh` [n][n][2] in place (host or device)."""
    _check(load().sdd_mesh_smooth(plan, _ptr(mesh), int(steps), float(dt), float(k),
                                  _stream(stream)), "sdd_mesh_smooth")


def sdd_mesh_smooth_subdomains(plan, mesh, steps: int, dt: float, k: float, shifted: bool = False,
                               stream=None) -> None:
    """Perona-Malik smoothing of `mesh` on each subdomain separately (interface
    lines held), or on the subdomains shifted by half a subdomain."""
    _check(load().sdd_mesh_smooth_subdomains(plan, _ptr(mesh), int(steps), float(dt), float(k),
                                             1 if shifted else 0, _stream(stream)),
           "sdd_mesh_smooth_subdomains")


def sdd_interface_mc_advance(plan, mc: sdd_mc_params, max_items: int, stream=None):
    """Runs the next work items of a split Monte Carlo run; returns
    (items_done, items_total)."""
    done, total = ctypes.c_uint64(), ctypes.c_uint64()
    _check(load().sdd_interface_mc_advance(plan, ctypes.byref(mc), int(max_items),
                                           ctypes.byref(done), ctypes.byref(total),
                                           _stream(stream)), "sdd_interface_mc_advance")
    return int(done.value), int(total.value)


def sdd_interface_mc_finish(plan, mc: sdd_mc_params, mean=None, stderr=None,
                            want_stats: bool = True, stream=None):
    st = sdd_mc_stats()
    _check(load().sdd_interface_mc_finish(plan, ctypes.byref(mc), _ptr(mean), _ptr(stderr),
                                          ctypes.byref(st) if want_stats else None,
                                          _stream(stream)), "sdd_interface_mc_finish")
    return st if want_stats else None


def sdd_mc_checkpoint_save(plan, stream=None) -> bytes:
    """The plan's split run as bytes (header + the sums of the items done)."""
    n = ctypes.c_uint64()
    _check(load().sdd_mc_checkpoint_bytes(plan, ctypes.byref(n)), "sdd_mc_checkpoint_bytes")
    buf = ctypes.create_string_buffer(int(n.value))
    _check(load().sdd_mc_checkpoint_save(plan, buf, n.value, _stream(stream)),
           "sdd_mc_checkpoint_save")
    return buf.raw


def sdd_mc_checkpoint_load(plan, data: bytes, stream=None) -> None:
    buf = ctypes.create_string_buffer(bytes(data), len(data))
    _check(load().sdd_mc_checkpoint_load(plan, buf, len(data), _stream(stream)),
           "sdd_mc_checkpoint_load")


def sdd_plan_destroy(plan) -> None:
    if plan:
        load().sdd_plan_destroy(plan)


def sdd_last_error() -> str:
    msg = load().sdd_last_error()
    return msg.decode() if msg else ""


def sdd_kernel_launches() -> int:
    v = ctypes.c_uint64()
    _check(load().sdd_kernel_launches(ctypes.byref(v)), "sdd_kernel_launches")
    return int(v.value)


# ----------------------------------------------------------- convenience --
class Plan:
    """Owning wrapper of a plan handle built from a request description with
    attributes n, sx, sy, family, params, coef_mode, bmap_mode (and, for
    SDD_BMAP_TABLE, `edges`)."""

    def __init__(self, spec, edges=None):
        self.spec = spec
        self.n = int(spec.n)
        self.density = make_density(spec.family, spec.params, getattr(spec, "coef_mode", 0))
        self.handle = sdd_mesh_plan(self.n, spec.sx, spec.sy, self.density,
                                    getattr(spec, "bmap_mode", SDD_BMAP_IDENTITY), edges)
        self.n_nodes = sdd_plan_num_nodes(self.handle)

    def nodes(self) -> np.ndarray:
        return sdd_plan_nodes(self.handle)

    def edges(self) -> np.ndarray:
        return sdd_plan_edges(self.handle, self.n)

    def mc_params(self, **kw) -> sdd_mc_params:
        s = self.spec
        args = dict(paths=s.paths, dt=s.dt, seed=s.seed, precision=s.precision,
                    max_steps=s.max_steps, tie_delta=s.tie_delta,
                    exit_test=getattr(s, "exit_test", SDD_EXIT_END_OF_STEP),
                    stepper=getattr(s, "stepper", SDD_STEP_EULER))
        args.update(kw)
        return mc_params(**args)

    def solve_params(self, **kw) -> sdd_solve_params:
        s = self.spec
        args = dict(solver=s.solver, tol=s.tol)
        args.update(kw)
        return solve_params(**args)

    def close(self):
        if self.handle:
            sdd_plan_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


class Batch:
    """Owning wrapper of a batch over `Plan` objects (which it keeps alive)."""

    def __init__(self, plans, mcs=None, sps=None):
        self.plans = list(plans)
        mcs = mcs or [p.mc_params() for p in self.plans]
        sps = sps or [p.solve_params() for p in self.plans]
        self.handle = sdd_batch_create([p.handle for p in self.plans], mcs, sps)

    def run(self, use_graph: bool = False, stream=None) -> None:
        sdd_batch_run(self.handle, use_graph, stream)

    def run_phases(self, phases: int, stream=None) -> None:
        sdd_batch_run_phases(self.handle, phases, stream)

    def stats(self, index: int, allow_not_converged: bool = False):
        return sdd_batch_plan_stats(self.handle, index, allow_not_converged)

    def close(self):
        if self.handle:
            sdd_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()
