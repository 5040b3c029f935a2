"""Plain FP64 CPU oracle of the stochastic-deterministic domain decomposition
(SDD) mesh generator of Bihlo & Haynes (arXiv 1310.3435).

TEST INFRASTRUCTURE ONLY.  Only tests/, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline leg import this package.  It shares no code with the
CUDA library in ``paper_1310_3435_gb300`` and imports nothing from it; the two
meet only through the seeded workload generator (``workloads.py``), which holds
none of the method's arithmetic.

Parts (each follows the passage it cites):

* ``interface_indices`` / ``interface_nodes``: the interface lines and the
  interface nodes where the stochastic representation is evaluated (§2.1,
  Fig. 1; the split rule I_k = round(k (n-1)/s) is this project's reading).
* ``bmap_tables``: the boundary map u|boundary = (f, g).  Identity map, or the
  paper's choice (§3.2): u1 = 0 / 1 on s = 0 / 1, u2 = 0 / 1 on t = 0 / 1, the
  other edges from the 1D form of the generator, -(c u')' = 0, solved by the
  same conservative differences as the 2D operator.
* ``mc_nodes``: the Monte Carlo estimate at interface nodes (§2.2), per node
  sums replayed in C (mc_oracle.c) over threads.
* ``edge_coefs`` / ``global_solve`` / ``stitch``: the finite
  difference form of eq. (WinslowTypeGridGenerator) (§3.2) in conservative form
  with c at edge midpoints; subdomains take the interface values as Dirichlet
  data (§2.1, §3.5).  The linear solve is scipy's sparse direct solver.
* ``closed_form_1d`` and ``torsion_exit_time``: the exact solutions used as pins.
* ``perona_malik``: FTCS anisotropic smoothing of a mesh (§3.4).
* ``cell_quality`` / ``mesh_quality``: Q(K), R_max, R_mean, l_inf (§3.1, §3.3);
  ``placement`` / ``interpolate_interface``: few-point interfaces (§3.6).
"""
from __future__ import annotations

import ctypes
import math
import os
from concurrent.futures import ThreadPoolExecutor

import numpy as np

from . import build as _build

FAMILY_BUMPS, FAMILY_RING, FAMILY_RIDGE, FAMILY_TABLE = 0, 1, 2, 3
COEF_W, COEF_INV_W = 0, 1
BMAP_IDENTITY, BMAP_PAPER_1D, BMAP_TABLE = 0, 1, 2
EDGE_BOTTOM, EDGE_TOP, EDGE_LEFT, EDGE_RIGHT = 0, 1, 2, 3

_lib = None


def lib():
    """The compiled C part (built on first use)."""
    global _lib
    if _lib is None:
        path = _build.build()
        L = ctypes.CDLL(path)
        dp = ctypes.POINTER(ctypes.c_double)
        u32p = ctypes.POINTER(ctypes.c_uint32)
        u64p = ctypes.POINTER(ctypes.c_uint64)
        ip = ctypes.POINTER(ctypes.c_int)
        L.oracle_philox4x32_10.argtypes = [u32p, u32p, u32p]
        L.oracle_philox4x32_10.restype = None
        L.oracle_normals.argtypes = [ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint32,
                                     ctypes.c_uint32, dp]
        L.oracle_normals.restype = None
        L.oracle_coef.argtypes = [ctypes.c_int, ctypes.c_int, dp, ctypes.c_double,
                                  ctypes.c_double]
        L.oracle_coef.restype = ctypes.c_double
        L.oracle_coef_array.argtypes = [ctypes.c_int, ctypes.c_int, dp, ctypes.c_int64,
                                        dp, dp, dp]
        L.oracle_coef_array.restype = None
        L.oracle_drift.argtypes = [ctypes.c_int, ctypes.c_int, dp, ctypes.c_double,
                                   ctypes.c_double, dp]
        L.oracle_drift.restype = None
        L.oracle_lookup.argtypes = [dp, ctypes.c_int, ctypes.c_double]
        L.oracle_lookup.restype = ctypes.c_double
        L.oracle_exit_point.argtypes = [ctypes.c_double] * 4 + [dp]
        L.oracle_exit_point.restype = ctypes.c_int
        L.oracle_path.argtypes = [ctypes.c_int, ctypes.c_double, ctypes.c_double,
                                  ctypes.c_uint32, ctypes.c_uint32, dp, ctypes.c_int,
                                  ctypes.c_int, dp, ctypes.c_uint64, ctypes.c_double,
                                  ctypes.c_uint64, ctypes.c_double, ctypes.c_int, ctypes.c_int,
                                  dp, u64p, ip, ip]
        L.oracle_path.restype = None
        L.oracle_mc_node.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                     ctypes.c_uint32, dp, ctypes.c_int, ctypes.c_int, dp,
                                     ctypes.c_uint64, ctypes.c_uint64, ctypes.c_uint64,
                                     ctypes.c_double, ctypes.c_uint64, ctypes.c_double,
                                     ctypes.c_int, ctypes.c_int, dp, u64p]
        L.oracle_mc_node.restype = None
        L.oracle_step_lengths.argtypes = [ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint32,
                                          ctypes.c_uint32, dp]
        L.oracle_step_lengths.restype = None
        L.oracle_bridge_exit.argtypes = [ctypes.c_double] * 5 + [ctypes.c_uint64, ctypes.c_uint32,
                                                                 ctypes.c_uint32, ctypes.c_uint32,
                                                                 dp, ip]
        L.oracle_bridge_exit.restype = ctypes.c_int
        _lib = L
    return _lib


def _dp(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _params(params) -> np.ndarray:
    """Family parameters as a C array (at least 32 entries; a TABLE density
    carries [tn, tn*tn values of ln w])."""
    q = np.asarray(params, dtype=np.float64).ravel()
    p = np.zeros(max(32, q.size), dtype=np.float64)
    p[: q.size] = q
    return p


# ------------------------------------------------------------------ RNG -----
def philox4x32_10(ctr, key) -> tuple:
    """Philox4x32-10 (Salmon et al., SC'11) of a 4-word counter and 2-word key."""
    c = (ctypes.c_uint32 * 4)(*[int(x) & 0xFFFFFFFF for x in ctr])
    k = (ctypes.c_uint32 * 2)(*[int(x) & 0xFFFFFFFF for x in key])
    o = (ctypes.c_uint32 * 4)()
    lib().oracle_philox4x32_10(c, k, o)
    return tuple(int(x) for x in o)


def normals(seed: int, node: int, path: int, step_pair: int) -> np.ndarray:
    """The four N(0,1) draws of steps 2*step_pair and 2*step_pair+1 (§2.2)."""
    z = np.zeros(4, dtype=np.float64)
    lib().oracle_normals(seed, node, path, step_pair, _dp(z))
    return z


# ------------------------------------------------------------- density -----
def coef(family: int, coef_mode: int, params, s, t) -> np.ndarray:
    """c(s,t) of -div(c grad u) = 0 (eq. WinslowTypeGridGenerator, c = w or 1/w)."""
    shape = np.broadcast(np.asarray(s), np.asarray(t)).shape
    s = np.array(np.broadcast_to(np.asarray(s, np.float64), shape), dtype=np.float64).ravel()
    t = np.array(np.broadcast_to(np.asarray(t, np.float64), shape), dtype=np.float64).ravel()
    out = np.empty(s.shape, dtype=np.float64)
    p = _params(params)
    lib().oracle_coef_array(family, coef_mode, _dp(p), s.size, _dp(s), _dp(t), _dp(out))
    return out.reshape(shape)


def drift(family: int, coef_mode: int, params, s: float, t: float) -> np.ndarray:
    """grad ln c at (s,t) (eq. WinslowTypeGridGeneratorExpanded)."""
    b = np.zeros(2, dtype=np.float64)
    p = _params(params)
    lib().oracle_drift(family, coef_mode, _dp(p), s, t, _dp(b))
    return b


# ---------------------------------------------------------------- plan -----
def interface_indices(n: int, s: int) -> list:
    """Grid lines of the s-1 interior interfaces of an s-way split of n points:
    I_k = round(k (n-1) / s), halves rounded up, in exact integer arithmetic."""
    return [(2 * k * (n - 1) + s) // (2 * s) for k in range(1, s)]


def interface_nodes(n: int, sx: int, sy: int) -> np.ndarray:
    """Interior grid nodes (i, j) lying on an interface line, each once, ordered
    by row j then column i.  Shape [n_nodes, 2] = (i, j)."""
    ix = set(interface_indices(n, sx))
    iy = set(interface_indices(n, sy))
    out = [(i, j) for j in range(1, n - 1) for i in range(1, n - 1) if i in ix or j in iy]
    return np.array(out, dtype=np.int64).reshape(-1, 2)


def subdomains(n: int, sx: int, sy: int) -> list:
    """Index boxes (i0, i1, j0, j1) of the subdomains: interior nodes are
    i0 < i < i1, j0 < j < j1 (the box edges are boundary or interface lines)."""
    X = [0] + interface_indices(n, sx) + [n - 1]
    Y = [0] + interface_indices(n, sy) + [n - 1]
    return [(X[a], X[a + 1], Y[b], Y[b + 1]) for b in range(sy) for a in range(sx)]


# -------------------------------------------------------- boundary map -----
def bmap_tables(n: int, mode: int, family: int = 0, coef_mode: int = 0, params=(0,),
                table=None) -> np.ndarray:
    """Boundary tables edges[comp][edge][k], k = node index along the edge.

    Edges: 0 bottom (t=0), 1 top (t=1), 2 left (s=0), 3 right (s=1).
    IDENTITY: u = (s, t).  PAPER_1D (§3.2): u1 = 0 on s=0, 1 on s=1, u2 = 0 on
    t=0, 1 on t=1; u1 on the bottom/top edge and u2 on the left/right edge solve
    the 1D generator -(c u')' = 0 with the conservative three-point difference
    (c at midpoints), i.e. u_k = sum_{m<k} 1/c_{m+1/2} / sum_m 1/c_{m+1/2}."""
    if mode == BMAP_TABLE:
        E = np.array(table, dtype=np.float64).reshape(2, 4, n)
        return E
    x = np.arange(n, dtype=np.float64) / float(n - 1)
    E = np.zeros((2, 4, n), dtype=np.float64)
    E[0, EDGE_BOTTOM] = x
    E[0, EDGE_TOP] = x
    E[0, EDGE_LEFT] = 0.0
    E[0, EDGE_RIGHT] = 1.0
    E[1, EDGE_BOTTOM] = 0.0
    E[1, EDGE_TOP] = 1.0
    E[1, EDGE_LEFT] = x
    E[1, EDGE_RIGHT] = x
    if mode == BMAP_IDENTITY:
        return E
    mid = (np.arange(n - 1, dtype=np.float64) + 0.5) / float(n - 1)

    def one_d(cvals):
        r = 1.0 / cvals
        cs = np.concatenate([[0.0], np.cumsum(r)])
        return cs / cs[-1]

    E[0, EDGE_BOTTOM] = one_d(coef(family, coef_mode, params, mid, 0.0))
    E[0, EDGE_TOP] = one_d(coef(family, coef_mode, params, mid, 1.0))
    E[1, EDGE_LEFT] = one_d(coef(family, coef_mode, params, 0.0, mid))
    E[1, EDGE_RIGHT] = one_d(coef(family, coef_mode, params, 1.0, mid))
    return E


def boundary_grid(n: int, edges: np.ndarray) -> np.ndarray:
    """[n, n, 2] array (index [j, i, comp]) holding the boundary map on the
    boundary rows/columns (rows j = 0, n-1 from the bottom/top tables, corners
    included; columns i = 0, n-1 from the left/right tables) and 0 inside."""
    U = np.zeros((n, n, 2), dtype=np.float64)
    for c in range(2):
        U[0, :, c] = edges[c, EDGE_BOTTOM]
        U[n - 1, :, c] = edges[c, EDGE_TOP]
        U[1:n - 1, 0, c] = edges[c, EDGE_LEFT, 1:n - 1]
        U[1:n - 1, n - 1, c] = edges[c, EDGE_RIGHT, 1:n - 1]
    return U


# ---------------------------------------------------------- Monte Carlo -----
def default_threads() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def mc_nodes(n: int, nodes, edges: np.ndarray, family: int, coef_mode: int, params,
             seed: int, paths: int, dt: float, max_steps: int, tie_delta: float = 0.0,
             node_ids=None, threads: int | None = None, path_begin: int = 0,
             exit_test: int = 0, stepper: int = 0) -> dict:
    """Per-node Monte Carlo sums (§2.2) for nodes [(i, j), ...].

    Node m uses counter word node_ids[m] (default: m) and paths
    [path_begin, path_begin + paths).  exit_test: 0 end-of-step test only,
    1 also the Brownian-bridge test (§2.2).  stepper: 0 constant step dt,
    1 exponential time stepping with mean step dt (§2.2).  Returns arrays
      S_all, Q_all, S_nt, Q_nt : [n_nodes, 2]  sums of d = F - X0 and d^2 over
                                 all paths / paths not flagged as ties
      paths, ties, non_exits, steps : [n_nodes] uint64
    """
    nodes = np.asarray(nodes, dtype=np.int64).reshape(-1, 2)
    m = nodes.shape[0]
    ids = np.arange(m, dtype=np.int64) if node_ids is None else np.asarray(node_ids)
    E = np.ascontiguousarray(edges, dtype=np.float64)
    p = _params(params)
    sums = np.zeros((m, 8), dtype=np.float64)
    counts = np.zeros((m, 4), dtype=np.uint64)
    L = lib()

    def run(k):
        i, j = int(nodes[k, 0]), int(nodes[k, 1])
        srow = sums[k]
        crow = counts[k]
        L.oracle_mc_node(n, i, j, int(ids[k]) & 0xFFFFFFFF, _dp(E), family, coef_mode,
                         _dp(p), seed, path_begin, path_begin + paths, dt, max_steps,
                         tie_delta, exit_test, stepper,
                         srow.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                         crow.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64)))

    nt = threads or default_threads()
    if nt <= 1 or m <= 1:
        for k in range(m):
            run(k)
    else:
        with ThreadPoolExecutor(max_workers=nt) as ex:
            list(ex.map(run, range(m)))
    return {
        "S_all": sums[:, 0:2].copy(), "Q_all": sums[:, 2:4].copy(),
        "S_nt": sums[:, 4:6].copy(), "Q_nt": sums[:, 6:8].copy(),
        "paths": counts[:, 0].copy(), "ties": counts[:, 1].copy(),
        "non_exits": counts[:, 2].copy(), "steps": counts[:, 3].copy(),
    }


def mc_estimate(nodes, n: int, S: np.ndarray, Q: np.ndarray, N) -> tuple:
    """Sample mean and its standard error from shifted sums (§2.2):
    mean = X0 + S/N,  stderr = sqrt((Q - S^2/N) / (N (N-1)))."""
    nodes = np.asarray(nodes, dtype=np.float64).reshape(-1, 2)
    x0 = nodes / float(n - 1)
    N = np.asarray(N, dtype=np.float64).reshape(-1, 1)
    mean = x0 + S / N
    var = np.maximum(Q - S * S / N, 0.0) / (N * (N - 1.0))
    return mean, np.sqrt(var)


def path(n: int, s0: float, t0: float, node: int, path_index: int, edges: np.ndarray,
         family: int, coef_mode: int, params, seed: int, dt: float, max_steps: int,
         tie_delta: float = 0.0, exit_test: int = 0, stepper: int = 0) -> dict:
    """One path from (s0, t0): score, step count, tie and cap flags."""
    E = np.ascontiguousarray(edges, dtype=np.float64)
    p = _params(params)
    F = np.zeros(2, dtype=np.float64)
    st = ctypes.c_uint64()
    tie = ctypes.c_int()
    cap = ctypes.c_int()
    lib().oracle_path(n, s0, t0, node, path_index, _dp(E), family, coef_mode, _dp(p),
                      seed, dt, max_steps, tie_delta, exit_test, stepper, _dp(F),
                      ctypes.byref(st),
                      ctypes.byref(tie), ctypes.byref(cap))
    return {"F": F, "steps": int(st.value), "tie": bool(tie.value), "capped": bool(cap.value)}


def step_lengths(seed: int, node: int, path: int, quad: int) -> np.ndarray:
    """Unit-mean exponentials of the lengths of steps 4 quad .. 4 quad + 3
    under exponential time stepping (§2.2)."""
    E = np.zeros(4, dtype=np.float64)
    lib().oracle_step_lengths(seed, node, path, quad, _dp(E))
    return E


def exit_point(xs: float, xt: float, ys: float, yt: float):
    """(edge or -1, exit point) of the Euler-Maruyama step x -> y (§2.2)."""
    e = np.zeros(2, dtype=np.float64)
    edge = lib().oracle_exit_point(xs, xt, ys, yt, _dp(e))
    return edge, e


def bridge_exit(xs, xt, ys, yt, dt, seed, node, path_index, k):
    """(edge or -1, exit point, tie) of the Brownian-bridge test of step k."""
    e = np.zeros(2, dtype=np.float64)
    tie = ctypes.c_int(0)
    edge = lib().oracle_bridge_exit(xs, xt, ys, yt, dt, seed, node, path_index, k, _dp(e),
                                    ctypes.byref(tie))
    return edge, e, bool(tie.value)


def lookup(table, tau: float) -> float:
    T = np.ascontiguousarray(table, dtype=np.float64)
    return lib().oracle_lookup(_dp(T), T.size, tau)


# ------------------------------------------------- finite differences -----
def edge_coefs(n: int, family: int, coef_mode: int, params) -> tuple:
    """c at the midpoints of the grid edges: cx[j, i] = c((i+1/2)h, jh) for
    i < n-1 and cy[j, i] = c(ih, (j+1/2)h) for j < n-1 (§3.2, conservative
    centred differences)."""
    h = 1.0 / (n - 1)
    i = np.arange(n, dtype=np.float64)
    mid = (np.arange(n - 1, dtype=np.float64) + 0.5) / float(n - 1)
    S, T = np.meshgrid(mid, i * h, indexing="xy")       # [n, n-1]: s = mid_i, t = j h
    cx = coef(family, coef_mode, params, S, T)
    S2, T2 = np.meshgrid(i * h, mid, indexing="xy")     # [n-1, n]: s = i h, t = mid_j
    cy = coef(family, coef_mode, params, S2, T2)
    return cx, cy


def _solve_box(U: np.ndarray, cx: np.ndarray, cy: np.ndarray, box) -> None:
    """Solve  sum_nbr c_edge (u_nbr - u_ij) = 0  at the interior nodes of the
    index box (i0, i1, j0, j1) with the values of U on the box's ring as
    Dirichlet data, for both components; writes the solution into U."""
    import scipy.sparse as sp
    import scipy.sparse.linalg as spla
    i0, i1, j0, j1 = box
    nx, ny = i1 - i0 - 1, j1 - j0 - 1
    if nx <= 0 or ny <= 0:
        return
    m = nx * ny

    def idx(i, j):
        return (j - j0 - 1) * nx + (i - i0 - 1)

    rows, cols, vals = [], [], []
    b = np.zeros((m, 2), dtype=np.float64)
    for j in range(j0 + 1, j1):
        for i in range(i0 + 1, i1):
            r = idx(i, j)
            nb = ((i + 1, j, cx[j, i]), (i - 1, j, cx[j, i - 1]),
                  (i, j + 1, cy[j, i]), (i, j - 1, cy[j - 1, i]))
            diag = 0.0
            for (ii, jj, c) in nb:
                diag += c
                if i0 < ii < i1 and j0 < jj < j1:
                    rows.append(r); cols.append(idx(ii, jj)); vals.append(-c)
                else:
                    b[r] += c * U[jj, ii]
            rows.append(r); cols.append(r); vals.append(diag)
    A = sp.csc_matrix((vals, (rows, cols)), shape=(m, m))
    x = spla.spsolve(A, b)
    x = np.asarray(x).reshape(m, 2)
    U[j0 + 1:j1, i0 + 1:i1, :] = x.reshape(ny, nx, 2)


def global_solve(n: int, edges: np.ndarray, family: int, coef_mode: int, params) -> np.ndarray:
    """Single-domain reference mesh (§3.2): the finite-difference system on the
    whole square with the boundary map as Dirichlet data.  [n, n, 2]."""
    cx, cy = edge_coefs(n, family, coef_mode, params)
    U = boundary_grid(n, edges)
    _solve_box(U, cx, cy, (0, n - 1, 0, n - 1))
    return U


def stitch(n: int, sx: int, sy: int, edges: np.ndarray, iface: np.ndarray, family: int,
           coef_mode: int, params) -> np.ndarray:
    """Non-iterative domain decomposition (§2.1, Fig. 1; §3.5): interface values
    (rows of ``iface`` in ``interface_nodes`` order) become Dirichlet data and
    every subdomain is solved once, independently.  Returns the mesh [n, n, 2]."""
    cx, cy = edge_coefs(n, family, coef_mode, params)
    U = boundary_grid(n, edges)
    nodes = interface_nodes(n, sx, sy)
    iface = np.asarray(iface, dtype=np.float64).reshape(-1, 2)
    U[nodes[:, 1], nodes[:, 0], :] = iface
    for box in subdomains(n, sx, sy):
        _solve_box(U, cx, cy, box)
    return U


def residual(U: np.ndarray, cx: np.ndarray, cy: np.ndarray) -> np.ndarray:
    """sum_nbr c_edge (u_nbr - u_ij) at every interior node, [n-2, n-2, 2]."""
    c = U[1:-1, 1:-1]
    r = (cx[1:-1, 1:, None] * (U[1:-1, 2:] - c) + cx[1:-1, :-1, None] * (U[1:-1, :-2] - c)
         + cy[1:, 1:-1, None] * (U[2:, 1:-1] - c) + cy[:-1, 1:-1, None] * (U[:-2, 1:-1] - c))
    return r


# --------------------------------------------------------- closed forms -----
def closed_form_1d(family: int, coef_mode: int, params, x: np.ndarray, axis: int = 0,
                   other: float = 0.5) -> np.ndarray:
    """Exact solution of the generator when c depends on one coordinate only
    (§3.2's 1D form): u(x) = int_0^x c^-1 / int_0^1 c^-1, by adaptive
    Gauss-Kronrod quadrature.  axis 0: c = c(s); axis 1: c = c(t)."""
    from scipy.integrate import quad

    def inv_c(y):
        s, t = (y, other) if axis == 0 else (other, y)
        return 1.0 / float(coef(family, coef_mode, params, s, t))

    # a tabulated density is smooth inside its cells only: integrate cell by cell
    tn = int(np.asarray(params, dtype=np.float64).ravel()[0]) if family == FAMILY_TABLE else 2
    edges = np.arange(tn) / (tn - 1.0)

    def integral(v):
        cuts = [0.0] + [e for e in edges[1:-1] if e < v] + [v]
        return sum(quad(inv_c, a, b, limit=400, epsabs=1e-15, epsrel=1e-13)[0]
                   for a, b in zip(cuts[:-1], cuts[1:]) if b > a)

    total = integral(1.0)
    return np.array([integral(float(v)) / total for v in np.atleast_1d(x)])


def torsion_exit_time(s: float, t: float, terms: int = 401) -> float:
    """Mean exit time from the unit square of X = sqrt(2) W started at (s,t):
    E[tau] = v with Lap v = -1, v = 0 on the boundary, by its sine series
    v = sum_{m,k odd} 16 sin(m pi s) sin(k pi t) / (pi^4 m k (m^2 + k^2))."""
    m = np.arange(1, terms + 1, 2, dtype=np.float64)
    M, K = np.meshgrid(m, m, indexing="ij")
    terms_ = 16.0 * np.sin(M * math.pi * s) * np.sin(K * math.pi * t) / (
        math.pi ** 4 * M * K * (M * M + K * K))
    return float(terms_.sum())


# ---------------------------------------------------- mesh smoothing -----
def perona_malik(U: np.ndarray, steps: int, dt: float, k: float) -> np.ndarray:
    """Anisotropic (Perona-Malik) smoothing of a mesh U[j, i, comp] (§3.4,
    eq. PeronaMalikDiffusion): `steps` forward-Euler, centred-in-space (FTCS)
    steps of length dt of u_t = div(g grad u) for each component separately,
    g = exp(-|grad u|^2 / k^2).  The conductance of each of a node's four
    edges comes from that edge's own difference, g(|u_nb - u| / h) (Perona
    and Malik's discrete scheme); boundary values stay fixed:
      u <- u + dt/h^2 sum_{nb in E,W,N,S} g(|u_nb - u| / h) (u_nb - u)."""
    U = np.array(U, dtype=np.float64, copy=True)
    return _perona_malik_spacing(U, steps, dt, k, 1.0 / (U.shape[0] - 1))


def _perona_malik_spacing(U: np.ndarray, steps: int, dt: float, k: float, h: float) -> np.ndarray:
    """The FTCS steps of `perona_malik` on a rectangular block of nodes
    U[j, i, comp] with node spacing h; the block's ring stays fixed."""
    U = np.array(U, dtype=np.float64, copy=True)
    r = dt / (h * h)

    def flux(d):
        return np.exp(-(d / h) ** 2 / (k * k)) * d

    for _ in range(steps):
        V = U.copy()
        for c in range(2):
            u = U[:, :, c]
            mid = u[1:-1, 1:-1]
            V[1:-1, 1:-1, c] = mid + r * (flux(u[1:-1, 2:] - mid) + flux(u[1:-1, :-2] - mid)
                                          + flux(u[2:, 1:-1] - mid) + flux(u[:-2, 1:-1] - mid))
        U = V
    return U


def smoothing_lines(n: int, s: int, shifted: bool) -> list:
    """Lines (grid indices, boundary included) that bound the blocks smoothed
    separately along one axis (§3.5, §4): the boundary and the interface lines
    of an s-way split; shifted, the midlines floor((a + b) / 2) of those
    blocks [a, b] instead, so that each original interface lies inside a block
    (the paper's second smoothing cycle over shifted subdomains)."""
    X = [0] + interface_indices(n, s) + [n - 1]
    if shifted:
        X = [0] + [(X[a] + X[a + 1]) // 2 for a in range(len(X) - 1)] + [n - 1]
    return sorted(set(X))


def perona_malik_subdomains(U: np.ndarray, steps: int, dt: float, k: float, sx: int, sy: int,
                            shifted: bool = False) -> np.ndarray:
    """Perona-Malik smoothing applied on each subdomain separately (§3.5, §4):
    every block between consecutive smoothing lines (`smoothing_lines`) is
    smoothed as a mesh of its own by `perona_malik`, its ring (the boundary and
    interface nodes around it) held fixed, with the spacing h of the whole
    grid.  The blocks only share their rings, so they are independent."""
    U = np.asarray(U, dtype=np.float64)
    n = U.shape[0]
    out = U.copy()
    X = smoothing_lines(n, sx, shifted)
    Y = smoothing_lines(n, sy, shifted)
    for b in range(len(Y) - 1):
        for a in range(len(X) - 1):
            i0, i1, j0, j1 = X[a], X[a + 1], Y[b], Y[b + 1]
            if i1 - i0 < 2 or j1 - j0 < 2:
                continue                       # no interior node
            block = U[j0:j1 + 1, i0:i1 + 1]
            sm = _perona_malik_spacing(block, steps, dt, k, 1.0 / (n - 1))
            out[j0 + 1:j1, i0 + 1:i1] = sm[1:-1, 1:-1]
    return out


# ------------------------------------------------------- mesh quality -----
def cell_quality(U: np.ndarray) -> np.ndarray:
    """Geometric quality Q(K) = 1/2 tr(J^T J) / sqrt(det(J^T J)) of every cell
    K of a mesh U[j, i, comp] (eq. Qmeasure, §3.1).  J is the Jacobian of the
    map (s, t) -> u on the cell, from the mean of the cell's two edge
    differences in each direction.  Q >= 1, Q = 1 for a square cell; inf for a
    folded cell (det J <= 0).  Shape [n-1, n-1]."""
    n = U.shape[0]
    h = 1.0 / (n - 1)
    du_ds = ((U[:-1, 1:] - U[:-1, :-1]) + (U[1:, 1:] - U[1:, :-1])) / (2 * h)
    du_dt = ((U[1:, :-1] - U[:-1, :-1]) + (U[1:, 1:] - U[:-1, 1:])) / (2 * h)
    a, c = du_ds[..., 0], du_ds[..., 1]          # J = [[a, b], [c, d]]
    b, d = du_dt[..., 0], du_dt[..., 1]
    det = a * d - b * c
    fro = a * a + b * b + c * c + d * d
    with np.errstate(divide="ignore", invalid="ignore"):
        q = np.where(det > 0, 0.5 * fro / np.where(det > 0, det, 1.0), np.inf)
    return q


def mesh_quality(U: np.ndarray, ref: np.ndarray | None = None, family: int = 0,
                 coef_mode: int = 0, params=(0.0,)) -> dict:
    """Q_max, Q_mean and folded cells of U; with a reference mesh also
    R_max = Q_max(ref)/Q_max(U), R_mean = Q_mean(ref)/Q_mean(U) and
    l_inf = max over nodes |rho(U) - rho(ref)|, rho = w (the mesh density)
    evaluated at the mesh points (§3.3)."""
    q = cell_quality(U)
    ok = np.isfinite(q)
    out = {"q_max": float(q[ok].max()) if ok.any() else math.inf,
           "q_mean": float(q[ok].mean()) if ok.any() else math.inf,
           "folds": int((~ok).sum())}
    if ref is not None:
        qr = cell_quality(ref)
        out["r_max"] = float(qr[np.isfinite(qr)].max() / out["q_max"])
        out["r_mean"] = float(qr[np.isfinite(qr)].mean() / out["q_mean"])
        c_u = coef(family, 0, params, U[..., 0], U[..., 1])
        c_r = coef(family, 0, params, ref[..., 0], ref[..., 1])
        out["l_inf"] = float(np.abs(c_u - c_r).max())
    return out


# ----------------------------------------------- few-point interfaces -----
def line_nodes(n: int, sx: int, sy: int) -> list:
    """Interface lines as lists of grid nodes, boundary endpoints included:
    ('v', i, [(i, j) for j = 0..n-1]) for each vertical line i in I_x and
    ('h', j, [(i, j) for i = 0..n-1]) for each horizontal line."""
    out = [("v", i, [(i, j) for j in range(n)]) for i in interface_indices(n, sx)]
    out += [("h", j, [(i, j) for i in range(n)]) for j in interface_indices(n, sy)]
    return out


def placement(n: int, sx: int, sy: int, mode: int, k: int = 7, family: int = 0,
              params=(0.0,)) -> np.ndarray:
    """Boolean mask over interface_nodes(n, sx, sy): the nodes where the Monte
    Carlo estimate is computed (§3.6).  Crossings of two lines are always
    included.  mode 0: every node; 1: k equispaced points per line
    (positions round(m (n-1)/(k+1)), m = 1..k); 2: the local extrema, along
    each line, of the first and second derivative of the density rho = w in
    the line's direction (centred differences of w at the line's nodes)."""
    nodes = interface_nodes(n, sx, sy)
    index = {(int(i), int(j)): q for q, (i, j) in enumerate(nodes)}
    mask = np.zeros(len(nodes), dtype=bool)
    if mode == 0:
        mask[:] = True
        return mask
    ix, iy = set(interface_indices(n, sx)), set(interface_indices(n, sy))
    for q, (i, j) in enumerate(nodes):
        if i in ix and j in iy:
            mask[q] = True
    h = 1.0 / (n - 1)
    for kind, _, pts in line_nodes(n, sx, sy):
        m = len(pts)
        if mode == 1:
            chosen = [int((2 * r * (m - 1) + (k + 1)) // (2 * (k + 1))) for r in range(1, k + 1)]
        else:
            s = np.array([p[0] for p in pts], dtype=np.float64) * h
            t = np.array([p[1] for p in pts], dtype=np.float64) * h
            rho = coef(family, 0, params, s, t)
            d1 = np.zeros(m)
            d2 = np.zeros(m)
            d1[1:-1] = (rho[2:] - rho[:-2]) / (2 * h)
            d2[1:-1] = (rho[2:] - 2 * rho[1:-1] + rho[:-2]) / (h * h)
            chosen = []
            for d in (d1, d2):
                for r in range(2, m - 2):
                    if (d[r] > d[r - 1] and d[r] >= d[r + 1]) or (d[r] < d[r - 1] and d[r] <= d[r + 1]):
                        chosen.append(r)
        for r in chosen:
            if 1 <= r <= m - 2:
                q = index.get(pts[r])
                if q is not None:
                    mask[q] = True
    return mask


def interpolate_interface(n: int, sx: int, sy: int, edges: np.ndarray, mask: np.ndarray,
                          values: np.ndarray) -> np.ndarray:
    """Fills every interface node from the values at the masked nodes by
    linear interpolation along its line, the line's boundary endpoints taking
    the boundary map (§3.6).  values: [n_nodes, 2] (rows of unmasked nodes
    ignored).  Vertical lines first, so crossings (always masked) and
    horizontal-line nodes never conflict."""
    nodes = interface_nodes(n, sx, sy)
    index = {(int(i), int(j)): q for q, (i, j) in enumerate(nodes)}
    U = boundary_grid(n, edges)
    out = np.array(values, dtype=np.float64).copy()
    for kind, _, pts in line_nodes(n, sx, sy):
        known_r, known_v = [], []
        for r, p in enumerate(pts):
            if r == 0 or r == len(pts) - 1:
                known_r.append(r)
                known_v.append(U[p[1], p[0]])
            else:
                q = index[p]
                if mask[q]:
                    known_r.append(r)
                    known_v.append(values[q])
        known_v = np.array(known_v)
        for r, p in enumerate(pts[1:-1], start=1):
            q = index[p]
            if not mask[q]:
                for c in range(2):
                    out[q, c] = np.interp(r, known_r, known_v[:, c])
    return out
