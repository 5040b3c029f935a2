"""Shared helpers of the GPU tests: run a request through the C ABI and the
same request through the oracle."""
import numpy as np

import workloads as W


def gpu_plan(spec, edges=None):
    from paper_1310_3435_gb300 import native as N
    return N.Plan(spec, edges=edges)


def gpu_sums(spec, **mc_kw):
    """Per-node sums from the CUDA path (host structured array)."""
    from paper_1310_3435_gb300 import native as N
    with gpu_plan(spec) as P:
        mc = P.mc_params(**mc_kw)
        return N.sdd_interface_mc_sums(P.handle, mc)


def oracle_edges(orc, spec):
    return orc.bmap_tables(spec.n, spec.bmap_mode, spec.family, spec.coef_mode, spec.params)


def oracle_sums(orc, spec, nodes=None, node_ids=None, paths=None, max_steps=None, tie=None,
                threads=None):
    E = oracle_edges(orc, spec)
    if nodes is None:
        nodes = orc.interface_nodes(spec.n, spec.sx, spec.sy)
    return orc.mc_nodes(spec.n, nodes, E, spec.family, spec.coef_mode, spec.params,
                        seed=spec.seed, paths=paths or spec.paths, dt=spec.dt,
                        max_steps=max_steps or spec.cap(),
                        tie_delta=spec.tie() if tie is None else tie,
                        node_ids=node_ids, threads=threads)


def gpu_means(g, n, nodes, nt=False):
    """Mean and stderr from GPU node sums (over non-tie paths if nt)."""
    S = g["sum_nt"] if nt else g["sum"]
    Q = g["sumsq_nt"] if nt else g["sumsq"]
    N = (g["paths"] - (g["ties"] if nt else 0)).astype(np.float64)[:, None]
    x0 = np.asarray(nodes, dtype=np.float64) / (n - 1.0)
    mean = x0 + S / N
    var = np.maximum(Q - S * S / N, 0.0) / (N * (N - 1.0))
    return mean, np.sqrt(var)
