"""Seeded synthetic workloads for the interface Monte Carlo and subdomain solves.

This module only draws and names inputs: grid size, subdomain split, density
family and parameters, boundary-map mode, paths per node, time step, seed.
It holds none of the method's arithmetic and imports neither the oracle nor
the CUDA library, so both can be fed the same inputs.

Density shapes follow the paper's monitor functions (all inputs are analytic,
there is no dataset):
  * Gaussian bump, as the running example (eq. MonitorFunctionRunningExample);
  * sech^2 ring, the building block of the five-ring monitor
    (eq. FiveRingMonitorFunction);
  * sinusoidal ridge, as the Mackenzie front (eq. MackenzieMonitorFunction).

Family parameter layouts (shared convention of both implementations):
  BUMPS (0): [nb, (A, cs, ct, ks, kt) * nb]   w = 1 + sum A exp(-ks(s-cs)^2 - kt(t-ct)^2)
  RING  (1): [A, cs, ct, k, r0]                w = 1 + A sech^2(k(|x-c| - r0))
  RIDGE (2): [A, k, t0, a, f]                  w = 1 + A exp(-k(t - t0 - a sin(2 pi f s))^2)
  TABLE (3): [tn, tn*tn values of ln w at the nodes (a/(tn-1), b/(tn-1)), row by row in b]
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field, replace

import numpy as np

FAMILY_BUMPS, FAMILY_RING, FAMILY_RIDGE, FAMILY_TABLE = 0, 1, 2, 3
COEF_W, COEF_INV_W = 0, 1
BMAP_IDENTITY, BMAP_PAPER_1D, BMAP_TABLE = 0, 1, 2
FP64, FP32_STEP = 0, 1
EXIT_END_OF_STEP, EXIT_BRIDGE = 0, 1
STEP_EULER, STEP_EXPONENTIAL = 0, 1
SOLVER_SOR, SOLVER_CG_FP32_REFINE, SOLVER_CG_JACOBI_FP32_REFINE = 0, 1, 2


@dataclass(frozen=True)
class MeshSpec:
    """One mesh-generation request."""
    n: int                       # grid points per side of the unit square
    sx: int                      # subdomains along s
    sy: int                      # subdomains along t
    family: int
    params: tuple
    coef_mode: int = COEF_W
    bmap_mode: int = BMAP_IDENTITY
    paths: int = 4000            # Monte Carlo paths per interface node
    dt: float = 1e-4             # Euler-Maruyama time step
    seed: int = 0
    precision: int = FP64
    max_steps: int = 0           # 0: default cap ceil(2/dt)
    tie_delta: float = -1.0      # <0: default (1e-11 in FP64 stepping, 0 in FP32)
    solver: int = SOLVER_SOR
    tol: float = 1e-10
    exit_test: int = EXIT_END_OF_STEP
    stepper: int = STEP_EULER    # EXPONENTIAL: step lengths ~ Exp(1/dt), mean dt
    label: str = ""

    def cap(self) -> int:
        return self.max_steps if self.max_steps > 0 else int(math.ceil(2.0 / self.dt))

    def tie(self) -> float:
        if self.tie_delta >= 0.0:
            return self.tie_delta
        return 1e-11 if self.precision == FP64 else 0.0

    def n_interface_nodes(self) -> int:
        """Unique interior nodes on interface lines: (sx-1)(n-2) + (sy-1)(n-2)
        minus the (sx-1)(sy-1) crossings."""
        return (self.sx - 1) * (self.n - 2) + (self.sy - 1) * (self.n - 2) - (
            self.sx - 1) * (self.sy - 1)


def bump(A, cs, ct, s) -> tuple:
    """One isotropic Gaussian bump with exponent -|x-c|^2 / s."""
    return (A, cs, ct, 1.0 / s, 1.0 / s)


def bumps(*bs) -> tuple:
    out = [float(len(bs))]
    for b in bs:
        out.extend(float(x) for x in b)
    return tuple(out)


def table_params(values) -> np.ndarray:
    """TABLE family parameters from a [tn, tn] array of ln w (row b = t
    index): a read-only flat array [tn, values...]."""
    v = np.asarray(values, dtype=np.float64)
    assert v.ndim == 2 and v.shape[0] == v.shape[1] and v.shape[0] >= 2
    out = np.concatenate([[float(v.shape[0])], v.ravel()])
    out.flags.writeable = False
    return out


def smooth_field(tn: int, seed: int = 0, amplitude: float = 1.0, modes: int = 4) -> np.ndarray:
    """A seeded smooth synthetic field on tn x tn nodes of the unit square (a
    sum of cosine modes with decaying random amplitudes), e.g. as a tabulated
    ln w standing in for a density that comes from a numerical solution."""
    rng = np.random.default_rng(seed)
    x = np.arange(tn) / (tn - 1.0)
    S, T = np.meshgrid(x, x, indexing="xy")
    out = np.zeros((tn, tn))
    for j in range(modes):
        for k in range(modes):
            c = rng.standard_normal() / (1.0 + j * j + k * k)
            out += c * np.cos(j * np.pi * S + rng.uniform(0, 2 * np.pi)) * np.cos(
                k * np.pi * T + rng.uniform(0, 2 * np.pi))
    return amplitude * out


# --------------------------------------------------------------- configs ----
def config1(**kw) -> MeshSpec:
    """Plain FP64, one mesh: 33x33, 2x2 split (61 unique interface nodes),
    w = 1 + 5 exp(-50 |x - (1/2,1/2)|^2), identity boundary map, 4000 paths,
    dt = 1e-4, seed 0; SOR to 1e-10."""
    spec = MeshSpec(n=33, sx=2, sy=2, family=FAMILY_BUMPS,
                    params=bumps((5.0, 0.5, 0.5, 50.0, 50.0)), paths=4000, dt=1e-4,
                    seed=0, precision=FP64, solver=SOLVER_SOR, tol=1e-10,
                    label="33x33 2x2 bump N=4000 dt=1e-4")
    return replace(spec, **kw)


def config2(**kw) -> MeshSpec:
    """257x257, 4x4 split (1521 unique interface nodes), ring
    w = 1 + 10 sech^2(50 (r - 1/4)), 1e5 paths, dt = 1e-5, FP32 stepping with
    FP64 accumulation; FP32 CG + FP64 refinement to 1e-10."""
    spec = MeshSpec(n=257, sx=4, sy=4, family=FAMILY_RING,
                    params=(10.0, 0.5, 0.5, 50.0, 0.25), paths=100000, dt=1e-5, seed=0,
                    precision=FP32_STEP, solver=SOLVER_CG_FP32_REFINE, tol=1e-10,
                    label="257x257 4x4 ring N=1e5 dt=1e-5")
    return replace(spec, **kw)


def config3(count: int = 256, seed: int = 0, **kw) -> list:
    """Batched uneven meshes: n uniform in {65,129,257,513}, sx, sy uniform in
    2..8, one bump with A ~ U[1,20], c ~ U[0.2,0.8]^2, s ~ U[0.002,0.05];
    2e4 paths, dt = 5e-5.  Drawn with numpy's PCG64 seeded by `seed`."""
    rng = np.random.default_rng(seed)
    out = []
    for m in range(count):
        n = int(rng.choice([65, 129, 257, 513]))
        sx, sy = int(rng.integers(2, 9)), int(rng.integers(2, 9))
        A = float(rng.uniform(1.0, 20.0))
        cs, ct = (float(v) for v in rng.uniform(0.2, 0.8, size=2))
        s = float(rng.uniform(0.002, 0.05))
        spec = MeshSpec(n=n, sx=sx, sy=sy, family=FAMILY_BUMPS,
                        params=bumps(bump(A, cs, ct, s)), paths=20000, dt=5e-5,
                        seed=seed * 100003 + m, precision=FP32_STEP,
                        solver=SOLVER_CG_FP32_REFINE, tol=1e-10,
                        label=f"batch{m} {n}x{n} {sx}x{sy}")
        out.append(replace(spec, **kw))
    return out


def config4(**kw) -> MeshSpec:
    """1025x1025, 8x8 split (14273 unique interface nodes), anisotropic ridge
    w = 1 + 20 exp(-200 (t - 0.3 - 0.2 sin 2 pi s)^2), 1e6 paths, dt = 1e-5,
    FP32 stepping with compensated FP64 sums."""
    spec = MeshSpec(n=1025, sx=8, sy=8, family=FAMILY_RIDGE,
                    params=(20.0, 200.0, 0.3, 0.2, 1.0), paths=1000000, dt=1e-5, seed=0,
                    precision=FP32_STEP, solver=SOLVER_CG_FP32_REFINE, tol=1e-10,
                    label="1025x1025 8x8 ridge N=1e6 dt=1e-5")
    return replace(spec, **kw)


@dataclass
class Arrival:
    t: float          # arrival time [s]
    spec: MeshSpec


def config5(count: int = 10000, rate: float = 200.0, seed: int = 0, paths: int = 0,
            n_max: int = 1025) -> list:
    """Serving stream: Poisson arrivals at `rate` req/s; n = round(exp U[ln 65,
    ln n_max]); sx, sy in 2..8; 1-3 bumps drawn as in the batched config.
    `paths` = 0 leaves the paths per node to the server's pilot (std-err
    target); otherwise fixed."""
    rng = np.random.default_rng(seed)
    t = 0.0
    out = []
    for m in range(count):
        t += float(rng.exponential(1.0 / rate))
        n = int(round(math.exp(rng.uniform(math.log(65), math.log(n_max)))))
        sx, sy = int(rng.integers(2, 9)), int(rng.integers(2, 9))
        sx, sy = min(sx, (n - 1) // 2), min(sy, (n - 1) // 2)
        nb = int(rng.integers(1, 4))
        bs = []
        for _ in range(nb):
            A = float(rng.uniform(1.0, 20.0))
            cs, ct = (float(v) for v in rng.uniform(0.2, 0.8, size=2))
            s = float(rng.uniform(0.002, 0.05))
            bs.append(bump(A, cs, ct, s))
        spec = MeshSpec(n=n, sx=sx, sy=sy, family=FAMILY_BUMPS, params=bumps(*bs),
                        paths=paths or 1024, dt=5e-5, seed=seed * 1000003 + m,
                        precision=FP32_STEP, solver=SOLVER_CG_FP32_REFINE, tol=1e-10,
                        label=f"req{m}")
        out.append(Arrival(t=t, spec=spec))
    return out


def small_parity_cases() -> list:
    """Small meshes spanning several work chunks and ragged tails, every
    density family and both coefficient modes; used by parity tests."""
    return [
        config1(paths=1000, label="cfg1 small N"),
        MeshSpec(n=17, sx=2, sy=3, family=FAMILY_RING, params=(10.0, 0.5, 0.5, 50.0, 0.25),
                 paths=777, dt=1e-4, seed=3, label="ring 17 2x3 ragged"),
        MeshSpec(n=21, sx=3, sy=2, family=FAMILY_RIDGE, params=(20.0, 200.0, 0.3, 0.2, 1.0),
                 paths=513, dt=1e-4, seed=5, coef_mode=COEF_INV_W, label="ridge 21 3x2 invw"),
        MeshSpec(n=13, sx=2, sy=2, family=FAMILY_BUMPS,
                 params=bumps((8.0, 0.3, 0.6, 30.0, 10.0), (3.0, 0.7, 0.2, 80.0, 80.0)),
                 paths=1500, dt=2e-4, seed=11, bmap_mode=BMAP_PAPER_1D,
                 label="2 bumps 13 paper1d"),
    ]
