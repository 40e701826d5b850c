"""Named synthetic workloads: node set, triangulation, stencil size, polynomial
degree, kernel, firing-rate parameters, initial state, step size and step count.

Five workloads mirror the benchmark configurations:

* ``flat``       unit square, 1,500 nodes (152 boundary + 1,348 Halton), k = 24, deg 2,
                 Mexican hat (1, 0.1, 0.5, 0.2), beta 20, theta 0.2, Gaussian bump u0,
                 RK4 dt = 0.05 to t = 5 (100 steps), one trajectory;
* ``sphere``     unit sphere, 20,000 jittered Fibonacci nodes, k = 32, deg 3,
                 manufactured forcing (z = 0.5 + 0.3 cos t (z/2 + x y)), dt = 0.01,
                 200 steps;
* ``precision``  torus R = 1, r = 0.4, 100,000 jittered spiral-lattice nodes, k = 48,
                 deg 4, beta 50, six phase-shifted bumps as u0, dt = 0.05;
* ``batched``    256 trajectories on a 40,000-node sphere plus 64 on each of three
                 ellipsoids (axes 1 : 0.8 : 0.6) with 8,000 / 15,000 / 30,000 nodes,
                 k = 32, deg 3, per-trajectory beta ~ U[10, 40], theta ~ U[0.1, 0.3];
* ``adjoint``    torus (R = 1, r = 0.4) with 40,000 nodes, k = 32, deg 3, 200 steps of
                 dt = 0.02, checkpoints every 20 steps; target trajectory from kernel
                 (1.2, 0.08, 0.6, 0.25), gradients at (1, 0.1, 0.5, 0.2).

Only sizes and parameters live here; the arithmetic of the method is elsewhere.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

from . import (NodeSet, bump_u0, ellipsoid_fibonacci, random_bumps, sphere_fibonacci, spiral_bumps_u0,
               square_halton, torus_lattice)

KERNEL = (1.0, 0.1, 0.5, 0.2)


@dataclass
class Workload:
    name: str
    ns: NodeSet
    k: int
    deg: int
    kernel: tuple
    beta: np.ndarray
    theta: np.ndarray
    u0: np.ndarray          # B x n
    dt: float
    nsteps: int
    forcing: dict | None = None   # {"kind": 1, "c": ..., "a0": ...} (eigenvalues computed by the user)
    extra: dict = field(default_factory=dict)

    @property
    def n(self):
        return self.ns.n

    @property
    def B(self):
        return self.u0.shape[0]


def flat(n: int = 1500, seed: int = 0) -> Workload:
    ns = square_halton(n, seed)
    u0 = bump_u0(ns.nodes[:, :2], (0.5, 0.5), 0.8, 0.1)[None, :]
    return Workload("flat", ns, 24, 2, KERNEL, np.array([20.0]), np.array([0.2]), u0, 0.05, 100)


def sphere_mms_u0(nodes: np.ndarray, beta: float, theta: float, c: float = 0.5, a0: float = 0.3) -> np.ndarray:
    """Initial state of the manufactured sphere solution, u*(0) = theta + ln(z/(1-z))/beta,
    z = c + a0 (z_coord/2 + x y)."""
    Y = 0.5 * nodes[:, 2] + nodes[:, 0] * nodes[:, 1]
    z = c + a0 * Y
    return theta + np.log(z / (1.0 - z)) / beta


def sphere(n: int = 20000, seed: int = 0) -> Workload:
    ns = sphere_fibonacci(n, 0.1, seed)
    beta, theta = 20.0, 0.2
    u0 = sphere_mms_u0(ns.nodes, beta, theta)[None, :]
    return Workload("sphere", ns, 32, 3, KERNEL, np.array([beta]), np.array([theta]), u0, 0.01, 200,
                    forcing={"kind": 1, "c": 0.5, "a0": 0.3},
                    extra={"Y1": 0.5 * ns.nodes[:, 2], "Y2": ns.nodes[:, 0] * ns.nodes[:, 1]})


def precision(n: int = 100000, seed: int = 0) -> Workload:
    ns = torus_lattice(n, 1.0, 0.4, 0.15, seed)
    u0 = spiral_bumps_u0(ns)[None, :]
    return Workload("precision", ns, 48, 4, KERNEL, np.array([50.0]), np.array([0.2]), u0, 0.05, 20)


def batched(sizes=(40000, 8000, 15000, 30000), B=(256, 64, 64, 64), seed: int = 0):
    out = []
    for g, (n, b) in enumerate(zip(sizes, B)):
        if g == 0:
            ns = sphere_fibonacci(n, 0.1, seed)
            axes = (1.0, 1.0, 1.0)
        else:
            axes = (1.0, 0.8, 0.6)
            ns = ellipsoid_fibonacci(n, axes, 0.1, seed + g)
        u0, beta, theta = random_bumps(ns, b, seed + 100 + g, axes)
        out.append(Workload(f"batched[{g}]", ns, 32, 3, KERNEL, beta, theta, u0, 0.05, 20))
    return out


def adjoint(n: int = 40000, seed: int = 0) -> Workload:
    ns = torus_lattice(n, 1.0, 0.4, 0.15, seed)
    u0 = spiral_bumps_u0(ns)[None, :]
    return Workload("adjoint", ns, 32, 3, KERNEL, np.array([20.0]), np.array([0.2]), u0, 0.02, 200,
                    extra={"target_kernel": (1.2, 0.08, 0.6, 0.25), "C": 20})
