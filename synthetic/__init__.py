"""Seeded synthetic inputs shared by the tests, the bench and the oracle legs.

This module holds no arithmetic of the method: only workload shapes, seeded
random vectors and the seeded serving request stream.  Both the CUDA path's
tests and the oracle draw their inputs from here.

Workloads (the heat problem u_t = Lap u + f on [0,1]^d with the manufactured
solution u = prod sin(pi x_a) cos t, homogeneous Dirichlet):

* ``HEAT2D_K2_N16_Q2``  : 2D, degree 2, 16^2 cells (1089 nodes), Q=2, tau=1e-2, 10 steps
* ``HEAT3D_K4_N32_Q3``  : 3D, degree 4, 32^3 cells (2,146,689 nodes), Q=3, tau=1e-3, 20 steps,
                          Chebyshev degree 3
* ``HEAT3D_K3_N64``     : 3D, degree 3, 64^3 cells (7,189,057 nodes), Q in 2..5, tau=1e-3
* ``HEAT3D_K2_N48_Q3``  : 3D, degree 2, 48^3 cells (912,673 nodes), Q=3, tau=1e-3
* serving stream        : 512 requests, Poisson arrivals at 200/s, dim in {2,3},
                          degree 1..4, N in {8,16,32,64}, Q in {2,3,4},
                          tau log-uniform in [1e-4, 1e-2]
"""
from dataclasses import dataclass

import numpy as np


@dataclass(frozen=True)
class Workload:
    name: str
    dim: int
    degree: int
    cells: int
    Q: int
    tau: float
    steps: int
    cheb_degree: int = 3

    @property
    def n1(self):
        return self.degree * self.cells + 1

    @property
    def ndofs(self):
        return self.n1 ** self.dim

    @property
    def n_interior(self):
        return (self.n1 - 2) ** self.dim


HEAT2D_K2_N16_Q2 = Workload("heat2d_k2_n16_q2", 2, 2, 16, 2, 1e-2, 10)
HEAT3D_K4_N32_Q3 = Workload("heat3d_k4_n32_q3", 3, 4, 32, 3, 1e-3, 20)
HEAT3D_K2_N48_Q3 = Workload("heat3d_k2_n48_q3", 3, 2, 48, 3, 1e-3, 10)


def heat3d_k3_n64(Q):
    return Workload(f"heat3d_k3_n64_q{Q}", 3, 3, 64, Q, 1e-3, 5)


def uniform_vectors(shape, seed=0):
    """uniform[-1, 1) float64 values from a seeded PCG64 generator (host array)."""
    return np.random.default_rng(seed).uniform(-1.0, 1.0, size=shape)


def zero_boundary(vec, dim, n1):
    """Copy of ``vec`` (..., n1^dim, x fastest) with the boundary nodes of the grid set to 0."""
    out = np.array(vec, copy=True)
    idx = np.arange(n1 ** dim)
    mask = np.zeros(n1 ** dim, dtype=bool)
    for a in range(dim):
        ia = (idx // (n1 ** a)) % n1
        mask |= (ia == 0) | (ia == n1 - 1)
    out[..., mask] = 0.0
    return out


@dataclass(frozen=True)
class Request:
    rid: int
    arrival_s: float
    dim: int
    degree: int
    cells: int
    Q: int
    tau: float


def serving_stream(n=512, rate=200.0, seed=0, cells=(8, 16, 32, 64), degrees=(1, 2, 3, 4),
                   stages=(2, 3, 4), dims=(2, 3), tau_range=(1e-4, 1e-2)):
    """Seeded request stream: exponential inter-arrival times, shapes drawn uniformly."""
    rng = np.random.default_rng(seed)
    t = 0.0
    out = []
    for i in range(n):
        t += rng.exponential(1.0 / rate)
        d = int(rng.choice(dims))
        k = int(rng.choice(degrees))
        N = int(rng.choice(cells))
        Q = int(rng.choice(stages))
        tau = float(np.exp(rng.uniform(np.log(tau_range[0]), np.log(tau_range[1]))))
        out.append(Request(i, t, d, k, N, Q, tau))
    return out
