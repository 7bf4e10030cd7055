"""The seeded input generators (synthetic/, no method arithmetic) follow their stated recipe (CPU):
workload sizes, the serving request stream, the operator test vectors."""
import numpy as np

from synthetic import (HEAT2D_K2_N16_Q2, HEAT3D_K2_N48_Q3, HEAT3D_K4_N32_Q3, heat3d_k3_n64, serving_stream,
                       uniform_vectors, zero_boundary)


def test_workload_node_counts():
    # (k N + 1)^d nodes, (k N - 1)^d interior
    assert (HEAT2D_K2_N16_Q2.ndofs, HEAT2D_K2_N16_Q2.n_interior) == (33 ** 2, 31 ** 2)
    assert (HEAT3D_K4_N32_Q3.ndofs, HEAT3D_K4_N32_Q3.n_interior) == (2_146_689, 2_048_383)
    assert (heat3d_k3_n64(3).ndofs, heat3d_k3_n64(3).n_interior) == (7_189_057, 6_967_871)
    assert (HEAT3D_K2_N48_Q3.ndofs, HEAT3D_K2_N48_Q3.n_interior) == (912_673, 857_375)


def test_serving_stream_is_seeded_and_follows_its_recipe():
    reqs = serving_stream(512)
    assert reqs == serving_stream(512) and reqs != serving_stream(512, seed=1)
    t = np.array([r.arrival_s for r in reqs])
    assert np.all(np.diff(t) > 0)
    gaps = np.diff(np.concatenate([[0.0], t]))
    assert abs(gaps.mean() * 200.0 - 1.0) < 0.15            # exponential gaps, rate 200/s (sd ~4.4 %)
    assert {r.dim for r in reqs} == {2, 3}
    assert {r.degree for r in reqs} == {1, 2, 3, 4}
    assert {r.cells for r in reqs} == {8, 16, 32, 64}
    assert {r.Q for r in reqs} == {2, 3, 4}
    tau = np.array([r.tau for r in reqs])
    assert tau.min() >= 1e-4 and tau.max() <= 1e-2
    assert abs(np.log10(tau).mean() + 3.0) < 0.1             # log-uniform on [1e-4, 1e-2] (sd ~0.026)
    assert [r.rid for r in reqs] == list(range(512))


def test_operator_vectors_and_boundary():
    u = uniform_vectors((2, 7 ** 3), seed=3)
    assert np.array_equal(u, uniform_vectors((2, 7 ** 3), seed=3))
    assert u.min() >= -1.0 and u.max() < 1.0 and abs(u.mean()) < 0.05
    z = zero_boundary(u, 3, 7)
    g = np.indices((7, 7, 7)).reshape(3, -1)[::-1]         # x fastest
    bnd = np.any((g == 0) | (g == 6), axis=0)
    assert np.all(z[:, bnd] == 0.0) and np.array_equal(z[:, ~bnd], u[:, ~bnd])
