"""The bench's workloads on the CPU: each problem's boundary data, initial
data and exact solution are one consistent manufactured solution, checked by
stepping the oracle a few steps at a small grid (no GPU), and each problem
names its configuration."""

import os
import sys

import numpy as np
import pytest

import oracle

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
import bench  # noqa: E402


class _Args:
    def __init__(self, workload, M):
        self.workload, self.M = workload, M


@pytest.mark.parametrize("workload,M,steps,bound", [
    ("wave1024", 64, 4, 5e-2),
    ("nls1024", 64, 4, 5e-2),
    ("heat1024-neumann", 64, 4, 2e-2),
])
def test_problem_is_a_consistent_manufactured_solution(workload, M, steps, bound):
    P = bench.make_problem(_Args(workload, M))
    d = oracle.make_domain(P.desc)
    st = P.oracle_stepper(oracle, d)
    for k in range(steps):
        P.oracle_step(st, k)
    err = np.abs(st.u - P.exact(steps))[d.interior_inside()].max()
    assert err < bound, err
    # and the error falls with the grid (the data are not merely small)
    P2 = bench.make_problem(_Args(workload, 2 * M))
    d2 = oracle.make_domain(P2.desc)
    st2 = P2.oracle_stepper(oracle, d2)
    t_end = steps * P.dt
    n2 = int(round(t_end / P2.dt))
    for k in range(n2):
        P2.oracle_step(st2, k)
    err2 = np.abs(st2.u - P2.exact(n2))[d2.interior_inside()].max()
    assert err2 < err, (err, err2)
    cfg = P.config("fp64")
    assert cfg["M"] == M and cfg["workload"].endswith(str(M))


@pytest.mark.parametrize("curve", ["ellipse", "star", "flower"])
def test_boundary_normal_is_the_outward_unit_normal(curve):
    from paper_2404_14864_gb300 import workloads as W
    c = {"ellipse": W.ellipse(), "star": W.star(), "flower": W.flower()}[curve]
    desc = W.domain_desc(64, c)
    d = oracle.make_domain(desc)
    t1, t2, _, _ = oracle.interface.tangent_data(d, d.theta)
    nx, ny = W.boundary_normal(desc)
    assert np.abs(np.hypot(nx, ny) - 1.0).max() < 1e-14
    assert np.abs(nx - t2).max() < 1e-13 and np.abs(ny + t1).max() < 1e-13
    # outward: a small step along n leaves the domain
    zx, zy = W.boundary_xy(desc)
    assert np.all(d.curve.level(zx + 1e-3 * nx, zy + 1e-3 * ny) > 0)
