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
