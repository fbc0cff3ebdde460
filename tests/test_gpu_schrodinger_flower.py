"""GPU runs of the Schroedinger flower workload (Strang splitting,
Eqs. 3.8-3.12, kappa = 2i/dt, dt = h/2, flower r = 0.6 + 0.15 cos 4 theta):

- the Gaussian packet in the harmonic potential with g = 0 at 256^2 (the
  norm-drift run): the FFT32 (complex64 planes, FP64 refinement) and
  float64 (complex128) paths match the oracle's steps to 1e-8 and 1e-10
  relative L-infinity, and the discrete L2 norm over Omega stays within the
  oracle's drift bound (2e-3) over 40 steps;
- the plane wave (V = 0) at 256^2: the FFT32 path's error against the
  exact solution is at most 1.1x the float64 path's after the same steps.
"""

import math

import numpy as np
import pytest

import oracle
from paper_2404_14864_gb300 import kfbi, workloads as W
from gpu_util import dev, ensure_built, host, rel_linf

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    ensure_built()


def _packet(desc, d):
    X, Y = W.grid_xy(desc)
    pk = W.GaussianPacket(0.1, 0.0, 0.1, 5.0, 0.0)
    mask = d.interior_inside()
    u0 = np.where(mask, pk.u(X, Y), 0.0)
    lap0 = np.where(mask, pk.lap(X, Y), 0.0)
    n0 = math.sqrt(np.sum(np.abs(u0[mask]) ** 2) * d.h ** 2)
    return u0 / n0, lap0 / n0, W.harmonic_potential(X, Y)


def test_packet_steps_match_oracle_and_keep_the_norm():
    M = 256
    desc = W.domain_desc(M, W.flower())
    d = oracle.make_domain(desc)
    dt = 0.5 * d.h
    u0, lap0, V = _packet(desc, d)
    mask = d.interior_inside()
    g = np.zeros(d.nb, dtype=np.complex128)
    orc = oracle.SchrodingerStepper(d, dt, 1e-12)
    orc.init(u0, lap0)
    steps = 4
    for _ in range(steps):
        U = orc.step(g, V)
    for prec, bound in ((kfbi.KFBI_MIXED_FFT32, 1e-8), (kfbi.KFBI_FP64, 1e-10)):
        dom = kfbi.Domain(desc, prec, tol=1e-12, maxit=800)
        st = kfbi.State(dom, kfbi.KFBI_SCHRODINGER)
        st.init_schrodinger(dt, dev(u0), dev(lap0))
        Vd, gd = dev(V), dev(g)
        for _ in range(steps):
            st.step_schrodinger(Vd, gd)
        assert rel_linf(host(st.get_u())[mask], U[mask]) <= bound, prec
        if prec == kfbi.KFBI_MIXED_FFT32:
            norms = []
            for _ in range(40 - steps):
                st.step_schrodinger(Vd, gd)
                u = host(st.get_u())
                norms.append(math.sqrt(np.sum(np.abs(u[mask]) ** 2) * d.h ** 2))
            assert np.abs(np.array(norms) - 1.0).max() < 2e-3, norms
        dom.close()


def test_plane_wave_error_mixed_within_fp64():
    M = 256
    desc = W.domain_desc(M, W.flower())
    d = oracle.make_domain(desc)
    dt = 0.5 * d.h
    ex = W.PlaneWaveExact(5.0, 0.0)
    X, Y = W.grid_xy(desc)
    zx, zy = W.boundary_xy(desc)
    mask = d.interior_inside()
    errs = {}
    for prec in (kfbi.KFBI_MIXED_FFT32, kfbi.KFBI_FP64):
        dom = kfbi.Domain(desc, prec, tol=1e-10, maxit=800)
        st = kfbi.State(dom, kfbi.KFBI_SCHRODINGER)
        st.init_schrodinger(dt, dev(ex.u(X, Y, 0)), dev(ex.lap(X, Y, 0)))
        z = dev(np.zeros_like(X))
        for k in range(12):
            st.step_schrodinger(z, dev(ex.u(zx, zy, (k + 1) * dt)))
        errs[prec] = np.abs(host(st.get_u()) - ex.u(X, Y, 12 * dt))[mask].max()
        dom.close()
    assert errs[kfbi.KFBI_MIXED_FFT32] <= 1.1 * errs[kfbi.KFBI_FP64], errs
