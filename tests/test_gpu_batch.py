"""GPU tests of the batched path (kfbi_batch_step): instances of uneven
size, curve and equation advance together in grouped launches (one
persistent tcgen05 launch over all TF32 instances' tiles per pass, one FFT
launch per grid size for the FFT32 instances, a CUDA graph per lockstep
GMRES iteration).  Each instance must agree with the same domain stepped
alone to 1e-10 relative (both solve the BIE to GMRES tolerance 1e-12;
observed ~2e-12) and match the oracle's steps to 1e-8 (the mixed step bound
of the single-domain tests), with every configuration the autotuner can
choose."""

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


def _instances():
    rng = np.random.Generator(np.random.PCG64(3))
    return [
        ("heat", W.domain_desc(128, W.star())),
        ("heat", W.domain_desc(192, W.random_star(rng))),
        ("wave", W.domain_desc(256, W.ellipse())),
        ("schr", W.domain_desc(128, W.flower())),
        ("heat", W.domain_desc(96, W.random_star(rng))),
    ]


class _Run:
    """Inputs of one instance over a few steps."""

    def __init__(self, kind, desc):
        self.kind, self.desc = kind, desc
        self.X, self.Y = W.grid_xy(desc)
        self.zx, self.zy = W.boundary_xy(desc)
        h = (desc["hi"] - desc["lo"]) / desc["M"]
        self.tau = {"heat": h, "wave": 4 * h, "schr": 0.5 * h}[kind]
        self.ex = {"heat": W.HeatExact(), "wave": W.WaveExact(),
                   "schr": W.PlaneWaveExact(2.0, 1.0)}[kind]

    def make_state(self, dom):
        X, Y, ex, tau = self.X, self.Y, self.ex, self.tau
        if self.kind == "heat":
            st = kfbi.State(dom, kfbi.KFBI_HEAT)
            st.init_heat(tau, dev(ex.u(X, Y, 0)), dev(ex.lap(X, Y, 0)),
                         dev(ex.src(X, Y, 0) + ex.src(X, Y, tau)))
        elif self.kind == "wave":
            st = kfbi.State(dom, kfbi.KFBI_WAVE)
            st.init_wave(tau, 0.25, dev(ex.u(X, Y, 0)), dev(ex.lap(X, Y, 0)),
                         dev(ex.u(X, Y, tau)), dev(ex.lap(X, Y, tau)))
        else:
            st = kfbi.State(dom, kfbi.KFBI_SCHRODINGER)
            st.init_schrodinger(tau, dev(ex.u(X, Y, 0)), dev(ex.lap(X, Y, 0)))
        return st

    def inputs(self, k):
        """(g_next, src_or_v) of step k (0-based)."""
        X, Y, ex, tau = self.X, self.Y, self.ex, self.tau
        if self.kind == "heat":
            t1 = (k + 1) * tau
            return dev(ex.u(self.zx, self.zy, t1)), dev(ex.src(X, Y, t1) + ex.src(X, Y, t1 + tau))
        if self.kind == "wave":
            return dev(ex.u(self.zx, self.zy, (k + 2) * tau)), None
        return dev(ex.u(self.zx, self.zy, (k + 1) * tau)), dev(np.zeros_like(X))

    def step_alone(self, st, k):
        g, s = self.inputs(k)
        if self.kind == "heat":
            return st.step_heat(g, s)
        if self.kind == "wave":
            return st.step_wave(g)
        return st.step_schrodinger(s, g)


def _prec(engine, desc):
    """The engine's precision, TF32 where the FFT pass has no transform of
    that size (an "fft32" batch then mixes both engines)."""
    if engine == "fft32" and kfbi.fft_supported(desc["M"]):
        return kfbi.KFBI_MIXED_FFT32
    return kfbi.KFBI_MIXED_TF32


@pytest.mark.parametrize("engine", ["tf32", "fft32"])
def test_batch_steps_equal_single_instance_steps(engine):
    runs = [_Run(k, d) for k, d in _instances()]
    steps = 3
    # batched
    doms = [kfbi.Domain(r.desc, _prec(engine, r.desc), tol=1e-12, maxit=800) for r in runs]
    states = [r.make_state(d) for r, d in zip(runs, doms)]
    batch = kfbi.Batch(doms)
    for k in range(steps):
        ins = [r.inputs(k) for r in runs]
        infos = batch.step(states, [g for g, _ in ins], [s for _, s in ins])
        assert all(i["converged"] for i in infos)
    ub = [host(s.get_u()) for s in states]
    # alone
    for r, u_b in zip(runs, ub):
        d1 = kfbi.Domain(r.desc, _prec(engine, r.desc), tol=1e-12, maxit=800)
        s1 = r.make_state(d1)
        for k in range(steps):
            r.step_alone(s1, k)
        u1 = host(s1.get_u())
        assert rel_linf(u_b, u1) <= 1e-10, r.desc["M"]
    # the autotuner timed every candidate of every group and kept the fastest
    t = batch.tuning()
    engines = {x["engine"] for x in t}
    assert "tf32" in engines
    if engine == "fft32":
        fft_ms = sorted(x["M"] for x in t if x["engine"] == "fft32")
        assert fft_ms == sorted({r.desc["M"] for r in runs if r.desc["M"] != 96})
    for x in t:
        us = [c["us"] for c in x["candidates"]]
        assert len(us) >= 1 and all(u > 0 for u in us)
        assert us[x["chosen"]] == min(us)


def _oracle_stepper(r):
    """The oracle's stepper for a run, initialised as make_state does."""
    d = oracle.make_domain(r.desc)
    X, Y, ex, tau = r.X, r.Y, r.ex, r.tau
    if r.kind == "heat":
        st = oracle.HeatStepper(d, tau, 1e-12)
        st.init(ex.u(X, Y, 0), ex.lap(X, Y, 0), ex.src(X, Y, 0) + ex.src(X, Y, tau))
    elif r.kind == "wave":
        st = oracle.WaveStepper(d, tau, 1e-12)
        st.init(ex.u(X, Y, 0), ex.lap(X, Y, 0), ex.u(X, Y, tau), ex.lap(X, Y, tau))
    else:
        st = oracle.SchrodingerStepper(d, tau, 1e-12)
        st.init(ex.u(X, Y, 0), ex.lap(X, Y, 0))
    return d, st


def _oracle_step(r, st, k):
    X, Y, ex, tau = r.X, r.Y, r.ex, r.tau
    if r.kind == "heat":
        t1 = (k + 1) * tau
        return st.step(ex.u(r.zx, r.zy, t1), ex.src(X, Y, t1) + ex.src(X, Y, t1 + tau))
    if r.kind == "wave":
        return st.step(ex.u(r.zx, r.zy, (k + 2) * tau))
    return st.step(ex.u(r.zx, r.zy, (k + 1) * tau), np.zeros_like(X))


def _check_batch_against_oracle(runs, engine, steps, force=None, fields=False):
    doms = [kfbi.Domain(x.desc, _prec(engine, x.desc), tol=1e-12, maxit=800) for x in runs]
    states = [x.make_state(d) for x, d in zip(runs, doms)]
    batch = kfbi.Batch(doms)
    if force is not None:
        batch.force_candidate(force)
    orcs = [_oracle_stepper(x) for x in runs]
    for k in range(steps):
        ins = [x.inputs(k) for x in runs]
        infos = batch.step(states, [g for g, _ in ins], [s for _, s in ins])
        assert all(i["converged"] for i in infos)
        Us = [_oracle_step(x, st, k) for x, (_, st) in zip(runs, orcs)]
    # every instance, not only the first
    for x, st, (d, _), U in zip(runs, states, orcs, Us):
        m = d.interior_inside()
        assert rel_linf(host(st.get_u())[m], U[m]) <= 1e-8, (x.kind, x.desc["M"])
    tun = batch.tuning()
    us = [host(st.get_u()) for st in states]
    batch.close()
    for d in doms:
        d.close()
    return (tun, us) if fields else tun


@pytest.mark.parametrize("engine", ["tf32", "fft32"])
def test_batch_matches_oracle_for_every_instance(engine):
    runs = [_Run("heat", W.domain_desc(128, W.star())), _Run("wave", W.domain_desc(96, W.ellipse())),
            _Run("schr", W.domain_desc(64, W.flower())), _Run("heat", W.domain_desc(192, W.ellipse()))]
    _check_batch_against_oracle(runs, engine, 2)


def test_batch_every_autotuner_candidate_matches_oracle():
    """Each launch configuration the autotuner may pick (rows per block of
    the FFT passes; tile order and persistent CTAs of the tensor passes),
    forced in turn, gives the oracle's steps: FFT instances of two sizes
    (one complex) and TF32 instances in one batch.  No candidate changes a
    tile's or a row's arithmetic, so all give the same bits."""
    runs = [_Run("heat", W.domain_desc(128, W.star())), _Run("schr", W.domain_desc(192, W.flower())),
            _Run("wave", W.domain_desc(96, W.ellipse())), _Run("heat", W.domain_desc(130, W.star()))]
    fields = []
    for candidate in range(4):
        tun, us = _check_batch_against_oracle(runs, "fft32", 2, force=candidate, fields=True)
        assert {x["engine"] for x in tun} == {"fft32", "tf32"}
        for x in tun:
            assert x["chosen"] == candidate % len(x["candidates"])
        fields.append(us)
    for us in fields[1:]:
        assert all(np.array_equal(a, b) for a, b in zip(us, fields[0]))


def test_batch_nonlinear_schrodinger_equals_single_steps():
    """w = 1 (the paper's nonlinear example) through kfbi_state_set_w in a
    batch with a linear instance: each equals its domain stepped alone."""
    ex = W.NonlinearSchrodingerExact()
    desc = W.domain_desc(64, W.ex5_star(0.2), lo=-math.pi, hi=math.pi)
    X, Y = W.grid_xy(desc)
    zx, zy = W.boundary_xy(desc)
    tau = 0.125
    V = dev(ex.v(X, Y))
    lin = _Run("schr", W.domain_desc(128, W.flower()))

    def nl_state(dom):
        st = kfbi.State(dom, kfbi.KFBI_SCHRODINGER)
        st.init_schrodinger(tau, dev(ex.u(X, Y, 0)), dev(ex.lap(X, Y, 0)))
        return st

    doms = [kfbi.Domain(desc, kfbi.KFBI_MIXED_TF32, tol=1e-12, maxit=800),
            kfbi.Domain(lin.desc, kfbi.KFBI_MIXED_TF32, tol=1e-12, maxit=800)]
    states = [nl_state(doms[0]), lin.make_state(doms[1])]
    states[0].set_w(ex.w)
    batch = kfbi.Batch(doms)
    for k in range(3):
        g1, v1 = lin.inputs(k)
        infos = batch.step(states, [dev(ex.u(zx, zy, (k + 1) * tau)), g1], [V, v1])
        assert all(i["converged"] for i in infos)
    d1 = kfbi.Domain(desc, kfbi.KFBI_MIXED_TF32, tol=1e-12, maxit=800)
    s1 = nl_state(d1)
    for k in range(3):
        s1.step_schrodinger(V, dev(ex.u(zx, zy, (k + 1) * tau)), w=ex.w)
    assert rel_linf(host(states[0].get_u()), host(s1.get_u())) <= 1e-10
    with pytest.raises(kfbi.KfbiError):
        states[0].set_w(float("inf"))
    batch.close()
    for d in doms + [d1]:
        d.close()


def test_batches_of_different_sizes_step_in_any_order():
    """Kernel limits that depend on a batch's sizes (the Arnoldi step stages
    a whole boundary vector in shared memory) belong to the kernel, not to
    the batch: a large batch still steps after a small one was bound."""
    rng = np.random.Generator(np.random.PCG64(11))
    big = _Run("heat", W.domain_desc(1024, W.random_star(rng)))
    small = _Run("heat", W.domain_desc(128, W.random_star(rng)))
    d_big = kfbi.Domain(big.desc, kfbi.KFBI_MIXED_FFT32, tol=1e-10, maxit=800)
    d_small = kfbi.Domain(small.desc, kfbi.KFBI_MIXED_FFT32, tol=1e-10, maxit=800)
    s_big, s_small = big.make_state(d_big), small.make_state(d_small)
    b_big = kfbi.Batch([d_big])
    b_small = kfbi.Batch([d_small])
    for k in range(2):
        g, s = small.inputs(k)
        assert all(i["converged"] for i in b_small.step([s_small], [g], [s]))
        g, s = big.inputs(k)
        assert all(i["converged"] for i in b_big.step([s_big], [g], [s]))
