"""Checkpoint and resume of time-stepping states (kfbi_state_export /
kfbi_state_import): a run interrupted after k steps, exported, imported into
a fresh state on a fresh domain of the same description and continued gives
the uninterrupted run's field and density bit for bit (the blob carries the
fields, the densities and their extrapolation history, and on mixed domains
the superposition caches).  Blobs of another equation or grid are refused.
"""

import numpy as np
import pytest

from paper_2404_14864_gb300 import kfbi, workloads as W
from gpu_util import dev, ensure_built, host

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    ensure_built()


def _wave(desc, prec):
    ex = W.WaveExact()
    X, Y = W.grid_xy(desc)
    zx, zy = W.boundary_xy(desc)
    tau = 4.0 * (desc["hi"] - desc["lo"]) / desc["M"]
    dom = kfbi.Domain(desc, prec, tol=1e-10, maxit=1000)
    st = kfbi.State(dom, kfbi.KFBI_WAVE)
    st.init_wave(tau, 0.25, dev(ex.u(X, Y, 0)), dev(ex.lap(X, Y, 0)), dev(ex.u(X, Y, tau)),
                 dev(ex.lap(X, Y, tau)))
    g = [dev(ex.u(zx, zy, (k + 2) * tau)) for k in range(8)]
    return dom, st, g


@pytest.mark.parametrize("prec", [kfbi.KFBI_FP64, kfbi.KFBI_MIXED_FFT32, kfbi.KFBI_MIXED_TF32],
                         ids=["fp64", "fft32", "tf32"])
def test_resumed_wave_run_is_bitwise_identical(prec):
    desc = W.domain_desc(128, W.ellipse())
    dom, st, g = _wave(desc, prec)
    for k in range(8):
        st.step_wave(g[k])
    u_ref, phi_ref = host(st.get_u()), host(st.get_phi())
    dom.close()
    dom1, st1, g = _wave(desc, prec)
    for k in range(5):
        st1.step_wave(g[k])
    blob = st1.export()
    dom1.close()
    dom2, st2, g = _wave(desc, prec)
    st2.import_(blob)
    for k in range(5, 8):
        st2.step_wave(g[k])
    assert np.array_equal(host(st2.get_u()), u_ref)
    assert np.array_equal(host(st2.get_phi()), phi_ref)
    dom2.close()


def test_blob_of_another_state_is_refused():
    desc = W.domain_desc(128, W.ellipse())
    dom, st, g = _wave(desc, kfbi.KFBI_FP64)
    st.step_wave(g[0])
    blob = st.export()
    heat = kfbi.State(dom, kfbi.KFBI_HEAT)
    with pytest.raises(kfbi.KfbiError) as e:
        heat.import_(blob)
    assert e.value.status == 1
    other = kfbi.Domain(W.domain_desc(64, W.ellipse()), kfbi.KFBI_FP64)
    st_o = kfbi.State(other, kfbi.KFBI_WAVE)
    with pytest.raises(kfbi.KfbiError):
        st_o.import_(blob)
    with pytest.raises(kfbi.KfbiError):
        st.import_(blob[:100])
    other.close()
    dom.close()


def test_resumed_nonlinear_schrodinger_batch_is_bitwise_identical():
    """A w = 1 Schroedinger state (the paper's Ex. 5) stepped in a batch,
    exported after 2 of 4 steps and imported into a fresh state on a fresh
    domain, continues bit for bit: the blob carries w (set by
    kfbi_state_set_w, which batched steps use)."""
    import math
    ex = W.NonlinearSchrodingerExact()
    desc = W.domain_desc(64, W.ex5_star(0.2), lo=-math.pi, hi=math.pi)
    X, Y = W.grid_xy(desc)
    zx, zy = W.boundary_xy(desc)
    tau = 0.125
    V = dev(ex.v(X, Y))
    g = [dev(ex.u(zx, zy, (k + 1) * tau)) for k in range(4)]

    def fresh():
        dom = kfbi.Domain(desc, kfbi.KFBI_MIXED_TF32, tol=1e-12, maxit=800)
        st = kfbi.State(dom, kfbi.KFBI_SCHRODINGER)
        st.init_schrodinger(tau, dev(ex.u(X, Y, 0)), dev(ex.lap(X, Y, 0)))
        return dom, st, kfbi.Batch([dom])

    dom, st, b = fresh()
    st.set_w(ex.w)
    for k in range(4):
        b.step([st], [g[k]], [V])
    u_ref = host(st.get_u())
    b.close()
    dom.close()
    dom1, st1, b1 = fresh()
    st1.set_w(ex.w)
    for k in range(2):
        b1.step([st1], [g[k]], [V])
    blob = st1.export()
    b1.close()
    dom1.close()
    dom2, st2, b2 = fresh()   # w is not set here: it comes with the blob
    st2.import_(blob)
    for k in range(2, 4):
        b2.step([st2], [g[k]], [V])
    assert np.array_equal(host(st2.get_u()), u_ref)
    # the same run without w differs: the blob's w was used
    dom3, st3, b3 = fresh()
    for k in range(4):
        b3.step([st3], [g[k]], [V])
    assert not np.array_equal(host(st3.get_u()), u_ref)
    for o in (b2, dom2, b3, dom3):
        o.close()
