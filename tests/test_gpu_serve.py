"""GPU tests of the served stream (kfbi_server_*): continuous batching of
heat, wave and Schroedinger requests of uneven size.

- A request's final field is the same, bit for bit, when it runs alone and
  when it shares every tick with other requests that come and go.
- A served request agrees with the single-domain steppers to 1e-10 relative
  (both solve the BIE to GMRES tolerance 1e-12), and served heat, wave and
  Schroedinger requests match the oracle's steps to the mixed path's step
  bound (1e-8), on KFBI_MIXED_TF32 and KFBI_MIXED_FFT32 domains alike.
- Admission: at most max_resident requests are on the device; a request
  that does not fit the memory budget waits (first come first served) until
  an earlier one retires; one larger than the whole budget fails alone.
- The device bytes the server charges are exact (plan-based count equals
  the allocations of the domain and state).
"""

import numpy as np
import pytest

import oracle
from paper_2404_14864_gb300 import kfbi, workloads as W
from gpu_util import dev, ensure_built, host, rel_linf

pytestmark = pytest.mark.gpu

TOL = 1e-12


@pytest.fixture(scope="module", autouse=True)
def _lib():
    ensure_built()


PRECS = {"tf32": kfbi.KFBI_MIXED_TF32, "fft32": kfbi.KFBI_MIXED_FFT32}


def _prec(name, desc):
    """FFT32 where the grid has an FFT pass (an "fft32" mix then holds both engines)."""
    if name == "fft32" and not kfbi.fft_supported(desc["M"]):
        return kfbi.KFBI_MIXED_TF32
    return PRECS[name]


def _submit(srv, kind, desc, steps, arrival, inputs=None, prec="tf32"):
    x = inputs or W.request_inputs(kind, desc, steps)
    return srv.submit(desc, x["equation"], steps, x["dt"], arrival, x["u0"], x["lap_u0"], x["g"],
                      theta=x.get("theta", 0.25), u1=x.get("u1"), lap_u1=x.get("lap_u1"),
                      src_init=x.get("src_init"), src_profile=x.get("src_profile"),
                      src_coef=x.get("src_coef"), potential=x.get("potential"), tol=TOL,
                      maxit=800, precision=_prec(prec, desc))


def _mix():
    rng = np.random.Generator(np.random.PCG64(11))
    # (kind, desc, steps, arrival tick)
    return [
        ("heat", W.domain_desc(128, W.random_star(rng)), 4, 0.0),
        ("wave", W.domain_desc(96, W.random_star(rng)), 3, 0.0),
        ("schrodinger", W.domain_desc(128, W.random_star(rng)), 3, 1.0),
        ("heat", W.domain_desc(64, W.random_star(rng)), 2, 2.0),
        ("wave", W.domain_desc(160, W.random_star(rng)), 3, 2.0),
        ("schrodinger", W.domain_desc(96, W.random_star(rng)), 2, 5.0),
    ]


def _drain(srv, n, max_ticks=200):
    """Tick on virtual time 0, 1, 2, ... until all n requests are final."""
    seen = []
    for t in range(max_ticks):
        seen.append(srv.tick(float(t)))
        if all(srv.info(i)["state"] in (kfbi.REQ_DONE, kfbi.REQ_FAILED) for i in range(n)):
            return seen
    raise AssertionError("requests did not finish")


@pytest.mark.parametrize("prec", ["tf32", "fft32"])
def test_served_result_is_the_same_alone_and_in_the_mix(prec):
    mix = _mix()
    srv = kfbi.Server(max_resident=3, plan_threads=0, restart=50)
    ids = [_submit(srv, k, d, s, a, prec=prec) for k, d, s, a in mix]
    seen = _drain(srv, len(ids))
    assert max(seen) == 3  # the slot limit was reached: requests overlapped
    mixed = []
    for i in ids:
        info = srv.info(i)
        assert info["state"] == kfbi.REQ_DONE, info
        mixed.append(srv.result(i).copy())
    st = srv.stats()
    assert st["completed"] == len(ids) and st["failed"] == 0
    assert st["peak_device_bytes"] > 0 and st["h2d_bytes"] > 0 and st["d2h_bytes"] > 0
    srv.close()
    for (k, d, s, a), u_mix in zip(mix, mixed):
        alone = kfbi.Server(max_resident=1, plan_threads=0, restart=50)
        j = _submit(alone, k, d, s, 0.0, prec=prec)
        _drain(alone, 1)
        u_alone = alone.result(j)
        assert np.array_equal(u_alone, u_mix), (k, d["M"], rel_linf(u_mix, u_alone))
        alone.close()


@pytest.mark.parametrize("prec", ["tf32", "fft32"])
def test_served_request_agrees_with_single_domain_steppers(prec):
    rng = np.random.Generator(np.random.PCG64(5))
    for kind in ("heat", "wave", "schrodinger"):
        desc = W.domain_desc(128, W.random_star(rng))
        steps = 3
        x = W.request_inputs(kind, desc, steps)
        srv = kfbi.Server(max_resident=2, plan_threads=1, restart=50)
        i = _submit(srv, kind, desc, steps, 0.0, x, prec=prec)
        _drain(srv, 1)
        u_srv = srv.result(i)
        srv.close()
        dom = kfbi.Domain(desc, _prec(prec, desc), restart=50, tol=TOL, maxit=800)
        st = kfbi.State(dom, x["equation"])
        if kind == "heat":
            st.init_heat(x["dt"], dev(x["u0"]), dev(x["lap_u0"]), dev(x["src_init"]))
            for n in range(steps):
                st.step_heat(dev(x["g"][n]), dev(x["src_coef"][n] * x["src_profile"]))
        elif kind == "wave":
            st.init_wave(x["dt"], x["theta"], dev(x["u0"]), dev(x["lap_u0"]), dev(x["u1"]),
                         dev(x["lap_u1"]))
            for n in range(steps):
                st.step_wave(dev(x["g"][n]))
        else:
            st.init_schrodinger(x["dt"], dev(x["u0"]), dev(x["lap_u0"]))
            v = dev(x["potential"])
            for n in range(steps):
                st.step_schrodinger(v, dev(x["g"][n]))
        u1 = host(st.get_u())
        assert rel_linf(u_srv, u1) <= 1e-10, kind


@pytest.mark.parametrize("prec", ["tf32", "fft32"])
def test_served_requests_match_oracle(prec):
    """Heat, wave and Schroedinger requests served together (one tick steps
    all three) against the oracle's steppers on the same inputs."""
    rng = np.random.Generator(np.random.PCG64(17))
    reqs = [("heat", W.domain_desc(128, W.star()), 2), ("wave", W.domain_desc(192, W.ellipse()), 2),
            ("schrodinger", W.domain_desc(64, W.random_star(rng)), 3)]
    xs = [W.request_inputs(k, d, n) for k, d, n in reqs]
    srv = kfbi.Server(max_resident=4, plan_threads=0, restart=50)
    ids = [_submit(srv, k, d, n, 0.0, x, prec=prec) for (k, d, n), x in zip(reqs, xs)]
    _drain(srv, len(ids))
    for (kind, desc, steps), x, i in zip(reqs, xs, ids):
        u = srv.result(i)
        d = oracle.make_domain(desc)
        if kind == "heat":
            orc = oracle.HeatStepper(d, x["dt"], 1e-12)
            orc.init(x["u0"], x["lap_u0"], x["src_init"])
            for n in range(steps):
                U = orc.step(x["g"][n], x["src_coef"][n] * x["src_profile"])
        elif kind == "wave":
            orc = oracle.WaveStepper(d, x["dt"], 1e-12)
            orc.init(x["u0"], x["lap_u0"], x["u1"], x["lap_u1"], theta=x["theta"])
            for n in range(steps):
                U = orc.step(x["g"][n])
        else:
            orc = oracle.SchrodingerStepper(d, x["dt"], 1e-12)
            orc.init(x["u0"], x["lap_u0"])
            for n in range(steps):
                U = orc.step(x["g"][n], x["potential"])
        m = d.interior_inside()
        assert rel_linf(u[m], U[m]) <= 1e-8, (kind, desc["M"])
    srv.close()


def test_admission_by_slots_memory_and_fifo():
    rng = np.random.Generator(np.random.PCG64(21))
    descs = [W.domain_desc(128, W.random_star(rng)) for _ in range(4)]
    steps = [2, 3, 2, 2]
    # bytes the server will charge for each request
    need = []
    for d, s in zip(descs, steps):
        p = kfbi.Plan(d, kfbi.KFBI_MIXED_TF32, 50)
        data = s * d["nb"] * 8 + (d["M"] - 1) ** 2 * 8
        need.append(p.device_bytes(kfbi.KFBI_HEAT) + data)
        p.close()
    # budget: any one request fits, no two do
    budget = max(need) + min(need) // 2
    srv = kfbi.Server(max_resident=8, hbm_budget_bytes=budget, hbm_reserve_bytes=0,
                      plan_threads=0, restart=50)
    ids = [_submit(srv, "heat", d, s, 0.0) for d, s in zip(descs, steps)]
    seen = _drain(srv, len(ids))
    assert max(seen) == 1
    infos = [srv.info(i) for i in ids]
    for a, b in zip(infos, infos[1:]):
        assert b["admit_tick"] == a["finish_tick"], (a, b)  # admitted as the earlier one retired
    for i, inf in enumerate(infos):
        assert inf["state"] == kfbi.REQ_DONE and inf["device_bytes"] == need[i]
    assert srv.stats()["peak_device_bytes"] == max(need)
    srv.close()
    # slots: four requests, two slots
    srv = kfbi.Server(max_resident=2, plan_threads=0, restart=50)
    ids = [_submit(srv, "heat", d, s, 0.0) for d, s in zip(descs, steps)]
    seen = _drain(srv, len(ids))
    assert max(seen) == 2
    infos = [srv.info(i) for i in ids]
    assert infos[0]["admit_tick"] == infos[1]["admit_tick"] == 0
    assert infos[2]["admit_tick"] == min(infos[0]["finish_tick"], infos[1]["finish_tick"])
    srv.close()
    # a request larger than the whole budget fails; the next one still runs
    big_desc = W.domain_desc(256, W.random_star(rng))
    p = kfbi.Plan(big_desc, kfbi.KFBI_MIXED_TF32, 50)
    need_big = p.device_bytes(kfbi.KFBI_HEAT)
    p.close()
    assert need_big > 2 * need[0]
    srv = kfbi.Server(max_resident=4, hbm_budget_bytes=(need_big + need[0]) // 2,
                      hbm_reserve_bytes=0, plan_threads=0, restart=50)
    big = _submit(srv, "heat", big_desc, 2, 0.0)
    small = _submit(srv, "heat", descs[0], 2, 0.0)
    _drain(srv, 2)
    assert srv.info(big)["state"] == kfbi.REQ_FAILED and srv.info(big)["status"] == 3
    assert srv.info(small)["state"] == kfbi.REQ_DONE
    srv.close()


def test_plan_device_bytes_equal_allocations():
    rng = np.random.Generator(np.random.PCG64(2))
    for M, prec, eq in [(64, kfbi.KFBI_FP64, kfbi.KFBI_HEAT), (128, kfbi.KFBI_MIXED_TF32, kfbi.KFBI_WAVE),
                        (200, kfbi.KFBI_MIXED_TF32, kfbi.KFBI_SCHRODINGER),
                        (96, kfbi.KFBI_MIXED_TF32, kfbi.KFBI_HEAT)]:
        desc = W.domain_desc(M, W.random_star(rng))
        p = kfbi.Plan(desc, prec, 30)
        want = p.device_bytes(eq)
        p.close()
        dom = kfbi.Domain(desc, prec, restart=30)
        st = kfbi.State(dom, eq)
        assert dom.device_bytes() + st.device_bytes() == want, (M, prec, eq)
        st.close()
        dom.close()


def test_shared_dst_tables_are_reused_per_grid():
    M = 352  # a grid no other test keeps alive
    base = kfbi.table_cache_bytes()
    d1 = kfbi.Domain(W.domain_desc(M, W.star()), kfbi.KFBI_MIXED_TF32)
    one = kfbi.table_cache_bytes() - base
    d2 = kfbi.Domain(W.domain_desc(M, W.flower()), kfbi.KFBI_MIXED_TF32)
    assert kfbi.table_cache_bytes() - base == one  # same grid: no new tables
    Mp = ((M - 1 + 127) // 128) * 128
    assert one >= 8 * Mp * Mp + 3 * 4 * Mp * Mp  # S (FP64) + hi, lo, FP32 copies
    d1.close()
    d2.close()
    assert kfbi.table_cache_bytes() == base


def test_server_run_on_the_wall_clock_with_plan_threads():
    mix = _mix()
    # the same requests with arrivals in milliseconds; results are batch
    # invariant, so they equal the virtual-time run of the same requests alone
    srv = kfbi.Server(max_resident=4, plan_threads=2, restart=50)
    ids = [_submit(srv, k, d, s, 0.002 * a) for k, d, s, a in mix]
    srv.run(time_limit=300.0)
    for i, (k, d, s, a) in zip(ids, mix):
        inf = srv.info(i)
        assert inf["state"] == kfbi.REQ_DONE
        assert inf["finished"] >= inf["admitted"] >= inf["arrival"] - 1e-9
        ref = kfbi.Server(max_resident=1, plan_threads=0, restart=50)
        j = _submit(ref, k, d, s, 0.0)
        _drain(ref, 1)
        assert np.array_equal(ref.result(j), srv.result(i))
        ref.close()
    srv.close()


def test_a_diverging_request_fails_alone():
    """A request whose data are not finite (injected on the host: NaN in its
    initial field) fails with KFBI_ERR_NONFINITE; the requests it shared
    ticks with complete with the same bits as alone."""
    mix = _mix()[:3]
    srv = kfbi.Server(max_resident=4, plan_threads=0, restart=50)
    ids = []
    for n, (k, d, s, a) in enumerate(mix):
        x = W.request_inputs(k, d, s)
        if n == 1:
            # at the centre node, inside every star (values outside Omega are masked)
            x["u0"] = x["u0"].copy()
            c = (d["M"] - 1) // 2
            x["u0"][c, c] = np.nan
        ids.append(_submit(srv, k, d, s, 0.0, x))
    _drain(srv, len(ids))
    bad = srv.info(ids[1])
    assert bad["state"] == kfbi.REQ_FAILED and bad["status"] == 5, bad
    for n in (0, 2):
        k, d, s, a = mix[n]
        assert srv.info(ids[n])["state"] == kfbi.REQ_DONE
        alone = kfbi.Server(max_resident=1, plan_threads=0, restart=50)
        j = _submit(alone, k, d, s, 0.0)
        _drain(alone, 1)
        assert np.array_equal(alone.result(j), srv.result(ids[n]))
        alone.close()
    srv.close()


def test_lanes_run_concurrently_with_identical_results():
    """Three size lanes driven by their own host threads (kfbi_server_run):
    every request gives the same bits as alone, and a small request
    finishes before the large one that arrived with it."""
    rng = np.random.Generator(np.random.PCG64(31))
    mix = [
        ("heat", W.domain_desc(128, W.random_star(rng)), 4, 0.000),
        ("schrodinger", W.domain_desc(256, W.random_star(rng)), 3, 0.001),
        ("wave", W.domain_desc(640, W.random_star(rng)), 3, 0.001),
        ("heat", W.domain_desc(1100, W.random_star(rng)), 3, 0.000),
        ("heat", W.domain_desc(96, W.random_star(rng)), 2, 0.002),
    ]
    srv = kfbi.Server(max_resident=8, plan_threads=2, restart=50, lanes=3)
    ids = [_submit(srv, k, d, s, a) for k, d, s, a in mix]
    srv.run(time_limit=300.0)
    infos = [srv.info(i) for i in ids]
    err = (kfbi.lib().kfbi_server_last_error(srv.h) or b"").decode()
    assert all(i["state"] == kfbi.REQ_DONE for i in infos), (
        [(i["state"], i["status"], i["steps_done"]) for i in infos], err)
    assert infos[0]["finished"] < infos[3]["finished"]
    for i, (k, d, s, a) in zip(ids, mix):
        ref = kfbi.Server(max_resident=1, plan_threads=0, restart=50)
        j = _submit(ref, k, d, s, 0.0)
        _drain(ref, 1)
        assert np.array_equal(ref.result(j), srv.result(i)), (k, d["M"])
        ref.close()
    srv.close()
