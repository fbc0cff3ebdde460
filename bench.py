#!/usr/bin/env python
"""Benchmark: KFBI wave time stepping at 1024^2 on one GB300 per rank.

Workload (one "step" = one implicit time step = the whole hot path: the
volume-source application, GMRES with one operator application per
iteration, the final interface solve and the F recurrence):
  wave equation u_tt = Delta u, theta-scheme theta = 1/4, ellipse a = 0.7,
  b = 0.4 rotated 30 deg in [-1, 1]^2, M = 1024 (1023^2 unknowns),
  N_b = M = 1024 boundary nodes, dt = 4h, GMRES(50) tol 1e-10, manufactured
  solution u = cos(sqrt(2) pi t) sin(pi x) sin(pi y) for the data.
The metric is grid-point*steps/s = M^2 * steps / seconds.

The default line also carries sub-records (bounded in time) for the
batched heat workload (256 random stars, M in {128..512}), the served
Poisson stream (a prefix of it at a load the GPU sustains, and one at the
stream's own rate), the 512^2 / 1024^2 convergence leg of the wave
workload, and the FP64 comparisons.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Multi-GPU (torchrun): every rank runs an independent replica (the method
has no exchange step); value = sum over ranks; timing = max over ranks.
"""

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = ("grid-point·steps/s at 1024² vs plain FP64 GPU at fixed L∞ error; "
          "p50/p99 latency")
UNIT = "grid-point*steps/s"


def max_over_ranks(values, world, device=None):
    """The slowest rank's times: an all-reduce (max) of a few floats over the
    default process group (the timing barrier is the only collective of the
    replica runs).  device: where the reduction tensor lives ("cuda" under
    NCCL, None for a CPU group)."""
    if world <= 1:
        return [float(v) for v in values]
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(v) for v in values], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return [float(v) for v in t.cpu()]


def replica_value(world, work_per_rank, seconds):
    """Whole-job throughput of independent replicas: all ranks' work over the
    slowest rank's time (weak scaling)."""
    return world * work_per_rank / seconds


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--M", type=int, default=1024)
    ap.add_argument("--precision", default="fft32", choices=["tf32", "fft32", "fp64"])
    ap.add_argument("--solver", default="gmres", choices=["gmres", "richardson"],
                    help="density solver: GMRES(50) or the Richardson iteration of Eq. 3.21")
    ap.add_argument("--gamma", type=float, default=0.5, help="Richardson step")
    ap.add_argument("--no-alt-path", action="store_true",
                    help="skip the second (TF32 tensor-core) measurement of the default run")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-fp64-compare", action="store_true")
    ap.add_argument("--cpu-steps", type=int, default=2)
    ap.add_argument("--workload", default="wave1024",
                    choices=["wave1024", "heat1024-neumann", "nls1024", "schr1024", "batched",
                             "served"],
                    help="wave1024: theta = 1/4 wave (headline); heat1024-neumann: the paper's "
                         "Neumann heat example at --M; nls1024: its nonlinear Schroedinger "
                         "example (w = 1) at --M; schr1024: the Strang-split Schroedinger "
                         "flower runs (norm drift, plane-wave error); batched, served: the "
                         "256-instance and Poisson-stream workloads")
    ap.add_argument("--batch", type=int, default=256)
    ap.add_argument("--batch-precision", default="fft32", choices=["tf32", "fft32"])
    ap.add_argument("--requests", type=int, default=60)
    ap.add_argument("--max-resident", type=int, default=64)
    ap.add_argument("--rate", type=float, default=200.0)
    ap.add_argument("--sustained-rate", type=float, default=3.0,
                    help="offered load (req/s) of the queue-free served run")
    ap.add_argument("--sustained-requests", type=int, default=40)
    ap.add_argument("--lanes", type=int, default=3)
    ap.add_argument("--schr-steps", type=int, default=400)
    ap.add_argument("--no-batched", action="store_true", help="skip the batched sub-record")
    ap.add_argument("--no-served", action="store_true", help="skip the served sub-record")
    ap.add_argument("--no-convergence", action="store_true",
                    help="skip the 512^2 / 1024^2 convergence leg")
    return ap.parse_args()


def workload(M):
    from paper_2404_14864_gb300 import workloads as W
    desc = W.domain_desc(M, W.ellipse(0.7, 0.4, 30.0))
    h = (desc["hi"] - desc["lo"]) / M
    return desc, 4.0 * h, 0.25


class WaveProblem:
    """The headline workload: theta = 1/4 wave on the rotated ellipse,
    u = cos(sqrt2 pi t) sin(pi x) sin(pi y), dt = 4h."""

    kind = "wave"

    def __init__(self, M):
        from paper_2404_14864_gb300 import workloads as W
        self.M = M
        self.desc, self.dt, self.theta = workload(M)
        self.ex = W.WaveExact()
        self.X, self.Y = W.grid_xy(self.desc)
        self.zx, self.zy = W.boundary_xy(self.desc)
        self.cplx = False

    def equation(self, kfbi):
        return kfbi.KFBI_WAVE

    def g(self, k):
        """Dirichlet data of step k (0-based): u at (k + 2) dt."""
        return self.ex.u(self.zx, self.zy, (k + 2) * self.dt)

    def exact(self, n):
        """u after n steps."""
        return self.ex.u(self.X, self.Y, (n + 1) * self.dt)

    def init(self, st, cu):
        ex, X, Y, dt = self.ex, self.X, self.Y, self.dt
        st.init_wave(dt, self.theta, cu(ex.u(X, Y, 0.0)), cu(ex.lap(X, Y, 0.0)),
                     cu(ex.u(X, Y, dt)), cu(ex.lap(X, Y, dt)))

    def step(self, st, g_dev):
        return st.step_wave(g_dev)

    def oracle_stepper(self, oracle, d):
        ex, X, Y, dt = self.ex, self.X, self.Y, self.dt
        st = oracle.WaveStepper(d, dt, 1e-10)
        st.init(ex.u(X, Y, 0.0), ex.lap(X, Y, 0.0), ex.u(X, Y, dt), ex.lap(X, Y, dt))
        return st

    def oracle_step(self, st, k):
        st.step(self.g(k))

    def config(self, precision, solver="gmres", gamma=0.5):
        return config(self.M, self.desc, self.dt, precision, solver, gamma)


class NlsProblem:
    """The paper's nonlinear Schroedinger example (Sec. 4, Ex. 5) at grid M:
    w = 1, v = 1 - cos^2 x cos^2 y, u = exp(i t) cos x cos y, star
    r = 1.5 (0.8 + 0.2 cos 3 theta), box [-pi, pi]^2, N_b = M, dt = 8 / M
    (the time steps of its Table 4)."""

    kind = "nls"

    def __init__(self, M):
        from paper_2404_14864_gb300 import workloads as W
        self.M = M
        self.desc = W.domain_desc(M, W.ex5_star(0.2), lo=-math.pi, hi=math.pi)
        self.dt = 8.0 / M
        self.ex = W.NonlinearSchrodingerExact()
        self.X, self.Y = W.grid_xy(self.desc)
        self.zx, self.zy = W.boundary_xy(self.desc)
        self.V = self.ex.v(self.X, self.Y)
        self.cplx = True
        self.Vd = None

    def equation(self, kfbi):
        return kfbi.KFBI_SCHRODINGER

    def g(self, k):
        return self.ex.u(self.zx, self.zy, (k + 1) * self.dt)

    def exact(self, n):
        return self.ex.u(self.X, self.Y, n * self.dt)

    def init(self, st, cu):
        if self.Vd is None:
            self.Vd = cu(self.V)
        st.init_schrodinger(self.dt, cu(self.ex.u(self.X, self.Y, 0.0)),
                            cu(self.ex.lap(self.X, self.Y, 0.0)))

    def step(self, st, g_dev):
        return st.step_schrodinger(self.Vd, g_dev, w=self.ex.w)

    def oracle_stepper(self, oracle, d):
        st = oracle.SchrodingerStepper(d, self.dt, 1e-10)
        st.init(self.ex.u(self.X, self.Y, 0.0), self.ex.lap(self.X, self.Y, 0.0))
        return st

    def oracle_step(self, st, k):
        st.step(self.g(k), self.V, self.ex.w)

    def config(self, precision, solver="gmres", gamma=0.5):
        sv = ("gmres restart 50, tol 1e-10" if solver == "gmres"
              else "richardson gamma %g, tol 1e-10" % gamma)
        return {"workload": "nonlinear-schrodinger-w1-star-%d" % self.M, "M": self.M,
                "unknowns": (self.M - 1) ** 2, "n_boundary": self.desc["nb"], "dt": "8/M",
                "w": 1.0, "solver": sv, "precision": precision,
                "l2": "flushed between timed steps (256 MiB write)",
                "box": [self.desc["lo"], self.desc["hi"]]}


class HeatNeumannProblem:
    """The paper's Neumann heat example (Sec. 4, Ex. 2) at grid M:
    u = exp(-t) sin(0.6 x + 0.8 y), u_t = Delta u, d_n u given on Gamma, on
    the star r = 1 + 0.2 sin 5 theta in [-1.5, 1.5]^2 (its heart curve is a
    spline), N_b = M, dt = 16 / M (the time steps of its Table 2)."""

    kind = "heat-neumann"
    cplx = False

    def __init__(self, M):
        from paper_2404_14864_gb300 import workloads as W
        self.M = M
        self.desc = W.domain_desc(M, W.star(1.0, 0.2, 5), lo=-1.5, hi=1.5)
        self.dt = 16.0 / M
        self.X, self.Y = W.grid_xy(self.desc)
        self.zx, self.zy = W.boundary_xy(self.desc)
        self.nx, self.ny = W.boundary_normal(self.desc)

    def equation(self, kfbi):
        return kfbi.KFBI_HEAT

    def _u(self, t):
        return math.exp(-t) * np.sin(0.6 * self.X + 0.8 * self.Y)

    def g(self, k):
        t = (k + 1) * self.dt
        c = math.exp(-t) * np.cos(0.6 * self.zx + 0.8 * self.zy)
        return c * (0.6 * self.nx + 0.8 * self.ny)

    def exact(self, n):
        return self._u(n * self.dt)

    def init(self, st, cu):
        st.set_neumann(True)
        st.init_heat(self.dt, cu(self._u(0.0)), cu(-self._u(0.0)))

    def step(self, st, g_dev):
        return st.step_heat(g_dev)

    def oracle_stepper(self, oracle, d):
        st = oracle.HeatStepper(d, self.dt, 1e-10, bc="neumann")
        st.init(self._u(0.0), -self._u(0.0))
        return st

    def oracle_step(self, st, k):
        st.step(self.g(k))

    def config(self, precision, solver="gmres", gamma=0.5):
        sv = ("gmres restart 50, tol 1e-10" if solver == "gmres"
              else "richardson gamma %g, tol 1e-10" % gamma)
        return {"workload": "heat-neumann-star-%d" % self.M, "M": self.M,
                "unknowns": (self.M - 1) ** 2, "n_boundary": self.desc["nb"], "dt": "16/M",
                "boundary": "neumann (Eq. 3.19)", "solver": sv, "precision": precision,
                "l2": "flushed between timed steps (256 MiB write)",
                "box": [self.desc["lo"], self.desc["hi"]]}


class SchrPacketProblem:
    """Run A of the Schroedinger flower workload for the oracle arm: the
    Gaussian packet in the harmonic potential with g = 0, dt = h/2."""

    kind = "schrodinger-packet"
    cplx = True

    def __init__(self, M):
        self.M = M
        self.desc, self.dt = schr_setup(M)
        self.u0, self.lap0, self.V = schr_packet(self.desc)

    def oracle_stepper(self, oracle, d):
        st = oracle.SchrodingerStepper(d, self.dt, 1e-10)
        st.init(self.u0, self.lap0)
        return st

    def oracle_step(self, st, k):
        import numpy as np
        st.step(np.zeros(self.desc["nb"], dtype=complex), self.V)

    def config(self, precision, solver="gmres", gamma=0.5):
        return {"workload": "schrodinger-strang-flower-%d" % self.M, "M": self.M,
                "n_boundary": self.desc["nb"], "dt": "h/2", "run": "A (Gaussian packet, V = |x|^2/2)",
                "precision": precision, "solver": "gmres restart 50, tol 1e-10"}


def make_problem(args):
    if args.workload == "nls1024":
        return NlsProblem(args.M)
    if args.workload == "heat1024-neumann":
        return HeatNeumannProblem(args.M)
    if args.workload == "schr1024":
        return SchrPacketProblem(args.M)
    return WaveProblem(args.M)


def config(M, desc, dt, precision, solver="gmres", gamma=0.5):
    sv = ("gmres restart 50, tol 1e-10" if solver == "gmres"
          else "richardson gamma %g, tol 1e-10" % gamma)
    return {"workload": "wave-theta0.25-ellipse-%d" % M, "M": M, "unknowns": (M - 1) ** 2,
            "n_boundary": desc["nb"], "dt": "4h", "theta": 0.25, "solver": sv,
            "precision": precision, "l2": "flushed between timed steps (256 MiB write)",
            "box": [desc["lo"], desc["hi"]]}


# ----------------------------------------------------------------------------
# clocks during the timed region
# ----------------------------------------------------------------------------


class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        time.sleep(0.05)
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            p = [x.strip() for x in ln.split(",")]
            if len(p) < 9:
                continue
            try:
                sm.append(float(p[1]))
                smax = float(p[2])
            except ValueError:
                continue
            for n, v in zip(names, p[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": smax, "samples": len(sm),
                "reasons": sorted(reasons)}


# ----------------------------------------------------------------------------
# our arm
# ----------------------------------------------------------------------------


def run_ours(args, rank, world, local_rank):
    import numpy as np
    import torch

    from paper_2404_14864_gb300 import build, kfbi, workloads as W

    build.build()
    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    M = args.M
    P = make_problem(args)
    desc, dt = P.desc, P.dt
    n1 = M - 1
    stream = torch.cuda.current_stream()

    def cu(a):
        return torch.from_numpy(np.ascontiguousarray(a)).to(dev)

    prec = {"tf32": kfbi.KFBI_MIXED_TF32, "fft32": kfbi.KFBI_MIXED_FFT32,
            "fp64": kfbi.KFBI_FP64}[args.precision]
    note = None
    sv = {"solver": kfbi.KFBI_RICHARDSON if args.solver == "richardson" else kfbi.KFBI_GMRES,
          "gamma": args.gamma}
    try:
        dom = kfbi.Domain(desc, prec, restart=50, tol=1e-10, maxit=2000, **sv)
    except kfbi.KfbiError as e:
        if prec == kfbi.KFBI_FP64 or e.status != 8:
            raise
        note = "mixed path unavailable in this build (%s); fp64 path timed" % e
        prec = kfbi.KFBI_FP64
        dom = kfbi.Domain(desc, prec, restart=50, tol=1e-10, maxit=2000, **sv)
    K, Wm = args.steps, args.warmup
    n_total = Wm + K
    # boundary data for every step, resident on the device before timing
    g_all = [cu(P.g(k)) for k in range(n_total)]

    def new_state(domain):
        st = kfbi.State(domain, P.equation(kfbi))
        P.init(st, cu)
        return st

    # inside mask for the error norm, from the library's host-side plan
    ins = kfbi.Plan(desc).field("inside").reshape(M + 1, M + 1)[1:-1, 1:-1].astype(bool)
    inside = torch.from_numpy(ins.copy()).to(dev)

    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)

    def run_steps(st, first, count, timed, lat):
        iters = []
        for k in range(first, first + count):
            if timed:
                flush.zero_()
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
            info = P.step(st, g_all[k])
            iters.append(info["iters"])
            if timed:
                e1.record(stream)
                e1.synchronize()
                lat.append(e0.elapsed_time(e1))
        return iters

    st = new_state(dom)
    run_steps(st, 0, Wm, False, [])
    torch.cuda.synchronize()
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
    torch.cuda.synchronize()
    clk = ClockSampler(local_rank if "CUDA_VISIBLE_DEVICES" not in os.environ
                       else os.environ["CUDA_VISIBLE_DEVICES"].split(",")[local_rank])
    clk.start()
    # timed region: per-step CUDA events only (an event between two kernels
    # would serialise the programmatic-dependent launches it measures)
    n_launch0 = kfbi.launch_count()
    lat = []
    t0 = time.perf_counter()
    iters = run_steps(st, Wm, K, True, lat)
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    n_launch = kfbi.launch_count() - n_launch0
    clocks = clk.stop()
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
    # second timed pass over the same steps with an event pair around every
    # launch of the dominant kernel class: its average launch duration and
    # the flops those launches issued, for the roofline
    st_r = new_state(dom)
    run_steps(st_r, 0, Wm, False, [])
    torch.cuda.synchronize()
    kfbi.kfbi_profile_reset()
    kfbi.kfbi_profile_enable([kfbi.PROF_DST])
    lat_r = []
    run_steps(st_r, Wm, K, True, lat_r)
    torch.cuda.synchronize()
    kfbi.kfbi_profile_enable(False)
    prof = {"dst": kfbi.kfbi_profile_read(kfbi.PROF_DST),
            "dst_flops": kfbi.kfbi_profile_work(kfbi.PROF_DST),
            "dst_bytes": kfbi.kfbi_profile_bytes(kfbi.PROF_DST),
            "ms_per_step_instrumented": sum(lat_r) / K}
    st_r.close()
    t_dev = sum(lat) / 1e3
    exact = torch.from_numpy(P.exact(Wm + K)).to(dev)
    u = st.get_u()
    err = float((u - exact).abs()[inside].max())
    # per-class breakdown: one extra (untimed) step with every class timed
    st_b = new_state(dom)
    kfbi.kfbi_profile_reset()
    kfbi.kfbi_profile_enable(True)
    P.step(st_b, g_all[0])
    kfbi.kfbi_profile_enable(False)
    breakdown = {kfbi.PROF_NAMES[c]: kfbi.kfbi_profile_read(c) for c in kfbi.PROF_NAMES}
    st_b.close()

    # end to end through the public API with host buffers: H2D of the step's
    # boundary data, the step, D2H of the solution grid
    st2 = new_state(dom)
    cdt = torch.complex128 if P.cplx else torch.float64
    g_host = [torch.from_numpy(P.g(k)).pin_memory() for k in range(K)]
    u_host = torch.empty(n1 * n1, dtype=cdt).pin_memory()
    g_dev = torch.empty(desc["nb"], dtype=cdt, device=dev)
    u_dev = torch.empty(n1 * n1, dtype=cdt, device=dev)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for k in range(K):
        g_dev.copy_(g_host[k], non_blocking=True)
        P.step(st2, g_dev)
        st2.get_u(u_dev)
        u_host.copy_(u_dev, non_blocking=True)
        torch.cuda.synchronize()
    t_e2e = time.perf_counter() - t0
    st2.close()

    # the plain FP64 GPU path on the same steps, for the fixed-error comparison
    fp64 = None
    if prec != kfbi.KFBI_FP64 and not args.no_fp64_compare:
        dom64 = kfbi.Domain(desc, kfbi.KFBI_FP64, restart=50, tol=1e-10, maxit=2000, **sv)
        st64 = new_state(dom64)
        run_steps(st64, 0, Wm, False, [])
        lat64 = []
        run_steps(st64, Wm, K, True, lat64)
        u64 = st64.get_u()
        err64 = float((u64 - exact).abs()[inside].max())
        diff = float((u64 - u).abs()[inside].max())
        fp64 = {"value": M * M * K / (sum(lat64) / 1e3), "unit": UNIT,
                "ms_per_step": sum(lat64) / K, "linf_vs_exact": err64,
                "linf_mixed_minus_fp64": diff}
        st64.close()
        dom64.close()

    out = {"t_dev": t_dev, "t_e2e": t_e2e, "lat": lat, "iters": iters, "err": err,
           "launches": n_launch, "prof": prof, "breakdown": breakdown, "clocks": clocks,
           "prec": prec, "note": note,
           "wall": wall, "fp64": fp64, "desc": desc, "dt": dt,
           "h2d": desc["nb"] * (16 if P.cplx else 8), "d2h": n1 * n1 * (16 if P.cplx else 8),
           "problem": P}
    st.close()
    dom.close()
    return out


# DRAM bytes per launch of the mixed DST pass at the 1024^2 wave workload
# (dram__bytes_read.sum + dram__bytes_write.sum of a dense pass, from one
# ncu --set full capture of the timed step).  Reset to None whenever
# k_tc_pass changes until it is captured again.
TC_PASS_TRAFFIC_1024 = 16.845824e6 + 0.0
# DRAM bytes per FFT32 DST launch at the 1024^2 wave workload (one real
# plane): dram__bytes_read.sum + dram__bytes_write.sum averaged over the
# captured k_dst_fft launches of the current kernel.  None whenever
# k_dst_fft changes until it is captured again.
FFT_PASS_TRAFFIC_1024 = 4.265e6


def load_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return {}


def fft_roofline(n, ms, nbytes, flops, how, traffic=None, kernel="k_dst_fft (FP32 FFT DST-I pass)"):
    """HBM roofline of the FFT DST launches: the algorithmic bytes they
    declare (each transformed row read and written once, 4 (M - 1) bytes
    each way) over their summed CUDA-event time, against the measured copy
    rate."""
    if n == 0 or ms <= 0:
        return None
    peak = load_peaks().get("hbm_gbs", 6800.0)
    gbs = nbytes / (ms / 1e3) / 1e9
    return {"bound": "hbm", "achieved": gbs, "peak": peak, "unit": "GB/s", "frac": gbs / peak,
            "traffic": traffic, "traffic_unit": "bytes per launch", "kernel": kernel,
            "peak_source": "of measured: STREAM-style copy (hbm_gbs)",
            "algorithmic_bytes_per_launch": nbytes / n, "avg_launch_us": 1e3 * ms / n,
            "launches": n, "flops_per_launch": flops / n, "timing": how}


_TF32_PEAK = None


def measure_tf32_peak():
    """Dense TF32 rate of this GPU, measured here like the bf16 figure of
    the peaks file: torch.matmul on 8192^3 FP32 operands with TF32 allowed,
    best of 5 (burst) and a back-to-back loop of about 1.5 s (sustained)."""
    global _TF32_PEAK
    if _TF32_PEAK is not None:
        return _TF32_PEAK
    import torch
    prev = torch.backends.cuda.matmul.allow_tf32
    torch.backends.cuda.matmul.allow_tf32 = True
    try:
        n = 8192
        a = torch.randn(n, n, device="cuda")
        b = torch.randn(n, n, device="cuda")
        c = torch.empty(n, n, device="cuda")
        for _ in range(2):
            torch.matmul(a, b, out=c)
        torch.cuda.synchronize()
        best = 1e9
        for _ in range(5):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record()
            torch.matmul(a, b, out=c)
            e1.record()
            e1.synchronize()
            best = min(best, e0.elapsed_time(e1))
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        t0 = time.perf_counter()
        k = 0
        e0.record()
        while time.perf_counter() - t0 < 1.5:
            for _ in range(10):
                torch.matmul(a, b, out=c)
            k += 10
            torch.cuda.synchronize()
        e1.record()
        e1.synchronize()
        flop = 2.0 * n ** 3
        _TF32_PEAK = {"burst": flop / (best / 1e3) / 1e12,
                      "sustained": flop * k / (e0.elapsed_time(e1) / 1e3) / 1e12,
                      "how": "torch.matmul FP32 8192^3 with TF32 allowed: best of 5 (burst), "
                             "back-to-back for 1.5 s (sustained), this run"}
        del a, b, c
        torch.cuda.empty_cache()
    finally:
        torch.backends.cuda.matmul.allow_tf32 = prev
    return _TF32_PEAK


def roofline(res, M):
    """Roofline of the dominant kernel class (the DST-I passes) over the
    timed launches of a second timed pass: FFT32 against HBM by algorithmic
    bytes, TF32 against the tensor rate by executed flops, FP64 against the
    nominal FP64 rate."""
    n, ms = res["prof"]["dst"]
    flops = res["prof"]["dst_flops"]
    if n == 0 or ms <= 0:
        return None
    how = ("CUDA event pair around every DST launch, on its stream, in a second timed pass "
           "of the same steps (%.3f ms/step with those events)" % res["prof"]["ms_per_step_instrumented"])
    avg_s = ms / n / 1e3
    from paper_2404_14864_gb300 import kfbi
    achieved = flops / (ms / 1e3) / 1e12
    if res["prec"] == kfbi.KFBI_FP64:
        return {"bound": "alu", "achieved": achieved, "peak": 1.25, "unit": "TFLOP/s",
                "frac": achieved / 1.25, "traffic": None,
                "kernel": "k_dgemm_t (float64 DST-I pass)",
                "peak_source": "nominal GB300 FP64 rate (1.25 TFLOP/s, profiling recipe table)",
                "avg_launch_us": avg_s * 1e6, "launches": n, "flops_per_launch": flops / n,
                "timing": how}
    if res["prec"] == kfbi.KFBI_MIXED_FFT32:
        return fft_roofline(n, ms, res["prof"]["dst_bytes"], flops, how,
                            FFT_PASS_TRAFFIC_1024 if M == 1024 else None)
    pk = measure_tf32_peak()
    peak = pk["sustained"]
    return {"bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
            "frac": achieved / peak, "traffic": TC_PASS_TRAFFIC_1024 if M == 1024 else None,
            "traffic_unit": "bytes per launch",
            "kernel": "k_tc_pass (tcgen05 TF32x3 DST-I pass)",
            "peak_source": "of measured: sustained dense TF32 rate (%s; burst %.0f)"
                           % (pk["how"], pk["burst"]),
            "avg_launch_us": avg_s * 1e6, "launches": n, "flops_per_launch": flops / n,
            "timing": how}


# ----------------------------------------------------------------------------
# batched heat workload (256 random stars of uneven size, one grouped step)
# ----------------------------------------------------------------------------


def pct(v, f):
    """The f-quantile of sorted values (nearest rank)."""
    return v[min(len(v) - 1, max(0, int(math.ceil(f * len(v))) - 1))] if v else None


def batched_record(args, K, Wm, prec_name="fft32", fp64=True):
    """The batched heat workload: 256 instances, M drawn from {128, 192, 256,
    384, 512}, random stars (PCG64 seed 0), dt = h, stepped together by
    kfbi_batch_step.  K timed steps after Wm warm-up steps (CUDA events per
    batch step, L2 flushed before each); a second timed pass with an event
    pair around every DST launch gives the roofline; the float64 path steps
    the same instances one domain at a time for the comparison."""
    import numpy as np
    import torch

    from paper_2404_14864_gb300 import kfbi, workloads as W
    dev = torch.device("cuda", torch.cuda.current_device())
    inst = W.batched_instances(args.batch, seed=0)
    ex = W.HeatExact()
    prec = {"tf32": kfbi.KFBI_MIXED_TF32, "fft32": kfbi.KFBI_MIXED_FFT32}[prec_name]

    def cu(a):
        return torch.from_numpy(np.ascontiguousarray(a)).to(dev)

    runs = []
    for M, curve in inst:
        desc = W.domain_desc(M, curve)
        h = 2.0 / M
        X, Y = W.grid_xy(desc)
        zx, zy = W.boundary_xy(desc)
        ins = kfbi.Plan(desc).field("inside").reshape(M + 1, M + 1)[1:-1, 1:-1].astype(bool)
        runs.append((M, h, X, Y, zx, zy, desc, ins))
    nsteps = Wm + K
    g = [[cu(ex.u(r[4], r[5], (k + 1) * r[1])) for r in runs] for k in range(nsteps)]
    src = [[cu(ex.src(r[2], r[3], (k + 1) * r[1]) + ex.src(r[2], r[3], (k + 2) * r[1])) for r in runs]
           for k in range(nsteps)]

    def make(p):
        doms, states = [], []
        for (M, h, X, Y, zx, zy, desc, ins) in runs:
            d = kfbi.Domain(desc, p if kfbi.fft_supported(M) or p != kfbi.KFBI_MIXED_FFT32
                            else kfbi.KFBI_MIXED_TF32, restart=50, tol=1e-10, maxit=2000)
            st = kfbi.State(d, kfbi.KFBI_HEAT)
            st.init_heat(h, cu(ex.u(X, Y, 0)), cu(ex.lap(X, Y, 0)), cu(ex.src(X, Y, 0) + ex.src(X, Y, h)))
            doms.append(d)
            states.append(st)
        return doms, states

    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    doms, states = make(prec)
    batch = kfbi.Batch(doms)
    for k in range(Wm):
        batch.step(states, g[k], src[k])
    torch.cuda.synchronize()
    lat, iters = [], []
    n0 = kfbi.launch_count()
    clk = ClockSampler(os.environ.get("CUDA_VISIBLE_DEVICES", "0").split(",")[0])
    clk.start()
    for k in range(Wm, nsteps):
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        infos = batch.step(states, g[k], src[k])
        e1.record()
        e1.synchronize()
        lat.append(e0.elapsed_time(e1))
        iters.append(max(i["iters"] for i in infos))
    launches = kfbi.launch_count() - n0
    clocks = clk.stop()
    t = sum(lat) / 1e3
    pts = sum(r[0] * r[0] for r in runs)
    errs = []
    for r, st in zip(runs, states):
        u = st.get_u().cpu().numpy()
        errs.append(float(np.abs(u - ex.u(r[2], r[3], nsteps * r[1]))[r[7]].max()))
    tuning = batch.tuning()
    batch.close()
    for d in doms:
        d.close()
    # second pass: event pairs around every DST launch (roofline)
    doms, states = make(prec)
    batch = kfbi.Batch(doms)
    for k in range(Wm):
        batch.step(states, g[k], src[k])
    torch.cuda.synchronize()
    kfbi.kfbi_profile_reset()
    kfbi.kfbi_profile_enable([kfbi.PROF_DST])
    for k in range(Wm, nsteps):
        flush.zero_()
        batch.step(states, g[k], src[k])
    torch.cuda.synchronize()
    kfbi.kfbi_profile_enable(False)
    n, ms = kfbi.kfbi_profile_read(kfbi.PROF_DST)
    how = ("CUDA event pair around every DST launch on its stream, second timed pass of the "
           "same batch steps")
    if prec == kfbi.KFBI_MIXED_FFT32:
        roof = fft_roofline(n, ms, kfbi.kfbi_profile_bytes(kfbi.PROF_DST),
                            kfbi.kfbi_profile_work(kfbi.PROF_DST), how,
                            kernel="k_dst_fft (FP32 FFT DST-I passes, grouped per grid size)")
    else:
        pk = measure_tf32_peak()
        fl = kfbi.kfbi_profile_work(kfbi.PROF_DST)
        ach = fl / (ms / 1e3) / 1e12 if ms > 0 else 0.0
        roof = {"bound": "tensor", "achieved": ach, "peak": pk["sustained"], "unit": "TFLOP/s",
                "frac": ach / pk["sustained"], "traffic": None,
                "kernel": "k_tc_pass (tcgen05 TF32x3, grouped over instances)",
                "peak_source": "of measured: sustained dense TF32 rate (%s)" % pk["how"],
                "avg_launch_us": 1e3 * ms / max(1, n), "launches": n, "timing": how}
    kfbi.kfbi_profile_reset()
    batch.close()
    for d in doms:
        d.close()
    lat_s = sorted(lat)
    rec = {"value": pts * K / t, "unit": UNIT, "ms_per_step": 1e3 * t / K, "steps": K, "warmup": Wm,
           "precision": {"fft32": "mixed-fp32-fft", "tf32": "mixed-tf32x3"}[prec_name],
           "instances": len(runs), "sizes": sorted(set(r[0] for r in runs)),
           "grid_points_per_step": pts,
           "latency_ms_per_batch_step": {"p50": pct(lat_s, 0.5), "p99": pct(lat_s, 0.99),
                                         "max": lat_s[-1]},
           "linf_vs_exact_max": max(errs), "gmres_iters_max_per_step": iters,
           "gpu_launches": launches, "tuning": tuning, "roofline": roof, "clocks": clocks,
           "workload": "batched-heat-%d (M in {128,192,256,384,512}, random stars, PCG64 seed 0, "
                       "dt = h)" % len(runs),
           "l2": "flushed before each timed batch step (256 MiB write)"}
    if fp64:
        # the plain float64 path on the same instances and steps, one domain
        # at a time (batches take mixed domains)
        t64, e64 = 0.0, []
        for i, r in enumerate(runs):
            M, h, X, Y, zx, zy, desc, ins = r
            d = kfbi.Domain(desc, kfbi.KFBI_FP64, restart=50, tol=1e-10, maxit=2000)
            st = kfbi.State(d, kfbi.KFBI_HEAT)
            st.init_heat(h, cu(ex.u(X, Y, 0)), cu(ex.lap(X, Y, 0)), cu(ex.src(X, Y, 0) + ex.src(X, Y, h)))
            for k in range(nsteps):
                if k >= Wm:
                    e0 = torch.cuda.Event(enable_timing=True)
                    e1 = torch.cuda.Event(enable_timing=True)
                    e0.record()
                st.step_heat(g[k][i], src[k][i])
                if k >= Wm:
                    e1.record()
                    e1.synchronize()
                    t64 += e0.elapsed_time(e1) / 1e3
            u = st.get_u().cpu().numpy()
            e64.append(float(np.abs(u - ex.u(X, Y, nsteps * h))[ins].max()))
            st.close()
            d.close()
        rec["fp64_gpu"] = {"value": pts * K / t64, "unit": UNIT, "ms_per_batch_step": 1e3 * t64 / K,
                           "linf_vs_exact_max": max(e64),
                           "how": "each instance stepped alone on a KFBI_FP64 domain (dense FP64 "
                                  "DST-I passes), the same steps; time summed over instances"}
        rec["speedup_vs_fp64_gpu"] = rec["value"] / rec["fp64_gpu"]["value"]
    return rec


def run_batched(args):
    import torch

    from paper_2404_14864_gb300 import build
    build.build()
    torch.cuda.set_device(0)
    rec = batched_record(args, args.steps, args.warmup, args.batch_precision, not args.no_fp64_compare)
    line = {"metric": "grid-point*steps/s, batched heat (aggregate over instances)",
            "value": rec["value"], "unit": UNIT, "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": rec["ms_per_step"], "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None,
            "dtype": {"fft32": "fp32-fft+f64", "tf32": "tf32x3-f32acc+f64"}[args.batch_precision],
            "data": "synthetic (manufactured solution)",
            "config": {"workload": "batched-heat-%d" % rec["instances"], "sizes": rec["sizes"],
                       "instances": rec["instances"], "seed": 0, "dt": "h",
                       "precision": rec["precision"], "l2": rec["l2"]},
            "latency_ms": rec["latency_ms_per_batch_step"],
            "linf_vs_exact_max": rec["linf_vs_exact_max"], "roofline": rec["roofline"],
            "gpu_launches": rec["gpu_launches"], "tuning": rec["tuning"], "clocks": rec["clocks"],
            "fp64_gpu": rec.get("fp64_gpu"),
            "gmres_iters_max_per_step": rec["gmres_iters_max_per_step"]}
    print(json.dumps(line))
    return 0


# ----------------------------------------------------------------------------
# served stream (Poisson arrivals, continuous batching, admission by HBM)
# ----------------------------------------------------------------------------


def served_record(args, n, rate, prec_name="fft32", profile=False):
    """Serve the first n requests of the Poisson request stream (kinds 1:1:1,
    M in {128, 256, 512, 1024, 2048}, 20..200 steps, random stars, PCG64
    seed 0) with arrival times scaled to the offered rate, on the wall
    clock.  Latency = finish - arrival per request; service = finish -
    admission; throughput = grid-point*steps of all requests / wall time."""
    import numpy as np
    import torch

    from paper_2404_14864_gb300 import kfbi, workloads as W
    reqs = W.served_requests(n, rate=rate, seed=0)
    t_prep = time.perf_counter()
    inputs = [W.request_inputs(kind, W.domain_desc(M, curve), steps)
              for (_, kind, M, curve, steps) in reqs]
    t_prep = time.perf_counter() - t_prep
    prec = {"tf32": kfbi.KFBI_MIXED_TF32, "fft32": kfbi.KFBI_MIXED_FFT32}[prec_name]
    srv = kfbi.Server(max_resident=args.max_resident, hbm_reserve_bytes=8 << 30, restart=50,
                      plan_threads=8, lanes=args.lanes)
    ids = []
    for (arr, kind, M, curve, steps), x in zip(reqs, inputs):
        desc = W.domain_desc(M, curve)
        p = prec if (prec != kfbi.KFBI_MIXED_FFT32 or kfbi.fft_supported(M)) else kfbi.KFBI_MIXED_TF32
        ids.append(srv.submit(desc, x["equation"], steps, x["dt"], arr, x["u0"], x["lap_u0"], x["g"],
                              theta=x.get("theta", 0.25), u1=x.get("u1"), lap_u1=x.get("lap_u1"),
                              src_init=x.get("src_init"), src_profile=x.get("src_profile"),
                              src_coef=x.get("src_coef"), potential=x.get("potential"),
                              tol=1e-10, maxit=2000, precision=p))
    torch.cuda.synchronize()
    clk = ClockSampler(os.environ.get("CUDA_VISIBLE_DEVICES", "0").split(",")[0])
    clk.start()
    if profile:
        kfbi.kfbi_profile_reset()
        kfbi.kfbi_profile_enable([kfbi.PROF_DST])
    n0 = kfbi.launch_count()
    t0 = time.perf_counter()
    srv.run(time_limit=3600.0)
    wall = time.perf_counter() - t0
    launches = kfbi.launch_count() - n0
    roof = None
    if profile:
        kfbi.kfbi_profile_enable(False)
        nl, ms = kfbi.kfbi_profile_read(kfbi.PROF_DST)
        roof = fft_roofline(nl, ms, kfbi.kfbi_profile_bytes(kfbi.PROF_DST),
                            kfbi.kfbi_profile_work(kfbi.PROF_DST),
                            "CUDA event pair around every DST launch on its lane's stream "
                            "(a separate profiled run of the same requests)",
                            kernel="k_dst_fft (FP32 FFT DST-I passes, grouped per grid size)")
        kfbi.kfbi_profile_reset()
    clocks = clk.stop()
    st = srv.stats()
    infos = [srv.info(i) for i in ids]
    done = [i for i in infos if i["state"] == kfbi.REQ_DONE]
    lat = sorted(i["finished"] - i["arrival"] for i in done)
    svc = sorted(i["finished"] - i["admitted"] for i in done)
    wait = sorted(i["admitted"] - i["arrival"] for i in infos if i["admitted"] >= 0)
    errs = {"heat": 0.0, "wave": 0.0, "schrodinger": 0.0}
    for (arr, kind, M, curve, steps), x, i in zip(reqs, inputs, ids):
        u = srv.result(i)
        if u is None:
            continue
        pl = kfbi.Plan(W.domain_desc(M, curve))
        ins = pl.field("inside").reshape(M + 1, M + 1)[1:-1, 1:-1].astype(bool)
        pl.close()
        errs[kind] = max(errs[kind], float(np.abs(u - x["exact"]())[ins].max()))
    srv.close()
    rec = {"value": st["grid_point_steps"] / wall, "unit": UNIT, "requests": n,
           "offered_rate_per_s": rate, "completed": st["completed"], "failed": st["failed"],
           "latency_s": {"p50": pct(lat, 0.5), "p99": pct(lat, 0.99), "max": lat[-1] if lat else None},
           "service_s": {"p50": pct(svc, 0.5), "p99": pct(svc, 0.99)},
           "queue_wait_s": {"p50": pct(wait, 0.5), "p99": pct(wait, 0.99)},
           "ticks": st["ticks"], "mean_resident": st["resident_ticks"] / max(1, st["ticks"]),
           "wall_s": wall, "grid_point_steps": st["grid_point_steps"],
           "peak_device_gib": st["peak_device_bytes"] / 2 ** 30, "linf_vs_exact_max": errs,
           "gpu_launches": launches, "clocks": clocks, "host_input_prep_s": t_prep,
           "h2d_bytes": st["h2d_bytes"], "d2h_bytes": st["d2h_bytes"]}
    if roof:
        rec["roofline"] = roof
    return rec, reqs


def fp64_served_estimate(reqs):
    """Throughput the plain float64 path would give the same requests, one
    at a time: per (kind, M) the time of one float64 step (median of 3 after
    a warm-up, CUDA events), times each request's steps."""
    import numpy as np
    import torch

    from paper_2404_14864_gb300 import kfbi, workloads as W
    per = {}
    for kind, M in sorted(set((r[1], r[2]) for r in reqs)):
        desc = W.domain_desc(M, W.star())
        x = W.request_inputs(kind, desc, 4)
        cu = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
        d = kfbi.Domain(desc, kfbi.KFBI_FP64, restart=50, tol=1e-10, maxit=2000)
        st = kfbi.State(d, x["equation"])
        if kind == "heat":
            st.init_heat(x["dt"], cu(x["u0"]), cu(x["lap_u0"]), cu(x["src_init"]))
            step = lambda n: st.step_heat(cu(x["g"][n]), cu(x["src_coef"][n] * x["src_profile"]))
        elif kind == "wave":
            st.init_wave(x["dt"], x["theta"], cu(x["u0"]), cu(x["lap_u0"]), cu(x["u1"]), cu(x["lap_u1"]))
            step = lambda n: st.step_wave(cu(x["g"][n]))
        else:
            st.init_schrodinger(x["dt"], cu(x["u0"]), cu(x["lap_u0"]))
            v = cu(x["potential"])
            step = lambda n: st.step_schrodinger(v, cu(x["g"][n]))
        step(0)
        ts = []
        for n in range(1, 4):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record()
            step(n)
            e1.record()
            e1.synchronize()
            ts.append(e0.elapsed_time(e1) / 1e3)
        per[(kind, M)] = sorted(ts)[1]
        st.close()
        d.close()
    pts = sum(r[2] * r[2] * r[4] for r in reqs)
    t = sum(per[(r[1], r[2])] * r[4] for r in reqs)
    return {"value": pts / t, "unit": UNIT,
            "seconds_per_step": {"%s-%d" % k: v for k, v in per.items()},
            "how": "float64 step time measured per (kind, M) on a star of that size (median of "
                   "3 after a warm-up), summed over the requests' steps: the same requests "
                   "served one at a time on KFBI_FP64 domains"}


def served_sub_record(args):
    """Two runs of the stream's prefix: at an offered load the GPU sustains
    (queue-free latency) and at the stream's own rate (saturated
    throughput), then a profiled run for the roofline and the float64
    estimate."""
    sus, _ = served_record(args, args.sustained_requests, args.sustained_rate, "fft32")
    sat, reqs = served_record(args, args.requests, args.rate, "fft32")
    prof, _ = served_record(args, min(args.requests, 20), args.rate, "fft32", profile=True)
    f64 = fp64_served_estimate(reqs)
    return {"precision": "mixed-fp32-fft (all sizes of the stream have an FFT pass)",
            "stream": "Poisson arrivals, kinds heat:wave:schrodinger 1:1:1, M in {128, 256, 512, "
                      "1024, 2048}, 20..200 steps, random stars, PCG64 seed 0; prefixes of %d and "
                      "%d requests (the full 1000-request stream takes minutes)"
                      % (args.sustained_requests, args.requests),
            "sustained": sus, "saturated": sat, "roofline": prof.get("roofline"),
            "fp64_gpu_estimate": f64, "speedup_vs_fp64_gpu": sat["value"] / f64["value"]}


def run_served(args):
    import torch

    from paper_2404_14864_gb300 import build
    build.build()
    torch.cuda.init()
    rec = served_sub_record(args)
    sat = rec["saturated"]
    line = {"metric": "grid-point*steps/s, served stream (Poisson arrivals, continuous batching)",
            "value": sat["value"], "unit": UNIT, "n_gpus": 1, "steps": sat["ticks"], "warmup": 0,
            "ms_per_step": 1e3 * sat["wall_s"] / max(1, sat["ticks"]), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "fp32-fft+f64",
            "data": "synthetic (manufactured solutions)",
            "config": {"workload": "served-%d-requests" % args.requests, "rate_per_s": args.rate,
                       "sustained_rate_per_s": args.sustained_rate,
                       "sizes": [128, 256, 512, 1024, 2048], "steps": [20, 200],
                       "kinds": "heat:wave:schrodinger 1:1:1", "seed": 0,
                       "max_resident": args.max_resident, "lanes": args.lanes,
                       "admission": "FIFO per size lane, exact device bytes, 8 GiB of free HBM kept",
                       "gmres": "restart 50, tol 1e-10"},
            "latency_s": sat["latency_s"], "served": rec, "gpu_launches": sat["gpu_launches"],
            "clocks": sat["clocks"], "roofline": rec["roofline"],
            "e2e": {"value": sat["value"], "unit": UNIT,
                    "h2d_bytes_per_step": sat["h2d_bytes"] / max(1, sat["ticks"]),
                    "d2h_bytes_per_step": sat["d2h_bytes"] / max(1, sat["ticks"])}}
    print(json.dumps(line))
    return 0


# ----------------------------------------------------------------------------
# convergence leg of the wave workload (512^2 and 1024^2 at T = 0.5)
# ----------------------------------------------------------------------------


def convergence_record():
    """L-infinity error of the wave workload at T = 0.5 (dt = 4h: 16, 32 and
    64 steps at 256^2, 512^2 and 1024^2) on the FFT32 path and the ratios of
    successive errors (4 for second order)."""
    import numpy as np
    import torch

    from paper_2404_14864_gb300 import kfbi
    out = {}
    for M in (256, 512, 1024):
        P = WaveProblem(M)
        cu = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
        d = kfbi.Domain(P.desc, kfbi.KFBI_MIXED_FFT32, restart=50, tol=1e-10, maxit=2000)
        st = kfbi.State(d, kfbi.KFBI_WAVE)
        P.init(st, cu)
        nsteps = int(round(0.5 / P.dt)) - 1   # from level 1 (t = dt) to t = 0.5
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        for k in range(nsteps):
            P.step(st, cu(P.g(k)))
        e1.record()
        e1.synchronize()
        ins = kfbi.Plan(P.desc).field("inside").reshape(M + 1, M + 1)[1:-1, 1:-1].astype(bool)
        err = float(np.abs(st.get_u().cpu().numpy() - P.exact(nsteps))[ins].max())
        out[str(M)] = {"linf_vs_exact": err, "steps": nsteps, "T": (nsteps + 1) * P.dt,
                       "ms_per_step": e0.elapsed_time(e1) / nsteps}
        st.close()
        d.close()
    out["ratio_256_over_512"] = out["256"]["linf_vs_exact"] / out["512"]["linf_vs_exact"]
    out["ratio_512_over_1024"] = out["512"]["linf_vs_exact"] / out["1024"]["linf_vs_exact"]
    out["workload"] = "wave theta = 1/4, ellipse, dt = 4h, T = 0.5, FFT32 path"
    return out


# ----------------------------------------------------------------------------
# Schroedinger flower runs (Strang splitting, complex kappa = 2i / dt)
# ----------------------------------------------------------------------------


def schr_setup(M):
    """Flower r = 0.6 + 0.15 cos 4 theta in [-1, 1]^2, N_b = M, dt = h / 2."""
    from paper_2404_14864_gb300 import workloads as W
    desc = W.domain_desc(M, W.flower(0.6, 0.15, 4))
    h = (desc["hi"] - desc["lo"]) / M
    return desc, 0.5 * h


def schr_packet(desc):
    """Gaussian packet at (0.1, 0), width 0.1, momentum (5, 0), scaled to
    unit discrete L2 norm h^2 sum |u|^2 = 1, and its Laplacian."""
    import numpy as np
    from paper_2404_14864_gb300 import workloads as W
    X, Y = W.grid_xy(desc)
    h = (desc["hi"] - desc["lo"]) / desc["M"]
    gp = W.GaussianPacket(0.1, 0.0, 0.1, 5.0, 0.0, 1.0)
    amp = 1.0 / math.sqrt(h * h * float(np.sum(np.abs(gp.u(X, Y)) ** 2)))
    gp = W.GaussianPacket(0.1, 0.0, 0.1, 5.0, 0.0, amp)
    return gp.u(X, Y), gp.lap(X, Y), W.harmonic_potential(X, Y)


def run_schr1024(args):
    """Config-3 runs at grid M (default 1024): (A) the Gaussian packet in the
    harmonic potential with g = 0 for --schr-steps steps, timed, with the
    discrete L2 norm over Omega sampled every 50 steps (its drift); (B) the
    plane wave u = exp(i (5 x + 25 t)) with V = 0 for the same steps, L-inf
    error against it; the float64 (complex128) path runs a bounded prefix of
    (B) for the fixed-error comparison."""
    import numpy as np
    import torch

    from paper_2404_14864_gb300 import build, kfbi, workloads as W
    build.build()
    torch.cuda.set_device(0)
    M = args.M
    desc, dt = schr_setup(M)
    h = 2.0 * dt
    n1 = M - 1
    X, Y = W.grid_xy(desc)
    zx, zy = W.boundary_xy(desc)
    cu = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    ins = kfbi.Plan(desc).field("inside").reshape(M + 1, M + 1)[1:-1, 1:-1].astype(bool)
    ins_d = torch.from_numpy(ins.copy()).cuda()
    steps = args.schr_steps
    Wm = args.warmup
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    # (A) norm drift
    u0, lap0, V = schr_packet(desc)
    Vd = cu(V)
    g0 = torch.zeros(desc["nb"], dtype=torch.complex128, device="cuda")
    dom = kfbi.Domain(desc, kfbi.KFBI_MIXED_FFT32, restart=50, tol=1e-10, maxit=2000)

    def norm(st):
        u = st.get_u()
        return math.sqrt(h * h * float((u.abs() ** 2)[ins_d].sum()))

    st = kfbi.State(dom, kfbi.KFBI_SCHRODINGER)
    st.init_schrodinger(dt, cu(u0), cu(lap0))
    nrm0 = norm(st)
    norms = [(0, nrm0)]
    lat, iters = [], []
    clk = ClockSampler(os.environ.get("CUDA_VISIBLE_DEVICES", "0").split(",")[0])
    clk.start()
    n0 = kfbi.launch_count()
    for k in range(steps):
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        info = st.step_schrodinger(Vd, g0)
        e1.record()
        e1.synchronize()
        lat.append(e0.elapsed_time(e1))
        iters.append(info["iters"])
        if (k + 1) % 50 == 0 or k + 1 == steps:
            norms.append((k + 1, norm(st)))
    launches = kfbi.launch_count() - n0
    clocks = clk.stop()
    st.close()
    drift = max(abs(v / nrm0 - 1.0) for _, v in norms)
    # (B) plane wave: error after the same steps; e2e through the public API
    ex = W.PlaneWaveExact(5.0, 0.0)
    zero = cu(np.zeros_like(X))

    def run_b(prec, nsteps, e2e=False):
        d = kfbi.Domain(desc, prec, restart=50, tol=1e-10, maxit=2000)
        sb = kfbi.State(d, kfbi.KFBI_SCHRODINGER)
        sb.init_schrodinger(dt, cu(ex.u(X, Y, 0.0)), cu(ex.lap(X, Y, 0.0)))
        g_host = [torch.from_numpy(ex.u(zx, zy, (k + 1) * dt)).pin_memory() for k in range(nsteps)]
        u_host = torch.empty(n1 * n1, dtype=torch.complex128).pin_memory()
        g_dev = torch.empty(desc["nb"], dtype=torch.complex128, device="cuda")
        u_dev = torch.empty(n1 * n1, dtype=torch.complex128, device="cuda")
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        tdev = 0.0
        for k in range(nsteps):
            g_dev.copy_(g_host[k], non_blocking=True)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record()
            sb.step_schrodinger(zero, g_dev)
            e1.record()
            if e2e:
                sb.get_u(u_dev)
                u_host.copy_(u_dev, non_blocking=True)
            torch.cuda.synchronize()
            tdev += e0.elapsed_time(e1) / 1e3
        twall = time.perf_counter() - t0
        u = sb.get_u().cpu().numpy()
        err = float(np.abs(u - ex.u(X, Y, nsteps * dt))[ins].max())
        sb.close()
        d.close()
        return err, tdev, twall
    err_b, tdev_b, twall_b = run_b(kfbi.KFBI_MIXED_FFT32, steps, e2e=True)
    pre = min(steps, 12)
    err_b_pre, _, _ = run_b(kfbi.KFBI_MIXED_FFT32, pre)
    err64_pre, t64_pre, _ = run_b(kfbi.KFBI_FP64, pre)
    dom.close()
    t = sum(lat) / 1e3
    lat_s = sorted(lat)
    line = {"metric": METRIC, "value": M * M * steps / t, "unit": UNIT, "n_gpus": 1, "steps": steps,
            "warmup": 0, "ms_per_step": 1e3 * t / steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "fp32-fft+f64 (complex)",
            "data": "synthetic (Gaussian packet; manufactured plane wave)",
            "config": {"workload": "schrodinger-strang-flower-%d" % M, "M": M, "n_boundary": desc["nb"],
                       "dt": "h/2", "steps": steps, "curve": "r = 0.6 + 0.15 cos 4 theta",
                       "run_A": "Gaussian packet at (0.1, 0), width 0.1, momentum (5, 0), V = |x|^2/2, "
                                "w = 0, g = 0 (timed)",
                       "run_B": "plane wave exp(i (5 x + 25 t)), V = 0",
                       "precision": "mixed-fp32-fft (complex64 planes) vs complex128 FP64 path",
                       "l2": "flushed between timed steps (256 MiB write)"},
            "latency_ms": {"p50": pct(lat_s, 0.5), "p99": pct(lat_s, 0.99), "max": lat_s[-1]},
            "l2_norm": {"initial": nrm0, "samples": norms, "max_relative_drift": drift},
            "linf_vs_exact_plane_wave": err_b,
            "gmres_iters_per_step_max": max(iters), "gpu_launches": launches, "clocks": clocks,
            "e2e": {"value": M * M * steps / twall_b, "unit": UNIT,
                    "h2d_bytes_per_step": desc["nb"] * 16, "d2h_bytes_per_step": n1 * n1 * 16,
                    "how": "run B through the public API with the boundary data copied from pinned "
                           "host memory and the field read back every step"},
            "fp64_gpu": {"value": M * M * pre / t64_pre, "unit": UNIT, "steps": pre,
                         "ms_per_step": 1e3 * t64_pre / pre, "linf_vs_exact_plane_wave": err64_pre,
                         "mixed_linf_same_steps": err_b_pre,
                         "how": "plane-wave run B on a KFBI_FP64 domain (complex128), first %d steps"
                                % pre}}
    print(json.dumps(line))
    return 0


# ----------------------------------------------------------------------------
# oracle (CPU baseline / reference arm)
# ----------------------------------------------------------------------------


def run_oracle(P, steps, budget_s=150.0):
    """The oracle stepping the problem's first `steps` time steps (stops
    after the step that crosses budget_s); returns (steps done, seconds)."""
    import oracle
    d = oracle.make_domain(P.desc)
    st = P.oracle_stepper(oracle, d)
    done = 0
    t0 = time.perf_counter()
    for k in range(steps):
        P.oracle_step(st, k)
        done += 1
        if time.perf_counter() - t0 > budget_s:
            break
    t = time.perf_counter() - t0
    return done, t


def main():
    args = parse()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    M = args.M
    P = make_problem(args)

    if args.impl == "reference":
        if rank != 0:
            return 0
        k = max(1, min(args.steps, 50))
        run_oracle(P, 1, 1e9)  # one untimed warm-up step
        done, t = run_oracle(P, k)
        v = M * M * done / t
        cores = os.cpu_count()
        line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT,
                "n_gpus": args.gpus, "steps": done, "warmup": 1, "ms_per_step": 1e3 * t / done,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
                "data": "synthetic (manufactured solution)",
                "config": P.config("fp64 CPU oracle", args.solver, args.gamma),
                "cpu_baseline": {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle",
                                 "sample": "%d time steps of the %d^2 %s workload after one "
                                           "untimed step (numpy float64 oracle)"
                                           % (done, M, P.kind)},
                "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0,
                        "d2h_bytes_per_step": 0}}
        print(json.dumps(line))
        return 0

    if args.workload == "batched":
        return run_batched(args)
    if args.workload == "served":
        return run_served(args)
    if args.workload == "schr1024":
        return run_schr1024(args)

    if world > 1:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(local_rank)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local_rank))

    res = run_ours(args, rank, world, local_rank)
    alt = None
    if world == 1 and args.precision == "fft32" and not args.no_alt_path:
        # the same workload with the TF32 tensor-core DST passes
        import copy
        a2 = copy.copy(args)
        a2.precision, a2.no_fp64_compare = "tf32", True
        r2 = run_ours(a2, rank, world, local_rank)
        alt = {"value": M * M * args.steps / r2["t_dev"], "unit": UNIT,
               "ms_per_step": 1e3 * r2["t_dev"] / args.steps, "linf_vs_exact": r2["err"],
               "roofline": roofline(r2, M),
               "e2e": {"value": M * M * args.steps / r2["t_e2e"], "unit": UNIT}}
    K = args.steps
    t_dev, t_e2e = max_over_ranks([res["t_dev"], res["t_e2e"]], world, "cuda")

    # sub-records of the default line (one GPU): the 512^2 / 1024^2
    # convergence leg, the batched workload and the served stream
    subs = {}
    if world == 1 and args.workload == "wave1024" and args.precision == "fft32":
        if not args.no_convergence:
            subs["convergence"] = convergence_record()
        if not args.no_batched:
            subs["batched"] = batched_record(args, min(args.steps, 10), min(args.warmup, 3), "fft32",
                                             not args.no_fp64_compare)
        if not args.no_served:
            subs["served"] = served_sub_record(args)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        done, t = run_oracle(res["problem"], args.cpu_steps)
        cpu = {"value": M * M * done / t, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
               "sample": "%d time steps of the %d^2 %s workload (numpy float64 oracle, "
                         "BLAS threads = host cores)" % (done, M, res["problem"].kind)}

    if rank == 0:
        from paper_2404_14864_gb300 import kfbi
        lat = sorted(res["lat"])
        p = lambda q: lat[min(len(lat) - 1, int(math.ceil(q * len(lat))) - 1)]
        line = {
            "metric": METRIC, "value": replica_value(world, M * M * K, t_dev), "unit": UNIT,
            "n_gpus": world,
            "steps": K, "warmup": args.warmup, "ms_per_step": 1e3 * t_dev / K,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": {kfbi.KFBI_FP64: "f64", kfbi.KFBI_MIXED_TF32: "tf32x3-f32acc+f64",
                      kfbi.KFBI_MIXED_FFT32: "fp32-fft+f64"}[res["prec"]],
            "data": "synthetic (manufactured solution)",
            "config": res["problem"].config({kfbi.KFBI_FP64: "fp64",
                                             kfbi.KFBI_MIXED_TF32: "mixed-tf32x3",
                                             kfbi.KFBI_MIXED_FFT32: "mixed-fp32-fft"}[res["prec"]],
                                            args.solver, args.gamma),
            "latency_ms": {"p50": p(0.5), "p99": p(0.99), "max": lat[-1]},
            "linf_vs_exact": res["err"],
            "%s_iters_per_step" % args.solver: res["iters"],
            "roofline": roofline(res, M),
            "kernel_time_ms_one_step": {k: {"launches": v[0], "ms": v[1]}
                                        for k, v in res["breakdown"].items()},
            "kernel_time_note": ("one extra untimed step with a CUDA event pair around every "
                                 "launch: the events serialise the programmatic dependent "
                                 "launches, so the classes add up to more than ms_per_step; "
                                 "read them as shares"),
            "gpu_launches": res["launches"],
            "clocks": res["clocks"],
            "e2e": {"value": replica_value(world, M * M * K, t_e2e), "unit": UNIT,
                    "h2d_bytes_per_step": res["h2d"], "d2h_bytes_per_step": res["d2h"]},
            "cpu_baseline": cpu,
            "fp64_gpu": res["fp64"],
            "wall_s_timed": res["wall"],
        }
        if alt:
            line["tf32_tensor_path"] = alt
        if res["fp64"]:
            # like for like: the TF32 path keeps the dense DST-I product of the
            # float64 path; the FFT32 path also changes the algorithm from an
            # O(M^3) product to an O(M^2 log M) transform
            r = {"fft32_over_fp64_dense": line["value"] / res["fp64"]["value"],
                 "note": "FFT32 vs FP64 compares an O(M^2 log M) FP32 FFT with the O(M^3) "
                         "dense FP64 product (algorithm and precision); TF32 vs FP64 is dense vs "
                         "dense (precision only)"}
            if alt:
                r["tf32_dense_over_fp64_dense"] = alt["value"] / res["fp64"]["value"]
            line["speedup_vs_fp64_gpu"] = r
        line.update(subs)
        if res["note"]:
            line["note"] = res["note"]
        print(json.dumps(line))
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
