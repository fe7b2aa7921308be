#!/usr/bin/env python
"""Benchmark of the ES adaptive moving-mesh 2D RHD scheme on GB300.

Workload (default): the 2D RHD four-quadrant Riemann problem on [-1,1]^2 with
400 x 400 nodes, outflow boundaries, Gamma = 5/3, seeded states (rho in
[0.1,1], |v| <= 0.9, p in [0.01,1]), adaptive moving mesh (sigma = ln rho,
alpha = 1200, 4 filter passes, 10 Jacobi sweeps), 4th-order EC flux (p = 2)
with WENO5 dissipation, SSP-RK3 at CFL 0.4.  A step is one full time step
(CFL reduction with the eq. cfl solve, mesh redistribution and three RK
stages), timed as one esmm_advance call that replays the step's CUDA graph
captured in the warm-up.

Metric: cell-updates/s per RK stage = nodes * 3 * steps / device time.  Every
timed step starts with the L2 cache flushed (a 256 MB write outside the timed
events).  Under torchrun the ranks share one problem: N such 400 x 400
problems stacked into one 400 x 400N grid, slab-decomposed along x_2 (one
400-row slab per rank, weak scaling), with the step's reductions and halo
exchanges between the ranks.

``--impl reference`` times the FP64 CPU oracle (the paper's method restated
plainly in C) on the host cores over a bounded sample of the same workload.

``--workload batched`` times the 256-problem batch alone (mixed form).

``--workload rotor`` (2D RMHD rotor, 512^2, Gamma = 4/3, alpha = 800) and
``--workload blast3d`` (3D RMHD blast, 128^3, CFL 0.3) time the RMHD paths in
FP64 on the same metric; ``--workload sphere3d`` (the 3D spherical Riemann
problem, 128^3) and ``--workload bubble3d`` (the 3D shock-bubble, 325 x 90 x
90) time the 3D RHD examples, MM-O5 on the RMHD system with B = 0.  Each timed step advances the workload's initial
state by one full step (the state is restored on the device between steps,
outside the timed events): the untapered rotor loses admissibility after a
few steps (the scheme has no positivity limiter), and restoring keeps every
timed step a valid one.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "cell-updates/s per RK stage"
UNIT = "cell-updates/s"
N_SIDE = 400
WORKLOAD = ("2D RHD four-quadrant Riemann problem, 400x400 nodes on [-1,1]^2, outflow, Gamma=5/3, seeded states "
            "(rho in [0.1,1], |v|<=0.9, p in [0.01,1]), adaptive moving mesh (sigma=ln rho, alpha=1200, 4 filter "
            "passes, 10 Jacobi sweeps), 4th-order EC flux (p=2) + WENO5 dissipation, SSP-RK3, CFL 0.4")
# Flops per interface of the interface kernels are EXECUTED operations, from
# the ncu SASS counters of one capture of each kernel: dadd + dmul + 2 dfma
# (FP64) or fadd + fmul + 2 ffma (FP32), i.e. an add, a mul, or half an FMA,
# including the FP64 instructions inside division, square-root and log
# sequences.  The FP64 interface kernel (p = 2, WENO5) on the 400^2 Riemann
# workload executed 1,395 per interface before the paired WENO reconstructions
# (not recaptured since: None).
FLOPS_PER_IFACE_F64 = None
# Unit counts for the derived peaks, reported beside the measured ones:
# 4 FP64 flop/clk/SM and 256 FP32 flop/clk/SM at the 2070 MHz maximum clock.
FP64_FLOP_PER_CLK_SM = 4
FP32_FLOP_PER_CLK_SM = 256
# DRAM bytes (read + write) of one interface-kernel launch in that capture;
# None whenever the kernel has changed since the counters were taken.
TRAFFIC_IFACE_F64 = None
# The mixed form's interface kernel on the same workload: FP32 flops per
# interface and DRAM bytes per launch.
FLOPS_PER_IFACE_F32 = None
TRAFFIC_IFACE_F32 = None
# The same for the RMHD interface kernels at p = 2, WENO5: the FP64 2D kernel
# on the 512^2 rotor (10,898 FP64 flops per interface; 1.019 GB of DRAM
# traffic per launch, the eigen-system's per-thread stack), its FP32 instance
# (10,712 FP32 flops per interface besides 103 FP64 ones; 0.467 GB), and the 3D
# kernel (16,265 FP64 flops per interface; 1.212 GB at 64^3, scaled by the
# 7.94x interfaces of a 128^3 launch -- the stack traffic grows with the
# threads).
FLOPS_PER_IFACE_MHD2 = 10898
TRAFFIC_IFACE_MHD2 = 1.019e9
FLOPS_PER_IFACE_MHD2_F32 = 10712
TRAFFIC_IFACE_MHD2_F32 = 0.467e9
FLOPS_PER_IFACE_MHD3 = 16265
TRAFFIC_IFACE_MHD3 = 9.62e9
# The fused sweep kernel (pair and interface fluxes in one launch) on the
# same workload, from one capture of each form: executed flops per interface
# (its pair fluxes included: 32 anchors per 31 interfaces) and DRAM bytes
# per launch; None whenever the kernel has changed since.
FLOPS_PER_SWEEP_F64 = 1573
TRAFFIC_SWEEP_F64 = 13.10e6
FLOPS_PER_SWEEP_F32 = 1363
TRAFFIC_SWEEP_F32 = 11.74e6
# The counters above were captured on kernels built from these sources. The
# bench reports a kernel's counters only while its sources still hash to the
# digest recorded at that capture: an edit of any of them drops that
# kernel's executed flops and traffic to null until they are captured again
# and the digest is recorded anew.
COUNTER_SOURCES = {
    "sweep": ("esmm_sweep.cuh", "esmm_flux.cuh", "esmm_device.cuh", "esmm_conv.h"),
    "mhd2": ("esmm_mhd.cuh", "esmm_device.cuh", "esmm_conv.h"),
    "mhd3": ("esmm_3d.cuh", "esmm_3d_iface.cu", "esmm_mhd.cuh", "esmm_device.cuh", "esmm_conv.h"),
}
COUNTER_DIGEST = {"sweep": "5c6fe845469dcca2", "mhd2": "154efcb90ff39846", "mhd3": "dd8daf5262c5c5b3"}


def source_digest(kind, csrc=None):
    """First 16 hex digits of the SHA-256 of a kernel's sources, in order."""
    import hashlib
    csrc = csrc or os.path.join(ROOT, "paper_2107_12027_gb300", "csrc")
    h = hashlib.sha256()
    for f in COUNTER_SOURCES[kind]:
        with open(os.path.join(csrc, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def counters_current(kind):
    return source_digest(kind) == COUNTER_DIGEST[kind]


N_SM = 152
SM_MAX_MHZ = 2070.0
# Algorithmic HBM bytes per node and RK stage of the whole step, fused to the
# minimum: each stage reads the state and J of the stage and of t^n, x^n and
# the mesh velocity and writes the new state and J (stage 1 reads t^n's only),
# averaged over the three stages; plus the mesh redistribution once per step
# (read rho and x^n, write the mesh velocity), a third of it per stage.
#   2D RHD  (m = 4): (112 + 152 + 152)/3 + 40/3 = 152.0 B
#   2D RMHD (m = 8): (176 + 248 + 248)/3 + 40/3 = 237.3 B
#   3D RMHD (m = 8): (192 + 264 + 264)/3 + 56/3 = 258.7 B
HBM_BYTES_PER_NODE_STAGE = {"rhd2": 152.0, "rmhd2": 237.3, "rmhd3": 258.7}
# The untapered 512^2 rotor loses admissibility in its first step at CFL 0.4
# on a static mesh and with the moving mesh under eq. cfl, in the oracle as
# on the GPU (the scheme has no positivity limiter); at CFL 0.3 the first
# step stays admissible.  Every timed rotor step starts from the initial
# state, so the workload runs at CFL 0.3.
ROTOR_CFL = 0.3


_PEAKS = {}


def alu_peak(precision):
    """(TFLOP/s, source) of the FP64 (precision "fp64") or FP32 pipe:
    measured once per process by the library's FMA-throughput kernel
    (esmm_fma_peak, ~1 s), else derived from the unit counts."""
    from paper_2107_12027_gb300 import esmm
    if precision not in _PEAKS:
        try:
            fl, _ = esmm.fma_peak(esmm.FP64 if precision == "fp64" else esmm.MIXED, 1.0)
            _PEAKS[precision] = (fl / 1e12, "measured: esmm_fma_peak (independent FMA chains, 8x256 threads per SM, "
                                            "CUDA events, ~1 s)")
        except Exception as e:   # noqa: BLE001 -- report the derived peak and why
            per = FP64_FLOP_PER_CLK_SM if precision == "fp64" else FP32_FLOP_PER_CLK_SM
            _PEAKS[precision] = (N_SM * per * SM_MAX_MHZ * 1e6 / 1e12, "derived (measurement failed: %s)" % e)
    return _PEAKS[precision]


def cpu_model():
    """The host CPU's model name and its number of hardware threads."""
    name = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.strip().startswith("Model name:"):
                name = line.split(":", 1)[1].strip()
                break
    except (OSError, subprocess.SubprocessError):
        pass
    return name or "unknown", os.cpu_count() or 1


def hbm_peak_gbs():
    """Measured HBM copy bandwidth of the GB300s (MEASURED_PEAKS.json),
    else the fallback measurement of 6.8 TB/s."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


def hbm_roofline(rate, kind):
    """Whole-step fraction of the HBM roofline: algorithmic bytes per
    node-stage x node-stages per second over the measured copy bandwidth."""
    peak, src = hbm_peak_gbs()
    ach = rate * HBM_BYTES_PER_NODE_STAGE[kind] / 1e9
    return {"bytes_per_node_stage": HBM_BYTES_PER_NODE_STAGE[kind], "achieved": ach, "peak": peak,
            "unit": "GB/s", "frac": ach / peak, "peak_source": src}


def kind_rates(g, torch, nodes, steps, restore=None):
    """Device time per step of each kernel kind (the library's per-launch
    event profiling, outside the timed region) and the RHS-only and
    mesh-only rates derived from it."""
    from paper_2107_12027_gb300 import esmm
    g.profile((1 << len(esmm.KINDS)) - 1)
    for _ in range(steps):
        if restore:
            restore()
        g.rk_step(sync=False)
    torch.cuda.synchronize()
    prof = g.profile_read()
    g.profile(0)
    per = {k: v[0] / steps for k, v in prof.items()}
    rhs = per["node"] + per["pairs"] + per["iface"] + per["update"]
    return {"ms_per_step": per,
            "rhs_only": {"value": nodes * 3 / (rhs * 1e-3), "unit": "cell-updates/s",
                         "note": "node, pair, interface and update kernels"},
            "mesh_only": {"value": nodes / (per["mesh"] * 1e-3) if per["mesh"] > 0 else None,
                          "unit": "node-updates/s", "note": "one mesh redistribution per step"}}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--form", default="fp64", choices=["fp64", "mixed"])
    ap.add_argument("--n", type=int, default=None, help="nodes per side (default per workload)")
    ap.add_argument("--workload", default="riemann",
                    choices=["riemann", "rotor", "blast3d", "sphere3d", "bubble3d", "batched"],
                    help="batched: only the batched leg (256 problems, mixed form), one JSON line")
    ap.add_argument("--no-extras", action="store_true", help="skip e2e, cpu baseline and mixed-form legs")
    ap.add_argument("--study", default=None, choices=["um-mm"],
                    help="um-mm: the efficiency of MM-O5 against UM-O5 on the Sec. 6 problems (one JSON line per run)")
    ap.add_argument("--problems", default="rp1,rp2,rp3,blast", help="problems of --study um-mm")
    return ap.parse_args()


def dist_env():
    return int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)), int(os.environ.get("LOCAL_RANK", 0))


def job_time_ms(total_ms, world, dist, device):
    """The job's time over the timed steps: the slowest rank's (a max
    all-reduce over the ranks; the only collective of a multi-rank run)."""
    import torch
    t = torch.tensor([total_ms], dtype=torch.float64, device=device)
    if world > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(nodes_per_rank, steps, world, job_ms):
    """Whole-job cell-updates per second per RK stage: every rank advances
    nodes_per_rank nodes of its own (its slab's own rows; weak scaling)."""
    return world * nodes_per_rank * 3 * steps / (job_ms * 1e-3)


def workload(n, rank=0):
    from paper_2107_12027_gb300 import workloads as wl
    return wl.riemann_config(n, offset=1 + rank)


def stacked_workload(n, world):
    """The sharded workload of a multi-rank run: `world` four-quadrant
    Riemann problems of n x n nodes stacked along x_2 into one grid of
    n x (n world) nodes on [-1,1] x [-1, 2 world - 1] (band k holds the
    seeded states of rank k's single-GPU problem, split at its centre)."""
    from paper_2107_12027_gb300 import workloads as wl
    x = wl.uniform_mesh(n, n * world, (-1.0, -1.0), (1.0, 2.0 * world - 1.0), (False, False))
    prim = np.empty((4, n * world, n))
    for k in range(world):
        band = slice(k * n, (k + 1) * n)
        prim[:, band] = wl.quadrant_riemann(x[:, band], wl.quadrant_states(wl.rng(1 + k)), split=(0.0, 2.0 * k))
    return x, np.ascontiguousarray(prim)


def grid_params(form):
    from paper_2107_12027_gb300 import esmm
    return dict(cfl=0.4, alpha=1200.0, monitor=esmm.MONITOR_LNRHO, n_filter=4, mu=10, move_mesh=1,
                precision=esmm.MIXED if form == "mixed" else esmm.FP64)


# ---------------------------------------------------------------- clocks
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (OSError, ValueError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
            out, _ = self.proc.communicate()
        sm, mx, reasons = [], 0.0, set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for line in out.splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = max(mx, float(f[2]))
            except ValueError:
                continue
            for name, val in zip(names, f[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(name)
        if not sm:
            return None
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": mx, "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------- CPU oracle
def oracle_sample_rate(n, budget_s, nsteps=1, rows=None, threads=0):
    """Time the FP64 oracle's rk_step on a 400-wide strip of the workload
    (rows chosen so the run takes about budget_s) on `threads` host threads
    (0: all); returns (cell-updates/s, description, rows, threads used)."""
    import oracle
    used = oracle.set_threads(threads)
    x, prim = workload(n)
    if rows is None:
        r0 = 16
        cfg = oracle.make_cfg(n, r0, bc=(1, 1), period=(2.0, 2.0), p=2, w=5, alpha=1200.0,
                              monitor=oracle.MONITOR_LNRHO)
        j0 = n // 2 - r0 // 2
        xs, ps = np.ascontiguousarray(x[:, j0:j0 + r0]), np.ascontiguousarray(prim[:, j0:j0 + r0])
        cons, J = oracle.init_state(cfg, ps, xs)
        t = time.perf_counter()
        oracle.rk_step(cfg, cons, J, xs)
        per_row = (time.perf_counter() - t) / r0
        rows = int(max(8, min(n, budget_s / max(nsteps * per_row, 1e-9))))
    j0 = max(0, n // 2 - rows // 2)
    cfg = oracle.make_cfg(n, rows, bc=(1, 1), period=(2.0, 2.0), p=2, w=5, alpha=1200.0,
                          monitor=oracle.MONITOR_LNRHO)
    xs, ps = np.ascontiguousarray(x[:, j0:j0 + rows]), np.ascontiguousarray(prim[:, j0:j0 + rows])
    cons, J = oracle.init_state(cfg, ps, xs)
    t = time.perf_counter()
    for _ in range(nsteps):
        cons, J, xs, _ = oracle.rk_step(cfg, cons, J, xs)
    el = time.perf_counter() - t
    rate = n * rows * 3 * nsteps / el
    desc = ("%d rk_step(s) of the FP64 C oracle (%d host thread%s, OpenMP over nodes and interfaces) on the "
            "central %dx%d strip of the %dx%d workload" % (nsteps, used, "" if used == 1 else "s", n, rows, n, n))
    return rate, desc, rows, used


def cpu_baseline(n, budget_s):
    """The oracle on all host threads (the reported baseline) and on one."""
    model, nthreads = cpu_model()
    rate, desc, _, used = oracle_sample_rate(n, budget_s, 1, threads=0)
    rate1, desc1, _, _ = oracle_sample_rate(n, budget_s, 1, threads=1)
    return {"value": rate, "unit": UNIT, "cores": used, "kind": "oracle", "sample": desc, "cpu_model": model,
            "host_threads": nthreads,
            "single_thread": {"value": rate1, "unit": UNIT, "cores": 1, "sample": desc1}}


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    K, W = args.steps, args.warmup
    budget = 150.0 / max(1, K + W)      # whole run in about 2.5 minutes
    model, _ = cpu_model()
    _, _, rows, used = oracle_sample_rate(args.n, budget, 1)
    rates = []
    for s in range(W + K):
        rate, desc, _, used = oracle_sample_rate(args.n, budget, 1, rows=rows)
        if s >= W:
            rates.append(rate)
    value = float(len(rates) / sum(1.0 / r for r in rates))
    ms = args.n * args.n * 3 / value * 1e3
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": K, "warmup": W, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "nodes": args.n * args.n, "form": "fp64 oracle"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": used, "kind": "oracle", "sample": desc,
                             "cpu_model": model},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------- GPU legs
def timed_steps(g, torch, K, W, flush, stream, clock=None):
    """K steps through esmm_advance, one call per step: the warm-up (W >= 2)
    captures the step as a CUDA graph with event nodes around the interface
    kernels, and each timed step replays it (the library reads the graph's
    events between replays); L2 is flushed before every step."""
    from paper_2107_12027_gb300 import esmm
    g.profile(1 << esmm.KIND_IFACE)
    g.advance(W)
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(K)]
    g.profile(1 << esmm.KIND_IFACE)   # counters from zero; the graph stays
    if clock:
        clock.start()
    with torch.cuda.stream(stream):
        for k in range(K):
            flush.zero_()
            ev[k][0].record(stream)
            g.advance(1)
            ev[k][1].record(stream)
    torch.cuda.synchronize()
    clk = clock.stop() if clock else None
    prof = g.profile_read()
    total_ms = sum(a.elapsed_time(b) for a, b in ev)
    return total_ms, prof, clk


def e2e_leg(torch, n, form, K, W, stream):
    """Same metric through the public API with host buffers: every step copies
    the state in from pinned host memory and reads it back."""
    from paper_2107_12027_gb300 import esmm
    x, prim = workload(n)
    with esmm.Grid((n, n), (-1, -1), (1, 1), bc=(esmm.OUTFLOW, esmm.OUTFLOW), p=2, w=5,
                   stream=stream.cuda_stream, **grid_params(form)) as g:
        g.state_set(prim, x)
        pin = lambda shape: torch.empty(shape, dtype=torch.float64, pin_memory=True).numpy()
        cons, J, xs = pin((4, n, n)), pin((n, n)), pin((2, n, n))
        g.state_get(esmm.GET_CONS, cons)
        g.state_get(esmm.GET_J, J)
        g.state_get(esmm.GET_X, xs)
        t = 0.0

        def one():
            g.state_set_cons(cons, J, xs, t)
            g.advance(1)
            g.state_get(esmm.GET_CONS, cons)
            g.state_get(esmm.GET_J, J)
            g.state_get(esmm.GET_X, xs)
        g.advance(2)   # captures the step graph that advance(1) replays
        for _ in range(W):
            one()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(K):
            one()
        torch.cuda.synchronize()
        el = time.perf_counter() - t0
    nb = (4 + 1 + 2) * n * n * 8
    return {"value": n * n * 3 * K / el, "unit": UNIT, "h2d_bytes_per_step": nb, "d2h_bytes_per_step": nb}


def mixed_vs_fp64(torch, n, stream, nsteps=20):
    """Mixed form against the FP64 form (itself at 1e-12 of the oracle) after
    nsteps steps with the same fixed dt: L1 density error and entropy drift."""
    from paper_2107_12027_gb300 import esmm
    x, prim = workload(n)
    out = {}
    for form in ("fp64", "mixed"):
        with esmm.Grid((n, n), (-1, -1), (1, 1), bc=(esmm.OUTFLOW, esmm.OUTFLOW), p=2, w=5,
                       stream=stream.cuda_stream, **grid_params(form)) as g:
            g.state_set(prim, x)
            if form == "fp64":
                dt = 0.9 * g.cfl_dt()
            S0 = g.totals()[0]
            g.advance(nsteps, dt)
            out[form] = (g.state_get(esmm.GET_PRIM)[0], g.totals()[0], S0)
    rf, rm = out["fp64"][0], out["mixed"][0]
    return {"steps": nsteps, "dt": dt,
            "l1_rho_rel": float(np.abs(rm - rf).mean() / np.abs(rf).mean()),
            "entropy_rel_diff": float(abs(out["mixed"][1] - out["fp64"][1]) / abs(out["fp64"][1])),
            "entropy_change_fp64": float((out["fp64"][1] - out["fp64"][2]) / abs(out["fp64"][2])),
            "entropy_change_mixed": float((out["mixed"][1] - out["mixed"][2]) / abs(out["mixed"][2]))}


def batch_leg(torch, stream, steps=50, warm=2):
    """Batched workload: 256 independent seeded four-quadrant Riemann
    problems with sides uniform in [64, 512] (|v| <= 0.5), FP32 bulk with FP64
    recovery, every kernel one launch over the whole batch, steps replayed
    from a CUDA graph, launch shapes autotuned; 50 RK3 steps.  The working
    set (~18 GB) is far larger than L2."""
    from paper_2107_12027_gb300 import esmm
    from paper_2107_12027_gb300 import workloads as wl
    sides = wl.batch_sizes()
    with esmm.Batch([(int(s), int(s)) for s in sides], lo=(-1, -1), hi=(1, 1), bc=(esmm.OUTFLOW, esmm.OUTFLOW),
                    p=2, w=5, stream=stream.cuda_stream, **grid_params("mixed")) as b:
        for k, s in enumerate(sides):
            x, prim = wl.batch_problem(k, int(s))
            b.state_set(k, prim, x)
        shapes = b.tune()
        b.advance(warm)
        torch.cuda.synchronize()
        b.profile(0)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        # the profiler range marks the timed steps for a profiler started
        # with profiling off (a no-op otherwise)
        torch.cuda.profiler.start()
        e0.record(stream)
        b.advance(steps)
        e1.record(stream)
        torch.cuda.synchronize()
        torch.cuda.profiler.stop()
        ms = e0.elapsed_time(e1)
        nfail, _ = b.last_error()
        launches = int(sum(v[1] for v in b.profile_read().values()))
        nodes = int(sum(int(s) ** 2 for s in sides))
    return {"value": nodes * 3 * steps / (ms * 1e-3), "unit": UNIT, "problems": len(sides), "nodes": nodes,
            "side_range": [int(sides.min()), int(sides.max())], "steps": steps, "ms_per_step": ms / steps,
            "precision": "f32 bulk + f64 recovery", "graph": True, "tile_shapes": shapes,
            "gpu_launches": launches, "failed_recoveries": int(nfail)}


def run_batched(args):
    """The batched leg alone (the default line carries it under forms)."""
    import torch
    torch.cuda.set_device(0)
    stream = torch.cuda.Stream()
    leg = batch_leg(torch, stream, steps=args.steps, warm=max(args.warmup, 1))
    line = {"metric": METRIC, "value": leg.pop("value"), "unit": leg.pop("unit"), "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": leg["ms_per_step"],
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64",
            "data": "synthetic", "config": {"workload": "256 seeded four-quadrant Riemann problems, sides in [64, 512]",
                                            "form": "mixed", **leg}}
    print(json.dumps(line), flush=True)


def run_gpu(args):
    import torch
    import torch.distributed as dist
    from paper_2107_12027_gb300 import esmm

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    esmm.lib()
    stream = torch.cuda.Stream()
    n, K, W = args.n, args.steps, args.warmup
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")   # 256 MB > L2
    if world > 1:
        # one problem sharded over the ranks: slab k of the stacked grid on
        # rank k, reductions and halo exchanges over a gloo group
        from paper_2107_12027_gb300.comm import TorchComm
        x, prim = stacked_workload(n, world)
        g = esmm.Slab((n, n * world), world, rank, TorchComm(dist.new_group(backend="gloo")), lo=(-1, -1),
                      hi=(1, 2 * world - 1), bc=(esmm.OUTFLOW, esmm.OUTFLOW), p=2, w=5, stream=stream.cuda_stream,
                      **grid_params(args.form))
    else:
        x, prim = workload(n, rank)
        g = esmm.Grid((n, n), (-1, -1), (1, 1), bc=(esmm.OUTFLOW, esmm.OUTFLOW), p=2, w=5,
                      stream=stream.cuda_stream, **grid_params(args.form))
    g.state_set(prim, x)
    if world > 1:
        x, prim = workload(n, rank)   # the single-GPU problem for the extras below
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    clock = ClockSampler(local) if rank == 0 else None
    total_ms, prof, clk = timed_steps(g, torch, K, W, flush, stream, clock)
    nfail, msg = g.last_error()
    if nfail:
        raise RuntimeError("primitive recovery failed at %d nodes: %s" % (nfail, msg))
    total_ms = job_time_ms(total_ms, world, dist, "cuda")
    if world > 1:
        dist.barrier()
    value = job_rate(n * n, K, world, total_ms)
    launches = int(sum(v[1] for v in prof.values()))
    fused = g.get_params()["sweep"] != esmm.SWEEP_SPLIT   # untuned: AUTO runs the fused sweep
    g.close()
    if rank != 0:
        if world > 1:
            dist.destroy_process_group()
        return

    # roofline of the dominant kernel, the flux kernel of a sweep (the fused
    # sweep kernel, or the interface kernel when the pair and interface
    # kernels run apart): bound by the FP64 pipe in the FP64 form (no dense
    # contraction, ~20 FP64 flop per byte), by the FP32 pipes in the mixed one
    iface_ms, iface_n, iface_timed = prof["iface"]
    ifaces_per_launch = ((n + 1) * n + (n + 1) * n) / 2.0
    avg_launch_s = iface_ms * 1e-3 / max(iface_timed, 1)
    # the method's operations per interface (the library's flux templates on
    # a counting type; each divide and root counts once) beside the executed ones
    ops = esmm.flux_ops(5.0 / 3.0, 2, 5)
    alg = ops["dissipation"] + ops["combination"] + (2 * ops["pair"] if fused else 0)
    f64 = args.form == "fp64"
    peak, src = alu_peak("fp64" if f64 else "fp32")
    if fused:
        flops = FLOPS_PER_SWEEP_F64 if f64 else FLOPS_PER_SWEEP_F32
        traffic = TRAFFIC_SWEEP_F64 if f64 else TRAFFIC_SWEEP_F32
        if not counters_current("sweep"):
            flops = traffic = None
        kname = "k_sweep<%s,2,5>" % ("double" if f64 else "float")
    else:
        flops = FLOPS_PER_IFACE_F64 if f64 else FLOPS_PER_IFACE_F32
        traffic = TRAFFIC_IFACE_F64 if f64 else TRAFFIC_IFACE_F32
        kname = "k_iface<%s,2,5>" % ("double" if f64 else "float")
    ach = flops * ifaces_per_launch / avg_launch_s / 1e12 if flops else None
    prec = "FP64" if f64 else "FP32"
    ops_names = "dadd + dmul + 2 dfma" if f64 else "fadd + fmul + 2 ffma"
    roof = {"bound": "alu", "achieved": ach, "peak": peak, "unit": "TFLOP/s",
            "frac": ach / peak if ach else None, "traffic": traffic, "kernel": kname,
            "avg_launch_ms": avg_launch_s * 1e3, "share_of_step": iface_ms / total_ms, "peak_source": src,
            "peak_derived": N_SM * (FP64_FLOP_PER_CLK_SM if f64 else FP32_FLOP_PER_CLK_SM) * SM_MAX_MHZ * 1e6 / 1e12,
            "flops_basis": ("executed %s operations per interface (ncu: %s), %d per interface"
                            % (prec, ops_names, flops)) if flops else "not measured for this kernel",
            "algorithmic": {"flops_per_interface": alg,
                            "achieved": alg * ifaces_per_launch / avg_launch_s / 1e12,
                            "frac": alg * ifaces_per_launch / avg_launch_s / 1e12 / peak,
                            "basis": "esmm_flux_ops: ES dissipation %d + pair combination %d%s operations per "
                                     "interface (add, mul, div, sqrt, rsqrt each 1)"
                                     % (ops["dissipation"], ops["combination"],
                                        " + two pair fluxes of %d" % ops["pair"] if fused else "")}}
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": K, "warmup": W,
            "ms_per_step": total_ms / K, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64" if args.form == "fp64" else "f32+f64",
            "data": "synthetic",
            "config": {"workload": WORKLOAD, "nodes": n * n, "form": args.form,
                       "l2": "flushed (256 MB write) before every timed step",
                       "parallelism": ("one %dx%d grid of %d stacked problems, slab-decomposed along x_2: %d own "
                                       "rows (+%d-row halos) per rank, halo exchange and reductions over gloo"
                                       % (n, n * world, world, n, esmm.SLAB_HALO)) if world > 1 else "single GPU"},
            "gpu_launches": launches, "roofline": roof, "clocks": clk,
            "hbm": hbm_roofline(value / world, "rhd2")}
    if not args.no_extras:
        with esmm.Grid((n, n), (-1, -1), (1, 1), bc=(esmm.OUTFLOW, esmm.OUTFLOW), p=2, w=5,
                       stream=stream.cuda_stream, **grid_params(args.form)) as gk:
            gk.state_set(prim, x)
            line["kinds"] = kind_rates(gk, torch, n * n, 10)
        line["e2e"] = e2e_leg(torch, n, args.form, max(3, min(K, 50)), 2, stream)
        line["cpu_baseline"] = cpu_baseline(n, 10.0)
        if args.form == "fp64":
            with esmm.Grid((n, n), (-1, -1), (1, 1), bc=(esmm.OUTFLOW, esmm.OUTFLOW), p=2, w=5,
                           stream=stream.cuda_stream, **grid_params("mixed")) as gm:
                gm.state_set(prim, x)
                tm, _, _ = timed_steps(gm, torch, K, W, flush, stream, None)
                forms = {"mixed": {"value": n * n * 3 * K / (tm * 1e-3), "ms_per_step": tm / K,
                                   "kinds": kind_rates(gm, torch, n * n, 10)}}
            forms["mixed"].update(mixed_vs_fp64(torch, n, stream))
            forms["batched"] = batch_leg(torch, stream)
            line["forms"] = forms
            # the other single-GPU configurations: the 512^2 RMHD rotor (FP64,
            # with its mixed form) and the 128^3 RMHD blast (FP64)
            sub = argparse.Namespace(workload="rotor", form="fp64", n=None, steps=5, warmup=3, no_extras=False)
            blast = argparse.Namespace(workload="blast3d", form="fp64", n=None, steps=3, warmup=2, no_extras=True)
            line["workloads"] = {"rotor512": rmhd_line(sub), "blast128": rmhd_line(blast)}
            line["peaks"] = {"fp64_tflops": alu_peak("fp64")[0], "fp32_tflops": alu_peak("fp32")[0],
                             "source": alu_peak("fp64")[1]}
    print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


# ---------------------------------------------------------------- RMHD workloads
def rotor_mixed_vs_fp64(torch, n, stream, nsteps=1):
    """Mixed form against the FP64 form on the rotor after nsteps steps with
    the FP64 form's time steps: L1 density error and total-entropy difference.
    The untapered 512^2 rotor loses admissibility in its second step in
    either form (the disk edge is a jump of 10 in density moving at 0.995),
    so the comparison takes one step."""
    from paper_2107_12027_gb300 import esmm
    from paper_2107_12027_gb300 import workloads as wl
    x, prim = wl.rotor_config(n)
    out = {}
    for form in ("fp64", "mixed"):
        with esmm.Grid((n, n), (-0.5, -0.5), (0.5, 0.5), bc=(1, 1), p=2, w=5, gamma=4.0 / 3.0, phys=esmm.RMHD,
                       stream=stream.cuda_stream, alpha=800.0, monitor=esmm.MONITOR_LNRHO, cfl=ROTOR_CFL,
                       precision=esmm.MIXED if form == "mixed" else esmm.FP64) as g:
            g.state_set(prim, x)
            S0 = g.totals()[0]
            if form == "fp64":
                dts = [g.rk_step() for _ in range(nsteps)]
            else:
                for dt in dts:
                    g.advance(1, dt)
            out[form] = (g.state_get(esmm.GET_PRIM)[0], g.totals()[0], S0)
    rf, rm = out["fp64"][0], out["mixed"][0]
    return {"steps": nsteps, "dt": dts,
            "l1_rho_rel": float(np.abs(rm - rf).mean() / np.abs(rf).mean()),
            "entropy_rel_diff": float(abs(out["mixed"][1] - out["fp64"][1]) / abs(out["fp64"][1])),
            "entropy_change_fp64": float((out["fp64"][1] - out["fp64"][2]) / abs(out["fp64"][2])),
            "entropy_change_mixed": float((out["mixed"][1] - out["mixed"][2]) / abs(out["mixed"][2]))}


def run_rmhd(args):
    print(json.dumps(rmhd_line(args)), flush=True)


def rmhd_line(args):
    """Time the 2D RMHD rotor (FP64 or mixed form) or a 3D workload (FP64) on
    one GPU; returns the bench line."""
    import torch
    from paper_2107_12027_gb300 import esmm
    from paper_2107_12027_gb300 import workloads as wl
    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    esmm.lib()
    stream = torch.cuda.Stream()
    three = args.workload in ("blast3d", "sphere3d", "bubble3d")
    if three and args.form != "fp64":
        raise SystemExit("the 3D workloads run in the FP64 form only")
    n = args.n or (128 if three else 512)
    K, W = args.steps, args.warmup
    if args.workload == "sphere3d":
        x = wl.uniform_mesh3((n, n, n), (-1.0,) * 3, (1.0,) * 3, (False, False, False))
        prim = wl.sphere_rp3(x)
        g = esmm.Grid3((n, n, n), (-1.0,) * 3, (1.0,) * 3, bc=(1, 1, 1), gamma=5.0 / 3.0, scheme="MM-O5",
                       alpha=800.0, monitor=esmm.MONITOR_LNRHO, stream=stream.cuda_stream)
        nodes = n ** 3
        ifaces = (n + 1) * n * n
        desc = ("3D spherical Riemann problem (an RHD problem on the RMHD system, B = 0), %d^3 nodes on [-1,1]^3, "
                "outflow, Gamma=5/3, r<0.5: rho=10, p=40/3; outside rho=1, p=1e-2; at rest; MM-O5 (6th-order EC "
                "flux p=3 + WENO5), adaptive moving mesh (sigma=ln rho, alpha=800), SSP-RK3, CFL 0.3" % n)
        flops, traffic, kname = None, None, "k3_iface<3,5>"
    elif args.workload == "bubble3d":
        m = (n, max(8, round(n * 90 / 325)), max(8, round(n * 90 / 325))) if args.n else (325, 90, 90)
        x, prim = wl.rhd_shock_bubble3_config(m)
        g = esmm.Grid3(m, (0.0, -45.0, -45.0), (325.0, 45.0, 45.0), bc=(1, 1, 1), gamma=5.0 / 3.0,
                       scheme="MM-O5", alpha=800.0, monitor=esmm.MONITOR_LNRHO, stream=stream.cuda_stream)
        nodes = m[0] * m[1] * m[2]
        ifaces = (m[0] + 1) * m[1] * m[2]
        desc = ("3D shock-bubble (an RHD problem on the RMHD system, B = 0), %dx%dx%d nodes on [0,325]x[-45,45]^2, "
                "outflow, Gamma=5/3, planar shock at x1=265 (post-shock rho=1.865225080631180, v1=-0.196781107378299, "
                "p=0.15) moving into rho=1, p=0.05 at rest, bubble r<=25 at (215,0,0) with rho=0.1358; MM-O5 "
                "(6th-order EC flux p=3 + WENO5), adaptive moving mesh (sigma=ln rho, alpha=800), SSP-RK3, CFL 0.3"
                % m)
        flops, traffic, kname = None, None, "k3_iface<3,5>"
    elif three:
        x, prim = wl.blast3_config(n)
        g = esmm.Grid3((n, n, n), (-0.5,) * 3, (0.5,) * 3, bc=(1, 1, 1), p=2, w=5, stream=stream.cuda_stream)
        nodes = n ** 3
        ifaces = (n + 1) * n * n
        desc = ("3D RMHD blast, %d^3 nodes on [-0.5,0.5]^3, outflow, Gamma=4/3, sphere r<0.1 with p=1, rho=1e-2, "
                "background p=5e-4, rho=1e-4, B=(0.1,0,0), at rest, adaptive moving mesh (sigma=ln rho, alpha=800), "
                "4th-order EC flux (p=2) + WENO5, SSP-RK3, CFL 0.3" % n)
        flops, traffic, kname = FLOPS_PER_IFACE_MHD3, TRAFFIC_IFACE_MHD3, "k3_iface<2,5>"
        if not counters_current("mhd3"):
            flops = traffic = None
    else:
        x, prim = wl.rotor_config(n)
        g = esmm.Grid((n, n), (-0.5, -0.5), (0.5, 0.5), bc=(1, 1), p=2, w=5, gamma=4.0 / 3.0, phys=esmm.RMHD,
                      stream=stream.cuda_stream, alpha=800.0, monitor=esmm.MONITOR_LNRHO, cfl=ROTOR_CFL,
                      precision=esmm.MIXED if args.form == "mixed" else esmm.FP64)
        nodes = n * n
        ifaces = (n + 1) * n
        desc = ("2D RMHD rotor, %dx%d nodes on [-0.5,0.5]^2, outflow, Gamma=4/3, disk r<0.1 with rho=10 at angular "
                "speed 9.95, background rho=1, p=1, B=(1,0,0), adaptive moving mesh (sigma=ln rho, alpha=800), "
                "4th-order EC flux (p=2) + WENO5 + Powell source, SSP-RK3, CFL %g" % (n, n, ROTOR_CFL))
        flops, traffic, kname = FLOPS_PER_IFACE_MHD2, TRAFFIC_IFACE_MHD2, "k_iface_mhd<double,2,5>"
        if args.form == "mixed":
            flops, traffic, kname = FLOPS_PER_IFACE_MHD2_F32, TRAFFIC_IFACE_MHD2_F32, "k_iface_mhd<float,2,5>"
        if not counters_current("mhd2"):
            flops = traffic = None
    g.state_set(prim, x)
    dev = torch.device("cuda", local)
    c0 = torch.empty(((8,) + tuple(prim.shape[1:])), dtype=torch.float64, device=dev)
    J0 = torch.empty(tuple(prim.shape[1:]), dtype=torch.float64, device=dev)
    x0 = torch.empty(((3 if three else 2,) + tuple(prim.shape[1:])), dtype=torch.float64, device=dev)
    g.state_get(esmm.GET_CONS, c0)
    g.state_get(esmm.GET_J, J0)
    g.state_get(esmm.GET_X, x0)
    torch.cuda.synchronize()
    for _ in range(W):
        g.state_set_cons(c0, J0, x0)
        g.rk_step()
    g.profile(1 << esmm.KIND_IFACE)
    flush = None if three else torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)   # 256 MB > L2
    clock = ClockSampler(local)
    clock.start()
    total_ms = 0.0
    for _ in range(K):
        g.state_set_cons(c0, J0, x0)
        if flush is not None:
            flush.zero_()
            torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        g.rk_step(sync=False)
        e1.record(stream)
        torch.cuda.synchronize()
        total_ms += e0.elapsed_time(e1)
    clk = clock.stop()
    nfail, msg = g.last_error()
    if nfail:
        raise RuntimeError("primitive recovery failed at %d nodes: %s" % (nfail, msg))
    prof = g.profile_read()
    launches = int(sum(v[1] for v in prof.values()))
    iface_ms, _, iface_timed = prof["iface"]
    avg = iface_ms * 1e-3 / max(iface_timed, 1)
    mixed = args.form == "mixed"
    per_clk = FP32_FLOP_PER_CLK_SM if mixed else FP64_FLOP_PER_CLK_SM
    peak, src = alu_peak("fp32" if mixed else "fp64")
    ach = flops * ifaces / avg / 1e12 if flops else None
    roof = {"bound": "alu", "achieved": ach, "peak": peak, "unit": "TFLOP/s",
            "frac": (ach / peak) if ach else None, "traffic": traffic, "kernel": kname,
            "avg_launch_ms": avg * 1e3, "share_of_step": iface_ms / total_ms, "peak_source": src,
            "peak_derived": N_SM * per_clk * SM_MAX_MHZ * 1e6 / 1e12,
            "flops_basis": ("executed %s operations per interface (ncu SASS counters), %s per interface"
                            % ("FP32" if mixed else "FP64", flops)) if flops else None}
    kinds = None
    if not args.no_extras:
        kinds = kind_rates(g, torch, nodes, 3, restore=lambda: g.state_set_cons(c0, J0, x0))
    g.close()
    line = {"metric": METRIC, "value": nodes * 3 * K / (total_ms * 1e-3), "unit": UNIT, "n_gpus": 1, "steps": K,
            "warmup": W, "ms_per_step": total_ms / K, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64" if args.form == "fp64" else "f32+f64", "data": "synthetic",
            "config": {"workload": desc, "nodes": nodes, "form": args.form,
                       "steps": "each from the initial state (restored on the device, outside the timed events)",
                       "l2": ("working set (~0.5 GB of node data) larger than L2" if three
                              else "flushed (256 MB write) before every timed step"),
                       "parallelism": "single GPU"},
            "roofline": roof, "clocks": clk,
            "hbm": hbm_roofline(nodes * 3 * K / (total_ms * 1e-3), "rmhd3" if three else "rmhd2")}
    line["gpu_launches"] = launches
    if kinds:
        line["kinds"] = kinds
    if not three and args.form == "fp64" and not args.no_extras:
        with esmm.Grid((n, n), (-0.5, -0.5), (0.5, 0.5), bc=(1, 1), p=2, w=5, gamma=4.0 / 3.0, phys=esmm.RMHD,
                       stream=stream.cuda_stream, alpha=800.0, monitor=esmm.MONITOR_LNRHO, cfl=ROTOR_CFL,
                       precision=esmm.MIXED) as gm:
            gm.state_set(prim, x)
            tm = 0.0
            for k in range(W + K):
                gm.state_set_cons(c0, J0, x0)
                flush.zero_()
                torch.cuda.synchronize()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                gm.rk_step(sync=False)
                e1.record(stream)
                torch.cuda.synchronize()
                if k >= W:
                    tm += e0.elapsed_time(e1)
            if gm.last_error()[0]:
                raise RuntimeError("mixed form: primitive recovery failed")
        line["forms"] = {"mixed": {"value": nodes * 3 * K / (tm * 1e-3), "ms_per_step": tm / K}}
        line["forms"]["mixed"].update(rotor_mixed_vs_fp64(torch, n, stream))
    return line


# ---------------------------------------------------------------- UM-O5 vs MM-O5
# The paper's efficiency claim (Sec. 6, Table 6.1 and the Riemann problem
# figures): MM-O5 on a coarse adaptive mesh resolves what UM-O5 needs a much
# finer static mesh for, at a fraction of the cost.  Each problem runs MM-O5
# and UM-O5 at the paper's coarse size, UM-O5 at the paper's fine size, and
# UM-O5 finer still as the reference (for the blast the fine run itself, as
# in the paper's comparison); every run is timed on the GPU (wall
# time of the whole run, synchronised) and its final ln rho is compared with
# the reference's on a common 400 x 400 sample grid and along the cut line
# of the paper's figures (x_2 = x_1 for the Riemann problems, x_2 = 0 for the
# blast), as L1 means.
STUDY = {   # problem: (sizes (MM-O5, UM-O5 coarse, UM-O5 fine, reference), final time)
    "rp1": ((200, 200, 500, 1000), 0.4),
    "rp2": ((200, 200, 500, 1000), 0.4),
    "rp3": ((200, 200, 600, 1000), 0.4),
    "blast": ((150, 150, 600, 600), 4.0),   # the fine run is the reference (as in the paper's comparison)
}


def study_grid(problem, n, scheme):
    from paper_2107_12027_gb300 import esmm
    from paper_2107_12027_gb300 import workloads as wl
    if problem == "blast":
        x, prim = wl.rmhd_blast2_config(n)
        g = esmm.Grid((n, n), (-6.0, -6.0), (6.0, 6.0), bc=(esmm.OUTFLOW, esmm.OUTFLOW), gamma=4.0 / 3.0,
                      phys=esmm.RMHD, scheme=scheme, cfl=0.4, alpha=800.0, monitor=esmm.MONITOR_LNRHO)
    else:
        x, prim = wl.rhd_rp_config(int(problem[2]), n)
        g = esmm.Grid((n, n), (0.0, 0.0), (1.0, 1.0), bc=(esmm.OUTFLOW, esmm.OUTFLOW), gamma=5.0 / 3.0,
                      scheme=scheme, cfl=0.4, alpha=1200.0, monitor=esmm.MONITOR_LNRHO)
    g.state_set(prim, x)
    return g


def study_run(torch, problem, n, scheme, t_end):
    """Advance to t_end (CFL steps, the last one cut to land on t_end); return
    (final nodes, final ln rho, steps, seconds)."""
    from paper_2107_12027_gb300 import esmm
    g = study_grid(problem, n, scheme)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    steps, t = 0, 0.0
    while t_end - t > 1e-12 * t_end:
        rest = t_end - t
        dt = g.rk_step(rest if rest <= 0.9 * g.cfl_dt() else 0.0)
        steps += 1
        t = g.time()
        if steps > 200000:
            raise RuntimeError("study run did not reach t_end")
    torch.cuda.synchronize()
    sec = time.perf_counter() - t0
    nfail, msg = g.last_error()
    x, prim = g.state_get(esmm.GET_X), g.state_get(esmm.GET_PRIM)
    g.close()
    if nfail:
        raise RuntimeError("primitive recovery failed at %d nodes: %s" % (nfail, msg))
    return x, np.log(prim[0]), steps, sec


def study_sample(x, f, pts, uniform=False):
    """f (given at the nodes x) at the points pts [2][...] (linear
    interpolation: on the grid's axes when uniform, else on the Delaunay
    triangulation of the nodes)."""
    from scipy.interpolate import RegularGridInterpolator, griddata
    if uniform:
        f_ = RegularGridInterpolator((x[1][:, 0], x[0][0, :]), f)
        return f_(np.stack([pts[1].ravel(), pts[0].ravel()], axis=1)).reshape(pts.shape[1:])
    return griddata((x[0].ravel(), x[1].ravel()), f.ravel(), (pts[0], pts[1]), method="linear")


def study_points(problem, lo, hi, m=400, mc=1000):
    s = lo + (hi - lo) * (np.arange(m) + 0.5) / m
    Y, X = np.meshgrid(s, s, indexing="ij")
    c = lo + (hi - lo) * (np.arange(mc) + 0.5) / mc
    cut = np.stack([c, 0.0 * c]) if problem == "blast" else np.stack([c, c])
    return np.stack([X, Y]), cut


def run_study(args):
    import torch
    from paper_2107_12027_gb300 import esmm
    esmm.lib()
    for problem in args.problems.split(","):
        (n_mm, n_um, n_fine, n_ref), t_end = STUDY[problem]
        lo, hi = (-6.0, 6.0) if problem == "blast" else (0.0, 1.0)
        grid, cut = study_points(problem, lo, hi)
        xr, fr, steps, sec = study_run(torch, problem, n_ref, "UM-O5", t_end)
        ref, ref_c = study_sample(xr, fr, grid, uniform=True), study_sample(xr, fr, cut, uniform=True)
        line = {"study": "um-mm", "problem": problem, "scheme": "UM-O5", "n": n_ref, "t": t_end, "steps": steps,
                "seconds": sec, "role": "reference"}
        print(json.dumps(line), flush=True)
        for scheme, n in (("MM-O5", n_mm), ("UM-O5", n_um), ("UM-O5", n_fine)):
            if scheme == "UM-O5" and n == n_ref:
                continue
            x, f, steps, sec = study_run(torch, problem, n, scheme, t_end)
            got = study_sample(x, f, grid, uniform=scheme == "UM-O5")
            got_c = study_sample(x, f, cut, uniform=scheme == "UM-O5")
            print(json.dumps({"study": "um-mm", "problem": problem, "scheme": scheme, "n": n, "t": t_end,
                              "steps": steps, "seconds": sec,
                              "l1_lnrho_vs_ref": float(np.nanmean(np.abs(got - ref))),
                              "l1_lnrho_cut_vs_ref": float(np.nanmean(np.abs(got_c - ref_c))),
                              "ref": "UM-O5 %d" % n_ref}), flush=True)


def main():
    args = parse()
    if args.study:
        run_study(args)
        return
    if args.workload == "batched":
        run_batched(args)
        return
    if args.workload != "riemann":
        run_rmhd(args)
        return
    if args.n is None:
        args.n = N_SIDE
    if args.impl == "reference":
        run_reference(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
