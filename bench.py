"""Benchmark of the Fisher-forecast hot path on GB300.

One step = one pass of the whole hot path over the 1e5-event uneven catalog
(70 % BBH / 30 % tidal BNS, rotating triangle, per-event log grid from 2 Hz to
f_ISCO): catalog preparation, network SNR + 11x11 Fisher matrix (mixed
precision by default), batched FP64 Cholesky inversion with conditioning
check, and the VJP of the network SNR with respect to all 11 source
parameters.  Inputs are resident in HBM before the timed region; L2 is
flushed (256 MiB write) before every timed step.

  python bench.py [--gpus N --steps K --warmup W] [--precision mixed|fp64]
                  [--grid literal|stress] [--impl ours|reference]

--impl reference times the CPU oracle (oracle/) on a bounded sample of the same
workload on the host cores (the paper's method has no GPU implementation).
Prints one JSON line.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np

import gwcat

METRIC = "events/s (SNR + 11x11 Fisher), mixed vs FP64 path at stated error; % FP peak"
WORKLOAD = "c3: 1e5 events, 70% BBH (5-80 Msun, spins) + 30% tidal BNS, ET-like triangle, " \
           "Earth rotation, per-event log grid 2 Hz..f_ISCO"
WORKLOAD_C4 = "c4: 1e6 events drawn as c3 on five interferometers (triangle + two L)"
WORKLOAD_GATED = ("c3-gated: the c3 catalog with a duty factor of 0.85 per triangle arm "
                  "(seeded per-event arm masks), an SNR pass over every event, the SNR > 12 "
                  "detection gate, then Fisher + inversion of the selected events")
GATE_SNR = 12.0       # default snr_th of the paper's forecast driver (Sec. 5)
GATE_DUTY = 0.85      # duty factor per arm of the gated workload
N_PAR = 11
SM_COUNT = 152
DFMA_PER_CLK_SM = 2          # measured on GB300: 2 FP64 FMA / clock / SM (1.26 TFLOP/s)
FFMA_PER_CLK_SM = 128        # FP32 FMA lanes per SM (measured 117 / clock with a plain FFMA loop)
# DRAM bytes (read + write) per grid point of the Fisher point kernel, from one
# ncu capture of the 2e4-event c3 catalog (4,376,070 points) of the current
# kernels (profiles/k_points_*_fisher_c3.md); scaled by points to a full launch
DRAM_BYTES_PER_POINT = {"mixed": (23.10528e6 + 11.52e3) / 4376070,
                        "fp64": (19.284224e6 + 91.136e3) / 4376070}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=60)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--precision", choices=["mixed", "fp64"], default="mixed")
    ap.add_argument("--grid", choices=["literal", "stress"], default="literal")
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--events", type=int, default=None)
    ap.add_argument("--workload", choices=["c3", "c4", "c3-gated"], default="c3",
                    help="c3: 1e5 events on the triangle (headline); c4: 1e6 events on five "
                         "interferometers, the step adding the log-det VJP over the two "
                         "L detectors' orientations; c3-gated: c3 with duty-factor arm masks, "
                         "an SNR pass and the SNR > 12 gate before the Fisher pass")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--eager", action="store_true",
                    help="launch the step call by call instead of replaying a CUDA graph")
    return ap.parse_args()


# ------------------------------------------------------------------ oracle leg
def _oracle_event_step(args):
    """Every row of the step for one event, on the CPU oracle."""
    import oracle
    raw, rule, det, psd, rot = args
    p = oracle.prepare(raw["m1"], raw["m2"], raw["chi1"], raw["chi2"], raw["lam1"], raw["lam2"],
                       raw["dL_Mpc"], raw["zflag"], raw["tcoal"])
    if rule[0] == "efold":
        npts = oracle.grid_npts(raw["fmin"], p["fisco"], *rule[1:])
    else:
        npts = raw["npts"]
    ev = np.stack([p["Mc"], p["eta"], p["dL"], raw["theta"], raw["phi"], raw["iota"], raw["psi"],
                   p["tc"], raw["Phic"], p["chi1z"], p["chi2z"], p["LamT"], p["dLamT"]], 1)
    cat = oracle.Catalog(ev, raw["pset"], raw["fmin"], p["fisco"], npts)
    F, s, err, st = oracle.fisher(cat, det, psd, rot, N_PAR)
    oracle.invert(F)
    oracle.snr_grad(cat, det, psd, rot, N_PAR)
    return 1


def _sample(raw, idx):
    out = {}
    for k, v in raw.items():
        if isinstance(v, np.ndarray) and v.shape[:1] == (len(raw["m1"]),):
            out[k] = v[idx]
    return out


def oracle_timing(raw, n_events, cores, budget_s=20.0):
    """Time the oracle on a bounded sample of the workload (spawn pool)."""
    import multiprocessing as mp
    import oracle
    oracle.build()
    det, psd, rot = gwcat.network("c3")
    rule = raw["npts_rule"]
    ctx = mp.get_context("spawn")
    rng = np.random.default_rng(1)
    with ctx.Pool(cores) as pool:
        pool.map(_oracle_event_step, [(_sample(raw, [0]), rule, det, psd, rot)])   # warm
        done, t0 = 0, time.time()
        while True:
            idx = rng.choice(len(raw["m1"]), cores, replace=False)
            tasks = [(_sample(raw, [i]), rule, det, psd, rot) for i in idx]
            done += sum(pool.map(_oracle_event_step, tasks))
            el = time.time() - t0
            if el >= budget_s or done >= n_events:
                return done / el, done, el


def run_reference(a):
    raw = gwcat.draw("c3", a.events, grid=a.grid)
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    cores = os.cpu_count() or 1
    det, psd, rot = gwcat.network("c3")
    import multiprocessing as mp
    import oracle
    oracle.build()
    rng = np.random.default_rng(2)
    times = []
    with mp.get_context("spawn").Pool(cores) as pool:
        for i in range(a.warmup + a.steps):
            idx = rng.choice(len(raw["m1"]), cores, replace=False)
            tasks = [(_sample(raw, [j]), raw["npts_rule"], det, psd, rot) for j in idx]
            t0 = time.time()
            pool.map(_oracle_event_step, tasks)
            if i >= a.warmup:
                times.append(time.time() - t0)
    per_step = float(np.mean(times))
    value = cores / per_step
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "events/s",
        "n_gpus": a.gpus, "steps": a.steps, "warmup": a.warmup, "ms_per_step": per_step * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64/long double",
        "data": "synthetic (seeded, gwcat)",
        "config": {"workload": WORKLOAD, "grid": a.grid, "sample_events_per_step": cores},
        "cpu_baseline": {"value": value, "unit": "events/s", "cores": cores, "kind": "oracle",
                         "sample": f"{cores} random events of the catalog per step, one per process"},
        "e2e": {"value": value, "unit": "events/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------ GPU leg
class Clocks:
    """nvidia-smi clock / throttle sampling during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, dev):
        self.dev = dev
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        self.p = None

    def start(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--id={self.dev}", f"--query-gpu={self.Q}",
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except OSError:
            self.p = None

    def stop(self):
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.p.terminate()
        self.p.wait()
        self.f.seek(0)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.f.read().splitlines():
            c = [x.strip() for x in line.split(",")]
            if len(c) < 9:
                continue
            try:
                sm.append(float(c[1]))
                mx.append(float(c[2]))
            except ValueError:
                continue
            for n, v in zip(names, c[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        os.unlink(self.f.name)
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": float(max(mx)) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def flops_per_point(n_site: int, n_ifo: int, precision: str) -> float:
    """Arithmetic of the fused Fisher kernel per grid point (P = 11, rotation on),
    counted from its straight-line formulas, one FMA = 2 flops.

    FP64 path (all FP64): basis powers 8, f/w 4, d Psi/d Mc 19, d Psi/d eta 20,
    slots 9/10 14, tau* and two derivatives 48, PSD weight with reciprocal and
    square root 35, recurrences 4; per site: Earth-angle sincos ~40, double
    angle 5, JKS/Doppler/phase combinations ~95; per virtual interferometer:
    patterns 38, tangents 46, sigma scaling 4, |Q|^2 3, 66-pair Gram update 265.
    Mixed path (FP32 pipe): double-float basis 80; compensated (Dot2) dot
    products with double-float coefficients, 13 flops per term and lane (the
    product error and the addend's roundoff folded into one FMA): d Psi/d Mc with
    d Psi/d eta (two lanes, 11 terms) 276, slots 9/10 (two lanes, 4 terms) 94,
    tau* (one lane, 8 terms, times v^-3) 111, d tau*/d Mc with d tau*/d eta (two
    lanes, 8 terms) 200; f 12, recurrences 41, PSD weight 23; per site 122
    (double-float Earth angle 44, sincosf ~20, JKS/Doppler ~58); per virtual
    interferometer 1343 (patterns 38, tangents 56, scaling 4, 69 compensated
    accumulations of 18 flops: product, two-sum of the high parts, one FMA for
    the product error and roundoff, compensation)."""
    if precision == "mixed":
        shared = 80 + 276 + 94 + 111 + 200 + 12 + 41 + 23
        return shared + 122 * n_site + 1343 * n_ifo
    shared = 8 + 4 + 19 + 20 + 14 + 48 + 35 + 4
    return shared + 140 * n_site + 356 * n_ifo


def shard_seed(rank: int) -> int:
    """Seed of rank's catalog shard: every rank owns its own full-size shard
    (weak scaling; events are independent, nothing is exchanged)."""
    return gwcat.SEED_BASE + 3 + 1000 * rank


def aggregate(times_ms, n_events: int, steps: int, world: int, dist=None, device="cpu"):
    """Max over ranks of each timed quantity (ms) and the whole-job rates:
    events/s = world * n_events * steps / max_time."""
    import torch
    t = torch.tensor([float(x) for x in times_ms], dtype=torch.float64, device=device)
    if world > 1 and dist is not None:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    t = t.tolist()
    rates = [world * n_events * steps / (x * 1e-3) for x in t]
    return t, rates


def sum_over_ranks(t, world: int, dist=None):
    """Whole-job value of a per-shard partial sum, in place: the log-det
    gradient is a sum over events, so the ranks' gradients over their shards
    add up (all-reduce SUM, 8 bytes per detector).  A no-op on one rank."""
    if world > 1 and dist is not None:
        dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return t


def run_ours(a):
    import torch
    import torch.distributed as dist

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl", init_method="env://")
    torch.cuda.set_device(local)
    import paper_2207_06910_gb300 as gw

    prec = gw.GW_MIXED if a.precision == "mixed" else gw.GW_FP64
    gated = a.workload == "c3-gated"
    cfg = "c3" if gated else a.workload
    if gated:
        a.eager = True      # the gate reads its count back: no single-graph step
    # weak scaling: every rank owns its own 1e5-event shard (seed offset by rank)
    raw = gwcat.draw(cfg, a.events, seed=shard_seed(rank), grid=a.grid)
    n = len(raw["m1"])
    rule = raw["npts_rule"]
    det, psd, rot = gwcat.network(cfg)
    net = gw.Network(det, psd, rot)
    n_arms = sum(1 if int(r[4]) == 0 else 3 for r in det)
    keys = ("m1", "m2", "chi1", "chi2", "lam1", "lam2", "dL_Mpc", "tcoal", "fmin",
            "theta", "phi", "iota", "psi", "Phic")
    host = {k: torch.as_tensor(np.ascontiguousarray(raw[k], np.float64)).pin_memory() for k in keys}
    host["zflag"] = torch.as_tensor(np.ascontiguousarray(raw["zflag"], np.uint8)).pin_memory()
    host["pset"] = torch.as_tensor(np.ascontiguousarray(raw["pset"], np.int8)).pin_memory()
    if rule[0] == "given":
        host["npts"] = torch.as_tensor(np.ascontiguousarray(raw["npts"], np.int32)).pin_memory()
    if gated:
        masks = gwcat.draw_arm_masks(n, n_arms, GATE_DUTY, seed=shard_seed(rank) + 7)
        host["arm_mask"] = torch.as_tensor(masks.view(np.int32)).pin_memory()
    dev = {k: v.cuda() for k, v in host.items()}
    stream = torch.cuda.current_stream()
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    grad_up = torch.ones(n, dtype=torch.float64, device="cuda")
    ctx = gw.context()
    lib = gw.load_library()

    def prepare(d):
        return gw_prepare_dev(gw, d, rule, n)

    with_logdet = a.workload == "c4"
    # the orientation gradient the c4 study asks for: the L-shaped detectors
    # (network rows of shape 0); the triangle's entry is not formed
    l_mask = sum(1 << k for k, r in enumerate(net.det_rows) if int(r[4]) == 0)

    def gate(d):
        """Prepared catalog of the step's Fisher pass: every event, or (gated
        workload) the events passing the SNR gate, with their arm masks."""
        cat = prepare(d)
        if not gated:
            return cat
        cat = cat.with_arm_mask(d["arm_mask"])
        snr_all, _ = gw.gw_snr(cat, net, prec)
        return cat.select(gw.gw_select_snr(snr_all, GATE_SNR))

    def step(d):
        cat = gate(d)
        F, snr, st, g = gw.gw_fisher(cat, net, N_PAR, prec, grad_snr=grad_up[:cat.n])
        cov, cond, err, sti = gw.gw_fisher_inverse(F, N_PAR)
        gg = None
        if with_logdet:
            gg = gw.gw_logdet_vjp_detangles(cat, net, N_PAR, cov, gw.GW_FP64, det_mask=l_mask)
        return cat, F, snr, cov, cond, g, st, gg

    # prepare 1; Fisher 7 (event setup, scan 3, point loop, finish, SNR VJP);
    # inversion 1; log-det VJP 6; gated: SNR pass 6 and gate 5
    launches_per_step = 1 + 7 + 1 + (6 if with_logdet else 0) + (11 if gated else 0)
    for _ in range(a.warmup):
        step(dev)
    torch.cuda.synchronize()
    # sanity of the timed configuration: no event flagged by the point loop
    cat, F, snr, cov, cond, g, st, gg = step(dev)
    torch.cuda.synchronize()
    assert int((st != 0).sum()) == 0, "events flagged in the benchmark catalog"
    n_sel = cat.n
    if gated:
        sel_rows = cat.sel
        n_points_all = int(cat.npts.to(torch.int64).sum().item())
        n_points = int(cat.npts[sel_rows].to(torch.int64).sum().item())
    else:
        n_points = n_points_all = int(cat.npts.to(torch.int64).sum().item())

    # ---- reserve the workspace (asynchronous calls) and capture the step
    gw.gw_reserve(n, gw.work_items(cat.npts), net.n_det)
    for _ in range(2):
        step(dev)
    torch.cuda.synchronize()
    graph, gout = None, None
    if not a.eager:
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(graph):
            gout = step(dev)
        graph.replay()
        torch.cuda.synchronize()
        assert int((gout[6] != 0).sum()) == 0 and torch.allclose(gout[2], snr, rtol=1e-12)

    def run_step():
        out = gout
        if graph is not None:
            graph.replay()
        else:
            out = step(dev)
        if with_logdet:   # the job's gradient: sum of the ranks' shard gradients
            sum_over_ranks(out[7], world, dist if world > 1 else None)
        return out

    # Fisher point-kernel duration: a few eager Fisher calls with the library's
    # event hooks (read before any later point kernel of the step)
    fisher_ms = []
    gw.gw_set_profiling(True)
    for _ in range(5):
        flush.zero_()
        cat_p = gate(dev)
        gw.gw_fisher(cat_p, net, N_PAR, prec, grad_snr=grad_up[:cat_p.n])
        fisher_ms.append(gw.gw_point_kernel_ms())
    gw.gw_set_profiling(False)
    torch.cuda.synchronize()

    # ---- device-resident timed loop
    clk = Clocks(local)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    clk.start()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(a.steps)]
    for i in range(a.steps):
        flush.zero_()
        ev[i][0].record(stream)
        run_step()
        ev[i][1].record(stream)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    clocks = clk.stop()
    step_ms = [s.elapsed_time(e) for s, e in ev]
    total_ms = float(sum(step_ms))

    # ---- end to end: host (pinned) -> device, step, device -> host.  Every step
    # copies its own inputs up and its results down; the copies run on a copy
    # stream, so the inputs of step i+1 go up and the results of step i come
    # down while the GPU computes.  Two input sets (and, with graphs, two
    # captured step graphs) alternate; one pair of events brackets all steps,
    # including their L2 flushes.
    dev2 = {k: v.clone() for k, v in dev.items()}
    bufs, graphs, gouts = [dev, dev2], [graph, None], [gout, None]
    if graph is not None:
        graph2 = torch.cuda.CUDAGraph()
        with torch.cuda.graph(graph2):
            gouts[1] = step(dev2)
        graph2.replay()
        torch.cuda.synchronize()
        graphs[1] = graph2

    def run_on(b):
        out = gouts[b]
        if graphs[b] is not None:
            graphs[b].replay()
        else:
            out = step(bufs[b])
        if with_logdet:
            sum_over_ranks(out[7], world, dist if world > 1 else None)
        return out

    outs_host = {"snr": torch.empty(n_sel, dtype=torch.float64).pin_memory(),
                 "F": torch.empty((N_PAR * (N_PAR + 1) // 2, n_sel), dtype=torch.float64).pin_memory(),
                 "cov": torch.empty((N_PAR * (N_PAR + 1) // 2, n_sel), dtype=torch.float64).pin_memory(),
                 "g": torch.empty((N_PAR, n_sel), dtype=torch.float64).pin_memory()}
    if with_logdet:
        outs_host["gg"] = torch.empty(net.n_det, dtype=torch.float64).pin_memory()
    h2d = sum(v.numel() * v.element_size() for v in host.values())
    d2h = sum(v.numel() * v.element_size() for v in outs_host.values())
    copy = torch.cuda.Stream()
    h2d_ev = [torch.cuda.Event(), torch.cuda.Event()]
    step_ev = [torch.cuda.Event(), torch.cuda.Event()]
    d2h_ev = [torch.cuda.Event(), torch.cuda.Event()]
    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    t0.record(stream)
    copy.wait_event(t0)
    with torch.cuda.stream(copy):
        for k, v in host.items():
            bufs[0][k].copy_(v, non_blocking=True)
        h2d_ev[0].record(copy)
    keep = [None, None]
    for i in range(a.steps):
        b = i % 2
        flush.zero_()
        stream.wait_event(h2d_ev[b])          # this step's inputs are up
        if i >= 2:
            stream.wait_event(d2h_ev[b])      # step i-2's results are down
        out = run_on(b)
        step_ev[b].record(stream)
        with torch.cuda.stream(copy):
            if i + 1 < a.steps:
                if i >= 1:
                    copy.wait_event(step_ev[1 - b])   # step i-1 is done with that set
                for k, v in host.items():
                    bufs[1 - b][k].copy_(v, non_blocking=True)
                h2d_ev[1 - b].record(copy)
            copy.wait_event(step_ev[b])
            cat, F, snr, cov, cond, g, st, gg = out
            res = ((snr, "snr"), (F, "F"), (cov, "cov"), (g, "g"))
            for t, name in res + (((gg, "gg"),) if with_logdet else ()):
                if graphs[b] is None:
                    t.record_stream(copy)
                outs_host[name].copy_(t, non_blocking=True)
            d2h_ev[b].record(copy)
        keep[b] = out
    stream.wait_stream(copy)
    t1.record(stream)
    torch.cuda.synchronize()
    e2e_ms = float(t0.elapsed_time(t1))
    gw.gw_reserve(0, 0, 0)

    (total_ms, e2e_ms, kern_ms), (value, e2e_value, _) = aggregate(
        [total_ms, e2e_ms, float(np.mean(fisher_ms))], n, a.steps, world,
        dist if world > 1 else None, device="cuda")

    if rank == 0:
        n_site = net.n_det
        n_ifo = sum(1 if int(r[4]) == 0 else 2 for r in det)
        if gated:
            # interferometers in use per selected event: a triangle with every arm
            # on is two virtual ones, otherwise one per arm that is on
            sel_np = sel_rows.cpu().numpy()
            m = masks[sel_np].astype(np.int64) & 7
            ifo_e = np.where(m == 7, 2, (m & 1) + ((m >> 1) & 1) + ((m >> 2) & 1))
            pts_e = cat.npts[sel_rows].cpu().numpy().astype(np.float64)
            flops = float(np.sum(pts_e * np.array([flops_per_point(n_site, int(k), a.precision)
                                                   for k in ifo_e])))
        else:
            flops = flops_per_point(n_site, n_ifo, a.precision) * n_points
        sm_mhz = clocks.get("sm_mhz") or 2070.0
        per_clk = FFMA_PER_CLK_SM if a.precision == "mixed" else DFMA_PER_CLK_SM
        peak = SM_COUNT * per_clk * 2 * sm_mhz * 1e6 / 1e12       # TFLOP/s at the sampled clock
        achieved = flops / (kern_ms * 1e-3) / 1e12
        cpu = None
        if not a.no_cpu_baseline:
            cores = os.cpu_count() or 1
            v, done, el = oracle_timing(raw, 10 ** 9, cores, budget_s=20.0)
            cpu = {"value": v, "unit": "events/s", "cores": cores, "kind": "oracle",
                   "sample": f"{done} random events of this catalog in {el:.1f} s "
                             f"(prepare + SNR + Fisher + inversion + SNR gradient), "
                             f"one event per process on {cores} host cores"}
        line = {
            "metric": METRIC, "value": value, "unit": "events/s", "n_gpus": world,
            "steps": a.steps, "warmup": a.warmup, "ms_per_step": total_ms / a.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32+f64 (mixed)" if a.precision == "mixed" else "f64",
            "data": "synthetic (seeded, gwcat)",
            "config": {"workload": {"c3": WORKLOAD, "c4": WORKLOAD_C4,
                                    "c3-gated": WORKLOAD_GATED}[a.workload],
                       "n_events_per_gpu": n, "grid": a.grid,
                       "points_per_step": n_points + (n_points_all if gated else 0),
                       "precision": a.precision, "n_par": N_PAR,
                       "step": ("prepare + SNR pass + gate + " if gated else "prepare + ")
                               + "SNR/Fisher with fused SNR VJP + Cholesky inversion"
                               + (" + log-det VJP (FP64) over the two L detectors' orientations"
                                  if with_logdet else ""),
                       **({"selected_events": n_sel, "fisher_points": n_points}
                          if gated else {}),
                       "l2": "flushed before every timed step (256 MiB write)",
                       "launch": "eager calls" if a.eager else "one CUDA graph replay per step",
                       "parallelism": f"event shards, {world} GPU(s), " + (
                           "log-det gradient all-reduced (SUM) per step" if with_logdet
                           and world > 1 else "no collective")},
            "clocks": clocks,
            "e2e": {"value": e2e_value, "unit": "events/s", "h2d_bytes_per_step": h2d,
                    "d2h_bytes_per_step": d2h,
                    "copies": "pinned host buffers, on a copy stream overlapping the "
                              "previous/next step's compute"},
            "gpu_launches": launches_per_step * a.steps,
            "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                         "frac": achieved / peak,
                         "traffic": DRAM_BYTES_PER_POINT[a.precision] * n_points
                         if a.grid == "literal" else None,
                         "kernel": f"k_points_{'mixed' if a.precision == 'mixed' else 'fp64'} (Fisher)",
                         "kernel_ms": kern_ms,
                         "flops_per_point": flops_per_point(n_site, n_ifo, a.precision),
                         "peak_basis": (f"{'FP32' if a.precision == 'mixed' else 'FP64'} pipe: "
                                        f"{SM_COUNT} SMs x {per_clk} FMA/clk x 2 flops x "
                                        f"{sm_mhz:.0f} MHz (median sampled SM clock)")},
            "cpu_baseline": cpu,
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def gw_prepare_dev(gw, d, rule, n):
    """gw_prepare_catalog on device-resident raw arrays (no host transfer)."""
    import ctypes
    import torch
    lib = gw.load_library()
    ctx = gw.context()
    dev = d["m1"].device
    out = {k: torch.empty(n, dtype=torch.float64, device=dev) for k in
           ("Mc", "eta", "dL", "chi1z", "chi2z", "LamT", "dLamT", "tc", "fmax")}
    npts = torch.empty(n, dtype=torch.int32, device=dev)
    fixed, per, lo, hi, given = 0, 0.0, 0, 0, None
    if rule[0] == "fixed":
        fixed = int(rule[1])
    elif rule[0] == "efold":
        per, lo, hi = float(rule[1]), int(rule[2]), int(rule[3])
    else:
        given = d["npts"]
    P = gw._ptr
    st = lib.gw_prepare_catalog(ctx, n, P(d["m1"]), P(d["m2"]), P(d["chi1"]), P(d["chi2"]),
                                P(d["lam1"]), P(d["lam2"]), P(d["dL_Mpc"]), P(d["zflag"]),
                                P(d["tcoal"]), P(d["fmin"]), P(given), fixed, per, lo, hi,
                                P(out["Mc"]), P(out["eta"]), P(out["dL"]), P(out["chi1z"]),
                                P(out["chi2z"]), P(out["LamT"]), P(out["dLamT"]), P(out["tc"]),
                                P(out["fmax"]), P(npts), gw._stream())
    gw._check(st, ctx)
    t = dict(out)
    for k in ("theta", "phi", "iota", "psi", "Phic"):
        t[k] = d[k]
    return gw.Catalog(t, d["pset"], d["fmin"], out["fmax"], npts)


def main():
    a = parse()
    if a.impl == "reference":
        run_reference(a)
    else:
        run_ours(a)


if __name__ == "__main__":
    main()
