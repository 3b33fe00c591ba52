"""Benchmark of the Fisher-forecast hot path on GB300.

One step = one pass of the whole hot path over a catalog: catalog preparation,
network SNR + 11x11 Fisher matrix with the fused SNR vector-Jacobian product,
batched FP64 Cholesky inversion with the conditioning check, and, in the mixed
path, the precision refinement (events whose mixed inversion fails or whose
condition number exceeds 1e7 are recomputed in FP64).  The default workload is
the 1e5-event uneven catalog (70 % BBH / 30 % tidal BNS, rotating triangle,
per-event log grid from 2 Hz to f_ISCO).  The headline is the routed step
(gw_fisher_routed: the precision chosen per event -- the double-float path,
every per-point quantity in double-float arithmetic on the FP32 pipe and the
Fisher matrix the exact Gram of the tangents on the tensor cores, for the BBH,
whose two spins make their Fisher matrices ill-conditioned; the mixed path for
the rest, with a double-float recomputation of any event whose condition
number exceeds 1e7); the FP64 path is timed on the same catalog as the second
arm, and the stored oracle results of 1000 stratified events give the error of
the FP64, mixed (with refinement), double-float and routed paths.
Inputs are resident in HBM before the timed region; L2 is flushed (256 MiB
write) before every timed step.

  python bench.py [--gpus N --steps K --warmup W] [--precision routed|dfloat|mixed|fp64]
                  [--grid literal|stress] [--workload c3|c4|c3-gated]
                  [--impl ours|reference]

With N > 1 (torchrun) one catalog of N x 1e5 events is split into contiguous
ranges of equal cost (grid points x interferometers), one per rank.
--impl reference times the CPU oracle (oracle/) on a bounded sample of the same
workload on the host cores (the paper's method has no GPU implementation).
Prints one JSON line.
"""
from __future__ import annotations

import argparse
import json
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
NPK = N_PAR * (N_PAR + 1) // 2
# nominal pipe widths per SM and clock (the peaks' unit counts): FP32 lanes x 2 for
# the packed FP32x2 FMA the mixed kernel issues; FP64 FMA units
FP32_FMA_PER_CLK_SM = 256
FP64_FMA_PER_CLK_SM = 2
# DRAM bytes (read + write) per grid point of the Fisher point kernels, from one
# ncu capture of the 2e4-event c3 catalog (4,376,070 points; profiles/
# k_points_*_fisher_c3.md), scaled by points to a full launch
DRAM_BYTES_PER_POINT = {"mixed": (23.10528e6 + 11.52e3) / 4376070,
                        "fp64": (19.284224e6 + 91.136e3) / 4376070,
                        "dfloat_tc": (20.592128e6 + 70.656e3) / 4376070}
# executed warp instructions per grid point of the double-float tensor-core
# kernel (the same capture, profiles/k_fisher_tc_dfloat_c3.md): the kernel is
# latency-bound, so its issue rate against the schedulers' peak (4 per SM and
# clock) is the roofline that explains its time
ISSUE_WARP_INSTR_PER_POINT = {"dfloat_tc": 1.028082637e9 / 4376070}
GOLDEN = os.path.join(ROOT, "tests", "golden", "parity_oracle.npz")


def _measured_peaks() -> dict:
    """The measured copy bandwidth and bf16 GEMM rates of this machine's GPUs."""
    try:
        with open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


MEASURED = _measured_peaks()


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=40)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--precision", choices=["routed", "mixed", "fp64", "dfloat"],
                    default="routed",
                    help="routed: precision chosen per event (gw_fisher_routed: double-float "
                         "for the BBH, whose two spins make them ill-conditioned, mixed for the "
                         "rest with a double-float recomputation of any ill-conditioned one); "
                         "dfloat: double-float tangents on the FP32 pipe with the exact "
                         "tensor-core Gram (FP64-class results in one pass); mixed: FP32 "
                         "tangents with compensated sums and FP64 refinement of the "
                         "ill-conditioned events; fp64: every operation in FP64")
    ap.add_argument("--grid", choices=["literal", "stress"], default="literal")
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--events", type=int, default=None, help="events per GPU")
    ap.add_argument("--workload", choices=["c3", "c4", "c3-gated"], default="c3",
                    help="c3: 1e5 events on the triangle (headline); c4: 1e6 events on five "
                         "interferometers, the step adding the log-det VJP over the two "
                         "L detectors' orientations; c3-gated: c3 with duty-factor arm masks, "
                         "an SNR pass and the SNR > 12 gate before the Fisher pass")
    ap.add_argument("--refine-cond", type=float, default=1e7,
                    help="condition number above which mixed events are recomputed in FP64")
    ap.add_argument("--no-fp64-arm", action="store_true",
                    help="do not time the FP64 path beside the mixed one")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--psd", choices=["power", "table"], default="power",
                    help="noise curves as the configuration's power sums, or as tables of "
                         "2000 log-spaced (f, S_n) points read by log-log interpolation "
                         "(Sec. 3.1 psd_path)")
    ap.add_argument("--fp64-gram", choices=["tensor", "pipe"], default="pipe",
                    help="Gram of the FP64 Fisher pass on the tensor cores (exact digit "
                         "products) or on the FP64 pipe")
    ap.add_argument("--autotune", action="store_true",
                    help="time the six Fisher-pass tiles on this catalog (per precision and "
                         "grid-length class, cached in a JSON file) before the arms")
    ap.add_argument("--eager", action="store_true",
                    help="launch the step call by call instead of replaying a CUDA graph")
    return ap.parse_args()


def bench_network(cfg: str, kind: str):
    """Detector table, PSD rows, rotation flag and PSD tables (None for power
    sums) of a workload."""
    if kind == "table":
        return gwcat.network_tabulated(cfg)
    det, psd, rot = gwcat.network(cfg)
    return det, psd, rot, None


# ------------------------------------------------------------------ oracle leg
def _oracle_event_step(args):
    """Every row of the step for one event, on the CPU oracle; returns the
    event's packed Fisher matrix, SNR, covariance and condition number."""
    import oracle
    raw, rule, det, psd, rot, tables = args
    if tables:
        oracle.set_psd_tables(tables)
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
    C, kappa, eps, sti = oracle.invert(F)
    oracle.snr_grad(cat, det, psd, rot, N_PAR)
    iu = np.triu_indices(N_PAR)
    return F[0][iu], float(s[0]), C[0][iu], float(kappa[0]), int(sti[0])


def _sample(raw, idx):
    out = {}
    for k, v in raw.items():
        if isinstance(v, np.ndarray) and v.shape[:1] == (len(raw["m1"]),):
            out[k] = v[idx]
    return out


def oracle_timing(raw, cfg, cores, budget_s=20.0, psd_kind="power"):
    """Time the oracle on a bounded random sample of the workload (spawn
    pool, one event per process); returns the rate and the sampled events'
    rows and oracle results."""
    import multiprocessing as mp
    import oracle
    oracle.build()
    det, psd, rot, tables = bench_network(cfg, psd_kind)
    rule = raw["npts_rule"]
    rng = np.random.default_rng(1)
    rows, res = [], []
    with mp.get_context("spawn").Pool(cores) as pool:
        pool.map(_oracle_event_step, [(_sample(raw, [0]), rule, det, psd, rot, tables)])   # warm
        t0 = time.time()
        while True:
            idx = rng.choice(len(raw["m1"]), cores, replace=False)
            res += pool.map(_oracle_event_step, [(_sample(raw, [i]), rule, det, psd, rot, tables)
                                                 for i in idx])
            rows += list(idx)
            el = time.time() - t0
            if el >= budget_s:
                return len(rows) / el, np.array(rows), res, el


def run_reference(a):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    raw = gwcat.draw("c3", a.events, grid=a.grid)
    cores = os.cpu_count() or 1
    det, psd, rot, tables = bench_network("c3", a.psd)
    import multiprocessing as mp
    import oracle
    oracle.build()
    rng = np.random.default_rng(2)
    times = []
    with mp.get_context("spawn").Pool(cores) as pool:
        for i in range(a.warmup + a.steps):
            idx = rng.choice(len(raw["m1"]), cores, replace=False)
            tasks = [(_sample(raw, [j]), raw["npts_rule"], det, psd, rot, tables) for j in idx]
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
    """Arithmetic per grid point of the fused Fisher kernel (P = 11, rotation on),
    counted from its straight-line formulas, one FMA = 2 flops.

    "fp64": the method's work, every operation once in FP64 (the roofline's
    algorithmic count for both paths): basis powers 8, f/w 4, d Psi/d Mc 19,
    d Psi/d eta 20, slots 9/10 14, tau* and two derivatives 48, PSD weight with
    reciprocal and square root 35, recurrences 4; per site: Earth-angle sincos
    ~40, double angle 5, JKS/Doppler/phase combinations ~95; per virtual
    interferometer: patterns 38, tangents 46, sigma scaling 4, |Q|^2 3, 66-pair
    Gram update 265.
    "mixed": what the mixed kernel executes on the FP32 pipe, compensations
    included: double-float basis 80; compensated (Dot2) dot products with
    double-float coefficients, 13 flops per term and lane: d Psi/d Mc with
    d Psi/d eta (two lanes, 11 terms) 276, slots 9/10 (two lanes, 4 terms) 94,
    tau* (one lane, 8 terms, times v^-3) 111, d tau*/d Mc with d tau*/d eta (two
    lanes, 8 terms) 200; f 12, recurrences 41, PSD weight 23; per site 122
    (double-float Earth angle 44, sincosf ~20, JKS/Doppler ~58); per virtual
    interferometer 1343 (patterns 38, tangents 56, scaling 4, 69 compensated
    accumulations of 18 flops)."""
    if precision == "mixed":
        shared = 80 + 276 + 94 + 111 + 200 + 12 + 41 + 23
        return shared + 122 * n_site + 1343 * n_ifo
    shared = 8 + 4 + 19 + 20 + 14 + 48 + 35 + 4
    return shared + 140 * n_site + 356 * n_ifo


def fp64_gram_flops_per_point(n_ifo: int) -> float:
    """The Gram update's share of the FP64 count above: 66 pairs x 2 products
    (real and imaginary parts) x 2 flops per virtual interferometer, plus the
    |Q|^2 sum (3 flops) that the Gram's (Phic, Phic) entry replaces."""
    return 265.0 * n_ifo


def tc_digit_flops_per_point(n_ifo: int, n_par: int = 11) -> float:
    """Tensor-core work of the exact Gram per grid point: 2 K rows (real and
    imaginary parts) per virtual interferometer, each entering one M = 128 by
    N = 8 n_par (padded to 16) digit product, 2 flops per multiply-add."""
    n = ((8 * n_par + 15) // 16) * 16
    return 2.0 * n_ifo * 128 * n * 2


def aggregate(times_ms, n_events: int, steps: int, world: int, dist=None, device="cpu"):
    """Max over ranks of each timed quantity (ms) and the whole-job rates:
    events/s = n_events (all ranks) * steps / max_time."""
    import torch
    t = torch.tensor([float(x) for x in times_ms], dtype=torch.float64, device=device)
    if world > 1 and dist is not None:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    t = t.tolist()
    rates = [n_events * steps / (x * 1e-3) if x > 0 else 0.0 for x in t]
    return t, rates


def gw_prepare_dev(gw, d, rule, n):
    """gw_prepare_catalog on device-resident raw arrays (no host transfer)."""
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


KEYS = ("m1", "m2", "chi1", "chi2", "lam1", "lam2", "dL_Mpc", "tcoal", "fmin",
        "theta", "phi", "iota", "psi", "Phic")


def golden_error(gw, refine_cond):
    """sqrt(diag C) error of the mixed path (with the FP64 refinement), the
    double-float path and the FP64 path against the stored oracle results of 1000 stratified events
    of the c3 catalog (tests/golden/parity_oracle.npz), per condition-number
    decade; worst = max of rel / max(1e-3, 1e-15 kappa) (pass: <= 1)."""
    import torch
    if not os.path.exists(GOLDEN):
        return None
    z = np.load(GOLDEN)
    if "c3lit_cov" not in z:
        return None
    det, psd, rot = gwcat.network("c3")
    net = gw.Network(det, psd, rot)
    cat = gw.Catalog.from_numpy(z["c3lit_ev"], z["c3lit_pset"], z["c3lit_fmin"], z["c3lit_fmax"],
                                z["c3lit_npts"])
    diag = [i * N_PAR - i * (i - 1) // 2 for i in range(N_PAR)]     # packed (i, i)
    so = np.sqrt(np.abs(z["c3lit_cov"][:, diag]))
    kappa = z["c3lit_kappa"]
    ok = (z["c3lit_inv_status"] & 33) == 0
    out = {"events": int(len(kappa)), "oracle_flagged": int((~ok).sum())}
    for name, prec in (("mixed_refined", gw.GW_MIXED), ("dfloat", gw.GW_DFLOAT),
                       ("fp64", gw.GW_FP64), ("routed", None)):
        if prec is None:
            # double-float for the BBH (pset 1), mixed + FP64 refinement for the rest
            r = gw.gw_fisher_routed(cat, net, N_PAR, 1 << 1, cond_th=refine_cond)
            inv, nref = r[3:7], r[-1]
        else:
            F, snr, st = gw.gw_fisher(cat, net, N_PAR, prec)
            inv = gw.gw_fisher_inverse(F, N_PAR)
            nref = gw.gw_fisher_refine(cat, net, N_PAR, F, snr, st, inv, cond_th=refine_cond) \
                if prec == gw.GW_MIXED else 0
        torch.cuda.synchronize()
        C = inv[0].cpu().numpy()
        sg = np.sqrt(np.abs(C[diag].T))
        with np.errstate(all="ignore"):
            rel = np.max(np.abs(sg / so - 1), axis=1)
        rel_ok = rel[ok]
        worst = float(np.nanmax(rel_ok / np.maximum(1e-3, 1e-15 * kappa[ok])))
        dec = np.floor(np.log10(kappa[ok])).astype(int)
        table = {f"1e{d}": [int((dec == d).sum()), round(float(np.mean(rel_ok[dec == d] <= 1e-3)), 3),
                            float(np.max(rel_ok[dec == d]))]
                 for d in range(dec.min(), dec.max() + 1) if (dec == d).any()}
        out[name] = {"worst_over_bound": worst, "max_rel_kappa_le_1e12":
                     float(np.max(rel_ok[kappa[ok] <= 1e12])),
                     "pass_1e-3_frac": float(np.mean(rel_ok <= 1e-3)),
                     "refined_frac": nref / len(kappa),
                     "per_decade_[events,pass_1e-3,max_rel]": table}
    return out


def tune_tiles(gw, a, cat, net, order, prec):
    """Autotuned Fisher-pass tiles of the arms: each precision on the step's
    catalog and, for the mixed arm, the FP64 pass on the events its
    refinement selects.  Returns, per pass, the chosen tile and (when timed
    here rather than read from the cache) the time of every tile, the fixed
    default 8x2 among them."""
    import torch
    from paper_2207_06910_gb300 import autotune

    def entry(e):
        return {"tile": f"{e['group']}x{e['blocks_per_sm']}", "cached": e["cached"],
                "length_class": gw.LENGTH_CLASSES[e["length_class"]],
                **({"ms": e["ms"]} if "ms" in e else {})}
    out = {}
    for p in order:
        if p < 0:
            continue        # the routed step: its passes are tuned as themselves
        if p == gw.GW_DFLOAT:
            continue     # one fixed shape (the tensor-core kernel)
        out["mixed" if p == gw.GW_MIXED else "fp64"] = entry(autotune.tune(cat, net, N_PAR, p))
    if prec == gw.GW_MIXED:
        F, snr, st = gw.gw_fisher(cat, net, N_PAR, gw.GW_MIXED)
        inv = gw.gw_fisher_inverse(F, N_PAR)
        flag = torch.zeros(cat.n, dtype=torch.uint8, device="cuda")
        gw.gw_fisher_refine(cat, net, N_PAR, F, snr, st, inv, cond_th=a.refine_cond, refined=flag)
        idx = torch.nonzero(flag).flatten()
        if idx.numel() > 0:
            out["fp64 refinement"] = entry(autotune.tune(cat.select(idx), net, N_PAR, gw.GW_FP64))
    return out


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
    from paper_2207_06910_gb300 import shard

    ROUTED = -1          # the routed step (not a library precision)
    prec = {"mixed": gw.GW_MIXED, "fp64": gw.GW_FP64, "dfloat": gw.GW_DFLOAT,
            "routed": ROUTED}[a.precision]
    routed_counts = {"dfloat": 0, "recomputed": 0}
    gw.gw_set_fp64_gram(a.fp64_gram == "tensor")
    gated = a.workload == "c3-gated"
    cfg = "c3" if gated else a.workload
    if gated:
        a.eager = True      # the gate reads its count back: no single-graph step
    with_logdet = a.workload == "c4"
    n_per_gpu = a.events or gwcat.SIZES[cfg]
    det, psd, rot, tables = bench_network(cfg, a.psd)
    net = gw.Network(det, psd, rot, tables)
    n_arms = sum(1 if int(r[4]) == 0 else 3 for r in det)
    n_site = net.n_det
    n_ifo = sum(1 if int(r[4]) == 0 else 2 for r in det)

    # ---- one catalog over all ranks, split into contiguous ranges of equal cost
    raw_all = gwcat.draw(cfg, n_per_gpu * world, grid=a.grid)
    rule = raw_all["npts_rule"]
    dev_all = {k: torch.as_tensor(np.ascontiguousarray(raw_all[k], np.float64), device="cuda")
               for k in KEYS}
    dev_all["zflag"] = torch.as_tensor(np.ascontiguousarray(raw_all["zflag"], np.uint8), device="cuda")
    dev_all["pset"] = torch.as_tensor(np.ascontiguousarray(raw_all["pset"], np.int8), device="cuda")
    if rule[0] == "given":
        dev_all["npts"] = torch.as_tensor(np.ascontiguousarray(raw_all["npts"], np.int32), device="cuda")
    npts_all = gw_prepare_dev(gw, dev_all, rule, len(raw_all["m1"])).npts.cpu().numpy()
    del dev_all
    bounds = shard.partition(shard.event_cost(npts_all, n_ifo), world)
    lo_r, hi_r = int(bounds[rank]), int(bounds[rank + 1])
    raw = {k: (v[lo_r:hi_r] if isinstance(v, np.ndarray) and v.shape[:1] == (len(raw_all["m1"]),)
               else v) for k, v in raw_all.items()}
    n = hi_r - lo_r
    n_total = len(raw_all["m1"])

    host = {k: torch.as_tensor(np.ascontiguousarray(raw[k], np.float64)).pin_memory() for k in KEYS}
    host["zflag"] = torch.as_tensor(np.ascontiguousarray(raw["zflag"], np.uint8)).pin_memory()
    host["pset"] = torch.as_tensor(np.ascontiguousarray(raw["pset"], np.int8)).pin_memory()
    if rule[0] == "given":
        host["npts"] = torch.as_tensor(np.ascontiguousarray(raw["npts"], np.int32)).pin_memory()
    masks = None
    if gated:
        masks = gwcat.draw_arm_masks(n_total, n_arms, GATE_DUTY)[lo_r:hi_r]
        host["arm_mask"] = torch.as_tensor(masks.view(np.int32)).pin_memory()
    dev = {k: v.cuda() for k, v in host.items()}
    stream = torch.cuda.current_stream()
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    grad_up = torch.ones(n, dtype=torch.float64, device="cuda")
    # the orientation gradient the c4 study asks for: the L-shaped detectors
    l_mask = sum(1 << k for k, r in enumerate(net.det_rows) if int(r[4]) == 0)

    def item_points(p):
        """Points per work item of the Fisher pass at precision p (the
        tensor-core pass takes shorter items)."""
        tc = p in (gw.GW_DFLOAT, ROUTED) or (p == gw.GW_FP64 and a.fp64_gram == "tensor")
        return gw.TC_ITEM_POINTS if (tc and n_ifo <= 2) else gw.ITEM_POINTS

    def gate(d):
        """Prepared catalog of the step's Fisher pass: every event, or (gated
        workload) the events passing the SNR gate, with their arm masks."""
        cat = gw_prepare_dev(gw, d, rule, n)
        if not gated:
            return cat
        cat = cat.with_arm_mask(d["arm_mask"])
        snr_all, _ = gw.gw_snr(cat, net, gw.GW_MIXED if prec == gw.GW_MIXED else gw.GW_FP64)
        return cat.select(gw.gw_select_snr(snr_all, GATE_SNR))

    def forward(d, p):
        """The capturable part of the step: prepare, Fisher with fused SNR VJP,
        inversion (and the gate for the gated workload); the routed step
        captures only the preparation."""
        cat = gate(d)
        if p == ROUTED:
            return [cat, None, None, None, None, None]
        F, snr, st, g = gw.gw_fisher(cat, net, N_PAR, p, grad_snr=grad_up[:cat.n])
        inv = gw.gw_fisher_inverse(F, N_PAR)
        return [cat, F, snr, st, g, inv]

    def finish(out, p):
        """The rest of the step: the routed Fisher pass and inversion (reads back
        its split and count), FP64 refinement of the mixed path's events (reads
        back its count), log-det VJP (c4) and its sum over ranks."""
        nref = 0
        if p == ROUTED:
            cr = out[0]
            r = gw.gw_fisher_routed(cr, net, N_PAR, 1 << 1, grad_snr=grad_up[:cr.n],
                                    cond_th=a.refine_cond)
            out[1:6] = [r[0], r[1], r[2], r[7], tuple(r[3:7])]
            routed_counts["dfloat"], routed_counts["recomputed"] = r[8], r[9]
            nref = r[9]
        cat, F, snr, st, g, inv = out
        if p == gw.GW_MIXED:
            nref = gw.gw_fisher_refine(cat, net, N_PAR, F, snr, st, inv, grad_snr=grad_up[:cat.n],
                                       grad_params=g, cond_th=a.refine_cond)
        gg = None
        if with_logdet:
            gg = gw.gw_logdet_vjp_detangles(cat, net, N_PAR, inv[0], gw.GW_FP64, det_mask=l_mask)
            shard.sum_partials(gg, world, dist if world > 1 else None)
        return nref, gg

    def make_arm(p, bufs):
        """Warm, reserve, capture; returns run(b) -> (outputs, n_refined)."""
        for _ in range(a.warmup):
            finish(forward(bufs[0], p), p)
        torch.cuda.synchronize()
        cat0 = forward(bufs[0], p)[0]
        gw.gw_reserve(n, gw.work_items(cat0.npts if cat0.sel is None else cat0.npts[cat0.sel],
                                       item_points(p)), net.n_det)
        for _ in range(2):
            finish(forward(bufs[0], p), p)
        torch.cuda.synchronize()
        graphs, outs = [None] * len(bufs), [None] * len(bufs)
        if not a.eager:
            for b, d in enumerate(bufs):
                graphs[b] = torch.cuda.CUDAGraph()
                with torch.cuda.graph(graphs[b]):
                    outs[b] = forward(d, p)
                graphs[b].replay()
            torch.cuda.synchronize()

        def run(b):
            if graphs[b] is not None:
                graphs[b].replay()
                out = outs[b]
            else:
                out = forward(bufs[b], p)
            nref, gg = finish(out, p)
            return out, nref, gg
        return run

    def timed_loop(run):
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
              for _ in range(a.steps)]
        nref = 0
        for i in range(a.steps):
            flush.zero_()
            ev[i][0].record(stream)
            out, nref, gg = run(0)
            ev[i][1].record(stream)
        torch.cuda.synchronize()
        return float(sum(s.elapsed_time(e) for s, e in ev)), out, nref

    def point_kernel_ms(p, refine):
        """Point-loop kernel durations from the library's CUDA events on the
        launching stream: the Fisher pass, and (mixed) the refinement's FP64 pass."""
        ms, ms_ref = [], []
        pts_ref = 0
        gw.gw_set_profiling(True)
        if p == ROUTED:
            # the routed step's dominant kernel: the double-float pass over its
            # BBH (pset 1) events, timed on its own (measurement only)
            cr = gate(dev)
            ps = cr.pset[cr.sel] if cr.sel is not None else cr.pset
            sub = cr.select(torch.nonzero(ps == 1).flatten())
            routed_counts["points_df"] = int(sub.npts[sub.sel].to(torch.int64).sum().item())
            for _ in range(4):
                flush.zero_()
                gw.gw_fisher(sub, net, N_PAR, gw.GW_DFLOAT, grad_snr=grad_up[:sub.n])
                ms.append(gw.gw_point_kernel_ms())
            gw.gw_set_profiling(False)
            torch.cuda.synchronize()
            return float(np.min(ms)), 0.0, 0
        for _ in range(4):
            flush.zero_()
            cat, F, snr, st, g, inv = forward(dev, p)
            ms.append(gw.gw_point_kernel_ms())
            if refine:
                flag = torch.zeros(cat.n, dtype=torch.uint8, device="cuda")
                gw.gw_fisher_refine(cat, net, N_PAR, F, snr, st, inv, grad_snr=grad_up[:cat.n],
                                    grad_params=g, cond_th=a.refine_cond, refined=flag)
                ms_ref.append(gw.gw_point_kernel_ms())
                npts = cat.npts if cat.sel is None else cat.npts[cat.sel]
                pts_ref = int(npts.to(torch.int64)[flag.bool()].sum().item())
        gw.gw_set_profiling(False)
        torch.cuda.synchronize()
        # (the minimum: a first call can include one-time module loading)
        return float(np.min(ms)), (float(np.min(ms_ref)) if ms_ref else 0.0), pts_ref

    # ---- the FP64 arm (same catalog, same launch), then the headline arm
    arms = {}
    order = [prec] if (a.no_fp64_arm or prec == gw.GW_FP64) else [gw.GW_FP64, prec]
    tiles = None
    if a.autotune:
        tiles = tune_tiles(gw, a, gate(dev), net, order, prec)
    dev2 = {k: v.clone() for k, v in dev.items()}
    clocks = None
    for p in order:
        run = make_arm(p, [dev, dev2])
        kern_ms, kern_ref_ms, pts_ref = point_kernel_ms(p, p == gw.GW_MIXED)
        clk = Clocks(local)
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()
        clk.start()
        total_ms, out, nref = timed_loop(run)
        if world > 1:
            dist.barrier()
        c = clk.stop()
        arms[p] = dict(run=run, total_ms=total_ms, out=out, nref=nref, kern_ms=kern_ms,
                       kern_ref_ms=kern_ref_ms, pts_ref=pts_ref, clocks=c)
        if p == prec:
            clocks = c
        gw.gw_reserve(0, 0, 0)
    # ---- the routed step beside the double-float headline (gw_fisher_routed:
    # double-float for the BBH, mixed for the rest with a double-float
    # recomputation of its ill-conditioned events; host synchronisations
    # inside, so launched call by call), same catalog and timing; one GPU
    routed = None
    if prec == gw.GW_DFLOAT and not a.no_fp64_arm and not gated and not with_logdet \
            and n_ifo <= 2 and world == 1:
        def run_routed():
            cr = gate(dev)
            return cr.n, gw.gw_fisher_routed(cr, net, N_PAR, 1 << 1, grad_snr=grad_up[:cr.n],
                                             cond_th=a.refine_cond)
        for _ in range(a.warmup):
            run_routed()
        torch.cuda.synchronize()
        rev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
               for _ in range(a.steps)]
        for i in range(a.steps):
            flush.zero_()
            rev[i][0].record(stream)
            nr, rr = run_routed()
            rev[i][1].record(stream)
        torch.cuda.synchronize()
        r_ms = float(sum(x.elapsed_time(y) for x, y in rev)) / a.steps
        routed = {"value": nr / (r_ms * 1e-3), "unit": "events/s", "ms_per_step": r_ms,
                  "events_dfloat": rr[-2], "events_recomputed": rr[-1],
                  "step": "prepare + gw_fisher_routed (split by parameter set, double-float "
                          "Fisher for the BBH, mixed Fisher + inversion check + double-float "
                          "recomputation of the ill-conditioned others, inversion, fused SNR "
                          "VJP), launched call by call"}
    head = arms[prec]
    cat, F, snr, st, g, inv = head["out"]
    assert int((st != 0).sum()) == 0, "events flagged in the benchmark catalog"
    n_sel = cat.n
    npts_sel = (cat.npts if cat.sel is None else cat.npts[cat.sel]).to(torch.int64)
    n_points = int(npts_sel.sum().item())
    n_points_all = int(cat.npts.to(torch.int64).sum().item())

    # ---- end to end: host (pinned) -> device, step, device -> host.  Every step
    # copies its own inputs up and its results down on a copy stream, so the
    # inputs of step i+1 go up and the results of step i come down while the GPU
    # computes; two input sets (and two captured graphs) alternate.
    gw.gw_reserve(n, gw.work_items(npts_sel, item_points(prec)), net.n_det)
    run = make_arm(prec, [dev, dev2])
    outs_host = {"snr": torch.empty(n_sel, dtype=torch.float64).pin_memory(),
                 "F": torch.empty((NPK, n_sel), dtype=torch.float64).pin_memory(),
                 "cov": torch.empty((NPK, n_sel), dtype=torch.float64).pin_memory(),
                 "g": torch.empty((N_PAR, n_sel), dtype=torch.float64).pin_memory(),
                 "cond": torch.empty(n_sel, dtype=torch.float64).pin_memory(),
                 "inv_err": torch.empty(n_sel, dtype=torch.float64).pin_memory(),
                 "status": torch.empty(n_sel, dtype=torch.int32).pin_memory(),
                 "inv_status": torch.empty(n_sel, dtype=torch.int32).pin_memory()}
    if with_logdet:
        outs_host["gg"] = torch.empty(net.n_det, dtype=torch.float64).pin_memory()
    h2d = sum(v.numel() * v.element_size() for v in host.values())
    d2h = sum(v.numel() * v.element_size() for v in outs_host.values())
    copy = torch.cuda.Stream()
    bufs = [dev, dev2]
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
    for i in range(a.steps):
        b = i % 2
        flush.zero_()
        stream.wait_event(h2d_ev[b])          # this step's inputs are up
        if i >= 2:
            stream.wait_event(d2h_ev[b])      # step i-2's results are down
        out, nref, gg = run(b)
        step_ev[b].record(stream)
        with torch.cuda.stream(copy):
            if i + 1 < a.steps:
                if i >= 1:
                    copy.wait_event(step_ev[1 - b])   # step i-1 is done with that set
                for k, v in host.items():
                    bufs[1 - b][k].copy_(v, non_blocking=True)
                h2d_ev[1 - b].record(copy)
            copy.wait_event(step_ev[b])
            c_, F_, snr_, st_, g_, inv_ = out
            res = [(snr_, "snr"), (F_, "F"), (inv_[0], "cov"), (g_, "g"), (inv_[1], "cond"),
                   (inv_[2], "inv_err"), (st_, "status"), (inv_[3], "inv_status")]
            if with_logdet:
                res.append((gg, "gg"))
            for t, name in res:
                t.record_stream(copy)
                outs_host[name].copy_(t, non_blocking=True)
            d2h_ev[b].record(copy)
    stream.wait_stream(copy)
    t1.record(stream)
    torch.cuda.synchronize()
    e2e_ms = float(t0.elapsed_time(t1))
    gw.gw_reserve(0, 0, 0)

    # ---- whole-job figures: max over ranks of the times
    fp64 = arms.get(gw.GW_FP64)
    times = [head["total_ms"], e2e_ms, head["kern_ms"], head["kern_ref_ms"],
             fp64["total_ms"] if fp64 else 0.0, fp64["kern_ms"] if fp64 else 0.0]
    t, rates = aggregate(times, n_total, a.steps, world, dist if world > 1 else None, device="cuda")
    total_ms, e2e_ms, kern_ms, kern_ref_ms, fp64_ms, fp64_kern_ms = t
    value, e2e_value = rates[0], rates[1]
    nref_t = torch.tensor([float(head["nref"])], dtype=torch.float64, device="cuda")
    if world > 1:
        dist.all_reduce(nref_t)
    n_refined = int(nref_t.item())

    if rank == 0:
        algo_fp = flops_per_point(n_site, n_ifo, "fp64")
        exec_fp = flops_per_point(n_site, n_ifo, a.precision)
        sm_mhz = (clocks or {}).get("sm_mhz") or 2070.0
        sms = torch.cuda.get_device_properties(local).multi_processor_count
        rate64 = gw.gw_fma_rate(True)
        rate32 = gw.gw_fma_rate(False)
        peak32 = sms * FP32_FMA_PER_CLK_SM * 2 * sm_mhz * 1e6 / 1e12
        peak64 = sms * FP64_FMA_PER_CLK_SM * 2 * sm_mhz * 1e6 / 1e12
        refined_frac = n_refined / max(1, n_total)
        # points of one rank's launch of each point kernel
        pts_mixed = n_points if prec == gw.GW_MIXED else 0
        pts_ref = head["pts_ref"] if prec == gw.GW_MIXED else n_points
        kernels = []
        # the FP64 Fisher pass runs the tensor-core Gram kernel for networks of at
        # most two interferometers per point
        tc_on = a.fp64_gram == "tensor" and n_ifo <= 2
        fp64_name = "k_fisher_fp64_tc" if tc_on else "k_points_fp64"
        fp64_pipe_fp = algo_fp - (fp64_gram_flops_per_point(n_ifo) if tc_on else 0.0)
        peak_bf16 = MEASURED.get("bf16_tflops")

        def fp64_entry(label, ms, points):
            k = {"kernel": f"{fp64_name} ({label})", "ms": ms, "points": points, "bound": "alu",
                 "peak": peak64, "executed_flops_per_point": fp64_pipe_fp,
                 "pipe_flops_per_point": fp64_pipe_fp,
                 "peak_basis": f"FP64 pipe: {sms} SMs x {FP64_FMA_PER_CLK_SM} FMA/clk "
                               f"x 2 flops x {sm_mhz:.0f} MHz"}
            if tc_on:
                tfl = tc_digit_flops_per_point(n_ifo, N_PAR)
                k["gram_on_tensor_cores"] = {
                    "digit_flops_per_point": tfl,
                    "achieved": tfl * points / (ms * 1e-3) / 1e12 if ms > 0 else None,
                    "peak": peak_bf16, "unit": "TFLOP/s",
                    "peak_basis": "measured cuBLAS bf16 (burst)",
                    "note": f"the method's {fp64_gram_flops_per_point(n_ifo):.0f} Gram flops per "
                            f"point as exact 7-bit digit products (8 digits per value)"}
            return k
        if prec == gw.GW_MIXED:
            kernels.append({"kernel": "k_points_mixed (Fisher)", "ms": kern_ms, "points": pts_mixed,
                            "bound": "alu", "peak": peak32,
                            "peak_basis": f"FP32 pipe: {sms} SMs x {FP32_FMA_PER_CLK_SM} FMA/clk "
                                          f"(packed FP32x2) x 2 flops x {sm_mhz:.0f} MHz",
                            "executed_flops_per_point": exec_fp})
            if kern_ref_ms > 0:
                kernels.append(fp64_entry("refinement of the ill-conditioned events", kern_ref_ms,
                                          pts_ref))
        elif prec in (gw.GW_DFLOAT, ROUTED) and n_ifo <= 2:
            # the method's FP64-class arithmetic against the FP64 pipe's peak:
            # the kernel runs it as double-float on the FP32 pipe and as exact
            # digit products on the tensor cores, so it can exceed that peak
            # (the routed step: the double-float pass over its BBH events)
            tfl = tc_digit_flops_per_point(n_ifo, N_PAR)
            pts_df = routed_counts["points_df"] if prec == ROUTED else n_points
            kernels.append({
                "kernel": "k_fisher_tc<double-float> (Fisher" +
                          (", the routed step's BBH events)" if prec == ROUTED else ")"),
                "ms": kern_ms, "points": pts_df,
                "bound": "alu", "peak": peak64,
                "peak_basis": f"FP64 pipe: {sms} SMs x {FP64_FMA_PER_CLK_SM} FMA/clk x 2 flops "
                              f"x {sm_mhz:.0f} MHz (the method's arithmetic in FP64; executed as "
                              f"double-float on the FP32 pipe and exact bf16 digit products on "
                              f"the tensor cores)",
                "executed_flops_per_point": None,
                "pipe_flops_per_point": algo_fp,
                "issue": {
                    "warp_instructions_per_point": ISSUE_WARP_INSTR_PER_POINT["dfloat_tc"],
                    "achieved": ISSUE_WARP_INSTR_PER_POINT["dfloat_tc"] * pts_df /
                                (kern_ms * 1e-3) / 1e9 if kern_ms > 0 else None,
                    "peak": sms * 4 * sm_mhz * 1e6 / 1e9, "unit": "G warp instructions/s",
                    "peak_basis": f"{sms} SMs x 4 schedulers x 1 instruction/clk x {sm_mhz:.0f} MHz",
                    "source": "instructions per point from one ncu capture of the 2e4-event "
                              "literal-grid catalog, scaled by this launch's points"},
                "gram_on_tensor_cores": {
                    "digit_flops_per_point": tfl,
                    "achieved": tfl * pts_df / (kern_ms * 1e-3) / 1e12 if kern_ms > 0 else None,
                    "peak": peak_bf16, "unit": "TFLOP/s",
                    "peak_basis": "measured cuBLAS bf16 (burst)"}})
        else:
            kernels.append(fp64_entry("Fisher", kern_ms,
                                      routed_counts["points_df"] if prec == ROUTED else n_points))
        for k in kernels:
            # the flops of the kernel's bound pipe: the method's FP64 count, less the
            # Gram where the tensor cores form it
            k["achieved"] = k.get("pipe_flops_per_point", algo_fp) * k["points"] / (k["ms"] * 1e-3) / 1e12
            k["frac"] = k["achieved"] / k["peak"]
            k["algorithmic_flops_per_point"] = algo_fp
            k["unit"] = "TFLOP/s"
            is_mixed = k["kernel"].startswith("k_points_mixed")
            # DRAM bytes per point from ncu captures of the literal-grid workload
            # (none for the FP64 tensor-core variant)
            is_df = k["kernel"].startswith("k_fisher_tc<double-float>")
            is_tc = k["kernel"].startswith("k_fisher_")
            per_pt = DRAM_BYTES_PER_POINT.get("mixed" if is_mixed else (
                "dfloat_tc" if is_df else ("fp64_tc" if is_tc else "fp64")))
            if "issue" in k and k["issue"]["achieved"] is not None:
                k["issue"]["frac"] = k["issue"]["achieved"] / k["issue"]["peak"]
            k["traffic"] = per_pt * k["points"] if (a.grid == "literal" and per_pt) else None
        dom = max(kernels, key=lambda k: k["ms"])
        roofline = {"bound": dom["bound"], "achieved": dom["achieved"], "peak": dom["peak"],
                    "unit": "TFLOP/s", "frac": dom["frac"], "traffic": dom["traffic"],
                    "kernel": dom["kernel"], "kernel_ms": dom["ms"],
                    "algorithmic_flops_per_point": algo_fp,
                    "executed_flops_per_point": dom["executed_flops_per_point"],
                    "pipe_flops_per_point": dom.get("pipe_flops_per_point", algo_fp),
                    **({"gram_on_tensor_cores": dom["gram_on_tensor_cores"]}
                       if "gram_on_tensor_cores" in dom else {}),
                    **({"issue": dom["issue"]} if "issue" in dom else {}),
                    "peak_basis": dom["peak_basis"] + " (median sampled SM clock)",
                    "kernels": kernels,
                    "measured_fma_per_clk_sm": {"fp64": rate64["fma_per_clk_sm"],
                                                "fp32_packed": rate32["fma_per_clk_sm"]}}
        cpu = None
        err_sample = None
        if not a.no_cpu_baseline:
            cores = os.cpu_count() or 1
            v, rows, ores, el = oracle_timing(raw, cfg, cores, budget_s=20.0, psd_kind=a.psd)
            cpu = {"value": v, "unit": "events/s", "cores": cores, "kind": "oracle",
                   "sample": f"{len(rows)} random events of this rank's catalog in {el:.1f} s "
                             f"(prepare + SNR + Fisher + inversion + SNR gradient), "
                             f"one event per process on {cores} host cores"}
            if not gated:
                # the timed step's results on the sampled events against the oracle's
                diag = [i * N_PAR - i * (i - 1) // 2 for i in range(N_PAR)]
                Fg = F.cpu().numpy()[:, rows].T
                sg = snr.cpu().numpy()[rows]
                Cg = inv[0].cpu().numpy()[:, rows].T
                Fo = np.array([r[0] for r in ores])
                so = np.array([r[1] for r in ores])
                Co = np.array([r[2] for r in ores])
                ko = np.array([r[3] for r in ores])
                okd = (np.array([r[4] for r in ores]) & 33) == 0
                dgo = np.sqrt(Fo[:, diag])
                iu = np.triu_indices(N_PAR)
                relF = np.max(np.abs(Fg - Fo) / (dgo[:, iu[0]] * dgo[:, iu[1]]), axis=1)
                with np.errstate(all="ignore"):
                    relC = np.max(np.abs(np.sqrt(np.abs(Cg[:, diag])) /
                                         np.sqrt(np.abs(Co[:, diag])) - 1), axis=1)
                err_sample = {"events": int(len(rows)),
                              "snr_max_rel": float(np.max(np.abs(sg / so - 1))),
                              "fisher_max_rel_of_sqrt_FiiFjj": float(relF.max()),
                              "sqrt_diag_cov_max_rel": float(np.nanmax(relC[okd])) if okd.any() else None,
                              "sqrt_diag_cov_worst_over_bound": float(np.nanmax(
                                  relC[okd] / np.maximum(1e-3, 1e-15 * ko[okd]))) if okd.any() else None}
        # (the stored oracle results use the power-sum noise curve)
        golden = golden_error(gw, a.refine_cond) if (cfg == "c3" and not gated and a.psd == "power") \
            else None
        line = {
            "metric": METRIC, "value": value, "unit": "events/s", "n_gpus": world,
            "steps": a.steps, "warmup": a.warmup, "ms_per_step": total_ms / a.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": {"mixed": "f32+f64 (mixed, FP64 refinement)", "fp64": "f64",
                      "dfloat": "double-float (f32 pairs) tangents, exact bf16-digit Gram, "
                                "f64 combination",
                      "routed": "per event: double-float (f32 pairs) + exact bf16-digit Gram "
                                "for the BBH, f32+f64 mixed for the rest (double-float "
                                "recomputation above kappa 1e7)"}[a.precision],
            "data": "synthetic (seeded, gwcat)",
            "config": {"workload": {"c3": WORKLOAD, "c4": WORKLOAD_C4,
                                    "c3-gated": WORKLOAD_GATED}[a.workload],
                       "n_events_total": n_total, "n_events_per_gpu": n_per_gpu,
                       "grid": a.grid, "psd": a.psd, "points_per_step_rank0": n_points + (n_points_all if gated else 0),
                       "precision": a.precision, "n_par": N_PAR,
                       "step": ("prepare + SNR pass + gate + " if gated else "prepare + ")
                               + "SNR/Fisher with fused SNR VJP + Cholesky inversion"
                               + (f" + FP64 refinement of events with condition number > "
                                  f"{a.refine_cond:g}" if prec == gw.GW_MIXED else "")
                               + (" + log-det VJP (FP64) over the two L detectors' orientations"
                                  if with_logdet else ""),
                       **({"selected_events_rank0": n_sel, "fisher_points_rank0": n_points}
                          if gated else {}),
                       "l2": "flushed before every timed step (256 MiB write)",
                       "launch": "eager calls" if a.eager else (
                                 "the preparation as a CUDA graph replay + gw_fisher_routed "
                                 "called per step (it reads back its split)" if prec == ROUTED
                                 else "one CUDA graph replay per step + the refinement's calls"),
                       "parallelism": f"one catalog split into {world} cost-balanced contiguous "
                                      f"ranges, one per GPU" + (
                                          "; log-det gradient all-reduced (SUM) per step"
                                          if with_logdet and world > 1 else "; no collective")},
            "clocks": clocks,
            "refined_fraction": refined_frac if prec in (gw.GW_MIXED, ROUTED) else None,
            "e2e": {"value": e2e_value, "unit": "events/s", "h2d_bytes_per_step": h2d,
                    "d2h_bytes_per_step": d2h,
                    "copies": "pinned host buffers, on a copy stream overlapping the "
                              "previous/next step's compute"},
            "gpu_launches": None,
            "roofline": roofline,
            "cpu_baseline": cpu,
            "error": {"bound": "sqrt(diag C): max(1e-3, 1e-15 kappa) relative to the oracle "
                               "(the FP64 rounding floor of an FP64 Fisher matrix above 1e12)",
                      "oracle_sample_of_this_run": err_sample,
                      "oracle_stratified_1000_c3_events": golden},
        }
        if tiles is not None:
            line["tiles"] = tiles
        if fp64 is not None and prec != gw.GW_FP64:
            line["fp64_arm"] = {"value": rates[4], "unit": "events/s", "ms_per_step": fp64_ms / a.steps,
                                "point_kernel_ms": fp64_kern_ms, "clocks": fp64["clocks"]}
            line[f"{a.precision}_over_fp64"] = value / rates[4]
            if routed is not None:
                line["routed_arm"] = routed
                line["routed_over_fp64"] = routed["value"] / rates[4]
        # launches per step: prepare 1; Fisher 7 (event setup, scan 3, point loop,
        # finish, SNR VJP); inversion 1; refinement (when it selects events) 15:
        # flag + scan 3 + compact, gather, Fisher 7, inversion, one scatter of
        # every result, else 5; log-det VJP 6; gated: SNR pass 6 and gate 5
        per_step = 1 + 7 + 1 + (6 if with_logdet else 0) + (11 if gated else 0)
        if prec == ROUTED:
            # prepare 1; split 9 (flag, two scans of 3, two compactions); per
            # part: gather, Fisher 7, inversion, one scatter; after the mixed
            # part the marking of its events to recompute, scan 3 and compaction
            per_step = 1 + 9 + 2 * 10 + 5 + (6 if with_logdet else 0) + (11 if gated else 0)
        if prec == gw.GW_MIXED:
            per_step += 15 if n_refined > 0 else 5
        line["gpu_launches"] = per_step * a.steps
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def main():
    a = parse()
    if a.impl == "reference":
        run_reference(a)
    else:
        run_ours(a)


if __name__ == "__main__":
    main()
