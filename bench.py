"""Benchmark: DNS points filtered (+ T_ij) per second on one GB300.

Workload (default, the Re_tau ~ 550 precision form): DNS 512 x 257 x 384 in
a 2 pi x 2 x pi box, tanh-stretched y, filtered with a Gaussian of constant
width Delta = Lx / 64 (wall extension of Eq. 7) onto a 64 x 65 x 48 LES grid
with split-BF16 tensor-core contractions; one step = ~bar(u_i), T_ij and the
plane means of 10 seeded synthetic snapshots.  Inputs are 10 x 607 MB = 6.1
GB per step, far larger than the 129 MB L2, so no flush is needed between
steps.  Ten snapshots are 2570 (snapshot, y-plane) items of the persistent
x-z kernel, 16.9 per SM on 152 SMs, so its last wave is 90 % full (eight
give 13.5 per SM and a last wave half full).  `--workload re550_d32` is the same with Delta = Lx / 32;
`--workload re180` selects the 192 x 129 x 192 -> 32 x 33 x 32,
Delta = Lx / 32 channel (10 snapshots per step).  `--precision` picks the
split form (bf16x3, the default, or tf32x2) or fp32 / fp64.

Output: one JSON line (rank 0).  `value` is whole-job throughput in DNS
points per second with inputs resident in HBM; `e2e` is the same metric
through the host-buffer C-ABI call (ef_subfilter_stress_host: pinned host
inputs and outputs, the copies in and out overlapped with the compute of
other snapshots) inside the timed region.  `roofline` reports the
x-contraction kernel (the dominant phase) against the measured HBM copy
bandwidth.  `cpu_baseline` times the CPU oracle on a bounded sample.
`closure` reports the learned closure in its own configuration: trained on the
exact T_ij of 32 seeded 256 x 193 x 256 snapshots filtered to 64 x 65 x 48 at
Delta = Lx / 32, its error per component on two held-out seeds beside the
gradient model's, the training rate, and tensor-core inference on 2^20 LES
points with its roofline.  `differential` times the
paper's own filter (Sec. 3, a = 0.1) on one snapshot in FP64 against the FP64
arithmetic bound.  `split_forms` runs the other split-precision form on the
same snapshots, and both forms with the configuration's other filter width
(Lx / 32 on the Lx / 64 workload), each with its x-z roofline and the T error
of snapshot 0 against the oracle per component.  `apost` runs the loop of
Fig. 2 on the workload: per step the filter of one DNS snapshot (T_ij and the
wall values of Eq. 10) and one RK3 step of the FP64 LES on the LES grid.

Multi-GPU: one process per GPU; snapshots are independent, so every rank
filters its own snapshots with no collective on the data path (weak
scaling, "replicas only").

--impl reference times the CPU oracle (the only reference that exists for
this method) on the same workload's unit.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

METRIC = "DNS pts filtered+tau_ij per s, TC split-prec vs FP64 plain at stated err; %roofline"
UNIT = "DNS points/s"

WORKLOADS = {
    # name: (nx, ny, nz, Lx, Lz, nlx, nly, nlz, delta/Lx, snapshots per step)
    "re180": (192, 129, 192, 4 * math.pi, 2 * math.pi, 32, 33, 32, 1 / 32, 10),
    "re550_d64": (512, 257, 384, 2 * math.pi, math.pi, 64, 65, 48, 1 / 64, 10),
    "re550_d32": (512, 257, 384, 2 * math.pi, math.pi, 64, 65, 48, 1 / 32, 10),
}
PREC = {"fp32": 1, "fp64": 0, "bf16x3": 3, "tf32x2": 2}
L2_BYTES = 129e6


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="re550_d64", choices=sorted(WORKLOADS) + ["batch64"])
    ap.add_argument("--precision", default="bf16x3", choices=sorted(PREC))
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-fp64", action="store_true")
    ap.add_argument("--no-closure", action="store_true")
    ap.add_argument("--no-forms", action="store_true")
    ap.add_argument("--no-apost", action="store_true")
    ap.add_argument("--snapshots", type=int, default=0, help="snapshots per step (default: the workload's)")
    return ap.parse_args()


def snapshot_recipe(rank, ns):
    """(seed, x shift, z shift) of each of a rank's ns snapshots: two seeded
    fields per rank, the rest periodic shifts of them.  Ranks never share a
    seed, so the ranks filter disjoint snapshots (no collective on the data)."""
    nbase = min(ns, 2)
    return [(1000 + rank * 1000 + s % nbase, 0 if s < nbase else 7 * s, 0 if s < nbase else 5 * s)
            for s in range(ns)]


def max_over_ranks(ms, device, world):
    """The step time of the job: the slowest rank's."""
    if world <= 1:
        return ms
    import torch
    import torch.distributed as dist
    t = torch.tensor([ms], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(world, units_per_rank_step, steps, ms):
    """Units all ranks processed per second (weak scaling: every rank its own)."""
    return world * units_per_rank_step * steps / (ms / 1e3)


def make_workload(name, rank=0, nsnap=0):
    from paper_1902_02508_gb300 import inputs as I
    nx, ny, nz, Lx, Lz, nlx, nly, nlz, dfrac, ns = WORKLOADS[name]
    ns = nsnap or ns
    dns = I.dns_grid(nx, ny, nz, Lx, Lz)
    les = I.les_grid(dns, nlx, nly, nlz)
    delta = dfrac * Lx
    recipe = snapshot_recipe(rank, ns)
    base = {seed: I.channel_velocity(dns, seed) for seed, sx, sz in recipe if sx == 0 and sz == 0}
    snaps = [base[seed] if (sx, sz) == (0, 0) else I.shifted(base[seed], sx, sz) for seed, sx, sz in recipe]
    return dns, les, delta, snaps


def workload_config(name, prec, nsnap=0):
    nx, ny, nz, Lx, Lz, nlx, nly, nlz, dfrac, ns = WORKLOADS[name]
    ns = nsnap or ns
    esz = 8 if prec == "fp64" else 4
    return {"workload": f"channel DNS {nx}x{ny}x{nz} -> LES {nlx}x{nly}x{nlz}, Delta=Lx/{round(1 / dfrac)}, "
                        f"Eq.7 wall extension, {ns} snapshots per step",
            "dns_grid": [nx, ny, nz], "les_grid": [nlx, nly, nlz], "box": [Lx, 2.0, Lz],
            "delta": dfrac * Lx, "snapshots_per_step": ns,
            "l2": f"inputs {ns * nx * ny * nz * 3 * esz / 1e6:.0f} MB per step > {L2_BYTES / 1e6:.0f} MB L2, no flush"}


# ------------------------------------------------------------ clocks ----
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (OSError, FileNotFoundError):
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *a):
        self.out = ""
        if self.proc:
            time.sleep(0.2)
            self.proc.terminate()
            try:
                self.out, _ = self.proc.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                self.out, _ = self.proc.communicate()

    def summary(self):
        if not self.proc or not self.out:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.out.strip().splitlines():
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax = float(parts[2])
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax,
                "reasons": sorted(reasons), "samples": len(sm)}


# ------------------------------------------------------------ oracle ----
def oracle_time(dns, les, delta, snaps, budget_s=10.0):
    """Time the CPU oracle (separable FP64 evaluation) on whole snapshots of
    the workload until ~budget_s has passed.  Returns (points/s, cores, sample)."""
    from oracle import oracle as O
    done, t0 = 0, time.perf_counter()
    while True:                                  # cycle through the snapshots for about budget_s
        O.subfilter_stress(dns, les, delta, snaps[done % len(snaps)])
        done += 1
        if time.perf_counter() - t0 > budget_s:
            break
    dt = time.perf_counter() - t0
    pts = done * dns.npts
    return pts / dt, O.num_threads(), f"{done} whole snapshot(s) of the workload ({len(snaps)} distinct), {dt:.1f} s"


def min_eigenvalue(tau):
    """Smallest eigenvalue of the symmetric 3 x 3 T_ij over all LES points."""
    T = np.empty(tau.shape[1:] + (3, 3))
    for q, (i, j) in enumerate(((0, 0), (0, 1), (0, 2), (1, 1), (1, 2), (2, 2))):
        T[..., i, j] = tau[q]
        T[..., j, i] = tau[q]
    return float(np.linalg.eigvalsh(T.reshape(-1, 3, 3)).min())


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    from oracle import oracle as O
    if args.workload == "batch64":
        # one step = one snapshot of each of the batch's plans in turn (a
        # bounded sample of the 64-snapshot batch)
        from paper_1902_02508_gb300 import inputs as I
        combos, base = batch64_setup(0)
        jobs = []
        for shape, w, _ in combos:
            dns, les = I.batch_grids(shape)
            jobs.append((dns, les, dns.Lx / w, base[shape][0]))
        for s in range(args.warmup):
            O.subfilter_stress(*jobs[s % len(jobs)])
        t0, npts = time.perf_counter(), 0
        for s in range(args.steps):
            O.subfilter_stress(*jobs[s % len(jobs)])
            npts += jobs[s % len(jobs)][0].npts
        dt = time.perf_counter() - t0
        value = npts / dt
        line = {"metric": METRIC, "value": value, "unit": UNIT, "impl": "reference", "n_gpus": args.gpus,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
                "data": "synthetic", "config": {"workload": "batched (64 snapshots, 9 plans): one snapshot of "
                                                            "each plan in turn per step"},
                "cpu_baseline": {"value": value, "unit": UNIT, "cores": O.num_threads(), "kind": "oracle",
                                 "sample": f"{args.steps} whole snapshots, one per plan in turn"},
                "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
        print(json.dumps(line), flush=True)
        return
    dns, les, delta, snaps = make_workload(args.workload, 0, args.snapshots)
    for s in range(args.warmup):
        O.subfilter_stress(dns, les, delta, snaps[s % len(snaps)])
    t0 = time.perf_counter()
    for s in range(args.steps):
        O.subfilter_stress(dns, les, delta, snaps[s % len(snaps)])
    dt = time.perf_counter() - t0
    value = args.steps * dns.npts / dt
    line = {"metric": METRIC, "value": value, "unit": UNIT, "impl": "reference", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": workload_config(args.workload, args.precision, args.snapshots),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": O.num_threads(), "kind": "oracle",
                             "sample": f"one whole snapshot per step ({dns.npts} DNS points)"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# --------------------------------------------------------------- ours ----
KERNEL_SOURCES = {"xz": ("fused_stage.cuh", "xz_ws.cuh", "xz_ws.cu", "eles_internal.h"),
                  "closure": ("closure_tc.cu", "fused_stage.cuh", "eles_internal.h")}


def kernel_source_hash(kind="xz"):
    import hashlib
    h = hashlib.sha256()
    for name in KERNEL_SOURCES[kind]:
        h.update(open(os.path.join(ROOT, "paper_1902_02508_gb300", "csrc", name), "rb").read())
    return h.hexdigest()[:16]


def traffic_from_profile(kernel_tag, points_per_launch, kind="xz"):
    """DRAM bytes per launch from the committed ncu summary, if it was taken
    on the current kernel source; scaled from the captured launch's points to
    this launch's points (the traffic is proportional to the points read)."""
    path = os.path.join(ROOT, "profiles", f"{kernel_tag}.json")
    try:
        prof = json.load(open(path))
        if prof.get("source_sha256_16") == kernel_source_hash(kind):
            return prof["dram_bytes_per_point"] * points_per_launch
    except (OSError, ValueError, KeyError):
        pass
    return None


def peak_of(peaks):
    """Measured HBM copy bandwidth (GB/s) of the GB300s, else the fallback."""
    if "hbm_gbs" in peaks:
        return peaks["hbm_gbs"], "measured"
    return 6800.0, "fallback"


def form_measure(eles, torch, workload, pname, dns, les, snaps, u, ub, tau, pm, stream, timed, steps, peak, rank):
    """One split-precision form on the workload's snapshots (same fields; the
    filter width of `workload`): throughput, the x-z kernel against the HBM
    roofline, and T of snapshot 0 against the oracle per component."""
    nx, ny, nz, Lx, Lz, nlx, nly, nlz, dfrac, _ = WORKLOADS[workload]
    delta = dfrac * Lx
    plan = eles.filter_setup(dns, les, delta, precision=PREC[pname])
    ns = u.shape[0]
    eles.plan_reserve(plan, ns)
    k = max(10, steps // 4)
    ms = timed(lambda: eles.subfilter_stress_batch(plan, u, ub, tau, pm, stream=stream), k, 3)
    eles.profile_enable(plan, True)
    timed(lambda: eles.subfilter_stress_batch(plan, u, ub, tau, pm, stream=stream), max(5, k // 2), 1)
    phase_ms, calls = eles.profile_read(plan)
    eles.profile_enable(plan, False)
    xz_ms = phase_ms[0] / max(calls, 1)
    alg = 12 * dns.npts * ns
    out = {"workload": workload_config(workload, pname)["workload"], "dtype": pname, "delta": delta,
           "value": dns.npts * ns * k / (ms / 1e3), "unit": UNIT, "ms_per_step": ms / k,
           "x_variant": eles.plan_info(plan, 10), "output_phases": eles.plan_info(plan, 15),
           "roofline": {"bound": "hbm", "achieved": alg / (xz_ms / 1e3) / 1e9, "peak": peak[0], "unit": "GB/s",
                        "frac": alg / (xz_ms / 1e3) / 1e9 / peak[0], "peak_source": peak[1],
                        "phase_ms_per_step": {"xz": xz_ms, "y_recovery": phase_ms[2] / max(calls, 1)}}}
    if rank == 0:
        from oracle import oracle as O
        _, tau_ref = O.subfilter_stress(dns, les, delta, snaps[0])
        got = tau[0].double().cpu().numpy()
        out["accuracy"] = {"tau_max_abs_err_utau2": [float(x) for x in np.abs(got - tau_ref).max(axis=(1, 2, 3))],
                           "tau_order": ["11", "12", "13", "22", "23", "33"]}
    plan.close()
    return out


def differential_measure(eles, torch, dns, les, u0, stream, timed, peaks):
    """EF_KERNEL_DIFFERENTIAL (FP64) on one snapshot, against the FP64 arithmetic
    bound.  Algorithmic flops: 5 N log2 N per complex transform of length N
    (two real x rows per transform), 10 per Thomas row, for the 9 fields."""
    delta_f = 0.1 * math.sqrt(40.0)                    # a = 0.1 (Sec. 3), a^2 = Delta_f^2 / 40
    plan = eles.filter_setup(dns, les, delta_f, kernel=eles.KERNEL_DIFFERENTIAL, precision=0)
    with torch.cuda.stream(stream):
        ud = u0.double().contiguous()
        ub = torch.empty((3, les.ny, les.nz, les.nx), device=ud.device, dtype=torch.float64)
        tau = torch.empty((6, les.ny, les.nz, les.nx), device=ud.device, dtype=torch.float64)
    torch.cuda.synchronize()
    k = 3
    ms = timed(lambda: eles.subfilter_stress(plan, ud, ub, tau, stream=stream), k, 1) / k
    assert eles.check_device_error(plan, stream) == 0
    plan.close()
    # the FP32 form: fluctuations about the plane means in FP32, profiles and recovery in FP64
    p32 = eles.filter_setup(dns, les, delta_f, kernel=eles.KERNEL_DIFFERENTIAL, precision=1)
    with torch.cuda.stream(stream):
        uf = u0.float().contiguous()
        ub32 = torch.empty((3, les.ny, les.nz, les.nx), device=ud.device)
        tau32 = torch.empty((6, les.ny, les.nz, les.nx), device=ud.device)
    torch.cuda.synchronize()
    ms32 = timed(lambda: eles.subfilter_stress(p32, uf, ub32, tau32, stream=stream), k, 1) / k
    p32.close()
    with torch.cuda.stream(stream):
        err32 = float((tau32.double() - tau).abs().max())
    torch.cuda.synchronize()
    nxh = dns.nx // 2 + 1
    lg = math.log2
    flop = 9 * (dns.ny * (dns.nz / 2) * 5 * dns.nx * lg(dns.nx)        # forward x, two rows per transform
                + dns.ny * nxh * 5 * dns.nz * lg(dns.nz)                  # forward z
                + dns.nz * nxh * dns.ny * 10                              # Thomas
                + les.ny * nxh * 5 * dns.nz * lg(dns.nz)                  # inverse z on the LES rows
                + les.ny * les.nz * 5 * dns.nx * lg(dns.nx))              # inverse x on the LES rows
    nsm = torch.cuda.get_device_properties(ud.device).multi_processor_count
    dpeak = 1.68 * 2 * nsm * peaks.get("sm_max_mhz", 2070.0) * 1e6
    ach = flop / (ms / 1e3)
    # the FP64 reference on a bounded sample: one 192 x 129 x 192 channel snapshot
    from oracle import differential as D
    from paper_1902_02508_gb300 import inputs as I
    d2 = I.dns_grid(192, 129, 192, 4 * math.pi, 2 * math.pi)
    l2 = I.les_grid(d2, 32, 33, 32)
    u2 = I.channel_velocity(d2, 1000)
    t0 = time.perf_counter()
    D.subfilter_stress(d2, l2, delta_f, u2)
    dt = time.perf_counter() - t0
    cpu = {"value": d2.npts / dt, "unit": UNIT, "cores": 1, "kind": "oracle",
           "sample": f"one 192x129x192 snapshot -> 32x33x32 (NumPy FFT + Thomas, FP64), {dt:.1f} s"}
    return {"workload": f"differential filter (1 - a^2 lap)^-1, a = 0.1, one {dns.nx}x{dns.ny}x{dns.nz} snapshot "
                        f"-> {les.nx}x{les.ny}x{les.nz}, ubar and T, FP64",
            "ms_per_snapshot": ms, "value": dns.npts / (ms / 1e3), "unit": UNIT,
            "roofline": {"bound": "alu", "achieved": ach / 1e12, "peak": dpeak / 1e12, "unit": "TFLOP/s",
                         "frac": ach / dpeak, "flop_per_snapshot": flop,
                         "peak_source": "FP64 FMA rate measured on GB300 (1.68 per SM per clock) x SMs x max clock"},
            "gpu_launches_per_snapshot": 3 * 5 + 1, "cpu_baseline": cpu,       # 3 groups of 3 fields x 5 steps, stress
            "fp32": {"ms_per_snapshot": ms32, "value": dns.npts / (ms32 / 1e3), "unit": UNIT,
                     "tau_max_abs_diff_vs_fp64_utau2": err32,
                     "form": "u', u'u' and U u' (18 fields) through FP32 transforms; profiles and recovery in FP64",
                     "gpu_launches_per_snapshot": 2 + 3 * 5 + 1}}     # profile, 3 groups of 6 x 5 steps, recovery


CLOSURE_FLOP_PER_POINT = 2 * (10 * 128 + 128 * 128 + 128 * 128 + 128 * 6)   # 69,632: the four layers' MACs
CLOSURE_POINTS = 1 << 20
# The SiLU of the 384 hidden activations per point takes one ex2.approx and one
# rcp.approx each; on GB300 these issue at 32 and 16 lanes per SM per clock
# (throughput of independent chains, measured), so a point needs
# 384 (1/32 + 1/16) = 36 SM-clocks of the special-function units.
CLOSURE_SFU_CLK_PER_POINT = 384 * (1 / 32 + 1 / 16)


CLOSURE_DNS = (256, 193, 256)      # 4 pi x 2 x 2 pi channel
CLOSURE_LES = (64, 65, 48)
CLOSURE_TRAIN, CLOSURE_HELDOUT, CLOSURE_EPOCHS = 32, 2, 8
# training flop per point and epoch, one product per multiply: forward (all
# four layers), weight gradients (all four) and input gradients (layers 1-3)
CLOSURE_TRAIN_FLOP_PER_POINT = 2 * CLOSURE_FLOP_PER_POINT + 2 * (128 * 128 + 128 * 128 + 128 * 6)
CLOSURE_LAUNCHES_PER_TRAIN_STEP = 34


def closure_measure(eles, torch, stream, peaks):
    """The learned closure in the configuration it is specified for: exact
    T_ij of 32 seeded 256 x 193 x 256 channel snapshots (4 pi x 2 x 2 pi)
    filtered to 64 x 65 x 48 at Delta = Lx / 32 train the network; two more
    seeds are held out.  Reports the held-out error per component against the
    exact stress for the network, the gradient model (formed from the same
    features) and no model; the training rate; and tensor-core inference on
    2^20 LES points.  Rank 0 only: its timings are local."""
    from concurrent.futures import ThreadPoolExecutor

    from paper_1902_02508_gb300 import inputs as I
    dev = torch.device("cuda", torch.cuda.current_device())
    dns = I.dns_grid(*CLOSURE_DNS, *I.BOX_LARGE)
    les = I.les_grid(dns, *CLOSURE_LES)
    delta = dns.Lx / 32
    plan = eles.filter_setup(dns, les, delta, precision=eles.PREC_FP32)
    n = les.nx * les.ny * les.nz
    seeds = [5000 + s for s in range(CLOSURE_TRAIN)] + [6000 + s for s in range(CLOSURE_HELDOUT)]

    def local_ms(fn, k, warm=2):
        for _ in range(warm):
            fn()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with torch.cuda.stream(stream):
            e0.record(stream)
            for _ in range(k):
                fn()
            e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / k

    feats, taus = [], []
    t0 = time.perf_counter()
    exact_ms = None
    with ThreadPoolExecutor(8) as ex, torch.cuda.stream(stream):
        for i in range(0, len(seeds), 8):
            for u in ex.map(lambda sd: I.channel_velocity(dns, sd).astype(np.float32), seeds[i:i + 8]):
                ud = torch.from_numpy(u).to(dev)
                ub = torch.empty((3, les.ny, les.nz, les.nx), device=dev)
                tau = torch.empty((6, les.ny, les.nz, les.nx), device=dev)
                call = lambda: eles.subfilter_stress(plan, ud, ub, tau, stream=stream)
                if exact_ms is None:
                    exact_ms = local_ms(call, 5)
                call()
                f = torch.empty((n, 10), device=dev)
                eles.closure_features(les, ub, f, re_tau=I.RE_TAU, stream=stream)
                feats.append(f)
                taus.append(tau.reshape(6, n))
    torch.cuda.synchronize()
    data_s = time.perf_counter() - t0
    ftr = torch.cat(feats[:CLOSURE_TRAIN], 0).contiguous()
    ttr = torch.cat(taus[:CLOSURE_TRAIN], 1).contiguous()
    ntr = ftr.shape[0]
    cl = eles.closure_create(batch=4096, lr=2e-3, seed=3)
    t0 = time.perf_counter()
    loss = eles.closure_train(cl, ftr, ttr, epochs=CLOSURE_EPOCHS, stream=stream)
    torch.cuda.synchronize()
    train_s = time.perf_counter() - t0
    del ftr, ttr
    fho = torch.cat(feats[CLOSURE_TRAIN:], 0).contiguous()
    tho = torch.cat(taus[CLOSURE_TRAIN:], 1).contiguous().double()
    nho = fho.shape[0]
    with torch.cuda.stream(stream):
        pred = torch.empty((6, nho), device=dev)
        nfall = eles.closure_infer(cl, fho, pred, stream=stream)
        # the gradient model T_ij = Delta^2 / 12 g_ik g_jk from the same features
        g = fho[:, :9].double().reshape(nho, 3, 3)
        pairs = ((0, 0), (0, 1), (0, 2), (1, 1), (1, 2), (2, 2))
        gm = torch.stack([delta * delta / 12.0 * (g[:, i, :] * g[:, j, :]).sum(dim=1) for i, j in pairs])

        def rel(a):
            d = a - tho
            return float(d.norm() / tho.norm()), [float(d[q].norm() / tho[q].norm()) for q in range(6)]
        mlp_rel, mlp_c = rel(pred.double())
        gm_rel, gm_c = rel(gm)
        reps = (CLOSURE_POINTS + nho - 1) // nho
        f1m = fho.repeat(reps, 1)[:CLOSURE_POINTS].contiguous()
        out = torch.empty((6, CLOSURE_POINTS), device=dev)
    torch.cuda.synchronize()
    ms = local_ms(lambda: eles.closure_infer(cl, f1m, out, stream=stream, count=False), 20, 3)
    assert eles.closure_check_device_error(cl, stream) == 0
    tflops = CLOSURE_FLOP_PER_POINT * CLOSURE_POINTS / (ms / 1e3) / 1e12
    tpeak = peaks.get("bf16_tflops", 1900.0)
    nsm = torch.cuda.get_device_properties(dev).multi_processor_count
    sm_hz = peaks.get("sm_max_mhz", 2070.0) * 1e6
    pts = CLOSURE_POINTS / (ms / 1e3)
    sfu_peak = nsm * sm_hz / CLOSURE_SFU_CLK_PER_POINT
    train_pts = ntr * CLOSURE_EPOCHS / train_s
    train_tflops = train_pts * CLOSURE_TRAIN_FLOP_PER_POINT / 1e12
    # the FP64 reference forward pass on a bounded sample of the same features
    from oracle import mlp as M
    params, stats = eles.closure_get_params(cl)
    cl.close()
    ncpu = 200000
    Xs = f1m[:ncpu].double().cpu().numpy()
    t0 = time.perf_counter()
    M.forward([(W.astype(np.float64), b.astype(np.float64)) for W, b in eles.closure_unpack(params)],
              (Xs - stats[:10]) / stats[10:20])
    dt = time.perf_counter() - t0
    cpu = {"value": ncpu / dt, "unit": "points/s", "cores": os.cpu_count(), "kind": "oracle",
           "sample": f"{ncpu} points, NumPy FP64 forward pass, {dt:.2f} s"}
    order = ["11", "12", "13", "22", "23", "33"]
    return {"workload": f"MLP 10-128-128-128-6 (SiLU) trained on the exact T_ij of {CLOSURE_TRAIN} synthetic "
                        f"{'x'.join(map(str, CLOSURE_DNS))} channel snapshots (4 pi x 2 x 2 pi) filtered to "
                        f"{'x'.join(map(str, CLOSURE_LES))} at Delta = Lx/32 ({ntr} LES points); inference on "
                        f"{CLOSURE_POINTS} LES points (held-out features, repeated)",
            "ms_per_call": ms, "points_per_s": pts,
            "precision": "BF16 weights, split-BF16 activations, FP32 accumulation (tcgen05, TMEM)",
            "roofline": {"bound": "alu", "achieved": pts, "peak": sfu_peak, "unit": "points/s",
                         "frac": pts / sfu_peak,
                         "peak_source": f"SiLU on the special-function units: {nsm} SMs x {sm_hz / 1e6:.0f} MHz / "
                                        f"{CLOSURE_SFU_CLK_PER_POINT:.0f} SM-clocks per point (ex2 32, rcp 16 "
                                        f"lanes per SM per clock, measured)",
                         "tensor": {"achieved": tflops, "peak": tpeak, "unit": "TFLOP/s", "frac": tflops / tpeak,
                                    "peak_source": "measured bf16 burst" if "bf16_tflops" in peaks else "fallback",
                                    "flop_per_point": CLOSURE_FLOP_PER_POINT},
                         "traffic": traffic_from_profile("closure_mlp_tc_1m", CLOSURE_POINTS, "closure")},
            "error_vs_exact": {"rel_l2": mlp_rel, "rel_l2_per_component": mlp_c,
                               "gradient_model_rel_l2": gm_rel, "gradient_model_rel_l2_per_component": gm_c,
                               "no_model_rel_l2": 1.0, "tau_order": order,
                               "test": f"{CLOSURE_HELDOUT} held-out seeds ({nho} LES points)",
                               "guarded_points": nfall},
            "train": {"points": ntr, "epochs": CLOSURE_EPOCHS, "batch": 4096, "s": train_s,
                      "points_per_s": train_pts, "final_loss_standardised": loss,
                      "gemms": "mma.sync m16n8k16 BF16, split-BF16 activations and gradients, FP32 accumulation, "
                               "fixed-order split-K",
                      "tflops_algorithmic": train_tflops, "flop_per_point": CLOSURE_TRAIN_FLOP_PER_POINT,
                      "tensor_frac": train_tflops / tpeak,
                      "launches_per_step": CLOSURE_LAUNCHES_PER_TRAIN_STEP,
                      "data": f"{len(seeds)} snapshots generated and filtered in {data_s:.1f} s "
                              f"(FP32 plan: the LES z nodes are not DNS nodes)"},
            "exact_ms_per_snapshot": exact_ms,
            "speedup_vs_exact_per_les_point": (exact_ms / n) / (ms / CLOSURE_POINTS), "cpu_baseline": cpu,
            "gpu_launches_per_call": 2}


def apost_measure(eles, torch, dns, les, plan, u, ub, tau, stream, timed, steps):
    """The loop of Fig. 2 on this workload: per step the filter of one DNS
    snapshot (T_ij and the wall values) and one RK3 step of the LES on the
    LES grid (FP64).  Snapshots are taken in turn from the batch."""
    solver = eles.les_create(les, 1.0 / 180.0, forcing=1.0)
    ns = u.shape[0]
    ub1, tau1 = ub[0], tau[0]
    eles.filter_fields(plan, u[0], ub1, stream=stream)
    ubar_les = ub1.to(torch.float64, copy=True)
    dt = 1e-3
    state = {"k": 0}

    def loop_step():
        k = state["k"]
        state["k"] = k + 1
        eles.apost_step(plan, solver, u[k % ns], ub1, tau1, ubar_les, dt, stream=stream)

    k = max(10, steps // 2)
    ms = timed(loop_step, k, 3)
    ms_les = timed(lambda: eles.les_step(solver, ubar_les, dt, tau=tau1, ubar_bc=ub1, stream=stream), k, 2)
    div = torch.empty(ubar_les.shape[1:], device=ubar_les.device, dtype=torch.float64)
    eles.les_divergence(solver, ubar_les, div, stream=stream)
    torch.cuda.synchronize()
    out = {"ms_per_step": ms / k, "les_step_ms": ms_les / k, "steps": k,
           "value": dns.npts * k / (ms / 1e3), "unit": "DNS points/s through the loop",
           "dns_grid": [dns.nx, dns.ny, dns.nz], "les_grid": [les.nx, les.ny, les.nz],
           "dt": dt, "scheme": "rk3 (3 projected substeps)",
           "les_launches_per_step": 1 + 3 * 8,
           "max_abs_divergence": float(div.abs().max().item()),
           "finite": bool(torch.isfinite(ubar_les).all().item()),
           "max_abs_ubar": float(ubar_les.abs().max().item())}
    solver.close()
    return out


def batch64_setup(rank=0):
    """The batched configuration: 64 seeded draws of (grid, width); one plan
    per drawn (grid, width), its snapshots the shifts of two seeded fields of
    that grid.  Returns [(shape, width, count)] and the base fields."""
    from collections import Counter
    from paper_1902_02508_gb300 import inputs as I
    combos = sorted(Counter(I.batch_draws(64, 7)).items())
    base = {}
    for (shape, w), count in combos:
        if shape not in base:
            dns, _ = I.batch_grids(shape)
            base[shape] = [I.channel_velocity(dns, 1000 + 1000 * rank + 10 * shape[0] + k) for k in range(2)]
    return [(shape, w, count) for (shape, w), count in combos], base


def run_batch64(args):
    """bench.py --workload batch64: the 64 snapshots (three grids, three
    filter widths, nine plans) through one batch (one CUDA graph: a
    persistent x-z launch per kernel class, then the plans' y stages)."""
    import torch
    import torch.distributed as dist
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        dist.init_process_group("nccl", device_id=dev)
    import __graft_entry__ as entry
    if rank == 0:
        entry.build()      # one rank builds; the others wait for the library
    if world > 1:
        dist.barrier()
    from paper_1902_02508_gb300 import eles
    from paper_1902_02508_gb300 import inputs as I
    prec = PREC[args.precision]
    combos, base = batch64_setup(rank)
    stream = torch.cuda.Stream(dev)
    plans, us, ubs, taus, info = [], [], [], [], []
    pts = 0
    for shape, w, count in combos:
        dns, les = I.batch_grids(shape)
        delta = dns.Lx / w
        plan = eles.filter_setup(dns, les, delta, precision=prec)
        b0 = [torch.from_numpy(f).to(dev, plan.dtype) for f in base[shape]]
        u = torch.stack([torch.roll(b0[k % 2], shifts=(5 * k, 7 * k), dims=(2, 3)) for k in range(count)])
        plans.append(plan)
        us.append(u)
        ubs.append(torch.empty((count, 3, les.ny, les.nz, les.nx), device=dev, dtype=plan.dtype))
        taus.append(torch.empty((count, 6, les.ny, les.nz, les.nx), device=dev, dtype=plan.dtype))
        info.append({"dns_grid": list(shape), "les_grid": [les.nx, les.ny, les.nz], "delta": f"Lx/{w}",
                     "snapshots": count, "x_variant": eles.plan_info(plan, 10),
                     "output_phases": eles.plan_info(plan, 15)})
        pts += count * dns.npts
    batch = eles.batch_create(plans, [c for _, _, c in combos])

    def step():
        eles.batch_run(batch, us, ubs, taus, stream=stream)

    def timed(fn, steps, warmup):
        with torch.cuda.stream(stream):
            for _ in range(warmup):
                fn()
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with torch.cuda.stream(stream):
            e0.record(stream)
            for _ in range(steps):
                fn()
            e1.record(stream)
        torch.cuda.synchronize()
        return max_over_ranks(e0.elapsed_time(e1), dev, world)

    timed(step, 0, args.warmup)
    for p in plans:
        assert eles.check_device_error(p, stream) == 0
    with ClockSampler(local) as clk:
        ms = timed(step, args.steps, 0)
    value = whole_job_rate(world, pts, args.steps, ms)
    captures = eles.batch_captures(batch)
    peak, peak_src = peak_of(json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
                             if os.path.exists(os.path.join(ROOT, "MEASURED_PEAKS.json")) else {})
    ach = 12 * pts / (ms / args.steps / 1e3) / 1e9
    roof = {"bound": "hbm", "kernel": "the whole batch step (x-z launches per kernel class and every plan's y "
                                      "stage, one CUDA graph): 12 B per DNS point read once",
            "achieved": ach, "peak": peak, "unit": "GB/s", "frac": ach / peak, "peak_source": peak_src,
            "traffic": None, "algorithmic_bytes_per_launch": 12 * pts}

    # end to end: every plan through the host-buffer entry point
    hosts = []
    for p, u, ub, tau in zip(plans, us, ubs, taus):
        hosts.append((eles.io_create(p, 1), u.cpu().pin_memory(), torch.empty(ub.shape, dtype=ub.dtype).pin_memory(),
                      torch.empty(tau.shape, dtype=tau.dtype).pin_memory()))

    def e2e_step():
        for io, hu, hb, ht in hosts:
            eles.subfilter_stress_host(io, hu, hb, ht, stream=stream)

    k_e2e = max(3, args.steps // 4)
    ms_e2e = timed(e2e_step, k_e2e, 1)
    e2e = {"value": world * pts * k_e2e / (ms_e2e / 1e3), "unit": UNIT,
           "h2d_bytes_per_step": sum(h[1].numel() * h[1].element_size() for h in hosts),
           "d2h_bytes_per_step": sum(h[2].numel() * h[2].element_size() + h[3].numel() * h[3].element_size()
                                     for h in hosts),
           "api": "ef_subfilter_stress_host per plan (pinned host buffers, 1-snapshot groups)"}
    for h in hosts:
        h[0].close()
    del hosts

    # accuracy: snapshot 0 of every plan against the oracle; the CPU baseline
    err = cpu = None
    step()
    torch.cuda.synchronize()
    if rank == 0:
        from oracle import oracle as O
        worst = np.zeros(6)
        for (shape, w, count), tau in zip(combos, taus):
            dns, les = I.batch_grids(shape)
            _, tau_ref = O.subfilter_stress(dns, les, dns.Lx / w, base[shape][0])
            worst = np.maximum(worst, np.abs(tau[0].double().cpu().numpy() - tau_ref).max(axis=(1, 2, 3)))
        err = {"tau_max_abs_err_utau2": [float(x) for x in worst], "tau_order": ["11", "12", "13", "22", "23", "33"],
               "over": "snapshot 0 of each of the nine plans"}
        if not args.no_cpu_baseline and world == 1:
            done, pdone, t0 = 0, 0, time.perf_counter()
            while time.perf_counter() - t0 < 10.0:
                shape, w, _ = combos[done % len(combos)]
                dns, les = I.batch_grids(shape)
                O.subfilter_stress(dns, les, dns.Lx / w, base[shape][0])
                done += 1
                pdone += dns.npts
            dt = time.perf_counter() - t0
            cpu = {"value": pdone / dt, "unit": UNIT, "cores": O.num_threads(), "kind": "oracle",
                   "sample": f"{done} whole snapshots of the batch's plans in turn, {dt:.1f} s"}
    launches = sum(6 for _ in plans) + len({(eles.plan_info(p, 2), eles.plan_info(p, 15)) for p in plans})
    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": args.precision,
                "data": "synthetic (seeded solenoidal channel fields, Reichardt mean profile)",
                "config": {"workload": "batched: 64 snapshots drawn (seed 7) over DNS grids 128x97x128, 192x129x192, "
                                       "256x193x256 (4 pi x 2 x 2 pi, LES = DNS / 4) and widths Lx/16, Lx/32, Lx/48; "
                                       "one batch (one CUDA graph) per step",
                           "dns_points_per_step": pts, "plans": info, "graph_captures": captures,
                           "l2": f"inputs {12 * pts / 1e6:.0f} MB per step > 129 MB L2, no flush"},
                "roofline": roof, "cpu_baseline": cpu, "e2e": e2e, "accuracy": err, "clocks": clk.summary(),
                "gpu_launches": launches * args.steps}
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
        return
    if args.workload == "batch64":
        run_batch64(args)
        return
    import torch
    import torch.distributed as dist

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        dist.init_process_group("nccl", device_id=dev)

    import __graft_entry__ as entry
    if rank == 0:
        entry.build()      # one rank builds; the others wait for the library
    if world > 1:
        dist.barrier()
    from paper_1902_02508_gb300 import eles

    dns, les, delta, snaps = make_workload(args.workload, rank, args.snapshots)
    ns = len(snaps)
    prec = PREC[args.precision]
    plan = eles.filter_setup(dns, les, delta, precision=prec)
    dt = plan.dtype
    stream = torch.cuda.Stream(dev)
    u = torch.empty((ns, 3, dns.ny, dns.nz, dns.nx), device=dev, dtype=dt)
    for k, sk in enumerate(snaps):
        u[k] = torch.from_numpy(sk).to(dev, dt)
    ub = torch.empty((ns, 3, les.ny, les.nz, les.nx), device=dev, dtype=dt)
    tau = torch.empty((ns, 6, les.ny, les.nz, les.nx), device=dev, dtype=dt)
    pm = torch.empty((ns, 3, dns.ny), device=dev, dtype=torch.float64)
    torch.cuda.synchronize()

    eles.plan_reserve(plan, ns)

    def step(pl, uu, bb, tt, mm):
        eles.subfilter_stress_batch(pl, uu, bb, tt, mm, stream=stream)

    def timed(fn, steps, warmup):
        with torch.cuda.stream(stream):
            for _ in range(warmup):
                fn()
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with torch.cuda.stream(stream):
            e0.record(stream)
            for _ in range(steps):
                fn()
            e1.record(stream)
        torch.cuda.synchronize()
        return max_over_ranks(e0.elapsed_time(e1), dev, world)

    # --- device-resident throughput, with phase timing and clocks
    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            step(plan, u, ub, tau, pm)
    torch.cuda.synchronize()
    assert eles.check_device_error(plan, stream) == 0
    # the headline pass (no phase events), then a pass with phase events for
    # the per-kernel timing of the roofline
    with ClockSampler(local) as clk:
        ms = timed(lambda: step(plan, u, ub, tau, pm), args.steps, 0)
    eles.profile_enable(plan, True)
    timed(lambda: step(plan, u, ub, tau, pm), max(10, args.steps // 4), 1)
    phase_ms, calls = eles.profile_read(plan)
    eles.profile_enable(plan, False)
    pts_step = ns * dns.npts
    value = whole_job_rate(world, pts_step, args.steps, ms)

    # --- end to end: pinned host in, results back to pinned host
    hu = torch.empty(u.shape, dtype=dt).pin_memory()
    for k, sk in enumerate(snaps):
        hu[k] = torch.from_numpy(sk).to(dt)
    hb = torch.empty(ub.shape, dtype=dt).pin_memory()
    ht = torch.empty(tau.shape, dtype=dt).pin_memory()

    hpm = torch.empty(pm.shape, dtype=torch.float64).pin_memory()
    # the host-buffer entry point: copies of one snapshot in and of another's
    # results out overlap the compute of a third (set up outside the timing)
    io = eles.io_create(plan, 1)

    def e2e_step():
        eles.subfilter_stress_host(io, hu, hb, ht, hpm, stream=stream)

    e2e_steps = max(3, args.steps // 2)
    ms_e2e = timed(e2e_step, e2e_steps, 2)
    e2e = {"value": world * pts_step * e2e_steps / (ms_e2e / 1e3), "unit": UNIT,
           "h2d_bytes_per_step": hu.numel() * hu.element_size(),
           "d2h_bytes_per_step": hb.numel() * hb.element_size() + ht.numel() * ht.element_size()
           + hpm.numel() * hpm.element_size(),
           "api": "ef_subfilter_stress_host (pinned host buffers, 1-snapshot groups)"}
    io.close()

    from_json = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))) \
        if os.path.exists(os.path.join(ROOT, "MEASURED_PEAKS.json")) else {}

    # --- plain FP64 GPU filter on the same workload (the metric's comparator)
    fp64 = None
    if not args.no_fp64 and prec != 0:
        p64 = eles.filter_setup(dns, les, delta, precision=0)
        eles.plan_reserve(p64, ns)
        u64 = u.double()
        b64 = torch.empty(ub.shape, device=dev, dtype=torch.float64)
        t64 = torch.empty(tau.shape, device=dev, dtype=torch.float64)
        k64 = max(2, args.steps // 4)
        ms64 = timed(lambda: step(p64, u64, b64, t64, pm), k64, 1)
        fp64 = {"value": world * pts_step * k64 / (ms64 / 1e3), "unit": UNIT, "ms_per_step": ms64 / k64}
        # FP64 arithmetic bound: algorithmic flops per DNS point from the plan's tap counts (9 fields
        # formed; x, z and y contractions; the y pass also contracts the 9 cross-term fields) against
        # the FP64 FMA rate measured on this GB300 (1.68 DFMA per SM per clock, independent chains)
        tx, tz, ty = (eles.plan_info(p64, i) for i in (7, 8, 9))
        fpp = (9 + 18 * les.nx * tx / dns.nx + 18 * les.nz * tz / dns.nz * les.nx / dns.nx
               + 36 * les.ny * ty / dns.ny * les.nx * les.nz / (dns.nx * dns.nz))
        nsm = torch.cuda.get_device_properties(dev).multi_processor_count
        dpeak = 1.68 * 2 * nsm * from_json.get("sm_max_mhz", 2070.0) * 1e6
        ach = fp64["value"] / world * fpp
        fp64["roofline"] = {"bound": "alu", "achieved": ach / 1e12, "peak": dpeak / 1e12, "unit": "TFLOP/s",
                            "frac": ach / dpeak, "flop_per_point": fpp,
                            "peak_source": "FP64 FMA rate measured on GB300 (1.68 per SM per clock) x SMs x max clock"}
        del u64
        p64.close()

    # --- the differential filter of Sec. 3 (the paper's own kernel, a = 0.1) on snapshot 0, FP64
    differential = None
    if not args.no_fp64:
        differential = differential_measure(eles, torch, dns, les, u[0], stream, timed, from_json)

    # --- the learned closure, in its own configuration (rank 0)
    closure = None
    if not args.no_closure and rank == 0:
        closure = closure_measure(eles, torch, stream, from_json)

    # --- accuracy at the stated tolerance: snapshot 0 against the CPU oracle
    err = None
    cpu = None
    if rank == 0:
        from oracle import oracle as O
        ub_ref, tau_ref = O.subfilter_stress(dns, les, delta, snaps[0])
        got = tau[0].double().cpu().numpy()
        err = {"tau_max_abs_err_utau2": [float(x) for x in np.abs(got - tau_ref).max(axis=(1, 2, 3))],
               "tau_order": ["11", "12", "13", "22", "23", "33"],
               "ubar_max_abs_err": float(np.abs(ub[0].double().cpu().numpy() - ub_ref).max()),
               "tau_min_eigenvalue": {"path": min_eigenvalue(got), "oracle": min_eigenvalue(tau_ref),
                                      "note": "T is a weighted covariance for a positive kernel (PSD); "
                                              "u_tau^2 units"}}
        if not args.no_cpu_baseline and world == 1:
            v, cores, sample = oracle_time(dns, les, delta, snaps)
            cpu = {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample}

    # --- the other split-precision form on this workload, and both forms with
    # the wider filter of the configuration (Delta = Lx/32 on the Lx/64 workload);
    # after the accuracy check, since they reuse the output buffers
    forms = None
    if not args.no_forms and prec in (2, 3) and args.workload in ("re550_d64", "re550_d32"):
        forms = {}
        other = {"re550_d64": "re550_d32", "re550_d32": "re550_d64"}[args.workload]
        cases = [(args.workload, "tf32x2" if prec == 3 else "bf16x3"), (other, "bf16x3"), (other, "tf32x2")]
        for wl, pname in cases:
            forms[f"{wl}_{pname}"] = form_measure(eles, torch, wl, pname, dns, les, snaps, u, ub, tau, pm,
                                                  stream, timed, args.steps, peak_of(from_json), rank)

    # --- the coupled loop of Fig. 2 (filter of a DNS snapshot + one LES step);
    # last, since it reuses the output buffers
    apost = None
    if not args.no_apost and rank == 0:
        try:
            apost = apost_measure(eles, torch, dns, les, plan, u, ub, tau, stream, timed, args.steps)
        except Exception as ex:          # reported, the headline line still prints
            apost = {"error": f"{type(ex).__name__}: {ex}"}

    # --- roofline of the dominant phase (x-contraction: it alone reads the input)
    peak, peak_src = peak_of(from_json)
    xz_ms = phase_ms[0] / max(calls, 1)
    alg_bytes = (12 if prec != 0 else 24) * dns.npts * ns      # one launch covers the whole batch
    achieved = alg_bytes / (xz_ms / 1e3) / 1e9
    fused = eles.plan_info(plan, 11) == 1
    roof = {"bound": "hbm",
            "kernel": "xz_fused (x and z contractions + reference profile, reads the input once)" if fused
            else "x and z contractions (unfused)",
            "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
            "peak_source": peak_src,
            "traffic": traffic_from_profile(f"xz_ws_{args.workload}_{args.precision}", dns.npts * ns),
            "algorithmic_bytes_per_launch": alg_bytes,
            "phase_ms_per_step": {"xz": xz_ms, "y_recovery": phase_ms[2] / max(calls, 1)},
            "path_frac": (value / world) * (alg_bytes / (dns.npts * ns)) / 1e9 / peak}
    # x-z: the reference profile and the warp-specialised kernel (2 launches),
    # one fused launch, or 5 per snapshot + 2 unfused; y: profile, then
    # fragments + velocities + products + recovery (tensor cores) or 2 passes
    ytc = eles.plan_info(plan, 13) == 1
    xv = eles.plan_info(plan, 10)
    per_call_launches = (2 if xv == 3 else 1 if fused else 2 + 5 * ns) + 1 + (4 if ytc else 2)
    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None,
                "dtype": {"fp32": "f32", "fp64": "f64", "bf16x3": "bf16x3", "tf32x2": "tf32x2"}[args.precision],
                "data": "synthetic (seeded solenoidal channel fields, Reichardt mean profile)",
                "config": workload_config(args.workload, args.precision, args.snapshots),
                "roofline": roof, "cpu_baseline": cpu, "e2e": e2e, "fp64_plain": fp64,
                "accuracy": err, "split_forms": forms, "closure": closure, "differential": differential,
                "apost": apost, "clocks": clk.summary(),
                "gpu_launches": per_call_launches * args.steps,
                "x_variant": eles.plan_info(plan, 10)}
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
