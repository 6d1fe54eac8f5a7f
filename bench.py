#!/usr/bin/env python3
"""Benchmark of the multi-RHS Dirac operators (Wilson, Brillouin, staggered).

Workload (one "step"): apply D_W, D_B and D_S once each to N_v = 12
right-hand sides on a 16^3 x 32 lattice, N_c = 3, complex FP32, random SU(3)
links exp(i 0.4 sum_k a_k lambda_k), Gaussian sources.  The metric is
Gflop/s counted with the paper's per-site flop numbers (App. E: 1368, 30168,
582 per site and RHS), whole job, inputs resident in HBM.

Also reported: per-operator Gflop/s, algorithmic GB/s and roofline
fractions, an N_v sweep, the end-to-end rate through the C ABI from pinned
host memory (copies inside the timed region), the FP64 CPU oracle on a
bounded sample of the same workload, and SM clocks sampled during the timed
region.  ``--solve`` adds the mixed-precision vs FP32-inner defect-correction
time to 1e-10.  ``--impl reference`` times the oracle alone.

Multi-GPU (torchrun): the operators do not shard here; every rank runs an
independent replica and the aggregate is the sum over ranks / max time.
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)
try:
    _CORES = len(os.sched_getaffinity(0))
except AttributeError:
    _CORES = os.cpu_count() or 1
os.environ.setdefault("OMP_NUM_THREADS", str(_CORES))

METRIC = "Gflop/s & HBM GB/s of D on Nv=12 RHS, FP32; mixed vs FP32 CG time to 1e-10"
DIMS = (16, 16, 16, 32)
NC = 3
NV = 12
BC = (1, 1, 1, -1)
EPS = 0.4
MASS = {0: 0.1, 1: 0.1, 2: 0.05, 3: 0.1, 4: 0.1, 5: 0.1, 6: 0.1}   # Laplace kinds: m of A
FP32_LANES_PER_SM = 128
# bare masses of the precision study (32^3x64, eps = 0.6, gauge seed 99)
# that put cond(D^dag D) near 1e6, from a Lanczos scan of FP32 CG on that
# field; every solve reports the Lanczos estimate it actually saw
SOLVE_MASS = {"staggered": 0.00265, "wilson": -1.961}


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=1000)
    p.add_argument("--warmup", type=int, default=20)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-sweep", action="store_true")
    p.add_argument("--solve", action="store_true", help="full config-3 study: every sloppy precision and mode")
    p.add_argument("--no-solve", action="store_true", help="skip the default config-3 FP32 vs mixed comparison")
    p.add_argument("--solve-budget", type=float, default=240.0,
                   help="wall-clock seconds the default solver comparison may use")
    p.add_argument("--no-large", action="store_true", help="skip the 32^3x64 operator timing")
    p.add_argument("--no-nc-sweep", action="store_true", help="skip the N_c sweep (24^3x48, N_v = 24)")
    p.add_argument("--no-batch", action="store_true", help="skip the config-4 batched-solve measurement")
    p.add_argument("--ncu", action="store_true", help="short run for profiler launch lists (no extras)")
    p.add_argument("--csw", type=float, default=0.0,
                   help="time D_W and D_B with the clover term of this c_SW (0: the plain operators)")
    p.add_argument("--no-clover", action="store_true", help="skip the separate clover-term measurement")
    p.add_argument("--no-laplace", action="store_true", help="skip the separate Laplace-operator measurement")
    p.add_argument("--ops", default="wilson,brillouin,staggered",
                   help="profiling only: subset of operators to create and time")
    p.add_argument("--fixed", default=None,
                   help="profiling only: LAYOUT:VR,MINB,BLOCK (LAYOUT outer|inner), or name=LAYOUT:...;name=... per "
                        "operator, instead of the autotuned choice")
    return p.parse_args()


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return dict(hbm=float(d["hbm_gbs"]), sm_max=float(d.get("sm_max_mhz", 2070.0)), source="measured")
    except Exception:
        return dict(hbm=6800.0, sm_max=2070.0, source="fallback")


def alg_bytes_per_site(kind, nc, nv, eb=4, clover=False):
    """Compulsory bytes per site and apply: spinor in + out once, links once
    (Brillouin: the 80 stored W links of this implementation), plus the four
    N_c x N_c clover blocks per site when the clover term is applied."""
    spin = 1 if kind in (2, 5, 6) else 4               # staggered, colour-only Laplace kinds
    vec = nc * spin * nv * 2 * eb
    links = (80 if kind in (1, 4, 6) else 4) * nc * nc * 2 * eb   # Brillouin kinds: W links
    return 2 * vec + links + (4 * nc * nc * 2 * eb if clover else 0)


def ncu_traffic(op_name):
    """DRAM bytes per launch (dram__bytes_read.sum + dram__bytes_write.sum) from
    the committed ncu summary of this kernel, or None when the kernel source
    changed since the counters were taken."""
    import hashlib
    prof = os.path.join(ROOT, "profiles", "%s_kernel_16x16x16x32_nv12.md" % op_name)
    csrc = os.path.join(ROOT, "paper_2112_14640_gb300", "csrc")
    try:
        text = open(prof).read()
        h = hashlib.sha256()
        srcs = {"wilson": ("wilson.cuh", "clover.cuh"), "staggered": ("staggered.cuh",),
                "brillouin": ("brillouin.cuh", "bril_dirs.h", "clover.cuh"),
                "wlap": ("laplace.cuh", "bril_dirs.h"), "blap": ("laplace.cuh", "bril_dirs.h")}[op_name] + \
            ("common.cuh",)
        for f in srcs:
            h.update(open(os.path.join(csrc, f), "rb").read())
        fields = dict(l.split(":", 1) for l in text.splitlines() if ":" in l and not l.startswith(("#", " ", "|")))
        if fields.get("kernel_source_sha256_16", "").strip() != h.hexdigest()[:16]:
            return None
        return int(fields["traffic_bytes_per_launch"].strip())
    except Exception:
        return None


class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.idx = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.idx), "--query-gpu=" + self.FIELDS, "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 9:
                rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        smax = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": reasons, "samples": len(rows)}


def dist_setup(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def max_over_ranks(x, world, device):
    """The largest x over all ranks (one all-reduce; x itself when world = 1)."""
    if world == 1:
        return float(x)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(units_per_rank, world, ms_step):
    """Whole-job throughput of independent replicas: the units all ranks
    processed per second of the slowest rank's step time."""
    return units_per_rank * world / (ms_step * 1e-3)


# ------------------------------------------------------------------ oracle leg
def oracle_rate(target_s, U_np, sources):
    """FP64 CPU oracle on a bounded sample of output sites of each operator.
    Returns (Gflop/s over the three operators, description of the sample)."""
    import numpy as np

    import oracle as O

    V = int(np.prod(DIMS))
    rng = np.random.default_rng(7)
    total_flop, total_t, desc = 0.0, 0.0, []
    for kind in (0, 1, 2):
        ref = O.Operator(kind, U_np, BC)
        src = sources[kind]
        fps = O.flops_per_site(kind, NC) * NV

        def run(ns):
            sites = rng.choice(V, ns, replace=False)
            field = O.build_w_sites(ref.Up, sites) if kind == 1 else ref.Up
            t0 = time.perf_counter()
            O.stencil_sites(kind, field, MASS[kind], src, sites)
            return time.perf_counter() - t0

        probe = 32 if kind == 1 else 512
        dt = run(probe)
        ns = int(min(V, max(probe, probe * target_s / max(dt, 1e-6))))
        dt = run(ns)
        total_flop += fps * ns
        total_t += dt
        desc.append("%s %d sites" % (O.KIND_NAMES[kind], ns))
    return total_flop / total_t / 1e9, "; ".join(desc) + " of 16^3x32, Nv=12 (FP64 oracle, sampled sites)"


def config_dict():
    return {"workload": "D_W + D_B + D_S apply, 16^3x32, Nc=3, Nv=12, FP32 storage+arithmetic",
            "lattice": "16x16x16x32", "nc": NC, "nv": NV, "bc": "antiperiodic t",
            "links": "random SU(3), eps=0.4", "l2": "working set > L2: each step streams >1 GB between reuses"}


def run_reference(args):
    world, rank, _ = dist_setup(args)
    if rank != 0:
        return
    import numpy as np  # noqa: F401

    from paper_2112_14640_gb300 import inputs as I
    U = I.gauge_field(DIMS, NC, EPS, 1234)
    sources = {k: I.source(DIMS, NC, NV, 4321 + k, staggered=(k == 2)) for k in (0, 1, 2)}
    per_step = max(0.05, min(5.0, 120.0 / max(1, args.steps + args.warmup)))
    for _ in range(min(args.warmup, 1)):
        oracle_rate(per_step / 3, U, sources)
    rates, descs, t0 = [], None, time.perf_counter()
    for _ in range(args.steps):
        r, descs = oracle_rate(per_step / 3, U, sources)
        rates.append(r)
    wall = time.perf_counter() - t0
    value = statistics.median(rates)
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "Gflop/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000 * wall / max(1, args.steps),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": config_dict(),
            "cpu_baseline": {"value": value, "unit": "Gflop/s", "cores": _CORES, "kind": "oracle",
                             "sample": descs},
            "e2e": {"value": value, "unit": "Gflop/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# -------------------------------------------------------------------- our leg
def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    import numpy as np
    import torch

    world, rank, local = dist_setup(args)
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    import __graft_entry__
    __graft_entry__.build()
    from paper_2112_14640_gb300 import dirac as D
    from paper_2112_14640_gb300 import inputs as I

    pk = peaks()
    U_np = I.gauge_field(DIMS, NC, EPS, 1234)
    U = torch.from_numpy(U_np).cuda()
    names = {v: k for k, v in D.KIND_NAMES.items()}
    kinds = tuple(names[o] for o in args.ops.split(","))
    sources = {k: I.source(DIMS, NC, NV, 4321 + k, staggered=(k in (D.STAGGERED, D.WSUV, D.BSUV))) for k in kinds}
    ops, xs, ys = {}, {}, {}
    launch, layout_ms = {}, {}
    stream0 = torch.cuda.current_stream()

    def quick_ms(op, x, y, m0, reps=20):
        for _ in range(3):
            op.apply(x, y, m0=m0)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream0)
        for _ in range(reps):
            op.apply(x, y, m0=m0)
        e1.record(stream0)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps

    for k in kinds:
        if args.fixed:
            spec = args.fixed
            if "=" in spec:   # per operator: name=LAYOUT:VR,MINB,BLOCK;...
                spec = dict(x.split("=") for x in spec.split(";"))[D.KIND_NAMES[k]]
            lay_s, var = spec.split(":")
            lay = D.SITE_INNER if lay_s == "inner" else D.SITE_OUTER
            op = D.DiracOp(k, U, NV, BC, D.F32, layout=lay)
            op.set_launch(*[int(v) for v in var.split(",")])
            xs[k] = op.to_prec(op.from_site_outer(torch.from_numpy(sources[k]).cuda()))
            ys[k] = op.new_vector(zero=False)
            ops[k] = op
            layout_ms[D.KIND_NAMES[k]] = {"chosen": lay_s, "fixed": True}
            launch[D.KIND_NAMES[k]] = op.get_launch()
            continue
        # untimed setup: for each vector layout pick the launch variant, then
        # keep the faster layout for the timed step
        cand = {}
        for lay in (D.SITE_OUTER, D.SITE_INNER):
            op = D.DiracOp(k, U, NV, BC, D.F32, layout=lay)
            x = op.to_prec(op.from_site_outer(torch.from_numpy(sources[k]).cuda()))
            y = op.new_vector(zero=False)
            op.autotune(MASS[k])
            cand[lay] = (quick_ms(op, x, y, MASS[k]), op, x, y)
        best = min(cand, key=lambda l: cand[l][0])
        layout_ms[D.KIND_NAMES[k]] = {"site_outer_ms": cand[D.SITE_OUTER][0], "site_inner_ms": cand[D.SITE_INNER][0],
                                      "chosen": "site_inner" if best == D.SITE_INNER else "site_outer"}
        _, ops[k], xs[k], ys[k] = cand[best]
        cand[1 - best][1].close()
        launch[D.KIND_NAMES[k]] = ops[k].get_launch()
    clov = {k: bool(args.csw) and k != D.STAGGERED for k in kinds}
    for k in kinds:
        if clov[k]:
            ops[k].set_clover(args.csw, U)
            if not args.fixed:
                ops[k].autotune(MASS[k])
                launch[D.KIND_NAMES[k]] = ops[k].get_launch()
    V = int(np.prod(DIMS))
    flop = {k: (D.flops_per_site(k, NC) + (D.clover_flops_per_site(NC) if clov[k] else 0)) * V * NV
            for k in kinds}
    step_flop = sum(flop.values())
    stream = torch.cuda.current_stream()

    def step(evs=None):
        for i, k in enumerate(kinds):
            if evs is not None:
                evs[i].record(stream)
            ops[k].apply(xs[k], ys[k], m0=MASS[k])
        if evs is not None:
            evs[len(kinds)].record(stream)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    K = args.steps
    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(len(kinds) + 1)] for _ in range(K)]
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    t_start = torch.cuda.Event(enable_timing=True)
    t_end = torch.cuda.Event(enable_timing=True)
    t_start.record(stream)
    for s in range(K):
        step(evs[s])
    t_end.record(stream)
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    clk = clocks.stop()
    ms_total = max_over_ranks(t_start.elapsed_time(t_end), world, "cuda")
    ms_step = ms_total / K
    value = job_rate(step_flop, world, ms_step) / 1e9

    per_op = {}
    # the ALU roof: the FMA probe kernel measured on this device (best of 3),
    # next to the nominal count from the device's own SM count
    sm_count = torch.cuda.get_device_properties(local).multi_processor_count
    fp32_peak = max(D.measure_fp32_peak()[0] for _ in range(3))        # TFLOP/s
    fp32_nominal = sm_count * FP32_LANES_PER_SM * 2 * pk["sm_max"] * 1e6 / 1e12
    for i, k in enumerate(kinds):
        times = [evs[s][i].elapsed_time(evs[s][i + 1]) for s in range(K)]
        t_ms = statistics.mean(times)
        gbytes = alg_bytes_per_site(k, NC, NV, clover=clov[k]) * V / 1e9
        per_op[D.KIND_NAMES[k]] = {
            "ms": t_ms, "gflops": flop[k] / (t_ms * 1e-3) / 1e9, "alg_GBps": gbytes / (t_ms * 1e-3),
            "hbm_frac": gbytes / (t_ms * 1e-3) / pk["hbm"],
            "alu_frac": flop[k] / (t_ms * 1e-3) / 1e12 / fp32_peak}
    dom = max(kinds, key=lambda k: per_op[D.KIND_NAMES[k]]["ms"])
    if len(kinds) < 3:
        if rank == 0:
            print(json.dumps({"profiling_subset": args.ops, "per_op": per_op, "ms_per_step": ms_step}), flush=True)
        return
    d = per_op[D.KIND_NAMES[dom]]
    if dom == D.BRILLOUIN:
        roof = {"bound": "alu", "achieved": d["gflops"] / 1e3, "peak": fp32_peak, "unit": "TFLOP/s",
                "frac": d["gflops"] / 1e3 / fp32_peak, "traffic": ncu_traffic("brillouin"),
                "traffic_unit": "bytes/launch", "kernel": "brillouin_kernel",
                "peak_source": "measured: FMA probe kernel (dirac_measure_fp32_peak) on %d SMs; nominal "
                               "%d x 128 lanes x 2 x %.0f MHz = %.1f TFLOP/s" % (sm_count, sm_count, pk["sm_max"],
                                                                               fp32_nominal)}
    else:
        roof = {"bound": "hbm", "achieved": d["alg_GBps"], "peak": pk["hbm"], "unit": "GB/s",
                "frac": d["hbm_frac"], "traffic": ncu_traffic(D.KIND_NAMES[dom]), "traffic_unit": "bytes/launch",
                "kernel": D.KIND_NAMES[dom] + "_kernel",
                "peak_source": pk["source"]}
    rooflines = {
        "wilson": {"bound": "hbm", "achieved": per_op["wilson"]["alg_GBps"], "peak": pk["hbm"], "unit": "GB/s",
                   "frac": per_op["wilson"]["hbm_frac"], "traffic": ncu_traffic("wilson")},
        "staggered": {"bound": "hbm", "achieved": per_op["staggered"]["alg_GBps"], "peak": pk["hbm"],
                      "unit": "GB/s", "frac": per_op["staggered"]["hbm_frac"], "traffic": ncu_traffic("staggered")},
        "brillouin": {"bound": "alu", "achieved": per_op["brillouin"]["gflops"] / 1e3, "peak": fp32_peak,
                      "unit": "TFLOP/s", "frac": per_op["brillouin"]["alu_frac"], "traffic": ncu_traffic("brillouin")},
    }

    cfg = config_dict()
    if args.csw:
        cfg["workload"] += ", clover term c_SW=%g on D_W and D_B" % args.csw
        cfg["csw"] = args.csw
    line = {"metric": METRIC, "value": value, "unit": "Gflop/s", "n_gpus": world, "steps": K,
            "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic", "config": cfg,
            "gpu_launches": K * len(kinds), "roofline": roof, "rooflines": rooflines, "per_op": per_op,
            "clocks": clk, "peaks_source": pk["source"], "launch_variants": launch, "layouts": layout_ms,
            "device": {"sm_count": sm_count, "fp32_peak_measured_tflops": fp32_peak,
                       "fp32_peak_nominal_tflops": fp32_nominal}}

    if not args.ncu:
        # end to end through the C ABI from pinned host memory, copies included
        hin = {k: xs[k].cpu().pin_memory() for k in kinds}
        hout = {k: torch.empty_like(hin[k]).pin_memory() for k in kinds}
        Ke = max(3, min(K, 30))
        for k in kinds:
            ops[k].apply_host(hin[k], hout[k], m0=MASS[k])
        # one step = the three host applies enqueued back to back (each
        # operator's copies overlap the others' stencils), one wait per step;
        # the longest stencil first, so that its copies go out last
        order = sorted(kinds, key=lambda k: -per_op[D.KIND_NAMES[k]]["ms"])
        for _ in range(max(3, args.warmup)):   # untimed steps of the same form
            for k in order:
                ops[k].apply_host_async(hin[k], hout[k], m0=MASS[k])
            torch.cuda.current_stream().synchronize()
        enq = 0.0
        t0 = time.perf_counter()
        for _ in range(Ke):
            te = time.perf_counter()
            for k in order:
                ops[k].apply_host_async(hin[k], hout[k], m0=MASS[k])
            enq += time.perf_counter() - te
            torch.cuda.current_stream().synchronize()
        dt = (time.perf_counter() - t0) / Ke
        nbytes = sum(ops[k].vec_bytes() for k in kinds)
        line["e2e"] = {"value": step_flop / dt / 1e9, "unit": "Gflop/s", "h2d_bytes_per_step": nbytes,
                       "d2h_bytes_per_step": nbytes, "ms_per_step": dt * 1e3,
                       "host_enqueue_ms_per_step": enq / Ke * 1e3,
                       "pinned_copy": pinned_copy_rate(torch, ops[kinds[0]].vec_bytes())}

    if not args.ncu and not args.no_sweep:
        sweep = {}
        for nv in (1, 4, 12, 24):
            row = {}
            for k in kinds:
                op = D.DiracOp(k, U, nv, BC, D.F32, layout=ops[k].layout)
                op.autotune(MASS[k])
                x = op.new_vector()
                x.real.normal_()
                y = op.new_vector(zero=False)
                for _ in range(3):
                    op.apply(x, y, m0=MASS[k])
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                reps = 20
                e0.record(stream)
                for _ in range(reps):
                    op.apply(x, y, m0=MASS[k])
                e1.record(stream)
                torch.cuda.synchronize()
                t = e0.elapsed_time(e1) / reps * 1e-3
                row[D.KIND_NAMES[k]] = {"gflops": D.flops_per_site(k, NC) * V * nv / t / 1e9,
                                        "alg_GBps": alg_bytes_per_site(k, NC, nv) * V / t / 1e9}
                op.close()
            sweep["nv=%d" % nv] = row
        line["nv_sweep"] = sweep

    if not args.ncu and not args.no_clover and not args.csw:
        line["clover"] = clover_measurement(D, U, ops, xs, ys, per_op, pk, fp32_peak, quick_ms)

    if not args.ncu and not args.no_laplace:
        line["laplace"] = laplace_measurement(D, U, pk, fp32_peak, quick_ms)

    if not args.ncu and not args.no_large:
        line["large_lattice"] = large_lattice_timing(D, I, torch, pk, fp32_peak)
    if not args.ncu:
        line["force"] = force_timing(D, I, torch)
        line["link_setup"] = link_setup_timing(D, I, torch)
    if not args.ncu and not args.no_nc_sweep:
        line["nc_sweep"] = nc_sweep(D, I, torch)
    if args.solve:
        line["solve"] = solver_comparison(D, I, torch)
    elif not args.ncu and not args.no_solve:
        line["solve"] = solve_default(D, I, torch, args.solve_budget)
    if not args.ncu and not args.no_batch:
        line["batch"] = batch_measurement(D, I, torch)

    if rank == 0 and world == 1 and not args.no_cpu_baseline and not args.ncu:
        rate, sample = oracle_rate(6.0, U_np, sources)
        line["cpu_baseline"] = {"value": rate, "unit": "Gflop/s", "cores": _CORES, "kind": "oracle",
                                "sample": sample}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


def pinned_copy_rate(torch, nbytes, reps=5):
    """Plain copies of one vector's bytes between pinned host memory and the
    device (one cudaMemcpyAsync each), GB/s per direction: the link rate the
    end-to-end apply's copies are measured against."""
    h = torch.empty(nbytes, dtype=torch.uint8).pin_memory()
    d = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
    st = torch.cuda.current_stream()
    out = {"bytes": nbytes}
    for name, fn in (("h2d_GBps", lambda: d.copy_(h, non_blocking=True)),
                     ("d2h_GBps", lambda: h.copy_(d, non_blocking=True))):
        fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(st)
        for _ in range(reps):
            fn()
        e1.record(st)
        torch.cuda.synchronize()
        out[name] = nbytes * reps / (e0.elapsed_time(e1) * 1e-3) / 1e9
    # both directions at once, on two streams: the rate the overlapped
    # end-to-end step can reach at best (bytes moved in both directions)
    h2 = torch.empty(nbytes, dtype=torch.uint8).pin_memory()
    d2 = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
    s1, s2 = torch.cuda.Stream(), torch.cuda.Stream()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(reps):
        with torch.cuda.stream(s1):
            d.copy_(h, non_blocking=True)
        with torch.cuda.stream(s2):
            h2.copy_(d2, non_blocking=True)
    torch.cuda.synchronize()
    out["bidirectional_GBps"] = 2 * nbytes * reps / (time.perf_counter() - t0) / 1e9
    del h, d, h2, d2
    return out


def large_lattice_timing(D, I, torch, pk, fp32_peak, dims=(32, 32, 32, 64)):
    """D_W, D_B and D_S at 32^3x64 (16x the benchmark volume: every operand is
    larger than L2), N_v = 12, FP32, site-inner, autotuned there; two input
    and output vector sets alternate between applies."""
    import numpy as np
    V = int(np.prod(dims))
    U = torch.from_numpy(I.gauge_field(dims, NC, EPS, 4242)).cuda()
    st = torch.cuda.current_stream()
    out = {"lattice": "x".join(map(str, dims)), "nv": NV}
    for k in (D.WILSON, D.STAGGERED, D.BRILLOUIN):
        op = D.DiracOp(k, U, NV, BC, D.F32, layout=D.SITE_INNER)
        op.autotune(MASS[k])
        xs = [op.new_vector() for _ in range(2)]
        for x in xs:
            x.real.normal_()
        ys = [op.new_vector(zero=False) for _ in range(2)]
        reps = 4 if k == D.BRILLOUIN else 20
        for i in range(2):
            op.apply(xs[i], ys[i], m0=MASS[k])
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(st)
        for i in range(reps):
            op.apply(xs[i % 2], ys[i % 2], m0=MASS[k])
        e1.record(st)
        torch.cuda.synchronize()
        t = e0.elapsed_time(e1) / reps * 1e-3
        flop = D.flops_per_site(k, NC) * V * NV
        gbytes = alg_bytes_per_site(k, NC, NV) * V / 1e9
        row = {"ms": t * 1e3, "gflops": flop / t / 1e9, "alg_GBps": gbytes / t, "launch": op.get_launch()}
        if k == D.BRILLOUIN:
            row["alu_frac"] = flop / t / 1e12 / fp32_peak
        else:
            row["hbm_frac"] = gbytes / t / pk["hbm"]
        out[D.KIND_NAMES[k]] = row
        op.close()
        del xs, ys
        torch.cuda.empty_cache()
    del U
    torch.cuda.empty_cache()
    return out


def nc_sweep(D, I, torch, dims=(24, 24, 24, 48), nv=24, ncs=(2, 3, 4, 6, 8)):
    """Gflop/s (App. E counts) of D_W, D_B and D_S as a function of N_c at
    24^3x48, N_v = 24, FP32, site-inner, autotuned: the workload of the
    paper's N_c table (Sec. "Dependence on compile-time parameters")."""
    import numpy as np
    V = int(np.prod(dims))
    st = torch.cuda.current_stream()
    out = {"lattice": "x".join(map(str, dims)), "nv": nv}
    for nc in ncs:
        U = torch.from_numpy(I.gauge_field(dims, nc, EPS, 900 + nc)).cuda().to(torch.complex64)
        row = {}
        for k in (D.WILSON, D.BRILLOUIN, D.STAGGERED):
            op = D.DiracOp(k, U, nv, BC, D.F32, layout=D.SITE_INNER)
            op.autotune(MASS[k])
            x = op.new_vector()
            x.real.normal_()
            y = op.new_vector(zero=False)
            op.apply(x, y, m0=MASS[k])
            reps = 2 if k == D.BRILLOUIN else 10
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(st)
            for _ in range(reps):
                op.apply(x, y, m0=MASS[k])
            e1.record(st)
            torch.cuda.synchronize()
            t = e0.elapsed_time(e1) / reps * 1e-3
            row[D.KIND_NAMES[k]] = {"ms": t * 1e3, "gflops": D.flops_per_site(k, nc) * V * nv / t / 1e9,
                                    "alg_GBps": alg_bytes_per_site(k, nc, nv) * V / t / 1e9}
            op.close()
            del x, y
            torch.cuda.empty_cache()
        out["nc=%d" % nc] = row
        del U
        torch.cuda.empty_cache()
    return out


def link_setup_timing(D, I, torch, dims=(16, 16, 16, 32), nv=12):
    """A new gauge field handed to an existing operator (dirac_op_update_links:
    boundary phases, and for D_B the 80 path-averaged W links of every site),
    as in every molecular-dynamics step of an HMC: time per update, FP32."""
    import numpy as np
    U = torch.from_numpy(I.gauge_field(dims, NC, EPS, 11)).cuda()
    st = torch.cuda.current_stream()
    out = {"lattice": "x".join(map(str, dims))}
    for k in (D.WILSON, D.BRILLOUIN):
        op = D.DiracOp(k, U, nv, BC, D.F32)
        op.update_links(U)
        reps = 5
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(st)
        for _ in range(reps):
            op.update_links(U)
        e1.record(st)
        torch.cuda.synchronize()
        out[D.KIND_NAMES[k] + "_ms"] = e0.elapsed_time(e1) / reps
        op.close()
    del U
    torch.cuda.empty_cache()
    return out


def force_timing(D, I, torch, dims=(16, 16, 16, 32), nv=4):
    """The fermion-force kernels of the differentiation workload (16^3x32,
    N_v = 4, FP32; Wilson, staggered and Brillouin): time per call and the algorithmic
    bytes it moves (psi and chi read once, links read once, the force
    written once)."""
    import numpy as np
    V = int(np.prod(dims))
    U = torch.from_numpy(I.gauge_field(dims, NC, EPS, 7)).cuda()
    st = torch.cuda.current_stream()
    out = {"lattice": "x".join(map(str, dims)), "nv": nv}
    for k in (D.WILSON, D.STAGGERED, D.BRILLOUIN):
        op = D.DiracOp(k, U, nv, BC, D.F32)
        psi, chi = op.new_vector(), op.new_vector()
        psi.real.normal_()
        chi.real.normal_()
        op.force(psi, chi)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        reps = 3 if k == D.BRILLOUIN else 20
        e0.record(st)
        for _ in range(reps):
            op.force(psi, chi)
        e1.record(st)
        torch.cuda.synchronize()
        t = e0.elapsed_time(e1) / reps * 1e-3
        spin = 1 if k == D.STAGGERED else 4
        gbytes = V * (2 * NC * spin * nv * 8 + 2 * 4 * NC * NC * 8) / 1e9
        out[D.KIND_NAMES[k]] = {"ms": t * 1e3, "alg_GBps": gbytes / t, "hbm_frac": gbytes / t / peaks()["hbm"]}
        if k == D.BRILLOUIN:   # plus the 216 link terms per site written and read back
            out[D.KIND_NAMES[k]]["scratch_GB"] = V * 216 * NC * NC * 8 / 1e9
        op.close()
    return out


def solve_default(D, I, torch, budget_s):
    """The precision comparison of the metric, bounded in time: CG on D^dag D
    to an FP64 residual of 1e-10 (32^3x64, N_c = 3, N_v = 12, eps = 0.6,
    masses at cond(D^dag D) ~ 1e6), the FP32 sloppy iteration (the baseline)
    against the adaptive FP16 (FP32 links) sloppy iteration, reliable updates
    in FP64.  The two modes alternate, up to three times each per operator,
    while the wall-clock budget lasts; every time is reported."""
    dims = (32, 32, 32, 64)
    U = torch.from_numpy(I.gauge_field(dims, NC, 0.6, 99)).cuda()
    out = {"lattice": "32x32x32x64", "nv": NV, "eps": 0.6, "tol": 1e-10, "budget_s": budget_s}
    t_start = time.perf_counter()
    modes = (("f32", D.F32, D.LINKS_NATIVE, D.MIXED_RELIABLE), ("f16+f32links+adaptive", D.F16, D.LINKS_F32,
                                                               D.MIXED_ADAPTIVE))
    per_kind = budget_s / 2
    for kind in (D.STAGGERED, D.WILSON):
        t_kind = time.perf_counter()
        name = D.KIND_NAMES[kind]
        m0 = SOLVE_MASS[name]
        op = D.DiracOp(kind, U, NV, BC, D.F64, layout=D.SITE_INNER)
        for prec, links in ((D.F32, D.LINKS_NATIVE), (D.F16, D.LINKS_F32)):
            tw = D.DiracOp(kind, U, NV, BC, prec, layout=D.SITE_INNER, link_storage=links)
            tw.autotune(m0)
            tw.close()
        b = op.to_prec(op.from_site_outer(torch.from_numpy(
            I.source(dims, NC, NV, 5, staggered=(kind == D.STAGGERED))).cuda()))
        row = {"m0": m0}
        for rep in range(3):
            for mname, inner, links, mode in modes:
                if rep > 0 and time.perf_counter() - t_kind > per_kind:
                    break
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                x, st = op.solve(b, m0=m0, solver=D.CG_NORMAL, tol=1e-10, maxit=60000, inner_prec=inner,
                                 sloppy_links=links, mixed_mode=mode)
                torch.cuda.synchronize()
                r = row.setdefault(mname, {"seconds": [], "iters": [], "status": [], "max_true_relres": [],
                                           "cond_lanczos": None})
                r["seconds"].append(time.perf_counter() - t0)
                r["iters"].append(st["iters"])
                r["status"].append(st["status"])
                r["max_true_relres"].append(max(st["true_relres"]))
                r["max_normal_relres"] = max(st["relres"])
                r["cond_lanczos"] = max(st["lambda_max"]) / max(min(st["lambda_min"]), 1e-300)
                r["ms_per_iter"] = 1e3 * st["seconds"] / max(st["iters"], 1)
                if inner != D.F32:
                    # the 16-bit phase: how far it carried the solve and what its iterations cost
                    r["iters_16bit"] = st["iters_16bit"]
                    r["ms_per_iter_16bit"] = 1e3 * st["seconds_16bit"] / max(st["iters_16bit"], 1)
                del x
        for mname, *_ in modes:
            if mname in row:
                sec = row[mname]["seconds"]
                row[mname]["median_s"] = statistics.median(sec)
                row[mname]["spread_s"] = max(sec) - min(sec)
        if "f32" in row and modes[1][0] in row:
            row["mixed_over_f32"] = row[modes[1][0]]["median_s"] / row["f32"]["median_s"]
        out[name] = row
        op.close()
        torch.cuda.empty_cache()
    out["wall_s"] = time.perf_counter() - t_start
    del U
    torch.cuda.empty_cache()
    return out


def clover_measurement(D, U, ops, xs, ys, per_op, pk, fp32_peak, quick_ms, csw=1.0):
    """D_W + C and D_B + C (c_SW = 1, F from the same field) on the timed
    workload, in the layout chosen for the plain operator and an autotuned
    launch variant: time per apply, Gflop/s with the 64 N_c^2 clover flops of
    App. E added, algorithmic bandwidth with the clover blocks added, and the
    cost over the plain operator timed the same way."""
    import numpy as np
    V = int(np.prod(DIMS))
    out = {"csw": csw}
    for k in (D.WILSON, D.BRILLOUIN):
        if k not in ops:
            continue
        op = D.DiracOp(k, U, NV, BC, D.F32, layout=ops[k].layout)
        op.set_clover(csw, U)
        op.autotune(MASS[k])
        plain_ms = quick_ms(ops[k], xs[k], ys[k], MASS[k], reps=50)
        ms = quick_ms(op, xs[k], ys[k], MASS[k], reps=50)
        flop = (D.flops_per_site(k, NC) + D.clover_flops_per_site(NC)) * V * NV
        gbytes = alg_bytes_per_site(k, NC, NV, clover=True) * V / 1e9
        out[D.KIND_NAMES[k]] = {
            "ms": ms, "plain_ms": plain_ms, "overhead": ms / plain_ms - 1.0,
            "gflops": flop / (ms * 1e-3) / 1e9, "alg_GBps": gbytes / (ms * 1e-3),
            "hbm_frac": gbytes / (ms * 1e-3) / pk["hbm"], "alu_frac": flop / (ms * 1e-3) / 1e12 / fp32_peak,
            "launch": op.get_launch()}
        op.close()
    return out


def laplace_measurement(D, U, pk, fp32_peak, quick_ms, m=0.1):
    """The Laplace operators A = -1/2 Lap + m^2/2 (wlap, blap on Wilson-type
    vectors; wsuv, bsuv on colour-only vectors) on the timed workload
    (16^3x32, N_c = 3, N_v = 12, FP32, site-inner, autotuned): time per
    apply, Gflop/s with the App. E counts, algorithmic bandwidth, and the
    fraction of the binding roof (FP32 peak for blap, HBM copy otherwise)."""
    import numpy as np
    import torch
    V = int(np.prod(DIMS))
    out = {"m": m}
    for k in (D.WLAP, D.BLAP, D.WSUV, D.BSUV):
        op = D.DiracOp(k, U, NV, BC, D.F32, layout=D.SITE_INNER)
        x = op.new_vector()
        x.real.normal_()
        y = op.new_vector(zero=False)
        op.autotune(m)
        ms = quick_ms(op, x, y, m, reps=50)
        flop = D.flops_per_site(k, NC) * V * NV
        gbytes = alg_bytes_per_site(k, NC, NV) * V / 1e9
        alu = k == D.BLAP
        out[D.KIND_NAMES[k]] = {
            "ms": ms, "gflops": flop / (ms * 1e-3) / 1e9, "alg_GBps": gbytes / (ms * 1e-3),
            "bound": "alu" if alu else "hbm",
            "frac": (flop / (ms * 1e-3) / 1e12 / fp32_peak) if alu else gbytes / (ms * 1e-3) / pk["hbm"],
            "traffic": ncu_traffic(D.KIND_NAMES[k]) if k in (D.WLAP, D.BLAP) else None,
            "launch": op.get_launch()}
        op.close()
        del x, y
        torch.cuda.empty_cache()
    return out


# FP32 CG on the normal equations of the light staggered operator sits at an
# FP32 floor of a few 1e-6 (measured); 1e-5 is reachable by every solve
TOL_BATCH = 1e-5


def batch_measurement(D, I, torch, nsolves=64, seed=2026):
    """64 independent Wilson/staggered CG solves (FP32, tol 1e-5) of random
    lattice size in {8^4, 12^4, 16^3x32, 24^3x48} and N_v ~ U{1..24} as one
    graph-captured batch: solves/s and per-solve latency p50/p99 from the
    device completion stamps."""
    import numpy as np
    rng = np.random.default_rng(seed)
    sizes = [(8, 8, 8, 8), (12, 12, 12, 12), (16, 16, 16, 32), (24, 24, 24, 48)]
    ops, bs, m0s, desc = [], [], [], []
    fields = {}
    for i in range(nsolves):
        kind = D.WILSON if rng.integers(2) == 0 else D.STAGGERED
        dims = sizes[rng.integers(len(sizes))]
        nv = int(rng.integers(1, 25))
        if dims not in fields:
            fields[dims] = torch.from_numpy(I.gauge_field(dims, NC, 0.4, 500 + len(fields))).cuda()
        op = D.DiracOp(kind, fields[dims], nv, BC, D.F32)
        op.autotune(MASS[kind])
        ops.append(op)
        bs.append(op.to_prec(torch.from_numpy(I.source(dims, NC, nv, 600 + i, staggered=(kind == D.STAGGERED))).cuda()))
        m0s.append(0.1 if kind == D.WILSON else 0.05)
        desc.append((D.KIND_NAMES[kind], "x".join(map(str, dims)), nv))
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    xs, stats, rc = D.solve_batched(ops, bs, m0s=m0s, solver=D.CG_NORMAL, tol=TOL_BATCH, maxit=20000)
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    lat = sorted(s["seconds"] for s in stats)
    res = {"nsolves": nsolves, "rc": rc, "wall_s": wall, "solves_per_s": nsolves / wall,
           "latency_p50_s": float(np.percentile(lat, 50)), "latency_p99_s": float(np.percentile(lat, 99)),
           "iters_total": int(sum(s["iters"] for s in stats)),
           "all_converged": all(s["status"] == 0 for s in stats),
           "rhs_total": int(sum(d[2] for d in desc)), "tol": TOL_BATCH,
           "host_graph_launches": int(stats[0]["host_launches"]),
           "lattices": sorted({d[1] for d in desc})}
    for op in ops:
        op.close()
    return res


def tune_mass(D, op32, b32, kind, target=1e6, iters=600, torch_mod=None):
    """Bare mass giving cond(D^dag D) ~ target, from Lanczos estimates of a
    short FP32 CG (App. F "cond").  Staggered: cond ~ lambda_max / m^2.
    Wilson: bisection on m0 for lambda_min = lambda_max / target."""
    def est(m):
        _, st = op32.solve(b32, m0=m, solver=D.CG_HPD, tol=1e-30, maxit=iters, recompute_every=100000)
        return min(st["lambda_min"]), max(st["lambda_max"])
    if kind == D.STAGGERED:
        lo, hi = est(0.05)
        return (hi / target) ** 0.5, {"lambda_max": hi}
    # Wilson: a coarse scan of m0 on a 16^3x32 field of the same roughness,
    # each point solved to 1e-8 so that the Lanczos extremes have converged,
    # then log-interpolation of cond(m0) to the target
    small = (16, 16, 16, 32)
    import numpy as np
    from paper_2112_14640_gb300 import inputs as I
    Us = torch_mod.from_numpy(I.gauge_field(small, NC, 0.6, 98)).cuda()
    ops = D.DiracOp(kind, Us, NV, BC, D.F32)
    bs = ops.to_prec(torch_mod.from_numpy(I.source(small, NC, NV, 6)).cuda())
    scan = []
    for m in (0.0, -0.4, -0.7, -1.0, -1.2, -1.4, -1.6, -1.7, -1.8, -1.9, -2.0, -2.1, -2.2, -2.3, -2.4, -2.5):
        _, st = ops.solve(bs, m0=m, solver=D.CG_HPD, tol=1e-8, maxit=30000)
        c = max(st["lambda_max"]) / max(min(st["lambda_min"]), 1e-300)
        scan.append((m, c, st["iters"]))
        if c >= target:
            break
    ops.close()
    # log-interpolate between the last two points (cond grows towards the
    # critical mass); if the target was never reached, the largest cond seen
    ms, cs = np.array([a for a, _, _ in scan]), np.log(np.array([b for _, b, _ in scan]))
    if cs[-1] >= np.log(target) and len(cs) > 1 and cs[-1] > cs[-2]:
        w = (np.log(target) - cs[-2]) / (cs[-1] - cs[-2])
        m = float(ms[-2] + w * (ms[-1] - ms[-2]))
    else:
        m = float(ms[int(np.argmax(cs))])
    return m, {"scan_16x16x16x32": [(round(a, 3), float(b), int(k)) for a, b, k in scan]}


def solver_comparison(D, I, torch):
    """Time to an FP64 residual of 1e-10 of mixed-precision CG on D^dag D
    (32^3x64, Nc=3, Nv=12, eps=0.6, mass tuned to cond ~1e6): the FP32
    sloppy iteration (the baseline) against BF16 and FP16 sloppy iterations,
    reliable updates in FP64."""
    dims = (32, 32, 32, 64)
    out = {}
    U = torch.from_numpy(I.gauge_field(dims, NC, 0.6, 99)).cuda()
    for kind in (D.STAGGERED, D.WILSON):
        op = D.DiracOp(kind, U, NV, BC, D.F64, layout=D.SITE_INNER)
        # tune the launch variants of the sloppy operators first: the solver's
        # internal lower-precision twins pick the tuning up by their shape
        for prec, links in ((D.F32, D.LINKS_NATIVE), (D.F16, D.LINKS_F32), (D.BF16, D.LINKS_F32),
                            (D.F16, D.LINKS_NATIVE), (D.BF16, D.LINKS_NATIVE)):
            tw = D.DiracOp(kind, U, NV, BC, prec, layout=D.SITE_INNER, link_storage=links)
            tw.autotune(0.1 if kind == D.WILSON else 0.05)
            tw.close()
        op32 = D.DiracOp(kind, U, NV, BC, D.F32, layout=D.SITE_INNER)
        src = op.from_site_outer(torch.from_numpy(I.source(dims, NC, NV, 5, staggered=(kind == D.STAGGERED))).cuda())
        m0, info = tune_mass(D, op32, op32.to_prec(src), kind, torch_mod=torch)
        op32.close()
        b = op.to_prec(src)
        row = {"m0": m0, "tuning": info}
        for inner, links, mode in ((D.F32, D.LINKS_NATIVE, D.MIXED_RELIABLE),
                                   (D.F16, D.LINKS_F32, D.MIXED_RELIABLE), (D.BF16, D.LINKS_F32, D.MIXED_RELIABLE),
                                   (D.F16, D.LINKS_NATIVE, D.MIXED_RELIABLE), (D.BF16, D.LINKS_NATIVE, D.MIXED_RELIABLE),
                                   (D.F16, D.LINKS_F32, D.MIXED_ADAPTIVE), (D.BF16, D.LINKS_F32, D.MIXED_ADAPTIVE)):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            x, st = op.solve(b, m0=m0, solver=D.CG_NORMAL, tol=1e-10, maxit=40000, inner_prec=inner,
                             sloppy_links=links, mixed_mode=mode)
            torch.cuda.synchronize()
            name = D.PREC_NAMES[inner] + ("+f32links" if links == D.LINKS_F32 else "") + \
                ("+adaptive" if mode == D.MIXED_ADAPTIVE else "")
            row[name] = {"seconds": time.perf_counter() - t0, "iters": st["iters"],
                                        "updates": st["outer_iters"], "status": st["status"],
                                        "max_relres": max(st["relres"]), "max_true_relres": max(st["true_relres"]),
                                        "cond_lanczos": max(st["lambda_max"]) / max(min(st["lambda_min"]), 1e-300)}
            del x
        out[D.KIND_NAMES[kind]] = row
        op.close()
    return out


if __name__ == "__main__":
    main()
