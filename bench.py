"""Benchmark of the compact-derivative hot path on one or more GPUs (one process per GPU).

Workload (default): a 512^3 periodic field, sum of 4 Fourier modes (k <= 100) plus N(0, 0.1)
noise, P = 8 chunks per line.  One step is one pass of the whole path, in FP64 and then in
FP32 storage:
    x layout:  D1 u, D2 u, D1^T u          (first, second derivative, adjoint of the first)
    reorder x -> y;  the same three along y
    reorder y -> z;  the same three along z
i.e. 18 directional operators of 512^3 points and 4 reorders.  The three operators of one
direction share one read of the field (``tds_deriv_multi``: one fused pass).  ``value`` is
directional-derivative points per second (Gpoints/s) over all ranks, with the field resident in
HBM; every field is 0.5-1 GiB, larger than L2, so no flush is needed between steps.
``value_f64`` / ``value_f32`` (and ``by_precision``) split it: the nine operators of each
precision over the time of that precision's launches.  After the timed steps each operator is
also timed on its own (``breakdown`` entries ``single/...``), and the FP64 half of the step runs
again, K steps, with split-precision plans (FP64 fields and results, the sweeps' recurrences in
float pairs on the FP32 pipes): ``value_f64_split`` and the ``f64s/...`` breakdown entries; a
copy with the fused pass's traffic shape (one read, three writes: ``fanout3``) gives that pass's
own ceiling.

``e2e`` repeats the step through host buffers: the x-layout field comes from pinned host
memory each step (``tds_deriv_host`` copies it in for the first operator) and every one of
the 18 results is copied back to pinned host memory by the host entry points, whose copies
overlap the compute slab by slab.

``--impl reference`` times the FP64 CPU oracle (plain C) on every host core, one spawn-pool
process per core, on a bounded sample of the same workload (slabs of lines along each
direction), with the same metric.

Multi-GPU (torchrun): every rank runs the same workload on its own field (independent
problems: weak scaling, no data exchange); timing is max over ranks.
"""
import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "Gpoints/s and % of HBM roofline per directional derivative, FP64 vs FP32"
UNIT = "Gpoints/s"
KERNEL_SRC = [os.path.join(ROOT, "paper_2411_13532_gb300", "csrc", f)
              for f in ("tds_resident.cuh", "tds_device.cuh", "tds_df.cuh")]

def fp64_ops_per_point(op, m, periodic=True):
    """FP64-pipe operations per interior point as the resident kernel issues them.

    Forward row with f folded into the coefficients: 2 adds (the stencil differences or sums)
    + 1 multiply + 2 FMAs (first derivative) or 3 FMAs (second: the centre tap).  Back-
    substitution: 1 FMA.  The accumulation S += pi_j d_j and the s^a_j F term of the back-
    substitution are issued only on the rows before the plan's cut-off, where those weights,
    decaying like lambda^j (lambda = 0.382 for alpha = 1/3, 0.188 for alpha = 2/11), fall
    below 2^-60: about 44 and 25 rows.  The adjoint on periodic lines is the forward form with
    the transposed stencil (A and B circulant commute); on closed lines it is the identity
    forward row (1 multiply + 1 FMA), the back-substitution and the B^T pass (4)."""
    lam = {"d1": 0.38196601125, "d2": 0.18826230851, "d1t": 0.38196601125}[op]
    cut = min(m, math.ceil(math.log(2.0 ** -60) / math.log(lam)))
    extra = 2.0 * cut / m
    base = {"d1": 5.0 + 1.0, "d2": 6.0 + 1.0, "d1t": (5.0 + 1.0) if periodic else (2.0 + 1.0 + 4.0)}
    return base[op] + extra


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=30)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--size", type=int, default=512)
    ap.add_argument("--P", type=int, default=8)
    ap.add_argument("--e2e-steps", type=int, default=3)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--sweep", action="store_true",
                    help="time every workload configuration one operator at a time (one JSON line per "
                         "case) instead of the benchmark step")
    ap.add_argument("--sweep-match", default="",
                    help="with --sweep: only the cases whose label contains this text")
    ap.add_argument("--transport", action="store_true",
                    help="time the momentum-transport right-hand side (Sec. 5) instead of the "
                         "derivative step: one JSON line")
    ap.add_argument("--nu", type=float, default=1e-3)
    ap.add_argument("--thomas", action="store_true",
                    help="the plain Thomas kernel (tds_deriv_thomas) beside the DistD2 kernels at P = 8 "
                         "and P = 1, 512^3 x lines, FP64 and FP32, periodic and closed, D1 and D2")
    ap.add_argument("--nsweep", action="store_true",
                    help="the single-rank sweep over the line length n = 32..8192 (one JSON line per "
                         "case): first derivative along x, 2^30 points, P = 1 and 8, FP64 and FP32, "
                         "against a device copy of the same bytes")
    ap.add_argument("--one", action="store_true",
                    help="a small fixed launch sequence for profiler captures: on a --size^3 Fourier field "
                         "along x (--bc lines, --P chunks), --reps launches of the first derivative (or its "
                         "transpose, --adjoint), then --reps of the second, in --dtype with --arith; prints "
                         "one JSON line of timings")
    ap.add_argument("--reps", type=int, default=3)
    ap.add_argument("--bc", default="periodic", choices=["periodic", "closed"], help="with --one: the lines' ends")
    ap.add_argument("--adjoint", action="store_true", help="with --one: the transposed operators")
    ap.add_argument("--width", type=int, default=0, help="with --one: lines per resident CTA (0: the plan's)")
    ap.add_argument("--dtype", default="f64", choices=["f64", "f32"])
    ap.add_argument("--arith", default="native", choices=["native", "split"],
                    help="with --one or --sweep: the arithmetic of FP64 plans (tds_plan_set_arith)")
    return ap.parse_args()


def run_one(args):
    """--one: the launch sequence a profiler capture selects from (-s / -c)."""
    import torch
    import __graft_entry__
    __graft_entry__.build()
    import paper_2411_13532_gb300 as tds
    from paper_2411_13532_gb300 import inputs
    S = args.size
    shape = (S, S, S)
    dt = torch.float64 if args.dtype == "f64" else torch.float32
    f, _ = inputs.fourier_field(shape, seed=2, kmax=100, noise=0.1, noise_kind="normal", device="cuda")
    x = tds.reorder(f.to(dt).reshape(-1), shape, "cart", "x")
    del f
    y = torch.empty_like(x)
    out = {"mode": "one", "size": S, "P": args.P, "dtype": args.dtype, "arith": args.arith, "bc": args.bc,
           "adjoint": args.adjoint}
    for order in (1, 2):
        p = tds.Plan(shape, "x", order, args.bc, P=args.P, dtype=dt, width=args.width or None,
                     arith=args.arith if args.dtype == "f64" else "native")
        call = p.adjoint if args.adjoint else p.deriv
        ms = []
        for _ in range(args.reps):
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record()
            call(x, y)
            b.record()
            b.synchronize()
            ms.append(round(a.elapsed_time(b), 4))
        out["D%d_ms" % order] = ms
        out["D%d_width" % order] = p.width
    if tds.device_status() != 0:
        raise RuntimeError("device status after --one")
    print(json.dumps(out))


def load_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return json.load(fh), "measured"
    except (OSError, ValueError):
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


def code_fingerprint(paths):
    """sha256[:12] of C/C++/CUDA sources (concatenated in order) with their comments and whitespace
    removed: the counters of a capture stay valid across edits that do not touch the code."""
    import re
    text = ""
    for path in paths:
        with open(path) as fh:
            text += fh.read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    text = re.sub(r"//[^\n]*", "", text)
    text = re.sub(r"\s+", "", text)
    return hashlib.sha256(text.encode()).hexdigest()[:12]


def traffic_from_profiles(kernel_key):
    """DRAM bytes per launch from profiles/traffic.txt: lines '<key> <bytes> <code fingerprint>'.
    None if absent or if the kernel code changed since the capture."""
    path = os.path.join(ROOT, "profiles", "traffic.txt")
    try:
        cur = code_fingerprint(KERNEL_SRC)
        with open(path) as fh:
            for line in fh:
                parts = line.split()
                if len(parts) == 3 and not line.startswith("#") and parts[0] == kernel_key:
                    return float(parts[1]) if parts[2] == cur else None
    except OSError:
        pass
    return None


class ClockSampler:
    """nvidia-smi sampling of SM clock and throttle reasons during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "50"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
        return self

    def __exit__(self, *exc):
        self.out = ""
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.out, _ = self.proc.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                self.out, _ = self.proc.communicate()

    def summary(self):
        rows = []
        for line in (self.out or "").splitlines():
            p = [v.strip() for v in line.split(",")]
            if len(p) >= 9:
                try:
                    rows.append((float(p[1]), float(p[2]), p[5:9]))
                except ValueError:
                    pass
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for _, _, r in rows for i in range(4) if r[i] == "Active"})
        return {"sm_mhz": statistics.median(r[0] for r in rows), "sm_max_mhz": rows[0][1],
                "reasons": reasons, "samples": len(rows)}


# --------------------------------------------------------------------------- multi-rank

def max_over_ranks(ms, world, device):
    """Max of a per-rank time over all ranks (the job is as slow as its slowest GPU)."""
    if world <= 1:
        return ms
    import torch
    import torch.distributed as dist
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(world, ops_per_step, npts, steps, ms):
    """Whole-job Gpoints/s: every rank processes its own field (weak scaling)."""
    return world * ops_per_step * npts * steps / (ms * 1e-3) / 1e9


# ------------------------------------------------------------------------------ our arm

def run_ours(args, rank, world, local_rank):
    import torch
    import torch.distributed as dist

    import __graft_entry__
    __graft_entry__.build()
    import paper_2411_13532_gb300 as tds
    from paper_2411_13532_gb300 import inputs

    dev = torch.device("cuda", local_rank)
    torch.cuda.set_device(dev)
    S, P = args.size, args.P
    shape = (S, S, S)
    bc = "periodic"
    npts = S ** 3
    f, _ = inputs.fourier_field(shape, seed=2 + rank, kmax=100, noise=0.1, noise_kind="normal",
                                device=dev)
    dtypes = [("f64", torch.float64), ("f32", torch.float32)]
    data = {}
    for name, dt in dtypes:
        cart = f.to(dt).reshape(-1)
        ux = tds.reorder(cart, shape, "cart", "x")
        del cart
        d = {"ux": ux, "uy": torch.empty_like(ux), "uz": torch.empty_like(ux),
             "o": [torch.empty_like(ux) for _ in range(3)], "plans": {}}
        for direc in "xyz":
            for order in (1, 2):
                d["plans"][(direc, order)] = tds.Plan(shape, direc, order, bc, P=P, dtype=dt)
        d["ws"] = {k: p.workspace() for k, p in d["plans"].items()}
        data[name] = d
    del f
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream(dev)

    # per-launch CUDA events on the launching stream
    timing = {}

    def timed(key, fn):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        fn()
        e1.record(stream)
        timing.setdefault(key, []).append((e0, e1))

    launches = [0]

    def fused(p1, p2):
        # one pass computes D1, D2 and D1^T when both plans run resident with one width and
        # the adjoint has the forward form (periodic lines)
        return (p1.variant == p2.variant == "resident" and p1.width == p2.width and bc == "periodic")

    def step(record, names=("f64", "f32")):
        # per direction: D1, D2 and D1^T of one input through tds_deriv_multi (one fused pass)
        for name in names:
            d = data[name]
            src = d["ux"]
            for direc, nxt in (("x", "uy"), ("y", "uz"), ("z", None)):
                p1, p2 = d["plans"][(direc, 1)], d["plans"][(direc, 2)]
                ws = d["ws"][(direc, 1)] if p1.ws_bytes >= p2.ws_bytes else d["ws"][(direc, 2)]
                fn = (lambda s=src, a=p1, b=p2, w=ws:
                      tds.deriv_multi([(a, False), (b, False), (a, True)], s, outs=d["o"], ws=w))
                if record:
                    timed((name, "multi", p1.variant), fn)
                else:
                    fn()
                launches[0] += 1 if fused(p1, p2) else sum(3 if p.variant == "streaming" else 1
                                                           for p in (p1, p2, p1))
                if nxt is not None:
                    rfn = (lambda s=src, t=d[nxt], a=direc, b={"uy": "y", "uz": "z"}[nxt]:
                           tds.reorder(s, shape, a, b, out=t))
                    if record:
                        timed((name, "reorder"), rfn)
                    else:
                        rfn()
                    launches[0] += 1
                    src = d[nxt]

    for _ in range(args.warmup):
        step(False)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    launches[0] = 0
    timing.clear()
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    with ClockSampler(local_rank) as clk:
        t0.record(stream)
        for _ in range(args.steps):
            step(True)
        t1.record(stream)
        torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    ms = max_over_ranks(t0.elapsed_time(t1), world, dev)
    gpu_launches = launches[0]
    ops_per_step = 18
    value = job_throughput(world, ops_per_step, npts, args.steps, ms)

    # per-kernel averages over the timed steps
    per = {}
    for key, evs in timing.items():
        per[key] = sum(a.elapsed_time(b) for a, b in evs) / len(evs)

    # the single operators, one launch each (after the timed region, not part of `value`):
    # the per-kernel fractions of HBM of D1, D2 and D1^T on their own
    single = {}
    for name, _ in dtypes:
        d = data[name]
        p1, p2 = d["plans"][("x", 1)], d["plans"][("x", 2)]
        w1, w2 = d["ws"][("x", 1)], d["ws"][("x", 2)]
        for key, fn, var in (("d1", lambda: p1.deriv(d["ux"], d["o"][0], w1), p1.variant),
                             ("d2", lambda: p2.deriv(d["ux"], d["o"][1], w2), p2.variant),
                             ("d1t", lambda: p1.adjoint(d["ux"], d["o"][2], w1), p1.variant)):
            for _ in range(2):
                fn()
            evs = []
            for _ in range(5):
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                fn()
                e1.record(stream)
                evs.append((e0, e1))
            torch.cuda.synchronize()
            single[(name, key, var)] = sum(a.elapsed_time(b) for a, b in evs) / len(evs)

    # the FP64 step again with split-precision plans (FP64 fields and results, the sweeps'
    # recurrences in float pairs on the FP32 pipes): K steps after W warm-up steps, not part of
    # `value`; reported as value_f64_split with its own per-launch breakdown
    d64 = data["f64"]
    data["f64s"] = dict(d64)
    data["f64s"]["plans"] = {k: tds.Plan(shape, k[0], k[1], bc, P=P, dtype=torch.float64, arith="split")
                             for k in d64["plans"]}
    for _ in range(args.warmup):
        step(False, ("f64s",))
    torch.cuda.synchronize()
    ts0 = torch.cuda.Event(enable_timing=True)
    ts1 = torch.cuda.Event(enable_timing=True)
    ts0.record(stream)
    for _ in range(args.steps):
        step(True, ("f64s",))
    ts1.record(stream)
    torch.cuda.synchronize()
    ms_split = max_over_ranks(ts0.elapsed_time(ts1), world, dev)
    for key in [k for k in timing if k[0] == "f64s"]:
        per[key] = sum(a.elapsed_time(b) for a, b in timing[key]) / len(timing[key])
    ds = data["f64s"]
    p1s, p2s = ds["plans"][("x", 1)], ds["plans"][("x", 2)]
    for key, fn, var in (("d1", lambda: p1s.deriv(ds["ux"], ds["o"][0]), p1s.variant),
                         ("d2", lambda: p2s.deriv(ds["ux"], ds["o"][1]), p2s.variant),
                         ("d1t", lambda: p1s.adjoint(ds["ux"], ds["o"][2]), p1s.variant)):
        for _ in range(2):
            fn()
        evs = []
        for _ in range(5):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            fn()
            e1.record(stream)
            evs.append((e0, e1))
        torch.cuda.synchronize()
        single[("f64s", key, var)] = sum(a.elapsed_time(b) for a, b in evs) / len(evs)

    # the fused pass's own ceiling: a copy with its traffic shape (one read, three writes)
    for name, _ in dtypes:
        d = data[name]
        fn = (lambda d=d: tds.fanout_copy(d["ux"], d["o"]))
        for _ in range(2):
            fn()
        evs = []
        for _ in range(5):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            fn()
            e1.record(stream)
            evs.append((e0, e1))
        torch.cuda.synchronize()
        single[(name, "fanout3", "copy")] = sum(a.elapsed_time(b) for a, b in evs) / len(evs)

    m_chunk = S // args.P

    def algorithmic(key):
        """(directional-derivative points, algorithmic HBM bytes, FP64 operations) of one launch."""
        name, kind = key[0], key[1]
        es = 8 if name in ("f64", "f64s") else 4
        if kind == "multi":   # one read of the field, three results written
            return 3 * npts, 4 * es * npts, sum(fp64_ops_per_point(o, m_chunk) for o in ("d1", "d2", "d1t")) * npts
        if kind == "fanout3":
            return 3 * npts, 4 * es * npts, 0.0
        if kind == "reorder":
            return npts, 2 * es * npts, 0.0
        return npts, 2 * es * npts, fp64_ops_per_point(kind, m_chunk) * npts

    peaks, peak_kind = load_peaks()
    hbm = float(peaks["hbm_gbs"])
    breakdown = {}
    for src_tab, tag in ((per, ""), (single, "single/")):
        for key, avg_ms in sorted(src_tab.items()):
            pts, nbytes, _ = algorithmic(key)
            gbs = nbytes / (avg_ms * 1e-3) / 1e9
            breakdown[tag + "/".join(str(k) for k in key)] = {
                "ms": round(avg_ms, 4), "gpoints_s": round(pts / (avg_ms * 1e-3) / 1e9, 2),
                "alg_GB_s": round(gbs, 1), "hbm_frac": round(gbs / hbm, 4)}
    # the headline split by precision: each precision's launches of the timed step (three fused
    # passes, two reorders) and the nine directional derivatives they compute
    by_precision = {}
    for name, _ in dtypes:
        keys = [k for k in per if k[0] == name]
        ms_p = sum(per[k] * len(timing[k]) for k in keys) / args.steps
        bytes_p = sum(algorithmic(k)[1] * len(timing[k]) for k in keys) / args.steps
        by_precision[name] = {
            "gpoints_s": round(job_throughput(world, ops_per_step // 2, npts, 1, ms_p), 3),
            "ms_per_step": round(ms_p, 4),
            "alg_GB_s": round(bytes_p / (ms_p * 1e-3) / 1e9, 1),
            "hbm_frac": round(bytes_p / (ms_p * 1e-3) / 1e9 / hbm, 4)}
    # the FP64 step with split-precision plans (timed on its own after the timed region)
    keys = [k for k in per if k[0] == "f64s"]
    bytes_s = sum(algorithmic(k)[1] * len(timing[k]) for k in keys) / args.steps
    ms_s = sum(per[k] * len(timing[k]) for k in keys) / args.steps
    by_precision["f64_split"] = {
        "gpoints_s": round(job_throughput(world, ops_per_step // 2, npts, args.steps, ms_split), 3),
        "ms_per_step": round(ms_split / args.steps, 4),
        "alg_GB_s": round(bytes_s / (ms_s * 1e-3) / 1e9, 1),
        "hbm_frac": round(bytes_s / (ms_s * 1e-3) / 1e9 / hbm, 4),
        "arith": "FP64 fields and results; sweeps in float pairs on the FP32 pipes (tds_plan_set_arith)"}
    # dominant kernel of the timed step by total time
    totals = {k: per[k] * len(timing[k]) for k in per if k[0] != "f64s"}
    dom = max(totals, key=totals.get)
    dom_ms = per[dom]
    pts, nbytes, ops = algorithmic(dom)
    clocks = clk.summary()
    if dom[0] == "f64" and dom[1] != "reorder":
        # FP64 pipe bound: FP64 operations issued vs the FP64 pipe's peak rate,
        # 2 FP64 instructions per clock per SM x 152 SMs x sampled SM clock
        sm_mhz = clocks["sm_mhz"] or 2070.0
        peak = 2 * 152 * sm_mhz * 1e6 / 1e9
        ach = ops / (dom_ms * 1e-3) / 1e9
        roofline = {"kernel": "/".join(str(k) for k in dom), "bound": "alu", "achieved": round(ach, 1),
                    "peak": round(peak, 1), "unit": "Gop/s (FP64 pipe)", "frac": round(ach / peak, 4),
                    "peak_source": "derived: 2 FP64 ops/clk/SM x 152 SMs x median SM clock",
                    "hbm_frac": round(nbytes / (dom_ms * 1e-3) / 1e9 / hbm, 4)}
    else:
        ach = nbytes / (dom_ms * 1e-3) / 1e9
        roofline = {"kernel": "/".join(str(k) for k in dom), "bound": "hbm", "achieved": round(ach, 1),
                    "peak": hbm, "unit": "GB/s", "frac": round(ach / hbm, 4), "peak_source": peak_kind}
    kkey = "%s_%s_%s_%d" % (dom[0], dom[1], dom[2] if len(dom) > 2 else "", S)
    traffic = traffic_from_profiles(kkey)
    roofline["traffic"] = traffic
    roofline["alg_bytes_per_launch"] = nbytes
    # the FP32 derivative kernels on their own against HBM (the 70 % target)
    f32 = [v for k, v in breakdown.items() if k.startswith("single/f32/d")]
    roofline["f32_deriv_hbm_frac_min"] = min(e["hbm_frac"] for e in f32) if f32 else None
    # the FP32 fused pass against a copy of the same traffic shape (one read, three writes)
    fan = breakdown.get("single/f32/fanout3/copy")
    mul = [v for k, v in breakdown.items() if k.startswith("f32/multi/")]
    if fan and mul:
        roofline["f32_multi_of_fanout_copy"] = round(fan["ms"] / mul[0]["ms"], 4)
    # the split-precision FP64 fused pass against HBM
    sm = [(k, v) for k, v in breakdown.items() if k.startswith("f64s/multi/")]
    if sm:
        roofline["f64_split_multi_hbm_frac"] = sm[0][1]["hbm_frac"]

    # ------------------------------------------------------------------ end to end
    e2e = None
    if args.e2e_steps > 0:
        host = {}
        for name, dt in dtypes:
            d = data[name]
            host[name] = {"in": torch.empty(d["ux"].numel(), dtype=dt, pin_memory=True),
                          "out": [torch.empty(d["ux"].numel(), dtype=dt, pin_memory=True)
                                  for _ in range(9)]}
            host[name]["in"].copy_(d["ux"])
        h2d = sum(host[n]["in"].numel() * host[n]["in"].element_size() for n in host)
        d2h = sum(o.numel() * o.element_size() for n in host for o in host[n]["out"])

        def e2e_step():
            # every operator through the host entry points (slab-pipelined copies): the field
            # comes in with the first x operator, every result goes back to pinned host memory
            for name, _ in dtypes:
                d, hb = data[name], host[name]
                i = 0
                src = d["ux"]
                for direc, nxt in (("x", "uy"), ("y", "uz"), ("z", None)):
                    p1, p2 = d["plans"][(direc, 1)], d["plans"][(direc, 2)]
                    w1, w2 = d["ws"][(direc, 1)], d["ws"][(direc, 2)]
                    p1.deriv_host(hb["in"] if direc == "x" else None, hb["out"][i], src, d["o"][0], w1)
                    p2.deriv_host(None, hb["out"][i + 1], src, d["o"][1], w2)
                    p1.adjoint_host(None, hb["out"][i + 2], src, d["o"][2], w1)
                    i += 3
                    if nxt is not None:
                        b = {"uy": "y", "uz": "z"}[nxt]
                        tds.reorder(src, shape, direc, b, out=d[nxt])
                        src = d[nxt]
        e2e_step()
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(args.e2e_steps):
            e2e_step()
        b.record(stream)
        torch.cuda.synchronize()
        ems = max_over_ranks(a.elapsed_time(b), world, dev)
        e2e = {"value": round(job_throughput(world, ops_per_step, npts, args.e2e_steps, ems), 3),
               "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
               "ms_per_step": round(ems / args.e2e_steps, 3)}

    status = tds.device_status()
    if status != 0:
        raise RuntimeError("device status %d after the timed region" % status)
    return {"value": value, "ms": ms, "roofline": roofline, "breakdown": breakdown, "by_precision": by_precision,
            "clocks": clocks, "e2e": e2e, "gpu_launches": gpu_launches}


# ------------------------------------------------------------------ per-configuration sweep

SWEEP_CASES = [
    # (label, shape (nz, ny, nx), directions, orders, bcs, Ps, dtypes,
    #  kind: "deriv" | "adjoint" | "solve" | "band", or "deriv+adjoint" for both on one plan)
    ("64^3 D1 x periodic P=1", (64, 64, 64), "x", (1,), ("periodic",), (1,), ("f64",), "deriv"),
    ("256^3 D1/D2 x,y,z periodic/closed P=1,4", (256, 256, 256), "xyz", (1, 2), ("periodic", "closed"),
     (1, 4), ("f64",), "deriv"),
    ("512^3 D1/D2 x,y,z periodic P=8 FP64/FP32", (512, 512, 512), "xyz", (1, 2), ("periodic",), (8,),
     ("f64", "f32"), "deriv"),
    ("512^3 D1^T x periodic P=8 FP64/FP32", (512, 512, 512), "x", (1,), ("periodic",), (8,), ("f64", "f32"),
     "adjoint"),
    ("256^3 D1^T z closed P=4 FP64/FP32", (256, 256, 256), "z", (1,), ("closed",), (4,), ("f64", "f32"), "adjoint"),
    ("512^3 D1/D2 and D1^T/D2^T x closed P=8 FP64/FP32", (512, 512, 512), "x", (1, 2), ("closed",), (8,),
     ("f64", "f32"), "deriv+adjoint"),
    ("1024^3 D1 x,y,z periodic P=8,2", (1024, 1024, 1024), "xyz", (1,), ("periodic",), (8, 2), ("f64",), "deriv"),
    ("256 x 262144 D1 x periodic P=64", (1, 256, 262144), "x", (1,), ("periodic",), (64,), ("f64", "f32"), "deriv"),
    ("512^3 solve A x = d, x periodic/closed P=8 FP64/FP32", (512, 512, 512), "x", (1, 2),
     ("periodic", "closed"), (8,), ("f64", "f32"), "solve"),
    ("512^3 compact filter (alpha_f 0.45) and mid-point interpolation, x, P=8 FP64/FP32", (512, 512, 512),
     "x", ("filter", "interp"), ("periodic", "closed"), (8,), ("f64", "f32"), "deriv"),
    ("512^3 batched tridiagonal solve, variable-coefficient band (implicit diffusion on a stretched grid), "
     "x, P=8 FP64/FP32", (512, 512, 512), "x", ("band",), ("periodic", "closed"), (8,), ("f64", "f32"), "band"),
]


def run_sweep(args):
    """Every workload configuration, one operator at a time: CUDA events around each launch,
    a 2x-L2 buffer written between launches, median of the timed launches."""
    import torch
    import __graft_entry__
    __graft_entry__.build()
    import paper_2411_13532_gb300 as tds
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    flush = torch.empty(2 * 135 * 2 ** 20 // 4, dtype=torch.float32, device=dev)
    peaks, peak_kind = load_peaks()
    hbm = float(peaks["hbm_gbs"])
    TD = {"f64": torch.float64, "f32": torch.float32}
    reps = max(args.steps, 5)
    import numpy as np
    import oracle
    from paper_2411_13532_gb300 import inputs
    oracle.build()

    def oracle_rate(n, order, bc, kind):
        """The FP64 oracle (one core) on a sample of about 2^21 points of whole lines of this
        case: points per second."""
        nl = max(1, 2 ** 21 // n)
        lines = np.random.default_rng(n).uniform(-1, 1, (nl, n))
        h = oracle.grid_spacing(n, bc)
        t = time.perf_counter()
        if order == "filter":
            oracle.filter_lines(lines, 0.45, bc)
        elif order == "interp":
            oracle.interp_lines(lines, bc)
        elif kind == "adjoint":
            oracle.deriv_adjoint_lines(lines, order, bc, h)
        elif kind == "solve":
            a, b, c, _ = oracle.bands(n, order, bc, h)
            for d in lines:
                oracle.tridiag_solve(a, b, c, d, bc == "periodic")
        elif kind == "band":
            a, b, c = inputs.diffusion_band(n, seed=1)
            for d in lines:
                oracle.tridiag_solve(a, b, c, d, bc == "periodic")
        else:
            oracle.deriv_lines(lines, order, bc, h)
        return nl * n / (time.perf_counter() - t) / 1e9
    for label, shape, dirs, orders, bcs, Ps, dts, kind in SWEEP_CASES:
        if args.sweep_match not in label:
            continue
        npts = shape[0] * shape[1] * shape[2]
        for dname in dts:
            dt = TD[dname]
            x = (torch.rand(npts, dtype=dt, device=dev) - 0.5) * 2
            y = torch.empty_like(x)
            for direc in dirs:
                for order in orders:
                    for bc in bcs:
                        for P in Ps:
                            n = shape[{"x": 2, "y": 1, "z": 0}[direc]]
                            if kind == "band":
                                plan = tds.Plan(shape, direc, 0, bc, P=P, dtype=dt,
                                                band=inputs.diffusion_band(n, seed=1))
                            else:
                                plan = tds.Plan(shape, direc, order, bc, P=P, dtype=dt,
                                                alpha_f=0.45 if order == "filter" else None,
                                                arith=args.arith if dname == "f64" else "native")
                            ws = plan.workspace()
                            for sub in kind.split("+"):
                                fn = {"adjoint": lambda: plan.adjoint(x, y, ws), "solve": lambda: plan.solve(x, y, ws),
                                      "band": lambda: plan.solve(x, y, ws), "deriv": lambda: plan.deriv(x, y, ws)}[sub]
                                for _ in range(max(args.warmup, 3)):
                                    fn()
                                times = []
                                for _ in range(reps):
                                    flush.fill_(1.0)
                                    a = torch.cuda.Event(enable_timing=True)
                                    b = torch.cuda.Event(enable_timing=True)
                                    a.record()
                                    fn()
                                    b.record()
                                    b.synchronize()
                                    times.append(a.elapsed_time(b))
                                ms = statistics.median(times)
                                es = x.element_size()
                                gbs = 2 * es * npts / (ms * 1e-3) / 1e9
                                print(json.dumps({
                                    "case": label, "dtype": dname,
                                    "op": (order if isinstance(order, str) else
                                           {"adjoint": "D%dT", "solve": "A%d^-1", "deriv": "D%d"}[sub] % order),
                                    "dir": direc, "bc": bc, "P": P, "variant": plan.variant, "width": plan.width,
                                    "arith": plan.arith,
                                    "ms": round(ms, 4), "gpoints_s": round(npts / (ms * 1e-3) / 1e9, 2),
                                    "alg_GB_s": round(gbs, 1), "hbm_frac": round(gbs / hbm, 4),
                                    "hbm_frac_nominal_7900": round(gbs / 7900.0, 4), "peak_source": peak_kind,
                                    "oracle_gpoints_s_1core": round(oracle_rate(shape[{"x": 2, "y": 1, "z": 0}[direc]],
                                                                                order, bc, sub), 5)}),
                                      flush=True)
                            del plan, ws
            del x, y
            torch.cuda.empty_cache()
    if tds.device_status() != 0:
        raise RuntimeError("device status after the sweep")


# ----------------------------------------------------------- plain Thomas beside DistD2

def run_thomas(args):
    """The single-rank baseline of the paper's bandwidth table (Table BW): the plain Thomas
    algorithm on whole lines (one thread per line; cyclic lines: Sherman-Morrison, a third pass)
    beside the resident DistD2 kernels at P = 8 and P = 1, each the median of the timed launches
    with a 2x-L2 write between launches.  Algorithmic traffic 2 fields per operator; the Thomas
    kernel moves 4 (closed) or 6 (cyclic), DistD2 resident 2."""
    import torch
    import __graft_entry__
    __graft_entry__.build()
    import paper_2411_13532_gb300 as tds
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    flush = torch.empty(2 * 135 * 2 ** 20 // 4, dtype=torch.float32, device=dev)
    peaks, peak_kind = load_peaks()
    hbm = float(peaks["hbm_gbs"])
    S = args.size
    shape = (S, S, S)
    npts = S ** 3
    reps = max(args.steps, 5)

    def timed(fn):
        for _ in range(max(args.warmup, 3)):
            fn()
        times = []
        for _ in range(reps):
            flush.fill_(1.0)
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record()
            fn()
            b.record()
            b.synchronize()
            times.append(a.elapsed_time(b))
        return statistics.median(times)
    with ClockSampler(0) as clk:
        for dname, dt in (("f64", torch.float64), ("f32", torch.float32)):
            x = (torch.rand(npts, dtype=dt, device=dev) - 0.5) * 2
            y = torch.empty_like(x)
            es = x.element_size()
            for bc in ("periodic", "closed"):
                for order in (1, 2):
                    row = {"case": "thomas_vs_distd2", "size": S, "dtype": dname, "op": "D%d" % order, "bc": bc}
                    p8 = tds.Plan(shape, "x", order, bc, P=args.P, dtype=dt)
                    p1 = tds.Plan(shape, "x", order, bc, P=1, dtype=dt)
                    w8, w1 = p8.workspace(), p1.workspace()
                    for key, fn, moved in (("thomas", lambda: p8.thomas(x, y), 6 if bc == "periodic" else 4),
                                           ("distd2_P%d" % args.P, lambda: p8.deriv(x, y, w8), 2),
                                           ("distd2_P1", lambda: p1.deriv(x, y, w1), 2)):
                        ms = timed(fn)
                        alg = 2 * es * npts / (ms * 1e-3) / 1e9
                        row[key] = {"ms": round(ms, 4), "gpoints_s": round(npts / (ms * 1e-3) / 1e9, 2),
                                    "alg_GB_s": round(alg, 1), "hbm_frac": round(alg / hbm, 4),
                                    "moved_fields": moved, "moved_hbm_frac": round(alg * moved / 2 / hbm, 4)}
                    row["variants"] = {"P%d" % args.P: p8.variant, "P1": p1.variant}
                    row["peak_source"] = peak_kind
                    print(json.dumps(row), flush=True)
                    del p8, p1, w8, w1
            del x, y
            torch.cuda.empty_cache()
    print(json.dumps({"case": "thomas_vs_distd2", "clocks": clk.summary()}), flush=True)
    if tds.device_status() != 0:
        raise RuntimeError("device status after the Thomas comparison")


# ----------------------------------------------------------- line-length sweep (single rank)

def run_nsweep(args):
    """The paper's single-rank sweep (Sec. 5: runtime against line length, normalised by a STREAM
    copy) on one GB300: D1 along x on 2^30 points cut into lines of n = 32..8192, P = 1 (one rank)
    and P = 8, FP64 and FP32; each time is the median of 5 launches with a 2x-L2 write between
    them, beside a device-to-device copy of the same bytes (the copy stand-in)."""
    import torch
    import __graft_entry__
    __graft_entry__.build()
    import paper_2411_13532_gb300 as tds
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    flush = torch.empty(2 * 135 * 2 ** 20 // 4, dtype=torch.float32, device=dev)
    peaks, kind = load_peaks()
    hbm = float(peaks["hbm_gbs"])
    total = 2 ** 30

    def timed(fn):
        for _ in range(3):
            fn()
        ts = []
        for _ in range(5):
            flush.fill_(1.0)
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record()
            fn()
            b.record()
            b.synchronize()
            ts.append(a.elapsed_time(b))
        return statistics.median(ts)

    for dname, dt in (("f64", torch.float64), ("f32", torch.float32)):
        x = (torch.rand(total, dtype=dt, device=dev) - 0.5) * 2
        y = torch.empty_like(x)
        copy_ms = timed(lambda: y.copy_(x))
        for n in (32, 64, 128, 256, 512, 1024, 2048, 4096, 8192):
            shape = (total // (n * 1024), 1024, n)
            for P in (1, 8):
                plan = tds.Plan(shape, "x", 1, "periodic", P=P, dtype=dt)
                ws = plan.workspace()
                ms = timed(lambda: plan.deriv(x, y, ws))
                gbs = 2 * x.element_size() * total / (ms * 1e-3) / 1e9
                print(json.dumps({"sweep": "line length", "dtype": dname, "n": n, "lines": total // n, "P": P,
                                  "variant": plan.variant, "width": plan.width, "ms": round(ms, 4),
                                  "gpoints_s": round(total / (ms * 1e-3) / 1e9, 2),
                                  "alg_GB_s": round(gbs, 1), "hbm_frac": round(gbs / hbm, 4),
                                  "copy_ms": round(copy_ms, 4), "time_over_copy": round(ms / copy_ms, 3),
                                  "peak_source": kind}), flush=True)
                del plan, ws
        del x, y
        torch.cuda.empty_cache()
    if tds.device_status() != 0:
        raise RuntimeError("device status after the line-length sweep")


# ------------------------------------------------------------------ transport right-hand side

# Field transfers (reads + writes of one N^3 field) per evaluation, Table transport's counting:
# the paper's GPU implementation and this one (x: the i = j term reads 1 field, the two i != j
# terms 2, each writes 1; y and z: 3 reorders (1 + 1), the same 8 for the terms, 3
# accumulations fused with the reorder back to x (read the term, read and write the output).
PAPER_TRANSFERS = {"abstract_ij": 96, "abstract_ii": 45, "reorder": 12, "accumulate": 18}
OUR_TRANSFERS = {"term": 3 * 8, "reorder": 6 * 2, "reorder_add": 6 * 3}


def transport_fp64_ops_per_point(m):
    """FP64-pipe operations per point of one fused term kernel: the three sweeps (D1 of u_i,
    D1 of the product, D2 of u_i), the product (1 multiply) and the epilogues (2 multiplies,
    2 FMAs)."""
    return 2 * fp64_ops_per_point("d1", m) + fp64_ops_per_point("d2", m) + 1 + 4


def run_transport(args):
    """The transport right-hand side (three components, nine term groups, six reorders, six
    accumulations) on an S^3 periodic box, FP64 and FP32: per-launch CUDA events on the
    launching stream, inputs larger than L2."""
    import torch
    import __graft_entry__
    __graft_entry__.build()
    import paper_2411_13532_gb300 as tds
    from paper_2411_13532_gb300 import inputs
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    S, P = args.size, args.P
    shape = (S, S, S)
    npts = S ** 3
    stream = torch.cuda.current_stream(dev)
    peaks, peak_kind = load_peaks()
    hbm = float(peaks["hbm_gbs"])
    res = {}
    launches = 0
    clocks = None
    e2e = None
    for name, dt in (("f64", torch.float64), ("f32", torch.float32)):
        es = 8 if name == "f64" else 4
        rhs = tds.TransportRHS(shape, P=P, dtype=dt)
        u = []
        for c in range(3):
            f, _ = inputs.fourier_field(shape, seed=31 + c, kmax=20, noise=1e-3, device=dev)
            u.append(tds.reorder(f.to(dt).reshape(-1), shape, "cart", "x"))
            del f
        out = [torch.empty_like(u[0]) for _ in range(3)]
        plan = rhs.launch_list(u, args.nu, out)
        for _ in range(max(args.warmup, 3)):
            for _, fn in plan:
                fn()
        torch.cuda.synchronize()
        per = {}
        t0 = torch.cuda.Event(enable_timing=True)
        t1 = torch.cuda.Event(enable_timing=True)
        evs = []
        with ClockSampler(0) as clk:
            t0.record(stream)
            for _ in range(args.steps):
                for key, fn in plan:
                    a = torch.cuda.Event(enable_timing=True)
                    b = torch.cuda.Event(enable_timing=True)
                    a.record(stream)
                    fn()
                    b.record(stream)
                    evs.append((key, a, b))
                    launches += 1
            t1.record(stream)
            torch.cuda.synchronize()
        if name == "f64" or clocks is None:
            clocks = clk.summary()
        ms = t0.elapsed_time(t1) / args.steps
        for key, a, b in evs:
            per.setdefault(key, []).append(a.elapsed_time(b))
        # the same evaluation replayed as one CUDA graph (no per-launch host work)
        g = rhs.graph(u, args.nu, out)
        for _ in range(2):
            g.replay()
        torch.cuda.synchronize()
        g0 = torch.cuda.Event(enable_timing=True)
        g1 = torch.cuda.Event(enable_timing=True)
        g0.record(stream)
        for _ in range(args.steps):
            g.replay()
        g1.record(stream)
        torch.cuda.synchronize()
        graph_ms = g0.elapsed_time(g1) / args.steps
        launches += 21 * args.steps
        del g
        field = es * npts
        kern = {}
        for key, v in sorted(per.items()):
            avg = sum(v) / len(v)
            kind = key.split("/")[0]
            transfers = {"term": 8.0 / 3.0, "reorder": 2.0, "reorder_add": 3.0}[kind]
            gbs = transfers * field / (avg * 1e-3) / 1e9
            kern[key] = {"ms": round(avg, 4), "launches_per_eval": len(v) // args.steps,
                         "alg_GB_s": round(gbs, 1), "hbm_frac": round(gbs / hbm, 4)}
            if kind == "term":
                ops = transport_fp64_ops_per_point(S // P) * npts
                kern[key]["fp64_Gop_s"] = round(ops / (avg * 1e-3) / 1e9, 1)
        ours = sum(OUR_TRANSFERS.values())
        paper = sum(PAPER_TRANSFERS.values())
        term_ms = sum(sum(v) for k, v in per.items() if k.startswith("term")) / args.steps
        reo_ms = sum(sum(v) for k, v in per.items() if k.startswith("reorder/")) / args.steps
        acc_ms = sum(sum(v) for k, v in per.items() if k.startswith("reorder_add")) / args.steps
        res[name] = {
            "ms_per_eval": round(ms, 3), "gpoints_s": round(npts / (ms * 1e-3) / 1e9, 3),
            "field_transfers": ours, "paper_field_transfers": paper,
            "alg_GB_s": round(ours * field / (ms * 1e-3) / 1e9, 1),
            "hbm_frac": round(ours * field / (ms * 1e-3) / 1e9 / hbm, 4),
            "paper_count_GB_s": round(paper * field / (ms * 1e-3) / 1e9, 1),
            "time_share": {"terms": round(term_ms / ms, 4), "reorders": round(reo_ms / ms, 4),
                           "reorder_add": round(acc_ms / ms, 4)},
            "reorder_traffic_share": round(OUR_TRANSFERS["reorder"] / ours, 4),
            "kernels": kern, "graph_ms_per_eval": round(graph_ms, 3)}
        if name == "f64" and args.e2e_steps > 0:
            # end to end: the three components from pinned host memory, the three results back
            hu = [torch.empty(npts, dtype=dt, pin_memory=True) for _ in range(3)]
            ho = [torch.empty(npts, dtype=dt, pin_memory=True) for _ in range(3)]
            for h, d in zip(hu, u):
                h.copy_(d)

            def e2e_step():
                # pinned host in and out, the copies overlapped with the kernels
                rhs.call_host(hu, ho, args.nu, u, out)
            e2e_step()
            torch.cuda.synchronize()
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(stream)
            for _ in range(args.e2e_steps):
                e2e_step()
            b.record(stream)
            torch.cuda.synchronize()
            ems = a.elapsed_time(b) / args.e2e_steps
            e2e = {"value": round(npts / (ems * 1e-3) / 1e9, 3), "unit": "Gpoints/s",
                   "h2d_bytes_per_step": 3 * field, "d2h_bytes_per_step": 3 * field,
                   "ms_per_step": round(ems, 3), "dtype": "f64"}
            del hu, ho
        del rhs, u, out, plan
        torch.cuda.empty_cache()
    if tds.device_status() != 0:
        raise RuntimeError("device status after the transport benchmark")
    # roofline of the dominant kernel (the FP64 term group): FP64 pipe bound
    t64 = res["f64"]["kernels"]["term/x"]
    sm_mhz = clocks["sm_mhz"] or 2070.0
    peak = 2 * 152 * sm_mhz * 1e6 / 1e9
    roofline = {"kernel": "f64/term/x (k_resident_transport)", "bound": "alu",
                "achieved": t64["fp64_Gop_s"], "peak": round(peak, 1), "unit": "Gop/s (FP64 pipe)",
                "frac": round(t64["fp64_Gop_s"] / peak, 4),
                "peak_source": "derived: 2 FP64 ops/clk/SM x 152 SMs x median SM clock",
                "traffic": traffic_from_profiles("f64_transport_term_%d" % S),
                "alg_bytes_per_launch": 3 * 8 * npts,
                "f32_term_hbm_frac": res["f32"]["kernels"]["term/x"]["hbm_frac"]}
    cpu = None
    if not args.no_cpu_baseline:
        import numpy as np
        import oracle
        oracle.build()
        n = 64
        rng = np.random.default_rng(0)
        u = [rng.uniform(-1, 1, (n, n, n)) for _ in range(3)]
        t = time.perf_counter()
        reps = 0
        while time.perf_counter() - t < 10.0:
            oracle.transport_rhs(u, args.nu, "periodic")
            reps += 1
        dtc = time.perf_counter() - t
        cpu = {"value": round(reps * n ** 3 / dtc / 1e9, 5), "unit": "Gpoints/s", "cores": 1, "kind": "oracle",
               "sample": "%d evaluations of the FP64 oracle on a %d^3 periodic box, %.1f s" % (reps, n, dtc)}
    line = {"metric": "momentum-transport RHS evaluations (grid points per second)",
            "value": res["f64"]["gpoints_s"], "unit": "Gpoints/s", "n_gpus": 1, "steps": args.steps,
            "warmup": max(args.warmup, 3), "ms_per_step": res["f64"]["ms_per_eval"], "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64 (f32 in breakdown)", "data": "synthetic",
            "config": {"workload": "skew-symmetric momentum transport RHS, %d^3 periodic, P=%d, nu=%g"
                                   % (S, P, args.nu),
                       "l2": "inputs larger than L2"},
            "clocks": clocks, "e2e": e2e, "gpu_launches": launches, "roofline": roofline,
            "breakdown": res, "cpu_baseline": cpu}
    print(json.dumps(line))


# ------------------------------------------------------------------------ CPU oracle arm

def oracle_sample_step(S, lines_per_dir, rng_seed=0):
    """One bounded sample of the step on the CPU oracle: for each direction, a slab of
    ``lines_per_dir`` whole lines of S points taken from a Cartesian field, the three
    operators, in FP64 and again on the FP32-rounded field.  Returns points processed."""
    import numpy as np
    import oracle
    side = int(math.sqrt(lines_per_dir))
    rng = np.random.default_rng(rng_seed)
    pts = 0
    for prec in ("f64", "f32"):
        for direc in "xyz":
            shp = {"x": (side, side, S), "y": (side, S, side), "z": (S, side, side)}[direc]
            cart = rng.normal(size=shp)
            if prec == "f32":
                cart = cart.astype(np.float32).astype(np.float64)
            oracle.deriv(cart, direc, 1, "periodic")
            oracle.deriv(cart, direc, 2, "periodic")
            oracle.deriv_adjoint(cart, direc, 1, "periodic")
            pts += 3 * cart.size
    return pts


def _oracle_worker(task):
    """One process of the all-core oracle timing: sample steps until ``seconds`` have passed."""
    S, lines, seed, seconds = task
    import oracle
    t = time.perf_counter()
    pts = 0
    k = 0
    while True:
        pts += oracle_sample_step(S, lines, rng_seed=seed * 1000 + k)
        k += 1
        if time.perf_counter() - t >= seconds:
            break
    return pts, time.perf_counter() - t


def time_oracle_all_cores(S, seconds=10.0, lines=1024):
    """The oracle as it stands, one process per host core (a spawn pool: the parent holds a CUDA
    context), each timing sample steps of independent lines; rate = all points / slowest worker."""
    import multiprocessing as mp
    import oracle
    oracle.build()
    workers = os.cpu_count() or 1
    ctx = mp.get_context("spawn")
    with ctx.Pool(workers) as pool:
        # bounded: a worker that died would otherwise leave map() waiting for ever
        res = pool.map_async(_oracle_worker, [(S, lines, w + 1, seconds) for w in range(workers)]).get(
            timeout=4 * seconds + 120)
    pts = sum(p for p, _ in res)
    wall = max(t for _, t in res)
    return pts / wall / 1e9, workers, pts


def time_oracle(S, seconds_target=10.0):
    import oracle
    oracle.build()
    lines = 1024
    t = time.perf_counter()
    pts = oracle_sample_step(S, lines)
    dt = time.perf_counter() - t
    # grow the sample to roughly the target duration
    reps = max(1, int(seconds_target / max(dt, 1e-3)))
    t = time.perf_counter()
    tot = 0
    for r in range(reps):
        tot += oracle_sample_step(S, lines, rng_seed=r + 1)
    dt = time.perf_counter() - t
    return tot / dt / 1e9, "%d x (18 operators on %d lines of %d points each, 3 directions, " \
        "FP64 and FP32-rounded input), %.1f s" % (reps, lines, S, dt)


def _oracle_step_worker(task):
    S, lines, seed = task
    return oracle_sample_step(S, lines, rng_seed=seed)


def run_reference(args, rank, world):
    """The oracle as it stands, on every host core: one spawn-pool process per core, each step a
    sample of ``lines`` whole lines per direction per process (all 18 operators)."""
    if rank != 0:
        return None
    import multiprocessing as mp
    import oracle
    oracle.build()
    S = args.size
    lines = 1024
    workers = os.cpu_count() or 1
    ctx = mp.get_context("spawn")
    with ctx.Pool(workers) as pool:
        def step(k):
            tasks = [(S, lines, 1000 * (k + 1) + w) for w in range(workers)]
            # bounded: a worker that died would otherwise leave the map waiting for ever
            return sum(pool.map_async(_oracle_step_worker, tasks).get(timeout=600))
        for k in range(args.warmup):
            step(args.steps + k)   # seeds apart from the timed steps
        t = time.perf_counter()
        pts = 0
        for k in range(args.steps):
            pts += step(k)
        dt = time.perf_counter() - t
    value = pts / dt / 1e9
    sample = ("per step: %d processes, each 18 operators (D1, D2, D1^T along x, y, z; FP64 and FP32-rounded "
              "input) on %d whole lines of %d points per direction" % (workers, lines, S))
    return {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt * 1e3 / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": "compact derivatives %d^3 periodic, sampled lines (CPU oracle)" % S,
                       "P": args.P, "l2": "n/a (CPU)"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": workers, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def main():
    args = parse()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        out = run_reference(args, rank, world)
        if out is not None:
            print(json.dumps(out))
        return
    if args.sweep:
        run_sweep(args)
        return
    if args.transport:
        run_transport(args)
        return
    if args.nsweep:
        run_nsweep(args)
        return
    if args.thomas:
        run_thomas(args)
        return
    if args.one:
        run_one(args)
        return
    if world > 1:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(local_rank)
        dist.init_process_group("nccl")
    res = run_ours(args, rank, world, local_rank)
    if rank == 0:
        cpu = None
        if not args.no_cpu_baseline and world == 1:
            v1, sample = time_oracle(args.size)
            vn, workers, pts = time_oracle_all_cores(args.size)
            cpu = {"value": round(vn, 4), "unit": UNIT, "cores": workers, "kind": "oracle",
                   "sample": "%d processes x sample steps (18 operators on 1024 lines of %d points, "
                             "3 directions, FP64 and FP32-rounded input) for 10 s each, %d points" % (
                                 workers, args.size, pts),
                   "single_core": {"value": round(v1, 4), "cores": 1, "sample": sample}}
        S = args.size
        line = {
            "metric": METRIC, "value": round(res["value"], 3), "unit": UNIT, "n_gpus": world,
            "value_f64": res["by_precision"]["f64"]["gpoints_s"],
            "value_f32": res["by_precision"]["f32"]["gpoints_s"],
            "value_f64_split": res["by_precision"]["f64_split"]["gpoints_s"],
            "by_precision": res["by_precision"],
            "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": round(res["ms"] / args.steps, 4), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64+f32",
            "data": "synthetic (seeded Fourier modes k<=100 + N(0,0.1) noise)",
            "config": {"workload": "compact derivatives %d^3 periodic, P=%d, D1/D2/D1^T along x,y,z "
                                   "in FP64 and FP32 + 4 reorders per step" % (S, args.P),
                       "grid": [S, S, S], "P": args.P, "operators_per_step": 18,
                       "l2": "inputs larger than L2 (%.2f GiB per FP64 field)" % (S ** 3 * 8 / 2 ** 30)},
            "clocks": res["clocks"], "e2e": res["e2e"], "gpu_launches": res["gpu_launches"],
            "roofline": res["roofline"], "breakdown": res["breakdown"], "cpu_baseline": cpu,
        }
        print(json.dumps(line))
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
