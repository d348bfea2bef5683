"""Benchmark: 512^3 cubic Klein-Gordon steps/s on one GB300 (or N independent replicas).

Workload (the paper-scale case): N = 512 (R2C storage 512 x 512 x 257 complex128),
cube side 32, u0 = 0.1 exp(-|x|^2) + 1e-3 lowpass(N(0,1), |m| <= 8) seeded 1501,
u_t(0) = 0, dt = 0.005, energy every 10 steps.  A "step" is one pass of the whole
hot path: x pass (C2R, cube, R2C), forward y and z passes, the FP64 update, inverse z
and y passes, plus the recorded energy sums every 10th level.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

Prints one JSON line.  --impl reference times the FP64 CPU oracle on the host cores
on a bounded sample of the same workload.  Under torchrun each rank runs its own
replica (the method is not sharded); rank 0 prints.
"""
import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

N_GRID = 512
L_BOX = 32.0
DT = 0.005
ENERGY_EVERY = 10
PRECISION = "df64"
STEP_LAUNCHES = 7
E2E_REPEATS = 3
METRIC = "512^3 KG steps/s"
L2_BYTES = 129 * 1000 * 1000          # GB300 L2
S_BYTES = N_GRID * N_GRID * (N_GRID // 2 + 1) * 16      # one complex128 half-spectrum array


# Table 1 of the paper: wall time (s) of 30 time steps of the same scheme at 512^3 in FP64
# on CPU clusters (2DECOMP&FFT); quoted as context, not as a target
PAPER_TABLE1 = [("Hornet", 12288, 0.319), ("Juqueen", 262144, 0.350), ("Stampede", 8162, 0.581),
                ("Shaheen", 16384, 1.66), ("MareNostrum III", 64, 4.00), ("Hector", 1024, 7.66),
                ("VSC2", 1024, 9.03), ("Beacon", 256, 9.13), ("Monte Rosa", 1024, 11.9), ("Titan", 256, 17.0),
                ("Vedur", 1024, 18.6), ("Aquila", 256, 22.4), ("Neser", 128, 27.9)]

# DRAM bytes (read + write) per launch of a step kernel at 512^3, from one ncu capture
# (dram__bytes_read.sum + dram__bytes_write.sum; the capture is summarised under
# profiles/), valid only for the kernel sources it was taken on: KERNEL_SOURCES hashed
TRAFFIC_512 = {("df64", "x"): 2099839488, ("df64", "yf"): 2096962304, ("df64", "z"): 5455137792,
               ("df64", "yi"): 2096292352}
TRAFFIC_SOURCES_SHA = "00869fe2215bc89a"
KERNEL_SOURCES = ["kg_arith.cuh", "kg_fft.cuh", "kg_kernels.cuh", "kg_complex.cuh", "kg_launch_impl.cuh"]


def kernel_sources_sha():
    """hash of the kernel sources' code: comments and blank space are dropped first, so that
    an edit of a comment keeps a capture valid and any change of code does not"""
    import hashlib
    import re
    h = hashlib.sha256()
    for f in KERNEL_SOURCES:
        with open(os.path.join(ROOT, "paper_1501_04552_gb300", "csrc", f), encoding="utf-8") as fh:
            text = fh.read()
        text = re.sub(r"/\*.*?\*/", " ", text, flags=re.S)
        text = re.sub(r"//[^\n]*", " ", text)
        h.update(" ".join(text.split()).encode())
    return h.hexdigest()[:16]


def measured_traffic(prec, kernel, n):
    if n != N_GRID or TRAFFIC_SOURCES_SHA is None or kernel_sources_sha() != TRAFFIC_SOURCES_SHA:
        return None
    return TRAFFIC_512.get((prec, kernel))


def algorithmic_bytes(prec, n=N_GRID):
    """bytes each kernel group of a step must move (W is S or S/2 by precision, the state
    arrays are S), and the bytes an ideal step moves: four passes reading and writing W
    plus reading uh^n, uh^{n-1} and writing uh^{n+1} (11 S, or 7 S with FP32 W)"""
    s_bytes = n * n * (n // 2 + 1) * 16
    w = s_bytes if prec in ("fp64", "df64") else s_bytes // 2
    per_kernel = {"x": 2 * w, "yf": 2 * w, "zf": 2 * w, "update": 2 * w + 3 * s_bytes, "zi": 2 * w, "yi": 2 * w,
                  "z": 2 * w + 3 * s_bytes, "xy": 2 * w}
    return per_kernel, 8 * w + 3 * s_bytes


def kernel_groups(k_ms):
    """names and device ms of a step's kernel groups from kg_step_timed: x, yf, z (the
    fused z pass: forward z FFT, update, inverse z FFT), yi when the update and inverse-z
    slots are empty; xy (the cluster-fused inverse y, x and forward y pass), z and yi
    (the inverse y pass that closes a kg_step call, once per call) when the forward-y slot
    is empty too; else the six separate groups"""
    if k_ms[1] == 0.0 and k_ms[3] == 0.0 and k_ms[4] == 0.0:
        return ["xy", "z", "yi"], [k_ms[0], k_ms[2], k_ms[5]]
    if k_ms[3] == 0.0 and k_ms[4] == 0.0:
        return ["x", "yf", "z", "yi"], [k_ms[0], k_ms[1], k_ms[2], k_ms[5]]
    return ["x", "yf", "zf", "update", "zi", "yi"], list(k_ms)


KERNEL_NAMES = {"x": "k_pass_x", "z": "k_zstep", "update": "k_update", "xy": "k_xy_cluster"}


# FP32 peak of the GPU's FMA pipes: 152 SMs x 128 FP32 lanes x 2.07 GHz (max SM clock), one
# operation per lane per clock, whether issued as scalar FP32 instructions or as packed
# FP32x2 ones (which take the pipe for two lane operations; profiles/fp_pipes_gb300.md)
FP32_ISSUE_PEAK = 152 * 128 * 2.07e9
# FP64 FMA rate measured on GB300 (2 per SM per clock; profiles/fp_pipes_gb300.md)
FP64_PEAK = 598e9


def df64_fp32_ops(n):
    """FP32 operations of the double-float FFT kernels at grid n, counted from the
    definitions of the double-float arithmetic (Knuth two-sum 6 + low parts 2 = 8 per
    unnormalised add, 16 per unnormalised FMA-split dot product = one component of a
    twiddle product, 4 per unnormalised product; sign flips and integer work not counted;
    no transform renormalises its outputs).  Radix-8 DFT: 24 complex adds (384) + the two
    sqrt(1/2) rotations (48) = 432; a stage after the first applies 7 twiddle products
    (+224).  The paired x pass per pair and point: packing 16, two transforms, scale 4,
    the max|u| key 2, the cube 24; unpacking 40 per output.  Returns per-launch counts for
    the paired x pass and for one column pass (n = 512: three radix-8 stages)."""
    assert n == 512
    fft_point = (432 + (432 + 224) + (432 + 224)) / 8.0      # 218 per point
    pairs = n * n // 2
    per_pair = n * (16 + fft_point + 4 + 2 + 24 + fft_point) + (n // 2 + 1) * 40
    col_points = n * n * (n // 2 + 1)
    return {"x": pairs * per_pair, "col": col_points * fft_point}


def df64_fft_point_ops(n):
    """FP32 operations per point of a length-n double-float transform of the FFT engine
    (the counts of df64_fp32_ops): a radix-8 DFT 432 per 8 points, radix-4 128 per 4,
    radix-2 32 per 2; every stage after the first applies a twiddle product (32) to
    (R-1)/R of the points"""
    lg = n.bit_length() - 1
    radices = [8] * (lg // 3) + ([1 << (lg % 3)] if lg % 3 else [])
    dft = {8: 432 / 8.0, 4: 128 / 4.0, 2: 32 / 2.0}
    ops = sum(dft[r] for r in radices)
    ops += sum((r - 1) / r * 32 for r in radices[1:])
    return ops


def df64_step_ops(n):
    """FP32 operations of one double-float step of an n^3 grid: the paired x pass and four
    column transforms (forward y, forward and inverse z, inverse y) of the half spectrum"""
    f = df64_fft_point_ops(n)
    pairs = n * n // 2
    x = pairs * (n * (16 + f + 4 + 2 + 24 + f) + (n // 2 + 1) * 40)
    return x + 4 * n * n * (n // 2 + 1) * f


def step_schedule(start, steps, every):
    """the kg_step chunks of a timed region that starts at level `start` and runs `steps`
    steps, and after which of them the energy is evaluated: at every level that is a multiple
    of `every`, except the last level of the region (an evaluation runs the next step's x pass
    ahead of time, work of a step outside the region)"""
    out, level, left = [], start, steps
    while left > 0:
        k = min(left, every - level % every)
        level += k
        left -= k
        out.append((k, level % every == 0 and left > 0))
    return out


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled while the timed region runs"""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS, "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
            time.sleep(0.25)
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            time.sleep(0.15)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for l in self.lines:
            parts = [p.strip() for p in l.split(",")]
            if len(parts) < 7:
                continue
            try:
                sm.append(float(parts[0]))
                smax = float(parts[1])
            except ValueError:
                continue
            for nm, v in zip(names, parts[3:7]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": smax,
                "reasons": sorted(reasons), "samples": len(sm)}


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def cpu_baseline(workload, sample_steps):
    """the FP64 oracle, as it stands, on a bounded sample: set-up + sample_steps steps"""
    from oracle import oracle as O
    t0 = time.perf_counter()
    s = O.Solver(workload["N"], workload["L"], workload["dt"], workload["u0"], workload["v0"])
    t1 = time.perf_counter()
    s.step(sample_steps)
    t2 = time.perf_counter()
    s.close()
    return {"value": sample_steps / (t2 - t1), "unit": "steps/s", "cores": O.num_threads(), "kind": "oracle",
            "sample": "%d steps of the %d^3 workload after a %.1f s set-up (set-up not counted)"
                      % (sample_steps, workload["N"], t1 - t0)}


REF_MAX_STEPS = 60      # oracle steps (warm-up + timed) one reference run may take: ~2 s each at 512^3


def run_reference(args):
    """the FP64 oracle as it stands on the host cores: W warm-up steps after its set-up, then
    K timed steps of the 512^3 workload (K and W as asked, while K + W <= REF_MAX_STEPS)"""
    rank, world, local = dist_env()
    if rank != 0:
        return 0
    from oracle import oracle as O
    from paper_1501_04552_gb300 import inputs as I
    w = I.bump_noise(N_GRID)
    steps = max(1, min(args.steps, REF_MAX_STEPS))
    warmup = max(0, min(args.warmup, REF_MAX_STEPS - steps))
    t0 = time.perf_counter()
    s = O.Solver(w["N"], w["L"], w["dt"], w["u0"], w["v0"])
    t1 = time.perf_counter()
    s.step(warmup)
    t2 = time.perf_counter()
    s.step(steps)
    t3 = time.perf_counter()
    s.close()
    value = steps / (t3 - t2)
    base = {"value": value, "unit": "steps/s", "cores": O.num_threads(), "kind": "oracle",
            "sample": "%d timed steps of the %d^3 workload after a %.1f s set-up and %d warm-up steps"
                      % (steps, N_GRID, t1 - t0, warmup)}
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "steps/s", "n_gpus": args.gpus,
            "steps": steps, "warmup": warmup, "ms_per_step": 1e3 / value, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "kg512_bump_noise", "N": N_GRID, "L": L_BOX, "dt": DT, "seed": 1501},
            "cpu_baseline": base,
            "e2e": {"value": value, "unit": "steps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    if steps != args.steps or warmup != args.warmup:
        line["capped"] = "steps + warm-up capped at %d oracle steps (about 2 s each)" % REF_MAX_STEPS
    print(json.dumps(line), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--precision", default=PRECISION, choices=["fp64", "df64", "mixed"])
    ap.add_argument("--cpu-sample-steps", type=int, default=2)
    ap.add_argument("--no-extras", action="store_true", help="skip the other precisions and the cuFFT point")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU-oracle sample (profiling runs)")
    ap.add_argument("--ens-steps", type=int, default=200, help="fixed steps of the ensemble comparison")
    ap.add_argument("--no-ranker", action="store_true", help="skip the learned-ranker study (about two minutes)")
    ap.add_argument("--xy-fusion", action="store_true",
                    help="time the FP32 passes with the cluster-fused xy pass (with --precision mixed)")
    ap.add_argument("--grid", type=int, default=N_GRID, help="grid size (512 is the benchmark; smaller for profiling)")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    if args.warmup < 3 or args.steps < 1:
        ap.error("--warmup must be >= 3 and --steps >= 1")

    import torch
    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)

    import __graft_entry__ as g
    if rank == 0:
        g.build_library()
    if world > 1:
        torch.distributed.barrier()
    from paper_1501_04552_gb300 import inputs as I
    from paper_1501_04552_gb300 import kg
    from paper_1501_04552_gb300 import replicas

    NG = args.grid
    w = I.bump_noise(NG)
    kg.kg_set_xy_fusion(args.xy_fusion)
    u0 = w["u0"]
    stream = torch.cuda.Stream()
    kg.kg_set_stream(stream)

    def barrier():
        if world > 1:
            torch.distributed.barrier()

    def device_warmup(seconds=0.5):
        """untimed steps until `seconds` of wall time have passed: a GPU that has been idle
        (the first process on a box) ran the first milliseconds of work 20x slower, more than
        a few warm-up steps of a small grid cover.  Not part of the W warm-up steps."""
        kg.kg_set_options(precision="df64", energy_every=0)
        d_u0 = torch.from_numpy(u0).to(f"cuda:{local}")
        kg.kg_init_device(NG, L_BOX, DT, d_u0, None)
        del d_u0
        t0 = time.perf_counter()
        while time.perf_counter() - t0 < seconds:
            kg.kg_step(5)
            stream.synchronize()
        kg.kg_finalize()

    def timed_steps(prec, steps, warmup):
        """warm-up, then `steps` timed steps with the energy evaluated whenever the level
        reaches a multiple of ENERGY_EVERY (the workload's cadence, counted from level 0)
        inside the timed region: an evaluation runs the next step's x pass ahead of time, so
        one at the last level would time work of a step beyond the region.  The warm-up runs
        the same kernels, an energy evaluation included, so that no kernel is loaded for the
        first time inside the timed region."""
        kg.kg_set_options(precision=prec, energy_every=ENERGY_EVERY)
        d_u0 = torch.from_numpy(u0).to(f"cuda:{local}")
        kg.kg_init_device(NG, L_BOX, DT, d_u0, None)
        del d_u0
        # the warm-up's energy evaluation comes one step before its end: kg_energy runs the next
        # step's x pass ahead (kg_step then skips it), and that step still belongs to the warm-up,
        # so the timed region holds the whole work of its steps
        if warmup >= 1:
            kg.kg_step(warmup - 1)
            kg.kg_energy(allow_drift=True)
            kg.kg_step(1)
        stream.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        barrier()
        torch.cuda.synchronize()
        e0.record(stream)
        energies = []
        for k, evaluate in step_schedule(warmup, steps, ENERGY_EVERY):
            kg.kg_step(k)
            if evaluate:
                energies.append(kg.kg_energy(allow_drift=True))
        e1.record(stream)
        e1.synchronize()
        torch.cuda.synchronize()
        barrier()
        ms = e0.elapsed_time(e1)
        timed_steps.energies = energies
        return replicas.max_over_ranks(ms, device=f"cuda:{local}")

    prec = args.precision
    device_warmup()
    with ClockSampler(local) as clk:
        ms = timed_steps(prec, args.steps, args.warmup)
    clocks = clk.summary()
    energies = list(getattr(timed_steps, "energies", []))
    ms_per_step = ms / args.steps
    value = replicas.throughput(args.steps, world, ms * 1e-3)

    # per-kernel device times (CUDA events on the library's stream) for the roofline
    kg.kg_step(1)   # a step whose x pass an energy evaluation ran ahead is not timed below
    names, k_avg = kernel_groups([t / args.steps for t in kg.kg_step_timed(args.steps)])
    k_bytes, step_bytes = algorithmic_bytes(prec, NG)
    dom = int(np.argmax(k_avg))
    peak, peak_kind = peaks()
    achieved = k_bytes[names[dom]] / (k_avg[dom] * 1e-3) / 1e9
    step_achieved = step_bytes / (ms_per_step * 1e-3) / 1e9
    per_kernel = {n: {"ms": round(t, 4), "GBps": round(k_bytes[n] / (t * 1e-3) / 1e9, 1),
                      "frac": round(k_bytes[n] / (t * 1e-3) / 1e9 / peak, 4)} for n, t in zip(names, k_avg)}
    roofline = {"bound": "hbm", "kernel": KERNEL_NAMES.get(names[dom], "k_col(%s)" % names[dom]),
                "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s", "frac": round(achieved / peak, 4),
                "traffic": measured_traffic(prec, names[dom], NG), "peak_kind": peak_kind,
                "step_achieved": round(step_achieved, 1), "step_frac": round(step_achieved / peak, 4),
                "kernels": per_kernel}
    if prec == "df64":
        roofline["limiter"] = ("arithmetic, not HBM: the double-float transforms are bound by the FP32 lanes of the "
                               "FMA pipes (packed FP32x2 instructions; x and y passes about 0.62-0.70 of their peak, "
                               "ncu FMA pipe 75 % busy with math-pipe-throttle stalls in the x pass), and the fused z "
                               "pass adds the FP64 update on the FP64 pipe (frac_pipes of roofline_alu.kernels.z); "
                               "their HBM fraction is low by construction")
    roofline_alu = None
    if prec == "df64" and NG == 512:
        ops = df64_fp32_ops(NG)
        # the fused z pass: two column transforms on the FP32 pipe and the update on the FP64
        # pipe (6 DFMA per mode); frac_pipes adds the two pipes' busy fractions, the share of
        # the kernel's time their minimum times fill when they do not overlap
        kops = {n: ops["x"] if n == "x" else (2 * ops["col"] if n == "z" else ops["col"]) for n in names}
        per = {n: {"ops": kops[n], "frac": round(kops[n] / (t * 1e-3) / FP32_ISSUE_PEAK, 4)}
               for n, t in zip(names, k_avg) if n != "update"}
        if "z" in per:
            t_z = k_avg[names.index("z")] * 1e-3
            fp64_ops = 6 * NG * NG * (NG // 2 + 1)
            per["z"]["fp64_ops"] = fp64_ops
            per["z"]["frac_fp64"] = round(fp64_ops / t_z / FP64_PEAK, 4)
            per["z"]["frac_pipes"] = round(per["z"]["frac"] + per["z"]["frac_fp64"], 4)
        x_rate = ops["x"] / (k_avg[names.index("x")] * 1e-3)
        roofline_alu = {"bound": "alu", "kernel": "k_pass_x", "achieved": round(x_rate / 1e12, 2),
                        "peak": round(FP32_ISSUE_PEAK / 1e12, 2), "unit": "T FP32 ops/s",
                        "frac": round(x_rate / FP32_ISSUE_PEAK, 4), "kernels": per,
                        "what": "double-float operation counts of the FFT kernels / event time; "
                                "peak = 152 SMs x 128 lanes x 2.07 GHz"}

    # end to end through the public API with host buffers: pinned u0 -> kg_init, K steps, kg_fetch -> host
    pinned_u0 = torch.from_numpy(u0).pin_memory()
    out = torch.empty((NG,) * 3, dtype=torch.float64).pin_memory()
    kg.kg_set_options(precision=prec, energy_every=ENERGY_EVERY)
    e2e_runs = []
    for _ in range(E2E_REPEATS):     # host-side phases vary from run to run: the median is reported
        barrier()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        kg.lib.kg_init(NG, L_BOX, DT, pinned_u0.data_ptr(), None)
        kg.kg_step(args.steps)
        kg.lib.kg_fetch(out.data_ptr())
        torch.cuda.synchronize()
        e2e_runs.append(replicas.max_over_ranks(time.perf_counter() - t0, device=f"cuda:{local}"))
    t_e2e = sorted(e2e_runs)[len(e2e_runs) // 2]
    e2e = {"value": replicas.throughput(args.steps, world, t_e2e), "unit": "steps/s",
           "runs_s": [round(t, 4) for t in e2e_runs],
           "h2d_bytes_per_step": u0.nbytes // args.steps, "d2h_bytes_per_step": out.numel() * 8 // args.steps,
           "what": "kg_init from pinned host u0 + %d steps + kg_fetch to pinned host; median of %d runs"
                   % (args.steps, E2E_REPEATS)}

    extras = {}
    if not args.no_extras and rank == 0:
        for other in ["fp64", "df64", "mixed"]:
            if other == prec:
                continue
            steps = ENERGY_EVERY * max(1, args.steps // (8 if other == "fp64" else 1) // ENERGY_EVERY)
            o_ms = timed_steps(other, steps, ENERGY_EVERY)
            kg.kg_step(1)
            o_names, o_k = kernel_groups([t / steps for t in kg.kg_step_timed(steps)])
            o_bytes, o_step_bytes = algorithmic_bytes(other, NG)
            extras[other] = {"steps_per_s": round(steps / (o_ms * 1e-3), 2), "ms_per_step": round(o_ms / steps, 4),
                             "kernel_ms": {n: round(t, 4) for n, t in zip(o_names, o_k)},
                             "step_hbm_frac": round(o_step_bytes / (o_ms / steps * 1e-3) / 1e9 / peak, 4)}
        extras["mixed_xy_fused"] = xy_fused_point(kg, stream, torch, u0, NG, local, peak)
        extras["cufft_torch"] = torch_fft_point(u0, local)
        if NG == 512:
            extras["paper_table1_protocol"] = {p: paper_protocol(kg, stream, torch, u0, NG, local, p)
                                               for p in ("df64", "fp64")}
        extras["complex_field"] = {p: complex_point(kg, stream, torch, u0, NG, local, p, peak)
                                   for p in ("df64", "mixed")}
        extras["composed4"] = composed_point(kg, stream, torch, u0, NG, local, "df64")
        if NG == 512:
            extras["precision_split_500"] = precision_split(kg, torch, u0, NG, local, 500)
    ens = None
    if not args.no_extras and rank == 0:
        ens = ensemble_point(kg, prec, args.ens_steps, torch, stream, early_exit=True)
        ens["mixed"] = ensemble_point(kg, "mixed", args.ens_steps, torch, stream)
    ranker_study = None
    if not args.no_extras and not args.no_ranker and rank == 0:
        # the learned blow-up ranker on the GPU: 4096 solver-labelled 64^3 runs (T = 10),
        # training of the 6-128-128-2 network, a 65 536-point Sobol sweep, the top 1024 and
        # 1024 uniform points re-solved by the plain solver as judge, the boundary bracketed
        # at 32 values of s with and without the network
        from paper_1501_04552_gb300 import ranker
        kg.kg_set_options()
        t0 = time.perf_counter()
        ranker_study = ranker.run()
        ranker_study["wall_seconds"] = round(time.perf_counter() - t0, 1)

    base = None
    if rank == 0 and world == 1 and not args.no_cpu:
        base = cpu_baseline(w, args.cpu_sample_steps)

    kg.kg_finalize()
    kg.kg_set_stream(None)
    if rank == 0:
        s_bytes = NG * NG * (NG // 2 + 1) * 16
        l2_note = ("inputs larger than L2 (each state array %.2f GB)" % (s_bytes / 1e9) if s_bytes > L2_BYTES
                   else "inputs fit in L2 (each state array %.0f MB): a small-grid run" % (s_bytes / 1e6))
        line = {"metric": METRIC if NG == N_GRID else "%d^3 KG steps/s" % NG, "value": round(value, 3), "unit": "steps/s", "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": round(ms_per_step, 4), "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": {"fp64": "f64", "df64": "f64 state+update, df64 FFT",
                                                                  "mixed": "f64 state+update, f32 FFT"}[prec],
                "data": "synthetic",
                "config": {"workload": "kg%d_bump_noise" % NG, "N": NG, "L": L_BOX, "dt": DT, "seed": 1501,
                           "precision": prec, "energy_every": ENERGY_EVERY, "parallelism": "replicas",
                           "l2": l2_note, "device_warmup_s": 0.5},
                "roofline": roofline, "roofline_alu": roofline_alu, "cpu_baseline": base, "e2e": e2e,
                "clocks": clocks,
                # per step: x pass, its finaliser, two forward column passes, update, the
                # second-stage Q sum, the z finaliser, two inverse column passes; per energy
                # evaluation: the peek x pass and its finaliser
                "gpu_launches": STEP_LAUNCHES * args.steps + 2 * len(energies),
                "energy_series": {"every": ENERGY_EVERY, "first": energies[0] if energies else None,
                                  "max_rel_drift": (max(abs(e - energies[0]) for e in energies) / abs(energies[0])
                                                    if energies else None)},
                "other_precisions": extras, "ensemble": ens, "ranker_study": ranker_study}
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


def precision_split(kg, torch, u0, NG, local, steps):
    """the workload for `steps` steps in each precision, energy every 10: relative L2 of the
    final field against the IEEE-FP64 path, and each path's energy drift (max |E - E_0| / |E_0|
    over the series); the scheme's own O(dt^2) drift is in every path"""
    out, fields = {}, {}
    for prec in ("fp64", "df64", "mixed"):
        kg.kg_set_options(precision=prec, energy_every=ENERGY_EVERY)
        d_u0 = torch.from_numpy(u0).to(f"cuda:{local}")
        kg.kg_init_device(NG, L_BOX, DT, d_u0, None)
        del d_u0
        es = [kg.kg_energy()]
        for _ in range(steps // ENERGY_EVERY):
            kg.kg_step(ENERGY_EVERY)
            es.append(kg.kg_energy(allow_drift=True))
        fields[prec] = kg.kg_fetch(NG)
        es = np.array(es)
        out[prec] = {"energy_drift": float(np.abs(es - es[0]).max() / abs(es[0]))}
        kg.kg_finalize()
    ref = fields["fp64"]
    nrm = float(np.linalg.norm(ref))
    for prec in ("df64", "mixed"):
        out[prec]["rel_l2_vs_fp64"] = float(np.linalg.norm(fields[prec] - ref) / nrm)
    out["steps"] = steps
    return out


def xy_fused_point(kg, stream, torch, u0, NG, local, peak):
    """the FP32 passes with the inverse y, x and forward y transforms of each z-plane fused
    in thread-block clusters (kg_set_xy_fusion): steps/s, the fused kernel's device time
    and its HBM fraction for its algorithmic 2 W (W = S/2), against the same steps with
    the separate passes (x, y, y: 6 W)"""
    out = {}
    for fused in (False, True):
        kg.kg_set_options(precision="mixed", energy_every=ENERGY_EVERY)
        kg.kg_set_xy_fusion(fused)
        d_u0 = torch.from_numpy(u0).to(f"cuda:{local}")
        kg.kg_init_device(NG, L_BOX, DT, d_u0, None)
        del d_u0
        kg.kg_step(4)
        kg.kg_energy(allow_drift=True)
        kg.kg_step(1)   # takes the x pass the energy evaluation ran ahead
        stream.synchronize()
        steps = 2 * ENERGY_EVERY
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        kg.kg_step(steps)
        e1.record(stream)
        e1.synchronize()
        ms = e0.elapsed_time(e1) / steps
        k = [t / steps for t in kg.kg_step_timed(steps)]
        kg.kg_finalize()
        w_bytes = NG * NG * (NG // 2 + 1) * 8
        if fused:
            out["fused"] = {"steps_per_s": round(1e3 / ms, 2), "ms_per_step": round(ms, 4),
                            "xy_kernel_ms": round(k[0], 4), "z_ms": round(k[2], 4),
                            "xy_hbm_frac": round(2 * w_bytes / (k[0] * 1e-3) / 1e9 / peak, 4)}
        else:
            out["separate"] = {"steps_per_s": round(1e3 / ms, 2), "ms_per_step": round(ms, 4),
                               "x_yf_yi_ms": round(k[0] + k[1] + k[5], 4),
                               "x_yf_yi_hbm_frac": round(6 * w_bytes / ((k[0] + k[1] + k[5]) * 1e-3) / 1e9 / peak, 4)}
    kg.kg_set_xy_fusion(False)
    return out


def complex_point(kg, stream, torch, u0, NG, local, prec, peak):
    """the complex-field path (|u|^2 u, full N^3 spectrum) on the same grid: u0 of the
    workload times a phase exp(0.5 i x / L), steps/s and per-kernel device times; the
    algorithmic bytes are those of the real path with S_c = N^3 16 B"""
    x = (np.arange(NG) * (L_BOX / NG) - L_BOX / 2)
    uc = (u0 * np.exp(0.5j * x / L_BOX)[None, None, :]).astype(np.complex128)
    kg.kg_set_options(precision=prec, energy_every=ENERGY_EVERY)
    d_u0 = torch.from_numpy(uc).to(f"cuda:{local}")
    kg.kg_init_complex_device(NG, L_BOX, DT, d_u0, None)
    del d_u0
    kg.kg_step(ENERGY_EVERY)
    stream.synchronize()
    steps = 2 * ENERGY_EVERY
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    runs = []
    for _ in range(3):       # the energy calls synchronise with the host: median of three
        e0.record(stream)
        for _ in range(steps // ENERGY_EVERY):
            kg.kg_step(ENERGY_EVERY)
            kg.kg_energy(allow_drift=True)
        e1.record(stream)
        e1.synchronize()
        runs.append(e0.elapsed_time(e1) / steps)
    ms = sorted(runs)[1]
    k_names, k_ms = kernel_groups([t / steps for t in kg.kg_step_timed(steps)])
    sc = NG ** 3 * 16
    w = sc if prec in ("fp64", "df64") else sc // 2
    step_bytes = 8 * w + 3 * sc
    kg.kg_finalize()
    return {"steps_per_s": round(1e3 / ms, 2), "ms_per_step": round(ms, 4),
            "kernel_ms": {n: round(t, 4) for n, t in zip(k_names, k_ms)},
            "step_hbm_frac": round(step_bytes / (ms * 1e-3) / 1e9 / peak, 4)}


def composed_point(kg, stream, torch, u0, NG, local, prec):
    """the fourth-order composed scheme (three substeps per step) on the workload: steps/s;
    and, on a 64^3 bump at a coarse dt, its error at t = 1 beside Eq. (2) at the same cost
    (dt / 3), both against a composed run at dt / 16 (IEEE FP64 passes)"""
    kg.kg_set_scheme("composed4")
    kg.kg_set_options(precision=prec, energy_every=0)
    d_u0 = torch.from_numpy(u0).to(f"cuda:{local}")
    kg.kg_init_device(NG, L_BOX, DT, d_u0, None)
    del d_u0
    kg.kg_step(3)
    stream.synchronize()
    steps = 20
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    kg.kg_step(steps)
    e1.record(stream)
    e1.synchronize()
    ms = e0.elapsed_time(e1) / steps
    # accuracy at equal cost on a small grid
    from paper_1501_04552_gb300 import inputs as I
    n, dt, T = 64, 0.05, 1.0
    ub = I.gaussian(n, L_BOX, 1.4, 2.5)

    def run(scheme, prec_, step):
        kg.kg_set_scheme(scheme)
        kg.kg_set_options(precision=prec_, energy_every=0)
        kg.kg_init(n, L_BOX, step, ub, None)
        kg.kg_step(int(round(T / step)))
        return kg.kg_fetch(n)

    ref = run("composed4", "fp64", dt / 16)
    err = {}
    for name, scheme, step in (("eq2_dt_over_3", "eq2", dt / 3), ("composed4_dt", "composed4", dt)):
        u = run(scheme, prec, step)
        err[name] = float(np.linalg.norm(u - ref) / np.linalg.norm(ref))
    kg.kg_finalize()
    kg.kg_set_scheme("eq2")
    kg.kg_set_options()
    return {"steps_per_s": round(1e3 / ms, 2), "ms_per_step": round(ms, 4), "passes_per_step": 3,
            "equal_cost_error_64": {"dt": dt, "T": T, "rel_l2": err}}


def paper_protocol(kg, stream, torch, u0, NG, local, prec):
    """the paper's Table 1 protocol: device time of 30 time steps at 512^3 with no output
    (energy recording off), placed beside the paper's 13 machines (context only)"""
    kg.kg_set_options(precision=prec, energy_every=0)
    d_u0 = torch.from_numpy(u0).to(f"cuda:{local}")
    kg.kg_init_device(NG, L_BOX, DT, d_u0, None)
    del d_u0
    kg.kg_step(3)
    stream.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    kg.kg_step(30)
    e1.record(stream)
    e1.synchronize()
    sec = e0.elapsed_time(e1) * 1e-3
    best = PAPER_TABLE1[0]
    return {"steps": 30, "seconds": round(sec, 5), "ms_per_step": round(sec / 30 * 1e3, 3),
            "faster_than_n_of_13": sum(1 for _, _, t in PAPER_TABLE1 if sec < t),
            "paper_fastest": {"machine": best[0], "cores": best[1], "seconds": best[2]},
            "ratio_to_paper_fastest": round(best[2] / sec, 2)}


def ensemble_point(kg, prec, steps, torch, stream, early_exit=False):
    """512 instances (256 x 64^3 + 256 x 128^3, A ~ U[0.5,4], s ~ U[0.5,2], seed 4, dt = 0.005):
    one persistent launch per step vs the plain one-instance-at-a-time loop (kg_init + kg_step),
    both for `steps` fixed steps without early exits, same precision; with early_exit also the
    blow-up run (up to 2000 steps, max|u| > 1e3 freezes an instance, only active instance-steps
    counted)"""
    from paper_1501_04552_gb300 import inputs as I
    Ns, A, s = I.ensemble_params(512, 4)
    kg.kg_set_options(precision=prec)
    kg.kg_ens_init(Ns, L_BOX, DT, A, s)
    bps, order = kg.kg_ens_tune(2)                 # tuned on a throw-away copy
    kg.kg_ens_init(Ns, L_BOX, DT, A, s)
    sched = kg.kg_ens_schedule()[0]
    kg.kg_ens_run(3)
    done, ms = kg.kg_ens_run(steps, 0.0)
    res = kg.kg_ens_results()
    ens_rate = float(res["level"].sum() - 3 * len(Ns)) / (ms * 1e-3)
    blowup = None
    if early_exit:
        kg.kg_ens_init(Ns, L_BOX, DT, A, s)
        bdone, bms = kg.kg_ens_run(2000, 1e3)
        br = kg.kg_ens_results()
        active = float(br["level"].sum())      # a frozen instance stops at its blow-up level
        blowup = {"max_steps": 2000, "threshold": 1e3, "steps_run": int(bdone),
                  "blown_up": int(br["frozen"].sum()), "active_instance_steps": int(active),
                  "seconds": round(bms * 1e-3, 3), "active_instance_steps_per_s": round(active / (bms * 1e-3), 1)}
    kg.kg_ens_finalize()
    # plain loop on a sample of the same instances
    sample = list(range(0, 256, 43)) + list(range(256, 512, 43))
    plain_steps = max(20, steps // 4)
    tot_ms, tot_steps = 0.0, 0
    by_size = {64: [0.0, 0], 128: [0.0, 0]}
    for i in sample:
        N = int(Ns[i])
        kg.kg_init(N, L_BOX, DT, I.gaussian(N, L_BOX, A[i], s[i]), None)
        kg.kg_step(3)
        stream.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        kg.kg_step(plain_steps)
        e1.record(stream)
        e1.synchronize()
        tot_ms += e0.elapsed_time(e1)
        tot_steps += plain_steps
        by_size[N][0] += e0.elapsed_time(e1)
        by_size[N][1] += plain_steps
    kg.kg_finalize()
    # the plain loop's mix is 50/50 in instances like the ensemble, so its rate is the
    # harmonic combination of the per-size rates
    plain_rate = tot_steps / (tot_ms * 1e-3)
    plain_by_size = {"%d^3" % n: round(v[1] / (v[0] * 1e-3), 1) for n, v in by_size.items() if v[1]}
    # roofline of the ensemble step: the double-float transforms are bound by the FP32 lanes of
    # the FMA pipes (operation count of df64_step_ops), the FP32 ones by HBM (11 S or 7 S per instance)
    n64, n128 = int((Ns == 64).sum()), int((Ns == 128).sum())
    if prec == "df64":
        ops = n64 * df64_step_ops(64) + n128 * df64_step_ops(128)
        bound_rate = FP32_ISSUE_PEAK / ops * len(Ns)
        roof = {"bound": "alu", "unit": "instance-steps/s", "peak": round(bound_rate, 1),
                "frac": round(ens_rate / bound_rate, 4), "peak_kind": "FP32 lane peak / double-float operations"}
    else:
        per = lambda n: n * n * (n // 2 + 1) * 16 * (11 if prec == "fp64" else 7)
        byts = n64 * per(64) + n128 * per(128)
        hbm, kind = peaks()
        bound_rate = hbm * 1e9 / byts * len(Ns)
        roof = {"bound": "hbm", "unit": "instance-steps/s", "peak": round(bound_rate, 1),
                "frac": round(ens_rate / bound_rate, 4), "peak_kind": kind + " HBM / algorithmic bytes"}
    return {"instances": int(len(Ns)), "grids": "256 x 64^3 + 256 x 128^3", "steps": int(done),
            "roofline": roof, "tuned_schedule": sched,
            "instance_steps_per_s": round(ens_rate, 1), "plain_loop_instance_steps_per_s": round(plain_rate, 1),
            "speedup_vs_plain": round(ens_rate / plain_rate, 3), "precision": prec,
            "plain_loop_by_grid": plain_by_size,
            "tuned_blocks_per_sm": bps, "tuned_order": order,
            "plain_sample": "%d instances x %d steps (kg_init + kg_step each)" % (len(sample), plain_steps),
            "blowup_run": blowup,
            "blowup_speedup_vs_plain": (round(blowup["active_instance_steps_per_s"] / plain_rate, 3)
                                        if blowup else None)}


def torch_fft_point(u0, local):
    """the same step written with torch.fft (cuFFT) in FP64 and FP32: a same-GPU reference point"""
    import torch
    out = {}
    N = u0.shape[0]
    kf = 2 * np.pi / L_BOX
    m = torch.fft.fftfreq(N, 1.0 / N, dtype=torch.float64, device=f"cuda:{local}")
    mx = torch.fft.rfftfreq(N, 1.0 / N, dtype=torch.float64, device=f"cuda:{local}")
    k2 = kf * kf * (mx[None, None, :] ** 2 + m[None, :, None] ** 2 + m[:, None, None] ** 2)
    om2 = 1 + k2
    a = DT * DT * om2 / 4
    c2 = 2 * (1 - a) / (1 + a)
    b2 = DT * DT / (1 + a)
    del k2, om2, a
    for dt_name, fdt in [("f64", torch.float64), ("f32", torch.float32)]:
        u = torch.from_numpy(u0).to(f"cuda:{local}")
        A = torch.fft.rfftn(u)
        B = A.clone()
        cdt = torch.complex128 if fdt == torch.float64 else torch.complex64
        c2f, b2f = c2.to(fdt), b2.to(fdt)

        def step(A, B):
            uu = torch.fft.irfftn(A.to(cdt), s=(N, N, N))
            F = torch.fft.rfftn(uu * uu * uu).to(torch.complex128)
            return c2 * A - B + b2 * F, A

        for _ in range(3):
            A, B = step(A, B)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        n = 10
        e0.record()
        for _ in range(n):
            A, B = step(A, B)
        e1.record()
        e1.synchronize()
        out[dt_name] = {"steps_per_s": round(n / (e0.elapsed_time(e1) * 1e-3), 2)}
        del A, B, u
        torch.cuda.empty_cache()
    return out


if __name__ == "__main__":
    sys.exit(main())
