"""Throughput benchmark of the GB300 min-max NB-LDPC decoder.

One step decodes the GF(64) (x^6+x+1) regular (2,4) rate-1/2 N=576 workload:
65536 frames at each of Eb/N0 = 1.5, 2.0 and 2.5 dB (196608 frames, one
nbldpc_decode call), up to 20 iterations with syndrome early stop.  Inputs
(7.2 GB of uint8 reliabilities) are synthetic, seeded, and resident in HBM
before the timed region; they are larger than L2, so no flush is needed.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

Prints one JSON line (rank 0).  With torchrun, every rank decodes its own
batch (weak scaling, no data-path collective); the timing is the max over
ranks.  --impl reference times the CPU oracle on the host cores instead.

At N=1 the line also carries: the integer min/max peak measured by the
throughput probe (the roofline's denominator), one sub-line per other
min-max workload (GF(4) N=48: 1000 frames, 10 fixed iterations, plain and
CUDA-graph replayed; GF(256) (2,6) N=384: 16384 frames, up to 20 iterations),
the four-code persistent batch against the plain decoder, and a short
serving sweep.
"""
from __future__ import annotations

import argparse
import hashlib
import gc
import json
import os
import platform
import re
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402
import torch  # noqa: E402

WORKLOAD = "gf64_n576_dv2_dc4"
SM_COUNT = 152
# Issue-bound min/max ceiling: an SM issues 4 warp instructions per clock; a
# min-max pair costs at best one instruction per lane per two 16-bit pairs
# (max on the ALU or, as relu(a-b)+b, on the FMA pipe; 3-input min on the ALU),
# i.e. 128 pairs = 256 16-bit min/max ops per clock per SM.
PEAK_OPS_PER_CLK_SM = 256
SM_MAX_MHZ_FALLBACK = 2070.0


def sm_max_mhz():
    """Maximum SM clock: the measured-peaks file written for this GPU pool, else 2070 MHz."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return float(json.load(fh)["sm_max_mhz"]), "measured"
    except (OSError, KeyError, ValueError):
        return SM_MAX_MHZ_FALLBACK, "fallback"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--workload", default="gf64",
                    choices=["gf64", "gf4", "gf256", "peak", "mixed", "serving", "width", "fftspa", "schedule"],
                    help="gf64: the GF(64) N=576 headline step; gf4: GF(4) N=48, 1000 frames, 10 fixed "
                         "iterations (plain and CUDA-graph replayed); gf256: GF(256) (2,6) N=384, 16384 frames; "
                         "peak: the integer min/max throughput probe; mixed: the four-code batch, persistent vs "
                         "plain; serving: Poisson request arrivals, continuous batching vs plain; width: 8-bit "
                         "against 16-bit messages (throughput and frame error rate); fftspa: the GF(64) step "
                         "decoded with FFT-SPA (Alg. 1) from float channel probabilities; schedule: 3(d_c-2) "
                         "against Table 1's 3 d_c - 4 check-node convolutions")
    ap.add_argument("--seconds", type=float, default=6.0, help="serving: arrival window per load point")
    ap.add_argument("--frames", type=int, default=None, help="frames per Eb/N0 point (default: 65536)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-autotune", action="store_true", help="keep the default layout / frames per block")
    ap.add_argument("--no-extras", action="store_true",
                    help="default line: skip the probe, the other workloads, the mixed batch and serving")
    ap.add_argument("--probe-seconds", type=float, default=0.6, help="peak: seconds per probe form")
    ap.add_argument("--probe-rounds", type=int, default=0,
                    help="peak: fixed rounds per launch, one launch per form (no calibration)")
    ap.add_argument("--probe-forms", default="", help="peak: comma-separated probe forms (default: all)")
    return ap.parse_args()


def dist_setup(args):
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if ws > 1 and args.impl == "gb300":
        torch.cuda.set_device(local)
        torch.distributed.init_process_group("nccl")
    return ws, rank, local


def strip_comments(text: str) -> str:
    """C/C++ source without comments, whitespace runs collapsed to one space (string and
    character literals kept as written)."""
    out, i, n = [], 0, len(text)
    while i < n:
        c = text[i]
        if c in "\"'":
            j = i + 1
            while j < n and text[j] != c:
                j += 2 if text[j] == "\\" else 1
            out.append(text[i:j + 1])
            i = j + 1
        elif text.startswith("//", i):
            j = text.find("\n", i)
            i = n if j < 0 else j
        elif text.startswith("/*", i):
            j = text.find("*/", i + 2)
            i = n if j < 0 else j + 2
            out.append(" ")
        else:
            out.append(c)
            i += 1
    return " ".join("".join(out).split())


def kernel_code_hash(source: str = "mma_kernels.cuh") -> str:
    """Fingerprint of a kernel header's code: sha256 of the source without comments and
    with whitespace collapsed, so that a comment edit keeps its profile."""
    with open(os.path.join(ROOT, "paper_2508_03567_gb300", "csrc", source), encoding="utf-8") as fh:
        code = strip_comments(fh.read())
    return hashlib.sha256(code.encode()).hexdigest()[:16]


def profiled_traffic(profile: str = "mma_decode_kernel_gf64_n576.md", source: str = "mma_kernels.cuh"):
    """DRAM bytes per frame from a committed ncu summary, if it was taken on the current kernel code."""
    path = os.path.join(ROOT, "profiles", profile)
    if not os.path.exists(path):
        return None, None
    txt = open(path).read()
    m_hash = re.search(r"kernel_code_sha256_16:\s*([0-9a-f]+)", txt)
    m_bpf = re.search(r"dram_bytes_per_frame:\s*([0-9.eE+]+)", txt)
    if not m_hash or not m_bpf or m_hash.group(1) != kernel_code_hash(source):
        return None, path
    return float(m_bpf.group(1)), path


class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
        return self

    def __exit__(self, *a):
        self.rows = []
        if self.proc is None:
            return
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
            out, _ = self.proc.communicate()
        for line in out.strip().splitlines():
            parts = [p.strip() for p in line.split(",")]
            if len(parts) == 7:
                self.rows.append(parts)

    def summary(self):
        if not getattr(self, "rows", None):
            return None
        sm = [float(r[0]) for r in self.rows if r[0].replace(".", "").isdigit()]
        mx = [float(r[1]) for r in self.rows if r[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in self.rows for i in range(4) if r[3 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(self.rows)}


def make_inputs(code, w, frames_per_point, device, rank):
    return make_inputs_cw(code, w, frames_per_point, device, rank)[0]


def cpu_model() -> str:
    """CPU model string of this host (lscpu, else /proc/cpuinfo, else the machine type)."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.strip().startswith("Model name"):
                return line.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    try:
        with open("/proc/cpuinfo") as fh:
            for line in fh:
                if line.lower().startswith("model name"):
                    return line.split(":", 1)[1].strip()
    except OSError:
        pass
    return platform.processor() or platform.machine()


def oracle_rate(name, frames_per_point, threads):
    """Info Mbit/s of the CPU oracle on a bounded sample of workload `name` (the
    first frames of each Eb/N0 point's stream), with `threads` threads."""
    import oracle
    from paper_2508_03567_gb300 import inputs as I
    w = I.WORKLOADS[name]
    code = I.workload_code(name)
    g = np.concatenate([I.make_batch(code, eb, I.workload_seed(name, i), frames_per_point).gamma.numpy()
                        for i, eb in enumerate(w["ebn0"])], 0)
    t0 = time.perf_counter()
    oracle.decode(code, g, w["max_iters"], w["early_stop"], threads=threads)
    dt = time.perf_counter() - t0
    return g.shape[0] * code.k * code.p / dt / 1e6, dt, g.shape[0]


def cpu_baseline(name, frames_all, frames_single):
    """The oracle as it stands, on this host: all cores (a thread pool over
    frames) and one thread, each on a bounded sample of the workload."""
    threads = os.cpu_count() or 1
    rate, dt, f = oracle_rate(name, frames_all, threads)
    rate1, dt1, f1 = oracle_rate(name, frames_single, 1)
    return {"value": rate, "unit": "Mbit/s", "cores": threads, "kind": "oracle",
            "sample": f"{f} frames ({frames_all} per Eb/N0 point) of the same workload, {dt:.1f} s wall",
            "single_thread": {"value": rate1, "unit": "Mbit/s", "cores": 1,
                              "sample": f"{f1} frames ({frames_single} per Eb/N0 point), {dt1:.1f} s wall"},
            "nproc": threads, "cpu_model": cpu_model(), "machine": platform.machine()}


def run_reference(args, ws, rank):
    if rank != 0:
        return 0
    from paper_2508_03567_gb300 import inputs as I
    w = I.WORKLOADS[WORKLOAD]
    code = I.workload_code(WORKLOAD)
    threads = os.cpu_count() or 1
    sample = 8
    for _ in range(args.warmup):
        oracle_rate(WORKLOAD, 2, threads)
    times, bits = [], 0
    for _ in range(args.steps):
        rate, dt, f = oracle_rate(WORKLOAD, sample, threads)
        times.append(dt)
        bits += f * code.k * code.p
    value = bits / sum(times) / 1e6
    line = {"metric": "decoded info Mbit/s", "value": value, "unit": "Mbit/s", "n_gpus": 0,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * statistics.mean(times),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u8",
            "data": "synthetic", "impl": "reference",
            "config": {"workload": WORKLOAD, "frames_per_step": 3 * sample, "max_iters": w["max_iters"],
                       "early_stop": True, "ebn0_db": list(w["ebn0"])},
            "cpu_baseline": {"value": value, "unit": "Mbit/s", "cores": threads, "kind": "oracle",
                             "sample": f"{sample} frames per Eb/N0 point per step (of 65536)",
                             "nproc": threads, "cpu_model": cpu_model(), "machine": platform.machine()},
            "e2e": {"value": value, "unit": "Mbit/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def convolutions_per_frame_iter(code, table1=False):
    """XOR min-max convolutions of one check-node pass: per check of degree d,
    3(d-2) (forward and backward over d-2 edges, d-2 middle outputs) or, with
    `table1`, the 3d-4 of Table 1 of the paper (forward and backward over d-1
    edges each)."""
    d = np.diff(code.row_ptr).astype(np.int64)
    return int((3 * d - 4).sum()) if table1 else int((3 * np.maximum(d - 2, 0)).sum())


def pairs_per_frame_iter(code):
    """Min-max pairs of one check-node pass: sum over checks of 3(d-2) q^2."""
    return convolutions_per_frame_iter(code) * code.q * code.q


# ---------------------------------------------------------------- integer peak
# Probe forms (nbldpc_probe_minmax): the instruction mixes of the convolution's
# inner loop on registers, and the convolution itself on shared memory.
PROBE_FORMS = (("alu", 0), ("fma_1_8", 1), ("fma_3_8", 2), ("fma_4_8", 3), ("fma_3_8_shfl", 4))
CONV_FORMS = (("conv_gf64", 5), ("conv_gf256", 6))


def sm_count(dev) -> int:
    return torch.cuda.get_device_properties(dev).multi_processor_count


def run_probe_form(binding, form, seconds, dev, stream, fixed_rounds=0):
    """One probe launch of about `seconds` (the round count calibrated on shorter launches),
    or of `fixed_rounds` rounds."""
    sink = torch.zeros(1, dtype=torch.int32, device=dev)
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    rounds, cap = (fixed_rounds or 64), 1 << 26
    for _ in range(0 if fixed_rounds else 10):
        a.record(stream)
        binding.nbldpc_probe_minmax(form, rounds, sink, stream=stream)
        b.record(stream)
        b.synchronize()
        ms = a.elapsed_time(b)
        if ms >= 0.5e3 * seconds or rounds >= cap:
            break
        rounds = int(min(cap, rounds * max(2.0, 1e3 * seconds / max(ms, 1e-3))))
    a.record(stream)
    pairs, blocks = binding.nbldpc_probe_minmax(form, rounds, sink, stream=stream)
    b.record(stream)
    b.synchronize()
    ms = a.elapsed_time(b)
    return {"pairs_per_s": pairs / (ms / 1e3), "ms": ms, "rounds": rounds, "blocks": blocks}


def measure_peak(binding, dev, local, seconds, forms=PROBE_FORMS + CONV_FORMS, fixed_rounds=0):
    """Min-max pairs per clock per SM of each probe form, using the SM clock
    sampled while the probes ran (time x median MHz); the best register form
    is the integer peak of the roofline."""
    stream = torch.cuda.Stream(device=dev)
    sms = sm_count(dev)
    res = {}
    with ClockSampler(local) as clk:
        for label, form in forms:
            res[label] = run_probe_form(binding, form, seconds, dev, stream, fixed_rounds)
    clocks = clk.summary() or {}
    mhz = clocks.get("sm_mhz") or sm_max_mhz()[0]
    for r in res.values():
        r["pairs_per_clk_sm"] = r["pairs_per_s"] / (sms * mhz * 1e6)
    reg = [lab for lab, _ in PROBE_FORMS if lab in res] or list(res)
    best = max(reg, key=lambda k: res[k]["pairs_per_clk_sm"])
    return {"forms": res, "best_form": best, "pairs_per_clk_sm": res[best]["pairs_per_clk_sm"], "sms": sms,
            "clock_mhz_used": mhz, "clocks": clocks}


def alu_peaks(peak_meas, dev):
    """(measured peak Gop/s, its description, issue-bound peak Gop/s) in 16-bit min/max ops
    (a min-max pair = 2 ops), both at the maximum SM clock."""
    mhz, mhz_kind = sm_max_mhz()
    sms = sm_count(dev)
    issue = sms * PEAK_OPS_PER_CLK_SM * mhz * 1e6 / 1e9
    if not peak_meas:
        return issue, (f"derived: {sms} SMs x {PEAK_OPS_PER_CLK_SM} u16 min/max ops/clk (issue-bound ALU+FMA "
                       f"mix) x {mhz:.0f} MHz ({mhz_kind} max SM clock)"), issue
    ppc = peak_meas["pairs_per_clk_sm"]
    meas = sms * 2 * ppc * mhz * 1e6 / 1e9
    return meas, (f"measured: probe form {peak_meas['best_form']} at {ppc:.1f} min-max pairs/clk/SM "
                  f"(x 2 u16 ops) x {sms} SMs x {mhz:.0f} MHz ({mhz_kind} max SM clock)"), issue


HBM_FALLBACK_GBS = 6800.0


def hbm_peak_gbs():
    """Measured HBM copy bandwidth of this GPU pool (the measured-peaks file), else the fallback."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return float(json.load(fh)["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return HBM_FALLBACK_GBS, "fallback"


def algorithmic_bytes_per_frame(code) -> int:
    """HBM bytes one frame must move: its reliabilities in, its symbols, iteration count and ok flag out."""
    return code.n * code.q + code.n + 5


def roofline_alu(achieved, peak, peak_kind, issue, traffic=None, hbm_bytes_per_s=None, dense=None):
    """achieved: 16-bit min/max ops per second the kernel executed (2 per visited pair); dense: the
    same rate counted as if every convolution visited all q^2 pairs (the paper's operation count),
    reported beside it when the convolutions are pruned."""
    r = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "Gop/s", "frac": achieved / peak,
         "traffic": traffic, "peak_kind": peak_kind, "peak_issue_bound": issue,
         "frac_issue_bound": achieved / issue}
    if dense is not None and abs(dense - achieved) > 1e-9 * max(dense, 1.0):
        r["work"] = "executed (pruned convolutions)"
        r["dense_equivalent"] = {"achieved": dense, "frac": dense / peak, "frac_issue_bound": dense / issue}
    if hbm_bytes_per_s is not None:
        # the other roof: algorithmic HBM bytes per second against the measured copy bandwidth
        gbs, kind = hbm_peak_gbs()
        r["hbm"] = {"achieved": hbm_bytes_per_s / 1e9, "peak": gbs, "unit": "GB/s",
                    "frac": hbm_bytes_per_s / 1e9 / gbs, "peak_kind": kind}
    return r


def visited_pairs(binding, dec, decodes, dev):
    """Pairs (x, y) the convolutions of `decodes` (callables queuing one decode each on the current
    stream) visit, from the library's work counter; an untimed run of the timed decodes' inputs."""
    cnt = torch.zeros(1, dtype=torch.int64, device=dev)
    binding.nbldpc_code_set_work_counter(dec.handle, cnt)
    try:
        for f in decodes:
            f()
        torch.cuda.synchronize()
    finally:
        binding.nbldpc_code_set_work_counter(dec.handle, None)
    return int(cnt.item())


def run_peak(args, ws, rank, local):
    """Every probe form for --probe-seconds each: min-max pairs per clock per SM."""
    import __graft_entry__
    __graft_entry__.build()
    from paper_2508_03567_gb300 import binding
    if rank != 0:
        return 0
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    forms = PROBE_FORMS + CONV_FORMS
    if args.probe_forms:
        want = args.probe_forms.split(",")
        forms = tuple(f for f in forms if f[0] in want)
    meas = measure_peak(binding, dev, local, args.probe_seconds, forms, args.probe_rounds)
    peak, kind, issue = alu_peaks(meas, dev)
    line = {"metric": "integer min/max throughput (min-max pairs per clock per SM)",
            "value": meas["pairs_per_clk_sm"], "unit": "pairs/clk/SM", "n_gpus": 1, "steps": 1, "warmup": 1,
            "ms_per_step": None, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "u16x2", "data": "synthetic",
            "config": {"workload": "throughput probe of the convolution's instruction forms",
                       "seconds_per_form": args.probe_seconds},
            "peak_gops": peak, "peak_kind": kind, "issue_bound_gops": issue, "probe": meas,
            "gpu_launches": None}
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------- one min-max workload
L2_BYTES = 129e6


def batch_pool(step_bytes: float) -> int:
    """Distinct batches a workload rotates through so that the inputs of one timed
    decode are not in L2: 1 when one step's inputs exceed L2, else enough batches
    for twice the L2 size."""
    return 1 if step_bytes > L2_BYTES else int(np.ceil(2 * L2_BYTES / step_bytes))


def measure_workload(binding, I, name, dev, local, args, peaks, steps, warmup, frames=None, graph=False,
                     cpu_frames=None, e2e=True, profile=None):
    """One min-max workload of inputs.WORKLOADS through nbldpc_decode: its frames
    at every Eb/N0 point (inputs resident in HBM), `warmup` untimed and `steps`
    timed decodes (CUDA events on the launching stream), info Mbit/s, frame
    error rate against the transmitted codewords, the ALU roofline, clocks,
    and optionally a CUDA-graph replay, the e2e host-buffer decode and the CPU
    oracle on a sample.  A step whose inputs are smaller than L2 is one batch
    of a pool of distinct batches, 2 x L2 in all, decoded in turn, so that no
    timed decode finds its inputs in L2; the graph then holds one decode per
    batch of the pool."""
    w = I.WORKLOADS[name]
    code = I.workload_code(name)
    fpp = frames or w["frames"]
    npts = len(w["ebn0"])
    step_bytes = npts * fpp * code.n * code.q
    pool = batch_pool(step_bytes)
    gam, cws = [], []
    for i, eb in enumerate(w["ebn0"]):
        bt = I.make_batch(code, eb, I.workload_seed(name, i), pool * fpp, device=dev, chunk=65536)
        gam.append(bt.gamma.view(pool, fpp, code.n, code.q))
        cws.append(bt.codewords.view(pool, fpp, code.n))
    gamma = torch.cat(gam, 1).contiguous()                 # [pool, frames per step, n, q]
    cw = torch.cat(cws, 1)
    del gam, cws
    nf = gamma.shape[1]
    dec = binding.Decoder.from_code(code)
    tuning = {"source": "default"}
    if not args.no_autotune:
        res = dec.autotune(gamma[0][: min(nf, 4096)], 3)
        tuning = {"source": "autotuned", "candidates_ms": {f"v{v}_fpb{f}": round(ms, 3) for v, f, ms in res}}
    v, fpb = dec.tuning()
    tuning.update({"variant": v, "frames_per_block": fpb})
    stream = torch.cuda.Stream(device=dev)
    sym = torch.empty((pool, nf, code.n), dtype=torch.uint8, device=dev)
    its = torch.empty((pool, nf), dtype=torch.int32, device=dev)
    ok = torch.empty((pool, nf), dtype=torch.uint8, device=dev)
    wsb = dec.workspace(nf, dev)
    mi, es = w["max_iters"], w["early_stop"]

    def step(i):
        b = i % pool
        binding.nbldpc_decode(dec.handle, gamma[b], nf, mi, es, sym[b], its[b], ok[b], wsb, stream=stream)

    with torch.cuda.stream(stream):
        for i in range(warmup):
            step(i)
        for i in range(warmup, pool):      # every batch of the pool decoded once (outputs for the FER)
            step(i)
    torch.cuda.synchronize()
    ksteps = max(steps, min(pool, 1000))
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(ksteps)]
    launches0 = binding.nbldpc_kernel_launch_count()
    with ClockSampler(local) as clk:
        for i, (a, b) in enumerate(ev):
            a.record(stream)
            step(warmup + i)
            b.record(stream)
        torch.cuda.synchronize()
    launches = binding.nbldpc_kernel_launch_count() - launches0
    step_ms = [a.elapsed_time(b) for a, b in ev]
    kernel_s = statistics.mean(step_ms) / 1e3
    its_h = its.cpu().numpy().astype(np.int64)
    pairs_step = int(its_h.sum()) * pairs_per_frame_iter(code) / pool
    with torch.cuda.stream(stream):
        visited_step = visited_pairs(binding, dec, [lambda b=b: step(b) for b in range(pool)], dev) / pool
    achieved = 2 * visited_step / kernel_s / 1e9
    peak, kind, issue = peaks
    bpf = profiled_traffic(profile)[0] if profile else None
    info_bits = nf * code.k * code.p
    out = {"workload": name, "value": info_bits / kernel_s / 1e6, "unit": "Mbit/s", "steps": ksteps,
           "warmup": warmup, "ms_per_step": 1e3 * kernel_s, "median_ms_per_step": statistics.median(step_ms),
           "config": {"q": code.q, "n": code.n, "k": code.k, "dv": w["dv"], "dc": w["dc"], "frames_per_step": nf,
                      "ebn0_db": list(w["ebn0"]), "max_iters": mi, "early_stop": bool(es), "tuning": tuning,
                      "l2": "inputs larger than L2 (no flush)" if pool == 1 else
                            f"each step decodes the next of {pool} distinct {nf}-frame batches "
                            f"({pool * step_bytes / 1e6:.0f} MB of inputs, > L2; no flush)"},
           "roofline": roofline_alu(achieved, peak, kind, issue, None if bpf is None else bpf * nf,
                                    nf * algorithmic_bytes_per_frame(code) / kernel_s,
                                    dense=2 * pairs_step / kernel_s / 1e9),
           "clocks": clk.summary(), "gpu_launches": int(launches),
           "fer": float((sym.to(torch.int64) != cw).any(-1).float().mean()),
           "not_ok": float(1 - ok.float().mean()), "mean_iters": float(its_h.mean()),
           "pairs_per_step": pairs_step, "visited_pairs_per_step": visited_step,
           "coded_mbps": info_bits / kernel_s / 1e6 * code.n / code.k}
    if graph:
        # one decode per batch of the pool (or `steps` decodes of the one batch) captured in a CUDA graph
        reps = pool if pool > 1 else steps
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=stream):
            for i in range(reps):
                step(i)

        def replay():
            with torch.cuda.stream(stream):
                g.replay()
        replay()
        torch.cuda.synchronize()
        nrep = 5
        gev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(nrep)]
        with ClockSampler(local) as gclk:
            for a, b in gev:
                a.record(stream)
                replay()
                b.record(stream)
            torch.cuda.synchronize()
        per = sum(a.elapsed_time(b) for a, b in gev) / (nrep * reps) / 1e3
        out["graph"] = {"value": info_bits / per / 1e6, "unit": "Mbit/s", "ms_per_decode": 1e3 * per,
                        "decodes_per_replay": reps, "replays": nrep, "clocks": gclk.summary(),
                        "roofline": roofline_alu(2 * pairs_step / per / 1e9, peak, kind, issue),
                        "form": f"{reps} nbldpc_decode calls captured in one CUDA graph, replayed"}
        if not out["clocks"]:
            out["clocks"] = gclk.summary()
    if e2e and not args.no_e2e:
        out["e2e"] = measure_e2e(binding, dec, code, gamma[0], mi, es, args, dev)
    if cpu_frames and not args.no_cpu:
        out["cpu_baseline"] = cpu_baseline(name, *cpu_frames)
    del gamma
    return out


def run_mixed(args, ws, rank, local, emit=True, steps=None, warmup=None, peaks=None):
    """Four codes in one persistent launch (graph-replayed) against one
    fixed-iteration launch per code (the plain batch decoder).  With emit=False
    the line is returned instead of printed."""
    import __graft_entry__
    __graft_entry__.build()
    from paper_2508_03567_gb300 import binding, inputs as I
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    counts = I.mixed_frame_counts()
    codes = [I.workload_code(n) for n in I.MIXED_SET]
    max_iters = 30
    gam, cws, decs, outs, tuning = [], [], [], [], {}
    for k, (code, f) in enumerate(zip(codes, counts)):
        b = I.make_batch(code, I.MIXED_EBN0, I.MIXED_SEED * 100 + k + 7919 * rank, f, device=dev)
        gam.append(b.gamma.contiguous())
        cws.append(b.codewords)
        d = binding.Decoder.from_code(code)
        if not args.no_autotune:
            d.autotune(gam[-1][: min(f, 2048)], 3)
        tuning[code.name] = dict(zip(("variant", "frames_per_block"), d.tuning()))
        decs.append(d)
        outs.append((torch.empty((f, code.n), dtype=torch.uint8, device=dev),
                     torch.empty((f,), dtype=torch.int32, device=dev),
                     torch.empty((f,), dtype=torch.uint8, device=dev)))
    steps = steps or args.steps
    warmup = warmup or args.warmup
    jobs = [(d.handle, g, g.shape[0], max_iters, 1, *o) for d, g, o in zip(decs, gam, outs)]
    wsb = torch.empty(binding.nbldpc_decode_batch_workspace_size(jobs), dtype=torch.uint8, device=dev)
    stream = torch.cuda.Stream(device=dev)
    info_bits = sum(f * c.k * c.p for c, f in zip(codes, counts))

    def fer_of(sym_list):
        bad = sum(int((s.to(torch.int64) != cw).any(1).sum()) for s, cw in zip(sym_list, cws))
        return bad / sum(counts)

    def timed(fn, steps):
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        torch.cuda.synchronize()
        for a, b in ev:
            a.record(stream)
            fn()
            b.record(stream)
        torch.cuda.synchronize()
        return sum(a.elapsed_time(b) for a, b in ev) / 1e3

    # persistent mixed batch, captured once and replayed
    for _ in range(warmup):
        binding.nbldpc_decode_batch(jobs, wsb, stream=stream)
    stream.synchronize()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=stream):
        binding.nbldpc_decode_batch(jobs, wsb, stream=stream)
    def replay():
        with torch.cuda.stream(stream):
            graph.replay()
    with ClockSampler(local) as clk:
        t_pers = timed(replay, steps)
    its_pers = [o[1].cpu().numpy().astype(np.int64) for o in outs]
    fer_pers = fer_of([o[0] for o in outs])
    pairs = sum(int(it.sum()) * pairs_per_frame_iter(c) for it, c in zip(its_pers, codes))
    # pairs the persistent batch's convolutions visit (an untimed decode with every code's counter set)
    cnt = torch.zeros(1, dtype=torch.int64, device=dev)
    for d in decs:
        binding.nbldpc_code_set_work_counter(d.handle, cnt)
    binding.nbldpc_decode_batch(jobs, wsb, stream=stream)
    torch.cuda.synchronize()
    for d in decs:
        binding.nbldpc_code_set_work_counter(d.handle, None)
    visited = int(cnt.item())

    # plain: one fixed-iteration launch per code
    def plain(early):
        for d, g, (sym, its, ok) in zip(decs, gam, outs):
            binding.nbldpc_decode(d.handle, g, g.shape[0], max_iters, early, sym, its, ok,
                                  d.workspace(g.shape[0], dev), stream=stream)
    for _ in range(warmup):
        plain(0)
    t_fixed = timed(lambda: plain(0), steps)
    fer_fixed = fer_of([o[0] for o in outs])
    for _ in range(2):
        plain(1)
    t_early = timed(lambda: plain(1), steps)
    peak, kind, issue = peaks or alu_peaks(None, dev)
    achieved = 2 * visited / (t_pers / steps) / 1e9
    if rank != 0:
        return 0
    line = {
        "metric": "decoded info Mbit/s", "value": ws * steps * info_bits / t_pers / 1e6, "unit": "Mbit/s",
        "n_gpus": ws, "steps": steps, "warmup": warmup,
        "ms_per_step": 1e3 * t_pers / steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "u8", "data": "synthetic",
        "config": {"workload": "mixed4: GF(16) N=1024 (2,4) + GF(64) N=576 (2,4) + GF(32) N=600 (3,6) "
                               "+ GF(256) N=128 (2,8)", "frames": dict(zip(I.MIXED_SET, counts)),
                   "ebn0_db": "uniform per frame in [1.5, 3.5)", "max_iters": max_iters,
                   "form": "one persistent launch per step (CUDA graph replay), early stop + refill",
                   "tuning": tuning},
        "roofline": roofline_alu(achieved, peak, kind, issue, dense=2 * pairs / (t_pers / steps) / 1e9),
        "clocks": clk.summary(),
        "gpu_launches": steps,   # one decode kernel per graph replay
        "fer": fer_pers,
        "plain_fixed_iterations": {"value": ws * steps * info_bits / t_fixed / 1e6, "unit": "Mbit/s",
                                   "ms_per_step": 1e3 * t_fixed / steps, "fer": fer_fixed,
                                   "form": "one launch per code, 30 iterations, no early stop"},
        "plain_early_stop": {"value": ws * steps * info_bits / t_early / 1e6, "unit": "Mbit/s",
                             "ms_per_step": 1e3 * t_early / steps,
                             "form": "one launch per code, early stop"},
        "mean_iters": {c.name: float(it.mean()) for c, it in zip(codes, its_pers)},
    }
    if not emit:
        return line
    print(json.dumps(line), flush=True)
    return 0


def run_serving(args, ws, rank, local, emit=True, loads_c=(0.10, 0.25, 0.50, 0.75, 0.90, 1.00),
                loads_p=(0.10, 0.25, 0.50), seconds=None):
    """Poisson arrivals of requests (one of the four mixed-set codes, uniform;
    1-256 frames, uniform; per-frame Eb/N0 uniform in [1.5, 3.5) dB) served by
    continuous batching, load swept over fractions of the measured peak, and
    by the plain one-launch-per-request decoder.  With emit=False the line is
    returned instead of printed."""
    import __graft_entry__
    __graft_entry__.build()
    from paper_2508_03567_gb300 import binding, inputs as I
    from paper_2508_03567_gb300.serving import CudaExecutor, Request, Server, percentile
    if rank != 0:
        return 0
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    codes = [I.workload_code(n) for n in I.MIXED_SET]
    decs = [binding.Decoder.from_code(c) for c in codes]
    max_iters = 30
    rng = np.random.Generator(np.random.PCG64(4242))
    pool = []
    for i in range(96):
        k = int(rng.integers(len(codes)))
        f = int(rng.integers(1, 257))
        g = I.make_batch(codes[k], I.MIXED_EBN0, 60000 + i, f, device=dev).gamma.cpu().pin_memory()
        pool.append((k, g))
    if not args.no_autotune:
        for k, d in enumerate(decs):
            g = torch.cat([gg for kk, gg in pool if kk == k][:8]).to(dev)
            d.autotune(g[:2048], 3)
    bits_of = lambda k, f: f * codes[k].k * codes[k].p
    mean_bits = float(np.mean([bits_of(k, g.shape[0]) for k, g in pool]))
    budget = 8 << 30

    def serve(mode, rate, seconds, seed, saturate=False, cap=60.0):
        ex = CudaExecutor(decs, max_iters=max_iters, streams=3)
        srv = Server(ex, budget_bytes=budget, streams=3, mode=mode)
        r = np.random.Generator(np.random.PCG64(seed))
        reqs = []
        # no garbage-collector pause inside the window: the polling loop is what
        # observes completions, so a pause would show up as request latency
        gc.collect()
        gc.disable()
        try:
            return window(srv, r, reqs, rate, seconds, saturate, cap)
        finally:
            gc.enable()

    def window(srv, r, reqs, rate, seconds, saturate, cap):
        t0 = time.perf_counter()
        if saturate:
            for i in range(2 * len(pool)):
                k, g = pool[i % len(pool)]
                reqs.append(Request(rid=i, code=k, gamma=g))
                srv.submit(reqs[-1], now=t0)
        else:
            t_next = t0 + r.exponential(1.0 / rate)
            while True:
                now = time.perf_counter()
                while t_next <= now and t_next - t0 < seconds:
                    k, g = pool[int(r.integers(len(pool)))]
                    reqs.append(Request(rid=len(reqs), code=k, gamma=g))
                    srv.submit(reqs[-1], now=t_next)
                    t_next += r.exponential(1.0 / rate)
                srv.poll()
                if now - t0 >= seconds:
                    break
        while not srv.idle() and time.perf_counter() - t0 < seconds + cap:
            srv.poll()
        done = [q for q in reqs if q.t_done >= 0]
        t_end = max(q.t_done for q in done)
        bits = sum(bits_of(q.code, q.frames) for q in done)
        lat = [1e3 * q.latency for q in done]
        return {"offered_mbps": None if saturate else rate * mean_bits / 1e6,
                "achieved_mbps": bits / (t_end - t0) / 1e6, "requests": len(reqs), "completed": len(done),
                "p50_ms": percentile(lat, 50), "p99_ms": percentile(lat, 99), "launches": srv.launches,
                "peak_resident_bytes": srv.peak_used}

    serve("continuous", 0, 0, 1, saturate=True)      # warm-up
    peak = serve("continuous", 0, 0, 2, saturate=True)
    peak_plain = serve("plain", 0, 0, 3, saturate=True)
    peak_bps = peak["achieved_mbps"] * 1e6
    loads = []
    seconds = seconds or args.seconds
    for i, load in enumerate(loads_c):
        res = serve("continuous", load * peak_bps / mean_bits, seconds, 5000 + i)
        res["load"] = load
        loads.append(res)
    plain = []
    for i, load in enumerate(loads_p):
        res = serve("plain", load * peak_bps / mean_bits, seconds, 5100 + i, cap=20.0)
        res["load"] = load
        plain.append(res)
    line = {"metric": "decoded info Mbit/s; p50/p99 request latency", "value": peak["achieved_mbps"],
            "unit": "Mbit/s", "n_gpus": 1, "steps": len(loads), "warmup": 1,
            "ms_per_step": None, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "u8", "data": "synthetic",
            "config": {"workload": "serving: Poisson requests, code uniform over the four-code set, 1-256 "
                                   "frames, Eb/N0 uniform per frame in [1.5, 3.5) dB, up to 30 iterations, "
                                   "early stop, 8 GB resident budget",
                       "streams": 3, "max_requests_per_launch": 32},
            "peak_continuous": peak, "peak_plain": peak_plain, "loads_continuous": loads,
            "loads_plain": plain}
    if not emit:
        return line
    print(json.dumps(line), flush=True)
    return 0


def run_width(args, ws, rank, local):
    """8-bit against 16-bit messages on the same frames: decoded Mbit/s and
    frame error rate (decided symbols against the transmitted codeword), for
    the GF(64) (2,4) N=576 step and the GF(32) (3,6) N=600 code (three
    messages per symbol, so the variable-node sums are larger)."""
    if args.warmup < 3:
        raise SystemExit("--warmup must be >= 3")
    import __graft_entry__
    __graft_entry__.build()
    from paper_2508_03567_gb300 import binding, inputs as I
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    stream = torch.cuda.Stream(device=dev)
    mhz, mhz_kind = sm_max_mhz()
    peak = SM_COUNT * PEAK_OPS_PER_CLK_SM * mhz * 1e6 / 1e9
    results = {}
    with ClockSampler(local) as clk:
        for name, fpp in ((WORKLOAD, args.frames or 65536), ("gf32_n600_dv3_dc6", args.frames or 65536)):
            w = I.WORKLOADS[name]
            code = I.workload_code(name)
            gam, cws = [], []
            for i, eb in enumerate(w["ebn0"]):
                b = I.make_batch(code, eb, I.workload_seed(name, i) + 7919 * rank, fpp, device=dev, chunk=8192)
                gam.append(b.gamma)
                cws.append(b.codewords)
            gamma = torch.cat(gam, 0).contiguous()
            cw = torch.cat(cws, 0)
            frames = gamma.shape[0]
            sym = torch.empty((frames, code.n), dtype=torch.uint8, device=dev)
            its = torch.empty((frames,), dtype=torch.int32, device=dev)
            ok = torch.empty((frames,), dtype=torch.uint8, device=dev)
            mi, es = w["max_iters"], w["early_stop"]
            row = {"frames": frames, "ebn0_db": list(w["ebn0"]), "max_iters": mi}
            for bits in (8, 16):
                dec = binding.Decoder.from_code(code)
                dec.set_message_bits(bits)
                if not args.no_autotune:
                    dec.autotune(gamma[: min(frames, 4096)], 3)
                wsb = dec.workspace(frames, dev)

                def step():
                    binding.nbldpc_decode(dec.handle, gamma, frames, mi, es, sym, its, ok, wsb, stream=stream)

                with torch.cuda.stream(stream):
                    for _ in range(args.warmup):
                        step()
                torch.cuda.synchronize()
                ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
                      for _ in range(args.steps)]
                for a, b in ev:
                    a.record(stream)
                    step()
                    b.record(stream)
                torch.cuda.synchronize()
                t = sum(a.elapsed_time(b) for a, b in ev) / 1e3
                its_h = its.cpu().numpy().astype(np.int64)
                pairs = int(its_h.sum()) * pairs_per_frame_iter(code)
                ach = 2 * pairs / (t / args.steps) / 1e9
                row[f"{bits}bit"] = {
                    "value": args.steps * frames * code.k * code.p / t / 1e6, "unit": "Mbit/s",
                    "ms_per_step": 1e3 * t / args.steps,
                    "fer": float((sym.to(torch.int64) != cw).any(1).float().mean()),
                    "mean_iters": float(its_h.mean()), "tuning": list(dec.tuning()),
                    "alu_frac": ach / peak}
            results[name] = row
    if rank != 0:
        return 0
    head = results[WORKLOAD]["16bit"]
    line = {
        "metric": "decoded info Mbit/s", "value": ws * head["value"], "unit": "Mbit/s", "n_gpus": ws,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": head["ms_per_step"],
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u16",
        "data": "synthetic",
        "config": {"workload": f"{WORKLOAD} with 16-bit messages (value); 8-bit alongside; "
                               "gf32_n600_dv3_dc6 both widths", "l2": "inputs larger than L2 (no flush)"},
        "roofline": {"bound": "alu", "achieved": head["alu_frac"] * peak, "peak": peak, "unit": "Gop/s",
                     "frac": head["alu_frac"], "traffic": None,
                     "peak_kind": f"derived: 152 SMs x 256 u16 min/max ops/clk x {mhz:.0f} MHz ({mhz_kind})"},
        "clocks": clk.summary(),
        "gpu_launches": 2 * len(results) * args.steps,
        "widths": results,
    }
    print(json.dumps(line), flush=True)
    return 0


FP32_LANES_PER_SM = 128


def fft_flops_per_frame_iter(code):
    """Float operations executed in one FFT-SPA iteration: per check of degree
    d, two radix-2 transforms of q log2 q additions per edge, d (d - 1) q
    products and d q scalings; per variable of degree v, v (v - 1) q + v q
    products, v q additions for the normalization sum and v q normalizing
    multiplications.  These are the FFT-SPA rows of Table 1 of the paper
    without loop control, less two entries that execute no float operation
    here: the transforms' multiplications (factors of +-1, folded into each
    butterfly's add or subtract) and the additions listed beside the
    check-node products."""
    d = np.diff(code.row_ptr).astype(np.int64)
    v = np.bincount(code.col_idx, minlength=code.n).astype(np.int64)
    q, lq = code.q, code.p
    cnp = int((2 * d * q * lq + d * (d - 1) * q + d * q).sum())
    vnp = int((v * (v - 1) * q + 3 * v * q).sum())
    return cnp + vnp


def run_fftspa(args, ws, rank, local):
    """The GF(64) (2,4) N=576 step (196,608 frames at 1.5 / 2.0 / 2.5 dB, up to
    20 iterations, early stop) decoded with FFT-SPA from float32 channel
    probabilities resident in HBM (29 GB, larger than L2)."""
    if args.warmup < 3:
        raise SystemExit("--warmup must be >= 3")
    import __graft_entry__
    __graft_entry__.build()
    from paper_2508_03567_gb300 import binding, inputs as I
    w = I.WORKLOADS[WORKLOAD]
    code = I.workload_code(WORKLOAD)
    fpp = args.frames or w["frames"]
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    parts, cws = [], []
    for i, eb in enumerate(w["ebn0"]):
        seed = I.workload_seed(WORKLOAD, i) + 7919 * rank
        b = I.make_batch(code, eb, seed, fpp, device=dev, chunk=8192, prob=True)
        parts.append(b.prob)
        cws.append(b.codewords)
        del b
    prob = torch.cat(parts, 0).contiguous()
    del parts
    cw = torch.cat(cws, 0)
    frames = prob.shape[0]
    dec = binding.Decoder.from_code(code)
    stream = torch.cuda.Stream(device=dev)
    sym = torch.empty((frames, code.n), dtype=torch.uint8, device=dev)
    its = torch.empty((frames,), dtype=torch.int32, device=dev)
    ok = torch.empty((frames,), dtype=torch.uint8, device=dev)
    wsb = dec.fftspa_workspace(frames, dev)
    mi, es = w["max_iters"], w["early_stop"]

    def step():
        binding.nbldpc_fftspa_decode(dec.handle, prob, frames, mi, es, sym, its, ok, None, wsb, stream=stream)

    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            step()
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    launches0 = binding.nbldpc_kernel_launch_count()
    if ws > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        for a, b in ev:
            a.record(stream)
            step()
            b.record(stream)
        torch.cuda.synchronize()
    launches = binding.nbldpc_kernel_launch_count() - launches0
    total_s = sum(a.elapsed_time(b) for a, b in ev) / 1e3
    if ws > 1:
        t = torch.tensor([total_s], device=dev, dtype=torch.float64)
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        total_s = float(t.item())
    its_h = its.cpu().numpy().astype(np.int64)
    fer = float((sym.to(torch.int64) != cw).any(1).float().mean())
    flops_fi = fft_flops_per_frame_iter(code)
    kernel_s = total_s / args.steps
    achieved = flops_fi * int(its_h.sum()) / kernel_s / 1e9
    mhz, mhz_kind = sm_max_mhz()
    peak = SM_COUNT * FP32_LANES_PER_SM * mhz * 1e6 / 1e9
    info_bits = frames * code.k * code.p
    fbpf, _ = profiled_traffic("fftspa_decode_kernel_gf64_n576.md", "fftspa_kernels.cuh")

    # end to end through nbldpc_fftspa_decode_host: 65,536 frames taken evenly from the step (every third
    # frame, so the three Eb/N0 points mix), pinned host probabilities copied in and outputs copied back
    # in chunks of 16,384 frames on two streams, copies timed
    e2e = None
    if not args.no_e2e:
        sel = prob[::3][:65536]
        ef = sel.shape[0]
        hp = torch.empty(sel.shape, dtype=torch.float32, pin_memory=True)
        hp.copy_(sel)
        del sel
        hs = torch.empty((ef, code.n), dtype=torch.uint8, pin_memory=True)
        hi = torch.empty((ef,), dtype=torch.int32, pin_memory=True)
        ho = torch.empty((ef,), dtype=torch.uint8, pin_memory=True)
        chunk = 16384
        hws = torch.empty(binding.nbldpc_fftspa_decode_host_workspace_size(dec.handle, chunk), dtype=torch.uint8,
                          device=dev)

        def e2e_step():
            binding.nbldpc_fftspa_decode_host(dec.handle, hp, ef, mi, es, hs, hi, ho, chunk, hws, stream=stream)
            stream.synchronize()

        for _ in range(2):
            e2e_step()
        t0 = time.perf_counter()
        for _ in range(3):
            e2e_step()
        dt = (time.perf_counter() - t0) / 3
        e2e = {"value": ef * code.k * code.p / dt / 1e6, "unit": "Mbit/s", "h2d_bytes_per_step": int(hp.numel() * 4),
               "d2h_bytes_per_step": int(hs.numel() + 4 * hi.numel() + ho.numel()), "ms_per_step": 1e3 * dt,
               "frames": ef, "chunk_frames": chunk,
               "form": "nbldpc_fftspa_decode_host: every third frame of the step, pinned host memory, two streams"}
    cpu = None
    if rank == 0 and not args.no_cpu:
        import oracle
        threads = os.cpu_count() or 1
        sample = []
        for i, eb in enumerate(w["ebn0"]):
            sample.append(I.make_batch(code, eb, I.workload_seed(WORKLOAD, i), 32, prob=True).prob.numpy())
        sp = np.concatenate(sample, 0)
        t0 = time.perf_counter()
        oracle.fftspa_decode(code, sp, mi, es, threads=threads)
        dt = time.perf_counter() - t0
        cpu = {"value": sp.shape[0] * code.k * code.p / dt / 1e6, "unit": "Mbit/s", "cores": threads,
               "kind": "oracle", "sample": f"{sp.shape[0]} frames (32 per Eb/N0 point) of the same workload, "
                                           f"{dt:.1f} s wall, float64"}
    if rank != 0:
        return 0
    line = {
        "metric": "decoded info Mbit/s", "value": ws * args.steps * info_bits / total_s / 1e6, "unit": "Mbit/s",
        "n_gpus": ws, "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * kernel_s,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": f"{WORKLOAD} decoded with FFT-SPA (Alg. 1)", "frames_per_step": frames,
                   "input": "float32 channel probabilities [F, N, q]", "ebn0_db": list(w["ebn0"]),
                   "max_iters": mi, "early_stop": bool(es), "l2": "inputs larger than L2 (no flush)",
                   "parallelism": f"frames sharded over {ws} GPU(s)"},
        "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "GFLOP/s",
                     "frac": achieved / peak, "traffic": None if fbpf is None else fbpf * frames,
                     "peak_kind": f"derived: 152 SMs x 128 fp32 lanes x {mhz:.0f} MHz ({mhz_kind} max SM clock), "
                                  "one add or multiply per lane per clock"},
        "clocks": clk.summary(),
        "gpu_launches": int(launches),
        "e2e": e2e,
        "cpu_baseline": cpu,
        "decode_stats": {"mean_iters": float(its_h.mean()), "fer": fer, "not_ok": float(1 - ok.float().mean()),
                         "flops_per_frame_iter": flops_fi},
    }
    print(json.dumps(line), flush=True)
    return 0


def run_schedule(args, ws, rank, local):
    """The GF(64) (2,4) N=576 step with the minimal check-node schedule (3(d_c - 2) = 6
    convolutions per check) and with the paper's Table 1 count (3 d_c - 4 = 8): same frames,
    same outputs, time per step."""
    if args.warmup < 3:
        raise SystemExit("--warmup must be >= 3")
    import __graft_entry__
    __graft_entry__.build()
    from paper_2508_03567_gb300 import binding, inputs as I
    w = I.WORKLOADS[WORKLOAD]
    code = I.workload_code(WORKLOAD)
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    gamma = make_inputs(code, w, args.frames or w["frames"], dev, rank)
    frames = gamma.shape[0]
    stream = torch.cuda.Stream(device=dev)
    mhz, mhz_kind = sm_max_mhz()
    peak = SM_COUNT * PEAK_OPS_PER_CLK_SM * mhz * 1e6 / 1e9
    res, outs = {}, {}
    with ClockSampler(local) as clk:
        for sched, label in ((binding.NBLDPC_CNP_MINIMAL, "minimal_3(dc-2)"), (binding.NBLDPC_CNP_TABLE1, "table1_3dc-4")):
            dec = binding.Decoder.from_code(code)
            binding.nbldpc_code_set_cnp_schedule(dec.handle, sched)
            sym, its, ok = (torch.empty((frames, code.n), dtype=torch.uint8, device=dev),
                            torch.empty((frames,), dtype=torch.int32, device=dev),
                            torch.empty((frames,), dtype=torch.uint8, device=dev))
            wsb = dec.workspace(frames, dev)

            def step():
                binding.nbldpc_decode(dec.handle, gamma, frames, w["max_iters"], w["early_stop"], sym, its, ok, wsb,
                                      stream=stream)

            with torch.cuda.stream(stream):
                for _ in range(args.warmup):
                    step()
            torch.cuda.synchronize()
            ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
                  for _ in range(args.steps)]
            for a, b in ev:
                a.record(stream)
                step()
                b.record(stream)
            torch.cuda.synchronize()
            t = sum(a.elapsed_time(b) for a, b in ev) / 1e3
            its_h = its.cpu().numpy().astype(np.int64)
            convs = convolutions_per_frame_iter(code, table1=sched == binding.NBLDPC_CNP_TABLE1)
            pairs = int(its_h.sum()) * convs * code.q * code.q
            res[label] = {"value": args.steps * frames * code.k * code.p / t / 1e6, "unit": "Mbit/s",
                          "ms_per_step": 1e3 * t / args.steps, "convolutions_per_check": convs // code.m,
                          "executed_alu_frac": 2 * pairs / (t / args.steps) / 1e9 / peak}
            outs[label] = sym.clone()
    same = bool(torch.equal(*outs.values()))
    if rank != 0:
        return 0
    head = res["minimal_3(dc-2)"]
    line = {
        "metric": "decoded info Mbit/s", "value": ws * head["value"], "unit": "Mbit/s", "n_gpus": ws,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": head["ms_per_step"], "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "u8", "data": "synthetic",
        "config": {"workload": f"{WORKLOAD}: minimal check-node schedule (value) against Table 1's",
                   "frames_per_step": frames, "l2": "inputs larger than L2 (no flush)"},
        "roofline": {"bound": "alu", "achieved": head["executed_alu_frac"] * peak, "peak": peak, "unit": "Gop/s",
                     "frac": head["executed_alu_frac"], "traffic": None,
                     "peak_kind": f"derived: 152 SMs x 256 u16 min/max ops/clk x {mhz:.0f} MHz ({mhz_kind})"},
        "clocks": clk.summary(),
        "gpu_launches": 2 * args.steps,
        "schedules": res,
        "identical_outputs": same,
    }
    print(json.dumps(line), flush=True)
    return 0


def make_inputs_cw(code, w, frames_per_point, device, rank):
    """The headline step's reliabilities and transmitted codewords (rank-specific seeds)."""
    from paper_2508_03567_gb300 import inputs as I
    gam, cws = [], []
    for i, eb in enumerate(w["ebn0"]):
        seed = I.workload_seed(WORKLOAD, i) + 7919 * rank
        b = I.make_batch(code, eb, seed, frames_per_point, device=device, chunk=8192)
        gam.append(b.gamma)
        cws.append(b.codewords)
    return torch.cat(gam, 0).contiguous(), torch.cat(cws, 0)


def run_single(args, ws, rank, local, name, graph=False, cpu_frames=None, profile=None):
    """--workload gf4 / gf256: one min-max workload as its own line."""
    if args.warmup < 3:
        raise SystemExit("--warmup must be >= 3")
    import __graft_entry__
    __graft_entry__.build()
    from paper_2508_03567_gb300 import binding, inputs as I
    if rank != 0:
        return 0
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    peaks = alu_peaks(None if args.no_extras else measure_peak(binding, dev, local, 0.3, PROBE_FORMS), dev)
    r = measure_workload(binding, I, name, dev, local, args, peaks, args.steps, args.warmup,
                         frames=args.frames, graph=graph, cpu_frames=cpu_frames, profile=profile)
    line = {"metric": "decoded info Mbit/s", "value": r.pop("value"), "unit": "Mbit/s", "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": r.pop("ms_per_step"),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u8", "data": "synthetic",
            "config": dict(workload=name, **r.pop("config")), **r}
    print(json.dumps(line), flush=True)
    return 0


# workloads beside the headline: (name, CUDA-graph replay, CPU sample (all cores, one thread) per Eb/N0
# point, committed ncu summary)
SIDE_WORKLOADS = (("gf4_n48_dv2_dc4", True, (1000, 1000), "mma_decode_kernel_gf4_n48.md"),
                  ("gf256_n384_dv2_dc6", False, (16, 2), "mma_decode_kernel_gf256_n384.md"))


def main():
    args = parse()
    ws, rank, local = dist_setup(args)
    if args.impl == "reference":
        return run_reference(args, ws, rank)
    if args.workload == "mixed":
        return run_mixed(args, ws, rank, local)
    if args.workload == "serving":
        return run_serving(args, ws, rank, local)
    if args.workload == "width":
        return run_width(args, ws, rank, local)
    if args.workload == "fftspa":
        return run_fftspa(args, ws, rank, local)
    if args.workload == "schedule":
        return run_schedule(args, ws, rank, local)
    if args.workload == "peak":
        return run_peak(args, ws, rank, local)
    if args.workload in ("gf4", "gf256"):
        name, rep, cpuf, prof = SIDE_WORKLOADS[0 if args.workload == "gf4" else 1]
        return run_single(args, ws, rank, local, name, rep, cpuf, prof)
    if args.warmup < 3:
        raise SystemExit("--warmup must be >= 3")
    import __graft_entry__
    __graft_entry__.build()
    from paper_2508_03567_gb300 import binding, inputs as I
    w = I.WORKLOADS[WORKLOAD]
    code = I.workload_code(WORKLOAD)
    fpp = args.frames or w["frames"]
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    extras = ws == 1 and not args.no_extras
    # the integer min/max peak of this GPU, measured before the timed region (probe kernels)
    peak_meas = measure_peak(binding, dev, local, args.probe_seconds) if extras else None
    peaks = alu_peaks(peak_meas, dev)
    gamma, cw = make_inputs_cw(code, w, fpp, dev, rank)
    frames = gamma.shape[0]
    dec = binding.Decoder.from_code(code)
    tuning = {"source": "default"}
    if not args.no_autotune:
        # time every (layout variant, frames per block) pair on 4096 of the step's frames, fixed 3 iterations
        res = dec.autotune(gamma[: min(frames, 4096)], 3)
        tuning = {"source": "autotuned", "candidates_ms": {f"v{v}_fpb{f}": round(ms, 3) for v, f, ms in res}}
    v, fpb = dec.tuning()
    tuning.update({"variant": v, "frames_per_block": fpb})
    stream = torch.cuda.Stream(device=dev)
    sym = torch.empty((frames, code.n), dtype=torch.uint8, device=dev)
    its = torch.empty((frames,), dtype=torch.int32, device=dev)
    ok = torch.empty((frames,), dtype=torch.uint8, device=dev)
    wsb = dec.workspace(frames, dev)
    mi, es = w["max_iters"], w["early_stop"]

    def step():
        binding.nbldpc_decode(dec.handle, gamma, frames, mi, es, sym, its, ok, wsb, stream=stream)

    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            step()
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    launches0 = binding.nbldpc_kernel_launch_count()
    if ws > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        t0 = time.perf_counter()
        for a, b in ev:
            a.record(stream)
            step()
            b.record(stream)
        torch.cuda.synchronize()
        t1 = time.perf_counter()
    launches = binding.nbldpc_kernel_launch_count() - launches0
    step_ms = [a.elapsed_time(b) for a, b in ev]
    total_s = sum(step_ms) / 1e3
    if ws > 1:
        t = torch.tensor([total_s], device=dev, dtype=torch.float64)
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        total_s = float(t.item())
        torch.distributed.barrier()

    # decode statistics and algorithmic work of one step (identical every step)
    its_h = its.cpu().numpy().astype(np.int64)
    ok_h = ok.cpu().numpy()
    fer = float((sym.to(torch.int64) != cw).any(1).float().mean())
    pairs_step = int(its_h.sum()) * pairs_per_frame_iter(code)
    info_bits_step = frames * code.k * code.p
    value = ws * args.steps * info_bits_step / total_s / 1e6
    kernel_s = statistics.mean(step_ms) / 1e3
    median_ms = statistics.median(step_ms)
    with torch.cuda.stream(stream):
        visited_step = visited_pairs(binding, dec, [step], dev)
    achieved_gops = 2 * visited_step / kernel_s / 1e9         # executed 16-bit min/max ops per second
    clocks = clk.summary()
    peak_gops, peak_kind, issue_gops = peaks
    bpf, _ = profiled_traffic()

    e2e = None
    if not args.no_e2e:
        e2e = measure_e2e(binding, dec, code, gamma, mi, es, args, dev)
    cpu = None
    if rank == 0 and not args.no_cpu:
        cpu = cpu_baseline(WORKLOAD, 64, 4)
    del gamma, cw, sym
    torch.cuda.empty_cache()

    side, mixed, serving = None, None, None
    if extras and rank == 0:
        ks, kw = min(args.steps, 5), 3
        side = {}
        for name, rep, cpuf, prof in SIDE_WORKLOADS:
            side[name] = measure_workload(binding, I, name, dev, local, args, peaks, ks, kw, graph=rep,
                                          cpu_frames=cpuf, profile=prof)
            torch.cuda.empty_cache()
        # GF(4) N=48 at a batch large enough that launch cost does not dominate (kernel rate)
        big = measure_workload(binding, I, "gf4_n48_dv2_dc4", dev, local, args, peaks, ks, kw, frames=262144,
                               e2e=False)
        side["gf4_n48_dv2_dc4"]["kernel_rate_262144_frames"] = {
            k: big[k] for k in ("value", "unit", "ms_per_step", "roofline", "fer", "mean_iters", "clocks")}
        m = run_mixed(args, ws, rank, local, emit=False, steps=ks, warmup=kw, peaks=peaks)
        mixed = {"value": m["value"], "unit": "Mbit/s", "ms_per_step": m["ms_per_step"], "fer": m["fer"],
                 "roofline_frac": m["roofline"]["frac"], "form": m["config"]["form"],
                 "plain_fixed_iterations": m["plain_fixed_iterations"], "plain_early_stop": m["plain_early_stop"],
                 "frames": m["config"]["frames"], "clocks": m["clocks"]}
        torch.cuda.empty_cache()
        sv = run_serving(args, ws, rank, local, emit=False, loads_c=(0.10, 0.50), loads_p=(0.10,), seconds=3.0)
        serving = {"saturated_mbps": sv["peak_continuous"]["achieved_mbps"],
                   "plain_saturated_mbps": sv["peak_plain"]["achieved_mbps"],
                   "loads": [{k: r[k] for k in ("load", "offered_mbps", "achieved_mbps", "p50_ms", "p99_ms",
                                                  "requests", "completed")} for r in sv["loads_continuous"]],
                   "plain_loads": [{k: r[k] for k in ("load", "offered_mbps", "achieved_mbps", "p50_ms", "p99_ms",
                                                        "requests", "completed")} for r in sv["loads_plain"]],
                   "form": "native server, continuous batching, 3 s Poisson window per load point"}

    if rank != 0:
        return 0
    line = {
        "metric": "decoded info Mbit/s", "value": value, "unit": "Mbit/s", "n_gpus": ws,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total_s / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u8",
        "data": "synthetic",
        "config": {"workload": WORKLOAD, "frames_per_step": frames, "q": code.q, "n": code.n,
                   "k": code.k, "dv": w["dv"], "dc": w["dc"], "ebn0_db": list(w["ebn0"]),
                   "max_iters": mi, "early_stop": bool(es), "l2": "inputs larger than L2 (no flush)",
                   "parallelism": f"frames sharded over {ws} GPU(s)", "tuning": tuning},
        "roofline": roofline_alu(achieved_gops, peak_gops, peak_kind, issue_gops,
                                 None if bpf is None else bpf * frames,
                                 frames * algorithmic_bytes_per_frame(code) / kernel_s,
                                 dense=2 * pairs_step / kernel_s / 1e9),
        "clocks": clocks,
        "gpu_launches": int(launches),
        "e2e": e2e,
        "cpu_baseline": cpu,
        "fer": fer,
        "decode_stats": {"mean_iters": float(its_h.mean()), "not_ok": float(1 - ok_h.mean()),
                         "pairs_per_step": pairs_step, "visited_pairs_per_step": visited_step,
                         "kernel_ms": 1e3 * kernel_s,
                         "median_ms_per_step": median_ms,
                         "wall_ms_per_step": 1e3 * (t1 - t0) / args.steps},
        # the paper's throughput formula counts coded bits (N p per frame)
        "coded_mbps": value * code.n / code.k,
        "integer_peak_probe": peak_meas,
        "configs": side,
        "mixed": mixed,
        "serving": serving,
    }
    print(json.dumps(line), flush=True)
    return 0


def measure_e2e(binding, dec, code, gamma_dev, mi, es, args, dev):
    """Same workload through nbldpc_decode_host: pinned host inputs, copies timed."""
    frames = gamma_dev.shape[0]
    g_host = torch.empty(gamma_dev.shape, dtype=torch.uint8, pin_memory=True)
    g_host.copy_(gamma_dev)
    sym = torch.empty((frames, code.n), dtype=torch.uint8, pin_memory=True)
    its = torch.empty((frames,), dtype=torch.int32, pin_memory=True)
    ok = torch.empty((frames,), dtype=torch.uint8, pin_memory=True)
    chunk = 16384
    need = binding.nbldpc_decode_host_workspace_size(dec.handle, chunk)
    wsb = torch.empty(need, dtype=torch.uint8, device=dev)
    stream = torch.cuda.Stream(device=dev)

    def step():
        binding.nbldpc_decode_host(dec.handle, g_host, frames, mi, es, sym, its, ok, chunk, wsb,
                                   stream=stream)
        stream.synchronize()

    for _ in range(2):
        step()
    steps = max(1, min(args.steps, 3))
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(steps):
        step()
    dt = (time.perf_counter() - t0) / steps
    # the host-to-device copy of the step's reliabilities alone (the paper times transfers apart)
    dst = torch.empty(gamma_dev.shape, dtype=torch.uint8, device=dev)
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with torch.cuda.stream(stream):
        dst.copy_(g_host, non_blocking=True)
        a.record(stream)
        dst.copy_(g_host, non_blocking=True)
        b.record(stream)
    stream.synchronize()
    h2d_ms = a.elapsed_time(b)
    del dst
    bits = frames * code.k * code.p
    return {"value": bits / dt / 1e6, "unit": "Mbit/s", "h2d_bytes_per_step": int(g_host.numel()),
            "d2h_bytes_per_step": int(sym.numel() + 4 * its.numel() + ok.numel()),
            "ms_per_step": 1e3 * dt, "steps": steps, "chunk_frames": chunk,
            "h2d_only_ms_per_step": h2d_ms, "h2d_only_gbs": g_host.numel() / h2d_ms / 1e6}


if __name__ == "__main__":
    sys.exit(main())
