#!/usr/bin/env python3
"""Benchmark of the compressed 3-vector add (the paper's Sec. 5 test, C = A + B)
on GB300, through the library's C ABI.

One step = one fused launch c = compress(decompress(a) + decompress(b)) over
N = 2^28 packed <0,7,22>-17-18 words per GPU (magnitudes 10^U(-3,3), uniform
directions), inputs resident in HBM.  Printed: one JSON line (rank 0).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ivc|reference]

Under torchrun (N > 1) each rank processes its own N = 2^28 shard (weak
scaling, no data-path collective); the time is the maximum over ranks.
``--impl reference`` times the oracle (plain CPU reference) on the host cores
on bounded samples of the same workload.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "compressed 3-vector add: Gvec/s and % HBM peak vs FP32x3 at stated error"
UNIT = "Gvec/s"
BYTES_PER_VEC = 24          # read two 8-byte words, write one
FP32_BYTES_PER_VEC = 36     # read two 12-byte vectors, write one
FALLBACK_HBM_GBS = 6800.0
NOMINAL_HBM_GBS = 7900.0    # GB300 HBM3e, nominal (the measured copy peak is the roofline)


def parse_args():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=200)
    p.add_argument("--warmup", type=int, default=10)
    p.add_argument("--impl", choices=["ivc", "reference"], default="ivc")
    p.add_argument("--log2n", type=int, default=28)
    p.add_argument("--no-extra", action="store_true", help="skip the baseline/extra measurements")
    p.add_argument("--cpu-seconds", type=float, default=10.0)
    p.add_argument("--workload", choices=["add", "tgv", "batched", "precision", "fdiv", "sweep",
                                          "gather", "fr", "codec"],
                   default="add",
                   help="add: the headline line; the others print their own JSON line")
    p.add_argument("--tgv-elements", type=int, default=96)
    p.add_argument("--fdiv-elements", type=int, default=96,
                   help="elements per axis of the flux-divergence mesh")
    p.add_argument("--fr-elements", type=int, default=96,
                   help="elements per axis of the mesh of the FR steps 5-11")
    return p.parse_args()


def kernel_source_hash() -> str:
    """Hash of the sources that define the compressed add kernel and its launch
    (the committed DRAM-traffic figure is valid only for that exact code)."""
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2003_02633_gb300", "csrc")
    files = [os.path.join(csrc, f) for f in ("ivc_internal.h", "ivc_device.cuh", "ivc_exact.cuh",
                                              "ivc_fast.cuh", "ivc_ops.cu")]
    for f in files:
        with open(f, "rb") as fh:
            h.update(os.path.basename(f).encode())
            h.update(fh.read())
    return h.hexdigest()[:16]


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "MEASURED_PEAKS.json hbm_gbs (measured copy, burst)"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback 6.8 TB/s"


def tf32_roofline(issued_tflops: float) -> dict:
    """TF32 tensor-core products issued against the dense TF32 peak, derived
    from the measured bf16 peak and the nominal tf32 : bf16 ratio (1.1 : 2.25
    PFLOP/s)."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            bf16 = float(json.load(f)["bf16_tflops"])
        src = "MEASURED_PEAKS.json bf16_tflops (burst) x 1.1 / 2.25"
    except Exception:
        bf16, src = 1900.0, "fallback 1.9 PFLOP/s bf16 x 1.1 / 2.25"
    peak = bf16 * 1.1 / 2.25
    return {"issued_tf32_tflops": round(issued_tflops, 1), "peak_tf32_tflops": round(peak, 1),
            "frac": round(issued_tflops / peak, 4), "peak_source": src}


def issue_roofline(prof, gvec_s, clocks):
    """The bound the compressed add actually meets: warp instructions issued per
    second (instructions per vector from the committed ncu capture of the same
    kernel sources x vectors per second) against the SMs' issue rate (4
    schedulers per SM, one warp instruction per cycle each, at the sampled
    maximum SM clock)."""
    if not prof or "warp_inst_per_vector" not in prof:
        return None
    import torch
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    mhz = (clocks or {}).get("sm_max_mhz") or 2070.0
    peak = sms * 4 * mhz * 1e6 / 1e9
    achieved = gvec_s * prof["warp_inst_per_vector"]
    return {"bound": "issue", "achieved": round(achieved, 1), "peak": round(peak, 1),
            "unit": "G warp-instructions/s", "frac": round(achieved / peak, 4),
            "warp_inst_per_vector": prof["warp_inst_per_vector"],
            "source": "ncu smsp__inst_executed.sum of the same kernel sources (profiles/)"}


def ncu_profile_entry(kernel: str):
    """The committed ncu figures of a kernel, or None when its sources changed
    since they were captured."""
    p = os.path.join(ROOT, "profiles", "ncu_traffic.json")
    try:
        with open(p) as f:
            e = json.load(f)[kernel]
        return e if e.get("source_hash") == kernel_source_hash() else None
    except Exception:
        return None


def ncu_traffic(kernel: str, n: int):
    """DRAM bytes per launch from the committed ncu summary, or None when the
    kernel source changed since it was captured."""
    p = os.path.join(ROOT, "profiles", "ncu_traffic.json")
    try:
        with open(p) as f:
            d = json.load(f)
        e = d[kernel]
        if e.get("source_hash") != kernel_source_hash():
            return None
        return float(e["dram_bytes_per_vector"]) * n
    except Exception:
        return None


# ----------------------------------------------------------------- clocks

class ClockSampler:
    """nvidia-smi clock/throttle sampling while the timed region runs."""
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.QUERY}",
                 "--format=csv,noheader,nounits", "-lms", "20"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        time.sleep(0.3)

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        rows = []
        with open(self.path) as f:
            for line in f:
                p = [x.strip() for x in line.split(",")]
                if len(p) >= 9:
                    rows.append(p)
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"], "samples": 0}

        def num(x):
            try:
                return float(x)
            except ValueError:
                return None
        sm = [num(r[1]) for r in rows if num(r[1]) is not None]
        smax = [num(r[2]) for r in rows if num(r[2]) is not None]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        pw = [num(r[3]) for r in rows if num(r[3]) is not None]
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None, "reasons": reasons,
                "samples": len(rows), "power_w_max": max(pw) if pw else None}


# ------------------------------------------------------------ distributed

def dist_setup(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    pg = None
    if world > 1:
        import torch
        import torch.distributed as dist
        backend = "nccl" if torch.cuda.is_available() else "gloo"
        if torch.cuda.is_available():
            torch.cuda.set_device(local)
        dist.init_process_group(backend=backend)
        pg = dist
    return world, rank, local, pg


def barrier(pg):
    if pg is not None:
        pg.barrier()


def max_over_ranks(pg, value: float, device) -> float:
    if pg is None:
        return value
    import torch
    t = torch.tensor([value], dtype=torch.float64, device=device)
    pg.all_reduce(t, op=pg.ReduceOp.MAX)
    return float(t.item())


# ---------------------------------------------------------------- helpers

def time_launches(fn, steps, warmup, stream, sync_all=None):
    """Warm-up, then time exactly `steps` launches with CUDA events on
    `stream`.  Returns (total_ms, per_launch_ms list)."""
    import torch
    for _ in range(warmup):
        fn()
    torch.cuda.synchronize()
    if sync_all:
        sync_all()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(steps)]
    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    t0.record(stream)
    for i in range(steps):
        ev[i][0].record(stream)
        fn()
        ev[i][1].record(stream)
    t1.record(stream)
    torch.cuda.synchronize()
    if sync_all:
        sync_all()
    return t0.elapsed_time(t1), [a.elapsed_time(b) for a, b in ev]


def run_ivc(args):
    import numpy as np
    import torch

    from paper_2003_02633_gb300 import ivc, synth

    world, rank, local, pg = dist_setup(args)
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    ivc.load()
    n = 1 << args.log2n
    fmt = ivc.default_format()
    stream = torch.cuda.current_stream()
    s_handle = stream.cuda_stream

    # Inputs: FP32 AoS vectors drawn on the device, compressed once (untimed).
    a = synth.device_vectors(n, seed=2 * rank, device=dev)
    b = synth.device_vectors(n, seed=2 * rank + 1, device=dev)
    wa = ivc.compress(fmt, a)
    wb = ivc.compress(fmt, b)
    wc = torch.empty_like(wa)
    torch.cuda.synchronize()

    def step():
        ivc.add(fmt, wa, wb, out=wc, stream=s_handle)

    sampler = ClockSampler(local) if rank == 0 else None
    # warm-up outside the clock window
    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    barrier(pg)
    if sampler:
        sampler.start()
    total_ms, per = time_launches(step, args.steps, 0, stream, lambda: barrier(pg))
    clocks = sampler.stop() if sampler else None
    total_ms = max_over_ranks(pg, total_ms, dev)
    ms_step = total_ms / args.steps
    kernel_ms = statistics.mean(per)
    value = world * n / (ms_step * 1e-3) / 1e9
    hbm_peak, peak_src = measured_peaks()
    achieved = BYTES_PER_VEC * n / (kernel_ms * 1e-3) / 1e9
    traffic = ncu_traffic("ivc_add", n)
    prof = ncu_profile_entry("ivc_add")

    # End to end through the public API: pinned host words in, result out.
    h_a = torch.empty(n, dtype=torch.int64, pin_memory=True)
    h_b = torch.empty(n, dtype=torch.int64, pin_memory=True)
    h_c = torch.empty(n, dtype=torch.int64, pin_memory=True)
    h_a.copy_(wa)
    h_b.copy_(wb)
    # ivc_add_host: pinned host words are read and written by the kernel over
    # the host link; the workspace serves pageable memory only
    ws = torch.empty(3 * 3 * (1 << 24), dtype=torch.int64, device=dev)

    def e2e_step():
        ivc.add_host(fmt, h_a, h_b, h_c, ws, stream=s_handle)

    e2e_steps = max(3, min(args.steps, 20))
    e2e_ms, _ = time_launches(e2e_step, e2e_steps, 2, stream, lambda: barrier(pg))
    e2e_ms = max_over_ranks(pg, e2e_ms, dev) / e2e_steps
    e2e_value = world * n / (e2e_ms * 1e-3) / 1e9
    del ws
    same = bool(torch.equal(h_c, wc.cpu()))

    extra = {}
    if not args.no_extra:
        extra = run_extras(args, fmt, a, b, wa, wb, stream, s_handle, n, pg, dev, value)

    cpu = None
    if rank == 0:
        cpu = cpu_baseline(args, a, b, wc, fmt)

    if rank == 0:
        line = {
            "metric": METRIC, "value": round(value, 4), "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms_step, 5),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic (seeded torch.Generator on device; uniform directions, "
                    "magnitudes 10^U(-3,3))",
            "config": {"workload": f"compressed vector add c = a + b, N = 2^{args.log2n} "
                                   f"3-vectors per GPU, <0,7,22>-17-18 words (Sec. 5)",
                       "n_per_gpu": n, "format": "<0,7,22>-17-18, b7=80",
                       "l2": "inputs larger than L2 (16 B read per vector, "
                             f"{16 * n / 2**30:.1f} GiB per launch)",
                       "parallelism": f"dp{world} (independent shards)"},
            "roofline": {"bound": "hbm", "achieved": round(achieved, 1), "peak": hbm_peak,
                         "unit": "GB/s", "frac": round(achieved / hbm_peak, 4),
                         "traffic": traffic, "peak_source": peak_src,
                         "frac_of_nominal": round(achieved / NOMINAL_HBM_GBS, 4),
                         "algorithmic_bytes_per_launch": BYTES_PER_VEC * n,
                         "kernel_ms": round(kernel_ms, 5)},
            "issue_roofline": issue_roofline(prof, value, clocks),
            "e2e": {"value": round(e2e_value, 4), "unit": UNIT,
                    "h2d_bytes_per_step": 16 * n, "d2h_bytes_per_step": 8 * n,
                    "matches_device_result": same,
                    "path": "ivc_add_host on pinned host words: the kernel reads and "
                            "writes them over the host link (zero-copy)"},
            "gpu_launches": args.steps,
            "clocks": clocks,
            "cpu_baseline": cpu,
            "extra": extra,
        }
        print(json.dumps(line), flush=True)
    if pg is not None:
        pg.destroy_process_group()


def run_extras(args, fmt, a, b, wa, wb, stream, s_handle, n, pg, dev, value):
    """Baselines and the other fused operations at the same N (not the headline)."""
    import torch

    from paper_2003_02633_gb300 import ivc
    steps = max(5, min(args.steps, 50))
    out = {}

    def t(fn):
        ms, per = time_launches(fn, steps, 3, stream, lambda: barrier(pg))
        return max_over_ranks(pg, ms / steps, dev), statistics.mean(per)

    c32 = torch.empty_like(a)
    ms, _ = t(lambda: ivc.f32_add(a, b, out=c32, stream=s_handle))
    out["fp32_aos_add_gvec_s"] = round(n / (ms * 1e-3) / 1e9, 4)
    out["fp32_aos_add_gbs"] = round(FP32_BYTES_PER_VEC * n / (ms * 1e-3) / 1e9, 1)
    ms, _ = t(lambda: ivc.f32_add(a, b, out=c32, layout=ivc.IVC_SOA, ld=n, n=n, stream=s_handle))
    out["fp32_soa_add_gvec_s"] = round(n / (ms * 1e-3) / 1e9, 4)
    out["speedup_vs_fp32_aos"] = round(value / max(out["fp32_aos_add_gvec_s"], 1e-9), 4)
    out["speedup_vs_fp32_soa"] = round(value / max(out["fp32_soa_add_gvec_s"], 1e-9), 4)
    del c32
    y = wb.clone()
    ms, kms = t(lambda: ivc.axpy(fmt, 0.7, wa, y, stream=s_handle))
    out["axpy_gvec_s"] = round(n / (ms * 1e-3) / 1e9, 4)
    out["axpy_gbs"] = round(BYTES_PER_VEC * n / (kms * 1e-3) / 1e9, 1)
    del y
    y32 = b.clone()
    ms, _ = t(lambda: ivc.f32_axpy(0.7, a, y32, stream=s_handle))
    out["fp32_aos_axpy_gvec_s"] = round(n / (ms * 1e-3) / 1e9, 4)
    del y32
    for kind, name in ((ivc.IVC_F16, "fp16"), (ivc.IVC_BF16, "bf16")):
        ha = ivc.half_from_f32(kind, a)
        hb = ivc.half_from_f32(kind, b)
        hc = torch.empty_like(ha)
        ms, _ = t(lambda: ivc.half_add(kind, ha, hb, out=hc, stream=s_handle))
        out[f"{name}_aos_add_gvec_s"] = round(n / (ms * 1e-3) / 1e9, 4)
        del ha, hb, hc
    # decompress and compress alone (12 B <-> 8 B per vector)
    d = torch.empty_like(a)
    ms, _ = t(lambda: ivc.decompress(fmt, wa, out=d, stream=s_handle))
    out["decompress_gvec_s"] = round(n / (ms * 1e-3) / 1e9, 4)
    cw = torch.empty_like(wa)
    ms, _ = t(lambda: ivc.compress(fmt, a, out=cw, stream=s_handle))
    out["compress_gvec_s"] = round(n / (ms * 1e-3) / 1e9, 4)
    del d, cw
    # the paper's other layouts and variants, same vectors (Sec. 2.3-2.5)
    variants = {"L1717": dict(exp_bits=7, man_bits=23, phi_bits=17, theta_bits=17, exp_bias=80),
                "L1617": dict(exp_bits=8, man_bits=23, phi_bits=16, theta_bits=17,
                              exp_bias=127),
                "fracsplit": dict(map=2, nphi_max_p1=185363),
                "tanh": dict(map=1, gamma=0.5)}
    va, vb = torch.empty_like(wa), torch.empty_like(wb)
    for name, kw in variants.items():
        f = ivc.make_format(**kw)
        ivc.compress(f, a, out=va, stream=s_handle)
        ivc.compress(f, b, out=vb, stream=s_handle)
        vc = torch.empty_like(va)
        ms, _ = t(lambda: ivc.add(f, va, vb, out=vc, stream=s_handle))
        out[f"add_{name}_gvec_s"] = round(n / (ms * 1e-3) / 1e9, 4)
        del vc
    del va, vb
    torch.cuda.synchronize()
    if n >= (1 << 26):
        # the secondary workloads, short versions (each prints its own line with
        # --workload at full size)
        torch.cuda.empty_cache()
        bt = batched_measure(5)
        out["batched"] = {k: bt[k] for k in ("fields", "total_vectors", "tuned",
                                              "graph_tuned_gvec_s", "status_tuned",
                                              "separate_launches_gvec_s", "single_field_gvec_s",
                                              "batched_over_single_field",
                                              "graph_tuned_hbm_frac", "single_field_hbm_frac")}
        torch.cuda.empty_cache()
        tg = tgv_measure(48, 20, errors=False)
        out["tgv_48"] = {k: tg[k] for k in ("n_vectors", "steps", "gvec_s", "gbs_36B",
                                             "hbm_frac", "fp32_gvec_s")}
        torch.cuda.empty_cache()
        fd = fdiv_measure(48, 10, 3, 0, simt=False)
        out["fdiv_48"] = {k: fd[k] for k in ("elements", "ms", "gbs_algorithmic", "hbm_frac",
                                              "fp32_ms", "speedup_vs_fp32")}
        out["fdiv_48"]["tensor_frac"] = fd["tensor"]["frac"]
        torch.cuda.empty_cache()
        fr = fr_measure(48, 10, 3, only=(7,))
        out["fr_step7_48"] = fr["per_step"][0]
        out["fr_step7_48"]["elements"] = fr["elements"]
        torch.cuda.empty_cache()
    return out


def _oracle_worker(job):
    """One host process of the CPU baseline: compresses its slices with the
    oracle (untimed), times the oracle's add over them, and compares the words
    with the GPU's.  job = (sample directory, first slice, slice count, slice)."""
    import numpy as np

    from oracle import oracle as O
    d, first, count, chunk = job
    A = np.load(os.path.join(d, "a.npy"), mmap_mode="r")
    B = np.load(os.path.join(d, "b.npy"), mmap_mode="r")
    W = np.load(os.path.join(d, "w.npy"), mmap_mode="r")
    secs, done, mism = 0.0, 0, 0
    for i in range(first, first + count):
        sl = slice(i * chunk, (i + 1) * chunk)
        wa, wb = O.compress(O.PRIMARY, np.array(A[sl])), O.compress(O.PRIMARY, np.array(B[sl]))
        t0 = time.perf_counter()
        c = O.add(O.PRIMARY, wa, wb)
        secs += time.perf_counter() - t0
        mism += int(np.sum(np.array(W[sl]) != c))
        done += chunk
    return done, secs, mism


def cpu_baseline(args, a, b, wc, fmt):
    """The oracle's add on a bounded sample of the same workload, on the host
    cores (one process per core, started with spawn after the GPU work; the
    sample goes to them through a temporary directory), plus agreement of its
    words with the GPU's."""
    import multiprocessing as mp

    import numpy as np
    import torch
    if args.cpu_seconds <= 0:
        return None
    n = a.shape[0]
    cores = max(1, min(16, os.cpu_count() or 1))
    rng = np.random.default_rng(123)
    chunk = 1 << 14
    # about cpu_seconds of timed add in total (one core adds ~1.6e6 vectors/s)
    per_proc = max(1, int(args.cpu_seconds * 1.6e6 / chunk / cores))
    nsl = min(cores * per_proc, max(1, n // chunk))
    per_proc = max(1, nsl // cores)
    nsl = per_proc * cores
    starts = rng.integers(0, max(1, n - chunk), nsl)
    idx = torch.from_numpy((starts[:, None] + np.arange(chunk)[None, :]).reshape(-1)).to(a.device)
    with tempfile.TemporaryDirectory() as d:
        np.save(os.path.join(d, "a.npy"), a[idx].cpu().numpy())
        np.save(os.path.join(d, "b.npy"), b[idx].cpu().numpy())
        np.save(os.path.join(d, "w.npy"), wc[idx].cpu().numpy().view(np.uint64))
        del idx
        jobs = [(d, k * per_proc, per_proc, chunk) for k in range(cores)]
        with mp.get_context("spawn").Pool(cores) as pool:
            res = pool.map(_oracle_worker, jobs)
    done = sum(r[0] for r in res)
    secs = max(r[1] for r in res)
    mism = sum(r[2] for r in res)
    return {"value": round(done / secs / 1e9, 8), "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"{done} vectors ({nsl} random contiguous slices of {chunk}) of the same "
                      f"N = 2^{args.log2n} workload over {cores} processes, the oracle's add "
                      f"timed in each; value = vectors / slowest process's add time",
            "seconds": round(secs, 2), "sample_word_mismatches_vs_gpu": mism}


# -------------------------------------------------------------- reference

_REF = {}


def _ref_init(counter, m):
    """Worker of the reference arm: its own seeded sample of m vectors per
    operand, compressed once by the oracle."""
    from oracle import oracle as O
    from paper_2003_02633_gb300 import synth
    with counter.get_lock():
        k = counter.value
        counter.value += 1
    av = synth.bandwidth_vectors(m, seed=2 * k)
    bv = synth.bandwidth_vectors(m, seed=2 * k + 1)
    _REF["w"] = (O.compress(O.PRIMARY, av), O.compress(O.PRIMARY, bv))


def _ref_step(_):
    from oracle import oracle as O
    wa, wb = _REF["w"]
    O.add(O.PRIMARY, wa, wb)
    return wa.shape[0]


def run_reference(args):
    """The reference arm: the oracle's add (Sec. 5 workload, bounded samples) on
    the host cores, one spawned process per core, each step one add over
    every process's sample; wall-clock time per step."""
    import multiprocessing as mp

    from oracle import oracle as O
    from paper_2003_02633_gb300 import synth
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    O.build()
    cores = max(1, min(16, os.cpu_count() or 1))
    # size each process's sample so the whole run takes about a minute
    probe_a = synth.bandwidth_vectors(4096, seed=0)
    probe_b = synth.bandwidth_vectors(4096, seed=1)
    pa, pb = O.compress(O.PRIMARY, probe_a), O.compress(O.PRIMARY, probe_b)
    t0 = time.perf_counter()
    O.add(O.PRIMARY, pa, pb)
    rate = 4096 / (time.perf_counter() - t0)
    per_step_s = min(2.0, max(0.01, 60.0 / max(1, args.steps + args.warmup)))
    m = int(max(1024, min(1 << 22, rate * per_step_s)))
    ctx = mp.get_context("spawn")
    counter = ctx.Value("i", 0)
    times = []
    with ctx.Pool(cores, initializer=_ref_init, initargs=(counter, m)) as pool:
        for _ in range(args.warmup):
            pool.map(_ref_step, range(cores), chunksize=1)
        done = 0
        for _ in range(args.steps):
            t0 = time.perf_counter()
            done = sum(pool.map(_ref_step, range(cores), chunksize=1))
            times.append(time.perf_counter() - t0)
    sec = sum(times) / len(times)
    value = done / sec / 1e9
    line = {"impl": "reference", "metric": METRIC, "value": round(value, 8), "unit": UNIT,
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": round(sec * 1e3, 4), "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64 (binary128 near boundaries)",
            "data": "synthetic (seeded numpy PCG64; uniform directions, magnitudes 10^U(-3,3))",
            "config": {"workload": f"compressed vector add c = a + b, bounded samples of the "
                                   f"N = 2^{args.log2n} workload", "sample_per_step": done,
                       "format": "<0,7,22>-17-18, b7=80"},
            "cpu_baseline": {"value": round(value, 8), "unit": UNIT, "cores": cores,
                             "kind": "oracle",
                             "sample": f"{m} vectors per process and step, {cores} processes"},
            "e2e": {"value": round(value, 8), "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ------------------------------------------------------- other workloads

def _gvec(n, ms):
    return round(n / (ms * 1e-3) / 1e9, 4)


def _time_ms(fn, steps, warmup, stream):
    ms, per = time_launches(fn, steps, warmup, stream)
    return ms / steps, per


def run_tgv(args):
    """Pointwise update of a TGV velocity field (Sec. 4.2 initial condition) at
    the 4^3 solution points of each hex of an E^3 mesh: v <- v + dt f with the
    pressure-gradient forcing, decompress -> update -> recompress, 100 steps;
    error against the FP64 trajectory, next to the same update on FP32x3."""
    print(json.dumps(tgv_measure(args.tgv_elements, 100)), flush=True)


def tgv_measure(E, nsteps, errors=True):
    import torch

    from paper_2003_02633_gb300 import ivc, synth
    dev = torch.device("cuda", 0)
    fmt = ivc.default_format()
    v, f, rho = synth.tgv_fields_device(E, dev)
    n = v.shape[0]
    dt = 1e-3
    wv, wf = ivc.compress(fmt, v), ivc.compress(fmt, f)
    wm = torch.empty_like(wv)
    stream = torch.cuda.current_stream()
    s = stream.cuda_stream
    # FP64 trajectory of the same FP32 inputs
    exact = v.double() + nsteps * dt * f.double()
    torch.cuda.synchronize()
    ms, per = time_launches(lambda: ivc.pointwise_update(fmt, dt, wv, wf, rho=rho, v_out=wv,
                                                          m_out=wm, stream=s),
                            nsteps, 0, stream)
    vc = ivc.decompress(fmt, wv)
    v32 = v.clone()
    ms32, _ = time_launches(lambda: ivc.f32_axpy(dt, f, v32, stream=s), nsteps, 0, stream)
    ex32 = exact.float()

    def err(xh):
        acc = ivc.error_stats(ex32, xh)
        d = ivc.stats_dict(acc.cpu())
        diff = (xh.double() - exact).norm(dim=1)
        d["max_abs_vs_fp64"] = float(diff.max())
        d["mean_abs_vs_fp64"] = float(diff.mean())
        return d
    hbm, _ = measured_peaks()
    line = {"workload": "tgv_pointwise_update", "elements": E ** 3, "n_vectors": n,
            "steps": nsteps, "dt": dt, "ms_per_step": round(ms / nsteps, 5),
            "gvec_s": _gvec(n, ms / nsteps),
            "gbs_36B": round(36 * n / (ms / nsteps * 1e-3) / 1e9, 1),
            "hbm_frac": round(36 * n / (ms / nsteps * 1e-3) / 1e9 / hbm, 4),
            "fp32_ms_per_step": round(ms32 / nsteps, 5), "fp32_gvec_s": _gvec(n, ms32 / nsteps),
            "note": "velocity w = 0 makes every initial vector a phi tie (z = 0); 36 B per "
                    "vector: v, f words and rho in, v and m words out"}
    if errors:
        line["error_compressed_vs_fp64"] = err(vc)
        line["error_fp32_vs_fp64"] = err(v32)
    return line


def run_batched(args):
    """256 fields of uneven length (log-uniform 2^10..2^24), each with its own
    magnitude window: one persistent launch from a CUDA graph, against 256
    separate launches and one launch over a single field of the total size."""
    print(json.dumps(batched_measure(max(5, min(args.steps, 50)), sweep=True)), flush=True)


def batched_measure(steps, sweep=False):
    """The batched workload; the plan's launch shape is the autotuner's
    (ivc_tune_batched), plus, with sweep, fixed tiles for comparison."""
    import torch

    from paper_2003_02633_gb300 import ivc, synth
    dev = torch.device("cuda", 0)
    fmt = ivc.default_format()
    lens, win = synth.batched_fields(256, seed=0)
    fields = []
    for i, m in enumerate(lens):
        m = int(m)
        a = synth.device_vectors(m, 1000 + 2 * i, dev, lo=float(win[i, 0]), hi=float(win[i, 1]))
        b = synth.device_vectors(m, 1001 + 2 * i, dev, lo=float(win[i, 0]), hi=float(win[i, 1]))
        fields.append((ivc.compress(fmt, a), ivc.compress(fmt, b),
                       torch.empty(m, dtype=torch.int64, device=dev), 0.0))
        del a, b
    total = int(sum(int(m) for m in lens))
    stream = torch.cuda.current_stream()
    s = stream.cuda_stream
    out = {"workload": "batched_add", "fields": len(fields), "total_vectors": total}
    best = ivc.tune_batched(fmt, ivc.IVC_OP_ADD, fields, stream=s)
    out["tuned"] = {"block": best.block, "vec_per_thread": best.vec_per_thread,
                    "tile": best.tile, "blocks_per_sm": best.blocks_per_sm}
    plan = ivc.BatchedPlan(fmt, ivc.IVC_OP_ADD, fields, cfg=best, stream=s)
    ms, _ = _time_ms(lambda: plan.launch(stream=s), steps, 3, stream)
    out["graph_tuned_gvec_s"] = _gvec(total, ms)
    out["status_tuned"] = plan.status(stream=s)
    plan.close()
    if sweep:
        for tile in (4096, 16384, 65536):
            cfg = ivc.ivc_launch_config(256, 2, tile, 0)
            plan = ivc.BatchedPlan(fmt, ivc.IVC_OP_ADD, fields, cfg=cfg, stream=s)
            ms, _ = _time_ms(lambda: plan.launch(stream=s), steps, 3, stream)
            out[f"graph_tile{tile}_gvec_s"] = _gvec(total, ms)
            ms, _ = _time_ms(lambda: plan.launch(stream=s, graph=False), steps, 3, stream)
            out[f"direct_tile{tile}_gvec_s"] = _gvec(total, ms)
            out[f"status_tile{tile}"] = plan.status(stream=s)
            plan.close()

    def separate():
        for fa, fb, fc, _ in fields:
            ivc.add(fmt, fa, fb, out=fc, stream=s)
    ms, _ = _time_ms(separate, steps, 2, stream)
    out["separate_launches_gvec_s"] = _gvec(total, ms)
    big_a = torch.cat([f[0] for f in fields])
    big_b = torch.cat([f[1] for f in fields])
    big_c = torch.empty_like(big_a)
    ms, _ = _time_ms(lambda: ivc.add(fmt, big_a, big_b, out=big_c, stream=s), steps, 3, stream)
    out["single_field_gvec_s"] = _gvec(total, ms)
    out["batched_over_single_field"] = round(out["graph_tuned_gvec_s"] /
                                             out["single_field_gvec_s"], 4)
    hbm, _ = measured_peaks()
    out["graph_tuned_hbm_frac"] = round(out["graph_tuned_gvec_s"] * BYTES_PER_VEC / hbm, 4)
    out["single_field_hbm_frac"] = round(out["single_field_gvec_s"] * BYTES_PER_VEC / hbm, 4)
    del big_a, big_b, big_c, fields
    return out


def run_precision(args):
    """Precision sweep: 2^26 vectors with magnitudes 10^U(-30,30), 10 % near the
    poles, stored as FP32x3, compressed (plain, tanh, fractional split), FP16x3
    and BF16x3; errors against the FP32 inputs in FP64, range events, and the
    add throughput of each storage."""
    import numpy as np
    import torch

    from paper_2003_02633_gb300 import ivc, synth
    dev = torch.device("cuda", 0)
    n = 1 << min(args.log2n, 26)
    x = torch.from_numpy(synth.precision_vectors(n, seed=0)).to(dev)
    y = torch.from_numpy(synth.precision_vectors(n, seed=1)).to(dev)
    stream = torch.cuda.current_stream()
    s = stream.cuda_stream
    steps = max(5, min(args.steps, 20))
    out = {"workload": "precision_sweep", "n_vectors": n}

    def stats(xh):
        return ivc.stats_dict(ivc.error_stats(x, xh).cpu())
    out["fp32x3"] = stats(x)
    for name, kw in (("compressed_plain", {}), ("compressed_tanh", dict(map=1, gamma=0.5)),
                     ("compressed_fracsplit", dict(map=2, nphi_max_p1=185363))):
        fmt = ivc.make_format(**kw)
        counts = torch.zeros(3, dtype=torch.int64, device=dev)
        w = ivc.compress(fmt, x, counts=counts)
        d = stats(ivc.decompress(fmt, w))
        c = counts.cpu().tolist()
        d.update(n_overflow=c[0], n_underflow=c[1], n_nonfinite=c[2])
        wy = ivc.compress(fmt, y)
        wc = torch.empty_like(w)
        ms, _ = _time_ms(lambda: ivc.add(fmt, w, wy, out=wc, stream=s), steps, 2, stream)
        d["add_gvec_s"] = _gvec(n, ms)
        out[name] = d
    for kind, name in ((ivc.IVC_F16, "fp16x3"), (ivc.IVC_BF16, "bf16x3")):
        h = ivc.half_from_f32(kind, x)
        back = ivc.half_to_f32(kind, h)
        d = stats(back)
        fin = torch.isfinite(x).all(dim=1)
        d["n_overflow"] = int((~torch.isfinite(back).all(dim=1) & fin).sum())
        d["n_underflow"] = int(((back == 0).all(dim=1) & (x != 0).any(dim=1)).sum())
        hy = ivc.half_from_f32(kind, y)
        hc = torch.empty_like(h)
        ms, _ = _time_ms(lambda: ivc.half_add(kind, h, hy, out=hc, stream=s), steps, 2, stream)
        d["add_gvec_s"] = _gvec(n, ms)
        out[name] = d
    c32 = torch.empty_like(x)
    ms, _ = _time_ms(lambda: ivc.f32_add(x, y, out=c32, stream=s), steps, 2, stream)
    out["fp32x3"]["add_gvec_s"] = _gvec(n, ms)
    print(json.dumps(out), flush=True)


def run_fdiv(args):
    """Algorithm 1 (Sec. 4; Table fr_nse, step 10): divergence of the compressed
    Euler flux of the TGV initial state on an E^3 hex mesh of degree 3 (64
    solution points, 5 flux rows per point), against the same operator on the
    uncompressed FP32 flux; FP32 arithmetic in both."""
    print(json.dumps(fdiv_measure(args.fdiv_elements, args.steps, args.warmup,
                                  args.cpu_seconds)), flush=True)


def fdiv_measure(E, steps_arg, warmup_arg, cpu_seconds, simt=True):
    import numpy as np
    import torch

    from paper_2003_02633_gb300 import ivc, synth
    dev = torch.device("cuda", 0)
    fmt = ivc.default_format()
    order, nv = 3, 5
    ns = (order + 1) ** 3
    F = synth.tgv_euler_flux(E, order, device=dev)               # (ns, nv, ne, 3)
    ne = F.shape[2]
    W = ivc.compress(fmt, F.reshape(-1, 3)).reshape(ns, nv, ne)
    Fc = F.permute(3, 0, 1, 2).contiguous()                        # (3, ns, nv, ne)
    del F
    D = torch.from_numpy(synth.fr_hex_operator(order, 2 * math.pi / E)).to(dev)
    out = torch.empty((ns, nv, ne), dtype=torch.float32, device=dev)
    out32 = torch.empty_like(out)
    stream = torch.cuda.current_stream()
    s = stream.cuda_stream
    steps, warmup = max(3, min(steps_arg, 50)), max(3, min(warmup_arg, 10))
    ms, per = time_launches(lambda: ivc.flux_divergence(fmt, W, D, out=out, stream=s), steps,
                            warmup, stream)
    ms32, per32 = time_launches(lambda: ivc.f32_flux_divergence(Fc, D, out=out32, stream=s),
                                steps, warmup, stream)
    # the same two on the CUDA cores (FP32 FMAs)
    out_s = torch.empty_like(out)
    ms_s = ms32_s = float("nan")
    if simt:
        ms_s, _ = time_launches(lambda: ivc.flux_divergence(fmt, W, D, out=out_s, stream=s,
                                                            simt=True), steps, warmup, stream)
        ms32_s, _ = time_launches(lambda: ivc.f32_flux_divergence(Fc, D, out=out_s, stream=s,
                                                                  simt=True), steps, warmup,
                                  stream)
    ivc.flux_divergence_check()
    t, t32 = ms / steps, ms32 / steps
    flop = 2.0 * 3 * ns * ns * nv                                   # per element
    bytes_c = ns * nv * 8 + ns * nv * 4
    bytes_32 = ns * nv * 12 + ns * nv * 4
    hbm_gbs, _ = measured_peaks()
    # FP32 FMA peak: 152 SMs x 128 lanes x 2 FLOP x 2.07 GHz (sm count from the device)
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    fp32_peak = sms * 128 * 2 * 2.07e9 / 1e12
    d = (out.double() - out32.double()).abs()
    scale = out32.double().abs().max()
    line = {"workload": "flux_divergence_alg1", "elements": ne, "ns": ns, "nvars": nv,
            "steps": steps, "ms": round(t, 4), "elements_per_s": round(ne / (t * 1e-3), 1),
            "gbs_algorithmic": round(bytes_c * ne / (t * 1e-3) / 1e9, 1),
            "hbm_frac": round(bytes_c * ne / (t * 1e-3) / 1e9 / hbm_gbs, 4),
            "tflops": round(flop * ne / (t * 1e-3) / 1e12, 2),
            "fp32_alu_peak_tflops": round(fp32_peak, 1),
            "alu_frac": round(flop * ne / (t * 1e-3) / 1e12 / fp32_peak, 4),
            "fp32_ms": round(t32, 4), "fp32_gbs_algorithmic": round(bytes_32 * ne / (t32 * 1e-3) / 1e9, 1),
            "fp32_tflops": round(flop * ne / (t32 * 1e-3) / 1e12, 2),
            "speedup_vs_fp32": round(t32 / t, 4),
            "engine": "tensor cores (tcgen05 kind::tf32, 3 products per FP32 term)",
            "tensor": tf32_roofline(3 * flop * ne / (t * 1e-3) / 1e12),
            "simt_ms": round(ms_s / steps, 4), "simt_fp32_ms": round(ms32_s / steps, 4),
            "tc_speedup_vs_simt": round(ms_s / ms, 4),
            "tc_fp32_speedup_vs_simt": round(ms32_s / ms32, 4),
            "max_abs_diff_vs_fp32_input": float(d.max()), "max_abs_fp32_result": float(scale),
            "bytes_per_element": {"compressed": bytes_c, "fp32": bytes_32},
            "data": "synthetic TGV initial state (Sec. 4.2), Euler flux rows, degree-3 hexes"}
    if not simt:
        for k in ("simt_ms", "simt_fp32_ms", "tc_speedup_vs_simt", "tc_fp32_speedup_vs_simt"):
            line.pop(k)
    if cpu_seconds > 0:
        from oracle import oracle as O
        rng = np.random.default_rng(0)
        sel = np.sort(rng.choice(ne, size=min(ne, 256), replace=False))
        Wh = W[:, :, torch.from_numpy(sel).to(dev)].cpu().numpy().view(np.uint64)
        t0 = time.perf_counter()
        ref = O.flux_divergence(O.PRIMARY, Wh, D.cpu().numpy(), ns, nv)
        dt = time.perf_counter() - t0
        got = out[:, :, torch.from_numpy(sel).to(dev)].cpu().numpy().astype(np.float64)
        line["cpu_baseline"] = {"value": round(sel.size / dt, 1), "unit": "elements/s",
                                "cores": 1, "kind": "oracle",
                                "sample": f"{sel.size} random elements of the same mesh",
                                "max_abs_diff_vs_gpu": float(np.abs(got - ref).max())}
    del W, Fc, out, out32, out_s
    return line


def run_fr(args):
    """Steps 5-11 of Table fr_nse (Sec. 4) of the flux-reconstruction
    Navier-Stokes right-hand side on a periodic E^3 hex mesh of degree 3, with
    the gradient, metric, normal and flux tensors as compressed rows and, as
    the baseline, as FP32 rows: the chain 5 -> 6 -> 7 -> 8, 9 -> 10 -> 11, each
    step timed on its own.  The bytes each step moves per element come from
    the memory model of Table mem_usage (fr_memory); its prediction is the
    byte ratio, the measurement the time ratio."""
    print(json.dumps(fr_measure(args.fr_elements, args.steps, args.warmup)), flush=True)


def fr_measure(E, steps_arg, warmup_arg, only=None):
    """The FR steps; with `only`, just those steps are timed (the chain still
    runs once in full so that every step has its inputs)."""
    import torch

    from paper_2003_02633_gb300 import fr_memory, ivc, synth
    dev = torch.device("cuda", 0)
    fmt = ivc.default_format()
    order = 3
    dims = (E, E, E)
    ne = E ** 3
    c = synth.fr_case(dims, order, device=dev)
    basis = ivc.fr_basis(synth.fr_basis(order))
    gas = ivc.fr_gas()
    ns, nf = (order + 1) ** 3, 6 * (order + 1) ** 2

    def rows32(t):
        return t.permute(3, 0, 1, 2).contiguous()

    def words(t):
        return ivc.compress(fmt, t.reshape(-1, 3)).reshape(t.shape[:3])

    geo = {}
    for k in ("S_s", "S_f", "n_f"):
        geo[k + "32"], geo[k + "w"] = rows32(c[k]), words(c[k])
        del c[k]
    w_s, q_s, det_s = c["w_s"], c["q_s"], c["detJ_s"]
    dw_f, q_f, det_f, nFi = c["dw_f"], c["q_f"], c["detJ_f"], c["nFinv_f"]
    D = torch.from_numpy(synth.fr_hex_operator(order, 2.0)).to(dev)   # reference element
    f32 = dict(grad=torch.empty((3, ns, 5, ne), device=dev), gradc=torch.empty((3, ns, 5, ne),
               device=dev), gradf=torch.empty((3, nf, 5, ne), device=dev),
               F=torch.empty((3, ns, 5, ne), device=dev))
    cw = {k: torch.empty((ns if k != "gradf" else nf, 5, ne), dtype=torch.int64, device=dev)
          for k in ("grad", "gradc", "gradf", "F")}
    out = {k: (torch.empty((nf, 5, ne), device=dev), torch.empty((nf, 5, ne), device=dev))
           for k in ("nF", "Fc")}
    out["div"] = (torch.empty((ns, 5, ne), device=dev), torch.empty((ns, 5, ne), device=dev))
    stream = torch.cuda.current_stream()
    s = stream.cuda_stream

    def chain(f, R, G, k):          # k: 0 FP32, 1 compressed
        g = "32" if k == 0 else "w"
        return {
            5: lambda: ivc.fr_gradient(f, basis, w_s, out=R["grad"], stream=s),
            6: lambda: ivc.fr_correct_gradient(f, basis, R["grad"], dw_f, out=R["gradc"],
                                               stream=s),
            7: lambda: ivc.fr_interp_rows(f, basis, R["gradc"], out=R["gradf"], stream=s),
            8: lambda: ivc.fr_common_viscous_flux(f, order, gas, dims, R["gradf"], G["n_f" + g],
                                                  G["S_f" + g], det_f, q_f, nFi,
                                                  out=out["nF"][k], stream=s),
            9: lambda: ivc.fr_flux(f, order, gas, q_s, R["gradc"], G["S_s" + g], det_s,
                                   out=R["F"], stream=s),
            10: (lambda: ivc.f32_flux_divergence(R["F"], D, out=out["div"][k], stream=s))
            if f is None else
            (lambda: ivc.flux_divergence(f, R["F"], D, out=out["div"][k], stream=s)),
            11: lambda: ivc.fr_flux_correction(f, basis, R["F"], out["nF"][k], out=out["Fc"][k],
                                               stream=s),
        }

    runs = (chain(None, f32, geo, 0), chain(fmt, cw, geo, 1))
    order_steps = (5, 6, 7, 8, 9, 10, 11)
    for r in runs:
        for st in order_steps:
            r[st]()
    torch.cuda.synchronize()
    ivc.flux_divergence_check()
    steps, warmup = max(3, min(steps_arg, 20)), max(3, min(warmup_arg, 5))
    hbm_gbs, _ = measured_peaks()
    rows = []
    tot = [0.0, 0.0]
    byt = [0, 0]
    for st in (only or order_steps):
        ms = [_time_ms(r[st], steps, warmup, stream)[0] for r in runs]
        b32 = fr_memory.step_bytes(order, st)
        bc = fr_memory.step_bytes(order, st, compressed=True)
        for i in range(2):
            tot[i] += ms[i]
        byt[0] += b32
        byt[1] += bc
        rows.append({"step": st, "fp32_ms": round(ms[0], 4), "compressed_ms": round(ms[1], 4),
                     "time_ratio": round(ms[1] / ms[0], 4), "gamma_bytes": round(bc / b32, 4),
                     "fp32_gbs": round(b32 * ne / (ms[0] * 1e-3) / 1e9, 1),
                     "compressed_gbs": round(bc * ne / (ms[1] * 1e-3) / 1e9, 1),
                     "compressed_hbm_frac": round(bc * ne / (ms[1] * 1e-3) / 1e9 / hbm_gbs, 4)})
    ivc.flux_divergence_check()
    t_all, g_all = fr_memory.totals(order)
    line = {"workload": "fr_steps_5_11", "elements": ne, "order": order, "nvars": 5,
            "steps": steps, "per_step": rows,
            "steps_5_11": {"fp32_ms": round(tot[0], 4), "compressed_ms": round(tot[1], 4),
                           "time_ratio": round(tot[1] / tot[0], 4),
                           "predicted_ratio_bytes": round(byt[1] / byt[0], 4)},
            "table_mem_usage_k3": {"total_kib": round(t_all, 2), "gamma": round(g_all, 4),
                                   "predicted_gain": round(1 - g_all, 4)},
            "hbm_peak_gbs": hbm_gbs,
            "data": "synthetic: Taylor-Green state (Sec. 4.2) with a 5% smooth perturbation "
                    "on a periodic hex mesh deformed by 0.1 sin-products, degree 3"}
    return line


def run_sweep(args):
    """The paper's size sweep of Sec. 5 (Fig. speedup): compressed add against
    the FP32x3 add (AoS) for N = 2^10 ... 2^28 on one GPU.  The L2 is flushed
    (a 512 MB write) before every timed launch, so every size reads its inputs
    from HBM; the smallest sizes measure launch latency."""
    import torch

    from paper_2003_02633_gb300 import ivc, synth
    dev = torch.device("cuda", 0)
    fmt = ivc.default_format()
    stream = torch.cuda.current_stream()
    s = stream.cuda_stream
    nmax = 1 << 28
    a = synth.device_vectors(nmax, 21, dev)
    b = synth.device_vectors(nmax, 22, dev)
    wa, wb = ivc.compress(fmt, a), ivc.compress(fmt, b)
    wc, c32 = torch.empty_like(wa), torch.empty_like(a)
    flush = torch.empty(1 << 27, dtype=torch.float32, device=dev)
    rows = []
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)

    def timed(fn, reps):
        ts = []
        for _ in range(reps):
            flush.fill_(1.0)
            e0.record(stream)
            fn()
            e1.record(stream)
            e1.synchronize()
            ts.append(e0.elapsed_time(e1))
        ts.sort()
        return ts[len(ts) // 2]

    for k in range(10, 29, 2):
        n = 1 << k
        for _ in range(3):
            ivc.add(fmt, wa[:n], wb[:n], out=wc[:n], stream=s)
            ivc.f32_add(a[:n], b[:n], out=c32[:n], stream=s)
        reps = 20 if k < 26 else 10
        tc = timed(lambda: ivc.add(fmt, wa[:n], wb[:n], out=wc[:n], stream=s), reps)
        tf = timed(lambda: ivc.f32_add(a[:n], b[:n], out=c32[:n], stream=s), reps)
        rows.append({"log2n": k, "compressed_ms": round(tc, 5), "fp32_ms": round(tf, 5),
                     "compressed_gvec_s": _gvec(n, tc), "fp32_gvec_s": _gvec(n, tf),
                     "speedup": round(tf / tc, 4)})
    print(json.dumps({"workload": "size_sweep_add", "format": "<0,7,22>-17-18",
                      "l2_flush_bytes": 1 << 29, "rows": rows}), flush=True)


def run_gather(args):
    """Random access (the unstructured access of Sec. 1): decompress the words at
    2^28 uniformly random indices into a table of 2^28 vectors, against the
    FP32 gather from an AoS and from an SoA table of the same vectors."""
    import torch

    from paper_2003_02633_gb300 import ivc, synth
    dev = torch.device("cuda", 0)
    fmt = ivc.default_format()
    stream = torch.cuda.current_stream()
    s = stream.cuda_stream
    n = 1 << args.log2n
    x = synth.device_vectors(n, 31, dev)
    w = ivc.compress(fmt, x)
    g = torch.Generator(device=dev)
    g.manual_seed(32)
    idx = torch.randint(0, n, (n,), generator=g, device=dev, dtype=torch.int64)
    soa = x.t().contiguous()
    out = torch.empty((n, 3), dtype=torch.float32, device=dev)
    steps, warmup = max(3, min(args.steps, 20)), max(3, min(args.warmup, 5))
    res = {}
    for name, fn in (("compressed", lambda: ivc.gather_decompress(fmt, w, idx, out=out, stream=s)),
                     ("fp32_aos", lambda: ivc.f32_gather(x, idx, out=out, stream=s)),
                     ("fp32_soa", lambda: ivc.f32_gather(soa, idx, out=out, layout=ivc.IVC_SOA,
                                                          ld=n, nsrc=n, stream=s))):
        ms, _ = time_launches(fn, steps, warmup, stream)
        res[name] = {"ms": round(ms / steps, 4), "gvec_s": _gvec(n, ms / steps)}
    # bytes moved per vector at 32-byte sector granularity for the random reads
    line = {"workload": "gather_decompress", "n": n, "table": n, "index": "uniform random int64",
            "results": res,
            "speedup_vs_fp32_aos": round(res["fp32_aos"]["ms"] / res["compressed"]["ms"], 4),
            "speedup_vs_fp32_soa": round(res["fp32_soa"]["ms"] / res["compressed"]["ms"], 4),
            "sector_bytes_per_vector": {"compressed": 8 + 32 + 12, "fp32_aos": 8 + 44 + 12,
                                        "fp32_soa": 8 + 96 + 12},
            "note": "random reads cost whole 32-byte sectors: 32 B for an 8-byte word, 32 or "
                    "64 B (mean 44) for a 12-byte AoS vector, 3 x 32 B for SoA"}
    print(json.dumps(line), flush=True)


def run_codec(args):
    """The fast codec's kernels once each, in a fixed order, at N = 2^log2n
    (the target of the per-kernel ncu captures under profiles/): compress a,
    compress b (k_compress_fast), add (k_fused_fast<0>), axpy in place on b's
    words (k_fused_fast<1>), decompress of the sum (k_decompress_fast), each
    launch timed with CUDA events after `warmup` untimed rounds of the same
    sequence."""
    import torch

    from paper_2003_02633_gb300 import ivc, synth
    dev = torch.device("cuda", 0)
    fmt = ivc.default_format()
    stream = torch.cuda.current_stream()
    s = stream.cuda_stream
    n = 1 << args.log2n
    a = synth.device_vectors(n, 41, dev)
    b = synth.device_vectors(n, 42, dev)
    wa, wb, wc = (torch.empty(n, dtype=torch.int64, device=dev) for _ in range(3))
    d = torch.empty_like(a)
    seq = (("compress_a", lambda: ivc.compress(fmt, a, out=wa, stream=s)),
           ("compress_b", lambda: ivc.compress(fmt, b, out=wb, stream=s)),
           ("add", lambda: ivc.add(fmt, wa, wb, out=wc, stream=s)),
           ("axpy", lambda: ivc.axpy(fmt, 0.7, wa, wb, stream=s)),
           ("decompress", lambda: ivc.decompress(fmt, wc, out=d, stream=s)))
    for _ in range(args.warmup):
        for _, fn in seq:
            fn()
    torch.cuda.synchronize()
    res = {}
    for name, fn in seq:
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        fn()
        e1.record(stream)
        torch.cuda.synchronize()
        res[name] = {"ms": round(e0.elapsed_time(e1), 4), "gvec_s": _gvec(n, e0.elapsed_time(e1))}
    print(json.dumps({"workload": "codec_kernels", "n": n, "results": res}), flush=True)


def main():
    args = parse_args()
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "tgv":
        run_tgv(args)
    elif args.workload == "batched":
        run_batched(args)
    elif args.workload == "precision":
        run_precision(args)
    elif args.workload == "fdiv":
        run_fdiv(args)
    elif args.workload == "sweep":
        run_sweep(args)
    elif args.workload == "codec":
        run_codec(args)
    elif args.workload == "gather":
        run_gather(args)
    elif args.workload == "fr":
        run_fr(args)
    else:
        run_ivc(args)


if __name__ == "__main__":
    main()
