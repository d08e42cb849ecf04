#!/usr/bin/env python3
"""Throughput of the fused adjusted 2-D transforms (forward + inverse) on one GB300.

A step is one forward and one inverse transform of the whole batch: the mixed-size
workload of 8 synthetic 3840x2160 frames (66.4 M coefficients, ~0.5 M blocks of
4..64 x 4..64, every block with its own core x adjustment per direction).  The
metric is coefficients / (t_forward + t_inverse) in Gcoef/s, with the inputs
resident in HBM; L2 is flushed (256 MiB write) before every timed kernel and the
kernels are timed with CUDA events on their stream.

Extra fields: `e2e` (the same metric through the host-buffer C-ABI entry points,
copies included), `roofline` (HBM roofline of the dominant kernel from
algorithmic bytes), `cpu_baseline` (the FP64 oracle on the host cores), the
SM clocks sampled during the timed region, and `multiple`: the encoder's
simultaneous DST-7 / DCT-8 forward (Section 2.3) on the same frame tiling against
five separate forwards.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
"""

from __future__ import annotations

import argparse
import hashlib
import json
import os
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Gcoef/s fwd+inv adjusted 2-D transforms (mixed 4-64) vs plain; % HBM roofline"
UNIT = "Gcoef/s"
FALLBACK_HBM_GBS = 6800.0
L2_FLUSH_BYTES = 256 << 20


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=300)
    p.add_argument("--warmup", type=int, default=5)
    p.add_argument("--impl", default="fused", choices=["fused", "reference"])
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--e2e-steps", type=int, default=5)
    p.add_argument("--frames", type=int, default=8, help="frames of the workload (profiling uses fewer)")
    p.add_argument("--autotune", type=int, default=48, help="autotuner evaluations before timing (0: off)")
    p.add_argument("--no-multiple", action="store_true", help="skip the Multiple-forward measurement")
    p.add_argument("--uhd8k", dest="uhd8k", action="store_true", default=True,
                   help="measure the large-frame workload (default)")
    p.add_argument("--no-uhd8k", dest="uhd8k", action="store_false")
    p.add_argument("--no-frame", action="store_true", help="skip the frame-layout measurement")
    p.add_argument("--no-bwd", action="store_true", help="skip the backward / fitter-step measurement")
    p.add_argument("--classes", action="store_true",
                   help="diagnostic: time uniform single-class workloads (one JSON line per class) instead")
    return p.parse_args()


def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def workload(rank=0, frames=8):
    import synth
    # every rank transforms its own seeded batch of the same shape (weak scaling)
    return synth.uhd_mixed(seed=3 + 1000 * rank, frames=frames)


def aggregate_max(t_local, device=None):
    """Max of a per-rank time over all ranks (identity on one rank)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(t_local)
    t = torch.tensor([float(t_local)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_rank, world, steps, t_max):
    """Weak scaling: every rank processes units_per_rank per step; the job takes t_max."""
    return units_per_rank * world * steps / t_max


def measured_peak():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback"


# FP32 peak of the ALU roofline: 152 SMs x 128 FP32 lanes x 2 flops (FMA) x 2.07 GHz.
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12
# Flops of one line through a fast core of length N (butterflies 2 flops, rotations 6: the
# operation counts of the generated core graphs).
CORE_LINE_FLOPS = {4: 16, 8: 46, 16: 120, 32: 302, 64: 740}


def line_flops(tf):
    """Algorithmic flops of one length-n line through H = C B A (same for the inverse): the fast
    core, 6 per band rotation, 2 K^2 for the K x K post block; 2 n^2 for the dense kind."""
    import synth
    if tf.kind == synth.KIND_DENSE:
        return 2 * tf.n * tf.n
    f = CORE_LINE_FLOPS[tf.n]
    if tf.kind == synth.KIND_BAND:
        f += 6 * len(tf.angles)
    elif tf.kind == synth.KIND_POST:
        f += 2 * tf.q.shape[0] ** 2
    return f


def alg_flops(blocks, tfs):
    """Algorithmic flops of one 2-D forward (or inverse) over a block list: h rows through the
    horizontal transform and w columns through the vertical one per block."""
    import numpy as np
    lf = np.array([line_flops(t) for t in tfs], dtype=np.float64)
    return float(np.sum(blocks["h"].astype(np.float64) * lf[blocks["tf_h"]] +
                        blocks["w"].astype(np.float64) * lf[blocks["tf_v"]]))


def alu_roofline(flops, ms):
    tflops = flops / (ms * 1e-3) / 1e12
    return {"bound": "alu", "achieved": round(tflops, 2), "peak": round(FP32_PEAK_TFLOPS, 1), "unit": "TFLOP/s",
            "frac": round(tflops / FP32_PEAK_TFLOPS, 4)}


def kernel_source_hash():
    h = hashlib.sha256()
    d = os.path.join(ROOT, "paper_2505_23618_gb300", "csrc")
    for f in sorted(os.listdir(d)):
        if f.endswith((".cu", ".cuh", ".h")):
            with open(os.path.join(d, f), "rb") as fh:
                h.update(f.encode() + fh.read())
    return h.hexdigest()[:16]


def profiled_traffic(kernel: str):
    """Per-launch DRAM bytes of `kernel` from the committed ncu summary, if it was
    taken on the current kernel source (else None)."""
    path = os.path.join(ROOT, "profiles", "traffic.txt")
    try:
        lines = open(path).read().splitlines()
    except OSError:
        return None
    src = None
    for ln in lines:
        if ln.startswith("source_hash"):
            src = ln.split()[-1]
    if src != kernel_source_hash():
        return None
    for ln in lines:
        parts = ln.split()
        if len(parts) >= 2 and parts[0] == kernel:
            return float(parts[1])
    return None


class ClockSampler:
    """nvidia-smi clock / throttle sampling while the timed region runs."""

    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", "50"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *a):
        self.out = ""
        if self.proc:
            self.proc.terminate()
            try:
                self.out, _ = self.proc.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                self.out, _ = self.proc.communicate()

    def summary(self):
        rows = []
        for ln in (self.out or "").splitlines():
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 7:
                continue
            try:
                rows.append((float(f[0]), float(f[1]), f[3:7]))
            except ValueError:
                continue
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"], "samples": 0}
        sm = sorted(r[0] for r in rows)
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i, v in enumerate(r[2]) if v.lower() == "active"})
        return {"sm_mhz": sm[len(sm) // 2], "sm_max_mhz": max(r[1] for r in rows), "reasons": reasons,
                "samples": len(rows)}


_ORACLE_JOBS = None


def _oracle_init(jobs):
    global _ORACLE_JOBS
    _ORACLE_JOBS = jobs


def _oracle_chunk_roundtrip(i):
    """One worker's share of the CPU baseline: FP64 oracle forward then inverse of a
    contiguous run of blocks (data rebased to the run's first sample), handed to the workers
    once when the pool starts."""
    import oracle
    data, blocks, tfs = _ORACLE_JOBS[i]
    oracle.inverse_blocks(oracle.forward_blocks(data, blocks, tfs), blocks, tfs)
    return int(data.size)


def oracle_chunks(data, blocks, tfs, n_chunks):
    """Cut a packed block list (offsets increasing, blocks back to back) into about n_chunks
    contiguous runs of similar coefficient counts, each with its own data slice."""
    import numpy as np
    sz = blocks["w"].astype(np.int64) * blocks["h"]
    cs = np.cumsum(sz)
    cuts = np.searchsorted(cs, np.linspace(0, cs[-1], n_chunks + 1)[1:-1])
    jobs = []
    for part in np.split(np.arange(blocks.size), cuts):
        if part.size == 0:
            continue
        b = blocks[part].copy()
        lo = int(b["offset"][0])
        hi = int(b["offset"][-1] + sz[part[-1]])
        b["offset"] -= lo
        jobs.append((np.ascontiguousarray(data[lo:hi]), b, tfs))
    return jobs


def oracle_pool(cores, jobs):
    """Process pool for the oracle, one single-threaded worker per core (BLAS pinned to one
    thread per process), each holding the jobs; started with spawn so that no worker inherits
    GPU state."""
    import multiprocessing as mp
    for v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ[v] = "1"
    return mp.get_context("spawn").Pool(cores, initializer=_oracle_init, initargs=(jobs,))


def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


# Wall time the CPU baseline aims for (seconds over all host cores: 1.5 s x 16 cores is about
# 24 s of CPU work); the number of timed passes over the workload follows from one untimed pass.
CPU_BASELINE_WALL_S = 1.5


def cpu_baseline(sample_desc="full workload (66.4 M coefficients), one forward + one inverse per pass"):
    """Time the FP64 oracle on the host cores: a process pool (one single-threaded worker
    per core) over contiguous runs of blocks, in a child process started before any GPU work
    of its own."""
    cores = host_cores()
    code = (
        "import time, json, sys; sys.path.insert(0, %r)\n"
        "import bench, synth\n"
        "if __name__ == '__main__':\n"
        "    wl = synth.uhd_mixed()\n"
        "    jobs = bench.oracle_chunks(wl.data, wl.blocks, wl.tfs, 4 * %d)\n"
        "    with bench.oracle_pool(%d, jobs) as pool:\n"
        "        t = time.perf_counter()\n"
        "        pool.map(bench._oracle_chunk_roundtrip, range(len(jobs)), chunksize=1)\n"
        "        reps = max(1, min(20, int(%r / max(time.perf_counter() - t, 1e-3)) + 1))\n"
        "        t = time.perf_counter()\n"
        "        n = 0\n"
        "        for _ in range(reps):\n"
        "            n += sum(pool.map(bench._oracle_chunk_roundtrip, range(len(jobs)), chunksize=1))\n"
        "        dt = time.perf_counter() - t\n"
        "    print(json.dumps({'coefs': int(n), 'seconds': dt, 'passes': reps}))\n"
        % (ROOT, cores, cores, CPU_BASELINE_WALL_S))
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1")
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env, timeout=1800)
    if r.returncode != 0:
        return {"value": None, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample_desc,
                "error": r.stderr[-300:]}
    d = json.loads(r.stdout.strip().splitlines()[-1])
    return {"value": d["coefs"] / d["seconds"] / 1e9, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": sample_desc + f", {d['passes']} timed passes after one untimed, {cores} single-threaded "
                                    "processes over contiguous block runs",
            "seconds": round(d["seconds"], 3)}


def run_reference(args):
    world, rank, _ = dist_env()
    if rank != 0:
        return 0
    import numpy as np
    import synth
    wl = workload(0)
    cores = host_cores()
    # each step transforms a bounded sample of the workload: its first ~1 M coefficients per
    # host core, split over the cores in contiguous runs of blocks
    cs = np.cumsum(wl.blocks["w"].astype(np.int64) * wl.blocks["h"])
    nb = int(np.searchsorted(cs, 1_000_000 * cores)) + 1
    nb = min(nb, int(wl.blocks.size))
    blocks, tot = wl.blocks[:nb], int(cs[nb - 1])
    jobs = oracle_chunks(wl.data[:tot], blocks, wl.tfs, 4 * cores)
    with oracle_pool(cores, jobs) as pool:
        for _ in range(args.warmup):
            pool.map(_oracle_chunk_roundtrip, range(len(jobs)), chunksize=1)
        t0 = time.perf_counter()
        for _ in range(args.steps):
            pool.map(_oracle_chunk_roundtrip, range(len(jobs)), chunksize=1)
        dt = time.perf_counter() - t0
    value = tot * args.steps / dt / 1e9
    sample = (f"first {nb} blocks ({tot} coefficients) of the workload per step, "
              f"{cores} single-threaded processes over contiguous block runs")
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": wl.name, "coefs": tot, "blocks": nb, "what": "FP64 CPU oracle"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores,
                         "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def bench_multiple(args, rank, dev, stream, flush, peak):
    """The encoder's DST-7 / DCT-8 search (Section 2.3) on the same frame tiling: one
    Multiple forward (2-D DCT-2 + the distinct coefficients of the four adjusted pairings)
    against five separate fused forwards (DCT-2 and each pairing with its own post
    transforms, Q or S Q S), every launch after an L2 flush, median of the timed repeats."""
    import numpy as np
    import torch

    import oracle
    import synth
    import paper_2505_23618_gb300 as adj

    wl = synth.uhd_mixed_multiple(seed=3 + 1000 * rank, frames=args.frames)
    coefs, nb = wl.total, int(wl.blocks.size)
    reps = max(3, min(args.steps, 30))
    x = torch.from_numpy(wl.data).to(dev)
    y = torch.empty(coefs, dtype=torch.float32, device=dev)

    def timed(fn):
        for _ in range(2):
            fn()
        ev = [[torch.cuda.Event(enable_timing=True) for _ in range(2)] for _ in range(reps)]
        for e in ev:
            flush.fill_(5.0)
            e[0].record(stream)
            fn()
            e[1].record(stream)
        torch.cuda.synchronize()
        return float(np.median([e[0].elapsed_time(e[1]) for e in ev]))

    with adj.Plan(wl.tfs) as plan:
        plan.set_blocks(wl.blocks, coefs)
        off = plan.prepare_multiple()
        side = torch.empty(int(off[-1]), dtype=torch.float32, device=dev)
        ms_multi = timed(lambda: plan.fwd_multiple(x, y, side, stream))
        n_tiles = plan.info()["n_tiles"]
    # the five transforms one by one: DCT-2, then (vertical, horizontal) = SS, SC, CS, CC
    n_dir = len(synth.SIZES)
    ms_sep = 0.0
    for combo in ("DD",) + tuple(oracle.MULTI_COMBOS):
        tfs = []
        for d, t in enumerate(wl.tfs):
            c = combo[1] if d < n_dir else combo[0]     # first half horizontal, second vertical
            if c == "D":
                tfs.append(synth.Tf(n=t.n, core=0))
            else:
                q = t.q if c == "S" else oracle.post_c8_from_s7(t.q)
                tfs.append(synth.Tf(n=t.n, core=0, kind=synth.KIND_POST, q=q))
        with adj.Plan(tfs) as p5:
            p5.set_blocks(wl.blocks, coefs)
            ms_sep += timed(lambda: p5.fwd(x, y, stream))
    algo = coefs * 6 + int(off[-1]) * 4 + n_tiles * 16 + nb * 8
    gbs = algo / (ms_multi * 1e-3) / 1e9
    return {"workload": wl.name, "value": round(coefs / (ms_multi * 1e-3) / 1e9, 3), "unit": UNIT,
            "ms": round(ms_multi, 4), "side_floats": int(off[-1]),
            "algorithmic_bytes": algo, "GB/s": round(gbs, 1), "frac": round(gbs / peak, 4),
            "five_separate_ms": round(ms_sep, 4), "vs_five_separate": round(ms_sep / ms_multi, 3),
            "how": "one launch for DCT-2 + 4 DST-7/DCT-8 pairings vs 5 fused forwards, median of "
                   f"{reps} L2-flushed repeats"}


FITTED = os.path.join(ROOT, "paper_2505_23618_gb300", "params", "fitted.json")


def uhd8k_tfs():
    """The large-frame workload's transforms: fitted DST-7 / DCT-8 approximations when the
    fitted parameter file is present (horizontal DST-3 + 12-layer band; vertical DCT-2 + post
    with the DCT-8 block S Q S of Eq. 5), else None (the workload's seeded parameters)."""
    import numpy as np
    import synth
    try:
        with open(FITTED) as f:
            fit = json.load(f)
        b = fit["band_dst3_64"]
        h_tf = synth.Tf(n=64, core=synth.CORE_DST3, kind=synth.KIND_BAND,
                        parities=np.array(b["parities"], np.uint8), angles=np.array(b["angles"]))
        v_tfs = {n: synth.Tf(n=n, core=synth.CORE_DCT2, kind=synth.KIND_POST,
                             q=np.array(fit[f"post_dct2_{n}"]["q_dct8"]))
                 for n in (64, 32)}
        return h_tf, v_tfs, "fitted (paper_2505_23618_gb300/params/fitted.json)"
    except (OSError, KeyError, ValueError):
        return None, None, "seeded"


def bench_uhd8k(args, rank, dev, stream, flush, peak):
    """Large-frame workload (16 frames of 7680x4320, 64x64 and 64x32 blocks; horizontal
    DST-7 approximation, vertical DCT-8 approximation): fused forward + inverse, and the exact
    dense DST-7 / DCT-8 product on the same blocks as context.  Median of L2-flushed repeats."""
    import numpy as np
    import torch

    import synth
    import paper_2505_23618_gb300 as adj
    from paper_2505_23618_gb300 import targets

    h_tf, v_tfs, src = uhd8k_tfs()
    wl = synth.uhd8k(seed=5 + 1000 * rank, h_tf=h_tf, v_tfs=v_tfs)
    coefs, nb = wl.total, int(wl.blocks.size)
    reps = max(3, min(args.steps, 10))
    x = torch.from_numpy(wl.data).to(dev)
    y = torch.empty(coefs, dtype=torch.float32, device=dev)
    xr = torch.empty(coefs, dtype=torch.float32, device=dev)

    def timed(fwd, inv):
        for _ in range(2):
            fwd()
            inv()
        ev = [[torch.cuda.Event(enable_timing=True) for _ in range(4)] for _ in range(reps)]
        for e in ev:
            flush.fill_(6.0)
            e[0].record(stream)
            fwd()
            e[1].record(stream)
            flush.fill_(7.0)
            e[2].record(stream)
            inv()
            e[3].record(stream)
        torch.cuda.synchronize()
        tf = float(np.median([e[0].elapsed_time(e[1]) for e in ev]))
        ti = float(np.median([e[2].elapsed_time(e[3]) for e in ev]))
        return tf, ti

    out = {"workload": wl.name, "params": src}
    with adj.Plan(wl.tfs) as plan:
        plan.set_blocks(wl.blocks, coefs)
        tiles = plan.info()["n_tiles"]
        tf, ti = timed(lambda: plan.fwd(x, y, stream), lambda: plan.inv(y, xr, stream))
        torch.cuda.synchronize()
        rt = float((xr - x.float()).abs().max())
    meta = tiles * 16 + nb * 4
    bf, bi = coefs * 6 + meta, coefs * 8 + meta
    fl = alg_flops(wl.blocks, wl.tfs)
    out.update({"value": round(coefs / ((tf + ti) * 1e-3) / 1e9, 3), "unit": UNIT, "coefs": coefs,
                "fwd_ms": round(tf, 4), "inv_ms": round(ti, 4),
                "fwd_frac": round(bf / (tf * 1e-3) / 1e9 / peak, 4), "inv_frac": round(bi / (ti * 1e-3) / 1e9 / peak, 4),
                "flops_per_coef": round(fl / coefs, 2), "alu_fwd": alu_roofline(fl, tf), "alu_inv": alu_roofline(fl, ti),
                "algorithmic_bytes": {"fwd": bf, "inv": bi},
                "traffic": {"fwd": profiled_traffic("uhd8k_fwd"), "inv": profiled_traffic("uhd8k_inv")},
                "roundtrip_max_abs_err": rt})
    # the exact transforms the adjustments stand in for, as dense products (Eq. 3)
    dense = [targets.dense_tf(targets.dst7(64)), targets.dense_tf(targets.dct8(64)), targets.dense_tf(targets.dct8(32))]
    with adj.Plan(dense) as plan:
        plan.set_blocks(wl.blocks, coefs)
        tf, ti = timed(lambda: plan.fwd(x, y, stream), lambda: plan.inv(y, xr, stream))
    out["dense_dst7_dct8"] = {"value": round(coefs / ((tf + ti) * 1e-3) / 1e9, 3), "unit": UNIT,
                              "fwd_ms": round(tf, 4), "inv_ms": round(ti, 4)}
    out["vs_dense"] = round(out["value"] / out["dense_dst7_dct8"]["value"], 3)
    out["how"] = f"median of {reps} L2-flushed repeats per kernel"
    del x, y, xr
    return out


def bench_bwd(args, rank, dev, stream, flush, peak):
    """Backward of the two DST-7 fits at their full size (65,536 AR(1) 64x64 blocks, one 1-D
    transform used in both directions): the 64-point DCT-2 with the 24-tap band (378 angles)
    and the 64-point DST-2 with the 32x32 Cayley post block.  Times adj_transform_bwd alone
    (dL/dparams from x and dL/dY, the fitter's call; CUDA events, median of L2-flushed
    repeats) and one whole fitter step (forward, coding-gain proxy, backward, host Adam;
    wall clock).  Algorithmic bytes: x (int16) and dL/dY (FP32), 6 per coefficient; flops:
    the outer products sum a b^T (2 m^2 per line and direction, m = 64 for the band, 32 for
    the post block) plus three line transforms per line and direction (the recomputed
    forward, the transposed pass of dL/dY and the recomputed input of the row gradients)."""
    import numpy as np
    import torch
    from paper_2505_23618_gb300.fit import FitConfig, Fitter

    reps = max(3, min(args.steps, 10))
    out = {"workload": "65536 blocks 64x64 AR(1) rho 0.95 sigma 40 (the fits' blocks)", "unit": UNIT}
    for name, cfg in (("band_dct2_378", FitConfig(core=0, kind=1, seed=4 + 1000 * rank)),
                      ("post_dst2_k32", FitConfig(core=2, kind=2, seed=4 + 1000 * rank))):
        f = Fitter(cfg, device=dev)
        coefs = int(f.x.numel())
        f.loss_and_grad()
        gy = torch.randn(coefs, device=dev)
        for _ in range(2):
            f.plan.bwd(f.x, gy, None, f.gp, stream)
        ev = [[torch.cuda.Event(enable_timing=True) for _ in range(2)] for _ in range(reps)]
        for e in ev:
            flush.fill_(3.0)
            e[0].record(stream)
            f.plan.bwd(f.x, gy, None, f.gp, stream)
            e[1].record(stream)
        torch.cuda.synchronize()
        ms = float(np.median([e[0].elapsed_time(e[1]) for e in ev]))
        t0 = time.perf_counter()
        steps = 3
        for _ in range(steps):
            f.step()
        step_ms = (time.perf_counter() - t0) / steps * 1e3
        lines = 2 * 64 * (coefs // 4096)
        m = 64 if cfg.kind == 1 else cfg.k
        import synth
        lf = line_flops(synth.Tf(n=64, core=cfg.core, kind=cfg.kind, angles=np.asarray(f.theta))
                        if cfg.kind == 1 else synth.Tf(n=64, core=cfg.core, kind=cfg.kind, q=f.q()))
        flops = lines * (2 * m * m + 3 * lf)
        gbs = coefs * 6 / (ms * 1e-3) / 1e9
        out[name] = {"bwd_ms": round(ms, 4), "GB/s": round(gbs, 1), "hbm_frac": round(gbs / peak, 4),
                     "flops_per_coef": round(flops / coefs, 1),
                     "alu": alu_roofline(flops, ms), "fit_step_ms": round(step_ms, 2),
                     "coef_per_s_bwd": round(coefs / (ms * 1e-3) / 1e9, 3)}
        f.plan.close()
        del f, gy
    out["how"] = f"median of {reps} L2-flushed repeats; fit step: wall clock of 3 steps"
    return out


def bench_frame(args, rank, dev, stream, flush, peak):
    """Blocks inside frames (no packing step): forward from an int16 residual frame and inverse
    back into an int16 frame (rounded), on 8 frames of 3840x2160 tiled like the mixed UHD
    workload and stacked into one frame (one launch per direction), median of L2-flushed
    repeats."""
    import numpy as np
    import torch

    import synth
    import paper_2505_23618_gb300 as adj

    reps = max(3, min(args.steps, 20))
    n_frames = max(1, args.frames)
    frame, blocks, tfs = synth.uhd_mixed_frame(seed=3 + 1000 * rank, frames=n_frames)
    plan = adj.Plan(tfs)
    plan.set_frame_blocks(blocks, 3840, frame.shape[0], frame.shape[1])
    x = torch.from_numpy(frame).to(dev)
    y = torch.empty(plan.total, dtype=torch.float32, device=dev)
    r = torch.empty_like(x)
    coefs = plan.total
    for _ in range(2):
        plan.fwd_frame(x, y, stream)
        plan.inv_frame(y, d_frame_i16=r, stream=stream)
    ev = [[torch.cuda.Event(enable_timing=True) for _ in range(4)] for _ in range(reps)]
    for e in ev:
        flush.fill_(8.0)
        e[0].record(stream)
        plan.fwd_frame(x, y, stream)
        e[1].record(stream)
        flush.fill_(9.0)
        e[2].record(stream)
        plan.inv_frame(y, d_frame_i16=r, stream=stream)
        e[3].record(stream)
    torch.cuda.synchronize()
    exact = bool(torch.equal(r[:, :3840], x[:, :3840]))
    tf = float(np.median([e[0].elapsed_time(e[1]) for e in ev]))
    ti = float(np.median([e[2].elapsed_time(e[3]) for e in ev]))
    plan.close()
    return {"workload": f"{n_frames} frames 3840x2160 (mixed 4-64 tiling) stacked, int16 frame in, int16 frame out",
            "value": round(coefs / ((tf + ti) * 1e-3) / 1e9, 3), "unit": UNIT, "fwd_ms": round(tf, 4),
            "inv_ms": round(ti, 4), "fwd_frac": round(coefs * 6 / (tf * 1e-3) / 1e9 / peak, 4),
            "inv_frac": round(coefs * 6 / (ti * 1e-3) / 1e9 / peak, 4),
            "int16_roundtrip_exact": exact, "how": f"median of {reps} L2-flushed repeats"}


def run_fused(args):
    import numpy as np
    import torch

    import paper_2505_23618_gb300 as adj

    world, rank, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    wl = workload(rank, args.frames)
    coefs = wl.total
    plan = adj.Plan(wl.tfs)
    plan.set_blocks(wl.blocks, coefs)
    stream = torch.cuda.current_stream(dev)

    x = torch.from_numpy(wl.data).to(dev)
    y = torch.empty(coefs, dtype=torch.float32, device=dev)
    xr = torch.empty(coefs, dtype=torch.float32, device=dev)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    # the planner's autotuner (tile capacity per block size, CTAs and ranges per SM), then one
    # CUDA graph per direction around the persistent launch
    if args.autotune > 0:
        plan.autotune(x, y, xr, None, args.autotune, stream)
    tuning = plan.tuning()
    info = plan.info()
    from paper_2505_23618_gb300 import _lib as L
    g_fwd_fused = plan.graph(L.GRAPH_FWD, x, y)
    g_inv_fused = plan.graph(L.GRAPH_INV, y, xr)

    def step(ev=None):
        flush.fill_(1.0)
        if ev:
            ev[0].record(stream)
        g_fwd_fused.launch(stream)
        if ev:
            ev[1].record(stream)
        flush.fill_(2.0)
        if ev:
            ev[2].record(stream)
        g_inv_fused.launch(stream)
        if ev:
            ev[3].record(stream)

    for _ in range(max(3, args.warmup)):
        step()
    torch.cuda.synchronize()
    # correctness guard on the timed buffers (round trip), outside the timed region
    rt = float((xr - x.float()).abs().max())

    events = [[torch.cuda.Event(enable_timing=True) for _ in range(4)] for _ in range(args.steps)]
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        for k in range(args.steps):
            step(events[k])
        torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    t_fwd = np.array([e[0].elapsed_time(e[1]) for e in events]) * 1e-3
    t_inv = np.array([e[2].elapsed_time(e[3]) for e in events]) * 1e-3
    t_total = aggregate_max(float(t_fwd.sum() + t_inv.sum()), dev)
    value = whole_job_rate(coefs, world, args.steps, t_total) / 1e9

    # the plain (unfused) form on the same blocks, replayed from CUDA graphs (its best case:
    # no per-launch host overhead); same flushes and event timing as the fused kernels
    yp = torch.empty_like(y)
    xrp = torch.empty_like(xr)
    g_fwd = plan.graph(L.GRAPH_FWD_PLAIN, x, yp)
    g_inv = plan.graph(L.GRAPH_INV_PLAIN, yp, xrp)
    plain_steps = max(3, min(args.steps, 30))
    for _ in range(2):
        g_fwd.launch(stream)
        g_inv.launch(stream)
    pev = [[torch.cuda.Event(enable_timing=True) for _ in range(4)] for _ in range(plain_steps)]
    for k in range(plain_steps):
        flush.fill_(3.0)
        pev[k][0].record(stream)
        g_fwd.launch(stream)
        pev[k][1].record(stream)
        flush.fill_(4.0)
        pev[k][2].record(stream)
        g_inv.launch(stream)
        pev[k][3].record(stream)
    torch.cuda.synchronize()
    pf = np.array([e[0].elapsed_time(e[1]) for e in pev]) * 1e-3
    pi = np.array([e[2].elapsed_time(e[3]) for e in pev]) * 1e-3
    plain_value = coefs * world / float(np.median(pf) + np.median(pi)) / 1e9
    plain_launches = 6 * len(set(zip(wl.blocks["w"].tolist(), wl.blocks["h"].tolist())))
    plain_rt = float((xrp - x.float()).abs().max())
    g_fwd.close()
    g_inv.close()
    del yp, xrp

    peak, peak_src = measured_peak()
    multiple = bench_multiple(args, rank, dev, stream, flush, peak) if not args.no_multiple else None
    uhd8k = bench_uhd8k(args, rank, dev, stream, flush, peak) if args.uhd8k else None
    frame = bench_frame(args, rank, dev, stream, flush, peak) if not args.no_frame else None
    bwd = bench_bwd(args, rank, dev, stream, flush, peak) if not args.no_bwd else None

    # end to end through the host-buffer C-ABI calls (pinned memory), copies included
    h_x = torch.from_numpy(wl.data).pin_memory()
    h_y = torch.empty(coefs, dtype=torch.float32).pin_memory()
    h_xr = torch.empty(coefs, dtype=torch.float32).pin_memory()
    plan.fwd_host(h_x, h_y, stream)
    plan.inv_host(h_y, h_xr, stream)
    t0 = time.perf_counter()
    for _ in range(args.e2e_steps):
        plan.fwd_host(h_x, h_y, stream)
        plan.inv_host(h_y, h_xr, stream)
    e2e_t = aggregate_max((time.perf_counter() - t0) / args.e2e_steps, dev)
    e2e_value = whole_job_rate(coefs, world, 1, e2e_t) / 1e9

    flops = alg_flops(wl.blocks, wl.tfs)  # per launch, forward or inverse
    # roofline of the dominant kernel (algorithmic bytes per launch / mean duration)
    nb = int(wl.blocks.size)
    meta = info["n_tiles"] * 16 + nb * 4
    kern = {
        "fwd": {"bytes": coefs * 6 + meta, "ms": float(t_fwd.mean() * 1e3)},
        "inv": {"bytes": coefs * 8 + meta, "ms": float(t_inv.mean() * 1e3)},
    }
    for k in kern.values():
        k["gbs"] = k["bytes"] / (k["ms"] * 1e-3) / 1e9
        k["frac"] = k["gbs"] / peak
    dom = max(kern, key=lambda k: kern[k]["ms"])
    traffic = profiled_traffic(dom)
    roof = {"bound": "hbm", "achieved": round(kern[dom]["gbs"], 1), "peak": peak, "unit": "GB/s",
            "frac": round(kern[dom]["frac"], 4), "traffic": traffic, "kernel": f"fused_kernel<{dom}>",
            "algorithmic_bytes_per_launch": kern[dom]["bytes"], "peak_source": peak_src + " hbm_gbs"}

    if rank == 0:
        line = {
            "metric": METRIC, "value": round(value, 3), "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": round(t_total / args.steps * 1e3, 4),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": wl.name, "coefs_per_gpu": coefs, "blocks_per_gpu": nb,
                       "tiles": info["n_tiles"], "grid": info["grid_fwd"], "threads": info["threads"],
                       "tuning": {"autotune_evals": args.autotune, "ctas_per_sm": tuning["ctas_per_sm"],
                                  "ranges_per_sm": tuning["ranges_per_sm"], "tail_pct": tuning["tail_pct"],
                                  "cap_div": {f"{4 << (i // 5)}x{4 << (i % 5)}": d
                                              for i, d in enumerate(tuning["cap_div"]) if d != 1}},
                       "launch": "one CUDA graph per direction around the persistent kernel",
                       "l2": "flushed by a 256 MiB write before every timed kernel",
                       "layout": "packed block-linear int16 in, FP32 coefficients / reconstruction out"},
            "e2e": {"value": round(e2e_value, 3), "unit": UNIT, "h2d_bytes_per_step": coefs * (2 + 4),
                    "d2h_bytes_per_step": coefs * (4 + 4)},
            "gpu_launches": 2 * args.steps,
            "vs_plain": round(value / plain_value, 3),
            "plain": {"value": round(plain_value, 3), "unit": UNIT, "fwd_ms": round(float(np.median(pf)) * 1e3, 4),
                      "inv_ms": round(float(np.median(pi)) * 1e3, 4), "launches_per_direction": plain_launches,
                      "timed_steps": plain_steps, "how": "CUDA-graph replay of one launch per block size and step",
                      "roundtrip_max_abs_err": plain_rt},
            "roofline": roof,
            "multiple": multiple,
            "uhd8k": uhd8k,
            "frame": frame,
            "bwd": bwd,
            "kernels": {k: {"ms": round(v["ms"], 4), "GB/s": round(v["gbs"], 1), "frac": round(v["frac"], 4)}
                        for k, v in kern.items()},
            "flops_per_coef": round(flops / coefs, 2),
            "alu_roofline": {k: alu_roofline(flops, v["ms"]) for k, v in kern.items()},
            "clocks": clk.summary(),
            "roundtrip_max_abs_err": rt,
        }
        if not args.no_cpu_baseline and world == 1 and args.frames == 8:
            line["cpu_baseline"] = cpu_baseline()
        print(json.dumps(line), flush=True)
    g_fwd_fused.close()
    g_inv_fused.close()
    plan.close()
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


# Uniform single-class workloads of the diagnostic mode: (w, h, core, kind); band = 2 layers
# (even, odd), post K = n / 2; about 2^26 coefficients each.
CLASSES = [(64, 64, 0, 0), (64, 64, 0, 1), (64, 64, 0, 2), (32, 32, 0, 0), (32, 32, 2, 1), (32, 32, 0, 2),
           (16, 16, 0, 0), (16, 16, 3, 1), (8, 8, 0, 0), (4, 4, 0, 0), (4, 64, 0, 0), (64, 4, 0, 0)]


def run_classes(args):
    """Forward and inverse times of uniform workloads, one block class each (L2 flushed before
    every timed kernel, CUDA events); a diagnostic of where the mixed workload spends its time."""
    import numpy as np
    import torch
    import synth
    import paper_2505_23618_gb300 as adj
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    rng = np.random.default_rng(0)
    peak, _ = measured_peak()
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)

    def tf(n, core, kind):
        if kind == synth.KIND_NONE:
            return synth.Tf(n=n, core=core)
        if kind == synth.KIND_BAND:
            return synth.random_band(rng, n, core, [0, 1])
        return synth.random_post(rng, n, core, n // 2)

    for w, h, core, kind in CLASSES:
        nb = (1 << 26) // (w * h)
        blocks = np.zeros(nb, dtype=synth.BLOCK_DTYPE)
        blocks["offset"] = np.arange(nb, dtype=np.int64) * w * h
        blocks["w"], blocks["h"], blocks["tf_h"], blocks["tf_v"] = w, h, 0, 1
        total = nb * w * h
        x = torch.randint(-500, 500, (total,), dtype=torch.int16, device=dev)
        y = torch.empty(total, device=dev)
        xr = torch.empty_like(y)
        with adj.Plan([tf(w, core, kind), tf(h, core, kind)]) as plan:
            plan.set_blocks(blocks, total)
            for _ in range(max(1, args.warmup)):
                plan.fwd(x, y)
                plan.inv(y, xr)
            tf_, ti_ = [], []
            for _ in range(max(1, args.steps)):
                ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
                flush.fill_(1.0)
                ev[0].record()
                plan.fwd(x, y)
                ev[1].record()
                flush.fill_(2.0)
                ev[2].record()
                plan.inv(y, xr)
                ev[3].record()
                torch.cuda.synchronize()
                tf_.append(ev[0].elapsed_time(ev[1]))
                ti_.append(ev[2].elapsed_time(ev[3]))
            mf, mi = float(np.median(tf_)), float(np.median(ti_))
            print(json.dumps({"class": f"{w}x{h} core {core} kind {kind}", "coefs": total, "tiles": plan.info()["n_tiles"],
                              "fwd_ms": round(mf, 4), "inv_ms": round(mi, 4),
                              "fwd_frac": round(total * 6 / (mf * 1e-3) / 1e9 / peak, 4),
                              "inv_frac": round(total * 8 / (mi * 1e-3) / 1e9 / peak, 4)}), flush=True)
        del x, y, xr
    return 0


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    if args.classes:
        return run_classes(args)
    return run_fused(args)


if __name__ == "__main__":
    sys.exit(main())
