"""The bench's algorithmic flop counts (ALU roofline): the per-line core counts agree with the
operation counts the generator wrote for every core graph, and a block list sums by hand."""

import os
import re

import numpy as np

import bench
import synth

HERE = os.path.dirname(os.path.abspath(__file__))
CORES = os.path.join(HERE, "..", "paper_2505_23618_gb300", "csrc", "cores_gen.cuh")


def test_core_line_flops_match_the_generated_graphs():
    pat = re.compile(r"^// (DCT2|DCT3|DST2|DST3) N=(\d+): (\d+) butterflies \(2 FADD\), (\d+) rotations")
    # packed 64-point cores: two 32-point graphs in FP32x2, 32 first / last step maps (3 flops
    # a lane) and the chain ops (1 flop each)
    pat64 = re.compile(r"^// (DCT2|DCT3|DST2|DST3) N=64 packed: two 32-point lines in FP32x2 \((\d+) "
                       r"butterflies \(2 FADD\), (\d+) rotations .*, (\d+) chain ops = (\d+) instructions, "
                       r"(\d+) FP32 ops$")
    seen, packed = set(), set()
    with open(CORES) as f:
        for ln in f:
            m = pat.match(ln)
            if m:
                n, bfly, rot = int(m.group(2)), int(m.group(3)), int(m.group(4))
                assert bench.CORE_LINE_FLOPS[n] == 2 * bfly + 6 * rot, (m.group(1), n)
                seen.add((m.group(1), n))
            m = pat64.match(ln)
            if m:
                bfly, rot, nc, flops = (int(m.group(i)) for i in (2, 3, 4, 6))
                assert flops == 2 * (2 * bfly + 6 * rot) + 6 * 32 + nc
                packed.add(m.group(1))
    assert len(seen) == 20 and len(packed) == 4


def test_line_and_block_flops():
    rng = np.random.default_rng(0)
    band = synth.random_band(rng, 16, 3, [0, 1, 0, 1])          # 8 + 7 + 8 + 7 rotations
    post = synth.random_post(rng, 8, 0, 4)
    none = synth.Tf(n=4, core=2)
    dense = synth.Tf(n=8, core=0, kind=synth.KIND_DENSE, q=np.eye(8))
    assert bench.line_flops(band) == 120 + 6 * 30
    assert bench.line_flops(post) == 46 + 2 * 16
    assert bench.line_flops(none) == 16
    assert bench.line_flops(dense) == 128
    tfs = [band, post, none, dense]
    blocks = np.zeros(2, dtype=synth.BLOCK_DTYPE)
    blocks["w"], blocks["h"] = (16, 4), (8, 8)
    blocks["tf_h"], blocks["tf_v"] = (0, 2), (1, 3)
    # block 0: 8 rows of 16 (band) + 16 columns of 8 (post); block 1: 8 rows of 4 + 4 columns of 8
    want = 8 * 300 + 16 * 78 + 8 * 16 + 4 * 128
    assert bench.alg_flops(blocks, tfs) == want


def test_profiled_traffic_only_for_the_source_it_was_taken_on(monkeypatch):
    """The bench reports the committed ncu traffic counters only while the kernel source hash
    matches the one they were captured on; any change to the sources makes them null."""
    with open(os.path.join(HERE, "..", "profiles", "traffic.txt")) as f:
        lines = f.read().splitlines()
    key = [ln.split()[-1] for ln in lines if ln.startswith("source_hash")][0]
    vals = {ln.split()[0]: float(ln.split()[1]) for ln in lines
            if ln and not ln.startswith("#") and not ln.startswith("source_hash")}
    monkeypatch.setattr(bench, "kernel_source_hash", lambda: key)
    for name, v in vals.items():
        assert bench.profiled_traffic(name) == v
    monkeypatch.setattr(bench, "kernel_source_hash", lambda: "0" * 16)
    assert all(bench.profiled_traffic(name) is None for name in vals)
