"""The generated fast cores are benign in FP32: their flow graphs (butterflies and plane
rotations with FP32-rounded constants), executed in float32 on random lines, stay within
a few FP32 roundings of the exact orthonormal transforms of the oracle.  This is the
arithmetic the kernels run, so it bounds the per-line error the GPU parity tests allow
(1e-5 of the block norm) from the CPU side."""

import importlib.util
import os

import numpy as np
import pytest

import oracle as O

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def gen():
    path = os.path.join(ROOT, "paper_2505_23618_gb300", "csrc", "gen_cores.py")
    spec = importlib.util.spec_from_file_location("gen_cores", path)
    g = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(g)
    return g


def run_f32(N, prog, X):
    """The program on the lines X (N x L, float32), every operation rounded to float32."""
    ins, ops, outs = prog
    V = np.zeros((N, X.shape[1]), dtype=np.float32)
    for n in range(N):
        V[ins[n]] = X[n]
    for op in ops:
        if op[0] == "add":
            _, i, j = op
            V[i], V[j] = V[i] + V[j], V[i] - V[j]
        elif op[0] == "mat":
            _, i, j, a, b, c, d = op
            a, b, c, d = (np.float32(v) for v in (a, b, c, d))
            V[i], V[j] = a * V[i] + b * V[j], c * V[i] + d * V[j]
        elif op[0] == "scale":
            V[op[1]] = np.float32(op[2]) * V[op[1]]
        else:
            V[op[1]] = -V[op[1]]
    return np.stack([V[outs[k]] for k in range(N)])


@pytest.mark.parametrize("N", [4, 8, 16, 32, 64])
@pytest.mark.parametrize("core", range(4))
def test_core_graph_in_fp32(gen, N, core):
    rng = np.random.default_rng(100 * N + core)
    X = (rng.standard_normal((N, 2000)) * 300).astype(np.float32)
    Y = run_f32(N, gen.core_program(N, core), X).astype(np.float64)
    ref = O.core_matrix(N, core) @ X.astype(np.float64)
    rel = np.linalg.norm(Y - ref, axis=0) / np.linalg.norm(X.astype(np.float64), axis=0)
    # unit roundoff 6e-8: measured at most 1.7e-7 of the line norm at every size (the
    # rotations keep the norm, so rounding errors do not grow through the stages)
    assert rel.max() < 4e-7, rel.max()


@pytest.mark.parametrize("core", range(4))
def test_packed_64_point_core_in_fp32(gen, core):
    """The packed-pair form of the 64-point cores (two 32-point cores and a prefix chain)."""
    rng = np.random.default_rng(7000 + core)
    X = (rng.standard_normal((64, 4000)) * 300).astype(np.float32)
    Y = run_f32(64, gen.core_program(64, core, pair=True), X).astype(np.float64)
    ref = O.core_matrix(64, core) @ X.astype(np.float64)
    rel = np.linalg.norm(Y - ref, axis=0) / np.linalg.norm(X.astype(np.float64), axis=0)
    # O_k of the chain is an alternating sum of k + 1 outputs of the 32-point core, so their
    # rounding errors add up: measured at most 1.8e-6 over 20,000 lines (median 2.3e-7), a
    # fifth of the 1e-5 block tolerance of the GPU parity tests
    assert rel.max() < 2.5e-6, rel.max()
