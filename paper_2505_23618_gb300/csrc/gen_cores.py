#!/usr/bin/env python3
"""Generate straight-line CUDA for the fast DCT-2 / DCT-3 / DST-2 / DST-3 cores.

The DCT-2 of length N is built as a flow graph of 2x2 operations on N register
slots by the even/odd recursion:

    DCT2_N x = interleave( DCT2_{N/2} u , DCT4_{N/2} d ),
    u_n = (x_n + x_{N-1-n}) / sqrt(2),  d_n = (x_n - x_{N-1-n}) / sqrt(2),

and the DCT-4 half by pairing (x_{2m}, x_{M-1-2m}) into complex values, a
pre-rotation, an M/2-point complex inverse DFT (radix-2) and a post-rotation.
Every non-trivial step is a plane rotation or a +/- butterfly, so the graph is
orthogonal and numerically benign in FP32.  All 1/sqrt(2) factors are folded
into the rotation constants of the base cases.

The other three cores come from the same graph through the relations of
Section 2.1 of Said, Egilmez & Chao:
    DCT-3 = DCT-2^T                       (reverse the graph, transpose each op)
    DST-2 = R DCT-2 S                     (negate odd inputs, reverse outputs)
    DST-3 = S DCT-2^T R                   (reverse inputs, negate odd outputs)
R (reversal) and S (alternating sign) cost nothing: they become register
renaming and negation modifiers that the compiler folds into the adds/FMAs.

The script checks each generated graph in FP64 against its own definition of
the orthonormal DCT-2 before writing ``cores_gen.cuh``.
"""

from __future__ import annotations

import math
import os
import sys

import numpy as np

SIZES = (4, 8, 16, 32, 64)
CORE_NAMES = {0: "DCT2", 1: "DCT3", 2: "DST2", 3: "DST3"}


class Graph:
    """In-place ops on register slots 0..n-1.

    ('add', i, j)            : (s_i, s_j) <- (s_i + s_j, s_i - s_j)
    ('mat', i, j, a, b, c, d): (s_i, s_j) <- (a s_i + b s_j, c s_i + d s_j)
    ('neg', i)               : s_i <- -s_i
    """

    def __init__(self, n):
        self.n = n
        self.ops = []

    def add(self, i, j):
        self.ops.append(("add", i, j))

    def mat(self, i, j, a, b, c, d):
        self.ops.append(("mat", i, j, a, b, c, d))

    def neg(self, i):
        self.ops.append(("neg", i))


def _dct2(g, slots, scale):
    M = len(slots)
    if M == 2:
        a = scale / math.sqrt(2.0)
        g.mat(slots[0], slots[1], a, a, a, -a)
        return list(slots)
    h = M // 2
    for n in range(h):
        g.add(slots[n], slots[M - 1 - n])
    ev = _dct2(g, slots[:h], scale / math.sqrt(2.0))
    od = _dct4(g, [slots[M - 1 - n] for n in range(h)], scale / math.sqrt(2.0))
    out = [None] * M
    out[0::2] = ev
    out[1::2] = od
    return out


def _dct4(g, slots, scale):
    """scale * orthonormal DCT-4 of the values in ``slots``; returns output slots."""
    M = len(slots)
    if M == 2:
        c, s = math.cos(math.pi / 8), math.sin(math.pi / 8)
        g.mat(slots[0], slots[1], scale * c, scale * s, scale * s, -scale * c)
        return list(slots)
    P = M // 2
    cpx = []
    for m in range(P):
        re, im = slots[2 * m], slots[M - 1 - 2 * m]     # a_m, b_m; z_m = a_m - i b_m
        if m == 0:
            g.neg(im)
        else:
            th = math.pi * m / M                        # z_m *= e^{i th}
            g.mat(re, im, math.cos(th), math.sin(th), math.sin(th), -math.cos(th))
        cpx.append((re, im))
    Z = _idft(g, cpx)
    out = [None] * M
    f = scale * math.sqrt(2.0 / M)
    for p, (re, im) in enumerate(Z):
        ph = math.pi * (4 * p + 1) / (4 * M)             # W_p = f Z_p e^{i ph}
        c, s = math.cos(ph), math.sin(ph)
        g.mat(re, im, f * c, -f * s, f * s, f * c)
        out[2 * p] = re
        out[M - 1 - 2 * p] = im
    return out


def _idft(g, cpx):
    """Z_p = sum_m z_m e^{+2 pi i m p / P}, radix-2 decimation in time."""
    P = len(cpx)
    if P == 1:
        return list(cpx)
    E = _idft(g, cpx[0::2])
    O = _idft(g, cpx[1::2])
    out = [None] * P
    half = P // 2
    for p in range(half):
        ore, oim = O[p]
        if p == 0:
            pass
        elif 4 * p == P:                                 # times i: (re, im) -> (-im, re)
            g.neg(oim)
            ore, oim = oim, ore
        else:
            th = 2 * math.pi * p / P
            c, s = math.cos(th), math.sin(th)
            g.mat(ore, oim, c, -s, s, c)
        ere, eim = E[p]
        g.add(ere, ore)
        g.add(eim, oim)
        out[p] = (ere, eim)
        out[p + half] = (ore, oim)
    return out


def dct2_program(N):
    g = Graph(N)
    outs = _dct2(g, list(range(N)), 1.0)
    return list(range(N)), g.ops, outs, [], []


def transpose_ops(ops):
    t = []
    for op in reversed(ops):
        if op[0] == "mat":
            _, i, j, a, b, c, d = op
            t.append(("mat", i, j, a, c, b, d))
        else:
            t.append(op)
    return t


def core_program(N, core):
    """(input slot of x_n, ops, output slot of y_k) for one of the four cores."""
    ins, ops, outs, _, _ = dct2_program(N)
    if core == 0:                                        # DCT-2
        return ins, ops, outs
    if core == 2:                                        # DST-2 = R DCT-2 S
        pre = [("neg", n) for n in range(1, N, 2)]
        return ins, pre + ops, [outs[N - 1 - k] for k in range(N)]
    tops = transpose_ops(ops)
    if core == 1:                                        # DCT-3 = DCT-2^T
        return list(outs), tops, list(range(N))
    if core == 3:                                        # DST-3 = S DCT-2^T R
        post = [("neg", m) for m in range(1, N, 2)]
        return [outs[N - 1 - n] for n in range(N)], tops + post, list(range(N))
    raise ValueError(core)


def simulate(N, prog):
    """FP64 matrix (rows = outputs, cols = inputs) computed by a program."""
    ins, ops, outs = prog
    V = np.zeros((N, N))
    for n in range(N):
        V[ins[n], n] = 1.0
    for op in ops:
        if op[0] == "add":
            _, i, j = op
            V[i], V[j] = V[i] + V[j], V[i] - V[j]
        elif op[0] == "mat":
            _, i, j, a, b, c, d = op
            V[i], V[j] = a * V[i] + b * V[j], c * V[i] + d * V[j]
        else:
            V[op[1]] = -V[op[1]]
    return np.stack([V[outs[k]] for k in range(N)])


def definition(N, core):
    """This generator's own closed forms, used only to check the graphs."""
    k = np.arange(N)[:, None]
    n = np.arange(N)[None, :]
    c2 = np.sqrt(2.0 / N) * np.cos(np.pi * (2 * n + 1) * k / (2 * N))
    c2[0] /= np.sqrt(2.0)
    s2 = np.sqrt(2.0 / N) * np.sin(np.pi * (2 * n + 1) * (k + 1) / (2 * N))
    s2[N - 1] /= np.sqrt(2.0)
    return {0: c2, 1: c2.T, 2: s2, 3: s2.T}[core]


def f32(x):
    v = float(np.float32(x))
    return "%.9ef" % v


def emit(N, core, prog):
    """Straight-line code of one core, templated on the element type T (float, or float2 for
    two lines at once); arithmetic goes through the helpers of vec_ops.cuh."""
    ins, ops, outs = prog
    lines = []
    cur = {}
    for n in range(N):
        cur[ins[n]] = (f"v[{n}]", 1)
    tmp = [0]

    def new():
        tmp[0] += 1
        return f"t{tmp[0]}"

    def comb(terms):
        """Expression for sum(coef * sign * name) over two terms."""
        ts = [(coef * sign, name) for coef, (name, sign) in terms if coef * sign != 0.0]
        if not ts:
            return "vzero(v[0])"
        if len(ts) == 1:
            c, a = ts[0]
            if c == 1.0:
                return a
            if c == -1.0:
                return f"vneg({a})"
            return f"vmul({f32(c)}, {a})"
        (c1, a), (c2, b) = ts
        if c1 == 1.0 and c2 == 1.0:
            return f"vadd({a}, {b})"
        if c1 == 1.0 and c2 == -1.0:
            return f"vsub({a}, {b})"
        if c1 == -1.0 and c2 == 1.0:
            return f"vsub({b}, {a})"
        return f"vmac({f32(c1)}, {a}, {f32(c2)}, {b})"

    n_add = n_mat = 0
    for op in ops:
        if op[0] == "add":
            _, i, j = op
            (a, sa), (b, sb) = cur[i], cur[j]
            ts, td = new(), new()
            if sa * sb > 0:
                lines.append(f"    const T {ts} = vadd({a}, {b});")
                lines.append(f"    const T {td} = vsub({a}, {b});")
            else:
                lines.append(f"    const T {ts} = vsub({a}, {b});")
                lines.append(f"    const T {td} = vadd({a}, {b});")
            cur[i], cur[j] = (ts, sa), (td, sa)
            n_add += 1
        elif op[0] == "mat":
            _, i, j, a, b, c, d = op
            x, y = cur[i], cur[j]
            ti, tj = new(), new()
            lines.append(f"    const T {ti} = {comb([(a, x), (b, y)])};")
            lines.append(f"    const T {tj} = {comb([(c, x), (d, y)])};")
            cur[i], cur[j] = (ti, 1), (tj, 1)
            n_mat += 1
        else:
            name, sign = cur[op[1]]
            cur[op[1]] = (name, -sign)
    for k in range(N):
        name, sign = cur[outs[k]]
        lines.append(f"    v[{k}] = {'vneg(' + name + ')' if sign < 0 else name};")
    head = (f"// {CORE_NAMES[core]} N={N}: {n_add} butterflies (2 FADD), {n_mat} rotations "
            f"(2 FMUL + 2 FFMA) = {2 * n_add + 4 * n_mat} FP32 ops, "
            f"{(2 * n_add + 4 * n_mat) / N:.2f} per sample")
    body = "\n".join(lines)
    return (f"{head}\ntemplate <> struct Core<{N}, {core}> {{\n"
            f"  template <class T>\n"
            f"  static __device__ __forceinline__ void apply(T (&v)[{N}]) {{\n{body}\n  }}\n}};\n")


def generate() -> str:
    chunks = [
        "// Generated by gen_cores.py: fast orthonormal DCT-2 / DCT-3 / DST-2 / DST-3 cores.\n"
        "// Do not edit; regenerate with `python gen_cores.py`.\n"
        "#pragma once\n\n"
        "#include \"vec_ops.cuh\"\n\n"
        "template <int N, int CORE> struct Core;\n\n"
    ]
    for N in SIZES:
        for core in range(4):
            prog = core_program(N, core)
            err = np.abs(simulate(N, prog) - definition(N, core)).max()
            if err > 1e-12:
                raise AssertionError(f"graph N={N} core={core} off by {err}")
            chunks.append(emit(N, core, prog) + "\n")
    return "".join(chunks)


def main(argv=None):
    here = os.path.dirname(os.path.abspath(__file__))
    out = os.path.join(here, "cores_gen.cuh")
    text = generate()
    old = open(out).read() if os.path.exists(out) else None
    if old != text:
        with open(out, "w") as f:
            f.write(text)
    return 0


if __name__ == "__main__":
    sys.exit(main(sys.argv[1:]))
