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

The 64-point cores run as two 32-point cores at once in packed FP32x2 arithmetic
(one thread holds one 64-sample line, and a 32-point graph on float2 values costs the
instructions of one 32-point line).  With a_n = x_n, b_n = x_{63-n} (n < 32):

    u_n = (a_n + b_n) / sqrt(2),   y_n = sqrt(2) cos(pi (2n+1) / 128) (a_n - b_n),
    (U, Y) = DCT2_32 of (u, y), both lanes of one packed pass,
    X_{2k} = U_k,   X_1 = Y_0 / sqrt(2),   X_{2k+1} = Y_k - X_{2k-1}  (k >= 1).

The last line follows from 2 cos(A) cos(B) = cos(A + B) + cos(A - B): the DCT-2 of the
cosine-weighted differences is the sum of neighbouring odd outputs of the DCT-2 of x, so a
prefix chain of 31 subtractions recovers them.  O_k is an alternating sum of k + 1 outputs of
the 32-point core, so their rounding errors add up: at most about 1.5e-6 of the line norm in
FP32, against 2e-7 for the flow graphs (tests/test_cores_fp32.py).  DCT-3 is the transpose
(the chain runs backwards); DST-2 / DST-3 fold the R / S maps into the constants of the first
step and the output (input) order.  The packed cores are emitted as CorePair64 beside the
scalar flow graphs of Core<64, c>; the kernels choose per direction.

The script checks each generated graph, and the structure of the packed 64-point cores, in
FP64 against its own definition of the orthonormal DCT-2 before writing ``cores_gen.cuh``.
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
    ('scale', i, a)          : s_i <- a s_i
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

    def scale(self, i, a):
        self.ops.append(("scale", i, a))


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


def pair64_beta(i):
    return math.sqrt(2.0) * math.cos(math.pi * (2 * i + 1) / 128.0)


def chain_ops():
    """The odd outputs X_{2k+1} = O_k from the second lane Y of the packed 32-point pass:
    O_0 = Y_0 / sqrt(2), O_k = Y_k - O_{k-1}.  Each op is ("scale", k, a): c_k <- a c_k, or
    (d, r, s): c_d <- c_d + s c_r.  (O_k is an alternating sum of Y_0 .. Y_k, so the rounding
    errors of the Y_j add up whatever the order of evaluation; splitting the chain into linked
    blocks measured no more accurate.)"""
    return [("scale", 0, 1.0 / math.sqrt(2.0))] + [(k, k - 1, -1.0) for k in range(1, 32)]


def transposed_chain_ops():
    """The transpose of chain_ops (for DCT-3): the ops in reverse order, c_r <- c_r + s c_d."""
    return [op if op[0] == "scale" else (op[1], op[0], op[2]) for op in reversed(chain_ops())]


def _dct2_64_pair(g):
    """The 64-point DCT-2 as two 32-point DCT-2 graphs (slots 0..31 and 63..32) between a
    first step of 2x2 maps and the chain; returns the output slots."""
    a = 1.0 / math.sqrt(2.0)
    for i in range(32):
        g.mat(i, 63 - i, a, a, pair64_beta(i), -pair64_beta(i))
    ev = _dct2(g, list(range(32)), 1.0)
    od = _dct2(g, [63 - i for i in range(32)], 1.0)
    for op in chain_ops():
        if op[0] == "scale":
            g.scale(od[op[1]], op[2])
        else:
            d, r, sgn = op
            g.mat(od[r], od[d], 1.0, 0.0, sgn, 1.0)
    out = [None] * 64
    out[0::2] = ev
    out[1::2] = od
    return out


def dct2_program(N, pair=False):
    """The DCT-2 graph: the even/odd recursion, or (N = 64, pair) the packed-pair form."""
    g = Graph(N)
    outs = _dct2_64_pair(g) if pair else _dct2(g, list(range(N)), 1.0)
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


def core_program(N, core, pair=False):
    """(input slot of x_n, ops, output slot of y_k) for one of the four cores (pair: the
    packed-pair form of the 64-point cores)."""
    ins, ops, outs, _, _ = dct2_program(N, pair)
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
        elif op[0] == "scale":
            V[op[1]] = op[2] * V[op[1]]
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


def pair64_spec(core):
    """What the packed 64-point code of `core` does (emit_pair64 writes it, simulate_pair64
    runs it).  Forward type (DCT-2, DST-2): z_i = (ca v[ia] + cb v[ib], cc v[ia] + cd v[ib]),
    32-point DCT-2 of both lanes, forward chain on one lane, then v[m] = z[k].lane.  Transpose
    type (DCT-3, DST-3): z_k = (v[ix], v[iy]), backward chain on one lane, 32-point DCT-3 of
    both lanes, then (v[oa], v[ob]) = (ca z.x + cb z.y, cc z.x + cd z.y).  The DST forms keep
    the odd part in lane x, so that the output (input) reversal still pairs neighbouring
    samples in one float2 (vector shared-memory stores and loads need no register moves)."""
    a = 1.0 / math.sqrt(2.0)
    sig = [1.0 if i % 2 == 0 else -1.0 for i in range(32)]
    if core in (0, 2):
        pre, out = [], {}
        for i in range(32):
            b = pair64_beta(i)
            if core == 0:
                pre.append((i, 63 - i, a, a, b, -b))
            else:                                        # S on the input; odd part in lane x
                s = sig[i]
                pre.append((i, 63 - i, s * b, s * b, s * a, -s * a))
        for k in range(32):
            if core == 0:
                out[2 * k], out[2 * k + 1] = (k, "x"), (k, "y")
            else:                                        # R on the output
                out[63 - 2 * k], out[62 - 2 * k] = (k, "y"), (k, "x")
        return {"type": "fwd", "chain": "y" if core == 0 else "x", "pre": pre,
                "out": [out[m] for m in range(64)]}
    inp, post = [], []
    for k in range(32):
        inp.append((2 * k, 2 * k + 1) if core == 1 else (62 - 2 * k, 63 - 2 * k))
    for i in range(32):
        b = pair64_beta(i)
        if core == 1:
            post.append((i, 63 - i, a, b, a, -b))
        else:                                            # R on the input, S on the output
            s = sig[i]
            post.append((i, 63 - i, s * b, s * a, s * b, -s * a))
    return {"type": "inv", "chain": "y" if core == 1 else "x", "inp": inp, "post": post}


def run_chain(c, ops):
    for op in ops:
        if op[0] == "scale":
            c[op[1]] = op[2] * c[op[1]]
        else:
            c[op[0]] = c[op[0]] + op[2] * c[op[1]]


def simulate_pair64(core):
    """FP64 matrix of the packed 64-point code described by pair64_spec(core)."""
    spec = pair64_spec(core)
    a = 1.0 / math.sqrt(2.0)
    X = np.eye(64)
    if spec["type"] == "fwd":
        C = simulate(32, core_program(32, 0))
        z = {"x": np.stack([ca * X[ia] + cb * X[ib] for ia, ib, ca, cb, cc, cd in spec["pre"]]),
             "y": np.stack([cc * X[ia] + cd * X[ib] for ia, ib, ca, cb, cc, cd in spec["pre"]])}
        z = {l: C @ m for l, m in z.items()}
        run_chain(z[spec["chain"]], chain_ops())
        return np.stack([z[lane][k] for k, lane in spec["out"]])
    C = simulate(32, core_program(32, 1))
    z = {"x": np.stack([X[ix] for ix, iy in spec["inp"]]), "y": np.stack([X[iy] for ix, iy in spec["inp"]])}
    run_chain(z[spec["chain"]], transposed_chain_ops())
    zx, zy = C @ z["x"], C @ z["y"]
    V = np.zeros((64, 64))
    for i, (oa, ob, ca, cb, cc, cd) in enumerate(spec["post"]):
        V[oa] = ca * zx[i] + cb * zy[i]
        V[ob] = cc * zx[i] + cd * zy[i]
    return V


def f32(x):
    v = float(np.float32(x))
    return "%.9ef" % v


def emit_chain(lane, ops):
    out = []
    for op in ops:
        if op[0] == "scale":
            out.append(f"    z[{op[1]}].{lane} = {f32(op[2])} * z[{op[1]}].{lane};")
        else:
            d, r, sgn = op
            out.append(f"    z[{d}].{lane} = z[{d}].{lane} {'+' if sgn > 0 else '-'} z[{r}].{lane};")
    return out


def emit_pair64(core, inner_counts):
    """Packed FP32x2 code of a 64-point core (see pair64_spec)."""
    spec = pair64_spec(core)
    nb, nr = inner_counts
    a = 1.0 / math.sqrt(2.0)
    lines = ["    static_assert(sizeof(T) == sizeof(float), \"64-sample lines are one per thread\");",
             "    float2 z[32];"]
    if spec["type"] == "fwd":
        for i, (ia, ib, ca, cb, cc, cd) in enumerate(spec["pre"]):
            lines.append(f"    z[{i}] = vpre2(v[{ia}], v[{ib}], make_float2({f32(ca)}, {f32(cc)}), "
                         f"make_float2({f32(cb)}, {f32(cd)}));")
        lines.append("    Core<32, 0>::apply(z);")
        lines += emit_chain(spec["chain"], chain_ops())
        for m, (k, lane) in enumerate(spec["out"]):
            lines.append(f"    v[{m}] = z[{k}].{lane};")
        name = "first step"
    else:
        for k, (ix, iy) in enumerate(spec["inp"]):
            lines.append(f"    z[{k}] = make_float2(v[{ix}], v[{iy}]);")
        lines += emit_chain(spec["chain"], transposed_chain_ops())
        lines.append("    Core<32, 1>::apply(z);")
        for i, (oa, ob, ca, cb, cc, cd) in enumerate(spec["post"]):
            lines.append(f"    {{ const float2 r = vpre2(z[{i}].x, z[{i}].y, make_float2({f32(ca)}, {f32(cc)}), "
                         f"make_float2({f32(cb)}, {f32(cd)})); v[{oa}] = r.x; v[{ob}] = r.y; }}")
        name = "last step"
    nc = len(chain_ops())
    n_ins = 2 * nb + 4 * nr + 64 + nc
    flops = 2 * (2 * nb + 6 * nr) + 6 * 32 + nc
    head = (f"// {CORE_NAMES[core]} N=64 packed: two 32-point lines in FP32x2 ({nb} butterflies (2 FADD), "
            f"{nr} rotations (2 FMUL + 2 FFMA) on float2), 32 {name} maps (FP32x2 FMUL + FFMA), "
            f"{nc} chain ops = {n_ins} instructions, {flops} FP32 ops")
    body = "\n".join(lines)
    return (f"{head}\ntemplate <> struct CorePair64<{core}> {{\n"
            f"  template <class T>\n"
            f"  static __device__ __forceinline__ void apply(T (&v)[64]) {{\n{body}\n  }}\n}};\n")


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
        "template <int N, int CORE> struct Core;\n"
        "template <int CORE> struct CorePair64;\n\n"
    ]
    inner = None
    for N in SIZES:
        for core in range(4):
            prog = core_program(N, core)
            err = np.abs(simulate(N, prog) - definition(N, core)).max()
            if err > 1e-12:
                raise AssertionError(f"graph N={N} core={core} off by {err}")
            chunks.append(emit(N, core, prog) + "\n")
            if N == 32 and core == 0:
                ops = prog[1]
                inner = (sum(op[0] == "add" for op in ops), sum(op[0] == "mat" for op in ops))
    for core in range(4):
        for err in (np.abs(simulate(64, core_program(64, core, pair=True)) - definition(64, core)).max(),
                    np.abs(simulate_pair64(core) - definition(64, core)).max()):
            if err > 1e-12:
                raise AssertionError(f"packed 64-point core {core} off by {err}")
        chunks.append(emit_pair64(core, inner) + "\n")
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
