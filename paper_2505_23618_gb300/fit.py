"""Gradient fit of the adjustment parameters (the design step of Eq. 2, driven by the GPU
backward kernel).

Loss (per fitted 1-D transform H of length N, used both horizontally and vertically):
    L = sum_{k<M} |h_k - d_k|^2  +  lam * P(H),
where h_k, d_k are the first M basis vectors (rows) of H and of the target D (DST-7), and
P is the coding-gain proxy of the 2-D coefficients of synthetic AR(1) blocks,
(1/N^2) sum_{kv,kh} log mean_b Y_b[kv,kh]^2.  Optionally the paper's weighted criterion of
Eq. 2 replaces the first term: sum_{i,j} e^{-alpha i} (H_ij - D_ij)^2, alpha = ln(100)/N.

Parameterisations (orthogonality by construction, Section 2 after Eq. 2):
    band  H = B A(theta), A a product of Givens layers; theta are the free parameters;
    post  H = diag(Q, I) B with Q = Dg (I + W)^{-1} (I - W), W skew-symmetric (the Cayley
          map; Dg a fixed +-1 diagonal taken from the start point, since the Cayley map only
          reaches det = +1 without an eigenvalue -1).

The GPU does the per-block work (forward of every block, the proxy and its gradient, the
backward into dL/dtheta or dL/dQ); the host keeps the N x N FP64 model of H for the basis
term, the Cayley map and Adam.
"""

from __future__ import annotations

import ctypes as C
import json
import math
import os
from dataclasses import dataclass, field

import numpy as np

from . import _lib, targets


# ---------------------------------------------------------------------------------------
# FP64 host model of one direction's H and of its parameter gradients.
# ---------------------------------------------------------------------------------------

def _layer_pairs(n, parity):
    return [(i, i + 1) for i in range(int(parity), n - 1, 2)]


def _rot_layer(n, parity, angles):
    G = np.eye(n)
    for (i, j), th in zip(_layer_pairs(n, parity), angles):
        c, s = math.cos(th), math.sin(th)
        G[i, i], G[i, j], G[j, i], G[j, j] = c, -s, s, c
    return G


def band_layers(n, parities, angles):
    out, pos = [], 0
    for p in parities:
        cnt = len(_layer_pairs(n, p))
        out.append(_rot_layer(n, p, angles[pos:pos + cnt]))
        pos += cnt
    return out


def band_H(n, core, parities, angles):
    A = np.eye(n)
    for G in band_layers(n, parities, angles):
        A = G @ A
    return targets.core(n, core) @ A


def band_angle_grad(n, core, parities, angles, dH):
    """dL/dtheta for H = B G_{L-1}...G_0 from dL/dH (FP64, by the product rule per layer)."""
    Gs = band_layers(n, parities, angles)
    dA = targets.core(n, core).T @ dH
    out = np.zeros(len(angles))
    pos = 0
    for l, p in enumerate(parities):
        left = np.eye(n)
        for m in range(len(Gs) - 1, l, -1):
            left = left @ Gs[m]
        right = np.eye(n)
        for m in range(l):
            right = Gs[m] @ right
        M = left.T @ dA @ right.T
        for q, (i, j) in enumerate(_layer_pairs(n, p)):
            c, s = math.cos(angles[pos + q]), math.sin(angles[pos + q])
            out[pos + q] = -s * M[i, i] - c * M[i, j] + c * M[j, i] - s * M[j, j]
        pos += len(_layer_pairs(n, p))
    return out


def skew(w, k):
    W = np.zeros((k, k))
    W[np.triu_indices(k, 1)] = w
    return W - W.T


def cayley_q(w, k, dg):
    W = skew(w, k)
    I = np.eye(k)
    return dg[:, None] * np.linalg.solve(I + W, I - W)


def cayley_grad(w, k, dg, gq):
    W = skew(w, k)
    I = np.eye(k)
    Cq = np.linalg.solve(I + W, I - W)
    M = -np.linalg.solve((I + W).T, dg[:, None] * gq) @ (Cq + I).T
    return (M - M.T)[np.triu_indices(k, 1)]


def cayley_init(q):
    """(w, dg) with Dg Cayley(W) = q for an orthogonal q.

    The Cayley map reaches the orthogonal matrices of determinant +1 without an eigenvalue -1.
    An orthogonal matrix of determinant -1 always has the eigenvalue -1, so the signs Dg are
    chosen to make det(Dg q) = +1: first so that Dg q has a non-negative diagonal (as close to I
    as the diagonal allows), then, if the determinant is still -1, flipping the row whose
    diagonal entry is smallest in magnitude.  (A determinant +1 matrix with the eigenvalue -1,
    a rotation by exactly pi in some plane, is not handled; it does not arise from a generic
    start.)"""
    k = q.shape[0]
    dg = np.where(np.diag(q) < 0, -1.0, 1.0)
    if np.linalg.det(dg[:, None] * q) < 0:
        i = int(np.argmin(np.abs(np.diag(q))))
        dg[i] = -dg[i]
    C0 = dg[:, None] * q
    I = np.eye(k)
    W = np.linalg.solve(I + C0, I - C0)   # inverse Cayley map
    W = 0.5 * (W - W.T)
    return W[np.triu_indices(k, 1)], dg


# ---------------------------------------------------------------------------------------
# The fit.
# ---------------------------------------------------------------------------------------

@dataclass
class FitConfig:
    n: int = 64
    core: int = 0                 # 0 DCT-2, 1 DCT-3, 2 DST-2, 3 DST-3
    kind: int = 1                 # 1 band, 2 post
    parities: tuple = (0, 1) * 6  # band layers
    k: int = 32                   # post block size
    target: str = "dst7"
    m: int = 16                   # basis vectors matched
    lam: float = 0.1              # weight of the coding-gain proxy
    eq2: bool = False             # use the paper's weighted criterion (Eq. 2) instead
    blocks: int = 65536
    rho: float = 0.95
    sigma: float = 40.0
    seed: int = 4
    steps: int = 200
    lr: float = 0.01
    history: list = field(default_factory=list)


class Fitter:
    """Fits one 1-D adjusted transform on the GPU (one plan, blocks of n x n)."""

    def __init__(self, cfg: FitConfig, data=None, device=None):
        import torch

        self.cfg = cfg
        self.torch = torch
        self.dev = torch.device(device or "cuda")
        n = cfg.n
        self.D = {"dst7": targets.dst7, "dct8": targets.dct8}[cfg.target](n)
        if data is None:
            import synth
            rng = np.random.default_rng(cfg.seed)
            data = synth.ar1_blocks(rng, cfg.blocks, n, n, cfg.rho, cfg.rho, cfg.sigma, 255).reshape(-1)
        self.nb = data.size // (n * n)
        self.x = torch.from_numpy(np.ascontiguousarray(data)).to(self.dev)
        blocks = np.zeros(self.nb, dtype=_lib.BLOCK_DTYPE)
        blocks["offset"] = np.arange(self.nb, dtype=np.int64) * n * n
        blocks["w"] = blocks["h"] = n
        if cfg.kind == 1:
            self.theta = np.zeros(sum(len(_layer_pairs(n, p)) for p in cfg.parities))
        else:
            B = targets.core(n, cfg.core)
            # start from the orthogonal Procrustes fit of the K x K block: Q = U V^T of D_K B_K^T
            u, _, vt = np.linalg.svd(self.D[:cfg.k, :] @ B[:cfg.k, :].T)
            self.w, self.dg = cayley_init(u @ vt)
        self.plan = _lib.Plan([self._tf()])
        self.plan.set_blocks(blocks, data.size)
        self.lay = self.plan.param_layout()
        self.y = torch.empty(data.size, dtype=torch.float32, device=self.dev)
        self.gy = torch.empty_like(self.y)
        self.gp = torch.zeros(max(1, self.lay[-1]), dtype=torch.float32, device=self.dev)
        self.work = torch.zeros(65 * n * n, dtype=torch.float64, device=self.dev)
        self.loss_dev = torch.zeros(1, dtype=torch.float64, device=self.dev)
        self.m1 = self.m2 = None
        self.t = 0

    # current transform -------------------------------------------------------------
    def q(self):
        return cayley_q(self.w, self.cfg.k, self.dg)

    def _tf(self):
        c = self.cfg
        if c.kind == 1:
            return {"n": c.n, "core": c.core, "kind": 1, "parities": np.array(c.parities, np.uint8),
                    "angles": self.theta}
        return {"n": c.n, "core": c.core, "kind": 2, "q": self.q()}

    def H(self):
        c = self.cfg
        if c.kind == 1:
            return band_H(c.n, c.core, c.parities, self.theta)
        C = np.eye(c.n)
        C[:c.k, :c.k] = self.q()
        return C @ targets.core(c.n, c.core)

    # loss and gradient -------------------------------------------------------------
    def basis_term(self):
        c = self.cfg
        H = self.H()
        if c.eq2:
            wts = np.exp(-math.log(100.0) / c.n * np.arange(c.n))[:, None]
            diff = H - self.D
            return float(np.sum(wts * diff ** 2)), 2.0 * wts * diff
        diff = np.zeros_like(H)
        diff[:c.m] = H[:c.m] - self.D[:c.m]
        return float(np.sum(diff ** 2)), 2.0 * diff

    def loss_and_grad(self):
        """Loss and gradient w.r.t. the free parameters (theta, or the Cayley w)."""
        c = self.cfg
        torch = self.torch
        lib = self.plan._lib
        stream = torch.cuda.current_stream(self.dev)
        self.plan.update_params([self._tf()])
        self.plan.fwd(self.x, self.y, stream)
        n2 = c.n * c.n
        _lib.check(lib.adj_coding_gain_proxy(self.y.data_ptr(), self.nb, n2, self.work.data_ptr(),
                                             self.loss_dev.data_ptr(), self.gy.data_ptr(), stream.cuda_stream))
        # the backward is linear in dL/dY: the proxy gradient is scaled by lam on the host
        self.plan.bwd(self.x, self.gy, None, self.gp, stream)
        torch.cuda.synchronize(self.dev)
        proxy = float(self.loss_dev.item())
        g_proxy = self.gp[self.lay[0]:self.lay[1]].double().cpu().numpy()
        basis, dH = self.basis_term()
        loss = basis + c.lam * proxy
        if c.kind == 1:
            g = band_angle_grad(c.n, c.core, c.parities, self.theta, dH) + c.lam * g_proxy
        else:
            B = targets.core(c.n, c.core)
            gq = (dH @ B.T)[:c.k, :c.k] + c.lam * g_proxy.reshape(c.k, c.k)
            g = cayley_grad(self.w, c.k, self.dg, gq)
        return loss, basis, proxy, g

    def params(self):
        return self.theta if self.cfg.kind == 1 else self.w

    def set_params(self, v):
        if self.cfg.kind == 1:
            self.theta = np.asarray(v, dtype=np.float64)
        else:
            self.w = np.asarray(v, dtype=np.float64)

    def step(self):
        """One Adam step; returns the loss before it."""
        loss, basis, proxy, g = self.loss_and_grad()
        b1, b2, eps = 0.9, 0.999, 1e-12
        if self.m1 is None:
            self.m1 = np.zeros_like(g)
            self.m2 = np.zeros_like(g)
        self.t += 1
        self.m1 = b1 * self.m1 + (1 - b1) * g
        self.m2 = b2 * self.m2 + (1 - b2) * g * g
        mh = self.m1 / (1 - b1 ** self.t)
        vh = self.m2 / (1 - b2 ** self.t)
        self.set_params(self.params() - self.cfg.lr * mh / (np.sqrt(vh) + eps))
        self.cfg.history.append({"step": self.t, "loss": loss, "basis": basis, "proxy": proxy,
                                 "grad_norm": float(np.linalg.norm(g))})
        return loss

    def run(self, steps=None, log_every=0):
        for i in range(steps or self.cfg.steps):
            loss = self.step()
            if log_every and (i % log_every == 0):
                print(f"step {self.t:4d} loss {loss:.6f}", flush=True)
        return self.loss_and_grad()[0]

    # checkpoint ------------------------------------------------------------------
    def state(self):
        c = self.cfg
        d = {"config": {k: getattr(c, k) for k in ("n", "core", "kind", "parities", "k", "target", "m", "lam",
                                                   "eq2", "blocks", "rho", "sigma", "seed", "lr")},
             "step": self.t, "params": self.params().tolist(),
             "adam": None if self.m1 is None else [self.m1.tolist(), self.m2.tolist()]}
        if c.kind == 2:
            d["dg"] = self.dg.tolist()
            d["q"] = self.q().tolist()
        else:
            d["angles"] = self.theta.tolist()
        d["history"] = c.history
        return d

    def save(self, path):
        os.makedirs(os.path.dirname(os.path.abspath(path)), exist_ok=True)
        with open(path, "w") as f:
            json.dump(self.state(), f)

    def load(self, path):
        with open(path) as f:
            d = json.load(f)
        self.t = d["step"]
        self.set_params(d["params"])
        if self.cfg.kind == 2:
            self.dg = np.array(d["dg"])
        if d.get("adam"):
            self.m1, self.m2 = (np.array(a) for a in d["adam"])
        self.cfg.history = d.get("history", [])

    def close(self):
        self.plan.close()


# ---------------------------------------------------------------------------------------
# The fits of the design step: the DST-7 approximations of the fitting workload (65536
# AR(1) 64x64 blocks, rho 0.95, M = 16) for both parameterisations, and the pairings the
# large-frame workload runs (DST-3 + band; DCT-2 + post at 64 and 32 points, whose DCT-8
# counterpart follows by Eq. 5).
# ---------------------------------------------------------------------------------------

FITS = {
    "band_dct2_64": dict(n=64, core=0, kind=1, parities=(0, 1) * 6),
    "post_dst2_64": dict(n=64, core=2, kind=2, k=32),
    "band_dst3_64": dict(n=64, core=3, kind=1, parities=(0, 1) * 6),
    "post_dct2_64": dict(n=64, core=0, kind=2, k=32),
    "post_dct2_32": dict(n=32, core=0, kind=2, k=16),
}
# The paper's own design criterion (Eq. 2: squared error to the DST-7 weighted by
# e^{-alpha i}, alpha = ln(100)/N, no coding-gain term) for the adjustments of Table 1: a
# 6-tap band (3 layers) before the DST-3 and the 8 x 8 block after the DCT-2, at 16, 32 and
# 64 points.
for _n in (16, 32, 64):
    FITS[f"eq2_band6_dst3_{_n}"] = dict(n=_n, core=3, kind=1, parities=(0, 1, 0), eq2=True, lam=0.0)
    FITS[f"eq2_post8_dct2_{_n}"] = dict(n=_n, core=0, kind=2, k=8, eq2=True, lam=0.0)
DESIGN_FITS = ("band_dct2_64", "post_dst2_64", "band_dst3_64", "post_dct2_64", "post_dct2_32")


def _proxy_of(fitter, tf):
    """Coding-gain proxy of the fitter's blocks under another 1-D transform `tf`."""
    torch = fitter.torch
    with _lib.Plan([tf]) as plan:
        blocks = np.zeros(fitter.nb, dtype=_lib.BLOCK_DTYPE)
        n = fitter.cfg.n
        blocks["offset"] = np.arange(fitter.nb, dtype=np.int64) * n * n
        blocks["w"] = blocks["h"] = n
        plan.set_blocks(blocks, fitter.nb * n * n)
        stream = torch.cuda.current_stream(fitter.dev)
        plan.fwd(fitter.x, fitter.y, stream)
        _lib.check(plan._lib.adj_coding_gain_proxy(fitter.y.data_ptr(), fitter.nb, n * n, fitter.work.data_ptr(),
                                                   fitter.loss_dev.data_ptr(), None, stream.cuda_stream))
        torch.cuda.synchronize(fitter.dev)
        return float(fitter.loss_dev.item())


def run_fit(name, steps, lr=0.01, log_every=0):
    """Runs one named fit; returns its record (parameters, history summary, metrics)."""
    cfg = FitConfig(**FITS[name], steps=steps, lr=lr)
    f = Fitter(cfg)
    n, m = cfg.n, cfg.m
    loss0, basis0, proxy0, _ = f.loss_and_grad()
    wts = np.exp(-math.log(100.0) / n * np.arange(n))[:, None]
    eq2_start = float(np.sum(wts * (f.H() - f.D) ** 2))
    f.run(steps, log_every=log_every)
    loss1, basis1, proxy1, g1 = f.loss_and_grad()
    H = f.H()
    D = f.D
    # coding gains relative to the DCT-2 on the same blocks: (10 / ln 10) (P_DCT2 - P_H)
    p_dct2 = _proxy_of(f, {"n": n, "core": 0, "kind": 0})
    p_core = _proxy_of(f, {"n": n, "core": cfg.core, "kind": 0})
    p_dst7 = _proxy_of(f, targets.dense_tf(D))
    db = 10.0 / math.log(10.0)
    rec = {
        "name": name,
        "config": {k: (list(v) if isinstance(v, tuple) else v) for k, v in FITS[name].items()},
        "criterion": "eq2" if cfg.eq2 else f"basis(M={m}) + lam * proxy",
        "eq2_error": {"start": eq2_start, "final": float(np.sum(wts * (H - D) ** 2))},
        "first_basis_vectors": {"fitted": H[:4].tolist(), "dst7": D[:4].tolist()},
        "target": cfg.target, "m": m, "lam": cfg.lam, "blocks": cfg.blocks, "rho": cfg.rho, "sigma": cfg.sigma,
        "seed": cfg.seed, "steps": steps, "lr": lr,
        "start": {"loss": loss0, "basis": basis0, "proxy": proxy0},
        "final": {"loss": loss1, "basis": basis1, "proxy": proxy1, "grad_norm": float(np.linalg.norm(g1)),
                  "max_abs_basis_dev_first_m": float(np.abs(H[:m] - D[:m]).max())},
        "coding_gain_db_vs_dct2": {"fitted": db * (p_dct2 - proxy1), "core_alone": db * (p_dct2 - p_core),
                                   "exact_dst7": db * (p_dct2 - p_dst7)},
        "history": [cfg.history[i] for i in range(0, len(cfg.history), max(1, len(cfg.history) // 20))],
    }
    if cfg.kind == 1:
        rec["parities"] = list(cfg.parities)
        rec["angles"] = f.theta.tolist()
    else:
        rec["k"] = cfg.k
        rec["q"] = f.q().tolist()
        rec["q_dct8"] = targets.chessboard(f.q()).tolist()
    f.close()
    return rec


def basis_table(rec):
    """Basis vector by basis vector comparison of a stored band fit with the DST-7 it
    approximates (the content of Fig. 3, in numbers): for every row k of the fitted transform
    H = B A, the distance |h_k - d_k|, the inner product <h_k, d_k>, the distance of the core
    B alone, and the weight e^{-alpha k} (alpha = ln(100)/N) that Eq. 2 gives the row.  Host
    FP64 only."""
    n, core = int(rec["config"]["n"]), int(rec["config"]["core"])
    H = band_H(n, core, tuple(rec["parities"]), np.asarray(rec["angles"], dtype=np.float64))
    D = targets.dst7(n)
    B = targets.core(n, core)
    alpha = math.log(100.0) / n
    rows = []
    for k in range(n):
        rows.append({"k": k, "dist": float(np.linalg.norm(H[k] - D[k])), "inner": float(H[k] @ D[k]),
                     "core_dist": float(np.linalg.norm(B[k] - D[k])), "weight": math.exp(-alpha * k)})
    return rows


def basis_table_markdown(rec):
    rows = basis_table(rec)
    out = ["| k | Eq. 2 weight | core alone: |b_k - d_k| | fitted: |h_k - d_k| | <h_k, d_k> |",
           "|---|---|---|---|---|"]
    for r in rows:
        out.append(f"| {r['k']} | {r['weight']:.3f} | {r['core_dist']:.4f} | {r['dist']:.4f} | {r['inner']:.4f} |")
    return "\n".join(out)


def main(argv=None):
    import argparse
    import time
    ap = argparse.ArgumentParser(description="Fit the DST-7 adjustments on the GPU and write them as JSON.")
    ap.add_argument("--basis-table", metavar="FIT", default=None,
                    help="print the basis-vector table of a stored band fit (host only; e.g. "
                         "eq2_band6_dst3_16 from params/fitted_eq2.json) instead of fitting")
    ap.add_argument("--params", default=os.path.join(os.path.dirname(os.path.abspath(__file__)), "params",
                                                     "fitted_eq2.json"),
                    help="stored fits for --basis-table")
    ap.add_argument("--out", help="output JSON file (fitting)")
    ap.add_argument("--steps", type=int, default=400)
    ap.add_argument("--lr", type=float, default=0.01)
    ap.add_argument("--only", nargs="*", default=None,
                    help="names of the fits to run (default: the five design fits; see FITS)")
    a = ap.parse_args(argv)
    if a.basis_table:
        with open(a.params) as fh:
            print(basis_table_markdown(json.load(fh)[a.basis_table]))
        return 0
    if not a.out:
        ap.error("--out is required when fitting")
    out = {}
    for name in (a.only or list(DESIGN_FITS)):
        t0 = time.time()
        rec = run_fit(name, a.steps, a.lr)
        rec["seconds"] = round(time.time() - t0, 2)
        out[name] = rec
        print(json.dumps({k: rec[k] for k in ("name", "start", "final", "eq2_error", "coding_gain_db_vs_dct2",
                                              "seconds")}),
              flush=True)
    os.makedirs(os.path.dirname(os.path.abspath(a.out)), exist_ok=True)
    with open(a.out, "w") as fh:
        json.dump(out, fh)
    return 0


if __name__ == "__main__":
    import sys
    sys.exit(main())
