"""Pins of the oracle's analytic gradients by central finite differences (FP64),
and by closed forms where one exists."""

import math

import numpy as np
import pytest

import oracle as O
import synth


def fd(f, x, h):
    x = np.array(x, dtype=np.float64)
    g = np.zeros_like(x)
    for i in range(x.size):
        xp, xm = x.copy(), x.copy()
        xp.flat[i] += h
        xm.flat[i] -= h
        # 4th-order central difference (Richardson of two step sizes)
        xpp, xmm = x.copy(), x.copy()
        xpp.flat[i] += 2 * h
        xmm.flat[i] -= 2 * h
        g.flat[i] = (8 * (f(xp) - f(xm)) - (f(xpp) - f(xmm))) / (12 * h)
    return g


def rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def test_grad_2d_matches_fd_and_closed_form():
    rng = np.random.default_rng(0)
    h, w, nb = 4, 8, 3
    X = rng.standard_normal((nb, h, w))
    R = rng.standard_normal((nb, h, w))
    Hh = O.adjusted_matrix(w, 3, 1, [0, 1], rng.uniform(-1, 1, 7))
    Hv = O.adjusted_matrix(h, 0, 2, Q=synth.haar_orthogonal(rng, 2))
    # linear loss L = <R, Y>: dL/dX is the inverse transform of R (closed form)
    gX, dHh, dHv = O.grad_2d(X, R, Hh, Hv)
    assert np.abs(gX - O.inverse_2d(R, Hh, Hv)).max() < 1e-12
    f_h = lambda m: float(np.sum(R * O.forward_2d(X, m.reshape(w, w), Hv)))
    f_v = lambda m: float(np.sum(R * O.forward_2d(X, Hh, m.reshape(h, h))))
    assert rel(dHh, fd(f_h, Hh.ravel(), 1e-3).reshape(w, w)) < 1e-10
    assert rel(dHv, fd(f_v, Hv.ravel(), 1e-3).reshape(h, h)) < 1e-10


@pytest.mark.parametrize("N,par", [(8, [0, 1]), (16, [1, 0, 1]), (64, [0, 1] * 6)])
def test_grad_band_angles_fd(N, par):
    rng = np.random.default_rng(N)
    cnt = sum(synth.n_pairs(N, p) for p in par)
    ang = rng.uniform(-0.5, 0.5, cnt)
    core = 2
    dH = rng.standard_normal((N, N))
    f = lambda a: float(np.sum(dH * O.adjusted_matrix(N, core, 1, par, a)))
    g = O.grad_band_angles(N, core, par, ang, dH)
    assert rel(g, fd(f, ang, 1e-3)) < 1e-8


def test_grad_post_and_cayley_fd():
    rng = np.random.default_rng(5)
    N, K = 16, 8
    w = rng.uniform(-0.3, 0.3, K * (K - 1) // 2)
    Dg = np.where(rng.random(K) < 0.5, -1.0, 1.0)
    dH = rng.standard_normal((N, N))
    Q = O.cayley(w, K, Dg)
    assert np.abs(Q.T @ Q - np.eye(K)).max() < 1e-12
    assert abs(np.linalg.det(Q) - np.prod(Dg)) < 1e-10
    gq = O.grad_post_q(N, 0, K, dH)
    fq = lambda q: float(np.sum(dH * (O.post_matrix(N, q.reshape(K, K)) @ O.dct2(N))))
    assert rel(gq, fd(fq, Q.ravel(), 1e-3).reshape(K, K)) < 1e-10
    gw = O.cayley_grad(w, K, gq, Dg)
    fw = lambda p: float(np.sum(dH * (O.post_matrix(N, O.cayley(p, K, Dg)) @ O.dct2(N))))
    assert rel(gw, fd(fw, w, 1e-4)) < 1e-8


def test_cayley_small_closed_form():
    # K = 2: W = [[0, a], [-a, 0]] gives (1/(1+a^2)) [[1-a^2, -2a], [2a, 1-a^2]],
    # the rotation by t = 2 atan(a)
    a = 0.37
    Q = O.cayley([a], 2)
    t = 2 * math.atan(a)
    assert np.abs(Q - np.array([[math.cos(t), -math.sin(t)], [math.sin(t), math.cos(t)]])).max() < 1e-14


def test_losses_fd():
    rng = np.random.default_rng(9)
    N = 8
    H = O.dct2(N)
    D = O.dst7(N)
    L, G = O.basis_loss(H, D, 3)
    assert L == pytest.approx(float(np.sum((H[:3] - D[:3]) ** 2)))
    assert rel(G, fd(lambda m: O.basis_loss(m.reshape(N, N), D, 3)[0], H.ravel(), 1e-4).reshape(N, N)) < 1e-9
    Y = rng.standard_normal((6, 4, 4))
    Lp, Gp = O.proxy_loss(Y)
    assert rel(Gp, fd(lambda y: O.proxy_loss(y.reshape(6, 4, 4))[0], Y.ravel(), 1e-5).reshape(6, 4, 4)) < 1e-7
    # minimised by the KLT: for independent coefficients, an orthogonal mixing raises it
    Z = rng.standard_normal((4000, 2, 2)) * np.array([[3.0, 1.0], [0.5, 0.2]])
    R = np.array([[math.cos(0.4), -math.sin(0.4)], [math.sin(0.4), math.cos(0.4)]])
    assert O.proxy_loss(Z)[0] < O.proxy_loss(R @ Z)[0]
