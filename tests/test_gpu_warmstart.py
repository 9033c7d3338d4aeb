"""Learned initial guess: the CUDA network (forward, gradient, Adam) against the numpy reference in
oracle/warmstart_oracle.py, training on solves of the method, and the guarded warm-started solve.
Needs a GB300 (sm_103a).

Tolerances: with FP32 activations every convolution is an FP32 sum of at most 432 products and
the network is 12 convolutions deep, so outputs agree to ~1e-6 relative; gradients (24 more
convolutions) to ~1e-5.  BF16 activations keep 8 significant bits: outputs within a few 1e-2.
"""
import numpy as np
import pytest
import torch

import synthetic
from oracle import warmstart_oracle as wo

pytestmark = pytest.mark.gpu

smg = pytest.importorskip("paper_2312_10615_gb300")
DEV = torch.device("cuda:0")
N = 16


def _vec(n, seed):
    m = (n + 1) * n * n * 3 + n ** 3
    return np.random.default_rng(seed).standard_normal(m)


def _weights(seed, gain=0.5):
    return (synthetic.net_weights(seed) * gain).astype(np.float32)


def _rel(a, b):
    a = a.cpu().numpy() if isinstance(a, torch.Tensor) else a
    return float(np.max(np.abs(a - b)) / np.max(np.abs(b)))


def test_forward_parity_fp32():
    w = _weights(3)
    ws = smg.WarmStart(N, smg.STORE_FP32, scale=0.7)
    ws.set_weights(w)
    b = _vec(N, 1)
    x0 = ws.predict(torch.from_numpy(b).to(DEV))
    ref = wo.predict(b, w.astype(np.float64), N, 0.7)
    assert _rel(x0, ref) < 1e-5
    ws.close()


def test_loss_and_gradient_parity_fp32():
    w = _weights(4)
    ws = smg.WarmStart(N, smg.STORE_FP32, scale=0.7)
    ws.set_weights(w)
    b, xs = _vec(N, 2), _vec(N, 3)
    loss, g = ws.loss_grad(torch.from_numpy(b).to(DEV), torch.from_numpy(xs).to(DEV), want_grad=True)
    L, G = wo.loss_and_grad(b, xs, w.astype(np.float64), N, 0.7)
    assert abs(loss - L) < 1e-5 * L
    assert _rel(g, G) < 1e-4
    # per weight tensor as well, so that a small layer cannot hide behind a large one
    off = 0
    for shp in wo.SHAPES:
        m = shp[0] * shp[1] * shp[2]
        assert _rel(g[off:off + m], G[off:off + m]) < 1e-3, shp
        off += m
    ws.close()


def test_residual_form_loss_and_gradient_parity_fp32():
    import oracle
    o = oracle.Oracle(N, coarsest_max=8)
    act, _ = o.masks()
    S = smg.Stokes(N)
    w = _weights(9)
    ws = smg.WarmStart(N, smg.STORE_FP32, scale=0.7)
    ws.set_weights(w)
    b, xs = _vec(N, 8), _vec(N, 9)
    b[~act] = 0.0
    xs[~act] = 0.0
    loss, g = ws.loss_grad(torch.from_numpy(b).to(DEV), torch.from_numpy(xs).to(DEV), S=S, want_grad=True)
    L, G = wo.loss_and_grad(b, xs, w.astype(np.float64), N, 0.7, apply=o.apply)
    assert abs(loss - L) < 1e-5 * L
    assert _rel(g, G) < 1e-4
    ws.close()
    S.close()


def test_bf16_activations_close():
    w = _weights(5)
    b, xs = _vec(N, 4), _vec(N, 5)
    ws = smg.WarmStart(N, smg.STORE_BF16, scale=0.7)
    ws.set_weights(w)
    x0 = ws.predict(torch.from_numpy(b).to(DEV))
    ref = wo.predict(b, w.astype(np.float64), N, 0.7)
    assert _rel(x0, ref) < 5e-2
    _, g = ws.loss_grad(torch.from_numpy(b).to(DEV), torch.from_numpy(xs).to(DEV), want_grad=True)
    _, G = wo.loss_and_grad(b, xs, w.astype(np.float64), N, 0.7)
    cos = float(g.astype(np.float64) @ G / (np.linalg.norm(g) * np.linalg.norm(G)))
    assert cos > 0.99
    ws.close()


def test_adam_step_parity():
    w = _weights(6)
    ws = smg.WarmStart(N, smg.STORE_FP32, scale=0.7)
    ws.set_weights(w)
    b, xs = _vec(N, 6), _vec(N, 7)
    _, g = ws.loss_grad(torch.from_numpy(b).to(DEV), torch.from_numpy(xs).to(DEV), want_grad=True)
    ws.adam_step(1e-3)
    torch.cuda.synchronize()
    got = ws.get_weights()
    ref = wo.adam(w.astype(np.float64), g.astype(np.float64), np.zeros(w.size), np.zeros(w.size), 1, 1e-3)
    assert np.max(np.abs(got - ref)) < 1e-6
    ws.close()


def _solved(n, seeds):
    S = smg.Stokes(n, precision=smg.PREC_FP32)
    data = []
    for sd in seeds:
        b = S.rhs(synthetic.bumps(n, seed=sd, nbumps=8, device=DEV)["f"], None)
        x, info = S.solve(b, tol=1e-10)
        assert info.status == 0
        data.append((b, x))
    return S, data


def test_training_on_solves_reduces_loss():
    S, data = _solved(N, range(100, 106))
    scale = float(np.mean([float(x.norm() / b.norm()) for b, x in data]))
    ws = smg.WarmStart(N, smg.STORE_BF16, scale=scale)
    ws.set_weights(_weights(7, gain=1.0))
    first = np.mean([ws.loss_grad(b, x)[0] for b, x in data])
    for step in range(300):
        b, x = data[step % len(data)]
        ws.train_step(b, x, lr=2e-3)
    last = np.mean([ws.loss_grad(b, x)[0] for b, x in data])
    assert last < 0.5 * first, (first, last)
    ws.close()
    S.close()


def test_warmstart_solve_guard_and_tolerance():
    S, data = _solved(N, [200])
    b, xref = data[0]
    ws = smg.WarmStart(N, smg.STORE_FP32, scale=1.0)
    ws.set_weights(np.zeros(smg.warmstart_num_weights(), dtype=np.float32))
    # a zero network predicts x0 = 0: tau_0 = ||M b|| is not a reduction, the guess is discarded
    x, info, used = ws.solve(S, b, tol=1e-8)
    assert not used and info.status == 0
    x_plain, info_plain = S.solve(b, tol=1e-8)
    assert info.iterations == info_plain.iterations
    assert float(torch.max(torch.abs(x - x_plain))) == 0.0
    # with an untrained network, whatever guess it returns, the solve meets the tolerance
    ws.set_weights(_weights(8))
    x, info, used = ws.solve(S, b, tol=1e-8)
    assert info.status == 0 and info.rel_residual < 1e-8
    assert S.residual_norm(b, x) / float(b.norm()) < 1e-8
    # a perfect guess (the method's own solution, here passed straight to SQMR) needs fewer iterations
    x = xref.clone()
    info_exact = smg.sqmr_solve(S.h, b, x, 1e-8, 200)
    assert info_exact.iterations < info_plain.iterations
    ws.close()
    S.close()


def test_invalid_sizes_rejected():
    with pytest.raises(smg.StokesError):
        smg.WarmStart(12)  # not a multiple of 8
    ws = smg.WarmStart(N)
    with pytest.raises(smg.StokesError):
        ws.predict(torch.zeros(10, dtype=torch.float64))  # host tensor
    ws.close()


def test_trained_network_on_held_out_seeds():
    """Train the BF16 network (tensor-core convolutions) on the method's own solves of 64^3 bump problems,
    then solve held-out seeds from the learned x0 and from x0 = 0 with the same handle and tolerance,
    and compare mean iterations and time (the same recipe as the bench's initial-guess mode, smaller)"""
    import time
    n, ntrain, ntest = 64, 240, 40
    S = smg.Stokes(n, precision=smg.PREC_FP32)
    seeds = [30000 + i for i in range(ntrain + ntest)]

    def rhs(sd):
        return S.rhs(synthetic.bumps(n, seed=sd, nbumps=8, device=DEV)["f"], None)

    xs, its0 = [], []
    for sd in seeds:
        b = rhs(sd)
        x = torch.zeros_like(b)
        info = smg.sqmr_solve(S.h, b, x, 1e-8, 200)
        assert info.status == 0
        its0.append(info.iterations)
        xs.append(x.float())
    scale = float(np.median([float(xs[i].double().norm() / rhs(seeds[i]).norm()) for i in range(32)]))
    ws = smg.WarmStart(n, smg.STORE_BF16, scale=scale)
    w = synthetic.net_weights(7).astype(np.float32)
    w[-16 * 4:] = 0.0  # output layer 0: training starts from x0 = 0
    ws.set_weights(w)
    rng = np.random.default_rng(5)
    steps = 2 * ntrain
    for st in range(steps):
        i = int(rng.integers(ntrain))
        ws.train_step(rhs(seeds[i]), xs[i].double(), 1e-3 * 0.5 * (1 + np.cos(np.pi * st / steps)))
    loss = np.mean([ws.loss_grad(rhs(seeds[ntrain + k]), xs[ntrain + k].double())[0] for k in range(ntest)])
    rows = []
    for k in range(ntest):
        b = rhs(seeds[ntrain + k])
        x = torch.zeros_like(b)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        info0 = smg.sqmr_solve(S.h, b, x, 1e-8, 200)
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        _, infow, used = ws.solve(S, b, tol=1e-8)
        torch.cuda.synchronize()
        t2 = time.perf_counter()
        assert info0.status == 0 and infow.status == 0 and infow.rel_residual < 1e-8
        rows.append((info0.iterations, t1 - t0, infow.iterations, t2 - t1, used))
    r = np.array(rows, dtype=np.float64)
    it0, itw = r[:, 0].mean(), r[:, 2].mean()
    ms0, msw = 1e3 * r[:, 1].mean(), 1e3 * r[:, 3].mean()
    print(f"held-out {n}^3 x{ntest}: x0 = 0 {it0:.2f} it {ms0:.2f} ms; learned x0 {itw:.2f} it {msw:.2f} ms; "
          f"guess used {r[:, 4].mean():.2f}; error-form loss {loss:.3f}")
    assert loss < 1.0          # the network learned a guess closer to x* than x0 = 0
    assert itw <= it0 + 0.25   # and starting from it never costs iterations on average
    ws.close()
    S.close()
