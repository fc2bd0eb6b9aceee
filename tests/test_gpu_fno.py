"""Learned warm start on the GPU against the oracle's network (include/fh_fno.h).

The oracle evaluates the same network in float64 from the bfloat16-rounded
parameters the GPU uses; the GPU computes in float32. Tolerances follow from
float32 rounding through about 15 chained contractions of up to 128 terms
(relative error of order 1e-6, amplified at most a few-fold by the layers):
prediction 1e-4 max-relative per component field, loss 1e-5 relative,
gradient 1e-3 max-relative per parameter block (the block gradients are sums
over every voxel of the batch), Adam 1e-6.

* forward pass and loss on a 24 x 32 x 24 grid, two cells;
* gradient of the loss with respect to every parameter block;
* one Adam step against the oracle's formula;
* the training target (F - Fbar)/s and the warm start Fbar + G(s q):
  compatible, with voxel mean Fbar, and a solve from it reaching the same
  homogenized stress as the solve from Fbar;
* a few Adam steps on a fixed batch lower the loss.
"""

import math

import numpy as np
import pytest
import torch

from gpu_helpers import dev, host, require_gpu
from oracle import fno as ofno
from oracle import spectral
from rve_inputs import random_spheres, two_phase_table

pytestmark = pytest.mark.gpu

SHAPE = (24, 32, 24)


@pytest.fixture(scope="module")
def fh():
    require_gpu()
    import paper_2408_03804_gb300 as fh

    return fh


def _theta(seed, spectral_scale=0.02):
    g = torch.Generator().manual_seed(seed)
    th = torch.empty(ofno.n_params(), dtype=torch.float32)
    o = 0
    for name, shape in ofno.layout():
        k = math.prod(shape)
        sc = spectral_scale if name.startswith("W") else 1.0 / math.sqrt(shape[-1])
        th[o:o + k] = (2 * torch.rand(k, generator=g) - 1) * sc
        o += k
    return th


def _bf16(th):
    return th.to(torch.bfloat16).to(torch.float64)


def _cells(seed, B, shape=SHAPE):
    rng = np.random.default_rng(seed)
    phases = [(rng.uniform(size=shape) < 0.3).astype(np.uint8) for _ in range(B)]
    Fbar = np.zeros((B, 9))
    for b in range(B):
        d = rng.uniform(-1, 1, 9)
        Fbar[b] = np.eye(3).reshape(9) + 0.05 * d / np.linalg.norm(d)
    return phases, Fbar


def _blocks():
    o = 0
    for name, shape in ofno.layout():
        k = math.prod(shape)
        yield name, o, k
        o += k


def test_forward_and_loss_match_oracle(fh):
    th = _theta(1)
    phases, Fbar = _cells(2, 2)
    rng = np.random.default_rng(3)
    targets = [rng.normal(size=(9,) + SHAPE).astype(np.float32) for _ in range(2)]
    with fh.Fno(*SHAPE, max_batch=2, train=True) as net:
        net.set_params(th.cuda())
        q = [torch.empty((9,) + SHAPE, dtype=torch.float32, device="cuda") for _ in range(2)]
        ph = [dev(p) for p in phases]  # must outlive the backward pass
        net.forward(ph, Fbar, q)
        L = net.loss_grad([dev(t) for t in targets])
        qg = np.stack([host(x) for x in q])
    phi = torch.as_tensor(np.stack(phases).astype(np.float64))
    qr, _ = ofno.forward(_bf16(th), phi, torch.as_tensor(Fbar))
    qr = qr.numpy()
    for b in range(2):
        for c in range(9):
            assert np.abs(qg[b, c] - qr[b, c]).max() <= 1e-4 * np.abs(qr[b, c]).max(), (b, c)
    Lr = float(ofno.loss(_bf16(th), phi, torch.as_tensor(Fbar), torch.as_tensor(np.stack(targets), dtype=torch.float64)))
    assert abs(L - Lr) <= 1e-5 * Lr


def test_gradient_matches_oracle(fh):
    th = _theta(4)
    phases, Fbar = _cells(5, 2)
    rng = np.random.default_rng(6)
    targets = [rng.normal(size=(9,) + SHAPE).astype(np.float32) * 0.5 for _ in range(2)]
    with fh.Fno(*SHAPE, max_batch=2, train=True) as net:
        net.set_params(th.cuda())
        ph = [dev(p) for p in phases]  # must outlive the backward pass
        net.forward(ph, Fbar)
        grad = torch.empty(ofno.n_params(), dtype=torch.float32, device="cuda")
        net.loss_grad([dev(t) for t in targets], grad)
        g = host(grad).astype(np.float64)
    phi = torch.as_tensor(np.stack(phases).astype(np.float64))
    _, gr = ofno.loss_and_grad(_bf16(th), phi, torch.as_tensor(Fbar),
                               torch.as_tensor(np.stack(targets), dtype=torch.float64))
    gr = gr.numpy()
    bad = []
    for name, o, k in _blocks():
        ref = gr[o:o + k]
        err = np.abs(g[o:o + k] - ref).max()
        if not err <= 1e-3 * np.abs(ref).max() + 1e-12:
            bad.append((name, float(err), float(np.abs(ref).max())))
    assert not bad, bad


def test_adam_step_matches_oracle(fh):
    n = ofno.n_params()
    rng = np.random.default_rng(9)
    th = rng.normal(size=n).astype(np.float32)
    g = (rng.normal(size=n) * 1e-2).astype(np.float32)
    m = (rng.normal(size=n) * 1e-3).astype(np.float32)
    v = (rng.uniform(size=n) * 1e-4).astype(np.float32)
    ref = ofno.adam_step(th.astype(np.float64), g.astype(np.float64), m.astype(np.float64), v.astype(np.float64),
                         7, 1e-3, 0.9, 0.999, 1e-8, 1e-4)
    with fh.Fno(*SHAPE, max_batch=1) as net:
        T, G, M, V = (torch.as_tensor(a).cuda() for a in (th, g, m, v))
        net.adam(T, G, M, V, 7, 1e-3, 0.9, 0.999, 1e-8, 1e-4)
        out = (host(T), host(M), host(V))
    for a, b in zip(out, ref):
        assert np.abs(a - b).max() <= 1e-6 * np.abs(b).max()


def test_target_and_warm_start(fh):
    n = 32
    shape = (n, n, n)
    phase = random_spheres(n, seed=7, r_min=2.0, r_max=4.0)
    params = two_phase_table(1.5, 1.0, 10.0)
    rng = np.random.default_rng(10)
    d = rng.uniform(-1, 1, 9)
    Fbar = np.eye(3).reshape(9) + 0.04 * d / np.linalg.norm(d)
    th = _theta(11, spectral_scale=0.005)
    opts = fh.default_options(newton_tol=1e-10)
    with fh.Context(*shape) as ctx, fh.Fno(*shape, max_batch=1) as net:
        net.set_params(th.cuda())
        mat = fh.Material(1, phase, params)
        F0 = torch.zeros((9,) + shape, dtype=torch.float64, device="cuda")
        p0, st0, _ = ctx.fft_homog_solve(mat, Fbar, F0, options=opts)
        tgt = torch.empty((9,) + shape, dtype=torch.float32, device="cuda")
        net.make_target(F0, Fbar, tgt)
        Fw = torch.empty_like(F0)
        net.warm_start(ctx, dev(phase), Fbar, Fw)
        Fw_h = host(Fw)
        p1, st1, _ = ctx.fft_homog_solve(mat, Fbar, Fw, options=fh.default_options(newton_tol=1e-10,
                                                                                   init=fh.INIT_GIVEN))
        tg = host(tgt)
    s = np.linalg.norm(Fbar - np.eye(3).reshape(9))
    ref_t = (host(F0) - Fbar.reshape(9, 1, 1, 1)) / s
    assert np.abs(tg - ref_t).max() <= 1e-6 * np.abs(ref_t).max()
    fluct = Fw_h - Fbar.reshape(9, 1, 1, 1)
    np.testing.assert_allclose(fluct.reshape(9, -1).mean(axis=1), 0.0, atol=1e-14)
    # compatible up to the rounding of F = Fbar + fluctuation (|F| ~ 1, |fluctuation| ~ 1e-5)
    assert np.abs(spectral.project(fluct) - fluct).max() <= 1e-9 * np.abs(fluct).max()
    assert np.abs(fluct).max() > 0
    np.testing.assert_allclose(p1, p0, rtol=1e-9, atol=1e-9 * np.abs(p0).max())


def test_adam_steps_lower_the_loss(fh):
    th = _theta(12).cuda()
    phases, Fbar = _cells(13, 2)
    # a target the network can represent: a multiple of the phase indicator per component
    targets = [dev(np.stack([(0.5 * p - 0.2) * (c + 1) / 9 for c in range(9)]).astype(np.float32)) for p in phases]
    ph = [dev(p) for p in phases]
    m = torch.zeros_like(th)
    v = torch.zeros_like(th)
    grad = torch.empty_like(th)
    with fh.Fno(*SHAPE, max_batch=2, train=True) as net:
        losses = []
        for t in range(1, 31):
            net.set_params(th)
            net.forward(ph, Fbar)
            losses.append(net.loss_grad(targets, grad))
            net.adam(th, grad, m, v, t, 3e-3)
    assert losses[-1] < 0.5 * losses[0], losses


def test_inference_buffers_give_the_training_forward(fh):
    """A network created without training buffers (activations ping-pong between two fields) predicts
    exactly what the training-mode network predicts, for a batch of two cells."""
    th = _theta(15)
    phases, Fbar = _cells(16, 2)
    ph = [dev(p) for p in phases]
    out = []
    for train in (True, False):
        with fh.Fno(*SHAPE, max_batch=2, train=train) as net:
            net.set_params(th.cuda())
            q = [torch.empty((9,) + SHAPE, dtype=torch.float32, device="cuda") for _ in range(2)]
            net.forward(ph, Fbar, q)
            out.append(np.stack([host(x) for x in q]))
    assert np.array_equal(out[0], out[1])


def test_projection_wait_that_runs_out_reports_timeout(fh):
    """The tcgen05 projection's bounded mbarrier wait: with the test hook set, no MMA is issued and nothing
    signals the barrier, so the wait runs out (about a second); the forward pass must report FH_ERR_TIMEOUT,
    and with the hook cleared the same network must run again and give the normal prediction."""
    th = _theta(4)
    phases, Fbar = _cells(5, 1)
    with fh.Fno(*SHAPE, max_batch=1) as net:
        net.set_params(th.cuda())
        ph = [dev(phases[0])]
        q0 = [torch.empty((9,) + SHAPE, dtype=torch.float32, device="cuda")]
        net.forward(ph, Fbar, q0)
        net.test_skip_mma(True)
        with pytest.raises(fh.FhError) as exc:
            net.forward(ph, Fbar, [torch.empty_like(q0[0])])
        assert exc.value.code == fh.FH_ERR_TIMEOUT
        net.test_skip_mma(False)
        q1 = [torch.empty_like(q0[0])]
        net.forward(ph, Fbar, q1)
        assert torch.equal(q0[0], q1[0])
