"""The differentiable form (ctfmnmf_grad_*) against the FP64 reference gradient
(oracle/ctfmnmf_autograd.py) and central differences of the FP64 oracle.

The library's loss is the batch mean of the per-mixture MSE, so its gradient with respect
to mixture s is (1/S) times that mixture's reference gradient."""
import numpy as np
import pytest

from oracle import ctfmnmf_autograd as A
from oracle import ctfmnmf_oracle as O
from paper_2510_02382_gb300 import synth

from gpu_helpers import rel_fro

pytestmark = pytest.mark.gpu

TOL = 1e-3   # relative (Frobenius) error of every gradient against the FP64 reference

SHAPES = [
    # (M, N, Ln, F, J, B, iterations, checkpoint every, batch)
    (3, 2, (2, 1), 9, 32, 8, 20, 5, 2),       # the finite-difference shape of the workload
    (2, 2, (1, 1), 5, 37, 3, 7, 3, 2),        # ragged frames and a short last segment
    (4, 3, (2, 1, 1), 6, 70, 5, 6, 4, 2),
    (3, 2, (2, 1), 4, 700, 10, 3, 2, 1),      # two frames per thread, several frame tiles
    (3, 2, (2, 1), 3, 130, 20, 2, 1, 3),      # B > 16, a checkpoint every iteration
    (3, 2, (2, 1), 7, 45, 6, 5, 8, 2),        # one segment: every iteration on the forward tape
]


def _batch(shape, seed0=0):
    M, N, Ln, F, J, B, K, C, S = shape
    return [synth.random_case(seed0 + 100 + k, M=M, N=N, F=F, J=J, B=B, Ln=Ln) for k in range(S)]


def _run(shape, mixes):
    import torch
    from paper_2510_02382_gb300.api import Grad
    M, N, Ln, F, J, B, K, C, S = shape
    g = Grad(M, N, max(Ln), B, F, J, batch=S, n_iter=K, ckpt_every=C, Ln=Ln)
    X = torch.from_numpy(np.stack([m.X for m in mixes])).cuda()
    T0 = torch.from_numpy(np.stack([m.T0 for m in mixes])).cuda()
    V0 = torch.from_numpy(np.stack([m.V0 for m in mixes])).cuda()
    Cref = torch.from_numpy(np.stack([m.images for m in mixes])).cuda()
    Cimg = g.forward(X, T0, V0)
    loss = torch.zeros((), dtype=torch.float64, device="cuda")
    gC = torch.empty_like(Cimg)
    g.mse(Cimg, Cref, loss=loss, gC=gC)
    gX, gT0, gV0 = g.backward(gC)
    torch.cuda.synchronize()
    out = {"C": Cimg.cpu().numpy(), "loss": float(loss.cpu()), "gX": gX.cpu().numpy(),
           "gT0": gT0.cpu().numpy(), "gV0": gV0.cpu().numpy(), "launches": g.launch_count()}
    g.close()
    return out


@pytest.mark.parametrize("shape", SHAPES)
def test_gradient_matches_fp64_reference(shape):
    M, N, Ln, F, J, B, K, C, S = shape
    mixes = _batch(shape)
    out = _run(shape, mixes)
    losses = []
    for k, mix in enumerate(mixes):
        loss, gx, gb, gv = A.loss_and_gradient(mix.X, mix.T0, mix.V0, mix.images, mix.Ln, K)
        losses.append(loss)
        r = O.run(mix.X, mix.Ln, mix.T0, mix.V0, K)
        img = O.source_images(r["W"], r["y"], mix.Ln)
        assert rel_fro(out["C"][k], img) < 1e-3, (k, rel_fro(out["C"][k], img))
        assert rel_fro(S * out["gX"][k], gx) < TOL, ("gX", k, rel_fro(S * out["gX"][k], gx))
        assert rel_fro(S * out["gT0"][k], gb) < TOL, ("gT0", k, rel_fro(S * out["gT0"][k], gb))
        assert rel_fro(S * out["gV0"][k], gv) < TOL, ("gV0", k, rel_fro(S * out["gV0"][k], gv))
    assert abs(out["loss"] - np.mean(losses)) <= 1e-4 * abs(np.mean(losses))


def test_directional_derivatives_match_oracle_differences():
    """F = 9, J = 32: <gradient, d> against central differences of the FP64 oracle's loss
    for random directions d in X (complex), T0 and V0."""
    shape = SHAPES[0]
    M, N, Ln, F, J, B, K, C, S = shape
    mixes = _batch(shape)
    out = _run(shape, mixes)
    rng = np.random.default_rng(3)
    for k, mix in enumerate(mixes):
        X, T0, V0 = mix.X.astype(np.complex128), mix.T0.astype(np.float64), mix.V0.astype(np.float64)

        def loss(X, T0, V0):
            r = O.run(X, mix.Ln, T0, V0, K)
            c = O.source_images(r["W"], r["y"], mix.Ln)
            return np.mean(np.abs(c - mix.images.astype(np.complex128)) ** 2) / S

        d = rng.standard_normal(X.shape) + 1j * rng.standard_normal(X.shape)
        h = 1e-6 * np.abs(X).mean()
        fd = (loss(X + h * d, T0, V0) - loss(X - h * d, T0, V0)) / (2 * h)
        assert abs(np.sum((out["gX"][k].astype(np.complex128).conj() * d).real) - fd) <= TOL * abs(fd)
        d = rng.standard_normal(T0.shape)
        fd = (loss(X, T0 + 1e-6 * d, V0) - loss(X, T0 - 1e-6 * d, V0)) / 2e-6
        assert abs(np.sum(out["gT0"][k] * d) - fd) <= TOL * abs(fd)
        d = rng.standard_normal(V0.shape)
        fd = (loss(X, T0, V0 + 1e-6 * d) - loss(X, T0, V0 - 1e-6 * d)) / 2e-6
        assert abs(np.sum(out["gV0"][k] * d) - fd) <= TOL * abs(fd)


def test_tape_and_recomputation_agree():
    """One segment (every state from the forward pass's tape) against a checkpoint every
    iteration (all but the last iteration recomputed in the backward pass): the same gradients
    up to the rounding of the recomputed 1/lambda."""
    M, N, Ln, F, J, B, K, C, S = SHAPES[0]
    mixes = _batch(SHAPES[0])
    taped = _run((M, N, Ln, F, J, B, K, K, S), mixes)
    recomputed = _run((M, N, Ln, F, J, B, K, 1, S), mixes)
    assert abs(taped["loss"] - recomputed["loss"]) <= 1e-6 * abs(taped["loss"])
    for key in ("C", "gX", "gT0", "gV0"):
        assert rel_fro(taped[key], recomputed[key]) < 1e-4, key


def test_autograd_function_matches_direct_calls():
    import torch
    from paper_2510_02382_gb300.api import Grad
    from paper_2510_02382_gb300.autograd import mse, separate
    shape = SHAPES[2]
    M, N, Ln, F, J, B, K, C, S = shape
    mixes = _batch(shape)
    ref = _run(shape, mixes)
    g = Grad(M, N, max(Ln), B, F, J, batch=S, n_iter=K, ckpt_every=C, Ln=Ln)
    X = torch.from_numpy(np.stack([m.X for m in mixes])).cuda().requires_grad_()
    T0 = torch.from_numpy(np.stack([m.T0 for m in mixes])).cuda().requires_grad_()
    V0 = torch.from_numpy(np.stack([m.V0 for m in mixes])).cuda().requires_grad_()
    Cref = torch.from_numpy(np.stack([m.images for m in mixes])).cuda()
    loss = mse(separate(X, T0, V0, g), Cref, g)
    (3.0 * loss).backward()
    assert abs(float(loss.detach()) - ref["loss"]) <= 1e-6 * abs(ref["loss"])
    assert rel_fro(X.grad.cpu().numpy(), 3.0 * ref["gX"]) < 1e-5
    assert rel_fro(T0.grad.cpu().numpy(), 3.0 * ref["gT0"]) < 1e-5
    assert rel_fro(V0.grad.cpu().numpy(), 3.0 * ref["gV0"]) < 1e-5
    g.close()


def test_backward_needs_a_forward_pass():
    import torch
    from paper_2510_02382_gb300.api import CtfMnmfError, Grad
    M, N, Ln, F, J, B, K, C, S = SHAPES[1]
    mixes = _batch(SHAPES[1])
    g = Grad(M, N, max(Ln), B, F, J, batch=S, n_iter=K, ckpt_every=C, Ln=Ln)
    gC = torch.zeros(g.shapes()["C"], dtype=torch.complex64, device="cuda")
    with pytest.raises(CtfMnmfError) as e:
        g.backward(gC)
    assert e.value.name == "ESTATE"
    X = torch.from_numpy(np.stack([m.X for m in mixes])).cuda()
    T0 = torch.from_numpy(np.stack([m.T0 for m in mixes])).cuda()
    V0 = torch.from_numpy(np.stack([m.V0 for m in mixes])).cuda()
    g.forward(X, T0, V0)
    g.backward(gC)
    with pytest.raises(CtfMnmfError) as e:
        g.backward(gC)
    assert e.value.name == "ESTATE"
    g.close()


def test_differentiable_workload_sampled():
    """The C5 workload (16 mixtures, N=2, M=3, L=4, F=257, J=500, B=8, 20 iterations,
    checkpoint every 5) as the benchmark runs it: images of two sampled mixtures against the
    oracle, and directional derivatives of their losses against oracle central differences."""
    import torch
    from paper_2510_02382_gb300.api import Grad
    specs = synth.grad_specs()
    mixes = [synth.make_mixture(sp) for sp in specs]
    sp = specs[0]
    S, K = len(specs), sp.iters
    g = Grad(sp.M, sp.N, sp.L, sp.B, sp.F, sp.J, batch=S, n_iter=K, ckpt_every=5)
    X = torch.from_numpy(np.stack([m.X for m in mixes])).cuda()
    T0 = torch.from_numpy(np.stack([m.T0 for m in mixes])).cuda()
    V0 = torch.from_numpy(np.stack([m.V0 for m in mixes])).cuda()
    Cref = torch.from_numpy(np.stack([m.images for m in mixes])).cuda()
    Cimg = g.forward(X, T0, V0)
    gC = torch.empty_like(Cimg)
    g.mse(Cimg, Cref, gC=gC)
    gX, gT0, gV0 = g.backward(gC)
    torch.cuda.synchronize()
    rng = np.random.default_rng(7)
    for k in (0, 15):
        mix = mixes[k]
        r = O.run(mix.X, mix.Ln, mix.T0, mix.V0, K)
        img = O.source_images(r["W"], r["y"], mix.Ln)
        assert rel_fro(Cimg[k].cpu().numpy(), img) < 1e-3
        Xk, T0k, V0k = mix.X.astype(np.complex128), mix.T0.astype(np.float64), mix.V0.astype(np.float64)

        def loss(X, T0, V0):
            r = O.run(X, mix.Ln, T0, V0, K)
            c = O.source_images(r["W"], r["y"], mix.Ln)
            return np.mean(np.abs(c - mix.images.astype(np.complex128)) ** 2) / S

        d = rng.standard_normal(Xk.shape) + 1j * rng.standard_normal(Xk.shape)
        h = 1e-6 * np.abs(Xk).mean()
        fd = (loss(Xk + h * d, T0k, V0k) - loss(Xk - h * d, T0k, V0k)) / (2 * h)
        got = np.sum((gX[k].cpu().numpy().astype(np.complex128).conj() * d).real)
        assert abs(got - fd) <= TOL * abs(fd), (k, got, fd)
        d = rng.standard_normal(T0k.shape)
        fd = (loss(Xk, T0k + 1e-6 * d, V0k) - loss(Xk, T0k - 1e-6 * d, V0k)) / 2e-6
        got = np.sum(gT0[k].cpu().numpy() * d)
        assert abs(got - fd) <= TOL * abs(fd), (k, got, fd)
        d = rng.standard_normal(V0k.shape)
        fd = (loss(Xk, T0k, V0k + 1e-6 * d) - loss(Xk, T0k, V0k - 1e-6 * d)) / 2e-6
        got = np.sum(gV0[k].cpu().numpy() * d)
        assert abs(got - fd) <= TOL * abs(fd), (k, got, fd)
    g.close()
