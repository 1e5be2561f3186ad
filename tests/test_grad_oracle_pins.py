"""Pins of the FP64 reference gradient (oracle/ctfmnmf_autograd.py), CPU only.

The autograd restatement is checked against things other than itself: its forward against
the NumPy oracle, its gradient against central finite differences of the NumPy oracle's
loss (directional and per coordinate, which also fixes the complex convention
dL/da + i dL/db), and the closed-form gradient with no iteration (W = I, so the images are
the microphone signals routed to their source).
"""
import numpy as np
import pytest
import torch

from oracle import ctfmnmf_autograd as A
from oracle import ctfmnmf_oracle as O
from paper_2510_02382_gb300 import synth

CASES = [
    # (seed, M, N, Ln, F, J, B, iterations)
    (5, 3, 2, (2, 1), 9, 32, 8, 20),      # the finite-difference shape of the differentiable workload
    (7, 4, 3, (2, 1, 1), 5, 24, 3, 6),
    (9, 2, 2, (1, 1), 4, 20, 2, 5),
]


def _mix(case):
    seed, M, N, Ln, F, J, B, K = case
    return synth.random_case(seed, M=M, N=N, F=F, J=J, B=B, Ln=Ln), K


def _oracle_loss(mix, K, X, T0, V0):
    r = O.run(X, mix.Ln, T0, V0, K)
    c = O.source_images(r["W"], r["y"], mix.Ln)
    return np.mean(np.abs(c - mix.images.astype(np.complex128)) ** 2)


@pytest.mark.parametrize("case", CASES)
def test_forward_equals_numpy_oracle(case):
    mix, K = _mix(case)
    r = O.run(mix.X, mix.Ln, mix.T0, mix.V0, K)
    ref = O.source_images(r["W"], r["y"], mix.Ln)
    with torch.no_grad():
        got = A.separate(torch.tensor(mix.X, dtype=torch.complex128),
                         torch.tensor(mix.T0, dtype=torch.float64),
                         torch.tensor(mix.V0, dtype=torch.float64), mix.Ln, K).numpy()
    assert np.abs(got - ref).max() <= 1e-10 * np.abs(ref).max()


@pytest.mark.parametrize("case", CASES)
def test_gradient_matches_central_differences(case):
    mix, K = _mix(case)
    loss, gx, gb, gv = A.loss_and_gradient(mix.X, mix.T0, mix.V0, mix.images, mix.Ln, K)
    X = mix.X.astype(np.complex128)
    T0 = mix.T0.astype(np.float64)
    V0 = mix.V0.astype(np.float64)
    assert abs(loss - _oracle_loss(mix, K, X, T0, V0)) <= 1e-12 * abs(loss)
    rng = np.random.default_rng(11)
    for _ in range(2):
        d = rng.standard_normal(X.shape) + 1j * rng.standard_normal(X.shape)
        h = 1e-6 * np.abs(X).mean()
        fd = (_oracle_loss(mix, K, X + h * d, T0, V0) - _oracle_loss(mix, K, X - h * d, T0, V0)) / (2 * h)
        assert abs(fd - np.sum((gx.conj() * d).real)) <= 1e-6 * abs(fd)
        d = rng.standard_normal(T0.shape)
        fd = (_oracle_loss(mix, K, X, T0 + 1e-6 * d, V0) - _oracle_loss(mix, K, X, T0 - 1e-6 * d, V0)) / 2e-6
        assert abs(fd - np.sum(gb * d)) <= 1e-6 * abs(fd)
        d = rng.standard_normal(V0.shape)
        fd = (_oracle_loss(mix, K, X, T0, V0 + 1e-6 * d) - _oracle_loss(mix, K, X, T0, V0 - 1e-6 * d)) / 2e-6
        assert abs(fd - np.sum(gv * d)) <= 1e-6 * abs(fd)


def test_gradient_coordinates_fix_the_complex_convention():
    mix, K = _mix(CASES[0])
    _, gx, _, _ = A.loss_and_gradient(mix.X, mix.T0, mix.V0, mix.images, mix.Ln, K)
    X = mix.X.astype(np.complex128)
    T0, V0 = mix.T0.astype(np.float64), mix.V0.astype(np.float64)
    h = 1e-6
    for idx in [(0, 0, 5), (1, 4, 17), (2, 8, 31)]:
        for unit, part in ((1.0, np.real), (1j, np.imag)):
            Xp, Xm = X.copy(), X.copy()
            Xp[idx] += h * unit
            Xm[idx] -= h * unit
            fd = (_oracle_loss(mix, K, Xp, T0, V0) - _oracle_loss(mix, K, Xm, T0, V0)) / (2 * h)
            assert abs(fd - part(gx[idx])) <= 1e-5 * max(abs(fd), 1e-3), (idx, unit)


def test_no_iteration_closed_form():
    """K = 0: W = I, so c_hat_n[m] = x_m for the rows m of source n and 0 elsewhere; the
    gradient of the mean squared error is 2 (x_m - c_{n(m), m}) / (N M F J), and b0, v0
    do not enter."""
    mix, _ = _mix(CASES[1])
    loss, gx, gb, gv = A.loss_and_gradient(mix.X, mix.T0, mix.V0, mix.images, mix.Ln, 0)
    N, M, F, J = mix.images.shape
    rows = [n for n, L in enumerate(mix.Ln) for _ in range(L)]
    X = mix.X.astype(np.complex128)
    C = mix.images.astype(np.complex128)
    expect_loss = 0.0
    for n in range(N):
        for m in range(M):
            pred = X[m] if rows[m] == n else 0.0
            expect_loss += np.sum(np.abs(pred - C[n, m]) ** 2)
    expect_loss /= N * M * F * J
    assert abs(loss - expect_loss) <= 1e-12 * expect_loss
    expect_gx = np.stack([2.0 * (X[m] - C[rows[m], m]) / (N * M * F * J) for m in range(M)])
    assert np.abs(gx - expect_gx).max() <= 1e-14
    assert not gb.any() and not gv.any()
