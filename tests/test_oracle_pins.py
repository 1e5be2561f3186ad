"""Pins of the FP64 oracle to facts fixed by the paper and by mathematics (CPU only).

Each test checks the oracle against something other than itself: a brute-force
minimisation, a closed form, an invariant, a finite-difference gradient, or a
special case with a textbook form.
"""
import os

import numpy as np
import pytest
from scipy.optimize import minimize

from oracle import ctfmnmf_oracle as O
from paper_2510_02382_gb300 import synth

HERE = os.path.dirname(os.path.abspath(__file__))


def _rand_hpd(rng, M, J=12):
    x = rng.standard_normal((M, J)) + 1j * rng.standard_normal((M, J))
    w = rng.uniform(0.2, 2.0, size=J)
    return (x * w) @ x.conj().T / J


def _rand_W(rng, M, I=1):
    return rng.standard_normal((I, M, M)) + 1j * rng.standard_normal((I, M, M))


def _small(seed=0, M=3, N=2, F=5, J=24, B=3, Ln=None):
    mix = synth.random_case(seed, M=M, N=N, F=F, J=J, B=B, Ln=Ln)
    x, W, b, v = O.init_state(mix.X, mix.T0, mix.V0)
    return mix, x, W, b, v


# --- ISS step: closed form (Eq. 16) vs brute-force minimisation of the ISS sub-objective (Eq. 12)

@pytest.mark.parametrize("M", [2, 3, 4])
@pytest.mark.parametrize("seed", [0, 1])
def test_iss_closed_form_is_the_minimiser(M, seed):
    rng = np.random.default_rng(100 + seed)
    W = _rand_W(rng, M)
    Q = np.stack([_rand_hpd(rng, M)[None] for _ in range(M)])        # [M][1][M][M]
    Wcur = W.copy()
    for r in range(M):
        # the sweep starts at r = 0; take step r by permuting the rows so r comes first
        perm = [r] + [p for p in range(M) if p != r]
        Wp = Wcur[:, perm, :]
        Qp = Q[perm]
        _, zsp = O.iss_sweep(Wp, Qp)
        z = np.empty(M, dtype=complex)
        z[perm] = zsp[0][0]

        wr_h = Wcur[0, r, :]

        def objective(par):
            zz = par[:M] + 1j * par[M:]
            Wn = Wcur[0] - np.outer(zz, wr_h)
            val = -2.0 * np.log(np.abs(np.linalg.det(Wn)))
            for p in range(M):
                val += (Wn[p] @ Q[p, 0] @ Wn[p].conj()).real
            return val

        res = minimize(objective, np.zeros(2 * M), method="BFGS", options={"gtol": 1e-11})
        zb = res.x[:M] + 1j * res.x[M:]
        for p in range(M):
            if p != r:
                assert abs(zb[p] - z[p]) < 1e-5, (r, p, zb[p], z[p])
        assert abs(abs(1 - zb[r]) - abs(1 - z[r])) < 1e-5
        assert abs((1 - z[r]).imag) < 1e-14 and (1 - z[r]).real > 0
        assert objective(np.concatenate([z.real, z.imag])) <= res.fun + 1e-9
        # advance the current W by step r to test the next row from a new point
        Wcur = Wcur - z[None, :, None] * wr_h[None, None, :]


def test_printed_conjugate_numerator_is_not_the_minimiser():
    """The numerator printed in Eq. 16 is the conjugate of the minimiser; on complex data
    it gives a strictly larger objective, so the oracle must not use it."""
    rng = np.random.default_rng(7)
    M = 3
    W = _rand_W(rng, M)
    Q = np.stack([_rand_hpd(rng, M)[None] for _ in range(M)])
    _, zs = O.iss_sweep(W, Q)
    z = zs[0][0]
    wr_h = W[0, 0]

    def rows_cost(zz):
        Wn = W[0] - np.outer(zz, wr_h)
        return sum((Wn[p] @ Q[p, 0] @ Wn[p].conj()).real for p in range(1, M))

    zc = z.copy()
    zc[1:] = np.conj(z[1:])
    assert rows_cost(z) < rows_cost(zc) - 1e-6


# --- Determinant lemma (Sec. III-A): det(W - z w_r^H) = det(W)(1 - z_rr)

def test_determinant_lemma_tracks_logdet():
    rng = np.random.default_rng(3)
    M, I = 4, 3
    W = _rand_W(rng, M, I)
    Q = np.stack([np.stack([_rand_hpd(rng, M) for _ in range(I)]) for _ in range(M)])
    W2, zs = O.iss_sweep(W, Q)
    tracked = O.logabsdet(W) + sum(np.log(np.abs(1 - zs[r][:, r])) for r in range(M))
    assert np.max(np.abs(tracked - O.logabsdet(W2))) < 1e-10


# --- Monotonicity: auxiliary function (Eq. 7) per row step; NLL (Eq. 5) per sub-step

def test_aux_nonincreasing_each_row_step():
    rng = np.random.default_rng(5)
    M, I = 4, 4
    W = _rand_W(rng, M, I)
    Q = np.stack([np.stack([_rand_hpd(rng, M) for _ in range(I)]) for _ in range(M)])
    prev = O.aux_value(W, Q)
    Wc = W.copy()
    for r in range(M):
        perm = [r] + [p for p in range(M) if p != r]
        _, zsp = O.iss_sweep(Wc[:, perm, :], Q[perm])
        z = np.empty((I, M), dtype=complex)
        z[:, perm] = zsp[0]
        Wc = Wc - z[:, :, None] * Wc[:, r, :][:, None, :]
        cur = O.aux_value(Wc, Q)
        assert np.all(cur <= prev + 1e-10)
        prev = cur


@pytest.mark.parametrize("Ln,M,N", [((2, 1), 3, 2), ((2, 1, 1), 4, 3), ((1, 1), 2, 2), ((2, 2), 4, 2)])
def test_nll_nonincreasing_each_substep(Ln, M, N):
    mix, x, W, b, v = _small(seed=11, M=M, N=N, Ln=Ln, F=4, J=20)
    y = O.demix(W, x)
    prev = O.nll(y, O.psd(b, v), W, Ln)
    for _ in range(4):
        lam = O.psd(b, v)
        Q = O.weighted_covariances(x, O.delayed_weights(lam, Ln))
        W, _ = O.iss_sweep(W, Q)
        y = O.demix(W, x)
        c1 = O.nll(y, lam, W, Ln)
        b, _, _ = O.update_basis(b, v, y, Ln)
        c2 = O.nll(y, O.psd(b, v), W, Ln)
        v, _, _ = O.update_activation(b, v, y, Ln, "all_taps")
        c3 = O.nll(y, O.psd(b, v), W, Ln)
        tol = 1e-9 * abs(prev)
        assert c1 <= prev + tol and c2 <= c1 + tol and c3 <= c2 + tol, (prev, c1, c2, c3)
        y, W, b, _ = O.normalise(y, W, b, Ln)
        prev = O.nll(y, O.psd(b, v), W, Ln)


# --- The cost of Eq. 5 equals J * (aux of Eq. 7 with Q of Eq. 8) + sum of log lambda

def test_cost_equals_auxiliary_form():
    Ln = (2, 1)
    mix, x, W, b, v = _small(seed=2, Ln=Ln, F=3, J=16)
    rng = np.random.default_rng(9)
    W = W + 0.3 * _rand_W(rng, 3, 3)
    lam = O.psd(b, v)
    Q = O.weighted_covariances(x, O.delayed_weights(lam, Ln))
    y = O.demix(W, x)
    J = x.shape[2]
    logs = sum(np.sum(np.log(lam[n, :, : J - l])) for n, l in O.row_map(Ln))
    assert abs(O.nll(y, lam, W, Ln) - (J * np.sum(O.aux_value(W, Q)) + logs)) < 1e-9 * J


# --- MU rules (Eqs. 17-18): fixed point and gradient split

def _matched_y(lam, Ln, rng):
    """y with |y_{(n,l),i,j}|^2 = lambda_{n,i,j-l} exactly on the unmasked frames."""
    N, I, J = lam.shape
    rows = O.row_map(Ln)
    y = np.zeros((len(rows), I, J), dtype=complex)
    for r, (n, l) in enumerate(rows):
        ph = np.exp(2j * np.pi * rng.uniform(size=(I, J)))
        y[r] = ph * rng.uniform(0.5, 2.0, size=(I, J))
        y[r, :, l:] = ph[:, l:] * np.sqrt(lam[n, :, : J - l])
    return y


def test_mu_fixed_point_when_power_matches_model():
    Ln = (2, 1)
    rng = np.random.default_rng(4)
    b = rng.uniform(0.2, 1.5, (2, 5, 3))
    v = rng.uniform(0.2, 1.5, (2, 3, 17))
    y = _matched_y(O.psd(b, v), Ln, rng)
    b2, _, _ = O.update_basis(b, v, y, Ln)
    v2, _, _ = O.update_activation(b, v, y, Ln, "all_taps")
    assert np.max(np.abs(b2 / b - 1)) < 1e-12
    assert np.max(np.abs(v2 / v - 1)) < 1e-12


def test_mu_sums_are_the_gradient_split():
    """dNLL/db = den - num and dNLL/dv = den - num (all-taps), by central differences."""
    Ln = (2, 1)
    mix, x, W, b, v = _small(seed=6, Ln=Ln, F=3, J=10, B=2)
    rng = np.random.default_rng(1)
    y = O.demix(W + 0.2 * _rand_W(rng, 3, 3), x)
    _, num_b, den_b = O.update_basis(b, v, y, Ln)
    _, num_v, den_v = O.update_activation(b, v, y, Ln, "all_taps")

    def f(bb, vv):
        return O.nll(y, O.psd(bb, vv), W, Ln)

    h = 1e-6
    for idx in [(0, 0, 0), (1, 2, 1), (0, 1, 1)]:
        e = np.zeros_like(b)
        e[idx] = h
        g = (f(b + e, v) - f(b - e, v)) / (2 * h)
        assert abs(g - (den_b[idx] - num_b[idx])) < 1e-5 * max(1.0, abs(g))
    for idx in [(0, 0, 0), (1, 1, 9), (0, 1, 4)]:
        e = np.zeros_like(v)
        e[idx] = h
        g = (f(b, v + e) - f(b, v - e)) / (2 * h)
        assert abs(g - (den_v[idx] - num_v[idx])) < 1e-5 * max(1.0, abs(g))


def test_mu_single_basis_is_the_geometric_mean_step():
    """With one basis (K = 1) the NLL of Eq. 5 in b_{n,i} (or in v_{n,j}) has the closed-form
    minimiser b* = mean over the unmasked (j, l) terms of |y_{(n,l),i,j}|^2 / v_{n,j-l}
    (v* = mean over (i, l) of |y_{(n,l),i,j+l}|^2 / b_{n,i}); the majorise-minimise steps of
    Eqs. 17-18 move halfway there in log scale: b_new = sqrt(b b*), v_new = sqrt(v v*)."""
    Ln = (2, 1)
    rng = np.random.default_rng(17)
    I, J = 3, 15
    b = rng.uniform(0.3, 2.0, (2, I, 1))
    v = rng.uniform(0.3, 2.0, (2, 1, J))
    y = rng.standard_normal((3, I, J)) + 1j * rng.standard_normal((3, I, J))
    rows = [(0, 0), (0, 1), (1, 0)]
    for n in range(2):
        taps = [(r, l) for r, (nn, l) in enumerate(rows) if nn == n]
        bstar = np.zeros(I)
        for i in range(I):
            terms = [abs(y[r, i, j]) ** 2 / v[n, 0, j - l] for r, l in taps for j in range(l, J)]
            bstar[i] = np.mean(terms)
        vstar = np.zeros(J)
        for j in range(J):
            terms = [abs(y[r, i, j + l]) ** 2 / b[n, i, 0] for r, l in taps for i in range(I) if j + l < J]
            vstar[j] = np.mean(terms)
        b_new, _, _ = O.update_basis(b, v, y, Ln)
        v_new, _, _ = O.update_activation(b, v, y, Ln, "all_taps")
        assert np.max(np.abs(b_new[n, :, 0] / np.sqrt(b[n, :, 0] * bstar) - 1)) < 1e-12
        assert np.max(np.abs(v_new[n, 0] / np.sqrt(v[n, 0] * vstar) - 1)) < 1e-12


def test_iteration_order_single_basis():
    """One whole iteration without normalisation, one basis (Sec. III order: demixing
    update, then the basis update on the new rows, then the activation update with the new
    bases): with y = W x from the returned W, the returned b is sqrt(b0 b*) with b* the
    closed-form minimiser for y and v0, and the returned v is sqrt(v0 v*) with v* the one
    for y and the returned b."""
    Ln = (2, 1)
    mix = synth.random_case(19, M=3, N=2, F=4, J=18, B=1, Ln=Ln)
    x, W0, b0, v0 = O.init_state(mix.X, mix.T0, mix.V0)
    W, b, v, y = O.iterate(x, W0, b0, v0, Ln, normalize=False)
    y = O.demix(W, x)
    rows = O.row_map(Ln)
    I, J = x.shape[0], x.shape[2]
    for n in range(2):
        taps = [(r, l) for r, (nn, l) in enumerate(rows) if nn == n]
        bstar = np.array([np.mean([abs(y[r, i, j]) ** 2 / v0[n, 0, j - l] for r, l in taps for j in range(l, J)])
                          for i in range(I)])
        vstar = np.array([np.mean([abs(y[r, i, j + l]) ** 2 / b[n, i, 0] for r, l in taps for i in range(I)
                                   if j + l < J]) for j in range(J)])
        assert np.max(np.abs(b[n, :, 0] / np.sqrt(b0[n, :, 0] * bstar) - 1)) < 1e-12
        assert np.max(np.abs(v[n, 0] / np.sqrt(v0[n, 0] * vstar) - 1)) < 1e-12


@pytest.mark.parametrize("Ln,M,N", [((2, 1), 3, 2), ((2, 1, 1), 4, 3), ((2, 2), 4, 2)])
def test_nll_nonincreasing_over_whole_iterations(Ln, M, N):
    """Without the normalisation every iteration is a chain of majorise-minimise steps of
    Eq. 5 (demixing update, basis MU, activation MU), so the NLL never rises."""
    mix = synth.random_case(30 + M + N, M=M, N=N, F=4, J=24, B=3, Ln=Ln)
    x, W, b, v = O.init_state(mix.X, mix.T0, mix.V0)
    out = O.run(mix.X, Ln, mix.T0, mix.V0, 12, normalize=False, trace=True)
    c = [O.nll(O.demix(W, x), O.psd(b, v), W, Ln)] + list(out["trace"])
    for a, bb in zip(c[:-1], c[1:]):
        assert bb <= a + 1e-9 * abs(a), (a, bb)


def test_tap0_mode_equals_all_taps_when_one_tap():
    Ln = (1, 1)
    mix, x, W, b, v = _small(seed=8, M=2, N=2, Ln=Ln, F=3, J=12)
    y = O.demix(W, x)
    v1, _, _ = O.update_activation(b, v, y, Ln, "all_taps")
    v2, _, _ = O.update_activation(b, v, y, Ln, "tap0")
    assert np.max(np.abs(v1 - v2)) < 1e-14


def test_tap0_single_basis_is_the_geometric_mean_step():
    """Eq. 18 as printed (tap 0 only), one basis (K = 1), sources with more than one tap:
    with lambda = b v the update reads v_new = v sqrt(sum_i |y_{(n,0),i,j}|^2 / (b_{n,i} v^2)
    / sum_i 1/v), i.e. the geometric mean of v and the minimiser v* = mean over bins i of
    |y_{(n,0),i,j}|^2 / b_{n,i} of the tap-0 terms of Eq. 5. Only row (n, 0) enters and the
    denominator counts one term per bin, whatever L_n is."""
    Ln = (3, 2)
    rows = O.row_map(Ln)
    rng = np.random.default_rng(23)
    I, J = 4, 11
    b = rng.uniform(0.3, 2.0, (2, I, 1))
    v = rng.uniform(0.3, 2.0, (2, 1, J))
    y = rng.standard_normal((5, I, J)) + 1j * rng.standard_normal((5, I, J))
    v_new, _, _ = O.update_activation(b, v, y, Ln, "tap0")
    for n in range(2):
        r0 = rows.index((n, 0))
        vstar = np.array([np.mean([abs(y[r0, i, j]) ** 2 / b[n, i, 0] for i in range(I)]) for j in range(J)])
        assert np.max(np.abs(v_new[n, 0] / np.sqrt(v[n, 0] * vstar) - 1)) < 1e-12


def test_nmf_factors_stay_positive():
    Ln = (2, 1)
    mix = synth.random_case(12, M=3, N=2, F=6, J=30, B=3, Ln=Ln)
    out = O.run(mix.X, Ln, mix.T0, mix.V0, 8)
    assert np.all(out["b"] > 0) and np.all(out["v"] > 0)
    assert np.all(np.isfinite(out["y"]))


# --- Normalisation (Eqs. 19-21)

def test_normalisation_gives_unit_row_power_and_keeps_y_equal_wx():
    Ln = (2, 1)
    mix, x, W, b, v = _small(seed=13, Ln=Ln)
    rng = np.random.default_rng(0)
    W = W + 0.4 * _rand_W(rng, 3, W.shape[0])
    y = O.demix(W, x)
    y2, W2, b2, mu = O.normalise(y, W, b, Ln)
    assert np.allclose(np.mean(np.abs(y2) ** 2, axis=(1, 2)), 1.0, atol=1e-12)
    assert np.max(np.abs(O.demix(W2, x) - y2)) < 1e-12
    assert np.allclose(b2[0], b[0] / mu[0] ** 2) and np.allclose(b2[1], b[1] / mu[2] ** 2)


# --- Source images (Eqs. 23-24): projection-back, sum to the mixture, literal MWF

def test_images_sum_to_mixture_and_equal_literal_mwf():
    Ln = (2, 1)
    mix, x, W, b, v = _small(seed=14, Ln=Ln, F=3, J=9)
    rng = np.random.default_rng(2)
    W = W + 0.5 * _rand_W(rng, 3, 3)
    y = O.demix(W, x)
    c = O.source_images(W, y, Ln)
    assert np.max(np.abs(c.sum(axis=0) - np.transpose(x, (1, 0, 2)))) < 1e-12
    c_mwf = O.mwf_images(W, O.psd(b, v), x, Ln)
    lmax = 1
    assert np.max(np.abs(c[..., lmax:] - c_mwf[..., lmax:])) < 1e-9


# --- IP (Eqs. 9-10) and the ISS/IP fixed points

def test_ip_last_row_satisfies_head():
    rng = np.random.default_rng(21)
    M, I = 3, 2
    W = _rand_W(rng, M, I)
    Q = np.stack([np.stack([_rand_hpd(rng, M) for _ in range(I)]) for _ in range(M)])
    W2 = O.ip_sweep(W, Q)
    r = M - 1
    for i in range(I):
        w = W2[i, r].conj()
        assert np.max(np.abs(W2[i] @ Q[r, i] @ w - np.eye(M)[r])) < 1e-10


def test_ip_row_update_determinant_factor():
    """Each IP row update (Eqs. 9-10) multiplies |det W| by (x^H Q_r x)^{1/2}, where
    x = (W Q_r)^{-1} e_r is taken before the update: replacing row r is the rank-one update
    W + e_r d^H, and the matrix determinant lemma with W^{-1} e_r = Q_r x gives the factor.
    The IP bin kernel returns |det W_new| / |det W_old| in this form; here the oracle's sweep
    is checked against it with determinants from slogdet. Step r changes row r only, so the
    matrix before step r is the swept rows 0..r-1 over the initial rows r..M-1."""
    rng = np.random.default_rng(23)
    for M in (2, 3, 4):
        I = 3
        W = _rand_W(rng, M, I)
        Q = np.stack([np.stack([_rand_hpd(rng, M) for _ in range(I)]) for _ in range(M)])
        W2 = O.ip_sweep(W, Q)
        expect = np.zeros(I)
        for r in range(M):
            Wb = np.concatenate([W2[:, :r], W[:, r:]], axis=1)
            for i in range(I):
                x = np.linalg.solve(Wb[i] @ Q[r, i], np.eye(M)[r])
                expect[i] += 0.5 * np.log((x.conj() @ Q[r, i] @ x).real)
        got = np.linalg.slogdet(W2)[1] - np.linalg.slogdet(W)[1]
        assert np.max(np.abs(got - expect)) < 1e-10, (M, got, expect)


def _head_residual(W, Q):
    M = W.shape[1]
    res = 0.0
    for i in range(W.shape[0]):
        for r in range(M):
            w = W[i, r].conj()
            res = max(res, np.max(np.abs(W[i] @ Q[r, i] @ w - np.eye(M)[r])))
    return res


def test_iss_and_ip_reach_the_same_fixed_point_cost():
    rng = np.random.default_rng(31)
    M, I = 3, 2
    Q = np.stack([np.stack([_rand_hpd(rng, M, J=40) for _ in range(I)]) for _ in range(M)])
    W = np.tile(np.eye(M, dtype=complex), (I, 1, 1))
    for _ in range(3000):
        W, _ = O.iss_sweep(W, Q)
    assert _head_residual(W, Q) < 1e-8
    a_iss = O.aux_value(W, Q)
    W_ip = O.ip_sweep(W, Q)
    assert np.max(np.abs(O.aux_value(W_ip, Q) - a_iss) / np.abs(a_iss)) < 1e-10
    W2 = np.tile(np.eye(M, dtype=complex), (I, 1, 1))
    for _ in range(300):
        W2 = O.ip_sweep(W2, Q)
    assert _head_residual(W2, Q) < 1e-8
    W2s, _ = O.iss_sweep(W2, Q)
    assert np.max(np.abs(O.aux_value(W2s, Q) - O.aux_value(W2, Q))) < 1e-10 * np.max(np.abs(a_iss))


def test_planted_joint_diagonalisation_closed_form():
    """Q_r = A D_r A^H: a stationary W is a scaled permutation of A^{-1}, and the
    auxiliary value there is M + sum_r log D_r[pi(r)] + 2 log|det A|."""
    rng = np.random.default_rng(41)
    M = 3
    A = rng.standard_normal((M, M)) + 1j * rng.standard_normal((M, M))
    D = np.exp(rng.uniform(-2.0, 2.0, size=(M, M)))             # D[r] diagonal of D_r
    Q = np.stack([(A * D[r]) @ A.conj().T for r in range(M)])[:, None]
    W = np.eye(M, dtype=complex)[None]
    for _ in range(4000):
        W, _ = O.iss_sweep(W, Q)
    G = W[0] @ A
    pi = np.argmax(np.abs(G), axis=1)
    assert sorted(pi) == list(range(M))
    off = np.abs(G).copy()
    off[np.arange(M), pi] = 0.0
    assert np.max(off) < 1e-7 * np.max(np.abs(G))
    expect = M + sum(np.log(D[r, pi[r]]) for r in range(M)) + 2 * np.log(abs(np.linalg.det(A)))
    assert abs(O.aux_value(W, Q)[0] - expect) < 1e-9


# --- Special case L_n = 1 (M = N): the sweep is ILRMA with ISS in its data-domain form

def test_single_tap_case_matches_data_domain_iss():
    """With one tap per source, the ISS step written on the separated signals
    (z_p = sum_j y_p conj(y_r)/lam_p / sum_j |y_r|^2/lam_p, z_r = 1 - (mean_j |y_r|^2/lam_r)^{-1/2},
    y_p <- y_p - z_p y_r) must reproduce the oracle's covariance-domain sweep."""
    Ln = (1, 1, 1)
    mix, x, W, b, v = _small(seed=15, M=3, N=3, Ln=Ln, F=4, J=32)
    rng = np.random.default_rng(3)
    W = W + 0.3 * _rand_W(rng, 3, 4)
    lam = O.psd(b, v)
    Q = O.weighted_covariances(x, O.delayed_weights(lam, Ln))
    W2, _ = O.iss_sweep(W, Q)
    y = O.demix(W, x)
    for r in range(3):
        yr = y[r].copy()
        for p in range(3):
            if p == r:
                continue
            z = np.sum(y[p] * yr.conj() / lam[p], axis=1) / np.sum(np.abs(yr) ** 2 / lam[p], axis=1)
            y[p] = y[p] - z[:, None] * yr
        q = np.mean(np.abs(yr) ** 2 / lam[r], axis=1)
        y[r] = yr / np.sqrt(q)[:, None]
    assert np.max(np.abs(O.demix(W2, x) - y)) < 1e-10 * np.max(np.abs(y))


# --- Table I (Sec. V-A): taps per source for 4/6/8 microphones and 2 sources

def test_default_taps_reproduce_table1():
    rows = np.loadtxt(os.path.join(HERE, "golden", "table1_taps.txt"), dtype=int)
    for M, N, Ln in rows:
        assert synth.default_taps(int(M), int(N), 8) == [int(Ln)] * int(N)


def test_zero_energy_bin_is_left_unchanged():
    """A bin with no signal (all-zero observations) keeps W = I and produces no NaN."""
    Ln = (2, 1)
    mix = synth.random_case(16, M=3, N=2, F=4, J=20, B=2, Ln=Ln)
    X = mix.X.copy()
    X[:, 1, :] = 0
    out = O.run(X, Ln, mix.T0, mix.V0, 3)
    assert np.all(np.isfinite(out["y"])) and np.isfinite(out["cost"])
    W1 = out["W"][1]
    assert np.allclose(W1, np.diag(np.diag(W1)))
