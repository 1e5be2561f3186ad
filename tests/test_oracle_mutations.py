"""The oracle's pins catch plausible mistakes (CPU only).

Each case below plants one mistake in a copy of one oracle function (a dropped term, a
conjugate, a wrong delay index, a transposed operand, a missing factor, a step taken on
stale values), installs it in place of the original for the duration of the test, and runs
every pin of test_oracle_pins.py against the mutated oracle. At least one pin must fail;
otherwise the pins would not tell that oracle apart from the correct one, and the GPU
parity that rests on the oracle would prove nothing about that part of the method.
"""
import itertools

import numpy as np
import pytest

import test_oracle_pins as pins
from oracle import ctfmnmf_oracle as O


# ---- mutated copies of oracle functions (one planted mistake each)

def _iss_sweep(conj_num=False, conj_update=False):
    """The ISS sweep of Eqs. 11-16 with a planted mistake: the printed conjugate numerator
    for p != r, or w_r^T in place of w_r^H in the rank-1 update."""
    def sweep(W, Q):
        W = W.copy()
        I, M, _ = W.shape
        zs = []
        for r in range(M):
            wr_h = W[:, r, :].copy()
            z = np.zeros((I, M), dtype=complex)
            for p in range(M):
                den = np.einsum("im,imk,ik->i", wr_h, Q[p], wr_h.conj()).real
                ok = den > 0
                if p != r:
                    num = np.einsum("im,imk,ik->i", W[:, p, :], Q[p], wr_h.conj())
                    if conj_num:
                        num = num.conj()
                    z[ok, p] = num[ok] / den[ok]
                else:
                    z[ok, p] = 1.0 - 1.0 / np.sqrt(den[ok])
            upd = wr_h.conj() if conj_update else wr_h
            W = W - z[:, :, None] * upd[:, None, :]
            zs.append(z)
        return W, zs
    return sweep


def _ip_sweep_unscaled(W, Q):
    """IP of Eqs. 9-10 without the (w^H Q_r w)^{-1/2} scaling."""
    W = W.copy()
    I, M, _ = W.shape
    for r in range(M):
        e = np.eye(M, dtype=complex)[r]
        for i in range(I):
            W[i, r, :] = np.linalg.solve(W[i] @ Q[r, i], e).conj()
    return W


def _delayed_weights_undelayed(lam, Ln):
    """phi_r(j) = 1/lambda_{n,i,j} (the delay l dropped from the index), masked j < l."""
    N, I, J = lam.shape
    rows = O.row_map(Ln)
    phi = np.zeros((len(rows), I, J))
    for r, (n, l) in enumerate(rows):
        phi[r, :, l:] = 1.0 / lam[n, :, l:]
    return phi


def _weighted_covariances_transposed(x, phi):
    """Q_r built as (x x^H)^T = conj(x x^H)."""
    J = x.shape[2]
    return np.einsum("rij,imj,ikj->rikm", phi, x, x.conj()) / J


def _update_basis(power=2, root=True):
    """Basis MU of Eq. 17 with lambda^{-power} in the numerator and optionally no sqrt."""
    def update(b, v, y, Ln):
        lam = O.psd(b, v)
        J = v.shape[2]
        num = np.zeros_like(b)
        den = np.zeros_like(b)
        for r, (n, l) in enumerate(O.row_map(Ln)):
            yy = np.abs(y[r, :, l:]) ** 2
            lm = lam[n, :, : J - l]
            vk = v[n, :, : J - l]
            num[n] += np.einsum("ij,kj->ik", yy / lm ** power, vk)
            den[n] += np.einsum("ij,kj->ik", 1.0 / lm, vk)
        ratio = num / den
        return np.maximum(b * (np.sqrt(ratio) if root else ratio), O.FLOOR_NMF), num, den
    return update


def _update_activation_no_count(b, v, y, Ln, mode="all_taps"):
    """Activation MU of Eq. 18 (all taps) with the count of valid taps dropped (1 everywhere)."""
    lam = O.psd(b, v)
    N, K, J = v.shape
    num = np.zeros_like(v)
    den = np.zeros_like(v)
    for n in range(N):
        P, _ = O._delayed_power(y, Ln, n, J)
        num[n] = np.einsum("ik,ij->kj", b[n], P / lam[n] ** 2)
        den[n] = np.einsum("ik,ij->kj", b[n], 1.0 / lam[n])
    return np.maximum(v * np.sqrt(num / den), O.FLOOR_NMF), num, den


_UPDATE_ACTIVATION = O.update_activation   # the unmutated function


def _update_activation_tap0(wrong_row=False, all_tap_count=False):
    """Eq. 18 as printed (tap 0) with a planted mistake: the last tap's row of the source in
    place of its tap-0 row, or the all-taps count of valid taps kept in the denominator."""
    def update(b, v, y, Ln, mode="all_taps"):
        if mode != "tap0":
            return _UPDATE_ACTIVATION(b, v, y, Ln, mode)
        lam = O.psd(b, v)
        N, K, J = v.shape
        rows = O.row_map(Ln)
        num = np.zeros_like(v)
        den = np.zeros_like(v)
        for n in range(N):
            r = rows.index((n, Ln[n] - 1 if wrong_row else 0))
            P = np.abs(y[r]) ** 2
            cnt = O._delayed_power(y, Ln, n, J)[1] if all_tap_count else np.ones(J)
            num[n] = np.einsum("ik,ij->kj", b[n], P / lam[n] ** 2)
            den[n] = np.einsum("ik,ij->kj", b[n], cnt[None, :] / lam[n])
        return np.maximum(v * np.sqrt(num / den), O.FLOOR_NMF), num, den
    return update


def _delayed_power_backwards(y, Ln, n, J):
    """Delayed power with the delay applied in the wrong direction: |y_{(n,l),j-l}|^2 at j."""
    I = y.shape[1]
    P = np.zeros((I, J))
    cnt = np.zeros(J)
    for r, (nn, l) in enumerate(O.row_map(Ln)):
        if nn != n:
            continue
        P[:, l:] += np.abs(y[r, :, : J - l]) ** 2
        cnt[l:] += 1.0
    return P, cnt


def _normalise_b_by_mu(y, W, b, Ln):
    """Eqs. 19-21 with b_n scaled by mu_{n,0}^{-1} instead of mu_{n,0}^{-2}."""
    mu = np.sqrt(np.mean(np.abs(y) ** 2, axis=(1, 2)))
    mu = np.where(mu > 0, mu, 1.0)
    b = b.copy()
    for r, (n, l) in enumerate(O.row_map(Ln)):
        if l == 0:
            b[n] = b[n] / mu[r]
    return y / mu[:, None, None], W / mu[None, :, None], b, mu


def _nll_without_J(y, lam, W, Ln):
    """Eq. 5 with the log-det term not multiplied by the number of frames J."""
    J = y.shape[2]
    total = 0.0
    for r, (n, l) in enumerate(O.row_map(Ln)):
        lm = lam[n, :, : J - l]
        total += np.sum(np.log(lm) + np.abs(y[r, :, l:]) ** 2 / lm)
    return total - 2.0 * np.sum(O.logabsdet(W))


def _source_images_transposed_H(W, y, Ln):
    """Projection-back images with row r of W^{-1} in place of its column r."""
    H = np.linalg.inv(W)
    rows = O.row_map(Ln)
    N = max(n for n, _ in rows) + 1
    I, M, _ = W.shape
    out = np.zeros((N, M, I, y.shape[2]), dtype=complex)
    for r, (n, l) in enumerate(rows):
        out[n] += np.einsum("im,ij->mij", H[:, r, :], y[r])
    return out


def _iterate(stale_bases=False, stale_rows=False):
    """One iteration with an ordering mistake: the activation update with the bases from
    before the basis update, or both NMF updates on the rows from before the demixing update."""
    def iterate(x, W, b, v, Ln, update="iss", v_mode="all_taps", normalize=True):
        lam = O.psd(b, v)
        y_old = O.demix(W, x)
        Q = O.weighted_covariances(x, O.delayed_weights(lam, Ln))
        W, _ = O.iss_sweep(W, Q) if update == "iss" else (O.ip_sweep(W, Q), None)
        y = O.demix(W, x)
        yn = y_old if stale_rows else y
        b_new, _, _ = O.update_basis(b, v, yn, Ln)
        v, _, _ = O.update_activation(b if stale_bases else b_new, v, yn, Ln, v_mode)
        b = b_new
        if normalize:
            y, W, b, _ = O.normalise(y, W, b, Ln)
        return W, b, v, y
    return iterate


def _iss_sweep_gauss_seidel(W, Q):
    """ISS with the rows updated one p at a time inside a step, so that later z_p of the same
    step see the already-updated rows (the step's z must all come from the same W)."""
    W = W.copy()
    I, M, _ = W.shape
    zs = []
    for r in range(M):
        z = np.zeros((I, M), dtype=complex)
        for p in range(M):
            wr_h = W[:, r, :].copy()
            den = np.einsum("im,imk,ik->i", wr_h, Q[p], wr_h.conj()).real
            ok = den > 0
            if p != r:
                num = np.einsum("im,imk,ik->i", W[:, p, :], Q[p], wr_h.conj())
                z[ok, p] = num[ok] / den[ok]
            else:
                z[ok, p] = 1.0 - 1.0 / np.sqrt(den[ok])
            W[:, p, :] = W[:, p, :] - z[:, p, None] * wr_h
        zs.append(z)
    return W, zs


def _ip_sweep_reversed_product(W, Q):
    """IP of Eqs. 9-10 solving (Q_r W) w = e_r instead of (W Q_r) w = e_r."""
    W = W.copy()
    I, M, _ = W.shape
    for r in range(M):
        e = np.eye(M, dtype=complex)[r]
        for i in range(I):
            w = np.linalg.solve(Q[r, i] @ W[i], e)
            W[i, r, :] = (w / np.sqrt((w.conj() @ Q[r, i] @ w).real)).conj()
    return W


def _weighted_covariances_without_1_over_J(x, phi):
    """Q_r of Eq. 8 without its 1/J."""
    return np.einsum("rij,imj,ikj->rimk", phi, x, x.conj())


_NORMALISE = O.normalise      # the unmutated function, captured before any test patches it


def _normalise_columns(y, W, b, Ln):
    """Eqs. 19-21 with the columns of W divided by mu instead of its rows."""
    y2, _, b2, mu = _NORMALISE(y, W, b, Ln)
    return y2, W / mu[None, None, :], b2, mu


MUTANTS = {
    "iterate_activation_with_stale_bases": {"iterate": _iterate(stale_bases=True)},
    "iterate_nmf_on_rows_before_the_sweep": {"iterate": _iterate(stale_rows=True)},
    "iss_rows_updated_within_a_step": {"iss_sweep": _iss_sweep_gauss_seidel},
    "ip_reversed_product": {"ip_sweep": _ip_sweep_reversed_product},
    "covariance_without_1_over_J": {"weighted_covariances": _weighted_covariances_without_1_over_J},
    "normalise_columns_of_W": {"normalise": _normalise_columns},
    "iss_conjugate_numerator": {"iss_sweep": _iss_sweep(conj_num=True)},
    "iss_conjugated_row_update": {"iss_sweep": _iss_sweep(conj_update=True)},
    "ip_without_scaling": {"ip_sweep": _ip_sweep_unscaled},
    "weights_without_delay": {"delayed_weights": _delayed_weights_undelayed},
    "covariance_transposed": {"weighted_covariances": _weighted_covariances_transposed},
    "basis_mu_lambda_inverse_for_inverse_square": {"update_basis": _update_basis(power=1)},
    "basis_mu_without_sqrt": {"update_basis": _update_basis(root=False)},
    "activation_mu_without_tap_count": {"update_activation": _update_activation_no_count},
    "activation_tap0_wrong_tap_row": {"update_activation": _update_activation_tap0(wrong_row=True)},
    "activation_tap0_all_taps_count": {"update_activation": _update_activation_tap0(all_tap_count=True)},
    "delayed_power_backwards": {"_delayed_power": _delayed_power_backwards},
    "normalise_b_by_mu": {"normalise": _normalise_b_by_mu},
    "cost_without_J": {"nll": _nll_without_J},
    "images_with_transposed_inverse": {"source_images": _source_images_transposed_H},
}


def _pin_calls():
    """Every pin of test_oracle_pins.py with each of its parameter sets, cheapest first."""
    calls = []
    for name in sorted(n for n in dir(pins) if n.startswith("test_")):
        fn = getattr(pins, name)
        marks = [m for m in getattr(fn, "pytestmark", []) if m.name == "parametrize"]
        grids = []
        for m in marks:
            argnames, argvalues = m.args[0], m.args[1]
            names = [a.strip() for a in argnames.split(",")] if isinstance(argnames, str) else list(argnames)
            grids.append([dict(zip(names, v if len(names) > 1 else (v,))) for v in argvalues])
        for combo in itertools.product(*grids) if grids else [()]:
            kw = {}
            for d in combo:
                kw.update(d)
            calls.append((name, fn, kw))
    slow = {"test_iss_and_ip_reach_the_same_fixed_point_cost", "test_planted_joint_diagonalisation_closed_form"}
    return sorted(calls, key=lambda c: c[0] in slow)


def test_every_pin_passes_on_the_unmutated_oracle():
    for name, fn, kw in _pin_calls():
        fn(**kw)


@pytest.mark.parametrize("mutant", sorted(MUTANTS))
def test_planted_mistake_fails_a_pin(mutant, monkeypatch):
    for attr, repl in MUTANTS[mutant].items():
        assert hasattr(O, attr)
        monkeypatch.setattr(O, attr, repl)
    caught = []
    for name, fn, kw in _pin_calls():
        try:
            with np.errstate(all="ignore"):
                fn(**kw)
        except (AssertionError, np.linalg.LinAlgError, FloatingPointError, ValueError):
            caught.append(name)
            break
    assert caught, f"no pin fails with the planted mistake {mutant!r}"
