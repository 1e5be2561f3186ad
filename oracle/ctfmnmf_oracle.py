"""FP64 CPU oracle for CTF-MNMF with ISS (and the IP update it replaces).

TEST INFRASTRUCTURE ONLY. This module is the plain, slow, double-precision
statement of the method used to check the CUDA library. Only the test suite,
the smoke check and the CPU-baseline leg of the benchmark may import it; the
library itself never does, and nothing here is shared with the CUDA code.

Notation follows the paper (Xie et al., "Accelerated CTF-Based Multichannel NMF
Using Iterative Source Steering"):
    I bins (index i), J frames (index j), M microphones, N sources,
    L_n taps of source n with sum_n L_n = M (Sec. II, square extended model),
    extended row r <-> (n, l), r = L_1 + ... + L_{n-1} + l   (0-based, Sec. III-A),
    W_i (M x M) demixing matrix whose row r is w_r^H, y_{r,i,j} = w_r^H x_{i,j} (Eq. 4),
    b[n,i,k], v[n,k,j] the NMF factors, lambda_{n,i,j} = sum_k b v (Sec. II).
Arrays: x [I][M][J], y [M][I][J], W [I][M][M], b [N][I][K], v [N][K][J], lam [N][I][J].

Readings of the paper that this oracle fixes (where it is silent or garbled):
  * masked delays: a term that needs lambda_{n,i,j-l} with j-l < 0 is left out of
    Q, of both MU sums and of the cost; the 1/J of Q and the 2J of the log-det keep J;
  * ISS, p != r: z_p = (w_p^H Q_p w_r) / (w_r^H Q_p w_r), the minimiser of the ISS
    sub-objective as written (the printed numerator is its complex conjugate);
  * ISS, p == r: z_r = 1 - (w_r^H Q_r w_r)^{-1/2} (the real positive root);
  * a zero denominator (a row with no energy) leaves that coefficient at 0;
  * the basis update sums l over the taps of its own source (l < L_n);
  * the activation update uses all taps of the source by default ("all_taps",
    the majorisation-minimisation form), or tap 0 only as printed ("tap0");
  * T and V are floored at 1e-12 after each MU, lambda at 1e-18 where it is formed;
  * order per iteration: ISS sweep -> basis MU -> activation MU -> normalisation,
    normalisation once per iteration with mu over all frames.
"""
from __future__ import annotations

import numpy as np

FLOOR_NMF = 1e-12   # floor of b and v after each multiplicative update
FLOOR_PSD = 1e-18   # floor of lambda where it is formed


def row_map(Ln):
    """Flattened extended rows: r -> (n, l), r = L_1 + ... + L_{n-1} + l (Sec. III-A)."""
    rows = []
    for n, L in enumerate(Ln):
        for l in range(L):
            rows.append((n, l))
    return rows


def psd(b, v):
    """lambda_{n,i,j} = sum_k b_{n,i,k} v_{n,k,j} (the NMF source model, Sec. II)."""
    return np.maximum(np.einsum("nik,nkj->nij", b, v), FLOOR_PSD)


def demix(W, x):
    """y_{r,i,j} = w_r^H x_{i,j} with row r of W_i holding w_r^H (Eq. 4)."""
    return np.einsum("irm,imj->rij", W, x)


def delayed_weights(lam, Ln):
    """phi[r,i,j] = 1 / lambda_{n,i,j-l} for j >= l, 0 for the masked j < l: the weight of
    extended row r = (n, l) in Eq. 8 (the delayed PSD of the extended model, Sec. II)."""
    N, I, J = lam.shape
    rows = row_map(Ln)
    phi = np.zeros((len(rows), I, J))
    for r, (n, l) in enumerate(rows):
        phi[r, :, l:] = 1.0 / lam[n, :, : J - l]
    return phi


def weighted_covariances(x, phi):
    """Q_{r,i} = (1/J) sum_j x_{i,j} x_{i,j}^H / lambda_{n,i,j-l}  (Eq. 8), [M][I][M][M]."""
    J = x.shape[2]
    return np.einsum("rij,imj,ikj->rimk", phi, x, x.conj()) / J


def aux_value(W, Q):
    """Auxiliary function of Eq. 7 per bin: -2 log|det W_i| + sum_r w_r^H Q_{r,i} w_r."""
    M = W.shape[1]
    val = -2.0 * np.log(np.abs(np.linalg.det(W)))
    for r in range(M):
        wr_h = W[:, r, :]                       # w_r^H, [I][M]
        val = val + np.einsum("im,imk,ik->i", wr_h, Q[r], wr_h.conj()).real
    return val


def iss_sweep(W, Q):
    """One ISS sweep (Eqs. 11-16): for r = 0..M-1 in order, W_i <- W_i - z_r w_r^H.

    z_p = (w_p^H Q_p w_r) / (w_r^H Q_p w_r) for p != r and z_r = 1 - (w_r^H Q_r w_r)^{-1/2},
    evaluated with the current W (the rows change after every step). Returns the new
    W and the list of z vectors [I][M] (one per r) for inspection.
    """
    W = W.copy()
    I, M, _ = W.shape
    zs = []
    for r in range(M):
        wr_h = W[:, r, :].copy()                 # w_r^H per bin, [I][M]
        z = np.zeros((I, M), dtype=complex)
        for p in range(M):
            wp_h = W[:, p, :]
            den = np.einsum("im,imk,ik->i", wr_h, Q[p], wr_h.conj()).real   # w_r^H Q_p w_r
            if p != r:
                num = np.einsum("im,imk,ik->i", wp_h, Q[p], wr_h.conj())    # w_p^H Q_p w_r
                safe = den > 0
                z[safe, p] = num[safe] / den[safe]
            else:
                safe = den > 0
                z[safe, p] = 1.0 - 1.0 / np.sqrt(den[safe])
        W = W - z[:, :, None] * wr_h[:, None, :]
        zs.append(z)
    return W, zs


def ip_sweep(W, Q):
    """One IP sweep (Eqs. 9-10): w_r <- (W Q_r)^{-1} e_r, w_r <- w_r (w_r^H Q_r w_r)^{-1/2}."""
    W = W.copy()
    I, M, _ = W.shape
    for r in range(M):
        e = np.zeros(M, dtype=complex)
        e[r] = 1.0
        for i in range(I):
            w = np.linalg.solve(W[i] @ Q[r, i], e)
            w = w / np.sqrt((w.conj() @ Q[r, i] @ w).real)
            W[i, r, :] = w.conj()
    return W


def _delayed_power(y, Ln, n, J):
    """P[i,j'] = sum_{l < L_n, j'+l < J} |y_{(n,l),i,j'+l}|^2 and the count of valid l: the
    delayed power of source n that the all-taps reading of Eq. 18 uses."""
    rows = row_map(Ln)
    I = y.shape[1]
    P = np.zeros((I, J))
    cnt = np.zeros(J)
    for r, (nn, l) in enumerate(rows):
        if nn != n:
            continue
        P[:, : J - l] += np.abs(y[r, :, l:]) ** 2
        cnt[: J - l] += 1.0
    return P, cnt


def update_basis(b, v, y, Ln):
    """Basis MU of Eq. 17 with l over the taps of source n and masked j-l < 0.

    b_{n,i,k} <- b sqrt( sum_{j,l} |y_{n,i,j,l}|^2 v_{n,k,j-l} lam_{n,i,j-l}^{-2}
                       / sum_{j,l} v_{n,k,j-l} lam_{n,i,j-l}^{-1} )
    """
    lam = psd(b, v)
    rows = row_map(Ln)
    J = v.shape[2]
    num = np.zeros_like(b)
    den = np.zeros_like(b)
    for r, (n, l) in enumerate(rows):
        yy = np.abs(y[r, :, l:]) ** 2                  # |y_{n,i,j,l}|^2 for j >= l
        lm = lam[n, :, : J - l]                        # lambda_{n,i,j-l}
        vk = v[n, :, : J - l]                          # v_{n,k,j-l}
        num[n] += np.einsum("ij,kj->ik", yy / lm ** 2, vk)
        den[n] += np.einsum("ij,kj->ik", 1.0 / lm, vk)
    return np.maximum(b * np.sqrt(num / den), FLOOR_NMF), num, den


def update_activation(b, v, y, Ln, mode="all_taps"):
    """Activation MU of Eq. 18.

    "tap0" (as printed): v_{n,k,j} <- v sqrt( sum_i |y_{n,i,j,0}|^2 b lam^{-2} / sum_i b lam^{-1} ).
    "all_taps" (default): the same with |y_{n,i,j,0}|^2 replaced by the delayed power of all
    taps, sum_{l, j+l<J} |y_{n,i,j+l,l}|^2, and the denominator by the number of such taps.
    """
    lam = psd(b, v)
    N, K, J = v.shape
    num = np.zeros_like(v)
    den = np.zeros_like(v)
    rows = row_map(Ln)
    for n in range(N):
        if mode == "all_taps":
            P, cnt = _delayed_power(y, Ln, n, J)
        elif mode == "tap0":
            r0 = rows.index((n, 0))
            P, cnt = np.abs(y[r0]) ** 2, np.ones(J)
        else:
            raise ValueError(mode)
        num[n] = np.einsum("ik,ij->kj", b[n], P / lam[n] ** 2)
        den[n] = np.einsum("ik,ij->kj", b[n], cnt[None, :] / lam[n])
    return np.maximum(v * np.sqrt(num / den), FLOOR_NMF), num, den


def normalise(y, W, b, Ln):
    """Scale normalisation (Eqs. 19-21): mu_{n,l} = sqrt(mean_{i,j} |y|^2),
    y_{n,l} /= mu_{n,l}, the matching row of W /= mu_{n,l}, b_n *= mu_{n,0}^{-2}."""
    rows = row_map(Ln)
    mu = np.sqrt(np.mean(np.abs(y) ** 2, axis=(1, 2)))     # [M]
    mu = np.where(mu > 0, mu, 1.0)
    y = y / mu[:, None, None]
    W = W / mu[None, :, None]
    b = b.copy()
    for r, (n, l) in enumerate(rows):
        if l == 0:
            b[n] = b[n] / mu[r] ** 2
    return y, W, b, mu


def logabsdet(W):
    """log|det W_i| per bin (the log-determinant term of Eq. 5), by LU."""
    return np.linalg.slogdet(W)[1]


def nll(y, lam, W, Ln):
    """Negative log-likelihood of Eq. 5 (constant dropped), masked delays left out:
    sum_{i,j,n,l} (log lam_{n,i,j-l} + |y_{n,i,j,l}|^2 / lam_{n,i,j-l}) - 2J sum_i log|det W_i|."""
    J = y.shape[2]
    total = 0.0
    for r, (n, l) in enumerate(row_map(Ln)):
        lm = lam[n, :, : J - l]
        total += np.sum(np.log(lm) + np.abs(y[r, :, l:]) ** 2 / lm)
    return total - 2.0 * J * np.sum(logabsdet(W))


def source_images(W, y, Ln):
    """MWF source images (Eqs. 23-24) under the square model reduce to
    c_n = sum_l [W_i^{-1}]_{:, (n,l)} y_{(n,l)}; returns [N][M][I][J]."""
    H = np.linalg.inv(W)                                    # [I][M][M]
    rows = row_map(Ln)
    N = max(n for n, _ in rows) + 1
    I, M, _ = W.shape
    out = np.zeros((N, M, I, y.shape[2]), dtype=complex)
    for r, (n, l) in enumerate(rows):
        out[n] += np.einsum("im,ij->mij", H[:, :, r], y[r])
    return out


def mwf_images(W, lam, x, Ln):
    """Literal multichannel Wiener filter of Eqs. 23-24, c_n = H_n Lam_n H_n^H (H Lam H^H)^{-1} x,
    with H_i = W_i^{-1} and Lam the diagonal of delayed PSDs lam_{n,i,j-l} (frames j >= max l)."""
    H = np.linalg.inv(W)
    rows = row_map(Ln)
    N = max(n for n, _ in rows) + 1
    I, M, J = x.shape
    out = np.zeros((N, M, I, J), dtype=complex)
    lmax = max(l for _, l in rows)
    for i in range(I):
        for j in range(lmax, J):
            d = np.array([lam[n, i, j - l] for n, l in rows])
            Rx = H[i] @ np.diag(d) @ H[i].conj().T
            g = np.linalg.solve(Rx, x[i, :, j])
            for n in range(N):
                sel = [r for r, (nn, _) in enumerate(rows) if nn == n]
                Hn = H[i][:, sel]
                out[n, :, i, j] = Hn @ np.diag(d[sel]) @ Hn.conj().T @ g
    return out


def init_state(x_mfj, b0, v0):
    """Initial state: W_i = I (Sec. V-A), y = x, and the given NMF factors."""
    x = np.transpose(np.asarray(x_mfj, dtype=complex), (1, 0, 2))    # [I][M][J]
    I, M, J = x.shape
    W = np.tile(np.eye(M, dtype=complex), (I, 1, 1))
    b = np.maximum(np.asarray(b0, dtype=float), FLOOR_NMF)
    v = np.maximum(np.asarray(v0, dtype=float), FLOOR_NMF)
    return x, W, b, v


def iterate(x, W, b, v, Ln, update="iss", v_mode="all_taps", normalize=True):
    """One iteration in the order of Sec. III: W update (ISS, Eqs. 11-16, or IP, Eqs. 9-10)
    -> basis MU (Eq. 17) on the new rows -> activation MU (Eq. 18) with the new bases ->
    normalisation (Eqs. 19-21)."""
    lam = psd(b, v)
    Q = weighted_covariances(x, delayed_weights(lam, Ln))
    if update == "iss":
        W, _ = iss_sweep(W, Q)
    elif update == "ip":
        W = ip_sweep(W, Q)
    else:
        raise ValueError(update)
    y = demix(W, x)
    b, _, _ = update_basis(b, v, y, Ln)
    v, _, _ = update_activation(b, v, y, Ln, v_mode)
    if normalize:
        y, W, b, _ = normalise(y, W, b, Ln)
    return W, b, v, y


def run(x_mfj, Ln, b0, v0, n_iter, update="iss", v_mode="all_taps", normalize=True, trace=False):
    """Run n_iter iterations from W = I (Sec. V-A). x_mfj is [M][I][J] (per-microphone STFTs).

    Returns a dict with W [I][M][M], y [M][I][J], b, v, cost, logdet [I] and,
    when trace is set, the cost after every iteration.
    """
    x, W, b, v = init_state(x_mfj, b0, v0)
    costs = []
    y = demix(W, x)
    for _ in range(n_iter):
        W, b, v, y = iterate(x, W, b, v, Ln, update, v_mode, normalize)
        if trace:
            costs.append(nll(y, psd(b, v), W, Ln))
    return {"W": W, "y": y, "b": b, "v": v, "logdet": logabsdet(W),
            "cost": nll(y, psd(b, v), W, Ln), "trace": costs}
