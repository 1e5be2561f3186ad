"""FP64 reference gradient of unrolled CTF-MNMF-ISS separation (PyTorch autograd, CPU).

TEST INFRASTRUCTURE ONLY. Only the test suite and the CPU legs of the benchmark may
import it; the library never does, and nothing here is shared with the CUDA code.

The paper (Xie et al., APSIPA ASC 2025) differentiates nothing: this module states the
same iteration as ``ctfmnmf_oracle`` (Sec. III: the ISS sweep of Eqs. 11-16 on the
weighted covariances of Eq. 8, the basis MU of Eq. 17, the activation MU of Eq. 18 in the
all-taps form, the normalisation of Eqs. 19-21, the projection-back images of Eq. 24)
written with differentiable complex128 torch operations, so that torch.autograd gives the
gradient of a loss on the separated images with respect to the observation x and the
initial factors b0, v0. It is written independently of the NumPy oracle (covariance form
again, but its own code) and is pinned against central finite differences of that oracle.

Gradient convention (PyTorch's): for a real loss L and a complex input z = a + ib the
gradient is dL/da + i dL/db.

Loss used by the differentiable workload: the mean over sources n, microphones m, bins i
and frames j of |c_hat_n - c_n|^2 (the MSE of the separated images to the true images),
with no permutation search.
"""
from __future__ import annotations

import torch

FLOOR_NMF = 1e-12   # b and v after each multiplicative update
FLOOR_PSD = 1e-18   # lambda where it is formed


def _rows(Ln):
    out = []
    for n, L in enumerate(Ln):
        out.extend((n, l) for l in range(L))
    return out


def _lam(b, v):
    """lambda_{n,i,j} = sum_k b v, floored (the NMF source model, Sec. II)."""
    return torch.clamp(torch.einsum("nik,nkj->nij", b, v), min=FLOOR_PSD)


def _phi(lam, Ln):
    """phi[r,i,j] = 1/lambda_{n,i,j-l} for j >= l, 0 for the masked frames j < l."""
    N, I, J = lam.shape
    rows = []
    for n, l in _rows(Ln):
        pad = torch.zeros((I, l), dtype=lam.dtype)
        rows.append(torch.cat([pad, 1.0 / lam[n, :, : J - l]], dim=1))
    return torch.stack(rows)


def _iss(W, Q):
    """ISS sweep of Eqs. 11-16 on W [I][M][M] (row r = w_r^H) with Q [M][I][M][M]:
    z_p = w_p^H Q_p w_r / w_r^H Q_p w_r (p != r), z_r = 1 - (w_r^H Q_r w_r)^{-1/2}."""
    I, M, _ = W.shape
    for r in range(M):
        wr = W[:, r, :]
        zs = []
        for p in range(M):
            den = torch.einsum("im,imk,ik->i", wr, Q[p], wr.conj()).real
            if p != r:
                num = torch.einsum("im,imk,ik->i", W[:, p, :], Q[p], wr.conj())
                z = torch.where(den > 0, num / torch.where(den > 0, den, 1.0), 0.0)
            else:
                z = torch.where(den > 0, 1.0 - torch.rsqrt(torch.where(den > 0, den, 1.0)), 0.0)
                z = z.to(W.dtype)
            zs.append(z)
        z = torch.stack(zs, dim=1)                                  # [I][M]
        W = W - z[:, :, None] * wr[:, None, :]
    return W


def _delayed_power(y, Ln, n, J):
    """S[i,j] = sum_{l < L_n, j+l < J} |y_{(n,l), j+l}|^2 and the count of such l."""
    I = y.shape[1]
    S = torch.zeros((I, J), dtype=torch.float64)
    cnt = torch.zeros(J, dtype=torch.float64)
    for r, (nn, l) in enumerate(_rows(Ln)):
        if nn != n:
            continue
        S = S + torch.cat([y[r, :, l:].abs() ** 2, torch.zeros((I, l), dtype=torch.float64)], dim=1)
        cnt = cnt + torch.cat([torch.ones(J - l, dtype=torch.float64), torch.zeros(l, dtype=torch.float64)])
    return S, cnt


def _basis_mu(b, v, y, Ln):
    """Eq. 17 (taps of the own source, masked delays), in terms of lag j' = j - l."""
    lam = _lam(b, v)
    N, K, J = v.shape
    out = []
    for n in range(N):
        S, cnt = _delayed_power(y, Ln, n, J)
        num = torch.einsum("ij,kj->ik", S / lam[n] ** 2, v[n])
        den = torch.einsum("ij,kj->ik", cnt[None, :] / lam[n], v[n])
        out.append(torch.clamp(b[n] * torch.sqrt(num / den), min=FLOOR_NMF))
    return torch.stack(out)


def _activation_mu(b, v, y, Ln):
    """Eq. 18 in the all-taps form (delayed power of every tap of the source)."""
    lam = _lam(b, v)
    N, K, J = v.shape
    out = []
    for n in range(N):
        S, cnt = _delayed_power(y, Ln, n, J)
        num = torch.einsum("ik,ij->kj", b[n], S / lam[n] ** 2)
        den = torch.einsum("ik,ij->kj", b[n], cnt[None, :] / lam[n])
        out.append(torch.clamp(v[n] * torch.sqrt(num / den), min=FLOOR_NMF))
    return torch.stack(out)


def _normalise(y, W, b, Ln):
    """Eqs. 19-21: mu_r = sqrt(mean_{i,j} |y_r|^2); y_r, row r of W divided by mu_r,
    b_n multiplied by mu_{(n,0)}^{-2}."""
    mu = torch.sqrt(torch.mean(y.abs() ** 2, dim=(1, 2)))
    mu = torch.where(mu > 0, mu, torch.ones_like(mu))
    y = y / mu[:, None, None]
    W = W / mu[None, :, None]
    scales = []
    for n in range(b.shape[0]):
        r0 = _rows(Ln).index((n, 0))
        scales.append(mu[r0] ** -2)
    b = b * torch.stack(scales)[:, None, None]
    return y, W, b


def separate(x_mfj, b0, v0, Ln, n_iter):
    """Images c_hat [N][M][I][J] after n_iter iterations from W = I (Eq. 24, projection-back).

    x_mfj: complex128 [M][I][J]; b0 [N][I][K], v0 [N][K][J] float64 (floored on entry).
    """
    x = x_mfj.permute(1, 0, 2)                                      # [I][M][J]
    I, M, J = x.shape
    W = torch.eye(M, dtype=torch.complex128).repeat(I, 1, 1)
    b = torch.clamp(b0, min=FLOOR_NMF)
    v = torch.clamp(v0, min=FLOOR_NMF)
    y = torch.einsum("irm,imj->rij", W, x)
    for _ in range(n_iter):
        lam = _lam(b, v)
        phi = _phi(lam, Ln).to(torch.complex128)
        Q = torch.einsum("rij,imj,ikj->rimk", phi, x, x.conj()) / J   # Eq. 8
        W = _iss(W, Q)
        y = torch.einsum("irm,imj->rij", W, x)                         # Eq. 4
        b = _basis_mu(b, v, y, Ln)
        v = _activation_mu(b, v, y, Ln)
        y, W, b = _normalise(y, W, b, Ln)
    H = torch.linalg.inv(W)
    rows = _rows(Ln)
    N = max(n for n, _ in rows) + 1
    imgs = [torch.zeros((M, I, J), dtype=torch.complex128) for _ in range(N)]
    for r, (n, _) in enumerate(rows):
        imgs[n] = imgs[n] + torch.einsum("im,ij->mij", H[:, :, r], y[r])
    return torch.stack(imgs)


def mse(c_hat, c_true):
    """Mean over all elements of |c_hat - c_true|^2."""
    return torch.mean((c_hat - c_true).abs() ** 2)


def loss_and_gradient(x_mfj, b0, v0, c_true, Ln, n_iter):
    """FP64 loss and its gradient with respect to x (complex, PyTorch convention), b0, v0.

    Inputs are NumPy arrays (any precision; upcast here). Returns (loss, gx, gb0, gv0) as
    NumPy arrays / float.
    """
    x = torch.tensor(x_mfj, dtype=torch.complex128, requires_grad=True)
    b = torch.tensor(b0, dtype=torch.float64, requires_grad=True)
    v = torch.tensor(v0, dtype=torch.float64, requires_grad=True)
    c = torch.tensor(c_true, dtype=torch.complex128)
    loss = mse(separate(x, b, v, Ln, n_iter), c)
    loss.backward()

    def grad(t):   # an input the loss does not reach (no iteration) has gradient 0
        return t.grad.numpy() if t.grad is not None else torch.zeros_like(t).detach().numpy()

    return float(loss.detach()), grad(x), grad(b), grad(v)
