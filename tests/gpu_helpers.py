"""Shared helpers of the GPU tests: run the CUDA library and the oracle on one mixture."""
import numpy as np

from oracle import ctfmnmf_oracle as O


def make_solver(mix, path="auto", **kw):
    """A solver for `mix`; skips the test when the requested path does not fit the shape."""
    import pytest
    from paper_2510_02382_gb300.api import CTFMNMF, CtfMnmfError
    sp = mix.spec
    try:
        return CTFMNMF(sp.M, sp.N, max(mix.Ln), sp.B, sp.F, sp.J, Ln=mix.Ln, path=path, **kw)
    except CtfMnmfError as e:
        if e.name == "EUNSUPPORTED":
            pytest.skip(f"{path} path unavailable for this shape: {e}")
        raise


def run_gpu(mix, n_iter, v_mode="all_taps", normalize=True, use_graph=True, set_init=True, path="auto", **kw):
    import torch
    s = make_solver(mix, path=path, v_update=v_mode, normalize=normalize, use_graph=use_graph, **kw)
    X = torch.from_numpy(mix.X).cuda()
    s.load_stft(X)
    if set_init:
        s.set_init(torch.from_numpy(mix.T0).cuda(), torch.from_numpy(mix.V0).cuda())
    s.iterate(n_iter)
    out = {
        "y": s.get_demixed().cpu().numpy(),
        "W": s.get_demix_matrix().cpu().numpy(),
        "logdet": s.get_logdet().cpu().numpy(),
        "cost": s.cost(),
        "images": s.get_separated().cpu().numpy(),
    }
    T, V = s.get_nmf()
    out["T"], out["V"] = T.cpu().numpy(), V.cpu().numpy()
    s.close()
    return out


def run_oracle(mix, n_iter, v_mode="all_taps", normalize=True, T0=None, V0=None):
    T0 = mix.T0 if T0 is None else T0
    V0 = mix.V0 if V0 is None else V0
    ref = O.run(mix.X, mix.Ln, T0, V0, n_iter, v_mode=v_mode, normalize=normalize)
    ref["images"] = O.source_images(ref["W"], ref["y"], mix.Ln)
    return ref


def rel_fro(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(np.asarray(b)), 1e-300))


def cost_close(c_gpu, c_ref, tol, F, J, M):
    """Cost agreement scaled by max(|L_ref|, F*J*M): the cost can sit near zero, where a
    purely relative test is ill-conditioned; F*J*M is the number of terms of Eq. 5."""
    scale = max(abs(c_ref), float(F) * J * M)
    return abs(c_gpu - c_ref) <= tol * scale, abs(c_gpu - c_ref) / scale


def per_bin_rel(a, b):
    """Largest per-bin relative Frobenius error of rows [M][F][J] (bin = axis 1): a whole-tensor
    norm dilutes one wrong bin among F, this does not."""
    a, b = np.asarray(a), np.asarray(b)
    num = np.sqrt(np.sum(np.abs(a - b) ** 2, axis=(0, 2)))
    den = np.maximum(np.sqrt(np.sum(np.abs(b) ** 2, axis=(0, 2))), 1e-300)
    return float(np.max(num / den))


def per_bin_logdet(a, b):
    """Largest per-bin |delta log|det W_i||, relative to max(1, |log|det W_i||)."""
    a, b = np.asarray(a), np.asarray(b)
    return float(np.max(np.abs(a - b) / np.maximum(1.0, np.abs(b))))


def expected_costs(name):
    """Stored FP64 oracle costs of a full-size workload (tests/golden/expected_costs.json, written
    by tests/golden/make_expected.py, which calls only the oracle), or a skip if absent."""
    import json
    import os
    import pytest
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "expected_costs.json")
    if not os.path.exists(path):
        pytest.skip("expected_costs.json not generated")
    with open(path) as f:
        return json.load(f)["entries"][name]


def check_fingerprint(entry, mix):
    """The stored costs belong to this mixture: the generator still draws the same inputs (to
    the last few bits, which numpy's elementary functions may round differently per platform)."""
    fp = entry["fingerprint"]
    got = {"x_power": float(np.sum(np.abs(mix.X.astype(np.complex128)) ** 2)),
           "t0_sum": float(np.sum(mix.T0, dtype=np.float64)), "v0_sum": float(np.sum(mix.V0, dtype=np.float64))}
    for k, v in fp.items():
        assert abs(got[k] - v) <= 1e-9 * abs(v), (k, got[k], v)
