"""ctfmnmf_cost_noalloc against ctfmnmf_cost (GPU).

The no-allocation entry point serves callers that cannot allocate device memory where they
need the cost (for example a real-time audio thread, where an allocation may synchronise
the device, or code running inside an allocator callback). It must give the same
negative log-likelihood as the handle-based ctfmnmf_cost, on consecutive calls that share
its static scratch. Collected last on purpose, so that a run stopping at the first failure
has run every other test before it.
"""
import numpy as np
import pytest

from paper_2510_02382_gb300 import synth

from gpu_helpers import cost_close, make_solver

pytestmark = pytest.mark.gpu


def _state(mix, n_iter):
    import torch
    s = make_solver(mix)
    s.load_stft(torch.from_numpy(mix.X).cuda())
    s.set_init(torch.from_numpy(mix.T0).cuda(), torch.from_numpy(mix.V0).cuda())
    s.iterate(n_iter)
    ref = s.cost()
    Y = s.get_demixed()
    T, V = s.get_nmf()
    ld = s.get_logdet()
    torch.cuda.synchronize()
    s.close()
    return ref, Y, T, V, ld


def test_cost_noalloc_matches_cost_on_consecutive_calls():
    import torch
    from paper_2510_02382_gb300.api import cost_noalloc
    a = synth.random_case(51, M=3, N=2, F=129, J=256, B=4, Ln=(2, 1))
    b = synth.random_case(52, M=4, N=3, F=65, J=301, B=10, Ln=(2, 1, 1))
    ref_a, *args_a = _state(a, 5)
    ref_b, *args_b = _state(b, 3)
    out = torch.empty(1, dtype=torch.float64, device="cuda")
    for ref, args, mix in [(ref_a, args_a, a), (ref_a, args_a, a), (ref_b, args_b, b)]:
        out.fill_(float("nan"))
        cost_noalloc(*args, mix.Ln, out)
        val = float(out.item())
        sp = mix.spec
        ok, err = cost_close(val, ref, 1e-5, sp.F, sp.J, sp.M)
        assert np.isfinite(val) and ok, (val, ref, err)


def test_cost_noalloc_rejects_too_many_bins():
    import torch
    from paper_2510_02382_gb300.api import CtfMnmfError, cost_noalloc
    F = 16385
    Y = torch.zeros((2, F, 4), dtype=torch.complex64, device="cuda")
    T = torch.ones((2, F, 1), dtype=torch.float32, device="cuda")
    V = torch.ones((2, 1, 4), dtype=torch.float32, device="cuda")
    ld = torch.zeros((F,), dtype=torch.float64, device="cuda")
    out = torch.empty(1, dtype=torch.float64, device="cuda")
    with pytest.raises(CtfMnmfError) as e:
        cost_noalloc(Y, T, V, ld, [1, 1], out)
    assert e.value.name == "EINVAL" and "16384" in str(e.value)
