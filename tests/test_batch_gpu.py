"""The batched form (ctfmnmf_batch_*) against the FP64 oracle and the single-mixture path."""
import numpy as np
import pytest

from paper_2510_02382_gb300 import synth

from gpu_helpers import (check_fingerprint, cost_close, expected_costs, make_solver, per_bin_rel, rel_fro,
                         run_oracle)

pytestmark = pytest.mark.gpu

RAGGED = [
    # (M, N, Ln, F, J, B)
    (3, 2, (2, 1), 9, 37, 4),
    (4, 3, (2, 1, 1), 7, 611, 10),
    (3, 2, (2, 1), 5, 1500, 10),
    (2, 2, (1, 1), 11, 300, 3),
    (6, 2, (3, 3), 4, 260, 16),
    (4, 2, (2, 2), 3, 2900, 32),
]


def _loaded(mixes, **kw):
    import torch
    out = []
    for mix in mixes:
        s = make_solver(mix, path="two_kernel", **kw)
        s.load_stft(torch.from_numpy(mix.X).cuda())
        s.set_init(torch.from_numpy(mix.T0).cuda(), torch.from_numpy(mix.V0).cuda())
        out.append(s)
    return out


def test_batch_of_ragged_mixtures_matches_oracle():
    from paper_2510_02382_gb300.api import Batch
    mixes = [synth.random_case(300 + k, M=M, N=N, F=F, J=J, B=B, Ln=Ln)
             for k, (M, N, Ln, F, J, B) in enumerate(RAGGED)]
    solvers = _loaded(mixes)
    batch = Batch(solvers)
    info = batch.info()
    assert info["mixtures"] == len(mixes) and info["bin_classes"] >= 1
    batch.iterate(1)
    for s, mix in zip(solvers, mixes):
        r = run_oracle(mix, 1)
        assert rel_fro(s.get_demixed().cpu().numpy(), r["y"]) < 1e-4
    batch.iterate(4)                     # 5 iterations in total
    for s, mix in zip(solvers, mixes):
        r = run_oracle(mix, 5)
        sp = mix.spec
        ok, err = cost_close(s.cost(), r["cost"], 1e-5, sp.F, sp.J, sp.M)
        assert ok, (sp, err)
        T, V = s.get_nmf()
        assert rel_fro(V.cpu().numpy(), r["v"]) < 1e-3 and rel_fro(T.cpu().numpy(), r["b"]) < 1e-3
    batch.close()
    for s in solvers:
        s.close()


def test_batch_creation_leaves_handles_unchanged_and_matches_single_path():
    from paper_2510_02382_gb300.api import Batch
    mixes = [synth.random_case(400 + k, M=3, N=2, F=6, J=J, B=4, Ln=(2, 1)) for k, J in enumerate((100, 700))]
    solvers = _loaded(mixes)
    before = [s.get_demixed().cpu().numpy() for s in solvers]
    batch = Batch(solvers)
    after = [s.get_demixed().cpu().numpy() for s in solvers]
    for a, b in zip(before, after):
        assert np.array_equal(a, b)
    batch.iterate(3)
    ys = [s.get_demixed().cpu().numpy() for s in solvers]
    single = _loaded(mixes)
    for s, y in zip(single, ys):
        s.iterate(3)
        assert rel_fro(s.get_demixed().cpu().numpy(), y) < 1e-5
        s.close()
    batch.close()
    for s in solvers:
        s.close()


def test_batch_rejects_unloaded_member():
    from paper_2510_02382_gb300.api import Batch, CtfMnmfError
    mixes = [synth.random_case(500 + k, M=3, N=2, F=4, J=64, B=3, Ln=(2, 1)) for k in range(2)]
    solvers = _loaded(mixes[:1]) + [make_solver(mixes[1], path="two_kernel")]
    batch = Batch(solvers)
    with pytest.raises(CtfMnmfError) as e:
        batch.iterate(1)
    assert e.value.name == "ESTATE"
    batch.close()
    for s in solvers:
        s.close()


def test_batched_workload_sampled_mixtures():
    """The 64-mixture ragged workload (J in [300, 3000], N in {2,3}, M = N+1, L in {2,4,8},
    F = 513, B = 10): one batched iteration, three sampled mixtures checked against the oracle."""
    from paper_2510_02382_gb300.api import Batch
    specs = synth.batched_specs()
    mixes = [synth.make_mixture(sp) for sp in specs]
    solvers = _loaded(mixes)
    batch = Batch(solvers)
    batch.iterate(1)
    for k in (0, 17, 63):
        r = run_oracle(mixes[k], 1)
        y = solvers[k].get_demixed().cpu().numpy()
        assert rel_fro(y, r["y"]) < 1e-4, k
        assert per_bin_rel(y, r["y"]) < 1e-3, k
    batch.close()
    for s in solvers:
        s.close()


def test_batch_ragged_buffers_match_per_handle_calls():
    """ctfmnmf_batch_load_stft / _set_init / _get_separated over one concatenated buffer
    with offsets give exactly what the per-handle calls give."""
    import torch
    from paper_2510_02382_gb300.api import Batch
    mixes = [synth.random_case(700 + k, M=M, N=N, F=F, J=J, B=B, Ln=Ln)
             for k, (M, N, Ln, F, J, B) in enumerate(RAGGED[:4])]
    # per-handle reference
    ref_solvers = _loaded(mixes)
    ref_batch = Batch(ref_solvers)
    ref_batch.iterate(3)
    ref = [s.get_separated().cpu().numpy() for s in ref_solvers]
    ref_batch.close()
    # the same through ragged buffers
    solvers = [make_solver(m, path="two_kernel") for m in mixes]
    batch = Batch(solvers)
    X = torch.from_numpy(np.concatenate([m.X.ravel() for m in mixes])).cuda()
    T0 = torch.from_numpy(np.concatenate([m.T0.ravel() for m in mixes])).cuda()
    V0 = torch.from_numpy(np.concatenate([m.V0.ravel() for m in mixes])).cuda()
    xo = np.cumsum([0] + [m.X.size for m in mixes])[:-1]
    to = np.cumsum([0] + [m.T0.size for m in mixes])[:-1]
    vo = np.cumsum([0] + [m.V0.size for m in mixes])[:-1]
    co = np.cumsum([0] + [m.images.size for m in mixes])
    batch.load_stft(X, xo)
    batch.set_init(T0, to, V0, vo)
    batch.iterate(3)
    C = torch.empty(int(co[-1]), dtype=torch.complex64, device="cuda")
    batch.get_separated(C, co[:-1])
    torch.cuda.synchronize()
    Cn = C.cpu().numpy()
    for k, m in enumerate(mixes):
        assert np.array_equal(Cn[co[k]:co[k + 1]].reshape(m.images.shape), ref[k]), k
    batch.close()
    for s in solvers + ref_solvers:
        s.close()


def test_batched_workload_50_iterations_cost_on_sampled_mixtures():
    """The whole 64-mixture workload in one batch, 50 iterations as the benchmark runs it; the
    costs of four sampled mixtures (the smallest and the largest J, the first M = 4 and the
    first M = 3) within 1e-5 of the FP64 oracle after 10 iterations and 1e-3 after 50
    (stored oracle costs, tests/golden/expected_costs.json)."""
    from paper_2510_02382_gb300.api import Batch
    import json
    import os
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "expected_costs.json")
    if not os.path.exists(path):
        pytest.skip("expected_costs.json not generated")
    with open(path) as f:
        names = [k for k in json.load(f)["entries"] if k.startswith("B")]
    assert len(names) >= 4
    specs = synth.batched_specs()
    mixes = [synth.make_mixture(sp) for sp in specs]
    solvers = _loaded(mixes)
    batch = Batch(solvers)
    batch.iterate(10)
    errs = {}
    for name in names:
        exp = expected_costs(name)
        k = exp["seed"]
        check_fingerprint(exp, mixes[k])
        sp = specs[k]
        ok, err = cost_close(solvers[k].cost(), exp["iss_cost"]["10"], 1e-5, sp.F, sp.J, sp.M)
        errs[(name, 10)] = err
        assert ok, (name, err)
    batch.iterate(40)
    for name in names:
        exp = expected_costs(name)
        k = exp["seed"]
        sp = specs[k]
        ok, err = cost_close(solvers[k].cost(), exp["iss_cost"]["50"], 1e-3, sp.F, sp.J, sp.M)
        errs[(name, 50)] = err
        assert ok, (name, err)
    print("batched cost errors:", {f"{n}@{it}": f"{e:.2e}" for (n, it), e in errs.items()})
    batch.close()
    for s in solvers:
        s.close()


@pytest.mark.parametrize("plan", range(6))
def test_every_batch_plan_matches_oracle(plan, monkeypatch):
    """Each candidate plan of the batch autotuner (CTFMNMF_BATCH_PLAN keeps one): single-mixture
    shapes, eight strided frames, eight consecutive frames where the taps allow (with the
    strided kernel for the rest), each merged or not; ragged mixtures against the oracle."""
    from paper_2510_02382_gb300.api import Batch
    monkeypatch.setenv("CTFMNMF_BATCH_PLAN", str(plan))
    mixes = [synth.random_case(800 + k, M=M, N=N, F=F, J=J, B=B, Ln=Ln)
             for k, (M, N, Ln, F, J, B) in enumerate(RAGGED)]
    solvers = _loaded(mixes)
    batch = Batch(solvers)
    assert batch.info()["plan"] == plan
    batch.iterate(2)
    for s, mix in zip(solvers, mixes):
        r = run_oracle(mix, 2)
        y = s.get_demixed().cpu().numpy()
        assert rel_fro(y, r["y"]) < 1e-4 and per_bin_rel(y, r["y"]) < 1e-3, mix.spec
        sp = mix.spec
        ok, err = cost_close(s.cost(), r["cost"], 1e-5, sp.F, sp.J, sp.M)
        assert ok, (sp, err)
    batch.close()
    for s in solvers:
        s.close()
