"""The seeded input generator (CPU): the workload shapes, the ragged batch's draws,
determinism, and the mixture as the sum of its source images (Eq. 2) plus the stated noise."""
import numpy as np
import pytest

from paper_2510_02382_gb300 import synth


@pytest.mark.parametrize("name,shape,taps", [
    ("C1", dict(N=2, M=3, L=2, F=129, J=256, B=4, iters=10), [2, 1]),
    ("C2", dict(N=2, M=3, L=4, F=513, J=1000, B=10, iters=100), [2, 1]),
    ("C3", dict(N=3, M=4, L=8, F=513, J=2000, B=16, iters=100), [2, 1, 1]),
    ("C5", dict(N=2, M=3, L=4, F=257, J=500, B=8, iters=20), [2, 1]),
    ("L1", dict(N=2, M=3, L=4, F=513, J=16000, B=10, iters=10), [2, 1]),
    ("P4", dict(N=2, M=4, F=513, J=501, B=3), [2, 2]),
    ("P6", dict(N=2, M=6, F=513, J=501, B=3), [3, 3]),
    ("P8", dict(N=2, M=8, F=513, J=501, B=3), [4, 4]),
])
def test_workload_shapes_and_taps(name, shape, taps):
    sp = synth.CONFIGS[name]
    for k, v in shape.items():
        assert getattr(sp, k) == v, (name, k)
    assert sp.taps() == taps and sum(sp.taps()) == sp.M


def test_workload_generator_parameters():
    assert synth.CONFIGS["C2"].snr_db == 30.0 and synth.CONFIGS["C2"].tau == 3.0
    c3 = synth.CONFIGS["C3"]
    assert (c3.gamma_shape, c3.gamma_scale, c3.tau) == (0.5, 2.0, 5.0)
    assert synth.CONFIGS["C1"].tau == 1.5 and synth.CONFIGS["C1"].snr_db is None


def test_batched_specs_follow_the_ragged_recipe():
    specs = synth.batched_specs()
    assert len(specs) == 64 and [s.seed for s in specs] == list(range(64))
    for s in specs:
        assert 300 <= s.J <= 3000 and s.N in (2, 3) and s.M == s.N + 1
        assert s.L in (2, 4, 8) and s.tau == {2: 1.5, 4: 3.0, 8: 5.0}[s.L]
        assert (s.F, s.B, s.iters) == (513, 10, 50)
        assert sum(s.taps()) == s.M and max(s.taps()) <= s.L
    # the first three draws of each seed's generator fix J, N and L
    rng = np.random.default_rng(7)
    assert (specs[7].J, specs[7].N, specs[7].L) == (int(rng.integers(300, 3001)), int(rng.choice([2, 3])),
                                                    int(rng.choice([2, 4, 8])))
    # the batch is ragged in every drawn dimension
    assert len({s.J for s in specs}) > 32 and {s.N for s in specs} == {2, 3} and {s.L for s in specs} == {2, 4, 8}
    assert [s.seed for s in synth.grad_specs()] == list(range(16))


def test_mixture_is_deterministic_per_seed():
    a = synth.random_case(5, M=3, N=2, F=4, J=20, B=2)
    b = synth.random_case(5, M=3, N=2, F=4, J=20, B=2)
    c = synth.random_case(6, M=3, N=2, F=4, J=20, B=2)
    for k in ("X", "images", "T0", "V0"):
        assert np.array_equal(getattr(a, k), getattr(b, k))
    assert not np.array_equal(a.X, c.X)
    assert a.X.dtype == np.complex64 and a.T0.dtype == np.float32 and a.V0.dtype == np.float32
    assert a.X.shape == (3, 4, 20) and a.images.shape == (2, 3, 4, 20)
    for f in (a.T0, a.V0):
        assert f.min() >= 0.1 and f.max() < 1.0


def test_mixture_is_the_sum_of_its_source_images():
    """Without noise the observation is exactly the sum over sources of the source images
    (Eq. 2), up to the complex64 rounding of each."""
    m = synth.random_case(3, M=4, N=2, F=5, J=40, B=3, Ln=(2, 2))
    s = m.images.astype(np.complex128).sum(axis=0)
    err = np.max(np.abs(m.X.astype(np.complex128) - s)) / np.max(np.abs(s))
    assert err < 1e-6


def test_noise_level_matches_the_stated_snr():
    sp = synth.scaled(synth.CONFIGS["C2"], F=16, J=400)
    noisy = synth.make_mixture(sp)
    clean = noisy.images.astype(np.complex128).sum(axis=0)
    n = noisy.X.astype(np.complex128) - clean
    snr = 10 * np.log10(np.mean(np.abs(clean) ** 2) / np.mean(np.abs(n) ** 2))
    assert abs(snr - 30.0) < 0.5, snr


def test_stored_oracle_costs_belong_to_the_generated_mixtures():
    """tests/golden/expected_costs.json (written by tests/golden/make_expected.py from the
    oracle) was made from the inputs this generator draws today: the fingerprint of every
    stored mixture matches, and the stored C4 samples are the seeds the script picks."""
    import importlib.util
    import json
    import os
    from gpu_helpers import check_fingerprint
    here = os.path.dirname(os.path.abspath(__file__))
    with open(os.path.join(here, "golden", "expected_costs.json")) as f:
        entries = json.load(f)["entries"]
    spec = importlib.util.spec_from_file_location("make_expected", os.path.join(here, "golden", "make_expected.py"))
    me = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(me)
    assert sorted(k for k in entries if k != "C3") == sorted(sp.name for sp in me.c4_samples())
    specs = {sp.name: sp for sp in synth.batched_specs()}
    for name, e in entries.items():
        sp = synth.CONFIGS["C3"] if name == "C3" else specs[name]
        check_fingerprint(e, synth.make_mixture(sp))
