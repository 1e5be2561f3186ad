"""Bins longer than one thread block (the cluster bin phase, cluster_bin.cu) against the
FP64 oracle: each shape below exceeds the one-block limit (J = 4096 for M <= 4, 1024 for
M = 5..8), so its bins are split over clusters of 2, 4 or 8 blocks, and taps up to 3 frames
long cross the blocks' chunk boundaries."""
import pytest

from paper_2510_02382_gb300 import synth

from gpu_helpers import cost_close, rel_fro, run_gpu, run_oracle

pytestmark = pytest.mark.gpu

SHAPES = [
    # (M, N, Ln, F, J, B)             cluster blocks
    (3, 2, (2, 1), 3, 5000, 4),        # 4
    (2, 2, (1, 1), 2, 9000, 3),        # 4 (8 frames per thread)
    (6, 2, (3, 3), 3, 1500, 5),        # 2, taps of 3 frames
    (8, 2, (4, 4), 2, 2600, 3),        # 2, taps of 4 frames
    (4, 3, (2, 1, 1), 2, 12000, 4),    # 8
]


@pytest.mark.parametrize("shape", SHAPES)
def test_long_bins_one_iteration(shape):
    M, N, Ln, F, J, B = shape
    mix = synth.random_case(1000 + J, M=M, N=N, F=F, J=J, B=B, Ln=Ln)
    got = run_gpu(mix, 1, path="two_kernel")
    ref = run_oracle(mix, 1)
    assert rel_fro(got["y"], ref["y"]) < 1e-4
    assert rel_fro(got["W"], ref["W"]) < 1e-4
    assert rel_fro(got["T"], ref["b"]) < 1e-4 and rel_fro(got["V"], ref["v"]) < 1e-4
    assert abs(got["logdet"] - ref["logdet"]).max() < 1e-4


@pytest.mark.parametrize("shape", SHAPES[:3])
def test_long_bins_five_iterations_cost(shape):
    M, N, Ln, F, J, B = shape
    mix = synth.random_case(2000 + J, M=M, N=N, F=F, J=J, B=B, Ln=Ln)
    got = run_gpu(mix, 5, path="two_kernel")
    ref = run_oracle(mix, 5)
    ok, err = cost_close(got["cost"], ref["cost"], 1e-5, F, J, M)
    assert ok, err


def test_long_bins_tap0_activation_update():
    mix = synth.random_case(3001, M=3, N=2, F=2, J=6000, B=3, Ln=(2, 1))
    got = run_gpu(mix, 2, v_mode="tap0", path="two_kernel")
    ref = run_oracle(mix, 2, v_mode="tap0")
    assert rel_fro(got["y"], ref["y"]) < 1e-4
    assert rel_fro(got["V"], ref["v"]) < 1e-4


def test_long_j_workload_one_iteration():
    """The long-J benchmark shape (F=513, J=16000: clusters of 8 blocks per bin), one
    iteration against the oracle on the whole mixture."""
    mix = synth.make_mixture(synth.CONFIGS["L1"])
    got = run_gpu(mix, 1, path="two_kernel")
    ref = run_oracle(mix, 1)
    assert rel_fro(got["y"], ref["y"]) < 1e-4
    assert rel_fro(got["T"], ref["b"]) < 1e-4 and rel_fro(got["V"], ref["v"]) < 1e-4


# the size limits of the two bin-phase forms: the largest bin one block holds (8 frames x
# 512 threads for M <= 4, 4 x 256 for M = 5..8), the first frame past it (a cluster of two
# blocks with a ragged second chunk), and the largest bin a cluster of 8 blocks holds
LIMIT_SHAPES = [
    # (M, N, Ln, F, J, B)
    (4, 2, (2, 2), 2, 4096, 4),        # one block, every thread full
    (6, 2, (3, 3), 2, 1024, 3),        # one block, M = 5..8
    (3, 2, (2, 1), 2, 4097, 3),        # cluster of 2, one frame in the last chunk row
    (7, 3, (3, 2, 2), 1, 1025, 3),     # cluster of 2, M = 5..8
    (3, 2, (2, 1), 1, 16384, 3),       # cluster of 8, M = 3..8 limit
    (2, 2, (1, 1), 1, 32768, 2),       # cluster of 8, M = 2 limit
]


@pytest.mark.parametrize("shape", LIMIT_SHAPES, ids=lambda s: f"M{s[0]}J{s[4]}")
def test_size_limits_one_iteration(shape):
    M, N, Ln, F, J, B = shape
    mix = synth.random_case(4000 + J, M=M, N=N, F=F, J=J, B=B, Ln=Ln)
    got = run_gpu(mix, 1, path="two_kernel")
    ref = run_oracle(mix, 1)
    assert rel_fro(got["y"], ref["y"]) < 1e-4
    assert rel_fro(got["W"], ref["W"]) < 1e-4
    assert rel_fro(got["T"], ref["b"]) < 1e-4 and rel_fro(got["V"], ref["v"]) < 1e-4
    assert abs(got["logdet"] - ref["logdet"]).max() < 1e-4
    assert rel_fro(got["images"], ref["images"]) < 1e-4
