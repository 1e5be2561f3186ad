"""ctfmnmf_options fields and the CTFMNMF_DEBUG build (GPU).

eps_floor      the floor of T and V (reading of the unstated floors) matches the oracle run with
               the same floor;
check_finite   a state driven to NaN/Inf (FP32 overflow of |y|^2 from a finite but huge STFT) is
               reported as ENONFINITE by the next synchronising call, and not without the scan;
deterministic_reduce
               the long-J cluster path repeats bit for bit with fixed-order sums;
CTFMNMF_DEBUG  a batched work-list entry naming a bin outside its mixture is caught by the
               device bounds check (EBOUNDS, no memory access with the bad index); a release
               build refuses to change a work list.
No case faults the GPU: the non-finite values are ordinary IEEE arithmetic and the bad index is
checked before it is used.
"""
import os
import subprocess
import sys

import numpy as np
import pytest

from oracle import ctfmnmf_oracle as O
from paper_2510_02382_gb300 import synth

from gpu_helpers import cost_close, make_solver, rel_fro

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _run(mix, n_iter, T0=None, V0=None, **kw):
    import torch
    s = make_solver(mix, path="two_kernel", **kw)
    s.load_stft(torch.from_numpy(mix.X).cuda())
    s.set_init(torch.from_numpy(mix.T0 if T0 is None else T0).cuda(),
               torch.from_numpy(mix.V0 if V0 is None else V0).cuda())
    s.iterate(n_iter)
    return s


def test_eps_floor_matches_the_oracle_with_the_same_floor(monkeypatch):
    mix = synth.random_case(91, M=3, N=2, F=6, J=120, B=4, Ln=(2, 1))
    T0 = (mix.T0 * 1e-3).astype(np.float32)           # below the floor: floored at set_init
    floor = 1e-3
    s = _run(mix, 3, T0=T0, eps_floor=floor)
    y, cost = s.get_demixed().cpu().numpy(), s.cost()
    T, V = (t.cpu().numpy() for t in s.get_nmf())
    s.close()
    monkeypatch.setattr(O, "FLOOR_NMF", floor)
    r = O.run(mix.X, mix.Ln, T0, mix.V0, 3)
    assert rel_fro(y, r["y"]) < 1e-4
    ok, err = cost_close(cost, r["cost"], 1e-5, 6, 120, 3)
    assert ok, err
    assert rel_fro(V, r["v"]) < 1e-4 and rel_fro(T, r["b"]) < 1e-4
    assert np.min(T) >= np.float32(floor) * (1 - 1e-6) and np.min(V) >= np.float32(floor) * (1 - 1e-6)


def test_check_finite_reports_a_state_driven_to_nan():
    from paper_2510_02382_gb300.api import CtfMnmfError
    mix = synth.random_case(92, M=3, N=2, F=5, J=64, B=3, Ln=(2, 1))
    mix.X = (mix.X * np.float32(1e25)).astype(np.complex64)     # finite, but |y|^2 overflows FP32
    assert np.all(np.isfinite(mix.X))
    quiet = _run(mix, 2)
    quiet.synchronize()                                        # no scan: nothing reported
    quiet.close()
    s = _run(mix, 2, check_finite=True)
    with pytest.raises(CtfMnmfError) as e:
        s.synchronize()
    assert e.value.name == "ENONFINITE"
    with pytest.raises(CtfMnmfError) as e:
        s.iterate(1)                                           # the state must be reloaded
    assert e.value.name == "ESTATE"
    good = synth.random_case(93, M=3, N=2, F=5, J=64, B=3, Ln=(2, 1))
    import torch
    s.load_stft(torch.from_numpy(good.X).cuda())
    s.set_init(torch.from_numpy(good.T0).cuda(), torch.from_numpy(good.V0).cuda())
    s.iterate(2)
    s.synchronize()
    r = O.run(good.X, good.Ln, good.T0, good.V0, 2)
    assert rel_fro(s.get_demixed().cpu().numpy(), r["y"]) < 1e-4
    s.close()


def test_deterministic_reduce_repeats_bit_for_bit_on_the_cluster_path():
    mix = synth.random_case(94, M=3, N=2, F=4, J=5000, B=4, Ln=(2, 1))   # J > 4096: a cluster per bin
    outs = []
    for _ in range(2):
        s = _run(mix, 3, deterministic_reduce=True)
        assert s.bin_shape() == (0, 0)                                   # the cluster bin phase
        outs.append((s.get_demixed().cpu().numpy(), s.cost()))
        s.close()
    assert np.array_equal(outs[0][0], outs[1][0]) and outs[0][1] == outs[1][1]
    s = _run(mix, 3, deterministic_reduce=False)
    assert rel_fro(s.get_demixed().cpu().numpy(), outs[0][0]) < 1e-5
    s.close()


def test_release_build_refuses_to_change_a_work_list():
    from paper_2510_02382_gb300.api import Batch, CtfMnmfError
    mixes = [synth.random_case(95 + k, M=3, N=2, F=4, J=64, B=3, Ln=(2, 1)) for k in range(2)]
    solvers = [_run(m, 0) for m in mixes]
    b = Batch(solvers)
    with pytest.raises(CtfMnmfError) as e:
        b.debug_set_work(0, 0, 0, 4)
    assert e.value.name == "EUNSUPPORTED"
    b.close()
    for s in solvers:
        s.close()


_DEBUG_CHILD = r"""
import sys
sys.path.insert(0, sys.argv[1]); sys.path.insert(0, sys.argv[1] + "/tests")
import numpy as np, torch
from paper_2510_02382_gb300 import synth
from paper_2510_02382_gb300.api import Batch, CTFMNMF, CtfMnmfError
mixes = [synth.random_case(97 + k, M=3, N=2, F=4, J=64, B=3, Ln=(2, 1)) for k in range(2)]
solvers = []
for m in mixes:
    s = CTFMNMF(3, 2, 2, 3, 4, 64, Ln=m.Ln, path="two_kernel")
    s.load_stft(torch.from_numpy(m.X).cuda())
    s.set_init(torch.from_numpy(m.T0).cuda(), torch.from_numpy(m.V0).cuda())
    solvers.append(s)
b = Batch(solvers)
b.iterate(1)
solvers[0].synchronize()
assert b.debug_set_work(0, 0, 0, 4)            # bin 4 of a 4-bin mixture: out of range
b.iterate(1)
try:
    solvers[0].synchronize()
    print("NO_ERROR")
except CtfMnmfError as e:
    print("STATUS", e.name)
"""


def test_debug_build_bounds_check_stops_a_bad_work_item():
    from paper_2510_02382_gb300 import build as Bld
    Bld.build(debug=True)
    env = dict(os.environ, CTFMNMF_DEBUG_BUILD="1")
    r = subprocess.run([sys.executable, "-c", _DEBUG_CHILD, ROOT], capture_output=True, text=True, env=env,
                       timeout=300)
    assert r.returncode == 0, r.stderr[-2000:]
    assert "STATUS EBOUNDS" in r.stdout, r.stdout + r.stderr[-2000:]
