"""Write tests/golden/expected_costs.json: FP64 oracle costs of the full-size workloads whose
oracle runs take minutes (the GPU tests compare against these stored values instead of
re-running the oracle on the GPU machine's host).

Calls only oracle/ (the FP64 CPU oracle) and the seeded input generator; nothing here comes
from the CUDA library. Each entry also stores a fingerprint of its inputs (sums of |X|^2, T0
and V0 in FP64) so that a test can tell whether the generator still produces the same
mixture before it trusts the stored costs.

    python tests/golden/make_expected.py      (about five minutes on eight cores)
"""
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle import ctfmnmf_oracle as O          # noqa: E402
from paper_2510_02382_gb300 import synth        # noqa: E402

OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "expected_costs.json")


def fingerprint(mix):
    import numpy as np
    return {"x_power": float(np.sum(np.abs(mix.X.astype(np.complex128)) ** 2)),
            "t0_sum": float(np.sum(mix.T0, dtype=np.float64)), "v0_sum": float(np.sum(mix.V0, dtype=np.float64))}


def c4_samples():
    """Four mixtures of the 64-mixture batched workload: the smallest J, the largest J, the
    first with M = 4 and the first with M = 3 (seed order), without repeats."""
    specs = synth.batched_specs()
    picks = [min(specs, key=lambda s: s.J), max(specs, key=lambda s: s.J)]
    for M in (4, 3):
        for s in specs:
            if s.M == M and s not in picks:
                picks.append(s)
                break
    return picks


def main():
    out = {"oracle": "oracle/ctfmnmf_oracle.py (FP64), default options: all-taps activation update, "
                     "normalisation every iteration", "entries": {}}
    c3 = synth.make_mixture(synth.CONFIGS["C3"])
    iss = O.run(c3.X, c3.Ln, c3.T0, c3.V0, 100, trace=True)
    ip = O.run(c3.X, c3.Ln, c3.T0, c3.V0, 100, update="ip", trace=True)
    out["entries"]["C3"] = {"fingerprint": fingerprint(c3), "iss_cost": {"10": iss["trace"][9], "100": iss["trace"][99]},
                            "ip_cost": {"10": ip["trace"][9], "100": ip["trace"][99]}}
    print("C3", out["entries"]["C3"], flush=True)
    for sp in c4_samples():
        mix = synth.make_mixture(sp)
        r = O.run(mix.X, mix.Ln, mix.T0, mix.V0, sp.iters, trace=True)
        out["entries"][sp.name] = {"fingerprint": fingerprint(mix), "seed": sp.seed, "M": sp.M, "N": sp.N,
                                   "L": sp.L, "J": sp.J, "iss_cost": {"10": r["trace"][9], "50": r["trace"][49]}}
        print(sp.name, out["entries"][sp.name], flush=True)
    with open(OUT, "w") as f:
        json.dump(out, f, indent=1)
        f.write("\n")


if __name__ == "__main__":
    main()
