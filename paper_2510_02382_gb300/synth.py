"""Seeded synthetic inputs for CTF-MNMF: mixtures drawn from the CTF mixing model.

This module draws random numbers and builds observations; it holds none of the
separation method's arithmetic, so both the FP64 oracle tests and the CUDA path
take their inputs from here.

Generative model (Sec. II, Eq. (2), the CTF convolutive mixing model):
    x_{m,i,j} = sum_n sum_{l < Lmix} h_{m,n,i,l} s_{n,i,j-l}   (s_{n,i,j<0} = 0)
with sources s_{n,i,j} ~ CN(0, lambda_{n,i,j}) whose power follows the NMF model
of Sec. II, lambda_{n,i,j} = sum_k b_{n,i,k} v_{n,k,j}.

Recipe (fixed order of draws from ``numpy.random.default_rng(seed)``):
  1. T_true [N][F][B], V_true [N][B][J] ~ Gamma(shape, scale)
  2. a, b [N][F][J] ~ N(0,1);  s = sqrt(lambda/2) (a + i b)
  3. h [M][N][F][Lmix] ~ CN(0,1) * exp(-l / tau)
  4. x = CTF convolution of s; source images c_n likewise per source
  5. optional white complex-Gaussian noise at ``snr_db`` below the mean mixture power
The observation is cast to complex64; the oracle upcasts exactly those values.
Initial NMF factors T0 [N][F][B], V0 [N][B][J] ~ Uniform[0.1, 1.0) are drawn
from ``default_rng(seed + 1_000_003)`` and cast to float32; both sides receive
identical values.
"""
from __future__ import annotations

import dataclasses
from typing import List, Optional, Sequence

import numpy as np

INIT_SEED_OFFSET = 1_000_003


def default_taps(M: int, N: int, L: int) -> List[int]:
    """Model taps per source so that sum(Ln) == M (the square extended model).

    Ln[n] = floor(M/N) + (n < M mod N), each capped at the mixing length L.
    M=4,N=2 -> (2,2); M=6,N=2 -> (3,3); M=8,N=2 -> (4,4) (the paper's Table I);
    M=3,N=2 -> (2,1); M=4,N=3 -> (2,1,1).
    """
    if N <= 0 or M < N:
        raise ValueError("need 0 < N <= M")
    Ln = [M // N + (1 if n < M % N else 0) for n in range(N)]
    if max(Ln) > L:
        raise ValueError(f"taps {Ln} exceed mixing length L={L}")
    return Ln


@dataclasses.dataclass(frozen=True)
class MixSpec:
    """Shape and generator parameters of one synthetic mixture."""
    name: str
    N: int
    M: int
    L: int            # length of the synthetic mixing CTF (and cap on model taps)
    tau: float        # tap decay: |h_l| ~ exp(-l / tau)
    F: int            # frequency bins (the paper's I)
    J: int            # frames
    B: int            # NMF bases per source (the paper's K_n)
    iters: int
    seed: int = 0
    gamma_shape: float = 1.0
    gamma_scale: float = 1.0
    snr_db: Optional[float] = None
    Ln: Optional[Sequence[int]] = None

    def taps(self) -> List[int]:
        return list(self.Ln) if self.Ln is not None else default_taps(self.M, self.N, self.L)


# Workloads. C1..C3: single mixtures; P4/P6/P8: the paper's Table I array shapes
# (2 sources, 8 s at 16 kHz with a 1024-point STFT and hop 256 -> 513 bins, 501 frames, K_n = 3).
CONFIGS = {
    "C1": MixSpec("C1", N=2, M=3, L=2, tau=1.5, F=129, J=256, B=4, iters=10),
    "C2": MixSpec("C2", N=2, M=3, L=4, tau=3.0, F=513, J=1000, B=10, iters=100, snr_db=30.0),
    "C3": MixSpec("C3", N=3, M=4, L=8, tau=5.0, F=513, J=2000, B=16, iters=100,
                  gamma_shape=0.5, gamma_scale=2.0),
    "P4": MixSpec("P4", N=2, M=4, L=2, tau=1.5, F=513, J=501, B=3, iters=100),
    "P6": MixSpec("P6", N=2, M=6, L=3, tau=2.0, F=513, J=501, B=3, iters=100),
    "P8": MixSpec("P8", N=2, M=8, L=4, tau=3.0, F=513, J=501, B=3, iters=100),
    # differentiable workload: 20 unrolled iterations, a batch of 16 mixtures (seeds 0..15)
    "C5": MixSpec("C5", N=2, M=3, L=4, tau=3.0, F=257, J=500, B=8, iters=20),
    # long-J workload: a 256 s recording at hop 256 (16 kHz), beyond one thread block per bin
    "L1": MixSpec("L1", N=2, M=3, L=4, tau=3.0, F=513, J=16000, B=10, iters=10, snr_db=30.0),
}

_TAU_BY_L = {2: 1.5, 4: 3.0, 8: 5.0}


def batched_specs(count: int = 64, F: int = 513, B: int = 10, iters: int = 50) -> List[MixSpec]:
    """The ragged batch: per seed s, J ~ U[300, 3000], N in {2,3}, M = N+1, L in {2,4,8}.

    J, N and L are the first three draws of ``default_rng(s)``; the mixture itself is
    then generated from ``default_rng(s)`` afresh by :func:`make_mixture`.
    """
    out = []
    for s in range(count):
        rng = np.random.default_rng(s)
        J = int(rng.integers(300, 3001))
        N = int(rng.choice([2, 3]))
        L = int(rng.choice([2, 4, 8]))
        out.append(MixSpec(f"B{s}", N=N, M=N + 1, L=L, tau=_TAU_BY_L[L], F=F, J=J, B=B,
                           iters=iters, seed=s))
    return out


def grad_specs(count: int = 16, **kw) -> List[MixSpec]:
    """The differentiable batch: the C5 shape with seeds 0..count-1 (fields in ``kw`` replaced)."""
    return [dataclasses.replace(CONFIGS["C5"], name=f"G{s}", seed=s, **kw) for s in range(count)]


def scaled(spec: MixSpec, **kw) -> MixSpec:
    """A copy of ``spec`` with some fields replaced (e.g. a smaller F or J for tests)."""
    return dataclasses.replace(spec, **kw)


@dataclasses.dataclass
class Mixture:
    spec: MixSpec
    Ln: List[int]
    X: np.ndarray        # [M][F][J] complex64 observation
    images: np.ndarray   # [N][M][F][J] complex64 true source images
    T0: np.ndarray       # [N][F][B] float32 initial basis
    V0: np.ndarray       # [N][B][J] float32 initial activation


def make_mixture(spec: MixSpec) -> Mixture:
    """Draw one mixture following the recipe in the module docstring."""
    N, M, F, J, B, L = spec.N, spec.M, spec.F, spec.J, spec.B, spec.L
    Ln = spec.taps()
    if sum(Ln) != M:
        raise ValueError("sum(Ln) must equal M")
    rng = np.random.default_rng(spec.seed)
    T_true = rng.gamma(spec.gamma_shape, spec.gamma_scale, size=(N, F, B))
    V_true = rng.gamma(spec.gamma_shape, spec.gamma_scale, size=(N, B, J))
    lam = np.einsum("nfk,nkj->nfj", T_true, V_true)
    s = np.sqrt(lam / 2.0) * (rng.standard_normal((N, F, J)) + 1j * rng.standard_normal((N, F, J)))
    decay = np.exp(-np.arange(L) / spec.tau)
    h = (rng.standard_normal((M, N, F, L)) + 1j * rng.standard_normal((M, N, F, L))) / np.sqrt(2.0)
    h = h * decay
    images = np.zeros((N, M, F, J), dtype=np.complex128)
    for l in range(L):
        # images[n, m, f, j] += h[m, n, f, l] * s[n, f, j - l]
        images[:, :, :, l:] += np.einsum("mnf,nfj->nmfj", h[:, :, :, l], s[:, :, : J - l])
    X = images.sum(axis=0)
    if spec.snr_db is not None:
        p = np.mean(np.abs(X) ** 2)
        sigma = np.sqrt(p * 10.0 ** (-spec.snr_db / 10.0) / 2.0)
        X = X + sigma * (rng.standard_normal(X.shape) + 1j * rng.standard_normal(X.shape))
    T0, V0 = initial_factors(N, F, B, J, spec.seed)
    return Mixture(spec=spec, Ln=Ln, X=X.astype(np.complex64), images=images.astype(np.complex64),
                   T0=T0, V0=V0)


def initial_factors(N: int, F: int, B: int, J: int, seed: int):
    """T0 [N][F][B], V0 [N][B][J] ~ Uniform[0.1, 1.0), float32, from seed + 1_000_003."""
    rng = np.random.default_rng(seed + INIT_SEED_OFFSET)
    T0 = rng.uniform(0.1, 1.0, size=(N, F, B)).astype(np.float32)
    V0 = rng.uniform(0.1, 1.0, size=(N, B, J)).astype(np.float32)
    return T0, V0


def random_case(seed: int, M: int, N: int, F: int, J: int, B: int, Ln=None, L=None):
    """A small mixture of arbitrary shape for tests (mixing length = max(Ln))."""
    Ln = list(Ln) if Ln is not None else default_taps(M, N, 8)
    L = L if L is not None else max(Ln)
    return make_mixture(MixSpec("rand", N=N, M=M, L=L, tau=2.0, F=F, J=J, B=B, iters=1,
                                seed=seed, Ln=tuple(Ln)))


def splitmix64(x: np.ndarray) -> np.ndarray:
    """splitmix64 (Steele, Lea, Flood 2014; constants of Vigna's splitmix64.c), uint64 wrap-around."""
    with np.errstate(over="ignore"):
        z = (x + np.uint64(0x9E3779B97F4A7C15)).astype(np.uint64)
        z = ((z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)).astype(np.uint64)
        z = ((z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)).astype(np.uint64)
        return z ^ (z >> np.uint64(31))


def library_default_factors(N: int, F: int, B: int, J: int, seed: int = 0):
    """The library's default NMF init: element e of T0 [N][F][B] is 0.1 + 0.9 u(2e), of
    V0 [N][B][J] 0.1 + 0.9 u(2e+1), u(c) = top 24 bits of splitmix64(seed*2^32 + c) / 2^24."""
    base = np.uint64(seed) << np.uint64(32)

    def vals(count, odd):
        c = np.arange(count, dtype=np.uint64) * np.uint64(2) + np.uint64(odd)
        u = (splitmix64(base + c) >> np.uint64(40)).astype(np.float64) / 16777216.0
        return (0.1 + 0.9 * u).astype(np.float32)

    return vals(N * F * B, 0).reshape(N, F, B), vals(N * B * J, 1).reshape(N, B, J)
