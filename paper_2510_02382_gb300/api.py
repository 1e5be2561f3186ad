"""Python binding of libctfmnmf (ctypes): the C ABI of include/ctfmnmf.h, same names.

Argument marshalling only: every step of the method runs in the CUDA library. Device
memory comes from torch tensors (their data pointers); work runs on the stream given
to the handle, by default torch's current stream at construction. If the library
has not been built, loading it raises; there is no other code path.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional, Sequence

from .build import lib_path

c_int, c_void_p, c_double, c_char_p = ctypes.c_int, ctypes.c_void_p, ctypes.c_double, ctypes.c_char_p

STATUS = {0: "OK", -1: "EINVAL", -2: "ESTATE", -3: "ECUDA", -4: "ENONFINITE", -5: "ETIMEOUT",
          -6: "ENOMEM", -7: "EUNSUPPORTED", -8: "EBOUNDS"}
V_ALL_TAPS, V_TAP0 = 0, 1
W_ISS, W_IP = 0, 1


class Dims(ctypes.Structure):
    _fields_ = [("M", c_int), ("N", c_int), ("L", c_int), ("B", c_int), ("F", c_int), ("J", c_int)]


class Options(ctypes.Structure):
    _fields_ = [("v_update", c_int), ("normalize", c_int), ("use_graph", c_int), ("path", c_int),
                ("wait_timeout_ms", c_int), ("w_update", c_int), ("bin_fpt", c_int), ("eps_floor", ctypes.c_float),
                ("deterministic_reduce", c_int), ("check_finite", c_int), ("reserved", c_int * 1)]


PATHS = {"auto": 0, "two_kernel": 1, "persistent": 2}


class CtfMnmfError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{STATUS.get(code, code)}: {msg}")
        self.code = code
        self.name = STATUS.get(code, str(code))


_LIB = None

_SIGS = {
    "ctfmnmf_default_options": (None, [c_void_p]),
    "ctfmnmf_create": (c_int, [c_int] * 6 + [c_void_p]),
    "ctfmnmf_create_ex": (c_int, [c_void_p, c_void_p, c_void_p, c_void_p]),
    "ctfmnmf_destroy": (c_int, [c_void_p]),
    "ctfmnmf_last_error": (c_char_p, [c_void_p]),
    "ctfmnmf_set_stream": (c_int, [c_void_p, c_void_p]),
    "ctfmnmf_get_taps": (c_int, [c_void_p, c_void_p]),
    "ctfmnmf_load_stft": (c_int, [c_void_p, c_void_p]),
    "ctfmnmf_load_stft_host": (c_int, [c_void_p, c_void_p]),
    "ctfmnmf_set_init": (c_int, [c_void_p, c_void_p, c_void_p]),
    "ctfmnmf_iterate": (c_int, [c_void_p, c_int]),
    "ctfmnmf_cost": (c_int, [c_void_p, c_void_p]),
    "ctfmnmf_get_separated": (c_int, [c_void_p, c_void_p]),
    "ctfmnmf_get_separated_host": (c_int, [c_void_p, c_void_p]),
    "ctfmnmf_get_demixed": (c_int, [c_void_p, c_void_p]),
    "ctfmnmf_get_demix_matrix": (c_int, [c_void_p, c_void_p]),
    "ctfmnmf_get_logdet": (c_int, [c_void_p, c_void_p]),
    "ctfmnmf_get_nmf": (c_int, [c_void_p, c_void_p, c_void_p]),
    "ctfmnmf_set_state": (c_int, [c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p]),
    "ctfmnmf_time_phases": (c_int, [c_void_p, c_int, c_void_p]),
    "ctfmnmf_get_launch_count": (c_int, [c_void_p, c_void_p]),
    "ctfmnmf_synchronize": (c_int, [c_void_p]),
    "ctfmnmf_get_path": (c_int, [c_void_p, c_void_p]),
    "ctfmnmf_get_bin_shape": (c_int, [c_void_p, c_void_p, c_void_p]),
    "ctfmnmf_time_persistent": (c_int, [c_void_p, c_int, c_void_p]),
    "ctfmnmf_debug_skip_arrival": (c_int, [c_void_p, c_int]),
    "ctfmnmf_debug_set_work": (c_int, [c_void_p, c_int, c_int, c_int, c_int, c_void_p]),
    "ctfmnmf_cost_noalloc": (c_int, [c_int, c_int, c_void_p, c_int, c_int, c_int, c_void_p, c_void_p,
                                     c_void_p, c_void_p, c_void_p, c_void_p]),
    "ctfmnmf_batch_create": (c_int, [c_int, c_void_p, c_void_p]),
    "ctfmnmf_batch_iterate": (c_int, [c_void_p, c_int]),
    "ctfmnmf_batch_time": (c_int, [c_void_p, c_int, c_void_p]),
    "ctfmnmf_batch_info": (c_int, [c_void_p, c_void_p]),
    "ctfmnmf_batch_destroy": (c_int, [c_void_p]),
    "ctfmnmf_batch_load_stft": (c_int, [c_void_p, c_void_p, c_void_p]),
    "ctfmnmf_batch_set_init": (c_int, [c_void_p, c_void_p, c_void_p, c_void_p, c_void_p]),
    "ctfmnmf_batch_get_separated": (c_int, [c_void_p, c_void_p, c_void_p]),
    "ctfmnmf_grad_create": (c_int, [c_void_p, c_void_p, c_int, c_int, c_int, c_void_p]),
    "ctfmnmf_grad_set_stream": (c_int, [c_void_p, c_void_p]),
    "ctfmnmf_grad_forward": (c_int, [c_void_p, c_void_p, c_void_p, c_void_p, c_void_p]),
    "ctfmnmf_grad_backward": (c_int, [c_void_p, c_void_p, c_void_p, c_void_p, c_void_p]),
    "ctfmnmf_grad_mse": (c_int, [c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p]),
    "ctfmnmf_grad_launch_count": (c_int, [c_void_p, c_void_p]),
    "ctfmnmf_grad_destroy": (c_int, [c_void_p]),
}


def lib():
    """Load libctfmnmf.so (raises if it has not been built). With CTFMNMF_DEBUG_BUILD=1 in the
    environment, the CTFMNMF_DEBUG build (device bounds checks, NaN/Inf scan every iteration)
    is loaded instead."""
    global _LIB
    if _LIB is None:
        p = lib_path(debug=os.environ.get("CTFMNMF_DEBUG_BUILD") == "1")
        if not os.path.exists(p):
            raise RuntimeError(f"{p} is missing: build it with `python -m paper_2510_02382_gb300.build`")
        L = ctypes.CDLL(p)
        for name, (res, args) in _SIGS.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _LIB = L
    return _LIB


def exported_symbols():
    return list(_SIGS)


def _check(rc: int, h=None):
    if rc != 0:
        msg = lib().ctfmnmf_last_error(h)
        raise CtfMnmfError(rc, msg.decode() if msg else "")


def _ptr(t) -> Optional[int]:
    if t is None:
        return None
    return t.data_ptr()


class Batch:
    """A ctfmnmf_batch_t over CTFMNMF solvers of one device: iterate() advances them all."""

    def __init__(self, solvers):
        self.solvers = list(solvers)
        arr = (c_void_p * len(self.solvers))(*[x._h.value for x in self.solvers])
        h = c_void_p()
        _check(lib().ctfmnmf_batch_create(len(self.solvers), arr, ctypes.byref(h)), None)
        self._h = h

    def iterate(self, n_iter: int):
        _check(lib().ctfmnmf_batch_iterate(self._h, int(n_iter)), None)

    def time(self, n_iter: int) -> float:
        ms = c_double()
        _check(lib().ctfmnmf_batch_time(self._h, int(n_iter), ctypes.byref(ms)), None)
        return ms.value

    def load_stft(self, X, offsets):
        """All mixtures' X from one complex64 device buffer; offsets[k] = element offset of
        mixture k's [M][F][J] block."""
        offs = (ctypes.c_longlong * len(self.solvers))(*[int(o) for o in offsets])
        _check(lib().ctfmnmf_batch_load_stft(self._h, c_void_p(X.data_ptr()), offs), None)

    def set_init(self, T0, t_offsets, V0, v_offsets):
        to = (ctypes.c_longlong * len(self.solvers))(*[int(o) for o in t_offsets])
        vo = (ctypes.c_longlong * len(self.solvers))(*[int(o) for o in v_offsets])
        _check(lib().ctfmnmf_batch_set_init(self._h, _ptr(T0), to, _ptr(V0), vo), None)

    def get_separated(self, C, offsets):
        offs = (ctypes.c_longlong * len(self.solvers))(*[int(o) for o in offsets])
        _check(lib().ctfmnmf_batch_get_separated(self._h, c_void_p(C.data_ptr()), offs), None)
        return C

    def debug_set_work(self, cls: int, entry: int, mixture: int, bin_: int) -> bool:
        """Test hook of CTFMNMF_DEBUG builds (ctfmnmf_debug_set_work); returns whether the loaded
        library is a debug build (a release build raises EUNSUPPORTED and changes nothing)."""
        dbg = c_int(0)
        _check(lib().ctfmnmf_debug_set_work(self._h, int(cls), int(entry), int(mixture), int(bin_), ctypes.byref(dbg)), None)
        return bool(dbg.value)

    def info(self):
        out = (c_int * 5)()
        _check(lib().ctfmnmf_batch_info(self._h, out), None)
        keys = ("mixtures", "bin_classes", "frame_classes", "plan", "launches")
        return dict(zip(keys, list(out)))

    def close(self):
        if getattr(self, "_h", None):
            lib().ctfmnmf_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Grad:
    """A ctfmnmf_grad_t: n_iter unrolled iterations on a batch of S mixtures of one shape,
    differentiable with respect to X [S][M][F][J] complex64, T0 [S][N][F][B] and
    V0 [S][N][B][J] float32 through the separated images C [S][N][M][F][J] complex64
    (checkpoint every ckpt_every iterations). See paper_2510_02382_gb300.autograd for the
    torch.autograd.Function wrappers."""

    def __init__(self, M: int, N: int, L: int, B: int, F: int, J: int, batch: int, n_iter: int,
                 ckpt_every: int = 5, Ln: Optional[Sequence[int]] = None, stream=None):
        import torch
        self.M, self.N, self.L, self.B, self.F, self.J = M, N, L, B, F, J
        self.S, self.n_iter, self.ckpt_every = batch, n_iter, ckpt_every
        d = Dims(M, N, L, B, F, J)
        ln_arr = (c_int * N)(*Ln) if Ln is not None else None
        h = c_void_p()
        _check(lib().ctfmnmf_grad_create(ctypes.byref(d), ln_arr, int(batch), int(n_iter), int(ckpt_every),
                                         ctypes.byref(h)), None)
        self._h = h
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        _check(lib().ctfmnmf_grad_set_stream(self._h, c_void_p(self.stream.cuda_stream)), None)

    def shapes(self):
        S, M, N, F, J, B = self.S, self.M, self.N, self.F, self.J, self.B
        return {"X": (S, M, F, J), "T0": (S, N, F, B), "V0": (S, N, B, J), "C": (S, N, M, F, J)}

    def forward(self, X, T0, V0, out=None):
        import torch
        sh = self.shapes()
        CTFMNMF._expect(X, sh["X"], torch.complex64, cuda=True)
        CTFMNMF._expect(T0, sh["T0"], torch.float32, cuda=True)
        CTFMNMF._expect(V0, sh["V0"], torch.float32, cuda=True)
        if out is None:
            out = torch.empty(sh["C"], dtype=torch.complex64, device=X.device)
        CTFMNMF._expect(out, sh["C"], torch.complex64, cuda=True)
        _check(lib().ctfmnmf_grad_forward(self._h, c_void_p(X.data_ptr()), c_void_p(T0.data_ptr()),
                                          c_void_p(V0.data_ptr()), c_void_p(out.data_ptr())), None)
        return out

    def backward(self, gC):
        import torch
        sh = self.shapes()
        CTFMNMF._expect(gC, sh["C"], torch.complex64, cuda=True)
        gX = torch.empty(sh["X"], dtype=torch.complex64, device=gC.device)
        gT0 = torch.empty(sh["T0"], dtype=torch.float32, device=gC.device)
        gV0 = torch.empty(sh["V0"], dtype=torch.float32, device=gC.device)
        _check(lib().ctfmnmf_grad_backward(self._h, c_void_p(gC.data_ptr()), c_void_p(gX.data_ptr()),
                                           c_void_p(gT0.data_ptr()), c_void_p(gV0.data_ptr())), None)
        return gX, gT0, gV0

    def mse(self, C, Cref, loss=None, dloss=None, gC=None):
        """Loss head: loss (0-dim float64 device tensor) = mean |C - Cref|^2 and/or gC =
        dloss * d(loss)/dC (dloss: 0-dim float64 device tensor, or None for 1)."""
        import torch
        sh = self.shapes()
        CTFMNMF._expect(C, sh["C"], torch.complex64, cuda=True)
        CTFMNMF._expect(Cref, sh["C"], torch.complex64, cuda=True)
        _check(lib().ctfmnmf_grad_mse(self._h, c_void_p(C.data_ptr()), c_void_p(Cref.data_ptr()), _ptr(loss),
                                      _ptr(dloss), _ptr(gC)), None)
        return loss, gC

    def launch_count(self) -> int:
        out = ctypes.c_longlong()
        _check(lib().ctfmnmf_grad_launch_count(self._h, ctypes.byref(out)), None)
        return int(out.value)

    def close(self):
        if getattr(self, "_h", None):
            lib().ctfmnmf_grad_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def cost_noalloc(Y, T, V, logdet, Ln, out, stream=None):
    """ctfmnmf_cost_noalloc: Eq. 5 from caller-held device tensors into `out` (one float64 on
    the device), without any device allocation by the library. Y [M][F][J] complex64,
    T [N][F][B], V [N][B][J] float32, logdet [F] float64."""
    import torch
    # the C side trusts every size it is given: check them all here, before any launch
    if Y.dim() != 3 or T.dim() != 3:
        raise ValueError("Y must be [M][F][J] and T [N][F][B]")
    M, F, J = Y.shape
    N, _, B = T.shape
    if len(Ln) != N:
        raise ValueError(f"Ln has {len(Ln)} entries for N={N} sources")
    CTFMNMF._expect(Y, (M, F, J), torch.complex64)
    CTFMNMF._expect(T, (N, F, B), torch.float32)
    CTFMNMF._expect(V, (N, B, J), torch.float32)
    CTFMNMF._expect(logdet, (F,), torch.float64)
    CTFMNMF._expect(out, (1,), torch.float64)
    st = stream if stream is not None else torch.cuda.current_stream()
    dev = st.device
    for t in (Y, T, V, logdet, out):
        if not t.is_cuda or t.device != dev:
            raise ValueError(f"every tensor must be on the stream's device {dev}, got {t.device}")
    ln_arr = (c_int * N)(*Ln)
    rc = lib().ctfmnmf_cost_noalloc(M, N, ln_arr, B, F, J, c_void_p(Y.data_ptr()), c_void_p(T.data_ptr()),
                                    c_void_p(V.data_ptr()), c_void_p(logdet.data_ptr()),
                                    c_void_p(out.data_ptr()), c_void_p(st.cuda_stream))
    _check(rc, None)
    return out


class CTFMNMF:
    """One mixture's solver on the current CUDA device (a handle of the C ABI).

    Shapes follow the C ABI: X [M][F][J] complex64, T [N][F][B], V [N][B][J] float32,
    images [N][M][F][J] complex64, W [F][M][M] complex64, logdet [F] float64.
    """

    def __init__(self, M: int, N: int, L: int, B: int, F: int, J: int,
                 Ln: Optional[Sequence[int]] = None, v_update: str = "all_taps",
                 normalize: bool = True, use_graph: bool = True, path: str = "auto",
                 wait_timeout_ms: int = 0, w_update: str = "iss", bin_fpt: int = 0, eps_floor: float = 0.0,
                 deterministic_reduce: bool = True, check_finite: bool = False, stream=None):
        import torch
        self.M, self.N, self.L, self.B, self.F, self.J = M, N, L, B, F, J
        d = Dims(M, N, L, B, F, J)
        o = Options()
        lib().ctfmnmf_default_options(ctypes.byref(o))
        o.v_update = {"all_taps": V_ALL_TAPS, "tap0": V_TAP0}[v_update]
        o.normalize = int(bool(normalize))
        o.use_graph = int(bool(use_graph))
        o.path = PATHS[path]
        o.wait_timeout_ms = int(wait_timeout_ms)
        o.w_update = {"iss": W_ISS, "ip": W_IP}[w_update]
        o.bin_fpt = int(bin_fpt)
        o.eps_floor = float(eps_floor)
        o.deterministic_reduce = int(bool(deterministic_reduce))
        o.check_finite = int(bool(check_finite))
        ln_arr = (c_int * N)(*Ln) if Ln is not None else None
        h = c_void_p()
        rc = lib().ctfmnmf_create_ex(ctypes.byref(d), ln_arr, ctypes.byref(o), ctypes.byref(h))
        _check(rc, None)
        self._h = h
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        _check(lib().ctfmnmf_set_stream(self._h, c_void_p(self.stream.cuda_stream)), self._h)
        taps = (c_int * N)()
        _check(lib().ctfmnmf_get_taps(self._h, taps), self._h)
        self.Ln = list(taps)
        p = c_int()
        _check(lib().ctfmnmf_get_path(self._h, ctypes.byref(p)), self._h)
        self.path = {1: "two_kernel", 2: "persistent"}[p.value]

    # -- lifecycle
    def close(self):
        if getattr(self, "_h", None):
            lib().ctfmnmf_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    # -- inputs
    def load_stft(self, X):
        import torch
        self._expect(X, (self.M, self.F, self.J), torch.complex64)
        if X.is_cuda:
            _check(lib().ctfmnmf_load_stft(self._h, c_void_p(X.data_ptr())), self._h)
        else:
            _check(lib().ctfmnmf_load_stft_host(self._h, c_void_p(X.data_ptr())), self._h)

    def set_init(self, T0=None, V0=None):
        import torch
        if T0 is not None:
            self._expect(T0, (self.N, self.F, self.B), torch.float32, cuda=True)
        if V0 is not None:
            self._expect(V0, (self.N, self.B, self.J), torch.float32, cuda=True)
        _check(lib().ctfmnmf_set_init(self._h, _ptr(T0), _ptr(V0)), self._h)

    def iterate(self, n_iter: int):
        _check(lib().ctfmnmf_iterate(self._h, int(n_iter)), self._h)

    def get_state(self):
        """The iteration state as tensors (checkpoint): Y [M][F][J] complex64, W [F][M][M]
        complex64, T [N][F][B], V [N][B][J] float32, logdet [F] float64."""
        T, V = self.get_nmf()
        return {"Y": self.get_demixed(), "W": self.get_demix_matrix(), "T": T, "V": V, "logdet": self.get_logdet()}

    def set_state(self, st):
        """Resume from a state returned by get_state (device tensors)."""
        import torch
        self._expect(st["Y"], (self.M, self.F, self.J), torch.complex64, cuda=True)
        self._expect(st["W"], (self.F, self.M, self.M), torch.complex64, cuda=True)
        self._expect(st["T"], (self.N, self.F, self.B), torch.float32, cuda=True)
        self._expect(st["V"], (self.N, self.B, self.J), torch.float32, cuda=True)
        self._expect(st["logdet"], (self.F,), torch.float64, cuda=True)
        _check(lib().ctfmnmf_set_state(self._h, _ptr(st["Y"]), _ptr(st["W"]), _ptr(st["T"]), _ptr(st["V"]),
                                       _ptr(st["logdet"])), self._h)

    # -- outputs
    def cost(self) -> float:
        out = c_double()
        _check(lib().ctfmnmf_cost(self._h, ctypes.byref(out)), self._h)
        return out.value

    def get_separated(self, out=None):
        import torch
        shape = (self.N, self.M, self.F, self.J)
        if out is None:
            out = torch.empty(shape, dtype=torch.complex64, device="cuda")
        self._expect(out, shape, torch.complex64)
        if out.is_cuda:
            _check(lib().ctfmnmf_get_separated(self._h, c_void_p(out.data_ptr())), self._h)
        else:
            _check(lib().ctfmnmf_get_separated_host(self._h, c_void_p(out.data_ptr())), self._h)
        return out

    def get_demixed(self):
        import torch
        out = torch.empty((self.M, self.F, self.J), dtype=torch.complex64, device="cuda")
        _check(lib().ctfmnmf_get_demixed(self._h, c_void_p(out.data_ptr())), self._h)
        return out

    def get_demix_matrix(self):
        import torch
        out = torch.empty((self.F, self.M, self.M), dtype=torch.complex64, device="cuda")
        _check(lib().ctfmnmf_get_demix_matrix(self._h, c_void_p(out.data_ptr())), self._h)
        return out

    def get_logdet(self):
        import torch
        out = torch.empty((self.F,), dtype=torch.float64, device="cuda")
        _check(lib().ctfmnmf_get_logdet(self._h, c_void_p(out.data_ptr())), self._h)
        return out

    def get_nmf(self):
        import torch
        T = torch.empty((self.N, self.F, self.B), dtype=torch.float32, device="cuda")
        V = torch.empty((self.N, self.B, self.J), dtype=torch.float32, device="cuda")
        _check(lib().ctfmnmf_get_nmf(self._h, c_void_p(T.data_ptr()), c_void_p(V.data_ptr())), self._h)
        return T, V

    # -- diagnostics
    def time_phases(self, n_iter: int):
        """Average device ms per launch of (bin phase, frame phase) over n_iter iterations."""
        ms = (c_double * 2)()
        _check(lib().ctfmnmf_time_phases(self._h, int(n_iter), ms), self._h)
        return float(ms[0]), float(ms[1])

    def synchronize(self):
        _check(lib().ctfmnmf_synchronize(self._h), self._h)

    def time_persistent(self, n_iter: int):
        """Device ms of one persistent launch of n_iter iterations, and of the closing kernels."""
        ms = (c_double * 2)()
        _check(lib().ctfmnmf_time_persistent(self._h, int(n_iter), ms), self._h)
        return float(ms[0]), float(ms[1])

    def debug_skip_arrival(self, cta: int):
        _check(lib().ctfmnmf_debug_skip_arrival(self._h, int(cta)), self._h)

    def launch_count(self) -> int:
        out = ctypes.c_longlong()
        _check(lib().ctfmnmf_get_launch_count(self._h, ctypes.byref(out)), self._h)
        return int(out.value)

    def bin_shape(self):
        """(frames per thread, threads) of the two-kernel bin phase; (0, 0) for cluster bins."""
        f, t = c_int(), c_int()
        _check(lib().ctfmnmf_get_bin_shape(self._h, ctypes.byref(f), ctypes.byref(t)), self._h)
        return f.value, t.value

    @staticmethod
    def _expect(t, shape, dtype, cuda=None):
        if tuple(t.shape) != tuple(shape) or t.dtype != dtype or not t.is_contiguous():
            raise ValueError(f"expected contiguous {dtype} {tuple(shape)}, got {t.dtype} {tuple(t.shape)}")
        if cuda and not t.is_cuda:
            raise ValueError("expected a CUDA tensor")
