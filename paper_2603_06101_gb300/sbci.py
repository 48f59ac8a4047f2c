"""Thin Python binding of the C ABI in include/sbci.h (ctypes, marshalling only).

Every computation runs in libsbci.so; this module converts numpy arrays and
torch CUDA tensors to pointers and raises on error statuses.  Importing it
fails loudly when the shared library has not been built: there is no CPU
fallback.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "libsbci.so")

SBCI_OK = 0
SBCI_ERR_INVALID = 1
SBCI_ERR_NOMEM = 2
SBCI_ERR_CUDA = 3
SBCI_ERR_NUMERIC = 4
SBCI_ERR_NOT_CONVERGED = 5
SBCI_ERR_TIMEOUT = 6
SBCI_ERR_CANCELLED = 7

SBCI_FP64 = 0
SBCI_TF32X3 = 1
SBCI_BF16X3 = 2
SBCI_FP32 = 3

_STATUS = {0: "OK", 1: "INVALID", 2: "NOMEM", 3: "CUDA", 4: "NUMERIC", 5: "NOT_CONVERGED",
           6: "TIMEOUT", 7: "CANCELLED"}


class SbciError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"sbci {_STATUS.get(status, status)}: {msg}")
        self.status = status


class sbci_params(C.Structure):
    _fields_ = [("eps0", C.c_double), ("r0", C.c_double), ("b_th", C.c_double), ("eps1", C.c_double),
                ("x_th1", C.c_double), ("x_th2", C.c_double), ("r1", C.c_double),
                ("max_cycle", C.c_int), ("max_sigma", C.c_int), ("guard", C.c_double),
                ("gs_tol", C.c_double), ("sector", C.c_int), ("n_init", C.c_int), ("init", C.c_int),
                ("prec", C.c_int), ("mixed_eps", C.c_double), ("mixed_r", C.c_double),
                ("refine_max_sigma", C.c_int), ("start_noise", C.c_double),
                ("noise_seed", C.c_longlong), ("init_stage", C.c_int)]


class sbci_report(C.Structure):
    _fields_ = [("energy", C.c_double), ("residual", C.c_double), ("converged", C.c_int),
                ("n_sigma", C.c_int), ("n_sigma_fp64", C.c_int), ("n_step", C.c_int),
                ("n_restart", C.c_int * 4), ("ctl_cycles", C.c_longlong), ("s136_ratio", C.c_double),
                ("s136_steps", C.c_int)]


class sbci_trace_record(C.Structure):
    _fields_ = [("state", C.c_int), ("t", C.c_int), ("energy", C.c_double), ("b", C.c_double),
                ("c", C.c_double), ("k", C.c_double), ("dE", C.c_double), ("dz", C.c_double),
                ("event", C.c_int), ("prec", C.c_int), ("s136", C.c_double)]


class sbci_kernel_stat(C.Structure):
    _fields_ = [("name", C.c_char * 32), ("launches", C.c_longlong), ("total_ms", C.c_double)]


class sbci_batch_class(C.Structure):
    _fields_ = [("Kp", C.c_int), ("Np", C.c_int), ("smem_bytes", C.c_int), ("tc_per_sm_max", C.c_int),
                ("tuned", C.c_int), ("ctas", C.c_int * 7), ("fKp", C.c_int), ("fNp", C.c_int),
                ("fused_smem_bytes", C.c_int), ("kernels", C.c_int)]


_lib = None

EXPORTS = ["sbci_params_init", "sbci_init_integrals", "sbci_dims", "sbci_string_table",
           "sbci_diagonal", "sbci_sigma", "sbci_begin", "sbci_step", "sbci_finish", "sbci_solve",
           "sbci_trace", "sbci_solve_sbci2", "sbci_davidson", "sbci_profile", "sbci_profile_read", "sbci_sigma_noalloc",
           "sbci_server_create", "sbci_server_submit", "sbci_server_progress", "sbci_server_poll",
           "sbci_server_set_batching", "sbci_server_destroy", "sbci_solve_batch", "sbci_batch_profile",
           "sbci_batch_profile_read", "sbci_batch_classes", "sbci_last_error", "sbci_destroy",
           "sbci_pool_stats", "sbci_pool_trim", "sbci_init_integrals_many"]
NOALLOC_SCRATCH_BYTES = 32 * 1024 * 1024


def load(path: str = LIB_PATH):
    """Loads libsbci.so and declares the prototypes.  Raises if it is missing."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError(f"libsbci.so not built ({path}); run __graft_entry__.build()")
    lib = C.CDLL(path)
    P, I, D, LL = C.c_void_p, C.c_int, C.c_double, C.c_longlong
    lib.sbci_params_init.argtypes = [C.POINTER(sbci_params)]
    lib.sbci_init_integrals.argtypes = [C.POINTER(P), I, I, I, P, P, D, P]
    lib.sbci_init_integrals_many.argtypes = [C.POINTER(P), I, I, I, I, P, P, D, C.POINTER(P)]
    lib.sbci_dims.argtypes = [P, C.POINTER(LL), C.POINTER(I), C.POINTER(I), C.POINTER(I),
                              C.POINTER(I), C.POINTER(I)]
    lib.sbci_string_table.argtypes = [P, I, P]
    lib.sbci_diagonal.argtypes = [P, P, I]
    lib.sbci_sigma.argtypes = [P, P, P, I, I, I]
    lib.sbci_begin.argtypes = [P, I, C.POINTER(sbci_params), P]
    lib.sbci_step.argtypes = [P, C.POINTER(sbci_trace_record), C.POINTER(I)]
    lib.sbci_finish.argtypes = [P, P, P, P]
    lib.sbci_solve.argtypes = [P, I, C.POINTER(sbci_params), P, P, P, P]
    lib.sbci_trace.argtypes = [P, C.POINTER(sbci_trace_record), I, C.POINTER(I)]
    lib.sbci_davidson.argtypes = [P, I, C.POINTER(sbci_params), I, P, P, P, C.POINTER(LL)]
    lib.sbci_solve_sbci2.argtypes = [P, I, C.POINTER(sbci_params), I, P, P, P]
    lib.sbci_sigma_noalloc.argtypes = [P, P, P, P]
    lib.sbci_server_create.argtypes = [C.POINTER(P), C.c_size_t, I]
    lib.sbci_server_submit.argtypes = [P, I, I, I, P, P, D, I, C.POINTER(sbci_params), C.POINTER(LL)]
    lib.sbci_server_progress.argtypes = [P, C.POINTER(I), C.POINTER(I)]
    lib.sbci_server_poll.argtypes = [P, LL, C.POINTER(I), P, P, P]
    lib.sbci_server_set_batching.argtypes = [P, I]
    lib.sbci_solve_batch.argtypes = [C.POINTER(P), I, I, C.POINTER(sbci_params), P, P, C.POINTER(LL)]
    lib.sbci_batch_profile.argtypes = [I]
    lib.sbci_batch_classes.argtypes = [C.POINTER(sbci_batch_class), I, C.POINTER(I)]
    lib.sbci_batch_profile_read.argtypes = [C.POINTER(sbci_kernel_stat), I, C.POINTER(I)]
    lib.sbci_server_destroy.argtypes = [P]
    lib.sbci_server_destroy.restype = None
    lib.sbci_profile.argtypes = [P, I]
    lib.sbci_profile_read.argtypes = [P, C.POINTER(sbci_kernel_stat), I, C.POINTER(I)]
    lib.sbci_last_error.restype = C.c_char_p
    lib.sbci_last_error.argtypes = []
    lib.sbci_destroy.argtypes = [P]
    lib.sbci_destroy.restype = None
    lib.sbci_pool_stats.argtypes = [C.POINTER(C.c_size_t), C.POINTER(LL), C.POINTER(LL)]
    lib.sbci_pool_trim.argtypes = []
    for name in EXPORTS:
        if name not in ("sbci_last_error", "sbci_destroy", "sbci_server_destroy"):
            getattr(lib, name).restype = C.c_int
    _lib = lib
    return lib


def _check(st: int, allow=()):
    if st != SBCI_OK and st not in allow:
        raise SbciError(st, _lib.sbci_last_error().decode())
    return st


def _ptr(a):
    """Pointer of a C-contiguous float64 numpy array or a CUDA torch tensor."""
    if isinstance(a, np.ndarray):
        assert a.flags["C_CONTIGUOUS"], "array must be C-contiguous"
        return a.ctypes.data_as(C.c_void_p), False
    if hasattr(a, "data_ptr"):
        assert a.is_contiguous(), "tensor must be contiguous"
        if a.is_cuda:
            # the library runs on its own stream: make torch's pending work visible
            import torch

            torch.cuda.current_stream(a.device).synchronize()
        return C.c_void_p(a.data_ptr()), bool(a.is_cuda)
    raise TypeError(type(a))


def _torch_float64():
    import torch

    return torch.float64


def params(**kw) -> sbci_params:
    lib = load()
    p = sbci_params()
    _check(lib.sbci_params_init(C.byref(p)))
    for k, v in kw.items():
        if not hasattr(p, k):
            raise KeyError(k)
        setattr(p, k, v)
    return p


class Context:
    """One active space on the current CUDA device (owns the device memory)."""

    def __init__(self, norb, nalpha, nbeta, h1, eri, e_core=0.0, stream=None, _handle=None):
        lib = load()
        self._lib = lib
        if _handle is not None:  # made by Context.many
            self._h = _handle
        else:
            h1 = np.ascontiguousarray(h1, dtype=np.float64)
            eri = np.ascontiguousarray(eri, dtype=np.float64)
            self._h = C.c_void_p()
            st = lib.sbci_init_integrals(C.byref(self._h), int(norb), int(nalpha), int(nbeta),
                                         h1.ctypes.data_as(C.c_void_p), eri.ctypes.data_as(C.c_void_p),
                                         float(e_core), C.c_void_p(stream) if stream else None)
            _check(st)
        nd, na, nb, la, lb, npair = C.c_longlong(), C.c_int(), C.c_int(), C.c_int(), C.c_int(), C.c_int()
        _check(lib.sbci_dims(self._h, C.byref(nd), C.byref(na), C.byref(nb), C.byref(la),
                             C.byref(lb), C.byref(npair)))
        self.ndet, self.na, self.nb = nd.value, na.value, nb.value
        self.nlink_a, self.nlink_b, self.npair = la.value, lb.value, npair.value
        self.norb, self.nalpha, self.nbeta = norb, nalpha, nbeta

    @classmethod
    def from_integrals(cls, I, stream=None):
        return cls(I.norb, I.nalpha, I.nbeta, I.h1, I.eri, I.e_core, stream)

    @classmethod
    def many(cls, norb, nalpha, nbeta, h1, eri, e_core=0.0, streams=None, n=None):
        """len(streams) (or n) contexts of the same integrals, created in
        parallel by sbci_init_integrals_many; streams: CUDA stream handles,
        one per context (None: each context makes its own)."""
        lib = load()
        if streams is None:
            streams = [None] * int(n)
        n = len(streams)
        h1 = np.ascontiguousarray(h1, dtype=np.float64)
        eri = np.ascontiguousarray(eri, dtype=np.float64)
        hs = (C.c_void_p * n)()
        ss = (C.c_void_p * n)(*[C.c_void_p(x) if x else None for x in streams])
        _check(lib.sbci_init_integrals_many(hs, n, int(norb), int(nalpha), int(nbeta),
                                            h1.ctypes.data_as(C.c_void_p), eri.ctypes.data_as(C.c_void_p),
                                            float(e_core), ss))
        return [cls(norb, nalpha, nbeta, None, None, e_core, _handle=C.c_void_p(hs[i])) for i in range(n)]

    def close(self):
        if getattr(self, "_h", None) and self._h.value:
            self._lib.sbci_destroy(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- entry points -------------------------------------------------------
    def string_table(self, spin: int) -> np.ndarray:
        nstr, nl = (self.na, self.nlink_a) if spin == 0 else (self.nb, self.nlink_b)
        out = np.zeros((nstr, nl, 3), dtype=np.int32)
        _check(self._lib.sbci_string_table(self._h, spin, out.ctypes.data_as(C.c_void_p)))
        return out

    def diagonal(self, out=None):
        if out is None:
            out = np.zeros(self.ndet)
        p, dev = _ptr(out)
        _check(self._lib.sbci_diagonal(self._h, p, int(dev)))
        return out

    def sigma(self, c, out=None, prec: int = SBCI_FP64):
        """sigma = H c for c of shape [..., Na, Nb] (numpy host or torch CUDA)."""
        if isinstance(c, np.ndarray):
            c = np.ascontiguousarray(c, dtype=np.float64)
            if out is None:
                out = np.zeros_like(c)
        elif out is None:
            out = c.new_zeros(c.shape)
        nvec = int(np.prod(c.shape)) // self.ndet
        pc, dev = _ptr(c)
        po, dev2 = _ptr(out)
        assert dev == dev2, "input and output must both be host or both be device"
        _check(self._lib.sbci_sigma(self._h, pc, po, nvec, int(prec), int(dev)))
        return out

    def sigma_noalloc(self, c, out, stream=None):
        """FP64 sigma of one device vector into ``out`` without any allocation.

        ``c`` and ``out``: contiguous float64 CUDA tensors of exactly ``ndet``
        elements on the context's device.  The call is queued on ``stream`` (a
        cudaStream_t handle) or, by default, on torch's current stream of that
        device, so torch work issued later on the same stream sees ``out``."""
        for name, t in (("c", c), ("out", out)):
            if not hasattr(t, "data_ptr"):
                raise TypeError(f"sigma_noalloc: {name} must be a torch tensor")
            if t.dtype != _torch_float64():
                raise TypeError(f"sigma_noalloc: {name} must be float64, got {t.dtype}")
            if t.numel() != self.ndet:
                raise ValueError(f"sigma_noalloc: {name} must hold ndet = {self.ndet} elements, got {t.numel()}")
            if not t.is_contiguous():
                raise ValueError(f"sigma_noalloc: {name} must be contiguous")
        if c.device != out.device:
            raise ValueError("sigma_noalloc: c and out must be on the same device")
        if not c.is_cuda:
            raise ValueError("sigma_noalloc: c and out must be CUDA tensors")
        if stream is None:
            import torch

            stream = torch.cuda.current_stream(c.device).cuda_stream
        _check(self._lib.sbci_sigma_noalloc(self._h, C.c_void_p(c.data_ptr()), C.c_void_p(out.data_ptr()),
                                            C.c_void_p(stream) if stream else None))
        return out

    def begin(self, k, p: sbci_params | None = None, c0=None):
        pc = None
        if c0 is not None:
            c0 = np.ascontiguousarray(c0, dtype=np.float64).reshape(-1)
            self._c0 = c0
            pc = c0.ctypes.data_as(C.c_void_p)
        _check(self._lib.sbci_begin(self._h, int(k), C.byref(p) if p is not None else None, pc))
        self._k = k

    def step(self):
        rec = sbci_trace_record()
        done = C.c_int()
        st = self._lib.sbci_step(self._h, C.byref(rec), C.byref(done))
        _check(st, allow=(SBCI_ERR_NOT_CONVERGED,))
        return rec, bool(done.value)

    def finish(self, want_vectors=False):
        k = self._k
        E = np.zeros(k)
        V = np.zeros((k, self.ndet)) if want_vectors else None
        R = (sbci_report * k)()
        st = self._lib.sbci_finish(self._h, E.ctypes.data_as(C.c_void_p),
                                   V.ctypes.data_as(C.c_void_p) if V is not None else None, R)
        _check(st, allow=(SBCI_ERR_NOT_CONVERGED,))
        return E, V, list(R), st

    def solve(self, k, p: sbci_params | None = None, c0=None, want_vectors=False):
        pc = None
        if c0 is not None:
            c0 = np.ascontiguousarray(c0, dtype=np.float64).reshape(-1)
            pc = c0.ctypes.data_as(C.c_void_p)
        E = np.zeros(k)
        V = np.zeros((k, self.ndet)) if want_vectors else None
        R = (sbci_report * k)()
        st = self._lib.sbci_solve(self._h, int(k), C.byref(p) if p is not None else None, pc,
                                  E.ctypes.data_as(C.c_void_p),
                                  V.ctypes.data_as(C.c_void_p) if V is not None else None, R)
        _check(st, allow=(SBCI_ERR_NOT_CONVERGED,))
        self._k = k
        return E, V, list(R), st

    def solve_sbci2(self, k, p: sbci_params | None = None, max_cycle2: int = 0, want_vectors=False):
        """SBCI2 (sbci_solve_sbci2): pairs of states, the last one by SBCI1."""
        E = np.zeros(k)
        V = np.zeros((k, self.ndet)) if want_vectors else None
        R = (sbci_report * k)()
        st = self._lib.sbci_solve_sbci2(self._h, int(k), C.byref(p) if p is not None else None, int(max_cycle2),
                                        E.ctypes.data_as(C.c_void_p),
                                        V.ctypes.data_as(C.c_void_p) if V is not None else None, R)
        _check(st, allow=(SBCI_ERR_NOT_CONVERGED,))
        self._k = k
        return E, V, list(R), st

    def davidson(self, k, p: sbci_params | None = None, max_space: int = 0, want_vectors=False):
        """Block Davidson-Liu on the same FP64 sigma (sbci_davidson).  Returns
        (energies, vectors or None, reports, status, subspace bytes)."""
        E = np.zeros(k)
        V = np.zeros((k, self.ndet)) if want_vectors else None
        R = (sbci_report * k)()
        nbytes = C.c_longlong()
        st = self._lib.sbci_davidson(self._h, int(k), C.byref(p) if p is not None else None, int(max_space),
                                     E.ctypes.data_as(C.c_void_p),
                                     V.ctypes.data_as(C.c_void_p) if V is not None else None, R,
                                     C.byref(nbytes))
        _check(st, allow=(SBCI_ERR_NOT_CONVERGED,))
        return E, V, list(R), st, int(nbytes.value)

    def profile(self, enable: bool = True):
        """Resets the per-kernel statistics; enable also times every launch."""
        _check(self._lib.sbci_profile(self._h, int(enable)))

    def profile_read(self) -> dict:
        buf = (sbci_kernel_stat * 32)()
        n = C.c_int()
        _check(self._lib.sbci_profile_read(self._h, buf, 32, C.byref(n)))
        return {b.name.decode(): (int(b.launches), float(b.total_ms)) for b in list(buf)[: n.value]}

    def trace(self):
        n = C.c_int()
        _check(self._lib.sbci_trace(self._h, None, 0, C.byref(n)))
        buf = (sbci_trace_record * max(n.value, 1))()
        _check(self._lib.sbci_trace(self._h, buf, n.value, C.byref(n)))
        return list(buf)[: n.value]


def solve_batch(contexts, k: int, p: sbci_params | None = None):
    """sbci_solve_batch over a list of Context objects: energies [n][k], reports, status."""
    lib = load()
    n = len(contexts)
    arr = (C.c_void_p * n)(*[c._h.value for c in contexts])
    E = np.zeros((n, k))
    R = (sbci_report * (n * k))()
    nl = C.c_longlong()
    st = lib.sbci_solve_batch(arr, n, int(k), C.byref(p) if p is not None else None,
                              E.ctypes.data_as(C.c_void_p), R, C.byref(nl))
    _check(st, allow=(SBCI_ERR_NOT_CONVERGED,))
    for c in contexts:
        c._k = k
    solve_batch.last_launches = nl.value
    return E, list(R), st


def last_error() -> str:
    """sbci_last_error: the calling thread's last error message."""
    return load().sbci_last_error().decode()


def batch_profile(enable: bool):
    """sbci_batch_profile: reset the batch engine's kernel statistics; enable
    event timing of every batched kernel launch."""
    _check(load().sbci_batch_profile(int(bool(enable))))


def batch_profile_read() -> dict:
    """sbci_batch_profile_read: {family: (launches, total_ms)}."""
    buf = (sbci_kernel_stat * 8)()
    n = C.c_int()
    _check(load().sbci_batch_profile_read(buf, 8, C.byref(n)))
    return {b.name.decode(): (int(b.launches), float(b.total_ms)) for b in list(buf)[: n.value]}


def pool_stats() -> dict:
    """The library's buffer cache: bytes cached now, requests served from the
    cache (hits) and from CUDA (misses) since the process started."""
    lib = load()
    cached, hits, misses = C.c_size_t(0), C.c_longlong(0), C.c_longlong(0)
    _check(lib.sbci_pool_stats(C.byref(cached), C.byref(hits), C.byref(misses)))
    return {"cached_bytes": cached.value, "hits": hits.value, "misses": misses.value}


def pool_trim():
    """Returns every cached buffer of the library to CUDA."""
    _check(load().sbci_pool_trim())


def batch_classes() -> list:
    """sbci_batch_classes: launch shapes of the batch engine per operand class."""
    buf = (sbci_batch_class * 16)()
    n = C.c_int()
    _check(load().sbci_batch_classes(buf, 16, C.byref(n)))
    names = ["update", "project", "tensor_core", "fused_column", "scatter", "symfinish", "end"]
    return [{"Kp": b.Kp, "Np": b.Np, "smem_bytes": b.smem_bytes, "tc_per_sm_max": b.tc_per_sm_max,
             "fKp": b.fKp, "fNp": b.fNp, "fused_smem_bytes": b.fused_smem_bytes, "tuned": bool(b.tuned),
             "ctas": {nm: b.ctas[i] for i, nm in enumerate(names) if b.kernels & (1 << i)}}
            for b in list(buf)[: min(n.value, 16)]]


class Server:
    """Continuous-batching request loop (sbci_server_*), one host thread."""

    def __init__(self, mem_budget_bytes: int, max_slots: int, batching: bool = True):
        lib = load()
        self._lib = lib
        self._h = C.c_void_p()
        _check(lib.sbci_server_create(C.byref(self._h), C.c_size_t(int(mem_budget_bytes)), int(max_slots)))
        _check(lib.sbci_server_set_batching(self._h, int(batching)))
        self._k = {}

    def submit(self, I, k: int, p: sbci_params | None = None) -> int:
        h1 = np.ascontiguousarray(I.h1, dtype=np.float64)
        eri = np.ascontiguousarray(I.eri, dtype=np.float64)
        t = C.c_longlong()
        _check(self._lib.sbci_server_submit(self._h, I.norb, I.nalpha, I.nbeta,
                                            h1.ctypes.data_as(C.c_void_p), eri.ctypes.data_as(C.c_void_p),
                                            float(I.e_core), int(k), C.byref(p) if p is not None else None,
                                            C.byref(t)))
        self._k[t.value] = k
        return t.value

    def progress(self):
        a, q = C.c_int(), C.c_int()
        _check(self._lib.sbci_server_progress(self._h, C.byref(a), C.byref(q)))
        return a.value, q.value

    def poll(self, ticket: int):
        """None while running, else (energies, reports, (queue_s, latency_s), status)."""
        k = self._k[ticket]
        done = C.c_int()
        E = np.zeros(k)
        R = (sbci_report * k)()
        T = np.zeros(2)
        st = self._lib.sbci_server_poll(self._h, C.c_longlong(ticket), C.byref(done),
                                        E.ctypes.data_as(C.c_void_p), R, T.ctypes.data_as(C.c_void_p))
        if not done.value:
            _check(st)
            return None
        return E, list(R), (float(T[0]), float(T[1])), st

    def close(self):
        if getattr(self, "_h", None) and self._h.value:
            self._lib.sbci_server_destroy(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
