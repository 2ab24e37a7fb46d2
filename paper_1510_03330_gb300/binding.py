"""Thin ctypes binding of the C ABI in include/parquet.h.

Argument marshalling only: every step of a parquet iteration runs in the CUDA
library libparquet_gb300.so.  Importing this module does not need a GPU;
creating a Solver does, and there is no CPU fallback.  Device memory of a
solve comes from PyTorch's caching allocator and its kernels run on the
current PyTorch stream unless told otherwise.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from .workloads import BETHE, FP64, SPLIT_BF16X3, SPLIT_BF16X6, SPLIT_FP16X3, SPLIT_TF32X3, Params

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libparquet_gb300.so")

PQ_OK, PQ_EINVAL, PQ_ENOMEM, PQ_ECUDA, PQ_ENOTCONV, PQ_ETIMEOUT, PQ_ENAN, PQ_ESTATE, PQ_EDIVERGED = range(9)
STATUS = {0: "PQ_OK", 1: "PQ_EINVAL", 2: "PQ_ENOMEM", 3: "PQ_ECUDA", 4: "PQ_ENOTCONV", 5: "PQ_ETIMEOUT",
          6: "PQ_ENAN", 7: "PQ_ESTATE", 8: "PQ_EDIVERGED"}
PRECISION = {FP64: 0, SPLIT_TF32X3: 1, SPLIT_BF16X3: 2, SPLIT_BF16X6: 3, SPLIT_FP16X3: 4}
PQ_NSTEPS = 9

ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p)
FREE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_size_t, C.c_void_p)


class Options(C.Structure):
    _fields_ = [
        ("precision", C.c_int),
        ("mix_alpha", C.c_double),
        ("sigma2_box_factor", C.c_int),
        ("hop", C.c_double),
        ("tau_panels", C.c_int),
        ("tau_order", C.c_int),
        ("tau_matsubara", C.c_int),
        ("time_steps", C.c_int),
        ("q_chunk", C.c_int),
        ("assembly", C.c_int),
        ("kernel_level", C.c_int),
        ("edge_rule", C.c_int),
        ("sde", C.c_int),
        ("bse_tile_cols", C.c_int),
        ("diverge_window", C.c_int),
        ("target_density", C.c_double),
        ("cuda_stream", C.c_void_p),
        ("dev_alloc", ALLOC_FN),
        ("dev_free", FREE_FN),
        ("alloc_ctx", C.c_void_p),
    ]


class BatchOptions(C.Structure):
    _fields_ = [("tile_cols", C.c_int), ("order", C.c_int), ("time_steps", C.c_int)]


class ParquetError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


_lib = None


def load_library(path: str = LIB_PATH):
    """Load libparquet_gb300.so and declare the prototypes (no GPU needed)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is missing: build it with paper_1510_03330_gb300.build.build()")
    lib = C.CDLL(path)
    P = C.c_void_p
    D = C.POINTER(C.c_double)
    lib.pq_default_options.argtypes = [C.POINTER(Options)]
    lib.pq_default_options.restype = None
    lib.pq_init.argtypes = [C.POINTER(P), C.c_int, C.c_double, C.c_double, C.c_double, C.c_int, C.c_int, C.c_int,
                            C.POINTER(Options)]
    lib.pq_init.restype = C.c_int
    lib.pq_set_Lambda.argtypes = [P, C.c_int, D, C.c_int]
    lib.pq_set_Lambda.restype = C.c_int
    lib.pq_iterate.argtypes = [P, C.c_int, C.c_double, C.POINTER(C.c_int), D]
    lib.pq_iterate.restype = C.c_int
    for name in ("pq_get_Sigma",):
        getattr(lib, name).argtypes = [P, D, C.c_size_t]
        getattr(lib, name).restype = C.c_int
    for name in ("pq_get_F", "pq_get_Phi"):
        getattr(lib, name).argtypes = [P, C.c_int, C.c_int, D, C.c_size_t]
        getattr(lib, name).restype = C.c_int
    lib.pq_get_chi.argtypes = [P, C.c_int, D, C.c_size_t]
    lib.pq_get_chi.restype = C.c_int
    lib.pq_sigma_second_order.argtypes = [P, D, D, C.c_size_t]
    lib.pq_sigma_second_order.restype = C.c_int
    lib.pq_sigma_second_order_noalloc.argtypes = [C.c_int, C.c_double, C.c_double, C.c_double, C.c_double,
                                                  C.c_int, C.c_int, C.c_int, C.c_int, C.c_int, C.c_int, P, P, P]
    lib.pq_sigma_second_order_noalloc.restype = C.c_int
    lib.pq_density.argtypes = [P, D]
    lib.pq_density.restype = C.c_int
    lib.pq_get_mu.argtypes = [P, D]
    lib.pq_get_mu.restype = C.c_int
    lib.pq_selftest_wait_timeout.argtypes = [P, C.c_int]
    lib.pq_selftest_wait_timeout.restype = C.c_int
    lib.pq_set_state.argtypes = [P, D, D]
    lib.pq_set_state.restype = C.c_int
    lib.pq_get_sizes.argtypes = [P, C.POINTER(C.c_longlong)]
    lib.pq_get_sizes.restype = C.c_int
    lib.pq_step_times.argtypes = [P, C.POINTER(C.c_float), C.c_int]
    lib.pq_step_times.restype = C.c_int
    lib.pq_step_name.argtypes = [C.c_int]
    lib.pq_step_name.restype = C.c_char_p
    lib.pq_last_error.argtypes = [P]
    lib.pq_last_error.restype = C.c_char_p
    lib.pq_destroy.argtypes = [P]
    lib.pq_destroy.restype = None
    lib.pq_batch_default_options.argtypes = [C.POINTER(BatchOptions)]
    lib.pq_batch_default_options.restype = None
    lib.pq_batch_create.argtypes = [C.POINTER(P), C.POINTER(P), C.c_int, C.POINTER(BatchOptions)]
    lib.pq_batch_create.restype = C.c_int
    lib.pq_batch_iterate.argtypes = [P, C.c_int, D]
    lib.pq_batch_iterate.restype = C.c_int
    lib.pq_batch_config.argtypes = [P, C.POINTER(C.c_int), C.POINTER(C.c_int), C.POINTER(C.c_float)]
    lib.pq_batch_config.restype = C.c_int
    lib.pq_batch_times.argtypes = [P, C.POINTER(C.c_float)]
    lib.pq_batch_times.restype = C.c_int
    lib.pq_batch_last_error.argtypes = [P]
    lib.pq_batch_last_error.restype = C.c_char_p
    lib.pq_batch_destroy.argtypes = [P]
    lib.pq_batch_destroy.restype = None
    _lib = lib
    return lib


def default_options() -> Options:
    o = Options()
    load_library().pq_default_options(C.byref(o))
    return o


def _dptr(a: np.ndarray):
    return a.ctypes.data_as(C.POINTER(C.c_double))


class _TorchAllocator:
    """Device memory from PyTorch's caching allocator on the solve's stream."""

    def __init__(self, stream_handle):
        import torch

        self.torch = torch
        self.dev = torch.cuda.current_device()
        self.stream = stream_handle

        def alloc(nbytes, _ctx):
            try:
                return int(torch.cuda.caching_allocator_alloc(int(nbytes), self.dev, self.stream))
            except Exception:  # out of memory: the library reports PQ_ENOMEM
                return None

        def free(ptr, _nbytes, _ctx):
            torch.cuda.caching_allocator_delete(int(ptr))

        self.alloc = ALLOC_FN(alloc)
        self.free = FREE_FN(free)


class Solver:
    """One parquet solve on the GPU (C ABI: pq_init ... pq_destroy)."""

    def __init__(self, p: Params, precision: str = FP64, time_steps: bool = False, use_torch: bool = True,
                 q_chunk: int = 0, assembly: int = 0, bse_tile_cols: int = 0, diverge_window: int = 0):
        lib = load_library()
        self.p = p
        self.lib = lib
        o = default_options()
        o.precision = PRECISION[precision]
        o.mix_alpha = p.mix
        o.sigma2_box_factor = p.sigma2_factor
        o.hop = p.hop
        o.tau_panels = p.tau_panels
        o.tau_order = p.tau_order
        o.tau_matsubara = p.tau_matsubara
        o.time_steps = 1 if time_steps else 0
        o.q_chunk = q_chunk
        o.assembly = assembly
        o.kernel_level = p.kernel_level
        o.edge_rule = {"both": 0, "lower": 1}[p.edge_rule]
        o.sde = {"regulated": 0, "truncated": 1}[p.sde]
        o.bse_tile_cols = bse_tile_cols
        o.diverge_window = diverge_window
        o.target_density = p.density
        self.last_status = PQ_OK
        self._alloc = None
        if use_torch:
            import torch

            if not torch.cuda.is_available():
                raise RuntimeError("the parquet solver needs a CUDA device")
            s = torch.cuda.current_stream()
            o.cuda_stream = s.cuda_stream
            self._alloc = _TorchAllocator(s.cuda_stream)
            o.dev_alloc = self._alloc.alloc
            o.dev_free = self._alloc.free
        self._opt = o
        h = C.c_void_p()
        lat = 0 if p.lattice == BETHE else 1
        st = lib.pq_init(C.byref(h), lat, p.beta, p.U, p.mu, p.L, p.n_nu, p.n_Omega, C.byref(o))
        if st != PQ_OK:
            raise ParquetError(st, lib.pq_last_error(None).decode())
        self.h = h
        sz = (C.c_longlong * 8)()
        lib.pq_get_sizes(h, sz)
        self.sizes = list(sz)

    # ------------------------------------------------------------------ helpers
    def _check(self, st, ok=(PQ_OK,)):
        if st not in ok:
            raise ParquetError(st, self.lib.pq_last_error(self.h).decode())
        return st

    def close(self):
        if getattr(self, "h", None):
            self.lib.pq_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    # ------------------------------------------------------------------ API
    def iterate(self, max_iter: int = 1, tol: float = 0.0):
        """Run pq_iterate; returns (iterations done, last max|dSigma|, converged).  A run that
        stops without converging (PQ_ENOTCONV, or PQ_EDIVERGED with divergence detection on)
        leaves a valid state; its status is kept in last_status."""
        it = C.c_int(0)
        d = C.c_double(0.0)
        st = self._check(self.lib.pq_iterate(self.h, max_iter, tol, C.byref(it), C.byref(d)),
                         (PQ_OK, PQ_ENOTCONV, PQ_EDIVERGED))
        self.last_status = st
        return it.value, d.value, st == PQ_OK

    def density(self) -> float:
        """Electrons per site (both spins) of the current state's G (pq_density)."""
        v = C.c_double(0.0)
        self._check(self.lib.pq_density(self.h, C.byref(v)))
        return v.value

    def mu(self) -> float:
        """Chemical potential of the last iteration (pq_get_mu)."""
        v = C.c_double(0.0)
        self._check(self.lib.pq_get_mu(self.h, C.byref(v)))
        return v.value

    def selftest_wait_timeout(self, limit_ms: int) -> int:
        """pq_selftest_wait_timeout: a device wait on a barrier nothing arrives at gives up after
        limit_ms; returns the status (PQ_ETIMEOUT, after which the context is poisoned)."""
        return self.lib.pq_selftest_wait_timeout(self.h, limit_ms)

    def sigma(self) -> np.ndarray:
        p = self.p
        out = np.empty((p.n_k, p.n_ext), dtype=np.complex128)
        self._check(self.lib.pq_get_Sigma(self.h, _dptr(out), out.size * 2))
        return out

    def F(self, channel: int, Q: int) -> np.ndarray:
        out = np.empty((self.p.n, self.p.n), dtype=np.complex128)
        self._check(self.lib.pq_get_F(self.h, channel, Q, _dptr(out), out.size * 2))
        return out

    def Phi(self, channel: int, Q: int) -> np.ndarray:
        out = np.empty((self.p.n, self.p.n), dtype=np.complex128)
        self._check(self.lib.pq_get_Phi(self.h, channel, Q, _dptr(out), out.size * 2))
        return out

    def chi(self, channel: int) -> np.ndarray:
        out = np.empty(self.p.n_Q, dtype=np.complex128)
        self._check(self.lib.pq_get_chi(self.h, channel, _dptr(out), out.size * 2))
        return out

    def sigma_second_order(self, sigma: np.ndarray | None = None) -> np.ndarray:
        """Second-order self-energy (the paper's Sigma~1) of G[sigma] (default: the state)."""
        p = self.p
        out = np.empty((p.n_k, p.n_ext), dtype=np.complex128)
        sa = None
        if sigma is not None:
            sa = np.ascontiguousarray(sigma, dtype=np.complex128)
            assert sa.shape == (p.n_k, p.n_ext)
        self._check(self.lib.pq_sigma_second_order(self.h, _dptr(sa) if sa is not None else None, _dptr(out),
                                                   out.size * 2))
        return out

    def set_Lambda(self, channel: int, table: np.ndarray, n_lambda: int):
        """Tabulated local Lambda of one channel, [2 n_lambda + 1][2 n_lambda][2 n_lambda] (m, n, n')."""
        t = np.ascontiguousarray(table, dtype=np.complex128)
        assert t.shape == (2 * n_lambda + 1, 2 * n_lambda, 2 * n_lambda)
        self._check(self.lib.pq_set_Lambda(self.h, channel, _dptr(t), n_lambda))

    def set_state(self, phi: np.ndarray | None = None, sigma: np.ndarray | None = None):
        p = self.p
        pa = sa = None
        if phi is not None:
            pa = np.ascontiguousarray(phi, dtype=np.complex128)
            assert pa.shape == (4, p.n_Q, p.n, p.n)
        if sigma is not None:
            sa = np.ascontiguousarray(sigma, dtype=np.complex128)
            assert sa.shape == (p.n_k, p.n_ext)
        self._check(self.lib.pq_set_state(self.h, _dptr(pa) if pa is not None else None,
                                          _dptr(sa) if sa is not None else None))

    def step_times(self) -> dict:
        out = (C.c_float * PQ_NSTEPS)()
        self._check(self.lib.pq_step_times(self.h, out, PQ_NSTEPS))
        return {self.lib.pq_step_name(i).decode(): float(out[i]) for i in range(PQ_NSTEPS)}

    @property
    def device_bytes(self) -> int:
        return int(self.sizes[6])


class Batch:
    """Several solves iterated together (C ABI: pq_batch_create ... pq_batch_destroy): per iteration
    one CUDA graph with one grouped tensor-core launch for all the Bethe-Salpeter products."""

    def __init__(self, solvers, tile_cols: int = 0, order: int = -1, time_steps: bool = False):
        lib = load_library()
        self.lib = lib
        self.solvers = list(solvers)
        o = BatchOptions()
        lib.pq_batch_default_options(C.byref(o))
        o.tile_cols, o.order, o.time_steps = tile_cols, order, 1 if time_steps else 0
        arr = (C.c_void_p * len(self.solvers))(*[s.h.value for s in self.solvers])
        h = C.c_void_p()
        st = lib.pq_batch_create(C.byref(h), arr, len(self.solvers), C.byref(o))
        if st != PQ_OK:
            raise ParquetError(st, lib.pq_last_error(None).decode())
        self.h = h

    def iterate(self, n_iter: int = 1) -> np.ndarray:
        """Run n_iter iterations of every member; returns each member's last max|dSigma|."""
        out = np.zeros(len(self.solvers))
        st = self.lib.pq_batch_iterate(self.h, n_iter, _dptr(out))
        if st != PQ_OK:
            raise ParquetError(st, self.lib.pq_batch_last_error(self.h).decode())
        return out

    def config(self):
        tc, od = C.c_int(0), C.c_int(0)
        tuned = (C.c_float * 4)()
        self.lib.pq_batch_config(self.h, C.byref(tc), C.byref(od), tuned)
        return {"tile_cols": tc.value, "order": od.value, "tuned_ms": [float(x) for x in tuned]}

    def times(self):
        out = (C.c_float * 2)()
        self.lib.pq_batch_times(self.h, out)
        return {"iteration": float(out[0]), "bse": float(out[1])}

    def close(self):
        if getattr(self, "h", None):
            self.lib.pq_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()
