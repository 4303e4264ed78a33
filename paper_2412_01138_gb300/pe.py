"""ctypes binding of libpe (include/pe.h): argument marshalling only.

Every step of the method runs in the CUDA library; this module converts
Python descriptors (``inputs.Problem``, ``inputs.Term``) into the C structs,
passes pointers (numpy host arrays or torch device tensors) and raises
``PEError`` with the library's message on any non-zero status.  Importing it
loads ``_lib/libpe.so`` and fails loudly when the library has not been built
(``python -m paper_2412_01138_gb300.build``).
"""
from __future__ import annotations

import ctypes as C
import os
from typing import Optional, Sequence

import numpy as np

from . import inputs as _in

_LIB_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "_lib", "libpe.so")

PE_OK, PE_EINVAL, PE_ENOMEM, PE_ECUDA, PE_ENOCONV, PE_ENONFINITE, PE_ETIMEOUT, PE_ESTATE = 0, -1, -2, -3, -4, -5, -6, -7
PE_FP64, PE_MIXED = 0, 1
PE_DST_AUTO, PE_DST_MATRIX, PE_DST_TC = 0, 1, 2
PE_FORCING_SEPARABLE, PE_FORCING_GENERAL = 0, 1
PE_FINE_SIMT, PE_FINE_TC = 0, 1
PE_FIELD_TERMS_SEPARABLE, PE_FIELD_TERMS_QUADRATURE, PE_FIELD_NODAL = 0, 1, 2
PE_MAX_TERMS = 32

_STATUS_NAMES = {0: "PE_OK", -1: "PE_EINVAL", -2: "PE_ENOMEM", -3: "PE_ECUDA", -4: "PE_ENOCONV",
                 -5: "PE_ENONFINITE", -6: "PE_ETIMEOUT", -7: "PE_ESTATE"}

#: every symbol include/pe.h declares (checked by the CPU test suite)
EXPORTED = ("pe_setup", "pe_set_problem", "pe_parareal_iter", "pe_refine", "pe_solve", "pe_get_solution", "pe_get_modal",
            "pe_get_lambda", "pe_get_coefficients", "pe_forcing_modal", "pe_get_nodes", "pe_save_state",
            "pe_load_state", "pe_dst", "pe_dst_f32", "pe_last_error", "pe_destroy", "pe_setup_batch",
            "pe_batch_autotune", "pe_batch_solve", "pe_batch_get_modal", "pe_batch_get_solution", "pe_batch_status",
            "pe_batch_destroy", "pe_mlp_create", "pe_mlp_num_params", "pe_mlp_train", "pe_mlp_gradient",
            "pe_mlp_forward", "pe_mlp_get_params", "pe_mlp_set_params", "pe_mlp_destroy", "pe_learned_samples",
            "pe_set_learned", "pe_dst_tc", "pe_dst_noalloc", "pe_set_dirichlet", "pe_measure_fma_peak",
            "pe_probe_wait_timeout", "pe_parareal_iter_sums", "pe_batch_set_learned", "pe_solve_out",
            "pe_solve_async", "pe_solve_wait", "pe_probe_widen_f32")


class PEError(RuntimeError):
    def __init__(self, status: int, msg: str, result: Optional[dict] = None):
        super().__init__(f"{_STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status
        #: what the call reported before it failed (pe_solve's pe_result on PE_ENOCONV), else None
        self.result = result


class pe_term(C.Structure):
    _fields_ = [("amp", C.c_double), ("tkind", C.c_int32), ("tp", C.c_double * 2), ("skind", C.c_int32 * 3),
                ("sp", (C.c_double * 4) * 3)]


class pe_tableau(C.Structure):
    _fields_ = [("s", C.c_int32), ("c", C.POINTER(C.c_double)), ("random", C.c_int32), ("seed", C.c_uint64)]


#: residual_reduce callback of pe_options: void (*)(double* sums, void* user)
REDUCE_FN = C.CFUNCTYPE(None, C.POINTER(C.c_double), C.c_void_p)


class pe_options(C.Structure):
    _fields_ = [("precision", C.c_int32), ("dst_backend", C.c_int32), ("quad_pts", C.c_int32),
                ("max_iter", C.c_int32), ("cuda_stream", C.c_void_p), ("forcing_path", C.c_int32),
                ("cache_forced", C.c_int32), ("periodic_mask", C.c_int32), ("fine_engine", C.c_int32),
                ("mode_begin", C.c_int32), ("mode_end", C.c_int32), ("residual_reduce", REDUCE_FN),
                ("residual_reduce_user", C.c_void_p), ("device_loop", C.c_int32)]


class pe_field(C.Structure):
    _fields_ = [("kind", C.c_int32), ("n_terms", C.c_int32), ("terms", C.POINTER(pe_term)),
                ("nodal", C.c_void_p)]


class pe_forcing(C.Structure):
    _fields_ = [("n_terms", C.c_int32), ("terms", C.POINTER(pe_term))]


class pe_result(C.Structure):
    _fields_ = [("k", C.c_int32), ("residual", C.c_double), ("residual_history", C.POINTER(C.c_double)),
                ("history_cap", C.c_int32), ("fine_sweeps", C.c_int64), ("ms_tables", C.c_double),
                ("ms_prepare", C.c_double), ("ms_iterations", C.c_double), ("ms_output", C.c_double),
                ("ms_fine_kernel", C.c_double), ("kernel_launches", C.c_int64),
                ("ms_correction_kernel", C.c_double), ("ms_coarse_kernel", C.c_double)]


class pe_problem(C.Structure):
    _fields_ = [("d", C.c_int32), ("n", C.c_int32 * 3), ("box", C.c_double * 6), ("D", C.c_double),
                ("t0", C.c_double), ("T", C.c_double), ("n_slices", C.c_int32), ("n_substeps", C.c_int32),
                ("fine", pe_tableau), ("coarse", pe_tableau), ("u0", pe_field), ("forcing", pe_forcing)]


class pe_batch_result(C.Structure):
    _fields_ = [("graph_replays", C.c_int32), ("max_k", C.c_int32), ("max_residual", C.c_double),
                ("fine_dof_substeps", C.c_int64), ("ms_prepare", C.c_double), ("ms_iterations", C.c_double),
                ("kernel_launches", C.c_int64), ("threads", C.c_int32), ("ctas_per_sm", C.c_int32)]


def load_library(path: str = _LIB_PATH) -> C.CDLL:
    if not os.path.exists(path):
        raise ImportError(f"libpe is not built ({path} missing); run python -m paper_2412_01138_gb300.build")
    lib = C.CDLL(path)
    P = C.c_void_p
    sig = {
        "pe_setup": (C.c_int, [C.POINTER(P), C.c_int32, C.POINTER(C.c_int32), C.POINTER(C.c_double), C.c_double,
                               C.c_double, C.c_double, C.c_int32, C.c_int32, C.POINTER(pe_tableau),
                               C.POINTER(pe_tableau), C.POINTER(pe_options)]),
        "pe_set_problem": (C.c_int, [P, C.POINTER(pe_field), C.POINTER(pe_forcing)]),
        "pe_parareal_iter": (C.c_int, [P, C.POINTER(C.c_double)]),
        "pe_parareal_iter_sums": (C.c_int, [P, C.POINTER(C.c_double)]),
        "pe_refine": (C.c_int, [P, C.POINTER(C.c_double)]),
        "pe_solve": (C.c_int, [P, C.POINTER(pe_field), C.POINTER(pe_forcing), C.c_double, C.POINTER(pe_result)]),
        "pe_solve_out": (C.c_int, [P, C.POINTER(pe_field), C.POINTER(pe_forcing), C.c_double, P,
                                   C.POINTER(pe_result)]),
        "pe_solve_async": (C.c_int, [P, C.POINTER(pe_field), C.POINTER(pe_forcing), C.c_double, P]),
        "pe_solve_wait": (C.c_int, [P, C.POINTER(pe_result)]),
        "pe_get_solution": (C.c_int, [P, C.c_int32, P]),
        "pe_get_modal": (C.c_int, [P, C.c_int32, P]),
        "pe_get_lambda": (C.c_int, [P, P]),
        "pe_get_coefficients": (C.c_int, [P, C.c_int32, P]),
        "pe_forcing_modal": (C.c_int, [P, C.c_double, P]),
        "pe_get_nodes": (C.c_int, [P, C.c_int32, C.POINTER(C.c_double)]),
        "pe_save_state": (C.c_int, [P, P, C.POINTER(C.c_size_t)]),
        "pe_load_state": (C.c_int, [P, P, C.c_size_t]),
        "pe_dst": (C.c_int, [C.c_int32, C.POINTER(C.c_int32), P, P, P]),
        "pe_dst_f32": (C.c_int, [C.c_int32, C.POINTER(C.c_int32), P, P, P]),
        "pe_last_error": (C.c_char_p, []),
        "pe_setup_batch": (C.c_int, [C.POINTER(P), C.c_int32, C.POINTER(pe_problem), C.POINTER(pe_options)]),
        "pe_batch_autotune": (C.c_int, [P, C.c_char_p]),
        "pe_batch_solve": (C.c_int, [P, C.c_double, C.POINTER(pe_batch_result)]),
        "pe_batch_get_modal": (C.c_int, [P, C.c_int32, C.c_int32, P]),
        "pe_batch_get_solution": (C.c_int, [P, C.c_int32, P]),
        "pe_batch_status": (C.c_int, [P, C.POINTER(C.c_double), C.POINTER(C.c_int32)]),
        "pe_batch_destroy": (None, [P]),
        "pe_mlp_create": (C.c_int, [C.POINTER(P), C.c_uint64]),
        "pe_mlp_num_params": (C.c_int32, []),
        "pe_mlp_train": (C.c_int, [P, P, P, C.c_int32, C.c_int32, C.c_int32, C.c_float, C.POINTER(C.c_float)]),
        "pe_mlp_gradient": (C.c_int, [P, P, P, C.c_int32, C.POINTER(C.c_float), C.POINTER(C.c_float)]),
        "pe_mlp_forward": (C.c_int, [P, P, C.c_int32, P]),
        "pe_mlp_get_params": (C.c_int, [P, C.POINTER(C.c_float)]),
        "pe_mlp_set_params": (C.c_int, [P, C.POINTER(C.c_float)]),
        "pe_mlp_destroy": (None, [P]),
        "pe_learned_samples": (C.c_int, [P, C.c_int32, P, P, P, P, P]),
        "pe_set_learned": (C.c_int, [P, P]),
        "pe_batch_set_learned": (C.c_int, [P, P]),
        "pe_dst_tc": (C.c_int, [C.c_int32, C.POINTER(C.c_int32), P, P, C.c_int32, P]),
        "pe_dst_noalloc": (C.c_int, [C.c_int32, C.POINTER(C.c_int32), P, P, P]),
        "pe_set_dirichlet": (C.c_int, [P, C.c_int32, P]),
        "pe_measure_fma_peak": (C.c_int, [C.c_int32, C.POINTER(C.c_double), P]),
        "pe_probe_wait_timeout": (C.c_int, [C.c_int64, P]),
        "pe_probe_widen_f32": (C.c_int, [P, P, C.c_int64, P]),
        "pe_destroy": (None, [P]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    return lib


_lib: Optional[C.CDLL] = None


def lib() -> C.CDLL:
    global _lib
    if _lib is None:
        _lib = load_library()
    return _lib


def _check(status: int):
    if status != PE_OK:
        raise PEError(status, lib().pe_last_error().decode())


def _ptr(x) -> int:
    """Raw address of a numpy array or a torch tensor (host or device)."""
    if isinstance(x, np.ndarray):
        if not x.flags.c_contiguous:
            raise ValueError("array must be C-contiguous")
        return x.ctypes.data
    if hasattr(x, "data_ptr"):
        if not x.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return x.data_ptr()
    raise TypeError(f"unsupported buffer type {type(x)}")


def _check_out(x, count: int):
    """An output buffer of the solver: float64, contiguous (checked by _ptr), >= count values."""
    if isinstance(x, np.ndarray):
        if x.dtype != np.float64 or x.size < count:
            raise ValueError(f"output must hold >= {count} float64 values, got {x.size} {x.dtype}")
    elif hasattr(x, "numel"):
        if str(x.dtype) != "torch.float64" or x.numel() < count:
            raise ValueError(f"output must hold >= {count} float64 values, got {x.numel()} {x.dtype}")
    else:
        raise TypeError(f"unsupported buffer type {type(x)}")


def make_terms(terms: Sequence["_in.Term"]):
    arr = (pe_term * max(1, len(terms)))()
    for k, t in enumerate(terms):
        arr[k].amp = t.amp
        arr[k].tkind = t.tkind
        arr[k].tp[0], arr[k].tp[1] = t.tp
        for a, f in enumerate(t.factors):
            arr[k].skind[a] = f.kind
            for i, v in enumerate(f.params4()):
                arr[k].sp[a][i] = v
    return arr


def stream_handle(stream) -> Optional[int]:
    if stream is None:
        return None
    if hasattr(stream, "cuda_stream"):
        return stream.cuda_stream
    return int(stream)


class Solver:
    """One pe_ctx: a Parareal EIFE-linear solver for a fixed grid and time partition."""

    def __init__(self, prob: "_in.Problem", precision: int = PE_FP64, stream=None, max_iter: int = 0,
                 random_coarse_seed: Optional[int] = None, forcing_path: int = PE_FORCING_SEPARABLE,
                 dst_backend: int = PE_DST_AUTO, cache_forced: bool = False, fine_engine: int = PE_FINE_SIMT,
                 mode_range: Optional[Sequence[int]] = None, residual_reduce=None, device_loop: int = 0):
        """mode_range = (begin, end): own only the modes with axis-0 index in [begin, end) (a shard of
        a mode-sharded solve); residual_reduce(sums) -> totals: combines the two residual sums of
        this context with those of the other shards (pe_options.residual_reduce)."""
        self.prob = prob
        self._lib = lib()
        b, e = mode_range if mode_range is not None else (0, 0)
        self.mode_range = (b, e) if mode_range is not None else (0, prob.n[0])
        self.ndof_local = prob.ndof // prob.n[0] * (self.mode_range[1] - self.mode_range[0])
        self._reduce = None
        if residual_reduce is not None:
            def _cb(sums, _user, fn=residual_reduce):
                tot = fn(np.array([sums[0], sums[1]]))
                sums[0], sums[1] = float(tot[0]), float(tot[1])
            self._reduce = REDUCE_FN(_cb)
        n = (C.c_int32 * prob.d)(*prob.n)
        box = (C.c_double * (2 * prob.d))(*[v for lohi in prob.box for v in lohi])
        self._cF = (C.c_double * prob.q)(*prob.fine_nodes)
        self._cG = (C.c_double * prob.p)(*prob.coarse_nodes)
        fine = pe_tableau(prob.q, C.cast(self._cF, C.POINTER(C.c_double)), 0, 0)
        if random_coarse_seed is None:
            coarse = pe_tableau(prob.p, C.cast(self._cG, C.POINTER(C.c_double)), 0, 0)
        else:
            coarse = pe_tableau(prob.p, None, 1, random_coarse_seed)
        mask = sum(1 << a for a, p in enumerate(getattr(prob, "periodic", ())) if p)
        opt = pe_options(precision, dst_backend, prob.quad_pts, max_iter, stream_handle(stream), forcing_path,
                         1 if cache_forced else 0, mask, fine_engine, b, e,
                         self._reduce if self._reduce is not None else REDUCE_FN(), None, device_loop)
        ctx = C.c_void_p()
        _check(self._lib.pe_setup(C.byref(ctx), prob.d, n, box, prob.D, prob.t0, prob.T, prob.N, prob.M,
                                  C.byref(fine), C.byref(coarse), C.byref(opt)))
        self.ctx = ctx
        self._keep = []
        if getattr(prob, "boundary", ()):
            self.set_dirichlet(prob.boundary)

    def set_dirichlet(self, terms) -> None:
        """Non-homogeneous Dirichlet data (separable terms on the closed box); () restores u = 0."""
        arr = make_terms(tuple(terms)) if terms else None
        _check(self._lib.pe_set_dirichlet(self.ctx, len(terms), C.cast(arr, C.c_void_p) if arr is not None else None))

    def close(self):
        if getattr(self, "ctx", None):
            self._lib.pe_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    # -- problem data -------------------------------------------------------
    # The term arrays of u0 and f are marshalled once per solver (the problem is fixed for
    # its lifetime; the library copies them in on every call and keeps no pointer).
    def _u0_terms(self):
        if getattr(self, "_u0_arr", None) is None:
            self._u0_arr = make_terms(self.prob.u0)
        return self._u0_arr

    def _field(self, kind: int, nodal=None):
        prob = self.prob
        if kind == PE_FIELD_NODAL:
            return pe_field(kind, 0, None, _ptr(nodal))
        return pe_field(kind, len(prob.u0), C.cast(self._u0_terms(), C.POINTER(pe_term)), None)

    def _forcing(self):
        if getattr(self, "_f_struct", None) is None:
            self._f_arr = make_terms(self.prob.forcing)
            self._f_struct = pe_forcing(len(self.prob.forcing), C.cast(self._f_arr, C.POINTER(pe_term)))
        return self._f_struct

    def set_problem(self, u0_kind: int = PE_FIELD_TERMS_SEPARABLE, nodal=None):
        f = self._field(u0_kind, nodal)
        _check(self._lib.pe_set_problem(self.ctx, C.byref(f), C.byref(self._forcing())))

    def iterate(self) -> float:
        r = C.c_double()
        _check(self._lib.pe_parareal_iter(self.ctx, C.byref(r)))
        return r.value

    def iterate_sums(self) -> np.ndarray:
        """One Parareal iteration; this context's residual sums (sum mu (dU)^2, sum mu U^2)."""
        out = (C.c_double * 2)()
        _check(self._lib.pe_parareal_iter_sums(self.ctx, out))
        return np.array([out[0], out[1]])

    def refine(self) -> float:
        """One float64 Parareal iteration (float64 refinement of a mixed-precision iterate)."""
        r = C.c_double()
        _check(self._lib.pe_refine(self.ctx, C.byref(r)))
        return r.value

    def solve(self, tol: Optional[float] = None, u0_kind: int = PE_FIELD_TERMS_SEPARABLE, nodal=None,
              history: int = 64, out=None) -> dict:
        """pe_solve; with ``out`` (host array or device tensor of ndof float64) pe_solve_out,
        which also writes the nodal solution of the last slice into it."""
        f = self._field(u0_kind, nodal)
        res, hist = self._result(history)
        tol = self.prob.tol if tol is None else tol
        if out is None:
            st = self._lib.pe_solve(self.ctx, C.byref(f), C.byref(self._forcing()), tol, C.byref(res))
        else:
            _check_out(out, self.prob.ndof)
            st = self._lib.pe_solve_out(self.ctx, C.byref(f), C.byref(self._forcing()), tol, _ptr(out),
                                        C.byref(res))
        return self._report(st, res, hist, history)

    def solve_async(self, tol: Optional[float] = None, u0_kind: int = PE_FIELD_TERMS_SEPARABLE, nodal=None,
                    out=None) -> None:
        """pe_solve_async: the whole solve enqueued on the context's stream; ``wait`` reports it.
        A device u0 and ``out`` must stay alive until then."""
        f = self._field(u0_kind, nodal)
        tol = self.prob.tol if tol is None else tol
        if out is not None:
            _check_out(out, self.prob.ndof)
        self._pending = (nodal, out)  # the buffers the enqueued work reads and writes
        _check(self._lib.pe_solve_async(self.ctx, C.byref(f), C.byref(self._forcing()), tol,
                                        None if out is None else _ptr(out)))

    def wait(self, history: int = 64) -> dict:
        """pe_solve_wait: the report of the pending solve (as ``solve`` returns it)."""
        res, hist = self._result(history)
        st = self._lib.pe_solve_wait(self.ctx, C.byref(res))
        self._pending = None
        return self._report(st, res, hist, history)

    @staticmethod
    def _result(history: int):
        hist = (C.c_double * history)()
        res = pe_result()
        res.residual_history = C.cast(hist, C.POINTER(C.c_double))
        res.history_cap = history
        return res, hist

    def _report(self, st: int, res, hist, history: int) -> dict:
        info = {"k": res.k, "residual": res.residual, "history": list(hist[: min(res.k, history)]),
                "fine_sweeps": res.fine_sweeps, "ms_tables": res.ms_tables, "ms_prepare": res.ms_prepare,
                "ms_iterations": res.ms_iterations, "ms_output": res.ms_output,
                "ms_fine_kernel": res.ms_fine_kernel, "kernel_launches": res.kernel_launches,
                "ms_correction_kernel": res.ms_correction_kernel, "ms_coarse_kernel": res.ms_coarse_kernel}
        if st != PE_OK:
            # PE_ENOCONV: the iterations ran and the result is filled in; the caller may want it
            raise PEError(st, self._lib.pe_last_error().decode(), info if st == PE_ENOCONV else None)
        return info

    # -- outputs ------------------------------------------------------------
    def _out(self, count: int, out):
        return np.empty(count, dtype=np.float64) if out is None else out

    def solution(self, slice_: int, out=None):
        """Nodal values of the whole grid (a shard: of its modes alone)."""
        out = self._out(self.prob.ndof, out)
        _check(self._lib.pe_get_solution(self.ctx, slice_, _ptr(out)))
        return out

    def modal(self, slice_: int, out=None):
        out = self._out(self.ndof_local, out)
        _check(self._lib.pe_get_modal(self.ctx, slice_, _ptr(out)))
        return out

    def lam(self, out=None):
        out = self._out(self.ndof_local, out)
        _check(self._lib.pe_get_lambda(self.ctx, _ptr(out)))
        return out

    def coefficients(self, which: int, out=None):
        s = self.prob.q if which == 0 else self.prob.p
        out = self._out((s + 1) * self.ndof_local, out)
        _check(self._lib.pe_get_coefficients(self.ctx, which, _ptr(out)))
        return out.reshape(s + 1, self.ndof_local) if isinstance(out, np.ndarray) else out

    def forcing_modal(self, t: float, out=None):
        out = self._out(self.ndof_local, out)
        _check(self._lib.pe_forcing_modal(self.ctx, t, _ptr(out)))
        return out

    def nodes(self, which: int):
        s = self.prob.q if which == 0 else self.prob.p
        out = (C.c_double * s)()
        _check(self._lib.pe_get_nodes(self.ctx, which, out))
        return tuple(out)

    def set_learned(self, mlp: Optional["MLP"]):
        """Attach a trained network as learned coarse correction (None detaches)."""
        _check(self._lib.pe_set_learned(self.ctx, mlp.ctx if mlp is not None else None))
        self._mlp = mlp

    def learned_samples(self, lam, omega, x, t, K=None):
        """Method-generated training pairs for (lam, omega) device arrays (see pe_learned_samples)."""
        n = int(lam.numel()) if hasattr(lam, "numel") else len(lam)
        _check(self._lib.pe_learned_samples(self.ctx, n, _ptr(lam), _ptr(omega), _ptr(x), _ptr(t),
                                            _ptr(K) if K is not None else None))

    def save_state(self) -> bytes:
        size = C.c_size_t()
        _check(self._lib.pe_save_state(self.ctx, None, C.byref(size)))
        buf = C.create_string_buffer(size.value)
        _check(self._lib.pe_save_state(self.ctx, buf, C.byref(size)))
        return buf.raw

    def load_state(self, blob: bytes):
        buf = C.create_string_buffer(blob, len(blob))
        _check(self._lib.pe_load_state(self.ctx, buf, len(blob)))


def _device_buffers(name: str, d: int, n: Sequence[int], dtype: str, *bufs):
    """Checks of the device buffers of a standalone transform before any pointer reaches the
    library (which trusts its arguments): torch CUDA tensors of the transform's dtype holding at
    least prod(n) elements, contiguous."""
    if len(n) != d or d < 1:
        raise ValueError(f"{name}: n must hold d = {d} sizes")
    count = 1
    for v in n:
        count *= int(v)
    for b in bufs:
        if not (hasattr(b, "is_cuda") and b.is_cuda):
            raise ValueError(f"{name}: buffers must be CUDA tensors")
        if str(b.dtype) != f"torch.{dtype}":
            raise ValueError(f"{name}: buffers must be {dtype}, got {b.dtype}")
        if b.numel() < count:
            raise ValueError(f"{name}: a buffer holds {b.numel()} values, the transform needs {count}")
        if not b.is_contiguous():
            raise ValueError(f"{name}: buffers must be contiguous")


def dst_tc(d: int, n: Sequence[int], x_in, x_out, nsplit: int = 3, stream=None):
    """Tensor-core (tcgen05) DST-I of a float32 device buffer, split-bfloat16 operands."""
    _device_buffers("dst_tc", d, n, "float32", x_in, x_out)
    nn = (C.c_int32 * d)(*n)
    _check(lib().pe_dst_tc(d, nn, _ptr(x_in), _ptr(x_out), nsplit, stream_handle(stream)))


def dst_noalloc(d: int, n: Sequence[int], x_in, x_out, stream=None):
    """Float64 DST-I that allocates nothing (scratch in a built-in device array); see pe_dst_noalloc."""
    _device_buffers("dst_noalloc", d, n, "float64", x_in, x_out)
    nn = (C.c_int32 * d)(*n)
    _check(lib().pe_dst_noalloc(d, nn, _ptr(x_in), _ptr(x_out), stream_handle(stream)))


def dst(d: int, n: Sequence[int], x_in, x_out, stream=None, f32: bool = False):
    """Orthonormal tensor DST-I of a device buffer (torch tensor), out may alias in."""
    _device_buffers("dst", d, n, "float32" if f32 else "float64", x_in, x_out)
    nn = (C.c_int32 * d)(*n)
    fn = lib().pe_dst_f32 if f32 else lib().pe_dst
    _check(fn(d, nn, _ptr(x_in), _ptr(x_out), stream_handle(stream)))


def measure_fma_peak(precision: int, stream=None) -> float:
    """Measured FMA throughput of the CUDA cores (TFLOP/s): PE_FP64 float64, PE_MIXED float32."""
    out = C.c_double()
    _check(lib().pe_measure_fma_peak(precision, C.byref(out), stream_handle(stream)))
    return out.value


def probe_wait_timeout(budget_cycles: int, stream=None) -> None:
    """Run the tensor-core kernels' bounded wait on a barrier nothing arrives at (raises PEError
    with status PE_ETIMEOUT when the wait expires, which is what it is for)."""
    _check(lib().pe_probe_wait_timeout(int(budget_cycles), stream_handle(stream)))


def probe_widen_f32(x, y, stream=None) -> None:
    """y = x widened to float64 by the coarse sweeps' integer widening (float32 and float64 CUDA
    tensors of equal length)."""
    if not (getattr(x, "is_cuda", False) and getattr(y, "is_cuda", False)):
        raise ValueError("probe_widen_f32: buffers must be CUDA tensors")
    if str(x.dtype) != "torch.float32" or str(y.dtype) != "torch.float64" or y.numel() < x.numel():
        raise ValueError("probe_widen_f32: x float32, y float64 with at least as many values")
    _check(lib().pe_probe_widen_f32(_ptr(x), _ptr(y), int(x.numel()), stream_handle(stream)))


class BatchSolver:
    """One pe_batch: many independent problems advanced by shared persistent launches."""

    def __init__(self, probs: Sequence["_in.Problem"], precision: int = PE_MIXED, stream=None,
                 fine_engine: int = PE_FINE_SIMT):
        self.probs = list(probs)
        self._lib = lib()
        arr = (pe_problem * len(self.probs))()
        self._keep = []
        for k, p in enumerate(self.probs):
            q = arr[k]
            q.d = p.d
            for a in range(p.d):
                q.n[a] = p.n[a]
                q.box[2 * a], q.box[2 * a + 1] = p.box[a]
            q.D, q.t0, q.T = p.D, p.t0, p.T
            q.n_slices, q.n_substeps = p.N, p.M
            cF = (C.c_double * p.q)(*p.fine_nodes)
            cG = (C.c_double * p.p)(*p.coarse_nodes)
            tu = make_terms(p.u0)
            tf = make_terms(p.forcing)
            self._keep += [cF, cG, tu, tf]
            q.fine = pe_tableau(p.q, C.cast(cF, C.POINTER(C.c_double)), 0, 0)
            q.coarse = pe_tableau(p.p, C.cast(cG, C.POINTER(C.c_double)), 0, 0)
            q.u0 = pe_field(PE_FIELD_TERMS_SEPARABLE, len(p.u0), C.cast(tu, C.POINTER(pe_term)), None)
            q.forcing = pe_forcing(len(p.forcing), C.cast(tf, C.POINTER(pe_term)))
        opt = pe_options(precision, PE_DST_AUTO, self.probs[0].quad_pts, 0, stream_handle(stream),
                         PE_FORCING_SEPARABLE, 0, 0, fine_engine, 0, 0, REDUCE_FN(), None, 0)
        ctx = C.c_void_p()
        _check(self._lib.pe_setup_batch(C.byref(ctx), len(self.probs), arr, C.byref(opt)))
        self.ctx = ctx

    def close(self):
        if getattr(self, "ctx", None):
            self._lib.pe_batch_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def set_learned(self, mlp: Optional["MLP"]):
        """Attach a trained network as learned coarse correction of every problem (None detaches)."""
        _check(self._lib.pe_batch_set_learned(self.ctx, mlp.ctx if mlp is not None else None))
        self._mlp = mlp

    def autotune(self, cache_path: Optional[str] = None):
        _check(self._lib.pe_batch_autotune(self.ctx, cache_path.encode() if cache_path else None))

    def solve(self, tol: float) -> dict:
        res = pe_batch_result()
        _check(self._lib.pe_batch_solve(self.ctx, tol, C.byref(res)))
        return {f: getattr(res, f) for f, _ in pe_batch_result._fields_}

    def modal(self, problem: int, slice_: int, out=None):
        out = np.empty(self.probs[problem].ndof) if out is None else out
        _check(self._lib.pe_batch_get_modal(self.ctx, problem, slice_, _ptr(out)))
        return out

    def solution(self, problem: int, out=None):
        out = np.empty(self.probs[problem].ndof) if out is None else out
        _check(self._lib.pe_batch_get_solution(self.ctx, problem, _ptr(out)))
        return out

    def status(self):
        r = np.empty(len(self.probs))
        k = np.empty(len(self.probs), dtype=np.int32)
        _check(self._lib.pe_batch_status(self.ctx, r.ctypes.data_as(C.POINTER(C.c_double)),
                                         k.ctypes.data_as(C.POINTER(C.c_int32))))
        return r, k


class MLP:
    """The learned coarse correction network (pe_mlp)."""

    def __init__(self, seed: int = 0):
        self._lib = lib()
        ctx = C.c_void_p()
        _check(self._lib.pe_mlp_create(C.byref(ctx), seed))
        self.ctx = ctx
        self.n_params = self._lib.pe_mlp_num_params()

    def close(self):
        if getattr(self, "ctx", None):
            self._lib.pe_mlp_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def train(self, x, t, epochs: int, batch: int = 4096, lr: float = 2e-3) -> float:
        n = int(x.shape[0])
        loss = C.c_float()
        _check(self._lib.pe_mlp_train(self.ctx, _ptr(x), _ptr(t), n, epochs, batch, lr, C.byref(loss)))
        return loss.value

    def gradient(self, x, t):
        g = np.empty(self.n_params, dtype=np.float32)
        loss = C.c_float()
        _check(self._lib.pe_mlp_gradient(self.ctx, _ptr(x), _ptr(t), int(x.shape[0]),
                                          g.ctypes.data_as(C.POINTER(C.c_float)), C.byref(loss)))
        return g, loss.value

    def forward(self, x, y):
        _check(self._lib.pe_mlp_forward(self.ctx, _ptr(x), int(x.shape[0]), _ptr(y)))

    def params(self):
        p = np.empty(self.n_params, dtype=np.float32)
        _check(self._lib.pe_mlp_get_params(self.ctx, p.ctypes.data_as(C.POINTER(C.c_float))))
        return p

    def set_params(self, p):
        p = np.ascontiguousarray(p, dtype=np.float32)
        _check(self._lib.pe_mlp_set_params(self.ctx, p.ctypes.data_as(C.POINTER(C.c_float))))
