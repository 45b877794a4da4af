"""Python binding of libstochq (include/stochq.h): the same entry points,
argument marshalling only. Every step of the computation runs in the CUDA
library; there is no Python or CPU fallback. If ``libstochq.so`` has not
been built, importing this module raises.

Host arrays are numpy ``complex128`` in the library's lexicographic layout:
links ``(T, Z, Y, X, 4, 3, 3)``, spinors ``(n, T, Z, Y, X, 4, 3)``. Device
buffers are torch CUDA tensors (any dtype; only ``data_ptr()`` is used) or
raw integer device addresses.
"""

from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
# STOCHQ_LIBRARY selects another build of the library (a build variant such
# as libstochq_sums64.so); by default the in-tree libstochq.so is loaded.
LIBPATH = os.environ.get("STOCHQ_LIBRARY") or os.path.join(_HERE, "libstochq.so")

SQ_F64, SQ_F32, SQ_F16 = 0, 1, 2
SQ_HOST, SQ_DEVICE = 0, 1
SQ_DS_CLOVER_INV, SQ_DS_XPAY, SQ_DS_SYNC, SQ_DS_F64_EMULATED = 1, 2, 4, 8
SQ_OUTER_RELIABLE, SQ_OUTER_DEFECT = 0, 1
SQ_DILUTE_TIME, SQ_DILUTE_SPIN_COLOUR, SQ_DILUTE_FULL = 1, 2, 3

STATUS = {
    0: "SQ_OK", 1: "SQ_ERR_ARG", 2: "SQ_ERR_CUDA", 3: "SQ_ERR_OOM",
    4: "SQ_ERR_NONFINITE", 5: "SQ_ERR_CLOVER", 6: "SQ_ERR_NOCONV",
    7: "SQ_ERR_BREAKDOWN", 8: "SQ_ERR_TIMEOUT", 9: "SQ_ERR_STATE",
}
globals().update({v: k for k, v in STATUS.items()})


class sq_solve_params(C.Structure):
    _fields_ = [
        ("inner_prec", C.c_int), ("outer", C.c_int), ("delta", C.c_double),
        ("max_iter", C.c_int), ("recon", C.c_int), ("sites_per_block", C.c_int),
        ("rhs_per_block", C.c_int), ("chunk", C.c_int), ("use_graph", C.c_int),
        ("io", C.c_int), ("use_x0", C.c_int), ("verbose", C.c_int),
        ("profile", C.c_int), ("pion", C.c_void_p), ("pion_tslice", C.c_void_p),
        ("breakdown_tol", C.c_double), ("fallback", C.c_int), ("fallback_max_iter", C.c_int),
    ]


class sq_solve_stats(C.Structure):
    _fields_ = [
        ("status", C.c_int), ("iterations", C.c_int), ("updates", C.c_int),
        ("restarts", C.c_int), ("true_residual", C.c_double), ("seconds", C.c_double),
        ("breakdowns", C.c_int), ("fallback", C.c_int),
    ]


class sq_kernel_stat(C.Structure):
    _fields_ = [
        ("name", C.c_char * 48), ("launches", C.c_longlong), ("ms", C.c_double),
        ("bytes", C.c_double), ("flops", C.c_double),
    ]


class sq_problem(C.Structure):
    _fields_ = [
        ("ctx", C.c_void_p), ("kappa", C.c_double), ("c_sw", C.c_double),
        ("sources", C.c_void_p), ("solutions", C.c_void_p), ("n_rhs", C.c_int),
        ("tol", C.c_double),
    ]


class StochqError(RuntimeError):
    def __init__(self, status, message, stats=None):
        self.status = status
        self.stats = stats
        super().__init__(f"{STATUS.get(status, status)}: {message}")


if not os.path.exists(LIBPATH):
    raise ImportError(
        f"{LIBPATH} is missing: build it with `python -m paper_1405_4524_gb300.build` "
        "(the CUDA library is required; there is no CPU fallback)")

_lib = C.CDLL(LIBPATH)
_vp, _i, _d = C.c_void_p, C.c_int, C.c_double

_SIG = {
    "sq_default_params": (None, [C.POINTER(sq_solve_params)]),
    "sq_create": (_i, [C.POINTER(_vp), C.POINTER(_i), _i, _vp]),
    "sq_destroy": (_i, [_vp]),
    "sq_load_gauge": (_i, [_vp, _vp, _i, _i]),
    "sq_build_clover": (_i, [_vp, _d, _d]),
    "sq_field_bytes": (_i, [_vp, _i, _i, C.POINTER(C.c_size_t)]),
    "sq_pack_spinor": (_i, [_vp, _vp, _vp, _i, _i, _i, _i]),
    "sq_unpack_spinor": (_i, [_vp, _vp, _vp, _i, _i, _i, _i]),
    "sq_dslash_eo": (_i, [_vp, _vp, _vp, _vp, _i, _i, _i, _i, _d]),
    "sq_norm2_eo": (_i, [_vp, _vp, _i, _i, _vp, _i]),
    "sq_norm2_eo_noalloc": (_i, [_vp, _vp, _i, _i, _vp, _i]),
    "sq_apply_M": (_i, [_vp, _vp, _vp, _i, _d, _d, _i]),
    "sq_solve": (_i, [_vp, _d, _d, _vp, _vp, _i, _d, C.POINTER(sq_solve_params),
                      C.POINTER(sq_solve_stats)]),
    "sq_solve_batch": (_i, [C.POINTER(sq_problem), _i, C.POINTER(sq_solve_params),
                            C.POINTER(sq_solve_stats)]),
    "sq_contract_pion": (_i, [_vp, _vp, _i, _vp, _vp, _i]),
    "sq_set_allocator": (_i, [_vp, _vp, _vp, _vp]),
    "sq_contract_stoch_op": (_i, [_vp, _vp, _vp, _i, _vp, _vp, _i]),
    "sq_contract_prop_trace": (_i, [_vp, _vp, _vp, _vp, _vp, _i, _vp, _i]),
    "sq_contract_stoch_op_z4": (_i, [_vp, _vp, _vp, _i, _vp, _vp, _i]),
    "sq_dilute": (_i, [_vp, _vp, _i, _i, _vp, _i]),
    "sq_contract_diagrams": (_i, [_vp, _vp, _vp, _vp, _vp, _vp, _i, _vp, _i]),
    "sq_diagrams_ensemble": (_i, [_vp, _vp, _i, _vp, _i]),
    "sq_get_profile": (_i, [_vp, C.POINTER(sq_kernel_stat), _i, C.POINTER(_i)]),
    "sq_kernel_launches": (_i, [_vp, C.POINTER(C.c_longlong)]),
    "sq_set_dslash_shape": (_i, [_vp, _i, _i, _i, C.POINTER(_i)]),
    "sq_get_dslash_shape": (_i, [_vp, _i, _i, C.POINTER(_i), C.POINTER(_i)]),
    "sq_set_wait_cycles": (_i, [_vp, C.c_longlong, _i]),
    "sq_tune_save": (_i, [_vp, C.c_char_p]),
    "sq_tune_load": (_i, [_vp, C.c_char_p, C.POINTER(_i)]),
    "sq_status_string": (C.c_char_p, [_i]),
    "sq_last_error": (C.c_char_p, [_vp]),
    "sq_inner_sum_bits": (_i, []),
}
for _name, (_res, _args) in _SIG.items():
    _f = getattr(_lib, _name)
    _f.restype = _res
    _f.argtypes = _args

EXPORTS = tuple(_SIG)


def _ptr(a):
    """Address of a numpy array, torch tensor or raw integer address."""
    if a is None:
        return None
    if isinstance(a, int):
        return a
    if isinstance(a, np.ndarray):
        if not a.flags["C_CONTIGUOUS"]:
            raise ValueError("host arrays must be C-contiguous")
        return a.ctypes.data
    if hasattr(a, "data_ptr"):
        if not a.is_contiguous():
            raise ValueError("device tensors must be contiguous")
        return a.data_ptr()
    raise TypeError(f"cannot take the address of {type(a)}")


def _where(a):
    if isinstance(a, np.ndarray):
        return SQ_HOST
    if hasattr(a, "is_cuda"):
        return SQ_DEVICE if a.is_cuda else SQ_HOST
    return SQ_DEVICE


def _check(ctx, status, stats=None):
    if status != 0:
        msg = sq_last_error(ctx) if ctx else STATUS.get(status, "")
        raise StochqError(status, msg, stats)


def _host_c128(a, name):
    if a.dtype != np.complex128:
        raise TypeError(f"{name} must be complex128 (FP64 re, im)")
    return a


# ---------------------------------------------------------------------------
# entry points (same names as the C ABI)
# ---------------------------------------------------------------------------

def sq_status_string(status: int) -> str:
    return _lib.sq_status_string(int(status)).decode()


def sq_last_error(ctx) -> str:
    return _lib.sq_last_error(ctx).decode()


def sq_inner_sum_bits() -> int:
    return int(_lib.sq_inner_sum_bits())


def sq_default_params(**overrides) -> sq_solve_params:
    p = sq_solve_params()
    _lib.sq_default_params(C.byref(p))
    for k, v in overrides.items():
        setattr(p, k, v)
    return p


def sq_create(dims, t_bc: int = -1, stream=None):
    """dims = (X, Y, Z, T); stream: torch.cuda.Stream, raw handle or None."""
    d = (C.c_int * 4)(*[int(x) for x in dims])
    h = _vp()
    s = None
    if stream is not None:
        s = stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)
    st = _lib.sq_create(C.byref(h), d, int(t_bc), s)
    _check(None, st)
    return h.value


def sq_destroy(ctx) -> None:
    _check(None, _lib.sq_destroy(ctx))
    _ALLOCATORS.pop(ctx, None)  # after the library has freed through them


_ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p, C.c_void_p)
_FREE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_size_t, C.c_void_p, C.c_void_p)
_ALLOCATORS = {}  # ctx -> the ctypes callbacks, alive as long as the context


def sq_set_allocator(ctx, alloc=None, free=None) -> None:
    """Persistent device buffers of the context from Python callables:
    alloc(nbytes, stream) -> device address (int, 0 on failure),
    free(address, nbytes, stream). Both None restores cudaMalloc / cudaFree.
    Call before sq_load_gauge."""
    if (alloc is None) != (free is None):
        raise ValueError("give both alloc and free, or neither")
    if alloc is None:
        _check(ctx, _lib.sq_set_allocator(ctx, None, None, None))
        _ALLOCATORS.pop(ctx, None)
        return
    a = _ALLOC_FN(lambda nbytes, stream, user: alloc(int(nbytes), stream) or None)
    f = _FREE_FN(lambda ptr, nbytes, stream, user: free(ptr, int(nbytes), stream))
    _check(ctx, _lib.sq_set_allocator(ctx, C.cast(a, _vp), C.cast(f, _vp), None))
    _ALLOCATORS[ctx] = (a, f)


def use_torch_allocator(ctx) -> None:
    """Take the context's persistent buffers from PyTorch's CUDA caching
    allocator (they then show in torch.cuda.memory_allocated)."""
    import torch

    dev = torch.cuda.current_device()
    sq_set_allocator(ctx,
                     lambda nbytes, stream: torch.cuda.caching_allocator_alloc(nbytes, dev, stream or 0),
                     lambda ptr, nbytes, stream: torch.cuda.caching_allocator_delete(ptr))


def sq_load_gauge(ctx, U, recon: int = 12) -> None:
    if isinstance(U, np.ndarray):
        U = np.ascontiguousarray(_host_c128(U, "U"))
    _check(ctx, _lib.sq_load_gauge(ctx, _ptr(U), int(recon), _where(U)))


def sq_build_clover(ctx, kappa: float, c_sw: float) -> None:
    _check(ctx, _lib.sq_build_clover(ctx, float(kappa), float(c_sw)))


def sq_field_bytes(ctx, prec: int, n_rhs: int) -> int:
    b = C.c_size_t()
    _check(ctx, _lib.sq_field_bytes(ctx, int(prec), int(n_rhs), C.byref(b)))
    return b.value


def sq_pack_spinor(ctx, eo_out, lex_in, parity: int, prec: int, n_rhs: int) -> None:
    if isinstance(lex_in, np.ndarray):
        lex_in = np.ascontiguousarray(_host_c128(lex_in, "lex_in"))
    _check(ctx, _lib.sq_pack_spinor(ctx, _ptr(eo_out), _ptr(lex_in), int(parity), int(prec),
                                    int(n_rhs), _where(lex_in)))


def sq_unpack_spinor(ctx, lex_out, eo_in, parity: int, prec: int, n_rhs: int) -> None:
    if isinstance(lex_out, np.ndarray):
        _host_c128(lex_out, "lex_out")
        if not lex_out.flags["C_CONTIGUOUS"]:
            raise ValueError("lex_out must be C-contiguous")
    _check(ctx, _lib.sq_unpack_spinor(ctx, _ptr(lex_out), _ptr(eo_in), int(parity), int(prec),
                                      int(n_rhs), _where(lex_out)))


def sq_dslash_eo(ctx, out, inp, x, out_parity: int, prec: int, n_rhs: int, flags: int = 0,
                 a: float = 0.0) -> None:
    _check(ctx, _lib.sq_dslash_eo(ctx, _ptr(out), _ptr(inp), _ptr(x), int(out_parity), int(prec),
                                  int(n_rhs), int(flags), float(a)))


def sq_norm2_eo(ctx, eo_field, prec: int, n_rhs: int, out=None) -> np.ndarray:
    """Per-source squared norms of a device even-odd field (float64 array)."""
    if out is None:
        out = np.zeros(int(n_rhs), dtype=np.float64)
    _check(ctx, _lib.sq_norm2_eo(ctx, _ptr(eo_field), int(prec), int(n_rhs), _ptr(out), _where(out)))
    return out


def sq_norm2_eo_noalloc(ctx, eo_field, prec: int, n_rhs: int, out=None) -> np.ndarray:
    """sq_norm2_eo without any device allocation (static scratch, at most
    256 sources; overlapping calls on one GPU race)."""
    if out is None:
        out = np.zeros(int(n_rhs), dtype=np.float64)
    _check(ctx, _lib.sq_norm2_eo_noalloc(ctx, _ptr(eo_field), int(prec), int(n_rhs), _ptr(out),
                                         _where(out)))
    return out


def sq_apply_M(ctx, out, inp, n_rhs: int, kappa: float, c_sw: float) -> None:
    if isinstance(inp, np.ndarray):
        inp = np.ascontiguousarray(_host_c128(inp, "in"))
    _check(ctx, _lib.sq_apply_M(ctx, _ptr(out), _ptr(inp), int(n_rhs), float(kappa), float(c_sw),
                                _where(inp)))


def sq_solve(ctx, kappa: float, c_sw: float, sources, solutions, n_rhs: int, tol: float,
             params: sq_solve_params | None = None, raise_on_error: bool = True,
             pion=None, pion_tslice=None):
    """Returns (status, list of per-source stats dicts). pion: optional
    (n_rhs, T) float64 output of the fused pion epilogue (same memory kind
    as the sources); pion_tslice: optional (n_rhs,) int32 time slices."""
    if params is None:
        params = sq_default_params()
    params = sq_solve_params.from_buffer_copy(params)
    params.io = _where(sources)
    if isinstance(sources, np.ndarray):
        _host_c128(sources, "sources")
        _host_c128(solutions, "solutions")
    keep = []
    if pion is not None:
        if _where(pion) != params.io:
            raise ValueError("pion must live where the sources live")
        if isinstance(pion, np.ndarray) and (pion.dtype != np.float64 or not pion.flags.c_contiguous):
            raise ValueError("pion must be a C-contiguous float64 array")
        shp = getattr(sources, "shape", None)
        if shp is not None and len(shp) == 7 and tuple(pion.shape) != (int(n_rhs), int(shp[1])):
            raise ValueError("pion must have shape (n_rhs, T)")
        params.pion = _ptr(pion)
        if pion_tslice is not None:
            if isinstance(pion_tslice, np.ndarray) or isinstance(pion_tslice, (list, tuple)):
                if params.io != SQ_HOST:
                    raise ValueError("pion_tslice must live where the sources live")
                pion_tslice = np.ascontiguousarray(pion_tslice, dtype=np.int32)
            if len(pion_tslice) != int(n_rhs):
                raise ValueError("pion_tslice must have n_rhs entries")
            keep.append(pion_tslice)
            params.pion_tslice = _ptr(pion_tslice)
    stats = (sq_solve_stats * int(n_rhs))()
    st = _lib.sq_solve(ctx, float(kappa), float(c_sw), _ptr(sources), _ptr(solutions), int(n_rhs),
                       float(tol), C.byref(params), stats)
    out = [dict(status=s.status, iterations=s.iterations, updates=s.updates,
                restarts=s.restarts, true_residual=s.true_residual, seconds=s.seconds,
                breakdowns=s.breakdowns, fallback=s.fallback)
           for s in stats]
    if raise_on_error:
        _check(ctx, st, out)
    return st, out


def sq_solve_batch(problems, params: sq_solve_params | None = None, raise_on_error: bool = True):
    """problems: list of dicts with ctx, kappa, c_sw, sources, solutions, n_rhs, tol."""
    if params is None:
        params = sq_default_params()
    params = sq_solve_params.from_buffer_copy(params)
    params.io = _where(problems[0]["sources"])
    arr = (sq_problem * len(problems))()
    total = 0
    for i, p in enumerate(problems):
        arr[i] = sq_problem(p["ctx"], float(p["kappa"]), float(p["c_sw"]), _ptr(p["sources"]),
                            _ptr(p["solutions"]), int(p["n_rhs"]), float(p["tol"]))
        total += int(p["n_rhs"])
    stats = (sq_solve_stats * total)()
    st = _lib.sq_solve_batch(arr, len(problems), C.byref(params), stats)
    out = [dict(status=s.status, iterations=s.iterations, updates=s.updates,
                restarts=s.restarts, true_residual=s.true_residual, seconds=s.seconds,
                breakdowns=s.breakdowns, fallback=s.fallback)
           for s in stats]
    if raise_on_error and st != 0:
        raise StochqError(st, sq_last_error(problems[0]["ctx"]), out)
    return st, out


def sq_dilute(ctx, noise, n_noise: int, scheme: int, out=None):
    """Diluted sources (n_noise * D, T, Z, Y, X, 4, 3), D = T, 12 or 12 T for
    SQ_DILUTE_TIME, SQ_DILUTE_SPIN_COLOUR, SQ_DILUTE_FULL; allocated like
    ``noise`` (host array or CUDA tensor) when not given."""
    where = _where(noise)
    T = int(noise.shape[1])
    D = {SQ_DILUTE_TIME: T, SQ_DILUTE_SPIN_COLOUR: 12, SQ_DILUTE_FULL: 12 * T}.get(int(scheme), 1)
    shape = (int(n_noise) * D,) + tuple(noise.shape[1:])
    if out is None:
        if where == SQ_HOST:
            out = np.zeros(shape, dtype=noise.dtype)
        else:
            import torch
            out = torch.zeros(shape, dtype=noise.dtype, device=noise.device)
    elif _where(out) != where:
        raise ValueError("out must live where noise does")
    _check(ctx, _lib.sq_dilute(ctx, _ptr(noise), int(n_noise), int(scheme), _ptr(out), where))
    return out


def sq_contract_pion(ctx, solutions, n_rhs: int, src_tslice=None) -> np.ndarray:
    """Returns C as a (n_rhs, T) float64 array."""
    ts = None
    if src_tslice is not None:
        ts = np.ascontiguousarray(np.asarray(src_tslice, dtype=np.int32))
    # T from the solutions' shape when on the host, else from the context
    T = int(solutions.shape[1]) if hasattr(solutions, "shape") else None
    if T is None:
        raise ValueError("solutions must be an array or tensor with shape (n, T, Z, Y, X, 4, 3)")
    Cout = np.zeros((int(n_rhs), T), dtype=np.float64)
    _check(ctx, _lib.sq_contract_pion(ctx, _ptr(solutions), int(n_rhs), _ptr(ts), _ptr(Cout),
                                      _where(solutions)))
    return Cout


def sq_contract_stoch_op(ctx, eta, X, n_rhs: int, O=None, C=None, correlator: bool = True,
                         tensor_cores: bool = False):
    """Operators O (T, n, n) complex128 and, if correlator, C (T,) complex128.

    eta, X: (n, T, Z, Y, X, 4, 3) float64 (or complex128 with the last axis
    folded) arrays, both on the host or both CUDA tensors. Outputs are
    allocated like the inputs when not given. tensor_cores: the exact
    digit-split tensor-core route (sq_contract_stoch_op_z4), for sources with
    components 0 or +-1."""
    where = _where(eta)
    if _where(X) != where:
        raise ValueError("eta and X must both be host arrays or both device tensors")
    T = int(eta.shape[1])
    n = int(n_rhs)
    if where == SQ_HOST:
        if O is None:
            O = np.zeros((T, n, n), dtype=np.complex128)
        if correlator and C is None:
            C = np.zeros(T, dtype=np.complex128)
    else:
        import torch
        if O is None:
            O = torch.zeros((T, n, n), dtype=torch.complex128, device=eta.device)
        if correlator and C is None:
            C = torch.zeros(T, dtype=torch.complex128, device=eta.device)
    if not correlator:
        C = None
    for a in (O, C):
        if a is not None and _where(a) != where:
            raise ValueError("O and C must live where eta and X do")
    fn = _lib.sq_contract_stoch_op_z4 if tensor_cores else _lib.sq_contract_stoch_op
    _check(ctx, fn(ctx, _ptr(eta), _ptr(X), n, _ptr(O), _ptr(C), where))
    return O, C


def sq_contract_stoch_op_z4(ctx, eta, X, n_rhs: int, O=None, C=None, correlator: bool = True):
    """sq_contract_stoch_op on the tensor cores (sources with components 0 or +-1)."""
    return sq_contract_stoch_op(ctx, eta, X, n_rhs, O, C, correlator, tensor_cores=True)


def sq_contract_prop_trace(ctx, etaA, XA, n_rhs: int, etaB=None, XB=None, C=None):
    """C (T, T) complex128: C[t0, t] = sum_{x in t0, z in t} tr[S_A S_B^dag].

    One source set when etaB and XB are None. Inputs all host arrays or all
    CUDA tensors; C is allocated like them when not given."""
    if (etaB is None) != (XB is None):
        raise ValueError("give both etaB and XB, or neither")
    fields = [f for f in (etaA, XA, etaB, XB) if f is not None]
    where = _where(etaA)
    if any(_where(f) != where for f in fields):
        raise ValueError("all fields must be host arrays or all device tensors")
    T = int(etaA.shape[1])
    if C is None:
        if where == SQ_HOST:
            C = np.zeros((T, T), dtype=np.complex128)
        else:
            import torch
            C = torch.zeros((T, T), dtype=torch.complex128, device=etaA.device)
    elif _where(C) != where:
        raise ValueError("C must live where the fields do")
    _check(ctx, _lib.sq_contract_prop_trace(ctx, _ptr(etaA), _ptr(XA), _ptr(etaB), _ptr(XB), int(n_rhs),
                                            _ptr(C), where))
    return C


DIAGRAM_NAMES = ("P", "Q0", "Qtt", "C0", "C1", "C2", "C3")
ENSEMBLE_NAMES = ("C0", "C1", "C2", "C3", "C")


def sq_contract_diagrams(ctx, Xp, etaA, XA, n_rhs: int, etaB=None, XB=None, out=None):
    """Per-configuration diagram quantities (DIAGRAM_NAMES) at every sink
    timeslice: complex (7, T), a numpy array for host inputs or the given /
    a new torch tensor for device inputs."""
    where = _where(XA)
    T = int(np.shape(XA)[1]) if where == SQ_HOST else int(XA.shape[1])
    if out is None:
        if where == SQ_HOST:
            out = np.zeros((7, T), dtype=np.complex128)
        else:
            import torch

            out = torch.zeros((7, T), dtype=torch.complex128, device=XA.device)
    if (etaB is None) != (XB is None):
        raise ValueError("etaB and XB go together")
    _check(ctx, _lib.sq_contract_diagrams(ctx, _ptr(Xp), _ptr(etaA), _ptr(XA), _ptr(etaB), _ptr(XB),
                                          int(n_rhs), _ptr(out), where))
    return out


def sq_diagrams_ensemble(ctx, rec, out=None):
    """Vacuum-subtracted ensemble averages (ENSEMBLE_NAMES) from records
    (n_cfg, 7, T) of sq_contract_diagrams; complex (5, T)."""
    where = _where(rec)
    n_cfg, _, T = (int(v) for v in rec.shape)
    if out is None:
        if where == SQ_HOST:
            out = np.zeros((5, T), dtype=np.complex128)
        else:
            import torch

            out = torch.zeros((5, T), dtype=torch.complex128, device=rec.device)
    _check(ctx, _lib.sq_diagrams_ensemble(ctx, _ptr(rec), n_cfg, _ptr(out), where))
    return out


def sq_get_profile(ctx):
    """Per kernel class totals of the last profiled solve (list of dicts)."""
    n = _i()
    _check(ctx, _lib.sq_get_profile(ctx, None, 0, C.byref(n)))
    arr = (sq_kernel_stat * n.value)()
    _check(ctx, _lib.sq_get_profile(ctx, arr, n.value, C.byref(n)))
    return [dict(name=a.name.decode(), launches=a.launches, ms=a.ms, bytes=a.bytes, flops=a.flops)
            for a in arr]


def sq_kernel_launches(ctx) -> int:
    n = C.c_longlong()
    _check(ctx, _lib.sq_kernel_launches(ctx, C.byref(n)))
    return n.value


def sq_set_dslash_shape(ctx, prec: int, n_rhs: int, kind: int, shape) -> None:
    """kind 0: shape = (sites per CTA, sources per CTA, order); kind 1 (halo
    tiles): shape = (rows in y, z, t, source slots per CTA, ring depth)."""
    v = (C.c_int * 5)(*(list(shape) + [0] * (5 - len(shape))))
    _check(ctx, _lib.sq_set_dslash_shape(ctx, int(prec), int(n_rhs), int(kind), v))


def sq_get_dslash_shape(ctx, prec: int, n_rhs: int):
    """(kind, shape tuple of 5) chosen for (prec, n_rhs) on this context."""
    k = C.c_int(0)
    v = (C.c_int * 5)()
    _check(ctx, _lib.sq_get_dslash_shape(ctx, int(prec), int(n_rhs), C.byref(k), v))
    return k.value, tuple(v)


def sq_tune_save(ctx, path: str) -> None:
    _check(ctx, _lib.sq_tune_save(ctx, os.fsencode(path)))


def sq_tune_load(ctx, path: str) -> int:
    """Number of shapes installed from the file."""
    n = C.c_int(0)
    _check(ctx, _lib.sq_tune_load(ctx, os.fsencode(path), C.byref(n)))
    return n.value


def sq_set_wait_cycles(ctx, cycles: int, stall_test: bool = False) -> None:
    _check(ctx, _lib.sq_set_wait_cycles(ctx, C.c_longlong(int(cycles)), int(bool(stall_test))))


class Lattice:
    """Owns one context: ``with Lattice(dims) as lat: lat.load(U) ...``."""

    def __init__(self, dims, t_bc: int = -1, stream=None):
        self.dims = tuple(int(d) for d in dims)
        self.ctx = sq_create(self.dims, t_bc, stream)

    def close(self):
        if self.ctx:
            sq_destroy(self.ctx)
            self.ctx = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
