"""Thin ctypes binding of libqmcdu (include/qmcdu.h): same names, argument
marshalling only. Every step of the delayed update runs in the library's CUDA
kernels; PyTorch only supplies device memory and streams here.

Array arguments may be torch tensors (CPU or CUDA) or numpy arrays; the C
functions are told only their addresses. Arrays that the header calls
"device" must be CUDA tensors; "host or device" arrays may be either.
Any non-zero status raises QmcduError with the library's error text.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIBRARY_PATH = os.path.join(_HERE, "libqmcdu.so")

QMCDU_FP64, QMCDU_FP32, QMCDU_FP32_BF16X3 = 0, 1, 2
PRECISIONS = {"fp64": QMCDU_FP64, "fp32": QMCDU_FP32, "bf16x3": QMCDU_FP32_BF16X3}
STATUS = {0: "OK", 1: "ERR_ARG", 2: "ERR_STATE", 3: "ERR_SINGULAR", 4: "ERR_OOM",
          5: "ERR_CUDA", 6: "ERR_TIMEOUT"}
QMCDU_MAX_N, QMCDU_MAX_K = 8192, 256

# Every function the header declares, with its ctypes signature.
_VP, _I, _D, _ULL = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_ulonglong
SIGNATURES = {
    "qmcdu_create": (_I, [_I, _I, _I, _I, _VP, ctypes.POINTER(_VP)]),
    "qmcdu_destroy": (_I, [_VP]),
    "qmcdu_set_matrix": (_I, [_VP, _VP]),
    "qmcdu_get_matrix": (_I, [_VP, _VP]),
    "qmcdu_get_inverse": (_I, [_VP, _VP]),
    "qmcdu_ratio": (_I, [_VP, _VP, _VP, _VP]),
    "qmcdu_accept": (_I, [_VP, _VP]),
    "qmcdu_flush": (_I, [_VP]),
    "qmcdu_recompute": (_I, [_VP, _VP]),
    "qmcdu_logdet": (_I, [_VP, _VP, _VP]),
    "qmcdu_logdet_product": (_I, [_VP, _VP, _VP, _VP]),
    "qmcdu_sweep": (_I, [_VP, _ULL, _I, _D, _VP, _VP, _VP, _VP]),
    "qmcdu_sync": (_I, [_VP]),
    "qmcdu_step": (_I, [_VP, _ULL, _I, _I, _D, _I, _I, _VP, _VP]),
    "qmcdu_step_results": (_I, [_VP, _I, _VP, _VP, _VP]),
    "qmcdu_group_create": (_I, [_VP, _I, ctypes.POINTER(_VP)]),
    "qmcdu_group_step": (_I, [_VP, _VP, _I, _I, _D, _I, _I]),
    "qmcdu_group_destroy": (_I, [_VP]),
    "qmcdu_last_error": (ctypes.c_char_p, [_VP]),
    "qmcdu_philox4x32_10": (_I, [_VP, _VP, _VP, _VP, _I, _ULL, _VP, _VP]),
    "qmcdu_proposal_draws": (_I, [_I, _I, _ULL, _I, _VP, _VP, _VP]),
    "qmcdu_set_option": (_I, [_VP, _I, ctypes.c_longlong]),
    "qmcdu_sweep_shape": (_I, [_VP, _VP]),
    "qmcdu_profile_enable": (_I, [_VP, _I]),
    "qmcdu_profile_read": (_I, [_VP, _VP, _I]),
    "qmcdu_profile_sweep_times": (_I, [_VP, _VP, _I, ctypes.POINTER(_I)]),
    "qmcdu_ratio_noalloc": (_I, [_I, _I, _VP, _VP, _VP, _VP, _VP, _VP, _VP]),
    "qmcdu_gemm_bf16x3": (_I, [_I, _I, _I, _VP, _I, _VP, _I, _I, _VP, _I, ctypes.c_float,
                               ctypes.c_float, _VP]),
    "qmcdu_footprint": (_I, [_I, _I, _I, _I, ctypes.POINTER(_ULL)]),
    "qmcdu_load_walkers": (_I, [_VP, _I, _I, _VP, _VP]),
    "qmcdu_recompute_walkers": (_I, [_VP, _I, _I, _VP]),
    "qmcdu_sweep_walkers": (_I, [_VP, _I, _VP, _VP, _VP, _D, _VP, _VP, _VP]),
    "qmcdu_server_create": (_I, [_VP, ctypes.POINTER(_VP)]),
    "qmcdu_server_submit": (_I, [_VP, _VP, _I]),
    "qmcdu_server_run": (_I, [_VP, _D]),
    "qmcdu_server_results": (_I, [_VP, _VP, _I, ctypes.POINTER(_I)]),
    "qmcdu_server_trace": (_I, [_VP, _ULL, _VP, _VP]),
    "qmcdu_server_stats": (_I, [_VP, _VP, _I]),
    "qmcdu_server_class_stats": (_I, [_VP, _I, _VP, _I]),
    "qmcdu_server_error": (ctypes.c_char_p, [_VP]),
    "qmcdu_server_destroy": (_I, [_VP]),
    "qmcdu_version": (ctypes.c_char_p, []),
    "qmcdu_md_create": (_I, [_VP, _I, _I, _VP, _VP, ctypes.POINTER(_VP)]),
    "qmcdu_md_destroy": (_I, [_VP]),
    "qmcdu_md_set_virtuals": (_I, [_VP, _VP]),
    "qmcdu_md_ratio": (_I, [_VP, _VP, _VP, _VP, _VP, _VP]),
    "qmcdu_md_accept": (_I, [_VP, _VP]),
    "qmcdu_md_logpsi": (_I, [_VP, _VP, _VP]),
    "qmcdu_md_last_error": (ctypes.c_char_p, [_VP]),
}


class QmcduError(RuntimeError):
    def __init__(self, fn, status, text):
        super().__init__("%s -> %s (%d): %s" % (fn, STATUS.get(status, "?"), status, text))
        self.status = status


_lib = None


def load():
    """Load libqmcdu.so. Raises if the CUDA library has not been built: there is
    no fallback path."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIBRARY_PATH):
            raise RuntimeError("libqmcdu.so is missing at %s; build it with "
                               "`python -m paper_1708_00744_b300.build`" % LIBRARY_PATH)
        lib = ctypes.CDLL(LIBRARY_PATH)
        for name, (res, args) in SIGNATURES.items():
            f = getattr(lib, name)
            f.restype, f.argtypes = res, args
        _lib = lib
    return _lib


def _ptr(x):
    """Address of a torch tensor or numpy array (None -> NULL)."""
    if x is None:
        return None
    if isinstance(x, np.ndarray):
        if not x.flags["C_CONTIGUOUS"]:
            raise ValueError("array must be C-contiguous")
        return x.ctypes.data
    if hasattr(x, "data_ptr"):
        if not x.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return x.data_ptr()
    if isinstance(x, int):
        return x
    raise TypeError("expected a torch tensor, numpy array or address, got %r" % type(x))


def _stream_ptr(stream):
    if stream is None:
        return None
    if hasattr(stream, "cuda_stream"):
        return stream.cuda_stream
    return int(stream)


def _check(name, status, h=None):
    if status != 0:
        text = load().qmcdu_last_error(h).decode() if h else ""
        raise QmcduError(name, status, text)


def _is_cuda(x):
    return hasattr(x, "is_cuda") and x.is_cuda


def _need(x, n, kind, name, device):
    if x is None:
        return
    size = x.numel() if hasattr(x, "numel") else x.size
    if size < n:
        raise ValueError("%s: need %d elements, got %d" % (name, n, size))
    dt = str(x.dtype).replace("torch.", "")
    if dt != kind:
        raise TypeError("%s: dtype %s, expected %s" % (name, dt, kind))
    if device and not _is_cuda(x):
        raise ValueError("%s must be a CUDA tensor" % name)


# ---------------------------------------------------------------- C functions
def qmcdu_version():
    return load().qmcdu_version().decode()


def qmcdu_create(N, K, precision, batch, stream=None):
    h = ctypes.c_void_p()
    prec = PRECISIONS.get(precision, precision)
    _check("qmcdu_create", load().qmcdu_create(N, K, prec, batch, _stream_ptr(stream), ctypes.byref(h)))
    return h.value


def qmcdu_destroy(h):
    _check("qmcdu_destroy", load().qmcdu_destroy(h))


def qmcdu_set_matrix(h, A, N, batch):
    _need(A, batch * N * N, "float64", "A", False)
    _check("qmcdu_set_matrix", load().qmcdu_set_matrix(h, _ptr(A)), h)


def qmcdu_get_matrix(h, A_out, N, batch):
    _need(A_out, batch * N * N, "float64", "A_out", False)
    _check("qmcdu_get_matrix", load().qmcdu_get_matrix(h, _ptr(A_out)), h)


def qmcdu_get_inverse(h, Ainv_out, N, batch):
    _need(Ainv_out, batch * N * N, "float64", "Ainv_out", False)
    _check("qmcdu_get_inverse", load().qmcdu_get_inverse(h, _ptr(Ainv_out)), h)


def qmcdu_ratio(h, elec, v, ratio_out, N, batch):
    elec = np.ascontiguousarray(elec, dtype=np.int32)
    if elec.size != batch:
        raise ValueError("elec: need %d entries" % batch)
    _need(v, batch * N, "float64", "v", True)
    _need(ratio_out, batch, "float64", "ratio_out", True)
    _check("qmcdu_ratio", load().qmcdu_ratio(h, _ptr(elec), _ptr(v), _ptr(ratio_out)), h)


def qmcdu_accept(h, mask, batch):
    mask = np.ascontiguousarray(mask, dtype=np.uint8)
    if mask.size != batch:
        raise ValueError("mask: need %d entries" % batch)
    _check("qmcdu_accept", load().qmcdu_accept(h, _ptr(mask)), h)


def qmcdu_flush(h):
    _check("qmcdu_flush", load().qmcdu_flush(h), h)


def qmcdu_recompute(h, drift_out=None, batch=None):
    if drift_out is not None:
        _need(drift_out, 2 * batch, "float64", "drift_out", False)
    _check("qmcdu_recompute", load().qmcdu_recompute(h, _ptr(drift_out)), h)


def qmcdu_logdet(h, logabs, sign, batch):
    _need(logabs, batch, "float64", "logabs", False)
    _need(sign, batch, "int32", "sign", False)
    _check("qmcdu_logdet", load().qmcdu_logdet(h, _ptr(logabs), _ptr(sign)), h)


def qmcdu_logdet_product(h1, h2, logabs, sign, batch):
    _need(logabs, batch, "float64", "logabs", False)
    _need(sign, batch, "int32", "sign", False)
    _check("qmcdu_logdet_product", load().qmcdu_logdet_product(h1, h2, _ptr(logabs), _ptr(sign)), h1)


def qmcdu_sweep(h, base_seed, sweep_index, sigma, N, batch, override=None, accepted_out=None,
                ratios_out=None, near_ties_out=None):
    _need(override, batch * N, "int8", "override", False)
    _need(accepted_out, batch * N, "uint8", "accepted_out", False)
    _need(ratios_out, batch * N, "float64", "ratios_out", False)
    _need(near_ties_out, batch, "int64", "near_ties_out", False)
    _check("qmcdu_sweep", load().qmcdu_sweep(h, base_seed, sweep_index, sigma, _ptr(override),
                                             _ptr(accepted_out), _ptr(ratios_out),
                                             _ptr(near_ties_out)), h)


def qmcdu_ratio_noalloc(N, k, ainv_col, u, P, V, Kinv, ratio_out, stream=None):
    """Ratio of one proposal through a caller-held queue, with no device
    allocation (see include/qmcdu.h): u is the move's change of its row
    (v - a_j), V's rows the queued changes, Kinv = (I + V P')^{-1}."""
    for name, x, n in (("ainv_col", ainv_col, N), ("u", u, N), ("ratio_out", ratio_out, 1)):
        _need(x, n, "float64", name, True)
    if k > 0:
        for name, x, n in (("P", P, k * N), ("V", V, k * N), ("Kinv", Kinv, k * k)):
            _need(x, n, "float64", name, True)
    st = load().qmcdu_ratio_noalloc(N, k, _ptr(ainv_col), _ptr(u), _ptr(P if k else None),
                                    _ptr(V if k else None), _ptr(Kinv if k else None),
                                    _ptr(ratio_out), _stream_ptr(stream))
    if st != 0:
        raise QmcduError("qmcdu_ratio_noalloc", st, load().qmcdu_last_error(None).decode())


def qmcdu_gemm_bf16x3(A, B, C, alpha=1.0, beta=0.0, b_trans=False, stream=None):
    """C = alpha A B' + beta C on the tensor cores (split-bf16 x3); fp32 CUDA
    tensors, A: M x K, B: N x K (or K x N with b_trans), C: M x N, row-major."""
    M, K = A.shape
    N = B.shape[1] if b_trans else B.shape[0]
    for name, x in (("A", A), ("B", B), ("C", C)):
        _need(x, x.numel(), "float32", name, True)
    st = load().qmcdu_gemm_bf16x3(M, N, K, _ptr(A), A.stride(0), _ptr(B), B.stride(0),
                                  1 if b_trans else 0, _ptr(C), C.stride(0), float(alpha),
                                  float(beta), _stream_ptr(stream))
    if st != 0:
        raise QmcduError("qmcdu_gemm_bf16x3", st, load().qmcdu_last_error(None).decode())


def qmcdu_step(h, base_seed, first_sweep, nsweeps, sigma, N, batch, recompute=True,
               use_graph=False, accepted_out=None, drift_out=None):
    _need(accepted_out, nsweeps * batch * N, "uint8", "accepted_out", False)
    _need(drift_out, 2 * batch, "float64", "drift_out", False)
    _check("qmcdu_step", load().qmcdu_step(h, base_seed, first_sweep, nsweeps, sigma,
                                           1 if recompute else 0, 1 if use_graph else 0,
                                           _ptr(accepted_out), _ptr(drift_out)), h)


def qmcdu_step_results(h, nsweeps, N, batch, accepted_out=None, ratios_out=None,
                       near_ties_out=None):
    _need(accepted_out, nsweeps * batch * N, "uint8", "accepted_out", False)
    _need(ratios_out, nsweeps * batch * N, "float64", "ratios_out", False)
    _need(near_ties_out, nsweeps * batch, "int64", "near_ties_out", False)
    _check("qmcdu_step_results", load().qmcdu_step_results(h, nsweeps, _ptr(accepted_out),
                                                           _ptr(ratios_out), _ptr(near_ties_out)), h)


def qmcdu_group_create(handles):
    arr = (ctypes.c_void_p * len(handles))(*handles)
    g = ctypes.c_void_p()
    _check("qmcdu_group_create", load().qmcdu_group_create(arr, len(handles), ctypes.byref(g)))
    return g.value


def qmcdu_group_step(g, seeds, first_sweep, nsweeps, sigma, recompute=True, use_graph=False):
    seeds = np.ascontiguousarray(seeds, dtype=np.uint64)
    _check("qmcdu_group_step", load().qmcdu_group_step(g, _ptr(seeds), first_sweep, nsweeps, sigma,
                                                       1 if recompute else 0,
                                                       1 if use_graph else 0))


def qmcdu_group_destroy(g):
    _check("qmcdu_group_destroy", load().qmcdu_group_destroy(g))


def qmcdu_sync(h):
    _check("qmcdu_sync", load().qmcdu_sync(h), h)


def qmcdu_last_error(h):
    return load().qmcdu_last_error(h).decode()


def qmcdu_philox4x32_10(c0, c1, c2, c3, seed, out, stream=None):
    n = c0.numel()
    for name, x in (("c0", c0), ("c1", c1), ("c2", c2), ("c3", c3)):
        _need(x, n, "int32", name, True)
    _need(out, 4 * n, "int32", "out", True)
    _check("qmcdu_philox4x32_10", load().qmcdu_philox4x32_10(
        _ptr(c0), _ptr(c1), _ptr(c2), _ptr(c3), n, seed, _ptr(out), _stream_ptr(stream)))


def qmcdu_proposal_draws(N, nwalkers, base_seed, sweep, gauss_out, unif_out, stream=None):
    """The Gaussians and uniforms of one sweep of walkers 0..nwalkers-1 as the
    device draws them (CUDA tensors [nwalkers][N][N] and [nwalkers][N] fp64)."""
    _need(gauss_out, nwalkers * N * N, "float64", "gauss_out", True)
    _need(unif_out, nwalkers * N, "float64", "unif_out", True)
    st = load().qmcdu_proposal_draws(N, nwalkers, base_seed, sweep, _ptr(gauss_out), _ptr(unif_out),
                                     _stream_ptr(stream))
    if st != 0:
        raise QmcduError("qmcdu_proposal_draws", st, load().qmcdu_last_error(None).decode())


OPTIONS = {"sweep_persistent": 1, "ratio_ctas": 2, "flush_ctas": 3, "wait_budget_ns": 4,
           "test_stall": 5, "max_ctas": 6, "group_ctas": 7, "fp64_flush": 8,
           "cluster": 9, "fixed_slot": 10}


def qmcdu_set_option(h, option, value):
    _check("qmcdu_set_option", load().qmcdu_set_option(h, OPTIONS.get(option, option), int(value)), h)


def qmcdu_sweep_shape(h):
    out = np.zeros(5, dtype=np.int32)
    _check("qmcdu_sweep_shape", load().qmcdu_sweep_shape(h, _ptr(out)), h)
    return dict(zip(("flush_ctas", "ratio_ctas", "groups", "chunk", "col_tile"), out.tolist()))


PROFILE_FIELDS = ("launches", "flushes", "flush_ms", "recomputes", "recompute_ms", "sweep_syncs",
                  "ratio_launches", "accept_launches", "sweep_dots_ms", "sweep_stage_ms",
                  "sweep_barrier_ms", "sweep_decide_ms", "sweep_accept_ms", "sweep_flushbar1_ms",
                  "sweep_flush_ms", "sweep_flushbar2_ms", "sweep_kernels", "sweep_kernel_ms",
                  "sweep_oz_products_ms", "sweep_oz_slicing_ms", "sweep_oz_update_ms")


def qmcdu_profile_enable(h, enable=True):
    _check("qmcdu_profile_enable", load().qmcdu_profile_enable(h, 1 if enable else 0), h)


def qmcdu_profile_sweep_times(h, max_n=1 << 16):
    """Per-launch device times (ms) of the persistent sweeps while profiling."""
    out = np.zeros(max_n)
    n = _I()
    _check("qmcdu_profile_sweep_times", load().qmcdu_profile_sweep_times(h, _ptr(out), max_n,
                                                                         ctypes.byref(n)), h)
    return out[:n.value].copy()


def qmcdu_profile_read(h):
    out = np.zeros(len(PROFILE_FIELDS))
    _check("qmcdu_profile_read", load().qmcdu_profile_read(h, _ptr(out), out.size), h)
    return dict(zip(PROFILE_FIELDS, out.tolist()))


# ---------------------------------------------------------------- walker subsets
def qmcdu_footprint(N, K, precision, batch):
    """Device bytes a handle of these sizes allocates (host only, no GPU needed)."""
    out = _ULL()
    _check("qmcdu_footprint", load().qmcdu_footprint(N, K, PRECISIONS.get(precision, precision),
                                                     batch, ctypes.byref(out)))
    return out.value


def qmcdu_load_walkers(h, first, count, N, A=None, seeds=None):
    if A is not None:
        _need(A, count * N * N, "float64", "A", False)
    if seeds is not None:
        seeds = np.ascontiguousarray(seeds, dtype=np.uint64)
        _need(seeds, count, "uint64", "seeds", False)
    _check("qmcdu_load_walkers", load().qmcdu_load_walkers(h, first, count, _ptr(A), _ptr(seeds)), h)


def qmcdu_recompute_walkers(h, first, count, drift_out=None):
    _need(drift_out, 2 * count, "float64", "drift_out", False)
    _check("qmcdu_recompute_walkers",
           load().qmcdu_recompute_walkers(h, first, count, _ptr(drift_out)), h)


def qmcdu_sweep_walkers(h, walkers, seeds, sweeps, sigma, N, accepted_out=None, ratios_out=None,
                        near_ties_out=None):
    walkers = np.ascontiguousarray(walkers, dtype=np.int32)
    seeds = np.ascontiguousarray(seeds, dtype=np.uint64)
    sweeps = np.ascontiguousarray(sweeps, dtype=np.int32)
    n = walkers.size
    if seeds.size != n or sweeps.size != n:
        raise ValueError("walkers, seeds and sweeps must have the same length")
    _need(accepted_out, n * N, "uint8", "accepted_out", False)
    _need(ratios_out, n * N, "float64", "ratios_out", False)
    _need(near_ties_out, n, "int64", "near_ties_out", False)
    _check("qmcdu_sweep_walkers",
           load().qmcdu_sweep_walkers(h, n, _ptr(walkers), _ptr(seeds), _ptr(sweeps), sigma,
                                      _ptr(accepted_out), _ptr(ratios_out), _ptr(near_ties_out)),
           h)


# ---------------------------------------------------------------- serving loop
SERVER_MAX_CLASSES = 16
_IARR = ctypes.c_int * SERVER_MAX_CLASSES


class ServerConfig(ctypes.Structure):
    _fields_ = [("precision", _I), ("recompute_every", _I), ("sigma", _D),
                ("hbm_budget", _ULL), ("num_classes", _I), ("class_N", _IARR),
                ("class_K", _IARR), ("class_slots", _IARR), ("class_group_ctas", _IARR),
                ("max_inflight", _I), ("max_walkers", _I), ("keep_traces", _I),
                ("simulate", _I), ("sim_flops", _D), ("sim_fp64_flops", _D),
                ("sim_proposal_s", _D), ("sm_oversubscription", _D)]


class Request(ctypes.Structure):
    _fields_ = [("id", _ULL), ("seed", _ULL), ("N", _I), ("nsweeps", _I), ("arrival_s", _D)]


class Result(ctypes.Structure):
    _fields_ = [("id", _ULL), ("N", _I), ("nsweeps", _I), ("status", _I), ("pool", _I),
                ("arrival_s", _D), ("admit_s", _D), ("done_s", _D), ("accepted", ctypes.c_longlong),
                ("near_ties", ctypes.c_longlong), ("recomputes", _I), ("sign", _I),
                ("logabs", _D), ("drift_logdet", _D), ("drift_inverse", _D),
                ("sweep_ms_mean", _D), ("sweep_ms_max", _D), ("first_round", ctypes.c_longlong),
                ("last_round", ctypes.c_longlong)]


SERVER_STATS = ("clock_s", "submitted", "finished", "failed", "walker_sweeps", "accepted",
                "proposals", "sweep_ms_p50", "sweep_ms_p99", "request_s_p50", "request_s_p99",
                "wait_s_p50", "wait_s_p99", "peak_bytes", "budget_bytes", "pools_created",
                "pools_destroyed", "rounds", "max_resident", "max_inflight",
                "mixed_walker_sweeps", "last_round_end_s")


def _server_check(name, status, s):
    if status != 0:
        raise QmcduError(name, status, load().qmcdu_server_error(s).decode() if s else "")


def qmcdu_server_create(cfg):
    s = _VP()
    _server_check("qmcdu_server_create", load().qmcdu_server_create(ctypes.byref(cfg), ctypes.byref(s)),
                  None)
    return s.value


def qmcdu_server_submit(s, reqs):
    arr = (Request * len(reqs))(*reqs)
    _server_check("qmcdu_server_submit", load().qmcdu_server_submit(s, ctypes.addressof(arr), len(reqs)), s)


def qmcdu_server_run(s, until_s=-1.0):
    _server_check("qmcdu_server_run", load().qmcdu_server_run(s, until_s), s)


def qmcdu_server_results(s, max_results=4096):
    arr = (Result * max_results)()
    n = _I()
    _server_check("qmcdu_server_results",
                  load().qmcdu_server_results(s, ctypes.addressof(arr), max_results, ctypes.byref(n)), s)
    return [{f: getattr(arr[i], f) for f, _ in Result._fields_} for i in range(n.value)]


def qmcdu_server_trace(s, req_id, nsweeps, N):
    acc = np.zeros((nsweeps, N), dtype=np.uint8)
    rat = np.zeros((nsweeps, N))
    _server_check("qmcdu_server_trace", load().qmcdu_server_trace(s, req_id, _ptr(acc), _ptr(rat)), s)
    return acc, rat


def qmcdu_server_stats(s):
    out = np.zeros(len(SERVER_STATS))
    _server_check("qmcdu_server_stats", load().qmcdu_server_stats(s, _ptr(out), out.size), s)
    return dict(zip(SERVER_STATS, out.tolist()))


SERVER_CLASS_STATS = ("walker_sweeps", "sweep_ms_p50", "sweep_ms_p99", "finished",
                      "request_s_p50", "request_s_p99", "accepted")


def qmcdu_server_class_stats(s, cls):
    out = np.zeros(len(SERVER_CLASS_STATS))
    _server_check("qmcdu_server_class_stats",
                  load().qmcdu_server_class_stats(s, cls, _ptr(out), out.size), s)
    return dict(zip(SERVER_CLASS_STATS, out.tolist()))


def qmcdu_server_destroy(s):
    _server_check("qmcdu_server_destroy", load().qmcdu_server_destroy(s), None)


class Server:
    """The library's serving loop (qmcdu_server_*).

    classes: list of dicts with N and optionally K, slots, group_ctas.
    """

    def __init__(self, classes, precision="fp32", sigma=0.1, recompute_every=10,
                 hbm_budget=150 * 10**9, max_inflight=0, max_walkers=0, keep_traces=False,
                 simulate=False, sim_flops=10e12, sim_fp64_flops=0.3e12, sim_proposal_s=10e-6,
                 sm_oversubscription=0.0):
        if not 1 <= len(classes) <= SERVER_MAX_CLASSES:
            raise ValueError("1..%d size classes" % SERVER_MAX_CLASSES)
        cfg = ServerConfig()
        cfg.precision = PRECISIONS.get(precision, precision)
        cfg.recompute_every = recompute_every
        cfg.sigma = sigma
        cfg.hbm_budget = int(hbm_budget)
        cfg.num_classes = len(classes)
        for i, c in enumerate(classes):
            cfg.class_N[i] = c["N"]
            cfg.class_K[i] = c.get("K", 0)
            cfg.class_slots[i] = c.get("slots", 0)
            cfg.class_group_ctas[i] = c.get("group_ctas", 0)
        cfg.max_inflight, cfg.max_walkers = max_inflight, max_walkers
        cfg.keep_traces, cfg.simulate = int(bool(keep_traces)), int(bool(simulate))
        cfg.sim_flops, cfg.sim_fp64_flops, cfg.sim_proposal_s = sim_flops, sim_fp64_flops, sim_proposal_s
        cfg.sm_oversubscription = sm_oversubscription
        self.s = qmcdu_server_create(cfg)

    def submit(self, requests):
        """requests: iterable of dicts with id, seed, N, nsweeps, arrival_s."""
        qmcdu_server_submit(self.s, [Request(int(r["id"]), int(r["seed"]), int(r["N"]),
                                             int(r["nsweeps"]), float(r["arrival_s"]))
                                     for r in requests])

    def run(self, until_s=-1.0):
        qmcdu_server_run(self.s, until_s)

    def results(self, max_results=4096):
        out = []
        while True:
            got = qmcdu_server_results(self.s, max_results)
            out += got
            if len(got) < max_results:
                return out

    def trace(self, req_id, nsweeps, N):
        return qmcdu_server_trace(self.s, req_id, nsweeps, N)

    def stats(self):
        return qmcdu_server_stats(self.s)

    def class_stats(self, cls):
        return qmcdu_server_class_stats(self.s, cls)

    def close(self):
        if self.s:
            qmcdu_server_destroy(self.s)
            self.s = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ---------------------------------------------------------------- handle object
class Walkers:
    """A qmcdu handle: `batch` walkers of N electrons with delay K.

    Methods forward to the C functions of the same name (without the prefix).
    """

    def __init__(self, N, K, precision="fp64", batch=1, stream=None):
        self.N, self.K, self.batch = int(N), int(K), int(batch)
        self.precision = precision
        self.h = qmcdu_create(self.N, self.K, precision, self.batch, stream)

    def close(self):
        if self.h:
            qmcdu_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def set_matrix(self, A):
        qmcdu_set_matrix(self.h, A, self.N, self.batch)

    def get_matrix(self, out):
        qmcdu_get_matrix(self.h, out, self.N, self.batch)
        return out

    def get_inverse(self, out):
        qmcdu_get_inverse(self.h, out, self.N, self.batch)
        return out

    def ratio(self, elec, v, ratio_out):
        qmcdu_ratio(self.h, elec, v, ratio_out, self.N, self.batch)

    def accept(self, mask):
        qmcdu_accept(self.h, mask, self.batch)

    def flush(self):
        qmcdu_flush(self.h)

    def recompute(self, drift_out=None):
        qmcdu_recompute(self.h, drift_out, self.batch)

    def logdet(self, logabs, sign):
        qmcdu_logdet(self.h, logabs, sign, self.batch)

    def sweep(self, base_seed, sweep_index, sigma, override=None, accepted_out=None,
              ratios_out=None, near_ties_out=None):
        qmcdu_sweep(self.h, base_seed, sweep_index, sigma, self.N, self.batch, override,
                    accepted_out, ratios_out, near_ties_out)

    def sync(self):
        qmcdu_sync(self.h)

    def step(self, base_seed, first_sweep, nsweeps, sigma, recompute=True, use_graph=False,
             accepted_out=None, drift_out=None):
        qmcdu_step(self.h, base_seed, first_sweep, nsweeps, sigma, self.N, self.batch, recompute,
                   use_graph, accepted_out, drift_out)

    def step_results(self, nsweeps, accepted_out=None, ratios_out=None, near_ties_out=None):
        qmcdu_step_results(self.h, nsweeps, self.N, self.batch, accepted_out, ratios_out,
                           near_ties_out)

    def set_option(self, option, value):
        qmcdu_set_option(self.h, option, value)

    def sweep_shape(self):
        return qmcdu_sweep_shape(self.h)

    def load_walkers(self, first, count, A=None, seeds=None):
        qmcdu_load_walkers(self.h, first, count, self.N, A, seeds)

    def recompute_walkers(self, first, count, drift_out=None):
        qmcdu_recompute_walkers(self.h, first, count, drift_out)

    def sweep_walkers(self, walkers, seeds, sweeps, sigma, accepted_out=None, ratios_out=None,
                      near_ties_out=None):
        qmcdu_sweep_walkers(self.h, walkers, seeds, sweeps, sigma, self.N, accepted_out,
                            ratios_out, near_ties_out)

    def profile_enable(self, enable=True):
        qmcdu_profile_enable(self.h, enable)

    def profile_read(self):
        return qmcdu_profile_read(self.h)

    def profile_sweep_times(self):
        return qmcdu_profile_sweep_times(self.h)


# ---------------------------------------------------------------- multideterminant walkers
def _md_check(name, status, m=None):
    if status != 0:
        text = load().qmcdu_md_last_error(m).decode() if m else load().qmcdu_last_error(None).decode()
        raise QmcduError(name, status, text)


class MultiDetWalkers:
    """Psi = sum_I coef_I det(A_I) over a handle's walkers (include/qmcdu.h,
    qmcdu_md_*): exc [ndet][4] (o1, a1, o2, a2; -1 unused), coef [ndet], nv
    virtual orbitals. Uses the handle's qmcdu_ratio / qmcdu_accept."""

    def __init__(self, walkers, nv, exc, coef):
        self.W = walkers
        self.nv = int(nv)
        exc = np.ascontiguousarray(exc, dtype=np.int32).reshape(-1, 4)
        coef = np.ascontiguousarray(coef, dtype=np.float64).reshape(-1)
        m = ctypes.c_void_p()
        _md_check("qmcdu_md_create", load().qmcdu_md_create(walkers.h, self.nv, exc.shape[0], _ptr(exc),
                                                            _ptr(coef), ctypes.byref(m)))
        self.m = m.value

    def set_virtuals(self, B):
        _need(B, self.W.batch * self.W.N * self.nv, "float64", "B", False)
        _md_check("qmcdu_md_set_virtuals", load().qmcdu_md_set_virtuals(self.m, _ptr(B)), self.m)

    def ratio(self, elec, v, w, ratio_out, ref_ratio_out=None):
        elec = np.ascontiguousarray(elec, dtype=np.int32)
        _need(v, self.W.batch * self.W.N, "float64", "v", True)
        _need(w, self.W.batch * self.nv, "float64", "w", True)
        _need(ratio_out, self.W.batch, "float64", "ratio_out", True)
        _need(ref_ratio_out, self.W.batch, "float64", "ref_ratio_out", True)
        _md_check("qmcdu_md_ratio", load().qmcdu_md_ratio(self.m, _ptr(elec), _ptr(v), _ptr(w), _ptr(ratio_out),
                                                          _ptr(ref_ratio_out)), self.m)

    def accept(self, mask):
        mask = np.ascontiguousarray(mask, dtype=np.uint8)
        _md_check("qmcdu_md_accept", load().qmcdu_md_accept(self.m, _ptr(mask)), self.m)

    def logpsi(self, logabs, sign):
        _need(logabs, self.W.batch, "float64", "logabs", False)
        _need(sign, self.W.batch, "int32", "sign", False)
        _md_check("qmcdu_md_logpsi", load().qmcdu_md_logpsi(self.m, _ptr(logabs), _ptr(sign)), self.m)

    def close(self):
        if getattr(self, "m", None):
            load().qmcdu_md_destroy(self.m)
            self.m = None
