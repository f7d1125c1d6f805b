"""CPU oracle for the delayed Slater-determinant update (fp64, plain C).

TEST INFRASTRUCTURE ONLY: the test suite, the smoke check and the CPU-baseline
leg of the benchmark are the only callers. The product path never imports it.

Readings of the paper, all in its column convention (one column of the
Slater matrix per electron, Sec. I), each loaded from qmc_oracle.c:
  BRUTE   ratio = det(M_new) / det(M) by two LU determinants (direct calculation)
  SM      ratio by the matrix determinant lemma (Eq. 1), inverse by the
          Sherman-Morrison rank-1 formula (Eq. 2)
  DELAYED ratios by look-ahead determinants of I_k + V'M^{-1}U (Eq. 3), queued
          accepted moves applied en bloc by Sherman-Morrison-Woodbury (Eq. 4)
          when k reaches K or the sweep ends (Sec. II)
  DELAYED_SLOT  the same with Sec. II's fixed slots: a rejected proposal also
          takes a queue slot, as an unchanged column (a zero change), so the
          queue is flushed every K proposals
plus LU log|det| and LU inverse. Inputs and outputs use the row convention of
the library (row j of A = electron j); inverses come back in the column-major
layout of A^{-1} (row c of the returned array is column c of A^{-1}).

Pins (tests/test_oracle_pins.py) tie every function to something other than
itself: Leibniz-formula determinants, exact rational arithmetic, closed forms
(Hilbert, Vandermonde, diagonal, permutation) and the paper's invariants.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "qmc_oracle.c")
_LIB = os.path.join(_HERE, "libqmc_oracle.so")

BRUTE, SM, DELAYED, DELAYED_SLOT = 0, 1, 2, 3
OK, ERR_ARG, ERR_SINGULAR, ERR_OOM = 0, 1, 3, 4


class OracleError(RuntimeError):
    pass


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (plain -O2, no FMA contraction, OpenMP for
    the loops over independent output elements)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".tmp.%d" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-fopenmp", "-fPIC", "-shared",
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


_lib = None


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        dp, ip, i8p, u8p = (ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int),
                            ctypes.POINTER(ctypes.c_int8), ctypes.POINTER(ctypes.c_uint8))
        lib.oracle_slogdet.argtypes = [ctypes.c_int, dp, dp, ip]
        lib.oracle_inverse.argtypes = [ctypes.c_int, dp, dp]
        lib.oracle_sweeps.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                      ctypes.c_double, dp, dp, dp, i8p, dp, dp, u8p, dp, dp, dp, ip,
                                      ctypes.POINTER(ctypes.c_longlong), ctypes.c_longlong]
        lib.oracle_moves.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, dp,
                                     ip, dp, u8p, u8p, dp, dp, dp, dp, dp, ip]
        lib.oracle_md_sweeps.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                         ctypes.c_double, dp, dp, dp, dp, dp, ctypes.c_int, ip, dp, i8p,
                                         dp, u8p, dp, dp, dp, ip]
        lib.oracle_md_sweeps.restype = ctypes.c_int
        lib.oracle_set_threads.argtypes = [ctypes.c_int]
        lib.oracle_last_update_seconds.argtypes = []
        lib.oracle_last_update_seconds.restype = ctypes.c_double
        for f in (lib.oracle_slogdet, lib.oracle_inverse, lib.oracle_sweeps, lib.oracle_moves,
                  lib.oracle_set_threads):
            f.restype = ctypes.c_int
        _lib = lib
    return _lib


def last_update_seconds() -> float:
    """Wall seconds of the last sweeps() call after its setup (the LU
    determinant and inverse of the starting matrix): the update work alone."""
    return _load().oracle_last_update_seconds()


def set_threads(n: int = 0) -> int:
    """Threads of the oracle's parallel loops (n <= 0: every processor of
    the host). Results are identical for every count: each output element is
    computed by one thread in the single-thread order. Returns the count."""
    return _load().oracle_set_threads(int(n))


def _p(a, ct):
    return a.ctypes.data_as(ctypes.POINTER(ct)) if a is not None else None


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def slogdet(a):
    """(sign, log|det a|) by LU with partial pivoting."""
    a = _f64(a)
    n = a.shape[0]
    la, sg = ctypes.c_double(), ctypes.c_int()
    st = _load().oracle_slogdet(n, _p(a, ctypes.c_double), ctypes.byref(la), ctypes.byref(sg))
    if st not in (OK, ERR_SINGULAR):
        raise OracleError("oracle_slogdet status %d" % st)
    return sg.value, la.value


def inverse(a):
    """a^{-1} (row-major) by LU and triangular solves."""
    a = _f64(a)
    n = a.shape[0]
    out = np.zeros((n, n))
    st = _load().oracle_inverse(n, _p(a, ctypes.c_double), _p(out, ctypes.c_double))
    if st != OK:
        raise OracleError("oracle_inverse status %d" % st)
    return out


def inverse_colmajor(a):
    """A^{-1} in the library's layout: row c holds column c of A^{-1}."""
    return np.ascontiguousarray(inverse(a).T)


ALT_INIT = 16      # added to a method: start from the inverse by the LU of A (not of A')


def sweeps(method, A0, G, U, sigma, K=1, override=None, max_moves=-1):
    """Metropolis sweeps from A0 with Gaussians G[s, j, :] and uniforms U[s, j].

    max_moves >= 0 stops after that many proposals (a bounded sample).
    method + ALT_INIT starts the walk from the inverse computed by the LU of
    A (then transposed) instead of the LU of the paper's M = A'.
    Returns dict(ratios, accepted, A, Ainv (column-major layout), logabs, sign,
    near_ties, terms). terms[s, j] = 1 + sum_i |(A^{-1})_ij (v - a_j)_i|, the
    size of the terms of proposal j's Eq. 1 dot product (with the inverse of
    the last flush for the delayed readings): it bounds that dot product's
    rounding error."""
    A0 = _f64(A0)
    n = A0.shape[0]
    G = _f64(G).reshape(-1, n, n)
    ns = G.shape[0]
    U = _f64(U).reshape(ns, n)
    ov = None if override is None else np.ascontiguousarray(override, dtype=np.int8).reshape(ns, n)
    ratios = np.zeros((ns, n))
    terms = np.zeros((ns, n))
    acc = np.zeros((ns, n), dtype=np.uint8)
    A = np.zeros((n, n))
    Ainv = np.zeros((n, n))
    la, sg, nt = ctypes.c_double(), ctypes.c_int(), ctypes.c_longlong()
    st = _load().oracle_sweeps(method, n, K, ns, float(sigma), _p(A0, ctypes.c_double),
                               _p(G, ctypes.c_double), _p(U, ctypes.c_double),
                               _p(ov, ctypes.c_int8), _p(ratios, ctypes.c_double),
                               _p(terms, ctypes.c_double),
                               _p(acc, ctypes.c_uint8), _p(A, ctypes.c_double),
                               _p(Ainv, ctypes.c_double), ctypes.byref(la), ctypes.byref(sg),
                               ctypes.byref(nt), int(max_moves))
    if st != OK:
        raise OracleError("oracle_sweeps status %d" % st)
    return dict(ratios=ratios, accepted=acc.astype(bool), A=A, Ainv=Ainv,
                logabs=la.value, sign=sg.value, near_ties=nt.value, terms=terms)


def moves(method, A0, elec, vrows, decisions, K=1, flush_after=None):
    """Explicit moves with given decisions. Returns dict(ratios, A, Ainv, logabs, sign,
    terms) (terms as in sweeps())."""
    A0 = _f64(A0)
    n = A0.shape[0]
    elec = np.ascontiguousarray(elec, dtype=np.int32)
    m = elec.shape[0]
    vrows = _f64(vrows).reshape(m, n)
    dec = np.ascontiguousarray(decisions, dtype=np.uint8).reshape(m)
    fa = None if flush_after is None else np.ascontiguousarray(flush_after, dtype=np.uint8)
    ratios = np.zeros(m)
    terms = np.zeros(m)
    A = np.zeros((n, n))
    Ainv = np.zeros((n, n))
    la, sg = ctypes.c_double(), ctypes.c_int()
    st = _load().oracle_moves(method, n, K, m, _p(A0, ctypes.c_double),
                              elec.ctypes.data_as(ctypes.POINTER(ctypes.c_int)),
                              _p(vrows, ctypes.c_double), _p(dec, ctypes.c_uint8),
                              _p(fa, ctypes.c_uint8), _p(ratios, ctypes.c_double),
                              _p(terms, ctypes.c_double),
                              _p(A, ctypes.c_double), _p(Ainv, ctypes.c_double),
                              ctypes.byref(la), ctypes.byref(sg))
    if st != OK:
        raise OracleError("oracle_moves status %d" % st)
    return dict(ratios=ratios, A=A, Ainv=Ainv, logabs=la.value, sign=sg.value, terms=terms)


MD_BRUTE, MD_TABLE, MD_TABLE_DELAYED = 0, 1, 2


def md_sweeps(method, A0, B0, G, H, U, sigma, exc, coef, override=None, K=1):
    """Metropolis sweeps of a multideterminant walker, Psi = sum_I coef_I
    det(A_I): A_I is A (electron rows, occupied orbital columns) with occupied
    columns o_p replaced by columns a_p of B (the virtual orbitals at the
    electrons), exc[I] = (o1, a1, o2, a2) with -1 for unused pairs.
    Proposals v = a_j + sigma G[s, j], w = b_j + sigma H[s, j]; accept iff
    u < min(1, R^2), R = Psi(new) / Psi(old).
      MD_BRUTE  R from every det(A_I) by LU (the definition)
      MD_TABLE  Clark et al.'s table T = A^{-1} B with the reference ratio of
                Eq. 1 and Sherman-Morrison updates of A^{-1} and T
      MD_TABLE_DELAYED  the same table with the reference inverse under the
                delayed update (Eq. 3-4, queue length K): the current column
                A^{-1} e_j by the Woodbury form, Eq. 4 when K moves wait or
                a queued electron moves again
    Returns dict(ratios, accepted, A, B, logabs, sign) (log|Psi|, sign Psi)."""
    A0, B0 = _f64(A0), _f64(B0)
    n, nv = A0.shape[0], B0.shape[1]
    G = _f64(G).reshape(-1, n, n)
    ns = G.shape[0]
    H = _f64(H).reshape(ns, n, nv)
    U = _f64(U).reshape(ns, n)
    exc = np.ascontiguousarray(exc, dtype=np.int32).reshape(-1, 4)
    coef = _f64(coef).reshape(-1)
    ov = None if override is None else np.ascontiguousarray(override, dtype=np.int8).reshape(ns, n)
    ratios = np.zeros((ns, n))
    acc = np.zeros((ns, n), dtype=np.uint8)
    A = np.zeros((n, n))
    B = np.zeros((n, nv))
    la, sg = ctypes.c_double(), ctypes.c_int()
    st = _load().oracle_md_sweeps(method, int(K), n, nv, ns, float(sigma), _p(A0, ctypes.c_double),
                                  _p(B0, ctypes.c_double), _p(G, ctypes.c_double), _p(H, ctypes.c_double),
                                  _p(U, ctypes.c_double), exc.shape[0],
                                  exc.ctypes.data_as(ctypes.POINTER(ctypes.c_int)),
                                  _p(coef, ctypes.c_double), _p(ov, ctypes.c_int8),
                                  _p(ratios, ctypes.c_double), _p(acc, ctypes.c_uint8),
                                  _p(A, ctypes.c_double), _p(B, ctypes.c_double),
                                  ctypes.byref(la), ctypes.byref(sg))
    if st != OK:
        raise OracleError("oracle_md_sweeps status %d" % st)
    return dict(ratios=ratios, accepted=acc.astype(bool), A=A, B=B, logabs=la.value, sign=sg.value)
