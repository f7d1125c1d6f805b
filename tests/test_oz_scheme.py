"""The arithmetic of the emulated-fp64 flush (Eq. 4 on 16-bit tensor
products), modelled on the CPU with exact integers: its exactness bounds and
its accuracy against an extended-precision evaluation of Eq. 4.

Scheme (the sweep kernel's flush): every fp64 operand is cut into NS signed
8-bit slices relative to a power of two shared by its row (V, W) or column
(A^{-1}, T), q = round(|x| 2^(1078 - Emax)) = sum_j s_j 2^(48 - 8 j); slice
products (at most 255^2) are summed exactly while partial sums stay below
2^24 (the fp32 accumulator's exact range); the pairs with j + l <= 6 are kept
and recombined per diagonal d = j + l. Phase A (T' = V A^{-1}) recombines the
d <= 3 diagonals exactly and d = 4..6 as an fp32 tail; phase C (A^{-1} -= W T)
folds the seventh diagonal in at half a unit and rounds once to fp64 before
the fp64 subtraction."""
import numpy as np
import pytest

AR, CK = 256, 32          # rows summed per phase A partial; contraction length in phase C


def bexp(x):
    return ((np.ascontiguousarray(x, dtype=np.float64).view(np.uint64) >> np.uint64(52))
            & np.uint64(0x7FF)).astype(np.int64)


def cut(x, emax, ns=7):
    """ns signed byte slices of x relative to the biased exponent emax
    (broadcast against x): returns s[j] (int64) with
    x ~ sum_j s[j] 2^(emax - 1030 - 8 j)."""
    x = np.ascontiguousarray(x, dtype=np.float64)
    b = x.view(np.uint64)
    E = ((b >> np.uint64(52)) & np.uint64(0x7FF)).astype(np.int64)
    m = ((b & np.uint64((1 << 52) - 1)) | np.uint64(1 << 52)).astype(np.int64)
    t = np.broadcast_to(emax, E.shape) - E                 # q = round(8 m / 2^t)
    m3 = m << 3
    q = np.where(t <= 0, m3 << np.clip(-t, 0, 3),
                 (m3 + (np.int64(1) << np.clip(t - 1, 0, 62))) >> np.clip(t, 0, 63))
    q = np.where((E == 0) | (t > 62), 0, np.minimum(q, (1 << 56) - 1))
    q >>= 8 * (7 - ns)                                     # fewer slices: drop the low bytes
    sg = np.where(x < 0, -1, 1)
    return [sg * ((q >> (8 * (ns - 1 - j))) & 0xFF) for j in range(ns)]


def pow2(e):
    return np.ldexp(1.0, np.asarray(e, dtype=np.int64))


def phase_a(V, Ainv, ns=7):
    """T'[m][c] = sum_i V[m][i] Ainv[i][c] as the flush recombines it."""
    em = bexp(V).max(axis=1)[:, None]
    ec = bexp(Ainv).max(axis=0)[None, :]
    v, a = cut(V, em, ns), cut(Ainv, ec, ns)
    N = V.shape[1]
    out = np.zeros((V.shape[0], Ainv.shape[1]))
    for r0 in range(0, N, AR):                             # partials over row chunks
        sl = slice(r0, r0 + AR)
        D = [sum(v[l][:, sl] @ a[d - l][sl, :] for l in range(max(0, d - ns + 1), min(d, ns - 1) + 1))
             for d in range(min(7, 2 * ns - 1))]
        S = np.zeros(out.shape, dtype=object)
        for d in range(min(4, len(D))):
            S = S * 256 + D[d].astype(object)
        g = np.zeros(out.shape, dtype=np.float32)
        for d in range(len(D) - 1, 3, -1):                 # the fp32 tail, d = 6, 5, 4
            g = (g / np.float32(256) if d < len(D) - 1 else g) + D[d].astype(np.float32)
        if len(D) > 4:
            g = g / np.float32(256) ** (6 - (len(D) - 1))
        val = (S.astype(np.float64) + g.astype(np.float64) / 256.0) * pow2(ec + em - 2084)
        out += val
    return out


def phase_c(W, T, ns=7):
    """U[i][c] = sum_m W[i][m] T[m][c] rounded once to fp64 as the flush does."""
    ei = bexp(W).max(axis=1)[:, None]
    et = bexp(T).max(axis=0)[None, :]
    w, t = cut(W, ei, ns), cut(T, et, ns)
    D = [sum(w[j] @ t[d - j] for j in range(max(0, d - ns + 1), min(d, ns - 1) + 1))
         for d in range(min(7, 2 * ns - 1))]
    for Dd in D:
        assert np.abs(Dd).max() < 2 ** 24                  # exact in the fp32 accumulator
    S = np.zeros(D[0].shape, dtype=object)
    for d in range(min(6, len(D))):
        S = S * 256 + D[d].astype(object)
    S = S * 2 + (((D[6] + 64) >> 7).astype(object) if len(D) > 6 else 0)
    scale = (ei + et - 2101) - 8 * (6 - min(6, len(D)))
    exact = np.vectorize(lambda s: float(s), otypes=[np.float64])(S)   # one rounding to fp64
    return exact * pow2(scale)


def flush_case(N, k, seed):
    rng = np.random.default_rng(seed)
    A = rng.standard_normal((N, N))
    Ainv = np.linalg.inv(A)
    idx = rng.choice(N, k, replace=False)
    V = A[idx] + 0.5 * rng.standard_normal((k, N))
    W = Ainv[:, idx] @ np.linalg.inv(V @ Ainv[:, idx])
    E = np.zeros((k, N))
    E[np.arange(k), idx] = 1.0
    L = np.longdouble
    ref = Ainv.astype(L) - W.astype(L) @ (V.astype(L) @ Ainv.astype(L) - E)
    return A, Ainv, V, W, E, ref


def rel(x, ref):
    return float(np.linalg.norm((x - ref).astype(np.float64)) / np.linalg.norm(ref.astype(np.float64)))


def test_exactness_bounds():
    # a slice product is at most 255^2; phase A sums one slice pair over AR
    # rows per accumulator block of the exact diagonals, phase C at most 7
    # pairs over a contraction of CK
    assert AR * 255 ** 2 < 2 ** 24
    assert 7 * CK * 255 ** 2 < 2 ** 24
    assert 8 * (2 ** 53 - 1) < 2 ** 56                     # q of the set's largest element fits


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_slices_reconstruct_to_fp64(seed):
    rng = np.random.default_rng(seed)
    x = rng.standard_normal((40, 40)) * np.exp2(rng.integers(-30, 30, (40, 40)))
    x[0, 0] = 0.0
    ec = bexp(x).max(axis=0)[None, :]
    s = cut(x, ec)
    back = sum(s[j].astype(np.float64) * pow2(ec - 1030 - 8 * j) for j in range(7))
    # each element within half a unit of the 2^-55 grid of its column's largest
    unit = pow2(ec - 1023 - 55)
    assert np.all(np.abs(back - x) <= 0.5 * unit * (1 + 1e-12))
    assert back[0, 0] == 0.0


@pytest.mark.parametrize("N,k,seed", [(96, 12, 0), (200, 16, 3)])
def test_emulated_flush_matches_fp64(N, k, seed):
    A, Ainv, V, W, E, ref = flush_case(N, k, seed)
    fp64 = Ainv - W @ (V @ Ainv - E)
    T = phase_a(V, Ainv) - E
    emulated = Ainv - phase_c(W, T)
    e64, e7 = rel(fp64, ref), rel(emulated, ref)
    assert e7 < 3.0 * e64 + 1e-16, (e7, e64)


def test_six_slices_fall_short():
    # the reason for the seventh slice: with six (the same j + l <= 6 pairs),
    # one flush is 40-50 times less accurate than fp64 arithmetic
    A, Ainv, V, W, E, ref = flush_case(200, 16, 3)
    fp64 = Ainv - W @ (V @ Ainv - E)
    T6 = phase_a(V, Ainv, ns=6) - E
    e6 = rel(Ainv - phase_c(W, T6, ns=6), ref)
    assert e6 > 10.0 * rel(fp64, ref), e6
