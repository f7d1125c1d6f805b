"""Pins for the CPU oracle: each oracle function is checked against something
other than itself -- the Leibniz definition of the determinant, exact rational
arithmetic, closed forms, and the invariants the paper states (Sec. II: the
delayed scheme is equivalent to one-move-at-a-time updating and does not change
the sampling).

A plausible mistake in the oracle (a dropped term, a wrong sign, a transposed
operand, a wrong pivot) changes at least one exact or closed-form value here.
"""
import itertools
import math
from fractions import Fraction

import numpy as np
import pytest

import oracle
from paper_1708_00744_b300 import inputs


# ---------------------------------------------------------------- exact helpers
def leibniz_det(a):
    """Determinant straight from its definition: sum over permutations."""
    n = len(a)
    total = 0
    for perm in itertools.permutations(range(n)):
        inv = sum(1 for i in range(n) for j in range(i + 1, n) if perm[i] > perm[j])
        term = -1 if inv % 2 else 1
        for i in range(n):
            term = term * a[i][perm[i]]
        total += term
    return total


def frac_matrix(a):
    return [[Fraction(int(x)) if float(x).is_integer() else Fraction(x) for x in row] for row in a]


def frac_inverse(a):
    """Exact inverse by Gauss-Jordan over the rationals."""
    n = len(a)
    m = [list(row) + [Fraction(int(i == j)) for j in range(n)] for i, row in enumerate(a)]
    for c in range(n):
        p = next(i for i in range(c, n) if m[i][c] != 0)
        m[c], m[p] = m[p], m[c]
        piv = m[c][c]
        m[c] = [x / piv for x in m[c]]
        for i in range(n):
            if i != c and m[i][c] != 0:
                f = m[i][c]
                m[i] = [x - f * y for x, y in zip(m[i], m[c])]
    return [row[n:] for row in m]


def to_float(m):
    return np.array([[float(x) for x in row] for row in m])


def random_int_matrix(rng, n, lo=-3, hi=4):
    while True:
        a = rng.integers(lo, hi, size=(n, n))
        if leibniz_det(a.tolist()) != 0 if n <= 6 else abs(np.linalg.det(a)) > 0.5:
            return a.astype(np.float64)


def rel(x, ref):
    return abs(x - ref) / max(abs(ref), 1e-300)


# ---------------------------------------------------------------- determinant
@pytest.mark.parametrize("n", [1, 2, 3, 4, 5, 6])
def test_slogdet_matches_leibniz_definition(n):
    rng = np.random.default_rng(100 + n)
    for _ in range(5):
        a = rng.standard_normal((n, n))
        d = leibniz_det(a.tolist())
        sg, la = oracle.slogdet(a)
        assert sg == (1 if d > 0 else -1)
        assert abs(la - math.log(abs(d))) < 1e-12 * max(1.0, abs(la))


def test_slogdet_closed_forms():
    # identity and diagonal: product of the diagonal
    assert oracle.slogdet(np.eye(7)) == (1, 0.0)
    d = np.array([2.0, -0.5, 3.0, -4.0, 0.25])
    sg, la = oracle.slogdet(np.diag(d))
    assert sg == 1 and abs(la - np.sum(np.log(np.abs(d)))) < 1e-14
    # permutation matrices: determinant = parity of the permutation
    rng = np.random.default_rng(3)
    for n in (2, 3, 6, 9):
        perm = rng.permutation(n)
        inv = sum(1 for i in range(n) for j in range(i + 1, n) if perm[i] > perm[j])
        p = np.zeros((n, n))
        p[np.arange(n), perm] = 1.0
        sg, la = oracle.slogdet(p)
        assert sg == (-1 if inv % 2 else 1) and la == 0.0
    # Vandermonde: det = prod_{i<j} (x_j - x_i)
    x = np.array([0.3, -1.2, 2.5, 0.9, -0.4, 1.7])
    v = np.vander(x, increasing=True)
    ref = np.prod([x[j] - x[i] for i in range(6) for j in range(i + 1, 6)])
    sg, la = oracle.slogdet(v)
    assert sg == np.sign(ref) and abs(la - math.log(abs(ref))) < 1e-12
    # Hilbert: det H_n = c_n^4 / c_{2n}, c_n = prod_{i=1}^{n-1} i!
    for n in (3, 5, 7):
        c = lambda m: math.prod(math.factorial(i) for i in range(1, m))
        ref = Fraction(c(n) ** 4, c(2 * n))
        h = np.array([[1.0 / (i + j + 1) for j in range(n)] for i in range(n)])
        sg, la = oracle.slogdet(h)
        assert sg == 1 and abs(la - math.log(ref)) < 1e-8


def test_slogdet_singular_and_empty():
    a = np.array([[1.0, 2.0], [2.0, 4.0]])
    sg, la = oracle.slogdet(a)
    assert sg == 0 and la == -math.inf
    assert oracle.slogdet(np.zeros((0, 0))) == (1, 0.0)


# ---------------------------------------------------------------- inverse
@pytest.mark.parametrize("n", [1, 2, 3, 5, 7])
def test_inverse_matches_exact_rational_inverse(n):
    rng = np.random.default_rng(200 + n)
    a = random_int_matrix(rng, n)
    ref = to_float(frac_inverse(frac_matrix(a)))
    got = oracle.inverse(a)
    assert np.linalg.norm(got - ref) <= 1e-12 * np.linalg.norm(ref)
    # column-major layout: row c is column c of A^{-1}
    assert np.array_equal(oracle.inverse_colmajor(a), got.T)


def test_inverse_hilbert_closed_form():
    n = 5
    h = np.array([[1.0 / (i + j + 1) for j in range(n)] for i in range(n)])
    ref = np.zeros((n, n))
    for i in range(1, n + 1):
        for j in range(1, n + 1):
            ref[i - 1, j - 1] = ((-1) ** (i + j) * (i + j - 1) * math.comb(n + i - 1, n - j)
                                 * math.comb(n + j - 1, n - i) * math.comb(i + j - 2, i - 1) ** 2)
    got = oracle.inverse(h)
    assert np.linalg.norm(got - ref) <= 1e-8 * np.linalg.norm(ref)


def test_inverse_is_not_transposed():
    a = np.array([[2.0, 1.0], [0.0, 1.0]])
    assert np.allclose(oracle.inverse(a), [[0.5, -0.5], [0.0, 1.0]], atol=0, rtol=1e-15)


# ---------------------------------------------------------------- ratios
def exact_ratio(a, j, v):
    a2 = np.array(a, dtype=np.float64)
    a2[j] = v
    return Fraction(leibniz_det(frac_matrix(a2))) / Fraction(leibniz_det(frac_matrix(a)))


@pytest.mark.parametrize("method", [oracle.BRUTE, oracle.SM, oracle.DELAYED])
def test_single_move_ratio_is_exact_determinant_ratio(method):
    rng = np.random.default_rng(7)
    n = 5
    a = random_int_matrix(rng, n)
    elec = np.array([0, 3, 1, 4, 2, 3])
    v = rng.integers(-3, 4, size=(len(elec), n)).astype(np.float64)
    out = oracle.moves(method, a, elec, v, np.zeros(len(elec)), K=3)   # all rejected
    for m, j in enumerate(elec):
        assert rel(out["ratios"][m], float(exact_ratio(a, j, v[m]))) < 1e-12
    assert np.array_equal(out["A"], a)                    # rejects change nothing


@pytest.mark.parametrize("method", [oracle.BRUTE, oracle.SM, oracle.DELAYED])
def test_ratio_closed_forms(method):
    n = 6
    rng = np.random.default_rng(11)
    v = rng.standard_normal((n, n))
    # A = I: r = v_j
    out = oracle.moves(method, np.eye(n), np.arange(n), v, np.zeros(n), K=4)
    assert np.allclose(out["ratios"], v[np.arange(n), np.arange(n)], rtol=1e-14, atol=0)
    # A = diag(d): r = v_j / d_j
    d = np.array([2.0, -0.5, 4.0, 1.5, -3.0, 0.75])
    out = oracle.moves(method, np.diag(d), np.arange(n), v, np.zeros(n), K=4)
    assert np.allclose(out["ratios"], v[np.arange(n), np.arange(n)] / d, rtol=1e-14, atol=0)


# ---------------------------------------------------------------- trajectories
@pytest.mark.parametrize("method,K", [(oracle.BRUTE, 1), (oracle.SM, 1), (oracle.DELAYED, 1),
                                      (oracle.DELAYED, 2), (oracle.DELAYED, 3), (oracle.DELAYED, 8)])
def test_accepted_moves_give_exact_inverse_and_logdet(method, K):
    """After accepted integer moves the matrix is integer: compare the running
    inverse, log|det| and sign with exact rational arithmetic."""
    rng = np.random.default_rng(5)
    n = 6
    a = random_int_matrix(rng, n)
    elec = np.array([2, 0, 5, 1, 2, 4, 3, 0, 5])          # repeats force delayed flushes
    cur = a.copy()
    vs, dec = [], []
    for j in elec:
        while True:
            v = rng.integers(-3, 4, size=n).astype(np.float64)
            trial = cur.copy()
            trial[j] = v
            if leibniz_det(trial.tolist()) != 0:
                break
        vs.append(v)
        acc = rng.random() < 0.7
        dec.append(acc)
        if acc:
            cur = trial
    out = oracle.moves(method, a, elec, np.array(vs), np.array(dec), K=K)
    assert np.array_equal(out["A"], cur)
    exact_inv = to_float(frac_inverse(frac_matrix(cur)))
    assert np.linalg.norm(out["Ainv"] - exact_inv.T) <= 1e-11 * np.linalg.norm(exact_inv)
    det = leibniz_det(frac_matrix(cur))
    assert out["sign"] == (1 if det > 0 else -1)
    assert abs(out["logabs"] - math.log(abs(det))) < 1e-11
    # each ratio equals det(A')/det(A) of the matrix at that point
    cur = a.copy()
    for m, j in enumerate(elec):
        assert rel(out["ratios"][m], float(exact_ratio(cur, j, vs[m]))) < 1e-11
        if dec[m]:
            cur[j] = vs[m]


def _sweep_inputs(seed, n, nsweeps):
    a = inputs.initial_matrix(seed, n)
    g = np.stack([inputs.proposal_gaussians(seed, s, n) for s in range(nsweeps)])
    u = np.stack([inputs.metropolis_uniforms(seed, s, n) for s in range(nsweeps)])
    return a, g, u


@pytest.mark.parametrize("sigma", [0.1, 1.0])
def test_sm_matches_brute_force_sweeps(sigma):
    a, g, u = _sweep_inputs(1, 12, 2)
    b = oracle.sweeps(oracle.BRUTE, a, g, u, sigma)
    s = oracle.sweeps(oracle.SM, a, g, u, sigma)
    assert b["near_ties"] == 0
    assert np.array_equal(b["accepted"], s["accepted"])
    assert np.max(np.abs(b["ratios"] - s["ratios"]) / np.abs(b["ratios"])) < 1e-11
    assert np.array_equal(b["A"], s["A"])
    assert np.linalg.norm(s["Ainv"] - b["Ainv"]) < 1e-11 * np.linalg.norm(b["Ainv"])


@pytest.mark.parametrize("sigma", [0.1, 1.0])
def test_delayed_equivalent_to_one_move_at_a_time(sigma):
    """Sec. II: same uniforms -> same accept sequence for every K."""
    n = 48
    a, g, u = _sweep_inputs(2, n, 3)
    ref = oracle.sweeps(oracle.SM, a, g, u, sigma)
    assert ref["near_ties"] == 0
    for K in (1, 2, 3, 5, 8, 16, 48):
        d = oracle.sweeps(oracle.DELAYED, a, g, u, sigma, K=K)
        assert np.array_equal(d["accepted"], ref["accepted"]), K
        assert np.max(np.abs(d["ratios"] - ref["ratios"]) / np.abs(ref["ratios"])) < 1e-10
        assert np.linalg.norm(d["Ainv"] - ref["Ainv"]) < 1e-10 * np.linalg.norm(ref["Ainv"])
        assert abs(d["logabs"] - ref["logabs"]) < 1e-10 * max(1.0, abs(ref["logabs"]))
        assert d["sign"] == ref["sign"]
        assert np.array_equal(d["A"], ref["A"])


def test_running_logdet_and_inverse_match_direct_calculation():
    """Sec. III checks determinants against direct calculation after a sweep."""
    n = 64
    a, g, u = _sweep_inputs(0, n, 2)
    for method, K in ((oracle.SM, 1), (oracle.DELAYED, 8)):
        out = oracle.sweeps(method, a, g, u, 0.1, K=K)
        sg, la = oracle.slogdet(out["A"])
        assert out["sign"] == sg and abs(out["logabs"] - la) < 1e-10 * max(1.0, abs(la))
        ref = oracle.inverse_colmajor(out["A"])
        assert np.linalg.norm(out["Ainv"] - ref) < 1e-10 * np.linalg.norm(ref)
        # residual: A A^{-1} = I  (Ainv layout is column-major: use its transpose)
        assert np.abs(out["A"] @ out["Ainv"].T - np.eye(n)).max() < 1e-10


def test_override_replays_decisions():
    n = 16
    a, g, u = _sweep_inputs(4, n, 1)
    rej = oracle.sweeps(oracle.DELAYED, a, g, u, 1.0, K=4, override=np.zeros((1, n)))
    assert not rej["accepted"].any() and np.array_equal(rej["A"], a)
    ref_inv = oracle.inverse_colmajor(a)
    assert np.linalg.norm(rej["Ainv"] - ref_inv) < 1e-13 * np.linalg.norm(ref_inv)
    acc = oracle.sweeps(oracle.DELAYED, a, g, u, 1.0, K=4, override=np.ones((1, n)))
    assert acc["accepted"].all()
    sm = oracle.sweeps(oracle.SM, a, g, u, 1.0, override=np.ones((1, n)))
    assert np.linalg.norm(acc["Ainv"] - sm["Ainv"]) < 1e-10 * np.linalg.norm(sm["Ainv"])


def test_metropolis_rule_is_strict_and_squared():
    """accept iff u < min(1, r^2): with A = I, r = v_j exactly."""
    n = 4
    a = np.eye(n)
    g = np.zeros((1, n, n))
    # v_j = 1 + sigma * g_jj ; choose g so that r = 0.5 (r^2 = 0.25)
    for j in range(n):
        g[0, j, j] = -0.5
    u = np.array([[0.2499, 0.25, 0.2501, 0.0]])
    out = oracle.sweeps(oracle.SM, a, g, u, 1.0)
    assert np.allclose(out["ratios"], 0.5)
    assert out["accepted"].tolist() == [[True, False, False, True]]
    assert out["near_ties"] == 1                             # |0.25 - 0.25| < 1e-10


def test_one_electron():
    a = np.array([[2.0]])
    g = np.array([[[1.0]]])
    u = np.array([[0.0]])
    out = oracle.sweeps(oracle.DELAYED, a, g, u, 1.0, K=4)
    assert out["ratios"][0, 0] == 1.5 and out["accepted"][0, 0]
    assert out["Ainv"][0, 0] == pytest.approx(1 / 3, rel=1e-15)
    assert out["logabs"] == pytest.approx(math.log(3.0), rel=1e-15)


def test_golden_fixture_reproduces():
    """tests/golden/sweep_n64_seed0.json was written by tests/golden/make_golden.py
    from this oracle; K=1 and K=8 must give the same accept string (Sec. II)."""
    import json
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", "sweep_n64_seed0.json")
    doc = json.load(open(path))
    k1, k8 = doc["cases"]
    assert k1["accepted"] == k8["accepted"]
    for c in doc["cases"]:
        a, g, u = _sweep_inputs(c["seed"], c["n"], c["nsweeps"])
        out = oracle.sweeps(oracle.SM if c["K"] == 1 else oracle.DELAYED, a, g, u, c["sigma"], K=c["K"])
        assert ["".join("1" if x else "0" for x in row) for row in out["accepted"]] == c["accepted"]
        assert np.max(np.abs(out["ratios"] - np.array(c["ratios"]))) == 0.0
        assert out["logabs"] == c["final_logabs"]


@pytest.mark.parametrize("method,K", [(oracle.SM, 1), (oracle.DELAYED, 16)])
def test_results_do_not_depend_on_thread_count(method, K):
    """The parallel loops write disjoint elements, each in the one-thread
    order: every output is bit-identical for 1 and several threads."""
    n, ns = 300, 2
    A, G, U = _sweep_inputs(77, n, ns)
    prev = oracle.set_threads(1)
    try:
        one = oracle.sweeps(method, A, G, U, 0.3, K=K)
        oracle.set_threads(4)
        many = oracle.sweeps(method, A, G, U, 0.3, K=K)
        inv1 = oracle.inverse(A)
        oracle.set_threads(1)
        inv0 = oracle.inverse(A)
    finally:
        oracle.set_threads(prev)
    for key in ("ratios", "accepted", "A", "Ainv"):
        assert np.array_equal(one[key], many[key]), key
    assert one["logabs"] == many["logabs"] and one["sign"] == many["sign"]
    assert np.array_equal(inv0, inv1)


@pytest.mark.parametrize("sigma", [0.3, 1.5])
def test_fixed_slot_reading_equivalent_to_one_move_at_a_time(sigma):
    """Sec. II's fixed slots (a rejected proposal takes a queue slot as an
    unchanged column): the same trajectory as Sherman-Morrison for every K,
    with many rejections (sigma 1.5) and with few."""
    n = 40
    a, g, u = _sweep_inputs(12, n, 3)
    ref = oracle.sweeps(oracle.SM, a, g, u, sigma)
    assert ref["near_ties"] == 0
    assert 0.2 < ref["accepted"].mean() < 0.98
    for K in (1, 2, 3, 7, 16, 40):
        d = oracle.sweeps(oracle.DELAYED_SLOT, a, g, u, sigma, K=K)
        assert np.array_equal(d["accepted"], ref["accepted"]), K
        assert np.max(np.abs(d["ratios"] - ref["ratios"]) / np.maximum(1.0, np.abs(ref["ratios"]))) < 1e-10
        assert np.linalg.norm(d["Ainv"] - ref["Ainv"]) < 1e-10 * np.linalg.norm(ref["Ainv"])
        assert abs(d["logabs"] - ref["logabs"]) < 1e-10 * max(1.0, abs(ref["logabs"]))
        assert d["sign"] == ref["sign"] and np.array_equal(d["A"], ref["A"])


def test_fixed_slot_rejections_change_nothing():
    """Every proposal rejected: the queue fills with zero changes, the flushes
    subtract exact zeros, and the inverse, A and log|det| stay bit for bit."""
    n, K = 30, 4
    a, g, u = _sweep_inputs(5, n, 2)
    ov = np.zeros((2, n), dtype=np.int8)
    d = oracle.sweeps(oracle.DELAYED_SLOT, a, g, u, 0.2, K=K, override=ov)
    s, l = oracle.slogdet(a)
    assert not d["accepted"].any()
    assert np.array_equal(d["A"], a)
    # the walker's inverse is the LU inverse of the paper's matrix M = A'
    # (one column per electron), exported as it is
    assert np.array_equal(d["Ainv"], oracle.inverse(np.ascontiguousarray(a.T)))
    assert d["logabs"] == l and d["sign"] == s


@pytest.mark.parametrize("method", [oracle.BRUTE, oracle.SM, oracle.DELAYED])
def test_ratio_terms_closed_form_and_bound(method):
    """terms = 1 + sum_i |(A^{-1})_ij u_i|: for A = I it is 1 + |u_j| (the
    only nonzero term of Eq. 1), and it bounds |r| (triangle inequality)."""
    n = 9
    rng = np.random.default_rng(4)
    v = rng.standard_normal((n, n))
    out = oracle.moves(method, np.eye(n), np.arange(n), v, np.zeros(n, np.uint8), K=4)
    u = v[np.arange(n), np.arange(n)] - 1.0
    assert np.allclose(out["terms"], 1.0 + np.abs(u), rtol=1e-15, atol=0)
    a, g, uu = _sweep_inputs(8, 24, 1)
    s = oracle.sweeps(method, a, g, uu, 0.5, K=4)
    assert np.all(s["terms"] >= np.abs(s["ratios"]) * (1 - 1e-14))


# ---------------------------------------------------------------- multideterminant walkers
def _md_exact_psi(A, B, exc, coef):
    """Psi = sum_I c_I det(A_I) in exact rational arithmetic (Leibniz)."""
    tot = Fraction(0)
    for (o1, a1, o2, a2), c in zip(exc, coef):
        M = [[Fraction(int(x)) for x in row] for row in A]
        for o, a in ((o1, a1), (o2, a2)):
            if o >= 0:
                for e in range(len(M)):
                    M[e][o] = Fraction(int(B[e][a]))
        tot += Fraction(c) * leibniz_det(M)
    return tot


def _md_case(seed, n=4, nv=3):
    rng = np.random.default_rng(seed)
    A = random_int_matrix(rng, n)
    B = rng.integers(-3, 4, size=(n, nv)).astype(np.float64)
    exc = [(-1, -1, -1, -1), (0, 1, -1, -1), (2, 0, -1, -1), (1, 2, 3, 0), (0, 0, 2, 1)]
    coef = [1.0, 0.5, -0.25, 0.125, 0.75]
    G = rng.integers(-2, 3, size=(1, n, n)).astype(np.float64)
    H = rng.integers(-2, 3, size=(1, n, nv)).astype(np.float64)
    return A, B, exc, coef, G, H


@pytest.mark.parametrize("method,K", [(oracle.MD_BRUTE, 1), (oracle.MD_TABLE, 1), (oracle.MD_TABLE_DELAYED, 2),
                                      (oracle.MD_TABLE_DELAYED, 4)])
def test_multideterminant_ratios_match_exact_rational(method, K):
    """Integer orbitals and integer moves (sigma = 1): every ratio of
    Psi = sum_I c_I det(A_I) against exact Leibniz determinants over the
    rationals, along the walk of given decisions (the delayed reading with
    queued moves, so that the Woodbury column of the current inverse is
    used)."""
    for seed in (1, 2, 3):
        A, B, exc, coef, G, H = _md_case(seed)
        n = A.shape[0]
        dec = np.array([1, 0, 1, 1], dtype=np.int8)[None]
        # a move onto a singular reference determinant is not taken (the table
        # is relative to it); its ratio is still checked
        cA = A.copy()
        for j in range(n):
            nA = cA.copy()
            nA[j] += G[0, j]
            if leibniz_det(nA.astype(int).tolist()) == 0:
                dec[0, j] = 0
            if dec[0, j]:
                cA = nA
        U = np.full((1, n), 0.5)
        out = oracle.md_sweeps(method, A, B, G, H, U, 1.0, exc, coef, override=dec, K=K)
        cur_A, cur_B = A.copy(), B.copy()
        psi = _md_exact_psi(cur_A, cur_B, exc, coef)
        for j in range(n):
            nA, nB = cur_A.copy(), cur_B.copy()
            nA[j] += G[0, j]
            nB[j] += H[0, j]
            npsi = _md_exact_psi(nA, nB, exc, coef)
            exact = float(npsi / psi) if psi != 0 else 0.0
            assert abs(out["ratios"][0, j] - exact) <= 1e-11 * max(1.0, abs(exact)), (seed, j)
            if dec[0, j]:
                cur_A, cur_B, psi = nA, nB, npsi
        assert np.array_equal(out["A"], cur_A) and np.array_equal(out["B"], cur_B)


def test_multideterminant_readings_agree_and_reduce_to_one_determinant():
    """The table method (Sherman-Morrison on A^{-1} and the table) follows the
    definition's trajectory, and an expansion of the reference alone is the
    one-determinant walk."""
    n, nv, ns = 24, 6, 2
    rng = np.random.default_rng(9)
    a, g, u = _sweep_inputs(31, n, ns)
    B = rng.standard_normal((n, nv))
    H = rng.standard_normal((ns, n, nv))
    exc = [(-1, -1, -1, -1)] + [(int(o), int(v), -1, -1) for o, v in zip(rng.integers(0, n, 6),
                                                                          rng.integers(0, nv, 6))]
    exc += [(0, 1, 5, 2), (3, 4, 7, 0)]
    coef = rng.standard_normal(len(exc)) * 0.3
    coef[0] = 1.0
    brute = oracle.md_sweeps(oracle.MD_BRUTE, a, B, g, H, u, 0.3, exc, coef)
    table = oracle.md_sweeps(oracle.MD_TABLE, a, B, g, H, u, 0.3, exc, coef)
    assert 0.2 < brute["accepted"].mean() < 0.99
    assert np.array_equal(brute["accepted"], table["accepted"])
    assert np.max(np.abs(brute["ratios"] - table["ratios"]) / np.maximum(1, np.abs(brute["ratios"]))) < 1e-10
    assert abs(brute["logabs"] - table["logabs"]) < 1e-10 * max(1, abs(brute["logabs"]))
    assert brute["sign"] == table["sign"]
    for K in (1, 5, n):
        dl = oracle.md_sweeps(oracle.MD_TABLE_DELAYED, a, B, g, H, u, 0.3, exc, coef,
                              override=brute["accepted"].astype(np.int8), K=K)
        assert np.max(np.abs(brute["ratios"] - dl["ratios"]) / np.maximum(1, np.abs(brute["ratios"]))) < 1e-10, K
        assert abs(brute["logabs"] - dl["logabs"]) < 1e-10 * max(1, abs(brute["logabs"]))
    one = oracle.md_sweeps(oracle.MD_TABLE, a, B, g, H, u, 0.3, exc[:1], [1.0])
    sm = oracle.sweeps(oracle.SM, a, g, u, 0.3)
    assert np.array_equal(one["accepted"], sm["accepted"])
    assert np.max(np.abs(one["ratios"] - sm["ratios"]) / np.maximum(1, np.abs(sm["ratios"]))) < 1e-12
