"""The recompute panels' pivot search compares integer keys instead of fp64
values: the key of x is the bit pattern of |x| as a signed 64-bit integer, and
-2 for NaN (below the empty key -1). The search takes the largest key, the
lowest row on ties; it must pick the row that partial pivoting by |x| picks with
fp64 comparisons, where a NaN candidate never wins (a comparison with NaN is
false). Checked here on the CPU over the values that could break the
correspondence: zeros of both signs, subnormals, the largest finite values,
infinities, NaNs of both signs and payloads, and ties."""
import numpy as np
import pytest


def key(x):
    b = np.asarray(x, dtype=np.float64).view(np.int64) & np.int64(0x7FFFFFFFFFFFFFFF)
    return np.where(b > np.int64(0x7FF0000000000000), np.int64(-2), b)


def pick_by_keys(col):
    best, bi = -1, len(col)
    for i, k in enumerate(key(col)):
        if k > best or (k == best and i < bi):
            best, bi = int(k), i
    return bi


def pick_by_fp64(col):
    best, bi = -1.0, len(col)
    for i, v in enumerate(np.abs(col)):
        if v > best or (v == best and i < bi):
            best, bi = v, i
    return bi


SPECIAL = np.array([0.0, -0.0, 5e-324, -5e-324, 2.2250738585072014e-308, 1e-300, 1.0, -1.0,
                    1.7976931348623157e308, -1.7976931348623157e308, np.inf, -np.inf, np.nan,
                    -np.nan, np.float64(np.frombuffer(np.int64(0x7FF0000000000001).tobytes(), np.float64)[0])])


def test_key_order_is_value_order_on_non_negative_doubles():
    rng = np.random.default_rng(5)
    bits = rng.integers(0, 0x7FF0000000000000, size=20000, dtype=np.int64)
    vals = np.sort(bits.view(np.float64))
    assert np.all(np.diff(key(vals)) >= 0)
    assert np.all((np.diff(key(vals)) == 0) == (np.diff(vals) == 0))


def test_nan_never_wins_and_the_empty_search_stays_empty():
    assert key(np.nan) < -1 and key(-np.nan) < -1
    assert pick_by_keys(np.array([np.nan, np.nan])) == 2 == pick_by_fp64(np.array([np.nan, np.nan]))


@pytest.mark.parametrize("seed", range(40))
def test_pivot_rows_agree_with_fp64_partial_pivoting(seed):
    rng = np.random.default_rng(seed)
    n = int(rng.integers(1, 40))
    col = rng.standard_normal(n) * 10.0 ** rng.integers(-300, 300, size=n)
    # sprinkle special values and exact ties
    for _ in range(int(rng.integers(0, 6))):
        col[rng.integers(0, n)] = SPECIAL[rng.integers(0, len(SPECIAL))]
    if n > 2 and rng.random() < 0.5:
        col[rng.integers(0, n)] = -col[rng.integers(0, n)]
    assert pick_by_keys(col) == pick_by_fp64(col)
