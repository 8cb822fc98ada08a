"""Pins of the oracle against facts fixed by the paper and by mathematics.

Nothing here compares the oracle with itself: every expectation comes from a
hand-worked example, a brute-force enumeration of warping paths, a closed
form, a library routine (numpy), or an inequality that holds for any
monotone warping path.
"""
import itertools
import math

import numpy as np
import pytest

import oracle
from tests.conftest import read_golden


# ------------------------------------------------------------ brute force --
def brute_force(x, y):
    """Every warping path of sDTW (Section 2.3): it starts at any cell of the
    first query row, moves by (1,0), (0,1) or (1,1), and ends in the last
    query row; its cost is the sum of |x_i - y_j| over its cells. Returns the
    smallest cost and the first end column reaching it."""
    M, N = len(x), len(y)
    best = {}

    def walk(i, j, acc):
        acc = acc + abs(x[i] - y[j])
        if i == M - 1:
            if j not in best or acc < best[j]:
                best[j] = acc
        if i + 1 < M:
            walk(i + 1, j, acc)
        if j + 1 < N:
            walk(i, j + 1, acc)
        if i + 1 < M and j + 1 < N:
            walk(i + 1, j + 1, acc)

    for s in range(N):
        walk(0, s, 0)
    cost = min(best.values())
    col = min(j for j, v in best.items() if v == cost)
    return cost, col


def small_cases():
    rng = np.random.default_rng(7)
    for M in range(1, 6):
        for N in range(M, 7):
            for _ in range(3):
                yield rng.integers(0, 4, M).astype(np.float64), rng.integers(0, 4, N).astype(np.float64)


@pytest.mark.parametrize("case", list(range(60)))
def test_brute_force_all_forms(case):
    x, y = list(small_cases())[case]
    c, j = brute_force(list(x), list(y))
    assert oracle.sdtw_full_f64(x, y) == (c, j)
    rc, rj, _ = oracle.sdtw_roll_f64(x, y)
    assert (rc, rj) == (c, j)
    assert oracle.sdtw_roll_f32(x.astype(np.float32), y.astype(np.float32)) == (c, j)
    xi, yi = x.astype(np.int16), y.astype(np.int16)
    assert oracle.sdtw_full_i16(xi, yi) == (c, j)
    assert oracle.sdtw_roll_i16(xi, yi) == (c, j)
    assert oracle.sdtw_roll_i32(xi, yi) == (c, j)


def test_brute_force_continuous_values():
    rng = np.random.default_rng(11)
    for _ in range(25):
        M = int(rng.integers(1, 6))
        N = int(rng.integers(M, 7))
        x, y = rng.normal(size=M), rng.normal(size=N)
        c, j = brute_force(list(x), list(y))
        oc, oj = oracle.sdtw_full_f64(x, y)
        assert oj == j
        assert math.isclose(oc, c, rel_tol=1e-12, abs_tol=1e-12)


# ----------------------------------------------------------- hand examples --
@pytest.mark.parametrize("row", read_golden("sdtw_hand.txt"))
def test_hand_worked_examples(row):
    name, xs, ys, cost, col, last = row
    x = np.array([float(v) for v in xs.split()])
    y = np.array([float(v) for v in ys.split()])
    assert oracle.sdtw_full_f64(x, y) == (float(cost), int(col)), name
    assert oracle.sdtw_roll_f64(x, y)[:2] == (float(cost), int(col)), name
    np.testing.assert_array_equal(oracle.sdtw_lastrow_f64(x, y), [float(v) for v in last.split()])


@pytest.mark.parametrize("row", read_golden("kmer_hand.txt"))
def test_kmer_reference_hand(row):
    g, k, levels = row
    bases = np.array(["ACGT".index(c) for c in g], dtype=np.uint8)
    k = int(k)
    model = np.arange(4 ** k, dtype=np.float32)
    np.testing.assert_array_equal(oracle.ref_levels(bases, model, k), [float(v) for v in levels.split()])


def test_kmer_reference_palindrome_and_sizes():
    # The reverse complement of a reverse-complement palindrome is itself, so
    # both strands give the same levels (Section 4.1 footnote: both strands).
    bases = np.array(["ACGT".index(c) for c in "GAATTC"], dtype=np.uint8)
    model = np.random.default_rng(0).normal(90, 12, 4 ** 3).astype(np.float32)
    lv = oracle.ref_levels(bases, model, 3)
    np.testing.assert_array_equal(lv[:4], lv[4:])
    # n bases give n - k + 1 levels per strand (29,903 bases -> 59,796 values)
    g = np.random.default_rng(1).integers(0, 4, 29903).astype(np.uint8)
    assert oracle.ref_levels(g, np.zeros(4 ** 6, np.float32), 6).shape[0] == 59796


# -------------------------------------------------------- planted copies --
def test_exact_copy_has_zero_cost_at_planted_end():
    rng = np.random.default_rng(3)
    y = rng.normal(size=400)
    for j0, M in [(0, 1), (17, 25), (100, 60), (400 - 30, 30)]:
        x = y[j0:j0 + M].copy()
        c, j, _ = oracle.sdtw_roll_f64(x, y)
        assert c == 0.0 and j == j0 + M - 1
        ci, ji = oracle.sdtw_roll_i16(np.round(x * 64).astype(np.int16), np.round(y * 64).astype(np.int16))
        assert ci == 0 and ji == j0 + M - 1


def test_dwelled_copy_has_zero_cost():
    # Repeating a sample is a vertical step with delta = 0 (Eq. 1), so a query
    # whose samples each repeat 1..3 times still costs 0 at the same column.
    rng = np.random.default_rng(4)
    y = rng.normal(size=300)
    seg = y[50:90]
    rep = rng.integers(1, 4, size=seg.shape[0])
    x = np.repeat(seg, rep)
    c, j, _ = oracle.sdtw_roll_f64(x, y)
    assert c == 0.0 and j == 89


# ---------------------------------------------------------- special cases --
def test_single_row_is_nearest_sample():
    rng = np.random.default_rng(5)
    for _ in range(20):
        y = rng.integers(-5, 6, size=50).astype(np.float64)
        x = np.array([float(rng.integers(-5, 6))])
        d = np.abs(y - x[0])
        c, j, _ = oracle.sdtw_roll_f64(x, y)
        assert c == d.min() and j == int(np.argmin(d))  # argmin: first occurrence


def test_query_equal_to_reference_length():
    rng = np.random.default_rng(6)
    y = rng.normal(size=40)
    x = y[::-1].copy()
    # M = N: every path spans all rows; the cost is bounded by the diagonal.
    c, j, _ = oracle.sdtw_roll_f64(x, y)
    assert c <= np.abs(x - y).sum() + 1e-12


def test_path_bounds():
    """Upper bound: the best diagonal (identity) path. Lower bound: every
    query row costs at least its nearest reference sample."""
    rng = np.random.default_rng(8)
    for _ in range(10):
        M, N = int(rng.integers(2, 40)), int(rng.integers(40, 300))
        x, y = rng.normal(size=M), rng.normal(size=N)
        c, _, _ = oracle.sdtw_roll_f64(x, y)
        diag = min(np.abs(x - y[s:s + M]).sum() for s in range(N - M + 1))
        rowmin = np.abs(x[:, None] - y[None, :]).min(axis=1).sum()
        assert rowmin - 1e-9 <= c <= diag + 1e-9


def test_last_row_and_runner_up():
    rng = np.random.default_rng(9)
    x, y = rng.normal(size=12), rng.normal(size=200)
    last = oracle.sdtw_lastrow_f64(x, y)
    c, j, r = oracle.sdtw_roll_f64(x, y)
    assert c == last.min() and j == int(np.argmin(last))
    assert r == np.delete(last, j).min()


# --------------------------------------------- Algorithm 1 == Algorithm 2 --
def test_full_matrix_equals_rolling_array():
    rng = np.random.default_rng(10)
    for _ in range(10):
        M, N = int(rng.integers(1, 60)), int(rng.integers(60, 400))
        x, y = rng.normal(size=M), rng.normal(size=N)
        assert oracle.sdtw_full_f64(x, y) == oracle.sdtw_roll_f64(x, y)[:2]
        xi = rng.integers(-2047, 2048, size=M).astype(np.int16)
        yi = rng.integers(-2047, 2048, size=N).astype(np.int16)
        assert oracle.sdtw_full_i16(xi, yi) == oracle.sdtw_roll_i16(xi, yi)


# ------------------------------------------- the PE chain's oblique order --
@pytest.mark.parametrize("case", list(range(60)))
def test_wavefront_order_matches_brute_force(case):
    """Section 4.3's processing-element chain evaluates Eq. 1 along oblique
    columns (PE i computes column t - i at step t, all PEs at once): the same
    cost and first end column as the enumeration of every warping path, in
    N + M - 1 steps."""
    x, y = list(small_cases())[case]
    c, j = brute_force(list(x), list(y))
    wc, wj, steps = oracle.sdtw_wavefront_f64(x, y)
    assert (wc, wj) == (c, j)
    assert steps == len(x) + len(y) - 1


def test_wavefront_order_equals_rolling_array():
    """The oblique order and Algorithm 2's column-by-column rolling array give
    the same bits (every cell is the same |x - y| + min of the same three
    values), on continuous values and on small integers full of ties."""
    rng = np.random.default_rng(13)
    for _ in range(20):
        M, N = int(rng.integers(1, 60)), int(rng.integers(60, 300))
        x, y = rng.normal(size=M), rng.normal(size=N)
        wc, wj, steps = oracle.sdtw_wavefront_f64(x, y)
        assert (wc, wj) == oracle.sdtw_roll_f64(x, y)[:2]
        assert steps == M + N - 1
        xi, yi = rng.integers(0, 3, M).astype(np.float64), rng.integers(0, 3, N).astype(np.float64)
        assert oracle.sdtw_wavefront_f64(xi, yi)[:2] == oracle.sdtw_roll_f64(xi, yi)[:2]


# ------------------------------------------------ int16 saturation identity --
def test_int16_is_capped_exact_integer_dp():
    """Saturating at CAP in every cell equals saturating the exact integer
    result once: min(CAP, d + min(a, b, c)) with a, b, c already capped is
    min(CAP, d + min(exact)). Checked against the FP64 form run on the same
    integers (exact in double), including inputs that do hit the cap."""
    rng = np.random.default_rng(12)
    cap = oracle.cap()
    assert cap == 32767 - 2 * oracle.qmax()
    hit = 0
    for trial in range(30):
        M, N = int(rng.integers(1, 40)), int(rng.integers(40, 200))
        hi = 2047 if trial % 2 else 300
        xi = rng.integers(-hi, hi + 1, size=M).astype(np.int16)
        yi = rng.integers(-hi, hi + 1, size=N).astype(np.int16)
        if trial % 3 == 0:
            xi[:] = 2047
            yi[:] = -2047
        last = oracle.sdtw_lastrow_f64(xi.astype(np.float64), yi.astype(np.float64))
        capped = np.minimum(last, cap)
        c, j = oracle.sdtw_roll_i16(xi, yi)
        assert c == capped.min() and j == int(np.argmin(capped))
        hit += int(c == cap)
    assert hit > 0


def test_wide_accumulation_is_unsaturated():
    """int16 inputs with 32-bit accumulation (Section 4.3's PE) equal the
    brute-force minimum over every warping path even where that minimum is
    above CAP (8 cells of |2047 - (-2047)| = 32,752 > 28,673), where the
    saturating form reports CAP; and in general min(CAP, wide) = saturating."""
    x = np.full(8, 2047, dtype=np.int16)
    y = np.array([-2047] * 8, dtype=np.int16)
    c, j = brute_force(list(x.astype(np.int64)), list(y.astype(np.int64)))
    assert c == 8 * 4094 > oracle.cap()
    assert oracle.sdtw_roll_i32(x, y) == (c, j)
    assert oracle.sdtw_roll_i16(x, y) == (oracle.cap(), 0)
    rng = np.random.default_rng(16)
    for _ in range(6):
        M, N = int(rng.integers(1, 8)), int(rng.integers(8, 9))
        xi = rng.choice([-2047, 2047, 0, 1000], M).astype(np.int16)
        yi = rng.choice([-2047, 2047, 5, -999], N).astype(np.int16)
        assert oracle.sdtw_roll_i32(xi, yi) == brute_force(list(xi.astype(np.int64)), list(yi.astype(np.int64)))
    for _ in range(10):
        M, N = int(rng.integers(1, 60)), int(rng.integers(60, 300))
        xi = rng.integers(-2047, 2048, size=M).astype(np.int16)
        yi = rng.integers(-2047, 2048, size=N).astype(np.int16)
        c32, j32 = oracle.sdtw_roll_i32(xi, yi)
        c16, j16 = oracle.sdtw_roll_i16(xi, yi)
        assert c16 == min(c32, oracle.cap())
        if c32 < oracle.cap():
            assert j16 == j32


# ------------------------------------------------------- start column --
def traceback_start(x, y):
    """Independent pin for the start column: the whole cost matrix in float64
    (numpy, Eq. 1), then a traceback from the first minimum of the last row
    that steps to the up neighbour if it is a minimum predecessor, else the
    diagonal one, else the left one; the path starts where it enters row 1."""
    M, N = len(x), len(y)
    g = np.full((M + 1, N + 1), np.inf)
    g[0, :] = 0.0
    for i in range(1, M + 1):
        for j in range(1, N + 1):
            g[i, j] = abs(x[i - 1] - y[j - 1]) + min(g[i - 1, j], g[i - 1, j - 1], g[i, j - 1])
    j = int(np.argmin(g[M, 1:])) + 1
    cost, end = g[M, j], j - 1
    i = M
    while i > 1:
        up, dg, lf = g[i - 1, j], g[i - 1, j - 1], g[i, j - 1]
        m = min(up, dg, lf)
        if up == m:
            i -= 1
        elif dg == m:
            i, j = i - 1, j - 1
        else:
            j -= 1
    return cost, end, j - 1


def test_start_column_matches_traceback():
    rng = np.random.default_rng(17)
    cases = [(rng.integers(0, 4, int(rng.integers(1, 7))), rng.integers(0, 4, 7)) for _ in range(40)]
    cases += [(rng.integers(-2047, 2048, int(rng.integers(1, 30))), rng.integers(-2047, 2048, 80)) for _ in range(20)]
    for x, y in cases:
        if len(x) > len(y):
            continue
        c, e, st = traceback_start(list(x.astype(np.float64)), list(y.astype(np.float64)))
        assert oracle.sdtw_span_i32(x.astype(np.int16), y.astype(np.int16)) == (c, e, st)
        assert oracle.sdtw_span_f32(x.astype(np.float32), y.astype(np.float32)) == (c, e, st)
        # cost and end column are the plain DP's; the start lies on an optimal path (brute force, small cases)
        assert oracle.sdtw_roll_i32(x.astype(np.int16), y.astype(np.int16)) == (c, e)
        if len(y) <= 7:
            bc, bj = brute_force(list(x.astype(np.float64)), list(y.astype(np.float64)))
            assert (bc, bj) == (c, e) and 0 <= st <= e


def test_start_column_of_planted_copies():
    rng = np.random.default_rng(18)
    y = rng.normal(size=3000).astype(np.float32)
    for s0, m, rep in ((0, 50, 1), (1234, 80, 1), (2900, 100, 1), (700, 60, 3)):
        x = np.repeat(y[s0:s0 + m], rep)  # a dwelled copy: vertical steps cost 0
        c, e, st = oracle.sdtw_span_f32(x, y)
        assert (c, e, st) == (0.0, s0 + m - 1, s0)


def test_int16_error_bound_vs_fp64():
    """Each quantised sample is within 0.5/s of its value, so every cell's
    distance moves by at most 1/s; any warping path has at most M + N - 1
    cells, which bounds |cost_q / s - cost|."""
    rng = np.random.default_rng(13)
    for k in (2, 5, 6):
        s = 2.0 ** k
        for _ in range(8):
            M, N = int(rng.integers(5, 50)), int(rng.integers(50, 300))
            x = rng.normal(size=M).astype(np.float32)
            y = rng.normal(size=N).astype(np.float32)
            c64, _, _ = oracle.sdtw_roll_f64(x.astype(np.float64), y.astype(np.float64))
            ci, _ = oracle.sdtw_roll_i16(oracle.quantise(x, k), oracle.quantise(y, k))
            assert abs(ci / s - c64) <= (M + N - 1) / s + 1e-9


# ------------------------------------------------------------ z-score, Q --
def test_zscore_matches_numpy_population_std():
    rng = np.random.default_rng(14)
    for n in (2, 250, 4096, 4097, 100_000):
        x = rng.normal(90, 12, size=n).astype(np.float32)
        z = oracle.zscore(x)
        xd = x.astype(np.float64)
        ref = (xd - xd.mean()) / xd.std()  # numpy: population std (ddof=0)
        np.testing.assert_allclose(z, ref.astype(np.float32), rtol=2e-6, atol=2e-6)
        assert abs(z.astype(np.float64).mean()) < 1e-6
        assert abs(z.astype(np.float64).std() - 1.0) < 1e-6


def test_zscore_closed_form_and_errors():
    z = oracle.zscore(np.array([1, 2, 3, 4], dtype=np.float32))
    s = math.sqrt(1.25)
    np.testing.assert_array_equal(z, np.array([-1.5 / s, -0.5 / s, 0.5 / s, 1.5 / s], dtype=np.float32))
    with pytest.raises(ValueError):
        oracle.zscore(np.full(10, 3.0, dtype=np.float32))


def test_quantiser_rounding_and_clamp():
    # round half to even of z * 2^k, clamp to +-2047
    z = np.array([0.5, 1.5, 2.5, -2.5, -0.5, 79.008, 0.0], dtype=np.float32) / 64.0
    np.testing.assert_array_equal(oracle.quantise(z, 6), [0, 2, 2, -2, 0, 79, 0])
    big = np.array([100.0, -100.0, 31.99, 31.98, -31.99], dtype=np.float32)  # z units: 2047.36, 2046.72
    np.testing.assert_array_equal(oracle.quantise(big, 6), [2047, -2047, 2047, 2047, -2047])
    np.testing.assert_array_equal(oracle.quantise(np.array([0.75, -0.25], np.float32), 1), [2, 0])


# -------------------------------------------------------------- the batch --
def test_batch_composes_the_steps():
    rng = np.random.default_rng(15)
    ref = rng.normal(90, 12, 2000).astype(np.float32)
    lens = rng.integers(5, 60, size=9)
    off = np.concatenate([[0], np.cumsum(lens)]).astype(np.uint32)
    ev = rng.normal(90, 12, off[-1]).astype(np.float32)
    rz = oracle.zscore(ref)
    b16 = oracle.batch(oracle.PREC_I16, ref, ev, off, scale_log2=5, threads=3)
    b32 = oracle.batch(oracle.PREC_F32, ref, ev, off, threads=1)
    b64 = oracle.batch(oracle.PREC_F64, ref, ev, off, threads=2)
    bw = oracle.batch(oracle.PREC_I32, ref, ev, off, scale_log2=5, threads=2)
    bws = oracle.batch(oracle.PREC_I32, ref, ev, off, scale_log2=5, threads=2, start=True)
    b32s = oracle.batch(oracle.PREC_F32, ref, ev, off, threads=2, start=True)
    for q in range(9):
        qz = oracle.zscore(ev[off[q]:off[q + 1]])
        ci, ji = oracle.sdtw_roll_i16(oracle.quantise(qz, 5), oracle.quantise(rz, 5))
        assert (b16.icost[q], b16.col[q]) == (ci, ji) and b16.cost[q] == ci / 32.0
        cw, jw = oracle.sdtw_roll_i32(oracle.quantise(qz, 5), oracle.quantise(rz, 5))
        assert (bw.icost[q], bw.col[q]) == (cw, jw) and bw.cost[q] == cw / 32.0
        assert (bws.icost[q], bws.col[q], bws.start[q]) == oracle.sdtw_span_i32(oracle.quantise(qz, 5),
                                                                               oracle.quantise(rz, 5))
        assert (b32s.cost[q], b32s.col[q], b32s.start[q]) == oracle.sdtw_span_f32(qz, rz)
        assert (b32.cost[q], b32.col[q]) == oracle.sdtw_roll_f32(qz, rz)
        assert (b64.cost[q], b64.col[q]) == oracle.sdtw_roll_f64(qz.astype(np.float64), rz.astype(np.float64))[:2]
    with pytest.raises(ValueError):
        oracle.batch(oracle.PREC_F32, ref[:10], ev, off)  # M > N


# ------------------------------------------------- FP32 rounding of Eq. 1 --
def full_matrix_float32(x, y, acc=np.float32, cell=None):
    """Eq. 1 as a full (M + 1) x (N + 1) matrix with every operation rounded
    in `acc` (numpy scalar arithmetic): delta = |x_i - y_j|, then
    delta + min(up, diagonal, left). With acc = float32 this is the FP32 form
    written out independently of the oracle. Two plausible slips for the
    sensitivity check: acc = float64 accumulates in double and rounds once at
    the end; cell = float32 with acc = float64 rounds each cell once to float32
    after forming |x - y| + min in double (no float32 rounding of delta)."""
    M, N = len(x), len(y)
    inf = acc(np.inf)
    g = [[acc(0.0)] * (N + 1)] + [[inf] + [acc(0.0)] * N for _ in range(M)]
    for i in range(1, M + 1):
        xi = acc(x[i - 1])
        up_row, row = g[i - 1], g[i]
        for j in range(1, N + 1):
            d = abs(xi - acc(y[j - 1]))
            m = min(up_row[j], up_row[j - 1], row[j - 1])
            row[j] = acc(d + m) if cell is None else acc(cell(d + acc(m)))
    last = g[M][1:]
    j = min(range(N), key=lambda k: (last[k], k))  # first column of the minimum
    return g, np.float32(last[j]), j


def float32_traceback_start(g, x, y, end):
    """Start column by a traceback through the FP32 matrix from `end`: step to
    the up neighbour if it is a minimum predecessor, else the diagonal one,
    else the left one; the path starts where it enters row 1."""
    i, j = len(x), end + 1
    while i > 1:
        up, dg, lf = g[i - 1][j], g[i - 1][j - 1], g[i][j - 1]
        m = min(up, dg, lf)
        if up == m:
            i -= 1
        elif dg == m:
            i, j = i - 1, j - 1
        else:
            j -= 1
    return j - 1


def fp32_cases():
    rng = np.random.default_rng(19)
    for _ in range(40):
        M, N = int(rng.integers(1, 41)), int(rng.integers(41, 301))
        yield rng.normal(size=M).astype(np.float32), rng.normal(size=N).astype(np.float32)
    # a planted copy with noise: costs small against their summands
    y = rng.normal(size=300).astype(np.float32)
    yield (y[100:140] + rng.normal(0.0, 0.05, 40)).astype(np.float32), y


def test_fp32_rounding_matches_float32_restatement():
    """The FP32 oracle (Algorithm 2 and the start-column carry) rounds every
    cell exactly as an independent float32 full-matrix Eq. 1 does, on
    continuous inputs where float32 and double sums differ. The same
    restatement accumulated in double disagrees with it on these inputs, so a
    double-accumulating oracle, or one that rounds each cell once from a
    double |x - y| + min, would fail this pin."""
    slips = [0, 0]
    for x, y in fp32_cases():
        g, c, j = full_matrix_float32(x, y)
        oc, oj = oracle.sdtw_roll_f32(x, y)
        assert np.float32(oc) == c and oj == j
        st = float32_traceback_start(g, x, y, j)
        assert oracle.sdtw_span_f32(x, y) == (float(c), j, st)
        for k, (acc, cell) in enumerate(((np.float64, None), (np.float64, np.float32))):
            _, cs, js = full_matrix_float32(x, y, acc=acc, cell=cell)
            slips[k] += int(np.float32(cs) != c or js != j)
    assert min(slips) >= 3, slips
