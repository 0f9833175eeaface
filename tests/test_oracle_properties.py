"""Randomised properties of the oracle (CPU only; hypothesis draws the cases).

Shapes, layouts, transposes, alpha, beta, verification-tile geometries and k-tile depths
are drawn at random. Each example checks facts that hold independently of the oracle's
code:

- Section II.A's checksum relations, e^T C = alpha (e^T op(A)) op(B) + beta e^T C_in and
  C e = alpha op(A) (op(B) e) + beta C_in e, summed here without rounding (math.fsum over
  the individual products) and compared within the rounding bound of the product;
- the product against a library matmul within the standard bound 2 gamma_{K+2}
  (|alpha| |A||B| + |beta| |C_in|);
- a clean protected run flags nothing and checks every tile;
- on integer operands, where every checksum is exact, one output error of any size and sign
  at any element (Section VI.C) is located at that element. Its row and column mismatches
  both equal the error exactly, and the recomputed C equals the fault-free C bit for bit.
"""
import math
from fractions import Fraction

import numpy as np
import pytest

import oracle as O
import synth as S
from tests.helpers import stored

hypothesis = pytest.importorskip("hypothesis")
from hypothesis import HealthCheck, assume, given, settings  # noqa: E402
from hypothesis import strategies as st  # noqa: E402

U = 2.0 ** -53
SETTINGS = settings(max_examples=120, deadline=None, suppress_health_check=[HealthCheck.too_slow])


def gamma(n):
    return n * U / (1 - n * U)


def c_store(layout, C_log, pad):
    ld = (C_log.shape[0] if layout == O.COL_MAJOR else C_log.shape[1]) + pad
    return S.store(C_log, layout, ld=max(1, ld))


def run(case, A, B, Cin, protected, inj=()):
    layout, ta, tb, alpha, beta, tm, tn, bk, pad = (case[k] for k in
                                                    ("layout", "ta", "tb", "alpha", "beta", "tm", "tn", "bk", "pad"))
    M, K = A.shape
    N = B.shape[1]
    a, lda = stored(layout, ta, A, pad=pad)
    b, ldb = stored(layout, tb, B, pad=pad)
    c, ldc = c_store(layout, Cin, pad)
    if not protected:
        return S.load(O.gemm(layout, ta, tb, M, N, K, alpha, a, lda, b, ldb, beta, c, ldc), layout, M, N, ldc)
    out, rep = O.ft_gemm(layout, ta, tb, M, N, K, alpha, a, lda, b, ldb, beta, c, ldc, tm, tn, bk, injections=inj)
    return S.load(out, layout, M, N, ldc), rep


def cases(alphas, betas):
    return st.fixed_dictionaries({
        "M": st.integers(1, 20), "N": st.integers(1, 20), "K": st.integers(1, 24),
        "layout": st.sampled_from([O.COL_MAJOR, O.ROW_MAJOR]),
        "ta": st.sampled_from([O.NO_TRANS, O.TRANS]), "tb": st.sampled_from([O.NO_TRANS, O.TRANS]),
        "alpha": st.sampled_from(alphas), "beta": st.sampled_from(betas),
        "tm": st.integers(1, 8), "tn": st.integers(1, 8), "bk": st.integers(1, 6),
        "pad": st.integers(0, 3), "seed": st.integers(0, 10 ** 6),
    })


@SETTINGS
@given(cases([1.0, -0.75, 1.5, 2.0], [0.0, 0.5, -1.0]))
def test_product_checksum_relations_and_library_bound(case):
    M, N, K, seed = case["M"], case["N"], case["K"], case["seed"]
    alpha, beta = case["alpha"], case["beta"]
    A = S.uniform_matrix(seed, 0, M, K)
    B = S.uniform_matrix(seed, 1, K, N)
    Cin = S.uniform_matrix(seed, 2, M, N)
    C = run(case, A, B, Cin, protected=False)
    mag = abs(alpha) * (np.abs(A) @ np.abs(B)) + abs(beta) * np.abs(Cin)
    # library cross-check
    lib = alpha * (A @ B) + beta * Cin
    assert np.all(np.abs(C - lib) <= 2 * gamma(K + 2) * mag + 1e-300)
    # Section II.A relations, right-hand sides summed without intermediate rounding
    g = gamma(K + 3)
    for j in range(N):
        rhs = math.fsum([alpha * A[i, k] * B[k, j] for i in range(M) for k in range(K)] +
                        [beta * Cin[i, j] for i in range(M)])
        assert abs(math.fsum(C[:, j]) - rhs) <= 2 * g * mag[:, j].sum() + 1e-300
    for i in range(M):
        rhs = math.fsum([alpha * A[i, k] * B[k, j] for j in range(N) for k in range(K)] +
                        [beta * Cin[i, j] for j in range(N)])
        assert abs(math.fsum(C[i, :]) - rhs) <= 2 * g * mag[i, :].sum() + 1e-300


@SETTINGS
@given(cases([1.0, -0.75, 1.5], [0.0, 0.5, -1.0]))
def test_clean_protected_run_checks_every_tile_and_flags_nothing(case):
    M, N, K, seed = case["M"], case["N"], case["K"], case["seed"]
    A = S.uniform_matrix(seed, 0, M, K)
    B = S.uniform_matrix(seed, 1, K, N)
    Cin = S.uniform_matrix(seed, 2, M, N)
    got, rep = run(case, A, B, Cin, protected=True)
    assert rep.detected == 0 and rep.input_nonfinite == 0 and rep.n_records == 0
    assert rep.tiles_checked == math.ceil(M / case["tm"]) * math.ceil(N / case["tn"])
    assert np.array_equal(got, run(case, A, B, Cin, protected=False))


@SETTINGS
@given(cases([1.0, 2.0, -1.0], [0.0, 1.0, -2.0]), st.integers(0, 10 ** 6), st.integers(-3, 6),
       st.sampled_from([1, -1]))
def test_one_output_error_anywhere_is_located_and_removed_exactly(case, where, p, sign):
    M, N, K, seed = case["M"], case["N"], case["K"], case["seed"]
    A = S.randint(seed, 0, M * K, -4, 4).reshape(M, K).astype(np.float64)
    B = S.randint(seed, 1, K * N, -4, 4).reshape(K, N).astype(np.float64)
    Cin = S.randint(seed, 2, M * N, -9, 9).reshape(M, N).astype(np.float64)
    clean = run(case, A, B, Cin, protected=False)
    i, j = (where // N) % M, where % N
    assume(clean[i, j] != 0)
    e = sign * 2.0 ** p * abs(clean[i, j])
    got, rep = run(case, A, B, Cin, protected=True,
                   inj=[dict(i=i, j=j, site=O.SITE_OUTPUT, mode=O.MODE_ADD_REL, rel_log2=p, sign=sign)])
    assert (rep.detected, rep.corrected, rep.uncorrectable, rep.checksum_only) == (1, 1, 0, 0)
    r = rep.records()[0]
    assert (r.i, r.j) == (i, j)
    assert (r.tile_row, r.tile_col) == (i // case["tm"], j // case["tn"])
    assert r.delta_row == e and r.delta_col == e
    assert np.array_equal(got, clean)


# ------------------------------------------------------------------------------------
# The binary32-accumulation model of the tensor-core forms (ACC32)
# ------------------------------------------------------------------------------------

def bf16_exact(X):
    return S.bf16_bits_to_f64(S.to_bf16_bits(X))


@SETTINGS
@given(cases([1.0, 2.0], [0.0, 1.0, -2.0]))
def test_acc32_output_is_the_exact_product_rounded_once_to_binary32(case):
    """A on the grid 2^-8 Z and B, C_in bfloat16 of magnitude 0 or at least 2^-12 in
    [-1, 1): every product is a multiple of 2^-27 below 1, so with K <= 24 and alpha, beta
    powers of two, alpha acc + beta C_in has at most 33 significant bits and is exact in
    binary64 in any order. C must be that value rounded to nearest binary32 (a real
    rounding: up to 33 bits into 24), and a clean run must flag nothing."""
    M, N, K, seed = case["M"], case["N"], case["K"], case["seed"]

    def bf16_not_tiny(X):
        X = bf16_exact(X)
        return np.where(np.abs(X) < 2.0 ** -12, 0.0, X)

    A = np.round(S.uniform_matrix(seed, 0, M, K) * 256.0) / 256.0
    B = bf16_not_tiny(S.uniform_matrix(seed, 1, K, N))
    Cin = bf16_not_tiny(S.uniform_matrix(seed, 2, M, N))
    exact = case["alpha"] * (A @ B) + case["beta"] * Cin  # every step exact here
    a, lda = stored(case["layout"], case["ta"], A, pad=case["pad"])
    b, ldb = stored(case["layout"], case["tb"], B, pad=case["pad"])
    c, ldc = c_store(case["layout"], Cin, case["pad"])
    out, rep = O.ft_gemm(case["layout"], case["ta"], case["tb"], M, N, K, case["alpha"], a, lda, b, ldb,
                         case["beta"], c, ldc, case["tm"], case["tn"], case["bk"], precision=O.PREC_ACC32)
    got = S.load(out, case["layout"], M, N, ldc)
    assert np.array_equal(got, exact.astype(np.float32).astype(np.float64))
    assert rep.detected == 0 and rep.tiles_checked == math.ceil(M / case["tm"]) * math.ceil(N / case["tn"])


@SETTINGS
@given(cases([1.0, -0.75, 1.5], [0.0, 0.5]), st.integers(-8, 8))
def test_acc32_clean_runs_never_flag_under_row_scaling(case, shift):
    M, N, K, seed = case["M"], case["N"], case["K"], case["seed"]
    A = bf16_exact(S.normal_matrix(seed, 0, M, K) * S.pow2_row_scales(seed, 5, M)[:, None] * 2.0 ** shift)
    B = bf16_exact(S.normal_matrix(seed, 1, K, N))
    Cin = S.normal_matrix(seed, 2, M, N)
    a, lda = stored(case["layout"], case["ta"], A, pad=case["pad"])
    b, ldb = stored(case["layout"], case["tb"], B, pad=case["pad"])
    c, ldc = c_store(case["layout"], Cin, case["pad"])
    _, rep = O.ft_gemm(case["layout"], case["ta"], case["tb"], M, N, K, case["alpha"], a, lda, b, ldb,
                       case["beta"], c, ldc, case["tm"], case["tn"], case["bk"], precision=O.PREC_ACC32)
    assert rep.detected == 0


@SETTINGS
@given(cases([1.0, 2.0, -1.0], [0.0, 1.0]), st.integers(0, 10 ** 6), st.integers(0, 6), st.sampled_from([1, -1]))
def test_acc32_one_output_error_anywhere_is_located_and_removed_exactly(case, where, p, sign):
    M, N, K, seed = case["M"], case["N"], case["K"], case["seed"]
    A = S.randint(seed, 0, M * K, -4, 4).reshape(M, K).astype(np.float64)
    B = S.randint(seed, 1, K * N, -4, 4).reshape(K, N).astype(np.float64)
    Cin = S.randint(seed, 2, M * N, -9, 9).reshape(M, N).astype(np.float64)
    a, lda = stored(case["layout"], case["ta"], A, pad=case["pad"])
    b, ldb = stored(case["layout"], case["tb"], B, pad=case["pad"])
    c, ldc = c_store(case["layout"], Cin, case["pad"])

    def call(inj):
        out, rep = O.ft_gemm(case["layout"], case["ta"], case["tb"], M, N, K, case["alpha"], a, lda, b, ldb,
                             case["beta"], c, ldc, case["tm"], case["tn"], case["bk"], injections=inj,
                             precision=O.PREC_ACC32)
        return S.load(out, case["layout"], M, N, ldc), rep

    clean, rep0 = call(())
    assert rep0.detected == 0
    assert np.array_equal(clean, case["alpha"] * (A @ B) + case["beta"] * Cin)  # small integers: exact
    i, j = (where // N) % M, where % N
    assume(clean[i, j] != 0)
    got, rep = call([dict(i=i, j=j, site=O.SITE_OUTPUT, mode=O.MODE_ADD_REL, rel_log2=p, sign=sign)])
    assert (rep.detected, rep.corrected) == (1, 1)
    r = rep.records()[0]
    assert (r.i, r.j) == (i, j)
    assert r.delta_row == sign * 2.0 ** p * abs(clean[i, j])
    assert np.array_equal(got, clean)


# ------------------------------------------------------------------------------------
# The triangular solve behind FT-DTRSM's reference
# ------------------------------------------------------------------------------------

@SETTINGS
@given(st.integers(1, 24), st.integers(1, 10), st.booleans(), st.integers(0, 10 ** 6))
def test_substitution_meets_its_componentwise_backward_error_bound(n, nrhs, lower, seed):
    """Substitution is componentwise backward stable: the computed X satisfies
    |T X - W| <= gamma_n |T| |X| (a textbook bound for forward and back substitution with
    any summation order). The unread triangle holds NaN, so reading it would show."""
    R = S.uniform_matrix(seed, 0, n, n)
    d = 0.5 + S.uniform(seed, 1, n) ** 2                      # diagonal away from zero
    T = np.tril(R, -1) if lower else np.triu(R, 1)
    T = T + np.diag(d * np.where(S.uniform(seed, 2, n) < 0, -1.0, 1.0))
    W = S.uniform_matrix(seed, 3, n, nrhs)
    Tn = np.where(np.tril(np.ones((n, n))) if lower else np.triu(np.ones((n, n))), T, np.nan)
    X = O.trsm_left(Tn, W, lower)
    # the residual formed exactly (rational arithmetic), so that only the solve's rounding shows
    Tf = [[Fraction(float(v)) for v in row] for row in T]
    bound = gamma(n) * (np.abs(T) @ np.abs(X)) * (1 + 1e-9)
    for j in range(nrhs):
        xj = [Fraction(float(v)) for v in X[:, j]]
        for i in range(n):
            res = sum((Tf[i][k] * xj[k] for k in range(n)), Fraction(0)) - Fraction(float(W[i, j]))
            assert abs(res) <= Fraction(float(bound[i, j])), (i, j, float(res), bound[i, j])


# ------------------------------------------------------------------------------------
# Online (mid-K) verification: one correctable error per interval
# ------------------------------------------------------------------------------------

@SETTINGS
@given(st.data())
def test_online_checks_correct_one_flip_per_interval(data):
    """Integer operands (exact partial checksums); checks every kc products. Two accumulator
    flips of an exponent bit in one tile, strictly inside two different intervals, are each
    corrected at the check that follows them (Section V.A's rank-K_c steps), and C equals
    the fault-free C bit for bit. Without online checks the pair is uncorrectable."""
    bk = data.draw(st.integers(1, 3))
    kc = bk * data.draw(st.integers(2, 3))
    K = kc * data.draw(st.integers(3, 4))
    M, N = data.draw(st.integers(1, 10)), data.draw(st.integers(2, 10))
    tm, tn = data.draw(st.integers(1, 6)), data.draw(st.integers(2, 6))
    seed = data.draw(st.integers(0, 10 ** 6))
    A = S.randint(seed, 0, M * K, 1, 4).reshape(M, K).astype(np.float64)   # positive: partial sums > 0
    B = S.randint(seed, 1, K * N, 1, 4).reshape(K, N).astype(np.float64)
    inside = [kt for kt in range(1, K // bk) if (kt * bk) % kc != 0]
    last = (K // bk - 1) * bk // kc
    kt1 = data.draw(st.sampled_from([kt for kt in inside if (kt * bk) // kc < last]))
    kt2 = data.draw(st.sampled_from([kt for kt in inside if (kt * bk) // kc > (kt1 * bk) // kc]))
    hi, hj = min(tm, M), min(tn, N)  # both flips in tile (0, 0), which has at least 2 elements
    e1 = data.draw(st.integers(0, hi * hj - 1))
    e2 = data.draw(st.integers(0, hi * hj - 2))
    e2 += e2 >= e1  # a different element: the injection model holds one accumulator point per element
    (i1, j1), (i2, j2) = divmod(e1, hj), divmod(e2, hj)
    bit = data.draw(st.integers(55, 60))
    a, lda = stored(O.COL_MAJOR, O.NO_TRANS, A)
    b, ldb = stored(O.COL_MAJOR, O.NO_TRANS, B)
    c, ldc = c_store(O.COL_MAJOR, np.zeros((M, N)), 0)

    def call(kc_, inj):
        out, rep = O.ft_gemm(O.COL_MAJOR, O.NO_TRANS, O.NO_TRANS, M, N, K, 1.0, a, lda, b, ldb, 0.0, c, ldc,
                             tm, tn, bk, injections=inj, kc=kc_)
        return S.load(out, O.COL_MAJOR, M, N, ldc), rep

    clean, rep0 = call(kc, ())
    assert rep0.detected == 0 and np.array_equal(clean, A @ B)  # small integers: exact
    pts = [dict(i=i1, j=j1, site=O.SITE_ACCUM, mode=O.MODE_BITFLIP, bit=bit, kt=kt1),
           dict(i=i2, j=j2, site=O.SITE_ACCUM, mode=O.MODE_BITFLIP, bit=bit, kt=kt2)]
    got, rep = call(kc, pts)
    assert rep.corrected == 2 and rep.uncorrectable == 0
    assert sorted((r.i, r.j) for r in rep.records()) == sorted([(i1, j1), (i2, j2)])
    assert np.array_equal(got, clean)
    _, rep_end = call(0, pts)
    assert rep_end.corrected == 0 and rep_end.uncorrectable == 1


# ------------------------------------------------------------------------------------
# Classification of several errors (G4)
# ------------------------------------------------------------------------------------

@SETTINGS
@given(st.data())
def test_two_errors_in_one_tile_are_uncorrectable_and_in_two_tiles_corrected(data):
    """Integer operands, so each flagged row and column carries the exact error. Two errors
    at different elements of one tile flag two rows and/or two columns: uncorrectable, with
    C left as computed (both errors stay). Two errors in different tiles: both corrected."""
    M, N, K = data.draw(st.integers(2, 12)), data.draw(st.integers(2, 12)), data.draw(st.integers(1, 12))
    tm, tn = data.draw(st.integers(1, 6)), data.draw(st.integers(1, 6))
    seed = data.draw(st.integers(0, 10 ** 6))
    A = S.randint(seed, 0, M * K, 1, 4).reshape(M, K).astype(np.float64)  # positive: C >= 1
    B = S.randint(seed, 1, K * N, 1, 4).reshape(K, N).astype(np.float64)
    case = dict(layout=O.COL_MAJOR, ta=O.NO_TRANS, tb=O.NO_TRANS, alpha=1.0, beta=0.0, tm=tm, tn=tn,
                bk=data.draw(st.integers(1, 4)), pad=0)
    Cin = np.zeros((M, N))
    clean = run(case, A, B, Cin, protected=False)
    err = lambda i, j: dict(i=i, j=j, site=O.SITE_OUTPUT, mode=O.MODE_ADD_REL, rel_log2=3, sign=1)
    tiles = [(r, c) for r in range(-(-M // tm)) for c in range(-(-N // tn))]
    tr, tc = data.draw(st.sampled_from(tiles))
    cells = [(i, j) for i in range(tr * tm, min(M, tr * tm + tm)) for j in range(tc * tn, min(N, tc * tn + tn))]
    if len(cells) >= 2:
        (i1, j1), (i2, j2) = data.draw(st.lists(st.sampled_from(cells), min_size=2, max_size=2, unique=True))
        got, rep = run(case, A, B, Cin, protected=True, inj=[err(i1, j1), err(i2, j2)])
        assert (rep.detected, rep.uncorrectable, rep.corrected) == (1, 1, 0)
        (r,) = rep.records()
        assert (r.rows_flagged, r.cols_flagged) == (len({i1, i2}), len({j1, j2}))
        assert got[i1, j1] == 9 * clean[i1, j1] and got[i2, j2] == 9 * clean[i2, j2]
    if len(tiles) >= 2:
        (ta_, tb_) = data.draw(st.lists(st.sampled_from(tiles), min_size=2, max_size=2, unique=True))
        pick = lambda t: (t[0] * tm, t[1] * tn)
        (i1, j1), (i2, j2) = pick(ta_), pick(tb_)
        got, rep = run(case, A, B, Cin, protected=True, inj=[err(i1, j1), err(i2, j2)])
        assert (rep.detected, rep.corrected, rep.uncorrectable) == (2, 2, 0)
        assert np.array_equal(got, clean)


@SETTINGS
@given(st.data())
def test_a_fault_in_a_predicted_checksum_alone_is_checksum_only(data):
    """A fault in the predicted checksum and nowhere in C flags one side only: reported as
    checksum-only, and C is left exactly as the fault-free product (G4)."""
    M, N, K = data.draw(st.integers(1, 12)), data.draw(st.integers(1, 12)), data.draw(st.integers(1, 12))
    layout = data.draw(st.sampled_from([O.COL_MAJOR, O.ROW_MAJOR]))
    case = dict(layout=layout, ta=O.NO_TRANS, tb=O.NO_TRANS, alpha=1.0, beta=0.0,
                tm=data.draw(st.integers(1, 6)), tn=data.draw(st.integers(1, 6)), bk=data.draw(st.integers(1, 4)), pad=0)
    seed = data.draw(st.integers(0, 10 ** 6))
    A = S.randint(seed, 0, M * K, 1, 4).reshape(M, K).astype(np.float64)
    B = S.randint(seed, 1, K * N, 1, 4).reshape(K, N).astype(np.float64)
    Cin = np.zeros((M, N))
    clean = run(case, A, B, Cin, protected=False)
    i, j = data.draw(st.integers(0, M - 1)), data.draw(st.integers(0, N - 1))
    got, rep = run(case, A, B, Cin, protected=True,
                   inj=[dict(i=i, j=j, site=O.SITE_CHECKSUM, mode=O.MODE_ADD_REL, rel_log2=2, sign=1)])
    assert (rep.detected, rep.checksum_only, rep.corrected, rep.uncorrectable) == (1, 1, 0, 0)
    assert np.array_equal(got, clean)


@SETTINGS
@given(st.data())
def test_acc32_error_in_the_smallest_row_is_located_and_removed_exactly(data):
    """Rows of A scaled by 2^u, u in [-8, 8] (config 3's structure), with small integer
    entries: every value is dyadic and exact in binary32. An output error 2^-4 |C(i,j)| in
    the row of smallest scale is far above that row's threshold (positive entries make
    C(i,j) at least the row's sum of |A|) but usually below the column thresholds, which the
    large rows of the tile dominate; the row-recompute locator (beta = 0) then finds it.
    Either way it is located, and the correction from the row checksum restores C exactly."""
    M, N, K = data.draw(st.integers(8, 16)), data.draw(st.integers(1, 16)), data.draw(st.integers(32, 64))
    seed = data.draw(st.integers(0, 10 ** 6))
    A = S.randint(seed, 0, M * K, 1, 3).reshape(M, K).astype(np.float64) * S.pow2_row_scales(seed, 5, M)[:, None]
    B = S.randint(seed, 1, K * N, 1, 3).reshape(K, N).astype(np.float64)
    case = dict(layout=O.COL_MAJOR, ta=O.TRANS, tb=O.NO_TRANS, alpha=1.0, beta=0.0,
                tm=16, tn=data.draw(st.integers(1, 16)), bk=64, pad=0)
    a, lda = stored(case["layout"], case["ta"], A)
    b, ldb = stored(case["layout"], case["tb"], B)
    c, ldc = c_store(case["layout"], np.zeros((M, N)), 0)

    def call(inj):
        out, rep = O.ft_gemm(case["layout"], case["ta"], case["tb"], M, N, K, 1.0, a, lda, b, ldb, 0.0, c, ldc,
                             case["tm"], case["tn"], case["bk"], injections=inj, precision=O.PREC_ACC32)
        return S.load(out, case["layout"], M, N, ldc), rep

    clean, rep0 = call(())
    assert rep0.detected == 0 and np.array_equal(clean, A @ B)
    i = int(np.argmin(np.abs(A).sum(axis=1)))
    j = data.draw(st.integers(0, N - 1))
    got, rep = call([dict(i=i, j=j, site=O.SITE_OUTPUT, mode=O.MODE_ADD_REL, rel_log2=-4, sign=1)])
    assert (rep.detected, rep.corrected) == (1, 1)
    assert (rep.records()[0].i, rep.records()[0].j) == (i, j)
    assert np.array_equal(got, clean)
