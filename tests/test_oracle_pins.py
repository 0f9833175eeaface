"""Pins for the CPU oracle: facts fixed by the mathematics and the paper, not by the oracle.

FT-BLAS Section II.A defines the checksum relations e^T C = (e^T A) B and C e = A (B e),
Section V.A/V.B the detect/locate scheme with beta*C folded in, and Section VI.C the
correction of an injected error by its located magnitude. Each test below checks the
oracle against something independent of its own code: closed-form products of integer
matrices (exact in binary64), special cases that reduce to textbook results, a library
matmul within the standard rounding bound, brute-force injection on tiny inputs with the
faulty value recomputed here in plain Python floats, and exact checksum differences on
integer data.
"""
import math
import os
import struct

import numpy as np
import pytest

import oracle as O
import synth as S

U = 2.0 ** -53
LAYOUTS = [O.COL_MAJOR, O.ROW_MAJOR]
TRANS = [O.NO_TRANS, O.TRANS]
COMBOS = [(l, a, b) for l in LAYOUTS for a in TRANS for b in TRANS]


def gamma(n):
    return n * U / (1 - n * U)


def stored(layout, trans, logical, pad=3):
    """BLAS storage of X such that op(X) == logical."""
    X = logical if trans == O.NO_TRANS else logical.T
    ld = (X.shape[0] if layout == O.COL_MAJOR else X.shape[1]) + pad
    return S.store(X, layout, ld=max(1, ld))


def c_store(layout, C_log, pad=2):
    ld = (C_log.shape[0] if layout == O.COL_MAJOR else C_log.shape[1]) + pad
    return S.store(C_log, layout, ld=max(1, ld))


def plain(layout, ta, tb, A_log, B_log, alpha=1.0, beta=0.0, C_log=None):
    M, K = A_log.shape
    N = B_log.shape[1]
    a, lda = stored(layout, ta, A_log)
    b, ldb = stored(layout, tb, B_log)
    if C_log is None:
        C_log = np.zeros((M, N))
    c, ldc = c_store(layout, C_log)
    out = O.gemm(layout, ta, tb, M, N, K, alpha, a, lda, b, ldb, beta, c, ldc)
    return S.load(out, layout, M, N, ldc)


def ft(layout, ta, tb, A_log, B_log, alpha=1.0, beta=0.0, C_log=None, tile=(4, 4), bk=2, inj=(), tiles=None):
    M, K = A_log.shape
    N = B_log.shape[1]
    a, lda = stored(layout, ta, A_log)
    b, ldb = stored(layout, tb, B_log)
    if C_log is None:
        C_log = np.zeros((M, N))
    c, ldc = c_store(layout, C_log)
    out, rep = O.ft_gemm(layout, ta, tb, M, N, K, alpha, a, lda, b, ldb, beta, c, ldc,
                         tile[0], tile[1], bk, injections=inj, tiles=tiles)
    return S.load(out, layout, M, N, ldc), rep


def flip(x, bit):
    (u,) = struct.unpack("<Q", struct.pack("<d", x))
    return struct.unpack("<d", struct.pack("<Q", u ^ (1 << bit)))[0]


# ------------------------------------------------------------------------------------
# The product itself
# ------------------------------------------------------------------------------------

@pytest.mark.parametrize("layout,ta,tb", COMBOS)
@pytest.mark.parametrize("M,N,K", [(1, 1, 1), (7, 5, 9), (33, 17, 64)])
def test_closed_form_linear_operands(layout, ta, tb, M, N, K):
    """A(i,k) = i + k, B(k,j) = k + j  =>  C(i,j) = K i j + (i + j) S1 + S2, exactly."""
    i = np.arange(M)[:, None]
    j = np.arange(N)[None, :]
    k = np.arange(K)
    A = (np.arange(M)[:, None] + k[None, :]).astype(np.float64)
    B = (k[:, None] + np.arange(N)[None, :]).astype(np.float64)
    S1 = K * (K - 1) // 2
    S2 = (K - 1) * K * (2 * K - 1) // 6
    expect = (K * i * j + (i + j) * S1 + S2).astype(np.float64)
    assert np.array_equal(plain(layout, ta, tb, A, B), expect)
    # alpha, beta with exact dyadic values and an integer C_in
    Cin = (i - 2 * j).astype(np.float64)
    got = plain(layout, ta, tb, A, B, alpha=0.5, beta=-2.0, C_log=Cin)
    assert np.array_equal(got, 0.5 * expect - 2.0 * Cin)


@pytest.mark.parametrize("layout,ta,tb", COMBOS)
def test_identity_and_ones(layout, ta, tb):
    K, N = 6, 5
    B = S.uniform_matrix(3, 1, K, N)
    assert np.array_equal(plain(layout, ta, tb, np.eye(K), B), B)
    Bi = S.randint(3, 2, K * N, -9, 9).reshape(K, N).astype(np.float64)
    ones = np.ones((4, K))
    expect = np.tile(Bi.sum(axis=0), (4, 1))  # integer column sums, exact
    assert np.array_equal(plain(layout, ta, tb, ones, Bi), expect)


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_library_matmul_within_rounding_bound(seed):
    M, N, K = 23, 19, 71
    A = S.uniform_matrix(seed, 0, M, K)
    B = S.uniform_matrix(seed, 1, K, N)
    got = plain(O.COL_MAJOR, O.NO_TRANS, O.NO_TRANS, A, B)
    bound = 2 * gamma(K) * (np.abs(A) @ np.abs(B))
    assert np.all(np.abs(got - A @ B) <= bound)


def test_storage_variants_give_identical_bits():
    """op() and layout change only where elements are read, never the order of a sum."""
    M, N, K = 13, 11, 29
    A = S.uniform_matrix(5, 0, M, K)
    B = S.uniform_matrix(5, 1, K, N)
    Cin = S.uniform_matrix(5, 2, M, N)
    ref = plain(O.COL_MAJOR, O.NO_TRANS, O.NO_TRANS, A, B, 1.5, 0.5, Cin)
    for layout, ta, tb in COMBOS:
        assert np.array_equal(plain(layout, ta, tb, A, B, 1.5, 0.5, Cin), ref)


@pytest.mark.parametrize("seed", [11, 12])
def test_checksum_invariants_of_the_product(seed):
    """Section II.A: e^T C = (e^T A) B and C e = A (B e), within rounding."""
    M, N, K = 40, 30, 50
    A = S.uniform_matrix(seed, 0, M, K)
    B = S.uniform_matrix(seed, 1, K, N)
    Cm = plain(O.COL_MAJOR, O.NO_TRANS, O.NO_TRANS, A, B)
    absprod = np.abs(A) @ np.abs(B)
    col_lhs = np.array([math.fsum(Cm[:, j]) for j in range(N)])
    col_rhs = np.array([math.fsum(A.sum(axis=0) * B[:, j]) for j in range(N)])
    row_lhs = np.array([math.fsum(Cm[i, :]) for i in range(M)])
    row_rhs = np.array([math.fsum(A[i, :] * B.sum(axis=1)) for i in range(M)])
    g = gamma(K + max(M, N) + 2)
    assert np.all(np.abs(col_lhs - col_rhs) <= 2 * g * absprod.sum(axis=0))
    assert np.all(np.abs(row_lhs - row_rhs) <= 2 * g * absprod.sum(axis=1))


# ------------------------------------------------------------------------------------
# The fault-tolerant path
# ------------------------------------------------------------------------------------

@pytest.mark.parametrize("layout,ta,tb", COMBOS)
@pytest.mark.parametrize("alpha,beta", [(1.0, 0.0), (1.5, 0.5), (-0.75, 2.0)])
def test_clean_runs_never_flag_and_match_plain(layout, ta, tb, alpha, beta):
    M, N, K = 37, 29, 45
    A = S.uniform_matrix(21, 0, M, K)
    B = S.uniform_matrix(21, 1, K, N)
    Cin = S.uniform_matrix(21, 2, M, N)
    for tile, bk in [((16, 8), 4), ((4, 4), 3), ((37, 29), 16), ((1, 29), 1)]:
        got, rep = ft(layout, ta, tb, A, B, alpha, beta, Cin, tile=tile, bk=bk)
        assert rep.detected == 0 and rep.input_nonfinite == 0
        assert rep.tiles_checked == math.ceil(M / tile[0]) * math.ceil(N / tile[1])
        assert np.array_equal(got, plain(layout, ta, tb, A, B, alpha, beta, Cin))


def test_clean_soak_structured_magnitudes():
    """Rows of A and columns of B scaled by 2^u, u in [-8, 8]: no false alarm."""
    for seed in range(6):
        M, N, K = 48, 40, 96
        A = S.normal_matrix(seed, 0, M, K) * S.pow2_row_scales(seed, 5, M)[:, None]
        B = S.normal_matrix(seed, 1, K, N) * S.pow2_row_scales(seed, 6, N)[None, :]
        Cin = S.normal_matrix(seed, 2, M, N)
        _, rep = ft(O.COL_MAJOR, O.NO_TRANS, O.NO_TRANS, A, B, 1.5, 0.5, Cin, tile=(16, 16), bk=8)
        assert rep.detected == 0


@pytest.mark.filterwarnings("ignore::RuntimeWarning")
@pytest.mark.parametrize("tile", [(2, 2), (4, 4), (3, 2), (1, 5), (4, 5)])
@pytest.mark.parametrize("bk", [1, 2])
def test_bruteforce_accumulator_bitflips_tiny(tile, bk):
    """Every element and every bit 40..62 of a 4x5x3 product: the flipped element is
    located exactly and the corrected output equals the fault-free output bit for bit."""
    M, N, K = 4, 5, 3
    A = S.uniform_matrix(7, 0, M, K)
    B = S.uniform_matrix(7, 1, K, N)
    clean = plain(O.COL_MAJOR, O.NO_TRANS, O.NO_TRANS, A, B)
    nk = -(-K // bk)
    kstar = bk * (nk // 2)
    for i in range(M):
        for j in range(N):
            for bit in range(40, 63):
                acc = 0.0
                for k in range(K):
                    if k == kstar:
                        acc = flip(acc, bit)
                    acc = acc + A[i, k] * B[k, j]
                bad = acc  # alpha = 1, beta = 0
                err = bad - clean[i, j]
                if math.isfinite(err) and abs(err) < 1e-9:
                    continue  # below any plausible threshold: not a detection case
                got, rep = ft(O.COL_MAJOR, O.NO_TRANS, O.NO_TRANS, A, B, tile=tile, bk=bk,
                              inj=[dict(i=i, j=j, site=O.SITE_ACCUM, bit=bit)])
                assert (rep.detected, rep.corrected, rep.uncorrectable, rep.checksum_only) == (1, 1, 0, 0)
                r = rep.records()[0]
                assert (r.i, r.j, r.kind) == (i, j, O.KIND_CORRECTED)
                assert struct.pack("<d", r.value_before) == struct.pack("<d", bad)
                assert np.array_equal(got, clean)


@pytest.mark.parametrize("layout,ta,tb", COMBOS)
def test_delta_is_the_injected_magnitude_on_integer_data(layout, ta, tb):
    """Integer operands make every checksum exact, so C^r_ref - C^r and C^c_ref - C^c
    equal the injected error e exactly, and subtracting it (Section VI.C) restores C."""
    M, N, K = 9, 7, 12
    A = S.randint(31, 0, M * K, -4, 4).reshape(M, K).astype(np.float64)
    B = S.randint(31, 1, K * N, -4, 4).reshape(K, N).astype(np.float64)
    Cin = S.randint(31, 2, M * N, -9, 9).reshape(M, N).astype(np.float64)
    clean = plain(layout, ta, tb, A, B, 1.0, 1.0, Cin)
    for (i, j, p, s) in [(0, 0, 0, 1), (8, 6, -3, -1), (4, 3, 2, 1), (5, 1, -7, -1)]:
        if clean[i, j] == 0:
            continue
        e = s * 2.0 ** p * abs(clean[i, j])
        got, rep = ft(layout, ta, tb, A, B, 1.0, 1.0, Cin, tile=(9, 7), bk=4,
                      inj=[dict(i=i, j=j, site=O.SITE_OUTPUT, mode=O.MODE_ADD_REL, rel_log2=p, sign=s)])
        r = rep.records()[0]
        assert (r.i, r.j, rep.corrected) == (i, j, 1)
        assert r.delta_row == e and r.delta_col == e
        assert r.value_before == clean[i, j] + e
        assert r.value_subtracted == clean[i, j]
        assert np.array_equal(got, clean)


def test_classification_multiple_and_checksum_faults():
    M, N, K = 16, 16, 20
    A = S.randint(41, 0, M * K, -3, 3).reshape(M, K).astype(np.float64)
    B = S.randint(41, 1, K * N, -3, 3).reshape(K, N).astype(np.float64)
    clean = plain(O.COL_MAJOR, O.NO_TRANS, O.NO_TRANS, A, B)
    add = lambda i, j, p=2: dict(i=i, j=j, site=O.SITE_OUTPUT, mode=O.MODE_ADD_REL, rel_log2=p, sign=1)
    nz = [(i, j) for i in range(M) for j in range(N) if clean[i, j] != 0]
    # two errors in one 8x8 tile, different rows and columns: uncorrectable, C kept as computed
    (i1, j1), (i2, j2) = [(i, j) for (i, j) in nz if i < 8 and j < 8][0], (7, 7)
    if clean[7, 7] == 0:
        pytest.skip("degenerate draw")
    got, rep = ft(O.COL_MAJOR, O.NO_TRANS, O.NO_TRANS, A, B, tile=(8, 8), inj=[add(i1, j1), add(i2, j2)])
    assert (rep.detected, rep.uncorrectable, rep.corrected) == (1, 1, 0)
    assert got[i1, j1] != clean[i1, j1]
    # two errors in one row of one tile: one row, two columns flagged -> uncorrectable
    row_pair = [(i, j) for (i, j) in nz if i == 9 and j >= 8][:2]
    _, rep = ft(O.COL_MAJOR, O.NO_TRANS, O.NO_TRANS, A, B, tile=(8, 8), inj=[add(*row_pair[0]), add(*row_pair[1])])
    assert (rep.detected, rep.uncorrectable) == (1, 1)
    r = rep.records()[0]
    assert (r.rows_flagged, r.cols_flagged) == (1, 2)
    # one error in each of two tiles: both corrected
    got, rep = ft(O.COL_MAJOR, O.NO_TRANS, O.NO_TRANS, A, B, tile=(8, 8),
                  inj=[add(*nz[0]), add(*[(i, j) for (i, j) in nz if i >= 8 and j >= 8][0])])
    assert (rep.detected, rep.corrected, rep.tiles_checked) == (2, 2, 4)
    assert np.array_equal(got, clean)
    # a fault in the predicted row checksum only: checksum-only, C untouched
    i_cs = [i for i in range(8) if clean[i, :8].sum() != 0][0]
    got, rep = ft(O.COL_MAJOR, O.NO_TRANS, O.NO_TRANS, A, B, tile=(8, 8),
                  inj=[dict(i=i_cs, j=0, site=O.SITE_CHECKSUM, mode=O.MODE_ADD_REL, rel_log2=0, sign=1)])
    assert (rep.detected, rep.checksum_only, rep.corrected) == (1, 1, 0)
    assert rep.records()[0].i == i_cs and rep.records()[0].j == -1
    assert np.array_equal(got, clean)


def test_quick_returns_and_beta_zero_ignores_nan():
    M, N, K = 6, 5, 4
    A = S.uniform_matrix(1, 0, M, K)
    B = S.uniform_matrix(1, 1, K, N)
    Cin = S.uniform_matrix(1, 2, M, N)
    # K = 0 and alpha = 0: C = beta * C, nothing checked
    for (Kq, alpha) in [(0, 1.0), (K, 0.0)]:
        Aq = A[:, :Kq]
        Bq = B[:Kq, :]
        got, rep = ft(O.COL_MAJOR, O.NO_TRANS, O.NO_TRANS, Aq, Bq, alpha, 0.5, Cin)
        assert np.array_equal(got, 0.5 * Cin) and rep.tiles_checked == 0
    # beta = 0: C_in is never read, NaN there does not propagate
    nanC = np.full((M, N), np.nan)
    got, rep = ft(O.COL_MAJOR, O.NO_TRANS, O.NO_TRANS, A, B, 1.0, 0.0, nanC)
    assert np.all(np.isfinite(got)) and rep.detected == 0
    got, rep = ft(O.COL_MAJOR, O.NO_TRANS, O.NO_TRANS, A, B, 0.0, 0.0, nanC)
    assert np.array_equal(got, np.zeros((M, N)))


def test_nonfinite_input_is_reported_not_corrected():
    M, N, K = 8, 8, 8
    A = S.uniform_matrix(2, 0, M, K)
    A[3, 2] = np.inf
    B = S.uniform_matrix(2, 1, K, N)
    _, rep = ft(O.COL_MAJOR, O.NO_TRANS, O.NO_TRANS, A, B, tile=(4, 4))
    assert rep.input_nonfinite == 2 and rep.corrected == 0  # tiles of row block 0


def test_exponent_flip_to_nonfinite_is_corrected():
    """A flip of bit 62 that makes the running sum infinite or huge is still located and
    recomputed (the paper's subtraction cannot restore a non-finite value)."""
    M, N, K = 8, 8, 16
    A = S.uniform_matrix(9, 0, M, K)
    B = S.uniform_matrix(9, 1, K, N)
    clean = plain(O.COL_MAJOR, O.NO_TRANS, O.NO_TRANS, A, B)
    got, rep = ft(O.COL_MAJOR, O.NO_TRANS, O.NO_TRANS, A, B, tile=(8, 8), bk=4,
                  inj=[dict(i=2, j=5, site=O.SITE_ACCUM, bit=62)])
    assert rep.corrected == 1 and np.array_equal(got, clean)


@pytest.mark.filterwarnings("ignore::RuntimeWarning")
def test_infinite_output_is_flagged_against_infinite_threshold():
    """C(3,5) == 1.0 exactly; flipping bit 62 of it gives +inf, which makes the row sum,
    the column sum and both thresholds infinite. It must still be located and recomputed."""
    M = N = K = 8
    A = np.eye(8)
    B = S.randint(51, 0, K * N, 2, 5).reshape(K, N).astype(np.float64)
    B[3, 5] = 1.0
    clean = plain(O.COL_MAJOR, O.NO_TRANS, O.NO_TRANS, A, B)
    assert clean[3, 5] == 1.0 and flip(1.0, 62) == math.inf
    got, rep = ft(O.COL_MAJOR, O.NO_TRANS, O.NO_TRANS, A, B, tile=(8, 8), bk=4,
                  inj=[dict(i=3, j=5, site=O.SITE_OUTPUT, mode=O.MODE_BITFLIP, bit=62)])
    r = rep.records()[0]
    assert (rep.corrected, r.i, r.j) == (1, 3, 5)
    assert math.isinf(r.delta_row) and math.isinf(r.tau_row)
    assert np.array_equal(got, clean)


def test_ragged_tiles_and_injection_in_last_tile():
    M, N, K = 37, 29, 33
    A = S.uniform_matrix(4, 0, M, K)
    B = S.uniform_matrix(4, 1, K, N)
    Cin = S.uniform_matrix(4, 2, M, N)
    clean = plain(O.ROW_MAJOR, O.TRANS, O.NO_TRANS, A, B, 1.5, 0.5, Cin)
    got, rep = ft(O.ROW_MAJOR, O.TRANS, O.NO_TRANS, A, B, 1.5, 0.5, Cin, tile=(16, 8), bk=8,
                  inj=[dict(i=36, j=28, site=O.SITE_ACCUM, bit=55), dict(i=0, j=0, site=O.SITE_ACCUM, bit=51)])
    assert rep.tiles_checked == 3 * 4 and rep.corrected == 2
    assert sorted((r.i, r.j) for r in rep.records()) == [(0, 0), (36, 28)]
    assert np.array_equal(got, clean)


def test_selected_tiles_only():
    M, N, K = 32, 32, 16
    A = S.uniform_matrix(6, 0, M, K)
    B = S.uniform_matrix(6, 1, K, N)
    clean = plain(O.COL_MAJOR, O.NO_TRANS, O.NO_TRANS, A, B)
    got, rep = ft(O.COL_MAJOR, O.NO_TRANS, O.NO_TRANS, A, B, tile=(8, 8), tiles=[0, 5, 15])
    assert rep.tiles_checked == 3
    for t in [0, 5, 15]:
        r0, c0 = (t % 4) * 8, (t // 4) * 8
        assert np.array_equal(got[r0:r0 + 8, c0:c0 + 8], clean[r0:r0 + 8, c0:c0 + 8])
    assert np.all(got[8:16, 0:8] == 0)


def test_seeded_draw_properties():
    M, N, tm, tn = 300, 260, 128, 64
    n_tiles = 3 * 5
    seen_launches = []
    for launch in range(30):
        pts = O.draw_injections(12345, launch, 10, 4, O.SITE_ACCUM, O.MODE_BITFLIP, 40, 62, -20, 4, M, N, tm, tn)
        if not pts:
            continue
        seen_launches.append(launch)
        tiles = {(p["i"] // tm, p["j"] // tn) for p in pts}
        assert len(pts) == 4 and len(tiles) == 4
        for p in pts:
            assert 0 <= p["i"] < M and 0 <= p["j"] < N and 40 <= p["bit"] <= 62 and -20 <= p["rel_log2"] <= 4
        assert pts == O.draw_injections(12345, launch, 10, 4, O.SITE_ACCUM, O.MODE_BITFLIP, 40, 62, -20, 4, M, N, tm, tn)
    assert seen_launches == [5, 15, 25]  # 12345 % 10 == 5
    pts = O.draw_injections(1, 0, 1, 100, O.SITE_ACCUM, O.MODE_BITFLIP, 40, 62, 0, 0, M, N, tm, tn)
    assert len(pts) == n_tiles


# ------------------------------------------------------------------------------------
# ACC32 precision (binary32 accumulation and output): pins on exact integer data
# ------------------------------------------------------------------------------------

def ft32(A_log, B_log, alpha=1.0, beta=0.0, C_log=None, tile=(8, 16), inj=(), precision=O.PREC_ACC32,
         u_acc=O.U_ACC32):
    M, K = A_log.shape
    N = B_log.shape[1]
    a, lda = stored(O.COL_MAJOR, O.TRANS, A_log)   # A k-contiguous
    b, ldb = stored(O.COL_MAJOR, O.NO_TRANS, B_log)
    if C_log is None:
        C_log = np.zeros((M, N))
    c, ldc = c_store(O.COL_MAJOR, C_log)
    out, rep = O.ft_gemm(O.COL_MAJOR, O.TRANS, O.NO_TRANS, M, N, K, alpha, a, lda, b, ldb, beta, c, ldc,
                         tile[0], tile[1], 64, injections=inj, precision=precision, u_acc=u_acc)
    return S.load(out, O.COL_MAJOR, M, N, ldc), rep


def test_acc32_closed_form_is_exact_after_binary32_rounding():
    M, N, K = 9, 13, 20
    i = np.arange(M)[:, None]
    j = np.arange(N)[None, :]
    k = np.arange(K)
    A = (np.arange(M)[:, None] + k[None, :]).astype(np.float64)
    B = (k[:, None] - np.arange(N)[None, :]).astype(np.float64)
    S1 = K * (K - 1) // 2
    S2 = (K - 1) * K * (2 * K - 1) // 6
    expect = (-K * i * j + (i - j) * S1 + S2).astype(np.float64)  # integers < 2^24: exact in binary32
    got, rep = ft32(A, B)
    assert np.array_equal(got, expect) and rep.detected == 0
    a, lda = stored(O.COL_MAJOR, O.NO_TRANS, A)
    b, ldb = stored(O.COL_MAJOR, O.NO_TRANS, B)
    plain32 = O.gemm(O.COL_MAJOR, O.NO_TRANS, O.NO_TRANS, M, N, K, 1.0, a, lda, b, ldb, 0.0, None, M,
                     precision=O.PREC_ACC32)
    assert np.array_equal(S.load(plain32, O.COL_MAJOR, M, N, M), expect)


def test_acc32_binary32_rounding_of_the_output():
    """C is rounded to binary32 once: 1 + 2^-30 becomes 1."""
    A = np.array([[1.0, 2.0 ** -30]])
    B = np.array([[1.0], [1.0]])
    got, _ = ft32(A, B, tile=(1, 1))
    assert got[0, 0] == 1.0


@pytest.mark.filterwarnings("ignore::RuntimeWarning")
def test_acc32_injections_on_integer_data():
    M, N, K = 16, 32, 24
    A = S.randint(71, 0, M * K, -3, 3).reshape(M, K).astype(np.float64)
    B = S.randint(71, 1, K * N, -3, 3).reshape(K, N).astype(np.float64)
    Cin = S.randint(71, 2, M * N, -5, 5).reshape(M, N).astype(np.float64)
    clean, rep = ft32(A, B, 1.0, 1.0, Cin)
    assert rep.detected == 0
    nz = [(i, j) for i in range(M) for j in range(N) if clean[i, j] != 0]
    (i, j) = nz[5]
    # a large output error: located, and subtracting it restores C exactly (exact checksums)
    got, rep = ft32(A, B, 1.0, 1.0, Cin, inj=[dict(i=i, j=j, site=O.SITE_OUTPUT, mode=O.MODE_ADD_REL, rel_log2=3,
                                                   sign=1)])
    assert (rep.corrected, rep.records()[0].i, rep.records()[0].j) == (1, i, j)
    assert rep.records()[0].delta_row == 8.0 * abs(clean[i, j])
    assert np.array_equal(got, clean)
    # an error far below the threshold is not detected
    got, rep = ft32(A, B, 1.0, 1.0, Cin, inj=[dict(i=i, j=j, site=O.SITE_OUTPUT, mode=O.MODE_ADD_REL, rel_log2=-60,
                                                   sign=1)])
    assert rep.detected == 0
    # an output flipped to infinity: recovered from the row checksum, exactly
    ones = [(i, j) for (i, j) in nz if abs(clean[i, j]) == 1.0]
    if ones:
        (i1, j1) = ones[0]
        got, rep = ft32(A, B, 1.0, 1.0, Cin, inj=[dict(i=i1, j=j1, site=O.SITE_OUTPUT, mode=O.MODE_BITFLIP, bit=30)])
        assert rep.corrected == 1 and math.isinf(rep.records()[0].value_before)
        assert np.array_equal(got, clean)
    # an accumulator flip of the binary32 sum (bit 29: exponent)
    got, rep = ft32(A, B, 1.0, 1.0, Cin, inj=[dict(i=i, j=j, site=O.SITE_ACCUM, mode=O.MODE_BITFLIP, bit=29)])
    assert (rep.corrected, rep.records()[0].i, rep.records()[0].j) == (1, i, j)
    assert np.array_equal(got, clean)
    # a fault in the predicted row checksum: checksum-only, C kept
    got, rep = ft32(A, B, 1.0, 1.0, Cin, inj=[dict(i=3, j=0, site=O.SITE_CHECKSUM, mode=O.MODE_ADD_REL, rel_log2=2,
                                                   sign=1)])
    assert (rep.checksum_only, rep.corrected) == (1, 0) and np.array_equal(got, clean)
    # two errors in one tile: uncorrectable
    (i2, j2) = [(a, b) for (a, b) in nz if a // 8 == i // 8 and b // 16 == j // 16 and a != i and b != j][0]
    _, rep = ft32(A, B, 1.0, 1.0, Cin, inj=[dict(i=i, j=j, site=O.SITE_OUTPUT, mode=O.MODE_ADD_REL, rel_log2=3),
                                            dict(i=i2, j=j2, site=O.SITE_OUTPUT, mode=O.MODE_ADD_REL, rel_log2=3)])
    assert rep.uncorrectable == 1


def test_acc32_clean_soak_bf16_like_values():
    """bfloat16-exact operands, rows scaled by 2^u: no false alarm at K = 512."""
    for seed in range(4):
        M, N, K = 32, 64, 512
        A = S.bf16_bits_to_f64(S.to_bf16_bits(S.normal_matrix(seed, 0, M, K) * S.pow2_row_scales(seed, 5, M)[:, None]))
        B = S.bf16_bits_to_f64(S.to_bf16_bits(S.normal_matrix(seed, 1, K, N)))
        _, rep = ft32(A, B, 1.0, 0.0, None, tile=(16, 32))
        assert rep.detected == 0


def _extreme_accumulation(terms, u, direction):
    """The sum of `terms` in ascending order with every step rounded at the extreme that a
    unit roundoff u allows (standard model fl(s + x) = (s + x)(1 + d), |d| <= u), all in
    one direction: d = -u (direction -1) or d = +u (direction +1). Binary64 carries the
    model; its own rounding (2^-53 per step) is far below u."""
    s = 0.0
    for x in terms:
        s = (s + x) * (1.0 + direction * u)
    return s


@pytest.mark.parametrize("precision,u_acc", [(O.PREC_ACC32, 2.0 ** -23), (O.PREC_ACC32_E4M3, 2.0 ** -22)])
def test_acc32_row_threshold_covers_the_extreme_accumulations(precision, u_acc):
    """The ACC32 row threshold claims to bound the row mismatch of every tensor-core run in
    which each binary32 accumulation step errs by at most u_acc in either direction: the
    K-term accumulations of the tile's outputs C(i, j) (the reference side) and those of A
    times the pieces of B e that the checksum columns hold (the prediction side). This
    builds the worst such run by hand: outputs accumulated with every step rounded down,
    the checksum products with every step rounded up, on data whose partial sums stay at
    their final size from the first product on (A(i, 0) = 1, later A(i, k) = 2^-16, B all
    ones). Here B e = 8 exactly, so each of its pieces (three bfloat16 or eight e4m3) is
    8 or 0. The mismatch then uses most of the threshold: it must stay within it, and it
    is well above the 0.44 to 0.5 of it that a threshold without the prediction side's
    term would be."""
    M, N, K = 1, 8, 2048
    A = np.full((M, K), 2.0 ** -16)
    A[:, 0] = 1.0
    B = np.ones((K, N))
    # the reference side: sum_j C(i, j), each C(i, j) an extreme accumulation of its products
    C = [_extreme_accumulation(A[0] * B[:, j], u_acc, -1) for j in range(N)]
    ref = math.fsum(C)
    # the prediction side: B e = 8 in every k, held as one nonzero piece (8) in either format
    Be = B.sum(axis=1)
    assert np.all(Be == 8.0)
    pred = _extreme_accumulation(A[0] * Be, u_acc, +1)
    delta = ref - pred
    # the oracle's threshold for row 0, read from the record of a flagged row (a checksum
    # fault far above any threshold; the threshold does not depend on it)
    _, rep = ft32(A, B, tile=(4, N), precision=precision, u_acc=u_acc,
                  inj=[dict(i=0, j=0, site=O.SITE_CHECKSUM, mode=O.MODE_ADD_REL, rel_log2=30, sign=1)])
    (r,) = rep.records()
    assert r.i == 0 and r.kind == O.KIND_CHECKSUM_ONLY
    tau = r.tau_row
    assert abs(delta) <= tau
    # the data is adversarial enough to need every term of it (0.97 of the threshold with
    # the bfloat16 pieces, 0.87 with the e4m3 pieces, whose magnitude bound is looser)
    assert abs(delta) > 0.8 * tau
    # and a clean run of the oracle itself never flags
    _, rep0 = ft32(A, B, tile=(4, N), precision=precision, u_acc=u_acc)
    assert rep0.detected == 0


# ------------------------------------------------------------------------------------
# Sampled rows of the plain product (the reference of the full-size GPU tests)
# ------------------------------------------------------------------------------------

@pytest.mark.parametrize("layout,ta,tb", COMBOS)
def test_gemm_rows_equals_the_full_product_row_by_row(layout, ta, tb):
    """oracle_gemm_rows gives, bit for bit, the rows of oracle_gemm, whatever rows are
    asked for (repeated, unordered, the last one), with alpha, beta and C_in."""
    M, N, K = 23, 17, 31
    A = S.uniform_matrix(61, 0, M, K)
    B = S.uniform_matrix(61, 1, K, N)
    Cin = S.uniform_matrix(61, 2, M, N)
    a, lda = stored(layout, ta, A)
    b, ldb = stored(layout, tb, B)
    c, ldc = c_store(layout, Cin)
    full = S.load(O.gemm(layout, ta, tb, M, N, K, 1.5, a, lda, b, ldb, 0.5, c, ldc), layout, M, N, ldc)
    rows = np.array([22, 0, 7, 7, 13])
    got = O.gemm_rows(layout, ta, tb, M, N, K, 1.5, a, lda, b, ldb, 0.5, c, ldc, rows)
    assert np.array_equal(got, full[rows, :])
    # quick returns: alpha = 0 gives beta C_in; K = 0 likewise
    got0 = O.gemm_rows(layout, ta, tb, M, N, K, 0.0, a, lda, b, ldb, 0.5, c, ldc, rows)
    assert np.array_equal(got0, 0.5 * Cin[rows, :])
    got_k0 = O.gemm_rows(layout, ta, tb, M, N, 0, 1.5, a, lda, b, ldb, -2.0, c, ldc, rows)
    assert np.array_equal(got_k0, -2.0 * Cin[rows, :])


@pytest.mark.parametrize("layout,ta,tb", COMBOS)
def test_gemm_rows_closed_form_linear_operands(layout, ta, tb):
    """A(i,k) = i + k, B(k,j) = k + j: row i of C is K i j + (i + j) S1 + S2 exactly, and
    with alpha = 0.5, beta = -2, C_in(i,j) = i - 2 j, 0.5 of that minus 2 C_in."""
    M, N, K = 40, 9, 57
    k = np.arange(K)
    A = (np.arange(M)[:, None] + k[None, :]).astype(np.float64)
    B = (k[:, None] + np.arange(N)[None, :]).astype(np.float64)
    i = np.arange(M)[:, None]
    j = np.arange(N)[None, :]
    S1 = K * (K - 1) // 2
    S2 = (K - 1) * K * (2 * K - 1) // 6
    expect = (K * i * j + (i + j) * S1 + S2).astype(np.float64)
    Cin = (i - 2 * j).astype(np.float64)
    a, lda = stored(layout, ta, A)
    b, ldb = stored(layout, tb, B)
    c, ldc = c_store(layout, Cin)
    rows = np.array([0, 39, 5])
    got = O.gemm_rows(layout, ta, tb, M, N, K, 0.5, a, lda, b, ldb, -2.0, c, ldc, rows)
    assert np.array_equal(got, (0.5 * expect - 2.0 * Cin)[rows, :])


# ------------------------------------------------------------------------------------
# The generator behind the seeded draw and the inputs, pinned to its published outputs
# ------------------------------------------------------------------------------------

def _golden_splitmix():
    path = os.path.join(os.path.dirname(__file__), "golden", "splitmix64_state0.txt")
    vals = [int(line, 16) for line in open(path) if line.strip() and not line.startswith("#")]
    assert len(vals) == 3
    return vals


def test_splitmix64_matches_published_outputs():
    g = _golden_splitmix()
    # synth: counter form, element idx of (seed 0, matrix 0) is output idx + 1 of state 0
    assert [int(x) for x in S.splitmix64(0, 0, np.arange(3, dtype=np.uint64))] == g
    # oracle draw, seed 0, launch 0 (state 0): the first point's tile, row and column come
    # from the first three outputs (tile t = out0 mod ntiles, numbered t = tile_row +
    # tile_col * n_tile_rows; offsets out1 mod rows, out2 mod columns of that tile)
    M = N = 1000
    tm = tn = 100
    (pt,) = O.draw_injections(0, 0, 1, 1, O.SITE_ACCUM, O.MODE_BITFLIP, 40, 62, 0, 0, M, N, tm, tn)
    t = g[0] % 100
    assert (pt["i"], pt["j"]) == ((t % 10) * tm + g[1] % tm, (t // 10) * tn + g[2] % tn)


# ------------------------------------------------------------------------------------
# Online verification every kc products (Section V.A's rank-kc steps)
# ------------------------------------------------------------------------------------

def _midk(A, B, kc, inj=(), tile=(4, 5), bk=2, alpha=1.0, beta=0.0, C=None):
    M, K = A.shape
    N = B.shape[1]
    a, lda = stored(O.COL_MAJOR, O.NO_TRANS, A)
    b, ldb = stored(O.COL_MAJOR, O.NO_TRANS, B)
    c, ldc = c_store(O.COL_MAJOR, np.zeros((M, N)) if C is None else C)
    out, rep = O.ft_gemm(O.COL_MAJOR, O.NO_TRANS, O.NO_TRANS, M, N, K, alpha, a, lda, b, ldb, beta, c, ldc,
                         tile[0], tile[1], bk, injections=inj, kc=kc)
    return S.load(out, O.COL_MAJOR, M, N, ldc), rep


def test_midk_two_faults_in_one_tile_both_corrected_bitwise():
    """Brute force on 4 x 5 x 12 (one tile, bk = 2, checks after 4 and 8 products): two
    accumulator flips in the same tile, in different rank-4 steps, are each located and
    corrected at the check that follows them; C equals the fault-free C bit for bit.
    Without online checks the same pair is uncorrectable."""
    A = S.uniform_matrix(81, 0, 4, 12)
    B = S.uniform_matrix(81, 1, 12, 5)
    clean = A @ B  # reference only for the final comparison below
    ref, rep0 = _midk(A, B, 4)
    assert rep0.detected == 0
    plain, _ = _midk(A, B, 0)
    assert np.array_equal(ref, plain)  # the checked steps change nothing on a clean run
    assert np.max(np.abs(ref - clean)) <= 2 * 12 * 2.0 ** -53 * np.max(np.abs(A) @ np.abs(B))
    hits = 0
    for (i1, j1, i2, j2) in [(0, 0, 3, 4), (1, 2, 2, 3), (3, 1, 0, 4)]:
        for bit in (44, 52, 60, 62):
            inj = [dict(i=i1, j=j1, site=O.SITE_ACCUM, mode=O.MODE_BITFLIP, bit=bit, kt=1),
                   dict(i=i2, j=j2, site=O.SITE_ACCUM, mode=O.MODE_BITFLIP, bit=bit, kt=3)]
            got, rep = _midk(A, B, 4, inj)
            recs = sorted((r.i, r.j, r.kind) for r in rep.records())
            if rep.corrected == 2:
                hits += 1
                assert recs == sorted([(i1, j1, O.KIND_CORRECTED), (i2, j2, O.KIND_CORRECTED)])
                assert np.array_equal(got, ref)
            _, rep_end = _midk(A, B, 0, inj)
            if rep.corrected == 2:
                assert rep_end.uncorrectable == 1 and rep_end.corrected == 0
    assert hits >= 10  # a flip is undetectable only when the partial sum is tiny


def test_midk_exact_delta_on_integer_data():
    """Integer operands: partial checksums are exact, so at the first check after the flip
    delta_row = delta_col = the flip's exact error, and the record carries it."""
    A = (np.arange(4)[:, None] + np.arange(8)[None, :]).astype(np.float64)
    B = (np.arange(8)[:, None] - np.arange(5)[None, :]).astype(np.float64)
    i, j = 2, 3
    acc_after_2 = sum(A[i, k] * B[k, j] for k in range(2))  # flip lands after kt * bk = 2 products
    bit = 55
    flipped = struct.unpack("<d", struct.pack("<Q", struct.unpack("<Q", struct.pack("<d", acc_after_2))[0] ^ (1 << bit)))[0]
    e = flipped - acc_after_2
    got, rep = _midk(A, B, 4, [dict(i=i, j=j, site=O.SITE_ACCUM, mode=O.MODE_BITFLIP, bit=bit, kt=1)])
    (r,) = rep.records()
    assert (r.i, r.j, r.kind) == (i, j, O.KIND_CORRECTED)
    assert r.delta_row == e and r.delta_col == e
    assert np.array_equal(got, A @ B)


def test_midk_clean_runs_never_flag():
    for seed in range(6):
        M, N, K = 40, 50, 96
        A = S.normal_matrix(seed, 0, M, K) * S.pow2_row_scales(seed, 3, M)[:, None]
        B = S.normal_matrix(seed, 1, K, N)
        _, rep = _midk(A, B, 16, tile=(16, 16), bk=8, alpha=1.5, beta=0.5, C=S.normal_matrix(seed, 2, M, N))
        assert rep.detected == 0


# ------------------------------------------------------------------------------------
# Triangular solve (the definition behind FT-DTRSM): plain substitution
# ------------------------------------------------------------------------------------

def test_trsm_identity_diagonal_and_exact_integer_solutions():
    W = S.uniform_matrix(61, 0, 7, 5)
    for lower in (True, False):
        assert np.array_equal(O.trsm_left(np.eye(7), W, lower), W)
        d = np.ldexp(1.0, S.randint(61, 1, 7, -3, 3).astype(int))
        assert np.array_equal(O.trsm_left(np.diag(d), W, lower), W / d[:, None])
    # unit lower bidiagonal with -1 below the diagonal: x_r = w_r + x_{r-1}, exact on integers
    n = 9
    T = np.eye(n) - np.eye(n, k=-1)
    Wi = S.randint(61, 2, n * 3, -5, 5).reshape(n, 3).astype(np.float64)
    assert np.array_equal(O.trsm_left(T, Wi, True), np.cumsum(Wi, axis=0))
    assert np.array_equal(O.trsm_left(T.T, Wi, False), np.cumsum(Wi[::-1], axis=0)[::-1])


def test_trsm_reads_only_its_triangle_and_has_small_residual():
    n = 40
    R = S.uniform_matrix(62, 0, n, n)
    T = np.tril(R) + n * np.eye(n)
    W = S.uniform_matrix(62, 1, n, 6)
    junk = T + np.triu(np.full((n, n), np.nan), 1)  # the unread triangle holds NaN
    X = O.trsm_left(junk, W, True)
    # componentwise backward error of substitution: |T X - W| <= gamma_n |T| |X|
    g = n * 2.0 ** -53 / (1 - n * 2.0 ** -53)
    assert np.all(np.abs(T @ X - W) <= 2 * g * (np.abs(T) @ np.abs(X)) + 1e-300)
    Xu = O.trsm_left(T.T + np.tril(np.full((n, n), np.nan), -1), W, False)
    assert np.all(np.abs(T.T @ Xu - W) <= 2 * g * (np.abs(T.T) @ np.abs(Xu)) + 1e-300)
