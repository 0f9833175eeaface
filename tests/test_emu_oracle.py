"""Pins for the oracle of the emulated FP64 GEMM (emu_oracle.c): binary64 operands as
integer slices, exact group products and exact integer checksums (Section II.A's relations
holding exactly), located and corrected by recomputation (Sections V.A, VI.C).

Each test checks the oracle against something its code does not contain: exact rational
arithmetic (fractions) for the slicing, the digits and the product's error bound; Python's
own correctly rounded integer-to-float conversion; closed-form integer products; a library
matmul; and, for injections, the fault-free run of the same problem.
"""
import math
import random
from fractions import Fraction

import numpy as np
import pytest

import oracle as O
import synth as S

U = 2.0 ** -53
COMBOS = [(l, a, b) for l in (O.COL_MAJOR, O.ROW_MAJOR) for a in (O.NO_TRANS, O.TRANS)
          for b in (O.NO_TRANS, O.TRANS)]


def stored(layout, trans, logical, pad=2):
    X = logical if trans == O.NO_TRANS else logical.T
    ld = (X.shape[0] if layout == O.COL_MAJOR else X.shape[1]) + pad
    return S.store(X, layout, ld=max(1, ld))


def emu(A, B, alpha=1.0, beta=0.0, Cin=None, layout=O.COL_MAJOR, ta=O.NO_TRANS, tb=O.NO_TRANS, slices=14,
        tile=(8, 12), inj=(), tiles=None):
    M, K = A.shape
    N = B.shape[1]
    a, lda = stored(layout, ta, A)
    b, ldb = stored(layout, tb, B)
    Cl = np.zeros((M, N)) if Cin is None else Cin
    c, ldc = S.store(Cl, layout, ld=(M if layout == O.COL_MAJOR else N) + 1)
    out, rep = O.emu_gemm(layout, ta, tb, M, N, K, alpha, a, lda, b, ldb, beta, c, ldc, slices=slices,
                          injections=inj, tiles=tiles, tile_m=tile[0], tile_n=tile[1])
    return S.load(out, layout, M, N, ldc), rep


def summary(rep):
    return (int(rep.tiles_checked), int(rep.detected), int(rep.corrected), int(rep.uncorrectable),
            int(rep.checksum_only), int(rep.input_nonfinite))


# ------------------------------------------------------------------------------------
# Slices and digits, against exact rationals
# ------------------------------------------------------------------------------------

def _sample_x(n, seed):
    rnd = random.Random(seed)
    xs = [0.0, 0.5, -0.5, 1 - 2 ** -53, -(1 - 2 ** -53), 15.5 / 16, -15.5 / 16, 2 ** -60, 0.5 + 2 ** -53,
          1 / 32, 3 / 32, 17 / 256]
    while len(xs) < n:
        e = -rnd.randint(1, 70)
        xs.append(rnd.choice([-1, 1]) * rnd.random() * 2.0 ** (e + 1))
    return [x for x in xs if abs(x) < 1]


@pytest.mark.parametrize("s", [1, 4, 9, 14])
def test_slices_are_small_integers_that_rebuild_x(s):
    """|a_0| <= 16, |a_p| <= 8 (E4M3 values), and |x - sum_p a_p 16^-(p+1)| <= 16^-s / 2,
    exactly; with 24 slices every x of magnitude >= 2^-40 is rebuilt exactly."""
    for x in _sample_x(400, s):
        a = O.emu_split(x, s)
        assert abs(a[0]) <= 16 and all(abs(v) <= 8 for v in a[1:]), (x, a)
        rebuilt = sum(Fraction(v, 16 ** (q + 1)) for q, v in enumerate(a))
        assert abs(Fraction(x) - rebuilt) <= Fraction(1, 2 * 16 ** s), (x, a)
        if abs(x) >= 2.0 ** -40:
            a24 = O.emu_split(x, 24)
            assert sum(Fraction(v, 16 ** (q + 1)) for q, v in enumerate(a24)) == Fraction(x)


def test_checksum_digits_rebuild_the_integer():
    """Four base-16 digits in [-8, 8] whose weighted sum is v, for every v the checksum of a
    248-column tile can take (|v| <= 248 * 16)."""
    for v in range(-3968, 3969):
        d = O.emu_digits(v)
        assert all(abs(x) <= 8 for x in d) and sum(x * 16 ** t for t, x in enumerate(d)) == v, (v, d)


def test_i128_to_double_is_correctly_rounded():
    """The oracle's conversion of 128-bit integers equals Python's float(int), which rounds
    to nearest with ties to even: ties, carries into the next binade, negatives, extremes."""
    rnd = random.Random(5)
    vals = [0, 1, -1, 2 ** 53, 2 ** 53 + 1, 2 ** 53 + 2, 2 ** 53 + 3, 2 ** 54 + 2, 2 ** 54 + 6, 2 ** 80 + 2 ** 27,
            2 ** 80 + 2 ** 27 + 1, (2 ** 53 - 1) * 2 ** 30 + 2 ** 29, 2 ** 127 - 1, -(2 ** 127), -(2 ** 64) - 1]
    for _ in range(3000):
        nb = rnd.randint(1, 126)
        v = rnd.getrandbits(nb)
        if rnd.random() < 0.3:  # a value with a tie or near-tie below bit 53
            v |= 1 << max(0, nb - 54)
        vals.append(v if rnd.random() < 0.5 else -v)
    for v in vals:
        assert O.emu_i128_to_double(v) == float(v), v


# ------------------------------------------------------------------------------------
# The product
# ------------------------------------------------------------------------------------

@pytest.mark.parametrize("layout,ta,tb", COMBOS)
def test_small_integer_operands_give_the_exact_product(layout, ta, tb):
    """Integer operands of magnitude < 16 are held exactly by the slices, so C equals the
    integer product exactly, with dyadic alpha and beta and an integer C_in."""
    M, N, K = 19, 29, 23
    i = np.arange(M)[:, None]
    j = np.arange(N)[None, :]
    k = np.arange(K)
    A = ((i + 2 * k[None, :]) % 13 - 6).astype(np.float64)
    B = ((3 * k[:, None] + j) % 11 - 5).astype(np.float64)
    Cin = (i - 2 * j).astype(np.float64)
    exact = (A.astype(np.int64) @ B.astype(np.int64)).astype(np.float64)
    C, rep = emu(A, B, 0.5, -2.0, Cin, layout, ta, tb)
    assert np.array_equal(C, 0.5 * exact - 2.0 * Cin)
    assert summary(rep)[1:] == (0, 0, 0, 0, 0)


@pytest.mark.parametrize("s", [6, 10, 14])
def test_error_within_the_slicing_bound(s):
    """|C - C_exact| <= |alpha| 2^(e_i + f_j) K 16^-s (s + 3) / 4 + 3 u |C_exact| elementwise,
    C_exact the exact rational product; normalised by max|A| max|B| K this is at most
    (s + 3) 16^-s + 3 u."""
    M, N, K = 7, 6, 9
    A = S.uniform_matrix(3 + s, 0, M, K) * 2.0 ** np.arange(M)[:, None]
    B = S.uniform_matrix(3 + s, 1, K, N) * 2.0 ** -np.arange(N)[None, :]
    C, _ = emu(A, B, slices=s, tile=(M, N))
    e = np.array([math.frexp(np.abs(A[r]).max())[1] for r in range(M)])
    f = np.array([math.frexp(np.abs(B[:, c]).max())[1] for c in range(N)])
    for r in range(M):
        for c in range(N):
            exact = sum(Fraction(A[r, q]) * Fraction(B[q, c]) for q in range(K))
            bound = Fraction(2.0 ** (e[r] + f[c])) * K * Fraction(s + 3, 4 * 16 ** s) + Fraction(3 * U) * abs(exact)
            assert abs(Fraction(C[r, c]) - exact) <= bound, (r, c)
    exact_all = A @ B
    if s == 14:
        assert np.abs(C - exact_all).max() / (np.abs(A).max() * np.abs(B).max() * K) <= 1e-15


def test_library_matmul_agrees_within_both_bounds():
    M, N, K = 40, 33, 300
    A = S.uniform_matrix(8, 0, M, K)
    B = S.uniform_matrix(8, 1, K, N)
    Cin = S.uniform_matrix(8, 2, M, N)
    C, rep = emu(A, B, 1.5, 0.5, Cin, tile=(16, 16))
    ref = 1.5 * (A @ B) + 0.5 * Cin
    g = K * U / (1 - K * U)
    bound = 1.5 * (2 * g * (np.abs(A) @ np.abs(B)) + 4 * K * 17 * 16.0 ** -14) + 4 * U * (np.abs(ref) + 1)
    assert np.all(np.abs(C - ref) <= bound)
    assert summary(rep)[1:] == (0, 0, 0, 0, 0)


@pytest.mark.parametrize("layout", [O.COL_MAJOR, O.ROW_MAJOR])
def test_clean_runs_never_flag(layout):
    """Rows and columns scaled by 2^u, u in [-20, 20], beta != 0, ragged tiles: no flag (the
    integer checks are exact; the binary64 stage's threshold bounds its rounding)."""
    for seed in range(3):
        M, N, K = 37, 41, 64
        A = S.normal_matrix(seed, 0, M, K) * S.pow2_row_scales(seed, 5, M, -20, 20)[:, None]
        B = S.normal_matrix(seed, 1, K, N) * S.pow2_row_scales(seed, 6, N, -20, 20)[None, :]
        Cin = S.normal_matrix(seed, 2, M, N)
        _, rep = emu(A, B, -0.75, 1.25, Cin, layout, tile=(8, 12))
        fm, fn = (M, N) if layout == O.COL_MAJOR else (N, M)   # the column-major frame
        assert summary(rep)[1:] == (0, 0, 0, 0, 0) and rep.tiles_checked == -(-fm // 8) * -(-fn // 12)


# ------------------------------------------------------------------------------------
# Injected errors against the fault-free run
# ------------------------------------------------------------------------------------

def test_every_accumulator_flip_is_detected_and_c_restored_bitwise():
    """Brute force: every element, every group and bits across the binary32 pattern of a
    3 x 4 x 5 product in 2 x 3 tiles. The exact check flags every flip (no threshold to
    hide under); the stored C equals the fault-free C bit for bit; a flip that changed C is
    located at its element, one that did not is checksum-only."""
    M, N, K = 3, 4, 5
    A = S.uniform_matrix(21, 0, M, K)
    B = S.uniform_matrix(21, 1, K, N)
    s = 6
    clean, rep0 = emu(A, B, slices=s, tile=(2, 3))
    assert rep0.detected == 0
    for i in range(M):
        for j in range(N):
            for g in range(s):
                for bit in (0, 5, 13, 22, 23, 24, 27, 30, 31):
                    pt = dict(i=i, j=j, site=O.SITE_ACCUM, mode=O.MODE_BITFLIP, bit=bit, kt=g)
                    C, rep = emu(A, B, slices=s, tile=(2, 3), inj=[pt])
                    assert rep.detected == 1, (i, j, g, bit)
                    assert np.array_equal(C.view(np.uint64), clean.view(np.uint64)), (i, j, g, bit)
                    recs = [(r.i, r.j, r.kind) for r in rep.records()]
                    if rep.corrected:
                        assert recs == [(i, j, O.KIND_CORRECTED)]
                    else:
                        assert rep.checksum_only == 1 and recs == [(i, -1, O.KIND_CHECKSUM_ONLY)]


@pytest.mark.parametrize("layout", [O.COL_MAJOR, O.ROW_MAJOR])
def test_output_and_checksum_faults(layout):
    M, N, K = 20, 30, 16
    A = S.uniform_matrix(22, 0, M, K)
    B = S.uniform_matrix(22, 1, K, N)
    Cin = S.uniform_matrix(22, 2, M, N)
    clean, _ = emu(A, B, 1.5, 0.5, Cin, layout, tile=(8, 12))
    # an output error above the binary64 stage's threshold: located there, C restored bitwise
    for rel, bit in ((-20, None), (3, None), (None, 62), (None, 52)):
        pt = (dict(i=13, j=17, site=O.SITE_OUTPUT, mode=O.MODE_ADD_REL, rel_log2=rel, sign=-1) if bit is None else
              dict(i=13, j=17, site=O.SITE_OUTPUT, mode=O.MODE_BITFLIP, bit=bit))
        C, rep = emu(A, B, 1.5, 0.5, Cin, layout, tile=(8, 12), inj=[pt])
        assert summary(rep)[1:] == (1, 1, 0, 0, 0) and [(r.i, r.j) for r in rep.records()] == [(13, 17)], pt
        assert np.array_equal(C.view(np.uint64), clean.view(np.uint64))
    # far below it: undetected, and the error stays where it was put
    pt = dict(i=13, j=17, site=O.SITE_OUTPUT, mode=O.MODE_ADD_REL, rel_log2=-70, sign=1)
    C, rep = emu(A, B, 1.5, 0.5, Cin, layout, tile=(8, 12), inj=[pt])
    assert rep.detected == 0
    # a fault in a predicted checksum: checksum-only, C kept
    pt = dict(i=5, j=4, site=O.SITE_CHECKSUM, mode=O.MODE_ADD_REL, rel_log2=-40, sign=1)
    C, rep = emu(A, B, 1.5, 0.5, Cin, layout, tile=(8, 12), inj=[pt])
    assert summary(rep)[1:] == (1, 0, 0, 1, 0) and np.array_equal(C, clean)


def test_several_errors_in_a_tile():
    """Errors in up to four rows of one tile are all located and corrected (each flagged row
    is recomputed); a fifth row makes the tile uncorrectable, C left as computed; errors in
    different tiles are corrected independently."""
    M, N, K = 16, 24, 8
    A = S.uniform_matrix(23, 0, M, K)
    B = S.uniform_matrix(23, 1, K, N)
    clean, _ = emu(A, B, tile=(8, 12))
    four = [dict(i=r, j=(3 * r) % 12, site=O.SITE_ACCUM, mode=O.MODE_BITFLIP, bit=27, kt=0) for r in range(4)]
    C, rep = emu(A, B, tile=(8, 12), inj=four)
    assert summary(rep)[1:] == (1, 1, 0, 0, 0)
    assert sorted((r.i, r.j) for r in rep.records()) == sorted((p["i"], p["j"]) for p in four)
    assert np.array_equal(C, clean)
    five = four + [dict(i=6, j=1, site=O.SITE_ACCUM, mode=O.MODE_BITFLIP, bit=27, kt=0)]
    C, rep = emu(A, B, tile=(8, 12), inj=five)
    assert summary(rep)[1:] == (1, 0, 1, 0, 0)
    assert not np.array_equal(C, clean)
    spread = [dict(i=1, j=2, site=O.SITE_ACCUM, mode=O.MODE_BITFLIP, bit=27, kt=1),
              dict(i=10, j=20, site=O.SITE_OUTPUT, mode=O.MODE_ADD_REL, rel_log2=2, sign=1)]
    C, rep = emu(A, B, tile=(8, 12), inj=spread)
    assert summary(rep)[1:] == (2, 2, 0, 0, 0) and np.array_equal(C, clean)


def test_nonfinite_inputs_quick_returns_and_limits():
    M, N, K = 10, 14, 6
    A = S.uniform_matrix(24, 0, M, K)
    B = S.uniform_matrix(24, 1, K, N)
    Cin = S.uniform_matrix(24, 2, M, N)
    A2 = A.copy()
    A2[3, 2] = np.inf
    C, rep = emu(A2, B, tile=(8, 12))
    assert np.all(np.isnan(C[3])) and np.all(np.isfinite(np.delete(C, 3, axis=0)))
    assert rep.input_nonfinite == 2 and rep.detected == 0  # the two tiles of row block 0
    # alpha = 0 and K = 0: C = beta C_in, no checks; beta = 0 never reads C_in
    C, rep = emu(A, B, 0.0, 2.0, Cin)
    assert np.array_equal(C, 2.0 * Cin) and rep.tiles_checked == 0
    Cnan = np.full((M, N), np.nan)
    C, rep = emu(A, B, 1.0, 0.0, Cnan)
    assert np.all(np.isfinite(C)) and rep.detected == 0
    # K beyond the exact range of the group accumulators is refused
    assert O.emu_max_k(14) == 16384 and O.emu_max_k(6) == 32768
    with pytest.raises(ValueError):
        emu(np.ones((2, 16385)), np.ones((16385, 2)))


def test_selected_tiles_match_the_full_run():
    M, N, K = 30, 50, 12
    A = S.uniform_matrix(25, 0, M, K)
    B = S.uniform_matrix(25, 1, K, N)
    for layout in (O.COL_MAJOR, O.ROW_MAJOR):
        full, _ = emu(A, B, layout=layout, tile=(8, 12))
        tr, tc = (8, 12) if layout == O.COL_MAJOR else (12, 8)   # caller's tile shape
        n_tr = -(-M // tr)
        t = 2 + 1 * n_tr
        part, rep = emu(A, B, layout=layout, tile=(8, 12), tiles=[t])
        rows = slice(2 * tr, min(M, 3 * tr))
        cols = slice(1 * tc, min(N, 2 * tc))
        assert rep.tiles_checked == 1 and np.array_equal(part[rows, cols], full[rows, cols])
