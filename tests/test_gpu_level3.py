"""FT-DSYMM and FT-DTRMM through the C ABI against the CPU oracle.

By definition DSYMM is the GEMM C = alpha S B + beta C (or alpha B S + beta C) with S the
symmetric matrix whose `uplo` triangle is stored, and DTRMM is B = alpha op(A) B (or
alpha B op(A)) with op(A) triangular (zeros outside the triangle, ones on a unit
diagonal). The oracle runs its protected GEMM on those matrices, formed here from the
definitions; the library reads only the stored triangle (the other one, and a unit
diagonal, hold NaN in these tests). Bar: FP64 values within 1e-15 normalised, the same
tiles checked, and injected errors detected, located and corrected as the oracle does.
"""
import itertools

import numpy as np
import pytest

import oracle as O
import synth as S
from tests.helpers import record_set, report_summary

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2104_00897_gb300 as fb  # noqa: E402


@pytest.fixture(autouse=True)
def _fresh_injection():
    fb.ftblas_set_injection(None)
    yield
    fb.ftblas_set_injection(None)


def dev(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def tile(layout, M, N, K):
    return fb.ftblas_verification_tile(layout, fb.R_64F, M, N, K)


def norm_err(got, ref, A, B, K):
    den = max(np.abs(A).max() * np.abs(B).max() * max(K, 1), 1e-300)
    return float(np.abs(got - ref).max() / den)


def oracle_gemm(layout, M, N, K, alpha, A, B, beta, C, inj=()):
    a, lda = S.store(A, layout)
    b, ldb = S.store(B, layout)
    c, ldc = S.store(C, layout)
    tr, tc, bk = tile(layout, M, N, K)
    out, rep = O.ft_gemm(layout, O.NO_TRANS, O.NO_TRANS, M, N, K, alpha, a, lda, b, ldb, beta, c, ldc, tr, tc, bk,
                         injections=inj)
    return S.load(out, layout, M, N, ldc), rep


def stored_triangle(X, upper, nan_diag=False):
    """X with the other triangle (and optionally the diagonal) replaced by NaN."""
    n = X.shape[0]
    r, c = np.indices((n, n))
    keep = (r <= c) if upper else (r >= c)
    Y = np.where(keep, X, np.nan)
    if nan_diag:
        Y[np.arange(n), np.arange(n)] = np.nan
    return Y


@pytest.mark.parametrize("layout,side,uplo", list(itertools.product((O.COL_MAJOR, O.ROW_MAJOR), (fb.LEFT, fb.RIGHT),
                                                                      (fb.UPPER, fb.LOWER))))
def test_dsymm_matches_oracle(layout, side, uplo):
    M, N = 300, 200
    dim = M if side == fb.LEFT else N
    X = S.uniform_matrix(51, 0, dim, dim)
    Sym = X + X.T
    B = S.uniform_matrix(51, 1, M, N)
    Cin = S.uniform_matrix(51, 2, M, N)
    alpha, beta = 1.5, -0.5
    a, lda = S.store(stored_triangle(Sym, uplo == fb.UPPER), layout, ld=dim + 3)
    b, ldb = S.store(B, layout)
    c, ldc = S.store(Cin, layout)
    dA, dB, dC = dev(a), dev(b), dev(c)
    pts = [dict(i=150, j=60, site=fb.SITE_OUTPUT, mode=fb.MODE_ADD_REL, rel_log2=3, sign=1)]
    for inj in ((), pts):
        dC.copy_(dev(c))
        fb.ftblas_set_injection(fb.make_injection(fixed=inj) if inj else None)
        rep = fb.new_report()
        fb.check(fb.ftblas_dsymm(layout, side, uplo, M, N, alpha, dA.data_ptr(), lda, dB.data_ptr(), ldb, beta,
                                 dC.data_ptr(), ldc, torch.cuda.current_stream().cuda_stream, rep.data_ptr()))
        torch.cuda.synchronize()
        got = S.load(dC.cpu().numpy(), layout, M, N, ldc)
        r = fb.report_from_device(rep)
        if side == fb.LEFT:
            ref, orep = oracle_gemm(layout, M, N, M, alpha, Sym, B, beta, Cin, inj)
        else:
            ref, orep = oracle_gemm(layout, M, N, N, alpha, B, Sym, beta, Cin, inj)
        assert report_summary(r) == report_summary(orep)
        assert record_set(r) == record_set(orep)
        assert norm_err(got, ref, Sym, B, dim) <= 1e-15


@pytest.mark.parametrize("layout,side,uplo,transa,diag", list(itertools.product(
    (O.COL_MAJOR, O.ROW_MAJOR), (fb.LEFT, fb.RIGHT), (fb.UPPER, fb.LOWER), (fb.NO_TRANS, fb.TRANS),
    (fb.NON_UNIT, fb.UNIT))))
def test_dtrmm_matches_oracle(layout, side, uplo, transa, diag):
    M, N = 330, 270
    dim = M if side == fb.LEFT else N
    A = S.uniform_matrix(52, 0, dim, dim)
    upper = uplo == fb.UPPER
    r, c = np.indices((dim, dim))
    tri = np.where((r <= c) if upper else (r >= c), A, 0.0)
    if diag == fb.UNIT:
        tri[np.arange(dim), np.arange(dim)] = 1.0
    T = tri.T if transa == fb.TRANS else tri  # op(A)
    B0 = S.uniform_matrix(52, 1, M, N)
    alpha = -1.25
    a, lda = S.store(stored_triangle(A, upper, nan_diag=diag == fb.UNIT), layout, ld=dim + 1)
    b, ldb = S.store(B0, layout, ld=(M if layout == O.COL_MAJOR else N) + 2)
    dA, dB = dev(a), dev(b)
    rep = fb.new_report()
    fb.check(fb.ftblas_dtrmm(layout, side, uplo, transa, diag, M, N, alpha, dA.data_ptr(), lda, dB.data_ptr(), ldb,
                             torch.cuda.current_stream().cuda_stream, rep.data_ptr()))
    torch.cuda.synchronize()
    got = S.load(dB.cpu().numpy(), layout, M, N, ldb)
    zero = np.zeros((M, N))
    if side == fb.LEFT:
        ref, orep = oracle_gemm(layout, M, N, M, alpha, T, B0, 0.0, zero)
    else:
        ref, orep = oracle_gemm(layout, M, N, N, alpha, B0, T, 0.0, zero)
    assert report_summary(fb.report_from_device(rep)) == report_summary(orep)
    assert norm_err(got, ref, T, B0, dim) <= 1e-15


@pytest.mark.parametrize("layout", [O.COL_MAJOR, O.ROW_MAJOR])
def test_dtrmm_faults_located_like_the_oracle(layout):
    """Output and accumulator faults (the latter inside the tile's k-range) in FT-DTRMM,
    side LEFT, upper: a tile starts at k = its first row (the tile of rows from 128 at k-tile 4)."""
    M, N = 384, 256
    A = S.uniform_matrix(53, 0, M, M)
    T = np.triu(A)
    B0 = S.uniform_matrix(53, 1, M, N)
    a, lda = S.store(stored_triangle(A, True), layout)
    b, ldb = S.store(B0, layout)
    cases = [[dict(i=200, j=100, site=fb.SITE_OUTPUT, mode=fb.MODE_ADD_REL, rel_log2=4, sign=1)],
             [dict(i=140, j=30, site=fb.SITE_ACCUM, mode=fb.MODE_BITFLIP, bit=56, kt=7)],
             [dict(i=300, j=250, site=fb.SITE_ACCUM, mode=fb.MODE_BITFLIP, bit=60, kt=10)]]
    for pts in cases:
        dA, dB = dev(a), dev(b)
        fb.ftblas_set_injection(fb.make_injection(fixed=pts))
        rep = fb.new_report()
        fb.check(fb.ftblas_dtrmm(layout, fb.LEFT, fb.UPPER, fb.NO_TRANS, fb.NON_UNIT, M, N, 1.0, dA.data_ptr(), lda,
                                 dB.data_ptr(), ldb, torch.cuda.current_stream().cuda_stream, rep.data_ptr()))
        torch.cuda.synchronize()
        r = fb.report_from_device(rep)
        _, orep = oracle_gemm(layout, M, N, M, 1.0, T, B0, 0.0, np.zeros((M, N)), pts)
        assert report_summary(r) == report_summary(orep), pts
        assert record_set(r) == record_set(orep), pts
        assert r.corrected == 1, pts


def trsm_system(layout, side, uplo, transa, diag, M, N, seed):
    """A well-conditioned triangular A (stored triangle only, NaN elsewhere and on a unit
    diagonal), B, and the left-form system T X = alpha W0 the definition gives."""
    dim = M if side == fb.LEFT else N
    R = S.uniform_matrix(seed, 0, dim, dim)
    upper = uplo == fb.UPPER
    r, c = np.indices((dim, dim))
    # off-diagonal entries below 1 / (2 dim): diagonally dominant, so well conditioned
    tri = np.where((r <= c) if upper else (r >= c), R / (2 * dim), 0.0)
    tri[np.arange(dim), np.arange(dim)] = 1.0 if diag == fb.UNIT else 1.0 + S.uniform(seed, 3, dim) ** 2
    opA = tri.T if transa == fb.TRANS else tri
    B = S.uniform_matrix(seed, 1, M, N)
    stored = stored_triangle(np.where((r <= c) if upper else (r >= c), tri, np.nan), upper,
                             nan_diag=diag == fb.UNIT)
    return dim, opA, B, stored


def run_trsm(layout, side, uplo, transa, diag, M, N, alpha, stored, B, inj=None):
    dim = M if side == fb.LEFT else N
    a, lda = S.store(stored, layout, ld=dim + 1)
    b, ldb = S.store(B, layout, ld=(M if layout == O.COL_MAJOR else N) + 3)
    dA, dB = dev(a), dev(b)
    fb.ftblas_set_injection(fb.make_injection(fixed=inj) if inj else None)
    rep = fb.new_report()
    fb.check(fb.ftblas_dtrsm(layout, side, uplo, transa, diag, M, N, alpha, dA.data_ptr(), lda, dB.data_ptr(), ldb,
                             torch.cuda.current_stream().cuda_stream, rep.data_ptr()))
    torch.cuda.synchronize()
    fb.ftblas_set_injection(None)
    return S.load(dB.cpu().numpy(), layout, M, N, ldb), fb.report_from_device(rep)


@pytest.mark.parametrize("layout,side,uplo,transa,diag", list(itertools.product(
    (O.COL_MAJOR, O.ROW_MAJOR), (fb.LEFT, fb.RIGHT), (fb.UPPER, fb.LOWER), (fb.NO_TRANS, fb.TRANS),
    (fb.NON_UNIT, fb.UNIT))))
def test_dtrsm_matches_oracle(layout, side, uplo, transa, diag):
    """X against the oracle's substitution on the same system (left form: T = op(A) or
    op(A)^T, W0 = B or B^T): |X - X_ref| within 2 gamma_{3n} of |T^-1| |alpha W0| growth,
    bounded here through the well-conditioned T; and a small residual op(A) X - alpha B."""
    M, N = 300, 200
    alpha = 0.75
    dim, opA, B, stored = trsm_system(layout, side, uplo, transa, diag, M, N, 54)
    X, rep = run_trsm(layout, side, uplo, transa, diag, M, N, alpha, stored, B)
    T = opA if side == fb.LEFT else opA.T
    W0 = alpha * (B if side == fb.LEFT else B.T)
    lower = np.allclose(np.triu(T, 1), 0.0)
    Xref = O.trsm_left(T, W0, lower)
    Xref = Xref if side == fb.LEFT else Xref.T
    g = 3 * dim * 2.0 ** -53
    assert np.max(np.abs(X - Xref)) <= 64 * g * np.max(np.abs(Xref))
    res = (opA @ X - alpha * B) if side == fb.LEFT else (X @ opA - alpha * B)
    mag = (np.abs(opA) @ np.abs(X)) if side == fb.LEFT else (np.abs(X) @ np.abs(opA))
    assert np.all(np.abs(res) <= 4 * g * mag + 1e-300)
    assert rep.detected == 0 and rep.status == 0 and rep.tiles_checked > 0


@pytest.mark.parametrize("side", [fb.LEFT, fb.RIGHT])
@pytest.mark.parametrize("layout", [O.COL_MAJOR, O.ROW_MAJOR])
def test_dtrsm_faults_in_every_step_are_corrected_bitwise(layout, side):
    """A fixed injection point applies to every internal step (each protected update GEMM
    and each diagonal solve, in that step's coordinates): every fault is detected and
    corrected, and X equals the fault-free X bit for bit."""
    M, N = 520, 300
    dim, opA, B, stored = trsm_system(layout, side, fb.LOWER, fb.NO_TRANS, fb.NON_UNIT, M, N, 55)
    clean, rep0 = run_trsm(layout, side, fb.LOWER, fb.NO_TRANS, fb.NON_UNIT, M, N, 1.0, stored, B)
    assert rep0.detected == 0
    pts = [dict(i=5, j=7, site=fb.SITE_OUTPUT, mode=fb.MODE_BITFLIP, bit=54)]
    got, rep = run_trsm(layout, side, fb.LOWER, fb.NO_TRANS, fb.NON_UNIT, M, N, 1.0, stored, B, inj=pts)
    leaves = -(-dim // 128)
    assert rep.detected == rep.corrected == 2 * leaves - 1  # every diagonal solve and every update
    assert rep.uncorrectable == 0 and rep.checksum_only == 0
    assert np.array_equal(got, clean)
