"""GPU parity of the BF16 tensor-core ABFT GEMM (tcgen05, FP32 accumulation) against the
CPU oracle's ACC32 precision, through the C ABI (ftblas_gemm_ex).

Values: the oracle forms each C(i,j) from the exact inner product of the same BF16
operands (binary64), rounded once to binary32; the kernel accumulates in binary32 on the
tensor core. They must agree within the stated accumulation bound,
|C - C_ref| <= 2 gamma_K(2^-23) |alpha| (|A||B|)_ij + 2^-22 (|C_ref| + |beta C_in|).
Detection, location and classification must match the oracle exactly where the injected
error is not within a factor 4 of the threshold (both sides evaluate the same threshold
formula from slightly different roundings).
"""
import ctypes

import numpy as np
import pytest

import oracle as O
import synth as S
from tests.helpers import record_set, report_summary

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2104_00897_gb300 as fb  # noqa: E402

U32 = 2.0 ** -23


def gamma(n, u):
    return n * u / (1 - n * u)


@pytest.fixture(autouse=True)
def _fresh_injection():
    fb.ftblas_set_injection(None)
    yield
    fb.ftblas_set_injection(None)


class Bf16Problem:
    """Seeded BF16 operands, K-contiguous in the kernel frame (the path's requirement)."""

    def __init__(self, M, N, K, layout=O.COL_MAJOR, alpha=1.0, beta=0.0, seed=1, row_scale=False, pad=8):
        self.M, self.N, self.K, self.layout, self.alpha, self.beta = M, N, K, layout, alpha, beta
        # column-major: A transposed, B not; row-major: A not, B transposed
        self.ta, self.tb = (O.TRANS, O.NO_TRANS) if layout == O.COL_MAJOR else (O.NO_TRANS, O.TRANS)
        A = S.normal_matrix(seed, 0, M, K)
        if row_scale:
            A = A * S.pow2_row_scales(seed, 5, M)[:, None]
        B = S.normal_matrix(seed, 1, K, N)
        self.Abits = S.to_bf16_bits(A)
        self.Bbits = S.to_bf16_bits(B)
        self.A = S.bf16_bits_to_f64(self.Abits)
        self.B = S.bf16_bits_to_f64(self.Bbits)
        self.Cin = S.bf16_bits_to_f64(S.to_bf16_bits(S.normal_matrix(seed, 2, M, N)))  # exact in binary32 too
        Xa = self.Abits if self.ta == O.NO_TRANS else self.Abits.T
        Xb = self.Bbits if self.tb == O.NO_TRANS else self.Bbits.T
        up8 = lambda x: (x + 7) // 8 * 8  # 16-byte rows for TMA
        lda = up8(Xa.shape[0] if layout == O.COL_MAJOR else Xa.shape[1]) + pad
        ldb = up8(Xb.shape[0] if layout == O.COL_MAJOR else Xb.shape[1]) + pad
        self.a16, self.lda = S.store(Xa, layout, ld=lda, pad_value=0)
        self.b16, self.ldb = S.store(Xb, layout, ld=ldb, pad_value=0)
        XaF = self.A if self.ta == O.NO_TRANS else self.A.T
        XbF = self.B if self.tb == O.NO_TRANS else self.B.T
        self.a64, _ = S.store(XaF, layout, ld=lda)
        self.b64, _ = S.store(XbF, layout, ld=ldb)
        self.ldc = (M if layout == O.COL_MAJOR else N) + 4
        self.c64, _ = S.store(self.Cin, layout, ld=self.ldc)

    def tile(self):
        return fb.ftblas_verification_tile(self.layout, fb.R_32F, self.M, self.N, self.K)

    def run(self, protect=True):
        dA = torch.from_numpy(self.a16.view(np.int16)).cuda()
        dB = torch.from_numpy(self.b16.view(np.int16)).cuda()
        dC = torch.from_numpy(np.nan_to_num(self.c64, nan=0.0).astype(np.float32)).cuda()
        rep = fb.new_report() if protect else None
        st = torch.cuda.current_stream().cuda_stream
        args = (self.layout, self.ta, self.tb, self.M, self.N, self.K, self.alpha, dA.data_ptr(), fb.R_16BF,
                self.lda, dB.data_ptr(), fb.R_16BF, self.ldb, self.beta, dC.data_ptr(), fb.R_32F, self.ldc, fb.R_32F,
                None, None, st)
        rc = fb.ftblas_gemm_ex(*args, rep.data_ptr()) if protect else fb.ftblas_gemm_ex_noabft(*args)
        fb.check(rc, "ftblas_gemm_ex")
        torch.cuda.synchronize()
        out = S.load(dC.cpu().numpy().astype(np.float64), self.layout, self.M, self.N, self.ldc)
        return out, (fb.report_from_device(rep) if protect else None)

    def oracle(self, injections=(), tiles=None):
        tr, tc, bk = self.tile()
        out, rep = O.ft_gemm(self.layout, self.ta, self.tb, self.M, self.N, self.K, self.alpha, self.a64, self.lda,
                             self.b64, self.ldb, self.beta, self.c64, self.ldc, tr, tc, bk, injections=injections,
                             tiles=tiles, precision=O.PREC_ACC32)
        return S.load(out, self.layout, self.M, self.N, self.ldc), rep

    def bound(self, ref):
        prod = np.abs(self.A) @ np.abs(self.B)
        return (2 * gamma(self.K, U32) * abs(self.alpha) * prod + 2.0 ** -22 * (np.abs(ref) + abs(self.beta) *
                np.abs(self.Cin)) + 1e-30)


@pytest.mark.parametrize("layout", [O.COL_MAJOR, O.ROW_MAJOR])
@pytest.mark.parametrize("shape", [(128, 256, 64), (300, 700, 200), (256, 512, 1000), (5, 3, 130)])
def test_bf16_values_match_oracle_within_bound(layout, shape):
    M, N, K = shape
    P = Bf16Problem(M, N, K, layout, alpha=1.25, beta=0.5, seed=M + N + K)
    plain, _ = P.run(protect=False)
    got, rep = P.run(protect=True)
    ref, orep = P.oracle()
    assert np.all(np.abs(got - ref) <= P.bound(ref))
    assert np.array_equal(got, plain)  # the checksum MMA does not touch the product
    assert report_summary(rep) == report_summary(orep)
    assert rep.detected == 0 and rep.status == 0


@pytest.mark.parametrize("layout", [O.COL_MAJOR, O.ROW_MAJOR])
def test_bf16_injections_match_oracle(layout):
    """Errors far above the rigorous threshold are detected, located and corrected as the
    oracle does; an error far below it is not detected by either side (undetectable by
    construction) and stays in C."""
    P = Bf16Problem(384, 768, 512, layout, alpha=1.0, beta=0.0, seed=3)
    clean, _ = P.run()
    big = np.argsort(np.abs(clean), axis=None)[::-1]
    (i1, j1), (i2, j2), (i3, j3) = [np.unravel_index(x, clean.shape) for x in big[[0, 40, 400]]]
    i4, j4 = np.unravel_index(np.argmin(np.where(clean != 0, np.abs(clean), np.inf)), clean.shape)
    assert abs(clean[i4, j4]) < 2.0  # bit 30 of its binary32 pattern is clear: the flip scales it by 2^128
    cases = [
        [dict(i=int(i1), j=int(j1), site=fb.SITE_OUTPUT, mode=fb.MODE_ADD_REL, rel_log2=4, sign=1)],
        [dict(i=int(i2), j=int(j2), site=fb.SITE_OUTPUT, mode=fb.MODE_ADD_REL, rel_log2=3, sign=-1)],
        [dict(i=int(i4), j=int(j4), site=fb.SITE_ACCUM, mode=fb.MODE_BITFLIP, bit=30)],
        [dict(i=int(i3), j=int(j3), site=fb.SITE_OUTPUT, mode=fb.MODE_BITFLIP, bit=29)],
        [dict(i=int(i1), j=int(j1), site=fb.SITE_OUTPUT, mode=fb.MODE_ADD_REL, rel_log2=4),
         dict(i=int(i1) ^ 1, j=int(j1) ^ 1, site=fb.SITE_OUTPUT, mode=fb.MODE_ADD_REL, rel_log2=20)],
        [dict(i=int(i1), j=int(j1), site=fb.SITE_OUTPUT, mode=fb.MODE_ADD_REL, rel_log2=-40)],
    ]
    if layout == O.COL_MAJOR:
        cases.append([dict(i=200, j=100, site=fb.SITE_CHECKSUM, mode=fb.MODE_ADD_REL, rel_log2=20, sign=1)])
    detected = 0
    for pts in cases:
        fb.ftblas_set_injection(fb.make_injection(fixed=pts))
        got, rep = P.run()
        ref, orep = P.oracle(injections=pts)
        assert report_summary(rep) == report_summary(orep), pts
        assert record_set(rep) == record_set(orep), pts
        detected += int(rep.detected)
        for r in rep.records():
            if r.kind == fb.KIND_CORRECTED:
                # corrected from the checksum: within the row threshold of the fault-free value
                assert abs(got[r.i, r.j] - clean[r.i, r.j]) <= r.tau_row + 2.0 ** -22 * abs(clean[r.i, r.j])
        if rep.uncorrectable == 0:
            mask = np.ones_like(got, dtype=bool)
            for r in rep.records():
                if r.i >= 0 and r.j >= 0:
                    mask[r.i, r.j] = False
            if rep.detected == 0:
                for q in pts:  # undetected (below threshold): the error stays where it was put
                    mask[q["i"], q["j"]] = False
            bad = np.argwhere(mask & (got != clean))
            assert bad.size == 0, (pts, [(int(a), int(b), float(got[a, b]), float(clean[a, b])) for a, b in bad[:6]],
                                   [(r.i, r.j, r.kind) for r in rep.records()])
    assert detected >= len(cases) - 1


def test_bf16_detection_threshold_sweep_agrees_with_oracle():
    """Config-3 style map: output errors 2^p |C|, p = -20 .. 8, at the largest |C(i,j)|,
    rows of A scaled by 2^u, u in [-8, 8]. Detection starts where the rigorous threshold
    allows and agrees with the oracle away from the threshold."""
    P = Bf16Problem(256, 512, 1024, O.COL_MAJOR, alpha=1.0, beta=0.0, seed=11, row_scale=True)
    clean, rep0 = P.run()
    _, orep0 = P.oracle()
    assert rep0.detected == 0 and orep0.detected == 0
    i, j = (int(x) for x in np.unravel_index(np.argmax(np.abs(clean)), clean.shape))
    first = None
    for p in range(-20, 9, 2):
        pts = [dict(i=i, j=j, site=fb.SITE_OUTPUT, mode=fb.MODE_ADD_REL, rel_log2=p, sign=1)]
        fb.ftblas_set_injection(fb.make_injection(fixed=pts))
        _, rep = P.run()
        _, orep = P.oracle(injections=pts)
        e = 2.0 ** p * abs(clean[i, j])
        tau = orep.records()[0].tau_row if orep.n_records else None
        if tau is not None and 0.25 < e / tau < 4:
            continue  # within a factor 4 of the threshold: the two roundings may decide apart
        assert report_summary(rep) == report_summary(orep), p
        if rep.corrected and first is None:
            first = p
    assert first is not None and first <= 8


def test_bf16_full_size_8192_sampled_rows():
    """8192^3 BF16 with an injected output error: sampled rows within the bound, the faulted
    tile's detection equal to the oracle's."""
    n = 8192
    P = Bf16Problem(n, n, n, O.COL_MAJOR, alpha=1.0, beta=0.0, seed=20210603, pad=0)
    i, j = 4321, 1234
    pt = dict(i=i, j=j, site=fb.SITE_OUTPUT, mode=fb.MODE_ADD_REL, rel_log2=12, sign=1)
    fb.ftblas_set_injection(fb.make_injection(fixed=[pt]))
    got, rep = P.run()
    tr, tc, _ = P.tile()
    assert report_summary(rep)[:5] == (-(-n // tr) * -(-n // tc), 1, 1, 0, 0)
    assert [(r.i, r.j) for r in rep.records()] == [(i, j)]
    rows = np.unique(np.concatenate([S.randint(9, 9, 3, 0, n - 1), [i]]))
    ref_rows = O.gemm_rows(O.COL_MAJOR, P.ta, P.tb, n, n, n, P.alpha, P.a64, P.lda, P.b64, P.ldb, P.beta, P.c64,
                           P.ldc, rows)
    prod = (np.abs(P.A[rows, :]) @ np.abs(P.B))
    bound = 2 * gamma(n, U32) * prod + 2.0 ** -22 * np.abs(ref_rows) + 1e-30
    sel = np.ones_like(ref_rows, dtype=bool)
    sel[list(rows).index(i), j] = False
    assert np.all(np.abs(got[rows, :] - ref_rows)[sel] <= bound[sel])
    r = rep.records()[0]
    assert abs(got[i, j] - ref_rows[list(rows).index(i), j]) <= r.tau_row + bound[list(rows).index(i), j]
    tr, tc, bk = P.tile()
    t = (i // tr) + (j // tc) * ((n + tr - 1) // tr)
    _, orep = P.oracle(injections=[pt], tiles=[t])
    assert record_set(orep) == record_set(rep)


@pytest.mark.parametrize("cta_group", [1, 2])
def test_bounded_wait_gives_up_and_reports_timeout(cta_group):
    """The tensor-core kernel's bounded waits: a staging barrier that never completes (the
    test-only stall point) ends the stalled CTA's (or CTA pair's) work after 20 ms, with no
    fault. With one unit per persistent CTA (pair), exactly that unit is left unwritten: the
    stalled tile, or with CTA pairs the two 128-row tiles that share the pair's staging
    barrier. The report carries FT_STATUS_TIMEOUT, the other tiles are stored as in a clean
    call, and the next call is clean."""
    prev = fb.ftblas_set_tc_cta_group(cta_group)
    try:
        P = Bf16Problem(256, 496, 512, O.COL_MAJOR, alpha=1.0, beta=0.0, seed=43)
        clean, rep0 = P.run()
        assert rep0.status == 0
        tr, tc, _ = P.tile()
        i, j = 130, 300
        fb.ftblas_set_injection(fb.make_injection(fixed=[dict(i=i, j=j, site=fb.SITE_STALL, kt=3)]))
        try:
            got, rep = P.run()
        finally:
            fb.ftblas_set_injection(None)
        assert rep.status & fb.STATUS_TIMEOUT
        ur = tr * cta_group  # rows of a unit
        stalled = np.zeros_like(got, dtype=bool)
        stalled[(i // ur) * ur:(i // ur + 1) * ur, (j // tc) * tc:(j // tc + 1) * tc] = True
        assert np.array_equal(got[~stalled], clean[~stalled])
        assert np.array_equal(got[stalled], P.Cin.astype(np.float32).astype(np.float64)[stalled])  # not stored
        assert rep.tiles_checked == -(-P.M // tr) * -(-P.N // tc) - cta_group
        again, rep2 = P.run()
        assert rep2.status == 0 and rep2.detected == 0 and np.array_equal(again, clean)
    finally:
        fb.ftblas_set_tc_cta_group(prev)
