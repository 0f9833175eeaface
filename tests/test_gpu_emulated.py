"""GPU parity of the emulated FP64 GEMM (ftblas_dgemm_emulated: binary64 operands as E4M3
integer slices on the tcgen05 tensor cores, exact group products, exact integer checksums)
against the oracle's definition of the same method (emu_oracle.c), through the C ABI.

Every step of the method is exact or rounded in a stated order on both sides, so parity is
bit for bit: C, the report's counters and the records (located elements, kinds) must equal
the oracle's exactly, for all layouts and transposes, ragged and multi-round shapes, and
every injection site. Beside it, the accuracy criterion of the FP64 path,
max|C - C_ref| / (max|A| max|B| K) <= 1e-15, against the oracle's binary64 product.
"""
import numpy as np
import pytest

import oracle as O
import synth as S
from tests.helpers import record_set, report_summary

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2104_00897_gb300 as fb  # noqa: E402

COMBOS = [(l, a, b) for l in (O.COL_MAJOR, O.ROW_MAJOR) for a in (O.NO_TRANS, O.TRANS)
          for b in (O.NO_TRANS, O.TRANS)]


@pytest.fixture(autouse=True)
def _fresh_state():
    fb.ftblas_set_injection(None)
    prev = fb.ftblas_set_emulation_slices(O.EMU_SLICES)
    yield
    fb.ftblas_set_injection(None)
    fb.ftblas_set_emulation_slices(prev)


def stored(layout, trans, logical, pad):
    X = logical if trans == O.NO_TRANS else logical.T
    ld = (X.shape[0] if layout == O.COL_MAJOR else X.shape[1]) + pad
    return S.store(X, layout, ld=ld)


class EmuProblem:
    def __init__(self, M, N, K, layout=O.COL_MAJOR, ta=O.NO_TRANS, tb=O.NO_TRANS, alpha=1.5, beta=0.5, seed=1,
                 pad=3, A=None, B=None):
        self.M, self.N, self.K, self.layout, self.ta, self.tb = M, N, K, layout, ta, tb
        self.alpha, self.beta = alpha, beta
        self.A = S.uniform_matrix(seed, 0, M, K) if A is None else A
        self.B = S.uniform_matrix(seed, 1, K, N) if B is None else B
        self.Cin = S.uniform_matrix(seed, 2, M, N)
        self.a, self.lda = stored(layout, ta, self.A, pad)
        self.b, self.ldb = stored(layout, tb, self.B, pad)
        self.c, self.ldc = S.store(self.Cin, layout, ld=(M if layout == O.COL_MAJOR else N) + pad)
        # padding beyond each leading dimension holds NaN: a kernel that read it would fail
        self.dA = torch.from_numpy(self.a).cuda()
        self.dB = torch.from_numpy(self.b).cuda()

    def tile(self):
        return fb.ftblas_verification_tile(self.layout, fb.R_8F_E4M3, self.M, self.N, self.K)

    def run(self, protect=True):
        dC = torch.from_numpy(self.c.copy()).cuda()
        st = torch.cuda.current_stream().cuda_stream
        args = (self.layout, self.ta, self.tb, self.M, self.N, self.K, self.alpha, self.dA.data_ptr(), self.lda,
                self.dB.data_ptr(), self.ldb, self.beta, dC.data_ptr(), self.ldc, st)
        rep = fb.new_report() if protect else None
        rc = fb.ftblas_dgemm_emulated(*args, rep.data_ptr()) if protect else fb.ftblas_dgemm_emulated_noabft(*args)
        fb.check(rc, "ftblas_dgemm_emulated")
        torch.cuda.synchronize()
        out = S.load(dC.cpu().numpy(), self.layout, self.M, self.N, self.ldc)
        return out, (fb.report_from_device(rep) if protect else None)

    def oracle(self, injections=(), tiles=None):
        out, rep = O.emu_gemm(self.layout, self.ta, self.tb, self.M, self.N, self.K, self.alpha, self.a, self.lda,
                              self.b, self.ldb, self.beta, self.c, self.ldc, injections=injections, tiles=tiles)
        return S.load(out, self.layout, self.M, self.N, self.ldc), rep

    def normalized_error(self, C, ref):
        return float(np.abs(C - ref).max() / (np.abs(self.A).max() * np.abs(self.B).max() * self.K))


def bits(x):
    return np.ascontiguousarray(x).view(np.uint64)


@pytest.mark.parametrize("layout,ta,tb", COMBOS)
def test_bitwise_parity_all_layouts(layout, ta, tb):
    P = EmuProblem(260, 530, 200, layout, ta, tb, seed=7 + layout + ta + tb)
    got, rep = P.run()
    ref, orep = P.oracle()
    assert np.array_equal(bits(got), bits(ref))
    assert report_summary(rep) == report_summary(orep) and rep.detected == 0 and rep.status == 0
    plain, _ = P.run(protect=False)
    assert np.array_equal(bits(plain), bits(got))  # the checksum digits do not touch the product
    exact = P.alpha * (P.A @ P.B) + P.beta * P.Cin
    assert P.normalized_error(got, exact) <= 1e-15


@pytest.mark.parametrize("layout", [O.COL_MAJOR, O.ROW_MAJOR])
def test_multi_round_ragged_shape(layout):
    """306 (column-major frame) or 330 (row-major frame) tiles on 152 SMs, a narrow last
    column block, beta != 0, rows and columns scaled by 2^u, u in [-30, 30]."""
    M, N, K = 2304, 4100, 136
    A = S.uniform_matrix(31, 0, M, K) * S.pow2_row_scales(31, 5, M, -30, 30)[:, None]
    B = S.uniform_matrix(31, 1, K, N) * S.pow2_row_scales(31, 6, N, -30, 30)[None, :]
    P = EmuProblem(M, N, K, layout, alpha=-0.75, beta=1.25, seed=31, A=A, B=B)
    got, rep = P.run()
    ref, orep = P.oracle()
    assert np.array_equal(bits(got), bits(ref))
    assert report_summary(rep) == report_summary(orep) and rep.detected == 0
    tr, tc, _ = P.tile()
    assert rep.tiles_checked == -(-M // tr) * -(-N // tc) > 2 * 152


@pytest.mark.parametrize("layout", [O.COL_MAJOR, O.ROW_MAJOR])
def test_injections_match_the_oracle(layout):
    """Accumulator flips in several groups and bits (every one detected: the checks are
    exact), output errors, a checksum fault, four faulted rows in one tile (all corrected)
    and five (uncorrectable), and faults in two tiles: reports, records and C bit for bit."""
    P = EmuProblem(300, 520, 160, layout, seed=11)
    clean, _ = P.run()
    cases = [
        [dict(i=5, j=7, site=fb.SITE_ACCUM, mode=fb.MODE_BITFLIP, bit=20, kt=0)],
        [dict(i=129, j=300, site=fb.SITE_ACCUM, mode=fb.MODE_BITFLIP, bit=30, kt=3)],
        [dict(i=200, j=511, site=fb.SITE_ACCUM, mode=fb.MODE_BITFLIP, bit=0, kt=13)],
        [dict(i=299, j=0, site=fb.SITE_ACCUM, mode=fb.MODE_BITFLIP, bit=23, kt=7)],
        [dict(i=50, j=250, site=fb.SITE_OUTPUT, mode=fb.MODE_ADD_REL, rel_log2=-30, sign=1)],
        [dict(i=51, j=25, site=fb.SITE_OUTPUT, mode=fb.MODE_BITFLIP, bit=62)],
        [dict(i=52, j=26, site=fb.SITE_OUTPUT, mode=fb.MODE_ADD_REL, rel_log2=-80, sign=-1)],  # below threshold
        [dict(i=60, j=40, site=fb.SITE_CHECKSUM, mode=fb.MODE_ADD_REL, rel_log2=-50, sign=1)],
        [dict(i=r, j=(37 * r) % 240, site=fb.SITE_ACCUM, mode=fb.MODE_BITFLIP, bit=27, kt=r % 5) for r in range(4)],
        [dict(i=r, j=(37 * r) % 240, site=fb.SITE_ACCUM, mode=fb.MODE_BITFLIP, bit=27, kt=1) for r in range(5)],
        [dict(i=3, j=3, site=fb.SITE_ACCUM, mode=fb.MODE_BITFLIP, bit=29, kt=2),
         dict(i=290, j=500, site=fb.SITE_OUTPUT, mode=fb.MODE_ADD_REL, rel_log2=4, sign=-1)],
    ]
    for pts in cases:
        fb.ftblas_set_injection(fb.make_injection(fixed=pts))
        got, rep = P.run()
        fb.ftblas_set_injection(None)
        ref, orep = P.oracle(injections=pts)
        assert report_summary(rep) == report_summary(orep), pts
        assert record_set(rep) == record_set(orep), pts
        assert np.array_equal(bits(got), bits(ref)), pts
        below = any(q.get("rel_log2") == -80 for q in pts)  # undetectable: the error stays
        if rep.uncorrectable == 0 and not below:
            assert np.array_equal(bits(got), bits(clean)), pts


def test_seeded_draw_and_accumulator_flips_over_launches():
    """The seeded plan (bits 0-31 of the group accumulators, one point per launch) equals the
    oracle's draw on the emulated tile, and every launch's flip is detected and removed."""
    P = EmuProblem(512, 744, 128, seed=12)
    clean, _ = P.run()
    tr, tc, _ = P.tile()
    fb.ftblas_set_injection(fb.make_injection(seed=77, site=fb.SITE_ACCUM, mode=fb.MODE_BITFLIP, bit_lo=0, bit_hi=31,
                                              every_n_launches=1, errors_per_launch=2))
    for launch in range(4):
        got, rep = P.run()
        pts = O.draw_injections(77, launch, 1, 2, O.SITE_ACCUM, O.MODE_BITFLIP, 0, 31, 0, 0, P.M, P.N, tr, tc)
        ref, orep = P.oracle(injections=pts)
        assert report_summary(rep) == report_summary(orep) and rep.detected == 2, launch
        assert record_set(rep) == record_set(orep)
        assert np.array_equal(bits(got), bits(clean))


def test_full_size_8192_sampled_tiles_and_accuracy():
    """Config 2's 8192^3 at alpha = 1.5, beta = 0.5 with one accumulator flip: the faulted
    tile and three others bit for bit against the oracle, and sampled rows within the FP64
    criterion of the oracle's binary64 product."""
    n = 8192
    P = EmuProblem(n, n, n, alpha=1.5, beta=0.5, seed=20210601, pad=0)
    i, j = 4321, 1234
    pt = dict(i=i, j=j, site=fb.SITE_ACCUM, mode=fb.MODE_BITFLIP, bit=26, kt=1)
    fb.ftblas_set_injection(fb.make_injection(fixed=[pt]))
    got, rep = P.run()
    fb.ftblas_set_injection(None)
    tr, tc, _ = P.tile()
    n_tr = -(-n // tr)
    assert report_summary(rep)[:5] == (n_tr * -(-n // tc), 1, 1, 0, 0) and rep.status == 0
    assert [(r.i, r.j, r.kind) for r in rep.records()] == [(i, j, fb.KIND_CORRECTED)]
    tiles = [(i // tr) + (j // tc) * n_tr, 0, n_tr - 1, n_tr * (-(-n // tc)) - 1]
    ref, orep = P.oracle(injections=[pt], tiles=tiles)
    assert record_set(orep) == record_set(rep)
    for t in tiles:
        r0, c0 = (t % n_tr) * tr, (t // n_tr) * tc
        blk = (slice(r0, min(n, r0 + tr)), slice(c0, min(n, c0 + tc)))
        assert np.array_equal(bits(got[blk]), bits(ref[blk])), t
    rows = np.unique(np.concatenate([S.randint(3, 9, 5, 0, n - 1), [i]]))
    ref_rows = O.gemm_rows(P.layout, P.ta, P.tb, n, n, n, P.alpha, P.a, P.lda, P.b, P.ldb, P.beta, P.c, P.ldc, rows)
    assert P.normalized_error(got[rows, :], ref_rows) <= 1e-15


def test_i128_conversion_is_correctly_rounded():
    """The kernel's 128-bit integer to binary64 conversion equals Python's float(int) (round
    to nearest, ties to even) on ties, carries, negatives and the extremes."""
    import random
    rnd = random.Random(9)
    vals = [0, 1, -1, 2 ** 53 + 1, 2 ** 53 + 3, 2 ** 54 + 2, 2 ** 54 + 6, 2 ** 64 + 2 ** 11, 2 ** 64 + 2 ** 11 + 1,
            2 ** 80 + 2 ** 27, 2 ** 80 + 2 ** 27 + 1, 2 ** 127 - 1, -(2 ** 127), -(2 ** 64) - 1, 2 ** 63, -(2 ** 63)]
    for _ in range(4000):
        nb = rnd.randint(1, 126)
        v = rnd.getrandbits(nb)
        if rnd.random() < 0.4:
            v = (v >> max(0, nb - 54) << max(0, nb - 54)) | (1 << max(0, nb - 55))  # exact ties
        vals.append(v if rnd.random() < 0.5 else -v)
    words = np.zeros(2 * len(vals), dtype=np.int64)
    for q, v in enumerate(vals):
        u = v & ((1 << 128) - 1)
        words[2 * q] = np.array([u & ((1 << 64) - 1)], dtype=np.uint64).view(np.int64)[0]
        words[2 * q + 1] = np.array([u >> 64], dtype=np.uint64).view(np.int64)[0]
    dw = torch.from_numpy(words).cuda()
    out = torch.empty(len(vals), dtype=torch.float64, device="cuda")
    fb.check(fb.ftblas_emu_convert_i128(dw.data_ptr(), out.data_ptr(), len(vals)))
    torch.cuda.synchronize()
    got = out.cpu().numpy()
    want = np.array([float(v) for v in vals])
    assert np.array_equal(got.view(np.uint64), want.view(np.uint64))
    assert fb.ftblas_emu_convert_i128(None, out.data_ptr(), 1) == -1
    assert fb.ftblas_emu_convert_i128(dw.data_ptr(), out.data_ptr(), -1) == -3


def test_nonfinite_inputs_quick_returns_and_limits():
    M, N, K = 200, 300, 64
    P = EmuProblem(M, N, K, seed=13)
    A = P.A.copy()
    A[130, 5] = np.nan
    Q = EmuProblem(M, N, K, seed=13, A=A)
    got, rep = Q.run()
    ref, orep = Q.oracle()
    assert report_summary(rep) == report_summary(orep) and rep.input_nonfinite == 2
    assert np.array_equal(bits(got), bits(ref)) and np.all(np.isnan(got[130]))
    # K = 0: C = beta C_in, nothing checked
    dC = torch.from_numpy(P.c.copy()).cuda()
    rep = fb.new_report()
    fb.check(fb.ftblas_dgemm_emulated(P.layout, P.ta, P.tb, M, N, 0, 1.0, P.dA.data_ptr(), P.lda, P.dB.data_ptr(),
                                      P.ldb, 2.0, dC.data_ptr(), P.ldc, None, rep.data_ptr()))
    torch.cuda.synchronize()
    assert np.array_equal(S.load(dC.cpu().numpy(), P.layout, M, N, P.ldc), 2.0 * P.Cin)
    assert fb.report_from_device(rep).tiles_checked == 0
    # K beyond the exact range of the group accumulators, and the slice setting
    assert fb.ftblas_emulation_max_k(14) == 16384 and fb.ftblas_emulation_max_k(1) == -1
    assert fb.ftblas_dgemm_emulated(P.layout, P.ta, P.tb, M, N, 16385, 1.0, P.dA.data_ptr(), 16385,
                                    P.dB.data_ptr(), 16385, 0.0, dC.data_ptr(), P.ldc, None, None) == 2
    assert fb.ftblas_set_emulation_slices(16) == -1


@pytest.mark.parametrize("slices", [6, 10, 15])
def test_other_slice_counts(slices):
    fb.ftblas_set_emulation_slices(slices)
    P = EmuProblem(140, 260, 96, seed=14)
    got, rep = P.run()
    out, orep = O.emu_gemm(P.layout, P.ta, P.tb, P.M, P.N, P.K, P.alpha, P.a, P.lda, P.b, P.ldb, P.beta, P.c, P.ldc,
                           slices=slices)
    assert np.array_equal(bits(got), bits(S.load(out, P.layout, P.M, P.N, P.ldc)))
    assert report_summary(rep) == report_summary(orep)


def test_bounded_wait_gives_up_and_reports_timeout():
    """A staging barrier that never completes (the test-only stall point) ends its CTA's
    work after 20 ms with no fault: with one tile per CTA exactly that tile is unwritten, the
    report carries FT_STATUS_TIMEOUT, and the next call is clean and identical."""
    P = EmuProblem(256, 496, 256, seed=15)
    clean, rep0 = P.run()
    tr, tc, _ = P.tile()
    i, j = 130, 300
    fb.ftblas_set_injection(fb.make_injection(fixed=[dict(i=i, j=j, site=fb.SITE_STALL, kt=1)]))
    try:
        got, rep = P.run()
    finally:
        fb.ftblas_set_injection(None)
    assert rep.status & fb.STATUS_TIMEOUT
    stalled = np.zeros_like(got, dtype=bool)
    stalled[(i // tr) * tr:(i // tr + 1) * tr, (j // tc) * tc:(j // tc + 1) * tc] = True
    assert np.array_equal(bits(got[~stalled]), bits(clean[~stalled]))
    assert np.array_equal(got[stalled], P.Cin[stalled])  # not stored
    assert rep.tiles_checked == -(-P.M // tr) * -(-P.N // tc) - 1
    again, rep2 = P.run()
    assert rep2.status == 0 and rep2.detected == 0 and np.array_equal(bits(again), bits(clean))
