"""GPU parity of the tensor-core forms (BF16 and FP8 E4M3, tcgen05, binary32 accumulation)
beyond one persistent round, against the oracle's ACC32 / ACC32_E4M3 precision, through the
C ABI (ftblas_gemm_ex).

The persistent product kernel runs one CTA per SM. A problem with more tiles than SMs makes
each CTA take several tiles in turn, hand TMEM accumulator buffers back and forth between
its MMA and epilogue warps, and, when N is not a multiple of the tile width, finish with the
narrow tiles of the last column block, which run narrower MMAs. These tests cover that
regime element by element:

- 2304 x 4100 x 520 in both layouts with beta != 0: 306 tiles in the column-major frame
  (18 x 17, the last column block 132 columns wide) and 330 in the row-major one (33 x 10,
  the last block 72 wide), so two to three rounds on 152 SMs. One output fault per call, in
  the bottom-right tile (narrow, last round) or in a full tile of the second round.
  Every element is compared with the oracle within the accumulation bound (the corrected
  element within its record's row threshold), and reports and records must equal the
  oracle's.
- FP8 at the full 16384^3 size of the benchmark, with one fault: sampled rows within the
  bound, the faulted tile's detection equal to the oracle's.
"""
import numpy as np
import pytest

import oracle as O
import synth as S
from tests.helpers import record_set, report_summary
from tests.test_gpu_fp8 import U_FP8, Fp8Problem
from tests.test_gpu_tc import Bf16Problem

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2104_00897_gb300 as fb  # noqa: E402


def gamma(n, u):
    return n * u / (1 - n * u)


@pytest.fixture(autouse=True)
def _fresh_injection():
    fb.ftblas_set_injection(None)
    yield
    fb.ftblas_set_injection(None)


def _tile_of(P, i, j):
    tr, tc, _ = P.tile()
    return (i // tr) + (j // tc) * (-(-P.M // tr))


def _largest_in_tile(clean, P, tile_row, tile_col):
    tr, tc, _ = P.tile()
    block = np.abs(clean[tile_row * tr:(tile_row + 1) * tr, tile_col * tc:(tile_col + 1) * tc])
    a, b = np.unravel_index(np.argmax(block), block.shape)
    return tile_row * tr + int(a), tile_col * tc + int(b)


@pytest.fixture
def cta_group(request):
    prev = fb.ftblas_set_tc_cta_group(request.param)
    yield request.param
    fb.ftblas_set_tc_cta_group(prev)


@pytest.mark.parametrize("cta_group", [1, 2], indirect=True)
@pytest.mark.parametrize("kind", ["bf16", "fp8"])
@pytest.mark.parametrize("layout", [O.COL_MAJOR, O.ROW_MAJOR])
def test_multi_round_parity_with_one_fault_per_call(kind, layout, cta_group):
    M, N, K = 2304, 4100, 520
    cls = Bf16Problem if kind == "bf16" else Fp8Problem
    P = cls(M, N, K, layout, alpha=1.25, beta=0.5, seed=2304 + layout)
    tr, tc, _ = P.tile()
    n_tr, n_tc = -(-M // tr), -(-N // tc)
    assert n_tr * n_tc > 2 * 152  # more than two persistent rounds
    clean, rep = P.run()
    ref, orep = P.oracle()
    bound = P.bound(ref)
    assert np.all(np.abs(clean - ref) <= bound)
    assert report_summary(rep) == report_summary(orep) and rep.detected == 0 and rep.status == 0
    assert rep.tiles_checked == n_tr * n_tc
    # faults: the bottom-right tile (the narrow last column block of the kernel frame, last
    # round) and a full-width tile of the second round
    spots = [_largest_in_tile(clean, P, n_tr - 1, n_tc - 1), _largest_in_tile(clean, P, n_tr // 2, n_tc // 2)]
    for (i, j) in spots:
        pt = dict(i=i, j=j, site=fb.SITE_OUTPUT, mode=fb.MODE_ADD_REL, rel_log2=12, sign=1)
        fb.ftblas_set_injection(fb.make_injection(fixed=[pt]))
        got, rep = P.run()
        fb.ftblas_set_injection(None)
        t = _tile_of(P, i, j)
        _, orep_t = P.oracle(injections=[pt], tiles=[t])
        assert report_summary(rep)[1:] == report_summary(orep_t)[1:] == (1, 1, 0, 0, 0), (i, j)
        assert rep.tiles_checked == n_tr * n_tc
        assert record_set(rep) == record_set(orep_t) == [(i, j, fb.KIND_CORRECTED)]
        (r,) = rep.records()
        b2 = bound.copy()
        b2[i, j] += r.tau_row + 2.0 ** -21 * abs(ref[i, j])
        assert np.all(np.abs(got - ref) <= b2), (i, j)
        others = np.ones_like(got, dtype=bool)
        others[i, j] = False
        assert np.array_equal(got[others], clean[others])  # nothing else moved


@pytest.mark.parametrize("kind", ["bf16", "fp8"])
@pytest.mark.parametrize("N", [256, 368, 369, 500])
def test_cta_pair_shapes_match_the_oracle(kind, N):
    """The CTA-pair kernel's unit shapes: an odd number of 128-row tiles (the last pair's odd
    CTA reads rows past M as zeros and stores nothing), and last column blocks of 8 and 120
    data columns (the narrow pair MMA with the checksum pieces staged by the odd CTA), 121
    (full width, rows past N zero), and 248. Protected and unprotected calls, with one CTA per
    tile and with CTA pairs: values within the accumulation bound of the oracle, reports equal
    to its clean report, and with a fault in the last tile of the ragged corner the oracle's
    record."""
    M, K = 300, 200
    cls = Bf16Problem if kind == "bf16" else Fp8Problem
    P = cls(M, N, K, O.COL_MAJOR, alpha=0.75, beta=-0.5, seed=300 + N)
    ref, orep = P.oracle()
    bound = P.bound(ref)
    tr, tc, _ = P.tile()
    i, j = _largest_in_tile(ref, P, -(-M // tr) - 1, -(-N // tc) - 1)
    pt = dict(i=i, j=j, site=fb.SITE_OUTPUT, mode=fb.MODE_ADD_REL, rel_log2=14, sign=-1)
    _, orep_f = P.oracle(injections=[pt], tiles=[_tile_of(P, i, j)])
    prev = fb.ftblas_set_tc_cta_group(2)
    try:
        for cg in (1, 2):
            fb.ftblas_set_tc_cta_group(cg)
            got, rep = P.run()
            assert np.all(np.abs(got - ref) <= bound), cg
            assert report_summary(rep) == report_summary(orep) and rep.detected == 0 and rep.status == 0, cg
            plain, _ = P.run(protect=False)
            assert np.all(np.abs(plain - ref) <= bound), cg
            fb.ftblas_set_injection(fb.make_injection(fixed=[pt]))
            fgot, frep = P.run()
            fb.ftblas_set_injection(None)
            assert report_summary(frep)[1:] == report_summary(orep_f)[1:] == (1, 1, 0, 0, 0), cg
            assert record_set(frep) == record_set(orep_f) == [(i, j, fb.KIND_CORRECTED)], cg
            (r,) = frep.records()
            assert abs(fgot[i, j] - ref[i, j]) <= bound[i, j] + r.tau_row + 2.0 ** -21 * abs(ref[i, j]), cg
    finally:
        fb.ftblas_set_injection(None)
        fb.ftblas_set_tc_cta_group(prev)


def test_fp8_full_size_16384_sampled_rows():
    """16384^3 FP8 (the benchmark's size) with an injected output error: sampled rows within
    the bound, the faulted tile's detection and record equal to the oracle's."""
    n = 16384
    threads = 16
    A = S.normal_matrix(20210605, 0, n, n, threads=threads)
    B = S.normal_matrix(20210605, 1, n, n, threads=threads)
    sa = float(np.float32(np.max(np.abs(A)) / 448.0))
    sb = float(np.float32(np.max(np.abs(B)) / 448.0))
    abits = S.map_elementwise(lambda x: S.to_e4m3_bits(x / sa), A, np.uint8, threads)          # op(A), rows k-contiguous
    bbits_t = S.map_elementwise(lambda x: S.to_e4m3_bits(x / sb), np.ascontiguousarray(B.T), np.uint8, threads)
    del A, B
    dA = torch.from_numpy(abits).cuda()
    dB = torch.from_numpy(bbits_t).cuda()
    dC = torch.zeros((n, n), dtype=torch.float32, device="cuda")  # column-major C: dC[j, i]
    dS = torch.tensor([sa, sb], dtype=torch.float32, device="cuda")
    i, j = 12345, 6789
    pt = dict(i=i, j=j, site=fb.SITE_OUTPUT, mode=fb.MODE_ADD_REL, rel_log2=14, sign=-1)
    fb.ftblas_set_injection(fb.make_injection(fixed=[pt]))
    rep = fb.new_report()
    fb.check(fb.ftblas_gemm_ex(O.COL_MAJOR, O.TRANS, O.NO_TRANS, n, n, n, 1.0, dA.data_ptr(), fb.R_8F_E4M3, n,
                               dB.data_ptr(), fb.R_8F_E4M3, n, 0.0, dC.data_ptr(), fb.R_32F, n, fb.R_32F,
                               dS.data_ptr(), dS.data_ptr() + 4, torch.cuda.current_stream().cuda_stream,
                               rep.data_ptr()))
    torch.cuda.synchronize()
    fb.ftblas_set_injection(None)
    r = fb.report_from_device(rep)
    tr, tc, bk = fb.ftblas_verification_tile(O.COL_MAJOR, fb.R_8F_E4M3, n, n, n)
    assert report_summary(r)[:5] == (-(-n // tr) * -(-n // tc), 1, 1, 0, 0) and r.status == 0
    assert [(x.i, x.j, x.kind) for x in r.records()] == [(i, j, fb.KIND_CORRECTED)]
    # oracle: dequantised operands, in the same storage (op(A) = A^T of a K x M column-major
    # array, B a K x N column-major array)
    a64 = S.e4m3_bits_to_f64(abits) * sa       # row r of abits is column r of the stored K x M array
    b64 = S.e4m3_bits_to_f64(bbits_t) * sb
    rows = np.unique(np.concatenate([S.randint(13, 9, 6, 0, n - 1), [i]]))
    ref_rows = O.gemm_rows(O.COL_MAJOR, O.TRANS, O.NO_TRANS, n, n, n, 1.0, a64.ravel(), n, b64.ravel(), n, 0.0,
                           None, n, rows)
    got_rows = dC[:, torch.from_numpy(rows).cuda()].t().double().cpu().numpy()
    prod = np.abs(a64[rows, :]) @ np.abs(b64).T
    bound = 2 * gamma(n, U_FP8) * prod + 2.0 ** -21 * np.abs(ref_rows) + 1e-30
    sel = np.ones_like(ref_rows, dtype=bool)
    ri = list(rows).index(i)
    sel[ri, j] = False
    assert np.all(np.abs(got_rows - ref_rows)[sel] <= bound[sel])
    (rec,) = r.records()
    assert abs(got_rows[ri, j] - ref_rows[ri, j]) <= rec.tau_row + bound[ri, j]
    t = (i // tr) + (j // tc) * (-(-n // tr))
    _, orep = O.ft_gemm(O.COL_MAJOR, O.TRANS, O.NO_TRANS, n, n, n, 1.0, a64.ravel(), n, b64.ravel(), n, 0.0, None, n,
                        tr, tc, bk, injections=[pt], tiles=[t], precision=O.PREC_ACC32_E4M3, u_acc=U_FP8)
    assert record_set(orep) == record_set(r)
