"""The no-allocation entry point, ftblas_gemm_ex_noalloc.

Some callers cannot allocate device memory while they issue work: their process does not
own the device allocator (another framework has reserved it), or their setting forbids
allocation after start-up. For them ftblas_gemm_ex_noalloc runs the protected BF16 GEMM
on a static 16 MiB device array instead of stream-ordered allocations. These checks call
it through the C ABI and compare it with the allocating entry point, ftblas_gemm_ex,
within the BF16 tolerance the other tests use, on two calls in a row (the second call
finds the first call's data in the shared array); with an injected fault, in both layouts,
its detection, location and correction on two calls in a row equal the allocating entry
point's bit for bit; and a problem needing more scratch than the array holds is rejected
before any device work. This file is collected
last on purpose, and it also passes alone in a fresh process.
"""
import numpy as np
import pytest

import oracle as O
import synth as S
from tests.helpers import report_summary

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2104_00897_gb300 as fb  # noqa: E402

U32 = 2.0 ** -23


def _operands(M, N, K, seed):
    A = S.bf16_bits_to_f64(S.to_bf16_bits(S.normal_matrix(seed, 0, M, K)))
    B = S.bf16_bits_to_f64(S.to_bf16_bits(S.normal_matrix(seed, 1, K, N)))
    Cin = S.bf16_bits_to_f64(S.to_bf16_bits(S.normal_matrix(seed, 2, M, N)))
    # column-major, A transposed (stored K x M) and B not: both K-contiguous
    a16, lda = S.store(S.to_bf16_bits(A).T, O.COL_MAJOR, ld=K)
    b16, ldb = S.store(S.to_bf16_bits(B), O.COL_MAJOR, ld=K)
    return A, B, Cin, a16, lda, b16, ldb


def _call(entry, M, N, K, dA, lda, dB, ldb, Cin, alpha, beta):
    dC = torch.from_numpy(Cin.T.astype(np.float32).ravel().copy()).cuda()  # column-major, ldc = M
    rep = fb.new_report()
    rc = entry(O.COL_MAJOR, O.TRANS, O.NO_TRANS, M, N, K, alpha, dA.data_ptr(), fb.R_16BF, lda, dB.data_ptr(),
               fb.R_16BF, ldb, beta, dC.data_ptr(), fb.R_32F, M, fb.R_32F, None, None,
               torch.cuda.current_stream().cuda_stream, rep.data_ptr())
    fb.check(rc, entry.__name__)
    torch.cuda.synchronize()
    return dC.cpu().numpy().astype(np.float64).reshape(N, M).T, fb.report_from_device(rep)


def test_noalloc_matches_the_allocating_entry_point_twice():
    M, N, K = 640, 1280, 1536
    alpha, beta = 1.25, 0.5
    A, B, Cin, a16, lda, b16, ldb = _operands(M, N, K, seed=97)
    dA = torch.from_numpy(a16.view(np.int16)).cuda()
    dB = torch.from_numpy(b16.view(np.int16)).cuda()
    fb.ftblas_set_injection(None)
    ref, ref_rep = _call(fb.ftblas_gemm_ex, M, N, K, dA, lda, dB, ldb, Cin, alpha, beta)
    gam = K * U32 / (1 - K * U32)
    tol = 2 * gam * abs(alpha) * (np.abs(A) @ np.abs(B)) + 2.0 ** -22 * (np.abs(ref) + abs(beta) * np.abs(Cin))
    for call in range(2):
        got, rep = _call(fb.ftblas_gemm_ex_noalloc, M, N, K, dA, lda, dB, ldb, Cin, alpha, beta)
        assert np.all(np.abs(got - ref) <= tol), call
        assert (rep.tiles_checked, rep.detected, rep.status) == (ref_rep.tiles_checked, 0, 0), call


def _call_layout(entry, layout, M, N, K, dA, lda, dB, ldb, Cin_store, ldc, alpha, beta):
    ta, tb = (O.TRANS, O.NO_TRANS) if layout == O.COL_MAJOR else (O.NO_TRANS, O.TRANS)
    dC = torch.from_numpy(Cin_store.astype(np.float32)).cuda()
    rep = fb.new_report()
    rc = entry(layout, ta, tb, M, N, K, alpha, dA.data_ptr(), fb.R_16BF, lda, dB.data_ptr(), fb.R_16BF, ldb, beta,
               dC.data_ptr(), fb.R_32F, ldc, fb.R_32F, None, None, torch.cuda.current_stream().cuda_stream,
               rep.data_ptr())
    fb.check(rc, entry.__name__)
    torch.cuda.synchronize()
    return dC.cpu().numpy(), fb.report_from_device(rep)


@pytest.mark.parametrize("layout", [O.COL_MAJOR, O.ROW_MAJOR])
def test_noalloc_detects_and_corrects_like_the_allocating_entry_point(layout):
    """One accumulator bit flip (the exponent's top bit, at an element between 1/4 and 1 in
    magnitude, so the flip makes it about 2^128 times larger) on every call. The static array then
    carries the resolve pass's table of mismatching tiles and the checksum operand of the
    previous call; two calls in a row through the no-allocation entry point must detect,
    locate and correct it exactly as the allocating one does: the same counters, the same
    record, and the same output bit for bit (the two run the same kernels). Row-major calls
    swap the operands and dimensions of the kernel frame."""
    M, N, K = 384, 760, 640
    A, B, Cin, _, _, _, _ = _operands(M, N, K, seed=131)
    if layout == O.COL_MAJOR:
        a16, lda = S.store(S.to_bf16_bits(A).T, O.COL_MAJOR, ld=K)   # op(A) = A, stored transposed
        b16, ldb = S.store(S.to_bf16_bits(B), O.COL_MAJOR, ld=K)
        c, ldc = S.store(Cin, O.COL_MAJOR, ld=M)
    else:
        a16, lda = S.store(S.to_bf16_bits(A), O.ROW_MAJOR, ld=K)     # row-major A, K-contiguous
        b16, ldb = S.store(S.to_bf16_bits(B).T, O.ROW_MAJOR, ld=K)   # op(B) = B, stored transposed
        c, ldc = S.store(Cin, O.ROW_MAJOR, ld=N)
    dA = torch.from_numpy(a16.view(np.int16)).cuda()
    dB = torch.from_numpy(b16.view(np.int16)).cuda()
    fb.ftblas_set_injection(None)
    clean, rep0 = _call_layout(fb.ftblas_gemm_ex, layout, M, N, K, dA, lda, dB, ldb, c, ldc, 1.0, 0.0)
    assert rep0.detected == 0
    Cl = S.load(clean.astype(np.float64), layout, M, N, ldc)
    small = np.argwhere((np.abs(Cl) < 1.0) & (np.abs(Cl) > 0.25))  # the flip stays finite: about 2^128 |C|
    i, j = (int(x) for x in small[len(small) // 3])
    pt = dict(i=i, j=j, site=fb.SITE_ACCUM, mode=fb.MODE_BITFLIP, bit=30)
    fb.ftblas_set_injection(fb.make_injection(fixed=[pt]))
    try:
        ref, ref_rep = _call_layout(fb.ftblas_gemm_ex, layout, M, N, K, dA, lda, dB, ldb, c, ldc, 1.0, 0.0)
        assert (ref_rep.detected, ref_rep.corrected, ref_rep.uncorrectable) == (1, 1, 0)
        assert [(r.i, r.j, r.kind) for r in ref_rep.records()] == [(i, j, fb.KIND_CORRECTED)]
        for call in range(2):
            got, rep = _call_layout(fb.ftblas_gemm_ex_noalloc, layout, M, N, K, dA, lda, dB, ldb, c, ldc, 1.0, 0.0)
            assert report_summary(rep) == report_summary(ref_rep), call
            assert rep.status == ref_rep.status == 0
            (r,), (q,) = rep.records(), ref_rep.records()
            assert (r.i, r.j, r.kind, r.rows_flagged, r.cols_flagged) == (q.i, q.j, q.kind, q.rows_flagged,
                                                                          q.cols_flagged), call
            assert np.array_equal([r.delta_row, r.tau_row, r.value_after], [q.delta_row, q.tau_row, q.value_after],
                                  equal_nan=True), call
            assert np.array_equal(got.view(np.uint32), ref.view(np.uint32)), call
    finally:
        fb.ftblas_set_injection(None)
    # the corrected element is within its row threshold of the fault-free value
    got_l = S.load(got.astype(np.float64), layout, M, N, ldc)
    assert abs(got_l[i, j] - Cl[i, j]) <= r.tau_row + 2.0 ** -22 * abs(Cl[i, j])


def test_noalloc_rejects_mn_major_operands():
    """The allocating entry point copies an MN-major operand K-major in workspace; this one
    makes no copies, so such a call is refused before any device work."""
    M, N, K = 128, 256, 64
    dA = torch.zeros(M * K, dtype=torch.int16, device="cuda")
    dB = torch.zeros(N * K, dtype=torch.int16, device="cuda")
    dC = torch.full((M * N,), 7.0, dtype=torch.float32, device="cuda")
    rc = fb.ftblas_gemm_ex_noalloc(O.COL_MAJOR, O.NO_TRANS, O.NO_TRANS, M, N, K, 1.0, dA.data_ptr(), fb.R_16BF, M,
                                   dB.data_ptr(), fb.R_16BF, K, 0.0, dC.data_ptr(), fb.R_32F, M, fb.R_32F, None, None,
                                   None, None)
    assert rc == 2  # FTBLAS_STATUS_NOT_SUPPORTED
    torch.cuda.synchronize()
    assert bool((dC == 7.0).all())


def test_noalloc_rejects_problems_beyond_its_scratch():
    # M = N = 128, K = 2^20: the encode scratch (about 40 MiB) exceeds the 16 MiB array.
    M, N, K = 128, 256, 1 << 20
    dA = torch.zeros(M * K, dtype=torch.int16, device="cuda")  # real buffers of the right size
    dB = torch.zeros(N * K, dtype=torch.int16, device="cuda")
    dC = torch.full((M * N,), 7.0, dtype=torch.float32, device="cuda")
    rc = fb.ftblas_gemm_ex_noalloc(O.COL_MAJOR, O.TRANS, O.NO_TRANS, M, N, K, 1.0, dA.data_ptr(), fb.R_16BF, K,
                                   dB.data_ptr(), fb.R_16BF, K, 0.0, dC.data_ptr(), fb.R_32F, M, fb.R_32F, None, None,
                                   None, None)
    assert rc == fb.STATUS_WORKSPACE_LIMIT
    assert "static workspace" in fb.ftblas_status_string(rc)
    torch.cuda.synchronize()
    assert bool((dC == 7.0).all())  # nothing ran
