"""The torch-level API: gemm() on tensors and the protected linear layer FTLinearFn
(Y = X W^T, whose backward runs dX = dY W and dW = dY^T X as two more protected GEMMs).

- FP64: central finite differences (torch.autograd.gradcheck) at X 64 x 48, W 32 x 48,
  i.e. the GEMM (M, N, K) = (64, 32, 48), pin the backward; forward and gradients equal
  the oracle's products within the FP64 criterion, with one corrected fault per pass.
- BF16: forward and gradients (bfloat16, rounded once by the library from the verified
  FP32 products) against the oracle's products of the same BF16 values (binary32
  accumulation) within the accumulation bound plus the bfloat16 rounding; one injected
  output fault per GEMM pass is corrected in all three.
"""
import numpy as np
import pytest

import oracle as O
import synth as S

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


def ref_gemm(A, B):
    """Oracle product A @ B of exact binary64 values, binary32-rounded (ACC32)."""
    M, K = A.shape
    N = B.shape[1]
    a, lda = S.store(A, O.COL_MAJOR)
    b, ldb = S.store(B, O.COL_MAJOR)
    out = O.gemm(O.COL_MAJOR, O.NO_TRANS, O.NO_TRANS, M, N, K, 1.0, a, lda, b, ldb, 0.0, None, M,
                 precision=O.PREC_ACC32)
    return S.load(out, O.COL_MAJOR, M, N, M)


def ref_gemm64(A, B):
    """Oracle product A @ B in binary64 (the GEMM definition, ascending k)."""
    M, K = A.shape
    N = B.shape[1]
    a, lda = S.store(np.ascontiguousarray(A), O.COL_MAJOR)
    b, ldb = S.store(np.ascontiguousarray(B), O.COL_MAJOR)
    out = O.gemm(O.COL_MAJOR, O.NO_TRANS, O.NO_TRANS, M, N, K, 1.0, a, lda, b, ldb, 0.0, None, M)
    return S.load(out, O.COL_MAJOR, M, N, M)


def test_fp64_linear_gradcheck():
    x = torch.from_numpy(S.uniform_matrix(41, 0, 64, 48)).cuda().requires_grad_(True)
    w = torch.from_numpy(S.uniform_matrix(41, 1, 32, 48)).cuda().requires_grad_(True)
    mon = fb.FTMonitor()
    assert torch.autograd.gradcheck(lambda a, b: fb.FTLinearFn.apply(a, b, mon), (x, w), eps=1e-6)
    s = mon.summary()
    assert s["calls"] > 0 and s["detected"] == 0 and s["status"] == 0


def test_fp64_linear_matches_oracle_and_corrects_one_fault_per_pass():
    X = S.uniform_matrix(42, 0, 200, 96)
    W = S.uniform_matrix(42, 1, 150, 96)
    dY = S.uniform_matrix(42, 2, 200, 150)
    x = torch.from_numpy(X).cuda().requires_grad_(True)
    w = torch.from_numpy(W).cuda().requires_grad_(True)
    fb.ftblas_set_injection(fb.make_injection(seed=5, site=fb.SITE_ACCUM, mode=fb.MODE_BITFLIP, bit_lo=52, bit_hi=60,
                                              every_n_launches=1, errors_per_launch=1))
    mon = fb.FTMonitor()
    y = fb.FTLinearFn.apply(x, w, mon)
    y.backward(torch.from_numpy(dY).cuda())
    s = mon.summary()
    assert (s["calls"], s["detected"], s["corrected"], s["uncorrectable"]) == (3, 3, 3, 0)
    fb.ftblas_set_injection(None)
    # the oracle's reference products Y = X W^T, dX = dY W, dW = dY^T X: within the FP64
    # criterion max|C - C_ref| / (max|A| max|B| K) <= 1e-15, and within the rounding bound
    for got, A, B in ((y, X, W.T), (x.grad, dY, W), (w.grad, dY.T, X)):
        ref = ref_gemm64(A, B)
        g = got.detach().cpu().numpy()
        K = A.shape[1]
        assert np.abs(g - ref).max() / (np.abs(A).max() * np.abs(B).max() * K) <= 1e-15
        bound = 2 * gamma(K, 2.0 ** -53) * (np.abs(A) @ np.abs(B)) + 1e-300
        assert np.all(np.abs(g - ref) <= bound)


def test_bf16_linear_forward_backward_with_faults():
    T, n_in, n_out = 512, 256, 384
    X = S.bf16_bits_to_f64(S.to_bf16_bits(S.normal_matrix(43, 0, T, n_in)))
    W = S.bf16_bits_to_f64(S.to_bf16_bits(S.normal_matrix(43, 1, n_out, n_in, std=0.02)))
    dY = S.normal_matrix(43, 2, T, n_out)
    x = torch.from_numpy(X).cuda().to(torch.bfloat16).requires_grad_(True)
    w = torch.from_numpy(W).cuda().to(torch.bfloat16).requires_grad_(True)
    fb.ftblas_set_injection(fb.make_injection(seed=9, site=fb.SITE_OUTPUT, mode=fb.MODE_ADD_REL, log2_lo=12,
                                              log2_hi=14, every_n_launches=1, errors_per_launch=1))
    mon = fb.FTMonitor()
    y = fb.FTLinearFn.apply(x, w, mon)
    assert y.dtype == torch.bfloat16
    dy = torch.from_numpy(dY).cuda().float()
    y.backward(dy.to(torch.bfloat16))
    s = mon.summary()
    assert (s["calls"], s["detected"], s["corrected"], s["uncorrectable"], s["status"]) == (3, 3, 3, 0, 0)
    fb.ftblas_set_injection(None)
    dYq = S.bf16_bits_to_f64(S.to_bf16_bits(dy.double().cpu().numpy()))  # dY rounded to bfloat16, as the layer does
    # forward and gradients in bfloat16 (the FP32 result rounded once: 2^-8 relative covers
    # it with the FP32 rounding). A corrected element comes from the row checksum: within
    # its record's row threshold instead.
    calls = ((y.detach(), X, W.T, 2.0 ** -8), (x.grad, dYq, W, 2.0 ** -8), (w.grad, dYq.T, X, 2.0 ** -8))
    for (got, A, B, out_round), buf in zip(calls, mon.reports):
        ref = ref_gemm(A, B)
        bound = 2 * gamma(A.shape[1], U32) * (np.abs(A) @ np.abs(B)) + out_round * np.abs(ref) + 1e-30
        (r,) = fb.report_from_device(buf).records()
        assert r.kind == fb.KIND_CORRECTED
        bound[r.i, r.j] += r.tau_row * (1 + out_round)
        assert np.all(np.abs(got.double().cpu().numpy() - ref) <= bound)
    assert x.grad.dtype == torch.bfloat16 and w.grad.dtype == torch.bfloat16


def test_gemm_api_fp8_and_column_major_output():
    f8 = getattr(torch, "float8_e4m3fn", None)
    if f8 is None:
        pytest.skip("torch without float8_e4m3fn")
    M, N, K = 256, 300, 512
    Aq = S.e4m3_bits_to_f64(S.to_e4m3_bits(S.normal_matrix(44, 0, M, K) * 64))
    Bq = S.e4m3_bits_to_f64(S.to_e4m3_bits(S.normal_matrix(44, 1, K, N) * 64))
    a = torch.from_numpy(Aq).cuda().to(f8)
    b = torch.from_numpy(Bq).cuda().to(f8)
    assert np.array_equal(a.double().cpu().numpy(), Aq)  # exact round trip: torch and synth agree on e4m3
    sa = torch.tensor([0.5], dtype=torch.float32, device="cuda")
    sb = torch.tensor([0.25], dtype=torch.float32, device="cuda")
    rep = fb.new_report()
    c = fb.gemm(a, b, report=rep, a_scale=sa, b_scale=sb)
    ref = 0.125 * ref_gemm(Aq, Bq)
    bound = 0.125 * 2 * gamma(K, 2.0 ** -22) * (np.abs(Aq) @ np.abs(Bq)) + 2.0 ** -21 * np.abs(ref) + 1e-30
    assert np.all(np.abs(c.double().cpu().numpy() - ref) <= bound)
    r = fb.report_from_device(rep)
    assert r.detected == 0 and r.tiles_checked > 0
    # column-major c (the transposed call) gives the same values
    cc = torch.empty((N, M), dtype=torch.float32, device="cuda").t()
    fb.gemm(a, b, c=cc, a_scale=sa, b_scale=sb)
    assert np.all(np.abs(cc.double().cpu().numpy() - ref) <= bound)
