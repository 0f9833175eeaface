"""GPU tests of a bfloat16 C on the tensor-core path (ftblas_gemm_ex with Ctype
FTBLAS_R_16BF): the product is verified, located and corrected in FP32 as for an FP32 C, and
rounded to nearest bfloat16 once: by the CTA-pair kernel's epilogue as it stores each element
(and by the resolve pass for a corrected one), or, with one CTA per tile, by a pass over an
FP32 buffer at the end. Each test runs with both kernel forms.

So a bfloat16-C call must give, bit for bit, the nearest bfloat16 of the FP32-C call on the
same operands (and, for beta != 0, on the same bfloat16 C_in), with the same report and
records, clean and with an injected fault; and the values must lie within the oracle's
accumulation bound plus one bfloat16 rounding.
"""
import numpy as np
import pytest

import oracle as O
import synth as S
from tests.helpers import record_set, report_summary

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2104_00897_gb300 as fb  # noqa: E402


def gamma(n, u):
    return n * u / (1 - n * u)


def bf16_round(x):
    """Nearest bfloat16 of binary32 values (ties to even), as float64."""
    return S.bf16_bits_to_f64(S.to_bf16_bits(np.asarray(x, dtype=np.float32).astype(np.float64)))


@pytest.fixture(params=[1, 2], ids=["one_cta", "cta_pair"])
def cta_group(request):
    prev = fb.ftblas_set_tc_cta_group(request.param)
    yield request.param
    fb.ftblas_set_tc_cta_group(prev)


@pytest.fixture(autouse=True)
def _fresh_injection():
    fb.ftblas_set_injection(None)
    yield
    fb.ftblas_set_injection(None)


class Problem:
    def __init__(self, kind, M, N, K, layout, alpha=1.25, beta=0.0, seed=1):
        self.kind, self.M, self.N, self.K, self.layout = kind, M, N, K, layout
        self.alpha, self.beta = alpha, beta
        A = S.normal_matrix(seed, 0, M, K)
        B = S.normal_matrix(seed, 1, K, N)
        if kind == "bf16":
            abits, bbits = S.to_bf16_bits(A), S.to_bf16_bits(B)
            self.A, self.B = S.bf16_bits_to_f64(abits), S.bf16_bits_to_f64(bbits)
            self.sa = self.sb = None
            self.dt, self.u, self.prec = fb.R_16BF, 2.0 ** -23, O.PREC_ACC32
        else:
            self.sa = float(np.float32(np.max(np.abs(A)) / 448.0))
            self.sb = float(np.float32(np.max(np.abs(B)) / 448.0))
            abits, bbits = S.to_e4m3_bits(A / self.sa), S.to_e4m3_bits(B / self.sb)
            self.A = self.sa * S.e4m3_bits_to_f64(abits)
            self.B = self.sb * S.e4m3_bits_to_f64(bbits)
            self.dt, self.u, self.prec = fb.R_8F_E4M3, 2.0 ** -22, O.PREC_ACC32_E4M3
        # op(A) K-contiguous in the kernel frame of either layout: column-major A^T, row-major A
        self.ta, self.tb = (O.TRANS, O.NO_TRANS) if layout == O.COL_MAJOR else (O.NO_TRANS, O.TRANS)
        Xa = abits.T if self.ta == O.TRANS else abits
        Xb = bbits.T if self.tb == O.TRANS else bbits
        self.lda = Xa.shape[0] if layout == O.COL_MAJOR else Xa.shape[1]
        self.ldb = Xb.shape[0] if layout == O.COL_MAJOR else Xb.shape[1]
        self.abits, _ = S.store(Xa, layout, ld=self.lda, pad_value=0)
        self.bbits, _ = S.store(Xb, layout, ld=self.ldb, pad_value=0)
        self.a64, _ = S.store(self.A.T if self.ta == O.TRANS else self.A, layout, ld=self.lda)
        self.b64, _ = S.store(self.B.T if self.tb == O.TRANS else self.B, layout, ld=self.ldb)
        self.ldc = (M if layout == O.COL_MAJOR else N) + 5
        self.Cin = bf16_round(S.normal_matrix(seed, 2, M, N))  # a bfloat16 C_in, exact in both forms
        self.c64, _ = S.store(self.Cin, layout, ld=self.ldc, pad_value=0.0)

    def run(self, c_bf16, protect=True):
        if self.kind == "bf16":
            dA = torch.from_numpy(self.abits.astype(np.uint16).view(np.int16)).cuda()
            dB = torch.from_numpy(self.bbits.astype(np.uint16).view(np.int16)).cuda()
            dS = None
        else:
            dA = torch.from_numpy(self.abits.astype(np.uint8)).cuda()
            dB = torch.from_numpy(self.bbits.astype(np.uint8)).cuda()
            dS = torch.tensor([self.sa, self.sb], dtype=torch.float32, device="cuda")
        if c_bf16:
            dC = torch.from_numpy(S.to_bf16_bits(self.c64).astype(np.uint16).view(np.int16)).cuda()
            ct = fb.R_16BF
        else:
            dC = torch.from_numpy(self.c64.astype(np.float32)).cuda()
            ct = fb.R_32F
        rep = fb.new_report() if protect else None
        st = torch.cuda.current_stream().cuda_stream
        args = (self.layout, self.ta, self.tb, self.M, self.N, self.K, self.alpha, dA.data_ptr(), self.dt, self.lda,
                dB.data_ptr(), self.dt, self.ldb, self.beta, dC.data_ptr(), ct, self.ldc, fb.R_32F,
                dS.data_ptr() if dS is not None else None, dS.data_ptr() + 4 if dS is not None else None, st)
        rc = fb.ftblas_gemm_ex(*args, rep.data_ptr()) if protect else fb.ftblas_gemm_ex_noabft(*args)
        fb.check(rc, "ftblas_gemm_ex")
        torch.cuda.synchronize()
        if c_bf16:
            raw = dC.cpu().numpy().view(np.uint16)
            out = S.bf16_bits_to_f64(raw)
        else:
            out = dC.cpu().numpy().astype(np.float64)
        return S.load(out, self.layout, self.M, self.N, self.ldc), (fb.report_from_device(rep) if protect else None)

    def tile(self):
        return fb.ftblas_verification_tile(self.layout, self.dt, self.M, self.N, self.K)

    def oracle(self, injections=(), tiles=None):
        tr, tc, bk = self.tile()
        out, rep = O.ft_gemm(self.layout, self.ta, self.tb, self.M, self.N, self.K, self.alpha, self.a64, self.lda,
                             self.b64, self.ldb, self.beta, self.c64, self.ldc, tr, tc, bk, injections=injections,
                             tiles=tiles, precision=self.prec, u_acc=self.u)
        return S.load(out, self.layout, self.M, self.N, self.ldc), rep

    def bound(self, ref):
        prod = np.abs(self.A) @ np.abs(self.B)
        return (2 * gamma(self.K, self.u) * abs(self.alpha) * prod + 2.0 ** -21 * (np.abs(ref) + abs(self.beta) *
                np.abs(self.Cin)) + 2.0 ** -8 * np.abs(ref) + 1e-30)


CASES = [("bf16", O.COL_MAJOR, 0.0), ("bf16", O.ROW_MAJOR, 0.5), ("fp8", O.COL_MAJOR, -0.75), ("fp8", O.ROW_MAJOR, 0.0)]


@pytest.mark.parametrize("kind,layout,beta", CASES)
def test_bf16_c_is_the_rounded_fp32_c(kind, layout, beta, cta_group):
    P = Problem(kind, 300, 517, 260, layout, beta=beta, seed=31 + layout)
    c32, r32 = P.run(False)
    c16, r16 = P.run(True)
    assert np.array_equal(c16, bf16_round(c32))
    assert report_summary(r16) == report_summary(r32) and r16.detected == 0 and r16.status == 0
    ref, orep = P.oracle()
    assert report_summary(r16) == report_summary(orep)
    assert np.all(np.abs(c16 - ref) <= P.bound(ref))
    # unprotected calls likewise
    u32, _ = P.run(False, protect=False)
    u16, _ = P.run(True, protect=False)
    assert np.array_equal(u16, bf16_round(u32))


@pytest.mark.parametrize("kind,layout,beta", CASES)
def test_bf16_c_fault_corrected_in_fp32(kind, layout, beta, cta_group):
    P = Problem(kind, 300, 517, 260, layout, beta=beta, seed=41 + layout)
    clean32, _ = P.run(False)
    i, j = (int(x) for x in np.unravel_index(np.argmax(np.abs(clean32)), clean32.shape))
    pt = dict(i=i, j=j, site=fb.SITE_OUTPUT, mode=fb.MODE_ADD_REL, rel_log2=12, sign=1)
    fb.ftblas_set_injection(fb.make_injection(fixed=[pt]))
    g32, r32 = P.run(False)
    g16, r16 = P.run(True)
    fb.ftblas_set_injection(None)
    assert report_summary(r16) == report_summary(r32) and r16.corrected == 1
    assert record_set(r16) == record_set(r32) == [(i, j, fb.KIND_CORRECTED)]
    assert np.array_equal(g16, bf16_round(g32))
    _, orep = P.oracle(injections=[pt])
    assert record_set(orep) == [(i, j, fb.KIND_CORRECTED)]


@pytest.mark.parametrize("kind", ["bf16", "fp8"])
def test_bf16_c_over_several_rounds(kind, cta_group):
    """More tiles than one persistent round, a ragged last column block, beta != 0 and one
    fault: the bfloat16 C is the rounded FP32 C of the same call form, bit for bit."""
    P = Problem(kind, 2304, 4100, 520, O.COL_MAJOR, beta=0.5, seed=57)
    clean32, _ = P.run(False)
    # the largest element of a tile of the ragged last column block (columns 3968..4099)
    blk = np.abs(clean32[1408:1536, 3968:])
    di, dj = np.unravel_index(np.argmax(blk), blk.shape)
    i, j = 1408 + int(di), 3968 + int(dj)
    pt = dict(i=i, j=j, site=fb.SITE_OUTPUT, mode=fb.MODE_ADD_REL, rel_log2=14, sign=-1)
    fb.ftblas_set_injection(fb.make_injection(fixed=[pt]))
    g32, r32 = P.run(False)
    g16, r16 = P.run(True)
    fb.ftblas_set_injection(None)
    assert record_set(r16) == record_set(r32) == [(i, j, fb.KIND_CORRECTED)]
    assert np.array_equal(g16, bf16_round(g32))
    others = np.ones_like(g32, dtype=bool)
    others[i, j] = False
    assert np.array_equal(g32[others], clean32[others])
    (r,) = r32.records()
    assert abs(g32[i, j] - clean32[i, j]) <= r.tau_row + 2.0 ** -21 * abs(clean32[i, j])
    c16, r = P.run(True)
    assert np.array_equal(c16, bf16_round(clean32)) and r.detected == 0
    u32, _ = P.run(False, protect=False)
    u16, _ = P.run(True, protect=False)
    assert np.array_equal(u16, bf16_round(u32))


def test_bf16_c_scaled_when_there_is_no_product():
    """K = 0 and alpha = 0 leave C = beta C, computed on the bfloat16 values."""
    for K, alpha in ((0, 1.0), (64, 0.0)):
        P = Problem("bf16", 70, 90, max(K, 1), O.COL_MAJOR, alpha=alpha, beta=1.5, seed=7)
        P.K = K
        got, rep = P.run(True)
        assert np.array_equal(got, bf16_round(1.5 * P.Cin))
        assert rep.detected == 0


def test_noalloc_refuses_a_bf16_c():
    M = N = K = 64
    a = torch.zeros((M, K), dtype=torch.bfloat16, device="cuda")
    b = torch.zeros((N, K), dtype=torch.bfloat16, device="cuda")
    c = torch.zeros((N, M), dtype=torch.bfloat16, device="cuda")
    rc = fb.ftblas_gemm_ex_noalloc(O.COL_MAJOR, O.TRANS, O.NO_TRANS, M, N, K, 1.0, a.data_ptr(), fb.R_16BF, K,
                                   b.data_ptr(), fb.R_16BF, K, 0.0, c.data_ptr(), fb.R_16BF, M, fb.R_32F, None, None,
                                   torch.cuda.current_stream().cuda_stream, None)
    assert rc == fb.STATUS_NOT_SUPPORTED


def test_gemm_api_bf16_output_and_linear_layer_dtype():
    a = torch.randn(256, 192, device="cuda").to(torch.bfloat16)
    b = torch.randn(192, 320, device="cuda").to(torch.bfloat16)
    c32 = fb.gemm(a, b)
    c16 = fb.gemm(a, b, out_dtype=torch.bfloat16)
    assert c16.dtype == torch.bfloat16
    assert torch.equal(c16, c32.to(torch.bfloat16))
    x = a.clone().requires_grad_(True)
    w = b.t().contiguous().requires_grad_(True)
    y = fb.FTLinearFn.apply(x, w, None)
    assert y.dtype == torch.bfloat16 and torch.equal(y, c16)
