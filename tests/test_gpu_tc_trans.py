"""GPU parity of the tensor-core forms for every transpose combination, through the C ABI
(ftblas_gemm_ex), against the oracle's ACC32 / ACC32_E4M3 model.

The product kernel reads operands K-contiguous; an operand stored the other way is copied
K-major by the library first. Every combination of layout and transposes must therefore give
the values of the K-contiguous call within the accumulation bound (in fact bit for bit: the
kernel sees the same K-major data), the oracle's reports, and with an injected fault the
oracle's records. Leading dimensions that are not multiples of 16 bytes exercise the copy's
element-by-element path.
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


def gamma(n, u):
    return n * u / (1 - n * u)


@pytest.fixture(autouse=True)
def _fresh_injection():
    fb.ftblas_set_injection(None)
    yield
    fb.ftblas_set_injection(None)


class TransProblem:
    def __init__(self, kind, M, N, K, layout, ta, tb, alpha=1.25, beta=0.5, seed=1, pad=0):
        self.kind, self.M, self.N, self.K = kind, M, N, K
        self.layout, self.ta, self.tb, self.alpha, self.beta = layout, ta, tb, alpha, beta
        A = S.normal_matrix(seed, 0, M, K)
        B = S.normal_matrix(seed, 1, K, N)
        if kind == "bf16":
            abits, bbits = S.to_bf16_bits(A), S.to_bf16_bits(B)
            self.A, self.B = S.bf16_bits_to_f64(abits), S.bf16_bits_to_f64(bbits)
            self.sa = self.sb = None
            self.dtype, self.u, self.prec, self.out_round = fb.R_16BF, 2.0 ** -23, O.PREC_ACC32, 2.0 ** -22
        else:
            self.sa = float(np.float32(np.max(np.abs(A)) / 448.0))
            self.sb = float(np.float32(np.max(np.abs(B)) / 448.0))
            abits, bbits = S.to_e4m3_bits(A / self.sa), S.to_e4m3_bits(B / self.sb)
            self.A = self.sa * S.e4m3_bits_to_f64(abits)
            self.B = self.sb * S.e4m3_bits_to_f64(bbits)
            self.dtype, self.u, self.prec, self.out_round = fb.R_8F_E4M3, 2.0 ** -22, O.PREC_ACC32_E4M3, 2.0 ** -21
        self.Cin = S.bf16_bits_to_f64(S.to_bf16_bits(S.normal_matrix(seed, 2, M, N)))
        Xa = abits if ta == O.NO_TRANS else abits.T
        Xb = bbits if tb == O.NO_TRANS else bbits.T
        lda = (Xa.shape[0] if layout == O.COL_MAJOR else Xa.shape[1]) + pad
        ldb = (Xb.shape[0] if layout == O.COL_MAJOR else Xb.shape[1]) + pad
        self.abits, self.lda = S.store(Xa, layout, ld=lda, pad_value=0)
        self.bbits, self.ldb = S.store(Xb, layout, ld=ldb, pad_value=0)
        XaF = self.A if ta == O.NO_TRANS else self.A.T
        XbF = self.B if tb == O.NO_TRANS else self.B.T
        self.a64, _ = S.store(XaF, layout, ld=lda)
        self.b64, _ = S.store(XbF, layout, ld=ldb)
        self.ldc = (M if layout == O.COL_MAJOR else N) + 3
        self.c64, _ = S.store(self.Cin, layout, ld=self.ldc)

    def tile(self):
        return fb.ftblas_verification_tile(self.layout, self.dtype, self.M, self.N, self.K)

    def run(self, protect=True):
        if self.kind == "bf16":
            dA = torch.from_numpy(self.abits.astype(np.uint16).view(np.int16)).cuda()
            dB = torch.from_numpy(self.bbits.astype(np.uint16).view(np.int16)).cuda()
            dS = None
        else:
            dA = torch.from_numpy(self.abits.astype(np.uint8)).cuda()
            dB = torch.from_numpy(self.bbits.astype(np.uint8)).cuda()
            dS = torch.tensor([self.sa, self.sb], dtype=torch.float32, device="cuda")
        dC = torch.from_numpy(np.nan_to_num(self.c64, nan=0.0).astype(np.float32)).cuda()
        rep = fb.new_report() if protect else None
        st = torch.cuda.current_stream().cuda_stream
        args = (self.layout, self.ta, self.tb, self.M, self.N, self.K, self.alpha, dA.data_ptr(), self.dtype,
                self.lda, dB.data_ptr(), self.dtype, self.ldb, self.beta, dC.data_ptr(), fb.R_32F, self.ldc,
                fb.R_32F, dS.data_ptr() if dS is not None else None, dS.data_ptr() + 4 if dS is not None else None,
                st)
        rc = fb.ftblas_gemm_ex(*args, rep.data_ptr()) if protect else fb.ftblas_gemm_ex_noabft(*args)
        fb.check(rc, "ftblas_gemm_ex")
        torch.cuda.synchronize()
        out = S.load(dC.cpu().numpy().astype(np.float64), self.layout, self.M, self.N, self.ldc)
        return out, (fb.report_from_device(rep) if protect else None)

    def oracle(self, injections=(), tiles=None):
        tr, tc, bk = self.tile()
        out, rep = O.ft_gemm(self.layout, self.ta, self.tb, self.M, self.N, self.K, self.alpha, self.a64, self.lda,
                             self.b64, self.ldb, self.beta, self.c64, self.ldc, tr, tc, bk, injections=injections,
                             tiles=tiles, precision=self.prec, u_acc=self.u)
        return S.load(out, self.layout, self.M, self.N, self.ldc), rep

    def bound(self, ref):
        prod = np.abs(self.A) @ np.abs(self.B)
        return (2 * gamma(self.K, self.u) * abs(self.alpha) * prod
                + self.out_round * (np.abs(ref) + abs(self.beta) * np.abs(self.Cin)) + 1e-30)


@pytest.mark.parametrize("kind", ["bf16", "fp8"])
@pytest.mark.parametrize("layout,ta,tb", COMBOS)
def test_every_transpose_combination_matches_the_oracle(kind, layout, ta, tb):
    P = TransProblem(kind, 300, 530, 260, layout, ta, tb, seed=3 + ta + tb, pad=0)
    got, rep = P.run()
    ref, orep = P.oracle()
    assert np.all(np.abs(got - ref) <= P.bound(ref))
    assert report_summary(rep) == report_summary(orep) and rep.detected == 0 and rep.status == 0
    plain, _ = P.run(protect=False)
    assert np.array_equal(got, plain)
    # the same product through the K-contiguous combination of this layout: identical bits
    kt = (O.TRANS, O.NO_TRANS) if layout == O.COL_MAJOR else (O.NO_TRANS, O.TRANS)
    Q = TransProblem(kind, 300, 530, 260, layout, *kt, seed=3 + ta + tb, pad=0)
    same, _ = Q.run()
    assert np.array_equal(got, same)


@pytest.mark.parametrize("kind", ["bf16", "fp8"])
@pytest.mark.parametrize("layout", [O.COL_MAJOR, O.ROW_MAJOR])
def test_unaligned_mn_major_operands_and_a_fault(kind, layout):
    """Both operands MN-major with leading dimensions that are not multiples of 16 bytes
    (the copy's element-by-element path), beta != 0, and one output fault located and
    corrected as the oracle does."""
    ta, tb = (O.NO_TRANS, O.TRANS) if layout == O.COL_MAJOR else (O.TRANS, O.NO_TRANS)
    P = TransProblem(kind, 257, 611, 333, layout, ta, tb, seed=17, pad=3)
    clean, rep = P.run()
    ref, orep = P.oracle()
    assert np.all(np.abs(clean - ref) <= P.bound(ref))
    assert report_summary(rep) == report_summary(orep)
    i, j = (int(x) for x in np.unravel_index(np.argmax(np.abs(clean)), clean.shape))
    pt = dict(i=i, j=j, site=fb.SITE_OUTPUT, mode=fb.MODE_ADD_REL, rel_log2=12, sign=1)
    fb.ftblas_set_injection(fb.make_injection(fixed=[pt]))
    got, rep = P.run()
    _, orep = P.oracle(injections=[pt])
    assert report_summary(rep) == report_summary(orep) and rep.corrected == 1
    assert record_set(rep) == record_set(orep) == [(i, j, fb.KIND_CORRECTED)]
    (r,) = rep.records()
    assert abs(got[i, j] - clean[i, j]) <= r.tau_row + P.out_round * abs(clean[i, j])
