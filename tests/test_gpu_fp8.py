"""GPU parity of the FP8 (E4M3) tensor-core ABFT GEMM (tcgen05 kind::f8f6f4, FP32
accumulation, per-tensor scales) against the CPU oracle's ACC32_E4M3 precision, through
the C ABI (ftblas_gemm_ex with A, B FTBLAS_R_8F_E4M3).

Quantisation: scale = amax / 448 in binary32, e4m3 = nearest (ties to even, saturating)
of x / scale, computed on the host. The oracle receives the dequantised operands
scale * e4m3 (exact in binary64) and the caller's alpha; the kernel forms
alpha * a_scale * b_scale in binary32, two more roundings. Values must agree within
|C - C_ref| <= 2 gamma_K(2^-22) |alpha| (|A||B|)_ij + 2^-21 (|C_ref| + |beta C_in|)
(2^-22: the accumulation unit assumed for kind::f8f6f4, twice binary32's, because a
group of 32 products is aligned to its largest term and each product truncated).
Detection, location and classification must match the oracle exactly where the injected
error is not within a factor 4 of the threshold.
"""
import numpy as np
import pytest

import oracle as O
import synth as S
from tests.helpers import record_set, report_summary

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2104_00897_gb300 as fb  # noqa: E402

U_FP8 = 2.0 ** -22


def gamma(n, u):
    return n * u / (1 - n * u)


@pytest.fixture(autouse=True)
def _fresh_injection():
    fb.ftblas_set_injection(None)
    yield
    fb.ftblas_set_injection(None)


def quantise(x):
    """Per-tensor e4m3 quantisation: (bits, binary32 scale, exact dequantised values)."""
    scale = float(np.float32(np.max(np.abs(x)) / 448.0))
    bits = S.to_e4m3_bits(x / scale)
    return bits, scale, scale * S.e4m3_bits_to_f64(bits)


class Fp8Problem:
    """Seeded FP8 operands, K-contiguous in the kernel frame (the path's requirement)."""

    def __init__(self, M, N, K, layout=O.COL_MAJOR, alpha=1.0, beta=0.0, seed=1, row_scale=False, pad=16):
        self.M, self.N, self.K, self.layout, self.alpha, self.beta = M, N, K, layout, alpha, beta
        self.ta, self.tb = (O.TRANS, O.NO_TRANS) if layout == O.COL_MAJOR else (O.NO_TRANS, O.TRANS)
        A = S.normal_matrix(seed, 0, M, K)
        if row_scale:
            A = A * S.pow2_row_scales(seed, 5, M)[:, None]
        B = S.normal_matrix(seed, 1, K, N)
        self.Abits, self.sa, self.A = quantise(A)
        self.Bbits, self.sb, self.B = quantise(B)
        self.Cin = S.bf16_bits_to_f64(S.to_bf16_bits(S.normal_matrix(seed, 2, M, N)))
        Xa = self.Abits if self.ta == O.NO_TRANS else self.Abits.T
        Xb = self.Bbits if self.tb == O.NO_TRANS else self.Bbits.T
        up16 = lambda x: (x + 15) // 16 * 16  # 16-byte rows for TMA
        lda = up16(Xa.shape[0] if layout == O.COL_MAJOR else Xa.shape[1]) + pad
        ldb = up16(Xb.shape[0] if layout == O.COL_MAJOR else Xb.shape[1]) + pad
        self.a8, self.lda = S.store(Xa, layout, ld=lda, pad_value=0)
        self.b8, self.ldb = S.store(Xb, layout, ld=ldb, pad_value=0)
        XaF = self.A if self.ta == O.NO_TRANS else self.A.T
        XbF = self.B if self.tb == O.NO_TRANS else self.B.T
        self.a64, _ = S.store(XaF, layout, ld=lda)
        self.b64, _ = S.store(XbF, layout, ld=ldb)
        self.ldc = (M if layout == O.COL_MAJOR else N) + 4
        self.c64, _ = S.store(self.Cin, layout, ld=self.ldc)

    def tile(self):
        return fb.ftblas_verification_tile(self.layout, fb.R_8F_E4M3, self.M, self.N, self.K)

    def run(self, protect=True):
        dA = torch.from_numpy(self.a8.astype(np.uint8)).cuda()
        dB = torch.from_numpy(self.b8.astype(np.uint8)).cuda()
        dC = torch.from_numpy(np.nan_to_num(self.c64, nan=0.0).astype(np.float32)).cuda()
        dS = torch.tensor([self.sa, self.sb], dtype=torch.float32, device="cuda")
        rep = fb.new_report() if protect else None
        st = torch.cuda.current_stream().cuda_stream
        args = (self.layout, self.ta, self.tb, self.M, self.N, self.K, self.alpha, dA.data_ptr(), fb.R_8F_E4M3,
                self.lda, dB.data_ptr(), fb.R_8F_E4M3, self.ldb, self.beta, dC.data_ptr(), fb.R_32F, self.ldc,
                fb.R_32F, dS.data_ptr(), dS.data_ptr() + 4, st)
        rc = fb.ftblas_gemm_ex(*args, rep.data_ptr()) if protect else fb.ftblas_gemm_ex_noabft(*args)
        fb.check(rc, "ftblas_gemm_ex")
        torch.cuda.synchronize()
        out = S.load(dC.cpu().numpy().astype(np.float64), self.layout, self.M, self.N, self.ldc)
        return out, (fb.report_from_device(rep) if protect else None)

    def oracle(self, injections=(), tiles=None):
        tr, tc, bk = self.tile()
        out, rep = O.ft_gemm(self.layout, self.ta, self.tb, self.M, self.N, self.K, self.alpha, self.a64, self.lda,
                             self.b64, self.ldb, self.beta, self.c64, self.ldc, tr, tc, bk, injections=injections,
                             tiles=tiles, precision=O.PREC_ACC32_E4M3, u_acc=U_FP8)
        return S.load(out, self.layout, self.M, self.N, self.ldc), rep

    def bound(self, ref):
        prod = np.abs(self.A) @ np.abs(self.B)
        return (2 * gamma(self.K, U_FP8) * abs(self.alpha) * prod + 2.0 ** -21 * (np.abs(ref) + abs(self.beta) *
                np.abs(self.Cin)) + 1e-30)


@pytest.mark.parametrize("layout", [O.COL_MAJOR, O.ROW_MAJOR])
@pytest.mark.parametrize("shape", [(128, 256, 128), (300, 700, 200), (256, 512, 1000), (5, 3, 130)])
def test_fp8_values_match_oracle_within_bound(layout, shape):
    M, N, K = shape
    P = Fp8Problem(M, N, K, layout, alpha=1.25, beta=0.5, seed=M + 2 * N + K)
    plain, _ = P.run(protect=False)
    got, rep = P.run(protect=True)
    ref, orep = P.oracle()
    assert np.all(np.abs(got - ref) <= P.bound(ref))
    assert np.array_equal(got, plain)  # the checksum columns do not touch the product
    assert report_summary(rep) == report_summary(orep)
    assert rep.detected == 0 and rep.status == 0


def test_fp8_scales_are_applied():
    """C = alpha * a_scale * b_scale * (A_q B_q): doubling a_scale doubles C (power-of-two
    change, exact)."""
    P = Fp8Problem(128, 240, 256, O.COL_MAJOR, alpha=1.0, beta=0.0, seed=5)
    c1, _ = P.run()
    P.sa *= 2.0
    c2, rep = P.run()
    assert np.array_equal(c2, 2.0 * c1) and rep.detected == 0


@pytest.mark.parametrize("layout", [O.COL_MAJOR, O.ROW_MAJOR])
def test_fp8_injections_match_oracle(layout):
    """Errors far above the threshold are located and corrected as the oracle does; an
    error far below it is undetected by both and stays in C."""
    P = Fp8Problem(384, 768, 512, layout, alpha=1.0, beta=0.0, seed=3)
    clean, _ = P.run()
    big = np.argsort(np.abs(clean), axis=None)[::-1]
    (i1, j1), (i2, j2) = [np.unravel_index(x, clean.shape) for x in big[[0, 40]]]
    cases = [
        [dict(i=int(i1), j=int(j1), site=fb.SITE_OUTPUT, mode=fb.MODE_ADD_REL, rel_log2=4, sign=1)],
        [dict(i=int(i2), j=int(j2), site=fb.SITE_OUTPUT, mode=fb.MODE_ADD_REL, rel_log2=3, sign=-1)],
        [dict(i=int(i2), j=int(j2), site=fb.SITE_OUTPUT, mode=fb.MODE_BITFLIP, bit=30)],
        [dict(i=int(i1), j=int(j1), site=fb.SITE_OUTPUT, mode=fb.MODE_ADD_REL, rel_log2=-40)],
    ]
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
                assert abs(got[r.i, r.j] - clean[r.i, r.j]) <= r.tau_row + 2.0 ** -21 * abs(clean[r.i, r.j])
        mask = np.ones_like(got, dtype=bool)
        for q in pts:
            mask[q["i"], q["j"]] = False
        assert np.array_equal(got[mask], clean[mask]), pts
    assert detected == len(cases) - 1


def test_fp8_row_scaled_clean_runs_have_no_false_alarm():
    """Rows of A scaled by 2^u, u in [-8, 8] before quantisation: no false alarm, and an
    error of 2^10 |C| at the largest element is corrected."""
    P = Fp8Problem(512, 960, 2048, O.COL_MAJOR, seed=17, row_scale=True)
    clean, rep = P.run()
    assert rep.detected == 0
    i, j = (int(x) for x in np.unravel_index(np.argmax(np.abs(clean)), clean.shape))
    pts = [dict(i=i, j=j, site=fb.SITE_OUTPUT, mode=fb.MODE_ADD_REL, rel_log2=10, sign=1)]
    fb.ftblas_set_injection(fb.make_injection(fixed=pts))
    got, rep = P.run()
    tr, tc, _ = P.tile()
    _, orep = P.oracle(injections=pts, tiles=[(i // tr) + (j // tc) * ((512 + tr - 1) // tr)])
    assert (rep.detected, rep.corrected) == (1, 1)
    assert record_set(rep) == record_set(orep)


def e4m3_from_definition(code):
    """Value of an E4M3 code from the format's definition (OCP 8-bit floating point: sign,
    4 exponent bits biased by 7, 3 mantissa bits; exponent field 0 subnormal; S.1111.111
    NaN; no infinities)."""
    s, e, m = code >> 7, (code >> 3) & 15, code & 7
    if e == 15 and m == 7:
        return float("nan")
    mag = (m / 8) * 2.0 ** -6 if e == 0 else (1 + m / 8) * 2.0 ** (e - 7)
    return -mag if s else mag


def test_e4m3_decoder_matches_the_format_definition_for_every_code():
    """The encode's E4M3 unpacking (paired hardware conversions) against the definition,
    code by code, and against torch's CPU float8_e4m3fn conversion; signed zeros and NaN
    included; a ragged count (not a multiple of 8) too."""
    codes = torch.arange(256, dtype=torch.int32).to(torch.uint8)
    d_codes = codes.cuda()
    out = torch.empty(256, dtype=torch.float32, device="cuda")
    fb.check(fb.ftblas_decode_e4m3(d_codes.data_ptr(), out.data_ptr(), 256, torch.cuda.current_stream().cuda_stream))
    torch.cuda.synchronize()
    got = out.cpu().numpy()
    want = np.array([e4m3_from_definition(c) for c in range(256)], dtype=np.float32)
    via_torch = codes.view(torch.float8_e4m3fn).float().numpy()
    nan = np.isnan(want)
    assert nan.sum() == 2 and np.array_equal(np.isnan(got), nan) and np.array_equal(np.isnan(via_torch), nan)
    assert np.array_equal(got[~nan].view(np.uint32), want[~nan].view(np.uint32))
    assert np.array_equal(via_torch[~nan].view(np.uint32), want[~nan].view(np.uint32))
    assert got[0x80] == 0.0 and np.signbit(got[0x80]) and got[0x7E] == 448.0 and got[0x01] == 2.0 ** -9
    part = torch.full((13,), -1.0, dtype=torch.float32, device="cuda")
    fb.check(fb.ftblas_decode_e4m3(d_codes[24:].data_ptr(), part.data_ptr(), 13, None))
    torch.cuda.synchronize()
    assert np.array_equal(part.cpu().numpy().view(np.uint32), want[24:37].view(np.uint32))
    assert fb.ftblas_decode_e4m3(None, out.data_ptr(), 1, None) == -1
    assert fb.ftblas_decode_e4m3(d_codes[3:].data_ptr(), out.data_ptr(), 1, None) == -1
    assert fb.ftblas_decode_e4m3(d_codes.data_ptr(), out.data_ptr(), -1, None) == -3
