"""The unfused comparator ftblas_dgemm_unfused (checksum passes around cuBLAS's DGEMM)
against the CPU oracle, through the C ABI.

Same tiles, detections, classifications and error locations as the oracle for errors far
from the threshold (its magnitude bound is looser than the fused kernel's); FP64 values
within max|C - C_ref| / (max|A| max|B| K) <= 1e-15; a corrected element within the row
threshold of the fault-free value (the checksum-form correction of a library product is
not bit-exact).
"""
import numpy as np
import pytest

import oracle as O
import synth as S
from tests.helpers import Problem, record_set, report_summary

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2104_00897_gb300 as fb  # noqa: E402

COMBOS = [(l, a, b) for l in (O.COL_MAJOR, O.ROW_MAJOR) for a in (O.NO_TRANS, O.TRANS) for b in (O.NO_TRANS, O.TRANS)]


@pytest.fixture(autouse=True)
def _fresh_injection():
    fb.ftblas_set_injection(None)
    yield
    fb.ftblas_set_injection(None)


def run_unfused(P: Problem):
    dA = torch.from_numpy(np.ascontiguousarray(P.a)).cuda()
    dB = torch.from_numpy(np.ascontiguousarray(P.b)).cuda()
    dC = torch.from_numpy(np.ascontiguousarray(P.c)).cuda()
    rep = fb.new_report()
    st = torch.cuda.current_stream().cuda_stream
    rc = fb.ftblas_dgemm_unfused(P.layout, P.ta, P.tb, P.M, P.N, P.K, P.alpha, dA.data_ptr(), P.lda, dB.data_ptr(),
                                 P.ldb, P.beta, dC.data_ptr(), P.ldc, st, rep.data_ptr())
    fb.check(rc, "ftblas_dgemm_unfused")
    torch.cuda.synchronize()
    return S.load(dC.cpu().numpy(), P.layout, P.M, P.N, P.ldc), fb.report_from_device(rep)


def tile_of(P):
    """The comparator verifies 128 x 128 tiles at every size (k-tile depth 32)."""
    return 128, 128, 32


@pytest.mark.parametrize("layout,ta,tb", COMBOS)
@pytest.mark.parametrize("shape", [(256, 256, 256), (300, 200, 130), (129, 385, 64)])
def test_unfused_values_and_clean_report(layout, ta, tb, shape):
    M, N, K = shape
    P = Problem(M, N, K, layout, ta, tb, alpha=1.5, beta=0.5, seed=M + N + K, pad=3)
    got, rep = run_unfused(P)
    tr, tc, bk = tile_of(P)
    ref, orep = P.oracle_ft(tr, tc, bk)
    assert P.normalized_error(got, ref) <= 1e-15
    assert report_summary(rep) == report_summary(orep)
    assert rep.detected == 0 and rep.status == 0


@pytest.mark.parametrize("layout", [O.COL_MAJOR, O.ROW_MAJOR])
def test_unfused_injections_match_oracle(layout):
    P = Problem(384, 256, 512, layout, O.NO_TRANS, O.NO_TRANS, alpha=1.0, beta=0.5, seed=7)
    clean, _ = run_unfused(P)
    tr, tc, bk = tile_of(P)
    cases = [
        [dict(i=17, j=33, site=fb.SITE_OUTPUT, mode=fb.MODE_ADD_REL, rel_log2=4, sign=1)],
        [dict(i=200, j=130, site=fb.SITE_OUTPUT, mode=fb.MODE_BITFLIP, bit=60)],
        [dict(i=300, j=5, site=fb.SITE_OUTPUT, mode=fb.MODE_BITFLIP, bit=62)],          # to infinity or tiny
        [dict(i=3, j=3, site=fb.SITE_OUTPUT, mode=fb.MODE_ADD_REL, rel_log2=3),
         dict(i=4, j=5, site=fb.SITE_OUTPUT, mode=fb.MODE_ADD_REL, rel_log2=3)],        # two in a tile
        [dict(i=10, j=140, site=fb.SITE_OUTPUT, mode=fb.MODE_ADD_REL, rel_log2=2),
         dict(i=300, j=20, site=fb.SITE_OUTPUT, mode=fb.MODE_ADD_REL, rel_log2=2)],     # two tiles
        [dict(i=99, j=99, site=fb.SITE_OUTPUT, mode=fb.MODE_ADD_REL, rel_log2=-70)],    # far below threshold
    ]
    if layout == O.COL_MAJOR:
        cases.append([dict(i=250, j=100, site=fb.SITE_CHECKSUM, mode=fb.MODE_ADD_REL, rel_log2=10, sign=1)])
    for pts in cases:
        fb.ftblas_set_injection(fb.make_injection(fixed=pts))
        got, rep = run_unfused(P)
        _, orep = P.oracle_ft(tr, tc, bk, injections=pts)
        assert report_summary(rep) == report_summary(orep), pts
        assert record_set(rep) == record_set(orep), pts
        for r in rep.records():
            if r.kind == fb.KIND_CORRECTED:
                err = abs(got[r.i, r.j] - clean[r.i, r.j])
                assert err <= 1e-15 * np.abs(P.A).max() * np.abs(P.B).max() * P.K, pts
                assert not np.isfinite(r.tau_row) or err <= r.tau_row, pts
        touched = {(q["i"], q["j"]) for q in pts}
        mask = np.ones_like(got, dtype=bool)
        for (i, j) in touched:
            mask[i, j] = False
        assert np.array_equal(got[mask], clean[mask]), pts


def test_unfused_seeded_draw_one_fault_per_launch():
    P = Problem(512, 512, 256, O.COL_MAJOR, O.NO_TRANS, O.NO_TRANS, alpha=1.0, beta=0.0, seed=9)
    fb.ftblas_set_injection(fb.make_injection(seed=3, site=fb.SITE_OUTPUT, mode=fb.MODE_BITFLIP, bit_lo=52,
                                              bit_hi=62, every_n_launches=1, errors_per_launch=3))
    got, rep = run_unfused(P)
    assert (rep.detected, rep.corrected, rep.uncorrectable) == (3, 3, 0)
    fb.ftblas_set_injection(None)
    clean, _ = run_unfused(P)
    for r in rep.records():
        # an exponent flip can leave NaN in the row, and then its threshold is NaN too
        if np.isfinite(r.tau_row):
            assert abs(got[r.i, r.j] - clean[r.i, r.j]) <= r.tau_row
        assert abs(got[r.i, r.j] - clean[r.i, r.j]) <= 1e-15 * np.abs(P.A).max() * np.abs(P.B).max() * P.K
