"""GPU parity of the FP64 ABFT GEMM against the CPU oracle, through the C ABI.

The bar (FT-BLAS Sections II.A, V, VI.C): the same tiles checked, the same detections,
corrections and error locations as the oracle, bit for bit; the corrected output equal
to the fault-free output of the same engine, bit for bit; and the FP64 values within
max|C - C_ref| / (max|A| max|B| K) <= 1e-15 of the oracle.
"""
import numpy as np
import pytest

import oracle as O
import synth as S
from tests.helpers import Problem, record_set, report_summary

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2104_00897_gb300 as fb  # noqa: E402

TOL = 1e-15
COMBOS = [(l, a, b) for l in (O.COL_MAJOR, O.ROW_MAJOR) for a in (O.NO_TRANS, O.TRANS) for b in (O.NO_TRANS, O.TRANS)]
# kernel variants: (engine, forced tile edge or 0 for the automatic choice, which is 64 for
# the small problems here and 128 from 4096 on)
ENGINES = [(fb.ENGINE_DFMA, 0), (fb.ENGINE_DFMA, 128), (fb.ENGINE_DMMA, 0)]
ENGINE_IDS = ["dfma-auto", "dfma-128", "dmma"]


def use(variant):
    engine, edge = variant
    fb.ftblas_set_fp64_engine(engine)
    fb.ftblas_set_fp64_tile(edge)


@pytest.fixture(autouse=True)
def _fresh_injection():
    fb.ftblas_set_injection(None)
    prev = fb.ftblas_set_fp64_engine(fb.ENGINE_DFMA)
    prev_tile = fb.ftblas_set_fp64_tile(0)
    yield
    fb.ftblas_set_injection(None)
    fb.ftblas_set_fp64_engine(prev)
    fb.ftblas_set_fp64_tile(prev_tile)


def dev(x):
    return torch.from_numpy(np.ascontiguousarray(x)).to("cuda")


def run_gpu(P: Problem, protect=True, c_init=None, a=None, b=None, lda=None, ldb=None):
    """Run the GEMM on the GPU through the C ABI; returns (logical C, FtReport or None)."""
    dA = dev(P.a if a is None else a)
    dB = dev(P.b if b is None else b)
    dC = dev(P.c if c_init is None else c_init)
    rep = fb.new_report() if protect else None
    st = torch.cuda.current_stream().cuda_stream
    args = (P.layout, P.ta, P.tb, P.M, P.N, P.K, P.alpha, dA.data_ptr(), P.lda if lda is None else lda,
            dB.data_ptr(), P.ldb if ldb is None else ldb, P.beta, dC.data_ptr(), P.ldc, st)
    if protect:
        rc = fb.ftblas_dgemm(*args, rep.data_ptr())
    else:
        rc = fb.ftblas_dgemm_noabft(*args)
    fb.check(rc)
    torch.cuda.synchronize()
    out = S.load(dC.cpu().numpy(), P.layout, P.M, P.N, P.ldc)
    return out, (fb.report_from_device(rep) if protect else None)


def tile_of(P):
    return fb.ftblas_verification_tile(P.layout, fb.R_64F, P.M, P.N, P.K)


def seeded_point(seed, M, N):
    i, j = S.randint(seed, 99, 2, 0, 1 << 30)
    return int(i % M), int(j % N)


# ---------------------------------------------------------------------------------------
@pytest.mark.parametrize("engine", ENGINES, ids=ENGINE_IDS)
def test_config1_256_fault_free_and_bit52_flip(engine):
    """FP64 column-major 256^3, alpha = 1, beta = 0, U[-1,1]: a fault-free run, then one
    flip of bit 52 of C(i,j) at seeded (i,j) after K/2 products."""
    use(engine)
    P = Problem(256, 256, 256, alpha=1.0, beta=0.0, seed=20210601)
    tr, tc, bk = tile_of(P)
    clean, rep = run_gpu(P)
    assert fb.ftblas_last_launch_used_tma() == 1
    oclean, orep = P.oracle_ft(tr, tc, bk)
    nt = (256 // tr) * (256 // tc)
    assert report_summary(rep) == report_summary(orep) == (nt, 0, 0, 0, 0, 0)
    assert P.normalized_error(clean, oclean) <= TOL
    assert bk * ((256 // bk) // 2) == 128  # the flip happens after K/2 products
    i, j = seeded_point(20210601, 256, 256)
    pt = dict(i=i, j=j, site=fb.SITE_ACCUM, mode=fb.MODE_BITFLIP, bit=52)
    fb.ftblas_set_injection(fb.make_injection(fixed=[pt]))
    fixed, rep = run_gpu(P)
    ofixed, orep = P.oracle_ft(tr, tc, bk, injections=[dict(pt, site=O.SITE_ACCUM)])
    assert report_summary(rep) == report_summary(orep) == (nt, 1, 1, 0, 0, 0)
    assert record_set(rep) == record_set(orep) == [(i, j, fb.KIND_CORRECTED)]
    r = rep.records()[0]
    assert abs(r.delta_row) > r.tau_row and abs(r.delta_col) > r.tau_col
    assert np.array_equal(fixed.view(np.uint64), clean.view(np.uint64))  # bit-exact correction
    assert np.array_equal(ofixed.view(np.uint64), oclean.view(np.uint64))
    assert r.value_after == clean[i, j] and r.value_before != clean[i, j]


@pytest.mark.parametrize("engine", ENGINES, ids=ENGINE_IDS)
@pytest.mark.parametrize("layout,ta,tb", COMBOS)
@pytest.mark.parametrize("shape", [(300, 200, 77), (129, 257, 33), (1, 1, 1), (5, 300, 1000)])
def test_layouts_and_ragged_shapes_match_oracle(engine, layout, ta, tb, shape):
    use(engine)
    M, N, K = shape
    P = Problem(M, N, K, layout, ta, tb, alpha=1.5, beta=0.5, seed=7 + M + N + K, pad="even")
    got, rep = run_gpu(P)
    assert fb.ftblas_last_launch_used_tma() == 1
    tr, tc, bk = tile_of(P)
    ref, orep = P.oracle_ft(tr, tc, bk)
    assert report_summary(rep) == report_summary(orep)
    assert rep.detected == 0 and rep.status == 0
    assert P.normalized_error(got, ref) <= TOL


@pytest.mark.parametrize("engine", ENGINES, ids=ENGINE_IDS)
@pytest.mark.parametrize("layout", [O.COL_MAJOR, O.ROW_MAJOR])
def test_seeded_draw_parity_over_launches(engine, layout):
    """The library's seeded draw and the oracle's (each its own SplitMix64) pick the same
    points; every launch detects, locates and corrects exactly what the oracle does."""
    use(engine)
    P = Problem(520, 390, 200, layout, O.NO_TRANS, O.TRANS, alpha=1.5, beta=0.5, seed=11)
    tr, tc, bk = tile_of(P)
    clean, _ = run_gpu(P)
    assert fb.ftblas_last_launch_used_tma() == 1
    seed = 424242
    fb.ftblas_set_injection(fb.make_injection(seed=seed, every_n_launches=2, errors_per_launch=5, bit_lo=40,
                                              bit_hi=62))
    injected_launches = 0
    for launch in range(4):
        got, rep = run_gpu(P)
        pts = O.draw_injections(seed, launch, 2, 5, O.SITE_ACCUM, O.MODE_BITFLIP, 40, 62, 0, 0, P.M, P.N, tr, tc)
        ref, orep = P.oracle_ft(tr, tc, bk, injections=pts)
        assert report_summary(rep) == report_summary(orep)
        assert record_set(rep) == record_set(orep)
        if pts:
            injected_launches += 1
            assert rep.corrected == len(pts) == 5
            assert sorted((r.i, r.j) for r in rep.records()) == sorted((p["i"], p["j"]) for p in pts)
        assert np.array_equal(got.view(np.uint64), clean.view(np.uint64))
    assert injected_launches == 2
    assert fb.ftblas_injection_launch_count() == 4


@pytest.mark.parametrize("engine", ENGINES, ids=ENGINE_IDS)
def test_output_checksum_and_multiple_error_sites(engine):
    use(engine)
    P = Problem(256, 256, 96, alpha=1.0, beta=1.0, seed=5)
    tr, tc, bk = tile_of(P)
    clean, _ = run_gpu(P)
    cases = [
        [dict(i=3, j=200, site=fb.SITE_OUTPUT, mode=fb.MODE_ADD_REL, rel_log2=-10, sign=-1)],
        [dict(i=130, j=7, site=fb.SITE_CHECKSUM, mode=fb.MODE_ADD_REL, rel_log2=0, sign=1)],
        [dict(i=10, j=10, site=fb.SITE_ACCUM, bit=50), dict(i=20, j=30, site=fb.SITE_ACCUM, bit=61)],
        [dict(i=10, j=10, site=fb.SITE_ACCUM, bit=50), dict(i=10, j=30, site=fb.SITE_OUTPUT, bit=58)],
        [dict(i=255, j=255, site=fb.SITE_OUTPUT, bit=62), dict(i=0, j=0, site=fb.SITE_ACCUM, bit=63)],
    ]
    for pts in cases:
        fb.ftblas_set_injection(fb.make_injection(fixed=pts))
        got, rep = run_gpu(P)
        opts = [dict(p, mode=p.get("mode", O.MODE_BITFLIP)) for p in pts]
        ref, orep = P.oracle_ft(tr, tc, bk, injections=opts)
        assert report_summary(rep) == report_summary(orep), pts
        assert record_set(rep) == record_set(orep), pts
        for (i, j, kind) in record_set(rep):
            if kind == fb.KIND_CORRECTED:
                assert got[i, j] == clean[i, j]
        if orep.uncorrectable == 0 and orep.input_nonfinite == 0:
            assert np.array_equal(got.view(np.uint64), clean.view(np.uint64))


@pytest.mark.parametrize("engine", ENGINES, ids=ENGINE_IDS)
def test_infinite_output_flagged_against_infinite_threshold(engine):
    """An output flipped to +inf makes its row/column sums and thresholds infinite; it is
    still located and recomputed (same data as the oracle's pin)."""
    use(engine)
    P = Problem(8, 8, 8, alpha=1.0, beta=0.0, seed=51, pad="even")
    P.A = np.eye(8)
    P.B = S.randint(51, 0, 64, 2, 5).reshape(8, 8).astype(np.float64)
    P.B[3, 5] = 1.0
    P.a, P.lda = S.store(P.A, O.COL_MAJOR, ld=8)
    P.b, P.ldb = S.store(P.B, O.COL_MAJOR, ld=8)
    clean, _ = run_gpu(P)
    pt = dict(i=3, j=5, site=fb.SITE_OUTPUT, mode=fb.MODE_BITFLIP, bit=62)
    fb.ftblas_set_injection(fb.make_injection(fixed=[pt]))
    got, rep = run_gpu(P)
    _, orep = P.oracle_ft(*tile_of(P), injections=[pt])
    assert report_summary(rep) == report_summary(orep) == (1, 1, 1, 0, 0, 0)
    assert record_set(rep) == record_set(orep) == [(3, 5, fb.KIND_CORRECTED)]
    assert np.array_equal(got, clean)


def test_huge_operands_use_the_binary64_threshold_path():
    """Operands near 1e20 overflow the binary32 magnitude sums of the mainloop; the tile
    then recomputes its threshold in binary64 and still matches the oracle."""
    P = Problem(200, 136, 64, alpha=1.0, beta=0.5, seed=61, pad="even")
    scale = 2.0 ** 70
    P.A = P.A * scale
    P.B = P.B * scale
    P.a, P.lda = S.store(P.A, O.COL_MAJOR, ld=P.lda)
    P.b, P.ldb = S.store(P.B, O.COL_MAJOR, ld=P.ldb)
    tr, tc, bk = tile_of(P)
    clean, rep = run_gpu(P)
    ref, orep = P.oracle_ft(tr, tc, bk)
    assert report_summary(rep) == report_summary(orep) and rep.detected == 0
    assert P.normalized_error(clean, ref) <= TOL
    pt = dict(i=150, j=100, site=fb.SITE_ACCUM, bit=44)
    fb.ftblas_set_injection(fb.make_injection(fixed=[pt]))
    got, rep = run_gpu(P)
    _, orep = P.oracle_ft(tr, tc, bk, injections=[pt])
    assert record_set(rep) == record_set(orep) == [(150, 100, fb.KIND_CORRECTED)]
    assert np.array_equal(got.view(np.uint64), clean.view(np.uint64))


def test_quick_returns_on_gpu():
    P = Problem(70, 50, 0, alpha=1.0, beta=0.5, seed=3)
    got, rep = run_gpu(P)
    assert np.array_equal(got, 0.5 * P.Cin) and rep.tiles_checked == 0
    P = Problem(70, 50, 40, alpha=0.0, beta=-2.0, seed=3)
    got, rep = run_gpu(P)
    assert np.array_equal(got, -2.0 * P.Cin) and rep.tiles_checked == 0
    P = Problem(70, 50, 40, alpha=1.0, beta=0.0, seed=3)
    nanc = np.full_like(P.c, np.nan)
    got, rep = run_gpu(P, c_init=nanc)
    assert np.all(np.isfinite(got)) and rep.detected == 0
    assert P.normalized_error(got, P.oracle_plain()) <= TOL


@pytest.mark.parametrize("engine", ENGINES, ids=ENGINE_IDS)
def test_untma_able_operands_use_the_fallback_loads(engine):
    """Odd leading dimensions and 8-byte-offset pointers cannot be described to TMA; the
    cooperative-load path must give the same answers."""
    use(engine)
    P = Problem(133, 71, 45, O.COL_MAJOR, O.NO_TRANS, O.NO_TRANS, alpha=1.5, beta=0.5, seed=9, pad=0)
    assert P.lda % 2 == 1  # 133: not a multiple of 16 bytes
    tr, tc, bk = tile_of(P)
    got, rep = run_gpu(P)
    assert fb.ftblas_last_launch_used_tma() == 0
    ref, orep = P.oracle_ft(tr, tc, bk)
    assert report_summary(rep) == report_summary(orep)
    assert P.normalized_error(got, ref) <= TOL
    # 8-byte-misaligned base pointer with even lda
    Q = Problem(128, 96, 64, alpha=1.0, beta=0.0, seed=10, pad=0)
    shifted = np.concatenate([[0.0], Q.a])
    dA = dev(shifted)
    dB, dC = dev(Q.b), dev(Q.c)
    rep = fb.new_report()
    fb.check(fb.ftblas_dgemm(Q.layout, Q.ta, Q.tb, Q.M, Q.N, Q.K, Q.alpha, dA.data_ptr() + 8, Q.lda,
                             dB.data_ptr(), Q.ldb, Q.beta, dC.data_ptr(), Q.ldc,
                             torch.cuda.current_stream().cuda_stream, rep.data_ptr()))
    assert fb.ftblas_last_launch_used_tma() == 0
    torch.cuda.synchronize()
    got = S.load(dC.cpu().numpy(), Q.layout, Q.M, Q.N, Q.ldc)
    assert Q.normalized_error(got, Q.oracle_plain()) <= TOL


@pytest.mark.parametrize("engine", ENGINES, ids=ENGINE_IDS)
def test_noabft_equals_protected_clean_output_bitwise(engine):
    use(engine)
    P = Problem(384, 256, 160, O.ROW_MAJOR, O.TRANS, O.NO_TRANS, alpha=1.5, beta=0.5, seed=12)
    ft_out, rep = run_gpu(P, protect=True)
    plain, _ = run_gpu(P, protect=False)
    assert rep.detected == 0
    assert np.array_equal(ft_out.view(np.uint64), plain.view(np.uint64))


def test_engines_agree_within_tolerance():
    P = Problem(256, 384, 512, alpha=1.5, beta=0.5, seed=13)
    fb.ftblas_set_fp64_engine(fb.ENGINE_DFMA)
    a, _ = run_gpu(P)
    fb.ftblas_set_fp64_engine(fb.ENGINE_DMMA)
    b, _ = run_gpu(P)
    assert P.normalized_error(a, b) <= TOL


def test_host_buffer_entry_point_matches_device_path():
    P = Problem(200, 150, 100, O.ROW_MAJOR, O.NO_TRANS, O.TRANS, alpha=1.5, beta=0.5, seed=14, pad=3)
    dev_out, _ = run_gpu(P)
    c = P.c.copy()
    rep = fb.FtReport()
    import ctypes
    fb.check(fb.ftblas_dgemm_host(P.layout, P.ta, P.tb, P.M, P.N, P.K, P.alpha, P.a.ctypes.data, P.lda,
                                  P.b.ctypes.data, P.ldb, P.beta, c.ctypes.data, P.ldc, None,
                                  ctypes.addressof(rep)))
    host_out = S.load(c, P.layout, P.M, P.N, P.ldc)
    assert np.array_equal(host_out.view(np.uint64), dev_out.view(np.uint64))
    tr, tc, _ = tile_of(P)
    assert rep.tiles_checked == -(-P.M // tr) * -(-P.N // tc) and rep.detected == 0
    # padding between leading dimensions was not touched
    assert np.isnan(c.reshape(P.M, P.ldc)[:, P.N:]).all()


@pytest.mark.parametrize("seed", range(6))
def test_clean_soak_no_false_alarms(seed):
    """Many seeds, shapes and magnitudes with no injection: zero detections."""
    rng = np.random.default_rng(seed)
    M, N, K = (int(x) for x in rng.integers(1, 700, size=3))
    layout, ta, tb = COMBOS[seed % len(COMBOS)]
    P = Problem(M, N, K, layout, ta, tb, alpha=float(rng.normal()), beta=float(rng.normal()), seed=seed,
                dist="normal")
    for engine in ENGINES:
        use(engine)
        got, rep = run_gpu(P)
        assert rep.detected == 0 and rep.input_nonfinite == 0
    assert P.normalized_error(got, P.oracle_plain()) <= TOL


@pytest.mark.parametrize("engine", [ENGINES[0], ENGINES[2]], ids=[ENGINE_IDS[0], ENGINE_IDS[2]])
def test_full_size_8192_sampled_rows_and_faulted_tile(engine):
    """The benchmark's launch configuration (8192^3, alpha 1.5, beta 0.5) checked on sampled
    rows and on the whole faulted tile, with one accumulator flip."""
    use(engine)
    n = 8192
    P = Problem(n, n, n, alpha=1.5, beta=0.5, seed=20210602)
    tr, tc, bk = tile_of(P)
    i, j = seeded_point(77, n, n)
    fb.ftblas_set_injection(fb.make_injection(fixed=[dict(i=i, j=j, site=fb.SITE_ACCUM, bit=45)]))
    got, rep = run_gpu(P)
    assert fb.ftblas_last_launch_used_tma() == 1
    assert report_summary(rep)[:5] == ((n // tr) * (n // tc), 1, 1, 0, 0)
    assert [(r.i, r.j) for r in rep.records()] == [(i, j)]
    rows = np.unique(np.concatenate([S.randint(5, 5, 6, 0, n - 1), [i]]))
    ref_rows = O.gemm_rows(P.layout, P.ta, P.tb, n, n, n, P.alpha, P.a, P.lda, P.b, P.ldb, P.beta, P.c, P.ldc, rows)
    den = np.abs(P.A).max() * np.abs(P.B).max() * n
    assert np.abs(got[rows, :] - ref_rows).max() / den <= TOL
    t = (i // tr) + (j // tc) * ((n + tr - 1) // tr)
    _, orep = P.oracle_ft(tr, tc, bk, injections=[dict(i=i, j=j, site=O.SITE_ACCUM, bit=45)], tiles=[t])
    assert record_set(orep) == record_set(rep)


# ---------------------------------------------------------------------------------------
# Online verification every kc products (ftblas_set_verification_interval)
# ---------------------------------------------------------------------------------------

@pytest.fixture
def _interval_off():
    yield
    fb.ftblas_set_verification_interval(0)


@pytest.mark.parametrize("engine", ENGINES, ids=ENGINE_IDS)
def test_online_checks_leave_clean_runs_bitwise_unchanged(engine, _interval_off):
    use(engine)
    P = Problem(300, 260, 700, O.COL_MAJOR, O.NO_TRANS, O.TRANS, alpha=1.5, beta=0.5, seed=31)
    base, rep0 = run_gpu(P)
    fb.ftblas_set_verification_interval(128)
    got, rep = run_gpu(P)
    assert np.array_equal(got, base)
    assert rep.detected == 0 and rep.tiles_checked == rep0.tiles_checked


@pytest.mark.parametrize("engine", ENGINES, ids=ENGINE_IDS)
@pytest.mark.parametrize("layout", [O.COL_MAJOR, O.ROW_MAJOR])
def test_online_checks_correct_two_faults_in_one_tile(engine, layout, _interval_off):
    """Two accumulator flips in one tile, in different intervals: with checks every 128
    products (4 k-tiles) both are corrected where they occur, as the oracle's interval mode
    does, and C equals the fault-free C of the same engine bit for bit; without online
    checks the pair is uncorrectable."""
    use(engine)
    P = Problem(256, 256, 512, layout, O.NO_TRANS, O.NO_TRANS, alpha=1.0, beta=0.0, seed=33)
    clean, _ = run_gpu(P)
    tr, tc, bk = tile_of(P)
    pts = [dict(i=5, j=7, site=fb.SITE_ACCUM, mode=fb.MODE_BITFLIP, bit=55, kt=2),
           dict(i=40, j=50, site=fb.SITE_ACCUM, mode=fb.MODE_BITFLIP, bit=58, kt=9),  # same tile as (5, 7)
           dict(i=200, j=140, site=fb.SITE_ACCUM, mode=fb.MODE_BITFLIP, bit=52, kt=5)]
    fb.ftblas_set_injection(fb.make_injection(fixed=pts))
    got_end, rep_end = run_gpu(P)
    _, orep_end = P.oracle_ft(tr, tc, bk, injections=pts)
    assert report_summary(rep_end) == report_summary(orep_end)
    assert rep_end.uncorrectable >= 1
    fb.ftblas_set_verification_interval(128)
    got, rep = run_gpu(P)
    _, orep = P.oracle_ft(tr, tc, bk, injections=pts, kc=128)
    assert report_summary(rep) == report_summary(orep)
    assert record_set(rep) == record_set(orep)
    assert (rep.corrected, rep.uncorrectable) == (3, 0)
    assert np.array_equal(got, clean)


@pytest.mark.parametrize("engine", ENGINES, ids=ENGINE_IDS)
def test_bounded_wait_gives_up_and_reports_timeout(engine):
    """A staging barrier that never completes (the test-only stall point: it expects 16 bytes
    more than TMA delivers) ends in a bounded wait, with no fault: the call returns, the
    report carries FT_STATUS_TIMEOUT, that tile is not stored while every other tile is,
    and the next call on the same context is clean and bit-identical."""
    use(engine)
    P = Problem(256, 320, 256, alpha=1.0, beta=0.0, seed=41)
    clean, rep0 = run_gpu(P)
    assert fb.ftblas_last_launch_used_tma() == 1 and rep0.status == 0
    tr, tc, _ = tile_of(P)
    i, j = 70, 200
    fb.ftblas_set_injection(fb.make_injection(fixed=[dict(i=i, j=j, site=fb.SITE_STALL, kt=3)]))
    got, rep = run_gpu(P)
    fb.ftblas_set_injection(None)
    assert rep.status & fb.STATUS_TIMEOUT
    rows = slice((i // tr) * tr, min((i // tr + 1) * tr, P.M))
    cols = slice((j // tc) * tc, min((j // tc + 1) * tc, P.N))
    stalled = np.zeros_like(got, dtype=bool)
    stalled[rows, cols] = True
    assert np.array_equal(got[~stalled], clean[~stalled])
    assert np.array_equal(got[stalled].view(np.uint64), P.Cin[stalled].view(np.uint64))  # not stored
    assert rep.tiles_checked == -(-P.M // tr) * -(-P.N // tc) - 1
    again, rep2 = run_gpu(P)
    assert rep2.status == 0 and rep2.detected == 0
    assert np.array_equal(again.view(np.uint64), clean.view(np.uint64))
