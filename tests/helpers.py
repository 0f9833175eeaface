"""Shared test helpers: seeded operands in BLAS storage, device copies, comparisons."""
import numpy as np

import oracle as O
import synth as S


def lead(extent, pad):
    """Leading dimension for a run of `extent`: + pad, or rounded up to even ("even": the
    16-byte rows TMA can address)."""
    if pad == "even":
        return max(2, extent + (extent & 1))
    return max(1, extent + pad)


def stored(layout, trans, logical, pad=0):
    """BLAS storage of X with op(X) == logical; returns (flat buffer, ld)."""
    X = logical if trans == O.NO_TRANS else logical.T
    return S.store(X, layout, ld=lead(X.shape[0] if layout == O.COL_MAJOR else X.shape[1], pad))


class Problem:
    """A seeded GEMM problem: logical operands plus their storage for one call layout."""

    def __init__(self, M, N, K, layout=O.COL_MAJOR, ta=O.NO_TRANS, tb=O.NO_TRANS, alpha=1.0, beta=0.0,
                 seed=20210601, pad=0, dist="uniform"):
        self.M, self.N, self.K = M, N, K
        self.layout, self.ta, self.tb = layout, ta, tb
        self.alpha, self.beta = alpha, beta
        gen = S.uniform_matrix if dist == "uniform" else S.normal_matrix
        self.A = gen(seed, 0, M, K)
        self.B = gen(seed, 1, K, N)
        self.Cin = gen(seed, 2, M, N)
        self.a, self.lda = stored(layout, ta, self.A, pad)
        self.b, self.ldb = stored(layout, tb, self.B, pad)
        self.c, self.ldc = S.store(self.Cin, layout, ld=lead(M if layout == O.COL_MAJOR else N, pad))

    def oracle_ft(self, tile_rows, tile_cols, bk, injections=(), tiles=None, kc=0):
        out, rep = O.ft_gemm(self.layout, self.ta, self.tb, self.M, self.N, self.K, self.alpha, self.a, self.lda,
                             self.b, self.ldb, self.beta, self.c, self.ldc, tile_rows, tile_cols, bk,
                             injections=injections, tiles=tiles, kc=kc)
        return S.load(out, self.layout, self.M, self.N, self.ldc), rep

    def oracle_plain(self):
        out = O.gemm(self.layout, self.ta, self.tb, self.M, self.N, self.K, self.alpha, self.a, self.lda, self.b,
                     self.ldb, self.beta, self.c, self.ldc)
        return S.load(out, self.layout, self.M, self.N, self.ldc)

    def normalized_error(self, got, ref):
        """max|C - C_ref| / (max|A| max|B| K), the FP64 accuracy criterion."""
        if got.size == 0:
            return 0.0
        den = max(np.abs(self.A).max(initial=0.0) * np.abs(self.B).max(initial=0.0) * max(self.K, 1), 1e-300)
        return float(np.abs(got - ref).max() / den)


def report_summary(rep):
    return (int(rep.tiles_checked), int(rep.detected), int(rep.corrected), int(rep.uncorrectable),
            int(rep.checksum_only), int(rep.input_nonfinite))


def record_set(rep):
    return sorted((int(r.i), int(r.j), int(r.kind)) for r in rep.records())
