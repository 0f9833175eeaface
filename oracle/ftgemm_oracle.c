/*
 * CPU oracle for the ABFT-protected GEMM of FT-BLAS (Zhai et al., ICS '21).
 *
 * TEST INFRASTRUCTURE ONLY. Only the tests, the smoke check and the benchmark's CPU
 * baseline and reference arm may load this library. The CUDA path never calls it and
 * shares no code with it: this file has its own element access, its own checksum
 * encode/verify/correct and its own SplitMix64 for the seeded injection draw.
 *
 * It is plain, slow and written to be checked by eye against the paper:
 *   - Section II.A: Huang-Abraham encoding A^c = [A; e^T A], B^r = [B, Be], so that
 *     A^c B^r = [[C, Ce], [e^T C, .]]; a disagreement of C with C^r = Ce or C^c = e^T C
 *     beyond the round-off threshold signals an error; one error per verification
 *     interval is corrected.
 *   - Section V.A: the reference row checksum is recomputed from C and compared; a
 *     mismatch is located with the column checksum.
 *   - Section V.B: C = beta*C is folded into the checksums; C^c and C^r are formed from
 *     the operands, the reference checksums from the computed C.
 *   - Section VI.C: the injected element and error magnitude follow from the checksum
 *     differences; correction subtracts the magnitude (kept as a cross-check here; the
 *     stored correction recomputes the element, see below).
 *
 * Readings where the paper is silent (each is listed in the design notes):
 *   - one verification interval = one tile_m x tile_n output tile over all of K;
 *   - threshold tau (below) is a rigorous rounding bound with gamma_n = n u / (1 - n u),
 *     u = 2^-53;
 *   - classification: 0 flagged rows and 0 flagged columns = clean; exactly one of each
 *     = located and corrected; flags on one side only = checksum-only; anything else =
 *     uncorrectable (C left as computed);
 *   - correction recomputes the located element from A and B (bit-exact fault-free
 *     value); the paper's subtract-the-magnitude value is recorded beside it;
 *   - accumulator injection flips bit b of the running sum of element (i, j) after
 *     bk * floor(nk / 2) products, nk = ceil(K / bk); output injection perturbs C(i, j)
 *     after alpha/beta and before verification.
 *
 * Parity unpinned, in one place, the binary32-accumulation model (ACC32) of the
 * tensor-core forms: the values of those forms against binary64 are checked only within
 * the stated accumulation bound; its unit roundoff u_acc is a property of the hardware,
 * not a figure of the paper. (The row threshold's term s gamma_K(u_acc), which this oracle's
 * own binary64 prediction never exercises, is pinned by a test that builds the extreme
 * binary32 accumulations the threshold must cover.)
 *
 * Arithmetic: binary64, products and sums as separate operations in ascending k. Build
 * with -ffp-contract=off so no multiply-add is contracted. OpenMP may split rows or
 * tiles across threads; it never changes the order of any individual sum.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define OR_ROW_MAJOR 101
#define OR_COL_MAJOR 102
#define OR_NO_TRANS 111
#define OR_TRANS 112

#define OR_SITE_ACCUM 1
#define OR_SITE_OUTPUT 2
#define OR_SITE_CHECKSUM 3   /* perturbs the predicted row checksum C^r(i): a fault in the encode path */
#define OR_MODE_BITFLIP 0
#define OR_MODE_ADD_REL 1

#define OR_KIND_CORRECTED 1
#define OR_KIND_CHECKSUM_ONLY 2
#define OR_KIND_UNCORRECTABLE 3
#define OR_KIND_INPUT_NONFINITE 4

#define OR_MAX_RECORDS 256

/* Precision of the protected product. FP64: binary64 throughout (the paper's setting).
 * ACC32: operands of any precision given as exact binary64 values, products accumulated
 * in binary32 (modelled by the binary64 sum and the threshold's u_acc), C rounded to
 * binary32; the row checksums are verified in every tile and the column checksums only in
 * tiles with a row mismatch (the lazy second side of Section V.A). */
#define OR_PREC_FP64 0
#define OR_PREC_ACC32 1
/* ACC32 for FP8 (E4M3) operands: the same arithmetic, with the row checksum's prediction
 * formed from B e split into eight e4m3 pieces instead of three bfloat16 ones, whose
 * magnitudes sum to at most 1.25 |B e| (1 + 2^-7 for the bfloat16 pieces). */
#define OR_PREC_ACC32_E4M3 2
#define IS_ACC32(p) ((p)->precision == OR_PREC_ACC32 || (p)->precision == OR_PREC_ACC32_E4M3)

/* ---------------------------------------------------------------------------------- */
/* Problem description and results                                                    */
/* ---------------------------------------------------------------------------------- */

typedef struct {
  int32_t layout, transa, transb, pad_;
  int64_t M, N, K;
  double alpha;
  const double* A; int64_t lda;
  const double* B; int64_t ldb;
  double beta;
  const double* Cin; int64_t ldc;   /* not read when beta == 0 */
  int64_t tile_m, tile_n;           /* verification tile, in rows x columns of C */
  int64_t bk;                       /* k-tile depth (sets the accumulator injection point) */
  int32_t precision;                /* OR_PREC_FP64, OR_PREC_ACC32 or OR_PREC_ACC32_E4M3 (binary32
                                       accumulation, binary32 C) */
  int32_t pad2_;
  double u_acc;                     /* OR_PREC_ACC32: unit roundoff of the accumulation */
  int64_t kc;                       /* OR_PREC_FP64: online verification every kc products (a
                                       multiple of bk; 0 or >= K: only the finished tile) */
} oracle_problem_t;

typedef struct {
  int64_t i, j;        /* element of C (row, column) */
  int32_t site;        /* OR_SITE_ACCUM, OR_SITE_OUTPUT or OR_SITE_CHECKSUM (j ignored there) */
  int32_t mode;        /* OR_MODE_BITFLIP or OR_MODE_ADD_REL */
  int32_t bit;         /* bit-flip: bit of the IEEE-754 binary64 pattern, 0 = lsb */
  int32_t rel_log2;    /* add-rel: e = sign * 2^rel_log2 * |c| */
  int32_t sign;        /* +1 or -1 */
  int32_t kt;          /* accumulator site: flip after kt * bk products (0: after bk * floor(nk / 2)) */
} oracle_injection_t;

typedef struct {
  int64_t tile_row, tile_col;  /* tile coordinates */
  int64_t i, j;                /* located element (or first flagged row / column, -1 if none) */
  double delta_row, delta_col; /* C^r_ref - C^r and C^c_ref - C^c at the flagged entries */
  double tau_row, tau_col;
  double value_before;         /* C(i, j) as computed (with the error) */
  double value_after;          /* C(i, j) after correction (recomputed) */
  double value_subtracted;     /* the paper's correction: value_before - delta_row */
  int32_t kind;                /* OR_KIND_* */
  int32_t rows_flagged, cols_flagged, pad_;
} oracle_record_t;

typedef struct {
  uint64_t tiles_checked, detected, corrected, uncorrectable, checksum_only, input_nonfinite;
  uint32_t n_records, pad_;
  oracle_record_t rec[OR_MAX_RECORDS];
} oracle_report_t;

/* ---------------------------------------------------------------------------------- */
/* Element access following the BLAS op() convention                                  */
/* ---------------------------------------------------------------------------------- */

/* Element (r, c) of op(X): X(r, c) without transpose, X(c, r) with it; X(p, q) lives at
 * p + q*ld in column-major storage and at p*ld + q in row-major storage. */
static double op_elem(const double* X, int64_t ld, int layout, int trans, int64_t r, int64_t c) {
  int64_t p = (trans == OR_TRANS) ? c : r;
  int64_t q = (trans == OR_TRANS) ? r : c;
  return (layout == OR_COL_MAJOR) ? X[p + q * ld] : X[p * ld + q];
}

static int64_t c_index(int layout, int64_t ldc, int64_t i, int64_t j) {
  return (layout == OR_COL_MAJOR) ? i + j * ldc : i * ldc + j;
}

static double a_elem(const oracle_problem_t* p, int64_t i, int64_t k) {
  return op_elem(p->A, p->lda, p->layout, p->transa, i, k);
}
static double b_elem(const oracle_problem_t* p, int64_t k, int64_t j) {
  return op_elem(p->B, p->ldb, p->layout, p->transb, k, j);
}
static double cin_elem(const oracle_problem_t* p, int64_t i, int64_t j) {
  return p->Cin[c_index(p->layout, p->ldc, i, j)];
}

static double flip_bit(double x, int bit) {
  uint64_t u;
  memcpy(&u, &x, 8);
  u ^= (uint64_t)1 << bit;
  memcpy(&x, &u, 8);
  return x;
}

static double round32(double x) { return (double)(float)x; }

static double flip_bit32(double x, int bit) {
  float f = (float)x;
  uint32_t u;
  memcpy(&u, &f, 4);
  u ^= (uint32_t)1 << bit;
  memcpy(&f, &u, 4);
  return (double)f;
}

/* ---------------------------------------------------------------------------------- */
/* The GEMM definition: C = alpha * op(A) * op(B) + beta * C                           */
/* ---------------------------------------------------------------------------------- */

/* Inner product of row i of op(A) with column j of op(B), k ascending, separate multiply
 * and add. When inj_bit >= 0 the running sum's bit inj_bit is flipped after the first
 * kstar products (kstar >= K flips the finished sum). */
static double dot_row_col(const oracle_problem_t* p, int64_t i, int64_t j, int64_t kstar, int inj_bit) {
  double acc = 0.0;
  for (int64_t k = 0; k < p->K; ++k) {
    if (inj_bit >= 0 && k == kstar) acc = flip_bit(acc, inj_bit);
    double prod = a_elem(p, i, k) * b_elem(p, k, j);
    acc = acc + prod;
  }
  if (inj_bit >= 0 && kstar >= p->K) acc = flip_bit(acc, inj_bit);
  return acc;
}

/* alpha * acc, then + beta * cin (cin not read when beta == 0). */
static double scale_out(const oracle_problem_t* p, double acc, int64_t i, int64_t j) {
  double t = p->alpha * acc;
  if (p->beta != 0.0) {
    double s = p->beta * cin_elem(p, i, j);
    t = t + s;
  }
  return t;
}

/* Triangular solve T X = W in place, T n x n column-major (leading dimension ldt), only
 * its lower (lower != 0) or upper triangle read, W n x nrhs column-major (ldw): the
 * textbook substitution for each column, x_r = (w_r - sum_c T(r,c) x_c) / T(r,r) with the
 * sum over the already solved rows in ascending c (forward for lower, backward for upper),
 * separate multiply and add. */
void oracle_trsm_left(int64_t n, int64_t nrhs, const double* T, int64_t ldt, int lower, double* W, int64_t ldw) {
#pragma omp parallel for schedule(static)
  for (int64_t j = 0; j < nrhs; ++j) {
    double* w = W + j * ldw;
    for (int64_t q = 0; q < n; ++q) {
      const int64_t r = lower ? q : n - 1 - q;
      double s = 0.0;
      if (lower) {
        for (int64_t c = 0; c < r; ++c) s = s + T[r + c * ldt] * w[c];
      } else {
        for (int64_t c = r + 1; c < n; ++c) s = s + T[r + c * ldt] * w[c];
      }
      w[r] = (w[r] - s) / T[r + r * ldt];
    }
  }
}

/* Plain product C = alpha*op(A)*op(B) + beta*C_in into Cout (same layout and ldc as Cin).
 * Returns 0, or -1 for bad arguments. */
int oracle_gemm(const oracle_problem_t* p, double* Cout) {
  if (p->M < 0 || p->N < 0 || p->K < 0) return -1;
  int64_t M = p->M, N = p->N;
#pragma omp parallel for schedule(dynamic, 1)
  for (int64_t i = 0; i < M; ++i) {
    for (int64_t j = 0; j < N; ++j) {
      double acc = (p->alpha == 0.0) ? 0.0 : dot_row_col(p, i, j, 0, -1);
      double v;
      if (p->alpha == 0.0) {
        v = (p->beta == 0.0) ? 0.0 : p->beta * cin_elem(p, i, j);
      } else {
        v = scale_out(p, acc, i, j);
      }
      if (IS_ACC32(p)) v = round32(v);
      Cout[c_index(p->layout, p->ldc, i, j)] = v;
    }
  }
  return 0;
}

/* Rows rows[0..nrows-1] of the plain product, written row by row into out[r*N + j]. */
int oracle_gemm_rows(const oracle_problem_t* p, int64_t nrows, const int64_t* rows, double* out) {
  int64_t N = p->N;
#pragma omp parallel for schedule(dynamic, 1)
  for (int64_t r = 0; r < nrows; ++r) {
    int64_t i = rows[r];
    for (int64_t j = 0; j < N; ++j) {
      double v;
      if (p->alpha == 0.0 || p->K == 0) {
        v = (p->beta == 0.0) ? 0.0 : p->beta * cin_elem(p, i, j);
      } else {
        v = scale_out(p, dot_row_col(p, i, j, 0, -1), i, j);
      }
      out[r * N + j] = v;
    }
  }
  return 0;
}

int oracle_num_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

/* ---------------------------------------------------------------------------------- */
/* Seeded injection draw (SplitMix64 of Steele, Lea and Flood, OOPSLA 2014)            */
/* ---------------------------------------------------------------------------------- */

static uint64_t sm64_next(uint64_t* state) {
  uint64_t z = (*state += 0x9E3779B97F4A7C15ULL);
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}

/* The injections of launch number `launch` (0-based count of protected launches since
 * the configuration was set). A launch injects when every_n > 0 and
 * launch % every_n == seed % every_n. Tiles (numbered t = tile_row + tile_col * n_tile_rows)
 * are drawn without replacement; per injection the stream yields, in this order: tile,
 * row offset, column offset, bit, log2 magnitude, sign. The stream state starts at
 * seed ^ (launch * 0xD1B54A32D192ED03). Returns the number written to out (<= cap). */
int64_t oracle_draw_injections(uint64_t seed, uint64_t launch, int32_t every_n, int32_t per_launch,
                               int32_t site, int32_t mode, int32_t bit_lo, int32_t bit_hi,
                               int32_t log2_lo, int32_t log2_hi,
                               int64_t M, int64_t N, int64_t tile_m, int64_t tile_n,
                               int64_t cap, oracle_injection_t* out) {
  if (every_n <= 0 || per_launch <= 0 || M <= 0 || N <= 0) return 0;
  if (launch % (uint64_t)every_n != seed % (uint64_t)every_n) return 0;
  int64_t tr = (M + tile_m - 1) / tile_m, tc = (N + tile_n - 1) / tile_n;
  int64_t ntiles = tr * tc;
  int64_t want = per_launch;
  if (want > ntiles) want = ntiles;
  if (want > cap) want = cap;
  uint64_t st = seed ^ (launch * 0xD1B54A32D192ED03ULL);
  int64_t n = 0;
  while (n < want) {
    uint64_t t = sm64_next(&st) % (uint64_t)ntiles;
    uint64_t ri = sm64_next(&st);
    uint64_t rj = sm64_next(&st);
    uint64_t rb = sm64_next(&st);
    uint64_t rp = sm64_next(&st);
    uint64_t rs = sm64_next(&st);
    int dup = 0;
    int64_t trow = (int64_t)t % tr, tcol = (int64_t)t / tr;
    for (int64_t q = 0; q < n; ++q)
      if (out[q].i / tile_m == trow && out[q].j / tile_n == tcol) dup = 1;
    if (dup) continue;
    int64_t rows = (trow == tr - 1) ? M - trow * tile_m : tile_m;
    int64_t cols = (tcol == tc - 1) ? N - tcol * tile_n : tile_n;
    out[n].i = trow * tile_m + (int64_t)(ri % (uint64_t)rows);
    out[n].j = tcol * tile_n + (int64_t)(rj % (uint64_t)cols);
    out[n].site = site;
    out[n].mode = mode;
    out[n].bit = bit_lo + (int32_t)(rb % (uint64_t)(bit_hi - bit_lo + 1));
    out[n].rel_log2 = log2_lo + (int32_t)(rp % (uint64_t)(log2_hi - log2_lo + 1));
    out[n].sign = (rs & 1) ? -1 : 1;
    out[n].kt = 0;
    ++n;
  }
  return n;
}

/* ---------------------------------------------------------------------------------- */
/* ABFT-protected GEMM                                                                */
/* ---------------------------------------------------------------------------------- */

static double gamma_n(double n) {
  const double u = 1.1102230246251565e-16; /* 2^-53 */
  return n * u / (1.0 - n * u);
}

static int isfinite_d(double x) { return isfinite(x) != 0; }

#define OR_TILE_RECORDS 32
typedef struct {
  uint64_t detected, corrected, uncorrectable, checksum_only, input_nonfinite;
  int32_t n_rec;
  oracle_record_t rec[OR_TILE_RECORDS];
} tile_result_t;

static void add_record(tile_result_t* res, const oracle_record_t* r) {
  if (res->n_rec < OR_TILE_RECORDS) res->rec[res->n_rec++] = *r;
}

/* Products over the tile with online verification every kc products (Section V.A: after
 * every rank-kc update of the outer-product formulation the checksum relation holds for
 * the partial product, so it can be checked, and one error corrected, at each step).
 * acc[ii + jj*nI] receives the tile's raw accumulators (alpha, beta not applied). At the
 * end of each step but the last, the row and column sums of the accumulators are
 * compared with the predicted partial checksums sum_{k < kh} A(i,k) (Be)(k) and
 * sum_{k < kh} (e^T A)(k) B(k,j) against
 *   tau = 2 [gamma_{kh + n + 3} P + gamma_n sum |acc|],  P = sum_{k < kh} |A(i,k)| (|B| e)(k)
 * (and symmetrically for columns), the threshold reading of the finished tile with K
 * replaced by kh and no alpha or beta. Exactly one flagged row and one flagged column
 * locate the error, whose accumulator is recomputed over k < kh (the fault-free partial
 * product) and recorded as corrected; other patterns are left for the check of the
 * finished tile. Accumulator flips land after kt * bk products as in dot_row_col. */
static void midk_products(const oracle_problem_t* p, int64_t tr, int64_t tc, int64_t i0, int64_t j0, int64_t nI,
                          int64_t nJ, const double* Ac, const double* Br, const double* Ac_abs, const double* Br_abs,
                          int64_t n_inj, const oracle_injection_t* inj, double* acc, tile_result_t* res) {
  const int64_t K = p->K, nk = (K + p->bk - 1) / p->bk;
  double* pr = (double*)calloc((size_t)nI, sizeof(double));
  double* Pr = (double*)calloc((size_t)nI, sizeof(double));
  double* pc = (double*)calloc((size_t)nJ, sizeof(double));
  double* Pc = (double*)calloc((size_t)nJ, sizeof(double));
  int64_t* kflip = (int64_t*)malloc((size_t)(nI * nJ) * sizeof(int64_t));
  int* bflip = (int*)malloc((size_t)(nI * nJ) * sizeof(int));
  for (int64_t e = 0; e < nI * nJ; ++e) { acc[e] = 0.0; kflip[e] = -1; bflip[e] = -1; }
  for (int64_t q = 0; q < n_inj; ++q) {
    if (inj[q].site != OR_SITE_ACCUM || inj[q].mode != OR_MODE_BITFLIP) continue;
    int64_t ii = inj[q].i - i0, jj = inj[q].j - j0;
    if (ii < 0 || ii >= nI || jj < 0 || jj >= nJ || bflip[ii + jj * nI] >= 0) continue;
    bflip[ii + jj * nI] = inj[q].bit;
    kflip[ii + jj * nI] = p->bk * (inj[q].kt > 0 ? inj[q].kt : nk / 2);
  }
  for (int64_t kl = 0; kl < K; kl += p->kc) {
    const int64_t kh = (kl + p->kc < K) ? kl + p->kc : K;
    for (int64_t jj = 0; jj < nJ; ++jj)
      for (int64_t ii = 0; ii < nI; ++ii) {
        double a_ = acc[ii + jj * nI];
        for (int64_t k = kl; k < kh; ++k) {
          if (bflip[ii + jj * nI] >= 0 && k == kflip[ii + jj * nI]) a_ = flip_bit(a_, bflip[ii + jj * nI]);
          double prod = a_elem(p, i0 + ii, k) * b_elem(p, k, j0 + jj);
          a_ = a_ + prod;
        }
        acc[ii + jj * nI] = a_;
      }
    for (int64_t ii = 0; ii < nI; ++ii)
      for (int64_t k = kl; k < kh; ++k) {
        double a = a_elem(p, i0 + ii, k);
        pr[ii] = pr[ii] + a * Br[k];
        Pr[ii] = Pr[ii] + fabs(a) * Br_abs[k];
      }
    for (int64_t jj = 0; jj < nJ; ++jj)
      for (int64_t k = kl; k < kh; ++k) {
        double b = b_elem(p, k, j0 + jj);
        pc[jj] = pc[jj] + Ac[k] * b;
        Pc[jj] = Pc[jj] + Ac_abs[k] * fabs(b);
      }
    if (kh >= K) break;
    /* online check of the partial product */
    const double g_row = gamma_n((double)(kh + nJ + 3)), g_rsum = gamma_n((double)nJ);
    const double g_col = gamma_n((double)(kh + nI + 3)), g_csum = gamma_n((double)nI);
    int64_t nr = 0, nc = 0, fr = -1, fc = -1;
    double fr_d = 0.0, fr_t = 0.0, fc_d = 0.0, fc_t = 0.0;
    for (int64_t ii = 0; ii < nI; ++ii) {
      double ref = 0.0, R = 0.0;
      for (int64_t jj = 0; jj < nJ; ++jj) { ref = ref + acc[ii + jj * nI]; R = R + fabs(acc[ii + jj * nI]); }
      double d = ref - pr[ii], tau = 2.0 * (g_row * Pr[ii] + g_rsum * R);
      if (!(fabs(d) <= tau) || isinf(d)) { if (fr < 0) { fr = ii; fr_d = d; fr_t = tau; } ++nr; }
    }
    for (int64_t jj = 0; jj < nJ; ++jj) {
      double ref = 0.0, R = 0.0;
      for (int64_t ii = 0; ii < nI; ++ii) { ref = ref + acc[ii + jj * nI]; R = R + fabs(acc[ii + jj * nI]); }
      double d = ref - pc[jj], tau = 2.0 * (g_col * Pc[jj] + g_csum * R);
      if (!(fabs(d) <= tau) || isinf(d)) { if (fc < 0) { fc = jj; fc_d = d; fc_t = tau; } ++nc; }
    }
    if (nr == 1 && nc == 1) {
      double fixed = 0.0;
      for (int64_t k = 0; k < kh; ++k) {
        double prod = a_elem(p, i0 + fr, k) * b_elem(p, k, j0 + fc);
        fixed = fixed + prod;
      }
      oracle_record_t r;
      memset(&r, 0, sizeof(r));
      r.tile_row = tr; r.tile_col = tc; r.i = i0 + fr; r.j = j0 + fc;
      r.delta_row = fr_d; r.delta_col = fc_d; r.tau_row = fr_t; r.tau_col = fc_t;
      r.value_before = acc[fr + fc * nI];
      r.value_after = fixed;
      r.value_subtracted = acc[fr + fc * nI] - fr_d;
      r.kind = OR_KIND_CORRECTED;
      r.rows_flagged = 1; r.cols_flagged = 1;
      add_record(res, &r);
      res->detected += 1;
      res->corrected += 1;
      acc[fr + fc * nI] = fixed;
    }
  }
  free(pr); free(Pr); free(pc); free(Pc); free(kflip); free(bflip);
}

/* One verification interval: the tile_m x tile_n tile (tr, tc) over all of K. */
static void ft_tile(const oracle_problem_t* p, int64_t tr, int64_t tc,
                    int64_t n_inj, const oracle_injection_t* inj,
                    double* Cout, tile_result_t* res) {
  const int64_t K = p->K;
  const int64_t i0 = tr * p->tile_m, j0 = tc * p->tile_n;
  const int64_t nI = (i0 + p->tile_m <= p->M) ? p->tile_m : p->M - i0;
  const int64_t nJ = (j0 + p->tile_n <= p->N) ? p->tile_n : p->N - j0;
  const int64_t nk = (K + p->bk - 1) / p->bk;
  const int64_t kstar = p->bk * (nk / 2);
  memset(res, 0, sizeof(*res));

  /* Encode (Section II.A, per tile): the checksum row of A^c = e^T A over the tile's
   * rows and the checksum column of B^r = B e over the tile's columns, plus the
   * absolute-value versions used by the threshold. */
  double* Ac = (double*)calloc((size_t)(K > 0 ? K : 1), sizeof(double));
  double* Br = (double*)calloc((size_t)(K > 0 ? K : 1), sizeof(double));
  double* Ac_abs = (double*)calloc((size_t)(K > 0 ? K : 1), sizeof(double));
  double* Br_abs = (double*)calloc((size_t)(K > 0 ? K : 1), sizeof(double));
  for (int64_t k = 0; k < K; ++k) {
    double s = 0.0, sa = 0.0;
    for (int64_t i = i0; i < i0 + nI; ++i) { double a = a_elem(p, i, k); s = s + a; sa = sa + fabs(a); }
    Ac[k] = s; Ac_abs[k] = sa;
    s = 0.0; sa = 0.0;
    for (int64_t j = j0; j < j0 + nJ; ++j) { double b = b_elem(p, k, j); s = s + b; sa = sa + fabs(b); }
    Br[k] = s; Br_abs[k] = sa;
  }
  int nonfinite_input = 0;
  for (int64_t k = 0; k < K; ++k)
    if (!isfinite_d(Ac[k]) || !isfinite_d(Br[k])) nonfinite_input = 1;

  /* Product over the tile, with the injections that fall inside it; with online
   * verification (kc) the accumulators come from the checked rank-kc steps. */
  double* T = (double*)malloc((size_t)(nI * nJ) * sizeof(double)); /* T[ii + jj*nI] */
  const int midk = p->kc > 0 && p->kc < K;
  if (midk) midk_products(p, tr, tc, i0, j0, nI, nJ, Ac, Br, Ac_abs, Br_abs, n_inj, inj, T, res);
  for (int64_t jj = 0; jj < nJ; ++jj) {
    for (int64_t ii = 0; ii < nI; ++ii) {
      int64_t i = i0 + ii, j = j0 + jj;
      double acc;
      if (midk) {
        acc = T[ii + jj * nI];
      } else {
        int acc_bit = -1;
        int64_t kq = kstar;
        for (int64_t q = 0; q < n_inj; ++q)
          if (inj[q].i == i && inj[q].j == j && inj[q].site == OR_SITE_ACCUM && inj[q].mode == OR_MODE_BITFLIP) {
            acc_bit = inj[q].bit;
            if (inj[q].kt > 0) kq = p->bk * inj[q].kt;
          }
        acc = dot_row_col(p, i, j, kq, acc_bit);
      }
      double v = scale_out(p, acc, i, j);
      for (int64_t q = 0; q < n_inj; ++q) {
        if (inj[q].i != i || inj[q].j != j || inj[q].site != OR_SITE_OUTPUT) continue;
        if (inj[q].mode == OR_MODE_BITFLIP) {
          v = flip_bit(v, inj[q].bit);
        } else {
          double e = ldexp(fabs(v), inj[q].rel_log2);
          v = (inj[q].sign < 0) ? v - e : v + e;
        }
      }
      T[ii + jj * nI] = v;
    }
  }

  /* Checksums of C predicted from the operands (Section II.A, with beta*C folded in as in
   * Section V.B): C^r(i) = alpha * sum_k A(i,k) * (Be)(k) + beta * sum_j Cin(i,j) and
   * C^c(j) = alpha * sum_k (e^T A)(k) * B(k,j) + beta * sum_i Cin(i,j); reference
   * checksums from the computed tile (Section V.A): C^r_ref(i) = sum_j C(i,j),
   * C^c_ref(j) = sum_i C(i,j). */
  double* dr = (double*)malloc((size_t)nI * sizeof(double));
  double* tr_tau = (double*)malloc((size_t)nI * sizeof(double));
  double* dc = (double*)malloc((size_t)nJ * sizeof(double));
  double* tc_tau = (double*)malloc((size_t)nJ * sizeof(double));
  const double g_row = gamma_n((double)(K + nJ + 3)), g_rsum = gamma_n((double)nJ);
  const double g_col = gamma_n((double)(K + nI + 3)), g_csum = gamma_n((double)nI);
  for (int64_t ii = 0; ii < nI; ++ii) {
    int64_t i = i0 + ii;
    double dotp = 0.0, P = 0.0;
    for (int64_t k = 0; k < K; ++k) {
      double a = a_elem(p, i, k);
      dotp = dotp + a * Br[k];
      P = P + fabs(a) * Br_abs[k];
    }
    double cin_sum = 0.0, Q = 0.0;
    if (p->beta != 0.0)
      for (int64_t jj = 0; jj < nJ; ++jj) { double c = cin_elem(p, i, j0 + jj); cin_sum = cin_sum + c; Q = Q + fabs(c); }
    double Cr = p->alpha * dotp;
    if (p->beta != 0.0) Cr = Cr + p->beta * cin_sum;
    for (int64_t q = 0; q < n_inj; ++q) {
      if (inj[q].site != OR_SITE_CHECKSUM || inj[q].i != i || inj[q].j / p->tile_n != tc) continue;
      double e = ldexp(fabs(Cr), inj[q].rel_log2);
      Cr = (inj[q].sign < 0) ? Cr - e : Cr + e;
    }
    double Cr_ref = 0.0, R = 0.0;
    for (int64_t jj = 0; jj < nJ; ++jj) { Cr_ref = Cr_ref + T[ii + jj * nI]; R = R + fabs(T[ii + jj * nI]); }
    dr[ii] = Cr_ref - Cr;
    tr_tau[ii] = 2.0 * (g_row * (fabs(p->alpha) * P + fabs(p->beta) * Q) + g_rsum * R);
    if (p->beta != 0.0 && !isfinite_d(cin_sum)) nonfinite_input = 1;
  }
  for (int64_t jj = 0; jj < nJ; ++jj) {
    int64_t j = j0 + jj;
    double dotp = 0.0, P = 0.0;
    for (int64_t k = 0; k < K; ++k) {
      double b = b_elem(p, k, j);
      dotp = dotp + Ac[k] * b;
      P = P + Ac_abs[k] * fabs(b);
    }
    double cin_sum = 0.0, Q = 0.0;
    if (p->beta != 0.0)
      for (int64_t ii = 0; ii < nI; ++ii) { double c = cin_elem(p, i0 + ii, j); cin_sum = cin_sum + c; Q = Q + fabs(c); }
    double Cc = p->alpha * dotp;
    if (p->beta != 0.0) Cc = Cc + p->beta * cin_sum;
    double Cc_ref = 0.0, R = 0.0;
    for (int64_t ii = 0; ii < nI; ++ii) { Cc_ref = Cc_ref + T[ii + jj * nI]; R = R + fabs(T[ii + jj * nI]); }
    dc[jj] = Cc_ref - Cc;
    tc_tau[jj] = 2.0 * (g_col * (fabs(p->alpha) * P + fabs(p->beta) * Q) + g_csum * R);
    if (p->beta != 0.0 && !isfinite_d(cin_sum)) nonfinite_input = 1;
  }

  /* Verify: an entry is flagged when |delta| > tau, or when delta is not finite (NaN, or
   * infinite even when an infinite C entry has made tau infinite too). */
  int64_t nr = 0, nc = 0, fr = -1, fc = -1;
  for (int64_t ii = 0; ii < nI; ++ii)
    if (!(fabs(dr[ii]) <= tr_tau[ii]) || isinf(dr[ii])) { if (fr < 0) fr = ii; ++nr; }
  for (int64_t jj = 0; jj < nJ; ++jj)
    if (!(fabs(dc[jj]) <= tc_tau[jj]) || isinf(dc[jj])) { if (fc < 0) fc = jj; ++nc; }

  oracle_record_t r;
  memset(&r, 0, sizeof(r));
  r.tile_row = tr; r.tile_col = tc;
  r.i = (fr >= 0) ? i0 + fr : -1;
  r.j = (fc >= 0) ? j0 + fc : -1;
  r.delta_row = (fr >= 0) ? dr[fr] : 0.0;
  r.delta_col = (fc >= 0) ? dc[fc] : 0.0;
  r.tau_row = (fr >= 0) ? tr_tau[fr] : 0.0;
  r.tau_col = (fc >= 0) ? tc_tau[fc] : 0.0;
  r.rows_flagged = (int32_t)nr; r.cols_flagged = (int32_t)nc;

  if (nonfinite_input) {
    /* Non-finite encoded checksums: the relation cannot be checked; C is kept. */
    res->input_nonfinite += 1;
    r.kind = OR_KIND_INPUT_NONFINITE;
    add_record(res, &r);
  } else if (nr == 0 && nc == 0) {
    /* clean */
  } else if (nr == 1 && nc == 1) {
    /* Locate at the crossing of the mismatching row and column and correct. */
    res->detected += 1; res->corrected += 1;
    r.kind = OR_KIND_CORRECTED;
    r.value_before = T[fr + fc * nI];
    r.value_subtracted = r.value_before - r.delta_row;
    double fixed = scale_out(p, dot_row_col(p, r.i, r.j, 0, -1), r.i, r.j);
    T[fr + fc * nI] = fixed;
    r.value_after = fixed;
    add_record(res, &r);
  } else if (nr == 0 || nc == 0) {
    res->detected += 1; res->checksum_only += 1;
    r.kind = OR_KIND_CHECKSUM_ONLY;
    add_record(res, &r);
  } else {
    res->detected += 1; res->uncorrectable += 1;
    r.kind = OR_KIND_UNCORRECTABLE;
    add_record(res, &r);
  }

  for (int64_t jj = 0; jj < nJ; ++jj)
    for (int64_t ii = 0; ii < nI; ++ii)
      Cout[c_index(p->layout, p->ldc, i0 + ii, j0 + jj)] = T[ii + jj * nI];

  free(Ac); free(Br); free(Ac_abs); free(Br_abs); free(T);
  free(dr); free(tr_tau); free(dc); free(tc_tau);
}

/* One verification interval of the ACC32 precision (operands exact in binary64, products
 * accumulated in binary32, C stored in binary32). Same encode and checksums as ft_tile;
 * the differences are the ones a binary32 accumulation brings:
 *   - C(i,j) = fl32(alpha * acc + beta * C_in), acc the binary64 inner product;
 *   - an accumulator injection flips bit b of the binary32 accumulator after all K products;
 *   - tau bounds, for any run whose binary32 accumulation steps each err by at most u_acc
 *     (either direction), the mismatch a clean tile can show. With P = (sum_k |A(i,k)|)
 *     (max_k sum_j |B(k,j)|) over the tile (an upper bound of sum_k |A(i,k)| sum_j |B(k,j)|):
 *       row:    |alpha| P (gamma_K(u_acc) (1 + s) + 2^-20 + gamma_{tile_n}(2^-24))
 *               + 2^-23 sum_j |C| + 2^-21 |beta| sum_j |C_in|
 *       term by term: gamma_K(u_acc) P, the K-term accumulations of the row's outputs;
 *       gamma_K(u_acc) s P, the accumulations of A times the pieces of B e that form the
 *       prediction, the pieces' magnitudes summing to at most s |B e| (s = 1 + 2^-7 for
 *       three bfloat16 pieces, 1.25 for eight e4m3 pieces); gamma_{tile_n}(2^-24) P, the
 *       binary32 sum B e over the tile's columns in any order; 2^-23 sum_j |C|, the
 *       compensated binary32 sum of the row (2 x 2^-24 of its value); 2^-21 |beta| sum_j
 *       |C_in|, the beta side of four roundings of 2^-24: beta C_in and the output's
 *       multiply-add, both binary32, and the compensated sum of C_in (2 x 2^-24), with a
 *       factor two to spare; 2^-20 P collects the alpha side of the output rounding
 *       (2^-24 (1 + gamma_K) P), the cross term gamma_K s gamma_{tile_n} (below 2^-24 for
 *       K <= 2^15) and the binary64 operations of the comparison (a few 2^-53), with a
 *       factor four to spare;
 *       column: |alpha| P_c (gamma_K(u_acc) + gamma_K(2^-24) + 2^-22 + gamma_{tile_m}(2^-24))
 *               + 2^-23 (sum_i |C| + 34 |beta| sum_i |C_in|),
 *               P_c = sum_k (sum_{i in tile} |A(i,k)|) |B(k,j)| (exact: it is formed only in the
 *               rare tiles with a row mismatch)
 *       term by term: gamma_K(u_acc) P_c, the column's outputs; gamma_K(2^-24) P_c, the
 *       prediction (e^T A) B as a binary32 dot product (round to nearest);
 *       gamma_{tile_m}(2^-24) P_c, e^T A as a binary32 sum over the tile's rows; 2^-23 sum_i
 *       |C|, the compensated column sum; 34 x 2^-23 |beta| sum_i |C_in|, the beta side:
 *       gamma_31(2^-24) for the binary32 sums of C_in over each group of 32 rows in any
 *       order (31 x 2^-24), beta C_in and the output's multiply-add (2 x 2^-24), 33 x 2^-24
 *       in all, with a factor two to spare; 2^-22 P_c collects the alpha side of the output
 *       rounding, the cross terms (gamma_K(2^-24) gamma_{tile_m}(2^-24), below 2^-26) and
 *       the binary64 operations;
 *   - column checksums are formed only when a row mismatches (Section V.A, lazy side);
 *     when they flag no column and beta == 0, the mismatching row is recomputed and each
 *     element compared with its own bound (locates errors in rows of small scale):
 *       |alpha| S (gamma_K(u_acc) + gamma_K(2^-24) + 2^-30) + 2^-23 |C(i,j)|,
 *       S = sum_k |A(i,k)| |B(k,j)|: the output's accumulation, the recomputation as a
 *       binary32 dot product (round to nearest), the output's rounding (2^-24, a factor two
 *       to spare) and 2^-30 S for the cross term and the binary64 operations;
 *   - a located error is corrected by subtracting the row mismatch (Section VI.C),
 *     evaluated as C(i,j) = C^r(i) - sum_{j' != j} C(i,j') (equal in exact arithmetic,
 *     stable for huge or non-finite errors); the result is rounded to binary32. */
static void ft_tile_acc32(const oracle_problem_t* p, int64_t tr, int64_t tc,
                          int64_t n_inj, const oracle_injection_t* inj,
                          double* Cout, tile_result_t* res) {
  const int64_t K = p->K;
  const int64_t i0 = tr * p->tile_m, j0 = tc * p->tile_n;
  const int64_t nI = (i0 + p->tile_m <= p->M) ? p->tile_m : p->M - i0;
  const int64_t nJ = (j0 + p->tile_n <= p->N) ? p->tile_n : p->N - j0;
  memset(res, 0, sizeof(*res));
  double* Ac = (double*)calloc((size_t)(K > 0 ? K : 1), sizeof(double));
  double* Ac_abs = (double*)calloc((size_t)(K > 0 ? K : 1), sizeof(double));
  double* Br = (double*)calloc((size_t)(K > 0 ? K : 1), sizeof(double));
  double maxAbsBe = 0.0;
  for (int64_t k = 0; k < K; ++k) {
    double s = 0.0, sa = 0.0;
    for (int64_t i = i0; i < i0 + nI; ++i) { double a = a_elem(p, i, k); s = s + a; sa = sa + fabs(a); }
    Ac[k] = s;
    Ac_abs[k] = sa;
    s = 0.0; sa = 0.0;
    for (int64_t j = j0; j < j0 + nJ; ++j) { double b = b_elem(p, k, j); s = s + b; sa = sa + fabs(b); }
    Br[k] = s;
    if (sa > maxAbsBe) maxAbsBe = sa;
  }
  double* T = (double*)malloc((size_t)(nI * nJ) * sizeof(double));
  for (int64_t jj = 0; jj < nJ; ++jj) {
    for (int64_t ii = 0; ii < nI; ++ii) {
      int64_t i = i0 + ii, j = j0 + jj;
      double acc = dot_row_col(p, i, j, 0, -1);
      for (int64_t q = 0; q < n_inj; ++q)
        if (inj[q].i == i && inj[q].j == j && inj[q].site == OR_SITE_ACCUM && inj[q].mode == OR_MODE_BITFLIP)
          acc = flip_bit32(acc, inj[q].bit);
      double v = round32(scale_out(p, acc, i, j));
      for (int64_t q = 0; q < n_inj; ++q) {
        if (inj[q].i != i || inj[q].j != j || inj[q].site != OR_SITE_OUTPUT) continue;
        if (inj[q].mode == OR_MODE_BITFLIP) {
          v = flip_bit32(v, inj[q].bit);
        } else {
          double e = ldexp(fabs(v), inj[q].rel_log2);
          v = round32((inj[q].sign < 0) ? v - e : v + e);
        }
      }
      T[ii + jj * nI] = v;
    }
  }
  const double gK = gamma_n((double)K * p->u_acc / 1.1102230246251565e-16);
  const double g24 = gamma_n((double)K * 5.9604644775390625e-08 / 1.1102230246251565e-16);  /* gamma_K(2^-24) */
  /* gamma_{tile_n}(2^-24) and gamma_{tile_m}(2^-24): rounding of the binary32 sums B e and e^T A */
  const double genc_r = gamma_n((double)p->tile_n * 5.9604644775390625e-08 / 1.1102230246251565e-16);
  const double genc_c = gamma_n((double)p->tile_m * 5.9604644775390625e-08 / 1.1102230246251565e-16);
  const double piece_sum = (p->precision == OR_PREC_ACC32_E4M3) ? 1.25 : 1.0078125;
  /* Row side, every row. */
  int64_t nr = 0, fr = -1;
  double fr_delta = 0.0, fr_tau = 0.0, fr_pred = 0.0;
  for (int64_t ii = 0; ii < nI; ++ii) {
    int64_t i = i0 + ii;
    double dotp = 0.0, rowAbsA = 0.0;
    for (int64_t k = 0; k < K; ++k) { double a = a_elem(p, i, k); dotp = dotp + a * Br[k]; rowAbsA = rowAbsA + fabs(a); }
    double cin_sum = 0.0, Q = 0.0;
    if (p->beta != 0.0)
      for (int64_t jj = 0; jj < nJ; ++jj) { double c = cin_elem(p, i, j0 + jj); cin_sum = cin_sum + c; Q = Q + fabs(c); }
    double Cr = p->alpha * dotp;
    if (p->beta != 0.0) Cr = Cr + p->beta * cin_sum;
    for (int64_t q = 0; q < n_inj; ++q) {
      if (inj[q].site != OR_SITE_CHECKSUM || inj[q].i != i || inj[q].j / p->tile_n != tc) continue;
      double e = ldexp(fabs(Cr), inj[q].rel_log2);
      Cr = (inj[q].sign < 0) ? Cr - e : Cr + e;
    }
    double Cr_ref = 0.0, R = 0.0;
    for (int64_t jj = 0; jj < nJ; ++jj) { Cr_ref = Cr_ref + T[ii + jj * nI]; R = R + fabs(T[ii + jj * nI]); }
    double P = rowAbsA * maxAbsBe;
    double tau = fabs(p->alpha) * P * (gK * (1.0 + piece_sum) + 9.5367431640625e-07 + genc_r) +
                 1.1920928955078125e-07 * R + 4.76837158203125e-07 * fabs(p->beta) * Q;
    double d = Cr_ref - Cr;
    if (!(fabs(d) <= tau) || isinf(d)) {
      if (fr < 0) { fr = ii; fr_delta = d; fr_tau = tau; fr_pred = Cr; }
      ++nr;
    }
  }
  /* Column side, only when a row mismatched. */
  int64_t nc = 0, fc = -1;
  double fc_delta = 0.0, fc_tau = 0.0;
  if (nr > 0) {
    for (int64_t jj = 0; jj < nJ; ++jj) {
      int64_t j = j0 + jj;
      double dotp = 0.0, P = 0.0;
      for (int64_t k = 0; k < K; ++k) { double b = b_elem(p, k, j); dotp = dotp + Ac[k] * b; P = P + Ac_abs[k] * fabs(b); }
      double cin_sum = 0.0, Q = 0.0;
      if (p->beta != 0.0)
        for (int64_t ii = 0; ii < nI; ++ii) { double c = cin_elem(p, i0 + ii, j); cin_sum = cin_sum + c; Q = Q + fabs(c); }
      double Cc = p->alpha * dotp;
      if (p->beta != 0.0) Cc = Cc + p->beta * cin_sum;
      double Cc_ref = 0.0, R = 0.0;
      for (int64_t ii = 0; ii < nI; ++ii) { Cc_ref = Cc_ref + T[ii + jj * nI]; R = R + fabs(T[ii + jj * nI]); }
      double tau = fabs(p->alpha) * P * (gK + g24 + 2.384185791015625e-07 + genc_c) +
                   1.1920928955078125e-07 * (R + 34.0 * fabs(p->beta) * Q);
      double d = Cc_ref - Cc;
      if (!(fabs(d) <= tau) || isinf(d)) {
        if (fc < 0) { fc = jj; fc_delta = d; fc_tau = tau; }
        ++nc;
      }
    }
  }
  /* Row-recompute locator: one mismatching row and no mismatching column (the column
   * checksums of a tile whose rows differ greatly in scale cannot resolve an error in a
   * small row), beta == 0. Each element of that row is compared with its own recomputed
   * value against |alpha| (gamma_K(u_acc) + 2^-30) sum_k |A(i,k)||B(k,j)| + 2^-23 |C(i,j)|. */
  int64_t ne = 0, fe = -1;
  const int recompute_row = (nr == 1 && nc == 0 && p->beta == 0.0);
  if (recompute_row) {
    int64_t i = i0 + fr;
    for (int64_t jj = 0; jj < nJ; ++jj) {
      int64_t j = j0 + jj;
      double rec = 0.0, S = 0.0;
      for (int64_t k = 0; k < K; ++k) {
        double a = a_elem(p, i, k), b = b_elem(p, k, j);
        rec = rec + a * b;
        S = S + fabs(a) * fabs(b);
      }
      rec = p->alpha * rec;
      double cij = T[fr + jj * nI];
      double te = fabs(p->alpha) * S * (gK + g24 + 9.313225746154785e-10) + 1.1920928955078125e-07 * fabs(cij);
      double d = cij - rec;
      if (!(fabs(d) <= te) || isinf(d)) {
        if (fe < 0) fe = jj;
        ++ne;
      }
    }
  }
  int64_t located = -1;
  if (nr == 1 && nc == 1) located = fc;
  else if (recompute_row && ne == 1) located = fe;
  oracle_record_t r;
  memset(&r, 0, sizeof(r));
  r.tile_row = tr; r.tile_col = tc;
  r.i = (fr >= 0) ? i0 + fr : -1;
  r.j = (fc >= 0) ? j0 + fc : (located >= 0 ? j0 + located : -1);
  r.delta_row = fr_delta; r.delta_col = fc_delta; r.tau_row = fr_tau; r.tau_col = fc_tau;
  r.rows_flagged = (int32_t)nr; r.cols_flagged = (int32_t)(nc > 0 ? nc : (recompute_row ? ne : 0));
  if (nr == 0) {
    /* clean */
  } else if (located >= 0) {
    res->detected += 1; res->corrected += 1;
    r.kind = OR_KIND_CORRECTED;
    const int64_t fcl = located;
    double before = T[fr + fcl * nI];
    r.value_before = before;
    r.value_subtracted = before - fr_delta;
    /* C(i,j) - delta_row equals C^r(i) - sum_{j' != j} C(i,j') in exact arithmetic; the
     * second form never touches the erroneous value, so a huge or non-finite error does
     * not cancel catastrophically. */
    double rest = 0.0;
    for (int64_t jj = 0; jj < nJ; ++jj)
      if (jj != fcl) rest = rest + T[fr + jj * nI];
    double after = fr_pred - rest;
    T[fr + fcl * nI] = round32(after);
    r.value_after = T[fr + fcl * nI];
    add_record(res, &r);
  } else if (nc == 0 && (!recompute_row || ne == 0)) {
    res->detected += 1; res->checksum_only += 1;
    r.kind = OR_KIND_CHECKSUM_ONLY;
    add_record(res, &r);
  } else {
    res->detected += 1; res->uncorrectable += 1;
    r.kind = OR_KIND_UNCORRECTABLE;
    add_record(res, &r);
  }
  for (int64_t jj = 0; jj < nJ; ++jj)
    for (int64_t ii = 0; ii < nI; ++ii)
      Cout[c_index(p->layout, p->ldc, i0 + ii, j0 + jj)] = T[ii + jj * nI];
  free(Ac); free(Ac_abs); free(Br); free(T);
}

/* ABFT-protected C = alpha*op(A)*op(B) + beta*C_in into Cout.
 * sel_tiles: NULL = every tile; otherwise n_sel tile numbers t = tile_row + tile_col *
 * n_tile_rows, and only those tiles of Cout are written. K == 0 or alpha == 0 is the
 * quick return C = beta*C with no checks (tiles_checked stays 0). Returns 0 or -1. */
int oracle_ft_gemm(const oracle_problem_t* p, int64_t n_inj, const oracle_injection_t* inj,
                   int64_t n_sel, const int64_t* sel_tiles, double* Cout, oracle_report_t* rep) {
  memset(rep, 0, sizeof(*rep));
  if (p->M < 0 || p->N < 0 || p->K < 0 || p->tile_m <= 0 || p->tile_n <= 0 || p->bk <= 0) return -1;
  if (p->M == 0 || p->N == 0) return 0;
  int64_t tr = (p->M + p->tile_m - 1) / p->tile_m, tc = (p->N + p->tile_n - 1) / p->tile_n;
  int64_t ntiles = tr * tc;
  int64_t nsel = sel_tiles ? n_sel : ntiles;
  if (p->K == 0 || p->alpha == 0.0) {
    for (int64_t s = 0; s < nsel; ++s) {
      int64_t t = sel_tiles ? sel_tiles[s] : s;
      int64_t r0 = (t % tr) * p->tile_m, c0 = (t / tr) * p->tile_n;
      for (int64_t j = c0; j < c0 + p->tile_n && j < p->N; ++j)
        for (int64_t i = r0; i < r0 + p->tile_m && i < p->M; ++i)
          Cout[c_index(p->layout, p->ldc, i, j)] =
              (p->beta == 0.0) ? 0.0
                               : (IS_ACC32(p) ? round32(p->beta * cin_elem(p, i, j))
                                                                : p->beta * cin_elem(p, i, j));
    }
    return 0;
  }
  tile_result_t* res = (tile_result_t*)calloc((size_t)nsel, sizeof(tile_result_t));
#pragma omp parallel for schedule(dynamic, 1)
  for (int64_t s = 0; s < nsel; ++s) {
    int64_t t = sel_tiles ? sel_tiles[s] : s;
    if (IS_ACC32(p))
      ft_tile_acc32(p, t % tr, t / tr, n_inj, inj, Cout, &res[s]);
    else
      ft_tile(p, t % tr, t / tr, n_inj, inj, Cout, &res[s]);
  }
  /* Merge in tile order (deterministic). */
  for (int64_t s = 0; s < nsel; ++s) {
    rep->tiles_checked += 1;
    rep->detected += res[s].detected;
    rep->corrected += res[s].corrected;
    rep->uncorrectable += res[s].uncorrectable;
    rep->checksum_only += res[s].checksum_only;
    rep->input_nonfinite += res[s].input_nonfinite;
    for (int32_t q = 0; q < res[s].n_rec; ++q)
      if (rep->n_records < OR_MAX_RECORDS) rep->rec[rep->n_records++] = res[s].rec[q];
  }
  free(res);
  return 0;
}
