/*
 * CPU oracle for the emulated FP64 ABFT GEMM: binary64 operands split into small integer
 * slices whose products the tensor cores form exactly, with exact integer checksums.
 *
 * TEST INFRASTRUCTURE ONLY. Only the tests, the smoke check and the benchmark's CPU legs
 * may load this library. The CUDA path never calls it and shares no code with it.
 *
 * The paper (FT-BLAS, Zhai et al., ICS '21) computes in binary64 throughout. Section V.A
 * argues that the checksum work, a matrix-vector product, costs little next to the
 * matrix-matrix product; on hardware whose binary64 units are far slower than its
 * low-precision tensor cores the product itself can be formed from exact integer pieces,
 * which also makes the checksum relations of Section II.A hold exactly. This file is the
 * definition of that method, step by step:
 *
 *   1. Scales. For row i of op(A), e_i is the binary exponent of max_k |A(i,k)| (the e of
 *      frexp: max < 2^e_i <= 2 max); 0 for a zero row. Likewise f_j for column j of op(B).
 *   2. Slices. x = A(i,k) 2^-e_i lies in (-1, 1). With r_0 = 16 x, each slice is the
 *      nearest integer a_p = rint(r_p) (ties to even) and r_{p+1} = 16 (r_p - a_p); every
 *      step is exact in binary64. |a_0| <= 16 and |a_p| <= 8 for p > 0, so every slice is an
 *      E4M3 value. x = sum_p a_p 16^-(p+1) up to 16^-s / 2 after s slices.
 *   3. Group products. G_g(i,j) = sum_{p+q=g} sum_k a_p(i,k) b_q(k,j) for g = 0 .. s-1 (the
 *      pairs with p + q < s). Each is an integer of magnitude at most 64 (s+2) K, below 2^24
 *      for K <= 2^18 / (s+2): a binary32 accumulator holds it, and every partial sum, exactly.
 *   4. Checksums, per verification tile (tile_m rows x tile_n columns). For each q and k,
 *      v = sum_{j in tile} b_q(k,j) is an integer of magnitude below 2^12, written as four
 *      base-16 digits d_t in [-8, 8] (nearest-integer division by 16, ties to even). The
 *      predicted row checksum of group g is P_g(i) = sum_t 16^t sum_{p+q=g} sum_k a_p(i,k)
 *      d_t(q,k); the reference is R_g(i) = sum_{j in tile} G_g(i,j). Both are exact
 *      integers: R_g(i) = P_g(i) on a clean run, so the threshold is zero (Section II.A's
 *      relation C e = A (B e) holds exactly). A row is flagged when they differ, or when a
 *      group value is not an integer of magnitude at most 2^24.
 *   5. Combination. S(i,j) = sum_g G_g(i,j) 16^(s-1-g), exact in 128-bit integers (each
 *      group value taken as the nearest 32-bit integer, NaN as 0, saturating, as the
 *      hardware's conversion does). v(i,j) = ldexp(double(S), e_i + f_j - 4 (s+1)), the
 *      conversion rounded to nearest; C = alpha v + beta C_in as two binary64 products and
 *      a sum (C_in not read when beta == 0).
 *   6. Final check of the binary64 stage (Section V.B's folded C = beta C, verified after
 *      the output is formed): R_C(i) = sum_j C(i,j) against Pi(i) = alpha sum_j v(i,j) +
 *      beta sum_j C_in(i,j), sums in ascending j; flagged when the difference exceeds
 *      tau_C = 2 gamma_{n+2} (|alpha| sum_j |v| + |beta| sum_j |C_in| + sum_j |C|),
 *      gamma_n = n u / (1 - n u), u = 2^-53, n the tile's column count: the rounding of
 *      both sides, doubled.
 *   7. Locate and correct (Sections V.A, VI.C). Each flagged row of a tile is recomputed
 *      from the slices without faults (its groups, S, v and C exactly as above); every
 *      element whose computed value differs from the recomputed one is located and
 *      replaced, so the stored C equals the fault-free C bit for bit. A tile whose flagged
 *      rows hold no differing element had its fault in a checksum: C kept, checksum-only.
 *      More than four flagged rows in one tile: uncorrectable, C left as computed.
 *   8. A row of op(A) or column of op(B) with a non-finite element gives NaN outputs in
 *      its row / column; tiles touching one are reported input_nonfinite and not checked.
 *
 * Injection (Section VI.C), all in the caller's coordinates: the accumulator site flips
 * bit (bit & 31) of the binary32 value of G_g(i,j), g = the point's k-tile field (0 = the
 * most significant group); the output site perturbs C(i,j) after alpha and beta; the
 * checksum site adds sign * max(1, floor(2^rel_log2 |P_0(i)|)) to group 0's predicted row
 * checksum of the tile holding (i,j).
 *
 * Row-major calls are computed in the column-major frame of C^T = op(B)^T op(A)^T (the
 * BLAS identity), so verified rows are the caller's columns there, as in the kernels; the
 * values are the same in both frames.
 *
 * Arithmetic: integers exact (64 and 128 bits), binary64 operations as written, in the
 * order written. Build with -ffp-contract=off.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>

#define EO_ROW_MAJOR 101
#define EO_COL_MAJOR 102
#define EO_TRANS 112

#define EO_SITE_ACCUM 1
#define EO_SITE_OUTPUT 2
#define EO_SITE_CHECKSUM 3
#define EO_MODE_BITFLIP 0

#define EO_KIND_CORRECTED 1
#define EO_KIND_CHECKSUM_ONLY 2
#define EO_KIND_UNCORRECTABLE 3
#define EO_KIND_INPUT_NONFINITE 4

#define EO_MAX_RECORDS 256
#define EO_MAX_FLAGGED_ROWS 4
#define EO_DIGITS 4

typedef __int128 i128;

typedef struct {
  int32_t layout, transa, transb, slices;
  int64_t M, N, K;
  double alpha;
  const double* A; int64_t lda;
  const double* B; int64_t ldb;
  double beta;
  const double* Cin; int64_t ldc;   /* not read when beta == 0 */
  int64_t tile_m, tile_n;           /* verification tile in the column-major (kernel) frame */
} emu_problem_t;

/* Same layout as the FP64 oracle's injection point; kt selects the group. */
typedef struct {
  int64_t i, j;
  int32_t site, mode, bit, rel_log2, sign, kt;
} emu_injection_t;

/* Same layouts as the FP64 oracle's record and report. */
typedef struct {
  int64_t tile_row, tile_col, i, j;
  double delta_row, delta_col, tau_row, tau_col;
  double value_before, value_after, value_subtracted;
  int32_t kind, rows_flagged, cols_flagged, pad_;
} emu_record_t;

typedef struct {
  uint64_t tiles_checked, detected, corrected, uncorrectable, checksum_only, input_nonfinite;
  uint32_t n_records, pad_;
  emu_record_t rec[EO_MAX_RECORDS];
} emu_report_t;

/* ---------------------------------------------------------------------------------- */
/* The column-major (kernel) frame: row-major calls compute C^T = op(B)^T op(A)^T      */
/* ---------------------------------------------------------------------------------- */

typedef struct {
  const emu_problem_t* p;
  int swap;          /* 1: row-major call, frame is the transposed problem */
  int64_t M, N, K;   /* frame dimensions */
  int s;
} frame_t;

/* Element (r, c) of op(X) in BLAS storage. */
static double op_at(const double* X, int64_t ld, int layout, int trans, int64_t r, int64_t c) {
  int64_t a = (trans == EO_TRANS) ? c : r;
  int64_t b = (trans == EO_TRANS) ? r : c;
  return (layout == EO_COL_MAJOR) ? X[a + b * ld] : X[a * ld + b];
}
/* op(A)(i,k) of the frame */
static double fa(const frame_t* f, int64_t i, int64_t k) {
  const emu_problem_t* p = f->p;
  return f->swap ? op_at(p->B, p->ldb, p->layout, p->transb, k, i) : op_at(p->A, p->lda, p->layout, p->transa, i, k);
}
/* op(B)(k,j) of the frame */
static double fb(const frame_t* f, int64_t k, int64_t j) {
  const emu_problem_t* p = f->p;
  return f->swap ? op_at(p->A, p->lda, p->layout, p->transa, j, k) : op_at(p->B, p->ldb, p->layout, p->transb, k, j);
}
/* storage index of C(i,j) of the frame: column-major, or the caller's row-major C(j,i),
 * which is the same index */
static int64_t fc_index(const frame_t* f, int64_t i, int64_t j) {
  return i + j * f->p->ldc;
}

/* ---------------------------------------------------------------------------------- */
/* Steps 1 and 2: scales and slices                                                    */
/* ---------------------------------------------------------------------------------- */

/* e with max = m 2^e, m in [0.5, 1) (0 for a zero maximum); *finite = 0 when a value of
 * the line is not finite. get(k) reads the line. */
static int line_exponent(const frame_t* f, int is_row, int64_t idx, int* finite) {
  double mx = 0.0;
  *finite = 1;
  for (int64_t k = 0; k < f->K; ++k) {
    double v = is_row ? fa(f, idx, k) : fb(f, k, idx);
    if (!isfinite(v)) *finite = 0;
    double a = fabs(v);
    if (a > mx) mx = a;
  }
  if (!(mx > 0.0) || !*finite) return 0;
  int e;
  (void)frexp(mx, &e);
  return e;
}

/* The s slices of x in (-1, 1): r_0 = 16 x, a_p = rint(r_p), r_{p+1} = 16 (r_p - a_p). */
void oracle_emu_split(double x, int s, int32_t* out) {
  double r = ldexp(x, 4);
  for (int q = 0; q < s; ++q) {
    double a = nearbyint(r);
    out[q] = (int32_t)a;
    r = ldexp(r - a, 4);
  }
}

/* Step 4: the four base-16 digits of v (|v| < 2^15), d_t in [-8, 8]. */
void oracle_emu_digits(int64_t v, int32_t* d) {
  for (int t = 0; t < EO_DIGITS; ++t) {
    double c = nearbyint((double)v / 16.0);
    d[t] = (int32_t)(v - 16 * (int64_t)c);
    v = (int64_t)c;
  }
}

/* The hardware's conversion of a binary32 value to a 32-bit integer: nearest (ties to
 * even), saturating, NaN to 0. */
static int32_t to_int32(float x) {
  if (isnan(x)) return 0;
  double r = nearbyint((double)x);
  if (r >= 2147483647.0) return INT32_MAX;
  if (r <= -2147483648.0) return INT32_MIN;
  return (int32_t)r;
}
/* A group value as the accumulator must hold it: an integer of magnitude <= 2^24. */
static int valid_group_value(float x) {
  return isfinite(x) && x == nearbyintf(x) && fabsf(x) <= 16777216.0f;
}
static float flip32(float x, int bit) {
  uint32_t u;
  memcpy(&u, &x, 4);
  u ^= (uint32_t)1 << (bit & 31);
  memcpy(&x, &u, 4);
  return x;
}
static double flip64(double x, int bit) {
  uint64_t u;
  memcpy(&u, &x, 8);
  u ^= (uint64_t)1 << bit;
  memcpy(&x, &u, 8);
  return x;
}

/* Rounded-to-nearest binary64 value of a 128-bit integer (the compiler's conversion),
 * exported so that a test can pin it to an independent exact conversion. */
double oracle_emu_i128_to_double(int64_t hi, uint64_t lo) {
  i128 x = ((i128)hi << 64) | (i128)lo;
  return (double)x;
}

static double gamma_u(double n) {
  const double u = 1.1102230246251565e-16; /* 2^-53 */
  return n * u / (1.0 - n * u);
}

/* ---------------------------------------------------------------------------------- */
/* Steps 3 to 7 on one verification tile                                               */
/* ---------------------------------------------------------------------------------- */

#define EO_TILE_RECORDS 64
typedef struct {
  uint64_t detected, corrected, uncorrectable, checksum_only, input_nonfinite;
  int32_t n_rec;
  emu_record_t rec[EO_TILE_RECORDS];
} emu_tile_result_t;

/* A record in the caller's coordinates (a row-major call swaps rows and columns). */
static void add_rec(const frame_t* f, emu_tile_result_t* res, int kind, int64_t tr, int64_t tc, int64_t i,
                    int64_t j, double delta, double tau, double before, double after, int nr, int nc) {
  if (res->n_rec >= EO_TILE_RECORDS) return;
  emu_record_t* r = &res->rec[res->n_rec++];
  memset(r, 0, sizeof(*r));
  if (f->swap) {
    r->tile_row = tc; r->tile_col = tr; r->i = j; r->j = i;
    r->delta_col = delta; r->tau_col = tau;
    r->rows_flagged = nc; r->cols_flagged = nr;
  } else {
    r->tile_row = tr; r->tile_col = tc; r->i = i; r->j = j;
    r->delta_row = delta; r->tau_row = tau;
    r->rows_flagged = nr; r->cols_flagged = nc;
  }
  r->value_before = before;
  r->value_after = after;
  r->kind = kind;
}

static uint64_t bits64(double x) {
  uint64_t u;
  memcpy(&u, &x, 8);
  return u;
}

/* Injection points of the call, in frame coordinates. */
typedef struct {
  int64_t i, j;
  int32_t site, mode, bit, rel_log2, sign, group;
} fpoint_t;

static void emu_tile(const frame_t* f, int64_t tr, int64_t tc, int64_t npts, const fpoint_t* pts,
                     const int* erow, const int* fin_row, const int* fcol, const int* fin_col, double* Cout,
                     emu_tile_result_t* res) {
  const emu_problem_t* p = f->p;
  const int s = f->s;
  const int64_t K = f->K;
  const int64_t i0 = tr * p->tile_m, j0 = tc * p->tile_n;
  const int64_t nI = (i0 + p->tile_m <= f->M) ? p->tile_m : f->M - i0;
  const int64_t nJ = (j0 + p->tile_n <= f->N) ? p->tile_n : f->N - j0;
  memset(res, 0, sizeof(*res));

  /* slices of the tile's rows of op(A) and columns of op(B) (step 2) */
  int32_t* as = (int32_t*)malloc(sizeof(int32_t) * (size_t)(nI * s * K));   /* as[(ii*s + p)*K + k] */
  int32_t* bs = (int32_t*)malloc(sizeof(int32_t) * (size_t)(nJ * s * K));   /* bs[(jj*s + q)*K + k] */
#pragma omp parallel for schedule(static)
  for (int64_t ii = 0; ii < nI; ++ii)
    for (int64_t k = 0; k < K; ++k) {
      int32_t sl[32];
      oracle_emu_split(fin_row[i0 + ii] ? ldexp(fa(f, i0 + ii, k), -erow[i0 + ii]) : 0.0, s, sl);
      for (int q = 0; q < s; ++q) as[(ii * s + q) * K + k] = sl[q];
    }
#pragma omp parallel for schedule(static)
  for (int64_t jj = 0; jj < nJ; ++jj)
    for (int64_t k = 0; k < K; ++k) {
      int32_t sl[32];
      oracle_emu_split(fin_col[j0 + jj] ? ldexp(fb(f, k, j0 + jj), -fcol[j0 + jj]) : 0.0, s, sl);
      for (int q = 0; q < s; ++q) bs[(jj * s + q) * K + k] = sl[q];
    }
  /* checksum digits of the tile's column block (step 4): dg[(q*EO_DIGITS + t)*K + k] */
  int32_t* dg = (int32_t*)malloc(sizeof(int32_t) * (size_t)(s * EO_DIGITS * K));
  for (int q = 0; q < s; ++q)
    for (int64_t k = 0; k < K; ++k) {
      int64_t v = 0;
      for (int64_t jj = 0; jj < nJ; ++jj) v += bs[(jj * s + q) * K + k];
      int32_t d[EO_DIGITS];
      oracle_emu_digits(v, d);
      for (int t = 0; t < EO_DIGITS; ++t) dg[(q * EO_DIGITS + t) * K + k] = d[t];
    }

  int tile_nonfinite = 0;
  for (int64_t ii = 0; ii < nI; ++ii) if (!fin_row[i0 + ii]) tile_nonfinite = 1;
  for (int64_t jj = 0; jj < nJ; ++jj) if (!fin_col[j0 + jj]) tile_nonfinite = 1;

  double* Cc = (double*)malloc(sizeof(double) * (size_t)(nI * nJ));  /* computed, Cc[ii*nJ + jj] */
  double* Ct = (double*)malloc(sizeof(double) * (size_t)(nI * nJ));  /* fault-free */
  int* flagged = (int*)calloc((size_t)nI, sizeof(int));
  double* fdelta = (double*)calloc((size_t)nI, sizeof(double));
  double* ftau = (double*)calloc((size_t)nI, sizeof(double));
  const int shift = -4 * (s + 1);

  /* rows are independent: OpenMP may split them across threads (every sum below is exact
   * or taken in the order written within one row) */
#pragma omp parallel for schedule(dynamic, 1)
  for (int64_t ii = 0; ii < nI; ++ii) {
    const int64_t i = i0 + ii;
    i128* S = (i128*)malloc(sizeof(i128) * (size_t)nJ);
    i128* St = (i128*)malloc(sizeof(i128) * (size_t)nJ);
    for (int64_t jj = 0; jj < nJ; ++jj) { S[jj] = 0; St[jj] = 0; }
    for (int g = 0; g < s; ++g) {
      /* step 3: group values as the accumulators hold them, and the reference row sum */
      int64_t R = 0;
      int invalid = 0;
      for (int64_t jj = 0; jj < nJ; ++jj) {
        int64_t G = 0;
        for (int pp = 0; pp <= g; ++pp) {
          const int32_t* a = &as[(ii * s + pp) * K];
          const int32_t* b = &bs[(jj * s + (g - pp)) * K];
          for (int64_t k = 0; k < K; ++k) G += (int64_t)a[k] * b[k];
        }
        St[jj] = St[jj] * 16 + G;
        float Gf = (float)G;
        for (int64_t e = 0; e < npts; ++e)
          if (pts[e].site == EO_SITE_ACCUM && pts[e].mode == EO_MODE_BITFLIP && pts[e].i == i && pts[e].j == j0 + jj &&
              pts[e].group == g)
            Gf = flip32(Gf, pts[e].bit);
        if (!valid_group_value(Gf)) invalid = 1;
        int32_t gi = to_int32(Gf);
        R += gi;
        S[jj] = S[jj] * 16 + gi;
      }
      /* step 4: the prediction from the checksum digits */
      int64_t P = 0, w = 1;
      for (int t = 0; t < EO_DIGITS; ++t, w *= 16) {
        int64_t acc = 0;
        for (int pp = 0; pp <= g; ++pp) {
          const int32_t* a = &as[(ii * s + pp) * K];
          const int32_t* d = &dg[((g - pp) * EO_DIGITS + t) * K];
          for (int64_t k = 0; k < K; ++k) acc += (int64_t)a[k] * d[k];
        }
        P += w * acc;
      }
      if (g == 0)
        for (int64_t e = 0; e < npts; ++e)
          if (pts[e].site == EO_SITE_CHECKSUM && pts[e].i == i && pts[e].j >= j0 && pts[e].j < j0 + nJ) {
            double m = floor(ldexp(fabs((double)P), pts[e].rel_log2));
            int64_t add = (m < 1.0) ? 1 : (int64_t)m;
            P += (pts[e].sign < 0) ? -add : add;
          }
      if (!flagged[ii] && (invalid || R != P)) { flagged[ii] = 1; fdelta[ii] = (double)(R - P); ftau[ii] = 0.0; }
    }
    /* steps 5 and 6: the binary64 stage and its check */
    double V = 0.0, aV = 0.0, Q = 0.0, aQ = 0.0, RC = 0.0, aC = 0.0;
    for (int64_t jj = 0; jj < nJ; ++jj) {
      const int64_t j = j0 + jj;
      double v, vt;
      if (!fin_row[i] || !fin_col[j]) {
        v = NAN; vt = NAN;
      } else {
        v = ldexp((double)S[jj], erow[i] + fcol[j] + shift);
        vt = ldexp((double)St[jj], erow[i] + fcol[j] + shift);
      }
      double cin = (p->beta != 0.0) ? p->Cin[fc_index(f, i, j)] : 0.0;
      double c = p->alpha * v, ct = p->alpha * vt;
      if (p->beta != 0.0) {
        double bc = p->beta * cin;
        c = c + bc;
        ct = ct + bc;
      }
      for (int64_t e = 0; e < npts; ++e) {
        if (pts[e].site != EO_SITE_OUTPUT || pts[e].i != i || pts[e].j != j) continue;
        if (pts[e].mode == EO_MODE_BITFLIP) {
          c = flip64(c, pts[e].bit);
        } else {
          double em = ldexp(fabs(c), pts[e].rel_log2);
          c = (pts[e].sign < 0) ? c - em : c + em;
        }
      }
      Cc[ii * nJ + jj] = c;
      Ct[ii * nJ + jj] = ct;
      V = V + v; aV = aV + fabs(v);
      if (p->beta != 0.0) { Q = Q + cin; aQ = aQ + fabs(cin); }
      RC = RC + c; aC = aC + fabs(c);
    }
    double Pi = p->alpha * V;
    if (p->beta != 0.0) Pi = Pi + p->beta * Q;
    double tauC = 2.0 * gamma_u((double)(nJ + 2)) * ((fabs(p->alpha) * aV + fabs(p->beta) * aQ) + aC);
    double d = RC - Pi;
    if (!flagged[ii] && (!(fabs(d) <= tauC) || isinf(d))) { flagged[ii] = 1; fdelta[ii] = d; ftau[ii] = tauC; }
    free(S);
    free(St);
  }

  /* step 7: classification, location by recomputation, correction */
  int64_t nf = 0, first = -1;
  for (int64_t ii = 0; ii < nI; ++ii)
    if (flagged[ii]) { if (first < 0) first = ii; ++nf; }
  int located_total = 0;
  if (!tile_nonfinite && nf > 0 && nf <= EO_MAX_FLAGGED_ROWS)
    for (int64_t ii = 0; ii < nI; ++ii)
      if (flagged[ii])
        for (int64_t jj = 0; jj < nJ; ++jj)
          if (bits64(Cc[ii * nJ + jj]) != bits64(Ct[ii * nJ + jj])) ++located_total;
  if (tile_nonfinite) {
    res->input_nonfinite += 1;
    add_rec(f, res, EO_KIND_INPUT_NONFINITE, tr, tc, -1, -1, 0.0, 0.0, 0.0, 0.0, 0, 0);
  } else if (nf > EO_MAX_FLAGGED_ROWS) {
    res->detected += 1; res->uncorrectable += 1;
    add_rec(f, res, EO_KIND_UNCORRECTABLE, tr, tc, i0 + first, -1, fdelta[first], ftau[first], 0.0, 0.0, (int)nf, 0);
  } else if (nf > 0) {
    res->detected += 1;
    if (located_total > 0) {
      res->corrected += 1;
      for (int64_t ii = 0; ii < nI; ++ii) {
        if (!flagged[ii]) continue;
        for (int64_t jj = 0; jj < nJ; ++jj) {
          double before = Cc[ii * nJ + jj], after = Ct[ii * nJ + jj];
          if (bits64(before) != bits64(after))
            add_rec(f, res, EO_KIND_CORRECTED, tr, tc, i0 + ii, j0 + jj, fdelta[ii], ftau[ii], before, after, (int)nf,
                    located_total);
          Cc[ii * nJ + jj] = after;   /* the flagged row is stored as recomputed */
        }
      }
    } else {
      res->checksum_only += 1;
      add_rec(f, res, EO_KIND_CHECKSUM_ONLY, tr, tc, i0 + first, -1, fdelta[first], ftau[first], 0.0, 0.0, (int)nf, 0);
    }
  }
  for (int64_t ii = 0; ii < nI; ++ii)
    for (int64_t jj = 0; jj < nJ; ++jj) Cout[fc_index(f, i0 + ii, j0 + jj)] = Cc[ii * nJ + jj];

  free(as); free(bs); free(dg); free(Cc); free(Ct); free(flagged); free(fdelta); free(ftau);
}

/* ---------------------------------------------------------------------------------- */
/* The protected product                                                               */
/* ---------------------------------------------------------------------------------- */

/* Largest K whose group values stay within 2^24 for s slices: 64 (s+2) K <= 2^24. */
int64_t oracle_emu_max_k(int s) { return ((int64_t)1 << 18) / (s + 2); }

/* The emulated protected C = alpha op(A) op(B) + beta C_in into Cout (caller's storage;
 * unselected tiles untouched). sel_tiles: NULL for all tiles, else tile numbers t = tile_row
 * + tile_col * n_tile_rows in the caller's coordinates, whose tiles are tile_m x tile_n in
 * the column-major frame (tile_n x tile_m for a row-major call). Returns 0, -1 for bad
 * arguments, -2 when K exceeds oracle_emu_max_k(slices). */
int oracle_emu_gemm(const emu_problem_t* p, int64_t n_inj, const emu_injection_t* inj, int64_t n_sel,
                    const int64_t* sel_tiles, double* Cout, emu_report_t* rep) {
  memset(rep, 0, sizeof(*rep));
  if (p->M < 0 || p->N < 0 || p->K < 0 || p->tile_m <= 0 || p->tile_n <= 0) return -1;
  if (p->slices < 1 || p->slices > 24) return -1;
  if (p->M == 0 || p->N == 0) return 0;
  if (p->K > oracle_emu_max_k(p->slices)) return -2;
  frame_t f;
  f.p = p;
  f.swap = p->layout == EO_ROW_MAJOR;
  f.M = f.swap ? p->N : p->M;
  f.N = f.swap ? p->M : p->N;
  f.K = p->K;
  f.s = p->slices;
  if (p->K == 0 || p->alpha == 0.0) {  /* quick return C = beta C, no checks */
    for (int64_t j = 0; j < f.N; ++j)
      for (int64_t i = 0; i < f.M; ++i) {
        int64_t x = fc_index(&f, i, j);
        Cout[x] = (p->beta == 0.0) ? 0.0 : p->beta * p->Cin[x];
      }
    return 0;
  }
  int* erow = (int*)malloc(sizeof(int) * (size_t)f.M);
  int* fin_row = (int*)malloc(sizeof(int) * (size_t)f.M);
  int* fcol = (int*)malloc(sizeof(int) * (size_t)f.N);
  int* fin_col = (int*)malloc(sizeof(int) * (size_t)f.N);
  for (int64_t i = 0; i < f.M; ++i) erow[i] = line_exponent(&f, 1, i, &fin_row[i]);
  for (int64_t j = 0; j < f.N; ++j) fcol[j] = line_exponent(&f, 0, j, &fin_col[j]);
  fpoint_t* pts = (fpoint_t*)malloc(sizeof(fpoint_t) * (size_t)(n_inj > 0 ? n_inj : 1));
  for (int64_t e = 0; e < n_inj; ++e) {
    pts[e].i = f.swap ? inj[e].j : inj[e].i;
    pts[e].j = f.swap ? inj[e].i : inj[e].j;
    pts[e].site = inj[e].site; pts[e].mode = inj[e].mode; pts[e].bit = inj[e].bit;
    pts[e].rel_log2 = inj[e].rel_log2; pts[e].sign = inj[e].sign; pts[e].group = inj[e].kt;
  }
  const int64_t ftr = (f.M + p->tile_m - 1) / p->tile_m, ftc = (f.N + p->tile_n - 1) / p->tile_n;
  const int64_t ctr = f.swap ? ftc : ftr;  /* tile rows in the caller's coordinates */
  const int64_t nsel = sel_tiles ? n_sel : ftr * ftc;
  emu_tile_result_t* res = (emu_tile_result_t*)calloc((size_t)(nsel > 0 ? nsel : 1), sizeof(emu_tile_result_t));
  for (int64_t q = 0; q < nsel; ++q) {
    int64_t tr, tc;
    if (sel_tiles) {
      int64_t c_r = sel_tiles[q] % ctr, c_c = sel_tiles[q] / ctr;
      tr = f.swap ? c_c : c_r;
      tc = f.swap ? c_r : c_c;
    } else {
      tr = q % ftr;
      tc = q / ftr;
    }
    emu_tile(&f, tr, tc, n_inj, pts, erow, fin_row, fcol, fin_col, Cout, &res[q]);
  }
  for (int64_t q = 0; q < nsel; ++q) {
    rep->tiles_checked += 1;
    rep->detected += res[q].detected;
    rep->corrected += res[q].corrected;
    rep->uncorrectable += res[q].uncorrectable;
    rep->checksum_only += res[q].checksum_only;
    rep->input_nonfinite += res[q].input_nonfinite;
    for (int32_t r = 0; r < res[q].n_rec; ++r)
      if (rep->n_records < EO_MAX_RECORDS) rep->rec[rep->n_records++] = res[q].rec[r];
  }
  free(res); free(pts); free(erow); free(fin_row); free(fcol); free(fin_col);
  return 0;
}
