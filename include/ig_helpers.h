/*
 * ig_helpers.h -- host helpers around the IG library: the preprocessing that
 * turns raw flow attributes into the codes ig_encode takes, the contradiction
 * filter, and the detection metrics of the evaluation.
 *
 * These functions run on the host over HOST arrays only (never device
 * pointers); they launch no kernel and need no GPU.  They return IG_OK (0) or
 * a negative status of ig.h, with the message readable via ig_last_error().
 * Floating-point work is plain IEEE double arithmetic in the order stated per
 * function, without contraction, so that its results are reproducible.
 */
#ifndef IG_GB300_HELPERS_H
#define IG_GB300_HELPERS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Discretiser of Section 3.1: numeric attributes are z-scored and rounded to
 * p decimals, categorical values are kept as they are, and each (column,
 * value) pair becomes one token (one item of the itemset).
 *
 * fit_values: double[n_fit][F], row-major.  The statistics and the token
 *   vocabulary come from these rows.  A non-finite value (NaN, +-inf) is a
 *   missing value.
 * values:     double[n][F], the rows to code (may be fit_values itself).
 * categorical: uint8[F]; non-zero marks a categorical column.
 * p: decimals kept after z-scoring, 0 <= p <= 9.
 *
 * Numeric column f: mu_f = (sum of its present fit values, in row order) /
 * count; sigma_f = sqrt((sum of (x - mu_f)^2, in row order) / count), the
 * population deviation.  The token of x is the integer
 * t = rint(((x - mu_f) / sigma_f) * 10^p) (round half to even), i.e. z
 * rounded to p decimals and scaled by 10^p; t = 0 where sigma_f is 0 or the
 * column has no fit value.  Categorical column: the token is x itself.
 *
 * codes_out: uint16[n][F]; codes_out[i][f] = rank of the token of
 *   values[i][f] among the distinct tokens of column f in fit_values
 *   (ascending), or 0xFFFF (missing: no item) where values[i][f] is
 *   missing or its token never occurs in fit_values.  -0 and +0 are one
 *   value.
 * cards_out: uint16[F], the number of distinct tokens per column.
 * Returns IG_E_INVAL for bad sizes or p, IG_E_OVERFLOW if a column has more
 * than 65535 distinct tokens or a fit value's token reaches 2^62 in
 * magnitude (a value of `values` with such a token is coded missing). */
int ig_discretize(const double* fit_values, int64_t n_fit, const double* values,
                  int64_t n, int32_t F, const uint8_t* categorical, int32_t p,
                  uint16_t* codes_out, uint16_t* cards_out);

/* Anti-contradiction filter (the last stage of the preprocessing pipeline of
 * Section 4): records with the same itemset but opposite labels contradict
 * each other.
 *
 * rows: uint64[n][K] (encoded records); labels: uint8[n] in {0, 1}.
 * mode 0: within each itemset, the k-th attack record and the k-th normal
 *   record (k counted in record order) form a contradicting pair and both
 *   are dropped; the surplus records of the majority label are kept.
 * mode 1: every record whose itemset occurs under both labels is dropped.
 * keep_out: uint8[n], 1 = kept.  *n_kept_out (may be NULL) = records kept.
 * Returns IG_E_INVAL for a bad mode, K or label. */
int ig_filter_contradictions(const uint64_t* rows, const uint8_t* labels,
                             int64_t n, int32_t K, int32_t mode,
                             uint8_t* keep_out, int64_t* n_kept_out);

/* Detection metrics of the evaluation (Section 4, Table 2): positive class =
 * attack (label 1). */
typedef struct {
  int64_t tp, fp, tn, fn;
  double accuracy;   /* (tp + tn) / m */
  double precision;  /* tp / (tp + fp) */
  double recall;     /* tp / (tp + fn) */
  double f1;         /* 2 tp / (2 tp + fp + fn) */
  /* Area under the ROC curve of the continuous score s = A - N: the
   * probability that an attack record scores above a normal one, ties
   * counting one half (Mann-Whitney).  Computed as the exact integer
   * 2U = sum over attack/normal pairs of (2 if s_a > s_n, 1 if equal), then
   * auc = (double)2U / (2.0 * (double)n_attack * (double)n_normal). */
  double auc;
} ig_metrics_t;

/* y_true, y_pred: uint8[m] in {0, 1}.  A, N: int64[m] evidence from
 * ig_score, or both NULL (auc is then NaN).  A ratio with a zero
 * denominator (and auc without both classes) is NaN.  m == 0 is valid. */
int ig_evaluate(const uint8_t* y_true, const uint8_t* y_pred, const int64_t* A,
                const int64_t* N, int64_t m, ig_metrics_t* out);

/* Regulation 3 sweep: metrics of the labels that Regulations 1-3 give for
 * each of n_r values of r, from evidence A, N (int64[m]) and the statistics
 * mu, sigma of a model fitted with Regulation 3 (ig_model_info_t's reg3_mu
 * and reg3_sigma).  For each r: thr = mu - (r * sigma), the product rounded
 * first; a record is labelled attack if A >= N (Regulation 1), A == N == 0
 * (Regulation 2) or (double)N < thr (Regulation 3) -- the rule ig_score
 * applies.  r = +inf switches Regulation 3 off.  out: ig_metrics_t[n_r]. */
int ig_reg3_sweep(const int64_t* A, const int64_t* N, const uint8_t* y_true,
                  int64_t m, double mu, double sigma, const double* r,
                  int32_t n_r, ig_metrics_t* out);

#ifdef __cplusplus
}
#endif
#endif /* IG_GB300_HELPERS_H */
