// Host helpers of ig_helpers.h: the discretiser of Section 3.1, the
// anti-contradiction filter of the Section 4 preprocessing pipeline, and the
// detection metrics of Section 4 (Table 2), plus a Regulation 3 sweep.
// Plain host code: no kernel is launched and no GPU is needed.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <numeric>
#include <string>
#include <vector>

#include "ig.h"
#include "ig_helpers.h"
#include "internal.h"

namespace {

int fail(int code, const std::string& msg) { return igk::report_error(code, msg.c_str()); }

constexpr uint16_t kMissing = 0xFFFF;
constexpr double kTokenLimit = 4611686018427387904.0;  // 2^62

// Tokens of one column: the value itself (categorical) or the z-score
// rounded to p decimals, as the integer rint(z * 10^p) (numeric).
struct Column {
  bool categorical = false;
  double mu = 0.0, sigma = 0.0, scale = 1.0;

  // false if the value is missing (non-finite); else *t is its token.
  // Tokens of both kinds are kept as doubles: a numeric token is an integer
  // below 2^62 in magnitude, which a double holds exactly.
  bool token(double x, double* t, bool* overflow) const {
    if (!std::isfinite(x)) return false;
    if (categorical) {
      *t = x == 0.0 ? 0.0 : x;  // -0 and +0 are one value
      return true;
    }
    if (!(sigma > 0.0)) {
      *t = 0.0;
      return true;
    }
    const double z = (x - mu) / sigma;
    const double zs = z * scale;
    if (!std::isfinite(zs) || std::fabs(zs) >= kTokenLimit) {
      *overflow = true;
      return false;
    }
    *t = std::nearbyint(zs);  // round half to even (default rounding mode)
    if (*t == 0.0) *t = 0.0;
    return true;
  }
};

double ratio(int64_t a, int64_t b) { return b ? double(a) / double(b) : std::nan(""); }

void fill_counts(const uint8_t* y_true, const uint8_t* y_pred, int64_t m, ig_metrics_t* o) {
  int64_t tp = 0, fp = 0, tn = 0, fn = 0;
  for (int64_t i = 0; i < m; ++i) {
    if (y_pred[i]) {
      if (y_true[i]) ++tp; else ++fp;
    } else {
      if (y_true[i]) ++fn; else ++tn;
    }
  }
  o->tp = tp;
  o->fp = fp;
  o->tn = tn;
  o->fn = fn;
  o->accuracy = ratio(tp + tn, m);
  o->precision = ratio(tp, tp + fp);
  o->recall = ratio(tp, tp + fn);
  o->f1 = ratio(2 * tp, 2 * tp + fp + fn);
}

// Mann-Whitney AUC of s = A - N (attack = positive), ties counting half.
double auc_of(const uint8_t* y_true, const int64_t* A, const int64_t* N, int64_t m) {
  std::vector<__int128> s(static_cast<size_t>(m));
  for (int64_t i = 0; i < m; ++i) s[i] = __int128(A[i]) - __int128(N[i]);
  std::vector<int64_t> order(static_cast<size_t>(m));
  std::iota(order.begin(), order.end(), int64_t(0));
  std::sort(order.begin(), order.end(), [&](int64_t a, int64_t b) { return s[a] < s[b]; });
  uint64_t two_u = 0, neg_below = 0, n_pos = 0, n_neg = 0;
  for (int64_t g0 = 0; g0 < m;) {
    int64_t g1 = g0;
    uint64_t pg = 0, ng = 0;
    while (g1 < m && s[order[g1]] == s[order[g0]]) {
      if (y_true[order[g1]]) ++pg; else ++ng;
      ++g1;
    }
    two_u += 2 * pg * neg_below + pg * ng;
    neg_below += ng;
    n_pos += pg;
    n_neg += ng;
    g0 = g1;
  }
  if (n_pos == 0 || n_neg == 0) return std::nan("");
  return double(two_u) / (2.0 * double(n_pos) * double(n_neg));
}

bool labels_ok(const uint8_t* y, int64_t m) {
  for (int64_t i = 0; i < m; ++i)
    if (y[i] > 1) return false;
  return true;
}

constexpr int64_t kMaxEvalRows = int64_t(1) << 31;  // keeps 2U below 2^63

}  // namespace

extern "C" int ig_discretize(const double* fit_values, int64_t n_fit, const double* values,
                             int64_t n, int32_t F, const uint8_t* categorical, int32_t p,
                             uint16_t* codes_out, uint16_t* cards_out) {
  return igk::guarded("ig_discretize", [&]() -> int {
    if (n_fit < 0 || n < 0 || F <= 0 || p < 0 || p > 9 || !categorical || !cards_out ||
        (n_fit > 0 && !fit_values) || (n > 0 && (!values || !codes_out)))
      return fail(IG_E_INVAL, "ig_discretize: bad arguments");
    double scale = 1.0;
    for (int k = 0; k < p; ++k) scale *= 10.0;
    std::vector<double> tok;
    for (int32_t f = 0; f < F; ++f) {
      Column col;
      col.categorical = categorical[f] != 0;
      col.scale = scale;
      if (!col.categorical) {
        // Population statistics over the column's present fit values, summed
        // in row order.
        double sum = 0.0;
        int64_t cnt = 0;
        for (int64_t i = 0; i < n_fit; ++i) {
          const double x = fit_values[i * F + f];
          if (std::isfinite(x)) {
            sum += x;
            ++cnt;
          }
        }
        if (cnt > 0) {
          col.mu = sum / double(cnt);
          double ss = 0.0;
          for (int64_t i = 0; i < n_fit; ++i) {
            const double x = fit_values[i * F + f];
            if (std::isfinite(x)) {
              const double d = x - col.mu;
              ss += d * d;
            }
          }
          col.sigma = std::sqrt(ss / double(cnt));
        }
      }
      // Vocabulary: the distinct tokens of the fit rows, ascending.
      tok.clear();
      bool overflow = false;
      for (int64_t i = 0; i < n_fit; ++i) {
        double t;
        if (col.token(fit_values[i * F + f], &t, &overflow)) tok.push_back(t);
      }
      if (overflow)
        return fail(IG_E_OVERFLOW, "ig_discretize: column " + std::to_string(f) +
                                       ": a z-score token exceeds 2^62");
      std::sort(tok.begin(), tok.end());
      tok.erase(std::unique(tok.begin(), tok.end()), tok.end());
      if (tok.size() > 65535u)
        return fail(IG_E_OVERFLOW, "ig_discretize: column " + std::to_string(f) +
                                       " has more than 65535 distinct tokens");
      cards_out[f] = uint16_t(tok.size());
      for (int64_t i = 0; i < n; ++i) {
        double t;
        bool ovf = false;
        uint16_t code = kMissing;
        if (col.token(values[i * F + f], &t, &ovf)) {
          auto it = std::lower_bound(tok.begin(), tok.end(), t);
          if (it != tok.end() && *it == t) code = uint16_t(it - tok.begin());
        }
        codes_out[i * F + f] = code;  // missing, unseen or out-of-range tokens: no item
      }
    }
    return IG_OK;
  });
}

extern "C" int ig_filter_contradictions(const uint64_t* rows, const uint8_t* labels, int64_t n,
                                        int32_t K, int32_t mode, uint8_t* keep_out,
                                        int64_t* n_kept_out) {
  return igk::guarded("ig_filter_contradictions", [&]() -> int {
    if (n < 0 || K < 1 || K > IG_MAX_WORDS || (mode != 0 && mode != 1) ||
        (n > 0 && (!rows || !labels || !keep_out)))
      return fail(IG_E_INVAL, "ig_filter_contradictions: bad arguments");
    if (!labels_ok(labels, n)) return fail(IG_E_INVAL, "ig_filter_contradictions: label > 1");
    // Group equal itemsets: sort record indices by their words, ties by index,
    // so that each group lists its records in record order.
    std::vector<int64_t> order(static_cast<size_t>(n));
    std::iota(order.begin(), order.end(), int64_t(0));
    auto less = [&](int64_t a, int64_t b) {
      const uint64_t* ra = rows + a * K;
      const uint64_t* rb = rows + b * K;
      for (int w = 0; w < K; ++w)
        if (ra[w] != rb[w]) return ra[w] < rb[w];
      return a < b;
    };
    std::sort(order.begin(), order.end(), less);
    auto same = [&](int64_t a, int64_t b) {
      return std::equal(rows + a * K, rows + a * K + K, rows + b * K);
    };
    int64_t kept = 0;
    for (int64_t g0 = 0; g0 < n;) {
      int64_t g1 = g0 + 1;
      while (g1 < n && same(order[g0], order[g1])) ++g1;
      int64_t n_att = 0, n_nor = 0;
      for (int64_t k = g0; k < g1; ++k) (labels[order[k]] ? n_att : n_nor)++;
      int64_t drop_att = 0, drop_nor = 0;
      if (mode == 0) {
        drop_att = drop_nor = std::min(n_att, n_nor);
      } else if (n_att > 0 && n_nor > 0) {
        drop_att = n_att;
        drop_nor = n_nor;
      }
      for (int64_t k = g0; k < g1; ++k) {
        const int64_t i = order[k];
        int64_t& left = labels[i] ? drop_att : drop_nor;
        if (left > 0) {
          --left;
          keep_out[i] = 0;
        } else {
          keep_out[i] = 1;
          ++kept;
        }
      }
      g0 = g1;
    }
    if (n_kept_out) *n_kept_out = kept;
    return IG_OK;
  });
}

extern "C" int ig_evaluate(const uint8_t* y_true, const uint8_t* y_pred, const int64_t* A,
                           const int64_t* N, int64_t m, ig_metrics_t* out) {
  return igk::guarded("ig_evaluate", [&]() -> int {
    if (m < 0 || !out || (m > 0 && (!y_true || !y_pred)) || ((A == nullptr) != (N == nullptr)))
      return fail(IG_E_INVAL, "ig_evaluate: bad arguments");
    if (m > kMaxEvalRows) return fail(IG_E_OVERFLOW, "ig_evaluate: more than 2^31 records");
    if (!labels_ok(y_true, m) || !labels_ok(y_pred, m))
      return fail(IG_E_INVAL, "ig_evaluate: label > 1");
    fill_counts(y_true, y_pred, m, out);
    out->auc = (A && m > 0) ? auc_of(y_true, A, N, m) : std::nan("");
    return IG_OK;
  });
}

extern "C" int ig_reg3_sweep(const int64_t* A, const int64_t* N, const uint8_t* y_true,
                             int64_t m, double mu, double sigma, const double* r, int32_t n_r,
                             ig_metrics_t* out) {
  return igk::guarded("ig_reg3_sweep", [&]() -> int {
    if (m < 0 || n_r < 0 || (n_r > 0 && (!r || !out)) || (m > 0 && (!A || !N || !y_true)))
      return fail(IG_E_INVAL, "ig_reg3_sweep: bad arguments");
    if (m > kMaxEvalRows) return fail(IG_E_OVERFLOW, "ig_reg3_sweep: more than 2^31 records");
    if (!labels_ok(y_true, m)) return fail(IG_E_INVAL, "ig_reg3_sweep: label > 1");
    const double auc = m > 0 ? auc_of(y_true, A, N, m) : std::nan("");
    std::vector<uint8_t> pred(static_cast<size_t>(m));
    for (int32_t k = 0; k < n_r; ++k) {
      const double scaled = r[k] * sigma;
      const double thr = mu - scaled;
      for (int64_t i = 0; i < m; ++i) {
        const bool r1 = A[i] >= N[i];
        const bool r2 = A[i] == 0 && N[i] == 0;
        const bool r3 = double(N[i]) < thr;
        pred[i] = uint8_t(r1 || r2 || r3);
      }
      fill_counts(y_true, pred.data(), m, out + k);
      out[k].auc = auc;
    }
    return IG_OK;
  });
}
