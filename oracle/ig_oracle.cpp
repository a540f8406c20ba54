// CPU oracle for Interpretable Generalization (IG).
//
// TEST INFRASTRUCTURE ONLY.  This file is the slow, plain, obviously-correct
// statement of what the IG hot path computes.  Only the test suite, the smoke
// check and the benchmark's CPU-baseline leg may build, load or call it; the
// product library never does, and the two share no code, header or table.
//
// Every function follows the paper's definitions literally:
//   * items and packing ............ Section 3.1 (tokens), Eq. 5 (packed words)
//   * candidates B^c ............... Eq. 1 (pairwise intersections i < j, plus
//                                     every record; the empty set is dropped)
//   * support and score S_c(b) ..... Eq. 2 (f_c(b) = number of class-c records
//                                     containing b; |b| = number of items in b)
//   * coherence P^c ................ Eq. 3, tested in the form of Eq. 6
//                                     ((p AND r) == p on every word)
//   * evidence A(x), N(x) .......... Eq. 4
//   * labels ....................... Regulations 1-3 (Section 3.1)
//
// Bit convention (Eq. 5): item j of a record is bit (j mod 64) of word
// (j div 64); K = ceil(L / 64).  Canonical order of a pattern list is
// ascending as a K-word unsigned integer whose most significant word is
// word K-1.
//
// Build: g++ -O2 -std=c++17 -pthread -ffp-contract=off -shared -fPIC
// (no SIMD intrinsics, no architecture flags).

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <thread>
#include <vector>

namespace {

// Number of items in a packed word, by clearing the lowest set bit until none
// is left.
int items_in_word(uint64_t w) {
  int c = 0;
  while (w != 0) {
    w &= w - 1;
    ++c;
  }
  return c;
}

int items_in_row(const uint64_t* b, int K) {
  int c = 0;
  for (int k = 0; k < K; ++k) c += items_in_word(b[k]);
  return c;
}

// Eq. 6 for one (pattern, record) pair: p is contained in r iff, on every
// word k, (p_k AND r_k) == p_k.
bool contained_in(const uint64_t* p, const uint64_t* r, int K) {
  for (int k = 0; k < K; ++k)
    if ((p[k] & r[k]) != p[k]) return false;
  return true;
}

bool is_empty(const uint64_t* b, int K) {
  for (int k = 0; k < K; ++k)
    if (b[k] != 0) return false;
  return true;
}

// Canonical order: compare as unsigned integers, word K-1 most significant.
bool less_than(const uint64_t* a, const uint64_t* b, int K) {
  for (int k = K - 1; k >= 0; --k) {
    if (a[k] != b[k]) return a[k] < b[k];
  }
  return false;
}

bool equal_rows(const uint64_t* a, const uint64_t* b, int K) {
  for (int k = 0; k < K; ++k)
    if (a[k] != b[k]) return false;
  return true;
}

// Runs body(lo, hi) over [0, n) split into contiguous chunks, one thread per
// chunk.  Every caller writes only the outputs of its own index range, so the
// result does not depend on the thread count.
template <class Body>
void parallel_ranges(int64_t n, int nthreads, Body body) {
  if (nthreads <= 1 || n < 2 * nthreads) {
    body(int64_t(0), n);
    return;
  }
  std::vector<std::thread> pool;
  int64_t chunk = (n + nthreads - 1) / nthreads;
  for (int t = 0; t < nthreads; ++t) {
    int64_t lo = t * chunk, hi = std::min<int64_t>(n, lo + chunk);
    if (lo >= hi) break;
    pool.emplace_back([=] { body(lo, hi); });
  }
  for (auto& th : pool) th.join();
}

struct RowList {
  int K = 0;
  std::vector<uint64_t> words;  // rows * K
  int64_t rows() const { return K ? int64_t(words.size()) / K : 0; }
};

}  // namespace

extern "C" {

// Section 3.1 and Eq. 5: the token (feature f, value v) is item
// offset_f + v, where offset_f is the sum of the cardinalities of the features
// before f; the code 0xFFFF marks a missing value (no token).  Returns 0, or
// -1 if a code is out of range or K is too small.
int oracle_encode(const uint16_t* codes, int64_t n, int32_t F,
                  const uint16_t* cards, int32_t K, uint64_t* out) {
  int64_t L = 0;
  for (int f = 0; f < F; ++f) L += cards[f];
  if (int64_t(K) * 64 < L) return -1;
  std::memset(out, 0, sizeof(uint64_t) * size_t(n) * size_t(K));
  for (int64_t i = 0; i < n; ++i) {
    int64_t offset = 0;
    for (int f = 0; f < F; ++f) {
      uint16_t v = codes[i * F + f];
      if (v == 0xFFFF) {  // missing value: the feature contributes no item
        offset += cards[f];
        continue;
      }
      if (v >= cards[f]) return -1;
      int64_t item = offset + v;
      out[i * K + item / 64] |= uint64_t(1) << (item % 64);
      offset += cards[f];
    }
  }
  return 0;
}

// Eq. 1: B^c = { x_i AND x_j : i < j } united with { x_i }, as a set (sorted,
// duplicates removed), without the empty itemset.
void* oracle_candidates(const uint64_t* rows, int64_t n, int32_t K) {
  RowList all;
  all.K = K;
  std::vector<uint64_t> b(K);
  auto push = [&](const uint64_t* v) {
    if (!is_empty(v, K)) all.words.insert(all.words.end(), v, v + K);
  };
  for (int64_t i = 0; i < n; ++i) {
    push(rows + i * K);
    for (int64_t j = i + 1; j < n; ++j) {
      for (int k = 0; k < K; ++k) b[k] = rows[i * K + k] & rows[j * K + k];
      push(b.data());
    }
  }
  int64_t m = all.rows();
  std::vector<int64_t> order(m);
  for (int64_t i = 0; i < m; ++i) order[i] = i;
  const uint64_t* w = all.words.data();
  std::sort(order.begin(), order.end(), [&](int64_t a, int64_t c) {
    return less_than(w + a * K, w + c * K, K);
  });
  RowList* out = new RowList;
  out->K = K;
  for (int64_t t = 0; t < m; ++t) {
    const uint64_t* v = w + order[t] * K;
    if (out->rows() > 0 &&
        equal_rows(out->words.data() + (out->rows() - 1) * K, v, K))
      continue;
    out->words.insert(out->words.end(), v, v + K);
  }
  return out;
}

int64_t oracle_list_rows(void* h) { return static_cast<RowList*>(h)->rows(); }

void oracle_list_copy(void* h, uint64_t* out) {
  RowList* r = static_cast<RowList*>(h);
  std::memcpy(out, r->words.data(), r->words.size() * sizeof(uint64_t));
}

void oracle_list_free(void* h) { delete static_cast<RowList*>(h); }

// Eq. 3 with the test of Eq. 6: candidate b is coherent iff no record x of
// the opposite class contains it.  out[u] = 1 for coherent candidates.
void oracle_coherent(const uint64_t* cand, int64_t U, const uint64_t* opp,
                     int64_t n_opp, int32_t K, uint8_t* out, int nthreads) {
  parallel_ranges(U, nthreads, [&](int64_t lo, int64_t hi) {
    for (int64_t u = lo; u < hi; ++u) {
      bool inside_some = false;
      for (int64_t t = 0; t < n_opp && !inside_some; ++t)
        inside_some = contained_in(cand + u * K, opp + t * K, K);
      out[u] = inside_some ? 0 : 1;
    }
  });
}

// Eq. 2: f_c(b) = number of class-c records (duplicates counted) that
// contain b, and S_c(b) = f_c(b) * |b|^2 with |b| the number of items of b.
void oracle_support(const uint64_t* pat, int64_t P, const uint64_t* same,
                    int64_t n_same, int32_t K, uint32_t* f, uint64_t* S,
                    int nthreads) {
  parallel_ranges(P, nthreads, [&](int64_t lo, int64_t hi) {
    for (int64_t p = lo; p < hi; ++p) {
      uint32_t count = 0;
      for (int64_t t = 0; t < n_same; ++t)
        if (contained_in(pat + p * K, same + t * K, K)) ++count;
      uint64_t size = uint64_t(items_in_row(pat + p * K, K));
      f[p] = count;
      S[p] = uint64_t(count) * size * size;
    }
  });
}

// Eq. 2 for given supports: S(b) = f(b) * |b|^2 (patterns learned elsewhere,
// e.g. a dictionary to be served).
void oracle_pattern_score(const uint64_t* pat, int64_t P, int32_t K, const uint32_t* f,
                          uint64_t* S) {
  for (int64_t p = 0; p < P; ++p) {
    uint64_t size = uint64_t(items_in_row(pat + p * K, K));
    S[p] = uint64_t(f[p]) * size * size;
  }
}

// Eq. 4: evidence(x) = sum over patterns b of S(b) * [b contained in x].
// Called once with P^+ (giving A) and once with P^- (giving N).
void oracle_evidence(const uint64_t* pat, const uint64_t* S, int64_t P,
                     const uint64_t* rows, int64_t m, int32_t K, int64_t* out,
                     int nthreads) {
  parallel_ranges(m, nthreads, [&](int64_t lo, int64_t hi) {
    for (int64_t t = lo; t < hi; ++t) {
      int64_t sum = 0;
      for (int64_t p = 0; p < P; ++p)
        if (contained_in(pat + p * K, rows + t * K, K)) sum += int64_t(S[p]);
      out[t] = sum;
    }
  });
}

// Regulation 3 statistics: mean and population standard deviation of the
// normal evidence N over the given records, accumulated in index order in
// double precision: mu = sum(N_i) / n; var = sum((N_i - mu)^2) / n.
void oracle_reg3_stats(const int64_t* N, int64_t n, double* mu,
                       double* sigma) {
  if (n <= 0) {
    *mu = 0.0;
    *sigma = 0.0;
    return;
  }
  double sum = 0.0;
  for (int64_t i = 0; i < n; ++i) sum += double(N[i]);
  double mean = sum / double(n);
  double ss = 0.0;
  for (int64_t i = 0; i < n; ++i) {
    double d = double(N[i]) - mean;
    ss += d * d;
  }
  *mu = mean;
  *sigma = std::sqrt(ss / double(n));
}

// Regulations 1-3, applied in the paper's order.  1 = attack, 0 = normal.
//   R1: attack iff A >= N.
//   R2: A == 0 and N == 0 overrides R1 with attack.
//   R3 (when enabled): N < mu_N - r * sigma_N gives attack even when R1 says
//       normal; otherwise the earlier label stands.  `threshold` is
//       mu_N - r * sigma_N, computed by the caller.
void oracle_labels(const int64_t* A, const int64_t* N, int64_t m, int reg3,
                   double threshold, uint8_t* out) {
  for (int64_t t = 0; t < m; ++t) {
    uint8_t label = (A[t] >= N[t]) ? 1 : 0;               // Regulation 1
    if (A[t] == 0 && N[t] == 0) label = 1;                 // Regulation 2
    if (reg3 && label == 0 && double(N[t]) < threshold)    // Regulation 3
      label = 1;
    out[t] = label;
  }
}

// Regulation 3 threshold mu - r * sigma, with no fused multiply-add (the
// file is compiled with -ffp-contract=off).
double oracle_reg3_threshold(double mu, double sigma, double r) {
  double scaled = r * sigma;
  return mu - scaled;
}

}  // extern "C"
