// CPU oracle for C = A*B on CSR inputs: TEST INFRASTRUCTURE ONLY.
//
// Only the tests, the smoke check and the bench's CPU-baseline leg may load this
// library. The product path never calls it; it shares no code, header or constant with
// the CUDA library.
//
// It is the row-by-row (Gustavson) formulation of the paper, Algorithm 1 (Sec. III-A),
// written out as its plain definition:
//   for each row i of A:
//     for each stored (k, a_ik) of row i, in stored order:        (the B rows named by A)
//       for each stored (j, b_kj) of row k of B, in stored order:
//         the partial product a_ik*b_kj is merged into the entry of column j
//   the row is emitted sorted by column, one entry for EVERY column that received a
//   partial product (structural: a sum that cancels to 0 is still emitted).
// The "sort then merge equal columns" of Algorithm 1 is realised by an ordered map keyed by
// column, which holds the partial products of one row already merged, or (the default for the
// stored-order sums) by a dense accumulator per thread: one slot per column of C, the columns a
// row touched listed as they are first hit and sorted at the end (Gustavson's own sparse
// accumulator). Both add each entry's products in the same stored order, so their values are
// bit-identical; the tests compare them.
//
// Arithmetic: FP64, each product rounded once (the build passes -ffp-contract=off so no
// multiply-add is fused), summed in stored order. A second variant (exact_sum) returns for each
// entry the sum of its rounded products rounded once to FP64 (round to nearest, ties to even):
// the exact sum of the same partial products, with no rounding in between. It keeps each
// entry's running sum as a list of non-overlapping partial sums (Shewchuk, "Adaptive precision
// floating-point arithmetic and fast robust geometric predicates", 1997: TwoSum growth of an
// expansion) and rounds it once at the end, from the largest partial down, with the half-way
// correction that makes the result correctly rounded. An entry with a non-finite product takes
// the stored-order sum. Beside each value it returns
// mag = sum of |a_ik*b_kj| (the scale of the entry's rounding error) and the number of
// terms that entry received. Inputs in FP32 are widened to FP64 by the caller; that is
// exact, and so is every FP32*FP32 product in FP64.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <map>
#include <memory>
#include <thread>
#include <vector>

namespace {

struct Entry {
  double sum = 0.0;
  double mag = 0.0;
  int32_t terms = 0;
};

struct RowOut {
  std::vector<int32_t> col;
  std::vector<double> val;
  std::vector<double> mag;
  std::vector<int32_t> terms;
};

}  // namespace

struct OracleResult {
  std::vector<RowOut> rows;
  int64_t nnz = 0;
  int threads = 0;
};

// Exact sum of one entry: partials[] hold non-overlapping FP64 values whose exact sum is the
// exact sum of the terms added so far (each TwoSum below is error-free).
struct ExactEntry {
  std::vector<double> partials;
  double plain = 0.0;   // stored-order sum (for non-finite terms)
  double mag = 0.0;
  int32_t terms = 0;
  bool finite = true;

  void add(double x) {
    plain = plain + x;
    if (!std::isfinite(x)) finite = false;
    if (!finite) return;
    size_t n = 0;
    for (size_t q = 0; q < partials.size(); ++q) {
      double y = partials[q];
      if (std::fabs(x) < std::fabs(y)) std::swap(x, y);
      const double hi = x + y;          // |x| >= |y|: hi + lo == x + y exactly
      const double lo = y - (hi - x);
      if (lo != 0.0) partials[n++] = lo;
      x = hi;
    }
    partials.resize(n);
    partials.push_back(x);
  }

  // The exact sum of the partials rounded once to FP64 (nearest, ties to even).
  double rounded() const {
    if (!finite) return plain;
    size_t n = partials.size();
    if (n == 0) return 0.0;
    double hi = partials[--n];
    double lo = 0.0;
    while (n > 0) {   // add partials from the top while the sum stays exact
      const double x = hi;
      const double y = partials[--n];
      hi = x + y;
      lo = y - (hi - x);
      if (lo != 0.0) break;
    }
    // hi is the sum rounded to nearest unless lo is exactly half an ulp of hi and the partials
    // below push the true sum past the half-way point (same sign as lo): then round away
    if (n > 0 && ((lo < 0.0 && partials[n - 1] < 0.0) || (lo > 0.0 && partials[n - 1] > 0.0))) {
      const double y = lo * 2.0;
      const double x = hi + y;
      if (y == x - hi) hi = x;
    }
    return hi;
  }
};

static void oracle_row_exact(int64_t i, const int64_t* a_rp, const int32_t* a_col, const double* a_val,
                             const int64_t* b_rp, const int32_t* b_col, const double* b_val, RowOut& out) {
  std::map<int32_t, ExactEntry> acc;
  for (int64_t p = a_rp[i]; p < a_rp[i + 1]; ++p) {
    const int32_t k = a_col[p];
    const double a = a_val ? a_val[p] : 1.0;
    for (int64_t q = b_rp[k]; q < b_rp[k + 1]; ++q) {
      const double prod = a * (b_val ? b_val[q] : 1.0);
      ExactEntry& e = acc[b_col[q]];
      e.add(prod);
      e.mag = e.mag + std::fabs(prod);
      e.terms += 1;
    }
  }
  for (const auto& kv : acc) {
    out.col.push_back(kv.first);
    out.val.push_back(kv.second.rounded());
    out.mag.push_back(kv.second.mag);
    out.terms.push_back(kv.second.terms);
  }
}

static void oracle_row(int64_t i, const int64_t* a_rp, const int32_t* a_col, const double* a_val,
                       const int64_t* b_rp, const int32_t* b_col, const double* b_val,
                       RowOut& out) {
  std::map<int32_t, Entry> acc;
  for (int64_t p = a_rp[i]; p < a_rp[i + 1]; ++p) {
    const int32_t k = a_col[p];
    const double a = a_val ? a_val[p] : 1.0;
    for (int64_t q = b_rp[k]; q < b_rp[k + 1]; ++q) {
      const double prod = a * (b_val ? b_val[q] : 1.0);
      Entry& e = acc[b_col[q]];
      e.sum = e.sum + prod;
      e.mag = e.mag + std::fabs(prod);
      e.terms += 1;
    }
  }
  out.col.reserve(acc.size());
  out.val.reserve(acc.size());
  out.mag.reserve(acc.size());
  out.terms.reserve(acc.size());
  for (const auto& kv : acc) {
    out.col.push_back(kv.first);
    out.val.push_back(kv.second.sum);
    out.mag.push_back(kv.second.mag);
    out.terms.push_back(kv.second.terms);
  }
}

// Dense accumulator of one thread: slots for every column of C, reset after each row.
struct DenseAcc {
  std::vector<double> sum, mag;
  std::vector<int32_t> terms;
  std::vector<int32_t> touched;
  explicit DenseAcc(int64_t n) : sum(n, 0.0), mag(n, 0.0), terms(n, 0) {}
};

static void oracle_row_dense(int64_t i, const int64_t* a_rp, const int32_t* a_col, const double* a_val,
                             const int64_t* b_rp, const int32_t* b_col, const double* b_val, DenseAcc& d,
                             RowOut& out) {
  d.touched.clear();
  for (int64_t p = a_rp[i]; p < a_rp[i + 1]; ++p) {
    const int32_t k = a_col[p];
    const double a = a_val ? a_val[p] : 1.0;
    for (int64_t q = b_rp[k]; q < b_rp[k + 1]; ++q) {
      const double prod = a * (b_val ? b_val[q] : 1.0);
      const int32_t j = b_col[q];
      if (d.terms[j] == 0) d.touched.push_back(j);
      d.sum[j] = d.sum[j] + prod;
      d.mag[j] = d.mag[j] + std::fabs(prod);
      d.terms[j] += 1;
    }
  }
  std::sort(d.touched.begin(), d.touched.end());
  const size_t len = d.touched.size();
  out.col.resize(len);
  out.val.resize(len);
  out.mag.resize(len);
  out.terms.resize(len);
  for (size_t t = 0; t < len; ++t) {
    const int32_t j = d.touched[t];
    out.col[t] = j;
    out.val[t] = d.sum[j];
    out.mag[t] = d.mag[j];
    out.terms[t] = d.terms[j];
    d.sum[j] = 0.0;
    d.mag[j] = 0.0;
    d.terms[j] = 0;
  }
}

extern "C" {

// Computes rows `rows[0..nrows)` of C = A*B (all m rows when rows == NULL).
// a_val / b_val may be NULL (pattern only: every stored value taken as 1).
// threads <= 0 uses std::thread::hardware_concurrency().
// exact_sum != 0: every value is the correctly rounded sum of the entry's partial products.
// method: 0 ordered map, 1 dense accumulator of n_cols slots per thread (stored-order sums only).
OracleResult* oracle_spgemm_ex(int64_t m, const int64_t* a_rp, const int32_t* a_col,
                               const double* a_val, const int64_t* b_rp, const int32_t* b_col,
                               const double* b_val, const int64_t* rows, int64_t nrows,
                               int threads, int exact_sum, int method, int64_t n_cols) {
  OracleResult* r = new OracleResult();
  const int64_t count = rows ? nrows : m;
  r->rows.resize(static_cast<size_t>(count));
  int nt = threads > 0 ? threads : static_cast<int>(std::thread::hardware_concurrency());
  if (nt < 1) nt = 1;
  if (count < 256) nt = 1;
  r->threads = nt;
  std::atomic<int64_t> next(0);
  const int64_t chunk = 64;
  const bool dense = !exact_sum && method == 1 && n_cols > 0;
  auto work = [&]() {
    std::unique_ptr<DenseAcc> d;
    if (dense) d.reset(new DenseAcc(n_cols));
    for (;;) {
      const int64_t s = next.fetch_add(chunk);
      if (s >= count) break;
      const int64_t e = s + chunk < count ? s + chunk : count;
      for (int64_t t = s; t < e; ++t) {
        const int64_t i = rows ? rows[t] : t;
        if (exact_sum) oracle_row_exact(i, a_rp, a_col, a_val, b_rp, b_col, b_val, r->rows[t]);
        else if (dense) oracle_row_dense(i, a_rp, a_col, a_val, b_rp, b_col, b_val, *d, r->rows[t]);
        else oracle_row(i, a_rp, a_col, a_val, b_rp, b_col, b_val, r->rows[t]);
      }
    }
  };
  if (nt == 1) {
    work();
  } else {
    std::vector<std::thread> pool;
    for (int t = 0; t < nt; ++t) pool.emplace_back(work);
    for (auto& th : pool) th.join();
  }
  int64_t nnz = 0;
  for (const auto& ro : r->rows) nnz += static_cast<int64_t>(ro.col.size());
  r->nnz = nnz;
  return r;
}

OracleResult* oracle_spgemm(int64_t m, const int64_t* a_rp, const int32_t* a_col,
                            const double* a_val, const int64_t* b_rp, const int32_t* b_col,
                            const double* b_val, const int64_t* rows, int64_t nrows,
                            int threads) {
  return oracle_spgemm_ex(m, a_rp, a_col, a_val, b_rp, b_col, b_val, rows, nrows, threads, 0, 0, 0);
}

int64_t oracle_nnz(const OracleResult* r) { return r->nnz; }

int oracle_threads(const OracleResult* r) { return r->threads; }

// rp has nrows+1 entries; col/val/mag/terms have oracle_nnz entries. Any output may be NULL.
void oracle_copy(const OracleResult* r, int64_t* rp, int32_t* col, double* val, double* mag,
                 int32_t* terms) {
  int64_t off = 0;
  if (rp) rp[0] = 0;
  for (size_t t = 0; t < r->rows.size(); ++t) {
    const RowOut& ro = r->rows[t];
    const size_t len = ro.col.size();
    if (len) {
      if (col) std::memcpy(col + off, ro.col.data(), len * sizeof(int32_t));
      if (val) std::memcpy(val + off, ro.val.data(), len * sizeof(double));
      if (mag) std::memcpy(mag + off, ro.mag.data(), len * sizeof(double));
      if (terms) std::memcpy(terms + off, ro.terms.data(), len * sizeof(int32_t));
    }
    off += static_cast<int64_t>(len);
    if (rp) rp[t + 1] = off;
  }
}

void oracle_free(OracleResult* r) { delete r; }

}  // extern "C"
