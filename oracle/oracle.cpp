/*
 * oracle.cpp -- plain, slow, obviously correct CPU implementation of the
 * relational hot path (filter, radix hash partition, hash-join build/probe,
 * exact group-by SUM, top-k, and the three-table filter/join/group-by/top-k
 * plan).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path may link, load or
 * call this file: only the tests, the smoke check and the benchmark's CPU
 * baseline use it.  It shares no code, header, table or constant generator
 * with the CUDA library; the two meet only at the raw input arrays.
 *
 * Every routine is the plain definition of the operation written out with
 * standard containers (std::vector, std::unordered_multimap, std::map,
 * std::sort), single-threaded, with int64 results accumulated in __int128 so
 * that an int64 overflow is detected instead of wrapping.
 *
 * Operation codes are plain integers (fixed by the C ABI's documentation):
 *   dtype: 1 = int8, 2 = int32, 3 = int64
 *   compare: 0 '<', 1 '<=', 2 '>', 3 '>=', 4 '==', 5 '!=', 6 always true
 * Status: 0 ok, 1 invalid argument, 7 int64 overflow.
 */
#include <algorithm>
#include <cstdint>
#include <cstring>
#include <map>
#include <unordered_map>
#include <unordered_set>
#include <utility>
#include <vector>

namespace {

int64_t load(const void* col, int type, int64_t i) {
  switch (type) {
    case 1: return static_cast<const int8_t*>(col)[i];
    case 2: return static_cast<const int32_t*>(col)[i];
    case 3: return static_cast<const int64_t*>(col)[i];
  }
  return 0;
}

void store(void* col, int type, int64_t i, int64_t v) {
  switch (type) {
    case 1: static_cast<int8_t*>(col)[i] = static_cast<int8_t>(v); break;
    case 2: static_cast<int32_t*>(col)[i] = static_cast<int32_t>(v); break;
    case 3: static_cast<int64_t*>(col)[i] = v; break;
  }
}

/* A predicate "column op constant" as written in a WHERE clause (the scan's
 * pushed-down filter, Sec. 4 and Sec. 6.1). */
bool pred(int op, int64_t v, int64_t c) {
  switch (op) {
    case 0: return v < c;
    case 1: return v <= c;
    case 2: return v > c;
    case 3: return v >= c;
    case 4: return v == c;
    case 5: return v != c;
    case 6: return true;
  }
  return false;
}

bool fits_int64(__int128 x) {
  return x >= static_cast<__int128>(INT64_MIN) && x <= static_cast<__int128>(INT64_MAX);
}

/* Radix bucket of a key: Fibonacci (multiplicative) hashing, Knuth TAOCP
 * vol. 3, Sec. 6.4 -- multiply the key, read as an unsigned 64-bit word, by
 * floor(2^64 / golden ratio) modulo 2^64 and keep the top log2P bits.  This
 * replaces the paper's "key modulo number of nodes" split (Sec. 3.1) by a
 * hash that also spreads clustered keys. */
uint64_t bucket_of(int64_t key, int log2P) {
  if (log2P == 0) return 0;
  const uint64_t golden = 11400714819323198485ULL;
  uint64_t h = static_cast<uint64_t>(key) * golden;
  return h >> (64 - log2P);
}

bool before(int64_t ka, int64_t sa, int64_t kb, int64_t sb) {
  /* Top-k order: larger sum first, ties broken by smaller key. */
  if (sa != sb) return sa > sb;
  return ka < kb;
}

}  // namespace

extern "C" {

/* Selection (filter pushdown into the scan, Sec. 4 / Sec. 6.1): the row ids
 * whose value satisfies the predicate, in ascending row order.  With a
 * selection vector, only its rows are tested (AND with the previous filter). */
int64_t oracle_filter(const void* col, int type, int64_t n, int op, int64_t c,
                      const int64_t* sel_in, int64_t n_in, int64_t* sel_out) {
  int64_t cnt = 0;
  if (sel_in == nullptr) {
    for (int64_t i = 0; i < n; ++i)
      if (pred(op, load(col, type, i), c)) sel_out[cnt++] = i;
  } else {
    for (int64_t j = 0; j < n_in; ++j) {
      int64_t r = sel_in[j];
      if (pred(op, load(col, type, r), c)) sel_out[cnt++] = r;
    }
  }
  return cnt;
}

/* Partitioning by join key ahead of the exchange (Sec. 3.1): rows grouped
 * into P = 2^log2P buckets, bucket b holding the rows with bucket_of(key) = b
 * in their input order (a stable counting sort).  offsets[b] .. offsets[b+1]
 * delimit bucket b. */
int oracle_partition(const void* key, int ktype, int64_t n, int log2P, int npay,
                     const void* const* pay, const int* ptypes, void* out_key,
                     void* const* out_pay, int64_t* offsets) {
  if (log2P < 0 || log2P > 16) return 1;
  const int64_t P = int64_t{1} << log2P;
  std::vector<int64_t> count(P, 0);
  for (int64_t i = 0; i < n; ++i) count[bucket_of(load(key, ktype, i), log2P)]++;
  offsets[0] = 0;
  for (int64_t b = 0; b < P; ++b) offsets[b + 1] = offsets[b] + count[b];
  std::vector<int64_t> cursor(offsets, offsets + P);
  for (int64_t i = 0; i < n; ++i) {
    int64_t k = load(key, ktype, i);
    int64_t pos = cursor[bucket_of(k, log2P)]++;
    store(out_key, ktype, pos, k);
    for (int j = 0; j < npay; ++j) store(out_pay[j], ptypes[j], pos, load(pay[j], ptypes[j], i));
  }
  return 0;
}

/* Equi-join (hash-table build on the left side, probe with the right side,
 * Sec. 3.1): every pair (probe row i, build value v) with probe[i] == build
 * key of the row holding v.  A null build value column means "build row id".
 * Output sorted by (probe row, build value); returns the full pair count and
 * writes at most cap pairs. */
int64_t oracle_join(const void* bkey, int bktype, const int64_t* bval, int64_t nb,
                    const void* pkey, int pktype, int64_t np, int64_t* out_probe_row,
                    int64_t* out_build_val, int64_t cap) {
  std::unordered_multimap<int64_t, int64_t> table;
  table.reserve(static_cast<size_t>(nb));
  for (int64_t j = 0; j < nb; ++j) table.emplace(load(bkey, bktype, j), bval ? bval[j] : j);
  std::vector<std::pair<int64_t, int64_t>> pairs;
  for (int64_t i = 0; i < np; ++i) {
    auto range = table.equal_range(load(pkey, pktype, i));
    for (auto it = range.first; it != range.second; ++it) pairs.emplace_back(i, it->second);
  }
  std::sort(pairs.begin(), pairs.end());
  int64_t total = static_cast<int64_t>(pairs.size());
  for (int64_t t = 0; t < total && t < cap; ++t) {
    out_probe_row[t] = pairs[t].first;
    out_build_val[t] = pairs[t].second;
  }
  return total;
}

/* Group-by aggregation (Sec. 3.2, Sec. 6.3): one output row per distinct key
 * with the exact SUM of its values, sorted by key.  Returns the number of
 * groups (writes at most cap); *overflow = 1 if any sum leaves int64. */
int64_t oracle_groupby_sum(const void* key, int ktype, const int64_t* val, int64_t n,
                           int64_t* out_keys, int64_t* out_sums, int64_t cap, int* overflow) {
  std::map<int64_t, __int128> groups;
  for (int64_t i = 0; i < n; ++i) groups[load(key, ktype, i)] += val[i];
  int ovf = 0;
  int64_t g = 0;
  for (const auto& kv : groups) {
    if (!fits_int64(kv.second)) ovf = 1;
    if (g < cap) {
      out_keys[g] = kv.first;
      out_sums[g] = static_cast<int64_t>(kv.second);
    }
    ++g;
  }
  if (overflow) *overflow = ovf;
  return g;
}

/* ORDER BY sum DESC, key ASC LIMIT k: a full sort, then the first
 * min(k, n) rows. */
int64_t oracle_topk(const int64_t* keys, const int64_t* sums, int64_t n, int k,
                    int64_t* out_keys, int64_t* out_sums) {
  std::vector<int64_t> idx(static_cast<size_t>(n));
  for (int64_t i = 0; i < n; ++i) idx[i] = i;
  std::sort(idx.begin(), idx.end(), [&](int64_t a, int64_t b) {
    return before(keys[a], sums[a], keys[b], sums[b]);
  });
  int64_t m = std::min<int64_t>(k, n);
  for (int64_t t = 0; t < m; ++t) {
    out_keys[t] = keys[idx[t]];
    out_sums[t] = sums[idx[t]];
  }
  return m;
}

/* The three-table plan (the paper's running example shape, Sec. 5.1):
 *   D' = { d.key : d.seg op_d c_d }
 *   M' = { m : m.date op_m c_m and m.dref in D' }
 *   for every pair (f, m) with f.date2 op_f c_f, m in M', f.mkey = m.key:
 *       sum[m.key] += f.price * (100 - f.disc)
 *   groups = M keys with at least one such pair.
 * Returns the groups as an ordered map key -> exact (__int128) sum. */
static std::map<int64_t, __int128> plan_groups(
    const int32_t* d_key, const int8_t* d_seg, int64_t n_d, const int64_t* m_key,
    const int32_t* m_dref, const int32_t* m_date, int64_t n_m, const int64_t* f_mkey,
    const int64_t* f_price, const int8_t* f_disc, const int32_t* f_date2, int64_t n_f, int d_op,
    int64_t d_c, int m_op, int64_t m_c, int f_op, int64_t f_c) {
  std::unordered_set<int64_t> d_pass;
  for (int64_t i = 0; i < n_d; ++i)
    if (pred(d_op, d_seg[i], d_c)) d_pass.insert(d_key[i]);

  std::unordered_multimap<int64_t, int64_t> m_pass;  // M.key -> M row
  for (int64_t i = 0; i < n_m; ++i) {
    const int64_t ref = m_dref[i];
    if (pred(m_op, m_date[i], m_c) && d_pass.count(ref)) m_pass.emplace(m_key[i], i);
  }

  std::map<int64_t, __int128> sums;
  for (int64_t i = 0; i < n_f; ++i) {
    if (!pred(f_op, f_date2[i], f_c)) continue;
    auto range = m_pass.equal_range(f_mkey[i]);
    for (auto it = range.first; it != range.second; ++it) {
      const __int128 revenue = static_cast<__int128>(f_price[i]) * (100 - f_disc[i]);
      sums[it->first] += revenue;
    }
  }
  return sums;
}

/* The plan's result: top-k of (key, sum) by sum desc, key asc, plus the
 * number of groups.  Returns 0, or 7 if a group sum leaves int64. */
int oracle_run_plan(const int32_t* d_key, const int8_t* d_seg, int64_t n_d,
                    const int64_t* m_key, const int32_t* m_dref, const int32_t* m_date,
                    int64_t n_m, const int64_t* f_mkey, const int64_t* f_price,
                    const int8_t* f_disc, const int32_t* f_date2, int64_t n_f, int d_op,
                    int64_t d_c, int m_op, int64_t m_c, int f_op, int64_t f_c, int k,
                    int64_t* out_keys, int64_t* out_sums, int64_t* n_out, int64_t* ngroups) {
  auto sums = plan_groups(d_key, d_seg, n_d, m_key, m_dref, m_date, n_m, f_mkey, f_price, f_disc,
                          f_date2, n_f, d_op, d_c, m_op, m_c, f_op, f_c);
  std::vector<int64_t> keys, vals;
  keys.reserve(sums.size());
  vals.reserve(sums.size());
  int status = 0;
  for (const auto& kv : sums) {
    if (!fits_int64(kv.second)) status = 7;
    keys.push_back(kv.first);
    vals.push_back(static_cast<int64_t>(kv.second));
  }
  *ngroups = static_cast<int64_t>(keys.size());
  *n_out = oracle_topk(keys.data(), vals.data(), static_cast<int64_t>(keys.size()), k, out_keys,
                       out_sums);
  return status;
}

/* The aggregate-first plan (a large materialised group-by filtered on its
 * aggregate, the shape of the paper's Q18 remark, Sec. 6.3):
 *   G  = for the F rows with f.date2 op_f c_f, grouped by f.mkey:
 *        sum = sum of f.price * (100 - f.disc)      (every group, materialised)
 *   M' = { m.key : m.date op_m c_m and m.dref in D' },  D' as above
 *   result = the groups with sum > having and key in M' (a semi-join: a key
 *            held by several M' rows counts once), top-k by sum desc, key asc,
 *            and their number.
 * Returns 0, or 7 if a group sum leaves int64. */
int oracle_run_plan_aggfirst(const int32_t* d_key, const int8_t* d_seg, int64_t n_d,
                             const int64_t* m_key, const int32_t* m_dref, const int32_t* m_date,
                             int64_t n_m, const int64_t* f_mkey, const int64_t* f_price,
                             const int8_t* f_disc, const int32_t* f_date2, int64_t n_f, int d_op,
                             int64_t d_c, int m_op, int64_t m_c, int f_op, int64_t f_c,
                             int64_t having, int k, int64_t* out_keys, int64_t* out_sums,
                             int64_t* n_out, int64_t* ngroups) {
  std::unordered_set<int64_t> d_pass;
  for (int64_t i = 0; i < n_d; ++i)
    if (pred(d_op, d_seg[i], d_c)) d_pass.insert(d_key[i]);
  std::unordered_map<int64_t, int64_t> m_keys;  // key -> M' rows holding it
  for (int64_t i = 0; i < n_m; ++i)
    if (pred(m_op, m_date[i], m_c) && d_pass.count(m_dref[i])) ++m_keys[m_key[i]];
  std::map<int64_t, __int128> g;
  for (int64_t i = 0; i < n_f; ++i)
    if (pred(f_op, f_date2[i], f_c))
      g[f_mkey[i]] += static_cast<__int128>(f_price[i]) * (100 - f_disc[i]);
  std::vector<int64_t> keys, vals;
  int status = 0;
  for (const auto& kv : g) {
    if (!fits_int64(kv.second)) status = 7;
    const auto m = m_keys.find(kv.first);
    const __int128 sum = kv.second;
    if (sum > having && m != m_keys.end()) {
      keys.push_back(kv.first);
      vals.push_back(static_cast<int64_t>(sum));
    }
  }
  *ngroups = static_cast<int64_t>(keys.size());
  *n_out = oracle_topk(keys.data(), vals.data(), static_cast<int64_t>(keys.size()), k, out_keys,
                       out_sums);
  return status;
}

/* Every group of the plan (key, sum) sorted by key.  Returns the group
 * count; writes at most cap rows. */
int64_t oracle_plan_groups(const int32_t* d_key, const int8_t* d_seg, int64_t n_d,
                           const int64_t* m_key, const int32_t* m_dref, const int32_t* m_date,
                           int64_t n_m, const int64_t* f_mkey, const int64_t* f_price,
                           const int8_t* f_disc, const int32_t* f_date2, int64_t n_f, int d_op,
                           int64_t d_c, int m_op, int64_t m_c, int f_op, int64_t f_c,
                           int64_t* out_keys, int64_t* out_sums, int64_t cap) {
  auto sums = plan_groups(d_key, d_seg, n_d, m_key, m_dref, m_date, n_m, f_mkey, f_price, f_disc,
                          f_date2, n_f, d_op, d_c, m_op, m_c, f_op, f_c);
  int64_t g = 0;
  for (const auto& kv : sums) {
    if (g < cap) {
      out_keys[g] = kv.first;
      out_sums[g] = static_cast<int64_t>(kv.second);
    }
    ++g;
  }
  return g;
}

}  // extern "C"
