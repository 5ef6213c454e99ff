// CPU oracle for the join and grouped-aggregation operators.
//
// TEST INFRASTRUCTURE ONLY. This file is the plain, slow, obviously correct
// statement of what the operators compute; only the test suite, the smoke check
// and the benchmark's CPU-baseline leg may load it. It shares no code with the
// CUDA library: no headers, no helpers, no constants.
//
// Every value is widened to int64 by the caller; every aggregate is int64.
// SUM accumulates in uint64 with two's-complement wrap-around, which is exact
// and independent of the order of additions.
//
// Definitions followed (paper: "Efficiently Processing Joins and Grouped
// Aggregations on GPUs"):
//   * inner equi-join T(key, r1.., s1..) of R(key, r1..) and S(key, s1..) -- Sec. 2.2
//   * group-by R(k, r1..rn) -> A(k, a1..an) with reducible aggregates -- Sec. 2.2, Alg. 1
//   * radix-partition(kin, vin, kout, vout, i, j): stable, partitions stored
//     contiguously, on bits [i, j) of the key -- Sec. 2.3
#include <algorithm>
#include <cstdint>
#include <cstring>
#include <numeric>
#include <unordered_map>
#include <vector>

namespace {

enum { AGG_SUM = 0, AGG_COUNT = 1, AGG_MIN = 2, AGG_MAX = 3 };


int64_t agg_init(int op) {
  switch (op) {
    case AGG_MIN: return INT64_MAX;
    case AGG_MAX: return INT64_MIN;
    default: return 0;
  }
}

int64_t agg_update(int op, int64_t acc, int64_t x) {
  switch (op) {
    case AGG_SUM: return (int64_t)((uint64_t)acc + (uint64_t)x);
    case AGG_COUNT: return acc + 1;
    case AGG_MIN: return x < acc ? x : acc;
    case AGG_MAX: return x > acc ? x : acc;
  }
  return acc;
}

// MurmurHash3 fmix32 / fmix64 finalizers (Appleby, public domain): bijections
// used as the "hashed key" digit source of radix-partition.
uint32_t fmix32(uint32_t h) {
  h ^= h >> 16; h *= 0x85ebca6bu; h ^= h >> 13; h *= 0xc2b2ae35u; h ^= h >> 16;
  return h;
}
uint64_t fmix64(uint64_t k) {
  k ^= k >> 33; k *= 0xff51afd7ed558ccdull; k ^= k >> 33; k *= 0xc4ceb9fe1a85ec53ull; k ^= k >> 33;
  return k;
}

}  // namespace

extern "C" {

// ---------------------------------------------------------------- join
// T = multiset { (r.key, r.cols.., s.cols..) : r in R, s in S, r.key = s.key }.
// Rows are emitted scanning S in order, and for each S row the matching R rows
// in R order. Output is row-major, (1 + ncr + ncs) int64 per row. Returns the
// number of result rows (which may exceed cap; only cap rows are written).
int64_t oracle_join(const int64_t* rkey, const int64_t* const* rcols, int64_t nr, int32_t ncr,
                    const int64_t* skey, const int64_t* const* scols, int64_t ns, int32_t ncs,
                    int64_t* out, int64_t cap) {
  std::unordered_map<int64_t, std::vector<int64_t>> build;
  build.reserve((size_t)nr * 2 + 1);
  for (int64_t i = 0; i < nr; ++i) build[rkey[i]].push_back(i);
  const int64_t w = 1 + ncr + ncs;
  int64_t m = 0;
  for (int64_t j = 0; j < ns; ++j) {
    auto it = build.find(skey[j]);
    if (it == build.end()) continue;
    for (int64_t i : it->second) {
      if (m < cap) {
        int64_t* row = out + m * w;
        row[0] = rkey[i];
        for (int c = 0; c < ncr; ++c) row[1 + c] = rcols[c][i];
        for (int c = 0; c < ncs; ++c) row[1 + ncr + c] = scols[c][j];
      }
      ++m;
    }
  }
  return m;
}

// ---------------------------------------------------------------- group-by
// For each distinct key k: a_j = f_j over { col[op_col[j]][i] : key[i] = k }
// (COUNT ignores its column). Output row-major, (1 + nagg) int64 per group.
// Two independent implementations: a hash map in first-occurrence order, and a
// sort by key followed by a scan of equal-key runs (ascending key order).
int64_t oracle_groupby_hash(const int64_t* key, const int64_t* const* cols, int64_t n, int32_t nagg,
                            const int32_t* ops, const int32_t* op_col, int64_t* out, int64_t cap) {
  std::unordered_map<int64_t, int64_t> slot;
  slot.reserve((size_t)n * 2 + 1);
  std::vector<int64_t> keys;
  std::vector<int64_t> acc;
  for (int64_t i = 0; i < n; ++i) {
    auto ins = slot.emplace(key[i], (int64_t)keys.size());
    int64_t s = ins.first->second;
    if (ins.second) {
      keys.push_back(key[i]);
      for (int j = 0; j < nagg; ++j) acc.push_back(agg_init(ops[j]));
    }
    for (int j = 0; j < nagg; ++j) {
      int64_t x = ops[j] == AGG_COUNT ? 0 : cols[op_col[j]][i];
      acc[s * nagg + j] = agg_update(ops[j], acc[s * nagg + j], x);
    }
  }
  const int64_t g = (int64_t)keys.size();
  for (int64_t s = 0; s < g && s < cap; ++s) {
    out[s * (1 + nagg)] = keys[s];
    for (int j = 0; j < nagg; ++j) out[s * (1 + nagg) + 1 + j] = acc[s * nagg + j];
  }
  return g;
}

int64_t oracle_groupby_sort(const int64_t* key, const int64_t* const* cols, int64_t n, int32_t nagg,
                            const int32_t* ops, const int32_t* op_col, int64_t* out, int64_t cap) {
  std::vector<int64_t> idx(n);
  std::iota(idx.begin(), idx.end(), 0);
  std::stable_sort(idx.begin(), idx.end(), [&](int64_t a, int64_t b) { return key[a] < key[b]; });
  int64_t g = 0;
  int64_t i = 0;
  std::vector<int64_t> acc(nagg);
  while (i < n) {
    int64_t k = key[idx[i]];
    for (int j = 0; j < nagg; ++j) acc[j] = agg_init(ops[j]);
    while (i < n && key[idx[i]] == k) {
      for (int j = 0; j < nagg; ++j) {
        int64_t x = ops[j] == AGG_COUNT ? 0 : cols[op_col[j]][idx[i]];
        acc[j] = agg_update(ops[j], acc[j], x);
      }
      ++i;
    }
    if (g < cap) {
      out[g * (1 + nagg)] = k;
      for (int j = 0; j < nagg; ++j) out[g * (1 + nagg) + 1 + j] = acc[j];
    }
    ++g;
  }
  return g;
}

// ---------------------------------------------------------------- join -> group-by
// GROUP BY gk over the join result, where gk is the join key (g_col < 0) or
// column g_col of side g_side (0 = R, 1 = S), reduced by C '%' when g_mod > 0.
// Aggregate j reads column agg_col[j] of side agg_side[j]. The join is
// computed first, exactly as oracle_join defines it; nothing is fused.
int64_t oracle_join_groupby(const int64_t* rkey, const int64_t* const* rcols, int64_t nr, int32_t ncr,
                            const int64_t* skey, const int64_t* const* scols, int64_t ns, int32_t ncs,
                            int32_t g_side, int32_t g_col, int64_t g_mod, int32_t nagg, const int32_t* ops,
                            const int32_t* agg_side, const int32_t* agg_col, int64_t* out, int64_t cap) {
  int64_t m = oracle_join(rkey, rcols, nr, ncr, skey, scols, ns, ncs, nullptr, 0);
  const int64_t w = 1 + ncr + ncs;
  std::vector<int64_t> t((size_t)(m * w));
  oracle_join(rkey, rcols, nr, ncr, skey, scols, ns, ncs, t.data(), m);
  std::vector<int64_t> gk(m);
  for (int64_t i = 0; i < m; ++i) {
    const int64_t* row = t.data() + i * w;
    int64_t v = g_col < 0 ? row[0] : (g_side == 0 ? row[1 + g_col] : row[1 + ncr + g_col]);
    gk[i] = g_mod > 0 ? v % g_mod : v;
  }
  std::vector<std::vector<int64_t>> acols(nagg, std::vector<int64_t>(m));
  std::vector<const int64_t*> cp(nagg);
  std::vector<int32_t> oc(nagg);
  for (int j = 0; j < nagg; ++j) {
    for (int64_t i = 0; i < m; ++i) {
      const int64_t* row = t.data() + i * w;
      acols[j][i] = ops[j] == AGG_COUNT ? 0 : (agg_side[j] == 0 ? row[1 + agg_col[j]] : row[1 + ncr + agg_col[j]]);
    }
    cp[j] = acols[j].data();
    oc[j] = j;
  }
  return oracle_groupby_hash(gk.data(), cp.data(), m, nagg, ops, oc.data(), out, cap);
}

// ---------------------------------------------------------------- radix-partition
// Digit of row i = bits [lo, hi) of d(key[i]) where d is the key's own binary
// representation (transform 0, unsigned, key_bytes wide), the key with its sign
// bit flipped (transform 1, ascending signed order), or the fmix32/fmix64 hash
// of the key (transform 2). perm[p] = input row placed at output position p;
// stability means rows of equal digit keep their input order, which
// std::stable_sort by digit gives by definition. offsets[d] = first position of
// digit d, offsets[2^(hi-lo)] = n (skipped when offsets is null).
void oracle_radix_partition(const int64_t* key, int64_t n, int32_t key_bytes, int32_t lo, int32_t hi,
                            int32_t transform, int64_t* perm, int64_t* offsets) {
  std::vector<uint64_t> dig(n);
  for (int64_t i = 0; i < n; ++i) {
    uint64_t bits;
    if (key_bytes == 4) {
      uint32_t k = (uint32_t)(int32_t)key[i];
      if (transform == 1) k ^= 0x80000000u;
      if (transform == 2) k = fmix32(k);
      bits = k;
    } else {
      uint64_t k = (uint64_t)key[i];
      if (transform == 1) k ^= 0x8000000000000000ull;
      if (transform == 2) k = fmix64(k);
      bits = k;
    }
    int width = hi - lo;
    dig[i] = (bits >> lo) & ((width >= 64) ? ~0ull : ((1ull << width) - 1));
  }
  std::iota(perm, perm + n, 0);
  std::stable_sort(perm, perm + n, [&](int64_t a, int64_t b) { return dig[a] < dig[b]; });
  if (offsets == nullptr) return;  // digit ranges too wide to tabulate
  const int64_t nd = (int64_t)1 << (hi - lo);
  std::fill(offsets, offsets + nd + 1, 0);
  for (int64_t i = 0; i < n; ++i) offsets[dig[i] + 1]++;
  for (int64_t d = 0; d < nd; ++d) offsets[d + 1] += offsets[d];
}

}  // extern "C"
