// Grouped aggregation (paper Sec. 3.2, 4.1.3, 4.2, 4.3, 4.4).
//
// HGB (Sec. 4.2, Algorithm 1): stage 1 inserts every key with its tuple id into
// a global hash table; the inserting tuple takes a dense group id from an atomic
// counter and writes the output key, every tuple records the id of the tuple
// its key was inserted with (groupIdLoc). Stage 2 decides on the device whether
// the g groups' aggregates fit in shared memory; if so each block aggregates
// into shared memory and merges into the result, otherwise it aggregates
// straight into global memory. Lanes of a warp holding the same key insert once
// (warp-level deduplication) so that few distinct keys do not serialise on the
// table.
//
// SGB-TR (Sec. 4.1.3): the key and every aggregated value column are sorted
// together (GFTR) by the stable LSD radix sort; a segmented reduction over the
// sorted rows writes each group once, at the row that ends its segment.
// Segments crossing tiles are carried by a decoupled look-back over (head
// count, open-segment aggregate) records, so long runs stay parallel.
//
// PGB-TR (Sec. 4.3): key and values are partitioned together on hashed key bits;
// one block per partition inserts all keys of the partition into a shared-memory
// table first (group discovery decoupled from aggregation), publishes the
// partition's group count through a look-back over partitions to get dense
// output offsets, then aggregates: one group -> block reduction, otherwise
// shared-memory slots flushed with plain stores (the block owns the groups). A
// partition with more distinct keys than the table holds is processed in 2^q
// sub-rounds split by a second hash, so no partition ever falls back to global
// atomics.
#include <cuda_runtime.h>

#include <algorithm>
#include <type_traits>

#include "gj_internal.cuh"

namespace gj {

namespace {

// ================================================================ HGB
template <typename K>
__global__ void __launch_bounds__(256) hgb_group_id_kernel(const K* __restrict__ key, int64_t n,
                                                           int32_t* __restrict__ ht, uint64_t mask,
                                                           int32_t* __restrict__ gid_of_row,
                                                           int32_t* __restrict__ gidloc,
                                                           unsigned long long* ngroups, K* __restrict__ out_keys,
                                                           int64_t cap, int* err) {
  const int lane = threadIdx.x & 31;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  const int64_t n_round = (n + 31) & ~int64_t(31);
  // kBatch rows per thread per step: their key loads and first table probes are
  // in flight together; a collision continues probing on its own
  constexpr int kBatch = 4;
  for (int64_t it = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; it < n_round; it += stride * kBatch) {
    K k[kBatch];
    bool valid[kBatch];
#pragma unroll
    for (int u = 0; u < kBatch; ++u) {
      const int64_t i = it + u * stride;
      valid[u] = i < n;
      k[u] = valid[u] ? key[i] : K(0);
    }
    int leader[kBatch], prev[kBatch];
    uint64_t sl[kBatch];
#pragma unroll
    for (int u = 0; u < kBatch; ++u) {
      const unsigned vmask = __ballot_sync(0xffffffffu, valid[u]);
      const unsigned peers = __match_any_sync(0xffffffffu, k[u]) & vmask;
      leader[u] = valid[u] ? __ffs(peers) - 1 : lane;
      sl[u] = KeyTraits<K>::hash64(k[u]) & mask;
      prev[u] = (valid[u] && lane == leader[u]) ? atomicCAS(&ht[sl[u]], 0, (int)(it + u * stride + 1)) : -1;
    }
    K pk[kBatch];
#pragma unroll
    for (int u = 0; u < kBatch; ++u) pk[u] = prev[u] > 0 ? key[prev[u] - 1] : K(0);
#pragma unroll
    for (int u = 0; u < kBatch; ++u) {
      const int64_t i = it + u * stride;
      int32_t loc = -1;
      if (prev[u] >= 0) {
        int pv = prev[u];
        K pkey = pk[u];
        uint64_t s2 = sl[u];
        for (uint64_t probe = 0; probe <= mask; ++probe) {
          if (pv == 0) {
            const unsigned long long g = atomicAdd(ngroups, 1ull);
            gid_of_row[i] = (int32_t)g;
            if ((int64_t)g < cap)
              out_keys[g] = k[u];
            else
              set_status(err, GJ_ERR_CAPACITY);
            loc = (int32_t)i;
            break;
          }
          if (pkey == k[u]) {
            loc = pv - 1;
            break;
          }
          s2 = (s2 + 1) & mask;
          pv = atomicCAS(&ht[s2], 0, (int)(i + 1));
          if (pv > 0) pkey = key[pv - 1];
        }
        if (loc < 0) set_status(err, GJ_ERR_CAPACITY);  // table full
      }
      loc = __shfl_sync(0xffffffffu, loc, leader[u]);
      if (valid[u]) gidloc[i] = loc;
    }
  }
}

// out[j][0..g) = the starting value of aggregate j, g read from the device
// counter. MIN/MAX over a 4-byte column start at the 32-bit identity
// (INT32_MAX / INT32_MIN): every group holds at least one row, whose value fits
// 32 bits, so the result is unchanged, and a block's shared-memory slot still at
// that identity has nothing to add (it may hold a real INT32_MAX, which then is
// already the starting value).
__global__ void agg_init_kernel(Aggs A, const int64_t* __restrict__ ngroups, int64_t cap) {
  const int64_t g = min64(*ngroups, cap);
  const int64_t total = g * A.n;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += stride) {
    const int j = (int)(t / g);
    const int op = A.op[j];
    int64_t v = agg_identity(op);
    if (A.size[j] == 4 && op == GJ_AGG_MIN) v = INT32_MAX;
    if (A.size[j] == 4 && op == GJ_AGG_MAX) v = INT32_MIN;
    A.out[j][t - (int64_t)j * g] = v;
  }
}

// Shared-memory slot widths per aggregate: COUNT 4 bytes (a block sees < 2^31
// rows), SUM 8, MIN/MAX as wide as their column. 8-byte arrays come first so
// every array is aligned whatever g is.
struct SmemAggLayout {
  int32_t width[kMaxAggs];
  int32_t order[kMaxAggs];  // aggregates in layout order
  int32_t bytes_per_group;
};

__device__ __forceinline__ void smem_update(int op, int width, unsigned char* slot, int64_t v) {
  if (width == 8) {
    agg_atomic(op, (int64_t*)slot, v);
  } else if (op == GJ_AGG_COUNT) {
    atomicAdd((unsigned int*)slot, 1u);
  } else if (op == GJ_AGG_MIN) {
    atomicMin((int*)slot, (int)v);
  } else {
    atomicMax((int*)slot, (int)v);
  }
}

__device__ __forceinline__ int64_t smem_read(int op, int width, const unsigned char* slot) {
  if (width == 8) return *(const int64_t*)slot;
  if (op == GJ_AGG_COUNT) return (int64_t) * (const unsigned int*)slot;
  return (int64_t) * (const int*)slot;
}

__device__ __forceinline__ void smem_init(int op, int width, unsigned char* slot) {
  if (width == 8)
    *(int64_t*)slot = agg_identity(op);
  else if (op == GJ_AGG_COUNT)
    *(unsigned int*)slot = 0u;
  else
    *(int*)slot = op == GJ_AGG_MIN ? INT32_MAX : INT32_MIN;
}

__global__ void __launch_bounds__(1024) hgb_agg_kernel(const int32_t* __restrict__ gidloc,
                                                       const int32_t* __restrict__ gid_of_row, int64_t n, Aggs A,
                                                       ColCache cc, SmemAggLayout L, const int64_t* __restrict__ ngroups,
                                                       int64_t cap, int smem_budget) {
  extern __shared__ __align__(16) unsigned char s_agg[];
  const int64_t g = min64(*ngroups, cap);
  const bool use_smem = g * (int64_t)L.bytes_per_group <= smem_budget;  // is_smem_enough
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  const int64_t first = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (use_smem) {
    int64_t offs[kMaxAggs];
    int64_t o = 0;
    for (int q = 0; q < A.n; ++q) {
      int j = L.order[q];
      offs[j] = o;
      o += g * L.width[j];
    }
    for (int q = 0; q < A.n; ++q) {
      int j = L.order[q];
      for (int64_t s = threadIdx.x; s < g; s += blockDim.x) smem_init(A.op[j], L.width[j], s_agg + offs[j] + s * L.width[j]);
    }
    __syncthreads();
    // kBatch rows per thread per step: dependent loads of the batch overlap
    constexpr int kBatch = 4;
    for (int64_t it = first; it < n; it += stride * kBatch) {
      int32_t loc[kBatch];
      int64_t gid[kBatch];
#pragma unroll
      for (int u = 0; u < kBatch; ++u) loc[u] = it + u * stride < n ? gidloc[it + u * stride] : -1;
#pragma unroll
      for (int u = 0; u < kBatch; ++u) gid[u] = loc[u] >= 0 ? gid_of_row[loc[u]] : g;  // < 0: insert failed
      int64_t row[kBatch];
      bool valid[kBatch];
#pragma unroll
      for (int u = 0; u < kBatch; ++u) {
        row[u] = it + u * stride;
        valid[u] = gid[u] < g;
      }
      int32_t cv[kColCache][kBatch];
      load_cached<kBatch>(cc, row, valid, cv);
      for (int j = 0; j < A.n; ++j) {
#pragma unroll
        for (int u = 0; u < kBatch; ++u)
          if (valid[u])
            smem_update(A.op[j], L.width[j], s_agg + offs[j] + gid[u] * L.width[j],
                        cached_value<kBatch>(A, cc, j, cv, u, row[u]));
      }
    }
    __syncthreads();
    for (int j = 0; j < A.n; ++j) {
      const int64_t idv = agg_identity(A.op[j]);
      for (int64_t s = threadIdx.x; s < g; s += blockDim.x) {
        int64_t v = smem_read(A.op[j], L.width[j], s_agg + offs[j] + s * L.width[j]);
        if (L.width[j] == 4 && A.op[j] == GJ_AGG_MIN && v == INT32_MAX) continue;
        if (L.width[j] == 4 && A.op[j] == GJ_AGG_MAX && v == INT32_MIN) continue;
        if (v == idv) continue;
        agg_atomic(A.op[j], &A.out[j][s], v);
      }
    }
  } else {
    constexpr int kBatch = 4;
    for (int64_t it = first; it < n; it += stride * kBatch) {
      int32_t loc[kBatch];
      int64_t gid[kBatch];
#pragma unroll
      for (int u = 0; u < kBatch; ++u) loc[u] = it + u * stride < n ? gidloc[it + u * stride] : -1;
#pragma unroll
      for (int u = 0; u < kBatch; ++u) gid[u] = loc[u] >= 0 ? gid_of_row[loc[u]] : g;
      int64_t row[kBatch];
      bool valid[kBatch];
#pragma unroll
      for (int u = 0; u < kBatch; ++u) {
        row[u] = it + u * stride;
        valid[u] = gid[u] < g;
      }
      int32_t cv[kColCache][kBatch];
      load_cached<kBatch>(cc, row, valid, cv);
      for (int j = 0; j < A.n; ++j) {
#pragma unroll
        for (int u = 0; u < kBatch; ++u)
          if (valid[u]) agg_atomic(A.op[j], &A.out[j][gid[u]], cached_value<kBatch>(A, cc, j, cv, u, row[u]));
      }
    }
  }
}

// ================================================================ SGB
constexpr int kSegItems = 16;
constexpr int kSegWarps = 8;
constexpr int kSegWarpRows = 32 * kSegItems;         // rows per warp
constexpr int kSegTile = kSegWarps * kSegWarpRows;   // rows per block tile

// Segmented combine: (ha, a) then (hb, b) -> b restarts when its part holds a head.
__device__ __forceinline__ int64_t seg_combine(int op, bool hb, int64_t a, int64_t b) {
  return hb ? b : agg_combine(op, a, b);
}

// Value columns a segmented reduction keeps in registers: slot[j] is the cached
// column of aggregate j, or -1 (COUNT, or read through Aggs).
constexpr int kSegCache = 3;
struct SegCols {
  int32_t n;
  const int32_t* src[kSegCache];
  int8_t slot[kMaxAggs];
  const int32_t* tid;  // GFUR: values of sorted row r at src[tid[r]]
};

// Aggregate OP over value source SLOT (a cached column, or -1: read through
// Aggs) with both fixed at compile time, so the per-row loops carry no branches.
template <int OP, int SLOT>
struct SegOp {
  // COUNT, and MIN/MAX over a cached 4-byte column, run in 32 bits: a count stays
  // below 2^30 and a MIN/MAX of 4-byte values is one of them, while the 32-bit
  // identities (INT32_MAX for MIN, INT32_MIN for MAX) leave such values unchanged,
  // so narrowing the 64-bit identity or carry to them is exact.
  using T = typename std::conditional<OP == GJ_AGG_COUNT || ((OP == GJ_AGG_MIN || OP == GJ_AGG_MAX) && SLOT >= 0),
                                      int32_t, int64_t>::type;
  static __device__ __forceinline__ T value(const Aggs& A, int j, const int32_t (&cv)[kSegCache][kSegItems], int r,
                                            int64_t row) {
    if (OP == GJ_AGG_COUNT) return 1;
    if (SLOT >= 0) return cv[SLOT][r];
    return (T)load_as_i64(A.src[j], A.size[j], A.tid ? (int64_t)A.tid[row] : row);
  }
  static __device__ __forceinline__ T comb(T a, T b) {
    if (OP == GJ_AGG_MIN) return a < b ? a : b;
    if (OP == GJ_AGG_MAX) return a > b ? a : b;
    return (T)((typename std::make_unsigned<T>::type)a + (typename std::make_unsigned<T>::type)b);
  }
  static __device__ __forceinline__ T ident() {
    if (sizeof(T) == 4) return OP == GJ_AGG_MIN ? INT32_MAX : (OP == GJ_AGG_MAX ? INT32_MIN : 0);
    return (T)agg_identity(OP);
  }
  static __device__ __forceinline__ T narrow(int64_t x) {
    if (sizeof(T) == 8) return (T)x;
    if (OP == GJ_AGG_COUNT) return (T)x;
    return (T)(x > INT32_MAX ? INT32_MAX : (x < INT32_MIN ? INT32_MIN : x));
  }
};

// Calls f(SegOp<op, slot>{}) for the runtime pair (op, slot); COUNT ignores slot.
template <typename F>
__device__ __forceinline__ void seg_dispatch(int op, int slot, F&& f) {
  if (op == GJ_AGG_COUNT) return f(SegOp<GJ_AGG_COUNT, -1>{});
#define GJ_SEG_CASE(OPV)                          \
  if (op == OPV) {                                \
    if (slot == 0) return f(SegOp<OPV, 0>{});     \
    if (slot == 1) return f(SegOp<OPV, 1>{});     \
    if (slot == 2) return f(SegOp<OPV, 2>{});     \
    return f(SegOp<OPV, -1>{});                   \
  }
  GJ_SEG_CASE(GJ_AGG_SUM)
  GJ_SEG_CASE(GJ_AGG_MIN)
  GJ_SEG_CASE(GJ_AGG_MAX)
#undef GJ_SEG_CASE
}

// Head bits of a lane's kSegItems sorted rows starting at rb (bit r: row rb + r
// starts a segment), and whether the row after its last row starts one (or the
// input ends there). tb is the warp's first row. Keys are read with 16-byte loads.
template <typename K>
__device__ __forceinline__ uint32_t seg_heads(const K* __restrict__ key, int64_t n, int64_t tb, int64_t rb, int nvalid,
                                              bool& last_ends) {
  const int lane = threadIdx.x & 31;
  K k[kSegItems];
  if (nvalid == kSegItems && (reinterpret_cast<uintptr_t>(key + rb) & 15) == 0) {
    constexpr int kVec = 16 / sizeof(K);
#pragma unroll
    for (int q = 0; q < kSegItems / kVec; ++q) {
      const int4 u = __ldcs(reinterpret_cast<const int4*>(key + rb) + q);
      const K* e = reinterpret_cast<const K*>(&u);
#pragma unroll
      for (int t = 0; t < kVec; ++t) k[q * kVec + t] = e[t];
    }
  } else {
#pragma unroll
    for (int r = 0; r < kSegItems; ++r) k[r] = r < nvalid ? key[rb + r] : K(0);
  }
  const K prev_last = __shfl_up_sync(0xffffffffu, k[kSegItems - 1], 1);
  bool first_is_head;
  if (lane == 0)
    first_is_head = tb == 0 || (tb < n && key[tb - 1] != k[0]);
  else
    first_is_head = prev_last != k[0];
  uint32_t hm = 0;
#pragma unroll
  for (int r = 0; r < kSegItems; ++r) {
    const bool h = r == 0 ? first_is_head : (k[r] != k[r - 1]);
    if (r < nvalid && h) hm |= 1u << r;
  }
  const uint32_t next_head = __shfl_down_sync(0xffffffffu, hm & 1u, 1);
  const int64_t lastrow = rb + kSegItems - 1;
  if (lastrow + 1 >= n)
    last_ends = true;
  else if (lane == 31)
    last_ends = key[lastrow + 1] != k[kSegItems - 1];
  else
    last_ends = next_head != 0;
  return hm;
}

// Up to kSegCache 4-byte value columns of a lane's rows [r0, nvalid) into registers.
__device__ __forceinline__ void seg_load_cols(const SegCols& sc, int64_t rb, int r0, int nvalid,
                                              int32_t (&cv)[kSegCache][kSegItems]) {
  if (sc.tid) {
    // GFUR: the rows' tuple ids first, then every column gathered through them
    int32_t id[kSegItems];
#pragma unroll
    for (int r = 0; r < kSegItems; ++r) id[r] = (sc.n > 0 && r >= r0 && r < nvalid) ? __ldcs(sc.tid + rb + r) : 0;
#pragma unroll
    for (int s = 0; s < kSegCache; ++s) {
      if (s >= sc.n) break;
#pragma unroll
      for (int r = 0; r < kSegItems; ++r) cv[s][r] = (r >= r0 && r < nvalid) ? __ldg(sc.src[s] + id[r]) : 0;
    }
    return;
  }
#pragma unroll
  for (int s = 0; s < kSegCache; ++s) {
    if (s >= sc.n) break;
    const int32_t* src = sc.src[s] + rb;
    if (r0 == 0 && nvalid == kSegItems && (reinterpret_cast<uintptr_t>(src) & 15) == 0) {
#pragma unroll
      for (int q = 0; q < kSegItems / 4; ++q) {
        const int4 u = __ldcs(reinterpret_cast<const int4*>(src) + q);
        cv[s][4 * q] = u.x;
        cv[s][4 * q + 1] = u.y;
        cv[s][4 * q + 2] = u.z;
        cv[s][4 * q + 3] = u.w;
      }
    } else {
#pragma unroll
      for (int r = 0; r < kSegItems; ++r) cv[s][r] = (r >= r0 && r < nvalid) ? src[r] : 0;
    }
  }
}

// Records: a run of sorted rows is summarised by (cnt: heads it holds, has: cnt
// > 0, val[j]: aggregate j over the rows after its last head, or over all of
// them if it holds none). (a then b) = (a.cnt + b.cnt, a.has | b.has, b.has ?
// b.val : op(a.val, b.val)), an associative combine, so the carry into every
// tile is an exclusive scan of the tile records.
//
// Pass 1: one block per tile of kSegTile rows writes the tile's record
// rec[tile][cnt, has, val[nagg]]; only the rows after each warp's last head are
// read beyond the keys.
template <typename K>
__global__ void __launch_bounds__(kSegWarps * 32) sgb_tile_kernel(const K* __restrict__ key, int64_t n, Aggs A,
                                                                  SegCols sc, int64_t* __restrict__ rec) {
  __shared__ int64_t s_w[kSegWarps][kMaxAggs + 2];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int nagg = A.n;
  const int64_t tile = blockIdx.x;
  const int64_t tb = tile * kSegTile + (int64_t)warp * kSegWarpRows;
  const int64_t rb = tb + (int64_t)lane * kSegItems;
  const int nvalid = (int)(rb >= n ? 0 : min64(n - rb, kSegItems));
  bool last_ends;
  const uint32_t hm = seg_heads<K>(key, n, tb, rb, nvalid, last_ends);
  const unsigned has_mask = __ballot_sync(0xffffffffu, hm != 0);
  // the warp's tail starts at its last head (the warp's first row if it has none)
  const int tail_lane = has_mask ? 31 - __clz(has_mask) : -1;
  const int r0 = lane < tail_lane ? kSegItems : (lane == tail_lane ? 31 - __clz(hm) : 0);
  int32_t cv[kSegCache][kSegItems];
  seg_load_cols(sc, rb, r0, nvalid, cv);
  for (int j = 0; j < nagg; ++j) {
    int64_t t64;
    seg_dispatch(A.op[j], sc.slot[j], [&](auto S) {
      using Op = decltype(S);
      typename Op::T t = Op::ident();
#pragma unroll
      for (int r = 0; r < kSegItems; ++r)
        if (r >= r0 && r < nvalid) t = Op::comb(t, Op::value(A, j, cv, r, rb + r));
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) t = Op::comb(t, __shfl_xor_sync(0xffffffffu, t, o));
      t64 = t;
    });
    if (lane == 0) s_w[warp][2 + j] = t64;
  }
  int cnt = __popc(hm);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
  if (lane == 0) {
    s_w[warp][0] = cnt;
    s_w[warp][1] = has_mask != 0;
  }
  __syncthreads();
  const int rw = nagg + 2;
  int64_t* my = rec + tile * rw;
  if (threadIdx.x < nagg) {
    const int j = threadIdx.x;
    const int op = A.op[j];
    int64_t v = agg_identity(op);
    for (int w = 0; w < kSegWarps; ++w) v = seg_combine(op, s_w[w][1] != 0, v, s_w[w][2 + j]);
    my[2 + j] = v;
  } else if (threadIdx.x == 32) {
    int64_t c = 0, h = 0;
    for (int w = 0; w < kSegWarps; ++w) {
      c += s_w[w][0];
      h |= s_w[w][1];
    }
    my[0] = c;
    my[1] = h;
  }
}

// Pass 2: exclusive scan of the tile records in two levels. sgb_scan_kernel
// gives every item of a block of kScanBlock items the record of the items before
// it within the block (excl) and writes the block's total record (totals); run
// once over the tiles and once, as a single block, over those totals. A tile's
// carry is then (block carry then in-block carry). Records and carries share the
// layout [cnt, has, val[nagg]]; d_total (if set) receives the total count.
constexpr int kScanBlock = 1024;

// does the range of 2^st items ending at idx (clamped at 0) hold a set bit of m?
__device__ __forceinline__ bool range_has(unsigned m, int idx, int st) {
  const int lo = idx - (1 << st) + 1;
  return ((m >> (lo > 0 ? lo : 0)) & (((2u << idx) - 1) >> (lo > 0 ? lo : 0))) != 0;
}

__global__ void __launch_bounds__(kScanBlock) sgb_scan_kernel(const int64_t* __restrict__ rec, int64_t count, Aggs A,
                                                              int64_t* __restrict__ excl, int64_t* __restrict__ totals,
                                                              int64_t* d_total) {
  __shared__ int64_t s_v[32];
  __shared__ unsigned s_wm;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int nwarps = blockDim.x >> 5;
  const int nagg = A.n, rw = nagg + 2;
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const bool valid = i < count;
  const bool h = valid && rec[i * rw + 1] != 0;
  const unsigned hmask = __ballot_sync(0xffffffffu, h);
  if (threadIdx.x == 0) s_wm = 0;
  __syncthreads();
  if (lane == 0 && hmask) atomicOr(&s_wm, 1u << warp);
  __syncthreads();
  const unsigned wmask = s_wm;
  const bool lanes_before = (hmask & ((1u << lane) - 1)) != 0;
  const bool warps_before = (wmask & ((1u << warp) - 1)) != 0;
  if (valid) excl[i * rw + 1] = lanes_before || warps_before;
  const bool last = threadIdx.x == blockDim.x - 1;
  if (totals && last) totals[(int64_t)blockIdx.x * rw + 1] = wmask != 0;
  // field -1 is the count (a plain sum); field f >= 0 aggregate f (segmented)
  for (int f = -1; f < nagg; ++f) {
    const int op = f < 0 ? (int)GJ_AGG_SUM : A.op[f];
    const int off = f < 0 ? 0 : 2 + f;
    const int64_t v = valid ? rec[i * rw + off] : agg_identity(op);
    int64_t x = v;
#pragma unroll
    for (int st = 0; st < 5; ++st) {
      const int64_t xp = __shfl_up_sync(0xffffffffu, x, 1 << st);
      if (lane >= (1 << st)) x = seg_combine(op, f >= 0 && range_has(hmask, lane, st), xp, x);
    }
    if (lane == 31) s_v[warp] = x;
    __syncthreads();
    if (warp == 0) {
      int64_t y = lane < nwarps ? s_v[lane] : agg_identity(op);
#pragma unroll
      for (int st = 0; st < 5; ++st) {
        const int64_t yp = __shfl_up_sync(0xffffffffu, y, 1 << st);
        if (lane >= (1 << st)) y = seg_combine(op, f >= 0 && range_has(wmask, lane, st), yp, y);
      }
      s_v[lane] = y;
    }
    __syncthreads();
    int64_t xe = __shfl_up_sync(0xffffffffu, x, 1);
    if (lane == 0) xe = agg_identity(op);
    const int64_t run = warp > 0 ? seg_combine(op, f >= 0 && lanes_before, s_v[warp - 1], xe) : xe;
    if (valid) excl[i * rw + off] = run;
    if (last) {
      const int64_t tot = seg_combine(op, f >= 0 && h, run, v);
      if (totals) totals[(int64_t)blockIdx.x * rw + off] = tot;
      if (d_total && f < 0) *d_total = tot;
    }
    __syncthreads();
  }
}

// Pass 3: one block per tile. Each lane walks its rows once: segments that start
// in the lane are written when they end; the rows before its first head continue
// a segment from earlier rows, whose value needs the carry into the lane and is
// written after the scans (if it ends in the lane). The carry into a lane is the
// tile carry, then the warps before it, then the lanes before it. Head counts
// need no values, so every group id is known before the row walk.
template <typename K>
__global__ void __launch_bounds__(kSegWarps * 32, 2) sgb_reduce_kernel(const K* __restrict__ key, int64_t n, Aggs A,
                                                                    SegCols sc, K* __restrict__ out_keys, int64_t cap,
                                                                    const int64_t* __restrict__ carry,
                                                                    const int64_t* __restrict__ bcarry, int* err) {
  extern __shared__ __align__(16) int64_t s_dyn[];
  __shared__ int64_t s_wcnt[kSegWarps];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int nagg = A.n;
  const int rw = nagg + 2;
  int64_t* s_inc = s_dyn + (int64_t)warp * nagg * 32;                          // [nagg][32] lane inclusive values
  int64_t* s_pre = s_dyn + (int64_t)kSegWarps * nagg * 32 + warp * nagg * 32;  // [nagg][32] open-segment folds
  int64_t* s_wrec = s_dyn + (int64_t)2 * kSegWarps * nagg * 32;                // [kSegWarps] warp records
  int64_t* s_carry = s_wrec + kSegWarps * rw;                                   // [kSegWarps] carry into each warp

  const int64_t tile = blockIdx.x;
  const int64_t* tc = carry + tile * rw;                      // carry within the scan block
  const int64_t* bc = bcarry + (tile / kScanBlock) * rw;      // carry of the scan block
  const int64_t tb = tile * kSegTile + (int64_t)warp * kSegWarpRows;
  const int64_t rb = tb + (int64_t)lane * kSegItems;
  const int nvalid = (int)(rb >= n ? 0 : min64(n - rb, kSegItems));
  bool last_ends;
  const uint32_t hm = seg_heads<K>(key, n, tb, rb, nvalid, last_ends);
  const uint32_t heads = __popc(hm);
  uint32_t hincl = heads;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    uint32_t y = __shfl_up_sync(0xffffffffu, hincl, o);
    if (lane >= o) hincl += y;
  }
  const uint32_t warp_heads = __shfl_sync(0xffffffffu, hincl, 31);
  const unsigned has_mask = __ballot_sync(0xffffffffu, hm != 0);
  if (lane == 0) s_wcnt[warp] = warp_heads;
  __syncthreads();
  int64_t cnt_before = bc[0] + tc[0] + (hincl - heads);
  for (int w = 0; w < warp; ++w) cnt_before += s_wcnt[w];
  // rows that end a segment; rows before the first head continue an open segment
  const uint32_t vmask = (1u << nvalid) - 1;
  const uint32_t em = ((hm >> 1) | (last_ends ? 1u << (kSegItems - 1) : 0u) |
                       (nvalid > 0 && nvalid < kSegItems ? 1u << (nvalid - 1) : 0u)) & vmask;
  const int fh = hm ? __ffs(hm) - 1 : kSegItems;
  const bool pre_ends = (em & ((1u << fh) - 1)) != 0;

  int32_t cv[kSegCache][kSegItems];
  seg_load_cols(sc, rb, 0, nvalid, cv);
  bool hstep[5];
#pragma unroll
  for (int st = 0; st < 5; ++st) hstep[st] = range_has(has_mask, lane, st);

  bool overflow = false;
  for (int j = 0; j < nagg; ++j) {
    int64_t x64, pre64;
    int64_t* out = A.out[j];
    seg_dispatch(A.op[j], sc.slot[j], [&](auto S) {
      using Op = decltype(S);
      typename Op::T run = Op::ident(), pre = Op::ident();
#pragma unroll
      for (int r = 0; r < kSegItems; ++r) {
        if (r < nvalid) {
          const typename Op::T v = Op::value(A, j, cv, r, rb + r);
          run = ((hm >> r) & 1u) ? v : Op::comb(run, v);
          if ((em >> r) & 1u) {
            if (r < fh) {
              pre = run;
            } else {
              const int64_t gid = cnt_before + __popc(hm & ((2u << r) - 1)) - 1;
              if (gid < cap)
                out[gid] = (int64_t)run;
              else
                overflow = true;
            }
          }
        }
      }
      // run is now the fold after the lane's last head (all its rows if it has
      // none): its record value, scanned over the warp's lanes
      typename Op::T x = run;
#pragma unroll
      for (int st = 0; st < 5; ++st) {
        const typename Op::T xp = __shfl_up_sync(0xffffffffu, x, 1 << st);
        if (lane >= (1 << st) && !hstep[st]) x = Op::comb(xp, x);
      }
      x64 = x;
      pre64 = pre;
    });
    s_inc[j * 32 + lane] = x64;
    s_pre[j * 32 + lane] = pre64;
  }
  __syncwarp();
  if (lane == 0) {
    s_wrec[warp * rw] = warp_heads;
    s_wrec[warp * rw + 1] = has_mask != 0;
  }
  for (int j = lane; j < nagg; j += 32) s_wrec[warp * rw + 2 + j] = s_inc[j * 32 + 31];
  __syncthreads();

  if (warp == 0) {
    const bool tc_has = tc[1] != 0;
    for (int j = lane; j < nagg; j += 32) {
      const int op = A.op[j];
      int64_t run = seg_combine(op, tc_has, bc[2 + j], tc[2 + j]);
      for (int w = 0; w < kSegWarps; ++w) {
        s_carry[w * rw + 2 + j] = run;
        run = seg_combine(op, s_wrec[w * rw + 1] != 0, run, s_wrec[w * rw + 2 + j]);
      }
    }
  }
  __syncthreads();

  // ---- the open segment's value, where it ends in this lane
  if (pre_ends) {
    const int64_t* wc = s_carry + warp * rw;
    const bool lanes_before = (has_mask & ((1u << lane) - 1)) != 0;
    const int64_t gid = cnt_before - 1;
    for (int j = 0; j < nagg; ++j) {
      const int op = A.op[j];
      const int64_t cin = lane == 0 ? wc[2 + j] : seg_combine(op, lanes_before, wc[2 + j], s_inc[j * 32 + lane - 1]);
      if (gid < cap)
        A.out[j][gid] = agg_combine(op, cin, s_pre[j * 32 + lane]);
      else
        overflow = true;
    }
  }
  {
    int64_t gcount = cnt_before;
    for (int r = 0; r < nvalid; ++r) {
      if ((hm >> r) & 1u) {
        if (gcount < cap)
          out_keys[gcount] = key[rb + r];  // re-read (cache hit) rather than kept live in registers
        else
          overflow = true;
        ++gcount;
      }
    }
  }
  if (overflow) set_status(err, GJ_ERR_CAPACITY);
}

// ================================================================ PGB
constexpr int kPgbThreads = 512;
constexpr int kPgbCap = 4096;        // distinct keys per shared-memory table
constexpr int kPgbSlots = 2 * kPgbCap;
constexpr int kPgbMaxQ = 12;

template <typename K>
__device__ __forceinline__ uint32_t pgb_sub(K k, int q) {
  if (q == 0) return 0;
  uint32_t h = fmix32((uint32_t)KeyTraits<K>::hash64(k) ^ 0x9e3779b9u);
  return h & ((1u << q) - 1);
}

template <typename K>
__device__ __forceinline__ uint32_t pgb_slot(K k, int pbits) {
  return (uint32_t)(KeyTraits<K>::hash64(k) >> pbits) & (kPgbSlots - 1);
}

// Inserts the keys of rows [r0, r1) with sub-round `round` into the table.
// Returns the distinct count, or -1 on overflow.
// Inserts the keys of rows [r0, r1) with sub-round `round` into the table. A
// slot holds (partition row + 1) of the first row seen with its key; keys are
// compared in global memory, so claiming a slot is one CAS and no thread ever
// waits on another. Occupied slots then get dense local ids in slot order
// (s_keys[lid], s_lid[slot]). Returns the distinct count, or -1 if it exceeds
// kPgbCap.
template <typename K>
__device__ int pgb_build(const K* __restrict__ key, int64_t r0, int64_t r1, int q, uint32_t round, int pbits,
                         int32_t* s_slots, K* s_keys, int* s_count, int* s_over) {
  int16_t* s_lid = (int16_t*)(s_keys + kPgbCap);
  for (int j = threadIdx.x; j < kPgbSlots; j += blockDim.x) s_slots[j] = 0;
  if (threadIdx.x == 0) {
    *s_count = 0;
    *s_over = 0;
  }
  __syncthreads();
  // rows in batches of kBatch per thread: the batch's key loads are in flight together
  constexpr int kBatch = 8;
  // the last key this thread inserted or found: a run of equal keys (few groups
  // per partition) skips the table after its first row
  K last = K(0);
  bool has_last = false;
  for (int64_t b0 = r0; b0 < r1; b0 += (int64_t)kBatch * blockDim.x) {
    K kk[kBatch];
#pragma unroll
    for (int u = 0; u < kBatch; ++u) {
      const int64_t i = b0 + (int64_t)u * blockDim.x + threadIdx.x;
      kk[u] = i < r1 ? key[i] : K(0);
    }
#pragma unroll
    for (int u = 0; u < kBatch; ++u) {
      const int64_t i = b0 + (int64_t)u * blockDim.x + threadIdx.x;
      if (i >= r1) continue;
      const K k = kk[u];
      if (has_last && k == last) continue;
      if (pgb_sub<K>(k, q) != round) continue;
      last = k;
      has_last = true;
      uint32_t sl = pgb_slot<K>(k, pbits);
      volatile int32_t* vs = s_slots;
      for (int probe = 0; probe < kPgbSlots; ++probe) {
        int v = vs[sl];  // a repeated key finds its slot without an atomic
        if (v == 0) {
          v = atomicCAS(&s_slots[sl], 0, (int)(i - r0 + 1));
          if (v == 0) break;
        }
        if (key[r0 + v - 1] == k) break;
        sl = (sl + 1) & (kPgbSlots - 1);
      }
    }
  }
  __syncthreads();
  // dense ids in slot order: block-wide count of occupied slots before each one
  constexpr int kPer = kPgbSlots / kPgbThreads;
  const int s0 = threadIdx.x * kPer;
  int mine = 0;
#pragma unroll
  for (int r = 0; r < kPer; ++r) mine += s_slots[s0 + r] != 0;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int x = mine;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  __shared__ int s_wsum[kPgbThreads / 32];
  if (lane == 31) s_wsum[warp] = x;
  __syncthreads();
  if (threadIdx.x == 0) {
    int run = 0;
    for (int w = 0; w < kPgbThreads / 32; ++w) {
      const int c = s_wsum[w];
      s_wsum[w] = run;
      run += c;
    }
    *s_count = run;
    *s_over = run > kPgbCap;
  }
  __syncthreads();
  const int total = *s_count;
  if (total <= kPgbCap) {
    int lid = s_wsum[warp] + x - mine;
#pragma unroll
    for (int r = 0; r < kPer; ++r) {
      const int v = s_slots[s0 + r];
      if (v != 0) {
        s_keys[lid] = key[r0 + v - 1];
        s_lid[s0 + r] = (int16_t)lid;
        ++lid;
      }
    }
  }
  __syncthreads();
  return total > kPgbCap ? -1 : total;
}

template <typename K>
__device__ __forceinline__ int pgb_lookup(K k, int pbits, const int32_t* s_slots, const K* s_keys) {
  const int16_t* s_lid = (const int16_t*)(s_keys + kPgbCap);
  uint32_t sl = pgb_slot<K>(k, pbits);
  for (int probe = 0; probe < kPgbSlots; ++probe) {
    const int v = s_slots[sl];
    if (v == 0) return -1;
    const int l = s_lid[sl];
    if (s_keys[l] == k) return l;
    sl = (sl + 1) & (kPgbSlots - 1);
  }
  return -1;
}

template <typename K>
__global__ void __launch_bounds__(kPgbThreads, 2) pgb_kernel(const K* __restrict__ key,
                                                          const int64_t* __restrict__ poff, int pbits, Aggs A,
                                                          ColCache cc, K* __restrict__ out_keys, int64_t cap, int mode,
                                                          int64_t* __restrict__ gcount, int8_t* __restrict__ qsel,
                                                          int* err) {
  extern __shared__ __align__(16) unsigned char s_raw[];
  int64_t* s_agg = (int64_t*)s_raw;                       // kPgbCap aggregates
  int32_t* s_slots = (int32_t*)(s_agg + kPgbCap);         // table: local id + 1
  K* s_keys = (K*)(s_slots + kPgbSlots);                  // distinct keys by local id
  __shared__ int s_count, s_over;
  __shared__ int64_t s_red[kPgbThreads / 32];

  const int64_t p = blockIdx.x;
  const int64_t r0 = poff[p], r1 = poff[p + 1];

  int q = 0;
  int64_t total = 0;
  if (mode == 0) {
    // ---- counting launch: the smallest split q whose sub-rounds all fit
    for (;;) {
      total = 0;
      bool ok = true;
      for (uint32_t round = 0; round < (1u << q); ++round) {
        int c = pgb_build<K>(key, r0, r1, q, round, pbits, s_slots, s_keys, &s_count, &s_over);
        if (c < 0) {
          ok = false;
          break;
        }
        total += c;
      }
      __syncthreads();
      if (ok) break;
      if (++q > kPgbMaxQ) {
        if (threadIdx.x == 0) set_status(err, GJ_ERR_CAPACITY);
        total = 0;
        q = -1;
        break;
      }
    }
    if (threadIdx.x == 0) {
      gcount[p] = total;
      qsel[p] = (int8_t)q;
    }
    return;
  }
  // ---- aggregating launch: offsets are known, no block waits on another
  q = qsel[p];
  if (q < 0) return;
  const int64_t goff = gcount[p];
  total = gcount[p + 1] - goff;
  if (total == 0) return;
  // one group needs no table: every row of the partition holds the key of its first
  if (q == 0 && total > 1) pgb_build<K>(key, r0, r1, 0, 0, pbits, s_slots, s_keys, &s_count, &s_over);

  // one group: register accumulators below
  constexpr int kOneGroupAggs = 8;
  const bool one_group = q == 0 && total == 1;

  // ---- few groups, one round: every aggregate in one pass over the partition.
  // When the slots are few, every warp updates its own copy (no contention
  // between warps) and the copies are combined at the end.
  if (q == 0 && !one_group && total * A.n <= kPgbCap) {
    const int g = (int)total;
    const int nsl = g * A.n;
    constexpr int kWarpsPgb = kPgbThreads / 32;
    const int ncopy = nsl * kWarpsPgb <= kPgbCap ? kWarpsPgb : 1;
    int64_t* my = s_agg + (ncopy > 1 ? (threadIdx.x >> 5) * nsl : 0);
    for (int l = threadIdx.x; l < g; l += blockDim.x) {
      if (goff + l < cap)
        out_keys[goff + l] = s_keys[l];
      else
        set_status(err, GJ_ERR_CAPACITY);
    }
    for (int s = threadIdx.x; s < nsl * ncopy; s += blockDim.x) s_agg[s] = agg_identity(A.op[(s % nsl) / g]);
    __syncthreads();
    constexpr int kBatch = 4;
    for (int64_t b0 = r0; b0 < r1; b0 += (int64_t)kBatch * blockDim.x) {
      K kk[kBatch];
#pragma unroll
      for (int u = 0; u < kBatch; ++u) {
        const int64_t i = b0 + (int64_t)u * blockDim.x + threadIdx.x;
        kk[u] = i < r1 ? key[i] : K(0);
      }
      int lid[kBatch];
      int64_t row[kBatch];
      bool valid[kBatch];
#pragma unroll
      for (int u = 0; u < kBatch; ++u) {
        row[u] = b0 + (int64_t)u * blockDim.x + threadIdx.x;
        valid[u] = row[u] < r1;
        lid[u] = valid[u] ? pgb_lookup<K>(kk[u], pbits, s_slots, s_keys) : -1;
      }
      int32_t cv[kColCache][kBatch];
      load_cached<kBatch>(cc, row, valid, cv);
      for (int j = 0; j < A.n; ++j) {
#pragma unroll
        for (int u = 0; u < kBatch; ++u)
          if (lid[u] >= 0) agg_atomic(A.op[j], &my[j * g + lid[u]], cached_value<kBatch>(A, cc, j, cv, u, row[u]));
      }
    }
    __syncthreads();
    for (int s = threadIdx.x; s < nsl; s += blockDim.x) {
      const int j = s / g, l = s - j * g;
      int64_t v = s_agg[s];
      for (int c = 1; c < ncopy; ++c) v = agg_combine(A.op[j], v, s_agg[c * nsl + s]);
      if (goff + l < cap) A.out[j][goff + l] = v;
    }
    return;
  }

  // ---- one group: aggregates accumulated in registers, kOneGroupAggs per pass
  // over the partition, then a block-wide reduction (no atomics)
  if (one_group) {
    if (threadIdx.x == 0) {
      if (goff < cap)
        out_keys[goff] = key[r0];
      else
        set_status(err, GJ_ERR_CAPACITY);
    }
    for (int j0 = 0; j0 < A.n; j0 += kOneGroupAggs) {
      int64_t acc[kOneGroupAggs];
#pragma unroll
      for (int j = 0; j < kOneGroupAggs; ++j) acc[j] = j0 + j < A.n ? agg_identity(A.op[j0 + j]) : 0;
      constexpr int kBatch = 4;
      for (int64_t b0 = r0; b0 < r1; b0 += (int64_t)kBatch * blockDim.x) {
        int64_t row[kBatch];
        bool valid[kBatch];
#pragma unroll
        for (int u = 0; u < kBatch; ++u) {
          row[u] = b0 + (int64_t)u * blockDim.x + threadIdx.x;
          valid[u] = row[u] < r1;
        }
        int32_t cv[kColCache][kBatch];
        load_cached<kBatch>(cc, row, valid, cv);
#pragma unroll
        for (int j = 0; j < kOneGroupAggs; ++j) {
          if (j0 + j < A.n) {
#pragma unroll
            for (int u = 0; u < kBatch; ++u)
              if (valid[u])
                acc[j] = agg_combine(A.op[j0 + j], acc[j], cached_value<kBatch>(A, cc, j0 + j, cv, u, row[u]));
          }
        }
      }
#pragma unroll
      for (int j = 0; j < kOneGroupAggs; ++j) {
        if (j0 + j >= A.n) break;
        for (int o = 16; o > 0; o >>= 1)
          acc[j] = agg_combine(A.op[j0 + j], acc[j], __shfl_down_sync(0xffffffffu, acc[j], o));
        if ((threadIdx.x & 31) == 0) s_agg[(threadIdx.x >> 5) * kOneGroupAggs + j] = acc[j];
      }
      __syncthreads();
      if (threadIdx.x < kOneGroupAggs && j0 + (int)threadIdx.x < A.n && goff < cap) {
        const int j = j0 + threadIdx.x;
        int64_t t = s_agg[threadIdx.x];
        for (int w = 1; w < kPgbThreads / 32; ++w) t = agg_combine(A.op[j], t, s_agg[w * kOneGroupAggs + threadIdx.x]);
        A.out[j][goff] = t;
      }
      __syncthreads();
    }
    return;
  }

  int64_t base = goff;
  for (uint32_t round = 0; round < (1u << q); ++round) {
    // with one round the table built during discovery is still in place
    int g = q == 0 ? (int)total : pgb_build<K>(key, r0, r1, q, round, pbits, s_slots, s_keys, &s_count, &s_over);
    if (g <= 0) continue;
    for (int l = threadIdx.x; l < g; l += blockDim.x) {
      if (base + l < cap)
        out_keys[base + l] = s_keys[l];
      else
        set_status(err, GJ_ERR_CAPACITY);
    }
    for (int j = 0; j < A.n; ++j) {
      const int op = A.op[j];
      if (g == 1) {
        // one group: block-wide reduction, no atomics
        int64_t acc = agg_identity(op);
        for (int64_t i = r0 + threadIdx.x; i < r1; i += blockDim.x)
          if (pgb_sub<K>(key[i], q) == round) acc = agg_combine(op, acc, agg_value(A, j, i));
        for (int o = 16; o > 0; o >>= 1) acc = agg_combine(op, acc, __shfl_down_sync(0xffffffffu, acc, o));
        if ((threadIdx.x & 31) == 0) s_red[threadIdx.x >> 5] = acc;
        __syncthreads();
        if (threadIdx.x == 0) {
          int64_t t = s_red[0];
          for (int w = 1; w < kPgbThreads / 32; ++w) t = agg_combine(op, t, s_red[w]);
          if (base < cap) A.out[j][base] = t;
        }
        __syncthreads();
      } else {
        for (int l = threadIdx.x; l < g; l += blockDim.x) s_agg[l] = agg_identity(op);
        __syncthreads();
        for (int64_t i = r0 + threadIdx.x; i < r1; i += blockDim.x) {
          K k = key[i];
          if (pgb_sub<K>(k, q) != round) continue;
          int lid = pgb_lookup<K>(k, pbits, s_slots, s_keys);
          if (lid >= 0) agg_atomic(op, &s_agg[lid], agg_value(A, j, i));
        }
        __syncthreads();
        for (int l = threadIdx.x; l < g; l += blockDim.x)
          if (base + l < cap) A.out[j][base + l] = s_agg[l];
        __syncthreads();
      }
    }
    base += g;
    __syncthreads();
  }
}

// In-place exclusive scan of v[0..n) (n <= 2^20) by one block; v[n] and *total
// receive the sum.
__global__ void __launch_bounds__(1024) excl_scan_kernel(int64_t* v, int64_t n, int64_t* total) {
  __shared__ int64_t s_w[32];
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  const int64_t per = (n + 1023) / 1024;
  const int64_t b = (int64_t)t * per, e = min64(n, b + per);
  int64_t sum = 0;
  for (int64_t i = b; i < e; ++i) sum += v[i];
  int64_t x = sum;
  for (int o = 1; o < 32; o <<= 1) {
    const int64_t y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) s_w[warp] = x;
  __syncthreads();
  if (warp == 0) {
    int64_t w = s_w[lane];
    for (int o = 1; o < 32; o <<= 1) {
      const int64_t y = __shfl_up_sync(0xffffffffu, w, o);
      if (lane >= o) w += y;
    }
    s_w[lane] = w;
  }
  __syncthreads();
  int64_t run = (warp ? s_w[warp - 1] : 0) + x - sum;
  for (int64_t i = b; i < e; ++i) {
    const int64_t c = v[i];
    v[i] = run;
    run += c;
  }
  if (t == 1023) {
    v[n] = run;
    *total = run;
  }
}

template <typename K>
constexpr size_t pgb_smem_bytes() {
  // aggregates, slots, keys by local id, local id by slot
  return (size_t)kPgbCap * 8 + (size_t)kPgbSlots * 4 + (size_t)kPgbCap * sizeof(K) + (size_t)kPgbSlots * 2;
}

// ================================================================ host
Aggs make_aggs(const gj_table* in, int nagg, const int32_t* ops, const int32_t* op_col, int64_t* const* out,
               const void* const* col_src) {
  Aggs A{};
  A.n = nagg;
  for (int j = 0; j < nagg; ++j) {
    A.op[j] = ops[j];
    A.out[j] = out[j];
    if (ops[j] != GJ_AGG_COUNT) {
      A.src[j] = col_src[op_col[j]];
      A.size[j] = dtype_size(in->col_type[op_col[j]]);
    } else {
      A.src[j] = nullptr;
      A.size[j] = 8;
    }
  }
  return A;
}

// The segmented reduction over sorted keys k2 (SGB): tile records, their
// two-level scan, then one walk of the rows; group keys go to out_keys in
// sorted order, aggregates to A.out, the group count to d_ngroups.
template <typename K>
gj_status sgb_reduce_run(const Ctx& ctx, Scratch& scr, const K* k2, int64_t n, const Aggs& A, int nagg,
                         const int32_t* ops, K* out_keys, int64_t cap, int64_t* d_ngroups) {
  cudaStream_t s = ctx.stream;
  const int64_t ntiles = (n + kSegTile - 1) / kSegTile;
  const int64_t nblk = (ntiles + kScanBlock - 1) / kScanBlock;  // <= kScanBlock while n < 2^32
  const int rw = nagg + 2;
  int64_t* rec = scr.get_as<int64_t>((size_t)ntiles * rw);
  int64_t* carry = scr.get_as<int64_t>((size_t)ntiles * rw);
  int64_t* btot = scr.get_as<int64_t>((size_t)nblk * rw);
  int64_t* bcarry = scr.get_as<int64_t>((size_t)nblk * rw);
  if (scr.failed()) return GJ_ERR_OOM;
  const size_t dyn = sizeof(int64_t) * ((size_t)2 * kSegWarps * nagg * 32 + (size_t)2 * kSegWarps * rw);
  gj_status st = ensure_smem_attr(
      ctx, (const void*)sgb_reduce_kernel<K>,
      (int)(sizeof(int64_t) * ((size_t)2 * kSegWarps * kMaxAggs * 32 + 2 * kSegWarps * (kMaxAggs + 2))));
  if (st != GJ_OK) return st;
  // the distinct 4-byte value columns (up to kSegCache) are kept in registers
  SegCols sc{};
  sc.tid = A.tid;
  for (int j = 0; j < nagg; ++j) {
    sc.slot[j] = -1;
    if (ops[j] == GJ_AGG_COUNT || A.size[j] != 4) continue;
    int s2 = -1;
    for (int q = 0; q < sc.n; ++q)
      if (sc.src[q] == A.src[j]) s2 = q;
    if (s2 < 0 && sc.n < kSegCache) {
      s2 = sc.n;
      sc.src[sc.n++] = (const int32_t*)A.src[j];
    }
    sc.slot[j] = (int8_t)s2;
  }
  {
    LaunchScope ls(ctx, KK_SGB_REDUCE);
    sgb_tile_kernel<K><<<(unsigned)ntiles, kSegWarps * 32, 0, s>>>(k2, n, A, sc, rec);
  }
  {
    LaunchScope ls(ctx, KK_SGB_REDUCE);
    sgb_scan_kernel<<<(unsigned)nblk, kScanBlock, 0, s>>>(rec, ntiles, A, carry, btot, nullptr);
  }
  {
    LaunchScope ls(ctx, KK_SGB_REDUCE);
    sgb_scan_kernel<<<1, kScanBlock, 0, s>>>(btot, nblk, A, bcarry, nullptr, d_ngroups);
  }
  LaunchScope ls(ctx, KK_SGB_REDUCE);
  sgb_reduce_kernel<K><<<(unsigned)ntiles, kSegWarps * 32, dyn, s>>>(k2, n, A, sc, out_keys, cap, carry, bcarry,
                                                                     ctx.d_status);
  return cuda_check(cudaGetLastError());
}

// code[i] = the dense group id of row i (HGB stage 1: gid_of_row at the row its key
// was inserted with), the dictionary code SGB-DE sorts.
__global__ void de_codes_kernel(const int32_t* __restrict__ gidloc, const int32_t* __restrict__ gid_of_row, int64_t n,
                                int32_t* __restrict__ code) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
    const int32_t loc = gidloc[i];
    code[i] = loc >= 0 ? gid_of_row[loc] : 0;  // a failed insert has set the status already
  }
}

template <typename K>
gj_status groupby_typed(const Ctx& ctx, const gj_table* in, int nagg, const int32_t* ops, const int32_t* op_col,
                        const gj_options* opt, int variant, void* out_keys, int64_t* const* out_aggs, int64_t cap,
                        int64_t* d_ngroups) {
  cudaStream_t s = ctx.stream;
  Scratch scr(s);
  gj_status st;
  const int64_t n = in->n;
  if ((st = cuda_check(cudaMemsetAsync(d_ngroups, 0, sizeof(int64_t), s))) != GJ_OK) return st;
  if (n == 0) return GJ_OK;

  if (variant == GJ_GB_HGB) {
    uint64_t want = (uint64_t)std::max<int64_t>(2, 2 * (opt->groups_hint > 0 ? std::min(opt->groups_hint, n) : n));
    uint64_t slots = 1;
    while (slots < want) slots <<= 1;
    int32_t* ht = scr.get_as<int32_t>(slots);
    int32_t* gid_of_row = scr.get_as<int32_t>(n);
    int32_t* gidloc = scr.get_as<int32_t>(n);
    if (scr.failed()) return GJ_ERR_OOM;
    if ((st = cuda_check(cudaMemsetAsync(ht, 0, sizeof(int32_t) * slots, s))) != GJ_OK) return st;
    Aggs A = make_aggs(in, nagg, ops, op_col, out_aggs, in->cols);
    {
      LaunchScope ls(ctx, KK_HGB_GROUP_ID);
      int blocks = (int)std::min<int64_t>((n + 255) / 256, (int64_t)ctx.num_sms * 8);
      hgb_group_id_kernel<K><<<blocks, 256, 0, s>>>((const K*)in->key, n, ht, slots - 1, gid_of_row, gidloc,
                                                     (unsigned long long*)d_ngroups, (K*)out_keys, cap,
                                                     ctx.d_status);
    }
    {
      LaunchScope ls(ctx, KK_AGG_INIT);
      agg_init_kernel<<<ctx.num_sms * 4, 256, 0, s>>>(A, d_ngroups, cap);
    }
    SmemAggLayout L{};
    int q = 0;
    for (int pass = 0; pass < 2; ++pass)
      for (int j = 0; j < nagg; ++j) {
        int w = ops[j] == GJ_AGG_SUM ? 8 : (ops[j] == GJ_AGG_COUNT ? 4 : A.size[j]);
        if ((pass == 0) == (w == 8)) {
          L.width[j] = w;
          L.order[q++] = j;
          L.bytes_per_group += w;
        }
      }
    const int budget = ctx.smem_optin - 1024;  // all of an SM's opt-in shared memory for one block
    if ((st = ensure_smem_attr(ctx, (const void*)hgb_agg_kernel, budget)) != GJ_OK) return st;
    {
      LaunchScope ls(ctx, KK_HGB_AGG);
      hgb_agg_kernel<<<ctx.num_sms, 1024, budget, s>>>(gidloc, gid_of_row, n, A, make_col_cache(A), L, d_ngroups,
                                                       cap, budget);
    }
    return cuda_check(cudaGetLastError());
  }

  // ---- SGB-DE (SGB-TR of Sec. 4.1.3 after the dictionary encoding of Sec. 4.4): HGB stage 1 gives every
  // row a dense code and writes the dictionary (code -> key) to out_keys; the
  // codes are then sorted with the values on their ceil(log2 g) bits only and
  // reduced by the SGB kernels, whose segment i is code i. Reading g to size the
  // sort synchronises the stream once.
  if (variant == GJ_GB_SGB_DE) {
    uint64_t want = (uint64_t)std::max<int64_t>(2, 2 * (opt->groups_hint > 0 ? std::min(opt->groups_hint, n) : n));
    uint64_t slots = 1;
    while (slots < want) slots <<= 1;
    int32_t* ht = scr.get_as<int32_t>(slots);
    int32_t* gid_of_row = scr.get_as<int32_t>(n);
    int32_t* gidloc = scr.get_as<int32_t>(n);
    int32_t* code = scr.get_as<int32_t>(n);
    int32_t* code2 = scr.get_as<int32_t>(n);
    int32_t* code_out = scr.get_as<int32_t>(n);  // the reduction's segment codes (0, 1, ...), unused
    if (scr.failed()) return GJ_ERR_OOM;
    if ((st = cuda_check(cudaMemsetAsync(ht, 0, sizeof(int32_t) * slots, s))) != GJ_OK) return st;
    {
      LaunchScope ls(ctx, KK_HGB_GROUP_ID);
      int blocks = (int)std::min<int64_t>((n + 255) / 256, (int64_t)ctx.num_sms * 8);
      hgb_group_id_kernel<K><<<blocks, 256, 0, s>>>((const K*)in->key, n, ht, slots - 1, gid_of_row, gidloc,
                                                     (unsigned long long*)d_ngroups, (K*)out_keys, cap,
                                                     ctx.d_status);
      de_codes_kernel<<<blocks, 256, 0, s>>>(gidloc, gid_of_row, n, code);
    }
    int64_t g = 0;
    if ((st = cuda_check(cudaMemcpyAsync(&g, d_ngroups, sizeof(int64_t), cudaMemcpyDeviceToHost, s))) != GJ_OK)
      return st;
    if ((st = cuda_check(cudaStreamSynchronize(s))) != GJ_OK) return st;
    g = std::min<int64_t>(std::max<int64_t>(g, 1), std::min<int64_t>(n, cap));
    int bits = 1;
    while ((int64_t(1) << bits) < g) ++bits;
    ColSet cs{};
    int colmap[kMaxCols];
    for (int c = 0; c < kMaxCols; ++c) colmap[c] = -1;
    for (int j = 0; j < nagg; ++j) {
      if (ops[j] == GJ_AGG_COUNT || colmap[op_col[j]] >= 0) continue;
      int c = op_col[j];
      colmap[c] = cs.n;
      cs.src[cs.n] = in->cols[c];
      cs.size[cs.n] = dtype_size(in->col_type[c]);
      cs.dst[cs.n] = scr.get((size_t)n * cs.size[cs.n]);
      cs.n++;
    }
    if (scr.failed()) return GJ_ERR_OOM;
    const void* moved[kMaxCols] = {nullptr};
    for (int c = 0; c < kMaxCols; ++c)
      if (colmap[c] >= 0) moved[c] = cs.dst[colmap[c]];
    Aggs A = make_aggs(in, nagg, ops, op_col, out_aggs, moved);
    if ((st = radix_partition_run(ctx, scr, GJ_I32, code, code2, cs, n, 0, bits, kRawBits, opt->bits_per_pass)) !=
        GJ_OK)
      return st;
    return sgb_reduce_run<int32_t>(ctx, scr, code2, n, A, nagg, ops, code_out, cap, d_ngroups);
  }

  // ---- SGB and PGB. TR (GFTR): move the key with every aggregated column; UR
  // (GFUR): move the key with a generated tuple id and read the values through it
  const bool ur = variant == GJ_GB_SGB_UR || variant == GJ_GB_PGB_UR;
  ColSet cs{};
  int colmap[kMaxCols];
  for (int c = 0; c < kMaxCols; ++c) colmap[c] = -1;
  if (ur) {
    cs.n = 1;
    cs.src[0] = nullptr;  // generated tuple ids
    cs.size[0] = 4;
    cs.dst[0] = scr.get((size_t)n * 4);
  } else {
    for (int j = 0; j < nagg; ++j) {
      if (ops[j] == GJ_AGG_COUNT || colmap[op_col[j]] >= 0) continue;
      int c = op_col[j];
      colmap[c] = cs.n;
      cs.src[cs.n] = in->cols[c];
      cs.size[cs.n] = dtype_size(in->col_type[c]);
      cs.dst[cs.n] = scr.get((size_t)n * cs.size[cs.n]);
      cs.n++;
    }
  }
  K* k2 = scr.get_as<K>(n);
  if (scr.failed()) return GJ_ERR_OOM;
  const void* moved[kMaxCols] = {nullptr};
  for (int c = 0; c < kMaxCols; ++c)
    if (colmap[c] >= 0) moved[c] = cs.dst[colmap[c]];
  Aggs A = make_aggs(in, nagg, ops, op_col, out_aggs, ur ? in->cols : moved);
  if (ur) A.tid = (const int32_t*)cs.dst[0];
  const int kbits = sizeof(K) * 8;

  if (variant == GJ_GB_SGB || variant == GJ_GB_SGB_UR) {
    if ((st = radix_partition_run(ctx, scr, sizeof(K) == 8 ? GJ_I64 : GJ_I32, in->key, k2, cs, n, 0, kbits,
                                  kSignedOrder, opt->bits_per_pass)) != GJ_OK)
      return st;
    return sgb_reduce_run<K>(ctx, scr, k2, n, A, nagg, ops, (K*)out_keys, cap, d_ngroups);
  }

  // PGB-TR / PGB-UR: partitions of about 2048 rows on hashed key bits (at most 16 bits)
  int bits = opt->radix_bits > 0 ? std::min(opt->radix_bits, 16) : 0;
  if (opt->radix_bits <= 0)
    while (bits < 16 && (n >> bits) > 2048) ++bits;
  const int64_t nparts = int64_t(1) << bits;
  if (bits > 0) {
    if ((st = radix_partition_run(ctx, scr, sizeof(K) == 8 ? GJ_I64 : GJ_I32, in->key, k2, cs, n, 0, bits, kHashed,
                                  opt->bits_per_pass)) != GJ_OK)
      return st;
  } else {
    if ((st = cuda_check(cudaMemcpyAsync(k2, in->key, sizeof(K) * n, cudaMemcpyDeviceToDevice, s))) != GJ_OK)
      return st;
    if (ur) {
      A.tid = nullptr;  // one partition: rows keep their order
    } else {
      for (int c = 0; c < cs.n; ++c)
        if ((st = cuda_check(cudaMemcpyAsync(cs.dst[c], cs.src[c], (size_t)n * cs.size[c],
                                             cudaMemcpyDeviceToDevice, s))) != GJ_OK)
          return st;
    }
  }
  int64_t* poff = scr.get_as<int64_t>(nparts + 1);
  int64_t* gcount = scr.get_as<int64_t>(nparts + 1);
  int8_t* qsel = scr.get_as<int8_t>(nparts);
  if (scr.failed()) return GJ_ERR_OOM;
  if ((st = partition_bounds_run(ctx, sizeof(K) == 8 ? GJ_I64 : GJ_I32, k2, n, 0, bits, kHashed, poff)) != GJ_OK)
    return st;
  const size_t dyn = pgb_smem_bytes<K>();
  if ((st = ensure_smem_attr(ctx, (const void*)pgb_kernel<K>, (int)dyn)) != GJ_OK) return st;
  const ColCache cc = make_col_cache(A);
  // group counts per partition, their exclusive scan (and g), then the aggregation
  {
    LaunchScope ls(ctx, KK_PGB);
    pgb_kernel<K><<<(unsigned)nparts, kPgbThreads, dyn, s>>>(k2, poff, bits, A, cc, (K*)out_keys, cap, 0, gcount, qsel,
                                                             ctx.d_status);
  }
  {
    LaunchScope ls(ctx, KK_PGB);
    excl_scan_kernel<<<1, 1024, 0, s>>>(gcount, nparts, d_ngroups);
  }
  LaunchScope ls(ctx, KK_PGB);
  pgb_kernel<K><<<(unsigned)nparts, kPgbThreads, dyn, s>>>(k2, poff, bits, A, cc, (K*)out_keys, cap, 1, gcount, qsel,
                                                           ctx.d_status);
  return cuda_check(cudaGetLastError());
}

}  // namespace

int choose_groupby_variant(const gj_table* in, int nagg, const int32_t* ops, const gj_options* opt, int smem_budget) {
  // Fig. groupby-dt without a mandated sort: HGB when the aggregates of the
  // expected groups fit in shared memory, else PGB-TR unless the keys are
  // highly skewed (z >= 1), where the sort-based variant is taken.
  int64_t bytes = 0;
  for (int j = 0; j < nagg; ++j) bytes += (!ops || ops[j] == GJ_AGG_SUM) ? 8 : 4;
  int64_t g = opt->groups_hint > 0 ? opt->groups_hint : in->n;
  if (g * bytes <= smem_budget) return GJ_GB_HGB;
  if (opt->zipf_hint >= 1.0f) return GJ_GB_SGB;
  return GJ_GB_PGB;
}

int resolve_groupby_variant(const gj_table* in, int nagg, const int32_t* ops, const gj_options* opt,
                            int smem_budget) {
  int variant = opt->groupby_variant;
  if (variant == GJ_GB_AUTO && opt->selector == GJ_SELECT_MLP) variant = mlp_choose(nullptr, in, nagg, opt, false, false);
  if (variant == GJ_GB_AUTO) variant = choose_groupby_variant(in, nagg, ops, opt, smem_budget);
  return variant;
}

gj_status groupby_run(const Ctx& ctx, const gj_table* in, int nagg, const int32_t* ops, const int32_t* op_col,
                      const gj_options* opt, void* out_keys, int64_t* const* out_aggs, int64_t cap,
                      int64_t* d_ngroups) {
  const int variant = resolve_groupby_variant(in, nagg, ops, opt, ctx.smem_optin - 1024);
  if (in->key_type == GJ_I64)
    return groupby_typed<int64_t>(ctx, in, nagg, ops, op_col, opt, variant, out_keys, out_aggs, cap, d_ngroups);
  return groupby_typed<int32_t>(ctx, in, nagg, ops, op_col, opt, variant, out_keys, out_aggs, cap, d_ngroups);
}

}  // namespace gj
