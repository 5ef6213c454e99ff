// Internal declarations shared by the CUDA translation units of libgj.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

#include "gj.h"

namespace gj {

constexpr int kMaxCols = GJ_MAX_COLS;
constexpr int kMaxAggs = GJ_MAX_AGGS;
constexpr int64_t kMaxRows = (int64_t(1) << 30) - 1;

// Bounded waits. Every kernel receives its device's status buffer: the status
// word at int [0] and, at bytes 8..15, the wait limit in nanoseconds (0 = the
// default of kDefaultWaitNs). A waiter reads %globaltimer every kWaitPollsPerCheck
// polls and, once the limit has passed since its first poll, records
// GJ_ERR_TIMEOUT and proceeds with what it has, so a kernel always terminates.
constexpr uint64_t kDefaultWaitNs = 2000000000ull;  // 2 s
constexpr uint32_t kWaitPollsPerCheck = 64;
constexpr int kStatusInts = 4;  // ints in a status buffer

// ------------------------------------------------------------------ hashing
// MurmurHash3 fmix32 / fmix64 finalisers (Appleby, public domain): bijective
// mixes; partition digits take the low bits, hash-table slots the bits above.
__host__ __device__ __forceinline__ uint32_t fmix32(uint32_t h) {
  h ^= h >> 16;
  h *= 0x85ebca6bu;
  h ^= h >> 13;
  h *= 0xc2b2ae35u;
  h ^= h >> 16;
  return h;
}
__host__ __device__ __forceinline__ uint64_t fmix64(uint64_t k) {
  k ^= k >> 33;
  k *= 0xff51afd7ed558ccdull;
  k ^= k >> 33;
  k *= 0xc4ceb9fe1a85ec53ull;
  k ^= k >> 33;
  return k;
}

enum KeyTransform { kRawBits = 0, kSignedOrder = 1, kHashed = 2 };

template <typename K>
struct KeyTraits;
template <>
struct KeyTraits<int32_t> {
  using U = uint32_t;
  static constexpr int kBits = 32;
  __host__ __device__ static uint32_t hash(int32_t k) { return fmix32((uint32_t)k); }
  __host__ __device__ static uint64_t hash64(int32_t k) { return fmix32((uint32_t)k); }
};
template <>
struct KeyTraits<int64_t> {
  using U = uint64_t;
  static constexpr int kBits = 64;
  __host__ __device__ static uint64_t hash(int64_t k) { return fmix64((uint64_t)k); }
  __host__ __device__ static uint64_t hash64(int64_t k) { return fmix64((uint64_t)k); }
};

// The bit pattern whose bits [lo, hi) form a key's radix digit.
template <typename K>
__host__ __device__ __forceinline__ typename KeyTraits<K>::U digit_source(K k, int transform) {
  using U = typename KeyTraits<K>::U;
  U u = (U)k;
  if (transform == kSignedOrder) u ^= (U(1) << (KeyTraits<K>::kBits - 1));
  if (transform == kHashed) u = (U)KeyTraits<K>::hash(k);
  return u;
}

template <typename K>
__host__ __device__ __forceinline__ uint32_t extract_digit(K k, int transform, int shift, int width) {
  auto u = digit_source<K>(k, transform);
  return (uint32_t)((u >> shift) & ((typename KeyTraits<K>::U(1) << width) - 1));
}

__host__ __device__ __forceinline__ int64_t min64(int64_t a, int64_t b) { return a < b ? a : b; }
__host__ __device__ __forceinline__ int64_t max64(int64_t a, int64_t b) { return a > b ? a : b; }

// ------------------------------------------------------------------ status
__device__ __forceinline__ void set_status(int* status, int code) { atomicCAS(status, 0, code); }

__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// The clock of one bounded wait. expired() is called once per poll; calls made in
// lockstep by the lanes of a warp see the same poll count, so a warp-wide vote on
// it (__any_sync) keeps the warp's decision uniform.
struct WaitGuard {
  uint64_t start;
  uint64_t limit;
  uint32_t polls;
  // a wait on other blocks: the device's current limit
  __device__ __forceinline__ explicit WaitGuard(const int* status) : start(0), polls(0) {
    const uint64_t l = *(const volatile uint64_t*)(status + 2);
    limit = l ? l : kDefaultWaitNs;
  }
  // a wait with a fixed limit
  __device__ __forceinline__ explicit WaitGuard(uint64_t limit_ns) : start(0), limit(limit_ns), polls(0) {}
  __device__ __forceinline__ bool expired() {
    if ((polls++ % kWaitPollsPerCheck) != 0) return false;
    const uint64_t now = global_ns();
    if (polls == 1) {
      start = now;
      return false;
    }
    return now - start >= limit;
  }
};

// ------------------------------------------------------------------ look-back
// Chained scan across tiles taken in order (decoupled look-back, Merrill &
// Garland 2016). A tile's 64-bit word holds a 2-bit flag in the top bits and a
// 62-bit count: 1 = aggregate of this tile only, 2 = inclusive prefix.
constexpr uint64_t kFlagAgg = 1ull << 62;
constexpr uint64_t kFlagInc = 2ull << 62;
constexpr uint64_t kValMask = (1ull << 62) - 1;

__device__ __forceinline__ uint64_t ld_volatile(const uint64_t* p) { return *(volatile const uint64_t*)p; }
__device__ __forceinline__ void st_volatile(uint64_t* p, uint64_t v) { *(volatile uint64_t*)p = v; }
__device__ __forceinline__ uint32_t ld_volatile32(const uint32_t* p) { return *(volatile const uint32_t*)p; }
__device__ __forceinline__ void st_volatile32(uint32_t* p, uint32_t v) { *(volatile uint32_t*)p = v; }

// Warp-wide look-back: called by all 32 lanes of one warp of tile `tile`. Lanes
// read 32 predecessors per round trip (lane l reads tile base - l), so a chain
// of n aggregate-only predecessors costs n / 32 round trips instead of n.
// Returns the exclusive prefix in every lane and publishes the inclusive value.
__device__ __forceinline__ uint64_t lookback_scan_warp(uint64_t* st, int64_t tile, uint64_t agg, int* status) {
  const int lane = threadIdx.x & 31;
  if (tile == 0) {
    if (lane == 0) st_volatile(&st[0], kFlagInc | agg);
    __syncwarp();
    return 0;
  }
  if (lane == 0) st_volatile(&st[tile], kFlagAgg | agg);
  uint64_t excl = 0;
  int64_t base = tile - 1;
  WaitGuard guard(status);
  bool timed_out = false;
  while (base >= 0) {
    const int64_t idx = base - lane;
    uint64_t w = idx >= 0 ? ld_volatile(&st[idx]) : kFlagInc;
    // every predecessor was taken by a running block: wait until all 32 have a flag
    while (__any_sync(0xffffffffu, (w & ~kValMask) == 0)) {
      if (__any_sync(0xffffffffu, guard.expired())) {  // every lane polls in lockstep: a uniform decision
        timed_out = true;
        break;
      }
      if ((w & ~kValMask) == 0) w = ld_volatile(&st[idx]);
    }
    if (timed_out) {
      if (lane == 0) set_status(status, GJ_ERR_TIMEOUT);
      break;
    }
    const unsigned inc = __ballot_sync(0xffffffffu, (w & ~kValMask) == kFlagInc);
    const int stop = inc ? __ffs(inc) - 1 : 31;  // nearest inclusive predecessor in this window
    uint64_t v = lane <= stop ? (w & kValMask) : 0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    excl += v;
    if (inc) break;
    base -= 32;
  }
  if (lane == 0) st_volatile(&st[tile], kFlagInc | (excl + agg));
  __syncwarp();
  return excl;
}

// Thread 0 waits until the counter *p reaches target (bounded), then the whole
// block proceeds: a task's wait for the tasks it depends on.
__device__ __forceinline__ void block_wait(const unsigned long long* p, unsigned long long target, int* err) {
  if (threadIdx.x == 0) {
    WaitGuard guard(err);
    while (ld_volatile((const uint64_t*)p) < target) {
      if (guard.expired()) {
        set_status(err, GJ_ERR_TIMEOUT);
        break;
      }
      __nanosleep(100);
    }
    __threadfence();
  }
  __syncthreads();
}

// Makes this block's writes visible, then counts its task as done.
__device__ __forceinline__ void block_done(unsigned long long* p) {
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) atomicAdd(p, 1ull);
}

// ------------------------------------------------------------------ bulk copies
// cp.async.bulk global -> shared with completion on an mbarrier (sm_90+). The
// source address, the shared destination and the size must be multiples of 16
// bytes; callers copy the aligned body this way and the ragged end with plain
// loads.
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_fence_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }
// Orders this thread's earlier generic-proxy shared-memory accesses (made visible to
// it by a barrier) before its later bulk-copy writes to the same bytes.
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   smem_u32(dst)),
               "l"(src), "r"(bytes), "r"(smem_u32(bar))
               : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t phase) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(phase)
      : "memory");
  return ok != 0;
}
// Bounded wait for this block's own bulk copies: after kDefaultWaitNs the error is
// recorded and the caller proceeds, so the kernel always ends. The limit is fixed
// (gj_set_wait_limit does not shorten it): a copy still in flight must land
// before its block may use or leave the shared memory it writes, and no working
// copy takes anywhere near that long.
__device__ __forceinline__ void mbar_wait(uint64_t* bar, uint32_t phase, int* err) {
  WaitGuard guard(kDefaultWaitNs);
  while (!mbar_try_wait(bar, phase)) {
    if (guard.expired()) {
      set_status(err, GJ_ERR_TIMEOUT);
      return;
    }
  }
}

// ------------------------------------------------------------------ columns
struct ColSet {
  const void* src[kMaxCols];
  void* dst[kMaxCols];
  int32_t size[kMaxCols];  // bytes per element: 4, 8 or 16
  int32_t n;
  // 1: the four 4-byte source columns are written interleaved, as one 16-byte
  // column at dst[0] (row r's values at dst[0] + 16 r)
  int32_t zip4;
};

__host__ __device__ __forceinline__ int dtype_size(int t) { return t == GJ_I64 ? 8 : 4; }

__device__ __forceinline__ int64_t load_as_i64(const void* p, int size, int64_t i) {
  return size == 8 ? ((const int64_t*)p)[i] : (int64_t)((const int32_t*)p)[i];
}

__device__ __forceinline__ void copy_elem(void* dst, int64_t o, const void* src, int64_t i, int size) {
  if (size == 8)
    ((int64_t*)dst)[o] = ((const int64_t*)src)[i];
  else
    ((int32_t*)dst)[o] = ((const int32_t*)src)[i];
}

// ------------------------------------------------------------------ aggregates
// Reducible aggregates (Sec. 2.2) in int64. SUM wraps in two's complement, so
// every combination order gives the same bits.
struct Aggs {
  int32_t n;
  int32_t op[kMaxAggs];
  const void* src[kMaxAggs];  // value column of aggregate j (unused for COUNT)
  int32_t size[kMaxAggs];     // 4 or 8
  int64_t* out[kMaxAggs];
  // GFUR: row r's values are at src[j][tid[r]] (the rows were moved with their
  // tuple ids only); null: at src[j][r]
  const int32_t* tid;
};

__host__ __device__ __forceinline__ int64_t agg_identity(int op) {
  return op == GJ_AGG_MIN ? INT64_MAX : (op == GJ_AGG_MAX ? INT64_MIN : 0);
}
__device__ __forceinline__ int64_t agg_combine(int op, int64_t a, int64_t b) {
  switch (op) {
    case GJ_AGG_MIN: return a < b ? a : b;
    case GJ_AGG_MAX: return a > b ? a : b;
    default: return (int64_t)((uint64_t)a + (uint64_t)b);
  }
}
// The value row `row` contributes to aggregate j (COUNT contributes 1).
__device__ __forceinline__ int64_t agg_value(const Aggs& A, int j, int64_t row) {
  if (A.op[j] == GJ_AGG_COUNT) return 1;
  return load_as_i64(A.src[j], A.size[j], A.tid ? (int64_t)A.tid[row] : row);
}
__device__ __forceinline__ void agg_atomic(int op, int64_t* p, int64_t v) {
  switch (op) {
    case GJ_AGG_MIN: atomicMin((long long*)p, (long long)v); break;
    case GJ_AGG_MAX: atomicMax((long long*)p, (long long)v); break;
    default: atomicAdd((unsigned long long*)p, (unsigned long long)v); break;
  }
}

// Up to kColCache distinct 4-byte value columns read once per row and shared by
// every aggregate over them: slot[j] is aggregate j's cached column or -1.
constexpr int kColCache = 3;
struct ColCache {
  int32_t n;
  const int32_t* src[kColCache];
  int8_t slot[kMaxAggs];
  const int32_t* tid;  // Aggs::tid
};

inline ColCache make_col_cache(const Aggs& A) {
  ColCache cc{};
  cc.tid = A.tid;
  for (int j = 0; j < A.n; ++j) {
    cc.slot[j] = -1;
    if (A.op[j] == GJ_AGG_COUNT || A.size[j] != 4) continue;
    int s = -1;
    for (int q = 0; q < cc.n; ++q)
      if (cc.src[q] == A.src[j]) s = q;
    if (s < 0 && cc.n < kColCache) {
      s = cc.n;
      cc.src[cc.n++] = (const int32_t*)A.src[j];
    }
    cc.slot[j] = (int8_t)s;
  }
  return cc;
}

// Loads the cached columns of B rows at once (predicated, no early exit, so all
// loads are in flight together).
template <int B>
__device__ __forceinline__ void load_cached(const ColCache& cc, const int64_t (&row)[B], const bool (&valid)[B],
                                            int32_t (&cv)[kColCache][B]) {
  int64_t r[B];
#pragma unroll
  for (int u = 0; u < B; ++u) r[u] = (cc.tid && valid[u] && cc.n > 0) ? (int64_t)__ldcs(cc.tid + row[u]) : row[u];
#pragma unroll
  for (int s = 0; s < kColCache; ++s)
#pragma unroll
    for (int u = 0; u < B; ++u) cv[s][u] = (s < cc.n && valid[u]) ? (cc.tid ? __ldg(cc.src[s] + r[u]) : __ldcs(cc.src[s] + r[u])) : 0;
}

template <int B>
__device__ __forceinline__ int64_t cached_value(const Aggs& A, const ColCache& cc, int j,
                                                const int32_t (&cv)[kColCache][B], int u, int64_t row) {
  if (A.op[j] == GJ_AGG_COUNT) return 1;
  const int s = cc.slot[j];
  if (s == 0) return cv[0][u];
  if (s == 1) return cv[1][u];
  if (s == 2) return cv[2][u];
  return load_as_i64(A.src[j], A.size[j], A.tid ? (int64_t)A.tid[row] : row);
}

// ------------------------------------------------------------------ host side
struct Ctx {
  cudaStream_t stream;
  int* d_status;  // per-device persistent status word
  int num_sms;
  int smem_optin;
  int device;
};

// Stream-ordered scratch allocations released when the object goes away.
class Scratch {
 public:
  explicit Scratch(cudaStream_t s) : stream_(s) {}
  ~Scratch();
  void* get(size_t bytes);  // NULL on failure (sticky failed() flag)
  template <typename T>
  T* get_as(size_t count) {
    return (T*)get(count * sizeof(T));
  }
  bool failed() const { return failed_; }

 private:
  cudaStream_t stream_;
  std::vector<void*> ptrs_;
  bool failed_ = false;
};

gj_status make_ctx(void* stream, Ctx* ctx);

// Raises `func`'s dynamic shared-memory limit to `bytes` on the context's device,
// once per (kernel, device) pair: the attribute belongs to the device context, so
// a process that drives several GPUs sets it on each of them.
gj_status ensure_smem_attr(const Ctx& ctx, const void* func, int bytes);

// Kernel kinds for launch counting and the optional per-kernel event timing.
enum KernelKind {
  KK_RADIX_HIST = 0,
  KK_RADIX_SCATTER,
  KK_PART_BOUNDS,
  KK_PHJ_PROBE,
  KK_NPHJ_BUILD,
  KK_NPHJ_PROBE,
  KK_HGB_GROUP_ID,
  KK_HGB_AGG,
  KK_PGB,
  KK_SGB_REDUCE,
  KK_AGG_INIT,
  KK_FUSED_PROBE,
  KK_GROUP_EMIT,
  KK_BATCH,
  KK_MLP,
  KK_SMJ_MERGE,
  KK_GATHER,
  KK_COUNT
};
// Brackets one kernel launch: counts it and, when timing is on, records CUDA
// events before and after it on the launching stream.
class LaunchScope {
 public:
  LaunchScope(const Ctx& ctx, int kind);
  ~LaunchScope();

 private:
  cudaStream_t stream_;
  int kind_;
  cudaEvent_t start_ = nullptr;
};
gj_status finish(const Ctx& ctx, const gj_options* opt, gj_status st);
gj_status cuda_check(cudaError_t e);

// ------------------------------------------------------------------ radix partition
// Per-pass plan for a stable partition on bits [lo, hi): LSD passes of <= 8 bits.
struct RadixPlan {
  int passes;
  int shift[16];
  int width[16];
};
RadixPlan make_radix_plan(int lo, int hi, int bits_per_pass);

// Partitions key + columns (cols.src -> cols.dst; src NULL with gen_tid set means
// "row index as int32") from kin to kout. Scratch ping-pong buffers come from `scr`.
gj_status radix_partition_run(const Ctx& ctx, Scratch& scr, int key_type, const void* kin, void* kout,
                              const ColSet& cols, int64_t n, int lo, int hi, int transform, int bits_per_pass);

// Partition bounds of already-partitioned keys: off[p] = first row with digit >= p.
gj_status partition_bounds_run(const Ctx& ctx, int key_type, const void* keys, int64_t n, int lo, int width,
                               int transform, int64_t* d_off);

// ------------------------------------------------------------------ operators
gj_status join_run(const Ctx& ctx, const gj_table* R, const gj_table* S, const gj_options* opt, gj_table* T,
                   int64_t cap, int64_t* d_count);
gj_status groupby_run(const Ctx& ctx, const gj_table* in, int nagg, const int32_t* ops, const int32_t* op_col,
                      const gj_options* opt, void* out_keys, int64_t* const* out_aggs, int64_t cap,
                      int64_t* d_ngroups);
gj_status join_groupby_run(const Ctx& ctx, const gj_table* R, const gj_table* S, gj_colref gk, int nagg,
                           const int32_t* ops, const gj_colref* agg_cols, const gj_options* opt, int64_t* out_keys,
                           int64_t* const* out_aggs, int64_t cap, int64_t* d_ngroups);

// The paper's rules (Sec. 7 for the join, Fig. groupby-dt for the group-by).
int heuristic_join_variant(const gj_table* R, const gj_options* opt);
int choose_groupby_variant(const gj_table* in, int nagg, const int32_t* ops, const gj_options* opt, int smem_budget);

// Learned selector: raw query features, and the network's choice (0 = no network).
// `fused` restricts a join choice to the variants the join -> group-by call runs
// (PHJ-TR, PHJ-UR, NPHJ).
void query_features(const gj_table* R, const gj_table* S, int nagg, const gj_options* opt, float* f);
int mlp_choose(const gj_table* R, const gj_table* S, int nagg, const gj_options* opt, bool join, bool fused);

// The GB300-calibrated cost model's choice (argmin of gj_cost_estimate; `fused`
// as for mlp_choose).
int cost_join_variant(const gj_table* R, const gj_table* S, const gj_options* opt, bool fused);
int cost_groupby_variant(const gj_table* in, int nagg, const int32_t* ops, const gj_options* opt);

// The variants an AUTO request runs: the trained network's choice when
// options.selector is GJ_SELECT_MLP and a network is installed, the paper's rules
// under GJ_SELECT_HEURISTIC, else the cost model; an explicit variant is returned
// unchanged.
int resolve_join_variant(const gj_table* R, const gj_table* S, int nagg, const gj_options* opt, bool fused);
int resolve_groupby_variant(const gj_table* in, int nagg, const int32_t* ops, const gj_options* opt,
                            int smem_budget);

// Total partition bits for a build side of nr rows so that a partition holds
// about `target` rows; at most 16 bits (two passes of 8).
int choose_join_bits(int64_t nr, int64_t target);

}  // namespace gj
