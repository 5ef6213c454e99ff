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
// The dictionary (Alg. 1, stage 1): a global open-addressing table of entries
// (key, g). g = 0 marks an empty slot; kClaim | (row + 1) a slot claimed by the
// row that is inserting its key; otherwise g - 1 is the key's dense group id,
// taken from the group counter by the inserting row, which also writes the
// output key. Stage 2 finds a row's id by looking its key up in this table.
constexpr uint32_t kClaim = 0x80000000u;

template <typename K>
struct alignas(2 * sizeof(K)) HEntry {
  K key;
  uint32_t g;
};

__device__ __forceinline__ uint32_t ld_acquire_u32(const uint32_t* p) {
  uint32_t v;
  asm volatile("ld.acquire.gpu.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_release_u32(uint32_t* p, uint32_t v) {
  asm volatile("st.release.gpu.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Inserts the key k of row i unless the table holds it already.
template <typename K>
__device__ __forceinline__ void hgb_insert(const K* __restrict__ key, HEntry<K>* ht, uint64_t mask, K k, int64_t i,
                                           unsigned long long* ngroups, K* __restrict__ out_keys, int64_t cap,
                                           int* err) {
  uint64_t sl = KeyTraits<K>::hash64(k) & mask;
  for (uint64_t probe = 0; probe <= mask;) {
    const uint32_t w = ld_acquire_u32(&ht[sl].g);
    if (w == 0) {
      if (atomicCAS(&ht[sl].g, 0u, kClaim | (uint32_t)(i + 1)) == 0u) {
        ht[sl].key = k;
        const unsigned long long gid = atomicAdd(ngroups, 1ull);
        if ((int64_t)gid < cap)
          out_keys[gid] = k;
        else
          set_status(err, GJ_ERR_CAPACITY);
        st_release_u32(&ht[sl].g, (uint32_t)gid + 1u);  // the key is written before the id is published
        return;
      }
      continue;  // another row claimed the slot first: read it again
    }
    const K other = (w & kClaim) ? key[(w & ~kClaim) - 1] : ht[sl].key;
    if (other == k) return;
    sl = (sl + 1) & mask;
    ++probe;
  }
  set_status(err, GJ_ERR_CAPACITY);  // the table is full
}

// Dense group id of key k, or -1 if the table does not hold it. Called after the
// dictionary kernel has finished, when every entry is final.
template <typename K>
__device__ __forceinline__ int32_t hgb_find(const HEntry<K>* __restrict__ ht, uint64_t mask, K k) {
  uint64_t sl = KeyTraits<K>::hash64(k) & mask;
  for (uint64_t probe = 0; probe <= mask; ++probe) {
    const HEntry<K> e = ht[sl];
    if (e.g == 0) return -1;
    if (e.key == k) return (int32_t)(e.g - 1);
    sl = (sl + 1) & mask;
  }
  return -1;
}

// Keys a block has already inserted or found: a shared-memory set of tagged keys,
// so that a key repeated across the block's rows reaches the global table once per
// block. 4-byte keys are tagged with bit 32 (empty = 0); 8-byte keys are stored as
// they are (empty = INT64_MIN, a key of that value is simply never cached).
constexpr int kSeenSlots = 16384;  // 192 KB with the rows: one 1024-thread block per SM
// Probes of the set per key: when the expected groups fit in half the set, every
// distinct key of a block must find a slot, or each of its rows goes to the global
// table (4 probes left a few percent of 4096 keys uncached and made the pass 7x
// slower); when they do not, the set caches only some keys and a key absent from
// it is looked for briefly (long probe runs of one lane stall its whole warp:
// 32 probes made the 2^20-group pass 1.8x slower).
constexpr int kSeenProbesFit = 32;
constexpr int kSeenProbesSome = 4;
template <typename K>
__device__ __forceinline__ unsigned long long seen_tag(K k) {
  return sizeof(K) == 4 ? ((1ull << 32) | (uint64_t)(uint32_t)k) : (unsigned long long)(int64_t)k;
}
template <typename K>
__device__ __forceinline__ unsigned long long seen_empty() {
  return sizeof(K) == 4 ? 0ull : 0x8000000000000000ull;
}

// Stage 1: build the dictionary. Writes nothing per row. A block first only
// collects its distinct keys in the shared-memory set (with one row holding each,
// which the global insert needs); keys that do not fit the set go to the global
// table at once. At the end all threads of the block insert the collected keys
// together, so the global round trips run in full warps rather than one diverged
// lane at a time.
template <typename K, int kProbes>
__global__ void __launch_bounds__(1024, 1) hgb_dict_kernel(const K* __restrict__ key, int64_t n, HEntry<K>* ht,
                                                       uint64_t mask, unsigned long long* ngroups,
                                                       K* __restrict__ out_keys, int64_t cap, const int* gate,
                                                       int* err) {
  if (gate && *gate == 0) return;  // the few-groups pass has produced the result
  extern __shared__ unsigned long long s_seen[];  // kSeenSlots tags, then kSeenSlots rows (int32)
  int32_t* s_row = reinterpret_cast<int32_t*>(s_seen + kSeenSlots);
  __shared__ int s_fill;  // keys cached; new keys stop being cached at half load
  const unsigned long long empty = seen_empty<K>();
  for (int j = threadIdx.x; j < kSeenSlots; j += blockDim.x) s_seen[j] = empty;
  if (threadIdx.x == 0) s_fill = 0;
  __syncthreads();
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  constexpr int kBatch = 4;  // rows per thread per step: their key loads are in flight together
  for (int64_t it = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; it < n; it += stride * kBatch) {
    K kk[kBatch];
#pragma unroll
    for (int u = 0; u < kBatch; ++u) {
      const int64_t i = it + u * stride;
      kk[u] = i < n ? __ldcs(key + i) : K(0);
    }
#pragma unroll
    for (int u = 0; u < kBatch; ++u) {
      const int64_t i = it + u * stride;
      if (i >= n) continue;
      const unsigned long long tag = seen_tag<K>(kk[u]);
      bool handled = false;
      if (tag != empty) {
        uint32_t sl = (uint32_t)KeyTraits<K>::hash64(kk[u]) & (kSeenSlots - 1);
        for (int p = 0; p < kProbes; ++p) {
          unsigned long long v = s_seen[sl];
          if (v == empty) {
            if (*(volatile int*)&s_fill >= kSeenSlots / 2) break;  // full enough: look up only
            v = atomicCAS(&s_seen[sl], empty, tag);
            if (v == empty) {
              s_row[sl] = (int32_t)i;  // inserted into the global table at the end
              atomicAdd(&s_fill, 1);
              handled = true;
              break;
            }
          }
          if (v == tag) {
            handled = true;  // collected already
            break;
          }
          sl = (sl + 1) & (kSeenSlots - 1);
        }
      }
      if (!handled) hgb_insert<K>(key, ht, mask, kk[u], i, ngroups, out_keys, cap, err);
    }
  }
  __syncthreads();
  for (int j = threadIdx.x; j < kSeenSlots; j += blockDim.x) {
    const unsigned long long tag = s_seen[j];
    if (tag == empty) continue;
    const K k = sizeof(K) == 4 ? (K)(int32_t)(uint32_t)tag : (K)(int64_t)tag;
    hgb_insert<K>(key, ht, mask, k, s_row[j], ngroups, out_keys, cap, err);
  }
}

// code[i] = the dense group id of row i: the dictionary code SGB-DE sorts.
template <typename K>
__global__ void hgb_codes_kernel(const K* __restrict__ key, int64_t n, const HEntry<K>* __restrict__ ht,
                                 uint64_t mask, int32_t* __restrict__ code, int* err) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
    const int32_t g = hgb_find<K>(ht, mask, __ldcs(key + i));
    if (g < 0) set_status(err, GJ_ERR_CAPACITY);  // its insert failed and was reported
    code[i] = g < 0 ? 0 : g;
  }
}

// out[j][0..g) = the starting value of aggregate j, g read from the device
// counter. MIN/MAX over a 4-byte column start at the 32-bit identity
// (INT32_MAX / INT32_MIN): every group holds at least one row, whose value fits
// 32 bits, so the result is unchanged, and a block's shared-memory slot still at
// that identity has nothing to add (it may hold a real INT32_MAX, which then is
// already the starting value).
__global__ void agg_init_kernel(Aggs A, const int64_t* __restrict__ ngroups, int64_t cap, const int* gate) {
  if (gate && *gate == 0) return;
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

// Starting value of a slot (zero for both SUM forms).
__device__ __forceinline__ void smem_init(int op, int width, unsigned char* slot) {
  if (width == 8)
    *(int64_t*)slot = agg_identity(op);
  else if (op == GJ_AGG_COUNT)
    *(unsigned int*)slot = 0u;
  else
    *(int*)slot = op == GJ_AGG_MIN ? INT32_MAX : INT32_MIN;
}

// Slot forms of an aggregate in shared memory: 32-bit (COUNT; MIN/MAX over a
// 4-byte column), int64, or a SUM split over two 32-bit words that add the
// value's low 16 bits (unsigned) and high 16 bits (signed) separately.
// Shared-memory 64-bit additions run as compare-and-swap loops that collapse
// when many lanes hit one slot, while 32-bit atomics are resolved in hardware;
// the split form is exact while a slot takes at most kSplitRows values (its
// words stay below 2^32 and 2^31), after which it is folded away.
enum SlotForm { kSlot32 = 0, kSlot64 = 1, kSlotSplit = 2 };

// One aggregate with its operation, value source (a cached 4-byte column 0..2, or
// -1: COUNT, or a column read through Aggs) and slot form fixed at compile time,
// so the per-row update is a handful of instructions.
template <int OP, int SRC, int FORM>
struct SlotUpd {
  static constexpr int kWidth = FORM == kSlot32 ? 4 : 8;
  template <int B>
  static __device__ __forceinline__ int64_t value(const Aggs& A, int j, const int32_t (&cv)[kColCache][B], int u,
                                                  int64_t row) {
    if (OP == GJ_AGG_COUNT) return 1;
    if (SRC >= 0) return cv[SRC][u];
    return load_as_i64(A.src[j], A.size[j], A.tid ? (int64_t)A.tid[row] : row);
  }
  static __device__ __forceinline__ void apply(unsigned char* slot, int64_t v) {
    if (FORM == kSlotSplit) {
      atomicAdd((unsigned int*)slot, (unsigned int)(v & 0xffff));
      atomicAdd((int*)slot + 1, (int)(v >> 16));
    } else if (FORM == kSlot64) {
      agg_atomic(OP, (int64_t*)slot, v);
    } else if (OP == GJ_AGG_COUNT) {
      atomicAdd((unsigned int*)slot, 1u);
    } else if (OP == GJ_AGG_MIN) {
      atomicMin((int*)slot, (int)v);
    } else {
      atomicMax((int*)slot, (int)v);
    }
  }
};

__host__ __device__ __forceinline__ int slot_code(int op, int src, int form) { return op * 16 + (src + 1) * 4 + form; }

// The form and dispatch code of aggregate j: split SUMs need a cached 4-byte column.
__device__ __forceinline__ int slot_form(const Aggs& A, const ColCache& cc, int j, bool split) {
  const int op = A.op[j];
  if (op == GJ_AGG_COUNT) return kSlot32;
  if (op == GJ_AGG_SUM) return split && cc.slot[j] >= 0 ? kSlotSplit : kSlot64;
  return A.size[j] == 4 ? kSlot32 : kSlot64;
}

// Calls f(SlotUpd<...>{}) for a code made by slot_code (a switch over the 18
// combinations that occur).
template <typename F>
__device__ __forceinline__ void slot_dispatch(int code, F&& f) {
#define GJ_UPD_CASE(OP, SRC, FORM) \
  case (OP) * 16 + ((SRC) + 1) * 4 + (FORM): f(SlotUpd<OP, SRC, FORM>{}); return;
  switch (code) {
    GJ_UPD_CASE(GJ_AGG_COUNT, -1, kSlot32)
    GJ_UPD_CASE(GJ_AGG_SUM, 0, kSlot64)
    GJ_UPD_CASE(GJ_AGG_SUM, 1, kSlot64)
    GJ_UPD_CASE(GJ_AGG_SUM, 2, kSlot64)
    GJ_UPD_CASE(GJ_AGG_SUM, -1, kSlot64)
    GJ_UPD_CASE(GJ_AGG_SUM, 0, kSlotSplit)
    GJ_UPD_CASE(GJ_AGG_SUM, 1, kSlotSplit)
    GJ_UPD_CASE(GJ_AGG_SUM, 2, kSlotSplit)
    GJ_UPD_CASE(GJ_AGG_MIN, 0, kSlot32)
    GJ_UPD_CASE(GJ_AGG_MIN, 1, kSlot32)
    GJ_UPD_CASE(GJ_AGG_MIN, 2, kSlot32)
    GJ_UPD_CASE(GJ_AGG_MIN, -1, kSlot32)
    GJ_UPD_CASE(GJ_AGG_MIN, -1, kSlot64)
    GJ_UPD_CASE(GJ_AGG_MAX, 0, kSlot32)
    GJ_UPD_CASE(GJ_AGG_MAX, 1, kSlot32)
    GJ_UPD_CASE(GJ_AGG_MAX, 2, kSlot32)
    GJ_UPD_CASE(GJ_AGG_MAX, -1, kSlot32)
    GJ_UPD_CASE(GJ_AGG_MAX, -1, kSlot64)
    default: return;
  }
#undef GJ_UPD_CASE
}

// Value of a slot of the given form.
__device__ __forceinline__ int64_t slot_read(int op, int form, const unsigned char* p) {
  if (form == kSlotSplit) return (int64_t)(*((const int*)p + 1)) * 65536 + (int64_t)(*(const unsigned int*)p);
  if (form == kSlot64) return *(const int64_t*)p;
  if (op == GJ_AGG_COUNT) return (int64_t) * (const unsigned int*)p;
  return (int64_t) * (const int*)p;
}

// Rows a split SUM slot may take before its 32-bit words are folded away.
constexpr int64_t kSplitRows = 65535;

// Stage 2: every row's group id from the dictionary, then its aggregates. When
// the g groups' slots fit in shared memory (is_smem_enough, decided here on the
// device from the group counter) each block aggregates into shared memory --
// one copy per warp, or per few warps, when several copies fit, so warps do not
// contend for the same slots -- and adds its slots into the result at the end;
// otherwise rows are aggregated straight into the result with global atomics.
template <typename K>
__global__ void __launch_bounds__(1024, 1) hgb_aggregate_kernel(const K* __restrict__ key, int64_t n,
                                                                const HEntry<K>* __restrict__ ht, uint64_t mask,
                                                                Aggs A, ColCache cc, SmemAggLayout L,
                                                                const int64_t* __restrict__ ngroups, int64_t cap,
                                                                int smem_budget, const int* gate, int* err) {
  if (gate && *gate == 0) return;
  extern __shared__ __align__(16) unsigned char s_agg[];
  __shared__ int64_t offs[kMaxAggs];  // aggregate j's slot array within a copy
  __shared__ int s_code[kMaxAggs];
  const int64_t g = min64(*ngroups, cap);
  const int64_t copy_bytes = (g * (int64_t)L.bytes_per_group + 15) & ~int64_t(15);
  const bool use_smem = copy_bytes <= smem_budget;  // is_smem_enough
  const int nwarps = blockDim.x >> 5;
  int ncopy = 1;
  while (use_smem && ncopy < nwarps && 2 * ncopy * copy_bytes <= smem_budget) ncopy *= 2;
  const int warp = threadIdx.x >> 5;
  // split SUMs (32-bit atomics only) whenever the slots are in shared memory,
  // folded into the result every epoch: a copy takes at most (nwarps / ncopy) * 32 *
  // kBatch rows per step
  constexpr int kBatch = 4;  // rows per thread per step: loads and lookups of the batch overlap
  const bool split = use_smem;
  const int epoch_steps = (int)(kSplitRows / ((nwarps / ncopy) * 32 * kBatch));
  if (threadIdx.x == 0) {
    int64_t o = 0;
    for (int q = 0; q < A.n; ++q) {
      const int j = L.order[q];
      offs[j] = o;
      o += g * L.width[j];
    }
  }
  if (threadIdx.x < A.n) {
    const int j = threadIdx.x;
    s_code[j] = slot_code(A.op[j], A.op[j] == GJ_AGG_COUNT ? -1 : cc.slot[j], slot_form(A, cc, j, split));
  }
  __syncthreads();
  if (use_smem) {
    for (int c = 0; c < ncopy; ++c)
      for (int q = 0; q < A.n; ++q) {
        const int j = L.order[q];
        for (int64_t s = threadIdx.x; s < g; s += blockDim.x)
          smem_init(A.op[j], L.width[j], s_agg + c * copy_bytes + offs[j] + s * L.width[j]);
      }
    __syncthreads();
  }
  // adds the split SUM words of every copy into the result and clears them
  auto fold_split = [&]() {
    for (int j = 0; j < A.n; ++j) {
      if ((s_code[j] & 3) != kSlotSplit) continue;
      for (int64_t s = threadIdx.x; s < g; s += blockDim.x) {
        int64_t v = 0;
        for (int c = 0; c < ncopy; ++c) {
          unsigned char* p = s_agg + c * copy_bytes + offs[j] + s * 8;
          v += slot_read(GJ_AGG_SUM, kSlotSplit, p);
          *(int64_t*)p = 0;
        }
        if (v != 0) agg_atomic(GJ_AGG_SUM, &A.out[j][s], v);
      }
    }
  };
  unsigned char* mine = s_agg + (warp & (ncopy - 1)) * copy_bytes;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  bool lost = false;
  int step = 0;
  // the loop bound is the block's first row: every thread runs the same steps
  for (int64_t it = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; it - threadIdx.x < n; it += stride * kBatch) {
    int64_t row[kBatch];
    bool valid[kBatch];
    K kk[kBatch];
#pragma unroll
    for (int u = 0; u < kBatch; ++u) {
      row[u] = it + u * stride;
      valid[u] = row[u] < n;
      kk[u] = valid[u] ? __ldcs(key + row[u]) : K(0);
    }
    int32_t gid[kBatch];
#pragma unroll
    for (int u = 0; u < kBatch; ++u) gid[u] = valid[u] ? hgb_find<K>(ht, mask, kk[u]) : -1;
    int32_t cv[kColCache][kBatch];
    load_cached<kBatch>(cc, row, valid, cv);
    bool ok[kBatch];
#pragma unroll
    for (int u = 0; u < kBatch; ++u) {
      lost |= valid[u] && gid[u] < 0;
      ok[u] = valid[u] && gid[u] >= 0 && gid[u] < g;
    }
    for (int j = 0; j < A.n; ++j) {
      unsigned char* base = mine + offs[j];
      int64_t* gout = A.out[j];
      slot_dispatch(s_code[j], [&](auto U) {
        using Up = decltype(U);
#pragma unroll
        for (int u = 0; u < kBatch; ++u) {
          if (!ok[u]) continue;
          const int64_t v = Up::template value<kBatch>(A, j, cv, u, row[u]);
          if (use_smem)
            Up::apply(base + (int64_t)gid[u] * Up::kWidth, v);
          else
            agg_atomic(A.op[j], &gout[gid[u]], v);
        }
      });
    }
    if (split && ++step == epoch_steps) {
      step = 0;
      __syncthreads();
      fold_split();
      __syncthreads();
    }
  }
  if (lost) set_status(err, GJ_ERR_CAPACITY);  // a key whose insert failed (reported by stage 1)
  if (!use_smem) return;
  __syncthreads();
  if (split) fold_split();
  for (int j = 0; j < A.n; ++j) {
    const int op = A.op[j], w = L.width[j], form = s_code[j] & 3;
    if (form == kSlotSplit) continue;
    const int64_t idv = agg_identity(op);
    for (int64_t s = threadIdx.x; s < g; s += blockDim.x) {
      int64_t v = slot_read(op, form, s_agg + offs[j] + s * w);
      for (int c = 1; c < ncopy; ++c) v = agg_combine(op, v, slot_read(op, form, s_agg + c * copy_bytes + offs[j] + s * w));
      if (w == 4 && op == GJ_AGG_MIN && v == INT32_MAX) continue;
      if (w == 4 && op == GJ_AGG_MAX && v == INT32_MIN) continue;
      if (v == idv) continue;
      agg_atomic(op, &A.out[j][s], v);
    }
  }
}

// ---------------------------------------------------------------- HGB, few groups
// When the groups hint says at most 32 groups, a single pass aggregates without
// the dictionary pass and without atomics: each block keeps a 64-slot
// shared-memory table of the keys it has seen (tagged 64-bit words, at most 32
// keys), and every warp keeps, per slot, the COUNT and the SUM/MIN/MAX of each
// cached 4-byte value column in registers -- lane l owns slots l and l + 32.
// In a warp step (one row per lane) lane l finds the lanes whose row is in its
// slot from six ballots on the slot number and pulls their values with
// shuffles. Blocks leave their per-slot results in scratch; one block merges
// them into the dense result (at most kTinyMerge groups). A block that meets a
// 33rd key, or a merge that meets too many, sets `overflow` and the general
// HGB kernels, which test it, run instead.
constexpr int kTinySlots = 64;
constexpr int kTinyKeys = 32;
constexpr int kTinyMerge = 1024;

struct TinyPart {  // one slot of one block: its key tag and the per-column results
  unsigned long long tag;
  unsigned int count;
  int32_t pad;
  int64_t sum[kColCache];
  int32_t mn[kColCache];
  int32_t mx[kColCache];
};

template <typename K>
__global__ void __launch_bounds__(1024, 1) hgb_tiny_kernel(const K* __restrict__ key, int64_t n, ColCache cc,
                                                           TinyPart* __restrict__ parts, int* overflow) {
  __shared__ unsigned long long s_tab[kTinySlots];
  __shared__ int s_nkeys;
  __shared__ unsigned int s_cnt[kTinySlots];
  __shared__ long long s_sum[kColCache][kTinySlots];
  __shared__ int s_mn[kColCache][kTinySlots];
  __shared__ int s_mx[kColCache][kTinySlots];
  const unsigned long long empty = seen_empty<K>();
  const int tid = threadIdx.x, lane = tid & 31;
  if (tid < kTinySlots) {
    s_tab[tid] = empty;
    s_cnt[tid] = 0;
    for (int c = 0; c < kColCache; ++c) {
      s_sum[c][tid] = 0;
      s_mn[c][tid] = INT32_MAX;
      s_mx[c][tid] = INT32_MIN;
    }
  }
  if (tid == 0) s_nkeys = 0;
  __syncthreads();
  // lane-owned results of slots lane and lane + 32
  unsigned int cnt[2] = {0u, 0u};
  int64_t sum[2][kColCache];
  int32_t mn[2][kColCache], mx[2][kColCache];
#pragma unroll
  for (int h = 0; h < 2; ++h)
#pragma unroll
    for (int c = 0; c < kColCache; ++c) {
      sum[h][c] = 0;
      mn[h][c] = INT32_MAX;
      mx[h][c] = INT32_MIN;
    }
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  bool bail = false, stop = false;
  // kTB rows per thread per step, their loads in flight together; the loop bound is
  // the warp's first row, so the lanes of a warp run the same steps (no block
  // barrier inside the loop: a warp that meets too many keys stops on its own)
  constexpr int kTB = 2;
  for (int64_t i0 = (int64_t)blockIdx.x * blockDim.x + tid; i0 - lane < n && !stop; i0 += stride * kTB) {
    K kk[kTB];
    int32_t v[kTB][kColCache];
    bool valid[kTB];
#pragma unroll
    for (int u = 0; u < kTB; ++u) {
      const int64_t i = i0 + u * stride;
      valid[u] = i < n;
      kk[u] = valid[u] ? __ldcs(key + i) : K(0);
#pragma unroll
      for (int c = 0; c < kColCache; ++c) v[u][c] = (valid[u] && c < cc.n) ? __ldcs(cc.src[c] + i) : 0;
    }
#pragma unroll
    for (int u = 0; u < kTB; ++u) {
      int slot = -1;
      if (valid[u]) {
        const unsigned long long tag = seen_tag<K>(kk[u]);
        if (tag != empty) {
          uint32_t sl = (uint32_t)KeyTraits<K>::hash64(kk[u]) & (kTinySlots - 1);
          for (int p = 0; p < kTinySlots; ++p) {
            unsigned long long w = ((volatile unsigned long long*)s_tab)[sl];
            if (w == empty) {
              w = atomicCAS(&s_tab[sl], empty, tag);
              if (w == empty) {
                if (atomicAdd(&s_nkeys, 1) >= kTinyKeys) bail = true;
                slot = (int)sl;
                break;
              }
            }
            if (w == tag) {
              slot = (int)sl;
              break;
            }
            sl = (sl + 1) & (kTinySlots - 1);
          }
        }
        if (slot < 0) bail = true;  // INT64_MIN as an 8-byte key, or a full table
      }
      if (__any_sync(0xffffffffu, bail)) {  // too many keys for this path
        stop = true;
        break;
      }
      // the lanes whose row is in slot lane (h = 0) and slot lane + 32 (h = 1)
      unsigned m0 = __ballot_sync(0xffffffffu, slot >= 0), m1 = m0;
#pragma unroll
      for (int b = 0; b < 5; ++b) {
        const unsigned bb = __ballot_sync(0xffffffffu, (slot >> b) & 1);
        const unsigned sel = ((lane >> b) & 1) ? bb : ~bb;
        m0 &= sel;
        m1 &= sel;
      }
      const unsigned b5 = __ballot_sync(0xffffffffu, (slot >> 5) & 1);
      m0 &= ~b5;
      m1 &= b5;
      cnt[0] += __popc(m0);
      cnt[1] += __popc(m1);
      const int rounds = __reduce_max_sync(0xffffffffu, (unsigned)max(__popc(m0), __popc(m1)));
      for (int r = 0; r < rounds; ++r) {
        const int s0 = m0 ? __ffs(m0) - 1 : lane, s1 = m1 ? __ffs(m1) - 1 : lane;
#pragma unroll
        for (int c = 0; c < kColCache; ++c) {
          const int32_t x0 = __shfl_sync(0xffffffffu, v[u][c], s0), x1 = __shfl_sync(0xffffffffu, v[u][c], s1);
          if (m0) {
            sum[0][c] += x0;
            mn[0][c] = min(mn[0][c], x0);
            mx[0][c] = max(mx[0][c], x0);
          }
          if (m1) {
            sum[1][c] += x1;
            mn[1][c] = min(mn[1][c], x1);
            mx[1][c] = max(mx[1][c], x1);
          }
        }
        m0 &= m0 - 1;
        m1 &= m1 - 1;
      }
    }
  }
  // every warp has left the loop before the key count is read
  const bool any_bail = __syncthreads_or(bail);
  if (any_bail || s_nkeys > kTinyKeys) {
    if (tid == 0) atomicExch(overflow, 1);
    return;
  }
  // the warps' results into the block's slots, then the block's slots out
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    const int sl = lane + 32 * h;
    if (cnt[h] == 0) continue;
    atomicAdd(&s_cnt[sl], cnt[h]);
#pragma unroll
    for (int c = 0; c < kColCache; ++c) {
      atomicAdd((unsigned long long*)&s_sum[c][sl], (unsigned long long)sum[h][c]);
      atomicMin(&s_mn[c][sl], mn[h][c]);
      atomicMax(&s_mx[c][sl], mx[h][c]);
    }
  }
  __syncthreads();
  if (tid < kTinySlots) {
    TinyPart t{};
    t.tag = s_cnt[tid] ? s_tab[tid] : empty;
    t.count = s_cnt[tid];
    for (int c = 0; c < kColCache; ++c) {
      t.sum[c] = s_sum[c][tid];
      t.mn[c] = s_mn[c][tid];
      t.mx[c] = s_mx[c][tid];
    }
    parts[(int64_t)blockIdx.x * kTinySlots + tid] = t;
  }
}

// ---------------------------------------------------------------- HGB, at most 16 groups
// When the groups hint says at most kFewKeys groups, each block counting-sorts
// every tile of kFewTile rows by local group id in shared memory and reduces the
// runs. Keys get local ids 0..15 from the block's 64-slot table of tagged keys;
// keys enter it only in insertion phases between block barriers, taken when some
// thread meets a key the table lacks, so the lookups in between read a table that
// nothing writes. Per tile:
//  A. every row's id; four ballots on its bits give each row its rank among the
//     warp's rows of its group, and one shared-memory atomic per group and warp
//     reserves the warp's places in that group's run;
//  B. the groups' sizes become run offsets (and are added to the groups' COUNTs);
//  C. every row's cached values go to their places;
//  D. one warp per group walks its run and folds it into registers: per lane the
//     64-bit SUM, the MIN and the MAX of each column for that group.
// No update of a result conflicts with another and no work crosses lanes except
// the ballots and shuffles of the ranking. The tiles' key and value columns reach
// shared memory by bulk copies kFewStages - 1 tiles ahead of their use (one thread
// refills a stage once the block has read it); the ragged last tile, and inputs
// whose columns do not start on 16 bytes, are read with plain loads. Two blocks
// share an SM, so that one block's work overlaps the other's barriers. At the end
// each warp reduces its lanes and the block leaves one TinyPart per id for the
// merge kernel. A 17th key in a block, or a key equal to the empty tag, sets
// `overflow`, and the general HGB kernels run instead.
constexpr int kFewKeys = 16;
constexpr int kFewThreads = 512;
constexpr int kFewRows = 4;  // rows per thread per tile
constexpr int kFewTile = kFewThreads * kFewRows;
constexpr int kFewStages = 2;  // two blocks per SM must fit: 2 x (2 stages + the sorted tile)
template <typename K, int NC>
constexpr int few_stage_bytes() {
  return kFewTile * (int)sizeof(K) + NC * kFewTile * 4;
}
static_assert(kFewKeys == 16 && kFewThreads == 32 * kFewKeys, "four ballots address the ids; one warp per group");

// Local id of `tag` in the block's table, or -1 when it is absent.
__device__ __forceinline__ int few_find(const unsigned long long* s_tab, const int* s_lid, unsigned long long tag,
                                        unsigned long long empty) {
  uint32_t sl = (uint32_t)((tag * 0x9e3779b97f4a7c15ull) >> 58);
  for (int p = 0; p < kTinySlots; ++p) {
    const unsigned long long w = s_tab[sl];
    if (w == tag) return s_lid[sl];
    if (w == empty) return -1;
    sl = (sl + 1) & (kTinySlots - 1);
  }
  return -1;
}

// Keys and cached columns of this thread's rows of tile t (rows past n read nothing).
template <typename K, int NV>
__device__ __forceinline__ void few_load(const K* __restrict__ key, const ColCache& cc, int64_t n, int64_t t,
                                         K (&kk)[kFewRows], int32_t (&v)[NV][kFewRows]) {
  const int64_t base = t * kFewTile + threadIdx.x;
#pragma unroll
  for (int u = 0; u < kFewRows; ++u) {
    const int64_t i = base + (int64_t)u * kFewThreads;
    const bool ok = i < n;
    kk[u] = ok ? __ldcs(key + i) : K(0);
#pragma unroll
    for (int c = 0; c < NV; ++c) v[c][u] = (ok && c < cc.n) ? __ldcs(cc.src[c] + i) : 0;
  }
}

template <typename K, int NC>
__global__ void __launch_bounds__(kFewThreads, 2) hgb_few_kernel(const K* __restrict__ key, int64_t n, ColCache cc,
                                                                 TinyPart* __restrict__ parts, int* overflow,
                                                                 bool bulk, int* err) {
  constexpr int NV = NC > 0 ? NC : 1;
  constexpr unsigned F = 0xffffffffu;
  constexpr int SB = few_stage_bytes<K, NC>();
  extern __shared__ __align__(16) unsigned char few_stage[];  // kFewStages x (keys, columns), when bulk
  __shared__ __align__(8) uint64_t s_bar[kFewStages];
  __shared__ int32_t s_val[NV][kFewTile];  // the tile's values in group order
  __shared__ unsigned long long s_tab[kTinySlots];
  __shared__ int s_lid[kTinySlots];
  __shared__ unsigned long long s_ltag[kFewKeys];
  __shared__ int s_nkeys;
  __shared__ int s_gcnt[kFewKeys];                  // the tile's rows per group (phase A)
  __shared__ int s_gstart[kFewKeys + 1];            // the tile's run offsets (phase B)
  __shared__ unsigned long long s_total[kFewKeys];  // COUNT per group over the block's tiles
  __shared__ long long s_rsum[NV][kFewKeys];
  __shared__ int s_rmn[NV][kFewKeys];
  __shared__ int s_rmx[NV][kFewKeys];
  const unsigned long long empty = seen_empty<K>();
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  if (tid < kTinySlots) {
    s_tab[tid] = empty;
    s_lid[tid] = -1;
  }
  if (tid < kFewKeys) {
    s_gcnt[tid] = 0;
    s_total[tid] = 0ull;
#pragma unroll
    for (int c = 0; c < NV; ++c) {
      s_rsum[c][tid] = 0;
      s_rmn[c][tid] = INT32_MAX;
      s_rmx[c][tid] = INT32_MIN;
    }
  }
  if (tid == 0) {
    s_nkeys = 0;
    if (bulk) {
      for (int j = 0; j < kFewStages; ++j) mbar_init(&s_bar[j], 1);
      mbar_fence_init();
    }
  }
  __syncthreads();
  const int64_t ntiles = (n + kFewTile - 1) / kFewTile;
  const int64_t nk = ntiles > blockIdx.x ? (ntiles - 1 - blockIdx.x) / gridDim.x + 1 : 0;  // this block's tiles
  // the block's k-th tile comes by bulk copy unless it is the ragged last one
  auto staged = [&](int64_t k) {
    return bulk && !((n % kFewTile) != 0 && (int64_t)blockIdx.x + k * gridDim.x == ntiles - 1);
  };
  auto issue = [&](int64_t k) {  // one thread: tile k's columns into stage k mod kFewStages
    const int64_t r = ((int64_t)blockIdx.x + k * gridDim.x) * kFewTile;
    unsigned char* d = few_stage + (k % kFewStages) * SB;
    uint64_t* bar = &s_bar[k % kFewStages];
    mbar_expect_tx(bar, SB);
    bulk_g2s(d, key + r, kFewTile * (int)sizeof(K), bar);
#pragma unroll
    for (int c = 0; c < NC; ++c) bulk_g2s(d + kFewTile * sizeof(K) + c * kFewTile * 4, cc.src[c] + r, kFewTile * 4, bar);
  };
  if (tid == 0)
    for (int64_t k = 0; k < kFewStages && k < nk; ++k)
      if (staged(k)) issue(k);
  // per id bit: all ones where this lane's group (lane & 15) has a 0, so that
  // (ballot ^ mask) keeps the lanes whose row agrees with the group on that bit
  const int G = lane & (kFewKeys - 1);
  const unsigned xm0 = (G & 1) ? 0u : F, xm1 = (G & 2) ? 0u : F, xm2 = (G & 4) ? 0u : F, xm3 = (G & 8) ? 0u : F;
  const unsigned below = (1u << lane) - 1u;
  const int dg = warp;  // phase D: this warp's group
  int64_t sum[NV];
  int32_t mn[NV], mx[NV];
#pragma unroll
  for (int c = 0; c < NV; ++c) {
    sum[c] = 0;
    mn[c] = INT32_MAX;
    mx[c] = INT32_MIN;
  }
  bool over = false;
  int64_t k = 0;
  // the bound is the same for all threads of the block: every barrier below is reached by all
  for (; k < nk; ++k) {
    const int64_t t = (int64_t)blockIdx.x + k * gridDim.x;
    const int64_t base = t * kFewTile + tid;
    K kk[kFewRows];
    int32_t v[NV][kFewRows];
    if (staged(k)) {
      mbar_wait(&s_bar[k % kFewStages], (uint32_t)((k / kFewStages) & 1), err);
      const unsigned char* d = few_stage + (k % kFewStages) * SB;
#pragma unroll
      for (int u = 0; u < kFewRows; ++u) {
        kk[u] = reinterpret_cast<const K*>(d)[tid + u * kFewThreads];
#pragma unroll
        for (int c = 0; c < NV; ++c)
          v[c][u] = c < NC ? reinterpret_cast<const int32_t*>(d + kFewTile * sizeof(K) + c * kFewTile * 4)[tid + u * kFewThreads] : 0;
      }
    } else {
      few_load<K, NV>(key, cc, n, t, kk, v);
    }
    int lid[kFewRows];
    bool miss = false;
#pragma unroll
    for (int u = 0; u < kFewRows; ++u) {
      lid[u] = -2;  // past the end
      if (base + (int64_t)u * kFewThreads < n) {
        const unsigned long long tag = seen_tag<K>(kk[u]);
        lid[u] = tag == empty ? -1 : few_find(s_tab, s_lid, tag, empty);
        miss |= lid[u] == -1;
      }
    }
    const bool any_miss = __syncthreads_or(miss);
    // every thread has read stage k: it takes tile k + kFewStages
    if (tid == 0 && k + kFewStages < nk && staged(k + kFewStages)) {
      fence_proxy_async();
      issue(k + kFewStages);
    }
    if (any_miss) {
      // insertion phase: absent keys claim a slot; the claiming thread hands out the id
      bool bail = false;
#pragma unroll
      for (int u = 0; u < kFewRows; ++u) {
        if (lid[u] != -1) continue;
        const unsigned long long tag = seen_tag<K>(kk[u]);
        if (tag == empty) {
          bail = true;
          continue;
        }
        uint32_t sl = (uint32_t)((tag * 0x9e3779b97f4a7c15ull) >> 58);
        bool placed = false;
        for (int p = 0; p < kTinySlots && !placed; ++p) {
          const unsigned long long w = atomicCAS(&s_tab[sl], empty, tag);
          if (w == empty) {
            const int l = atomicAdd(&s_nkeys, 1);
            if (l < kFewKeys) {
              s_lid[sl] = l;
              s_ltag[l] = tag;
            } else {
              bail = true;
            }
            placed = true;
          } else if (w == tag) {
            placed = true;
          } else {
            sl = (sl + 1) & (kTinySlots - 1);
          }
        }
        if (!placed) bail = true;
      }
      if (__syncthreads_or(bail)) {  // the same for all threads of the block
        over = true;
        break;
      }
      bool lost = false;
#pragma unroll
      for (int u = 0; u < kFewRows; ++u)
        if (lid[u] == -1) {
          lid[u] = few_find(s_tab, s_lid, seen_tag<K>(kk[u]), empty);
          lost |= lid[u] < 0;
        }
      if (__syncthreads_or(lost)) {
        over = true;
        break;
      }
    }
    // A: ranks within the warp's rows of each group, the warp's places reserved per group
    int off[kFewRows];
#pragma unroll
    for (int u = 0; u < kFewRows; ++u) {
      const bool valid = lid[u] >= 0;
      const int l = valid ? lid[u] : 0;
      const unsigned V = __ballot_sync(F, valid);
      const unsigned b0 = __ballot_sync(F, l & 1), b1 = __ballot_sync(F, l & 2);
      const unsigned b2 = __ballot_sync(F, l & 4), b3 = __ballot_sync(F, l & 8);
      const unsigned m = V & (b0 ^ xm0) & (b1 ^ xm1) & (b2 ^ xm2) & (b3 ^ xm3);  // rows of group G
      int wb = 0;
      if (lane < kFewKeys && m) wb = atomicAdd(&s_gcnt[lane], __popc(m));
      const unsigned pm = __shfl_sync(F, m, l);  // rows of this row's group
      off[u] = __shfl_sync(F, wb, l) + __popc(pm & below);
    }
    __syncthreads();
    // B: run offsets (exclusive sums of the groups' sizes from independent loads,
    // no shuffle chain) and COUNTs; the sizes are cleared after the next barrier
    if (warp == 0 && lane <= kFewKeys) {
      int x = 0, c = 0;
#pragma unroll
      for (int j = 0; j < kFewKeys; ++j) {
        const int y = s_gcnt[j];
        x += j < lane ? y : 0;
        c = j == lane ? y : c;
      }
      s_gstart[lane] = x;
      if (lane < kFewKeys) s_total[lane] += (unsigned long long)c;
    }
    __syncthreads();
    if (tid < kFewKeys) s_gcnt[tid] = 0;  // read only in B; next written after two more barriers
    // C: values to their places
#pragma unroll
    for (int u = 0; u < kFewRows; ++u)
      if (lid[u] >= 0) {
        const int p = s_gstart[lid[u]] + off[u];
#pragma unroll
        for (int c = 0; c < NC; ++c) s_val[c][p] = v[c][u];
      }
    __syncthreads();
    // D: this warp's half of its group's run
    const int s1 = s_gstart[dg + 1];
    for (int i = s_gstart[dg] + lane; i < s1; i += 32) {
#pragma unroll
      for (int c = 0; c < NC; ++c) {
        const int32_t x = s_val[c][i];
        sum[c] += x;
        mn[c] = min(mn[c], x);
        mx[c] = max(mx[c], x);
      }
    }
  }
  if (over) {
    // the copies still in flight (tiles k + 1 .. k + kFewStages) land before the block leaves
    if (tid == 0) {
      atomicExch(overflow, 1);
      for (int64_t j = k + 1; j <= k + kFewStages && j < nk; ++j)
        if (staged(j)) mbar_wait(&s_bar[j % kFewStages], (uint32_t)((j / kFewStages) & 1), err);
    }
    return;
  }
  // each warp's lanes reduced into its group's results, one TinyPart per id
#pragma unroll
  for (int c = 0; c < NC; ++c) {
    long long s = sum[c];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(F, s, o);
    const int a = __reduce_min_sync(F, mn[c]), b = __reduce_max_sync(F, mx[c]);
    if (lane == 0 && dg < s_nkeys) {
      atomicAdd((unsigned long long*)&s_rsum[c][dg], (unsigned long long)s);
      atomicMin(&s_rmn[c][dg], a);
      atomicMax(&s_rmx[c][dg], b);
    }
  }
  __syncthreads();
  if (tid < kTinySlots) {
    TinyPart tp{};
    tp.tag = empty;
    if (tid < s_nkeys) {
      tp.tag = s_ltag[tid];
      tp.count = (unsigned int)s_total[tid];
#pragma unroll
      for (int c = 0; c < NC; ++c) {
        tp.sum[c] = s_rsum[c][tid];
        tp.mn[c] = s_rmn[c][tid];
        tp.mx[c] = s_rmx[c][tid];
      }
    }
    parts[(int64_t)blockIdx.x * kTinySlots + tid] = tp;
  }
}

// Merges the blocks' slots (one block): dense group ids in order of first
// appearance, the aggregates of Aggs from the per-column results, g into
// *ngroups. Sets `overflow` instead when the union of keys is too large.
template <typename K>
__global__ void __launch_bounds__(1024) hgb_tiny_merge_kernel(const TinyPart* __restrict__ parts, int nparts,
                                                              Aggs A, ColCache cc, K* __restrict__ out_keys,
                                                              int64_t cap, int64_t* ngroups, int* overflow, int* err) {
  __shared__ unsigned long long s_key[2 * kTinyMerge];  // tags
  __shared__ int s_id[2 * kTinyMerge];
  __shared__ int s_n;
  const unsigned long long empty = seen_empty<K>();
  if (*(volatile int*)overflow) return;
  for (int j = threadIdx.x; j < 2 * kTinyMerge; j += blockDim.x) {
    s_key[j] = empty;
    s_id[j] = -1;
  }
  if (threadIdx.x == 0) s_n = 0;
  __syncthreads();
  // ids: one thread per slot entry inserts the tag; the inserting thread takes the id
  for (int e = threadIdx.x; e < nparts * kTinySlots; e += blockDim.x) {
    const unsigned long long tag = parts[e].tag;
    if (tag == empty) continue;
    uint32_t sl = (uint32_t)(tag * 0x9e3779b97f4a7c15ull >> 40) & (2 * kTinyMerge - 1);
    for (int p = 0; p < 2 * kTinyMerge; ++p) {
      const unsigned long long w = atomicCAS(&s_key[sl], empty, tag);
      if (w == empty) {
        s_id[sl] = atomicAdd(&s_n, 1);
        break;
      }
      if (w == tag) break;
      sl = (sl + 1) & (2 * kTinyMerge - 1);
    }
  }
  __syncthreads();
  const int g = s_n;
  if (g > kTinyMerge) {
    if (threadIdx.x == 0) atomicExch(overflow, 1);
    return;
  }
  // starting values, then every entry combined into its group (64-bit atomics on
  // the result; at most nparts * 64 entries)
  for (int t = threadIdx.x; t < g * A.n; t += blockDim.x) {
    const int j = t / g, id = t - j * g;
    if (id < cap) A.out[j][id] = agg_identity(A.op[j]);
  }
  for (int sl = threadIdx.x; sl < 2 * kTinyMerge; sl += blockDim.x) {
    if (s_key[sl] == empty) continue;
    const int id = s_id[sl];
    const unsigned long long tag = s_key[sl];
    const K k = sizeof(K) == 4 ? (K)(int32_t)(uint32_t)tag : (K)(int64_t)tag;
    if (id < cap)
      out_keys[id] = k;
    else
      set_status(err, GJ_ERR_CAPACITY);
  }
  __syncthreads();
  for (int e = threadIdx.x; e < nparts * kTinySlots; e += blockDim.x) {
    const TinyPart& t = parts[e];
    if (t.tag == empty) continue;
    uint32_t sl = (uint32_t)(t.tag * 0x9e3779b97f4a7c15ull >> 40) & (2 * kTinyMerge - 1);
    while (s_key[sl] != t.tag) sl = (sl + 1) & (2 * kTinyMerge - 1);
    const int id = s_id[sl];
    if (id >= cap) continue;
    for (int j = 0; j < A.n; ++j) {
      const int op = A.op[j], c = cc.slot[j];
      const int64_t v = op == GJ_AGG_COUNT ? (int64_t)t.count
                        : op == GJ_AGG_SUM ? t.sum[c]
                        : op == GJ_AGG_MIN ? (int64_t)t.mn[c] : (int64_t)t.mx[c];
      agg_atomic(op, &A.out[j][id], v);
    }
  }
  if (threadIdx.x == 0) *ngroups = g;
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
// One block per partition (Sec. 4.3). The block inserts the partition's keys into
// a shared-memory table sized to the partition (a slot holds the partition row +
// 1 of its key's first row; keys are compared in global memory, where the small
// partition stays cached), gives the keys dense local ids in slot order,
// reserves the round's output rows from the global group counter, aggregates
// every row into shared-memory slots by local id (one copy per warp, or per few
// warps, when the round's groups leave room; 32-bit atomics only, SUMs split and
// folded into the output rows every kSplitRows rows) and writes the rest of the
// output rows with plain stores.
// A partition whose distinct keys exceed the block's group capacity C is split by
// a second hash into two halves, recursively, each processed as above.
constexpr int kPgbThreads = 512;
constexpr int kPgbMaxQ = 12;
constexpr int kPgbSmem = 110 * 1024;  // dynamic shared memory budget of a block (two blocks per SM)
constexpr int kPgbMaxCap = 4096;      // groups per round (local ids fit int16)

// Work of a PGB launch beyond one block per partition. Partitions with many more
// rows than the others (identical keys: few groups, Zipf skew) are cut into slices
// taken by several blocks (items); a slice's groups go to partial rows in the
// partition's own range of part_keys / part_agg (a partition's partial rows never
// outnumber its rows), counted by pcount; a second launch with pcount set (and
// no items) then aggregates each sliced partition's partial rows into the result
// (Sec. 4.3: overly large partitions get a group-by of their own).
struct PgbItem {
  int32_t part;
  int32_t nslices;
  int64_t r0, r1;
};
template <typename K>
struct PgbWork {
  const PgbItem* items;        // non-null: block b takes items[b]
  const int64_t* nitems;       // non-null: blocks from *nitems on have no item
  unsigned long long* pcount;  // partial rows per partition (the second launch reads them)
  const int64_t* pbase;        // first partial row of each sliced partition
  K* part_keys;                // partial rows: keys and one int64 value per aggregate
  int64_t* part_agg[kMaxAggs];
};

// Items of the first PGB launch (one block): every non-empty partition whole, or,
// when it has more than `thresh` rows, in slices of about `slice` rows. info[0] =
// the item count, info[1] = the rows of the sliced partitions; pbase[p] = where
// partition p's partial rows start (sliced partitions packed in order).
__global__ void __launch_bounds__(1024) pgb_items_kernel(const int64_t* __restrict__ poff, int nparts, int64_t thresh,
                                                         int64_t slice, PgbItem* __restrict__ items,
                                                         int64_t* __restrict__ pbase, int64_t* info) {
  __shared__ int64_t s_w[2][32];
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  const int per = (nparts + 1023) / 1024;
  const int p0 = min(t * per, nparts), p1 = min(p0 + per, nparts);
  auto nslices = [&](int p) -> int64_t {
    const int64_t rows = poff[p + 1] - poff[p];
    if (rows <= 0) return 0;
    return rows > thresh ? (rows + slice - 1) / slice : 1;
  };
  int64_t cnt = 0, srows = 0;
  for (int p = p0; p < p1; ++p) {
    const int64_t k = nslices(p);
    cnt += k;
    if (k > 1) srows += poff[p + 1] - poff[p];
  }
  // block-wide exclusive scans of both
  int64_t x = cnt, y = srows;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int64_t a = __shfl_up_sync(0xffffffffu, x, o), b = __shfl_up_sync(0xffffffffu, y, o);
    if (lane >= o) {
      x += a;
      y += b;
    }
  }
  if (lane == 31) {
    s_w[0][warp] = x;
    s_w[1][warp] = y;
  }
  __syncthreads();
  if (t == 0) {
    int64_t a = 0, b = 0;
    for (int w = 0; w < 32; ++w) {
      const int64_t ca = s_w[0][w], cb = s_w[1][w];
      s_w[0][w] = a;
      s_w[1][w] = b;
      a += ca;
      b += cb;
    }
    info[0] = a;
    info[1] = b;
  }
  __syncthreads();
  int64_t ib = s_w[0][warp] + x - cnt, rb = s_w[1][warp] + y - srows;
  for (int p = p0; p < p1; ++p) {
    const int64_t k = nslices(p), r0 = poff[p], r1 = poff[p + 1];
    pbase[p] = rb;
    if (k > 1) rb += r1 - r0;
    const int64_t len = k > 1 ? (r1 - r0 + k - 1) / k : r1 - r0;
    for (int64_t q = 0; q < k; ++q)
      items[ib + q] = PgbItem{p, (int32_t)k, r0 + q * len, min64(r1, r0 + (q + 1) * len)};
    ib += k;
  }
}

template <typename K>
__device__ __forceinline__ uint32_t pgb_sub(K k, int q) {
  if (q == 0) return 0;
  uint32_t h = fmix32((uint32_t)KeyTraits<K>::hash64(k) ^ 0x9e3779b9u);
  return h & ((1u << q) - 1);
}

template <typename K>
__device__ __forceinline__ uint32_t pgb_slot(K k, int pbits, int tslots) {
  return (uint32_t)(KeyTraits<K>::hash64(k) >> pbits) & (uint32_t)(tslots - 1);
}

// Dynamic shared memory of a PGB block with group capacity C: table (2C int32
// slots, 2C int16 local ids), keys by local id, then the aggregate arrays.
template <typename K>
__host__ __device__ constexpr int pgb_key_off(int C) {
  return (C * 2 * 4 + C * 2 * 2 + 15) & ~15;
}
template <typename K>
__host__ __device__ constexpr int pgb_agg_off(int C) {
  return (pgb_key_off<K>(C) + C * (int)sizeof(K) + 15) & ~15;
}

template <typename K>
__global__ void __launch_bounds__(kPgbThreads, 2) pgb_kernel(const K* __restrict__ key,
                                                          const int64_t* __restrict__ poff, int pbits, Aggs A,
                                                          ColCache cc, SmemAggLayout L, int C,
                                                          K* __restrict__ out_keys, int64_t cap,
                                                          unsigned long long* ngroups, PgbWork<K> W, int* err) {
  extern __shared__ __align__(16) unsigned char s_raw[];
  int32_t* s_slot = (int32_t*)s_raw;
  int16_t* s_lid = (int16_t*)(s_slot + 2 * C);
  K* s_key = (K*)(s_raw + pgb_key_off<K>(C));
  unsigned char* s_agg = s_raw + pgb_agg_off<K>(C);
  __shared__ int64_t offs[kMaxAggs];
  __shared__ int s_code[kMaxAggs];
  __shared__ int s_wsum[kPgbThreads / 32];
  __shared__ int s_count;
  __shared__ unsigned long long s_base;
  __shared__ int s_stack_q[kPgbMaxQ + 2];
  __shared__ uint32_t s_stack_r[kPgbMaxQ + 2];
  __shared__ int s_top;

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  // the block's rows: a whole partition, one slice of a large one (whose groups go
  // to the partial rows of the partition), or the partial rows of a sliced one
  int64_t p = blockIdx.x, r0, r1;
  bool partial = false;
  if (W.items) {
    if (W.nitems && (int64_t)blockIdx.x >= *W.nitems) return;
    const PgbItem it = W.items[blockIdx.x];
    p = it.part;
    r0 = it.r0;
    r1 = it.r1;
    partial = it.nslices > 1;
  } else if (W.pcount) {
    r0 = W.pbase[p];
    r1 = r0 + (int64_t)W.pcount[p];
  } else {
    r0 = poff[p];
    r1 = poff[p + 1];
  }
  if (r1 <= r0) return;
  const int64_t rows = r1 - r0;
  K* __restrict__ okeys = partial ? W.part_keys : out_keys;
  // the destination column of each aggregate, read from shared memory in the loops
  __shared__ int64_t* oagg[kMaxAggs];
  if (tid < A.n) oagg[tid] = partial ? W.part_agg[tid] : A.out[tid];
  const int64_t ocap = partial ? INT64_MAX : cap;  // a partition's partial rows never exceed its rows
  int tslots = 64;  // table slots: about twice the rows, at most 2C
  while (tslots < 2 * C && tslots < 2 * rows) tslots <<= 1;
  if (tid == 0) {
    s_stack_q[0] = 0;
    s_stack_r[0] = 0;
    s_top = 1;
  }
  __syncthreads();
  bool over_cap = false;
  const int nwarps = blockDim.x >> 5;
  // rounds (q, r): the rows whose second hash has r in its low q bits
  while (s_top > 0) {
    const int q = s_stack_q[s_top - 1];
    const uint32_t round = s_stack_r[s_top - 1];
    __syncthreads();
    if (tid == 0) {
      --s_top;
      s_count = 0;
    }
    for (int j = tid; j < tslots; j += blockDim.x) s_slot[j] = 0;
    __syncthreads();
    // ---- insert the round's keys
    constexpr int kBatch = 4;
    for (int64_t b0 = r0; b0 < r1; b0 += (int64_t)kBatch * blockDim.x) {
      K kk[kBatch];
#pragma unroll
      for (int u = 0; u < kBatch; ++u) {
        const int64_t i = b0 + (int64_t)u * blockDim.x + tid;
        kk[u] = i < r1 ? key[i] : K(0);
      }
#pragma unroll
      for (int u = 0; u < kBatch; ++u) {
        const int64_t i = b0 + (int64_t)u * blockDim.x + tid;
        if (i >= r1 || pgb_sub<K>(kk[u], q) != round) continue;
        uint32_t sl = pgb_slot<K>(kk[u], pbits, tslots);
        for (int probe = 0; probe < tslots; ++probe) {
          int v = ((volatile int32_t*)s_slot)[sl];  // a repeated key finds its slot without an atomic
          if (v == 0) {
            v = atomicCAS(&s_slot[sl], 0, (int)(i - r0 + 1));
            if (v == 0) break;
          }
          if (key[r0 + v - 1] == kk[u]) break;
          sl = (sl + 1) & (uint32_t)(tslots - 1);
        }
      }
    }
    __syncthreads();
    // ---- dense local ids in slot order
    const int per = (tslots + (int)blockDim.x - 1) / (int)blockDim.x;
    const int s0 = min(tid * per, tslots), s1 = min(s0 + per, tslots);
    int mine = 0;
    for (int j = s0; j < s1; ++j) mine += s_slot[j] != 0;
    int x = mine;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += y;
    }
    if (lane == 31) s_wsum[warp] = x;
    __syncthreads();
    if (tid == 0) {
      int run = 0;
      for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
        const int c = s_wsum[w];
        s_wsum[w] = run;
        run += c;
      }
      s_count = run;
    }
    __syncthreads();
    const int count = s_count;
    if (count > C) {
      // too many keys for one round: split it by the next bit of the second hash
      if (tid == 0) {
        if (q < kPgbMaxQ) {
          s_stack_q[s_top] = q + 1;
          s_stack_r[s_top] = round | (1u << q);
          s_stack_q[s_top + 1] = q + 1;
          s_stack_r[s_top + 1] = round;
          s_top += 2;
        } else {
          set_status(err, GJ_ERR_CAPACITY);
        }
      }
      __syncthreads();
      continue;
    }
    {
      int lid = s_wsum[warp] + x - mine;
      for (int j = s0; j < s1; ++j) {
        const int v = s_slot[j];
        if (v != 0) {
          s_key[lid] = key[r0 + v - 1];
          s_lid[j] = (int16_t)lid;
          ++lid;
        }
      }
    }
    // copies of the round's slots: as many (up to one per warp) as fit in C groups
    int ncopy = 1;
    while (ncopy < nwarps && 2 * ncopy * count <= C) ncopy *= 2;
    const int cc_cap = C / ncopy;  // groups per copy
    const int64_t copy_bytes = (int64_t)cc_cap * L.bytes_per_group;
    if (tid == 0) {
      int64_t o = 0;
      for (int q2 = 0; q2 < A.n; ++q2) {
        const int j = L.order[q2];
        offs[j] = o;
        o += (int64_t)cc_cap * L.width[j];
      }
      // the round's output rows: from the global group counter, or the partition's
      // next partial rows
      s_base = partial ? (unsigned long long)W.pbase[p] + atomicAdd(&W.pcount[p], (unsigned long long)count)
                       : atomicAdd(ngroups, (unsigned long long)count);
    }
    if (tid < A.n) s_code[tid] = slot_code(A.op[tid], A.op[tid] == GJ_AGG_COUNT ? -1 : cc.slot[tid],
                                           slot_form(A, cc, tid, true));
    __syncthreads();
    const int64_t base = (int64_t)s_base;
    for (int c = 0; c < ncopy; ++c)
      for (int jq = 0; jq < A.n; ++jq)
        for (int l = tid; l < count; l += blockDim.x)
          smem_init(A.op[jq], L.width[jq], s_agg + c * copy_bytes + offs[jq] + (int64_t)l * L.width[jq]);
    // split SUMs accumulate in the output rows, folded in every kSplitRows rows
    for (int j = 0; j < A.n; ++j)
      if ((s_code[j] & 3) == kSlotSplit)
        for (int l = tid; l < count && base + l < ocap; l += blockDim.x) oagg[j][base + l] = 0;
    __syncthreads();
    auto fold_split = [&]() {
      for (int j = 0; j < A.n; ++j) {
        if ((s_code[j] & 3) != kSlotSplit) continue;
        for (int l = tid; l < count; l += blockDim.x) {
          int64_t v = 0;
          for (int c = 0; c < ncopy; ++c) {
            unsigned char* pp = s_agg + c * copy_bytes + offs[j] + (int64_t)l * 8;
            v += slot_read(GJ_AGG_SUM, kSlotSplit, pp);
            *(int64_t*)pp = 0;
          }
          if (base + l < ocap) oagg[j][base + l] += v;  // this block owns the row
        }
      }
    };
    unsigned char* my_agg = s_agg + (warp & (ncopy - 1)) * copy_bytes;
    // ---- aggregate the round's rows by local id, in epochs of kSplitRows rows
    for (int64_t e0 = r0; e0 < r1; e0 += kSplitRows) {
      const int64_t e1 = min64(r1, e0 + kSplitRows);
      for (int64_t b0 = e0; b0 < e1; b0 += (int64_t)kBatch * blockDim.x) {
        int64_t row[kBatch];
        bool valid[kBatch];
        int32_t lid[kBatch];
#pragma unroll
        for (int u = 0; u < kBatch; ++u) {
          row[u] = b0 + (int64_t)u * blockDim.x + tid;
          valid[u] = row[u] < e1;
          lid[u] = -1;
          if (!valid[u]) continue;
          const K k = key[row[u]];
          if (pgb_sub<K>(k, q) != round) continue;
          uint32_t sl = pgb_slot<K>(k, pbits, tslots);
          for (int probe = 0; probe < tslots; ++probe) {
            if (s_slot[sl] == 0) break;
            const int l = s_lid[sl];
            if (s_key[l] == k) {
              lid[u] = l;
              break;
            }
            sl = (sl + 1) & (uint32_t)(tslots - 1);
          }
        }
        int32_t cv[kColCache][kBatch];
        load_cached<kBatch>(cc, row, valid, cv);
        for (int j = 0; j < A.n; ++j) {
          unsigned char* sb = my_agg + offs[j];
          slot_dispatch(s_code[j], [&](auto U) {
            using Up = decltype(U);
#pragma unroll
            for (int u = 0; u < kBatch; ++u)
              if (lid[u] >= 0)
                Up::apply(sb + (int64_t)lid[u] * Up::kWidth, Up::template value<kBatch>(A, j, cv, u, row[u]));
          });
        }
      }
      __syncthreads();
      fold_split();
      __syncthreads();
    }
    // ---- the round's groups: keys and the other aggregates, copies combined
    for (int l = tid; l < count; l += blockDim.x) {
      const int64_t o = base + l;
      if (o >= ocap) {
        over_cap = true;
        continue;
      }
      okeys[o] = s_key[l];
      for (int j = 0; j < A.n; ++j) {
        const int form = s_code[j] & 3;
        if (form == kSlotSplit) continue;
        const unsigned char* sl = s_agg + offs[j] + (int64_t)l * L.width[j];
        int64_t v = slot_read(A.op[j], form, sl);
        // copies a group never reached hold the identity, which combining leaves out
        for (int c = 1; c < ncopy; ++c) v = agg_combine(A.op[j], v, slot_read(A.op[j], form, sl + c * copy_bytes));
        oagg[j][o] = v;
      }
    }
    __syncthreads();
  }
  if (over_cap) set_status(err, GJ_ERR_CAPACITY);
}

// Smallest and largest signed-order bit pattern of the keys: mm[0] = min, mm[1] =
// max (mm starts at {~0, 0}).
template <typename K>
__global__ void __launch_bounds__(256) key_range_kernel(const K* __restrict__ key, int64_t n,
                                                         unsigned long long* mm) {
  unsigned long long lo = ~0ull, hi = 0ull;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
    const unsigned long long u = (unsigned long long)digit_source<K>(__ldcs(key + i), kSignedOrder);
    lo = u < lo ? u : lo;
    hi = u > hi ? u : hi;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long a = __shfl_xor_sync(0xffffffffu, lo, o), b = __shfl_xor_sync(0xffffffffu, hi, o);
    lo = a < lo ? a : lo;
    hi = b > hi ? b : hi;
  }
  if ((threadIdx.x & 31) == 0) {
    atomicMin(&mm[0], lo);
    atomicMax(&mm[1], hi);
  }
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

  // HGB with at most 32 expected groups: a few-groups pass first (tiles sorted by
  // group in shared memory for at most 16, the lane-slot pass for 17 to 32); the general
  // kernels below run only if it reports overflow
  int* gate = nullptr;
  if (variant == GJ_GB_HGB && opt->groups_hint > 0 && opt->groups_hint <= kTinyKeys) {
    Aggs A0 = make_aggs(in, nagg, ops, op_col, out_aggs, in->cols);
    const ColCache cc0 = make_col_cache(A0);
    bool eligible = true;
    for (int j = 0; j < nagg; ++j)
      if (ops[j] != GJ_AGG_COUNT && (A0.size[j] != 4 || cc0.slot[j] < 0)) eligible = false;
    if (eligible) {
      const bool few = opt->groups_hint <= kFewKeys;
      const int64_t few_block_rows = kFewTile;
      const int blocks =
          few ? (int)std::max<int64_t>(1, std::min<int64_t>((n + few_block_rows - 1) / few_block_rows,
                                                            (int64_t)ctx.num_sms * 2))
              : (int)std::max<int64_t>(1, std::min<int64_t>((n + 1023) / 1024, (int64_t)ctx.num_sms * 2));
      TinyPart* parts = scr.get_as<TinyPart>((size_t)blocks * kTinySlots);
      gate = scr.get_as<int>(1);
      if (scr.failed()) return GJ_ERR_OOM;
      if ((st = cuda_check(cudaMemsetAsync(gate, 0, sizeof(int), s))) != GJ_OK) return st;
      if (few) {
        static_assert(kColCache == 3, "one instantiation per cached-column count");
        auto kern = cc0.n == 0   ? hgb_few_kernel<K, 0>
                    : cc0.n == 1 ? hgb_few_kernel<K, 1>
                    : cc0.n == 2 ? hgb_few_kernel<K, 2>
                                 : hgb_few_kernel<K, 3>;
        const int sb = cc0.n == 0   ? few_stage_bytes<K, 0>()
                       : cc0.n == 1 ? few_stage_bytes<K, 1>()
                       : cc0.n == 2 ? few_stage_bytes<K, 2>()
                                    : few_stage_bytes<K, 3>();
        // bulk copies need every column to start on 16 bytes (tiles then do too)
        bool bulk = ((uintptr_t)in->key & 15) == 0;
        for (int c = 0; c < cc0.n; ++c) bulk = bulk && ((uintptr_t)cc0.src[c] & 15) == 0;
        const int bytes = bulk ? kFewStages * sb : 0;
        if ((st = ensure_smem_attr(ctx, (const void*)kern, kFewStages * sb)) != GJ_OK) return st;
        LaunchScope ls(ctx, KK_HGB_AGG);
        kern<<<blocks, kFewThreads, bytes, s>>>((const K*)in->key, n, cc0, parts, gate, bulk, ctx.d_status);
      } else {
        LaunchScope ls(ctx, KK_HGB_AGG);
        hgb_tiny_kernel<K><<<blocks, 1024, 0, s>>>((const K*)in->key, n, cc0, parts, gate);
      }
      {
        LaunchScope ls(ctx, KK_HGB_AGG);
        hgb_tiny_merge_kernel<K><<<1, 1024, 0, s>>>(parts, blocks, A0, cc0, (K*)out_keys, cap, d_ngroups, gate,
                                                     ctx.d_status);
      }
    }
  }

  // HGB and SGB-DE share the dictionary of Alg. 1, stage 1: a table of (key, dense
  // id) entries sized for twice the expected groups (the hint, else n), filled
  // by one pass over the keys; out_keys receives the dictionary (id -> key).
  HEntry<K>* ht = nullptr;
  uint64_t slots = 1;
  if (variant == GJ_GB_HGB || variant == GJ_GB_SGB_DE) {
    const uint64_t want =
        (uint64_t)std::max<int64_t>(2, 2 * (opt->groups_hint > 0 ? std::min(opt->groups_hint, n) : n));
    while (slots < want) slots <<= 1;
    ht = scr.get_as<HEntry<K>>(slots);
    if (scr.failed()) return GJ_ERR_OOM;
    if ((st = cuda_check(cudaMemsetAsync(ht, 0, sizeof(HEntry<K>) * slots, s))) != GJ_OK) return st;
    LaunchScope ls(ctx, KK_HGB_GROUP_ID);
    // one block per SM with its key cache
    const int blocks = (int)std::max<int64_t>(1, std::min<int64_t>((n + 1023) / 1024, (int64_t)ctx.num_sms));
    const int cache_bytes = kSeenSlots * (int)(sizeof(unsigned long long) + sizeof(int32_t));
    const bool fit = opt->groups_hint > 0 && opt->groups_hint <= kSeenSlots / 2;
    auto kern = fit ? hgb_dict_kernel<K, kSeenProbesFit> : hgb_dict_kernel<K, kSeenProbesSome>;
    if ((st = ensure_smem_attr(ctx, (const void*)kern, cache_bytes)) != GJ_OK) return st;
    kern<<<blocks, 1024, cache_bytes, s>>>((const K*)in->key, n, ht, slots - 1, (unsigned long long*)d_ngroups,
                                           (K*)out_keys, cap, gate, ctx.d_status);
  }

  if (variant == GJ_GB_HGB) {
    Aggs A = make_aggs(in, nagg, ops, op_col, out_aggs, in->cols);
    {
      LaunchScope ls(ctx, KK_AGG_INIT);
      agg_init_kernel<<<ctx.num_sms * 4, 256, 0, s>>>(A, d_ngroups, cap, gate);
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
    if ((st = ensure_smem_attr(ctx, (const void*)hgb_aggregate_kernel<K>, budget)) != GJ_OK) return st;
    {
      LaunchScope ls(ctx, KK_HGB_AGG);
      hgb_aggregate_kernel<K><<<ctx.num_sms, 1024, budget, s>>>((const K*)in->key, n, ht, slots - 1, A,
                                                                 make_col_cache(A), L, d_ngroups, cap, budget, gate,
                                                                 ctx.d_status);
    }
    return cuda_check(cudaGetLastError());
  }

  // ---- SGB-DE (SGB-TR of Sec. 4.1.3 after the dictionary encoding of Sec. 4.4): HGB stage 1 gives every
  // row a dense code and writes the dictionary (code -> key) to out_keys; the
  // codes are then sorted with the values on their ceil(log2 g) bits only and
  // reduced by the SGB kernels, whose segment i is code i. Reading g to size the
  // sort synchronises the stream once.
  if (variant == GJ_GB_SGB_DE) {
    int32_t* code = scr.get_as<int32_t>(n);
    int32_t* code2 = scr.get_as<int32_t>(n);
    int32_t* code_out = scr.get_as<int32_t>(n);  // the reduction's segment codes (0, 1, ...), unused
    if (scr.failed()) return GJ_ERR_OOM;
    {
      LaunchScope ls(ctx, KK_HGB_GROUP_ID);
      const int blocks = (int)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, (int64_t)ctx.num_sms * 8));
      hgb_codes_kernel<K><<<blocks, 256, 0, s>>>((const K*)in->key, n, ht, slots - 1, code, ctx.d_status);
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
    // only the key bits that vary are sorted: keys between min and max (in
    // signed order) share every bit above the highest bit where min and max
    // differ. Reading the range synchronises the stream once.
    unsigned long long* d_mm = scr.get_as<unsigned long long>(2);
    if (scr.failed()) return GJ_ERR_OOM;
    const unsigned long long init[2] = {~0ull, 0ull};
    if ((st = cuda_check(cudaMemcpyAsync(d_mm, init, sizeof(init), cudaMemcpyHostToDevice, s))) != GJ_OK) return st;
    {
      LaunchScope ls(ctx, KK_RADIX_HIST);
      const int blocks = (int)std::max<int64_t>(1, std::min<int64_t>((n + 1023) / 1024, (int64_t)ctx.num_sms * 4));
      key_range_kernel<K><<<blocks, 256, 0, s>>>((const K*)in->key, n, d_mm);
    }
    unsigned long long mm[2] = {0, 0};
    if ((st = cuda_check(cudaMemcpyAsync(mm, d_mm, sizeof(mm), cudaMemcpyDeviceToHost, s))) != GJ_OK) return st;
    if ((st = cuda_check(cudaStreamSynchronize(s))) != GJ_OK) return st;
    int live = 0;
    while (live < kbits && ((mm[0] ^ mm[1]) >> live) != 0) ++live;
    if (live == 0) {
      // one key value: the input is already sorted
      Aggs A0 = make_aggs(in, nagg, ops, op_col, out_aggs, in->cols);
      return sgb_reduce_run<K>(ctx, scr, (const K*)in->key, n, A0, nagg, ops, (K*)out_keys, cap, d_ngroups);
    }
    if ((st = radix_partition_run(ctx, scr, sizeof(K) == 8 ? GJ_I64 : GJ_I32, in->key, k2, cs, n, 0, live,
                                  kSignedOrder, opt->bits_per_pass)) != GJ_OK)
      return st;
    return sgb_reduce_run<K>(ctx, scr, k2, n, A, nagg, ops, (K*)out_keys, cap, d_ngroups);
  }

  // shared-memory slot widths as in HGB; the group capacity C of a round is what
  // fits the block's budget (at most kPgbMaxCap)
  SmemAggLayout L{};
  {
    int q = 0;
    for (int pass = 0; pass < 2; ++pass)
      for (int j = 0; j < nagg; ++j) {
        const int w = ops[j] == GJ_AGG_SUM ? 8 : (ops[j] == GJ_AGG_COUNT ? 4 : A.size[j]);
        if ((pass == 0) == (w == 8)) {
          L.width[j] = w;
          L.order[q++] = j;
          L.bytes_per_group += w;
        }
      }
  }
  int C = kPgbMaxCap;
  while (C > 32 && pgb_agg_off<K>(C) + C * L.bytes_per_group > kPgbSmem) C >>= 1;
  // PGB-TR / PGB-UR: hashed partitions of about 2048 rows (at most 16 bits). With
  // a groups hint, fewer bits while a partition still holds about C / 2 groups,
  // but at least 8 (or the row-derived count if smaller), so that every SM gets
  // several partitions
  int bits = opt->radix_bits > 0 ? std::min(opt->radix_bits, 16) : 0;
  if (opt->radix_bits <= 0) {
    int by_rows = 0;
    while (by_rows < 16 && (n >> by_rows) > 2048) ++by_rows;
    bits = by_rows;
    if (opt->groups_hint > 0) {
      int by_groups = 0;
      while (by_groups < 16 && (opt->groups_hint >> by_groups) > C / 2) ++by_groups;
      bits = std::max(std::min(by_rows, 8), std::min(by_rows, by_groups));
    }
  }
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
  if (scr.failed()) return GJ_ERR_OOM;
  if ((st = partition_bounds_run(ctx, sizeof(K) == 8 ? GJ_I64 : GJ_I32, k2, n, 0, bits, kHashed, poff)) != GJ_OK)
    return st;
  const size_t dyn = (size_t)pgb_agg_off<K>(C) + (size_t)C * L.bytes_per_group;
  if ((st = ensure_smem_attr(ctx, (const void*)pgb_kernel<K>, (int)dyn)) != GJ_OK) return st;
  // partitions of more than four slices' rows (few groups, hot keys) are cut into
  // slices of about `slice` rows: an SM's fair share of the rows (a sixteenth of
  // that when the average partition is smaller), at least 16384
  const int64_t avg = std::max<int64_t>(1, n / nparts);
  const int64_t slice = std::max<int64_t>(16384, std::min<int64_t>(avg, n / ((int64_t)ctx.num_sms * 8)));
  const int64_t thresh = 4 * slice;
  PgbItem* items = scr.get_as<PgbItem>((size_t)(nparts + n / slice + 2));
  int64_t* pbase = scr.get_as<int64_t>(nparts);
  int64_t* info = scr.get_as<int64_t>(2);
  unsigned long long* pcount = scr.get_as<unsigned long long>(nparts);
  if (scr.failed()) return GJ_ERR_OOM;
  if ((st = cuda_check(cudaMemsetAsync(pcount, 0, sizeof(unsigned long long) * nparts, s))) != GJ_OK) return st;
  {
    LaunchScope ls(ctx, KK_PGB);
    pgb_items_kernel<<<1, 1024, 0, s>>>(poff, (int)nparts, thresh, slice, items, pbase, info);
  }
  PgbWork<K> W{};
  W.items = items;
  W.pcount = pcount;
  W.pbase = pbase;
  // partial rows never outnumber the sliced partitions' rows. Small inputs take
  // scratch for all n rows and launch for the largest item count (blocks past it
  // leave at once); large ones read the item count and the sliced rows first
  // (one synchronisation) to size both exactly
  const size_t part_row_bytes = sizeof(K) + (size_t)8 * nagg;
  const bool sized_up_front = (size_t)n * part_row_bytes <= ((size_t)256 << 20);
  int64_t nitems = nparts + n / slice + 2, sliced_rows = n;
  if (sized_up_front) {
    W.nitems = info;
  } else {
    int64_t h_info[2] = {0, 0};
    if ((st = cuda_check(cudaMemcpyAsync(h_info, info, sizeof(h_info), cudaMemcpyDeviceToHost, s))) != GJ_OK)
      return st;
    if ((st = cuda_check(cudaStreamSynchronize(s))) != GJ_OK) return st;
    nitems = h_info[0];
    sliced_rows = h_info[1];
    if (nitems == 0) return GJ_OK;
  }
  if (sliced_rows > 0) {
    W.part_keys = scr.get_as<K>((size_t)sliced_rows);
    for (int j = 0; j < nagg; ++j) W.part_agg[j] = scr.get_as<int64_t>((size_t)sliced_rows);
    if (scr.failed()) return GJ_ERR_OOM;
  }
  {
    LaunchScope ls(ctx, KK_PGB);
    pgb_kernel<K><<<(unsigned)nitems, kPgbThreads, dyn, s>>>(k2, poff, bits, A, make_col_cache(A), L, C,
                                                             (K*)out_keys, cap, (unsigned long long*)d_ngroups, W,
                                                             ctx.d_status);
  }
  if (sliced_rows == 0) return cuda_check(cudaGetLastError());
  // the sliced partitions' partial rows, one block each: COUNTs add up, SUM / MIN /
  // MAX combine as themselves, over int64 values
  Aggs A2 = A;
  A2.tid = nullptr;
  for (int j = 0; j < nagg; ++j) {
    A2.op[j] = ops[j] == GJ_AGG_COUNT ? GJ_AGG_SUM : ops[j];
    A2.src[j] = W.part_agg[j];
    A2.size[j] = 8;
  }
  SmemAggLayout L2{};
  {
    int q = 0;
    for (int j = 0; j < nagg; ++j) {
      L2.width[j] = 8;
      L2.order[q++] = j;
      L2.bytes_per_group += 8;
    }
  }
  int C2 = kPgbMaxCap;
  while (C2 > 32 && pgb_agg_off<K>(C2) + C2 * L2.bytes_per_group > kPgbSmem) C2 >>= 1;
  const size_t dyn2 = (size_t)pgb_agg_off<K>(C2) + (size_t)C2 * L2.bytes_per_group;
  if ((st = ensure_smem_attr(ctx, (const void*)pgb_kernel<K>, (int)std::max(dyn, dyn2))) != GJ_OK) return st;
  PgbWork<K> W2 = W;
  W2.items = nullptr;
  W2.nitems = nullptr;
  {
    LaunchScope ls(ctx, KK_PGB);
    pgb_kernel<K><<<(unsigned)nparts, kPgbThreads, dyn2, s>>>(W.part_keys, poff, bits, A2, make_col_cache(A2), L2, C2,
                                                              (K*)out_keys, cap, (unsigned long long*)d_ngroups, W2,
                                                              ctx.d_status);
  }
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
  if (variant == GJ_GB_AUTO)
    variant = opt->selector == GJ_SELECT_HEURISTIC ? choose_groupby_variant(in, nagg, ops, opt, smem_budget)
                                                   : cost_groupby_variant(in, nagg, ops, opt);
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
