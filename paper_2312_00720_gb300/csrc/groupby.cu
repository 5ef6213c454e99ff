// Grouped aggregation (paper Sec. 3.2, 4.1.3, 4.2, 4.3).
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
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n_round; i += stride) {
    const bool valid = i < n;
    const K k = valid ? key[i] : K(0);
    const unsigned vmask = __ballot_sync(0xffffffffu, valid);
    unsigned peers = __match_any_sync(0xffffffffu, k) & vmask;
    const int leader = valid ? __ffs(peers) - 1 : lane;
    int32_t loc = -1;
    if (valid && lane == leader) {
      uint64_t sl = KeyTraits<K>::hash64(k) & mask;
      for (uint64_t probe = 0; probe <= mask; ++probe) {
        int prev = atomicCAS(&ht[sl], 0, (int)(i + 1));
        if (prev == 0) {
          unsigned long long g = atomicAdd(ngroups, 1ull);
          gid_of_row[i] = (int32_t)g;
          if ((int64_t)g < cap)
            out_keys[g] = k;
          else
            set_status(err, GJ_ERR_CAPACITY);
          loc = (int32_t)i;
          break;
        }
        if (key[prev - 1] == k) {
          loc = prev - 1;
          break;
        }
        sl = (sl + 1) & mask;
      }
      if (loc < 0) set_status(err, GJ_ERR_CAPACITY);  // table full
    }
    loc = __shfl_sync(0xffffffffu, loc, leader);
    if (valid) gidloc[i] = loc;
  }
}

// out[j][0..g) = identity of op j, g read from the device counter.
__global__ void agg_init_kernel(Aggs A, const int64_t* __restrict__ ngroups, int64_t cap) {
  const int64_t g = min64(*ngroups, cap);
  const int64_t total = g * A.n;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += stride) {
    int j = (int)(t / g);
    A.out[j][t - (int64_t)j * g] = agg_identity(A.op[j]);
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
                                                       SmemAggLayout L, const int64_t* __restrict__ ngroups,
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
    for (int64_t i = first; i < n; i += stride) {
      const int32_t loc = gidloc[i];
      if (loc < 0) continue;  // insert failed (reported as GJ_ERR_CAPACITY)
      int64_t gid = gid_of_row[loc];
      if (gid >= g) continue;
      for (int j = 0; j < A.n; ++j)
        smem_update(A.op[j], L.width[j], s_agg + offs[j] + gid * L.width[j], agg_value(A, j, i));
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
    for (int64_t i = first; i < n; i += stride) {
      const int32_t loc = gidloc[i];
      if (loc < 0) continue;
      int64_t gid = gid_of_row[loc];
      if (gid >= g) continue;
      for (int j = 0; j < A.n; ++j) agg_atomic(A.op[j], &A.out[j][gid], agg_value(A, j, i));
    }
  }
}

// ================================================================ SGB
constexpr int kSegItems = 16;
constexpr int kSegWarps = 8;
constexpr int kSegTile = 32 * kSegItems;

// Segmented combine: (ha, a) then (hb, b) -> b restarts when its part holds a head.
__device__ __forceinline__ int64_t seg_combine(int op, bool hb, int64_t a, int64_t b) {
  return hb ? b : agg_combine(op, a, b);
}

template <typename K>
__global__ void __launch_bounds__(kSegWarps * 32) sgb_reduce_kernel(const K* __restrict__ key, int64_t n, Aggs A,
                                                                    K* __restrict__ out_keys, int64_t cap,
                                                                    int64_t* d_ngroups, int64_t* rec, int* counter,
                                                                    int64_t ntiles, int* err) {
  extern __shared__ __align__(16) int64_t s_dyn[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int nagg = A.n;
  int64_t* s_inc = s_dyn + (int64_t)warp * nagg * 32;            // [nagg][32] lane inclusive values
  int64_t* s_carry = s_dyn + (int64_t)kSegWarps * nagg * 32 + (int64_t)warp * (nagg + 2);
  const int rstride = 5 + 2 * nagg;  // flag | agg cnt, agg has | inc cnt, inc has | agg[nagg] | inc[nagg]

  int64_t tile = 0;
  if (lane == 0) tile = atomicAdd(counter, 1);
  tile = __shfl_sync(0xffffffffu, tile, 0);
  if (tile >= ntiles) return;
  const int64_t tb = tile * kSegTile;
  const int64_t rb = tb + (int64_t)lane * kSegItems;

  K k[kSegItems];
#pragma unroll
  for (int r = 0; r < kSegItems; ++r) k[r] = rb + r < n ? key[rb + r] : K(0);
  K prev_last = __shfl_up_sync(0xffffffffu, k[kSegItems - 1], 1);
  bool first_is_head;
  if (lane == 0)
    first_is_head = tb == 0 || key[tb - 1] != k[0];
  else
    first_is_head = prev_last != k[0];
  uint32_t hm = 0;  // head bits of valid rows
#pragma unroll
  for (int r = 0; r < kSegItems; ++r) {
    if (rb + r >= n) break;
    bool h = r == 0 ? first_is_head : (k[r] != k[r - 1]);
    if (h) hm |= 1u << r;
  }
  // does the row after this lane's last row start a new segment (or end the input)?
  uint32_t next_head = __shfl_down_sync(0xffffffffu, hm & 1u, 1);
  bool last_ends;
  const int64_t lastrow = rb + kSegItems - 1;
  if (lastrow + 1 >= n)
    last_ends = true;
  else if (lane == 31)
    last_ends = key[lastrow + 1] != k[kSegItems - 1];
  else
    last_ends = next_head != 0;

  const uint32_t heads = __popc(hm);
  const bool has = hm != 0;
  uint32_t hincl = heads;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    uint32_t y = __shfl_up_sync(0xffffffffu, hincl, o);
    if (lane >= o) hincl += y;
  }
  const uint32_t tile_heads = __shfl_sync(0xffffffffu, hincl, 31);
  const bool tile_has = __any_sync(0xffffffffu, has);
  // lanes before me hold a head?
  const unsigned has_mask = __ballot_sync(0xffffffffu, has);

  for (int j = 0; j < nagg; ++j) {
    const int op = A.op[j];
    int64_t tv = agg_identity(op);
    for (int r = 0; r < kSegItems; ++r) {
      const int64_t row = rb + r;
      if (row >= n) break;
      int64_t v = agg_value(A, j, row);
      tv = ((hm >> r) & 1u) ? v : agg_combine(op, tv, v);
    }
    // warp inclusive segmented scan over lanes
    bool h = has;
    int64_t x = tv;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      int64_t xp = __shfl_up_sync(0xffffffffu, x, o);
      bool hp = __shfl_up_sync(0xffffffffu, (int)h, o) != 0;
      if (lane >= o) {
        x = seg_combine(op, h, xp, x);
        h = h || hp;
      }
    }
    s_inc[j * 32 + lane] = x;
  }
  __syncwarp();

  // ---- publish the tile aggregate, look back, publish the inclusive record
  if (lane == 0) {
    int64_t* my = rec + tile * rstride;
    int64_t carry_cnt = 0;
    bool carry_has = false;
    for (int j = 0; j < nagg; ++j) s_carry[2 + j] = agg_identity(A.op[j]);
    if (tile > 0) {
      my[1] = tile_heads;
      my[2] = tile_has;
      for (int j = 0; j < nagg; ++j) my[5 + j] = s_inc[j * 32 + 31];
      __threadfence();
      st_volatile((uint64_t*)&my[0], 1);
      int64_t t = tile - 1;
      uint32_t spins = 0;
      while (t >= 0) {
        const int64_t* rt = rec + t * rstride;
        int64_t f = (int64_t)ld_volatile((const uint64_t*)&rt[0]);
        if (f == 0) {
          if (++spins > kSpinLimit) {
            set_status(err, GJ_ERR_TIMEOUT);
            break;
          }
          continue;
        }
        __threadfence();
        const int base = f == 2 ? 3 : 1;
        const int vbase = f == 2 ? 5 + nagg : 5;
        int64_t c = (int64_t)ld_volatile((const uint64_t*)&rt[base]);
        bool hh = ld_volatile((const uint64_t*)&rt[base + 1]) != 0;
        for (int j = 0; j < nagg; ++j) {
          int64_t v = (int64_t)ld_volatile((const uint64_t*)&rt[vbase + j]);
          if (!carry_has) s_carry[2 + j] = agg_combine(A.op[j], v, s_carry[2 + j]);
        }
        carry_cnt += c;
        carry_has = carry_has || hh;
        if (f == 2) break;
        --t;
      }
    }
    s_carry[0] = carry_cnt;
    s_carry[1] = carry_has;
    my[3] = carry_cnt + tile_heads;
    my[4] = carry_has || tile_has;
    for (int j = 0; j < nagg; ++j) my[5 + nagg + j] = seg_combine(A.op[j], tile_has, s_carry[2 + j], s_inc[j * 32 + 31]);
    __threadfence();
    st_volatile((uint64_t*)&my[0], 2);
    if (tile == ntiles - 1) *d_ngroups = carry_cnt + tile_heads;
  }
  __syncwarp();

  // ---- each lane walks its rows; a segment's value is written at its last row
  const int64_t cnt_before = s_carry[0] + (hincl - heads);
  const bool prev_lanes_have_head = (has_mask & ((1u << lane) - 1)) != 0;
  bool overflow = false;
  for (int j = 0; j < nagg; ++j) {
    const int op = A.op[j];
    int64_t run;
    if (lane == 0)
      run = s_carry[2 + j];
    else
      run = seg_combine(op, prev_lanes_have_head, s_carry[2 + j], s_inc[j * 32 + lane - 1]);
    int64_t gcount = cnt_before;
    for (int r = 0; r < kSegItems; ++r) {
      const int64_t row = rb + r;
      if (row >= n) break;
      int64_t v = agg_value(A, j, row);
      const bool h = (hm >> r) & 1u;
      if (h) {
        ++gcount;
        run = v;
      } else {
        run = agg_combine(op, run, v);
      }
      const bool ends = r == kSegItems - 1 ? last_ends : ((hm >> (r + 1)) & 1u) || row + 1 >= n;
      if (ends) {
        const int64_t gid = gcount - 1;
        if (gid < cap)
          A.out[j][gid] = run;
        else
          overflow = true;
      }
    }
  }
  {
    int64_t gcount = cnt_before;
    for (int r = 0; r < kSegItems; ++r) {
      if (rb + r >= n) break;
      if ((hm >> r) & 1u) {
        if (gcount < cap)
          out_keys[gcount] = k[r];
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
template <typename K>
__device__ int pgb_build(const K* __restrict__ key, int64_t r0, int64_t r1, int q, uint32_t round, int pbits,
                         int32_t* s_slots, K* s_keys, int* s_count, int* s_over) {
  for (int j = threadIdx.x; j < kPgbSlots; j += blockDim.x) s_slots[j] = 0;
  if (threadIdx.x == 0) {
    *s_count = 0;
    *s_over = 0;
  }
  __syncthreads();
  for (int64_t i = r0 + threadIdx.x; i < r1; i += blockDim.x) {
    if (*s_over) break;
    K k = key[i];
    if (pgb_sub<K>(k, q) != round) continue;
    uint32_t sl = pgb_slot<K>(k, pbits);
    volatile int32_t* vs = s_slots;
    volatile K* vk = s_keys;
    int probes = 0;
    uint32_t spins = 0;
    while (probes < kPgbSlots) {
      int v = vs[sl];
      if (v == 0) {
        // claim the slot (-1 = being written), then take a dense local id
        if (atomicCAS(&s_slots[sl], 0, -1) == 0) {
          int lid = atomicAdd(s_count, 1);
          if (lid >= kPgbCap) {
            *s_over = 1;
            atomicExch(&s_slots[sl], 0);
            break;
          }
          s_keys[lid] = k;
          __threadfence_block();
          atomicExch(&s_slots[sl], lid + 1);
          break;
        }
        continue;  // lost the race: re-read this slot
      }
      if (v < 0) {  // being written by another thread: re-read, with a bound
        if (++spins > kSpinLimit) {
          *s_over = 1;
          break;
        }
        continue;
      }
      if (vk[v - 1] == k) break;  // present
      sl = (sl + 1) & (kPgbSlots - 1);
      ++probes;
    }
  }
  __syncthreads();
  return *s_over ? -1 : *s_count;
}

template <typename K>
__device__ __forceinline__ int pgb_lookup(K k, int pbits, const int32_t* s_slots, const K* s_keys) {
  uint32_t sl = pgb_slot<K>(k, pbits);
  for (int probe = 0; probe < kPgbSlots; ++probe) {
    int v = s_slots[sl];
    if (v == 0) return -1;
    if (v > 0 && s_keys[v - 1] == k) return v - 1;
    sl = (sl + 1) & (kPgbSlots - 1);
  }
  return -1;
}

template <typename K>
__global__ void __launch_bounds__(kPgbThreads) pgb_kernel(const K* __restrict__ key,
                                                          const int64_t* __restrict__ poff, int64_t nparts,
                                                          int pbits, Aggs A, K* __restrict__ out_keys,
                                                          int64_t cap, int64_t* d_ngroups, uint64_t* pstat,
                                                          int* counter, int* err) {
  extern __shared__ __align__(16) unsigned char s_raw[];
  int64_t* s_agg = (int64_t*)s_raw;                       // kPgbCap aggregates
  int32_t* s_slots = (int32_t*)(s_agg + kPgbCap);         // table: local id + 1
  K* s_keys = (K*)(s_slots + kPgbSlots);                  // distinct keys by local id
  __shared__ int s_count, s_over;
  __shared__ int64_t s_part, s_goff;
  __shared__ int64_t s_red[kPgbThreads / 32];

  if (threadIdx.x == 0) s_part = atomicAdd(counter, 1);
  __syncthreads();
  const int64_t p = s_part;
  const int64_t r0 = poff[p], r1 = poff[p + 1];

  // ---- group discovery: the smallest split q whose sub-rounds all fit
  int q = 0;
  int64_t total = 0;
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
  if (threadIdx.x < 32) {
    const int64_t goff = (int64_t)lookback_scan_warp(pstat, p, (uint64_t)total, err);
    if (threadIdx.x == 0) {
      s_goff = goff;
      if (p == nparts - 1) *d_ngroups = goff + total;
    }
  }
  __syncthreads();
  if (q < 0) return;
  const int64_t goff = s_goff;

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

template <typename K>
constexpr size_t pgb_smem_bytes() {
  return (size_t)kPgbCap * 8 + (size_t)kPgbSlots * 4 + (size_t)kPgbCap * sizeof(K);
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
    const int budget = std::min(ctx.smem_optin, 200 * 1024);
    static bool attr = false;
    if (!attr) {
      cudaFuncSetAttribute(hgb_agg_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, budget);
      attr = true;
    }
    {
      LaunchScope ls(ctx, KK_HGB_AGG);
      hgb_agg_kernel<<<ctx.num_sms, 1024, budget, s>>>(gidloc, gid_of_row, n, A, L, d_ngroups, cap, budget);
    }
    return cuda_check(cudaGetLastError());
  }

  // ---- SGB-TR and PGB-TR: move the key with every aggregated column (GFTR)
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
  K* k2 = scr.get_as<K>(n);
  if (scr.failed()) return GJ_ERR_OOM;
  const void* moved[kMaxCols] = {nullptr};
  for (int c = 0; c < kMaxCols; ++c)
    if (colmap[c] >= 0) moved[c] = cs.dst[colmap[c]];
  Aggs A = make_aggs(in, nagg, ops, op_col, out_aggs, moved);
  const int kbits = sizeof(K) * 8;

  if (variant == GJ_GB_SGB) {
    if ((st = radix_partition_run(ctx, scr, sizeof(K) == 8 ? GJ_I64 : GJ_I32, in->key, k2, cs, n, 0, kbits,
                                  kSignedOrder, opt->bits_per_pass)) != GJ_OK)
      return st;
    const int64_t ntiles = (n + kSegTile - 1) / kSegTile;
    const int rstride = 5 + 2 * nagg;
    int64_t* rec = scr.get_as<int64_t>((size_t)ntiles * rstride);
    int* counter = scr.get_as<int>(1);
    if (scr.failed()) return GJ_ERR_OOM;
    if ((st = cuda_check(cudaMemsetAsync(rec, 0, sizeof(int64_t) * ntiles * rstride, s))) != GJ_OK) return st;
    if ((st = cuda_check(cudaMemsetAsync(counter, 0, sizeof(int), s))) != GJ_OK) return st;
    const size_t dyn = sizeof(int64_t) * ((size_t)kSegWarps * nagg * 32 + (size_t)kSegWarps * (nagg + 2));
    static bool attr[2] = {false, false};
    if (!attr[sizeof(K) == 8]) {
      cudaFuncSetAttribute(sgb_reduce_kernel<K>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)(sizeof(int64_t) * ((size_t)kSegWarps * kMaxAggs * 32 + kSegWarps * (kMaxAggs + 2))));
      attr[sizeof(K) == 8] = true;
    }
    const int64_t blocks = (ntiles + kSegWarps - 1) / kSegWarps;
    LaunchScope ls(ctx, KK_SGB_REDUCE);
    sgb_reduce_kernel<K><<<(unsigned)blocks, kSegWarps * 32, dyn, s>>>(k2, n, A, (K*)out_keys, cap, d_ngroups, rec,
                                                                       counter, ntiles, ctx.d_status);
    return cuda_check(cudaGetLastError());
  }

  // PGB-TR: partitions of about 2048 rows on hashed key bits (at most 16 bits)
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
    for (int c = 0; c < cs.n; ++c)
      if ((st = cuda_check(cudaMemcpyAsync(cs.dst[c], cs.src[c], (size_t)n * cs.size[c], cudaMemcpyDeviceToDevice,
                                           s))) != GJ_OK)
        return st;
  }
  int64_t* poff = scr.get_as<int64_t>(nparts + 1);
  uint64_t* pstat = scr.get_as<uint64_t>(nparts);
  int* counter = scr.get_as<int>(1);
  if (scr.failed()) return GJ_ERR_OOM;
  if ((st = partition_bounds_run(ctx, sizeof(K) == 8 ? GJ_I64 : GJ_I32, k2, n, 0, bits, kHashed, poff)) != GJ_OK)
    return st;
  if ((st = cuda_check(cudaMemsetAsync(pstat, 0, sizeof(uint64_t) * nparts, s))) != GJ_OK) return st;
  if ((st = cuda_check(cudaMemsetAsync(counter, 0, sizeof(int), s))) != GJ_OK) return st;
  const size_t dyn = pgb_smem_bytes<K>();
  static bool attr[2] = {false, false};
  if (!attr[sizeof(K) == 8]) {
    cudaFuncSetAttribute(pgb_kernel<K>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn);
    attr[sizeof(K) == 8] = true;
  }
  LaunchScope ls(ctx, KK_PGB);
  pgb_kernel<K><<<(unsigned)nparts, kPgbThreads, dyn, s>>>(k2, poff, nparts, bits, A, (K*)out_keys, cap, d_ngroups,
                                                           pstat, counter, ctx.d_status);
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

gj_status groupby_run(const Ctx& ctx, const gj_table* in, int nagg, const int32_t* ops, const int32_t* op_col,
                      const gj_options* opt, void* out_keys, int64_t* const* out_aggs, int64_t cap,
                      int64_t* d_ngroups) {
  int variant = opt->groupby_variant;
  if (variant == GJ_GB_AUTO && opt->selector == GJ_SELECT_MLP) variant = mlp_choose(nullptr, in, nagg, opt, false);
  if (variant == GJ_GB_AUTO) variant = choose_groupby_variant(in, nagg, ops, opt, std::min(ctx.smem_optin, 200 * 1024));
  if (in->key_type == GJ_I64)
    return groupby_typed<int64_t>(ctx, in, nagg, ops, op_col, opt, variant, out_keys, out_aggs, cap, d_ngroups);
  return groupby_typed<int32_t>(ctx, in, nagg, ops, op_col, opt, variant, out_keys, out_aggs, cap, d_ngroups);
}

}  // namespace gj
