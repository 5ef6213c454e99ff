// Joins (paper Sec. 3.1 and 4.1.4).
//
// PHJ-TR / PHJ-UR: both relations are radix-partitioned on hashed key bits with
// the stable radix-partition primitive (contiguous partitions, bounds from a
// histogram-like pass), then matches are found with a shared-memory hash table
// per build-side partition, and the result is materialised.
//   * TR (GFTR, Sec. 4.1.2 / 4.1.4): payload columns are partitioned together
//     with the key, so S payloads are read sequentially and R payloads from the
//     small, contiguous partition R'_p (clustered).
//   * UR (GFUR, Fig. gfur): (key, tuple id) pairs are partitioned and payloads
//     are gathered from the untransformed inputs through the ids.
// The probe side is walked in fixed-size units of the partitioned S'. A unit
// covers the tail of one partition, whole partitions or a slice of a large
// one; a table of R'_p is built once per unit that holds rows of partition p
// (the paper's decomposition of large probe partitions, Sec. 3.1.2 / 4.1.4, by
// construction), so skewed foreign keys do not unbalance the blocks. Output
// positions come from a decoupled look-back over units, so the result is
// compact, ordered by S' and identical on every run. The fused join->group-by
// walks the same partitions in tiles of kTileS rows.
//
// NPHJ (Sec. 3.1.3): one global open-addressing table on R (key -> row), S
// probed in its own order; R payloads are gathered randomly, S sequentially.
#include <cuda_runtime.h>

#include <algorithm>

#include "gj_internal.cuh"

namespace gj {

namespace {

constexpr int kThreads = 256;
constexpr int kTileS = 2048;          // probe rows per tile
constexpr int kItems = kTileS / kThreads;
constexpr int kBuildCap = 1024;       // build rows per shared-memory table
constexpr int kSlots = 2 * kBuildCap; // load factor <= 1/2

struct JoinIO {
  // R side: value of R column c for match m = rsrc[c][ r_tid ? r_tid[m] : m ]
  const void* rsrc[kMaxCols];
  int32_t rsize[kMaxCols];
  int32_t nr_cols;
  const int32_t* r_tid;  // UR: tuple ids carried through the partitioning of R
  // S side: value of S column c for probe row i = ssrc[c][ s_tid ? s_tid[i] : i ]
  const void* ssrc[kMaxCols];
  int32_t ssize[kMaxCols];
  int32_t ns_cols;
  const int32_t* s_tid;
  // T
  void* tkey;
  void* tcols[2 * kMaxCols];
  int64_t cap;
  int64_t* d_count;
  int32_t stage_bulk;  // 1: probe keys 16-byte aligned, bulk-copied into shared memory
  int32_t narrow4;     // 1: every payload column 4 bytes wide, at most 4 per side
  // GFTR with four 4-byte payloads on a side: that side's partitioned payloads as
  // interleaved 16-byte rows (one load per row) instead of rsrc / ssrc
  const int4* r_zip;
  const int4* s_zip;
};

template <typename K>
__device__ __forceinline__ uint32_t smem_slot(K k, int pbits) {
  uint64_t h = KeyTraits<K>::hash64(k);
  return (uint32_t)(h >> pbits) & (kSlots - 1);
}

// Copies g (<= G) consecutive T columns starting at c for the thread's kItems rows.
template <typename T, int G>
__device__ __forceinline__ void emit_group(const JoinIO& io, int c, int g, bool rside, const uint32_t* idx,
                                           const uint32_t* o, const bool* ok) {
  // loads are unconditional (rows without a match read row 0, which exists), so
  // nothing orders them after one another: all G x kItems are in flight at once.
  T v[G][kItems];
#pragma unroll
  for (int q = 0; q < G; ++q) {
    const int cq = c + (q < g ? q : 0);
    const T* __restrict__ src = (const T*)(rside ? io.rsrc[cq] : io.ssrc[cq - io.nr_cols]);
#pragma unroll
    for (int j = 0; j < kItems; ++j) {
      const uint32_t r = ok[j] ? idx[j] : 0u;
      v[q][j] = rside ? __ldg(src + r) : __ldcs(src + r);
    }
  }
#pragma unroll
  for (int q = 0; q < G; ++q) {
    T* __restrict__ dst = (T*)io.tcols[c + (q < g ? q : 0)];
#pragma unroll
    for (int j = 0; j < kItems; ++j)
      if (q < g && ok[j]) __stcs(dst + o[j], v[q][j]);
  }
}

// Compaction + materialisation of one probe tile. s_midx[i] is the matching
// build row (index into the R-side source arrays, or into r_tid) or -1.
template <typename K>
__device__ void emit_tile(int64_t tile, int64_t ntiles, int64_t tile_base, int tile_n, const K* s_key,
                          const int32_t* s_midx, int32_t* s_pos, const JoinIO& io, uint64_t* tile_status,
                          int* err, uint32_t* s_scan, uint64_t* s_base) {
  const int t = threadIdx.x;
  // blocked exclusive scan of match flags
  uint32_t cnt = 0;
#pragma unroll
  for (int j = 0; j < kItems; ++j) {
    int i = t * kItems + j;
    cnt += (i < tile_n && s_midx[i] >= 0) ? 1u : 0u;
  }
  const int lane = t & 31, warp = t >> 5;
  uint32_t x = cnt;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) s_scan[warp] = x;
  __syncthreads();
  if (warp == 0) {
    uint32_t run = 0;
    for (int w = 0; w < kThreads / 32; ++w) run += s_scan[w];
    __syncwarp();
    if (lane == 0) {
      uint32_t r = 0;
      for (int w = 0; w < kThreads / 32; ++w) {
        const uint32_t c = s_scan[w];
        s_scan[w] = r;
        r += c;
      }
    }
    const uint64_t excl = lookback_scan_warp(tile_status, tile, run, err);
    if (lane == 0) {
      *s_base = excl;
      if (tile == ntiles - 1 && io.d_count) *io.d_count = (int64_t)(excl + run);
    }
  }
  __syncthreads();
  uint32_t pos = s_scan[warp] + x - cnt;
#pragma unroll
  for (int j = 0; j < kItems; ++j) {
    int i = t * kItems + j;
    if (i < tile_n && s_midx[i] >= 0) s_pos[i] = (int32_t)pos++;
  }
  __syncthreads();
  // Each thread owns rows t, t + kThreads, ...: outputs of a warp are contiguous.
  // All loads of a column are issued before its stores, so a thread keeps
  // kItems gathers in flight instead of waiting on one at a time.
  const int64_t base = (int64_t)*s_base;
  const int64_t cap = io.cap;
  // output rows < cap and source rows < 2^30: 32-bit indices
  uint32_t o[kItems], ridx[kItems], sidx[kItems];
  bool ok[kItems];
  bool overflow = false;
#pragma unroll
  for (int j = 0; j < kItems; ++j) {
    const int i = t + j * kThreads;
    const int32_t m = i < tile_n ? s_midx[i] : -1;
    const int64_t oo = m >= 0 ? base + s_pos[i] : 0;
    ok[j] = m >= 0 && oo < cap;
    overflow |= m >= 0 && oo >= cap;
    o[j] = (uint32_t)oo;
    ridx[j] = (uint32_t)m;
    sidx[j] = (uint32_t)(tile_base + i);
  }
  if (overflow) set_status(err, GJ_ERR_CAPACITY);
  if (io.r_tid) {
#pragma unroll
    for (int j = 0; j < kItems; ++j)
      if (ok[j]) ridx[j] = (uint32_t)__ldg(io.r_tid + ridx[j]);
  }
  if (io.s_tid) {
#pragma unroll
    for (int j = 0; j < kItems; ++j)
      if (ok[j]) sidx[j] = (uint32_t)__ldcs(io.s_tid + sidx[j]);
  }
  {
    K* __restrict__ tk = (K*)io.tkey;
#pragma unroll
    for (int j = 0; j < kItems; ++j)
      if (ok[j]) __stcs(tk + o[j], s_key[t + j * kThreads]);
  }
  // columns in groups of one width and side (two 4-byte or one 8-byte column):
  // all loads of a group are in flight before its first store
  const int ncols = io.nr_cols + io.ns_cols;
  int c = 0;
  while (c < ncols) {
    const bool rside = c < io.nr_cols;
    const int size = rside ? io.rsize[c] : io.ssize[c - io.nr_cols];
    const int gmax = size == 8 ? 1 : 2;
    int g = 1;
    while (g < gmax && c + g < ncols && (c + g < io.nr_cols) == rside &&
           (rside ? io.rsize[c + g] : io.ssize[c + g - io.nr_cols]) == size)
      ++g;
    const uint32_t* idx = rside ? ridx : sidx;
    if (size == 8)
      emit_group<int64_t, 1>(io, c, g, rside, idx, o, ok);
    else
      emit_group<int32_t, 2>(io, c, g, rside, idx, o, ok);
    c += g;
  }
}

// Shared memory of one probe tile walked by probe_tile: probe keys, partition and
// match of each row, the table and the build chunk's keys.
template <typename K>
constexpr size_t phj_smem_bytes() {
  return (size_t)kTileS * sizeof(K) + 2 * (size_t)kTileS * 4 + (size_t)kSlots * 4 + (size_t)kBuildCap * sizeof(K);
}

// Finds, for every probe row of S'[tile_base, tile_base + tile_n), the build row
// of R' with the same key (s_midx, -1 = none): one shared-memory table per build
// partition (or per chunk of kBuildCap rows of it) present in the tile.
template <typename K>
__device__ void probe_tile(const K* __restrict__ rkey, const int64_t* __restrict__ roff, int pbits,
                           const K* __restrict__ skey, int64_t tile_base, int tile_n, K* s_key, int32_t* s_part,
                           int32_t* s_midx, int32_t* s_slots, K* s_rkey, int* err) {
  const int t = threadIdx.x;
  const uint32_t pmask = pbits >= 32 ? 0xffffffffu : ((1u << pbits) - 1);
#pragma unroll 8
  for (int i = t; i < tile_n; i += kThreads) {
    K k = __ldcs(skey + tile_base + i);
    s_key[i] = k;
    s_part[i] = (int32_t)((uint32_t)KeyTraits<K>::hash64(k) & pmask);
    s_midx[i] = -1;
  }
  __syncthreads();

  // walk the partitions present in this tile (non-decreasing in S')
  int a = 0;
  while (a < tile_n) {
    const int32_t p = s_part[a];
    int lo = a, hi = tile_n;  // first row with partition > p
    while (lo < hi) {
      int mid = (lo + hi) >> 1;
      if (s_part[mid] <= p) lo = mid + 1; else hi = mid;
    }
    const int b = lo;
    const int64_t r_lo = roff[p], r_hi = roff[p + 1];
    for (int64_t c0 = r_lo; c0 < r_hi; c0 += kBuildCap) {
      const int cn = (int)min64(kBuildCap, r_hi - c0);
      for (int j = t; j < kSlots; j += kThreads) s_slots[j] = 0;
      // stage the chunk's keys first so the loads overlap, then insert
#pragma unroll 8
      for (int j = t; j < cn; j += kThreads) s_rkey[j] = __ldg(rkey + c0 + j);
      __syncthreads();
      for (int j = t; j < cn; j += kThreads) {
        const K k = s_rkey[j];
        uint32_t sl = smem_slot<K>(k, pbits);
        for (int probe = 0; probe < kSlots; ++probe) {
          int prev = atomicCAS(&s_slots[sl], 0, j + 1);
          if (prev == 0) break;
          if (s_rkey[prev - 1] == k) {
            set_status(err, GJ_ERR_DUPLICATE_KEY);
            break;
          }
          sl = (sl + 1) & (kSlots - 1);
        }
      }
      __syncthreads();
      for (int i = a + t; i < b; i += kThreads) {
        K k = s_key[i];
        uint32_t sl = smem_slot<K>(k, pbits);
        for (int probe = 0; probe < kSlots; ++probe) {
          int v = s_slots[sl];
          if (v == 0) break;
          if (s_rkey[v - 1] == k) {
            if (s_midx[i] >= 0) set_status(err, GJ_ERR_DUPLICATE_KEY);
            s_midx[i] = (int32_t)(c0 + v - 1);
            break;
          }
          sl = (sl + 1) & (kSlots - 1);
        }
      }
      __syncthreads();
    }
    a = b;
  }
  __syncthreads();
}

// ---------------------------------------------------------------- PHJ probe by units
// A block takes a unit of kUnitRows consecutive rows of S' (taken in order from a
// counter). Phase 1 walks the unit in sub-tiles of kTileS rows whose keys arrive
// by bulk copy into a double buffer (the next sub-tile's copy is in flight while
// the current one is probed) and finds each row's build row; the table of the
// partition last built stays resident, so a partition spanning sub-tiles is
// built once per unit. Phase 2 takes the unit's output offset from a decoupled
// look-back over units and materialises the matches: every warp owns a
// contiguous range of the unit and writes it without block barriers, all loads
// of a group of columns in flight before its stores.
constexpr int kUnitSub = 2;                   // sub-tiles per unit
constexpr int kUnitRows = kUnitSub * kTileS;  // probe rows per unit
constexpr int kRoffCache = 64;              // partition bounds cached per unit
constexpr int kEmitU = 4;                     // rows per lane per emit step

template <typename K>
constexpr size_t phj_unit_smem_bytes() {
  return (size_t)kUnitRows * 4 + 2 * (size_t)kTileS * sizeof(K) + (size_t)kSlots * 4 + (size_t)kBuildCap * sizeof(K);
}

// T columns c .. c + g - 1 (g <= G, one side and one width) for U rows per lane:
// every load is issued before the first store. Rows without a match load row 0.
template <typename T, int G, int U>
__device__ __forceinline__ void emit_cols(const JoinIO& io, int c, int g, bool rside, const uint32_t (&idx)[U],
                                          const uint32_t (&o)[U], const bool (&ok)[U]) {
  T v[G][U];
#pragma unroll
  for (int q = 0; q < G; ++q) {
    const int cq = c + (q < g ? q : 0);
    const T* __restrict__ src = (const T*)(rside ? io.rsrc[cq] : io.ssrc[cq - io.nr_cols]);
#pragma unroll
    for (int j = 0; j < U; ++j) {
      const uint32_t r = ok[j] ? idx[j] : 0u;
      v[q][j] = rside ? __ldg(src + r) : __ldcs(src + r);
    }
  }
#pragma unroll
  for (int q = 0; q < G; ++q) {
    T* __restrict__ dst = (T*)io.tcols[c + (q < g ? q : 0)];
#pragma unroll
    for (int j = 0; j < U; ++j)
      if (q < g && ok[j]) __stcs(dst + o[j], v[q][j]);
  }
}

// One warp materialises unit rows [w0, wend) (s_midx[r]: the build row of unit
// row r, or -1) at output positions from `pos` on, in row order; all loads of a
// group of columns are in flight before its stores. Returns true when a match fell
// beyond the output capacity (its row is dropped).
template <typename K>
__device__ __forceinline__ bool emit_range(const K* __restrict__ skey, int64_t u0, int w0, int wend, int64_t pos,
                                           const int32_t* s_midx, const JoinIO& io) {
  const int lane = threadIdx.x & 31;
  const int64_t cap = io.cap;
  const unsigned lt = (1u << lane) - 1;
  const int ncols = io.nr_cols + io.ns_cols;
  bool overflow = false;
  for (int b0 = w0; b0 < wend; b0 += 32 * kEmitU) {
    uint32_t o[kEmitU], ridx[kEmitU], sidx[kEmitU];
    bool ok[kEmitU];
#pragma unroll
    for (int j = 0; j < kEmitU; ++j) {
      const int r = b0 + j * 32 + lane;
      const int32_t m = r < wend ? s_midx[r] : -1;
      const unsigned bal = __ballot_sync(0xffffffffu, m >= 0);
      const int64_t oo = pos + __popc(bal & lt);
      pos += __popc(bal);
      ok[j] = m >= 0 && oo < cap;
      overflow |= m >= 0 && oo >= cap;
      o[j] = (uint32_t)oo;
      ridx[j] = (uint32_t)m;
      sidx[j] = (uint32_t)(u0 + r);
    }
    if (io.r_tid) {
#pragma unroll
      for (int j = 0; j < kEmitU; ++j) ridx[j] = ok[j] ? (uint32_t)__ldg(io.r_tid + ridx[j]) : 0u;
    }
    if (io.s_tid) {
#pragma unroll
      for (int j = 0; j < kEmitU; ++j) sidx[j] = ok[j] ? (uint32_t)__ldcs(io.s_tid + sidx[j]) : 0u;
    }
    {
      K kv[kEmitU];
#pragma unroll
      for (int j = 0; j < kEmitU; ++j) kv[j] = skey[ok[j] ? u0 + b0 + j * 32 + lane : u0];
      K* __restrict__ tk = (K*)io.tkey;
#pragma unroll
      for (int j = 0; j < kEmitU; ++j)
        if (ok[j]) __stcs(tk + o[j], kv[j]);
    }
    if (io.narrow4) {
      // every column 4 bytes wide, at most 4 per side: all loads of the step in flight together
      int32_t vr[4][kEmitU], vs[4][kEmitU];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int32_t* __restrict__ rs = (const int32_t*)io.rsrc[q < io.nr_cols ? q : 0];
        const int32_t* __restrict__ ss = (const int32_t*)io.ssrc[q < io.ns_cols ? q : 0];
#pragma unroll
        for (int j = 0; j < kEmitU; ++j) {
          vr[q][j] = (q < io.nr_cols && !io.r_zip) ? __ldg(rs + (ok[j] ? ridx[j] : 0u)) : 0;
          vs[q][j] = (q < io.ns_cols && !io.s_zip) ? __ldcs(ss + (ok[j] ? sidx[j] : 0u)) : 0;
        }
      }
      if (io.r_zip) {
#pragma unroll
        for (int j = 0; j < kEmitU; ++j) {
          const int4 v = __ldg(io.r_zip + (ok[j] ? ridx[j] : 0u));
          vr[0][j] = v.x;
          vr[1][j] = v.y;
          vr[2][j] = v.z;
          vr[3][j] = v.w;
        }
      }
      if (io.s_zip) {
#pragma unroll
        for (int j = 0; j < kEmitU; ++j) {
          const int4 v = __ldcs(io.s_zip + (ok[j] ? sidx[j] : 0u));
          vs[0][j] = v.x;
          vs[1][j] = v.y;
          vs[2][j] = v.z;
          vs[3][j] = v.w;
        }
      }
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        int32_t* __restrict__ dr = (int32_t*)io.tcols[q < io.nr_cols ? q : 0];
        int32_t* __restrict__ ds = (int32_t*)io.tcols[io.nr_cols + (q < io.ns_cols ? q : 0)];
#pragma unroll
        for (int j = 0; j < kEmitU; ++j) {
          if (q < io.nr_cols && ok[j]) __stcs(dr + o[j], vr[q][j]);
          if (q < io.ns_cols && ok[j]) __stcs(ds + o[j], vs[q][j]);
        }
      }
      continue;
    }
    int c = 0;
    while (c < ncols) {
      const bool rside = c < io.nr_cols;
      const int size = rside ? io.rsize[c] : io.ssize[c - io.nr_cols];
      const int gmax = size == 8 ? 2 : 4;
      int g = 1;
      while (g < gmax && c + g < ncols && (c + g < io.nr_cols) == rside &&
             (rside ? io.rsize[c + g] : io.ssize[c + g - io.nr_cols]) == size)
        ++g;
      if (size == 8)
        emit_cols<int64_t, 2, kEmitU>(io, c, g, rside, rside ? ridx : sidx, o, ok);
      else
        emit_cols<int32_t, 4, kEmitU>(io, c, g, rside, rside ? ridx : sidx, o, ok);
      c += g;
    }
  }
  return overflow;
}

// Output offset of a probe unit (decoupled look-back over units) and the
// materialisation of its matches: s_midx[r] is the build row of unit row r (or
// -1). Every warp owns a contiguous range of the unit and writes it without
// block barriers, all loads of a group of columns in flight before its stores.
// Called by all threads of the block after s_midx is complete.
template <typename K, int NT = kThreads>
__device__ __forceinline__ void phj_emit_unit(const K* __restrict__ skey, int64_t u0, int un, int64_t unit,
                                              int64_t nunits, const int32_t* s_midx, const JoinIO& io,
                                              uint64_t* unit_status, int* err, uint32_t* s_wcnt, uint64_t* s_base_p) {
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  uint64_t& s_base = *s_base_p;
  constexpr int kWarpRows = kUnitRows / (NT / 32);
  const int w0 = warp * kWarpRows, wend = min(w0 + kWarpRows, un);
  uint32_t cnt = 0;
  for (int i = w0 + lane; i < wend; i += 32) cnt += s_midx[i] >= 0 ? 1u : 0u;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
  if (lane == 0) s_wcnt[warp] = cnt;
  __syncthreads();
  if (warp == 0) {
    uint32_t tot = lane < NT / 32 ? s_wcnt[lane] : 0u;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) tot += __shfl_xor_sync(0xffffffffu, tot, o);
    const uint64_t excl = lookback_scan_warp(unit_status, unit, tot, err);
    if (lane == 0) {
      s_base = excl;
      if (unit == nunits - 1 && io.d_count) *io.d_count = (int64_t)(excl + tot);
    }
  }
  __syncthreads();

  // ---- phase 2: each warp materialises its range, no block barriers
  int64_t pos = (int64_t)s_base;
  for (int w = 0; w < warp; ++w) pos += s_wcnt[w];
  if (emit_range<K>(skey, u0, w0, wend, pos, s_midx, io)) set_status(err, GJ_ERR_CAPACITY);
}

template <typename K>
__global__ void __launch_bounds__(kThreads, 4) phj_unit_kernel(const K* __restrict__ rkey,
                                                            const int64_t* __restrict__ roff, int pbits,
                                                            const K* __restrict__ skey, int64_t ns, JoinIO io,
                                                            uint64_t* unit_status, int* unit_counter, int64_t nunits,
                                                            int* err) {
  extern __shared__ __align__(128) unsigned char s_raw[];
  int32_t* s_midx = (int32_t*)s_raw;                 // kUnitRows: matching build row or -1
  K* s_kbuf = (K*)(s_midx + kUnitRows);              // 2 x kTileS probe keys
  int32_t* s_slots = (int32_t*)(s_kbuf + 2 * kTileS);  // table: build row + 1, 0 = empty
  K* s_rkey = (K*)(s_slots + kSlots);                 // keys of the resident build chunk
  __shared__ __align__(8) uint64_t s_bar[2];
  __shared__ int64_t s_unit;
  __shared__ uint32_t s_wcnt[kThreads / 32];
  __shared__ uint64_t s_base;
  __shared__ int64_t s_roff[kRoffCache];  // roff[s_p0 .. s_p0 + s_nroff) of the unit's partitions
  __shared__ uint32_t s_p0;
  __shared__ int s_nroff;

  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  if (t == 0) {
    s_unit = atomicAdd(unit_counter, 1);
    mbar_init(&s_bar[0], 1);
    mbar_init(&s_bar[1], 1);
    mbar_fence_init();
  }
  __syncthreads();
  const int64_t unit = s_unit;
  if (unit >= nunits) return;
  const int64_t u0 = unit * kUnitRows;
  const int un = (int)min64(kUnitRows, ns - u0);
  const int nsub = (un + kTileS - 1) / kTileS;
  const uint32_t pmask = pbits >= 32 ? 0xffffffffu : ((1u << pbits) - 1);

  // ---- phase 1: build rows of every probe row of the unit
  // the 16-byte aligned body of sub-tile k's keys is bulk-copied into buffer k & 1
  auto body_rows = [&](int k) {
    const int rows = min(kTileS, un - k * kTileS);
    return io.stage_bulk ? (int)((((uint32_t)rows * sizeof(K)) & ~15u) / sizeof(K)) : 0;
  };
  if (t == 0) {
    const uint32_t kb = (uint32_t)body_rows(0) * sizeof(K);
    mbar_expect_tx(&s_bar[0], kb);
    if (kb) bulk_g2s(s_kbuf, skey + u0, kb, &s_bar[0]);
  }
  // while the keys arrive, one warp fetches the partition bounds the unit needs:
  // its rows are sorted by partition, so they lie between those of its first and
  // last row
  if (warp == 0) {
    uint32_t p0 = 0, p1 = 0;
    if (lane == 0) {
      const K kf = skey[u0], kl = skey[u0 + un - 1];
      p0 = (uint32_t)KeyTraits<K>::hash64(kf) & pmask;
      p1 = (uint32_t)KeyTraits<K>::hash64(kl) & pmask;
    }
    p0 = __shfl_sync(0xffffffffu, p0, 0);
    p1 = __shfl_sync(0xffffffffu, p1, 0);
    const int nr = min((int)(p1 - p0) + 2, kRoffCache);
    for (int e = lane; e < nr; e += 32) s_roff[e] = roff[p0 + e];
    if (lane == 0) {
      s_p0 = p0;
      s_nroff = nr;
    }
  }
  int64_t cur_p = -1;  // partition whose whole build side is in the table
  for (int k = 0; k < nsub; ++k) {
    const int rows = min(kTileS, un - k * kTileS);
    K* kb = s_kbuf + (k & 1) * kTileS;
    int32_t* mid = s_midx + k * kTileS;
    const int64_t sbase = u0 + (int64_t)k * kTileS;
    __syncthreads();  // sub-tile k - 1 is done with its buffer: it takes sub-tile k + 1
    if (t == 0 && k + 1 < nsub) {
      fence_proxy_async();  // the buffer's previous contents were read and written by threads
      const uint32_t nb = (uint32_t)body_rows(k + 1) * sizeof(K);
      mbar_expect_tx(&s_bar[(k + 1) & 1], nb);
      if (nb) bulk_g2s(s_kbuf + ((k + 1) & 1) * kTileS, skey + sbase + kTileS, nb, &s_bar[(k + 1) & 1]);
    }
    for (int i = body_rows(k) + t; i < rows; i += kThreads) kb[i] = skey[sbase + i];
    mbar_wait(&s_bar[k & 1], (uint32_t)((k >> 1) & 1), err);
    __syncthreads();
    // the partitions present in the sub-tile (non-decreasing in S')
    auto part_of = [&](int i) { return (uint32_t)KeyTraits<K>::hash64(kb[i]) & pmask; };
    int a = 0;
    while (a < rows) {
      const uint32_t p = part_of(a);
      int lo = a, hi = rows;  // first row with partition > p
      while (lo < hi) {
        const int m = (lo + hi) >> 1;
        if (part_of(m) <= p) lo = m + 1; else hi = m;
      }
      const int b = lo;
      const int e = (int)(p - s_p0);  // the unit's partitions come from its bound cache
      const int64_t r_lo = e + 1 < s_nroff ? s_roff[e] : roff[p];
      const int64_t r_hi = e + 1 < s_nroff ? s_roff[e + 1] : roff[p + 1];
      // rows of a partition without build rows match nothing
      if (r_hi == r_lo)
        for (int i = a + t; i < b; i += kThreads) mid[i] = -1;
      const bool whole = r_hi - r_lo <= kBuildCap;
      for (int64_t c0 = r_lo; c0 < r_hi; c0 += kBuildCap) {
        const int cn = (int)min64(kBuildCap, r_hi - c0);
        if (!(whole && p == cur_p)) {
          for (int j = t; j < kSlots; j += kThreads) s_slots[j] = 0;
#pragma unroll 8
          for (int j = t; j < cn; j += kThreads) s_rkey[j] = __ldg(rkey + c0 + j);
          __syncthreads();
          for (int j = t; j < cn; j += kThreads) {
            const K kk = s_rkey[j];
            uint32_t sl = smem_slot<K>(kk, pbits);
            for (int probe = 0; probe < kSlots; ++probe) {
              const int prev = atomicCAS(&s_slots[sl], 0, j + 1);
              if (prev == 0) break;
              if (s_rkey[prev - 1] == kk) {
                set_status(err, GJ_ERR_DUPLICATE_KEY);
                break;
              }
              sl = (sl + 1) & (kSlots - 1);
            }
          }
          __syncthreads();
        }
        // the first chunk decides every row (match or -1); later chunks of a large
        // partition only add matches
        const bool first_chunk = c0 == r_lo;
        for (int i = a + t; i < b; i += kThreads) {
          const K kk = kb[i];
          uint32_t sl = smem_slot<K>(kk, pbits);
          int32_t m = -1;
          for (int probe = 0; probe < kSlots; ++probe) {
            const int v = s_slots[sl];
            if (v == 0) break;
            if (s_rkey[v - 1] == kk) {
              m = (int32_t)(c0 + v - 1);
              break;
            }
            sl = (sl + 1) & (kSlots - 1);
          }
          if (first_chunk) {
            mid[i] = m;
          } else if (m >= 0) {
            if (mid[i] >= 0) set_status(err, GJ_ERR_DUPLICATE_KEY);
            mid[i] = m;
          }
        }
        __syncthreads();  // the table may be rebuilt next
      }
      if (r_hi > r_lo) cur_p = whole ? (int64_t)p : -1;
      a = b;
    }
  }
  // the last partition may have had no build rows: its -1 entries were written
  // without a barrier after them
  __syncthreads();
  phj_emit_unit<K>(skey, u0, un, unit, nunits, s_midx, io, unit_status, err, s_wcnt, &s_base);
}

// ---------------------------------------------------------------- PHJ, L2-sized partitions
// With a large build side, one 8-bit hashed pass per side replaces the two passes
// that shared-memory-sized partitions need. Each of the 256 build partitions R'_P
// gets an open-addressing table in global memory at toff[P] (a power of two of
// at least twice its rows, holding R' row + 1), built once; a probe unit of S'
// rows of partition P looks its keys up there. R'_P and its table (a few MB) stay
// in the 129 MB L2 while the units of S'_P run, so the gathers from R'_P are
// clustered in L2 the way GFTR clusters them in shared memory for small
// partitions. Output offsets and materialisation are those of phj_unit_kernel.
constexpr int kL2Parts = 256;
constexpr int kL2Bits = 8;

// toff[P] = sum of the table sizes of partitions < P, toff[kL2Parts] = the total.
__global__ void __launch_bounds__(kL2Parts) l2_table_offsets_kernel(const int64_t* __restrict__ roff,
                                                                   int64_t* __restrict__ toff) {
  __shared__ int64_t s[kL2Parts];
  const int p = threadIdx.x;
  const int64_t rows = roff[p + 1] - roff[p];
  int64_t sz = 2;
  while (sz < 2 * rows) sz <<= 1;
  s[p] = sz;
  __syncthreads();
  for (int o = 1; o < kL2Parts; o <<= 1) {
    const int64_t v = p >= o ? s[p - o] : 0;
    __syncthreads();
    s[p] += v;
    __syncthreads();
  }
  toff[p + 1] = s[p];
  if (p == 0) toff[0] = 0;
}

// Table entries: for 4-byte keys one 64-bit word, (row + 1) << 32 | key, claimed
// by a single compare-and-swap, so a probe reads key and row in one access; for
// 8-byte keys a 32-bit row + 1 with the key compared in R'.
template <typename K>
struct L2Slot;
template <>
struct L2Slot<int32_t> {
  using W = unsigned long long;
  static constexpr int kWords = 2;  // int32 words per entry
  static __device__ __forceinline__ W make(int32_t k, int64_t i) {
    return ((W)(uint32_t)(i + 1) << 32) | (W)(uint32_t)k;
  }
};
template <>
struct L2Slot<int64_t> {
  using W = int32_t;
  static constexpr int kWords = 1;
};

// Build: blocks take chunks of R' in order from a counter, so the tables being
// filled at any time are those of a few neighbouring partitions (in L2).
constexpr int kL2BuildChunk = 1024;  // rows per build chunk (measured: 0.74 ms at 2^25 rows, 0.94 ms for 4096, 1.05 ms for 256)
// A partition's table is cleared just before it is filled, by the blocks whose
// chunks reach it (in segments of kL2ClearWords words taken from a per-partition
// counter), so its lines are written to L2 and filled there instead of being
// cleared to DRAM by a separate pass and read back. A chunk covers the partitions
// of its rows and any empty ones up to the next chunk's first partition; the
// first and last chunks also cover the partitions before and after all rows.
constexpr int kL2ClearWords = 8192;  // 32 KB per clearing segment

__device__ __forceinline__ int l2_part_of_hash(uint64_t h) { return (int)(h & (kL2Parts - 1)); }

template <typename K>
__device__ __forceinline__ void l2_clear_partition(int p, const int64_t* __restrict__ toff, int32_t* table, int kw,
                                                   int* pseg, int* pdone, int* s_seg, int* err) {
  const int64_t w0 = toff[p] * kw, w1 = toff[p + 1] * kw;  // even word counts: 8-byte stores
  const int nseg = (int)((w1 - w0 + kL2ClearWords - 1) / kL2ClearWords);
  for (;;) {
    if (threadIdx.x == 0) *s_seg = atomicAdd(&pseg[p], 1);
    __syncthreads();
    const int seg = *s_seg;
    __syncthreads();
    if (seg >= nseg) break;
    const int64_t a = w0 + (int64_t)seg * kL2ClearWords, b = min64(w1, a + kL2ClearWords);
    for (int64_t e = a + 2 * threadIdx.x; e < b; e += 2 * blockDim.x)
      *reinterpret_cast<uint2*>(table + e) = make_uint2(0u, 0u);
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) atomicAdd(&pdone[p], 1);
  }
  // every segment of the partition cleared (by this block or others)
  if (threadIdx.x == 0) {
    WaitGuard guard(err);
    while (*(volatile int*)&pdone[p] < nseg) {
      if (guard.expired()) {
        set_status(err, GJ_ERR_TIMEOUT);
        break;
      }
    }
    __threadfence();
  }
  __syncthreads();
}

template <typename K>
__global__ void __launch_bounds__(256) l2_build_kernel(const K* __restrict__ rkey, int64_t nr,
                                                       const int64_t* __restrict__ toff, int32_t* __restrict__ table,
                                                       int* chunk_counter, int* pseg, int* pdone, int* err) {
  __shared__ int64_t s_chunk;
  __shared__ int s_pa, s_pb, s_seg;
  for (;;) {
    if (threadIdx.x == 0) s_chunk = atomicAdd(chunk_counter, 1);
    __syncthreads();
    const int64_t c0 = s_chunk * kL2BuildChunk;
    __syncthreads();
    if (c0 >= nr) return;
    const int64_t c1 = min64(nr, c0 + kL2BuildChunk);
    if (threadIdx.x == 0) {
      const int pf = l2_part_of_hash(KeyTraits<K>::hash64(rkey[c0]));
      const int pl = l2_part_of_hash(KeyTraits<K>::hash64(rkey[c1 - 1]));
      s_pa = c0 == 0 ? 0 : pf;
      s_pb = c1 == nr ? kL2Parts - 1 : max(pl, l2_part_of_hash(KeyTraits<K>::hash64(rkey[c1])) - 1);
    }
    __syncthreads();
    for (int p = s_pa; p <= s_pb; ++p) l2_clear_partition<K>(p, toff, table, L2Slot<K>::kWords, pseg, pdone, &s_seg, err);
    if constexpr (sizeof(K) == 4) {
      // one row per thread in flight (batching several rows' compare-and-swaps
      // per thread made the build 1.7x slower)
      for (int64_t i = c0 + threadIdx.x; i < c1; i += blockDim.x) {
        const K k = rkey[i];
        const uint64_t h = KeyTraits<K>::hash64(k);
        const int P = (int)(h & (kL2Parts - 1));
        const int64_t base = toff[P];
        const uint64_t msk = (uint64_t)(toff[P + 1] - base) - 1;
        uint64_t sl = (h >> kL2Bits) & msk;
        auto* t = reinterpret_cast<unsigned long long*>(table) + base;
        const unsigned long long w = L2Slot<int32_t>::make((int32_t)k, i);
        for (uint64_t probe = 0; probe <= msk; ++probe) {
          const unsigned long long prev = atomicCAS(&t[sl], 0ull, w);
          if (prev == 0ull) break;
          if ((uint32_t)prev == (uint32_t)w) {
            set_status(err, GJ_ERR_DUPLICATE_KEY);
            break;
          }
          sl = (sl + 1) & msk;
        }
      }
    } else {
      for (int64_t i = c0 + threadIdx.x; i < c1; i += blockDim.x) {
        const K k = rkey[i];
        const uint64_t h = KeyTraits<K>::hash64(k);
        const int P = (int)(h & (kL2Parts - 1));
        const int64_t base = toff[P];
        const uint64_t msk = (uint64_t)(toff[P + 1] - base) - 1;
        uint64_t sl = (h >> kL2Bits) & msk;
        int32_t* t = table + base;
        for (uint64_t probe = 0; probe <= msk; ++probe) {
          const int prev = atomicCAS(&t[sl], 0, (int)(i + 1));
          if (prev == 0) break;
          if (rkey[prev - 1] == k) {
            set_status(err, GJ_ERR_DUPLICATE_KEY);
            break;
          }
          sl = (sl + 1) & msk;
        }
      }
    }
  }
}

// The R' row of key k in the table of its partition, or -1, given the word w
// already read at its first slot sl.
template <typename K>
__device__ __forceinline__ int32_t l2_resolve(const K* __restrict__ rkey, const int32_t* __restrict__ table,
                                              int64_t base, uint64_t msk, uint64_t sl, typename L2Slot<K>::W w, K k) {
  if constexpr (sizeof(K) == 4) {
    const auto* t = reinterpret_cast<const unsigned long long*>(table) + base;
    for (uint64_t probe = 0; probe <= msk; ++probe) {
      if (w == 0ull) return -1;
      if ((int32_t)(uint32_t)w == (int32_t)k) return (int32_t)(w >> 32) - 1;
      sl = (sl + 1) & msk;
      w = __ldg(t + sl);
    }
  } else {
    const int32_t* t = table + base;
    for (uint64_t probe = 0; probe <= msk; ++probe) {
      if (w == 0) return -1;
      if (__ldg(rkey + w - 1) == k) return w - 1;
      sl = (sl + 1) & msk;
      w = __ldg(t + sl);
    }
  }
  return -1;
}

constexpr int kL2ProbeThreads = 256;
template <typename K, int NT = kL2ProbeThreads>
__global__ void __launch_bounds__(NT, 1024 / NT) phj_l2_probe_kernel(const K* __restrict__ rkey,
                                                                const int64_t* __restrict__ toff,
                                                                const int32_t* __restrict__ table,
                                                                const K* __restrict__ skey, int64_t ns, JoinIO io,
                                                                uint64_t* unit_status, int* unit_counter,
                                                                int64_t nunits, int* err) {
  __shared__ int32_t s_midx[kUnitRows];
  __shared__ int64_t s_toff[kL2Parts + 1];
  __shared__ int64_t s_unit;
  __shared__ uint32_t s_wcnt[NT / 32];
  __shared__ uint64_t s_base;
  const int t = threadIdx.x;
  if (t == 0) s_unit = atomicAdd(unit_counter, 1);
  for (int p = t; p <= kL2Parts; p += NT) s_toff[p] = toff[p];
  __syncthreads();
  const int64_t unit = s_unit;
  if (unit >= nunits) return;
  const int64_t u0 = unit * kUnitRows;
  const int un = (int)min64(kUnitRows, ns - u0);
  // every row's build row: kLook rows per thread in flight
  constexpr int kLook = 4;
  for (int r0 = 0; r0 < un; r0 += NT * kLook) {
    K k[kLook];
#pragma unroll
    for (int q = 0; q < kLook; ++q) {
      const int r = r0 + q * NT + t;
      k[q] = r < un ? __ldcs(skey + u0 + r) : K(0);
    }
    // the first slot of every row of the batch is read before any is resolved, so
    // the batch's L2 round trips overlap; a collision continues on its own
    int64_t base[kLook];
    uint64_t msk[kLook], sl[kLook];
    typename L2Slot<K>::W w[kLook];
#pragma unroll
    for (int q = 0; q < kLook; ++q) {
      const uint64_t h = KeyTraits<K>::hash64(k[q]);
      const int P = (int)(h & (kL2Parts - 1));
      base[q] = s_toff[P];  // in entries
      msk[q] = (uint64_t)(s_toff[P + 1] - s_toff[P]) - 1;
      sl[q] = (h >> kL2Bits) & msk[q];
      const bool in = r0 + q * NT + t < un;
      w[q] = in ? __ldg(reinterpret_cast<const typename L2Slot<K>::W*>(table) + base[q] + sl[q])
                : typename L2Slot<K>::W(0);
    }
#pragma unroll
    for (int q = 0; q < kLook; ++q) {
      const int r = r0 + q * NT + t;
      if (r >= un) continue;
      s_midx[r] = l2_resolve<K>(rkey, table, base[q], msk[q], sl[q], w[q], k[q]);
    }
  }
  __syncthreads();
  phj_emit_unit<K, NT>(skey, u0, un, unit, nunits, s_midx, io, unit_status, err, s_wcnt, &s_base);
}

// ---------------------------------------------------------------- NPHJ
template <typename K>
__global__ void nphj_build_kernel(const K* __restrict__ rkey, int64_t nr, int32_t* __restrict__ ht, uint64_t mask,
                                  int* err) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nr; i += stride) {
    K k = rkey[i];
    uint64_t sl = KeyTraits<K>::hash64(k) & mask;
    for (uint64_t probe = 0; probe <= mask; ++probe) {
      int prev = atomicCAS(&ht[sl], 0, (int)(i + 1));
      if (prev == 0) break;
      if (rkey[prev - 1] == k) {
        set_status(err, GJ_ERR_DUPLICATE_KEY);
        break;
      }
      sl = (sl + 1) & mask;
    }
  }
}

template <typename K>
__global__ void __launch_bounds__(kThreads) nphj_probe_kernel(const K* __restrict__ rkey,
                                                              const int32_t* __restrict__ ht, uint64_t mask,
                                                              const K* __restrict__ skey, int64_t ns, JoinIO io,
                                                              uint64_t* tile_status, int* tile_counter,
                                                              int64_t ntiles, int* err) {
  __shared__ K s_key[kTileS];
  __shared__ int32_t s_pos[kTileS];
  __shared__ int32_t s_midx[kTileS];
  __shared__ uint32_t s_scan[kThreads / 32];
  __shared__ uint64_t s_base;
  __shared__ int64_t s_tile;
  const int t = threadIdx.x;
  if (t == 0) s_tile = atomicAdd(tile_counter, 1);
  __syncthreads();
  const int64_t tile = s_tile;
  const int64_t tile_base = tile * kTileS;
  const int tile_n = (int)min64(kTileS, ns - tile_base);
  // first probe of every owned row issued together; collisions continue serially
  K k[kItems];
  uint64_t sl[kItems];
  int v[kItems];
  K rk[kItems];
#pragma unroll
  for (int j = 0; j < kItems; ++j) {
    const int i = t + j * kThreads;
    k[j] = i < tile_n ? __ldcs(skey + tile_base + i) : K(0);
  }
#pragma unroll
  for (int j = 0; j < kItems; ++j) {
    const int i = t + j * kThreads;
    sl[j] = KeyTraits<K>::hash64(k[j]) & mask;
    v[j] = i < tile_n ? __ldg(ht + sl[j]) : 0;
  }
#pragma unroll
  for (int j = 0; j < kItems; ++j) rk[j] = v[j] ? __ldg(rkey + v[j] - 1) : K(0);
#pragma unroll
  for (int j = 0; j < kItems; ++j) {
    const int i = t + j * kThreads;
    if (i >= tile_n) continue;
    s_key[i] = k[j];
    int32_t m = -1;
    int vv = v[j];
    K kk = rk[j];
    uint64_t s2 = sl[j];
    for (uint64_t probe = 0; probe <= mask && vv != 0; ++probe) {
      if (kk == k[j]) {
        m = vv - 1;
        break;
      }
      s2 = (s2 + 1) & mask;
      vv = ht[s2];
      if (vv) kk = rkey[vv - 1];
    }
    s_midx[i] = m;
  }
  __syncthreads();
  emit_tile<K>(tile, ntiles, tile_base, tile_n, s_key, s_midx, s_pos, io, tile_status, err, s_scan, &s_base);
}

// ---------------------------------------------------------------- SMJ
// Sort-merge join (Sec. 3.1.1; the paper's comparison point, with Merge Path
// partitioning): R and S are radix-sorted on the whole key (signed order), with
// their payloads (TR) or tuple ids (UR). Each tile of kTileS sorted S rows finds
// its range of R rows by two warp-wide 33-way searches over R (the tile's first
// and last key: the merge-path split points), stages those R keys in shared
// memory when they fit, and matches every row by binary search in them. The
// NPHJ emitter then compacts and writes the tile through a decoupled look-back.
constexpr int kSmjRBytes = 12288;  // staged R keys per tile

// First index in sorted a[0, n) whose element is not below key (Upper: above key),
// found by all 32 lanes of a warp: 32 pivots per round trip.
template <typename K, bool Upper>
__device__ int64_t warp_bound(const K* __restrict__ a, int64_t n, K key) {
  const int lane = threadIdx.x & 31;
  int64_t lo = 0, hi = n;  // the answer lies in [lo, hi]
  while (hi - lo > 32) {
    const int64_t len = hi - lo;
    const int64_t p = lo + (len * (lane + 1)) / 33;
    const K v = a[p];
    const bool before = Upper ? !(key < v) : (v < key);  // the answer lies after p
    const int c = __popc(__ballot_sync(0xffffffffu, before));
    const int64_t nlo = c == 0 ? lo : lo + (len * c) / 33 + 1;
    const int64_t nhi = c == 32 ? hi : lo + (len * (c + 1)) / 33;
    lo = nlo;
    hi = nhi;
  }
  const int64_t p = lo + lane;
  bool before = false;
  if (p < hi) {
    const K v = a[p];
    before = Upper ? !(key < v) : (v < key);
  }
  return lo + __popc(__ballot_sync(0xffffffffu, before));
}

template <typename K>
__global__ void __launch_bounds__(kThreads) smj_merge_kernel(const K* __restrict__ rkey, int64_t nr,
                                                             const K* __restrict__ skey, int64_t ns, JoinIO io,
                                                             uint64_t* tile_status, int* tile_counter, int64_t ntiles,
                                                             int* err) {
  constexpr int kStageR = kSmjRBytes / (int)sizeof(K);
  __shared__ K s_key[kTileS];
  __shared__ K s_r[kStageR];
  __shared__ int32_t s_pos[kTileS];
  __shared__ int32_t s_midx[kTileS];
  __shared__ uint32_t s_scan[kThreads / 32];
  __shared__ uint64_t s_base;
  __shared__ int64_t s_tile, s_ra, s_rb;
  const int t = threadIdx.x;
  if (t == 0) s_tile = atomicAdd(tile_counter, 1);
  __syncthreads();
  const int64_t tile = s_tile;
  const int64_t tile_base = tile * kTileS;
  const int tile_n = (int)min64(kTileS, ns - tile_base);
  for (int i = t; i < tile_n; i += kThreads) s_key[i] = __ldcs(skey + tile_base + i);
  if (t < 32) {
    // the merge-path split: R rows with keys in [first, last] of the tile
    const int64_t ra = warp_bound<K, false>(rkey, nr, skey[tile_base]);
    const int64_t rb = warp_bound<K, true>(rkey, nr, skey[tile_base + tile_n - 1]);
    if (t == 0) {
      s_ra = ra;
      s_rb = rb;
    }
  }
  __syncthreads();
  const int64_t ra = s_ra, rb = s_rb;
  const bool staged = rb - ra <= kStageR;
  if (staged)
    for (int64_t j = t; j < rb - ra; j += kThreads) s_r[j] = __ldg(rkey + ra + j);
  __syncthreads();
  for (int i = t; i < tile_n; i += kThreads) {
    const K k = s_key[i];
    int64_t lo = ra, hi = rb;  // first R row in [ra, rb) not below k
    while (lo < hi) {
      const int64_t m = (lo + hi) >> 1;
      const K v = staged ? s_r[m - ra] : rkey[m];
      if (v < k) lo = m + 1; else hi = m;
    }
    int32_t mi = -1;
    if (lo < rb && (staged ? s_r[lo - ra] : rkey[lo]) == k) {
      mi = (int32_t)lo;
      if (lo + 1 < rb && (staged ? s_r[lo + 1 - ra] : rkey[lo + 1]) == k) set_status(err, GJ_ERR_DUPLICATE_KEY);
    }
    s_midx[i] = mi;
  }
  __syncthreads();
  emit_tile<K>(tile, ntiles, tile_base, tile_n, s_key, s_midx, s_pos, io, tile_status, err, s_scan, &s_base);
}

// ---------------------------------------------------------------- many-to-many
// R.key may repeat (Sec. 5.1, many-to-many joins). The global table keeps, per
// key, the last R row inserted (row + 1); next[r] links each R row to the one
// inserted before it with the same key (-1 ends the chain), so the rows of a key
// are one chain. Chain order follows the insertions and is not fixed, which only
// reorders T.
//
// Non-partitioned (NPHJ-MN) the table is indexed by the key's hash. Partitioned
// (PHJ-MN, GFTR: R and S radix-partitioned on the low cbits hash bits with their
// payloads) the slot puts the partition id in the top cbits of the slot index, so
// the keys of one partition occupy one contiguous stretch of the table: probe
// rows taken in S' order stay inside a few KB of it, and a key's chain of R' rows
// lies inside its partition.
__device__ __forceinline__ uint64_t mn_slot(uint64_t h, uint64_t mask, int cbits, int logslots) {
  if (cbits == 0) return h & mask;
  const uint64_t p = h & ((uint64_t(1) << cbits) - 1);
  const uint64_t rest = (h >> cbits) & ((uint64_t(1) << (logslots - cbits)) - 1);
  return (p << (logslots - cbits)) | rest;
}

template <typename K>
__global__ void nphj_mn_build_kernel(const K* __restrict__ rkey, int64_t nr, int32_t* __restrict__ ht, uint64_t mask,
                                     int cbits, int logslots, int32_t* __restrict__ next, int* err) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nr; i += stride) {
    const K k = rkey[i];
    uint64_t sl = mn_slot(KeyTraits<K>::hash64(k), mask, cbits, logslots);
    bool done = false;
    for (uint64_t probe = 0; probe <= mask; ++probe) {
      const int prev = atomicCAS(&ht[sl], 0, (int)(i + 1));
      if (prev == 0) {
        next[i] = -1;
        done = true;
        break;
      }
      if (rkey[prev - 1] == k) {
        // the key's slot: this row becomes the head, linked to the previous head
        next[i] = atomicExch(&ht[sl], (int)(i + 1)) - 1;
        done = true;
        break;
      }
      sl = (sl + 1) & mask;
    }
    if (!done) set_status(err, GJ_ERR_CAPACITY);
  }
}

// One block per tile of kTileS probe rows (a contiguous run of kItems rows per
// thread): count every row's matches by walking its key's chain, take the tile's
// output offset from a decoupled look-back over tiles, then walk the chains again
// and write each (r, s) pair. Output rows of a thread are contiguous.
template <typename K>
__global__ void __launch_bounds__(kThreads) nphj_mn_probe_kernel(const K* __restrict__ rkey,
                                                                 const int32_t* __restrict__ ht, uint64_t mask,
                                                                 int cbits, int logslots,
                                                                 const int32_t* __restrict__ next,
                                                                 const K* __restrict__ skey, int64_t ns, JoinIO io,
                                                                 uint64_t* tile_status, int* tile_counter,
                                                                 int64_t ntiles, int* err) {
  __shared__ uint64_t s_warp[kThreads / 32];
  __shared__ uint64_t s_base;
  __shared__ int64_t s_tile;
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  if (t == 0) s_tile = atomicAdd(tile_counter, 1);
  __syncthreads();
  const int64_t tile = s_tile;
  const int64_t r0 = tile * kTileS + (int64_t)t * kItems;  // this thread's rows [r0, r0 + kItems)
  int32_t head[kItems];
  uint32_t cnt[kItems];
  uint64_t mine = 0;
#pragma unroll
  for (int j = 0; j < kItems; ++j) {
    const int64_t i = r0 + j;
    head[j] = -1;
    cnt[j] = 0;
    if (i >= ns) continue;
    const K k = skey[i];
    uint64_t sl = mn_slot(KeyTraits<K>::hash64(k), mask, cbits, logslots);
    for (uint64_t probe = 0; probe <= mask; ++probe) {
      const int v = __ldg(ht + sl);
      if (v == 0) break;
      if (__ldg(rkey + v - 1) == k) {
        head[j] = v - 1;
        break;
      }
      sl = (sl + 1) & mask;
    }
    for (int32_t r = head[j]; r >= 0; r = __ldg(next + r)) ++cnt[j];
    mine += cnt[j];
  }
  // block exclusive scan of the per-thread match counts, then the tile's offset
  uint64_t x = mine;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint64_t y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) s_warp[warp] = x;
  __syncthreads();
  if (warp == 0) {
    uint64_t w = lane < kThreads / 32 ? s_warp[lane] : 0;
    uint64_t wx = w;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint64_t y = __shfl_up_sync(0xffffffffu, wx, o);
      if (lane >= o) wx += y;
    }
    const uint64_t total = __shfl_sync(0xffffffffu, wx, 31);
    if (lane < kThreads / 32) s_warp[lane] = wx - w;
    const uint64_t excl = lookback_scan_warp(tile_status, tile, total, err);
    if (lane == 0) {
      s_base = excl;
      if (tile == ntiles - 1 && io.d_count) *io.d_count = (int64_t)(excl + total);
    }
  }
  __syncthreads();
  uint64_t pos = s_base + s_warp[warp] + (x - mine);
  const int ncols = io.nr_cols + io.ns_cols;
  bool overflow = false;
#pragma unroll
  for (int j = 0; j < kItems; ++j) {
    const int64_t i = r0 + j;
    if (i >= ns) continue;
    const K k = head[j] >= 0 ? skey[i] : K(0);
    for (int32_t r = head[j]; r >= 0; r = __ldg(next + r)) {
      if ((int64_t)pos >= io.cap) {
        overflow = true;
        break;
      }
      ((K*)io.tkey)[pos] = k;
      for (int c = 0; c < ncols; ++c) {
        const bool rside = c < io.nr_cols;
        const int sz = rside ? io.rsize[c] : io.ssize[c - io.nr_cols];
        const int64_t src_row = rside ? (int64_t)r : i;
        const void* src = rside ? io.rsrc[c] : io.ssrc[c - io.nr_cols];
        copy_elem(io.tcols[c], (int64_t)pos, src, src_row, sz);
      }
      ++pos;
    }
  }
  if (overflow) set_status(err, GJ_ERR_CAPACITY);
}

// ---------------------------------------------------------------- join -> group-by
// The group-by that follows a join (Sec. 1) fused into the probe: each match is
// aggregated where it is found and T is never written. Groups live either in a
// dense slot array indexed by the key's residue (the group key is `x % m`, so
// it lies in (-m, m)) with per-block shared-memory pre-aggregation, or in a
// global open-addressing table of int64 group keys.
constexpr int64_t kEmptyKey = INT64_MIN;

struct FusedRef {
  int32_t is_key;  // the join key itself
  int32_t side;    // 0 = R (indexed by the build-side match), 1 = S (by the probe row)
  int32_t size;
  int64_t mod;
  const void* src;
  const int32_t* tid;  // UR: ids carried through the partitioning
};

struct GroupSink {
  int32_t dense;
  int32_t smem;
  int64_t dense_off;
  int64_t nslots;  // dense domain or table capacity; table mode has one more slot for kEmptyKey
  uint64_t mask;
  int64_t* keys;
  unsigned long long* cnt;  // matches per slot: a slot holds a group iff cnt > 0
  int32_t nagg;
  int32_t op[kMaxAggs];
  int64_t* agg[kMaxAggs];
  FusedRef gk;
  FusedRef val[kMaxAggs];
};

__device__ __forceinline__ int64_t fused_value(const FusedRef& f, int64_t m, int64_t i, int64_t key) {
  int64_t v;
  if (f.is_key) {
    v = key;
  } else {
    int64_t idx = f.side == 0 ? m : i;
    if (f.tid) idx = f.tid[idx];
    v = load_as_i64(f.src, f.size, idx);
  }
  return f.mod > 0 ? v % f.mod : v;
}

__device__ __forceinline__ int64_t sink_slot(const GroupSink& G, int64_t gk, int* err) {
  if (G.dense) return gk + G.dense_off;
  if (gk == kEmptyKey) return G.nslots;
  uint64_t sl = fmix64((uint64_t)gk) & G.mask;
  for (uint64_t probe = 0; probe <= G.mask; ++probe) {
    int64_t cur = (int64_t)ld_volatile((const uint64_t*)&G.keys[sl]);
    if (cur == gk) return (int64_t)sl;
    if (cur == kEmptyKey) {
      unsigned long long old = atomicCAS((unsigned long long*)&G.keys[sl], (unsigned long long)kEmptyKey,
                                         (unsigned long long)gk);
      if ((int64_t)old == kEmptyKey || (int64_t)old == gk) return (int64_t)sl;
    }
    sl = (sl + 1) & G.mask;
  }
  set_status(err, GJ_ERR_CAPACITY);
  return -1;
}

// Aggregates one match (build index m, probe index i, join key) into the sink.
__device__ __forceinline__ void sink_add(const GroupSink& G, int64_t m, int64_t i, int64_t key,
                                         unsigned long long* s_cnt, int64_t* s_agg, int* err) {
  const int64_t gk = fused_value(G.gk, m, i, key);
  const int64_t sl = sink_slot(G, gk, err);
  if (sl < 0) return;
  if (G.smem) {
    atomicAdd(&s_cnt[sl], 1ull);
    for (int j = 0; j < G.nagg; ++j)
      agg_atomic(G.op[j], &s_agg[(int64_t)j * G.nslots + sl],
                 G.op[j] == GJ_AGG_COUNT ? 1 : fused_value(G.val[j], m, i, key));
  } else {
    atomicAdd(&G.cnt[sl], 1ull);
    for (int j = 0; j < G.nagg; ++j)
      agg_atomic(G.op[j], &G.agg[j][sl], G.op[j] == GJ_AGG_COUNT ? 1 : fused_value(G.val[j], m, i, key));
  }
}

__device__ void sink_smem_init(const GroupSink& G, unsigned long long* s_cnt, int64_t* s_agg) {
  if (!G.smem) return;
  for (int64_t s = threadIdx.x; s < G.nslots; s += blockDim.x) {
    s_cnt[s] = 0;
    for (int j = 0; j < G.nagg; ++j) s_agg[(int64_t)j * G.nslots + s] = agg_identity(G.op[j]);
  }
  __syncthreads();
}

__device__ void sink_smem_flush(const GroupSink& G, const unsigned long long* s_cnt, const int64_t* s_agg) {
  if (!G.smem) return;
  __syncthreads();
  for (int64_t s = threadIdx.x; s < G.nslots; s += blockDim.x) {
    if (s_cnt[s] == 0) continue;
    atomicAdd(&G.cnt[s], s_cnt[s]);
    for (int j = 0; j < G.nagg; ++j) agg_atomic(G.op[j], &G.agg[j][s], s_agg[(int64_t)j * G.nslots + s]);
  }
}

__global__ void sink_init_kernel(GroupSink G) {
  const int64_t total = G.nslots + (G.dense ? 0 : 1);
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; s < total; s += stride) {
    if (!G.dense) G.keys[s] = kEmptyKey;
    G.cnt[s] = 0;
    for (int j = 0; j < G.nagg; ++j) G.agg[j][s] = agg_identity(G.op[j]);
  }
}

template <typename K>
__global__ void __launch_bounds__(kThreads, 2) phj_probe_agg_kernel(const K* __restrict__ rkey,
                                                                 const int64_t* __restrict__ roff, int pbits,
                                                                 const K* __restrict__ skey, int64_t ns, GroupSink G,
                                                                 int* tile_counter, int64_t ntiles, int* err) {
  extern __shared__ __align__(128) unsigned char s_raw[];
  K* s_key = (K*)s_raw;
  int32_t* s_part = (int32_t*)(s_key + kTileS);
  int32_t* s_midx = s_part + kTileS;
  int32_t* s_slots = s_midx + kTileS;
  K* s_rkey = (K*)(s_slots + kSlots);
  unsigned long long* s_cnt = (unsigned long long*)(s_rkey + kBuildCap);
  int64_t* s_agg = (int64_t*)(s_cnt + (G.smem ? G.nslots : 0));
  __shared__ int64_t s_tile;
  sink_smem_init(G, s_cnt, s_agg);
  for (;;) {
    if (threadIdx.x == 0) s_tile = atomicAdd(tile_counter, 1);
    __syncthreads();
    const int64_t tile = s_tile;
    if (tile >= ntiles) break;
    const int64_t tile_base = tile * kTileS;
    const int tile_n = (int)min64(kTileS, ns - tile_base);
    probe_tile<K>(rkey, roff, pbits, skey, tile_base, tile_n, s_key, s_part, s_midx, s_slots, s_rkey, err);
    for (int i = threadIdx.x; i < tile_n; i += kThreads) {
      const int32_t m = s_midx[i];
      if (m >= 0) sink_add(G, m, tile_base + i, (int64_t)s_key[i], s_cnt, s_agg, err);
    }
    __syncthreads();
  }
  sink_smem_flush(G, s_cnt, s_agg);
}

template <typename K>
__global__ void __launch_bounds__(kThreads) nphj_probe_agg_kernel(const K* __restrict__ rkey,
                                                                  const int32_t* __restrict__ ht, uint64_t mask,
                                                                  const K* __restrict__ skey, int64_t ns, GroupSink G,
                                                                  int* err) {
  extern __shared__ __align__(128) unsigned char s_raw[];
  unsigned long long* s_cnt = (unsigned long long*)s_raw;
  int64_t* s_agg = (int64_t*)(s_cnt + (G.smem ? G.nslots : 0));
  sink_smem_init(G, s_cnt, s_agg);
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < ns; i += stride) {
    const K k = skey[i];
    uint64_t sl = KeyTraits<K>::hash64(k) & mask;
    for (uint64_t probe = 0; probe <= mask; ++probe) {
      int v = ht[sl];
      if (v == 0) break;
      if (rkey[v - 1] == k) {
        sink_add(G, v - 1, i, (int64_t)k, s_cnt, s_agg, err);
        break;
      }
      sl = (sl + 1) & mask;
    }
  }
  sink_smem_flush(G, s_cnt, s_agg);
}

// Writes the occupied slots densely: out_keys / out_aggs[j], g = *d_ngroups.
constexpr int kEmitItems = 8;
constexpr int kEmitTile = kThreads * kEmitItems;

__global__ void __launch_bounds__(kThreads) group_emit_kernel(GroupSink G, int64_t* __restrict__ out_keys,
                                                              Aggs out, int64_t cap, int64_t* d_ngroups,
                                                              uint64_t* tstat, int* counter, int64_t ntiles,
                                                              int* err) {
  __shared__ uint32_t s_scan[kThreads / 32];
  __shared__ uint64_t s_base;
  __shared__ int64_t s_tile;
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  if (t == 0) s_tile = atomicAdd(counter, 1);
  __syncthreads();
  const int64_t tile = s_tile;
  const int64_t total = G.nslots + (G.dense ? 0 : 1);
  const int64_t tb = tile * kEmitTile + (int64_t)t * kEmitItems;
  uint32_t cnt = 0;
  for (int r = 0; r < kEmitItems; ++r) cnt += (tb + r < total && G.cnt[tb + r] > 0) ? 1u : 0u;
  uint32_t x = cnt;
  for (int o = 1; o < 32; o <<= 1) {
    uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) s_scan[warp] = x;
  __syncthreads();
  if (warp == 0) {
    uint32_t run = 0;
    for (int w = 0; w < kThreads / 32; ++w) run += s_scan[w];
    __syncwarp();
    if (lane == 0) {
      uint32_t r = 0;
      for (int w = 0; w < kThreads / 32; ++w) {
        const uint32_t c = s_scan[w];
        s_scan[w] = r;
        r += c;
      }
    }
    const uint64_t excl = lookback_scan_warp(tstat, tile, run, err);
    if (lane == 0) {
      s_base = excl;
      if (tile == ntiles - 1) *d_ngroups = (int64_t)(excl + run);
    }
  }
  __syncthreads();
  int64_t o = (int64_t)s_base + s_scan[warp] + x - cnt;
  bool overflow = false;
  for (int r = 0; r < kEmitItems; ++r) {
    const int64_t sl = tb + r;
    if (sl >= total || G.cnt[sl] == 0) continue;
    if (o >= cap) {
      overflow = true;
      ++o;
      continue;
    }
    out_keys[o] = G.dense ? sl - G.dense_off : (sl == G.nslots ? kEmptyKey : G.keys[sl]);
    for (int j = 0; j < out.n; ++j) out.out[j][o] = G.agg[j][sl];
    ++o;
  }
  if (overflow) set_status(err, GJ_ERR_CAPACITY);
}

// The tables of the L2-sized build partitions of R' (rk2, nr rows): partition
// bounds, table offsets, clearing and the build (scratch taken up front).
struct L2Tables {
  int64_t* roff;
  int64_t* toff;
  int32_t* table;
  int* bcounter;
};

template <typename K>
gj_status l2_tables_alloc(Scratch& scr, int64_t nr, L2Tables* t) {
  constexpr int kW = L2Slot<K>::kWords;  // int32 words per entry
  t->roff = scr.get_as<int64_t>(kL2Parts + 1);
  t->toff = scr.get_as<int64_t>(kL2Parts + 1);
  t->table = scr.get_as<int32_t>(((size_t)4 * nr + 2 * kL2Parts) * kW);  // sizes < 4 rows + 2 each
  t->bcounter = scr.get_as<int>(1 + 2 * kL2Parts);
  return scr.failed() ? GJ_ERR_OOM : GJ_OK;
}

template <typename K>
gj_status l2_tables_run(const Ctx& ctx, const K* rk2, int64_t nr, const L2Tables* t) {
  gj_status st;
  cudaStream_t s = ctx.stream;
  // the chunk counter, then per partition its clearing-segment and cleared-segment counters
  if ((st = cuda_check(cudaMemsetAsync(t->bcounter, 0, sizeof(int) * (1 + 2 * kL2Parts), s))) != GJ_OK) return st;
  if ((st = partition_bounds_run(ctx, sizeof(K) == 8 ? GJ_I64 : GJ_I32, rk2, nr, 0, kL2Bits, kHashed, t->roff)) !=
      GJ_OK)
    return st;
  {
    LaunchScope ls(ctx, KK_PART_BOUNDS);
    l2_table_offsets_kernel<<<1, kL2Parts, 0, s>>>(t->roff, t->toff);
  }
  LaunchScope ls(ctx, KK_NPHJ_BUILD);
  // blocks take build chunks in order: the tables being cleared and filled are
  // those of a few neighbouring partitions
  const int bblocks =
      (int)std::max<int64_t>(1, std::min<int64_t>((nr + kL2BuildChunk - 1) / kL2BuildChunk, (int64_t)ctx.num_sms * 8));
  l2_build_kernel<K><<<bblocks, 256, 0, s>>>(rk2, nr, t->toff, t->table, t->bcounter, t->bcounter + 1,
                                             t->bcounter + 1 + kL2Parts, ctx.d_status);
  return cuda_check(cudaGetLastError());
}

template <typename K>
gj_status join_typed(const Ctx& ctx, const gj_table* R, const gj_table* S, int variant, int bits, int bpp, bool l2,
                     gj_table* T, int64_t cap, int64_t* d_count) {
  cudaStream_t s = ctx.stream;
  Scratch scr(s);
  gj_status st;
  if ((st = cuda_check(cudaMemsetAsync(d_count, 0, sizeof(int64_t), s))) != GJ_OK) return st;
  const int64_t nr = R->n, ns = S->n;
  JoinIO io{};
  io.nr_cols = R->ncols;
  io.ns_cols = S->ncols;
  io.tkey = T->key;
  for (int c = 0; c < R->ncols + S->ncols; ++c) io.tcols[c] = T->cols[c];
  io.cap = cap;
  io.d_count = d_count;
  for (int c = 0; c < R->ncols; ++c) io.rsize[c] = dtype_size(R->col_type[c]);
  for (int c = 0; c < S->ncols; ++c) io.ssize[c] = dtype_size(S->col_type[c]);
  // no rows on either side: no matches (the emit reads row 0 of each source, which must exist)
  if (ns == 0 || nr == 0) return GJ_OK;

  const int64_t ntiles = (ns + kTileS - 1) / kTileS;
  uint64_t* tstat = scr.get_as<uint64_t>(ntiles);
  int* counter = scr.get_as<int>(1);
  if (scr.failed()) return GJ_ERR_OOM;
  if ((st = cuda_check(cudaMemsetAsync(tstat, 0, sizeof(uint64_t) * ntiles, s))) != GJ_OK) return st;
  if ((st = cuda_check(cudaMemsetAsync(counter, 0, sizeof(int), s))) != GJ_OK) return st;

  if (variant == GJ_JOIN_SMJ_TR || variant == GJ_JOIN_SMJ_UR) {
    // sort both sides on every key bit; TR moves the payloads along, UR a tuple id
    const bool tr = variant == GJ_JOIN_SMJ_TR;
    const int kbits = sizeof(K) * 8;
    K* rk2 = scr.get_as<K>(nr);
    K* sk2 = scr.get_as<K>(ns);
    ColSet rc{}, sc{};
    if (tr) {
      rc.n = R->ncols;
      for (int c = 0; c < R->ncols; ++c) {
        rc.src[c] = R->cols[c];
        rc.size[c] = dtype_size(R->col_type[c]);
        rc.dst[c] = scr.get((size_t)nr * rc.size[c]);
      }
      sc.n = S->ncols;
      for (int c = 0; c < S->ncols; ++c) {
        sc.src[c] = S->cols[c];
        sc.size[c] = dtype_size(S->col_type[c]);
        sc.dst[c] = scr.get((size_t)ns * sc.size[c]);
      }
    } else {
      rc.n = sc.n = 1;
      rc.src[0] = sc.src[0] = nullptr;  // generated tuple ids
      rc.size[0] = sc.size[0] = 4;
      rc.dst[0] = scr.get((size_t)nr * 4);
      sc.dst[0] = scr.get((size_t)ns * 4);
    }
    if (scr.failed()) return GJ_ERR_OOM;
    const int kt = sizeof(K) == 8 ? GJ_I64 : GJ_I32;
    if ((st = radix_partition_run(ctx, scr, kt, R->key, rk2, rc, nr, 0, kbits, kSignedOrder, bpp)) != GJ_OK) return st;
    if ((st = radix_partition_run(ctx, scr, kt, S->key, sk2, sc, ns, 0, kbits, kSignedOrder, bpp)) != GJ_OK) return st;
    if (tr) {
      for (int c = 0; c < R->ncols; ++c) io.rsrc[c] = rc.dst[c];
      for (int c = 0; c < S->ncols; ++c) io.ssrc[c] = sc.dst[c];
    } else {
      for (int c = 0; c < R->ncols; ++c) io.rsrc[c] = R->cols[c];
      for (int c = 0; c < S->ncols; ++c) io.ssrc[c] = S->cols[c];
      io.r_tid = (const int32_t*)rc.dst[0];
      io.s_tid = (const int32_t*)sc.dst[0];
    }
    LaunchScope ls(ctx, KK_SMJ_MERGE);
    smj_merge_kernel<K><<<(unsigned)ntiles, kThreads, 0, s>>>(rk2, nr, sk2, ns, io, tstat, counter, ntiles,
                                                               ctx.d_status);
    return cuda_check(cudaGetLastError());
  }

  if (variant == GJ_JOIN_NPHJ_MN || variant == GJ_JOIN_PHJ_MN) {
    const K* rk = (const K*)R->key;
    const K* sk = (const K*)S->key;
    for (int c = 0; c < R->ncols; ++c) io.rsrc[c] = R->cols[c];
    for (int c = 0; c < S->ncols; ++c) io.ssrc[c] = S->cols[c];
    int cbits = 0;
    if (variant == GJ_JOIN_PHJ_MN && bits > 0) {
      // GFTR: both sides partitioned on the low hash bits with their payloads
      K* rk2 = scr.get_as<K>(nr);
      K* sk2 = scr.get_as<K>(ns);
      ColSet rc{}, sc{};
      rc.n = R->ncols;
      for (int c = 0; c < R->ncols; ++c) {
        rc.src[c] = R->cols[c];
        rc.size[c] = dtype_size(R->col_type[c]);
        rc.dst[c] = scr.get((size_t)nr * rc.size[c]);
      }
      sc.n = S->ncols;
      for (int c = 0; c < S->ncols; ++c) {
        sc.src[c] = S->cols[c];
        sc.size[c] = dtype_size(S->col_type[c]);
        sc.dst[c] = scr.get((size_t)ns * sc.size[c]);
      }
      if (scr.failed()) return GJ_ERR_OOM;
      const int kt = sizeof(K) == 8 ? GJ_I64 : GJ_I32;
      if ((st = radix_partition_run(ctx, scr, kt, rk, rk2, rc, nr, 0, bits, kHashed, bpp)) != GJ_OK) return st;
      if ((st = radix_partition_run(ctx, scr, kt, sk, sk2, sc, ns, 0, bits, kHashed, bpp)) != GJ_OK) return st;
      rk = rk2;
      sk = sk2;
      for (int c = 0; c < R->ncols; ++c) io.rsrc[c] = rc.dst[c];
      for (int c = 0; c < S->ncols; ++c) io.ssrc[c] = sc.dst[c];
      cbits = bits;
    }
    uint64_t slots = 1;
    int logslots = 0;
    while (slots < (uint64_t)std::max<int64_t>(2 * nr, 2)) {
      slots <<= 1;
      ++logslots;
    }
    if (cbits > logslots) cbits = 0;  // more partitions than slots: plain hashing
    int32_t* ht = scr.get_as<int32_t>(slots);
    int32_t* next = scr.get_as<int32_t>(std::max<int64_t>(nr, 1));
    if (scr.failed()) return GJ_ERR_OOM;
    if ((st = cuda_check(cudaMemsetAsync(ht, 0, sizeof(int32_t) * slots, s))) != GJ_OK) return st;
    {
      int blocks = (int)std::min<int64_t>((nr + 255) / 256, (int64_t)ctx.num_sms * 16);
      LaunchScope ls(ctx, KK_NPHJ_BUILD);
      nphj_mn_build_kernel<K><<<blocks, 256, 0, s>>>(rk, nr, ht, slots - 1, cbits, logslots, next, ctx.d_status);
    }
    LaunchScope ls(ctx, KK_NPHJ_PROBE);
    nphj_mn_probe_kernel<K><<<(unsigned)ntiles, kThreads, 0, s>>>(rk, ht, slots - 1, cbits, logslots, next, sk, ns,
                                                                   io, tstat, counter, ntiles, ctx.d_status);
    return cuda_check(cudaGetLastError());
  }

  if (variant == GJ_JOIN_NPHJ) {
    uint64_t slots = 1;
    while (slots < (uint64_t)std::max<int64_t>(2 * nr, 2)) slots <<= 1;
    int32_t* ht = scr.get_as<int32_t>(slots);
    if (scr.failed()) return GJ_ERR_OOM;
    if ((st = cuda_check(cudaMemsetAsync(ht, 0, sizeof(int32_t) * slots, s))) != GJ_OK) return st;
    for (int c = 0; c < R->ncols; ++c) io.rsrc[c] = R->cols[c];
    for (int c = 0; c < S->ncols; ++c) io.ssrc[c] = S->cols[c];
    if (nr > 0) {
      int blocks = (int)std::min<int64_t>((nr + 255) / 256, (int64_t)ctx.num_sms * 16);
      LaunchScope ls(ctx, KK_NPHJ_BUILD);
      nphj_build_kernel<K><<<blocks, 256, 0, s>>>((const K*)R->key, nr, ht, slots - 1, ctx.d_status);
    }
    LaunchScope ls(ctx, KK_NPHJ_PROBE);
    nphj_probe_kernel<K><<<(unsigned)ntiles, kThreads, 0, s>>>((const K*)R->key, ht, slots - 1, (const K*)S->key,
                                                                ns, io, tstat, counter, ntiles, ctx.d_status);
    return cuda_check(cudaGetLastError());
  }

  // ---- partitioned hash joins
  const bool gftr = variant == GJ_JOIN_PHJ_TR;
  L2Tables l2t{};
  const K* rk = (const K*)R->key;
  const K* sk = (const K*)S->key;
  if (bits > 0) {
    K* rk2 = scr.get_as<K>(std::max<int64_t>(nr, 1));
    K* sk2 = scr.get_as<K>(ns);
    ColSet rc{}, sc{};
    if (gftr) {
      // four 4-byte payloads on a side travel as one interleaved 16-byte row, read
      // by the probe's path for sides of one to four 4-byte payloads
      auto narrow = [](const gj_table* t) {
        if (t->ncols < 1 || t->ncols > 4) return false;
        for (int c = 0; c < t->ncols; ++c)
          if (dtype_size(t->col_type[c]) != 4) return false;
        return true;
      };
      const bool both_narrow = narrow(R) && narrow(S);
      rc.n = R->ncols;
      rc.zip4 = both_narrow && R->ncols == 4 ? 1 : 0;
      for (int c = 0; c < R->ncols; ++c) {
        rc.src[c] = R->cols[c];
        rc.size[c] = dtype_size(R->col_type[c]);
        if (!rc.zip4) rc.dst[c] = scr.get((size_t)std::max<int64_t>(nr, 1) * rc.size[c]);
      }
      if (rc.zip4) rc.dst[0] = scr.get((size_t)std::max<int64_t>(nr, 1) * 16);
      sc.n = S->ncols;
      sc.zip4 = both_narrow && S->ncols == 4 ? 1 : 0;
      for (int c = 0; c < S->ncols; ++c) {
        sc.src[c] = S->cols[c];
        sc.size[c] = dtype_size(S->col_type[c]);
        if (!sc.zip4) sc.dst[c] = scr.get((size_t)ns * sc.size[c]);
      }
      if (sc.zip4) sc.dst[0] = scr.get((size_t)ns * 16);
    } else {
      rc.n = sc.n = 1;
      rc.src[0] = sc.src[0] = nullptr;  // generated tuple ids
      rc.size[0] = sc.size[0] = 4;
      rc.dst[0] = scr.get((size_t)std::max<int64_t>(nr, 1) * 4);
      sc.dst[0] = scr.get((size_t)ns * 4);
    }
    if (scr.failed()) return GJ_ERR_OOM;
    if (l2 && (st = l2_tables_alloc<K>(scr, nr, &l2t)) != GJ_OK) return st;
    if ((st = radix_partition_run(ctx, scr, sizeof(K) == 8 ? GJ_I64 : GJ_I32, rk, rk2, rc, nr, 0, bits, kHashed,
                                  bpp)) != GJ_OK)
      return st;
    if ((st = radix_partition_run(ctx, scr, sizeof(K) == 8 ? GJ_I64 : GJ_I32, sk, sk2, sc, ns, 0, bits, kHashed,
                                  bpp)) != GJ_OK)
      return st;
    // the build right before the probe: run on a second stream beside S's partition
    // pass it gained under 1 % (the streaming pass evicts the tables being filled)
    if (l2 && (st = l2_tables_run<K>(ctx, rk2, nr, &l2t)) != GJ_OK) return st;
    rk = rk2;
    sk = sk2;
    if (gftr) {
      // zipped payloads are read through r_zip / s_zip; rsrc / ssrc keep a valid
      // address for the unused column slots
      for (int c = 0; c < R->ncols; ++c) io.rsrc[c] = rc.zip4 ? rc.dst[0] : rc.dst[c];
      for (int c = 0; c < S->ncols; ++c) io.ssrc[c] = sc.zip4 ? sc.dst[0] : sc.dst[c];
      if (rc.zip4) io.r_zip = (const int4*)rc.dst[0];
      if (sc.zip4) io.s_zip = (const int4*)sc.dst[0];
    } else {
      for (int c = 0; c < R->ncols; ++c) io.rsrc[c] = R->cols[c];
      for (int c = 0; c < S->ncols; ++c) io.ssrc[c] = S->cols[c];
      io.r_tid = (const int32_t*)rc.dst[0];
      io.s_tid = (const int32_t*)sc.dst[0];
    }
  } else {
    for (int c = 0; c < R->ncols; ++c) io.rsrc[c] = R->cols[c];
    for (int c = 0; c < S->ncols; ++c) io.ssrc[c] = S->cols[c];
  }
  int64_t* roff = l2t.roff;
  if (!l2) {
    roff = scr.get_as<int64_t>(((size_t)1 << bits) + 1);
    if (scr.failed()) return GJ_ERR_OOM;
    if ((st = partition_bounds_run(ctx, sizeof(K) == 8 ? GJ_I64 : GJ_I32, rk, nr, 0, bits, kHashed, roff)) != GJ_OK)
      return st;
  }
  // probe keys arrive by bulk copy when S' keys are 16-byte aligned
  io.stage_bulk = (reinterpret_cast<uintptr_t>(sk) & 15) == 0 ? 1 : 0;
  io.narrow4 = io.nr_cols >= 1 && io.nr_cols <= 4 && io.ns_cols >= 1 && io.ns_cols <= 4;
  for (int c = 0; c < io.nr_cols; ++c) io.narrow4 &= io.rsize[c] == 4;
  for (int c = 0; c < io.ns_cols; ++c) io.narrow4 &= io.ssize[c] == 4;
  const int64_t nunits = (ns + kUnitRows - 1) / kUnitRows;
  uint64_t* ustat = scr.get_as<uint64_t>(nunits);
  int* ucounter = scr.get_as<int>(1);
  if (scr.failed()) return GJ_ERR_OOM;
  if ((st = cuda_check(cudaMemsetAsync(ustat, 0, sizeof(uint64_t) * nunits, s))) != GJ_OK) return st;
  if ((st = cuda_check(cudaMemsetAsync(ucounter, 0, sizeof(int), s))) != GJ_OK) return st;
  if (l2) {
    LaunchScope ls(ctx, KK_PHJ_PROBE);
    phj_l2_probe_kernel<K><<<(unsigned)nunits, kL2ProbeThreads, 0, s>>>(rk, l2t.toff, l2t.table, sk, ns, io, ustat,
                                                                         ucounter, nunits, ctx.d_status);
    return cuda_check(cudaGetLastError());
  }
  const size_t dyn = phj_unit_smem_bytes<K>();
  if ((st = ensure_smem_attr(ctx, (const void*)phj_unit_kernel<K>, (int)dyn)) != GJ_OK) return st;
  LaunchScope ls(ctx, KK_PHJ_PROBE);
  phj_unit_kernel<K><<<(unsigned)nunits, kThreads, dyn, s>>>(rk, roff, bits, sk, ns, io, ustat, ucounter, nunits,
                                                              ctx.d_status);
  return cuda_check(cudaGetLastError());
}

template <typename K>
gj_status join_groupby_typed(const Ctx& ctx, const gj_table* R, const gj_table* S, int variant, int bits, int bpp,
                             gj_colref gkref, int nagg, const int32_t* ops, const gj_colref* agg_cols,
                             const gj_options* opt, int64_t* out_keys, int64_t* const* out_aggs, int64_t cap,
                             int64_t* d_ngroups) {
  cudaStream_t s = ctx.stream;
  Scratch scr(s);
  gj_status st;
  if ((st = cuda_check(cudaMemsetAsync(d_ngroups, 0, sizeof(int64_t), s))) != GJ_OK) return st;
  const int64_t nr = R->n, ns = S->n;
  if (nr == 0 || ns == 0) return GJ_OK;
  const int kt = sizeof(K) == 8 ? GJ_I64 : GJ_I32;

  GroupSink G{};
  G.nagg = nagg;
  G.dense = gkref.modulus > 0 && gkref.modulus <= (int64_t(1) << 21);
  if (G.dense) {
    G.nslots = 2 * gkref.modulus - 1;
    G.dense_off = gkref.modulus - 1;
  } else {
    int64_t est = opt->groups_hint > 0 ? std::min<int64_t>(opt->groups_hint, ns) : ns;
    uint64_t c = 1;
    while (c < (uint64_t)std::max<int64_t>(2, 2 * est)) c <<= 1;
    G.nslots = (int64_t)c;
    G.mask = c - 1;
  }
  const int64_t total = G.nslots + (G.dense ? 0 : 1);
  const size_t smem_agg = (size_t)G.nslots * 8 * (nagg + 1);
  G.smem = G.dense && smem_agg <= 96 * 1024;
  G.cnt = scr.get_as<unsigned long long>(total);
  if (!G.dense) G.keys = scr.get_as<int64_t>(total);
  for (int j = 0; j < nagg; ++j) {
    G.op[j] = ops[j];
    G.agg[j] = scr.get_as<int64_t>(total);
  }
  int* counter = scr.get_as<int>(2);
  if (scr.failed()) return GJ_ERR_OOM;
  if ((st = cuda_check(cudaMemsetAsync(counter, 0, 2 * sizeof(int), s))) != GJ_OK) return st;
  {
    LaunchScope ls(ctx, KK_AGG_INIT);
    int blocks = (int)std::min<int64_t>((total + 255) / 256, (int64_t)ctx.num_sms * 8);
    sink_init_kernel<<<std::max(blocks, 1), 256, 0, s>>>(G);
  }

  // columns the query reads on each side
  bool need[2][kMaxCols] = {};
  auto mark = [&](const gj_colref& c) {
    if (c.col >= 0) need[c.side][c.col] = true;
  };
  mark(gkref);
  for (int j = 0; j < nagg; ++j)
    if (ops[j] != GJ_AGG_COUNT) mark(agg_cols[j]);
  const void* src[2][kMaxCols];
  for (int c = 0; c < R->ncols; ++c) src[0][c] = R->cols[c];
  for (int c = 0; c < S->ncols; ++c) src[1][c] = S->cols[c];
  const int32_t* tids[2] = {nullptr, nullptr};
  const gj_table* side_tab[2] = {R, S};
  const K* rk = (const K*)R->key;
  const K* sk = (const K*)S->key;
  int64_t* roff = nullptr;
  int32_t* ht = nullptr;
  uint64_t ht_slots = 0;

  if (variant == GJ_JOIN_NPHJ) {
    ht_slots = 1;
    while (ht_slots < (uint64_t)std::max<int64_t>(2 * nr, 2)) ht_slots <<= 1;
    ht = scr.get_as<int32_t>(ht_slots);
    if (scr.failed()) return GJ_ERR_OOM;
    if ((st = cuda_check(cudaMemsetAsync(ht, 0, sizeof(int32_t) * ht_slots, s))) != GJ_OK) return st;
    LaunchScope ls(ctx, KK_NPHJ_BUILD);
    int blocks = (int)std::min<int64_t>((nr + 255) / 256, (int64_t)ctx.num_sms * 16);
    nphj_build_kernel<K><<<blocks, 256, 0, s>>>(rk, nr, ht, ht_slots - 1, ctx.d_status);
  } else {
    const bool gftr = variant == GJ_JOIN_PHJ_TR;
    if (bits > 0) {
      for (int side = 0; side < 2; ++side) {
        const gj_table* T = side_tab[side];
        ColSet cs{};
        int pos[kMaxCols];
        if (gftr) {
          for (int c = 0; c < T->ncols; ++c) {
            if (!need[side][c]) continue;
            pos[c] = cs.n;
            cs.src[cs.n] = T->cols[c];
            cs.size[cs.n] = dtype_size(T->col_type[c]);
            cs.dst[cs.n] = scr.get((size_t)T->n * cs.size[cs.n]);
            cs.n++;
          }
        } else {
          cs.n = 1;
          cs.src[0] = nullptr;
          cs.size[0] = 4;
          cs.dst[0] = scr.get((size_t)T->n * 4);
        }
        K* k2 = scr.get_as<K>(T->n);
        if (scr.failed()) return GJ_ERR_OOM;
        if ((st = radix_partition_run(ctx, scr, kt, T->key, k2, cs, T->n, 0, bits, kHashed, bpp)) != GJ_OK) return st;
        if (side == 0)
          rk = k2;
        else
          sk = k2;
        if (gftr) {
          for (int c = 0; c < T->ncols; ++c)
            if (need[side][c]) src[side][c] = cs.dst[pos[c]];
        } else {
          tids[side] = (const int32_t*)cs.dst[0];
        }
      }
    }
    roff = scr.get_as<int64_t>(((size_t)1 << bits) + 1);
    if (scr.failed()) return GJ_ERR_OOM;
    if ((st = partition_bounds_run(ctx, kt, rk, nr, 0, bits, kHashed, roff)) != GJ_OK) return st;
  }

  auto ref = [&](const gj_colref& c) {
    FusedRef f{};
    f.mod = c.modulus;
    if (c.col < 0) {
      f.is_key = 1;
      return f;
    }
    f.side = c.side;
    f.src = src[c.side][c.col];
    f.size = dtype_size(side_tab[c.side]->col_type[c.col]);
    f.tid = tids[c.side];
    return f;
  };
  G.gk = ref(gkref);
  for (int j = 0; j < nagg; ++j)
    if (ops[j] != GJ_AGG_COUNT) G.val[j] = ref(agg_cols[j]);

  const size_t agg_dyn = G.smem ? smem_agg : 0;
  if (variant == GJ_JOIN_NPHJ) {
    if ((st = ensure_smem_attr(ctx, (const void*)nphj_probe_agg_kernel<K>, 96 * 1024)) != GJ_OK) return st;
    LaunchScope ls(ctx, KK_FUSED_PROBE);
    int blocks = (int)std::min<int64_t>((ns + kThreads - 1) / kThreads, (int64_t)ctx.num_sms * 4);
    nphj_probe_agg_kernel<K><<<blocks, kThreads, agg_dyn, s>>>(rk, ht, ht_slots - 1, sk, ns, G, ctx.d_status);
  } else {
    const int64_t ntiles = (ns + kTileS - 1) / kTileS;
    const size_t dyn = phj_smem_bytes<K>() + agg_dyn;
    if ((st = ensure_smem_attr(ctx, (const void*)phj_probe_agg_kernel<K>, (int)(phj_smem_bytes<K>() + 96 * 1024))) !=
        GJ_OK)
      return st;
    int per_sm = 1;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, phj_probe_agg_kernel<K>, kThreads, dyn);
    int blocks = (int)std::min<int64_t>(ntiles, (int64_t)ctx.num_sms * std::max(per_sm, 1));
    LaunchScope ls(ctx, KK_FUSED_PROBE);
    phj_probe_agg_kernel<K><<<blocks, kThreads, dyn, s>>>(rk, roff, bits, sk, ns, G, counter, ntiles, ctx.d_status);
  }

  const int64_t etiles = (total + kEmitTile - 1) / kEmitTile;
  uint64_t* tstat = scr.get_as<uint64_t>(etiles);
  if (scr.failed()) return GJ_ERR_OOM;
  if ((st = cuda_check(cudaMemsetAsync(tstat, 0, sizeof(uint64_t) * etiles, s))) != GJ_OK) return st;
  Aggs out{};
  out.n = nagg;
  for (int j = 0; j < nagg; ++j) out.out[j] = out_aggs[j];
  LaunchScope ls(ctx, KK_GROUP_EMIT);
  group_emit_kernel<<<(unsigned)etiles, kThreads, 0, s>>>(G, out_keys, out, cap, d_ngroups, tstat, counter + 1,
                                                          etiles, ctx.d_status);
  return cuda_check(cudaGetLastError());
}

}  // namespace

gj_status join_groupby_run(const Ctx& ctx, const gj_table* R, const gj_table* S, gj_colref gk, int nagg,
                           const int32_t* ops, const gj_colref* agg_cols, const gj_options* opt, int64_t* out_keys,
                           int64_t* const* out_aggs, int64_t cap, int64_t* d_ngroups) {
  const int variant = resolve_join_variant(R, S, nagg, opt, true);
  int bits = opt->radix_bits > 0 ? std::min(opt->radix_bits, 16) : choose_join_bits(R->n, 512);
  if (R->key_type == GJ_I64)
    return join_groupby_typed<int64_t>(ctx, R, S, variant, bits, opt->bits_per_pass, gk, nagg, ops, agg_cols, opt,
                                       out_keys, out_aggs, cap, d_ngroups);
  return join_groupby_typed<int32_t>(ctx, R, S, variant, bits, opt->bits_per_pass, gk, nagg, ops, agg_cols, opt,
                                     out_keys, out_aggs, cap, d_ngroups);
}

int choose_join_bits(int64_t nr, int64_t target) {
  int bits = 0;
  while (bits < 16 && (nr >> bits) > target) ++bits;
  return bits;
}

int heuristic_join_variant(const gj_table* R, const gj_options* opt) {
  // Sec. 7: GFTR when the match ratio is >= 25 %, the foreign keys are skewed or
  // keys are 8 bytes wide; otherwise the GFUR partitioned join. Unknown hints
  // read as the common case (all rows match, no skew); "skewed" is read as a
  // Zipf factor of at least 0.5.
  const float mr = opt->match_ratio_hint < 0 ? 1.0f : opt->match_ratio_hint;
  const float z = opt->zipf_hint < 0 ? 0.0f : opt->zipf_hint;
  return (mr >= 0.25f || z >= 0.5f || R->key_type == GJ_I64) ? GJ_JOIN_PHJ_TR : GJ_JOIN_PHJ_UR;
}

int resolve_join_variant(const gj_table* R, const gj_table* S, int nagg, const gj_options* opt, bool fused) {
  int variant = opt->join_variant;
  if (variant == GJ_JOIN_AUTO && opt->selector == GJ_SELECT_MLP) variant = mlp_choose(R, S, nagg, opt, true, fused);
  if (variant == GJ_JOIN_AUTO)
    variant = opt->selector == GJ_SELECT_HEURISTIC ? heuristic_join_variant(R, opt) : cost_join_variant(R, S, opt, fused);
  return variant;
}

gj_status join_run(const Ctx& ctx, const gj_table* R, const gj_table* S, const gj_options* opt, gj_table* T,
                   int64_t cap, int64_t* d_count) {
  const int variant = resolve_join_variant(R, S, 0, opt, false);
  int bits = opt->radix_bits > 0 ? std::min(opt->radix_bits, 16) : choose_join_bits(R->n, 512);
  // a build side that shared-memory partitions would need two passes for, but whose
  // 256 partitions stay L2-sized: one pass per side and L2-resident tables
  const bool l2 = (variant == GJ_JOIN_PHJ_TR || variant == GJ_JOIN_PHJ_UR) && opt->radix_bits <= 0 &&
                  bits > kL2Bits && R->n <= (int64_t(1) << 27);
  if (l2) bits = kL2Bits;
  if (R->key_type == GJ_I64)
    return join_typed<int64_t>(ctx, R, S, variant, bits, opt->bits_per_pass, l2, T, cap, d_count);
  return join_typed<int32_t>(ctx, R, S, variant, bits, opt->bits_per_pass, l2, T, cap, d_count);
}

}  // namespace gj
