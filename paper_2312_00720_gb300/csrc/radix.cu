// radix-partition (paper Sec. 2.3): stable partition of a key column and any
// number of payload columns on bits [lo, hi) of the key, partitions stored
// contiguously. Each pass of <= 8 bits reads key and columns once and writes
// them once.
//
// Per pass, a histogram kernel counts the digits of every tile of the pass's
// input (the paper's "histogram pass", per tile), and one block per digit scans
// those counts: every tile then knows where its rows of each digit go before the
// scatter starts, so tiles need no ordering or waiting between them. In the
// scatter, thread 0 of a block bulk-copies (cp.async.bulk, completion on an
// mbarrier) the tile's key into shared memory and prefetches its payload columns
// into L2 (cp.async.bulk.prefetch.L2). Keys are ranked stably per warp by a
// ballot multisplit (the warp's rows are contiguous, lanes in row order); per-digit warp
// counts give each row its position inside the tile's digit-sorted order. Every
// column is then gathered and written in that order through one permutation word
// per row, so warps store contiguous runs of each digit.
//
// Moving every payload column with the key in the same pass is what the GFTR
// pattern needs (Sec. 4.1.2): one rank computation places all columns. Four
// 4-byte columns can be written interleaved as one 16-byte row (ColSet::zip4),
// which later passes and the join's probe move with one access per row.
#include <cuda_runtime.h>

#include <algorithm>
#include <mutex>

#include "gj_internal.cuh"

namespace gj {

namespace {

constexpr int kRadixMax = 256;
constexpr int kHistThreads = 256;
constexpr int kThreads = 512;
constexpr int kWarps = kThreads / 32;
constexpr int kMaxChunks = 8;  // 32-row chunks per warp: tiles of up to 4096 rows
constexpr int kSmemBudget = 48 * 1024;  // staged key + per-row arrays; three blocks per SM

// 32-row chunks per warp for a key of key_size bytes: the staged key and 4 bytes of
// permutation per row within the budget. Tiles hold kThreads * chunks rows (4096
// for 4- and 8-byte keys).
constexpr int scatter_chunks(int key_size) {
  return kSmemBudget / (kThreads * (key_size + 4)) < 1 ? 1
         : (kSmemBudget / (kThreads * (key_size + 4)) > kMaxChunks ? kMaxChunks
                                                                    : kSmemBudget / (kThreads * (key_size + 4)));
}


// Exclusive scan of one value per thread over the block.
__device__ __forceinline__ uint32_t block_excl_scan(uint32_t v, uint32_t* s_warp) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  uint32_t x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) s_warp[warp] = x;
  __syncthreads();
  if (warp == 0) {
    uint32_t w = lane < kWarps ? s_warp[lane] : 0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      uint32_t y = __shfl_up_sync(0xffffffffu, w, o);
      if (lane >= o) w += y;
    }
    if (lane < kWarps) s_warp[lane] = w;
  }
  __syncthreads();
  uint32_t before = warp ? s_warp[warp - 1] : 0;
  __syncthreads();
  return before + x - v;
}

// ---------------------------------------------------------------- tile histograms
// Digit counts of every tile of tile_rows rows: tcount[d * ld + tile] (ld >= ntiles,
// a multiple of 4); the digit totals are added into total[d] (zeroed by the
// caller). Blocks stride over the tiles.
template <typename K>
__global__ void __launch_bounds__(kHistThreads) tile_hist_kernel(const K* __restrict__ kin, int64_t n, int shift,
                                                                  int width, int transform, int tile_rows,
                                                                  int64_t ld, uint32_t* __restrict__ tcount,
                                                                  uint32_t* __restrict__ total) {
  __shared__ uint32_t s_h[kRadixMax];
  __shared__ uint32_t s_tot[kRadixMax];
  const int radix = 1 << width;
  const int64_t ntiles = (n + tile_rows - 1) / tile_rows;
  constexpr int kVec = 16 / sizeof(K);
  const bool vec = (reinterpret_cast<uintptr_t>(kin) & 15) == 0;  // tile_rows * sizeof(K) is a multiple of 16
  for (int d = threadIdx.x; d < radix; d += kHistThreads) s_tot[d] = 0;
  for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    for (int d = threadIdx.x; d < radix; d += kHistThreads) s_h[d] = 0;
    __syncthreads();
    const int64_t tb = tile * tile_rows;
    const int tn = (int)min64(tile_rows, n - tb);
    const K* kt = kin + tb;
    int from = 0;
    if (vec) {
      const int nvec = tn / kVec;
      const uint4* body = reinterpret_cast<const uint4*>(kt);
      // all of a thread's loads first, then its counts
      constexpr int kLoads = 4;
      for (int v0 = 0; v0 < nvec; v0 += kLoads * kHistThreads) {
        uint4 u[kLoads];
#pragma unroll
        for (int q = 0; q < kLoads; ++q) {
          const int v = v0 + q * kHistThreads + threadIdx.x;
          u[q] = v < nvec ? __ldcs(body + v) : make_uint4(0, 0, 0, 0);
        }
#pragma unroll
        for (int q = 0; q < kLoads; ++q) {
          if (v0 + q * kHistThreads + threadIdx.x >= nvec) continue;
          const K* ks = reinterpret_cast<const K*>(&u[q]);
#pragma unroll
          for (int e = 0; e < kVec; ++e) atomicAdd(&s_h[extract_digit<K>(ks[e], transform, shift, width)], 1u);
        }
      }
      from = nvec * kVec;
    }
    for (int r = from + threadIdx.x; r < tn; r += kHistThreads)
      atomicAdd(&s_h[extract_digit<K>(kt[r], transform, shift, width)], 1u);
    __syncthreads();
    for (int d = threadIdx.x; d < radix; d += kHistThreads) {
      const uint32_t c = s_h[d];
      tcount[(int64_t)d * ld + tile] = c;
      s_tot[d] += c;
    }
  }
  __syncthreads();
  for (int d = threadIdx.x; d < radix; d += kHistThreads)
    if (s_tot[d]) atomicAdd(&total[d], s_tot[d]);
}

// In place: tcount[d * ld + t] -> the output position of tile t's first row with
// digit d = (rows of digits < d) + (rows with digit d in tiles < t). One block per
// digit; each thread scans a contiguous chunk of tiles, a multiple of 4 long, read
// and written with 16-byte accesses.
__global__ void __launch_bounds__(1024) tile_offsets_kernel(uint32_t* __restrict__ tcount,
                                                            const uint32_t* __restrict__ total, int64_t ld) {
  __shared__ uint32_t s_warp[32];
  __shared__ uint32_t s_base;
  const int d = blockIdx.x;
  if (threadIdx.x < 32) {
    uint32_t b = 0;
    for (int e = threadIdx.x; e < d; e += 32) b += total[e];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) b += __shfl_xor_sync(0xffffffffu, b, o);
    if (threadIdx.x == 0) s_base = b;
  }
  uint4* row = reinterpret_cast<uint4*>(tcount + (int64_t)d * ld);
  // entries past ntiles come after every real tile: what they hold changes no real offset
  const int64_t nv = ld / 4;
  const int64_t chunk = (nv + blockDim.x - 1) / blockDim.x;
  const int64_t v0 = min64((int64_t)threadIdx.x * chunk, nv), v1 = min64(v0 + chunk, nv);
  uint32_t sum = 0;
#pragma unroll 4
  for (int64_t v = v0; v < v1; ++v) {
    const uint4 u = row[v];
    sum += u.x + u.y + u.z + u.w;
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  uint32_t x = sum;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) s_warp[warp] = x;
  __syncthreads();
  if (warp == 0) {
    uint32_t w = lane < (int)(blockDim.x >> 5) ? s_warp[lane] : 0u;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(0xffffffffu, w, o);
      if (lane >= o) w += y;
    }
    s_warp[lane] = w;
  }
  __syncthreads();
  uint32_t run = s_base + (warp ? s_warp[warp - 1] : 0u) + x - sum;
#pragma unroll 4
  for (int64_t v = v0; v < v1; ++v) {
    uint4 u = row[v];
    uint4 o;
    o.x = run;
    o.y = run + u.x;
    o.z = o.y + u.y;
    o.w = o.z + u.z;
    run = o.w + u.w;
    row[v] = o;
  }
}

// ---------------------------------------------------------------- scatter
struct ScatterArgs {
  const void* kin;
  void* kout;
  ColSet cols;
  uint32_t gen_mask;  // columns whose values are the input row index (tuple ids)
  int64_t n;
  int shift, width, transform;
  const uint32_t* offs;  // [2^width][ld]: output position of each tile's first row of each digit
  int64_t ld;
  int* err;
  int tile_rows;  // 512 * chunks
  int chunks;     // 32-row chunks per warp
  int bulk;       // 1: every source is 16-byte aligned, copy with cp.async.bulk
  int32_t perm_off, wcnt_off;
  int4* zip_dst;  // non-null: the four 4-byte columns are written interleaved here instead
};

// Shared-memory layout for tiles of tile_rows rows: the staged key, the
// permutation words and the per-warp digit counts. Returns the dynamic
// shared-memory bytes.
int scatter_layout(ScatterArgs& a, int tile_rows, int key_size) {
  int off = tile_rows * key_size;
  off = (off + 15) & ~15;
  a.perm_off = off;
  off += tile_rows * 4;
  a.wcnt_off = off;
  off += kWarps * kRadixMax * 2;
  return off;
}

__device__ __forceinline__ void prefetch_l2(const void* p, uint32_t bytes) {
  asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(p), "r"(bytes) : "memory");
}

template <typename T>
__device__ __forceinline__ void stage_tail(unsigned char* stage, const T* src, int64_t tile_base, int tile_n,
                                           int from) {
  for (int r = from + threadIdx.x; r < tile_n; r += kThreads) ((T*)stage)[r] = src[tile_base + r];
}

// The valid lanes of the warp whose digit (< 2^width, width <= 8) equals this
// lane's: the AND, over the digit's bits, of each bit's ballot or its complement
// (warp-level multisplit; a handful of ballots cost less than one match.any).
__device__ __forceinline__ unsigned digit_peers(uint32_t d, int width, bool valid) {
  unsigned m = __ballot_sync(0xffffffffu, valid);
#pragma unroll
  for (int b = 0; b < 8; ++b) {
    if (b >= width) break;
    const bool bit = (d >> b) & 1u;
    const unsigned bb = __ballot_sync(0xffffffffu, bit);
    m &= bit ? bb : ~bb;
  }
  return m;
}

template <typename K>
__global__ void __launch_bounds__(kThreads, 3) radix_scatter_kernel(ScatterArgs a) {
  extern __shared__ __align__(128) unsigned char smem[];
  __shared__ uint32_t s_tstart[kRadixMax];
  __shared__ int32_t s_gdst[kRadixMax];  // output position of sorted position 0 of each digit
  __shared__ uint32_t s_scan[kWarps];
  __shared__ __align__(8) uint64_t s_bar[1];

  const int radix = 1 << a.width;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const unsigned lt_mask = (1u << lane) - 1;
  K* s_key = (K*)smem;
  uint32_t* s_perm = (uint32_t*)(smem + a.perm_off);  // sorted position -> digit << 16 | row of the tile
  uint16_t* s_wcnt = (uint16_t*)(smem + a.wcnt_off);  // [kWarps][kRadixMax]

  if (threadIdx.x == 0) {
    mbar_init(&s_bar[0], 1);
    mbar_fence_init();
  }
  __syncthreads();
  const int64_t tile = blockIdx.x;
  const int64_t tile_base = (int64_t)tile * a.tile_rows;
  const int tile_n = (int)min64(a.tile_rows, a.n - tile_base);

  // ---- stage the tile's key in shared memory (ranking needs only it); the columns
  // are prefetched into L2 and gathered from there in digit order, which keeps
  // shared memory small enough for three blocks per SM
  if (a.bulk) {
    if (threadIdx.x == 0) {
      uint32_t kb = ((uint32_t)tile_n * sizeof(K)) & ~15u;
      mbar_expect_tx(&s_bar[0], kb);
      if (kb) bulk_g2s(s_key, (const K*)a.kin + tile_base, kb, &s_bar[0]);
      for (int c = 0; c < a.cols.n; ++c) {
        if ((a.gen_mask >> c) & 1u) continue;
        uint32_t b = ((uint32_t)tile_n * a.cols.size[c]) & ~15u;
        if (b) prefetch_l2((const unsigned char*)a.cols.src[c] + tile_base * a.cols.size[c], b);
      }
    }
    stage_tail<K>(smem, (const K*)a.kin, tile_base, tile_n, (int)((((uint32_t)tile_n * sizeof(K)) & ~15u) / sizeof(K)));
  } else {
    stage_tail<K>(smem, (const K*)a.kin, tile_base, tile_n, 0);
  }
  for (int i = threadIdx.x; i < kWarps * kRadixMax; i += kThreads) s_wcnt[i] = 0;
  if (a.bulk) mbar_wait(&s_bar[0], 0, a.err);
  __syncthreads();

  // ---- stable rank inside the warp's contiguous rows
  uint16_t rank[kMaxChunks];
  uint8_t dg[kMaxChunks];
  const int seg = warp * a.chunks * 32;
#pragma unroll
  for (int i = 0; i < kMaxChunks; ++i) {
    if (i >= a.chunks) break;
    const int row = seg + i * 32 + lane;
    const bool valid = row < tile_n;
    const uint32_t d = valid ? extract_digit<K>(s_key[row], a.transform, a.shift, a.width) : 0u;
    const unsigned peers = digit_peers(d, a.width, valid);
    uint32_t cnt = 0;
    if (valid) cnt = s_wcnt[warp * kRadixMax + d];
    __syncwarp();
    if (valid && (peers & lt_mask) == 0) s_wcnt[warp * kRadixMax + d] = (uint16_t)(cnt + __popc(peers));
    __syncwarp();
    rank[i] = (uint16_t)(cnt + __popc(peers & lt_mask));
    dg[i] = (uint8_t)d;
  }
  __syncthreads();

  // ---- per digit: warp offsets, tile count, tile-local starts; the tile's output
  // position for each digit comes from the tile histograms of the pass
  const int d = threadIdx.x;
  uint32_t tcnt = 0;
  if (d < radix) {
#pragma unroll
    for (int w = 0; w < kWarps; ++w) {
      uint32_t c = s_wcnt[w * kRadixMax + d];
      s_wcnt[w * kRadixMax + d] = (uint16_t)tcnt;
      tcnt += c;
    }
  }
  const uint32_t tstart = block_excl_scan(tcnt, s_scan);
  if (d < radix) {
    s_tstart[d] = tstart;
    s_gdst[d] = (int32_t)(a.offs[(int64_t)d * a.ld + tile] - tstart);  // rows < 2^31
  }
  __syncthreads();

  // ---- inverse index: sorted position -> row of the tile
#pragma unroll
  for (int i = 0; i < kMaxChunks; ++i) {
    if (i >= a.chunks) break;
    const int row = seg + i * 32 + lane;
    if (row < tile_n) {
      const uint32_t p = s_tstart[dg[i]] + s_wcnt[warp * kRadixMax + dg[i]] + rank[i];
      s_perm[p] = (uint32_t)dg[i] << 16 | (uint32_t)row;
    }
  }
  __syncthreads();

  // ---- write every column in digit-sorted order. Thread t owns sorted positions
  // t, t + kThreads, ...: their destinations and source rows are computed once
  // and reused for every column.
  uint32_t dst_at[kMaxChunks];
  uint16_t src_at[kMaxChunks];
#pragma unroll
  for (int i = 0; i < kMaxChunks; ++i) {
    if (i >= a.chunks) break;
    const int p = threadIdx.x + i * kThreads;
    if (p < tile_n) {
      const uint32_t e = s_perm[p];
      dst_at[i] = (uint32_t)(s_gdst[e >> 16] + p);
      src_at[i] = (uint16_t)(e & 0xffffu);
    }
  }
  {
    K* __restrict__ kout = (K*)a.kout;
#pragma unroll
    for (int i = 0; i < kMaxChunks; ++i) {
      if (i >= a.chunks) break;
      if (threadIdx.x + i * kThreads < tile_n) kout[dst_at[i]] = s_key[src_at[i]];
    }
  }
  if (a.zip_dst) {
    // four 4-byte columns -> one 16-byte row each
    const int32_t* st0 = (const int32_t*)a.cols.src[0] + tile_base;
    const int32_t* st1 = (const int32_t*)a.cols.src[1] + tile_base;
    const int32_t* st2 = (const int32_t*)a.cols.src[2] + tile_base;
    const int32_t* st3 = (const int32_t*)a.cols.src[3] + tile_base;
#pragma unroll
    for (int i = 0; i < kMaxChunks; ++i) {
      if (i >= a.chunks) break;
      if (threadIdx.x + i * kThreads < tile_n) {
        const int r = src_at[i];
        a.zip_dst[dst_at[i]] = make_int4(st0[r], st1[r], st2[r], st3[r]);
      }
    }
    return;
  }
  for (int c = 0; c < a.cols.n; ++c) {
    const bool gen = (a.gen_mask >> c) & 1u;
    if (a.cols.size[c] == 16) {
      const int4* st = (const int4*)a.cols.src[c] + tile_base;
      int4* __restrict__ dst = (int4*)a.cols.dst[c];
#pragma unroll
      for (int i = 0; i < kMaxChunks; ++i) {
        if (i >= a.chunks) break;
        if (threadIdx.x + i * kThreads < tile_n) dst[dst_at[i]] = st[src_at[i]];
      }
    } else if (a.cols.size[c] == 8) {
      const int64_t* st = gen ? nullptr : (const int64_t*)a.cols.src[c] + tile_base;
      int64_t* __restrict__ dst = (int64_t*)a.cols.dst[c];
#pragma unroll
      for (int i = 0; i < kMaxChunks; ++i) {
        if (i >= a.chunks) break;
        if (threadIdx.x + i * kThreads < tile_n) dst[dst_at[i]] = gen ? tile_base + src_at[i] : st[src_at[i]];
      }
    } else {
      const int32_t* st = gen ? nullptr : (const int32_t*)a.cols.src[c] + tile_base;
      int32_t* __restrict__ dst = (int32_t*)a.cols.dst[c];
#pragma unroll
      for (int i = 0; i < kMaxChunks; ++i) {
        if (i >= a.chunks) break;
        if (threadIdx.x + i * kThreads < tile_n)
          dst[dst_at[i]] = gen ? (int32_t)(tile_base + src_at[i]) : st[src_at[i]];
      }
    }
  }
}

template <typename K>
__global__ void bounds_kernel(const K* __restrict__ keys, int64_t n, int shift, int width, int transform,
                              int64_t* __restrict__ off) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  const int64_t nparts = int64_t(1) << width;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i <= n; i += stride) {
    int64_t di = i < n ? (int64_t)extract_digit<K>(keys[i], transform, shift, width) : nparts;
    int64_t dp = i > 0 ? (int64_t)extract_digit<K>(keys[i - 1], transform, shift, width) : -1;
    for (int64_t p = dp + 1; p <= di; ++p) off[p] = i;
  }
}

bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15) == 0; }

template <typename K>
gj_status radix_partition_typed(const Ctx& ctx, Scratch& scr, const K* kin, K* kout, const ColSet& cols_in,
                                int64_t n, int lo, int hi, int transform, int bits_per_pass) {
  RadixPlan plan = make_radix_plan(lo, hi, bits_per_pass);
  if (n == 0) return GJ_OK;
  uint32_t gen_mask = 0;
  for (int c = 0; c < cols_in.n; ++c)
    if (cols_in.src[c] == nullptr) gen_mask |= 1u << c;
  const int chunks = scatter_chunks((int)sizeof(K));
  const int tile_rows = kThreads * chunks;
  const int64_t tiles = (n + tile_rows - 1) / tile_rows;

  // the columns every pass after the first reads and writes: with zip4 the
  // interleaved 16-byte rows, else the input's columns
  const bool zip = cols_in.zip4 != 0;
  ColSet out_set = cols_in;
  out_set.zip4 = 0;
  if (zip) {
    out_set.n = 1;
    out_set.size[0] = 16;
  }
  ColSet tmp = out_set;
  K* ktmp = nullptr;
  uint32_t* total = scr.get_as<uint32_t>((size_t)plan.passes * kRadixMax);
  const int64_t ld = (tiles + 3) & ~int64_t(3);                      // row stride of the tile offsets
  uint32_t* offs = scr.get_as<uint32_t>((size_t)ld * kRadixMax);     // reused by every pass
  if (plan.passes > 1) {
    ktmp = scr.get_as<K>(n);
    for (int c = 0; c < out_set.n; ++c) tmp.dst[c] = scr.get((size_t)n * out_set.size[c]);
  }
  if (scr.failed()) return GJ_ERR_OOM;
  cudaStream_t s = ctx.stream;
  gj_status st;
  if ((st = cuda_check(cudaMemsetAsync(total, 0, sizeof(uint32_t) * plan.passes * kRadixMax, s))) != GJ_OK) return st;
  if ((st = ensure_smem_attr(ctx, (const void*)radix_scatter_kernel<K>, kSmemBudget + 16 * 1024)) != GJ_OK) return st;
  for (int q = 0; q < plan.passes; ++q) {
    const bool to_out = ((plan.passes - 1 - q) % 2) == 0;
    ScatterArgs a{};
    a.n = n;
    a.transform = transform;
    a.tile_rows = tile_rows;
    a.chunks = chunks;
    a.kin = q == 0 ? (const void*)kin : (to_out ? (const void*)ktmp : (const void*)kout);
    a.kout = to_out ? (void*)kout : (void*)ktmp;
    const ColSet& dst_set = to_out ? out_set : tmp;
    const ColSet& prev_set = to_out ? tmp : out_set;  // where the previous pass wrote
    if (q == 0) {
      a.cols = cols_in;
      if (zip)
        a.zip_dst = (int4*)dst_set.dst[0];
      else
        for (int c = 0; c < cols_in.n; ++c) a.cols.dst[c] = dst_set.dst[c];
    } else {
      a.cols = out_set;
      for (int c = 0; c < out_set.n; ++c) {
        a.cols.src[c] = prev_set.dst[c];
        a.cols.dst[c] = dst_set.dst[c];
      }
    }
    bool bulk = aligned16(a.kin);
    for (int c = 0; c < a.cols.n; ++c)
      if (a.cols.src[c] && !aligned16(a.cols.src[c])) bulk = false;
    a.gen_mask = q == 0 ? gen_mask : 0u;
    a.bulk = bulk ? 1 : 0;
    a.shift = plan.shift[q];
    a.width = plan.width[q];
    a.offs = offs;
    a.ld = ld;
    a.err = ctx.d_status;
    // tuple ids are generated in the first pass and staged like any column after it
    const size_t dyn = (size_t)scatter_layout(a, tile_rows, (int)sizeof(K));
    {
      // where each tile's rows of each digit go: tile histograms, then their scan
      LaunchScope ls(ctx, KK_RADIX_HIST);
      const unsigned hb = (unsigned)std::min<int64_t>(tiles, (int64_t)ctx.num_sms * 8);
      tile_hist_kernel<K><<<hb, kHistThreads, 0, s>>>((const K*)a.kin, n, a.shift, a.width, transform, tile_rows, ld,
                                                      offs, total + q * kRadixMax);
    }
    {
      LaunchScope ls(ctx, KK_RADIX_HIST);
      tile_offsets_kernel<<<1u << a.width, 1024, 0, s>>>(offs, total + q * kRadixMax, ld);
    }
    LaunchScope ls(ctx, KK_RADIX_SCATTER);
    radix_scatter_kernel<K><<<(unsigned)tiles, kThreads, dyn, s>>>(a);
  }
  return cuda_check(cudaGetLastError());
}

}  // namespace

RadixPlan make_radix_plan(int lo, int hi, int bits_per_pass) {
  RadixPlan p{};
  int total = hi - lo;
  if (total <= 0) {
    p.passes = 0;
    return p;
  }
  int bpp = bits_per_pass > 0 ? std::min(bits_per_pass, 8) : 8;
  int passes = (total + bpp - 1) / bpp;
  // balanced widths: e.g. 14 bits -> 7 + 7 rather than 8 + 6
  int base = total / passes, extra = total % passes, sh = lo;
  for (int q = 0; q < passes; ++q) {
    int w = base + (q < extra ? 1 : 0);
    p.shift[q] = sh;
    p.width[q] = w;
    sh += w;
  }
  p.passes = passes;
  return p;
}

gj_status radix_partition_run(const Ctx& ctx, Scratch& scr, int key_type, const void* kin, void* kout,
                              const ColSet& cols, int64_t n, int lo, int hi, int transform, int bits_per_pass) {
  if (key_type == GJ_I64)
    return radix_partition_typed<int64_t>(ctx, scr, (const int64_t*)kin, (int64_t*)kout, cols, n, lo, hi,
                                          transform, bits_per_pass);
  return radix_partition_typed<int32_t>(ctx, scr, (const int32_t*)kin, (int32_t*)kout, cols, n, lo, hi, transform,
                                        bits_per_pass);
}

// ---------------------------------------------------------------- allocation-free variant
// For callers that cannot allocate device memory: a single-pass partition whose
// scratch (digit totals, per-tile digit offsets) is this file-scope
// array instead of stream-ordered allocations. It holds kNoAllocWords 32-bit
// words (about 0.5 MB) on every device that loads the library, until exit.
namespace {
constexpr int64_t kNoAllocMaxRows = int64_t(1) << 21;
// tiles of the smaller of the two key widths' tile sizes bound the tile count
constexpr int kNoAllocTileRows =
    kThreads * (scatter_chunks(4) < scatter_chunks(8) ? scatter_chunks(4) : scatter_chunks(8));
constexpr int kNoAllocMaxTiles = (int)((kNoAllocMaxRows + kNoAllocTileRows - 1) / kNoAllocTileRows);
static_assert(kNoAllocMaxTiles % 4 == 0, "the offset rows are padded to a multiple of 4 tiles");
constexpr size_t kNoAllocHead = 320;                                  // digit totals (256), padded
constexpr size_t kNoAllocWords = kNoAllocHead + (size_t)kNoAllocMaxTiles * kRadixMax;
__device__ __align__(256) uint32_t g_noalloc_scratch[kNoAllocWords];
__device__ __align__(256) int g_noalloc_status[64];
constexpr int kNoAllocDevices = 64;
uint32_t* g_noalloc_ptr[kNoAllocDevices] = {nullptr};
int* g_noalloc_err[kNoAllocDevices] = {nullptr};
std::mutex g_noalloc_mu;

template <typename K>
gj_status noalloc_partition(const Ctx& ctx, uint32_t* scratch, const gj_table* in, gj_table* out, int lo, int hi,
                            int transform, int64_t* d_off) {
  const int64_t n = in->n;
  const int width = hi - lo;
  ColSet cols{};
  cols.n = in->ncols;
  for (int c = 0; c < in->ncols; ++c) {
    cols.src[c] = in->cols[c];
    cols.dst[c] = out->cols[c];
    cols.size[c] = dtype_size(in->col_type[c]);
  }
  const int chunks = scatter_chunks((int)sizeof(K));
  const int tile_rows = kThreads * chunks;
  const int64_t tiles = (n + tile_rows - 1) / tile_rows;
  if (tiles > kNoAllocMaxTiles) return GJ_ERR_UNSUPPORTED;  // not reached: n <= kNoAllocMaxRows
  ScatterArgs a{};
  a.kin = in->key;
  a.kout = out->key;
  a.cols = cols;
  a.n = n;
  a.shift = lo;
  a.width = width;
  a.transform = transform;
  a.offs = scratch + kNoAllocHead;
  a.ld = (tiles + 3) & ~int64_t(3);
  a.err = ctx.d_status;
  a.tile_rows = tile_rows;
  a.chunks = chunks;
  bool bulk = aligned16(in->key);
  for (int c = 0; c < cols.n; ++c)
    if (!aligned16(cols.src[c])) bulk = false;
  a.bulk = bulk ? 1 : 0;
  const int off = scatter_layout(a, tile_rows, (int)sizeof(K));
  cudaStream_t s = ctx.stream;
  gj_status st;
  // the array keeps the previous call's contents: clear what must start at zero (the
  // digit totals; every tile writes all of its offsets)
  if ((st = cuda_check(cudaMemsetAsync(scratch, 0, sizeof(uint32_t) * kNoAllocHead, s))) != GJ_OK) return st;
  {
    LaunchScope ls(ctx, KK_RADIX_HIST);
    const unsigned hb = (unsigned)std::min<int64_t>(tiles, (int64_t)ctx.num_sms * 8);
    tile_hist_kernel<K><<<hb, kHistThreads, 0, s>>>((const K*)in->key, n, lo, width, transform, tile_rows, a.ld,
                                                    scratch + kNoAllocHead, scratch);
  }
  {
    LaunchScope ls(ctx, KK_RADIX_HIST);
    tile_offsets_kernel<<<1u << width, 1024, 0, s>>>(scratch + kNoAllocHead, scratch, a.ld);
  }
  if ((st = ensure_smem_attr(ctx, (const void*)radix_scatter_kernel<K>, kSmemBudget + 16 * 1024)) != GJ_OK) return st;
  {
    LaunchScope ls(ctx, KK_RADIX_SCATTER);
    radix_scatter_kernel<K><<<(unsigned)tiles, kThreads, (size_t)off, s>>>(a);
  }
  if ((st = cuda_check(cudaGetLastError())) != GJ_OK) return st;
  if (d_off) return partition_bounds_run(ctx, in->key_type, out->key, n, lo, width, transform, d_off);
  return GJ_OK;
}
}  // namespace

gj_status partition_bounds_run(const Ctx& ctx, int key_type, const void* keys, int64_t n, int lo, int width,
                               int transform, int64_t* d_off) {
  int blocks = (int)std::max<int64_t>(1, std::min<int64_t>((n + 256) / 256, (int64_t)ctx.num_sms * 8));
  LaunchScope ls(ctx, KK_PART_BOUNDS);
  if (key_type == GJ_I64)
    bounds_kernel<int64_t><<<blocks, 256, 0, ctx.stream>>>((const int64_t*)keys, n, lo, width, transform, d_off);
  else
    bounds_kernel<int32_t><<<blocks, 256, 0, ctx.stream>>>((const int32_t*)keys, n, lo, width, transform, d_off);
  return cuda_check(cudaGetLastError());
}

}  // namespace gj

extern "C" gj_status gj_radix_partition_noalloc(const gj_table* in, int32_t bit_lo, int32_t bit_hi,
                                                int32_t key_transform, gj_table* out, int64_t* d_offsets,
                                                int32_t sync, void* stream) {
  using namespace gj;
  if (!in || !out) return GJ_ERR_INVALID_ARG;
  for (const gj_table* t : {in, (const gj_table*)out}) {
    if ((t->key_type != GJ_I32 && t->key_type != GJ_I64) || t->ncols < 0 || t->ncols > GJ_MAX_COLS || t->n < 0)
      return GJ_ERR_INVALID_ARG;
    if (in->n > 0 && !t->key) return GJ_ERR_INVALID_ARG;
    for (int c = 0; c < t->ncols; ++c)
      if ((t->col_type[c] != GJ_I32 && t->col_type[c] != GJ_I64) || (in->n > 0 && !t->cols[c]))
        return GJ_ERR_INVALID_ARG;
  }
  if (out->key_type != in->key_type || out->ncols != in->ncols || out->n < in->n) return GJ_ERR_INVALID_ARG;
  for (int c = 0; c < in->ncols; ++c)
    if (out->col_type[c] != in->col_type[c]) return GJ_ERR_INVALID_ARG;
  const int kbits = in->key_type == GJ_I64 ? 64 : 32;
  if (bit_lo < 0 || bit_hi <= bit_lo || bit_hi > kbits || key_transform < 0 || key_transform > 2)
    return GJ_ERR_INVALID_ARG;
  // beyond the fixed scratch: one pass of at most 8 bits over at most 2^21 rows
  if (bit_hi - bit_lo > 8 || in->n > kNoAllocMaxRows) return GJ_ERR_UNSUPPORTED;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kNoAllocDevices) return GJ_ERR_CUDA;
  Ctx ctx{};
  {
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (!g_noalloc_ptr[dev]) {
      // one-time set-up on this device: the device addresses of the arrays
      void* p = nullptr;
      void* e = nullptr;
      if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess) return GJ_ERR_CUDA;
      if (cudaGetSymbolAddress(&e, g_noalloc_status) != cudaSuccess) return GJ_ERR_CUDA;
      g_noalloc_ptr[dev] = (uint32_t*)p;
      g_noalloc_err[dev] = (int*)e;
    }
    ctx.d_status = g_noalloc_err[dev];
  }
  ctx.stream = (cudaStream_t)stream;
  ctx.device = dev;
  cudaDeviceGetAttribute(&ctx.num_sms, cudaDevAttrMultiProcessorCount, dev);
  cudaDeviceGetAttribute(&ctx.smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  gj_status st;
  if (in->n == 0)  // nothing to move; the bounds are all zero
    st = d_offsets ? partition_bounds_run(ctx, in->key_type, out->key, 0, bit_lo, bit_hi - bit_lo, key_transform,
                                          d_offsets)
                   : GJ_OK;
  else
    st = in->key_type == GJ_I64
             ? noalloc_partition<int64_t>(ctx, g_noalloc_ptr[dev], in, out, bit_lo, bit_hi, key_transform, d_offsets)
             : noalloc_partition<int32_t>(ctx, g_noalloc_ptr[dev], in, out, bit_lo, bit_hi, key_transform, d_offsets);
  // every call, empty or not, ends the same way: with sync = 1 it returns (and
  // clears) what its kernels and earlier sync = 0 calls recorded
  if (st != GJ_OK || !sync) return st;
  int h = 0;
  if (cudaStreamSynchronize(ctx.stream) != cudaSuccess) return GJ_ERR_CUDA;
  if (cudaMemcpy(&h, ctx.d_status, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) return GJ_ERR_CUDA;
  if (h != 0 && cudaMemset(ctx.d_status, 0, sizeof(int)) != cudaSuccess) return GJ_ERR_CUDA;
  return (gj_status)h;
}
