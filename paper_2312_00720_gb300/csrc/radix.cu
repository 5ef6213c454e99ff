// radix-partition (paper Sec. 2.3): stable partition of a key column and any
// number of payload columns on bits [lo, hi) of the key, partitions stored
// contiguously. One read of the keys builds the digit histogram of every pass
// (the paper's "histogram pass"); then each pass of <= 8 bits reads key and
// columns once and writes them once, sequentially, in tiles that are ranked
// stably in shared memory and placed with a decoupled look-back over tiles.
//
// Moving every payload column with the key in the same pass is what the GFTR
// pattern needs (Sec. 4.1.2): all columns land in the same positions because
// one rank computation drives all of them.
#include <cuda_runtime.h>

#include <algorithm>

#include "gj_internal.cuh"

namespace gj {

namespace {

constexpr int kRadixMax = 256;
constexpr int kScatterThreads = 256;
constexpr int kScatterItems = 16;
constexpr int kTile = kScatterThreads * kScatterItems;
constexpr int kWarps = kScatterThreads / 32;
constexpr uint32_t kSFlagAgg = 1u << 30;
constexpr uint32_t kSFlagInc = 2u << 30;
constexpr uint32_t kSVal = (1u << 30) - 1;

struct PassDigits {
  int passes;
  int shift[16];
  int width[16];
};

// Exclusive scan of one value per thread over a 256-thread block.
__device__ __forceinline__ uint32_t block_excl_scan256(uint32_t v, uint32_t* s_warp, uint32_t* total) {
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
  if (total) *total = s_warp[kWarps - 1];
  __syncthreads();
  return before + x - v;
}

template <typename K>
__global__ void __launch_bounds__(256) radix_hist_kernel(const K* __restrict__ kin, int64_t n, PassDigits pd,
                                                         int transform, uint32_t* __restrict__ hist) {
  __shared__ uint32_t sh[16][kRadixMax];
  for (int i = threadIdx.x; i < pd.passes * kRadixMax; i += blockDim.x) (&sh[0][0])[i] = 0;
  __syncthreads();
  // 16-byte vector loads over the aligned body, scalar loads for the ragged ends
  constexpr int kVec = 16 / sizeof(K);
  const uintptr_t addr = reinterpret_cast<uintptr_t>(kin);
  int64_t head = (int64_t)(((16 - (addr & 15)) & 15) / sizeof(K));
  if ((addr % sizeof(K)) != 0 || head > n) head = n;
  const int64_t nvec = (n - head) / kVec;
  const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  auto count = [&](K k) {
    for (int q = 0; q < pd.passes; ++q) atomicAdd(&sh[q][extract_digit<K>(k, transform, pd.shift[q], pd.width[q])], 1u);
  };
  const uint4* body = reinterpret_cast<const uint4*>(kin + head);
  for (int64_t v = tid; v < nvec; v += stride) {
    uint4 u = __ldcs(body + v);
    const K* ks = reinterpret_cast<const K*>(&u);
#pragma unroll
    for (int e = 0; e < kVec; ++e) count(ks[e]);
  }
  for (int64_t i = tid; i < head; i += stride) count(kin[i]);
  for (int64_t i = head + nvec * kVec + tid; i < n; i += stride) count(kin[i]);
  __syncthreads();
  for (int i = threadIdx.x; i < pd.passes * kRadixMax; i += blockDim.x) {
    uint32_t c = (&sh[0][0])[i];
    if (c) atomicAdd(&hist[i], c);
  }
}

template <typename T>
__device__ __forceinline__ void scatter_column(const T* __restrict__ src, T* __restrict__ dst, bool gen_tid,
                                               int64_t seg, int lane, const uint32_t* spos, int nvalid_mask_items,
                                               int64_t n, T* staging, const int64_t* s_gdst, const uint8_t* s_sdig,
                                               int tile_n, int64_t tile_base) {
#pragma unroll
  for (int i = 0; i < kScatterItems; ++i) {
    int64_t row = seg + i * 32 + lane;
    if (row < n) {
      T v = gen_tid ? (T)row : src[row];
      staging[spos[i]] = v;
    }
  }
  __syncthreads();
  for (int p = threadIdx.x; p < tile_n; p += kScatterThreads) dst[s_gdst[s_sdig[p]] + p] = staging[p];
  __syncthreads();
}

template <typename K>
__global__ void __launch_bounds__(kScatterThreads) radix_scatter_kernel(
    const K* __restrict__ kin, K* __restrict__ kout, ColSet cols, uint32_t gen_tid_mask, int64_t n, int shift,
    int width, int transform, const uint32_t* __restrict__ hist, uint32_t* status, int* tile_counter, int* err) {
  extern __shared__ __align__(16) unsigned char s_stage_raw[];
  __shared__ uint32_t s_wcnt[kWarps][kRadixMax];
  __shared__ uint32_t s_tstart[kRadixMax];
  __shared__ uint32_t s_dbase[kRadixMax];
  __shared__ int64_t s_gdst[kRadixMax];
  __shared__ uint8_t s_sdig[kTile];
  __shared__ uint32_t s_scan[kWarps];
  __shared__ int s_tile;

  const int radix = 1 << width;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const unsigned lt_mask = (1u << lane) - 1;

  if (threadIdx.x == 0) s_tile = atomicAdd(tile_counter, 1);
  for (int i = threadIdx.x; i < kWarps * kRadixMax; i += kScatterThreads) (&s_wcnt[0][0])[i] = 0;
  __syncthreads();
  const int tile = s_tile;
  const int64_t tile_base = (int64_t)tile * kTile;
  const int tile_n = (int)min64(kTile, n - tile_base);
  const int64_t seg = tile_base + (int64_t)warp * (32 * kScatterItems);

  // ---- load keys, rank stably within the warp's contiguous segment
  K key[kScatterItems];
  uint32_t dig[kScatterItems];
  uint32_t spos[kScatterItems];
#pragma unroll
  for (int i = 0; i < kScatterItems; ++i) {
    int64_t row = seg + i * 32 + lane;
    key[i] = row < n ? kin[row] : K(0);
  }
#pragma unroll
  for (int i = 0; i < kScatterItems; ++i) {
    int64_t row = seg + i * 32 + lane;
    const bool valid = row < n;
    uint32_t d = valid ? extract_digit<K>(key[i], transform, shift, width) : 0xffffffffu;
    unsigned peers = __match_any_sync(0xffffffffu, d);
    uint32_t cnt = 0;
    if (valid) cnt = s_wcnt[warp][d];
    __syncwarp();
    if (valid && (peers & lt_mask) == 0) s_wcnt[warp][d] = cnt + __popc(peers);
    __syncwarp();
    dig[i] = d;
    spos[i] = cnt + __popc(peers & lt_mask);  // rank among equal digits of this warp so far
  }
  __syncthreads();

  // ---- per digit: exclusive offsets of the warps, tile count, publish aggregate
  const int d = threadIdx.x;  // kScatterThreads == kRadixMax
  uint32_t tcnt = 0;
  if (d < radix) {
#pragma unroll
    for (int w = 0; w < kWarps; ++w) {
      uint32_t c = s_wcnt[w][d];
      s_wcnt[w][d] = tcnt;
      tcnt += c;
    }
    st_volatile32(&status[(int64_t)tile * radix + d], (tile == 0 ? kSFlagInc : kSFlagAgg) | tcnt);
  }
  uint32_t hv = d < radix ? hist[d] : 0;
  uint32_t tstart = block_excl_scan256(tcnt, s_scan, nullptr);
  uint32_t dbase = block_excl_scan256(hv, s_scan, nullptr);
  if (d < radix) {
    s_tstart[d] = tstart;
    s_dbase[d] = dbase;
    // ---- decoupled look-back over preceding tiles for this digit
    uint32_t excl = 0;
    if (tile > 0) {
      int64_t t = tile - 1;
      uint32_t spins = 0;
      while (t >= 0) {
        uint32_t w = ld_volatile32(&status[t * radix + d]);
        uint32_t flag = w & ~kSVal;
        if (flag == 0) {
          if (++spins > kSpinLimit) {
            set_status(err, GJ_ERR_TIMEOUT);
            break;
          }
          continue;
        }
        excl += w & kSVal;
        if (flag == kSFlagInc) break;
        --t;
      }
      st_volatile32(&status[(int64_t)tile * radix + d], kSFlagInc | (excl + tcnt));
    }
    s_gdst[d] = (int64_t)dbase + excl - tstart;
  }
  __syncthreads();

  // ---- sorted position inside the tile; digit of every sorted position
#pragma unroll
  for (int i = 0; i < kScatterItems; ++i) {
    int64_t row = seg + i * 32 + lane;
    if (row < n) {
      uint32_t p = s_tstart[dig[i]] + s_wcnt[warp][dig[i]] + spos[i];
      spos[i] = p;
      s_sdig[p] = (uint8_t)dig[i];
    }
  }
  // keys
  {
    K* st = (K*)s_stage_raw;
#pragma unroll
    for (int i = 0; i < kScatterItems; ++i) {
      int64_t row = seg + i * 32 + lane;
      if (row < n) st[spos[i]] = key[i];
    }
    __syncthreads();
    for (int p = threadIdx.x; p < tile_n; p += kScatterThreads) kout[s_gdst[s_sdig[p]] + p] = st[p];
    __syncthreads();
  }
  // payload columns, all through the same positions
  for (int c = 0; c < cols.n; ++c) {
    const bool gen = (gen_tid_mask >> c) & 1u;
    if (cols.size[c] == 8)
      scatter_column<int64_t>((const int64_t*)cols.src[c], (int64_t*)cols.dst[c], gen, seg, lane, spos, 0, n,
                              (int64_t*)s_stage_raw, s_gdst, s_sdig, tile_n, tile_base);
    else
      scatter_column<int32_t>((const int32_t*)cols.src[c], (int32_t*)cols.dst[c], gen, seg, lane, spos, 0, n,
                              (int32_t*)s_stage_raw, s_gdst, s_sdig, tile_n, tile_base);
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

template <typename K>
gj_status radix_partition_typed(const Ctx& ctx, Scratch& scr, const K* kin, K* kout, const ColSet& cols_in,
                                int64_t n, int lo, int hi, int transform, int bits_per_pass) {
  RadixPlan plan = make_radix_plan(lo, hi, bits_per_pass);
  if (n == 0) return GJ_OK;
  PassDigits pd;
  pd.passes = plan.passes;
  for (int q = 0; q < plan.passes; ++q) {
    pd.shift[q] = plan.shift[q];
    pd.width[q] = plan.width[q];
  }
  const int64_t tiles = (n + kTile - 1) / kTile;
  uint32_t* hist = scr.get_as<uint32_t>((size_t)plan.passes * kRadixMax);
  size_t status_words = (size_t)tiles * kRadixMax;
  uint32_t* status = scr.get_as<uint32_t>(status_words * plan.passes);
  int* counters = scr.get_as<int>(plan.passes);
  // one scratch buffer (keys + columns) ping-pongs with the output
  K* ktmp = nullptr;
  ColSet tmp = cols_in;
  if (plan.passes > 1) {
    ktmp = scr.get_as<K>(n);
    for (int c = 0; c < cols_in.n; ++c) tmp.dst[c] = scr.get((size_t)n * cols_in.size[c]);
  }
  if (scr.failed()) return GJ_ERR_OOM;
  cudaStream_t s = ctx.stream;
  gj_status st;
  if ((st = cuda_check(cudaMemsetAsync(hist, 0, sizeof(uint32_t) * plan.passes * kRadixMax, s))) != GJ_OK) return st;
  if ((st = cuda_check(cudaMemsetAsync(status, 0, sizeof(uint32_t) * status_words * plan.passes, s))) != GJ_OK)
    return st;
  if ((st = cuda_check(cudaMemsetAsync(counters, 0, sizeof(int) * plan.passes, s))) != GJ_OK) return st;

  int hist_blocks = (int)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, (int64_t)ctx.num_sms * 8));
  {
    LaunchScope ls(ctx, KK_RADIX_HIST);
    radix_hist_kernel<K><<<hist_blocks, 256, 0, s>>>(kin, n, pd, transform, hist);
  }

  int max_size = sizeof(K);
  uint32_t gen_mask = 0;
  for (int c = 0; c < cols_in.n; ++c) {
    max_size = std::max(max_size, cols_in.size[c]);
    if (cols_in.src[c] == nullptr) gen_mask |= 1u << c;
  }
  const size_t dyn = (size_t)kTile * max_size;
  static bool attr_set[2] = {false, false};
  if (!attr_set[sizeof(K) == 8]) {
    cudaFuncSetAttribute(radix_scatter_kernel<K>, cudaFuncAttributeMaxDynamicSharedMemorySize, kTile * 8);
    attr_set[sizeof(K) == 8] = true;
  }
  for (int q = 0; q < plan.passes; ++q) {
    const bool to_out = ((plan.passes - 1 - q) % 2) == 0;
    const K* ki = q == 0 ? kin : (to_out ? ktmp : kout);
    K* ko = to_out ? kout : ktmp;
    ColSet cs = cols_in;
    for (int c = 0; c < cols_in.n; ++c) {
      const void* prev_dst = to_out ? tmp.dst[c] : cols_in.dst[c];  // where the previous pass wrote
      cs.src[c] = q == 0 ? cols_in.src[c] : prev_dst;
      cs.dst[c] = to_out ? cols_in.dst[c] : tmp.dst[c];
    }
    uint32_t gm = q == 0 ? gen_mask : 0u;
    LaunchScope ls(ctx, KK_RADIX_SCATTER);
    radix_scatter_kernel<K><<<(unsigned)tiles, kScatterThreads, dyn, s>>>(
        ki, ko, cs, gm, n, plan.shift[q], plan.width[q], transform, hist + q * kRadixMax,
        status + status_words * q, counters + q, ctx.d_status);
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
