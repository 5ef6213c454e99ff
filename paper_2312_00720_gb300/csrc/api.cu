// C ABI entry points of libgj: argument validation, scratch allocation,
// per-device status word, and dispatch to the operator pipelines.
#include <cuda_runtime.h>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <map>
#include <mutex>
#include <utility>

#include "gj_internal.cuh"

namespace gj {

namespace {

struct Allocator {
  void* (*alloc)(size_t, void*, void*) = nullptr;
  void (*free_fn)(void*, void*, void*) = nullptr;
  void* ctx = nullptr;
};
Allocator g_alloc;

constexpr int kMaxDevices = 64;
int* g_status_word[kMaxDevices] = {nullptr};
int g_num_sms[kMaxDevices] = {0};
int g_smem_optin[kMaxDevices] = {0};
bool g_pool_configured[kMaxDevices] = {false};
std::mutex g_mu;

bool valid_dtype(int t) { return t == GJ_I32 || t == GJ_I64; }

gj_status check_table(const gj_table* t, bool need_key) {
  if (!t) return GJ_ERR_INVALID_ARG;
  if (!valid_dtype(t->key_type) || t->ncols < 0 || t->ncols > GJ_MAX_COLS || t->n < 0) return GJ_ERR_INVALID_ARG;
  if (t->n > kMaxRows) return GJ_ERR_UNSUPPORTED;
  if (t->n > 0 && need_key && !t->key) return GJ_ERR_INVALID_ARG;
  for (int c = 0; c < t->ncols; ++c) {
    if (!valid_dtype(t->col_type[c])) return GJ_ERR_INVALID_ARG;
    if (t->n > 0 && !t->cols[c]) return GJ_ERR_INVALID_ARG;
  }
  return GJ_OK;
}

std::atomic<int64_t> g_launches{0};
std::atomic<int> g_timing{0};
struct TimedLaunch {
  int kind;
  cudaEvent_t a, b;
};
std::vector<TimedLaunch> g_timed;
std::vector<cudaEvent_t> g_event_pool;
std::mutex g_prof_mu;

cudaEvent_t take_event() {
  if (!g_event_pool.empty()) {
    cudaEvent_t e = g_event_pool.back();
    g_event_pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  cudaEventCreate(&e);
  return e;
}

const char* const kKindNames[KK_COUNT] = {
    "radix_hist", "radix_scatter", "partition_bounds", "phj_probe", "nphj_build", "nphj_probe",
    "hgb_group_id", "hgb_aggregate", "pgb", "sgb_reduce", "agg_init", "fused_probe", "group_emit",
    "batch", "mlp", "smj_merge", "gather"};

}  // namespace

LaunchScope::LaunchScope(const Ctx& ctx, int kind) : stream_(ctx.stream), kind_(kind) {
  g_launches.fetch_add(1, std::memory_order_relaxed);
  if (g_timing.load(std::memory_order_relaxed)) {
    std::lock_guard<std::mutex> lock(g_prof_mu);
    start_ = take_event();
    cudaEventRecord(start_, stream_);
  }
}

LaunchScope::~LaunchScope() {
  if (!start_) return;
  std::lock_guard<std::mutex> lock(g_prof_mu);
  cudaEvent_t end = take_event();
  cudaEventRecord(end, stream_);
  g_timed.push_back({kind_, start_, end});
}

gj_status cuda_check(cudaError_t e) { return e == cudaSuccess ? GJ_OK : GJ_ERR_CUDA; }

Scratch::~Scratch() {
  for (void* p : ptrs_) {
    if (g_alloc.free_fn)
      g_alloc.free_fn(p, (void*)stream_, g_alloc.ctx);
    else
      cudaFreeAsync(p, stream_);
  }
}

void* Scratch::get(size_t bytes) {
  if (failed_) return nullptr;
  bytes = (bytes + 255) & ~size_t(255);
  if (bytes == 0) bytes = 256;
  void* p = nullptr;
  if (g_alloc.alloc) {
    p = g_alloc.alloc(bytes, (void*)stream_, g_alloc.ctx);
  } else if (cudaMallocAsync(&p, bytes, stream_) != cudaSuccess) {
    cudaGetLastError();
    p = nullptr;
  }
  if (!p) {
    failed_ = true;
    return nullptr;
  }
  ptrs_.push_back(p);
  return p;
}

gj_status make_ctx(void* stream, Ctx* ctx) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return GJ_ERR_CUDA;
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_status_word[dev]) {
    // status word at [0], the wait limit (ns, 0 = default) at bytes 8..15
    int* p = nullptr;
    if (cudaMalloc(&p, sizeof(int) * kStatusInts) != cudaSuccess) return GJ_ERR_OOM;
    if (cudaMemset(p, 0, sizeof(int) * kStatusInts) != cudaSuccess) return GJ_ERR_CUDA;
    g_status_word[dev] = p;
    cudaDeviceGetAttribute(&g_num_sms[dev], cudaDevAttrMultiProcessorCount, dev);
    cudaDeviceGetAttribute(&g_smem_optin[dev], cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  }
  if (!g_pool_configured[dev]) {
    // keep freed scratch in the stream-ordered pool instead of returning it to
    // the CUDA driver after every call
    cudaMemPool_t pool;
    if (cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
      uint64_t thr = UINT64_MAX;
      cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
    }
    cudaGetLastError();
    g_pool_configured[dev] = true;
  }
  ctx->stream = (cudaStream_t)stream;
  ctx->d_status = g_status_word[dev];
  ctx->num_sms = g_num_sms[dev];
  ctx->smem_optin = g_smem_optin[dev];
  ctx->device = dev;
  return GJ_OK;
}

namespace {
std::mutex g_attr_mu;
std::map<std::pair<const void*, int>, int> g_attr_bytes;  // (kernel, device) -> limit set
}  // namespace

gj_status ensure_smem_attr(const Ctx& ctx, const void* func, int bytes) {
  std::lock_guard<std::mutex> lock(g_attr_mu);
  auto key = std::make_pair(func, ctx.device);
  auto it = g_attr_bytes.find(key);
  if (it != g_attr_bytes.end() && it->second >= bytes) return GJ_OK;
  if (cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes) != cudaSuccess) {
    cudaGetLastError();
    return GJ_ERR_CUDA;
  }
  g_attr_bytes[key] = bytes;
  return GJ_OK;
}

// Waits that nothing ever releases, one kind per launch, for gj_check_bounded_wait:
// 0 the warp-wide look-back over a predecessor that never publishes, 1 an mbarrier
// that nothing arrives at, 2 a task counter that never reaches its target.
__global__ void wait_check_kernel(int kind, uint64_t* words, int* status) {
  __shared__ __align__(8) uint64_t s_bar;
  if (kind == 0) {
    if (threadIdx.x < 32) lookback_scan_warp(words, 1, 1, status);  // tile 0 never publishes
  } else if (kind == 1) {
    if (threadIdx.x == 0) {
      mbar_init(&s_bar, 1);
      mbar_fence_init();
    }
    __syncthreads();
    if (threadIdx.x == 0) mbar_wait(&s_bar, 0, status);  // no arrival, no copy in flight
  } else {
    block_wait((const unsigned long long*)words + 1, 1ull, status);  // word 1 stays 0
  }
}

// out[i] = in[map[i]] (the gather primitive): map read and out written in order,
// in read wherever map points. An index outside [0, n_in) records
// GJ_ERR_INVALID_ARG and leaves out[i] as it was.
template <typename T>
__global__ void __launch_bounds__(256) gather_kernel(const T* __restrict__ in, int64_t n_in,
                                                     const int32_t* __restrict__ map, int64_t n, T* __restrict__ out,
                                                     int* status) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  constexpr int kBatch = 4;  // loads of the batch in flight together
  for (int64_t i0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i0 < n; i0 += stride * kBatch) {
    int32_t m[kBatch];
    T v[kBatch];
#pragma unroll
    for (int u = 0; u < kBatch; ++u) m[u] = i0 + u * stride < n ? __ldcs(map + i0 + u * stride) : 0;
#pragma unroll
    for (int u = 0; u < kBatch; ++u) {
      const bool ok = i0 + u * stride < n && m[u] >= 0 && m[u] < n_in;
      v[u] = ok ? in[m[u]] : T(0);
    }
#pragma unroll
    for (int u = 0; u < kBatch; ++u) {
      const int64_t i = i0 + u * stride;
      if (i >= n) continue;
      if (m[u] < 0 || m[u] >= n_in) {
        set_status(status, GJ_ERR_INVALID_ARG);
        continue;
      }
      __stcs(out + i, v[u]);
    }
  }
}

gj_status read_and_clear_status(const Ctx& ctx) {
  int h = 0;
  if (cudaStreamSynchronize(ctx.stream) != cudaSuccess) return GJ_ERR_CUDA;
  if (cudaMemcpy(&h, ctx.d_status, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) return GJ_ERR_CUDA;
  if (h != 0 && cudaMemset(ctx.d_status, 0, sizeof(int)) != cudaSuccess) return GJ_ERR_CUDA;
  return (gj_status)h;
}

gj_status finish(const Ctx& ctx, const gj_options* opt, gj_status st) {
  if (st != GJ_OK) return st;
  if (opt && opt->sync) return read_and_clear_status(ctx);
  return GJ_OK;
}

}  // namespace gj

using namespace gj;

extern "C" {

void gj_options_default(gj_options* opt) {
  if (!opt) return;
  memset(opt, 0, sizeof(*opt));
  opt->join_variant = GJ_JOIN_AUTO;
  opt->groupby_variant = GJ_GB_AUTO;
  opt->selector = GJ_SELECT_COST;
  opt->zipf_hint = -1.0f;
  opt->match_ratio_hint = -1.0f;
}

const char* gj_status_string(gj_status s) {
  switch (s) {
    case GJ_OK: return "GJ_OK";
    case GJ_ERR_INVALID_ARG: return "GJ_ERR_INVALID_ARG";
    case GJ_ERR_UNSUPPORTED: return "GJ_ERR_UNSUPPORTED";
    case GJ_ERR_OOM: return "GJ_ERR_OOM";
    case GJ_ERR_CAPACITY: return "GJ_ERR_CAPACITY";
    case GJ_ERR_DUPLICATE_KEY: return "GJ_ERR_DUPLICATE_KEY";
    case GJ_ERR_TIMEOUT: return "GJ_ERR_TIMEOUT";
    case GJ_ERR_CUDA: return "GJ_ERR_CUDA";
  }
  return "GJ_UNKNOWN_STATUS";
}

gj_status gj_set_allocator(void* (*alloc)(size_t, void*, void*), void (*free_fn)(void*, void*, void*), void* ctx) {
  if ((alloc == nullptr) != (free_fn == nullptr)) return GJ_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lock(g_mu);
  g_alloc.alloc = alloc;
  g_alloc.free_fn = free_fn;
  g_alloc.ctx = ctx;
  return GJ_OK;
}

gj_status gj_get_device_status(void* stream) {
  Ctx ctx;
  gj_status st = make_ctx(stream, &ctx);
  if (st != GJ_OK) return st;
  return read_and_clear_status(ctx);
}

gj_status gj_radix_partition(const gj_table* in, int32_t bit_lo, int32_t bit_hi, int32_t key_transform,
                             gj_table* out, int64_t* d_offsets, const gj_options* opt, void* stream) {
  gj_status st;
  if ((st = check_table(in, true)) != GJ_OK) return st;
  if ((st = check_table(out, true)) != GJ_OK) return st;
  if (out->key_type != in->key_type || out->ncols != in->ncols || out->n < in->n) return GJ_ERR_INVALID_ARG;
  for (int c = 0; c < in->ncols; ++c)
    if (out->col_type[c] != in->col_type[c]) return GJ_ERR_INVALID_ARG;
  const int kbits = in->key_type == GJ_I64 ? 64 : 32;
  if (bit_lo < 0 || bit_hi <= bit_lo || bit_hi > kbits) return GJ_ERR_INVALID_ARG;
  if (key_transform < 0 || key_transform > 2) return GJ_ERR_INVALID_ARG;
  if (d_offsets && bit_hi - bit_lo > 24) return GJ_ERR_INVALID_ARG;
  gj_options defaults;
  gj_options_default(&defaults);
  if (!opt) opt = &defaults;
  if (opt->bits_per_pass < 0 || opt->bits_per_pass > 8) return GJ_ERR_INVALID_ARG;
  Ctx ctx;
  if ((st = make_ctx(stream, &ctx)) != GJ_OK) return st;
  ColSet cs{};
  cs.n = in->ncols;
  for (int c = 0; c < in->ncols; ++c) {
    cs.src[c] = in->cols[c];
    cs.dst[c] = out->cols[c];
    cs.size[c] = dtype_size(in->col_type[c]);
  }
  {
    Scratch scr(ctx.stream);
    st = radix_partition_run(ctx, scr, in->key_type, in->key, out->key, cs, in->n, bit_lo, bit_hi, key_transform,
                             opt->bits_per_pass);
    if (st == GJ_OK && d_offsets)
      st = partition_bounds_run(ctx, in->key_type, out->key, in->n, bit_lo, bit_hi - bit_lo, key_transform,
                                d_offsets);
  }
  return finish(ctx, opt, st);
}

gj_status gj_join(const gj_table* R, const gj_table* S, const gj_options* opt, gj_table* T, int64_t T_capacity,
                  int64_t* d_T_count, void* stream) {
  gj_status st;
  if ((st = check_table(R, true)) != GJ_OK) return st;
  if ((st = check_table(S, true)) != GJ_OK) return st;
  if (!T || !d_T_count || T_capacity < 0) return GJ_ERR_INVALID_ARG;
  if (R->key_type != S->key_type || T->key_type != R->key_type) return GJ_ERR_INVALID_ARG;
  if (T->ncols != R->ncols + S->ncols || T->ncols > GJ_MAX_COLS) return GJ_ERR_INVALID_ARG;
  for (int c = 0; c < R->ncols; ++c)
    if (T->col_type[c] != R->col_type[c]) return GJ_ERR_INVALID_ARG;
  for (int c = 0; c < S->ncols; ++c)
    if (T->col_type[R->ncols + c] != S->col_type[c]) return GJ_ERR_INVALID_ARG;
  if (T_capacity > 0) {
    if (!T->key) return GJ_ERR_INVALID_ARG;
    for (int c = 0; c < T->ncols; ++c)
      if (!T->cols[c]) return GJ_ERR_INVALID_ARG;
  }
  gj_options defaults;
  gj_options_default(&defaults);
  if (!opt) opt = &defaults;
  if (opt->join_variant < GJ_JOIN_AUTO || opt->join_variant > GJ_JOIN_PHJ_MN) return GJ_ERR_INVALID_ARG;
  if (opt->radix_bits < 0 || opt->radix_bits > 16 || opt->bits_per_pass < 0 || opt->bits_per_pass > 8)
    return GJ_ERR_INVALID_ARG;
  Ctx ctx;
  if ((st = make_ctx(stream, &ctx)) != GJ_OK) return st;
  st = join_run(ctx, R, S, opt, T, T_capacity, d_T_count);
  return finish(ctx, opt, st);
}

gj_status gj_groupby(const gj_table* in, int32_t nagg, const int32_t* ops, const int32_t* op_col,
                     const gj_options* opt, void* out_keys, int64_t* const* out_aggs, int64_t capacity,
                     int64_t* d_ngroups, void* stream) {
  gj_status st;
  if ((st = check_table(in, true)) != GJ_OK) return st;
  if (nagg < 1 || nagg > GJ_MAX_AGGS || !ops || !op_col || !out_aggs || !d_ngroups || capacity < 0)
    return GJ_ERR_INVALID_ARG;
  for (int j = 0; j < nagg; ++j) {
    if (ops[j] < GJ_AGG_SUM || ops[j] > GJ_AGG_MAX) return GJ_ERR_INVALID_ARG;
    if (ops[j] != GJ_AGG_COUNT && (op_col[j] < 0 || op_col[j] >= in->ncols)) return GJ_ERR_INVALID_ARG;
    if (capacity > 0 && !out_aggs[j]) return GJ_ERR_INVALID_ARG;
  }
  if (capacity > 0 && !out_keys) return GJ_ERR_INVALID_ARG;
  gj_options defaults;
  gj_options_default(&defaults);
  if (!opt) opt = &defaults;
  if (opt->groupby_variant < GJ_GB_AUTO || opt->groupby_variant > GJ_GB_SGB_DE) return GJ_ERR_INVALID_ARG;
  if (opt->radix_bits < 0 || opt->radix_bits > 24 || opt->bits_per_pass < 0 || opt->bits_per_pass > 8)
    return GJ_ERR_INVALID_ARG;
  Ctx ctx;
  if ((st = make_ctx(stream, &ctx)) != GJ_OK) return st;
  st = groupby_run(ctx, in, nagg, ops, op_col, opt, out_keys, out_aggs, capacity, d_ngroups);
  return finish(ctx, opt, st);
}

gj_status gj_join_groupby(const gj_table* R, const gj_table* S, gj_colref group_key, int32_t nagg,
                          const int32_t* ops, const gj_colref* agg_cols, const gj_options* opt, int64_t* out_keys,
                          int64_t* const* out_aggs, int64_t capacity, int64_t* d_ngroups, void* stream) {
  gj_status st;
  if ((st = check_table(R, true)) != GJ_OK) return st;
  if ((st = check_table(S, true)) != GJ_OK) return st;
  if (R->key_type != S->key_type) return GJ_ERR_INVALID_ARG;
  auto ref_ok = [&](const gj_colref& r) {
    if (r.side != 0 && r.side != 1) return false;
    const gj_table* t = r.side == 0 ? R : S;
    return r.col >= -1 && r.col < t->ncols && r.modulus >= 0;
  };
  if (!ref_ok(group_key)) return GJ_ERR_INVALID_ARG;
  if (nagg < 1 || nagg > GJ_MAX_AGGS || !ops || !agg_cols || !out_aggs || !d_ngroups || capacity < 0)
    return GJ_ERR_INVALID_ARG;
  for (int j = 0; j < nagg; ++j) {
    if (ops[j] < GJ_AGG_SUM || ops[j] > GJ_AGG_MAX) return GJ_ERR_INVALID_ARG;
    if (ops[j] != GJ_AGG_COUNT && !ref_ok(agg_cols[j])) return GJ_ERR_INVALID_ARG;
    if (capacity > 0 && !out_aggs[j]) return GJ_ERR_INVALID_ARG;
  }
  if (capacity > 0 && !out_keys) return GJ_ERR_INVALID_ARG;
  gj_options defaults;
  gj_options_default(&defaults);
  if (!opt) opt = &defaults;
  if (opt->join_variant < GJ_JOIN_AUTO || opt->join_variant > GJ_JOIN_NPHJ) return GJ_ERR_INVALID_ARG;
  if (opt->radix_bits < 0 || opt->radix_bits > 16 || opt->bits_per_pass < 0 || opt->bits_per_pass > 8)
    return GJ_ERR_INVALID_ARG;
  Ctx ctx;
  if ((st = make_ctx(stream, &ctx)) != GJ_OK) return st;
  st = join_groupby_run(ctx, R, S, group_key, nagg, ops, agg_cols, opt, out_keys, out_aggs, capacity, d_ngroups);
  return finish(ctx, opt, st);
}

gj_status gj_heuristic_choose(const gj_table* R, const gj_table* S, int32_t nagg, const gj_options* opt,
                              int32_t* join_variant, int32_t* gb_variant) {
  gj_options defaults;
  gj_options_default(&defaults);
  if (!opt) opt = &defaults;
  if (join_variant) {
    if (!R) return GJ_ERR_INVALID_ARG;
    *join_variant = heuristic_join_variant(R, opt);
  }
  if (gb_variant) {
    if (!S || nagg < 1) return GJ_ERR_INVALID_ARG;
    int dev = 0, smem = 200 * 1024;
    if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    cudaGetLastError();
    *gb_variant = choose_groupby_variant(S, nagg, nullptr, opt, std::min(smem, 200 * 1024));
  }
  return GJ_OK;
}

gj_status gj_auto_variants(const gj_table* R, const gj_table* S, int32_t nagg, const int32_t* ops,
                           const gj_options* opt, int32_t fused, int32_t* join_variant, int32_t* gb_variant) {
  gj_options defaults;
  gj_options_default(&defaults);
  if (!opt) opt = &defaults;
  if (join_variant) {
    if (!R || !S) return GJ_ERR_INVALID_ARG;
    *join_variant = resolve_join_variant(R, S, fused ? nagg : 0, opt, fused != 0);
  }
  if (gb_variant) {
    if (!S || nagg < 1) return GJ_ERR_INVALID_ARG;
    int dev = 0, smem = 200 * 1024;
    if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    cudaGetLastError();
    *gb_variant = resolve_groupby_variant(S, nagg, ops, opt, std::min(smem, 200 * 1024) - 1024);
  }
  return GJ_OK;
}

gj_status gj_gather(const void* in, int64_t n_in, int32_t elem_bytes, const int32_t* map, int64_t n, void* out,
                    const gj_options* opt, void* stream) {
  if (n < 0 || n_in < 0 || (elem_bytes != 4 && elem_bytes != 8)) return GJ_ERR_INVALID_ARG;
  if (n > 0 && (!in || !map || !out)) return GJ_ERR_INVALID_ARG;
  if (n > kMaxRows || n_in > kMaxRows) return GJ_ERR_UNSUPPORTED;
  Ctx ctx;
  gj_status st = make_ctx(stream, &ctx);
  if (st != GJ_OK) return st;
  if (n > 0) {
    LaunchScope ls(ctx, KK_GATHER);
    const int blocks = (int)std::max<int64_t>(1, std::min<int64_t>((n + 1023) / 1024, (int64_t)ctx.num_sms * 8));
    if (elem_bytes == 4)
      gather_kernel<int32_t><<<blocks, 256, 0, ctx.stream>>>((const int32_t*)in, n_in, map, n, (int32_t*)out,
                                                             ctx.d_status);
    else
      gather_kernel<int64_t><<<blocks, 256, 0, ctx.stream>>>((const int64_t*)in, n_in, map, n, (int64_t*)out,
                                                             ctx.d_status);
    st = cuda_check(cudaGetLastError());
  }
  return finish(ctx, opt, st);
}

gj_status gj_set_wait_limit(uint64_t ns) {
  Ctx ctx;
  gj_status st = make_ctx(nullptr, &ctx);
  if (st != GJ_OK) return st;
  return cuda_check(cudaMemcpy(ctx.d_status + 2, &ns, sizeof(ns), cudaMemcpyHostToDevice));
}

gj_status gj_check_bounded_wait(int32_t kind, void* stream) {
  if (kind < 0 || kind > 2) return GJ_ERR_INVALID_ARG;
  Ctx ctx;
  gj_status st = make_ctx(stream, &ctx);
  if (st != GJ_OK) return st;
  {
    Scratch scr(ctx.stream);
    uint64_t* words = scr.get_as<uint64_t>(2);
    if (scr.failed()) return GJ_ERR_OOM;
    if ((st = cuda_check(cudaMemsetAsync(words, 0, 2 * sizeof(uint64_t), ctx.stream))) != GJ_OK) return st;
    wait_check_kernel<<<1, 64, 0, ctx.stream>>>(kind, words, ctx.d_status);
    if ((st = cuda_check(cudaGetLastError())) != GJ_OK) return st;
  }
  return read_and_clear_status(ctx);
}

void gj_profile_enable(int32_t on) { g_timing.store(on ? 1 : 0); }

int32_t gj_profile_read(double* ms, int64_t* launches, int32_t max_kinds) {
  cudaDeviceSynchronize();
  std::lock_guard<std::mutex> lock(g_prof_mu);
  for (int k = 0; k < max_kinds && k < KK_COUNT; ++k) {
    if (ms) ms[k] = 0.0;
    if (launches) launches[k] = 0;
  }
  for (auto& t : g_timed) {
    float e = 0.f;
    cudaEventElapsedTime(&e, t.a, t.b);
    if (t.kind < max_kinds) {
      if (ms) ms[t.kind] += e;
      if (launches) launches[t.kind] += 1;
    }
    g_event_pool.push_back(t.a);
    g_event_pool.push_back(t.b);
  }
  g_timed.clear();
  return KK_COUNT;
}

const char* gj_kernel_name(int32_t kind) { return kind >= 0 && kind < KK_COUNT ? kKindNames[kind] : "unknown"; }

int64_t gj_kernel_launches(void) { return g_launches.load(); }

}  // extern "C"
