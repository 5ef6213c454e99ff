// Batched join -> group-by: many queries in one persistent launch.
//
// The queue holds, per query q, tasks of four kinds:
//   ZERO  clear a chunk of q's build table and group slots,
//   BUILD insert a tile of R_q into q's global open-addressing table (key -> row),
//   PROBE look a tile of S_q up in the table and aggregate every match into q's
//         dense group slots (the group key is a residue, slot = key + m - 1),
//         pre-aggregating in shared memory when q's slots fit,
//   EMIT  compact a tile of q's occupied slots into the output (look-back over
//         q's emit tiles gives dense positions; the last tile writes g).
// BUILD waits for all of q's ZERO tasks, PROBE for all BUILD tasks, EMIT for all
// PROBE tasks. The queue puts the ZERO and BUILD tasks of query q + L (the
// lookahead) before the PROBE tasks of q and every EMIT after its PROBEs, so a
// task's dependencies always sit earlier in the queue: they were taken by CTAs
// that are running and never wait on later tasks, hence every wait ends
// (each is bounded anyway). Each query computes what gj_join_groupby computes
// with the non-partitioned table; the batch only removes per-query launches
// and host round trips, and keeps a small query's table in L2 while it runs.
// The paper has no batched mode: this is a scheduling layer over the group-by
// that follows a join (Sec. 1) with the non-partitioned hash join of Sec. 3.1.3.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <map>
#include <mutex>
#include <tuple>
#include <vector>

#include "gj_internal.cuh"

struct gj_batch_plan;

namespace gj {

namespace {

constexpr int kBThreads = 256;
constexpr int kBMaxAggs = GJ_BATCH_MAX_AGGS;
constexpr int kEmitTile = 2048;
constexpr int64_t kZeroChunk = 1 << 16;
constexpr int kSmemAgg = 64 * 1024;

enum TaskKind { TK_ZERO = 0, TK_BUILD = 1, TK_PROBE = 2, TK_EMIT = 3 };

// Shared-memory slots of a probe task. 64-bit shared-memory atomics are
// compare-and-swap loops that collapse when many lanes hit one slot (a handful
// of groups), so values that fit 32 bits use 32-bit slots: COUNT, MIN/MAX, and
// SUM split over two words (the value's low 16 bits unsigned, its high 16 bits
// signed), exact while a task has at most 65535 rows; merged into the int64
// results at the end of the task.
enum SlotKind { SK_COUNT32 = 0, SK_MINMAX32 = 1, SK_SPLIT = 2, SK_64 = 3 };

struct BRef {
  int32_t is_key;
  int32_t side;
  int32_t size;
  int32_t pad;
  int64_t mod;
  const void* src;
};

struct BInst {
  const int32_t* rkey;
  const int32_t* skey;
  int64_t nr, ns;
  int32_t* ht;
  uint64_t ht_slots;  // power of two
  unsigned long long* cnt;
  int64_t* agg[kBMaxAggs];
  int64_t nslots, dense_off;
  int32_t nagg, smem;  // smem: the probe aggregates into shared memory (layout below)
  int32_t op[kBMaxAggs];
  // shared-memory slot form of aggregate j (SlotKind) and its byte offset; the
  // 32-bit row counts of the slots come first
  int32_t sform[kBMaxAggs];
  int32_t soff[kBMaxAggs];
  int32_t fits32;  // bit j: aggregate j's values fit 32 bits
  int32_t prows;   // rows per probe task
  BRef gk;
  BRef val[kBMaxAggs];
  int64_t* out_keys;
  int64_t* out_aggs[kBMaxAggs];
  int64_t cap;
  int64_t* d_ngroups;
  int32_t nzero, nbuild, nprobe, nemit;
  int64_t ctl;  // control words: zero_done, build_done, probe_done, -, emit look-back words
};

struct BTask {
  int32_t inst;
  int32_t kind;
  int64_t begin, end;
  int32_t idx;
  int32_t pad;
};

__device__ __forceinline__ int64_t bref_value(const BRef& f, int64_t m, int64_t i, int32_t key) {
  int64_t v;
  if (f.is_key)
    v = key;
  else
    v = load_as_i64(f.src, f.size, f.side == 0 ? m : i);
  return f.mod > 0 ? v % f.mod : v;
}

__global__ void __launch_bounds__(kBThreads) batch_kernel(const BInst* __restrict__ insts,
                                                          const BTask* __restrict__ tasks, int ntasks,
                                                          unsigned long long* ctl, int* err) {
  extern __shared__ __align__(16) unsigned char s_dyn[];
  __shared__ int s_t;
  __shared__ uint32_t s_scan[kBThreads / 32];
  __shared__ uint64_t s_base;
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  for (;;) {
    if (t == 0) s_t = (int)atomicAdd(&ctl[0], 1ull);
    __syncthreads();
    const int ti = s_t;
    __syncthreads();
    if (ti >= ntasks) break;
    const BTask T = tasks[ti];
    const BInst& I = insts[T.inst];
    unsigned long long* c = ctl + I.ctl;

    if (T.kind == TK_ZERO) {
      for (int64_t x = T.begin + t; x < T.end; x += kBThreads) {
        if ((uint64_t)x < I.ht_slots) {
          I.ht[x] = 0;
        } else {
          const int64_t s = x - (int64_t)I.ht_slots;
          I.cnt[s] = 0;
          for (int j = 0; j < I.nagg; ++j) I.agg[j][s] = agg_identity(I.op[j]);
        }
      }
      block_done(&c[0]);
    } else if (T.kind == TK_BUILD) {
      block_wait(&c[0], (unsigned long long)I.nzero, err);
      const uint64_t mask = I.ht_slots - 1;
      for (int64_t i = T.begin + t; i < T.end; i += kBThreads) {
        const int32_t k = I.rkey[i];
        uint64_t sl = fmix32((uint32_t)k) & mask;
        for (uint64_t probe = 0; probe <= mask; ++probe) {
          const int prev = atomicCAS(&I.ht[sl], 0, (int)(i + 1));
          if (prev == 0) break;
          if (I.rkey[prev - 1] == k) {
            set_status(err, GJ_ERR_DUPLICATE_KEY);
            break;
          }
          sl = (sl + 1) & mask;
        }
      }
      block_done(&c[1]);
    } else if (T.kind == TK_PROBE) {
      block_wait(&c[1], (unsigned long long)I.nbuild, err);
      uint32_t* s_cnt = (uint32_t*)s_dyn;
      if (I.smem) {
        for (int64_t s = t; s < I.nslots; s += kBThreads) {
          s_cnt[s] = 0u;
          for (int j = 0; j < I.nagg; ++j) {
            unsigned char* base = s_dyn + I.soff[j];
            switch (I.sform[j]) {
              case SK_COUNT32: ((uint32_t*)base)[s] = 0u; break;
              case SK_MINMAX32: ((int32_t*)base)[s] = I.op[j] == GJ_AGG_MIN ? INT32_MAX : INT32_MIN; break;
              case SK_SPLIT: ((int64_t*)base)[s] = 0; break;
              default: ((int64_t*)base)[s] = agg_identity(I.op[j]); break;
            }
          }
        }
        __syncthreads();
      }
      const uint64_t mask = I.ht_slots - 1;
      for (int64_t i = T.begin + t; i < T.end; i += kBThreads) {
        const int32_t k = __ldcs(I.skey + i);
        uint64_t sl = fmix32((uint32_t)k) & mask;
        int v = __ldcg(I.ht + sl);
        int64_t m = -1;
        for (uint64_t probe = 0; probe <= mask && v != 0; ++probe) {
          if (__ldg(I.rkey + v - 1) == k) {
            m = v - 1;
            break;
          }
          sl = (sl + 1) & mask;
          v = __ldcg(I.ht + sl);
        }
        if (m < 0) continue;
        const int64_t slot = bref_value(I.gk, m, i, k) + I.dense_off;
        if (I.smem) {
          atomicAdd(&s_cnt[slot], 1u);
          for (int j = 0; j < I.nagg; ++j) {
            unsigned char* base = s_dyn + I.soff[j];
            switch (I.sform[j]) {
              case SK_COUNT32: atomicAdd((uint32_t*)base + slot, 1u); break;
              case SK_MINMAX32: {
                const int32_t v = (int32_t)bref_value(I.val[j], m, i, k);
                if (I.op[j] == GJ_AGG_MIN) atomicMin((int32_t*)base + slot, v); else atomicMax((int32_t*)base + slot, v);
                break;
              }
              case SK_SPLIT: {
                const int32_t v = (int32_t)bref_value(I.val[j], m, i, k);
                atomicAdd((uint32_t*)base + 2 * slot, (uint32_t)v & 0xffffu);
                atomicAdd((int32_t*)base + 2 * slot + 1, v >> 16);
                break;
              }
              default:
                agg_atomic(I.op[j], (int64_t*)base + slot, I.op[j] == GJ_AGG_COUNT ? 1 : bref_value(I.val[j], m, i, k));
            }
          }
        } else {
          atomicAdd(&I.cnt[slot], 1ull);
          for (int j = 0; j < I.nagg; ++j)
            agg_atomic(I.op[j], &I.agg[j][slot], I.op[j] == GJ_AGG_COUNT ? 1 : bref_value(I.val[j], m, i, k));
        }
      }
      if (I.smem) {
        __syncthreads();
        for (int64_t s = t; s < I.nslots; s += kBThreads) {
          if (s_cnt[s] == 0u) continue;
          atomicAdd(&I.cnt[s], (unsigned long long)s_cnt[s]);
          for (int j = 0; j < I.nagg; ++j) {
            const unsigned char* base = s_dyn + I.soff[j];
            int64_t v;
            switch (I.sform[j]) {
              case SK_COUNT32: v = (int64_t)((const uint32_t*)base)[s]; break;
              case SK_MINMAX32: v = (int64_t)((const int32_t*)base)[s]; break;
              case SK_SPLIT:
                v = (int64_t)((const int32_t*)base)[2 * s + 1] * 65536 + (int64_t)((const uint32_t*)base)[2 * s];
                break;
              default: v = ((const int64_t*)base)[s]; break;
            }
            agg_atomic(I.op[j], &I.agg[j][s], v);
          }
        }
      }
      block_done(&c[2]);
    } else {  // TK_EMIT: slots [begin, end) are one tile of 8 slots per thread
      block_wait(&c[2], (unsigned long long)I.nprobe, err);
      const int64_t sb = T.begin + (int64_t)t * (kEmitTile / kBThreads);
      constexpr int kPer = kEmitTile / kBThreads;
      uint32_t cnt = 0;
      for (int r = 0; r < kPer; ++r) cnt += (sb + r < T.end && __ldcg(&I.cnt[sb + r]) > 0) ? 1u : 0u;
      uint32_t x = cnt;
      for (int o = 1; o < 32; o <<= 1) {
        uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
      }
      if (lane == 31) s_scan[warp] = x;
      __syncthreads();
      if (warp == 0) {
        uint32_t run = 0;
        for (int w = 0; w < kBThreads / 32; ++w) run += s_scan[w];
        __syncwarp();
        if (lane == 0) {
          uint32_t r = 0;
          for (int w = 0; w < kBThreads / 32; ++w) {
            const uint32_t cc = s_scan[w];
            s_scan[w] = r;
            r += cc;
          }
        }
        const uint64_t excl = lookback_scan_warp((uint64_t*)(c + 4), T.idx, run, err);
        if (lane == 0) {
          s_base = excl;
          if (T.idx == I.nemit - 1) *I.d_ngroups = (int64_t)(excl + run);
        }
      }
      __syncthreads();
      int64_t o = (int64_t)s_base + s_scan[warp] + x - cnt;
      bool overflow = false;
      for (int r = 0; r < kPer; ++r) {
        const int64_t s = sb + r;
        if (s >= T.end || __ldcg(&I.cnt[s]) == 0) continue;
        if (o < I.cap) {
          I.out_keys[o] = s - I.dense_off;
          for (int j = 0; j < I.nagg; ++j) I.out_aggs[j][o] = __ldcg(&I.agg[j][s]);
        } else {
          overflow = true;
        }
        ++o;
      }
      if (overflow) set_status(err, GJ_ERR_CAPACITY);
      __syncthreads();
    }
  }
}

int64_t ceil_div(int64_t a, int64_t b) { return (a + b - 1) / b; }

}  // namespace

}  // namespace gj

using namespace gj;

struct gj_batch_plan {
  int device = 0;
  int num_sms = 0;
  int nq = 0;
  std::vector<BInst> h_insts;
  BInst* d_insts = nullptr;
  BTask* d_tasks = nullptr;
  int ntasks = 0;
  unsigned long long* d_ctl = nullptr;
  size_t ctl_words = 0;
  std::vector<void*> allocs;
  gj_batch_config cfg{};
  size_t dyn = 0;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  int* d_status = nullptr;
  // per query of the request: the join variant it runs; queries not run by the
  // persistent kernel go through the one-query path after it, with these options
  int nq_total = 0;
  std::vector<int32_t> variant;
  std::vector<int> solo;
  std::vector<gj_query> queries;
  gj_options solo_opt{};
};

namespace gj {
namespace {

std::mutex g_tune_mu;
std::map<std::tuple<int, int, int64_t, int64_t, int64_t>, gj_batch_config> g_tune_cache;

bool valid_ref(const gj_query& q, const gj_colref& r) {
  if (r.side != 0 && r.side != 1) return false;
  const gj_table& t = r.side == 0 ? q.R : q.S;
  return r.col >= -1 && r.col < t.ncols && r.modulus >= 0;
}

// Checks every query must pass; batchable() adds the persistent kernel's limits.
gj_status check_query(const gj_query& q) {
  for (const gj_table* t : {&q.R, &q.S}) {
    if (t->key_type != GJ_I32 && t->key_type != GJ_I64) return GJ_ERR_INVALID_ARG;
    if (t->ncols < 0 || t->ncols > GJ_MAX_COLS || t->n < 0) return GJ_ERR_INVALID_ARG;
    if (t->n > 0 && !t->key) return GJ_ERR_INVALID_ARG;
    for (int c = 0; c < t->ncols; ++c)
      if ((t->col_type[c] != GJ_I32 && t->col_type[c] != GJ_I64) || (t->n > 0 && !t->cols[c]))
        return GJ_ERR_INVALID_ARG;
  }
  if (q.R.key_type != q.S.key_type) return GJ_ERR_INVALID_ARG;
  if (!valid_ref(q, q.group_key)) return GJ_ERR_INVALID_ARG;
  if (q.nagg < 1 || q.nagg > GJ_BATCH_MAX_AGGS) return GJ_ERR_INVALID_ARG;
  for (int j = 0; j < q.nagg; ++j) {
    if (q.ops[j] < GJ_AGG_SUM || q.ops[j] > GJ_AGG_MAX) return GJ_ERR_INVALID_ARG;
    if (q.ops[j] != GJ_AGG_COUNT && !valid_ref(q, q.agg_cols[j])) return GJ_ERR_INVALID_ARG;
    if (q.capacity > 0 && !q.out_aggs[j]) return GJ_ERR_INVALID_ARG;
  }
  if (q.capacity < 0 || !q.d_ngroups || (q.capacity > 0 && !q.out_keys)) return GJ_ERR_INVALID_ARG;
  return GJ_OK;
}

bool batchable(const gj_query& q) {
  return q.R.key_type == GJ_I32 && q.R.n <= kMaxRows && q.S.n <= kMaxRows && q.group_key.modulus >= 1 &&
         q.group_key.modulus <= (1 << 20);
}

BRef make_ref(const gj_query& q, const gj_colref& r) {
  BRef f{};
  f.mod = r.modulus;
  if (r.col < 0) {
    f.is_key = 1;
    return f;
  }
  const gj_table& t = r.side == 0 ? q.R : q.S;
  f.side = r.side;
  f.src = t.cols[r.col];
  f.size = dtype_size(t.col_type[r.col]);
  return f;
}

// Builds the task queue for `cfg` and uploads it; sets the per-instance task
// counts and control offsets.
gj_status build_tasks(gj_batch_plan* P, const gj_batch_config& cfg) {
  std::vector<BTask> tasks;
  size_t ctl = 1;  // word 0: queue head
  for (auto& I : P->h_insts) {
    // rows per probe task (at least four rows per shared-memory slot measured no faster)
    I.prows = cfg.probe_rows;
    // a split SUM slot is exact for at most 65535 rows: longer probe tasks take 64-bit SUMs
    for (int j = 0; j < I.nagg; ++j)
      if (I.op[j] == GJ_AGG_SUM && ((I.fits32 >> j) & 1)) I.sform[j] = I.prows <= 65535 ? SK_SPLIT : SK_64;
    I.nzero = (int32_t)ceil_div((int64_t)I.ht_slots + I.nslots, kZeroChunk);
    I.nbuild = (int32_t)ceil_div(I.nr, cfg.build_rows);
    I.nprobe = (int32_t)ceil_div(I.ns, I.prows);
    I.nemit = (int32_t)ceil_div(I.nslots, kEmitTile);
    I.ctl = (int64_t)ctl;
    ctl += 4 + I.nemit;
  }
  const int nq = P->nq, L = cfg.lookahead;
  auto push_zb = [&](int q) {
    const BInst& I = P->h_insts[q];
    const int64_t total = (int64_t)I.ht_slots + I.nslots;
    for (int z = 0; z < I.nzero; ++z)
      tasks.push_back({q, TK_ZERO, z * kZeroChunk, std::min<int64_t>(total, (z + 1) * kZeroChunk), z, 0});
    for (int b = 0; b < I.nbuild; ++b)
      tasks.push_back({q, TK_BUILD, (int64_t)b * cfg.build_rows,
                       std::min<int64_t>(I.nr, (int64_t)(b + 1) * cfg.build_rows), b, 0});
  };
  auto push_p = [&](int q) {
    const BInst& I = P->h_insts[q];
    for (int p = 0; p < I.nprobe; ++p)
      tasks.push_back({q, TK_PROBE, (int64_t)p * I.prows, std::min<int64_t>(I.ns, (int64_t)(p + 1) * I.prows), p, 0});
  };
  auto push_e = [&](int q) {
    const BInst& I = P->h_insts[q];
    for (int e = 0; e < I.nemit; ++e)
      tasks.push_back({q, TK_EMIT, (int64_t)e * kEmitTile, std::min<int64_t>(I.nslots, (int64_t)(e + 1) * kEmitTile),
                       e, 0});
  };
  for (int s = 0; s < nq + L + 1; ++s) {
    if (s < nq) push_zb(s);
    if (s - L >= 0 && s - L < nq) push_p(s - L);
    if (s - L - 1 >= 0 && s - L - 1 < nq) push_e(s - L - 1);
  }
  if (P->d_tasks) cudaFree(P->d_tasks);
  if (P->d_ctl) cudaFree(P->d_ctl);
  P->d_tasks = nullptr;
  P->d_ctl = nullptr;
  P->ntasks = (int)tasks.size();
  P->ctl_words = ctl;
  if (cudaMalloc(&P->d_tasks, sizeof(BTask) * std::max<size_t>(1, tasks.size())) != cudaSuccess) return GJ_ERR_OOM;
  if (cudaMalloc(&P->d_ctl, sizeof(unsigned long long) * ctl) != cudaSuccess) return GJ_ERR_OOM;
  if (cudaMemcpy(P->d_tasks, tasks.data(), sizeof(BTask) * tasks.size(), cudaMemcpyHostToDevice) != cudaSuccess)
    return GJ_ERR_CUDA;
  if (cudaMemcpy(P->d_insts, P->h_insts.data(), sizeof(BInst) * P->nq, cudaMemcpyHostToDevice) != cudaSuccess)
    return GJ_ERR_CUDA;
  return GJ_OK;
}

gj_status capture(gj_batch_plan* P, const gj_batch_config& cfg) {
  gj_status st = build_tasks(P, cfg);
  if (st != GJ_OK) return st;
  if (P->exec) cudaGraphExecDestroy(P->exec);
  if (P->graph) cudaGraphDestroy(P->graph);
  P->exec = nullptr;
  P->graph = nullptr;
  int per_sm = 1;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, batch_kernel, kBThreads, P->dyn);
  const int bps = std::max(1, std::min(cfg.blocks_per_sm, per_sm));
  const int grid = P->num_sms * bps;
  cudaStream_t cs;
  if (cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) != cudaSuccess) return GJ_ERR_CUDA;
  cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
  cudaMemsetAsync(P->d_ctl, 0, sizeof(unsigned long long) * P->ctl_words, cs);
  batch_kernel<<<grid, kBThreads, P->dyn, cs>>>(P->d_insts, P->d_tasks, P->ntasks, P->d_ctl, P->d_status);
  cudaError_t e = cudaStreamEndCapture(cs, &P->graph);
  cudaStreamDestroy(cs);
  if (e != cudaSuccess) return GJ_ERR_CUDA;
  if (cudaGraphInstantiate(&P->exec, P->graph, 0) != cudaSuccess) return GJ_ERR_CUDA;
  P->cfg = cfg;
  P->cfg.blocks_per_sm = bps;
  return GJ_OK;
}

float time_plan(gj_batch_plan* P, cudaStream_t s, int reps) {
  cudaEvent_t a, b;
  cudaEventCreate(&a);
  cudaEventCreate(&b);
  cudaGraphLaunch(P->exec, s);
  std::vector<float> ts;
  for (int r = 0; r < reps; ++r) {
    cudaEventRecord(a, s);
    cudaGraphLaunch(P->exec, s);
    cudaEventRecord(b, s);
    cudaEventSynchronize(b);
    float ms = 0;
    cudaEventElapsedTime(&ms, a, b);
    ts.push_back(ms);
  }
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  std::sort(ts.begin(), ts.end());
  return ts[ts.size() / 2];
}

}  // namespace
}  // namespace gj

extern "C" {

gj_status gj_batch_create(const gj_query* queries, int32_t nq, const gj_batch_config* cfg_in, const gj_options* opt,
                          gj_batch_plan** out, void* stream) {
  if (!out || nq < 0 || (nq > 0 && !queries)) return GJ_ERR_INVALID_ARG;
  gj_options o;
  gj_options_default(&o);
  if (opt) o = *opt;
  if (o.join_variant != GJ_JOIN_AUTO && o.join_variant != GJ_JOIN_PHJ_TR && o.join_variant != GJ_JOIN_PHJ_UR &&
      o.join_variant != GJ_JOIN_NPHJ)
    return GJ_ERR_INVALID_ARG;
  if (o.radix_bits < 0 || o.radix_bits > 16 || o.bits_per_pass < 0 || o.bits_per_pass > 8) return GJ_ERR_INVALID_ARG;
  for (int q = 0; q < nq; ++q) {
    gj_status st = check_query(queries[q]);
    if (st != GJ_OK) return st;
  }
  gj_batch_config want{};
  if (cfg_in) want = *cfg_in;
  if (want.build_rows < 0 || want.probe_rows < 0 || want.lookahead < 0 || want.blocks_per_sm < 0)
    return GJ_ERR_INVALID_ARG;
  Ctx ctx;
  gj_status st = make_ctx(stream, &ctx);
  if (st != GJ_OK) return st;
  auto* P = new gj_batch_plan();
  P->device = ctx.device;
  P->num_sms = ctx.num_sms;
  P->nq_total = nq;
  P->d_status = ctx.d_status;
  P->queries.assign(queries, queries + nq);
  P->solo_opt = o;
  P->solo_opt.sync = 0;
  auto fail = [&](gj_status e) {
    gj_batch_destroy(P);
    return e;
  };
  int64_t sum_r = 0, sum_s = 0, sum_slots = 0;
  bool any_smem = false;
  for (int q = 0; q < nq; ++q) {
    const gj_query& Q = queries[q];
    // the variant this query runs (Sec. 7's choice made per query); the persistent
    // kernel runs the non-partitioned join, every other choice and every query
    // outside its limits runs alone after it
    const int v = resolve_join_variant(&Q.R, &Q.S, Q.nagg, &o, true);
    P->variant.push_back(v);
    if (v != GJ_JOIN_NPHJ || !batchable(Q)) {
      P->solo.push_back(q);
      continue;
    }
    BInst I{};
    I.rkey = (const int32_t*)Q.R.key;
    I.skey = (const int32_t*)Q.S.key;
    I.nr = Q.R.n;
    I.ns = Q.S.n;
    uint64_t hs = 2;
    while (hs < (uint64_t)(2 * I.nr)) hs <<= 1;
    I.ht_slots = hs;
    I.nslots = 2 * Q.group_key.modulus - 1;
    I.dense_off = Q.group_key.modulus - 1;
    I.nagg = Q.nagg;
    void* p = nullptr;
    const size_t bytes = sizeof(int32_t) * hs + sizeof(unsigned long long) * I.nslots +
                         sizeof(int64_t) * I.nslots * Q.nagg + 64 * (2 + Q.nagg);
    if (cudaMalloc(&p, bytes) != cudaSuccess) return fail(GJ_ERR_OOM);
    P->allocs.push_back(p);
    unsigned char* b = (unsigned char*)p;
    I.ht = (int32_t*)b;
    b += (sizeof(int32_t) * hs + 63) & ~size_t(63);
    I.cnt = (unsigned long long*)b;
    b += (sizeof(unsigned long long) * I.nslots + 63) & ~size_t(63);
    for (int j = 0; j < Q.nagg; ++j) {
      I.op[j] = Q.ops[j];
      I.agg[j] = (int64_t*)b;
      b += (sizeof(int64_t) * I.nslots + 63) & ~size_t(63);
      I.out_aggs[j] = Q.out_aggs[j];
      if (Q.ops[j] != GJ_AGG_COUNT) I.val[j] = make_ref(Q, Q.agg_cols[j]);
    }
    I.gk = make_ref(Q, Q.group_key);
    // shared-memory layout of a probe task: 32-bit row counts, then each aggregate
    // (32-bit COUNT / MIN / MAX when the values fit 32 bits, else 8 bytes: a split
    // or 64-bit SUM, 64-bit MIN / MAX)
    {
      int64_t off = 4 * I.nslots;
      for (int j = 0; j < Q.nagg; ++j) {
        const BRef& v = I.val[j];
        const bool fits32 = v.is_key || v.size == 4 || (v.mod > 0 && v.mod <= (int64_t(1) << 31));
        if (fits32) I.fits32 |= 1 << j;
        int kind = SK_64;
        if (Q.ops[j] == GJ_AGG_COUNT) kind = SK_COUNT32;
        else if (fits32) kind = Q.ops[j] == GJ_AGG_SUM ? SK_SPLIT : SK_MINMAX32;
        const int w = (kind == SK_COUNT32 || kind == SK_MINMAX32) ? 4 : 8;
        off = (off + w - 1) / w * w;
        I.sform[j] = kind;
        I.soff[j] = (int32_t)std::min<int64_t>(off, INT32_MAX);
        off += (int64_t)w * I.nslots;
      }
      I.smem = off <= kSmemAgg;
      any_smem |= I.smem != 0;
    }
    I.out_keys = Q.out_keys;
    I.cap = Q.capacity;
    I.d_ngroups = Q.d_ngroups;
    P->h_insts.push_back(I);
    sum_r += I.nr;
    sum_s += I.ns;
    sum_slots += I.nslots;
  }
  P->nq = (int)P->h_insts.size();
  if (P->nq == 0) {  // nothing for the persistent kernel
    *out = P;
    return GJ_OK;
  }
  nq = P->nq;
  P->dyn = any_smem ? kSmemAgg : 0;
  if (cudaFuncSetAttribute(batch_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemAgg) != cudaSuccess)
    return fail(GJ_ERR_CUDA);
  if (cudaMalloc(&P->d_insts, sizeof(BInst) * std::max(1, nq)) != cudaSuccess) return fail(GJ_ERR_OOM);

  // ---- autotuner: time every candidate for the fields left at zero
  gj_batch_config best = want;
  const auto key = std::make_tuple(ctx.device, nq, sum_r, sum_s, sum_slots);
  bool cached = false;
  {
    std::lock_guard<std::mutex> lock(g_tune_mu);
    auto it = g_tune_cache.find(key);
    if (it != g_tune_cache.end() && !want.build_rows && !want.probe_rows && !want.lookahead && !want.blocks_per_sm) {
      best = it->second;
      cached = true;
    }
  }
  const bool tune = !cached && (!want.build_rows || !want.probe_rows || !want.lookahead || !want.blocks_per_sm);
  if (tune) {
    std::vector<int> br = want.build_rows ? std::vector<int>{want.build_rows} : std::vector<int>{8192, 32768};
    std::vector<int> pr = want.probe_rows ? std::vector<int>{want.probe_rows} : std::vector<int>{8192, 32768};
    std::vector<int> la = want.lookahead ? std::vector<int>{want.lookahead} : std::vector<int>{1, 4};
    std::vector<int> bs = want.blocks_per_sm ? std::vector<int>{want.blocks_per_sm} : std::vector<int>{2, 3};
    float best_ms = 1e30f;
    for (int a : br)
      for (int b : pr)
        for (int c : la)
          for (int d : bs) {
            gj_batch_config cand{a, b, c, d};
            if ((st = capture(P, cand)) != GJ_OK) return fail(st);
            const float ms = time_plan(P, ctx.stream, 3);
            if (ms < best_ms) {
              best_ms = ms;
              best = cand;
            }
          }
    std::lock_guard<std::mutex> lock(g_tune_mu);
    g_tune_cache[key] = best;
  } else if (!cached) {
    best = want;
  }
  if (!best.build_rows) best.build_rows = 32768;
  if (!best.probe_rows) best.probe_rows = 32768;
  if (!best.lookahead) best.lookahead = 1;
  if (!best.blocks_per_sm) best.blocks_per_sm = 2;
  if ((st = capture(P, best)) != GJ_OK) return fail(st);
  if (cudaStreamSynchronize((cudaStream_t)stream) != cudaSuccess) return fail(GJ_ERR_CUDA);
  *out = P;
  return GJ_OK;
}

gj_status gj_batch_launch(gj_batch_plan* P, void* stream) {
  if (!P || (P->nq > 0 && !P->exec)) return GJ_ERR_INVALID_ARG;
  Ctx ctx;
  gj_status st = make_ctx(stream, &ctx);
  if (st != GJ_OK) return st;
  if (P->exec) {
    LaunchScope ls(ctx, KK_BATCH);
    if ((st = cuda_check(cudaGraphLaunch(P->exec, (cudaStream_t)stream))) != GJ_OK) return st;
  }
  for (int q : P->solo) {
    const gj_query& Q = P->queries[q];
    gj_options o = P->solo_opt;
    o.join_variant = P->variant[q];
    if ((st = join_groupby_run(ctx, &Q.R, &Q.S, Q.group_key, Q.nagg, Q.ops, Q.agg_cols, &o, Q.out_keys, Q.out_aggs,
                               Q.capacity, Q.d_ngroups)) != GJ_OK)
      return st;
  }
  return GJ_OK;
}

gj_status gj_batch_get_variants(const gj_batch_plan* P, int32_t* variants) {
  if (!P || (P->nq_total > 0 && !variants)) return GJ_ERR_INVALID_ARG;
  std::copy(P->variant.begin(), P->variant.end(), variants);
  return GJ_OK;
}

gj_status gj_batch_get_config(const gj_batch_plan* P, gj_batch_config* cfg) {
  if (!P || !cfg) return GJ_ERR_INVALID_ARG;
  *cfg = P->cfg;
  return GJ_OK;
}

gj_status gj_batch_destroy(gj_batch_plan* P) {
  if (!P) return GJ_ERR_INVALID_ARG;
  cudaDeviceSynchronize();
  if (P->exec) cudaGraphExecDestroy(P->exec);
  if (P->graph) cudaGraphDestroy(P->graph);
  for (void* p : P->allocs) cudaFree(p);
  if (P->d_insts) cudaFree(P->d_insts);
  if (P->d_tasks) cudaFree(P->d_tasks);
  if (P->d_ctl) cudaFree(P->d_ctl);
  delete P;
  return GJ_OK;
}

}  // extern "C"
