// Variant-selector network: hand-written FP32 forward, backward and optimiser
// kernels, and the selector state used by the AUTO variants. Once installed, the
// network stands in for the paper's variant rules (the join rule of Sec. 7 and
// the group-by decision tree of Fig. groupby-dt), which stay the fallback.
//
// Forward: one block of 64 threads per sample, thread j owns hidden unit j of
// both layers; the 11 outputs are reduced by threads 0..10. Backward: each block
// processes a fixed slice of the batch and accumulates its partial gradient in
// shared memory; a second kernel adds the partials in block order, so the
// gradient does not depend on scheduling. The net is far too small for tensor
// cores to matter (5,707 parameters).
#include <cuda_runtime.h>
#include <math.h>
#include <string.h>

#include <mutex>
#include <vector>

#include "gj_internal.cuh"

namespace gj {
namespace {

constexpr int kIn = GJ_MLP_IN, kH = GJ_MLP_HIDDEN, kOut = GJ_MLP_OUT, kP = GJ_MLP_PARAMS;
constexpr int kW1 = 0, kB1 = kW1 + kH * kIn, kW2 = kB1 + kH, kB2 = kW2 + kH * kH, kW3 = kB2 + kH,
              kB3 = kW3 + kOut * kH;
static_assert(kB3 + kOut == kP, "parameter layout");
constexpr int kSamplesPerBlock = 32;
constexpr int kJoinOut = GJ_MLP_JOIN_OUT;  // y[0, kJoinOut): join variants; the rest group-by variants
static_assert(kOut - kJoinOut == 6, "six group-by outputs");

// The join variant of output o < kJoinOut.
__host__ __device__ __forceinline__ int join_variant_of(int o) {
  return o < 3 ? GJ_JOIN_PHJ_TR + o : (o == 3 ? GJ_JOIN_SMJ_TR : GJ_JOIN_SMJ_UR);
}

__device__ __forceinline__ void mlp_forward_sample(const float* th, const float* x, float* z1, float* h1, float* z2,
                                                   float* h2, float* y) {
  const int j = threadIdx.x;
  float a = th[kB1 + j];
  for (int i = 0; i < kIn; ++i) a += th[kW1 + j * kIn + i] * x[i];
  z1[j] = a;
  h1[j] = a > 0.f ? a : 0.f;
  __syncthreads();
  float b = th[kB2 + j];
  for (int k = 0; k < kH; ++k) b += th[kW2 + j * kH + k] * h1[k];
  z2[j] = b;
  h2[j] = b > 0.f ? b : 0.f;
  __syncthreads();
  if (j < kOut) {
    float c = th[kB3 + j];
    for (int k = 0; k < kH; ++k) c += th[kW3 + j * kH + k] * h2[k];
    y[j] = c;
  }
  __syncthreads();
}

__global__ void __launch_bounds__(kH) mlp_forward_kernel(const float* __restrict__ th, const float* __restrict__ x,
                                                         int batch, float* __restrict__ y) {
  __shared__ float s_x[kIn], z1[kH], h1[kH], z2[kH], h2[kH], s_y[kOut];
  const int b = blockIdx.x;
  if (threadIdx.x < kIn) s_x[threadIdx.x] = x[(int64_t)b * kIn + threadIdx.x];
  __syncthreads();
  mlp_forward_sample(th, s_x, z1, h1, z2, h2, s_y);
  if (threadIdx.x < kOut) y[(int64_t)b * kOut + threadIdx.x] = s_y[threadIdx.x];
}

__global__ void __launch_bounds__(kH) mlp_select_kernel(const float* __restrict__ th, const float* __restrict__ x,
                                                        int n, int32_t* jv, int32_t* gv) {
  __shared__ float s_x[kIn], z1[kH], h1[kH], z2[kH], h2[kH], s_y[kOut];
  const int b = blockIdx.x;
  if (threadIdx.x < kIn) s_x[threadIdx.x] = x[(int64_t)b * kIn + threadIdx.x];
  __syncthreads();
  mlp_forward_sample(th, s_x, z1, h1, z2, h2, s_y);
  if (threadIdx.x == 0) {
    int bj = 0, bg = kJoinOut;
    for (int o = 1; o < kJoinOut; ++o)
      if (s_y[o] < s_y[bj]) bj = o;
    for (int o = kJoinOut + 1; o < kOut; ++o)
      if (s_y[o] < s_y[bg]) bg = o;
    jv[b] = join_variant_of(bj);
    gv[b] = GJ_GB_HGB + (bg - kJoinOut);
  }
}

// Partial gradient of the loss over samples [blockIdx.x * kSamplesPerBlock, ...).
__global__ void __launch_bounds__(kH) mlp_grad_partial_kernel(const float* __restrict__ th,
                                                              const float* __restrict__ x,
                                                              const float* __restrict__ t,
                                                              const float* __restrict__ mask, int batch,
                                                              float* __restrict__ part, float* __restrict__ part_loss) {
  __shared__ float g[kP];
  __shared__ float s_x[kIn], z1[kH], h1[kH], z2[kH], h2[kH], s_y[kOut], dy[kOut], dh2[kH], dz1[kH];
  __shared__ float s_loss;
  const int j = threadIdx.x;
  for (int p = j; p < kP; p += kH) g[p] = 0.f;
  if (j == 0) s_loss = 0.f;
  __syncthreads();
  const float inv_b = 1.0f / (float)batch;
  const int b0 = blockIdx.x * kSamplesPerBlock;
  const int b1 = min(batch, b0 + kSamplesPerBlock);
  for (int b = b0; b < b1; ++b) {
    if (j < kIn) s_x[j] = x[(int64_t)b * kIn + j];
    __syncthreads();
    mlp_forward_sample(th, s_x, z1, h1, z2, h2, s_y);
    if (j < kOut) {
      const float m = mask[(int64_t)b * kOut + j];
      const float d = (s_y[j] - t[(int64_t)b * kOut + j]) * m;
      dy[j] = 2.0f * d * inv_b;
      if (j == 0) {
        float l = 0.f;
        for (int o = 0; o < kOut; ++o) {
          const float mo = mask[(int64_t)b * kOut + o];
          const float dd = (s_y[o] - t[(int64_t)b * kOut + o]) * mo;
          l += dd * dd;
        }
        s_loss += l * inv_b;
      }
    }
    __syncthreads();
    // layer 3: thread j owns input unit j of w3 and h2's gradient
    float acc = 0.f;
    for (int o = 0; o < kOut; ++o) {
      g[kW3 + o * kH + j] += dy[o] * h2[j];
      acc += dy[o] * th[kW3 + o * kH + j];
    }
    if (j < kOut) g[kB3 + j] += dy[j];
    dh2[j] = z2[j] > 0.f ? acc : 0.f;  // dz2
    __syncthreads();
    // layer 2: thread j owns output unit j (row j of w2)
    for (int k = 0; k < kH; ++k) g[kW2 + j * kH + k] += dh2[j] * h1[k];
    g[kB2 + j] += dh2[j];
    float acc1 = 0.f;
    for (int k = 0; k < kH; ++k) acc1 += dh2[k] * th[kW2 + k * kH + j];
    dz1[j] = z1[j] > 0.f ? acc1 : 0.f;
    __syncthreads();
    // layer 1
    for (int i = 0; i < kIn; ++i) g[kW1 + j * kIn + i] += dz1[j] * s_x[i];
    g[kB1 + j] += dz1[j];
    __syncthreads();
  }
  for (int p = j; p < kP; p += kH) part[(int64_t)blockIdx.x * kP + p] = g[p];
  if (j == 0) part_loss[blockIdx.x] = s_loss;
}

__global__ void mlp_grad_reduce_kernel(const float* __restrict__ part, const float* __restrict__ part_loss, int nblk,
                                       float* __restrict__ grad, float* __restrict__ loss) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p < kP) {
    float s = 0.f;
    for (int b = 0; b < nblk; ++b) s += part[(int64_t)b * kP + p];
    grad[p] = s;
  }
  if (p == 0 && loss) {
    float s = 0.f;
    for (int b = 0; b < nblk; ++b) s += part_loss[b];
    *loss = s;
  }
}

__global__ void mlp_adam_kernel(float* th, const float* g, float* m, float* v, float lr, float b1, float b2,
                                float eps, float c1, float c2) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= kP) return;
  const float gp = g[p];
  const float mp = b1 * m[p] + (1.f - b1) * gp;
  const float vp = b2 * v[p] + (1.f - b2) * gp * gp;
  m[p] = mp;
  v[p] = vp;
  th[p] -= lr * (mp / c1) / (sqrtf(vp / c2) + eps);
}

__global__ void mlp_sgd_kernel(float* th, const float* g, float lr) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p < kP) th[p] -= lr * g[p];
}

// ---------------------------------------------------------------- selector state
std::mutex g_sel_mu;
bool g_sel_on = false;
std::vector<float> g_sel_theta, g_sel_mean, g_sel_std;

void host_forward(const float* th, const float* x, float* y) {
  float h1[kH], h2[kH];
  for (int j = 0; j < kH; ++j) {
    float a = th[kB1 + j];
    for (int i = 0; i < kIn; ++i) a += th[kW1 + j * kIn + i] * x[i];
    h1[j] = a > 0.f ? a : 0.f;
  }
  for (int j = 0; j < kH; ++j) {
    float a = th[kB2 + j];
    for (int k = 0; k < kH; ++k) a += th[kW2 + j * kH + k] * h1[k];
    h2[j] = a > 0.f ? a : 0.f;
  }
  for (int o = 0; o < kOut; ++o) {
    float a = th[kB3 + o];
    for (int k = 0; k < kH; ++k) a += th[kW3 + o * kH + k] * h2[k];
    y[o] = a;
  }
}

}  // namespace

void query_features(const gj_table* R, const gj_table* S, int nagg, const gj_options* opt, float* f) {
  const double nr = R ? (double)R->n : 0.0, ns = S ? (double)S->n : (R ? (double)R->n : 0.0);
  const gj_table* K = R ? R : S;
  const double groups = opt && opt->groups_hint > 0 ? (double)opt->groups_hint : ns;
  int sbytes = 0;
  if (S)
    for (int c = 0; c < S->ncols; ++c) sbytes += dtype_size(S->col_type[c]);
  f[0] = (float)log2(nr + 1.0);
  f[1] = (float)log2(ns + 1.0);
  f[2] = K ? (float)dtype_size(K->key_type) : 4.0f;
  f[3] = R ? (float)R->ncols : 0.0f;
  f[4] = S ? (float)S->ncols : 0.0f;
  f[5] = opt && opt->zipf_hint >= 0 ? opt->zipf_hint : 0.0f;
  f[6] = opt && opt->match_ratio_hint >= 0 ? opt->match_ratio_hint : 1.0f;
  f[7] = (float)log2(groups + 1.0);
  f[8] = (float)nagg;
  f[9] = (float)log2((nr + 1.0) / (ns + 1.0));
  f[10] = (float)sbytes;
  f[11] = (float)(log2(groups + 1.0) / log2(ns + 2.0));
}

// Variant choice of the trained network, or 0 when no network is set.
int mlp_choose(const gj_table* R, const gj_table* S, int nagg, const gj_options* opt, bool join, bool fused) {
  std::lock_guard<std::mutex> lock(g_sel_mu);
  if (!g_sel_on) return 0;
  float f[kIn], y[kOut];
  query_features(R, S, nagg, opt, f);
  for (int i = 0; i < kIn; ++i) f[i] = (f[i] - g_sel_mean[i]) / g_sel_std[i];
  // features the call knows nothing about take the training mean (0 once
  // normalised): the group-by's for a join alone, the join's for a group-by alone
  if (join && !fused) f[7] = f[8] = f[11] = 0.f;
  if (!join) f[0] = f[3] = f[6] = f[9] = 0.f;
  host_forward(g_sel_theta.data(), f, y);
  if (join) {
    // the join -> group-by call runs PHJ-TR, PHJ-UR and NPHJ only
    const int nj = fused ? 3 : kJoinOut;
    int b = 0;
    for (int o = 1; o < nj; ++o)
      if (y[o] < y[b]) b = o;
    return join_variant_of(b);
  }
  int b = kJoinOut;
  for (int o = kJoinOut + 1; o < kOut; ++o)
    if (y[o] < y[b]) b = o;
  return GJ_GB_HGB + (b - kJoinOut);
}

}  // namespace gj

using namespace gj;

extern "C" {

gj_status gj_mlp_forward(const float* theta, const float* x, int32_t batch, float* y, void* stream) {
  if (!theta || batch < 0 || (batch > 0 && (!x || !y))) return GJ_ERR_INVALID_ARG;
  if (batch == 0) return GJ_OK;
  Ctx ctx;
  gj_status st = make_ctx(stream, &ctx);
  if (st != GJ_OK) return st;
  LaunchScope ls(ctx, KK_MLP);
  mlp_forward_kernel<<<batch, kH, 0, ctx.stream>>>(theta, x, batch, y);
  return cuda_check(cudaGetLastError());
}

gj_status gj_mlp_select(const float* theta, const float* x, int32_t n, int32_t* jv, int32_t* gv, void* stream) {
  if (!theta || n < 0 || (n > 0 && (!x || !jv || !gv))) return GJ_ERR_INVALID_ARG;
  if (n == 0) return GJ_OK;
  Ctx ctx;
  gj_status st = make_ctx(stream, &ctx);
  if (st != GJ_OK) return st;
  LaunchScope ls(ctx, KK_MLP);
  mlp_select_kernel<<<n, kH, 0, ctx.stream>>>(theta, x, n, jv, gv);
  return cuda_check(cudaGetLastError());
}

gj_status gj_mlp_loss_grad(const float* theta, const float* x, const float* t, const float* mask, int32_t batch,
                           float* grad, float* loss, void* stream) {
  if (!theta || !x || !t || !mask || !grad || batch < 1) return GJ_ERR_INVALID_ARG;
  Ctx ctx;
  gj_status st = make_ctx(stream, &ctx);
  if (st != GJ_OK) return st;
  const int nblk = (batch + kSamplesPerBlock - 1) / kSamplesPerBlock;
  Scratch scr(ctx.stream);
  float* part = scr.get_as<float>((size_t)nblk * kP);
  float* part_loss = scr.get_as<float>(nblk);
  if (scr.failed()) return GJ_ERR_OOM;
  {
    LaunchScope ls(ctx, KK_MLP);
    mlp_grad_partial_kernel<<<nblk, kH, 0, ctx.stream>>>(theta, x, t, mask, batch, part, part_loss);
  }
  {
    LaunchScope ls(ctx, KK_MLP);
    mlp_grad_reduce_kernel<<<(kP + 255) / 256, 256, 0, ctx.stream>>>(part, part_loss, nblk, grad, loss);
  }
  return cuda_check(cudaGetLastError());
}

gj_status gj_mlp_adam_step(float* theta, const float* grad, float* m, float* v, int32_t step, float lr, float beta1,
                           float beta2, float eps, void* stream) {
  if (!theta || !grad || !m || !v || step < 1) return GJ_ERR_INVALID_ARG;
  Ctx ctx;
  gj_status st = make_ctx(stream, &ctx);
  if (st != GJ_OK) return st;
  const float c1 = 1.0f - powf(beta1, (float)step), c2 = 1.0f - powf(beta2, (float)step);
  LaunchScope ls(ctx, KK_MLP);
  mlp_adam_kernel<<<(kP + 255) / 256, 256, 0, ctx.stream>>>(theta, grad, m, v, lr, beta1, beta2, eps, c1, c2);
  return cuda_check(cudaGetLastError());
}

gj_status gj_mlp_sgd_step(float* theta, const float* grad, float lr, void* stream) {
  if (!theta || !grad) return GJ_ERR_INVALID_ARG;
  Ctx ctx;
  gj_status st = make_ctx(stream, &ctx);
  if (st != GJ_OK) return st;
  LaunchScope ls(ctx, KK_MLP);
  mlp_sgd_kernel<<<(kP + 255) / 256, 256, 0, ctx.stream>>>(theta, grad, lr);
  return cuda_check(cudaGetLastError());
}

gj_status gj_selector_set(const float* theta, const float* mean, const float* stdev) {
  std::lock_guard<std::mutex> lock(g_sel_mu);
  if (!theta) {
    g_sel_on = false;
    return GJ_OK;
  }
  if (!mean || !stdev) return GJ_ERR_INVALID_ARG;
  for (int i = 0; i < kIn; ++i)
    if (!(stdev[i] > 0.f)) return GJ_ERR_INVALID_ARG;
  g_sel_theta.assign(theta, theta + kP);
  g_sel_mean.assign(mean, mean + kIn);
  g_sel_std.assign(stdev, stdev + kIn);
  g_sel_on = true;
  return GJ_OK;
}

gj_status gj_query_features(const gj_table* R, const gj_table* S, int32_t nagg, const gj_options* opt, float* out) {
  if (!out || (!R && !S)) return GJ_ERR_INVALID_ARG;
  query_features(R, S, nagg, opt, out);
  return GJ_OK;
}

}  // extern "C"
