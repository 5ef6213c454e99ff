// Cost-model selector: the paper's bandwidth models (M1-M4, Sec. 4.1.1, 4.1.3,
// 4.1.4, 4.4) extended to every variant this library implements and evaluated
// with GB300 constants, for AUTO requests under GJ_SELECT_COST (and under
// GJ_SELECT_MLP while no network is installed).
//
// Every variant's cost is the bytes it moves, in units of sequential global-memory
// bytes (so a cost divided by B_G is a time):
//   * sequential reads and writes count their bytes;
//   * unclustered accesses into a structure larger than the L2 share count
//     B_G / B_R times their bytes (M1; B_G / B_R measured on GB300 with the
//     clustered-vs-unclustered gather of 2^27 4-byte items, Table gather-profile);
//   * unclustered accesses into an L2-resident structure count B_G / B_L2 times
//     their bytes (the form of M4's B_M / min(g, 24) for an L2-resident table);
//   * each kernel launch and each host synchronisation inside a call adds a fixed
//     cost, which dominates small inputs;
//   * the partition-based group-by pays for its hottest partition (share 1 / H(g, z)
//     of the rows under a Zipf factor z): sliced over several blocks, it still
//     costs its rows' contention on the hot keys, counted as if one SM took them
//     at hot_row_bytes each.
// Host code only; it reads sizes, types and hints, never the data.
#include <algorithm>
#include <cmath>
#include <mutex>

#include "gj_internal.cuh"

namespace gj {
namespace {

std::mutex g_cost_mu;
bool g_cost_set = false;
gj_cost_params g_cost;

gj_cost_params installed_params() {
  std::lock_guard<std::mutex> lk(g_cost_mu);
  if (g_cost_set) return g_cost;
  gj_cost_params p;
  gj_cost_params_default(&p);
  return p;
}

// Device figures the parameters leave open (0), else GB300's.
void device_figures(const gj_cost_params& p, double* l2, double* smem, double* sms) {
  int dev = 0, l2b = 0, sm = 0, smem_b = 0;
  if (cudaGetDevice(&dev) == cudaSuccess) {
    cudaDeviceGetAttribute(&l2b, cudaDevAttrL2CacheSize, dev);
    cudaDeviceGetAttribute(&sm, cudaDevAttrMultiProcessorCount, dev);
    cudaDeviceGetAttribute(&smem_b, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  }
  cudaGetLastError();
  *l2 = p.l2_bytes > 0 ? p.l2_bytes : 0.5 * (l2b > 0 ? (double)l2b : 126.5 * 1048576.0);
  *smem = p.smem_bytes > 0 ? p.smem_bytes : (smem_b > 0 ? (double)std::min(smem_b, 200 * 1024) : 200.0 * 1024);
  *sms = p.num_sms > 0 ? (double)p.num_sms : (sm > 0 ? (double)sm : 152.0);
}

double dtype_bytes(int t) { return t == GJ_I64 ? 8.0 : 4.0; }

double payload_bytes(const gj_table* t) {
  double b = 0;
  for (int c = 0; c < t->ncols; ++c) b += dtype_bytes(t->col_type[c]);
  return b;
}

// Share of the rows carried by the most frequent of g keys under Zipf factor z:
// 1 / H(g, z), with H's first 1024 terms summed and the rest integrated.
double zipf_top_share(double g, double z) {
  if (g <= 1) return 1.0;
  if (z <= 0) return 1.0 / g;
  const double head = std::min(g, 1024.0);
  double h = 0;
  for (int i = 1; i <= (int)head; ++i) h += std::pow((double)i, -z);
  if (g > head) {
    const double a = head + 0.5, b = g + 0.5;
    h += std::fabs(z - 1.0) < 1e-9 ? std::log(b / a) : (std::pow(b, 1.0 - z) - std::pow(a, 1.0 - z)) / (1.0 - z);
  }
  return 1.0 / h;
}

struct Model {
  gj_cost_params p;
  double l2, smem, sms;
  double rnd(double bytes, double footprint) const {
    return bytes * (footprint <= l2 ? p.bg_over_bl2 : p.bg_over_br);
  }
};

double pow2_ceil(double x) {
  double v = 1;
  while (v < x) v *= 2;
  return v;
}

// join_cost[0..4]: PHJ-TR, PHJ-UR, NPHJ, SMJ-TR, SMJ-UR.
void join_costs(const Model& m, const gj_table* R, const gj_table* S, const gj_options* opt, double* c) {
  const double nr = (double)R->n, ns = (double)S->n, k = dtype_bytes(R->key_type);
  const double wr = payload_bytes(R), ws = payload_bytes(S);
  const double mr = opt->match_ratio_hint < 0 ? 1.0 : std::min(1.0, (double)opt->match_ratio_hint);
  const double M = mr * ns;                 // result rows: each S row matches at most one R row
  const double out = M * (k + wr + ws);     // the result, written once by every variant
  const double L = m.p.launch_bytes;
  // PHJ: one 8-bit pass per side up to 2^27 build rows, else two
  const double pp = nr > (double)(1 << 27) ? 2 : 1;
  const double build_probe = k * (nr + ns) + 8.0 * (nr + ns);  // per-partition tables stay on chip / in L2
  c[0] = (k + 2 * pp * (k + wr)) * nr + (k + 2 * pp * (k + ws)) * ns + build_probe + M * (wr + ws) + out + 10 * L;
  c[1] = (k + 2 * pp * (k + 4)) * (nr + ns) + build_probe + m.rnd(M * wr, nr * wr) + m.rnd(M * ws, ns * ws) +
         8.0 * M + out + 11 * L;
  // NPHJ: a global table of row ids, 2 |R| slots rounded up to a power of two
  const double table = 4.0 * pow2_ceil(std::max(2.0 * nr, 2.0)) + k * nr;
  c[2] = k * nr + 4.0 * nr + k * ns + m.rnd(4.0 * ns + k * M, table) + m.rnd(M * wr, nr * wr) + ns * ws + out + 3 * L;
  // SMJ: both sides sorted on the whole key, one 8-bit pass per key byte
  const double ps = k;
  c[3] = (k + 2 * ps * (k + wr)) * nr + (k + 2 * ps * (k + ws)) * ns + k * (nr + ns) + out + 26 * L;
  c[4] = (k + 2 * ps * (k + 4)) * (nr + ns) + k * (nr + ns) + m.rnd(M * wr, nr * wr) + m.rnd(M * ws, ns * ws) + out +
         27 * L;
}

// gb_cost[0..5]: HGB, SGB, PGB, SGB-UR, PGB-UR, SGB-DE.
void groupby_costs(const Model& m, const gj_table* in, int nagg, const int32_t* ops, const gj_options* opt,
                   double* c) {
  const double n = (double)in->n, k = dtype_bytes(in->key_type), w = payload_bytes(in);
  const double g = std::max(1.0, opt->groups_hint > 0 ? (double)opt->groups_hint : n);
  const double z = opt->zipf_hint < 0 ? 0.0 : (double)opt->zipf_hint;
  double slot = 0;
  for (int j = 0; j < nagg; ++j) slot += (!ops || ops[j] == GJ_AGG_SUM) ? 8 : 4;
  const double out = g * (k + 8.0 * nagg);
  const double L = m.p.launch_bytes, Y = m.p.sync_bytes;
  // HGB: dictionary of 2g (key, id) entries; lookups hit each block's shared-memory
  // cache of 16384 keys when g is at most that; aggregates in shared memory when
  // the g slots fit, else global atomics
  const double dict = 2.0 * g * (k + 4);
  const double look = g <= 16384 ? 0.0 : m.rnd((k + 4) * n, dict);
  const double agg = g * slot <= m.smem ? 0.0 : m.rnd(8.0 * nagg * n, 8.0 * nagg * g);
  c[0] = 2 * k * n + m.rnd((k + 4) * g, dict) + w * n + look + agg + out + 5 * L;
  // SGB: one 8-bit pass per byte of the varying key bits (about log2 g of them)
  const double ps = std::ceil(std::max(1.0, std::ceil(std::log2(g))) / 8.0);
  c[1] = (k + 2 * ps * (k + w)) * n + (k + w) * n + out + 9 * L + Y;
  c[3] = (k + 2 * ps * (k + 4)) * n + (k + 4) * n + m.rnd(w * n, w * n) + out + 10 * L + Y;
  c[5] = 2 * k * n + m.rnd((k + 4) * g, dict) + m.rnd((k + 4) * n, dict) + (4 + 2 * ps * (4 + w)) * n + (4 + w) * n +
         out + 12 * L;
  // PGB: one pass up to 2^20 groups, else two; the hottest partition's contention
  const double pb = g <= (double)(1 << 20) ? 1 : 2;
  const double hot = zipf_top_share(g, z) * n * m.sms * m.p.hot_row_bytes;
  const double pgb_sync = n * (k + 8.0 * nagg) > 256.0 * 1048576.0 ? Y : 0.0;  // sizing its partial rows
  c[2] = (k + 2 * pb * (k + w)) * n + (k + w) * n + out + 5 * L + hot + pgb_sync;
  c[4] = (k + 2 * pb * (k + 4)) * n + (k + 4) * n + m.rnd(w * n, w * n) + out + 6 * L + hot + pgb_sync;
}

Model make_model() {
  Model m;
  m.p = installed_params();
  device_figures(m.p, &m.l2, &m.smem, &m.sms);
  return m;
}

constexpr int kJoinOrder[5] = {GJ_JOIN_PHJ_TR, GJ_JOIN_PHJ_UR, GJ_JOIN_NPHJ, GJ_JOIN_SMJ_TR, GJ_JOIN_SMJ_UR};

}  // namespace

int cost_join_variant(const gj_table* R, const gj_table* S, const gj_options* opt, bool fused) {
  double c[5];
  join_costs(make_model(), R, S, opt, c);
  const int nv = fused ? 3 : 5;
  int best = 0;
  for (int i = 1; i < nv; ++i)
    if (c[i] < c[best]) best = i;
  return kJoinOrder[best];
}

int cost_groupby_variant(const gj_table* in, int nagg, const int32_t* ops, const gj_options* opt) {
  double c[6];
  groupby_costs(make_model(), in, nagg, ops, opt, c);
  int best = 0;
  for (int i = 1; i < 6; ++i)
    if (c[i] < c[best]) best = i;
  return GJ_GB_HGB + best;
}

}  // namespace gj

using namespace gj;

extern "C" {

void gj_cost_params_default(gj_cost_params* p) {
  if (!p) return;
  p->bg_over_br = 27.5;         // GB300: unclustered / clustered gather time of 2^27 int32 = 9.82 -> 3r - 2
  p->bg_over_bl2 = 27.5 / 4.5;  // B_L2 = 4.5 B_G as Sec. 4.4 gives for the A100, over the GB300 ratio
  p->l2_bytes = 0;              // half the device's L2 (its near die)
  p->smem_bytes = 0;            // the device's opt-in shared memory per block (at most 200 KB)
  p->launch_bytes = 2.0e7;      // about 3 us at 6.8 TB/s
  p->sync_bytes = 6.0e7;        // a host round trip inside the call
  p->hot_row_bytes = 10.0;  // PGB slices its hottest partitions; what remains is contention on the hot keys
  p->num_sms = 0;
}

gj_status gj_set_cost_params(const gj_cost_params* p) {
  if (p && (!(p->bg_over_br >= 1.0) || !(p->bg_over_bl2 >= 1.0) || p->l2_bytes < 0 || p->smem_bytes < 0 ||
            p->launch_bytes < 0 || p->sync_bytes < 0 || p->hot_row_bytes < 0 || p->num_sms < 0))
    return GJ_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(g_cost_mu);
  g_cost_set = p != nullptr;
  if (p) g_cost = *p;
  return GJ_OK;
}

gj_status gj_cost_estimate(const gj_table* R, const gj_table* S, int32_t nagg, const int32_t* ops,
                           const gj_options* opt, double* join_cost, double* gb_cost) {
  gj_options defaults;
  gj_options_default(&defaults);
  if (!opt) opt = &defaults;
  if (!S || S->n < 0 || (R && R->n < 0)) return GJ_ERR_INVALID_ARG;
  const Model m = make_model();
  if (join_cost) {
    if (!R) return GJ_ERR_INVALID_ARG;
    join_costs(m, R, S, opt, join_cost);
  }
  if (gb_cost) {
    if (nagg < 1) return GJ_ERR_INVALID_ARG;
    groupby_costs(m, S, nagg, ops, opt, gb_cost);
  }
  return GJ_OK;
}

}  // extern "C"
