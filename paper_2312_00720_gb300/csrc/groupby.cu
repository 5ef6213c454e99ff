#include "gj_internal.cuh"
namespace gj {
gj_status groupby_run(const Ctx& ctx, const gj_table* in, int nagg, const int32_t* ops, const int32_t* op_col,
                      const gj_options* opt, void* out_keys, int64_t* const* out_aggs, int64_t cap,
                      int64_t* d_ngroups) {
  return GJ_ERR_UNSUPPORTED;
}
gj_status join_groupby_run(const Ctx& ctx, const gj_table* R, const gj_table* S, gj_colref gk, int nagg,
                           const int32_t* ops, const gj_colref* agg_cols, const gj_options* opt, int64_t* out_keys,
                           int64_t* const* out_aggs, int64_t cap, int64_t* d_ngroups) {
  return GJ_ERR_UNSUPPORTED;
}
}
