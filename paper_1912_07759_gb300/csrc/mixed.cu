// mixed.cu -- mixed-precision path: FP16 log10 sigma tables and the tau contraction on
// tensor cores as BF16 hi+lo split products.
#include "tr_internal.h"

namespace tr {

int build_fp16_log_tables(tr_ctx* ctx, tr_tables*) {
  return set_error(ctx, TR_ERR_UNSUPPORTED, "FP16 log10 tables are not built in this version");
}

int forward_mixed(tr_ctx* ctx, const tr_tables*, int, const ItemBuffers&, int, int, int,
                  double*, long long, cudaStream_t) {
  return set_error(ctx, TR_ERR_UNSUPPORTED, "mixed precision is not built in this version");
}

}  // namespace tr
