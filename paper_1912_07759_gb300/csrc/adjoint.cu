// adjoint.cu -- hand-written reverse-mode derivative of the batched forward model.
#include "tr_internal.h"

namespace tr {
size_t adjoint_extra_bytes(const tr_tables*, const tr_batch_desc*, const tr_bins*, int) {
  return 0;
}
}  // namespace tr

extern "C" int tr_adjoint_transit(tr_ctx* ctx, const tr_tables*, const tr_batch_desc*, int,
                                  const double*, const int32_t*, const tr_bins*, const double*,
                                  const double*, const double*, double*, double*, double*,
                                  int32_t*, int, void*, size_t, void*) {
  return tr::set_error(ctx, TR_ERR_UNSUPPORTED, "adjoint is not built in this version");
}
