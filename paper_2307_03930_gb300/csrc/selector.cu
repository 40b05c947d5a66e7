// Learned schedule selector (placeholder until the MLP is trained).
#include "handle.hpp"

namespace rosko {
rosko_status select_learned(rosko_packed_s* h, int64_t N, rosko_tile* out, cudaStream_t st) {
  (void)h;
  (void)N;
  (void)out;
  (void)st;
  return ROSKO_ERR_UNSUPPORTED;
}
}  // namespace rosko
