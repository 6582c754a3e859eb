// Wing decomposition (Sec. 3.3) -- under construction.
#include "internal.cuh"

namespace pbng {
void wing_decompose(Arena &a, Graph &G, const TipParams &p, uint64_t *theta_out, pbng_stats *st) {
  (void)a; (void)G; (void)p; (void)theta_out; (void)st;
  fail(PBNG_EINVAL, "wing decomposition is not available in this build");
}
}  // namespace pbng
