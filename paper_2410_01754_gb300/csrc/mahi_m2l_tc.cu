// Tensor-core M2L (tcgen05, sm_103a).  Placeholder entry points until the
// kernel lands: creation of a MAHI_MIXED handle fails with INVALID_ARG.
#include <vector>

#include "mahi_internal.h"

namespace mahi {

size_t tc_ops_bytes(int p) { (void)p; return 16; }
void tc_pack_ops(int p, const std::vector<std::vector<double>> &m2l, void *host_image) {
  (void)p; (void)m2l; (void)host_image;
}
int tc_build_units(mahi_ctx *h, std::vector<int> &units) {
  (void)h; (void)units;
  return -1;
}
int tc_m2l(mahi_ctx *h) {
  (void)h;
  return -1;
}

}  // namespace mahi
