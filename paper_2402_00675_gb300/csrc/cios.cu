// Multi-limb Montgomery multiplication (REDC at R = 2^{32k}).
#include "tune.h"

namespace montgb {

int launch_multilimb_op(mont_ctx_t, Mode, const void*, const void*, void*, size_t, void*) {
  return MONT_EINVAL;
}

}  // namespace montgb
