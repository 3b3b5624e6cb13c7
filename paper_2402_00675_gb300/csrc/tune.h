// Launch-shape selection for the element-wise kernels.
#pragma once

#include "internal.h"
#include "montgb.h"

namespace montgb {

// Shape the element-wise launcher uses for (word width, variant, mode):
// the autotuner's choice for the current device when one is recorded,
// otherwise the built-in default.
LaunchShape tuned_shape(int width, int variant, int mode);

// Record a shape for the current device (used by the autotuner).
void set_tuned_shape(int width, int variant, int mode, const LaunchShape& shape);

// Shape of the batched kernel for a word width (threads, unroll, tile_iters).
LaunchShape tuned_batched_shape(int width);
void set_tuned_batched_shape(int width, const LaunchShape& shape);

// Multi-limb element-wise operations (cios.cu).
int launch_multilimb_op(mont_ctx_t ctx, Mode mode, const void* x, const void* y, void* out,
                        size_t n, void* stream);
// Whether the multi-limb REDC kernels have a build for k limbs at this many
// lanes per element (others run at the default team).
bool multilimb_team_supported(int k, int team);

}  // namespace montgb
