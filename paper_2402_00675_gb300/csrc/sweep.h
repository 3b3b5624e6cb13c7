// The verify sweep in steps (sweep.cu), for callers that place its device
// scratch themselves and launch its chunks in pieces: mont_verify_sweep runs
// them back to back on memory it allocates; the serving loop runs them in
// bounded pieces on memory from its arena, checking a deadline in between.
#pragma once

#include <cuda_runtime.h>

#include <cstddef>
#include <cstdint>
#include <vector>

#include "montgb.h"

namespace montgb {

// One swept modulus: its constants, T interval and claimed output range.
struct SweepN {
  int32_t N;
  uint32_t nprime;   // -N^{-1} mod R
  uint32_t ninv;     // N^{-1} mod R (two's complement reading gives N^{-1} mods R)
  uint32_t step;     // s R^{-1} mod N
  int64_t t_lo;      // first T of this modulus
  int64_t t_hi;      // last T
  int32_t r_lo;      // claimed range (inclusive)
  int32_t r_hi;
  uint64_t item0;    // index of this modulus's first chunk
};

struct SweepParams {
  int log2R;
  int n;            // log2R / 2 (Plantard family)
  int alpha;
  uint32_t chunk;   // T per chunk
  int range_kind;   // how the claimed range is tested (see sweep.cu)
  uint32_t one;     // 1 (a multiplier the kernel cannot fold; see sweep.cu)
};

// A sweep prepared on the host: the table of swept moduli (odd N that pass
// the variant's condition, or all with MONT_SWEEP_INCLUDE_OUT_OF_SPEC, and
// whose domain is not empty), where each entry's count belongs among the odd
// N of the request, and the chunking.
struct SweepPlan {
  int variant = 0;
  SweepParams p{};
  std::vector<SweepN> tab;
  std::vector<size_t> tab_index;   // position of each entry among the odd N
  size_t n_odd = 0;                // odd N in [N_lo, N_hi]
  uint64_t items = 0;              // chunks of the whole sweep
  uint64_t total_T = 0;            // checks of the whole sweep
  size_t cex_cap = 0;
};

// Validate the arguments (the limits of mont_verify_sweep) and build the plan;
// sets per_N_checked (if not NULL) and clears per_N_counts.  MONT_EINVAL on
// bad arguments.  Allocates host memory only.
int sweep_plan(int variant, int log2R, int alpha, uint32_t N_lo, uint32_t N_hi,
               const mont_bounds* claimed, int flags, size_t cex_cap, uint64_t* per_N_counts,
               uint64_t* per_N_checked, SweepPlan* plan);

// Device scratch a plan of n_tab entries and cex_cap examples needs (an upper
// bound for n_tab = the number of odd N of the request); 256-byte aligned
// start required.
size_t sweep_scratch_bytes(size_t n_tab, size_t cex_cap);

// Enqueue on s: the table into scratch, the counters cleared.
cudaError_t sweep_upload(const SweepPlan& plan, void* scratch, cudaStream_t s);

// Enqueue on s the chunks [item_lo, item_hi) of the plan.
cudaError_t sweep_launch(const SweepPlan& plan, void* scratch, uint64_t item_lo, uint64_t item_hi,
                         cudaStream_t s);

// Chunks per launch that keep one launch to about `checks` checks.
uint64_t sweep_items_for_checks(const SweepPlan& plan, uint64_t checks);

// After every launch has been enqueued: copy the counts and the examples back
// (synchronises s), sort the examples by (N, T) and report the total.
// MONT_EOVERFLOW when the total exceeds cex_cap.
int sweep_collect(const SweepPlan& plan, void* scratch, cudaStream_t s, uint64_t* per_N_counts,
                  mont_cex* cex, size_t* n_cex_total);

}  // namespace montgb
