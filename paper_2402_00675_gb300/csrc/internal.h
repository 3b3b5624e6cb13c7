// Internal declarations shared by the library's translation units.
//
// The per-modulus constants travel to the kernels by value (kernel parameter
// space is broadcast through the constant bank), so a ctx owns host memory
// only and the word kernels read nothing from global memory except their
// operands.
#pragma once

#include <cuda_runtime.h>

#include <cstddef>
#include <cstdint>
#include <vector>

#include "montgb.h"

namespace montgb {

// Constants of one modulus for the 32-bit word kernels.
struct WordConst32 {
  uint32_t N;       // modulus
  uint32_t nprime;  // N' = -N^{-1} mod 2^32 (REDC, Section 1)
  uint32_t ninv;    // N^{-1} mod 2^32; read as a signed word it is N^{-1} mods 2^32 (Algorithm 1)
  uint32_t half;    // (N - 1) / 2, bound of the mods-N range
  uint64_t ninv2;   // N^{-1} mod 2^64 for the Plantard family (R = 2^{2n}, n = 32)
  uint32_t r2;      // domain constant (R^2 mod N, or its mods-N form as a two's complement word)
  int32_t alpha;    // Algorithm 4's parameter
};

// Constants of one modulus for the 64-bit word kernels.
struct WordConst64 {
  uint64_t N;
  uint64_t nprime;   // -N^{-1} mod 2^64
  uint64_t ninv;     // N^{-1} mod 2^64
  uint64_t half;     // (N - 1) / 2
  uint64_t ninv2_lo; // N^{-1} mod 2^128, low word   (Plantard family, n = 64)
  uint64_t ninv2_hi; // N^{-1} mod 2^128, high word
  uint64_t r2;       // domain constant
  int32_t alpha;
};

// Constants of one modulus for the multi-limb kernels (R = 2^{32k}).
struct LimbConst {
  uint32_t n0prime;             // -N^{-1} mod 2^32: the only inverse CIOS needs
  uint32_t N[MONT_MAX_LIMBS];   // modulus, little-endian limbs (k used)
  uint32_t r2[MONT_MAX_LIMBS];  // R^2 mod N
  uint32_t dom[MONT_MAX_LIMBS]; // Algorithm 1's domain constant: (R^2 mod N) mods N, two's complement
};

// Constants of one modulus for the multi-limb kernels of Algorithms 1-4
// (R = 2^{32k} for Algorithm 1, 2^{64k} for the Plantard family).
struct LimbVarConst {
  int variant;
  int alpha;
  uint32_t N[MONT_MAX_LIMBS];
  uint32_t ninv[2 * MONT_MAX_LIMBS];  // N^{-1} mod R: k limbs (Algorithm 1) or 2k (Algorithms 2-4)
  uint32_t dom[MONT_MAX_LIMBS];       // mont_to_domain constant, two's complement for signed variants
  uint32_t half[MONT_MAX_LIMBS];      // (N - 1) / 2
};

// Launch shape of an element-wise kernel.
struct LaunchShape {
  int threads = 256;        // threads per block
  int unroll = 2;           // vectors in flight per thread per operand
  int vec_bytes = 32;       // 32 (256-bit), 16 (128-bit) or 0 (scalar path)
  int blocks_per_sm = 0;    // 0: as many as the occupancy calculator allows
  int tile_iters = 2;       // batched kernel: CTA iterations per tile
  int team = 0;             // multi-limb: lanes per element (0: default for k)
};

enum class Mode : int { kMul = 0, kToDomain = 1, kFromDomain = 2, kRedc = 3 };

// Element-wise launchers (word.cu).  Return a cudaError_t.
cudaError_t launch_word32(int variant, Mode mode, const WordConst32& c, const void* x,
                          const void* y, void* out, size_t n, cudaStream_t s,
                          const LaunchShape& shape);
cudaError_t launch_word64(int variant, Mode mode, const WordConst64& c, const void* x,
                          const void* y, void* out, size_t n, cudaStream_t s,
                          const LaunchShape& shape);

// Multi-limb Algorithms 1-4 (limb_variants.cu); k in {4, 8, 12, 16, 32, 64}.
cudaError_t launch_limb_variant(int k, Mode mode, const LimbVarConst& c, const uint32_t* x,
                                const uint32_t* y, uint32_t* o, size_t n, cudaStream_t s,
                                int vec16, const LaunchShape& shape);

// Launch a kernel with programmatic stream serialization: it may be
// scheduled while the kernel before it in the stream drains.  The kernel must
// execute `griddepcontrol.wait` before its first memory access (and may then
// execute `griddepcontrol.launch_dependents`).  Used for the HBM-bound word
// kernels only: blocks scheduled early land in whatever slots the previous
// grid frees, unevenly over the SMs, which a bandwidth-bound kernel does not
// notice but a compute-bound grid-stride kernel does (the multi-limb REDC
// kernel at 1024 bits measured 57 -> 63-76 us with it).
template <typename... KArgs, typename... Args>
cudaError_t launch_pdl(void (*kernel)(KArgs...), unsigned grid, unsigned threads, size_t smem,
                       cudaStream_t s, Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(threads);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kernel, args...);
}

// The first statements of a kernel launched by launch_pdl: wait for the
// kernel before it, then let the next one's blocks be scheduled into slots
// this grid frees (a dependent kernel is scheduled only once every block of
// this grid has started, so it never holds slots this grid still needs).
__device__ __forceinline__ void pdl_enter() {
  asm volatile("griddepcontrol.wait;" ::: "memory");
  asm volatile("griddepcontrol.launch_dependents;" :::);
}

// Number of SMs of the current device (cached per device).
int device_sm_count();

// Occupancy-derived resident blocks per SM of a kernel at a block size
// (cached per kernel, block size and device).
int resident_blocks(const void* kernel, int threads);

}  // namespace montgb

// The opaque ctx of the C ABI.
struct mont_ctx {
  int variant = 0;
  int alpha = 0;
  int log2R = 0;
  int n_limbs = 0;     // limbs of one element (1, 2 or k)
  int width = 0;       // 32, 64 or 32k
  std::vector<uint32_t> N, ninv, nprime, r_mod_n, r2_mod_n, domain_r2;
  montgb::WordConst32 w32{};
  montgb::WordConst64 w64{};
  montgb::LimbConst limb{};
  montgb::LimbVarConst limbv{};
};

namespace montgb {
// Set the per-thread CUDA error and map it to a status.
int cuda_status(cudaError_t e);
}  // namespace montgb
