/*
 * montgb -- Montgomery-type modular multiplication on NVIDIA GB300 (sm_103a).
 *
 * C ABI of the library.  The arithmetic follows Xu, Jia and Yang, "Chinese
 * Remainder Theorem Approach to Montgomery-Type Algorithms": REDC (Section 1,
 * derived from Qin's identity in Section 2, Eqs. (1)-(4)), the signed
 * Montgomery reduction (Algorithm 1), Plantard's reduction (Algorithm 2) and
 * the two signed Plantard reductions (Algorithms 3 and 4).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * - Every function returns an int status: MONT_OK (0) or one of the MONT_E*
 *   codes below.  Nothing aborts, prints or throws.  On MONT_ECUDA the CUDA
 *   error code of the failing runtime call is kept per thread and returned by
 *   mont_last_cuda_error().
 * - "device pointer" arguments are addresses in the current CUDA device's
 *   global memory, allocated and owned by the caller; the library never frees
 *   or retains them past the call.  "host pointer" arguments are ordinary
 *   process memory, also owned by the caller.
 * - `stream` is a cudaStream_t passed as void*; NULL is the legacy default
 *   stream.  Calls that take a stream only enqueue work on it and return
 *   without synchronising, unless their comment says otherwise; the caller
 *   must keep every buffer alive until that work completes.
 * - Element layout: all integers are little-endian.  A ctx of word width 32
 *   works on uint32_t (REDC, Plantard) or int32_t (signed variants) elements,
 *   width 64 on uint64_t / int64_t elements, and a multi-limb ctx of k limbs
 *   on elements of k consecutive uint32_t limbs, least significant first,
 *   element i occupying limbs [i*k, (i+1)*k).
 * - Alignment: device pointers must be aligned to their element's word size
 *   (4 bytes for 32-bit words and limbs, 8 for 64-bit words, 16 for the
 *   128-bit T of mont_redc at width 64); otherwise MONT_EINVAL.  Buffers that
 *   are also 32-byte aligned take the 256-bit vector path; others take a
 *   scalar path with identical results.
 * - Inputs out of the range a variant's algorithm requires are not checked on
 *   the device; the result for them is whatever the algorithm's formula
 *   yields in the word arithmetic described at each variant.
 */
#ifndef MONTGB_H
#define MONTGB_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---------------------------------------------------------------- status */
#define MONT_OK        0
#define MONT_EINVAL    1  /* bad argument, unsupported (variant, width), precondition on N violated */
#define MONT_ENOMEM    2  /* a host or device allocation failed */
#define MONT_ECUDA     3  /* a CUDA runtime call failed; see mont_last_cuda_error() */
#define MONT_ETIMEOUT  4  /* a bounded wait (device work-queue or host event) gave up */
#define MONT_EOVERFLOW 5  /* an output buffer was too small; counts stay exact */

/* -------------------------------------------------------------- variants */
/* REDC (Section 1): returns T R^{-1} mod N in [0, N); requires N < R, 0 <= T < RN. */
#define MONT_REDC              0
/* SigRedc (Algorithm 1): returns r = T R^{-1} (mod N), -N < r < N;
 * requires 2N < R and -NR/2 < T < NR/2. */
#define MONT_SIGNED            1
/* PRedc (Algorithm 2), R = 2^{2n}: returns -T R^{-1} mod N in [0, N);
 * requires N < 2^n/phi (phi the golden ratio) and 0 <= T <= N^2. */
#define MONT_PLANTARD          2
/* SigPRedc1 (Algorithm 3), R = 2^{2n}: returns -T R^{-1} mods N;
 * requires N < 2^{n-1} and |T| <= 2^{2n-2}. */
#define MONT_SIGNED_PLANTARD   3
/* SigPRedc2 (Algorithm 4), R = 2^{2n}, parameter alpha: returns
 * -T R^{-1} mods N for alpha >= 1; requires N < 2^{n-alpha-1} and
 * |T| <= 2^{2 alpha} N^2.  Section 3.3 shows alpha = 0 is wrong (Example 3.1);
 * a ctx with alpha = 0 is refused, and the sweep below can test it. */
#define MONT_SIGNED_PLANTARD2  4

/* Largest multi-limb width: 64 limbs of 32 bits (2048-bit moduli). */
#define MONT_MAX_LIMBS 64

typedef struct mont_ctx* mont_ctx_t;  /* opaque; owned by the library */

/*
 * mont_ctx_create -- per-modulus precomputation (the constants of Section 1
 * and Theorem 2.1: N^{-1} mod R, N' = R - N^{-1}, R mod N, R^2 mod N).
 *
 *   out      host pointer; receives the new ctx (left untouched on error).
 *   N_limbs  host pointer to n_limbs little-endian 32-bit limbs of the odd
 *            modulus N >= 3.  Upper limbs may be zero.
 *   n_limbs  1 -> 32-bit word kernels, 2 -> 64-bit word kernels,
 *            4, 8, 12, 16, 32 or 64 -> multi-limb kernels (every variant;
 *            signed elements are k-limb two's complement integers).
 *   log2R    R = 2^log2R.  Must be 32*n_limbs for MONT_REDC and MONT_SIGNED,
 *            and 64*n_limbs (the paper's R = 2^{2n} with n the word size) for
 *            the three Plantard variants.
 *   variant  one of the MONT_* variant codes.
 *   alpha    Algorithm 4's parameter (>= 1); ignored by other variants.
 *
 * Errors: MONT_EINVAL if N is even or < 3, if N violates the variant's
 * condition on N listed above, if (variant, n_limbs, log2R) is not a
 * supported combination, or if a pointer is NULL; MONT_ENOMEM.
 * The ctx holds host memory only; it can be used from any thread and on any
 * stream, concurrently, and is freed by mont_ctx_destroy.
 */
int mont_ctx_create(mont_ctx_t* out, const uint32_t* N_limbs, int n_limbs,
                    int log2R, int variant, int alpha);

/* Free a ctx.  NULL is accepted.  Work already enqueued that used the ctx is
 * unaffected (kernels receive the constants by value). */
int mont_ctx_destroy(mont_ctx_t ctx);

/* Which precomputed constant mont_ctx_constant returns. */
#define MONT_CONST_N          0  /* N                                              */
#define MONT_CONST_NINV       1  /* N^{-1} mod R, in [1, R)                         */
#define MONT_CONST_NPRIME     2  /* N' = R - N^{-1} (Section 1)                     */
#define MONT_CONST_R_MOD_N    3  /* R mod N                                         */
#define MONT_CONST_R2_MOD_N   4  /* R^2 mod N, in [0, N)                            */
#define MONT_CONST_DOMAIN_R2  5  /* constant mont_to_domain multiplies by: R^2 mod N
                                    for unsigned variants, (R^2 mod N) mods N for
                                    signed ones (two's complement in the limbs)    */

/*
 * mont_ctx_constant -- copy one precomputed constant out of a ctx, as
 * little-endian 32-bit limbs (log2R/32 limbs for NINV and NPRIME, n_limbs
 * limbs for the others), into the host buffer `limbs` of `cap` limbs.
 * *n_out receives the number of limbs written.  MONT_EOVERFLOW if cap is too
 * small (nothing written); MONT_EINVAL on a bad `which` or NULL pointer.
 */
int mont_ctx_constant(mont_ctx_t ctx, int which, uint32_t* limbs, int cap, int* n_out);

/*
 * mont_ctx_query -- shape of a ctx: word width in bits (32, 64 or 32*k),
 * number of limbs of one element, bytes per element, variant, log2R, alpha.
 * Any output pointer may be NULL.
 */
int mont_ctx_query(mont_ctx_t ctx, int* width_bits, int* n_limbs, int* elem_bytes,
                   int* variant, int* log2R, int* alpha);

/*
 * mont_mul -- out[i] = reduce(a[i] * b[i]) for i in [0, n): the Montgomery-
 * type product a b R^{-1} (REDC, Algorithm 1) or -a b R^{-1} (Algorithms 2-4)
 * in the variant's output range.  a, b, out: device pointers of n elements
 * each (element type per the ctx); out may alias a or b exactly (in place),
 * but must not partially overlap them.  Inputs must lie in the variant's
 * output range (so that T = a b is in the algorithm's input domain):
 * [0, N) for REDC, Plantard and multi-limb; (-N, N) for Algorithm 1;
 * the mods-N range [-(N-1)/2, (N-1)/2] for Algorithms 3 and 4.
 * n = 0 is a no-op.  Asynchronous on `stream`.
 */
int mont_mul(mont_ctx_t ctx, const void* a, const void* b, void* out, size_t n,
             void* stream);

/*
 * mont_redc -- out[i] = reduce(T[i]) for a caller-supplied double-width T:
 * int64/uint64 at width 32, 128-bit two's complement (16 bytes, low word
 * first) at width 64, 2k limbs at k limbs.  T must lie in the algorithm's
 * input domain (see the variant codes).  Device pointers; asynchronous.
 */
int mont_redc(mont_ctx_t ctx, const void* T, void* out, size_t n, void* stream);

/*
 * mont_to_domain -- out[i] = reduce(x[i] * MONT_CONST_DOMAIN_R2): the
 * representation x R mod N of Section 1's map Phi for REDC and Algorithm 1,
 * and -x R mod N for the Plantard variants (whose reductions return
 * -T R^{-1}, so products stay closed).  x must lie in the variant's input
 * range as for mont_mul.  Device pointers; asynchronous; out may alias x.
 */
int mont_to_domain(mont_ctx_t ctx, const void* x, void* out, size_t n, void* stream);

/*
 * mont_from_domain -- out[i] = canonical(reduce(y[i])): leaves the
 * representation; the result is in [0, N) for unsigned variants and in
 * [-(N-1)/2, (N-1)/2] for signed ones, so from(to(x)) = x.  Device pointers;
 * asynchronous; out may alias y.
 */
int mont_from_domain(mont_ctx_t ctx, const void* y, void* out, size_t n, void* stream);

/* --------------------------------------------------- host-buffer pipeline */
/*
 * The element-wise operations above on vectors that live in HOST memory.
 * The paper has no counterpart (it states the reductions, not where their
 * operands live); this is the library's transfer layer.
 *
 * A pipe owns one device staging buffer, cut into MONT_PIPE_SLOTS fixed
 * slots, and three CUDA streams.  mont_pipe_run splits the element range
 * into chunks and, for chunk c in slot c mod MONT_PIPE_SLOTS, copies the
 * chunk of every distinct input to the device, runs every operation on it
 * with the element-wise kernels above and copies every result chunk back, so
 * that host-to-device copies, kernels and device-to-host copies of
 * consecutive chunks overlap.  An input that several operations name (the
 * same host address, element size and length) is copied once per chunk.
 * The results are bit-identical to the device-pointer entry points.
 */
#define MONT_PIPE_SLOTS    3    /* chunks in flight                              */
#define MONT_PIPE_MAX_OPS  256  /* operations in one mont_pipe_run               */
#define MONT_PIPE_MIN_CHUNK 256 /* smallest chunk, in elements                   */

/* The operation of one mont_host_op. */
#define MONT_OP_MUL         0   /* out = reduce(a b)          (mont_mul)          */
#define MONT_OP_REDC        1   /* out = reduce(a), a double-width (mont_redc)    */
#define MONT_OP_TO_DOMAIN   2   /* out = to(a)                (mont_to_domain)    */
#define MONT_OP_FROM_DOMAIN 3   /* out = from(a)              (mont_from_domain)  */

typedef struct mont_host_op {
  mont_ctx_t ctx;   /* any ctx (word or multi-limb); fixes the element size e   */
  int op;           /* MONT_OP_*                                                  */
  const void* a;    /* HOST pointer: n elements of e bytes (2e for MONT_OP_REDC)  */
  const void* b;    /* HOST pointer: n elements of e bytes (MONT_OP_MUL only)     */
  void* out;        /* HOST pointer: n elements of e bytes                        */
  size_t n;         /* elements; 0 skips the operation                            */
} mont_host_op;

typedef struct mont_pipe* mont_pipe_t;

/*
 * mont_pipe_create -- a pipe on the current device with `staging_bytes` of
 * device memory (split into MONT_PIPE_SLOTS equal slots).  MONT_EINVAL if
 * out is NULL or staging_bytes < MONT_PIPE_SLOTS * 64 KiB; MONT_ENOMEM if the
 * staging memory cannot be allocated; MONT_ECUDA if a stream or event
 * cannot be created.
 */
int mont_pipe_create(mont_pipe_t* out, size_t staging_bytes);

/*
 * mont_pipe_run -- run `count` operations on host vectors.
 *
 * Ordering: the pipe's work starts after all work enqueued on `stream`
 * before the call, and `stream` waits for the last result copy, so a later
 * call or mont_sync(stream) sees every result in host memory.  The call
 * itself only enqueues (it returns before the copies finish); the host
 * buffers must stay valid, and the inputs unmodified, until `stream` has
 * passed that point.  Calls on one pipe are serialised by an internal lock;
 * back-to-back calls on one pipe reuse its slots safely without a
 * synchronisation in between.
 *
 * Host memory: page-locked (pinned) memory gives overlapped copies in both
 * directions; pageable memory gives the same results but copies that do not
 * overlap.
 *
 * Chunk C: the largest multiple of MONT_PIPE_MIN_CHUNK elements for which one
 * chunk of every distinct input and every output fits one slot, capped so
 * that one chunk of the widest vector is at most 16 MiB.
 *
 * Errors (nothing is enqueued): MONT_EINVAL if pipe or ops is NULL, count is
 * outside 0..MONT_PIPE_MAX_OPS, an operation has a NULL ctx or pointer or an
 * unknown op code; MONT_EINVAL too if an output range
 * overlaps an input range or another output range in host memory, or if the
 * current device is not the pipe's; MONT_ENOMEM if one slot cannot hold
 * MONT_PIPE_MIN_CHUNK elements of every vector.  MONT_ECUDA if enqueueing
 * fails part-way, or the status of an operation's own mont_* call if that
 * fails part-way: no further chunk is started, `stream` still waits for what
 * was enqueued, and the host outputs of the run are unspecified.  count = 0
 * is a no-op.
 */
int mont_pipe_run(mont_pipe_t pipe, const mont_host_op* ops, int count, void* stream);

/* Chunk (elements) and number of distinct inputs mont_pipe_run would use for
 * these operations (no work enqueued); errors as mont_pipe_run's argument
 * checks. */
int mont_pipe_plan(mont_pipe_t pipe, const mont_host_op* ops, int count, size_t* chunk,
                   int* distinct_inputs);

/* Wait for the pipe's streams, then free its staging memory, streams and
 * events.  NULL is accepted. */
int mont_pipe_destroy(mont_pipe_t pipe);

/* -------------------------------------------- fixed multipliers (Plantard) */
/*
 * Section 3.2: Plantard's reduction lets a fixed multiplier b be prepared once
 * as b' = b N^{-1} mod R (R = 2^{2n}); the reduction of a b then needs only
 * m = a b' mod R, a word-by-double-word low product of which one word is
 * used, instead of T = a b and T N^{-1} mod R.  Plantard-family contexts at
 * word widths only (MONT_EINVAL otherwise).
 *
 * mont_const_prepare -- b_pre[i] = b[i] N^{-1} mod R.  b: device array of n
 *   ctx elements in the variant's input range; b_pre: device array of n double
 *   words (uint64_t at 32 bits; two little-endian uint64_t at 64 bits),
 *   aligned to its double-word size.  Asynchronous.
 * mont_mul_pre -- out[i] = the variant's reduction of a[i] b[i], using b_pre:
 *   bit-identical to mont_mul(a, b).  out may alias a exactly; b_pre must not
 *   overlap a or out.  Asynchronous.
 */
int mont_const_prepare(mont_ctx_t ctx, const void* b, void* b_pre, size_t n, void* stream);
int mont_mul_pre(mont_ctx_t ctx, const void* a, const void* b_pre, void* out, size_t n,
                 void* stream);

/* ------------------------------------------------------- lazy reduction */
/*
 * mont_dot_lazy -- out[j] = SigPRedc2(sum_{i<k} a[j k + i] b[j k + i]): row dot
 * products reduced once each with Algorithm 4, which Section 3.3 proves
 * correct for |T| <= 2^{2 alpha} N^2 (alpha >= 1).  With inputs in the mods-N
 * range each product has |a b| <= N^2/4, so any k <= 4^{alpha+1} keeps the
 * sum within that bound; the result is -(sum a b) R^{-1} mods N.
 *
 *   ctx   MONT_SIGNED_PLANTARD2 at 32- or 64-bit words (its alpha sets the
 *         largest k); MONT_EINVAL otherwise or when k = 0 or k > 4^{alpha+1}.
 *   a, b  device arrays of rows * k elements, row-major; out: device array of
 *         `rows` elements, not overlapping a or b.  Asynchronous.
 */
int mont_dot_lazy(mont_ctx_t ctx, const void* a, const void* b, void* out, size_t rows,
                  uint32_t k, void* stream);

/* ------------------------------------------------------------------ NTT */
/*
 * Batched negacyclic number-theoretic transform over Z_N, the application the
 * paper gives for word-size Montgomery-type reductions (Section 1); each
 * butterfly's twiddle product is a REDC product with the twiddle in
 * Montgomery form, or a Plantard product with the twiddle in the prepared
 * form of Section 3.2, so the data stays in the plain representation.
 *
 *   forward: A[i] = sum_j a[j] psi^{(2 brv(i) + 1) j} mod N   (bit-reversed output)
 *   inverse: a[j] = n^{-1} sum_i A[i] psi^{-(2 brv(i) + 1) j} mod N
 *
 * with n = 2^log2n, brv the log2n-bit reversal and psi a primitive 2n-th root
 * of unity mod N (psi^n = -1 mod N).
 *
 * mont_ntt_create -- plan for ctx (MONT_REDC or MONT_PLANTARD, 32- or 64-bit
 *   words), 5 <= log2n <= 10, psi as ctx->n_limbs little-endian 32-bit limbs.
 *   Builds the twiddle tables on the host and copies them to a device
 *   allocation owned by the plan (synchronous).  MONT_EINVAL when psi^n != -1
 *   mod N or the parameters are unsupported.  The plan copies the ctx's
 *   constants; the ctx may be destroyed afterwards.
 * mont_ntt_forward / mont_ntt_inverse -- transform `batch` polynomials of n
 *   coefficients in [0, N), stored one after another (polynomial p occupies
 *   elements [p n, (p+1) n)); device pointers; in == out allowed (in place),
 *   partial overlap refused.  Asynchronous on `stream`.
 * mont_ntt_destroy -- free the plan (NULL accepted); work already enqueued
 *   must have completed.
 */
typedef struct mont_ntt* mont_ntt_t;
int mont_ntt_create(mont_ntt_t* out, mont_ctx_t ctx, int log2n, const uint32_t* psi_limbs);
int mont_ntt_forward(mont_ntt_t plan, const void* in, void* out, size_t batch, void* stream);
int mont_ntt_inverse(mont_ntt_t plan, const void* in, void* out, size_t batch, void* stream);
int mont_ntt_destroy(mont_ntt_t plan);

/* ------------------------------------------------ RNS <-> big integers */
/*
 * Conversions between big integers and their residues modulo pairwise coprime
 * odd moduli p_0 .. p_{count-1} (the multi-modulus CRT, which Section 2
 * derives for two moduli from Qin's identity, Eq. (2), and states extends).
 *
 * mont_rns_create -- host array of `count` (1..64) odd, pairwise coprime
 *   moduli, 3 <= p < 2^63, with product P < 2^2047.  Precomputes the Montgomery
 *   constants (R = 2^64), M_i = P / p_i with M_i^{-1} mod p_i, and floor(2^128 /
 *   p_i), copied to a device allocation owned by the object (synchronous).
 *   MONT_EINVAL otherwise.
 * mont_rns_query -- number of moduli, and `limbs`: the 32-bit limbs of every
 *   big integer these calls read or write (8, 16, 32 or 64: the least with
 *   32 limbs > the bits of P).
 * mont_rns_to_residues -- residues[i n + e] = X_e mod p_i for n big integers X
 *   (element e at X[e limbs .. (e+1) limbs), little-endian, any value below
 *   2^(32 limbs)).  X 16-byte aligned, residues 8-byte aligned, not
 *   overlapping; device pointers; asynchronous.
 * mont_rns_from_residues -- X_e = the unique integer in [0, P) with
 *   X_e = residues[i n + e] (mod p_i) for all i; residues must lie in [0, p_i).
 *   Same layout rules; asynchronous.
 * mont_rns_destroy -- free the object (NULL accepted).
 */
typedef struct mont_rns* mont_rns_t;
int mont_rns_create(mont_rns_t* out, const uint64_t* moduli, int count);
int mont_rns_query(mont_rns_t rns, int* count, int* limbs);
int mont_rns_to_residues(mont_rns_t rns, const uint32_t* X, uint64_t* residues, size_t n,
                         void* stream);
int mont_rns_from_residues(mont_rns_t rns, const uint64_t* residues, uint32_t* X, size_t n,
                           void* stream);
int mont_rns_destroy(mont_rns_t rns);

/* ---------------------------------------------------------- batched RNS */
/*
 * mont_mul_batched -- many independent mont_mul problems in one persistent
 * launch: for each j in [0, count), out[j][i] = reduce(a[j][i] * b[j][i]) for
 * i in [0, lens[j]) with the modulus, variant and constants of ctxs[j]
 * (Section 1 / Algorithms 1-4, as mont_mul).  This is the residue-number-system
 * pattern: one vector per modulus, lengths as uneven as the caller likes.
 *
 *   ctxs, a, b, out, lens  host arrays of `count` entries; a[j], b[j], out[j]
 *          are device pointers with mont_mul's rules (element alignment, in
 *          place allowed, no partial overlap).  lens[j] = 0 is allowed (the
 *          pointers of that entry are then ignored).
 *   Every ctx must have the same word width, 32 or 64 (multi-limb contexts
 *   are refused); variants may differ.  Asynchronous on `stream`.  Vectors of
 *   up to 128 moduli go into one launch; larger batches take one launch per
 *   128.  No device memory is allocated: the per-modulus constants travel in
 *   the launch's parameters and are staged in shared memory.
 * Errors: MONT_EINVAL on mixed widths, NULL or misaligned pointers.
 */
int mont_mul_batched(const mont_ctx_t* ctxs, const void* const* a, const void* const* b,
                     void* const* out, const size_t* lens, int count, void* stream);

/*
 * A batch plan: the launches of mont_mul_batched for one fixed set of
 * (ctx, length) pairs, recorded once in a CUDA graph and replayed with a single
 * graph launch.  The plan copies everything it needs; ctxs may be destroyed
 * after mont_batch_create returns.
 *
 * mont_batch_create  -- same arguments and rules as mont_mul_batched (host
 *                       arrays; device operand pointers); builds and
 *                       instantiates the graph on the current device.
 * mont_batch_launch  -- enqueue the graph on `stream` (asynchronous).  A plan
 *                       must not be launched concurrently with itself
 *                       while its pointers are being updated.
 * mont_batch_update  -- replace the operand pointers (host arrays of `count`
 *                       device pointers; entries with length 0 are ignored);
 *                       shapes stay fixed.  Affects later launches only.
 * mont_batch_destroy -- free the plan (NULL accepted); launches already
 *                       enqueued complete normally.
 */
typedef struct mont_batch* mont_batch_t;
int mont_batch_create(mont_batch_t* out_batch, const mont_ctx_t* ctxs, const void* const* a,
                      const void* const* b, void* const* out, const size_t* lens, int count);
int mont_batch_launch(mont_batch_t batch, void* stream);
int mont_batch_update(mont_batch_t batch, const void* const* a, const void* const* b,
                      void* const* out);
int mont_batch_destroy(mont_batch_t batch);

/* ------------------------------------------------------- verify sweep */
/*
 * The exhaustive check of Section 3: for every odd N in [N_lo, N_hi] and every T
 * of a domain, evaluate the variant's algorithm (REDC of Section 1, Algorithms
 * 1-4) exactly as written, at R = 2^log2R, and count T whose output r is a
 * counterexample to the claim derived from Eq. (5):
 *     r != s T R^{-1} (mod N)   or   r outside the claimed range,
 * with s = +1 for REDC and Algorithm 1, s = -1 for the Plantard family.
 * Example 3.1 is such a counterexample of Algorithm 4 with alpha = 0.
 */
#define MONT_DOMAIN_DEFAULT   0  /* the algorithm's own Require line (inclusive bounds)        */
#define MONT_DOMAIN_REDC      1  /* 0 <= T < R N, Section 1's domain, for every variant        */
#define MONT_DOMAIN_EXPLICIT  2  /* t_lo <= T <= t_hi for every N                             */
#define MONT_RANGE_DEFAULT    0  /* the algorithm's own Ensure line                           */
#define MONT_RANGE_UNSIGNED   1  /* 0 <= r <= N-1                                             */
#define MONT_RANGE_WIDE       2  /* -(N-1) <= r <= N-1                                        */
#define MONT_RANGE_CENTRED    3  /* -(N-1)/2 <= r <= (N-1)/2                                  */
#define MONT_RANGE_EXPLICIT   4  /* r_lo <= r <= r_hi for every N                             */

typedef struct mont_bounds {
  int domain_rule;   /* MONT_DOMAIN_*                                  */
  int range_rule;    /* MONT_RANGE_*                                   */
  int64_t t_lo, t_hi; /* used by MONT_DOMAIN_EXPLICIT (inclusive)      */
  int64_t r_lo, r_hi; /* used by MONT_RANGE_EXPLICIT (inclusive)       */
} mont_bounds;

typedef struct mont_cex {  /* one counterexample                        */
  uint32_t N;
  uint32_t reserved;
  int64_t T;
  int64_t r;         /* the algorithm's output                          */
  int64_t expected;  /* the canonical target: s T R^{-1} mod N (REDC, Algorithm 2)
                        or mods N (Algorithms 1, 3, 4)                   */
} mont_cex;

#define MONT_SWEEP_INCLUDE_OUT_OF_SPEC 1  /* also sweep N that violate the variant's
                                             condition on N (skipped by default) */

/* Limits of the sweep: 2 <= log2R <= 16 (even for the Plantard family);
 * 3 <= N_lo <= N_hi < 2^15; every swept T and every claimed bound within
 * [-2^31, 2^31 - 1]; 0 <= alpha <= 14.  These keep every intermediate of the
 * algorithms inside a 32-bit register (64-bit for REDC's T + mN). */
#define MONT_SWEEP_MAX_LOG2R 16
#define MONT_SWEEP_MAX_N     32767

/*
 * mont_verify_sweep -- run the sweep on the device and return its results on
 * the host.  Synchronous: returns after the results are copied back.
 *
 *   variant, log2R, alpha  the algorithm under test and its R = 2^log2R; alpha
 *                  (Algorithm 4 only) may be 0 here, unlike in mont_ctx_create.
 *   N_lo, N_hi     inclusive range; even values are skipped.
 *   claimed        host pointer to the domain and range rules, or NULL for
 *                  (MONT_DOMAIN_DEFAULT, MONT_RANGE_DEFAULT).
 *   flags          0 or MONT_SWEEP_INCLUDE_OUT_OF_SPEC.
 *   per_N_counts   host array of n_odd = number of odd N in [N_lo, N_hi]
 *                  entries, entry i for the i-th odd N: the exact number of
 *                  counterexamples (0 for skipped N).
 *   per_N_checked  host array of n_odd entries receiving the number of T
 *                  checked per N (0 for skipped N), or NULL.
 *   cex, cex_cap   host array for up to cex_cap counterexamples, sorted by
 *                  (N, T); may be NULL when cex_cap = 0.
 *   n_cex_total    host pointer receiving the total number of counterexamples.
 *   stream         the stream the sweep runs on (it is synchronised).
 *
 * Returns MONT_EOVERFLOW when n_cex_total > cex_cap: the counts are exact, and
 * cex holds cex_cap of the counterexamples (which ones is unspecified), sorted.
 * MONT_EINVAL outside the limits above; MONT_ENOMEM / MONT_ECUDA on device
 * failures.  Device scratch (the counters and the example buffer) is allocated
 * and freed on the stream by the call.
 */
int mont_verify_sweep(int variant, int log2R, int alpha, uint32_t N_lo, uint32_t N_hi,
                      const mont_bounds* claimed, int flags, uint64_t* per_N_counts,
                      uint64_t* per_N_checked, mont_cex* cex, size_t cex_cap,
                      size_t* n_cex_total, void* stream);

/*
 * mont_verify_sweep_noalloc -- mont_verify_sweep for callers that must not
 * allocate memory during the call: for example a program that sets its
 * device-memory budget once at start-up, a host whose device memory is owned
 * by another allocator, or a latency-critical loop that cannot afford the
 * implicit device synchronisation cudaMalloc may perform.  The paper has no
 * counterpart; this is a property of the library interface, not of the
 * method.
 *
 * Same arguments, results, sorting and status codes as mont_verify_sweep,
 * with two differences:
 *  - It allocates nothing, on the device or on the host.  Its device
 *    scratch is one fixed array of about 0.6 MB compiled into the library,
 *    which every GPU that loads the library keeps until the process exits.
 *    The host side writes only into the caller's buffers.
 *  - That array bounds the request: at most MONT_SWEEP_NOALLOC_MAX_MODULI odd
 *    N in [N_lo, N_hi], and cex_cap at most MONT_SWEEP_NOALLOC_MAX_CEX;
 *    larger requests return MONT_EINVAL before any GPU work.
 * Every call on a device shares the one array and it keeps the previous
 * call's contents (the call clears its counters itself), so calls whose GPU
 * work overlaps in time -- on different streams or host threads -- race and
 * must be serialised by the caller.  Each call looks up the array's device
 * address in the current device's context (cudaGetSymbolAddress, which
 * allocates nothing) and synchronises `stream` before it returns.
 */
#define MONT_SWEEP_NOALLOC_MAX_MODULI 8192
#define MONT_SWEEP_NOALLOC_MAX_CEX    4096
int mont_verify_sweep_noalloc(int variant, int log2R, int alpha, uint32_t N_lo, uint32_t N_hi,
                              const mont_bounds* claimed, int flags, uint64_t* per_N_counts,
                              uint64_t* per_N_checked, mont_cex* cex, size_t cex_cap,
                              size_t* n_cex_total, void* stream);

/* ------------------------------------------------------------- serving */
/*
 * A serving loop for a stream of independent requests (jobs): modular
 * multiplications (the paper's reductions applied with mont_mul) and
 * verify sweeps (Section 3's check), batched continuously on one GPU.
 *
 * The server owns a device arena of mem_budget_bytes and `slots` worker
 * threads, each with a high-priority CUDA stream (modmul jobs) and a
 * low-priority one (sweep jobs).  Jobs wait in two FIFO queues, modmul and
 * sweep; the job at a queue's head is admitted by the next idle worker that
 * serves that queue as soon as its device memory fits in the arena
 * (3 * n * element bytes for a modmul job; the table, counters and example
 * buffer for a sweep), so requests arriving while others run start as soon
 * as a slot and memory free up, and up to `slots` jobs overlap on the device.
 * Workers 0 .. max(1, slots/4) - 1 take sweeps first and modmul jobs
 * otherwise; the rest take modmul jobs only, so a modmul job never queues
 * behind a sweep.  A modmul job copies a and b from host memory into the
 * arena, runs mont_mul and copies the products back into `out`; pinned host
 * buffers let the copies run asynchronously.  A sweep job runs the sweep of
 * mont_verify_sweep in launches of about 2^31 checks each, so that modmul
 * jobs' kernels run between them.  Contexts stay with the caller (resident
 * across jobs).
 *
 * Every wait for the device is bounded by the job's timeout (its own
 * timeout_ms, else the server's job_timeout_ms; <= 0: 60 s).  A job past its
 * timeout completes with MONT_ETIMEOUT while its device work may still run:
 * until that work ends, its arena region stays reserved and -- for a modmul
 * job -- the device may still read a and b and write out.  The caller must
 * keep a, b, out and ctx valid until mont_server_job_busy reports 0 for the
 * job (or until mont_server_destroy has returned MONT_OK).  A timed-out sweep
 * writes none of its result buffers.
 */
#define MONT_JOB_MODMUL 0
#define MONT_JOB_SWEEP  1

typedef struct mont_job {
  int kind;                    /* MONT_JOB_MODMUL or MONT_JOB_SWEEP                     */
  /* MODMUL: out[i] = reduce(a[i] b[i]) for ctx; a, b, out HOST pointers of n elements;
   * ctx and the buffers must stay valid until the job completes (and, after
   * MONT_ETIMEOUT, until mont_server_job_busy reports 0).                                */
  mont_ctx_t ctx;
  const void* a;
  const void* b;
  void* out;
  size_t n;
  /* SWEEP: the arguments of mont_verify_sweep; the result buffers must stay valid
   * until the job completes (claimed is copied, and the request checked, at submission). */
  int variant, log2R, alpha;
  uint32_t N_lo, N_hi;
  const mont_bounds* claimed;
  int flags;
  uint64_t* per_N_counts;
  uint64_t* per_N_checked;
  mont_cex* cex;
  size_t cex_cap;
  size_t* n_cex_total;
  int timeout_ms;              /* this job's bound on device waits; <= 0: the server's  */
} mont_job;

typedef struct mont_job_result {
  int status;        /* the job's status (a sweep's MONT_EOVERFLOW is reported as MONT_OK) */
  double t_submit;   /* seconds since the server was created                       */
  double t_admit;    /* admitted to a slot                                        */
  double t_done;     /* results in host memory                                    */
} mont_job_result;

typedef struct mont_server* mont_server_t;

/* Create a server on the current device.  MONT_EINVAL for slots outside
 * 1..64 or a budget below 256 bytes; MONT_ENOMEM if the arena cannot be
 * allocated. */
int mont_server_create(mont_server_t* out, size_t mem_budget_bytes, int slots,
                       int job_timeout_ms);
/* Queue a job (copied; never blocks on the device) and return its id.
 * MONT_ENOMEM if the job alone exceeds the budget; MONT_EINVAL on bad fields
 * (for a sweep, any request mont_verify_sweep would refuse).  A job that can
 * never be admitted -- nothing running, and the memory held by timed-out jobs
 * not given back within its timeout -- completes with MONT_ENOMEM. */
int mont_server_submit(mont_server_t server, const mont_job* job, uint64_t* id);
/* Wait for job `id` (timeout_ms < 0: no limit) and retrieve its result; the
 * id is then forgotten.  MONT_ETIMEOUT if it is not done in time (it can be
 * waited for again); MONT_EINVAL for an unknown or already retrieved id. */
int mont_server_wait(mont_server_t server, uint64_t id, int timeout_ms, mont_job_result* res);
/* *busy = 1 while job `id` timed out and its device work may still use its
 * buffers (see above), else 0; valid before and after mont_server_wait. */
int mont_server_job_busy(mont_server_t server, uint64_t id, int* busy);
/* Snapshot: jobs queued, jobs running, free arena bytes, server clock. */
int mont_server_query(mont_server_t server, size_t* queued, size_t* running,
                      size_t* arena_free, double* now_s);
/* Finish every queued job, stop the workers, wait (per stream, at most twice
 * the job timeout) for the device work of timed-out jobs and free the server.
 * MONT_ETIMEOUT if that work did not end: the arena is then left allocated
 * (the device may still write it) and the buffers of those jobs stay in use. */
int mont_server_destroy(mont_server_t server);

/* ------------------------------------------------------------ autotuner */
/*
 * Launch shapes.  Every kernel family has a few launch knobs; a per-process
 * table maps (current device, word width in bits, variant, mode) to a shape,
 * and entries that are not set use built-in defaults.  Shapes change speed
 * only, never results.
 */
typedef struct mont_launch_shape {
  int threads;        /* threads per block: 64..512 (word kernels), 32, 64, 128 or 256
                         (multi-limb), 128 or 256 (batched); multi-limb REDC reports 0
                         when untuned: the block size then follows the element count */
  int unroll;         /* 256-bit vectors in flight per thread per operand: 1, 2 or 4      */
  int vec_bytes;      /* word kernels: 32, 16 or 0 (scalar loads)                         */
  int blocks_per_sm;  /* resident blocks per SM the grid is sized for; 0 = occupancy max   */
  int tile_iters;     /* reserved; keep 0                                                   */
  int team;           /* multi-limb REDC: lanes per element (1, 2, 4, 8, 16); 0 = default;
                         the other multi-limb variants run one thread per element      */
} mont_launch_shape;

#define MONT_TUNE_MODE_MUL          0  /* mont_mul (also used by the other modes when tuned) */
#define MONT_TUNE_MODE_TO_DOMAIN    1
#define MONT_TUNE_MODE_FROM_DOMAIN  2
#define MONT_TUNE_MODE_REDC         3
#define MONT_TUNE_MODE_BATCHED     (-1)  /* mont_mul_batched; variant is ignored */

/* Set (or, with shape = NULL, clear) the shape of one table entry for the
 * current device.  MONT_EINVAL for out-of-range knobs. */
int mont_tune_set(int width_bits, int variant, int mode, const mont_launch_shape* shape);
/* The shape the library would use now for that entry (defaults filled in). */
int mont_tune_get(int width_bits, int variant, int mode, mont_launch_shape* shape);

#define MONT_TUNE_ELEMENTWISE 1  /* tune mont_mul and the domain maps of ctx's width/variant */
#define MONT_TUNE_BATCHED     2  /* tune mont_mul_batched for ctx's word width             */

/*
 * mont_autotune -- time every candidate shape on n elements of ctx's type,
 * with CUDA events on `stream`, and record the fastest in the table.
 * Allocates 3 n elements of device scratch on `stream` and frees it before
 * returning; synchronous.  Timing uses arbitrary operand bits, which is safe:
 * the kernels have no data-dependent memory access.
 */
int mont_autotune(mont_ctx_t ctx, size_t n, int flags, void* stream);

/* Persist the current device's table entries to a text file / load the
 * entries of a file whose device name and SM count match the current device
 * (others are ignored).  MONT_EINVAL on I/O or format errors. */
int mont_tune_save(const char* path);
int mont_tune_load(const char* path);

/* ----------------------------------------------------------------- probe */
/*
 * mont_probe_int_rate -- measured integer throughput of the current GPU for
 * the instruction mixes of the multi-limb kernels and the sweep: kind 0
 * mad.lo.u32, 1 mad.hi.u32, 2 mad.lo.cc + madc.hi pairs (the high product
 * dependent on the low one; counted as two), 3 add.u32, 4 mad.wide.u32 (one
 * 32x32->64 multiply-add), 5 a mad.lo.u32 and a mad.hi.u32 on independent
 * accumulators (counted as two).  A full-occupancy grid runs `iters`
 * iterations of 8 independent chains per thread; *ops_per_s receives
 * instructions per second (thread instructions).  MONT_EINVAL for another
 * kind.  Synchronous on `stream`.  Measurement support: the paper has no
 * counterpart.
 */
int mont_probe_int_rate(int kind, int iters, void* stream, double* ops_per_s);

/* ------------------------------------------------------------- utilities */
/* Static description of a status code; never NULL. */
const char* mont_strerror(int status);
/* CUDA error code (cudaError_t as int) of the last MONT_ECUDA on this thread. */
int mont_last_cuda_error(void);
/* cudaStreamSynchronize(stream); MONT_ECUDA on failure. */
int mont_sync(void* stream);
/* Library version as major*10000 + minor*100 + patch. */
int mont_version(void);

#ifdef __cplusplus
}
#endif
#endif /* MONTGB_H */
