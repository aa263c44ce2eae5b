/*
 * libpolymul -- exact negacyclic polynomial multiplication on GB300 (sm_103a).
 *
 * The operation (paper: "TPU as Cryptographic Accelerator", arXiv 2307.06554):
 * for operands a, b in the ring Z_q[x]/(x^n+1) (Sec. 2.1, ring and Eq.
 * equ-poly-coef: coefficient vectors a_0..a_{n-1} in Z_q) compute
 *
 *     c_j = ( sum_{i+k=j} a_i b_k  -  sum_{i+k=j+n} a_i b_k ) mod q,
 *
 * i.e. the product in Z[x] reduced by x^n = -1 (Sec. 2.2 fold rule) and taken
 * mod q, which is the row vector a times the negacyclic matrix of b of
 * Eq. equ-genereal-mat.  Results are canonical residues in [0, q) and are
 * bit-exact: no floating-point rounding can reach them.  With
 * POLYMUL_FLAG_CYCLIC the ring is Z_q[x]/(x^n-1), the other ring Sec. 2.1
 * names: x^n = 1, so the second sum is added, and the matrix is the
 * circulant of b (Sec. 2.5 notes that the matrix form adapts to the modulus).
 *
 * Algorithm 1 of the paper maps onto this interface as follows:
 * GenConfig / ExtractModuli / ExtractDimensions  ->  polymul_create
 * ConvertPoly / TPUMul / ConvertMatrix            ->  inside polymul_batch.
 * Several moduli ("RNS primes", Sec. 2.4, where residues are kept until they
 * are needed) are handled as independent rings of the same n.
 *
 * Conventions for every call below.
 *  - Data layout: operand and result arrays are C-contiguous
 *    [batch][k][n] (product, prime, coefficient) with coefficients
 *    contiguous.  Entry (p, j, i) belongs to the ring with modulus q_list[j].
 *    Inputs must be canonical (in [0, q_j)); behaviour for larger inputs is
 *    unspecified unless POLYMUL_FLAG_VALIDATE is set.
 *  - Element type: uint32_t when every modulus of the plan is < 2^32,
 *    otherwise uint64_t (query with polymul_plan_info).
 *  - Ownership: the caller owns a, b and c; the plan owns its tables and any
 *    staging memory.  c must not overlap a or b.
 *  - Streams: `stream` is a cudaStream_t passed as void* (NULL = the legacy
 *    default stream).  Device-pointer calls are asynchronous with respect to
 *    the host; results are visible once the stream has been synchronised.
 *  - Errors: every int-returning call returns POLYMUL_OK (0) or one of the
 *    codes below; polymul_last_error() gives a message for the calling
 *    thread's most recent failure.  A failing call has no other effect.
 *  - Threads: distinct plans may be used concurrently from different
 *    threads; one plan must not be used by two threads at once.
 */
#ifndef POLYMUL_H
#define POLYMUL_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ---- */
#define POLYMUL_OK        0
#define POLYMUL_EINVAL    1  /* bad argument: n, q, k, null pointer, size   */
#define POLYMUL_ENOTSUP   2  /* valid request this build cannot serve        */
#define POLYMUL_EDOMAIN   3  /* validate flag set and an input is >= q       */
#define POLYMUL_ENOMEM    4  /* device or host allocation failed             */
#define POLYMUL_ETIMEOUT  5  /* a bounded device wait gave up                */
#define POLYMUL_ECUDA     6  /* CUDA runtime error (message has the detail)  */

/* ---- computation paths ---- */
#define POLYMUL_PATH_AUTO    0  /* pick the fastest exact path (tuned)        */
#define POLYMUL_PATH_NTT     1  /* path (a): number-theoretic transform       */
#define POLYMUL_PATH_TENSOR  2  /* path (b): Toeplitz matrix on tensor cores  */

/* ---- flags ---- */
#define POLYMUL_FLAG_VALIDATE 1u  /* check that inputs are < q (slower)       */
#define POLYMUL_FLAG_TUNE     2u  /* time the candidate kernels at creation    */
#define POLYMUL_FLAG_CYCLIC   4u  /* the ring Z_q[x]/(x^n - 1) instead of
                                     Z_q[x]/(x^n + 1) (Sec. 2.1 names it as the
                                     other common ring): the NTT path then needs
                                     q = 1 mod n; every path supports it      */
#define POLYMUL_FLAG_TERNARY_B 8u /* every coefficient of b is 0, 1 or q - 1
                                     (a ternary polynomial lifted mod q, as the
                                     secrets and errors of lattice schemes):
                                     the tensor path splits b into a single
                                     digit and computes c = b * T(a), one MMA
                                     chain per block instead of L.  The NTT
                                     path ignores it.  A tensor-path launch
                                     that meets a b coefficient whose centred
                                     value does not fit one digit leaves its
                                     results invalid and makes
                                     polymul_plan_status return EDOMAIN     */
#define POLYMUL_FLAG_OVERLAP 16u  /* let a batch on the NTT path start before
                                     the previous kernel on its stream has
                                     finished, when that kernel is a batch
                                     launch of this library (any plan) that
                                     writes none of this batch's operands and
                                     reads or writes none of its results: the
                                     new batch loads and multiplies its first
                                     products while the previous one drains,
                                     so back-to-back batches do not each pay
                                     a fill and a drain.  Results and stream
                                     order are otherwise unchanged.  The
                                     caller guarantees one thing the library
                                     cannot see: no kernel of the caller's
                                     own that lets its dependents start early
                                     (programmatic dependent launch) is
                                     enqueued right before a batch and
                                     produces that batch's a or b.  Ignored
                                     on the legacy and per-thread default
                                     streams                                */

#define POLYMUL_FLAG_HOST_STAGED 32u /* polymul_batch_host always streams
                                     through the plan's device staging
                                     buffers and copy engines, never takes
                                     its direct route (see there)           */

typedef struct polymul_opts {
    uint32_t path;        /* POLYMUL_PATH_*                                   */
    uint32_t flags;       /* POLYMUL_FLAG_*                                   */
    uint32_t tune_batch;  /* batch size to tune for (0: 1024)                 */
    uint32_t reserved[5];
} polymul_opts;

typedef struct polymul_plan_info {
    uint32_t n;
    uint32_t k;
    uint32_t elem_bytes;  /* 4 (uint32_t) or 8 (uint64_t)                     */
    uint32_t path;        /* the path actually used (NTT or TENSOR)           */
    uint32_t aux_primes;  /* NTT only: number of auxiliary primes (0 = direct)*/
    uint32_t block;       /* threads per CTA of the main kernel               */
    uint32_t grid;        /* CTAs of the main kernel (persistent grid)        */
    uint32_t smem_bytes;  /* dynamic shared memory per CTA                    */
    uint32_t ctas_per_sm; /* resident CTAs per SM of the main kernel          */
    uint32_t digit_bits;  /* tensor path: digit width w (0 for NTT plans)     */
    uint32_t digits;      /* tensor path: digits per coefficient L            */
    uint32_t radix_bits;  /* NTT path: stage bits per register pass           */
    uint32_t candidates;  /* kernels the autotuner chooses among              */
    uint32_t tuned;       /* 1 once polymul_tune has chosen                   */
    uint32_t tuned_batch; /* batch bucket of that choice (0: not tuned)       */
    uint32_t launch_flags;/* bit 1: the main kernel takes a programmatic
                             dependent launch (its CTAs start as the previous
                             kernel on the stream drains and wait for it to
                             complete before touching memory); set for the
                             NTT batch kernels.  Bit 2: POLYMUL_FLAG_OVERLAP
                             is in effect for it                            */
    uint32_t ntt_mode;    /* NTT path: reduction mode of the main kernel:
                             0 = values in [0, 2q), 1 = [0, 4q) (Harvey),
                             2 = unreduced (small q)                        */
    uint32_t regs;        /* NTT path: register budget per thread of the main
                             kernel (fewer registers, more resident warps)  */
    uint32_t cyclic;      /* 1: the ring Z_q[x]/(x^n-1); 0: Z_q[x]/(x^n+1) */
    uint32_t tensor_groups;/* tensor path: 0 for the whole-product kernel
                             (n = 1024, 2048); else the tiled or RNS
                             kernel's units of work per (product, prime):
                             output groups of up to 1024 coefficients each  */
    uint32_t rns_moduli;  /* tensor path, RNS kernel: small moduli in the
                             base (0 for the digit kernels)                 */
    uint32_t exchange_pad;/* NTT path: shared-memory exchange layout of the
                             main kernel: 0 = XOR swizzle, s > 0 = one
                             padding word after every 2^s words             */
    uint32_t one_operand; /* NTT path: 1 when the main kernel holds one
                             operand in registers at a time (a's transform
                             parked in shared memory during b's)            */
    uint32_t tensor_kernel;/* tensor path: the main kernel, coded as
                             polymul_tensor_shape_info.kernel (1 whole
                             product, 2 tiled, 3 RNS, 4 tiled drained, 5
                             tiled drained warp-specialised)                 */
    uint32_t kernel_regs;  /* registers per thread the main kernel was
                             compiled to (from the CUDA runtime)            */
    uint32_t kernel_max_block;/* the largest CTA the main kernel can launch
                             with (from the CUDA runtime)                   */
    uint32_t host_direct; /* polymul_batch_host calls on this plan that took
                             the direct route (saturates at 2^32 - 1)       */
} polymul_plan_info;

typedef struct polymul_plan polymul_plan; /* opaque, owned by the library */

/*
 * polymul_create -- build a plan for products in Z_q[x]/(x^n+1) (or in
 * Z_q[x]/(x^n-1) with POLYMUL_FLAG_CYCLIC) for each q of q_list
 * (Algorithm 1, GenConfig: parameters are fixed here, once).
 *   n       power of two, 16 <= n <= 65536.
 *   q_list  k moduli, each 2 <= q < 2^62, pairwise distinct (host memory,
 *           read during the call only).
 *   opts    NULL for defaults (PATH_AUTO, no flags).
 *   out     receives the plan; untouched on failure.
 * Device tables (roots of unity, constants) are computed and uploaded on the
 * current CUDA device; the plan must be used on that device.
 * Routes (PATH_AUTO takes the NTT where it exists; the tensor kernels are
 * then autotuner candidates):
 *   NTT      prime q = 1 mod 2n (mod n for the cyclic ring), q < 2^31 in
 *            4-byte words or q < 2^62 in 8-byte words; else, for q < 2^31
 *            and n <= 2^14, one 31-bit auxiliary prime when 2n floor(q/2)^2
 *            fits it.
 *   TENSOR   (the matrix form, Sec. 2.2) n = 2^6 .. 2^14 for q < 2^31:
 *            balanced bf16 digits, at most five digits whose fp32 sums
 *            stay exact over the whole of K (whole-product kernel at
 *            n = 1024, 2048, tiled kernel at every n), or four 8-bit digits
 *            whose sums are drained into 64-bit integers after every K
 *            chunk of at most 1024 (also as a warp-specialised pipeline);
 *            64-bit words at n = 2^10 .. 2^16: five to eight drained 8-bit
 *            digits; the residue number system of small moduli for any
 *            q < 2^62 whose base needs at most 32 moduli
 *            (polymul_tensor_rns_base).  polymul_plan_info reports which
 *            kernel a plan holds (tensor_kernel).
 * Errors: EINVAL (n, q, k, duplicates, null out), ENOTSUP (no path can serve
 * the moduli at this n, or a forced path cannot), ENOMEM, ECUDA.
 */
int polymul_create(uint32_t n, const uint64_t *q_list, uint32_t k,
                   const polymul_opts *opts, polymul_plan **out);

/*
 * polymul_batch -- c = a*b for `batch` products (each with all k moduli).
 *   a, b, c  device pointers, [batch][k][n] of the plan's element type,
 *            16-byte aligned.  batch == 0 is a no-op.
 *   stream   cudaStream_t or NULL.
 * Asynchronous.  The tensor path's residue-number-system kernel keeps
 * residue planes in plan-owned scratch, allocated (or grown) on the first
 * call with a larger batch: make one such call before capturing the stream
 * into a CUDA graph.  Errors: EINVAL (null pointers with batch > 0,
 * misaligned), EDOMAIN (validate flag and an input >= q; c is then
 * unspecified), ENOMEM (scratch), ECUDA.
 */
int polymul_batch(polymul_plan *plan, const void *a, const void *b, void *c,
                  uint64_t batch, void *stream);

/*
 * polymul_batch_shared -- c_i = a * b_i (i < batch) for one operand a shared
 * by every product: the paper's many-vector batching (Sec. 2.2: one matrix
 * times many vectors is one matrix product).
 *   a        device pointer, [k][n] (one polynomial per modulus).
 *   b, c     device pointers, [batch][k][n].  All 16-byte aligned.
 * The plan's path decides how:
 *   tensor path: with c_i = b_i * T(a) the batch is the GEMM
 *     C = B * T(a) (M = batch, N = K = n), every digit pair in tensor memory;
 *     needs 2 digits per coefficient (n = 1024 with q < 2^15, n = 2048 with
 *     q < 2^14);
 *   NTT path: a's transform once per modulus, then one forward and one
 *     inverse transform per product (instead of two forward and one
 *     inverse); needs 32-bit words, 1024 <= n <= 8192, a direct NTT.
 * The cyclic flag is honoured.  The plan keeps scratch (digit planes of b
 * and T(a), or a's transforms), grown (cudaMalloc) when a call needs more.
 * Asynchronous; a call must not overlap another call on the same plan (they
 * share the scratch).
 * Errors: EINVAL (pointers, alignment, batch > 2^32), ENOTSUP (a plan
 * outside the cases above), ENOMEM, ECUDA.
 */
int polymul_batch_shared(polymul_plan *plan, const void *a, const void *b, void *c,
                         uint64_t batch, void *stream);

/*
 * polymul_batch_host -- as polymul_batch with HOST arrays a, b, c (layout as
 * there).  Two routes, both overlapping the transfer of operands and
 * results with the arithmetic (Sec. 4, "optimizing computation and I/O"):
 *   direct: when polymul_batch_mapped accepts the call (a, b and c in
 *     mapped page-locked host memory, an NTT plan it serves) and the plan
 *     lacks POLYMUL_FLAG_HOST_STAGED: that call on `stream`, then a
 *     synchronisation of `stream`.
 *   staged: otherwise the library streams chunks through plan-owned device
 *     buffers, overlapping the host-to-device copy of one chunk with the
 *     kernel of another and with the device-to-host copy of a third.
 *     Page-locked memory gives full overlap; pageable memory works but
 *     copies synchronously.
 * polymul_plan_info.host_direct counts the calls that took the direct
 * route.  Returns after c has been written (synchronous).  Calls on one plan
 * must not overlap.
 */
int polymul_batch_host(polymul_plan *plan, const void *a, const void *b, void *c,
                       uint64_t batch, void *stream);

/*
 * polymul_batch_mapped -- as polymul_batch with a, b and c in page-locked
 * HOST memory that the device maps (cudaHostAlloc, cudaHostRegister or a
 * page-locked allocator; each range is checked at both ends with
 * cudaPointerGetAttributes).  The NTT batch kernel, in its direct form,
 * loads every row of a and b and stores every row of c in host memory
 * itself: on a coherent host link (NVLink-C2C) the operands travel in and
 * the results out at the same time, inside the kernel, with no staging
 * buffer or copy engine (Sec. 4, overlapping computation with I/O).  The
 * operands cross the link at every call; nothing of them stays on the
 * device.
 *   a, b, c  host pointers (as the device sees them with unified
 *            addressing), [batch][k][n], aligned to the word size; c
 *            writable by the device (not registered read-only).
 *   stream   cudaStream_t or NULL.
 * Asynchronous like polymul_batch: c holds the results once `stream` has
 * been synchronised; until then a and b must not change and c must not be
 * read.  POLYMUL_FLAG_OVERLAP lets consecutive batches on a stream overlap
 * as for polymul_batch (below the thread-block-cluster degrees);
 * POLYMUL_FLAG_VALIDATE is honoured (an extra pass over a and b,
 * synchronous).  Needs an NTT-path plan (its own primes or one auxiliary
 * prime); every degree: the batch kernel's direct form up to n = 2^14
 * (32-bit words) or 2^13 (64-bit words), the plan's thread-block-cluster
 * kernel above (it reads and writes with plain accesses already).
 * Errors: EINVAL (null pointers with batch > 0, a range that is not mapped
 * page-locked host memory, misalignment, batch > 2^40), ENOTSUP (a
 * tensor-path plan), EDOMAIN (validation), ECUDA.
 */
int polymul_batch_mapped(polymul_plan *plan, const void *a, const void *b, void *c,
                         uint64_t batch, void *stream);

/*
 * polymul_plan_status -- synchronise `stream`, then report whether a kernel
 * of this plan abandoned a bounded device wait (an asynchronous copy that
 * never completed) since the previous call.  Returns POLYMUL_ETIMEOUT in
 * that case (the outputs of the affected launches are invalid) and resets
 * the plan's device-side state so that it can be used again; else
 * POLYMUL_EDOMAIN if a tensor-path launch of a POLYMUL_FLAG_TERNARY_B plan
 * met a b coefficient that does not fit one digit (its outputs are
 * invalid); POLYMUL_OK otherwise.  Kernels never spin without a bound.
 */
int polymul_plan_status(polymul_plan *plan, void *stream);

/*
 * polymul_batch_static -- c = a*b in Z_q[x]/(x^n+1) for `batch` products of
 * one prime modulus, WITHOUT any device allocation.  (Not an operation of
 * the paper: it has no counterpart there.  It is polymul_batch's NTT kernel
 * run from library-owned fixed memory.)
 *
 * For callers that cannot allocate device memory: code running while any
 * thread of the process captures a CUDA graph in global capture mode (where
 * cudaMalloc/cudaFree are not permitted), latency-critical code that cannot
 * take the device-wide synchronisation of an allocation, and hosts whose
 * memory manager owns all device memory.  polymul_create allocates tables,
 * so these callers cannot hold a plan; this call needs none.
 *   n      power of two, 16 <= n <= 4096 (the fixed memory's limit).
 *   q      prime, q < 2^31, 2n | q - 1 (an NTT-friendly modulus).
 *   a,b,c  device pointers, [batch][n] uint32_t, 16-byte aligned, canonical
 *          inputs; the caller owns and provides them.
 * The library keeps the twiddle tables, constants and the kernel's work
 * counter in one fixed device array (64 KiB + 64 bytes) that every GPU using
 * the library holds until the process exits.  Every call shares that array:
 * calls whose kernels may overlap on the GPU race (issue them on one stream
 * or order them with events); tables are refreshed only when (n, q) changes,
 * and the work counter and error word are cleared on every call.  The first
 * call on a device looks up the array's device address; make it before any
 * stream capture.  Asynchronous like polymul_batch.  Errors: EINVAL,
 * ENOTSUP, ECUDA; a bounded device wait that expired is reported by
 * polymul_static_status.
 */
int polymul_batch_static(uint32_t n, uint64_t q, const void *a, const void *b, void *c,
                         uint64_t batch, void *stream);

/*
 * polymul_static_status -- synchronise `stream`, then report whether the
 * kernel of the most recent polymul_batch_static call on the current device
 * abandoned a bounded device wait (POLYMUL_ETIMEOUT: its results are
 * invalid; the word is cleared).  Call it after that call and before the
 * next one (each call clears the word).  Allocates nothing, like the call
 * it checks.  POLYMUL_OK when no call has run on the device yet.  Errors:
 * ETIMEOUT, ENOTSUP (device ordinal >= 64), ECUDA.
 */
int polymul_static_status(void *stream);

/*
 * polymul_tune -- choose the plan's kernel by measurement (the paper leaves
 * the matrix dimensions to "experimentation", Sec. 2.6): every candidate --
 * the default NTT kernel, NTT kernels with other register radices, and the
 * tensor path where it applies -- runs on a batch of `batch` products
 * (rounded up to a power of two) and the fastest is kept.  Choices are
 * cached per (GPU, word size, n, k, reduction mode, modulus size, batch
 * bucket) for the process, and in the file named by the environment
 * variable POLYMUL_TUNE_CACHE if set (read on first use, appended after each
 * new measurement).  Allocates scratch buffers for the measurement only.
 * Synchronous.  Errors: EINVAL, ENOMEM, ECUDA.
 */
int polymul_tune(polymul_plan *plan, uint64_t batch, void *stream);

/*
 * polymul_tensor_shape -- the tensor path's default kernel for degree n and
 * moduli up to qmax, as a POLYMUL_PATH_TENSOR plan with `flags` would take
 * it (POLYMUL_FLAG_TERNARY_B matters; the cyclic flag does not change the
 * shape), without creating a plan: host only, no device is touched.
 * Errors: EINVAL (n not a power of two in [16, 65536], qmax outside
 * [2, 2^62), info NULL), ENOTSUP (the tensor path has no kernel for it).
 */
typedef struct polymul_tensor_shape_info {
    uint32_t kernel;      /* 1 whole-product digit kernel, 2 tiled digit
                             kernel, 3 residue number system of small moduli,
                             4 tiled digit kernel that drains each K chunk
                             (8-bit digits at every degree), 5 the same as
                             a warp-specialised pipeline (one CTA per SM) */
    uint32_t candidates;  /* tensor kernels the plan holds (the autotuner
                             chooses among them)                            */
    uint32_t digit_bits;  /* digit kernels: digit width w (0 for the RNS one) */
    uint32_t digits_a;    /* digits of the operand on the MMA's A side (1 for
                             a ternary b, which takes that side)            */
    uint32_t digits_b;    /* digits of the operand on the B side            */
    uint32_t shifts;      /* tiled and RNS kernels: shifted copies of b that
                             share one A slice                              */
    uint32_t slices;      /* A slices (1024 outputs each) per unit of work  */
    uint32_t groups;      /* units of work per (product, prime); 0 for the
                             whole-product kernel                           */
    uint32_t rns_moduli;  /* RNS kernel: moduli in the base                 */
    uint32_t smem_bytes;  /* dynamic shared memory per CTA                  */
    uint32_t tmem_cols;   /* tensor-memory columns per CTA                  */
    uint32_t reserved[5];
} polymul_tensor_shape_info;

int polymul_tensor_shape(uint32_t n, uint64_t qmax, uint32_t flags, polymul_tensor_shape_info *info);

/*
 * polymul_tensor_rns_base -- the residue number system of small moduli that
 * the tensor path's RNS kernel uses for degree n and moduli up to qmax
 * (Sec. 2.4 and the RNS-base selection of the key-parameter section): odd,
 * pairwise coprime moduli below 2^8, the largest first, each small enough
 * that n ((m-1)/2)^2 <= 2^24 (every fp32 partial sum of centred residues
 * exact), until their product exceeds 16 n floor(qmax/2)^2.  Writes up to
 * `cap` moduli to `moduli` (may be NULL when cap is 0) and their number to
 * *count.  Host only (no device is touched).  Errors: EINVAL (n not a power
 * of two in [64, 16384], qmax < 2, count NULL), ENOTSUP (no base of at most
 * 32 moduli reaches the bound).
 */
int polymul_tensor_rns_base(uint32_t n, uint64_t qmax, uint32_t *moduli, uint32_t cap, uint32_t *count);

/* Use candidate kernel `candidate` (0 .. info.candidates - 1; 0 is the
 * default) instead of the tuned or default choice.  Errors: EINVAL. */
int polymul_plan_select(polymul_plan *plan, uint32_t candidate);

/* Fill *info with the plan's shape and launch configuration. */
int polymul_plan_info_get(const polymul_plan *plan, polymul_plan_info *info);

/* Release the plan and its device memory.  NULL is a no-op.  The caller must
 * make sure no launch of the plan is still running. */
void polymul_destroy(polymul_plan *plan);

/* ------------------------------------------------------------------------
 * Uneven batches (products of different degrees and prime counts) in
 * persistent launches.  Every modulus is a prime of a shared pool; each product
 * has its own degree n and its own subset of the pool (its RNS primes,
 * Sec. 2.4).  Operands and results live in flat caller-owned arrays of
 * uint32_t: product p occupies rows [offset, offset + k*n) laid out [k][n].
 * ---------------------------------------------------------------------- */
typedef struct polymul_ragged polymul_ragged;             /* pool + tables   */
typedef struct polymul_ragged_batch polymul_ragged_batch; /* a prepared list */

typedef struct polymul_desc {
    uint32_t n;            /* degree: power of two, 1024 <= n <= n_max        */
    uint32_t k;            /* number of primes of this product (>= 1)         */
    uint32_t prime_offset; /* its primes: prime_idx[prime_offset .. +k)       */
    uint32_t reserved;
    uint64_t offset;       /* element offset of its [k][n] rows (multiple of 4) */
} polymul_desc;

/*
 * polymul_ragged_create -- tables for a pool of primes (each prime < 2^31,
 * 2 n_max | q - 1, distinct) at the largest degree n_max (power of two in
 * [1024, 16384]); a product of degree n <= n_max uses the length-n prefix.
 * Errors: EINVAL, ENOMEM, ECUDA.
 */
int polymul_ragged_create(const uint64_t *pool, uint32_t pool_size, uint32_t n_max,
                          polymul_ragged **out);

/*
 * polymul_ragged_prepare -- plan a list of `count` products: validates every
 * descriptor (degree, prime indices < pool size, rows inside `total_elems`
 * elements of the operand arrays), flattens them into (product, prime) units
 * and sorts the units into degree segments, largest degree first (the
 * kernel's teams take the units of a segment one at a time).  The plan is
 * uploaded once and reused by every run.  Products must not overlap in c.
 */
int polymul_ragged_prepare(polymul_ragged *ctx, const polymul_desc *descs, uint32_t count,
                           const uint32_t *prime_idx, uint64_t prime_idx_len,
                           uint64_t total_elems, polymul_ragged_batch **out);

/* The whole prepared list (asynchronous, stream-ordered on `stream`): one
 * persistent launch for the degrees 2^10 .. 2^13 and one for 2^14, the
 * second forked onto a stream owned by the batch and joined back into
 * `stream` before the call returns, so that work queued on `stream` after
 * the call sees every result.  Also valid while `stream` is being captured
 * into a CUDA graph.  Errors: EINVAL (NULL, misaligned), ECUDA. */
int polymul_ragged_run(polymul_ragged_batch *batch, const void *a, const void *b, void *c,
                       void *stream);

/* The same launches as a CUDA graph of independent kernel nodes: built on
 * the first call, replayed after; new operand pointers update the recorded
 * launches in place. */
int polymul_ragged_run_graph(polymul_ragged_batch *batch, const void *a, const void *b, void *c,
                             void *stream);

/* As polymul_plan_status, for a prepared list. */
int polymul_ragged_status(polymul_ragged_batch *batch, void *stream);

/*
 * polymul_ragged_tune -- choose the kernel shapes and paths of a prepared
 * list by measurement on the caller's operands (the paper leaves such
 * dimensions to experiment, Sec. 2.6).  Each of the list's two NTT launches
 * (degrees 2^10 .. 2^13; 2^14) exists in two shape sets -- 0: swizzled
 * exchanges, both operands in registers; 1: padded exchanges, one operand
 * in registers at 2^10, 2^11 and 2^14 (the default) -- and each launch
 * keeps the faster set; then each degree class runs on the path that is
 * faster for its rows: its NTT segment alone, or the tensor path (Sec. 2.2
 * matrix form: the tiled digit kernel with 8-bit digits drained per K
 * chunk, one launch per class, behind the NTT launches).  Best of three
 * timed runs after a warm-up each.  a, b, c as for polymul_ragged_run (c is
 * overwritten with the products).  *choice (may be NULL) receives bit 0 =
 * set of the smaller degrees, bit 1 = set of 2^14, bit 2 + (log2 n - 10) =
 * degree class n on the tensor path.  A recorded graph is rebuilt on its
 * next replay.  Synchronous; returns as polymul_ragged_status afterwards.
 * Errors: EINVAL, ETIMEOUT, ECUDA.
 */
int polymul_ragged_tune(polymul_ragged_batch *batch, const void *a, const void *b, void *c,
                        void *stream, uint32_t *choice);

/* Use the shape sets and paths `choice` (bits as for polymul_ragged_tune;
 * tensor bits of classes the list does not hold are ignored) instead of the
 * default (every class on the NTT path, set 1) or tuned ones.  Waits for
 * the device to finish its work first (the NTT launches' segment list is
 * rewritten).  Errors: EINVAL (choice >= 128, or a class with units and no
 * tensor kernel for the pool: each pool prime needs at most four 8-bit
 * digits, i.e. q < 2^31), ECUDA. */
int polymul_ragged_select(polymul_ragged_batch *batch, uint32_t choice);

/* Units, degree segments (`items`) and CTAs of a prepared list (any pointer
 * may be NULL). */
int polymul_ragged_batch_info(const polymul_ragged_batch *batch, uint64_t *units, uint64_t *items,
                              uint32_t *grid);

void polymul_ragged_batch_destroy(polymul_ragged_batch *batch); /* NULL-safe */
void polymul_ragged_destroy(polymul_ragged *ctx);               /* NULL-safe */

/* ------------------------------------------------------------------------
 * Serving: a continuously batching request loop.  Requests are products of
 * any degree n <= n_max with their own subset of a prime pool (64-bit
 * words, each prime < 2^62 with 2 n_max | q - 1), operands in HOST memory.
 * A server thread admits queued requests in arrival order as soon as device
 * memory (an arena of `device_bytes`) and an in-flight slot free up, runs
 * each on one of `lanes` streams (copy in, kernel, copy out) so that work of
 * different requests overlaps on the device, and retires finished ones.
 * A request whose a, b and c all lie in page-locked host memory the device
 * maps (checked at submission as for polymul_batch_mapped) takes the direct
 * route: its kernel loads a and b and stores c in host memory itself over
 * the host link, with no arena memory and no copies
 * (polymul_server_set_route turns this off).
 * Twiddle tables of the whole pool stay resident (Sec. 4, "fine-tuning the
 * design" (i)); copies overlap computation (Sec. 4 (ii)).
 * ---------------------------------------------------------------------- */
typedef struct polymul_server polymul_server;

typedef struct polymul_request {
    uint32_t n;                  /* degree, power of two, 16 <= n <= n_max */
    uint32_t k;                  /* number of primes (>= 1)                */
    const uint32_t *prime_idx;   /* k pool indices (read during submit)     */
    const void *a;               /* host [k][n] uint64_t operands; must stay */
    const void *b;               /*   valid until the request completes;    */
    void *c;                     /*   page-locked memory overlaps copies     */
} polymul_request;

typedef struct polymul_server_stats {
    uint64_t submitted, completed, failed, queued, in_flight;
    uint64_t arena_bytes, arena_peak_bytes;
    double p50_us, p99_us, mean_us, max_us; /* submit -> completion latency */
    double queue_p50_us, queue_p99_us;      /* submit -> admission (waiting
                                               for memory, a slot or the
                                               server thread)               */
    double service_p50_us, service_p99_us;  /* admission -> observed
                                               completion (copies in, kernel,
                                               copy out)                    */
    double issue_us_mean;                   /* host time the server thread
                                               spends enqueuing one request */
    double server_busy_s;                   /* server-thread time in passes
                                               that admitted or retired work */
    uint64_t completed_direct;              /* completed requests that took
                                               the direct route             */
} polymul_server_stats;

#define POLYMUL_ROUTE_DIRECT 0  /* operands in mapped page-locked host memory
                                   are read and written in place (default) */
#define POLYMUL_ROUTE_STAGED 1  /* always copy through device memory       */

/* Start a server on the current device.  Each lane is three streams (copies
 * in, kernels, copies out); with more than 8 streams in the process, set
 * CUDA_DEVICE_MAX_CONNECTIONS (up to 32) before the CUDA context is created,
 * or streams share hardware queues and lanes wait on each other.  Errors:
 * EINVAL, ENOMEM, ENOTSUP. */
int polymul_server_create(const uint64_t *pool, uint32_t pool_size, uint32_t n_max,
                          uint64_t device_bytes, uint32_t lanes, polymul_server **out);
/* Queue one request (asynchronous); *ticket identifies it. */
int polymul_server_submit(polymul_server *srv, const polymul_request *req, uint64_t *ticket);
/* The path of requests submitted after the call: POLYMUL_PATH_NTT (the
 * default) or POLYMUL_PATH_TENSOR -- the matrix form (Sec. 2.2) as the
 * 64-bit-word digit kernel: 5 .. 8 balanced 8-bit digits of each centred
 * residue per operand (as many as the pool's largest prime needs, at least
 * five), the exact fp32 sums of each K chunk of at most 1024 drained into
 * 64-bit modular sums, for degrees 2^10 .. n_max (smaller degrees stay on
 * the NTT path).  The first switch to the tensor path sets up its kernels
 * and the pool's constants (synchronous).  Errors: EINVAL (path), ENOTSUP
 * (n_max below 1024), ENOMEM, ECUDA. */
int polymul_server_set_path(polymul_server *srv, uint32_t path);
/* The host route of requests submitted after the call: POLYMUL_ROUTE_DIRECT
 * (the default; requests whose buffers are not all mapped page-locked
 * memory, and tensor-path requests, are copied all the same) or
 * POLYMUL_ROUTE_STAGED.  Errors: EINVAL. */
int polymul_server_set_route(polymul_server *srv, uint32_t route);
/* *done = 1 once the result is in req->c (the ticket is then released).  A
 * request that failed releases its ticket and returns its error: ETIMEOUT
 * when a bounded device wait of its kernel expired (c is invalid), ECUDA for
 * a CUDA error. */
int polymul_server_poll(polymul_server *srv, uint64_t ticket, int *done);
/* Block until the request completes; its failure as for polymul_server_poll,
 * or ETIMEOUT after timeout_s seconds with the request still pending. */
int polymul_server_wait(polymul_server *srv, uint64_t ticket, double timeout_s);
/* Load generator: submit reqs[i] at arrival_s[i] seconds after the call,
 * wait for all, and store each submit-to-completion latency (microseconds)
 * in latency_us (may be NULL). */
int polymul_server_replay(polymul_server *srv, const polymul_request *reqs, uint32_t count,
                          const double *arrival_s, double *latency_us);
/* Counters and latency percentiles of completed requests; reset != 0
 * clears them afterwards. */
int polymul_server_stats_get(polymul_server *srv, polymul_server_stats *out, int reset);
/* Stop the loop (finishing work in flight) and free everything.  NULL-safe. */
void polymul_server_destroy(polymul_server *srv);

/*
 * polymul_selftest_wait -- diagnostics (the paper has no counterpart).
 * Runs one small kernel whose bounded mbarrier wait has nothing to wait for
 * and therefore gives up after `polls` polls (1 .. 2^22), the path every
 * kernel of the library takes when a copy or MMA never completes.  Returns
 * POLYMUL_ETIMEOUT when the wait expired and was reported (the expected
 * outcome; the CUDA context stays usable), EINVAL for polls outside the
 * range, ECUDA otherwise.  Synchronises `stream`.
 */
int polymul_selftest_wait(uint32_t polls, void *stream);

/*
 * polymul_selftest_inject_wait -- diagnostics (the paper has no counterpart).
 * The next `launches` launches of the NTT batch kernel in this process (by
 * any plan, server or polymul_batch_static; the thread-block-cluster kernel
 * for n >= 2^14 does not count) expect 16 bytes more than their operand
 * copies deliver, so every bounded wait they make expires after `polls`
 * polls: the path of a copy that never completes, taken without any device
 * fault.  Their results are invalid and they report it like a real expiry
 * (polymul_plan_status and polymul_static_status return POLYMUL_ETIMEOUT; a
 * server request completes as failed with POLYMUL_ETIMEOUT).  launches = 0
 * cancels what is left.  Errors: EINVAL (polls outside [1, 2^22], launches
 * > 2^20).
 */
int polymul_selftest_inject_wait(uint32_t launches, uint32_t polls);

/* Message for the calling thread's most recent failing call ("" if none).
 * The pointer stays valid until the next call from the same thread. */
const char *polymul_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* POLYMUL_H */
