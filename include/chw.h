/*
 * chw.h -- C ABI of the GB300 (sm_103a) Cascading Haar Wavelet Walsh-Hadamard library.
 *
 * The library computes y = H_m x for batches of signals of length n = 2^m, where H_m is
 * the 2^m x 2^m Hadamard matrix in dyadic (Paley) order defined by the recursion of
 * eq. (1) of "The Cascading Haar Wavelet algorithm for computing the Walsh-Hadamard
 * Transform" (arXiv 1609.06641):
 *
 *     H_0 = 1,   H_{m+1} = 2^{-1/2} [ H_m (x) (1 1) ; H_m (x) (1 -1) ].
 *
 * It computes it by the CHW algorithm of Theorem 1 (eq. (3)): the Haar transform Psi_m of
 * eq. (2), followed by stages r = 1..m-1, each applying Psi_{m-r} to the second half of
 * every block of length 2^{m-r+1}.  The cascade's butterflies are fused into register,
 * shared-memory, cluster (DSMEM) and HBM tiers; every schedule performs the same
 * butterflies on the same operands, so results round exactly as the cascade taken in
 * the paper's stage order does.  Signals of 2^15 and 2^16 elements are held on one SM,
 * their rows in shared memory and the whole signal in the SM's tensor memory (tcgen05),
 * between the row butterflies and the last ones; signals of 2^17 on a pair of SMs, half
 * in each, the last label bit exchanged through L2.
 *
 * Conventions for every call below:
 *   - Pointers named x, y, exp_*, diag are DEVICE pointers unless the name says _host.
 *     The caller owns them.  Data buffers must be 16-byte aligned.
 *   - Layout: batch-major, contiguous: signal b occupies elements [b*n, (b+1)*n).
 *   - stream is a cudaStream_t passed as void* (NULL = the legacy default stream).
 *     Device calls are asynchronous on that stream and never synchronise; a plan must
 *     be used from one stream at a time.
 *   - Errors are returned as chw_status_t; nothing aborts and no C++ exception crosses
 *     the boundary.  chw_last_error_message() gives a one-line reason (per host thread).
 *     Errors found on the device (a bounded wait that ran out, a checked-mode index
 *     fault) are latched in the plan and reported by chw_last_device_status().
 *   - In-place operation (x == y) is allowed for every call except the Haar transforms
 *     (chw_haar, chw_haar_inverse, chw_forward_haar), whose input and output must not
 *     overlap.
 */
#ifndef CHW_H
#define CHW_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum chw_status_e {
  CHW_OK = 0,
  CHW_ERR_INVALID_ARG = 1,  /* bad m, batch, dtype/norm pairing, null pointer, ...   */
  CHW_ERR_UNSUPPORTED = 2,  /* valid request this library does not implement        */
  CHW_ERR_ALIGNMENT = 3,    /* a data pointer is not 16-byte aligned                 */
  CHW_ERR_OOM = 4,          /* the plan's device workspace could not be allocated    */
  CHW_ERR_CUDA = 5,         /* a CUDA runtime call failed (no device, launch error)  */
  CHW_ERR_TIMEOUT = 6,      /* a bounded device-side wait gave up                    */
  CHW_ERR_DEVICE_CHECK = 7  /* a device-side consistency check failed                */
} chw_status_t;

typedef enum chw_dtype_e {
  CHW_I32 = 0,   /* int32, unnormalised only; two's-complement wrap on overflow        */
  CHW_F32 = 1,   /* fp32 in, fp32 out                                                  */
  CHW_BF16 = 2,  /* bf16 codes with an int32 power-of-two exponent per signal          */
  CHW_F16 = 3    /* fp16 codes with an int32 power-of-two exponent per signal          */
} chw_dtype_t;

/* Placement of the 2^{-1/2} factors of eq. (1)-(2) (the paper counts additions only). */
typedef enum chw_norm_e {
  CHW_NORM_NONE = 0,      /* unscaled butterflies: result 2^{m/2} H_m x                   */
  CHW_NORM_PER_LEVEL = 1, /* (a+b)*c and (a-b)*c at every level, c = fp32(1/sqrt2)       */
  CHW_NORM_END = 2        /* unscaled butterflies, then one multiply by fp32(2^{-m/2})   */
} chw_norm_t;

#define CHW_MAX_M 30

/* Plan flags. */
#define CHW_FLAG_NONE 0u
#define CHW_FLAG_FORCE_SIMPLE 1u    /* use the plain one-CTA-per-signal kernel (tests)  */
#define CHW_FLAG_FORCE_MULTIPASS 2u /* split m into two HBM passes even if one fits     */
#define CHW_FLAG_ROWSTACK 4u        /* m = 15..17: one CTA per signal with its rows through */
                                    /* L2 instead of a thread-block cluster (DSMEM)        */
#define CHW_FLAG_HAAR_WALSH 8u      /* also prepare chw_from_haar / chw_forward_haar       */
#define CHW_FLAG_ORDER_NATURAL 16u  /* store outputs in natural (Sylvester) order          */
#define CHW_FLAG_ORDER_SEQUENCY 32u /* store outputs in sequency (Walsh) order             */
#define CHW_FLAG_TEST_STALL 64u     /* test hook, cluster tier (m = 15..17): one CTA       */
                                    /* withholds a signal and waits give up after a few    */
                                    /* thousand polls, so chw_last_device_status() reports */
                                    /* CHW_ERR_TIMEOUT; the output is then undefined       */
#define CHW_FLAG_CLUSTER 128u       /* m = 15..17: thread-block-cluster (DSMEM) tier of     */
                                    /* shared-memory tiles instead of the tensor-memory    */
                                    /* tier (one SM per signal at 15, 16; two at 17)       */
#define CHW_FLAG_AUTOTUNE 256u      /* pick the tier, two-pass split and CTA tile by timing */
                                    /* the candidates (chw_tune_candidates) on the device  */
                                    /* when the plan is made; CHW_AUTOTUNE=1 in the        */
                                    /* environment turns it on for every plan              */
#define CHW_FLAG_CHECKED 512u       /* checked mode: the kernels that compute global indices */
                                    /* from offsets (tiles, tensor-memory rows and columns, */
                                    /* two-pass scratch, ragged offset tables) range-check  */
                                    /* every input tile and output address before using it; */
                                    /* a bad one is skipped and latches                     */
                                    /* CHW_ERR_DEVICE_CHECK with the offending element index */
                                    /* (chw_last_device_status, chw_last_error_message); the */
                                    /* output is then undefined.  Results are otherwise      */
                                    /* identical; the checks cost a few instructions per     */
                                    /* store                                                 */
#define CHW_FLAG_TEST_CORRUPT 1024u /* test hook, ragged plans, only with CHW_FLAG_CHECKED  */
                                    /* (else CHW_ERR_INVALID_ARG): the plan overwrites, on   */
                                    /* the host before upload, the offset of its first       */
                                    /* signal with m >= 13 and of its first signal with      */
                                    /* m <= 12 by an element index past the end of x and y,  */
                                    /* so the device checks must catch them                  */

typedef struct chw_plan_s* chw_plan_t;

/* Read-only description of what a plan will launch (for tests and reports). */
typedef struct chw_plan_info_s {
  int m;                     /* transform bits (-1 for a ragged plan)                 */
  int64_t batch;             /* signals per call (ragged: number of signals)          */
  int dtype;                 /* chw_dtype_t                                            */
  int norm;                  /* chw_norm_t                                             */
  int tier;                  /* 0 simple, 1 fused CTA, 2 fused cluster, 3 two-pass, 4 ragged,
                                5 fused 16-bit, 6 row-stack (one CTA, L2-resident rows),
                                7 tensor memory (one CTA per signal, m = 15, 16),
                                8 tensor memory over a cluster (m = 17: two SMs hold a
                                  signal and exchange its last label bit through L2) */
  int passes;                /* HBM round trips per call                               */
  int row_bits;              /* two-pass: bits transformed in pass 1 (else m)          */
  int cluster;               /* CTAs per cluster in the fused (or first) pass          */
  int kernels_per_call;      /* kernel launches per forward/adjoint call               */
  int64_t workspace_bytes;   /* device scratch owned by the plan                       */
  int64_t total_elements;    /* elements per call (sum over the batch)                 */
  int order;                 /* output order: 0 dyadic, 1 natural, 2 sequency          */
  int tile_bits;             /* CTA tile of the fused/cluster kernels (13, 14; 0 default) */
  int tuned;                 /* 0 built-in choice, 1 timed by the autotuner, 2 its cache */
  float tune_us;             /* the autotuner's time for the chosen configuration (us) */
} chw_plan_info_t;

/* One configuration the autotuner can choose for a plan. */
typedef struct chw_tune_choice_s {
  int tier;                  /* as chw_plan_info_t.tier                                */
  int row_bits;              /* two-pass: bits of the first (row) pass; otherwise m     */
  int tile_bits;             /* CTA tile of the fused/cluster kernels: 13 or 14; 0 none */
} chw_tune_choice_t;

/*
 * chw_plan -- prepare y = H_m x for `batch` signals of length 2^m (eq. (1), Theorem 1).
 *   m      0..CHW_MAX_M (m = 0 is the identity: H_0 = 1).
 *   batch  >= 1.
 *   dtype/norm: CHW_I32 requires CHW_NORM_NONE; CHW_F32 takes any norm; CHW_BF16 and
 *          CHW_F16 take CHW_NORM_END or CHW_NORM_PER_LEVEL (the stored exponent carries
 *          the scale) and need m <= 13.
 *   flags  CHW_FLAG_* bits.
 * Output order.  By default outputs are in dyadic order, y = H_m x with H_m of eq. (1).
 * CHW_FLAG_ORDER_NATURAL stores the same values in natural (Sylvester-Hadamard) order,
 * y_nat[k] = y[bitrev_m(k)], and CHW_FLAG_ORDER_SEQUENCY in sequency (Walsh) order,
 * y_seq[k] = y[k ^ (k >> 1)] (row k has k sign changes).  The butterflies, and so every
 * value, are those of the dyadic transform; only the store changes.  Both ordered
 * matrices are symmetric, so chw_adjoint of an ordered plan is the same ordered transform
 * (D then applied to its input).  Natural order takes m <= 23 (m >= 17 runs as two HBM
 * passes); ordered plans cannot be combined with CHW_FLAG_ROWSTACK or ragged plans.
 * Tiers by m (chw_plan_get_info reports the one chosen): m <= 14 one CTA per tile in
 * registers and shared memory; m = 15, 16 one SM per signal with the signal held in tensor
 * memory; m = 17 in dyadic order two SMs per signal (a 2-CTA cluster, half of the signal
 * in each SM's tensor memory, the last label bit exchanged through L2); m = 17 in natural
 * order .. 30 two HBM passes; m = 17 in sequency order a thread-block cluster.
 * CHW_FLAG_AUTOTUNE replaces these built-in choices by measured ones.
 * Allocates the plan (host) and its device workspace on the current device: the two-pass
 * intermediate (batch x 2^m elements), or for the m = 17 pair tier its exchange slots
 * (128 KB per pair of SMs, 9.5 MB on 152 SMs).  Returns
 * CHW_ERR_INVALID_ARG / CHW_ERR_UNSUPPORTED / CHW_ERR_OOM / CHW_ERR_CUDA on failure, in
 * which case *plan is set to NULL.
 */
chw_status_t chw_plan(chw_plan_t* plan, int m, int64_t batch, chw_dtype_t dtype, chw_norm_t norm,
                      uint32_t flags);

/*
 * chw_plan_ragged -- prepare one call over `count` signals of uneven lengths 2^{ms[i]}
 * (the transform of eq. (1) applied to each signal independently).
 *   ms_host   host array of `count` bit counts, each in 0..20.  The signals are packed
 *             in that order, each starting on a 32-element (128-byte) boundary, and a
 *             signal with 15 <= m <= 17 on a multiple of 2^{m-8} elements:
 *             e[0] = 0, offset[i] = round_up(e[i], a(ms[i])), e[i+1] =
 *             round_up(offset[i] + 2^{ms[i]}, 32), a(m) = 2^{m-8} for m = 15..17, else 32;
 *             the total is e[count] (chw_ragged_offsets() returns the offsets; the
 *             padding elements are neither read into results nor written).
 *   dtype     CHW_F32 or CHW_I32 (with norm as for chw_plan).
 * The plan sorts the signals by length once and records one launch per length present
 * (signals up to 2^12 share one persistent kernel over a work list; 2^13..2^17 run as
 * batched one-pass launches -- 2^15..2^17 on the tensor-memory tiers when every offset of
 * that length is aligned as above, else on clusters of shared-memory tiles -- and
 * 2^18..2^20 as two-pass launches, reading and writing each signal at its own offset);
 * chw_forward_ragged() replays them as one CUDA graph launch.
 * chw_plan_get_info() reports the kernels in the graph (kernels_per_call).  With
 * CHW_FLAG_AUTOTUNE each length's configuration is timed and chosen when the plan is made
 * (tuned = 1 in chw_plan_get_info).
 */
chw_status_t chw_plan_ragged(chw_plan_t* plan, const uint8_t* ms_host, int64_t count, chw_dtype_t dtype,
                             chw_norm_t norm, uint32_t flags);

/*
 * chw_plan_ragged_at -- as chw_plan_ragged, with the caller's own layout: signal i occupies
 * elements [offsets_host[i], offsets_host[i] + 2^{ms[i]}) of x and y, which hold `total`
 * elements.  Validated on the host before anything is uploaded: every signal must lie in
 * [0, total) and no two may overlap (CHW_ERR_INVALID_ARG otherwise), and signals with
 * m >= 13 must start on a 32-element (128-byte) boundary, because their kernels load them
 * as rows of 32 words by TMA (CHW_ERR_ALIGNMENT otherwise); shorter signals may start
 * anywhere.  Elements outside every signal are neither read into results nor written.
 * The offsets are copied into the plan's device tables, which the recorded CUDA graph
 * reads, so a call does not take offsets of its own.
 */
chw_status_t chw_plan_ragged_at(chw_plan_t* plan, const uint8_t* ms_host, const int64_t* offsets_host, int64_t count,
                                int64_t total, chw_dtype_t dtype, chw_norm_t norm, uint32_t flags);

/* Element offsets of a ragged plan's signals: offsets_host[0..count] (count+1 entries). */
chw_status_t chw_ragged_offsets(chw_plan_t plan, int64_t* offsets_host);

/*
 * chw_forward -- y = D H_m x for every signal of the plan's batch (eq. (1); computed by
 * the cascade of Theorem 1).
 *   x, y     device buffers of batch * 2^m elements of the plan's dtype.
 *   exp_in   bf16/fp16 only: int32[batch], signal b of x means 2^{exp_in[b]} * x_b.
 *   exp_out  bf16/fp16 only: int32[batch] written with the output exponents: y_b means
 *            2^{exp_out[b]} * y_b, chosen so max|y_b| is in [1, 2) for bf16 and
 *            [2^14, 2^15) for fp16.  Must be NULL for int32/fp32.
 *   diag     optional int8[2^m] of +-1 (the diagonal of D, shared by all signals), NULL
 *            for D = I.  Applied to the transform's output.
 */
chw_status_t chw_forward(chw_plan_t plan, const void* x, void* y, const int32_t* exp_in, int32_t* exp_out,
                         const int8_t* diag, void* stream);

/*
 * chw_adjoint -- x = H_m^T D y, the transpose of chw_forward (used for gradients).
 * H_m^T is the reversed cascade of inverse Haar transforms Psi^T.  Each butterfly of the
 * cascade is a symmetric 2x2 matrix and the dyadic reorder is an involution, so the
 * reversed cascade performs the forward cascade's butterflies with inputs and outputs
 * relabelled; it runs on the same kernels and rounds identically.  diag (if given) is
 * applied to y before the transform.  Arguments as for chw_forward.
 */
chw_status_t chw_adjoint(chw_plan_t plan, const void* y, void* x, const int32_t* exp_in, int32_t* exp_out,
                         const int8_t* diag, void* stream);

/* chw_forward_ragged -- transform every signal of a ragged plan (packed layout above). */
chw_status_t chw_forward_ragged(chw_plan_t plan, const void* x, void* y, void* stream);

/*
 * Haar wavelet transforms.  A plan made by chw_plan (dtype CHW_F32 or CHW_I32, any m) also
 * runs the Haar transform Psi_m of eq. (2), its transpose, and the Haar-Walsh transform
 * H_m Psi_m^T of eq. (4), on the same `batch` signals of 2^m elements.
 *
 * Haar layout (what eq. (2) produces): z = Psi_m x holds, per signal,
 *   z[0]                          the approximation after all m levels,
 *   z[2^{m-l} .. 2^{m-l+1} - 1]   the 2^{m-l} details of level l = 1..m,
 * where level l maps the current approximation v (2^{m-l+1} values) to pair sums
 * v_{2i} + v_{2i+1} (the next approximation) and differences v_{2i} - v_{2i+1}.
 *
 * Normalisation (the plan's norm): PER_LEVEL multiplies every butterfly output by
 * fp32(1/sqrt2) (Psi_m exactly as eq. (2) scales it); NONE leaves the butterflies unscaled
 * (int32: exact unnormalised Haar with two's-complement wrap); END leaves them unscaled
 * and multiplies each coefficient once by fp32(2^{-L/2}), where L is the number of levels
 * behind it (m for z[0], l for a level-l detail) -- after the butterflies for chw_haar,
 * before them for chw_haar_inverse.
 *
 * chw_haar          z = Psi_m x.  x and z must not overlap.
 * chw_haar_inverse  x = Psi_m^T z (= Psi_m^{-1} z for PER_LEVEL and END), the synthesis
 *                   butterflies v_{2i} = u_i + d_i, v_{2i+1} = u_i - d_i from coarse to
 *                   fine.  z and x must not overlap.
 * Both read their input once and write their output once (plus 2^{-13} of the data in
 * plan-owned scratch when m > 13); errors as for chw_forward.
 */
chw_status_t chw_haar(chw_plan_t plan, const void* x, void* z, void* stream);
chw_status_t chw_haar_inverse(chw_plan_t plan, const void* z, void* x, void* stream);

/*
 * chw_from_haar -- the Haar-Walsh transform y = H_m Psi_m^T z of eq. (4): Haar
 * coefficients z (layout above) to Walsh-Hadamard coefficients in dyadic order.  These are
 * stages r = 1..m-1 of Theorem 1; by eq. (4) they act on each Haar scale separately, the
 * level-l details (2^k values, k = m - l) going through H_k and z[0] through 1, so the
 * call transforms the scales independently: every scale below 2^14 of every signal in one
 * tile kernel (the head), the scales 2^14..2^17 as batched launches over strided units
 * (with the head on branches forked from the caller's stream and joined again), each
 * larger scale as a two-pass transform; a batch whose total is not a multiple of 32
 * elements (m < 5) runs as one ragged task set.  With PER_LEVEL or NONE the result equals
 * chw_forward(x) bit for bit when z = chw_haar(x); with END each scale k is scaled once by
 * fp32(2^{-k/2}).  In-place (z == y) allowed.  The plan must have been made with
 * CHW_FLAG_HAAR_WALSH (which builds the task set); otherwise CHW_ERR_INVALID_ARG.
 *
 * chw_forward_haar -- y = H_m x together with its Haar side output z = Psi_m x (stage 0 of
 * Theorem 1, "for free" from the cascade): y is bit for bit chw_forward's result and z
 * chw_haar's, in every normalisation.  Where the plan's tier holds whole signals on one SM
 * (single-CTA tiles, m <= 14; the tensor-memory tier, m = 15, 16; dyadic order) the
 * kernels capture z from the same pass -- each detail right after the butterfly of its level, the approximation at
 * the end -- so x is read once and y and z written once; other tiers run chw_haar and then
 * the forward transform.  z must not overlap x or y (x == y is allowed).
 */
chw_status_t chw_from_haar(chw_plan_t plan, const void* z, void* y, void* stream);
chw_status_t chw_forward_haar(chw_plan_t plan, const void* x, void* y, void* z, void* stream);

/*
 * chw_forward_host -- chw_forward for HOST buffers: copies x_host to the device, runs
 * the transform and copies the result to y_host, pipelined in chunks over the plan's
 * own streams and staging buffers; returns when y_host (and exp_out_host) are written.
 * Pinned (page-locked) host memory gives full copy bandwidth.  exp_*_host and diag_host
 * follow chw_forward's rules (diag_host: int8[2^m] on the host, or NULL).
 */
chw_status_t chw_forward_host(chw_plan_t plan, const void* x_host, void* y_host, const int32_t* exp_in_host,
                              int32_t* exp_out_host, const int8_t* diag_host);

/*
 * chw_forward_noalloc -- y = H_m x for `batch` signals through the two-HBM-pass kernels,
 * without allocating anything.  (The paper has no counterpart; this is a library entry
 * point for callers that cannot allocate device memory when they transform: processes
 * whose device memory has been handed in full to another allocator, such as a caching
 * pool that reserved it all; latency-critical code that cannot take cudaMalloc's implicit
 * device-wide synchronisation; and code running where the CUDA runtime's allocator may
 * not be called.)
 *   m, batch, dtype, norm  as for chw_plan.  m outside 18..22 and dtypes other than
 *          CHW_F32 / CHW_I32 return CHW_ERR_UNSUPPORTED; batch * 2^m above 2^22 elements
 *          returns CHW_ERR_INVALID_ARG: the pass-1 intermediate lives in a fixed 16 MiB
 *          device array of the library, which every GPU that loads the library holds
 *          until the process exits.
 *   x, y   device buffers as for chw_forward (16-byte aligned); stream as elsewhere.
 * It launches exactly what chw_forward does for a two-pass plan of the same shape (same
 * split, same kernels, bit-identical results).  No plan object, no cudaMalloc/cudaFree.
 * The first call on a device looks up the array's device address (once per device, with
 * that device current); make that first call before any stream capture.  Each device has
 * its own copy of the array, and all calls on a device share it, keeping the previous
 * call's contents: calls on one device whose work overlaps (different streams with no
 * order between them) race on it and must be serialised by the caller.  A bounded device
 * wait that gives up latches CHW_ERR_TIMEOUT into the
 * array's header word, which each call clears first; read it with
 * chw_noalloc_device_status().
 */
chw_status_t chw_forward_noalloc(int m, int64_t batch, chw_dtype_t dtype, chw_norm_t norm, const void* x, void* y,
                                 void* stream);

/*
 * chw_noalloc_device_status -- the device-side status of chw_forward_noalloc on the current
 * device: synchronises the device, returns the error latched by the calls since the last
 * read (CHW_ERR_TIMEOUT) or CHW_OK, and clears it.  Allocates nothing.
 */
chw_status_t chw_noalloc_device_status(void);

/* Fill *info with what the plan launches. */
chw_status_t chw_plan_get_info(chw_plan_t plan, chw_plan_info_t* info);

/*
 * Autotuner.  A plan made with CHW_FLAG_AUTOTUNE (or with CHW_AUTOTUNE=1 in the
 * environment) times every candidate configuration of its shape on the device -- on
 * min(batch, 2^26 / 2^m) synthetic signals, two warm-up runs and the mean of five, CUDA
 * events -- and keeps the fastest; chw_plan_get_info reports the choice (tier, row_bits,
 * tile_bits, tuned = 1) and its time.  Every candidate computes the same result bit for bit.
 * Choices are cached per process under (device name, m, floor(log2 batch), dtype, norm,
 * order); a later plan with the same key takes the cached choice (tuned = 2).  When
 * CHW_TUNE_CACHE names a file, it is read on the first autotuned plan and rewritten after
 * each new measurement.  Plans with a single configuration (m <= 13; m = 15 and 16, where
 * the tensor-memory tier is the only candidate; m = 30; bf16/fp16; or a flag that fixes
 * the tier) are not timed.
 *
 * chw_tune_candidates   host only: writes up to `cap` candidates for this shape to `out`
 *                       and returns how many there are (0: nothing to choose).
 * chw_tune_cache_put/get host only: set / read the process cache entry of a key, the device
 *                       named by `device` (as cudaDeviceProp.name); get returns
 *                       CHW_ERR_UNSUPPORTED when the key has no entry.
 * chw_tune_cache_load   merges a cache file into the process cache; returns the number of
 *                       entries read (malformed lines are skipped) or -1 if unreadable.
 * chw_tune_cache_save   writes the process cache to `path` (CHW_ERR_INVALID_ARG on I/O error).
 * chw_tune_cache_clear  empties the process cache.
 */
int chw_tune_candidates(int m, chw_dtype_t dtype, chw_norm_t norm, uint32_t flags, chw_tune_choice_t* out, int cap);
chw_status_t chw_tune_cache_put(const char* device, int m, int64_t batch, chw_dtype_t dtype, chw_norm_t norm,
                                uint32_t flags, const chw_tune_choice_t* choice, float us);
chw_status_t chw_tune_cache_get(const char* device, int m, int64_t batch, chw_dtype_t dtype, chw_norm_t norm,
                                uint32_t flags, chw_tune_choice_t* choice, float* us);
int chw_tune_cache_load(const char* path);
chw_status_t chw_tune_cache_save(const char* path);
void chw_tune_cache_clear(void);

/*
 * chw_last_device_status -- synchronise the plan's device work and report the first
 * device-side error latched since the previous call (CHW_ERR_TIMEOUT,
 * CHW_ERR_DEVICE_CHECK) or an asynchronous CUDA error (CHW_ERR_CUDA); clears the latch.
 * For CHW_ERR_DEVICE_CHECK, chw_last_error_message() names the first offending element
 * index.
 */
chw_status_t chw_last_device_status(chw_plan_t plan);

/* Release the plan and its device workspace.  NULL is accepted. */
chw_status_t chw_plan_destroy(chw_plan_t plan);

/* Static description of a status code. */
const char* chw_status_string(chw_status_t status);

/* One-line reason for the last error returned on this host thread ("" if none). */
const char* chw_last_error_message(void);

#ifdef __cplusplus
}
#endif

#endif /* CHW_H */
