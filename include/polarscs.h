/*
 * polarscs.h - C ABI of the GB300 (sm_103a) stack decoder for polar codes.
 *
 * The method is successive-cancellation stack (SCS) decoding with the fast
 * simplified nodes and the reduced-memory in-place partial sums of Aurora &
 * Gross, "Towards Practical Software Stack Decoding of Polar Codes"
 * (arXiv 1809.03606), Sec. 2.2.5, Sec. 3.3 and Sec. 4.
 *
 * Conventions shared by every call:
 *  - A code PC(N, K) is given by N (a power of two), K information bits and a
 *    frozen mask of N bytes, 1 = frozen (Sec. 2.1).  With a CRC of crc bits the
 *    message has K - crc bits; the CRC register (initial value 0, no
 *    reflection, no final XOR, polynomial 0x07 for crc = 8, 0x1021 for 16,
 *    0xB2B117 for 24) follows the message MSB first on the last crc
 *    information positions.  Message bit j sits on the j-th information index
 *    in increasing order.
 *  - Codewords are c = u F^{(x)n} with the XOR tree of Fig. encoder
 *    (non-systematic encoding), or systematic ones for a plan switched by
 *    polar_plan_set_systematic.
 *  - Decoding uses min-sum (Eq. minsum) unless a plan is switched to the
 *    exact box-plus rule by polar_plan_set_exact.
 *  - Channel LLRs are float32, LLR = ln P(0)/P(1); they must be finite.
 *  - Device buffers are row-major per frame.  Packed bit buffers are uint32
 *    words, bit j of a row in word j/32 at bit position j%32 (LSB first).
 *  - "stream" is a cudaStream_t passed as void* (NULL = the legacy default
 *    stream).  Batched calls are asynchronous on that stream; the caller
 *    owns every buffer and must keep it alive until the stream has passed the
 *    call.  The library keeps no pointer to caller memory after that.
 *  - Return values: 0 = OK; > 0 is a per-frame decode status (single-frame
 *    calls only); < 0 is an error and nothing was launched.
 *  - Every function is thread-safe.  A plan may be shared between threads
 *    and streams once created.
 */
#ifndef POLARSCS_H
#define POLARSCS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* decode status of one frame (also the int8 entries of a status buffer) */
#define POLAR_OK 0
#define POLAR_CRC_FAIL 1 /* no complete path passed the CRC: the first complete
                            path popped is returned (Sec. 2.2.5, CRC rule) */
#define POLAR_TIMEOUT 2  /* iteration guard tripped; never expected, output zero */
#define POLAR_DEBUG_FAIL 4 /* bounds-checked debug builds only (POLAR_DEBUG): an
                              internal index check failed in this frame; its
                              output is not meaningful */

/* errors */
#define POLAR_EINVAL (-1) /* bad argument: N not a power of 2 in range, K not in
                             [1, N], D < 1, L < 1, crc not in {0, 8, 16, 24},
                             crc >= K, frozen count != N - K, NULL pointer */
#define POLAR_ENOMEM (-2) /* host or device allocation failed */
#define POLAR_ECUDA (-3)  /* a CUDA call failed (no device, launch error) */
#define POLAR_ELIMIT (-4) /* valid code, but beyond the GPU kernel's limits:
                             N > 8192, L > 255, D > 65536 (scs_decode_batch,
                             min-sum plans) or D > 64 (the other decoders
                             and exact-f plans) */
#define POLAR_ESCRATCH (-5) /* scs_decode_batch_noalloc only: the plan's tables
                               exceed its 1 MiB static table area, or one
                               warp's scratch exceeds its 16 MiB static array */

#define POLAR_ETIMEOUT (-6) /* polar_serve*: a bounded wait ran out (requests left
                               undecoded; the engine stopped cleanly) */

/* Maximum sizes the GPU decoder accepts. */
#define POLAR_MAX_N_GPU 8192
#define POLAR_MAX_D_GPU 64          /* register stack: every decoder */
#define POLAR_MAX_D_GPU_DEEP 65536  /* memory stack: scs_decode_batch only */
#define POLAR_MAX_L_GPU 255

/* Opaque decoding plan: the precomputed schedule of Sec. 3.1 (Fig. fsscsch)
 * plus the tables the kernels need.  Created on the host; its device copy is
 * made on first use on a GPU. */
typedef struct polar_plan polar_plan;

/* Frozen mask by Bhattacharyya-parameter construction at a design Eb/N0 in dB
 * (the paper uses the 5G sequence, Sec. 5, which this library does not ship):
 * z0 = exp(-(K/N) 10^(dB/10)), an f child gets 2z - z^2, a g child z^2, the K
 * positions of smallest z are information bits (ties: higher index).  Double
 * precision, host only.  frozen: out, N bytes (1 = frozen).  Returns 0 or
 * POLAR_EINVAL (N not a power of 2 in [2, 32768], K not in [1, N]). */
int polar_construct(int N, int K, float design_snr_db, uint8_t *frozen);

/* Build a plan for PC(N, K) with the given frozen mask (host memory, N bytes,
 * copied).  fast_nodes != 0 recognises the Rate-0, Rate-1, repetition and SPC
 * nodes of Sec. 2.2.2 (precedence R-0 > R-1 > REP > SPC, SPC from 4 leaves);
 * 0 decodes bit by bit (Sec. 2.2.1).  crc in {0, 8, 16, 24}.  *out receives a
 * plan owned by the caller (free with polar_plan_destroy).  Host only: no GPU
 * is needed to create or inspect a plan.  Errors: POLAR_EINVAL, POLAR_ENOMEM. */
int polar_plan_create(int N, int K, const uint8_t *frozen, int fast_nodes, int crc, polar_plan **out);

/* Per-stage min-sum scales (not in the paper; the learnable form trained by
 * gsc_loss_grad below): every f output written at stage lambda is multiplied
 * by scales[lambda] (float32), lambda = 0 .. n-1.  NULL restores plain
 * min-sum.  Host memory, n floats, copied (and pushed to the plan's device
 * copy if it exists).  Not while a call using the plan is in flight.
 * Errors: POLAR_EINVAL (NULL plan, non-finite scale), POLAR_ECUDA. */
int polar_plan_set_scales(polar_plan *plan, const float *scales);

/* Systematic encoding (Sec. 2.2.2, Sec. 4): with on != 0 the codeword
 * itself carries the K information bits (message, then CRC) on the
 * information set, x_A = info with u frozen = 0, and decoders read the
 * message straight from the decoded codeword (no re-encode); on = 0 restores
 * the non-systematic code.  The encoder computes x as two passes of the XOR
 * tree with the frozen positions cleared in between, which is systematic
 * exactly when the information set is closed under the bit-subset order
 * between its members (true of the constructions this library makes); a set
 * for which the two passes are not systematic is rejected.  Host only; call
 * before the plan's first GPU use (its device tables are made then).
 * Errors: POLAR_EINVAL (NULL plan, plan already on a device, unsupported
 * information set), POLAR_ENOMEM. */
int polar_plan_set_systematic(polar_plan *plan, int on);

/* Exact-f decoding: with on != 0, scs_decode_batch(_noalloc) decodes the
 * plan with the box-plus f of Eq. llrcalc itself, 2 atanh(tanh(a/2)
 * tanh(b/2)) evaluated as sgn(a) sgn(b) min(|a|,|b|) + ln(1 + e^-|a+b|) -
 * ln(1 + e^-|a-b|), and the exact leaf metric of Eq. PMupd, PM += ln(1 +
 * exp(-(1 - 2u) alpha)) at every leaf, in float32, instead of min-sum.  The
 * plan must be bit-level (fast_nodes = 0: the fast-node decoders of Sec.
 * 2.2.2 are min-sum rules) and without scales; exact plans are decoded by the
 * uniform decoder only (not in plan sets).  Host only; call before the plan's
 * first GPU use.  Counters keep the min-sum counting convention.
 * Errors: POLAR_EINVAL (NULL plan, fast nodes, scales set, plan already on a
 * device). */
int polar_plan_set_exact(polar_plan *plan, int on);

/* Release a plan and its device copy (synchronous; no call using it may be
 * in flight).  NULL is ignored. */
void polar_plan_destroy(polar_plan *plan);

/* The plan's schedule (Fig. fsscsch), host logic.  ops_out receives up to
 * max_ops triples (op, lambda, phi): op 0 = alpha (Eq. llrcalc, node
 * (lambda, phi) from its parent), 1 = beta (Eq. bitcalc, odd node (lambda, phi)
 * into its parent), 2 = R-0, 3 = R-1, 4 = REP, 5 = SPC, 6 = frozen leaf,
 * 7 = information leaf.  Returns the number of operations, or < 0. */
int polar_plan_schedule(const polar_plan *plan, int32_t *ops_out, int max_ops);

/* Encode B messages on the GPU (Sec. 2.1; the CRC of the plan is appended;
 * systematic when the plan is, see polar_plan_set_systematic).
 * d_msg: device, [B, ceil((K-crc)/32)] packed message bits.  d_codeword:
 * device, [B, ceil(N/32)] packed codeword bits.  Asynchronous on stream. */
int polar_encode_batch(const polar_plan *plan, const uint32_t *d_msg, int B, uint32_t *d_codeword, void *stream);

/* Encode one message (host memory, synchronous): msg holds K - crc bits, one
 * per byte; codeword receives N bytes.  Runs polar_encode_batch on the
 * current device. */
int polar_encode(const uint8_t *msg, int N, int K, const uint8_t *frozen, int crc, uint8_t *codeword);

/* Decode B frames on the GPU with FSSCS-RM (Sec. 2.2.5, Sec. 3.3, Sec. 4):
 * best-first search over a stack of at most D paths, at most L extensions
 * per branching node, the CRC of the plan checked on complete paths.
 *  d_llr    device, [B, N] float32 channel LLRs (Eq. llrcalc, stage n)
 *  d_info   device out, [B, ceil((K-crc)/32)] packed message bits
 *  d_pm     device out, [B] float32 final path metric (Eq. PMupd)
 *  d_status device out, [B] int8 POLAR_OK / POLAR_CRC_FAIL / POLAR_TIMEOUT
 *  d_stats  device out or NULL, [B, 4] uint32: pops, path switches, counted
 *           operations (the ALU-roofline convention of the design notes),
 *           expansions.
 * D <= 64 keeps the stack in registers.  64 < D <= POLAR_MAX_D_GPU_DEEP
 * (e.g. the D = 8192 of Sec. 5) keeps it in per-warp scratch memory with the
 * same search order (min-sum plans only; an exact-f plan gives POLAR_ELIMIT);
 * that scratch holds one beta snapshot per iteration, L * (branching nodes +
 * 9) + 3 of them, and up to min(D, 7 * iterations + 1) entries of 16 bytes,
 * and a launch holds at most 8 GiB of it (fewer resident warps when one
 * warp's share is large; POLAR_ELIMIT when one warp's exceeds it).
 * Scratch (the in-place beta arrays of stacked paths) is allocated
 * stream-ordered per call.  Asynchronous on stream; errors are returned
 * before launch (POLAR_EINVAL, POLAR_ELIMIT) or from the launch
 * (POLAR_ECUDA, POLAR_ENOMEM). */
int scs_decode_batch(const polar_plan *plan, const float *d_llr, int B, int D, int L, uint32_t *d_info,
                     float *d_pm, int8_t *d_status, uint32_t *d_stats, void *stream);

/* scs_decode_batch without any allocation by the library (the paper has no
 * counterpart; this is a deployment variant).  For callers that cannot
 * allocate device memory at decode time -- a fixed budget reserved at
 * start-up, a real-time loop where cudaMalloc/cudaMallocAsync may block or
 * fail, or device memory owned by another allocator.  Same arguments, outputs
 * and results as scs_decode_batch for D <= POLAR_MAX_D_GPU (the register
 * stack); the memory stack of larger D needs per-call scratch and is not
 * offered here (POLAR_ELIMIT).  The caller still provides every input and
 * output buffer.
 *  - The scratch lives in a file-scope static device array of 16 MiB and the
 *    plan's tables are copied into a static 1 MiB device area; every GPU that
 *    loads the library holds both until the process exits.  The decoder runs
 *    as many resident warps as the 16 MiB hold, so large D and N run on fewer
 *    warps (slower, same result).  Returns POLAR_ESCRATCH when the plan's
 *    tables exceed 1 MiB or one warp's scratch, (D+1) * (ceil(N/32)+4 rounded
 *    up to 8) * 4 bytes, exceeds 16 MiB.
 *  - The table area remembers the plan (and the version of its tables) it
 *    holds.  A call with another plan, or after polar_plan_set_scales changed
 *    the plan, copies the tables from the plan's pageable host memory: CUDA
 *    may make the host wait for earlier work on the stream before such a
 *    copy.  A call with the plan already in the area issues no copy, only a
 *    reset of the frame counter (a memset) and the kernel launch; it relies on the earlier
 *    call's copy being ordered before it (the same stream, or synchronised).
 *  - No cudaMalloc, cudaMallocAsync or cudaFree is called.  The first call on
 *    a device looks up the arrays' device addresses (cudaGetSymbolAddress)
 *    with that device current; make that first call before any stream
 *    capture.
 *  - Every call shares the two arrays, which keep the previous call's
 *    contents (the frame counter is cleared on each call).  Calls whose work
 *    overlaps on the GPU (different streams, or different host threads)
 *    race on them and give wrong results; serialise them, e.g. on one
 *    stream. */
int scs_decode_batch_noalloc(const polar_plan *plan, const float *d_llr, int B, int D, int L, uint32_t *d_info,
                             float *d_pm, int8_t *d_status, uint32_t *d_stats, void *stream);

/* ---- Mixed batches (one persistent launch for frames of different codes) ----
 * Not a construct of the paper: a batching form of the same decoder.  Every
 * frame is decoded exactly as scs_decode_batch would decode it alone with its
 * own plan, D and L. */
typedef struct polar_plan_set polar_plan_set;

/* Group 1..64 plans (not copied: they must outlive the set).  Host only.
 * Errors: POLAR_EINVAL, POLAR_ELIMIT (a plan with N > 8192), POLAR_ENOMEM. */
int polar_plan_set_create(const polar_plan *const *plans, int nplans, polar_plan_set **out);
void polar_plan_set_destroy(polar_plan_set *set);

/* Decode B frames of mixed codes in one persistent launch.
 *  d_frames   device, [B, 4] int32 per frame: plan index in the set, D
 *             (1..Dmax), L (1..255), unused; 16-byte aligned
 *  d_order    device, [B] int32 permutation of 0..B-1 giving the order in
 *             which frames are started (e.g. polar_mixed_order), or NULL
 *  Dmax       largest D of the batch (<= 64); sizes the scratch
 *  d_llr      device float32 LLRs of all frames, packed; frame b's N values
 *             start at d_llr[d_llr_off[b]] (16-byte aligned starts are read
 *             with vector loads)
 *  d_info     device packed message words; frame b's ceil(K_msg/32) words
 *             start at d_info[d_info_off[b]]
 *  d_pm, d_status, d_stats as in scs_decode_batch, indexed by frame.  A frame
 *  whose descriptor is invalid (bad plan index, D or L) gets status 3 and
 *  pm = +inf, and nothing else of it is read or written.
 * The set's device tables are made on the first call on a device (make that
 * call before any stream capture; later calls can be captured in a CUDA
 * graph).  Asynchronous on stream. */
int scs_decode_mixed(const polar_plan_set *set, const int32_t *d_frames, const int32_t *d_order, int B, int Dmax,
                     const float *d_llr, const int64_t *d_llr_off, uint32_t *d_info, const int64_t *d_info_off,
                     float *d_pm, int8_t *d_status, uint32_t *d_stats, void *stream);

/* Longest-first claim order for scs_decode_mixed (host): h_frames is the host
 * copy of the [B, 4] descriptors, h_order receives a permutation of 0..B-1
 * sorted by decreasing N * (8 + D).  Pass it (on the device) as d_order so
 * that expensive frames start first.  Errors: POLAR_EINVAL. */
int polar_mixed_order(const polar_plan_set *set, const int32_t *h_frames, int B, int32_t *h_order);

/* Claim order for scs_decode_mixed_split (host): the frames that need two
 * stack rows a lane (valid descriptors with 32 < D <= 64) first, then all
 * others, each part sorted like polar_mixed_order (decreasing N * (8 + D),
 * ties in frame order).  *n_two receives the size of the first part.
 * Errors: POLAR_EINVAL. */
int polar_mixed_split_order(const polar_plan_set *set, const int32_t *h_frames, int B, int32_t *h_order, int *n_two);

/* scs_decode_mixed in two persistent launches (a GPU mapping, not a
 * construct of the paper; every frame's result is the one scs_decode_mixed
 * gives): d_order[0, n_two) are decoded by the kernel with two stack rows a
 * lane (D <= 64) on a second stream of the library, forked from `stream`
 * with an event, and d_order[n_two, B) by the one-row kernel (D <= 32) on
 * `stream`, which then waits for the other launch; so frames with D <= 32
 * no longer carry the second row, and each launch fills the other's tail.
 * d_order is required: polar_mixed_split_order gives it and n_two (a frame
 * of the second part with D > 32 gets status 3, as an invalid descriptor).
 * Dmax bounds the first part's D (it must exceed 32 when n_two > 0).  The
 * side stream and its two events are made on the first call on a device
 * (make it before any stream capture; later calls can be captured, the
 * fork and join becoming graph dependencies).  Calls from several host
 * threads are serialised while they enqueue.  Other arguments, outputs and
 * errors as scs_decode_mixed. */
int scs_decode_mixed_split(const polar_plan_set *set, const int32_t *d_frames, const int32_t *d_order, int B,
                           int n_two, int Dmax, const float *d_llr, const int64_t *d_llr_off, uint32_t *d_info,
                           const int64_t *d_info_off, float *d_pm, int8_t *d_status, uint32_t *d_stats,
                           void *stream);

/* Autotuner for scs_decode_mixed: decodes the given batch (same arguments)
 * with every combination of 1, 2 or 4 warps (frames in flight) per block and
 * 1, 4 or 16 frames claimed per atomic, times each on the stream with CUDA
 * events (synchronising), and keeps the fastest in the set for later calls.
 * *wpb_out and *chunk_out (optional) receive the choice. */
int scs_tune_mixed(polar_plan_set *set, const int32_t *d_frames, const int32_t *d_order, int B, int Dmax,
                   const float *d_llr, const int64_t *d_llr_off, uint32_t *d_info, const int64_t *d_info_off,
                   float *d_pm, int8_t *d_status, void *stream, int *wpb_out, int *chunk_out);

/* The launch shape scs_decode_mixed and scs_decode_mixed_split use for the
 * set, as scs_tune_mixed leaves it: warps_per_block in {1, 2, 4} and
 * frames_per_claim in 1 .. 1024, or both 0 for the defaults (4 warps, 1
 * frame).  For restoring a tuning result saved earlier instead of timing
 * again (the paper has no counterpart; the binding keeps such results in a
 * JSON file keyed by GPU and codes).  Host only, no device work; thread-safe.
 * Errors: POLAR_EINVAL (null set, values out of range). */
int polar_plan_set_tuning(polar_plan_set *set, int warps_per_block, int frames_per_claim);

/* The set's current launch shape (0, 0 when it was never tuned or set).
 * Host only.  Errors: POLAR_EINVAL (a null argument). */
int polar_plan_set_get_tuning(const polar_plan_set *set, int *warps_per_block, int *frames_per_claim);

/* ---- Genie-aided SC with per-stage min-sum scales (differentiation) ----
 * Built on Eq. minsum and Eq. llrcalc: with the transmitted bits known, every
 * g uses the true partial sums, and the f output written at stage lambda is
 * multiplied by scales[lambda] (lambda = 0 .. n-1).  The loss is the mean over
 * frames and information leaves of softplus(-(1 - 2 u_i) L_i), the binary
 * cross-entropy of the leaf LLR L_i against the transmitted bit u_i.
 *  d_llr     device, [B, N] channel LLRs
 *  d_u       device, [B, ceil(N/32)] packed transmitted bits u (frozen = 0)
 *  d_scales  device, [n] stage scales
 *  d_loss    device out, one value
 *  d_leaf    device out or NULL, [B, N] leaf LLRs
 *  d_grad_scales  device out, [n] d loss / d scales
 *  d_grad_llr     device out or NULL, [B, N] d loss / d llr
 * The reverse pass recomputes the forward tree (nothing is stored between
 * calls).  Per-frame sums are reduced over frames in a fixed order:
 * results are bit-reproducible.  Limits: the (n+1) x N tree must fit in
 * shared memory (N <= 2048 in float, N <= 1024 in double), else POLAR_ELIMIT.
 * Asynchronous on stream. */
int gsc_loss(const polar_plan *plan, const float *d_llr, const uint32_t *d_u, int B, const float *d_scales,
             float *d_loss, float *d_leaf, void *stream);
int gsc_loss_grad(const polar_plan *plan, const float *d_llr, const uint32_t *d_u, int B, const float *d_scales,
                  float *d_loss, float *d_grad_scales, float *d_grad_llr, void *stream);
int gsc_loss_f64(const polar_plan *plan, const double *d_llr, const uint32_t *d_u, int B, const double *d_scales,
                 double *d_loss, double *d_leaf, void *stream);
int gsc_loss_grad_f64(const polar_plan *plan, const double *d_llr, const uint32_t *d_u, int B,
                      const double *d_scales, double *d_loss, double *d_grad_scales, double *d_grad_llr,
                      void *stream);

/* ---- Serving (continuous batching) ----
 * Not a construct of the paper: a serving form of the same decoder.  Requests
 * arrive at given times (seconds from the start of the call, non-decreasing).
 * Request r is (plan index in the set, D, L, pool frame) = req[4r .. 4r+3];
 * its N LLRs are pool_llr[pool_off[frame] ..] (host memory, read during the
 * call).
 *  polar_serve keeps one persistent kernel resident: each warp claims the
 *  next request, waits until the host has released it, decodes it and
 *  raises its completion flag, so requests that arrive while others are
 *  being decoded start as soon as a warp and arena space free up.  A request
 *  is released once it has arrived and its LLRs fit in the device arena of
 *  arena_floats floats (the HBM budget; space is returned when the oldest
 *  outstanding requests complete).  The requests released together are
 *  gathered on the host into a pinned mirror of the arena (arena_floats
 *  floats of pinned host memory for the duration of the call) and copied in
 *  one transfer.  Every device and host wait is bounded by
 *  wait_s seconds; on time-out the engine stops and returns POLAR_ETIMEOUT.
 *  polar_serve_baseline decodes one size per launch: every interval_s the
 *  arrived requests are grouped by (plan, D, L) and each group is a separate
 *  scs_decode_batch launch.
 * Outputs per request: pm_out, status_out (as scs_decode_batch; 127 if never
 * decoded), latency_out (completion - arrival, seconds; NaN if not completed)
 * and, for polar_serve, the packed message words at info_off[r] of info_out
 * (both may be NULL) and service_out (may be NULL): the seconds from the
 * moment a warp starts the request, after its release, to its completion,
 * both on the device clock (latency - service = waiting for release and for
 * a warp).  report (6 doubles): seconds from start to the last
 * completion, arena-full stalls, error flag, most requests in flight (serve) or
 * launches (baseline), requests completed, arena bytes. */
int polar_serve(const polar_plan_set *set, const int32_t *req, const double *arrival_s, int R, const float *pool_llr,
                const int64_t *pool_off, int P, int64_t arena_floats, double wait_s, float *pm_out,
                int8_t *status_out, uint32_t *info_out, const int64_t *info_off, double *latency_out,
                double *service_out, double *report);
int polar_serve_baseline(const polar_plan_set *set, const int32_t *req, const double *arrival_s, int R,
                         const float *pool_llr, const int64_t *pool_off, int P, int64_t arena_floats,
                         double interval_s, double wait_s, float *pm_out, int8_t *status_out, double *latency_out,
                         double *report);

/* Decode one frame held in host memory (synchronous), fast nodes on:
 * llr N floats in, info_out K - crc bytes (one bit per byte) out, *pm_out the
 * final path metric.  Runs scs_decode_batch on the current device, so D may be
 * up to POLAR_MAX_D_GPU_DEEP.  Returns the frame status (>= 0) or an error
 * (< 0). */
int scs_decode(const float *llr, int N, int K, const uint8_t *frozen, int D, int L, int crc, uint8_t *info_out,
               float *pm_out);

/* Number of SMs and the library's build architecture string, for reports. */
int polar_device_info(int *sm_count, int *cc_major, int *cc_minor);

#ifdef __cplusplus
}
#endif

#endif /* POLARSCS_H */
