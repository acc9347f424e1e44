/*
 * cwth.h - C ABI of libcwth.so, the GB300 (sm_103a) hop-size continuous
 * wavelet transform (CWTH).
 *
 * The operation (paper Sec. II.A, Eq. 1, discretised with dt = 1 sample, and
 * Sec. II.B, which evaluates it only at samples spaced by a hop H):
 *
 *     W_s[k] = a_s^{-1/2} * sum_n x[n] * conj(psi((n - k*H) / a_s)),
 *     k = 0 .. ceil(len/H) - 1,  x[n] = 0 outside [0, len),
 *     psi(t) = (pi*B)^{-1/2} * exp(-t^2/B) * exp(i*2*pi*C*t)   (complex Morlet),
 *
 * and the library returns the scalogram |W_s[k]| in float32.
 *
 * Conventions shared by every call:
 *   - No call throws; each returns a cwth_status.
 *   - "device" pointers are CUDA device memory of the device that was current
 *     when the plan was made; "host" pointers are ordinary or pinned host
 *     memory.  The caller owns every buffer it passes in; a plan owns its
 *     tables and staging buffers and frees them in cwth_destroy.
 *   - Calls that take a stream (a cudaStream_t passed as void*, NULL = the
 *     legacy default stream) enqueue their work on it and return without
 *     synchronising, except cwth_execute_host, which returns once the result
 *     is in host memory.
 *   - A plan may be used by one stream at a time; plans are independent.
 */
#ifndef CWTH_H
#define CWTH_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    CWTH_OK = 0,
    CWTH_ERR_INVALID_ARG = 1, /* a pointer, size, scale or flag is out of range */
    CWTH_ERR_OOM = 2,         /* device or host allocation failed             */
    CWTH_ERR_CUDA = 3,        /* a CUDA runtime call or kernel launch failed  */
    CWTH_ERR_UNSUPPORTED = 4, /* valid request this build cannot serve        */
    CWTH_ERR_TIMEOUT = 5,     /* a bounded device wait ran out                */
    CWTH_ERR_BAD_PLAN = 6     /* NULL, destroyed or foreign plan handle       */
} cwth_status;

/* Complex Morlet parameters, "cmor B-C": bandwidth B > 0, centre frequency
 * C > 0 (cycles per unit of t).  The wavelet's spectrum is
 * exp(-pi^2 B (f - C)^2), peak 1 at f = C. */
typedef struct {
    double bandwidth;
    double center_freq;
} cwth_morlet;

typedef struct cwth_plan_s *cwth_plan_t;

/* Arithmetic of the direct (time-domain, tensor-core) path.  The spectral
 * path always computes in float32.  The split variants write the samples
 * and the taps as sums of bf16 parts and accumulate part products in
 * float32: BF16X2 (hi + lo, all four products) holds each tap product to
 * about 2^-17 relative, so a scalogram value is within about 2^-17 of the
 * sum of |x g| over its taps (tight where the taps do not cancel);
 * BF16X3 (hi + mid + lo, the six products of order up to 2^-16) holds each
 * tap product to about 2^-24, i.e. float32 accuracy even where the taps
 * cancel. */
enum {
    CWTH_PREC_FP32 = 0,   /* float32 everywhere                          */
    CWTH_PREC_BF16 = 1,   /* bf16 operands, float32 accumulation         */
    CWTH_PREC_BF16X2 = 2, /* hi+lo split bf16 operands, fp32 accumulate  */
    CWTH_PREC_BF16X3 = 3  /* hi+mid+lo split bf16, fp32 accumulate      */
};

/* Which evaluation each scale takes. */
enum {
    CWTH_PATH_AUTO = 0,     /* per scale, by the plan's cost model      */
    CWTH_PATH_SPECTRAL = 1, /* every scale through the FFT path         */
    CWTH_PATH_DIRECT = 2    /* every scale through the direct sum       */
};

/*
 * Build a plan for clips of up to max_len samples.
 *
 *   w           host, the Morlet parameters (Eq. 1's psi).
 *   scales      host, S scales a_s in samples (Eq. 1's a; a_s = C*fs/f_s
 *               for a centre frequency f_s in Hz).  Output row s is scale s.
 *   S           number of scales, >= 1.
 *   hop         H of Sec. II.B, >= 1 (H = 1 is the plain CWT).
 *   sample_rate fs in Hz, > 0 (recorded for cwth_plan_query; scales are
 *               already in samples).
 *   max_len     longest clip the plan accepts, >= 1.
 *   precision   CWTH_PREC_*; path CWTH_PATH_*.
 *   out         host, receives the handle.
 *
 * Makes the float64-generated tables (FFT twiddles, per-scale Morlet band
 * limits, direct-path tap banks) on the current device and synchronises
 * with them.  Errors: CWTH_ERR_INVALID_ARG for a NULL pointer, S/hop/max_len
 * < 1, a scale that is not finite and positive, B/C/fs not finite and
 * positive, or an unknown flag; CWTH_ERR_UNSUPPORTED when the forced path
 * cannot serve the request (the spectral path needs hop = 2^e d with d a
 * product of 3, 5 and 7 no larger than 27, e.g. 3, 96 or 100, and
 * hop <= 2048, and a segment of at most 16384 samples with M / hop <= 8192
 * must hold a valid frame beside the largest scale's support: about
 * a <= 1390 samples at hops >= 2, a <= 690 at hop 1; the direct path needs
 * hop % 8 == 0 for bf16 operands and at most 4096 taps);
 * CWTH_ERR_OOM / CWTH_ERR_CUDA otherwise.  On error *out is set to NULL.
 */
cwth_status cwth_plan(const cwth_morlet *w, const double *scales, int32_t S, int32_t hop,
                      double sample_rate, int64_t max_len, int32_t precision,
                      int32_t path, cwth_plan_t *out);

/*
 * cwth_plan with the spectral path's FFT segment length M fixed instead of
 * chosen by the plan's cost model (an autotuner's knob; results agree with
 * any other segment length within the float32 tolerance: every valid
 * segment gives the linear correlation of Eq. 1 at its frames).
 *
 *   seg_len   0: automatic (exactly cwth_plan); else M in [512, 32768] of
 *             the form 2^k d, d a product of 3, 5 and 7 no larger than 27
 *             (a power of two for power-of-two hops).  The spectral path
 *             uses M = 2 d N2 with d the odd part of the hop, N2 a power of
 *             two in [256, 8192 / d] and M / hop >= 8.
 *
 * Errors: those of cwth_plan; CWTH_ERR_INVALID_ARG for a seg_len that is
 * negative, out of range or of another form; CWTH_ERR_UNSUPPORTED when the
 * plan has spectral-path scales and M cannot serve them (its odd part is
 * not the hop's, M / hop < 8, the wavelet support leaves no valid frame, or
 * the segment's shared-memory footprint exceeds a CTA's).
 */
cwth_status cwth_plan_segment(const cwth_morlet *w, const double *scales, int32_t S,
                              int32_t hop, double sample_rate, int64_t max_len,
                              int32_t precision, int32_t path, int32_t seg_len,
                              cwth_plan_t *out);

/*
 * Scalograms of a batch of clips, asynchronous on `stream`.
 *
 *   d_x       device, float32, clip i occupies d_x[i*ld_x .. i*ld_x + len_i).
 *   ld_x      row stride in elements, >= max_len.
 *   d_lengths device, int64 per clip, each in [0, max_len]; NULL means every
 *             clip has max_len samples.  Lengths are read on the device.
 *   batch     number of clips, >= 0 (0 is a no-op).
 *   d_out     device, float32 [batch][S][F_max], F_max = cwth_num_frames(
 *             max_len, hop).  out[i][s][k] = |W_s[k]| of clip i for
 *             k < ceil(len_i/H); frames at and beyond ceil(len_i/H) are not
 *             written.  d_out must not overlap d_x.
 *   stream    cudaStream_t as void*, NULL for the legacy default stream.
 *
 * Workspace: plans with direct-path scales at a bf16 precision stage the
 * batch as bf16 parts, and resample-first plans re-sample it, in device
 * buffers the plan owns and keeps at the largest batch seen.  A call with a
 * larger batch than any before frees and re-allocates them (cudaFree /
 * cudaMalloc, which wait for the device to go idle); calls with smaller or
 * equal batches allocate nothing.  cwth_plan_reserve sizes them up front.
 * Float32 plans whose scales all take the spectral path never allocate here.
 * Within one call, the tensor-core kernel, a spectral part after it and
 * every later spectral part are launched with programmatic stream
 * serialisation (each may start while the kernel before it ends; none
 * reads what that kernel writes, except the tensor-core kernel, which
 * waits for its staging kernel first); every one of them completes after
 * the kernel before it, so work enqueued on `stream` after the call still
 * follows the whole transform.
 *
 * Errors: CWTH_ERR_BAD_PLAN, CWTH_ERR_INVALID_ARG (NULL buffer with
 * batch > 0, ld_x < max_len, batch < 0), CWTH_ERR_OOM (a workspace could
 * not grow), CWTH_ERR_CUDA (launch failure).  Kernel faults surface later,
 * at the caller's next synchronisation.
 */
cwth_status cwth_execute(cwth_plan_t plan, const float *d_x, int64_t ld_x,
                         const int64_t *d_lengths, int32_t batch, float *d_out,
                         void *stream);

/*
 * Resample-first reading of the hop (paper Sec. III.B and Fig. 2, against
 * the output-decimation reading of Sec. II.B that cwth_plan implements): each
 * clip x of n samples is re-sampled at the hop spacing, y[m] = x[m H] for
 * m < ceil(n / H), and the CWT of Eq. 1 is evaluated at every sample of y
 * with scales a_s / H:
 *
 *     W_s[m] = (a_s/H)^{-1/2} sum_j y[j] conj(psi((j - m) / (a_s/H))),
 *
 * so the output has the same [clip][scale][ceil(n / H)] shape as
 * cwth_plan's.  Arguments are as for cwth_plan (scales are given in samples
 * of x, max_len is the longest x); the plan re-samples on the device inside
 * cwth_execute / cwth_execute_host (inputs and lengths are those of x) and
 * then runs the hop-1 transform of y.  No anti-alias filter is applied
 * (plain re-sampling, as the reading states).
 * Errors: as cwth_plan.
 */
cwth_status cwth_plan_resampled(const cwth_morlet *w, const double *scales, int32_t S, int32_t hop,
                                double sample_rate, int64_t max_len, int32_t precision,
                                int32_t path, cwth_plan_t *plan);

/*
 * Same transform from and to host memory.  The batch runs in chunks of
 * whole clips: chunk c is uploaded on a copy stream of the plan, transformed
 * on `stream` and downloaded on a second copy stream, so the upload of chunk
 * c + 1 and the download of chunk c - 1 overlap the transform of chunk c.
 * The copies start after the work already enqueued on `stream`; the call
 * synchronises `stream` (which ends with the last download) before
 * returning.  h_lengths is host memory (or NULL); with lengths, only the
 * written prefix ceil(len_b / H) of each output row is copied back and the
 * rest of h_out is left untouched.  The other arguments are as in
 * cwth_execute.  Device staging is owned by the plan and grows to the
 * largest batch seen.  Pinned host buffers make the copies asynchronous DMA
 * transfers (pageable ones serialise them).
 * Errors: as cwth_execute; after a failure the call still waits for what it
 * enqueued.
 */
cwth_status cwth_execute_host(cwth_plan_t plan, const float *h_x, int64_t ld_x,
                              const int64_t *h_lengths, int32_t batch, float *h_out,
                              void *stream);

/*
 * Chunk count of cwth_execute_host: 0 (the default) chooses it from the
 * input size (spectral-only plans: about 7 MiB per chunk, at most 8 chunks;
 * plans with direct-path scales: 2 chunks from 16 MiB on); n >= 1 asks for
 * n chunks (never more than the batch has clips).  Results do not depend on
 * it.
 * Errors: CWTH_ERR_BAD_PLAN, CWTH_ERR_INVALID_ARG (n < 0).
 */
cwth_status cwth_plan_set_host_chunks(cwth_plan_t plan, int32_t n);

/*
 * Pass plan of the spectral path's inverse FFTs (an autotuner's knob; the
 * result agrees with any other plan within the float32 tolerance):
 * radix 0 restores the plan's cost-model choice, 16 takes radix-16 passes
 * (with a leading 8 / 4), 8 takes radix-8 passes (with a leading 4 / 4,4),
 * which keeps more warps busy when a pass holds few points.  Applies to
 * every spectral part of the plan; later executes use it.
 * Errors: CWTH_ERR_BAD_PLAN; CWTH_ERR_INVALID_ARG for another radix;
 * CWTH_ERR_UNSUPPORTED for 8 when a part's passes cannot take it (pruned
 * inverse FFTs, 1024-thread segments, or more points per pass than eight
 * per thread).
 */
cwth_status cwth_plan_set_inverse_radix(cwth_plan_t plan, int32_t radix);

/*
 * Sizes a plan's growable device workspaces for batches of up to `batch`
 * clips, so that later cwth_execute calls with batch' <= batch allocate
 * nothing (and, with host != 0, cwth_execute_host calls with batch' <= batch
 * and row stride ld_x as well: it also creates the host pipeline's streams
 * and events).  Which workspaces exist depends on the plan (see
 * cwth_execute); a plan without any returns CWTH_OK at once.  Synchronous:
 * growing frees the old buffers (cudaFree waits for the device) and
 * allocates new ones.  No paper counterpart: it only moves allocation out
 * of the calls that transform.
 *   batch  clips, >= 0 (0 is a no-op).
 *   ld_x   row stride in elements of the host input (ignored when host is
 *          0), >= max_len (for a resample-first plan, the longest clip
 *          before re-sampling).
 *   host   nonzero to size cwth_execute_host's staging too.
 * Errors: CWTH_ERR_BAD_PLAN, CWTH_ERR_INVALID_ARG (batch < 0, host != 0 and
 * ld_x too small), CWTH_ERR_UNSUPPORTED (the staged direct-path signal would
 * exceed 2^31 rows), CWTH_ERR_OOM, CWTH_ERR_CUDA.
 */
cwth_status cwth_plan_reserve(cwth_plan_t plan, int32_t batch, int64_t ld_x, int32_t host);

/* Bytes of device memory the direct path's staged bf16 signal needs for
 * `batch` clips (0 for plans without tensor-core scales), written to
 * *bytes: the size a buffer bound by cwth_plan_bind_stage must have for an
 * execute of that batch.  No paper counterpart.
 * Errors: CWTH_ERR_BAD_PLAN, CWTH_ERR_INVALID_ARG (bytes NULL, batch < 0).
 */
cwth_status cwth_plan_stage_bytes(cwth_plan_t plan, int32_t batch, size_t *bytes);

/* Bind a caller-owned device buffer (16-byte aligned, `bytes` long) in
 * which later executes of this plan stage the direct path's bf16 signal,
 * instead of the plan's own growable workspace; NULL unbinds.  The buffer
 * stays the caller's: it must outlive the work enqueued with it bound, and
 * two executes that may run at once must use different buffers (one plan
 * can then serve several streams, each with its own buffer).  An execute
 * whose batch needs more than `bytes` (cwth_plan_stage_bytes) fails with
 * CWTH_ERR_INVALID_ARG before enqueuing anything.  No paper counterpart.
 * Errors: CWTH_ERR_BAD_PLAN, CWTH_ERR_INVALID_ARG (unaligned buffer, or a
 * buffer with bytes == 0).
 */
cwth_status cwth_plan_bind_stage(cwth_plan_t plan, void *buf, size_t bytes);

/* Release a plan's device tables and staging.  NULL is accepted.  The caller
 * must not destroy a plan while work it enqueued may still be running. */
cwth_status cwth_destroy(cwth_plan_t plan);

/* ceil(n / hop), the number of frames b = 0, H, 2H, ... inside [0, n);
 * 0 when n <= 0 or hop <= 0. */
int64_t cwth_num_frames(int64_t n, int32_t hop);

/* Static, human-readable name of a status code. */
const char *cwth_status_string(cwth_status s);

/* Detail of the most recent CUDA or driver failure seen by this library in
 * the calling thread (CUDA error name and text, or which request the driver
 * rejected); "" if none.  The string stays valid until the thread's next
 * failing call. */
const char *cwth_last_error(void);

/* What a plan decided, for tests and benchmarks. */
typedef struct {
    int32_t num_scales;        /* S                                            */
    int32_t hop;               /* H                                            */
    int64_t max_len;           /* longest clip                                 */
    int64_t frames_max;        /* cwth_num_frames(max_len, hop)                */
    int32_t num_spectral;      /* scales on the FFT path                       */
    int32_t num_direct;        /* scales on the direct path                    */
    int32_t seg_len;           /* FFT segment length M (spectral path)         */
    int32_t seg_frames;        /* frames each segment produces                 */
    int32_t seg_halo;          /* samples of left context per segment          */
    int32_t fold_len;          /* P = M / H, the inverse-FFT length            */
    int32_t num_segments;      /* segments per max_len clip                    */
    int32_t direct_taps;       /* padded tap count of the direct path          */
    int64_t table_bytes;       /* device bytes held by the plan's tables       */
    double sample_rate;        /* as given to cwth_plan                        */
    int32_t resample;          /* 1, or H of a cwth_plan_resampled plan (whose
                                  other fields describe its hop-1 transform of
                                  the re-sampled signal)                       */
    int32_t spectral_threads;  /* threads per spectral CTA: 512 (two CTAs per
                                  SM) or 1024 (one); 0 without spectral scales */
    int32_t spectral_pass_scales; /* most scales one spectral CTA folds and
                                  inverts together                             */
    int32_t spectral_pruned;   /* 1 if the inverse FFTs skip the leading passes
                                  that narrow Morlet bands leave trivial       */
    int32_t num_fused;         /* of num_direct: short-support scales summed in
                                  the time domain inside the spectral kernel   */
    int64_t workspace_bytes;   /* device bytes the plan's growable workspaces
                                  hold now (see cwth_execute, cwth_plan_reserve) */
    int32_t spectral_parts;    /* spectral launches per execute: more than 1
                                  when the smallest spectral scales run in
                                  parts with their own, shorter-halo segments
                                  (the other fields describe the part with
                                  the largest scales), 1, or 0 without
                                  spectral scales                            */
    int32_t inverse_radix;     /* main radix of the spectral inverse FFTs'
                                  pass plan (16, or 8 for the radix-8 plan),
                                  0 without folded scales                    */
} cwth_plan_info;

/* Fill *info.  Errors: CWTH_ERR_BAD_PLAN, CWTH_ERR_INVALID_ARG (NULL info). */
cwth_status cwth_plan_query(cwth_plan_t plan, cwth_plan_info *info);

/* Wait for the work enqueued on `stream` and report device-side errors of
 * this plan: CWTH_ERR_TIMEOUT if one of its kernels gave up a bounded wait
 * (the flag is then cleared), CWTH_ERR_CUDA if the stream reported a fault.
 * Errors: CWTH_ERR_BAD_PLAN. */
cwth_status cwth_sync(cwth_plan_t plan, void *stream);

/*
 * Failure-path self-test (the paper has no counterpart): enqueues on
 * `stream` a one-thread kernel that waits on an mbarrier nothing arrives on,
 * for budget_cycles SM clock cycles (1 .. 4e9, i.e. at most about 2 s), and
 * then records CWTH_ERR_TIMEOUT in the plan's device status word, exactly as
 * the tensor-core kernels do when a copy or MMA stage never completes.  The
 * next cwth_sync(plan, stream) returns CWTH_ERR_TIMEOUT and clears the word;
 * the CUDA context stays usable.  Nothing faults or hangs.  plan == NULL
 * targets the status word of cwth_execute_direct_noalloc on the current
 * device instead, which cwth_noalloc_status then reports and clears.
 * Errors: CWTH_ERR_BAD_PLAN (a destroyed or foreign handle),
 * CWTH_ERR_INVALID_ARG (budget out of range), CWTH_ERR_CUDA (allocation of
 * the plan's status word or launch failed).
 */
cwth_status cwth_selftest_wait_timeout(cwth_plan_t plan, int64_t budget_cycles, void *stream);

/*
 * FP32 FMA throughput of the current device in TFLOP/s (no paper
 * counterpart): the roofline denominator of the spectral path.  Runs a few
 * launches of an FMA-only kernel (8 independent chains per thread, every SM
 * full) on `stream`, times them with CUDA events and returns the best.
 * Synchronous; about 10 ms.
 * Errors: CWTH_ERR_INVALID_ARG (NULL tflops), CWTH_ERR_CUDA.
 */
cwth_status cwth_measure_fp32_fma(double *tflops, void *stream);

/* Per-scale path decision: paths[s] = CWTH_PATH_SPECTRAL or CWTH_PATH_DIRECT
 * for s < S (host array of S entries). */
cwth_status cwth_plan_scale_paths(cwth_plan_t plan, int32_t *paths);

/*
 * Uneven batches in one launch (paper Sec. II.B applied to clips of mixed
 * lengths, sample rates, scale counts and hops: one plan per group of
 * clips that share rate, scales and hop).
 *
 * cwth_batch_create binds n groups, each a plan with its device batch,
 * exactly as cwth_execute takes them:
 *   plans[i]      a plan whose every scale takes the float32 spectral path
 *                 (with the short-support scales it sums in the time domain:
 *                 CWTH_PREC_FP32 with CWTH_PATH_AUTO or CWTH_PATH_SPECTRAL),
 *                 without pruned inverse FFTs (cwth_plan_query reports
 *                 spectral_pruned = 0; pruning is taken at hops 1 and 2)
 *                 and not re-sampled;
 *   d_x[i], ld_x[i], d_lengths[i] (may be NULL), batch[i], d_out[i]
 *                 as cwth_execute's arguments for that plan (device memory);
 *   h_lengths     NULL, or n host pointers (each NULL or batch[i] lengths,
 *                 the same as d_lengths[i]): only the segments a clip needs
 *                 become work items.
 * It builds a device work list of (group, clip, segment) items, ordered by
 * the plans' cost models, largest first, and allocates it (the only
 * allocation; cwth_batch_destroy frees it).  cwth_batch_execute then runs
 * every group with ONE kernel launch on `stream` (one block per item, the
 * hardware's block scheduler dealing them to the SMs as they free up); it
 * allocates nothing and can be repeated, also from a captured CUDA graph.
 * The result is the same as cwth_execute of each group within the float32
 * tolerance (the groups' plans fold their scales in one pass).  The bound
 * buffers and plans must outlive the batch; a batch may be executed on one
 * stream at a time.
 *
 * Errors: CWTH_ERR_INVALID_ARG (NULL arrays, n outside 1..96, a batch
 * outside 0..65535, ld_x below the plan's max_len, plans on different
 * devices), CWTH_ERR_BAD_PLAN, CWTH_ERR_UNSUPPORTED (a plan with
 * tensor-core or SIMT direct scales, pruned inverse FFTs, re-sampling, or
 * the one-CTA-per-SM shape), CWTH_ERR_OOM / CWTH_ERR_CUDA.
 */
typedef struct cwth_batch_s *cwth_batch_t;
cwth_status cwth_batch_create(int32_t n, const cwth_plan_t *plans, const float *const *d_x,
                              const int64_t *ld_x, const int64_t *const *d_lengths,
                              const int64_t *const *h_lengths, const int32_t *batch,
                              float *const *d_out, cwth_batch_t *out);
/* One launch over the batch's work list, asynchronous on `stream`.
 * Errors: CWTH_ERR_BAD_PLAN (not a live batch), CWTH_ERR_CUDA. */
cwth_status cwth_batch_execute(cwth_batch_t batch, void *stream);
/* Work items of the batch (blocks per launch), or -1 for a bad handle. */
int64_t cwth_batch_items(cwth_batch_t batch);
/* Release the batch's work list; NULL is accepted.  Not while a launch of
 * it may still be running. */
cwth_status cwth_batch_destroy(cwth_batch_t batch);

/*
 * Allocation-free direct-path scalograms.
 *
 * For callers that cannot allocate device memory while they run: code whose
 * device memory is owned by another allocator (a framework's caching pool),
 * real-time loops where cudaMalloc/cudaFree would synchronise the device or
 * block, and processes that must not grow their footprint after start-up.
 * This call needs no plan and allocates nothing:
 * the tap bank, the per-scale tables, the staged bf16 signal and a status
 * word all live in one array of CWTH_NOALLOC_SCRATCH_BYTES compiled into
 * libcwth.so, which every GPU that loads the library holds until the process
 * exits.  The paper has no counterpart of this call.
 *
 * Computes the same |W| as cwth_plan(..., CWTH_PATH_DIRECT) + cwth_execute:
 *   w, scales, S (1..1024), hop (a multiple of 8), precision
 *   (CWTH_PREC_BF16, CWTH_PREC_BF16X2 or CWTH_PREC_BF16X3) as in
 *   cwth_plan; d_x, ld_x,
 *   d_lengths, batch, d_out, stream as in cwth_execute, with max_len the
 *   longest clip and d_out laid out [batch][S][cwth_num_frames(max_len, hop)].
 *
 * The first call on a device sets that device up (looks up the array's
 * device address, sets the kernels' shared-memory limit, fetches the
 * tensor-map encoder).
 * Every call on a device reuses the same array and leaves the previous call's
 * contents in it (each call rewrites what it reads), so calls whose work
 * overlaps on the GPU - on different streams, or from different threads -
 * race: serialise them, e.g. on one stream.
 *
 * Device-side failures: the tensor-core kernels wait on their copies and
 * MMAs with bounded waits; one that runs out records CWTH_ERR_TIMEOUT in a
 * status word inside the array and its frames are left unwritten.  The word
 * stays set (later calls then skip their work) until cwth_noalloc_status
 * reads and clears it, so check it after the calls whose results you use.
 *
 * Errors: CWTH_ERR_INVALID_ARG for bad arguments and for a request whose
 * scratch would exceed CWTH_NOALLOC_SCRATCH_BYTES (cwth_last_error() states
 * the bytes needed); CWTH_ERR_UNSUPPORTED for a scale needing more than 4096
 * taps; CWTH_ERR_CUDA for a launch failure.  Asynchronous on `stream`.
 */
#define CWTH_NOALLOC_SCRATCH_BYTES (64u << 20)
cwth_status cwth_execute_direct_noalloc(const cwth_morlet *w, const double *scales, int32_t S,
                                        int32_t hop, int32_t precision, const float *d_x,
                                        int64_t ld_x, int64_t max_len, const int64_t *d_lengths,
                                        int32_t batch, float *d_out, void *stream);

/*
 * Status of cwth_execute_direct_noalloc on the current device (no paper
 * counterpart): waits for the work enqueued on `stream`, then reads the
 * status word the allocation-free kernels share and clears it.  Returns
 * CWTH_ERR_TIMEOUT if one of them gave up a bounded wait since the last
 * query, CWTH_OK otherwise; CWTH_ERR_CUDA if the stream reported a fault.
 * Allocates nothing (a synchronous 4-byte copy and, after a timeout, a
 * 4-byte memset of the array).  Sets the device up like the entry point's
 * first call if it has not run yet.
 */
cwth_status cwth_noalloc_status(void *stream);

/* ------------------------------------------------------------------------
 * Continuous-batching server (no paper counterpart: the paper transforms
 * one clip at a time).  Requests, each one clip with its own length, sample
 * rate, scale count and hop, are queued by cwth_server_submit; every
 * cwth_server_poll completes finished batches and launches waiting requests
 * while a stream slot is free and the device-memory budget allows, grouping
 * requests of the same (sample rate, scale count, hop, power-of-two length
 * bucket) into batches of up to max_batch clips.  Plans are cached with
 * their device tables; their bytes count against the budget and the cache
 * evicts the least recently used idle plan when it would exceed
 * plan_cache_bytes.  Each request's samples are read straight from the
 * caller's memory (when page-locked, by one gather kernel per batch that
 * reads them in place over the host link; otherwise one upload per
 * request) and its scalogram is downloaded straight into the caller's
 * buffer (one copy per request; page-locked buffers make it asynchronous).
 * Each slot keeps device buffers for its batches' samples and scalograms
 * (and, for plans with tensor-core scales, the bf16 staged signal, bound
 * to the shared plan for each execute: cwth_plan_bind_stage), grown on
 * demand (at least by half) from a memory pool the server owns,
 * which keeps the blocks a slot outgrew for reuse until
 * cwth_server_destroy; these are not charged to the budget, which limits
 * the bytes of the batches in flight.
 * Not thread-safe: one thread drives a server.
 */
typedef struct cwth_server_s *cwth_server_t;

typedef struct {
    double budget_bytes;      /* device bytes the server may hold: staging
                                 of the batches in flight + cached plans   */
    double plan_cache_bytes;  /* bound on the cached plans' device bytes   */
    int32_t max_batch;        /* clips per batch, 1 .. 4096                */
    int32_t slots;            /* batches in flight (one stream each), 1..64 */
    int32_t precision;        /* CWTH_PREC_* of every plan                 */
    int32_t path;             /* CWTH_PATH_* of every plan                 */
    double f_lo, f_hi;        /* scale band in Hz: S centre frequencies
                                 f_hi (f_lo/f_hi)^(s/(S-1)), s = 0..S-1, with
                                 f_hi capped at fs/2; a_s = C fs / f_s     */
    cwth_morlet wavelet;
    int32_t dry_run;          /* nonzero: no device work at all; plans are
                                 costed by cwth_server_plan_bytes and every
                                 launched batch completes at the next poll
                                 (tests of the admission logic)            */
} cwth_server_config;

typedef struct {
    int64_t rid;              /* caller's id, returned in the completion   */
    const float *x;           /* host, n float32 samples; must stay valid
                                 until the request completes               */
    int64_t n;                /* samples, >= 1                             */
    double fs;                /* sample rate in Hz, > 0                    */
    int32_t n_scales;         /* S >= 1                                    */
    int32_t hop;              /* H >= 1                                    */
    float *out;               /* host, [S][ceil(n / H)] float32 |W|, written
                                 before the completion is reported         */
} cwth_request;

typedef struct {
    int64_t rid;
    int32_t status;           /* CWTH_OK, or the error that failed it      */
    int32_t batch_size;       /* clips in the batch that carried it        */
    double t_done;            /* seconds on the server's clock (since
                                 cwth_server_create) when the poll saw it  */
} cwth_completion;

typedef struct {
    double bytes_in_use;      /* in-flight staging + cached plans          */
    double peak_bytes;
    double plan_bytes;        /* cached plans' device bytes                */
    int32_t plans;            /* cached plans                              */
    int32_t evictions;        /* plans evicted (LRU)                       */
    int64_t launched_batches;
    int64_t completed;
    int64_t rejected;         /* requests that can never fit the budget    */
    int32_t pending;          /* queued, not yet launched                  */
    int32_t in_flight;        /* batches on the GPU                        */
} cwth_server_stats;

/*
 * Creates a server on the current device (streams, events; staging grows on
 * demand).  Errors: CWTH_ERR_INVALID_ARG for a NULL pointer or a field out
 * of range; CWTH_ERR_CUDA.
 */
cwth_status cwth_server_create(const cwth_server_config *cfg, cwth_server_t *out);

/*
 * Queues n requests (host work only).  Errors: CWTH_ERR_INVALID_ARG for a
 * NULL server or request array, or a request with a NULL buffer or a field
 * out of range (nothing is queued then).
 */
cwth_status cwth_server_submit(cwth_server_t s, const cwth_request *reqs, int32_t n);

/*
 * Completes the batches the GPU has finished (their requests' outputs are
 * in place), then admits and launches waiting requests.  Writes up to
 * max_done completions (further ones are kept for the next poll) and
 * returns how many it wrote, or a negative cwth_status.  Requests that
 * could never fit the budget complete with CWTH_ERR_OOM; a plan the path
 * cannot build completes its requests with that plan's error.
 */
int32_t cwth_server_poll(cwth_server_t s, cwth_completion *done, int32_t max_done);

cwth_status cwth_server_stats_query(cwth_server_t s, cwth_server_stats *st);

/*
 * Builds (or finds) the cached plan that requests of (fs, n_scales, hop)
 * with up to n_max samples will use (one plan per key, shared by the
 * slots), so that the first such request does not wait for a plan.
 * Cached plans count against the budget and may be evicted like any other
 * (least recently used first when the plan cache is full).
 * Errors: CWTH_ERR_INVALID_ARG for a NULL server or a field out of range;
 * the plan's own error when the path cannot serve the key.
 */
cwth_status cwth_server_prepare(cwth_server_t s, double fs, int32_t n_scales, int32_t hop,
                                int64_t n_max);

/*
 * Device bytes a plan of the server holds for (fs, S, hop, bucket length):
 * its tables and workspaces (as cwth_plan_query reports table_bytes), the
 * figure the budget charges for it.  In dry-run mode an estimate from the
 * scale count and segment sizes.
 */
double cwth_server_plan_bytes(cwth_server_t s, double fs, int32_t n_scales, int32_t hop,
                              int64_t bucket);

/*
 * Open-loop replay: submits request i at arrival_s[i] seconds after the
 * call starts (host clock) and polls until every request has completed;
 * latency_s[i] = completion time - arrival time, batch_sizes[i] the size of
 * the batch that carried it, status[i] its completion status (any of the
 * three may be NULL).  Requests must be sorted by arrival and have distinct
 * rids.  Returns the wall time in seconds through *wall_s (may be NULL).
 */
cwth_status cwth_server_replay(cwth_server_t s, const cwth_request *reqs,
                               const double *arrival_s, int32_t n, double *latency_s,
                               int32_t *batch_sizes, int32_t *status, double *wall_s);

/* Waits for the batches in flight, then frees plans, staging and streams. */
cwth_status cwth_server_destroy(cwth_server_t s);

#ifdef __cplusplus
}
#endif

#endif /* CWTH_H */
