/*
 * vbw.h - C ABI of libvbw: overlap-save (OLS) fast-convolution filtering with a variable-bandwidth
 * (VBW) filter whose DFT coefficients follow the hybrid frequency-sampling / optimization (HFSO)
 * rule of Moryakova & Johansson, "Efficient Design and Implementation of Fast-Convolution-Based
 * Variable-Bandwidth Filters". GB300 (sm_103a) only.
 *
 * The method (paper Sec. II and Sec. III-B):
 *   - the input is cut into blocks of N samples that overlap by O = N - M samples (Sec. II);
 *   - each block goes through an N-point DFT, a multiply by H(k,b), an N-point IDFT with +j and
 *     1/N (eq. (OLS_dn)), and the first O outputs are discarded (Sec. II, steps 1-5);
 *   - H(k,b) = H_R(k,b) exp(-j 2 pi k (L-1)/2 / N) with L - 1 = O (eq. (FS_Hk_exp)); H_R is 1 in
 *     the passband, V(r) on the L_V transition bins at each band edge and 0 in the stopband
 *     (eq. (FS_Hk_real)), so a bandwidth change moves the table V and computes nothing.
 *
 * Conventions used by every call:
 *   - Samples are complex64: interleaved (re, im) float32 pairs, 8 bytes per sample.
 *   - N is a power of two in [128, 2048]; overlap 0 < O < N; M = N - O. The delay (L-1)/2 = O/2
 *     is a whole number of samples for even O. For odd O it is a half sample: the phase of
 *     eq. (FS_Hk_exp) then uses the signed bin index (k - N above N/2), which keeps the filter
 *     real. FP32 plans only.
 *   - "band" is k1 of eq. (k_var): bins 0..k1-1 (and their mirrors) are passband, the transition
 *     band is k1..k2 with k2 = k1 + L_V - 1, and 1 <= k1 <= N/2 - L_V - 1 (the paper's bounds
 *     Delta_N/2 <= b_N <= N/2 - Delta_N/2 - 1 with b_N = k1 + Delta_N/2 - 1, L_V = Delta_N - 1).
 *   - Stream alignment: O zero samples precede a stream's first sample, so output y(t) is the
 *     filtered x(t) delayed by the filter's group delay O/2 and every input sample yields one
 *     output sample. A final partial block is zero padded; only its valid outputs are written.
 *   - Device pointers are caller-owned (e.g. PyTorch allocations); all filtering calls are
 *     asynchronous on the CUDA stream given at stream or batch creation. Input and output
 *     ranges must not overlap (an overlapping pair is VBW_ERR_INVALID_ARG).
 *   - Errors are return codes; vbw_last_error() gives a thread-local message for the last
 *     failing call on this thread.
 */
#ifndef VBW_H
#define VBW_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct vbw_plan_s* vbw_plan_t;     /* library-owned: N, overlap, V and device tables */
typedef struct vbw_stream_s* vbw_stream_t; /* library-owned: device tail, band, position    */
typedef struct vbw_batch_s* vbw_batch_t;   /* library-owned: device work list of a batch     */

typedef enum {
    VBW_OK = 0,
    VBW_ERR_INVALID_ARG = 1, /* a size, pointer or geometry outside the documented range   */
    VBW_ERR_BAND_RANGE = 2,  /* band (k1) outside [1, N/2 - L_V - 1]                       */
    VBW_ERR_NOMEM = 3,       /* a device or host allocation failed                          */
    VBW_ERR_CUDA = 4,        /* a CUDA runtime call failed (message has the CUDA error)     */
    VBW_ERR_TIMEOUT = 5,     /* a bounded device-side wait gave up                          */
    VBW_ERR_BUSY = 6,        /* no free slot or memory for the request right now            */
    VBW_ERR_STATE = 7,       /* call not allowed in the object's current state              */
    VBW_ERR_UNSUPPORTED = 8  /* valid request that the library does not provide             */
} vbw_status;

/* Arithmetic of a plan's DFT stages:
 *   VBW_PREC_FP32          FP32 register/shared-memory FFT on the CUDA cores (any N, any overlap);
 *   VBW_PREC_BF16_SPLIT    DFT-matrix GEMMs on the tensor cores (tcgen05), operands split into
 *                          bfloat16 hi + lo, products hi*hi + hi*lo + lo*hi, FP32 accumulation;
 *   VBW_PREC_FP16_SCALED   the same with float16 hi + lo pieces of each data row scaled into
 *                          (-1, 1) by a power of two (scaled back exactly after the product);
 *   VBW_PREC_BF16_SPLIT3   bfloat16 hi + mid + lo, six products.
 * The tensor-core precisions take N in {256, 512} with overlap N/4 (VBW_ERR_UNSUPPORTED otherwise).
 * The DFT matrices and twiddles are generated in FP64 on the GPU at plan time, then split. */
enum { VBW_PREC_FP32 = 0, VBW_PREC_BF16_SPLIT = 1, VBW_PREC_FP16_SCALED = 2, VBW_PREC_BF16_SPLIT3 = 3 };

/* Creates a plan for N-point OLS with the given overlap and the L_V transition samples
 * V(0..L_V-1) of eq. (FS_Hk_real) (host array, read during the call; any finite values, the
 * paper does not restrict them). The device keeps V rounded to float32 and the FFT twiddles,
 * generated in FP64 on the GPU and rounded once. Needs a current CUDA device.
 * Errors: VBW_ERR_INVALID_ARG (N not a power of two in [128, 2048], overlap outside (0, N),
 * L_V outside [1, N/2 - 2], non-finite V, precision unknown), VBW_ERR_NOMEM, VBW_ERR_CUDA. */
vbw_status vbw_plan(int N, int overlap, const double* transition_samples, int L_V, int precision,
                    vbw_plan_t* out);
vbw_status vbw_plan_destroy(vbw_plan_t plan);

/* Geometry of a plan: any output pointer may be NULL. */
vbw_status vbw_plan_info(vbw_plan_t plan, int* N, int* overlap, int* L_V, int* M);

/* Creates a filtering stream on the plan: device state holds the last O input samples (zeros at
 * the start); the band (k1) is validated against the plan. cuda_stream is a cudaStream_t (NULL =
 * legacy default stream); every call on this stream object is ordered on it.
 * Errors: VBW_ERR_BAND_RANGE, VBW_ERR_INVALID_ARG, VBW_ERR_NOMEM, VBW_ERR_CUDA. */
vbw_status vbw_stream_create(vbw_plan_t plan, int band, void* cuda_stream, vbw_stream_t* out);
vbw_status vbw_stream_destroy(vbw_stream_t s);

/* Back to the stream's start: tail zeroed (stream-ordered), position 0, pending changes dropped,
 * band set to `band`. */
vbw_status vbw_stream_reset(vbw_stream_t s, int band);

/* Bandwidth change (eq. (k_var) re-indexing, Sec. III-E: no coefficient is computed). Takes effect
 * at the first block not yet submitted to vbw_filter, i.e. at a block boundary. */
vbw_status vbw_set_bandwidth(vbw_stream_t s, int band);

/* Bandwidth change at an absolute block index of the stream (block >= blocks submitted so far).
 * A later call for the same block replaces the earlier one. Errors: VBW_ERR_BAND_RANGE,
 * VBW_ERR_INVALID_ARG (block in the past). */
vbw_status vbw_set_bandwidth_at(vbw_stream_t s, int64_t block, int band);

/* Filters the next nblocks * M samples of the stream: `in` and `out` are device complex64 arrays
 * of nblocks * M samples (Sec. II: block m reads the O previous samples and these M). nblocks = 0
 * is a no-op. Asynchronous; `in` must stay valid until the stream's work completes.
 * Errors: VBW_ERR_INVALID_ARG (NULL or overlapping pointers, nblocks < 0), VBW_ERR_STATE (after
 * vbw_flush), VBW_ERR_CUDA. */
vbw_status vbw_filter(vbw_stream_t s, const void* in, void* out, int64_t nblocks);

/* Ends the stream with a partial block of nvalid samples (0 <= nvalid < M): the block is zero
 * padded after them and only nvalid outputs are written to `out`. After it only vbw_stream_reset
 * is allowed. nvalid = 0 only ends the stream. */
vbw_status vbw_flush(vbw_stream_t s, const void* in, void* out, int nvalid);

/* Same as vbw_filter but `in` and `out` are HOST arrays (pageable or pinned): the call copies the
 * input to the device, filters and copies the result back, pipelined in chunks on the stream's
 * CUDA stream with library-owned device staging, and returns when `out` holds the result. */
vbw_status vbw_filter_host(vbw_stream_t s, const void* in, void* out, int64_t nblocks);

/* Blocks submitted so far (the absolute index of the next block). */
vbw_status vbw_stream_position(vbw_stream_t s, int64_t* blocks);

/* Checkpoint / resume of a stream: the serialized state is (N, overlap, band, position, pending
 * changes, flushed flag, the O-sample tail). vbw_stream_save synchronizes the stream's CUDA
 * stream. With host_buf == NULL it only reports the size in *bytes. vbw_stream_restore needs a
 * stream created on a plan with the same N, overlap and L_V. */
vbw_status vbw_stream_save(vbw_stream_t s, void* host_buf, size_t* bytes);
vbw_status vbw_stream_restore(vbw_stream_t s, const void* host_buf, size_t bytes);

/* One signal of a batch: a whole stream filtered from a zero history (the paper's stream start).
 * band_per_block (host, ceil(nsamples / M) entries) gives k1 for every block; when it is NULL
 * every block uses `band`. */
typedef struct {
    vbw_plan_t plan;               /* geometry and transition table of this signal          */
    const void* in;                /* device complex64 [nsamples]                           */
    void* out;                     /* device complex64 [nsamples]                           */
    int64_t nsamples;              /* >= 0; the final partial block is zero padded          */
    int32_t band;                  /* k1 for every block when band_per_block is NULL        */
    const int32_t* band_per_block; /* host, optional                                       */
} vbw_signal;

/* Prepares a batch of signals, which may use different plans (mixed N): validates every band,
 * builds and uploads the device work list (synchronous, allocates). The batch records the
 * signal pointers; the caller keeps those arrays allocated while the batch is used. */
vbw_status vbw_batch_create(const vbw_signal* signals, int nsignals, vbw_batch_t* out);

/* Prepares a batch of REAL signals (the paper's setting, Sec. III-D): `in` and `out` are device
 * float32 arrays of nsamples real samples (4-byte aligned), band_per_block has one entry per real
 * block of M samples. The filter is real (H(N-k) = conj H(k), eq. (FS_Hk_exp)), so the kernels
 * take two consecutive real blocks as the real and imaginary parts of one complex block. One
 * N-point transform pair then yields 2 M real outputs.
 * Where a band change falls on an odd block, the pair would mix two bands. The signal is then cut
 * there into pieces, and each later piece reads its O samples of history from the signal itself.
 * Results equal the complex path on x + 0j (real part).
 * Errors: VBW_ERR_INVALID_ARG, VBW_ERR_BAND_RANGE, VBW_ERR_UNSUPPORTED (tensor-core plans,
 * overlap > N/2), VBW_ERR_NOMEM. vbw_batch_run runs it (PER_PLAN launches);
 * vbw_batch_run_host returns VBW_ERR_UNSUPPORTED for it. */
vbw_status vbw_batch_create_real(const vbw_signal* signals, int nsignals, vbw_batch_t* out);

/* Runs a prepared batch on cuda_stream: asynchronous, no allocation, no host-device copy, so it
 * can be captured in a CUDA graph. */
vbw_status vbw_batch_run(vbw_batch_t batch, void* cuda_stream);

/* Runs a prepared batch from HOST buffers: host_in[i] and host_out[i] hold signal i's nsamples
 * samples; the call returns when every host_out is written, ordered after the work already queued
 * on cuda_stream.
 *   - All buffers pinned (cudaHostAlloc / cudaHostRegister, e.g. torch pin_memory): zero copy. The
 *     kernels read and write host memory directly over the coherent CPU-GPU link (Grace-Blackwell
 *     NVLink-C2C), with plain loads and stores; nothing is staged. VBW_ZERO_COPY=0 disables it.
 *   - Otherwise: staged. The batch's device in/out arrays hold the data; copies in (merged where
 *     signals are contiguous on both sides), kernels and copies out are pipelined over groups of
 *     signals on library-owned streams (pageable memory works but serializes the copies). */
vbw_status vbw_batch_run_host(vbw_batch_t batch, const void* const* host_in, void* const* host_out,
                              void* cuda_stream);
vbw_status vbw_batch_destroy(vbw_batch_t batch);

/* Number of kernel launches the last vbw_batch_run of this batch issued (for accounting). */
vbw_status vbw_batch_launches(vbw_batch_t batch, int* launches);

/* How vbw_batch_run executes a batch whose signals use several plans:
 *   VBW_BATCH_PER_PLAN  one persistent full-GPU launch per plan, in sequence;
 *   VBW_BATCH_MIXED     one persistent launch over every plan with overlap N/4 and N <= 1024
 *                       (warps switch the transform size per tile), the other plans launched
 *                       beside it on a forked stream; mixed_share is the share of the SMs for the
 *                       mixed launch (0 = in proportion to the transform work);
 *   VBW_BATCH_AUTO      MIXED when at least two plans mix, else PER_PLAN (the default).
 * Errors: VBW_ERR_INVALID_ARG. */
enum { VBW_BATCH_AUTO = 0, VBW_BATCH_PER_PLAN = 1, VBW_BATCH_MIXED = 2 };
vbw_status vbw_batch_set_mode(vbw_batch_t batch, int mode, double mixed_share);

/* Tuning of the single-plan kernel for transform size N, for every later launch in this process:
 * warps per CTA (4 or 8; 0 = default) and a cap on resident CTAs per SM (0 = as many as fit).
 * The autotuner (paper_2406_14116_gb300/tune.py) measures the choices on the current GPU, keeps
 * them in a JSON cache and applies them through this call. Errors: VBW_ERR_INVALID_ARG. */
vbw_status vbw_tune_set(int N, int warps, int ctas_per_sm);

/* Device status word of a plan's launches (synchronizes the device): bit 0 = a bounded device-side
 * wait gave up (a tensor-core kernel's CTA waited for its MMAs in vain, stopped, and left its
 * remaining outputs unwritten). Returns VBW_ERR_TIMEOUT when bit 0 is set. clear != 0 resets the
 * word. */
vbw_status vbw_plan_status(vbw_plan_t plan, int* flags, int clear);

/* Test hooks, process-wide; 0 turns them off.
 *   bit 0: the failure-detection path. Later launches of tensor-core plans issue no MMAs and
 *          shorten the device wait limit to about a millisecond, so the bounded waits for the
 *          accumulators run out, set the status word and stop the CTA, with no fault. (The FP32
 *          kernels wait on nothing.)
 *   bit 1: the full-band identity. Band checks also accept k1 = N/2 + 1, which puts every bin in
 *          the passband (H_R = 1 in eq. (FS_Hk_real)); the filter then returns its input delayed
 *          by D = O/2 (eq. (FS_Hk_exp)). */
vbw_status vbw_debug_set(int flags);

/* Test hook: D (128 x NN) = A (128 x K) B (K x NN) on the tensor cores through the operand
 * layouts, descriptors, TMEM accumulator and waits the tensor-core OLS kernel uses, with A and B
 * rounded once to 16 bits. flags: bit 0 set = bfloat16, clear = float16; bit 1 set = A stored in
 * MN-major core matrices (the layout of rounds 2 and 4), clear = K-major. K, NN in {32, 64}; host
 * float arrays, row-major. Synchronous; allocates. */
vbw_status vbw_debug_tc_gemm(int flags, int K, int NN, const float* A, const float* B, float* D);

/* Test hook: writes the H_R(k) values (k = 0..N-1) that the filtering kernel applies for `band`,
 * produced by the same device code and register layout, to host_out (N floats). For N = 2048 with
 * overlap N/4 that is the split kernel's (two de-interleaved tables, bins 2k and 2k + 1), which
 * filters every launch that fills the GPU; shorter launches use the four-step kernel's layout.
 * Synchronous. */
vbw_status vbw_debug_export_HR(vbw_plan_t plan, int band, float* host_out);

/* ---- Overlap-add: the other fast-convolution method -----------------------------------------
 *
 * Sec. I names overlap-save (OLS) and overlap-add (OLA) as the two fast-convolution methods and
 * chooses OLS. This call filters with OLA and the same coefficients H(k, b) (eq. (FS_Hk_exp),
 * eq. (FS_Hk_real)): block m takes the M = N - O input samples x(mM .. mM + M - 1), zero padded
 * to N, through the N-point DFT, the multiply by H and the N-point IDFT with 1/N (Sec. II steps
 * 1-3); the N-sample results overlap by O and are added:
 *     y(t) = sum_m z_m(t - mM),  0 <= t - mM < N,
 * written for t = 0..nsamples-1 (samples past the end are zero, the last block's tail beyond the
 * signal is dropped). Like OLS with the frequency-sampled H, OLA is periodically time-varying; the
 * two outputs differ by their aliasing terms and agree exactly when h = IDFT(H) has length L = O + 1.
 *
 * Arguments: plan (FP32 precision, even overlap O <= N/2, else VBW_ERR_UNSUPPORTED); in, out:
 * device complex64, nsignals rows of nsamples samples each, back to back (8-byte aligned, not
 * overlapping); band: k1 of every block, checked against the plan (eq. (k_var)), used when
 * band_per_block is NULL; band_per_block: device int32, nsignals x ceil(nsamples / M) values of k1
 * (row-major, 4-byte aligned), or NULL. Values of band_per_block are not checked: a k1 outside
 * eq. (k_var)'s range gives that block other gains (the kernel still reads only V). Whole signals
 * only (no stream state); asynchronous on cuda_stream (a cudaStream_t, NULL = legacy stream); no
 * allocation.
 * Errors: VBW_ERR_INVALID_ARG, VBW_ERR_BAND_RANGE, VBW_ERR_UNSUPPORTED, VBW_ERR_CUDA. */
vbw_status vbw_filter_ola(vbw_plan_t plan, const void* in, void* out, int64_t nsamples, int nsignals,
                          int band, const int* band_per_block, void* cuda_stream);

/* ---- Design analysis: the PTVIR errors of the filter a plan applies ---------------------------
 *
 * OLS with frequency-sampled coefficients is a periodically time-varying system (Sec. II): output
 * phase n = 0..M-1 of every block is a time-invariant filter H_n(w, b) (eq. (OLS_Hn)), and the
 * minimax design of V (eq. (minimax), Sec. III-C) bounds the error
 *     E_n(w, b) = H_n(w, b) e^{j w (L-1)/2} - d(w)            (eq. (err_min), eq. (VBW_des))
 * over every phase, band and grid frequency. This call evaluates that error on the GPU for the
 * plan's geometry (N, overlap O = L - 1) and its transition samples V (as the filter applies
 * them, rounded to float32), building each band's impulse response h = IDFT(H) (eq. (OLS_dn)) in
 * the kernel from (k1, V) alone.
 *
 * Arguments (all arrays are device memory, row-major, owned by the caller):
 *   bands    nbands int32 values k1 (one band per row; 0 <= nbands <= 65535)
 *   omega    nbands x K doubles: the grid frequencies w of each row, radians per sample
 *   desired  nbands x K floats: the desired value d(w) at each point (1 passband, 0 stopband for
 *            eq. (VBW_des); any real value is accepted)
 *   err      nbands x K floats written: max over n of |E_n(w, b)|
 *   phase    nbands x K int32 written: the smallest n reaching that maximum (may be NULL)
 * A row whose k1 lies outside the range of eq. (k_var) (1 <= k1 <= N/2 - L_V - 1) gets NaN in err
 * and -1 in phase. Asynchronous on cuda_stream (a cudaStream_t, NULL = legacy stream); no
 * allocation. Arithmetic is float32 with exactly reduced angles and compensated running sums: each
 * err value is within 1e-6 x max(1, sum_q |h(q)|) of the exact modulus (measured: about 1e-7 x
 * that sum).
 * Errors: VBW_ERR_INVALID_ARG (null plan or array, sizes, misaligned arrays, plan of another
 * device), VBW_ERR_CUDA (launch). */
vbw_status vbw_ptvir_error(vbw_plan_t plan, const int* bands, int nbands, const double* omega,
                           const float* desired, int K, float* err, int* phase, void* cuda_stream);

/* Filters one whole signal without allocating anything. This is for callers that cannot
 * allocate device memory: a host framework that owns every device allocation through its own
 * pool, a real-time loop that cannot afford cudaMalloc's device synchronization and latency, or
 * code that must not touch the CUDA allocator at all. The paper has no counterpart; it is a
 * deployment convenience.
 *
 * Behaviour: as a batch of one signal (zero history, final partial block zero padded), with plan
 * geometry (N, overlap, L_V = transition samples, host doubles read during the call) and band
 * k1, on cuda_stream (a cudaStream_t, NULL = legacy stream). The caller passes device complex64
 * `in` and `out` of nsamples samples (8-byte aligned, not overlapping). The twiddle rows and the
 * float32 transition table live in one fixed 64 KiB array of device memory that belongs to the
 * library image. Every GPU that loads the library holds it until the
 * process exits.
 *
 * The first call on a device looks up that array's device address, with the device current, and
 * the library keeps that address for the life of the process: make the first call before any
 * stream capture, and do not call this entry point on a device after a cudaDeviceReset of it.
 * Every call shares the array: a call rewrites its tables unless they already hold the same
 * geometry and transition table as the previous call on that device, so calls that overlap on the
 * GPU race. Order them on one stream, or synchronize between them. The transition table reaches
 * the GPU inside the launch parameters (no copy from host memory), so the call does not wait on
 * the host for the stream. The call itself makes no cudaMalloc/cudaFree and calls no allocating
 * library routine. Requests beyond the array's capacity are rejected with VBW_ERR_INVALID_ARG;
 * every geometry vbw_plan accepts fits.
 *
 * Errors: VBW_ERR_INVALID_ARG, VBW_ERR_BAND_RANGE, VBW_ERR_CUDA. Device-side wait timeouts are not
 * reported by this call. */
vbw_status vbw_filter_static(int N, int overlap, const double* transition_samples, int L_V,
                             int band, const void* in, void* out, int64_t nsamples,
                             void* cuda_stream);

/* ---- Serving: continuous batching of many live streams ----------------------------------------
 *
 * The paper filters one stream whose band changes at block boundaries (Sec. II, Sec. III-B). A
 * serving deployment runs that filter on many independent streams at once, each sending chunks of
 * any length at any time. The server keeps each stream's OLS state on the device (the O-sample
 * tail and the fewer than M input samples that do not fill a block yet), merges the chunks queued
 * at a moment into batches, and runs them through the fused kernels of the batch path.
 *
 * Chunks are admitted first in first out into one of `slots` batch slots, each an equal share of
 * a device pool of `pool_bytes`. A batch takes chunks from the head of the queue while their input
 * and output blocks fit its slot (admission by memory). A slot is free again once its batch's
 * outputs are on the host. Up to `slots` batches are in flight, so one batch's copies overlap
 * another's kernels.
 *
 * Semantics per stream. The output is the same as vbw_filter over the concatenated chunks,
 * followed by vbw_flush at close, bit for bit, whatever other streams share the batches:
 *   - a chunk's output is every block its samples complete: ((S + n) / M - S / M) * M samples,
 *     with S the samples submitted before it. It is written to host_out from the stream's output
 *     position floor(S / M) * M onward;
 *   - a band change carried by a chunk (new_band >= 0) takes effect at block ceil(S / M), the first
 *     block boundary at or after the chunk's first sample. Of several changes due at one block,
 *     the last one submitted wins;
 *   - vbw_server_close_stream emits the final partial block (S mod M samples, zero padded); the
 *     stream slot can then be opened again.
 * host_in must stay unchanged and host_out untouched until the chunk's completion is returned.
 * Pinned host memory (cudaHostAlloc) gives asynchronous copies. Pageable memory works but is
 * copied synchronously by the CUDA runtime.
 *
 * Threading: a server is not thread safe; one host thread drives it. */
typedef struct vbw_server_s* vbw_server_t;

typedef struct {
    uint64_t tag;        /* the tag given at submit / close                                      */
    int32_t stream;      /* stream index                                                         */
    int32_t final_flush; /* 1 for the completion of vbw_server_close_stream                      */
    int64_t produced;    /* output samples written to the chunk's host_out                       */
    double t_submit;     /* vbw_server_clock() when the chunk was submitted                      */
    double t_done;       /* vbw_server_clock() when the engine saw the chunk's outputs on the host */
} vbw_completion;

typedef struct {
    int64_t queued;            /* chunks submitted, not yet admitted                             */
    int64_t inflight_batches;  /* batches launched, not yet retired                              */
    int64_t completions_ready; /* completions retired, not yet returned                          */
    int64_t batches;           /* batches launched since creation                                */
    int64_t launches;          /* kernel launches since creation                                 */
    int64_t admitted;          /* chunks admitted since creation                                 */
    int64_t slot_bytes;        /* device bytes per batch slot                                    */
    int64_t slots;             /* batch slots                                                    */
} vbw_server_stats;

/* Creates a server for streams that use one of `plans` (all on the current device; the plans
 * must outlive the server). max_streams: stream indices 0..max_streams-1; their state is
 * allocated here (2 O + M samples each). pool_bytes: device memory for batch inputs and outputs,
 * split into `slots` (1..64) equal slots.
 * Errors: VBW_ERR_INVALID_ARG (a NULL plan, more than 64 plans, a slot smaller than 8 M samples),
 * VBW_ERR_NOMEM. */
vbw_status vbw_server_create(const vbw_plan_t* plans, int nplans, int max_streams, size_t pool_bytes,
                             int slots, vbw_server_t* out);

/* Waits for every batch in flight, then frees the server. Chunks still queued are dropped. */
vbw_status vbw_server_destroy(vbw_server_t server);

/* Opens stream index `stream` with plan plans[plan] and band k1 = band: zero history, position 0.
 * Errors: VBW_ERR_INVALID_ARG, VBW_ERR_BAND_RANGE, VBW_ERR_STATE (the stream is open or closing). */
vbw_status vbw_server_open_stream(vbw_server_t server, int stream, int plan, int band);

/* Queues n input samples (host, complex64, 8-byte aligned) of an open stream. new_band: k1 from
 * block ceil(S / M) on, or -1 for none. host_out: room for out_capacity samples, at least the
 * chunk's output count (it may be NULL when that count is 0). tag comes back in the completion.
 * Nothing runs until vbw_server_poll or vbw_server_wait.
 * Errors: VBW_ERR_INVALID_ARG (bad pointer, too small an output, a chunk whose job cannot fit
 * one slot), VBW_ERR_BAND_RANGE, VBW_ERR_STATE (stream not open, or closing). */
vbw_status vbw_server_submit(vbw_server_t server, int stream, const void* host_in, int64_t n, int new_band,
                             void* host_out, int64_t out_capacity, uint64_t tag);

/* One chunk for vbw_server_submit_many: the arguments of vbw_server_submit. */
typedef struct {
    int32_t stream;
    int32_t new_band;      /* -1: no change */
    const void* host_in;
    int64_t n;
    void* host_out;
    int64_t out_capacity;
    uint64_t tag;
} vbw_request;

/* vbw_server_submit for count chunks in order, in one call (no per-chunk call overhead for the
 * caller). Stops at the first chunk that fails and returns its status; *submitted is the number
 * queued before it. */
vbw_status vbw_server_submit_many(vbw_server_t server, const vbw_request* requests, int count, int* submitted);

/* Queues the end of an open stream. Its completion carries the final partial block (S mod M
 * samples, written to host_out) and final_flush = 1. The stream can be opened again after
 * this call returns. Errors: VBW_ERR_INVALID_ARG (output too small), VBW_ERR_STATE. */
vbw_status vbw_server_close_stream(vbw_server_t server, int stream, void* host_out, int64_t out_capacity,
                                   uint64_t tag);

/* Progresses the engine without blocking: retires finished batches, launches batches into free
 * slots, and returns up to max_out completions (oldest first) in out[0 .. *nout). Completions come
 * in submission order. Errors: VBW_ERR_INVALID_ARG, VBW_ERR_CUDA (a batch failed). */
vbw_status vbw_server_poll(vbw_server_t server, vbw_completion* out, int max_out, int* nout);

/* As vbw_server_poll, but if no completion is ready and a batch is in flight, blocks until the
 * oldest batch finishes. Returns *nout = 0 only when nothing is queued or in flight. */
vbw_status vbw_server_wait(vbw_server_t server, vbw_completion* out, int max_out, int* nout);

/* Counters of the engine (see vbw_server_stats). */
vbw_status vbw_server_info(vbw_server_t server, vbw_server_stats* out);

/* The clock of t_submit / t_done: seconds of a monotonic host clock. */
double vbw_server_clock(void);

/* Thread-local description of the last error on this thread ("" if none). */
const char* vbw_last_error(void);

/* Library version string. */
const char* vbw_version(void);

#ifdef __cplusplus
}
#endif

#endif /* VBW_H */
