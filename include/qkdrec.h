/*
 * qkdrec -- GPU hot path of CV-QKD slice reconciliation (B300, sm_103a).
 *
 * The calls follow the paper's statement of reverse slice reconciliation
 * (Ai & Malaney, "Optimised Multithreaded CV-QKD Reconciliation for Global
 * Quantum Networks", arXiv:2108.08418):
 *   Bob quantises y with a constant-step quantiser M(.) into m bits per sample
 *   (Sec. III-B step 1, LSB = l_0), forms slices S_j = bit plane j (step 2) and
 *   sends syndromes s_j = H_j S_j (Sec. II Step 5, Sec. III-B steps 2-3);
 *   Alice computes soft information for slice j from her quadratures x and the
 *   already reconciled lower slices (steps 4-5) and decodes the N_d = N/N_R
 *   sub-blocks of every slice in parallel with BP, all sub-blocks sharing one
 *   H_j (Sec. III-A, Fig. 2; BP decoder of Sec. III-C).
 *
 * Conventions shared by every call
 *   - LLR = ln P(b = 0) / P(b = 1); the hard decision is b = 1 iff LLR < 0.
 *   - A "frame" is one sub-block of length n of one slice (N_R = n).
 *   - Pointers marked DEVICE are CUDA device pointers owned by the caller; the
 *     library never frees them.  Pointers marked HOST are read or written
 *     during the call only.
 *   - `stream` is a cudaStream_t (NULL = the legacy default stream).  Device
 *     work is enqueued asynchronously on it; argument errors are returned
 *     synchronously before anything is enqueued; a CUDA launch error is
 *     returned as QKDREC_ERR_CUDA; a fault inside a kernel surfaces at the
 *     caller's next synchronisation.
 *   - Every call is thread-safe for distinct outputs; the only global state is
 *     a per-thread error string (qkdrec_last_error).
 *   - Sizes of zero are valid and enqueue nothing.
 */
#ifndef QKDREC_H
#define QKDREC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    QKDREC_OK = 0,
    QKDREC_ERR_ARG = 1,          /* bad pointer, size, option or workspace too small */
    QKDREC_ERR_CSR = 2,          /* malformed parity-check matrix */
    QKDREC_ERR_CUDA = 3,         /* a CUDA runtime call or launch failed */
    QKDREC_ERR_NOMEM = 4,        /* device or host allocation failed (code objects only) */
    QKDREC_ERR_TIMEOUT = 5,      /* a bounded device-side wait gave up */
    QKDREC_ERR_UNSUPPORTED = 6   /* valid request this build does not implement */
} qkdrec_status;

typedef enum {
    QKDREC_SP_FLOOD = 0,         /* sum-product, flooding schedule */
    QKDREC_OMS_FLOOD = 1,        /* offset min-sum, flooding schedule */
    QKDREC_OMS_LAYERED = 2       /* offset min-sum, layered schedule (greedy layers) */
} qkdrec_algo;

typedef enum {
    QKDREC_F32 = 0,              /* FP32 messages and posteriors */
    QKDREC_F16MSG = 1,           /* FP16 stored messages, FP32 arithmetic and posteriors */
    QKDREC_I8SAT = 2             /* 6-bit integer min-sum: int8 messages (+-31), int16 posteriors */
} qkdrec_prec;

typedef enum {
    QKDREC_LABEL_GRAY = 0,       /* label(k) = k xor (k >> 1)  (Sec. II Step 4) */
    QKDREC_LABEL_BINARY = 1      /* label(k) = k */
} qkdrec_label;

/* Opaque parity-check matrix H_j, with device copies and derived schedules. */
typedef struct qkdrec_code_s *qkdrec_code_t;

/* ------------------------------------------------------------------ codes */

/*
 * Create a code from H (m_checks x n) in CSR form (the matrix Bob and Alice
 * agree on for one slice, Sec. II Step 5; shared by all sub-blocks, Sec. III-A).
 *   row_ptr  HOST int32 [m_checks + 1], row_ptr[0] = 0, non-decreasing.
 *   col_idx  HOST int32 [row_ptr[m_checks]], variable indices in [0, n).
 *   seed     provenance only (recorded, not used).
 * The arrays are copied; the caller keeps ownership.  The call builds the
 * variable-to-edge map and the layer partition (greedy first fit of checks in
 * index order: check c joins the lowest layer holding none of its variables).
 * Synchronous (allocates and copies to the current device).
 * Errors: QKDREC_ERR_ARG (NULL out/arrays, n <= 0, m_checks <= 0),
 *         QKDREC_ERR_CSR (bad row_ptr, index out of range, a variable twice in
 *         one row), QKDREC_ERR_NOMEM, QKDREC_ERR_CUDA.
 */
qkdrec_status qkdrec_code_create(int32_t n, int32_t m_checks, const int32_t *row_ptr,
                                 const int32_t *col_idx, uint64_t seed, qkdrec_code_t *out);

/* Free a code and its device memory (synchronous).  NULL is ignored. */
void qkdrec_code_destroy(qkdrec_code_t code);

/*
 * Sizes of a code: n, checks M, edges E, number of layers, largest check degree.
 * Any output pointer may be NULL.  HOST outputs.
 */
qkdrec_status qkdrec_code_info(qkdrec_code_t code, int32_t *n, int32_t *m_checks,
                               int64_t *edges, int32_t *n_layers, int32_t *dc_max);

/*
 * Build the seeded parity-check matrix of one slice code (Sec. II Step 5: Bob
 * and Alice agree on H_j; Sec. III-A: one H_j shared by all sub-blocks of the
 * slice).  The paper's code database (Sec. V-B) is not public; this is the
 * random left-regular family that stands in for it:
 *   - n variables of degree dv, m_checks checks; with E = dv n, the first
 *     E - m_checks floor(E / m_checks) checks have degree floor(E / m_checks) + 1,
 *     the others floor(E / m_checks);
 *   - the E variable sockets (socket s belongs to variable s / dv) are placed on
 *     the check sockets in edge order by a uniformly random permutation drawn
 *     from Philox-4x64-10 keyed by (seed, 0) (Fisher-Yates from the last
 *     position, masked-rejection draws; numpy's Generator(Philox(seed)) draws
 *     the same permutation);
 *   - edges on 4-cycles or double edges are swapped with uniformly drawn other
 *     edges (splitmix64 stream of the seed; at most 100 passes; degrees are
 *     kept), then any repeated (check, variable) pair left in dense codes is
 *     swapped away alone, so H never holds a pair twice.
 *   row_ptr   out: HOST int32 [m_checks + 1], allocated by the library;
 *   col_idx   out: HOST int32 [dv n], allocated by the library, check-major edge
 *             order (the layout qkdrec_code_create takes);
 *             release both with qkdrec_free.
 *   cycles4_left  out (may be NULL): 4-cycle / double-edge detections left
 *             after the passes (0 = girth >= 6; dense high-rate codes may keep
 *             some), saturated at INT32_MAX.
 * Synchronous, host only (no device work).  Deterministic in (seed, n,
 * m_checks, dv).
 * Errors: QKDREC_ERR_ARG (NULL outputs, n, dv or m_checks <= 0, m_checks > dv n,
 *         dv n >= 2^31, a check degree above n), QKDREC_ERR_NOMEM.
 */
qkdrec_status qkdrec_make_regular_code(uint64_t seed, int32_t n, int32_t m_checks, int32_t dv,
                                       int32_t **row_ptr, int32_t **col_idx, int32_t *cycles4_left);

/* Release an array the library allocated for the caller (qkdrec_make_regular_code).
 * NULL is ignored. */
void qkdrec_free(void *p);

/* HOST int32 [M]: the layer of every check (the partition the layered decoder uses). */
qkdrec_status qkdrec_code_layers(qkdrec_code_t code, int32_t *layer_of_check);

/*
 * Declare the code quasi-cyclic: H is an mb x nb base matrix of Z x Z circulant
 * permutations, check c = i Z + z holding, in edge order k = 0..nb-1, variable
 * k Z + (z + shifts[i nb + k]) mod Z (HOST int32 shifts [mb][nb], in [0, Z)).
 * The CSR given to qkdrec_code_create is checked against this (QKDREC_ERR_CSR
 * on a mismatch) and the layer partition must be the base rows
 * (QKDREC_ERR_UNSUPPORTED otherwise).  tma_staging = 1: the layered FP32
 * decoder stages each layer chunk's posteriors (a circulant block row is a
 * contiguous run of variables) and messages in shared memory with TMA tile
 * copies instead of per-edge loads; results are identical.  Measured on B300
 * the per-edge path is faster on these codes (their gathers are already
 * sequential), so 0 keeps it.  Synchronous.  The paper's codes (Sec. V-B) are
 * not quasi-cyclic; this is a code layout the decoder can exploit.
 */
qkdrec_status qkdrec_code_set_qc(qkdrec_code_t code, int32_t Z, int32_t mb, int32_t nb, const int32_t *shifts,
                                 int32_t tma_staging);
/* Number of times a quasi-cyclic layer kernel gave up waiting for its tile
 * copies (bounded wait; the chunk is then left undecoded) since the library
 * was loaded.  Synchronous read of a device counter; 0 in normal operation. */
qkdrec_status qkdrec_qc_timeouts(int32_t *count);

/* ------------------------------------------------------- quantiser (Bob) */

/*
 * Constant-step quantiser and bit slicing (Sec. III-B step 1-2; 2^m bins
 * centred on zero, text after Eq. beta).
 *   y         DEVICE float [count]          Bob's quadratures.
 *   m_slices  1..8; bins k = 0 .. 2^m - 1 on [lo, hi], step (hi - lo)/2^m,
 *             interior thresholds t_k = lo + k (hi - lo)/2^m evaluated in FP64;
 *             interval k = number of thresholds t <= y (a sample on a
 *             threshold goes to the upper bin; the outer bins are unbounded).
 *   label     labelling of the interval index (Gray default).
 *   idx_out   DEVICE uint8 [count]          interval index k (may be NULL).
 *   bits_out  DEVICE uint8 [m_slices][count] bit j of label(k), j = 0 the LSB
 *             (may be NULL).
 * Errors: QKDREC_ERR_ARG (count < 0, m out of range, lo >= hi, y NULL with count > 0).
 */
qkdrec_status qkdrec_quantise_slices(const float *y, int64_t count, int32_t m_slices,
                                     double lo, double hi, qkdrec_label label,
                                     uint8_t *idx_out, uint8_t *bits_out, void *stream);

/* -------------------------------------------------------- slice LLR (Alice) */

/*
 * Soft information of slice j for Alice (Sec. III-B steps 4-5, multi-stage
 * hard decoding, Sec. II footnote):
 *   L_j(i) = ln sum_{k in K0(i)} P(k | x_i) - ln sum_{k in K1(i)} P(k | x_i),
 *   K_b(i) = { k : bit j of label(k) = b and bits 0..j-1 of label(k) equal the
 *             reconciled lower bits of sample i },
 *   P(k | x) = Phi((t_{k+1} - x)/sigma_n) - Phi((t_k - x)/sigma_n), t_0 = -inf,
 *   t_{2^m} = +inf, the thresholds of qkdrec_quantise_slices.
 * The result is clipped to [-30, 30].  Three evaluation paths, chosen per
 * sample from each set's nearest candidate (distance d in units of sigma_n):
 *  - saturation: bounds on the two set masses (above: |K_b| times the nearest
 *    term's Gaussian bound; below: a strip of the interval's width at d + width)
 *    show one set more than e^30 below the other -> +-30, no tail evaluated;
 *  - linear FP32 (both nearest candidates within 9 sigma, the common case):
 *    P(k | x) as differences of Gaussian upper tails Q, each from a fitted
 *    Mills ratio (about 1.2e-6 relative), over every candidate or over the
 *    window of candidates whose bound is within e^-16 of its set's lower
 *    bound; L = ln(S0 / S1);
 *  - log domain (a nearest candidate beyond 9 sigma, e.g. wrong lower bits):
 *    each set summed relative to its nearest term in FP32 through the scaled
 *    complementary error function, terms below e^-25 of it skipped, and in
 *    FP64 when both sets lie below e^-50.
 * The result is within 1e-4 max(|L|, 1) of the exact value.
 *   x           DEVICE float [count]       Alice's quadratures.
 *   lower_bits  DEVICE uint8 [j][count]    reconciled slices 0..j-1 (NULL iff j = 0).
 *   llr_out     DEVICE float [count].
 * Errors: QKDREC_ERR_ARG (j outside [0, m), sigma_n <= 0, lo >= hi, NULLs).
 */
qkdrec_status qkdrec_slice_llr(const float *x, int64_t count, int32_t m_slices, int32_t j,
                               double lo, double hi, double sigma_n, qkdrec_label label,
                               const uint8_t *lower_bits, float *llr_out, void *stream);

/* ------------------------------------------------------------------ syndrome */

/*
 * s = H b (mod 2) for F frames (Sec. II Step 5: Bob encodes each slice into
 * syndrome bits; the decoder's stopping test uses the same product).
 *   bits      DEVICE uint8 [F][n]  (values 0/1; only bit 0 is used).
 *   synd_out  DEVICE uint8 [F][M].
 */
qkdrec_status qkdrec_syndrome(qkdrec_code_t code, const uint8_t *bits, int32_t F,
                              uint8_t *synd_out, void *stream);

/* ------------------------------------------------------------------ decoder */

typedef struct {
    int32_t algo;          /* qkdrec_algo */
    int32_t prec;          /* qkdrec_prec; QKDREC_I8SAT needs an OMS algorithm */
    int32_t max_iter;      /* >= 0 */
    float offset;          /* OMS offset beta (float modes); default 0.5 */
    float llr_step;        /* integer mode: LSB of the 6-bit LLR grid; default 0.5 (offset = 1 LSB) */
    int32_t early_stop;    /* 1: stop each frame at the first satisfied syndrome */
    int32_t fallback_f32;  /* frames a low-precision decode leaves unsatisfied are decoded
                              again in FP32: 0 never, 1 with the same algorithm,
                              2 with FP32 sum-product flooding (the plain form).  The
                              failed frames are packed together on the device first, so
                              the second pass costs what they need; each gets exactly the
                              outputs a plain FP32 decode would give it (iterations of
                              both passes added), the other frames keep the first pass's */
} qkdrec_decode_opts;

/* Defaults: SP flooding, FP32, 50 iterations, offset 0.5, step 0.5, early stop on, no fallback. */
void qkdrec_decode_opts_default(qkdrec_decode_opts *opts);

/* Bytes of DEVICE workspace qkdrec_decode_batch needs for F frames of `code`. */
qkdrec_status qkdrec_decode_workspace_size(qkdrec_code_t code, int32_t F,
                                           const qkdrec_decode_opts *opts, size_t *bytes);

/*
 * Syndrome-based BP decoding of F frames that share one code (Sec. III-A:
 * N_d decoders loaded with the same matrix; Sec. III-C: BP decoder).
 * Per frame: L = channel LLR; the syndrome of the hard decision is tested
 * before the first iteration and after every iteration; with early_stop the
 * frame stops at the first success.  The check rule carries the syndrome:
 * a check with s_c = 1 flips the sign of its outgoing messages.
 *   llr         DEVICE float [F][n]   channel LLRs (qkdrec_slice_llr).
 *   synd        DEVICE uint8 [F][M]   Bob's syndrome bits.
 *   bits_out    DEVICE uint8 [F][n]   last hard decision.
 *   iters_out   DEVICE int32 [F]      iterations executed.
 *   conv_out    DEVICE uint8 [F]      1 iff the output satisfies the syndrome.
 *   post_out    DEVICE float [F][n]   final posterior LLRs (may be NULL); in
 *                                     integer mode the integer posterior * llr_step.
 *   workspace   DEVICE, >= qkdrec_decode_workspace_size bytes, 256-byte
 *               aligned; contents need not be initialised and are clobbered.
 * Errors: QKDREC_ERR_ARG (NULLs, F < 0, bad options, workspace too small or
 *         misaligned), QKDREC_ERR_UNSUPPORTED (integer mode with SP),
 *         QKDREC_ERR_CUDA.
 */
qkdrec_status qkdrec_decode_batch(qkdrec_code_t code, const float *llr, const uint8_t *synd,
                                  int32_t F, const qkdrec_decode_opts *opts, uint8_t *bits_out,
                                  int32_t *iters_out, uint8_t *conv_out, float *post_out,
                                  void *workspace, size_t workspace_bytes, void *stream);

/*
 * Slice LLR with the lower slices known softly (Sec. III-B step 4 and its
 * footnote: the soft decoding output of the lower slices gives a-priori
 * reliabilities for slice j):
 *   L_j = ln sum_{k: b_j(k)=0} P(k|x) w_k - ln sum_{k: b_j(k)=1} P(k|x) w_k,
 *   w_k = prod_{l<j} P(b_l = bit l of label(k) | L_l),  P(b = 0 | L) = 1/(1 + e^-L).
 *   lower_post  DEVICE float [j][count]: LLRs of slices 0..j-1 (the decoders'
 *               posteriors; +-inf = a known bit, see qkdrec_bits_to_llr);
 *               NULL allowed when j == 0.
 * With every lower LLR infinite this equals qkdrec_slice_llr with those bits.
 * Other arguments and errors as qkdrec_slice_llr; clipped to +-30.
 */
qkdrec_status qkdrec_slice_llr_soft(const float *x, int64_t count, int32_t m_slices, int32_t j, double lo,
                                    double hi, double sigma_n, qkdrec_label label, const float *lower_post,
                                    float *llr_out, void *stream);

/* Known bits as certain LLRs (0 -> +inf, 1 -> -inf): DEVICE uint8 [count] ->
 * DEVICE float [count]; for slices that are disclosed rather than decoded. */
qkdrec_status qkdrec_bits_to_llr(const uint8_t *bits, int64_t count, float *llr_out, void *stream);

/* ------------------------------------------- whole reconciliation of a block */

/*
 * One sub-block partition of a block (Sec. III-A: the block of N samples is
 * decoded as N_d = N / N_R sub-blocks of length N_R = n, all sharing the
 * slice's parity-check matrix).
 *   n             sub-block length: a positive multiple of 32 dividing count.
 *   codes         HOST array [m_slices]: the code of slice j (length n), or
 *                 NULL for a slice that is disclosed (rate 0: Bob's bits are
 *                 sent in the clear, Sec. II Step 5).
 *   alice_packed  out [m_slices][count / 8]: Alice's reconciled slices, sample i
 *                 of slice j in bit i % 8 of byte j count / 8 + i / 8.
 *   converged     out [m_slices][count / n] (may be NULL): 1 iff the decoded
 *                 sub-block satisfies Bob's syndrome (1 for disclosed slices).
 *   iters         out int32 [m_slices][count / n] (may be NULL): iterations
 *                 (0 for disclosed slices).
 * Each output may be HOST or DEVICE memory (told apart with
 * cudaPointerGetAttributes); host outputs are written by copies on the stream,
 * so they are complete after the caller synchronises the stream.
 */
typedef struct {
    int32_t n;
    const qkdrec_code_t *codes;
    uint8_t *alice_packed;
    uint8_t *converged;
    int32_t *iters;
} qkdrec_point;

/* DEVICE workspace bytes qkdrec_reconcile needs for these arguments (the
 * sizes of the codes, the frame counts and the decoder options) with every
 * partition in flight at once (at most 8); the _limited form sizes it for at
 * most max_in_flight (>= 1) partitions in flight, 1 = one after another. */
qkdrec_status qkdrec_reconcile_workspace_size(int64_t count, int32_t m_slices, const qkdrec_decode_opts *opts,
                                              const qkdrec_point *points, int32_t n_points, size_t *bytes);
qkdrec_status qkdrec_reconcile_workspace_size_limited(int64_t count, int32_t m_slices, const qkdrec_decode_opts *opts,
                                                      const qkdrec_point *points, int32_t n_points,
                                                      int32_t max_in_flight, size_t *bytes);

/*
 * Reverse slice reconciliation of one block of count quadrature pairs, end to
 * end (Sec. II Steps 4-5, Sec. III-B steps 1-5, Sec. III-A):
 *   Bob quantises y (qkdrec_quantise_slices with lo, hi, label) into m_slices
 *   bit planes; for every partition in `points` and every decoded slice j
 *   (LSB first) he forms the syndromes of the sub-blocks; Alice computes the
 *   slice LLRs from x and her already reconciled slices 0..j-1
 *   (qkdrec_slice_llr with sigma_n) and decodes every sub-block
 *   (qkdrec_decode_batch with opts; the FP32 re-decode of opts applies).
 *   Disclosed slices take Bob's bits.  The slices are packed eight to a byte.
 *   The partitions are independent reconciliations of the same block (the
 *   sub-block lengths N_R of the paper's Sec. IV-V comparison).
 *   x, y        float [count], HOST or DEVICE; host memory is copied into the
 *               workspace on the stream (pinned memory lets the copy overlap).
 *   bob_packed  out [m_slices][count / 8] (may be NULL, HOST or DEVICE): Bob's
 *               slices, packed like alice_packed, for checking the result.
 *   workspace   DEVICE, 256-byte aligned, clobbered: at least
 *               qkdrec_reconcile_workspace_size_limited(..., 1) bytes.  The
 *               partitions are decoded concurrently, as many at once as the
 *               workspace holds slots for (qkdrec_reconcile_workspace_size:
 *               all of them, up to 8), each on one of this device's side
 *               streams, forked from `stream` after Bob's slices and joined
 *               back before the call's work ends; with one slot everything
 *               runs on `stream` in order.  Nothing is allocated (the side
 *               streams and their events are created once per device, at the
 *               first call that runs partitions concurrently, which should
 *               come before any stream capture; calls that run partitions
 *               concurrently share them, so two such calls must not be issued
 *               at the same time from different host threads).
 * Asynchronous on `stream`; all argument checks happen before anything is
 * enqueued.  Errors: QKDREC_ERR_ARG (sizes, NULLs, a code whose length is not
 * its partition's n, workspace too small), the errors of the calls above.
 */
qkdrec_status qkdrec_reconcile(const float *x, const float *y, int64_t count, int32_t m_slices, double lo,
                               double hi, double sigma_n, qkdrec_label label, const qkdrec_decode_opts *opts,
                               const qkdrec_point *points, int32_t n_points, uint8_t *bob_packed,
                               void *workspace, size_t workspace_bytes, void *stream);

/* Bits (DEVICE uint8 [count], values 0/1) -> DEVICE packed [count / 8], bit
 * i % 8 of byte i / 8; count a multiple of 32, bits 16-byte and packed 4-byte
 * aligned.  qkdrec_unpack_bits is the inverse (writes 0/1 bytes). */
qkdrec_status qkdrec_pack_bits(const uint8_t *bits, int64_t count, uint8_t *packed, void *stream);
qkdrec_status qkdrec_unpack_bits(const uint8_t *packed, int64_t count, uint8_t *bits, void *stream);

/* ------------------------------------------------ uneven batches (one launch) */

/*
 * Frames whose own SNR sets their quantiser range and noise level: frame f
 * covers samples [frame_offsets[f], frame_offsets[f+1]) of the concatenated
 * arrays (frames of different lengths allowed).  Same results, sample by
 * sample, as qkdrec_quantise_slices / qkdrec_slice_llr called on each frame
 * with its parameters.
 *   frame_offsets  DEVICE int64 [F + 1], non-decreasing, last = count.
 *   frame_ranges   DEVICE double [F][2]: lo, hi of the frame's quantiser.
 *   frame_params   DEVICE double [F][3]: lo, hi, sigma_n of the frame.
 *   bits_out / lower_bits are [m][count] / [j][count] planes of the whole batch.
 *   The per-frame data live on the device and are not validated: ordered
 *   offsets, lo < hi and sigma_n > 0 are the caller's duty (otherwise the values
 *   are meaningless; the kernels clamp each frame's range to [0, count), so every
 *   access stays inside the arrays).
 */
qkdrec_status qkdrec_quantise_slices_frames(const float *y, int64_t count, const int64_t *frame_offsets,
                                            const double *frame_ranges, int32_t F, int32_t m_slices,
                                            qkdrec_label label, uint8_t *idx_out, uint8_t *bits_out,
                                            void *stream);
qkdrec_status qkdrec_slice_llr_frames(const float *x, int64_t count, const int64_t *frame_offsets,
                                      const double *frame_params, int32_t F, int32_t m_slices, int32_t j,
                                      qkdrec_label label, const uint8_t *lower_bits, float *llr_out,
                                      void *stream);

/* One group of an uneven batch: frames that share one code (Sec. III-A: the
 * sub-blocks of a slice share H_j; here many slices and block lengths at once). */
typedef struct {
    qkdrec_code_t code;
    int32_t frames;          /* F_g >= 0 */
    const float *llr;        /* DEVICE float [F_g][n] */
    const uint8_t *synd;     /* DEVICE uint8 [F_g][M] */
    uint8_t *bits_out;       /* DEVICE uint8 [F_g][n] */
    int32_t *iters_out;      /* DEVICE int32 [F_g] */
    uint8_t *conv_out;       /* DEVICE uint8 [F_g] */
} qkdrec_group;

/* Launch shape of a plan; the autotuner searches all combinations.
 *   frames_per_tile 8, 16 or 32: frames decoded together
 *   frames_per_lane 1, 2 or 4, with frames_per_tile / frames_per_lane >= 8:
 *                   frames one lane updates together (2- or 4-wide loads);
 *                   a check of a tile is served by frames_per_tile /
 *                   frames_per_lane lanes
 *   threads_per_cta 256, 512 or 1024
 *   stage_depth     4, 8 or 16: edge loads in flight per lane; with at most
 *                   1024, 512 or 256 threads per CTA at one frame per lane,
 *                   512 or 256 (depth 4 or 8) at two or four (a launch
 *                   outside these pairs returns QKDREC_ERR_UNSUPPORTED)
 *   ctas_per_tile   1, 2, 4 or 8: CTAs of a thread-block cluster sharing one
 *                   tile (they split each layer's checks and meet at the
 *                   cluster barrier after every layer)
 *   tiles_per_item  1, 2 or 4: tiles of one group a team decodes together,
 *                   layer by layer, so one barrier interval holds that many
 *                   tiles' checks of the layer
 *   sparse_frames   0 .. 32: once at most this many frames of a work item are
 *                   still decoding, each lane serves one (check, frame) pair
 *                   (0: never); the tail of a batch -- frames that need many
 *                   iterations -- then spreads every layer over all lanes
 * Every tuning gives the same bits, iteration counts and flags. */
typedef struct {
    int32_t frames_per_tile;
    int32_t threads_per_cta;
    int32_t stage_depth;
    int32_t ctas_per_tile;
    int32_t tiles_per_item;
    int32_t frames_per_lane;
    int32_t sparse_frames;
} qkdrec_tuning;

typedef struct qkdrec_plan_s *qkdrec_plan_t;

/* Defaults: 32 frames per tile, 512 threads, depth 8, 4 CTAs per tile, 1 tile per item,
 * 1 frame per lane, sparse mode from 4 decoding frames. */
void qkdrec_tuning_default(qkdrec_tuning *tuning);

/*
 * Plan the decode of an uneven batch in ONE persistent launch: work items
 * (group, tile of frames_per_tile frames), longest first, taken from a device
 * queue (one atomic increment per item) by thread-block clusters of
 * ctas_per_tile CTAs; no cluster waits for another.  A cluster runs the full
 * layered offset min-sum decode of its tile (Sec. III-C, layered schedule) with
 * the per-frame stopping test, its CTAs splitting each layer's checks.  The plan binds the groups' device pointers (the caller keeps
 * those buffers alive and may refill them between launches).  Synchronous;
 * allocates the plan's small device tables.  Only opts->algo OMS_LAYERED with
 * prec F32 is supported (QKDREC_ERR_UNSUPPORTED otherwise).
 */
qkdrec_status qkdrec_plan_create(const qkdrec_group *groups, int32_t n_groups, const qkdrec_decode_opts *opts,
                                 const qkdrec_tuning *tuning, qkdrec_plan_t *out);
void qkdrec_plan_destroy(qkdrec_plan_t plan);
/* DEVICE workspace bytes for any tuning of the plan. */
qkdrec_status qkdrec_plan_workspace_size(qkdrec_plan_t plan, size_t *bytes);
/*
 * Enqueue the batch decode on `stream`: a memset of the queue head and one
 * kernel launch; no allocation and no host synchronisation, so it can be
 * captured in a CUDA graph.  Launches of one plan must not overlap on the GPU
 * (they share the queue head).
 */
qkdrec_status qkdrec_plan_launch(qkdrec_plan_t plan, void *workspace, size_t workspace_bytes, void *stream);
qkdrec_status qkdrec_plan_get_tuning(qkdrec_plan_t plan, qkdrec_tuning *out);
/*
 * Autotuner: times every launch shape on this plan's batch (iterations capped
 * at max_iter if > 0), then at the fastest shape the sparse-mode thresholds
 * 0, 1, 2, 4, 8; keeps the fastest tuning in the plan and returns it (best_ms = its time).
 * Synchronous; runs real decodes (the outputs are overwritten).
 */
qkdrec_status qkdrec_plan_autotune(qkdrec_plan_t plan, void *workspace, size_t workspace_bytes,
                                   int32_t max_iter, void *stream, qkdrec_tuning *best_out, float *best_ms);

/* ------------------------------------------- differentiable weighted min-sum */

/*
 * Unrolled weighted offset min-sum: T flooding iterations without a stopping
 * test, iteration t scaling and offsetting the check-to-variable magnitudes with
 * learnable weights of the check's degree class (class 0 = the smallest check
 * degree of the code, class 1 = any other):
 *   m_cv = (-1)^{s_c} prod sgn(q) * alpha[t][cls] * max(min_{v'!=v}|q| - beta[t][cls], 0),
 * the min-sum form of the BP check rule of Sec. III-C with per-iteration
 * weights fitted on frames the channel model generates.  Loss = mean over
 * frames and variables of the binary cross-entropy of P(b = 1) = sigmoid(-L^T)
 * against target bits b (Bob's slice bits).
 *   llr     DEVICE float [F][n];  synd DEVICE uint8 [F][M];  target DEVICE uint8 [F][n]
 *   alpha, beta  DEVICE float [T][2]
 *   ckpt_every   iterations between stored message checkpoints (K >= 1); the
 *                backward recomputes each K-iteration segment from them.
 *   workspace    DEVICE, >= qkdrec_woms_workspace_size bytes, 256-byte aligned;
 *                qkdrec_woms_backward must get the same workspace (holding the
 *                forward's checkpoints), inputs and weights as the forward.
 * Forward: loss_out DEVICE float [1]; post_out DEVICE float [F][n] final
 * posteriors (may be NULL).
 * Backward: grad_alpha, grad_beta DEVICE float [T][2], d loss / d weights.  The
 * gradient of a minimum goes to its argmin (ties: lowest edge index),
 * max(x, 0)' = 0 at x <= 0, signs carry no gradient.  Gradients are summed in
 * FP64 over the frames.
 * Errors: QKDREC_ERR_ARG (NULLs, F/T/ckpt_every < 1, workspace too small),
 *         QKDREC_ERR_UNSUPPORTED (check degree above 32).
 */
qkdrec_status qkdrec_woms_workspace_size(qkdrec_code_t code, int32_t F, int32_t T, int32_t ckpt_every,
                                         size_t *bytes);
qkdrec_status qkdrec_woms_forward(qkdrec_code_t code, const float *llr, const uint8_t *synd,
                                  const uint8_t *target, int32_t F, int32_t T, const float *alpha,
                                  const float *beta, int32_t ckpt_every, float *loss_out, float *post_out,
                                  void *workspace, size_t workspace_bytes, void *stream);
qkdrec_status qkdrec_woms_backward(qkdrec_code_t code, const float *llr, const uint8_t *synd,
                                   const uint8_t *target, int32_t F, int32_t T, const float *alpha,
                                   const float *beta, int32_t ckpt_every, float *grad_alpha,
                                   float *grad_beta, void *workspace, size_t workspace_bytes, void *stream);

/*
 * No-allocation variant of qkdrec_decode_batch.  The paper has no counterpart:
 * this serves callers that cannot allocate device memory when they decode --
 * for example code running under a memory manager that owns all of the
 * device's memory, or a latency-critical reconciliation loop in which an
 * allocation (which may synchronise the device) is not allowed.
 * It runs the same decoder on a fixed workspace of
 * qkdrec_decode_static_capacity() bytes (32 MiB) compiled into the library as
 * a device array; every device that uses it holds that array until the process
 * exits.  The caller still passes the inputs and outputs, exactly
 * as for qkdrec_decode_batch.
 *  - A request whose workspace (qkdrec_decode_workspace_size) is larger than
 *    the array fails with QKDREC_ERR_ARG before anything is enqueued; split
 *    the frames over several calls.
 *  - Each call made outside stream capture looks up the array's device
 *    address (cudaGetSymbolAddress) and keeps it; a call made while its stream
 *    is capturing uses the address the last such call found on that device, so
 *    make the first call on a device before any stream capture (otherwise
 *    QKDREC_ERR_ARG).  Under lazy module loading (the CUDA default) the array's
 *    memory is committed by the first call on each device, not when the
 *    library is loaded; if the device has no room left for it then, that call
 *    fails with QKDREC_ERR_NOMEM.
 *  - All calls share the one array.  Calls whose work overlaps on the GPU
 *    (other streams, other host threads) race and corrupt each other's
 *    results: serialise them.  Each call initialises every part of the array
 *    it reads, so what a previous call left there does not matter.
 *  - No cudaMalloc, cudaFree or other allocating routine is called.
 */
size_t qkdrec_decode_static_capacity(void);
qkdrec_status qkdrec_decode_batch_static(qkdrec_code_t code, const float *llr, const uint8_t *synd,
                                         int32_t F, const qkdrec_decode_opts *opts, uint8_t *bits_out,
                                         int32_t *iters_out, uint8_t *conv_out, float *post_out,
                                         void *stream);

/* ------------------------------------------------------------- measurement */

/* Per-kernel-class totals collected between qkdrec_profile_begin/end. */
typedef struct {
    char name[40];         /* kernel class, e.g. "check_flood_sp_f32" */
    int64_t launches;      /* launches recorded */
    double ms;             /* sum of CUDA-event durations of those launches */
    double units;          /* work done: edge updates (check kernels), variable
                              updates (variable kernels), samples (quantiser, LLR),
                              check evaluations (syndrome) -- active frames only */
    double bytes;          /* algorithmic bytes of that work (what the method must
                              move: messages read+written, posteriors gathered, ...) */
} qkdrec_kernel_stat;

/*
 * Start recording: every library launch made after this call (on any stream,
 * from any thread) is bracketed by CUDA events on its stream, and its kernels
 * add their work to device counters.  Allocates a small device buffer.
 * Errors: QKDREC_ERR_ARG if already recording; QKDREC_ERR_CUDA.
 */
qkdrec_status qkdrec_profile_begin(void);

/*
 * Stop recording, synchronise the device, and write up to `capacity` kernel
 * classes (HOST array) with their totals; *count gets the number written.
 * Errors: QKDREC_ERR_ARG if not recording or NULL pointers; QKDREC_ERR_CUDA.
 */
qkdrec_status qkdrec_profile_end(qkdrec_kernel_stat *stats, int32_t capacity, int32_t *count);

/* ------------------------------------------------------------ host helpers */

/*
 * Conditional capacity C_j = 1 - H(B_j | X, B_0 .. B_{j-1}) in bits per sample
 * for x ~ N(0, va), y = x + N(0, 1/snr), the quantiser on [lo, hi] with 2^m
 * bins, by composite Simpson integration over x in [-12 sqrt(va), 12 sqrt(va)]
 * (Sec. II Step 5: the code rate is chosen from the slice's capacity).  HOST.
 */
qkdrec_status qkdrec_slice_capacity(double snr, int32_t m_slices, int32_t j, double lo, double hi,
                                    qkdrec_label label, double va, double *capacity);

/*
 * Rate rule of a slice code (Sec. II Step 5: the code rate is chosen close to
 * the slice's capacity; the workloads take a fraction of it):
 *   rate = k / denom, k = floor(fraction * capacity * denom + 1/2) clamped to
 *   [0, denom - 1] (nearest multiple of 1/denom, ties up; at most
 *   (denom - 1)/denom).  rate = 0 means the slice is disclosed, not decoded.
 * Errors: QKDREC_ERR_ARG (NULL, non-finite capacity or fraction, fraction < 0,
 *         denom outside [2, 2^20]).  HOST.
 */
qkdrec_status qkdrec_code_rate(double capacity, double fraction, int32_t denom, double *rate);

/* Checks of a rate-r code of length n: m = n (1 - rate) rounded to the nearest
 * integer (ties to even).  Errors: QKDREC_ERR_ARG (n <= 0, rate outside [0, 1),
 * m outside [1, n]).  HOST. */
qkdrec_status qkdrec_checks_for_rate(int32_t n, double rate, int32_t *m_checks);

/* Quantiser range of the workloads: [lo, hi] = [-4 sigma_y, 4 sigma_y] with the
 * model value sigma_y^2 = va + 1/snr of y = x + n (the paper's quantiser has a
 * constant step whose size depends on the SNR, Sec. III-B).  Errors:
 * QKDREC_ERR_ARG (NULL, snr or va not positive and finite).  HOST. */
qkdrec_status qkdrec_quantiser_range(double snr, double va, double *lo, double *hi);

/*
 * Reconciliation efficiency of slice reconciliation with code rates R_j
 * (Eq. beta):  beta = (Pi(M(Y)) - m + sum_j R_j) / I_AB,  where Pi(M(Y)) is the
 * entropy in bits of Bob's quantised value (y ~ N(0, va + 1/snr), 2^m bins on
 * [lo, hi] as qkdrec_quantise_slices) and I_AB = 1/2 log2(1 + va snr).  A
 * disclosed slice has R_j = 0 (its bits are revealed).
 *   rates    HOST double [m], each in [0, 1).
 *   beta     out;  entropy  out (may be NULL): Pi(M(Y)) in bits per sample.
 * Errors: QKDREC_ERR_ARG.  HOST.
 */
qkdrec_status qkdrec_reconciliation_efficiency(double snr, int32_t m_slices, double lo, double hi, double va,
                                               const double *rates, double *beta, double *entropy);

/* ------------------------------------------- optimum sub-block length N_R */

/*
 * Parameters of the key-rate optimisation over the sub-block length
 * (Sec. IV-B, Eqs. R_Finite, AEP, FiniteK, BPSRate, simplifiedOpt, diff_eq2;
 * the appendix for S_BE).  The paper's standard settings: N = 1e9, m = 5,
 * eps_EC = 2 eps_s = eps_PA = eps_PE = 2.5e-10, V_A = 5, T = 0.9,
 * xi_ch = 0.0186, xi_d = 0.0133, eta_d = 1, c_h = 3.2e-9 s.
 */
typedef struct {
    double n_signals;                 /* N, quantum signals of the block */
    int32_t m_slices;                 /* m, 1..16 */
    double eps_ec, eps_s, eps_pa, eps_pe;   /* failure probabilities, each in (0, 1/2) */
    double va;                        /* modulation variance V_A */
    double transmissivity;            /* T in (0, 1] */
    double xi_ch, xi_d;               /* channel excess noise, detector noise */
    double eta_d;                     /* detection efficiency in (0, 1] */
    double n_estimation;              /* N_e signals for parameter estimation; <= 0: N / 2 */
    double c_h;                       /* seconds per arithmetic operation of the decoder (Eq. DeltaT) */
    const double *edges_per_sample;   /* HOST [m]: G_j / N_R of slice j's code (0: disclosed slice) */
    const double *iterations;         /* HOST [m]: D_j, decoding iterations of slice j */
    int32_t dispersion_form;          /* 0: A = gamma (gamma+2) / (2 (gamma+1)^2) (log2 e)^2, the
                                         AWGN channel dispersion; 1: as printed, with (log2 eps_EC)^2 */
    double nr_min;                    /* lower end of the N_R range; <= 0: 1e5 (Sec. IV-B) */
} qkdrec_nr_params;

typedef struct {
    double snr;                       /* gamma = (V_A T / 2) / (1 + (xi_ch + xi_d) / 2)   (Eq. SNR) */
    double i_ab;                      /* C(gamma) = 1/2 log2(1 + gamma), bits per sample */
    double dispersion;                /* A */
    double qinv_ec;                   /* Q^-1(eps_EC) */
    double delta_aep;                 /* Delta_AEP (Eq. AEP) */
    double s_be;                      /* S_BE: chi_BE at T^L, xi_ch^U (appendix) */
    double t_low, xi_up;              /* the worst-case estimates T^L, xi_ch^U */
    double b1, b2;                    /* B_1, B_2 of Eq. simplifiedOpt */
    double nr_stationary;             /* root of dK'/dN_R = 0 in the range (0: none) */
    double nr_opt;                    /* maximiser of K'_Finite over the range */
    double key_rate_opt;              /* K'_Finite there, bits per second */
    double d2_key_rate;               /* d^2 K'/dN_R^2 at nr_opt (< 0 at an interior maximum) */
    int32_t at_boundary;              /* 1 if the maximum is at an end of the range */
} qkdrec_nr_result;

/*
 * The N_R that maximises the finite-length key rate in bits per second,
 *   K'(N_R) = (N C_Finite(N_R) - B_1) / (B_2 N_R),
 *   C_Finite(N_R) = C(gamma) - (sqrt(N_R A) Q^-1(eps_EC) + 1/2 log2 N_R) / N_R,
 *   B_1 = N S_BE + sqrt(N) Delta_AEP + 2 log2(1 / (2 eps_PA)),
 *   B_2 = sum_j 7 (G_j / N_R) D_j c_h,
 * over nr_min <= N_R <= N: the stationary point (bisection on ln N_R) or an
 * end of the range, whichever gives the larger K'.  Readings where the paper's
 * formulas are garbled: base-2 logarithms throughout; S_BE from the standard
 * symplectic eigenvalues of reverse reconciliation with heterodyne detection
 * (the squares the appendix drops restored, chi_ch in Psi_2, the detector
 * term (2 - eta_d + 2 xi_d) / eta_d); T^L and xi_ch^U from t^ = sqrt(eta_d T),
 * sigma^2 = T eta_d xi_ch + 1 + xi_d, tau = Q^-1(eps_PE / 2).  HOST only.
 * Errors: QKDREC_ERR_ARG (parameters out of range, B_2 = 0, T^L <= 0).
 */
qkdrec_status qkdrec_nr_optimise(const qkdrec_nr_params *params, qkdrec_nr_result *out);
/* K'_Finite(N_R) in bits per second for one N_R >= 1 (same parameters). */
qkdrec_status qkdrec_nr_key_rate(const qkdrec_nr_params *params, double nr, double *key_rate);

/* Message of the last failing call on this thread ("" if none). */
const char *qkdrec_last_error(void);

/* Library version string. */
const char *qkdrec_version(void);

#ifdef __cplusplus
}
#endif
#endif /* QKDREC_H */
