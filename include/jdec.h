/*
 * jdec.h -- C ABI of the GB300 (sm_103a) back-end of baseline JPEG decoding.
 *
 * The library runs the data-parallel part of the decoder path of Fig. 1
 * (Sodsong et al., PMAM'14, Sec. 2): per-component dequantisation, the 8x8
 * fixed-point IDCT as a column pass (Eq. 1) followed by a row pass (Eq. 2)
 * with range-limit clamping (Sec. 4.1), chroma upsampling by replication or
 * by the triangular filter of Alg. 1 (Sec. 4.2; 4:2:2 as printed, 4:2:0 as the
 * separable extension, 4:4:0 as Alg. 1 along columns), and YCbCr -> RGB by Alg. 2 in 16-bit fixed point
 * (Sec. 4.3), writing interleaved RGB in raster order (Sec. 4.3, Fig. 3-4).
 * Entropy (Huffman) decoding stays on the host (Sec. 2, Sec. 4.5) and is not
 * part of this interface: callers pass entropy-decoded coefficients.
 *
 * Input layout (Sec. 4: "Y blocks followed by Cb blocks followed by Cr
 * blocks"; "an array of short"): one int16 plane per component, blocks in
 * block-row-major order over the padded MCU grid, 64 coefficients per block in
 * natural order (index 8*v + u: row v = vertical frequency, column u =
 * horizontal frequency; zig-zag already undone).  For an image of W x H with
 * Hmax = max h_samp, Vmax = max v_samp: MCUs_x = ceil(W / (8*Hmax)),
 * MCUs_y = ceil(H / (8*Vmax)), component c has blocks_w[c] = MCUs_x*h_samp[c]
 * by blocks_h[c] = MCUs_y*v_samp[c] blocks.  The MCU is 8x8 pixels for 4:4:4
 * and 16x8 for 4:2:2 (Sec. 2), 16x16 for 4:2:0, 8x16 for 4:4:0.
 *
 * Output: 8-bit interleaved R,G,B, rgb_pitch bytes between rows; only the
 * W x H pixels are written, padding bytes of a row are left untouched.
 *
 * The integer result is fully specified (two's-complement int32 wrap,
 * arithmetic shifts, fixed multipliers) and is bit-identical to the CPU
 * oracle for every input; see the repository's design notes for the exact
 * arithmetic.
 *
 * Threading: a context is not thread-safe; use one per host thread.  All
 * decode calls are asynchronous on the given stream (a cudaStream_t passed as
 * void*; NULL = the legacy default stream).  Argument errors are reported
 * synchronously and launch nothing.
 */
#ifndef JDEC_H
#define JDEC_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define JDEC_API __attribute__((visibility("default")))
#else
#define JDEC_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef struct jdec_ctx jdec_ctx;

typedef enum {
    JDEC_OK = 0,
    JDEC_EINVAL = -1,        /* invalid argument or inconsistent geometry   */
    JDEC_ENOMEM = -2,        /* device or pinned-host allocation failed     */
    JDEC_ECUDA = -3,         /* a CUDA runtime call failed                  */
    JDEC_EUNSUPPORTED = -4,  /* valid JPEG, but a sampling or mode the library lacks */
    JDEC_EBUSY = -5,         /* request exceeds the context's HBM budget    */
    JDEC_ETIMEOUT = -6       /* a device-side bounded wait gave up          */
} jdec_status;

/* Upsampling selection (jdec_image.flags).  Fancy = triangular filter
 * (Alg. 1; default), replicate = nearest chroma sample. */
#define JDEC_UPSAMPLE_FANCY     0u
#define JDEC_UPSAMPLE_REPLICATE 1u

/* IDCT selection (jdec_image.flags).  Default: the LLM-form integer IDCT
 * (13-bit multipliers, 2 fractional bits between the passes).  JDEC_IDCT_AAN:
 * the Arai-Agui-Nakajima scaled IDCT that Sec. 2 names -- the 2-D scale
 * factors are folded into the dequantisation table (Q x round(2^12 s_v s_u),
 * s_0 = 1, s_k = sqrt(2) cos(k pi/16)) and each 8-point pass takes five
 * constant products, each an integer part plus the high word of a 32-bit
 * fraction, with 12 fractional bits throughout and one rounding at the end.
 * Both meet the IEEE 1180-1990 accuracy bounds; their samples differ by at
 * most one level on ordinary content.  Each is bit-exact with its oracle. */
#define JDEC_IDCT_AAN 2u

/* Testing aid for failure detection (jdec_image.flags, jdec_decode_coeffs
 * only): the kernel arms its coefficient-load barriers but issues no loads,
 * so every CTA's bounded wait gives up after its limit (2 s), the CTA stops
 * without writing any pixel, and jdec_sync_status returns JDEC_ETIMEOUT.
 * The context stays usable.  Also accepted by jdec_decode_batch_static
 * (jdec_batch_static_status then returns JDEC_ETIMEOUT); rejected
 * (JDEC_EINVAL) by the context-owned batched and host-buffer calls.  Environment variable JDEC_TEST_FAIL_ALLOCS=n (read by
 * jdec_create) makes the context's next n device-buffer allocations fail
 * with JDEC_ENOMEM, for the same purpose. */
#define JDEC_TEST_WITHHOLD_LOADS 0x80000000u

typedef struct {
    int device;               /* CUDA device ordinal                         */
    size_t hbm_budget_bytes;  /* 0 = no limit; bounds context-owned buffers  */
    int max_batch;            /* 0 = default (4096); images per batch call   */
    int autotune;             /* 1 = time tile shapes on first use per shape */
    const char *tune_file;    /* NULL or a JSON file to load/save tile picks */
    int jpeg_chunk_rows;      /* MCU rows per chunk of jdec_decode_jpeg's
                                 pipeline (rounded up to whole restart
                                 intervals when decoding in parallel);
                                 <= 0 = automatic                            */
} jdec_options;               /* a NULL options pointer = all defaults       */

typedef struct {
    int32_t width, height;        /* pixels, 1..65535                          */
    int32_t ncomp;                /* 3 (Y, Cb, Cr), or 1: grayscale -- coef[0],
                                     qtab[0] only, h_samp[0] = v_samp[0] = 1,
                                     blocks = ceil(W/8) x ceil(H/8), output
                                     R = G = B = Y                             */
    uint8_t h_samp[3], v_samp[3]; /* luma (1,1) | (2,1) | (2,2) | (1,2) (4:4:4,
                                     4:2:2, 4:2:0, 4:4:0); chroma (1,1)         */
    const int16_t *coef[3];       /* DEVICE pointers, 16-byte aligned, planes
                                     as described above                         */
    int32_t blocks_w[3], blocks_h[3]; /* must equal MCUs_x*h, MCUs_y*v         */
    const uint16_t *qtab[3];      /* HOST pointers, 64 entries, natural order;
                                     read during the call, not retained         */
    uint8_t *rgb;                 /* DEVICE pointer to the RGB output          */
    int64_t rgb_pitch;            /* bytes per output row, >= 3*width          */
    uint32_t flags;               /* JDEC_UPSAMPLE_* | JDEC_IDCT_AAN
                                     (| JDEC_TEST_*)                            */
} jdec_image;

/* Creates a context on opt->device (default 0).  *out receives the context.
 * No paper passage: context plumbing (device, HBM budget, tile tuner, staging
 * buffers).  Returns JDEC_EINVAL for a NULL `out` or a bad device ordinal,
 * JDEC_ENOMEM/JDEC_ECUDA if the runtime cannot set the context up; *out is
 * then NULL.  The caller owns the context and releases it with jdec_destroy. */
JDEC_API jdec_status jdec_create(jdec_ctx **out, const jdec_options *opt);

/* Decodes one image with one launch of the fused kernel on `stream`: the
 * stages of Sec. 4.1 (dequantisation, Eq. 1 column pass, Eq. 2 row pass with
 * range-limit clamp), Sec. 4.2 (upsampling, Alg. 1), Sec. 4.3 (colour
 * conversion, Alg. 2) merged into one kernel as Sec. 4.4 merges upsampling
 * and colour conversion.  Coefficient and RGB buffers are owned by the caller
 * and must stay valid until the stream has executed the launch.  Returns
 * JDEC_EINVAL without launching for inconsistent descriptions (see
 * jdec_image), JDEC_EUNSUPPORTED for other samplings, JDEC_ECUDA if the
 * launch fails; device-side timeouts are reported by jdec_sync_status. */
JDEC_API jdec_status jdec_decode_coeffs(jdec_ctx *ctx, const jdec_image *img, void *stream);

/* Decodes n images (any mix of sizes and samplings): per variant class one
 * persistent launch over a flattened work list of (image, strip of MCUs, MCU
 * rows) items -- the paper's grouping of MCUs into work-groups of 4 to 32
 * MCUs (Sec. 4; sizes profiled per platform, Sec. 5.1) applied across images
 * -- the launches recorded once per work-list shape as a CUDA graph and
 * replayed with the descriptors of each call.  Per-image results are
 * identical to jdec_decode_coeffs.  1 <= n <= max_batch; the first invalid
 * description's status is returned and nothing is launched.  Buffers as for
 * jdec_decode_coeffs; descriptors are copied into context-owned buffers. */
JDEC_API jdec_status jdec_decode_batch(jdec_ctx *ctx, const jdec_image *imgs, int32_t n, void *stream);

/* Same as jdec_decode_coeffs, but coef[] and rgb point to HOST memory
 * (page-locked for full speed).  The library copies the planes to device
 * buffers it owns, decodes, and copies the RGB back, all on `stream`, in
 * row bands so that copies overlap decoding.  The host buffers must stay
 * valid until the stream has executed the copies. */
JDEC_API jdec_status jdec_decode_host(jdec_ctx *ctx, const jdec_image *img, void *stream);

/* jdec_decode_host for n images in one call: the images are decoded in order,
 * and the copies and decoding of consecutive images overlap (the library
 * stages them in two alternating sets of device buffers it owns; each set
 * grows to the largest image staged in it and counts against the HBM
 * budget).  Stream-ordered on `stream` as a whole: the call
 * starts after earlier work on the stream, and later work waits for the last
 * copy back.  Every description is validated before anything is enqueued
 * (first invalid one -> its status, nothing launched).  Results are identical
 * to n jdec_decode_host calls. */
JDEC_API jdec_status jdec_decode_host_batch(jdec_ctx *ctx, const jdec_image *imgs, int32_t n, void *stream);

/* Synchronises `stream` and reports any device-side error recorded by earlier
 * launches of this context (a bounded wait that gave up -> JDEC_ETIMEOUT).
 * Clears the recorded error.  No paper passage: error plumbing. */
JDEC_API jdec_status jdec_sync_status(jdec_ctx *ctx, void *stream);

/* Releases the context and every buffer, graph and tensor map it owns
 * (synchronising its streams first).  No paper passage: context plumbing.
 * A NULL context returns JDEC_EINVAL. */
JDEC_API jdec_status jdec_destroy(jdec_ctx *ctx);

/* ---- Host-side entropy decoding (Sec. 2: the sequential stage; Sec. 4.5:
 * it runs on the CPU while the GPU back-end works) -------------------------
 * Baseline (SOF0/SOF1), 8-bit, 3-component, single interleaved scan,
 * Huffman coding, optional restart intervals.  Thread-safe; no GPU needed. */
typedef struct {
    int32_t width, height, ncomp;
    uint8_t h_samp[3], v_samp[3];
    int32_t blocks_w[3], blocks_h[3];   /* padded MCU grid, as jdec_image   */
    uint16_t qtab[3][64];               /* natural order                    */
    int32_t restart_interval;           /* MCUs per interval, 0 = none      */
    int64_t scan_offset, scan_bytes;    /* entropy-coded data in the stream */
} jdec_jpeg_info;

/* Parses the headers of a JPEG stream (no entropy decoding).  Returns
 * JDEC_EUNSUPPORTED for progressive, arithmetic or 12-bit streams, for
 * component counts other than 1 and 3 and for sampling factors above 2, and
 * JDEC_EINVAL for malformed ones. */
JDEC_API jdec_status jdec_jpeg_parse(const uint8_t *data, size_t size, jdec_jpeg_info *info);

/* Huffman-decodes the stream into natural-order int16 coefficient planes laid
 * out as jdec_image expects (HOST memory, planes[c] holds blocks_w[c] *
 * blocks_h[c] * 64 int16 as reported by jdec_jpeg_parse). */
JDEC_API jdec_status jdec_entropy_decode(const uint8_t *data, size_t size, int16_t *const planes[3]);

/* Same result with up to `threads` host threads: chunks of MCU rows that
 * start at restart intervals are decoded independently.  A stream without
 * restart intervals is decoded by the calling thread. */
JDEC_API jdec_status jdec_entropy_decode_mt(const uint8_t *data, size_t size, int16_t *const planes[3],
                                            int32_t threads);

/* Decodes a baseline JPEG stream held in HOST memory into DEVICE RGB
 * (rgb_pitch >= 3*width; flags: JDEC_UPSAMPLE_* | JDEC_IDCT_AAN), overlapping host entropy
 * decoding with the device back-end (Sec. 4.5): the MCU rows are cut into
 * chunks; each decoded chunk is copied to context-owned device planes and
 * transformed while the host decodes the next ones.  With restart intervals
 * that fall on chunk boundaries, chunks are entropy-decoded by up to
 * `threads` host threads in parallel; otherwise by the calling thread in
 * order.  Returns when host decoding is done; the device work completes in
 * order on `stream`.  The stream bytes are not needed after the call.
 * Malformed streams return JDEC_EINVAL (rows before the error may already be
 * written); unsupported ones JDEC_EUNSUPPORTED. */
JDEC_API jdec_status jdec_decode_jpeg(jdec_ctx *ctx, const uint8_t *data, size_t size, uint8_t *rgb,
                                      int64_t rgb_pitch, uint32_t flags, int32_t threads, void *stream);

/* Batched decode for callers that cannot allocate device memory (no
 * counterpart in the paper: a deployment need).  Some callers cannot call
 * cudaMalloc: processes whose device memory is all reserved by another
 * allocator (a framework's caching pool that holds the whole HBM), and
 * latency-critical paths where the implicit device-wide synchronisation of
 * cudaMalloc/cudaFree would stall every other stream.  This call needs no
 * context and allocates nothing: descriptors, work list and error word live
 * in one static device array of 512 KiB that every GPU loading the library
 * holds until exit.  Limits: 1 <= n <= 128 images and a work list of at most
 * 16384 items (about 64 strips of one MCU row per image at 128 images);
 * larger requests return JDEC_EINVAL and launch nothing.  Results equal
 * jdec_decode_batch.  Runs on the CURRENT device; the first call on a device
 * looks up the array's device address (cudaGetSymbolAddress) and later calls
 * reuse it.  The descriptors are copied from a
 * static host buffer with a pageable copy, which waits for earlier work on
 * `stream` before it starts; the call returns once they are staged.  All calls
 * share the array and it keeps the last call's contents: calls whose work
 * overlaps on the GPU (different streams) race.  Device-side wait timeouts are
 * recorded in the array's error word, which the next call clears; read it
 * with jdec_batch_static_status before then.  Buffers as for
 * jdec_decode_batch. */
JDEC_API jdec_status jdec_decode_batch_static(const jdec_image *imgs, int32_t n, void *stream);

/* Waits for `stream`, then reports the device-side error word that the last
 * jdec_decode_batch_static call on the current device left in the static
 * array: JDEC_ETIMEOUT if a bounded device wait gave up (that call's output is
 * then incomplete), JDEC_OK if none did.  Clears the word.  Allocates nothing
 * (no counterpart in the paper, like the call it reports on); read it before
 * the next jdec_decode_batch_static call, which clears the word itself. */
JDEC_API jdec_status jdec_batch_static_status(void *stream);

/* Static description of a status code. */
JDEC_API const char *jdec_status_str(jdec_status s);

#ifdef __cplusplus
}
#endif
#endif /* JDEC_H */
