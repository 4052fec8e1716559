/*
 * orc.h -- CPU oracle for the data-parallel back-end of baseline JPEG decoding
 * (Sodsong et al., "Dynamic Partitioning-based JPEG Decompression on
 * Heterogeneous Multicore Architectures", PMAM'14; Sec. 2 Fig. 1, Sec. 4).
 *
 * TEST INFRASTRUCTURE ONLY.  This code is the plain, slow, obviously correct
 * statement of what the GPU back-end computes.  It is used by the test-suite,
 * by the smoke check and by the CPU-baseline leg of the benchmark, and by
 * nothing else: the product library never links, loads or calls it, and it
 * shares no source, header, table or constant generator with the CUDA path.
 *
 * Integer semantics: every intermediate is int32 with two's-complement wrap
 * (the library is compiled with -fwrapv) and ">>" is an arithmetic shift, so
 * results are defined for every input, including adversarial coefficients.
 *
 * Parity pins (tests/test_oracle_*.py): double-precision Eq. 1-2, the
 * IEEE 1180-1990 accuracy procedure (both IDCT factorisations), the DC-only closed form (exhaustive),
 * DCT->IDCT round trips, Alg. 2 in floating point (exhaustive over 2^24),
 * Alg. 1 as printed, upsampling invariants, and a second naive per-pixel
 * implementation on tiny images.  The particular 13-bit LLM flowgraph is the
 * one choice those pins cannot single out (any accurate factorisation passes
 * them).  It is pinned instead by an independent decoder: NVIDIA's nvJPEG
 * library gives exactly the oracle's RGB bytes (replicated chroma) on the
 * encoder's streams at several qualities, for 4:4:4, 4:2:2, 4:2:0, 4:4:0 and grayscale
 * (tests/test_gpu_nvjpeg.py, which needs a GPU).
 */
#ifndef ORC_H
#define ORC_H
#include <stdint.h>
#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- IDCT (Sec. 4.1, Eq. 1 column pass then Eq. 2 row pass) ---------- */

/* Dequantise (Sec. 2 / Sec. 4.1: F = coefficient x quantisation step) and
 * run the 2-D fixed-point IDCT on one 8x8 block, natural (row-major, row =
 * vertical frequency v, column = horizontal frequency u) order.
 * out[y*8+x] = clamp(level-shifted sample, 0, 255). */
void orc_idct_block(const int16_t coef[64], const uint16_t q[64], uint8_t out[64]);

/* Same transform without level shift or clamp: the rounded 2-D IDCT value
 * (P + 2^17) >> 18 that the IEEE 1180 procedure examines. */
void orc_idct_core(const int16_t coef[64], const uint16_t q[64], int32_t out[64]);

/* Batched forms of the two calls above over n consecutive blocks that share
 * one table (used by the accuracy tests). */
void orc_idct_blocks(const int16_t *coef, const uint16_t q[64], uint8_t *out, int64_t n);
void orc_idct_core_blocks(const int16_t *coef, const uint16_t q[64], int32_t *out, int64_t n);

/* The 12 fixed-point multipliers round(k * 2^13), k from the cosine
 * expressions of the flowgraph; written to k[12] in the order documented in
 * orc_idct.c.  Exposed so a test can pin them to their definitions. */
void orc_idct_constants(int32_t k[12]);

/* The AAN scaled IDCT (orc_idct_aan.c; the algorithm Sec. 2 names): the same
 * transform with the scale factors folded into the dequantisation table and
 * five constant multiplications per 8-point pass, 12 fractional bits.  Same
 * calling conventions as the four calls above; the core value is
 * (Y + 2^14) >> 15. */
void orc_idct_aan_block(const int16_t coef[64], const uint16_t q[64], uint8_t out[64]);
void orc_idct_aan_core(const int16_t coef[64], const uint16_t q[64], int32_t out[64]);
void orc_idct_aan_blocks(const int16_t *coef, const uint16_t q[64], uint8_t *out, int64_t n);
void orc_idct_aan_core_blocks(const int16_t *coef, const uint16_t q[64], int32_t *out, int64_t n);
/* The integer scale table S(v,u) = round(2^12 s_v s_u) ([v*8+u]) and the four
 * 32-bit product constants K1..K4 documented in orc_idct_aan.c. */
void orc_idct_aan_constants(int32_t scale[64], int32_t k[4]);

/* ---- Colour conversion (Sec. 4.3, Alg. 2) ------------------------------ */
void orc_ycc_to_rgb(int y, int cb, int cr, uint8_t rgb[3]);
/* Whole-cube form: rgb[((y*256+cb)*256+cr)*3 + c] for all 2^24 inputs. */
void orc_ycc_to_rgb_all(uint8_t *rgb);

/* ---- Upsampling (Sec. 4.2, Alg. 1) -------------------------------------
 * in: a component plane of its true size cw x ch (row pitch in_pitch);
 * out: the upsampled plane of size (cw*sx) x (ch*sy) (row pitch out_pitch).
 * sx, sy in {1, 2}.  fancy = 0: replication; fancy = 1: triangular. */
void orc_upsample(const uint8_t *in, int cw, int ch, int64_t in_pitch,
                  int sx, int sy, int fancy, uint8_t *out, int64_t out_pitch);

/* ---- Whole back-end (Fig. 1 after entropy decoding) ------------------- */
typedef struct {
    int32_t width, height;        /* image size in pixels */
    int32_t h_samp[3], v_samp[3]; /* sampling factors per component */
    const int16_t *coef[3];       /* component planes, block-row-major,
                                     64 coefficients per block, natural order */
    int32_t blocks_w[3], blocks_h[3];
    const uint16_t *qtab[3];      /* 64 entries, natural order */
    int32_t fancy;                /* 1: triangular upsampling, 0: replication */
    int32_t idct;                 /* 0: LLM IDCT (orc_idct.c), 1: AAN (orc_idct_aan.c) */
} orc_image;

/* Decodes to interleaved RGB, rgb_pitch bytes per row; writes only the
 * W x H pixels.  Returns 0, or -1 if the description is inconsistent. */
int orc_backend_decode(const orc_image *img, uint8_t *rgb, int64_t rgb_pitch);

/* Single-component (grayscale) image: one plane of blocks_w x blocks_h blocks
 * with blocks_w = ceil(W/8), blocks_h = ceil(H/8) (a one-component frame has
 * 8x8 MCUs, T.81 A.2.2), one table.  Each sample Y is written as the RGB
 * triple (Y, Y, Y): the output format is interleaved RGB (Sec. 4.3), and
 * Alg. 2 maps (Y, 128, 128) to (Y, Y, Y).  Returns 0, or -1 if inconsistent. */
int orc_backend_decode_gray(int32_t width, int32_t height, const int16_t *coef, int32_t blocks_w,
                            int32_t blocks_h, const uint16_t q[64], uint8_t *rgb, int64_t rgb_pitch,
                            int32_t idct);

/* Number of threads used by orc_backend_decode_mt (images are split into
 * bands of output rows; the arithmetic is orc_backend_decode's). */
int orc_backend_decode_mt(const orc_image *img, uint8_t *rgb, int64_t rgb_pitch,
                          int nthreads);

/* ---- Entropy decoding (Sec. 2: Huffman, off the data-parallel path) ---- */
/* Parses a baseline (SOF0) JFIF byte stream and Huffman-decodes it into
 * natural-order coefficient planes laid out as orc_image expects.
 * planes[c] must hold blocks_w[c]*blocks_h[c]*64 int16; pass NULL planes to
 * query the geometry only.  Returns 0 on success, < 0 on malformed input. */
typedef struct {
    int32_t width, height, ncomp;
    int32_t h_samp[3], v_samp[3];
    int32_t blocks_w[3], blocks_h[3];
    uint16_t qtab[3][64];         /* natural order */
} orc_jpeg_info;
int orc_jpeg_decode_coefs(const uint8_t *data, int64_t size, orc_jpeg_info *info,
                          int16_t *planes[3]);

#ifdef __cplusplus
}
#endif
#endif
