// jdec_device.cuh -- device building blocks of the fused back-end kernel:
// PTX wrappers (TMA, mbarrier, saturating pack), the 1-D integer IDCT, the
// per-block 2-D IDCT over a TMA-swizzled tile, and the per-8-pixel
// upsampling + colour-conversion stage.
//
// Integer arithmetic (Sec. 4.1, Eq. 1 column pass then Eq. 2 row pass):
// the 1-D transform y = M x uses the 13-bit fixed-point matrix of the
// Loeffler-Ligtenberg-Moschytz flowgraph (multipliers round(k * 2^13) of the
// twelve cosine expressions), written here in its collapsed even/odd form:
//   even:  e0 = 8192(x0 + x4) + 10703 x2 +  4433 x6     e3 = ... - (b0)
//          e1 = 8192(x0 - x4) +  4433 x2 - 10704 x6     e2 = ... - (b1)
//   odd:   o_n = sum_k O[n][k] x_k over k = 1, 3, 5, 7
//   y_n = e_n + o_n,  y_{7-n} = e_n - o_n
// Every entry is an exact integer combination of the flowgraph's products,
// so the sums are identical mod 2^32 to evaluating the flowgraph itself.
// Column pass: (y + 2^10) >> 11.  Row pass: (y + 2^17 + 128 * 2^18) >> 18,
// saturated to [0, 255].  int32 arithmetic wraps (two's complement).
#pragma once

#include <cstdint>
#include <cuda.h>
#include "jdec_common.h"

namespace jdec {

// ---------------------------------------------------------------------------
// PTX wrappers
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void *p)
{
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint32_t bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}

__device__ __forceinline__ uint32_t mbar_try_wait(uint32_t bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok;
}

__device__ __forceinline__ uint64_t global_timer_ns()
{
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Bounded wait on an mbarrier phase: returns false if `budget_ns` passed
// without the phase completing (the caller then reports kErrTimeout).
__device__ __forceinline__ bool mbar_wait_bounded(uint32_t bar, uint32_t parity, uint64_t budget_ns)
{
    if (mbar_try_wait(bar, parity)) return true;
    const uint64_t t0 = global_timer_ns();
    for (uint32_t it = 1;; ++it) {
        if (mbar_try_wait(bar, parity)) return true;
        if ((it & 63) == 0 && global_timer_ns() - t0 > budget_ns) return false;
        if (it > (1u << 30)) return false;
    }
}

// Named CTA barriers (ids 1..15): `count` threads (a multiple of 32) take part.
__device__ __forceinline__ void named_sync(int id, int count)
{
    asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(count) : "memory");
}

__device__ __forceinline__ void named_arrive(int id, int count)
{
    asm volatile("bar.arrive %0, %1;" ::"r"(id), "r"(count) : "memory");
}

__device__ __forceinline__ void fence_barrier_init()
{
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void fence_proxy_async_smem()
{
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// 3-D tiled TMA load into shared memory, completion counted on `bar`.
// Coordinates are element indices {inner, block column, block row}; the
// inner coordinate is always 0 (16-byte aligned by construction).
__device__ __forceinline__ void tma_load_3d(uint32_t dst, const CUtensorMap *map, uint32_t bar,
                                            int c0, int c1, int c2)
{
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cta.global.tile.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(dst),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(bar)
        : "memory");
}

// Orders this thread's later TMA uses of a tensor map in global memory after
// the generic-proxy writes that produced it (the host copy of the batch
// descriptors).
__device__ __forceinline__ void tensormap_acquire(const CUtensorMap *map)
{
    asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" ::"l"(reinterpret_cast<uint64_t>(map))
                 : "memory");
}

__device__ __forceinline__ void tma_prefetch_map(const CUtensorMap *map)
{
    asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(map)) : "memory");
}

__device__ __forceinline__ uint4 lds128(uint32_t a)
{
    uint4 v;
    asm volatile("ld.shared.v4.u32 {%0, %1, %2, %3}, [%4];"
                 : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
                 : "r"(a));
    return v;
}

// Saturate four int32 to [0, 255] and pack them as bytes [a, b, c, d].
__device__ __forceinline__ uint32_t pack_sat4(int a, int b, int c, int d)
{
    uint32_t t, r;
    asm("cvt.pack.sat.u8.s32.b32 %0, %1, %2, %3;" : "=r"(t) : "r"(d), "r"(c), "r"(0u));
    asm("cvt.pack.sat.u8.s32.b32 %0, %1, %2, %3;" : "=r"(r) : "r"(b), "r"(a), "r"(t));
    return r;
}

// ---------------------------------------------------------------------------
// 1-D transform (see the header comment).  `rnd` is added to the even
// butterfly inputs, so every output carries it exactly once.  EVEN_ALU: the
// even half leans on the integer ALU instead of the multiply pipe -- the 2^13
// scaling as shifts, the x2/x6 rotation through one shared product
// (4433 (x2 + x6) + 6270 x2 = 10703 x2 + 4433 x6 and 4433 (x2 + x6) - 15137 x6
// = 4433 x2 - 10704 x6, identical mod 2^32); measured faster for the 4:4:4
// kernel only, whose IDCT warps run beside a colour warp.
// ---------------------------------------------------------------------------
template <bool EVEN_ALU = false>
__device__ __forceinline__ void idct8(const int x0, const int x1, const int x2, const int x3,
                                      const int x4, const int x5, const int x6, const int x7,
                                      const int rnd, int y[8])
{
    int a0, a1, b0, b1;
    if constexpr (EVEN_ALU) {
        a0 = ((x0 + x4) << 13) + rnd;
        a1 = ((x0 - x4) << 13) + rnd;
        const int z1 = (x2 + x6) * 4433;
        b0 = z1 + x2 * 6270;
        b1 = z1 - x6 * 15137;
    } else {
        a0 = (x0 + x4) * 8192 + rnd;
        a1 = (x0 - x4) * 8192 + rnd;
        b0 = x2 * 10703 + x6 * 4433;
        b1 = x2 * 4433 - x6 * 10704;
    }
    const int o0 = x1 * 11363 + x3 * 9633 + x5 * 6437 + x7 * 2260;
    const int o1 = x1 * 9633 - x3 * 2259 - x5 * 11362 - x7 * 6436;
    const int o2 = x1 * 6437 - x3 * 11362 + x5 * 2261 + x7 * 9633;
    const int o3 = x1 * 2260 - x3 * 6436 + x5 * 9633 - x7 * 11363;
    // y_n = e_n + o_n, y_{7-n} = e_n - o_n with e_0,3 = a0 +- b0 and
    // e_1,2 = a1 +- b1, each output written as one three-term sum (no shared
    // e_n), so that it is a single three-input add
    y[0] = a0 + (b0 + o0); y[7] = a0 + (b0 - o0);
    y[1] = a1 + (b1 + o1); y[6] = a1 + (b1 - o1);
    y[2] = a1 - (b1 - o2); y[5] = a1 - (b1 + o2);
    y[3] = a0 - (b0 - o3); y[4] = a0 - (b0 + o3);
}

__device__ __forceinline__ int sext_lo(uint32_t w) { return static_cast<int>(static_cast<int16_t>(w & 0xffffu)); }
__device__ __forceinline__ int sext_hi(uint32_t w) { return static_cast<int>(w) >> 16; }

// Two-way dot product of packed signed 16-bit lanes of `a` with unsigned
// bytes of `b` (low: bytes 0,1; high: bytes 2,3), accumulated into c.
__device__ __forceinline__ int dp2a_lo(uint32_t a, uint32_t b, int c)
{
    int d;
    asm("dp2a.lo.s32.u32 %0, %1, %2, %3;" : "=r"(d) : "r"(a), "r"(b), "r"(c));
    return d;
}
__device__ __forceinline__ int dp2a_hi(uint32_t a, uint32_t b, int c)
{
    int d;
    asm("dp2a.hi.s32.u32 %0, %1, %2, %3;" : "=r"(d) : "r"(a), "r"(b), "r"(c));
    return d;
}

// Row pass (Eq. 2) from the column-pass workspace, level shift and
// range-limit clamp; 8 samples per row to dst.
template <bool EVEN_ALU = false>
__device__ __forceinline__ void idct_rows(const int ws[8][8], uint8_t *dst, int pitch)
{
#pragma unroll
    for (int yy = 0; yy < 8; ++yy) {
        int y[8];
        idct8<EVEN_ALU>(ws[yy][0], ws[yy][1], ws[yy][2], ws[yy][3], ws[yy][4], ws[yy][5], ws[yy][6], ws[yy][7],
              (1 << 17) + (128 << 18), y);
        uint2 out;
        out.x = pack_sat4(y[0] >> 18, y[1] >> 18, y[2] >> 18, y[3] >> 18);
        out.y = pack_sat4(y[4] >> 18, y[5] >> 18, y[6] >> 18, y[7] >> 18);
        *reinterpret_cast<uint2 *>(dst + yy * pitch) = out;
    }
}

// Dequantise + 2-D IDCT one block that TMA placed at shared address `blk`
// with the 128-byte swizzle (16-byte chunk c of the 128-byte row at address
// A lives at chunk c ^ ((A >> 7) & 7)).  qt: dequantisation table (int32,
// shared memory, 16-byte aligned) stored transposed, qt[8*u + v] = Q(u, v),
// so each column's eight steps are two 16-byte loads.  Writes the 8x8
// samples to `dst` (shared memory, row pitch `pitch` bytes, 8-byte aligned
// rows).
template <bool EVEN_ALU = false>
__device__ __forceinline__ void idct_block(uint32_t blk, const int *__restrict__ qt, uint8_t *dst, int pitch)
{
    const uint32_t sw = (blk >> 7) & 7u;
    uint32_t w[8][4];
#pragma unroll
    for (int v = 0; v < 8; ++v) {
        const uint4 r = lds128(blk + ((static_cast<uint32_t>(v) ^ sw) << 4));
        w[v][0] = r.x; w[v][1] = r.y; w[v][2] = r.z; w[v][3] = r.w;
    }
    // Eq. 1: column pass over the vertical frequency v for each u.
    int ws[8][8];   // [y][u], 2 fractional bits
#pragma unroll
    for (int u = 0; u < 8; ++u) {
        const int4 qa = *reinterpret_cast<const int4 *>(qt + 8 * u);
        const int4 qb = *reinterpret_cast<const int4 *>(qt + 8 * u + 4);
        const int qv[8] = {qa.x, qa.y, qa.z, qa.w, qb.x, qb.y, qb.z, qb.w};
        int x[8];
#pragma unroll
        for (int v = 0; v < 8; ++v) {
            const uint32_t word = w[v][u >> 1];
            x[v] = ((u & 1) ? sext_hi(word) : sext_lo(word)) * qv[v];
        }
        int y[8];
        idct8<EVEN_ALU>(x[0], x[1], x[2], x[3], x[4], x[5], x[6], x[7], 1 << 10, y);
#pragma unroll
        for (int yy = 0; yy < 8; ++yy) ws[yy][u] = y[yy] >> 11;
    }
    // Eq. 2: row pass over u for each spatial row, level shift, clamp.
    idct_rows<EVEN_ALU>(ws, dst, pitch);
}

// Same transform for quantisation steps that fit in 8 bits: sign extension
// and dequantisation of a coefficient pair take one dp2a each.  qw: 32 words,
// qw[8*p + v] = Q(2p, v) | Q(2p+1, v) << 24 (column pair p, row v).
template <bool EVEN_ALU = false>
__device__ __forceinline__ void idct_block_q8(uint32_t blk, const uint32_t *__restrict__ qw, uint8_t *dst, int pitch)
{
    const uint32_t sw = (blk >> 7) & 7u;
    uint32_t w[8][4];
#pragma unroll
    for (int v = 0; v < 8; ++v) {
        const uint4 r = lds128(blk + ((static_cast<uint32_t>(v) ^ sw) << 4));
        w[v][0] = r.x; w[v][1] = r.y; w[v][2] = r.z; w[v][3] = r.w;
    }
    int ws[8][8];
#pragma unroll
    for (int p = 0; p < 4; ++p) {
        const uint4 qa = *reinterpret_cast<const uint4 *>(qw + 8 * p);
        const uint4 qb = *reinterpret_cast<const uint4 *>(qw + 8 * p + 4);
        const uint32_t qv[8] = {qa.x, qa.y, qa.z, qa.w, qb.x, qb.y, qb.z, qb.w};
        int xl[8], xh[8];
#pragma unroll
        for (int v = 0; v < 8; ++v) {
            xl[v] = dp2a_lo(w[v][p], qv[v], 0);
            xh[v] = dp2a_hi(w[v][p], qv[v], 0);
        }
        int y[8];
        idct8<EVEN_ALU>(xl[0], xl[1], xl[2], xl[3], xl[4], xl[5], xl[6], xl[7], 1 << 10, y);
#pragma unroll
        for (int yy = 0; yy < 8; ++yy) ws[yy][2 * p] = y[yy] >> 11;
        idct8<EVEN_ALU>(xh[0], xh[1], xh[2], xh[3], xh[4], xh[5], xh[6], xh[7], 1 << 10, y);
#pragma unroll
        for (int yy = 0; yy < 8; ++yy) ws[yy][2 * p + 1] = y[yy] >> 11;
    }
    idct_rows<EVEN_ALU>(ws, dst, pitch);
}

// ---------------------------------------------------------------------------
// AAN scaled IDCT (the algorithm Sec. 2 names).  With s_0 = 1 and
// s_k = sqrt(2) cos(k pi / 16), inputs w_k = s_k X_k make the 8-point
// transform cost five constant products: even half P = w2 + w6,
// q = sqrt2 (w2 - w6) - P, e = w0 + w4 +- P, w0 - w4 +- q; odd half
// a = w5 + w3, b = w5 - w3, c = w1 + w7, d = w1 - w7, o0 = a + c,
// z = 2cos(pi/8)(b + d), o1 = z - (2cos(pi/8) + 2sin(pi/8)) b - o0,
// o2 = sqrt2 (c - a) - o1, o3 = z - (2cos(pi/8) - 2sin(pi/8)) d - o2;
// y[n] = e[n] + o[n], y[7-n] = e[n] - o[n].  The 2-D scale factors
// s_v s_u * 2^12 are folded into the dequantisation table on the host, so the
// working values carry 12 fractional bits and need no descale between the
// passes.  Each product is an integer part plus the high word of a 32-bit
// fraction (one mad.hi):
//   sqrt2 t          = t  + hi(t * kA1),  kA1 = round((sqrt2 - 1) 2^32)
//   2c t             = 2t + hi(t * -kA2), kA2 = round((2 - 2c) 2^32)
//   (2c + 2s) t      = 3t - hi(t * kA3),  kA3 = round((3 - 2c - 2s) 2^32)
//   (2c - 2s) t      = t  - hi(t * -kA4), kA4 = round((2c - 2s - 1) 2^32)
// (c = cos(pi/8), s = sin(pi/8)).  Sample = clamp(((Y + 2^14) >> 15) + 128).
// ---------------------------------------------------------------------------
constexpr int kA1 = 1779033704;
constexpr int kA2 = 653869837;
constexpr int kA3 = 1661611479;
constexpr int kA4 = 353871806;

// hi(a * b) + c: the high word of the exact 64-bit product, plus c.
__device__ __forceinline__ int mad_hi(int a, int b, int c)
{
    int d;
    asm("mad.hi.s32 %0, %1, %2, %3;" : "=r"(d) : "r"(a), "r"(b), "r"(c));
    return d;
}

// One 8-point AAN transform of scaled inputs; `bias` reaches every output
// once (it enters through w0, which no product touches).
__device__ __forceinline__ void idct8_aan(const int w0, const int w1, const int w2, const int w3,
                                          const int w4, const int w5, const int w6, const int w7,
                                          const int bias, int y[8])
{
    const int t10 = w0 + bias + w4, t11 = w0 + bias - w4;
    const int P = w2 + w6, D = w2 - w6;
    const int q = mad_hi(D, kA1, D - P);
    const int e0 = t10 + P, e3 = t10 - P, e1 = t11 + q, e2 = t11 - q;
    const int a = w5 + w3, b = w5 - w3, c = w1 + w7, d = w1 - w7;
    const int o0 = a + c, r = c - a, bd = b + d;
    const int z = mad_hi(bd, -kA2, 2 * bd);
    const int o1 = mad_hi(b, kA3, z - 3 * b) - o0;
    const int o2 = mad_hi(r, kA1, r - o1);
    const int o3 = mad_hi(d, -kA4, z - d) - o2;
    y[0] = e0 + o0; y[7] = e0 - o0;
    y[1] = e1 + o1; y[6] = e1 - o1;
    y[2] = e2 + o2; y[5] = e2 - o2;
    y[3] = e3 + o3; y[4] = e3 - o3;
}

// Dequantise with the prescaled table and run both AAN passes on one block
// (layout, swizzle and output as idct_block; qt[8*u + v] = Q(v,u) S(v,u)).
__device__ __forceinline__ void idct_block_aan(uint32_t blk, const int *__restrict__ qt, uint8_t *dst, int pitch)
{
    const uint32_t sw = (blk >> 7) & 7u;
    uint32_t w[8][4];
#pragma unroll
    for (int v = 0; v < 8; ++v) {
        const uint4 r = lds128(blk + ((static_cast<uint32_t>(v) ^ sw) << 4));
        w[v][0] = r.x; w[v][1] = r.y; w[v][2] = r.z; w[v][3] = r.w;
    }
    int ws[8][8];   // [y][u], 12 fractional bits, scaled by s_u
#pragma unroll
    for (int u = 0; u < 8; ++u) {
        const int4 qa = *reinterpret_cast<const int4 *>(qt + 8 * u);
        const int4 qb = *reinterpret_cast<const int4 *>(qt + 8 * u + 4);
        const int qv[8] = {qa.x, qa.y, qa.z, qa.w, qb.x, qb.y, qb.z, qb.w};
        int x[8];
#pragma unroll
        for (int v = 0; v < 8; ++v) {
            const uint32_t word = w[v][u >> 1];
            x[v] = ((u & 1) ? sext_hi(word) : sext_lo(word)) * qv[v];
        }
        int y[8];
        idct8_aan(x[0], x[1], x[2], x[3], x[4], x[5], x[6], x[7], 0, y);
#pragma unroll
        for (int yy = 0; yy < 8; ++yy) ws[yy][u] = y[yy];
    }
#pragma unroll
    for (int yy = 0; yy < 8; ++yy) {
        int y[8];
        idct8_aan(ws[yy][0], ws[yy][1], ws[yy][2], ws[yy][3], ws[yy][4], ws[yy][5], ws[yy][6], ws[yy][7],
                  (1 << 14) + (128 << 15), y);
        uint2 out;
        out.x = pack_sat4(y[0] >> 15, y[1] >> 15, y[2] >> 15, y[3] >> 15);
        out.y = pack_sat4(y[4] >> 15, y[5] >> 15, y[6] >> 15, y[7] >> 15);
        *reinterpret_cast<uint2 *>(dst + yy * pitch) = out;
    }
}

// ---------------------------------------------------------------------------
// Colour conversion (Sec. 4.3, Alg. 2) in 16-bit fixed point.  The chroma
// samples reach it already offset (C' = C - 128: the upsampling filters fold
// the -128 into their rounding constants, and unfiltered samples are read as
// signed bytes of the word XOR 0x80808080), and the luma sample arrives as
// Y * 2^16 + 2^15 (one byte permute places Y and the rounding constant), so
// each channel is one multiply-add and one shift:
//   R = (Y 2^16 + 2^15 + 91881 Cr') >> 16
//   G = (Y 2^16 + 2^15 - 22554 Cb' - 46802 Cr') >> 16
//   B = (Y 2^16 + 2^15 + 116130 Cb') >> 16
// (91881 = round(1.402 * 2^16), 22554, 46802, 116130 likewise); the same
// integers as Y + ((c Cr' + 2^15) >> 16), because Y * 2^16 is a multiple of
// 2^16.  Saturation happens in the byte pack.
// ---------------------------------------------------------------------------

// Byte k of w as an int (PRMT with zero fill).
__device__ __forceinline__ int byte_of(uint32_t w, int k) { return static_cast<int>(__byte_perm(w, 0u, 0x4440u | k)); }

// Byte k of w as a sign-extended int (PRMT sign mode: the msb of a selector
// nibble replicates the sign of the selected byte).  On a word XORed with
// 0x80808080 this is the sample minus 128.
__device__ __forceinline__ int sbyte_of(uint32_t w, int k)
{
    const uint32_t s = static_cast<uint32_t>(k) | ((8u | k) << 4) | ((8u | k) << 8) | ((8u | k) << 12);
    uint32_t r;
    asm("prmt.b32 %0, %1, %2, %3;" : "=r"(r) : "r"(w), "r"(0u), "r"(s));
    return static_cast<int>(r);
}

// Byte k of w placed at bits 16..23 with 0x80 at bits 8..15: Y * 2^16 + 2^15.
__device__ __forceinline__ int y_term(uint32_t w, int k)
{
    return static_cast<int>(__byte_perm(w, 0x8000u, 0x4054u | (static_cast<uint32_t>(k) << 8)));
}

// Bytes [i, i+4) and [i, i+2) of the 24 little-endian bytes in w (i a
// compile-time constant after inlining).
__device__ __forceinline__ uint32_t bytes32(const uint32_t w[6], int i)
{
    return (i & 3) ? __funnelshift_r(w[i >> 2], w[(i >> 2) + 1], 8 * (i & 3)) : w[i >> 2];
}
__device__ __forceinline__ uint16_t bytes16(const uint32_t w[6], int i)
{
    return static_cast<uint16_t>((i & 3) == 3 ? __funnelshift_r(w[i >> 2], w[(i >> 2) + 1], 24) : w[i >> 2] >> (8 * (i & 3)));
}

// Writes 24 bytes to `out` with out % 8 == A (1..7): naturally aligned 1-,
// 2- and 4-byte stores up to the 8-byte boundary, two 8-byte stores, then
// the A remaining bytes with 4-, 2- and 1-byte stores.
template <int A>
__device__ __forceinline__ void store24_at(uint8_t *out, const uint32_t w[6])
{
    constexpr int S = 8 - A;   // bytes below the first 8-byte boundary
    int o = 0;
    if (S & 1) {
        out[0] = static_cast<uint8_t>(w[0]);
        o = 1;
    }
    if ((S - o) & 2) {
        *reinterpret_cast<uint16_t *>(out + o) = bytes16(w, o);
        o += 2;
    }
    if (S - o >= 4) *reinterpret_cast<uint32_t *>(out + o) = bytes32(w, o);
    reinterpret_cast<uint2 *>(out + S)[0] = make_uint2(bytes32(w, S), bytes32(w, S + 4));
    reinterpret_cast<uint2 *>(out + S)[1] = make_uint2(bytes32(w, S + 8), bytes32(w, S + 12));
    int t = S + 16;
    if (A & 4) {
        *reinterpret_cast<uint32_t *>(out + t) = bytes32(w, t);
        t += 4;
    }
    if (A & 2) {
        *reinterpret_cast<uint16_t *>(out + t) = bytes16(w, t);
        t += 2;
    }
    if (A & 1) out[t] = static_cast<uint8_t>(w[5] >> 24);
}

// Writes 24 bytes (little-endian words w[0..5]) to global memory at any
// alignment with naturally aligned stores (three 8-byte stores when out is
// 8-byte aligned).  Neighbouring tasks touch disjoint bytes, so the partial
// words at the ends never race.
__device__ __forceinline__ void store24(uint8_t *out, const uint32_t w[6])
{
    switch (static_cast<int>(reinterpret_cast<uintptr_t>(out) & 7)) {
    case 0: {
        uint2 *o = reinterpret_cast<uint2 *>(out);
        o[0] = make_uint2(w[0], w[1]);
        o[1] = make_uint2(w[2], w[3]);
        o[2] = make_uint2(w[4], w[5]);
        break;
    }
    case 1: store24_at<1>(out, w); break;
    case 2: store24_at<2>(out, w); break;
    case 3: store24_at<3>(out, w); break;
    case 4: store24_at<4>(out, w); break;
    case 5: store24_at<5>(out, w); break;
    case 6: store24_at<6>(out, w); break;
    default: store24_at<7>(out, w); break;
    }
}

// The rarely taken stores of an 8-pixel group, kept out of line so that the
// hot path stays small: the 24 bytes w[0..5] (saturated R, G, B of 8 pixels)
// to a row that is not 8-byte aligned, or the first 3n bytes only (n < 8
// pixels inside the image, at its right edge).
static __device__ __noinline__ void store_group_slow(uint8_t *out, uint32_t w0, uint32_t w1, uint32_t w2, uint32_t w3,
                                              uint32_t w4, uint32_t w5, int n)
{
    const uint32_t w[6] = {w0, w1, w2, w3, w4, w5};
    if (n >= 8) {
        store24(out, w);
        return;
    }
    for (int k = 0; k < 3 * n; ++k) out[k] = static_cast<uint8_t>(w[k >> 2] >> (8 * (k & 3)));
}

// Converts 8 pixels and writes 24 bytes to `out` (global).  yw: the 8 luma
// samples as two words; Cb, Cr: chroma minus 128; `n` = pixels inside the
// image (1..8); `vec`: out is 8-byte aligned.
__device__ __forceinline__ void cc_store8(uint2 yw, const int Cb[8], const int Cr[8], uint8_t *out, int n, bool vec)
{
    int R[8], G[8], B[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        const int ys = y_term(k < 4 ? yw.x : yw.y, k & 3);
        R[k] = (ys + Cr[k] * 91881) >> 16;
        G[k] = (ys - Cb[k] * 22554 - Cr[k] * 46802) >> 16;
        B[k] = (ys + Cb[k] * 116130) >> 16;
    }
    uint32_t w[6];
    w[0] = pack_sat4(R[0], G[0], B[0], R[1]);
    w[1] = pack_sat4(G[1], B[1], R[2], G[2]);
    w[2] = pack_sat4(B[2], R[3], G[3], B[3]);
    w[3] = pack_sat4(R[4], G[4], B[4], R[5]);
    w[4] = pack_sat4(G[5], B[5], R[6], G[6]);
    w[5] = pack_sat4(B[6], R[7], G[7], B[7]);
    if (n == 8 && vec) {
        uint2 *o = reinterpret_cast<uint2 *>(out);
        o[0] = make_uint2(w[0], w[1]);
        o[1] = make_uint2(w[2], w[3]);
        o[2] = make_uint2(w[4], w[5]);
    } else {
        store_group_slow(out, w[0], w[1], w[2], w[3], w[4], w[5], n);
    }
}

// Ten samples p[-1 .. 8] around eight chroma centres starting at the 4-byte
// aligned address p.
__device__ __forceinline__ void load10(const uint8_t *p, int c[10])
{
    const uint32_t l = *reinterpret_cast<const uint32_t *>(p - 4);
    const uint2 m = *reinterpret_cast<const uint2 *>(p);
    const uint32_t r = *reinterpret_cast<const uint32_t *>(p + 8);
    c[0] = byte_of(l, 3);
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        c[1 + k] = byte_of(m.x, k);
        c[5 + k] = byte_of(m.y, k);
    }
    c[9] = byte_of(r, 0);
}

// Alg. 1 (h2v1 triangular) for four centres c[1..4] with neighbours c[0],
// c[5]; outputs minus 128 ((x - 512) >> 2 = (x >> 2) - 128).
__device__ __forceinline__ void tri_h2v1(const int c[6], int o[8])
{
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const int t = 3 * c[k + 1];
        o[2 * k] = (t + c[k] + 1 - 512) >> 2;
        o[2 * k + 1] = (t + c[k + 2] + 2 - 512) >> 2;
    }
}

// h2v2 triangular on 16-bit lane pairs (two samples per 32-bit operation; no
// lane carries out: 3 * 1020 + 1020 + 2056 < 2^16).  The 6 samples c[-1..4]
// of a row around four chroma centres are the bytes l.3, m.0-3, r.0 of three
// words; lanes4 forms the pairs (c0,c2), (c1,c3), (c-1,c1), (c2,c4).
__device__ __forceinline__ void lanes4(uint32_t l, uint32_t m, uint32_t r, uint32_t &e, uint32_t &o, uint32_t &lp,
                                       uint32_t &rp)
{
    e = __byte_perm(m, 0u, 0x4240);
    o = __byte_perm(m, 0u, 0x4341);
    lp = __byte_perm(o, l, 0x1017);
    rp = __byte_perm(e, r, 0x1412);
}

// The 8 outputs (minus 128) of one output row from the near row's pairs
// (ne, no, nl, nr) and the far row's words: S = 3 near + far per lane, then
// out[2k] = (3 S_k + S_{k-1} + 8) >> 4 and out[2k+1] = (3 S_k + S_{k+1} + 7) >> 4
// with 2048 more in each sum, so that the low byte of each lane's result is
// the sample XOR 0x80 (read back as a signed byte: the sample minus 128).
__device__ __forceinline__ void tri_h2v2_pairs(uint32_t ne, uint32_t no, uint32_t nl, uint32_t nr, uint32_t fl,
                                               uint32_t fm, uint32_t fr, int out[8])
{
    uint32_t fe, fo, flp, frp;
    lanes4(fl, fm, fr, fe, fo, flp, frp);
    const uint32_t se = ne * 3u + fe, so = no * 3u + fo, sl = nl * 3u + flp, sr = nr * 3u + frp;
    const uint32_t te = se * 3u, to = so * 3u;
    const uint32_t p04 = (te + sl + 0x08080808u) >> 4;   // outputs 0, 4
    const uint32_t p26 = (to + se + 0x08080808u) >> 4;   // 2, 6
    const uint32_t p15 = (te + so + 0x08070807u) >> 4;   // 1, 5
    const uint32_t p37 = (to + sr + 0x08070807u) >> 4;   // 3, 7
    out[0] = sbyte_of(p04, 0); out[4] = sbyte_of(p04, 2);
    out[2] = sbyte_of(p26, 0); out[6] = sbyte_of(p26, 2);
    out[1] = sbyte_of(p15, 0); out[5] = sbyte_of(p15, 2);
    out[3] = sbyte_of(p37, 0); out[7] = sbyte_of(p37, 2);
}

}  // namespace jdec
