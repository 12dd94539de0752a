// rklt_tc.cuh -- 32 x 32 blocks on the tensor cores (warp-level fp16 mma.sync with
// fp32 accumulation) for retained supports inside i + j < 16 (r <= 136).  Included by
// rklt_fused_impl.cuh after the tile constants; used by fused_kernel<32, TC_V>.
//
// One warp transforms one block.  Lane l has g = l / 4 and t = l % 4, the MMA
// fragment coordinates.  The chain of contractions (Sec. 4.1: C = T A T^T, zonal
// mask, A' = T^{-1} C' T^{-T}) is laid out so that each MMA's accumulator is the next
// MMA's A operand wherever the contraction runs over the accumulator's columns:
//
//   F1  Z^T[j][y]  = sum_x T[j][x] A[y][x]        A operand T (rows j < 16), B = pixels
//   F2  C^T[j][i]  = sum_y Z^T[j][y] T[i][y]      y-parity: even i from Z[y] + Z[31-y],
//                                                 odd i from Z[y] - Z[31-y] (y < 16)
//   M   zonal mask, normalised coefficients s_i s_j C[i][j] staged in zig-zag order
//   I1  Y^T[j][y'] = sum_i C'^T[j][i] T^{-1}[y'][i]   i-parity: E (even i), O (odd i),
//                                                 Y[y'] = E + O, Y[31-y'] = E - O
//   --  Y^T -> Y by 8x8 register transposes (movmatrix)
//   I2  A'[y'][x'] = sum_j Y[y'][j] T^{-1}[x'][j]     j-parity as in I1, x' < 16 mirrored
//   E   error, SSE, 8-bit output clip(floor(A' + 1/2), 0, 255) in place
//
// Only frequencies below 16 are formed: every retained (i, j) has i + j < 16.  The
// row parity T[i][31-x] = (-1)^i T[i][x] and T^{-1}[31-l][j] = (-1)^j T^{-1}[l][j]
// halves F2, I1 and I2.
//
// Exactness of the forward part: pixels (biased by 1024 in F1, the bias removed by
// the accumulator start value), T in {0, +1, -1}, and every partial sum of F1 are
// integers below 2^16; F2 takes S = Z[y] +- Z[31-y] (|S| <= 16320) as two binary16
// digits hi + lo that sum to S exactly, and T scaled by 2^-12, so every partial sum of
// F2 is a multiple of 2^-12 below 2^6: C is exact.  The inverse takes C' (exact, in two
// digits) and 2^6 T^{-1} (two digits) with three products hi*hi + lo*hi + hi*lo, then
// Y (scaled by 2^-6) in two digits: about 22 significant bits per operand, inside
// the FP32 reconstruction bound.
#pragma once

namespace rklt {

constexpr int TC_V = 4;                    // kernel variant number of this path
constexpr int TC_DMAX = 16;                // handles diagonal bounds D <= 16
constexpr int TC_HALF = (TW / 2) * TH;     // bytes of one 128-byte-wide half tile
constexpr int TC_ZS = 140;                 // per-warp coefficient staging stride (floats)

// Byte offset of pixel (y, x) of a 64 x 256 tile held as two 64 x 128 halves, each
// in the 128-byte swizzled layout of a TMA copy: the 16-byte chunk index of row y is
// XORed with y mod 8, so eight rows read at the same column hit eight different
// bank groups.
__host__ __device__ constexpr int swz_off(int y, int x) {
    return (x >> 7) * TC_HALF + y * 128 + ((((x & 127) >> 4) ^ (y & 7)) << 4) + (x & 15);
}

// d = a * b + c, m16n8k16, fp16 operands, fp32 accumulation.
__device__ __forceinline__ void mma16(float (&d)[4], const float (&c)[4], uint32_t a0, uint32_t a1, uint32_t a2,
                                      uint32_t a3, uint32_t b0, uint32_t b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.f16.f16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%10,%11,%12,%13};"
        : "=f"(d[0]), "=f"(d[1]), "=f"(d[2]), "=f"(d[3])
        : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1), "f"(c[0]), "f"(c[1]), "f"(c[2]), "f"(c[3]));
}

// d += a * b, m16n8k8.
__device__ __forceinline__ void mma8(float (&d)[4], uint32_t a0, uint32_t a1, uint32_t b0) {
    asm volatile(
        "mma.sync.aligned.m16n8k8.row.col.f32.f16.f16.f32 {%0,%1,%2,%3}, {%4,%5}, {%6}, {%0,%1,%2,%3};"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a0), "r"(a1), "r"(b0));
}

// 8 x 8 transpose of 16-bit elements across the warp.
__device__ __forceinline__ uint32_t movm_t(uint32_t x) {
    uint32_t y;
    asm volatile("movmatrix.sync.aligned.m8n8.trans.b16 %0, %1;" : "=r"(y) : "r"(x));
    return y;
}

__device__ __forceinline__ uint32_t pack_h2(float lo, float hi) { return as_u32(__floats2half2_rn(lo, hi)); }

// v - h with a single rounding (mixed-precision FMA h * (-1) + v).
__device__ __forceinline__ float sub_f_h(float v, __half h) {
    float d;
    asm("fma.rn.f32.f16 %0, %1, %2, %3;" : "=f"(d) : "h"(__half_as_ushort(h)), "h"(uint16_t(0xBC00u)), "f"(v));
    return d;
}

// (v0, v1) = hi + lo with hi = binary16(v), lo = binary16(v - hi).
__device__ __forceinline__ void split_pair(float v0, float v1, uint32_t &hi, uint32_t &lo) {
    const __half2 h = __floats2half2_rn(v0, v1);
    hi = as_u32(h);
    lo = as_u32(__floats2half2_rn(sub_f_h(v0, __low2half(h)), sub_f_h(v1, __high2half(h))));
}

// Per-lane constant operands of the forward passes, kept in registers.
struct TcLane {
    uint32_t a1[2][4];   // F1 A fragments per k-step: T[j][x], rows j = 2g (even), 2g + 1 (odd)
    float init1[2];      // F1 accumulator start for those rows: -1024 sum_x T[j][x]
    uint32_t b2[2][2];   // F2 B per n-tile (even i, odd i): 2^-12 T[i][y], y < 16
};

// The other per-lane constants live in a shared-memory table of 8 x 32 uint4,
// entry [k][lane] (16-byte loads by consecutive lanes hit distinct banks):
//   k = 0, 1  I1 B of y' n-tile k: hi, lo of 2^6 T^{-1}[y'][i] (even i), then (odd i)
//   k = 2, 3  I2 B of x' n-tile k - 2: the same for T^{-1}[x'][j]
//   k = 4, 5  zig-zag positions of accumulator elements q = 4 (k - 4) .. + 3, -1 if dropped
//   k = 6, 7  2^12 s_i s_j of those elements
constexpr int TC_TAB_BYTES = 8 * 32 * 16;

__device__ __forceinline__ float tc_T(const PlanK<32> &P, int i, int x) {
    return x < 16 ? P.T[i][x] : ((i & 1) ? -P.T[i][31 - x] : P.T[i][31 - x]);
}

// Builds the lane's registers and (when `write_tab`) its column of the table.
// Element q = 4 * nt + e of a lane's F2 accumulator holds C[i][j] with
// j = 2g + (e >> 1) and i = 4t + 2 (e & 1) + nt.
__device__ inline void tc_setup(const PlanK<32> &P, TcLane &c, uint4 *tab, bool write_tab, int lane, int r) {
    const int g = lane >> 2, t = lane & 3;
    const int j0 = 2 * g, j1 = 2 * g + 1;
#pragma unroll
    for (int ks = 0; ks < 2; ks++) {
        const int x0 = 16 * ks + 4 * t;
        c.a1[ks][0] = pack_h2(tc_T(P, j0, x0), tc_T(P, j0, x0 + 1));
        c.a1[ks][1] = pack_h2(tc_T(P, j1, x0), tc_T(P, j1, x0 + 1));
        c.a1[ks][2] = pack_h2(tc_T(P, j0, x0 + 2), tc_T(P, j0, x0 + 3));
        c.a1[ks][3] = pack_h2(tc_T(P, j1, x0 + 2), tc_T(P, j1, x0 + 3));
    }
    float s0 = 0.0f, s1 = 0.0f;
    for (int x = 0; x < 32; x++) {
        s0 += tc_T(P, j0, x);
        s1 += tc_T(P, j1, x);
    }
    c.init1[0] = -1024.0f * s0;
    c.init1[1] = -1024.0f * s1;
    const float q12 = 1.0f / 4096.0f, s6 = 64.0f;
#pragma unroll
    for (int nt = 0; nt < 2; nt++) {
        const int i = 2 * g + nt;
        c.b2[nt][0] = pack_h2(q12 * P.T[i][2 * t], q12 * P.T[i][2 * t + 1]);
        c.b2[nt][1] = pack_h2(q12 * P.T[i][2 * t + 8], q12 * P.T[i][2 * t + 9]);
    }
    if (!write_tab) return;
#pragma unroll
    for (int nt = 0; nt < 2; nt++) {
        const int yp = 8 * nt + g;                              // I1 n-tile column y'
        const int xp = 4 * (g >> 1) + 2 * nt + (g & 1);         // I2 n-tile column x'
        uint4 v3, v4;
        split_pair(s6 * P.Ti[yp][4 * t], s6 * P.Ti[yp][4 * t + 2], v3.x, v3.y);
        split_pair(s6 * P.Ti[yp][4 * t + 1], s6 * P.Ti[yp][4 * t + 3], v3.z, v3.w);
        split_pair(s6 * P.Ti[xp][4 * t], s6 * P.Ti[xp][4 * t + 2], v4.x, v4.y);
        split_pair(s6 * P.Ti[xp][4 * t + 1], s6 * P.Ti[xp][4 * t + 3], v4.z, v4.w);
        tab[nt * 32 + lane] = v3;
        tab[(2 + nt) * 32 + lane] = v4;
    }
    int zp[8];
    float bs[8];
#pragma unroll
    for (int q = 0; q < 8; q++) {
        const int nt = q >> 2, e = q & 3;
        const int j = 2 * g + (e >> 1), i = 4 * t + 2 * (e & 1) + nt;
        const int z = zz_index(32, i, j);
        zp[q] = z < r ? z : -1;
        bs[q] = 4096.0f * P.sij[i][j];
    }
    tab[4 * 32 + lane] = make_uint4(zp[0], zp[1], zp[2], zp[3]);
    tab[5 * 32 + lane] = make_uint4(zp[4], zp[5], zp[6], zp[7]);
    tab[6 * 32 + lane] = make_uint4(__float_as_uint(bs[0]), __float_as_uint(bs[1]), __float_as_uint(bs[2]),
                                    __float_as_uint(bs[3]));
    tab[7 * 32 + lane] = make_uint4(__float_as_uint(bs[4]), __float_as_uint(bs[5]), __float_as_uint(bs[6]),
                                    __float_as_uint(bs[7]));
}

// One 32 x 32 block (block row `by`, block column `bx` of the tile) by one warp.
// Returns the lane's share of the block's SSE; writes the 8-bit reconstruction in
// place when `recon`, and the r normalised coefficients to zg (if not null) through
// the warp's staging buffer zs.
__device__ __forceinline__ float tc_block32(const TcLane &c, const uint4 *tab, uint8_t *tile, int by, int bx,
                                            int lane, int r, float *zg, float *zs, bool recon, bool vec4) {
    const int g = lane >> 2, t = lane & 3;
    uint8_t *base = tile + (bx >> 2) * TC_HALF + by * 32 * 128;
    const int cb = (bx & 3) * 2;  // first 16-byte chunk of the block in its half-tile row
    // The lane's rows: F1 n-tile q and output row q are y = g, 8 + g, 31 - g, 23 - g
    // (y mod 8 = g, g, 7 - g, 7 - g).
    const auto row_ptr = [&](int q, int chunk, int byte) -> uint8_t * {
        const int y = (q == 0) ? g : (q == 1) ? 8 + g : (q == 2) ? 31 - g : 23 - g;
        const int s = q < 2 ? g : 7 - g;
        return base + y * 128 + (((cb + chunk) ^ s) << 4) + byte;
    };

    // ---- F1: Z^T = T A^T (16 frequencies j x 32 rows y), pixels biased by 1024
    float d1[4][4];
#pragma unroll
    for (int nt = 0; nt < 4; nt++) {
        const float ci[4] = {c.init1[0], c.init1[0], c.init1[1], c.init1[1]};
        const uint32_t w0 = *reinterpret_cast<const uint32_t *>(row_ptr(nt, 0, 4 * t));
        const uint32_t w1 = *reinterpret_cast<const uint32_t *>(row_ptr(nt, 1, 4 * t));
        mma16(d1[nt], ci, c.a1[0][0], c.a1[0][1], c.a1[0][2], c.a1[0][3], bytes_to_biased_h2(w0, 0, 1),
              bytes_to_biased_h2(w0, 2, 3));
        mma16(d1[nt], d1[nt], c.a1[1][0], c.a1[1][1], c.a1[1][2], c.a1[1][3], bytes_to_biased_h2(w1, 0, 1),
              bytes_to_biased_h2(w1, 2, 3));
    }
    // ---- y-parity: S = Z[y] + Z[31-y], Dd = Z[y] - Z[31-y] (y < 16), as binary16 digits
    const float2 neg1 = make_float2(-1.0f, -1.0f);
    uint32_t sh[2][2], sl[2][2], dh[2][2], dl[2][2];
#pragma unroll
    for (int nt = 0; nt < 2; nt++) {
#pragma unroll
        for (int p = 0; p < 2; p++) {
            const float2 u = make_float2(d1[nt][2 * p], d1[nt][2 * p + 1]);
            const float2 v = make_float2(d1[nt + 2][2 * p], d1[nt + 2][2 * p + 1]);
            const float2 s = __fadd2_rn(u, v), d = __ffma2_rn(v, neg1, u);
            split_pair(s.x, s.y, sh[nt][p], sl[nt][p]);
            split_pair(d.x, d.y, dh[nt][p], dl[nt][p]);
        }
    }
    // ---- F2: C^T * 2^-12 (rows j, columns i: n-tile 0 even i, n-tile 1 odd i)
    const float z4[4] = {0.0f, 0.0f, 0.0f, 0.0f};
    float d2[2][4];
    mma16(d2[0], z4, sh[0][0], sh[0][1], sh[1][0], sh[1][1], c.b2[0][0], c.b2[0][1]);
    mma16(d2[0], d2[0], sl[0][0], sl[0][1], sl[1][0], sl[1][1], c.b2[0][0], c.b2[0][1]);
    mma16(d2[1], z4, dh[0][0], dh[0][1], dh[1][0], dh[1][1], c.b2[1][0], c.b2[1][1]);
    mma16(d2[1], d2[1], dl[0][0], dl[0][1], dl[1][0], dl[1][1], c.b2[1][0], c.b2[1][1]);
    // ---- M: coefficients (staged in zig-zag order), zonal mask, C' as binary16 digits
    uint32_t ch[2][2], cl[2][2];
    {
        const uint4 zp0 = tab[4 * 32 + lane], zp1 = tab[5 * 32 + lane];
        const int zp[8] = {int(zp0.x), int(zp0.y), int(zp0.z), int(zp0.w),
                           int(zp1.x), int(zp1.y), int(zp1.z), int(zp1.w)};
        if (zg) {
            const uint4 b0 = tab[6 * 32 + lane], b1 = tab[7 * 32 + lane];
            const float bs[8] = {__uint_as_float(b0.x), __uint_as_float(b0.y), __uint_as_float(b0.z),
                                 __uint_as_float(b0.w), __uint_as_float(b1.x), __uint_as_float(b1.y),
                                 __uint_as_float(b1.z), __uint_as_float(b1.w)};
#pragma unroll
            for (int q = 0; q < 8; q++)
                if (zp[q] >= 0) zs[zp[q]] = bs[q] * d2[q >> 2][q & 3];
        }
#pragma unroll
        for (int nt = 0; nt < 2; nt++) {
#pragma unroll
            for (int p = 0; p < 2; p++) {
                const float v0 = zp[4 * nt + 2 * p] >= 0 ? d2[nt][2 * p] : 0.0f;
                const float v1 = zp[4 * nt + 2 * p + 1] >= 0 ? d2[nt][2 * p + 1] : 0.0f;
                split_pair(v0, v1, ch[nt][p], cl[nt][p]);
            }
        }
    }
    // ---- I1: E (even i) and O (odd i) for y' < 16; Y^T * 2^-6 = E + O (y'), E - O (31 - y')
    uint32_t yh[4][2], yl[4][2];  // [group][row half]: groups y' = 0..7, 8..15, 31..24, 23..16
#pragma unroll
    for (int nt = 0; nt < 2; nt++) {
        const uint4 b3 = tab[nt * 32 + lane];
        float E[4], O[4];
        mma16(E, z4, ch[0][0], ch[0][1], cl[0][0], cl[0][1], b3.x, b3.x);
        mma8(E, ch[0][0], ch[0][1], b3.y);
        mma16(O, z4, ch[1][0], ch[1][1], cl[1][0], cl[1][1], b3.z, b3.z);
        mma8(O, ch[1][0], ch[1][1], b3.w);
#pragma unroll
        for (int p = 0; p < 2; p++) {
            const float2 e2 = make_float2(E[2 * p], E[2 * p + 1]), o2 = make_float2(O[2 * p], O[2 * p + 1]);
            const float2 top = __fadd2_rn(e2, o2), bot = __ffma2_rn(o2, neg1, e2);
            split_pair(top.x, top.y, yh[nt][p], yl[nt][p]);
            split_pair(bot.x, bot.y, yh[2 + nt][p], yl[2 + nt][p]);
        }
    }
    // ---- per m-tile: transpose to Y (rows y', columns j), I2 for x' < 16 (E' + O') and
    //      31 - x' (E' - O'), then error and 8-bit output for the m-tile's two rows.
    //      Row q of the lane: m-tile q >> 1, accumulator row half q & 1; top word
    //      x' = 4t .. 4t+3, bottom word x' = 28-4t .. 31-4t.
    const __half2 k10235 = __float2half2_rn(1023.5f);
    const float half4[4] = {0.5f, 0.5f, 0.5f, 0.5f};
    float2 sse2 = make_float2(0.0f, 0.0f);
#pragma unroll
    for (int mt = 0; mt < 2; mt++) {
        const uint32_t ah0 = movm_t(yh[2 * mt][0]), ah1 = movm_t(yh[2 * mt + 1][0]);
        const uint32_t al0 = movm_t(yl[2 * mt][0]), al1 = movm_t(yl[2 * mt + 1][0]);
        const uint32_t oh0 = movm_t(yh[2 * mt][1]), oh1 = movm_t(yh[2 * mt + 1][1]);
        const uint32_t ol0 = movm_t(yl[2 * mt][1]), ol1 = movm_t(yl[2 * mt + 1][1]);
        float E2[2][4], O2[2][4];  // [n-tile][4]
#pragma unroll
        for (int nt = 0; nt < 2; nt++) {
            const uint4 b4 = tab[(2 + nt) * 32 + lane];
            mma16(E2[nt], half4, ah0, ah1, al0, al1, b4.x, b4.x);
            mma8(E2[nt], ah0, ah1, b4.y);
            mma16(O2[nt], z4, oh0, oh1, ol0, ol1, b4.z, b4.z);
            mma8(O2[nt], oh0, oh1, b4.w);
        }
#pragma unroll
        for (int h = 0; h < 2; h++) {
            const int q = 2 * mt + h;
            uint32_t *pt = reinterpret_cast<uint32_t *>(row_ptr(q, 0, 4 * t));
            uint32_t *pb = reinterpret_cast<uint32_t *>(row_ptr(q, 1, 12 - 4 * t));
            const float2 e0 = make_float2(E2[0][2 * h], E2[0][2 * h + 1]);
            const float2 o0 = make_float2(O2[0][2 * h], O2[0][2 * h + 1]);
            const float2 e1 = make_float2(E2[1][2 * h], E2[1][2 * h + 1]);
            const float2 o1 = make_float2(O2[1][2 * h], O2[1][2 * h + 1]);
            const float2 ta = __fadd2_rn(e0, o0), tb = __fadd2_rn(e1, o1);              // x' = 4t + {0,1}, {2,3}
            const float2 ba = __ffma2_rn(o0, neg1, e0), bb = __ffma2_rn(o1, neg1, e1);  // bytes {3,2}, {1,0}
            const uint32_t wt = *pt, wb = *pb;
            const __half2 p01 = __hsub2(as_h2(bytes_to_biased_h2(wt, 0, 1)), k10235);   // pixel + 1/2
            const __half2 p23 = __hsub2(as_h2(bytes_to_biased_h2(wt, 2, 3)), k10235);
            const __half2 q01 = __hsub2(as_h2(bytes_to_biased_h2(wb, 0, 1)), k10235);
            const __half2 q23 = __hsub2(as_h2(bytes_to_biased_h2(wb, 2, 3)), k10235);
            const float2 et0 = make_float2(sub_h_f(__low2half(p01), ta.x), sub_h_f(__high2half(p01), ta.y));
            const float2 et1 = make_float2(sub_h_f(__low2half(p23), tb.x), sub_h_f(__high2half(p23), tb.y));
            const float2 eb0 = make_float2(sub_h_f(__low2half(q01), bb.y), sub_h_f(__high2half(q01), bb.x));
            const float2 eb1 = make_float2(sub_h_f(__low2half(q23), ba.y), sub_h_f(__high2half(q23), ba.x));
            sse2 = __ffma2_rn(et0, et0, sse2);
            sse2 = __ffma2_rn(et1, et1, sse2);
            sse2 = __ffma2_rn(eb0, eb0, sse2);
            sse2 = __ffma2_rn(eb1, eb1, sse2);
            if (recon) {
                *pt = floor_sat_u8(ta.x) | (floor_sat_u8(ta.y) << 8) | (floor_sat_u8(tb.x) << 16) |
                      (floor_sat_u8(tb.y) << 24);
                *pb = floor_sat_u8(bb.y) | (floor_sat_u8(bb.x) << 8) | (floor_sat_u8(ba.y) << 16) |
                      (floor_sat_u8(ba.x) << 24);
            }
        }
    }
    // ---- coefficients of the block, contiguous in the output
    if (zg) {
        __syncwarp();
        if (vec4) {
            for (int k = 4 * lane; k < r; k += 128)
                *reinterpret_cast<float4 *>(zg + k) = *reinterpret_cast<const float4 *>(zs + k);
        } else {
            for (int k = lane; k < r; k += 32) zg[k] = zs[k];
        }
        __syncwarp();
    }
    return sse2.x + sse2.y;
}

// All blocks of one tile: warp w takes block column w of both block rows.
__device__ __forceinline__ float tile_tc(const TcLane &c, const uint4 *tab, const FusedGeom &g, uint8_t *tile,
                                         int64_t tile_id, int ct, float *Zs) {
    const TileCoord tc = tile_coord(g, tile_id);
    const int w = ct >> 5, lane = ct & 31;
    const int bw = g.W / 32;
    const int rows_in = min(TH / 32, (g.H - tc.ty * TH) / 32);
    const int nb_in = min(TW / 32, bw - tc.tx * (TW / 32));
    float sse = 0.0f;
    if (w < nb_in) {
        for (int by = 0; by < rows_in; by++) {
            float *zg = g.zcoef ? g.zcoef + (int64_t(tc.img) * g.blocks_per_img +
                                             int64_t(tc.ty * (TH / 32) + by) * bw + tc.tx * (TW / 32) + w) *
                                                g.r
                                : nullptr;
            sse += tc_block32(c, tab, tile, by, w, lane, g.r, zg, Zs + w * TC_ZS, g.recon != nullptr,
                              g.coef_vec4 != 0);
        }
    }
    return sse;
}

}  // namespace rklt
