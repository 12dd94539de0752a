// rklt_tc.cuh -- 32 x 32 and 16 x 16 blocks on the tensor cores (warp-level fp16
// mma.sync with fp32 accumulation): N = 32 with retained supports inside i + j < 16
// (r <= 136), N = 16 inside i + j < 8 (r <= 36).  Included by rklt_fused_impl.cuh
// after the tile constants; used by fused_kernel<32, TC_V> and fused_kernel<16, TC_V>.
// The N = 32 chain is described first; the N = 16 form follows at tc16_setup.
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
constexpr int TC_DMAX = 16;                // N = 32: handles diagonal bounds D <= 16
constexpr int TC_DMAX16 = 8;               // N = 16: handles D <= 8
constexpr int TC_HALF = (TW / 2) * TH;     // bytes of one 128-byte-wide half tile
constexpr int TC_ZS = 148;                 // per-warp coefficient staging stride (floats)

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
    asm(
        "mma.sync.aligned.m16n8k16.row.col.f32.f16.f16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%10,%11,%12,%13};"
        : "=f"(d[0]), "=f"(d[1]), "=f"(d[2]), "=f"(d[3])
        : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1), "f"(c[0]), "f"(c[1]), "f"(c[2]), "f"(c[3]));
}

// d += a * b, m16n8k8.
__device__ __forceinline__ void mma8(float (&d)[4], uint32_t a0, uint32_t a1, uint32_t b0) {
    asm(
        "mma.sync.aligned.m16n8k8.row.col.f32.f16.f16.f32 {%0,%1,%2,%3}, {%4,%5}, {%6}, {%0,%1,%2,%3};"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a0), "r"(a1), "r"(b0));
}

// 8 x 8 transpose of 16-bit elements across the warp.
__device__ __forceinline__ uint32_t movm_t(uint32_t x) {
    uint32_t y;
    asm("movmatrix.sync.aligned.m8n8.trans.b16 %0, %1;" : "=r"(y) : "r"(x));
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

// Shared-memory accesses through 32-bit shared-window addresses.
__device__ __forceinline__ uint32_t lds32(uint32_t a) {
    uint32_t v;
    asm volatile("ld.shared.u32 %0, [%1];" : "=r"(v) : "r"(a));
    return v;
}
__device__ __forceinline__ void sts32(uint32_t a, uint32_t v) {
    asm volatile("st.shared.u32 [%0], %1;" ::"r"(a), "r"(v));
}
template <int OFF>
__device__ __forceinline__ uint32_t lds32o(uint32_t a) {
    uint32_t v;
    asm volatile("ld.shared.u32 %0, [%1+%2];" : "=r"(v) : "r"(a), "n"(OFF));
    return v;
}
template <int OFF>
__device__ __forceinline__ void sts32o(uint32_t a, uint32_t v) {
    asm volatile("st.shared.u32 [%0+%1], %2;" ::"r"(a), "n"(OFF), "r"(v));
}
__device__ __forceinline__ uint4 lds128(uint32_t a) {
    uint4 v;
    asm volatile("ld.shared.v4.u32 {%0,%1,%2,%3}, [%4];" : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w) : "r"(a));
    return v;
}
__device__ __forceinline__ void sts_f32(uint32_t a, float v) {
    asm volatile("st.shared.f32 [%0], %1;" ::"r"(a), "f"(v));
}

// Per-lane constants kept in registers: F1's accumulator start and the lane's
// shared-memory offsets inside a tile.
struct TcLane {
    float init1[2];      // F1 accumulator start for rows j = 2g, 2g + 1: -1024 sum_x T[j][x]
    // byte offsets in the tile of the lane's words for the warp's block column:
    // [class][word]; class 0 = row g (row 8 + g is +1024), class 1 = row 31 - g
    // (row 23 - g is -1024); word 0 = x 4t..4t+3, 1 = x 16+4t.., 2 = x 28-4t..31-4t
    uint32_t off[2][3];
};

// The other per-lane constants live in a shared-memory table of TC_TAB x 32 uint4,
// entry [k][lane] (16-byte loads by consecutive lanes hit distinct banks).  Operands
// that an MMA takes as a register pair are stored as such (a k16 B operand whose two
// halves are equal appears twice), so they load straight into place:
//   k = 0, 1  I1 B of y' n-tile k: hi, hi (even i), hi, hi (odd i) of 2^6 T^{-1}[y'][i]
//   k = 2, 3  I2 B of x' n-tile k - 2: the same for T^{-1}[x'][j]
//   k = 4, 5  staging byte offsets of accumulator elements q = 4 (k - 4) .. + 3: 4 x the
//             zig-zag position when retained, else 4 x the spare slot TC_ZS - 1
//   k = 6, 7  2^12 s_i s_j of those elements
//   k = 8, 9  1.0 when retained, else 0.0
//   k = 10, 11  F1 A fragments of k-step k - 10: T[j][x], rows j = 2g (even), 2g + 1 (odd)
//   k = 12    F2 B: 2^-12 T[i][y] (y < 16) for i = 2g (even n-tile), then i = 2g + 1
//   k = 13, 14  lo digits: I1 n-tile k - 13 (even i, odd i), then I2 n-tile k - 13
//   k = 15, 16  (quantised calls) 2^12 w_ij of those elements, w = fl32(s_i s_j / Q_ij)
//   k = 17, 18  (quantised calls) 2^-12 fl32(Q_ij / (s_i s_j))
constexpr int TC_TAB = 19;
constexpr int TC_TAB_BYTES = 19 * 32 * 16;   // the larger of the two tables

__device__ __forceinline__ float tc_T(const PlanK<32> &P, int i, int x) {
    return x < 16 ? P.T[i][x] : ((i & 1) ? -P.T[i][31 - x] : P.T[i][31 - x]);
}

// Builds the lane's registers and (when `write_tab`) its column of the table.
// Element q = 4 * nt + e of a lane's F2 accumulator holds C[i][j] with
// j = 2g + (e >> 1) and i = 4t + 2 (e & 1) + nt.  bx is the warp's block column.
__device__ inline void tc_setup(const PlanK<32> &P, TcLane &c, uint4 *tab, bool write_tab, int lane, int r,
                                int bx, bool quant) {
    const int g = lane >> 2, t = lane & 3;
    const int j0 = 2 * g, j1 = 2 * g + 1;
    float s0 = 0.0f, s1 = 0.0f;
    for (int x = 0; x < 32; x++) {
        s0 += tc_T(P, j0, x);
        s1 += tc_T(P, j1, x);
    }
    c.init1[0] = -1024.0f * s0;
    c.init1[1] = -1024.0f * s1;
    const float q12 = 1.0f / 4096.0f, s6 = 64.0f;
    const int cb = (bx & 3) * 2;
#pragma unroll
    for (int cls = 0; cls < 2; cls++) {
        const int y = cls ? 31 - g : g, sw = y & 7;
        const uint32_t rb = uint32_t((bx >> 2) * TC_HALF + y * 128);
        c.off[cls][0] = rb + uint32_t(((cb ^ sw) << 4) + 4 * t);
        c.off[cls][1] = rb + uint32_t((((cb + 1) ^ sw) << 4) + 4 * t);
        c.off[cls][2] = rb + uint32_t((((cb + 1) ^ sw) << 4) + 12 - 4 * t);
    }
    if (!write_tab) return;
#pragma unroll
    for (int ks = 0; ks < 2; ks++) {
        const int x0 = 16 * ks + 4 * t;
        tab[(10 + ks) * 32 + lane] = make_uint4(pack_h2(tc_T(P, j0, x0), tc_T(P, j0, x0 + 1)),
                                                pack_h2(tc_T(P, j1, x0), tc_T(P, j1, x0 + 1)),
                                                pack_h2(tc_T(P, j0, x0 + 2), tc_T(P, j0, x0 + 3)),
                                                pack_h2(tc_T(P, j1, x0 + 2), tc_T(P, j1, x0 + 3)));
    }
    tab[12 * 32 + lane] = make_uint4(pack_h2(q12 * P.T[j0][2 * t], q12 * P.T[j0][2 * t + 1]),
                                     pack_h2(q12 * P.T[j0][2 * t + 8], q12 * P.T[j0][2 * t + 9]),
                                     pack_h2(q12 * P.T[j1][2 * t], q12 * P.T[j1][2 * t + 1]),
                                     pack_h2(q12 * P.T[j1][2 * t + 8], q12 * P.T[j1][2 * t + 9]));
#pragma unroll
    for (int nt = 0; nt < 2; nt++) {
        const int yp = 8 * nt + g;                              // I1 n-tile column y'
        const int xp = 4 * (g >> 1) + 2 * nt + (g & 1);         // I2 n-tile column x'
        uint32_t h3e, l3e, h3o, l3o, h4e, l4e, h4o, l4o;
        split_pair(s6 * P.Ti[yp][4 * t], s6 * P.Ti[yp][4 * t + 2], h3e, l3e);
        split_pair(s6 * P.Ti[yp][4 * t + 1], s6 * P.Ti[yp][4 * t + 3], h3o, l3o);
        split_pair(s6 * P.Ti[xp][4 * t], s6 * P.Ti[xp][4 * t + 2], h4e, l4e);
        split_pair(s6 * P.Ti[xp][4 * t + 1], s6 * P.Ti[xp][4 * t + 3], h4o, l4o);
        tab[nt * 32 + lane] = make_uint4(h3e, h3e, h3o, h3o);
        tab[(2 + nt) * 32 + lane] = make_uint4(h4e, h4e, h4o, h4o);
        tab[(13 + nt) * 32 + lane] = make_uint4(l3e, l3o, l4e, l4o);
    }
    uint32_t zp[8], bs[8], kp[8], qw[8], qt[8];
#pragma unroll
    for (int q = 0; q < 8; q++) {
        const int nt = q >> 2, e = q & 3;
        const int j = 2 * g + (e >> 1), i = 4 * t + 2 * (e & 1) + nt;
        const int z = zz_index(32, i, j);
        zp[q] = uint32_t(4 * (z < r ? z : TC_ZS - 1));
        bs[q] = __float_as_uint(4096.0f * P.sij[i][j]);
        kp[q] = __float_as_uint(z < r ? 1.0f : 0.0f);
        qw[q] = __float_as_uint(4096.0f * P.qw[i][j]);
        qt[q] = __float_as_uint(P.qt[i][j] * (1.0f / 4096.0f));
    }
#pragma unroll
    for (int h = 0; h < 2; h++) {
        tab[(4 + h) * 32 + lane] = make_uint4(zp[4 * h], zp[4 * h + 1], zp[4 * h + 2], zp[4 * h + 3]);
        tab[(6 + h) * 32 + lane] = make_uint4(bs[4 * h], bs[4 * h + 1], bs[4 * h + 2], bs[4 * h + 3]);
        tab[(8 + h) * 32 + lane] = make_uint4(kp[4 * h], kp[4 * h + 1], kp[4 * h + 2], kp[4 * h + 3]);
        if (quant) {
            tab[(15 + h) * 32 + lane] = make_uint4(qw[4 * h], qw[4 * h + 1], qw[4 * h + 2], qw[4 * h + 3]);
            tab[(17 + h) * 32 + lane] = make_uint4(qt[4 * h], qt[4 * h + 1], qt[4 * h + 2], qt[4 * h + 3]);
        }
    }
}

// The quantiser's integer decision on an F2 accumulator element d = C 2^-12 with
// the table value w12 = 2^12 w: fl32(d w12) = fl32(C w) exactly (scaling by powers of
// two), then floor(fl32(q + 1/2)) -- the binary32 decision of the register path.
__device__ __forceinline__ float tc_quant_code(float d, uint32_t w12) {
    return floorf(__fadd_rn(__fmul_rn(d, __uint_as_float(w12)), 0.5f));
}

// One 32 x 32 block by one warp: `blk` is the shared-window address of the tile
// plus 4096 * (block row); tabl is the table address plus 16 * lane; zs the warp's
// staging buffer (shared-window address).  Returns the lane's share of the block's
// SSE; writes the 8-bit reconstruction in place when `recon`, and the r normalised
// coefficients to zg (if not null).
template <bool FAST, bool Q = false>
__device__ __forceinline__ float tc_block32(const TcLane &c, uint32_t tabl, uint32_t blk, int lane, int r,
                                            float *zg, uint32_t zs, bool recon_, bool vec4_) {
    // FAST: coefficients (16-byte aligned, r % 4 == 0) and reconstruction both wanted
    const bool recon = FAST || recon_, vec4 = FAST || vec4_;
    // the lane's rows: q = 0: g, 1: 8 + g, 2: 31 - g, 3: 23 - g
    // rows q = 0, 1 are [off[0][.]] and [off[0][.] + 1024], rows 2, 3 [off[1][.]] and
    // [off[1][.] - 1024]
    const auto ld_word = [&](int q, int word) -> uint32_t {
        const uint32_t a = blk + c.off[q >> 1][word];
        return q == 0 ? lds32o<0>(a) : q == 1 ? lds32o<1024>(a) : q == 2 ? lds32o<0>(a) : lds32o<-1024>(a);
    };
    const auto st_word = [&](int q, int word, uint32_t v) {
        const uint32_t a = blk + c.off[q >> 1][word];
        if (q == 0) sts32o<0>(a, v);
        else if (q == 1) sts32o<1024>(a, v);
        else if (q == 2) sts32o<0>(a, v);
        else sts32o<-1024>(a, v);
    };

    // ---- F1: Z^T = T A^T (16 frequencies j x 32 rows y), pixels biased by 1024
    float d1[4][4];
    {
        const uint4 a0 = lds128(tabl + 10 * 512), a1 = lds128(tabl + 11 * 512);
        const float ci[4] = {c.init1[0], c.init1[0], c.init1[1], c.init1[1]};
#pragma unroll
        for (int nt = 0; nt < 4; nt++) {
            const uint32_t w0 = ld_word(nt, 0), w1 = ld_word(nt, 1);
            mma16(d1[nt], ci, a0.x, a0.y, a0.z, a0.w, bytes_to_biased_h2(w0, 0, 1), bytes_to_biased_h2(w0, 2, 3));
            mma16(d1[nt], d1[nt], a1.x, a1.y, a1.z, a1.w, bytes_to_biased_h2(w1, 0, 1),
                  bytes_to_biased_h2(w1, 2, 3));
        }
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
    {
        const uint4 b2 = lds128(tabl + 12 * 512);
        mma16(d2[0], z4, sh[0][0], sh[0][1], sh[1][0], sh[1][1], b2.x, b2.y);
        mma16(d2[0], d2[0], sl[0][0], sl[0][1], sl[1][0], sl[1][1], b2.x, b2.y);
        mma16(d2[1], z4, dh[0][0], dh[0][1], dh[1][0], dh[1][1], b2.z, b2.w);
        mma16(d2[1], d2[1], dl[0][0], dl[0][1], dl[1][0], dl[1][1], b2.z, b2.w);
    }
    // ---- M: coefficients staged in zig-zag order (dropped ones land in the spare
    //      slot), zonal mask, C' as binary16 digits
    uint32_t ch[2][2], cl[2][2];
#pragma unroll
    for (int nt = 0; nt < 2; nt++) {
        if constexpr (Q) {
            // quantised: Bbar (int32) where the coefficients go; C' = Bbar Qtilde 2^-12
            const uint4 qw = lds128(tabl + (15 + nt) * 512), qt = lds128(tabl + (17 + nt) * 512);
            const float b0 = tc_quant_code(d2[nt][0], qw.x), b1 = tc_quant_code(d2[nt][1], qw.y);
            const float b2 = tc_quant_code(d2[nt][2], qw.z), b3 = tc_quant_code(d2[nt][3], qw.w);
            if (FAST || zg) {
                const uint4 zp = lds128(tabl + (4 + nt) * 512);
                sts_f32(zs + zp.x, __int_as_float(int(b0)));
                sts_f32(zs + zp.y, __int_as_float(int(b1)));
                sts_f32(zs + zp.z, __int_as_float(int(b2)));
                sts_f32(zs + zp.w, __int_as_float(int(b3)));
            }
            d2[nt][0] = __fmul_rn(b0, __uint_as_float(qt.x));
            d2[nt][1] = __fmul_rn(b1, __uint_as_float(qt.y));
            d2[nt][2] = __fmul_rn(b2, __uint_as_float(qt.z));
            d2[nt][3] = __fmul_rn(b3, __uint_as_float(qt.w));
        } else if (FAST || zg) {
            const uint4 zp = lds128(tabl + (4 + nt) * 512), bs = lds128(tabl + (6 + nt) * 512);
            sts_f32(zs + zp.x, __uint_as_float(bs.x) * d2[nt][0]);
            sts_f32(zs + zp.y, __uint_as_float(bs.y) * d2[nt][1]);
            sts_f32(zs + zp.z, __uint_as_float(bs.z) * d2[nt][2]);
            sts_f32(zs + zp.w, __uint_as_float(bs.w) * d2[nt][3]);
        }
        const uint4 kp = lds128(tabl + (8 + nt) * 512);
        const float2 v0 = __fmul2_rn(make_float2(d2[nt][0], d2[nt][1]),
                                     make_float2(__uint_as_float(kp.x), __uint_as_float(kp.y)));
        const float2 v1 = __fmul2_rn(make_float2(d2[nt][2], d2[nt][3]),
                                     make_float2(__uint_as_float(kp.z), __uint_as_float(kp.w)));
        split_pair(v0.x, v0.y, ch[nt][0], cl[nt][0]);
        split_pair(v1.x, v1.y, ch[nt][1], cl[nt][1]);
    }
    // ---- I1: E (even i) and O (odd i) for y' < 16; Y^T * 2^-6 = E + O (y'), E - O (31 - y')
    uint32_t yh[4][2], yl[4][2];  // [group][row half]: groups y' = 0..7, 8..15, 31..24, 23..16
#pragma unroll
    for (int nt = 0; nt < 2; nt++) {
        const uint4 b3 = lds128(tabl + nt * 512), lo = lds128(tabl + (13 + nt) * 512);
        float E[4], O[4];
        mma16(E, z4, ch[0][0], ch[0][1], cl[0][0], cl[0][1], b3.x, b3.y);
        mma8(E, ch[0][0], ch[0][1], lo.x);
        mma16(O, z4, ch[1][0], ch[1][1], cl[1][0], cl[1][1], b3.z, b3.w);
        mma8(O, ch[1][0], ch[1][1], lo.y);
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
    // the even sums start at 1024 + 1/2: E + O and E - O are A' + 1024 + 1/2, whose
    // binary16 truncation is the rounded byte biased by 1024 (bytes4_biased), and whose
    // difference from the biased pixel 1024 + a is the error less 1/2
    const float k10245[4] = {1024.5f, 1024.5f, 1024.5f, 1024.5f};
    const float2 half2f = make_float2(0.5f, 0.5f);
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
            const uint4 b4 = lds128(tabl + (2 + nt) * 512);
            const uint32_t l4e = lds32(tabl + (13 + nt) * 512 + 8), l4o = lds32(tabl + (13 + nt) * 512 + 12);
            mma16(E2[nt], k10245, ah0, ah1, al0, al1, b4.x, b4.y);
            mma8(E2[nt], ah0, ah1, l4e);
            mma16(O2[nt], z4, oh0, oh1, ol0, ol1, b4.z, b4.w);
            mma8(O2[nt], oh0, oh1, l4o);
        }
#pragma unroll
        for (int h = 0; h < 2; h++) {
            const int q = 2 * mt + h;
            const float2 e0 = make_float2(E2[0][2 * h], E2[0][2 * h + 1]);
            const float2 o0 = make_float2(O2[0][2 * h], O2[0][2 * h + 1]);
            const float2 e1 = make_float2(E2[1][2 * h], E2[1][2 * h + 1]);
            const float2 o1 = make_float2(O2[1][2 * h], O2[1][2 * h + 1]);
            const float2 ta = __fadd2_rn(e0, o0), tb = __fadd2_rn(e1, o1);              // x' = 4t + {0,1}, {2,3}
            const float2 ba = __ffma2_rn(o0, neg1, e0), bb = __ffma2_rn(o1, neg1, e1);  // bytes {3,2}, {1,0}
            const uint32_t wt = ld_word(q, 0), wb = ld_word(q, 2);
            const __half2 p01 = as_h2(bytes_to_biased_h2(wt, 0, 1));   // 1024 + pixel
            const __half2 p23 = as_h2(bytes_to_biased_h2(wt, 2, 3));
            const __half2 q01 = as_h2(bytes_to_biased_h2(wb, 0, 1));
            const __half2 q23 = as_h2(bytes_to_biased_h2(wb, 2, 3));
            const float2 et0 = __fadd2_rn(make_float2(sub_h_f(__low2half(p01), ta.x), sub_h_f(__high2half(p01), ta.y)), half2f);
            const float2 et1 = __fadd2_rn(make_float2(sub_h_f(__low2half(p23), tb.x), sub_h_f(__high2half(p23), tb.y)), half2f);
            const float2 eb0 = __fadd2_rn(make_float2(sub_h_f(__low2half(q01), bb.y), sub_h_f(__high2half(q01), bb.x)), half2f);
            const float2 eb1 = __fadd2_rn(make_float2(sub_h_f(__low2half(q23), ba.y), sub_h_f(__high2half(q23), ba.x)), half2f);
            sse2 = __ffma2_rn(et0, et0, sse2);
            sse2 = __ffma2_rn(et1, et1, sse2);
            sse2 = __ffma2_rn(eb0, eb0, sse2);
            sse2 = __ffma2_rn(eb1, eb1, sse2);
            if (recon) {
                st_word(q, 0, bytes4_biased(ta.x, ta.y, tb.x, tb.y));
                st_word(q, 2, bytes4_biased(bb.y, bb.x, ba.y, ba.x));
            }
        }
    }
    // ---- coefficients of the block, contiguous in the output
    if (FAST || zg) {
        __syncwarp();
        if (FAST) {  // r <= 136 (D <= 16): at most two float4 per lane
            if (4 * lane < r) *reinterpret_cast<uint4 *>(zg + 4 * lane) = lds128(zs + 16 * lane);
            if (4 * lane + 128 < r) *reinterpret_cast<uint4 *>(zg + 4 * lane + 128) = lds128(zs + 16 * lane + 512);
        } else if (vec4) {
            for (int k = 4 * lane; k < r; k += 128) {
                const uint4 v = lds128(zs + 4 * k);
                *reinterpret_cast<uint4 *>(zg + k) = v;
            }
        } else {
            for (int k = lane; k < r; k += 32) zg[k] = __uint_as_float(lds32(zs + 4 * k));
        }
        __syncwarp();
    }
    return sse2.x + sse2.y;
}

// The 16 blocks of one tile: warp w takes block columns w and w + 4 of both block
// rows.  Column w + 4 lies in the second 128-byte half of the tile at the same
// swizzle phase, so its addresses are column w's plus TC_HALF.
template <bool FAST, bool Q = false>
__device__ __forceinline__ float tile_tc(const TcLane &c, uint32_t tabl, const FusedGeom &g, uint8_t *tile,
                                         const TileCoord &tc, int ct, uint32_t zs) {
    const int w = ct >> 5, lane = ct & 31;
    const int bw = g.W / 32;
    const int rows_in = min(TH / 32, (g.H - tc.ty * TH) / 32);
    const int nb_in = min(TW / 32, bw - tc.tx * (TW / 32));
    float sse = 0.0f;
    float *zt = (FAST || g.zcoef) ? g.zcoef + (int64_t(tc.img) * g.blocks_per_img + int64_t(tc.ty * (TH / 32)) * bw +
                                               tc.tx * (TW / 32) + w) * g.r
                                  : nullptr;
#pragma unroll 1
    for (int cg = 0; cg < 2; cg++) {
        if (w + 4 * cg >= nb_in) break;
        for (int by = 0; by < rows_in; by++) {
            float *zg = zt ? zt + (int64_t(by) * bw + 4 * cg) * g.r : nullptr;
            sse += tc_block32<FAST, Q>(c, tabl, smem_u32(tile) + by * 32 * 128 + cg * TC_HALF, lane, g.r, zg, zs,
                                       g.recon != nullptr, g.coef_vec4 != 0);
        }
    }
    return sse;
}

// ---------------------------------------------------------------------------
// N = 16: one warp takes a 32 x 32 region of four blocks (vb, hb) (block row, block
// column) and runs the same chain with the block index folded into the MMA shapes:
//   F1  rows (hb, j), j < 8; k-step hb' = x block; the A operand is block diagonal
//       (T[j][x] where hb = hb', else 0), so each row sums its own block's columns
//   F2  per class (even i from S = Z[y] + Z[15-y], odd i from Z[y] - Z[15-y]) and per
//       k-step vb: K = (digit, y < 8), columns (vb', i) with B zero unless vb' = vb
//   I1  K = D2 columns (vb, i) of one class with [hi | lo] digits, columns (vb3, y'),
//       y' < 8, B zero unless vb = vb3; E (even i) + O (odd i) and E - O give rows
//       y' and 15 - y' of block row vb3
//   I2  per block column hb: the transposed 8 x 8 digit blocks (rows y, columns j)
//       times 2^6 T^{-1}[x][j] for all 16 x, 4 adjacent x per lane
// Row order of the lane: q = 0: y = g, 1: 16 + g, 2: 15 - g, 3: 31 - g (region rows).
//
// Table entries [k][lane] (uint4), register pairs and quads stored in place:
//   k = 0, 1  F1 A quads of k-step 0 and 1: (P01, 0, P23, 0), (0, P01, 0, P23) with
//             P01 = (T[g][4t], T[g][4t+1]), P23 = (T[g][4t+2], T[g][4t+3])
//   k = 2, 3  F2 B pairs of class k - 2 for k-step vb = 0, then 1: 2^-12 (T[i][2t],
//             T[i][2t+1]), i = 2 (g & 3) + class, nonzero only on lanes with g >> 2 = vb
//   k = 4, 5  I1 B (hi, hi) for column block vb3 = 0, then 1; class k - 4
//   k = 6     I1 lo digits: class 0 vb3 0, 1, class 1 vb3 0, 1
//   k = 7     I2 B: (hi, hi) of 2^6 T^{-1}[x][2t, 2t+1] for n-tile 0, then n-tile 1
//   k = 8     I2 lo digits for n-tile 0, 1
//   k = 9, 10   staging byte offsets 4 ((2 vb + hb) r + z) of accumulator elements q = 4 class + e
//   k = 11, 12  2^12 s_i s_j;  k = 13, 14  1.0 when retained, else 0.0
//   k = 15, 16 and 17, 18  (quantised calls) as for N = 32
constexpr int TC16_TAB = 19;
// ---------------------------------------------------------------------------
__device__ __forceinline__ float tc16_T(const PlanK<16> &P, int i, int x) {
    return x < 8 ? P.T[i][x] : ((i & 1) ? -P.T[i][15 - x] : P.T[i][15 - x]);
}
__device__ __forceinline__ float tc16_Ti(const PlanK<16> &P, int l, int j) {  // T^{-1}[l][j], any l
    return l < 8 ? P.Ti[l][j] : ((j & 1) ? -P.Ti[15 - l][j] : P.Ti[15 - l][j]);
}

__device__ inline void tc16_setup(const PlanK<16> &P, TcLane &c, uint4 *tab, bool write_tab, int lane, int r,
                                  int bx, bool quant) {
    const int g = lane >> 2, t = lane & 3;
    float s0 = 0.0f;
    for (int x = 0; x < 16; x++) s0 += tc16_T(P, g, x);
    c.init1[0] = c.init1[1] = -1024.0f * s0;
    const int cb = (bx & 3) * 2;
#pragma unroll
    for (int cls = 0; cls < 2; cls++) {
        const int y = cls ? 15 - g : g, sw = y & 7;
        const uint32_t rb = uint32_t((bx >> 2) * TC_HALF + y * 128);
        c.off[cls][0] = rb + uint32_t(((cb ^ sw) << 4) + 4 * t);
        c.off[cls][1] = rb + uint32_t((((cb + 1) ^ sw) << 4) + 4 * t);
        c.off[cls][2] = 0;
    }
    if (!write_tab) return;
    const float q12 = 1.0f / 4096.0f, s6 = 64.0f;
    const int i0 = 2 * (g & 3), i1 = 2 * (g & 3) + 1;
    const uint32_t p01 = pack_h2(tc16_T(P, g, 4 * t), tc16_T(P, g, 4 * t + 1));
    const uint32_t p23 = pack_h2(tc16_T(P, g, 4 * t + 2), tc16_T(P, g, 4 * t + 3));
    tab[0 * 32 + lane] = make_uint4(p01, 0u, p23, 0u);
    tab[1 * 32 + lane] = make_uint4(0u, p01, 0u, p23);
    {
        const uint32_t b0 = pack_h2(q12 * P.T[i0][2 * t], q12 * P.T[i0][2 * t + 1]);
        const uint32_t b1 = pack_h2(q12 * P.T[i1][2 * t], q12 * P.T[i1][2 * t + 1]);
        const bool v0 = (g >> 2) == 0;
        tab[2 * 32 + lane] = make_uint4(v0 ? b0 : 0u, v0 ? b0 : 0u, v0 ? 0u : b0, v0 ? 0u : b0);
        tab[3 * 32 + lane] = make_uint4(v0 ? b1 : 0u, v0 ? b1 : 0u, v0 ? 0u : b1, v0 ? 0u : b1);
    }
    uint32_t l1[4];
#pragma unroll
    for (int cls = 0; cls < 2; cls++) {
        // K index k = 2t, 2t+1 <-> D2 column (vb = t >> 1, i = 4 (t & 1) + {0, 2} + cls)
        const int ia = 4 * (t & 1) + cls, ib = ia + 2;
        uint32_t h, l;
        split_pair(s6 * P.Ti[g][ia], s6 * P.Ti[g][ib], h, l);
        const bool v0 = (t >> 1) == 0;
        const uint32_t h0 = v0 ? h : 0u, h1 = v0 ? 0u : h;
        tab[(4 + cls) * 32 + lane] = make_uint4(h0, h0, h1, h1);
        l1[2 * cls] = v0 ? l : 0u;
        l1[2 * cls + 1] = v0 ? 0u : l;
    }
    tab[6 * 32 + lane] = make_uint4(l1[0], l1[1], l1[2], l1[3]);
    {
        uint32_t ha, la, hb2, lb;
        const int xa = 4 * (g >> 1) + (g & 1), xb = xa + 2;  // n-tile 0 and 1 columns x
        split_pair(s6 * tc16_Ti(P, xa, 2 * t), s6 * tc16_Ti(P, xa, 2 * t + 1), ha, la);
        split_pair(s6 * tc16_Ti(P, xb, 2 * t), s6 * tc16_Ti(P, xb, 2 * t + 1), hb2, lb);
        tab[7 * 32 + lane] = make_uint4(ha, ha, hb2, hb2);
        tab[8 * 32 + lane] = make_uint4(la, lb, 0u, 0u);
    }
    uint32_t zp[8], bs[8], kp[8], qw[8], qt[8];
#pragma unroll
    for (int q = 0; q < 8; q++) {
        const int cls = q >> 2, e = q & 3;
        const int vb = t >> 1, hb = e >> 1;
        const int i = 2 * ((2 * t + (e & 1)) & 3) + cls, j = g;
        const int z = zz_index(16, i, j);
        zp[q] = uint32_t(4 * (z < r ? (2 * vb + hb) * r + z : TC_ZS - 1));
        bs[q] = __float_as_uint(4096.0f * P.sij[i][j]);
        kp[q] = __float_as_uint(z < r ? 1.0f : 0.0f);
        qw[q] = __float_as_uint(4096.0f * P.qw[i][j]);
        qt[q] = __float_as_uint(P.qt[i][j] * (1.0f / 4096.0f));
    }
#pragma unroll
    for (int h = 0; h < 2; h++) {
        tab[(9 + h) * 32 + lane] = make_uint4(zp[4 * h], zp[4 * h + 1], zp[4 * h + 2], zp[4 * h + 3]);
        tab[(11 + h) * 32 + lane] = make_uint4(bs[4 * h], bs[4 * h + 1], bs[4 * h + 2], bs[4 * h + 3]);
        tab[(13 + h) * 32 + lane] = make_uint4(kp[4 * h], kp[4 * h + 1], kp[4 * h + 2], kp[4 * h + 3]);
        if (quant) {
            tab[(15 + h) * 32 + lane] = make_uint4(qw[4 * h], qw[4 * h + 1], qw[4 * h + 2], qw[4 * h + 3]);
            tab[(17 + h) * 32 + lane] = make_uint4(qt[4 * h], qt[4 * h + 1], qt[4 * h + 2], qt[4 * h + 3]);
        }
    }
}

// One 32 x 32 region (four 16 x 16 blocks) by one warp.  `in` has bit 2 vb + hb set
// for the blocks inside the image (all four in the interior); only those add to the
// SSE.  The staging buffer receives each block's r coefficients at (2 vb + hb) r.
template <bool ALL_IN, bool FAST, bool Q = false>
__device__ __forceinline__ float tc16_region(const TcLane &c, uint32_t tabl, uint32_t blk, int lane, uint32_t zs,
                                             bool coef_, bool recon_, int in) {
    const bool coef = FAST || coef_, recon = FAST || recon_;
    const int t = lane & 3;
    // word w (x block) of row q: q = 0 [off[0][w]], 1 [+2048], 2 [off[1][w]], 3 [+2048]
    const auto ld_word = [&](int q, int w) -> uint32_t {
        const uint32_t a = blk + c.off[q >> 1 ? 1 : 0][w];
        return (q & 1) ? lds32o<2048>(a) : lds32o<0>(a);
    };
    const auto st_word = [&](int q, int w, uint32_t v) {
        const uint32_t a = blk + c.off[q >> 1 ? 1 : 0][w];
        if (q & 1) sts32o<2048>(a, v);
        else sts32o<0>(a, v);
    };
    // ---- F1 (n-tiles 0..3 = rows y = g, 15 - g, 16 + g, 31 - g = lane rows q 0, 2, 1, 3)
    float d1[4][4];
    {
        const uint4 f0 = lds128(tabl), f1 = lds128(tabl + 512);
        const float ci[4] = {c.init1[0], c.init1[0], c.init1[0], c.init1[0]};
#pragma unroll
        for (int nt = 0; nt < 4; nt++) {
            const int q = (nt == 0) ? 0 : (nt == 1) ? 2 : (nt == 2) ? 1 : 3;
            const uint32_t w0 = ld_word(q, 0), w1 = ld_word(q, 1);
            mma16(d1[nt], ci, f0.x, f0.y, f0.z, f0.w, bytes_to_biased_h2(w0, 0, 1), bytes_to_biased_h2(w0, 2, 3));
            mma16(d1[nt], d1[nt], f1.x, f1.y, f1.z, f1.w, bytes_to_biased_h2(w1, 0, 1),
                  bytes_to_biased_h2(w1, 2, 3));
        }
    }
    // ---- y-parity per block row vb: S = Z[y'] + Z[15-y'], Dd = Z[y'] - Z[15-y'], digits
    const float2 neg1 = make_float2(-1.0f, -1.0f);
    uint32_t sh[2][2], sl[2][2], dh[2][2], dl[2][2];  // [vb][row half = hb]
#pragma unroll
    for (int vb = 0; vb < 2; vb++) {
#pragma unroll
        for (int p = 0; p < 2; p++) {
            const float2 u = make_float2(d1[2 * vb][2 * p], d1[2 * vb][2 * p + 1]);
            const float2 v = make_float2(d1[2 * vb + 1][2 * p], d1[2 * vb + 1][2 * p + 1]);
            const float2 s = __fadd2_rn(u, v), d = __ffma2_rn(v, neg1, u);
            split_pair(s.x, s.y, sh[vb][p], sl[vb][p]);
            split_pair(d.x, d.y, dh[vb][p], dl[vb][p]);
        }
    }
    // ---- F2: class 0 (even i) from S, class 1 (odd i) from Dd; k-step vb
    const float z4[4] = {0.0f, 0.0f, 0.0f, 0.0f};
    float d2[2][4];
    {
        const uint4 be = lds128(tabl + 2 * 512), bo = lds128(tabl + 3 * 512);
        mma16(d2[0], z4, sh[0][0], sh[0][1], sl[0][0], sl[0][1], be.x, be.y);
        mma16(d2[0], d2[0], sh[1][0], sh[1][1], sl[1][0], sl[1][1], be.z, be.w);
        mma16(d2[1], z4, dh[0][0], dh[0][1], dl[0][0], dl[0][1], bo.x, bo.y);
        mma16(d2[1], d2[1], dh[1][0], dh[1][1], dl[1][0], dl[1][1], bo.z, bo.w);
    }
    // ---- M: staged coefficients, zonal mask, C' digits
    uint32_t ch[2][2], cl[2][2];
#pragma unroll
    for (int cls = 0; cls < 2; cls++) {
        if constexpr (Q) {
            const uint4 qw = lds128(tabl + (15 + cls) * 512), qt = lds128(tabl + (17 + cls) * 512);
            const float b0 = tc_quant_code(d2[cls][0], qw.x), b1 = tc_quant_code(d2[cls][1], qw.y);
            const float b2 = tc_quant_code(d2[cls][2], qw.z), b3 = tc_quant_code(d2[cls][3], qw.w);
            if (coef) {
                const uint4 zp = lds128(tabl + (9 + cls) * 512);
                sts_f32(zs + zp.x, __int_as_float(int(b0)));
                sts_f32(zs + zp.y, __int_as_float(int(b1)));
                sts_f32(zs + zp.z, __int_as_float(int(b2)));
                sts_f32(zs + zp.w, __int_as_float(int(b3)));
            }
            d2[cls][0] = __fmul_rn(b0, __uint_as_float(qt.x));
            d2[cls][1] = __fmul_rn(b1, __uint_as_float(qt.y));
            d2[cls][2] = __fmul_rn(b2, __uint_as_float(qt.z));
            d2[cls][3] = __fmul_rn(b3, __uint_as_float(qt.w));
        } else if (coef) {
            const uint4 zp = lds128(tabl + (9 + cls) * 512), bs = lds128(tabl + (11 + cls) * 512);
            sts_f32(zs + zp.x, __uint_as_float(bs.x) * d2[cls][0]);
            sts_f32(zs + zp.y, __uint_as_float(bs.y) * d2[cls][1]);
            sts_f32(zs + zp.z, __uint_as_float(bs.z) * d2[cls][2]);
            sts_f32(zs + zp.w, __uint_as_float(bs.w) * d2[cls][3]);
        }
        const uint4 kp = lds128(tabl + (13 + cls) * 512);
        const float2 v0 = __fmul2_rn(make_float2(d2[cls][0], d2[cls][1]),
                                     make_float2(__uint_as_float(kp.x), __uint_as_float(kp.y)));
        const float2 v1 = __fmul2_rn(make_float2(d2[cls][2], d2[cls][3]),
                                     make_float2(__uint_as_float(kp.z), __uint_as_float(kp.w)));
        split_pair(v0.x, v0.y, ch[cls][0], cl[cls][0]);
        split_pair(v1.x, v1.y, ch[cls][1], cl[cls][1]);
    }
    // ---- I1: n-tile vb3; top (y' < 8) = E + O, bottom (15 - y') = E - O
    uint32_t yh[4][2], yl[4][2];  // groups q: 0 = vb0 top, 1 = vb1 top, 2 = vb0 bottom, 3 = vb1 bottom
    {
        const uint4 be = lds128(tabl + 4 * 512), bo = lds128(tabl + 5 * 512), bl = lds128(tabl + 6 * 512);
#pragma unroll
        for (int vb3 = 0; vb3 < 2; vb3++) {
            const uint32_t eh0 = vb3 ? be.z : be.x, eh1 = vb3 ? be.w : be.y;
            const uint32_t oh0 = vb3 ? bo.z : bo.x, oh1 = vb3 ? bo.w : bo.y;
            const uint32_t el = vb3 ? bl.y : bl.x, ol = vb3 ? bl.w : bl.z;
            float E[4], O[4];
            mma16(E, z4, ch[0][0], ch[0][1], cl[0][0], cl[0][1], eh0, eh1);
            mma8(E, ch[0][0], ch[0][1], el);
            mma16(O, z4, ch[1][0], ch[1][1], cl[1][0], cl[1][1], oh0, oh1);
            mma8(O, ch[1][0], ch[1][1], ol);
#pragma unroll
            for (int p = 0; p < 2; p++) {
                const float2 e2 = make_float2(E[2 * p], E[2 * p + 1]), o2 = make_float2(O[2 * p], O[2 * p + 1]);
                const float2 top = __fadd2_rn(e2, o2), bot = __ffma2_rn(o2, neg1, e2);
                split_pair(top.x, top.y, yh[vb3][p], yl[vb3][p]);
                split_pair(bot.x, bot.y, yh[2 + vb3][p], yl[2 + vb3][p]);
            }
        }
    }
    // ---- I2 per (m-tile, block column hb), then error and 8-bit output.  m-tile mt has
    //      rows g (group 2 mt) and g + 8 (group 2 mt + 1): y = g, 16 + g (mt 0) and
    //      15 - g, 31 - g (mt 1); lane word x = 16 hb + 4t .. 4t + 3
    const uint4 b4 = lds128(tabl + 7 * 512), b4l = lds128(tabl + 8 * 512);
    // accumulators start at 1024 + 1/2 (see tc_block32)
    const float k10245[4] = {1024.5f, 1024.5f, 1024.5f, 1024.5f};
    const float2 half2f = make_float2(0.5f, 0.5f);
    float2 sse2 = make_float2(0.0f, 0.0f);
#pragma unroll
    for (int mt = 0; mt < 2; mt++) {
#pragma unroll
        for (int hb = 0; hb < 2; hb++) {
            const uint32_t ah0 = movm_t(yh[2 * mt][hb]), ah1 = movm_t(yh[2 * mt + 1][hb]);
            const uint32_t al0 = movm_t(yl[2 * mt][hb]), al1 = movm_t(yl[2 * mt + 1][hb]);
            float R[2][4];
            mma16(R[0], k10245, ah0, ah1, al0, al1, b4.x, b4.y);
            mma8(R[0], ah0, ah1, b4l.x);
            mma16(R[1], k10245, ah0, ah1, al0, al1, b4.z, b4.w);
            mma8(R[1], ah0, ah1, b4l.y);
#pragma unroll
            for (int h = 0; h < 2; h++) {
                const int q = 2 * mt + h;            // group; region row y as listed above
                const int vb = (q == 1 || q == 3) ? 1 : 0;
                const float2 va = make_float2(R[0][2 * h], R[0][2 * h + 1]);   // x = 4t, 4t + 1
                const float2 vc = make_float2(R[1][2 * h], R[1][2 * h + 1]);   // x = 4t + 2, 4t + 3
                const int lq = (q == 0) ? 0 : (q == 1) ? 1 : (q == 2) ? 2 : 3;
                // lane rows: ld_word's q follows y = g, 16 + g, 15 - g, 31 - g
                const uint32_t wt = ld_word(lq, hb);
                const __half2 p01 = as_h2(bytes_to_biased_h2(wt, 0, 1));   // 1024 + pixel
                const __half2 p23 = as_h2(bytes_to_biased_h2(wt, 2, 3));
                float2 e0 = __fadd2_rn(make_float2(sub_h_f(__low2half(p01), va.x), sub_h_f(__high2half(p01), va.y)), half2f);
                float2 e1 = __fadd2_rn(make_float2(sub_h_f(__low2half(p23), vc.x), sub_h_f(__high2half(p23), vc.y)), half2f);
                if (!ALL_IN && !((in >> (2 * vb + hb)) & 1)) e0 = e1 = make_float2(0.0f, 0.0f);
                sse2 = __ffma2_rn(e0, e0, sse2);
                sse2 = __ffma2_rn(e1, e1, sse2);
                if (recon) st_word(lq, hb, bytes4_biased(va.x, va.y, vc.x, vc.y));
            }
        }
    }
    (void)t;
    return sse2.x + sse2.y;
}

// The 16 regions of one tile (N = 16): warp w takes region columns w and w + 4 (the
// latter TC_HALF further in the swizzled tile) of both region rows.
template <bool FAST, bool Q = false>
__device__ __forceinline__ float tile_tc16(const TcLane &c, uint32_t tabl, const FusedGeom &g, uint8_t *tile,
                                           const TileCoord &tc, int ct, uint32_t zs) {
    const int lane = ct & 31;
    const int bw = g.W / 16;
    const int rows_in = min(TH / 16, (g.H - tc.ty * TH) / 16);   // block rows of the tile inside
    const int nb_in = min(TW / 16, bw - tc.tx * (TW / 16));       // block columns inside
    const int r = g.r;
    float sse = 0.0f;
    const bool coef = FAST || g.zcoef != nullptr;
#pragma unroll 1
    for (int cg = 0; cg < 2; cg++) {
    const int w = (ct >> 5) + 4 * cg;
    const uint32_t t32 = smem_u32(tile) + cg * TC_HALF;
    if (2 * w >= nb_in) break;
    const bool cols2 = 2 * w + 1 < nb_in;   // both block columns of the warp inside
    for (int ry = 0; ry < 2; ry++) {
        if (2 * ry >= rows_in) break;
        const bool rows2 = 2 * ry + 1 < rows_in;
        const int in = (rows2 && cols2) ? 15 : (1 | (cols2 ? 2 : 0) | (rows2 ? 4 | (cols2 ? 8 : 0) : 0));
        const uint32_t blk = t32 + ry * 32 * 128;
        if (in == 15) sse += tc16_region<true, FAST, Q>(c, tabl, blk, lane, zs, coef, g.recon != nullptr, in);
        else sse += tc16_region<false, FAST, Q>(c, tabl, blk, lane, zs, coef, g.recon != nullptr, in);
        if (coef) {
            // coefficients of the region's first block
            float *zrow0 = g.zcoef + (int64_t(tc.img) * g.blocks_per_img + int64_t(tc.ty * (TH / 16) + 2 * ry) * bw +
                                      tc.tx * (TW / 16) + 2 * w) * r;
            __syncwarp();
#pragma unroll
            for (int vb = 0; vb < 2; vb++) {
                if (!((in >> (2 * vb)) & 1)) continue;
                const int n = ((in >> (2 * vb + 1)) & 1) ? 2 * r : r;   // floats of this block row
                float *dst = zrow0 + (vb ? int64_t(bw) * r : int64_t(0));
                const uint32_t src = zs + 4 * (2 * vb * r);
                if (FAST) {  // n <= 72 (D <= 8): one float4 per lane at most
                    if (4 * lane < n) *reinterpret_cast<uint4 *>(dst + 4 * lane) = lds128(src + 16 * lane);
                } else if (g.coef_vec4) {
                    for (int k = 4 * lane; k < n; k += 128) *reinterpret_cast<uint4 *>(dst + k) = lds128(src + 4 * k);
                } else {
                    for (int k = lane; k < n; k += 32) dst[k] = __uint_as_float(lds32(src + 4 * k));
                }
            }
            __syncwarp();
        }
    }
    }
    return sse;
}

}  // namespace rklt
