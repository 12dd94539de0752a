// rklt_fused_impl.cuh -- the fused single-pass rounded-KLT kernel (included once
// per block size by rklt_fused_n{4,8,16,32}.cu so that the sizes compile in parallel).
//
// One pass per N x N block (Sec. 4.1 of arXiv 2111.14239 and its Appendix):
//   C  = T A T^T                exact: integers < 2^24 summed in FP32 registers
//   B  = (s s^T) o C            normalised coefficients, zig-zag order, first r kept
//   A' = T^{-1} (M o C) T^{-T}  inverse; equals That^{-1} B' That^{-T} (S cancels)
//   SSE += sum (A - A')^2       FP32 per thread, fixed-order tree per tile, FP64 per image
// with T = round(alpha K) (Sec. 2.3) in {0, +1, -1}.  Each 1-D transform uses the
// row parity of the Markov-1 KLT, T[i][N-1-j] = (-1)^i T[i][j]: a first butterfly
// stage forms sums s_j and differences d_j of mirrored samples, then even rows
// combine the sums and odd rows the differences (half the products of a dense
// product; the entries of T enter as constant-bank operands of FFMA).  Only the
// coefficients on the retained zig-zag support (anti-diagonals i + j < D) are
// formed, and only their inverse contributions are summed.
//
// Data movement: the image is cut into 64-row x 256-byte tiles.  When pointers
// and pitches are 16-byte aligned a producer warp streams tiles into a 3- to 6-stage
// shared-memory ring with 3-D TMA bulk tensor copies (mbarrier completion), the
// eight consumer warps transform them in place, and the producer writes the
// rounded 8-bit reconstruction back with TMA bulk tensor stores.  Otherwise the
// consumers copy each tile in and out with plain vector loads.  Both modes run the
// same per-block code in the same order, so their results are identical.
//
// JPEG-like quantisation (N = 4, 8; Appendix): the same kernels with the
// retained C quantised in place, Bbar = floor(fl32(C w) + 1/2) with
// w = fl32(s_i s_j / Q_ij), written as int32 where the coefficients go, and the
// inverse run on the dequantised Bbar o Qtilde (Qtilde = Q / (s s^T)).
//
// Work split inside a tile:
//   register path  (N = 4, and N = 8 with D <= 5): one thread owns a whole block;
//   tensor-core path (N = 32 with D <= 16, rklt_tc.cuh): one warp owns a block and
//     runs every contraction as fp16 mma.sync; tiles then arrive as two 128-byte
//     swizzled halves;
//   cooperative path (N = 16, N = 32 with D > 16, N = 8 with D > 5, and exact-KLT /
//     DCT plans): threads own columns for the column passes and (block, row) pairs
//     for the row passes, exchanging through a padded shared-memory buffer (all
//     block-rows of a tile at once for N >= 8; block-row by block-row for N = 4).
#pragma once

#include <cudaTypedefs.h>

#include <algorithm>
#include <mutex>

#include "rklt_device.cuh"
#include "rklt_internal.h"

namespace rklt {

constexpr int TW = 256;          // tile width in bytes (pixels)
constexpr int TH = 64;           // tile height in rows
constexpr int TILE_BYTES = TW * TH;
constexpr int STAGES = 8;        // deepest TMA ring (barrier and reduction slots)
constexpr int NCONS = 256;       // consumer threads (8 warps) of the FMA variants; one producer warp follows
constexpr int NCONS_TC = 128;    // consumer threads (4 warps) of the tensor-core variant: three CTAs of
                                 // 4 + 1 warps per SM leave each thread up to 128 registers
constexpr int NCONS_MAX = 256;
constexpr int LDY = TW + 1;      // padded row stride of the cooperative exchange buffer (floats)
static_assert(TW == kTileW && TH == kTileH, "tile geometry is declared in rklt_internal.h");
constexpr int REG_DMAX8 = 5;     // N = 8: two-CTA register path up to this diagonal bound
constexpr int REG8_FULL = 5;     // variant number of the N = 8 register path for any D (one CTA per SM)
constexpr int REG_REAL = 6;      // variant number of the register path for real (exact KLT / DCT) plans
constexpr uint64_t DRAIN_NS = 2000000000ull;  // limit on waits for copies already in flight
constexpr int QV = 8;            // added to a variant number: quantised coefficients
__host__ __device__ constexpr int vbase(int V) { return V & 7; }

// The quantiser's integer decision for one retained C (binary32, no contraction).
template <int N>
__device__ __forceinline__ float quant_code(const PlanK<N> &P, int i, int j, float c) {
    return floorf(__fadd_rn(__fmul_rn(c, P.qw[i][j]), 0.5f));
}

// ---------------------------------------------------------------------------
// Register path: one N x N block per thread.  D is a compile-time constant.
//
// The column pass runs as byte dot products (dp4a) on the transposed block: T's
// rows as packed signed bytes against four pixels of one column, exact in int32.
// The row pass, the inverse and the error run in FP32; the error takes each pixel
// straight from its exact binary16 form with a mixed-precision subtraction.
// ---------------------------------------------------------------------------
// Loads the N x N block at src (row stride ld bytes) as N/4 words per row.
template <int N>
__device__ __forceinline__ void load_block_words(const uint8_t *src, int64_t ld, uint32_t (&w)[N][N / 4]) {
#pragma unroll
    for (int k = 0; k < N; k++) {
        if constexpr (N == 8) {
            const uint2 v = *reinterpret_cast<const uint2 *>(src + k * ld);
            w[k][0] = v.x;
            w[k][1] = v.y;
        } else {
            w[k][0] = *reinterpret_cast<const uint32_t *>(src + k * ld);
        }
    }
}

// The whole per-block computation on a block held in registers (w); the 8-bit
// reconstruction is written to dst (row stride ldd bytes) when recon is set.
// FAST: coefficients and reconstruction both wanted (the branches resolved).
// REAL: a real (exact KLT / DCT) matrix: the column pass in FP32 instead of exact
// binary16 sums of {0, +1, -1} entries.
// (Rounded plans with T T^T diagonal run the register path of rklt_reg.cuh, which
// takes the error from Parseval's identity; this one serves the others.)
template <int N, int D, bool Q = false, bool FAST = false, bool REAL = false>
__device__ __forceinline__ float block_core(const PlanK<N> &P, const uint32_t (&w)[N][N / 4], uint8_t *dst,
                                            int64_t ldd, int r, float *coef_, bool vec4, bool recon_) {
    float *coef = coef_;
    const bool recon = FAST || recon_;
    constexpr int H2 = N / 2;
    constexpr int NP = N / 2;           // column pairs
    constexpr int DR = D < N ? D : N;   // rows / columns of C that carry retained terms
    constexpr int DA = DR > 0 ? DR : 1; // array extent (D = 0 keeps nothing)
    // every diagonal present, or one copy serving every D up to its own (real plans):
    // mask each entry by its zig-zag index
    constexpr bool FULL = D >= 2 * N - 1 || REAL;
    const __half2 k1024 = __float2half2_rn(1024.0f);
    // pixels (A[k][2p], A[k][2p+1]) of column pair p as exact binary16 pairs
    auto px = [&](int k, int p) -> __half2 {
        return __hsub2(as_h2(bytes_to_biased_h2(w[k][p >> 1], (2 * p) & 3, (2 * p + 1) & 3)), k1024);
    };
    // column transform Y = T A (rows i < DR), two columns per instruction
    float Y[DA][N];
    if constexpr (REAL) {
        // FP32: mirrored sums / differences of the exact pixels, then the real
        // entries of M as constant-bank FFMA operands
        const float2 neg1f = make_float2(-1.0f, -1.0f);
#pragma unroll
        for (int p = 0; p < NP; p++) {
            float2 sp[H2], dp[H2];
#pragma unroll
            for (int j = 0; j < H2; j++) {
                const float2 top = __half22float2(px(j, p)), bot = __half22float2(px(N - 1 - j, p));
                sp[j] = __fadd2_rn(top, bot);
                dp[j] = __ffma2_rn(bot, neg1f, top);
            }
#pragma unroll
            for (int i = 0; i < DR; i++) {
                float ax = 0.0f, ay = 0.0f;
#pragma unroll
                for (int j = 0; j < H2; j++) {
                    const float2 v = (i & 1) ? dp[j] : sp[j];
                    ax = fmaf(P.T[i][j], v.x, ax);
                    ay = fmaf(P.T[i][j], v.y, ay);
                }
                Y[i][2 * p] = ax;
                Y[i][2 * p + 1] = ay;
            }
        }
    } else {
        // byte dot products on the transposed block (T as signed bytes): exact int32
        uint32_t tw[N][N / 4];   // [column][row group]
#pragma unroll
        for (int h = 0; h < N / 4; h++)
#pragma unroll
            for (int q = 0; q < N / 4; q++) {
                uint32_t o[4];
                transpose4x4(w[4 * h][q], w[4 * h + 1][q], w[4 * h + 2][q], w[4 * h + 3][q], o);
#pragma unroll
                for (int c = 0; c < 4; c++) tw[4 * q + c][h] = o[c];
            }
#pragma unroll
        for (int i = 0; i < DR; i++)
#pragma unroll
            for (int c = 0; c < N; c++) {
                int y = 0;
#pragma unroll
                for (int h = 0; h < N / 4; h++) y = dp4a_su(P.T8[i][h], tw[c][h], y);
                Y[i][c] = float(y);
            }
    }
    // row transform: C = Y T^T on the support i + j < D; zonal mask on the last diagonal
    // (quantised: only Bq = Bbar is kept, as exact FP32 integers; the inverse forms
    // Bbar o Qtilde where it reads it)
    [[maybe_unused]] float Cm[Q ? 1 : DA][Q ? 1 : DA];
    [[maybe_unused]] float Bq[Q ? DA : 1][Q ? DA : 1];
#pragma unroll
    for (int i = 0; i < DR; i++) {
        float s[H2], d[H2];
#pragma unroll
        for (int l = 0; l < H2; l++) {
            s[l] = Y[i][l] + Y[i][N - 1 - l];
            d[l] = Y[i][l] - Y[i][N - 1 - l];
        }
#pragma unroll
        for (int j = 0; j < DR; j++) {
            if (i + j < D) {
                float acc = 0.0f;
#pragma unroll
                for (int l = 0; l < H2; l++) acc = fmaf(P.T[j][l], (j & 1) ? d[l] : s[l], acc);
                const bool keep = FULL ? zz_index(N, i, j) < r : (i + j < D - 1 || zz_index(N, i, j) < r);
                if constexpr (Q) {
                    const float bq = keep ? quant_code<N>(P, i, j, acc) : 0.0f;
                    Bq[i][j] = bq;
                } else {
                    Cm[i][j] = keep ? acc : 0.0f;
                }
            }
        }
    }
    // normalised coefficients B = s_i s_j C in zig-zag order, first r
    if (FAST || coef) {
        if (vec4) {
#pragma unroll
            for (int k4 = 0; k4 < (N * N) / 4; k4++) {
                if (zz_row(N, 4 * k4) + zz_col(N, 4 * k4) < D && 4 * k4 < r) {
                    float v[4];
#pragma unroll
                    for (int q = 0; q < 4; q++) {
                        const int k = 4 * k4 + q, i = zz_row(N, k), j = zz_col(N, k);
                        if constexpr (Q) v[q] = (i + j < D) ? __int_as_float(int(Bq[i < DA ? i : 0][j < DA ? j : 0])) : 0.0f;
                        else v[q] = (i + j < D) ? P.sij[i][j] * Cm[Q ? 0 : (i < DA ? i : 0)][Q ? 0 : (j < DA ? j : 0)] : 0.0f;
                    }
                    *reinterpret_cast<float4 *>(coef + 4 * k4) = make_float4(v[0], v[1], v[2], v[3]);
                }
            }
        } else {
#pragma unroll
            for (int k = 0; k < N * N; k++) {
                const int i = zz_row(N, k), j = zz_col(N, k);
                if (i + j < D && k < r) {
                    if constexpr (Q) coef[k] = __int_as_float(int(Bq[i < DA ? i : 0][j < DA ? j : 0]));
                    else coef[k] = P.sij[i][j] * Cm[Q ? 0 : (i < DA ? i : 0)][Q ? 0 : (j < DA ? j : 0)];
                }
            }
        }
    }
    // inverse row transform: X[i][l] = sum_j C[i][j] T^{-1}[l][j]  (i < DR)
    // (j outer, l inner: each C'[i][j] is formed once and feeds the H2 sums; every
    // sum still runs over j in ascending order)
    float X[DA][N];
#pragma unroll
    for (int i = 0; i < DR; i++) {
        float e[H2], o[H2];
#pragma unroll
        for (int l = 0; l < H2; l++) e[l] = o[l] = 0.0f;
#pragma unroll
        for (int j = 0; j < DR; j++) {
            if (i + j < D) {
                float cm;
                if constexpr (Q) cm = Bq[i][j] * P.qt[i][j];
                else cm = Cm[i][j];
#pragma unroll
                for (int l = 0; l < H2; l++) {
                    if (j & 1) o[l] = fmaf(cm, P.Ti[l][j], o[l]);
                    else e[l] = fmaf(cm, P.Ti[l][j], e[l]);
                }
            }
        }
#pragma unroll
        for (int l = 0; l < H2; l++) {
            X[i][l] = e[l] + o[l];
            X[i][N - 1 - l] = e[l] - o[l];
        }
    }
    // inverse column transform A'[k][c] = sum_i T^{-1}[k][i] X[i][c], one mirrored row
    // pair (k, N-1-k) at a time, two columns per packed-FP32 instruction; error;
    // 8-bit output clip(floor(A' + 1/2), 0, 255)
    float2 sse2 = make_float2(0.0f, 0.0f);
    const float2 half2f = make_float2(0.5f, 0.5f), neg1 = make_float2(-1.0f, -1.0f);
#pragma unroll
    for (int k = 0; k < H2; k++) {
        uint32_t wt[N / 4], wb[N / 4];
#pragma unroll
        for (int q = 0; q < N / 4; q++) {
            uint32_t bt[4], bb[4];
#pragma unroll
            for (int h = 0; h < 2; h++) {
                const int p = 2 * q + h;
                float2 e2 = make_float2(0.0f, 0.0f), o2 = make_float2(0.0f, 0.0f);
#pragma unroll
                for (int i = 0; i < DR; i++) {
                    const float t = P.Ti[k][i];
                    const float2 x2 = make_float2(X[i][2 * p], X[i][2 * p + 1]);
                    if (i & 1) o2 = __ffma2_rn(make_float2(t, t), x2, o2);
                    else e2 = __ffma2_rn(make_float2(t, t), x2, e2);
                }
                const float2 top = __fadd2_rn(e2, o2), bot = __ffma2_rn(o2, neg1, e2);
                const __half2 at2 = px(k, p), ab2 = px(N - 1 - k, p);
                const float2 et = make_float2(sub_h_f(__low2half(at2), top.x), sub_h_f(__high2half(at2), top.y));
                const float2 eb = make_float2(sub_h_f(__low2half(ab2), bot.x), sub_h_f(__high2half(ab2), bot.y));
                sse2 = __ffma2_rn(et, et, sse2);
                sse2 = __ffma2_rn(eb, eb, sse2);
                const float2 vt = __fadd2_rn(top, half2f), vb = __fadd2_rn(bot, half2f);
                bt[2 * h] = floor_sat_u8(vt.x);
                bt[2 * h + 1] = floor_sat_u8(vt.y);
                bb[2 * h] = floor_sat_u8(vb.x);
                bb[2 * h + 1] = floor_sat_u8(vb.y);
            }
            wt[q] = __byte_perm(__byte_perm(bt[0], bt[1], 0x0040), __byte_perm(bt[2], bt[3], 0x0040), 0x5410);
            wb[q] = __byte_perm(__byte_perm(bb[0], bb[1], 0x0040), __byte_perm(bb[2], bb[3], 0x0040), 0x5410);
        }
        if (recon) {
            if constexpr (N == 8) {
                *reinterpret_cast<uint2 *>(dst + k * ldd) = make_uint2(wt[0], wt[1]);
                *reinterpret_cast<uint2 *>(dst + (N - 1 - k) * ldd) = make_uint2(wb[0], wb[1]);
            } else {
                *reinterpret_cast<uint32_t *>(dst + k * ldd) = wt[0];
                *reinterpret_cast<uint32_t *>(dst + (N - 1 - k) * ldd) = wb[0];
            }
        }
    }
    return sse2.x + sse2.y;
}

// One block of a shared-memory tile, transformed in place.
template <int N, int D, bool Q, bool FAST = false, bool REAL = false>
__device__ __forceinline__ float block_reg(const PlanK<N> &P, uint8_t *blk, int r, float *coef, bool vec4,
                                           bool recon) {
    uint32_t w[N][N / 4];
    load_block_words<N>(blk, TW, w);
    return block_core<N, D, Q, FAST, REAL>(P, w, blk, TW, r, coef, vec4, recon);
}

struct TileCoord {
    int img, ty, tx;
};

__device__ __forceinline__ TileCoord tile_coord(const FusedGeom &g, int64_t tile_id) {
    const int64_t per_img = int64_t(g.tiles_x) * g.tiles_y;
    TileCoord t;
    t.img = int(tile_id / per_img);
    const int rem = int(tile_id - int64_t(t.img) * per_img);
    t.ty = rem / g.tiles_x;
    t.tx = rem - t.ty * g.tiles_x;
    return t;
}

// Coordinates of the tiles a CTA visits (ids blockIdx.x, + gridDim.x, ...), advanced
// with two carries per step instead of a 64-bit division per tile.  The grid stride
// in (img, ty, tx) form comes with the launch (g.step_*, step_tx < tiles_x,
// step_ty < tiles_y).
struct TileWalker {
    TileCoord c;
    __device__ __forceinline__ void init(const FusedGeom &g) { c = tile_coord(g, blockIdx.x); }
    __device__ __forceinline__ void next(const FusedGeom &g) {
        c.tx += g.step_tx;
        int carry = 0;
        if (c.tx >= g.tiles_x) {
            c.tx -= g.tiles_x;
            carry = 1;
        }
        c.ty += g.step_ty + carry;
        carry = 0;
        if (c.ty >= g.tiles_y) {
            c.ty -= g.tiles_y;
            carry = 1;
        }
        c.img += g.step_img + carry;
    }
};

// Per-warp coefficient staging for N = 8: lane l's block writes its r coefficients at
// stage + l * STG8_LD (16-byte aligned, and lanes 272 bytes apart hit distinct
// banks); then the warp copies the first nb blocks' runs to dst as one contiguous
// run of nb * r floats (float4 when vec4).  Called by all 32 lanes.
constexpr int STG8_LD = 68;
__device__ __forceinline__ void warp_coef_copy8(float *dst, const float *src, int nb, int r, bool vec4, int lane) {
    // element c = b n + k of the run (n per block), advanced by 32 without a division
    if (vec4) {
        const int n = r >> 2, sb = 32 / n, sk = 32 - sb * n;
        int b = lane / n, k = lane - b * n;
        for (int c = lane; c < nb * n; c += 32) {
            reinterpret_cast<float4 *>(dst)[c] = *reinterpret_cast<const float4 *>(src + b * STG8_LD + 4 * k);
            b += sb;
            k += sk;
            if (k >= n) {
                k -= n;
                ++b;
            }
        }
    } else {
        const int sb = 32 / r, sk = 32 - sb * r;
        int b = lane / r, k = lane - b * r;
        for (int c = lane; c < nb * r; c += 32) {
            dst[c] = src[b * STG8_LD + k];
            b += sb;
            k += sk;
            if (k >= r) {
                k -= r;
                ++b;
            }
        }
    }
}

// N = 8 with any D (one CTA per SM): one block per consumer thread, warp w owning
// block-row w of the tile (32 blocks, one per lane).  Coefficients are staged per
// warp in shared memory and leave as one contiguous run per block-row.
template <bool Q>
__device__ __forceinline__ float tile_reg8_full(const PlanK<8> &P, const FusedGeom &g, uint8_t *tile,
                                                const TileCoord &tc, int ct, float *Zs) {
    constexpr int BPR = TW / 8;
    static_assert((TH / 8) * BPR == NCONS, "one block per consumer thread");
    const int lane = ct & 31, w = ct >> 5;
    const int bw = g.W / 8, r = g.r;
    const int gy = tc.ty * (TH / 8) + w, gx = tc.tx * BPR + lane;
    const bool row_in = gy * 8 < g.H;
    const bool coef = g.zcoef != nullptr && r > 0;
    float *stage = coef ? Zs + (w * 32 + lane) * STG8_LD : nullptr;
    float sse = 0.0f;
    if (row_in && gx * 8 < g.W)
        sse = block_reg<8, 15, Q>(P, tile + w * 8 * TW + lane * 8, r, stage, (r & 3) == 0, g.recon != nullptr);
    if (coef && row_in) {
        __syncwarp();
        const int nb = min(BPR, bw - tc.tx * BPR);  // blocks of this block-row inside the image
        float *dst = g.zcoef + (int64_t(tc.img) * g.blocks_per_img + int64_t(gy) * bw + tc.tx * BPR) * r;
        warp_coef_copy8(dst, Zs + w * 32 * STG8_LD, nb, r, g.coef_vec4 != 0, lane);
        __syncwarp();  // the staging area is rewritten by the next tile
    }
    return sse;
}

// The register path over one tile for a compile-time diagonal bound D: the bounds
// test per block only on tiles that reach past the image, the coefficient base of
// the image hoisted.
template <int N, int D, bool Q, bool FAST, bool REAL>
__device__ __forceinline__ float tile_reg_d(const PlanK<N> &P, const FusedGeom &g, uint8_t *tile, const TileCoord &tc,
                                            int ct) {
    constexpr int BPR = TW / N, BPT = (TH / N) * BPR;
    const int bw = g.W / N, r = g.r;
    const bool full = (tc.ty + 1) * TH <= g.H && (tc.tx + 1) * TW <= g.W;
    float *zimg = (FAST || g.zcoef) ? g.zcoef + int64_t(tc.img) * g.blocks_per_img * r : nullptr;
    // the 8-bit result is always written into the shared tile: a tile is stored back
    // only when a reconstruction is wanted, so the write needs no branch
    const bool vec4 = g.coef_vec4 != 0, recon = true;
    float sse = 0.0f;
#pragma unroll 1
    for (int q = ct; q < BPT; q += NCONS) {
        const int by = q / BPR, bx = q % BPR;
        const int gy = tc.ty * (TH / N) + by, gx = tc.tx * BPR + bx;
        if (!full && (gy * N >= g.H || gx * N >= g.W)) continue;
        float *coef = zimg ? zimg + (int64_t(gy) * bw + gx) * r : nullptr;
        sse += block_reg<N, D, Q, FAST, REAL>(P, tile + by * N * TW + bx * N, r, coef, vec4, recon);
    }
    return sse;
}

template <int N, bool Q, bool FAST, bool REAL>
__device__ __forceinline__ float tile_reg_f(const PlanK<N> &P, const FusedGeom &g, uint8_t *tile, const TileCoord &tc,
                                            int ct) {
    if constexpr (REAL) {  // one copy for every D it serves (N = 4: all; N = 8: D <= REG_DMAX8)
        return tile_reg_d<N, (N == 4 ? 2 * N - 1 : REG_DMAX8), Q, FAST, true>(P, g, tile, tc, ct);
    } else if constexpr (N == 4) {
        switch (g.D) {
            case 0: return tile_reg_d<4, 0, Q, FAST, REAL>(P, g, tile, tc, ct);
            case 1: return tile_reg_d<4, 1, Q, FAST, REAL>(P, g, tile, tc, ct);
            case 2: return tile_reg_d<4, 2, Q, FAST, REAL>(P, g, tile, tc, ct);
            case 3: return tile_reg_d<4, 3, Q, FAST, REAL>(P, g, tile, tc, ct);
            case 4: return tile_reg_d<4, 4, Q, FAST, REAL>(P, g, tile, tc, ct);
            case 5: return tile_reg_d<4, 5, Q, FAST, REAL>(P, g, tile, tc, ct);
            case 6: return tile_reg_d<4, 6, Q, FAST, REAL>(P, g, tile, tc, ct);
            default: return tile_reg_d<4, 7, Q, FAST, REAL>(P, g, tile, tc, ct);
        }
    } else {
        switch (g.D) {
            case 0: return tile_reg_d<N, 0, Q, FAST, REAL>(P, g, tile, tc, ct);
            case 1: return tile_reg_d<N, 1, Q, FAST, REAL>(P, g, tile, tc, ct);
            case 2: return tile_reg_d<N, 2, Q, FAST, REAL>(P, g, tile, tc, ct);
            case 3: return tile_reg_d<N, 3, Q, FAST, REAL>(P, g, tile, tc, ct);
            case 4: return tile_reg_d<N, 4, Q, FAST, REAL>(P, g, tile, tc, ct);
            default: return tile_reg_d<N, 5, Q, FAST, REAL>(P, g, tile, tc, ct);
        }
    }
}

// The D dispatch happens once per tile; calls with coefficients and reconstruction
// and no quantiser run a copy with those branches resolved (N = 4).
template <int N, bool Q, bool REAL = false>
__device__ __forceinline__ float tile_reg(const PlanK<N> &P, const FusedGeom &g, uint8_t *tile, const TileCoord &tc,
                                          int ct) {
    if constexpr (!Q && !REAL && N == 4) {
        if (g.zcoef != nullptr && g.recon != nullptr) return tile_reg_f<N, false, true, false>(P, g, tile, tc, ct);
    }
    return tile_reg_f<N, Q, false, REAL>(P, g, tile, tc, ct);
}

// ---------------------------------------------------------------------------
// Cooperative path: per block-row of the tile (N rows x 256 columns = 256/N
// blocks), column passes by thread-per-column, row passes by thread-per-(block,
// row), exchange through Ys (row stride LDY, conflict-free for both access
// patterns).  Coefficients are staged in Zs in zig-zag order and written out
// contiguously.  D and r are runtime values.
// ---------------------------------------------------------------------------
template <int N, bool Q>
__device__ __forceinline__ float tile_coop(const PlanK<N> &P, const FusedGeom &g, uint8_t *tile, const TileCoord &tc,
                                           int ct, float *Ys, float *Zs) {
    constexpr int H2 = N / 2;
    constexpr int BPR = TW / N;
    const int bw = g.W / N;
    const int D = g.D, r = g.r;
    const int Dr = D < N ? D : N;
    const bool col_in = (tc.tx * TW + ct) < g.W;
    float sse = 0.0f;

#pragma unroll 1
    for (int round = 0; round < TH / N; round++) {
        const int gy = tc.ty * (TH / N) + round;
        if (gy * N >= g.H) break;  // uniform across the consumers
        uint8_t *rows = tile + round * N * TW;
        // ---- pass 1: thread = column ct; Y = T A on rows i < Dr
        {
            float a[N];
#pragma unroll
            for (int k = 0; k < N; k++) a[k] = float(rows[k * TW + ct]);
            float s[H2], d[H2];
#pragma unroll
            for (int j = 0; j < H2; j++) {
                s[j] = a[j] + a[N - 1 - j];
                d[j] = a[j] - a[N - 1 - j];
            }
#pragma unroll
            for (int i = 0; i < N; i++) {
                if (i < Dr) {
                    float acc = 0.0f;
#pragma unroll
                    for (int j = 0; j < H2; j++) acc = fmaf(P.T[i][j], (i & 1) ? d[j] : s[j], acc);
                    Ys[i * LDY + ct] = acc;
                }
            }
        }
        named_sync(1, NCONS);
        // ---- pass 2: thread = (block b, row i); C[i][j] for i + j < D; coefficients; inverse row pass
        {
            const int b = ct / N, i = ct - (ct / N) * N;
            if (i < Dr) {
                float s[H2], d[H2];
#pragma unroll
                for (int l = 0; l < H2; l++) {
                    const float y0 = Ys[i * LDY + b * N + l], y1 = Ys[i * LDY + b * N + (N - 1 - l)];
                    s[l] = y0 + y1;
                    d[l] = y0 - y1;
                }
                float xe[H2], xo[H2];
#pragma unroll
                for (int l = 0; l < H2; l++) xe[l] = xo[l] = 0.0f;
                const int jmax = D - i;  // j < jmax
                const float si = P.s[i];
#pragma unroll
                for (int j = 0; j < N; j++) {
                    if (j < jmax) {
                        float acc = 0.0f;
#pragma unroll
                        for (int l = 0; l < H2; l++) acc = fmaf(P.T[j][l], (j & 1) ? d[l] : s[l], acc);
                        const int z = zz_index(N, i, j);
                        float c;
                        if constexpr (Q) {
                            const float bq = (z < r) ? quant_code<N>(P, i, j, acc) : 0.0f;
                            if (z < r) Zs[b * r + z] = __int_as_float(int(bq));
                            c = bq * P.qt[i][j];
                        } else {
                            c = (z < r) ? acc : 0.0f;
                            if (z < r) Zs[b * r + z] = (si * P.s[j]) * c;
                        }
#pragma unroll
                        for (int l = 0; l < H2; l++) {
                            if (j & 1) xo[l] = fmaf(c, P.Ti[l][j], xo[l]);
                            else xe[l] = fmaf(c, P.Ti[l][j], xe[l]);
                        }
                    }
                }
#pragma unroll
                for (int l = 0; l < H2; l++) {
                    Ys[i * LDY + b * N + l] = xe[l] + xo[l];
                    Ys[i * LDY + b * N + (N - 1 - l)] = xe[l] - xo[l];
                }
            }
        }
        named_sync(1, NCONS);
        // ---- coefficients of the round's blocks are contiguous in the output
        if (g.zcoef) {
            const int nb = min(BPR, bw - tc.tx * BPR);
            if (nb > 0) {
                float *dst = g.zcoef + (int64_t(tc.img) * g.blocks_per_img + int64_t(gy) * bw + tc.tx * BPR) * r;
                for (int q = ct; q < nb * r; q += NCONS) dst[q] = Zs[q];
            }
        }
        // ---- pass 3: thread = column; A' = T^{-1} X; error; 8-bit output in place
        {
            float xcol[N];
#pragma unroll
            for (int i = 0; i < N; i++) xcol[i] = (i < Dr) ? Ys[i * LDY + ct] : 0.0f;
#pragma unroll
            for (int k = 0; k < H2; k++) {
                float e = 0.0f, o = 0.0f;
#pragma unroll
                for (int i = 0; i < N; i++) {
                    if (i < Dr) {
                        if (i & 1) o = fmaf(P.Ti[k][i], xcol[i], o);
                        else e = fmaf(P.Ti[k][i], xcol[i], e);
                    }
                }
                const float top = e + o, bot = e - o;
                if (col_in) {
                    const float et = float(rows[k * TW + ct]) - top;
                    const float eb = float(rows[(N - 1 - k) * TW + ct]) - bot;
                    sse = fmaf(et, et, sse);
                    sse = fmaf(eb, eb, sse);
                }
                if (g.recon) {
                    rows[k * TW + ct] = uint8_t(recon_byte(top));
                    rows[(N - 1 - k) * TW + ct] = uint8_t(recon_byte(bot));
                }
            }
        }
        named_sync(1, NCONS);  // Ys / Zs are reused by the next round
    }
    return sse;
}

// ---------------------------------------------------------------------------
// Cooperative path for N = 16 and 32.  All block-rows of the tile (R = 64/N of
// them, NB = 256/N blocks each) are transformed together in three phases
// separated by barriers:
//   1. column pass: a thread takes two adjacent columns of one block-row and forms
//      Y = T A for rows i < Dr with packed-FP32 FMAs; Y goes to Ys;
//   2. row pass + inverse row pass: a thread takes one row i of one block; it forms
//      C[i][j] for i + j < D (masked to the first r zig-zag positions), stages the
//      normalised coefficients in Zs, and writes X[i][.] = sum_j C[i][j] T^{-1}[.][j]
//      back over its row of Ys.  Tasks are ordered by i so that each warp shares i
//      and the triangular bound j < D - i stays warp-uniform;
//   3. inverse column pass, two columns per thread: A' = T^{-1} X, error, 8-bit
//      output in place.
// Ys holds rows i < Dr of every block: index ((round * Dr + i) * NB + b) * (N + 4) + c,
// rows 16-byte aligned and padded by 4 floats per block against bank conflicts.
// ---------------------------------------------------------------------------
template <int N>
__host__ __device__ constexpr int coop2_rounds() { return TH / N; }

// Whether the coefficients are staged in shared memory (then written out
// contiguously per block-row) rather than stored from the row pass directly.
__host__ __device__ inline bool coop2_stage_coef(int N, int r) {
    return int64_t(TH / N) * (TW / N) * (r | 1) * 4 <= 32 * 1024;
}

template <int N, int DRM, bool Q = false>
__device__ __forceinline__ float tile_coop2(const PlanK<N> &P, const FusedGeom &g, uint8_t *tile, const TileCoord &tc,
                                            int ct, float *Ys, float *Zs) {
    constexpr int H2 = N / 2;
    constexpr int R = TH / N;
    constexpr int NB = TW / N;
    constexpr int LB = N + 4;  // padded block row in Ys
    const int bw = g.W / N;
    const int D = g.D, r = g.r;
    const int Dr = D < N ? D : N;
    const bool stage = coop2_stage_coef(N, r);
    const int rows_in = min(R, (g.H - tc.ty * TH) / N);  // block-rows of this tile inside the image
    const int nb_in = min(NB, bw - tc.tx * NB);           // blocks per block-row inside the image
    const float2 neg1 = make_float2(-1.0f, -1.0f);
    const float2 bias24 = make_float2(-16777216.0f, -16777216.0f);
    float sse = 0.0f;

    // ---- phase 1: column pass, two columns per task
    for (int t = ct; t < R * (TW / 2); t += NCONS) {
        const int round = t / (TW / 2), cp = t - round * (TW / 2);
        if (round >= rows_in) continue;
        const int b = (2 * cp) / N, cc = (2 * cp) - b * N;
        const uint8_t *col = tile + round * N * TW + 2 * cp;
        float2 sp[H2], dp[H2];
#pragma unroll
        for (int j = 0; j < H2; j++) {
            const uint32_t top = *reinterpret_cast<const uint16_t *>(col + j * TW);
            const uint32_t bot = *reinterpret_cast<const uint16_t *>(col + (N - 1 - j) * TW);
            // biased floats 2^23 + byte (exact); s = (t - 2^24) + b is exact, d = t - b is exact
            const float2 tf = make_float2(__uint_as_float(0x4B000000u | (top & 0xffu)),
                                          __uint_as_float(0x4B000000u | (top >> 8)));
            const float2 bf = make_float2(__uint_as_float(0x4B000000u | (bot & 0xffu)),
                                          __uint_as_float(0x4B000000u | (bot >> 8)));
            sp[j] = __fadd2_rn(__fadd2_rn(tf, bias24), bf);
            dp[j] = __ffma2_rn(bf, neg1, tf);
        }
        float *dst = Ys + (round * Dr * NB + b) * LB + cc;
#pragma unroll
        for (int i = 0; i < DRM; i++) {
            if (i < Dr) {
                // scalar FFMA: T's entries stay constant-bank operands
                float ax = 0.0f, ay = 0.0f;
#pragma unroll
                for (int j = 0; j < H2; j++) {
                    const float2 v = (i & 1) ? dp[j] : sp[j];
                    ax = fmaf(P.T[i][j], v.x, ax);
                    ay = fmaf(P.T[i][j], v.y, ay);
                }
                *reinterpret_cast<float2 *>(dst + i * NB * LB) = make_float2(ax, ay);
            }
        }
    }
    named_sync(1, NCONS);

    // ---- phase 2: row pass, coefficients, inverse row pass; one (block, row) per task
    for (int t = ct; t < R * NB * Dr; t += NCONS) {
        const int i = t / (R * NB), rb = t - i * (R * NB);
        const int round = rb / NB, b = rb - round * NB;
        if (round >= rows_in || b >= nb_in) continue;
        float *row = Ys + ((round * Dr + i) * NB + b) * LB;
        float s[H2], d[H2];
#pragma unroll
        for (int l4 = 0; l4 < N / 8; l4++) {
            const float4 lo = *reinterpret_cast<const float4 *>(row + 4 * l4);
            const float4 hi = *reinterpret_cast<const float4 *>(row + N - 4 - 4 * l4);
            // lo holds Y[4l4 .. 4l4+3], hi holds Y[N-4-4l4 .. N-1-4l4]
            s[4 * l4 + 0] = lo.x + hi.w; d[4 * l4 + 0] = lo.x - hi.w;
            s[4 * l4 + 1] = lo.y + hi.z; d[4 * l4 + 1] = lo.y - hi.z;
            s[4 * l4 + 2] = lo.z + hi.y; d[4 * l4 + 2] = lo.z - hi.y;
            s[4 * l4 + 3] = lo.w + hi.x; d[4 * l4 + 3] = lo.w - hi.x;
        }
        float xe[H2], xo[H2];
#pragma unroll
        for (int l = 0; l < H2; l++) xe[l] = xo[l] = 0.0f;
        const int jmax = D - i;
        const float si = P.s[i];
        float *zs = Zs + (round * NB + b) * (r | 1);  // odd block stride: no bank conflicts
        float *zg = g.zcoef ? g.zcoef + (int64_t(tc.img) * g.blocks_per_img +
                                         int64_t(tc.ty * R + round) * bw + tc.tx * NB + b) * r
                            : nullptr;
        // D <= DRM in every variant but the last, so C[i][j] != 0 only for j < min(DRM, N)
        constexpr int JM = DRM < N ? DRM : N;
#pragma unroll
        for (int j = 0; j < JM; j++) {
            if (j < jmax) {
                float acc = 0.0f;
#pragma unroll
                for (int l = 0; l < H2; l++) acc = fmaf(P.T[j][l], (j & 1) ? d[l] : s[l], acc);
                const int z = zz_index(N, i, j);
                const bool keep = z < r;
                float c, bval;
                if constexpr (Q) {
                    const float bq = keep ? quant_code<N>(P, i, j, acc) : 0.0f;
                    c = bq * P.qt[i][j];
                    bval = __int_as_float(int(bq));
                } else {
                    c = keep ? acc : 0.0f;
                    bval = (si * P.s[j]) * c;
                }
                if (keep) {
                    if (stage) zs[z] = bval;
                    else if (zg) zg[z] = bval;
                }
#pragma unroll
                for (int l = 0; l < H2; l++) {
                    if (j & 1) xo[l] = fmaf(c, P.Ti[l][j], xo[l]);
                    else xe[l] = fmaf(c, P.Ti[l][j], xe[l]);
                }
            }
        }
#pragma unroll
        for (int l4 = 0; l4 < N / 8; l4++) {
            float4 lo, hi;
            lo.x = xe[4 * l4 + 0] + xo[4 * l4 + 0]; hi.w = xe[4 * l4 + 0] - xo[4 * l4 + 0];
            lo.y = xe[4 * l4 + 1] + xo[4 * l4 + 1]; hi.z = xe[4 * l4 + 1] - xo[4 * l4 + 1];
            lo.z = xe[4 * l4 + 2] + xo[4 * l4 + 2]; hi.y = xe[4 * l4 + 2] - xo[4 * l4 + 2];
            lo.w = xe[4 * l4 + 3] + xo[4 * l4 + 3]; hi.x = xe[4 * l4 + 3] - xo[4 * l4 + 3];
            *reinterpret_cast<float4 *>(row + 4 * l4) = lo;
            *reinterpret_cast<float4 *>(row + N - 4 - 4 * l4) = hi;
        }
    }
    named_sync(1, NCONS);

    // ---- staged coefficients: each block-row's blocks are contiguous in the output
    if (stage && g.zcoef && r > 0) {
        for (int round = 0; round < rows_in; round++) {
            float *dst = g.zcoef + (int64_t(tc.img) * g.blocks_per_img + int64_t(tc.ty * R + round) * bw +
                                    tc.tx * NB) * r;
            const float *src = Zs + round * NB * (r | 1);
            // q = bq r + kq, advanced by NCONS = step_b r + step_k without a division
            const int step_b = NCONS / r, step_k = NCONS - step_b * r;
            int bq = ct / r, kq = ct - bq * r;
            for (int q = ct; q < nb_in * r; q += NCONS) {
                dst[q] = src[bq * (r | 1) + kq];
                bq += step_b;
                kq += step_k;
                if (kq >= r) {
                    kq -= r;
                    ++bq;
                }
            }
        }
    }

    // ---- phase 3: inverse column pass, two columns per task; error; 8-bit output in place
    const float2 half2f = make_float2(0.5f, 0.5f);
    const float2 bias23 = make_float2(-8388608.0f, -8388608.0f);
    const int x_in = g.W - tc.tx * TW;  // columns of this tile inside the image
    for (int t = ct; t < R * (TW / 2); t += NCONS) {
        const int round = t / (TW / 2), cp = t - round * (TW / 2);
        if (round >= rows_in) continue;
        const int b = (2 * cp) / N, cc = (2 * cp) - b * N;
        const bool col_in = 2 * cp < x_in;  // W is a multiple of N, so both columns are in or out
        uint8_t *col = tile + round * N * TW + 2 * cp;
        const float *src = Ys + (round * Dr * NB + b) * LB + cc;
        float2 xv[DRM];
#pragma unroll
        for (int i = 0; i < DRM; i++)
            xv[i] = (i < Dr) ? *reinterpret_cast<const float2 *>(src + i * NB * LB) : make_float2(0.0f, 0.0f);
        float2 sse2 = make_float2(0.0f, 0.0f);
#pragma unroll
        for (int k = 0; k < H2; k++) {
            float ex = 0.0f, ey = 0.0f, ox = 0.0f, oy = 0.0f;
#pragma unroll
            for (int i = 0; i < DRM; i++) {
                if (i < Dr) {
                    if (i & 1) {
                        ox = fmaf(P.Ti[k][i], xv[i].x, ox);
                        oy = fmaf(P.Ti[k][i], xv[i].y, oy);
                    } else {
                        ex = fmaf(P.Ti[k][i], xv[i].x, ex);
                        ey = fmaf(P.Ti[k][i], xv[i].y, ey);
                    }
                }
            }
            const float2 e2 = make_float2(ex, ey), o2 = make_float2(ox, oy);
            const float2 top = __fadd2_rn(e2, o2), bot = __ffma2_rn(o2, neg1, e2);
            uint16_t *pt = reinterpret_cast<uint16_t *>(col + k * TW);
            uint16_t *pb = reinterpret_cast<uint16_t *>(col + (N - 1 - k) * TW);
            const uint32_t wt = *pt, wb = *pb;
            if (col_in) {
                const float2 at = __fadd2_rn(make_float2(__uint_as_float(0x4B000000u | (wt & 0xffu)),
                                                         __uint_as_float(0x4B000000u | (wt >> 8))), bias23);
                const float2 ab = __fadd2_rn(make_float2(__uint_as_float(0x4B000000u | (wb & 0xffu)),
                                                         __uint_as_float(0x4B000000u | (wb >> 8))), bias23);
                const float2 et = __ffma2_rn(top, neg1, at), eb = __ffma2_rn(bot, neg1, ab);
                sse2 = __ffma2_rn(et, et, sse2);
                sse2 = __ffma2_rn(eb, eb, sse2);
            }
            if (g.recon) {
                const float2 vt = __fadd2_rn(top, half2f), vb = __fadd2_rn(bot, half2f);
                *pt = uint16_t(floor_sat_u8(vt.x) | (floor_sat_u8(vt.y) << 8));
                *pb = uint16_t(floor_sat_u8(vb.x) | (floor_sat_u8(vb.y) << 8));
            }
        }
        sse += sse2.x + sse2.y;
    }
    named_sync(1, NCONS);  // Ys / Zs are reused by the next tile
    return sse;
}

}  // namespace rklt

#include "rklt_tc.cuh"

namespace rklt {

// Kernel variant V (picked on the host from the diagonal bound D):
//   N = 4: 0 (register path, any D);  N = 8: 0 register path (D <= REG_DMAX8), else
//   REG8_FULL (the register path for the full block, one CTA per SM);
//   N = 32 with D <= 16, N = 16 with D <= 8: TC_V (tensor cores);
//   N >= 16 otherwise: 1, 2, 3 = cooperative path (all block-rows at once) sized for
//   Dr <= N/4, N/2, N;  real (exact KLT / DCT) plans: REG_REAL for N = 4 and for N = 8
//   with D <= REG_DMAX8, else 1 = cooperative path block-row by block-row.
// QV is added for the quantised form.
__host__ __device__ inline int fused_variant(int N, int D) {
    if (N == 4) return 0;
    if (N == 8) return D <= REG_DMAX8 ? 0 : REG8_FULL;
    if (N == 32 && D <= TC_DMAX) return TC_V;
    if (N == 16 && D <= TC_DMAX16) return TC_V;
    const int Dr = D < N ? D : N;
    return Dr <= N / 4 ? 1 : (Dr <= N / 2 ? 2 : 3);
}

// Variant for a real (exact KLT / DCT) plan: only the FP32 paths, since the register
// and tensor-core paths rely on T having entries in {0, +1, -1}.
__host__ __device__ inline int real_variant(int N, int D) {
    if (N == 4) return REG_REAL;
    if (N == 8) return D <= REG_DMAX8 ? REG_REAL : 1;
    const int Dr = D < N ? D : N;
    return Dr <= N / 4 ? 1 : (Dr <= N / 2 ? 2 : 3);
}

// Consumer threads of kernel variant V, and the CTAs per SM its registers are sized for.
__host__ __device__ constexpr int ncons(int V) { return vbase(V) == TC_V ? NCONS_TC : NCONS; }
__host__ __device__ constexpr int kminb(int V) { return vbase(V) == REG8_FULL ? 1 : (vbase(V) == TC_V ? 3 : 2); }

template <int N, int V>
__device__ __forceinline__ float process_tile(const PlanK<N> &P, const FusedGeom &g, uint8_t *tile, const TileCoord &tc,
                                              int ct, float *Ys, float *Zs) {
    if constexpr (N == 4 || N == 8) {
        constexpr bool Q = V >= QV;
        constexpr int VB = vbase(V);
        if constexpr (VB == 0) return tile_reg<N, Q>(P, g, tile, tc, ct);
        else if constexpr (VB == REG_REAL) return tile_reg<N, false, true>(P, g, tile, tc, ct);
        else if constexpr (N == 8 && VB == REG8_FULL) return tile_reg8_full<Q>(P, g, tile, tc, ct, Zs);
        else return tile_coop<N, Q>(P, g, tile, tc, ct, Ys, Zs);
    } else {
        constexpr bool Q = V >= QV;
        if constexpr (vbase(V) == 1) return tile_coop2<N, N / 4, Q>(P, g, tile, tc, ct, Ys, Zs);
        else if constexpr (vbase(V) == 2) return tile_coop2<N, N / 2, Q>(P, g, tile, tc, ct, Ys, Zs);
        else return tile_coop2<N, N, Q>(P, g, tile, tc, ct, Ys, Zs);
    }
}

// Sum of the NC / 32 consumer warps' partials of one tile, in warp order.
template <int NC>
__device__ __forceinline__ float sum_warp_partials(const float *w) {
    float t = 0.0f;
#pragma unroll
    for (int i = 0; i < NC / 32; i++) t += w[i];
    return t;
}

// Fixed-order reduction over the NC consumer threads; thread 0 returns the sum.
template <int NC>
__device__ __forceinline__ float reduce_consumers(float v, float *red, int ct) {
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
    if ((ct & 31) == 0) red[ct >> 5] = v;
    named_sync(2, NC);
    float t = 0.0f;
    if (ct == 0) {
#pragma unroll
        for (int w = 0; w < NC / 32; w++) t += red[w];
    }
    named_sync(2, NC);
    return t;
}

__device__ __forceinline__ void tile_origin(const TileCoord &t, int &x, int &y, int &z) {
    z = t.img;
    y = t.ty * TH;
    x = t.tx * TW;
}

// Tile layout in shared memory: row-major 64 x 256 bytes, or (tensor-core variant)
// two 64 x 128 halves in the 128-byte swizzled layout.
template <int V>
__device__ __forceinline__ int tile_off(int y, int x) {
    if constexpr (vbase(V) == TC_V) return swz_off(y, x);
    else return y * TW + x;
}

// TMA copies of one tile: one 256 x 64 box, or two 128 x 64 swizzled boxes (the
// second only when it starts inside the image).
template <int V>
__device__ __forceinline__ void load_tile(const CUtensorMap *map, const FusedGeom &g, int x, int y, int z,
                                          uint8_t *dst, uint64_t *bar) {
    if constexpr (vbase(V) == TC_V) {
        const bool two = x + TW / 2 < g.W;
        mbar_arrive_expect_tx(bar, two ? TILE_BYTES : TC_HALF);
        tma_load_3d(dst, map, x, y, z, bar);
        if (two) tma_load_3d(dst + TC_HALF, map, x + TW / 2, y, z, bar);
    } else {
        mbar_arrive_expect_tx(bar, TILE_BYTES);
        tma_load_3d(dst, map, x, y, z, bar);
    }
}

template <int V>
__device__ __forceinline__ void store_tile(const CUtensorMap *map, const FusedGeom &g, int x, int y, int z,
                                           const uint8_t *src) {
    tma_store_3d(map, x, y, z, src);
    if constexpr (vbase(V) == TC_V) {
        if (x + TW / 2 < g.W) tma_store_3d(map, x + TW / 2, y, z, src + TC_HALF);
    }
}

// Shared memory after 1 KB alignment: tile ring | barriers | reduction | Ys | Zs.
struct SmemLayout {
    int bar_off, red_off, ys_off, zs_off, total;
};

template <int N>
__host__ __device__ inline SmemLayout smem_layout(int stages, int r, int D, int V) {
    SmemLayout L{};
    L.bar_off = stages * TILE_BYTES;
    L.red_off = L.bar_off + 2 * STAGES * 8;
    L.ys_off = L.red_off + STAGES * (NCONS_MAX / 32) * 4;  // barrier and reduction slots, deepest ring
    int ys = 0, zs = 0;
    if (V == TC_V) {
        zs = (NCONS_TC / 32) * TC_ZS * 4 + TC_TAB_BYTES;
    } else if (N >= 16) {  // all block-rows at once
        const int Dr = D < N ? D : N;
        ys = (TH / N) * Dr * (TW / N) * (N + 4) * 4;
        zs = coop2_stage_coef(N, r) ? (TH / N) * (TW / N) * (r | 1) * 4 : 0;
    } else if (N == 8 && V == REG8_FULL) {  // per-warp coefficient staging
        zs = NCONS * STG8_LD * 4;
    } else if (V == 1) {  // N = 4, 8 cooperative path, block-row by block-row
        ys = N * LDY * 4;
        zs = (TW / N) * r * 4;
    }
    L.zs_off = L.ys_off + ((ys + 15) / 16) * 16;
    L.total = L.zs_off + zs + 1024;  // + slack for aligning the dynamic base
    return L;
}

// ---------------------------------------------------------------------------
// The kernel: warps 0..7 consume; warp 8 produces in TMA mode (idle otherwise).
// ---------------------------------------------------------------------------
template <int N, int V>
__global__ void __launch_bounds__(ncons(V) + 32, kminb(V))
    fused_kernel(const __grid_constant__ PlanK<N> P, const __grid_constant__ CUtensorMap tm_in,
                 const __grid_constant__ CUtensorMap tm_out, const FusedGeom g) {
    constexpr int NC = ncons(V);
    extern __shared__ uint8_t smem_raw[];
    // 1 KB aligned, by an offset from the shared array (so that every pointer derived
    // from it stays a shared-space pointer: LDS / STS with immediate offsets)
    uint8_t *smem = smem_raw + ((1024u - (smem_u32(smem_raw) & 1023u)) & 1023u);
    const int NST = g.stages;  // ring depth (<= STAGES)
    const SmemLayout L = smem_layout<N>(g.use_tma ? NST : 1, g.r, g.D, vbase(V));
    uint64_t *full = reinterpret_cast<uint64_t *>(smem + L.bar_off);
    uint64_t *empty = full + STAGES;
    float *red = reinterpret_cast<float *>(smem + L.red_off);
    float *Ys = reinterpret_cast<float *>(smem + L.ys_off);
    float *Zs = reinterpret_cast<float *>(smem + L.zs_off);
    const int tid = threadIdx.x;

    if (g.use_tma && tid == NC) {
        for (int s = 0; s < NST; s++) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], NC / 32);
        }
        fence_mbar_init();
    }
    __syncthreads();

    if (tid >= NC) {
        // ---------------- producer: one elected lane of warp 8 ----------------
        if (!g.use_tma || tid != NC) return;
        int64_t it = 0;
        bool ok = true;
        TileWalker lw, sw;  // tiles being loaded; tiles being written back (NST behind)
        lw.init(g);
        sw = lw;
        for (int64_t tile = blockIdx.x; tile < g.ntiles; tile += gridDim.x, ++it) {
            const int s = int(it % NST);
            if (it >= NST) {
                // slot s last held tile (it - STAGES): wait for its release, write it back
                if (!mbar_wait_bounded(&empty[s], uint32_t(((it / NST) - 1) & 1), g.timeout_ns)) {
                    ok = false;
                    break;
                }
                const int64_t prev = tile - int64_t(NST) * gridDim.x;
                g.partials[prev] = sum_warp_partials<NC>(red + s * (NC / 32));
                if (g.recon) {
                    int x, y, z;
                    tile_origin(sw.c, x, y, z);
                    store_tile<V>(&tm_out, g, x, y, z, smem + s * TILE_BYTES);
                    bulk_commit();
                    bulk_wait_read_all();  // the store has read the slot before it is refilled
                }
                sw.next(g);
            }
            if (g.inject_stall) continue;  // test hook: nothing ever completes full[s]
            int x, y, z;
            tile_origin(lw.c, x, y, z);
            lw.next(g);
            load_tile<V>(&tm_in, g, x, y, z, smem + s * TILE_BYTES, &full[s]);
        }
        // drain: write back the slots still holding consumed tiles
        const int64_t issued = it;
        for (int64_t j = issued > NST ? issued - NST : 0; j < issued; j++) {
            const int s = int(j % NST);
            const uint32_t par = uint32_t((j / NST) & 1);
            if (!ok || !mbar_wait_bounded(&empty[s], par, g.timeout_ns)) {
                // the consumers gave up: let this slot's load land before the CTA exits
                ok = false;
                if (!g.inject_stall) mbar_wait_bounded(&full[s], par, DRAIN_NS);
                continue;
            }
            const int64_t tj = int64_t(blockIdx.x) + j * gridDim.x;
            g.partials[tj] = sum_warp_partials<NC>(red + s * (NC / 32));
            if (g.recon) {
                int x, y, z;
                tile_origin(sw.c, x, y, z);
                store_tile<V>(&tm_out, g, x, y, z, smem + s * TILE_BYTES);
                bulk_commit();
            }
            sw.next(g);
        }
        bulk_wait_all();
        return;
    }

    // ---------------- consumers ----------------
    const bool al8 = ((reinterpret_cast<uintptr_t>(g.img) | uintptr_t(g.ld) | uintptr_t(g.img_stride)) & 7) == 0;
    const bool al8o =
        ((reinterpret_cast<uintptr_t>(g.recon) | uintptr_t(g.ld_recon) | uintptr_t(g.recon_stride)) & 7) == 0;
    // the cooperative path synchronises the consumer warps with named barriers, so
    // they must give up together; the register path has no such barrier
    constexpr bool coop = vbase(V) != 0 && vbase(V) != TC_V;
    TcLane tcl;
    uint4 *tctab = reinterpret_cast<uint4 *>(Zs + (NC / 32) * TC_ZS);
    const uint32_t tctabl = smem_u32(tctab) + 16 * (tid & 31);
    const uint32_t tczs = smem_u32(Zs + (tid >> 5) * TC_ZS);
    if constexpr (vbase(V) == TC_V) {
        if constexpr (N == 32) tc_setup(P, tcl, tctab, tid < 32, tid & 31, g.r, (tid >> 5) & 7, V >= QV);
        else tc16_setup(P, tcl, tctab, tid < 32, tid & 31, g.r, (tid >> 5) & 7, V >= QV);
        named_sync(1, NC);  // the table is written before any warp reads it
    }
    int64_t it = 0;
    TileWalker cw;
    cw.init(g);
    for (int64_t tile = blockIdx.x; tile < g.ntiles; tile += gridDim.x, ++it, cw.next(g)) {
        uint8_t *buf;
        int s = 0;
        int x0 = 0, y0 = 0, z = 0, hv = 0, wv = 0;
        if (g.use_tma) {
            s = int(it % NST);
            const bool got = mbar_wait_bounded(&full[s], uint32_t((it / NST) & 1), g.timeout_ns);
            if (coop ? named_any(3, NC, !got) : !got) break;
            buf = smem + s * TILE_BYTES;
        } else {
            buf = smem;
            tile_origin(cw.c, x0, y0, z);
            hv = min(TH, g.H - y0);
            wv = min(TW, g.W - x0);
            const uint8_t *src = g.img + int64_t(z) * g.img_stride + int64_t(y0) * g.ld + x0;
            named_sync(1, NC);  // the previous tile's copy-out has read the buffer
            if (al8) {
                for (int q = tid; q < TH * (TW / 8); q += NC) {
                    const int y = q / (TW / 8), x = (q - y * (TW / 8)) * 8;
                    uint2 v = make_uint2(0u, 0u);
                    if (y < hv && x + 8 <= wv) {
                        v = *reinterpret_cast<const uint2 *>(src + int64_t(y) * g.ld + x);
                    } else if (y < hv && x < wv) {  // ragged edge: only bytes inside the image
                        for (int e = 0; e < wv - x; e++) {
                            const uint32_t b = src[int64_t(y) * g.ld + x + e];
                            if (e < 4) v.x |= b << (8 * e);
                            else v.y |= b << (8 * (e - 4));
                        }
                    }
                    *reinterpret_cast<uint2 *>(buf + tile_off<V>(y, x)) = v;
                }
            } else {
                for (int q = tid; q < TILE_BYTES; q += NC) {
                    const int y = q / TW, x = q - y * TW;
                    buf[tile_off<V>(y, x)] = (y < hv && x < wv) ? src[int64_t(y) * g.ld + x] : uint8_t(0);
                }
            }
            named_sync(1, NC);
        }
        float v;
        if constexpr (vbase(V) == TC_V) {
            // the benchmark configuration (coefficients 16-byte aligned with r % 4 == 0,
            // and the reconstruction) runs a copy with those branches resolved
            constexpr bool Q = V >= QV;
            const bool fast = g.zcoef != nullptr && g.recon != nullptr && g.coef_vec4;
            if constexpr (N == 32) v = fast ? tile_tc<true, Q>(tcl, tctabl, g, buf, cw.c, tid, tczs)
                                            : tile_tc<false, Q>(tcl, tctabl, g, buf, cw.c, tid, tczs);
            else v = fast ? tile_tc16<true, Q>(tcl, tctabl, g, buf, cw.c, tid, tczs)
                          : tile_tc16<false, Q>(tcl, tctabl, g, buf, cw.c, tid, tczs);
        }
        else v = process_tile<N, V>(P, g, buf, cw.c, tid, Ys, Zs);
        if (g.use_tma) {
            // warp partial -> red[s][warp]; the producer sums the eight in order
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
            if ((tid & 31) == 0) red[s * (NC / 32) + (tid >> 5)] = v;
            if (g.recon) fence_proxy_async_smem();
            __syncwarp();
            if ((tid & 31) == 0) mbar_arrive(&empty[s]);
        } else {
            const float t = reduce_consumers<NC>(v, red, tid);
            if (tid == 0) g.partials[tile] = t;
        }
        if (!g.use_tma && g.recon) {
            named_sync(1, NC);
            uint8_t *dst = g.recon + int64_t(z) * g.recon_stride + int64_t(y0) * g.ld_recon + x0;
            if (al8o) {
                for (int q = tid; q < TH * (TW / 8); q += NC) {
                    const int y = q / (TW / 8), x = (q - y * (TW / 8)) * 8;
                    if (y < hv && x + 8 <= wv) {
                        *reinterpret_cast<uint2 *>(dst + int64_t(y) * g.ld_recon + x) =
                            *reinterpret_cast<const uint2 *>(buf + tile_off<V>(y, x));
                    } else if (y < hv && x < wv) {
                        for (int e = 0; e < wv - x; e++)
                            dst[int64_t(y) * g.ld_recon + x + e] = buf[tile_off<V>(y, x + e)];
                    }
                }
            } else {
                for (int q = tid; q < TILE_BYTES; q += NC) {
                    const int y = q / TW, x = q - y * TW;
                    if (y < hv && x < wv) dst[int64_t(y) * g.ld_recon + x] = buf[tile_off<V>(y, x)];
                }
            }
        }
    }
}

// Per-image FP64 sum of the tile partials in a fixed order, then
// PSNR = 10 log10(255^2 H W / SSE) (+inf for SSE = 0, NaN for an empty image).
static __global__ void finalize_kernel(const float *partials, int64_t tiles_per_img, int nimg, int H, int W,
                                       double *sse, float *psnr) {
    __shared__ double red[256];
    const int img = blockIdx.x;
    if (img >= nimg) return;
    double acc = 0.0;
    for (int64_t t = threadIdx.x; t < tiles_per_img; t += blockDim.x)
        acc += double(partials[int64_t(img) * tiles_per_img + t]);
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int off = blockDim.x / 2; off > 0; off >>= 1) {
        if (threadIdx.x < off) red[threadIdx.x] += red[threadIdx.x + off];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        const double s = red[0];
        const double npx = double(H) * double(W);
        if (sse) sse[img] = s;
        if (psnr) {
            float p;
            if (npx == 0.0) p = __int_as_float(0x7fc00000);
            else if (s == 0.0) p = __int_as_float(0x7f800000);
            else p = float(10.0 * log10(255.0 * 255.0 * npx / s));
            psnr[img] = p;
        }
    }
}

// Host launcher (arguments already validated by the C ABI layer).
template <int N>
rklt_status launch_fused(const Plan &plan, const FusedArgs &a, cudaStream_t st) {
    // rounded plans with T T^T diagonal on the register path: the error by Parseval
    if constexpr (N == 4 || N == 8) {
        const rklt_status ps = N == 4 ? launch_pars_n4(plan, a, st) : launch_pars_n8(plan, a, st);
        if (ps != RKLT_ERR_UNSUPPORTED) return ps;
    }
    FusedGeom g{};
    g.img = a.img;
    g.recon = a.recon;
    g.zcoef = a.zcoef;
    g.ld = a.ld;
    g.img_stride = a.nimg > 1 ? a.img_stride : a.ld * int64_t(a.H);
    g.ld_recon = a.ld_recon;
    g.recon_stride = a.nimg > 1 ? a.recon_stride : a.ld_recon * int64_t(a.H);
    g.H = a.H;
    g.W = a.W;
    g.nimg = a.nimg;
    g.tiles_x = (a.W + TW - 1) / TW;
    g.tiles_y = (a.H + TH - 1) / TH;
    g.ntiles = int64_t(g.tiles_x) * g.tiles_y * a.nimg;
    g.blocks_per_img = int64_t(a.H / N) * (a.W / N);
    g.r = a.r;
    g.D = diag_bound(N, a.r);
    g.coef_vec4 = (a.r % 4 == 0) && ((reinterpret_cast<uintptr_t>(a.zcoef) & 15) == 0);
    g.timeout_ns = wait_timeout_ns();
    g.inject_stall = inject_stall();
    const int64_t tiles_per_img = int64_t(g.tiles_x) * g.tiles_y;
    if (a.H == 0 || a.W == 0) {
        finalize_kernel<<<a.nimg, 256, 0, st>>>(nullptr, 0, a.nimg, a.H, a.W, a.sse, a.psnr);
        const cudaError_t e = cudaGetLastError();
        return e == cudaSuccess ? RKLT_OK : cuda_fail(e, "finalize launch");
    }

    // scratch: one FP32 SSE partial per tile, stream-ordered from a library pool
    void *scratch = nullptr;
    if (a.partials) {
        if (g.ntiles * int64_t(sizeof(float)) > a.scratch_cap)
            return fail(RKLT_ERR_ARG, "scratch array too small for this call");
        g.partials = a.partials;
    } else {
        cudaMemPool_t pool = scratch_pool();
        if (!pool) return fail(RKLT_ERR_CUDA, "could not create the scratch memory pool");
        if (cudaMallocFromPoolAsync(&scratch, size_t(g.ntiles) * sizeof(float), pool, st) != cudaSuccess)
            return fail(RKLT_ERR_OOM, "scratch allocation failed");
        g.partials = static_cast<float *>(scratch);
    }

    const auto is16 = [](const void *p, int64_t x, int64_t y) {
        return ((reinterpret_cast<uintptr_t>(p) | uintptr_t(x) | uintptr_t(y)) & 15) == 0;
    };
    bool tma = !a.force_plain && is16(a.img, a.ld, g.img_stride) &&
               (!a.recon || is16(a.recon, a.ld_recon, g.recon_stride));
    int V = plan.kind == 0 ? fused_variant(N, g.D) : real_variant(N, g.D);
    // quantised call: the plan's constants plus this call's quantiser tables
    PlanK<N> pq;
    const PlanK<N> *pk = &plan.kparams<N>();
    if (a.Q) {
        V += QV;
        pq = *pk;
        for (int i = 0; i < N; i++)
            for (int j = 0; j < N; j++) {
                pq.qw[i][j] = float(plan.s[i] * plan.s[j] / a.Q[i * N + j]);
                pq.qt[i][j] = float(a.Q[i * N + j] / (plan.s[i] * plan.s[j]));
            }
        pk = &pq;
    }
    const bool swz = vbase(V) == TC_V;
    const int box_w = swz ? TW / 2 : TW;
    CUtensorMap tin{}, tout{};
    if (tma) {
        tma = make_map_u8(&tin, a.img, a.W, a.H, a.nimg, a.ld, g.img_stride, box_w, TH, swz);
        if (tma && a.recon)
            tma = make_map_u8(&tout, a.recon, a.W, a.H, a.nimg, a.ld_recon, g.recon_stride, box_w, TH, swz);
        if (tma && !a.recon) tout = tin;
    }
    g.use_tma = tma ? 1 : 0;
    g.stages = swz ? 3 : (N >= 16 ? 3 : 4);
    const SmemLayout L = smem_layout<N>(tma ? g.stages : 1, a.r, g.D, vbase(V));
    const void *fn = nullptr;
    if constexpr (N == 4) {
        switch (V) {
            case 0: fn = reinterpret_cast<const void *>(fused_kernel<4, 0>); break;
            case REG_REAL: fn = reinterpret_cast<const void *>(fused_kernel<4, REG_REAL>); break;
            default: fn = reinterpret_cast<const void *>(fused_kernel<4, QV>); break;
        }
    } else if constexpr (N == 8) {
        switch (V) {
            case 0: fn = reinterpret_cast<const void *>(fused_kernel<8, 0>); break;
            case 1: fn = reinterpret_cast<const void *>(fused_kernel<8, 1>); break;
            case REG_REAL: fn = reinterpret_cast<const void *>(fused_kernel<8, REG_REAL>); break;
            case REG8_FULL: fn = reinterpret_cast<const void *>(fused_kernel<8, REG8_FULL>); break;
            case QV: fn = reinterpret_cast<const void *>(fused_kernel<8, QV>); break;
            default: fn = reinterpret_cast<const void *>(fused_kernel<8, QV + REG8_FULL>); break;
        }
    } else {
        switch (V) {
            case 1: fn = reinterpret_cast<const void *>(fused_kernel<N, 1>); break;
            case 2: fn = reinterpret_cast<const void *>(fused_kernel<N, 2>); break;
            case 3: fn = reinterpret_cast<const void *>(fused_kernel<N, 3>); break;
            case TC_V: fn = reinterpret_cast<const void *>(fused_kernel<N, TC_V>); break;
            case QV + 1: fn = reinterpret_cast<const void *>(fused_kernel<N, QV + 1>); break;
            case QV + 2: fn = reinterpret_cast<const void *>(fused_kernel<N, QV + 2>); break;
            case QV + 3: fn = reinterpret_cast<const void *>(fused_kernel<N, QV + 3>); break;
            default: fn = reinterpret_cast<const void *>(fused_kernel<N, QV + TC_V>); break;
        }
    }
    const int dev = ensure_smem_attr(fn);
    const int threads = ncons(V) + 32;
    int per_sm = occupancy(fn, threads, L.total);
    if (per_sm < 1) per_sm = 1;
    const int64_t grid = std::min<int64_t>(g.ntiles, int64_t(per_sm) * sm_count(dev));
    {
        const int64_t per_img = int64_t(g.tiles_x) * g.tiles_y;
        g.step_img = int(grid / per_img);
        const int rem = int(grid - int64_t(g.step_img) * per_img);
        g.step_ty = rem / g.tiles_x;
        g.step_tx = rem - g.step_ty * g.tiles_x;
    }
    {
        void *args[] = {const_cast<PlanK<N> *>(pk), &tin, &tout, &g};
        const cudaError_t le = cudaLaunchKernel(fn, dim3(unsigned(grid)), dim3(threads), args, L.total, st);
        if (le != cudaSuccess) {
            if (scratch) cudaFreeAsync(scratch, st);
            return cuda_fail(le, "fused kernel launch");
        }
    }
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) {
        finalize_kernel<<<a.nimg, 256, 0, st>>>(g.partials, tiles_per_img, a.nimg, a.H, a.W, a.sse, a.psnr);
        e = cudaGetLastError();
    }
    if (scratch) cudaFreeAsync(scratch, st);
    return e == cudaSuccess ? RKLT_OK : cuda_fail(e, "fused kernel launch");
}

// Reads and clears this translation unit's latched device status.
static unsigned int take_tu_status() {
    unsigned int v = 0, zero = 0;
    if (cudaMemcpyFromSymbol(&v, g_dev_status, sizeof(v)) != cudaSuccess) return 0;
    cudaMemcpyToSymbol(g_dev_status, &zero, sizeof(zero));
    return v;
}

}  // namespace rklt
