// rklt_reg.cuh -- the register path for rounded plans whose T T^T is diagonal
// (N = 4 for every rho; N = 8 with T1 or T4, i.e. rho below 0.39 or from 0.8 on),
// one N x N block per thread, with the error taken from Parseval's identity in
// integers.  Included by rklt_reg_n4.cu and rklt_reg_n8.cu.
//
// Per block (Sec. 4.1 and the Appendix of arXiv 2111.14239):
//   C  = T A T^T                 exact (int32 byte-dot-product column pass, FP32 row pass)
//   B  = (s s^T) o C             first r zig-zag coefficients (Eq. 1, Sec. 4.1)
//   A' = T^{-1} (M o C) T^{-T}   8-bit output clip(floor(A' + 1/2), 0, 255)
//   SSE of the block = sum a^2 - sum_retained C_ij^2 / (d_i d_j),  d = diag(T T^T)
// The last line is Parseval's identity for T^{-1} = T^T diag(1/d) (Eq. 1's orthogonal
// branch); with m = lcm(d) it is (m^2 sum a^2 - sum pw_ij C_ij^2) / m^2, pw_ij =
// (m/d_i)(m/d_j), all integers: the per-block error is exact, so the per-image sums
// are exact 64-bit integer sums (order-free: identical alone, in a batch, in any
// grid) and the SSE is exactly that of the unrounded reconstruction A'.
//
// Column pass: dp4a on transposed bytes, four terms per instruction, T's rows as
// packed signed bytes (T is in {0, +1, -1}).
// Operand pairing for the packed FP32 instructions (FADD2 / FFMA2 / FMUL2):
//   row pass      two rows (i, i+1) per pair; T's entries as (t, t) constant pairs
//   U = T^{-1} C' two rows of C' per pair against (T^{-1}[k][i], T^{-1}[k][i+1]): the
//                 lanes collect the even-i and odd-i sums, U[k] = e + o, U[N-1-k] = e - o
//   A' = U T^{-T} rows (k, N-1-k) per pair; (t, t) constant pairs; even-j and odd-j
//                 sums give columns c and N-1-c (the row parity of T^{-1})
// so no pass needs a register shuffle.  The 1/2 of the rounding rides in the even
// accumulator's start value; the 8-bit conversion adds 1024 and truncates in
// binary16, where the spacing on [1024, 2048) is 1 (no conversion-unit instruction).
// Each thread transforms two blocks at once (PARS_B).
#pragma once

#include "rklt_fused_impl.cuh"

namespace rklt {

constexpr int PARS_DMAX8 = 5;   // N = 8: diagonal bounds served here (r <= 15)

__device__ __forceinline__ float2 ld_pair(const float *p) { return *reinterpret_cast<const float2 *>(p); }

// B blocks held in registers (w[b], N/4 words per row), transformed together: every
// constant operand is loaded once for the B blocks and the B instruction streams
// are independent.  Returns the blocks' error times m^2 as an exact integer (blocks
// with act[b] false -- outside the image -- add nothing and store no coefficients);
// writes the coefficients (COEF) and the 8-bit reconstruction over each block's
// bytes at dst[b], row stride LDD (RECON).
template <int N, int D, bool COEF, bool RECON, int B, int LDD = TW>
__device__ __forceinline__ uint64_t pars_blocks(const PlanK<N> &P, const uint32_t (&w)[B][N][N / 4],
                                                uint8_t *const (&dst)[B], int r, float *const (&coef)[B],
                                                const bool (&act)[B], int cvec) {
    constexpr int H2 = N / 2;
    constexpr int NP = N / 2;             // column pairs
    constexpr int DR = D < N ? D : N;     // rows / columns of C that carry retained terms
    constexpr int DA = DR > 0 ? DR : 1;
    const float2 neg1 = make_float2(-1.0f, -1.0f);

    // ---- pixel energy, exact: four bytes per dp4a
    uint32_t sa[B][2];
#pragma unroll
    for (int b = 0; b < B; b++) {
        sa[b][0] = sa[b][1] = 0;
#pragma unroll
        for (int k = 0; k < N; k++)
#pragma unroll
            for (int q = 0; q < N / 4; q++) {
                const int h = (k + q) & 1;
                sa[b][h] = __dp4a(w[b][k][q], w[b][k][q], sa[b][h]);
            }
    }

    // ---- column pass Y = T A (rows i < DR) by byte dot products: the block's columns
    // become words of four rows (PRMT 4 x 4 transposes), and Y[i][c] = sum_k T[i][k]
    // A[k][c] is exact in int32 (T as signed bytes, pixels unsigned); |Y| < 2^11, so
    // the conversion to FP32 is exact
    float Y[B][DA][N];
#pragma unroll
    for (int b = 0; b < B; b++) {
        uint32_t tw[N][N / 4];   // [column][row group]
#pragma unroll
        for (int h = 0; h < N / 4; h++)
#pragma unroll
            for (int q = 0; q < N / 4; q++) {
                uint32_t o[4];
                transpose4x4(w[b][4 * h][q], w[b][4 * h + 1][q], w[b][4 * h + 2][q], w[b][4 * h + 3][q], o);
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
                Y[b][i][c] = float(y);
            }
    }

    // ---- row pass C = Y T^T on the support i + j < D, rows in pairs (exact: integers
    // below 2^24 in FP32)
    float C[B][DA][DA];
#pragma unroll
    for (int i = 0; i < DR; i += 2) {
        if (i + 1 < DR) {
            float2 s[B][H2], d[B][H2];
#pragma unroll
            for (int b = 0; b < B; b++)
#pragma unroll
                for (int l = 0; l < H2; l++) {
                    const float2 a = make_float2(Y[b][i][l], Y[b][i + 1][l]);
                    const float2 c = make_float2(Y[b][i][N - 1 - l], Y[b][i + 1][N - 1 - l]);
                    s[b][l] = __fadd2_rn(a, c);
                    d[b][l] = __ffma2_rn(c, neg1, a);
                }
#pragma unroll
            for (int j = 0; j < DR; j++) {
                if (i + 1 + j < D) {
                    float2 acc[B];
#pragma unroll
                    for (int l = 0; l < H2; l++) {
                        const float2 t = P.Td[j][l];
#pragma unroll
                        for (int b = 0; b < B; b++) {
                            const float2 v = (j & 1) ? d[b][l] : s[b][l];
                            acc[b] = l == 0 ? __fmul2_rn(t, v) : __ffma2_rn(t, v, acc[b]);
                        }
                    }
#pragma unroll
                    for (int b = 0; b < B; b++) {
                        C[b][i][j] = acc[b].x;
                        C[b][i + 1][j] = acc[b].y;
                    }
                } else if (i + j < D) {
                    float acc[B];
#pragma unroll
                    for (int l = 0; l < H2; l++) {
                        const float t = P.T[j][l];
#pragma unroll
                        for (int b = 0; b < B; b++)
                            acc[b] = fmaf(t, (j & 1) ? d[b][l].x : s[b][l].x, l == 0 ? 0.0f : acc[b]);
                    }
#pragma unroll
                    for (int b = 0; b < B; b++) C[b][i][j] = acc[b];
                }
            }
        } else {
            float s[B][H2], d[B][H2];
#pragma unroll
            for (int b = 0; b < B; b++)
#pragma unroll
                for (int l = 0; l < H2; l++) {
                    s[b][l] = Y[b][i][l] + Y[b][i][N - 1 - l];
                    d[b][l] = Y[b][i][l] - Y[b][i][N - 1 - l];
                }
#pragma unroll
            for (int j = 0; j < DR; j++) {
                if (i + j < D) {
                    float acc[B];
#pragma unroll
                    for (int l = 0; l < H2; l++) {
                        const float t = P.T[j][l];
#pragma unroll
                        for (int b = 0; b < B; b++)
                            acc[b] = fmaf(t, (j & 1) ? d[b][l] : s[b][l], l == 0 ? 0.0f : acc[b]);
                    }
#pragma unroll
                    for (int b = 0; b < B; b++) C[b][i][j] = acc[b];
                }
            }
        }
    }
    // zonal mask: only the last diagonal can hold dropped positions
#pragma unroll
    for (int i = 0; i < DR; i++)
#pragma unroll
        for (int j = 0; j < DR; j++)
            if (i + j == D - 1) {
                const bool keep = zz_index(N, i, j) < r;
#pragma unroll
                for (int b = 0; b < B; b++) C[b][i][j] = keep ? C[b][i][j] : 0.0f;
            }

    // ---- normalised coefficients B = s_i s_j C in zig-zag order, first r
    if constexpr (COEF) {
#pragma unroll
        for (int b = 0; b < B; b++) {
            if (!act[b]) continue;
            const auto val = [&](int k) -> float {
                const int i = zz_row(N, k), j = zz_col(N, k);
                return (i + j < D) ? P.sij[i][j] * C[b][i < DA ? i : 0][j < DA ? j : 0] : 0.0f;
            };
            if (cvec == 4) {
#pragma unroll
                for (int k4 = 0; k4 < (N * N) / 4; k4++)
                    if (zz_row(N, 4 * k4) + zz_col(N, 4 * k4) < D && 4 * k4 < r)
                        *reinterpret_cast<float4 *>(coef[b] + 4 * k4) =
                            make_float4(val(4 * k4), val(4 * k4 + 1), val(4 * k4 + 2), val(4 * k4 + 3));
            } else if (cvec == 2) {
#pragma unroll
                for (int k2 = 0; k2 < (N * N) / 2; k2++)
                    if (zz_row(N, 2 * k2) + zz_col(N, 2 * k2) < D && 2 * k2 < r)
                        *reinterpret_cast<float2 *>(coef[b] + 2 * k2) = make_float2(val(2 * k2), val(2 * k2 + 1));
            } else {
#pragma unroll
                for (int k = 0; k < N * N; k++)
                    if (zz_row(N, k) + zz_col(N, k) < D && k < r) coef[b][k] = val(k);
            }
        }
    }

    // ---- block errors by Parseval, in integers: |C| < 2^15, so C^2 fits 32 bits, and
    // the retained energy of a block (pw-weighted) never exceeds m^2 sum a^2
    uint64_t err = 0;
#pragma unroll
    for (int b = 0; b < B; b++) {
        uint64_t kept = 0;
#pragma unroll
        for (int i = 0; i < DR; i++)
#pragma unroll
            for (int j = 0; j < DR; j++)
                if (i + j < D) {
                    const int c = __float2int_rn(C[b][i][j]);
                    kept += static_cast<uint64_t>(uint32_t(c * c)) * uint32_t(P.pw[i][j]);
                }
        const uint64_t e = static_cast<uint64_t>(uint32_t(P.pm2)) * (sa[b][0] + sa[b][1]) - kept;
        err += act[b] ? e : 0ull;
    }

    if constexpr (RECON) {
        // ---- U = T^{-1} C' (rows k and N-1-k of U as one pair), j < DR
        float2 U[B][H2][DA];
#pragma unroll
        for (int k = 0; k < H2; k++) {
#pragma unroll
            for (int j = 0; j < DR; j++) {
                float2 eo[B];   // (sum over even i, sum over odd i)
                bool odd = false, first = true;
#pragma unroll
                for (int i = 0; i < DR; i += 2) {
                    if (i + 1 < DR && i + 1 + j < D) {
                        const float2 t = ld_pair(&P.Ti[k][i]);
#pragma unroll
                        for (int b = 0; b < B; b++) {
                            const float2 c = make_float2(C[b][i][j], C[b][i + 1][j]);
                            eo[b] = first ? __fmul2_rn(c, t) : __ffma2_rn(c, t, eo[b]);
                        }
                        odd = true;
                        first = false;
                    } else if (i + j < D) {
                        const float t = P.Ti[k][i];
#pragma unroll
                        for (int b = 0; b < B; b++) {
                            if (first) eo[b] = make_float2(C[b][i][j] * t, 0.0f);
                            else eo[b].x = fmaf(C[b][i][j], t, eo[b].x);
                        }
                        first = false;
                    }
                }
#pragma unroll
                for (int b = 0; b < B; b++)
                    U[b][k][j] = odd ? make_float2(eo[b].x + eo[b].y, eo[b].x - eo[b].y)
                                     : make_float2(eo[b].x, eo[b].x);
            }
        }
        // ---- A' + 1/2 = U T^{-T} + 1/2: rows (k, N-1-k) per pair, columns c and N-1-c
        // from the even-j and odd-j sums; floor and saturate to bytes
        const float2 half2f = make_float2(0.5f, 0.5f);
#pragma unroll
        for (int k = 0; k < H2; k++) {
            float top[B][N], bot[B][N];
#pragma unroll
            for (int c = 0; c < H2; c++) {
                float2 e[B], o[B];
#pragma unroll
                for (int b = 0; b < B; b++) {
                    e[b] = half2f;
                    o[b] = make_float2(0.0f, 0.0f);
                }
#pragma unroll
                for (int j = 0; j < DR; j++) {
                    const float2 t = P.Tid[c][j];
#pragma unroll
                    for (int b = 0; b < B; b++) {
                        if (j & 1) o[b] = j == 1 ? __fmul2_rn(U[b][k][j], t) : __ffma2_rn(U[b][k][j], t, o[b]);
                        else e[b] = __ffma2_rn(U[b][k][j], t, e[b]);
                    }
                }
#pragma unroll
                for (int b = 0; b < B; b++) {
                    // + 1024: binary16 truncation is the floor on [1024, 2048) (bytes4_biased)
                    e[b] = __fadd2_rn(e[b], make_float2(1024.0f, 1024.0f));
                    const float2 lft = __fadd2_rn(e[b], o[b]);          // columns c     of rows k, N-1-k
                    const float2 rgt = __ffma2_rn(o[b], neg1, e[b]);    // columns N-1-c of rows k, N-1-k
                    top[b][c] = lft.x;
                    bot[b][c] = lft.y;
                    top[b][N - 1 - c] = rgt.x;
                    bot[b][N - 1 - c] = rgt.y;
                }
            }
#pragma unroll
            for (int b = 0; b < B; b++) {
                uint32_t wt[N / 4], wb[N / 4];
#pragma unroll
                for (int q = 0; q < N / 4; q++) {
                    wt[q] = bytes4_biased(top[b][4 * q], top[b][4 * q + 1], top[b][4 * q + 2], top[b][4 * q + 3]);
                    wb[q] = bytes4_biased(bot[b][4 * q], bot[b][4 * q + 1], bot[b][4 * q + 2], bot[b][4 * q + 3]);
                }
                if constexpr (N == 8) {
                    *reinterpret_cast<uint2 *>(dst[b] + k * LDD) = make_uint2(wt[0], wt[1]);
                    *reinterpret_cast<uint2 *>(dst[b] + (N - 1 - k) * LDD) = make_uint2(wb[0], wb[1]);
                } else {
                    *reinterpret_cast<uint32_t *>(dst[b] + k * LDD) = wt[0];
                    *reinterpret_cast<uint32_t *>(dst[b] + (N - 1 - k) * LDD) = wb[0];
                }
            }
        }
    }
    return err;
}

// Sum of a u64 over the warp; every lane gets the total.
__device__ __forceinline__ uint64_t warp_sum_u64(uint64_t v) {
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
    return v;
}

// Sum of the NC / 32 consumer warps' tile errors.
template <int NC>
__device__ __forceinline__ uint64_t pars_red_sum(const uint64_t *w) {
    uint64_t t = 0;
#pragma unroll
    for (int i = 0; i < NC / 32; i++) t += w[i];
    return t;
}

// The blocks of one tile owned by consumer thread ct (NC consumers), B at a time;
// errors added to acc.
template <int N, int D, bool COEF, bool RECON, int NC, int B>
__device__ __forceinline__ void pars_tile(const PlanK<N> &P, const FusedGeom &g, uint8_t *tile, const TileCoord &tc,
                                          int ct, uint64_t &acc) {
    constexpr int BPR = TW / N, BPT = (TH / N) * BPR;
    static_assert(BPT % (NC * B) == 0, "whole steps of B blocks per consumer");
    const int bw = g.W / N, r = g.r;
    const bool full = (tc.ty + 1) * TH <= g.H && (tc.tx + 1) * TW <= g.W;
    float *zimg = COEF ? g.zcoef + int64_t(tc.img) * g.blocks_per_img * r : nullptr;
#pragma unroll 1
    for (int q0 = ct; q0 < BPT; q0 += NC * B) {
        uint32_t w[B][N][N / 4];
        uint8_t *blk[B];
        float *coef[B];
        bool act[B];
#pragma unroll
        for (int b = 0; b < B; b++) {
            const int q = q0 + b * NC;
            const int by = q / BPR, bx = q % BPR;
            const int gy = tc.ty * (TH / N) + by, gx = tc.tx * BPR + bx;
            act[b] = full || (gy * N < g.H && gx * N < g.W);
            blk[b] = tile + by * N * TW + bx * N;
            coef[b] = COEF ? zimg + (int64_t(gy) * bw + gx) * r : nullptr;
            load_block_words<N>(blk[b], TW, w[b]);
        }
        acc += pars_blocks<N, D, COEF, RECON, B>(P, w, blk, r, coef, act, g.coef_vec4);
    }
}

// Copies one tile into the shared buffer with plain loads (bytes outside the image
// read as 0); the consumers call it together.
template <int NC>
__device__ __forceinline__ void plain_tile_in(const FusedGeom &g, const TileCoord &c, uint8_t *buf, int tid) {
    int x0, y0, z;
    tile_origin(c, x0, y0, z);
    const int hv = min(TH, g.H - y0), wv = min(TW, g.W - x0);
    const uint8_t *src = g.img + int64_t(z) * g.img_stride + int64_t(y0) * g.ld + x0;
    const bool al8 = ((reinterpret_cast<uintptr_t>(g.img) | uintptr_t(g.ld) | uintptr_t(g.img_stride)) & 7) == 0;
    if (al8) {
        for (int q = tid; q < TH * (TW / 8); q += NC) {
            const int y = q / (TW / 8), x = (q - y * (TW / 8)) * 8;
            uint2 v = make_uint2(0u, 0u);
            if (y < hv && x + 8 <= wv) {
                v = *reinterpret_cast<const uint2 *>(src + int64_t(y) * g.ld + x);
            } else if (y < hv && x < wv) {
                for (int e = 0; e < wv - x; e++) {
                    const uint32_t b = src[int64_t(y) * g.ld + x + e];
                    if (e < 4) v.x |= b << (8 * e);
                    else v.y |= b << (8 * (e - 4));
                }
            }
            *reinterpret_cast<uint2 *>(buf + y * TW + x) = v;
        }
    } else {
        for (int q = tid; q < TILE_BYTES; q += NC) {
            const int y = q / TW, x = q - y * TW;
            buf[y * TW + x] = (y < hv && x < wv) ? src[int64_t(y) * g.ld + x] : uint8_t(0);
        }
    }
}

// Copies the tile's reconstruction out with plain stores (only pixels inside the image).
template <int NC>
__device__ __forceinline__ void plain_tile_out(const FusedGeom &g, const TileCoord &c, const uint8_t *buf, int tid) {
    int x0, y0, z;
    tile_origin(c, x0, y0, z);
    const int hv = min(TH, g.H - y0), wv = min(TW, g.W - x0);
    uint8_t *dst = g.recon + int64_t(z) * g.recon_stride + int64_t(y0) * g.ld_recon + x0;
    const bool al8 =
        ((reinterpret_cast<uintptr_t>(g.recon) | uintptr_t(g.ld_recon) | uintptr_t(g.recon_stride)) & 7) == 0;
    if (al8) {
        for (int q = tid; q < TH * (TW / 8); q += NC) {
            const int y = q / (TW / 8), x = (q - y * (TW / 8)) * 8;
            if (y < hv && x + 8 <= wv) {
                *reinterpret_cast<uint2 *>(dst + int64_t(y) * g.ld_recon + x) =
                    *reinterpret_cast<const uint2 *>(buf + y * TW + x);
            } else if (y < hv && x < wv) {
                for (int e = 0; e < wv - x; e++) dst[int64_t(y) * g.ld_recon + x + e] = buf[y * TW + x + e];
            }
        }
    } else {
        for (int q = tid; q < TILE_BYTES; q += NC) {
            const int y = q / TW, x = q - y * TW;
            if (y < hv && x < wv) dst[int64_t(y) * g.ld_recon + x] = buf[y * TW + x];
        }
    }
}

// ---------------------------------------------------------------------------
// The kernel: warps 0..3 consume (PARS_B blocks per thread per step over the tile);
// warp 4 is the TMA producer (idle with plain loads).  OUT: bit 0 coefficients,
// bit 1 8-bit reconstruction.  Each tile's error (an exact integer, times m^2) goes
// to g.sse_acc[tile]: every tile is written exactly once, so the scratch needs no
// clearing, and the per-image sums of exact integers do not depend on their order.
// ---------------------------------------------------------------------------
// Consumer threads per CTA and blocks per consumer step.  Two blocks per thread:
// each constant operand load and each per-tile step serves two blocks, and a warp
// carries two independent instruction streams (measured faster than one block per
// thread with twice the warps, and than four).
constexpr int PARS_B = 2;
constexpr int PARS_NC = 128;

template <int N, int D, int OUT>
__global__ void __launch_bounds__(PARS_NC + 32, 2)
    pars_kernel(const __grid_constant__ PlanK<N> P, const __grid_constant__ CUtensorMap tm_in,
                const __grid_constant__ CUtensorMap tm_out, const FusedGeom g) {
    constexpr bool COEF = (OUT & 1) != 0, RECON = (OUT & 2) != 0;
    constexpr int PNC = PARS_NC;
    extern __shared__ uint8_t smem_raw[];
    uint8_t *smem = smem_raw + ((1024u - (smem_u32(smem_raw) & 1023u)) & 1023u);
    const int NST = g.stages;
    uint64_t *full = reinterpret_cast<uint64_t *>(smem + (g.use_tma ? NST : 1) * TILE_BYTES);
    uint64_t *empty = full + STAGES;
    uint64_t *red = empty + STAGES;   // [stage][consumer warp] tile errors
    const int tid = threadIdx.x;

    if (g.use_tma && tid == PNC) {
        for (int s = 0; s < NST; s++) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], PNC / 32);
        }
        fence_mbar_init();
    }
    __syncthreads();

    if (tid >= PNC) {
        // ---------------- producer: one elected lane of warp 8 ----------------
        if (!g.use_tma || tid != PNC) return;
        int64_t it = 0;
        bool ok = true;
        TileWalker lw, sw;  // tiles being loaded; tiles being written back (NST behind)
        lw.init(g);
        sw = lw;
        for (int64_t tile = blockIdx.x; tile < g.ntiles; tile += gridDim.x, ++it) {
            const int s = int(it % NST);
            if (it >= NST) {
                if (!mbar_wait_bounded(&empty[s], uint32_t(((it / NST) - 1) & 1), g.timeout_ns)) {
                    ok = false;
                    break;
                }
                g.sse_acc[tile - int64_t(NST) * gridDim.x] = pars_red_sum<PNC>(red + s * (PNC / 32));
                if (RECON) {
                    int x, y, z;
                    tile_origin(sw.c, x, y, z);
                    tma_store_3d(&tm_out, x, y, z, smem + s * TILE_BYTES);
                    bulk_commit();
                    bulk_wait_read_all();  // the store has read the slot before it is refilled
                }
                sw.next(g);
            }
            if (g.inject_stall) continue;  // test hook: nothing ever completes full[s]
            int x, y, z;
            tile_origin(lw.c, x, y, z);
            lw.next(g);
            mbar_arrive_expect_tx(&full[s], TILE_BYTES);
            tma_load_3d(smem + s * TILE_BYTES, &tm_in, x, y, z, &full[s]);
        }
        const int64_t issued = it;
        for (int64_t j = issued > NST ? issued - NST : 0; j < issued; j++) {
            const int s = int(j % NST);
            const uint32_t par = uint32_t((j / NST) & 1);
            if (!ok || !mbar_wait_bounded(&empty[s], par, g.timeout_ns)) {
                ok = false;
                if (!g.inject_stall) mbar_wait_bounded(&full[s], par, DRAIN_NS);
                continue;
            }
            g.sse_acc[int64_t(blockIdx.x) + j * gridDim.x] = pars_red_sum<PNC>(red + s * (PNC / 32));
            if (RECON) {
                int x, y, z;
                tile_origin(sw.c, x, y, z);
                tma_store_3d(&tm_out, x, y, z, smem + s * TILE_BYTES);
                bulk_commit();
            }
            sw.next(g);
        }
        bulk_wait_all();
        return;
    }

    // ---------------- consumers ----------------
    int64_t it = 0;
    TileWalker cw;
    cw.init(g);
    for (int64_t tile = blockIdx.x; tile < g.ntiles; tile += gridDim.x, ++it, cw.next(g)) {
        uint8_t *buf;
        int s = 0;
        if (g.use_tma) {
            s = int(it % NST);
            const bool got = mbar_wait_bounded(&full[s], uint32_t((it / NST) & 1), g.timeout_ns);
            if (!__all_sync(0xffffffffu, got)) break;  // the warp leaves together (it shuffles below)
            buf = smem + s * TILE_BYTES;
        } else {
            buf = smem;
            named_sync(1, PNC);  // the previous tile's copy-out has read the buffer
            plain_tile_in<PNC>(g, cw.c, buf, tid);
            named_sync(1, PNC);
        }
        uint64_t acc = 0;
        pars_tile<N, D, COEF, RECON, PNC, PARS_B>(P, g, buf, cw.c, tid, acc);
        acc = warp_sum_u64(acc);
        if (g.use_tma) {
            // warp errors -> red[s][warp]; the producer adds the four and writes the tile's
            if ((tid & 31) == 0) red[s * (PNC / 32) + (tid >> 5)] = acc;
            if (RECON) fence_proxy_async_smem();
            __syncwarp();
            if ((tid & 31) == 0) mbar_arrive(&empty[s]);
        } else {
            if ((tid & 31) == 0) red[tid >> 5] = acc;
            named_sync(1, PNC);
            if (tid == 0) g.sse_acc[tile] = pars_red_sum<PNC>(red);
            if (RECON) plain_tile_out<PNC>(g, cw.c, buf, tid);
        }
    }
}

// Per image (one CTA each): the exact integer sum of its tiles' errors, then
// SSE = sum / m^2 (exact quotient rounded once) and PSNR.
static __global__ void pars_finalize(const unsigned long long *tiles, int64_t tiles_per_img, int nimg, int H, int W,
                                     double m2, double *sse, float *psnr) {
    __shared__ unsigned long long red[256 / 32];
    const int img = blockIdx.x;
    if (img >= nimg) return;
    unsigned long long acc = 0;
    for (int64_t t = threadIdx.x; t < tiles_per_img; t += blockDim.x) acc += tiles[int64_t(img) * tiles_per_img + t];
    acc = warp_sum_u64(acc);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x != 0) return;
    unsigned long long tot = 0;
    for (int w = 0; w < int(blockDim.x) / 32; w++) tot += red[w];
    const double s = double(tot) / m2;
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

template <int N>
using PKernel = void (*)(PlanK<N>, CUtensorMap, CUtensorMap, FusedGeom);

template <int N, int D>
PKernel<N> pars_pick_out(int out) {
    switch (out) {
        case 0: return pars_kernel<N, D, 0>;
        case 1: return pars_kernel<N, D, 1>;
        case 2: return pars_kernel<N, D, 2>;
        default: return pars_kernel<N, D, 3>;
    }
}

// Kernel for diagonal bound D in [D0, D1] and output set `out`, or null.  The
// N = 8 kernels are split over two translation units by D so that they compile
// in parallel.
template <int N, int D0, int D1>
const void *pars_pick_range(int D, int out) {
    if constexpr (D0 > D1) {
        return nullptr;
    } else {
        if (D == D0) return reinterpret_cast<const void *>(pars_pick_out<N, D0>(out));
        return pars_pick_range<N, D0 + 1, D1>(D, out);
    }
}
using PickFn = const void *(*)(int D, int out);

// Whether launch_pars serves this call: a rounded plan with T T^T diagonal and a
// Parseval form, N = 4 (any r) or N = 8 with r <= 15, no quantiser.
template <int N>
bool pars_applies(const Plan &plan, const FusedArgs &a) {
    if (N > 8 || plan.kind != 0 || a.Q) return false;
    if (plan.kparams<N>().pm2 == 0) return false;
    return N == 4 || diag_bound(N, a.r) <= PARS_DMAX8;
}

// Host launcher (arguments validated by the C ABI layer; pars_applies checked).
template <int N>
rklt_status launch_pars(const Plan &plan, const FusedArgs &a, cudaStream_t st, PickFn pick) {
    const PlanK<N> &pk = plan.kparams<N>();
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
    const uintptr_t za = reinterpret_cast<uintptr_t>(a.zcoef);
    g.coef_vec4 = (a.r % 4 == 0 && (za & 15) == 0) ? 4 : ((a.r % 2 == 0 && (za & 7) == 0) ? 2 : 1);
    g.timeout_ns = wait_timeout_ns();
    g.inject_stall = inject_stall();

    // scratch: one u64 error per tile (each written once by the kernel)
    const int64_t tiles_per_img = int64_t(g.tiles_x) * g.tiles_y;
    const size_t acc_bytes = size_t(std::max<int64_t>(g.ntiles, 1)) * sizeof(unsigned long long);
    void *scratch = nullptr;
    if (a.partials) {
        if (int64_t(acc_bytes) > a.scratch_cap) return fail(RKLT_ERR_ARG, "scratch array too small for this call");
        g.sse_acc = reinterpret_cast<unsigned long long *>(a.partials);
    } else {
        cudaMemPool_t pool = scratch_pool();
        if (!pool) return fail(RKLT_ERR_CUDA, "could not create the scratch memory pool");
        if (cudaMallocFromPoolAsync(&scratch, acc_bytes, pool, st) != cudaSuccess)
            return fail(RKLT_ERR_OOM, "scratch allocation failed");
        g.sse_acc = static_cast<unsigned long long *>(scratch);
    }
    cudaError_t e = cudaSuccess;

    const bool empty = a.H == 0 || a.W == 0;
    if (!empty) {
        const auto is16 = [](const void *p, int64_t x, int64_t y) {
            return ((reinterpret_cast<uintptr_t>(p) | uintptr_t(x) | uintptr_t(y)) & 15) == 0;
        };
        bool tma = !a.force_plain && is16(a.img, a.ld, g.img_stride) &&
                   (!a.recon || is16(a.recon, a.ld_recon, g.recon_stride));
        CUtensorMap tin{}, tout{};
        if (tma) {
            tma = make_map_u8(&tin, a.img, a.W, a.H, a.nimg, a.ld, g.img_stride, TW, TH);
            if (tma && a.recon) tma = make_map_u8(&tout, a.recon, a.W, a.H, a.nimg, a.ld_recon, g.recon_stride, TW, TH);
            if (tma && !a.recon) tout = tin;
        }
        g.use_tma = tma ? 1 : 0;
        const int out = (a.zcoef && a.r > 0 ? 1 : 0) | (a.recon ? 2 : 0);
        // ring depth: with outputs, four tiles; error only (1 B/px, no store-back),
        // a shallower ring leaves room for more CTAs per SM, which measured faster
        // (N = 4: 0.0707 -> 0.0653 ms with two stages; N = 8: 0.0653 -> 0.0637 with three)
        g.stages = out != 0 ? 4 : (N == 4 ? 2 : 3);
        const int nthreads = PARS_NC + 32;
        const void *fn = pick(g.D, out);
        if (!fn) {
            if (scratch) cudaFreeAsync(scratch, st);
            return fail(RKLT_ERR_UNSUPPORTED, "register path: no kernel for this diagonal bound");
        }
        const int smem = (tma ? g.stages : 1) * TILE_BYTES + 2 * STAGES * 8 + STAGES * (PARS_NC / 32) * 8 + 1024;
        const int dev = ensure_smem_attr(fn);
        int per_sm = occupancy(fn, nthreads, smem);
        if (per_sm < 1) per_sm = 1;
        const int64_t grid = std::min<int64_t>(g.ntiles, int64_t(per_sm) * sm_count(dev));
        const int64_t per_img = int64_t(g.tiles_x) * g.tiles_y;
        g.step_img = int(grid / per_img);
        const int rem = int(grid - int64_t(g.step_img) * per_img);
        g.step_ty = rem / g.tiles_x;
        g.step_tx = rem - g.step_ty * g.tiles_x;
        void *args[] = {const_cast<PlanK<N> *>(&pk), &tin, &tout, &g};
        e = cudaLaunchKernel(fn, dim3(unsigned(grid)), dim3(nthreads), args, smem, st);
        if (e != cudaSuccess) {
            if (scratch) cudaFreeAsync(scratch, st);
            return cuda_fail(e, "register-path kernel launch");
        }
    }
    pars_finalize<<<a.nimg, 256, 0, st>>>(g.sse_acc, empty ? 0 : tiles_per_img, a.nimg, a.H, a.W, double(pk.pm2),
                                          a.sse, a.psnr);
    e = cudaGetLastError();
    if (scratch) cudaFreeAsync(scratch, st);
    return e == cudaSuccess ? RKLT_OK : cuda_fail(e, "register-path finalize launch");
}

}  // namespace rklt
