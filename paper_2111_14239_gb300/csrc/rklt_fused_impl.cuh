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
// and pitches are 16-byte aligned a producer warp streams tiles into a 4-stage
// shared-memory ring with 3-D TMA bulk tensor copies (mbarrier completion), the
// eight consumer warps transform them in place, and the producer writes the
// rounded 8-bit reconstruction back with TMA bulk tensor stores.  Otherwise the
// consumers copy each tile in and out with plain vector loads.  Both modes run the
// same per-block code in the same order, so their results are identical.
//
// Work split inside a tile:
//   register path  (N = 4, and N = 8 with D <= 5): one thread owns a whole block;
//   cooperative path (N = 16, 32, and N = 8 with D > 5): per block-row of the
//     tile, threads own columns for the column passes and (block, row) pairs for
//     the row passes, exchanging through a padded shared-memory buffer.
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
constexpr int STAGES = 4;        // TMA ring depth
constexpr int NCONS = 256;       // consumer threads (8 warps); one producer warp follows
constexpr int LDY = TW + 1;      // padded row stride of the cooperative exchange buffer (floats)
static_assert(TW == kTileW && TH == kTileH, "tile geometry is declared in rklt_internal.h");
constexpr int REG_DMAX8 = 5;     // N = 8: register path up to this diagonal bound
constexpr uint64_t DRAIN_NS = 2000000000ull;  // limit on waits for copies already in flight

// ---------------------------------------------------------------------------
// Register path: one N x N block per thread.  D is a compile-time constant.
// ---------------------------------------------------------------------------
template <int N, int D>
__device__ __forceinline__ float block_reg(const PlanK<N> &P, uint8_t *blk, int r, float *coef, bool vec4,
                                           bool recon) {
    constexpr int H2 = N / 2;
    constexpr int W32 = N / 4;          // 32-bit words per block row
    constexpr int DR = D < N ? D : N;   // rows / columns of C that carry retained terms
    constexpr int DA = DR > 0 ? DR : 1; // array extent (D = 0 keeps nothing)
    uint32_t raw[N][W32];
#pragma unroll
    for (int k = 0; k < N; k++) {
        if constexpr (N == 8) {
            const uint2 w = *reinterpret_cast<const uint2 *>(blk + k * TW);
            raw[k][0] = w.x;
            raw[k][1] = w.y;
        } else {
            raw[k][0] = *reinterpret_cast<const uint32_t *>(blk + k * TW);
        }
    }
    // column transform: Y = T A, rows i < DR
    float Y[DA][N];
#pragma unroll
    for (int c = 0; c < N; c++) {
        float s[H2], d[H2];
#pragma unroll
        for (int j = 0; j < H2; j++) {
            const float top = byte_f(raw[j][c >> 2], c & 3), bot = byte_f(raw[N - 1 - j][c >> 2], c & 3);
            s[j] = top + bot;
            d[j] = top - bot;
        }
#pragma unroll
        for (int i = 0; i < DR; i++) {
            float acc = 0.0f;
#pragma unroll
            for (int j = 0; j < H2; j++) acc = fmaf(P.T[i][j], (i & 1) ? d[j] : s[j], acc);
            Y[i][c] = acc;
        }
    }
    // row transform: C = Y T^T on the support i + j < D; zonal mask on the last diagonal
    float Cm[DA][DA];
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
                if (i + j == D - 1) acc = (zz_index(N, i, j) < r) ? acc : 0.0f;
                Cm[i][j] = acc;
            }
        }
    }
    // normalised coefficients B = s_i s_j C in zig-zag order, first r
    if (coef) {
        if (vec4) {
#pragma unroll
            for (int k4 = 0; k4 < (N * N) / 4; k4++) {
                if (zz_row(N, 4 * k4) + zz_col(N, 4 * k4) < D && 4 * k4 < r) {
                    float v[4];
#pragma unroll
                    for (int q = 0; q < 4; q++) {
                        const int k = 4 * k4 + q, i = zz_row(N, k), j = zz_col(N, k);
                        v[q] = (i + j < D) ? P.sij[i][j] * Cm[i < DA ? i : 0][j < DA ? j : 0] : 0.0f;
                    }
                    *reinterpret_cast<float4 *>(coef + 4 * k4) = make_float4(v[0], v[1], v[2], v[3]);
                }
            }
        } else {
#pragma unroll
            for (int k = 0; k < N * N; k++) {
                const int i = zz_row(N, k), j = zz_col(N, k);
                if (i + j < D && k < r) coef[k] = P.sij[i][j] * Cm[i < DA ? i : 0][j < DA ? j : 0];
            }
        }
    }
    // inverse row transform: X[i][l] = sum_j C[i][j] T^{-1}[l][j]  (i < DR)
    float X[DA][N];
#pragma unroll
    for (int i = 0; i < DR; i++) {
#pragma unroll
        for (int l = 0; l < H2; l++) {
            float e = 0.0f, o = 0.0f;
#pragma unroll
            for (int j = 0; j < DR; j++) {
                if (i + j < D) {
                    if (j & 1) o = fmaf(Cm[i][j], P.Ti[l][j], o);
                    else e = fmaf(Cm[i][j], P.Ti[l][j], e);
                }
            }
            X[i][l] = e + o;
            X[i][N - 1 - l] = e - o;
        }
    }
    // inverse column transform A'[k][c] = sum_i T^{-1}[k][i] X[i][c], one mirrored row
    // pair (k, N-1-k) at a time; error; 8-bit output
    float sse = 0.0f;
#pragma unroll
    for (int k = 0; k < H2; k++) {
        uint32_t ot[W32], ob[W32];
#pragma unroll
        for (int w = 0; w < W32; w++) ot[w] = ob[w] = 0u;
#pragma unroll
        for (int c = 0; c < N; c++) {
            float e = 0.0f, o = 0.0f;
#pragma unroll
            for (int i = 0; i < DR; i++) {
                if (i & 1) o = fmaf(P.Ti[k][i], X[i][c], o);
                else e = fmaf(P.Ti[k][i], X[i][c], e);
            }
            const float top = e + o, bot = e - o;
            const float et = byte_f(raw[k][c >> 2], c & 3) - top;
            const float eb = byte_f(raw[N - 1 - k][c >> 2], c & 3) - bot;
            sse = fmaf(et, et, sse);
            sse = fmaf(eb, eb, sse);
            if (recon) {
                ot[c >> 2] |= recon_byte(top) << (8 * (c & 3));
                ob[c >> 2] |= recon_byte(bot) << (8 * (c & 3));
            }
        }
        if (recon) {
            if constexpr (N == 8) {
                *reinterpret_cast<uint2 *>(blk + k * TW) = make_uint2(ot[0], ot[1]);
                *reinterpret_cast<uint2 *>(blk + (N - 1 - k) * TW) = make_uint2(ob[0], ob[1]);
            } else {
                *reinterpret_cast<uint32_t *>(blk + k * TW) = ot[0];
                *reinterpret_cast<uint32_t *>(blk + (N - 1 - k) * TW) = ob[0];
            }
        }
    }
    return sse;
}

template <int N>
__device__ __forceinline__ float block_reg_dispatch(const PlanK<N> &P, uint8_t *blk, int D, int r, float *coef,
                                                    bool vec4, bool recon) {
    if constexpr (N == 4) {
        switch (D) {
            case 0: return block_reg<4, 0>(P, blk, r, coef, vec4, recon);
            case 1: return block_reg<4, 1>(P, blk, r, coef, vec4, recon);
            case 2: return block_reg<4, 2>(P, blk, r, coef, vec4, recon);
            case 3: return block_reg<4, 3>(P, blk, r, coef, vec4, recon);
            case 4: return block_reg<4, 4>(P, blk, r, coef, vec4, recon);
            case 5: return block_reg<4, 5>(P, blk, r, coef, vec4, recon);
            case 6: return block_reg<4, 6>(P, blk, r, coef, vec4, recon);
            default: return block_reg<4, 7>(P, blk, r, coef, vec4, recon);
        }
    } else {
        switch (D) {
            case 0: return block_reg<N, 0>(P, blk, r, coef, vec4, recon);
            case 1: return block_reg<N, 1>(P, blk, r, coef, vec4, recon);
            case 2: return block_reg<N, 2>(P, blk, r, coef, vec4, recon);
            case 3: return block_reg<N, 3>(P, blk, r, coef, vec4, recon);
            case 4: return block_reg<N, 4>(P, blk, r, coef, vec4, recon);
            default: return block_reg<N, 5>(P, blk, r, coef, vec4, recon);
        }
    }
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

template <int N>
__device__ __forceinline__ float tile_reg(const PlanK<N> &P, const FusedGeom &g, uint8_t *tile, int64_t tile_id,
                                          int ct) {
    constexpr int BPR = TW / N, BPT = (TH / N) * BPR;
    const TileCoord tc = tile_coord(g, tile_id);
    const int bw = g.W / N;
    float sse = 0.0f;
#pragma unroll 1
    for (int q = ct; q < BPT; q += NCONS) {
        const int by = q / BPR, bx = q - (q / BPR) * BPR;
        const int gy = tc.ty * (TH / N) + by, gx = tc.tx * BPR + bx;
        if (gy * N >= g.H || gx * N >= g.W) continue;
        float *coef = nullptr;
        if (g.zcoef) coef = g.zcoef + (int64_t(tc.img) * g.blocks_per_img + int64_t(gy) * bw + gx) * g.r;
        sse += block_reg_dispatch<N>(P, tile + by * N * TW + bx * N, g.D, g.r, coef, g.coef_vec4 != 0,
                                     g.recon != nullptr);
    }
    return sse;
}

// ---------------------------------------------------------------------------
// Cooperative path: per block-row of the tile (N rows x 256 columns = 256/N
// blocks), column passes by thread-per-column, row passes by thread-per-(block,
// row), exchange through Ys (row stride LDY, conflict-free for both access
// patterns).  Coefficients are staged in Zs in zig-zag order and written out
// contiguously.  D and r are runtime values.
// ---------------------------------------------------------------------------
template <int N>
__device__ __forceinline__ float tile_coop(const PlanK<N> &P, const FusedGeom &g, uint8_t *tile, int64_t tile_id,
                                           int ct, float *Ys, float *Zs) {
    constexpr int H2 = N / 2;
    constexpr int BPR = TW / N;
    const TileCoord tc = tile_coord(g, tile_id);
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
                        const float c = (z < r) ? acc : 0.0f;
                        if (z < r) Zs[b * r + z] = (si * P.s[j]) * c;
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

template <int N>
__device__ __forceinline__ float process_tile(const PlanK<N> &P, const FusedGeom &g, uint8_t *tile, int64_t tile_id,
                                              int ct, float *Ys, float *Zs) {
    if constexpr (N == 4) {
        return tile_reg<4>(P, g, tile, tile_id, ct);
    } else if constexpr (N == 8) {
        if (g.D <= REG_DMAX8) return tile_reg<8>(P, g, tile, tile_id, ct);
        return tile_coop<8>(P, g, tile, tile_id, ct, Ys, Zs);
    } else {
        return tile_coop<N>(P, g, tile, tile_id, ct, Ys, Zs);
    }
}

// Fixed-order reduction over the consumer threads; thread 0 returns the sum.
__device__ __forceinline__ float reduce_consumers(float v, float *red, int ct) {
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
    if ((ct & 31) == 0) red[ct >> 5] = v;
    named_sync(2, NCONS);
    float t = 0.0f;
    if (ct == 0) {
#pragma unroll
        for (int w = 0; w < NCONS / 32; w++) t += red[w];
    }
    named_sync(2, NCONS);
    return t;
}

__device__ __forceinline__ void tile_origin(const FusedGeom &g, int64_t tile_id, int &x, int &y, int &z) {
    const TileCoord t = tile_coord(g, tile_id);
    z = t.img;
    y = t.ty * TH;
    x = t.tx * TW;
}

// Shared memory after 1 KB alignment: tile ring | barriers | reduction | Ys | Zs.
struct SmemLayout {
    int bar_off, red_off, ys_off, zs_off, total;
};

template <int N>
__host__ __device__ inline SmemLayout smem_layout(int stages, int r, int D) {
    SmemLayout L{};
    L.bar_off = stages * TILE_BYTES;
    L.red_off = L.bar_off + 2 * STAGES * 8;
    L.ys_off = L.red_off + 64;
    const bool coop = (N >= 16) || (N == 8 && D > REG_DMAX8);
    const int ys = coop ? N * LDY * 4 : 0;
    L.zs_off = L.ys_off + ((ys + 15) / 16) * 16;
    const int zs = coop ? (TW / N) * r * 4 : 0;
    L.total = L.zs_off + zs + 1024;  // + slack for aligning the dynamic base
    return L;
}

// ---------------------------------------------------------------------------
// The kernel: warps 0..7 consume; warp 8 produces in TMA mode (idle otherwise).
// ---------------------------------------------------------------------------
template <int N>
__global__ void __launch_bounds__(NCONS + 32, 2)
    fused_kernel(const __grid_constant__ PlanK<N> P, const __grid_constant__ CUtensorMap tm_in,
                 const __grid_constant__ CUtensorMap tm_out, const FusedGeom g) {
    extern __shared__ uint8_t smem_raw[];
    uint8_t *smem = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    const SmemLayout L = smem_layout<N>(g.use_tma ? STAGES : 1, g.r, g.D);
    uint64_t *full = reinterpret_cast<uint64_t *>(smem + L.bar_off);
    uint64_t *empty = full + STAGES;
    float *red = reinterpret_cast<float *>(smem + L.red_off);
    float *Ys = reinterpret_cast<float *>(smem + L.ys_off);
    float *Zs = reinterpret_cast<float *>(smem + L.zs_off);
    const int tid = threadIdx.x;

    if (g.use_tma && tid == NCONS) {
        for (int s = 0; s < STAGES; s++) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], NCONS / 32);
        }
        fence_mbar_init();
    }
    __syncthreads();

    if (tid >= NCONS) {
        // ---------------- producer: one elected lane of warp 8 ----------------
        if (!g.use_tma || tid != NCONS) return;
        int64_t it = 0;
        bool ok = true;
        for (int64_t tile = blockIdx.x; tile < g.ntiles; tile += gridDim.x, ++it) {
            const int s = int(it % STAGES);
            if (it >= STAGES) {
                // slot s last held tile (it - STAGES): wait for its release, write it back
                if (!mbar_wait_bounded(&empty[s], uint32_t(((it / STAGES) - 1) & 1), g.timeout_ns)) {
                    ok = false;
                    break;
                }
                if (g.recon) {
                    int x, y, z;
                    tile_origin(g, tile - int64_t(STAGES) * gridDim.x, x, y, z);
                    tma_store_3d(&tm_out, x, y, z, smem + s * TILE_BYTES);
                    bulk_commit();
                    bulk_wait_read_all();  // the store has read the slot before it is refilled
                }
            }
            if (g.inject_stall) continue;  // test hook: nothing ever completes full[s]
            int x, y, z;
            tile_origin(g, tile, x, y, z);
            mbar_arrive_expect_tx(&full[s], TILE_BYTES);
            tma_load_3d(smem + s * TILE_BYTES, &tm_in, x, y, z, &full[s]);
        }
        // drain: write back the slots still holding consumed tiles
        const int64_t issued = it;
        for (int64_t j = issued > STAGES ? issued - STAGES : 0; j < issued; j++) {
            const int s = int(j % STAGES);
            const uint32_t par = uint32_t((j / STAGES) & 1);
            if (!ok || !mbar_wait_bounded(&empty[s], par, g.timeout_ns)) {
                // the consumers gave up: let this slot's load land before the CTA exits
                ok = false;
                if (!g.inject_stall) mbar_wait_bounded(&full[s], par, DRAIN_NS);
                continue;
            }
            if (g.recon) {
                int x, y, z;
                tile_origin(g, int64_t(blockIdx.x) + j * gridDim.x, x, y, z);
                tma_store_3d(&tm_out, x, y, z, smem + s * TILE_BYTES);
                bulk_commit();
            }
        }
        bulk_wait_all();
        return;
    }

    // ---------------- consumers ----------------
    const bool al8 = ((reinterpret_cast<uintptr_t>(g.img) | uintptr_t(g.ld) | uintptr_t(g.img_stride)) & 7) == 0;
    const bool al8o =
        ((reinterpret_cast<uintptr_t>(g.recon) | uintptr_t(g.ld_recon) | uintptr_t(g.recon_stride)) & 7) == 0;
    int64_t it = 0;
    for (int64_t tile = blockIdx.x; tile < g.ntiles; tile += gridDim.x, ++it) {
        uint8_t *buf;
        int s = 0;
        int x0 = 0, y0 = 0, z = 0, hv = 0, wv = 0;
        if (g.use_tma) {
            s = int(it % STAGES);
            const bool got = mbar_wait_bounded(&full[s], uint32_t((it / STAGES) & 1), g.timeout_ns);
            // all consumers leave together if any of them gave up (they share named barriers)
            if (named_any(3, NCONS, !got)) break;
            buf = smem + s * TILE_BYTES;
        } else {
            buf = smem;
            tile_origin(g, tile, x0, y0, z);
            hv = min(TH, g.H - y0);
            wv = min(TW, g.W - x0);
            const uint8_t *src = g.img + int64_t(z) * g.img_stride + int64_t(y0) * g.ld + x0;
            named_sync(1, NCONS);  // the previous tile's copy-out has read the buffer
            if (al8) {
                for (int q = tid; q < TH * (TW / 8); q += NCONS) {
                    const int y = q / (TW / 8), x = (q - y * (TW / 8)) * 8;
                    uint2 v = make_uint2(0u, 0u);
                    if (y < hv && x + 8 <= wv) {
                        v = *reinterpret_cast<const uint2 *>(src + int64_t(y) * g.ld + x);
                    } else if (y < hv && x < wv) {  // ragged edge: only bytes inside the image
                        uint32_t b[8] = {0u, 0u, 0u, 0u, 0u, 0u, 0u, 0u};
                        for (int e = 0; e < wv - x; e++) b[e] = src[int64_t(y) * g.ld + x + e];
                        v.x = b[0] | (b[1] << 8) | (b[2] << 16) | (b[3] << 24);
                        v.y = b[4] | (b[5] << 8) | (b[6] << 16) | (b[7] << 24);
                    }
                    *reinterpret_cast<uint2 *>(buf + y * TW + x) = v;
                }
            } else {
                for (int q = tid; q < TILE_BYTES; q += NCONS) {
                    const int y = q / TW, x = q - y * TW;
                    buf[q] = (y < hv && x < wv) ? src[int64_t(y) * g.ld + x] : uint8_t(0);
                }
            }
            named_sync(1, NCONS);
        }
        const float v = process_tile<N>(P, g, buf, tile, tid, Ys, Zs);
        if (g.use_tma) {
            if (g.recon) fence_proxy_async_smem();
            __syncwarp();
            if ((tid & 31) == 0) mbar_arrive(&empty[s]);
        }
        const float t = reduce_consumers(v, red, tid);
        if (tid == 0) g.partials[tile] = t;
        if (!g.use_tma && g.recon) {
            named_sync(1, NCONS);
            uint8_t *dst = g.recon + int64_t(z) * g.recon_stride + int64_t(y0) * g.ld_recon + x0;
            if (al8o) {
                for (int q = tid; q < TH * (TW / 8); q += NCONS) {
                    const int y = q / (TW / 8), x = (q - y * (TW / 8)) * 8;
                    if (y < hv && x + 8 <= wv) {
                        *reinterpret_cast<uint2 *>(dst + int64_t(y) * g.ld_recon + x) =
                            *reinterpret_cast<const uint2 *>(buf + y * TW + x);
                    } else if (y < hv && x < wv) {
                        for (int e = 0; e < wv - x; e++) dst[int64_t(y) * g.ld_recon + x + e] = buf[y * TW + x + e];
                    }
                }
            } else {
                for (int q = tid; q < TILE_BYTES; q += NCONS) {
                    const int y = q / TW, x = q - y * TW;
                    if (y < hv && x < wv) dst[int64_t(y) * g.ld_recon + x] = buf[q];
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
    CUtensorMap tin{}, tout{};
    if (tma) {
        tma = make_map_u8(&tin, a.img, a.W, a.H, a.nimg, a.ld, g.img_stride, TW, TH);
        if (tma && a.recon) tma = make_map_u8(&tout, a.recon, a.W, a.H, a.nimg, a.ld_recon, g.recon_stride, TW, TH);
        if (tma && !a.recon) tout = tin;
    }
    g.use_tma = tma ? 1 : 0;
    const SmemLayout L = smem_layout<N>(tma ? STAGES : 1, a.r, g.D);
    const int dev = ensure_smem_attr(reinterpret_cast<const void *>(fused_kernel<N>));
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fused_kernel<N>, NCONS + 32, L.total);
    if (per_sm < 1) per_sm = 1;
    const int64_t grid = std::min<int64_t>(g.ntiles, int64_t(per_sm) * sm_count(dev));
    fused_kernel<N><<<unsigned(grid), NCONS + 32, L.total, st>>>(plan.kparams<N>(), tin, tout, g);
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
