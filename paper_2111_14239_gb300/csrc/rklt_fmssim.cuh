// rklt_fmssim.cuh -- the fused pass with the structural similarity: forward,
// zonal retention, inverse and error of every N x N block (Sec. 4.1, Appendix) and,
// in the same launch, the mean SSIM of the original against its 8-bit
// reconstruction (Sec. 4.1's second quality measure; Wang et al. 2004: 11 x 11
// Gaussian window, sigma 1.5, C1 = (0.01 * 255)^2, C2 = (0.03 * 255)^2, mean over the
// (H - 10) x (W - 10) positions where the window fits).  Included by
// rklt_fmssim_n4.cu and rklt_fmssim_n8.cu; N = 4 or 8, plans of the register path
// (T T^T diagonal, Parseval error).
//
// A CTA takes a unit: 256 columns of one image (a strip) x one segment of rows, and
// walks down it 88 rows at a time (88 = 8 x 11: whole blocks and whole 11-row
// window chunks):
//   load       the 88 rows of the original, 256 + 16 columns (TMA boxes into a
//              256-wide and a 16-wide part; rows or columns outside the image read
//              as 0), or plain loads when the pointers are not 16-byte aligned;
//   transform  every block of the 88 x 272 window into a shared-memory copy of the
//              reconstruction, two blocks per thread (the register path's block
//              code); the unit's own blocks (the first 256 columns) also write their
//              coefficients and add their error; the 16 columns on the right are
//              the next strip's blocks, transformed again here for the window halo;
//   store      the unit's reconstruction rows (one TMA store of the 256-wide part);
//   SSIM       eight chunks of 11 rows: horizontal 11-tap sums of x, y, x^2 + y^2
//              and x y straight from the two byte copies (eight outputs per task),
//              then one thread per output column adds the chunk's rows into 11
//              rolling vertical accumulators and finishes one output row per input
//              row, exactly as the standalone MSSIM pass does.
// A segment other than the first starts with a lead: the last block rows above it
// (16 rows for N = 8, 12 for N = 4) are transformed again (nothing stored) and their
// last 11 rows fill the accumulators, so that every window position has one owner:
// a unit owns the positions whose window ends in its rows (first segment: from row
// 0) and its columns.  During a transform the 44 accumulators per thread wait in
// the horizontal-sum buffer, which is idle then.
//
// Numerics: the blocks are those of the register path, so the coefficients, the
// reconstruction and the exact integer error are bit for bit the fused call's.  The
// SSIM of each window position is computed with the same operations in the same
// order as the standalone pass (bit-identical per position); only the grouping of
// the per-position values into FP32 chunk sums differs, so the mean agrees with the
// standalone pass on the same reconstruction to about 1e-7.
#pragma once

#include <algorithm>
#include <cmath>

#include "rklt_reg.cuh"

namespace rklt {

constexpr int FM_T = 256;         // threads per CTA (8 warps)
constexpr int FM_SC = 88;         // rows per step: 8 window chunks of 11
constexpr int FM_S = 11;          // window side
constexpr int FM_R = 5;           // window radius
constexpr int FM_WS = 256;        // output columns of a strip (one per thread)
constexpr int FM_HW = 16;         // halo columns
constexpr int FM_G = 8;           // horizontal outputs per task
constexpr int FM_B = 2;           // blocks per thread per transform step
constexpr int FM_HS_BYTES = FM_S * FM_WS * 16;
constexpr int FM_MAIN_BYTES = FM_SC * FM_WS, FM_HALO_BYTES = FM_SC * FM_HW;
// shared memory: original (main, halo), reconstruction (main, halo), horizontal
// sums (float4 per position), CTA reduction slots, one mbarrier
constexpr int FM_OFF_OM = 0;
constexpr int FM_OFF_OH = FM_OFF_OM + FM_MAIN_BYTES;
constexpr int FM_OFF_RM = FM_OFF_OH + FM_HALO_BYTES;
constexpr int FM_OFF_RH = FM_OFF_RM + FM_MAIN_BYTES;
constexpr int FM_OFF_HS = FM_OFF_RH + FM_HALO_BYTES;
constexpr int FM_OFF_RED = FM_OFF_HS + FM_HS_BYTES;
constexpr int FM_OFF_BAR = FM_OFF_RED + (FM_T / 32) * 16;
constexpr int FM_SMEM = FM_OFF_BAR + 16 + 1024;   // + alignment slack
static_assert(FM_OFF_OH % 128 == 0 && FM_OFF_RM % 128 == 0 && FM_OFF_RH % 128 == 0, "TMA destinations");
static_assert(FM_S * 4 * FM_T * 4 <= FM_HS_BYTES, "the accumulators fit the horizontal-sum buffer");
constexpr uint64_t FM_DRAIN_NS = 2000000000ull;

// rows of the lead: whole blocks covering at least the 11 rows above a segment
__host__ __device__ constexpr int fm_lead_rows(int N) { return N * ((FM_S + N - 1) / N); }

// The Gaussian's weights are symmetric (g[t] = g[10 - t] exactly: the same exponent
// and divisor on the host), so six register pairs hold all eleven taps.
__host__ __device__ constexpr int fm_tap(int t) { return t <= FM_R ? t : FM_S - 1 - t; }

// float4 column c of a horizontal-sum row sits at c with its low 3 bits XOR (c / 8)
// mod 8: lanes writing columns 8 apart and lanes reading consecutive columns both
// hit distinct bank groups
__device__ __forceinline__ int fm_phys(int c) { return (c & ~7) | ((c ^ (c >> 3)) & 7); }

struct FmGeom {
    const uint8_t *img;
    uint8_t *recon;                 // null: the reconstruction stays on chip
    float *zcoef;                   // null: no coefficients
    int64_t ld, img_stride, ld_recon, recon_stride;
    unsigned long long *sse_part;   // one per unit: the owned blocks' error times m^2
    double *ms_part;                // one per unit: sum of the owned positions' SSIM
    int H, W, nimg, r, cvec;
    int strips, segs, seg_rows;     // seg_rows: a multiple of FM_SC
    int64_t nunits;
    int use_tma;
    uint64_t timeout_ns;
    float g[FM_S];                  // 1-D Gaussian, normalised; the window is g g^T
};

struct FmMaps {
    CUtensorMap in256, in16;        // original: boxes of 256 and 16 columns x 88 rows
    CUtensorMap lead256, lead16;    // original: the same x lead rows
    CUtensorMap out256;             // reconstruction: 256 columns x 88 rows
};

// One unit's place: image, strip, segment rows [R0, R1).
struct FmUnit {
    int img, c0, R0, R1;
    __device__ __forceinline__ void set(const FmGeom &g, int64_t u) {
        const int64_t per_img = int64_t(g.strips) * g.segs;
        img = int(u / per_img);
        const int rem = int(u - int64_t(img) * per_img);
        const int sy = rem / g.strips, sx = rem - sy * g.strips;
        c0 = sx * FM_WS;
        R0 = sy * g.seg_rows;
        R1 = min(R0 + g.seg_rows, g.H);
    }
    // steps of this unit: the lead (when R0 > 0), then one per 88 rows
    __device__ __forceinline__ int first_step() const { return R0 > 0 ? -1 : 0; }
    __device__ __forceinline__ int nsteps() const { return (R1 - R0 + FM_SC - 1) / FM_SC; }
};

// Blocks of nbr block rows of the window buffers, two per thread: main part
// (256 / N block columns, row pitch 256) and halo part (16 / N block columns, pitch
// 16).  Block row 0 of the buffers is block row gy0 of the image, main block column
// 0 is block column gx0.  own: the main blocks belong to this unit (not in the
// lead).  The reconstruction goes to the rec buffers; returns the owned blocks'
// error times m^2.
template <int N, int D, bool COEF>
__device__ __forceinline__ uint64_t fm_transform(const PlanK<N> &P, const FmGeom &g, const uint8_t *om,
                                                 const uint8_t *oh, uint8_t *rm, uint8_t *rh, int nbr, int gy0,
                                                 int gx0, bool own, float *zimg, int tid) {
    constexpr int B = FM_B;
    constexpr int BM = FM_WS / N, BH = FM_HW / N;
    const int pm = nbr * BM / B, ph = nbr * BH / B, pm32 = (pm + 31) & ~31;
    const int bh = g.H / N, bw = g.W / N;
    uint64_t err = 0;
#pragma unroll 1
    for (int p = tid; p < pm32 + ph; p += FM_T) {
        if (p < pm) {
            uint32_t w[B][N][N / 4];
            uint8_t *dst[B];
            float *coef[B];
            bool act[B];
#pragma unroll
            for (int b = 0; b < B; b++) {
                const int q = p + b * pm;
                const int by = q / BM, bx = q - by * BM;
                const int gy = gy0 + by, gx = gx0 + bx;
                act[b] = own && gy < bh && gx < bw;
                load_block_words<N>(om + by * N * FM_WS + bx * N, FM_WS, w[b]);
                dst[b] = rm + by * N * FM_WS + bx * N;
                coef[b] = COEF ? zimg + (int64_t(gy) * bw + gx) * g.r : nullptr;
            }
            err += pars_blocks<N, D, COEF, true, B, FM_WS>(P, w, dst, g.r, coef, act, g.cvec);
        } else if (p >= pm32) {
            uint32_t w[B][N][N / 4];
            uint8_t *dst[B];
            float *coef[B];
            bool act[B];
#pragma unroll
            for (int b = 0; b < B; b++) {
                const int q = p - pm32 + b * ph;
                const int by = q / BH, bx = q - by * BH;
                load_block_words<N>(oh + by * N * FM_HW + bx * N, FM_HW, w[b]);
                dst[b] = rh + by * N * FM_HW + bx * N;
                coef[b] = nullptr;
                act[b] = false;
            }
            (void)pars_blocks<N, D, false, true, B, FM_HW>(P, w, dst, g.r, coef, act, g.cvec);
        }
    }
    return err;
}

// Plain loads of rows [y, y + rows) x columns [c0, c0 + 272) of image img into the
// window buffers (bytes outside the image read as 0).
__device__ __forceinline__ void fm_plain_in(const FmGeom &g, int img, int y, int rows, int c0, uint8_t *om,
                                            uint8_t *oh, int tid) {
    constexpr int G8 = (FM_WS + FM_HW) / 8;
    const uint8_t *src = g.img + int64_t(img) * g.img_stride;
    const bool al8 = ((reinterpret_cast<uintptr_t>(g.img) | uintptr_t(g.ld) | uintptr_t(g.img_stride)) & 7) == 0;
    for (int q = tid; q < rows * G8; q += FM_T) {
        const int rr = q / G8, k = q - rr * G8;
        const int yy = y + rr, x = c0 + 8 * k;
        uint2 v = make_uint2(0u, 0u);
        if (yy >= 0 && yy < g.H) {
            const uint8_t *s = src + int64_t(yy) * g.ld + x;
            if (al8 && x + 8 <= g.W) {
                v = *reinterpret_cast<const uint2 *>(s);
            } else {
                for (int e = 0; e < 8 && x + e < g.W; e++) {
                    const uint32_t b = s[e];
                    if (e < 4) v.x |= b << (8 * e);
                    else v.y |= b << (8 * (e - 4));
                }
            }
        }
        uint8_t *d = k < FM_WS / 8 ? om + rr * FM_WS + 8 * k : oh + rr * FM_HW + 8 * (k - FM_WS / 8);
        *reinterpret_cast<uint2 *>(d) = v;
    }
}

// Plain stores of the unit's reconstruction rows [y, y + rows), columns [c0, c0 + 256)
// inside the image.
__device__ __forceinline__ void fm_plain_out(const FmGeom &g, int img, int y, int rows, int c0, const uint8_t *rm,
                                             int tid) {
    uint8_t *dst = g.recon + int64_t(img) * g.recon_stride;
    const bool al8 =
        ((reinterpret_cast<uintptr_t>(g.recon) | uintptr_t(g.ld_recon) | uintptr_t(g.recon_stride)) & 7) == 0;
    for (int q = tid; q < rows * (FM_WS / 8); q += FM_T) {
        const int rr = q / (FM_WS / 8), x = c0 + 8 * (q - rr * (FM_WS / 8));
        if (x >= g.W) continue;
        const uint8_t *s = rm + rr * FM_WS + (x - c0);
        uint8_t *d = dst + int64_t(y + rr) * g.ld_recon + x;
        if (al8 && x + 8 <= g.W) {
            *reinterpret_cast<uint2 *>(d) = *reinterpret_cast<const uint2 *>(s);
        } else {
            for (int e = 0; e < 8 && x + e < g.W; e++) d[e] = s[e];
        }
    }
}

// Horizontal pass over buffer rows s0 .. s0 + 10: for each row and output column c,
// the 11-tap sums of (x, y) and (x^2 + y^2, x y), x and y centred at 128, in tap order
// (t = 0 a product, then fused multiply-adds), into hs.
__device__ __forceinline__ void fm_hpass(const uint8_t *om, const uint8_t *oh, const uint8_t *rm, const uint8_t *rh,
                                         float4 *hs, int s0, const float2 (&gw)[FM_R + 1], int tid) {
    constexpr int TPR = FM_WS / FM_G;   // tasks per row
#pragma unroll 1
    for (int q = tid; q < FM_S * TPR; q += FM_T) {
        const int rr = q / TPR, gc = (q - rr * TPR) * FM_G;
        const int row = s0 + rr;
        // words of columns gc .. gc + 19 (18 used) of both images; a word lies wholly
        // in the main or the halo part
        uint32_t xw[5], yw[5];
        const auto at = [&](const uint8_t *m, const uint8_t *h, int c) -> const uint8_t * {
            return c < FM_WS ? m + row * FM_WS + c : h + row * FM_HW + (c - FM_WS);
        };
#pragma unroll
        for (int h = 0; h < 2; h++) {
            const int c = gc + 8 * h;
            const uint2 a = *reinterpret_cast<const uint2 *>(at(om, oh, c));
            const uint2 b = *reinterpret_cast<const uint2 *>(at(rm, rh, c));
            xw[2 * h] = a.x;
            xw[2 * h + 1] = a.y;
            yw[2 * h] = b.x;
            yw[2 * h + 1] = b.y;
        }
        xw[4] = *reinterpret_cast<const uint32_t *>(at(om, oh, gc + 16));
        yw[4] = *reinterpret_cast<const uint32_t *>(at(rm, rh, gc + 16));
        float2 p[FM_G], s[FM_G];
#pragma unroll
        for (int k = 0; k < FM_G + FM_S - 1; k++) {
            // byte k under the exponent of 2^23 is the float 2^23 + byte (exact)
            const uint32_t sel = 0x7440u | uint32_t(k & 3);
            const float a = __uint_as_float(__byte_perm(xw[k >> 2], 0x4B000000u, sel)) - 8388736.0f;
            const float b = __uint_as_float(__byte_perm(yw[k >> 2], 0x4B000000u, sel)) - 8388736.0f;
            // products and sum of integers below 2^15: exact in any order
            const float2 vp = make_float2(a, b), vs = make_float2(fmaf(a, a, b * b), a * b);
#pragma unroll
            for (int o = 0; o < FM_G; o++) {
                const int t = k - o;
                if (t < 0 || t >= FM_S) continue;
                if (t == 0) {
                    p[o] = __fmul2_rn(gw[0], vp);
                    s[o] = __fmul2_rn(gw[0], vs);
                } else {
                    p[o] = __ffma2_rn(gw[fm_tap(t)], vp, p[o]);
                    s[o] = __ffma2_rn(gw[fm_tap(t)], vs, s[o]);
                }
            }
        }
        float4 *dst = hs + rr * FM_WS;
#pragma unroll
        for (int o = 0; o < FM_G; o++) dst[fm_phys(gc + o)] = make_float4(p[o].x, p[o].y, s[o].x, s[o].y);
    }
}

// ---------------------------------------------------------------------------
// The kernel: a persistent grid over the units; thread 0 issues the TMA copies.
// ---------------------------------------------------------------------------
template <int N, int D, bool COEF>
__global__ void __launch_bounds__(FM_T, 2)
    fm_kernel(const __grid_constant__ PlanK<N> P, const __grid_constant__ FmMaps maps,
              const __grid_constant__ FmGeom g) {
    constexpr int LEAD = fm_lead_rows(N);
    extern __shared__ uint8_t fm_smem_raw[];
    uint8_t *smem = fm_smem_raw + ((1024u - (smem_u32(fm_smem_raw) & 1023u)) & 1023u);
    uint8_t *om = smem + FM_OFF_OM, *oh = smem + FM_OFF_OH, *rm = smem + FM_OFF_RM, *rh = smem + FM_OFF_RH;
    float4 *hs = reinterpret_cast<float4 *>(smem + FM_OFF_HS);
    float *hsf = reinterpret_cast<float *>(smem + FM_OFF_HS);
    unsigned long long *red_u = reinterpret_cast<unsigned long long *>(smem + FM_OFF_RED);
    double *red_d = reinterpret_cast<double *>(red_u + FM_T / 32);
    uint64_t *bar = reinterpret_cast<uint64_t *>(smem + FM_OFF_BAR);
    const int tid = threadIdx.x;
    if (g.use_tma && tid == 0) {
        mbar_init(bar, 1);
        fence_mbar_init();
    }
    __syncthreads();

    const int OH = g.H - FM_S + 1, OW = g.W - FM_S + 1;
    const bool do_ssim = OH > 0 && OW > 0;
    const float C1 = (0.01f * 255.0f) * (0.01f * 255.0f), C2 = (0.03f * 255.0f) * (0.03f * 255.0f);
    float2 gw[FM_R + 1];   // taps 0..5 (the window is symmetric: tap t = tap 10 - t)
#pragma unroll
    for (int k = 0; k <= FM_R; k++) gw[k] = make_float2(g.g[k], g.g[k]);

    uint32_t consumed = 0, issued = 0;   // TMA loads waited for / issued (barrier phases)
    // issue the load of step k of unit u (thread 0)
    const auto issue = [&](int64_t u, int k) {
        FmUnit t;
        t.set(g, u);
        const bool box16 = t.c0 + FM_WS < g.W;
        const int rows = k < 0 ? LEAD : FM_SC;
        const int y = k < 0 ? t.R0 - LEAD : t.R0 + k * FM_SC;
        mbar_arrive_expect_tx(bar, uint32_t(rows * (FM_WS + (box16 ? FM_HW : 0))));
        tma_load_3d(om, k < 0 ? &maps.lead256 : &maps.in256, t.c0, y, t.img, bar);
        if (box16) tma_load_3d(oh, k < 0 ? &maps.lead16 : &maps.in16, t.c0 + FM_WS, y, t.img, bar);
        ++issued;
    };

    float2 ap[FM_S], as[FM_S];   // rolling vertical accumulators, slot = output row mod 11
#pragma unroll
    for (int k = 0; k < FM_S; k++) ap[k] = as[k] = make_float2(0.0f, 0.0f);
    uint64_t err = 0;
    double total = 0.0;

    int64_t u = blockIdx.x;
    FmUnit cu;
    if (u < g.nunits) {
        cu.set(g, u);
        if (g.use_tma && tid == 0) issue(u, cu.first_step());
    }
    int k = u < g.nunits ? cu.first_step() : 0;
    bool ok = true;
    while (u < g.nunits) {
        const int rows = k < 0 ? LEAD : FM_SC;
        const int y = k < 0 ? cu.R0 - LEAD : cu.R0 + k * FM_SC;
        // ---- the step's original rows
        if (g.use_tma) {
            if (tid == 0) bulk_wait_read_all();   // the last reconstruction store has read rm
            ok = mbar_wait_bounded(bar, consumed & 1u, g.timeout_ns);
            ++consumed;
        } else {
            fm_plain_in(g, cu.img, y, rows, cu.c0, om, oh, tid);
        }
        if (__syncthreads_or(!ok)) {
            ok = false;
            break;
        }
        // ---- transform (the accumulators wait in hs)
#pragma unroll
        for (int s = 0; s < FM_S; s++) {
            hsf[(4 * s + 0) * FM_T + tid] = ap[s].x;
            hsf[(4 * s + 1) * FM_T + tid] = ap[s].y;
            hsf[(4 * s + 2) * FM_T + tid] = as[s].x;
            hsf[(4 * s + 3) * FM_T + tid] = as[s].y;
        }
        float *zimg = COEF ? g.zcoef + int64_t(cu.img) * (g.H / N) * (g.W / N) * g.r : nullptr;
        err += fm_transform<N, D, COEF>(P, g, om, oh, rm, rh, rows / N, y / N, cu.c0 / N, k >= 0, zimg, tid);
        if (g.recon && g.use_tma) fence_proxy_async_smem();
        __syncthreads();
        if (g.recon && k >= 0) {
            if (g.use_tma) {
                if (tid == 0) {
                    tma_store_3d(&maps.out256, cu.c0, y, cu.img, rm);
                    bulk_commit();
                }
            } else {
                fm_plain_out(g, cu.img, y, min(FM_SC, cu.R1 - y), cu.c0, rm, tid);
            }
        }
#pragma unroll
        for (int s = 0; s < FM_S; s++) {
            ap[s] = make_float2(hsf[(4 * s + 0) * FM_T + tid], hsf[(4 * s + 1) * FM_T + tid]);
            as[s] = make_float2(hsf[(4 * s + 2) * FM_T + tid], hsf[(4 * s + 3) * FM_T + tid]);
        }
        __syncthreads();

        // ---- the next step (this unit's or the next unit's)
        int64_t nu = u;
        int nk = k + 1;
        if (nk >= cu.nsteps()) {
            nu = u + gridDim.x;
            nk = 0;
            if (nu < g.nunits) {
                FmUnit t;
                t.set(g, nu);
                nk = t.first_step();
            }
        }

        // ---- SSIM over the step's 11-row chunks: input rows j0 .. j0 + 10 at buffer
        // rows s0 ..; the unit owns output rows [lo, hi) and columns [c0, c0 + 256)
        const int nsub = !do_ssim ? 0 : (k < 0 ? 1 : min(FM_SC / FM_S, (cu.R1 - y + FM_S - 1) / FM_S));
        const int lo = max(cu.R0 - (FM_S - 1), 0), hi = min(cu.R1 - (FM_S - 1), OH);
        const bool col_ok = cu.c0 + tid < OW;
        for (int m = 0; m < nsub; m++) {
            const int s0 = k < 0 ? LEAD - FM_S : m * FM_S;
            const int j0 = k < 0 ? cu.R0 - FM_S : y + m * FM_S;
            if (m > 0) __syncthreads();   // the previous chunk's vertical pass has read hs
            fm_hpass(om, oh, rm, rh, hs, s0, gw, tid);
            __syncthreads();
            // the original is read: the next step's copy may land
            if (m == nsub - 1 && g.use_tma && tid == 0 && nu < g.nunits) issue(nu, nk);
            float csum = 0.0f;
            const float4 *col = hs + fm_phys(tid);
#pragma unroll
            for (int qq = 0; qq < FM_S; qq++) {
                const float4 v = col[qq * FM_WS];
                const float2 vp = make_float2(v.x, v.y), vs = make_float2(v.z, v.w);
#pragma unroll
                for (int d = 0; d < FM_S; d++) {
                    const int slot = (qq - d + FM_S) % FM_S;   // output row j - d
                    if (d == 0) {
                        ap[slot] = __fmul2_rn(gw[0], vp);
                        as[slot] = __fmul2_rn(gw[0], vs);
                    } else {
                        ap[slot] = __ffma2_rn(gw[fm_tap(d)], vp, ap[slot]);
                        as[slot] = __ffma2_rn(gw[fm_tap(d)], vs, as[slot]);
                    }
                }
                // output row o = j - 10 is complete (slot (qq + 1) mod 11)
                const int o = j0 + qq - (FM_S - 1);
                const int slot = (qq + 1) % FM_S;
                const bool valid = o >= lo && o < hi && col_ok;
                const float mx = ap[slot].x, my = ap[slot].y;
                const float vsum = __fsub_rn(as[slot].x, __fadd_rn(__fmul_rn(mx, mx), __fmul_rn(my, my)));
                const float cxy = __fsub_rn(as[slot].y, __fmul_rn(mx, my));
                const float ux = mx + 128.0f, uy = my + 128.0f;
                const float num = __fmul_rn(__fadd_rn(__fmul_rn(2.0f * ux, uy), C1), __fadd_rn(2.0f * cxy, C2));
                const float den =
                    __fmul_rn(__fadd_rn(__fadd_rn(__fmul_rn(ux, ux), __fmul_rn(uy, uy)), C1), __fadd_rn(vsum, C2));
                const float ssim = num == den ? 1.0f : __fdividef(num, den);
                csum += valid ? ssim : 0.0f;   // a select: positions outside add nothing
            }
            total += double(csum);
        }
        if (nsub == 0 && g.use_tma && tid == 0 && nu < g.nunits) issue(nu, nk);

        // ---- end of the unit: fixed-order CTA sums
        if (nu != u) {
            const uint64_t ew = warp_sum_u64(err);
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) total += __shfl_xor_sync(0xffffffffu, total, off);
            if ((tid & 31) == 0) {
                red_u[tid >> 5] = ew;
                red_d[tid >> 5] = total;
            }
            __syncthreads();
            if (tid == 0) {
                unsigned long long e = 0;
                double t = 0.0;
                for (int w = 0; w < FM_T / 32; w++) {
                    e += red_u[w];
                    t += red_d[w];
                }
                g.sse_part[u] = e;
                g.ms_part[u] = t;
            }
            err = 0;
            total = 0.0;
            u = nu;
            if (u < g.nunits) cu.set(g, u);
        }
        k = nk;
    }
    if (!ok && tid == 0) {
        // a copy never arrived: mark the unit, let loads still in flight land
        // (bounded) before the CTA leaves
        g.ms_part[u] = __longlong_as_double(0x7ff8000000000000ll);
        while (consumed < issued) {
            mbar_wait_bounded(bar, consumed & 1u, FM_DRAIN_NS);
            ++consumed;
        }
    }
    if (g.use_tma && tid == 0) bulk_wait_all();
}

// Per image (one CTA each): SSE and PSNR from the exact integer sum of its units'
// errors (as the fused call), MSSIM = sum of the units' SSIM sums / positions.
static __global__ void fm_finalize(const unsigned long long *sse_part, const double *ms_part, int64_t per_img,
                                   int nimg, int H, int W, double m2, double *sse, float *psnr, double *mssim) {
    __shared__ unsigned long long ru[256 / 32];
    __shared__ double rd[256];
    const int img = blockIdx.x;
    if (img >= nimg) return;
    unsigned long long acc = 0;
    double am = 0.0;
    for (int64_t t = threadIdx.x; t < per_img; t += blockDim.x) {
        acc += sse_part[int64_t(img) * per_img + t];
        am += ms_part[int64_t(img) * per_img + t];
    }
    acc = warp_sum_u64(acc);
    if ((threadIdx.x & 31) == 0) ru[threadIdx.x >> 5] = acc;
    rd[threadIdx.x] = am;
    __syncthreads();
    for (int off = blockDim.x / 2; off > 0; off >>= 1) {
        if (int(threadIdx.x) < off) rd[threadIdx.x] += rd[threadIdx.x + off];
        __syncthreads();
    }
    if (threadIdx.x != 0) return;
    unsigned long long tot = 0;
    for (int w = 0; w < int(blockDim.x) / 32; w++) tot += ru[w];
    const double s = double(tot) / m2;
    const double npx = double(H) * double(W);
    sse[img] = s;
    float p;
    if (npx == 0.0) p = __int_as_float(0x7fc00000);
    else if (s == 0.0) p = __int_as_float(0x7f800000);
    else p = float(10.0 * log10(255.0 * 255.0 * npx / s));
    psnr[img] = p;
    const double npos = double(H - FM_S + 1) * double(W - FM_S + 1);
    mssim[img] = (H < FM_S || W < FM_S) ? __longlong_as_double(0x7ff8000000000000ll) : rd[0] / npos;
}

template <int N>
using FmKernel = void (*)(PlanK<N>, FmMaps, FmGeom);

template <int N, int D0, int D1>
const void *fm_pick(int D, bool coef) {
    if constexpr (D0 > D1) {
        return nullptr;
    } else {
        if (D == D0)
            return coef ? reinterpret_cast<const void *>(fm_kernel<N, D0, true>)
                        : reinterpret_cast<const void *>(fm_kernel<N, D0, false>);
        return fm_pick<N, D0 + 1, D1>(D, coef);
    }
}

// Arguments of one fused-with-SSIM call (validated by the caller).
struct FmArgs {
    const uint8_t *img;
    int nimg, H, W;
    int64_t ld, img_stride;
    int r;
    float *zcoef;
    uint8_t *recon;
    int64_t ld_recon, recon_stride;
    double *sse, *mssim;
    float *psnr;
    int force_plain;
};

// Rows per segment: a multiple of 88, about an eighth of the image (at most 528
// rows), from the image height alone so that the result does not depend on nimg.
inline int fm_seg_rows(int H) {
    const int steps = (H + FM_SC - 1) / FM_SC;
    return FM_SC * std::min(6, std::max(1, (steps + 7) / 8));
}

// Host launcher (the plan is on the register path for N; arguments validated).
template <int N, int D0, int D1>
rklt_status launch_fm(const Plan &plan, const FmArgs &a, cudaStream_t st) {
    const PlanK<N> &pk = plan.kparams<N>();
    FmGeom g{};
    g.img = a.img;
    g.recon = a.recon;
    g.zcoef = a.r > 0 ? a.zcoef : nullptr;
    g.ld = a.ld;
    g.img_stride = a.nimg > 1 ? a.img_stride : a.ld * int64_t(a.H);
    g.ld_recon = a.ld_recon;
    g.recon_stride = a.nimg > 1 ? a.recon_stride : a.ld_recon * int64_t(a.H);
    g.H = a.H;
    g.W = a.W;
    g.nimg = a.nimg;
    g.r = a.r;
    const uintptr_t za = reinterpret_cast<uintptr_t>(a.zcoef);
    g.cvec = (a.r % 4 == 0 && (za & 15) == 0) ? 4 : ((a.r % 2 == 0 && (za & 7) == 0) ? 2 : 1);
    g.strips = (a.W + FM_WS - 1) / FM_WS;
    g.seg_rows = fm_seg_rows(a.H);
    g.segs = (a.H + g.seg_rows - 1) / g.seg_rows;
    g.nunits = int64_t(g.strips) * g.segs * a.nimg;
    g.timeout_ns = wait_timeout_ns();
    {
        double e[FM_S], tot = 0.0;
        for (int k = 0; k < FM_S; k++) {
            const double d = k - (FM_S - 1) / 2;
            e[k] = std::exp(-d * d / (2.0 * 1.5 * 1.5));
            tot += e[k];
        }
        for (int k = 0; k < FM_S; k++) g.g[k] = float(e[k] / tot);
    }
    const bool empty = a.H == 0 || a.W == 0;
    const int64_t per_img = empty ? 0 : int64_t(g.strips) * g.segs;
    const size_t nu = size_t(std::max<int64_t>(g.nunits, 1));
    cudaMemPool_t pool = scratch_pool();
    if (!pool) return fail(RKLT_ERR_CUDA, "could not create the scratch memory pool");
    void *scratch = nullptr;
    if (cudaMallocFromPoolAsync(&scratch, nu * 16, pool, st) != cudaSuccess)
        return fail(RKLT_ERR_OOM, "scratch allocation failed");
    g.sse_part = static_cast<unsigned long long *>(scratch);
    g.ms_part = reinterpret_cast<double *>(g.sse_part + nu);
    cudaError_t e = cudaSuccess;
    if (!empty) {
        const auto is16 = [](const void *p, int64_t x, int64_t y) {
            return ((reinterpret_cast<uintptr_t>(p) | uintptr_t(x) | uintptr_t(y)) & 15) == 0;
        };
        bool tma = !a.force_plain && is16(a.img, a.ld, g.img_stride) &&
                   (!a.recon || is16(a.recon, a.ld_recon, g.recon_stride));
        FmMaps maps{};
        constexpr int LEAD = fm_lead_rows(N);
        if (tma) tma = make_map_u8(&maps.in256, a.img, a.W, a.H, a.nimg, a.ld, g.img_stride, FM_WS, FM_SC);
        if (tma) tma = make_map_u8(&maps.in16, a.img, a.W, a.H, a.nimg, a.ld, g.img_stride, FM_HW, FM_SC);
        if (tma) tma = make_map_u8(&maps.lead256, a.img, a.W, a.H, a.nimg, a.ld, g.img_stride, FM_WS, LEAD);
        if (tma) tma = make_map_u8(&maps.lead16, a.img, a.W, a.H, a.nimg, a.ld, g.img_stride, FM_HW, LEAD);
        if (tma && a.recon)
            tma = make_map_u8(&maps.out256, a.recon, a.W, a.H, a.nimg, a.ld_recon, g.recon_stride, FM_WS, FM_SC);
        g.use_tma = tma ? 1 : 0;
        const void *fn = fm_pick<N, D0, D1>(diag_bound(N, a.r), g.zcoef != nullptr);
        if (!fn) {
            cudaFreeAsync(scratch, st);
            return fail(RKLT_ERR_UNSUPPORTED, "fused SSIM pass: no kernel for this diagonal bound");
        }
        const int dev = ensure_smem_attr(fn);
        int per_sm = occupancy(fn, FM_T, FM_SMEM);
        if (per_sm < 1) per_sm = 1;
        const int64_t grid = std::min<int64_t>(g.nunits, int64_t(per_sm) * sm_count(dev));
        void *args[] = {const_cast<PlanK<N> *>(&pk), &maps, &g};
        e = cudaLaunchKernel(fn, dim3(unsigned(grid)), dim3(FM_T), args, FM_SMEM, st);
        if (e != cudaSuccess) {
            cudaFreeAsync(scratch, st);
            return cuda_fail(e, "fused SSIM kernel launch");
        }
    }
    fm_finalize<<<a.nimg, 256, 0, st>>>(g.sse_part, g.ms_part, per_img, a.nimg, a.H, a.W, double(pk.pm2), a.sse,
                                        a.psnr, a.mssim);
    e = cudaGetLastError();
    cudaFreeAsync(scratch, st);
    return e == cudaSuccess ? RKLT_OK : cuda_fail(e, "fused SSIM finalize launch");
}

rklt_status launch_fm_n4(const Plan &plan, const FmArgs &a, cudaStream_t st);
rklt_status launch_fm_n8(const Plan &plan, const FmArgs &a, cudaStream_t st);

}  // namespace rklt
