// rklt_mssim.cu -- mean structural similarity (MSSIM) of two 8-bit images, the
// quality measure of Sec. 4.1 (Wang et al. 2004): 11 x 11 Gaussian window
// (sigma = 1.5, weights normalised to sum 1), C1 = (0.01 * 255)^2, C2 = (0.03 * 255)^2,
// mean over the (H - 10) x (W - 10) positions where the window fits.
//
// A second pass over (original, decoded image): the window straddles the N x N
// blocks of the transform, so it needs its own traversal.  A CTA takes a unit of
// 256 output columns x MS_SEG output rows and walks down it in chunks of 11 input
// rows:
//   load   the chunk's 11 x 266 bytes of both images: when pointers and pitches are
//          16-byte aligned, TMA boxes of 256 + 16 columns (rows past the image read
//          as 0) issued one chunk ahead, completion on an mbarrier; else plain loads;
//   stage  the pixel pairs, centred at 128, as float4 (x, y, x^2 + y^2, x y) in
//          shared memory (one conversion per pixel, four pixels per task);
//   H      11-tap horizontal sums of the four quantities, four adjacent outputs
//          per thread, each staged column read once and scattered into the four
//          accumulators (packed FP32 FMAs: (x, y) and (x^2 + y^2, x y) pairs);
//   V      one thread per output column keeps 11 rolling accumulators in registers
//          (slot = output row mod 11, static because a chunk is 11 rows), adds the
//          chunk's rows with the vertical weights, and finishes one output row per
//          input row: SSIM from mu_x, mu_y, sigma_x^2 + sigma_y^2 and sigma_xy.
// The float4 rows are XOR-swizzled within groups of 8 columns, so that lanes 1 or 4
// columns apart hit distinct banks.
// Only x^2 + y^2 is needed (the SSIM denominator uses sigma_x^2 + sigma_y^2), so four
// window sums suffice.  Per thread, each chunk's SSIM values are summed in FP32 and
// added to an FP64 total; per unit the totals are summed in a fixed order in FP64,
// per image the units in index order.
//
// Precision: with values centred at 128 the second moments are below 2^15 and each
// is a sum of 121 products rounded in FP32 (22 rounding steps along the two passes);
// sigma_x^2 + sigma_y^2 = E[x^2 + y^2] - mu_x^2 - mu_y^2 then carries an absolute error
// of about 22 u (E[(x-128)^2] + E[(y-128)^2]), u = 2^-24, sigma_xy half that, and SSIM
// an error of at most four such terms over C2 (= 58.5).  The final quotient is taken
// with the fast reciprocal (2 ulp), except that num = den gives 1; the products and
// differences are not contracted, so identical images give SSIM = 1 exactly.
#include <algorithm>
#include <cmath>

#include "rklt_device.cuh"
#include "rklt_internal.h"

namespace rklt {

constexpr int MS_S = 11, MS_R = 5;
constexpr int MS_WS = 256;                             // output columns per unit (one per thread)
constexpr int MS_IW = 268;                             // input columns staged (266 used), a multiple of 4
constexpr int MS_CH = MS_S;                            // input rows per chunk
constexpr int MS_NCH = 48;                             // chunks per unit
constexpr int MS_SEG = MS_NCH * MS_CH - (MS_S - 1);    // 518 output rows per unit
constexpr int MS_THREADS = 256;
constexpr int MS_G = 4;                                // outputs per thread in the horizontal pass
// float4 column c of a row sits at c with its low 3 bits XOR (c / 4) mod 8
__host__ __device__ constexpr int ms_phys(int c) { return (c & ~7) | ((c ^ (c >> 2)) & 7); }
constexpr int MS_LDI = 272;                            // staged float4 per row
constexpr int MS_LDH = MS_WS;                          // horizontal-sum float4 per row
constexpr int MS_RAW = 3072;                           // one image's chunk: 11 x 256 bytes, then 11 x 16
constexpr int MS_RAW_OFF = (MS_CH * MS_LDI + MS_CH * MS_LDH) * 16 + (MS_THREADS / 32) * 8;
constexpr int MS_RAW_AL = (MS_RAW_OFF + 127) / 128 * 128;
constexpr int MS_SMEM = MS_RAW_AL + 2 * MS_RAW + 16;  // + the chunk's mbarrier
constexpr uint64_t MS_DRAIN_NS = 2000000000ull;

struct MsGeom {
    const uint8_t *x, *y;
    int64_t ldx, xstride, ldy, ystride;
    double *partials;      // one per unit
    int H, W, nimg, units_x, units_y;
    int64_t nunits;
    int use_tma;
    uint64_t timeout_ns;
    float g[MS_S];         // 1-D Gaussian, normalised; the window is g g^T
};

struct MsMaps {
    CUtensorMap x256, x16, y256, y16;   // boxes of 256 and 16 columns x 11 rows
};

__global__ void __launch_bounds__(MS_THREADS, 2)
    mssim_kernel(const __grid_constant__ MsGeom g, const __grid_constant__ MsMaps maps) {
    extern __shared__ __align__(128) float4 ms_smem4[];
    float4 *stg = ms_smem4;                              // [MS_CH][MS_LDI]
    float4 *hs = stg + MS_CH * MS_LDI;                   // [MS_CH][MS_LDH]
    double *red = reinterpret_cast<double *>(hs + MS_CH * MS_LDH);
    uint8_t *raw = reinterpret_cast<uint8_t *>(ms_smem4) + MS_RAW_AL;   // [x, y][MS_RAW]
    uint64_t *bar = reinterpret_cast<uint64_t *>(raw + 2 * MS_RAW);
    const int tid = threadIdx.x;
    if (g.use_tma && tid == 0) {
        mbar_init(bar, 1);
        fence_mbar_init();
    }
    __syncthreads();
    uint32_t consumed = 0;   // chunk loads waited for (the barrier's phase parity)
    uint32_t issued = 0;
    const int OH = g.H - MS_S + 1, OW = g.W - MS_S + 1;
    const float C1 = (0.01f * 255.0f) * (0.01f * 255.0f), C2 = (0.03f * 255.0f) * (0.03f * 255.0f);
    const int64_t per_img = int64_t(g.units_x) * g.units_y;
    float2 gw[MS_S];
#pragma unroll
    for (int k = 0; k < MS_S; k++) gw[k] = make_float2(g.g[k], g.g[k]);

    for (int64_t unit = blockIdx.x; unit < g.nunits; unit += gridDim.x) {
        const int img = int(unit / per_img);
        const int rem = int(unit - int64_t(img) * per_img);
        const int uy = rem / g.units_x, ux = rem - uy * g.units_x;
        const int r0 = uy * MS_SEG, c0 = ux * MS_WS;
        const uint8_t *xp = g.x + int64_t(img) * g.xstride;
        const uint8_t *yp = g.y + int64_t(img) * g.ystride;
        const int orows = min(MS_SEG, OH - r0);            // output rows of this unit
        const int nch = (orows + MS_S - 1 + MS_CH - 1) / MS_CH;
        const bool col_ok = c0 + tid < OW;
        const bool box16 = c0 + 256 < g.W;   // the 16-column box starts inside the image

        // TMA: chunk m's rows of both images into raw (one elected thread)
        const auto issue = [&](int m) {
            const int y = r0 + m * MS_CH;
            mbar_arrive_expect_tx(bar, 2 * MS_CH * (256 + (box16 ? 16 : 0)));
            tma_load_3d(raw, &maps.x256, c0, y, img, bar);
            tma_load_3d(raw + MS_RAW, &maps.y256, c0, y, img, bar);
            if (box16) {
                tma_load_3d(raw + MS_CH * 256, &maps.x16, c0 + 256, y, img, bar);
                tma_load_3d(raw + MS_RAW + MS_CH * 256, &maps.y16, c0 + 256, y, img, bar);
            }
        };
        // stage chunk m: input rows r0 + 11 m .. + 10, columns c0 .. c0 + 267 (266 used),
        // four columns per task
        const auto stage = [&](int m) {
            for (int q = tid; q < MS_CH * (MS_IW / 4); q += MS_THREADS) {
                const int rr = q / (MS_IW / 4), c4 = (q - rr * (MS_IW / 4)) * 4;
                uint32_t wx = 0u, wy = 0u;
                if (g.use_tma) {
                    if (c4 < 256 || box16) {
                        const int o = c4 < 256 ? rr * 256 + c4 : MS_CH * 256 + rr * 16 + (c4 - 256);
                        wx = *reinterpret_cast<const uint32_t *>(raw + o);
                        wy = *reinterpret_cast<const uint32_t *>(raw + MS_RAW + o);
                    }
                } else {
                    const int r = r0 + m * MS_CH + rr;
                    if (r < g.H) {
#pragma unroll
                        for (int e = 0; e < 4; e++) {
                            const int c = c0 + c4 + e;
                            if (c < g.W) {
                                wx |= uint32_t(xp[int64_t(r) * g.ldx + c]) << (8 * e);
                                wy |= uint32_t(yp[int64_t(r) * g.ldy + c]) << (8 * e);
                            }
                        }
                    }
                }
                float4 *dst = stg + rr * MS_LDI;
#pragma unroll
                for (int e = 0; e < 4; e++) {
                    // byte e under the exponent of 2^23 is the float 2^23 + byte (exact)
                    const uint32_t sel = 0x7440u | uint32_t(e);
                    const float a = __uint_as_float(__byte_perm(wx, 0x4B000000u, sel)) - 8388736.0f;
                    const float b = __uint_as_float(__byte_perm(wy, 0x4B000000u, sel)) - 8388736.0f;
                    // products and sum of integers below 2^15: exact in any order
                    dst[ms_phys(c4 + e)] = make_float4(a, b, fmaf(a, a, b * b), a * b);
                }
            }
        };
        // wait for chunk m (TMA mode), stage it; false on a timeout (uniform over the CTA)
        const auto take = [&](int m) -> bool {
            bool ok = true;
            if (g.use_tma) ok = mbar_wait_bounded(bar, consumed & 1u, g.timeout_ns);
            ++consumed;
            if (ok) stage(m);
            return !__syncthreads_or(!ok);
        };
        // horizontal pass over the staged chunk
        const auto hpass = [&]() {
            for (int q = tid; q < MS_CH * (MS_WS / MS_G); q += MS_THREADS) {
                const int rr = q / (MS_WS / MS_G), gc = (q - rr * (MS_WS / MS_G)) * MS_G;
                const float4 *src = stg + rr * MS_LDI;
                float2 p[MS_G], s[MS_G];
#pragma unroll
                for (int k = 0; k < MS_G + MS_S - 1; k++) {
                    const float4 v = src[ms_phys(gc + k)];
                    const float2 vp = make_float2(v.x, v.y), vs = make_float2(v.z, v.w);
#pragma unroll
                    for (int o = 0; o < MS_G; o++) {
                        const int t = k - o;  // tap of output o
                        if (t < 0 || t >= MS_S) continue;
                        if (t == 0) {
                            p[o] = __fmul2_rn(gw[0], vp);
                            s[o] = __fmul2_rn(gw[0], vs);
                        } else {
                            p[o] = __ffma2_rn(gw[t], vp, p[o]);
                            s[o] = __ffma2_rn(gw[t], vs, s[o]);
                        }
                    }
                }
                float4 *dst = hs + rr * MS_LDH;
#pragma unroll
                for (int o = 0; o < MS_G; o++) dst[ms_phys(gc + o)] = make_float4(p[o].x, p[o].y, s[o].x, s[o].y);
            }
        };

        float2 ap[MS_S], as[MS_S];  // rolling vertical accumulators, slot = output row mod 11
#pragma unroll
        for (int k = 0; k < MS_S; k++) ap[k] = as[k] = make_float2(0.0f, 0.0f);
        double total = 0.0;
        if (g.use_tma && tid == 0) {
            issue(0);
            ++issued;
        }
        bool ok = take(0);
        if (ok) {
            if (g.use_tma && tid == 0 && nch > 1) {
                issue(1);  // raw was consumed before the barrier in take()
                ++issued;
            }
            hpass();
            __syncthreads();
        }
        for (int m = 0; ok && m < nch; m++) {
            // vertical pass over chunk m (input rows j = 11 m + qq)
            float csum = 0.0f;
            const float4 *col = hs + ms_phys(tid);
#pragma unroll
            for (int qq = 0; qq < MS_CH; qq++) {
                const float4 v = col[qq * MS_LDH];
                const float2 vp = make_float2(v.x, v.y), vs = make_float2(v.z, v.w);
#pragma unroll
                for (int d = 0; d < MS_S; d++) {
                    const int slot = (qq - d + MS_S) % MS_S;  // output row j - d
                    if (d == 0) {
                        ap[slot] = __fmul2_rn(gw[0], vp);
                        as[slot] = __fmul2_rn(gw[0], vs);
                    } else {
                        ap[slot] = __ffma2_rn(gw[d], vp, ap[slot]);
                        as[slot] = __ffma2_rn(gw[d], vs, as[slot]);
                    }
                }
                // output row o = j - 10 is complete (slot (qq + 1) mod 11)
                const int o = m * MS_CH + qq - (MS_S - 1);
                const int slot = (qq + 1) % MS_S;
                {
                    const bool valid = o >= 0 && o < orows && col_ok;
                    const float mx = ap[slot].x, my = ap[slot].y;
                    const float vsum = __fsub_rn(as[slot].x, __fadd_rn(__fmul_rn(mx, mx), __fmul_rn(my, my)));
                    const float cxy = __fsub_rn(as[slot].y, __fmul_rn(mx, my));
                    const float ux = mx + 128.0f, uy = my + 128.0f;
                    const float num = __fmul_rn(__fadd_rn(__fmul_rn(2.0f * ux, uy), C1), __fadd_rn(2.0f * cxy, C2));
                    const float den = __fmul_rn(__fadd_rn(__fadd_rn(__fmul_rn(ux, ux), __fmul_rn(uy, uy)), C1),
                                                __fadd_rn(vsum, C2));
                    const float ssim = num == den ? 1.0f : __fdividef(num, den);
                    csum += valid ? ssim : 0.0f;   // a select: rows and columns outside add nothing
                }
            }
            total += double(csum);
            if (m + 1 < nch) {
                // the staging buffer is not read by the vertical pass
                if (!(ok = take(m + 1))) break;
                if (g.use_tma && tid == 0 && m + 2 < nch) {
                    issue(m + 2);
                    ++issued;
                }
                hpass();
                __syncthreads();
            }
        }
        if (!ok) {
            // a chunk never arrived: record NaN for the unit, let any load still in
            // flight land (bounded) before the CTA leaves, and stop
            if (tid == 0) {
                g.partials[unit] = __longlong_as_double(0x7ff8000000000000ll);
                while (consumed < issued) {
                    mbar_wait_bounded(bar, consumed & 1u, MS_DRAIN_NS);
                    ++consumed;
                }
            }
            return;
        }
        // fixed-order CTA sum in FP64
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) total += __shfl_xor_sync(0xffffffffu, total, off);
        if ((tid & 31) == 0) red[tid >> 5] = total;
        __syncthreads();
        if (tid == 0) {
            double t = 0.0;
            for (int w = 0; w < MS_THREADS / 32; w++) t += red[w];
            g.partials[unit] = t;
        }
        __syncthreads();  // the shared buffers are refilled by the next unit
    }
}

static __global__ void mssim_finalize(const double *partials, int64_t per_img, int nimg, int H, int W, double *out) {
    __shared__ double red[256];
    const int img = blockIdx.x;
    if (img >= nimg) return;
    double acc = 0.0;
    for (int64_t t = threadIdx.x; t < per_img; t += blockDim.x) acc += partials[int64_t(img) * per_img + t];
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int off = blockDim.x / 2; off > 0; off >>= 1) {
        if (threadIdx.x < off) red[threadIdx.x] += red[threadIdx.x + off];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        const double n = double(H - MS_S + 1) * double(W - MS_S + 1);
        out[img] = (H < MS_S || W < MS_S) ? __longlong_as_double(0x7ff8000000000000ll) : red[0] / n;
    }
}

}  // namespace rklt

using namespace rklt;

namespace rklt {
unsigned int take_status_mssim() {
    unsigned int v = 0, zero = 0;
    if (cudaMemcpyFromSymbol(&v, g_dev_status, sizeof(v)) != cudaSuccess) return 0;
    cudaMemcpyToSymbol(g_dev_status, &zero, sizeof(zero));
    return v;
}
}  // namespace rklt

extern "C" rklt_status rklt_mssim(const uint8_t *d_x, const uint8_t *d_y, int nimg, int H, int W, int64_t ldx,
                                  int64_t x_stride, int64_t ldy, int64_t y_stride, double *d_mssim, void *stream) {
    if (!d_mssim) return fail(RKLT_ERR_ARG, "d_mssim is NULL");
    if (nimg < 1) return fail(RKLT_ERR_ARG, "nimg must be >= 1");
    if (H < 0 || W < 0) return fail(RKLT_ERR_SHAPE, "H and W must be non-negative");
    if (ldx < W || ldy < W) return fail(RKLT_ERR_SHAPE, "ldx and ldy must be >= W");
    if (nimg > 1 && (x_stride < ldx * int64_t(H) || y_stride < ldy * int64_t(H)))
        return fail(RKLT_ERR_SHAPE, "image stride smaller than one image");
    if (H > 0 && W > 0 && (!d_x || !d_y)) return fail(RKLT_ERR_ARG, "d_x or d_y is NULL");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    MsGeom g{};
    g.x = d_x;
    g.y = d_y;
    g.ldx = ldx;
    g.ldy = ldy;
    g.xstride = nimg > 1 ? x_stride : ldx * int64_t(H);
    g.ystride = nimg > 1 ? y_stride : ldy * int64_t(H);
    g.H = H;
    g.W = W;
    g.nimg = nimg;
    {
        double e[MS_S], tot = 0.0;
        for (int k = 0; k < MS_S; k++) {
            const double d = k - MS_R;
            e[k] = std::exp(-d * d / (2.0 * 1.5 * 1.5));
            tot += e[k];
        }
        for (int k = 0; k < MS_S; k++) g.g[k] = float(e[k] / tot);
    }
    const int OH = H - MS_S + 1, OW = W - MS_S + 1;
    if (OH < 1 || OW < 1) {
        mssim_finalize<<<nimg, 256, 0, st>>>(nullptr, 0, nimg, H, W, d_mssim);
        const cudaError_t e = cudaGetLastError();
        return e == cudaSuccess ? RKLT_OK : cuda_fail(e, "mssim finalize launch");
    }
    g.units_x = (OW + MS_WS - 1) / MS_WS;
    g.units_y = (OH + MS_SEG - 1) / MS_SEG;
    g.nunits = int64_t(g.units_x) * g.units_y * nimg;
    cudaMemPool_t pool = scratch_pool();
    if (!pool) return fail(RKLT_ERR_CUDA, "could not create the scratch memory pool");
    void *scratch = nullptr;
    if (cudaMallocFromPoolAsync(&scratch, size_t(g.nunits) * sizeof(double), pool, st) != cudaSuccess)
        return fail(RKLT_ERR_OOM, "scratch allocation failed");
    g.partials = static_cast<double *>(scratch);
    MsMaps maps{};
    const auto is16 = [](const void *p, int64_t a, int64_t b) {
        return ((reinterpret_cast<uintptr_t>(p) | uintptr_t(a) | uintptr_t(b)) & 15) == 0;
    };
    bool tma = transport_mode() != 1 && is16(d_x, ldx, g.xstride) && is16(d_y, ldy, g.ystride);
    if (tma) tma = make_map_u8(&maps.x256, d_x, W, H, nimg, ldx, g.xstride, 256, MS_CH);
    if (tma) tma = make_map_u8(&maps.x16, d_x, W, H, nimg, ldx, g.xstride, 16, MS_CH);
    if (tma) tma = make_map_u8(&maps.y256, d_y, W, H, nimg, ldy, g.ystride, 256, MS_CH);
    if (tma) tma = make_map_u8(&maps.y16, d_y, W, H, nimg, ldy, g.ystride, 16, MS_CH);
    g.use_tma = tma ? 1 : 0;
    g.timeout_ns = wait_timeout_ns();
    const int dev = ensure_smem_attr(reinterpret_cast<const void *>(mssim_kernel));
    const int64_t grid = std::min<int64_t>(g.nunits, int64_t(sm_count(dev)) * 2);
    mssim_kernel<<<unsigned(grid), MS_THREADS, MS_SMEM, st>>>(g, maps);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) {
        mssim_finalize<<<nimg, 256, 0, st>>>(g.partials, int64_t(g.units_x) * g.units_y, nimg, H, W, d_mssim);
        e = cudaGetLastError();
    }
    cudaFreeAsync(scratch, st);
    return e == cudaSuccess ? RKLT_OK : cuda_fail(e, "mssim kernel launch");
}
