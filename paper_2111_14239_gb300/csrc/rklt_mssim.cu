// rklt_mssim.cu -- mean structural similarity (MSSIM) of two 8-bit images, the
// quality measure of Sec. 4.1 (Wang et al. 2004): 11 x 11 Gaussian window
// (sigma = 1.5, weights normalised to sum 1), C1 = (0.01 * 255)^2, C2 = (0.03 * 255)^2,
// mean over the (H - 10) x (W - 10) positions where the window fits.
//
// A second pass over (original, decoded image): the window straddles the N x N
// blocks of the transform, so it needs its own tile shape with a 5-pixel halo.
// Each CTA takes 16 x 128 output positions: it loads the 26 x 138 input region of
// both images into shared memory (centred at 128), runs the separable window as an
// 11-tap horizontal pass over the five sums (x, y, x^2, y^2, xy) and an 11-tap
// vertical pass, and forms SSIM per position.  Per-tile FP32 partials are summed
// per image in FP64 in a fixed order.
//
// Precision: with values centred at 128 the second moments are below 2^14 and each
// is a sum of 121 products rounded in FP32 (22 rounding steps along the two passes);
// the variance E[x^2] - mu^2 then carries an absolute error of about
// 22 u (E[(x-128)^2] + E[(y-128)^2]), u = 2^-24, and SSIM an error of at most
// four such terms over C2 (= 58.5).
#include <algorithm>
#include <cmath>

#include "rklt_device.cuh"
#include "rklt_internal.h"

namespace rklt {

constexpr int MS_S = 11, MS_R = 5;
constexpr int MS_TR = 16, MS_TC = 128;                 // output positions per tile
constexpr int MS_IR = MS_TR + MS_S - 1;                // 26 input rows
constexpr int MS_IC = MS_TC + MS_S - 1;                // 138 input columns
constexpr int MS_LD = 140;                             // shared row stride of the inputs (floats)
constexpr int MS_THREADS = 256;
constexpr int MS_SMEM = (2 * MS_IR * MS_LD + 5 * MS_IR * MS_TC + MS_THREADS / 32) * 4;

struct MsGeom {
    const uint8_t *x, *y;
    int64_t ldx, xstride, ldy, ystride;
    float *partials;       // one per tile
    int H, W, nimg, tiles_x, tiles_y;
    int64_t ntiles;
    float g[MS_S];         // 1-D Gaussian, normalised; the window is g g^T
};

__global__ void __launch_bounds__(MS_THREADS) mssim_kernel(const __grid_constant__ MsGeom g) {
    extern __shared__ float ms_smem[];
    float *xs = ms_smem;                          // [MS_IR][MS_LD]
    float *ys = xs + MS_IR * MS_LD;               // [MS_IR][MS_LD]
    float *hb = ys + MS_IR * MS_LD;               // [5][MS_IR][MS_TC]
    float *red = hb + 5 * MS_IR * MS_TC;          // [warps]
    const int tid = threadIdx.x;
    const int OH = g.H - MS_S + 1, OW = g.W - MS_S + 1;
    const float C1 = (0.01f * 255.0f) * (0.01f * 255.0f), C2 = (0.03f * 255.0f) * (0.03f * 255.0f);
    const int64_t per_img = int64_t(g.tiles_x) * g.tiles_y;
    for (int64_t tile = blockIdx.x; tile < g.ntiles; tile += gridDim.x) {
        const int img = int(tile / per_img);
        const int rem = int(tile - int64_t(img) * per_img);
        const int ty = rem / g.tiles_x, tx = rem - ty * g.tiles_x;
        const int r0 = ty * MS_TR, c0 = tx * MS_TC;
        const uint8_t *xp = g.x + int64_t(img) * g.xstride;
        const uint8_t *yp = g.y + int64_t(img) * g.ystride;
        // ---- inputs, centred at 128 (0 outside the image: those feed no valid output)
        for (int q = tid; q < MS_IR * MS_IC; q += MS_THREADS) {
            const int rr = q / MS_IC, cc = q - rr * MS_IC;
            const int r = r0 + rr, c = c0 + cc;
            const bool in = r < g.H && c < g.W;
            xs[rr * MS_LD + cc] = in ? float(xp[int64_t(r) * g.ldx + c]) - 128.0f : 0.0f;
            ys[rr * MS_LD + cc] = in ? float(yp[int64_t(r) * g.ldy + c]) - 128.0f : 0.0f;
        }
        __syncthreads();
        // ---- horizontal pass: the five sums over 11 columns
        for (int q = tid; q < MS_IR * MS_TC; q += MS_THREADS) {
            const int rr = q / MS_TC, t = q - rr * MS_TC;
            const float *xr = xs + rr * MS_LD + t, *yr = ys + rr * MS_LD + t;
            float sx = 0.0f, sy = 0.0f, sxx = 0.0f, syy = 0.0f, sxy = 0.0f;
#pragma unroll
            for (int k = 0; k < MS_S; k++) {
                const float a = xr[k], b = yr[k], w = g.g[k];
                sx = fmaf(w, a, sx);
                sy = fmaf(w, b, sy);
                sxx = fmaf(w, a * a, sxx);
                syy = fmaf(w, b * b, syy);
                sxy = fmaf(w, a * b, sxy);
            }
            hb[(0 * MS_IR + rr) * MS_TC + t] = sx;
            hb[(1 * MS_IR + rr) * MS_TC + t] = sy;
            hb[(2 * MS_IR + rr) * MS_TC + t] = sxx;
            hb[(3 * MS_IR + rr) * MS_TC + t] = syy;
            hb[(4 * MS_IR + rr) * MS_TC + t] = sxy;
        }
        __syncthreads();
        // ---- vertical pass and SSIM per position
        float acc = 0.0f;
        for (int q = tid; q < MS_TR * MS_TC; q += MS_THREADS) {
            const int o = q / MS_TC, t = q - o * MS_TC;
            if (r0 + o >= OH || c0 + t >= OW) continue;
            float m[5] = {0.0f, 0.0f, 0.0f, 0.0f, 0.0f};
#pragma unroll
            for (int k = 0; k < MS_S; k++) {
                const float w = g.g[k];
#pragma unroll
                for (int v = 0; v < 5; v++) m[v] = fmaf(w, hb[(v * MS_IR + o + k) * MS_TC + t], m[v]);
            }
            const float vx = m[2] - m[0] * m[0], vy = m[3] - m[1] * m[1], cxy = m[4] - m[0] * m[1];
            const float mx = m[0] + 128.0f, my = m[1] + 128.0f;
            const float num = (2.0f * mx * my + C1) * (2.0f * cxy + C2);
            const float den = (mx * mx + my * my + C1) * (vx + vy + C2);
            acc += num / den;
        }
        // ---- fixed-order CTA sum
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
        if ((tid & 31) == 0) red[tid >> 5] = acc;
        __syncthreads();
        if (tid == 0) {
            float t = 0.0f;
            for (int w = 0; w < MS_THREADS / 32; w++) t += red[w];
            g.partials[tile] = t;
        }
        __syncthreads();  // the shared buffers are refilled by the next tile
    }
}

static __global__ void mssim_finalize(const float *partials, int64_t per_img, int nimg, int H, int W, double *out) {
    __shared__ double red[256];
    const int img = blockIdx.x;
    if (img >= nimg) return;
    double acc = 0.0;
    for (int64_t t = threadIdx.x; t < per_img; t += blockDim.x) acc += double(partials[int64_t(img) * per_img + t]);
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
    g.tiles_x = (OW + MS_TC - 1) / MS_TC;
    g.tiles_y = (OH + MS_TR - 1) / MS_TR;
    g.ntiles = int64_t(g.tiles_x) * g.tiles_y * nimg;
    cudaMemPool_t pool = scratch_pool();
    if (!pool) return fail(RKLT_ERR_CUDA, "could not create the scratch memory pool");
    void *scratch = nullptr;
    if (cudaMallocFromPoolAsync(&scratch, size_t(g.ntiles) * sizeof(float), pool, st) != cudaSuccess)
        return fail(RKLT_ERR_OOM, "scratch allocation failed");
    g.partials = static_cast<float *>(scratch);
    const int dev = ensure_smem_attr(reinterpret_cast<const void *>(mssim_kernel));
    const int64_t grid = std::min<int64_t>(g.ntiles, int64_t(sm_count(dev)) * 2);
    mssim_kernel<<<unsigned(grid), MS_THREADS, MS_SMEM, st>>>(g);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) {
        mssim_finalize<<<nimg, 256, 0, st>>>(g.partials, int64_t(g.tiles_x) * g.tiles_y, nimg, H, W, d_mssim);
        e = cudaGetLastError();
    }
    cudaFreeAsync(scratch, st);
    return e == cudaSuccess ? RKLT_OK : cuda_fail(e, "mssim kernel launch");
}
