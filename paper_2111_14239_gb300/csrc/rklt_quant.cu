// rklt_quant.cu -- JPEG-like quantisation with S absorbed into the quantiser
// (Appendix of arXiv 2111.14239): for every N x N block (N = 4, 8)
//   C    = T A T^T                     exact integers (FP32 sums below 2^24)
//   Bbar = round(C / Qtilde)           Qtilde = Q / (s s^T), round(x) = floor(x + 1/2)
//   B'   = Bbar o Q                    the decoder's dequantised coefficients
//   A'   = That^{-1} B' That^{-T} = T^{-1} (Bbar o Qtilde) T^{-T}   (S cancels again)
// with the first r zig-zag positions kept, the 8-bit reconstruction, and the
// per-image SSE / PSNR as in the fused pass.
//
// Floating point decides the integer Bbar, so the decision is fixed in binary32:
// w_ij = fl32(s_i s_j / Q_ij) (FP64 quotient rounded once, on the host),
// q = fl32(C_ij * w_ij) (__fmul_rn, no contraction), Bbar = floor(q + 1/2) (exact
// for |q| < 2^22).  One thread transforms one block; 32 adjacent blocks per warp.
#include <algorithm>
#include <cmath>
#include <cstring>

#include "rklt_device.cuh"
#include "rklt_internal.h"

namespace rklt {

template <int N>
struct QuantK {
    float T[N][N];    // bare integer T
    float Ti[N][N];   // T^{-1}
    float w[N][N];    // fl32(s_i s_j / Q_ij)
    float qt[N][N];   // fl32(Q_ij / (s_i s_j)) = Qtilde (dequantisation in the C domain)
};

struct QuantGeom {
    const uint8_t *img;
    uint8_t *recon;
    int32_t *qcoef;
    float *partials;      // one FP32 SSE per block
    int64_t ld, img_stride, ld_recon, recon_stride;
    int64_t blocks_per_img, nblk;
    int H, W, nimg, bw, r;
};

template <int N>
__global__ void __launch_bounds__(256) quant_kernel(const __grid_constant__ QuantK<N> K, const QuantGeom g) {
    for (int64_t b = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; b < g.nblk; b += int64_t(gridDim.x) * blockDim.x) {
        const int64_t img = b / g.blocks_per_img;
        const int64_t lb = b - img * g.blocks_per_img;
        const int by = int(lb / g.bw), bx = int(lb - int64_t(by) * g.bw);
        const uint8_t *src = g.img + img * g.img_stride + int64_t(by) * N * g.ld + int64_t(bx) * N;
        // Y = T A (integers)
        float y1[N][N];
        {
            float a[N][N];
#pragma unroll
            for (int y = 0; y < N; y++)
#pragma unroll
                for (int x = 0; x < N; x++) a[y][x] = float(src[int64_t(y) * g.ld + x]);
#pragma unroll
            for (int i = 0; i < N; i++)
#pragma unroll
                for (int x = 0; x < N; x++) {
                    float acc = 0.0f;
#pragma unroll
                    for (int y = 0; y < N; y++) acc = fmaf(K.T[i][y], a[y][x], acc);
                    y1[i][x] = acc;
                }
        }
        // C = Y T^T, quantised in place for the first r zig-zag positions (Bbar), and
        // replaced by the dequantised C-domain value Bbar * Qtilde (0 when dropped)
        float c[N][N];
        int32_t *qdst = g.qcoef ? g.qcoef + b * g.r : nullptr;
#pragma unroll
        for (int i = 0; i < N; i++)
#pragma unroll
            for (int j = 0; j < N; j++) {
                float acc = 0.0f;
#pragma unroll
                for (int x = 0; x < N; x++) acc = fmaf(y1[i][x], K.T[j][x], acc);
                const int z = zz_index(N, i, j);
                float v = 0.0f;
                if (z < g.r) {
                    const float bq = floorf(__fadd_rn(__fmul_rn(acc, K.w[i][j]), 0.5f));
                    if (qdst) qdst[z] = int32_t(bq);
                    v = bq * K.qt[i][j];
                }
                c[i][j] = v;
            }
        // A' = T^{-1} C' T^{-T}: X = T^{-1} C' first (reusing y1)
#pragma unroll
        for (int y = 0; y < N; y++)
#pragma unroll
            for (int j = 0; j < N; j++) {
                float acc = 0.0f;
#pragma unroll
                for (int i = 0; i < N; i++) acc = fmaf(K.Ti[y][i], c[i][j], acc);
                y1[y][j] = acc;
            }
        uint8_t *dst = g.recon ? g.recon + img * g.recon_stride + int64_t(by) * N * g.ld_recon + int64_t(bx) * N
                               : nullptr;
        float sse = 0.0f;
#pragma unroll
        for (int y = 0; y < N; y++)
#pragma unroll
            for (int x = 0; x < N; x++) {
                float acc = 0.0f;
#pragma unroll
                for (int j = 0; j < N; j++) acc = fmaf(y1[y][j], K.Ti[x][j], acc);
                const float e = float(src[int64_t(y) * g.ld + x]) - acc;
                sse = fmaf(e, e, sse);
                if (dst) dst[int64_t(y) * g.ld_recon + x] = uint8_t(recon_byte(acc));
            }
        g.partials[b] = sse;
    }
}

// Per-image FP64 sum of the block partials in index order, then PSNR.
static __global__ void quant_finalize(const float *partials, int64_t per_img, int nimg, int H, int W, double *sse,
                                      float *psnr) {
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

template <int N>
static void fill_quant(const Plan &p, const double *Q, QuantK<N> &k) {
    std::memset(&k, 0, sizeof(k));
    for (int i = 0; i < N; i++)
        for (int j = 0; j < N; j++) {
            k.T[i][j] = float(p.T[size_t(i) * N + j]);
            k.Ti[i][j] = float(p.Tinv[size_t(i) * N + j]);
            k.w[i][j] = float(p.s[i] * p.s[j] / Q[i * N + j]);
            k.qt[i][j] = float(Q[i * N + j] / (p.s[i] * p.s[j]));
        }
}

template <int N>
static rklt_status launch_quant(const Plan &p, const double *Q, const QuantGeom &g0, double *sse, float *psnr,
                                cudaStream_t st) {
    QuantK<N> k;
    fill_quant<N>(p, Q, k);
    QuantGeom g = g0;
    if (g.nblk == 0) {
        quant_finalize<<<g.nimg, 256, 0, st>>>(nullptr, 0, g.nimg, g.H, g.W, sse, psnr);
        const cudaError_t e = cudaGetLastError();
        return e == cudaSuccess ? RKLT_OK : cuda_fail(e, "quant finalize launch");
    }
    cudaMemPool_t pool = scratch_pool();
    if (!pool) return fail(RKLT_ERR_CUDA, "could not create the scratch memory pool");
    void *scratch = nullptr;
    if (cudaMallocFromPoolAsync(&scratch, size_t(g.nblk) * sizeof(float), pool, st) != cudaSuccess)
        return fail(RKLT_ERR_OOM, "scratch allocation failed");
    g.partials = static_cast<float *>(scratch);
    int dev = 0;
    cudaGetDevice(&dev);
    const int64_t grid = std::min<int64_t>((g.nblk + 255) / 256, int64_t(sm_count(dev)) * 8);
    quant_kernel<N><<<unsigned(grid), 256, 0, st>>>(k, g);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) {
        quant_finalize<<<g.nimg, 256, 0, st>>>(g.partials, g.blocks_per_img, g.nimg, g.H, g.W, sse, psnr);
        e = cudaGetLastError();
    }
    cudaFreeAsync(scratch, st);
    return e == cudaSuccess ? RKLT_OK : cuda_fail(e, "quant kernel launch");
}

}  // namespace rklt

using namespace rklt;

extern "C" rklt_status rklt_fused_quant(const rklt_plan *plan, const uint8_t *d_img, int nimg, int H, int W,
                                        int64_t ld, int64_t img_stride, int r, const double *h_Q, int32_t *d_qcoef,
                                        uint8_t *d_recon, int64_t ld_recon, int64_t recon_stride, double *d_sse,
                                        float *d_psnr, void *stream) {
    if (!plan) return fail(RKLT_ERR_ARG, "plan is NULL");
    const Plan &p = plan->p;
    const int N = p.N;
    if (p.kind != 0) return fail(RKLT_ERR_UNSUPPORTED, "quantisation with S absorbed needs a rounded (integer) plan");
    if (N != 4 && N != 8) return fail(RKLT_ERR_UNSUPPORTED, "quantisation is built for N = 4 and N = 8");
    if (!h_Q) return fail(RKLT_ERR_ARG, "h_Q is NULL");
    for (int k = 0; k < N * N; k++)
        if (!(h_Q[k] > 0.0) || !std::isfinite(h_Q[k])) return fail(RKLT_ERR_ARG, "Q entries must be positive and finite");
    if (!d_sse || !d_psnr) return fail(RKLT_ERR_ARG, "d_sse and d_psnr are required");
    if (nimg < 1) return fail(RKLT_ERR_ARG, "nimg must be >= 1");
    if (r < 0 || r > N * N) return fail(RKLT_ERR_ARG, "r must lie in [0, N*N]");
    if (H < 0 || W < 0 || H % N || W % N) return fail(RKLT_ERR_SHAPE, "H and W must be non-negative multiples of N");
    if (ld < W) return fail(RKLT_ERR_SHAPE, "ld must be >= W");
    if (nimg > 1 && img_stride < ld * int64_t(H)) return fail(RKLT_ERR_SHAPE, "img_stride smaller than one image");
    if (H > 0 && W > 0 && !d_img) return fail(RKLT_ERR_ARG, "d_img is NULL");
    if (d_recon && ld_recon < W) return fail(RKLT_ERR_SHAPE, "ld_recon must be >= W");
    if (d_recon && nimg > 1 && recon_stride < ld_recon * int64_t(H))
        return fail(RKLT_ERR_SHAPE, "recon_stride smaller than one image");
    QuantGeom g{};
    g.img = d_img;
    g.recon = d_recon;
    g.qcoef = r > 0 ? d_qcoef : nullptr;
    g.ld = ld;
    g.img_stride = nimg > 1 ? img_stride : ld * int64_t(H);
    g.ld_recon = ld_recon;
    g.recon_stride = nimg > 1 ? recon_stride : ld_recon * int64_t(H);
    g.H = H;
    g.W = W;
    g.nimg = nimg;
    g.bw = N ? W / N : 0;
    g.r = r;
    g.blocks_per_img = int64_t(H / N) * (W / N);
    g.nblk = g.blocks_per_img * nimg;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    return N == 4 ? launch_quant<4>(p, h_Q, g, d_sse, d_psnr, st) : launch_quant<8>(p, h_Q, g, d_sse, d_psnr, st);
}
