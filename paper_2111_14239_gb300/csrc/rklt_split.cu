// rklt_split.cu -- the split path of Sec. 4.1: forward (integer or normalised),
// zonal retention, inverse and squared error / PSNR as separate kernels.  These
// materialise every intermediate in device memory; the fused kernel is the fast
// path.  Each CTA takes KB blocks with one thread per matrix entry.
#include <algorithm>

#include "rklt_device.cuh"
#include "rklt_internal.h"

namespace rklt {
namespace {

// Full N x N matrix from the stored half: T[i][N-1-j] = (-1)^i T[i][j].
template <int N>
__device__ float t_full(const PlanK<N> &P, int i, int j) {
    if (j < N / 2) return P.T[i][j];
    const float v = P.T[i][N - 1 - j];
    return (i & 1) ? -v : v;
}

// Full That^{-1} from its stored upper rows: That^{-1}[N-1-l][j] = (-1)^j That^{-1}[l][j].
template <int N>
__device__ float tih_full(const PlanK<N> &P, int l, int j) {
    if (l < N / 2) return P.Tih[l][j];
    const float v = P.Tih[N - 1 - l][j];
    return (j & 1) ? -v : v;
}

template <int N>
__host__ __device__ constexpr int blocks_per_cta() { return N >= 16 ? 1 : (256 / (N * N)); }

// Forward transform per block: C = T A T^T (exact in FP32); mode 0 writes int32
// raster, mode 1 writes B = s_i s_j C in zig-zag order.
template <int N>
__global__ void split_forward_kernel(const __grid_constant__ PlanK<N> P, const uint8_t *img, int H, int W,
                                     int64_t ld, int64_t nblk, int mode, int32_t *Cout, float *Bout) {
    constexpr int KB = blocks_per_cta<N>();
    __shared__ float As[KB][N][N + 1];
    __shared__ float Xs[KB][N][N + 1];
    const int j = threadIdx.x, i = threadIdx.y, kb = threadIdx.z;
    const int64_t b = int64_t(blockIdx.x) * KB + kb;
    const bool live = b < nblk;
    const int bw = W / N;
    int64_t by = 0, bx = 0;
    if (live) {
        by = b / bw;
        bx = b - by * bw;
        As[kb][i][j] = float(img[(by * N + i) * ld + bx * N + j]);
    }
    __syncthreads();
    if (live) {
        float acc = 0.0f;  // X[i][j] = sum_k T[i][k] A[k][j]
        for (int k = 0; k < N; k++) acc += t_full(P, i, k) * As[kb][k][j];
        Xs[kb][i][j] = acc;
    }
    __syncthreads();
    if (!live) return;
    float c = 0.0f;  // C[i][j] = sum_l X[i][l] T[j][l]
    for (int l = 0; l < N; l++) c += Xs[kb][i][l] * t_full(P, j, l);
    if (mode == 0) Cout[b * N * N + i * N + j] = int32_t(c);
    else Bout[b * N * N + zz_index(N, i, j)] = P.sij[i][j] * c;
}

// Inverse per block from compact coefficients: A' = That^{-1} B' That^{-T}.
template <int N>
__global__ void split_inverse_kernel(const __grid_constant__ PlanK<N> P, const float *zc, int r, int H, int W,
                                     float *recon, int64_t ldo, int64_t nblk) {
    constexpr int KB = blocks_per_cta<N>();
    __shared__ float Bs[KB][N][N + 1];
    __shared__ float Xs[KB][N][N + 1];
    const int j = threadIdx.x, i = threadIdx.y, kb = threadIdx.z;
    const int64_t b = int64_t(blockIdx.x) * KB + kb;
    const bool live = b < nblk;
    if (live) {
        const int z = zz_index(N, i, j);
        Bs[kb][i][j] = (z < r) ? zc[b * r + z] : 0.0f;
    }
    __syncthreads();
    if (live) {
        float acc = 0.0f;  // X[i][j] = sum_m B'[i][m] That^{-1}[j][m]
        for (int m = 0; m < N; m++) acc += Bs[kb][i][m] * tih_full(P, j, m);
        Xs[kb][i][j] = acc;
    }
    __syncthreads();
    if (!live) return;
    float a = 0.0f;  // A'[i][j] = sum_m That^{-1}[i][m] X[m][j]
    for (int m = 0; m < N; m++) a += tih_full(P, i, m) * Xs[kb][m][j];
    const int bw = W / N;
    const int64_t by = b / bw, bx = b - (b / bw) * bw;
    recon[(by * N + i) * ldo + bx * N + j] = a;
}

__global__ void zonal_kernel(const float *in, int nn, int64_t nblk, int r, float *out) {
    const int64_t total = nblk * r;
    for (int64_t q = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; q < total; q += int64_t(gridDim.x) * blockDim.x) {
        const int64_t b = q / r;
        out[q] = in[b * nn + (q - b * r)];
    }
}

// One CTA: SSE over the image in FP64 (fixed order), then PSNR.
__global__ void psnr_kernel(const uint8_t *img, int64_t ld, const float *rec, int64_t ldr, int H, int W, double *sse,
                            float *psnr) {
    __shared__ double red[1024];
    double acc = 0.0;
    const int64_t total = int64_t(H) * W;
    for (int64_t q = threadIdx.x; q < total; q += blockDim.x) {
        const int64_t y = q / W, x = q - (q / W) * W;
        const double e = double(img[y * ld + x]) - double(rec[y * ldr + x]);
        acc += e * e;
    }
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int off = blockDim.x / 2; off > 0; off >>= 1) {
        if (threadIdx.x < off) red[threadIdx.x] += red[threadIdx.x + off];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        const double s = red[0];
        *sse = s;
        float p;
        if (total == 0) p = __int_as_float(0x7fc00000);
        else if (s == 0.0) p = __int_as_float(0x7f800000);
        else p = float(10.0 * log10(255.0 * 255.0 * double(total) / s));
        *psnr = p;
    }
}

template <int N>
rklt_status launch_forward(const Plan &p, const uint8_t *img, int H, int W, int64_t ld, int mode, int32_t *C,
                           float *B, cudaStream_t st) {
    constexpr int KB = blocks_per_cta<N>();
    const int64_t nblk = int64_t(H / N) * (W / N);
    if (nblk == 0) return RKLT_OK;
    const int64_t grid = (nblk + KB - 1) / KB;
    if (grid > 0x7fffffffLL) return fail(RKLT_ERR_ARG, "image too large for the split path");
    split_forward_kernel<N><<<unsigned(grid), dim3(N, N, KB), 0, st>>>(p.kparams<N>(), img, H, W, ld, nblk, mode, C,
                                                                      B);
    const cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? RKLT_OK : cuda_fail(e, "forward launch");
}

template <int N>
rklt_status launch_inverse(const Plan &p, const float *zc, int r, int H, int W, float *rec, int64_t ldo,
                           cudaStream_t st) {
    constexpr int KB = blocks_per_cta<N>();
    const int64_t nblk = int64_t(H / N) * (W / N);
    if (nblk == 0) return RKLT_OK;
    const int64_t grid = (nblk + KB - 1) / KB;
    if (grid > 0x7fffffffLL) return fail(RKLT_ERR_ARG, "image too large for the split path");
    split_inverse_kernel<N><<<unsigned(grid), dim3(N, N, KB), 0, st>>>(p.kparams<N>(), zc, r, H, W, rec, ldo, nblk);
    const cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? RKLT_OK : cuda_fail(e, "inverse launch");
}

rklt_status check_image(const Plan &p, const void *d, int H, int W, int64_t ld) {
    if (H < 0 || W < 0 || H % p.N || W % p.N) return fail(RKLT_ERR_SHAPE, "H and W must be non-negative multiples of N");
    if (ld < W) return fail(RKLT_ERR_SHAPE, "pitch smaller than W");
    if (H > 0 && W > 0 && !d) return fail(RKLT_ERR_ARG, "image pointer is NULL");
    return RKLT_OK;
}

}  // namespace

unsigned int take_status_split() { return 0; }

}  // namespace rklt

using namespace rklt;

extern "C" {

rklt_status rklt_forward_int(const rklt_plan *plan, const uint8_t *d_img, int H, int W, int64_t ld, int32_t *d_C,
                             void *stream) {
    if (!plan) return fail(RKLT_ERR_ARG, "plan is NULL");
    if (plan->p.kind != 0) return fail(RKLT_ERR_UNSUPPORTED, "the integer stage needs a rounded (integer) plan");
    rklt_status s = check_image(plan->p, d_img, H, W, ld);
    if (s) return s;
    if (H > 0 && W > 0 && !d_C) return fail(RKLT_ERR_ARG, "d_C is NULL");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    switch (plan->p.N) {
        case 4: return launch_forward<4>(plan->p, d_img, H, W, ld, 0, d_C, nullptr, st);
        case 8: return launch_forward<8>(plan->p, d_img, H, W, ld, 0, d_C, nullptr, st);
        case 16: return launch_forward<16>(plan->p, d_img, H, W, ld, 0, d_C, nullptr, st);
        default: return launch_forward<32>(plan->p, d_img, H, W, ld, 0, d_C, nullptr, st);
    }
}

rklt_status rklt_forward(const rklt_plan *plan, const uint8_t *d_img, int H, int W, int64_t ld, float *d_coef,
                         void *stream) {
    if (!plan) return fail(RKLT_ERR_ARG, "plan is NULL");
    rklt_status s = check_image(plan->p, d_img, H, W, ld);
    if (s) return s;
    if (H > 0 && W > 0 && !d_coef) return fail(RKLT_ERR_ARG, "d_coef is NULL");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    switch (plan->p.N) {
        case 4: return launch_forward<4>(plan->p, d_img, H, W, ld, 1, nullptr, d_coef, st);
        case 8: return launch_forward<8>(plan->p, d_img, H, W, ld, 1, nullptr, d_coef, st);
        case 16: return launch_forward<16>(plan->p, d_img, H, W, ld, 1, nullptr, d_coef, st);
        default: return launch_forward<32>(plan->p, d_img, H, W, ld, 1, nullptr, d_coef, st);
    }
}

rklt_status rklt_zonal(const rklt_plan *plan, const float *d_coef, int64_t nblk, int r, float *d_out, void *stream) {
    if (!plan) return fail(RKLT_ERR_ARG, "plan is NULL");
    const int nn = plan->p.N * plan->p.N;
    if (nblk < 0 || r < 0 || r > nn) return fail(RKLT_ERR_ARG, "need nblk >= 0 and 0 <= r <= N*N");
    if (nblk == 0 || r == 0) return RKLT_OK;
    if (!d_coef || !d_out) return fail(RKLT_ERR_ARG, "NULL buffer");
    if (d_out == d_coef && r != nn) return fail(RKLT_ERR_ARG, "in-place zonal retention needs r == N*N");
    if (d_out == d_coef) return RKLT_OK;
    const int64_t total = nblk * r;
    const unsigned grid = unsigned(std::min<int64_t>((total + 255) / 256, 65535LL * 32));
    zonal_kernel<<<grid, 256, 0, static_cast<cudaStream_t>(stream)>>>(d_coef, nn, nblk, r, d_out);
    const cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? RKLT_OK : cuda_fail(e, "zonal launch");
}

rklt_status rklt_inverse(const rklt_plan *plan, const float *d_zcoef, int r, int H, int W, float *d_recon,
                         int64_t ld_out, void *stream) {
    if (!plan) return fail(RKLT_ERR_ARG, "plan is NULL");
    const int N = plan->p.N;
    if (r < 0 || r > N * N) return fail(RKLT_ERR_ARG, "r must lie in [0, N*N]");
    rklt_status s = check_image(plan->p, d_recon, H, W, ld_out);
    if (s) return s;
    if (H > 0 && W > 0 && r > 0 && !d_zcoef) return fail(RKLT_ERR_ARG, "d_zcoef is NULL");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    switch (N) {
        case 4: return launch_inverse<4>(plan->p, d_zcoef, r, H, W, d_recon, ld_out, st);
        case 8: return launch_inverse<8>(plan->p, d_zcoef, r, H, W, d_recon, ld_out, st);
        case 16: return launch_inverse<16>(plan->p, d_zcoef, r, H, W, d_recon, ld_out, st);
        default: return launch_inverse<32>(plan->p, d_zcoef, r, H, W, d_recon, ld_out, st);
    }
}

rklt_status rklt_psnr(const uint8_t *d_img, int64_t ld, const float *d_recon, int64_t ldr, int H, int W,
                      double *d_sse, float *d_psnr, void *stream) {
    if (H < 0 || W < 0) return fail(RKLT_ERR_SHAPE, "negative size");
    if (ld < W || ldr < W) return fail(RKLT_ERR_SHAPE, "pitch smaller than W");
    if (!d_sse || !d_psnr) return fail(RKLT_ERR_ARG, "d_sse and d_psnr are required");
    if (H > 0 && W > 0 && (!d_img || !d_recon)) return fail(RKLT_ERR_ARG, "NULL image");
    psnr_kernel<<<1, 1024, 0, static_cast<cudaStream_t>(stream)>>>(d_img, ld, d_recon, ldr, H, W, d_sse, d_psnr);
    const cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? RKLT_OK : cuda_fail(e, "psnr launch");
}

}  // extern "C"
