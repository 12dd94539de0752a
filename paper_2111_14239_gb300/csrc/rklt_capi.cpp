// rklt_capi.cpp -- C ABI of the fused path and the device status.
#include <cuda_runtime.h>

#include "rklt_internal.h"

using namespace rklt;

namespace {

rklt_status fused_common(const rklt_plan *plan, FusedArgs &a, void *stream) {
    if (!plan) return fail(RKLT_ERR_ARG, "plan is NULL");
    const int N = plan->p.N;
    if (a.nimg < 1 || a.nimg > 65535) return fail(RKLT_ERR_ARG, "nimg must lie in [1, 65535]");
    if (!a.sse || !a.psnr) return fail(RKLT_ERR_ARG, "d_sse and d_psnr are required");
    if (a.r < 0 || a.r > N * N) return fail(RKLT_ERR_ARG, "r must lie in [0, N*N]");
    if (a.H < 0 || a.W < 0 || a.H % N || a.W % N)
        return fail(RKLT_ERR_SHAPE, "H and W must be non-negative multiples of N");
    if (a.ld < a.W) return fail(RKLT_ERR_SHAPE, "ld must be >= W");
    const bool empty = a.H == 0 || a.W == 0;
    if (!empty && !a.img) return fail(RKLT_ERR_ARG, "d_img is NULL");
    if (a.nimg > 1 && a.img_stride < a.ld * int64_t(a.H))
        return fail(RKLT_ERR_SHAPE, "img_stride smaller than one image");
    if (a.recon) {
        if (a.ld_recon < a.W) return fail(RKLT_ERR_SHAPE, "ld_recon must be >= W");
        if (a.nimg > 1 && a.recon_stride < a.ld_recon * int64_t(a.H))
            return fail(RKLT_ERR_SHAPE, "recon_stride smaller than one image");
    }
    if (!empty && (int64_t(a.H) * a.W) / int64_t(a.H) != a.W) return fail(RKLT_ERR_SHAPE, "image too large");
    a.force_plain = transport_mode() == 1;
    a.engine = tensor_engine();
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    switch (N) {
        case 4: return launch_fused_n4(plan->p, a, st);
        case 8: return launch_fused_n8(plan->p, a, st);
        case 16: return launch_fused_n16(plan->p, a, st);
        case 32: return launch_fused_n32(plan->p, a, st);
        default: return fail(RKLT_ERR_ARG, "bad plan");
    }
}

}  // namespace

extern "C" {

rklt_status rklt_fused_batched(const rklt_plan *plan, const uint8_t *d_img, int nimg, int H, int W, int64_t ld,
                               int64_t img_stride, int r, float *d_zcoef, uint8_t *d_recon, int64_t ld_recon,
                               int64_t recon_stride, double *d_sse, float *d_psnr, void *stream) {
    FusedArgs a{};
    a.img = d_img;
    a.nimg = nimg;
    a.H = H;
    a.W = W;
    a.ld = ld;
    a.img_stride = img_stride;
    a.r = r;
    a.zcoef = d_zcoef;
    a.recon = d_recon;
    a.ld_recon = ld_recon;
    a.recon_stride = recon_stride;
    a.sse = d_sse;
    a.psnr = d_psnr;
    return fused_common(plan, a, stream);
}

rklt_status rklt_fused(const rklt_plan *plan, const uint8_t *d_img, int H, int W, int64_t ld, int r, float *d_zcoef,
                       uint8_t *d_recon, int64_t ld_recon, double *d_sse, float *d_psnr, void *stream) {
    return rklt_fused_batched(plan, d_img, 1, H, W, ld, 0, r, d_zcoef, d_recon, ld_recon, 0, d_sse, d_psnr, stream);
}

rklt_status rklt_device_status(void) {
    const cudaError_t e = cudaDeviceSynchronize();
    if (e != cudaSuccess) return cuda_fail(e, "cudaDeviceSynchronize");
    unsigned int v = take_status_n4() | take_status_n8() | take_status_n16() | take_status_n32() | take_status_split() |
                     take_status_mssim() | take_status_reg_n4() | take_status_reg_n8() |
                     take_status_reg_n8b() | take_status_fm_n4() | take_status_fm_n8();
    if (v) return fail(RKLT_ERR_TIMEOUT, "a bounded device-side wait gave up");
    return RKLT_OK;
}

}  // extern "C"
