// rklt_fmssim_n8.cu -- the fused pass with the structural similarity, N = 8
// (diagonal bounds up to 5, r <= 15), and its C ABI entry point.
#include "rklt_fmssim.cuh"

namespace rklt {
rklt_status launch_fm_n8(const Plan &plan, const FmArgs &a, cudaStream_t st) {
    return launch_fm<8, 0, PARS_DMAX8>(plan, a, st);
}
unsigned int take_status_fm_n8() { return take_tu_status(); }
}  // namespace rklt

using namespace rklt;

extern "C" rklt_status rklt_fused_mssim(const rklt_plan *plan, const uint8_t *d_img, int nimg, int H, int W,
                                        int64_t ld, int64_t img_stride, int r, float *d_zcoef, uint8_t *d_recon,
                                        int64_t ld_recon, int64_t recon_stride, double *d_sse, float *d_psnr,
                                        double *d_mssim, void *stream) {
    if (!plan) return fail(RKLT_ERR_ARG, "plan is NULL");
    const int N = plan->p.N;
    if (nimg < 1 || nimg > 65535) return fail(RKLT_ERR_ARG, "nimg must lie in [1, 65535]");
    if (!d_sse || !d_psnr || !d_mssim) return fail(RKLT_ERR_ARG, "d_sse, d_psnr and d_mssim are required");
    if (r < 0 || r > N * N) return fail(RKLT_ERR_ARG, "r must lie in [0, N*N]");
    if (H < 0 || W < 0 || H % N || W % N) return fail(RKLT_ERR_SHAPE, "H and W must be non-negative multiples of N");
    if (ld < W) return fail(RKLT_ERR_SHAPE, "ld must be >= W");
    const bool empty = H == 0 || W == 0;
    if (!empty && !d_img) return fail(RKLT_ERR_ARG, "d_img is NULL");
    if (nimg > 1 && img_stride < ld * int64_t(H)) return fail(RKLT_ERR_SHAPE, "img_stride smaller than one image");
    if (d_recon) {
        if (ld_recon < W) return fail(RKLT_ERR_SHAPE, "ld_recon must be >= W");
        if (nimg > 1 && recon_stride < ld_recon * int64_t(H))
            return fail(RKLT_ERR_SHAPE, "recon_stride smaller than one image");
    }
    if (!empty && (int64_t(H) * W) / int64_t(H) != W) return fail(RKLT_ERR_SHAPE, "image too large");
    cudaStream_t st = static_cast<cudaStream_t>(stream);

    FusedArgs fa{};
    fa.r = r;
    const bool one_pass = (N == 4 && pars_applies<4>(plan->p, fa)) || (N == 8 && pars_applies<8>(plan->p, fa));
    if (one_pass) {
        FmArgs a{};
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
        a.mssim = d_mssim;
        a.force_plain = transport_mode() == 1;
        return N == 4 ? launch_fm_n4(plan->p, a, st) : launch_fm_n8(plan->p, a, st);
    }
    // other plans: the fused pass, then the SSIM pass over its reconstruction (kept in
    // a stream-ordered scratch image when the caller wants none)
    uint8_t *rec = d_recon;
    int64_t ldr = ld_recon, rstr = recon_stride;
    void *tmp = nullptr;
    if (!rec && !empty) {
        ldr = (int64_t(W) + 15) / 16 * 16;
        rstr = ldr * H;
        cudaMemPool_t pool = scratch_pool();
        if (!pool) return fail(RKLT_ERR_CUDA, "could not create the scratch memory pool");
        if (cudaMallocFromPoolAsync(&tmp, size_t(rstr) * size_t(nimg), pool, st) != cudaSuccess)
            return fail(RKLT_ERR_OOM, "scratch allocation failed");
        rec = static_cast<uint8_t *>(tmp);
    }
    rklt_status s = rklt_fused_batched(plan, d_img, nimg, H, W, ld, img_stride, r, d_zcoef, rec, ldr, rstr, d_sse,
                                       d_psnr, stream);
    if (s == RKLT_OK) s = rklt_mssim(d_img, rec, nimg, H, W, ld, img_stride, ldr, rstr, d_mssim, stream);
    if (tmp) cudaFreeAsync(tmp, st);
    return s;
}
