// rklt_quant.cu -- JPEG-like quantisation with S absorbed into the quantiser
// (Appendix of arXiv 2111.14239): for every N x N block (N = 4, 8, 16, 32)
//   C    = T A T^T                     exact integers (FP32 sums below 2^24)
//   Bbar = round(C / Qtilde)           Qtilde = Q / (s s^T), round(x) = floor(x + 1/2)
//   B'   = Bbar o Q                    the decoder's dequantised coefficients
//   A'   = That^{-1} B' That^{-T} = T^{-1} (Bbar o Qtilde) T^{-T}   (S cancels again)
// with the first r zig-zag positions kept, the 8-bit reconstruction, and the
// per-image SSE / PSNR as in the fused pass.
//
// This file validates the call; the work runs in the fused kernel's quantised
// variants (rklt_fused_impl.cuh; for N = 16, 32 the tensor-core and cooperative
// paths, rklt_tc.cuh): the same TMA tile pipeline, with the integer
// decision fixed in binary32 there: w_ij = fl32(s_i s_j / Q_ij) (FP64 quotient
// rounded once, on the host), q = fl32(C_ij * w_ij) (no contraction),
// Bbar = floor(q + 1/2) (exact for |q| < 2^22).
#include <cmath>

#include "rklt_internal.h"

using namespace rklt;

extern "C" rklt_status rklt_fused_quant(const rklt_plan *plan, const uint8_t *d_img, int nimg, int H, int W,
                                        int64_t ld, int64_t img_stride, int r, const double *h_Q, int32_t *d_qcoef,
                                        uint8_t *d_recon, int64_t ld_recon, int64_t recon_stride, double *d_sse,
                                        float *d_psnr, void *stream) {
    if (!plan) return fail(RKLT_ERR_ARG, "plan is NULL");
    const Plan &p = plan->p;
    const int N = p.N;
    if (p.kind != 0) return fail(RKLT_ERR_UNSUPPORTED, "quantisation with S absorbed needs a rounded (integer) plan");
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
    if (nimg > 65535) return fail(RKLT_ERR_ARG, "nimg must lie in [1, 65535]");
    if (H > 0 && W > 0 && (int64_t(H) * W) / int64_t(H) != W) return fail(RKLT_ERR_SHAPE, "image too large");
    FusedArgs a{};
    a.img = d_img;
    a.nimg = nimg;
    a.H = H;
    a.W = W;
    a.ld = ld;
    a.img_stride = img_stride;
    a.r = r;
    a.zcoef = r > 0 ? reinterpret_cast<float *>(d_qcoef) : nullptr;
    a.recon = d_recon;
    a.ld_recon = ld_recon;
    a.recon_stride = recon_stride;
    a.sse = d_sse;
    a.psnr = d_psnr;
    a.force_plain = transport_mode() == 1;
    a.Q = h_Q;
    a.engine = 0;   // the quantised N = 32 path runs on the warp-level tensor-core engine
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    switch (N) {
        case 4: return launch_fused_n4(p, a, st);
        case 8: return launch_fused_n8(p, a, st);
        case 16: return launch_fused_n16(p, a, st);
        default: return launch_fused_n32(p, a, st);
    }
}
