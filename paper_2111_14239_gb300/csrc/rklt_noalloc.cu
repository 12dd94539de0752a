// rklt_noalloc.cu -- rklt_fused without any allocation.
//
// rklt_fused takes its scratch (one error partial per 64 x 256 tile, or per 32 x 256
// strip for the N = 32 tensor-memory kernel: a float, or a 64-bit integer on the
// register path whose error comes from Parseval's identity) from a stream-ordered
// memory pool.  This variant takes it from a fixed array in the library's own
// device memory instead, so a call performs no allocation of any kind.  The array
// is a file-scope __device__ object: every GPU that loads the library holds it
// (512 KB) until the process exits.  Host code cannot pass the array's name to a
// kernel -- on the host that name denotes a stand-in object, not device memory --
// so its device address is looked up with cudaGetSymbolAddress, with the device
// current, once per device and context.
#include <cudaTypedefs.h>

#include <mutex>

#include "rklt_internal.h"

namespace rklt {

constexpr int64_t kNoAllocMaxTiles = 65536;  // 2^16 tiles: 2^30 pixels (2^29 for 32-row strips)

static __device__ __align__(256) unsigned long long g_noalloc_partials[kNoAllocMaxTiles];  // 8 bytes per tile

namespace {

std::mutex g_mu;
struct Cached {
    unsigned long long ctx = 0;  // context the address belongs to (0: none yet)
    float *addr = nullptr;
};
Cached g_addr[64];

// Unique id of the calling thread's current context, or 0 when none is current or
// the driver entry points are missing.  Ids are never reused, so an address cached
// under one id cannot outlive the context it came from (a device reset makes a new
// context with a new id, and the next call looks the address up again).
unsigned long long current_ctx_id() {
    static PFN_cuCtxGetCurrent_v4000 get_cur = nullptr;
    static PFN_cuCtxGetId_v12000 get_id = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        cudaDriverEntryPointQueryResult q;
        void *p = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_cur = reinterpret_cast<PFN_cuCtxGetCurrent_v4000>(p);
        p = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_id = reinterpret_cast<PFN_cuCtxGetId_v12000>(p);
    });
    if (!get_cur || !get_id) return 0;
    CUcontext c = nullptr;
    if (get_cur(&c) != CUDA_SUCCESS || !c) return 0;
    unsigned long long id = 0;
    return get_id(c, &id) == CUDA_SUCCESS ? id : 0;
}

// Device address of g_noalloc_partials on the current device and context (looked
// up on the first call there).
rklt_status partials_address(float **out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
    if (dev < 0 || dev >= 64) return fail(RKLT_ERR_UNSUPPORTED, "device ordinal above 63");
    std::lock_guard<std::mutex> lk(g_mu);
    const unsigned long long id = current_ctx_id();
    if (!g_addr[dev].addr || id == 0 || g_addr[dev].ctx != id) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_partials);
        if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress of the no-alloc scratch array");
        g_addr[dev].addr = static_cast<float *>(p);
        g_addr[dev].ctx = current_ctx_id();   // the lookup made the device's context current
    }
    *out = g_addr[dev].addr;
    return RKLT_OK;
}

}  // namespace
}  // namespace rklt

using namespace rklt;

extern "C" rklt_status rklt_fused_noalloc(const rklt_plan *plan, const uint8_t *d_img, int H, int W, int64_t ld,
                                          int r, float *d_zcoef, uint8_t *d_recon, int64_t ld_recon,
                                          double *d_sse, float *d_psnr, void *stream) {
    if (!plan) return fail(RKLT_ERR_ARG, "plan is NULL");
    const int N = plan->p.N;
    if (!d_sse || !d_psnr) return fail(RKLT_ERR_ARG, "d_sse and d_psnr are required");
    if (r < 0 || r > N * N) return fail(RKLT_ERR_ARG, "r must lie in [0, N*N]");
    if (H < 0 || W < 0 || H % N || W % N) return fail(RKLT_ERR_SHAPE, "H and W must be non-negative multiples of N");
    if (ld < W) return fail(RKLT_ERR_SHAPE, "ld must be >= W");
    if (H > 0 && W > 0 && !d_img) return fail(RKLT_ERR_ARG, "d_img is NULL");
    if (d_recon && ld_recon < W) return fail(RKLT_ERR_SHAPE, "ld_recon must be >= W");
    // the kernel is decided here, once: the size check and the launch see the same one
    const int engine = tensor_engine();
    const int rows = fused_tile_rows(plan->p, diag_bound(N, r), engine);
    const int64_t tiles = int64_t((H + rows - 1) / rows) * ((W + kTileW - 1) / kTileW);
    if (tiles > kNoAllocMaxTiles)
        return fail(RKLT_ERR_ARG, "image too large for rklt_fused_noalloc: it needs " + std::to_string(tiles) +
                                      " tiles of " + std::to_string(rows) +
                                      " x 256 pixels and the fixed scratch array holds 65536");
    float *partials = nullptr;
    rklt_status st = partials_address(&partials);
    if (st != RKLT_OK) return st;
    FusedArgs a{};
    a.img = d_img;
    a.nimg = 1;
    a.H = H;
    a.W = W;
    a.ld = ld;
    a.r = r;
    a.zcoef = d_zcoef;
    a.recon = d_recon;
    a.ld_recon = ld_recon;
    a.sse = d_sse;
    a.psnr = d_psnr;
    a.partials = partials;
    a.scratch_cap = kNoAllocMaxTiles * int64_t(sizeof(unsigned long long));
    a.force_plain = transport_mode() == 1;
    a.engine = engine;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    switch (N) {
        case 4: return launch_fused_n4(plan->p, a, s);
        case 8: return launch_fused_n8(plan->p, a, s);
        case 16: return launch_fused_n16(plan->p, a, s);
        case 32: return launch_fused_n32(plan->p, a, s);
        default: return fail(RKLT_ERR_ARG, "bad plan");
    }
}
