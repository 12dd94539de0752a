// rklt_internal.h -- declarations shared by the library's translation units.
// Not installed; the public boundary is include/rklt.h.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>

#include <cstdint>
#include <string>
#include <vector>

#include "../../include/rklt.h"

namespace rklt {

// Tile geometry of the fused kernel: 64 rows x 256 bytes per tile.
constexpr int kTileW = 256;
constexpr int kTileH = 64;

// Per-plan tables passed to kernels by value (they land in the constant bank,
// so the transform loops read T and T^{-1} as immediate-style operands).
//
// Parity of the KLT rows (R is centrosymmetric): T[i][N-1-j] = (-1)^i T[i][j],
// hence T^{-1}[N-1-l][j] = (-1)^j T^{-1}[l][j].  Only half of each matrix is
// stored; the kernels' butterflies rebuild the rest.
template <int N>
struct PlanK {
    // Operand pairs of the packed-FP32 register path (N <= 8; one unused entry otherwise):
    // both lanes of Td[j][l] hold T[j][l], both lanes of Tid[c][j] hold T^{-1}[c][j].
    static constexpr int RN = N <= 8 ? N : 2;
    float2 Td[RN][RN / 2];
    float2 Tid[RN / 2][RN];
    uint32_t T8[RN][RN / 4];     // T[i][4h .. 4h+3] as packed signed bytes (byte dot products)
    float T[N][N / 2];    // T[i][j], j < N/2           (entries 0, +1, -1)
    alignas(8) float Ti[N / 2][N];   // T^{-1}[l][j], l < N/2 (inverse of the bare integer T); pairs
                                     // (Ti[l][2m], Ti[l][2m+1]) are 8-byte aligned
    float Tih[N / 2][N];  // That^{-1}[l][j] = T^{-1}[l][j] / s_j
    float sij[N][N];      // s_i * s_j (B = sij o C), rounded once from FP64
    float s[N];           // s_i
    uint32_t T2[N][N / 2]; // T[i][j] as a packed pair of IEEE halves (both lanes equal)
    // JPEG-like quantiser of one call (filled per launch, zero in the plan):
    static constexpr int QN = N;
    float qw[QN][QN];      // fl32(s_i s_j / Q_ij): Bbar = floor(fl32(C qw) + 1/2)
    float qt[QN][QN];      // fl32(Q_ij / (s_i s_j)): the dequantised value in the C domain
    // Parseval form of a rounded plan whose T T^T is diagonal (N <= 8; zero otherwise).
    // With d_i = (T T^T)_ii, m = lcm(d_0 .. d_{N-1}) and e_i = m / d_i, T^{-1} =
    // T^T diag(1/d), so a block's error is sum a^2 - sum_retained C_ij^2 / (d_i d_j)
    // = (m^2 sum a^2 - sum_retained pw_ij C_ij^2) / m^2 with pw_ij = e_i e_j: integers.
    static constexpr int PN = N <= 8 ? N : 1;
    int32_t pw[PN][PN];
    int32_t pm2;           // m^2; 0 when the plan has no Parseval form
    float pinv;            // fl32(1 / m^2)
};

// Host-side plan object behind the opaque rklt_plan handle.
struct Plan {
    int N = 0;
    double rho = 0.0, alpha = 0.0;
    int orthogonal = 0;
    int kind = 0;                // 0 rounded KLT (integer T), 1 exact KLT, 2 DCT-II (real M)
    std::vector<double> M;       // N*N real analysis matrix (kinds 1, 2)
    std::vector<int8_t> T;       // N*N
    std::vector<double> s;       // N
    std::vector<double> Tinv;    // N*N, FP64 inverse of T
    std::vector<unsigned char> k; // bytes of PlanK<N>
    template <int M>
    const PlanK<M> &kparams() const { return *reinterpret_cast<const PlanK<M> *>(k.data()); }
};

// Geometry and outputs of one fused launch (kernel parameter).
struct FusedGeom {
    const uint8_t *img;          // source (plain-load mode)
    uint8_t *recon;              // 8-bit reconstruction (may be null)
    float *zcoef;                // compact coefficients (may be null)
    float *partials;             // one FP32 SSE partial per tile
    unsigned long long *sse_acc; // register path with a Parseval form: per-image error x m^2
    int64_t ld, img_stride;      // source pitch / image stride (bytes)
    int64_t ld_recon, recon_stride;
    int64_t ntiles;              // nimg * tiles_y * tiles_x
    int64_t blocks_per_img;      // (H/N) * (W/N)
    int H, W, nimg;
    int tiles_x, tiles_y;
    int step_img, step_ty, step_tx;  // the grid stride (tiles) in (image, tile row, tile column) form
    int r, D;                    // retained coefficients, diagonal bound
    int coef_vec4;               // r % 4 == 0 and zcoef 16-byte aligned (register path with a
                                 // Parseval form: widest coefficient store, 4, 2 or 1 floats)
    int use_tma;                 // tiles move by TMA (else plain loads)
    int stages;                  // TMA ring depth
    int inject_stall;            // test hook: the producer issues no loads
    uint64_t timeout_ns;
};

// Validated arguments of a fused call.
struct FusedArgs {
    const uint8_t *img;
    int nimg, H, W;
    int64_t ld, img_stride;
    int r;
    float *zcoef;
    uint8_t *recon;
    int64_t ld_recon, recon_stride;
    double *sse;
    float *psnr;
    float *partials;   // caller-provided scratch, or null (library pool)
    int64_t scratch_cap;  // bytes available at partials (when not null)
    int engine;        // N = 32: tensor engine of this call (0 mma.sync, 1 tcgen05), decided once
    int force_plain;   // 1: plain loads even when TMA would apply
    const double *Q;   // N = 4, 8: JPEG-like quantiser (N*N, host); zcoef then holds int32 Bbar
};

rklt_status launch_fused_n4(const Plan &p, const FusedArgs &a, cudaStream_t st);
rklt_status launch_fused_n8(const Plan &p, const FusedArgs &a, cudaStream_t st);
rklt_status launch_fused_n16(const Plan &p, const FusedArgs &a, cudaStream_t st);
rklt_status launch_fused_n32(const Plan &p, const FusedArgs &a, cudaStream_t st);
// Register path with the error by Parseval's identity (rklt_reg_n{4,8}.cu): serves the
// call and returns its status, or returns RKLT_ERR_UNSUPPORTED without doing anything
// when the plan or r is outside its scope.
rklt_status launch_pars_n4(const Plan &p, const FusedArgs &a, cudaStream_t st);
rklt_status launch_pars_n8(const Plan &p, const FusedArgs &a, cudaStream_t st);
unsigned int take_status_n4();
unsigned int take_status_n8();
unsigned int take_status_n16();
unsigned int take_status_n32();
unsigned int take_status_split();
unsigned int take_status_reg_n4();
unsigned int take_status_reg_n8();
unsigned int take_status_reg_n8b();
unsigned int take_status_mssim();
unsigned int take_status_fm_n4();
unsigned int take_status_fm_n8();

// host helpers (rklt_host.cpp)
rklt_status fail(rklt_status st, const std::string &msg);
rklt_status cuda_fail(cudaError_t err, const char *what);
cudaMemPool_t scratch_pool();                 // per-device stream-ordered pool for library scratch
int sm_count(int dev);
int ensure_smem_attr(const void *kernel);     // opt in to 227 KB dynamic smem; returns the device
int occupancy(const void *kernel, int threads, size_t smem);  // resident CTAs per SM (cached per device)
// 3-D tensor map over nimg images of W x H bytes; swizzle128 selects the 128-byte
// swizzled shared-memory layout (box_w must then be 128).
bool make_map_u8(CUtensorMap *m, const void *base, int W, int H, int nimg, int64_t ld, int64_t stride,
                 int box_w, int box_h, bool swizzle128 = false);
int transport_mode();                         // 0 auto, 1 plain loads only
int tensor_engine();                          // N = 32, D <= 16: 0 mma.sync, 1 tcgen05 / TMEM
int inject_stall();                           // fault-injection hook for the bounded-wait test

// Largest zig-zag diagonal touched by the first r coefficients, plus one:
// every retained (i, j) has i + j < diag_bound(N, r).
int diag_bound(int N, int r);

// Whether the fused call for (N, D) runs the tensor-memory (tcgen05) kernel, and the
// rows per tile of the kernel it runs: 32-row strips for that kernel, 64-row tiles
// otherwise.  The fused call needs one SSE partial per tile.
// `engine` is the call's tensor engine (FusedArgs::engine), read once from the
// library setting when the call enters the C ABI, so that the size check of a
// caller-provided scratch array and the launch see the same kernel.
inline bool uses_tmem_kernel(const Plan &p, int D, int engine) {
    return p.kind == 0 && p.N == 32 && D <= 16 && engine == 1;
}
inline int fused_tile_rows(const Plan &p, int D, int engine) { return uses_tmem_kernel(p, D, engine) ? 32 : kTileH; }

// Frees the constant-memory plan slots the batch kernels gave `p` (rklt_batch.cu).
void plan_registry_release(const Plan *p);

// Device wait timeout (nanoseconds) for the next launches.
uint64_t wait_timeout_ns();

}  // namespace rklt

struct rklt_plan {
    rklt::Plan p;
};
