// rklt_sweep.cu -- PSNR for every zonal size r = 1..N*N in one pass (r-sweep).
//
// For a block with exact integer coefficients c_k = C[i_k][j_k] (zig-zag order k),
// keeping the first r coefficients leaves the error A - A' = T^{-1} E_r T^{-T},
// E_r = the discarded c_k.  Its energy is
//   SSE(r) = sum_{k,l >= r} c_k c_l G_kl,   G_kl = H[i_k][i_l] H[j_k][j_l],
//   H = (T T^T)^{-1},
// so SSE(r) = SSE(r+1) + c_r (c_r G_rr + 2 sum_{l>r} c_l G_rl), SSE(N*N) = 0.
// For a T with diagonal T T^T (Eq. 1's orthogonal branch) G is diagonal and this
// is Parseval on the normalised coefficients, SSE(r) = sum_{k>=r} B_k^2.  H has
// the parity structure of the KLT rows (H[a][b] = 0 when a + b is odd), so pairs
// with i_k + i_l or j_k + j_l odd are skipped at compile time.
//
// One CTA per (image, chunk of SWEEP_CHUNK blocks) and distinct T: each thread takes
// blocks of the chunk, keeps its N*N - 1 running sums in registers, and the CTA adds
// them in a fixed order (FP64); the chunks of an image are then summed in order, so
// each image's values do not depend on the rest of the batch.
#include <algorithm>
#include <vector>

#include "rklt_fused_impl.cuh"

namespace rklt {

// Zig-zag positions as compile-time tables (cheap for the compiler to fold).
template <int N>
struct ZZTab {
    int row[N * N], col[N * N];
    constexpr ZZTab() : row(), col() {
        for (int k = 0; k < N * N; k++) {
            row[k] = zz_row(N, k);
            col[k] = zz_col(N, k);
        }
    }
};
template <int N>
__device__ constexpr ZZTab<N> kZZ{};

// Zig-zag positions split by (row parity, column parity), ascending.  G_kl is zero
// unless k and l share both parities, so the Gram sums stay inside one class.
template <int N>
struct ZZClass {
    int idx[4][N * N / 4];
    constexpr ZZClass() : idx() {
        int n[4] = {0, 0, 0, 0};
        for (int k = 0; k < N * N; k++) {
            const int q = (zz_row(N, k) & 1) * 2 + (zz_col(N, k) & 1);
            idx[q][n[q]++] = k;
        }
    }
};
template <int N>
__device__ constexpr ZZClass<N> kCls{};

template <int N>
struct SweepK {
    uint32_t T2[N][N / 2];     // T as binary16 pairs (column pass)
    float T[N][N / 2];         // T (row pass)
    float G[N * N][N * N];     // Gram matrix in zig-zag order
    int orthogonal;
};

// Full C = T A T^T of a register block (exact), in zig-zag order.
template <int N>
__device__ __forceinline__ void block_forward_full(const SweepK<N> &P, const uint32_t (&w)[N][N / 4],
                                                   float (&c)[N * N]) {
    constexpr int H2 = N / 2, NP = N / 2;
    const __half2 k1024 = __float2half2_rn(1024.0f);
    auto px = [&](int k, int p) -> __half2 {
        return __hsub2(as_h2(bytes_to_biased_h2(w[k][p >> 1], (2 * p) & 3, (2 * p + 1) & 3)), k1024);
    };
    float Y[N][N];
#pragma unroll
    for (int p = 0; p < NP; p++) {
        __half2 sp[H2], dp[H2];
#pragma unroll
        for (int j = 0; j < H2; j++) {
            const __half2 top = px(j, p), bot = px(N - 1 - j, p);
            sp[j] = __hadd2(top, bot);
            dp[j] = __hsub2(top, bot);
        }
#pragma unroll
        for (int i = 0; i < N; i++) {
            __half2 acc = __hmul2(as_h2(P.T2[i][0]), (i & 1) ? dp[0] : sp[0]);
#pragma unroll
            for (int j = 1; j < H2; j++) acc = __hfma2(as_h2(P.T2[i][j]), (i & 1) ? dp[j] : sp[j], acc);
            Y[i][2 * p] = __low2float(acc);
            Y[i][2 * p + 1] = __high2float(acc);
        }
    }
#pragma unroll
    for (int i = 0; i < N; i++) {
        float s[H2], d[H2];
#pragma unroll
        for (int l = 0; l < H2; l++) {
            s[l] = Y[i][l] + Y[i][N - 1 - l];
            d[l] = Y[i][l] - Y[i][N - 1 - l];
        }
#pragma unroll
        for (int j = 0; j < N; j++) {
            float acc = 0.0f;
#pragma unroll
            for (int l = 0; l < H2; l++) acc = fmaf(P.T[j][l], (j & 1) ? d[l] : s[l], acc);
            c[zz_index(N, i, j)] = acc;
        }
    }
}

constexpr int SWEEP_CHUNK = 1024;  // blocks per CTA (4 per thread): short waves, a small tail

// grid: (nimg, nchunk), one launch per distinct T; block: 256 threads; dynamic smem:
// 8 warps * (N*N - 1) floats.  sse_out: [image][chunk][distinct T][N*N].
template <int N>
__global__ void __launch_bounds__(256, 1)
    sweep_kernel(const __grid_constant__ SweepK<N> P, const uint8_t *__restrict__ imgs, int H, int W, int64_t ld,
                 int64_t img_stride, int tslot, int ntslots, double *__restrict__ sse_out) {
    constexpr int K = N * N;
    extern __shared__ float red[];  // [warps][K - 1]
    const int img = blockIdx.x, chunk = blockIdx.y, nchunk = gridDim.y;
    const uint8_t *base = imgs + int64_t(img) * img_stride;
    const int bw = W / N, nblk = (H / N) * bw;
    const int b_end = min(nblk, (chunk + 1) * SWEEP_CHUNK);
    float acc[K - 1];
#pragma unroll
    for (int q = 0; q < K - 1; q++) acc[q] = 0.0f;
    for (int b = chunk * SWEEP_CHUNK + int(threadIdx.x); b < b_end; b += blockDim.x) {
        const int by = b / bw, bx = b - by * bw;
        uint32_t w[N][N / 4];
        load_block_words<N>(base + int64_t(by) * N * ld + bx * N, ld, w);
        float c[K];
        block_forward_full<N>(P, w, c);
        // v_k = c_k (c_k G_kk + 2 sum_{l > k} c_l G_kl), written over c_k: within a
        // class, member a reads only members b > a, so c_k is no longer needed once
        // its own v_k is formed (every index below is a compile-time constant)
        constexpr int M = K / 4;
        if (!P.orthogonal) {
#pragma unroll
            for (int q = 0; q < 4; q++) {
#pragma unroll
                for (int a = 0; a < M; a++) {
                    const int ka = kCls<N>.idx[q][a];
                    float t = 0.0f;
#pragma unroll
                    for (int b = a + 1; b < M; b++) {
                        const int kb = kCls<N>.idx[q][b];
                        t = fmaf(c[kb], P.G[ka][kb], t);
                    }
                    c[ka] = c[ka] * fmaf(c[ka], P.G[ka][ka], 2.0f * t);
                }
            }
        } else {
#pragma unroll
            for (int k = 0; k < K; k++) c[k] = c[k] * (c[k] * P.G[k][k]);
        }
        float run = 0.0f;  // SSE(r) for the current r, from r = K - 1 down to 1
#pragma unroll
        for (int rr = K - 1; rr >= 1; rr--) {
            run += c[rr];
            acc[rr - 1] += run;  // keep the first rr coefficients
        }
    }
    // per warp: a fixed xor-butterfly in FP32; then the warps in order in FP64
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
#pragma unroll
    for (int q = 0; q < K - 1; q++) {
        float v = acc[q];
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
        if (lane == 0) red[warp * (K - 1) + q] = v;
    }
    __syncthreads();
    for (int q = threadIdx.x; q < K - 1; q += blockDim.x) {
        double s = 0.0;
        for (int t = 0; t < nwarp; t++) s += double(red[t * (K - 1) + q]);
        sse_out[((int64_t(img) * nchunk + chunk) * ntslots + tslot) * K + q] = s;
    }
    if (threadIdx.x == 0) sse_out[((int64_t(img) * nchunk + chunk) * ntslots + tslot) * K + (K - 1)] = 0.0;  // r = N*N
}

// Scatter per-distinct-T SSE to the callers' [image][plan][r] layout with PSNR.
__global__ void sweep_scatter(const double *__restrict__ sse_t, int nimg, int nchunk, int ntslots,
                              const int *__restrict__ slot_of, int nplans, int K, int64_t npx, double *sse, float *psnr) {
    const int64_t total = int64_t(nimg) * nplans * K;
    for (int64_t q = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; q < total; q += int64_t(gridDim.x) * blockDim.x) {
        const int r = int(q % K);
        const int64_t ip = q / K;
        const int p = int(ip % nplans), img = int(ip / nplans);
        double s = 0.0;  // the image's chunks in order
        for (int c = 0; c < nchunk; c++) s += sse_t[((int64_t(img) * nchunk + c) * ntslots + slot_of[p]) * K + r];
        if (sse) sse[q] = s;
        float v;
        if (npx == 0) v = __int_as_float(0x7fc00000);
        else if (s <= 0.0) v = __int_as_float(0x7f800000);
        else v = float(10.0 * log10(255.0 * 255.0 * double(npx) / s));
        psnr[q] = v;
    }
}

namespace {

template <int N>
void fill_sweep(const Plan &p, std::vector<unsigned char> &blob) {
    blob.assign(sizeof(SweepK<N>), 0);
    SweepK<N> &k = *reinterpret_cast<SweepK<N> *>(blob.data());
    const PlanK<N> &pk = p.kparams<N>();
    for (int i = 0; i < N; i++)
        for (int j = 0; j < N / 2; j++) {
            k.T2[i][j] = pk.T2[i][j];
            k.T[i][j] = pk.T[i][j];
        }
    // H = (T T^T)^{-1} = T^{-T} T^{-1}
    double Hm[N][N];
    for (int a = 0; a < N; a++)
        for (int b = 0; b < N; b++) {
            double acc = 0.0;
            for (int m = 0; m < N; m++) acc += p.Tinv[size_t(m) * N + a] * p.Tinv[size_t(m) * N + b];
            Hm[a][b] = acc;
        }
    for (int kk = 0; kk < N * N; kk++)
        for (int ll = 0; ll < N * N; ll++)
            k.G[kk][ll] = float(Hm[zz_row(N, kk)][zz_row(N, ll)] * Hm[zz_col(N, kk)][zz_col(N, ll)]);
    k.orthogonal = p.orthogonal;
}

template <int N>
rklt_status launch_sweep(const std::vector<const Plan *> &distinct, const std::vector<int> &slot_of,
                         const uint8_t *d_imgs, int nimg, int H, int W, int64_t ld, int64_t istride, double *d_sse,
                         float *d_psnr, cudaStream_t st) {
    constexpr int K = N * N;
    const int nt = int(distinct.size());
    cudaMemPool_t pool = scratch_pool();
    if (!pool) return fail(RKLT_ERR_CUDA, "could not create the scratch memory pool");
    const int nblk = (H / N) * (W / N);
    const int nchunk = std::max(1, (nblk + SWEEP_CHUNK - 1) / SWEEP_CHUNK);
    const size_t tb = size_t(nimg) * nchunk * nt * K * sizeof(double);
    const size_t sb = slot_of.size() * sizeof(int);
    void *scratch = nullptr;
    if (cudaMallocFromPoolAsync(&scratch, tb + sb, pool, st) != cudaSuccess)
        return fail(RKLT_ERR_OOM, "scratch allocation failed");
    double *sse_t = static_cast<double *>(scratch);
    int *d_slot = reinterpret_cast<int *>(static_cast<char *>(scratch) + tb);
    cudaError_t e = cudaMemcpyAsync(d_slot, slot_of.data(), sb, cudaMemcpyHostToDevice, st);
    const int threads = 256;
    const size_t smem = size_t(threads / 32) * (K - 1) * sizeof(float);
    static std::once_flag once;
    std::call_once(once, [] {
        cudaFuncSetAttribute(sweep_kernel<N>, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
    });
    std::vector<unsigned char> blob;
    for (int t = 0; t < nt && e == cudaSuccess; t++) {
        fill_sweep<N>(*distinct[t], blob);
        sweep_kernel<N><<<dim3(nimg, nchunk), threads, smem, st>>>(*reinterpret_cast<const SweepK<N> *>(blob.data()),
                                                                   d_imgs, H, W, ld, istride, t, nt, sse_t);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) {
        const int64_t total = int64_t(nimg) * slot_of.size() * K;
        const unsigned grid = unsigned(std::min<int64_t>((total + 255) / 256, 4096));
        sweep_scatter<<<grid, 256, 0, st>>>(sse_t, nimg, nchunk, nt, d_slot, int(slot_of.size()), K, int64_t(H) * W,
                                            d_sse, d_psnr);
        e = cudaGetLastError();
    }
    cudaFreeAsync(scratch, st);
    return e == cudaSuccess ? RKLT_OK : cuda_fail(e, "sweep launch");
}

}  // namespace
}  // namespace rklt

using namespace rklt;

extern "C" rklt_status rklt_rsweep(const rklt_plan *const *plans, int nplans, const uint8_t *d_imgs, int nimg, int H,
                                   int W, int64_t ld, int64_t img_stride, double *d_sse, float *d_psnr,
                                   void *stream) {
    if (!plans || nplans < 1) return fail(RKLT_ERR_ARG, "need at least one plan");
    if (!d_psnr) return fail(RKLT_ERR_ARG, "d_psnr is required");
    if (nimg < 1 || nimg > 2147483647) return fail(RKLT_ERR_ARG, "nimg must be >= 1");
    int N = 0;
    for (int p = 0; p < nplans; p++) {
        if (!plans[p]) return fail(RKLT_ERR_ARG, "NULL plan");
        if (plans[p]->p.kind != 0) return fail(RKLT_ERR_UNSUPPORTED, "the r-sweep needs rounded (integer) plans");
        if (N == 0) N = plans[p]->p.N;
        if (plans[p]->p.N != N) return fail(RKLT_ERR_ARG, "all plans must share N");
    }
    if (N != 4 && N != 8) return fail(RKLT_ERR_UNSUPPORTED, "the r-sweep supports N = 4 and N = 8");
    if (H < 0 || W < 0 || H % N || W % N) return fail(RKLT_ERR_SHAPE, "H and W must be non-negative multiples of N");
    if (ld < W) return fail(RKLT_ERR_SHAPE, "ld must be >= W");
    if (nimg > 1 && img_stride < ld * int64_t(H)) return fail(RKLT_ERR_SHAPE, "img_stride smaller than one image");
    if (H > 0 && W > 0 && !d_imgs) return fail(RKLT_ERR_ARG, "d_imgs is NULL");
    const uintptr_t amask = N == 8 ? 7 : 3;
    if ((reinterpret_cast<uintptr_t>(d_imgs) | uintptr_t(ld) | uintptr_t(nimg > 1 ? img_stride : 0)) & amask)
        return fail(RKLT_ERR_UNSUPPORTED, "image rows must be N-byte aligned");
    // plans with the same integer matrix are computed once
    std::vector<const Plan *> distinct;
    std::vector<int> slot_of(nplans);
    for (int p = 0; p < nplans; p++) {
        int found = -1;
        for (size_t t = 0; t < distinct.size(); t++)
            if (distinct[t]->T == plans[p]->p.T) found = int(t);
        if (found < 0) {
            found = int(distinct.size());
            distinct.push_back(&plans[p]->p);
        }
        slot_of[p] = found;
    }
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    return N == 4 ? launch_sweep<4>(distinct, slot_of, d_imgs, nimg, H, W, ld, img_stride, d_sse, d_psnr, st)
                  : launch_sweep<8>(distinct, slot_of, d_imgs, nimg, H, W, ld, img_stride, d_sse, d_psnr, st);
}
