// rklt_umma.cuh -- 32 x 32 blocks with retained support inside i + j < 16 on the
// fifth-generation tensor cores: tcgen05.mma with accumulators in tensor memory
// (TMEM), operands staged in shared memory, one elected thread per warp group
// issuing the MMAs.  Included by rklt_fused_n32.cu after rklt_fused_impl.cuh.
//
// Work unit: a strip of 32 rows x 256 columns = 8 blocks b = 0..7 (tile), handled by
// one warp group of 128 threads; thread (q, l) = (warp in group, lane) owns TMEM lane
// 32q + l.  The chain (Sec. 4.1: C = T A T^T, zonal mask, A' = T^{-1} C' T^{-T}):
//
//   S0  pixels of blocks q and 4 + q, row l, as binary16 (biased by 1024) into the
//       F1 A operand (K-major, rows (b, y), K = x)
//   F1  D1[(b, y)][j] = sum_x A[b][y][x] T[j][x]          M = 128 (4 blocks), N = 16, K = 32
//   S1  D1 rows -> two binary16 digits of Z^T into the F2 A operand (MN-major:
//       column y, rows (b, j))
//   F2  D2[(b, j)][i] = sum_y Z[b][y][j] 2^-12 T[i][y]     M = 128 (8 blocks), N = 16, K = 32
//   S2  bias removed, coefficients s_i s_j C staged in zig-zag order, zonal mask,
//       C' as two digits into the I1 A operand (K-major, rows (b, j), K = i)
//   I1  D3[(b, j)][y'] = sum_i C'[b][i][j] 2^6 T^{-1}[y'][i]   M = 128, N = 32, K = 16, 3 products
//   S3  D3 rows -> two digits of Y into the I2 A operand (MN-major: column j,
//       rows (b, y'))
//   I2  D4[(b, y')][x'] = sum_j Y[b][y'][j] 2^6 T^{-1}[x'][j]  M = 128 (4 blocks), N = 32, K = 16
//   S4  error against the pixels, SSE, 8-bit output clip(floor(A' + 1/2)) in place
//
// Exactness is the same argument as the warp-level path (rklt_tc.cuh): pixels and T
// are exact in binary16, D1 holds integers below 2^16 (the 1024 bias included), its
// two digits sum to it exactly, F2's partial sums are multiples of 2^-12 below 2^9,
// and the bias term 1024 (sum_x T[j][x]) (sum_y T[i][y]) is subtracted exactly in
// FP32; C is exact.  The inverse runs on two digits of each operand (three products).
//
// Shared-memory operand layouts are the canonical no-swizzle ("interleaved") ones:
// 8-row x 16-byte core matrices.  K-major: element (row, k) at (row / 8) SBO +
// (k / 8) LBO + (row % 8) 16 + (k % 8) 2.  MN-major: element (row, k) at (row / 8) SBO
// + (k / 8) LBO + (k % 8) 16 + (row % 8) 2.
#pragma once

namespace rklt {

constexpr int U_WG = 3;                       // warp groups (pipelines) per CTA
constexpr int U_NCONS = 128 * U_WG;           // consumer threads
constexpr int U_TH = 32;                      // strip height
constexpr int U_TILE = U_TH * TW;             // 8 KB: two 128 x 32 swizzled halves
constexpr int U_HALF = U_TH * 128;
constexpr int U_STAGES = 6;                   // TMA ring depth
constexpr int U_TCOL = 160;                   // TMEM columns per warp group
constexpr int U_ZS = 8 * 136 + 4;             // coefficient staging floats per group

// Per-group shared buffers (bytes)
constexpr int U_A1 = 16384;   // F1 A (2 chunks x 8 KB), reused as I2 A (2 chunks x 2 digits x 4 KB)
constexpr int U_A2 = 16384;   // F2 A, 2 digits x 8 KB
constexpr int U_A3 = 8192;    // I1 A, 2 digits x 4 KB
constexpr int U_GROUP_BYTES = U_A1 + U_A2 + U_A3;
// Constant operands (bytes): F1 B (T), F2 B (2^-12 T), I B hi / lo (2^6 T^{-1})
constexpr int U_CONST_BYTES = 4 * 1024;

// Byte offset of pixel (y, x) in a strip held as two 32 x 128 halves in the 128-byte
// swizzled layout of a TMA copy.
__host__ __device__ constexpr int u_pix_off(int y, int x) {
    return (x >> 7) * U_HALF + y * 128 + ((((x & 127) >> 4) ^ (y & 7)) << 4) + (x & 15);
}

struct UmmaLayout {
    int ring, bar, red, cst, grp, zs, total;
};

__host__ __device__ inline UmmaLayout umma_layout(int stages) {
    UmmaLayout L{};
    L.ring = 0;
    L.bar = stages * U_TILE;                            // full[ST], empty[ST], mma[U_WG], tmem slot
    L.red = L.bar + 8 * (2 * U_STAGES + U_WG) + 16;     // per-slot SSE of the strip; per-warp partials
    L.cst = ((L.red + 4 * (U_STAGES + U_NCONS / 32) + 1023) / 1024) * 1024;
    L.grp = L.cst + U_CONST_BYTES;
    L.zs = L.grp + U_WG * U_GROUP_BYTES;
    L.total = L.zs + U_WG * U_ZS * 4 + 1024;
    return L;
}

// ---------------------------------------------------------------------------
// tcgen05 wrappers
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint64_t u_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
    // start >> 4 | LBO >> 4 << 16 | SBO >> 4 << 32 | version 1 << 46 | no swizzle
    return uint64_t((addr >> 4) & 0x3FFFu) | (uint64_t((lbo >> 4) & 0x3FFFu) << 16) |
           (uint64_t((sbo >> 4) & 0x3FFFu) << 32) | (uint64_t(1) << 46);
}

// Instruction descriptor, kind::f16: fp16 A and B, fp32 accumulator, M = 128.
__host__ __device__ constexpr uint32_t u_idesc(int n, bool a_mn_major) {
    return (1u << 4) | (uint32_t(a_mn_major) << 15) | (uint32_t(n >> 3) << 17) | (uint32_t(128 >> 4) << 24);
}

__device__ __forceinline__ void u_mma(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc, bool accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
        "l"(a), "l"(b), "r"(idesc), "r"(uint32_t(accumulate))
        : "memory");
}

__device__ __forceinline__ void u_commit(uint64_t *bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
                 : "memory");
}

__device__ __forceinline__ void u_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void u_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// 16 consecutive FP32 columns of this thread's TMEM lane.  The registers pass through
// the wait as operands, so no use of them can be scheduled before the load completes.
__device__ __forceinline__ void u_ld16(uint32_t taddr, float (&v)[16]) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;"
                 : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5]), "+r"(r[6]), "+r"(r[7]),
                   "+r"(r[8]), "+r"(r[9]), "+r"(r[10]), "+r"(r[11]), "+r"(r[12]), "+r"(r[13]), "+r"(r[14]),
                   "+r"(r[15])
                 :
                 : "memory");
#pragma unroll
    for (int k = 0; k < 16; k++) v[k] = __uint_as_float(r[k]);
}

__device__ __forceinline__ void sts128(uint32_t a, uint32_t x, uint32_t y, uint32_t z, uint32_t w) {
    asm volatile("st.shared.v4.u32 [%0], {%1,%2,%3,%4};" ::"r"(a), "r"(x), "r"(y), "r"(z), "r"(w));
}

// Eight FP32 values as two binary16 digits (hi, lo), packed in pairs.
__device__ __forceinline__ void split8(const float *v, uint32_t (&h)[4], uint32_t (&l)[4]) {
#pragma unroll
    for (int p = 0; p < 4; p++) split_pair(v[2 * p], v[2 * p + 1], h[p], l[p]);
}

// ---------------------------------------------------------------------------
// Per-thread constants (its j for the F2/I1 rows it owns)
// ---------------------------------------------------------------------------
struct UmmaThread {
    float corr[16];   // 2^-12 * 1024 (sum_x T[j][x]) (sum_y T[i][y]), i = 0..15
    float bs[16];     // 2^12 s_i s_j
    int zp[16];       // zig-zag position of (i, j), or -1 if not retained
};

__device__ inline void umma_setup_thread(const PlanK<32> &P, UmmaThread &u, int j, int r) {
    float rs_j = 0.0f;
    for (int x = 0; x < 32; x++) rs_j += tc_T(P, j, x);
#pragma unroll
    for (int i = 0; i < 16; i++) {
        float rs_i = 0.0f;
        for (int x = 0; x < 32; x++) rs_i += tc_T(P, i, x);
        u.corr[i] = (1024.0f * rs_j * rs_i) * (1.0f / 4096.0f);
        u.bs[i] = 4096.0f * P.sij[i][j];
        const int z = zz_index(32, i, j);
        u.zp[i] = z < r ? z : -1;
    }
}

// Constant operands in shared memory (K-major, no swizzle), written by all consumers.
//   cst + 0     F1 B: T[j][x], rows j < 16, K = x < 32         (LBO 128, SBO 512)
//   cst + 1024  F2 B: 2^-12 T[i][y], rows i < 16, K = y < 32   (LBO 128, SBO 512)
//   cst + 2048  I  B hi: 2^6 T^{-1}[l][c], rows l < 32, K = c < 16  (LBO 128, SBO 256)
//   cst + 3072  I  B lo
__device__ inline void umma_setup_consts(const PlanK<32> &P, uint8_t *cst, int tid, int nthreads) {
    for (int e = tid; e < 16 * 32; e += nthreads) {
        const int row = e / 32, k = e % 32;
        const int off = (row / 8) * 512 + (k / 8) * 128 + (row % 8) * 16 + (k % 8) * 2;
        *reinterpret_cast<__half *>(cst + off) = __float2half_rn(tc_T(P, row, k));
        *reinterpret_cast<__half *>(cst + 1024 + off) = __float2half_rn(tc_T(P, row, k) * (1.0f / 4096.0f));
    }
    for (int e = tid; e < 32 * 16; e += nthreads) {
        const int l = e / 16, c = e % 16;
        // T^{-1}[l][c] for l >= 16 by the parity T^{-1}[31-l][c] = (-1)^c T^{-1}[l][c]
        const float ti = l < 16 ? P.Ti[l][c] : ((c & 1) ? -P.Ti[31 - l][c] : P.Ti[31 - l][c]);
        const float v = 64.0f * ti;
        const __half h = __float2half_rn(v);
        const int off = (l / 8) * 256 + (c / 8) * 128 + (l % 8) * 16 + (c % 8) * 2;
        *reinterpret_cast<__half *>(cst + 2048 + off) = h;
        *reinterpret_cast<__half *>(cst + 3072 + off) = __float2half_rn(v - __half2float(h));
    }
}

// ---------------------------------------------------------------------------
// One strip (8 blocks) by one warp group.  Returns the thread's SSE share.
// ---------------------------------------------------------------------------
struct UmmaCtx {
    uint32_t cst;      // shared-window address of the constant operands
    uint32_t a1, a2, a3;
    uint32_t zs;       // staging buffer (shared window)
    float *zs_ptr;
    uint32_t tmem;     // TMEM address of the group's first column, lane 0
    uint64_t *mbar;
    int q, l, gtid, wg;
};

// Waits for the group's MMA barrier phase.  The group decides together (barrier with
// an OR vote) whether any thread gave up, so no thread is left waiting at a later
// barrier for threads that returned.
__device__ __forceinline__ bool u_wait_mma(const UmmaCtx &x, uint32_t &phase, uint64_t timeout_ns) {
    const bool got = mbar_wait_poll(x.mbar, phase, timeout_ns);
    phase ^= 1u;
    const bool fail = named_any(1 + x.wg, 128, !got);
    u_fence_after();
    return !fail;
}

__device__ __forceinline__ void u_group_sync(const UmmaCtx &x) { named_sync(1 + x.wg, 128); }

__device__ __forceinline__ float umma_strip(const UmmaCtx &x, const UmmaThread &u, uint8_t *tile, int nb_in, int r,
                                            float *zg, bool recon, bool vec4, uint32_t &phase, uint64_t timeout_ns,
                                            bool &ok) {
    const int q = x.q, l = x.l;
    const uint32_t t32 = smem_u32(tile);
    const bool leader = x.gtid == 0;
    const uint32_t lane_base = x.tmem + (uint32_t(32 * q) << 16);
    constexpr uint32_t C_D1 = 0, C_D2 = 32, C_D3 = 48, C_D4 = 80;

    // ---- S0: pixel rows (blocks q and 4 + q, row l) -> F1 A (binary16, biased)
#pragma unroll
    for (int c = 0; c < 2; c++) {
        const int b = 4 * c + q;
        const uint32_t src = t32 + u_pix_off(l, 32 * b);
        const uint4 w0 = lds128(src);
        const uint4 w1 = lds128(t32 + u_pix_off(l, 32 * b + 16));
        const int m = 32 * q + l;  // row in chunk c
        const uint32_t dst = x.a1 + 8192 * c + (m / 8) * 512 + (m % 8) * 16;
        const uint32_t ws[8] = {w0.x, w0.y, w0.z, w0.w, w1.x, w1.y, w1.z, w1.w};
#pragma unroll
        for (int kb = 0; kb < 4; kb++)  // 8 pixels per core-matrix row
            sts128(dst + kb * 128, bytes_to_biased_h2(ws[2 * kb], 0, 1), bytes_to_biased_h2(ws[2 * kb], 2, 3),
                   bytes_to_biased_h2(ws[2 * kb + 1], 0, 1), bytes_to_biased_h2(ws[2 * kb + 1], 2, 3));
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    u_fence_before();
    u_group_sync(x);
    if (leader) {
        u_fence_after();
        constexpr uint32_t id = u_idesc(16, false);
#pragma unroll
        for (int c = 0; c < 2; c++)
#pragma unroll
            for (int ks = 0; ks < 2; ks++)
                u_mma(x.tmem + C_D1 + 16 * c, u_desc(x.a1 + 8192 * c + 256 * ks, 128, 512),
                      u_desc(x.cst + 256 * ks, 128, 512), id, ks > 0);
        u_commit(x.mbar);
    }
    if (!(ok = u_wait_mma(x, phase, timeout_ns))) return 0.0f;

    // ---- S1: D1 rows (b, y = l) -> digits of Z^T into F2 A (MN-major, rows (b, j), K = y)
#pragma unroll
    for (int c = 0; c < 2; c++) {
        const int b = 4 * c + q;
        float v[16];
        u_ld16(lane_base + C_D1 + 16 * c, v);
        uint32_t h[2][4], lo[2][4];
        split8(v, h[0], lo[0]);
        split8(v + 8, h[1], lo[1]);
#pragma unroll
        for (int jh = 0; jh < 2; jh++) {
            const uint32_t off = (2 * b + jh) * 128 + (l / 8) * 2048 + (l % 8) * 16;
            sts128(x.a2 + off, h[jh][0], h[jh][1], h[jh][2], h[jh][3]);
            sts128(x.a2 + 8192 + off, lo[jh][0], lo[jh][1], lo[jh][2], lo[jh][3]);
        }
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    u_fence_before();
    u_group_sync(x);
    if (leader) {
        u_fence_after();
        constexpr uint32_t id = u_idesc(16, true);
#pragma unroll
        for (int d = 0; d < 2; d++)
#pragma unroll
            for (int ks = 0; ks < 2; ks++)
                u_mma(x.tmem + C_D2, u_desc(x.a2 + 8192 * d + 4096 * ks, 2048, 128),
                      u_desc(x.cst + 1024 + 256 * ks, 128, 512), id, d > 0 || ks > 0);
        u_commit(x.mbar);
    }
    if (!(ok = u_wait_mma(x, phase, timeout_ns))) return 0.0f;

    // ---- S2: thread owns D2 row (b, j): b = 2q + l / 16, j = l % 16
    {
        const int b = 2 * q + (l >> 4);
        float v[16];
        u_ld16(lane_base + C_D2, v);
#pragma unroll
        for (int i = 0; i < 16; i++) v[i] -= u.corr[i];  // exact: C * 2^-12
        if (zg) {
            const uint32_t zb = x.zs + 4 * (b * r);
#pragma unroll
            for (int i = 0; i < 16; i++)
                if (u.zp[i] >= 0) sts_f32(zb + 4 * u.zp[i], u.bs[i] * v[i]);
        }
#pragma unroll
        for (int i = 0; i < 16; i++) v[i] = u.zp[i] >= 0 ? v[i] : 0.0f;
        uint32_t h[2][4], lo[2][4];
        split8(v, h[0], lo[0]);
        split8(v + 8, h[1], lo[1]);
        const int m = 16 * b + (l & 15);
#pragma unroll
        for (int ih = 0; ih < 2; ih++) {
            const uint32_t off = (m / 8) * 256 + ih * 128 + (m % 8) * 16;
            sts128(x.a3 + off, h[ih][0], h[ih][1], h[ih][2], h[ih][3]);
            sts128(x.a3 + 4096 + off, lo[ih][0], lo[ih][1], lo[ih][2], lo[ih][3]);
        }
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    u_fence_before();
    u_group_sync(x);
    if (leader) {
        u_fence_after();
        constexpr uint32_t id = u_idesc(32, false);
        u_mma(x.tmem + C_D3, u_desc(x.a3, 128, 256), u_desc(x.cst + 2048, 128, 256), id, false);
        u_mma(x.tmem + C_D3, u_desc(x.a3 + 4096, 128, 256), u_desc(x.cst + 2048, 128, 256), id, true);
        u_mma(x.tmem + C_D3, u_desc(x.a3, 128, 256), u_desc(x.cst + 3072, 128, 256), id, true);
        u_commit(x.mbar);
    }
    // the staged coefficients are complete once every thread passed the barrier above
    if (zg) {
        const int n = nb_in * r;
        const float *src = x.zs_ptr;
        if (vec4) {
            for (int k = 4 * x.gtid; k < n; k += 4 * 128)
                *reinterpret_cast<float4 *>(zg + k) = *reinterpret_cast<const float4 *>(src + k);
        } else {
            for (int k = x.gtid; k < n; k += 128) zg[k] = src[k];
        }
    }
    if (!(ok = u_wait_mma(x, phase, timeout_ns))) return 0.0f;

    // ---- S3: thread owns D3 row (b, j) -> digits of Y into I2 A (MN-major, rows (b, y'), K = j)
    {
        const int b = 2 * q + (l >> 4), j = l & 15;
        const int c = b >> 2, bb = b & 3;
#pragma unroll
        for (int half = 0; half < 2; half++) {
            float v[16];
            u_ld16(lane_base + C_D3 + 16 * half, v);
            uint32_t h[2][4], lo[2][4];
            split8(v, h[0], lo[0]);
            split8(v + 8, h[1], lo[1]);
#pragma unroll
            for (int g8 = 0; g8 < 2; g8++) {
                const int m = 32 * bb + 16 * half + 8 * g8;   // rows y' of this 8-group
                const uint32_t off = (m / 8) * 128 + (j / 8) * 2048 + (j % 8) * 16;
                sts128(x.a1 + 8192 * c + off, h[g8][0], h[g8][1], h[g8][2], h[g8][3]);
                sts128(x.a1 + 8192 * c + 4096 + off, lo[g8][0], lo[g8][1], lo[g8][2], lo[g8][3]);
            }
        }
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    u_fence_before();
    u_group_sync(x);
    if (leader) {
        u_fence_after();
        constexpr uint32_t id = u_idesc(32, true);
#pragma unroll
        for (int c = 0; c < 2; c++) {
            const uint32_t a = x.a1 + 8192 * c;
            u_mma(x.tmem + C_D4 + 32 * c, u_desc(a, 2048, 128), u_desc(x.cst + 2048, 128, 256), id, false);
            u_mma(x.tmem + C_D4 + 32 * c, u_desc(a + 4096, 2048, 128), u_desc(x.cst + 2048, 128, 256), id, true);
            u_mma(x.tmem + C_D4 + 32 * c, u_desc(a, 2048, 128), u_desc(x.cst + 3072, 128, 256), id, true);
        }
        u_commit(x.mbar);
    }
    if (!(ok = u_wait_mma(x, phase, timeout_ns))) return 0.0f;

    // ---- S4: rows (b = q, 4 + q; y = l): error, SSE, 8-bit output in place
    const __half2 k10235 = __float2half2_rn(1023.5f);
    const float2 half2f = make_float2(0.5f, 0.5f);
    float2 sse2 = make_float2(0.0f, 0.0f);
#pragma unroll
    for (int c = 0; c < 2; c++) {
        const int b = 4 * c + q;
        float a[32];
        u_ld16(lane_base + C_D4 + 32 * c, *reinterpret_cast<float(*)[16]>(a));
        u_ld16(lane_base + C_D4 + 32 * c + 16, *reinterpret_cast<float(*)[16]>(a + 16));
        const bool in = b < nb_in;
#pragma unroll
        for (int hh = 0; hh < 2; hh++) {
            const uint32_t pa = t32 + u_pix_off(l, 32 * b + 16 * hh);
            const uint4 w = lds128(pa);
            const uint32_t ws[4] = {w.x, w.y, w.z, w.w};
            uint32_t outw[4];
#pragma unroll
            for (int k = 0; k < 4; k++) {
                const float *av = a + 16 * hh + 4 * k;
                const float2 v01 = __fadd2_rn(make_float2(av[0], av[1]), half2f);
                const float2 v23 = __fadd2_rn(make_float2(av[2], av[3]), half2f);
                const __half2 p01 = __hsub2(as_h2(bytes_to_biased_h2(ws[k], 0, 1)), k10235);
                const __half2 p23 = __hsub2(as_h2(bytes_to_biased_h2(ws[k], 2, 3)), k10235);
                const float2 e01 = make_float2(sub_h_f(__low2half(p01), v01.x), sub_h_f(__high2half(p01), v01.y));
                const float2 e23 = make_float2(sub_h_f(__low2half(p23), v23.x), sub_h_f(__high2half(p23), v23.y));
                if (in) {
                    sse2 = __ffma2_rn(e01, e01, sse2);
                    sse2 = __ffma2_rn(e23, e23, sse2);
                }
                outw[k] = __byte_perm(__byte_perm(floor_sat_u8(v01.x), floor_sat_u8(v01.y), 0x0040),
                                      __byte_perm(floor_sat_u8(v23.x), floor_sat_u8(v23.y), 0x0040), 0x5410);
            }
            if (recon) sts128(pa, outw[0], outw[1], outw[2], outw[3]);
        }
    }
    u_fence_before();
    return sse2.x + sse2.y;
}

// ---------------------------------------------------------------------------
// The kernel: warp groups 0..U_WG-1 consume strips round-robin; the last warp
// produces (TMA mode).  One CTA per SM (it holds all 512 TMEM columns).
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(U_NCONS + 32, 1)
    umma32_kernel(const __grid_constant__ PlanK<32> P, const __grid_constant__ CUtensorMap tm_in,
                  const __grid_constant__ CUtensorMap tm_out, const FusedGeom g) {
    extern __shared__ uint8_t smem_raw[];
    uint8_t *smem = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    const int NST = g.stages;
    const UmmaLayout L = umma_layout(g.use_tma ? NST : U_WG);
    uint64_t *full = reinterpret_cast<uint64_t *>(smem + L.bar);
    uint64_t *empty = full + U_STAGES;
    uint64_t *mbar = empty + U_STAGES;
    uint32_t *tslot = reinterpret_cast<uint32_t *>(mbar + U_WG);
    float *red = reinterpret_cast<float *>(smem + L.red);   // [slot] strip SSE; then per-warp partials
    float *wred = red + U_STAGES;
    const int tid = threadIdx.x;

    if (tid == U_NCONS) {
        for (int s = 0; s < NST; s++) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        for (int w = 0; w < U_WG; w++) mbar_init(&mbar[w], 1);
        fence_mbar_init();
    }
    if (tid < 32) {  // warp 0 takes all of TMEM for the CTA
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tslot)),
                     "r"(512)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (tid < U_NCONS) umma_setup_consts(P, smem + L.cst, tid, U_NCONS);
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    u_fence_before();
    __syncthreads();
    u_fence_after();
    const uint32_t tmem_base = *tslot;

    if (tid >= U_NCONS) {
        // ---------------- producer: one elected lane ----------------
        if (!g.use_tma || tid != U_NCONS) return;
        int64_t it = 0;
        bool ok = true;
        TileWalker lw, sw;
        lw.init(g);
        sw = lw;
        for (int64_t tile = blockIdx.x; tile < g.ntiles; tile += gridDim.x, ++it) {
            const int s = int(it % NST);
            if (it >= NST) {
                if (!mbar_wait_bounded(&empty[s], uint32_t(((it / NST) - 1) & 1), g.timeout_ns)) {
                    ok = false;
                    break;
                }
                const int64_t prev = tile - int64_t(NST) * gridDim.x;
                g.partials[prev] = red[s];
                if (g.recon) {
                    const int x = sw.c.tx * TW, y = sw.c.ty * U_TH;
                    tma_store_3d(&tm_out, x, y, sw.c.img, smem + s * U_TILE);
                    if (x + TW / 2 < g.W) tma_store_3d(&tm_out, x + TW / 2, y, sw.c.img, smem + s * U_TILE + U_HALF);
                    bulk_commit();
                    bulk_wait_read_all();
                }
                sw.next(g);
            }
            if (g.inject_stall) continue;
            const int x = lw.c.tx * TW, y = lw.c.ty * U_TH, z = lw.c.img;
            lw.next(g);
            const bool two = x + TW / 2 < g.W;
            mbar_arrive_expect_tx(&full[s], two ? U_TILE : U_HALF);
            tma_load_3d(smem + s * U_TILE, &tm_in, x, y, z, &full[s]);
            if (two) tma_load_3d(smem + s * U_TILE + U_HALF, &tm_in, x + TW / 2, y, z, &full[s]);
        }
        const int64_t issued = it;
        for (int64_t j = issued > NST ? issued - NST : 0; j < issued; j++) {
            const int s = int(j % NST);
            const uint32_t par = uint32_t((j / NST) & 1);
            if (!ok || !mbar_wait_bounded(&empty[s], par, g.timeout_ns)) {
                ok = false;
                if (!g.inject_stall) mbar_wait_bounded(&full[s], par, DRAIN_NS);
                continue;
            }
            const int64_t tj = int64_t(blockIdx.x) + j * gridDim.x;
            g.partials[tj] = red[s];
            if (g.recon) {
                const int x = sw.c.tx * TW, y = sw.c.ty * U_TH;
                tma_store_3d(&tm_out, x, y, sw.c.img, smem + s * U_TILE);
                if (x + TW / 2 < g.W) tma_store_3d(&tm_out, x + TW / 2, y, sw.c.img, smem + s * U_TILE + U_HALF);
                bulk_commit();
            }
            sw.next(g);
        }
        bulk_wait_all();
        return;
    }

    // ---------------- consumers: warp group wg, thread gtid ----------------
    const int wg = tid >> 7, gtid = tid & 127;
    UmmaCtx x;
    x.wg = wg;
    x.gtid = gtid;
    x.q = gtid >> 5;
    x.l = gtid & 31;
    x.cst = smem_u32(smem + L.cst);
    x.a1 = smem_u32(smem + L.grp + wg * U_GROUP_BYTES);
    x.a2 = x.a1 + U_A1;
    x.a3 = x.a2 + U_A2;
    x.zs_ptr = reinterpret_cast<float *>(smem + L.zs) + wg * U_ZS;
    x.zs = smem_u32(x.zs_ptr);
    x.tmem = tmem_base + uint32_t(wg * U_TCOL);
    x.mbar = &mbar[wg];
    UmmaThread u;
    umma_setup_thread(P, u, x.l & 15, g.r);
    uint32_t phase = 0;
    const bool al8 = ((reinterpret_cast<uintptr_t>(g.img) | uintptr_t(g.ld) | uintptr_t(g.img_stride)) & 7) == 0;
    const bool al8o =
        ((reinterpret_cast<uintptr_t>(g.recon) | uintptr_t(g.ld_recon) | uintptr_t(g.recon_stride)) & 7) == 0;
    const int bw = g.W / 32;

    int64_t it = 0;
    TileWalker cw;
    cw.init(g);
    bool ok = true;
    for (int64_t tile = blockIdx.x; tile < g.ntiles; tile += gridDim.x, ++it, cw.next(g)) {
        if (int(it % U_WG) != wg) continue;
        uint8_t *buf;
        int s = 0;
        const int x0 = cw.c.tx * TW, y0 = cw.c.ty * U_TH, z = cw.c.img;
        const int wv = min(TW, g.W - x0);
        if (g.use_tma) {
            s = int(it % NST);
            const bool got = mbar_wait_bounded(&full[s], uint32_t((it / NST) & 1), g.timeout_ns);
            if (named_any(1 + wg, 128, !got)) break;
            buf = smem + s * U_TILE;
        } else {
            buf = smem + wg * U_TILE;  // this group's own slot
            const uint8_t *src = g.img + int64_t(z) * g.img_stride + int64_t(y0) * g.ld + x0;
            for (int qq = gtid; qq < U_TH * (TW / 8); qq += 128) {
                const int y = qq / (TW / 8), xx = (qq - y * (TW / 8)) * 8;
                uint2 v = make_uint2(0u, 0u);
                if (xx + 8 <= wv && al8) {
                    v = *reinterpret_cast<const uint2 *>(src + int64_t(y) * g.ld + xx);
                } else {
                    for (int e = 0; e < 8 && xx + e < wv; e++) {
                        const uint32_t bt = src[int64_t(y) * g.ld + xx + e];
                        if (e < 4) v.x |= bt << (8 * e);
                        else v.y |= bt << (8 * (e - 4));
                    }
                }
                *reinterpret_cast<uint2 *>(buf + u_pix_off(y, xx)) = v;
            }
            u_group_sync(x);
        }
        const int nb_in = min(TW / 32, bw - cw.c.tx * (TW / 32));
        float *zg = g.zcoef ? g.zcoef + (int64_t(z) * g.blocks_per_img + int64_t(cw.c.ty) * bw + cw.c.tx * (TW / 32)) *
                                            g.r
                            : nullptr;
        float v = umma_strip(x, u, buf, nb_in, g.r, zg, g.recon != nullptr, g.coef_vec4 != 0, phase, g.timeout_ns, ok);
        if (!ok) break;
        // group SSE in a fixed order: warp sums, then the four warps
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
        if (x.l == 0) wred[tid >> 5] = v;
        if (g.recon) asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        u_group_sync(x);
        if (gtid == 0) {
            const float t = wred[4 * wg] + wred[4 * wg + 1] + wred[4 * wg + 2] + wred[4 * wg + 3];
            if (g.use_tma) {
                red[s] = t;
                mbar_arrive(&empty[s]);
            } else {
                g.partials[tile] = t;
            }
        }
        if (!g.use_tma && g.recon) {
            uint8_t *dst = g.recon + int64_t(z) * g.recon_stride + int64_t(y0) * g.ld_recon + x0;
            for (int qq = gtid; qq < U_TH * (TW / 8); qq += 128) {
                const int y = qq / (TW / 8), xx = (qq - y * (TW / 8)) * 8;
                const uint2 vv = *reinterpret_cast<const uint2 *>(buf + u_pix_off(y, xx));
                if (xx + 8 <= wv && al8o) {
                    *reinterpret_cast<uint2 *>(dst + int64_t(y) * g.ld_recon + xx) = vv;
                } else {
                    for (int e = 0; e < 8 && xx + e < wv; e++)
                        dst[int64_t(y) * g.ld_recon + xx + e] = uint8_t((e < 4 ? vv.x >> (8 * e) : vv.y >> (8 * (e - 4))) & 0xffu);
                }
            }
        }
        if (!g.use_tma) u_group_sync(x);  // the slot is reused by this group's next strip
    }
    // all groups done with TMEM before warp 0 frees it
    u_fence_before();
    named_sync(5, U_NCONS);
    u_fence_after();
    if (tid < 32)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem_base), "r"(512) : "memory");
}


// Host launcher for N = 32 with D <= 16 (arguments validated by the C ABI layer).
inline rklt_status launch_umma32(const Plan &plan, const FusedArgs &a, cudaStream_t st) {
    constexpr int N = 32;
    FusedGeom g{};
    g.img = a.img;
    g.recon = a.recon;
    g.zcoef = a.zcoef;
    g.ld = a.ld;
    g.img_stride = a.nimg > 1 ? a.img_stride : a.ld * int64_t(a.H);
    g.ld_recon = a.ld_recon;
    g.recon_stride = a.nimg > 1 ? a.recon_stride : a.ld_recon * int64_t(a.H);
    g.H = a.H;
    g.W = a.W;
    g.nimg = a.nimg;
    g.tiles_x = (a.W + TW - 1) / TW;
    g.tiles_y = (a.H + U_TH - 1) / U_TH;
    g.ntiles = int64_t(g.tiles_x) * g.tiles_y * a.nimg;
    g.blocks_per_img = int64_t(a.H / N) * (a.W / N);
    g.r = a.r;
    g.D = diag_bound(N, a.r);
    g.coef_vec4 = (a.r % 4 == 0) && ((reinterpret_cast<uintptr_t>(a.zcoef) & 15) == 0);
    g.timeout_ns = wait_timeout_ns();
    g.inject_stall = inject_stall();
    const int64_t tiles_per_img = int64_t(g.tiles_x) * g.tiles_y;

    void *scratch = nullptr;
    if (a.partials) {
        if (g.ntiles * int64_t(sizeof(float)) > a.scratch_cap)
            return fail(RKLT_ERR_ARG, "scratch array too small for this call");
        g.partials = a.partials;
    } else {
        cudaMemPool_t pool = scratch_pool();
        if (!pool) return fail(RKLT_ERR_CUDA, "could not create the scratch memory pool");
        if (cudaMallocFromPoolAsync(&scratch, size_t(g.ntiles) * sizeof(float), pool, st) != cudaSuccess)
            return fail(RKLT_ERR_OOM, "scratch allocation failed");
        g.partials = static_cast<float *>(scratch);
    }
    const auto is16 = [](const void *p, int64_t x, int64_t y) {
        return ((reinterpret_cast<uintptr_t>(p) | uintptr_t(x) | uintptr_t(y)) & 15) == 0;
    };
    bool tma = !a.force_plain && is16(a.img, a.ld, g.img_stride) &&
               (!a.recon || is16(a.recon, a.ld_recon, g.recon_stride));
    CUtensorMap tin{}, tout{};
    if (tma) {
        tma = make_map_u8(&tin, a.img, a.W, a.H, a.nimg, a.ld, g.img_stride, TW / 2, U_TH, true);
        if (tma && a.recon)
            tma = make_map_u8(&tout, a.recon, a.W, a.H, a.nimg, a.ld_recon, g.recon_stride, TW / 2, U_TH, true);
        if (tma && !a.recon) tout = tin;
    }
    g.use_tma = tma ? 1 : 0;
    g.stages = U_STAGES;
    const UmmaLayout L = umma_layout(tma ? U_STAGES : U_WG);
    const void *fn = reinterpret_cast<const void *>(umma32_kernel);
    const int dev = ensure_smem_attr(fn);
    const int64_t grid = std::min<int64_t>(g.ntiles, int64_t(sm_count(dev)));  // one CTA per SM (all of TMEM)
    {
        const int64_t per_img = tiles_per_img;
        g.step_img = int(grid / per_img);
        const int rem = int(grid - int64_t(g.step_img) * per_img);
        g.step_ty = rem / g.tiles_x;
        g.step_tx = rem - g.step_ty * g.tiles_x;
    }
    {
        const PlanK<N> &pk = plan.kparams<N>();
        void *args[] = {const_cast<PlanK<N> *>(&pk), &tin, &tout, &g};
        const cudaError_t le =
            cudaLaunchKernel(fn, dim3(unsigned(grid)), dim3(U_NCONS + 32), args, L.total, st);
        if (le != cudaSuccess) {
            if (scratch) cudaFreeAsync(scratch, st);
            return cuda_fail(le, "tensor-memory kernel launch");
        }
    }
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) {
        finalize_kernel<<<a.nimg, 256, 0, st>>>(g.partials, tiles_per_img, a.nimg, a.H, a.W, a.sse, a.psnr);
        e = cudaGetLastError();
    }
    if (scratch) cudaFreeAsync(scratch, st);
    return e == cudaSuccess ? RKLT_OK : cuda_fail(e, "tensor-memory kernel launch");
}

}  // namespace rklt
