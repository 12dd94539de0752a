// rklt_device.cuh -- device helpers shared by the library's kernels: TMA and
// mbarrier PTX wrappers, bounded waits, the zig-zag walk, the latched device
// error word, and byte/float conversions.
#pragma once

#include <cuda.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <cstdint>
#include <cstring>

namespace rklt {

// Latched device-side status (RKLT_OK or RKLT_ERR_TIMEOUT).  Without relocatable
// device code every translation unit has its own copy; each unit exports a host
// function that reads and clears it.
static __device__ unsigned int g_dev_status = 0;

// --------------------------------------------------------------------------
// Zig-zag walk over an N x N coefficient block (Sec. 4.1, "standard zig-zag"):
// anti-diagonals d = i + j in increasing order, odd d walked with the row
// increasing, even d with the row decreasing; JPEG order for N = 8.  For even N
// the walk is point-symmetric: position N*N-1-k mirrors position k.
// --------------------------------------------------------------------------
__host__ __device__ constexpr int zz_index(int N, int i, int j) {
    int d = i + j;
    if (d < N) return d * (d + 1) / 2 + ((d & 1) ? i : d - i);
    int m = 2 * N - 2 - d;
    int base = N * N - (m + 1) * (m + 2) / 2;
    return base + ((d & 1) ? i - (d - (N - 1)) : (N - 1 - i));
}

__host__ __device__ constexpr int zz_upper_diag(int k) {
    int d = 0;
    while ((d + 1) * (d + 2) / 2 <= k) d++;
    return d;
}

__host__ __device__ constexpr int zz_row(int N, int k) {
    if (k < N * (N + 1) / 2) {
        int d = zz_upper_diag(k), off = k - d * (d + 1) / 2;
        return (d & 1) ? off : d - off;
    }
    int kk = N * N - 1 - k;
    int d = zz_upper_diag(kk), off = kk - d * (d + 1) / 2;
    return N - 1 - ((d & 1) ? off : d - off);
}

__host__ __device__ constexpr int zz_col(int N, int k) {
    if (k < N * (N + 1) / 2) {
        int d = zz_upper_diag(k), off = k - d * (d + 1) / 2;
        return d - ((d & 1) ? off : d - off);
    }
    int kk = N * N - 1 - k;
    int d = zz_upper_diag(kk), off = kk - d * (d + 1) / 2;
    return N - 1 - (d - ((d & 1) ? off : d - off));
}

// --------------------------------------------------------------------------
// PTX wrappers (sm_90+ forms that sm_103a keeps)
// --------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void fence_mbar_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

__device__ __forceinline__ uint64_t global_timer_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
    return t;
}

// try_wait with a suspend-time hint: a thread whose phase is not complete sleeps
// in hardware until the phase completes or about hint_ns pass, instead of spinning
// (a spinning warp takes issue slots from the working warps of its scheduler).
__device__ __forceinline__ bool mbar_try_wait_sleep(uint64_t *bar, uint32_t parity, uint32_t hint_ns) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity), "r"(hint_ns)
        : "memory");
    return ok != 0;
}

// Wait for phase `parity` of an mbarrier by polling (for short waits such as an MMA's
// completion), giving up after timeout_ns of GPU time like mbar_wait_bounded.
__device__ __forceinline__ bool mbar_wait_poll(uint64_t *bar, uint32_t parity, uint64_t timeout_ns) {
    if (mbar_try_wait(bar, parity)) return true;
    const uint64_t t0 = global_timer_ns();
    while (true) {
        for (int k = 0; k < 64; k++)
            if (mbar_try_wait(bar, parity)) return true;
        if (global_timer_ns() - t0 > timeout_ns) {
            atomicExch(&g_dev_status, 7u);
            return false;
        }
    }
}

// Wait for phase `parity` of an mbarrier, giving up after timeout_ns of GPU
// time; on give-up the device status latches RKLT_ERR_TIMEOUT (7).  Each retry
// sleeps up to 0.5 ms (or the remaining limit, if shorter) unless the phase completes.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, uint32_t parity, uint64_t timeout_ns) {
    if (mbar_try_wait(bar, parity)) return true;
    const uint64_t t0 = global_timer_ns();
    const uint32_t hint = timeout_ns < 500000ull ? uint32_t(timeout_ns) : 500000u;
    while (true) {
        if (mbar_try_wait_sleep(bar, parity, hint)) return true;
        if (global_timer_ns() - t0 > timeout_ns) {
            atomicExch(&g_dev_status, 7u);
            return false;
        }
    }
}

__device__ __forceinline__ void fence_proxy_async_smem() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// 3-D tiled bulk tensor load global -> shared, completion counted on `bar`.
__device__ __forceinline__ void tma_load_3d(void *smem_dst, const CUtensorMap *map, int x, int y, int z,
                                            uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(smem_u32(smem_dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(smem_u32(bar))
        : "memory");
}

// 3-D tiled bulk tensor store shared -> global (out-of-range elements are dropped).
__device__ __forceinline__ void tma_store_3d(const CUtensorMap *map, int x, int y, int z, const void *smem_src) {
    asm volatile(
        "cp.async.bulk.tensor.3d.global.shared::cta.tile.bulk_group"
        " [%0, {%1, %2, %3}], [%4];" ::"l"(reinterpret_cast<uint64_t>(map)),
        "r"(x), "r"(y), "r"(z), "r"(smem_u32(smem_src))
        : "memory");
}

__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }
__device__ __forceinline__ void bulk_wait_read_all() {
    asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");
}
__device__ __forceinline__ void bulk_wait_all() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }

// Barrier over the first `count` threads of the CTA that also ORs a predicate.
__device__ __forceinline__ bool named_any(int id, int count, bool pred) {
    uint32_t r;
    asm volatile(
        "{\n\t.reg .pred p, q;\n\t"
        "setp.ne.u32 p, %1, 0;\n\t"
        "bar.red.or.pred q, %2, %3, p;\n\t"
        "selp.u32 %0, 1, 0, q;\n\t}"
        : "=r"(r)
        : "r"(uint32_t(pred)), "r"(id), "r"(count)
        : "memory");
    return r != 0;
}

// Barrier over the first `count` threads of the CTA (named barrier `id`).
__device__ __forceinline__ void named_sync(int id, int count) {
    asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(count) : "memory");
}

// --------------------------------------------------------------------------
// Numeric helpers
// --------------------------------------------------------------------------
// Byte k of a 32-bit word as an exact float.
__device__ __forceinline__ float byte_f(uint32_t w, int k) { return float((w >> (8 * k)) & 0xffu); }

// Packed binary16 pairs held in 32-bit registers.
__device__ __forceinline__ __half2 as_h2(uint32_t u) {
    __half2 h;
    memcpy(&h, &u, 4);
    return h;
}
__device__ __forceinline__ uint32_t as_u32(__half2 h) {
    uint32_t u;
    memcpy(&u, &h, 4);
    return u;
}

// Bytes c0 and c1 of w as the pair (1024 + b0, 1024 + b1) of binary16 values:
// 0x64 in the high byte of each lane makes the half 1024 + byte exactly.
__device__ __forceinline__ uint32_t bytes_to_biased_h2(uint32_t w, int c0, int c1) {
    return __byte_perm(w, 0x6464u, uint32_t(c0) | (4u << 4) | (uint32_t(c1) << 8) | (5u << 12));
}

// FP32 difference (half a) - (float c) with a single rounding (mixed-precision sub).
__device__ __forceinline__ float sub_h_f(__half a, float c) {
    float d;
    asm("sub.rn.f32.f16 %0, %1, %2;" : "=f"(d) : "h"(__half_as_ushort(a)), "f"(c));
    return d;
}

// clip(floor(x), 0, 255) as an integer 0..255 (float-to-integer conversions saturate).
__device__ __forceinline__ uint32_t floor_sat_u8(float x) {
    uint32_t u;
    asm("cvt.rmi.sat.u8.f32 %0, %1;" : "=r"(u) : "f"(x));
    return u;
}

// Bytes clip(floor(v0..v3 - 1024), 0, 255) packed little-endian, for v = 1024 + x:
// binary16 has unit spacing on [1024, 2048), so conversion toward zero is the floor
// there, and the half 1024 + n has n as its low byte.  The clamp to [1024, 1279] runs
// on the halves' bit patterns as signed 16-bit integers (negative halves are negative
// integers, positive ones are ordered like their values), i.e. on the integer ALU,
// not the floating-point pipe; one permute gathers the four low bytes.
__device__ __forceinline__ uint32_t bytes4_biased(float v0, float v1, float v2, float v3) {
    uint32_t h01, h23;
    asm("cvt.rz.f16x2.f32 %0, %1, %2;" : "=r"(h01) : "f"(v1), "f"(v0));
    asm("cvt.rz.f16x2.f32 %0, %1, %2;" : "=r"(h23) : "f"(v3), "f"(v2));
    const uint32_t lo = 0x64006400u, hi = 0x64FF64FFu;
    asm("max.s16x2 %0, %0, %1;" : "+r"(h01) : "r"(lo));
    asm("min.s16x2 %0, %0, %1;" : "+r"(h01) : "r"(hi));
    asm("max.s16x2 %0, %0, %1;" : "+r"(h23) : "r"(lo));
    asm("min.s16x2 %0, %0, %1;" : "+r"(h23) : "r"(hi));
    return __byte_perm(h01, h23, 0x6420);
}

// Sum of the four signed byte products a_k b_k (a signed, b unsigned) plus c.
__device__ __forceinline__ int dp4a_su(uint32_t a, uint32_t b, int c) {
    int d;
    asm("dp4a.s32.u32 %0, %1, %2, %3;" : "=r"(d) : "r"(a), "r"(b), "r"(c));
    return d;
}

// 4 x 4 byte transpose: out[c] holds byte c of r0, r1, r2, r3 (in that order).
__device__ __forceinline__ void transpose4x4(uint32_t r0, uint32_t r1, uint32_t r2, uint32_t r3, uint32_t (&out)[4]) {
    const uint32_t x0 = __byte_perm(r0, r1, 0x5140), x1 = __byte_perm(r0, r1, 0x7362);
    const uint32_t x2 = __byte_perm(r2, r3, 0x5140), x3 = __byte_perm(r2, r3, 0x7362);
    out[0] = __byte_perm(x0, x2, 0x5410);
    out[1] = __byte_perm(x0, x2, 0x7632);
    out[2] = __byte_perm(x1, x3, 0x5410);
    out[3] = __byte_perm(x1, x3, 0x7632);
}

// clip(floor(x + 1/2), 0, 255): round-half-up then saturate to 8 bits.
__device__ __forceinline__ uint32_t recon_byte(float x) {
    float v = fminf(fmaxf(x + 0.5f, 0.0f), 255.0f);
    return __float2uint_rd(v);
}

}  // namespace rklt
