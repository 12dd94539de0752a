// rklt_batch.cu -- many images of uneven sizes (and their own r) in one launch.
//
// Work is a flattened queue of "units": 32 horizontally adjacent N x N blocks of
// one block-row of one image.  Each warp takes units round-robin; lane l owns
// block 32u + l and runs the same per-block computation as the fused kernel
// (block_core: exact column/row pass, zonal mask, inverse, error, 8-bit output).
// A unit's pixels arrive by cp.async in a per-warp staging ring one unit ahead;
// the 8-bit output goes straight to global memory (a warp's 32 blocks are 256
// contiguous bytes per row); for N = 8 the coefficients go through a per-warp
// shared-memory stage and leave as one contiguous run per unit.  D =
// diag_bound(N, r) is per image and selects a register-resident variant of
// block_core.  The SSE of a unit goes to a fixed slot, and a per-image kernel sums
// an image's slots in order, so results do not depend on the rest of the batch.
//
// rklt_fused_items launches immediately (continuous batching of requests);
// rklt_batch_* builds the queue once, captures the launches in a CUDA graph
// and picks the launch shape with a small autotuner (timed candidates).
#include <algorithm>
#include <cstring>
#include <mutex>
#include <map>
#include <utility>
#include <vector>

#include "rklt_fused_impl.cuh"

namespace rklt {

struct BatchItem {
    const uint8_t *img;
    uint8_t *recon;
    float *zcoef;
    int64_t ld, ld_recon;
    int64_t unit_base;  // first unit of this item in the queue
    int H, W, r, D;
    int bw, units_x;    // blocks per block-row, units per block-row
    int vec4;           // coefficients as float4 (r % 4 == 0, 16-byte aligned)
    int out_index;      // position of this item in the caller's d_sse / d_psnr
    int slot;           // the plan's slot in the constant-memory plan table (queue kernel)
    int64_t nunits;     // units of this item
};

// Last item whose unit range starts at or before u, searching forward from lo
// (items[lo].unit_base <= u): a galloping step, then a binary search.
__device__ __forceinline__ int item_of(const BatchItem *__restrict__ items, int nitems, int lo, int64_t u) {
    int a = lo, step = 1, b = lo + 1;
    while (b < nitems && items[b].unit_base <= u) {
        a = b;
        step <<= 1;
        b = a + step;
    }
    int hi = (b < nitems ? b : nitems) - 1;
    while (a < hi) {
        const int mid = (a + hi + 1) >> 1;
        if (items[mid].unit_base <= u) a = mid;
        else hi = mid - 1;
    }
    return a;
}

// Asynchronous copies global -> shared (cp.async, cached in L1 and L2).
template <int BYTES>
__device__ __forceinline__ void cp_async(void *smem_dst, const void *gmem_src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], %2;" ::"r"(smem_u32(smem_dst)), "l"(gmem_src), "n"(BYTES)
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int PENDING>
__device__ __forceinline__ void cp_async_wait() {
    asm volatile("cp.async.wait_group %0;" ::"n"(PENDING) : "memory");
}

// Position of lane's block in unit u of item it; false past the image's right edge.
// An item has fewer than 2^31 units (checked when the queue is built), so the
// division runs in 32 bits.
__device__ __forceinline__ bool unit_block(const BatchItem &it, int64_t u, int lane, int &by, int &bx) {
    const uint32_t local = uint32_t(u - it.unit_base);
    const uint32_t q = local / uint32_t(it.units_x);
    by = int(q);
    bx = int(local - q * uint32_t(it.units_x)) * 32 + lane;
    return bx < it.bw;
}

// Stage lane's block (N rows of N bytes) into dst with asynchronous copies; row k
// goes to dst + k * 32 N, so that the 32 lanes' rows are contiguous.
template <int N>
__device__ __forceinline__ void stage_block(const BatchItem &it, int by, int bx, uint8_t *dst) {
    const uint8_t *src = it.img + int64_t(by) * N * it.ld + bx * N;
#pragma unroll
    for (int k = 0; k < N; k++) cp_async<N>(dst + k * 32 * N, src + k * it.ld);
}

// Staging slots per warp: a warp transforms one unit while the copies of the next
// BRING - 1 are in flight.  (Four and eight slots measured no faster on the
// 2000-image batch than two: its kernels are bound by the per-block arithmetic at
// high diagonal bounds, not by the copies.)
constexpr int BRING = 2;

// Walks the warp's units u = warp0, warp0 + nwarps, ... through the ring: the copy of
// unit u + (BRING - 1) nwarps is issued into the slot just freed, then unit u (landed)
// is handed to body(u, item index, by, bx, have, staged block of this lane).  The
// pending units' positions form a register FIFO (shifted once per unit), so the body
// appears once in the loop.  mine: this lane's byte in slot 0 of the warp's ring
// (slot s at + s * 32 N N).
template <int N, class Body>
__device__ __forceinline__ void walk_units(const BatchItem *__restrict__ items, int nitems, int64_t nunits,
                                           int64_t warp0, int64_t nwarps, int lane, uint8_t *mine, Body body) {
    int idx[BRING], by[BRING], bx[BRING];   // FIFO: entry j is unit u + j nwarps
    bool have[BRING];
    int lo = item_of(items, nitems, 0, warp0);
    // stages unit un into ring slot s as FIFO entry j (nothing past the queue's end);
    // one copy group
    const auto stage = [&](int j, int s, int64_t un) {
        have[j] = false;
        idx[j] = lo;
        by[j] = bx[j] = 0;
        if (un < nunits) {
            lo = item_of(items, nitems, lo, un);
            idx[j] = lo;
            const BatchItem &it = items[lo];
            have[j] = unit_block(it, un, lane, by[j], bx[j]);
            if (have[j]) stage_block<N>(it, by[j], bx[j], mine + s * 32 * N * N);
        }
        cp_async_commit();
    };
#pragma unroll
    for (int j = 0; j < BRING - 1; j++) stage(j, j, warp0 + j * nwarps);
    int slot = 0;   // ring slot of FIFO entry 0
#pragma unroll 1
    for (int64_t u = warp0; u < nunits; u += nwarps) {
        const int last = slot == 0 ? BRING - 1 : slot - 1;
        stage(BRING - 1, last, u + (BRING - 1) * nwarps);
        cp_async_wait<BRING - 1>();   // unit u's group (the oldest pending) has landed
        body(u, idx[0], by[0], bx[0], have[0], mine + slot * 32 * N * N);
#pragma unroll
        for (int j = 0; j + 1 < BRING; j++) {
            idx[j] = idx[j + 1];
            by[j] = by[j + 1];
            bx[j] = bx[j + 1];
            have[j] = have[j + 1];
        }
        slot = slot == BRING - 1 ? 0 : slot + 1;
    }
    cp_async_wait<0>();
}

// Each warp walks units u = warp0, warp0 + nwarps, ... (walk_units): the pixels of the
// next BRING - 1 units are copied into the warp's staging ring (cp.async) while the
// current unit is transformed.  N = 8: the coefficients (up to 64 per block) go
// through a per-warp shared-memory stage and leave as one contiguous run per unit
// (warp_coef_copy8) instead of 32 strided per-lane runs.
// Dynamic shared memory (batch_smem): warps x BRING slots x N rows x 32 lanes x N
// bytes, then for N = 8 warps x 32 lanes x STG8_LD floats.
template <int N>
__device__ __forceinline__ float *coef_stage(uint8_t *bsm, int warp) {
    if constexpr (N == 8)
        return reinterpret_cast<float *>(bsm + (blockDim.x / 32) * BRING * 32 * N * N) + warp * 32 * STG8_LD;
    else
        return nullptr;
}

// The unit's coefficient destination and staging: where lane's block writes its
// coefficients (its global run for N = 4, the warp stage for N = 8), and for N = 8
// the copy of the warp's run to global memory afterwards (all lanes).
template <int N>
struct UnitCoef {
    float *run = nullptr;     // global run of the unit's first block (N = 8)
    float *mine = nullptr;    // where this lane's block writes
    int nb = 0;               // blocks of the unit inside the image
    bool vec4 = false;        // this lane's block writes float4
    __device__ __forceinline__ UnitCoef(const BatchItem &it, int by, int bx, int lane, float *stage) {
        if (!it.zcoef || it.r == 0) return;
        if constexpr (N == 8) {
            const int bx0 = bx - lane;
            run = it.zcoef + (int64_t(by) * it.bw + bx0) * it.r;
            mine = stage + lane * STG8_LD;
            nb = min(32, it.bw - bx0);
            vec4 = (it.r & 3) == 0;
        } else {
            mine = it.zcoef + (int64_t(by) * it.bw + bx) * it.r;
            vec4 = it.vec4 != 0;
        }
    }
    __device__ __forceinline__ void flush(const BatchItem &it, float *stage, int lane) const {
        if constexpr (N == 8) {
            if (!run) return;
            __syncwarp();
            warp_coef_copy8(run, stage, nb, it.r, it.vec4 != 0, lane);
            __syncwarp();   // the stage is rewritten by the next unit
        }
    }
};

template <int N, int D>
__global__ void __launch_bounds__(256, 1)
    batch_kernel(const __grid_constant__ PlanK<N> P, const BatchItem *__restrict__ items, int nitems, int64_t nunits,
                 float *__restrict__ partials) {
    extern __shared__ __align__(16) uint8_t bsm[];
    const int lane = threadIdx.x & 31, warp = int(threadIdx.x >> 5);
    const int64_t warp0 = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = (int64_t(gridDim.x) * blockDim.x) >> 5;
    if (warp0 >= nunits) return;
    uint8_t *mine = bsm + warp * (BRING * 32 * N * N) + lane * N;
    float *stage = coef_stage<N>(bsm, warp);
    walk_units<N>(items, nitems, nunits, warp0, nwarps, lane, mine,
                  [&](int64_t u, int k, int by, int bx, bool have, const uint8_t *src) {
                      const BatchItem &it = items[k];
                      const UnitCoef<N> uc(it, by, bx, lane, stage);
                      float sse = 0.0f;
                      if (have) {
                          uint32_t w[N][N / 4];
                          load_block_words<N>(src, 32 * N, w);
                          uint8_t *dst = it.recon ? it.recon + int64_t(by) * N * it.ld_recon + bx * N : nullptr;
                          sse = block_core<N, D>(P, w, dst, it.ld_recon, it.r, uc.mine, uc.vec4, dst != nullptr);
                      }
                      uc.flush(it, stage, lane);
#pragma unroll
                      for (int off = 16; off > 0; off >>= 1) sse += __shfl_xor_sync(0xffffffffu, sse, off);
                      if (lane == 0) partials[u] = sse;
                  });
}

// Sum of an item's unit partials by one warp, in a fixed order (lane-strided
// FP64 sums, then a fixed shuffle tree), then SSE and PSNR.
__device__ __forceinline__ void finalize_item(const BatchItem &it, const float *partials, double *sse, float *psnr,
                                              int lane) {
    double acc = 0.0;
    for (int64_t u = it.unit_base + lane; u < it.unit_base + it.nunits; u += 32)
        acc += double(__ldcg(partials + u));
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
    if (lane == 0) {
        const double npx = double(it.H) * double(it.W);
        sse[it.out_index] = acc;
        float p;
        if (npx == 0.0) p = __int_as_float(0x7fc00000);
        else if (acc == 0.0) p = __int_as_float(0x7f800000);
        else p = float(10.0 * log10(255.0 * 255.0 * npx / acc));
        psnr[it.out_index] = p;
    }
}

// One warp per item (grouped launches): the same sum as the queue kernel's, so
// both forms give bit-identical results.
__global__ void batch_finalize(const BatchItem *__restrict__ items, int nitems, int64_t nunits,
                               const float *__restrict__ partials, double *sse, float *psnr) {
    const int i = blockIdx.x;
    if (i >= nitems) return;
    finalize_item(items[i], partials, sse, psnr, int(threadIdx.x));
}

// ---------------------------------------------------------------------------
// One persistent launch for a whole batch (all plans, all diagonal bounds), then one
// finalize warp per item.  Plans live in a constant-memory table (one slot per plan
// and device, written once before first use); each unit dispatches on its item's D.
// Units are queued heaviest first (larger D) and dealt round-robin to the warps.
// (Finishing an item inside the kernel, by the warp whose unit completes it, needs a
// fence and an atomic per unit; that made the launch 3x slower than the separate
// finalize.)
// ---------------------------------------------------------------------------
constexpr int kPlanSlots = 16;
// Each slot padded to whole 256-byte lines, so that no cached constant line holds
// bytes of two plans (a slot is written while kernels reading other slots may run).
template <int N>
struct alignas(256) PlanSlot {
    PlanK<N> k;
};
__constant__ PlanSlot<8> c_plans8[kPlanSlots];
__constant__ PlanSlot<4> c_plans4[kPlanSlots];

template <int N>
__device__ __forceinline__ const PlanK<N> &plan_slot(int k) {
    if constexpr (N == 8) return c_plans8[k].k;
    else return c_plans4[k].k;
}

// The per-block computation for one diagonal bound, out of line: the queue kernel
// calls the variant of each unit's D (each variant is compiled once, and the kernel
// stays a small dispatcher).  slot: the unit's plan in the constant-memory table,
// read inside so that its operands are constant-bank loads; src: the staged block,
// row stride 32 N bytes.
template <int N, int D>
__device__ __noinline__ float block_d(int slot, const uint8_t *src, uint8_t *dst, int64_t ldd, int r, float *coef,
                                      bool vec4, bool recon) {
    uint32_t w[N][N / 4];
    load_block_words<N>(src, 32 * N, w);
    return block_core<N, D>(plan_slot<N>(slot), w, dst, ldd, r, coef, vec4, recon);
}

template <int N, int D = 0>
__device__ __forceinline__ float block_any_d(int slot, int Dr, const uint8_t *src, uint8_t *dst, int64_t ldd, int r,
                                             float *coef, bool vec4, bool recon) {
    if constexpr (D >= 2 * N - 1) {
        return block_d<N, 2 * N - 1>(slot, src, dst, ldd, r, coef, vec4, recon);
    } else {
        if (Dr == D) return block_d<N, D>(slot, src, dst, ldd, r, coef, vec4, recon);
        return block_any_d<N, D + 1>(slot, Dr, src, dst, ldd, r, coef, vec4, recon);
    }
}

template <int N>
__global__ void __launch_bounds__(256, 1)
    queue_kernel(const BatchItem *__restrict__ items, int nitems, int64_t nunits, float *__restrict__ partials) {
    extern __shared__ __align__(16) uint8_t bsm[];
    const int lane = threadIdx.x & 31;
    const int64_t warp0 = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = (int64_t(gridDim.x) * blockDim.x) >> 5;
    if (warp0 >= nunits) return;
    const int warp = int(threadIdx.x >> 5);
    uint8_t *mine = bsm + warp * (BRING * 32 * N * N) + lane * N;
    float *stage = coef_stage<N>(bsm, warp);
    walk_units<N>(items, nitems, nunits, warp0, nwarps, lane, mine,
                  [&](int64_t u, int k, int by, int bx, bool have, const uint8_t *src) {
                      const BatchItem &it = items[k];
                      const UnitCoef<N> uc(it, by, bx, lane, stage);
                      float e = 0.0f;
                      if (have) {
                          uint8_t *dst = it.recon ? it.recon + int64_t(by) * N * it.ld_recon + bx * N : nullptr;
                          e = block_any_d<N>(it.slot, it.D, src, dst, it.ld_recon, it.r, uc.mine, uc.vec4,
                                             dst != nullptr);
                      }
                      uc.flush(it, stage, lane);
#pragma unroll
                      for (int off = 16; off > 0; off >>= 1) e += __shfl_xor_sync(0xffffffffu, e, off);
                      if (lane == 0) partials[u] = e;
                  });
}

namespace {

// Constant-memory plan table: one slot per (device, plan), written once (on a
// private stream, so no other stream waits) before the plan's first queued use and
// released when the plan is destroyed.
struct Registry {
    const Plan *slot_plan[kPlanSlots] = {};
};
std::mutex g_reg_mu;
Registry g_reg[64][2];   // [device][N == 8]

// Slot of `p` on the current device, writing it if new; -1 when every slot is taken.
int plan_slot_for(const Plan &p) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return -1;
    std::lock_guard<std::mutex> lk(g_reg_mu);
    Registry &R = g_reg[dev][p.N == 8 ? 1 : 0];
    int free_k = -1;
    for (int k = 0; k < kPlanSlots; k++) {
        if (R.slot_plan[k] == &p) return k;
        if (!R.slot_plan[k] && free_k < 0) free_k = k;
    }
    if (free_k < 0) return -1;
    static cudaStream_t up[64] = {};
    if (!up[dev] && cudaStreamCreateWithFlags(&up[dev], cudaStreamNonBlocking) != cudaSuccess) return -1;
    const size_t bytes = p.N == 8 ? sizeof(PlanK<8>) : sizeof(PlanK<4>);
    const size_t off = size_t(free_k) * (p.N == 8 ? sizeof(PlanSlot<8>) : sizeof(PlanSlot<4>));
    const cudaError_t e = p.N == 8 ? cudaMemcpyToSymbolAsync(c_plans8, p.k.data(), bytes, off,
                                                              cudaMemcpyHostToDevice, up[dev])
                                   : cudaMemcpyToSymbolAsync(c_plans4, p.k.data(), bytes, off,
                                                              cudaMemcpyHostToDevice, up[dev]);
    if (e != cudaSuccess || cudaStreamSynchronize(up[dev]) != cudaSuccess) return -1;
    R.slot_plan[free_k] = &p;
    return free_k;
}

}  // namespace

void plan_registry_release(const Plan *p) {
    std::lock_guard<std::mutex> lk(g_reg_mu);
    for (auto &dev : g_reg)
        for (auto &R : dev)
            for (auto &sp : R.slot_plan)
                if (sp == p) sp = nullptr;
}

namespace {

struct Group {
    const Plan *plan = nullptr;
    int D = 0;  // every item of a group has the same retained support
    std::vector<BatchItem> items;
    int64_t nunits = 0;
};

// Validate items and split them by plan, building each group's unit queue.
rklt_status build_groups(const rklt_item *h, int n, const rklt_plan *const *plans, int nplans, std::vector<Group> &out,
                         int &N) {
    if (n < 1 || !h) return fail(RKLT_ERR_ARG, "need at least one item");
    if (nplans < 1 || !plans) return fail(RKLT_ERR_ARG, "need at least one plan");
    N = 0;
    for (int p = 0; p < nplans; p++) {
        if (!plans[p]) return fail(RKLT_ERR_ARG, "NULL plan");
        if (plans[p]->p.kind != 0) return fail(RKLT_ERR_UNSUPPORTED, "uneven batches need rounded (integer) plans");
        if (N == 0) N = plans[p]->p.N;
        if (plans[p]->p.N != N) return fail(RKLT_ERR_ARG, "all plans of a batch must share N");
    }
    if (N != 4 && N != 8) return fail(RKLT_ERR_UNSUPPORTED, "batched launches support N = 4 and N = 8");
    const uintptr_t amask = N == 8 ? 7 : 3;
    std::map<std::pair<int, int>, int> gidx;
    out.clear();
    for (int i = 0; i < n; i++) {
        const rklt_item &x = h[i];
        if (x.plan < 0 || x.plan >= nplans) return fail(RKLT_ERR_ARG, "item plan index out of range");
        if (x.r < 0 || x.r > N * N) return fail(RKLT_ERR_ARG, "item r must lie in [0, N*N]");
        if (x.H < 0 || x.W < 0 || x.H % N || x.W % N)
            return fail(RKLT_ERR_SHAPE, "item H and W must be non-negative multiples of N");
        if (x.ld < x.W) return fail(RKLT_ERR_SHAPE, "item ld must be >= W");
        if (x.H > 0 && x.W > 0 && !x.d_img) return fail(RKLT_ERR_ARG, "item image is NULL");
        if ((reinterpret_cast<uintptr_t>(x.d_img) | uintptr_t(x.ld)) & amask)
            return fail(RKLT_ERR_UNSUPPORTED, "batched items need N-byte aligned image rows");
        if (x.d_recon) {
            if (x.ld_recon < x.W) return fail(RKLT_ERR_SHAPE, "item ld_recon must be >= W");
            if ((reinterpret_cast<uintptr_t>(x.d_recon) | uintptr_t(x.ld_recon)) & amask)
                return fail(RKLT_ERR_UNSUPPORTED, "batched items need N-byte aligned reconstruction rows");
        }
        if (x.d_zcoef && (reinterpret_cast<uintptr_t>(x.d_zcoef) & 3))
            return fail(RKLT_ERR_ARG, "item coefficient pointer must be 4-byte aligned");
        const int D = diag_bound(N, x.r);
        auto f = gidx.find({x.plan, D});
        if (f == gidx.end()) {
            f = gidx.emplace(std::make_pair(x.plan, D), int(out.size())).first;
            out.emplace_back();
            out.back().plan = &plans[x.plan]->p;
            out.back().D = D;
        }
        Group &g = out[f->second];
        BatchItem b{};
        b.img = x.d_img;
        b.recon = x.d_recon;
        b.zcoef = x.d_zcoef;
        b.ld = x.ld;
        b.ld_recon = x.ld_recon;
        b.H = x.H;
        b.W = x.W;
        b.r = x.r;
        b.D = D;
        b.bw = x.W / N;
        b.units_x = (b.bw + 31) / 32;
        b.vec4 = (x.r % 4 == 0) && ((reinterpret_cast<uintptr_t>(x.d_zcoef) & 15) == 0);
        b.out_index = i;
        b.unit_base = g.nunits;
        b.nunits = int64_t(x.H / N) * b.units_x;
        if (b.nunits >= (int64_t(1) << 31)) return fail(RKLT_ERR_SHAPE, "image too large for a batch item");
        g.nunits += b.nunits;
        g.items.push_back(b);
    }
    return RKLT_OK;
}

template <int N, int D>
const void *batch_fn() { return reinterpret_cast<const void *>(batch_kernel<N, D>); }

// Host-side table of the batch kernels, indexed by D.
template <int N, int... Ds>
const void *pick_fn(int D, std::integer_sequence<int, Ds...>) {
    const void *tab[] = {batch_fn<N, Ds>()...};
    return tab[D];
}

// Dynamic shared memory of a batch launch: BRING staging slots per warp, and the
// per-warp coefficient stage for N = 8.
size_t batch_smem(int N, int threads) {
    return size_t(threads / 32) * (BRING * 32 * N * N + (N == 8 ? 32 * STG8_LD * 4 : 0));
}

const void *batch_kernel_for(int N, int D) {
    return N == 4 ? pick_fn<4>(D, std::make_integer_sequence<int, 8>{})
                  : pick_fn<8>(D, std::make_integer_sequence<int, 16>{});
}

cudaError_t launch_group(int N, const Group &g, const BatchItem *d_items, float *partials, double *sse, float *psnr,
                         int threads, int grid, cudaStream_t st) {
    const int nitems = int(g.items.size());
    int64_t nunits = g.nunits;
    if (nunits > 0) {
        const void *fn = batch_kernel_for(N, g.D);
        const void *kp = g.plan->k.data();
        void *args[] = {const_cast<void *>(kp), &d_items, const_cast<int *>(&nitems), &nunits, &partials};
        const cudaError_t e = cudaLaunchKernel(fn, dim3(grid), dim3(threads), args, batch_smem(N, threads), st);
        if (e != cudaSuccess) return e;
    }
    batch_finalize<<<nitems, 32, 0, st>>>(d_items, nitems, nunits, partials, sse, psnr);
    return cudaGetLastError();
}

const void *queue_kernel_for(int N);

// The staging ring needs more than the default 48 KB of dynamic shared memory: opt
// every batch kernel of N in, once per device (before its first launch or occupancy
// query, and so before any graph capture of the launches).
void batch_smem_attrs(int N, int dev) {
    static std::mutex mu;
    static bool done[2][64] = {};
    const int n = N == 4 ? 0 : 1;
    std::lock_guard<std::mutex> lk(mu);
    if (dev < 0 || dev >= 64 || done[n][dev]) return;
    for (int D = 0; D < 2 * N; D++) ensure_smem_attr(batch_kernel_for(N, D));
    ensure_smem_attr(queue_kernel_for(N));
    done[n][dev] = true;
}

// Largest useful persistent grid for `threads` per CTA and `per_sm` CTAs per SM.
int grid_for(int N, int threads, int per_sm, int64_t nunits) {
    int dev = 0;
    cudaGetDevice(&dev);
    batch_smem_attrs(N, dev);
    int occ = 0;
    occ = occupancy(batch_kernel_for(N, N == 4 ? 7 : 15), threads, batch_smem(N, threads));
    const int use = std::max(1, std::min(per_sm, occ));
    const int64_t warps_needed = nunits;
    const int64_t ctas_needed = (warps_needed * 32 + threads - 1) / threads;
    return int(std::max<int64_t>(1, std::min<int64_t>(int64_t(use) * sm_count(dev), ctas_needed)));
}

// One queue over every group: groups ordered by D (heaviest first), then plan;
// unit bases run over the whole queue; each item carries its plan's constant slot.
// Items without units (empty images) go to `empty`.  False if a plan gets no slot.
bool build_queue(const std::vector<Group> &groups, std::vector<BatchItem> &q, std::vector<BatchItem> &empty,
                 int64_t &nunits) {
    std::vector<size_t> order(groups.size());
    for (size_t i = 0; i < order.size(); i++) order[i] = i;
    std::stable_sort(order.begin(), order.end(), [&](size_t a, size_t b) { return groups[a].D > groups[b].D; });
    q.clear();
    empty.clear();
    nunits = 0;
    for (size_t gi : order) {
        const int slot = plan_slot_for(*groups[gi].plan);
        if (slot < 0) return false;
        for (BatchItem b : groups[gi].items) {
            b.slot = slot;
            if (b.nunits == 0) {
                b.unit_base = 0;
                empty.push_back(b);
                continue;
            }
            b.unit_base = nunits;
            nunits += b.nunits;
            q.push_back(b);
        }
    }
    return true;
}

const void *queue_kernel_for(int N) {
    return N == 8 ? reinterpret_cast<const void *>(queue_kernel<8>) : reinterpret_cast<const void *>(queue_kernel<4>);
}

int queue_grid(int N, int threads, int per_sm, int64_t nunits) {
    int dev = 0;
    cudaGetDevice(&dev);
    batch_smem_attrs(N, dev);
    const int occ = occupancy(queue_kernel_for(N), threads, batch_smem(N, threads));
    const int use = std::max(1, std::min(per_sm, occ));
    const int64_t ctas_needed = (nunits * 32 + threads - 1) / threads;
    return int(std::max<int64_t>(1, std::min<int64_t>(int64_t(use) * sm_count(dev), ctas_needed)));
}

// Empty items (H or W = 0): SSE 0, PSNR NaN.
__global__ void empty_items(const BatchItem *__restrict__ items, int n, double *sse, float *psnr) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    sse[items[i].out_index] = 0.0;
    psnr[items[i].out_index] = __int_as_float(0x7fc00000);
}

// The queue kernel over every unit, then one finalize warp per item (the unit
// partials summed in order, as for the grouped launches).
cudaError_t launch_queue(int N, const BatchItem *d_items, int nitems, int64_t nunits, const BatchItem *d_empty,
                         int nempty, float *partials, double *sse, float *psnr, int threads, int per_sm,
                         cudaStream_t st) {
    if (nunits > 0) {
        const int grid = queue_grid(N, threads, per_sm, nunits);
        void *args[] = {&d_items, &nitems, &nunits, &partials};
        const cudaError_t e =
            cudaLaunchKernel(queue_kernel_for(N), dim3(grid), dim3(threads), args, batch_smem(N, threads), st);
        if (e != cudaSuccess) return e;
        batch_finalize<<<nitems, 32, 0, st>>>(d_items, nitems, nunits, partials, sse, psnr);
    }
    if (nempty > 0) empty_items<<<(nempty + 127) / 128, 128, 0, st>>>(d_empty, nempty, sse, psnr);
    return cudaGetLastError();
}

}  // namespace
}  // namespace rklt

struct rklt_batch {
    int N = 0;
    std::vector<rklt::Group> groups;
    std::vector<rklt::BatchItem *> d_items;
    std::vector<float *> d_partials;
    double *sse = nullptr;
    float *psnr = nullptr;
    int threads = 256, per_sm = 1;
    double tuned_us = 0.0;
    cudaStream_t stream = nullptr;
    // the groups fan out over side streams (fork on one event, join on one per stream),
    // so that one group's last wave overlaps the next groups' launches
    std::vector<cudaStream_t> side;
    cudaEvent_t fork = nullptr;
    std::vector<cudaEvent_t> join;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    // one persistent launch over the whole queue (mode 1)
    int mode = 0;                      // 0 grouped launches, 1 queue kernel
    struct Timed {
        int mode, threads, per_sm;
        double us;
    };
    std::vector<Timed> tuned;          // every candidate the autotuner timed
    int64_t q_units = 0;
    int q_items = 0, q_empty = 0;
    rklt::BatchItem *dq_items = nullptr, *dq_empty = nullptr;
    float *dq_partials = nullptr;
};

using namespace rklt;

namespace {

void batch_free(rklt_batch *b) {
    if (!b) return;
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    for (auto p : b->d_items) cudaFree(p);
    for (auto p : b->d_partials) cudaFree(p);
    cudaFree(b->dq_items);
    cudaFree(b->dq_empty);
    cudaFree(b->dq_partials);
    if (b->stream) cudaStreamDestroy(b->stream);
    for (auto s : b->side) cudaStreamDestroy(s);
    for (auto e : b->join) cudaEventDestroy(e);
    if (b->fork) cudaEventDestroy(b->fork);
    delete b;
}

constexpr int kBatchSideStreams = 4;

cudaError_t batch_enqueue_groups(rklt_batch *b, int threads, int per_sm, cudaStream_t st);

// One run of the batch in mode 0 (grouped launches) or 1 (one queue launch).
cudaError_t batch_enqueue(rklt_batch *b, int mode, int threads, int per_sm, cudaStream_t st) {
    if (mode == 1)
        return launch_queue(b->N, b->dq_items, b->q_items, b->q_units, b->dq_empty, b->q_empty, b->dq_partials,
                            b->sse, b->psnr, threads, per_sm, st);
    return batch_enqueue_groups(b, threads, per_sm, st);
}

// Groups go round-robin over the side streams, largest first (the groups are
// independent: each has its own items, partials and outputs).
cudaError_t batch_enqueue_groups(rklt_batch *b, int threads, int per_sm, cudaStream_t st) {
    const bool fan = !b->side.empty();
    cudaError_t e = cudaSuccess;
    if (fan) {
        e = cudaEventRecord(b->fork, st);
        for (size_t k = 0; k < b->side.size() && e == cudaSuccess; k++) e = cudaStreamWaitEvent(b->side[k], b->fork, 0);
        if (e != cudaSuccess) return e;
    }
    std::vector<size_t> order(b->groups.size());
    for (size_t i = 0; i < order.size(); i++) order[i] = i;
    std::stable_sort(order.begin(), order.end(),
                     [&](size_t x, size_t y) { return b->groups[x].nunits > b->groups[y].nunits; });
    for (size_t k = 0; k < order.size(); k++) {
        const size_t gi = order[k];
        const Group &g = b->groups[gi];
        const int grid = grid_for(b->N, threads, per_sm, g.nunits);
        const cudaStream_t s = fan ? b->side[k % b->side.size()] : st;
        e = launch_group(b->N, g, b->d_items[gi], b->d_partials[gi], b->sse, b->psnr, threads, grid, s);
        if (e != cudaSuccess) return e;
    }
    if (fan) {
        for (size_t k = 0; k < b->side.size() && e == cudaSuccess; k++) {
            e = cudaEventRecord(b->join[k], b->side[k]);
            if (e == cudaSuccess) e = cudaStreamWaitEvent(st, b->join[k], 0);
        }
    }
    return e;
}

// Pinned staging for the item descriptors of immediate launches.  A copy from
// pageable memory would be staged by the runtime, and once its staging buffers are
// busy the host waits for earlier copies, which wait for the kernels queued before
// them: the request loop would stall behind work already on the GPU.  The ring is
// reused in order; a region is handed out again only after the event recorded
// behind its copy has completed.
class ItemRing {
  public:
    static constexpr size_t kBytes = size_t(4) << 20;
    // A pinned region of `bytes` (<= kBytes) for a copy enqueued on `st`; the caller
    // fills it, enqueues the copy and then calls done(st).  Null if no pinned memory.
    void *get(size_t bytes) {
        if (!base_ && cudaHostAlloc(&base_, kBytes, cudaHostAllocDefault) != cudaSuccess) base_ = nullptr;
        if (!base_ || bytes > kBytes) return nullptr;
        bytes = (bytes + 255) & ~size_t(255);
        for (;;) {
            if (used_ == 0) head_ = 0;  // empty: start over at the front
            // live regions occupy [head_ - used_, head_) in ring order; allocate after them
            size_t off = head_;
            if (off + bytes > kBytes) off = 0;  // wrap: never split a region
            const size_t skip = (off == 0 && head_ != 0) ? kBytes - head_ : 0;
            if (used_ + skip + bytes <= kBytes) {
                used_ += skip + bytes;
                pending_ = {off, skip + bytes};
                head_ = off + bytes;
                return static_cast<char *>(base_) + off;
            }
            if (regions_.empty()) return nullptr;
            // the oldest copy has read its bytes (a region without an event was
            // copied synchronously in done())
            if (regions_.front().ev) cudaEventSynchronize(regions_.front().ev);
            release_front();
        }
    }
    void done(cudaStream_t st) {
        cudaEvent_t ev = nullptr;
        if (!free_ev_.empty()) {
            ev = free_ev_.back();
            free_ev_.pop_back();
        } else if (cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) != cudaSuccess) {
            ev = nullptr;
        }
        if (ev && cudaEventRecord(ev, st) != cudaSuccess) {
            free_ev_.push_back(ev);
            ev = nullptr;
        }
        if (!ev) cudaStreamSynchronize(st);  // untracked: let the copy finish before reuse
        regions_.push_back({pending_.first, pending_.second, ev});
        while (!regions_.empty() && (!regions_.front().ev || cudaEventQuery(regions_.front().ev) == cudaSuccess))
            release_front();
    }

  private:
    struct Region {
        size_t off, len;
        cudaEvent_t ev;
    };
    void release_front() {
        const Region r = regions_.front();
        regions_.erase(regions_.begin());
        used_ -= r.len;
        if (r.ev) free_ev_.push_back(r.ev);
    }
    void *base_ = nullptr;
    size_t head_ = 0, used_ = 0;
    std::pair<size_t, size_t> pending_{0, 0};
    std::vector<Region> regions_;
    std::vector<cudaEvent_t> free_ev_;
};

std::mutex g_ring_mu;
ItemRing g_ring[64];  // per device

// Item descriptors to the device through the pinned ring (pageable when the ring is
// full, or under stream capture, where the copy would run at replay after the region
// is reused).
cudaError_t copy_items(BatchItem *d_items, const BatchItem *h_items, size_t bytes, cudaStream_t st) {
    int dev = 0;
    cudaGetDevice(&dev);
    std::lock_guard<std::mutex> lk(g_ring_mu);
    ItemRing &ring = g_ring[dev >= 0 && dev < 64 ? dev : 0];
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    cudaStreamIsCapturing(st, &cs);
    void *pinned = cs == cudaStreamCaptureStatusNone ? ring.get(bytes) : nullptr;
    if (!pinned) return cudaMemcpyAsync(d_items, h_items, bytes, cudaMemcpyHostToDevice, st);
    std::memcpy(pinned, h_items, bytes);
    const cudaError_t e = cudaMemcpyAsync(d_items, pinned, bytes, cudaMemcpyHostToDevice, st);
    ring.done(st);
    return e;
}

// Immediate batches with at least this many groups take the one-launch queue form.
constexpr size_t kQueueGroups = 3;

}  // namespace

extern "C" {

rklt_status rklt_fused_items(const rklt_item *h_items, int n, const rklt_plan *const *plans, int nplans,
                             double *d_sse, float *d_psnr, void *stream) {
    std::vector<Group> groups;
    int N = 0;
    rklt_status s = build_groups(h_items, n, plans, nplans, groups, N);
    if (s != RKLT_OK) return s;
    if (!d_sse || !d_psnr) return fail(RKLT_ERR_ARG, "d_sse and d_psnr are required");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    cudaMemPool_t pool = scratch_pool();
    if (!pool) return fail(RKLT_ERR_CUDA, "could not create the scratch memory pool");
    // Several (plan, support) groups: one queue launch and one finalize for all of them
    // instead of a launch pair per group (fewer commands on the stream; a request loop
    // issuing a batch per pass otherwise fills the stream's command queue and blocks).
    if (groups.size() >= kQueueGroups) {
        std::vector<BatchItem> q, em;
        int64_t nunits = 0;
        if (build_queue(groups, q, em, nunits)) {
            std::vector<BatchItem> all(q);
            all.insert(all.end(), em.begin(), em.end());
            const size_t ab = all.size() * sizeof(BatchItem);
            const size_t off_p = (ab + 255) & ~size_t(255);
            const size_t pb = size_t(std::max<int64_t>(nunits, 1)) * sizeof(float);
            void *scratch = nullptr;
            if (cudaMallocFromPoolAsync(&scratch, off_p + pb, pool, st) != cudaSuccess)
                return fail(RKLT_ERR_OOM, "scratch allocation failed");
            BatchItem *d_all = static_cast<BatchItem *>(scratch);
            float *partials = reinterpret_cast<float *>(static_cast<char *>(scratch) + off_p);
            cudaError_t e = copy_items(d_all, all.data(), ab, st);
            if (e == cudaSuccess)
                e = launch_queue(N, d_all, int(q.size()), nunits, d_all + q.size(), int(em.size()), partials, d_sse,
                                 d_psnr, 256, 1, st);
            cudaFreeAsync(scratch, st);
            if (e != cudaSuccess) return cuda_fail(e, "queued launch");
            return RKLT_OK;
        }
    }
    for (const Group &g : groups) {
        const size_t ib = g.items.size() * sizeof(BatchItem);
        const size_t pb = size_t(std::max<int64_t>(g.nunits, 1)) * sizeof(float);
        void *scratch = nullptr;
        if (cudaMallocFromPoolAsync(&scratch, ib + pb, pool, st) != cudaSuccess)
            return fail(RKLT_ERR_OOM, "scratch allocation failed");
        BatchItem *d_items = static_cast<BatchItem *>(scratch);
        float *partials = reinterpret_cast<float *>(static_cast<char *>(scratch) + ib);
        // descriptors through the pinned ring (an asynchronous copy); pageable if it is full
        cudaError_t e = copy_items(d_items, g.items.data(), ib, st);
        if (e == cudaSuccess)
            e = launch_group(N, g, d_items, partials, d_sse, d_psnr, 256, grid_for(N, 256, 1, g.nunits), st);
        cudaFreeAsync(scratch, st);
        if (e != cudaSuccess) return cuda_fail(e, "batched launch");
    }
    return RKLT_OK;
}

rklt_status rklt_batch_create(const rklt_item *h_items, int n, const rklt_plan *const *plans, int nplans,
                              double *d_sse, float *d_psnr, int flags, rklt_batch **out) {
    if (!out) return fail(RKLT_ERR_ARG, "out is NULL");
    *out = nullptr;
    if (!d_sse || !d_psnr) return fail(RKLT_ERR_ARG, "d_sse and d_psnr are required");
    rklt_batch *b = new (std::nothrow) rklt_batch;
    if (!b) return fail(RKLT_ERR_OOM, "host allocation failed");
    rklt_status s = build_groups(h_items, n, plans, nplans, b->groups, b->N);
    if (s != RKLT_OK) {
        delete b;
        return s;
    }
    b->sse = d_sse;
    b->psnr = d_psnr;
    {
        int dev = 0;
        cudaGetDevice(&dev);
        batch_smem_attrs(b->N, dev);   // before any capture of the launches
    }
    cudaError_t e = cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming);
    for (int k = 0; k < kBatchSideStreams && e == cudaSuccess; k++) {
        cudaStream_t s = nullptr;
        cudaEvent_t j = nullptr;
        e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
        if (e == cudaSuccess) b->side.push_back(s);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&j, cudaEventDisableTiming);
        if (e == cudaSuccess) b->join.push_back(j);
    }
    for (const Group &g : b->groups) {
        if (e != cudaSuccess) break;
        BatchItem *di = nullptr;
        float *dp = nullptr;
        e = cudaMalloc(&di, g.items.size() * sizeof(BatchItem));
        if (e == cudaSuccess) e = cudaMalloc(&dp, size_t(std::max<int64_t>(g.nunits, 1)) * sizeof(float));
        b->d_items.push_back(di);
        b->d_partials.push_back(dp);
        if (e == cudaSuccess)
            e = cudaMemcpy(di, g.items.data(), g.items.size() * sizeof(BatchItem), cudaMemcpyHostToDevice);
    }
    if (e != cudaSuccess) {
        batch_free(b);
        return e == cudaErrorMemoryAllocation ? fail(RKLT_ERR_OOM, "device allocation for the batch failed")
                                              : cuda_fail(e, "batch set-up");
    }
    // the whole batch as one queue for the persistent kernel (when every plan gets a
    // constant-memory slot)
    bool queue_ok = false;
    if (e == cudaSuccess) {
        std::vector<BatchItem> q, em;
        queue_ok = build_queue(b->groups, q, em, b->q_units);
        if (queue_ok) {
            b->q_items = int(q.size());
            b->q_empty = int(em.size());
            e = cudaMalloc(&b->dq_items, std::max<size_t>(q.size(), 1) * sizeof(BatchItem));
            if (e == cudaSuccess) e = cudaMalloc(&b->dq_empty, std::max<size_t>(em.size(), 1) * sizeof(BatchItem));
            if (e == cudaSuccess) e = cudaMalloc(&b->dq_partials, size_t(std::max<int64_t>(b->q_units, 1)) * 4);
            if (e == cudaSuccess && !q.empty())
                e = cudaMemcpy(b->dq_items, q.data(), q.size() * sizeof(BatchItem), cudaMemcpyHostToDevice);
            if (e == cudaSuccess && !em.empty())
                e = cudaMemcpy(b->dq_empty, em.data(), em.size() * sizeof(BatchItem), cudaMemcpyHostToDevice);
        }
    }
    if (e != cudaSuccess) {
        batch_free(b);
        return cuda_fail(e, "batch queue set-up");
    }
    // autotuner: time every candidate twice on the batch's own data and keep the
    // fastest.  Candidates: one persistent queue launch (threads per CTA x CTAs per
    // SM) and the grouped launches fanned over side streams (the same shapes).
    struct Cand {
        int mode, threads, per_sm;
    };
    std::vector<Cand> cands = {{0, 256, 1}, {0, 128, 2}, {0, 128, 1}, {0, 256, 2}};
    if (queue_ok) cands.insert(cands.end(), {{1, 256, 1}, {1, 128, 2}, {1, 128, 1}});
    if (!(flags & 1)) cands.resize(1);
    double best = 1e30;
    b->tuned.clear();
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    for (const Cand &c : cands) {
        if (batch_enqueue(b, c.mode, c.threads, c.per_sm, b->stream) != cudaSuccess) continue;  // warm-up
        cudaEventRecord(e0, b->stream);
        for (int rep = 0; rep < 2; rep++) batch_enqueue(b, c.mode, c.threads, c.per_sm, b->stream);
        cudaEventRecord(e1, b->stream);
        if (cudaEventSynchronize(e1) != cudaSuccess) continue;
        float ms = 0.0f;
        cudaEventElapsedTime(&ms, e0, e1);
        b->tuned.push_back({c.mode, c.threads, c.per_sm, ms / 2 * 1e3});
        if (ms / 2 < best) {
            best = ms / 2;
            b->mode = c.mode;
            b->threads = c.threads;
            b->per_sm = c.per_sm;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    b->tuned_us = (flags & 1) ? best * 1e3 : 0.0;
    // capture the chosen launch sequence once; runs replay the graph
    e = cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
        const cudaError_t le = batch_enqueue(b, b->mode, b->threads, b->per_sm, b->stream);
        e = cudaStreamEndCapture(b->stream, &b->graph);
        if (le != cudaSuccess) e = le;
    }
    if (e == cudaSuccess) e = cudaGraphInstantiate(&b->exec, b->graph, 0);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess) {
        batch_free(b);
        return cuda_fail(e, "batch graph capture");
    }
    *out = b;
    return RKLT_OK;
}

rklt_status rklt_batch_run(rklt_batch *b, void *stream) {
    if (!b) return fail(RKLT_ERR_ARG, "batch is NULL");
    const cudaError_t e = cudaGraphLaunch(b->exec, static_cast<cudaStream_t>(stream));
    return e == cudaSuccess ? RKLT_OK : cuda_fail(e, "graph launch");
}

rklt_status rklt_batch_info(const rklt_batch *b, int *threads, int *ctas_per_sm, int *groups, double *tuned_us,
                            int *mode) {
    if (!b) return fail(RKLT_ERR_ARG, "batch is NULL");
    if (threads) *threads = b->threads;
    if (ctas_per_sm) *ctas_per_sm = b->per_sm;
    if (groups) *groups = int(b->groups.size());
    if (tuned_us) *tuned_us = b->tuned_us;
    if (mode) *mode = b->mode;
    return RKLT_OK;
}

rklt_status rklt_batch_candidates(const rklt_batch *b, int *modes, int *threads, int *ctas_per_sm, double *us,
                                  int max_out, int *count) {
    if (!b || !count) return fail(RKLT_ERR_ARG, "batch and count are required");
    *count = int(b->tuned.size());
    for (int k = 0; k < *count && k < max_out; k++) {
        if (modes) modes[k] = b->tuned[size_t(k)].mode;
        if (threads) threads[k] = b->tuned[size_t(k)].threads;
        if (ctas_per_sm) ctas_per_sm[k] = b->tuned[size_t(k)].per_sm;
        if (us) us[k] = b->tuned[size_t(k)].us;
    }
    return RKLT_OK;
}

void rklt_batch_destroy(rklt_batch *b) {
    if (b && b->stream) cudaStreamSynchronize(b->stream);
    batch_free(b);
}

}  // extern "C"
