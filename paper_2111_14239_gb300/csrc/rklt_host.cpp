// rklt_host.cpp -- host helpers of the CUDA launchers: error plumbing, the
// per-device scratch pool, SM counts, shared-memory opt-in and TMA descriptors.
#include <cudaTypedefs.h>

#include <atomic>
#include <map>
#include <mutex>
#include <set>
#include <tuple>
#include <utility>

#include "rklt_internal.h"

namespace rklt {

static std::atomic<int> g_transport{0};
static std::atomic<int> g_tensor_engine{0};
static std::atomic<int> g_inject_stall{0};

int transport_mode() { return g_transport.load(std::memory_order_relaxed); }
int tensor_engine() { return g_tensor_engine.load(std::memory_order_relaxed); }
int inject_stall() { return g_inject_stall.load(std::memory_order_relaxed); }

rklt_status cuda_fail(cudaError_t err, const char *what) {
    return fail(RKLT_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(err));
}

cudaMemPool_t scratch_pool() {
    static std::mutex mu;
    static cudaMemPool_t pools[64] = {};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return nullptr;
    std::lock_guard<std::mutex> lk(mu);
    if (!pools[dev]) {
        cudaMemPoolProps props = {};
        props.allocType = cudaMemAllocationTypePinned;
        props.location.type = cudaMemLocationTypeDevice;
        props.location.id = dev;
        cudaMemPool_t p;
        if (cudaMemPoolCreate(&p, &props) != cudaSuccess) return nullptr;
        uint64_t keep = ~0ull;  // keep freed scratch cached in the pool
        cudaMemPoolSetAttribute(p, cudaMemPoolAttrReleaseThreshold, &keep);
        pools[dev] = p;
    }
    return pools[dev];
}

int sm_count(int dev) {
    static std::mutex mu;
    static int cache[64] = {};
    std::lock_guard<std::mutex> lk(mu);
    if (dev >= 0 && dev < 64 && cache[dev]) return cache[dev];
    int n = 0;
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    if (dev >= 0 && dev < 64) cache[dev] = n;
    return n;
}

int ensure_smem_attr(const void *kernel) {
    static std::mutex mu;
    static std::set<std::pair<int, const void *>> done;
    int dev = 0;
    cudaGetDevice(&dev);
    std::lock_guard<std::mutex> lk(mu);
    if (done.insert({dev, kernel}).second)
        cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
    return dev;
}

int occupancy(const void *kernel, int threads, size_t smem) {
    static std::mutex mu;
    static std::map<std::tuple<int, const void *, int, size_t>, int> cache;
    int dev = 0;
    cudaGetDevice(&dev);
    const auto key = std::make_tuple(dev, kernel, threads, smem);
    std::lock_guard<std::mutex> lk(mu);
    const auto f = cache.find(key);
    if (f != cache.end()) return f->second;
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, kernel, threads, smem) != cudaSuccess) n = 0;
    cache.emplace(key, n);
    return n;
}

static PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        cudaDriverEntryPointQueryResult q;
        void *p = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    });
    return fn;
}

namespace {

// Recent tensor-map encodings: a descriptor is a pure function of its arguments, so
// repeated calls on the same buffers (a serving or benchmark loop) reuse it instead
// of encoding it again on the host.
struct MapKey {
    const void *base;
    int W, H, nimg;
    int64_t ld, stride;
    int box_w, box_h;
    bool swz;
    bool operator==(const MapKey &o) const {
        return base == o.base && W == o.W && H == o.H && nimg == o.nimg && ld == o.ld && stride == o.stride &&
               box_w == o.box_w && box_h == o.box_h && swz == o.swz;
    }
};
constexpr int kMapCache = 16;
std::mutex g_map_mu;
MapKey g_map_key[kMapCache];
CUtensorMap g_map_val[kMapCache];
int g_map_used = 0, g_map_next = 0;

}  // namespace

// 3-D uint8 tensor map (x = column, y = row, z = image) with a box_w x box_h x 1 box.
bool make_map_u8(CUtensorMap *m, const void *base, int W, int H, int nimg, int64_t ld, int64_t stride, int box_w,
                 int box_h, bool swizzle128) {
    const MapKey key{base, W, H, nimg, ld, stride, box_w, box_h, swizzle128};
    {
        std::lock_guard<std::mutex> lk(g_map_mu);
        for (int k = 0; k < g_map_used; k++)
            if (g_map_key[k] == key) {
                *m = g_map_val[k];
                return true;
            }
    }
    auto fn = encode_fn();
    if (!fn) return false;
    cuuint64_t dims[3] = {cuuint64_t(W), cuuint64_t(H), cuuint64_t(nimg)};
    cuuint64_t strides[2] = {cuuint64_t(ld), cuuint64_t(stride)};
    cuuint32_t box[3] = {cuuint32_t(box_w), cuuint32_t(box_h), 1};
    cuuint32_t estr[3] = {1, 1, 1};
    const bool ok = fn(m, CU_TENSOR_MAP_DATA_TYPE_UINT8, 3, const_cast<void *>(base), dims, strides, box, estr,
                       CU_TENSOR_MAP_INTERLEAVE_NONE,
                       swizzle128 ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_NONE,
                       CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
    if (ok) {
        std::lock_guard<std::mutex> lk(g_map_mu);
        g_map_key[g_map_next] = key;
        g_map_val[g_map_next] = *m;
        g_map_next = (g_map_next + 1) % kMapCache;
        if (g_map_used < kMapCache) g_map_used++;
    }
    return ok;
}

}  // namespace rklt

extern "C" void rklt_set_transport(int mode) { rklt::g_transport.store(mode == 1 ? 1 : 0); }
extern "C" void rklt_set_tensor_engine(int mode) { rklt::g_tensor_engine.store(mode == 1 ? 1 : 0); }
extern "C" void rklt_debug_inject_stall(int on) { rklt::g_inject_stall.store(on ? 1 : 0); }
