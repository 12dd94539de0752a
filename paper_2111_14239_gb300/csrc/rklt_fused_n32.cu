// rklt_fused_n32.cu -- fused kernels instantiated for 32 x 32 blocks: the warp-level
// tensor-core kernel and the FMA kernels of rklt_fused_impl.cuh, and the
// tensor-memory (tcgen05) kernel selected by rklt_set_tensor_engine(1).
#include "rklt_fused_impl.cuh"
#include "rklt_umma.cuh"

namespace rklt {
rklt_status launch_fused_n32(const Plan &p, const FusedArgs &a, cudaStream_t st) {
    if (uses_tmem_kernel(p, diag_bound(32, a.r), a.engine)) return launch_umma32(p, a, st);
    return launch_fused<32>(p, a, st);
}
unsigned int take_status_n32() { return take_tu_status(); }
}  // namespace rklt
