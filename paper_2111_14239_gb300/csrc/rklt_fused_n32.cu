// rklt_fused_n32.cu -- fused kernel instantiated for 32 x 32 blocks.
#include "rklt_fused_impl.cuh"

namespace rklt {
rklt_status launch_fused_n32(const Plan &p, const FusedArgs &a, cudaStream_t st) { return launch_fused<32>(p, a, st); }
unsigned int take_status_n32() { return take_tu_status(); }
}  // namespace rklt
