// rklt_fused_n16.cu -- fused kernel instantiated for 16 x 16 blocks.
#include "rklt_fused_impl.cuh"

namespace rklt {
rklt_status launch_fused_n16(const Plan &p, const FusedArgs &a, cudaStream_t st) { return launch_fused<16>(p, a, st); }
unsigned int take_status_n16() { return take_tu_status(); }
}  // namespace rklt
