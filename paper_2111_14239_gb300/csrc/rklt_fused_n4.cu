// rklt_fused_n4.cu -- fused kernel instantiated for 4 x 4 blocks.
#include "rklt_fused_impl.cuh"

namespace rklt {
rklt_status launch_fused_n4(const Plan &p, const FusedArgs &a, cudaStream_t st) { return launch_fused<4>(p, a, st); }
unsigned int take_status_n4() { return take_tu_status(); }
}  // namespace rklt
