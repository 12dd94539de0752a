// rklt_fused_n8.cu -- fused kernel instantiated for 8 x 8 blocks.
#include "rklt_fused_impl.cuh"

namespace rklt {
rklt_status launch_fused_n8(const Plan &p, const FusedArgs &a, cudaStream_t st) { return launch_fused<8>(p, a, st); }
unsigned int take_status_n8() { return take_tu_status(); }
}  // namespace rklt
