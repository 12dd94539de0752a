// rklt_fmssim_n4.cu -- the fused pass with the structural similarity, N = 4
// (every diagonal bound).
#include "rklt_fmssim.cuh"

namespace rklt {
rklt_status launch_fm_n4(const Plan &plan, const FmArgs &a, cudaStream_t st) { return launch_fm<4, 0, 7>(plan, a, st); }
unsigned int take_status_fm_n4() { return take_tu_status(); }
}  // namespace rklt
