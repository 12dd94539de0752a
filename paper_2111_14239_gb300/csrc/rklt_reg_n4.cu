// rklt_reg_n4.cu -- register path with the error by Parseval's identity, 4 x 4 blocks.
#include "rklt_reg.cuh"

namespace rklt {
rklt_status launch_pars_n4(const Plan &p, const FusedArgs &a, cudaStream_t st) {
    if (!pars_applies<4>(p, a)) return RKLT_ERR_UNSUPPORTED;
    return launch_pars<4>(p, a, st, pars_pick_range<4, 0, 7>);
}
unsigned int take_status_reg_n4() { return take_tu_status(); }
}  // namespace rklt
