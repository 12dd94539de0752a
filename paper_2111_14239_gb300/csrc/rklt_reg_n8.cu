// rklt_reg_n8.cu -- register path with the error by Parseval's identity, 8 x 8 blocks:
// the launcher and the kernels for diagonal bounds D = 0..3 (r <= 10).
#include "rklt_reg.cuh"

namespace rklt {
const void *pars_pick_n8_hi(int D, int out);  // D = 4, 5: rklt_reg_n8b.cu

static const void *pick_n8(int D, int out) {
    return D <= 3 ? pars_pick_range<8, 0, 3>(D, out) : pars_pick_n8_hi(D, out);
}

rklt_status launch_pars_n8(const Plan &p, const FusedArgs &a, cudaStream_t st) {
    if (!pars_applies<8>(p, a)) return RKLT_ERR_UNSUPPORTED;
    return launch_pars<8>(p, a, st, pick_n8);
}
unsigned int take_status_reg_n8() { return take_tu_status(); }
}  // namespace rklt
