// rklt_reg_n8b.cu -- register path with the error by Parseval's identity, 8 x 8 blocks:
// the kernels for diagonal bounds D = 4, 5 (11 <= r <= 15).
#include "rklt_reg.cuh"

namespace rklt {
const void *pars_pick_n8_hi(int D, int out) { return pars_pick_range<8, 4, 5>(D, out); }
unsigned int take_status_reg_n8b() { return take_tu_status(); }
}  // namespace rklt
