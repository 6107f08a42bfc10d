// Instantiation of the FP32 paired-FFT convolution kernels for one N
// (compiled once per N with -DSE2_FN=<N>, in parallel).
#include "se2_internal.h"

#if !defined(SE2_FN)
#error "compile with -DSE2_FN=<N>"
#endif

namespace se2 {

namespace {
template <int N, int M>
bool fill_fast_nm(FastTable* t) {
    constexpr size_t sx = fast_xt_smem<N, M>(), sy = fast_lines_smem<N, M>();
    if constexpr (sx <= kMaxDynSmem && sy <= kMaxDynSmem) {
        t->fwd = kf_fwd_xt<N, M>;
        t->lines = kf_lines<N, M, FL_CONV>;
        t->lines_sep = kf_lines<N, M, FL_SEP>;
        t->lines_fwd = kf_lines<N, M, FL_FWD>;
        t->lines_adj = kf_lines<N, M, FL_ADJ>;
        t->lines_acc = kf_lines<N, M, FL_ACC>;
        t->inv = kf_inv_tx<N, M>;
        t->smem_xt = sx;
        t->smem_y = sy;
        t->lines_per_block = fast_lines<N>();
        t->yr = fast_yr<N, M>();
        if constexpr (fast2_ok<N>()) {
            constexpr size_t s2 = fast2_smem<N, M>();
            if constexpr (s2 <= kMaxDynSmem) {
                t->fwd2 = kf2_fwd_xt<N, M>;
                t->inv2 = kf2_inv_tx<N, M>;
                t->smem_xt2 = s2;
            }
        }
        if constexpr (flow_ok<N, M>()) {
            t->flow = kflow_conv<N, M>;
            t->smem_flow = FlowGeom<N, M>::SMEM;
        }
        return true;
    }
    return false;
}
}  // namespace

template <int N>
bool get_fast_n(int M, FastTable* t) {
    switch (M) {
        case 8: return fill_fast_nm<N, 8>(t);
        case 16: return fill_fast_nm<N, 16>(t);
        case 32: return fill_fast_nm<N, 32>(t);
        case 64: return fill_fast_nm<N, 64>(t);
        case 128: return fill_fast_nm<N, 128>(t);
        default: return false;
    }
}
template bool get_fast_n<SE2_FN>(int M, FastTable* t);

}  // namespace se2
