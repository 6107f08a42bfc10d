// Template instantiation and run-time dispatch of the kernels for one real
// type.  Included once per real type by se2_inst_f32.cu / se2_inst_f64.cu.
#pragma once
#include "se2_internal.h"

namespace se2 {

template <typename T>
__global__ void k_twiddles(c2<T>* tw, int L) {
    const int n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n < L) {
        double s, c;
        sincospi(2.0 * n / L, &s, &c);        // exact argument for power-of-two L
        tw[n] = mk<T>((T)c, (T)(-s));
    }
}

template <typename T>
cudaError_t make_twiddles(c2<T>* tw, int L, cudaStream_t st) {
    k_twiddles<T><<<(L + 127) / 128, 128, 0, st>>>(tw, L);
    return cudaGetLastError();
}

template <typename T, int N, int M>
void fill_fused(KTable<T>* kt) {
    constexpr size_t sm = fused_smem<T, N, M>();
    kt->persist = nullptr;
    kt->persist_sep = nullptr;
    kt->smem_persist = 0;
    if constexpr (N >= 32 && M >= 8 && sm <= kMaxDynSmem) {
        kt->fwd_xt = k_fwd_xt<T, N, M>;
        kt->inv_tx = k_inv_tx<T, N, M>;
        kt->smem_xt = sm;
        if constexpr (sizeof(T) == 4) {
            kt->persist = k_conv_persist<T, N, M, LM_CONV>;
            kt->persist_sep = k_conv_persist<T, N, M, LM_SEP>;
            kt->smem_persist = sm > lines_smem<T, N>() ? sm : lines_smem<T, N>();
        }
    } else {
        kt->fwd_xt = nullptr;
        kt->inv_tx = nullptr;
        kt->smem_xt = 0;
    }
}

template <typename T, int M>
void fill_theta(KTable<T>* kt) {
    kt->t_fwd = k_lines<T, M, LM_FWD>;
    kt->t_inv = k_lines<T, M, LM_INV>;
    kt->smem_t = lines_smem<T, M>();
    kt->lines_t = kThreads / team_size<M>();
}

template <typename T, int N>
bool fill_n(int M, KTable<T>* kt) {
    kt->fwd_x = k_fwd_x<T, N>;
    kt->inv_x = k_inv_x<T, N>;
    kt->smem_x = xsplit_smem<T, N>();
    kt->teams_x = kThreads / team_size<N>();
    kt->y_conv = k_lines<T, N, LM_CONV>;
    kt->y_coef = k_lines<T, N, LM_COEF>;
    kt->y_adj = k_lines<T, N, LM_ADJ>;
    kt->y_sep = k_lines<T, N, LM_SEP>;
    kt->smem_y = lines_smem<T, N>();
    kt->lines_y = kThreads / team_size<N>();
    switch (M) {
        case 2: fill_fused<T, N, 2>(kt); fill_theta<T, 2>(kt); return true;
        case 4: fill_fused<T, N, 4>(kt); fill_theta<T, 4>(kt); return true;
        case 8: fill_fused<T, N, 8>(kt); fill_theta<T, 8>(kt); return true;
        case 16: fill_fused<T, N, 16>(kt); fill_theta<T, 16>(kt); return true;
        case 32: fill_fused<T, N, 32>(kt); fill_theta<T, 32>(kt); return true;
        case 64: fill_fused<T, N, 64>(kt); fill_theta<T, 64>(kt); return true;
        case 128: fill_fused<T, N, 128>(kt); fill_theta<T, 128>(kt); return true;
        default: return false;
    }
}

}  // namespace se2
