// Instantiation of the tensor-core angular DFT kernels and host helpers.
#include <cmath>
#include <cstring>
#include <vector>

#include "se2_internal.h"
#include "se2_tc.cuh"

namespace se2 {

bool tc_kernel(int M, int dir, int split, TcKernel* out, size_t* smem) {
    TcKernel k = nullptr;
    size_t sm = 0;
    if (M == 64 && dir < 0 && split == 3) { k = k_theta_tc<64, -1, 3>; sm = tc_smem<64, 3>(); }
    else if (M == 64 && dir > 0 && split == 3) { k = k_theta_tc<64, +1, 3>; sm = tc_smem<64, 3>(); }
    else if (M == 64 && dir < 0 && split == 1) { k = k_theta_tc<64, -1, 1>; sm = tc_smem<64, 1>(); }
    else if (M == 64 && dir > 0 && split == 1) { k = k_theta_tc<64, +1, 1>; sm = tc_smem<64, 1>(); }
    else if (M == 128 && dir < 0 && split == 3) { k = k_theta_tc<128, -1, 3>; sm = tc_smem<128, 3>(); }
    else if (M == 128 && dir > 0 && split == 3) { k = k_theta_tc<128, +1, 3>; sm = tc_smem<128, 3>(); }
    else if (M == 128 && dir < 0 && split == 1) { k = k_theta_tc<128, -1, 1>; sm = tc_smem<128, 1>(); }
    else if (M == 128 && dir > 0 && split == 1) { k = k_theta_tc<128, +1, 1>; sm = tc_smem<128, 1>(); }
    else return false;
    *out = k;
    *smem = sm;
    return true;
}

// Host image of the constant operand: the real form of the 64-point DFT
// matrix in direction `dir`, B[n = 2m + a][k = 2l + b], split into bf16 hi and
// lo, in the K-major core-matrix layout (hi operand, then lo operand).
void tc_dft_matrix(int dir, std::vector<unsigned char>& img) {
    img.assign(2 * kTcOpBytes, 0);
    const double PI = 3.14159265358979323846;
    for (int m = 0; m < 64; ++m)
        for (int l = 0; l < 64; ++l) {
            const int ml = (m * l) % 64;
            const double c = std::cos(2 * PI * ml / 64.0), s = dir * std::sin(2 * PI * ml / 64.0);
            const double vals[2][2] = {{c, -s}, {s, c}};        // [a][b]
            for (int aa = 0; aa < 2; ++aa)
                for (int bb = 0; bb < 2; ++bb) {
                    const float v = (float)vals[aa][bb];
                    const __nv_bfloat16 hi = __float2bfloat16_rn(v);
                    const __nv_bfloat16 lo = __float2bfloat16_rn((float)(vals[aa][bb] - (double)__bfloat162float(hi)));
                    const int off = tc_off(2 * m + aa, 2 * l + bb);
                    std::memcpy(&img[off], &hi, 2);
                    std::memcpy(&img[kTcOpBytes + off], &lo, 2);
                }
        }
}

}  // namespace se2
