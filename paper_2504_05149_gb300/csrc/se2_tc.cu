// Instantiation of the tensor-core angular DFT kernels and host helpers.
#include <cmath>
#include <cstring>
#include <vector>

#include "se2_internal.h"
#include "se2_tc.cuh"

namespace se2 {

template <int M, int FMT>
static bool tc_pick(int dir, int split, TcKernel* k, size_t* sm) {
    if (dir < 0 && split == 3) { *k = k_theta_tc<M, -1, 3, FMT>; *sm = tc_smem<M, 3>(); return true; }
    if (dir > 0 && split == 3) { *k = k_theta_tc<M, +1, 3, FMT>; *sm = tc_smem<M, 3>(); return true; }
    if (FMT == 0 && dir < 0 && split == 1) { *k = k_theta_tc<M, -1, 1, 0>; *sm = tc_smem<M, 1>(); return true; }
    if (FMT == 0 && dir > 0 && split == 1) { *k = k_theta_tc<M, +1, 1, 0>; *sm = tc_smem<M, 1>(); return true; }
    return false;
}

bool tc_kernel(int M, int dir, int split, int fmt, TcKernel* out, size_t* smem) {
    if (M == 64) return fmt == 0 ? tc_pick<64, 0>(dir, split, out, smem) : tc_pick<64, 1>(dir, split, out, smem);
    if (M == 128) return fmt == 0 ? tc_pick<128, 0>(dir, split, out, smem) : tc_pick<128, 1>(dir, split, out, smem);
    return false;
}

// Host image of the constant operand: the real form of the 64-point DFT
// matrix in direction `dir`, B[n = 2m + a][k = 2l + b], split into 16-bit hi
// and lo (bf16 for fmt 0, fp16 for fmt 1), in the K-major core-matrix layout
// (hi operand, then lo operand).
void tc_dft_matrix(int dir, int fmt, std::vector<unsigned char>& img) {
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
                    const int off = tc_off(2 * m + aa, 2 * l + bb);
                    if (fmt == 0) {
                        const __nv_bfloat16 hi = __float2bfloat16_rn(v);
                        const __nv_bfloat16 lo = __float2bfloat16_rn((float)(vals[aa][bb] - (double)__bfloat162float(hi)));
                        std::memcpy(&img[off], &hi, 2);
                        std::memcpy(&img[kTcOpBytes + off], &lo, 2);
                    } else {
                        const __half hi = __float2half_rn(v);
                        const __half lo = __float2half_rn((float)(vals[aa][bb] - (double)__half2float(hi)));
                        std::memcpy(&img[off], &hi, 2);
                        std::memcpy(&img[kTcOpBytes + off], &lo, 2);
                    }
                }
        }
}

}  // namespace se2
