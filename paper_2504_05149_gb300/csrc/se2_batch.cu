// Instantiation of the one-launch batch kernel and its host-side geometry.
#include "se2_internal.h"

namespace se2 {

namespace {
template <int N, int M>
void units_nm(unsigned* nA, unsigned* nB, unsigned* nC, long long* s4) {
    *nA = (unsigned)(N / fast_yr<N, M>());
    *nC = *nA;
    *nB = (unsigned)((M * (N / 4 + 1) + fast_lines<N>() - 1) / fast_lines<N>());
    *s4 = (long long)M * N * ftp4<N>();
}
}  // namespace

bool batch_persist_units(int N, int M, unsigned* nA, unsigned* nB, unsigned* nC, long long* s4) {
    switch (batch_kind(N, M)) {
        case 0: units_nm<32, 16>(nA, nB, nC, s4); return true;
        case 1: units_nm<32, 32>(nA, nB, nC, s4); return true;
        case 2: units_nm<32, 64>(nA, nB, nC, s4); return true;
        case 3: units_nm<64, 16>(nA, nB, nC, s4); return true;
        case 4: units_nm<64, 32>(nA, nB, nC, s4); return true;
        case 5: units_nm<64, 64>(nA, nB, nC, s4); return true;
        case 6: units_nm<128, 16>(nA, nB, nC, s4); return true;
        case 7: units_nm<128, 32>(nA, nB, nC, s4); return true;
        case 8: units_nm<128, 64>(nA, nB, nC, s4); return true;
        case 9: units_nm<256, 16>(nA, nB, nC, s4); return true;
        case 10: units_nm<256, 32>(nA, nB, nC, s4); return true;
        case 11: units_nm<256, 64>(nA, nB, nC, s4); return true;
        default: return false;
    }
}

cudaError_t batch_persist_prepare(int* blocks_per_sm) {
    constexpr size_t smem = batch_persist_smem();
    static_assert(smem <= kMaxDynSmem, "the largest class fits one block");
    cudaError_t e = cudaFuncSetAttribute(kf_batch_persist<0>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, kf_batch_persist<0>, kThreads, smem);
    return e;
}

void launch_batch_persist(int grid, cudaStream_t s, const BPArgs& a) {
    kf_batch_persist<0><<<grid, kThreads, batch_persist_smem(), s>>>(a);
}

}  // namespace se2
