// Kernels of the FP32 path.
#include "se2_inst.cuh"

namespace se2 {
template <> bool get_kernels<float>(int N, int M, KTable<float>* kt) { return get_kernels_impl<float>(N, M, kt); }
template cudaError_t make_twiddles<float>(c2<float>*, int, cudaStream_t);
}  // namespace se2
