// Kernels of the FP64 path.
#include "se2_inst.cuh"

namespace se2 {
template <> bool get_kernels<double>(int N, int M, KTable<double>* kt) { return get_kernels_impl<double>(N, M, kt); }
template cudaError_t make_twiddles<double>(c2<double>*, int, cudaStream_t);
}  // namespace se2
