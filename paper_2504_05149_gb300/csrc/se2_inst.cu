// Explicit instantiation of the kernels for one (real type, N): compiled once
// per pair with -DSE2_T=float|double -DSE2_N=<N> so that the units build in
// parallel.
#include "se2_inst.cuh"

#if !defined(SE2_T) || !defined(SE2_N)
#error "compile with -DSE2_T=<float|double> -DSE2_N=<N>"
#endif

namespace se2 {
template bool fill_n<SE2_T, SE2_N>(int M, KTable<SE2_T>* kt);
#if SE2_N == 8
template cudaError_t make_twiddles<SE2_T>(c2<SE2_T>*, int, cudaStream_t);
#endif
}  // namespace se2
