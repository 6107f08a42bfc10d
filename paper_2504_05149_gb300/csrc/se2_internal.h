// Internal declarations shared by the C-ABI implementation and the kernel
// instantiation units.
#pragma once
#include <cuda_runtime.h>
#include <stddef.h>

#include <vector>

#include "se2_flow.cuh"
#include "se2_batch_persist.cuh"

namespace se2 {

constexpr size_t kMaxDynSmem = 226 * 1024;   // opt-in limit per block minus static use

template <typename T>
struct KTable {
    using XK = void (*)(XArgs<T>);
    using LK = void (*)(LArgs<T>);
    XK fwd_xt = nullptr, inv_tx = nullptr;   // fused x+theta (null: use split path)
    size_t smem_xt = 0;
    XK fwd_x = nullptr, inv_x = nullptr;     // split path, x only
    size_t smem_x = 0;
    LK y_conv = nullptr, y_coef = nullptr, y_adj = nullptr, y_sep = nullptr;   // lines of length N along y
    size_t smem_y = 0;
    int lines_y = 0;                          // lines per block
    LK t_fwd = nullptr, t_inv = nullptr;     // lines of length M along theta
    size_t smem_t = 0;
    int lines_t = 0;
    int teams_x = 0;                          // row pairs per block (split fwd_x/inv_x)
    using PK = void (*)(PArgs<T>);
    PK persist = nullptr;                     // persistent convolution (null: three kernels)
    PK persist_sep = nullptr;                 // same with separable coefficient tables
    size_t smem_persist = 0;
};

// Fills the kernel table for (N, M); false if M is unsupported.  Defined in
// se2_inst.cuh and instantiated per (T, N) by se2_inst.cu.
template <typename T, int N>
bool fill_n(int M, KTable<T>* kt);

template <typename T>
bool get_kernels(int N, int M, KTable<T>* kt) {
    switch (N) {
        case 8: return fill_n<T, 8>(M, kt);
        case 16: return fill_n<T, 16>(M, kt);
        case 32: return fill_n<T, 32>(M, kt);
        case 64: return fill_n<T, 64>(M, kt);
        case 128: return fill_n<T, 128>(M, kt);
        case 256: return fill_n<T, 256>(M, kt);
        case 512: return fill_n<T, 512>(M, kt);
        default: return false;
    }
}

// FP32 paired-FFT convolution kernels (se2_fast.cu), N in {32, 64, 128, 256},
// M in {8, ..., 128}.
struct FastTable {
    using FK = void (*)(FArgs);
    FK fwd = nullptr, lines = nullptr, lines_sep = nullptr, lines_fwd = nullptr, lines_adj = nullptr, lines_acc = nullptr,
       inv = nullptr;
    size_t smem_xt = 0, smem_y = 0;
    int lines_per_block = 0;
    int yr = 1;                  // y rows per block of fwd and inv (grid N / yr)
    // units A and C with bulk row copies and the real-FFT split in registers
    // (se2_fast2.cuh, N = 64, 256); they copy rows of f and out, so a call
    // whose f (or out) is not 16-byte aligned runs fwd (or inv) instead
    FK fwd2 = nullptr, inv2 = nullptr;
    size_t smem_xt2 = 0;
    // the whole convolution of a batch as one persistent dataflow launch
    // (se2_flow.cuh); null where (N, M) has none
    void (*flow)(FlowArgs) = nullptr;
    size_t smem_flow = 0;
};
template <int N>
bool get_fast_n(int M, FastTable* t);
bool get_fast(int N, int M, FastTable* t);   // se2_capi.cu

// Tensor-core angular DFT (se2_tc.cu).
struct TcArgs;
using TcKernel = void (*)(TcArgs);
bool tc_kernel(int M, int dir, int split, int fmt, TcKernel* out, size_t* smem);
void tc_dft_matrix(int dir, int fmt, std::vector<unsigned char>& img);

// The one-launch batch kernel (se2_batch.cu): its launch, and its unit
// counts per problem for (N, M) (false where the kernel has no such class).
void launch_batch_persist(int grid, cudaStream_t s, const BPArgs& a);
cudaError_t batch_persist_prepare(int* blocks_per_sm);
bool batch_persist_units(int N, int M, unsigned* nA, unsigned* nB, unsigned* nC, long long* s_pstride4);

// Device allocations of the library (plans, grid plans): counted, and made
// to fail on request (se2_debug_alloc_stats, se2_debug_fail_alloc).
cudaError_t dev_alloc(void** p, size_t bytes);
void dev_free(void* p);

// Sets the thread-local text returned by se2_last_error().
void set_last_error(const char* msg);

// FP64 twiddle generation (sincospi), rounded to T.
template <typename T>
cudaError_t make_twiddles(c2<T>* tw, int L, cudaStream_t st);

template <typename T, int N, int M>
constexpr size_t fused_smem() {
    return ((size_t)slab_elems<M, slab_pitch<N>()>() + (size_t)(kThreads / team_size<N>()) * xbuf_elems<N>()) * sizeof(c2<T>);
}
template <typename T, int N>
constexpr size_t xsplit_smem() {
    return (size_t)(kThreads / team_size<N>()) * xbuf_elems<N>() * sizeof(c2<T>);
}
template <typename T, int L>
constexpr size_t lines_smem() {   // no exchange buffer when one lane holds a line
    return Fac<L>::R2 == 1 ? 0 : (size_t)(kThreads / team_size<L>()) * ((Fac<L>::R1 * (Fac<L>::R2 + 1)) | 1) * sizeof(c2<T>);
}

}  // namespace se2
