// se2_convolve_noalloc: the FP32 single-kernel convolution of se2_convolve
// for callers that cannot create a plan.  A plan reserves device memory with
// cudaMalloc when it is created; some callers are not allowed to do that at
// the point where they need a convolution (for example, code running inside a
// host framework's execution step that forbids device allocation, or code
// that must not risk the implicit device-wide synchronisation that
// cudaMalloc / cudaFree can cause).  This entry point allocates nothing: its
// twiddle tables and its spectrum scratch live in one fixed, file-scope device
// array that exists from the moment the library is loaded until the process
// exits, on every GPU that loads the library.
//
// The array holds 64 MiB: 8 KiB of twiddle tables for every power-of-two
// length 2..512, then the scratch spectrum.  A call processes its batch in
// chunks of as many problems as fit in the scratch; a single problem must fit
// (N = 256, M = 64 needs 18.9 MB; N = 512, M = 128 does not fit and is
// rejected).
#include <cuda_runtime.h>

#include <cstdint>
#include <cstdio>
#include <mutex>
#include <string>

#include "../../include/se2.h"
#include "se2_internal.h"

using namespace se2;

namespace {

constexpr size_t kNoAllocBytes = (size_t)64 << 20;
constexpr size_t kTwBytes = 8192;           // 1022 float2 twiddles, padded
constexpr int kMaxDevices = 64;

// The fixed scratch.  Device code could name it directly; host code must use
// the address cudaGetSymbolAddress returns for the current device (the
// symbol itself is only a host-side stand-in).
static __device__ __align__(256) unsigned char g_se2_noalloc[kNoAllocBytes];

struct DeviceSetup {
    std::once_flag once;
    cudaError_t err = cudaSuccess;
    unsigned char* base = nullptr;          // device address of g_se2_noalloc
};
DeviceSetup g_setup[kMaxDevices];

se2_status nfail(se2_status st, const std::string& msg) {
    set_last_error(msg.c_str());       // read back with se2_last_error()
    return st;
}

// Offset (in float2 elements) of the length-L table: tables for 2, 4, ...,
// L/2 come first and hold 2 + 4 + ... + L/2 = L - 2 elements.
int tw_offset(int L) { return L - 2; }

// Once per device, with that device current: resolve the array's device
// address and fill the twiddle tables (then wait for them, so that calls on
// any stream see them).
void setup_device(DeviceSetup* d) {
    void* ptr = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&ptr, g_se2_noalloc);
    if (e != cudaSuccess) { d->err = e; return; }
    float2* tw = reinterpret_cast<float2*>(ptr);
    for (int L = 2; L <= 512; L *= 2) {
        e = make_twiddles<float>(tw + tw_offset(L), L, 0);
        if (e != cudaSuccess) { d->err = e; return; }
    }
    e = cudaDeviceSynchronize();
    if (e != cudaSuccess) { d->err = e; return; }
    d->base = reinterpret_cast<unsigned char*>(ptr);
}

}  // namespace

extern "C" se2_status se2_convolve_noalloc(const void* f, const void* coeffs, void* out, int N, int M, int B,
                                           void* stream) {
    if (f == nullptr || coeffs == nullptr || out == nullptr)
        return nfail(SE2_ERR_INVALID_ARG, "se2_convolve_noalloc: NULL pointer argument");
    if (N < 8 || N > 512 || (N & (N - 1)) || M < 2 || M > 128 || (M & (M - 1)))
        return nfail(SE2_ERR_UNSUPPORTED, "se2_convolve_noalloc: N must be a power of two in [8, 512] and M in [2, 128]");
    if (B < 1) return nfail(SE2_ERR_INVALID_ARG, "se2_convolve_noalloc: B must be >= 1");
    if (((uintptr_t)f % 4) || ((uintptr_t)out % 4) || ((uintptr_t)coeffs % 8))
        return nfail(SE2_ERR_INVALID_ARG, "se2_convolve_noalloc: misaligned pointer");
    if (f == out) return nfail(SE2_ERR_INVALID_ARG, "se2_convolve_noalloc: out aliases f");

    const int tp = ((N / 2 + 1) + 15) / 16 * 16;
    const size_t s_pstride = (size_t)M * N * tp;                  // complex elements per problem
    const size_t per = s_pstride * sizeof(float2);
    const size_t room = kNoAllocBytes - kTwBytes;
    if (per > room) {
        char buf[256];
        snprintf(buf, sizeof buf,
                 "se2_convolve_noalloc: one N=%d M=%d problem needs %zu bytes of scratch, more than the fixed %zu",
                 N, M, per, room);
        return nfail(SE2_ERR_UNSUPPORTED, buf);
    }
    KTable<float> kt;
    if (!get_kernels<float>(N, M, &kt)) return nfail(SE2_ERR_UNSUPPORTED, "se2_convolve_noalloc: no kernels for this size");

    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess || dev < 0 || dev >= kMaxDevices)
        return nfail(SE2_ERR_CUDA, "se2_convolve_noalloc: no usable current device");
    DeviceSetup* d = &g_setup[dev];
    std::call_once(d->once, setup_device, d);
    if (d->err != cudaSuccess)
        return nfail(SE2_ERR_CUDA, std::string("se2_convolve_noalloc: set-up failed: ") + cudaGetErrorString(d->err));

    // smem limits of the kernels this size uses (no allocation)
    const void* fns[] = {(const void*)kt.fwd_xt, (const void*)kt.inv_tx, (const void*)kt.fwd_x, (const void*)kt.inv_x,
                         (const void*)kt.y_conv, (const void*)kt.t_fwd, (const void*)kt.t_inv};
    const size_t sms[] = {kt.smem_xt, kt.smem_xt, kt.smem_x, kt.smem_x, kt.smem_y, kt.smem_t, kt.smem_t};
    for (int i = 0; i < 7; ++i) {
        if (fns[i] == nullptr) continue;
        e = cudaFuncSetAttribute(fns[i], cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sms[i]);
        if (e != cudaSuccess) return nfail(SE2_ERR_CUDA, std::string("se2_convolve_noalloc: ") + cudaGetErrorString(e));
    }

    const float2* twN = reinterpret_cast<const float2*>(d->base) + tw_offset(N);
    const float2* twM = reinterpret_cast<const float2*>(d->base) + tw_offset(M);
    float2* scratch = reinterpret_cast<float2*>(d->base + kTwBytes);
    const int chunk = (int)(room / per);
    const size_t g = (size_t)N * N * M;
    const long long cps = (long long)M * N * (N / 2 + 1);
    cudaStream_t st = (cudaStream_t)stream;
    const bool fused = kt.fwd_xt != nullptr;

    // Nothing in the scratch has to start at zero: every scratch element this
    // sequence reads was written earlier in the same chunk.
    for (int c0 = 0; c0 < B; c0 += chunk) {
        const int nb = (B - c0 < chunk) ? (B - c0) : chunk;
        XArgs<float> xa{};
        xa.f = (const float*)f + c0 * g;
        xa.out = (float*)out + c0 * g;
        xa.g_pstride = g;
        xa.s = scratch;
        xa.s_pstride = s_pstride;
        xa.tp = tp;
        xa.M = M;
        xa.twN = twN;
        xa.twM = twM;
        LArgs<float> tl{};                       // theta lines (split sizes)
        tl.s = scratch;
        tl.s_pstride = s_pstride;
        tl.outer_stride = tp;
        tl.elem_stride = (long long)N * tp;
        tl.n_outer = N;
        tl.nk = N / 2;
        tl.N = N;
        tl.tw = twM;
        const long long tlines = (long long)N * (N / 2 + 1);
        const unsigned tblocks = kt.lines_t ? (unsigned)((tlines + kt.lines_t - 1) / kt.lines_t) : 0;
        const int pairs = M / 2;
        if (fused) {
            kt.fwd_xt<<<dim3(N, nb), kThreads, kt.smem_xt, st>>>(xa);
        } else {
            kt.fwd_x<<<dim3(N, (pairs + kt.teams_x - 1) / kt.teams_x, nb), kThreads, kt.smem_x, st>>>(xa);
            kt.t_fwd<<<dim3(tblocks, nb), kThreads, kt.smem_t, st>>>(tl);
        }
        LArgs<float> yl{};
        yl.s = scratch;
        yl.s_pstride = s_pstride;
        yl.outer_stride = (long long)N * tp;
        yl.elem_stride = tp;
        yl.n_outer = M;
        yl.nk = N / 2;
        yl.N = N;
        yl.tw = twN;
        yl.cp = N / 2 + 1;
        yl.inv_L = 1.0 / ((double)N * N * M);
        yl.wsign = 1;                      // grids on Omega_L
        yl.k = 1;
        yl.C[0] = (const float2*)coeffs + c0 * cps;
        yl.ls[0] = nullptr;
        yl.c_pstride = cps;
        yl.ls_pstride = 1;
        const long long ylines = (long long)M * (N / 2 + 1);
        kt.y_conv<<<dim3((unsigned)((ylines + kt.lines_y - 1) / kt.lines_y), nb), kThreads, kt.smem_y, st>>>(yl);
        if (fused) {
            kt.inv_tx<<<dim3(N, nb), kThreads, kt.smem_xt, st>>>(xa);
        } else {
            kt.t_inv<<<dim3(tblocks, nb), kThreads, kt.smem_t, st>>>(tl);
            kt.inv_x<<<dim3(N, (pairs + kt.teams_x - 1) / kt.teams_x, nb), kThreads, kt.smem_x, st>>>(xa);
        }
    }
    e = cudaGetLastError();
    if (e != cudaSuccess) return nfail(SE2_ERR_CUDA, std::string("se2_convolve_noalloc: launch failed: ") + cudaGetErrorString(e));
    return SE2_OK;
}
