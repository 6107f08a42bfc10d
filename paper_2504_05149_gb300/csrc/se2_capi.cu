// C ABI of the SE(2) convolution library (declared in include/se2.h).
//
// Host side: argument validation, plan (twiddle tables, scratch), and the
// launch sequences of Algorithm 3 (se2_convolve), Algorithms 4/6
// (se2_convolve_chain) and the coefficient transform (se2_coeffs, Eq. FkLv).
#include <cuda_runtime.h>

#include <cstdarg>
#include <cstdint>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>
#include <string>

#include "../../include/se2.h"
#include "se2_internal.h"

using namespace se2;

namespace {

thread_local std::string g_err = "no error";

se2_status fail(se2_status st, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_err = buf;
    return st;
}

se2_status cuda_fail(cudaError_t e, const char* what) {
    return fail(SE2_ERR_CUDA, "%s: %s (%s)", what, cudaGetErrorName(e), cudaGetErrorString(e));
}

bool is_pow2(int v) { return v > 0 && (v & (v - 1)) == 0; }

struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev) {
        if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
        if (prev != dev) cudaSetDevice(dev);
    }
    ~DeviceGuard() {
        int cur = -1;
        if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
    }
};

}  // namespace

struct se2_plan_s {
    int N = 0, M = 0, batch = 0, dev = 0;
    se2_precision prec = SE2_F32;
    unsigned flags = 0;
    int tp = 0;                 // scratch row pitch (complex elements)
    size_t s_pstride = 0;       // complex elements per problem in scratch
    int chunk = 0;              // problems per scratch pass
    size_t elem = 0;            // bytes per complex element
    void* scratch = nullptr;
    void* twN = nullptr;
    void* twM = nullptr;
    double* abs_sum = nullptr;  // [chunk]
    size_t ws_bytes = 0;
    KTable<float> kf;
    KTable<double> kd;
    bool fused = false;
};

namespace {

template <typename T>
KTable<T>& table(se2_plan_s* p);
template <>
KTable<float>& table<float>(se2_plan_s* p) { return p->kf; }
template <>
KTable<double>& table<double>(se2_plan_s* p) { return p->kd; }

template <typename T>
se2_status set_smem(const KTable<T>& kt) {
    struct { const void* fn; size_t sm; } list[] = {
        {(const void*)kt.fwd_xt, kt.smem_xt}, {(const void*)kt.inv_tx, kt.smem_xt},
        {(const void*)kt.fwd_x, kt.smem_x},   {(const void*)kt.inv_x, kt.smem_x},
        {(const void*)kt.y_conv, kt.smem_y},  {(const void*)kt.y_coef, kt.smem_y},
        {(const void*)kt.t_fwd, kt.smem_t},   {(const void*)kt.t_inv, kt.smem_t},
    };
    for (auto& e : list) {
        if (e.fn == nullptr) continue;
        cudaError_t r = cudaFuncSetAttribute(e.fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)e.sm);
        if (r != cudaSuccess) return cuda_fail(r, "cudaFuncSetAttribute");
    }
    return SE2_OK;
}

template <typename T>
se2_status plan_init(se2_plan_s* p) {
    KTable<T>& kt = table<T>(p);
    if (!get_kernels<T>(p->N, p->M, &kt))
        return fail(SE2_ERR_UNSUPPORTED, "no kernels for N=%d M=%d", p->N, p->M);
    // SE2_FORCE_SPLIT=1 (environment) selects the separate x / theta passes
    // even where the fused slab kernels exist (used to test both paths).
    const char* split = getenv("SE2_FORCE_SPLIT");
    p->fused = kt.fwd_xt != nullptr && !(split && split[0] == '1');
    se2_status st = set_smem<T>(kt);
    if (st != SE2_OK) return st;
    p->elem = sizeof(c2<T>);
    cudaError_t e;
    if ((e = cudaMalloc(&p->twN, sizeof(c2<T>) * p->N)) != cudaSuccess) return fail(SE2_ERR_OOM, "twiddles: %s", cudaGetErrorString(e));
    if ((e = cudaMalloc(&p->twM, sizeof(c2<T>) * p->M)) != cudaSuccess) return fail(SE2_ERR_OOM, "twiddles: %s", cudaGetErrorString(e));
    if ((e = make_twiddles<T>((c2<T>*)p->twN, p->N, 0)) != cudaSuccess) return cuda_fail(e, "twiddle kernel");
    if ((e = make_twiddles<T>((c2<T>*)p->twM, p->M, 0)) != cudaSuccess) return cuda_fail(e, "twiddle kernel");
    return SE2_OK;
}

void plan_free(se2_plan_s* p) {
    if (p->scratch) cudaFree(p->scratch);
    if (p->twN) cudaFree(p->twN);
    if (p->twM) cudaFree(p->twM);
    if (p->abs_sum) cudaFree(p->abs_sum);
    p->scratch = p->twN = p->twM = nullptr;
    p->abs_sum = nullptr;
}

bool aligned(const void* ptr, size_t a) { return ((uintptr_t)ptr % a) == 0; }

// ---------------------------------------------------------------------------
// Launch helpers
// ---------------------------------------------------------------------------
template <typename T>
XArgs<T> xargs(se2_plan_s* p) {
    XArgs<T> a{};
    a.s = (c2<T>*)p->scratch;
    a.s_pstride = p->s_pstride;
    a.tp = p->tp;
    a.M = p->M;
    a.g_pstride = (size_t)p->N * p->N * p->M;
    a.twN = (const c2<T>*)p->twN;
    a.twM = (const c2<T>*)p->twM;
    return a;
}

// Forward x and theta transforms of nb real grids into the scratch.
template <typename T>
void launch_forward(se2_plan_s* p, const T* f, int nb, double* abs_sum, cudaStream_t st) {
    KTable<T>& kt = table<T>(p);
    XArgs<T> a = xargs<T>(p);
    a.f = f;
    a.abs_sum = abs_sum;
    if (p->fused) {
        kt.fwd_xt<<<dim3(p->N, nb), kThreads, kt.smem_xt, st>>>(a);
    } else {
        const int pairs = p->M / 2;
        kt.fwd_x<<<dim3(p->N, (pairs + kt.teams_x - 1) / kt.teams_x, nb), kThreads, kt.smem_x, st>>>(a);
        LArgs<T> l{};
        l.s = (c2<T>*)p->scratch;
        l.s_pstride = p->s_pstride;
        l.outer_stride = p->tp;                      // outer = y
        l.elem_stride = (long long)p->N * p->tp;     // along theta
        l.n_outer = p->N;
        l.nk = p->N / 2;
        l.N = p->N;
        l.tw = (const c2<T>*)p->twM;
        const long long lines = (long long)p->N * (p->N / 2 + 1);
        kt.t_fwd<<<dim3((unsigned)((lines + kt.lines_t - 1) / kt.lines_t), nb), kThreads, kt.smem_t, st>>>(l);
    }
}

template <typename T>
void launch_inverse(se2_plan_s* p, T* out, int nb, cudaStream_t st) {
    KTable<T>& kt = table<T>(p);
    XArgs<T> a = xargs<T>(p);
    a.out = out;
    if (p->fused) {
        kt.inv_tx<<<dim3(p->N, nb), kThreads, kt.smem_xt, st>>>(a);
    } else {
        LArgs<T> l{};
        l.s = (c2<T>*)p->scratch;
        l.s_pstride = p->s_pstride;
        l.outer_stride = p->tp;
        l.elem_stride = (long long)p->N * p->tp;
        l.n_outer = p->N;
        l.nk = p->N / 2;
        l.N = p->N;
        l.tw = (const c2<T>*)p->twM;
        const long long lines = (long long)p->N * (p->N / 2 + 1);
        kt.t_inv<<<dim3((unsigned)((lines + kt.lines_t - 1) / kt.lines_t), nb), kThreads, kt.smem_t, st>>>(l);
        const int pairs = p->M / 2;
        kt.inv_x<<<dim3(p->N, (pairs + kt.teams_x - 1) / kt.teams_x, nb), kThreads, kt.smem_x, st>>>(a);
    }
}

template <typename T>
LArgs<T> yargs(se2_plan_s* p) {
    LArgs<T> l{};
    l.s = (c2<T>*)p->scratch;
    l.s_pstride = p->s_pstride;
    l.outer_stride = (long long)p->N * p->tp;   // outer = theta bin
    l.elem_stride = p->tp;                      // along y
    l.n_outer = p->M;
    l.nk = p->N / 2;
    l.N = p->N;
    l.tw = (const c2<T>*)p->twN;
    l.cp = p->N / 2 + 1;
    l.inv_L = 1.0 / ((double)p->N * p->N * p->M);
    return l;
}

template <typename T>
unsigned y_blocks(se2_plan_s* p) {
    const long long lines = (long long)p->M * (p->N / 2 + 1);
    const int per = table<T>(p).lines_y;
    return (unsigned)((lines + per - 1) / per);
}

template <typename T>
se2_status run_chain(se2_plan_s* p, const void* f, int B, const void* const* coeffs,
                     const double* const* log_scales, int k, void* out, cudaStream_t st) {
    KTable<T>& kt = table<T>(p);
    const size_t g = (size_t)p->N * p->N * p->M;
    const long long cps = (p->flags & SE2_SHARED_KERNEL) ? 0 : (long long)p->M * p->N * (p->N / 2 + 1);
    const long long lps = (p->flags & SE2_SHARED_KERNEL) ? 0 : 1;
    for (int c0 = 0; c0 < B; c0 += p->chunk) {
        const int nb = (B - c0 < p->chunk) ? (B - c0) : p->chunk;
        launch_forward<T>(p, (const T*)f + c0 * g, nb, nullptr, st);
        LArgs<T> l = yargs<T>(p);
        l.k = k;
        l.c_pstride = cps;
        l.ls_pstride = lps;
        for (int i = 0; i < k; ++i) {
            l.C[i] = (const c2<T>*)coeffs[i] + c0 * cps;
            l.ls[i] = (log_scales && log_scales[i]) ? log_scales[i] + c0 * lps : nullptr;
        }
        kt.y_conv<<<dim3(y_blocks<T>(p), nb), kThreads, kt.smem_y, st>>>(l);
        launch_inverse<T>(p, (T*)out + c0 * g, nb, st);
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "kernel launch");
    return SE2_OK;
}

template <typename T>
se2_status run_coeffs(se2_plan_s* p, const void* samples, int n, void* coeffs, double* log_scale,
                      cudaStream_t st) {
    KTable<T>& kt = table<T>(p);
    const size_t g = (size_t)p->N * p->N * p->M;
    const long long cps = (long long)p->M * p->N * (p->N / 2 + 1);
    for (int c0 = 0; c0 < n; c0 += p->chunk) {
        const int nb = (n - c0 < p->chunk) ? (n - c0) : p->chunk;
        if (log_scale) {
            cudaError_t e = cudaMemsetAsync(p->abs_sum, 0, sizeof(double) * nb, st);
            if (e != cudaSuccess) return cuda_fail(e, "cudaMemsetAsync");
        }
        launch_forward<T>(p, (const T*)samples + c0 * g, nb, log_scale ? p->abs_sum : nullptr, st);
        LArgs<T> l = yargs<T>(p);
        l.cout = (c2<T>*)coeffs + c0 * cps;
        l.cout_pstride = cps;
        l.abs_sum = log_scale ? p->abs_sum : nullptr;
        l.log_scale = log_scale;
        l.problem0 = c0;
        kt.y_coef<<<dim3(y_blocks<T>(p), nb), kThreads, kt.smem_y, st>>>(l);
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "kernel launch");
    return SE2_OK;
}

se2_status check_plan(se2_plan_t p) {
    if (p == nullptr) return fail(SE2_ERR_INVALID_ARG, "plan is NULL");
    return SE2_OK;
}

}  // namespace

extern "C" {

const char* se2_last_error(void) { return g_err.c_str(); }

const char* se2_version(void) { return "se2-gb300 0.1 (sm_103a)"; }

se2_status se2_plan_create(se2_plan_t* out, int N, int M, int batch, se2_precision precision,
                           unsigned flags, int device) {
    if (out == nullptr) return fail(SE2_ERR_INVALID_ARG, "plan output pointer is NULL");
    *out = nullptr;
    if (!is_pow2(N) || N < 8 || N > 512) return fail(SE2_ERR_UNSUPPORTED, "N=%d: need a power of two in [8, 512]", N);
    if (!is_pow2(M) || M < 2 || M > 128) return fail(SE2_ERR_UNSUPPORTED, "M=%d: need a power of two in [2, 128]", M);
    if (batch < 1) return fail(SE2_ERR_INVALID_ARG, "batch=%d must be >= 1", batch);
    if (precision != SE2_F32 && precision != SE2_F64) return fail(SE2_ERR_UNSUPPORTED, "precision %d not supported", (int)precision);
    if (flags & ~SE2_SHARED_KERNEL) return fail(SE2_ERR_INVALID_ARG, "unknown flags 0x%x", flags);
    int ndev = 0;
    cudaError_t e = cudaGetDeviceCount(&ndev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDeviceCount");
    if (device < 0 || device >= ndev) return fail(SE2_ERR_INVALID_ARG, "device %d out of range (%d devices)", device, ndev);
    DeviceGuard guard(device);

    se2_plan_s* p = new (std::nothrow) se2_plan_s();
    if (p == nullptr) return fail(SE2_ERR_OOM, "host allocation failed");
    p->N = N;
    p->M = M;
    p->batch = batch;
    p->dev = device;
    p->prec = precision;
    p->flags = flags;
    p->tp = ((N / 2 + 1) + 15) / 16 * 16;           // 128-byte aligned scratch rows (FP32)
    p->s_pstride = (size_t)M * N * p->tp;
    se2_status st = (precision == SE2_F32) ? plan_init<float>(p) : plan_init<double>(p);
    if (st != SE2_OK) { plan_free(p); delete p; return st; }
    // scratch for `chunk` problems at a time (whole batch up to 1 GiB);
    // SE2_MAX_CHUNK (environment) caps it, e.g. to exercise ragged chunks.
    const size_t per = p->s_pstride * p->elem;
    size_t chunk = (size_t)1 << 30;
    chunk = chunk / per;
    if (const char* env = getenv("SE2_MAX_CHUNK")) {
        const long v = strtol(env, nullptr, 10);
        if (v >= 1 && (size_t)v < chunk) chunk = (size_t)v;
    }
    if (chunk < 1) chunk = 1;
    if (chunk > (size_t)batch) chunk = batch;
    p->chunk = (int)chunk;
    e = cudaMalloc(&p->scratch, per * chunk);
    if (e != cudaSuccess) { plan_free(p); delete p; return fail(SE2_ERR_OOM, "scratch (%zu bytes): %s", per * chunk, cudaGetErrorString(e)); }
    e = cudaMalloc((void**)&p->abs_sum, sizeof(double) * chunk);
    if (e != cudaSuccess) { plan_free(p); delete p; return fail(SE2_ERR_OOM, "accumulators: %s", cudaGetErrorString(e)); }
    e = cudaDeviceSynchronize();
    if (e != cudaSuccess) { plan_free(p); delete p; return cuda_fail(e, "plan setup"); }
    p->ws_bytes = per * chunk + p->elem * (N + M) + sizeof(double) * chunk;
    *out = p;
    return SE2_OK;
}

se2_status se2_plan_destroy(se2_plan_t p) {
    if (p == nullptr) return SE2_OK;
    DeviceGuard guard(p->dev);
    cudaDeviceSynchronize();
    plan_free(p);
    delete p;
    return SE2_OK;
}

size_t se2_plan_workspace_bytes(se2_plan_t p) { return p ? p->ws_bytes : 0; }

se2_status se2_coeffs(se2_plan_t p, const void* samples, int n, void* coeffs, double* log_scale,
                      void* stream) {
    se2_status st = check_plan(p);
    if (st != SE2_OK) return st;
    if (samples == nullptr || coeffs == nullptr) return fail(SE2_ERR_INVALID_ARG, "samples/coeffs is NULL");
    if (n < 1) return fail(SE2_ERR_INVALID_ARG, "n=%d must be >= 1", n);
    const size_t re = p->elem / 2;
    if (!aligned(samples, re) || !aligned(coeffs, p->elem) || (log_scale && !aligned(log_scale, 8)))
        return fail(SE2_ERR_INVALID_ARG, "misaligned pointer");
    DeviceGuard guard(p->dev);
    cudaStream_t s = (cudaStream_t)stream;
    return p->prec == SE2_F32 ? run_coeffs<float>(p, samples, n, coeffs, log_scale, s)
                              : run_coeffs<double>(p, samples, n, coeffs, log_scale, s);
}

se2_status se2_convolve_chain(se2_plan_t p, const void* f, int B, const void* const* coeffs,
                              const double* const* log_scales, int k, void* out, void* stream) {
    se2_status st = check_plan(p);
    if (st != SE2_OK) return st;
    if (f == nullptr || out == nullptr || coeffs == nullptr) return fail(SE2_ERR_INVALID_ARG, "NULL pointer argument");
    if (B < 1 || B > p->batch) return fail(SE2_ERR_INVALID_ARG, "B=%d outside [1, %d]", B, p->batch);
    if (k < 1 || k > kMaxChain) return fail(SE2_ERR_INVALID_ARG, "chain length k=%d outside [1, %d]", k, kMaxChain);
    const size_t re = p->elem / 2;
    if (!aligned(f, re) || !aligned(out, re)) return fail(SE2_ERR_INVALID_ARG, "misaligned f/out");
    for (int i = 0; i < k; ++i) {
        if (coeffs[i] == nullptr) return fail(SE2_ERR_INVALID_ARG, "coeffs[%d] is NULL", i);
        if (!aligned(coeffs[i], p->elem)) return fail(SE2_ERR_INVALID_ARG, "coeffs[%d] misaligned", i);
        if (log_scales && log_scales[i] && !aligned(log_scales[i], 8)) return fail(SE2_ERR_INVALID_ARG, "log_scales[%d] misaligned", i);
    }
    if (f == out) return fail(SE2_ERR_INVALID_ARG, "out aliases f");
    DeviceGuard guard(p->dev);
    cudaStream_t s = (cudaStream_t)stream;
    return p->prec == SE2_F32 ? run_chain<float>(p, f, B, coeffs, log_scales, k, out, s)
                              : run_chain<double>(p, f, B, coeffs, log_scales, k, out, s);
}

se2_status se2_convolve(se2_plan_t p, const void* f, int B, const void* coeffs, const double* log_scale,
                        void* out, void* stream) {
    const void* c[1] = {coeffs};
    const double* l[1] = {log_scale};
    return se2_convolve_chain(p, f, B, c, l, 1, out, stream);
}

}  // extern "C"
