// C ABI of the SE(2) convolution library (declared in include/se2.h).
//
// Host side: argument validation, plan (twiddle tables, scratch), and the
// launch sequences of Algorithm 3 (se2_convolve), Algorithms 4/6
// (se2_convolve_chain) and the coefficient transform (se2_coeffs, Eq. FkLv).
#include <cuda.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cstdarg>
#include <cstdint>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>
#include <string>
#include <algorithm>
#include <vector>

#include "../../include/se2.h"
#include "se2_internal.h"
#include "se2_nvtx.h"
#include "se2_tc.cuh"

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

void se2::set_last_error(const char* msg) { g_err = msg; }

namespace {
std::atomic<long long> g_live_allocs{0}, g_total_allocs{0}, g_fail_countdown{0};
}
cudaError_t se2::dev_alloc(void** p, size_t bytes) {
    // the countdown reaches 1 at the allocation that is to fail
    long long c = g_fail_countdown.load();
    while (c > 0 && !g_fail_countdown.compare_exchange_weak(c, c - 1)) {
    }
    if (c == 1) {
        *p = nullptr;
        return cudaErrorMemoryAllocation;
    }
    const cudaError_t e = cudaMalloc(p, bytes);
    if (e == cudaSuccess) {
        ++g_live_allocs;
        ++g_total_allocs;
    }
    return e;
}
void se2::dev_free(void* p) {
    if (p != nullptr && cudaFree(p) == cudaSuccess) --g_live_allocs;
}

se2_status se2_debug_alloc_stats(long long* live, long long* total) {
    SE2_RANGE("se2_debug_alloc_stats");
    if (live == nullptr || total == nullptr) return fail(SE2_ERR_INVALID_ARG, "NULL pointer argument");
    *live = g_live_allocs.load();
    *total = g_total_allocs.load();
    return SE2_OK;
}

se2_status se2_debug_fail_alloc(long long n) {
    SE2_RANGE("se2_debug_fail_alloc");
    if (n < 0) return fail(SE2_ERR_INVALID_ARG, "n=%lld must be >= 0", n);
    g_fail_countdown.store(n);
    return SE2_OK;
}

constexpr int kMaxPipe = 4;
constexpr int kPipeDepth = 2, kPipeGroup = 2;   // default pipelining of the FP32 fast path
constexpr long long kPipePoints = 2ll * 256 * 256 * 64;
constexpr int kHostBufs = 3, kHostGroup = 2;    // staging of se2_convolve_host

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
    double* mass = nullptr;     // [2 batch]: sum(f), sum(out) (SE2_MASS_RENORM)
    size_t ws_bytes = 0;
    // persistent path
    bool persist = false;
    int slots = 0;              // scratch slots in the persistent ring
    int persist_grid = 0;       // blocks of the persistent launch
    unsigned* ctr = nullptr;    // [1 + 3 * batch] work counter + unit counters
    int* err = nullptr;         // sticky device error word
    int nslots = 0;             // problem slots in the scratch (>= 2)
    // mixed precision: angular DFT on the tensor cores (0 = off, 1 or 3 products)
    int tc = 0;
    void* tcB = nullptr;        // B images: [dir -1: hi, lo][dir +1: hi, lo]
    TcKernel tc_fwd = nullptr, tc_inv = nullptr;
    size_t tc_smem = 0;
    int nsm = 0;
    double* tab = nullptr;      // [2N + 2M] FP64 tables of the Gaussian kernel family
    KTable<float> kf;
    KTable<double> kd;
    bool fused = false;
    unsigned long long launches = 0;   // kernels launched by this plan so far
    // per-launch timing of the FP32 fast path's units (se2_plan_timing)
    bool timing = false;
    std::vector<cudaEvent_t> tev;       // event pool, 2 per timed launch
    std::vector<int> tkind;             // unit of each timed launch (0 A, 1 B, 2 C)
    size_t tused = 0;                   // timed launches recorded
    // FP32 paired-FFT kernels for the convolution and chain (null: generic ones)
    bool fast = false;
    // unit C drops consumed scratch rows from L2 (SE2_L2_DISCARD=1 in the
    // environment): DRAM traffic falls to ~1.04x the algorithmic bytes, the
    // step measured 1.5% slower on GB300
    bool l2_discard = false;
    FastTable ft;
    // pipelined fast path: problem groups of pipe_group on pipe_depth streams
    // (the caller's and pipe_depth - 1 of the plan's), each group with its own
    // scratch slots, so that kernels of different groups overlap
    int pipe_depth = 1, pipe_group = 0;
    cudaStream_t aux[kMaxPipe] = {};
    cudaEvent_t ev_fork = nullptr, ev_join[kMaxPipe] = {};
    // se2_convolve_host: device staging for kHostBufs groups of host_group
    // problems (f then out per group), copy streams and their events
    int host_group = 0;
    void* hstage = nullptr;
    cudaStream_t hin = nullptr, hout = nullptr;
    cudaEvent_t hev_start = nullptr, hev_in[kHostBufs] = {}, hev_done[kHostBufs] = {}, hev_out[kHostBufs] = {};
    // tensor maps of the dataflow kernel's B items over the scratch
    CUtensorMap tm_blk{}, tm_nyq{};
};

bool se2::get_fast(int N, int M, FastTable* t) {
    switch (N) {
        case 32: return get_fast_n<32>(M, t);
        case 64: return get_fast_n<64>(M, t);
        case 128: return get_fast_n<128>(M, t);
        case 256: return get_fast_n<256>(M, t);
        default: return false;
    }
}

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
        {(const void*)kt.y_adj, kt.smem_y},   {(const void*)kt.y_sep, kt.smem_y},
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
    // The persistent dataflow kernel is opt-in (SE2_PERSIST=1): on 256^2 x 64
    // it measured slower than the three-kernel sequence.
    const char* per = getenv("SE2_PERSIST");
    p->persist = p->fused && kt.persist != nullptr &&
                 ((p->flags & SE2_PERSISTENT) || (per && per[0] == '1'));
    if (p->persist) {
        cudaError_t r = cudaFuncSetAttribute((const void*)kt.persist, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)kt.smem_persist);
        if (r == cudaSuccess)
            r = cudaFuncSetAttribute((const void*)kt.persist_sep, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)kt.smem_persist);
        if (r != cudaSuccess) return cuda_fail(r, "cudaFuncSetAttribute");
        int per_sm = 0, nsm = 0;
        r = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kt.persist, kThreads, kt.smem_persist);
        if (r != cudaSuccess) return cuda_fail(r, "occupancy");
        r = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, p->dev);
        if (r != cudaSuccess) return cuda_fail(r, "device attribute");
        if (per_sm < 1) p->persist = false;
        p->persist_grid = per_sm * nsm;
    }
    p->elem = sizeof(c2<T>);
    if (p->prec == SE2_SPLIT_BF16 || p->prec == SE2_BF16 || p->prec == SE2_SPLIT_F16) {
        p->tc = p->prec == SE2_BF16 ? 1 : 3;
        const int fmt = p->prec == SE2_SPLIT_F16 ? 1 : 0;
        p->fused = false;                    // x and theta as separate passes
        p->persist = false;
        if (!tc_kernel(p->M, -1, p->tc, fmt, &p->tc_fwd, &p->tc_smem) ||
            !tc_kernel(p->M, +1, p->tc, fmt, &p->tc_inv, &p->tc_smem))
            return fail(SE2_ERR_UNSUPPORTED, "tensor-core angular DFT needs M = 64 or 128 (M=%d)", p->M);
        cudaError_t r = cudaFuncSetAttribute((const void*)p->tc_fwd, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)p->tc_smem);
        if (r == cudaSuccess)
            r = cudaFuncSetAttribute((const void*)p->tc_inv, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)p->tc_smem);
        if (r != cudaSuccess) return cuda_fail(r, "cudaFuncSetAttribute");
        std::vector<unsigned char> img, all;
        tc_dft_matrix(-1, fmt, img);
        all.insert(all.end(), img.begin(), img.end());
        tc_dft_matrix(+1, fmt, img);
        all.insert(all.end(), img.begin(), img.end());
        r = dev_alloc((void**)&p->tcB, all.size());
        if (r != cudaSuccess) return fail(SE2_ERR_OOM, "tensor-core DFT matrix: %s", cudaGetErrorString(r));
        r = cudaMemcpy(p->tcB, all.data(), all.size(), cudaMemcpyHostToDevice);
        if (r != cudaSuccess) return cuda_fail(r, "cudaMemcpy");
        r = cudaDeviceGetAttribute(&p->nsm, cudaDevAttrMultiProcessorCount, p->dev);
        if (r != cudaSuccess) return cuda_fail(r, "device attribute");
    }
    // FP32 convolutions run on the paired-FFT kernels where they exist;
    // SE2_FAST=0 (environment) keeps the generic ones (used to test both).
    if constexpr (sizeof(T) == 4) {
        const char* fe = getenv("SE2_FAST");
        if (p->prec == SE2_F32 && p->fused && !p->persist && !(fe && fe[0] == '0') && get_fast(p->N, p->M, &p->ft)) {
            cudaError_t r = cudaFuncSetAttribute((const void*)p->ft.fwd, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)p->ft.smem_xt);
            if (r == cudaSuccess)
                r = cudaFuncSetAttribute((const void*)p->ft.inv, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)p->ft.smem_xt);
            if (r == cudaSuccess)
                r = cudaFuncSetAttribute((const void*)p->ft.lines, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)p->ft.smem_y);
            if (r == cudaSuccess)
                r = cudaFuncSetAttribute((const void*)p->ft.lines_sep, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)p->ft.smem_y);
            if (r == cudaSuccess)
                r = cudaFuncSetAttribute((const void*)p->ft.lines_fwd, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)p->ft.smem_y);
            if (r == cudaSuccess)
                r = cudaFuncSetAttribute((const void*)p->ft.lines_adj, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)p->ft.smem_y);
            if (r == cudaSuccess)
                r = cudaFuncSetAttribute((const void*)p->ft.lines_acc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)p->ft.smem_y);
            // The bulk-copy units A and C are opt-in (SE2_FAST2=1, or "a" / "c"
            // for one of them): measured inside the two-stream pipeline they are
            // 1-4% slower than the original units.
            const char* f2 = getenv("SE2_FAST2");
            if (!(f2 && (f2[0] == '1' || f2[0] == 'a'))) p->ft.fwd2 = nullptr;
            if (!(f2 && (f2[0] == '1' || f2[0] == 'c'))) p->ft.inv2 = nullptr;
            const char* dl = getenv("SE2_L2_DISCARD");
            p->l2_discard = dl && dl[0] == '1';
            const char* fl = getenv("SE2_FLOW");   // the whole-batch dataflow kernel is opt-in
            if (!(fl && fl[0] == '1')) p->ft.flow = nullptr;
            if (r == cudaSuccess && p->ft.flow != nullptr)
                r = cudaFuncSetAttribute((const void*)p->ft.flow, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)p->ft.smem_flow);
            if (r == cudaSuccess) r = cudaDeviceGetAttribute(&p->nsm, cudaDevAttrMultiProcessorCount, p->dev);
            if (r == cudaSuccess && p->ft.fwd2 != nullptr)
                r = cudaFuncSetAttribute((const void*)p->ft.fwd2, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)p->ft.smem_xt2);
            if (r == cudaSuccess && p->ft.inv2 != nullptr)
                r = cudaFuncSetAttribute((const void*)p->ft.inv2, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)p->ft.smem_xt2);
            if (r != cudaSuccess) return cuda_fail(r, "cudaFuncSetAttribute");
            p->fast = true;
        }
    }
    cudaError_t e;
    if ((e = dev_alloc((void**)&p->twN, sizeof(c2<T>) * p->N)) != cudaSuccess) return fail(SE2_ERR_OOM, "twiddles: %s", cudaGetErrorString(e));
    if ((e = dev_alloc((void**)&p->twM, sizeof(c2<T>) * p->M)) != cudaSuccess) return fail(SE2_ERR_OOM, "twiddles: %s", cudaGetErrorString(e));
    if ((e = make_twiddles<T>((c2<T>*)p->twN, p->N, 0)) != cudaSuccess) return cuda_fail(e, "twiddle kernel");
    if ((e = make_twiddles<T>((c2<T>*)p->twM, p->M, 0)) != cudaSuccess) return cuda_fail(e, "twiddle kernel");
    return SE2_OK;
}

void plan_free(se2_plan_s* p) {
    for (cudaEvent_t ev : p->tev) cudaEventDestroy(ev);
    p->tev.clear();
    p->tkind.clear();
    for (int k = 0; k < kHostBufs; ++k) {
        if (p->hev_in[k]) cudaEventDestroy(p->hev_in[k]);
        if (p->hev_done[k]) cudaEventDestroy(p->hev_done[k]);
        if (p->hev_out[k]) cudaEventDestroy(p->hev_out[k]);
        p->hev_in[k] = p->hev_done[k] = p->hev_out[k] = nullptr;
    }
    if (p->hev_start) cudaEventDestroy(p->hev_start);
    if (p->hin) cudaStreamDestroy(p->hin);
    if (p->hout) cudaStreamDestroy(p->hout);
    if (p->hstage) dev_free(p->hstage);
    p->hev_start = nullptr;
    p->hin = p->hout = nullptr;
    p->hstage = nullptr;
    for (int d = 0; d < kMaxPipe; ++d) {
        if (p->aux[d]) cudaStreamDestroy(p->aux[d]);
        if (p->ev_join[d]) cudaEventDestroy(p->ev_join[d]);
        p->aux[d] = nullptr;
        p->ev_join[d] = nullptr;
    }
    if (p->ev_fork) cudaEventDestroy(p->ev_fork);
    p->ev_fork = nullptr;
    if (p->ctr) dev_free(p->ctr);
    if (p->err) dev_free(p->err);
    if (p->tab) dev_free(p->tab);
    if (p->tcB) dev_free(p->tcB);
    p->tcB = nullptr;
    p->ctr = nullptr;
    p->err = nullptr;
    p->tab = nullptr;
    if (p->scratch) dev_free(p->scratch);
    if (p->twN) dev_free(p->twN);
    if (p->twM) dev_free(p->twM);
    if (p->abs_sum) dev_free(p->abs_sum);
    if (p->mass) dev_free(p->mass);
    p->scratch = p->twN = p->twM = nullptr;
    p->abs_sum = nullptr;
    p->mass = nullptr;
}

bool aligned(const void* ptr, size_t a) { return ((uintptr_t)ptr % a) == 0; }

// SE2_MASS_RENORM: FP64 sums of B problems' samples into sums[0..B).
template <typename T>
cudaError_t launch_mass_sum(se2_plan_s* p, const void* x, int B, double* sums, cudaStream_t s) {
    const long long n = (long long)p->N * p->N * p->M;
    const int bx = (int)((n + 256 * 8 - 1) / (256 * 8) < 64 ? (n + 256 * 8 - 1) / (256 * 8) : 64);
    k_mass_sum<T><<<dim3(bx, B), 256, 0, s>>>(static_cast<const T*>(x), n, sums);
    ++p->launches;
    return cudaGetLastError();
}

// Then the outputs' sums into p->mass[B..2B) and the correction.
template <typename T>
cudaError_t launch_mass_fix(se2_plan_s* p, void* out, int B, const void* const* coeffs,
                            const double* const* log_scales, int k, cudaStream_t s) {
    cudaError_t e = launch_mass_sum<T>(p, out, B, p->mass + B, s);
    if (e != cudaSuccess) return e;
    MassArgs<T> a = {};
    const bool shared = (p->flags & SE2_SHARED_KERNEL) != 0;
    for (int i = 0; i < k; ++i) {
        a.C[i] = static_cast<const c2<T>*>(coeffs[i]);
        a.ls[i] = log_scales ? log_scales[i] : nullptr;
    }
    a.k = k;
    a.B = B;
    a.c_pstride = shared ? 0 : (long long)p->M * p->N * (p->N / 2 + 1);
    a.ls_pstride = shared ? 0 : 1;
    const long long n = (long long)p->N * p->N * p->M;
    const long long per_block = 256LL * kMassRun;    // 8 warps x 32 lanes x kMassRun samples
    const int bx = (int)((n + per_block - 1) / per_block);
    k_mass_fix<T><<<dim3(bx, B), 256, 0, s>>>(static_cast<T*>(out), n, p->mass, a);
    ++p->launches;
    return cudaGetLastError();
}

// FP64 plans use double kernels; every other precision keeps float storage.
bool is_f64(const se2_plan_s* p) { return p->prec == SE2_F64; }

// Polls before a device-side wait gives up (each poll sleeps ~64 ns plus an
// L2 round trip, so this is of the order of a second).
constexpr long long kSpinLimit = 1ll << 21;

// ---------------------------------------------------------------------------
// Launch helpers
// ---------------------------------------------------------------------------
template <typename T>
XArgs<T> xargs(se2_plan_s* p, int slot0 = 0) {
    XArgs<T> a{};
    a.s = (c2<T>*)p->scratch + (size_t)slot0 * p->s_pstride;
    a.s_pstride = p->s_pstride;
    a.tp = p->tp;
    a.M = p->M;
    a.g_pstride = (size_t)p->N * p->N * p->M;
    a.twN = (const c2<T>*)p->twN;
    a.twM = (const c2<T>*)p->twM;
    return a;
}

// Angular DFT of nb scratch spectra on the tensor cores (mixed precision).
template <typename T>
void launch_tc(se2_plan_s* p, c2<T>* s, int nb, int dir, cudaStream_t st) {
    if constexpr (sizeof(T) == 4) {
        TcArgs t{};
        t.s = s;
        t.s_pstride = p->s_pstride;
        t.N = p->N;
        t.tp = p->tp;
        t.bmat = reinterpret_cast<const uint4*>((const unsigned char*)p->tcB + (dir < 0 ? 0 : 2 * kTcOpBytes));
        t.tw = (const float2*)p->twM;
        t.err = p->err;
        const long long lines = (long long)p->N * (p->N / 2 + 1);
        const int tiles = (int)((lines + kTcLines - 1) / kTcLines);
        int gx = (p->nsm + nb - 1) / nb;
        if (gx > tiles) gx = tiles;
        if (gx < 1) gx = 1;
        (dir < 0 ? p->tc_fwd : p->tc_inv)<<<dim3(gx, nb), kTcThreads, p->tc_smem, st>>>(t);
    }
}

// Forward x and theta transforms of nb real grids into the scratch.
template <typename T>
void launch_forward(se2_plan_s* p, const T* f, int nb, double* abs_sum, cudaStream_t st, int slot0 = 0) {
    KTable<T>& kt = table<T>(p);
    XArgs<T> a = xargs<T>(p, slot0);
    a.f = f;
    a.abs_sum = abs_sum;
    if (p->fused) {
        kt.fwd_xt<<<dim3(p->N, nb), kThreads, kt.smem_xt, st>>>(a);
        ++p->launches;
    } else {
        const int pairs = p->M / 2;
        kt.fwd_x<<<dim3(p->N, (pairs + kt.teams_x - 1) / kt.teams_x, nb), kThreads, kt.smem_x, st>>>(a);
        ++p->launches;
        LArgs<T> l{};
        l.s = a.s;
        l.s_pstride = p->s_pstride;
        l.outer_stride = p->tp;                      // outer = y
        l.elem_stride = (long long)p->N * p->tp;     // along theta
        l.n_outer = p->N;
        l.nk = p->N / 2;
        l.N = p->N;
        l.tw = (const c2<T>*)p->twM;
        const long long lines = (long long)p->N * (p->N / 2 + 1);
        if (p->tc) launch_tc<T>(p, a.s, nb, -1, st);
        else kt.t_fwd<<<dim3((unsigned)((lines + kt.lines_t - 1) / kt.lines_t), nb), kThreads, kt.smem_t, st>>>(l);
        ++p->launches;
    }
}

template <typename T>
void launch_inverse(se2_plan_s* p, T* out, int nb, cudaStream_t st, int slot0 = 0) {
    KTable<T>& kt = table<T>(p);
    XArgs<T> a = xargs<T>(p, slot0);
    a.out = out;
    if (p->fused) {
        kt.inv_tx<<<dim3(p->N, nb), kThreads, kt.smem_xt, st>>>(a);
        ++p->launches;
    } else {
        LArgs<T> l{};
        l.s = a.s;
        l.s_pstride = p->s_pstride;
        l.outer_stride = p->tp;
        l.elem_stride = (long long)p->N * p->tp;
        l.n_outer = p->N;
        l.nk = p->N / 2;
        l.N = p->N;
        l.tw = (const c2<T>*)p->twM;
        const long long lines = (long long)p->N * (p->N / 2 + 1);
        if (p->tc) launch_tc<T>(p, a.s, nb, +1, st);
        else kt.t_inv<<<dim3((unsigned)((lines + kt.lines_t - 1) / kt.lines_t), nb), kThreads, kt.smem_t, st>>>(l);
        ++p->launches;
        const int pairs = p->M / 2;
        kt.inv_x<<<dim3(p->N, (pairs + kt.teams_x - 1) / kt.teams_x, nb), kThreads, kt.smem_x, st>>>(a);
        ++p->launches;
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
    l.wsign = (p->flags & SE2_GRID_ORIGIN_ZERO) ? 0 : 1;
    return l;
}

template <typename T>
unsigned y_blocks(se2_plan_s* p) {
    const long long lines = (long long)p->M * (p->N / 2 + 1);
    const int per = table<T>(p).lines_y;
    return (unsigned)((lines + per - 1) / per);
}

template <typename T>
se2_status run_persist(se2_plan_s* p, const void* f, int B, const void* const* coeffs,
                       const double* const* log_scales, int k, void* out, cudaStream_t st,
                       unsigned dep_extra, long long spin_limit, const void* sep_tables = nullptr) {
    KTable<T>& kt = table<T>(p);
    const long long cps = (p->flags & SE2_SHARED_KERNEL) ? 0 : (long long)p->M * p->N * (p->N / 2 + 1);
    const long long lps = (p->flags & SE2_SHARED_KERNEL) ? 0 : 1;
    PArgs<T> a{};
    a.x = xargs<T>(p);
    a.x.f = (const T*)f;
    a.x.out = (T*)out;
    a.l = yargs<T>(p);
    a.l.k = k;
    a.l.c_pstride = cps;
    a.l.ls_pstride = lps;
    for (int i = 0; i < k && coeffs; ++i) {
        a.l.C[i] = (const c2<T>*)coeffs[i];
        a.l.ls[i] = (log_scales && log_scales[i]) ? log_scales[i] : nullptr;
    }
    if (sep_tables) {
        a.l.sep = (const c2<T>*)sep_tables;
        a.l.sep_pstride = (p->flags & SE2_SHARED_KERNEL) ? 0 : (long long)(p->N / 2 + 1 + p->N + p->M);
    }
    a.B = B;
    a.D = p->slots;
    a.nA = p->N;
    a.nC = p->N;
    a.nB = (int)y_blocks<T>(p);
    a.work = p->ctr;
    a.cnt = p->ctr + 1;
    a.err = p->err;
    a.spin_limit = spin_limit;
    a.dep_extra = dep_extra;
    cudaError_t e = cudaMemsetAsync(p->ctr, 0, sizeof(unsigned) * (1 + 3 * (size_t)B), st);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMemsetAsync");
    const long long units = (long long)B * (a.nA + a.nB + a.nC);
    const int grid = (int)(units < p->persist_grid ? units : p->persist_grid);
    if (sep_tables) kt.persist_sep<<<grid, kThreads, kt.smem_persist, st>>>(a);
    else kt.persist<<<grid, kThreads, kt.smem_persist, st>>>(a);
    ++p->launches;
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "kernel launch");
    return SE2_OK;
}

// Convolution / chain on the FP32 paired-FFT kernels (paired scratch layout).
// With pipe_depth > 1 the batch goes in groups of pipe_group problems,
// round-robin over pipe_depth streams forked from (and joined back into) st,
// each stream with its own scratch slots; a group's three kernels stay in
// order on its stream while groups on other streams overlap them.
// Unit timing (se2_plan_timing): an event before and after a launch, on the
// stream the launch runs on.  Returns the slot, or SIZE_MAX when not timing.
constexpr size_t kMaxTimed = 32768;
size_t time_begin(se2_plan_s* p, int kind, cudaStream_t s) {
    if (!p->timing || p->tused >= kMaxTimed) return SIZE_MAX;
    const size_t i = p->tused;
    while (p->tev.size() < 2 * (i + 1)) {
        cudaEvent_t ev = nullptr;
        if (cudaEventCreate(&ev) != cudaSuccess) return SIZE_MAX;
        p->tev.push_back(ev);
    }
    if (p->tkind.size() < i + 1) p->tkind.resize(i + 1);
    p->tkind[i] = kind;
    if (cudaEventRecord(p->tev[2 * i], s) != cudaSuccess) return SIZE_MAX;
    p->tused = i + 1;
    return i;
}
void time_end(se2_plan_s* p, size_t i, cudaStream_t s) {
    if (i != SIZE_MAX) cudaEventRecord(p->tev[2 * i + 1], s);
}

// Units A and C of the FP32 fast path: the bulk-copy kernels where they
// exist and the grid is 16-byte aligned, the original ones otherwise.
void launch_unit_a(const FastTable& ft, int N, int nb, cudaStream_t s, const FArgs& a) {
    if (ft.fwd2 != nullptr && aligned(a.f, 16))
        ft.fwd2<<<dim3(N, nb), kThreads, ft.smem_xt2, s>>>(a);
    else
        ft.fwd<<<dim3(N / ft.yr, nb), kThreads, ft.smem_xt, s>>>(a);
}
void launch_unit_c(const FastTable& ft, int N, int nb, cudaStream_t s, const FArgs& a) {
    if (ft.inv2 != nullptr && aligned(a.out, 16))
        ft.inv2<<<dim3(N, nb), kThreads, ft.smem_xt2, s>>>(a);
    else
        ft.inv<<<dim3(N / ft.yr, nb), kThreads, ft.smem_xt, s>>>(a);
}

// SE2_CHECK_FINITE: one pass over an output; the first NaN or infinity sets
// the plan's error word to 5 (se2_plan_status: SE2_ERR_NUMERIC).
template <typename T>
__global__ void k_check_finite(const T* x, size_t n, int* err) {
    bool bad = false;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        bad |= !isfinite(x[i]);
    if (__syncthreads_or(bad) && threadIdx.x == 0) atomicCAS(err, 0, 5);
}
se2_status check_finite(se2_plan_s* p, const void* x, size_t n, cudaStream_t s) {
    if (!(p->flags & SE2_CHECK_FINITE)) return SE2_OK;
    const int grid = 4 * (p->nsm > 0 ? p->nsm : 152);
    if (p->prec == SE2_F64)
        k_check_finite<double><<<grid, 256, 0, s>>>(static_cast<const double*>(x), n, p->err);
    else
        k_check_finite<float><<<grid, 256, 0, s>>>(static_cast<const float*>(x), n, p->err);
    ++p->launches;
    const cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? SE2_OK : cuda_fail(e, "finite check");
}

// Tensor maps of the dataflow kernel over the scratch [nslots M][N][4 tp/2
// floats]: boxes of 16 entries x N rows x 1 theta bin (B items of entry
// blocks) and 1 entry x N rows x 16 bins (Nyquist items).  The encoder is
// the driver's, reached through the runtime (no link to the driver library).
bool encode_flow_maps(se2_plan_s* p) {
    using Enc = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*, const cuuint64_t*,
                             const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave, CUtensorMapSwizzle,
                             CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
    void* fn = nullptr;
    cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess || fn == nullptr)
        return false;
    const Enc enc = (Enc)fn;
    const cuuint64_t row4 = (cuuint64_t)p->tp / 2;   // float4 entries per scratch row
    const cuuint64_t dims[3] = {row4 * 4, (cuuint64_t)p->N, (cuuint64_t)p->nslots * p->M};
    const cuuint64_t strides[2] = {row4 * 16, (cuuint64_t)p->N * row4 * 16};
    const cuuint32_t box_blk[3] = {4 * kFlowLines, (cuuint32_t)p->N, 1}, box_nyq[3] = {4, (cuuint32_t)p->N, kFlowLines};
    const cuuint32_t es[3] = {1, 1, 1};
    const CUresult r1 = enc(&p->tm_blk, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, p->scratch, dims, strides, box_blk, es,
                            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    const CUresult r2 = enc(&p->tm_nyq, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, p->scratch, dims, strides, box_nyq, es,
                            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r1 == CUDA_SUCCESS && r2 == CUDA_SUCCESS;
}

// The convolution (or chain) of B problems as one persistent dataflow launch
// (se2_flow.cuh): units A, B, C of every problem in one kernel, problems in
// flight in the plan's scratch slots.
bool flow_usable(const se2_plan_s* p, int B, const float* f, const float* out) {
    const int slots = p->nslots < kFlowSlots ? p->nslots : kFlowSlots;
    return p->ft.flow != nullptr && aligned(f, 16) && aligned(out, 16) && (slots >= 3 || B <= slots);
}
se2_status run_flow(se2_plan_s* p, const float* f, int B, const void* const* coeffs, const double* const* log_scales,
                    int k, float* out, cudaStream_t st) {
    const long long cps = (p->flags & SE2_SHARED_KERNEL) ? 0 : (long long)p->M * p->N * (p->N / 2 + 1);
    const long long lps = (p->flags & SE2_SHARED_KERNEL) ? 0 : 1;
    FlowArgs fa{};
    FArgs& a = fa.a;
    a.err = p->err;
    a.f = f;
    a.out = out;
    a.s = (float4*)p->scratch;
    a.s_pstride = (long long)(p->s_pstride / 2);
    a.twN = (const float2*)p->twN;
    a.twM = (const float2*)p->twM;
    a.k = k;
    a.c_pstride = cps;
    a.ls_pstride = lps;
    a.inv_L = 1.0 / ((double)p->N * p->N * p->M);
    a.wsign = (p->flags & SE2_GRID_ORIGIN_ZERO) ? 0 : 1;
    a.ymirror = (p->flags & SE2_KERNEL_YSYM) ? 1 : 0;
    for (int q = 0; q < k; ++q) {
        a.C[q] = (const float2*)coeffs[q];
        a.ls[q] = (log_scales && log_scales[q]) ? log_scales[q] : nullptr;
    }
    fa.tm_blk = p->tm_blk;
    fa.tm_nyq = p->tm_nyq;
    fa.work = p->ctr;
    fa.cnt = (int*)(p->ctr + 1);
    fa.P = B;
    fa.slots = p->nslots < kFlowSlots ? p->nslots : kFlowSlots;
    cudaError_t e = cudaMemsetAsync(p->ctr, 0, sizeof(unsigned) * (1 + 3 * (size_t)B), st);
    if (e != cudaSuccess) return cuda_fail(e, "counter reset");
    int grid = p->nsm > 0 ? p->nsm : 1;
    const size_t t = time_begin(p, 3, st);
    p->ft.flow<<<grid, kFlowThreads, p->ft.smem_flow, st>>>(fa);
    ++p->launches;
    time_end(p, t, st);
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "kernel launch");
    return SE2_OK;
}

se2_status run_chain_fast(se2_plan_s* p, const float* f, int B, const void* const* coeffs,
                          const double* const* log_scales, int k, float* out, cudaStream_t st,
                          const float2* sep_tables = nullptr) {
    if (sep_tables == nullptr && flow_usable(p, B, f, out)) return run_flow(p, f, B, coeffs, log_scales, k, out, st);
    const FastTable& ft = p->ft;
    const size_t g = (size_t)p->N * p->N * p->M;
    const long long cps = (p->flags & SE2_SHARED_KERNEL) ? 0 : (long long)p->M * p->N * (p->N / 2 + 1);
    const long long lps = (p->flags & SE2_SHARED_KERNEL) ? 0 : 1;
    const long long pairs = (long long)p->M * (p->N / 4 + 1);
    const unsigned yb = (unsigned)((pairs + ft.lines_per_block - 1) / ft.lines_per_block);
    const bool pipe = p->pipe_depth > 1 && B > p->pipe_group;
    const int group = pipe ? p->pipe_group : p->chunk;
    const int depth = pipe ? p->pipe_depth : 1;
    cudaError_t e = cudaSuccess;
    if (pipe) {
        e = cudaEventRecord(p->ev_fork, st);
        for (int d = 1; d < depth && e == cudaSuccess; ++d) e = cudaStreamWaitEvent(p->aux[d], p->ev_fork, 0);
        if (e != cudaSuccess) return cuda_fail(e, "stream fork");
    }
    int i = 0;
    for (int c0 = 0; c0 < B; c0 += group, ++i) {
        const int nb = (B - c0 < group) ? (B - c0) : group;
        const int d = i % depth;
        cudaStream_t s = d == 0 ? st : p->aux[d];
        FArgs a{};
        a.err = p->err;
        a.discard = p->l2_discard ? 1 : 0;
        a.f = f + c0 * g;
        a.out = out + c0 * g;
        a.s = (float4*)p->scratch + (size_t)d * group * (p->s_pstride / 2);
        a.s_pstride = (long long)(p->s_pstride / 2);
        a.twN = (const float2*)p->twN;
        a.twM = (const float2*)p->twM;
        a.k = k;
        a.c_pstride = cps;
        a.ls_pstride = lps;
        a.inv_L = 1.0 / ((double)p->N * p->N * p->M);
        a.wsign = (p->flags & SE2_GRID_ORIGIN_ZERO) ? 0 : 1;
        a.ymirror = (p->flags & SE2_KERNEL_YSYM) ? 1 : 0;
        if (sep_tables != nullptr) {
            const long long tps = (p->flags & SE2_SHARED_KERNEL) ? 0 : (long long)(p->N / 2 + 1 + p->N + p->M);
            a.sep = sep_tables + c0 * tps;
            a.sep_pstride = tps;
        } else {
            for (int q = 0; q < k; ++q) {
                a.C[q] = (const float2*)coeffs[q] + c0 * cps;
                a.ls[q] = (log_scales && log_scales[q]) ? log_scales[q] + c0 * lps : nullptr;
            }
        }
        const size_t t0 = time_begin(p, 0, s);
        launch_unit_a(ft, p->N, nb, s, a);
        ++p->launches;
        time_end(p, t0, s);
        const size_t t1 = time_begin(p, 1, s);
        (sep_tables != nullptr ? ft.lines_sep : ft.lines)<<<dim3(yb, nb), kLineThreads, ft.smem_y, s>>>(a);
        ++p->launches;
        time_end(p, t1, s);
        const size_t t2 = time_begin(p, 2, s);
        launch_unit_c(ft, p->N, nb, s, a);
        ++p->launches;
        time_end(p, t2, s);
    }
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "kernel launch");
    if (pipe) {
        for (int d = 1; d < depth && e == cudaSuccess; ++d) {
            e = cudaEventRecord(p->ev_join[d], p->aux[d]);
            if (e == cudaSuccess) e = cudaStreamWaitEvent(st, p->ev_join[d], 0);
        }
        if (e != cudaSuccess) return cuda_fail(e, "stream join");
    }
    return SE2_OK;
}

template <typename T>
se2_status run_chain(se2_plan_s* p, const void* f, int B, const void* const* coeffs,
                     const double* const* log_scales, int k, void* out, cudaStream_t st) {
    KTable<T>& kt = table<T>(p);
    if (p->persist) return run_persist<T>(p, f, B, coeffs, log_scales, k, out, st, 0, kSpinLimit);
    if constexpr (sizeof(T) == 4) {
        if (p->fast) return run_chain_fast(p, (const float*)f, B, coeffs, log_scales, k, (float*)out, st);
    }
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
        ++p->launches;
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
        ++p->launches;
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "kernel launch");
    return SE2_OK;
}

// The adjoint on the FP32 paired kernels: unit A on grad_out (slots 0..nb-1)
// and on f (slots nb..2nb-1), the forward y FFT of f's spectrum, the adjoint y
// pass (partials + correlation spectrum), unit C into grad_f.
se2_status run_backward_fast(se2_plan_s* p, const float* g, const float* f, int B, const void* coeffs,
                             const double* log_scale, int n_params, const void* const* dcoeffs,
                             double* grad_params, float* grad_f, cudaStream_t st) {
    const FastTable& ft = p->ft;
    const size_t gs = (size_t)p->N * p->N * p->M;
    const long long cps = (p->flags & SE2_SHARED_KERNEL) ? 0 : (long long)p->M * p->N * (p->N / 2 + 1);
    const long long lps = (p->flags & SE2_SHARED_KERNEL) ? 0 : 1;
    const long long pairs = (long long)p->M * (p->N / 4 + 1);
    const unsigned yb = (unsigned)((pairs + ft.lines_per_block - 1) / ft.lines_per_block);
    const int per_pass = n_params > 0 ? p->nslots / 2 : p->nslots;
    for (int c0 = 0; c0 < B; c0 += per_pass) {
        const int nb = (B - c0 < per_pass) ? (B - c0) : per_pass;
        FArgs a{};
        a.err = p->err;
        a.discard = p->l2_discard ? 1 : 0;
        a.s_pstride = (long long)(p->s_pstride / 2);
        a.twN = (const float2*)p->twN;
        a.twM = (const float2*)p->twM;
        a.inv_L = 1.0 / ((double)p->N * p->N * p->M);
        a.wsign = (p->flags & SE2_GRID_ORIGIN_ZERO) ? 0 : 1;
        float4* s0 = (float4*)p->scratch;
        float4* s1 = s0 + (size_t)nb * (p->s_pstride / 2);
        a.f = g + c0 * gs;
        a.s = s0;
        launch_unit_a(ft, p->N, nb, st, a);
        ++p->launches;
        if (n_params > 0) {
            a.f = f + c0 * gs;
            a.s = s1;
            launch_unit_a(ft, p->N, nb, st, a);
            ++p->launches;
            ft.lines_fwd<<<dim3(yb, nb), kLineThreads, ft.smem_y, st>>>(a);
            ++p->launches;
        }
        a.s = s0;
        a.s2 = s1;
        a.k = 1;
        a.c_pstride = cps;
        a.ls_pstride = lps;
        a.C[0] = (const float2*)coeffs + c0 * cps;
        a.ls[0] = log_scale ? log_scale + c0 * lps : nullptr;
        a.n_params = n_params;
        for (int i = 0; i < n_params; ++i) a.dC[i] = (const float2*)dcoeffs[i] + c0 * cps;
        a.grad_params = grad_params;
        a.want_grad = grad_f != nullptr;
        ft.lines_adj<<<dim3(yb, nb), kLineThreads, ft.smem_y, st>>>(a);
        ++p->launches;
        if (grad_f) {
            a.out = grad_f + c0 * gs;
            launch_unit_c(ft, p->N, nb, st, a);
            ++p->launches;
        }
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "kernel launch");
    return SE2_OK;
}

template <typename T>
se2_status run_backward(se2_plan_s* p, const void* g, const void* f, int B, const void* coeffs,
                        const double* log_scale, int n_params, const void* const* dcoeffs,
                        double* grad_params, void* grad_f, cudaStream_t st) {
    KTable<T>& kt = table<T>(p);
    if constexpr (sizeof(T) == 4) {
        if (p->fast)
            return run_backward_fast(p, (const float*)g, (const float*)f, B, coeffs, log_scale, n_params, dcoeffs,
                                     grad_params, (float*)grad_f, st);
    }
    const size_t gs = (size_t)p->N * p->N * p->M;
    const long long cps = (p->flags & SE2_SHARED_KERNEL) ? 0 : (long long)p->M * p->N * (p->N / 2 + 1);
    const long long lps = (p->flags & SE2_SHARED_KERNEL) ? 0 : 1;
    const int per_pass = n_params > 0 ? p->nslots / 2 : p->nslots;
    for (int c0 = 0; c0 < B; c0 += per_pass) {
        const int nb = (B - c0 < per_pass) ? (B - c0) : per_pass;
        launch_forward<T>(p, (const T*)g + c0 * gs, nb, nullptr, st, 0);
        if (n_params > 0) launch_forward<T>(p, (const T*)f + c0 * gs, nb, nullptr, st, nb);
        LArgs<T> l = yargs<T>(p);
        l.s2 = n_params > 0 ? (c2<T>*)p->scratch + (size_t)nb * p->s_pstride : nullptr;
        l.want_grad = grad_f != nullptr;
        l.k = 1;
        l.c_pstride = cps;
        l.ls_pstride = lps;
        l.C[0] = (const c2<T>*)coeffs + c0 * cps;
        l.ls[0] = log_scale ? log_scale + c0 * lps : nullptr;
        l.n_params = n_params;
        for (int i = 0; i < n_params; ++i) l.dC[i] = (const c2<T>*)dcoeffs[i] + c0 * cps;
        l.grad_params = grad_params;
        kt.y_adj<<<dim3(y_blocks<T>(p), nb), kThreads, kt.smem_y, st>>>(l);
        ++p->launches;
        if (grad_f) launch_inverse<T>(p, (T*)grad_f + c0 * gs, nb, st, 0);
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "kernel launch");
    return SE2_OK;
}

template <typename T>
se2_status run_sep(se2_plan_s* p, const void* f, int B, const void* tables, void* out, cudaStream_t st) {
    KTable<T>& kt = table<T>(p);
    if (p->persist) return run_persist<T>(p, f, B, nullptr, nullptr, 1, out, st, 0, kSpinLimit, tables);
    if constexpr (sizeof(T) == 4) {
        if (p->fast) return run_chain_fast(p, (const float*)f, B, nullptr, nullptr, 1, (float*)out, st, (const float2*)tables);
    }
    const size_t g = (size_t)p->N * p->N * p->M;
    const long long tps = (p->flags & SE2_SHARED_KERNEL) ? 0 : (long long)(p->N / 2 + 1 + p->N + p->M);
    for (int c0 = 0; c0 < B; c0 += p->chunk) {
        const int nb = (B - c0 < p->chunk) ? (B - c0) : p->chunk;
        launch_forward<T>(p, (const T*)f + c0 * g, nb, nullptr, st);
        LArgs<T> l = yargs<T>(p);
        l.k = 1;
        l.sep = (const c2<T>*)tables + c0 * tps;
        l.sep_pstride = tps;
        kt.y_sep<<<dim3(y_blocks<T>(p), nb), kThreads, kt.smem_y, st>>>(l);
        ++p->launches;
        launch_inverse<T>(p, (T*)out + c0 * g, nb, st);
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

// Staging of se2_convolve_host (plan flag SE2_HOST_STAGING): kHostBufs
// groups of f and out in device memory, two copy streams and their events,
// made once at plan creation so that no convolve call allocates.
se2_status host_staging_init(se2_plan_s* p) {
    const size_t gbytes = (size_t)p->N * p->N * p->M * (p->elem / 2);   // one grid
    int G = kHostGroup;   // SE2_HOST_GROUP (environment) overrides the group size
    if (const char* v = getenv("SE2_HOST_GROUP")) G = (int)strtol(v, nullptr, 10);
    if (G < 1) G = 1;
    if (G > p->batch) G = p->batch;
    cudaError_t e = dev_alloc((void**)&p->hstage, 2 * gbytes * (size_t)G * kHostBufs);
    if (e != cudaSuccess) { p->hstage = nullptr; return fail(SE2_ERR_OOM, "host staging: %s", cudaGetErrorString(e)); }
    p->host_group = G;
    e = cudaStreamCreateWithFlags(&p->hin, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&p->hout, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&p->hev_start, cudaEventDisableTiming);
    for (int k = 0; k < kHostBufs && e == cudaSuccess; ++k) {
        e = cudaEventCreateWithFlags(&p->hev_in[k], cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&p->hev_done[k], cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&p->hev_out[k], cudaEventDisableTiming);
    }
    if (e != cudaSuccess) return cuda_fail(e, "host staging streams");
    return SE2_OK;
}

namespace {
se2_status plan_create_impl(se2_plan_t* out, int N, int M, int batch, se2_precision precision, unsigned flags,
                            int device, size_t max_scratch);
}

se2_status se2_plan_create(se2_plan_t* out, int N, int M, int batch, se2_precision precision,
                           unsigned flags, int device) {
    SE2_RANGE("se2_plan_create");
    return plan_create_impl(out, N, M, batch, precision, flags, device, 0);
}

namespace {
// max_scratch > 0 caps the scratch (problem slots) below the default 1 GiB.
se2_status plan_create_impl(se2_plan_t* out, int N, int M, int batch, se2_precision precision, unsigned flags,
                            int device, size_t max_scratch) {
    if (out == nullptr) return fail(SE2_ERR_INVALID_ARG, "plan output pointer is NULL");
    *out = nullptr;
    if (!is_pow2(N) || N < 8 || N > 512) return fail(SE2_ERR_UNSUPPORTED, "N=%d: need a power of two in [8, 512]", N);
    if (!is_pow2(M) || M < 2 || M > 128) return fail(SE2_ERR_UNSUPPORTED, "M=%d: need a power of two in [2, 128]", M);
    if (batch < 1) return fail(SE2_ERR_INVALID_ARG, "batch=%d must be >= 1", batch);
    if (precision != SE2_F32 && precision != SE2_F64 && precision != SE2_SPLIT_BF16 && precision != SE2_BF16 &&
        precision != SE2_SPLIT_F16)
        return fail(SE2_ERR_UNSUPPORTED, "precision %d not supported", (int)precision);
    if (flags & ~(SE2_SHARED_KERNEL | SE2_PERSISTENT | SE2_GRID_ORIGIN_ZERO | SE2_MASS_RENORM | SE2_KERNEL_YSYM |
                  SE2_HOST_STAGING | SE2_CHECK_FINITE))
        return fail(SE2_ERR_INVALID_ARG, "unknown flags 0x%x", flags);
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
    se2_status st = (precision != SE2_F64) ? plan_init<float>(p) : plan_init<double>(p);
    if (st != SE2_OK) { plan_free(p); delete p; return st; }
    // scratch for `chunk` problems at a time (whole batch up to 1 GiB);
    // SE2_MAX_CHUNK (environment) caps it, e.g. to exercise ragged chunks.
    const size_t per = p->s_pstride * p->elem;
    size_t chunk = max_scratch > 0 ? max_scratch : (size_t)1 << 30;
    chunk = chunk / per;
    if (const char* env = getenv("SE2_MAX_CHUNK")) {
        const long v = strtol(env, nullptr, 10);
        if (v >= 1 && (size_t)v < chunk) chunk = (size_t)v;
    }
    if (chunk < 1) chunk = 1;
    if (p->persist) {
        // a ring of 4 slots: problems in flight between a unit A and its C
        chunk = 4;
        p->slots = 4;
    }
    if (chunk > (size_t)batch) chunk = batch;
    p->chunk = (int)chunk;
    if (p->persist && p->slots > (int)chunk) p->slots = (int)chunk;
    // at least two slots: the adjoint transforms grad_out and f side by side
    p->nslots = chunk < 2 ? 2 : (int)chunk;
    const size_t scratch_bytes = per * p->nslots;
    e = dev_alloc((void**)&p->scratch, scratch_bytes);
    if (e != cudaSuccess) { plan_free(p); delete p; return fail(SE2_ERR_OOM, "scratch (%zu bytes): %s", scratch_bytes, cudaGetErrorString(e)); }
    if (p->fast && p->ft.flow != nullptr && !encode_flow_maps(p)) p->ft.flow = nullptr;   // keep the pipelined units
    if (p->fast) {
        // pipelined groups (SE2_PIPE_DEPTH / SE2_PIPE_GROUP in the environment
        // override the defaults); depth * group scratch slots must exist
        // a group holds at least kPipePoints grid points (2 problems at
        // 256^2 x 64), so that small problems are not split into tiny launches
        const long long pts = (long long)N * N * M;
        int depth = kPipeDepth, group = (int)((kPipePoints + pts - 1) / pts);
        if (group < kPipeGroup) group = kPipeGroup;
        if (const char* v = getenv("SE2_PIPE_DEPTH")) depth = (int)strtol(v, nullptr, 10);
        if (const char* v = getenv("SE2_PIPE_GROUP")) group = (int)strtol(v, nullptr, 10);
        if (depth > kMaxPipe) depth = kMaxPipe;
        if (group < 1) group = 1;
        while (depth > 1 && depth * group > p->nslots) --depth;
        if (depth > 1) {
            e = cudaEventCreateWithFlags(&p->ev_fork, cudaEventDisableTiming);
            for (int d = 1; d < depth && e == cudaSuccess; ++d) {
                e = cudaStreamCreateWithFlags(&p->aux[d], cudaStreamNonBlocking);
                if (e == cudaSuccess) e = cudaEventCreateWithFlags(&p->ev_join[d], cudaEventDisableTiming);
            }
            if (e != cudaSuccess) { plan_free(p); delete p; return cuda_fail(e, "pipeline streams"); }
            p->pipe_depth = depth;
            p->pipe_group = group;
        }
    }
    e = dev_alloc((void**)&p->tab, sizeof(double) * 2 * ((size_t)N + M));
    if (e != cudaSuccess) { plan_free(p); delete p; return fail(SE2_ERR_OOM, "tables: %s", cudaGetErrorString(e)); }
    e = dev_alloc((void**)&p->abs_sum, sizeof(double) * chunk);
    if (e != cudaSuccess) { plan_free(p); delete p; return fail(SE2_ERR_OOM, "accumulators: %s", cudaGetErrorString(e)); }
    if (flags & SE2_MASS_RENORM) {
        e = dev_alloc((void**)&p->mass, sizeof(double) * 2 * (size_t)batch);
        if (e != cudaSuccess) { plan_free(p); delete p; return fail(SE2_ERR_OOM, "mass sums: %s", cudaGetErrorString(e)); }
    }
    e = dev_alloc((void**)&p->ctr, sizeof(unsigned) * (1 + 3 * (size_t)batch));
    if (e != cudaSuccess) { plan_free(p); delete p; return fail(SE2_ERR_OOM, "counters: %s", cudaGetErrorString(e)); }
    e = dev_alloc((void**)&p->err, sizeof(int));
    if (e == cudaSuccess) e = cudaMemset(p->err, 0, sizeof(int));
    if (e != cudaSuccess) { plan_free(p); delete p; return fail(SE2_ERR_OOM, "error word: %s", cudaGetErrorString(e)); }
    if (flags & SE2_HOST_STAGING) {
        st = host_staging_init(p);
        if (st != SE2_OK) { plan_free(p); delete p; return st; }
    }
    e = cudaDeviceSynchronize();
    if (e != cudaSuccess) { plan_free(p); delete p; return cuda_fail(e, "plan setup"); }
    p->ws_bytes = per * p->nslots + sizeof(double) * 2 * ((size_t)N + M) + p->elem * (N + M) + sizeof(double) * chunk + sizeof(unsigned) * (1 + 3 * (size_t)batch) + sizeof(int);
    *out = p;
    return SE2_OK;
}
}  // namespace

se2_status se2_plan_destroy(se2_plan_t p) {
    SE2_RANGE("se2_plan_destroy");
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
    SE2_RANGE("se2_coeffs");
    se2_status st = check_plan(p);
    if (st != SE2_OK) return st;
    if (samples == nullptr || coeffs == nullptr) return fail(SE2_ERR_INVALID_ARG, "samples/coeffs is NULL");
    if (n < 1) return fail(SE2_ERR_INVALID_ARG, "n=%d must be >= 1", n);
    const size_t re = p->elem / 2;
    if (!aligned(samples, re) || !aligned(coeffs, p->elem) || (log_scale && !aligned(log_scale, 8)))
        return fail(SE2_ERR_INVALID_ARG, "misaligned pointer");
    DeviceGuard guard(p->dev);
    cudaStream_t s = (cudaStream_t)stream;
    return !is_f64(p) ? run_coeffs<float>(p, samples, n, coeffs, log_scale, s)
                              : run_coeffs<double>(p, samples, n, coeffs, log_scale, s);
}

se2_status se2_convolve_chain(se2_plan_t p, const void* f, int B, const void* const* coeffs,
                              const double* const* log_scales, int k, void* out, void* stream) {
    SE2_RANGE("se2_convolve_chain");
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
    const bool renorm = (p->flags & SE2_MASS_RENORM) != 0;
    if (renorm) {
        cudaError_t e = cudaMemsetAsync(p->mass, 0, sizeof(double) * 2 * (size_t)B, s);
        if (e == cudaSuccess) e = !is_f64(p) ? launch_mass_sum<float>(p, f, B, p->mass, s)
                                             : launch_mass_sum<double>(p, f, B, p->mass, s);
        if (e != cudaSuccess) return cuda_fail(e, "mass sums");
    }
    st = !is_f64(p) ? run_chain<float>(p, f, B, coeffs, log_scales, k, out, s)
                    : run_chain<double>(p, f, B, coeffs, log_scales, k, out, s);
    if (st != SE2_OK) return st;
    if (renorm) {
        cudaError_t e = !is_f64(p) ? launch_mass_fix<float>(p, out, B, coeffs, log_scales, k, s)
                                   : launch_mass_fix<double>(p, out, B, coeffs, log_scales, k, s);
        if (e != cudaSuccess) return cuda_fail(e, "mass renormalisation");
    }
    return check_finite(p, out, (size_t)p->N * p->N * p->M * B, s);
}

se2_status se2_convolve_host(se2_plan_t p, const void* f, int B, const void* coeffs, const double* log_scale,
                             void* out, void* stream) {
    SE2_RANGE("se2_convolve_host");
    se2_status st = check_plan(p);
    if (st != SE2_OK) return st;
    if (f == nullptr || out == nullptr || coeffs == nullptr) return fail(SE2_ERR_INVALID_ARG, "NULL pointer argument");
    if (B < 1 || B > p->batch) return fail(SE2_ERR_INVALID_ARG, "B=%d outside [1, %d]", B, p->batch);
    if (!aligned(coeffs, p->elem)) return fail(SE2_ERR_INVALID_ARG, "coeffs misaligned");
    if (log_scale && !aligned(log_scale, 8)) return fail(SE2_ERR_INVALID_ARG, "log_scale misaligned");
    const size_t re = p->elem / 2;
    const size_t gbytes = (size_t)p->N * p->N * p->M * re;   // one grid
    const uintptr_t fa = (uintptr_t)f, oa = (uintptr_t)out, len = gbytes * (size_t)B;
    if (fa < oa + len && oa < fa + len) return fail(SE2_ERR_INVALID_ARG, "out overlaps f");
    DeviceGuard guard(p->dev);
    cudaError_t e = cudaSuccess;
    if (p->hstage == nullptr)
        return fail(SE2_ERR_INVALID_ARG, "the plan was created without SE2_HOST_STAGING (no staging buffers)");
    const int G = p->host_group;
    const long long cps = (p->flags & SE2_SHARED_KERNEL) ? 0 : (long long)p->M * p->N * (p->N / 2 + 1);
    const long long lps = (p->flags & SE2_SHARED_KERNEL) ? 0 : 1;
    cudaStream_t s = (cudaStream_t)stream;
    e = cudaEventRecord(p->hev_start, s);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(p->hin, p->hev_start, 0);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(p->hout, p->hev_start, 0);
    if (e != cudaSuccess) return cuda_fail(e, "host staging fork");
    int g = 0;
    for (int c0 = 0; c0 < B; c0 += G, ++g) {
        const int k = g % kHostBufs, nb = (B - c0 < G) ? (B - c0) : G;
        unsigned char* fdev = (unsigned char*)p->hstage + 2 * gbytes * (size_t)G * k;
        unsigned char* odev = fdev + gbytes * (size_t)G;
        const size_t bytes = gbytes * (size_t)nb, off = gbytes * (size_t)c0;
        // in: slot k's f is free once the convolution of the group before finished
        e = cudaStreamWaitEvent(p->hin, p->hev_done[k], 0);
        if (e == cudaSuccess) e = cudaMemcpyAsync(fdev, (const unsigned char*)f + off, bytes, cudaMemcpyHostToDevice, p->hin);
        if (e == cudaSuccess) e = cudaEventRecord(p->hev_in[k], p->hin);
        // convolve after the copy in, and after slot k's previous out left
        if (e == cudaSuccess) e = cudaStreamWaitEvent(s, p->hev_in[k], 0);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(s, p->hev_out[k], 0);
        if (e != cudaSuccess) return cuda_fail(e, "host staging copy in");
        const void* cg[1] = {(const unsigned char*)coeffs + (size_t)c0 * cps * p->elem};
        const double* lg[1] = {log_scale ? log_scale + (size_t)c0 * lps : nullptr};
        st = !is_f64(p) ? run_chain<float>(p, fdev, nb, cg, lg, 1, odev, s)
                        : run_chain<double>(p, fdev, nb, cg, lg, 1, odev, s);
        if (st != SE2_OK) return st;
        e = cudaEventRecord(p->hev_done[k], s);
        // out
        if (e == cudaSuccess) e = cudaStreamWaitEvent(p->hout, p->hev_done[k], 0);
        if (e == cudaSuccess) e = cudaMemcpyAsync((unsigned char*)out + off, odev, bytes, cudaMemcpyDeviceToHost, p->hout);
        if (e == cudaSuccess) e = cudaEventRecord(p->hev_out[k], p->hout);
        if (e != cudaSuccess) return cuda_fail(e, "host staging copy out");
    }
    for (int k = 0; k < kHostBufs && e == cudaSuccess; ++k) e = cudaStreamWaitEvent(s, p->hev_out[k], 0);
    if (e != cudaSuccess) return cuda_fail(e, "host staging join");
    return SE2_OK;
}

se2_status se2_convolve_chain_all(se2_plan_t p, const void* f, int B, const void* const* coeffs,
                                  const double* const* log_scales, int k, void* out, void* stream) {
    SE2_RANGE("se2_convolve_chain_all");
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
    const size_t gs = (size_t)p->N * p->N * p->M;
    const uintptr_t fa = (uintptr_t)f, oa = (uintptr_t)out;
    if (fa < oa + gs * re * (size_t)k * B && oa < fa + gs * re * (size_t)B) return fail(SE2_ERR_INVALID_ARG, "out overlaps f");
    DeviceGuard guard(p->dev);
    cudaStream_t s = (cudaStream_t)stream;
    if (!p->fast) {
        // without the FP32 fast path (FP64, N = 512, the tensor-core modes):
        // each V_p as its own chain of the first p kernels
        for (int q = 1; q <= k; ++q) {
            unsigned char* op = static_cast<unsigned char*>(out) + (size_t)(q - 1) * B * gs * re;
            st = !is_f64(p) ? run_chain<float>(p, f, B, coeffs, log_scales, q, op, s)
                            : run_chain<double>(p, f, B, coeffs, log_scales, q, op, s);
            if (st != SE2_OK) return st;
        }
        return check_finite(p, out, gs * (size_t)k * B, s);
    }
    const FastTable& ft = p->ft;
    const long long cps = (p->flags & SE2_SHARED_KERNEL) ? 0 : (long long)p->M * p->N * (p->N / 2 + 1);
    const long long lps = (p->flags & SE2_SHARED_KERNEL) ? 0 : 1;
    const long long pairs = (long long)p->M * (p->N / 4 + 1);
    const unsigned yb = (unsigned)((pairs + ft.lines_per_block - 1) / ft.lines_per_block);
    const int per_pass = p->nslots / 2;
    for (int c0 = 0; c0 < B; c0 += per_pass) {
        const int nb = (B - c0 < per_pass) ? (B - c0) : per_pass;
        FArgs a{};
        a.err = p->err;
        a.discard = p->l2_discard ? 1 : 0;
        a.s_pstride = (long long)(p->s_pstride / 2);
        a.twN = (const float2*)p->twN;
        a.twM = (const float2*)p->twM;
        a.inv_L = 1.0 / ((double)p->N * p->N * p->M);
        a.wsign = (p->flags & SE2_GRID_ORIGIN_ZERO) ? 0 : 1;
        a.ymirror = (p->flags & SE2_KERNEL_YSYM) ? 1 : 0;   // the running-product pass folds rows too
        a.k = k;
        a.c_pstride = cps;
        a.ls_pstride = lps;
        for (int i = 0; i < k; ++i) {
            a.C[i] = (const float2*)coeffs[i] + c0 * cps;
            a.ls[i] = (log_scales && log_scales[i]) ? log_scales[i] + c0 * lps : nullptr;
        }
        float4* s0 = (float4*)p->scratch;
        float4* s1 = s0 + (size_t)nb * (p->s_pstride / 2);
        a.f = (const float*)f + c0 * gs;
        a.s = s0;
        a.sout = s1;
        launch_unit_a(ft, p->N, nb, s, a);       // x, theta
        ++p->launches;
        ft.lines_fwd<<<dim3(yb, nb), kLineThreads, ft.smem_y, s>>>(a);     // y: the full spectrum of f
        ++p->launches;
        for (int q = 1; q <= k; ++q) {
            a.p = q;
            ft.lines_acc<<<dim3(yb, nb), kLineThreads, ft.smem_y, s>>>(a);   // R_q = R_{q-1} C_q; iDFT_y -> s1
            ++p->launches;
            FArgs c = a;
            c.s = s1;
            c.out = (float*)out + ((size_t)(q - 1) * B + c0) * gs;
            launch_unit_c(ft, p->N, nb, s, c);
            ++p->launches;
        }
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "kernel launch");
    return check_finite(p, out, gs * (size_t)k * B, s);
}

se2_status se2_backward(se2_plan_t p, const void* grad_out, const void* f, int B, const void* coeffs,
                        const double* log_scale, int n_params, const void* const* dcoeffs,
                        double* grad_params, void* grad_f, void* stream) {
    SE2_RANGE("se2_backward");
    se2_status st = check_plan(p);
    if (st != SE2_OK) return st;
    if (grad_out == nullptr || coeffs == nullptr) return fail(SE2_ERR_INVALID_ARG, "grad_out/coeffs is NULL");
    if (B < 1 || B > p->batch) return fail(SE2_ERR_INVALID_ARG, "B=%d outside [1, %d]", B, p->batch);
    if (n_params < 0 || n_params > kMaxParams) return fail(SE2_ERR_INVALID_ARG, "n_params=%d outside [0, %d]", n_params, kMaxParams);
    if (n_params > 0 && (f == nullptr || dcoeffs == nullptr || grad_params == nullptr))
        return fail(SE2_ERR_INVALID_ARG, "parameter gradients need f, dcoeffs and grad_params");
    if (n_params == 0 && grad_f == nullptr) return fail(SE2_ERR_INVALID_ARG, "nothing to compute");
    const size_t re = p->elem / 2;
    if (!aligned(grad_out, re) || (f && !aligned(f, re)) || (grad_f && !aligned(grad_f, re)) ||
        !aligned(coeffs, p->elem) || (log_scale && !aligned(log_scale, 8)) || (grad_params && !aligned(grad_params, 8)))
        return fail(SE2_ERR_INVALID_ARG, "misaligned pointer");
    for (int i = 0; i < n_params; ++i)
        if (dcoeffs[i] == nullptr || !aligned(dcoeffs[i], p->elem)) return fail(SE2_ERR_INVALID_ARG, "dcoeffs[%d] NULL or misaligned", i);
    if (grad_f != nullptr && (grad_f == grad_out || grad_f == f)) return fail(SE2_ERR_INVALID_ARG, "grad_f aliases an input");
    DeviceGuard guard(p->dev);
    cudaStream_t s = (cudaStream_t)stream;
    st = !is_f64(p)
             ? run_backward<float>(p, grad_out, f, B, coeffs, log_scale, n_params, dcoeffs, grad_params, grad_f, s)
             : run_backward<double>(p, grad_out, f, B, coeffs, log_scale, n_params, dcoeffs, grad_params, grad_f, s);
    if (st != SE2_OK || grad_f == nullptr) return st;
    return check_finite(p, grad_f, (size_t)p->N * p->N * p->M * B, s);
}

se2_status se2_sample_radial_gaussian(se2_plan_t p, double sigma, double sigma_theta, double nu, void* P,
                                      void* dP_dsigma, void* dP_dsigma_theta, void* stream) {
    SE2_RANGE("se2_sample_radial_gaussian");
    se2_status st = check_plan(p);
    if (st != SE2_OK) return st;
    if (!(sigma > 0) || !(sigma_theta > 0)) return fail(SE2_ERR_INVALID_ARG, "sigma and sigma_theta must be > 0");
    if (P == nullptr && dP_dsigma == nullptr && dP_dsigma_theta == nullptr) return fail(SE2_ERR_INVALID_ARG, "no output");
    const size_t re = p->elem / 2;
    if ((P && !aligned(P, re)) || (dP_dsigma && !aligned(dP_dsigma, re)) || (dP_dsigma_theta && !aligned(dP_dsigma_theta, re)))
        return fail(SE2_ERR_INVALID_ARG, "misaligned pointer");
    DeviceGuard guard(p->dev);
    cudaStream_t s = (cudaStream_t)stream;
    const double x0 = (p->flags & SE2_GRID_ORIGIN_ZERO) ? 0.0 : -0.5;
    k_gauss_tables<<<(p->N + p->M + 127) / 128, 128, 0, s>>>(p->tab, p->N, p->M, sigma, sigma_theta, nu, x0);
    ++p->launches;
    const long long total = (long long)p->N * p->N * p->M;
    const int blocks = (int)((total + 255) / 256 < 4096 ? (total + 255) / 256 : 4096);
    if (!is_f64(p))
        k_gauss_fill<float><<<blocks, 256, 0, s>>>(p->tab, p->N, p->M, (float*)P, (float*)dP_dsigma, (float*)dP_dsigma_theta);
    else
        k_gauss_fill<double><<<blocks, 256, 0, s>>>(p->tab, p->N, p->M, (double*)P, (double*)dP_dsigma, (double*)dP_dsigma_theta);
    ++p->launches;
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "kernel launch");
    return SE2_OK;
}

static int sampler_blocks(const se2_plan_s* p) {
    const long long total = (long long)p->N * p->N * p->M;
    return (int)((total + 255) / 256 < 4096 ? (total + 255) / 256 : 4096);
}

se2_status se2_sample_se2_gaussian(se2_plan_t p, const double* beta, const double* Sigma, int images, void* P,
                                   void* stream) {
    SE2_RANGE("se2_sample_se2_gaussian");
    se2_status st = check_plan(p);
    if (st != SE2_OK) return st;
    if (beta == nullptr || Sigma == nullptr || P == nullptr) return fail(SE2_ERR_INVALID_ARG, "NULL pointer argument");
    if (images < 0 || images > 8) return fail(SE2_ERR_INVALID_ARG, "images=%d must be in [0, 8]", images);
    if (!aligned(P, p->elem / 2)) return fail(SE2_ERR_INVALID_ARG, "misaligned pointer");
    GaussSE2Args a;
    if (const char* why = make_gauss_args(beta, Sigma, &a)) return fail(SE2_ERR_INVALID_ARG, "%s", why);
    a.Nx = a.Ny = p->N;
    a.M = p->M;
    a.images = images;
    a.x0 = (p->flags & SE2_GRID_ORIGIN_ZERO) ? 0.0 : -0.5;
    DeviceGuard guard(p->dev);
    cudaStream_t s = (cudaStream_t)stream;
    if (!is_f64(p))
        k_se2_gauss_fill<float><<<sampler_blocks(p), 256, 0, s>>>(a, (float*)P);
    else
        k_se2_gauss_fill<double><<<sampler_blocks(p), 256, 0, s>>>(a, (double*)P);
    ++p->launches;
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "kernel launch");
    return SE2_OK;
}

se2_status se2_sample_deformed_gaussian(se2_plan_t p, const double* H, double nu, double s_theta, int images, void* P,
                                        void* stream) {
    SE2_RANGE("se2_sample_deformed_gaussian");
    se2_status st = check_plan(p);
    if (st != SE2_OK) return st;
    if (H == nullptr || P == nullptr) return fail(SE2_ERR_INVALID_ARG, "NULL pointer argument");
    if (images < 0 || images > 8) return fail(SE2_ERR_INVALID_ARG, "images=%d must be in [0, 8]", images);
    if (!aligned(P, p->elem / 2)) return fail(SE2_ERR_INVALID_ARG, "misaligned pointer");
    DeformedArgs a;
    if (const char* why = make_deformed_args(H, nu, s_theta, &a)) return fail(SE2_ERR_INVALID_ARG, "%s", why);
    a.Nx = a.Ny = p->N;
    a.M = p->M;
    a.images = images;
    a.x0 = (p->flags & SE2_GRID_ORIGIN_ZERO) ? 0.0 : -0.5;
    DeviceGuard guard(p->dev);
    cudaStream_t s = (cudaStream_t)stream;
    if (!is_f64(p))
        k_deformed_fill<float><<<sampler_blocks(p), 256, 0, s>>>(a, (float*)P);
    else
        k_deformed_fill<double><<<sampler_blocks(p), 256, 0, s>>>(a, (double*)P);
    ++p->launches;
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "kernel launch");
    return SE2_OK;
}

se2_status se2_separable_tables(se2_plan_t p, const double* params, const int* k, int kmax, int B, void* tables,
                                void* stream) {
    SE2_RANGE("se2_separable_tables");
    se2_status st = check_plan(p);
    if (st != SE2_OK) return st;
    if (params == nullptr || k == nullptr || tables == nullptr) return fail(SE2_ERR_INVALID_ARG, "NULL pointer argument");
    if (kmax < 1 || B < 1) return fail(SE2_ERR_INVALID_ARG, "kmax=%d and B=%d must be >= 1", kmax, B);
    if (!aligned(params, 8) || !aligned(k, 4) || !aligned(tables, p->elem)) return fail(SE2_ERR_INVALID_ARG, "misaligned pointer");
    DeviceGuard guard(p->dev);
    cudaStream_t s = (cudaStream_t)stream;
    const long long tps = (long long)(p->N / 2 + 1 + p->N + p->M);
    const size_t sm = sizeof(double) * 3 * ((size_t)p->N + p->M);
    const bool oz = (p->flags & SE2_GRID_ORIGIN_ZERO) != 0;
    const double x0 = oz ? 0.0 : -0.5;
    const int wfold = oz ? 0 : 1;
    if (!is_f64(p))
        k_sep_tables<float><<<B, 128, sm, s>>>(params, k, kmax, p->N, p->M, (float2*)tables, tps, x0, wfold);
    else
        k_sep_tables<double><<<B, 128, sm, s>>>(params, k, kmax, p->N, p->M, (double2*)tables, tps, x0, wfold);
    ++p->launches;
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "kernel launch");
    return SE2_OK;
}

se2_status se2_convolve_separable(se2_plan_t p, const void* f, int B, const void* tables, void* out, void* stream) {
    SE2_RANGE("se2_convolve_separable");
    se2_status st = check_plan(p);
    if (st != SE2_OK) return st;
    if (f == nullptr || tables == nullptr || out == nullptr) return fail(SE2_ERR_INVALID_ARG, "NULL pointer argument");
    if (B < 1 || B > p->batch) return fail(SE2_ERR_INVALID_ARG, "B=%d outside [1, %d]", B, p->batch);
    const size_t re = p->elem / 2;
    if (!aligned(f, re) || !aligned(out, re) || !aligned(tables, p->elem)) return fail(SE2_ERR_INVALID_ARG, "misaligned pointer");
    if (f == out) return fail(SE2_ERR_INVALID_ARG, "out aliases f");
    DeviceGuard guard(p->dev);
    cudaStream_t s = (cudaStream_t)stream;
    st = !is_f64(p) ? run_sep<float>(p, f, B, tables, out, s) : run_sep<double>(p, f, B, tables, out, s);
    if (st != SE2_OK) return st;
    return check_finite(p, out, (size_t)p->N * p->N * p->M * B, s);
}

se2_status se2_plan_status(se2_plan_t p, void* stream) {
    SE2_RANGE("se2_plan_status");
    se2_status st = check_plan(p);
    if (st != SE2_OK) return st;
    DeviceGuard guard(p->dev);
    cudaError_t e = cudaStreamSynchronize((cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(e, "cudaStreamSynchronize");
    int h = 0;
    e = cudaMemcpy(&h, p->err, sizeof(int), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMemcpy");
    if (h != 0) {
        e = cudaMemset(p->err, 0, sizeof(int));
        if (e != cudaSuccess) return cuda_fail(e, "cudaMemset");
        if (h == 5) return fail(SE2_ERR_NUMERIC, "an output held NaN or infinity (SE2_CHECK_FINITE)");
        return fail(SE2_ERR_TIMEOUT, "a bounded device-side wait gave up (code %d: 1 persistent kernel, 2 tensor cores, "
                                     "3 bulk-copy units, 4 dataflow kernel)", h);
    }
    return SE2_OK;
}

se2_status se2_debug_wait_timeout(se2_plan_t p, const void* f, const void* coeffs, void* out, void* stream) {
    SE2_RANGE("se2_debug_wait_timeout");
    se2_status st = check_plan(p);
    if (st != SE2_OK) return st;
    if (!p->persist) return fail(SE2_ERR_UNSUPPORTED, "plan does not use the persistent kernel");
    if (f == nullptr || coeffs == nullptr || out == nullptr) return fail(SE2_ERR_INVALID_ARG, "NULL pointer argument");
    DeviceGuard guard(p->dev);
    const void* c[1] = {coeffs};
    // one problem whose A->B wait can never be met; 4096 polls end it quickly
    return run_persist<float>(p, f, 1, c, nullptr, 1, out, (cudaStream_t)stream, 1u, 4096);
}

unsigned long long se2_plan_launches(se2_plan_t p) { return p == nullptr ? 0ull : p->launches; }

se2_status se2_plan_timing(se2_plan_t p, int on) {
    SE2_RANGE("se2_plan_timing");
    se2_status st = check_plan(p);
    if (st != SE2_OK) return st;
    p->timing = on != 0;
    p->tused = 0;
    return SE2_OK;
}

se2_status se2_plan_timing_read(se2_plan_t p, double* ms, long long* count) {
    SE2_RANGE("se2_plan_timing_read");
    se2_status st = check_plan(p);
    if (st != SE2_OK) return st;
    if (ms == nullptr || count == nullptr) return fail(SE2_ERR_INVALID_ARG, "NULL pointer argument");
    for (int u = 0; u < 4; ++u) {
        ms[u] = 0.0;
        count[u] = 0;
    }
    DeviceGuard guard(p->dev);
    for (size_t i = 0; i < p->tused; ++i) {
        cudaError_t e = cudaEventSynchronize(p->tev[2 * i + 1]);
        float t = 0.f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&t, p->tev[2 * i], p->tev[2 * i + 1]);
        if (e != cudaSuccess) return cuda_fail(e, "timing events");
        ms[p->tkind[i]] += t;
        ++count[p->tkind[i]];
    }
    return SE2_OK;
}

se2_status se2_convolve(se2_plan_t p, const void* f, int B, const void* coeffs, const double* log_scale,
                        void* out, void* stream) {
    SE2_RANGE("se2_convolve");
    const void* c[1] = {coeffs};
    const double* l[1] = {log_scale};
    return se2_convolve_chain(p, f, B, c, l, 1, out, stream);
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Batch plans: many independent problems of uneven sizes (N, M), each with a
// chain of separable radial kernels in factored form.
// ---------------------------------------------------------------------------
struct se2_batch_plan_s {
    struct Class {
        int N = 0, M = 0, count = 0, first = 0;   // first: packed position of its first problem
        long long goff = 0, toff = 0;             // offsets of its block in the packed grids / tables
        se2_plan_s* plan = nullptr;               // sub-plan (the chosen path)
        se2_plan_s* alt = nullptr;                // the other path's plan while tuning
        bool persistent = false;
        cudaStream_t st = nullptr;                // own stream (class 0 uses the caller's)
        cudaEvent_t done = nullptr;
        double tuned_ms = 0;
        int lane = 0;                             // stream lane it runs on (0: the caller's stream)
    };
    int n = 0, dev = 0;
    se2_precision prec = SE2_F32;
    unsigned flags = 0;
    std::vector<Class> cls;
    std::vector<int> pos;                         // problem -> packed position
    std::vector<long long> goff, toff;            // per problem: packed grid / table offset
    long long gtotal = 0, ttotal = 0;
    cudaEvent_t fork = nullptr;
    int lanes = 1;                                // concurrent stream lanes (1: classes one after another)
    std::vector<double> lane_ms;                  // tuned whole-batch ms per lane count (index = lanes)
    // the whole batch as one persistent launch (kf_batch_persist)
    struct OneLaunch {
        bool ready = false, on = false;
        se2::BClass* cls = nullptr;               // device [n_classes]
        unsigned* units = nullptr;                // device work list
        unsigned n_units = 0;
        unsigned* ctr = nullptr;                  // device [1 + 3 n]
        void* ring = nullptr;                     // scratch rings of all classes
        int* err = nullptr;
        int grid = 0;
        double tuned_ms = 0;
        unsigned long long launches = 0;
    } one;
};

namespace {

constexpr size_t kBatchScratch = (size_t)512 << 20;   // scratch cap of one class's sub-plan

void batch_one_free(se2_batch_plan_s* b) {
    auto& o = b->one;
    if (o.cls) dev_free(o.cls);
    if (o.units) dev_free(o.units);
    if (o.ctr) dev_free(o.ctr);
    if (o.ring) dev_free(o.ring);
    if (o.err) dev_free(o.err);
    o = se2_batch_plan_s::OneLaunch{};
}

void batch_free(se2_batch_plan_s* b) {
    batch_one_free(b);
    for (auto& c : b->cls) {
        if (c.plan) se2_plan_destroy(c.plan);
        if (c.alt) se2_plan_destroy(c.alt);
        if (c.st) cudaStreamDestroy(c.st);
        if (c.done) cudaEventDestroy(c.done);
    }
    if (b->fork) cudaEventDestroy(b->fork);
    delete b;
}

// Pipeline streams (depth 2) for a sub-plan whose creation chose depth 1, so
// that the tuner can try both.
se2_status ensure_pipe_streams(se2_plan_s* p) {
    if (p->aux[1] != nullptr) return SE2_OK;
    cudaError_t e = cudaSuccess;
    if (p->ev_fork == nullptr) e = cudaEventCreateWithFlags(&p->ev_fork, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&p->aux[1], cudaStreamNonBlocking);
    if (e == cudaSuccess && p->ev_join[1] == nullptr) e = cudaEventCreateWithFlags(&p->ev_join[1], cudaEventDisableTiming);
    return e == cudaSuccess ? SE2_OK : cuda_fail(e, "pipeline streams");
}

se2_status batch_check(se2_batch_plan_s* b) {
    if (b == nullptr) return fail(SE2_ERR_INVALID_ARG, "NULL batch plan");
    return SE2_OK;
}

// Spread the classes over `lanes` stream lanes: longest first, each to the
// lane with the least work so far (tuned ms once tuned, grid points before).
// Lane l > 0 runs on the stream of class l.
void batch_assign_lanes(se2_batch_plan_s* b, int lanes) {
    const int nc = (int)b->cls.size();
    lanes = lanes < 1 ? 1 : (lanes > nc ? nc : lanes);
    b->lanes = lanes;
    auto weight = [&](const se2_batch_plan_s::Class& c) {
        return c.tuned_ms > 0 ? c.tuned_ms : (double)c.N * c.N * c.M * c.count;
    };
    std::vector<int> order(nc);
    for (int i = 0; i < nc; ++i) order[i] = i;
    std::stable_sort(order.begin(), order.end(), [&](int a, int c) { return weight(b->cls[a]) > weight(b->cls[c]); });
    std::vector<double> load(lanes, 0.0);
    for (int i : order) {
        int l = 0;
        for (int q = 1; q < lanes; ++q)
            if (load[q] < load[l]) l = q;
        b->cls[i].lane = l;
        load[l] += weight(b->cls[i]);
    }
}

// One class's convolutions on stream s with its current sub-plan.
se2_status batch_run_class(se2_batch_plan_s* b, se2_batch_plan_s::Class& c, const unsigned char* f, const unsigned char* tab,
                           unsigned char* out, cudaStream_t s) {
    const size_t re = b->prec == SE2_F64 ? sizeof(double) : sizeof(float);
    return se2_convolve_separable(c.plan, f + c.goff * re, c.count, tab + c.toff * 2 * re, out + c.goff * re, s);
}

// The one-launch path: per class its unit counts, lag L (rounds; at least
// ~1.5 waves of units between a producer and its consumer) and ring of
// D = 3L + 1 scratch slots; the work list merges the classes' rounds (a
// class starts when the one before it stops issuing units A).  Allocates
// (not a convolve call).  SE2_ERR_UNSUPPORTED where the kernel carries a
// class's (N, M) not, or for FP64.
struct OneClass { unsigned nA, nB, nC; long long s4; int L, D, n, start; };

// The work list of the one-launch kernel for classes (N, M, count) in plan
// order and `grid` resident blocks (host only).  Fills per class its unit
// counts, lag L, ring slots D and first round; SE2_ERR_UNSUPPORTED where the
// kernel carries a class not.
se2_status batch_work_list(const se2_shape* shapes, const int* counts, int nc, int grid, std::vector<OneClass>& ci,
                           std::vector<unsigned>& units) {
    if (nc > 16) return fail(SE2_ERR_UNSUPPORTED, "the one-launch batch kernel carries at most 16 classes");
    if (grid < 1) return fail(SE2_ERR_INVALID_ARG, "grid=%d must be >= 1", grid);
    ci.assign(nc, OneClass{});
    for (int c = 0; c < nc; ++c) {
        OneClass& x = ci[c];
        if (counts[c] < 1 || counts[c] > 65535 || !batch_persist_units(shapes[c].N, shapes[c].M, &x.nA, &x.nB, &x.nC, &x.s4))
            return fail(SE2_ERR_UNSUPPORTED, "class N=%d, M=%d (%d problems) is not carried by the one-launch kernel",
                        shapes[c].N, shapes[c].M, counts[c]);
        const unsigned upr = x.nA + x.nB + x.nC;
        x.L = (int)((3u * (unsigned)grid / 2u + upr - 1) / upr);
        if (x.L < 1) x.L = 1;
        x.D = 3 * x.L + 1 < counts[c] ? 3 * x.L + 1 : counts[c];
        x.n = counts[c];
        x.start = c == 0 ? 0 : ci[c - 1].start + ci[c - 1].n;
    }
    // rounds: class c's round r = R - start holds A of r, B of r - L, C of r - 2L
    units.clear();
    int last = 0;
    for (int c = 0; c < nc; ++c) last = std::max(last, ci[c].start + ci[c].n + 2 * ci[c].L);
    for (int R = 0; R < last; ++R) {
        for (int c = 0; c < nc; ++c) {
            const OneClass& x = ci[c];
            const int r = R - x.start;
            if (r < 0 || r >= x.n + 2 * x.L) continue;
            if (r < x.n)
                for (unsigned u = 0; u < x.nA; ++u) units.push_back(unit_code(c, 0, (int)u, r));
            if (r - x.L >= 0 && r - x.L < x.n)
                for (unsigned u = 0; u < x.nB; ++u) units.push_back(unit_code(c, 1, (int)u, r - x.L));
            if (r - 2 * x.L >= 0 && r - 2 * x.L < x.n)
                for (unsigned u = 0; u < x.nC; ++u) units.push_back(unit_code(c, 2, (int)u, r - 2 * x.L));
        }
    }
    return SE2_OK;
}

se2_status batch_one_init(se2_batch_plan_s* b) {
    auto& o = b->one;
    if (o.ready) return SE2_OK;
    if (b->prec != SE2_F32) return fail(SE2_ERR_UNSUPPORTED, "the one-launch batch kernel is FP32 only");
    const int nc = (int)b->cls.size();
    int bps = 0, nsm = 0;
    cudaError_t e = batch_persist_prepare(&bps);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, b->dev);
    if (e != cudaSuccess) return cuda_fail(e, "one-launch kernel attributes");
    if (bps < 1) return fail(SE2_ERR_UNSUPPORTED, "the one-launch batch kernel does not fit an SM");
    const int grid = bps * nsm;
    std::vector<se2_shape> shp(nc);
    std::vector<int> cnt(nc);
    for (int c = 0; c < nc; ++c) {
        shp[c] = se2_shape{b->cls[c].N, b->cls[c].M};
        cnt[c] = b->cls[c].count;
    }
    std::vector<OneClass> ci;
    std::vector<unsigned> units;
    se2_status st = batch_work_list(shp.data(), cnt.data(), nc, grid, ci, units);
    if (st != SE2_OK) return st;
    size_t ring_bytes = 0;
    for (int c = 0; c < nc; ++c) ring_bytes += (size_t)ci[c].D * (size_t)ci[c].s4 * 16;
    // device state
    std::vector<BClass> hc(nc);
    {
        e = dev_alloc((void**)&o.cls, sizeof(BClass) * nc);
        if (e == cudaSuccess) e = dev_alloc((void**)&o.units, sizeof(unsigned) * units.size());
        if (e == cudaSuccess) e = dev_alloc((void**)&o.ctr, sizeof(unsigned) * (1 + 3 * (size_t)b->n));
        if (e == cudaSuccess) e = dev_alloc(&o.ring, ring_bytes);
        if (e == cudaSuccess) e = dev_alloc((void**)&o.err, sizeof(int));
        if (e != cudaSuccess) {
            batch_one_free(b);
            return fail(SE2_ERR_OOM, "one-launch batch state: %s", cudaGetErrorString(e));
        }
    }
    size_t at = 0;
    for (int c = 0; c < nc; ++c) {
        const auto& k = b->cls[c];
        const se2_plan_s* p = k.plan;
        BClass& h = hc[c];
        h = BClass{};
        h.a.s = (float4*)((unsigned char*)o.ring + at);
        h.a.s_pstride = ci[c].s4;
        h.a.twN = (const float2*)p->twN;
        h.a.twM = (const float2*)p->twM;
        h.a.k = 1;
        h.a.inv_L = 1.0 / ((double)k.N * k.N * k.M);
        h.a.wsign = (b->flags & SE2_GRID_ORIGIN_ZERO) ? 0 : 1;
        h.a.err = o.err;
        h.goff = k.goff;
        h.toff = k.toff;
        h.grid = (long long)k.N * k.N * k.M;
        h.tabs = (long long)(k.N / 2 + 1 + k.N + k.M);
        h.kind = batch_kind(k.N, k.M);
        h.first = k.first;
        h.slots = ci[c].D;
        h.nA = ci[c].nA;
        h.nB = ci[c].nB;
        h.nC = ci[c].nC;
        at += (size_t)ci[c].D * (size_t)ci[c].s4 * 16;
    }
    e = cudaMemcpy(o.cls, hc.data(), sizeof(BClass) * nc, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(o.units, units.data(), sizeof(unsigned) * units.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemset(o.err, 0, sizeof(int));
    if (e != cudaSuccess) {
        batch_one_free(b);
        return cuda_fail(e, "one-launch batch state");
    }
    o.n_units = (unsigned)units.size();
    o.grid = grid;
    o.ready = true;
    return SE2_OK;
}

se2_status batch_one_run(se2_batch_plan_s* b, const unsigned char* f, const unsigned char* tab, unsigned char* out,
                         cudaStream_t s, unsigned dep_extra, long long spin_limit) {
    auto& o = b->one;
    cudaError_t e = cudaMemsetAsync(o.ctr, 0, sizeof(unsigned) * (1 + 3 * (size_t)b->n), s);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMemsetAsync");
    BPArgs a{};
    a.cls = o.cls;
    a.units = o.units;
    a.n_units = o.n_units;
    a.f = (const float*)f;
    a.out = (float*)out;
    a.tables = (const float2*)tab;
    a.work = o.ctr;
    a.cnt = o.ctr + 1;
    a.err = o.err;
    a.spin_limit = spin_limit;
    a.dep_extra = dep_extra;
    launch_batch_persist((int)std::min<unsigned>(o.n_units, (unsigned)o.grid), s, a);
    ++o.launches;
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "kernel launch");
    return SE2_OK;
}

// Every class, on its lane: lane 0 is the caller's stream, lanes 1.. are
// class streams forked from it and joined back (events only: capturable).
// Inside a lane the classes run in class order.
se2_status batch_run(se2_batch_plan_s* b, const unsigned char* f, const unsigned char* tab, unsigned char* out,
                     cudaStream_t s) {
    const int L = b->lanes;
    cudaError_t e = cudaSuccess;
    if (L > 1) {
        e = cudaEventRecord(b->fork, s);
        for (int l = 1; l < L && e == cudaSuccess; ++l) e = cudaStreamWaitEvent(b->cls[l].st, b->fork, 0);
        if (e != cudaSuccess) return cuda_fail(e, "class fork");
    }
    for (auto& c : b->cls) {
        se2_status st = batch_run_class(b, c, f, tab, out, c.lane == 0 ? s : b->cls[c.lane].st);
        if (st != SE2_OK) return st;
    }
    for (int l = 1; l < L && e == cudaSuccess; ++l) {
        e = cudaEventRecord(b->cls[l].done, b->cls[l].st);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(s, b->cls[l].done, 0);
    }
    if (e != cudaSuccess) return cuda_fail(e, "class join");
    return SE2_OK;
}

}  // namespace

se2_status se2_batch_plan_create(se2_batch_plan_t* out, const se2_shape* shapes, int n, se2_precision precision,
                                 unsigned flags, int device) {
    SE2_RANGE("se2_batch_plan_create");
    if (out == nullptr || shapes == nullptr) return fail(SE2_ERR_INVALID_ARG, "NULL pointer argument");
    *out = nullptr;
    if (n < 1) return fail(SE2_ERR_INVALID_ARG, "n_problems=%d must be >= 1", n);
    if (flags & ~(SE2_GRID_ORIGIN_ZERO | SE2_CHECK_FINITE)) return fail(SE2_ERR_INVALID_ARG, "unsupported flags 0x%x", flags);
    for (int i = 0; i < n; ++i) {
        const int N = shapes[i].N, M = shapes[i].M;
        if (!is_pow2(N) || N < 8 || N > 512 || !is_pow2(M) || M < 2 || M > 128)
            return fail(SE2_ERR_UNSUPPORTED, "problem %d: N=%d, M=%d outside the plan sizes", i, N, M);
    }
    se2_batch_plan_s* b = new (std::nothrow) se2_batch_plan_s();
    if (b == nullptr) return fail(SE2_ERR_OOM, "host allocation failed");
    b->n = n;
    b->dev = device;
    b->prec = precision;
    b->flags = flags;
    // size classes, largest total work first; problems keep their order inside a class
    std::vector<std::pair<long long, long long>> key;   // (N, M) packed -> index
    std::vector<std::vector<int>> members;
    for (int i = 0; i < n; ++i) {
        const long long k = (long long)shapes[i].N << 32 | (unsigned)shapes[i].M;
        size_t c = 0;
        while (c < key.size() && key[c].first != k) ++c;
        if (c == key.size()) {
            key.push_back({k, (long long)c});
            members.emplace_back();
        }
        members[c].push_back(i);
    }
    std::vector<size_t> order(key.size());
    for (size_t c = 0; c < order.size(); ++c) order[c] = c;
    auto work = [&](size_t c) {
        const long long N = key[c].first >> 32, M = key[c].first & 0xffffffffll;
        return N * N * M * (long long)members[c].size();
    };
    std::sort(order.begin(), order.end(), [&](size_t a, size_t c) { return work(a) > work(c) || (work(a) == work(c) && a < c); });
    b->pos.assign(n, 0);
    b->goff.assign(n, 0);
    b->toff.assign(n, 0);
    int at = 0;
    for (size_t oc : order) {
        se2_batch_plan_s::Class c;
        c.N = (int)(key[oc].first >> 32);
        c.M = (int)(key[oc].first & 0xffffffffll);
        c.count = (int)members[oc].size();
        c.first = at;
        c.goff = b->gtotal;
        c.toff = b->ttotal;
        for (int i : members[oc]) {
            b->pos[i] = at++;
            b->goff[i] = b->gtotal;
            b->toff[i] = b->ttotal;
            b->gtotal += (long long)c.N * c.N * c.M;
            b->ttotal += (long long)(c.N / 2 + 1 + c.N + c.M);
        }
        b->cls.push_back(c);
    }
    DeviceGuard guard(device);
    se2_status st = SE2_OK;
    cudaError_t e = cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming);
    if (e != cudaSuccess) { batch_free(b); return cuda_fail(e, "events"); }
    for (size_t ci = 0; ci < b->cls.size(); ++ci) {
        auto& c = b->cls[ci];
        st = plan_create_impl(&c.plan, c.N, c.M, c.count, precision, flags, device, kBatchScratch);
        if (st == SE2_OK && c.plan->fast && c.plan->nslots >= 2) st = ensure_pipe_streams(c.plan);
        if (st == SE2_OK && ci > 0) {
            e = cudaStreamCreateWithFlags(&c.st, cudaStreamNonBlocking);
            if (e == cudaSuccess) e = cudaEventCreateWithFlags(&c.done, cudaEventDisableTiming);
            if (e != cudaSuccess) st = cuda_fail(e, "class streams");
        }
        if (st != SE2_OK) { batch_free(b); return st; }
    }
    batch_assign_lanes(b, 1);
    *out = b;
    return SE2_OK;
}

se2_status se2_batch_plan_destroy(se2_batch_plan_t b) {
    SE2_RANGE("se2_batch_plan_destroy");
    se2_status st = batch_check(b);
    if (st != SE2_OK) return st;
    DeviceGuard guard(b->dev);
    cudaDeviceSynchronize();
    batch_free(b);
    return SE2_OK;
}

se2_status se2_batch_plan_layout(se2_batch_plan_t b, int* position, long long* grid_offset, long long* table_offset,
                                 long long* grid_total, long long* table_total) {
    se2_status st = batch_check(b);
    if (st != SE2_OK) return st;
    for (int i = 0; i < b->n; ++i) {
        if (position) position[i] = b->pos[i];
        if (grid_offset) grid_offset[i] = b->goff[i];
        if (table_offset) table_offset[i] = b->toff[i];
    }
    if (grid_total) *grid_total = b->gtotal;
    if (table_total) *table_total = b->ttotal;
    return SE2_OK;
}

se2_status se2_batch_separable_tables(se2_batch_plan_t b, const double* params, const int* k, int kmax, void* tables,
                                      void* stream) {
    SE2_RANGE("se2_batch_separable_tables");
    se2_status st = batch_check(b);
    if (st != SE2_OK) return st;
    if (params == nullptr || k == nullptr || tables == nullptr) return fail(SE2_ERR_INVALID_ARG, "NULL pointer argument");
    const size_t re = b->prec == SE2_F64 ? sizeof(double) : sizeof(float);
    DeviceGuard guard(b->dev);
    cudaStream_t s = (cudaStream_t)stream;
    for (auto& c : b->cls) {
        st = se2_separable_tables(c.plan, params + (size_t)c.first * kmax * 3, k + c.first, kmax, c.count,
                                  static_cast<unsigned char*>(tables) + c.toff * 2 * re, s);
        if (st != SE2_OK) return st;
    }
    return SE2_OK;
}

se2_status se2_batch_convolve_separable(se2_batch_plan_t b, const void* f, const void* tables, void* out, void* stream) {
    SE2_RANGE("se2_batch_convolve_separable");
    se2_status st = batch_check(b);
    if (st != SE2_OK) return st;
    if (f == nullptr || tables == nullptr || out == nullptr) return fail(SE2_ERR_INVALID_ARG, "NULL pointer argument");
    const size_t re = b->prec == SE2_F64 ? sizeof(double) : sizeof(float);
    if (!aligned(f, re) || !aligned(out, re) || !aligned(tables, 2 * re)) return fail(SE2_ERR_INVALID_ARG, "misaligned pointer");
    const uintptr_t fa = (uintptr_t)f, oa = (uintptr_t)out, len = (uintptr_t)b->gtotal * re;
    if (fa < oa + len && oa < fa + len) return fail(SE2_ERR_INVALID_ARG, "out overlaps f");
    DeviceGuard guard(b->dev);
    cudaStream_t s = (cudaStream_t)stream;
    const auto* fb = static_cast<const unsigned char*>(f);
    const auto* tb = static_cast<const unsigned char*>(tables);
    auto* ob = static_cast<unsigned char*>(out);
    if (b->one.on) return batch_one_run(b, fb, tb, ob, s, 0, kSpinLimit);
    return batch_run(b, fb, tb, ob, s);
}

// The autotuner: per class, time the candidate schedules on the caller's data
// and keep the fastest.  Candidates: the FP32 fast path with pipeline depth 1
// (groups of the scratch size) or depth 2 with groups of 1, 2, 4, 8 .. 64
// problems (as the scratch allows), and the persistent dataflow kernel
// (SE2_PERSISTENT).  Then the number of stream lanes for the whole batch.
// Synchronous; not for stream capture.
se2_status se2_batch_tune(se2_batch_plan_t b, const void* f, const void* tables, void* out, int reps, void* stream) {
    SE2_RANGE("se2_batch_tune");
    se2_status st = batch_check(b);
    if (st != SE2_OK) return st;
    if (f == nullptr || tables == nullptr || out == nullptr) return fail(SE2_ERR_INVALID_ARG, "NULL pointer argument");
    if (reps < 1) reps = 1;
    DeviceGuard guard(b->dev);
    cudaStream_t s = (cudaStream_t)stream;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    if (e != cudaSuccess) return cuda_fail(e, "events");
    const auto* fb = static_cast<const unsigned char*>(f);
    const auto* tb = static_cast<const unsigned char*>(tables);
    auto* ob = static_cast<unsigned char*>(out);
    auto time_class = [&](se2_batch_plan_s::Class& c, float* ms) -> se2_status {
        se2_status r = batch_run_class(b, c, fb, tb, ob, s);   // warm-up
        if (r != SE2_OK) return r;
        cudaEventRecord(e0, s);
        for (int i = 0; i < reps && r == SE2_OK; ++i) r = batch_run_class(b, c, fb, tb, ob, s);
        cudaEventRecord(e1, s);
        if (r != SE2_OK) return r;
        cudaError_t x = cudaEventSynchronize(e1);
        if (x == cudaSuccess) x = cudaEventElapsedTime(ms, e0, e1);
        if (x != cudaSuccess) return cuda_fail(x, "tuning events");
        *ms /= reps;
        return SE2_OK;
    };
    for (auto& c : b->cls) {
        float best = 0.f, ms = 0.f;
        int bd = c.plan->pipe_depth, bg = c.plan->pipe_group;
        bool bp = false;
        if (c.plan->fast) {
            std::vector<std::pair<int, int>> cand{{1, c.plan->chunk}};
            if (c.plan->aux[1] != nullptr)
                for (int g = 1; g <= 64 && g < c.count; g *= 2)
                    if (2 * g <= c.plan->nslots) cand.push_back({2, g});
            bool first = true;
            for (auto [d, g] : cand) {
                c.plan->pipe_depth = d;
                c.plan->pipe_group = d > 1 ? g : 0;
                st = time_class(c, &ms);
                if (st != SE2_OK) break;
                if (first || ms < best) {
                    best = ms;
                    bd = d;
                    bg = c.plan->pipe_group;
                }
                first = false;
            }
            c.plan->pipe_depth = bd;
            c.plan->pipe_group = bg;
            if (st != SE2_OK) break;
            if (b->prec == SE2_F32) {   // the persistent dataflow kernel
                se2_plan_s* fast = c.plan;
                se2_plan_s* pers = nullptr;
                if (plan_create_impl(&pers, c.N, c.M, c.count, b->prec, b->flags | SE2_PERSISTENT, b->dev, kBatchScratch) == SE2_OK) {
                    c.plan = pers;
                    st = time_class(c, &ms);
                    c.plan = fast;
                    if (st == SE2_OK && ms < best) {
                        best = ms;
                        bp = true;
                        c.alt = fast;
                        c.plan = pers;
                    } else {
                        se2_plan_destroy(pers);
                    }
                    if (st != SE2_OK) break;
                }
            }
        } else {
            st = time_class(c, &best);
            if (st != SE2_OK) break;
        }
        c.persistent = bp;
        c.tuned_ms = best;
        if (c.alt) {   // keep only the chosen path's scratch
            se2_plan_destroy(c.alt);
            c.alt = nullptr;
        }
    }
    // then the concurrency of the classes: the whole batch with 1, 2, 3, 4 ..
    // and all lanes; concurrent classes compete for L2, where each pipeline
    // keeps its scratch, so more lanes is not always faster
    const int nc = (int)b->cls.size();
    b->lane_ms.assign(nc + 1, 0.0);
    if (st == SE2_OK) {
        int best_l = 1;
        double best_ms = 0;
        for (int L = 1; L <= nc && st == SE2_OK; L = (L < 4 || L == nc) ? L + 1 : nc) {
            batch_assign_lanes(b, L);
            st = batch_run(b, fb, tb, ob, s);   // warm-up
            cudaEventRecord(e0, s);
            for (int i = 0; i < reps && st == SE2_OK; ++i) st = batch_run(b, fb, tb, ob, s);
            cudaEventRecord(e1, s);
            if (st != SE2_OK) break;
            float ms = 0.f;
            e = cudaEventSynchronize(e1);
            if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
            if (e != cudaSuccess) { st = cuda_fail(e, "tuning events"); break; }
            b->lane_ms[L] = ms / reps;
            if (L == 1 || b->lane_ms[L] < best_ms) {
                best_ms = b->lane_ms[L];
                best_l = L;
            }
            if (L == nc) break;
        }
        batch_assign_lanes(b, best_l);
        // and the whole batch as one persistent launch, where the kernel
        // carries every class; kept only if it beats the best lanes
        b->one.on = false;
        if (st == SE2_OK && batch_one_init(b) == SE2_OK) {
            st = batch_one_run(b, fb, tb, ob, s, 0, kSpinLimit);   // warm-up
            // its first launch may also set up the kernel's local memory
            // (about 4 KB of stack per thread): keep that out of the timing
            if (st == SE2_OK && (e = cudaStreamSynchronize(s)) != cudaSuccess) st = cuda_fail(e, "warm-up");
            cudaEventRecord(e0, s);
            for (int i = 0; i < reps && st == SE2_OK; ++i) st = batch_one_run(b, fb, tb, ob, s, 0, kSpinLimit);
            cudaEventRecord(e1, s);
            float ms = 0.f;
            if (st == SE2_OK) {
                e = cudaEventSynchronize(e1);
                if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
                if (e != cudaSuccess) st = cuda_fail(e, "tuning events");
            }
            int h = 0;
            if (st == SE2_OK && cudaMemcpy(&h, b->one.err, sizeof(int), cudaMemcpyDeviceToHost) == cudaSuccess && h == 0) {
                b->one.tuned_ms = ms / reps;
                b->one.on = b->one.tuned_ms < best_ms;
            }
            if (!b->one.on) {   // keep the measurement, drop the state
                const double t = b->one.tuned_ms;
                batch_one_free(b);
                b->one.tuned_ms = t;
            }
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return st;
}

se2_status se2_batch_plan_one_launch(se2_batch_plan_t b, int mode, int* current, double* tuned_ms) {
    SE2_RANGE("se2_batch_plan_one_launch");
    se2_status st = batch_check(b);
    if (st != SE2_OK) return st;
    if (mode > 0) {
        DeviceGuard guard(b->dev);
        st = batch_one_init(b);
        if (st != SE2_OK) return st;
        b->one.on = true;
    } else if (mode == 0) {
        b->one.on = false;
    }
    if (current) *current = b->one.on ? 1 : 0;
    if (tuned_ms) *tuned_ms = b->one.tuned_ms;
    return SE2_OK;
}

se2_status se2_batch_plan_status(se2_batch_plan_t b, void* stream) {
    SE2_RANGE("se2_batch_plan_status");
    se2_status st = batch_check(b);
    if (st != SE2_OK) return st;
    DeviceGuard guard(b->dev);
    cudaError_t e = cudaStreamSynchronize((cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(e, "cudaStreamSynchronize");
    if (b->one.err != nullptr) {
        int h = 0;
        e = cudaMemcpy(&h, b->one.err, sizeof(int), cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) return cuda_fail(e, "cudaMemcpy");
        if (h != 0) {
            e = cudaMemset(b->one.err, 0, sizeof(int));
            if (e != cudaSuccess) return cuda_fail(e, "cudaMemset");
            return fail(SE2_ERR_TIMEOUT, "a bounded wait of the one-launch batch kernel gave up (code %d)", h);
        }
    }
    for (auto& c : b->cls) {
        st = se2_plan_status(c.plan, stream);
        if (st != SE2_OK) return st;
    }
    return SE2_OK;
}

se2_status se2_debug_batch_work_list(const se2_shape* shapes, const int* counts, int n_classes, int grid,
                                     unsigned* units, long long* n_units, int* slots, int* lag) {
    if (shapes == nullptr || counts == nullptr || n_units == nullptr) return fail(SE2_ERR_INVALID_ARG, "NULL pointer argument");
    std::vector<OneClass> ci;
    std::vector<unsigned> list;
    se2_status st = batch_work_list(shapes, counts, n_classes, grid, ci, list);
    if (st != SE2_OK) return st;
    if (units != nullptr) {
        if (*n_units < (long long)list.size()) return fail(SE2_ERR_INVALID_ARG, "units holds %lld codes, %zu needed", *n_units, list.size());
        std::copy(list.begin(), list.end(), units);
    }
    *n_units = (long long)list.size();
    for (int c = 0; c < n_classes; ++c) {
        if (slots) slots[c] = ci[c].D;
        if (lag) lag[c] = ci[c].L;
    }
    return SE2_OK;
}

se2_status se2_debug_batch_wait_timeout(se2_batch_plan_t b, const void* f, const void* tables, void* out, void* stream) {
    SE2_RANGE("se2_debug_batch_wait_timeout");
    se2_status st = batch_check(b);
    if (st != SE2_OK) return st;
    if (f == nullptr || tables == nullptr || out == nullptr) return fail(SE2_ERR_INVALID_ARG, "NULL pointer argument");
    DeviceGuard guard(b->dev);
    st = batch_one_init(b);
    if (st != SE2_OK) return st;
    // every unit B waits for one more unit A than its problem has; 4096 polls end the wait
    return batch_one_run(b, static_cast<const unsigned char*>(f), static_cast<const unsigned char*>(tables),
                         static_cast<unsigned char*>(out), (cudaStream_t)stream, 1u, 4096);
}

se2_status se2_batch_plan_lanes(se2_batch_plan_t b, int lanes, int* current, int* lane_of_class, double* lane_ms) {
    se2_status st = batch_check(b);
    if (st != SE2_OK) return st;
    if (lanes > 0) batch_assign_lanes(b, lanes);
    if (current) *current = b->lanes;
    const int nc = (int)b->cls.size();
    for (int ci = 0; ci < nc; ++ci) {
        if (lane_of_class) lane_of_class[ci] = b->cls[ci].lane;
        if (lane_ms) lane_ms[ci] = (size_t)(ci + 1) < b->lane_ms.size() ? b->lane_ms[ci + 1] : 0.0;
    }
    return SE2_OK;
}

se2_status se2_batch_plan_config(se2_batch_plan_t b, int* n_classes, se2_shape* shape, int* count, int* depth,
                                 int* group, int* persistent, double* tuned_ms) {
    se2_status st = batch_check(b);
    if (st != SE2_OK) return st;
    if (n_classes) *n_classes = (int)b->cls.size();
    for (size_t ci = 0; ci < b->cls.size(); ++ci) {
        const auto& c = b->cls[ci];
        if (shape) shape[ci] = se2_shape{c.N, c.M};
        if (count) count[ci] = c.count;
        if (depth) depth[ci] = c.persistent ? 0 : c.plan->pipe_depth;
        if (group) group[ci] = c.persistent ? 0 : (c.plan->pipe_depth > 1 ? c.plan->pipe_group : c.plan->chunk);
        if (persistent) persistent[ci] = c.persistent ? 1 : 0;
        if (tuned_ms) tuned_ms[ci] = c.tuned_ms;
    }
    return SE2_OK;
}

unsigned long long se2_batch_plan_launches(se2_batch_plan_t b) {
    if (b == nullptr) return 0;
    unsigned long long n = b->one.launches;
    for (const auto& c : b->cls) n += c.plan->launches;
    return n;
}
