// Odd sampling grids L = 2K+1 per axis with the output on an N-grid >= L
// (Section 4.2, Eq. MatSKfonG; Section 6.1, Eqs. Qf, W, MatSKfgonG;
// Algorithm SKLAlg).  Sizes here are the paper's own experiment shapes
// (e.g. L = (31, 33, 61) -> N = (36, 38, 76)): a few tens to a few hundred
// points per axis, anisotropic, not powers of two.  Each axis is a direct DFT
// (a small dense complex matrix applied to every line), which at these
// lengths costs a few hundred flops per point and needs no mixed-radix plan.
//
// Zero padding (Eq. Qf) never materialises: the inverse passes sum only the
// 2K+1 stored bins, with the exponentials of the output grid, which is what
// Proposition LtoN1D states.  The product of coefficient arrays, the sign
// W^k (Eq. W, signed frequencies) and 1/|L| are applied while the theta
// inverse pass loads its input.
//
// Passes, for a batch of problems (x fastest everywhere):
//   f [B][Lr][Ly][Lx] real
//   -> x forward, real to half spectrum  [B][Lr][Ly][Hx]   (Hx = Kx + 1)
//   -> y forward                          [B][Lr][Ly][Hx]
//   -> theta forward = DFT(F)             [B][Lr][Ly][Hx]
//   -> theta inverse onto Nr (x product)  [B][Nr][Ly][Hx]
//   -> y inverse onto Ny                  [B][Nr][Ny][Hx]
//   -> x inverse onto Nx, complex to real [B][Nr][Ny][Nx]
#include <cuda_runtime.h>

#include <cstdarg>
#include <cstdint>
#include <cmath>
#include <cstdio>
#include <new>
#include <type_traits>

#include "../../include/se2.h"
#include "se2_internal.h"
#include "se2_nvtx.h"
#include "se2_kernels.cuh"

using namespace se2;

struct se2_grid_plan_s {
    int Lx = 0, Ly = 0, Lr = 0, Nx = 0, Ny = 0, Nr = 0, Hx = 0;
    int batch = 0, prec = 0, dev = 0;
    unsigned flags = 0;
    size_t celem = 0;              // bytes of one complex element
    void* tab = nullptr;           // the six DFT tables, complex
    size_t toff[6] = {};           // their offsets, in complex elements
    void* buf[3] = {nullptr, nullptr, nullptr};   // ping-pong workspace; running product of Algorithm 6
    unsigned long long launches = 0;
};

namespace {

constexpr int kGridMaxK = 32;      // kernels in one chain
constexpr int kGridMaxL = 255;     // largest sampling size per axis
constexpr int kGridMaxN = 1024;    // largest output size per axis
constexpr int kGridThreads = 256;

se2_status gfail(se2_status st, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    set_last_error(buf);
    return st;
}

se2_status gcuda(cudaError_t e, const char* what) {
    return gfail(SE2_ERR_CUDA, "%s: %s (%s)", what, cudaGetErrorName(e), cudaGetErrorString(e));
}

struct GDevice {
    int prev = -1;
    explicit GDevice(int dev) {
        if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
        if (prev != dev) cudaSetDevice(dev);
    }
    ~GDevice() {
        int cur = -1;
        if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
    }
};

// Signed frequency of bin b for an odd length L = 2K+1 (Eq. tauKk inverted).
__host__ __device__ inline int sfreq(int b, int L) { return b <= (L - 1) / 2 ? b : b - L; }

// ---------------------------------------------------------------------------
// DFT tables, FP64 (sincospi of the exactly reduced rational angle), rounded
// to T.  Layouts follow the pass that reads them:
//   0: x forward  [Lx][Hx]  e^{-2 pi i kx n / Lx}                (row passes: [in][out])
//   1: y forward  [Ly][Ly]  e^{-2 pi i ky m / Ly}                (column passes: [out][in])
//   2: theta fwd  [Lr][Lr]  e^{-2 pi i kr l / Lr}
//   3: theta inv  [Nr][Lr]  e^{+2 pi i s(kr) l' / Nr}
//   4: y inverse  [Ny][Ly]  e^{+2 pi i s(ky) m' / Ny}
//   5: x inverse  [Hx][Nx]  w(kx) e^{+2 pi i kx n' / Nx}, w = 1 at kx = 0, else 2
// ---------------------------------------------------------------------------
struct TabArgs {
    int Lx, Ly, Lr, Nx, Ny, Nr, Hx;
    long long off[6], total;
};

__device__ inline void cis_frac(long long num, long long den, int sign, double& c, double& s) {
    long long r = num % den;
    if (r < 0) r += den;
    double sp, cp;
    sincospi(2.0 * (double)r / (double)den, &sp, &cp);
    c = cp;
    s = sign * sp;
}

template <typename T>
__global__ void k_grid_tables(TabArgs a, c2<T>* tab) {
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < a.total;
         e += (long long)gridDim.x * blockDim.x) {
        double c = 0, s = 0, w = 1;
        if (e < a.off[1]) {                                  // x forward [n][kx]
            const long long t = e - a.off[0];
            const int n = (int)(t / a.Hx), kx = (int)(t % a.Hx);
            cis_frac((long long)kx * n, a.Lx, -1, c, s);
        } else if (e < a.off[2]) {                           // y forward [ky][m]
            const long long t = e - a.off[1];
            const int ky = (int)(t / a.Ly), m = (int)(t % a.Ly);
            cis_frac((long long)ky * m, a.Ly, -1, c, s);
        } else if (e < a.off[3]) {                           // theta forward [kr][l]
            const long long t = e - a.off[2];
            const int kr = (int)(t / a.Lr), l = (int)(t % a.Lr);
            cis_frac((long long)kr * l, a.Lr, -1, c, s);
        } else if (e < a.off[4]) {                           // theta inverse [l'][kr]
            const long long t = e - a.off[3];
            const int l = (int)(t / a.Lr), kb = (int)(t % a.Lr);
            cis_frac((long long)sfreq(kb, a.Lr) * l, a.Nr, +1, c, s);
        } else if (e < a.off[5]) {                           // y inverse [m'][ky]
            const long long t = e - a.off[4];
            const int m = (int)(t / a.Ly), kb = (int)(t % a.Ly);
            cis_frac((long long)sfreq(kb, a.Ly) * m, a.Ny, +1, c, s);
        } else {                                             // x inverse [kx][n']
            const long long t = e - a.off[5];
            const int kx = (int)(t / a.Nx), n = (int)(t % a.Nx);
            cis_frac((long long)kx * n, a.Nx, +1, c, s);
            w = kx == 0 ? 1.0 : 2.0;
        }
        tab[e] = mk<T>((T)(w * c), (T)(w * s));
    }
}

// ---------------------------------------------------------------------------
// One axis pass.  Column q of the pass (a line along the axis) has its element
// i at  (q / inner) * so + (q % inner) + i * si  (input and output alike, with
// their own strides).  Row passes (x, inner = 1) put the output index on the
// lanes; column passes (y, theta) put 32 neighbouring columns on the lanes.
// ---------------------------------------------------------------------------
enum GridMode { GM_R2C = 0, GM_C2C = 1, GM_MUL = 2, GM_C2R = 3 };

template <typename T>
struct GridPass {
    const void* in;
    void* out;
    const c2<T>* E;
    int n_in, n_out, inner;
    long long Q, in_so, in_si, out_so, out_sj;
    T out_scale;
    // GM_MUL: input times scale * W^k * C_1 ... C_k at the same bin
    const c2<T>* C[kGridMaxK];
    long long c_bstride;          // per problem (0: one array for the batch)
    int k, Ly, Hx;
    int wpow;                     // W^wpow (k for a chain, p for step p of Algorithm 6)
    T in_scale;
    c2<T>* acc;                   // when set: the unscaled product is stored back here (running product)
};

__device__ __forceinline__ long long gaddr(long long q, int inner, long long so) {
    return (q / inner) * so + (q % inner);
}

// Row passes: x forward (real input) and x inverse (real output).  A block
// holds kRows lines in shared memory.  Work items are (group of 4 lines,
// output index) pairs, numbered output-fastest, so that the lanes of a warp
// read neighbouring table entries and write neighbouring outputs whatever
// the output length; every item accumulates its 4 lines at once, so one
// table load feeds 4 multiply-adds.
constexpr int kRows = 64;
constexpr int kRowGroup = 4;

template <typename T, int MODE>
__global__ void __launch_bounds__(kGridThreads) k_grid_rows(GridPass<T> a) {
    extern __shared__ __align__(16) unsigned char g_smem[];
    using In = typename std::conditional<MODE == GM_R2C, T, c2<T>>::type;
    In* s = reinterpret_cast<In*>(g_smem);                                // [kRows][n_in]
    const long long q0 = (long long)blockIdx.x * kRows;
    const int tid = threadIdx.x;
    const In* in = static_cast<const In*>(a.in);
    for (int idx = tid; idx < kRows * a.n_in; idx += kGridThreads) {
        const int r = idx / a.n_in, i = idx % a.n_in;
        const long long q = q0 + r;
        In v;
        if constexpr (MODE == GM_R2C) v = T(0); else v = mk<T>(0, 0);
        if (q < a.Q) v = in[q * a.in_so + i * a.in_si];
        s[idx] = v;
    }
    __syncthreads();
    const long long left = a.Q - q0;
    const int groups = (int)((left < kRows ? left : kRows) + kRowGroup - 1) / kRowGroup;
    for (int w = tid; w < groups * a.n_out; w += kGridThreads) {
        const int g = w / a.n_out, j = w % a.n_out;
        const int r0 = g * kRowGroup;
        const In* sr = s + r0 * a.n_in;
        const c2<T>* e = a.E + j;
        if constexpr (MODE == GM_R2C) {
            T ar[kRowGroup] = {}, ai[kRowGroup] = {};
            for (int i = 0; i < a.n_in; ++i) {
                const c2<T> wv = e[(long long)i * a.n_out];
#pragma unroll
                for (int rr = 0; rr < kRowGroup; ++rr) {
                    const T x = sr[rr * a.n_in + i];
                    ar[rr] += wv.x * x;
                    ai[rr] += wv.y * x;
                }
            }
            c2<T>* out = static_cast<c2<T>*>(a.out);
#pragma unroll
            for (int rr = 0; rr < kRowGroup; ++rr) {
                const long long q = q0 + r0 + rr;
                if (q < a.Q) out[q * a.out_so + j * a.out_sj] = mk<T>(ar[rr], ai[rr]);
            }
        } else {
            T acc[kRowGroup] = {};
            for (int i = 0; i < a.n_in; ++i) {
                const c2<T> wv = e[(long long)i * a.n_out];
#pragma unroll
                for (int rr = 0; rr < kRowGroup; ++rr) {
                    const c2<T> v = sr[rr * a.n_in + i];
                    acc[rr] += wv.x * v.x - wv.y * v.y;                // Re(e v)
                }
            }
            T* out = static_cast<T*>(a.out);
#pragma unroll
            for (int rr = 0; rr < kRowGroup; ++rr) {
                const long long q = q0 + r0 + rr;
                if (q < a.Q) out[q * a.out_so + j * a.out_sj] = acc[rr];
            }
        }
    }
}

// Column passes: y and theta, forward and inverse; GM_MUL forms the product
// of the spectra while loading.  A block holds cols_tile<T>() neighbouring
// columns; each lane owns 2 (FP32) or 1 (FP64) of them and each warp 4
// outputs at a time, so per input sample a thread issues 2 shared loads and
// 4 (warp-uniform) table loads for 32 multiply-adds.
template <typename T>
constexpr int cols_tile() { return sizeof(T) == 4 ? 64 : 32; }
constexpr int kOutGroup = 4;
constexpr size_t kTableSmem = 48 * 1024;   // column-pass tables up to this size sit in shared memory

template <typename T>
__host__ __device__ inline bool table_in_smem(int n_in, int n_out) {
    return (size_t)n_in * n_out * sizeof(c2<T>) <= kTableSmem;
}

template <typename T, int MODE>
__global__ void __launch_bounds__(kGridThreads) k_grid_cols(GridPass<T> a) {
    constexpr int TC = cols_tile<T>(), CPT = TC / 32;
    extern __shared__ __align__(16) unsigned char g_smem[];
    c2<T>* s = reinterpret_cast<c2<T>*>(g_smem);                          // [n_in][TC]
    const long long q0 = (long long)blockIdx.x * TC;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const c2<T>* in = static_cast<const c2<T>*>(a.in);
    // the table follows the tile when it is small enough (table_in_smem)
    const c2<T>* E = a.E;
    if (table_in_smem<T>(a.n_in, a.n_out)) {
        c2<T>* es = s + (size_t)TC * a.n_in;
        for (int idx = tid; idx < a.n_in * a.n_out; idx += kGridThreads) es[idx] = a.E[idx];
        E = es;
    }
    for (int idx = tid; idx < TC * a.n_in; idx += kGridThreads) {
        const int c = idx % TC, i = idx / TC;
        const long long q = q0 + c;
        c2<T> v = mk<T>(0, 0);
        if (q < a.Q) {
            const long long off = gaddr(q, a.inner, a.in_so) + i * a.in_si;
            v = in[off];
            if (MODE == GM_MUL) {
                // column q = b * inner + (ky * Hx + kx); the bin index along theta is i
                const long long b = q / a.inner;
                const int cc = (int)(q % a.inner), ky = cc / a.Hx, kx = cc % a.Hx;
                const long long coff = b * a.c_bstride + (off - b * a.in_so);
                for (int t = 0; t < a.k; ++t) {
                    const c2<T> w = a.C[t][coff];
                    const T xr = v.x * w.x - v.y * w.y, xi = v.x * w.y + v.y * w.x;
                    v.x = xr;
                    v.y = xi;
                }
                if (a.acc != nullptr) a.acc[off] = v;   // each bin is loaded by one thread only
                T sr = a.in_scale;
                if ((a.wpow & 1) && ((kx + sfreq(ky, a.Ly)) & 1)) sr = -sr;
                v.x *= sr;
                v.y *= sr;
            }
        }
        s[idx] = v;
    }
    __syncthreads();
    c2<T>* out = static_cast<c2<T>*>(a.out);
    long long obase[CPT];
    bool ok[CPT];
    bool any = false;
#pragma unroll
    for (int cc = 0; cc < CPT; ++cc) {
        const long long q = q0 + lane + 32 * cc;
        ok[cc] = q < a.Q;
        obase[cc] = ok[cc] ? gaddr(q, a.inner, a.out_so) : 0;
        any |= ok[cc];
    }
    if (!any) return;
    for (int j0 = warp * kOutGroup; j0 < a.n_out; j0 += (kGridThreads / 32) * kOutGroup) {
        const c2<T>* e[kOutGroup];
#pragma unroll
        for (int r = 0; r < kOutGroup; ++r) e[r] = E + (long long)min(j0 + r, a.n_out - 1) * a.n_in;
        T ar[kOutGroup][CPT] = {}, ai[kOutGroup][CPT] = {};
#pragma unroll 4
        for (int i = 0; i < a.n_in; ++i) {
            c2<T> v[CPT];
#pragma unroll
            for (int cc = 0; cc < CPT; ++cc) v[cc] = s[i * TC + lane + 32 * cc];
#pragma unroll
            for (int r = 0; r < kOutGroup; ++r) {
                const c2<T> w = e[r][i];
#pragma unroll
                for (int cc = 0; cc < CPT; ++cc) {
                    ar[r][cc] += w.x * v[cc].x - w.y * v[cc].y;
                    ai[r][cc] += w.x * v[cc].y + w.y * v[cc].x;
                }
            }
        }
#pragma unroll
        for (int r = 0; r < kOutGroup; ++r) {
            if (j0 + r >= a.n_out) break;
#pragma unroll
            for (int cc = 0; cc < CPT; ++cc)
                if (ok[cc])
                    out[obase[cc] + (long long)(j0 + r) * a.out_sj] =
                        mk<T>(ar[r][cc] * a.out_scale, ai[r][cc] * a.out_scale);
        }
    }
}

template <typename T>
size_t pass_smem(int mode, int n_in, int n_out) {
    if (mode == GM_R2C) return (size_t)kRows * n_in * sizeof(T);
    if (mode == GM_C2R) return (size_t)kRows * n_in * sizeof(c2<T>);
    return ((size_t)cols_tile<T>() * n_in + (table_in_smem<T>(n_in, n_out) ? (size_t)n_in * n_out : 0)) *
           sizeof(c2<T>);
}

template <typename T>
cudaError_t launch_pass(se2_grid_plan_s* p, int mode, const GridPass<T>& a, cudaStream_t s) {
    const size_t sm = pass_smem<T>(mode, a.n_in, a.n_out);
    const int tile = (mode == GM_R2C || mode == GM_C2R) ? kRows : cols_tile<T>();
    const unsigned blocks = (unsigned)((a.Q + tile - 1) / tile);
    if (blocks == 0) return cudaSuccess;
    switch (mode) {
        case GM_R2C: k_grid_rows<T, GM_R2C><<<blocks, kGridThreads, sm, s>>>(a); break;
        case GM_C2R: k_grid_rows<T, GM_C2R><<<blocks, kGridThreads, sm, s>>>(a); break;
        case GM_C2C: k_grid_cols<T, GM_C2C><<<blocks, kGridThreads, sm, s>>>(a); break;
        default: k_grid_cols<T, GM_MUL><<<blocks, kGridThreads, sm, s>>>(a); break;
    }
    ++p->launches;
    return cudaGetLastError();
}

// Largest dynamic shared memory any pass asks for: rows of up to 255 real or
// 128 complex samples, columns of up to 255 samples.
template <typename T>
int max_pass_smem() {
    const size_t a = pass_smem<T>(GM_R2C, kGridMaxL, 1), b = pass_smem<T>(GM_C2R, (kGridMaxL - 1) / 2 + 1, 1),
                 c = (size_t)cols_tile<T>() * kGridMaxL * sizeof(c2<T>) + kTableSmem;
    return (int)(a > b ? (a > c ? a : c) : (b > c ? b : c));
}

template <typename T>
cudaError_t set_smem_attrs() {
    const int big = max_pass_smem<T>();
    cudaError_t e;
    if ((e = cudaFuncSetAttribute(k_grid_rows<T, GM_R2C>, cudaFuncAttributeMaxDynamicSharedMemorySize, big))) return e;
    if ((e = cudaFuncSetAttribute(k_grid_rows<T, GM_C2R>, cudaFuncAttributeMaxDynamicSharedMemorySize, big))) return e;
    if ((e = cudaFuncSetAttribute(k_grid_cols<T, GM_C2C>, cudaFuncAttributeMaxDynamicSharedMemorySize, big))) return e;
    return cudaFuncSetAttribute(k_grid_cols<T, GM_MUL>, cudaFuncAttributeMaxDynamicSharedMemorySize, big);
}

template <typename T>
const c2<T>* table(const se2_grid_plan_s* p, int i) {
    return static_cast<const c2<T>*>(p->tab) + p->toff[i];
}

// The three forward passes of B problems: real [B][Lr][Ly][Lx] -> DFT on
// [B][Lr][Ly][Hx] in `dst`, times `scale` (the last pass writes dst).
template <typename T>
cudaError_t forward(se2_grid_plan_s* p, const T* src, int B, c2<T>* dst, T scale, cudaStream_t s) {
    const long long slab = (long long)p->Lr * p->Ly * p->Hx;
    c2<T>* A = static_cast<c2<T>*>(p->buf[0]);
    c2<T>* Bf = static_cast<c2<T>*>(p->buf[1]);
    cudaError_t e;
    GridPass<T> a = {};
    a.out_scale = T(1);
    // x: lines (b, l, m), real Lx -> Hx bins
    a.in = src; a.out = A; a.E = table<T>(p, 0);
    a.n_in = p->Lx; a.n_out = p->Hx; a.inner = 1;
    a.Q = (long long)B * p->Lr * p->Ly;
    a.in_so = p->Lx; a.in_si = 1; a.out_so = p->Hx; a.out_sj = 1;
    if ((e = launch_pass<T>(p, GM_R2C, a, s))) return e;
    // y: columns (b, l, kx)
    a.in = A; a.out = Bf; a.E = table<T>(p, 1);
    a.n_in = p->Ly; a.n_out = p->Ly; a.inner = p->Hx;
    a.Q = (long long)B * p->Lr * p->Hx;
    a.in_so = (long long)p->Ly * p->Hx; a.in_si = p->Hx; a.out_so = a.in_so; a.out_sj = p->Hx;
    if ((e = launch_pass<T>(p, GM_C2C, a, s))) return e;
    // theta: columns (b, ky, kx)
    a.in = Bf; a.out = dst; a.E = table<T>(p, 2);
    a.n_in = p->Lr; a.n_out = p->Lr; a.inner = p->Ly * p->Hx;
    a.Q = (long long)B * p->Ly * p->Hx;
    a.in_so = slab; a.in_si = (long long)p->Ly * p->Hx; a.out_so = slab; a.out_sj = a.in_si;
    a.out_scale = scale;
    return launch_pass<T>(p, GM_C2C, a, s);
}

// The three inverse passes from the spectrum `spec` ([B][Lr][Ly][Hx]) to
// out ([B][Nr][Ny][Nx]): theta inverse with the product of the k coefficient
// arrays, W^wpow and 1/|L| formed while loading (and the unscaled product
// stored back into `acc` when given), then y and x.
template <typename T>
cudaError_t inverse_from(se2_grid_plan_s* p, c2<T>* spec, int B, const void* const* coeffs, int k, int wpow,
                         c2<T>* acc, T* out, cudaStream_t s) {
    const long long slab = (long long)p->Lr * p->Ly * p->Hx;
    c2<T>* A = static_cast<c2<T>*>(p->buf[0]);
    c2<T>* Bf = static_cast<c2<T>*>(p->buf[1]);
    cudaError_t e;
    GridPass<T> a = {};
    a.out_scale = T(1);
    // theta inverse onto Nr, with the product: columns (b, ky, kx)
    a.in = spec; a.out = Bf; a.E = table<T>(p, 3);
    a.n_in = p->Lr; a.n_out = p->Nr; a.inner = p->Ly * p->Hx;
    a.Q = (long long)B * p->Ly * p->Hx;
    a.in_so = slab; a.in_si = (long long)p->Ly * p->Hx;
    a.out_so = (long long)p->Nr * p->Ly * p->Hx; a.out_sj = a.in_si;
    for (int t = 0; t < k; ++t) a.C[t] = static_cast<const c2<T>*>(coeffs[t]);
    a.c_bstride = (p->flags & SE2_SHARED_KERNEL) ? 0 : slab;
    a.k = k; a.Ly = p->Ly; a.Hx = p->Hx;
    a.wpow = wpow;
    a.acc = acc;
    a.in_scale = (T)(1.0 / ((double)p->Lx * p->Ly * p->Lr));
    if ((e = launch_pass<T>(p, GM_MUL, a, s))) return e;
    // y inverse onto Ny: columns (b, l', kx)
    GridPass<T> y = {};
    y.out_scale = T(1);
    y.in = Bf; y.out = A; y.E = table<T>(p, 4);
    y.n_in = p->Ly; y.n_out = p->Ny; y.inner = p->Hx;
    y.Q = (long long)B * p->Nr * p->Hx;
    y.in_so = (long long)p->Ly * p->Hx; y.in_si = p->Hx;
    y.out_so = (long long)p->Ny * p->Hx; y.out_sj = p->Hx;
    if ((e = launch_pass<T>(p, GM_C2C, y, s))) return e;
    // x inverse onto Nx, complex to real: lines (b, l', m')
    GridPass<T> x = {};
    x.out_scale = T(1);
    x.in = A; x.out = out; x.E = table<T>(p, 5);
    x.n_in = p->Hx; x.n_out = p->Nx; x.inner = 1;
    x.Q = (long long)B * p->Nr * p->Ny;
    x.in_so = p->Hx; x.in_si = 1; x.out_so = p->Nx; x.out_sj = 1;
    return launch_pass<T>(p, GM_C2R, x, s);
}

template <typename T>
cudaError_t run_chain(se2_grid_plan_s* p, const T* f, int B, const void* const* coeffs, int k, T* out,
                      cudaStream_t s) {
    c2<T>* A = static_cast<c2<T>*>(p->buf[0]);
    cudaError_t e = forward<T>(p, f, B, A, T(1), s);
    if (e != cudaSuccess) return e;
    // the theta inverse reads A; the y inverse then overwrites it
    return inverse_from<T>(p, A, B, coeffs, k, k, nullptr, out, s);
}

// Algorithm 6 on the grid: one forward transform into the running product
// R (buf[2]), then per step p: R <- R C_p (stored back) and out_p from
// W^p R / |L|.
template <typename T>
cudaError_t run_chain_all(se2_grid_plan_s* p, const T* f, int B, const void* const* coeffs, int k, T* out,
                          cudaStream_t s) {
    c2<T>* R = static_cast<c2<T>*>(p->buf[2]);
    cudaError_t e = forward<T>(p, f, B, R, T(1), s);
    if (e != cudaSuccess) return e;
    const size_t per = (size_t)B * p->Nr * p->Ny * p->Nx;
    for (int q = 0; q < k; ++q) {
        const void* cq[1] = {coeffs[q]};
        if ((e = inverse_from<T>(p, R, B, cq, 1, q + 1, R, out + (size_t)q * per, s))) return e;
    }
    return cudaSuccess;
}

bool galigned(const void* ptr, size_t a) { return ((uintptr_t)ptr % a) == 0; }

se2_status check_gplan(se2_grid_plan_t p) {
    if (p == nullptr) return gfail(SE2_ERR_INVALID_ARG, "plan is NULL");
    return SE2_OK;
}

}  // namespace

namespace {
// f^[k; L] = (-1)^(k1 + k2) C(tau(k)) (Eq. FkLv) from the half spectrum C of
// real samples; a negative k1 reads the Hermitian partner -k and conjugates.
template <typename T>
__global__ void k_ffc_at(const c2<T>* C, int Lx, int Ly, int Lr, int Hx, int k1, int k2, int k3, double* out) {
    const bool conj = k1 < 0;
    if (conj) {
        k1 = -k1;
        k2 = -k2;
        k3 = -k3;
    }
    const int ty = ((k2 % Ly) + Ly) % Ly, tr = ((k3 % Lr) + Lr) % Lr;
    const c2<T> v = C[((size_t)tr * Ly + ty) * Hx + k1];
    double re = (double)v.x, im = conj ? -(double)v.y : (double)v.y;
    if ((k1 + k2) & 1) {
        re = -re;
        im = -im;
    }
    out[0] = re;
    out[1] = im;
    (void)Lx;
}
}  // namespace

extern "C" {

se2_status se2_grid_plan_create(se2_grid_plan_t* out, const int* L, const int* N, int batch, int precision,
                                unsigned flags, int device) {
    SE2_RANGE("se2_grid_plan_create");
    if (out == nullptr) return gfail(SE2_ERR_INVALID_ARG, "plan pointer is NULL");
    *out = nullptr;
    if (L == nullptr || N == nullptr) return gfail(SE2_ERR_INVALID_ARG, "L or N is NULL");
    for (int i = 0; i < 3; ++i) {
        if (L[i] < 1 || L[i] > kGridMaxL || (L[i] & 1) == 0)
            return gfail(SE2_ERR_UNSUPPORTED, "L[%d]=%d: sampling sizes must be odd (L = 2K+1) in [1, %d]", i, L[i],
                         kGridMaxL);
        if (N[i] < L[i] || N[i] > kGridMaxN)
            return gfail(SE2_ERR_INVALID_ARG, "N[%d]=%d: output sizes must satisfy L <= N <= %d", i, N[i], kGridMaxN);
    }
    if (batch < 1) return gfail(SE2_ERR_INVALID_ARG, "batch=%d must be >= 1", batch);
    if (precision != SE2_F32 && precision != SE2_F64)
        return gfail(SE2_ERR_UNSUPPORTED, "precision %d: the grid path runs SE2_F32 or SE2_F64", precision);
    if (flags & ~(unsigned)SE2_SHARED_KERNEL) return gfail(SE2_ERR_UNSUPPORTED, "flags 0x%x: only SE2_SHARED_KERNEL", flags);
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev)
        return gfail(SE2_ERR_INVALID_ARG, "device %d not available", device);
    se2_grid_plan_s* p = new (std::nothrow) se2_grid_plan_s();
    if (p == nullptr) return gfail(SE2_ERR_OOM, "host allocation failed");
    p->Lx = L[0]; p->Ly = L[1]; p->Lr = L[2];
    p->Nx = N[0]; p->Ny = N[1]; p->Nr = N[2];
    p->Hx = (p->Lx - 1) / 2 + 1;
    p->batch = batch;
    p->prec = precision;
    p->dev = device;
    p->flags = flags;
    p->celem = precision == SE2_F64 ? 16 : 8;
    GDevice guard(device);
    TabArgs ta;
    ta.Lx = p->Lx; ta.Ly = p->Ly; ta.Lr = p->Lr; ta.Nx = p->Nx; ta.Ny = p->Ny; ta.Nr = p->Nr; ta.Hx = p->Hx;
    const long long sz[6] = {(long long)p->Lx * p->Hx, (long long)p->Ly * p->Ly, (long long)p->Lr * p->Lr,
                             (long long)p->Nr * p->Lr, (long long)p->Ny * p->Ly, (long long)p->Hx * p->Nx};
    long long acc = 0;
    for (int i = 0; i < 6; ++i) {
        ta.off[i] = acc;
        p->toff[i] = (size_t)acc;
        acc += sz[i];
    }
    ta.total = acc;
    const size_t ws = (size_t)batch * p->Nr * p->Ny * p->Hx * p->celem;
    cudaError_t e = dev_alloc((void**)&p->tab, (size_t)acc * p->celem);
    if (e == cudaSuccess) e = dev_alloc((void**)&p->buf[0], ws);
    if (e == cudaSuccess) e = dev_alloc((void**)&p->buf[1], ws);
    if (e == cudaSuccess) e = dev_alloc((void**)&p->buf[2], (size_t)batch * p->Lr * p->Ly * p->Hx * p->celem);
    if (e != cudaSuccess) {
        cudaGetLastError();
        se2_grid_plan_destroy(p);
        return gfail(SE2_ERR_OOM, "device allocation of %zu bytes failed",
                     2 * ws + (size_t)acc * p->celem + (size_t)batch * p->Lr * p->Ly * p->Hx * p->celem);
    }
    const int blocks = (int)((acc + 255) / 256 < 1024 ? (acc + 255) / 256 : 1024);
    if (precision == SE2_F64) {
        e = set_smem_attrs<double>();
        if (e == cudaSuccess) k_grid_tables<double><<<blocks, 256>>>(ta, static_cast<c2<double>*>(p->tab));
    } else {
        e = set_smem_attrs<float>();
        if (e == cudaSuccess) k_grid_tables<float><<<blocks, 256>>>(ta, static_cast<c2<float>*>(p->tab));
    }
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e != cudaSuccess) {
        se2_grid_plan_destroy(p);
        return gcuda(e, "grid plan setup");
    }
    *out = p;
    return SE2_OK;
}

se2_status se2_grid_plan_destroy(se2_grid_plan_t p) {
    SE2_RANGE("se2_grid_plan_destroy");
    if (p == nullptr) return SE2_OK;
    {
        GDevice guard(p->dev);
        if (p->tab) dev_free(p->tab);
        if (p->buf[0]) dev_free(p->buf[0]);
        if (p->buf[1]) dev_free(p->buf[1]);
        if (p->buf[2]) dev_free(p->buf[2]);
    }
    delete p;
    return SE2_OK;
}

unsigned long long se2_grid_plan_launches(se2_grid_plan_t p) { return p ? p->launches : 0ull; }

static int grid_sampler_blocks(const se2_grid_plan_s* p) {
    const long long total = (long long)p->Lx * p->Ly * p->Lr;
    return (int)((total + 255) / 256 < 4096 ? (total + 255) / 256 : 4096);
}

se2_status se2_grid_sample_se2_gaussian(se2_grid_plan_t p, const double* beta, const double* Sigma, int images,
                                        void* P, void* stream) {
    SE2_RANGE("se2_grid_sample_se2_gaussian");
    se2_status st = check_gplan(p);
    if (st != SE2_OK) return st;
    if (beta == nullptr || Sigma == nullptr || P == nullptr) return gfail(SE2_ERR_INVALID_ARG, "NULL pointer argument");
    if (images < 0 || images > 8) return gfail(SE2_ERR_INVALID_ARG, "images=%d must be in [0, 8]", images);
    if (!galigned(P, p->celem / 2)) return gfail(SE2_ERR_INVALID_ARG, "misaligned pointer");
    GaussSE2Args a;
    if (const char* why = make_gauss_args(beta, Sigma, &a)) return gfail(SE2_ERR_INVALID_ARG, "%s", why);
    a.Nx = p->Lx;
    a.Ny = p->Ly;
    a.M = p->Lr;
    a.images = images;
    a.x0 = -0.5;
    GDevice guard(p->dev);
    cudaStream_t s = (cudaStream_t)stream;
    if (p->prec == SE2_F64)
        k_se2_gauss_fill<double><<<grid_sampler_blocks(p), 256, 0, s>>>(a, static_cast<double*>(P));
    else
        k_se2_gauss_fill<float><<<grid_sampler_blocks(p), 256, 0, s>>>(a, static_cast<float*>(P));
    ++p->launches;
    const cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? SE2_OK : gcuda(e, "kernel launch");
}

se2_status se2_grid_sample_deformed_gaussian(se2_grid_plan_t p, const double* H, double nu, double s_theta,
                                             int images, void* P, void* stream) {
    SE2_RANGE("se2_grid_sample_deformed_gaussian");
    se2_status st = check_gplan(p);
    if (st != SE2_OK) return st;
    if (H == nullptr || P == nullptr) return gfail(SE2_ERR_INVALID_ARG, "NULL pointer argument");
    if (images < 0 || images > 8) return gfail(SE2_ERR_INVALID_ARG, "images=%d must be in [0, 8]", images);
    if (!galigned(P, p->celem / 2)) return gfail(SE2_ERR_INVALID_ARG, "misaligned pointer");
    DeformedArgs a;
    if (const char* why = make_deformed_args(H, nu, s_theta, &a)) return gfail(SE2_ERR_INVALID_ARG, "%s", why);
    a.Nx = p->Lx;
    a.Ny = p->Ly;
    a.M = p->Lr;
    a.images = images;
    a.x0 = -0.5;
    GDevice guard(p->dev);
    cudaStream_t s = (cudaStream_t)stream;
    if (p->prec == SE2_F64)
        k_deformed_fill<double><<<grid_sampler_blocks(p), 256, 0, s>>>(a, static_cast<double*>(P));
    else
        k_deformed_fill<float><<<grid_sampler_blocks(p), 256, 0, s>>>(a, static_cast<float*>(P));
    ++p->launches;
    const cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? SE2_OK : gcuda(e, "kernel launch");
}

se2_status se2_accuracy_order(double eps, double grad_inf, int k_inf, double constant, long long* K) {
    SE2_RANGE("se2_accuracy_order");
    if (K == nullptr) return gfail(SE2_ERR_INVALID_ARG, "K is NULL");
    *K = 0;
    if (!(eps > 0) || !(eps < 1e300)) return gfail(SE2_ERR_INVALID_ARG, "eps=%g must be finite and > 0", eps);
    if (!(grad_inf >= 0) || !(grad_inf < 1e300))
        return gfail(SE2_ERR_INVALID_ARG, "grad_inf=%g must be finite and >= 0", grad_inf);
    if (k_inf < 0) return gfail(SE2_ERR_INVALID_ARG, "k_inf=%d must be >= 0", k_inf);
    const double c = constant > 0 ? constant : 32.0;   // Theorem fkLmain's constant
    const double beta = c * grad_inf / eps;
    if (!(beta < 4.0e18)) return gfail(SE2_ERR_UNSUPPORTED, "K = %g does not fit", beta);
    long long k = (long long)ceil(beta);
    if (k < k_inf) k = k_inf;
    if (k < 1) k = 1;                                    // K in N
    *K = k;
    return SE2_OK;
}

se2_status se2_grid_coeffs(se2_grid_plan_t p, const void* samples, int n, void* coeffs, void* stream) {
    SE2_RANGE("se2_grid_coeffs");
    se2_status st = check_gplan(p);
    if (st != SE2_OK) return st;
    if (samples == nullptr || coeffs == nullptr) return gfail(SE2_ERR_INVALID_ARG, "NULL pointer argument");
    if (n < 1 || n > p->batch) return gfail(SE2_ERR_INVALID_ARG, "n=%d must be in [1, batch=%d]", n, p->batch);
    if (!galigned(samples, p->celem / 2) || !galigned(coeffs, p->celem))
        return gfail(SE2_ERR_INVALID_ARG, "misaligned pointer");
    GDevice guard(p->dev);
    cudaStream_t s = (cudaStream_t)stream;
    const double inv = 1.0 / ((double)p->Lx * p->Ly * p->Lr);
    cudaError_t e = p->prec == SE2_F64
                        ? forward<double>(p, static_cast<const double*>(samples), n, static_cast<c2<double>*>(coeffs),
                                          inv, s)
                        : forward<float>(p, static_cast<const float*>(samples), n, static_cast<c2<float>*>(coeffs),
                                         (float)inv, s);
    if (e != cudaSuccess) return gcuda(e, "kernel launch");
    return SE2_OK;
}

se2_status se2_grid_ffc_at(se2_grid_plan_t p, const void* coeffs, int index, int k1, int k2, int k3, double* out,
                           void* stream) {
    SE2_RANGE("se2_grid_ffc_at");
    se2_status st = check_gplan(p);
    if (st != SE2_OK) return st;
    if (coeffs == nullptr || out == nullptr) return gfail(SE2_ERR_INVALID_ARG, "NULL pointer argument");
    if (index < 0 || index >= p->batch) return gfail(SE2_ERR_INVALID_ARG, "index=%d outside [0, %d)", index, p->batch);
    const int Kx = (p->Lx - 1) / 2, Ky = (p->Ly - 1) / 2, Kr = (p->Lr - 1) / 2;
    if (k1 < -Kx || k1 > Kx || k2 < -Ky || k2 > Ky || k3 < -Kr || k3 > Kr)
        return gfail(SE2_ERR_INVALID_ARG, "k = (%d, %d, %d) outside |k| <= K = (%d, %d, %d)", k1, k2, k3, Kx, Ky, Kr);
    if (!galigned(coeffs, p->celem) || !galigned(out, 8)) return gfail(SE2_ERR_INVALID_ARG, "misaligned pointer");
    GDevice guard(p->dev);
    cudaStream_t s = (cudaStream_t)stream;
    const size_t per = (size_t)p->Lr * p->Ly * p->Hx;
    if (p->prec == SE2_F64)
        k_ffc_at<double><<<1, 1, 0, s>>>(static_cast<const c2<double>*>(coeffs) + (size_t)index * per, p->Lx, p->Ly, p->Lr,
                                         p->Hx, k1, k2, k3, out);
    else
        k_ffc_at<float><<<1, 1, 0, s>>>(static_cast<const c2<float>*>(coeffs) + (size_t)index * per, p->Lx, p->Ly, p->Lr,
                                        p->Hx, k1, k2, k3, out);
    ++p->launches;
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return gcuda(e, "kernel launch");
    return SE2_OK;
}

se2_status se2_grid_convolve_chain(se2_grid_plan_t p, const void* f, int B, const void* const* coeffs, int k,
                                   void* out, void* stream) {
    SE2_RANGE("se2_grid_convolve_chain");
    se2_status st = check_gplan(p);
    if (st != SE2_OK) return st;
    if (f == nullptr || out == nullptr) return gfail(SE2_ERR_INVALID_ARG, "NULL pointer argument");
    if (B < 1 || B > p->batch) return gfail(SE2_ERR_INVALID_ARG, "B=%d must be in [1, batch=%d]", B, p->batch);
    if (k < 0 || k > kGridMaxK) return gfail(SE2_ERR_INVALID_ARG, "k=%d must be in [0, %d]", k, kGridMaxK);
    if (k > 0 && coeffs == nullptr) return gfail(SE2_ERR_INVALID_ARG, "coeffs is NULL");
    if (!galigned(f, p->celem / 2) || !galigned(out, p->celem / 2)) return gfail(SE2_ERR_INVALID_ARG, "misaligned pointer");
    for (int t = 0; t < k; ++t)
        if (coeffs[t] == nullptr || !galigned(coeffs[t], p->celem))
            return gfail(SE2_ERR_INVALID_ARG, "coeffs[%d] NULL or misaligned", t);
    if (f == out) return gfail(SE2_ERR_INVALID_ARG, "out aliases f");
    GDevice guard(p->dev);
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e = p->prec == SE2_F64
                        ? run_chain<double>(p, static_cast<const double*>(f), B, coeffs, k, static_cast<double*>(out), s)
                        : run_chain<float>(p, static_cast<const float*>(f), B, coeffs, k, static_cast<float*>(out), s);
    if (e != cudaSuccess) return gcuda(e, "kernel launch");
    return SE2_OK;
}

se2_status se2_grid_convolve_chain_all(se2_grid_plan_t p, const void* f, int B, const void* const* coeffs, int k,
                                       void* out, void* stream) {
    SE2_RANGE("se2_grid_convolve_chain_all");
    se2_status st = check_gplan(p);
    if (st != SE2_OK) return st;
    if (f == nullptr || out == nullptr || coeffs == nullptr) return gfail(SE2_ERR_INVALID_ARG, "NULL pointer argument");
    if (B < 1 || B > p->batch) return gfail(SE2_ERR_INVALID_ARG, "B=%d must be in [1, batch=%d]", B, p->batch);
    if (k < 1 || k > kGridMaxK) return gfail(SE2_ERR_INVALID_ARG, "k=%d must be in [1, %d]", k, kGridMaxK);
    if (!galigned(f, p->celem / 2) || !galigned(out, p->celem / 2)) return gfail(SE2_ERR_INVALID_ARG, "misaligned pointer");
    for (int t = 0; t < k; ++t)
        if (coeffs[t] == nullptr || !galigned(coeffs[t], p->celem))
            return gfail(SE2_ERR_INVALID_ARG, "coeffs[%d] NULL or misaligned", t);
    const size_t re = p->celem / 2;
    const uintptr_t fa = (uintptr_t)f, oa = (uintptr_t)out;
    const size_t flen = (size_t)B * p->Lr * p->Ly * p->Lx * re, olen = (size_t)k * B * p->Nr * p->Ny * p->Nx * re;
    if (fa < oa + olen && oa < fa + flen) return gfail(SE2_ERR_INVALID_ARG, "out overlaps f");
    GDevice guard(p->dev);
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e = p->prec == SE2_F64
                        ? run_chain_all<double>(p, static_cast<const double*>(f), B, coeffs, k, static_cast<double*>(out), s)
                        : run_chain_all<float>(p, static_cast<const float*>(f), B, coeffs, k, static_cast<float*>(out), s);
    if (e != cudaSuccess) return gcuda(e, "kernel launch");
    return SE2_OK;
}

}  // extern "C"
