// CUDA kernels of the SE(2) convolution path (arXiv 2504.05149, Algorithms
// 3, 4 and 6 at output grid N = L).  All grids are [theta][y][x], x fastest.
//
// Work units for one problem (|L| = N*N*M points):
//   A  fwd_xt  (one y row):  real FFT along x of the M rows (two rows packed
//                            as one complex line), then the angular DFT of the
//                            N/2+1 columns in shared memory  -> scratch S
//   B  lines<CONV> (a group of (theta-bin, x-bin) lines): FFT along y,
//                            multiply by W^k . C_1 ... C_k / |L| (Eq. MatSqKfgG),
//                            inverse FFT along y, in place in S
//   C  inv_tx  (one y row):  inverse angular DFT, then complex-to-real inverse
//                            FFT along x of row pairs -> out
// They run either as three kernels (one unit per block), or inside one
// persistent kernel that takes units from a work list and waits (bounded) on
// per-problem counters, so that problems pipeline through a small ring of
// scratch slots that stays resident in L2.
// When the [M][N/2+1] slab of one y row does not fit in shared memory the
// x and theta steps run as separate passes (fwd_x, lines<FWD> along theta,
// ..., lines<INV> along theta, inv_x).
#pragma once
#include "se2_fft.cuh"

namespace se2 {

constexpr int kThreads = 256;
constexpr int kMaxChain = 32;
constexpr int kMaxParams = 4;

enum LineMode { LM_FWD = 0, LM_INV = 1, LM_CONV = 2, LM_COEF = 3, LM_ADJ = 4, LM_SEP = 5 };

// Slab pitch (complex elements) for the [M][N/2+1] slab: = 2 mod 16 so that
// the 8-lane angular teams of one warp hit distinct bank pairs.
template <int N> __host__ __device__ constexpr int slab_pitch() {
    constexpr int H = N / 2 + 1;
    return H + ((2 - H % 16) + 16) % 16;
}

// ---------------------------------------------------------------------------
// Global-memory access with L2 eviction hints: the scratch spectrum is kept
// (evict_last), streamed inputs/outputs are let go first (evict_first).
// Scratch is read through L2 only (.cg): another SM may have written it.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint64_t pol_keep() {
    uint64_t p;
    asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(p));
    return p;
}
__device__ __forceinline__ uint64_t pol_stream() {
    uint64_t p;
    asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
    return p;
}
__device__ __forceinline__ float2 ld_s(const float2* a, uint64_t pol) {
    float2 v;
    asm volatile("ld.global.cg.L2::cache_hint.v2.f32 {%0, %1}, [%2], %3;" : "=f"(v.x), "=f"(v.y) : "l"(a), "l"(pol));
    return v;
}
__device__ __forceinline__ double2 ld_s(const double2* a, uint64_t pol) {
    double2 v;
    asm volatile("ld.global.cg.L2::cache_hint.v2.f64 {%0, %1}, [%2], %3;" : "=d"(v.x), "=d"(v.y) : "l"(a), "l"(pol));
    return v;
}
__device__ __forceinline__ void st_s(float2* a, float2 v, uint64_t pol) {
    asm volatile("st.global.L2::cache_hint.v2.f32 [%0], {%1, %2}, %3;" :: "l"(a), "f"(v.x), "f"(v.y), "l"(pol) : "memory");
}
__device__ __forceinline__ void st_s(double2* a, double2 v, uint64_t pol) {
    asm volatile("st.global.L2::cache_hint.v2.f64 [%0], {%1, %2}, %3;" :: "l"(a), "d"(v.x), "d"(v.y), "l"(pol) : "memory");
}
// read-only streamed inputs (never written during a launch)
__device__ __forceinline__ float ld_in(const float* a, uint64_t pol) {
    float v;
    asm volatile("ld.global.nc.L1::no_allocate.L2::cache_hint.f32 %0, [%1], %2;" : "=f"(v) : "l"(a), "l"(pol));
    return v;
}
__device__ __forceinline__ double ld_in(const double* a, uint64_t pol) {
    double v;
    asm volatile("ld.global.nc.L1::no_allocate.L2::cache_hint.f64 %0, [%1], %2;" : "=d"(v) : "l"(a), "l"(pol));
    return v;
}
__device__ __forceinline__ float2 ld_in(const float2* a, uint64_t pol) {
    float2 v;
    asm volatile("ld.global.nc.L1::no_allocate.L2::cache_hint.v2.f32 {%0, %1}, [%2], %3;" : "=f"(v.x), "=f"(v.y) : "l"(a), "l"(pol));
    return v;
}
__device__ __forceinline__ double2 ld_in(const double2* a, uint64_t pol) {
    double2 v;
    asm volatile("ld.global.nc.L1::no_allocate.L2::cache_hint.v2.f64 {%0, %1}, [%2], %3;" : "=d"(v.x), "=d"(v.y) : "l"(a), "l"(pol));
    return v;
}
__device__ __forceinline__ void st_out(float* a, float v, uint64_t pol) {
    asm volatile("st.global.L2::cache_hint.f32 [%0], %1, %2;" :: "l"(a), "f"(v), "l"(pol) : "memory");
}
__device__ __forceinline__ void st_out(double* a, double v, uint64_t pol) {
    asm volatile("st.global.L2::cache_hint.f64 [%0], %1, %2;" :: "l"(a), "d"(v), "l"(pol) : "memory");
}

__device__ __forceinline__ float4 ld_s4(const float4* a, uint64_t pol) {
    float4 v;
    asm volatile("ld.global.cg.L2::cache_hint.v4.f32 {%0, %1, %2, %3}, [%4], %5;"
                 : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w) : "l"(a), "l"(pol));
    return v;
}
__device__ __forceinline__ void st_s4(float4* a, float4 v, uint64_t pol) {
    asm volatile("st.global.L2::cache_hint.v4.f32 [%0], {%1, %2, %3, %4}, %5;"
                 :: "l"(a), "f"(v.x), "f"(v.y), "f"(v.z), "f"(v.w), "l"(pol) : "memory");
}

// Copy one slab row of H complex elements between shared memory and the
// scratch (both 16-byte aligned) with 16-byte accesses, lanes 0..31 of a warp.
template <typename T, int H>
__device__ __forceinline__ void row_to_global(c2<T>* g, const c2<T>* sm, int lane, uint64_t pol) {
    if constexpr (sizeof(c2<T>) == 8) {
        constexpr int NV = (H - 1) / 2;
        const float4* sv = reinterpret_cast<const float4*>(sm);
        float4* gv = reinterpret_cast<float4*>(g);
        for (int i = lane; i < NV; i += 32) st_s4(gv + i, sv[i], pol);
        if (lane == 0) st_s(g + (H - 1), sm[H - 1], pol);
    } else {
        for (int i = lane; i < H; i += 32) st_s(g + i, sm[i], pol);
    }
}
template <typename T, int H>
__device__ __forceinline__ void row_from_global(c2<T>* sm, const c2<T>* g, int lane, uint64_t pol) {
    if constexpr (sizeof(c2<T>) == 8) {
        constexpr int NV = (H - 1) / 2;
        float4* sv = reinterpret_cast<float4*>(sm);
        const float4* gv = reinterpret_cast<const float4*>(g);
        for (int i = lane; i < NV; i += 32) sv[i] = ld_s4(gv + i, pol);
        if (lane == 0) sm[H - 1] = ld_s(g + (H - 1), pol);
    } else {
        for (int i = lane; i < H; i += 32) sm[i] = ld_s(g + i, pol);
    }
}

// Load the [M][N/2+1] slab of one y row (rows `rstride` apart in the scratch)
// into shared memory: every thread issues all of its loads before its first
// shared-memory store, so the loads are in flight together.
template <typename T, int N, int M>
__device__ __forceinline__ void slab_from_global(c2<T>* S, const c2<T>* g, size_t rstride, uint64_t pol) {
    constexpr int H = N / 2 + 1, SP = slab_pitch<N>();
    const int tid = threadIdx.x;
    if constexpr (sizeof(c2<T>) == 8) {
        constexpr int NV = (H - 1) / 2;                  // float4 per row
        constexpr int TOT = M * NV;
        constexpr int PER = (TOT + kThreads - 1) / kThreads;
        float4 v[PER];
#pragma unroll
        for (int q = 0; q < PER; ++q) {
            const int e = tid + q * kThreads;
            if (e < TOT) {
                const int r = e / NV, c = e - r * NV;
                v[q] = ld_s4(reinterpret_cast<const float4*>(g + r * rstride) + c, pol);
            }
        }
        c2<T> last = mk<T>(0, 0);
        if (tid < M) last = ld_s(g + tid * rstride + (H - 1), pol);
#pragma unroll
        for (int q = 0; q < PER; ++q) {
            const int e = tid + q * kThreads;
            if (e < TOT) {
                const int r = e / NV, c = e - r * NV;
                reinterpret_cast<float4*>(S + rowoff<M, SP>(r))[c] = v[q];
            }
        }
        if (tid < M) S[rowoff<M, SP>(tid) + H - 1] = last;
    } else {
        constexpr int TOT = M * H;
        constexpr int PER = (TOT + kThreads - 1) / kThreads;
        for (int q0 = 0; q0 < PER; q0 += 8) {
            c2<T> v[8];
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                const int e = tid + (q0 + q) * kThreads;
                if (q0 + q < PER && e < TOT) { const int r = e / H, c = e - r * H; v[q] = ld_s(g + r * rstride + c, pol); }
            }
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                const int e = tid + (q0 + q) * kThreads;
                if (q0 + q < PER && e < TOT) { const int r = e / H, c = e - r * H; S[rowoff<M, SP>(r) + c] = v[q]; }
            }
        }
    }
}

template <typename T>
struct XArgs {                 // fwd_xt / fwd_x / inv_tx / inv_x
    const T* f;                // real grids (fwd) or nullptr
    T* out;                    // real grids (inv) or nullptr
    size_t g_pstride;          // real elements per problem
    c2<T>* s;                  // scratch spectrum base
    size_t s_pstride;          // complex elements per problem in scratch
    int tp;                    // scratch row pitch (complex), >= N/2+1
    int M;                     // runtime M (split-path kernels)
    const c2<T>* twN;          // e^{-2 pi i n / N}, n < N
    const c2<T>* twM;          // e^{-2 pi i n / M}, n < M
    double* abs_sum;           // [problems] accumulators of sum |f|, or nullptr
};

template <typename T>
struct LArgs {
    c2<T>* s;                  // scratch spectrum base
    size_t s_pstride;
    long long outer_stride;    // complex elements between outer indices
    long long elem_stride;     // complex elements between consecutive points of a line
    int n_outer;               // number of outer indices
    int nk;                    // regular x bins per outer index (= N/2); bin nk is Nyquist
    int N;                     // grid size (for the C layout)
    const c2<T>* tw;           // e^{-2 pi i n / L}, n < L
    // LM_CONV: chain of coefficient arrays
    int k;
    const c2<T>* C[kMaxChain];
    const double* ls[kMaxChain];
    long long c_pstride;       // complex elements per problem in C (0 = shared)
    long long ls_pstride;      // doubles per problem in log_scale (0 = shared)
    int cp;                    // C row pitch (= N/2+1)
    double inv_L;              // 1 / |L|
    // LM_COEF: output coefficient arrays and normalisation
    c2<T>* cout;
    long long cout_pstride;
    const double* abs_sum;     // [problems] sum |P| or nullptr
    double* log_scale;         // [problems] out or nullptr
    int problem0;              // index of the first problem of this launch (for log_scale)
    // LM_ADJ: second spectrum (the forward input f), parameter derivatives
    c2<T>* s2;                 // scratch base of the f spectra (same problem stride)
    int want_grad;             // write the grad_f spectrum back in place of G
    int n_params;
    const c2<T>* dC[kMaxParams];
    double* grad_params;       // [n_params], accumulated
    // LM_SEP: separable coefficients C = tt[ktheta] ty[ky] tx[kx] per problem,
    // tables [problem][(N/2+1) + N + M] complex (tx, ty, tt), W^(k-1) folded in
    const c2<T>* sep;
    long long sep_pstride;
    int wsign;                 // 1: apply W (grids on Omega_L); 0: grids at x_i = i/N
};

// ---------------------------------------------------------------------------
// Unit A: forward x (real, packed row pairs) and theta of y row j.
// fprob / sprob: this problem's real grid and scratch spectrum.
// ---------------------------------------------------------------------------
template <typename T, int N, int M>
__device__ __forceinline__ void unit_fwd_xt(const XArgs<T>& a, const T* fprob, c2<T>* sprob, int j,
                                            double* abs_out, unsigned char* smem_raw, double* red) {
    constexpr int H = N / 2 + 1, SP = slab_pitch<N>();
    constexpr int R1 = Fac<N>::R1, R2 = Fac<N>::R2, TS = team_size<N>(), RM = reg_count<N>();
    constexpr int TEAMS = kThreads / TS, XS = xbuf_elems<N>();
    using TO = TeamOut<R1, R2>;
    c2<T>* S = reinterpret_cast<c2<T>*>(smem_raw);
    c2<T>* XB = S + slab_elems<M, SP>();
    const int tid = threadIdx.x;
    const T* fb = fprob + (size_t)j * N;
    const int team = tid / TS, lane = tid % TS;
    c2<T>* xb = XB + team * XS;
    const uint64_t pin = pol_stream(), pk = pol_keep();
    T abs_acc = 0;
    T wr[R1], wi[R1];
    load_twiddles<N, -1, T>(a.twN, lane, wr, wi);

    constexpr int NP = M / 2;
    for (int p0 = 0; p0 < NP; p0 += TEAMS) {
        const int p = p0 + team;
        const bool act = p < NP;
        T re[RM], im[RM];
#pragma unroll
        for (int i = 0; i < RM; ++i) { re[i] = 0; im[i] = 0; }
        if (act && lane < R2) {
            const T* r0 = fb + (size_t)(2 * p) * N * N;
            const T* r1 = r0 + (size_t)N * N;
#pragma unroll
            for (int q = 0; q < R1; ++q) {
                re[q] = ld_in(r0 + lane + R2 * q, pin);
                im[q] = ld_in(r1 + lane + R2 * q, pin);
            }
            if (abs_out != nullptr) {
#pragma unroll
                for (int q = 0; q < R1; ++q) abs_acc += fabs(re[q]) + fabs(im[q]);
            }
        }
        team_fft_r<R1, R2, -1, T>(re, im, lane, xb, wr, wi, SyncWarp());
        // lane holds Z at TO::idx; publish Z linearly to split the pair
        if (lane < TO::lanes) {
#pragma unroll
            for (int k = 0; k < TO::regs; ++k) xb[TO::idx(lane, k)] = mk<T>(re[k], im[k]);
        }
        __syncwarp();
        if (act && lane < TO::lanes) {
            c2<T>* s0 = S + rowoff<M, SP>(2 * p);
            c2<T>* s1 = S + rowoff<M, SP>(2 * p + 1);
#pragma unroll
            for (int k2 = 0; k2 < TO::regs; ++k2) {
                const int kk = TO::idx(lane, k2);
                if (kk <= N / 2) {
                    const c2<T> zm = xb[(N - kk) & (N - 1)];
                    const T zr = re[k2], zi = im[k2];
                    // X0 = (Z[k] + conj Z[N-k]) / 2, X1 = (Z[k] - conj Z[N-k]) / (2i)
                    s0[kk] = mk<T>((zr + zm.x) * (T)0.5, (zi - zm.y) * (T)0.5);
                    s1[kk] = mk<T>((zi + zm.y) * (T)0.5, (zm.x - zr) * (T)0.5);
                }
            }
        }
        __syncwarp();
    }
    if (abs_out != nullptr) {
        double v = (double)abs_acc;
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if ((tid & 31) == 0) red[tid >> 5] = v;
    }
    __syncthreads();
    if (abs_out != nullptr && tid == 0) {
        double v = 0;
        for (int w = 0; w < kThreads / 32; ++w) v += red[w];
        atomicAdd(abs_out, v);
    }
    {
        constexpr int TSM = team_size<M>(), TEAMSM = kThreads / TSM;
        const int tm = tid / TSM, lm = tid % TSM;
        T vr[Fac<M>::R1], vi[Fac<M>::R1];
        load_twiddles<M, -1, T>(a.twM, lm, vr, vi);
        for (int c0 = 0; c0 < H; c0 += TEAMSM) {
            const int c = c0 + tm;
            const bool act = c < H;
            column_fft_r<M, SP, -1, T>(S, act ? c : 0, lm, act, vr, vi, SyncWarp());
        }
    }
    __syncthreads();
    {
        const int w = tid >> 5, l32 = tid & 31;
        c2<T>* sb = sprob + (size_t)j * a.tp;
        for (int r = w; r < M; r += kThreads / 32)
            row_to_global<T, H>(sb + (size_t)r * N * a.tp, S + rowoff<M, SP>(r), l32, pk);
    }
}

// ---------------------------------------------------------------------------
// Unit C: inverse theta then complex-to-real x of y row j.
// ---------------------------------------------------------------------------
template <typename T, int N, int M>
__device__ __forceinline__ void unit_inv_tx(const XArgs<T>& a, const c2<T>* sprob, T* oprob, int j,
                                            unsigned char* smem_raw) {
    constexpr int H = N / 2 + 1, SP = slab_pitch<N>();
    constexpr int R1 = Fac<N>::R1, R2 = Fac<N>::R2, TS = team_size<N>(), RM = reg_count<N>();
    constexpr int TEAMS = kThreads / TS, XS = xbuf_elems<N>();
    using TO = TeamOut<R1, R2>;
    c2<T>* S = reinterpret_cast<c2<T>*>(smem_raw);
    c2<T>* XB = S + slab_elems<M, SP>();
    const int tid = threadIdx.x;
    const uint64_t pk = pol_keep(), po = pol_stream();
    slab_from_global<T, N, M>(S, sprob + (size_t)j * a.tp, (size_t)N * a.tp, pk);
    __syncthreads();
    {
        constexpr int TSM = team_size<M>(), TEAMSM = kThreads / TSM;
        const int tm = tid / TSM, lm = tid % TSM;
        T vr[Fac<M>::R1], vi[Fac<M>::R1];
        load_twiddles<M, +1, T>(a.twM, lm, vr, vi);
        for (int c0 = 0; c0 < H; c0 += TEAMSM) {
            const int c = c0 + tm;
            const bool act = c < H;
            column_fft_r<M, SP, +1, T>(S, act ? c : 0, lm, act, vr, vi, SyncWarp());
        }
    }
    __syncthreads();
    const int team = tid / TS, lane = tid % TS;
    c2<T>* xb = XB + team * XS;
    T* ob = oprob + (size_t)j * N;
    T wr[R1], wi[R1];
    load_twiddles<N, +1, T>(a.twN, lane, wr, wi);
    constexpr int NP = M / 2;
    for (int p0 = 0; p0 < NP; p0 += TEAMS) {
        const int p = p0 + team;
        const bool act = p < NP;
        T re[RM], im[RM];
#pragma unroll
        for (int i = 0; i < RM; ++i) { re[i] = 0; im[i] = 0; }
        if (act && lane < R2) {
            const c2<T>* s0 = S + rowoff<M, SP>(2 * p);
            const c2<T>* s1 = S + rowoff<M, SP>(2 * p + 1);
#pragma unroll
            for (int q = 0; q < R1; ++q) {
                const int kk = lane + R2 * q;
                c2<T> A, B;
                if (kk <= N / 2) {
                    A = s0[kk];
                    B = s1[kk];
                    if (kk == 0 || kk == N / 2) { A.y = 0; B.y = 0; }
                } else {
                    A = s0[N - kk];
                    B = s1[N - kk];
                    A.y = -A.y;
                    B.y = -B.y;
                }
                re[q] = A.x - B.y;      // Z = A + i B
                im[q] = A.y + B.x;
            }
        }
        team_fft_r<R1, R2, +1, T>(re, im, lane, xb, wr, wi, SyncWarp());
        if (act && lane < TO::lanes) {
            T* o0 = ob + (size_t)(2 * p) * N * N;
            T* o1 = o0 + (size_t)N * N;
#pragma unroll
            for (int k = 0; k < TO::regs; ++k) {
                st_out(o0 + TO::idx(lane, k), re[k], po);
                st_out(o1 + TO::idx(lane, k), im[k], po);
            }
        }
    }
}

// ---------------------------------------------------------------------------
// Unit B (and the split-path theta passes): FFTs of length L along one axis
// of the scratch spectrum for LINES consecutive lines (outer index o, x bin
// kx; kx fastest for coalescing) starting at line g * LINES.
//   LM_FWD / LM_INV: forward / unscaled inverse FFT in place
//   LM_CONV (y axis): forward, multiply by W^k C_1..C_k exp(sum ls) / |L|,
//                     inverse, in place
//   LM_COEF (y axis): forward, scale by 1 / (|L| s_b), write the external
//                     coefficient layout
// b is the problem index used for C / log_scale / coefficient output.
// ---------------------------------------------------------------------------
template <typename T, int L, int MODE>
__device__ __forceinline__ void unit_lines(const LArgs<T>& a, c2<T>* sprob, int b, long long g,
                                           unsigned char* smem_raw, double* sh_scale,
                                           c2<T>* sprob2 = nullptr, double* red = nullptr) {
    constexpr int R1 = Fac<L>::R1, R2 = Fac<L>::R2, TS = team_size<L>(), RM = reg_count<L>();
    constexpr int LINES = kThreads / TS;
    constexpr int XS = (Fac<L>::R1 * (Fac<L>::R2 + 1)) | 1;   // odd stride: lines in distinct banks
    using TO = TeamOut<R1, R2>;
    c2<T>* XB = reinterpret_cast<c2<T>*>(smem_raw);
    const int tid = threadIdx.x;
    const int c = tid % LINES, t = tid / LINES;
    const long long NR = (long long)a.n_outer * a.nk;
    const long long total = NR + a.n_outer;
    const long long line = g * LINES + c;
    const bool act = line < total;
    int o, kx;
    if (line < NR) { o = (int)(line / a.nk); kx = (int)(line - (long long)o * a.nk); }
    else { o = act ? (int)(line - NR) : 0; kx = a.nk; }
    c2<T>* base = sprob + o * a.outer_stride + kx;
    c2<T>* xb = XB + c * XS;
    const uint64_t pk = pol_keep();

    if constexpr (MODE == LM_CONV || MODE == LM_COEF || MODE == LM_ADJ || MODE == LM_SEP) {
        if (tid == 0) {
            double sc = a.inv_L;
            if constexpr (MODE == LM_CONV || MODE == LM_ADJ) {
                double lsum = 0;
                for (int i = 0; i < a.k; ++i)
                    if (a.ls[i] != nullptr) lsum += a.ls[i][b * a.ls_pstride];
                sc *= exp(lsum);
            } else {
                if (a.abs_sum != nullptr) {
                    const double s = a.abs_sum[b] * a.inv_L;   // mean |P|
                    double lg = 0;
                    if (s > 0) { sc /= s; lg = log(s); }
                    if (g == 0 && a.log_scale != nullptr) a.log_scale[a.problem0 + b] = lg;
                }
            }
            *sh_scale = sc;
        }
        __syncthreads();
    }

    T re[RM], im[RM];
#pragma unroll
    for (int i = 0; i < RM; ++i) { re[i] = 0; im[i] = 0; }
    if (act && t < R2) {
#pragma unroll
        for (int q = 0; q < R1; ++q) {
            const c2<T> v = ld_s(base + (long long)(t + R2 * q) * a.elem_stride, pk);
            re[q] = v.x;
            im[q] = v.y;
        }
    }
    if constexpr (MODE == LM_INV) {
        team_fft<R1, R2, +1, T>(re, im, t, xb, a.tw, SyncBlock());
    } else {
        team_fft<R1, R2, -1, T>(re, im, t, xb, a.tw, SyncBlock());
    }
    // lane t < TO::lanes now holds X[TO::idx(t, k)], k < TO::regs
    if constexpr (MODE == LM_FWD || MODE == LM_INV) {
        if (act && t < TO::lanes) {
#pragma unroll
            for (int k = 0; k < TO::regs; ++k) st_s(base + (long long)TO::idx(t, k) * a.elem_stride, mk<T>(re[k], im[k]), pk);
        }
    } else if constexpr (MODE == LM_COEF) {
        if (act && t < TO::lanes) {
            const T sc = (T)*sh_scale;
            c2<T>* cb = a.cout + b * a.cout_pstride + (long long)o * a.N * a.cp + kx;
#pragma unroll
            for (int k = 0; k < TO::regs; ++k) cb[(long long)TO::idx(t, k) * a.cp] = mk<T>(re[k] * sc, im[k] * sc);
        }
    } else if constexpr (MODE == LM_SEP) {
        // C from three 1-D tables (a chain of separable kernels), then W
        if (act && t < TO::lanes) {
            const T sc = (T)*sh_scale;
            const c2<T>* tb = a.sep + b * a.sep_pstride;
            const c2<T> cx = tb[kx];
            const c2<T> ct = tb[a.nk + 1 + a.N + o];
            // cx * ct, then * ty per ky
            const T xr = cx.x * ct.x - cx.y * ct.y, xi = cx.x * ct.y + cx.y * ct.x;
            c2<T> cy[TO::regs];
#pragma unroll
            for (int k = 0; k < TO::regs; ++k) cy[k] = tb[a.nk + 1 + TO::idx(t, k)];
#pragma unroll
            for (int k = 0; k < TO::regs; ++k) {
                const int ky = TO::idx(t, k);
                const T cr = xr * cy[k].x - xi * cy[k].y, ci = xr * cy[k].y + xi * cy[k].x;
                const T r = re[k] * cr - im[k] * ci;
                const T i2 = re[k] * ci + im[k] * cr;
                const bool neg = a.wsign && ((kx + ky) & 1);              // W
                re[k] = neg ? -r * sc : r * sc;
                im[k] = neg ? -i2 * sc : i2 * sc;
            }
        }
        if constexpr (R2 == 1) {
            fft_reg<R1, +1>(re, im);
            if (act) {
#pragma unroll
                for (int q = 0; q < R1; ++q) st_s(base + (long long)q * a.elem_stride, mk<T>(re[q], im[q]), pk);
            }
        } else {
            team_fft<R2, R1, +1, T>(re, im, t, xb, a.tw, SyncBlock());
            if (act && t < R2) {
#pragma unroll
                for (int q = 0; q < R1; ++q) st_s(base + (long long)(t + R2 * q) * a.elem_stride, mk<T>(re[q], im[q]), pk);
            }
        }
    } else if constexpr (MODE == LM_ADJ) {
        // transpose of the convolution (grad_f spectrum W conj(C) G^ e^{ls} / |L|)
        // and kernel-parameter partials (1/|L|) sum_k m_k Re(W dC_i conj(G^) F^)
        const uint64_t pin = pol_stream();
        T fr[RM], fi[RM];
        if (a.n_params > 0) {
#pragma unroll
            for (int i = 0; i < RM; ++i) { fr[i] = 0; fi[i] = 0; }
            c2<T>* base2 = sprob2 + o * a.outer_stride + kx;
            if (act && t < R2) {
#pragma unroll
                for (int q = 0; q < R1; ++q) {
                    const c2<T> v = ld_s(base2 + (long long)(t + R2 * q) * a.elem_stride, pk);
                    fr[q] = v.x;
                    fi[q] = v.y;
                }
            }
            team_fft<R1, R2, -1, T>(fr, fi, t, xb, a.tw, SyncBlock());
        }
        T acc[kMaxParams];
#pragma unroll
        for (int i = 0; i < kMaxParams; ++i) acc[i] = 0;
        if (act && t < TO::lanes) {
            const T sc = (T)*sh_scale;
            const long long coff = (long long)o * a.N * a.cp + kx;
            const T mk_ = (kx == 0 || kx == a.nk) ? (T)1 : (T)2;
            for (int i = 0; i < a.n_params; ++i) {
                const c2<T>* Db = a.dC[i] + b * a.c_pstride + coff;
                c2<T> d[TO::regs];
#pragma unroll
                for (int k = 0; k < TO::regs; ++k) d[k] = ld_in(Db + (long long)TO::idx(t, k) * a.cp, pin);
#pragma unroll
                for (int k = 0; k < TO::regs; ++k) {
                    const int ky = TO::idx(t, k);
                    const T w = (a.wsign && ((kx + ky) & 1)) ? (T)-1 : (T)1;
                    // Re(W dC conj(G^) F^)
                    const T pr = re[k] * fr[k] + im[k] * fi[k];
                    const T pi = re[k] * fi[k] - im[k] * fr[k];
                    const T v = mk_ * w * (d[k].x * pr - d[k].y * pi);
#pragma unroll
                    for (int q = 0; q < kMaxParams; ++q) if (q == i) acc[q] += v;
                }
            }
            if (a.want_grad) {
                const c2<T>* Cb = a.C[0] + b * a.c_pstride + coff;
                c2<T> cv[TO::regs];
#pragma unroll
                for (int k = 0; k < TO::regs; ++k) cv[k] = ld_in(Cb + (long long)TO::idx(t, k) * a.cp, pin);
#pragma unroll
                for (int k = 0; k < TO::regs; ++k) {
                    const int ky = TO::idx(t, k);
                    const T w = (a.wsign && ((kx + ky) & 1)) ? (T)-1 : (T)1;
                    // W conj(C) G^ * scale
                    const T xr = (cv[k].x * re[k] + cv[k].y * im[k]) * sc * w;
                    const T xi = (cv[k].x * im[k] - cv[k].y * re[k]) * sc * w;
                    re[k] = xr;
                    im[k] = xi;
                }
            }
        }
        if (a.n_params > 0) {
            // block reduction of the partial sums (FP64), one atomic per parameter
            for (int i = 0; i < a.n_params; ++i) {
                double v = (double)acc[i];
                for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
                if ((tid & 31) == 0) red[tid >> 5] = v;
                __syncthreads();
                if (tid == 0) {
                    double tsum = 0;
                    for (int w_ = 0; w_ < kThreads / 32; ++w_) tsum += red[w_];
                    atomicAdd(a.grad_params + i, tsum * a.inv_L);
                }
                __syncthreads();
            }
        }
        if (a.want_grad) {
            if constexpr (R2 == 1) {
                fft_reg<R1, +1>(re, im);
                if (act) {
#pragma unroll
                    for (int q = 0; q < R1; ++q) st_s(base + (long long)q * a.elem_stride, mk<T>(re[q], im[q]), pk);
                }
            } else {
                team_fft<R2, R1, +1, T>(re, im, t, xb, a.tw, SyncBlock());
                if (act && t < R2) {
#pragma unroll
                    for (int q = 0; q < R1; ++q) st_s(base + (long long)(t + R2 * q) * a.elem_stride, mk<T>(re[q], im[q]), pk);
                }
            }
        }
    } else {  // LM_CONV
        const uint64_t pin = pol_stream();
        if (act && t < TO::lanes) {
            const T sc = (T)*sh_scale;
            const long long coff = (long long)o * a.N * a.cp + kx;
            // all loads of one coefficient array first, then the products
            for (int i = 0; i < a.k; ++i) {
                const c2<T>* Cb = a.C[i] + b * a.c_pstride + coff;
                c2<T> cv[TO::regs];
#pragma unroll
                for (int k = 0; k < TO::regs; ++k) cv[k] = ld_in(Cb + (long long)TO::idx(t, k) * a.cp, pin);
#pragma unroll
                for (int k = 0; k < TO::regs; ++k) {
                    const T r = re[k] * cv[k].x - im[k] * cv[k].y;
                    im[k] = re[k] * cv[k].y + im[k] * cv[k].x;
                    re[k] = r;
                }
            }
#pragma unroll
            for (int k = 0; k < TO::regs; ++k) {
                const int ky = TO::idx(t, k);
                const bool neg = a.wsign && (a.k & 1) && ((kx + ky) & 1);   // W^k
                re[k] = neg ? -re[k] * sc : re[k] * sc;
                im[k] = neg ? -im[k] * sc : im[k] * sc;
            }
        }
        if constexpr (R2 == 1) {
            fft_reg<R1, +1>(re, im);       // one lane holds the whole line
            if (act) {
#pragma unroll
                for (int q = 0; q < R1; ++q) st_s(base + (long long)q * a.elem_stride, mk<T>(re[q], im[q]), pk);
            }
        } else {
            // the transposed factorisation maps lane t back to x[t + R2 n]
            team_fft<R2, R1, +1, T>(re, im, t, xb, a.tw, SyncBlock());
            if (act && t < R2) {
#pragma unroll
                for (int q = 0; q < R1; ++q) st_s(base + (long long)(t + R2 * q) * a.elem_stride, mk<T>(re[q], im[q]), pk);
            }
        }
    }
}

// ---------------------------------------------------------------------------
// One-unit-per-block kernels
// ---------------------------------------------------------------------------
template <typename T, int N, int M>
__global__ void __launch_bounds__(kThreads) k_fwd_xt(XArgs<T> a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ double red[kThreads / 32];
    const int b = blockIdx.y;
    unit_fwd_xt<T, N, M>(a, a.f + b * a.g_pstride, a.s + b * a.s_pstride, blockIdx.x,
                         a.abs_sum ? a.abs_sum + b : nullptr, smem_raw, red);
}

template <typename T, int N, int M>
__global__ void __launch_bounds__(kThreads) k_inv_tx(XArgs<T> a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int b = blockIdx.y;
    unit_inv_tx<T, N, M>(a, a.s + b * a.s_pstride, a.out + b * a.g_pstride, blockIdx.x, smem_raw);
}

// FP32 line kernels are held to 85 registers so that three blocks share an SM.
template <typename T, int L, int MODE>
__global__ void __launch_bounds__(kThreads, sizeof(T) == 4 ? 3 : 1) k_lines(LArgs<T> a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ double sh_scale;
    __shared__ double red[kThreads / 32];
    const int b = blockIdx.y;
    unit_lines<T, L, MODE>(a, a.s + b * a.s_pstride, b, blockIdx.x, smem_raw, &sh_scale,
                           a.s2 ? a.s2 + b * a.s_pstride : nullptr, red);
}

// ---------------------------------------------------------------------------
// Radial kernel family for differentiation: Gaussian of width sigma in x, y
// (normalised over R^2, periodised over the lattice, images |n| <= 2) times
// 2 pi times a wrapped normal of width sigma_t centred at nu (|m| <= 4), on
// Omega_L; plus the derivatives in sigma and sigma_t.  The 1-D factors are
// computed in FP64 (tables: gx, dgx [N], gt, dgt [M]), then multiplied out.
// ---------------------------------------------------------------------------
static __global__ void k_gauss_tables(double* tab, int N, int M, double sigma, double sigma_t, double nu,
                                      double x0) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const double PI = 3.14159265358979323846;
    if (i < N) {
        const double d = x0 + (double)i / N;                // x_i (x0 = -1/2 on Omega_L, 0 at origin zero)
        double g = 0, dg = 0;
        for (int n = -2; n <= 2; ++n) {
            const double u2 = (d + n) * (d + n);
            const double e = exp(-u2 / (2 * sigma * sigma));
            g += e;
            dg += e * (-1.0 / (sigma * sigma) + u2 / (sigma * sigma * sigma * sigma));
        }
        tab[i] = g / (sqrt(2 * PI) * sigma);
        tab[N + i] = dg / sqrt(2 * PI);
    } else if (i < N + M) {
        const int l = i - N;
        double v = 2 * PI * l / M - nu + PI;
        v = v - 2 * PI * floor(v / (2 * PI)) - PI;          // [-pi, pi)
        double t = 0, dt = 0;
        for (int m = -4; m <= 4; ++m) {
            const double v2 = (v + 2 * PI * m) * (v + 2 * PI * m);
            const double e = exp(-v2 / (2 * sigma_t * sigma_t));
            t += e;
            dt += e * (-1.0 / (sigma_t * sigma_t) + v2 / (sigma_t * sigma_t * sigma_t * sigma_t));
        }
        tab[2 * N + l] = t * sqrt(2 * PI) / sigma_t;
        tab[2 * N + M + l] = dt * sqrt(2 * PI);
    }
}

// Separable chain tables: for problem b with k_b kernels (sigma, sigma_t, nu)
// from params[b][j][3], the 1-D factor spectra of each kernel (FP64 samples,
// FP64 direct DFT divided by the length) multiplied over the chain:
//   tx[kx] (kx <= N/2), ty[ky] (ky < N), tt[kt] (kt < M),
// with W^(k_b - 1) = (-1)^((kx + ky)(k_b - 1)) folded into tx and ty, so that
// the convolution applies W once.  One block per problem.
template <typename T>
__global__ void k_sep_tables(const double* params, const int* kcount, int kmax, int N, int M,
                             c2<T>* tab, long long tab_pstride, double x0, int wfold) {
    const int b = blockIdx.x;
    const int k = kcount[b];
    const double PI = 3.14159265358979323846;
    extern __shared__ double sh[];                 // g[N], gt[M], e^{-2 pi i n/N} [N], e^{-2 pi i n/M} [M]
    double* g = sh;
    double* gt = sh + N;
    double2* twN = reinterpret_cast<double2*>(sh + N + M);
    double2* twM = twN + N;
    for (int i = threadIdx.x; i < N + M; i += blockDim.x) {
        double sn, cn;
        if (i < N) { sincospi(2.0 * i / N, &sn, &cn); twN[i] = make_double2(cn, -sn); }
        else { sincospi(2.0 * (i - N) / M, &sn, &cn); twM[i - N] = make_double2(cn, -sn); }
    }
    c2<T>* tb = tab + b * tab_pstride;
    const int H = N / 2 + 1;
    const int tot = H + N + M;
    // accumulate in registers: each thread owns entries e = tid, tid + blockDim, ...
    double ar[8], ai[8];
    for (int q = 0; q < 8; ++q) { ar[q] = 1.0; ai[q] = 0.0; }
    for (int j = 0; j < k; ++j) {
        const double sigma = params[((size_t)b * kmax + j) * 3 + 0];
        const double sigma_t = params[((size_t)b * kmax + j) * 3 + 1];
        const double nu = params[((size_t)b * kmax + j) * 3 + 2];
        __syncthreads();
        for (int i = threadIdx.x; i < N + M; i += blockDim.x) {
            if (i < N) {
                const double d = x0 + (double)i / N;
                double acc = 0;
                for (int n = -2; n <= 2; ++n) acc += exp(-(d + n) * (d + n) / (2 * sigma * sigma));
                g[i] = acc / (sqrt(2 * PI) * sigma);
            } else {
                const int l = i - N;
                double v = 2 * PI * l / M - nu + PI;
                v = v - 2 * PI * floor(v / (2 * PI)) - PI;
                double acc = 0;
                for (int m = -4; m <= 4; ++m) acc += exp(-(v + 2 * PI * m) * (v + 2 * PI * m) / (2 * sigma_t * sigma_t));
                gt[l] = acc * sqrt(2 * PI) / sigma_t;
            }
        }
        __syncthreads();
        for (int q = 0; q < 8; ++q) {
            const int e = threadIdx.x + q * blockDim.x;
            if (e >= tot) break;
            const double* src;
            const double2* tw;
            int L, kk;
            if (e < H) { src = g; L = N; kk = e; tw = twN; }
            else if (e < H + N) { src = g; L = N; kk = e - H; tw = twN; }
            else { src = gt; L = M; kk = e - H - N; tw = twM; }
            double sr = 0, si = 0;
            int idx = 0;                                   // (kk * n) mod L
            for (int n = 0; n < L; ++n) {
                sr += src[n] * tw[idx].x;
                si += src[n] * tw[idx].y;
                idx += kk;
                if (idx >= L) idx -= L;
            }
            sr /= L;
            si /= L;
            const double r = ar[q] * sr - ai[q] * si;
            ai[q] = ar[q] * si + ai[q] * sr;
            ar[q] = r;
        }
    }
    for (int q = 0; q < 8; ++q) {
        const int e = threadIdx.x + q * blockDim.x;
        if (e >= tot) break;
        double sgn = 1.0;
        if (wfold && e < H + N && ((k - 1) & 1)) {
            const int kk = e < H ? e : e - H;
            if (kk & 1) sgn = -1.0;
        }
        tb[e] = mk<T>((T)(ar[q] * sgn), (T)(ai[q] * sgn));
    }
}

template <typename T>
__global__ void k_gauss_fill(const double* tab, int N, int M, T* P, T* dPs, T* dPt) {
    const long long total = (long long)M * N * N;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(e % N), j = (int)((e / N) % N), l = (int)(e / ((long long)N * N));
        const double gx = tab[i], gy = tab[j], dgx = tab[N + i], dgy = tab[N + j];
        const double gt = tab[2 * N + l], dgt = tab[2 * N + M + l];
        if (P) P[e] = (T)(gt * gy * gx);
        if (dPs) dPs[e] = (T)(gt * (dgy * gx + gy * dgx));
        if (dPt) dPt[e] = (T)(dgt * gy * gx);
    }
}

// ---------------------------------------------------------------------------
// Mass renormalisation (FP64).  k_mass_sum adds each problem's samples into
// sums[b] (grid: (blocks, B)); k_mass_fix adds (target - sum(out)) / n to
// every sample of problem b, target = sum(f) C_1[0] ... C_k[0] exp(sum ls).
// Adding one constant to samples already on the T grid would round the same
// way within a binade, so the total would drift by up to n/2 ulp; each lane
// therefore carries its rounding residual along its kMassRun samples (error
// feedback), which leaves at most half an ulp per lane.
// ---------------------------------------------------------------------------
constexpr int kMassRun = 256;   // samples per lane in k_mass_fix
template <typename T>
__global__ void k_mass_sum(const T* x, long long n, double* sums) {
    __shared__ double red[32];
    const T* xb = x + (size_t)blockIdx.y * n;
    double acc = 0.0;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x)
        acc += (double)xb[e];
    for (int off = 16; off > 0; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
        atomicAdd(sums + blockIdx.y, t);
    }
}

template <typename T>
struct MassArgs {
    const c2<T>* C[32];
    const double* ls[32];
    int k, B;
    long long c_pstride, ls_pstride;
};

template <typename T>
__global__ void k_mass_fix(T* out, long long n, const double* sums, MassArgs<T> a) {
    const int b = blockIdx.y;
    double prod = 1.0, lsum = 0.0;
    for (int i = 0; i < a.k; ++i) {
        prod *= (double)a.C[i][(size_t)b * a.c_pstride].x;
        if (a.ls[i] != nullptr) lsum += a.ls[i][(size_t)b * a.ls_pstride];
    }
    const double delta = (sums[b] * prod * exp(lsum) - sums[a.B + b]) / (double)n;
    T* ob = out + (size_t)b * n;
    // warp w of the grid row owns the segment [w * 32 * kMassRun, +32 * kMassRun)
    const long long w = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const long long seg = w * 32 * kMassRun + (threadIdx.x & 31);
    double carry = 0.0;
    for (int i = 0; i < kMassRun; ++i) {
        const long long e = seg + 32LL * i;
        if (e >= n) break;
        const double v = (double)ob[e] + delta + carry;
        const T r = (T)v;
        carry = v - (double)r;
        ob[e] = r;
    }
}

// ---------------------------------------------------------------------------
// Analytic inputs of the paper's experiments, sampled in FP64 on the plan's
// grid: the Gaussian on SE(2) (Section 5, Eq. fbS; Eq. gbS0 is the case
// beta = (0, R_nu), Sigma = sigma^2 I) and the 3D deformed Gaussian (Eq. fHsnu).
// Both sum the left translates by lattice vectors |n1|, |n2| <= images, which
// makes them functions on Z^2\SE(2).
// ---------------------------------------------------------------------------
struct GaussSE2Args {
    int Nx, Ny, M, images;   // grid x_i = x0 + i / Nx, y_j = x0 + j / Ny, theta_l = 2 pi l / M
    double x0;          // first grid coordinate: -1/2 on Omega_L, 0 at x_i = i/N
    double b1, b2;      // translation of the mean beta
    double nu_turns;    // rotation of the mean beta, in turns (nu / 2 pi)
    double q11, q12, q13, q22, q23, q33;  // Sigma^-1 (symmetric)
};

// f(g) = exp(-w^T Sigma^-1 w / 2) with w = log(beta^-1 o g)^v = (v, phi).
// beta^-1 o (x, R_theta) = (R_-nu (x - b), R_(theta - nu)); phi is the angle of
// R_(theta - nu) in (-pi, pi].  V(phi) = int_0^1 exp(t phi J) dt equals
// (2 sin(phi/2) / phi) R_(phi/2), so v = V(phi)^-1 R_-nu (x - b)
// = ((phi/2) / sin(phi/2)) R_-(nu + phi/2) (x - b).
template <typename T>
__global__ void k_se2_gauss_fill(GaussSE2Args a, T* P) {
    const long long total = (long long)a.M * a.Ny * a.Nx;
    const double inv_nx = 1.0 / a.Nx, inv_ny = 1.0 / a.Ny;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(e % a.Nx), j = (int)((e / a.Nx) % a.Ny), l = (int)(e / ((long long)a.Nx * a.Ny));
        // angle of theta_l - nu in turns, reduced to (-1/2, 1/2]
        double t = (double)l / a.M - a.nu_turns;
        t -= rint(t);
        if (t == -0.5) t = 0.5;
        const double PI = 3.14159265358979323846;
        const double phi = 2.0 * PI * t;
        const double ah = (t == 0.0) ? 1.0 : (PI * t) / sinpi(t);  // (phi/2)/sin(phi/2)
        double sr, cr;
        sincospi(2.0 * a.nu_turns + t, &sr, &cr);  // rotation by nu + phi/2
        const double px = a.x0 + i * inv_nx - a.b1, py = a.x0 + j * inv_ny - a.b2;
        double acc = 0.0;
        for (int n2 = -a.images; n2 <= a.images; ++n2) {
            for (int n1 = -a.images; n1 <= a.images; ++n1) {
                const double d1 = px + n1, d2 = py + n2;
                const double v1 = ah * (cr * d1 + sr * d2);
                const double v2 = ah * (-sr * d1 + cr * d2);
                const double q = a.q11 * v1 * v1 + a.q22 * v2 * v2 + a.q33 * phi * phi +
                                 2.0 * (a.q12 * v1 * v2 + a.q13 * v1 * phi + a.q23 * v2 * phi);
                acc += exp(-0.5 * q);
            }
        }
        P[e] = (T)acc;
    }
}

// Host-side preparation of GaussSE2Args from beta = {b1, b2, nu} and a
// row-major 3x3 Sigma: checks symmetry and positive definiteness (leading
// minors) and inverts by the adjugate.  Returns nullptr or why it refused.
inline const char* make_gauss_args(const double* beta, const double* Sigma, GaussSE2Args* a) {
    for (int i = 0; i < 3; ++i)
        if (!(fabs(beta[i]) < 1e300)) return "beta is not finite";
    double S[9], amax = 0.0;
    for (int i = 0; i < 9; ++i) {
        S[i] = Sigma[i];
        if (!(fabs(S[i]) < 1e300)) return "Sigma is not finite";
        amax = fabs(S[i]) > amax ? fabs(S[i]) : amax;
    }
    for (int r = 0; r < 3; ++r)
        for (int c = r + 1; c < 3; ++c)
            if (fabs(S[3 * r + c] - S[3 * c + r]) > 1e-12 * amax) return "Sigma is not symmetric";
    const double m1 = S[0], m2 = S[0] * S[4] - S[1] * S[3];
    const double c00 = S[4] * S[8] - S[5] * S[7], c01 = -(S[3] * S[8] - S[5] * S[6]), c02 = S[3] * S[7] - S[4] * S[6];
    const double det = S[0] * c00 + S[1] * c01 + S[2] * c02;
    if (!(m1 > 0) || !(m2 > 0) || !(det > 0)) return "Sigma is not positive definite";
    const double c11 = S[0] * S[8] - S[2] * S[6], c12 = -(S[0] * S[7] - S[1] * S[6]);
    const double c22 = S[0] * S[4] - S[1] * S[3];
    a->b1 = beta[0];
    a->b2 = beta[1];
    a->nu_turns = beta[2] / (2.0 * 3.14159265358979323846);
    a->q11 = c00 / det;
    a->q12 = c01 / det;
    a->q13 = c02 / det;
    a->q22 = c11 / det;
    a->q23 = c12 / det;
    a->q33 = c22 / det;
    return nullptr;
}

struct DeformedArgs {
    int Nx, Ny, M, images;
    double x0, nu, s;
    double h11, h12, h22;  // symmetric part of H
};

// Host-side preparation of DeformedArgs from a row-major 2x2 H (its
// symmetric part must be positive definite), nu and s > 0.
inline const char* make_deformed_args(const double* H, double nu, double s_theta, DeformedArgs* a) {
    if (!(s_theta > 0) || !(s_theta < 1e300) || !(fabs(nu) < 1e300)) return "s must be finite and > 0, nu finite";
    const double h11 = H[0], h12 = 0.5 * (H[1] + H[2]), h22 = H[3];
    if (!(h11 > 0) || !(h11 * h22 - h12 * h12 > 0) || !(h22 < 1e300) || !(fabs(h12) < 1e300))
        return "H is not positive definite";
    a->nu = nu;
    a->s = s_theta;
    a->h11 = h11;
    a->h12 = h12;
    a->h22 = h22;
    return nullptr;
}

// f(x, R_theta) = exp(-x^T H x) exp(-(theta - nu)^2 / s), theta = 2 pi l / M
// taken as it is (no wrapping), as Eq. fHsnu is printed.
template <typename T>
__global__ void k_deformed_fill(DeformedArgs a, T* P) {
    const long long total = (long long)a.M * a.Ny * a.Nx;
    const double inv_nx = 1.0 / a.Nx, inv_ny = 1.0 / a.Ny;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(e % a.Nx), j = (int)((e / a.Nx) % a.Ny), l = (int)(e / ((long long)a.Nx * a.Ny));
        const double PI = 3.14159265358979323846;
        const double dt = 2.0 * PI * l / a.M - a.nu;
        const double ang = exp(-dt * dt / a.s);
        const double px = a.x0 + i * inv_nx, py = a.x0 + j * inv_ny;
        double acc = 0.0;
        for (int n2 = -a.images; n2 <= a.images; ++n2) {
            for (int n1 = -a.images; n1 <= a.images; ++n1) {
                const double u1 = px + n1, u2 = py + n2;
                acc += exp(-(a.h11 * u1 * u1 + 2.0 * a.h12 * u1 * u2 + a.h22 * u2 * u2));
            }
        }
        P[e] = (T)(ang * acc);
    }
}

// ---------------------------------------------------------------------------
// Split path: x only (forward real FFT of packed theta-row pairs), runtime M.
// grid = (N rows y, ceil(M/2 / TEAMS), problems)
// ---------------------------------------------------------------------------
template <typename T, int N>
__global__ void __launch_bounds__(kThreads) k_fwd_x(XArgs<T> a) {
    constexpr int R1 = Fac<N>::R1, R2 = Fac<N>::R2, TS = team_size<N>(), RM = reg_count<N>();
    constexpr int TEAMS = kThreads / TS, XS = xbuf_elems<N>();
    using TO = TeamOut<R1, R2>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    c2<T>* XB = reinterpret_cast<c2<T>*>(smem_raw);
    __shared__ double red[kThreads / 32];
    const int j = blockIdx.x, b = blockIdx.z, tid = threadIdx.x;
    const int team = tid / TS, lane = tid % TS;
    const int p = blockIdx.y * TEAMS + team;
    const bool act = p < a.M / 2;
    c2<T>* xb = XB + team * XS;
    const T* fb = a.f + b * a.g_pstride + (size_t)j * N;
    const uint64_t pin = pol_stream(), pk = pol_keep();
    T re[RM], im[RM];
    T abs_acc = 0;
#pragma unroll
    for (int i = 0; i < RM; ++i) { re[i] = 0; im[i] = 0; }
    if (act && lane < R2) {
        const T* r0 = fb + (size_t)(2 * p) * N * N;
        const T* r1 = r0 + (size_t)N * N;
#pragma unroll
        for (int q = 0; q < R1; ++q) {
            re[q] = ld_in(r0 + lane + R2 * q, pin);
            im[q] = ld_in(r1 + lane + R2 * q, pin);
            abs_acc += fabs(re[q]) + fabs(im[q]);
        }
    }
    team_fft<R1, R2, -1, T>(re, im, lane, xb, a.twN, SyncWarp());
    if (lane < TO::lanes) {
#pragma unroll
        for (int k = 0; k < TO::regs; ++k) xb[TO::idx(lane, k)] = mk<T>(re[k], im[k]);
    }
    __syncwarp();
    if (act && lane < TO::lanes) {
        c2<T>* s0 = a.s + b * a.s_pstride + ((size_t)(2 * p) * N + j) * a.tp;
        c2<T>* s1 = s0 + (size_t)N * a.tp;
#pragma unroll
        for (int k2 = 0; k2 < TO::regs; ++k2) {
            const int kk = TO::idx(lane, k2);
            if (kk <= N / 2) {
                const c2<T> zm = xb[(N - kk) & (N - 1)];
                const T zr = re[k2], zi = im[k2];
                st_s(s0 + kk, mk<T>((zr + zm.x) * (T)0.5, (zi - zm.y) * (T)0.5), pk);
                st_s(s1 + kk, mk<T>((zi + zm.y) * (T)0.5, (zm.x - zr) * (T)0.5), pk);
            }
        }
    }
    if (a.abs_sum != nullptr) {
        double v = (double)abs_acc;
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if ((tid & 31) == 0) red[tid >> 5] = v;
        __syncthreads();
        if (tid == 0) {
            double t = 0;
            for (int w = 0; w < kThreads / 32; ++w) t += red[w];
            atomicAdd(a.abs_sum + b, t);
        }
    }
}

template <typename T, int N>
__global__ void __launch_bounds__(kThreads) k_inv_x(XArgs<T> a) {
    constexpr int R1 = Fac<N>::R1, R2 = Fac<N>::R2, TS = team_size<N>(), RM = reg_count<N>();
    constexpr int TEAMS = kThreads / TS, XS = xbuf_elems<N>();
    using TO = TeamOut<R1, R2>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    c2<T>* XB = reinterpret_cast<c2<T>*>(smem_raw);
    const int j = blockIdx.x, b = blockIdx.z, tid = threadIdx.x;
    const int team = tid / TS, lane = tid % TS;
    const int p = blockIdx.y * TEAMS + team;
    const bool act = p < a.M / 2;
    c2<T>* xb = XB + team * XS;
    const uint64_t pk = pol_keep(), po = pol_stream();
    T re[RM], im[RM];
#pragma unroll
    for (int i = 0; i < RM; ++i) { re[i] = 0; im[i] = 0; }
    if (act && lane < R2) {
        const c2<T>* s0 = a.s + b * a.s_pstride + ((size_t)(2 * p) * N + j) * a.tp;
        const c2<T>* s1 = s0 + (size_t)N * a.tp;
#pragma unroll
        for (int q = 0; q < R1; ++q) {
            const int kk = lane + R2 * q;
            c2<T> A, B;
            if (kk <= N / 2) {
                A = ld_s(s0 + kk, pk);
                B = ld_s(s1 + kk, pk);
                if (kk == 0 || kk == N / 2) { A.y = 0; B.y = 0; }
            } else {
                A = ld_s(s0 + N - kk, pk);
                B = ld_s(s1 + N - kk, pk);
                A.y = -A.y;
                B.y = -B.y;
            }
            re[q] = A.x - B.y;
            im[q] = A.y + B.x;
        }
    }
    team_fft<R1, R2, +1, T>(re, im, lane, xb, a.twN, SyncWarp());
    if (act && lane < TO::lanes) {
        T* o0 = a.out + b * a.g_pstride + ((size_t)(2 * p) * N + j) * N;
        T* o1 = o0 + (size_t)N * N;
#pragma unroll
        for (int k = 0; k < TO::regs; ++k) {
            st_out(o0 + TO::idx(lane, k), re[k], po);
            st_out(o1 + TO::idx(lane, k), im[k], po);
        }
    }
}

// ---------------------------------------------------------------------------
// Persistent convolution kernel: all units of all B problems of one call.
// Work list in rounds r = 0 .. B+2: round r holds A(r), then C(r-3), then
// B(r-1) (for the problems that exist), so a unit's inputs were produced
// about a round earlier.  Problem p uses scratch slot p % D (D = 4).
// Dependencies (waited on by the unit's thread 0, bounded):
//   B(p) needs all nA units A(p); C(p) needs all nB units B(p);
//   A(p), p >= D, needs all nC units C(p - D) (its slot is then free).
// Units are taken in list order from an atomic counter and every unit only
// waits on units earlier in the list, which were taken by running blocks, so
// the waits end.  A wait longer than `spin_limit` polls sets err = 1; then
// every block stops taking units and the kernel returns.
// Thread 0 fetches the next list index and that unit's dependency counter
// one unit ahead, so their latency overlaps the current unit's work.
// ---------------------------------------------------------------------------
template <typename T>
struct PArgs {
    XArgs<T> x;
    LArgs<T> l;
    int B;                     // problems in this launch
    int D;                     // scratch slots
    int nA, nB, nC;            // units per stage per problem
    unsigned* work;            // [1] next unit
    unsigned* cnt;             // [3 * B] completed units per (stage, problem)
    int* err;                  // device error word (0 = ok), sticky until read by the host
    long long spin_limit;      // polls before a wait gives up
    unsigned dep_extra;        // added to the A->B wait target; nonzero only to test the timeout path
};

__device__ __forceinline__ unsigned ld_acquire(const unsigned* p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ unsigned ld_relaxed(const unsigned* p) {
    unsigned v;
    asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// Map a work-list index to (stage 0=A,1=B,2=C, problem, unit); false if past the end.
__device__ __forceinline__ bool decode_unit(unsigned g, int B, int nA, int nB, int nC,
                                            int& stage, int& p, int& u) {
    long long rem = g;
    const long long full = (long long)nA + nB + nC;
    for (int r = 0; r < B + 3; ++r) {
        if (r >= 3 && r <= B - 1) {            // full rounds r .. B-1: skip whole ones
            const long long nfull = (long long)B - r;
            long long skip = rem / full;
            if (skip > nfull - 1) skip = nfull - 1;
            r += (int)skip;
            rem -= skip * full;
        }
        const bool ha = r < B, hc = r >= 3 && r <= B + 2, hb = r >= 1 && r <= B;
        if (ha) { if (rem < nA) { stage = 0; p = r; u = (int)rem; return true; } rem -= nA; }
        if (hc) { if (rem < nC) { stage = 2; p = r - 3; u = (int)rem; return true; } rem -= nC; }
        if (hb) { if (rem < nB) { stage = 1; p = r - 1; u = (int)rem; return true; } rem -= nB; }
    }
    return false;
}

// Dependency of a unit: counter and target (dep = nullptr: none).
template <typename T>
__device__ __forceinline__ const unsigned* unit_dep(const PArgs<T>& a, int stage, int p, unsigned& target) {
    if (stage == 1) { target = (unsigned)a.nA + a.dep_extra; return a.cnt + p; }
    if (stage == 2) { target = (unsigned)a.nB; return a.cnt + a.B + p; }
    if (p >= a.D) { target = (unsigned)a.nC; return a.cnt + 2 * a.B + (p - a.D); }
    return nullptr;
}

__device__ __forceinline__ void prefetch_l2(const void* p) {
    asm volatile("prefetch.global.L2 [%0];" :: "l"(p));
}

// Pull the HBM-resident inputs of a unit towards L2 ahead of its turn: the
// f rows of a unit A, the first coefficient tile of a unit B (units C read
// scratch, which is already in L2).
template <typename T, int N, int M>
__device__ __forceinline__ void prefetch_unit(const PArgs<T>& a, int stage, int p, int u) {
    const int tid = threadIdx.x;
    if (stage == 0) {
        const char* fb = reinterpret_cast<const char*>(a.x.f + p * a.x.g_pstride + (size_t)u * N);
        constexpr int LPR = (N * (int)sizeof(T) + 127) / 128;       // 128-byte lines per row
        for (int e = tid; e < M * LPR; e += kThreads) {
            const int r = e / LPR, c = e - r * LPR;
            prefetch_l2(fb + (size_t)r * N * N * sizeof(T) + c * 128);
        }
    } else if (stage == 1 && a.l.C[0] != nullptr) {
        constexpr int LINES = kThreads / team_size<N>();
        const long long line = (long long)u * LINES;
        const long long NR = (long long)a.l.n_outer * a.l.nk;
        if (line < NR) {
            const int o = (int)(line / a.l.nk), kx = (int)(line - (long long)o * a.l.nk);
            const char* cb = reinterpret_cast<const char*>(a.l.C[0] + p * a.l.c_pstride + (long long)o * a.l.N * a.l.cp + kx);
            for (int ky = tid; ky < N; ky += kThreads) prefetch_l2(cb + (size_t)ky * a.l.cp * sizeof(c2<T>));
        }
    }
}

template <typename T, int N, int M, int BMODE>
__global__ void __launch_bounds__(kThreads) k_conv_persist(PArgs<T> a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ double red[kThreads / 32];
    __shared__ double sh_scale;
    __shared__ int sh_unit[6];
    const int tid = threadIdx.x;
    // thread-0 pipeline state: the current unit, its early dependency read,
    // and the list index of the next unit (atomic in flight)
    int cs = -1, cp = 0, cu = 0;
    unsigned cv = 0, g_next = 0;
    if (tid == 0) {
        const unsigned g0 = atomicAdd(a.work, 1u);
        g_next = atomicAdd(a.work, 1u);
        if (decode_unit(g0, a.B, a.nA, a.nB, a.nC, cs, cp, cu)) {
            unsigned tg;
            const unsigned* d = unit_dep(a, cs, cp, tg);
            cv = d ? ld_relaxed(d) : 0u;
        } else {
            cs = -1;
        }
    }
    for (;;) {
        int ns = -1, np = 0, nu = 0;
        unsigned nv = 0;
        if (tid == 0) {
            int stage = cs;
            if (stage >= 0 && *(volatile int*)a.err != 0) stage = -1;
            if (stage >= 0) {
                unsigned target = 0;
                const unsigned* dep = unit_dep(a, cs, cp, target);
                if (dep != nullptr) {
                    if (cv >= target) {
                        __threadfence();        // the early relaxed read, upgraded to acquire
                    } else {
                        long long it = 0;
                        while (ld_acquire(dep) < target) {
                            if (++it > a.spin_limit || *(volatile int*)a.err != 0) {
                                atomicCAS(a.err, 0, 1);
                                stage = -1;
                                break;
                            }
                            __nanosleep(64);
                        }
                    }
                }
            }
            sh_unit[0] = stage;
            sh_unit[1] = cp;
            sh_unit[2] = cu;
            if (stage >= 0) {
                // look one unit ahead
                if (decode_unit(g_next, a.B, a.nA, a.nB, a.nC, ns, np, nu)) {
                    g_next = atomicAdd(a.work, 1u);
                    unsigned tg;
                    const unsigned* d = unit_dep(a, ns, np, tg);
                    nv = d ? ld_relaxed(d) : 0u;
                } else {
                    ns = -1;
                }
            }
            sh_unit[3] = ns;
            sh_unit[4] = np;
            sh_unit[5] = nu;
        }
        __syncthreads();
        const int stage = sh_unit[0], p = sh_unit[1], u = sh_unit[2];
        const int pst = sh_unit[3], pp = sh_unit[4], pu = sh_unit[5];
        __syncthreads();     // everyone has read sh_unit before it is rewritten
        if (stage < 0) break;
        if (pst >= 0) prefetch_unit<T, N, M>(a, pst, pp, pu);
        c2<T>* sprob = a.x.s + (size_t)(p % a.D) * a.x.s_pstride;
        if (stage == 0) {
            unit_fwd_xt<T, N, M>(a.x, a.x.f + p * a.x.g_pstride, sprob, u, nullptr, smem_raw, red);
        } else if (stage == 1) {
            unit_lines<T, N, BMODE>(a.l, sprob, p, u, smem_raw, &sh_scale);
        } else {
            unit_inv_tx<T, N, M>(a.x, sprob, a.x.out + p * a.x.g_pstride, u, smem_raw);
        }
        __syncthreads();
        if (tid == 0) {
            __threadfence();
            atomicAdd(a.cnt + stage * a.B + p, 1u);
            cs = ns; cp = np; cu = nu; cv = nv;
        }
    }
}

}  // namespace se2
