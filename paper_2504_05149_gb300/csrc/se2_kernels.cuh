// CUDA kernels of the SE(2) convolution path (arXiv 2504.05149, Algorithms
// 3, 4 and 6 at output grid N = L).  All grids are [theta][y][x], x fastest.
//
// Pass structure for one problem (|L| = N*N*M points):
//   fwd_xt  (per y row):   real FFT along x of the M rows (two rows packed
//                          as one complex line), then the angular DFT of the
//                          N/2+1 columns in shared memory  -> scratch S
//   lines<CONV> (per (theta-bin, x-bin) line): FFT along y, multiply by
//                          W^k . C_1 ... C_k / |L| (Eq. MatSqKfgG), inverse
//                          FFT along y, in place in S
//   inv_tx  (per y row):   inverse angular DFT, then complex-to-real inverse
//                          FFT along x of row pairs -> out
// When the [M][N/2+1] slab of one y row does not fit in shared memory the
// x and theta steps run as separate passes (fwd_x, lines<FWD> along theta,
// ..., lines<INV> along theta, inv_x).
#pragma once
#include "se2_fft.cuh"

namespace se2 {

constexpr int kThreads = 256;
constexpr int kMaxChain = 32;

enum LineMode { LM_FWD = 0, LM_INV = 1, LM_CONV = 2, LM_COEF = 3 };

// Slab pitch (complex elements) for the [M][N/2+1] slab: = 2 mod 16 so that
// the 8-lane angular teams of one warp hit distinct bank pairs.
template <int N> __host__ __device__ constexpr int slab_pitch() {
    constexpr int H = N / 2 + 1;
    return H + ((2 - H % 16) + 16) % 16;
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
};

// ---------------------------------------------------------------------------
// Forward x (real, packed row pairs) and theta, one y row per block.
// ---------------------------------------------------------------------------
template <typename T, int N, int M>
__global__ void __launch_bounds__(kThreads) k_fwd_xt(XArgs<T> a) {
    constexpr int H = N / 2 + 1, SP = slab_pitch<N>();
    constexpr int R1 = Fac<N>::R1, R2 = Fac<N>::R2, TS = team_size<N>(), RM = reg_count<N>();
    constexpr int TEAMS = kThreads / TS, XS = xbuf_elems<N>();
    using TO = TeamOut<R1, R2>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    c2<T>* S = reinterpret_cast<c2<T>*>(smem_raw);
    c2<T>* XB = S + M * SP;
    __shared__ double red[kThreads / 32];

    const int j = blockIdx.x, b = blockIdx.y, tid = threadIdx.x;
    const T* fb = a.f + b * a.g_pstride + (size_t)j * N;
    const int team = tid / TS, lane = tid % TS;
    c2<T>* xb = XB + team * XS;
    T abs_acc = 0;

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
                re[q] = __ldg(r0 + lane + R2 * q);
                im[q] = __ldg(r1 + lane + R2 * q);
                abs_acc += fabs(re[q]) + fabs(im[q]);
            }
        }
        team_fft<R1, R2, -1, T>(re, im, lane, xb, a.twN, SyncWarp());
        // lane s < R1 holds Z[s + R1 k]; publish Z linearly to split the pair
        if (lane < TO::lanes) {
#pragma unroll
            for (int k = 0; k < TO::regs; ++k) xb[TO::idx(lane, k)] = mk<T>(re[k], im[k]);
        }
        __syncwarp();
        if (act && lane < TO::lanes) {
#pragma unroll
            for (int k2 = 0; k2 < TO::regs; ++k2) {
                const int kk = TO::idx(lane, k2);
                if (kk <= N / 2) {
                    const c2<T> zm = xb[(N - kk) & (N - 1)];
                    const T zr = re[k2], zi = im[k2];
                    // X0 = (Z[k] + conj Z[N-k]) / 2, X1 = (Z[k] - conj Z[N-k]) / (2i)
                    S[(2 * p) * SP + kk] = mk<T>((zr + zm.x) * (T)0.5, (zi - zm.y) * (T)0.5);
                    S[(2 * p + 1) * SP + kk] = mk<T>((zi + zm.y) * (T)0.5, (zm.x - zr) * (T)0.5);
                }
            }
        }
        __syncwarp();
    }
    if (a.abs_sum != nullptr) {
        double v = (double)abs_acc;
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if ((tid & 31) == 0) red[tid >> 5] = v;
    }
    __syncthreads();
    if (a.abs_sum != nullptr && tid == 0) {
        double v = 0;
        for (int w = 0; w < kThreads / 32; ++w) v += red[w];
        atomicAdd(a.abs_sum + b, v);
    }
    // angular DFT of the H columns
    {
        constexpr int TSM = team_size<M>(), TEAMSM = kThreads / TSM;
        const int tm = tid / TSM, lm = tid % TSM;
        for (int c0 = 0; c0 < H; c0 += TEAMSM) {
            const int c = c0 + tm;
            const bool act = c < H;
            column_fft<M, -1, T>(S + (act ? c : 0), SP, lm, act, a.twM, SyncWarp());
        }
    }
    __syncthreads();
    c2<T>* sb = a.s + b * a.s_pstride + (size_t)j * a.tp;
    for (int e = tid; e < M * H; e += kThreads) {
        const int r = e / H, k = e - r * H;
        sb[(size_t)r * N * a.tp + k] = S[r * SP + k];
    }
}

// ---------------------------------------------------------------------------
// Inverse theta then complex-to-real x, one y row per block.
// ---------------------------------------------------------------------------
template <typename T, int N, int M>
__global__ void __launch_bounds__(kThreads) k_inv_tx(XArgs<T> a) {
    constexpr int H = N / 2 + 1, SP = slab_pitch<N>();
    constexpr int R1 = Fac<N>::R1, R2 = Fac<N>::R2, TS = team_size<N>(), RM = reg_count<N>();
    constexpr int TEAMS = kThreads / TS, XS = xbuf_elems<N>();
    using TO = TeamOut<R1, R2>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    c2<T>* S = reinterpret_cast<c2<T>*>(smem_raw);
    c2<T>* XB = S + M * SP;

    const int j = blockIdx.x, b = blockIdx.y, tid = threadIdx.x;
    const c2<T>* sb = a.s + b * a.s_pstride + (size_t)j * a.tp;
    for (int e = tid; e < M * H; e += kThreads) {
        const int r = e / H, k = e - r * H;
        S[r * SP + k] = sb[(size_t)r * N * a.tp + k];
    }
    __syncthreads();
    {
        constexpr int TSM = team_size<M>(), TEAMSM = kThreads / TSM;
        const int tm = tid / TSM, lm = tid % TSM;
        for (int c0 = 0; c0 < H; c0 += TEAMSM) {
            const int c = c0 + tm;
            const bool act = c < H;
            column_fft<M, +1, T>(S + (act ? c : 0), SP, lm, act, a.twM, SyncWarp());
        }
    }
    __syncthreads();
    const int team = tid / TS, lane = tid % TS;
    c2<T>* xb = XB + team * XS;
    T* ob = a.out + b * a.g_pstride + (size_t)j * N;
    constexpr int NP = M / 2;
    for (int p0 = 0; p0 < NP; p0 += TEAMS) {
        const int p = p0 + team;
        const bool act = p < NP;
        T re[RM], im[RM];
#pragma unroll
        for (int i = 0; i < RM; ++i) { re[i] = 0; im[i] = 0; }
        if (act && lane < R2) {
            const c2<T>* s0 = S + (2 * p) * SP;
            const c2<T>* s1 = s0 + SP;
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
        team_fft<R1, R2, +1, T>(re, im, lane, xb, a.twN, SyncWarp());
        if (act && lane < TO::lanes) {
            T* o0 = ob + (size_t)(2 * p) * N * N;
            T* o1 = o0 + (size_t)N * N;
#pragma unroll
            for (int k = 0; k < TO::regs; ++k) {
                o0[TO::idx(lane, k)] = re[k];
                o1[TO::idx(lane, k)] = im[k];
            }
        }
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
    T re[RM], im[RM];
    T abs_acc = 0;
#pragma unroll
    for (int i = 0; i < RM; ++i) { re[i] = 0; im[i] = 0; }
    if (act && lane < R2) {
        const T* r0 = fb + (size_t)(2 * p) * N * N;
        const T* r1 = r0 + (size_t)N * N;
#pragma unroll
        for (int q = 0; q < R1; ++q) {
            re[q] = __ldg(r0 + lane + R2 * q);
            im[q] = __ldg(r1 + lane + R2 * q);
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
                s0[kk] = mk<T>((zr + zm.x) * (T)0.5, (zi - zm.y) * (T)0.5);
                s1[kk] = mk<T>((zi + zm.y) * (T)0.5, (zm.x - zr) * (T)0.5);
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
                A = s0[kk];
                B = s1[kk];
                if (kk == 0 || kk == N / 2) { A.y = 0; B.y = 0; }
            } else {
                A = s0[N - kk];
                B = s1[N - kk];
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
            o0[TO::idx(lane, k)] = re[k];
            o1[TO::idx(lane, k)] = im[k];
        }
    }
}

// ---------------------------------------------------------------------------
// Line pass: FFTs of length L along one axis of the scratch spectrum, for
// all lines (outer index o, x bin kx), kx fastest for coalescing.
//   LM_FWD / LM_INV: forward / unscaled inverse FFT in place
//   LM_CONV (y axis): forward, multiply by W^k C_1..C_k exp(sum ls) / |L|,
//                     inverse, in place
//   LM_COEF (y axis): forward, scale by 1 / (|L| s_b), write the external
//                     coefficient layout
// grid = (ceil(lines / LINES), problems)
// ---------------------------------------------------------------------------
template <typename T, int L, int MODE>
__global__ void __launch_bounds__(kThreads) k_lines(LArgs<T> a) {
    constexpr int R1 = Fac<L>::R1, R2 = Fac<L>::R2, TS = team_size<L>(), RM = reg_count<L>();
    constexpr int LINES = kThreads / TS;
    constexpr int XS = (Fac<L>::R1 * (Fac<L>::R2 + 1)) | 1;   // odd stride: lines in distinct banks
    extern __shared__ __align__(16) unsigned char smem_raw[];
    c2<T>* XB = reinterpret_cast<c2<T>*>(smem_raw);
    __shared__ double sh_scale;

    const int b = blockIdx.y, tid = threadIdx.x;
    const int c = tid % LINES, t = tid / LINES;
    const long long NR = (long long)a.n_outer * a.nk;
    const long long total = NR + a.n_outer;
    const long long line = (long long)blockIdx.x * LINES + c;
    const bool act = line < total;
    int o, kx;
    if (line < NR) { o = (int)(line / a.nk); kx = (int)(line - (long long)o * a.nk); }
    else { o = act ? (int)(line - NR) : 0; kx = a.nk; }
    c2<T>* base = a.s + b * a.s_pstride + o * a.outer_stride + kx;
    c2<T>* xb = XB + c * XS;

    if constexpr (MODE == LM_CONV || MODE == LM_COEF) {
        if (tid == 0) {
            double sc = a.inv_L;
            if constexpr (MODE == LM_CONV) {
                double lsum = 0;
                for (int i = 0; i < a.k; ++i)
                    if (a.ls[i] != nullptr) lsum += a.ls[i][b * a.ls_pstride];
                sc *= exp(lsum);
            } else {
                if (a.abs_sum != nullptr) {
                    const double s = a.abs_sum[b] * a.inv_L;   // mean |P|
                    double lg = 0;
                    if (s > 0) { sc /= s; lg = log(s); }
                    if (blockIdx.x == 0 && a.log_scale != nullptr) a.log_scale[a.problem0 + b] = lg;
                }
            }
            sh_scale = sc;
        }
        __syncthreads();
    }

    T re[RM], im[RM];
#pragma unroll
    for (int i = 0; i < RM; ++i) { re[i] = 0; im[i] = 0; }
    if (act && t < R2) {
#pragma unroll
        for (int q = 0; q < R1; ++q) {
            const c2<T> v = base[(long long)(t + R2 * q) * a.elem_stride];
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
    using TO = TeamOut<R1, R2>;
    if constexpr (MODE == LM_FWD || MODE == LM_INV) {
        if (act && t < TO::lanes) {
#pragma unroll
            for (int k = 0; k < TO::regs; ++k) base[(long long)TO::idx(t, k) * a.elem_stride] = mk<T>(re[k], im[k]);
        }
    } else if constexpr (MODE == LM_COEF) {
        if (act && t < TO::lanes) {
            const T sc = (T)sh_scale;
            c2<T>* cb = a.cout + b * a.cout_pstride + (long long)o * a.N * a.cp + kx;
#pragma unroll
            for (int k = 0; k < TO::regs; ++k) cb[(long long)TO::idx(t, k) * a.cp] = mk<T>(re[k] * sc, im[k] * sc);
        }
    } else {  // LM_CONV
        if (act && t < TO::lanes) {
            const T sc = (T)sh_scale;
            const long long coff = (long long)o * a.N * a.cp + kx;
#pragma unroll
            for (int k = 0; k < TO::regs; ++k) {
                const int ky = TO::idx(t, k);
                T xr = re[k] * sc, xi = im[k] * sc;
                for (int i = 0; i < a.k; ++i) {
                    const c2<T> cv = a.C[i][b * a.c_pstride + coff + (long long)ky * a.cp];
                    const T r = xr * cv.x - xi * cv.y;
                    xi = xr * cv.y + xi * cv.x;
                    xr = r;
                }
                if ((a.k & 1) && ((kx + ky) & 1)) { xr = -xr; xi = -xi; }   // W^k
                re[k] = xr;
                im[k] = xi;
            }
        }
        if constexpr (R2 == 1) {
            fft_reg<R1, +1>(re, im);       // one lane holds the whole line
            if (act) {
#pragma unroll
                for (int q = 0; q < R1; ++q) base[(long long)q * a.elem_stride] = mk<T>(re[q], im[q]);
            }
        } else {
            // the transposed factorisation maps lane t back to x[t + R2 n]
            team_fft<R2, R1, +1, T>(re, im, t, xb, a.tw, SyncBlock());
            if (act && t < R2) {
#pragma unroll
                for (int q = 0; q < R1; ++q) base[(long long)(t + R2 * q) * a.elem_stride] = mk<T>(re[q], im[q]);
            }
        }
    }
}

}  // namespace se2
