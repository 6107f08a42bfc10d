// FP32 fast path of the three-kernel convolution (units A, B, C of the
// convolution of Algorithm 3 / the chain of Eq. MatSqKfgG at output grid
// N = L).  Every FFT here runs on two independent lines at once, one in each
// half of a float2 register ("paired"), so that each butterfly, twiddle and
// coefficient product is one sm_100+ f32x2 instruction (add/mul/fma.f32x2)
// acting on both lines.
//
// Scratch layout of this path ("paired spectrum"), Q = N/4, per (theta bin
// m, y or ky) row of Q + 1 float4 entries:
//   entry u < Q : (Re X[u], Re X[u+Q], Im X[u], Im X[u+Q])
//   entry Q     : (Re X[N/2], 0, Im X[N/2], 0)
// where X[kx] is the spectrum at x frequency kx.  The x-frequency pairs
// (u, u+Q) are the two lines that the y pass transforms together.  Spectra in
// this scratch are twice the true ones (the factor 1/2 of the real-FFT split
// is folded into the product's scale).
//
// Shared-memory slab (units A and C): M rows of odd pitch P >= Q + 1 entries,
// row r at r * P + (r >> 3); with P odd the strided row accesses of the
// angular teams fall in distinct 16-byte bank groups.  The x FFTs exchange
// through their own four slab rows (no separate buffer), so 4 P also covers a
// padded exchange of R1 (R2 + 1) entries.
//
// Global accesses use the cache-hint intrinsics (scratch: .cg, through L2
// only; inputs, coefficients and outputs: .cs, streamed) so that the compiler
// folds address offsets and forms 128-bit register quads itself.
#pragma once
#include "se2_kernels.cuh"

namespace se2 {

// ---------------------------------------------------------------------------
// Paired FP32 arithmetic
// ---------------------------------------------------------------------------
__device__ __forceinline__ float2 pf(float a, float b) { return make_float2(a, b); }
__device__ __forceinline__ float2 bc2(float a) { return make_float2(a, a); }
__device__ __forceinline__ float2 pneg(float2 a) { return make_float2(-a.x, -a.y); }
__device__ __forceinline__ float2 padd(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 psub(float2 a, float2 b) { return __fadd2_rn(a, pneg(b)); }
__device__ __forceinline__ float2 pmul(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 pfma(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }

// Two in-register DFTs of R <= 32 points (radix-2 decimation in frequency,
// natural order in and out), one per half of re/im.  A rotation by +-i is a
// swap of the real and imaginary registers with a sign that the following
// butterfly absorbs: in decimation in frequency that rotated element is always
// the second operand of the next butterfly, so nr/ni never outlive one stage.
template <int R, int DIR>
__device__ __forceinline__ void fft2_reg(float2* re, float2* im) {
    if constexpr (R > 1) {
        bool nr[R], ni[R];
#pragma unroll
        for (int i = 0; i < R; ++i) { nr[i] = false; ni[i] = false; }
#pragma unroll
        for (int half = R / 2; half >= 1; half >>= 1) {
#pragma unroll
            for (int base = 0; base < R; base += 2 * half) {
#pragma unroll
                for (int j = 0; j < half; ++j) {
                    const int a = base + j, b = a + half;
                    const float2 ar = re[a], ai = im[a], br = re[b], bi = im[b];
                    float2 sr, si, dr, di;
                    if (!nr[b]) { sr = padd(ar, br); dr = psub(ar, br); } else { sr = psub(ar, br); dr = padd(ar, br); }
                    if (!ni[b]) { si = padd(ai, bi); di = psub(ai, bi); } else { si = psub(ai, bi); di = padd(ai, bi); }
                    re[a] = sr;
                    im[a] = si;
                    nr[b] = false;
                    ni[b] = false;
                    const int q = j * (16 / half);          // rotation e^{DIR i pi q / 16}
                    if (q == 0) {
                        re[b] = dr;
                        im[b] = di;
                    } else if (q == 8) {                    // (r, i) * DIR i = (-DIR i, DIR r)
                        re[b] = di;
                        nr[b] = (DIR == 1);
                        im[b] = dr;
                        ni[b] = (DIR == -1);
                    } else {
                        const float c = (float)cpi16(q), s = (float)(DIR * spi16(q));
                        re[b] = pfma(dr, bc2(c), pmul(di, bc2(-s)));
                        im[b] = pfma(dr, bc2(s), pmul(di, bc2(c)));
                    }
                }
            }
        }
        float2 tr[R], ti[R];
#pragma unroll
        for (int i = 0; i < R; ++i) { tr[i] = re[i]; ti[i] = im[i]; }
#pragma unroll
        for (int i = 0; i < R; ++i) { re[i] = tr[bitrev<R>(i)]; im[i] = ti[bitrev<R>(i)]; }
    }
}

// (re + i im) *= w for DIR = -1 and *= conj(w) for DIR = +1, w = (wr, wi) the
// forward twiddle e^{-2 pi i n / L} broadcast to both halves.
template <int DIR>
__device__ __forceinline__ void ptw(float2& re, float2& im, float2 wr, float2 wi) {
    if constexpr (DIR < 0) {
        const float2 r = pfma(re, wr, pneg(pmul(im, wi)));
        im = pfma(re, wi, pmul(im, wr));
        re = r;
    } else {
        const float2 r = pfma(re, wr, pmul(im, wi));
        im = pfma(im, wr, pneg(pmul(re, wi)));
        re = r;
    }
}

// Exchange slot of step-A output k1 of lane t: rows of R2 + 1 slots, so that
// both the row writes and the column reads of 8 lanes (one 128-bit access
// phase) hit distinct bank groups, with compile-time offsets from a per-lane
// base.
template <int R1, int R2>
__device__ __forceinline__ constexpr int xslot(int k1, int t) { return k1 * (R2 + 1) + t; }
template <int R1, int R2> __host__ __device__ constexpr int xslots() { return R1 * (R2 + 1); }

// Paired team FFT of length L = R1 * R2 (two lines, one per register half).
//  in : lane t < R2 holds x[t + R2 j], j < R1
//  out: lane s < R1 holds X[s + R1 k], k < R2
// xb: the team's R1 * R2 float4 exchange slots; tw4: this factorisation's
// step-A twiddles, tw4[k1 * R2 + t] = e^{-2 pi i t k1 / L} as (wr, wr, wi, wi)
// (consecutive lanes read consecutive entries).  Lanes with act = false only
// synchronise.
template <int R1, int R2, int DIR, typename Sync>
__device__ __forceinline__ void team_fft2(float2* re, float2* im, int lane, bool act, float4* xb,
                                          const float4* tw4, Sync sync) {
    if constexpr (R2 == 1) {
        fft2_reg<R1, DIR>(re, im);
    } else {
        if (lane < R2) {
            fft2_reg<R1, DIR>(re, im);
#pragma unroll
            for (int k1 = 1; k1 < R1; ++k1) {
                const float4 w = tw4[k1 * R2 + lane];
                ptw<DIR>(re[k1], im[k1], pf(w.x, w.y), pf(w.z, w.w));
            }
            if (act) {
#pragma unroll
                for (int k1 = 0; k1 < R1; ++k1)
                    xb[xslot<R1, R2>(k1, lane)] = make_float4(re[k1].x, re[k1].y, im[k1].x, im[k1].y);
            }
        }
        sync();
        if (lane < R1) {
            if (act) {
#pragma unroll
                for (int t = 0; t < R2; ++t) {
                    const float4 v = xb[xslot<R1, R2>(lane, t)];
                    re[t] = pf(v.x, v.y);
                    im[t] = pf(v.z, v.w);
                }
            }
            fft2_reg<R2, DIR>(re, im);
        }
        sync();
    }
}

__host__ __device__ __forceinline__ constexpr int frow(int r, int P) { return r * P + (r >> 3); }
// Slab pitch: odd, >= N/4 + 1, and four rows hold the padded x exchange and
// the N + 1 linear slots of the real-FFT split.
template <int N> __host__ __device__ constexpr int fpitch() {
    constexpr int x = xslots<Fac<N>::R1, Fac<N>::R2>() > N + 1 ? xslots<Fac<N>::R1, Fac<N>::R2>() : N + 1;
    constexpr int p = (x + 3) / 4 > N / 4 + 1 ? (x + 3) / 4 : N / 4 + 1;
    return p | 1;
}
template <int N, int M> __host__ __device__ constexpr int fslab4() { return M * fpitch<N>() + (M >> 3) + 1; }
// Scratch row pitch (float4) of the paired layout: the plan's pitch of
// round_up(N/2 + 1, 16) complex elements.
template <int N> __host__ __device__ constexpr int ftp4() { return ((N / 2 + 1 + 15) / 16 * 16) / 2; }
// Lane part of frow(lane + R j) for lane < R, R a power of two: the row
// shift (lane + R j) >> 3 equals (lane >> 3) + ((R j) >> 3), so frow(lane + R j)
// = frow_lane(lane) + frow(R j) with the second term a compile-time constant.
__device__ __forceinline__ int frow_lane(int lane, int P) { return lane * P + (lane >> 3); }

// Paired in-place FFT of slab column pair u (rows r at frow(r, P) + u) by a
// team of team_size<L>() lanes; (wr, wi): this lane's step-A twiddles
// e^{-2 pi i lane k / L} as broadcast pairs.
template <int L, int P, int DIR, typename Sync>
__device__ __forceinline__ void column_fft2(float4* S, int u, int lane, bool act, const float2* wr,
                                            const float2* wi, Sync sync) {
    constexpr int R1 = Fac<L>::R1, R2 = Fac<L>::R2, RM = reg_count<L>();
    float2 re[RM], im[RM];
    if constexpr (R2 == 1) {
        if (act) {
#pragma unroll
            for (int r = 0; r < L; ++r) { const float4 v = S[frow(r, P) + u]; re[r] = pf(v.x, v.y); im[r] = pf(v.z, v.w); }
            fft2_reg<L, DIR>(re, im);
#pragma unroll
            for (int r = 0; r < L; ++r) S[frow(r, P) + u] = make_float4(re[r].x, re[r].y, im[r].x, im[r].y);
        }
    } else {
        // rows lane + R2 j, k1 + R1 lane and lane + R1 t: (a + b) >> 3 splits
        // into a >> 3 plus b >> 3 because R1, R2 are powers of two and lane < R
        float4* Su = S + u;
        float4* SA = Su + frow_lane(lane, P);                              // rows lane + R * j
        float4* SS = Su + lane * (R1 * P) + ((R1 * lane) >> 3);            // rows k1 + R1 lane
        if (act && lane < R2) {
#pragma unroll
            for (int j = 0; j < R1; ++j) {
                const float4 v = SA[R2 * j * P + ((R2 * j) >> 3)];
                re[j] = pf(v.x, v.y);
                im[j] = pf(v.z, v.w);
            }
            fft2_reg<R1, DIR>(re, im);
#pragma unroll
            for (int k1 = 1; k1 < R1; ++k1) ptw<DIR>(re[k1], im[k1], wr[k1], wi[k1]);
        }
        sync();     // every step-A load is done before any step-A store
        if (act && lane < R2) {
#pragma unroll
            for (int k1 = 0; k1 < R1; ++k1)
                SS[k1 * P + (k1 >> 3)] = make_float4(re[k1].x, re[k1].y, im[k1].x, im[k1].y);
        }
        sync();
        if (act && lane < R1) {
#pragma unroll
            for (int t = 0; t < R2; ++t) {
                const float4 v = SA[R1 * t * P + ((R1 * t) >> 3)];
                re[t] = pf(v.x, v.y);
                im[t] = pf(v.z, v.w);
            }
            fft2_reg<R2, DIR>(re, im);
#pragma unroll
            for (int k = 0; k < R2; ++k) SA[R1 * k * P + ((R1 * k) >> 3)] = make_float4(re[k].x, re[k].y, im[k].x, im[k].y);
        }
    }
}

struct FArgs {
    const float* f;
    float* out;
    float4* s;                   // paired scratch of the first problem of the launch
    long long s_pstride;         // float4 entries per problem (rows of ftp4<N>() entries)
    const float2* twN;           // forward twiddles of length N and M
    const float2* twM;
    int k;                       // kernels in the chain
    const float2* C[kMaxChain];  // coefficient arrays [B][M][N][N/2+1] (or shared)
    const double* ls[kMaxChain]; // per-problem log scales (or null)
    long long c_pstride, ls_pstride;
    double inv_L;
    // separable coefficients instead of C (kf_lines<.., true>): per problem
    // tables tx[N/2+1], ty[N], tt[M] with C = tx[kx] ty[ky] tt[m], W^(k-1)
    // folded in (the multiply applies W once)
    const float2* sep;
    long long sep_pstride;
    // adjoint y pass (kf_lines<.., FL_ADJ>): s2 = the y-transformed paired
    // spectrum of f; dC = derivative spectra; partials accumulate (FP64
    // atomics) into grad_params; want_grad: also the correlation spectrum
    const float4* s2;
    int n_params;
    const float2* dC[kMaxParams];
    double* grad_params;
    int want_grad;
    int wsign;                   // 1: apply W (grids on Omega_L); 0: grids at x_i = i/N
    int ymirror;                 // 1: C(ky) = C(N - ky) is promised; rows ky > N/2 are not read
    // running-product y pass (kf_lines<.., FL_ACC>): s holds the full spectrum
    // product R_{p-1} in ky order; R_p = R_{p-1} C_p is stored back and the
    // inverse y FFT of W^p R_p exp(sum_{i<=p} ls_i) / |L| goes to sout
    float4* sout;
    int p;                       // 1-based index of C_p in C[] (chain step)
    int* err;                    // plan's device error word (bounded waits of the bulk-copy units)
    int discard;                 // 1: unit C drops the scratch rows it has read from L2 (no write-back)
};

// y-pass modes: the convolution / chain product, the separable product, the
// forward y FFT only (in place), the adjoint (correlation + parameter partials)
enum FastLineMode { FL_CONV = 0, FL_SEP = 1, FL_FWD = 2, FL_ADJ = 3, FL_ACC = 4 };

// Step-A twiddle table of the team FFT of length L = R1 * R2 (layout of
// team_fft2) from the forward table src of length L.
template <int R1, int R2>
__device__ __forceinline__ void fill_tw4(float4* tw, const float2* src) {
    for (int n = threadIdx.x; n < R1 * R2; n += blockDim.x) {
        const int k1 = n / R2, t = n - k1 * R2;
        const float2 w = src[k1 * t];
        tw[n] = make_float4(w.x, w.x, w.y, w.y);
    }
}
__device__ __forceinline__ void copy_tw(float2* dst, const float2* src, int L) {
    for (int n = threadIdx.x; n < L; n += blockDim.x) dst[n] = src[n];
}

// This lane's step-A twiddles of the length-M angular team FFT, broadcast.
template <int M>
__device__ __forceinline__ void angular_twiddles(const float2* twM, int lm, float2* wr, float2* wi) {
    constexpr int R1 = Fac<M>::R1, R2 = Fac<M>::R2;
    const int l = lm < R2 ? lm : 0;
#pragma unroll
    for (int k = 0; k < R1; ++k) {
        const float2 w = twM[(l * k) % M];
        wr[k] = bc2(w.x);
        wi[k] = bc2(w.y);
    }
}

// y rows per block of units A and C.  One y row gives M / 4 x jobs (four
// theta rows each) and N / 4 angular columns; at small M that leaves most
// teams idle, so a block takes YR consecutive y rows, enough that every x
// team has a job (YR * M / 4 >= teams), and its slab holds YR * M rows.
template <int N, int M> __host__ __device__ constexpr int fast_yr() {
    constexpr int want = (kThreads / team_size<N>()) * 4 / M;
    return want < 1 ? 1 : (want > 8 ? 8 : want);
}

// ---------------------------------------------------------------------------
// Unit A: forward real x FFT of the M theta rows of y row j (rows 4q, 4q+1
// packed as one complex line, rows 4q+2, 4q+3 as the other half), the split
// into row spectra, then the paired angular FFT of the slab columns; the DC
// and Nyquist columns (both real along x) travel as one complex column.
// ---------------------------------------------------------------------------
// Unit A's body (se2_unit_a.inc), for the batch kernel: K = false, block
// bx_ of one problem whose grid f is fp and scratch slot sp.  With K = true
// (the kernel below) the block and problem come from the grid and the
// addresses from a, where they are used.
template <int N, int M, bool K>
__device__ __forceinline__ void fwd_xt_body(const FArgs& a, int bx_, int b_, const float* fp, float4* sp) {
#include "se2_unit_a.inc"
}

// The kernel expands the same body with K = true: its own parameter a, and
// block and problem from the grid (a function that takes a by reference
// measured 2% more instructions).
template <int N, int M>
__global__ void __launch_bounds__(kThreads, 2) kf_fwd_xt(FArgs a) {
    constexpr bool K = true;
    const int bx_ = 0, b_ = 0;
    const float* fp = nullptr;
    float4* sp = nullptr;
#include "se2_unit_a.inc"
}

// ---------------------------------------------------------------------------
// Unit B: for LINES pairs of (theta bin, x bins u, u + N/4) lines: paired FFT
// along y, multiply by W^k C_1 ... C_k exp(sum ls) / |L| (and the 1/2 of the
// split), inverse FFT along y, in place.
// ---------------------------------------------------------------------------
// Exchange entries per line pair of the y pass: both factorisations' padded
// slots, rounded to 1 (mod 8) so that 8 consecutive line pairs start in
// distinct bank groups.
template <int N> __host__ __device__ constexpr int fast_xs() {
    constexpr int a = xslots<Fac<N>::R1, Fac<N>::R2>(), b = xslots<Fac<N>::R2, Fac<N>::R1>();
    return ((a > b ? a : b) + 7) / 8 * 8 + 1;
}
// Threads of a unit-B block (its line pairs x team lanes); blocks per SM
// such that the SM holds as many threads as with units A and C.
constexpr int kLineThreads = 256;
template <int N> __host__ __device__ constexpr int fast_lines() { return kLineThreads / team_size<N>(); }

// Unit B's body (se2_unit_b.inc), for the batch kernel: K = false, block
// bx_ of problem b_ with scratch slot sp and separable tables tsep (FL_SEP).
template <int N, int M, int MODE, bool K>
__device__ __forceinline__ void lines_body(const FArgs& a, int bx_, int b_, float4* sp, const float2* tsep) {
#include "se2_unit_b.inc"
}

template <int N, int M, int MODE>
__global__ void __launch_bounds__(kLineThreads, 2 * kThreads / kLineThreads) kf_lines(FArgs a) {
    constexpr bool K = true;
    const int bx_ = 0, b_ = 0;
    float4* sp = nullptr;
    const float2* tsep = nullptr;
#include "se2_unit_b.inc"
}

// Unit C is the last reader of a y row's scratch rows (m, j): once the block
// holds them in shared memory they can be dropped from L2 without being
// written back (discard.global.L2; the slot is rewritten by a later unit A
// before it is read again), so that dead scratch costs no DRAM writes (opt-in,
// FArgs::discard).  Rows are ftp4<N>() float4 = a whole number of 128-byte
// lines, 128-byte aligned.
template <int N, int M>
__device__ __forceinline__ void discard_scratch_rows(const float4* row0) {
    constexpr int TP4 = ftp4<N>();
    constexpr int LPR = TP4 * 16 / 128;
    static_assert(TP4 * 16 % 128 == 0, "scratch rows are whole 128-byte lines");
    const char* base = reinterpret_cast<const char*>(row0);
    for (int i = threadIdx.x; i < M * LPR; i += blockDim.x) {
        const int r = i / LPR, l = i - (i / LPR) * LPR;
        asm volatile("discard.global.L2 [%0], 128;" :: "l"(base + ((size_t)r * N * TP4) * 16 + l * 128) : "memory");
    }
}

// ---------------------------------------------------------------------------
// Unit C: paired inverse angular FFT of the slab columns (DC and Nyquist
// columns recombined into one complex column first), then the inverse x FFTs
// of row pairs (4q, 4q+1) and (4q+2, 4q+3) as the two halves.
// ---------------------------------------------------------------------------
// Unit C's body (se2_unit_c.inc), for the batch kernel: K = false, block
// bx_ of one problem with scratch slot sp and grid out op.
template <int N, int M, bool K>
__device__ __forceinline__ void inv_tx_body(const FArgs& a, int bx_, int b_, const float4* sp, float* op) {
#include "se2_unit_c.inc"
}

template <int N, int M>
__global__ void __launch_bounds__(kThreads, 2) kf_inv_tx(FArgs a) {
    constexpr bool K = true;
    const int bx_ = 0, b_ = 0;
    const float4* sp = nullptr;
    float* op = nullptr;
#include "se2_unit_c.inc"
}

template <int N, int M> constexpr size_t fast_xt_smem() {
    return (size_t)(fslab4<N, fast_yr<N, M>() * M>() + N + M / 2) * sizeof(float4);
}
template <int N, int M> constexpr size_t fast_lines_smem() {
    return (size_t)(fast_lines<N>() * fast_xs<N>() + 2 * N) * sizeof(float4) + (size_t)(N / 2 + 1 + N + M) * sizeof(float2);
}

}  // namespace se2
