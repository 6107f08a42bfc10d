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
// Body of unit A for block bx of one problem: fp its grid f, sp its scratch
// rows (the kernel passes the problem's slot; the batch kernel a ring slot).
template <int N, int M>
__device__ __forceinline__ void fwd_xt_body(const FArgs& a, int bx, const float* fp, float4* sp, float4* fsm) {
    constexpr int YR = fast_yr<N, M>(), MR = YR * M;   // slab rows: YR y rows of M theta rows
    constexpr int Q = N / 4, P = fpitch<N>(), TP4 = ftp4<N>();
    constexpr int R1 = Fac<N>::R1, R2 = Fac<N>::R2, TS = team_size<N>(), RM = reg_count<N>();
    constexpr int TEAMS = kThreads / TS, JOBS = MR / 4, JY = M / 4;
    constexpr int QK = Q / R1;            // register distance between x bins u and u + Q
    constexpr int HK = N / (2 * R1);      // register of bin N/2 on lane 0
    constexpr size_t NN = (size_t)N * N;
    static_assert(Q % R1 == 0 && Q % R2 == 0, "pairing needs N/4 divisible by the radices");
    static_assert(M % 8 == 0 && MR <= kThreads && N % YR == 0, "slab of whole y rows");
    float4* S = fsm;
    float4* TW = fsm + fslab4<N, MR>();
    float2* TWM = reinterpret_cast<float2*>(TW + N);
    const int tid = threadIdx.x, j0 = bx * YR;
    const float* fb = fp + (size_t)j0 * N;
    const int team = tid / TS, lane = tid % TS;
    for (int q0 = 0; q0 < JOBS; q0 += TEAMS) {
        const int q = q0 + team;            // slab rows 4q .. 4q + 3: y row q / JY, theta rows 4 (q % JY) ..
        const bool act = q < JOBS;
        float2 re[RM], im[RM];
#pragma unroll
        for (int i = 0; i < RM; ++i) { re[i] = pf(0.f, 0.f); im[i] = pf(0.f, 0.f); }
        if (act && lane < R2) {
            const float* r0 = fb + (size_t)(q / JY) * N + (size_t)(4 * (q % JY)) * NN;
#pragma unroll
            for (int jj = 0; jj < R1; ++jj) {
                const int x = lane + R2 * jj;
                re[jj] = pf(__ldcs(r0 + x), __ldcs(r0 + 2 * NN + x));
                im[jj] = pf(__ldcs(r0 + NN + x), __ldcs(r0 + 3 * NN + x));
            }
        }
        if (q0 == 0) {   // the table fills overlap the first loads
            fill_tw4<R1, R2>(TW, a.twN);
            copy_tw(TWM, a.twM, M);
            __syncthreads();
        }
        float4* xb = S + frow(4 * (act ? q : 0), P);
        team_fft2<R1, R2, -1>(re, im, lane, act, xb, TW, SyncWarp());
        // lane s < R1 holds Z[s + R1 k], k < R2 (half a: rows 4q/4q+1, b: 4q+2/4q+3)
        if (act && lane < R1) {
#pragma unroll
            for (int k = 0; k < R2; ++k) xb[lane + R1 * k] = make_float4(re[k].x, re[k].y, im[k].x, im[k].y);
            if (lane == 0) xb[N] = make_float4(re[0].x, re[0].y, im[0].x, im[0].y);   // Z[N] = Z[0]
        }
        __syncwarp();
        float4 zm[HK + 1];
        if (act && lane < R1) {
            const float4* zb = xb + (N - lane);
#pragma unroll
            for (int k = 0; k < HK; ++k) zm[k] = zb[-R1 * k];
            zm[HK] = lane == 0 ? xb[N / 2] : make_float4(0.f, 0.f, 0.f, 0.f);
        }
        __syncwarp();   // every read of Z is done before the rows take the spectra
        if (act && lane < R1) {
            // X0 = Z + conj Z[N-k], X1 = -i (Z - conj Z[N-k]): twice the spectra of the two rows
            float4* row0 = S + frow(4 * q, P);
            const float2 n0 = padd(re[HK], pf(zm[HK].x, zm[HK].y));   // Re X0[N/2] (lane 0)
            const float2 n1 = padd(im[HK], pf(zm[HK].z, zm[HK].w));   // Re X1[N/2]
#pragma unroll
            for (int k = 0; k < QK; ++k) {
                const int u = lane + R1 * k, h = k + QK;
                const float2 lr = pf(zm[k].x, zm[k].y), li = pf(zm[k].z, zm[k].w);
                const float2 hr = pf(zm[h].x, zm[h].y), hi = pf(zm[h].z, zm[h].w);
                const float2 a0r = padd(re[k], lr), a0i = psub(im[k], li), a1r = padd(im[k], li), a1i = psub(lr, re[k]);
                const float2 b0r = padd(re[h], hr), b0i = psub(im[h], hi), b1r = padd(im[h], hi), b1i = psub(hr, re[h]);
                float4 e0 = make_float4(a0r.x, b0r.x, a0i.x, b0i.x);
                float4 e1 = make_float4(a1r.x, b1r.x, a1i.x, b1i.x);
                float4 e2 = make_float4(a0r.y, b0r.y, a0i.y, b0i.y);
                float4 e3 = make_float4(a1r.y, b1r.y, a1i.y, b1i.y);
                if (k == 0 && lane == 0) {   // X[0], X[N/2] are real: one complex DC entry
                    e0.z = n0.x;
                    e1.z = n1.x;
                    e2.z = n0.y;
                    e3.z = n1.y;
                }
                row0[u] = e0;
                row0[P + u] = e1;
                row0[2 * P + u] = e2;
                row0[3 * P + u] = e3;
            }
        }
    }
    __syncthreads();
    {
        constexpr int TSM = team_size<M>(), TEAMSM = kThreads / TSM;
        const int tm = tid / TSM, lm = tid % TSM;
        float2 wr[Fac<M>::R1], wi[Fac<M>::R1];
        angular_twiddles<M>(TWM, lm, wr, wi);
        for (int c0 = 0; c0 < YR * Q; c0 += TEAMSM) {
            const int c = c0 + tm;          // column u = c % Q of y row c / Q (M % 8 == 0: frow adds)
            const bool act = c < YR * Q;
            column_fft2<M, P, -1>(S + frow((act ? c / Q : 0) * M, P), act ? c % Q : 0, lm, act, wr, wi, SyncWarp());
        }
    }
    __syncthreads();
    // split the DC column's transform Y = F(X[.,0] + i X[.,N/2]) into the two
    // real columns' transforms: (Y + conj Y[-m]) / 2 and (Y - conj Y[-m]) / 2i
    float4 yv = make_float4(0.f, 0.f, 0.f, 0.f), ym = yv;
    if (tid < MR) {
        yv = S[frow(tid, P)];
        ym = S[frow((tid & ~(M - 1)) + ((M - tid) & (M - 1)), P)];
    }
    __syncthreads();
    if (tid < MR) {
        float4 e = yv;
        e.x = 0.5f * (yv.x + ym.x);
        e.z = 0.5f * (yv.z - ym.z);
        S[frow(tid, P)] = e;
        S[frow(tid, P) + Q] = make_float4(0.5f * (yv.z + ym.z), 0.f, 0.5f * (ym.x - yv.x), 0.f);
    }
    __syncthreads();
    {
        constexpr int E = Q + 1;
        float4* sb = sp + (size_t)j0 * TP4;
        for (int e = tid; e < MR * E; e += kThreads) {
            const int r = e / E, u = e - r * E;      // slab row r: theta row r % M of y row j0 + r / M
            __stcg(sb + (size_t)(r / M) * TP4 + (size_t)(r % M) * N * TP4 + u, S[frow(r, P) + u]);
        }
    }
}

template <int N, int M>
__global__ void __launch_bounds__(kThreads, 2) kf_fwd_xt(FArgs a) {
    extern __shared__ float4 fsm[];
    fwd_xt_body<N, M>(a, blockIdx.x, a.f + (size_t)blockIdx.y * N * N * M, a.s + (size_t)blockIdx.y * a.s_pstride, fsm);
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

// Body of unit B for block bx of problem b: sp its scratch, tsep its
// separable tables (FL_SEP).
template <int N, int M, int MODE>
__device__ __forceinline__ void lines_body(const FArgs& a, int bx, int b, float4* sp, const float2* tsep, float4* fsm) {
    constexpr bool SEP = MODE == FL_SEP;
    constexpr int Q = N / 4, P1 = Q + 1, CP = N / 2 + 1, TP4 = ftp4<N>();
    constexpr int TL = N / 2 + 1 + N + M;    // separable table length
    constexpr int R1 = Fac<N>::R1, R2 = Fac<N>::R2, RM = reg_count<N>();
    constexpr int LINES = fast_lines<N>(), XS = fast_xs<N>();
    static_assert(R1 % 2 == 0, "ky parity is the lane parity");
    float4* XB = fsm;
    float4* TWF = fsm + LINES * XS;     // forward (R1 x R2) and inverse (R2 x R1) tables
    float4* TWI = TWF + N;
    float2* TSEP = reinterpret_cast<float2*>(TWI + N);   // this problem's separable tables
    __shared__ double sh_scale;
    __shared__ double red[kLineThreads / 32];
    const int tid = threadIdx.x;
    const int c = tid % LINES, t = tid / LINES;
    const int pl = bx * LINES + c;
    const bool act = pl < M * P1;
    const int o = act ? pl / P1 : 0, u = act ? pl - (pl / P1) * P1 : 0;
    float4* base = sp + (size_t)o * N * TP4 + u + (size_t)t * TP4;
    float4* xb = XB + c * XS;
    float2 re[RM], im[RM];
#pragma unroll
    for (int i = 0; i < RM; ++i) { re[i] = pf(0.f, 0.f); im[i] = pf(0.f, 0.f); }
    if constexpr (MODE == FL_ACC) {
        if (act && t < R1) {
#pragma unroll
            for (int k = 0; k < R2; ++k) {
                const float4 v = __ldcg(base + (size_t)(R1 * k) * TP4);
                re[k] = pf(v.x, v.y);
                im[k] = pf(v.z, v.w);
            }
        }
    } else if (act && t < R2) {
#pragma unroll
        for (int jj = 0; jj < R1; ++jj) {
            const float4 v = __ldcg(base + (size_t)(R2 * jj) * TP4);
            re[jj] = pf(v.x, v.y);
            im[jj] = pf(v.z, v.w);
        }
    }
    // table fills and the scale overlap the loads
    fill_tw4<R1, R2>(TWF, a.twN);
    fill_tw4<R2, R1>(TWI, a.twN);
    if constexpr (SEP) {
        copy_tw(TSEP, tsep, TL);
        if (tid == 0) sh_scale = 0.5 * a.inv_L;
    } else if (tid == 0) {
        double lsum = 0;
        const int upto = MODE == FL_ACC ? a.p : a.k;
        for (int i = 0; i < upto; ++i)
            if (a.ls[i] != nullptr) lsum += a.ls[i][b * a.ls_pstride];
        sh_scale = 0.5 * a.inv_L * exp(lsum);
    }
    __syncthreads();
    if constexpr (MODE != FL_ACC) team_fft2<R1, R2, -1>(re, im, t, act, xb, TWF, SyncBlock());
    // lane s < R1 holds ky = s + R1 k, k < R2
    if constexpr (MODE == FL_FWD) {
        if (act && t < R1) {
#pragma unroll
            for (int k = 0; k < R2; ++k)
                __stcg(base + (size_t)(R1 * k) * TP4, make_float4(re[k].x, re[k].y, im[k].x, im[k].y));
        }
        return;
    }
    if constexpr (MODE == FL_ADJ) {
        // parameter partials sum_k m_k W Re(dC_i conj(G) F) over this lane's bins
        // (m_k = 1 at x bins 0 and N/2, 2 elsewhere; both spectra are doubled)
        float2 acc[kMaxParams];
#pragma unroll
        for (int i = 0; i < kMaxParams; ++i) acc[i] = pf(0.f, 0.f);
        if (a.n_params > 0 && act && t < R1) {
            const bool hasb = u < Q;
            const int kxa = hasb ? u : N / 2;
            const float sg = (a.wsign && ((u + t) & 1)) ? -1.f : 1.f;
            const float2 mw = pf(sg * ((u == 0 || u == Q) ? 1.f : 2.f), sg * 2.f);
            // F at this lane's bins, staged in the (now idle) exchange area
            const float4* fb2 = a.s2 + (size_t)b * a.s_pstride + (size_t)o * N * TP4 + u + (size_t)t * TP4;
#pragma unroll
            for (int k = 0; k < R2; ++k)
                asm volatile("cp.async.cg.shared.global [%0], [%1], 16;"
                             :: "r"((unsigned)__cvta_generic_to_shared(xb + t + R1 * k)), "l"(fb2 + (size_t)(R1 * k) * TP4)
                             : "memory");
            asm volatile("cp.async.commit_group;\ncp.async.wait_all;" ::: "memory");
            const size_t coff = (size_t)b * a.c_pstride + (size_t)o * N * CP + kxa + (size_t)t * CP;
#pragma unroll
            for (int i = 0; i < kMaxParams; ++i) {
                if (i < a.n_params) {
#pragma unroll
                    for (int h = 0; h < 4; ++h) {
                        constexpr int KH = R2 / 4;
                        float2 da[KH], dq[KH];
#pragma unroll
                        for (int kk = 0; kk < KH; ++kk) {
                            const float2* db = a.dC[i] + coff + (size_t)(R1 * (h * KH + kk)) * CP;
                            da[kk] = __ldcs(db);
                            dq[kk] = hasb ? __ldcs(db + Q) : pf(0.f, 0.f);
                        }
#pragma unroll
                        for (int kk = 0; kk < KH; ++kk) {
                            const int k = h * KH + kk;
                            const float4 v = xb[t + R1 * k];
                            const float2 fr = pf(v.x, v.y), fi = pf(v.z, v.w);
                            const float2 pr = pfma(re[k], fr, pmul(im[k], fi));      // conj(G) F
                            const float2 pi = pfma(re[k], fi, pneg(pmul(im[k], fr)));
                            const float2 vv = pfma(pf(da[kk].x, dq[kk].x), pr, pneg(pmul(pf(da[kk].y, dq[kk].y), pi)));
                            acc[i] = pfma(vv, mw, acc[i]);
                        }
                        asm volatile("" ::: "memory");   // bounds the loads in flight
                    }
                }
            }
        }
        __syncthreads();   // the exchange area is free again before the inverse FFT
#pragma unroll
        for (int i = 0; i < kMaxParams; ++i) {
            if (i < a.n_params) {   // uniform over the block
                double v = (double)acc[i].x + (double)acc[i].y;
                for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
                if ((tid & 31) == 0) red[tid >> 5] = v;
                __syncthreads();
                if (tid == 0) {
                    double tsum = 0;
                    for (int w = 0; w < kLineThreads / 32; ++w) tsum += red[w];
                    atomicAdd(a.grad_params + i, 0.25 * a.inv_L * tsum);
                }
                __syncthreads();
            }
        }
        if (!a.want_grad) return;
    }
    if (act && t < R1) {
        const bool hasb = u < Q;
        const int kxa = hasb ? u : N / 2;
        const float sc = (float)sh_scale;
        const int kpar = MODE == FL_ACC ? a.p : a.k;
        const bool neg = a.wsign && (SEP || (kpar & 1)) && ((u + t) & 1);   // W^k at (kx, ky), both halves alike
        const float2 s2 = bc2(neg ? -sc : sc);
        if constexpr (SEP) {
            // C = (tx[kx] tt[m]) ty[ky]: the x and theta factors once per lane
            const float2 ct = TSEP[N / 2 + 1 + N + o];
            const float2 xa = TSEP[kxa], xq = hasb ? TSEP[kxa + Q] : pf(0.f, 0.f);
            const float2 xr = pf(xa.x * ct.x - xa.y * ct.y, xq.x * ct.x - xq.y * ct.y);
            const float2 xi = pf(xa.x * ct.y + xa.y * ct.x, xq.x * ct.y + xq.y * ct.x);
#pragma unroll
            for (int k = 0; k < R2; ++k) {
                const float2 ty = TSEP[N / 2 + 1 + t + R1 * k];
                const float2 tyr = bc2(ty.x), tyi = bc2(ty.y);
                const float2 cr = pfma(xr, tyr, pneg(pmul(xi, tyi))), ci = pfma(xr, tyi, pmul(xi, tyr));
                const float2 r = pfma(re[k], cr, pneg(pmul(im[k], ci)));
                im[k] = pfma(re[k], ci, pmul(im[k], cr));
                re[k] = r;
            }
        }
        // coefficient loads in chunks of CK bins (the adjoint keeps fewer in flight)
        constexpr int CK = MODE == FL_ADJ ? R2 / 2 : R2;
        const int i0 = MODE == FL_ACC ? a.p - 1 : 0, i1 = SEP ? 0 : (MODE == FL_ACC ? a.p : a.k);
        const bool ym = a.ymirror != 0;
        for (int i = i0; i < i1; ++i) {
            const float2* cb = a.C[i] + (size_t)b * a.c_pstride + (size_t)o * N * CP + kxa;
#pragma unroll
            for (int k0 = 0; k0 < R2; k0 += CK) {
                float2 ca[CK], cq[CK];
#pragma unroll
                for (int kk = 0; kk < CK; ++kk) {
                    // row ky of this lane's bin, folded to N - ky for mirror-symmetric kernels
                    int row = t + R1 * (k0 + kk);
                    if (ym && row > N / 2) row = N - row;
                    ca[kk] = __ldcs(cb + (size_t)row * CP);
                    cq[kk] = hasb ? __ldcs(cb + (size_t)row * CP + Q) : pf(0.f, 0.f);
                }
#pragma unroll
                for (int kk = 0; kk < CK; ++kk) {
                    const int k = k0 + kk;
                    const float2 cr = pf(ca[kk].x, cq[kk].x);
                    // the adjoint multiplies by conj(C)
                    const float2 ci = MODE == FL_ADJ ? pf(-ca[kk].y, -cq[kk].y) : pf(ca[kk].y, cq[kk].y);
                    const float2 r = pfma(re[k], cr, pneg(pmul(im[k], ci)));
                    im[k] = pfma(re[k], ci, pmul(im[k], cr));
                    re[k] = r;
                }
                if (CK < R2) asm volatile("" ::: "memory");
            }
        }
        if constexpr (MODE == FL_ACC) {   // keep the running product R_p (unscaled, no W)
#pragma unroll
            for (int k = 0; k < R2; ++k)
                __stcg(base + (size_t)(R1 * k) * TP4, make_float4(re[k].x, re[k].y, im[k].x, im[k].y));
        }
#pragma unroll
        for (int k = 0; k < R2; ++k) {
            re[k] = pmul(re[k], s2);
            im[k] = pmul(im[k], s2);
        }
    }
    team_fft2<R2, R1, +1>(re, im, t, act, xb, TWI, SyncBlock());
    if (act && t < R2) {
        float4* dst = MODE == FL_ACC ? a.sout + (base - a.s) : base;
#pragma unroll
        for (int k = 0; k < R1; ++k)
            __stcg(dst + (size_t)(R2 * k) * TP4, make_float4(re[k].x, re[k].y, im[k].x, im[k].y));
    }
}

template <int N, int M, int MODE>
__global__ void __launch_bounds__(kLineThreads, 2 * kThreads / kLineThreads) kf_lines(FArgs a) {
    extern __shared__ float4 fsm[];
    lines_body<N, M, MODE>(a, blockIdx.x, blockIdx.y, a.s + (size_t)blockIdx.y * a.s_pstride,
                           MODE == FL_SEP ? a.sep + (size_t)blockIdx.y * a.sep_pstride : nullptr, fsm);
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
// Body of unit C for block bx of one problem: sp its scratch, op its grid out.
template <int N, int M>
__device__ __forceinline__ void inv_tx_body(const FArgs& a, int bx, const float4* sp, float* op, float4* fsm) {
    constexpr int YR = fast_yr<N, M>(), MR = YR * M;   // slab rows: YR y rows of M theta rows
    constexpr int Q = N / 4, P = fpitch<N>(), TP4 = ftp4<N>(), E = Q + 1;
    constexpr int R1 = Fac<N>::R1, R2 = Fac<N>::R2, TS = team_size<N>(), RM = reg_count<N>();
    constexpr int TEAMS = kThreads / TS, JOBS = MR / 4, JY = M / 4;
    constexpr int QJ = Q / R2, HJ = N / (2 * R2);
    constexpr size_t NN = (size_t)N * N;
    constexpr int LOADS = (MR * E + kThreads - 1) / kThreads;
    static_assert(M % 8 == 0 && MR <= kThreads && N % YR == 0, "slab of whole y rows");
    float4* S = fsm;
    float4* TW = fsm + fslab4<N, MR>();
    float2* TWM = reinterpret_cast<float2*>(TW + N);
    const int tid = threadIdx.x, j0 = bx * YR;
    {
        // batches of at most ~20 loads in flight per thread (registers)
        constexpr int CH = LOADS <= 20 ? LOADS : (LOADS + 1) / 2;
        const float4* sb = sp + (size_t)j0 * TP4;
        for (int i0 = 0; i0 < LOADS; i0 += CH) {
            float4 v[CH];
#pragma unroll
            for (int i = 0; i < CH; ++i) {
                const int e = tid + kThreads * (i0 + i);
                if (i0 + i < LOADS && e < MR * E) {
                    const int r = e / E, u = e - r * E;
                    v[i] = __ldcg(sb + (size_t)(r / M) * TP4 + (size_t)(r % M) * N * TP4 + u);
                }
            }
            if (i0 == 0) {   // the table fills overlap the loads
                fill_tw4<R1, R2>(TW, a.twN);
                copy_tw(TWM, a.twM, M);
            }
#pragma unroll
            for (int i = 0; i < CH; ++i) {
                const int e = tid + kThreads * (i0 + i);
                if (i0 + i < LOADS && e < MR * E) {
                    const int r = e / E, u = e - r * E;
                    S[frow(r, P) + u] = v[i];
                }
            }
        }
    }
    __syncthreads();
    if (a.discard)
        for (int yr = 0; yr < YR; ++yr) discard_scratch_rows<N, M>(sp + (size_t)(j0 + yr) * TP4);
    if (tid < MR) {   // DC column + i * Nyquist column
        float4 e = S[frow(tid, P)];
        const float4 ny = S[frow(tid, P) + Q];
        e.x -= ny.z;
        e.z += ny.x;
        S[frow(tid, P)] = e;
    }
    __syncthreads();
    {
        constexpr int TSM = team_size<M>(), TEAMSM = kThreads / TSM;
        const int tm = tid / TSM, lm = tid % TSM;
        float2 wr[Fac<M>::R1], wi[Fac<M>::R1];
        angular_twiddles<M>(TWM, lm, wr, wi);
        for (int c0 = 0; c0 < YR * Q; c0 += TEAMSM) {
            const int c = c0 + tm;          // column u = c % Q of y row c / Q
            const bool act = c < YR * Q;
            column_fft2<M, P, +1>(S + frow((act ? c / Q : 0) * M, P), act ? c % Q : 0, lm, act, wr, wi, SyncWarp());
        }
    }
    __syncthreads();
    // entry (m, 0) now holds (X_m[0], X_m[Q].re, X_m[N/2], X_m[Q].im) with
    // X_m[0], X_m[N/2] real
    const int team = tid / TS, lane = tid % TS;
    float* ob = op + (size_t)j0 * N;
    for (int q0 = 0; q0 < JOBS; q0 += TEAMS) {
        const int q = q0 + team;
        const bool act = q < JOBS;
        float2 re[RM], im[RM];
#pragma unroll
        for (int i = 0; i < RM; ++i) { re[i] = pf(0.f, 0.f); im[i] = pf(0.f, 0.f); }
        const float4* row0 = S + frow(4 * (act ? q : 0), P);
        if (act && lane < R2) {
            // Z_a[kk] = X_{4q}[kk] + i X_{4q+1}[kk], Z_b likewise with rows 4q+2, 4q+3,
            // kk = lane + R2 jj; bins above N/2 are conjugates of N - kk
#pragma unroll
            for (int jj = 0; jj < QJ; ++jj) {
                const int e = lane + R2 * jj;
                const float4 v0 = row0[e], v1 = row0[P + e], v2 = row0[2 * P + e], v3 = row0[3 * P + e];
                const bool dc = (jj == 0) && lane == 0;
                // kk = e (low half; the DC entry's imaginary slot holds X[N/2])
                const float i0 = dc ? 0.f : v0.z, i1 = dc ? 0.f : v1.z, i2 = dc ? 0.f : v2.z, i3 = dc ? 0.f : v3.z;
                re[jj] = pf(v0.x - i1, v2.x - i3);
                im[jj] = pf(i0 + v1.x, i2 + v3.x);
                // kk = e + Q (high half)
                re[jj + QJ] = pf(v0.y - v1.w, v2.y - v3.w);
                im[jj + QJ] = pf(v0.w + v1.y, v2.w + v3.y);
            }
#pragma unroll
            for (int jj = HJ; jj < HJ + QJ; ++jj) {
                // kk = lane + R2 jj in [N/2, N/2 + Q): X[kk] = conj X[N - kk], N - kk - Q < Q
                const bool ny = (jj == HJ) && lane == 0;
                const int e = ny ? 0 : N - lane - R2 * jj - Q;
                const float4 v0 = row0[e], v1 = row0[P + e], v2 = row0[2 * P + e], v3 = row0[3 * P + e];
                // kk: high half of entry e, conjugated; the Nyquist bin is the DC entry's z
                const float r0 = ny ? v0.z : v0.y, r1 = ny ? v1.z : v1.y, r2 = ny ? v2.z : v2.y, r3 = ny ? v3.z : v3.y;
                const float n0 = ny ? 0.f : -v0.w, n1 = ny ? 0.f : -v1.w, n2 = ny ? 0.f : -v2.w, n3 = ny ? 0.f : -v3.w;
                re[jj] = pf(r0 - n1, r2 - n3);
                im[jj] = pf(n0 + r1, n2 + r3);
                // kk + Q: low half of entry e, conjugated (Nyquist lane: X[Q] = high half of entry 0)
                const float s0 = ny ? v0.y : v0.x, s1 = ny ? v1.y : v1.x, s2 = ny ? v2.y : v2.x, s3 = ny ? v3.y : v3.x;
                const float m0 = ny ? -v0.w : -v0.z, m1 = ny ? -v1.w : -v1.z, m2 = ny ? -v2.w : -v2.z, m3 = ny ? -v3.w : -v3.z;
                re[jj + QJ] = pf(s0 - m1, s2 - m3);
                im[jj + QJ] = pf(m0 + s1, m2 + s3);
            }
        }
        __syncwarp();   // every read of the team's rows is done before the exchange reuses them
        float4* xb = S + frow(4 * (act ? q : 0), P);
        team_fft2<R1, R2, +1>(re, im, lane, act, xb, TW, SyncWarp());
        if (act && lane < R1) {
            float* o0 = ob + (size_t)(q / JY) * N + (size_t)(4 * (q % JY)) * NN;
#pragma unroll
            for (int k = 0; k < R2; ++k) {
                const int x = lane + R1 * k;
                __stcs(o0 + x, re[k].x);
                __stcs(o0 + NN + x, im[k].x);
                __stcs(o0 + 2 * NN + x, re[k].y);
                __stcs(o0 + 3 * NN + x, im[k].y);
            }
        }
    }
}

template <int N, int M>
__global__ void __launch_bounds__(kThreads, 2) kf_inv_tx(FArgs a) {
    extern __shared__ float4 fsm[];
    inv_tx_body<N, M>(a, blockIdx.x, a.s + (size_t)blockIdx.y * a.s_pstride, a.out + (size_t)blockIdx.y * N * N * M, fsm);
}

template <int N, int M> constexpr size_t fast_xt_smem() {
    return (size_t)(fslab4<N, fast_yr<N, M>() * M>() + N + M / 2) * sizeof(float4);
}
template <int N, int M> constexpr size_t fast_lines_smem() {
    return (size_t)(fast_lines<N>() * fast_xs<N>() + 2 * N) * sizeof(float4) + (size_t)(N / 2 + 1 + N + M) * sizeof(float2);
}

}  // namespace se2
