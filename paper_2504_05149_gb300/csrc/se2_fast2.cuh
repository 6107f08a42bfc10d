// FP32 units A and C of the convolution (Algorithm 3 / Eq. MatSqKfgG at
// output grid N = L) for N = R * R, with every global transfer a bulk
// asynchronous copy of one contiguous row and the real-FFT split done in
// registers.  Same scratch layout as se2_fast.cuh ("paired spectrum", entries
// (u, u + N/4) per float4), so unit B is shared.
//
// Data movement of one y row (a block):
//   unit A  f rows (theta, y = j) --bulk--> slab --x FFT, split--> slab
//           --angular FFT--> slab --bulk--> scratch rows (m, j)
//   unit C  scratch rows --bulk--> slab --inverse angular FFT--> slab
//           --inverse x FFT--> slab --bulk--> out rows
// Bulk copies move whole rows through the copy engine instead of warp-wide
// loads and stores that touch many rows per instruction; the block waits for
// its inputs on one mbarrier (bounded: on time-out it sets the plan's error
// word to 3 and returns).
//
// x FFT of one complex line z = row a + i row b (two real theta rows) by a
// team of R/2 lanes, n = t + R j:
//   pass 1 (DFT over j, per t)   lane p holds t = 2p, 2p + 1 (the two register
//                                halves), read as float2;
//   twiddle e^{-2 pi i t k1 / N};
//   pass 2 (DFT over t, per k1)  lane p holds the column pair (p, R - p)
//                                ((0, R/2) for p = 0); X[k1 + R k2] in
//                                register k2.
// The column pair is closed under k -> N - k, so the split of Z into the two
// rows' spectra (Z[k] + conj Z[N-k], -i (Z[k] - conj Z[N-k])) reads only the
// lane's own registers.  The inverse (unit C) runs the same passes backwards.
#pragma once
#include "se2_fast.cuh"

namespace se2 {

template <int N> struct X2 {
    static constexpr int R = N == 256 ? 16 : (N == 64 ? 8 : 0);   // N = R * R
    static constexpr int TL = R / 2;                               // lanes per x line
    static constexpr int XP = R + 1;                               // exchange pitch (odd)
};
template <int N> constexpr bool fast2_ok() { return X2<N>::R > 0; }

// Slab pitch: odd, >= N/4 + 1 entries, >= N/4 entries of real data (a row of
// f), and two rows hold one team's exchange.
template <int N> __host__ __device__ constexpr int f2pitch() {
    constexpr int ex = X2<N>::TL * X2<N>::XP;
    constexpr int a = (ex + 1) / 2 > N / 4 + 1 ? (ex + 1) / 2 : N / 4 + 1;
    return a | 1;
}
template <int N, int M> __host__ __device__ constexpr int f2slab4() { return M * f2pitch<N>() + (M >> 3) + 1; }
// slab + x twiddles [R-1][TL] (float4) + angular twiddles [M] (float2)
template <int N, int M> constexpr size_t fast2_smem() {
    return (size_t)(f2slab4<N, M>() + (X2<N>::R - 1) * X2<N>::TL + M / 2) * sizeof(float4);
}

// Second-pass column pair of lane p.
template <int R> __device__ __forceinline__ int col_b(int p) { return p == 0 ? R / 2 : R - p; }

// x-pass twiddle table: tw[(k - 1) * TL + p] = (w_a.re, w_b.re, w_a.im, w_b.im)
// with w = e^{-2 pi i n k / N}; forward: n = 2p, 2p + 1 (the pass-1 t pair),
// inverse: n = p, col_b(p) (the pass-1 columns), k = 1 .. R-1.
template <int N, bool INV>
__device__ __forceinline__ void fill_tw_x2(float4* tw, const float2* twN) {
    constexpr int R = X2<N>::R, TL = X2<N>::TL;
    for (int n = threadIdx.x; n < (R - 1) * TL; n += blockDim.x) {
        const int k = n / TL + 1, p = n - (n / TL) * TL;
        const int na = INV ? p : 2 * p, nb = INV ? col_b<R>(p) : 2 * p + 1;
        const float2 w0 = twN[(na * k) % N], w1 = twN[(nb * k) % N];
        tw[n] = make_float4(w0.x, w1.x, w0.y, w1.y);
    }
}

// ---------------------------------------------------------------------------
// Bulk asynchronous copies (copy engine) and the mbarrier that tracks them
// ---------------------------------------------------------------------------
__device__ __forceinline__ unsigned sm_u32(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void mbar_init(unsigned long long* bar, unsigned count) {
    asm volatile("mbarrier.init.shared.b64 [%0], %1;" :: "r"(sm_u32(bar)), "r"(count) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_arrive_expect(unsigned long long* bar, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared.b64 _, [%0], %1;" :: "r"(sm_u32(bar)), "r"(bytes) : "memory");
}
// global -> shared, `bytes` a multiple of 16, both addresses 16-byte aligned
__device__ __forceinline__ void bulk_load(void* dst, const void* src, unsigned bytes, unsigned long long* bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                 :: "r"(sm_u32(dst)), "l"(src), "r"(bytes), "r"(sm_u32(bar)) : "memory");
}
// shared -> global, same rules; completes in the issuing thread's bulk group
__device__ __forceinline__ void bulk_store(void* dst, const void* src, unsigned bytes) {
    asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;" :: "l"(dst), "r"(sm_u32(src)), "r"(bytes) : "memory");
}
__device__ __forceinline__ void bulk_commit_and_drain() {
    asm volatile("cp.async.bulk.commit_group;" ::: "memory");
    asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");
}
// generic-proxy shared-memory writes become visible to the copy engine
__device__ __forceinline__ void fence_to_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
// Poll phase `parity` of the barrier at most `limit` times.
__device__ __forceinline__ bool mbar_wait(unsigned long long* bar, unsigned parity, long limit) {
    unsigned done = 0;
    for (long it = 0; it < limit && !done; ++it)
        asm volatile("{ .reg .pred p; mbarrier.try_wait.parity.shared.b64 p, [%1], %2; selp.u32 %0, 1, 0, p; }"
                     : "=r"(done) : "r"(sm_u32(bar)), "r"(parity) : "memory");
    return done != 0;
}
constexpr long kBulkPolls = 1l << 22;

// Block-uniform wait for the block's input copies; false (error word set)
// when they did not arrive within the poll budget.
__device__ __forceinline__ bool block_wait_inputs(unsigned long long* bar, int* err) {
    bool ok = mbar_wait(bar, 0, kBulkPolls);
    ok = __syncthreads_and(ok) != 0;
    if (!ok) {
        mbar_wait(bar, 0, kBulkPolls);   // give copies still in flight a last chance to land
        if (threadIdx.x == 0 && err != nullptr) atomicExch(err, 3);
    }
    return ok;
}

// Forward x pass of line q (theta rows 2q, 2q + 1, read from the slab) by
// lane p of its team, the split in registers, and the rows' spectra written
// back over the same two slab rows (which also serve as the exchange).
template <int N>
__device__ __forceinline__ void x_fwd_line(float4* S, int q, int p, bool act, const float4* TWX) {
    constexpr int R = X2<N>::R, TL = X2<N>::TL, XP = X2<N>::XP, P = f2pitch<N>();
    const int ca = p, cb = col_b<R>(p);
    float2 re[R], im[R];
    float4* xb = S + frow(2 * (act ? q : 0), P);
    if (act) {
        const float* r0 = reinterpret_cast<const float*>(xb) + 2 * p;
        const float* r1 = reinterpret_cast<const float*>(xb + P) + 2 * p;
#pragma unroll
        for (int jj = 0; jj < R; ++jj) {
            re[jj] = *reinterpret_cast<const float2*>(r0 + R * jj);
            im[jj] = *reinterpret_cast<const float2*>(r1 + R * jj);
        }
    } else {
#pragma unroll
        for (int i = 0; i < R; ++i) { re[i] = pf(0.f, 0.f); im[i] = pf(0.f, 0.f); }
    }
    __syncwarp();   // the team's rows are read before they take the exchange
    // pass 1: DFT over j for t = 2p (.x) and 2p + 1 (.y)
    fft2_reg<R, -1>(re, im);
#pragma unroll
    for (int k1 = 1; k1 < R; ++k1) {
        const float4 w = TWX[(k1 - 1) * TL + p];
        ptw<-1>(re[k1], im[k1], pf(w.x, w.y), pf(w.z, w.w));
    }
    // exchange: slot (c, t) holds column pair c of pass-1 output t, t stored
    // at (t >> 1) + TL (t & 1)
    if (act) {
#pragma unroll
        for (int c = 0; c < TL; ++c) {
            const int A_ = c, B_ = c == 0 ? R / 2 : R - c;
            xb[c * XP + p] = make_float4(re[A_].x, re[B_].x, im[A_].x, im[B_].x);
            xb[c * XP + p + TL] = make_float4(re[A_].y, re[B_].y, im[A_].y, im[B_].y);
        }
    }
    __syncwarp();
    if (act) {
#pragma unroll
        for (int t = 0; t < R; ++t) {
            const float4 v = xb[p * XP + (t >> 1) + TL * (t & 1)];
            re[t] = pf(v.x, v.y);
            im[t] = pf(v.z, v.w);
        }
    }
    __syncwarp();   // the exchange is read before the rows take the spectra
    // pass 2: DFT over t; register k2 = (Z[ca + R k2], Z[cb + R k2])
    fft2_reg<R, -1>(re, im);
    if (act) {
        // X0 = Z + conj Z[N-k], X1 = -i (Z - conj Z[N-k]): twice the spectra of
        // rows 2q and 2q + 1 at bins ca + R k (.x) and cb + R k (.y), k < R/2
        float2 x0r[R / 2], x0i[R / 2], x1r[R / 2], x1i[R / 2];
#pragma unroll
        for (int k = 0; k < R / 2; ++k) {
            // mirror partners: lane 0's columns 0 and R/2 are each closed under
            // k -> N - k; lane p's columns p and R - p map onto each other
            const float2 mr = p == 0 ? pf(re[(R - k) & (R - 1)].x, re[R - 1 - k].y) : pf(re[R - 1 - k].y, re[R - 1 - k].x);
            const float2 mi = p == 0 ? pf(im[(R - k) & (R - 1)].x, im[R - 1 - k].y) : pf(im[R - 1 - k].y, im[R - 1 - k].x);
            x0r[k] = padd(re[k], mr);
            x0i[k] = psub(im[k], mi);
            x1r[k] = padd(im[k], mi);
            x1i[k] = psub(mr, re[k]);
        }
        // Nyquist bin N/2 (real): lane 0, column 0, register R/2
        const float ny0 = 2.f * re[R / 2].x, ny1 = 2.f * im[R / 2].x;
        constexpr int H = R / 4;   // register distance between bins u and u + N/4
#pragma unroll
        for (int k = 0; k < H; ++k) {
            const int ua = ca + R * k, ub = cb + R * k;
            float4 e0 = make_float4(x0r[k].x, x0r[k + H].x, x0i[k].x, x0i[k + H].x);
            float4 e1 = make_float4(x1r[k].x, x1r[k + H].x, x1i[k].x, x1i[k + H].x);
            if (k == 0 && p == 0) {   // X[0], X[N/2] are real: one complex DC entry
                e0.z = ny0;
                e1.z = ny1;
            }
            xb[ua] = e0;
            xb[P + ua] = e1;
            xb[ub] = make_float4(x0r[k].y, x0r[k + H].y, x0i[k].y, x0i[k + H].y);
            xb[P + ub] = make_float4(x1r[k].y, x1r[k + H].y, x1i[k].y, x1i[k + H].y);
        }
    }
}

// ---------------------------------------------------------------------------
// Unit A: forward real x FFT of the M theta rows of y row j, split into the
// rows' spectra, angular FFT of the slab columns (the DC and Nyquist x bins,
// both real, travel as one complex column and are split afterwards), the
// slab rows copied to scratch rows (m, j).  f must be 16-byte aligned.
// ---------------------------------------------------------------------------
template <int N, int M>
__global__ void __launch_bounds__(kThreads, 2) kf2_fwd_xt(FArgs a) {
    constexpr int R = X2<N>::R, TL = X2<N>::TL;
    constexpr int Q = N / 4, P = f2pitch<N>(), TP4 = ftp4<N>();
    constexpr int LINES = M / 2, TEAMS = kThreads / TL;
    constexpr size_t NN = (size_t)N * N;
    static_assert(R >= 4 && R * R == N, "N = R * R");
    extern __shared__ float4 fsm[];
    __shared__ __align__(8) unsigned long long bar;
    float4* S = fsm;
    float4* TWX = fsm + f2slab4<N, M>();
    float2* TWM = reinterpret_cast<float2*>(TWX + (R - 1) * TL);
    const int tid = threadIdx.x, j = blockIdx.x, b = blockIdx.y;
    if (tid == 0) {
        mbar_init(&bar, 1);
        mbar_arrive_expect(&bar, (unsigned)(M * N * 4));
    }
    __syncthreads();
    if (tid < 32) {
        const float* src = a.f + (size_t)b * NN * M + (size_t)j * N;
        for (int r = tid; r < M; r += 32) bulk_load(S + frow(r, P), src + (size_t)r * NN, N * 4, &bar);
    }
    fill_tw_x2<N, false>(TWX, a.twN);   // the table fills overlap the copies
    copy_tw(TWM, a.twM, M);
    if (!block_wait_inputs(&bar, a.err)) return;
    {
        const int team = tid / TL, p = tid % TL;
        for (int q0 = 0; q0 < LINES; q0 += TEAMS) x_fwd_line<N>(S, q0 + team, p, q0 + team < LINES, TWX);
    }
    __syncthreads();
    {
        constexpr int TSM = team_size<M>(), TEAMSM = kThreads / TSM;
        const int tm = tid / TSM, lm = tid % TSM;
        float2 wr[Fac<M>::R1], wi[Fac<M>::R1];
        angular_twiddles<M>(TWM, lm, wr, wi);
        for (int c0 = 0; c0 < Q; c0 += TEAMSM) {
            const int u = c0 + tm;
            const bool act = u < Q;
            column_fft2<M, P, -1>(S, act ? u : 0, lm, act, wr, wi, SyncWarp());
        }
    }
    __syncthreads();
    // split the DC column's transform Y = F(X[.,0] + i X[.,N/2]) into the two
    // real columns' transforms: (Y + conj Y[-m]) / 2 and (Y - conj Y[-m]) / 2i
    float4 yv = make_float4(0.f, 0.f, 0.f, 0.f), ym = yv;
    if (tid < M) {
        yv = S[frow(tid, P)];
        ym = S[frow((M - tid) & (M - 1), P)];
    }
    __syncthreads();
    if (tid < M) {
        float4 e = yv;
        e.x = 0.5f * (yv.x + ym.x);
        e.z = 0.5f * (yv.z - ym.z);
        S[frow(tid, P)] = e;
        S[frow(tid, P) + Q] = make_float4(0.5f * (yv.z + ym.z), 0.f, 0.5f * (ym.x - yv.x), 0.f);
    }
    fence_to_async();
    __syncthreads();
    if (tid < 32) {
        float4* dst = a.s + (size_t)b * a.s_pstride + (size_t)j * TP4;
        for (int m = tid; m < M; m += 32) bulk_store(dst + (size_t)m * N * TP4, S + frow(m, P), (Q + 1) * 16);
        bulk_commit_and_drain();
    }
}

// Inverse x pass of line q by lane p: reads the half spectra of slab rows
// 2q, 2q + 1 (entry (l, 0) = (X[0], X[Q].re, X[N/2], X[Q].im) with X[0] and
// X[N/2] real), forms Z = X0 + i X1 on the lane's column pair (Hermitian
// extension X[N-k] = conj X[k]), inverse FFT, and writes the two real rows
// over the same slab rows.
template <int N>
__device__ __forceinline__ void x_inv_line(float4* S, int q, int p, bool act, const float4* TWX) {
    constexpr int R = X2<N>::R, TL = X2<N>::TL, XP = X2<N>::XP, P = f2pitch<N>();
    const int ca = p, cb = col_b<R>(p);
    float2 re[R], im[R];
    float4* xb = S + frow(2 * (act ? q : 0), P);
    if (act) {
        // bins ca + R k and cb + R k (k < R/2) of rows 2q (0) and 2q + 1 (1)
        constexpr int H = R / 4;
        float2 a0[R / 2], a1[R / 2], b0[R / 2], b1[R / 2];   // (re, im) of each bin
        float nyq0 = 0.f, nyq1 = 0.f;
#pragma unroll
        for (int k = 0; k < H; ++k) {
            const float4 va0 = xb[ca + R * k], va1 = xb[P + ca + R * k];
            const float4 vb0 = xb[cb + R * k], vb1 = xb[P + cb + R * k];
            a0[k] = pf(va0.x, va0.z);
            a0[k + H] = pf(va0.y, va0.w);
            a1[k] = pf(va1.x, va1.z);
            a1[k + H] = pf(va1.y, va1.w);
            b0[k] = pf(vb0.x, vb0.z);
            b0[k + H] = pf(vb0.y, vb0.w);
            b1[k] = pf(vb1.x, vb1.z);
            b1[k + H] = pf(vb1.y, vb1.w);
            if (k == 0) {   // lane 0, entry 0: the imaginary slot holds X[N/2]
                nyq0 = va0.z;
                nyq1 = va1.z;
            }
        }
        if (p == 0) {
            a0[0].y = 0.f;
            a1[0].y = 0.f;
        }
#pragma unroll
        for (int k2 = 0; k2 < R; ++k2) {
            float2 za0, za1, zb0, zb1;   // X0, X1 at column a and column b of register k2
            if (k2 < R / 2) {
                za0 = a0[k2];
                za1 = a1[k2];
                zb0 = b0[k2];
                zb1 = b1[k2];
            } else if (p == 0) {
                // column 0: bin R k2 mirrors bin R (R - k2); k2 = R/2 is the Nyquist bin
                const int m = (R - k2) & (R / 2 - 1);
                za0 = k2 == R / 2 ? pf(nyq0, 0.f) : pf(a0[m].x, -a0[m].y);
                za1 = k2 == R / 2 ? pf(nyq1, 0.f) : pf(a1[m].x, -a1[m].y);
                zb0 = pf(b0[R - 1 - k2].x, -b0[R - 1 - k2].y);
                zb1 = pf(b1[R - 1 - k2].x, -b1[R - 1 - k2].y);
            } else {
                za0 = pf(b0[R - 1 - k2].x, -b0[R - 1 - k2].y);
                za1 = pf(b1[R - 1 - k2].x, -b1[R - 1 - k2].y);
                zb0 = pf(a0[R - 1 - k2].x, -a0[R - 1 - k2].y);
                zb1 = pf(a1[R - 1 - k2].x, -a1[R - 1 - k2].y);
            }
            re[k2] = pf(za0.x - za1.y, zb0.x - zb1.y);
            im[k2] = pf(za0.y + za1.x, zb0.y + zb1.x);
        }
    } else {
#pragma unroll
        for (int i = 0; i < R; ++i) { re[i] = pf(0.f, 0.f); im[i] = pf(0.f, 0.f); }
    }
    __syncwarp();   // every read of the team's rows is done before the exchange reuses them
    // pass 1: inverse DFT over k2 for columns ca (.x) and cb (.y), then twiddle
    // e^{+2 pi i t k1 / N}
    fft2_reg<R, +1>(re, im);
#pragma unroll
    for (int t = 1; t < R; ++t) {
        const float4 w = TWX[(t - 1) * TL + p];
        ptw<+1>(re[t], im[t], pf(w.x, w.y), pf(w.z, w.w));
    }
    // exchange: slot (i, k1) holds outputs t = 2i, 2i + 1 of column k1
    if (act) {
#pragma unroll
        for (int i = 0; i < TL; ++i) {
            xb[i * XP + ca] = make_float4(re[2 * i].x, re[2 * i + 1].x, im[2 * i].x, im[2 * i + 1].x);
            xb[i * XP + cb] = make_float4(re[2 * i].y, re[2 * i + 1].y, im[2 * i].y, im[2 * i + 1].y);
        }
    }
    __syncwarp();
    if (act) {
#pragma unroll
        for (int k1 = 0; k1 < R; ++k1) {
            const float4 v = xb[p * XP + k1];
            re[k1] = pf(v.x, v.y);
            im[k1] = pf(v.z, v.w);
        }
    }
    __syncwarp();   // the exchange is read before the rows take the output
    // pass 2: inverse DFT over k1; register jj = x = 2p + R jj (.x), 2p + 1 + R jj (.y)
    fft2_reg<R, +1>(re, im);
    if (act) {
        float* r0 = reinterpret_cast<float*>(xb) + 2 * p;
        float* r1 = reinterpret_cast<float*>(xb + P) + 2 * p;
#pragma unroll
        for (int jj = 0; jj < R; ++jj) {
            *reinterpret_cast<float2*>(r0 + R * jj) = re[jj];
            *reinterpret_cast<float2*>(r1 + R * jj) = im[jj];
        }
    }
}

// ---------------------------------------------------------------------------
// Unit C: scratch rows (m, j) copied into the slab, inverse angular FFT of the
// slab columns (DC and Nyquist columns recombined into one complex column
// first), inverse x FFT of the row pairs (2q, 2q + 1), the real rows copied
// to out.  out must be 16-byte aligned.
// ---------------------------------------------------------------------------
template <int N, int M>
__global__ void __launch_bounds__(kThreads, 2) kf2_inv_tx(FArgs a) {
    constexpr int R = X2<N>::R, TL = X2<N>::TL;
    constexpr int Q = N / 4, P = f2pitch<N>(), TP4 = ftp4<N>();
    constexpr int LINES = M / 2, TEAMS = kThreads / TL;
    constexpr size_t NN = (size_t)N * N;
    extern __shared__ float4 fsm[];
    __shared__ __align__(8) unsigned long long bar;
    float4* S = fsm;
    float4* TWX = fsm + f2slab4<N, M>();
    float2* TWM = reinterpret_cast<float2*>(TWX + (R - 1) * TL);
    const int tid = threadIdx.x, j = blockIdx.x, b = blockIdx.y;
    if (tid == 0) {
        mbar_init(&bar, 1);
        mbar_arrive_expect(&bar, (unsigned)(M * (Q + 1) * 16));
    }
    __syncthreads();
    if (tid < 32) {
        const float4* src = a.s + (size_t)b * a.s_pstride + (size_t)j * TP4;
        for (int m = tid; m < M; m += 32) bulk_load(S + frow(m, P), src + (size_t)m * N * TP4, (Q + 1) * 16, &bar);
    }
    fill_tw_x2<N, true>(TWX, a.twN);   // the table fills overlap the copies
    copy_tw(TWM, a.twM, M);
    if (!block_wait_inputs(&bar, a.err)) return;
    if (tid < M) {   // DC column + i * Nyquist column
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
        for (int c0 = 0; c0 < Q; c0 += TEAMSM) {
            const int u = c0 + tm;
            const bool act = u < Q;
            column_fft2<M, P, +1>(S, act ? u : 0, lm, act, wr, wi, SyncWarp());
        }
    }
    __syncthreads();
    {
        const int team = tid / TL, p = tid % TL;
        for (int q0 = 0; q0 < LINES; q0 += TEAMS) x_inv_line<N>(S, q0 + team, p, q0 + team < LINES, TWX);
    }
    fence_to_async();
    __syncthreads();
    if (tid < 32) {
        float* dst = a.out + (size_t)b * NN * M + (size_t)j * N;
        for (int r = tid; r < M; r += 32) bulk_store(dst + (size_t)r * NN, S + frow(r, P), N * 4);
        bulk_commit_and_drain();
    }
}

}  // namespace se2
