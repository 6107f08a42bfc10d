// FP32 convolution (Algorithm 3 / the chain of Eq. MatSqKfgG at N = L) of a
// whole batch as one persistent dataflow launch: one block per SM runs work
// items of three kinds in a dependency-safe global order,
//   A(p, j)  x FFT + split + angular FFT of y row j of problem p (unit A),
//   B(p, i)  y FFT, product with the coefficients, inverse y FFT of 16
//            line pairs (unit B),
//   C(p, j)  inverse angular FFT + inverse x FFT of y row j (unit C),
// emitted step by step: step t holds A(t), B(t-1), C(t-2).  Problem p keeps
// its spectrum in scratch slot p mod S (S >= 3 slots, L2-resident), so A(p)
// waits until C(p - S) has finished, B(p) until A(p), C(p) until B(p); all
// waits point at items earlier in the order.
//
// Inside a block a producer warp takes items from a global counter, waits
// for their dependencies, and moves each item's input rows into one of
// NBUF shared-memory buffers with bulk asynchronous copies (completion on an
// mbarrier); 8 compute warps transform the buffer in place and hand it back;
// the producer copies the result rows out, waits for the writes, and counts
// the item done for its problem.  So the next items' inputs arrive while the
// current one is computed.
//
// Every wait is bounded; on time-out the waiting side sets the plan's error
// word to 4 and the block winds down (later waits on its items time out
// too), so a launch always ends.
#pragma once
#include <cuda.h>   // CUtensorMap (the maps are encoded on the host)

#include "se2_fast2.cuh"

namespace se2 {

constexpr int kFlowCompute = 256;                 // compute threads (8 warps)
constexpr int kFlowThreads = kFlowCompute + 32;   // + the producer warp
constexpr int kFlowBufs = 3;
constexpr int kFlowLines = 16;                    // line pairs of a B item
constexpr int kFlowSlots = 4;                     // scratch slots wanted (problems in flight)
constexpr long kFlowPolls = 1l << 24;             // poll budget of one wait

enum FlowKind { FK_A = 0, FK_B = 1, FK_C = 2, FK_STOP = 3 };

// B items of a problem: (theta bin o, entries 16 b .. 16 b + 15) for b < N/64,
// then the Nyquist entry N/4 of 16 theta bins at a time.  Each item's tile is
// one box of a tensor map over the scratch.
template <int N, int M> struct FlowGeom {
    static constexpr int Q = N / 4, P = f2pitch<N>(), TP4 = ftp4<N>();
    static constexpr int NA = N;                                        // A (and C) items per problem
    static constexpr int NBLK = Q / kFlowLines;                         // entry blocks per theta bin
    static constexpr int NB = M * NBLK + M / kFlowLines;                // B items per problem
    static constexpr int SLAB = f2slab4<N, M>();
    static constexpr int TILE = N * kFlowLines;                          // B tile [ky][line pair]
    static constexpr int XB = kFlowLines * fast_xs<N>();                 // B exchange
    static constexpr int BUF0 = SLAB > TILE ? (SLAB > XB ? SLAB : XB) : (TILE > XB ? TILE : XB);
    static constexpr int BUF = (BUF0 + 7) / 8 * 8;                     // 128-byte aligned buffers
    // buffers, then unit B's forward/inverse team tables (2N), units A/C's x
    // tables (2 (R-1) TL) and the angular table (M float2)
    static constexpr int TABLES = 2 * N + 2 * (X2<N>::R - 1) * X2<N>::TL + M / 2;
    static constexpr size_t SMEM = (size_t)(kFlowBufs * BUF + TABLES) * sizeof(float4);
};
template <int N, int M> constexpr bool flow_ok() {
    // B items are 16 line pairs of one 16-lane team each: N = 256
    return N == 256 && M >= 16 && M % kFlowLines == 0 && FlowGeom<N, M>::SMEM <= 226 * 1024;
}

// Steps of the item order: step t holds A(t) (t < P), B(t-1) (1 <= t <= P),
// C(t-2) (2 <= t <= P+1).
__host__ __device__ inline long long flow_items(int P, int na, int nb) { return (long long)P * (2 * na + nb); }
__device__ inline void flow_decode(long long i, int P, int na, int nb, int* kind, int* prob, int* idx) {
    for (int t = 0; t < P + 2; ++t) {
        if (t < P) {
            if (i < na) { *kind = FK_A; *prob = t; *idx = (int)i; return; }
            i -= na;
        }
        if (t >= 1 && t <= P) {
            if (i < nb) { *kind = FK_B; *prob = t - 1; *idx = (int)i; return; }
            i -= nb;
        }
        if (t >= 2) {
            if (i < na) { *kind = FK_C; *prob = t - 2; *idx = (int)i; return; }
            i -= na;
        }
    }
    *kind = FK_STOP;
}

__device__ __forceinline__ void group_sync() { asm volatile("bar.sync 1, 256;" ::: "memory"); }
struct GroupSync { __device__ __forceinline__ void operator()() const { group_sync(); } };
__device__ __forceinline__ bool group_and(bool v) {
    unsigned r;
    asm volatile("{ .reg .pred p, q; setp.ne.u32 p, %1, 0; bar.red.and.pred q, 1, 256, p; selp.u32 %0, 1, 0, q; }"
                 : "=r"(r) : "r"((unsigned)v) : "memory");
    return r != 0;
}
__device__ __forceinline__ void mbar_arrive(unsigned long long* bar) {
    asm volatile("mbarrier.arrive.shared.b64 _, [%0];" :: "r"(sm_u32(bar)) : "memory");
}
__device__ __forceinline__ void fence_async_global() { asm volatile("fence.proxy.async.global;" ::: "memory"); }
// Tensor-map copies of a 3-D box (coordinates x fastest)
__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* map, int x, int y, int z, unsigned long long* bar) {
    asm volatile("cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];"
                 :: "r"(sm_u32(dst)), "l"((unsigned long long)map), "r"(x), "r"(y), "r"(z), "r"(sm_u32(bar)) : "memory");
}
__device__ __forceinline__ void tma_store_3d(const CUtensorMap* map, int x, int y, int z, const void* src) {
    asm volatile("cp.async.bulk.tensor.3d.global.shared::cta.bulk_group [%0, {%1, %2, %3}], [%4];"
                 :: "l"((unsigned long long)map), "r"(x), "r"(y), "r"(z), "r"(sm_u32(src)) : "memory");
}
__device__ __forceinline__ int ld_acquire(const int* p) {
    int v;
    asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// ---------------------------------------------------------------------------
// Compute parts (the 256 compute threads; tid < 256).  Buffers hold, for A
// and C items, the slab of one y row ([M] rows at frow(r, P)); for B items the
// tile [N ky][16 line pairs] of paired entries.
// ---------------------------------------------------------------------------
template <int N, int M>
__device__ __forceinline__ void flow_unit_a(float4* S, const float4* TWX, const float2* TWM, int tid) {
    constexpr int TL = X2<N>::TL, Q = N / 4, P = f2pitch<N>();
    constexpr int LINES = M / 2, TEAMS = kFlowCompute / TL;
    {
        const int team = tid / TL, p = tid % TL;
        for (int q0 = 0; q0 < LINES; q0 += TEAMS) x_fwd_line<N>(S, q0 + team, p, q0 + team < LINES, TWX);
    }
    group_sync();
    {
        constexpr int TSM = team_size<M>(), TEAMSM = kFlowCompute / TSM;
        const int tm = tid / TSM, lm = tid % TSM;
        float2 wr[Fac<M>::R1], wi[Fac<M>::R1];
        angular_twiddles<M>(TWM, lm, wr, wi);
        for (int c0 = 0; c0 < Q; c0 += TEAMSM) {
            const int u = c0 + tm;
            const bool act = u < Q;
            column_fft2<M, P, -1>(S, act ? u : 0, lm, act, wr, wi, SyncWarp());
        }
    }
    group_sync();
    // DC column Y = F(X[.,0] + i X[.,N/2]) -> (Y + conj Y[-m]) / 2, (Y - conj Y[-m]) / 2i
    float4 yv = make_float4(0.f, 0.f, 0.f, 0.f), ym = yv;
    if (tid < M) {
        yv = S[frow(tid, P)];
        ym = S[frow((M - tid) & (M - 1), P)];
    }
    group_sync();
    if (tid < M) {
        float4 e = yv;
        e.x = 0.5f * (yv.x + ym.x);
        e.z = 0.5f * (yv.z - ym.z);
        S[frow(tid, P)] = e;
        S[frow(tid, P) + Q] = make_float4(0.5f * (yv.z + ym.z), 0.f, 0.5f * (ym.x - yv.x), 0.f);
    }
}

template <int N, int M>
__device__ __forceinline__ void flow_unit_c(float4* S, const float4* TWX, const float2* TWM, int tid) {
    constexpr int TL = X2<N>::TL, Q = N / 4, P = f2pitch<N>();
    constexpr int LINES = M / 2, TEAMS = kFlowCompute / TL;
    if (tid < M) {   // DC column + i * Nyquist column
        float4 e = S[frow(tid, P)];
        const float4 ny = S[frow(tid, P) + Q];
        e.x -= ny.z;
        e.z += ny.x;
        S[frow(tid, P)] = e;
    }
    group_sync();
    {
        constexpr int TSM = team_size<M>(), TEAMSM = kFlowCompute / TSM;
        const int tm = tid / TSM, lm = tid % TSM;
        float2 wr[Fac<M>::R1], wi[Fac<M>::R1];
        angular_twiddles<M>(TWM, lm, wr, wi);
        for (int c0 = 0; c0 < Q; c0 += TEAMSM) {
            const int u = c0 + tm;
            const bool act = u < Q;
            column_fft2<M, P, +1>(S, act ? u : 0, lm, act, wr, wi, SyncWarp());
        }
    }
    group_sync();
    {
        const int team = tid / TL, p = tid % TL;
        for (int q0 = 0; q0 < LINES; q0 += TEAMS) x_inv_line<N>(S, q0 + team, p, q0 + team < LINES, TWX);
    }
}

// Unit B on one tile.  Line pair c = tid % 16 is (theta bin o, entry u): for
// a block item (o, 16 b + c), tile index ky * 16 + c; for a Nyquist item
// (o0 + c, N/4), tile index c * N + ky.  Lane t = tid / 16 holds ky = t + 16 j.
// The producer has asked L2 for the item's coefficient rows when it copied
// the tile in.
template <int N, int M>
__device__ __forceinline__ void flow_unit_b(float4* S, const float4* TWF, const float4* TWI, const FArgs& a, int prob,
                                            int item, int tid, double* sh_scale) {
    using G = FlowGeom<N, M>;
    constexpr int Q = N / 4, CP = N / 2 + 1, L16 = kFlowLines;
    constexpr int R1 = Fac<N>::R1, R2 = Fac<N>::R2, RM = reg_count<N>();
    constexpr int XS = fast_xs<N>();
    static_assert(kFlowCompute / team_size<N>() == L16 && R1 == R2, "16 line pairs of 16 lanes per item");
    const int c = tid % L16, t = tid / L16;
    const bool nyq = item >= M * G::NBLK;
    const int o = nyq ? (item - M * G::NBLK) * L16 + c : item / G::NBLK;
    const int u = nyq ? Q : (item % G::NBLK) * L16 + c;
    const int sk = nyq ? 1 : L16, sc = nyq ? N : 1;
    const bool hasb = u < Q;
    const int kxa = hasb ? u : N / 2;
    const bool ym = a.ymirror != 0;
    float2 re[RM], im[RM];
#pragma unroll
    for (int jj = 0; jj < R1; ++jj) {
        const float4 v = S[(t + R2 * jj) * sk + c * sc];
        re[jj] = pf(v.x, v.y);
        im[jj] = pf(v.z, v.w);
    }
    if (tid == 0) {
        double lsum = 0;
        for (int i = 0; i < a.k; ++i)
            if (a.ls[i] != nullptr) lsum += a.ls[i][prob * a.ls_pstride];
        *sh_scale = 0.5 * a.inv_L * exp(lsum);
    }
    group_sync();   // the tile is in registers before the exchange reuses it
    float4* xb = S + c * XS;
    team_fft2<R1, R2, -1>(re, im, t, true, xb, TWF, GroupSync());
    // lane s < R1 holds ky = s + R1 k
    {
        const float sc2 = (float)*sh_scale;
        const bool neg = a.wsign && (a.k & 1) && ((u + t) & 1);   // W^k at (kx, ky), both halves alike
        const float2 s2 = bc2(neg ? -sc2 : sc2);
        for (int i = 0; i < a.k; ++i) {
            float2 ca[R2], cq[R2];
            {
                const float2* cb = a.C[i] + (size_t)prob * a.c_pstride + (size_t)o * N * CP + kxa;
#pragma unroll
                for (int kk = 0; kk < R2; ++kk) {
                    int row = t + R1 * kk;
                    if (ym && row > N / 2) row = N - row;
                    ca[kk] = __ldcs(cb + (size_t)row * CP);
                    cq[kk] = hasb ? __ldcs(cb + (size_t)row * CP + Q) : pf(0.f, 0.f);
                }
            }
#pragma unroll
            for (int kk = 0; kk < R2; ++kk) {
                const float2 cr = pf(ca[kk].x, cq[kk].x), ci = pf(ca[kk].y, cq[kk].y);
                const float2 r = pfma(re[kk], cr, pneg(pmul(im[kk], ci)));
                im[kk] = pfma(re[kk], ci, pmul(im[kk], cr));
                re[kk] = r;
            }
        }
#pragma unroll
        for (int kk = 0; kk < R2; ++kk) {
            re[kk] = pmul(re[kk], s2);
            im[kk] = pmul(im[kk], s2);
        }
    }
    team_fft2<R2, R1, +1>(re, im, t, true, xb, TWI, GroupSync());
    // team_fft2 ends with a group barrier: the exchange is free
#pragma unroll
    for (int k = 0; k < R1; ++k) S[(t + R2 * k) * sk + c * sc] = make_float4(re[k].x, re[k].y, im[k].x, im[k].y);
}

// ---------------------------------------------------------------------------
// The persistent kernel
// ---------------------------------------------------------------------------
struct FlowArgs {
    // tensor maps over the scratch as [slots * M][N ky][4 * TP4 floats]:
    // boxes of 16 entries x N ky x 1 theta bin, and 1 entry x N ky x 16 bins
    CUtensorMap tm_blk, tm_nyq;
    FArgs a;                    // f, out, scratch slot 0, tables, coefficients, error word
    unsigned* work;             // next item (zeroed before the launch)
    int* cnt;                   // [3 P] items done per problem and kind (zeroed before the launch)
    int P;                      // problems
    int slots;                  // scratch slots; >= 3, or >= P (then no problem waits for a slot)
};

__device__ __forceinline__ unsigned long long gtime() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
constexpr unsigned long long kFlowWaitNs = 2000000000ull;   // 2 s per wait
__device__ __forceinline__ bool mbar_wait_ns(unsigned long long* bar, unsigned parity) {
    const unsigned long long t0 = gtime();
    for (;;) {
        unsigned done;
        asm volatile("{ .reg .pred p; mbarrier.try_wait.parity.shared.b64 p, [%1], %2; selp.u32 %0, 1, 0, p; }"
                     : "=r"(done) : "r"(sm_u32(bar)), "r"(parity) : "memory");
        if (done) return true;
        if (gtime() - t0 > kFlowWaitNs) return false;
    }
}
__device__ __forceinline__ bool wait_count(const int* c, int target) {
    const unsigned long long t0 = gtime();
    while (ld_acquire(c) < target) {
        if (gtime() - t0 > kFlowWaitNs) return false;
        __nanosleep(128);
    }
    return true;
}

// Input (ld) or output (!ld) row copies of one item between buffer S and
// global memory, spread over the producer lanes.
template <int N, int M, bool LD>
__device__ __forceinline__ void flow_copies(const FlowArgs& fa, int kind, int prob, int idx, float4* S, int lane,
                                            unsigned long long* bar) {
    using G = FlowGeom<N, M>;
    constexpr int Q = G::Q, P = G::P, TP4 = G::TP4, P1 = Q + 1;
    constexpr size_t NN = (size_t)N * N;
    const FArgs& a = fa.a;
    float4* slot = a.s + (size_t)(prob % fa.slots) * a.s_pstride;
    if (kind == FK_A || kind == FK_C) {
        const int j = idx;
        for (int r = lane; r < M; r += 32) {
            float4* row = S + frow(r, P);
            float4* sp = slot + (size_t)r * N * TP4 + (size_t)j * TP4;                  // scratch row (r, j)
            float* fp = (kind == FK_A ? const_cast<float*>(a.f) : a.out) + (size_t)prob * NN * M + (size_t)r * NN + (size_t)j * N;
            if (LD) {
                if (kind == FK_A) bulk_load(row, fp, N * 4, bar);
                else bulk_load(row, sp, P1 * 16, bar);
            } else {
                if (kind == FK_A) bulk_store(sp, row, P1 * 16);
                else bulk_store(fp, row, N * 4);
            }
        }
    } else {
        const bool nyq = idx >= M * G::NBLK;
        if (LD && !nyq) {   // coefficient rows of the first two kernels: 2 x 128 bytes per ky
            constexpr int CP = N / 2 + 1;
            const int o = idx / G::NBLK, kx = kFlowLines * (idx % G::NBLK);
            for (int i = 0; i < a.k && i < 2; ++i) {
                const float2* cb = a.C[i] + (size_t)prob * a.c_pstride + (size_t)o * N * CP + kx;
                for (int ky = lane; ky < N; ky += 32) {
                    const float2* r = cb + (size_t)ky * CP;
                    asm volatile("prefetch.global.L2 [%0];" :: "l"(r));
                    asm volatile("prefetch.global.L2 [%0];" :: "l"(r + kFlowLines - 1));
                    asm volatile("prefetch.global.L2 [%0];" :: "l"(r + Q));
                    asm volatile("prefetch.global.L2 [%0];" :: "l"(r + Q + kFlowLines - 1));
                }
            }
        }
        if (lane != 0) return;
        const int z = (prob % fa.slots) * M + (nyq ? (idx - M * G::NBLK) * kFlowLines : idx / G::NBLK);
        const int x = nyq ? 4 * Q : 4 * kFlowLines * (idx % G::NBLK);
        const CUtensorMap* map = nyq ? &fa.tm_nyq : &fa.tm_blk;
        if (LD) tma_load_3d(S, map, x, 0, z, bar);
        else tma_store_3d(map, x, 0, z, S);
    }
}

template <int N, int M>
__device__ __forceinline__ unsigned flow_bytes(int kind) {
    constexpr int P1 = N / 4 + 1;
    if (kind == FK_A) return (unsigned)(M * N * 4);
    if (kind == FK_C) return (unsigned)(M * P1 * 16);
    return (unsigned)(N * kFlowLines * 16);
}

template <int N, int M>
__global__ void __launch_bounds__(kFlowThreads, 1) kflow_conv(const __grid_constant__ FlowArgs fa) {
    using G = FlowGeom<N, M>;
    constexpr int NA = G::NA, NB = G::NB, BUF = G::BUF;
    constexpr int R = X2<N>::R, TL = X2<N>::TL, R1 = Fac<N>::R1, R2 = Fac<N>::R2;
    extern __shared__ __align__(128) float4 fsm[];
    __shared__ __align__(8) unsigned long long full[kFlowBufs], done[kFlowBufs];
    __shared__ int info[kFlowBufs][3];
    __shared__ double sh_scale;
    float4* TWF = fsm + kFlowBufs * BUF;
    float4* TWI = TWF + N;
    float4* TWXF = TWI + N;
    float4* TWXI = TWXF + (R - 1) * TL;
    float2* TWM = reinterpret_cast<float2*>(TWXI + (R - 1) * TL);
    const FArgs& a = fa.a;
    const int tid = threadIdx.x;
    if (tid == 0) {
        for (int s = 0; s < kFlowBufs; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&done[s], 1);
        }
    }
    fill_tw4<R1, R2>(TWF, a.twN);
    fill_tw4<R2, R1>(TWI, a.twN);
    fill_tw_x2<N, false>(TWXF, a.twN);
    fill_tw_x2<N, true>(TWXI, a.twN);
    copy_tw(TWM, a.twM, M);
    __syncthreads();
    if (tid >= kFlowCompute) {
        // ------------------------------ producer warp ------------------------------
        // Items are taken in increasing order; k counts the block's items, kfin
        // those copied out.  Item k uses buffer k % NBUF.  While an item waits for
        // its dependencies the warp keeps copying out its own finished items:
        // a dependency may be one of them, and the lowest unfinished item of the
        // whole order always progresses.
        const int lane = tid - kFlowCompute;
        const long long total = flow_items(fa.P, NA, NB);
        long long k = 0, kfin = 0;
        bool alive = true;
        // An item is counted done for its problem only once its output copies
        // have completed; its buffer is reused as soon as they have read it.
        // One item's copies stay in flight while the next ones proceed.
        int pend_prob = -1, pend_kind = 0;
        auto count_pending = [&](bool all) {
            if (pend_prob < 0) return;
            if (all) asm volatile("cp.async.bulk.wait_group 0;" ::: "memory");
            else asm volatile("cp.async.bulk.wait_group 1;" ::: "memory");
            fence_async_global();
            __syncwarp();
            if (lane == 0) {
                __threadfence();
                atomicAdd(fa.cnt + 3 * pend_prob + pend_kind, 1);
            }
            pend_prob = -1;
        };
        auto finish = [&](long long kk) -> bool {   // copy out item kk once computed
            const int s = (int)(kk % kFlowBufs);
            bool ok = true;
            if (lane == 0) ok = mbar_wait_ns(&done[s], (unsigned)((kk / kFlowBufs) & 1));
            ok = __shfl_sync(0xffffffffu, ok, 0);
            __syncwarp();
            if (!ok) return false;
            const int kind = info[s][0], prob = info[s][1], idx = info[s][2];
            flow_copies<N, M, false>(fa, kind, prob, idx, fsm + s * BUF, lane, nullptr);
            asm volatile("cp.async.bulk.commit_group;" ::: "memory");
            asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");   // the buffer is free
            count_pending(false);   // the previous item's copies have completed
            pend_prob = prob;
            pend_kind = kind;
            return true;
        };
        auto computed = [&](long long kk) -> bool {   // non-blocking: item kk is computed
            unsigned r = 0;
            if (lane == 0)
                asm volatile("{ .reg .pred p; mbarrier.test_wait.parity.shared.b64 p, [%1], %2; selp.u32 %0, 1, 0, p; }"
                             : "=r"(r) : "r"(sm_u32(&done[kk % kFlowBufs])), "r"((unsigned)((kk / kFlowBufs) & 1)) : "memory");
            return __shfl_sync(0xffffffffu, r, 0) != 0;
        };
        while (alive) {
            unsigned i = 0;
            if (lane == 0) i = atomicAdd(fa.work, 1u);
            i = __shfl_sync(0xffffffffu, i, 0);
            if ((long long)i >= total) break;
            if (k - kfin >= kFlowBufs) {   // free buffer k % NBUF
                if (!finish(kfin)) { alive = false; break; }
                ++kfin;
            }
            int kind = FK_STOP, prob = 0, idx = 0;
            flow_decode((long long)i, fa.P, NA, NB, &kind, &prob, &idx);
            const int* dep = nullptr;
            int target = 0;
            if (kind == FK_A && prob >= fa.slots) { dep = fa.cnt + 3 * (prob - fa.slots) + FK_C; target = NA; }
            else if (kind == FK_B) { dep = fa.cnt + 3 * prob + FK_A; target = NA; }
            else if (kind == FK_C) { dep = fa.cnt + 3 * prob + FK_B; target = NB; }
            if (dep != nullptr) {
                const unsigned long long t0 = gtime();
                for (;;) {
                    int v = 0;
                    if (lane == 0) v = ld_acquire(dep);
                    v = __shfl_sync(0xffffffffu, v, 0);
                    if (v >= target) break;
                    if (kfin < k && computed(kfin)) {
                        if (!finish(kfin)) { alive = false; break; }
                        ++kfin;
                        continue;
                    }
                    count_pending(true);   // another block may be waiting for it
                    if (gtime() - t0 > kFlowWaitNs) { alive = false; break; }
                    __nanosleep(256);
                }
                if (!alive) break;
            }
            __syncwarp();
            fence_async_global();   // the inputs written by other blocks' copies are read by ours
            const int s = (int)(k % kFlowBufs);
            if (lane == 0) {
                info[s][0] = kind;
                info[s][1] = prob;
                info[s][2] = idx;
                mbar_arrive_expect(&full[s], flow_bytes<N, M>(kind));
            }
            __syncwarp();
            flow_copies<N, M, true>(fa, kind, prob, idx, fsm + s * BUF, lane, &full[s]);
            ++k;
        }
        while (alive && kfin < k) {
            if (!finish(kfin)) alive = false;
            ++kfin;
        }
        count_pending(true);
        if (!alive && lane == 0) atomicExch(a.err, 4);
        if (lane == 0) {   // stop the compute warps (on the error path they may have stopped already)
            const int s = (int)(k % kFlowBufs);
            info[s][0] = FK_STOP;
            mbar_arrive(&full[s]);
        }
        return;
    }
    // ------------------------------ compute warps ------------------------------
    for (long long k = 0;; ++k) {
        const int s = (int)(k % kFlowBufs);
        const bool ok = group_and(mbar_wait_ns(&full[s], (unsigned)((k / kFlowBufs) & 1)));
        if (!ok) {
            if (tid == 0) atomicExch(a.err, 4);
            break;
        }
        const int kind = info[s][0], prob = info[s][1], idx = info[s][2];
        if (kind == FK_STOP) break;
        float4* S = fsm + s * BUF;
        if (kind == FK_A) flow_unit_a<N, M>(S, TWXF, TWM, tid);
        else if (kind == FK_B) flow_unit_b<N, M>(S, TWF, TWI, a, prob, idx, tid, &sh_scale);
        else flow_unit_c<N, M>(S, TWXI, TWM, tid);
        fence_to_async();
        group_sync();
        if (tid == 0) mbar_arrive(&done[s]);
    }
}

}  // namespace se2
