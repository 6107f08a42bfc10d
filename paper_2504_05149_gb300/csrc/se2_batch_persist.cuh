// One persistent launch over a whole batch of uneven problems: every problem
// is a separable-chain convolution (Algorithm 4 / Eq. MatSqKfgG at N = L,
// the chain's product in factored form) on its own N x N x M grid, and the
// units A, B, C of every problem of every size class run inside one kernel.
//
// Work list.  The host lays the units out in one array (one 32-bit code per
// unit: class, stage, block index, problem index inside the class).  Each
// class is a software pipeline of rounds; round r holds unit A of problem
// r, unit B of problem r - L and unit C of problem r - 2L, where the lag L
// (rounds) gives every dependency at least ~1.5 waves of other units between
// producer and consumer.  A class's rounds start when the class before it
// stops issuing units A, so the two overlap.  Blocks claim units in list
// order with one atomic counter (looking one unit ahead).
//
// Dependencies.  Per problem and stage a counter of finished units:
//   B of p waits for all units A of p, C of p for all units B of p, and A of
//   p for all units C of p - D, whose scratch slot (p mod D) it reuses.
// Every dependency points to an earlier place in the list, and blocks claim
// in list order, so the earliest unfinished unit can always run: no
// deadlock.  Each wait is bounded: a wait that gives up sets the error word
// to 6, and every block stops at its next wait.
#pragma once
#include "se2_fast.cuh"

namespace se2 {

static_assert(kLineThreads == kThreads, "units A, B and C run in blocks of one size");

// Size classes the kernel carries: N in {32, 64, 128, 256}, M in {16, 32, 64}.
constexpr int kBatchKinds = 12;
__host__ __device__ constexpr int batch_kind(int N, int M) {
    const int n = N == 32 ? 0 : N == 64 ? 1 : N == 128 ? 2 : N == 256 ? 3 : -1;
    const int m = M == 16 ? 0 : M == 32 ? 1 : M == 64 ? 2 : -1;
    return n < 0 || m < 0 ? -1 : 3 * n + m;
}

// One class of the batch, as the kernel sees it (device memory).
struct BClass {
    FArgs a;                 // twiddles, scale, W flag; s: the class's scratch ring
    long long goff, toff;    // offsets of its first problem in the packed grids / tables (elements)
    long long grid, tabs;    // elements of one grid / one problem's tables
    int kind;                // batch_kind(N, M)
    int first;               // batch index of its first problem (counters)
    int slots;               // ring slots D
    unsigned nA, nB, nC;     // units per stage of one problem
};

struct BPArgs {
    const BClass* cls;       // [n_classes]
    const unsigned* units;   // work list, n_units codes
    unsigned n_units;
    const float* f;          // packed grids (caller's)
    float* out;
    const float2* tables;    // packed separable tables
    unsigned* work;          // [1] next unit
    unsigned* cnt;           // [3 * n_problems] finished units per (problem, stage)
    int* err;                // error word (6: a wait gave up)
    long long spin_limit;    // polls before a wait gives up
    unsigned dep_extra;      // added to the A -> B target; nonzero only to test the timeout path
};

// Unit code: class (4 bits) | stage (2) | block index (10) | problem in class (16).
__host__ __device__ constexpr unsigned unit_code(int cls, int stage, int u, int p) {
    return ((unsigned)cls << 28) | ((unsigned)stage << 26) | ((unsigned)u << 16) | (unsigned)p;
}

// One unit of one class: a separate (not inlined) function per class and
// stage, so that each is compiled and register-allocated on its own, as the
// three kernels of the class are.
// g: the problem's grid (f for unit A, out for unit C) or tables (unit B);
// sp: its ring slot.
template <int N, int M>
__device__ __noinline__ void batch_unit_a(const BClass& c, int u, const float* g, float4* sp) {
    fwd_xt_body<N, M, false>(c.a, u, 0, g, sp);
}
template <int N, int M>
__device__ __noinline__ void batch_unit_b(const BClass& c, int u, int p, const float2* t, float4* sp) {
    lines_body<N, M, FL_SEP, false>(c.a, u, p, sp, t);
}
template <int N, int M>
__device__ __noinline__ void batch_unit_c(const BClass& c, int u, float* g, const float4* sp) {
    inv_tx_body<N, M, false>(c.a, u, 0, sp, g);
}
template <int N, int M>
__device__ __forceinline__ void batch_unit(const BPArgs& ba, const BClass& c, int stage, int u, int p) {
    float4* sp = c.a.s + (size_t)(p % c.slots) * c.a.s_pstride;
    if (stage == 0) batch_unit_a<N, M>(c, u, ba.f + c.goff + (size_t)p * c.grid, sp);
    else if (stage == 1) batch_unit_b<N, M>(c, u, p, ba.tables + c.toff + (size_t)p * c.tabs, sp);
    else batch_unit_c<N, M>(c, u, ba.out + c.goff + (size_t)p * c.grid, sp);
}

__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned* p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// Dependency of a unit: the counter it waits on and the count it needs
// (nullptr: none).
__device__ __forceinline__ const unsigned* unit_dep(const BPArgs& ba, unsigned code, unsigned* target) {
    const int ci = (int)(code >> 28), stage = (int)((code >> 26) & 3u), p = (int)(code & 0xffffu);
    const BClass& c = ba.cls[ci];
    if (stage == 1) {
        *target = c.nA + ba.dep_extra;
        return ba.cnt + 3 * (size_t)(c.first + p);
    }
    if (stage == 2) {
        *target = c.nB;
        return ba.cnt + 3 * (size_t)(c.first + p) + 1;
    }
    if (p >= c.slots) {
        *target = c.nC;
        return ba.cnt + 3 * (size_t)(c.first + p - c.slots) + 2;
    }
    *target = 0;
    return nullptr;
}

// The bookkeeping stays off the units' critical path: thread 0 knows the
// next unit's code and has claimed the one after it; at the start of each
// unit it issues the next unit's dependency read (acquire), the load of the
// following code and the next claim, whose results it uses only after the
// unit.  After a unit, lane 0 of the last warp publishes its completion
// (fence, then count) while thread 0 checks the next unit's dependency, so
// no block waits on its own unpublished unit.
// A template so that only the translation unit that takes its address
// compiles it (se2_batch.cu).
template <int UNUSED = 0>
__global__ void __launch_bounds__(kThreads, 2) kf_batch_persist(BPArgs ba) {
    __shared__ unsigned sh_code;
    __shared__ int sh_go;
    const int tid = threadIdx.x;
    const unsigned n = ba.n_units;
    unsigned g0 = 0, g1 = 0, g2 = 0, c0 = 0, c1 = 0;   // thread 0: units i, i+1 (codes), i+2 (claimed)
    int go0 = 0;
    if (tid == 0) {
        g0 = atomicAdd(ba.work, 1u);
        g1 = atomicAdd(ba.work, 1u);
        g2 = atomicAdd(ba.work, 1u);
        c0 = g0 < n ? ba.units[g0] : 0u;
        c1 = g1 < n ? ba.units[g1] : 0u;
        go0 = g0 < n;
    }
    unsigned ev1 = 0, t1 = 0;
    const unsigned* d1 = nullptr;
    bool early = false;
    for (;;) {
        if (tid == 0) {
            // the error word is read only while waiting: after a time-out every
            // block stops at its next wait or when the list is exhausted
            if (go0) {
                unsigned target;
                const unsigned* dep = early ? d1 : unit_dep(ba, c0, &target);
                if (early) target = t1;
                if (dep != nullptr && !(early && ev1 >= target)) {
                    long long it = 0;
                    while (ld_acquire_u32(dep) < target) {
                        if (++it > ba.spin_limit || *(volatile int*)ba.err != 0) {
                            atomicCAS(ba.err, 0, 6);
                            go0 = 0;
                            break;
                        }
                        __nanosleep(64);
                    }
                }
            }
            sh_go = go0;
            sh_code = c0;
        }
        __syncthreads();
        const int go = sh_go;
        const unsigned cd = sh_code;
        if (!go) break;
        unsigned c2 = 0, g3 = 0;
        if (tid == 0) {   // issued now, used after the unit
            c2 = g2 < n ? ba.units[g2] : 0u;
            g3 = atomicAdd(ba.work, 1u);
            d1 = g1 < n ? unit_dep(ba, c1, &t1) : nullptr;
            ev1 = d1 != nullptr ? ld_acquire_u32(d1) : 0u;
        }
        const int ci = (int)(cd >> 28), stage = (int)((cd >> 26) & 3u);
        const int u = (int)((cd >> 16) & 0x3ffu), p = (int)(cd & 0xffffu);
        const BClass& c = ba.cls[ci];
        switch (c.kind) {
            case 0: batch_unit<32, 16>(ba, c, stage, u, p); break;
            case 1: batch_unit<32, 32>(ba, c, stage, u, p); break;
            case 2: batch_unit<32, 64>(ba, c, stage, u, p); break;
            case 3: batch_unit<64, 16>(ba, c, stage, u, p); break;
            case 4: batch_unit<64, 32>(ba, c, stage, u, p); break;
            case 5: batch_unit<64, 64>(ba, c, stage, u, p); break;
            case 6: batch_unit<128, 16>(ba, c, stage, u, p); break;
            case 7: batch_unit<128, 32>(ba, c, stage, u, p); break;
            case 8: batch_unit<128, 64>(ba, c, stage, u, p); break;
            case 9: batch_unit<256, 16>(ba, c, stage, u, p); break;
            case 10: batch_unit<256, 32>(ba, c, stage, u, p); break;
            default: batch_unit<256, 64>(ba, c, stage, u, p); break;
        }
        __syncthreads();   // every thread's stores are issued; the slab is free
        if (tid == kThreads - 32) {   // publish this unit
            __threadfence();
            atomicAdd(ba.cnt + 3 * (size_t)(c.first + p) + stage, 1u);
        }
        if (tid == 0) {    // advance: unit i+1 becomes current
            g0 = g1;
            c0 = c1;
            g1 = g2;
            c1 = c2;
            g2 = g3;
            go0 = g0 < n;
            early = true;
        }
    }
}

// Shared memory of the kernel: the largest unit of any class it carries.
template <int N, int M> constexpr size_t batch_smem_nm() {
    return fast_xt_smem<N, M>() > fast_lines_smem<N, M>() ? fast_xt_smem<N, M>() : fast_lines_smem<N, M>();
}
constexpr size_t cmax(size_t a, size_t b) { return a > b ? a : b; }
constexpr size_t batch_persist_smem() {
    return cmax(cmax(cmax(batch_smem_nm<32, 16>(), batch_smem_nm<32, 32>()), cmax(batch_smem_nm<32, 64>(), batch_smem_nm<64, 16>())),
                cmax(cmax(cmax(batch_smem_nm<64, 32>(), batch_smem_nm<64, 64>()), cmax(batch_smem_nm<128, 16>(), batch_smem_nm<128, 32>())),
                     cmax(cmax(batch_smem_nm<128, 64>(), batch_smem_nm<256, 16>()), cmax(batch_smem_nm<256, 32>(), batch_smem_nm<256, 64>()))));
}

}  // namespace se2
