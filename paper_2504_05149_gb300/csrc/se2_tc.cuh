// Angular DFT on the 5th-generation tensor cores (tcgen05), for the mixed
// precision mode of the split pass structure.
//
// For a tile of 128 (y, x-bin) lines of the scratch spectrum, the length-M
// DFT along theta is a dense real contraction: with the real form of the
// DFT matrix B (row n = 2m + {re, im} of the output bin m, column k =
// 2l + {re, im} of the input sample l),
//     D[line][n] = sum_k A[line][k] B[n][k],   A[line][2l + b] = x_l (re/im).
// A (the data) and B are staged in shared memory as bf16 in the K-major
// no-swizzle core-matrix layout, the products run as tcgen05.mma kind::f16
// (M = 128 lines, N = 128, K = 16 per instruction) into an FP32 accumulator
// in tensor memory, and each warp reads its 32 lines back with tcgen05.ld.
// Split precision: x = x_hi + x_lo and B = B_hi + B_lo in bf16, and
// D = A_hi B_hi + A_hi B_lo + A_lo B_hi (the lo*lo term is below FP32
// rounding of the accumulation), which keeps about 16 significant bits.
// The FP16 variant (FMT = 1) splits into fp16 halves instead (about 22
// significant bits).  fp16 has a narrow exponent range, so every line is
// scaled by a power of two that puts its largest sample in [2^13, 2^14)
// before the split, and its outputs are scaled back (exactly) after.
// M = 64 is one contraction; M = 128 splits even and odd samples into two
// 64-point contractions and combines them with the radix-2 butterfly
// Y[m] = E[m] + w^m O[m], Y[m + 64] = E[m] - w^m O[m] in FP32.
#pragma once
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "se2_kernels.cuh"

namespace se2 {

constexpr int kTcLines = 128;            // lines per tile (tensor-memory lanes)
constexpr int kTcThreads = 256;          // two threads per line
constexpr int kTcK = 128;                // K of one contraction (64 complex samples)
constexpr int kTcOpBytes = kTcLines * kTcK * 2;   // one 16-bit operand: 32 KB

// byte offset of element (row r, k) of a K-major no-swizzle bf16 operand with
// K = kTcK: 8x8 core matrices (8 rows x 16 bytes), K-adjacent core matrices
// 128 bytes apart (LBO), 8-row groups (K/8)*128 bytes apart (SBO).
__host__ __device__ constexpr int tc_off(int r, int k) {
    return (r / 8) * (kTcK / 8) * 128 + (k / 8) * 128 + (r % 8) * 16 + (k % 8) * 2;
}

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// Shared-memory matrix descriptor (sm_100 format): start >> 4, LBO >> 4,
// SBO >> 4, version 1, no swizzle.
__device__ __forceinline__ uint64_t tc_desc(const void* p) {
    uint64_t d = 0;
    d |= (uint64_t)((smem_u32(p) >> 4) & 0x3FFF);
    d |= (uint64_t)((128u >> 4) & 0x3FFF) << 16;
    d |= (uint64_t)(((kTcK / 8) * 128u >> 4) & 0x3FFF) << 32;
    d |= (uint64_t)1 << 46;
    return d;
}
// Instruction descriptor: kind::f16, D = f32, both K-major; A and B share
// one type: bf16 (fmt 0, type code 1) or fp16 (fmt 1, type code 0).
__host__ __device__ constexpr uint32_t tc_idesc(int M, int N, int fmt) {
    return (1u << 4) | (fmt == 0 ? ((1u << 7) | (1u << 10)) : 0u) | ((uint32_t)(N >> 3) << 17) |
           ((uint32_t)(M >> 4) << 24);
}

template <int FMT>
__device__ __forceinline__ void tc_mma(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t acc) {
    asm volatile("{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
                 "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}"
                 :: "r"(d_tmem), "l"(a), "l"(b), "r"(tc_idesc(kTcLines, kTcK, FMT)), "r"(acc));
}

// 32 consecutive FP32 columns of this warp's 32 lanes.
__device__ __forceinline__ void tc_ld32(uint32_t taddr, float* v) {
    uint32_t r[32];
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
                 "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
                   "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
                   "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
                   "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
                 : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int j = 0; j < 32; ++j) v[j] = __uint_as_float(r[j]);
}

struct TcArgs {
    float2* s;                 // scratch spectrum base
    size_t s_pstride;          // complex elements per problem
    int N, tp;                 // grid size, scratch row pitch
    const uint4* bmat;         // B_hi then B_lo (kTcOpBytes each) for this direction
    const float2* tw;          // e^{-2 pi i m / 128}, m < 128 (M = 128 only)
    int* err;                  // set to 2 when a wait for the tensor cores gives up
};

// Split x into 16-bit hi + lo (bf16 for FMT 0, fp16 for FMT 1), as the raw bits.
template <int FMT>
__device__ __forceinline__ void split16(float x, uint32_t& hi, uint32_t& lo) {
    if constexpr (FMT == 0) {
        const __nv_bfloat16 h = __float2bfloat16_rn(x);
        hi = __bfloat16_as_ushort(h);
        lo = __bfloat16_as_ushort(__float2bfloat16_rn(x - __bfloat162float(h)));
    } else {
        const __half h = __float2half_rn(x);
        hi = __half_as_ushort(h);
        lo = __half_as_ushort(__float2half_rn(x - __half2float(h)));
    }
}

template <int M, int DIR, int SPLIT, int FMT>
__global__ void __launch_bounds__(kTcThreads, 1) k_theta_tc(TcArgs a) {
    static_assert(M == 64 || M == 128, "tensor-core angular DFT: M = 64 or 128");
    constexpr int NPART = (M == 128) ? 2 : 1;              // even / odd contractions
    constexpr int NLO = (SPLIT == 3) ? 1 : 0;
    extern __shared__ __align__(1024) unsigned char smem[];
    unsigned char* sB = smem;                              // B_hi [, B_lo]
    unsigned char* sA = smem + (1 + NLO) * kTcOpBytes;     // per part: A_hi [, A_lo]
    __shared__ uint32_t tmem_base;
    __shared__ __align__(8) uint64_t mbar;
    __shared__ float lmax[kTcThreads];       // FMT 1: per-thread maxima, then per-line scales
    __shared__ float lscale[kTcLines];
    const int tid = threadIdx.x, warp = tid >> 5;
    const int row = tid % kTcLines, half = tid / kTcLines;   // line of the tile, which half of it
    const int b = blockIdx.y;
    const int H = a.N / 2 + 1;
    const long long nlines = (long long)a.N * H;
    const int ntiles = (int)((nlines + kTcLines - 1) / kTcLines);
    float2* sp = a.s + b * a.s_pstride;

    // constant operand B (linear copy: the global array is already in the layout)
    {
        const uint4* src = a.bmat;
        uint4* dst = reinterpret_cast<uint4*>(sB);
        for (int i = tid; i < (1 + NLO) * kTcOpBytes / 16; i += kTcThreads) dst[i] = src[i];
    }
    if (tid == 0) asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(smem_u32(&mbar)));
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                     :: "r"(smem_u32(&tmem_base)), "n"(128 * NPART));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = tmem_base;
    bool ok = true;
    uint32_t phase = 0;

    for (int tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x) {
        const long long line = (long long)tile * kTcLines + row;
        const bool act = line < nlines;
        const int y = act ? (int)(line / H) : 0;
        const int kx = act ? (int)(line - (long long)y * H) : 0;
        float2* base = sp + (size_t)y * a.tp + kx;          // sample l at base + l * N * tp
        const size_t ls = (size_t)a.N * a.tp;
        // 1. this thread's half of its line -> A rows (8 bf16 = 4 samples per
        //    16-byte store); 16 loads in flight per batch.  M = 128: half =
        //    even / odd samples (the two contractions); M = 64: half = samples
        //    [0, 32) / [32, 64) of the one contraction.
        {
            const int part = (NPART == 2) ? half : 0;
            const int lbeg = (NPART == 2) ? 0 : 32 * half;
            unsigned char* Ahi = sA + part * (1 + NLO) * kTcOpBytes;
            unsigned char* Alo = Ahi + kTcOpBytes;
            constexpr int lcount = (NPART == 2) ? 64 : 32;   // samples of this thread
            float sc = 1.f;
            if constexpr (FMT == 1) {
                // the line's largest |re|, |im| over both threads' samples
                float mx = 0.f;
#pragma unroll 1
                for (int l0 = lbeg; l0 < lbeg + lcount; l0 += 16) {
#pragma unroll
                    for (int q = 0; q < 16; ++q) {
                        const int l = (l0 + q) * NPART + part;
                        const float2 w = act ? __ldcg(base + (size_t)l * ls) : make_float2(0.f, 0.f);
                        mx = fmaxf(mx, fmaxf(fabsf(w.x), fabsf(w.y)));
                    }
                }
                lmax[tid] = mx;
                __syncthreads();
                const float lm = fmaxf(lmax[row], lmax[row + kTcLines]);
                int ex = 0;
                if (lm > 0.f && lm <= 3.0e38f) frexpf(lm, &ex);     // lm = f 2^ex, f in [0.5, 1)
                // 2^e and 2^-e stay finite normal floats (subnormal lines are
                // scaled by 2^126 only; what stays below fp16's range is lost)
                const int e = lm > 0.f ? min(max(14 - ex, -126), 126) : 0;
                sc = ldexpf(1.f, e);
                if (half == 0) lscale[row] = ldexpf(1.f, -e);
            }
#pragma unroll 1
            for (int l0 = lbeg; l0 < lbeg + lcount; l0 += 16) {
                float2 v[16];
#pragma unroll
                for (int q = 0; q < 16; ++q) {
                    const int l = (l0 + q) * NPART + part;      // sample index
                    v[q] = act ? __ldcg(base + (size_t)l * ls) : make_float2(0.f, 0.f);
                }
#pragma unroll
                for (int g = 0; g < 4; ++g) {
                    uint32_t h[4], o[4];
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        uint32_t hr, lr, hi_, li;
                        split16<FMT>(v[4 * g + q].x * sc, hr, lr);
                        split16<FMT>(v[4 * g + q].y * sc, hi_, li);
                        // (re, im) -> one 32-bit word, re in the low half (lower address)
                        h[q] = hr | (hi_ << 16);
                        o[q] = lr | (li << 16);
                    }
                    const int off = tc_off(row, 2 * (l0 + 4 * g));
                    *reinterpret_cast<uint4*>(Ahi + off) = make_uint4(h[0], h[1], h[2], h[3]);
                    if (NLO) *reinterpret_cast<uint4*>(Alo + off) = make_uint4(o[0], o[1], o[2], o[3]);
                }
            }
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncthreads();
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        // 2. one thread issues the contractions
        if (tid == 0) {
#pragma unroll 1
            for (int part = 0; part < NPART; ++part) {
                const unsigned char* Ahi = sA + part * (1 + NLO) * kTcOpBytes;
                const unsigned char* Alo = Ahi + kTcOpBytes;
                const uint32_t d = tmem + 128 * part;
#pragma unroll 1
                for (int kk = 0; kk < kTcK / 16; ++kk) {
                    const int ko = kk * 256;                     // 16 K elements = 2 core matrices
                    tc_mma<FMT>(d, tc_desc(Ahi + ko), tc_desc(sB + ko), kk > 0 ? 1u : 0u);
                    if (NLO) {
                        tc_mma<FMT>(d, tc_desc(Ahi + ko), tc_desc(sB + kTcOpBytes + ko), 1u);
                        tc_mma<FMT>(d, tc_desc(Alo + ko), tc_desc(sB + ko), 1u);
                    }
                }
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                         :: "r"(smem_u32(&mbar)) : "memory");
        }
        // 3. bounded wait for the tensor cores
        uint32_t done = 0;
        for (long it = 0; it < (1L << 22) && !done; ++it) {
            asm volatile("{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}"
                         : "=r"(done) : "r"(smem_u32(&mbar)), "r"(phase) : "memory");
        }
        phase ^= 1u;
        ok = __syncthreads_and((int)done) != 0;      // one decision for the whole block
        if (!ok) {
            // the block leaves the tile loop: no further operand writes or MMAs;
            // one more bounded wait lets the MMAs in flight finish before the
            // tensor memory is released
            if (tid == 0) atomicExch(a.err, 2);
            uint32_t late = done;
            for (long it = 0; it < (1L << 22) && !late; ++it) {
                asm volatile("{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}"
                             : "=r"(late) : "r"(smem_u32(&mbar)), "r"(phase ^ 1u) : "memory");
            }
            break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        // 4. read the lines back and write them in place: warps w and w + 4
        //    share the lanes 32 (w % 4) .. +31 and take columns [0, 64) and
        //    [64, 128) (output bins [0, 32) and [32, 64) of each contraction)
        if (ok) {
            const uint32_t lane_base = tmem + ((uint32_t)(32 * (warp & 3)) << 16);
            const int cbeg = 64 * half;
            // this lane's line (tensor-memory lane) and its scale back
            const float us = FMT == 1 ? lscale[32 * (warp & 3) + (tid & 31)] : 1.f;
            if constexpr (M == 64) {
#pragma unroll 1
                for (int c0 = cbeg; c0 < cbeg + 64; c0 += 32) {
                    float v[32];
                    tc_ld32(lane_base + c0, v);
                    if (act) {
#pragma unroll
                        for (int q = 0; q < 16; ++q)
                            base[(size_t)(c0 / 2 + q) * ls] = make_float2(v[2 * q] * us, v[2 * q + 1] * us);
                    }
                }
            } else {
#pragma unroll 1
                for (int c0 = cbeg; c0 < cbeg + 64; c0 += 32) {
                    float e[32], o[32];
                    tc_ld32(lane_base + c0, e);
                    tc_ld32(lane_base + 128 + c0, o);
                    if (act) {
#pragma unroll
                        for (int q = 0; q < 16; ++q) {
                            const int m = c0 / 2 + q;
                            const float2 w = a.tw[m];
                            const float wr = w.x, wi = (DIR < 0) ? w.y : -w.y;
                            const float orr = o[2 * q] * wr - o[2 * q + 1] * wi;
                            const float oi = o[2 * q] * wi + o[2 * q + 1] * wr;
                            base[(size_t)m * ls] = make_float2((e[2 * q] + orr) * us, (e[2 * q + 1] + oi) * us);
                            base[(size_t)(m + 64) * ls] = make_float2((e[2 * q] - orr) * us, (e[2 * q + 1] - oi) * us);
                        }
                    }
                }
            }
        }
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncthreads();                 // A is rewritten by the next tile
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" :: "r"(tmem), "n"(128 * NPART));
}

template <int M, int SPLIT>
constexpr size_t tc_smem() {
    return (size_t)((SPLIT == 3 ? 2 : 1) * (1 + (M == 128 ? 2 : 1))) * kTcOpBytes;
}

}  // namespace se2
