// Device building blocks for the batched power-of-two FFTs of the SE(2)
// convolution path: in-register radix-2 DFTs of up to 32 points, and a
// two-step ("four-step") line FFT executed by a team of threads that swaps
// partial results through shared memory.
//
// Conventions: DIR = -1 is the forward transform e^{-2 pi i n k / L}
// (Eq. 3DFT), DIR = +1 the unscaled inverse (Eq. 3iDFT without 1/L).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace se2 {

template <typename T> struct C2;
template <> struct C2<float> { using t = float2; };
template <> struct C2<double> { using t = double2; };
template <typename T> using c2 = typename C2<T>::t;

template <typename T> __device__ __forceinline__ c2<T> mk(T x, T y) { c2<T> v; v.x = x; v.y = y; return v; }

// cos(pi q / 16) for q in [0, 8]; other q by symmetry.
__host__ __device__ constexpr double cos_pi16_tab(int q) {
    return q == 0 ? 1.0
         : q == 1 ? 0.9807852804032304491262
         : q == 2 ? 0.9238795325112867561282
         : q == 3 ? 0.8314696123025452370788
         : q == 4 ? 0.7071067811865475244008
         : q == 5 ? 0.5555702330196022247428
         : q == 6 ? 0.3826834323650897717285
         : q == 7 ? 0.1950903220161282678483
         : 0.0;
}
__host__ __device__ constexpr double cpi16(int q) {
    q = ((q % 32) + 32) % 32;
    if (q > 16) q = 32 - q;             // cos is even about 2 pi
    return q <= 8 ? cos_pi16_tab(q) : -cos_pi16_tab(16 - q);
}
__host__ __device__ constexpr double spi16(int q) { return cpi16(q - 8); }  // sin x = cos(x - pi/2)

// (re, im) *= exp(DIR * i * pi * q / 16), q a compile-time-foldable integer.
template <int DIR, typename T>
__device__ __forceinline__ void rot16(int q, T& re, T& im) {
    if (q == 0) return;
    if (q == 8) { const T t = re; re = (T)(-DIR) * im; im = (T)DIR * t; return; }
    const T c = (T)cpi16(q), s = (T)(DIR * spi16(q));
    const T r = re * c - im * s;
    im = re * s + im * c;
    re = r;
}

template <int R> __device__ __forceinline__ constexpr int bitrev(int i) {
    int r = 0;
    for (int b = 1, rb = R >> 1; b < R; b <<= 1, rb >>= 1) if (i & b) r |= rb;
    return r;
}

// In-register DFT of R <= 32 points: radix-2 decimation in frequency, then a
// compile-time register permutation back to natural order.
template <int R, int DIR, typename T>
__device__ __forceinline__ void fft_reg(T* re, T* im) {
    if constexpr (R > 1) {
#pragma unroll
        for (int half = R / 2; half >= 1; half >>= 1) {
#pragma unroll
            for (int base = 0; base < R; base += 2 * half) {
#pragma unroll
                for (int j = 0; j < half; ++j) {
                    const int a = base + j, b = a + half;
                    const T ar = re[a], ai = im[a], br = re[b], bi = im[b];
                    re[a] = ar + br;
                    im[a] = ai + bi;
                    T dr = ar - br, di = ai - bi;
                    rot16<DIR>(j * (16 / half), dr, di);   // e^{DIR 2 pi i j / (2 half)}
                    re[b] = dr;
                    im[b] = di;
                }
            }
        }
        T tr[R], ti[R];
#pragma unroll
        for (int i = 0; i < R; ++i) { tr[i] = re[i]; ti[i] = im[i]; }
#pragma unroll
        for (int i = 0; i < R; ++i) { re[i] = tr[bitrev<R>(i)]; im[i] = ti[bitrev<R>(i)]; }
    }
}

// L = R1 * R2 factorisation used by the team FFT.
template <int L> struct Fac;
template <> struct Fac<2>   { static constexpr int R1 = 2,  R2 = 1; };
template <> struct Fac<4>   { static constexpr int R1 = 4,  R2 = 1; };
template <> struct Fac<8>   { static constexpr int R1 = 8,  R2 = 1; };
template <> struct Fac<16>  { static constexpr int R1 = 16, R2 = 1; };
template <> struct Fac<32>  { static constexpr int R1 = 8,  R2 = 4; };
template <> struct Fac<64>  { static constexpr int R1 = 8,  R2 = 8; };
template <> struct Fac<128> { static constexpr int R1 = 16, R2 = 8; };
template <> struct Fac<256> { static constexpr int R1 = 16, R2 = 16; };
template <> struct Fac<512> { static constexpr int R1 = 32, R2 = 16; };
// Lanes per line: one lane holds a whole line when R2 == 1.
template <int L> __host__ __device__ constexpr int team_size() {
    return Fac<L>::R2 == 1 ? 1 : (Fac<L>::R1 > Fac<L>::R2 ? Fac<L>::R1 : Fac<L>::R2);
}
template <int L> __host__ __device__ constexpr int reg_count() { return Fac<L>::R1 > Fac<L>::R2 ? Fac<L>::R1 : Fac<L>::R2; }
// Exchange buffer (complex elements) one team needs: R1 rows of pitch R2+1,
// at least L for linear scratch, plus one so that consecutive buffers start
// in different banks.
template <int L> __host__ __device__ constexpr int xbuf_elems() {
    return (Fac<L>::R1 * (Fac<L>::R2 + 1) > L ? Fac<L>::R1 * (Fac<L>::R2 + 1) : L) + 1;
}

// Multiply by the twiddle e^{DIR 2 pi i n / L} from the forward table
// tw[n] = e^{-2 pi i n / L} (conjugated for the inverse).
template <int DIR, typename T>
__device__ __forceinline__ void twid(const c2<T>* __restrict__ tw, int n, T& re, T& im) {
    const c2<T> w = tw[n];
    const T wr = w.x, wi = (DIR < 0) ? w.y : -w.y;
    const T r = re * wr - im * wi;
    im = re * wi + im * wr;
    re = r;
}

// Where team_fft leaves its output: lane s < lanes holds X[idx(s, k)] in
// register k < regs.  With R2 == 1 a single lane holds everything.
template <int R1, int R2> struct TeamOut {
    static constexpr int lanes = (R2 > 1) ? R1 : 1;
    static constexpr int regs = (R2 > 1) ? R2 : R1;
    __device__ __forceinline__ static constexpr int idx(int lane, int k) { return (R2 > 1) ? lane + R1 * k : k; }
};

struct SyncWarp  { __device__ __forceinline__ void operator()() const { __syncwarp(); } };
struct SyncBlock { __device__ __forceinline__ void operator()() const { __syncthreads(); } };

// Team FFT of length L = R1 * R2.
//  in : lane t < R2 holds x[t + R2 j], j < R1, in re/im[0..R1)
//  out: lane s < R1 holds X[s + R1 k], k < R2, in re/im[0..R2)
// Every lane of the team must call it (it synchronises twice through `sync`).
// xb is the team's exchange buffer (R1 rows of pitch R2 + 1).
template <int R1, int R2, int DIR, typename T, typename Sync>
__device__ __forceinline__ void team_fft(T* re, T* im, int lane, c2<T>* xb,
                                         const c2<T>* __restrict__ tw, Sync sync) {
    if constexpr (R2 == 1) {
        fft_reg<R1, DIR>(re, im);
    } else {
        if (lane < R2) {
            fft_reg<R1, DIR>(re, im);
#pragma unroll
            for (int k1 = 1; k1 < R1; ++k1) twid<DIR, T>(tw, lane * k1, re[k1], im[k1]);
#pragma unroll
            for (int k1 = 0; k1 < R1; ++k1) xb[k1 * (R2 + 1) + lane] = mk<T>(re[k1], im[k1]);
        }
        sync();
        if (lane < R1) {
#pragma unroll
            for (int t = 0; t < R2; ++t) {
                const c2<T> v = xb[lane * (R2 + 1) + t];
                re[t] = v.x;
                im[t] = v.y;
            }
            fft_reg<R2, DIR>(re, im);
        }
        sync();
    }
}

// Same as team_fft, with this lane's step-A twiddles e^{DIR 2 pi i lane k / L}
// (k < R1) already in registers (wr, wi), so loops over several lines do not
// reload them.
template <int R1, int R2, int DIR, typename T, typename Sync>
__device__ __forceinline__ void team_fft_r(T* re, T* im, int lane, c2<T>* xb,
                                           const T* wr, const T* wi, Sync sync) {
    if constexpr (R2 == 1) {
        fft_reg<R1, DIR>(re, im);
    } else {
        if (lane < R2) {
            fft_reg<R1, DIR>(re, im);
#pragma unroll
            for (int k1 = 1; k1 < R1; ++k1) {
                const T r = re[k1] * wr[k1] - im[k1] * wi[k1];
                im[k1] = re[k1] * wi[k1] + im[k1] * wr[k1];
                re[k1] = r;
            }
#pragma unroll
            for (int k1 = 0; k1 < R1; ++k1) xb[k1 * (R2 + 1) + lane] = mk<T>(re[k1], im[k1]);
        }
        sync();
        if (lane < R1) {
#pragma unroll
            for (int t = 0; t < R2; ++t) {
                const c2<T> v = xb[lane * (R2 + 1) + t];
                re[t] = v.x;
                im[t] = v.y;
            }
            fft_reg<R2, DIR>(re, im);
        }
        sync();
    }
}

// Load this lane's step-A twiddles for a length-L team FFT.
template <int L, int DIR, typename T>
__device__ __forceinline__ void load_twiddles(const c2<T>* __restrict__ tw, int lane, T* wr, T* wi) {
    constexpr int R1 = Fac<L>::R1, R2 = Fac<L>::R2;
    const int l = lane < R2 ? lane : 0;
#pragma unroll
    for (int k = 0; k < R1; ++k) {
        const c2<T> w = tw[(l * k) % L];
        wr[k] = w.x;
        wi[k] = (DIR < 0) ? w.y : -w.y;
    }
}

// Row offset (complex elements) of row r in a column-transformed slab of pitch
// SP: rows are shifted by 2 elements per group of R1 rows, so that the strided
// row accesses of column_fft fall in distinct shared-memory banks.
template <int L> __host__ __device__ constexpr int row_group() { return Fac<L>::R2 == 1 ? (1 << 30) : Fac<L>::R1; }
template <int L, int SP> __device__ __forceinline__ constexpr int rowoff(int r) { return r * SP + (r / row_group<L>()) * 2; }
template <int L, int SP> __host__ __device__ constexpr int slab_elems() { return L * SP + (L / row_group<L>() + 1) * 2; }

// In-place FFT of the column c of an L-row slab in shared memory (row r at
// rowoff<L, SP>(r) + c), natural order in and out, by a team of
// team_size<L>() lanes with their step-A twiddles in (wr, wi).  Step A places
// A[t][k1] at row k1 + R1 t, step B reads rows s + R1 t and writes X[s + R1 k]
// back to the same rows.  `act` = false lanes only synchronise.
template <int L, int SP, int DIR, typename T, typename Sync>
__device__ __forceinline__ void column_fft_r(c2<T>* S, int c, int lane, bool act,
                                             const T* wr, const T* wi, Sync sync) {
    constexpr int R1 = Fac<L>::R1, R2 = Fac<L>::R2, RM = reg_count<L>();
    T re[RM], im[RM];
    if constexpr (R2 == 1) {
        if (act) {
#pragma unroll
            for (int r = 0; r < L; ++r) { const c2<T> v = S[rowoff<L, SP>(r) + c]; re[r] = v.x; im[r] = v.y; }
            fft_reg<L, DIR>(re, im);
#pragma unroll
            for (int r = 0; r < L; ++r) S[rowoff<L, SP>(r) + c] = mk<T>(re[r], im[r]);
        }
    } else {
        if (act && lane < R2) {
#pragma unroll
            for (int j = 0; j < R1; ++j) { const c2<T> v = S[rowoff<L, SP>(lane + R2 * j) + c]; re[j] = v.x; im[j] = v.y; }
            fft_reg<R1, DIR>(re, im);
#pragma unroll
            for (int k1 = 1; k1 < R1; ++k1) {
                const T r = re[k1] * wr[k1] - im[k1] * wi[k1];
                im[k1] = re[k1] * wi[k1] + im[k1] * wr[k1];
                re[k1] = r;
            }
        }
        sync();     // every step-A load is done before any step-A store
        if (act && lane < R2) {
#pragma unroll
            for (int k1 = 0; k1 < R1; ++k1) S[rowoff<L, SP>(k1 + R1 * lane) + c] = mk<T>(re[k1], im[k1]);
        }
        sync();
        if (act && lane < R1) {
#pragma unroll
            for (int t = 0; t < R2; ++t) { const c2<T> v = S[rowoff<L, SP>(lane + R1 * t) + c]; re[t] = v.x; im[t] = v.y; }
            fft_reg<R2, DIR>(re, im);
#pragma unroll
            for (int k = 0; k < R2; ++k) S[rowoff<L, SP>(lane + R1 * k) + c] = mk<T>(re[k], im[k]);
        }
    }
}

// In-place FFT of a strided column of L complex values in shared memory,
// col[r * pitch], r < L, by a team of team_size<L>() lanes (natural order in
// and out).  `act` = false lanes only take part in the synchronisation.
template <int L, int DIR, typename T, typename Sync>
__device__ __forceinline__ void column_fft(c2<T>* col, int pitch, int lane, bool act,
                                           const c2<T>* __restrict__ tw, Sync sync) {
    constexpr int R1 = Fac<L>::R1, R2 = Fac<L>::R2, RM = reg_count<L>();
    T re[RM], im[RM];
    if constexpr (R2 == 1) {
        if (act) {
#pragma unroll
            for (int r = 0; r < L; ++r) { const c2<T> v = col[r * pitch]; re[r] = v.x; im[r] = v.y; }
            fft_reg<L, DIR>(re, im);
#pragma unroll
            for (int r = 0; r < L; ++r) col[r * pitch] = mk<T>(re[r], im[r]);
        }
    } else {
        if (act && lane < R2) {
#pragma unroll
            for (int j = 0; j < R1; ++j) { const c2<T> v = col[(lane + R2 * j) * pitch]; re[j] = v.x; im[j] = v.y; }
            fft_reg<R1, DIR>(re, im);
#pragma unroll
            for (int k1 = 1; k1 < R1; ++k1) twid<DIR, T>(tw, lane * k1, re[k1], im[k1]);
#pragma unroll
            for (int k1 = 0; k1 < R1; ++k1) col[(lane + R2 * k1) * pitch] = mk<T>(re[k1], im[k1]);
        }
        sync();
        if (act && lane < R1) {
#pragma unroll
            for (int t = 0; t < R2; ++t) { const c2<T> v = col[(R2 * lane + t) * pitch]; re[t] = v.x; im[t] = v.y; }
            fft_reg<R2, DIR>(re, im);
        }
        sync();
        if (act && lane < R1) {
#pragma unroll
            for (int k = 0; k < R2; ++k) col[(lane + R1 * k) * pitch] = mk<T>(re[k], im[k]);
        }
    }
}

}  // namespace se2
