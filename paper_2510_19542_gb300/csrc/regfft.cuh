// Register-resident FFTs of compile-time length for the persistent frame kernel.
//
// A transform of length M = R1 * R2 (R1 = 2^floor(log2(M)/2), R2 = M/R1, so
// R2 is R1 or 2 R1) is computed by R1 threads in two steps (the "four-step"
// factorisation of the DFT):
//   step A: thread n1 holds x[n1 + R1 n2] (n2 < R2) in registers, takes the
//           R2-point DFT over n2, multiplies by W_M^(n1 k2) and writes
//           T[k2][n1] to shared memory;
//   step B: thread t takes the R1-point DFTs over n1 of the columns
//           k2 = t + c R1 (c < R2/R1), giving X[k2 + R2 k1] for k1 < R1.
// X[k2 + R2 k1] = sum_n1 W_R1^(n1 k1) W_M^(n1 k2) sum_n2 W_R2^(n2 k2) x[n1 + R1 n2].
// The small DFTs (N <= 32) are recursive radix-2 decimation in time, fully
// unrolled; their twiddles are the exact constants cos(pi m / 16).  The
// W_M^(n1 k2) twiddles come from a table built on the host in FP64.  T is
// padded (row stride R1 + 1) so both steps are free of bank conflicts.
#pragma once

#include <cuda_runtime.h>

namespace safr {

// cos(pi m / 16), m = 0..8
__host__ __device__ constexpr double cos_pi16(int m)
{
    return m == 0 ? 1.0
         : m == 1 ? 0.98078528040323044912618223613424
         : m == 2 ? 0.92387953251128675612818318939679
         : m == 3 ? 0.83146961230254523707878837761791
         : m == 4 ? 0.70710678118654752440084436210485
         : m == 5 ? 0.55557023301960222474283081394853
         : m == 6 ? 0.38268343236508977172845998403040
         : m == 7 ? 0.19509032201612826784828486847702
         : 0.0;
}

template <typename C>
__device__ __forceinline__ C c_add(C a, C b) { return C{a.x + b.x, a.y + b.y}; }
template <typename C>
__device__ __forceinline__ C c_sub(C a, C b) { return C{a.x - b.x, a.y - b.y}; }
template <typename C>
__device__ __forceinline__ C c_mul(C a, C b) { return C{a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x}; }
template <typename C>
__device__ __forceinline__ C c_mulc(C a, C b) { return C{a.x * b.x + a.y * b.y, a.y * b.x - a.x * b.y}; }  // a conj(b)

// v * W_N^k with W_N = exp(-2 pi i / N) (forward) or its conjugate (inverse), N <= 32
template <int N, int K, bool INV, typename C>
__device__ __forceinline__ C twiddle_const(C v)
{
    using R = decltype(v.x);
    constexpr int m = (32 / N) * K;  // angle 2 pi K / N = pi m / 16, 0 <= m < 16
    if constexpr (m == 0) {
        return v;
    } else if constexpr (m == 8) {  // -i (forward) / +i (inverse)
        return INV ? C{-v.y, v.x} : C{v.y, -v.x};
    } else {
        constexpr double cd = m <= 8 ? cos_pi16(m) : -cos_pi16(16 - m);
        constexpr double sd = m <= 8 ? cos_pi16(8 - m) : cos_pi16(m - 8);
        const R c = (R)cd, s = INV ? (R)sd : (R)(-sd);
        return C{v.x * c - v.y * s, v.x * s + v.y * c};
    }
}

template <int N, int K, bool INV, typename C>
__device__ __forceinline__ void dft_combine(C *v, const C *e, const C *o)
{
    if constexpr (K < N / 2) {
        const C t = twiddle_const<N, K, INV>(o[K]);
        v[K] = c_add(e[K], t);
        v[K + N / 2] = c_sub(e[K], t);
        dft_combine<N, K + 1, INV>(v, e, o);
    }
}

// In-register DFT of N points (N = 1, 2, 4, 8, 16, 32), natural order in and out.
template <int N, bool INV, typename C>
__device__ __forceinline__ void dft_reg(C *v)
{
    if constexpr (N == 2) {
        const C a = v[0];
        v[0] = c_add(a, v[1]);
        v[1] = c_sub(a, v[1]);
    } else if constexpr (N > 2) {
        C e[N / 2], o[N / 2];
#pragma unroll
        for (int i = 0; i < N / 2; ++i) {
            e[i] = v[2 * i];
            o[i] = v[2 * i + 1];
        }
        dft_reg<N / 2, INV>(e);
        dft_reg<N / 2, INV>(o);
        dft_combine<N, 0, INV>(v, e, o);
    }
}

constexpr int ilog2c(int n) { return n <= 1 ? 0 : 1 + ilog2c(n / 2); }

template <int M>
struct FftShape {
    static constexpr int LOG = ilog2c(M);
    static constexpr int R1 = 1 << (LOG / 2);  // threads per transform
    static constexpr int R2 = M / R1;          // points per thread in step A
    static constexpr int CB = R2 / R1;         // columns per thread in step B (1 or 2)
    // shared-memory words of one transform's transpose buffer, padded so that
    // neighbouring transforms in a half-warp start 16 banks apart
    static constexpr int TS_RAW = R2 * (R1 + 1);
    static constexpr int TS = R1 >= 16 ? TS_RAW : ((TS_RAW + 15) / 16) * 16 + 8;
};

// Step A of a length-M transform: v[n2] = x[t + R1 n2] on entry.
template <int M, bool INV, typename C>
__device__ __forceinline__ void fft_step_a(C *v, int t, C *T, const C *twq)
{
    using S = FftShape<M>;
    dft_reg<S::R2, INV>(v);
#pragma unroll
    for (int k2 = 0; k2 < S::R2; ++k2) {
        C y = v[k2];
        if (k2 > 0) {
            const C w = twq[k2 * S::R1 + t];
            y = INV ? c_mulc(y, w) : c_mul(y, w);
        }
        T[k2 * (S::R1 + 1) + t] = y;
    }
}

// Step B: out[c][k1] = X[(t + c R1) + R2 k1].
template <int M, bool INV, typename C>
__device__ __forceinline__ void fft_step_b(C (*out)[FftShape<M>::R1], int t, const C *T)
{
    using S = FftShape<M>;
#pragma unroll
    for (int c = 0; c < S::CB; ++c) {
        const int k2 = t + c * S::R1;
#pragma unroll
        for (int n1 = 0; n1 < S::R1; ++n1) out[c][n1] = T[k2 * (S::R1 + 1) + n1];
        dft_reg<S::R1, INV>(out[c]);
    }
}

// One length-M transform per group of R1 threads ("slot"), in place on
// shared memory: buf + slot * TS holds x[0..M) in natural order on entry and
// X[0..M) on return.  inv != 0 gives the unnormalised inverse through
// IDFT(x) = conj(DFT(conj(x))).  Slots >= nact only take part in the block
// barriers.  Not inlined: every phase of the frame kernel calls this one copy,
// which keeps the kernel's instruction footprint small.
template <int M, typename C>
__device__ __noinline__ void fft_core(C *buf, int nact, int inv, const C *twq)
{
    using S = FftShape<M>;
    const int slot = threadIdx.x / S::R1, t = threadIdx.x % S::R1;
    const bool act = slot < nact;
    C *x = buf + (size_t)slot * S::TS;
    C v[S::R2];
    if (act) {
#pragma unroll
        for (int n2 = 0; n2 < S::R2; ++n2) {
            v[n2] = x[t + S::R1 * n2];
            if (inv) v[n2].y = -v[n2].y;
        }
    }
    __syncthreads();
    if (act) {
        dft_reg<S::R2, false>(v);
#pragma unroll
        for (int k2 = 0; k2 < S::R2; ++k2) {
            C y = v[k2];
            if (k2 > 0) y = c_mul(y, twq[k2 * S::R1 + t]);
            x[k2 * (S::R1 + 1) + t] = y;
        }
    }
    __syncthreads();
    C out[S::CB][S::R1];
    if (act) {
#pragma unroll
        for (int c = 0; c < S::CB; ++c) {
            const int k2 = t + c * S::R1;
#pragma unroll
            for (int n1 = 0; n1 < S::R1; ++n1) out[c][n1] = x[k2 * (S::R1 + 1) + n1];
            dft_reg<S::R1, false>(out[c]);
        }
    }
    __syncthreads();
    if (act) {
#pragma unroll
        for (int c = 0; c < S::CB; ++c)
#pragma unroll
            for (int k1 = 0; k1 < S::R1; ++k1) {
                C o = out[c][k1];
                if (inv) o.y = -o.y;
                x[t + c * S::R1 + S::R2 * k1] = o;
            }
    }
    __syncthreads();
}

}  // namespace safr
