// Shared-memory Stockham FFT for the SAFR frame kernels.
//
// DFT2 of Section 3.2 is separable: the frame kernels run it as 1-D
// transforms of length M (a power of two) along rows and then columns.  A
// transform of length M is a sequence of radix-8 / radix-4 passes in the
// Stockham autosort form (each pass reads with stride M/R, applies the
// twiddles W_{Ns R}^{r k}, does an R-point DFT in registers and writes with
// stride Ns), ping-ponging between two shared-memory buffers, so the result
// comes out in natural order without a bit-reversal pass.  Twiddles come
// from a table exp(-2 pi i t / M) computed on the host in FP64.
#pragma once

#include <cuda_runtime.h>

namespace safr {

template <typename C>
__device__ __forceinline__ C cadd(C a, C b) { return C{a.x + b.x, a.y + b.y}; }
template <typename C>
__device__ __forceinline__ C csub(C a, C b) { return C{a.x - b.x, a.y - b.y}; }
template <typename C>
__device__ __forceinline__ C cmul(C a, C b) { return C{a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x}; }
template <typename C>
__device__ __forceinline__ C cconj(C a) { return C{a.x, -a.y}; }
// multiply by -i (forward) or +i (inverse)
template <bool INV, typename C>
__device__ __forceinline__ C mul_mi(C a) { return INV ? C{-a.y, a.x} : C{a.y, -a.x}; }

template <bool INV, typename C>
__device__ __forceinline__ void dft4(C &v0, C &v1, C &v2, C &v3)
{
    C a0 = cadd(v0, v2), a1 = csub(v0, v2), a2 = cadd(v1, v3), a3 = mul_mi<INV>(csub(v1, v3));
    v0 = cadd(a0, a2);
    v2 = csub(a0, a2);
    v1 = cadd(a1, a3);
    v3 = csub(a1, a3);
}

// v * exp(-+ 2 pi i m / 8), m = 1, 3
template <int m, bool INV, typename C>
__device__ __forceinline__ C mul_w8(C v)
{
    using R = decltype(v.x);
    const R h = R(0.70710678118654752440);
    if (m == 1)
        return INV ? C{h * (v.x - v.y), h * (v.x + v.y)} : C{h * (v.x + v.y), h * (v.y - v.x)};
    else
        return INV ? C{-h * (v.x + v.y), h * (v.x - v.y)} : C{h * (v.y - v.x), -h * (v.x + v.y)};
}

template <bool INV, typename C>
__device__ __forceinline__ void dft8(C *v)
{
    // even / odd halves, then combine with the eighth roots of unity
    dft4<INV>(v[0], v[2], v[4], v[6]);
    dft4<INV>(v[1], v[3], v[5], v[7]);
    C o0 = v[1], o1 = mul_w8<1, INV>(v[3]), o2 = mul_mi<INV>(v[5]), o3 = mul_w8<3, INV>(v[7]);
    C e0 = v[0], e1 = v[2], e2 = v[4], e3 = v[6];
    v[0] = cadd(e0, o0); v[4] = csub(e0, o0);
    v[1] = cadd(e1, o1); v[5] = csub(e1, o1);
    v[2] = cadd(e2, o2); v[6] = csub(e2, o2);
    v[3] = cadd(e3, o3); v[7] = csub(e3, o3);
}

template <int RADIX, bool INV, typename C>
__device__ __forceinline__ void dft_radix(C *v)
{
    if constexpr (RADIX == 2) {
        C a = v[0];
        v[0] = cadd(a, v[1]);
        v[1] = csub(a, v[1]);
    } else if constexpr (RADIX == 4) {
        dft4<INV>(v[0], v[1], v[2], v[3]);
    } else {
        dft8<INV>(v);
    }
}

// One Stockham pass over `nfft` sequences of length M (sequence f starts at
// f * fstride in both buffers).  Ns is the length of the sub-transforms
// already done (1 for the first pass).
template <int RADIX, bool INV, typename C>
__device__ __forceinline__ void stockham_pass(const C *__restrict__ src, C *__restrict__ dst, int logM,
                                              int logNs, int nfft, int fstride, const C *__restrict__ tw,
                                              int tid, int nth)
{
    constexpr int LR = RADIX == 8 ? 3 : (RADIX == 4 ? 2 : 1);
    const int lognb = logM - LR;           // butterflies per sequence: M / RADIX
    const int nb = 1 << lognb;
    const int Ns = 1 << logNs;
    const int ltstep = logM - logNs - LR;  // twiddle stride M / (Ns RADIX)
    for (int idx = tid; idx < (nfft << lognb); idx += nth) {
        const int f = idx >> lognb, j = idx & (nb - 1);
        const C *s = src + f * fstride;
        C *d = dst + f * fstride;
        C v[RADIX];
#pragma unroll
        for (int r = 0; r < RADIX; ++r) v[r] = s[j + r * nb];
        const int k = j & (Ns - 1);
        if (Ns > 1) {
#pragma unroll
            for (int r = 1; r < RADIX; ++r) {
                C w = tw[(r * k) << ltstep];
                v[r] = cmul(v[r], INV ? cconj(w) : w);
            }
        }
        dft_radix<RADIX, INV>(v);
        const int base = ((j - k) << LR) + k;
#pragma unroll
        for (int r = 0; r < RADIX; ++r) d[base + r * Ns] = v[r];
    }
}

// Radix of pass `pass` for M = 2^logM: radix-8 passes, with one or two
// radix-4 passes when logM is not a multiple of three (8 = 8, 16 = 4.4,
// 32 = 4.8, 64 = 8.8, 128 = 4.4.8, 256 = 4.8.8, 512 = 8.8.8, 1024 = 4.4.8.8).
__host__ __device__ inline int fft_num_passes(int logM)
{
    int r = logM % 3;
    return r == 0 ? logM / 3 : (r == 2 ? logM / 3 + 1 : (logM - 4) / 3 + 2);
}
__host__ __device__ inline int fft_radix(int logM, int pass)
{
    int r = logM % 3;
    int n4 = r == 0 ? 0 : (r == 2 ? 1 : 2);
    return pass < n4 ? 4 : 8;
}

// Length-M transforms of `nfft` sequences held in `a`; `b` is scratch of the
// same size.  Returns the buffer that holds the result.  All threads of the
// block must call it; it synchronises the block between passes and before
// returning.
template <bool INV, typename C>
__device__ C *block_fft(C *a, C *b, int logM, int nfft, int fstride, const C *tw, int tid, int nth)
{
    int logNs = 0;
    C *s = a, *d = b;
    const int np = fft_num_passes(logM);
    for (int pass = 0; pass < np; ++pass) {
        if (fft_radix(logM, pass) == 8) {
            stockham_pass<8, INV>(s, d, logM, logNs, nfft, fstride, tw, tid, nth);
            logNs += 3;
        } else {
            stockham_pass<4, INV>(s, d, logM, logNs, nfft, fstride, tw, tid, nth);
            logNs += 2;
        }
        __syncthreads();
        C *t = s;
        s = d;
        d = t;
    }
    return s;
}

}  // namespace safr
