// Warp-level FFTs of compile-time length M for the persistent frame kernel.
//
// A transform of length M = LW * R (LW = min(M, 32) lanes, R = M / LW values
// per lane) runs in one group of LW lanes with all data in registers:
//
//   forward, natural order in, permuted order out.  Lane t holds x[t + LW r]
//     in register r.  Step A: R-point DFT over r in registers, then multiply
//     register k_r by W_M^(t k_r).  Step B: LW-point DFT across the lanes by
//     radix-2 decimation in frequency with __shfl_xor_sync.  Lane t ends with
//     X[k_r + R brev(t)] in register k_r (brev: reversal of log2(LW) bits).
//   inverse, permuted order in, natural order out: the same steps in reverse
//     with conjugate twiddles, unnormalised.  Lane t ends with
//     y[t + LW r] = sum_k Y[k] W_M^(-k (t + LW r)) in register r.
//
// This is the four-step factorisation of the DFT with N1 = LW, N2 = R:
//   X[k2 + R k1] = sum_t W_LW^(t k1) W_M^(t k2) sum_r W_R^(r k2) x[t + LW r].
// No shared memory and no block barrier: every lane of the warp must call the
// functions together (lanes of unused transforms compute on any values).
// The R-point DFTs are recursive radix-2 decimation in time, fully unrolled,
// with the exact constants cos(pi m / 16); the lane-stage twiddles W_LW^e and
// the W_M^(t k_r) twiddles come from a table built on the host in FP64.
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
struct WShape {
    static constexpr int LW = M < 32 ? M : 32;  // lanes per transform
    static constexpr int R = M / LW;            // values per lane
    static constexpr int LB = ilog2c(LW);       // lane bits
    static constexpr int TPW = 32 / LW;         // transforms per warp
    static constexpr int LOG = ilog2c(M);
};

// Per-lane twiddles W_M^(t k_r) and the lane-stage twiddles W_LW^e, e < LW, from one
// table built on the host in FP64 and copied into shared memory (layout:
// tab[k_r * LW + t], then tab[M + e]).
template <int M, typename C>
struct WTw {
    using S = WShape<M>;
    C tw[S::R];
    const C *wlw;  // W_LW^e, e < LW
    __device__ __forceinline__ void load(const C *tab, int t)
    {
#pragma unroll
        for (int k = 0; k < S::R; ++k) tw[k] = tab[k * S::LW + t];
        wlw = tab + M;
    }
};

template <typename C>
__device__ __forceinline__ C shfl_xor_c(C v, int m)
{
    return C{__shfl_xor_sync(0xffffffffu, v.x, m), __shfl_xor_sync(0xffffffffu, v.y, m)};
}

// Whether the last two lane stages (first two of the inverse) run without complex products.
// Measured: 21.04 -> 20.20 us per back-to-back 256-grid frame (8 values per lane); at 16 values per
// lane (the 512 grid) the peeled stages made the frame 4 us slower, so it keeps the plain loop.
template <int M>
__host__ __device__ constexpr bool wfft_peel() { return WShape<M>::R <= 8 && WShape<M>::LW >= 4; }

// Forward transform, natural order in, permuted order out (see above).
// Lane stage h multiplies the lower lane's difference by W_(2h)^(t mod h).  For h >= 4 that is a
// general complex product; the last two stages need none: for h = 2 the factor is 1 or -i (a swap
// with a sign), for h = 1 it is 1, so their chains carry one add per value instead of three
// dependent operations.
template <int M, typename C>
__device__ __forceinline__ void wfft_fwd(C (&v)[WShape<M>::R], const WTw<M, C> &w, int t)
{
    using S = WShape<M>;
    using R = decltype(C{}.x);
    constexpr int HLAST = wfft_peel<M>() ? 4 : 1;  // the general loop's last stage
    dft_reg<S::R, false>(v);
#pragma unroll
    for (int k = 1; k < S::R; ++k) v[k] = c_mul(v[k], w.tw[k]);
    // stage h: W_(2h)^(t mod h) = W_LW^((t mod h) * LW / (2h))
#pragma unroll 1
    for (int h = S::LW / 2; h >= HLAST; h >>= 1) {
        // upper lane: v + p; lower lane: (p - v) W.  As (sg v + p) wp with sg = -1, wp = W on the
        // lower lane and sg = 1, wp = 1 on the upper one.
        const bool low = (t & h) != 0;
        const C ws = w.wlw[(t & (h - 1)) * (S::LW / (2 * h))];
        const C wp = low ? ws : C{R(1), R(0)};
        const R sg = low ? R(-1) : R(1);
#pragma unroll
        for (int k = 0; k < S::R; ++k) {
            const C p = shfl_xor_c(v[k], h);
            v[k] = c_mul(C{sg * v[k].x + p.x, sg * v[k].y + p.y}, wp);
        }
    }
    if constexpr (wfft_peel<M>()) {
        {  // h = 2: the lower lanes with t odd multiply by -i: (x, y) -> (y, -x)
            const bool low = (t & 2) != 0, rot = low && (t & 1);
            const R sg = low ? R(-1) : R(1);
#pragma unroll
            for (int k = 0; k < S::R; ++k) {
                const C p = shfl_xor_c(v[k], 2);
                const C u = C{sg * v[k].x + p.x, sg * v[k].y + p.y};
                v[k] = rot ? C{u.y, -u.x} : u;
            }
        }
        {  // h = 1: factor 1
            const R sg = (t & 1) ? R(-1) : R(1);
#pragma unroll
            for (int k = 0; k < S::R; ++k) {
                const C p = shfl_xor_c(v[k], 1);
                v[k] = C{sg * v[k].x + p.x, sg * v[k].y + p.y};
            }
        }
    }
}

// Inverse transform (unnormalised), permuted order in, natural order out.  The first two lane
// stages need no complex product (factor 1; then 1 or +i, a swap with a sign).
template <int M, typename C>
__device__ __forceinline__ void wfft_inv(C (&v)[WShape<M>::R], const WTw<M, C> &w, int t)
{
    using S = WShape<M>;
    using R = decltype(C{}.x);
    if constexpr (wfft_peel<M>()) {
        {  // h = 1: factor 1
            const R sg = (t & 1) ? R(-1) : R(1);
#pragma unroll
            for (int k = 0; k < S::R; ++k) {
                const C p = shfl_xor_c(v[k], 1);
                v[k] = C{sg * v[k].x + p.x, sg * v[k].y + p.y};
            }
        }
        {  // h = 2: the lower lanes with t odd multiply by +i: (x, y) -> (-y, x)
            const bool low = (t & 2) != 0, rot = low && (t & 1);
            const R sg = low ? R(-1) : R(1);
#pragma unroll
            for (int k = 0; k < S::R; ++k) {
                const C u = rot ? C{-v[k].y, v[k].x} : v[k];
                const C p = shfl_xor_c(u, 2);
                v[k] = C{sg * u.x + p.x, sg * u.y + p.y};
            }
        }
    }
#pragma unroll 1
    for (int h = wfft_peel<M>() ? 4 : 1; h < S::LW; h <<= 1) {
        // lower lane: u = v conj(W), result p - u; upper lane: u = v, result u + p
        const bool low = (t & h) != 0;
        const C ws = w.wlw[(t & (h - 1)) * (S::LW / (2 * h))];
        const C wc = low ? C{ws.x, -ws.y} : C{R(1), R(0)};
        const R sg = low ? R(-1) : R(1);
#pragma unroll
        for (int k = 0; k < S::R; ++k) {
            const C u = c_mul(v[k], wc);
            const C p = shfl_xor_c(u, h);
            v[k] = C{sg * u.x + p.x, sg * u.y + p.y};
        }
    }
#pragma unroll
    for (int k = 1; k < S::R; ++k) v[k] = c_mulc(v[k], w.tw[k]);
    dft_reg<S::R, true>(v);
}

// N independent inverse transforms in lockstep (the same steps, interleaved stage by
// stage, so that one warp keeps N dependency chains in flight).
template <int M, int N, typename C>
__device__ __forceinline__ void wfft_inv_n(C (&v)[N][WShape<M>::R], const WTw<M, C> &w, int t)
{
    using S = WShape<M>;
    using R = decltype(C{}.x);
    if constexpr (wfft_peel<M>()) {
        {  // h = 1: factor 1
            const R sg = (t & 1) ? R(-1) : R(1);
#pragma unroll
            for (int k = 0; k < S::R; ++k)
#pragma unroll
                for (int n = 0; n < N; ++n) {
                    const C p = shfl_xor_c(v[n][k], 1);
                    v[n][k] = C{sg * v[n][k].x + p.x, sg * v[n][k].y + p.y};
                }
        }
        {  // h = 2: +i on the lower lanes with t odd
            const bool low = (t & 2) != 0, rot = low && (t & 1);
            const R sg = low ? R(-1) : R(1);
#pragma unroll
            for (int k = 0; k < S::R; ++k)
#pragma unroll
                for (int n = 0; n < N; ++n) {
                    const C u = rot ? C{-v[n][k].y, v[n][k].x} : v[n][k];
                    const C p = shfl_xor_c(u, 2);
                    v[n][k] = C{sg * u.x + p.x, sg * u.y + p.y};
                }
        }
    }
#pragma unroll 1
    for (int h = wfft_peel<M>() ? 4 : 1; h < S::LW; h <<= 1) {
        const bool low = (t & h) != 0;
        const C ws = w.wlw[(t & (h - 1)) * (S::LW / (2 * h))];
        const C wc = low ? C{ws.x, -ws.y} : C{R(1), R(0)};
        const R sg = low ? R(-1) : R(1);
#pragma unroll
        for (int k = 0; k < S::R; ++k)
#pragma unroll
            for (int n = 0; n < N; ++n) {
                const C u = c_mul(v[n][k], wc);
                const C p = shfl_xor_c(u, h);
                v[n][k] = C{sg * u.x + p.x, sg * u.y + p.y};
            }
    }
#pragma unroll
    for (int n = 0; n < N; ++n) {
#pragma unroll
        for (int k = 1; k < S::R; ++k) v[n][k] = c_mulc(v[n][k], w.tw[k]);
        dft_reg<S::R, true>(v[n]);
    }
}

}  // namespace safr
