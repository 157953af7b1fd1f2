// Algorithm 1 as ONE persistent cooperative kernel per frame, for a grid
// size M fixed at compile time (instantiated per precision in frame_*.cu).
//
// All CTAs are co-resident (cooperative launch, one per SM, 512 threads) and
// run three phases separated by two grid-wide barriers:
//
//   prologue  TMA bulk copy of the B block of this CTA's first column k
//             (all groups, layers and stars; contiguous in memory) into shared
//             memory, and an L2 bulk prefetch of the B of its later columns, so
//             the dominant byte stream lands during phase 1;
//   phase 1   row pairs of the zero-padded wavefronts (Section 2): two real
//             rows packed into one complex length-M FFT along q, split into
//             two half spectra -> w1[g][k][p] (k < M/2).  LGS rows of a mixed
//             plan also contribute their share of the two linear functionals
//             that give the tip and tilt of the least-squares plane over the
//             pupil (Algorithm 3, line 3);
//   phase 2   columns k: FFT along p of every star's column -> d_g(j, k);
//             removeTT in the frequency domain, d_g -= b_g X(j,k) + c_g Y(j,k)
//             with X, Y = DFT2 of x and y on the mask (DFT2 is linear); per
//             frequency and layer b_l = sum_g B_lg d_g (Algorithm 1, line 5)
//             straight into the registers of the inverse FFT along j ->
//             w2[group][l][k][p];
//   phase 3   (layer, tile of output rows): complex-to-real inverse FFT of
//             the needed rows (IDFT2, 1/M^2), bilinear resample of LGS layers
//             from pitch c_l*delta to delta, sum of the groups (Algorithm 3,
//             line 4), optional FP16 with a power-of-two scale from the layer
//             energy (Parseval), store.
//
// Every wait is bounded: the grid barriers and the TMA completion waits read
// %globaltimer and give up after a time limit, recording SAFR_ERR_TIMEOUT in
// the plan's status word; a CTA that gives up first waits (again with a
// limit) for its own bulk copies, then returns.
#pragma once

#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <type_traits>
#include <vector>

#include "common.cuh"
#include "plan.h"
#include "regfft.cuh"

namespace safr {

template <typename R>
struct Frame2Params {
    using C = typename std::conditional<sizeof(R) == 8, double2, float2>::type;
    int P, L, G, o, ngroups, sumLG;
    int npr, n1;               // row pairs per star, phase-1 items
    int ntask2;                // phase-2 (group, layer) tasks = ngroups * L
    int rt3, tiles3, n3;       // phase-3 rows per item, tiles per layer, items
    int st3[2];                // staged source rows per group (odd stride)
    int cap3;                  // row-pair transforms in flight in phase 3
    int nsrc3[2];              // max source rows per group and item
    int any_tt, any_resample;
    int stage_b;               // 1: B column block staged in shared memory by TMA
    int skip_cta;              // test hook (-1: none)
    unsigned long long timeout_ns;
    R inv_M2;
    // shared-memory carve-up (bytes from the dynamic base)
    unsigned off_b, off_s12, off_s3;
    const void *in;
    const float *in_scales;
    void *out;
    float *out_scales;
    const C *B;                // [M/2][sumLG][M]
    C *w1;                     // [G][M/2][P]
    C *w2;                     // [ngroups][L][M/2][M]
    float *energy;             // [ngroups][L][M/2]
    const C *twq;              // [R2][R1] W_M^(n1 k2)
    const int *rs_i0;          // [L][M]
    const R *rs_w;             // [L][M]
    const R *tt_w;             // [2][P][P]
    const C *xy_hat;           // [2][M/2][M]
    R *pm;                     // [G][P][2]
    unsigned *bar;             // [2]
    unsigned long long *stamps;
    int *status;
    int star_tt[SAFR_MAX_G];
    GroupDev grp[2];
};

__device__ __forceinline__ unsigned long long gtimer()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ unsigned smem_u32(const void *p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t *mbar, unsigned count)
{
    asm volatile("mbarrier.init.shared.b64 [%0], %1;" ::"r"(smem_u32(mbar)), "r"(count) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t *mbar, unsigned bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared.b64 _, [%0], %1;" ::"r"(smem_u32(mbar)), "r"(bytes) : "memory");
}

// one 1-D bulk copy global -> this CTA's shared memory, completing on mbar
__device__ __forceinline__ void tma_load_1d(void *dst, const void *src, unsigned bytes, uint64_t *mbar)
{
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(mbar))
        : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *mbar, unsigned parity)
{
    unsigned ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_u32(mbar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// bounded wait for phase `parity` of mbar; false (and SAFR_ERR_TIMEOUT) if it never completes
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *mbar, unsigned parity, unsigned long long timeout_ns,
                                                  int *status)
{
    if (mbar_try_wait(mbar, parity)) return true;
    const unsigned long long t0 = gtimer();
    while (!mbar_try_wait(mbar, parity)) {
        if (gtimer() - t0 > timeout_ns) {
            atomicExch(status, (int)SAFR_ERR_TIMEOUT);
            return false;
        }
    }
    return true;
}

// Grid-wide barrier of the cooperative launch; false if it timed out.
__device__ __forceinline__ bool grid_sync_bounded(unsigned *bar, int *status, unsigned long long timeout_ns, int *flag)
{
    __syncthreads();
    if (threadIdx.x == 0) {
        volatile unsigned *vgen = bar + 1;
        const unsigned gen = *vgen;
        __threadfence();
        const unsigned arrived = atomicAdd(bar, 1u);
        int ok = 1;
        if (arrived == gridDim.x - 1) {
            atomicExch(bar, 0u);
            __threadfence();
            atomicAdd(bar + 1, 1u);
        } else {
            const unsigned long long t0 = gtimer();
            while (*vgen == gen) {
                if (gtimer() - t0 > timeout_ns) {
                    atomicExch(status, (int)SAFR_ERR_TIMEOUT);
                    ok = 0;
                    break;
                }
            }
        }
        __threadfence();
        *flag = ok;
    }
    __syncthreads();
    return *flag != 0;
}

template <int M, typename R, typename TIN, typename TOUT>
__global__ void __launch_bounds__(512, 1) k_frame2(Frame2Params<R> fp)
{
    using C = typename Frame2Params<R>::C;
    using S = FftShape<M>;
    constexpr int R1 = S::R1, R2 = S::R2, CB = S::CB, TS = S::TS;
    constexpr int Mh = M / 2;
    constexpr int NTH = 512;
    constexpr int SLOTS = NTH / R1;
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ __align__(8) uint64_t mbar;
    __shared__ int bar_flag;
    __shared__ R tt_b[SAFR_MAX_G], tt_c[SAFR_MAX_G];
    __shared__ R red[32];

    const int P = fp.P, o = fp.o, L = fp.L, G = fp.G;
    const int tid = threadIdx.x, b = blockIdx.x, nb = gridDim.x;
    const int lane = tid & 31, warp = tid >> 5;
    const int slot = tid / R1, t = tid % R1;
    unsigned long long *stamp = fp.stamps ? fp.stamps + (size_t)b * SAFR_TRACE_MARKS : nullptr;
    if (stamp && tid == 0) stamp[0] = gtimer();

    C *twq = (C *)smem;                      // [M]
    C *Bs = (C *)(smem + fp.off_b);          // staged B column block
    unsigned char *s12 = smem + fp.off_s12;  // phase 1 / 2 scratch
    unsigned char *s3 = smem + fp.off_s3;    // phase 3 scratch (may overlap Bs)
    const size_t colB = (size_t)fp.sumLG * M;  // complex per B column block
    const unsigned colB_bytes = (unsigned)(colB * sizeof(C));

    // ---- prologue ------------------------------------------------------------
    unsigned tma_phase = 0;
    bool tma_pending = false;
    if (tid == 0 && fp.stage_b) mbar_init(&mbar, 1);
    __syncthreads();
    if (fp.stage_b && b < Mh && tid == 0) {
        const C *src = fp.B + (size_t)b * colB;
        mbar_expect_tx(&mbar, colB_bytes);
        for (unsigned off = 0; off < colB_bytes; off += 32768u)
            tma_load_1d((unsigned char *)Bs + off, (const unsigned char *)src + off, min(32768u, colB_bytes - off), &mbar);
    }
    if (fp.stage_b && b < Mh) tma_pending = true;
    {   // later columns of this CTA (or every column when B is not staged): into L2
        const int k0 = fp.stage_b ? b + nb : b;
        for (int k = k0; k < Mh; k += nb) {
            const char *base = (const char *)(fp.B + (size_t)k * colB);
            for (unsigned off = (unsigned)tid * 4096u; off < colB_bytes; off += NTH * 4096u)
                prefetch_l2(base + off, min(4096u, colB_bytes - off));
        }
    }
    for (int i = tid; i < M; i += NTH) twq[i] = fp.twq[i];
    __syncthreads();
    if (stamp && tid == 0) stamp[1] = gtimer();

    // leave early (timeout or test hook) only after this CTA's own bulk copy landed
    auto drain = [&]() {
        if (tma_pending) mbar_wait_bounded(&mbar, tma_phase, fp.timeout_ns, fp.status);
    };

    // ---- phase 1: row pairs ----------------------------------------------------
    {
        const int lo = (int)(((long long)b * fp.n1) / nb), hi = (int)(((long long)(b + 1) * fp.n1) / nb);
        const int cap1 = min(SLOTS, (fp.n1 + nb - 1) / nb);  // row pairs in flight
        C *T = (C *)s12;                               // [cap1][TS]
        C *Z = T + (size_t)cap1 * TS;                  // [cap1][M]
        const R *wb = fp.tt_w, *wc = fp.tt_w + (size_t)P * P;
        for (int base = lo; base < hi; base += cap1) {
            const int nact = min(cap1, hi - base);
            const int item = base + slot;
            const bool act = slot < nact;
            int g = 0, a0 = 0;
            if (act) {
                g = item / fp.npr;
                a0 = 2 * (item - g * fp.npr);
            }
            const bool two = act && a0 + 1 < P;
            const bool tt = act && fp.star_tt[g];
            C v[R2];
            R sb0 = 0, sc0 = 0, sb1 = 0, sc1 = 0;
            const TIN *psi = (const TIN *)fp.in + (size_t)g * P * P;
            const R sc = (act && fp.in_scales) ? (R)fp.in_scales[g] : R(1);
#pragma unroll
            for (int n2 = 0; n2 < R2; ++n2) {
                const int qq = t + R1 * n2 - o;
                R re = 0, im = 0;
                if (act && qq >= 0 && qq < P) {
                    re = load_in<R>(psi + (size_t)a0 * P + qq) * sc;
                    if (two) im = load_in<R>(psi + (size_t)(a0 + 1) * P + qq) * sc;
                    if (tt) {
                        sb0 += wb[a0 * P + qq] * re;
                        sc0 += wc[a0 * P + qq] * re;
                        if (two) {
                            sb1 += wb[(a0 + 1) * P + qq] * im;
                            sc1 += wc[(a0 + 1) * P + qq] * im;
                        }
                    }
                }
                v[n2] = C{re, im};
            }
            if (fp.any_tt) {
#pragma unroll
                for (int off = R1 / 2; off > 0; off >>= 1) {
                    sb0 += __shfl_xor_sync(0xffffffffu, sb0, off);
                    sc0 += __shfl_xor_sync(0xffffffffu, sc0, off);
                    sb1 += __shfl_xor_sync(0xffffffffu, sb1, off);
                    sc1 += __shfl_xor_sync(0xffffffffu, sc1, off);
                }
                if (tt && t == 0) {
                    R *d = fp.pm + ((size_t)g * P + a0) * 2;
                    d[0] = sb0;
                    d[1] = sc0;
                    if (two) {
                        d[2] = sb1;
                        d[3] = sc1;
                    }
                }
            }
            if (act) fft_step_a<M, false>(v, t, T + (size_t)slot * TS, twq);
            __syncthreads();
            if (act) {
                C out[CB][R1];
                fft_step_b<M, false>(out, t, T + (size_t)slot * TS);
#pragma unroll
                for (int c = 0; c < CB; ++c)
#pragma unroll
                    for (int k1 = 0; k1 < R1; ++k1) Z[(size_t)slot * M + t + c * R1 + R2 * k1] = out[c][k1];
            }
            __syncthreads();
            if (stamp && tid == 0 && base == lo) stamp[2] = gtimer();
            // X1 = (Z[k] + conj Z[M-k]) / 2, X2 = (Z[k] - conj Z[M-k]) / 2i, row pair fastest
            for (int idx = tid; idx < nact * Mh; idx += NTH) {
                const int k = idx / nact, i = idx - k * nact;
                const int it2 = base + i, g2 = it2 / fp.npr, b0 = 2 * (it2 - g2 * fp.npr);
                const C z = Z[(size_t)i * M + k];
                const C zc = Z[(size_t)i * M + ((M - k) & (M - 1))];
                C *dst = fp.w1 + ((size_t)g2 * Mh + k) * P + b0;
                dst[0] = C{R(0.5) * (z.x + zc.x), R(0.5) * (z.y - zc.y)};
                if (b0 + 1 < P) dst[1] = C{R(0.5) * (z.y + zc.y), R(0.5) * (zc.x - z.x)};
            }
            __syncthreads();
        }
    }
    if (b == fp.skip_cta) {  // test hook: every other CTA's first barrier must time out
        drain();
        return;
    }
    if (stamp) {
        __syncthreads();
        if (tid == 0) stamp[3] = gtimer();
    }
    if (!grid_sync_bounded(fp.bar, fp.status, fp.timeout_ns, &bar_flag)) {
        drain();
        return;
    }
    if (stamp && tid == 0) stamp[4] = gtimer();

    // ---- phase 2: columns --------------------------------------------------------
    {
        for (int g = warp; fp.any_tt && g < G; g += NTH / 32) {
            R sb = 0, sc = 0;
            if (fp.star_tt[g])
                for (int a = lane; a < P; a += 32) {
                    const R *d = fp.pm + ((size_t)g * P + a) * 2;
                    sb += __ldcg(d);
                    sc += __ldcg(d + 1);
                }
            for (int off = 16; off > 0; off >>= 1) {
                sb += __shfl_xor_sync(0xffffffffu, sb, off);
                sc += __shfl_xor_sync(0xffffffffu, sc, off);
            }
            if (lane == 0) {
                tt_b[g] = sb;
                tt_c[g] = sc;
            }
        }
        C *D = (C *)s12;                 // [G][M] spectra d_g(j) of the column
        C *T = D + (size_t)G * M;        // [SLOTS][TS]
        __syncthreads();
        for (int k = b; k < Mh; k += nb) {
            // forward FFT of each star's column (p = t + R1 n2), zero outside the pupil
            for (int base = 0; base < G; base += SLOTS) {
                const int s = base + slot;
                const bool act = s < G;
                if (act) {
                    C v[R2];
                    const C *col = fp.w1 + ((size_t)s * Mh + k) * P;
#pragma unroll
                    for (int n2 = 0; n2 < R2; ++n2) {
                        const int pp = t + R1 * n2 - o;
                        v[n2] = (pp >= 0 && pp < P) ? __ldcg(col + pp) : C{0, 0};
                    }
                    fft_step_a<M, false>(v, t, T + (size_t)slot * TS, twq);
                }
                __syncthreads();
                if (act) {
                    C out[CB][R1];
                    fft_step_b<M, false>(out, t, T + (size_t)slot * TS);
                    const bool tt = fp.star_tt[s] != 0;
                    const R tb = tt ? tt_b[s] : R(0), tc = tt ? tt_c[s] : R(0);
#pragma unroll
                    for (int c = 0; c < CB; ++c)
#pragma unroll
                        for (int k1 = 0; k1 < R1; ++k1) {
                            const int j = t + c * R1 + R2 * k1;
                            C d = out[c][k1];
                            if (tt) {
                                const C xh = fp.xy_hat[(size_t)k * M + j];
                                const C yh = fp.xy_hat[(size_t)(Mh + k) * M + j];
                                d.x -= tb * xh.x + tc * yh.x;
                                d.y -= tb * xh.y + tc * yh.y;
                            }
                            D[(size_t)s * M + j] = d;
                        }
                }
                __syncthreads();
            }
            if (stamp && tid == 0 && k == b) stamp[5] = gtimer();
            const C *Bcol;
            if (fp.stage_b) {
                if (tid == 0 && !mbar_wait_bounded(&mbar, tma_phase, fp.timeout_ns, fp.status)) bar_flag = -1;
                else if (tid == 0) bar_flag = 1;
                __syncthreads();
                tma_pending = false;
                tma_phase ^= 1u;
                if (bar_flag < 0) return;  // the copy never landed: nothing in flight any more to wait for
                Bcol = Bs;
            } else {
                Bcol = fp.B + (size_t)k * colB;
            }
            // per-frequency apply straight into the inverse FFT along j
            for (int base = 0; base < fp.ntask2; base += SLOTS) {
                const int task = base + slot;
                const bool act = task < fp.ntask2;
                int gi = 0, l = 0;
                if (act) {
                    gi = task / L;
                    l = task - gi * L;
                }
                R en = 0;
                if (act) {
                    const GroupDev &gr = fp.grp[gi];
                    const int Gg = gr.G;
                    const C *Bl = Bcol + (size_t)(gr.b_row0 + l * Gg) * M;
                    C acc[R2];
#pragma unroll
                    for (int n2 = 0; n2 < R2; ++n2) acc[n2] = C{0, 0};
                    for (int gg = 0; gg < Gg; ++gg) {
                        const C *Brow = Bl + (size_t)gg * M + t;
                        const C *Drow = D + (size_t)gr.star[gg] * M + t;
#pragma unroll
                        for (int n2 = 0; n2 < R2; ++n2) {
                            const C bv = Brow[R1 * n2];
                            const C dv = Drow[R1 * n2];
                            acc[n2].x += bv.x * dv.x - bv.y * dv.y;
                            acc[n2].y += bv.x * dv.y + bv.y * dv.x;
                        }
                    }
                    if (fp.energy) {
#pragma unroll
                        for (int n2 = 0; n2 < R2; ++n2) en += acc[n2].x * acc[n2].x + acc[n2].y * acc[n2].y;
                    }
                    fft_step_a<M, true>(acc, t, T + (size_t)slot * TS, twq);
                }
                if (fp.energy) {  // all lanes take part in the shuffles
#pragma unroll
                    for (int off = R1 / 2; off > 0; off >>= 1) en += __shfl_xor_sync(0xffffffffu, en, off);
                    if (act && t == 0) fp.energy[((size_t)gi * L + l) * Mh + k] = (float)(k == 0 ? en : R(2) * en);
                }
                __syncthreads();
                if (act) {
                    C out[CB][R1];
                    fft_step_b<M, true>(out, t, T + (size_t)slot * TS);
                    C *dst = fp.w2 + (((size_t)gi * L + l) * Mh + k) * M;
#pragma unroll
                    for (int c = 0; c < CB; ++c)
#pragma unroll
                        for (int k1 = 0; k1 < R1; ++k1) dst[t + c * R1 + R2 * k1] = out[c][k1];
                }
                __syncthreads();
            }
            // next column of this CTA: bring its B block in while the rest runs
            if (fp.stage_b && k + nb < Mh && tid == 0) {
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                const C *src = fp.B + (size_t)(k + nb) * colB;
                mbar_expect_tx(&mbar, colB_bytes);
                for (unsigned off = 0; off < colB_bytes; off += 32768u)
                    tma_load_1d((unsigned char *)Bs + off, (const unsigned char *)src + off,
                                min(32768u, colB_bytes - off), &mbar);
            }
            if (fp.stage_b && k + nb < Mh) tma_pending = true;
        }
    }
    if (stamp) {
        __syncthreads();
        if (tid == 0) stamp[6] = gtimer();
    }
    if (!grid_sync_bounded(fp.bar, fp.status, fp.timeout_ns, &bar_flag)) {
        drain();
        return;
    }
    if (stamp && tid == 0) stamp[7] = gtimer();

    // ---- phase 3: (layer, row tile) ----------------------------------------------
    {
        const int RT = fp.rt3;
        int *ti0 = (int *)s3;                                   // [M]
        R *tfw = (R *)(ti0 + M);                                // [M]
        const int st0 = fp.st3[0], st1 = fp.st3[1];
        C *stg0 = (C *)(tfw + M);                               // [Mh][st0]
        C *stg1 = stg0 + (size_t)Mh * st0;                      // [Mh][st1]
        C *T = stg1 + (size_t)Mh * st1;                         // [cap3][TS]
        R *rows0 = (R *)(T + (size_t)fp.cap3 * TS);             // [nsrc3[0]][M] real rows
        R *rows1 = rows0 + (size_t)fp.nsrc3[0] * M;             // [nsrc3[1]][M]
        const bool rs0 = fp.grp[0].resample != 0, rs1 = fp.ngroups > 1 && fp.grp[1].resample != 0;
        for (int it = b; it < fp.n3; it += nb) {
            const int l = it / fp.tiles3, p0 = (it - l * fp.tiles3) * RT;
            const int nr = min(RT, M - p0);
            if (fp.any_resample)
                for (int i = tid; i < M; i += NTH) {
                    ti0[i] = fp.rs_i0[l * M + i];
                    tfw[i] = fp.rs_w[l * M + i];
                }
            __syncthreads();
            const int first0 = rs0 ? ti0[p0] : p0;
            const int nsrc0 = rs0 ? ti0[p0 + nr - 1] + 2 - first0 : nr;
            const int first1 = rs1 ? ti0[p0] : p0;
            const int nsrc1 = fp.ngroups > 1 ? (rs1 ? ti0[p0 + nr - 1] + 2 - first1 : nr) : 0;
            const int npair0 = (nsrc0 + 1) >> 1, npair1 = (nsrc1 + 1) >> 1;
            if (nsrc0 > fp.nsrc3[0] || nsrc1 > fp.nsrc3[1]) {  // sized on the host for every tile; never expected
                if (tid == 0) atomicExch(fp.status, (int)SAFR_ERR_DEVICE);
                continue;
            }
            // stage the needed rows of every column: stg[k][s] = w2[gi][l][k][first + s]
            {
                const C *src0 = fp.w2 + (size_t)l * Mh * M;
                for (int idx = tid; idx < Mh * nsrc0; idx += NTH) {
                    const int k = idx / nsrc0, s = idx - k * nsrc0;
                    stg0[k * st0 + s] = __ldcg(src0 + (size_t)k * M + ((first0 + s) & (M - 1)));
                }
                const C *src1 = fp.w2 + ((size_t)L + l) * Mh * M;
                for (int idx = tid; idx < Mh * nsrc1; idx += NTH) {
                    const int k = idx / nsrc1, s = idx - k * nsrc1;
                    stg1[k * st1 + s] = __ldcg(src1 + (size_t)k * M + ((first1 + s) & (M - 1)));
                }
            }
            __syncthreads();
            if (stamp && tid == 0 && it == b) stamp[8] = gtimer();
            // complex-to-real transforms of row pairs, both groups in one batch
            const int ntot = npair0 + npair1;
            for (int base = 0; base < ntot; base += fp.cap3) {
                const int task = base + slot;
                const bool act = slot < fp.cap3 && task < ntot;
                const bool g1 = act && task >= npair0;
                const int i = act ? (g1 ? task - npair0 : task) : 0;
                const int nsg = g1 ? nsrc1 : nsrc0;
                const bool hasb = act && 2 * i + 1 < nsg;
                if (act) {
                    const C *sg = g1 ? stg1 : stg0;
                    const int st = g1 ? st1 : st0;
                    C v[R2];
#pragma unroll
                    for (int n2 = 0; n2 < R2; ++n2) {
                        const int k = t + R1 * n2;
                        C z = C{0, 0};
                        if (k < Mh) {
                            C x1 = sg[k * st + 2 * i];
                            C x2 = hasb ? sg[k * st + 2 * i + 1] : C{0, 0};
                            if (k == 0) {
                                x1.y = 0;
                                x2.y = 0;
                            }
                            z = C{x1.x - x2.y, x1.y + x2.x};
                        } else if (k > Mh) {
                            const int kk = M - k;
                            const C x1 = sg[kk * st + 2 * i];
                            const C x2 = hasb ? sg[kk * st + 2 * i + 1] : C{0, 0};
                            z = C{x1.x + x2.y, x2.x - x1.y};
                        }
                        v[n2] = z;
                    }
                    fft_step_a<M, true>(v, t, T + (size_t)slot * TS, twq);
                }
                __syncthreads();
                if (act) {
                    C out[CB][R1];
                    fft_step_b<M, true>(out, t, T + (size_t)slot * TS);
                    R *ra = (g1 ? rows1 : rows0) + (size_t)(2 * i) * M;
#pragma unroll
                    for (int c = 0; c < CB; ++c)
#pragma unroll
                        for (int k1 = 0; k1 < R1; ++k1) {
                            const int q = t + c * R1 + R2 * k1;
                            ra[q] = out[c][k1].x;
                            if (hasb) ra[M + q] = out[c][k1].y;
                        }
                }
                __syncthreads();
            }
            if (stamp && tid == 0 && it == b) stamp[9] = gtimer();
            R inv_scale = R(1);
            if (fp.out_scales) {
                // layer energy sum_n |b(n)|^2 over the groups (fixed order) -> mean square / M^4
                R e = 0;
                for (int gi = 0; gi < fp.ngroups; ++gi)
                    for (int k = tid; k < Mh; k += NTH) e += (R)__ldcg(fp.energy + ((size_t)gi * L + l) * Mh + k);
                e = block_sum(e, red);
                const double ms = (double)e / ((double)M * M * (double)M * M);
                const double sc = ms > 0 ? exp2(rint(0.5 * log2(ms))) : 1.0;
                inv_scale = (R)(1.0 / sc);
                if (p0 == 0 && tid == 0) fp.out_scales[l] = (float)sc;
            }
            const R f = fp.inv_M2 * inv_scale;
            TOUT *outp = (TOUT *)fp.out + ((size_t)l * M + p0) * M;
            for (int idx = tid; idx < nr * M; idx += NTH) {
                const int r = idx / M, q = idx & (M - 1);
                R v = 0;
                if (rs0 || rs1) {  // bilinear weights of output (p0 + r, q) in the LGS layer grid
                    const R fu = tfw[p0 + r], fv = tfw[q];
                    const int j0u = ti0[q];
                    const int ja = j0u & (M - 1), jb = (j0u + 1) & (M - 1);
                    const R *r0 = (rs0 ? rows0 : rows1) + (size_t)(ti0[p0 + r] - (rs0 ? first0 : first1)) * M;
                    const R *r1 = r0 + M;
                    v += (R(1) - fu) * ((R(1) - fv) * r0[ja] + fv * r0[jb]) + fu * ((R(1) - fv) * r1[ja] + fv * r1[jb]);
                }
                if (!rs0) v += rows0[(size_t)r * M + q];
                if (fp.ngroups > 1 && !rs1) v += rows1[(size_t)r * M + q];
                if constexpr (std::is_same<TOUT, double>::value)
                    store_out_d(outp + idx, (double)(v * f));
                else
                    store_out<TOUT>(outp + idx, (float)(v * f));
            }
            __syncthreads();
        }
    }
    if (stamp && tid == 0) stamp[10] = gtimer();
}

// ----------------------------------------------------------------------------
// host side (instantiated per precision)
// ----------------------------------------------------------------------------
template <int M, typename R>
struct Frame2Host {
    using C = typename Frame2Params<R>::C;
    using S = FftShape<M>;

    // phase-3 staged-row stride: at least n, odd (conflict-free column reads)
    static int odd_at_least(int n) { return n | 1; }

    // Sizes the kernel for the plan; false if it cannot hold it.
    static bool configure(safr_plan_s *pl, int nsm, void *kernel)
    {
        const int Mh = M / 2, G = pl->G, L = pl->L, P = pl->P;
        const size_t cs = sizeof(C), rs = sizeof(R);
        const size_t limit = 227 * 1024 - 1024;  // dynamic shared memory budget
        const int SLOTS = 512 / S::R1;
        const int nb = nsm;
        auto al = [](size_t x) { return (x + 127) & ~(size_t)127; };
        const size_t twq_b = al((size_t)M * cs);
        // phase 1 / 2 scratch, sized for the transforms actually in flight
        const int n1 = G * ((P + 1) / 2);
        const int cap1 = std::min(SLOTS, (n1 + nb - 1) / nb);
        const int cap2 = std::min(SLOTS, std::max(G, pl->ngroups * L));
        const size_t s1 = (size_t)cap1 * S::TS * cs + (size_t)cap1 * M * cs;
        const size_t s2 = (size_t)G * M * cs + (size_t)cap2 * S::TS * cs;
        const size_t s12 = al(std::max(s1, s2));
        const size_t colB = (size_t)pl->sumLG * M * cs;
        if (G > 32) return false;
        // phase 3 tiles
        int best_rt = 0;
        size_t best_s3 = 0;
        int st[2] = {0, 0}, ns[2] = {0, 0};
        for (int rt = std::min(32, M); rt >= 2; rt -= 2) {
            int nsm_[2] = {0, 0};
            for (int gi = 0; gi < pl->ngroups; ++gi) {
                int mx = rt;
                if (pl->grp[gi].resample)
                    for (int l = 0; l < L; ++l) {
                        const double c = pl->grp[gi].c[l];
                        for (int p0 = 0; p0 < M; p0 += rt) {
                            const int p1 = std::min(M, p0 + rt) - 1;
                            const int a = (int)std::floor(M / 2.0 + (p0 - M / 2.0) / c);
                            const int bq = (int)std::floor(M / 2.0 + (p1 - M / 2.0) / c);
                            mx = std::max(mx, bq + 2 - a);
                        }
                    }
                nsm_[gi] = mx + (mx & 1);  // even: whole row pairs
            }
            size_t s3 = (size_t)M * (4 + rs);
            for (int gi = 0; gi < pl->ngroups; ++gi) s3 += (size_t)Mh * odd_at_least(nsm_[gi]) * cs;
            const int cap3 = std::min(SLOTS, (nsm_[0] + nsm_[1]) / 2);
            s3 += (size_t)cap3 * S::TS * cs;
            for (int gi = 0; gi < pl->ngroups; ++gi) s3 += (size_t)nsm_[gi] * M * rs;
            s3 = al(s3);
            const long long items = (long long)L * ((M + rt - 1) / rt);
            // largest tile that fits and still gives every CTA an item
            if (twq_b + s3 <= limit && (items >= nb || rt == 2 || best_rt == 0)) {
                if (best_rt == 0 || items >= nb) {
                    best_rt = rt;
                    best_s3 = s3;
                    pl->f2_cap3 = cap3;
                    for (int gi = 0; gi < 2; ++gi) {
                        ns[gi] = nsm_[gi];
                        st[gi] = gi < pl->ngroups ? odd_at_least(nsm_[gi]) : 0;
                    }
                    if (items >= nb) break;
                }
            }
        }
        if (best_rt == 0) return false;
        // B staging if it fits beside the phase 1/2 scratch
        const bool stage = twq_b + al(colB) + s12 <= limit;
        pl->f2_stage_b = stage ? 1 : 0;
        pl->f2_off_b = (unsigned)twq_b;
        pl->f2_off_s12 = (unsigned)(twq_b + (stage ? al(colB) : 0));
        pl->f2_off_s3 = (unsigned)twq_b;
        const size_t total = std::max((size_t)pl->f2_off_s12 + s12, twq_b + best_s3);
        if (total > limit) return false;
        pl->f2_smem = total;
        pl->f2_rt3 = best_rt;
        pl->f2_tiles3 = (M + best_rt - 1) / best_rt;
        pl->f2_n3 = L * pl->f2_tiles3;
        for (int gi = 0; gi < 2; ++gi) {
            pl->f2_st3[gi] = st[gi];
            pl->f2_nsrc3[gi] = ns[gi];
        }
        pl->f2_grid = nb;
        (void)P;
        if (cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)total) != cudaSuccess) {
            cudaGetLastError();
            return false;
        }
        int occ = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kernel, 512, total) != cudaSuccess || occ < 1) {
            cudaGetLastError();
            return false;
        }
        return true;
    }

    static Frame2Params<R> params(safr_plan_s *pl, const void *in, const float *in_scales, void *out,
                                  float *out_scales)
    {
        Frame2Params<R> fp;
        memset(&fp, 0, sizeof(fp));
        fp.P = pl->P;
        fp.L = pl->L;
        fp.G = pl->G;
        fp.o = pl->o;
        fp.ngroups = pl->ngroups;
        fp.sumLG = pl->sumLG;
        fp.npr = (pl->P + 1) / 2;
        fp.n1 = pl->G * fp.npr;
        fp.ntask2 = pl->ngroups * pl->L;
        fp.rt3 = pl->f2_rt3;
        fp.cap3 = pl->f2_cap3;
        fp.tiles3 = pl->f2_tiles3;
        fp.n3 = pl->f2_n3;
        for (int gi = 0; gi < 2; ++gi) {
            fp.st3[gi] = pl->f2_st3[gi];
            fp.nsrc3[gi] = pl->f2_nsrc3[gi];
        }
        fp.any_tt = pl->remove_tt;
        for (int gi = 0; gi < pl->ngroups; ++gi) fp.any_resample |= pl->grp[gi].resample ? 1 : 0;
        fp.stage_b = pl->f2_stage_b;
        fp.skip_cta = pl->debug_skip_cta;
        fp.timeout_ns = pl->barrier_timeout_ns;
        fp.inv_M2 = (R)(1.0 / ((double)M * M));
        fp.off_b = pl->f2_off_b;
        fp.off_s12 = pl->f2_off_s12;
        fp.off_s3 = pl->f2_off_s3;
        fp.in = in;
        fp.in_scales = in_scales;
        fp.out = out;
        fp.out_scales = out_scales;
        fp.B = (const C *)pl->d_B;
        fp.w1 = (C *)pl->d_w1;
        fp.w2 = (C *)pl->d_w2;
        fp.energy = out_scales ? pl->d_energy : nullptr;
        fp.twq = (const C *)pl->d_twq;
        fp.rs_i0 = pl->d_rs_i0;
        fp.rs_w = (const R *)pl->d_rs_w;
        fp.tt_w = (const R *)pl->d_tt_w;
        fp.xy_hat = (const C *)pl->d_xy_hat;
        fp.pm = (R *)pl->d_pm;
        fp.bar = pl->d_bar;
        fp.stamps = pl->trace ? pl->d_stamps : nullptr;
        fp.status = pl->d_status;
        for (int g = 0; g < pl->G; ++g) fp.star_tt[g] = pl->star_tt[g];
        for (int gi = 0; gi < pl->ngroups; ++gi) {
            fp.grp[gi].G = pl->grp[gi].G;
            fp.grp[gi].b_row0 = pl->grp[gi].b_row0;
            fp.grp[gi].resample = pl->grp[gi].resample ? 1 : 0;
            for (int q = 0; q < pl->grp[gi].G; ++q) fp.grp[gi].star[q] = pl->grp[gi].stars[q];
        }
        return fp;
    }
};

// Host-side table of the four-step twiddles W_M^(n1 k2), laid out [k2][n1].
inline void frame2_twiddles_impl(int M, std::vector<double> &re, std::vector<double> &im)
{
    int logM = 0;
    while ((1 << logM) < M) ++logM;
    const int R1 = 1 << (logM / 2), R2 = M / R1;
    re.assign(M, 0.0);
    im.assign(M, 0.0);
    const double pi = 3.14159265358979323846264338327950288;
    for (int k2 = 0; k2 < R2; ++k2)
        for (int n1 = 0; n1 < R1; ++n1) {
            const long long e = ((long long)n1 * k2) % M;
            re[k2 * R1 + n1] = std::cos(2.0 * pi * (double)e / M);
            im[k2 * R1 + n1] = -std::sin(2.0 * pi * (double)e / M);
        }
}

}  // namespace safr
