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
    unsigned long long *bar;   // [2] arrival count, launch epoch
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

__device__ __forceinline__ unsigned long long ld_acquire_u64(const unsigned long long *p)
{
    unsigned long long v;
    asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

// Grid-wide barrier number `which` (0, 1) of the cooperative launch with epoch
// `epoch`.  bar[0] counts arrivals over the plan's lifetime: every launch adds
// 2 * gridDim.x, so barrier `which` of epoch E is complete when the count
// reaches (2E + which + 1) * gridDim.x.  Arrival is one release reduction (no
// round trip); one thread per CTA polls with acquire loads until the count is
// reached or the time limit passes.  Returns false (SAFR_ERR_TIMEOUT recorded)
// on a timeout.
__device__ __forceinline__ bool grid_sync_bounded(unsigned long long *bar, unsigned long long epoch, int which,
                                                  int *status, unsigned long long timeout_ns, int *flag)
{
    __syncthreads();
    if (threadIdx.x == 0) {
        const unsigned long long target = (2ull * epoch + (unsigned long long)which + 1ull) * gridDim.x;
        asm volatile("red.release.gpu.global.add.u64 [%0], 1;" ::"l"(bar) : "memory");
        int ok = 1;
        if (ld_acquire_u64(bar) < target) {
            const unsigned long long t0 = gtimer();
            while (ld_acquire_u64(bar) < target) {
                if (gtimer() - t0 > timeout_ns) {
                    atomicExch(status, (int)SAFR_ERR_TIMEOUT);
                    ok = 0;
                    break;
                }
            }
        }
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
    constexpr int TS = S::TS;
    constexpr int Mh = M / 2;
    constexpr int LOGM = S::LOG;
    constexpr int NTH = 512;
    constexpr int SLOTS = NTH / S::R1;
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ __align__(8) uint64_t mbar;
    __shared__ int bar_flag;
    __shared__ unsigned long long epoch_s;
    __shared__ R tt_b[SAFR_MAX_G], tt_c[SAFR_MAX_G];
    __shared__ R red[32];

    const int P = fp.P, o = fp.o, L = fp.L, G = fp.G;
    const int tid = threadIdx.x, b = blockIdx.x, nb = gridDim.x;
    const int lane = tid & 31, warp = tid >> 5;
    unsigned long long *stamp = fp.stamps ? fp.stamps + (size_t)b * SAFR_TRACE_MARKS : nullptr;
    if (stamp && tid == 0) stamp[0] = gtimer();
    // epoch of this launch: advanced by CTA 0 once every CTA is past the last barrier
    if (tid == 0) epoch_s = ld_acquire_u64(fp.bar + 1);

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
    // B of the first column is requested once this CTA's phase-1 input has
    // arrived, so the 20+ MB stream does not queue ahead of those loads
    auto issue_first_b = [&]() {
        if (fp.stage_b && b < Mh && !tma_pending) {
            if (tid == 0) {
                const C *src = fp.B + (size_t)b * colB;
                mbar_expect_tx(&mbar, colB_bytes);
                for (unsigned off = 0; off < colB_bytes; off += 32768u)
                    tma_load_1d((unsigned char *)Bs + off, (const unsigned char *)src + off,
                                min(32768u, colB_bytes - off), &mbar);
            }
            tma_pending = true;
        }
    };
    {   // later columns of this CTA (or every column when B is not staged): into L2
        const int k0 = fp.stage_b ? b + nb : b;
        for (int k = k0; k < Mh; k += nb) {
            const char *base = (const char *)(fp.B + (size_t)k * colB);
            for (unsigned off = (unsigned)tid * 4096u; off < colB_bytes; off += NTH * 4096u)
                prefetch_l2(base + off, min(4096u, colB_bytes - off));
        }
    }
    for (int i = tid; i < M; i += NTH) twq[i] = fp.twq[i];
    if (stamp && tid == 0) stamp[1] = gtimer();

    // leave early (timeout or test hook) only after this CTA's own bulk copy landed
    auto drain = [&]() {
        if (tma_pending) mbar_wait_bounded(&mbar, tma_phase, fp.timeout_ns, fp.status);
    };

    // ---- phase 1: row pairs ----------------------------------------------------
    {
        const int lo = (int)(((long long)b * fp.n1) / nb), hi = (int)(((long long)(b + 1) * fp.n1) / nb);
        const int cap1 = min(SLOTS, (fp.n1 + nb - 1) / nb);  // row pairs per batch
        C *X = (C *)s12;                                      // [cap1][TS]
        for (int base = lo; base < hi; base += cap1) {
            const int nact = min(cap1, hi - base);
            // z[q] = psi[row a0][q - o] + i psi[row a0 + 1][q - o], zero outside the pupil
            for (int idx = tid; idx < (nact << LOGM); idx += NTH) {
                const int i = idx >> LOGM, q = idx & (M - 1);
                const int item = base + i, g = item / fp.npr, a0 = 2 * (item - g * fp.npr);
                const int qq = q - o;
                R re = 0, im = 0;
                if (qq >= 0 && qq < P) {
                    const TIN *psi = (const TIN *)fp.in + (size_t)g * P * P;
                    const R sc = fp.in_scales ? (R)fp.in_scales[g] : R(1);
                    re = load_in<R>(psi + (size_t)a0 * P + qq) * sc;
                    if (a0 + 1 < P) im = load_in<R>(psi + (size_t)(a0 + 1) * P + qq) * sc;
                }
                X[(size_t)i * TS + q] = C{re, im};
            }
            __syncthreads();
            issue_first_b();
            // per-row shares of the tip/tilt functionals (one warp per row pair)
            if (fp.any_tt)
                for (int i = warp; i < nact; i += NTH / 32) {
                    const int item = base + i, g = item / fp.npr, a0 = 2 * (item - g * fp.npr);
                    if (!fp.star_tt[g]) continue;
                    const R *wb = fp.tt_w, *wc = fp.tt_w + (size_t)P * P;
                    R s0b = 0, s0c = 0, s1b = 0, s1c = 0;
                    for (int q = lane; q < P; q += 32) {
                        const C v = X[(size_t)i * TS + o + q];
                        s0b += wb[a0 * P + q] * v.x;
                        s0c += wc[a0 * P + q] * v.x;
                        if (a0 + 1 < P) {
                            s1b += wb[(a0 + 1) * P + q] * v.y;
                            s1c += wc[(a0 + 1) * P + q] * v.y;
                        }
                    }
                    for (int off = 16; off > 0; off >>= 1) {
                        s0b += __shfl_xor_sync(0xffffffffu, s0b, off);
                        s0c += __shfl_xor_sync(0xffffffffu, s0c, off);
                        s1b += __shfl_xor_sync(0xffffffffu, s1b, off);
                        s1c += __shfl_xor_sync(0xffffffffu, s1c, off);
                    }
                    if (lane == 0) {
                        R *d = fp.pm + ((size_t)g * P + a0) * 2;
                        d[0] = s0b;
                        d[1] = s0c;
                        if (a0 + 1 < P) {
                            d[2] = s1b;
                            d[3] = s1c;
                        }
                    }
                }
            fft_core<M>(X, nact, 0, twq);
            if (stamp && tid == 0 && base == lo) stamp[2] = gtimer();
            // X1 = (Z[k] + conj Z[M-k]) / 2, X2 = (Z[k] - conj Z[M-k]) / 2i, row pair fastest
            for (int idx = tid; idx < nact * Mh; idx += NTH) {
                const int k = idx / nact, i = idx - k * nact;
                const int it2 = base + i, g2 = it2 / fp.npr, b0 = 2 * (it2 - g2 * fp.npr);
                const C z = X[(size_t)i * TS + k];
                const C zc = X[(size_t)i * TS + ((M - k) & (M - 1))];
                C *dst = fp.w1 + ((size_t)g2 * Mh + k) * P + b0;
                dst[0] = C{R(0.5) * (z.x + zc.x), R(0.5) * (z.y - zc.y)};
                if (b0 + 1 < P) dst[1] = C{R(0.5) * (z.y + zc.y), R(0.5) * (zc.x - z.x)};
            }
            __syncthreads();
        }
    }
    issue_first_b();  // CTAs without phase-1 rows
    if (b == fp.skip_cta) {  // test hook: every other CTA's first barrier must time out
        drain();
        return;
    }
    if (stamp) {
        __syncthreads();
        if (tid == 0) stamp[3] = gtimer();
    }
    if (!grid_sync_bounded(fp.bar, epoch_s, 0, fp.status, fp.timeout_ns, &bar_flag)) {
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
        const int cap2 = min(SLOTS, fp.ntask2);
        C *D = (C *)s12;                  // [G][TS] spectra d_g(j) of the column
        C *Y = D + (size_t)G * TS;        // [cap2][TS] layer spectra -> inverse transforms
        for (int k = b; k < Mh; k += nb) {
            // every star's column of w1, zero-padded (p contiguous: coalesced)
            for (int idx = tid; idx < (G << LOGM); idx += NTH) {
                const int s = idx >> LOGM, p = idx & (M - 1), pp = p - o;
                D[(size_t)s * TS + p] = (pp >= 0 && pp < P) ? __ldcg(fp.w1 + ((size_t)s * Mh + k) * P + pp) : C{0, 0};
            }
            __syncthreads();
            for (int base = 0; base < G; base += SLOTS) fft_core<M>(D + (size_t)base * TS, min(SLOTS, G - base), 0, twq);
            if (fp.any_tt) {  // d_g -= b_g X(j, k) + c_g Y(j, k) for the LGS stars
                for (int idx = tid; idx < (G << LOGM); idx += NTH) {
                    const int s = idx >> LOGM, j = idx & (M - 1);
                    if (!fp.star_tt[s]) continue;
                    const C xh = fp.xy_hat[((size_t)k << LOGM) + j];
                    const C yh = fp.xy_hat[((size_t)(Mh + k) << LOGM) + j];
                    C &d = D[(size_t)s * TS + j];
                    d.x -= tt_b[s] * xh.x + tt_c[s] * yh.x;
                    d.y -= tt_b[s] * xh.y + tt_c[s] * yh.y;
                }
                __syncthreads();
            }
            if (stamp && tid == 0 && k == b) stamp[5] = gtimer();
            const C *Bcol;
            if (fp.stage_b) {
                if (tid == 0) bar_flag = mbar_wait_bounded(&mbar, tma_phase, fp.timeout_ns, fp.status) ? 1 : -1;
                __syncthreads();
                tma_pending = false;
                tma_phase ^= 1u;
                if (bar_flag < 0) return;  // the copy never landed: nothing in flight any more to wait for
                Bcol = Bs;
            } else {
                Bcol = fp.B + (size_t)k * colB;
            }
            // b_l(j) = sum_g B_lg(j) d_g(j) for each (group, layer), then inverse transforms along j
            for (int base = 0; base < fp.ntask2; base += cap2) {
                const int nact = min(cap2, fp.ntask2 - base);
                for (int idx = tid; idx < (nact << LOGM); idx += NTH) {
                    const int i = idx >> LOGM, j = idx & (M - 1);
                    const int task = base + i, gi = task / L, l = task - gi * L;
                    const GroupDev &gr = fp.grp[gi];
                    const C *Bj = Bcol + ((size_t)(gr.b_row0 + l * gr.G) << LOGM) + j;
                    R ar = 0, ai = 0;
                    for (int gg = 0; gg < gr.G; ++gg) {
                        const C bv = Bj[(size_t)gg << LOGM];
                        const C dv = D[(size_t)gr.star[gg] * TS + j];
                        ar += bv.x * dv.x - bv.y * dv.y;
                        ai += bv.x * dv.y + bv.y * dv.x;
                    }
                    Y[(size_t)i * TS + j] = C{ar, ai};
                }
                __syncthreads();
                if (fp.energy)  // Parseval partial sums, one warp per (group, layer)
                    for (int i = warp; i < nact; i += NTH / 32) {
                        const int task = base + i, gi = task / L, l = task - gi * L;
                        R e = 0;
                        for (int j = lane; j < M; j += 32) {
                            const C v = Y[(size_t)i * TS + j];
                            e += v.x * v.x + v.y * v.y;
                        }
                        for (int off = 16; off > 0; off >>= 1) e += __shfl_xor_sync(0xffffffffu, e, off);
                        if (lane == 0) fp.energy[((size_t)gi * L + l) * Mh + k] = (float)(k == 0 ? e : R(2) * e);
                    }
                fft_core<M>(Y, nact, 1, twq);
                for (int idx = tid; idx < (nact << LOGM); idx += NTH) {
                    const int i = idx >> LOGM, p = idx & (M - 1);
                    const int task = base + i, gi = task / L, l = task - gi * L;
                    fp.w2[((((size_t)gi * L + l) * Mh + k) << LOGM) + p] = Y[(size_t)i * TS + p];
                }
                __syncthreads();
            }
            // next column of this CTA: bring its B block in while the rest runs
            if (fp.stage_b && k + nb < Mh) {
                if (tid == 0) {
                    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                    const C *src = fp.B + (size_t)(k + nb) * colB;
                    mbar_expect_tx(&mbar, colB_bytes);
                    for (unsigned off = 0; off < colB_bytes; off += 32768u)
                        tma_load_1d((unsigned char *)Bs + off, (const unsigned char *)src + off,
                                    min(32768u, colB_bytes - off), &mbar);
                }
                tma_pending = true;
            }
        }
    }
    if (stamp) {
        __syncthreads();
        if (tid == 0) stamp[6] = gtimer();
    }
    if (!grid_sync_bounded(fp.bar, epoch_s, 1, fp.status, fp.timeout_ns, &bar_flag)) {
        drain();
        return;
    }
    if (stamp && tid == 0) stamp[7] = gtimer();
    if (b == 0 && tid == 0) {  // every CTA has read this launch's epoch: open the next one
        asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(fp.bar + 1), "l"(epoch_s + 1ull) : "memory");
    }

    // ---- phase 3: (layer, row tile) ----------------------------------------------
    {
        const int RT = fp.rt3;
        int *ti0 = (int *)s3;                                   // [M]
        R *tfw = (R *)(ti0 + M);                                // [M]
        const int st0 = fp.st3[0], st1 = fp.st3[1];
        C *stg0 = (C *)(tfw + M);                               // [Mh][st0]
        C *stg1 = stg0 + (size_t)Mh * st0;                      // [Mh][st1]
        C *Z = stg1 + (size_t)Mh * st1;                         // [cap3][TS] row-pair transforms
        const bool rs0 = fp.grp[0].resample != 0;               // only an LGS group (group 0) is resampled
        const bool two = fp.ngroups > 1;
        for (int it = b; it < fp.n3; it += nb) {
            const int l = it / fp.tiles3, p0 = (it - l * fp.tiles3) * RT;
            const int nr = min(RT, M - p0);
            if (rs0)
                for (int i = tid; i < M; i += NTH) {
                    ti0[i] = fp.rs_i0[l * M + i];
                    tfw[i] = fp.rs_w[l * M + i];
                }
            __syncthreads();
            const int first0 = rs0 ? ti0[p0] : p0;
            const int nsrc0 = rs0 ? ti0[p0 + nr - 1] + 2 - first0 : nr;
            const int nsrc1 = two ? nr : 0;  // the NGS group is never resampled
            const int npair0 = (nsrc0 + 1) >> 1, npair1 = (nsrc1 + 1) >> 1;
            const int ntot = npair0 + npair1;
            if (nsrc0 > fp.nsrc3[0] || nsrc1 > fp.nsrc3[1] || ntot > fp.cap3) {  // sized on the host; never expected
                if (tid == 0) atomicExch(fp.status, (int)SAFR_ERR_DEVICE);
                continue;
            }
            // stage the needed rows of every column: stg[k][s] = w2[gi][l][k][first + s]
            {
                const C *src0 = fp.w2 + (size_t)l * Mh * M;
                for (int idx = tid; idx < Mh * nsrc0; idx += NTH) {
                    const int k = idx / nsrc0, s = idx - k * nsrc0;
                    stg0[k * st0 + s] = __ldcg(src0 + ((size_t)k << LOGM) + ((first0 + s) & (M - 1)));
                }
                const C *src1 = fp.w2 + ((size_t)L + l) * Mh * M;
                for (int idx = tid; idx < Mh * nsrc1; idx += NTH) {
                    const int k = idx / nsrc1, s = idx - k * nsrc1;
                    stg1[k * st1 + s] = __ldcg(src1 + ((size_t)k << LOGM) + p0 + s);
                }
            }
            __syncthreads();
            if (stamp && tid == 0 && it == b) stamp[8] = gtimer();
            // Z[k] = X1[k] + i X2[k] over the full length M from the stored half spectra of a row pair
            for (int idx = tid; idx < (ntot << LOGM); idx += NTH) {
                const int task = idx >> LOGM, k = idx & (M - 1);
                const bool g1 = task >= npair0;
                const int i = g1 ? task - npair0 : task;
                const C *sg = g1 ? stg1 : stg0;
                const int st = g1 ? st1 : st0;
                const bool hasb = 2 * i + 1 < (g1 ? nsrc1 : nsrc0);
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
                Z[(size_t)task * TS + k] = z;
            }
            __syncthreads();
            fft_core<M>(Z, ntot, 1, twq);
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
            // source row s of group 0 is Z[s / 2] (real part for even s, imaginary for odd)
            const R f = fp.inv_M2 * inv_scale;
            TOUT *outp = (TOUT *)fp.out + ((size_t)l * M + p0) * M;
            for (int idx = tid; idx < nr * M; idx += NTH) {
                const int r = idx >> LOGM, q = idx & (M - 1);
                R v;
                if (rs0) {  // bilinear in the LGS layer grid (pitch c_l delta)
                    const R fu = tfw[p0 + r], fv = tfw[q];
                    const int j0u = ti0[q];
                    const int ja = j0u & (M - 1), jb = (j0u + 1) & (M - 1);
                    const int s0 = ti0[p0 + r] - first0, s1 = s0 + 1;
                    const C *za = Z + (size_t)(s0 >> 1) * TS, *zb = Z + (size_t)(s1 >> 1) * TS;
                    const R a0 = (s0 & 1) ? za[ja].y : za[ja].x, a1 = (s0 & 1) ? za[jb].y : za[jb].x;
                    const R b0v = (s1 & 1) ? zb[ja].y : zb[ja].x, b1v = (s1 & 1) ? zb[jb].y : zb[jb].x;
                    v = (R(1) - fu) * ((R(1) - fv) * a0 + fv * a1) + fu * ((R(1) - fv) * b0v + fv * b1v);
                } else {
                    const C zz = Z[(size_t)(r >> 1) * TS + q];
                    v = (r & 1) ? zz.y : zz.x;
                }
                if (two) {  // the NGS group's rows follow group 0's pairs
                    const C zz = Z[(size_t)(npair0 + (r >> 1)) * TS + q];
                    v += (r & 1) ? zz.y : zz.x;
                }
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
        const int cap2 = std::min(SLOTS, pl->ngroups * L);
        const size_t s1 = (size_t)cap1 * S::TS * cs;
        const size_t s2 = (size_t)G * S::TS * cs + (size_t)cap2 * S::TS * cs;
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
            const int cap3 = (nsm_[0] + nsm_[1]) / 2;  // every row pair of a tile in one batch
            if (cap3 > SLOTS) continue;
            s3 += (size_t)cap3 * S::TS * cs;
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
