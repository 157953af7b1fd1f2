// Algorithm 1 as ONE persistent cooperative kernel per frame, for a grid
// size M fixed at compile time (instantiated per precision in frame_*.cu).
//
// All CTAs are co-resident (one per SM, 512 threads: the grid is at most the
// SM count and the kernel's shared memory allows one CTA per SM) and run three
// phases separated by two grid-wide barriers.  The kernel is launched with
// programmatic stream serialization: a frame launched right after another
// one takes the SMs as that frame's CTAs leave, runs its prologue (tables, B
// copy), and waits (griddepcontrol.wait) before it reads its inputs.  Every transform is a
// warp-level FFT (warpfft.cuh): one group of min(M, 32) lanes per transform,
// all data in registers, lanes exchanged by shuffles.
//
//   prologue  per-lane twiddles and this CTA's later-phase tables are loaded
//             into registers; B of every column after this CTA's first goes
//             to L2 by bulk prefetch;
//   phase 1   once warp 0 has issued its wavefront loads, the first half of
//             the CTA's first B column block (all groups, layers and stars;
//             contiguous) is copied into shared memory by TMA
//             (cp.async.bulk), the second half once the CTA has arrived at the
//             first grid barrier;
//             one transform per row pair of the zero-padded wavefronts
//             (Section 2): rows a0, a0 + 1 packed as z = psi_a0 + i psi_a0+1,
//             forward FFT along q, split into the two half spectra
//             -> w1[g][k][p] (k < M/2).  LGS rows of a mixed plan also give
//             their share of the two linear functionals that yield the tip and
//             tilt of the least-squares plane over the pupil (Algorithm 3,
//             line 3);
//   phase 2   column k: one transform per star, FFT along p -> d_g(j, k);
//             removeTT in the frequency domain, d_g -= b_g X(j,k) + c_g Y(j,k)
//             with X, Y = DFT2 of x and y on the mask (DFT2 is linear); then
//             one transform per (group, layer): b_l = sum_g B_lg d_g at every
//             frequency (Algorithm 1, line 5) straight into the registers of
//             the inverse FFT along j -> w2[group][l][k][p];
//   phase 3   (layer, tile of output rows): the needed rows of w2 staged in
//             shared memory; for LGS layers the row half of the bilinear
//             resample from pitch c_l*delta to delta is taken on the staged
//             spectra (a real combination of two rows commutes with the
//             transform along q), so every group needs one transform per
//             output row pair; inverse transforms (complex-to-real, IDFT2 with
//             1/M^2), the column half of the resample, sum of the groups
//             (Algorithm 3, line 4), optional FP16 with a power-of-two scale
//             from the layer energy (Parseval), store.
//
// The forward transforms leave the frequency index j in the permuted order
// of freqorder.h; B, the removeTT spectra and the column spectra are stored
// in that order, and the inverse transforms take it back to natural order.
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
#include "freqorder.h"
#include "plan.h"
#include "warpfft.cuh"

namespace safr {

template <typename R>
struct Frame2Params {
    using C = typename std::conditional<sizeof(R) == 8, double2, float2>::type;
    int P, L, G, o, ngroups, sumLG;
    int npr, n1;               // row pairs per star, phase-1 items
    int ntask2;                // phase-2 (group, layer) tasks = ngroups * L
    int rt3, tiles3, n3;       // phase-3 rows per item, tiles per layer, items
    int st3[2];                // staged source rows per group (odd stride)
    int cap3;                  // row-pair transforms of one phase-3 item (rows of Z)
    int nsrc3[2];              // max source rows per group and item
    int any_tt, any_resample;
    int stage_b;               // 1: B column block staged in shared memory by TMA
    int skip_cta;              // test hook (-1: none)
    unsigned long long timeout_ns;
    R inv_M2;
    int blend;                 // 1: out <- (1 - gain) out + gain layers (the AO loop's integrator)
    R gain;
    // phase 0 of an AO loop step (polc_tab non-null): in <- mask (polc_psi + A(out)), the pseudo open
    // loop data, from the POLC sample table of loop.cu; in is then the plan's staging buffer
    const unsigned char *polc_tab;
    const void *polc_psi;
    // shared-memory carve-up (bytes from the dynamic base)
    unsigned off_rs, off_tw, off_b, off_d, off_xy, off_s3;
    const void *in;
    const float *in_scales;
    void *out;
    float *out_scales;
    const C *B;                // [M/2][sumLG][M], j in the permuted order
    C *w1;                     // [G][M/2][P]
    C *w2;                     // [ngroups][L][M/2][M]
    float *energy;             // [ngroups][L][M/2]
    const C *twq;              // [M + LW] warp-FFT twiddles (WTw layout)
    const int *rs_i0;          // [L][M]
    const R *rs_w;             // [L][M]
    const R *tt_w;             // [2][P][P] (not read by this kernel)
    R tt_n[6];                 // removeTT: w_b = mask (n0 + n1 x + n2 y), w_c = mask (n3 + n4 x + n5 y)
    R tt_delta;                // pixel pitch for x, y
    const unsigned *mask_bits; // [P][mask_words] pupil mask, one bit per pixel
    int mask_words;
    const C *xy_hat;           // [2][M/2][M], j in the permuted order
    R *pm;                     // [G][P][2]
    unsigned long long *bar;   // [2] arrival count, and the arrival count when the previous launch ended
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

// One element global -> shared without registers (cp.async; 8 bytes through L1, 16 bytes around it).
// The copies of a thread complete at cp_async_wait_all.
template <typename C>
__device__ __forceinline__ void cp_async_el(C *dst, const C *src)
{
    static_assert(sizeof(C) == 8 || sizeof(C) == 16, "complex float or double");
    if constexpr (sizeof(C) == 16)
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_u32(dst)), "l"(src) : "memory");
    else
        asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(smem_u32(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

__device__ __forceinline__ void mbar_init(uint64_t *mbar, unsigned count)
{
    asm volatile("mbarrier.init.shared.b64 [%0], %1;" ::"r"(smem_u32(mbar)), "r"(count) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t *mbar, unsigned bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared.b64 _, [%0], %1;" ::"r"(smem_u32(mbar)), "r"(bytes) : "memory");
}

// raises the transaction count of mbar's current phase without arriving
__device__ __forceinline__ void mbar_expect_tx_only(uint64_t *mbar, unsigned bytes)
{
    asm volatile("mbarrier.expect_tx.relaxed.cta.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(mbar)), "r"(bytes) : "memory");
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

// Grid-wide barrier on the arrival counter bar[0], which counts arrivals over
// the counter's lifetime (gridDim.x per barrier).  `index` is the number of grid
// barriers completed on the counter before this one (thread 0's value counts;
// the others' is not used), so this barrier is complete when the count reaches
// (index + 1) * gridDim.x.  Arrival is one release reduction (no round trip);
// one thread per CTA polls with acquire loads until the count is reached or
// the time limit passes.  Returns false (SAFR_ERR_TIMEOUT recorded) on a
// timeout.
struct NoHook {
    __device__ __forceinline__ void operator()() const {}
};
template <typename Hook = NoHook>
__device__ __forceinline__ bool grid_sync_bounded(unsigned long long *bar, unsigned long long index, int *status,
                                                  unsigned long long timeout_ns, int *flag,
                                                  unsigned long long *arrive_mark, Hook after_arrive = Hook())
{
    __syncthreads();
    if (threadIdx.x == 0) {
        const unsigned long long target = index + gridDim.x;  // index: arrivals counted before this barrier
        asm volatile("red.release.gpu.global.add.u64 [%0], 1;" ::"l"(bar) : "memory");
        after_arrive();
        if (arrive_mark) *arrive_mark = gtimer();
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


// Threads per CTA of the persistent kernel for grid size M (16 warps: measured
// faster than 32 warps with half the registers each at M = 256).
__host__ __device__ constexpr int frame2_threads(int) { return 512; }

// Phase 0 of an AO loop step: psi~_g = mask (psi_g + sum_l a_l(sample point)), bilinear in the
// state a = out (the sample table is described in loop.cu).  A CTA computes exactly the rows that
// its own phase 1 transforms (the same row pairs, contiguous in the [G][P] row space), one sample
// per thread, so a block barrier orders phase 0 before phase 1 and no grid barrier is needed.
// Not inlined: its registers stay out of the frame's own allocation.
template <int M, typename R, typename TIN, typename TOUT>
__device__ __noinline__ void polc_phase(const Frame2Params<R> &fp, int G, int L, int P, int b, int nb)
{
    const size_t nn = (size_t)G * L * P;
    const R *fx = (const R *)fp.polc_tab, *fy = fx + nn;
    const int *ix = (const int *)(fy + nn), *iy = ix + nn;
    const unsigned char *pmask = (const unsigned char *)(iy + nn);
    const TIN *ps = (const TIN *)fp.polc_psi;
    const TOUT *aa = (const TOUT *)fp.out;
    TIN *dst = (TIN *)fp.in;
    const int nth = blockDim.x;
    const int lo = (int)(((long long)b * fp.n1) / nb), hi = (int)(((long long)(b + 1) * fp.n1) / nb);
    if (lo >= hi) return;
    const int g0 = lo / fp.npr, g1 = (hi - 1) / fp.npr;
    const long r0 = (long)g0 * P + 2 * (lo - g0 * fp.npr);                            // first row
    const long r1 = (long)g1 * P + min(2 * (hi - 1 - g1 * fp.npr) + 1, P - 1) + 1;    // past the last
    for (long idx = r0 * P + threadIdx.x; idx < r1 * P; idx += nth) {
        const int g = (int)(idx / ((long)P * P)), pq = (int)(idx % ((long)P * P)), p = pq / P, q = pq % P;
        R acc = 0;
        if (pmask[pq]) {
            acc = load_in<R>(ps + idx);
#pragma unroll 8
            for (int l = 0; l < L; ++l) {  // the layers' loads in flight together
                const size_t k = ((size_t)g * L + l) * P;
                const R fu = fx[k + p], fv = fy[k + q];
                const int i0 = ix[k + p], j0 = iy[k + q];
                const int i1 = i0 + 1 == M ? 0 : i0 + 1, j1 = j0 + 1 == M ? 0 : j0 + 1;
                const TOUT *al = aa + (size_t)l * M * M;
                const R v00 = (R)al[(size_t)i0 * M + j0], v01 = (R)al[(size_t)i0 * M + j1];
                const R v10 = (R)al[(size_t)i1 * M + j0], v11 = (R)al[(size_t)i1 * M + j1];
                acc += (R(1) - fu) * ((R(1) - fv) * v00 + fv * v01) + fu * ((R(1) - fv) * v10 + fv * v11);
            }
        }
        dst[idx] = (TIN)acc;
    }
}

// Reads, at the start of a launch (thread 0), the arrival count the counter held when the previous
// launch on it ended.  That launch wrote it; stream order makes the write visible, so a plain load
// does (an acquire load would stall thread 0 until it lands).  After its last grid barrier, CTA 0
// stores the count plus this launch's arrivals (barriers x its own grid): every CTA has read the old
// value by then, and the next launch may use another grid size.
__device__ __forceinline__ unsigned long long bar_count_read(const unsigned long long *bar)
{
    return threadIdx.x == 0 ? __ldcg(bar + 1) : 0ull;
}
// One frame of Algorithm 1 on the whole grid (all CTAs call it together).
//   bar_base   the arrivals counted on fp.bar before this frame (thread 0); the first frame of the
//              launch reads it once the kernels before this one in the stream have finished
//   bph, tph   parities of the B and table mbarriers for this frame's first waits
//   first      the first frame of the launch: initialises the mbarriers
//   fidx       frame index within the launch: its wavefronts, layers and scales are the fidx-th of
//              contiguous arrays (fp.in + fidx G P^2, fp.out + fidx L M^2, G and L scales per frame)
// Returns false if a bounded wait gave up (status recorded); the caller then stops.
template <int M, typename R, typename TIN, typename TOUT, int CKT>
__device__ __forceinline__ bool frame_body(const Frame2Params<R> &fp, unsigned long long &bar_base, unsigned &bph,
                                           unsigned tph, bool first_frame, int fidx = 0)
{
    using C = typename Frame2Params<R>::C;
    using S = WShape<M>;
    constexpr int LW = S::LW, RR = S::R, LB = S::LB;
    constexpr int Mh = M / 2;
    constexpr int LOGM = S::LOG;
    constexpr int NTH = frame2_threads(M);
    constexpr int LPS = (NTH >= 1024 || M >= 512) ? 1 : 2;  // layers per transform slot in the phase-2 apply
    constexpr int NW = NTH / 32;
    constexpr int UNITS = NW * S::TPW;  // transforms in flight per CTA
    constexpr int QC = 4;               // per-lane loads in flight in the pupil loops
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ __align__(8) uint64_t mbar;
    __shared__ int bar_flag;
    __shared__ R red[32];
    // kernel-parameter arrays indexed at run time, copied once: indexing the
    // parameter block with a run-time index would place it in local memory
    __shared__ int s_star_tt[SAFR_MAX_G];
    __shared__ GroupDev s_grp[2];
    __shared__ R s_ttb[SAFR_MAX_G], s_ttc[SAFR_MAX_G];  // tip and tilt of each LGS star (phase 2)

    const int P = fp.P, o = fp.o, L = fp.L, G = fp.G;
    const int tid = threadIdx.x, b = blockIdx.x, nb = gridDim.x;
    const int lane = tid & 31, warp = tid >> 5;
    const int t = lane & (LW - 1);                             // lane within the transform
    const int unit = warp * S::TPW + (lane >> LB);             // transform slot of this lane
    const int bt = LB > 0 ? (int)(__brev((unsigned)t) >> (32 - LB)) : 0;  // brev(t)
    // parameter copies by warps 2 and 3 (warp 0 issues the table copies first).  The kernel parameter
    // is __grid_constant__, so these loops read it in place through generic pointers: one round of
    // loads in parallel.  Written as copies with constant indices (a chain of predicated constant-bank
    // reads), they cost 1.8 us per frame in a several-frames launch and 1.7 us back to back with B in
    // the L2 (the parameter lines miss once the kernel's code has streamed through the SM's caches).
    if (warp == 2) {
        for (int i = lane; i < SAFR_MAX_G; i += 32) s_star_tt[i] = fp.star_tt[i];
    } else if (warp == 3) {
        const int *src = reinterpret_cast<const int *>(&fp.grp[0]);
        int *dst = reinterpret_cast<int *>(&s_grp[0]);
        constexpr int NWD = (int)(2 * sizeof(GroupDev) / sizeof(int));
        for (int i = lane; i < NWD; i += 32) dst[i] = src[i];
    }
    unsigned long long *stamp = fp.stamps ? fp.stamps + (size_t)b * SAFR_TRACE_MARKS : nullptr;
#define SAFR_MARK(n, cond)                                   \
    do {                                                     \
        if (stamp && tid == 0 && (cond)) stamp[n] = gtimer(); \
    } while (0)
    SAFR_MARK(0, true);

    C *Bs = (C *)(smem + fp.off_b);   // staged B column block
    C *Dp = (C *)(smem + fp.off_d);   // [G][M] column spectra (permuted j)
    C *xys = (C *)(smem + fp.off_xy); // [2][M] removeTT spectra of this CTA's first column (permuted j)
    unsigned char *s3 = smem + fp.off_s3;
    const size_t colB = (size_t)fp.sumLG * M;  // complex per B column block
    const unsigned colB_bytes = (unsigned)(colB * sizeof(C));
    const bool rs0 = fp.grp[0].resample != 0;  // only an LGS group (group 0) is resampled

    // ---- prologue ------------------------------------------------------------
    // Each phase issues all of its global loads before it consumes any of
    // them.  The per-lane twiddles and the values this CTA needs in later
    // phases are loaded into registers here and land while phase 1 runs.
    bool tma_pending = false;
    if (tid == 0 && first_frame) mbar_init(&mbar, 1);
    auto copy_b = [&](int k) {  // thread 0 only
        const C *src = fp.B + (size_t)k * colB;
        mbar_expect_tx(&mbar, colB_bytes);
        for (unsigned off = 0; off < colB_bytes; off += 32768u)
            tma_load_1d((unsigned char *)Bs + off, (const unsigned char *)src + off, min(32768u, colB_bytes - off),
                        &mbar);
    };
    // The first pass's B block in two halves: the first in phase 1 (its bytes on mbar, no arrival),
    // the second once this CTA's arrival at the first grid barrier is out (the arrival and its bytes).
    // The barrier's release waits for the CTA's bulk copies in flight, so only half the block's
    // stream stands before it (MORFEO-like frames back to back with B from HBM: 19.34 -> 18.49 us).
    const unsigned half_b = (colB_bytes / 2) & ~15u;
    auto copy_b1 = [&](int k) {  // thread 0 only
        const unsigned char *src = (const unsigned char *)(fp.B + (size_t)k * colB);
        mbar_expect_tx_only(&mbar, half_b);
        for (unsigned off = 0; off < half_b; off += 32768u)
            tma_load_1d((unsigned char *)Bs + off, src + off, min(32768u, half_b - off), &mbar);
    };
    auto copy_b2 = [&](int k) {  // thread 0 only
        const unsigned char *src = (const unsigned char *)(fp.B + (size_t)k * colB);
        mbar_expect_tx(&mbar, colB_bytes - half_b);
        for (unsigned off = half_b; off < colB_bytes; off += 32768u)
            tma_load_1d((unsigned char *)Bs + off, src + off, min(32768u, colB_bytes - off), &mbar);
    };
    WTw<M, C> tw;
    // tables, one bulk copy each into shared memory of their own, completing on
    // mbar_t: the warp-FFT twiddles, this CTA's first phase-2 column of the
    // removeTT spectra and its first phase-3 item's resample tables
    __shared__ __align__(8) uint64_t mbar_t;
    C *twq_s = (C *)(smem + fp.off_tw);     // [M + LW]
    int *ti0 = (int *)(smem + fp.off_rs);  // [M]
    R *tfw = (R *)(ti0 + M);               // [M]
    const bool xy_pre = fp.any_tt && b < Mh;
    const bool rs_pre = rs0 && b < fp.n3;
    if (tid == 0) {
        if (first_frame) {
            mbar_init(&mbar_t, 1);
        } else {  // this CTA's reads of the previous frame's tables and B are done (block barrier)
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        }
        const unsigned cb = (unsigned)(M * sizeof(C)), ib = (unsigned)(M * 4), wb = (unsigned)(M * sizeof(R));
        const unsigned tb = (unsigned)((M + LW) * sizeof(C));
        mbar_expect_tx(&mbar_t, tb + (xy_pre ? 2 * cb : 0u) + (rs_pre ? ib + wb : 0u));
        tma_load_1d(twq_s, fp.twq, tb, &mbar_t);
        if (xy_pre) {
            tma_load_1d(xys, fp.xy_hat + ((size_t)b << LOGM), cb, &mbar_t);
            tma_load_1d(xys + M, fp.xy_hat + ((size_t)(Mh + b) << LOGM), cb, &mbar_t);
        }
        if (rs_pre) {
            const int l = b / fp.tiles3;
            tma_load_1d(ti0, fp.rs_i0 + (size_t)l * M, ib, &mbar_t);
            tma_load_1d(tfw, fp.rs_w + (size_t)l * M, wb, &mbar_t);
        }
        // this CTA's first B column block is copied in phase 1 (first half, right after warp 0 has
        // issued its wavefront loads) and at the first grid barrier (second half, after the CTA's
        // arrival): issued here, the 21 MB stream (from HBM when B is not in the L2) delayed the frame
        // data by about 2.4 us; issued whole in phase 1, it held the first grid barrier back (a release
        // at GPU scope waits for the CTA's bulk copies in flight)
    }
    // every thread waits for the tables before its first transform (no thread leaves
    // on a timeout here: the status word records it and the barriers stay balanced)
    auto tables = [&]() {
        mbar_wait_bounded(&mbar_t, tph, fp.timeout_ns, fp.status);
        tw.load(twq_s, t);
    };
    {   // later columns of this CTA (or every column when B is not staged): into L2
        const int k0 = fp.stage_b ? b + nb : b;
        for (int k = k0; k < Mh; k += nb) {
            const char *base = (const char *)(fp.B + (size_t)k * colB);
            for (unsigned off = (unsigned)tid * 4096u; off < colB_bytes; off += NTH * 4096u)
                prefetch_l2(base + off, min(4096u, colB_bytes - off));
        }
    }
    // Everything above reads only the plan's own tables and B, which no frame writes.  A frame
    // launched right after another one starts while that one finishes (programmatic dependent
    // launch); its inputs, the workspaces and the barrier counter are touched only after the
    // kernels before it in the stream have finished and their writes are visible.
    if (first_frame) {
        pdl_wait();
        bar_base = bar_count_read(fp.bar);
    }
    __syncthreads();  // the parameter copies
    SAFR_MARK(1, true);

    tma_pending = fp.stage_b && b < Mh;  // the B block copy, issued in phase 1 before any early return
    // leave early (timeout or test hook) only after this CTA's own bulk copy landed
    auto drain = [&]() {
        if (tma_pending) mbar_wait_bounded(&mbar, bph, fp.timeout_ns, fp.status);
    };

    unsigned long long bar_next = bar_base;  // arrivals counted before this frame's next grid barrier
    // ---- phase 0 (AO loop step): pseudo open loop data ---------------------------
    // psi~_g = mask (psi_g + sum_l a_l(sample point)), bilinear in the state a = out, one
    // sample per thread over the whole grid; the samples' table is described in loop.cu
    if (fp.polc_tab) {
        polc_phase<M, R, TIN, TOUT>(fp, G, L, P, b, nb);
        __syncthreads();  // the samples of this CTA's phase-1 rows, written by its own threads
    }

    // ---- phase 1: row pairs ----------------------------------------------------
    {
        // 32-bit products: the grid is at most the SM count and n1 = G ceil(P / 2) <= 32 * 512, so
        // (b + 1) n1 < 2^31 (a 64-bit division here cost 0.2 us per frame in code fetch)
        const int lo = (b * fp.n1) / nb, hi = ((b + 1) * fp.n1) / nb;
        bool first = true;
        for (int base = lo; base < hi; base += UNITS) {
            const int i = base + unit;
            const bool act = i < hi;
            if (!__any_sync(0xffffffffu, act)) continue;  // a warp with no transform in this round stays idle
            const int item = act ? i : lo, g = item / fp.npr, a0 = 2 * (item - g * fp.npr);
            const bool has1 = a0 + 1 < P;
            const TIN *psi = (const TIN *)fp.in + ((size_t)fidx * G + g) * P * P;
            const R sc = fp.in_scales ? (R)fp.in_scales[(size_t)fidx * G + g] : R(1);
            const bool tt = act && fp.any_tt && s_star_tt[g];
            // z[q] = psi[a0][q - o] + i psi[a0 + 1][q - o]: lane t holds q = t + LW r.
            // All loads (the two rows and, for removeTT, their pupil-mask words) are issued
            // from clamped in-range addresses before any is used; values out of range are
            // selected away.  The tip/tilt shares of a row are
            //   sum_q w_b[a][q] psi[a][q] = (n0 + n1 x_a) S0 + n2 S1,  S0 = sum_q m psi, S1 = sum_q m y_q psi
            // (w_b = mask (n0 + n1 x + n2 y), likewise w_c with n3..n5).
            C v[RR];
            R s0b = 0, s0c = 0, s1b = 0, s1c = 0;
            const int a1 = has1 ? a0 + 1 : a0;
            {
                const unsigned *mb0 = fp.mask_bits + (size_t)a0 * fp.mask_words;
                const unsigned *mb1 = fp.mask_bits + (size_t)a1 * fp.mask_words;
                R S00 = 0, S01 = 0, S10 = 0, S11 = 0;
                const R half = R(0.5) * (R)(P - 1);
                if constexpr (RR <= 8) {  // one batch of loads
                    R x0[RR], x1[RR];
                    unsigned m0[RR], m1[RR];
#pragma unroll
                    for (int r = 0; r < RR; ++r) {
                        const int qc = min(max(t + LW * r - o, 0), P - 1);
                        x0[r] = load_in_cg<R>(psi + (size_t)a0 * P + qc);
                        x1[r] = load_in_cg<R>(psi + (size_t)a1 * P + qc);
                        if (tt) {
                            m0[r] = mb0[qc >> 5];
                            m1[r] = mb1[qc >> 5];
                        }
                    }
                    if (first && tid == 0 && fp.stage_b && b < Mh) copy_b1(b);  // B after this warp's loads
#pragma unroll
                    for (int r = 0; r < RR; ++r) {
                        const int qq = t + LW * r - o;
                        const bool in = act && qq >= 0 && qq < P;
                        v[r] = C{in ? x0[r] * sc : R(0), in && has1 ? x1[r] * sc : R(0)};
                    }
                    if (tt) {
#pragma unroll
                        for (int r = 0; r < RR; ++r) {
                            const int qc = min(max(t + LW * r - o, 0), P - 1);
                            const R y = ((R)qc - half) * fp.tt_delta;
                            const R k0 = ((m0[r] >> (qc & 31)) & 1u) ? v[r].x : R(0);
                            const R k1 = ((m1[r] >> (qc & 31)) & 1u) ? v[r].y : R(0);
                            S00 += k0;
                            S01 += y * k0;
                            S10 += k1;
                            S11 += y * k1;
                        }
                    }
                } else {  // batches of 8 values (bounds the registers at large M)
                    constexpr int RB = 8;
#pragma unroll
                    for (int r0 = 0; r0 < RR; r0 += RB) {
                        R x0[RB], x1[RB];
                        unsigned m0[RB], m1[RB];
#pragma unroll
                        for (int u = 0; u < RB; ++u) {
                            const int qc = min(max(t + LW * (r0 + u) - o, 0), P - 1);
                            x0[u] = load_in_cg<R>(psi + (size_t)a0 * P + qc);
                            x1[u] = load_in_cg<R>(psi + (size_t)a1 * P + qc);
                            if (tt) {
                                m0[u] = mb0[qc >> 5];
                                m1[u] = mb1[qc >> 5];
                            }
                        }
                        if (r0 == 0 && first && tid == 0 && fp.stage_b && b < Mh) copy_b1(b);  // B after the first batch
#pragma unroll
                        for (int u = 0; u < RB; ++u) {
                            const int r = r0 + u, qq = t + LW * r - o;
                            const bool in = act && qq >= 0 && qq < P;
                            v[r] = C{in ? x0[u] * sc : R(0), in && has1 ? x1[u] * sc : R(0)};
                            if (tt) {
                                const int qc = min(max(qq, 0), P - 1);
                                const R y = ((R)qc - half) * fp.tt_delta;
                                const R k0 = ((m0[u] >> (qc & 31)) & 1u) ? v[r].x : R(0);
                                const R k1 = ((m1[u] >> (qc & 31)) & 1u) ? v[r].y : R(0);
                                S00 += k0;
                                S01 += y * k0;
                                S10 += k1;
                                S11 += y * k1;
                            }
                        }
                    }
                }
                if (tt) {
                    const R xa0 = ((R)a0 - half) * fp.tt_delta, xa1 = ((R)a1 - half) * fp.tt_delta;
                    s0b = (fp.tt_n[0] + fp.tt_n[1] * xa0) * S00 + fp.tt_n[2] * S01;
                    s0c = (fp.tt_n[3] + fp.tt_n[4] * xa0) * S00 + fp.tt_n[5] * S01;
                    s1b = (fp.tt_n[0] + fp.tt_n[1] * xa1) * S10 + fp.tt_n[2] * S11;
                    s1c = (fp.tt_n[3] + fp.tt_n[4] * xa1) * S10 + fp.tt_n[5] * S11;
                }
            }
            if (fp.any_tt) {  // per-row shares of the tip/tilt functionals
#pragma unroll
                for (int off = LW / 2; off > 0; off >>= 1) {
                    s0b += __shfl_xor_sync(0xffffffffu, s0b, off);
                    s0c += __shfl_xor_sync(0xffffffffu, s0c, off);
                    s1b += __shfl_xor_sync(0xffffffffu, s1b, off);
                    s1c += __shfl_xor_sync(0xffffffffu, s1c, off);
                }
                if (tt && t == 0) {
                    R *d = fp.pm + ((size_t)g * P + a0) * 2;
                    d[0] = s0b;
                    d[1] = s0c;
                    if (has1) {
                        d[2] = s1b;
                        d[3] = s1c;
                    }
                }
            }
            SAFR_MARK(2, first);
            SAFR_MARK(3, first);
            if (first) tables();
            wfft_fwd<M>(v, tw, t);
            SAFR_MARK(4, first);
            // Z[k] sits in register k_r of lane t for k = k_r + R brev(t); Z[M - k] in
            // register R - k_r of lane t ^ (LW - 1) (k_r > 0), or register 0 of lane
            // brev(LW - brev(t)) (k_r = 0).  Even lanes hold k < M/2.
            C zc[RR];
            zc[0] = C{__shfl_sync(0xffffffffu, v[0].x, (int)(__brev((unsigned)((LW - bt) & (LW - 1))) >> (32 - LB)), LW),
                      __shfl_sync(0xffffffffu, v[0].y, (int)(__brev((unsigned)((LW - bt) & (LW - 1))) >> (32 - LB)), LW)};
#pragma unroll
            for (int k = 1; k < RR; ++k) zc[k] = shfl_xor_c(v[RR - k], LW - 1);
            if (act && (t & 1) == 0) {
                C *dst = fp.w1 + (size_t)g * Mh * P + a0;
#pragma unroll
                for (int k = 0; k < RR; ++k) {
                    const int kk = k + RR * bt;
                    const C z = v[k], w = zc[k];
                    // X1 = (Z[k] + conj Z[M-k]) / 2, X2 = (Z[k] - conj Z[M-k]) / 2i
                    dst[(size_t)kk * P] = C{R(0.5) * (z.x + w.x), R(0.5) * (z.y - w.y)};
                    if (has1) dst[(size_t)kk * P + 1] = C{R(0.5) * (z.y + w.y), R(0.5) * (w.x - z.x)};
                }
            }
            first = false;
        }
        if (first) tables();  // a warp without phase-1 rows
        if (first && tid == 0 && fp.stage_b && b < Mh) copy_b1(b);  // warp 0 had no rows
    }
    if (b == fp.skip_cta) {  // test hook: every other CTA's first barrier must time out
        if (tid == 0 && fp.stage_b && b < Mh) copy_b2(b);  // complete the B block's phase before draining
        drain();
        return false;
    }
    SAFR_MARK(5, true);
    auto b_second = [&]() {  // thread 0, right after its arrival
        if (fp.stage_b && b < Mh) copy_b2(b);
    };
    if (!grid_sync_bounded(fp.bar, bar_next, fp.status, fp.timeout_ns, &bar_flag, stamp ? stamp + 6 : nullptr,
                           b_second)) {
        drain();
        return false;
    }
    SAFR_MARK(7, true);

    // ---- phase 2: columns --------------------------------------------------------
    // CKT columns per pass (2 when B is read from global memory and the CTA has several
    // columns): their star transforms share one round and their layer slots are packed
    // into common rounds of the warps
    {
        constexpr int CK = CKT;
        for (int kb = b; kb < Mh; kb += CK * nb) {
            const bool first = kb == b;
            const int ncols = min(CK, (Mh - 1 - kb) / nb + 1);
            // one transform per (column, star): the column of w1 (p contiguous), forward FFT along p
            const int ntask1 = ncols * G;
#pragma unroll 1
            for (int s0 = 0; s0 < ntask1; s0 += UNITS) {
                const int task = s0 + unit;
                const bool act = task < ntask1;
                if (!__any_sync(0xffffffffu, act)) continue;
                const int tk = act ? task : 0, c = tk / G, ss = tk - c * G, k = kb + c * nb;
                const C *src = fp.w1 + ((size_t)ss * Mh + k) * P;
                const bool tt = fp.any_tt && act && s_star_tt[ss];
                // the star's tip/tilt from the row shares of phase 1 (first pass: every column of the
                // pass needs them): the first batch of shares is loaded together with the column, so
                // the two L2 round trips overlap
                const bool tt_sum = first && fp.any_tt;
                R pb[QC], pc[QC];
                auto load_shares = [&](int a0) {
#pragma unroll
                    for (int u = 0; u < QC; ++u) {
                        const int a = a0 + t + LW * u;
                        pb[u] = tt && a < P ? __ldcg(fp.pm + ((size_t)ss * P + a) * 2) : R(0);
                        pc[u] = tt && a < P ? __ldcg(fp.pm + ((size_t)ss * P + a) * 2 + 1) : R(0);
                    }
                };
                C v[RR];
                if constexpr (M >= 512) {
                    // the column's P values go to this task's own row of Dp by asynchronous copies (the
                    // row later receives the task's transform), then into registers, zero-extended.
                    // Measured on the 512 grid: 113.7 -> 102.5 us per frame, and fewer spills; at 256
                    // the direct loads below are 0.2 us faster.
                    C *stg = Dp + ((size_t)c * G + ss) * M;
#pragma unroll
                    for (int r = 0; r < RR; ++r) {
                        const int pp = t + LW * r - o;
                        if (act && pp >= 0 && pp < P) cp_async_el(stg + pp, src + pp);
                    }
                    if (tt_sum) load_shares(0);
                    cp_async_wait_all();
                    __syncwarp();
#pragma unroll
                    for (int r = 0; r < RR; ++r) {
                        const int pp = t + LW * r - o;
                        v[r] = act && pp >= 0 && pp < P ? stg[pp] : C{0, 0};
                    }
                } else {
#pragma unroll
                    for (int r = 0; r < RR; ++r) v[r] = __ldcg(src + min(max(t + LW * r - o, 0), P - 1));
                    if (tt_sum) load_shares(0);
#pragma unroll
                    for (int r = 0; r < RR; ++r) {  // loads first (clamped addresses), then the zero extension
                        const int pp = t + LW * r - o;
                        if (!(act && pp >= 0 && pp < P)) v[r] = C{0, 0};
                    }
                }
                R tb = 0, tc = 0;  // tip/tilt of the star
                if (tt_sum) {
                    R sb = 0, scs = 0;
                    for (int a0 = 0;;) {
#pragma unroll
                        for (int u = 0; u < QC; ++u) {
                            sb += pb[u];
                            scs += pc[u];
                        }
                        a0 += LW * QC;
                        if (a0 >= P) break;
                        load_shares(a0);  // rows beyond the first batch (P > LW * QC)
                    }
#pragma unroll
                    for (int off = LW / 2; off > 0; off >>= 1) {
                        sb += __shfl_xor_sync(0xffffffffu, sb, off);
                        scs += __shfl_xor_sync(0xffffffffu, scs, off);
                    }
                    if (tt && c == 0 && t == 0) {  // for this CTA's later passes
                        s_ttb[ss] = sb;
                        s_ttc[ss] = scs;
                    }
                    tb = sb;
                    tc = scs;
                } else if (tt) {
                    tb = s_ttb[ss];
                    tc = s_ttc[ss];
                }
                __syncwarp();
                wfft_fwd<M>(v, tw, t);
                if (tt) {  // d_g -= b_g X(j, k) + c_g Y(j, k)
#pragma unroll
                    for (int r = 0; r < RR; ++r) {
                        const int pos = r * LW + t;
                        C xh, yh;
                        if (first && c == 0 && xy_pre) {  // column b's spectra came with the prologue
                            xh = xys[pos];
                            yh = xys[M + pos];
                        } else {
                            xh = fp.xy_hat[((size_t)k << LOGM) + pos];
                            yh = fp.xy_hat[((size_t)(Mh + k) << LOGM) + pos];
                        }
                        v[r].x -= tb * xh.x + tc * yh.x;
                        v[r].y -= tb * xh.y + tc * yh.y;
                    }
                }
                if (act)
#pragma unroll
                    for (int r = 0; r < RR; ++r) Dp[((size_t)c * G + ss) * M + r * LW + t] = v[r];
            }
            SAFR_MARK(8, first);
            __syncthreads();
            SAFR_MARK(9, first);
            if (fp.stage_b) {  // one column per pass (ck = 1)
                if (tid == 0) bar_flag = mbar_wait_bounded(&mbar, bph, fp.timeout_ns, fp.status) ? 1 : -1;
                __syncthreads();
                tma_pending = false;
                bph ^= 1u;
                if (bar_flag < 0) return false;  // the copy never landed: nothing in flight any more to wait for
            }
            SAFR_MARK(10, first);
            // one transform slot per (column, group, LPS layers): b_l = sum_g B_lg d_g (permuted j)
            // for the slot's layers from one read of d_g, then the inverse FFTs along j
            const int per = (L + LPS - 1) / LPS, nslot = fp.ngroups * per, ntask2 = ncols * nslot;
            for (int u0 = 0; u0 < ntask2; u0 += UNITS) {
                const int task = u0 + unit;
                const bool act = task < ntask2;
                if (!__any_sync(0xffffffffu, act)) continue;
                const int tk = act ? task : 0, c = tk / nslot, ptk = tk - c * nslot, k = kb + c * nb;
                const int gi = ptk >= per ? 1 : 0, l0 = LPS * (ptk - gi * per);
                const int nl = min(LPS, L - l0);
                const int gG = s_grp[gi].G;
                const C *Bcol = fp.stage_b ? Bs : fp.B + (size_t)k * colB;
                const C *Bl = Bcol + ((size_t)(s_grp[gi].b_row0 + l0 * gG) << LOGM);
                const C *Dc = Dp + (size_t)c * G * M;
                C v[LPS][RR];
#pragma unroll
                for (int q = 0; q < LPS; ++q)
#pragma unroll
                    for (int r = 0; r < RR; ++r) v[q][r] = C{0, 0};
                // B from shared memory (staged) or from global memory, through generic loads: one copy of
                // the code for both (measured 0.2 us faster per MORFEO-like frame, 1.3 us on the 512 grid,
                // than two copies specialised by ld.shared and ld.global.cg)
                auto apply = [&](auto loadB) {
                    for (int gg = 0; gg < gG; ++gg) {
                        const C *Dg = Dc + (size_t)s_grp[gi].star[gg] * M;
#pragma unroll
                        for (int r = 0; r < RR; ++r) {
                            const int pos = r * LW + t;
                            const C dv = Dg[pos];
#pragma unroll
                            for (int q = 0; q < LPS; ++q) {
                                const C bv = loadB(((size_t)(gg + (q < nl ? q : 0) * gG) << LOGM) + pos);
                                v[q][r].x += bv.x * dv.x - bv.y * dv.y;
                                v[q][r].y += bv.x * dv.y + bv.y * dv.x;
                            }
                        }
                    }
                };
                apply([&](size_t i) { return Bl[i]; });
                SAFR_MARK(11, first && u0 == 0);
                if (fp.energy) {  // Parseval partial sums of |b_l(j, k)|^2 over j
#pragma unroll
                    for (int q = 0; q < LPS; ++q) {
                        R e = 0;
#pragma unroll
                        for (int r = 0; r < RR; ++r) e += v[q][r].x * v[q][r].x + v[q][r].y * v[q][r].y;
#pragma unroll
                        for (int off = LW / 2; off > 0; off >>= 1) e += __shfl_xor_sync(0xffffffffu, e, off);
                        if (act && t == 0 && q < nl)
                            fp.energy[((size_t)gi * L + l0 + q) * Mh + k] = (float)(k == 0 ? e : R(2) * e);
                    }
                }
                // the slot's layers: their transforms interleaved
                wfft_inv_n<M, LPS>(v, tw, t);
#pragma unroll
                for (int q = 0; q < LPS; ++q)
                    if (act && q < nl) {
                        C *dst = fp.w2 + ((((size_t)gi * L + l0 + q) * Mh + k) << LOGM);
#pragma unroll
                        for (int r = 0; r < RR; ++r) dst[t + LW * r] = v[q][r];
                    }
                SAFR_MARK(12, first && u0 == 0);
            }
            SAFR_MARK(13, first);
            // next pass of this CTA: B block and column spectra are free once every warp is done
            if (kb + CK * nb < Mh) {
                __syncthreads();
                if (fp.stage_b) {
                    if (tid == 0) {
                        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                        copy_b(kb + nb);
                    }
                    tma_pending = true;
                }
            }
        }
    }
    SAFR_MARK(14, true);
    if (!grid_sync_bounded(fp.bar, bar_next + (unsigned long long)nb, fp.status, fp.timeout_ns, &bar_flag,
                           stamp ? stamp + 15 : nullptr)) {
        drain();
        return false;
    }
    SAFR_MARK(16, true);

    // ---- phase 3: (layer, row tile) ----------------------------------------------
    {
        const int RT = fp.rt3;
        const int st0 = fp.st3[0], st1 = fp.st3[1];
        // staged rows: column k's run of source rows starts at k * st + skew(k); the skew
        // spreads the permuted-order reads of the row transforms over the banks
        C *stg0 = (C *)s3;                                      // [Mh][st0]
        C *stg1 = stg0 + (size_t)Mh * st0;                      // [Mh][st1]
        C *Z = stg1 + (size_t)Mh * st1;                         // [cap3][M] inverse row transforms
        const bool two = fp.ngroups > 1;
        constexpr int KW = (Mh + NW - 1) / NW;  // staged columns per warp
        // M >= 512 without a resample: an item's staging copies are issued while the previous
        // item stores (the staging buffers are free once its transforms are done)
        bool staged_ahead = false;
        for (int it = b; it < fp.n3; it += nb) {
            const int l = it / fp.tiles3, p0 = (it - l * fp.tiles3) * RT;
            const int nr = min(RT, M - p0);
            if (rs0 && !(it == b && rs_pre)) {  // tables of a later item (the first one came with the prologue)
                __syncthreads();
                for (int i = tid; i < M; i += NTH) {
                    ti0[i] = fp.rs_i0[l * M + i];
                    tfw[i] = fp.rs_w[l * M + i];
                }
            }
            __syncthreads();
            SAFR_MARK(17, it == b);
            const int first0 = rs0 ? ti0[p0] : p0;
            const int nsrc0 = rs0 ? ti0[p0 + nr - 1] + 2 - first0 : nr;
            const int nsrc1 = two ? nr : 0;  // the NGS group is never resampled
            const int npair = (nr + 1) >> 1;  // transforms per group: one per output row pair
            const int ntot = two ? 2 * npair : npair;
            if (nsrc0 > fp.nsrc3[0] || nsrc1 > fp.nsrc3[1] || ntot > fp.cap3) {  // sized on the host; never expected
                if (tid == 0) atomicExch(fp.status, (int)SAFR_ERR_DEVICE);
                cp_async_wait_all();
                staged_ahead = false;
                continue;
            }
            // stage the needed rows of every column, one warp per column k:
            // stg0[k][s] = w2[0][l][k][first0 + s], stg1[k][s] = w2[1][l][k][p0 + s],
            // as asynchronous copies: all of a lane's copies are in flight at once
            if (M < 512 || !staged_ahead) {
                const C *src0 = fp.w2 + (size_t)l * Mh * M;
                const C *src1 = fp.w2 + ((size_t)L + l) * Mh * M;
                for (int s = lane; s < nsrc0 || s < nsrc1; s += 32) {
#pragma unroll 4
                    for (int u = 0; u < KW; ++u) {
                        const int k = warp + NW * u;
                        const int sk = ((k / RR) >> 1) & 15;
                        if (k < Mh && s < nsrc0)
                            cp_async_el(stg0 + k * st0 + sk + s, src0 + ((size_t)k << LOGM) + ((first0 + s) & (M - 1)));
                        if (k < Mh && s < nsrc1) cp_async_el(stg1 + k * st1 + sk + s, src1 + ((size_t)k << LOGM) + p0 + s);
                    }
                }
            }
            // the power-of-two output scale of an FP16 layer (1 otherwise)
            auto out_scale = [&]() -> R {
                R inv_scale = R(1);
                if constexpr (std::is_same<TOUT, __half>::value) {
                    // layer energy sum_n |b(n)|^2 over the groups (fixed order) -> RMS = sqrt(energy) / M^2;
                    // scale = 2^round(log2 RMS): 2^(e-1) for RMS = f 2^e, f in [1/2, 1), rounded at f = 2^-1/2
                    R e = 0;
                    for (int gi = 0; gi < fp.ngroups; ++gi)
                        for (int k = tid; k < Mh; k += NTH) e += (R)__ldcg(fp.energy + ((size_t)gi * L + l) * Mh + k);
                    e = block_sum(e, red);
                    const float rms = sqrtf((float)e) / ((float)M * (float)M);
                    float sc = 1.0f;
                    if (rms > 0.0f && rms < INFINITY) {
                        int ex;
                        const float f = frexpf(rms, &ex);
                        sc = ldexpf(1.0f, f < 0.70710678f ? ex - 1 : ex);
                    }
                    inv_scale = (R)(1.0f / sc);
                    if (p0 == 0 && tid == 0) fp.out_scales[(size_t)fidx * L + l] = sc;
                }
                return inv_scale;
            };
            R inv_scale = R(1);
            if constexpr (M < 512) inv_scale = out_scale();  // while the staging copies are in flight
            cp_async_wait_all();
            __syncthreads();
            SAFR_MARK(18, it == b);
            // The spectrum of output row pair r = 2i, 2i + 1 of a group, ready for its inverse
            // transform: Z[k] = X1[k] + i X2[k] over the full length M from the stored half
            // spectra, built directly in the permuted order.  An LGS row's spectrum is the
            // combination (1 - f) S[s] + f S[s + 1] of its two staged source rows.
            auto build_v = [&](bool g1, int i, bool act, C(&v)[RR]) {
                const C *sg = g1 ? stg1 : stg0;
                const int st = g1 ? st1 : st0;
                const bool hasb = 2 * i + 1 < nr;
                // frequency k < M/2 reads stored column k; k > M/2 reads column M - k (conjugate
                // symmetry); every lane loads from a valid address first, then selects
                constexpr int RB = RR < 8 ? RR : 8;  // values loaded per batch (bounds the registers at large M)
                if (!g1 && rs0) {  // warp-uniform: the LGS group's rows, resampled along p
                    const int ra = p0 + 2 * i, rb = hasb ? ra + 1 : ra;
                    const int sa = ti0[ra] - first0, sb = ti0[rb] - first0;
                    const R fa = tfw[ra], fb = tfw[rb];
#pragma unroll
                    for (int r0 = 0; r0 < RR; r0 += RB) {
                        C x1[RB], y1[RB], x2[RB], y2[RB];
#pragma unroll
                        for (int u = 0; u < RB; ++u) {
                            const int k = r0 + u + RR * bt;
                            const int kk = k < Mh ? k : (k > Mh ? M - k : 0);
                            const C *row = sg + kk * st + (((kk / RR) >> 1) & 15);
                            x1[u] = row[sa];
                            y1[u] = row[sa + 1];
                            x2[u] = row[sb];
                            y2[u] = row[sb + 1];
                        }
#pragma unroll
                        for (int u = 0; u < RB; ++u) {
                            const int k = r0 + u + RR * bt;
                            C a = C{(R(1) - fa) * x1[u].x + fa * y1[u].x, (R(1) - fa) * x1[u].y + fa * y1[u].y};
                            C c = hasb ? C{(R(1) - fb) * x2[u].x + fb * y2[u].x, (R(1) - fb) * x2[u].y + fb * y2[u].y}
                                       : C{0, 0};
                            if (k == 0) {
                                a.y = 0;
                                c.y = 0;
                            }
                            const C lo = C{a.x - c.y, a.y + c.x}, hi = C{a.x + c.y, c.x - a.y};
                            v[r0 + u] = !act || k == Mh ? C{0, 0} : (k < Mh ? lo : hi);
                        }
                    }
                } else {
                    const int ib = hasb ? 2 * i + 1 : 2 * i;
#pragma unroll
                    for (int r0 = 0; r0 < RR; r0 += RB) {
                        C x1[RB], x2[RB];
#pragma unroll
                        for (int u = 0; u < RB; ++u) {
                            const int k = r0 + u + RR * bt;
                            const int kk = k < Mh ? k : (k > Mh ? M - k : 0);
                            const C *row = sg + kk * st + (((kk / RR) >> 1) & 15);
                            x1[u] = row[2 * i];
                            x2[u] = row[ib];
                        }
#pragma unroll
                        for (int u = 0; u < RB; ++u) {
                            const int k = r0 + u + RR * bt;
                            C a = x1[u], c = hasb ? x2[u] : C{0, 0};
                            if (k == 0) {
                                a.y = 0;
                                c.y = 0;
                            }
                            const C lo = C{a.x - c.y, a.y + c.x}, hi = C{a.x + c.y, c.x - a.y};
                            v[r0 + u] = !act || k == Mh ? C{0, 0} : (k < Mh ? lo : hi);
                        }
                    }
                }
            };
            const R f = fp.inv_M2 * inv_scale;
            TOUT *outp = (TOUT *)fp.out + (((size_t)fidx * L + l) * M + p0) * M;
            auto put = [&](TOUT *dst, R val) {
                if constexpr (!std::is_same<TOUT, __half>::value)
                    if (fp.blend) val = (R(1) - fp.gain) * (R)*dst + fp.gain * val;
                if constexpr (std::is_same<TOUT, double>::value)
                    store_out_d(dst, (double)val);
                else
                    store_out<TOUT>(dst, (float)val);
            };
            if constexpr (M < 512) {
                // Units in pairs: with two groups, units 2m and 2m + 1 take row pair i of group 0 and
                // of group 1.  The group-0 unit leaves its rows in Z (row i); the group-1 unit, once the
                // pair has met at a barrier of its own (a named barrier of two warps, or the warp), adds
                // them (resampled along q for an LGS group) to its own rows and stores output rows 2i
                // and 2i + 1.  With one group every unit stores its own row pair (through Z when it is
                // resampled along q).  No block barrier separates the transforms from the stores.
                const int PR = two ? UNITS / 2 : UNITS;  // row pairs per round
                for (int i0 = 0; i0 < npair; i0 += PR) {
                    const int i = i0 + (two ? unit >> 1 : unit);
                    const bool act = i < npair;
                    if (!__any_sync(0xffffffffu, act)) continue;  // the same for both units of a pair
                    const bool g1 = two && (unit & 1);
                    const int ii = act ? i : 0;  // an idle unit reads row pair 0 (always staged)
                    C v[RR];
                    build_v(g1, ii, act, v);
                    wfft_inv<M>(v, tw, t);
                    C *zr = Z + (size_t)ii * M;
                    const bool storer = g1 || !two;
                    if (act && (two ? !storer : rs0))  // group 0's rows, or a resampled single group's own
#pragma unroll
                        for (int r = 0; r < RR; ++r) zr[t + LW * r] = v[r];
                    if (two) {
                        if constexpr (S::TPW == 1)
                            asm volatile("bar.sync %0, 64;" ::"r"(8 + (warp >> 1)) : "memory");
                        else
                            __syncwarp();
                    } else if (rs0) {
                        __syncwarp();
                    }
                    if (storer && act) {
                        // output row 2i is the real part, row 2i + 1 the imaginary part
                        TOUT *oa = outp + (size_t)(2 * ii) * M;
                        const bool hasb = 2 * ii + 1 < nr;
                        R e[RR], od[RR];
#pragma unroll
                        for (int r = 0; r < RR; ++r) {
                            const int q = t + LW * r;
                            if (rs0) {  // the column half of the bilinear resample (the row half was taken on the spectra)
                                const R fv = tfw[q];
                                const int j0u = ti0[q];
                                const C za = zr[j0u & (M - 1)], zb = zr[(j0u + 1) & (M - 1)];
                                e[r] = (R(1) - fv) * za.x + fv * zb.x;
                                od[r] = (R(1) - fv) * za.y + fv * zb.y;
                            } else if (two) {
                                const C z = zr[q];
                                e[r] = z.x;
                                od[r] = z.y;
                            } else {
                                e[r] = v[r].x;
                                od[r] = v[r].y;
                            }
                            if (two) {  // the NGS group's rows
                                e[r] += v[r].x;
                                od[r] += v[r].y;
                            }
                            e[r] *= f;
                            od[r] *= f;
                        }
                        if constexpr (!std::is_same<TOUT, __half>::value)
                            if (fp.blend) {  // the integrator: every old value is loaded before any store
                                R pa[RR], pb[RR];
#pragma unroll
                                for (int r = 0; r < RR; ++r) {
                                    pa[r] = (R)oa[t + LW * r];
                                    pb[r] = hasb ? (R)oa[M + t + LW * r] : R(0);
                                }
#pragma unroll
                                for (int r = 0; r < RR; ++r) {
                                    e[r] = (R(1) - fp.gain) * pa[r] + fp.gain * e[r];
                                    od[r] = (R(1) - fp.gain) * pb[r] + fp.gain * od[r];
                                }
                            }
#pragma unroll
                        for (int r = 0; r < RR; ++r) {
                            const int q = t + LW * r;
                            if constexpr (std::is_same<TOUT, double>::value) {
                                store_out_d(oa + q, (double)e[r]);
                                if (hasb) store_out_d(oa + M + q, (double)od[r]);
                            } else {
                                store_out<TOUT>(oa + q, (float)e[r]);
                                if (hasb) store_out<TOUT>(oa + M + q, (float)od[r]);
                            }
                        }
                    }
                }
                SAFR_MARK(19, it == b);
                SAFR_MARK(20, it == b);
            } else {
                for (int u0 = 0; u0 < ntot; u0 += UNITS) {
                    const int task = u0 + unit;
                    const bool act = task < ntot;
                    if (!__any_sync(0xffffffffu, act)) continue;
                    const int tk = act ? task : 0;  // an idle slot reads row pair 0 of group 0 (always staged)
                    const bool g1 = tk >= npair;
                    const int i = g1 ? tk - npair : tk;
                    C v[RR];
                    build_v(g1, i, act, v);
                    wfft_inv<M>(v, tw, t);
                    if (act)
#pragma unroll
                        for (int r = 0; r < RR; ++r) Z[(size_t)task * M + t + LW * r] = v[r];
                }
                SAFR_MARK(19, it == b);
                __syncthreads();
                SAFR_MARK(20, it == b);
                {  // the next item's rows, while this one stores (no resample: rows p0..)
                    staged_ahead = false;
                    const int itn = it + nb;
                    if (!rs0 && itn < fp.n3) {
                        const int ln = itn / fp.tiles3, p0n = (itn - ln * fp.tiles3) * RT, nrn = min(RT, M - p0n);
                        const int ns1 = two ? nrn : 0;
                        const C *src0 = fp.w2 + (size_t)ln * Mh * M;
                        const C *src1 = fp.w2 + ((size_t)L + ln) * Mh * M;
                        for (int s = lane; s < nrn || s < ns1; s += 32) {
#pragma unroll 4
                            for (int u = 0; u < KW; ++u) {
                                const int k = warp + NW * u;
                                const int sk = ((k / RR) >> 1) & 15;
                                if (k < Mh && s < nrn) cp_async_el(stg0 + k * st0 + sk + s, src0 + ((size_t)k << LOGM) + p0n + s);
                                if (k < Mh && s < ns1) cp_async_el(stg1 + k * st1 + sk + s, src1 + ((size_t)k << LOGM) + p0n + s);
                            }
                        }
                        staged_ahead = true;
                    }
                }
                inv_scale = out_scale();
                const R f3 = fp.inv_M2 * inv_scale;
                // output row r of a group is Z[r / 2] of that group (real part for even r, imaginary for odd)
                for (int idx = tid; idx < nr * M; idx += NTH) {
                    const int r = idx >> LOGM, q = idx & (M - 1);
                    const C *zr = Z + (size_t)(r >> 1) * M;
                    R v;
                    if (rs0) {  // the column half of the bilinear resample (the row half was taken on the spectra)
                        const R fv = tfw[q];
                        const int j0u = ti0[q];
                        const int ja = j0u & (M - 1), jb = (j0u + 1) & (M - 1);
                        const R a0 = (r & 1) ? zr[ja].y : zr[ja].x, a1 = (r & 1) ? zr[jb].y : zr[jb].x;
                        v = (R(1) - fv) * a0 + fv * a1;
                    } else {
                        v = (r & 1) ? zr[q].y : zr[q].x;
                    }
                    if (two) {  // the NGS group's rows follow group 0's pairs
                        const C zz = Z[(size_t)(npair + (r >> 1)) * M + q];
                        v += (r & 1) ? zz.y : zz.x;
                    }
                    put(outp + idx, v * f3);
                }
            }
            __syncthreads();
            SAFR_MARK(21, it == b);
        }
    }
    SAFR_MARK(22, true);
#undef SAFR_MARK
    return true;
}

__device__ __forceinline__ void bar_count_advance(unsigned long long *bar, unsigned long long base,
                                                  unsigned long long arrivals)
{
    if (blockIdx.x == 0 && threadIdx.x == 0)
        asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(bar + 1), "l"(base + arrivals) : "memory");
}

// One frame per launch; CK phase-2 columns per pass.  The launch of the next kernel in the stream
// may begin at once (its CTAs take the SMs this frame's CTAs leave, and it waits for this frame to
// finish before it touches its data).
template <int M, typename R, typename TIN, typename TOUT, int CK = 1>
__global__ void __launch_bounds__(frame2_threads(M), 1) k_frame2(const __grid_constant__ Frame2Params<R> fp)
{
    pdl_trigger();
    unsigned long long base = 0;
    unsigned bph = 0;
    if (frame_body<M, R, TIN, TOUT, CK>(fp, base, bph, 0u, true))
        bar_count_advance(fp.bar, base, 2ull * gridDim.x);
}

// `nframes` frames of one plan in one launch, one after the other (contiguous input and output
// arrays).  Each frame is the same sequence of three phases and two grid barriers; between frames
// there is no launch and no prologue wait: a CTA that finished frame f's last phase starts frame
// f + 1's first at once.  The workspaces need no second copy.  Frame f + 1 writes the row spectra
// after frame f's second grid barrier, which a CTA passes only once every CTA is done with frame f's
// column phase, their only reader; it writes the layer spectra after its own first grid barrier,
// which a CTA passes only once every CTA is done with frame f's last phase, their only reader.
template <int M, typename R, typename TIN, typename TOUT, int CK = 1>
__global__ void __launch_bounds__(frame2_threads(M), 1) k_frame2_frames(const __grid_constant__ Frame2Params<R> fp, int nframes)
{
    pdl_trigger();
    unsigned long long base = 0;
    unsigned bph = 0;
    for (int f = 0; f < nframes; ++f) {
        unsigned long long bf = base + 2ull * gridDim.x * (unsigned long long)f;  // frame 0 reads it
        if (!frame_body<M, R, TIN, TOUT, CK>(fp, bf, bph, (unsigned)(f & 1), f == 0, f)) return;
        if (f == 0) base = bf;
    }
    bar_count_advance(fp.bar, base, 2ull * gridDim.x * (unsigned long long)nframes);
}

// ----------------------------------------------------------------------------
// host side (instantiated per precision)
// ----------------------------------------------------------------------------
template <int M, typename R>
struct Frame2Host {
    using C = typename Frame2Params<R>::C;
    using S = WShape<M>;

    // phase-3 staged-row stride: at least n, odd (conflict-free column reads)
    static int odd_at_least(int n) { return n | 1; }

    // Sizes the kernel for the plan; false if it cannot hold it.
    static bool configure(safr_plan_s *pl, int nsm, void *kernel)
    {
        const int Mh = M / 2, G = pl->G, L = pl->L;
        const size_t cs = sizeof(C), rs = sizeof(R);
        const size_t limit = 227 * 1024 - 1024;  // dynamic shared memory budget
        const int units = frame2_threads(M) / 32 * S::TPW;  // transforms in flight per CTA
        const int nb = nsm;
        auto al = [](size_t x) { return (x + 127) & ~(size_t)127; };
        if (G > SAFR_MAX_G) return false;
        // phase 1 / 2: B column block, column spectra, removeTT stash
        bool any_rs = false;
        for (int gi = 0; gi < pl->ngroups; ++gi) any_rs |= pl->grp[gi].resample;
        // resample tables and the twiddle table [M + LW] (both read for the whole kernel)
        const size_t rsb = (any_rs ? al((size_t)M * (4 + rs)) : 0) + al((size_t)(M + wfft_lanes(M)) * cs);
        const size_t colB = (size_t)pl->sumLG * M * cs;
        const size_t db = al((size_t)G * M * cs);
        const size_t xyb = pl->remove_tt ? al(2 * (size_t)M * cs) : 0;
        const bool stage = rsb + al(colB) + db + xyb <= limit;
        pl->f2_stage_b = stage ? 1 : 0;
        pl->f2_off_rs = 0;
        pl->f2_off_tw = (unsigned)(any_rs ? al((size_t)M * (4 + rs)) : 0);
        pl->f2_off_b = (unsigned)rsb;
        pl->f2_off_d = (unsigned)(rsb + (stage ? al(colB) : 0));
        // two phase-2 columns per pass: B read from global memory, CTAs with several columns,
        // and a kernel instance that has it (M >= 512)
        pl->f2_ck = (!stage && pl->f2_ck_allow && M >= 512 && Mh > nb && rsb + 2 * db + xyb <= limit) ? 2 : 1;
        pl->f2_off_xy = pl->f2_off_d + (unsigned)(pl->f2_ck * db);
        const size_t s12 = pl->f2_off_xy + xyb;
        if (s12 > limit) return false;
        // phase 3 tiles: every CTA takes ceil(items / grid) items one after the
        // other, each with ceil(pairs / units) rounds of transforms; minimise
        // rounds x (rows per item + about 4 rows of fixed cost + about 6 rows per
        // transform round)
        int best_rt = 0;
        size_t best_s3 = 0;
        long long best_cost = 0;
        int st[2] = {0, 0}, ns[2] = {0, 0};
        for (int rt = std::min(32, M); rt >= 2; rt -= 2) {
            if (pl->f2_rt_force > 0 && rt != pl->f2_rt_force) continue;  // a tile height the autotuner picked
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
                nsm_[gi] = mx + (mx & 1);  // staged source rows
            }
            const int cap3 = pl->ngroups * ((rt + 1) / 2);  // row-pair transforms of one item
            size_t s3 = rsb;
            for (int gi = 0; gi < pl->ngroups; ++gi) s3 += (size_t)Mh * odd_at_least(nsm_[gi] + 15) * cs;
            s3 += (size_t)cap3 * M * cs;
            s3 = al(s3);
            const long long items = (long long)L * ((M + rt - 1) / rt);
            const long long cost = ((items + nb - 1) / nb) * (rt + 4 + 6LL * ((cap3 + units - 1) / units));
            if (s3 <= limit && (best_rt == 0 || cost <= best_cost)) {
                best_cost = cost;
                best_rt = rt;
                best_s3 = s3;
                pl->f2_cap3 = cap3;
                for (int gi = 0; gi < 2; ++gi) {
                    ns[gi] = nsm_[gi];
                    st[gi] = gi < pl->ngroups ? odd_at_least(nsm_[gi] + 15) : 0;  // room for the skew
                }
            }
        }
        if (best_rt == 0) return false;
        pl->f2_off_s3 = (unsigned)rsb;
        const size_t total = std::max(s12, best_s3);
        pl->f2_smem = total;
        pl->f2_rt3 = best_rt;
        pl->f2_tiles3 = (M + best_rt - 1) / best_rt;
        pl->f2_n3 = L * pl->f2_tiles3;
        for (int gi = 0; gi < 2; ++gi) {
            pl->f2_st3[gi] = st[gi];
            pl->f2_nsrc3[gi] = ns[gi];
        }
        pl->f2_grid = nb;
        if (!smem_limit_allows(kernel, total)) return false;
        int occ = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kernel, frame2_threads(M), total) != cudaSuccess ||
            occ < 1) {
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
        fp.blend = pl->loop_blend;
        fp.gain = (R)pl->loop_gain;
        fp.polc_tab = pl->loop_polc_psi ? pl->d_polc : nullptr;
        fp.polc_psi = pl->loop_polc_psi;
        fp.off_rs = pl->f2_off_rs;
        fp.off_tw = pl->f2_off_tw;
        fp.off_b = pl->f2_off_b;
        fp.off_d = pl->f2_off_d;
        fp.off_xy = pl->f2_off_xy;
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
        for (int i = 0; i < 6; ++i) fp.tt_n[i] = (R)pl->tt_n[i];
        fp.tt_delta = (R)pl->delta;
        fp.mask_bits = pl->d_mask_bits;
        fp.mask_words = (pl->P + 31) / 32;
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

// Host-side table of the warp-FFT twiddles (WTw layout): W_M^(t k_r) at
// [k_r * LW + t] for k_r < M / LW, then W_LW^e at [M + e], from FP64.
inline void frame2_twiddles_impl(int M, std::vector<double> &re, std::vector<double> &im)
{
    const int LW = wfft_lanes(M), R = M / LW;
    re.assign(M + LW, 0.0);
    im.assign(M + LW, 0.0);
    const double pi = 3.14159265358979323846264338327950288;
    for (int k = 0; k < R; ++k)
        for (int t = 0; t < LW; ++t) {
            const long long e = ((long long)t * k) % M;
            re[k * LW + t] = std::cos(2.0 * pi * (double)e / M);
            im[k * LW + t] = -std::sin(2.0 * pi * (double)e / M);
        }
    for (int e = 0; e < LW; ++e) {
        re[M + e] = std::cos(2.0 * pi * (double)e / LW);
        im[M + e] = -std::sin(2.0 * pi * (double)e / LW);
    }
}

}  // namespace safr
