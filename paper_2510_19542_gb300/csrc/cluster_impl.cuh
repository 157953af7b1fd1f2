// Algorithm 1 for small grids (M <= 64) as ONE thread-block cluster per frame.
//
// A small frame is a chain of latencies, not of bytes: the 32-grid frame moves
// 64 KB.  The persistent kernel spends most of such a frame in its two grid
// barriers and in the round trips of the row and column spectra through L2.
// Here the whole frame stays on CS <= 16 SMs of one cluster (CS = min(16, M/2)):
// the spectra never leave shared memory, the CTAs exchange them through
// distributed shared memory, and the two exchange points are hardware cluster
// barriers.  Column k < M/2 belongs to CTA k mod CS (local column k / CS).
//
//   prologue  by bulk copy (cp.async.bulk) into shared memory: the warp-FFT
//             twiddles, the resample tables of every layer, the removeTT
//             spectra of this CTA's columns (tables barrier), and this CTA's
//             B column blocks when they fit (B barrier; else a bulk prefetch
//             to L2 and loads from global memory in the apply);
//   phase 1   row pairs i = c, c + CS, ... of the zero-padded wavefronts
//             (Section 2): z = psi_a0 + i psi_a0+1, forward FFT along q, split
//             into the two half spectra, and each value stored straight into
//             the shared memory of its column's CTA (st.shared::cluster: no
//             waiting on the remote side); LGS rows of a mixed plan also give
//             their shares of the tip and tilt of the least-squares plane
//             (Algorithm 3, line 3), summed per star in the CTA and sent to
//             every CTA;
//   cluster barrier;
//   phase 2   this CTA's columns k: per star, FFT along p of the gathered
//             column -> d_g(j, k); removeTT in the frequency domain (d_g -=
//             b_g X + c_g Y, X, Y = DFT2 of x and y on the mask); per (group,
//             two layers): b_l = sum_g B_lg d_g (Algorithm 1, line 5) into the
//             inverse FFT along j; the layer columns stay in shared memory;
//   cluster barrier;
//   phase 3   output row pairs (l, p0) strided over the CTAs: the row
//             spectra read from the column owners' shared memory (for an LGS
//             layer the row half of the bilinear resample taken on the
//             spectra), inverse FFT along q (IDFT2 with 1/M^2), the
//             column half of the resample, the sum of the groups (Algorithm 3,
//             line 4), optional FP16 with a power-of-two scale per layer from
//             its energy (Parseval), store;
//   cluster barrier (no CTA leaves while another still reads its spectra).
//
// The transforms are the warp FFTs of warpfft.cuh in the frequency order of
// freqorder.h, so B and the removeTT spectra are the same arrays the other
// schedules read.  The bulk-copy waits are bounded (SAFR_ERR_TIMEOUT in the
// status word); a CTA that gives up still runs every cluster barrier.
#pragma once

#include "frame_impl.cuh"

namespace safr {

template <typename R>
struct ClusterParams {
    using C = typename std::conditional<sizeof(R) == 8, double2, float2>::type;
    int P, L, G, o, ngroups, sumLG;
    int npr, n1;        // row pairs per star, phase-1 items (G * npr)
    int cs;             // CTAs of the cluster (= the grid)
    int slots1;         // phase-1 items per CTA: ceil(n1 / cs)
    int ncol;           // columns per CTA: (M / 2) / cs
    int tiles3, n3;     // phase-3 items (output row pairs) per layer (M / 2), items (L * tiles3)
    int ipr3;           // phase-3 items per round of transforms (one transform per group)
    int any_tt, any_resample, stage_b;
    unsigned long long timeout_ns;
    R inv_M2;
    // shared-memory carve-up (bytes from the dynamic base)
    unsigned off_tw, off_rs, off_xy, off_b, off_d1, off_tt, off_d, off_w2, off_e, off_sc, off_z;
    const void *in;
    const float *in_scales;
    void *out;
    float *out_scales;
    const C *B;                // [M/2][sumLG][M], j in the permuted order
    const C *twq;              // [M + LW] warp-FFT twiddles
    const int *rs_i0;          // [L][M]
    const R *rs_w;             // [L][M]
    R tt_n[6];                 // removeTT: w_b = mask (n0 + n1 x + n2 y), w_c = mask (n3 + n4 x + n5 y)
    R tt_delta;
    const unsigned *mask_bits; // [P][mask_words]
    int mask_words;
    const C *xy_hat;           // [2][M/2][M], j in the permuted order
    unsigned long long *stamps; // [cs][SAFR_TRACE_MARKS] %globaltimer marks of a traced frame, or null
    int *status;
    int star_tt[SAFR_MAX_G];
    GroupDev grp[2];
};

__device__ __forceinline__ unsigned cluster_rank()
{
    unsigned r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}

// the address of the same shared-memory byte in CTA `rank` of the cluster
__device__ __forceinline__ unsigned dsmem_map(unsigned local, unsigned rank)
{
    unsigned r;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(local), "r"(rank));
    return r;
}

template <typename C>
__device__ __forceinline__ C dsmem_ld_c(unsigned a);
template <>
__device__ __forceinline__ float2 dsmem_ld_c<float2>(unsigned a)
{
    float2 v;
    asm volatile("ld.shared::cluster.v2.f32 {%0, %1}, [%2];" : "=f"(v.x), "=f"(v.y) : "r"(a));
    return v;
}
template <>
__device__ __forceinline__ double2 dsmem_ld_c<double2>(unsigned a)
{
    double2 v;
    asm volatile("ld.shared::cluster.v2.f64 {%0, %1}, [%2];" : "=d"(v.x), "=d"(v.y) : "r"(a));
    return v;
}

__device__ __forceinline__ void dsmem_st_c(unsigned a, float2 v)
{
    asm volatile("st.shared::cluster.v2.f32 [%0], {%1, %2};" ::"r"(a), "f"(v.x), "f"(v.y) : "memory");
}
__device__ __forceinline__ void dsmem_st_c(unsigned a, double2 v)
{
    asm volatile("st.shared::cluster.v2.f64 [%0], {%1, %2};" ::"r"(a), "d"(v.x), "d"(v.y) : "memory");
}
__device__ __forceinline__ void dsmem_st_r(unsigned a, float v)
{
    asm volatile("st.shared::cluster.f32 [%0], %1;" ::"r"(a), "f"(v) : "memory");
}
__device__ __forceinline__ void dsmem_st_r(unsigned a, double v)
{
    asm volatile("st.shared::cluster.f64 [%0], %1;" ::"r"(a), "d"(v) : "memory");
}
__device__ __forceinline__ float dsmem_ld_f(unsigned a)
{
    float v;
    asm volatile("ld.shared::cluster.f32 %0, [%1];" : "=f"(v) : "r"(a));
    return v;
}

// every thread of every CTA of the cluster (release: this thread's shared-memory writes, local and
// remote, are visible to the cluster after the wait; acquire: the others' writes to this thread)
__device__ __forceinline__ void cluster_barrier()
{
    asm volatile("barrier.cluster.arrive.release.aligned;" ::: "memory");
    asm volatile("barrier.cluster.wait.acquire.aligned;" ::: "memory");
}

__host__ __device__ constexpr int cluster_threads() { return 512; }

template <int M, typename R, typename TIN, typename TOUT>
__global__ void __launch_bounds__(cluster_threads(), 1) k_cluster(const __grid_constant__ ClusterParams<R> cp)
{
    using C = typename ClusterParams<R>::C;
    using S = WShape<M>;
    constexpr int LW = S::LW, RR = S::R, LB = S::LB, LOGM = S::LOG;
    constexpr int Mh = M / 2;
    constexpr int NTH = cluster_threads();
    constexpr int NW = NTH / 32;
    constexpr int UNITS = NW * S::TPW;  // transforms in flight per CTA
    constexpr int LPS = 2;              // layers per transform slot in the apply
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ __align__(8) uint64_t mbar_t, mbar_b;
    __shared__ int s_star_tt[SAFR_MAX_G];
    __shared__ GroupDev s_grp[2];
    __shared__ R s_ttb[SAFR_MAX_G], s_ttc[SAFR_MAX_G];
    __shared__ int s_flag;

    const int P = cp.P, o = cp.o, L = cp.L, G = cp.G, cs = cp.cs, ng = cp.ngroups;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int c = (int)cluster_rank();
    const int t = lane & (LW - 1);
    const int unit = warp * S::TPW + (lane >> LB);
    const int bt = LB > 0 ? (int)(__brev((unsigned)t) >> (32 - LB)) : 0;

    C *twq_s = (C *)(smem + cp.off_tw);          // [M + LW]
    int *ti0 = (int *)(smem + cp.off_rs);         // [L][M]
    R *tfw = (R *)(ti0 + (size_t)L * M);          // [L][M]
    C *xys = (C *)(smem + cp.off_xy);             // [ncol][2][M]
    C *Bs = (C *)(smem + cp.off_b);               // [ncol][sumLG][M]
    C *D1 = (C *)(smem + cp.off_d1);              // [ncol][G][P] row spectra of this CTA's columns
    R *ttp = (R *)(smem + cp.off_tt);             // [cs][G][2] tip/tilt partial sums from each CTA
    C *Dp = (C *)(smem + cp.off_d);               // [G][M] column spectra (permuted j)
    C *w2s = (C *)(smem + cp.off_w2);             // [ncol][ngroups][L][M] layer columns (natural p)
    float *eps = (float *)(smem + cp.off_e);      // [ncol][ngroups][L] layer energy of this CTA's columns
    R *isc = (R *)(smem + cp.off_sc);             // [L] inverse output scales (FP16 storage)
    C *Z = (C *)(smem + cp.off_z);                // [UNITS][M] inverse row transforms of a round
    const size_t colB = (size_t)cp.sumLG * M;
    const unsigned colB_bytes = (unsigned)(colB * sizeof(C));
    // trace marks (traced frames only): 0 start, 1 prologue issued, 2 phase-1 input in, 3 phase 1 done,
    // 4 barrier 1 passed, 5 first column's star transforms done, 6 B landed, 7 first column done,
    // 8 phase 2 done, 9 barrier 2 passed, 10 first phase-3 round transformed, 11 phase 3 done,
    // 12 last barrier passed, 13 thread 0's bulk copies issued, 15 first phase-3 round stored
    unsigned long long *stamp = cp.stamps ? cp.stamps + (size_t)c * SAFR_TRACE_MARKS : nullptr;
#define SAFR_CMARK(n)                               \
    do {                                            \
        if (stamp && tid == 0) stamp[n] = gtimer(); \
    } while (0)
    SAFR_CMARK(0);

    // ---- prologue ----------------------------------------------------------------
    if (tid == 0) {
        mbar_init(&mbar_t, 1);
        mbar_init(&mbar_b, 1);
        const unsigned tb = (unsigned)((M + LW) * sizeof(C));
        const unsigned rb = cp.any_resample ? (unsigned)((size_t)L * M * (4 + sizeof(R))) : 0u;
        const unsigned xb = cp.any_tt ? (unsigned)(cp.ncol * 2 * M * sizeof(C)) : 0u;
        mbar_expect_tx(&mbar_t, tb + rb + xb);
        tma_load_1d(twq_s, cp.twq, tb, &mbar_t);
        if (cp.any_resample) {
            tma_load_1d(ti0, cp.rs_i0, (unsigned)((size_t)L * M * 4), &mbar_t);
            tma_load_1d(tfw, cp.rs_w, (unsigned)((size_t)L * M * sizeof(R)), &mbar_t);
        }
        if (cp.any_tt)
            for (int q = 0; q < cp.ncol; ++q) {
                const int k = c + cs * q;
                tma_load_1d(xys + (size_t)q * 2 * M, cp.xy_hat + ((size_t)k << LOGM), (unsigned)(M * sizeof(C)),
                            &mbar_t);
                tma_load_1d(xys + (size_t)q * 2 * M + M, cp.xy_hat + ((size_t)(Mh + k) << LOGM),
                            (unsigned)(M * sizeof(C)), &mbar_t);
            }
        if (cp.stage_b) {
            mbar_expect_tx(&mbar_b, (unsigned)cp.ncol * colB_bytes);
            for (int q = 0; q < cp.ncol; ++q) {
                const int k = c + cs * q;
                const unsigned char *src = (const unsigned char *)(cp.B + (size_t)k * colB);
                unsigned char *dst = (unsigned char *)(Bs + (size_t)q * colB);
                for (unsigned off = 0; off < colB_bytes; off += 32768u)
                    tma_load_1d(dst + off, src + off, min(32768u, colB_bytes - off), &mbar_b);
            }
        }
        if (stamp) stamp[13] = gtimer();
    } else if (warp == 2) {  // the __grid_constant__ parameter read in place: one round of loads
        for (int i = lane; i < SAFR_MAX_G; i += 32) s_star_tt[i] = cp.star_tt[i];
    } else if (warp == 3) {
        const int *src = reinterpret_cast<const int *>(&cp.grp[0]);
        int *dst = reinterpret_cast<int *>(&s_grp[0]);
        constexpr int NWD = (int)(2 * sizeof(GroupDev) / sizeof(int));
        for (int i = lane; i < NWD; i += 32) dst[i] = src[i];
    }
    if (!cp.stage_b)  // this CTA's B columns, into L2 while phase 1 runs
        for (int q = 0; q < cp.ncol; ++q) {
            const char *base = (const char *)(cp.B + (size_t)(c + cs * q) * colB);
            for (unsigned off = (unsigned)tid * 4096u; off < colB_bytes; off += NTH * 4096u)
                prefetch_l2(base + off, min(4096u, colB_bytes - off));
        }
    for (int i = tid; i < cp.ncol * ng * L; i += NTH) eps[i] = 0.f;
    __syncthreads();  // mbarrier init, parameter copies
    SAFR_CMARK(1);
    if (stamp && tid == 0)
        for (int i = 2; i < SAFR_TRACE_MARKS; ++i)
            if (i != 13) stamp[i] = 0;  // 13 is thread 0's own, already taken

    WTw<M, C> tw;
    auto tables = [&]() {
        mbar_wait_bounded(&mbar_t, 0u, cp.timeout_ns, cp.status);
        tw.load(twq_s, t);
    };
    const unsigned d1_base = smem_u32(D1), tt_base = smem_u32(ttp), w2_base = smem_u32(w2s);

    // ---- phase 1: row pairs c, c + cs, ... -> the columns' CTAs -----------------------
    {
        R *tts = (R *)Z;  // [slots1][4] this CTA's per-item shares (Z is free until phase 3)
        bool first = true;
        for (int base = 0; base < cp.slots1; base += UNITS) {
            const int s = base + unit;
            const int i = c + cs * s;
            const bool act = s < cp.slots1 && i < cp.n1;
            if (!__any_sync(0xffffffffu, act)) continue;
            const int item = act ? i : 0, g = item / cp.npr, a0 = 2 * (item - g * cp.npr);
            const bool has1 = a0 + 1 < P;
            const int a1 = has1 ? a0 + 1 : a0;
            const TIN *psi = (const TIN *)cp.in + (size_t)g * P * P;
            const R sc = cp.in_scales ? (R)cp.in_scales[g] : R(1);
            const bool tt = act && cp.any_tt && s_star_tt[g];
            C v[RR];
            R s0b = 0, s0c = 0, s1b = 0, s1c = 0;
            {
                const unsigned *mb0 = cp.mask_bits + (size_t)a0 * cp.mask_words;
                const unsigned *mb1 = cp.mask_bits + (size_t)a1 * cp.mask_words;
                R x0[RR], x1[RR];
                unsigned m0[RR], m1[RR];
#pragma unroll
                for (int r = 0; r < RR; ++r) {  // loads from clamped in-range addresses first
                    const int qc = min(max(t + LW * r - o, 0), P - 1);
                    x0[r] = load_in<R>(psi + (size_t)a0 * P + qc);
                    x1[r] = load_in<R>(psi + (size_t)a1 * P + qc);
                    m0[r] = tt ? mb0[qc >> 5] : 0u;
                    m1[r] = tt ? mb1[qc >> 5] : 0u;
                }
                R S00 = 0, S01 = 0, S10 = 0, S11 = 0;
                const R half = R(0.5) * (R)(P - 1);
#pragma unroll
                for (int r = 0; r < RR; ++r) {
                    const int qq = t + LW * r - o;
                    const bool in = act && qq >= 0 && qq < P;
                    v[r] = C{in ? x0[r] * sc : R(0), in && has1 ? x1[r] * sc : R(0)};
                    if (tt) {
                        const int qc = min(max(qq, 0), P - 1);
                        const R y = ((R)qc - half) * cp.tt_delta;
                        const R k0 = ((m0[r] >> (qc & 31)) & 1u) ? v[r].x : R(0);
                        const R k1 = ((m1[r] >> (qc & 31)) & 1u) ? v[r].y : R(0);
                        S00 += k0;
                        S01 += y * k0;
                        S10 += k1;
                        S11 += y * k1;
                    }
                }
                if (tt) {  // shares of the two linear functionals (as in the persistent kernel)
                    const R xa0 = ((R)a0 - half) * cp.tt_delta, xa1 = ((R)a1 - half) * cp.tt_delta;
                    s0b = (cp.tt_n[0] + cp.tt_n[1] * xa0) * S00 + cp.tt_n[2] * S01;
                    s0c = (cp.tt_n[3] + cp.tt_n[4] * xa0) * S00 + cp.tt_n[5] * S01;
                    s1b = (cp.tt_n[0] + cp.tt_n[1] * xa1) * S10 + cp.tt_n[2] * S11;
                    s1c = (cp.tt_n[3] + cp.tt_n[4] * xa1) * S10 + cp.tt_n[5] * S11;
                }
            }
            if (cp.any_tt) {
#pragma unroll
                for (int off = LW / 2; off > 0; off >>= 1) {
                    s0b += __shfl_xor_sync(0xffffffffu, s0b, off);
                    s0c += __shfl_xor_sync(0xffffffffu, s0c, off);
                    s1b += __shfl_xor_sync(0xffffffffu, s1b, off);
                    s1c += __shfl_xor_sync(0xffffffffu, s1c, off);
                }
                if (act && t == 0) {
                    tts[(size_t)s * 2] = tt ? s0b + (has1 ? s1b : R(0)) : R(0);
                    tts[(size_t)s * 2 + 1] = tt ? s0c + (has1 ? s1c : R(0)) : R(0);
                }
            }
            if (first) {
                SAFR_CMARK(2);
                tables();
            }
            first = false;
            wfft_fwd<M>(v, tw, t);
            // Z[k] in register k_r of lane t for k = k_r + R brev(t); the partner Z[M - k] as in the
            // persistent kernel's phase 1.  Even lanes hold k < M/2.
            C zc[RR];
            {
                const int src = LB > 0 ? (int)(__brev((unsigned)((LW - bt) & (LW - 1))) >> (32 - LB)) : 0;
                zc[0] = C{__shfl_sync(0xffffffffu, v[0].x, src, LW), __shfl_sync(0xffffffffu, v[0].y, src, LW)};
            }
#pragma unroll
            for (int k = 1; k < RR; ++k) zc[k] = shfl_xor_c(v[RR - k], LW - 1);
            if (act && (t & 1) == 0) {
#pragma unroll
                for (int k = 0; k < RR; ++k) {  // X_a0[kk], X_a0+1[kk] -> D1[kk / cs][g][a0 (+1)] of CTA kk mod cs
                    const int kk = k + RR * bt;
                    const C z = v[k], w = zc[k];
                    const unsigned rk = (unsigned)(kk % cs);
                    const unsigned a = d1_base + (unsigned)((((size_t)(kk / cs) * G + g) * P + a0) * sizeof(C));
                    dsmem_st_c(dsmem_map(a, rk), C{R(0.5) * (z.x + w.x), R(0.5) * (z.y - w.y)});
                    if (has1) dsmem_st_c(dsmem_map(a + (unsigned)sizeof(C), rk), C{R(0.5) * (z.y + w.y), R(0.5) * (w.x - z.x)});
                }
            }
        }
        if (first) tables();  // a warp without phase-1 rows
        if (cp.any_tt) {  // this CTA's tip/tilt partial sums per star -> every CTA
            __syncthreads();
            for (int idx = tid; idx < cs * G; idx += NTH) {
                const int gg = idx % G, dst = idx / G;
                R sb = 0, sc2 = 0;
                for (int s = 0; s < cp.slots1; ++s) {
                    const int it = c + cs * s;
                    if (it < cp.n1 && it / cp.npr == gg) {
                        sb += tts[(size_t)s * 2];
                        sc2 += tts[(size_t)s * 2 + 1];
                    }
                }
                const unsigned a = tt_base + (unsigned)((((size_t)c * G + gg) * 2) * sizeof(R));
                dsmem_st_r(dsmem_map(a, (unsigned)dst), sb);
                dsmem_st_r(dsmem_map(a + (unsigned)sizeof(R), (unsigned)dst), sc2);
            }
        }
    }
    SAFR_CMARK(3);
    cluster_barrier();
    SAFR_CMARK(4);

    // ---- phase 2: columns c, c + cs, ... ---------------------------------------------
    if (cp.any_tt) {  // tip and tilt of each LGS star: the CTAs' partial sums, in a fixed order
        for (int gg = tid; gg < G; gg += NTH) {
            R sb = 0, sc2 = 0;
            for (int cc = 0; cc < cs; ++cc) {
                sb += ttp[((size_t)cc * G + gg) * 2];
                sc2 += ttp[((size_t)cc * G + gg) * 2 + 1];
            }
            s_ttb[gg] = sb;
            s_ttc[gg] = sc2;
        }
        __syncthreads();
    }
    for (int q = 0; q < cp.ncol; ++q) {
        const int k = c + cs * q;
        // one transform per star: its row spectra at column k (stored here in phase 1), FFT along p
        for (int s0 = 0; s0 < G; s0 += UNITS) {
            const int ss = s0 + unit;
            const bool act = ss < G;
            if (!__any_sync(0xffffffffu, act)) continue;
            const int st = act ? ss : 0;
            const C *col = D1 + ((size_t)q * G + st) * P;
            C v[RR];
#pragma unroll
            for (int r = 0; r < RR; ++r) {
                const int pp = t + LW * r - o;
                v[r] = (act && pp >= 0 && pp < P) ? col[pp] : C{0, 0};
            }
            const bool tt = cp.any_tt && act && s_star_tt[st];
            const R tb = tt ? s_ttb[st] : R(0), tc = tt ? s_ttc[st] : R(0);
            wfft_fwd<M>(v, tw, t);
            if (tt) {  // d_g -= b_g X(j, k) + c_g Y(j, k)
                const C *X = xys + (size_t)q * 2 * M;
#pragma unroll
                for (int r = 0; r < RR; ++r) {
                    const int pos = r * LW + t;
                    const C xh = X[pos], yh = X[M + pos];
                    v[r].x -= tb * xh.x + tc * yh.x;
                    v[r].y -= tb * xh.y + tc * yh.y;
                }
            }
            if (act)
#pragma unroll
                for (int r = 0; r < RR; ++r) Dp[(size_t)st * M + r * LW + t] = v[r];
        }
        if (q == 0) SAFR_CMARK(5);
        if (cp.stage_b && q == 0) {
            if (tid == 0) s_flag = mbar_wait_bounded(&mbar_b, 0u, cp.timeout_ns, cp.status) ? 1 : 0;
        }
        __syncthreads();  // the column spectra (and, for the first column, the landed B blocks)
        if (q == 0) SAFR_CMARK(6);
        // one slot per (group, LPS layers): b_l = sum_g B_lg d_g, then the inverse FFTs along j
        const int per = (L + LPS - 1) / LPS, nslot = ng * per;
        const C *Bcol = cp.stage_b ? Bs + (size_t)q * colB : cp.B + (size_t)k * colB;
        for (int u0 = 0; u0 < nslot; u0 += UNITS) {
            const int task = u0 + unit;
            const bool act = task < nslot;
            if (!__any_sync(0xffffffffu, act)) continue;
            const int tk = act ? task : 0;
            const int gi = tk >= per ? 1 : 0, l0 = LPS * (tk - gi * per);
            const int nl = min(LPS, L - l0);
            const int gG = s_grp[gi].G;
            const C *Bl = Bcol + ((size_t)(s_grp[gi].b_row0 + l0 * gG) << LOGM);
            C v[LPS][RR];
#pragma unroll
            for (int qq = 0; qq < LPS; ++qq)
#pragma unroll
                for (int r = 0; r < RR; ++r) v[qq][r] = C{0, 0};
            for (int gg = 0; gg < gG; ++gg) {
                const C *Dg = Dp + (size_t)s_grp[gi].star[gg] * M;
#pragma unroll
                for (int r = 0; r < RR; ++r) {
                    const int pos = r * LW + t;
                    const C dv = Dg[pos];
#pragma unroll
                    for (int qq = 0; qq < LPS; ++qq) {
                        const size_t bi = ((size_t)(gg + (qq < nl ? qq : 0) * gG) << LOGM) + pos;
                        const C bv = cp.stage_b ? Bl[bi] : __ldcg(Bl + bi);
                        v[qq][r].x += bv.x * dv.x - bv.y * dv.y;
                        v[qq][r].y += bv.x * dv.y + bv.y * dv.x;
                    }
                }
            }
            if constexpr (std::is_same<TOUT, __half>::value) {  // Parseval partial sums of |b_l(j, k)|^2 over j
#pragma unroll
                for (int qq = 0; qq < LPS; ++qq) {
                    R e = 0;
#pragma unroll
                    for (int r = 0; r < RR; ++r) e += v[qq][r].x * v[qq][r].x + v[qq][r].y * v[qq][r].y;
#pragma unroll
                    for (int off = LW / 2; off > 0; off >>= 1) e += __shfl_xor_sync(0xffffffffu, e, off);
                    if (act && t == 0 && qq < nl)
                        eps[((size_t)q * ng + gi) * L + l0 + qq] = (float)(k == 0 ? e : R(2) * e);
                }
            }
            wfft_inv_n<M, LPS>(v, tw, t);
#pragma unroll
            for (int qq = 0; qq < LPS; ++qq)
                if (act && qq < nl) {
                    C *dst = w2s + (((size_t)q * ng + gi) * L + l0 + qq) * M;
#pragma unroll
                    for (int r = 0; r < RR; ++r) dst[t + LW * r] = v[qq][r];
                }
        }
        __syncthreads();  // the column spectra are free for the next column
        if (q == 0) SAFR_CMARK(7);
    }
    SAFR_CMARK(8);
    cluster_barrier();
    SAFR_CMARK(9);

    // ---- phase 3: items (layer, tile of rows) c, c + cs, ... ------------------------------
    if constexpr (std::is_same<TOUT, __half>::value) {
        // layer energy over the whole spectrum (all CTAs' columns, fixed order) -> RMS = sqrt(E) / M^2;
        // scale = 2^round(log2 RMS): 2^(e-1) for RMS = f 2^e, f in [1/2, 1), rounded at f = 2^-1/2
        const unsigned e_base = smem_u32(eps);
        for (int l = tid; l < L; l += NTH) {
            float e = 0.f;
            for (int cc = 0; cc < cs; ++cc)
                for (int q = 0; q < cp.ncol; ++q)
                    for (int gi = 0; gi < ng; ++gi)
                        e += dsmem_ld_f(dsmem_map(e_base + (unsigned)((((size_t)q * ng + gi) * L + l) * 4), (unsigned)cc));
            const float rms = sqrtf(e) / ((float)M * (float)M);
            float sc = 1.0f;
            if (rms > 0.0f && rms < INFINITY) {
                int ex;
                const float f = frexpf(rms, &ex);
                sc = ldexpf(1.0f, f < 0.70710678f ? ex - 1 : ex);
            }
            isc[l] = (R)(1.0f / sc);
            if (c == 0) cp.out_scales[l] = sc;
        }
        __syncthreads();
    }
    const bool rs0 = s_grp[0].resample != 0;  // only an LGS group (group 0) is resampled
    const int mine3 = cp.n3 > c ? (cp.n3 - c + cs - 1) / cs : 0;
    for (int s0 = 0; s0 < mine3; s0 += cp.ipr3) {
        // one transform per (item, group): output rows p0, p0 + 1 of layer l.  Z[k] = X_p0[k] + i
        // X_p0+1[k] over the full length, the upper half by conjugate symmetry, in the permuted order,
        // each value read from its column's CTA; an LGS row's spectrum is (1 - f) S[s] + f S[s + 1]
        // of its two source rows
        {
            const int it = unit / ng, gi = unit - it * ng;
            const bool act = it < cp.ipr3 && s0 + it < mine3;
            if (__any_sync(0xffffffffu, act)) {
                const int j = c + cs * (act ? s0 + it : 0);
                const int l = j / cp.tiles3, p0 = 2 * (j - l * cp.tiles3);
                const bool rsm = gi == 0 && rs0;
                int ra0 = p0, ra1 = p0, rb0 = p0 + 1, rb1 = p0 + 1;
                R fa = 0, fb = 0;
                if (rsm) {
                    const int sa = ti0[(size_t)l * M + p0], sb = ti0[(size_t)l * M + p0 + 1];
                    ra0 = sa & (M - 1);
                    ra1 = (sa + 1) & (M - 1);
                    rb0 = sb & (M - 1);
                    rb1 = (sb + 1) & (M - 1);
                    fa = tfw[(size_t)l * M + p0];
                    fb = tfw[(size_t)l * M + p0 + 1];
                }
                C xa[RR], xb[RR], ya[RR], yb[RR];
#pragma unroll
                for (int r = 0; r < RR; ++r) {  // every remote load issued before any is used
                    const int kf = r + RR * bt;
                    const int kk = kf < Mh ? kf : (kf > Mh ? M - kf : 0);
                    const unsigned col = dsmem_map(
                        w2_base + (unsigned)(((((size_t)(kk / cs) * ng + gi) * L + l) * M) * sizeof(C)), (unsigned)(kk % cs));
                    xa[r] = dsmem_ld_c<C>(col + (unsigned)(ra0 * sizeof(C)));
                    xb[r] = dsmem_ld_c<C>(col + (unsigned)(rb0 * sizeof(C)));
                    if (rsm) {
                        ya[r] = dsmem_ld_c<C>(col + (unsigned)(ra1 * sizeof(C)));
                        yb[r] = dsmem_ld_c<C>(col + (unsigned)(rb1 * sizeof(C)));
                    }
                }
                C v[RR];
#pragma unroll
                for (int r = 0; r < RR; ++r) {
                    const int kf = r + RR * bt;
                    C a = xa[r], cc = xb[r];
                    if (rsm) {
                        a = C{(R(1) - fa) * xa[r].x + fa * ya[r].x, (R(1) - fa) * xa[r].y + fa * ya[r].y};
                        cc = C{(R(1) - fb) * xb[r].x + fb * yb[r].x, (R(1) - fb) * xb[r].y + fb * yb[r].y};
                    }
                    if (kf == 0) {
                        a.y = 0;
                        cc.y = 0;
                    }
                    const C lo = C{a.x - cc.y, a.y + cc.x}, hi = C{a.x + cc.y, cc.x - a.y};
                    v[r] = !act || kf == Mh ? C{0, 0} : (kf < Mh ? lo : hi);
                }
                wfft_inv<M>(v, tw, t);
                if (act)
#pragma unroll
                    for (int r = 0; r < RR; ++r) Z[(size_t)unit * M + t + LW * r] = v[r];
            }
        }
        __syncthreads();
        if (s0 == 0) SAFR_CMARK(10);
        // output rows p0 + r of the round's items: real part row p0, imaginary part row p0 + 1
        const int nit = min(cp.ipr3, mine3 - s0);
        for (int idx = tid; idx < nit * 2 * M; idx += NTH) {
            const int it = idx >> (LOGM + 1), r = (idx >> LOGM) & 1, qq = idx & (M - 1);
            const int j = c + cs * (s0 + it);
            const int l = j / cp.tiles3, p = 2 * (j - l * cp.tiles3) + r;
            const C *z0 = Z + (size_t)(it * ng) * M;
            R v;
            if (rs0) {  // the column half of the bilinear resample
                const int j0u = ti0[(size_t)l * M + qq];
                const R fv = tfw[(size_t)l * M + qq];
                const int ja = j0u & (M - 1), jb = (j0u + 1) & (M - 1);
                const R a0 = r ? z0[ja].y : z0[ja].x, a1 = r ? z0[jb].y : z0[jb].x;
                v = (R(1) - fv) * a0 + fv * a1;
            } else {
                v = r ? z0[qq].y : z0[qq].x;
            }
            if (ng > 1) v += r ? z0[M + qq].y : z0[M + qq].x;
            const R val = v * cp.inv_M2;
            TOUT *outp = (TOUT *)cp.out + ((size_t)l * M + p) * M + qq;
            if constexpr (std::is_same<TOUT, __half>::value) {
                store_out<TOUT>(outp, (float)(val * isc[l]));
            } else if constexpr (std::is_same<TOUT, double>::value) {
                store_out_d(outp, (double)val);
            } else {
                store_out<TOUT>(outp, (float)val);
            }
        }
        __syncthreads();
        if (s0 == 0) SAFR_CMARK(15);
    }
    SAFR_CMARK(11);
    cluster_barrier();  // every CTA's reads of the others' spectra are done
    SAFR_CMARK(12);
#undef SAFR_CMARK
}

// ----------------------------------------------------------------------------
// host side
// ----------------------------------------------------------------------------
template <int M, typename R>
struct ClusterHost {
    using C = typename ClusterParams<R>::C;
    using S = WShape<M>;

    static bool configure(safr_plan_s *pl, void *kernel)
    {
        if (M > 64 || pl->G > SAFR_MAX_G) return false;
        const int Mh = M / 2, G = pl->G, L = pl->L, P = pl->P, ng = pl->ngroups;
        const size_t cb = sizeof(C), rb = sizeof(R);
        auto al = [](size_t x) { return (x + 127) & ~(size_t)127; };
        bool any_rs = false;
        for (int gi = 0; gi < ng; ++gi) any_rs |= pl->grp[gi].resample;
        const int units = cluster_threads() / 32 * S::TPW;
        const int npr = (P + 1) / 2, n1 = G * npr;
        if (units < ng) return false;
        int dev = 0, optin = 0;
        if (cudaGetDevice(&dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess) {
            cudaGetLastError();
            return false;
        }
        cudaFuncAttributes fa;
        if (cudaFuncGetAttributes(&fa, kernel) != cudaSuccess) {
            cudaGetLastError();
            return false;
        }
        const size_t limit = (size_t)optin - fa.sharedSizeBytes;
        if (cudaFuncSetAttribute(kernel, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess)
            cudaGetLastError();
        // the largest cluster (a power of two dividing M/2, at most 16) that fits and can be scheduled
        for (int cs = std::min(16, Mh); cs >= 2; cs >>= 1) {
            const int ncol = Mh / cs, slots1 = (n1 + cs - 1) / cs;
            size_t off = 0;
            const size_t o_tw = off;
            off += al((size_t)(M + S::LW) * cb);
            const size_t o_rs = off;
            off += any_rs ? al((size_t)L * M * (4 + rb)) : 0;
            const size_t o_xy = off;
            off += pl->remove_tt ? al((size_t)ncol * 2 * M * cb) : 0;
            const size_t o_d1 = off;
            off += al((size_t)ncol * G * P * cb);
            const size_t o_tt = off;
            off += pl->remove_tt ? al((size_t)cs * G * 2 * rb) : 0;
            const size_t o_d = off;
            off += al((size_t)G * M * cb);
            const size_t o_w2 = off;
            off += al((size_t)ncol * ng * L * M * cb);
            const size_t o_e = off;
            off += al((size_t)ncol * ng * L * 4);
            const size_t o_sc = off;
            off += al((size_t)L * rb);
            const size_t o_z = off;
            off += al(std::max((size_t)units * M * cb, (size_t)slots1 * 2 * rb));  // also the phase-1 shares
            const size_t colB = (size_t)pl->sumLG * M * cb;
            const bool stage = off + al((size_t)ncol * colB) <= limit;
            const size_t o_b = off;
            const size_t total = off + (stage ? al((size_t)ncol * colB) : 0);
            if (total > limit) continue;
            if (!smem_limit_allows(kernel, total)) continue;
            cudaLaunchConfig_t cfg = {};
            cfg.gridDim = dim3(cs);
            cfg.blockDim = dim3(cluster_threads());
            cfg.dynamicSmemBytes = total;
            cudaLaunchAttribute attr[1];
            attr[0].id = cudaLaunchAttributeClusterDimension;
            attr[0].val.clusterDim.x = cs;
            attr[0].val.clusterDim.y = 1;
            attr[0].val.clusterDim.z = 1;
            cfg.attrs = attr;
            cfg.numAttrs = 1;
            int nclusters = 0;
            if (cudaOccupancyMaxActiveClusters(&nclusters, kernel, &cfg) != cudaSuccess || nclusters < 1) {
                cudaGetLastError();
                continue;
            }
            // preferred by SAFR_PATH_AUTO when phase 2 and phase 3 each take one round of transforms
            // per CTA: the kernel then trades the persistent kernel's grid barriers and L2 round trips
            // for a few SMs' worth of work (measured faster there; slower on larger frames, whose
            // work the persistent kernel spreads over every SM)
            const int ipr3 = units / ng;
            pl->cl_auto = (L * Mh + cs * ipr3 - 1) / (cs * ipr3) <= 1 && ncol * ng * ((L + 1) / 2) <= units ? 1 : 0;
            pl->cl_cs = cs;
            pl->cl_ncol = ncol;
            pl->cl_slots1 = slots1;
            pl->cl_stage_b = stage ? 1 : 0;
            const size_t offs[11] = {o_tw, o_rs, o_xy, o_b, o_d1, o_tt, o_d, o_w2, o_e, o_sc, o_z};
            for (int i = 0; i < 11; ++i) pl->cl_off[i] = (unsigned)offs[i];
            pl->cl_smem = total;
            return true;
        }
        return false;
    }

    static ClusterParams<R> params(safr_plan_s *pl, const void *in, const float *in_scales, void *out,
                                   float *out_scales)
    {
        ClusterParams<R> cp;
        memset(&cp, 0, sizeof(cp));
        cp.P = pl->P;
        cp.L = pl->L;
        cp.G = pl->G;
        cp.o = pl->o;
        cp.ngroups = pl->ngroups;
        cp.sumLG = pl->sumLG;
        cp.npr = (pl->P + 1) / 2;
        cp.n1 = pl->G * cp.npr;
        cp.cs = pl->cl_cs;
        cp.slots1 = pl->cl_slots1;
        cp.ncol = pl->cl_ncol;
        cp.tiles3 = M / 2;
        cp.n3 = pl->L * cp.tiles3;
        cp.ipr3 = (cluster_threads() / 32 * S::TPW) / pl->ngroups;
        cp.any_tt = pl->remove_tt;
        for (int gi = 0; gi < pl->ngroups; ++gi) cp.any_resample |= pl->grp[gi].resample ? 1 : 0;
        cp.stage_b = pl->cl_stage_b;
        cp.timeout_ns = pl->barrier_timeout_ns;
        cp.inv_M2 = (R)(1.0 / ((double)M * M));
        cp.off_tw = pl->cl_off[0];
        cp.off_rs = pl->cl_off[1];
        cp.off_xy = pl->cl_off[2];
        cp.off_b = pl->cl_off[3];
        cp.off_d1 = pl->cl_off[4];
        cp.off_tt = pl->cl_off[5];
        cp.off_d = pl->cl_off[6];
        cp.off_w2 = pl->cl_off[7];
        cp.off_e = pl->cl_off[8];
        cp.off_sc = pl->cl_off[9];
        cp.off_z = pl->cl_off[10];
        cp.in = in;
        cp.in_scales = in_scales;
        cp.out = out;
        cp.out_scales = out_scales;
        cp.B = (const C *)pl->d_B;
        cp.twq = (const C *)pl->d_twq;
        cp.rs_i0 = pl->d_rs_i0;
        cp.rs_w = (const R *)pl->d_rs_w;
        for (int i = 0; i < 6; ++i) cp.tt_n[i] = (R)pl->tt_n[i];
        cp.tt_delta = (R)pl->delta;
        cp.mask_bits = pl->d_mask_bits;
        cp.mask_words = (pl->P + 31) / 32;
        cp.xy_hat = (const C *)pl->d_xy_hat;
        cp.stamps = pl->trace ? pl->d_stamps : nullptr;
        cp.status = pl->d_status;
        for (int g = 0; g < pl->G; ++g) cp.star_tt[g] = pl->star_tt[g];
        for (int gi = 0; gi < pl->ngroups; ++gi) {
            cp.grp[gi].G = pl->grp[gi].G;
            cp.grp[gi].b_row0 = pl->grp[gi].b_row0;
            cp.grp[gi].resample = pl->grp[gi].resample ? 1 : 0;
            for (int q = 0; q < pl->grp[gi].G; ++q) cp.grp[gi].star[q] = pl->grp[gi].stars[q];
        }
        return cp;
    }

    static cudaError_t launch(void *kernel, safr_plan_s *pl, const void *in, const float *isc, void *out,
                              float *osc, cudaStream_t st)
    {
        ClusterParams<R> cp = params(pl, in, isc, out, osc);
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3(pl->cl_cs);
        cfg.blockDim = dim3(cluster_threads());
        cfg.dynamicSmemBytes = pl->cl_smem;
        cfg.stream = st;
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeClusterDimension;
        attr[0].val.clusterDim.x = pl->cl_cs;
        attr[0].val.clusterDim.y = 1;
        attr[0].val.clusterDim.z = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        void *args[] = {&cp};
        return cudaLaunchKernelExC(&cfg, kernel, args);
    }
};

}  // namespace safr
