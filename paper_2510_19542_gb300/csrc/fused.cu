// Algorithm 1 as ONE persistent cooperative kernel per frame.
//
// Every CTA of a grid that fills the GPU (all CTAs co-resident, cooperative
// launch) runs three phases separated by two grid-wide barriers:
//
//   prologue  each CTA streams the B columns it will use in phase 2 from HBM
//             into L2 (bulk prefetch), so the dominant byte stream overlaps
//             phase 1 and the first barrier;
//   phase 1   row pairs of the zero-padded wavefronts (Section 2): two real
//             rows per complex FFT along q, split into two half spectra
//             -> w1[g][k][p] (p contiguous, k < M/2).  For the LGS stars of
//             a mixed plan each row also contributes its share of the two
//             linear functionals that give the tip and tilt of the
//             least-squares plane (Algorithm 3, line 3);
//   phase 2   columns k: FFT along p of every star's column -> d_g(j, k);
//             removeTT in the frequency domain, d_g -= b_g X(j,k) + c_g Y(j,k)
//             with X, Y = DFT2 of x and y on the pupil mask (DFT2 is linear);
//             per frequency and layer b_l = sum_g B_lg d_g (Algorithm 1,
//             line 5); inverse FFT along j -> w2[group][l][k][p];
//   phase 3   (layer, row tile): complex-to-real inverse FFT of the source
//             rows (IDFT2, 1/M^2), bilinear resample of LGS layers from pitch
//             c_l*delta to delta, sum of the groups (Algorithm 3, line 4),
//             optional FP16 with a power-of-two scale from the layer energy
//             (Parseval), store.
//
// The barriers spin on a generation word with a time limit read from
// %globaltimer: a CTA that waits longer records SAFR_ERR_TIMEOUT in the plan's
// status word and leaves, so a broken barrier never hangs the GPU.
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <type_traits>

#include "common.cuh"
#include "fft.cuh"
#include "plan.h"

namespace safr {

template <typename R>
struct FusedParams {
    using C = typename std::conditional<sizeof(R) == 8, double2, float2>::type;
    int M, P, L, G, Mh, o, logM, ngroups, sumLG;
    int npr;       // row pairs per star
    int n1;        // phase-1 items (row pairs)
    int lchunk;    // layers per inverse-FFT batch in phase 2
    int rt3;       // output rows per phase-3 item
    int tiles3;    // row tiles per layer
    int n3;        // phase-3 items
    int sp3;       // source row pairs per group and item (max)
    int stage3;    // source rows staged per group and item (max)
    int any_tt;
    int any_resample;
    int skip_cta;  // test hook: this CTA leaves before the first barrier (-1: none)
    unsigned long long timeout_ns;
    R inv_M2;
    const void *in;
    const float *in_scales;
    void *out;
    float *out_scales;
    const C *B;           // [Mh][sumLG][M]
    C *w1;                // [G][Mh][P]
    C *w2;                // [ngroups][L][Mh][M]
    float *energy;        // [ngroups][L][Mh]
    const C *tw;          // [M]
    const int *rs_i0;     // [L][M]
    const R *rs_w;        // [L][M]
    const R *tt_w;        // [2][P][P]
    const C *xy_hat;      // [2][Mh][M] DFT2 of x*mask and y*mask (column k contiguous in j)
    R *pm;                // [G][P][2] per-row tip/tilt functionals
    unsigned *bar;        // [2] arrival count, generation
    unsigned long long *stamps;  // [gridDim][6] phase timestamps (traced calls only)
    int *status;
    int star_tt[SAFR_MAX_G];
    GroupDev grp[2];
};

__device__ __forceinline__ unsigned long long globaltimer_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Grid-wide barrier of a cooperative launch; false if it timed out.
__device__ __forceinline__ bool grid_barrier(unsigned *bar, int *status, unsigned long long timeout_ns, int *flag)
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
            const unsigned long long t0 = globaltimer_ns();
            while (*vgen == gen) {
                if (globaltimer_ns() - t0 > timeout_ns) {
                    atomicExch(status, (int)SAFR_ERR_TIMEOUT);
                    ok = 0;
                    break;
                }
                __nanosleep(64);
            }
        }
        __threadfence();
        *flag = ok;
    }
    __syncthreads();
    return *flag != 0;
}

template <typename R, typename TIN, typename TOUT, int GMAX>
__global__ void __launch_bounds__(512, 1) k_frame(FusedParams<R> fp)
{
    using C = typename FusedParams<R>::C;
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ int bar_flag;
    __shared__ R tt_b[SAFR_MAX_G], tt_c[SAFR_MAX_G];
    __shared__ R red[32];

    const int M = fp.M, P = fp.P, Mh = fp.Mh, o = fp.o, L = fp.L, logM = fp.logM, G = fp.G;
    const int tid = threadIdx.x, nth = blockDim.x, b = blockIdx.x, nb = gridDim.x;
    const int lane = tid & 31, warp = tid >> 5, nwarps = nth >> 5;
    unsigned long long *stamp = fp.stamps ? fp.stamps + (size_t)b * 6 : nullptr;
    if (stamp && tid == 0) stamp[0] = globaltimer_ns();
    C *tw = (C *)smem;
    C *work = tw + M;  // phase scratch starts after the twiddles

    // ---- prologue: B of this CTA's phase-2 columns into L2 -------------------
    {
        const size_t colbytes = (size_t)fp.sumLG * M * sizeof(C);
        for (int k = b; k < Mh; k += nb) {
            const char *base = (const char *)(fp.B + (size_t)k * fp.sumLG * M);
            for (size_t off = (size_t)tid * 4096; off < colbytes; off += (size_t)nth * 4096)
                prefetch_l2(base + off, (unsigned)min((size_t)4096, colbytes - off));
        }
    }
    for (int i = tid; i < M; i += nth) tw[i] = fp.tw[i];

    // ---- phase 1: row FFTs -------------------------------------------------
    {
        const int lo = (int)(((long long)b * fp.n1) / nb), hi = (int)(((long long)(b + 1) * fp.n1) / nb);
        const int cnt = hi - lo;
        C *bufA = work, *bufB = work + ((size_t)max(cnt, 1) << logM);
        for (int idx = tid; idx < (cnt << logM); idx += nth) {
            const int i = idx >> logM, q = idx & (M - 1);
            const int item = lo + i, g = item / fp.npr, a0 = 2 * (item - g * fp.npr);
            const int qq = q - o;
            R re = 0, im = 0;
            if (qq >= 0 && qq < P) {
                const TIN *psi = (const TIN *)fp.in + (size_t)g * P * P;
                const R sc = fp.in_scales ? (R)fp.in_scales[g] : R(1);
                re = load_in<R>(psi + (size_t)a0 * P + qq) * sc;
                if (a0 + 1 < P) im = load_in<R>(psi + (size_t)(a0 + 1) * P + qq) * sc;
            }
            bufA[idx] = C{re, im};
        }
        __syncthreads();
        // per-row shares of the tip/tilt functionals (one warp per row pair)
        if (fp.any_tt) {
            for (int i = warp; i < cnt; i += nwarps) {
                const int item = lo + i, g = item / fp.npr, a0 = 2 * (item - g * fp.npr);
                if (!fp.star_tt[g]) continue;
                const R *wb = fp.tt_w, *wc = fp.tt_w + (size_t)P * P;
                R s0b = 0, s0c = 0, s1b = 0, s1c = 0;
                for (int q = lane; q < P; q += 32) {
                    const C v = bufA[(i << logM) + o + q];
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
        }
        if (cnt > 0) {
            C *res = block_fft<false>(bufA, bufB, logM, cnt, M, tw, tid, nth);
            // X1 = (Z[k] + conj Z[M-k]) / 2, X2 = (Z[k] - conj Z[M-k]) / 2i; item fastest
            for (int idx = tid; idx < cnt * Mh; idx += nth) {
                const int k = idx / cnt, i = idx - k * cnt;
                const int item = lo + i, g = item / fp.npr, a0 = 2 * (item - g * fp.npr);
                const C z = res[(i << logM) + k];
                const C zc = res[(i << logM) + ((M - k) & (M - 1))];
                C *dst = fp.w1 + ((size_t)g * Mh + k) * P + a0;
                dst[0] = C{R(0.5) * (z.x + zc.x), R(0.5) * (z.y - zc.y)};
                if (a0 + 1 < P) dst[1] = C{R(0.5) * (z.y + zc.y), R(0.5) * (zc.x - z.x)};
            }
        }
    }
    if (b == fp.skip_cta) return;  // test hook: the others' first barrier must time out
    if (stamp) {
        __syncthreads();
        if (tid == 0) stamp[1] = globaltimer_ns();
    }
    if (!grid_barrier(fp.bar, fp.status, fp.timeout_ns, &bar_flag)) return;
    if (stamp && tid == 0) stamp[2] = globaltimer_ns();

    // ---- phase 2: columns --------------------------------------------------
    {
        if (fp.any_tt) {
            for (int g = warp; g < G; g += nwarps) {
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
        }
        const int W = max(G, fp.lchunk);
        C *dcol = work;                          // [G][M]
        C *bufA = dcol + ((size_t)G << logM);    // [W][M]
        C *bufB = bufA + ((size_t)W << logM);    // [W][M]
        for (int k = b; k < Mh; k += nb) {
            for (int idx = tid; idx < (G << logM); idx += nth) {
                const int t = idx >> logM, p = idx & (M - 1), pp = p - o;
                C v = C{0, 0};
                if (pp >= 0 && pp < P) v = __ldcg(fp.w1 + ((size_t)t * Mh + k) * P + pp);
                dcol[idx] = v;
            }
            __syncthreads();
            C *res = block_fft<false>(dcol, bufA, logM, G, M, tw, tid, nth);
            // copy back (and remove the LGS tip/tilt: d -= b X - c Y at this column)
            for (int idx = tid; idx < (G << logM); idx += nth) {
                const int t = idx >> logM, j = idx & (M - 1);
                C v = res[idx];
                if (fp.star_tt[t]) {
                    const C xh = fp.xy_hat[((size_t)k << logM) + j];
                    const C yh = fp.xy_hat[((size_t)(Mh + k) << logM) + j];
                    v.x -= tt_b[t] * xh.x + tt_c[t] * yh.x;
                    v.y -= tt_b[t] * xh.y + tt_c[t] * yh.y;
                }
                dcol[idx] = v;
            }
            __syncthreads();
            for (int gi = 0; gi < fp.ngroups; ++gi) {
                const GroupDev &gr = fp.grp[gi];
                const int Gg = gr.G;
                const C *Bk = fp.B + ((size_t)k * fp.sumLG + gr.b_row0) * M;
                for (int l0 = 0; l0 < L; l0 += fp.lchunk) {
                    const int lc = min(fp.lchunk, L - l0);
                    for (int idx = tid; idx < (lc << logM); idx += nth) {
                        const int l = idx >> logM, j = idx & (M - 1);
                        const C *Bj = Bk + ((size_t)(l0 + l) * Gg << logM) + j;
                        C bv[GMAX];
#pragma unroll
                        for (int t = 0; t < GMAX; ++t)
                            if (t < Gg) bv[t] = __ldg(Bj + ((size_t)t << logM));
                        R ar = 0, ai = 0;
#pragma unroll
                        for (int t = 0; t < GMAX; ++t)
                            if (t < Gg) {
                                const C d = dcol[(gr.star[t] << logM) + j];
                                ar += bv[t].x * d.x - bv[t].y * d.y;
                                ai += bv[t].x * d.y + bv[t].y * d.x;
                            }
                        bufA[idx] = C{ar, ai};
                    }
                    __syncthreads();
                    if (fp.energy) {
                        for (int l = warp; l < lc; l += nwarps) {
                            R e = 0;
                            for (int j = lane; j < M; j += 32) {
                                const C v = bufA[(l << logM) + j];
                                e += v.x * v.x + v.y * v.y;
                            }
                            for (int off = 16; off > 0; off >>= 1) e += __shfl_xor_sync(0xffffffffu, e, off);
                            if (lane == 0)
                                fp.energy[((size_t)gi * L + l0 + l) * Mh + k] = (float)(k == 0 ? e : R(2) * e);
                        }
                    }
                    res = block_fft<true>(bufA, bufB, logM, lc, M, tw, tid, nth);
                    for (int idx = tid; idx < (lc << logM); idx += nth) {
                        const int l = idx >> logM, p = idx & (M - 1);
                        fp.w2[((((size_t)gi * L + l0 + l) * Mh + k) << logM) + p] = res[idx];
                    }
                    __syncthreads();
                }
            }
        }
    }
    if (stamp) {
        __syncthreads();
        if (tid == 0) stamp[3] = globaltimer_ns();
    }
    if (!grid_barrier(fp.bar, fp.status, fp.timeout_ns, &bar_flag)) return;
    if (stamp && tid == 0) stamp[4] = globaltimer_ns();

    // ---- phase 3: rows -----------------------------------------------------
    {
        const int SP = fp.sp3, ST = fp.stage3, RT = fp.rt3;
        C *stage = work;                                 // [Mh][ST]
        C *bufA = stage + (size_t)Mh * ST;               // [SP][M]
        C *bufB = bufA + ((size_t)SP << logM);           // [SP][M]
        R *acc = (R *)(bufB + ((size_t)SP << logM));     // [RT][M]
        int *ti0 = (int *)(acc + ((size_t)RT << logM));  // [M]
        R *tfw = (R *)(ti0 + M);                         // [M]
        for (int it = b; it < fp.n3; it += nb) {
            const int l = it / fp.tiles3, p0 = (it - l * fp.tiles3) * RT;
            const int nr = min(RT, M - p0);
            if (fp.any_resample)
                for (int i = tid; i < M; i += nth) {
                    ti0[i] = fp.rs_i0[l * M + i];
                    tfw[i] = fp.rs_w[l * M + i];
                }
            for (int i = tid; i < (nr << logM); i += nth) acc[i] = 0;
            __syncthreads();
            for (int gi = 0; gi < fp.ngroups; ++gi) {
                const bool rs = fp.grp[gi].resample;
                const int first = rs ? ti0[p0] : p0;
                const int nsrc = rs ? ti0[p0 + nr - 1] + 2 - first : nr;
                const int npairs = (nsrc + 1) >> 1;
                if (npairs > SP || nsrc > ST) {  // sized on the host for every tile; never expected
                    if (tid == 0) atomicExch(fp.status, (int)SAFR_ERR_DEVICE);
                    break;
                }
                // stage the needed rows of every column: stage[k][s] = w2[gi][l][k][first + s]
                const C *src = fp.w2 + (((size_t)gi * L + l) * Mh << logM);
                for (int idx = tid; idx < Mh * nsrc; idx += nth) {
                    const int k = idx / nsrc, s = idx - k * nsrc;
                    stage[k * ST + s] = __ldcg(src + ((size_t)k << logM) + ((first + s) & (M - 1)));
                }
                __syncthreads();
                // Z[k] = X1[k] + i X2[k] over the full length M (Hermitian rows)
                for (int idx = tid; idx < (npairs << logM); idx += nth) {
                    const int i = idx >> logM, k = idx & (M - 1);
                    const bool hasb = 2 * i + 1 < nsrc;
                    C z = C{0, 0};
                    if (k < Mh) {
                        C x1 = stage[k * ST + 2 * i];
                        C x2 = hasb ? stage[k * ST + 2 * i + 1] : C{0, 0};
                        if (k == 0) {
                            x1.y = 0;
                            x2.y = 0;
                        }
                        z = C{x1.x - x2.y, x1.y + x2.x};
                    } else if (k > Mh) {
                        const int kk = M - k;
                        const C x1 = stage[kk * ST + 2 * i];
                        const C x2 = hasb ? stage[kk * ST + 2 * i + 1] : C{0, 0};
                        z = C{x1.x + x2.y, x2.x - x1.y};
                    }
                    bufA[idx] = z;
                }
                __syncthreads();
                const C *res = block_fft<true>(bufA, bufB, logM, npairs, M, tw, tid, nth);
                for (int idx = tid; idx < (nr << logM); idx += nth) {
                    const int r = idx >> logM, q = idx & (M - 1);
                    R v;
                    if (rs) {
                        const int i0 = ti0[p0 + r] - first;
                        const R fu = tfw[p0 + r];
                        const int j0u = ti0[q];
                        const R fv = tfw[q];
                        const int ja = j0u & (M - 1), jb = (j0u + 1) & (M - 1);
                        const C ra = res[((i0 >> 1) << logM) + ja], rb = res[((i0 >> 1) << logM) + jb];
                        const C sa = res[(((i0 + 1) >> 1) << logM) + ja], sb = res[(((i0 + 1) >> 1) << logM) + jb];
                        const R v00 = (i0 & 1) ? ra.y : ra.x, v01 = (i0 & 1) ? rb.y : rb.x;
                        const R v10 = ((i0 + 1) & 1) ? sa.y : sa.x, v11 = ((i0 + 1) & 1) ? sb.y : sb.x;
                        v = (R(1) - fu) * ((R(1) - fv) * v00 + fv * v01) + fu * ((R(1) - fv) * v10 + fv * v11);
                    } else {
                        const C c = res[((r >> 1) << logM) + q];
                        v = (r & 1) ? c.y : c.x;
                    }
                    acc[idx] += v;
                }
                __syncthreads();
            }
            R inv_scale = R(1);
            if (fp.out_scales) {
                // layer energy sum_n |b(n)|^2 over both groups (fixed order) -> mean square / M^4
                R e = 0;
                for (int gi = 0; gi < fp.ngroups; ++gi)
                    for (int k = tid; k < Mh; k += nth) e += (R)__ldcg(fp.energy + ((size_t)gi * L + l) * Mh + k);
                e = block_sum(e, red);
                const double ms = (double)e / ((double)M * M * (double)M * M);
                const double sc = ms > 0 ? exp2(rint(0.5 * log2(ms))) : 1.0;
                inv_scale = (R)(1.0 / sc);
                if (p0 == 0 && tid == 0) fp.out_scales[l] = (float)sc;
            }
            TOUT *out = (TOUT *)fp.out + ((size_t)l * M + p0) * M;
            const R f = fp.inv_M2 * inv_scale;
            for (int idx = tid; idx < (nr << logM); idx += nth) {
                if constexpr (std::is_same<TOUT, double>::value)
                    store_out_d(out + idx, (double)(acc[idx] * f));
                else
                    store_out<TOUT>(out + idx, (float)(acc[idx] * f));
            }
            __syncthreads();
        }
    }
    if (stamp && tid == 0) stamp[5] = globaltimer_ns();
}

// ----------------------------------------------------------------------------
// host side
// ----------------------------------------------------------------------------
template <typename R, typename TIN, typename TOUT>
static void *frame_kernel(int gmax)
{
    if (gmax == 4) return (void *)k_frame<R, TIN, TOUT, 4>;
    if (gmax == 8) return (void *)k_frame<R, TIN, TOUT, 8>;
    return (void *)k_frame<R, TIN, TOUT, 16>;
}

static void *frame_kernel_for(const safr_plan_s *pl)
{
    if (pl->precision == SAFR_FP64) return frame_kernel<double, double, double>(pl->gmax);
    if (pl->precision == SAFR_FP16_STORAGE) return frame_kernel<float, __half, __half>(pl->gmax);
    return frame_kernel<float, float, float>(pl->gmax);
}

// Shapes of the fused kernel and whether it can run at all (false: the plan
// uses the three-kernel path).
bool configure_fused(safr_plan_s *pl)
{
    const int M = pl->M, Mh = pl->Mh, P = pl->P, G = pl->G, L = pl->L;
    const size_t cs = pl->precision == SAFR_FP64 ? 16 : 8, rs = pl->precision == SAFR_FP64 ? 8 : 4;
    int dev = 0, nsm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return false;
    if (cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return false;
    int coop = 0;
    cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev);
    if (!coop) return false;
    const size_t limit = 220 * 1024;
    const int nb = nsm;  // one CTA per SM
    pl->f_grid = nb;
    pl->f_npr = (P + 1) / 2;
    pl->f_n1 = G * pl->f_npr;
    const int p1max = (pl->f_n1 + nb - 1) / nb;
    size_t s1 = 2 * (size_t)std::max(p1max, 1) * M * cs;
    // phase 2
    int lc = L;
    auto s2f = [&](int c) { return ((size_t)G * M + 2 * (size_t)std::max(G, c) * M) * cs; };
    while (lc > 1 && s2f(lc) + (size_t)M * cs > limit) --lc;
    pl->f_lchunk = lc;
    size_t s2 = s2f(lc);
    // phase 3: rows per item so that items roughly fill the grid, capped by smem
    int rt = (int)(((long long)L * M + nb - 1) / nb);
    rt = std::max(2, std::min(rt, 32));
    rt += rt & 1;
    size_t s3 = 0;
    for (;;) {
        int st = rt;  // rows staged per group
        for (int gi = 0; gi < pl->ngroups; ++gi) {
            if (!pl->grp[gi].resample) continue;
            for (int l = 0; l < L; ++l) {
                const double c = pl->grp[gi].c[l];
                for (int p0 = 0; p0 < M; p0 += rt) {
                    const int p1 = std::min(M, p0 + rt) - 1;
                    const int a = (int)std::floor(M / 2.0 + (p0 - M / 2.0) / c);
                    const int bq = (int)std::floor(M / 2.0 + (p1 - M / 2.0) / c);
                    st = std::max(st, bq + 2 - a);
                }
            }
        }
        const int sp = (st + 1) / 2;
        s3 = (size_t)Mh * st * cs + 2 * (size_t)sp * M * cs + (size_t)rt * M * rs + (size_t)M * (4 + rs);
        pl->f_rt3 = rt;
        pl->f_stage3 = st;
        pl->f_sp3 = sp;
        if (s3 + (size_t)M * cs <= limit || rt <= 2) break;
        rt -= 2;
    }
    pl->f_tiles3 = (M + pl->f_rt3 - 1) / pl->f_rt3;
    pl->f_n3 = L * pl->f_tiles3;
    pl->f_smem = (size_t)M * cs + std::max(s1, std::max(s2, s3));
    if (pl->f_smem > limit) return false;
    void *kern = frame_kernel_for(pl);
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)pl->f_smem) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    int occ = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, 512, pl->f_smem) != cudaSuccess || occ < 1) {
        cudaGetLastError();
        return false;
    }
    return true;
}

template <typename R>
static FusedParams<R> fused_params(safr_plan_s *pl, const void *in, const float *in_scales, void *out,
                                   float *out_scales)
{
    using C = typename FusedParams<R>::C;
    FusedParams<R> fp;
    memset(&fp, 0, sizeof(fp));
    fp.M = pl->M;
    fp.P = pl->P;
    fp.L = pl->L;
    fp.G = pl->G;
    fp.Mh = pl->Mh;
    fp.o = pl->o;
    int lm = 0;
    while ((1 << lm) < pl->M) ++lm;
    fp.logM = lm;
    fp.ngroups = pl->ngroups;
    fp.sumLG = pl->sumLG;
    fp.npr = pl->f_npr;
    fp.n1 = pl->f_n1;
    fp.lchunk = pl->f_lchunk;
    fp.rt3 = pl->f_rt3;
    fp.tiles3 = pl->f_tiles3;
    fp.n3 = pl->f_n3;
    fp.sp3 = pl->f_sp3;
    fp.stage3 = pl->f_stage3;
    fp.any_tt = pl->remove_tt;
    fp.any_resample = 0;
    for (int gi = 0; gi < pl->ngroups; ++gi) fp.any_resample |= pl->grp[gi].resample ? 1 : 0;
    fp.skip_cta = pl->debug_skip_cta;
    fp.timeout_ns = pl->barrier_timeout_ns;
    fp.inv_M2 = (R)(1.0 / ((double)pl->M * pl->M));
    fp.in = in;
    fp.in_scales = in_scales;
    fp.out = out;
    fp.out_scales = out_scales;
    fp.B = (const C *)pl->d_B;
    fp.w1 = (C *)pl->d_w1;
    fp.w2 = (C *)pl->d_w2;
    fp.energy = out_scales ? pl->d_energy : nullptr;
    fp.tw = (const C *)pl->d_tw;
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
        for (int t = 0; t < pl->grp[gi].G; ++t) fp.grp[gi].star[t] = pl->grp[gi].stars[t];
    }
    return fp;
}

template <typename R>
static cudaError_t run_fused(safr_plan_s *pl, const void *in, const float *in_scales, void *out,
                             float *out_scales, cudaStream_t st)
{
    FusedParams<R> fp = fused_params<R>(pl, in, in_scales, out, out_scales);
    void *args[] = {&fp};
    if (pl->trace) cudaEventRecord(pl->ev[0], st);
    cudaError_t e = cudaLaunchCooperativeKernel(frame_kernel_for(pl), dim3(pl->f_grid), dim3(512), args, pl->f_smem, st);
    if (pl->trace) {
        cudaEventRecord(pl->ev[1], st);
        pl->traced = 1;
    }
    return e;
}

cudaError_t launch_fused(safr_plan_s *pl, const void *in, const float *in_scales, void *out, float *out_scales,
                         cudaStream_t st)
{
    if (pl->precision == SAFR_FP64) return run_fused<double>(pl, in, in_scales, out, out_scales, st);
    return run_fused<float>(pl, in, in_scales, out, out_scales, st);
}

}  // namespace safr
