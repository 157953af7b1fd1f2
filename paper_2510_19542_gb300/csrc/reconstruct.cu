// Algorithm 1 (hard real-time) on the GPU, as three passes over the frame.
//
//   pass 1 (rows):    zero-pad each pupil wavefront into the M x M grid
//                     (Section 2), remove the LGS tip/tilt of a mixed plan
//                     (Algorithm 3, line 3), real-to-complex FFT of the P
//                     non-zero rows (two real rows per complex transform)
//                     -> w1[g][p][k], k < M/2.  Its CTAs also start streaming
//                     B from HBM into L2 for pass 2.
//   pass 2 (columns): per column k and star group: FFT of the G columns
//                     (P non-zero inputs each) -> d_g(j, k); per frequency
//                     b_l = sum_g B_lg d_g for every layer (Algorithm 1,
//                     line 5), from registers; inverse FFT over j
//                     -> w2[group][l][p][k].
//   pass 3 (rows):    complex-to-real inverse FFT of the rows (IDFT2 of
//                     Section 3.2, 1/M^2), bilinear resample of LGS-group
//                     layers from pitch c_l*delta to delta (metric output),
//                     sum of the two groups (Algorithm 3, line 4), store.
//
// The passes are chained with programmatic dependent launch: each kernel
// lets the next one launch at its start, and waits (griddepcontrol.wait, a
// hardware wait with no spinning) for its predecessor before it reads or
// writes any frame buffer.  Work before the wait touches only constant plan
// data, so the launch latency of passes 2 and 3 is hidden.
//
// The Nyquist row and column of the even grid carry no B (B = 0 there), so
// only k in [0, M/2) is kept between the passes.
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <type_traits>
#include <utility>

#include "common.cuh"
#include "fft.cuh"
#include "freqorder.h"
#include "plan.h"

namespace safr {

// ----------------------------------------------------------------------------
// pass 1: pad + removeTT + row FFT
// ----------------------------------------------------------------------------
template <typename R, typename TIN>
__global__ void __launch_bounds__(256) k_rows_forward(FrameParams<R> fp)
{
    using C = typename FrameParams<R>::C;
    extern __shared__ __align__(16) unsigned char smem[];
    pdl_trigger();
    const int M = fp.M, P = fp.P, Mh = fp.Mh, o = fp.o, logM = fp.logM;
    const int tid = threadIdx.x, nth = blockDim.x;

    // stream this CTA's share of B into L2 for pass 2 (constant plan data)
    if (fp.prefetch_bytes) {
        const int nb = gridDim.x * gridDim.y;
        const int b = blockIdx.y * gridDim.x + blockIdx.x;
        const size_t share = ((fp.prefetch_bytes + nb - 1) / nb + 4095) & ~(size_t)4095;
        const size_t lo = (size_t)b * share;
        const size_t hi = min(fp.prefetch_bytes, lo + share);
        for (size_t off = lo + (size_t)tid * 4096; off < hi; off += (size_t)nth * 4096)
            prefetch_l2(fp.prefetch + off, (unsigned)min((size_t)4096, hi - off));
    }

    const int g = blockIdx.y;
    const int rows = fp.rows_per_cta;  // even
    const int row0 = blockIdx.x * rows;
    if (row0 >= P) return;
    const int nrows = min(rows, P - row0);
    const int npairs = (nrows + 1) >> 1;
    C *bufA = (C *)smem;
    C *bufB = bufA + ((size_t)npairs << logM);
    R *red = (R *)(bufB + ((size_t)npairs << logM));
    C *tw = (C *)(red + 32);
    for (int i = tid; i < M; i += nth) tw[i] = fp.tw[i];

    pdl_wait();
    const TIN *psi = (const TIN *)fp.in + (size_t)g * P * P;
    const R scale = fp.in_scales ? (R)fp.in_scales[g] : R(1);
    const R half = R(0.5) * (R)(P - 1);
    const bool tt = fp.star_tt[g] != 0;

    // tip and tilt of the least-squares plane over the pupil mask: linear
    // functionals sum_i w_b[i] psi[i], sum_i w_c[i] psi[i] (weights from the
    // host FP64 inverse of the 3x3 normal matrix)
    R tb = 0, tc = 0;
    if (tt) {
        const R *wb = fp.tt_w, *wc = fp.tt_w + (size_t)P * P;
        R sb = 0, sc = 0;
        for (int i = tid; i < P * P; i += nth) {
            const R v = load_in<R>(psi + i);
            sb += wb[i] * v;
            sc += wc[i] * v;
        }
        tb = block_sum(sb, red) * scale;
        tc = block_sum(sc, red) * scale;
    }

    // z[q] = psi[row 2i][q - o] + i psi[row 2i+1][q - o], zero outside the pupil
    for (int idx = tid; idx < (npairs << logM); idx += nth) {
        const int i = idx >> logM, q = idx & (M - 1);
        const int qq = q - o;
        R re = 0, im = 0;
        if (qq >= 0 && qq < P) {
            const int a0 = row0 + 2 * i, a1 = a0 + 1;
            const R y = ((R)qq - half) * fp.delta;
            re = load_in<R>(psi + (size_t)a0 * P + qq) * scale;
            if (tt && fp.mask[a0 * P + qq]) re -= tb * (((R)a0 - half) * fp.delta) + tc * y;
            if (2 * i + 1 < nrows) {
                im = load_in<R>(psi + (size_t)a1 * P + qq) * scale;
                if (tt && fp.mask[a1 * P + qq]) im -= tb * (((R)a1 - half) * fp.delta) + tc * y;
            }
        }
        bufA[idx] = C{re, im};
    }
    __syncthreads();
    C *res = block_fft<false>(bufA, bufB, logM, npairs, M, tw, tid, nth);

    // split the two real transforms: X1 = (Z[k] + conj Z[M-k]) / 2, X2 = (Z[k] - conj Z[M-k]) / 2i
    const int logMh = logM - 1;
    for (int idx = tid; idx < (npairs << logMh); idx += nth) {
        const int i = idx >> logMh, k = idx & (Mh - 1);
        const C z = res[(i << logM) + k];
        const C zc = res[(i << logM) + ((M - k) & (M - 1))];
        const C x1 = C{R(0.5) * (z.x + zc.x), R(0.5) * (z.y - zc.y)};
        const C x2 = C{R(0.5) * (z.y + zc.y), R(0.5) * (zc.x - z.x)};
        const int a0 = row0 + 2 * i;
        fp.w1[((size_t)g * P + a0) * Mh + k] = x1;
        if (2 * i + 1 < nrows) fp.w1[((size_t)g * P + a0 + 1) * Mh + k] = x2;
    }
}

// ----------------------------------------------------------------------------
// pass 2: column FFT + per-frequency apply + inverse column FFT
// ----------------------------------------------------------------------------
template <typename R, int GMAX>
__global__ void __launch_bounds__(256) k_cols_apply(FrameParams<R> fp)
{
    using C = typename FrameParams<R>::C;
    extern __shared__ __align__(16) unsigned char smem[];
    pdl_trigger();
    const int M = fp.M, P = fp.P, Mh = fp.Mh, o = fp.o, L = fp.L, logM = fp.logM;
    const int k = blockIdx.x;
    const int gi = blockIdx.y;
    const GroupDev &gr = fp.grp[gi];
    const int Gg = gr.G;
    const int W = max(Gg, fp.lchunk);
    C *dcol = (C *)smem;                    // [Gg][M]
    C *bufA = dcol + ((size_t)Gg << logM);  // [W][M]
    C *bufB = bufA + ((size_t)W << logM);   // [W][M]
    C *tw = bufB + ((size_t)W << logM);     // [M]
    R *red = (R *)(tw + M);
    const int tid = threadIdx.x, nth = blockDim.x;
    for (int i = tid; i < M; i += nth) tw[i] = fp.tw[i];

    pdl_wait();
    for (int idx = tid; idx < (Gg << logM); idx += nth) {
        const int t = idx >> logM, p = idx & (M - 1);
        const int pp = p - o;
        C v = C{0, 0};
        if (pp >= 0 && pp < P) v = fp.w1[((size_t)gr.star[t] * P + pp) * Mh + k];
        dcol[idx] = v;
    }
    __syncthreads();
    // forward column transforms, result copied back into dcol if it landed in bufA
    C *res = block_fft<false>(dcol, bufA, logM, Gg, M, tw, tid, nth);
    if (res != dcol) {
        for (int idx = tid; idx < (Gg << logM); idx += nth) dcol[idx] = res[idx];
        __syncthreads();
    }

    const C *Bk = fp.B + ((size_t)k * fp.sumLG + gr.b_row0) * M;
    for (int l0 = 0; l0 < L; l0 += fp.lchunk) {
        const int lc = min(fp.lchunk, L - l0);
        for (int j = tid; j < M; j += nth) {
            C d[GMAX];
#pragma unroll
            for (int t = 0; t < GMAX; ++t)
                if (t < Gg) d[t] = dcol[(t << logM) + j];
            // B is stored with j in the persistent kernel's warp-FFT order
            const C *Bj = Bk + (size_t)l0 * Gg * M + wfft_pos_of_j(j, M);
#pragma unroll 2
            for (int l = 0; l < lc; ++l) {
                C bv[GMAX];
#pragma unroll
                for (int t = 0; t < GMAX; ++t)
                    if (t < Gg) bv[t] = __ldg(Bj + ((size_t)(l * Gg + t) << logM));
                R ar = 0, ai = 0;
#pragma unroll
                for (int t = 0; t < GMAX; ++t)
                    if (t < Gg) {
                        ar += bv[t].x * d[t].x - bv[t].y * d[t].y;
                        ai += bv[t].x * d[t].y + bv[t].y * d[t].x;
                    }
                bufA[(l << logM) + j] = C{ar, ai};
            }
        }
        __syncthreads();
        if (fp.energy) {
            // Parseval partial sum of |b_l(j, k)|^2 over j (column k counts twice
            // in the full spectrum unless k = 0)
            for (int l = 0; l < lc; ++l) {
                R e = 0;
                for (int j = tid; j < M; j += nth) {
                    const C v = bufA[(l << logM) + j];
                    e += v.x * v.x + v.y * v.y;
                }
                e = block_sum(e, red);
                if (tid == 0) fp.energy[((size_t)gi * L + l0 + l) * Mh + k] = (float)(k == 0 ? e : R(2) * e);
            }
        }
        res = block_fft<true>(bufA, bufB, logM, lc, M, tw, tid, nth);
        for (int idx = tid; idx < (lc << logM); idx += nth) {
            const int l = idx >> logM, p = idx & (M - 1);
            fp.w2[(((size_t)gi * L + l0 + l) * M + p) * Mh + k] = res[idx];
        }
        __syncthreads();
    }
}

// ----------------------------------------------------------------------------
// pass 3: inverse row FFT (complex to real) + resample + group sum + store
// ----------------------------------------------------------------------------
template <typename R, typename TOUT>
__global__ void __launch_bounds__(256) k_rows_inverse(FrameParams<R> fp)
{
    using C = typename FrameParams<R>::C;
    extern __shared__ __align__(16) unsigned char smem[];
    pdl_trigger();
    const int M = fp.M, Mh = fp.Mh, L = fp.L, logM = fp.logM;
    const int l = blockIdx.y;
    const int p0 = blockIdx.x * fp.rows_per_cta;
    const int nr = min(fp.rows_per_cta, M - p0);
    const int SP = fp.src_pairs;
    C *bufA = (C *)smem;                    // [SP][M]
    C *bufB = bufA + ((size_t)SP << logM);  // [SP][M]
    C *tw = bufB + ((size_t)SP << logM);    // [M]
    R *acc = (R *)(tw + M);                 // [rows][M]
    const int tid = threadIdx.x, nth = blockDim.x;
    for (int i = tid; i < M; i += nth) tw[i] = fp.tw[i];
    for (int i = tid; i < (nr << logM); i += nth) acc[i] = 0;

    pdl_wait();
    for (int gi = 0; gi < fp.ngroups; ++gi) {
        const bool rs = fp.grp[gi].resample;
        int first, nsrc;
        if (rs) {
            first = fp.rs_i0[l * M + p0];
            nsrc = fp.rs_i0[l * M + p0 + nr - 1] + 2 - first;
        } else {
            first = p0;
            nsrc = nr;
        }
        const int npairs = (nsrc + 1) >> 1;
        if (npairs > SP) {  // the host sizes SP for every tile; never expected
            if (tid == 0) atomicExch(fp.status, (int)SAFR_ERR_DEVICE);
            return;
        }
        const C *src = fp.w2 + ((size_t)gi * L + l) * M * Mh;
        // Z[k] = X1[k] + i X2[k] over the full length M from the stored half (Hermitian rows)
        for (int idx = tid; idx < (npairs << logM); idx += nth) {
            const int i = idx >> logM, k = idx & (M - 1);
            const int ra = (first + 2 * i) & (M - 1);
            const bool hasb = 2 * i + 1 < nsrc;
            const int rb = (first + 2 * i + 1) & (M - 1);
            C z = C{0, 0};
            if (k < Mh) {
                C x1 = src[(size_t)ra * Mh + k];
                C x2 = hasb ? src[(size_t)rb * Mh + k] : C{0, 0};
                if (k == 0) {
                    x1.y = 0;
                    x2.y = 0;
                }
                z = C{x1.x - x2.y, x1.y + x2.x};
            } else if (k > Mh) {
                const int kk = M - k;
                const C x1 = src[(size_t)ra * Mh + kk];
                const C x2 = hasb ? src[(size_t)rb * Mh + kk] : C{0, 0};
                // conj(x1) + i conj(x2)
                z = C{x1.x + x2.y, x2.x - x1.y};
            }
            bufA[idx] = z;
        }
        __syncthreads();
        const C *res = block_fft<true>(bufA, bufB, logM, npairs, M, tw, tid, nth);
        // source row s (local) = res[s/2].x or .y
        for (int idx = tid; idx < (nr << logM); idx += nth) {
            const int r = idx >> logM, q = idx & (M - 1);
            R v;
            if (rs) {
                const int pr = p0 + r;
                const int i0 = fp.rs_i0[l * M + pr] - first;
                const R fu = fp.rs_w[l * M + pr];
                const int j0u = fp.rs_i0[l * M + q];
                const R fv = fp.rs_w[l * M + q];
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

    // per-layer power-of-two scale from the Parseval energy (FP16 storage)
    R inv_scale = R(1);
    if (fp.out_scales) {
        double e = 0;
        for (int gi = 0; gi < fp.ngroups; ++gi)
            for (int k = 0; k < Mh; ++k) e += (double)fp.energy[((size_t)gi * L + l) * Mh + k];
        // mean square of the layer: sum_n |b(n)|^2 / M^4
        const double ms = e / ((double)M * M * (double)M * M);
        double sc = 1.0;
        if (ms > 0) sc = exp2(rint(0.5 * log2(ms)));
        inv_scale = (R)(1.0 / sc);
        if (blockIdx.x == 0 && tid == 0) fp.out_scales[l] = (float)sc;
    }
    TOUT *out = (TOUT *)fp.out + ((size_t)l * M + p0) * M;
    const R f = fp.inv_M2 * inv_scale;
    for (int idx = tid; idx < (nr << logM); idx += nth) {
        if constexpr (std::is_same<TOUT, double>::value)
            store_out_d(out + idx, (double)(acc[idx] * f));
        else
            store_out<TOUT>(out + idx, (float)(acc[idx] * f));
    }
}

// ----------------------------------------------------------------------------
// host side
// ----------------------------------------------------------------------------
static size_t csize(const safr_plan_s *pl) { return pl->precision == SAFR_FP64 ? 16 : 8; }
static size_t rsize(const safr_plan_s *pl) { return pl->precision == SAFR_FP64 ? 8 : 4; }

template <typename R>
static FrameParams<R> make_params(safr_plan_s *pl, const void *in, const float *in_scales, void *out,
                                  float *out_scales)
{
    using C = typename FrameParams<R>::C;
    FrameParams<R> fp;
    memset(&fp, 0, sizeof(fp));
    fp.M = pl->M;
    fp.P = pl->P;
    fp.L = pl->L;
    fp.G = pl->G;
    fp.Mh = pl->Mh;
    fp.o = pl->o;
    fp.ngroups = pl->ngroups;
    fp.sumLG = pl->sumLG;
    int lm = 0;
    while ((1 << lm) < pl->M) ++lm;
    fp.logM = lm;
    fp.lchunk = pl->lchunk;
    fp.rows_per_cta = pl->rows_per_cta;
    fp.src_pairs = pl->src_pairs;
    fp.delta = (R)pl->delta;
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
    fp.mask = pl->d_mask;
    fp.tt_w = (const R *)pl->d_tt_w;
    fp.prefetch = (const char *)pl->d_B;
    fp.prefetch_bytes = pl->b_bytes;
    for (int g = 0; g < pl->G; ++g) fp.star_tt[g] = pl->star_tt[g];
    for (int gi = 0; gi < pl->ngroups; ++gi) {
        fp.grp[gi].G = pl->grp[gi].G;
        fp.grp[gi].b_row0 = pl->grp[gi].b_row0;
        fp.grp[gi].resample = pl->grp[gi].resample ? 1 : 0;
        for (int t = 0; t < pl->grp[gi].G; ++t) fp.grp[gi].star[t] = pl->grp[gi].stars[t];
    }
    fp.status = pl->d_status;
    return fp;
}

int launches_per_frame(const safr_plan_s *pl) { return use_fused(pl) || use_cluster(pl) ? 1 : 3; }

// column-pass instance for the largest star group of the plan
template <typename R>
static void (*cols_kernel(int gmax))(FrameParams<R>)
{
    return gmax == 4 ? k_cols_apply<R, 4> : (gmax == 8 ? k_cols_apply<R, 8> : k_cols_apply<R, 16>);
}

template <typename K1, typename K2, typename K3>
static safr_status set_smem(K1 k1, K2 k2, K3 k3, const safr_plan_s *pl)
{
    const int f[3] = {smem_fit((const void *)k1, pl->smem_k1), smem_fit((const void *)k2, pl->smem_k2),
                      smem_fit((const void *)k3, pl->smem_k3)};
    for (int i = 0; i < 3; ++i)
        if (f[i] < 0) return SAFR_ERR_CUDA;
    for (int i = 0; i < 3; ++i)
        if (f[i] == 0) return SAFR_ERR_UNSUPPORTED_SIZE;
    return SAFR_OK;
}

// Shared-memory sizes and launch shapes; called once at plan creation.  SAFR_ERR_UNSUPPORTED_SIZE
// when a pass needs more shared memory than one CTA may have, SAFR_ERR_CUDA when a query failed.
safr_status configure_frame_kernels(safr_plan_s *pl)
{
    const int M = pl->M;
    const size_t cs = csize(pl), rs = rsize(pl);
    int maxGg = 1;
    for (int gi = 0; gi < pl->ngroups; ++gi) maxGg = std::max(maxGg, pl->grp[gi].G);
    const size_t budget = 200 * 1024;

    // pass 1: rows per CTA (even), two buffers of rows/2 transforms
    pl->k1_rows = 8;
    pl->smem_k1 = 2 * (size_t)(pl->k1_rows / 2) * M * cs + 32 * rs + (size_t)M * cs;

    // pass 2: layers per inverse chunk so that dcol + 2 * max(Gg, chunk) rows fit
    int lc = pl->L;
    auto k2_bytes = [&](int c) {
        const int W = std::max(maxGg, c);
        return ((size_t)maxGg * M + 2 * (size_t)W * M + M) * cs + 32 * rs;
    };
    while (lc > 1 && k2_bytes(lc) > budget) --lc;
    pl->lchunk = lc;
    pl->smem_k2 = k2_bytes(lc);

    // pass 3: output rows per CTA and the source row pairs they need
    pl->rows_per_cta = 8;
    int sp = (pl->rows_per_cta + 1) / 2;
    for (int gi = 0; gi < pl->ngroups; ++gi) {
        if (!pl->grp[gi].resample) continue;
        for (int l = 0; l < pl->L; ++l) {
            const double c = pl->grp[gi].c[l];
            for (int p0 = 0; p0 < M; p0 += pl->rows_per_cta) {
                const int p1 = std::min(M, p0 + pl->rows_per_cta) - 1;
                const int a = (int)std::floor(M / 2.0 + (p0 - M / 2.0) / c);
                const int b = (int)std::floor(M / 2.0 + (p1 - M / 2.0) / c);
                sp = std::max(sp, (b + 2 - a + 1) / 2);
            }
        }
    }
    pl->src_pairs = sp;
    pl->smem_k3 = (2 * (size_t)sp * M + M) * cs + (size_t)pl->rows_per_cta * M * rs;

    pl->gmax = maxGg <= 4 ? 4 : (maxGg <= 8 ? 8 : 16);
    if (pl->precision == SAFR_FP64)
        return set_smem(k_rows_forward<double, double>, cols_kernel<double>(pl->gmax), k_rows_inverse<double, double>, pl);
    if (pl->precision == SAFR_FP16_STORAGE)
        return set_smem(k_rows_forward<float, __half>, cols_kernel<float>(pl->gmax), k_rows_inverse<float, __half>, pl);
    return set_smem(k_rows_forward<float, float>, cols_kernel<float>(pl->gmax), k_rows_inverse<float, float>, pl);
}

template <typename... KArgs, typename... Args>
static cudaError_t launch(void (*kernel)(KArgs...), dim3 grid, size_t smem, cudaStream_t st, bool pdl,
                          Args &&...args)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = dim3(256);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = pdl ? 1 : 0;
    return cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...);
}

template <typename R, typename TIN, typename TOUT>
static cudaError_t run_frame(safr_plan_s *pl, const void *in, const float *in_scales, void *out,
                             float *out_scales, cudaStream_t st)
{
    FrameParams<R> fp = make_params<R>(pl, in, in_scales, out, out_scales);
    const dim3 g1((pl->P + pl->k1_rows - 1) / pl->k1_rows, pl->G);
    const dim3 g2(pl->Mh, pl->ngroups);
    const dim3 g3((pl->M + pl->rows_per_cta - 1) / pl->rows_per_cta, pl->L);
    // events between the passes would break the programmatic overlap, so a
    // traced call runs the passes plainly serialised
    const bool pdl = pl->pdl && !pl->trace;
    cudaError_t e;
    if (pl->trace) cudaEventRecord(pl->ev[0], st);
    fp.rows_per_cta = pl->k1_rows;
    e = launch(k_rows_forward<R, TIN>, g1, pl->smem_k1, st, pdl, fp);
    if (e != cudaSuccess) return e;
    if (pl->trace) cudaEventRecord(pl->ev[1], st);
    fp.rows_per_cta = pl->rows_per_cta;
    e = launch(cols_kernel<R>(pl->gmax), g2, pl->smem_k2, st, pdl, fp);
    if (e != cudaSuccess) return e;
    if (pl->trace) cudaEventRecord(pl->ev[2], st);
    e = launch(k_rows_inverse<R, TOUT>, g3, pl->smem_k3, st, pdl, fp);
    if (e != cudaSuccess) return e;
    if (pl->trace) {
        cudaEventRecord(pl->ev[3], st);
        pl->traced = 1;
    }
    return cudaGetLastError();
}

cudaError_t launch_frame(safr_plan_s *pl, const void *in, const float *in_scales, void *out,
                         float *out_scales, cudaStream_t st)
{
    if (pl->precision == SAFR_FP64) return run_frame<double, double, double>(pl, in, in_scales, out, out_scales, st);
    if (pl->precision == SAFR_FP16_STORAGE)
        return run_frame<float, __half, __half>(pl, in, in_scales, out, out_scales, st);
    return run_frame<float, float, float>(pl, in, in_scales, out, out_scales, st);
}

}  // namespace safr
