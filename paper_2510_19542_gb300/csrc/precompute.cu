// Algorithm 2 (soft real-time) on the GPU: B for every stored frequency.
//
// For frequency labels n = (n(j), n(k)) (Section 3.2) and one star group:
//   A_n[g][l] = s_l(n) exp(i pi n.(alpha_g h_l) / (c_l T))
//             = s_l(n) exp(2 pi i (n_x sx_gl + n_y sy_gl) / M),  s_gl = alpha_g h_l / (c_l delta)
//   s_l(n)    = gamma_l^{1/2} / c_l (1 + tau_l |n|^2)^{-beta/2},  tau_l = pi^2 / (c_l T)^2
// (the matrix A_jk = (2T) w^(beta)_{jk,l}(alpha_g h_l) of Section 3.1), and
//   B_n = diag(s(n)) R_alpha(A_n),  R_alpha(A) = V g_alpha(Sigma^T) U^H,  g_alpha(s) = s/(s^2+alpha).
// For the Tikhonov filter R_alpha(A) = A^H (A A^H + alpha I)^{-1}, so each
// thread forms the G x G Hermitian matrix K = A A^H + alpha I, factors it by
// Cholesky (K = C C^H) and solves K x_l = a_l for every column a_l of A:
// B_lg = s_l conj(x_l[g]).  Everything is FP64; B is stored in the frame
// kernels' precision.  Layout: B[k][b_row0 + l*G + g][pos(j)], k in [0, M/2), with
// j in the warp-FFT order of freqorder.h.
// The Nyquist row j = M/2 is zero (and the Nyquist column k = M/2 is not stored).
#include <cuda_runtime.h>

#include "common.cuh"
#include "freqorder.h"
#include "plan.h"

namespace safr {

template <typename C>
__device__ __forceinline__ void store_c(C *p, double re, double im);
template <>
__device__ __forceinline__ void store_c<float2>(float2 *p, double re, double im) { *p = make_float2((float)re, (float)im); }
template <>
__device__ __forceinline__ void store_c<double2>(double2 *p, double re, double im) { *p = make_double2(re, im); }

// CACHE: s_l(n) and the phase factors of A_n, computed once in the first pass, are kept in
// shared memory for the solves (element e of thread t at [e * blockDim + t]); otherwise the
// solves evaluate them again (large G * L).
template <typename C, bool CACHE>
__global__ void __launch_bounds__(128) precompute_kernel(int M, int Mh, int sumLG, double beta, PreGroupDev gr, C *B,
                                                         int *status)
{
    extern __shared__ double pc_cache[];
    const long idx = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (long)M * Mh) return;
    const int j = (int)(idx % M), k = (int)(idx / M);
    const int G = gr.G, L = gr.L;
    // stored with j in the frame kernels' warp-FFT order
    C *Bk = B + ((size_t)k * sumLG + gr.b_row0) * M + wfft_pos_of_j(j, M);
    if (j == M / 2) {
        for (int r = 0; r < L * G; ++r) store_c(Bk + (size_t)r * M, 0.0, 0.0);
        return;
    }
    const double nx = j < M / 2 ? j : j - M;
    const double ny = k;
    const double n2 = nx * nx + ny * ny;
    const double twoM = 2.0 / M;

    // K = A A^H + alpha I: K[g][h] = sum_l s_l^2 exp(i (theta_gl - theta_hl))
    double Kr[SAFR_MAX_GROUP_G][SAFR_MAX_GROUP_G], Ki[SAFR_MAX_GROUP_G][SAFR_MAX_GROUP_G];
    for (int g = 0; g < G; ++g)
        for (int h = 0; h < G; ++h) Kr[g][h] = Ki[g][h] = 0.0;
    const int nt = blockDim.x, tl = threadIdx.x;
    double *cs_ = pc_cache, *sn_ = pc_cache + (size_t)G * L * nt, *s_ = pc_cache + 2 * (size_t)G * L * nt;
    for (int l = 0; l < L; ++l) {
        const double s = gr.sw[l] * pow(1.0 + gr.tau[l] * n2, -0.5 * beta);
        const double s2 = s * s;
        double cr[SAFR_MAX_GROUP_G], ci[SAFR_MAX_GROUP_G];
        for (int g = 0; g < G; ++g) sincospi(twoM * (nx * gr.sx[g * L + l] + ny * gr.sy[g * L + l]), &ci[g], &cr[g]);
        if constexpr (CACHE) {
            s_[(size_t)l * nt + tl] = s;
            for (int g = 0; g < G; ++g) {
                cs_[((size_t)g * L + l) * nt + tl] = cr[g];
                sn_[((size_t)g * L + l) * nt + tl] = ci[g];
            }
        }
        for (int g = 0; g < G; ++g)
            for (int h = 0; h <= g; ++h) {
                // e^{i th_g} e^{-i th_h}
                Kr[g][h] += s2 * (cr[g] * cr[h] + ci[g] * ci[h]);
                Ki[g][h] += s2 * (ci[g] * cr[h] - cr[g] * ci[h]);
            }
    }
    for (int g = 0; g < G; ++g) Kr[g][g] += gr.alpha;

    // Cholesky K = C C^H, C lower triangular (stored over the lower half of K)
    for (int c = 0; c < G; ++c) {
        double d = Kr[c][c];
        for (int m = 0; m < c; ++m) d -= Kr[c][m] * Kr[c][m] + Ki[c][m] * Ki[c][m];
        if (!(d > 0.0)) {
            atomicExch(status, (int)SAFR_ERR_DEVICE);
            d = 1e-300;
        }
        const double dc = sqrt(d);
        Kr[c][c] = dc;
        Ki[c][c] = 0.0;
        for (int r = c + 1; r < G; ++r) {
            double xr = Kr[r][c], xi = Ki[r][c];
            for (int m = 0; m < c; ++m) {  // x -= C[r][m] conj(C[c][m])
                xr -= Kr[r][m] * Kr[c][m] + Ki[r][m] * Ki[c][m];
                xi -= Ki[r][m] * Kr[c][m] - Kr[r][m] * Ki[c][m];
            }
            Kr[r][c] = xr / dc;
            Ki[r][c] = xi / dc;
        }
    }

    // every layer: solve K x = a_l, B_lg = s_l conj(x_g)
    for (int l = 0; l < L; ++l) {
        double s;
        double yr[SAFR_MAX_GROUP_G], yi[SAFR_MAX_GROUP_G];
        if constexpr (CACHE) {
            s = s_[(size_t)l * nt + tl];
            for (int g = 0; g < G; ++g) {
                yr[g] = s * cs_[((size_t)g * L + l) * nt + tl];
                yi[g] = s * sn_[((size_t)g * L + l) * nt + tl];
            }
        } else {
            s = gr.sw[l] * pow(1.0 + gr.tau[l] * n2, -0.5 * beta);
            for (int g = 0; g < G; ++g) {
                double sn, cs;
                sincospi(twoM * (nx * gr.sx[g * L + l] + ny * gr.sy[g * L + l]), &sn, &cs);
                yr[g] = s * cs;
                yi[g] = s * sn;
            }
        }
        // forward: C y = a
        for (int r = 0; r < G; ++r) {
            double xr = yr[r], xi = yi[r];
            for (int m = 0; m < r; ++m) {
                xr -= Kr[r][m] * yr[m] - Ki[r][m] * yi[m];
                xi -= Kr[r][m] * yi[m] + Ki[r][m] * yr[m];
            }
            yr[r] = xr / Kr[r][r];
            yi[r] = xi / Kr[r][r];
        }
        // backward: C^H x = y
        for (int r = G - 1; r >= 0; --r) {
            double xr = yr[r], xi = yi[r];
            for (int m = r + 1; m < G; ++m) {  // (C^H)[r][m] = conj(C[m][r])
                xr -= Kr[m][r] * yr[m] + Ki[m][r] * yi[m];
                xi -= Kr[m][r] * yi[m] - Ki[m][r] * yr[m];
            }
            yr[r] = xr / Kr[r][r];
            yi[r] = xi / Kr[r][r];
        }
        for (int g = 0; g < G; ++g) store_c(Bk + (size_t)(l * G + g) * M, s * yr[g], -s * yi[g]);
    }
}

template <typename C>
cudaError_t launch_group(const safr_plan_s *plan, const PreGroupDev &d, long n, cudaStream_t stream)
{
    // threads per block so that the cache (2 G L + L doubles per thread) fits in 200 KB; below 32, no cache
    const size_t per = (2 * (size_t)d.G * d.L + d.L) * sizeof(double);
    int threads = 128;
    while (threads >= 32 && per * threads > 200 * 1024) threads /= 2;
    if (threads >= 32 && smem_limit_allows((const void *)precompute_kernel<C, true>, per * threads)) {
        const int blocks = (int)((n + threads - 1) / threads);
        precompute_kernel<C, true><<<blocks, threads, per * threads, stream>>>(plan->M, plan->Mh, plan->sumLG, plan->beta,
                                                                             d, (C *)plan->d_B, plan->d_status);
    } else {
        const int blocks = (int)((n + 127) / 128);
        precompute_kernel<C, false><<<blocks, 128, 0, stream>>>(plan->M, plan->Mh, plan->sumLG, plan->beta, d,
                                                                (C *)plan->d_B, plan->d_status);
    }
    return cudaGetLastError();
}

cudaError_t launch_precompute(safr_plan_s *plan, cudaStream_t stream)
{
    const int M = plan->M, Mh = plan->Mh, L = plan->L;
    const long n = (long)M * Mh;
    size_t off = 0;
    for (int gi = 0; gi < plan->ngroups; ++gi) {
        const Group &g = plan->grp[gi];
        PreGroupDev d;
        d.G = g.G;
        d.L = L;
        d.b_row0 = g.b_row0;
        d.alpha = g.alpha;
        d.sx = plan->d_pre + off;
        d.sy = d.sx + (size_t)g.G * L;
        d.sw = d.sy + (size_t)g.G * L;
        d.tau = d.sw + L;
        off += 2 * (size_t)g.G * L + 2 * L;
        cudaError_t e = plan->precision == SAFR_FP64 ? launch_group<double2>(plan, d, n, stream)
                                                       : launch_group<float2>(plan, d, n, stream);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

}  // namespace safr
