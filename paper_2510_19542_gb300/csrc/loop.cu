// The steps of the three-step AO loop (Algorithm 3) around SAFR: pseudo open
// loop control (POLC, Algorithm 3 line 2) and the integrator (line 5).
//
// POLC adds the tomography operator of Section 2 applied to the current
// mirror/layer state a to the closed-loop wavefronts:
//
//     psi~_g(r) = psi_g(r) + (A_g a)(r),   (A_g a)(r) = sum_l a_l(c_l r + alpha_g h_l),
//
// evaluated at the pupil samples r and zero off the pupil (the zero extension
// of Section 2).  The layers a_l are samples on the plan's output grid, and
// the operator interpolates them bilinearly, matrix-free, in O(N) (Section 3.4
// computational cost).  The sample point of star g, layer l, pupil pixel
// (p, q) in output-grid pixels is
//     native grid (pitch c_l delta):  u = o + p + s_gl
//     metric grid (pitch delta):      u = M/2 + c_l (o + p - M/2 + s_gl)
// with s_gl = alpha_g h_l / (c_l delta) and o = (M - P)/2 (likewise for q),
// wrapped periodically onto [0, M).
//
// The integrator: a <- (1 - gain) a + gain Phi, Phi the new reconstruction.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <vector>

#include "plan.h"
#include "safr.h"

namespace safr {

// Sample points of the POLC operator, in one byte array (built in FP64 on the host):
//   fx [G][L][P], fy [G][L][P]  fractional parts (plan precision R)
//   ix [G][L][P], iy [G][L][P]  whole parts wrapped onto [0, M) (int)
//   mask [P][P]                 pupil (1 inside)
// for star g (geometry order), layer l and pupil row p (x) or column q (y).
void polc_table(const safr_plan_s *pl, std::vector<unsigned char> &bytes)
{
    const int L = pl->L, M = pl->M, o = pl->o, P = pl->P, G = pl->G;
    const size_t n = (size_t)G * L * P, rs = pl->precision == SAFR_FP64 ? 8 : 4;
    bytes.assign(2 * n * rs + 2 * n * 4 + (size_t)P * P, 0);
    unsigned char *fx = bytes.data(), *fy = fx + n * rs;
    int *ix = (int *)(fy + n * rs), *iy = ix + n;
    unsigned char *mask = (unsigned char *)(iy + n);
    auto put = [&](unsigned char *f, int *i, size_t k, double u) {
        const double fl = std::floor(u);
        long w = (long)fl % M;
        if (w < 0) w += M;
        i[k] = (int)w;
        if (rs == 8) ((double *)f)[k] = u - fl;
        else ((float *)f)[k] = (float)(u - fl);
    };
    for (int gi = 0; gi < pl->ngroups; ++gi) {
        const Group &grp = pl->grp[gi];
        for (int gg = 0; gg < grp.G; ++gg) {
            const int g = grp.stars[gg];
            for (int l = 0; l < L; ++l) {
                const double c = grp.c[l], sx = grp.sx[(size_t)gg * L + l], sy = grp.sy[(size_t)gg * L + l];
                for (int p = 0; p < P; ++p) {
                    const size_t k = ((size_t)g * L + l) * P + p;
                    if (pl->output_metric) {
                        put(fx, ix, k, M / 2.0 + c * (o + p - M / 2.0 + sx));
                        put(fy, iy, k, M / 2.0 + c * (o + p - M / 2.0 + sy));
                    } else {
                        put(fx, ix, k, o + p + sx);
                        put(fy, iy, k, o + p + sy);
                    }
                }
            }
        }
    }
    const double ro = pl->diameter / 2.0, ri = pl->obstruction * pl->diameter / 2.0;
    for (int a = 0; a < P; ++a)
        for (int b = 0; b < P; ++b) {
            const double x = (a - (P - 1) / 2.0) * pl->delta, y = (b - (P - 1) / 2.0) * pl->delta;
            const double r2 = x * x + y * y;
            mask[(size_t)a * P + b] = pl->diameter <= 0 ? 1 : (r2 <= ro * ro && r2 >= ri * ri);
        }
}

// One thread per (star, pupil pixel); q fastest, so neighbouring threads read neighbouring layer samples.
template <typename R>
__global__ void __launch_bounds__(256) k_polc(int M, int P, int L, int G, const unsigned char *tab, const R *psi,
                                              const R *a, R *out)
{
    const long idx = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (long)G * P * P) return;
    const size_t n = (size_t)G * L * P;
    const R *fx = (const R *)tab, *fy = fx + n;
    const int *ix = (const int *)(fy + n), *iy = ix + n;
    const unsigned char *mask = (const unsigned char *)(iy + n);
    const int g = (int)(idx / ((long)P * P)), pq = (int)(idx % ((long)P * P)), p = pq / P, q = pq % P;
    R acc = 0;
    if (mask[pq]) {
        acc = psi[idx];
#pragma unroll 4
        for (int l = 0; l < L; ++l) {
            const size_t k = ((size_t)g * L + l) * P;
            const R fu = fx[k + p], fv = fy[k + q];
            const int i0 = ix[k + p], j0 = iy[k + q];
            const int i1 = i0 + 1 == M ? 0 : i0 + 1, j1 = j0 + 1 == M ? 0 : j0 + 1;
            const R *al = a + (size_t)l * M * M;
            const R v00 = al[(size_t)i0 * M + j0], v01 = al[(size_t)i0 * M + j1];
            const R v10 = al[(size_t)i1 * M + j0], v11 = al[(size_t)i1 * M + j1];
            acc += ((R)1 - fu) * (((R)1 - fv) * v00 + fv * v01) + fu * (((R)1 - fv) * v10 + fv * v11);
        }
    }
    out[idx] = acc;
}

// a <- (1 - gain) a + gain phi, n elements, vectors of 16 bytes (n a multiple of the vector width)
__global__ void __launch_bounds__(256) k_integrate_f32(long n4, const float4 *phi, float4 *a, float gain)
{
    const float keep = 1.0f - gain;
    for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < n4; i += (long)gridDim.x * blockDim.x) {
        const float4 f = phi[i];
        float4 x = a[i];
        x.x = keep * x.x + gain * f.x;
        x.y = keep * x.y + gain * f.y;
        x.z = keep * x.z + gain * f.z;
        x.w = keep * x.w + gain * f.w;
        a[i] = x;
    }
}

__global__ void __launch_bounds__(256) k_integrate_f64(long n2, const double2 *phi, double2 *a, double gain)
{
    const double keep = 1.0 - gain;
    for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < n2; i += (long)gridDim.x * blockDim.x) {
        const double2 f = phi[i];
        double2 x = a[i];
        x.x = keep * x.x + gain * f.x;
        x.y = keep * x.y + gain * f.y;
        a[i] = x;
    }
}

}  // namespace safr

namespace {

bool aligned16(const void *p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

struct LoopDeviceGuard {
    int prev = -1;
    bool ok = false;
    explicit LoopDeviceGuard(int dev)
    {
        if (cudaGetDevice(&prev) != cudaSuccess) return;
        if (prev != dev && cudaSetDevice(dev) != cudaSuccess) return;
        ok = true;
    }
    ~LoopDeviceGuard()
    {
        if (ok && prev >= 0) cudaSetDevice(prev);
    }
};

safr_status polc_launch(safr_plan_t pl, const void *psi, const void *a, void *out, cudaStream_t st)
{
    const long n = (long)pl->G * pl->P * pl->P;
    const int th = 256;
    const int nb = (int)((n + th - 1) / th);
    if (pl->precision == SAFR_FP64)
        safr::k_polc<double><<<nb, th, 0, st>>>(pl->M, pl->P, pl->L, pl->G, pl->d_polc, (const double *)psi,
                                                (const double *)a, (double *)out);
    else
        safr::k_polc<float><<<nb, th, 0, st>>>(pl->M, pl->P, pl->L, pl->G, pl->d_polc, (const float *)psi,
                                               (const float *)a, (float *)out);
    return cudaGetLastError() == cudaSuccess ? SAFR_OK : SAFR_ERR_CUDA;
}

safr_status integrate_launch(safr_plan_t pl, const void *phi, void *a, double gain, cudaStream_t st)
{
    const long n = (long)pl->L * pl->M * pl->M;  // M >= 8: a multiple of 4
    const int th = 256;
    int nsm = 152;
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, pl->device);
    if (pl->precision == SAFR_FP64) {
        const long n2 = n / 2;
        const int nb = (int)std::min<long>((n2 + th - 1) / th, (long)nsm * 8);
        safr::k_integrate_f64<<<nb, th, 0, st>>>(n2, (const double2 *)phi, (double2 *)a, gain);
    } else {
        const long n4 = n / 4;
        const int nb = (int)std::min<long>((n4 + th - 1) / th, (long)nsm * 8);
        safr::k_integrate_f32<<<nb, th, 0, st>>>(n4, (const float4 *)phi, (float4 *)a, (float)gain);
    }
    return cudaGetLastError() == cudaSuccess ? SAFR_OK : SAFR_ERR_CUDA;
}

safr_status check_plan(safr_plan_t pl)
{
    if (!pl) return SAFR_ERR_INVALID_ARG;
    if (pl->precision == SAFR_FP16_STORAGE) return SAFR_ERR_UNSUPPORTED_SIZE;
    if (!pl->d_polc) return SAFR_ERR_CUDA;
    return SAFR_OK;
}

bool gain_ok(double gain) { return std::isfinite(gain) && gain >= 0.0 && gain <= 1.0; }

}  // namespace

extern "C" {

safr_status safr_polc(safr_plan_t plan, const void *d_wavefronts, const void *d_a, void *d_out, cudaStream_t stream)
{
    safr_status s = check_plan(plan);
    if (s != SAFR_OK) return s;
    if (!d_wavefronts || !d_a || !d_out) return SAFR_ERR_INVALID_ARG;
    if (!aligned16(d_wavefronts) || !aligned16(d_a) || !aligned16(d_out)) return SAFR_ERR_MISALIGNED;
    LoopDeviceGuard guard(plan->device);
    if (!guard.ok) return SAFR_ERR_CUDA;
    return polc_launch(plan, d_wavefronts, d_a, d_out, stream);
}

safr_status safr_integrate(safr_plan_t plan, const void *d_layers, void *d_a, double gain, cudaStream_t stream)
{
    safr_status s = check_plan(plan);
    if (s != SAFR_OK) return s;
    if (!d_layers || !d_a || !gain_ok(gain)) return SAFR_ERR_INVALID_ARG;
    if (!aligned16(d_layers) || !aligned16(d_a)) return SAFR_ERR_MISALIGNED;
    LoopDeviceGuard guard(plan->device);
    if (!guard.ok) return SAFR_ERR_CUDA;
    return integrate_launch(plan, d_layers, d_a, gain, stream);
}

safr_status safr_loop_step(safr_plan_t plan, const void *d_wavefronts, void *d_a, double gain, cudaStream_t stream)
{
    safr_status s = check_plan(plan);
    if (s != SAFR_OK) return s;
    if (!d_wavefronts || !d_a || !gain_ok(gain)) return SAFR_ERR_INVALID_ARG;
    if (!plan->precomputed) return SAFR_ERR_NOT_PRECOMPUTED;
    if (!aligned16(d_wavefronts) || !aligned16(d_a)) return SAFR_ERR_MISALIGNED;
    LoopDeviceGuard guard(plan->device);
    if (!guard.ok) return SAFR_ERR_CUDA;
    if (safr::use_fused(plan)) {
        // one launch: the persistent kernel computes the POLC data into the staging buffer (phase 0:
        // each CTA the rows of its own phase 1), reconstructs, and blends its layers into the state
        // as it stores them
        plan->loop_blend = 1;
        plan->loop_gain = gain;
        plan->loop_polc_psi = d_wavefronts;
        const cudaError_t e = safr::launch_fused(plan, plan->d_in_stage, nullptr, d_a, nullptr, stream);
        plan->loop_blend = 0;
        plan->loop_polc_psi = nullptr;
        return e == cudaSuccess ? SAFR_OK : SAFR_ERR_CUDA;
    }
    s = polc_launch(plan, d_wavefronts, d_a, plan->d_in_stage, stream);
    if (s != SAFR_OK) return s;
    s = safr_reconstruct(plan, plan->d_in_stage, nullptr, plan->d_out_stage, nullptr, stream);
    if (s != SAFR_OK) return s;
    return integrate_launch(plan, plan->d_out_stage, d_a, gain, stream);
}

}  // extern "C"
