// Learned spectral filter.  Section 3.1 builds the regularised inverse from
// any regularising filter g_alpha acting on the singular values (the paper's
// experiments use Tikhonov); here the filter is learned.
//
// SAFR's B(n) = diag(s) V g(Sigma) U^H applies one filter g(sigma_r) to every
// singular direction r of A(n) = U Sigma V^H.  Here the filter factor is
// phi_theta(x) in (0, 1), an MLP of the point x = (|n|, h_l, sigma_r, noise
// level), and the weight of direction r in layer l is w_lr = phi_theta / sigma_r
// (phi = 1 is the pseudo-inverse, phi = sigma^2 / (sigma^2 + alpha) is
// Tikhonov):
//
//     B_lg(n) = s_l(n) sum_r V_lr(n) w_lr(n) conj(U_gr(n)).
//
// The MLP is 4 -> 64 -> 64 -> 64 -> 1 with GELU (exact erf form) after the
// hidden layers and a logistic output; its parameters are BF16, its
// arithmetic FP32.  Its inputs are fixed per plan, so inference runs once,
// when B is built, and the per-frame kernels are unchanged.
//
// Training (hand-written kernels, all on the GPU): frames of the layered model
// of Section 2 through the aperture.  Layer spectra phi_l(n) are drawn with the
// von Karman variance of a layer's DFT and made Hermitian (real screens); star
// g's spectrum c_g(n) = sum_l e^{i theta_gl(n)} phi_l(n) is taken back to real
// space, restricted to the plan's pupil (the operator A_g acts on the aperture
// Omega_A), given white pixel noise with standard deviation noise level x the
// RMS of the masked noise-free wavefront, and transformed again: d_g =
// DFT2(psi_g).  All random numbers come from a counter-based generator
// (Philox4x32-10, Salmon et al., SC 2011).  The loss is the relative squared
// error of the reconstructed layer spectra (Parseval: the squared error of the
// layers); its gradient flows through the MLP; Adam updates FP32 master
// weights.  Held-out frames compare the learned filter against plain SAFR,
// which stays in the plan if it is not beaten.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <vector>

#include "common.cuh"
#include "freqorder.h"
#include "plan.h"
#include "safr.h"

namespace safr {

constexpr int kH = 64;  // hidden width
// parameter layout: W0[64][4], b0[64], W1[64][64], b1[64], W2[64][64], b2[64], W3[64], b3
constexpr int kOffW0 = 0, kOffB0 = kOffW0 + kH * 4, kOffW1 = kOffB0 + kH, kOffB1 = kOffW1 + kH * kH,
              kOffW2 = kOffB1 + kH, kOffB2 = kOffW2 + kH * kH, kOffW3 = kOffB2 + kH, kOffB3 = kOffW3 + kH,
              kParams = kOffB3 + 1;
static_assert(kParams == SAFR_FILTER_PARAMS, "parameter count");

// ---------------------------------------------------------------------------
// Philox4x32-10 (counter-based generator) and normal variates
// ---------------------------------------------------------------------------
struct U4 {
    uint32_t x, y, z, w;
};

__device__ __forceinline__ U4 philox4x32_10(U4 c, uint32_t k0, uint32_t k1)
{
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint64_t p0 = (uint64_t)0xD2511F53u * c.x, p1 = (uint64_t)0xCD9E8D57u * c.z;
        c = U4{(uint32_t)(p1 >> 32) ^ c.y ^ k0, (uint32_t)p1, (uint32_t)(p0 >> 32) ^ c.w ^ k1, (uint32_t)p0};
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    return c;
}

// two independent standard normals (Box-Muller) from the counter (a, b, c, d)
__device__ __forceinline__ float2 normal2(uint32_t a, uint32_t b, uint32_t c, uint32_t d, uint32_t k0, uint32_t k1)
{
    const U4 u = philox4x32_10(U4{a, b, c, d}, k0, k1);
    const float u1 = ((float)u.x + 0.5f) * 2.3283064365386963e-10f;  // (0, 1)
    const float u2 = ((float)u.y + 0.5f) * 2.3283064365386963e-10f;
    const float rad = sqrtf(-2.0f * logf(u1));
    float sn, cs;
    sincospif(2.0f * u2, &sn, &cs);
    return make_float2(rad * cs, rad * sn);
}

// ---------------------------------------------------------------------------
// per-frequency basis: A(n) = U Sigma V^H of one star group
// ---------------------------------------------------------------------------
struct Basis {
    int NF;           // frequencies: f = k * M + j, k < M/2, j < M
    double2 *U;       // [NF][G][G]      left singular vectors (columns r)
    double *sig;      // [NF][G]         singular values (descending not required)
    double2 *Q;       // [NF][L][G]      s_l V_lr = s_l (A^H U)_lr / sigma_r
    float2 *E;        // [NF][G][L]      e^{i theta_gl} (forward model of the training frames)
    double *s;        // [NF][L]         s_l(n)
    float *var;       // [NF][L]         variance of a layer's spectrum in the training frames
};

// One thread per frequency: build A (G x L), one-sided Jacobi on the columns of
// A^H (L x G, held in Q), accumulate the rotations in U.  After convergence the
// columns of A^H U are orthogonal: A^H U = V Sigma, so A = U Sigma V^H.
__global__ void __launch_bounds__(64) k_filter_basis(int M, int Mh, double beta, PreGroupDev gr, Basis bs, int *status)
{
    const int f = blockIdx.x * blockDim.x + threadIdx.x;
    if (f >= M * Mh) return;
    const int j = f % M, k = f / M, G = gr.G, L = gr.L;
    double2 *U = bs.U + (size_t)f * G * G;
    double *sg = bs.sig + (size_t)f * G;
    double2 *W = bs.Q + (size_t)f * L * G;  // A^H, rotated in place
    float2 *E = bs.E + (size_t)f * G * L;
    double *s = bs.s + (size_t)f * L;
    const double nx = j < M / 2 ? j : j - M, ny = k, n2 = nx * nx + ny * ny, twoM = 2.0 / M;
    for (int l = 0; l < L; ++l) {
        s[l] = gr.sw[l] * pow(1.0 + gr.tau[l] * n2, -0.5 * beta);
        for (int g = 0; g < G; ++g) {
            double sn, cs;
            sincospi(twoM * (nx * gr.sx[g * L + l] + ny * gr.sy[g * L + l]), &sn, &cs);
            E[g * L + l] = make_float2((float)cs, (float)sn);
            W[l * G + g] = make_double2(s[l] * cs, -s[l] * sn);  // (A^H)_lg = conj(A_gl)
        }
    }
    for (int g = 0; g < G; ++g)
        for (int r = 0; r < G; ++r) U[g * G + r] = make_double2(g == r ? 1.0 : 0.0, 0.0);
    if (j == M / 2) {  // Nyquist row: no B (zero singular values mark every direction unused)
        for (int r = 0; r < G; ++r) sg[r] = 0.0;
        return;
    }
    bool done = false;
    for (int sweep = 0; sweep < 40 && !done; ++sweep) {
        done = true;
        for (int p = 0; p < G - 1; ++p)
            for (int q = p + 1; q < G; ++q) {
                double a = 0, bq = 0, gr_ = 0, gi = 0;  // ||W_p||^2, ||W_q||^2, W_p^H W_q
                for (int l = 0; l < L; ++l) {
                    const double2 wp = W[l * G + p], wq = W[l * G + q];
                    a += wp.x * wp.x + wp.y * wp.y;
                    bq += wq.x * wq.x + wq.y * wq.y;
                    gr_ += wp.x * wq.x + wp.y * wq.y;
                    gi += wp.x * wq.y - wp.y * wq.x;
                }
                const double ga = sqrt(gr_ * gr_ + gi * gi);
                if (!(ga > 1e-14 * sqrt(a * bq))) continue;
                done = false;
                // rotation [W_p, W_q] <- [c W_p - s e^{-i ph} W_q, s e^{i ph} W_p + c W_q] with
                // g = |g| e^{i ph} zeroes W_p^H W_q when t = s / c solves t^2 - 2 z t - 1 = 0,
                // z = (a - b) / (2 |g|), taking the root of smaller magnitude
                const double z = (a - bq) / (2.0 * ga);
                const double t = -(z >= 0 ? 1.0 : -1.0) / (fabs(z) + sqrt(1.0 + z * z));
                const double c = 1.0 / sqrt(1.0 + t * t), sn = c * t;
                const double er = gr_ / ga, ei = gi / ga;  // e^{i ph}
                auto rot = [&](double2 *X, int rows, int stride) {
                    for (int i = 0; i < rows; ++i) {
                        const double2 xp = X[i * stride + p], xq = X[i * stride + q];
                        // e^{-i ph} xq and e^{i ph} xp
                        const double qr = er * xq.x + ei * xq.y, qi = er * xq.y - ei * xq.x;
                        const double pr = er * xp.x - ei * xp.y, pi = er * xp.y + ei * xp.x;
                        X[i * stride + p] = make_double2(c * xp.x - sn * qr, c * xp.y - sn * qi);
                        X[i * stride + q] = make_double2(sn * pr + c * xq.x, sn * pi + c * xq.y);
                    }
                };
                rot(W, L, G);
                rot(U, G, G);
            }
    }
    if (!done) atomicExch(status, (int)SAFR_ERR_DEVICE);
    // sigma_r = ||W_r||; Q_lr = s_l W_lr / sigma_r (= s_l V_lr); unused directions keep sigma = 0
    double smax = 0;
    for (int r = 0; r < G; ++r) {
        double nr = 0;
        for (int l = 0; l < L; ++l) nr += W[l * G + r].x * W[l * G + r].x + W[l * G + r].y * W[l * G + r].y;
        sg[r] = sqrt(nr);
        smax = fmax(smax, sg[r]);
    }
    for (int r = 0; r < G; ++r) {
        const bool use = sg[r] > 1e-13 * smax && sg[r] > 0;
        const double inv = use ? 1.0 / sg[r] : 0.0;
        if (!use) sg[r] = 0.0;
        for (int l = 0; l < L; ++l)
            W[l * G + r] = make_double2(s[l] * W[l * G + r].x * inv, s[l] * W[l * G + r].y * inv);
    }
}


// ---------------------------------------------------------------------------
// MLP: points p = (f * L + l) * G + r
// ---------------------------------------------------------------------------
__device__ __forceinline__ float gelu(float x) { return 0.5f * x * (1.0f + erff(x * 0.70710678118654752f)); }
__device__ __forceinline__ float gelu_d(float x)
{
    return 0.5f * (1.0f + erff(x * 0.70710678118654752f)) + x * 0.39894228040143268f * expf(-0.5f * x * x);
}

struct MlpArgs {
    int M, L, G, NP;
    const __nv_bfloat16 *w;  // [kParams]
    const double *sig;       // [NF][G]
    const float *hn;         // [L] h_l / 20 km
    float noise_feat;        // noise level / 0.05
    float *wout;             // [NP] w_lr = phi / sigma_r (0 where sigma_r = 0)
    float *phi;              // [NP] or null
    float *act;              // [NP][3][64] pre-activations, or null
    int *nonfinite;          // set if a weight is not finite
};

constexpr int kMlpThreads = 128;
constexpr int kRow = kH + 1;  // padded per-thread row in shared memory

// The four inputs of point p: |n| / (M/2), h_l / 20 km, (log10 sigma_r + 4) / 4, noise / 0.05.
__device__ __forceinline__ void mlp_features(const MlpArgs &a, int p, float x[4], double &sigma)
{
    const int r = p % a.G, fl = p / a.G, l = fl % a.L, f = fl / a.L;
    const int j = f % a.M, k = f / a.M;
    const double nx = j < a.M / 2 ? j : j - a.M;
    sigma = a.sig[(size_t)f * a.G + r];
    x[0] = (float)(sqrt(nx * nx + (double)k * k) / (0.5 * a.M));
    x[1] = a.hn[l];
    x[2] = (float)((log10(fmax(sigma, 1e-12)) + 4.0) / 4.0);
    x[3] = a.noise_feat;
}

// hidden layer: out[i] = b[i] + sum_j W[i][j] in[j] (pre-activation), in and out rows of one thread
__device__ __forceinline__ void dense64(const float *W, const float *b, const float *in, float *out)
{
    for (int i = 0; i < kH; ++i) {
        float acc = b[i];
#pragma unroll 16
        for (int j = 0; j < kH; ++j) acc += W[i * kH + j] * in[j];
        out[i] = acc;
    }
}

__global__ void __launch_bounds__(kMlpThreads) k_mlp_forward(MlpArgs a)
{
    extern __shared__ float sm[];
    float *wt = sm;                                            // [kParams] FP32 copy of the BF16 weights
    float *r0 = sm + ((kParams + 31) & ~31) + threadIdx.x * 2 * kRow;  // two rows of this thread
    float *r1 = r0 + kRow;
    for (int i = threadIdx.x; i < kParams; i += blockDim.x) wt[i] = __bfloat162float(a.w[i]);
    __syncthreads();
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= a.NP) return;
    float x[4];
    double sigma;
    mlp_features(a, p, x, sigma);
    float *act = a.act ? a.act + (size_t)p * 3 * kH : nullptr;
    // layer 0 (4 -> 64)
    for (int i = 0; i < kH; ++i) {
        float acc = wt[kOffB0 + i];
#pragma unroll
        for (int q = 0; q < 4; ++q) acc += wt[kOffW0 + i * 4 + q] * x[q];
        if (act) act[i] = acc;
        r0[i] = gelu(acc);
    }
    dense64(wt + kOffW1, wt + kOffB1, r0, r1);
    for (int i = 0; i < kH; ++i) {
        if (act) act[kH + i] = r1[i];
        r1[i] = gelu(r1[i]);
    }
    dense64(wt + kOffW2, wt + kOffB2, r1, r0);
    for (int i = 0; i < kH; ++i) {
        if (act) act[2 * kH + i] = r0[i];
        r0[i] = gelu(r0[i]);
    }
    float o = wt[kOffB3];
    for (int j = 0; j < kH; ++j) o += wt[kOffW3 + j] * r0[j];
    const float ph = 1.0f / (1.0f + expf(-o));
    const float w = sigma > 0.0 ? (float)(ph / sigma) : 0.0f;
    if (!isfinite(w) && a.nonfinite) atomicExch(a.nonfinite, 1);
    a.wout[p] = w;
    if (a.phi) a.phi[p] = ph;
}

struct MlpBackArgs {
    int M, L, G, NP;
    const __nv_bfloat16 *w;
    const double *sig;
    const float *hn;
    float noise_feat;
    const float *act, *phi;
    const float *gw;   // [NP] dLoss / dw
    float *partial;    // [gridDim.x][kParams]
};

// Gradient of the loss with respect to the parameters, summed over this block's
// points in a fixed order (per-block partials; k_sum_partials adds the blocks).
__global__ void __launch_bounds__(kMlpThreads) k_mlp_backward(MlpBackArgs a)
{
    extern __shared__ float sm[];
    float *wt = sm;
    float *dl = sm + ((kParams + 31) & ~31);  // [128][kRow] delta of the current layer
    float *hh = dl + kMlpThreads * kRow;      // [128][kRow] input of the current layer
    float *xs = hh + kMlpThreads * kRow;      // [128][4] network inputs
    float *go = xs + kMlpThreads * 4;         // [128] dLoss / d(output)
    const int t = threadIdx.x;
    for (int i = t; i < kParams; i += blockDim.x) wt[i] = __bfloat162float(a.w[i]);
    const int p = blockIdx.x * blockDim.x + t;
    const bool act = p < a.NP;
    float *D = dl + t * kRow, *Hh = hh + t * kRow;
    float x[4] = {0, 0, 0, 0};
    double sigma = 0;
    float g = 0;
    const float *ac = act ? a.act + (size_t)p * 3 * kH : nullptr;
    if (act) {
        MlpArgs fa{a.M, a.L, a.G, a.NP, a.w, a.sig, a.hn, a.noise_feat, nullptr, nullptr, nullptr, nullptr};
        mlp_features(fa, p, x, sigma);
        if (sigma > 0.0) {
            const float ph = a.phi[p];
            g = (float)(a.gw[p] / sigma) * ph * (1.0f - ph);  // w = phi / sigma, phi = logistic(o)
        }
    }
    for (int q = 0; q < 4; ++q) xs[t * 4 + q] = x[q];
    go[t] = g;
    __syncthreads();
    // output layer: h3 = gelu(a3); delta3_i = g W3_i gelu'(a3_i)
    for (int i = 0; i < kH; ++i) {
        const float a3 = ac ? ac[2 * kH + i] : 0.0f;
        Hh[i] = ac ? gelu(a3) : 0.0f;
        D[i] = g * wt[kOffW3 + i] * gelu_d(a3);
    }
    __syncthreads();
    float *out = a.partial + (size_t)blockIdx.x * kParams;
    if (t < kH) {
        float s3 = 0;
        for (int q = 0; q < kMlpThreads; ++q) s3 += go[q] * hh[q * kRow + t];
        out[kOffW3 + t] = s3;
    }
    if (t == 0) {
        float s3 = 0;
        for (int q = 0; q < kMlpThreads; ++q) s3 += go[q];
        out[kOffB3] = s3;
    }
    // hidden layers 2 and 1: dW = sum_points delta (x) input, delta_prev = (W^T delta) * gelu'(a_prev)
    for (int layer = 2; layer >= 1; --layer) {
        const int offW = layer == 2 ? kOffW2 : kOffW1, offB = layer == 2 ? kOffB2 : kOffB1;
        const int aprev = layer - 1;  // pre-activation index of this layer's input
        __syncthreads();
        for (int i = 0; i < kH; ++i) Hh[i] = ac ? gelu(ac[aprev * kH + i]) : 0.0f;
        __syncthreads();
        for (int e = t; e < kH * kH; e += blockDim.x) {
            const int i = e / kH, jj = e % kH;
            float sacc = 0;
            for (int q = 0; q < kMlpThreads; ++q) sacc += dl[q * kRow + i] * hh[q * kRow + jj];
            out[offW + e] = sacc;
        }
        if (t < kH) {
            float sb = 0;
            for (int q = 0; q < kMlpThreads; ++q) sb += dl[q * kRow + t];
            out[offB + t] = sb;
        }
        __syncthreads();
        // delta of the previous layer (own row): sum_i W[i][j] delta_i, times gelu'(a_prev_j)
        float nd[kH];
        for (int jj = 0; jj < kH; ++jj) {
            float sacc = 0;
            for (int i = 0; i < kH; ++i) sacc += wt[offW + i * kH + jj] * D[i];
            nd[jj] = sacc * (ac ? gelu_d(ac[aprev * kH + jj]) : 0.0f);
        }
        __syncthreads();
        for (int jj = 0; jj < kH; ++jj) D[jj] = nd[jj];
    }
    __syncthreads();
    // input layer: dW0[i][q] = sum_points delta1_i x_q
    for (int e = t; e < kH * 4; e += blockDim.x) {
        const int i = e / 4, q = e % 4;
        float sacc = 0;
        for (int u = 0; u < kMlpThreads; ++u) sacc += dl[u * kRow + i] * xs[u * 4 + q];
        out[kOffW0 + e] = sacc;
    }
    if (t < kH) {
        float sb = 0;
        for (int u = 0; u < kMlpThreads; ++u) sb += dl[u * kRow + t];
        out[kOffB0 + t] = sb;
    }
}

// grad[i] = scale * sum over blocks (fixed order) of partial[block][i]
__global__ void k_sum_partials(const float *partial, int nblocks, float scale, float *grad)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= kParams) return;
    float s = 0;
    for (int b = 0; b < nblocks; ++b) s += partial[(size_t)b * kParams + i];
    grad[i] = s * scale;
}

// Adam on FP32 master weights; the BF16 copy is what the MLP kernels read
__global__ void k_adam(float *master, float *m, float *v, const float *grad, __nv_bfloat16 *wb, float lr, float b1,
                       float b2, float eps, float c1, float c2)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= kParams) return;
    const float g = grad[i];
    const float mi = b1 * m[i] + (1.0f - b1) * g, vi = b2 * v[i] + (1.0f - b2) * g * g;
    m[i] = mi;
    v[i] = vi;
    const float w = master[i] - lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    master[i] = w;
    wb[i] = __float2bfloat16_rn(w);
}

// ---------------------------------------------------------------------------
// training frames: the layered model of Section 2 seen through the aperture,
// and the loss with its gradient with respect to the weights w
// ---------------------------------------------------------------------------
constexpr int kFrameThreads = 256;  // frames per step (one thread per frame in the per-frequency kernels)

// phi_l(n) of frame F at stored frequency (j, k), k < M/2: complex normal with
// variance var, from the Box-Muller pair of Philox counter (F, k M + j, l, 0).
// On the row k = 0 the frequencies j > M/2 are the conjugates of M - j, so
// every layer is a real screen.
__device__ __forceinline__ float2 layer_coeff(int M, int L, const float *var, uint32_t F, int j, int k, int l,
                                              uint32_t k0, uint32_t k1)
{
    const bool flip = k == 0 && j > M / 2;
    const int f = k * M + (flip ? M - j : j);
    const float sd = sqrtf(0.5f * var[(size_t)f * L + l]);
    const float2 z = normal2(F, (uint32_t)f, (uint32_t)l, 0u, k0, k1);
    return make_float2(sd * z.x, flip ? -sd * z.y : sd * z.y);
}

struct CleanArgs {
    int M, L, G, NF;
    const float2 *E;          // [NF][G][L] e^{i theta_gl}
    const float *var;         // [NF][L]
    uint32_t k0, k1, frame0, nwrap;
    float2 *c;                // [256][G][NF] noise-free data spectra
};

// One block per stored frequency, one thread per frame: c_g(n) = sum_l e^{i theta_gl(n)} phi_l(n).
__global__ void __launch_bounds__(kFrameThreads) k_tf_clean(CleanArgs a)
{
    const int f = blockIdx.x, j = f % a.M, k = f / a.M, t = threadIdx.x;
    const uint32_t F = (a.frame0 + (uint32_t)t) % a.nwrap;
    float cr[SAFR_MAX_GROUP_G], ci[SAFR_MAX_GROUP_G];
#pragma unroll
    for (int g = 0; g < SAFR_MAX_GROUP_G; ++g) cr[g] = ci[g] = 0.0f;
    if (j != a.M / 2) {
        const float2 *E = a.E + (size_t)f * a.G * a.L;
        for (int l = 0; l < a.L; ++l) {
            const float2 p = layer_coeff(a.M, a.L, a.var, F, j, k, l, a.k0, a.k1);
#pragma unroll
            for (int g = 0; g < SAFR_MAX_GROUP_G; ++g)
                if (g < a.G) {
                    const float2 e = E[g * a.L + l];
                    cr[g] += e.x * p.x - e.y * p.y;
                    ci[g] += e.x * p.y + e.y * p.x;
                }
        }
    }
#pragma unroll
    for (int g = 0; g < SAFR_MAX_GROUP_G; ++g)
        if (g < a.G) a.c[((size_t)t * a.G + g) * a.NF + f] = make_float2(cr[g], ci[g]);
}

struct MaskArgs {
    int M, G, NF;
    const float2 *c;              // [256][G][NF]
    const unsigned char *mask;    // [M][M] pupil on the grid (zero outside the P x P pupil square)
    float noise;                  // per-pixel noise std / RMS of the noise-free wavefront over the mask
    uint32_t k0, k1, frame0, nwrap;
    float2 *d;                    // [256][G][NF] data spectra
};

constexpr int kMaskThreads = 256;
constexpr int kMaxTrainM = 64;  // the direct DFTs of the aperture step hold two M x M complex tiles in shared memory

// One block per (frame, star): psi = IDFT2(c) (a real field), psi <- mask (psi + noise), d = DFT2(psi).
// The noise at grid pixel (p, q) is sigma z, z the first normal of Philox counter (F, p M + q, g, 1),
// sigma = noise x RMS of the masked noise-free wavefront.  Direct DFTs (M <= 64), twiddles from a table
// indexed by the exact residue (j p) mod M.
__global__ void __launch_bounds__(kMaskThreads) k_tf_mask(MaskArgs a)
{
    extern __shared__ float2 sm2[];
    const int M = a.M, MM = M * M, Mh = M / 2;
    float2 *X = sm2, *Y = sm2 + MM, *tw = sm2 + 2 * MM;
    float *red = (float *)(tw + M);
    const int t = blockIdx.x / a.G, g = blockIdx.x % a.G;
    const uint32_t F = (a.frame0 + (uint32_t)t) % a.nwrap;
    const float2 *c = a.c + ((size_t)t * a.G + g) * a.NF;
    for (int i = threadIdx.x; i < M; i += blockDim.x) {
        float s, co;
        sincospif(2.0f * (float)i / (float)M, &s, &co);
        tw[i] = make_float2(co, s);  // e^{+2 pi i i / M}
    }
    // full Hermitian spectrum X[j][k]
    for (int i = threadIdx.x; i < MM; i += blockDim.x) {
        const int j = i / M, k = i % M;
        float2 v = make_float2(0.0f, 0.0f);
        if (k < Mh) v = c[k * M + j];
        else if (k > Mh) {
            const float2 u = c[(M - k) * M + (M - j) % M];
            v = make_float2(u.x, -u.y);
        }
        X[i] = v;
    }
    __syncthreads();
    // inverse along j: Y[p][k] = sum_j X[j][k] e^{+2 pi i j p / M}
    for (int i = threadIdx.x; i < MM; i += blockDim.x) {
        const int p = i / M, k = i % M;
        float re = 0.0f, im = 0.0f;
        for (int j = 0; j < M; ++j) {
            const float2 x = X[j * M + k], w = tw[(j * p) % M];
            re += x.x * w.x - x.y * w.y;
            im += x.x * w.y + x.y * w.x;
        }
        Y[i] = make_float2(re, im);
    }
    __syncthreads();
    // inverse along k, real part, 1/M^2; mask; sums for the RMS
    const float inv = 1.0f / (float)MM;
    float s2 = 0.0f, cnt = 0.0f;
    for (int i = threadIdx.x; i < MM; i += blockDim.x) {
        const int p = i / M, q = i % M;
        float re = 0.0f;
        for (int k = 0; k < M; ++k) {
            const float2 y = Y[p * M + k], w = tw[(k * q) % M];
            re += y.x * w.x - y.y * w.y;
        }
        const float m = a.mask[i] ? 1.0f : 0.0f;
        const float v = m * re * inv;
        X[i] = make_float2(v, m);
        s2 += v * v;
        cnt += m;
    }
    for (int o = 16; o > 0; o >>= 1) {
        s2 += __shfl_xor_sync(0xffffffffu, s2, o);
        cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
    }
    if ((threadIdx.x & 31) == 0) {
        red[threadIdx.x >> 5] = s2;
        red[8 + (threadIdx.x >> 5)] = cnt;
    }
    __syncthreads();
    float S2 = 0.0f, N = 0.0f;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
        S2 += red[w];
        N += red[8 + w];
    }
    const float sigma = N > 0.0f ? a.noise * sqrtf(S2 / N) : 0.0f;
    // noise on the mask pixels, then forward along q for k < M/2: Y[p][k] = sum_q psi[p][q] e^{-2 pi i k q / M}
    for (int i = threadIdx.x; i < MM; i += blockDim.x) {
        const float2 v = X[i];
        if (v.y != 0.0f && sigma > 0.0f) {
            const float2 z = normal2(F, (uint32_t)i, (uint32_t)g, 1u, a.k0, a.k1);
            X[i] = make_float2(v.x + sigma * z.x, v.y);
        }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < M * Mh; i += blockDim.x) {
        const int p = i / Mh, k = i % Mh;
        float re = 0.0f, im = 0.0f;
        for (int q = 0; q < M; ++q) {
            const float x = X[p * M + q].x;
            const float2 w = tw[(k * q) % M];
            re += x * w.x;
            im -= x * w.y;
        }
        Y[p * Mh + k] = make_float2(re, im);
    }
    __syncthreads();
    // forward along p: d[k][j] = sum_p Y[p][k] e^{-2 pi i j p / M}
    float2 *d = a.d + ((size_t)t * a.G + g) * a.NF;
    for (int i = threadIdx.x; i < M * Mh; i += blockDim.x) {
        const int k = i / M, j = i % M;
        float re = 0.0f, im = 0.0f;
        for (int p = 0; p < M; ++p) {
            const float2 y = Y[p * Mh + k], w = tw[(j * p) % M];
            re += y.x * w.x + y.y * w.y;
            im += y.y * w.x - y.x * w.y;
        }
        d[k * M + j] = make_float2(re, im);
    }
}

inline size_t mask_smem(int M) { return (size_t)(2 * M * M + M) * sizeof(float2) + 16 * sizeof(float); }

struct FrameArgs {
    int M, L, G, NF;
    Basis bs;
    const float *w;           // [NP]
    uint32_t k0, k1;          // generator key
    uint32_t frame0, nwrap;   // thread t holds frame (frame0 + t) mod nwrap
    const float2 *d;          // [256][G][NF] data spectra (k_tf_mask)
    float *gw;                // [NP] or null: sum over the block's frames of dLoss / dw
    float *loss, *energy;     // [NF]: sums over the block's frames of |error|^2 and |phi_l(n)|^2
};

// sum over the block of v[0..G) per thread; thread r < G holds the sum of component r
__device__ __forceinline__ void block_sum_g(float (&v)[SAFR_MAX_GROUP_G], int G, float *red, float *out)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
    for (int r = 0; r < SAFR_MAX_GROUP_G; ++r)
        if (r < G) {
            float x = v[r];
            for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
            if (lane == 0) red[warp * SAFR_MAX_GROUP_G + r] = x;
        }
    __syncthreads();
    if ((int)threadIdx.x < G) {
        float sacc = 0;
        for (int q = 0; q < nw; ++q) sacc += red[q * SAFR_MAX_GROUP_G + threadIdx.x];
        *out = sacc;
    }
    __syncthreads();
}

// One block per stored frequency f = k * M + j, one thread per frame.  The frequency's
// weight in the full spectrum is 2 for k > 0 (its conjugate partner) and 1 for k = 0
// (both j and M - j are stored).
__global__ void __launch_bounds__(kFrameThreads) k_filter_frames(FrameArgs a)
{
    __shared__ float red[(kFrameThreads / 32) * SAFR_MAX_GROUP_G];
    const int f = blockIdx.x, j = f % a.M, k = f / a.M, G = a.G, L = a.L, t = threadIdx.x;
    if (j == a.M / 2) {  // Nyquist row: nothing is reconstructed there
        if (a.gw)
            for (int i = t; i < L * G; i += blockDim.x) a.gw[(size_t)f * L * G + i] = 0.0f;
        if (t == 0) a.loss[f] = a.energy[f] = 0.0f;
        return;
    }
    const float wf = k == 0 ? 1.0f : 2.0f;
    const uint32_t F = (a.frame0 + (uint32_t)t) % a.nwrap;
    const double2 *U = a.bs.U + (size_t)f * G * G;
    const double2 *Q = a.bs.Q + (size_t)f * L * G;
    const float *w = a.w + (size_t)f * L * G;
    float dr[SAFR_MAX_GROUP_G], di[SAFR_MAX_GROUP_G];
#pragma unroll
    for (int g = 0; g < SAFR_MAX_GROUP_G; ++g) {
        dr[g] = di[g] = 0.0f;
        if (g < G) {
            const float2 v = a.d[((size_t)t * G + g) * a.NF + f];
            dr[g] = v.x;
            di[g] = v.y;
        }
    }
    // y_r = sum_g conj(U_gr) d_g
    float yr[SAFR_MAX_GROUP_G], yi[SAFR_MAX_GROUP_G];
#pragma unroll
    for (int r = 0; r < SAFR_MAX_GROUP_G; ++r) {
        yr[r] = yi[r] = 0.0f;
        if (r < G)
            for (int g = 0; g < G; ++g) {
                const double2 u = U[g * G + r];
                yr[r] += (float)u.x * dr[g] + (float)u.y * di[g];
                yi[r] += (float)u.x * di[g] - (float)u.y * dr[g];
            }
    }
    float lsum = 0.0f, esum = 0.0f;
    for (int l = 0; l < L; ++l) {
        const float2 ph = layer_coeff(a.M, L, a.bs.var, F, j, k, l, a.k0, a.k1);
        float qyr[SAFR_MAX_GROUP_G], qyi[SAFR_MAX_GROUP_G];
        float er = -ph.x, ei = -ph.y;  // rec_l - phi_l, rec_l = sum_r Q_lr w_lr y_r
#pragma unroll
        for (int r = 0; r < SAFR_MAX_GROUP_G; ++r) {
            qyr[r] = qyi[r] = 0.0f;
            if (r < G) {
                const double2 q = Q[l * G + r];
                qyr[r] = (float)q.x * yr[r] - (float)q.y * yi[r];
                qyi[r] = (float)q.x * yi[r] + (float)q.y * yr[r];
                er += w[l * G + r] * qyr[r];
                ei += w[l * G + r] * qyi[r];
            }
        }
        lsum += er * er + ei * ei;
        esum += ph.x * ph.x + ph.y * ph.y;
        if (a.gw) {  // d|e|^2 / dw_lr = 2 Re(conj(e) Q_lr y_r)
            float gv[SAFR_MAX_GROUP_G];
#pragma unroll
            for (int r = 0; r < SAFR_MAX_GROUP_G; ++r) gv[r] = 2.0f * wf * (er * qyr[r] + ei * qyi[r]);
            float sum_r = 0.0f;
            block_sum_g(gv, G, red, &sum_r);
            if (t < G) a.gw[((size_t)f * L + l) * G + t] = sum_r;
        }
    }
    float pair[SAFR_MAX_GROUP_G];
    pair[0] = wf * lsum;
    pair[1] = wf * esum;
    float tot = 0.0f;
    block_sum_g(pair, 2, red, &tot);
    if (t == 0) a.loss[f] = tot;
    if (t == 1) a.energy[f] = tot;
}

// plain SAFR's weights w_lr = g(sigma_r) = sigma_r / (sigma_r^2 + alpha) (Tikhonov)
__global__ void k_filter_tikhonov(int NP, int L, int G, const double *sig, double alpha, float *w)
{
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= NP) return;
    const int r = p % G, f = p / (G * L);
    const double s = sig[(size_t)f * G + r];
    w[p] = s > 0.0 ? (float)(s / (s * s + alpha)) : 0.0f;
}

template <typename C>
__device__ __forceinline__ void store_b(C *p, double re, double im);
template <>
__device__ __forceinline__ void store_b<float2>(float2 *p, double re, double im) { *p = make_float2((float)re, (float)im); }
template <>
__device__ __forceinline__ void store_b<double2>(double2 *p, double re, double im) { *p = make_double2(re, im); }

// B_lg(n) = sum_r Q_lr w_lr conj(U_gr) in the frame kernels' layout (j in warp-FFT order).
template <typename C>
__global__ void k_filter_assemble(int M, int Mh, int L, int G, int sumLG, int b_row0, Basis bs, const float *w, C *B)
{
    const long idx = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (long)M * Mh * L) return;
    const int l = (int)(idx % L);
    const int f = (int)(idx / L), j = f % M, k = f / M;
    C *Bl = B + ((size_t)k * sumLG + b_row0 + (size_t)l * G) * M + wfft_pos_of_j(j, M);
    for (int g = 0; g < G; ++g) {
        double re = 0.0, im = 0.0;
        if (j != M / 2)
            for (int r = 0; r < G; ++r) {
                const double2 q = bs.Q[((size_t)f * L + l) * G + r], u = bs.U[((size_t)f * G + g) * G + r];
                const double ww = w[((size_t)f * L + l) * G + r];
                // q w conj(u)
                re += ww * (q.x * u.x + q.y * u.y);
                im += ww * (q.y * u.x - q.x * u.y);
            }
        store_b(Bl + (size_t)g * M, re, im);
    }
}

}  // namespace safr

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
namespace safr {

struct FilterState {
    int NF = 0, NP = 0;
    Basis bs{};
    float *hn = nullptr, *w = nullptr, *wplain = nullptr, *phi = nullptr, *act = nullptr, *gw = nullptr;
    float *partial = nullptr, *grad = nullptr, *master = nullptr, *m = nullptr, *v = nullptr;
    float *loss = nullptr, *energy = nullptr;
    float2 *cbuf = nullptr, *dbuf = nullptr;  // [256][G][NF] noise-free and measured data spectra of a step
    unsigned char *mask = nullptr;            // [M][M] pupil on the grid
    __nv_bfloat16 *wb = nullptr;
    int *flag = nullptr;
    bool basis_ready = false, training = false;
};

void filter_invalidate(safr_plan_s *pl)
{
    FilterState *fs = (FilterState *)pl->filter;
    if (fs) fs->basis_ready = false;
    pl->filter_learned = 0;
}

void filter_free(safr_plan_s *pl)
{
    FilterState *fs = (FilterState *)pl->filter;
    if (!fs) return;
    void *bufs[] = {fs->bs.U, fs->bs.sig, fs->bs.Q, fs->bs.E, fs->bs.s, fs->bs.var, fs->hn, fs->w, fs->wplain,
                    fs->phi, fs->act, fs->gw, fs->partial, fs->grad, fs->master, fs->m, fs->v, fs->loss,
                    fs->energy, fs->wb, fs->flag, fs->cbuf, fs->dbuf, fs->mask};
    for (void *b : bufs)
        if (b) cudaFree(b);
    delete fs;
    pl->filter = nullptr;
}

}  // namespace safr

namespace {

using safr::FilterState;

struct FilterDeviceGuard {
    int prev = -1;
    bool ok = false;
    explicit FilterDeviceGuard(int dev)
    {
        if (cudaGetDevice(&prev) != cudaSuccess) return;
        if (prev != dev && cudaSetDevice(dev) != cudaSuccess) return;
        ok = true;
    }
    ~FilterDeviceGuard()
    {
        if (ok && prev >= 0) cudaSetDevice(prev);
    }
};

constexpr size_t kMaxTrainPoints = (size_t)4 << 20;  // activations of 4M points: 3 GB

template <typename T>
bool dalloc(T **p, size_t n)
{
    return cudaMalloc((void **)p, n * sizeof(T)) == cudaSuccess;
}

size_t fwd_smem() { return (((size_t)safr::kParams + 31) & ~(size_t)31) * 4 + (size_t)safr::kMlpThreads * 2 * safr::kRow * 4; }
size_t bwd_smem()
{
    return (((size_t)safr::kParams + 31) & ~(size_t)31) * 4 + (size_t)safr::kMlpThreads * (2 * safr::kRow + 5) * 4;
}

// The basis and the inference buffers (and, for training, the training buffers).
safr_status filter_prepare(safr_plan_s *pl, bool training, cudaStream_t st)
{
    if (pl->ngroups != 1) return SAFR_ERR_UNSUPPORTED_SIZE;  // one star group (no split tomography)
    if (!pl->precomputed) return SAFR_ERR_NOT_PRECOMPUTED;
    FilterState *fs = (FilterState *)pl->filter;
    if (!fs) {
        fs = new (std::nothrow) FilterState();
        if (!fs) return SAFR_ERR_OOM;
        pl->filter = fs;
    }
    const int M = pl->M, Mh = pl->Mh, L = pl->L, G = pl->grp[0].G;
    fs->NF = M * Mh;
    fs->NP = fs->NF * L * G;
    if (training && ((size_t)fs->NP > kMaxTrainPoints || M > safr::kMaxTrainM)) return SAFR_ERR_UNSUPPORTED_SIZE;
    if (!fs->bs.U) {
        fs->bs.NF = fs->NF;
        if (!dalloc(&fs->bs.U, (size_t)fs->NF * G * G) || !dalloc(&fs->bs.sig, (size_t)fs->NF * G) ||
            !dalloc(&fs->bs.Q, (size_t)fs->NP) || !dalloc(&fs->bs.E, (size_t)fs->NF * G * L) ||
            !dalloc(&fs->bs.s, (size_t)fs->NF * L) || !dalloc(&fs->bs.var, (size_t)fs->NF * L) ||
            !dalloc(&fs->hn, (size_t)L) || !dalloc(&fs->w, (size_t)fs->NP) || !dalloc(&fs->wb, (size_t)safr::kParams) ||
            !dalloc(&fs->flag, 1))
            return SAFR_ERR_OOM;
        std::vector<float> hn(L);
        for (int l = 0; l < L; ++l) hn[l] = (float)(pl->h[l] / 20e3);
        if (cudaMemcpy(fs->hn, hn.data(), L * sizeof(float), cudaMemcpyHostToDevice) != cudaSuccess)
            return SAFR_ERR_CUDA;
    }
    if (training && !fs->training) {
        const int nblk = (fs->NP + safr::kMlpThreads - 1) / safr::kMlpThreads;
        if (!dalloc(&fs->wplain, (size_t)fs->NP) || !dalloc(&fs->phi, (size_t)fs->NP) ||
            !dalloc(&fs->act, (size_t)fs->NP * 3 * safr::kH) || !dalloc(&fs->gw, (size_t)fs->NP) ||
            !dalloc(&fs->partial, (size_t)nblk * safr::kParams) || !dalloc(&fs->grad, (size_t)safr::kParams) ||
            !dalloc(&fs->master, (size_t)safr::kParams) || !dalloc(&fs->m, (size_t)safr::kParams) ||
            !dalloc(&fs->v, (size_t)safr::kParams) || !dalloc(&fs->loss, (size_t)fs->NF) ||
            !dalloc(&fs->energy, (size_t)fs->NF) ||
            !dalloc(&fs->cbuf, (size_t)safr::kFrameThreads * G * fs->NF) ||
            !dalloc(&fs->dbuf, (size_t)safr::kFrameThreads * G * fs->NF) || !dalloc(&fs->mask, (size_t)M * M))
            return SAFR_ERR_OOM;
        // the pupil of the geometry (an annulus, or the whole P x P square) at offset (M - P) / 2
        std::vector<unsigned char> mk((size_t)M * M, 0);
        const int P = pl->P, o = (M - P) / 2;
        const double ro = pl->diameter / 2.0, ri = pl->obstruction * pl->diameter / 2.0;
        for (int a = 0; a < P; ++a)
            for (int b = 0; b < P; ++b) {
                const double x = (a - (P - 1) / 2.0) * pl->delta, y = (b - (P - 1) / 2.0) * pl->delta;
                const double r2 = x * x + y * y;
                mk[(size_t)(o + a) * M + o + b] = pl->diameter <= 0 ? 1 : (r2 <= ro * ro && r2 >= ri * ri);
            }
        if (cudaMemcpy(fs->mask, mk.data(), mk.size(), cudaMemcpyHostToDevice) != cudaSuccess) return SAFR_ERR_CUDA;
        fs->training = true;
    }
    if (!safr::smem_limit_allows((const void *)safr::k_mlp_forward, fwd_smem()) ||
        !safr::smem_limit_allows((const void *)safr::k_mlp_backward, bwd_smem()) ||
        (training && !safr::smem_limit_allows((const void *)safr::k_tf_mask, safr::mask_smem(M))))
        return SAFR_ERR_UNSUPPORTED_SIZE;
    if (!fs->basis_ready) {
        const safr::Group &g = pl->grp[0];
        safr::PreGroupDev d;
        d.G = g.G;
        d.L = L;
        d.b_row0 = g.b_row0;
        d.alpha = g.alpha;
        d.sx = pl->d_pre;
        d.sy = d.sx + (size_t)g.G * L;
        d.sw = d.sy + (size_t)g.G * L;
        d.tau = d.sw + L;
        safr::k_filter_basis<<<(fs->NF + 63) / 64, 64, 0, st>>>(M, Mh, pl->beta, d, fs->bs, pl->d_status);
        if (cudaGetLastError() != cudaSuccess) return SAFR_ERR_CUDA;
        fs->basis_ready = true;
    }
    return SAFR_OK;
}

safr::MlpArgs mlp_args(safr_plan_s *pl, FilterState *fs, double noise_level, float *wout, float *phi, float *act)
{
    return safr::MlpArgs{pl->M, pl->L, pl->grp[0].G, fs->NP, fs->wb, fs->bs.sig, fs->hn, (float)(noise_level / 0.05),
                         wout, phi, act, fs->flag};
}

cudaError_t mlp_forward(safr_plan_s *pl, FilterState *fs, double noise, float *wout, float *phi, float *act,
                        cudaStream_t st)
{
    const int nblk = (fs->NP + safr::kMlpThreads - 1) / safr::kMlpThreads;
    safr::k_mlp_forward<<<nblk, safr::kMlpThreads, fwd_smem(), st>>>(mlp_args(pl, fs, noise, wout, phi, act));
    return cudaGetLastError();
}

cudaError_t assemble(safr_plan_s *pl, FilterState *fs, const float *w, cudaStream_t st)
{
    const long n = (long)pl->M * pl->Mh * pl->L;
    const int th = 128, nb = (int)((n + th - 1) / th);
    if (pl->precision == SAFR_FP64)
        safr::k_filter_assemble<double2><<<nb, th, 0, st>>>(pl->M, pl->Mh, pl->L, pl->grp[0].G, pl->sumLG,
                                                              pl->grp[0].b_row0, fs->bs, w, (double2 *)pl->d_B);
    else
        safr::k_filter_assemble<float2><<<nb, th, 0, st>>>(pl->M, pl->Mh, pl->L, pl->grp[0].G, pl->sumLG,
                                                             pl->grp[0].b_row0, fs->bs, w, (float2 *)pl->d_B);
    return cudaGetLastError();
}

// sum of the loss and energy arrays (host)
bool read_loss(FilterState *fs, double &loss, double &energy, cudaStream_t st)
{
    std::vector<float> a(fs->NF), b(fs->NF);
    if (cudaMemcpyAsync(a.data(), fs->loss, fs->NF * sizeof(float), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaMemcpyAsync(b.data(), fs->energy, fs->NF * sizeof(float), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
        return false;
    loss = energy = 0;
    for (int i = 0; i < fs->NF; ++i) {
        loss += a[i];
        energy += b[i];
    }
    return true;
}

// deterministic host generator for the initial weights (splitmix64, Box-Muller)
struct InitRng {
    uint64_t s;
    uint64_t next()
    {
        uint64_t z = (s += 0x9E3779B97F4A7C15ull);
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
        return z ^ (z >> 31);
    }
    double normal()
    {
        const double u1 = ((double)(next() >> 11) + 0.5) * (1.0 / 9007199254740992.0);
        const double u2 = ((double)(next() >> 11) + 0.5) * (1.0 / 9007199254740992.0);
        return std::sqrt(-2.0 * std::log(u1)) * std::cos(2.0 * 3.14159265358979323846 * u2);
    }
};

}  // namespace

extern "C" {

safr_status safr_filter_apply(safr_plan_t pl, const float *weights, double noise_level, cudaStream_t st)
{
    if (!pl || !weights || !(noise_level >= 0) || !std::isfinite(noise_level)) return SAFR_ERR_INVALID_ARG;
    FilterDeviceGuard guard(pl->device);
    if (!guard.ok) return SAFR_ERR_CUDA;
    safr_status s = filter_prepare(pl, false, st);
    if (s != SAFR_OK) return s;
    FilterState *fs = (FilterState *)pl->filter;
    std::vector<__nv_bfloat16> wb(safr::kParams);
    for (int i = 0; i < safr::kParams; ++i) {
        if (!std::isfinite(weights[i])) return SAFR_ERR_INVALID_ARG;
        wb[i] = __float2bfloat16_rn(weights[i]);
    }
    int flag = 0;
    if (cudaMemcpyAsync(fs->wb, wb.data(), wb.size() * sizeof(__nv_bfloat16), cudaMemcpyHostToDevice, st) !=
            cudaSuccess ||
        cudaMemsetAsync(fs->flag, 0, sizeof(int), st) != cudaSuccess ||
        mlp_forward(pl, fs, noise_level, fs->w, nullptr, nullptr, st) != cudaSuccess ||
        cudaMemcpyAsync(&flag, fs->flag, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
        return SAFR_ERR_CUDA;
    if (flag) {  // a weight is not finite: plain SAFR stays
        if (safr::launch_precompute(pl, st) != cudaSuccess || cudaStreamSynchronize(st) != cudaSuccess)
            return SAFR_ERR_CUDA;
        pl->filter_learned = 0;
        return SAFR_ERR_DEVICE;
    }
    if (assemble(pl, fs, fs->w, st) != cudaSuccess || cudaStreamSynchronize(st) != cudaSuccess)
        return SAFR_ERR_CUDA;
    pl->filter_learned = 1;
    return SAFR_OK;
}

safr_status safr_filter_reset(safr_plan_t pl, cudaStream_t st)
{
    if (!pl) return SAFR_ERR_INVALID_ARG;
    FilterDeviceGuard guard(pl->device);
    if (!guard.ok) return SAFR_ERR_CUDA;
    if (safr::launch_precompute(pl, st) != cudaSuccess) return SAFR_ERR_CUDA;
    pl->precomputed = 1;
    pl->filter_learned = 0;
    return SAFR_OK;
}

}  // extern "C"

namespace {

// E|phi_l(n)|^2 of a layer's DFT over its own M x M grid (pitch c_l delta, period
// 2 c_l T) for the von Karman phase spectrum 0.023 r0_l^{-5/3} (f^2 + L0^{-2})^{-11/6},
// r0_l = r0 gamma_l^{-3/5}, of a real screen whose complex Fourier coefficients
// carry half the spectrum's power each; no piston, nothing on the Nyquist row.
double layer_variance(const safr_plan_s *pl, int l, int j, int k, double r0, double L0)
{
    const int M = pl->M;
    if (j == M / 2 || (j == 0 && k == 0)) return 0.0;
    const double nx = j < M / 2 ? j : j - M, ny = k;
    const double period = 2.0 * pl->grp[0].c[l] * pl->T;
    const double f2 = (nx * nx + ny * ny) / (period * period);
    const double psd = 0.023 * std::pow(r0, -5.0 / 3.0) * pl->gamma[l] * std::pow(f2 + 1.0 / (L0 * L0), -11.0 / 6.0);
    const double m2 = (double)M * M;
    return m2 * m2 * 0.5 * psd / (period * period);
}

// The data spectra of the 256 frames (frame0 + t) mod nwrap, t < 256, drawn with key (k0, k1).
cudaError_t make_frames(safr_plan_s *pl, FilterState *fs, uint32_t k0, uint32_t k1, uint32_t frame0, uint32_t nwrap,
                        double noise, cudaStream_t st)
{
    const int G = pl->grp[0].G;
    safr::CleanArgs ca{pl->M, pl->L, G, fs->NF, fs->bs.E, fs->bs.var, k0, k1, frame0, nwrap, fs->cbuf};
    safr::k_tf_clean<<<fs->NF, safr::kFrameThreads, 0, st>>>(ca);
    safr::MaskArgs ma{pl->M, G, fs->NF, fs->cbuf, fs->mask, (float)noise, k0, k1, frame0, nwrap, fs->dbuf};
    safr::k_tf_mask<<<safr::kFrameThreads * G, safr::kMaskThreads, safr::mask_smem(pl->M), st>>>(ma);
    return cudaGetLastError();
}

// Sum of loss and energy over nframes frames (chunks of kFrameThreads) drawn with
// key (k0, k1) for weights w.
bool eval_frames(safr_plan_s *pl, FilterState *fs, const float *w, uint32_t k0, uint32_t k1, uint32_t frame0,
                 uint32_t nwrap, int nframes, double noise, double &loss, double &energy, cudaStream_t st)
{
    loss = energy = 0;
    for (int c = 0; c < nframes; c += safr::kFrameThreads) {
        const uint32_t f0 = (uint32_t)((frame0 + (uint32_t)c) % nwrap);
        if (make_frames(pl, fs, k0, k1, f0, nwrap, noise, st) != cudaSuccess) return false;
        safr::FrameArgs fa{pl->M, pl->L, pl->grp[0].G, fs->NF, fs->bs, w, k0, k1, f0, nwrap, fs->dbuf, nullptr,
                           fs->loss, fs->energy};
        safr::k_filter_frames<<<fs->NF, safr::kFrameThreads, 0, st>>>(fa);
        if (cudaGetLastError() != cudaSuccess) return false;
        double a, b;
        if (!read_loss(fs, a, b, st)) return false;
        loss += a;
        energy += b;
    }
    return true;
}

}  // namespace

extern "C" safr_status safr_filter_train(safr_plan_t pl, const safr_filter_config *cfg, float *weights_out,
                                         safr_filter_result *res, cudaStream_t st)
{
    if (!pl || !cfg) return SAFR_ERR_INVALID_ARG;
    if (!(cfg->r0 > 0) || !(cfg->L0 > 0) || !std::isfinite(cfg->r0) || !std::isfinite(cfg->L0) ||
        !(cfg->noise_level >= 0) || !std::isfinite(cfg->noise_level) || cfg->train_frames < 1 ||
        cfg->valid_frames < 1 || cfg->epochs < 1 || !(cfg->lr > 0) || !std::isfinite(cfg->lr))
        return SAFR_ERR_INVALID_ARG;
    FilterDeviceGuard guard(pl->device);
    if (!guard.ok) return SAFR_ERR_CUDA;
    safr_status s = filter_prepare(pl, true, st);
    if (s != SAFR_OK) return s;
    FilterState *fs = (FilterState *)pl->filter;
    const int M = pl->M, Mh = pl->Mh, L = pl->L, G = pl->grp[0].G, NF = fs->NF, NP = fs->NP;
    const int T = safr::kFrameThreads;

    // layer spectra of the training frames and the frame energy (full spectrum)
    std::vector<float> var((size_t)NF * L);
    double Ef = 0;
    for (int k = 0; k < Mh; ++k)
        for (int j = 0; j < M; ++j)
            for (int l = 0; l < L; ++l) {
                const double v = layer_variance(pl, l, j, k, cfg->r0, cfg->L0);
                var[((size_t)k * M + j) * L + l] = (float)v;
                Ef += (k == 0 ? 1.0 : 2.0) * v;
            }
    if (!(Ef > 0)) return SAFR_ERR_INVALID_ARG;

    // initial weights: N(0, 1 / fan_in), zero biases
    std::vector<float> w0(safr::kParams, 0.0f);
    InitRng rng{cfg->seed * 0x9E3779B97F4A7C15ull + 0x632BE59BD9B4E019ull};
    auto fill = [&](int off, int n, int fan_in) {
        const double sd = 1.0 / std::sqrt((double)fan_in);
        for (int i = 0; i < n; ++i) w0[off + i] = (float)(sd * rng.normal());
    };
    fill(safr::kOffW0, safr::kH * 4, 4);
    fill(safr::kOffW1, safr::kH * safr::kH, safr::kH);
    fill(safr::kOffW2, safr::kH * safr::kH, safr::kH);
    fill(safr::kOffW3, safr::kH, safr::kH);
    std::vector<__nv_bfloat16> wb(safr::kParams);
    for (int i = 0; i < safr::kParams; ++i) wb[i] = __float2bfloat16_rn(w0[i]);
    const size_t pb = (size_t)safr::kParams * sizeof(float);
    if (cudaMemcpyAsync(fs->bs.var, var.data(), var.size() * sizeof(float), cudaMemcpyHostToDevice, st) !=
            cudaSuccess ||
        cudaMemcpyAsync(fs->master, w0.data(), pb, cudaMemcpyHostToDevice, st) != cudaSuccess ||
        cudaMemcpyAsync(fs->wb, wb.data(), wb.size() * sizeof(__nv_bfloat16), cudaMemcpyHostToDevice, st) !=
            cudaSuccess ||
        cudaMemsetAsync(fs->m, 0, pb, st) != cudaSuccess || cudaMemsetAsync(fs->v, 0, pb, st) != cudaSuccess ||
        cudaMemsetAsync(fs->flag, 0, sizeof(int), st) != cudaSuccess)
        return SAFR_ERR_CUDA;
    safr::k_filter_tikhonov<<<(NP + 255) / 256, 256, 0, st>>>(NP, L, G, fs->bs.sig, pl->grp[0].alpha, fs->wplain);
    if (cudaGetLastError() != cudaSuccess) return SAFR_ERR_CUDA;

    const uint32_t k0 = (uint32_t)cfg->seed, k1 = (uint32_t)(cfg->seed >> 32) ^ 0x5AFEu;
    const uint32_t v0 = k0 + 1u, v1 = k1;  // held-out frames: another key
    const uint32_t ntrain = (uint32_t)cfg->train_frames;
    const int probe = std::min(cfg->train_frames, 4 * T);
    double l_a, e_a;

    // training loss on the first frames before training
    if (mlp_forward(pl, fs, cfg->noise_level, fs->w, nullptr, nullptr, st) != cudaSuccess ||
        !eval_frames(pl, fs, fs->w, k0, k1, 0, ntrain, probe, cfg->noise_level, l_a, e_a, st))
        return SAFR_ERR_CUDA;
    const double first = l_a / e_a;

    const int nblk = (NP + safr::kMlpThreads - 1) / safr::kMlpThreads;
    const long steps_per_epoch = (cfg->train_frames + T - 1) / T;
    const long steps = steps_per_epoch * cfg->epochs;
    const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
    double c1 = 1, c2 = 1;
    const float scale = (float)(1.0 / ((double)T * Ef));
    for (long it = 0; it < steps; ++it) {
        const uint32_t frame0 = (uint32_t)(((uint64_t)(it % steps_per_epoch) * T) % ntrain);
        if (mlp_forward(pl, fs, cfg->noise_level, fs->w, fs->phi, fs->act, st) != cudaSuccess) return SAFR_ERR_CUDA;
        if (make_frames(pl, fs, k0, k1, frame0, ntrain, cfg->noise_level, st) != cudaSuccess) return SAFR_ERR_CUDA;
        safr::FrameArgs fa{M, L, G, NF, fs->bs, fs->w, k0, k1, frame0, ntrain, fs->dbuf, fs->gw, fs->loss, fs->energy};
        safr::k_filter_frames<<<NF, T, 0, st>>>(fa);
        safr::MlpBackArgs ba{M,  L,      G,      NP,      fs->wb, fs->bs.sig, fs->hn, (float)(cfg->noise_level / 0.05),
                             fs->act, fs->phi, fs->gw, fs->partial};
        safr::k_mlp_backward<<<nblk, safr::kMlpThreads, bwd_smem(), st>>>(ba);
        safr::k_sum_partials<<<(safr::kParams + 255) / 256, 256, 0, st>>>(fs->partial, nblk, scale, fs->grad);
        c1 *= b1;
        c2 *= b2;
        safr::k_adam<<<(safr::kParams + 255) / 256, 256, 0, st>>>(fs->master, fs->m, fs->v, fs->grad, fs->wb,
                                                                   (float)cfg->lr, b1, b2, eps, (float)(1.0 - c1),
                                                                   (float)(1.0 - c2));
        if (cudaGetLastError() != cudaSuccess) return SAFR_ERR_CUDA;
    }

    // learned weights in BF16 (what inference reads), their training loss, and the held-out comparison
    double lv_learned, ev, lv_plain, ev2;
    int flag = 0;
    if (mlp_forward(pl, fs, cfg->noise_level, fs->w, nullptr, nullptr, st) != cudaSuccess ||
        !eval_frames(pl, fs, fs->w, k0, k1, 0, ntrain, probe, cfg->noise_level, l_a, e_a, st) ||
        !eval_frames(pl, fs, fs->w, v0, v1, 0, (uint32_t)cfg->valid_frames, cfg->valid_frames, cfg->noise_level, lv_learned,
                     ev, st) ||
        !eval_frames(pl, fs, fs->wplain, v0, v1, 0, (uint32_t)cfg->valid_frames, cfg->valid_frames, cfg->noise_level,
                     lv_plain, ev2, st) ||
        cudaMemcpyAsync(&flag, fs->flag, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
        return SAFR_ERR_CUDA;
    const double last = l_a / e_a, vl = lv_learned / ev, vp = lv_plain / ev2;
    const bool use = flag == 0 && std::isfinite(vl) && std::isfinite(last) && vl < vp;
    if (use) {
        if (assemble(pl, fs, fs->w, st) != cudaSuccess) return SAFR_ERR_CUDA;
    } else if (safr::launch_precompute(pl, st) != cudaSuccess) {
        return SAFR_ERR_CUDA;
    }
    pl->filter_learned = use ? 1 : 0;
    if (weights_out) {
        std::vector<float> wm(safr::kParams);
        if (cudaMemcpyAsync(wm.data(), fs->master, pb, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
            cudaStreamSynchronize(st) != cudaSuccess)
            return SAFR_ERR_CUDA;
        for (int i = 0; i < safr::kParams; ++i) weights_out[i] = __bfloat162float(__float2bfloat16_rn(wm[i]));
    }
    if (res) {
        res->train_loss_first = first;
        res->train_loss_last = last;
        res->valid_loss_learned = vl;
        res->valid_loss_plain = vp;
        res->steps = steps;
        res->used_learned = use ? 1 : 0;
        res->nonfinite = flag;
    }
    return cudaStreamSynchronize(st) == cudaSuccess ? SAFR_OK : SAFR_ERR_CUDA;
}
