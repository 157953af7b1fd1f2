// C ABI of the SAFR library: plan creation (host geometry in FP64), the
// precompute and frame entry points, status and inspection calls.
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <complex>
#include <cstdint>
#include <cstring>
#include <new>
#include <vector>

#include "freqorder.h"
#include "plan.h"
#include "safr.h"

namespace {

const double kPi = 3.14159265358979323846264338327950288;

// Makes `dev` current for the lifetime of the guard and restores the
// caller's device afterwards.
struct DeviceGuard {
    int prev = -1;
    bool ok = false;
    explicit DeviceGuard(int dev)
    {
        if (cudaGetDevice(&prev) != cudaSuccess) return;
        if (prev != dev && cudaSetDevice(dev) != cudaSuccess) return;
        ok = true;
    }
    ~DeviceGuard()
    {
        if (ok && prev >= 0) cudaSetDevice(prev);
    }
};

size_t elem_size(int precision) { return precision == SAFR_FP64 ? 8 : (precision == SAFR_FP16_STORAGE ? 2 : 4); }

bool aligned16(const void *p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

void free_plan_memory(safr_plan_s *p)
{
    void *bufs[] = {p->d_B, p->d_w1, p->d_w2, p->d_energy, p->d_tw, p->d_rs_i0, p->d_rs_w, p->d_mask, p->d_tt_w,
                    p->d_xy_hat, p->d_pm, p->d_bar, p->d_stamps, p->d_twq,
                    p->d_pre, p->d_status, p->d_in_stage, p->d_out_stage, p->d_in_scales_stage,
                    p->d_out_scales_stage, p->d_polc, p->d_mask_bits};
    for (void *b : bufs)
        if (b) cudaFree(b);
    for (auto &e : p->ev)
        if (e) cudaEventDestroy(e);
    safr::filter_free(p);
}

// Inverse of a 3x3 matrix by cofactors; false if singular.
bool invert3(const double a[3][3], double inv[3][3])
{
    const double det = a[0][0] * (a[1][1] * a[2][2] - a[1][2] * a[2][1]) -
                       a[0][1] * (a[1][0] * a[2][2] - a[1][2] * a[2][0]) +
                       a[0][2] * (a[1][0] * a[2][1] - a[1][1] * a[2][0]);
    if (!(std::fabs(det) > 0)) return false;
    inv[0][0] = (a[1][1] * a[2][2] - a[1][2] * a[2][1]) / det;
    inv[0][1] = (a[0][2] * a[2][1] - a[0][1] * a[2][2]) / det;
    inv[0][2] = (a[0][1] * a[1][2] - a[0][2] * a[1][1]) / det;
    inv[1][0] = (a[1][2] * a[2][0] - a[1][0] * a[2][2]) / det;
    inv[1][1] = (a[0][0] * a[2][2] - a[0][2] * a[2][0]) / det;
    inv[1][2] = (a[0][2] * a[1][0] - a[0][0] * a[1][2]) / det;
    inv[2][0] = (a[1][0] * a[2][1] - a[1][1] * a[2][0]) / det;
    inv[2][1] = (a[0][1] * a[2][0] - a[0][0] * a[2][1]) / det;
    inv[2][2] = (a[0][0] * a[1][1] - a[0][1] * a[1][0]) / det;
    return true;
}

// In-place radix-2 FFT of length n (power of two), FP64, forward sign.
void host_fft(std::vector<std::complex<double>> &a)
{
    const size_t n = a.size();
    for (size_t i = 1, j = 0; i < n; ++i) {
        size_t bit = n >> 1;
        for (; j & bit; bit >>= 1) j ^= bit;
        j ^= bit;
        if (i < j) std::swap(a[i], a[j]);
    }
    for (size_t len = 2; len <= n; len <<= 1) {
        for (size_t i = 0; i < n; i += len)
            for (size_t k = 0; k < len / 2; ++k) {
                const double ang = -2.0 * kPi * (double)k / (double)len;
                const std::complex<double> w(std::cos(ang), std::sin(ang));
                const std::complex<double> u = a[i + k], v = a[i + k + len / 2] * w;
                a[i + k] = u + v;
                a[i + k + len / 2] = u - v;
            }
    }
}

// DFT2 (Section 3.2) of an M x M real image, returned for k < M/2 as [k][j].
std::vector<std::complex<double>> host_dft2_half(const std::vector<double> &img, int M)
{
    std::vector<std::complex<double>> rows((size_t)M * M), line(M);
    for (int p = 0; p < M; ++p) {
        for (int q = 0; q < M; ++q) line[q] = img[(size_t)p * M + q];
        host_fft(line);
        for (int k = 0; k < M; ++k) rows[(size_t)p * M + k] = line[k];
    }
    std::vector<std::complex<double>> out((size_t)(M / 2) * M);
    for (int k = 0; k < M / 2; ++k) {
        for (int p = 0; p < M; ++p) line[p] = rows[(size_t)p * M + k];
        host_fft(line);
        for (int j = 0; j < M; ++j) out[(size_t)k * M + j] = line[j];
    }
    return out;
}

safr_status validate(const safr_geometry *g)
{
    if (!g) return SAFR_ERR_INVALID_ARG;
    if (g->M < 8 || g->M > SAFR_MAX_M || (g->M & (g->M - 1))) return SAFR_ERR_UNSUPPORTED_SIZE;
    if (g->P < 1 || g->P > g->M) return SAFR_ERR_INVALID_ARG;
    if (g->L < 1 || g->G < 1) return SAFR_ERR_INVALID_ARG;
    if (g->L > SAFR_MAX_L || g->G > SAFR_MAX_G) return SAFR_ERR_UNSUPPORTED_SIZE;
    if (!g->h_m || !g->cn2 || !g->dir_x || !g->dir_y || !g->kind) return SAFR_ERR_INVALID_ARG;
    if (!(g->pitch_m > 0) || !std::isfinite(g->pitch_m)) return SAFR_ERR_INVALID_ARG;
    if (!(g->alpha > 0) || !std::isfinite(g->alpha)) return SAFR_ERR_INVALID_ARG;
    if (!(g->beta >= 0) || !std::isfinite(g->beta)) return SAFR_ERR_INVALID_ARG;
    if (g->precision != SAFR_FP32 && g->precision != SAFR_FP16_STORAGE && g->precision != SAFR_FP64)
        return SAFR_ERR_INVALID_ARG;
    if (g->output_grid != SAFR_NATIVE && g->output_grid != SAFR_METRIC) return SAFR_ERR_INVALID_ARG;
    int nl = 0, nn = 0;
    for (int i = 0; i < g->G; ++i) {
        if (g->kind[i] == SAFR_LGS)
            ++nl;
        else if (g->kind[i] == SAFR_NGS)
            ++nn;
        else
            return SAFR_ERR_INVALID_ARG;
        if (!std::isfinite(g->dir_x[i]) || !std::isfinite(g->dir_y[i])) return SAFR_ERR_INVALID_ARG;
    }
    if (nl > SAFR_MAX_GROUP_G || nn > SAFR_MAX_GROUP_G) return SAFR_ERR_UNSUPPORTED_SIZE;
    const bool mixed = nl > 0 && nn > 0;
    if (mixed && g->output_grid != SAFR_METRIC) return SAFR_ERR_INVALID_ARG;
    if (mixed && (!(g->alpha_tt > 0) || !std::isfinite(g->alpha_tt))) return SAFR_ERR_INVALID_ARG;
    if (nl > 0 && !(g->h_lgs_m > 0)) return SAFR_ERR_INVALID_ARG;
    for (int l = 0; l < g->L; ++l) {
        if (!(g->cn2[l] > 0) || !std::isfinite(g->cn2[l])) return SAFR_ERR_INVALID_ARG;
        if (!(g->h_m[l] >= 0) || !std::isfinite(g->h_m[l])) return SAFR_ERR_INVALID_ARG;
        if (l > 0 && !(g->h_m[l] > g->h_m[l - 1])) return SAFR_ERR_INVALID_ARG;  // ascending (Section 2)
        if (nl > 0 && !(g->h_m[l] < g->h_lgs_m)) return SAFR_ERR_INVALID_ARG;  // h_l in [0, h_LGS)
    }
    return SAFR_OK;
}

template <typename T>
cudaError_t upload(T **dst, const std::vector<T> &src)
{
    cudaError_t e = cudaMalloc((void **)dst, src.size() * sizeof(T));
    if (e != cudaSuccess) return e;
    return cudaMemcpy(*dst, src.data(), src.size() * sizeof(T), cudaMemcpyHostToDevice);
}

safr_status build_plan(const safr_geometry *g, safr_plan_s *p)
{
    p->M = g->M;
    p->P = g->P;
    p->L = g->L;
    p->G = g->G;
    p->Mh = g->M / 2;
    p->o = (g->M - g->P) / 2;
    p->precision = g->precision;
    p->output_metric = g->output_grid == SAFR_METRIC;
    p->delta = g->pitch_m;
    p->diameter = g->diameter_m;
    p->obstruction = g->obstruction;
    p->T = g->M * g->pitch_m / 2.0;
    p->beta = g->beta;
    p->h.assign(g->h_m, g->h_m + g->L);
    // the geometry as given (plan files, refresh)
    p->geo = *g;
    p->geo_cn2.assign(g->cn2, g->cn2 + g->L);
    p->geo_dir_x.assign(g->dir_x, g->dir_x + g->G);
    p->geo_dir_y.assign(g->dir_y, g->dir_y + g->G);
    p->geo_kind.assign(g->kind, g->kind + g->G);
    p->geo.h_m = p->h.data();
    p->geo.cn2 = p->geo_cn2.data();
    p->geo.dir_x = p->geo_dir_x.data();
    p->geo.dir_y = p->geo_dir_y.data();
    p->geo.kind = p->geo_kind.data();
    double sum = 0;
    for (int l = 0; l < g->L; ++l) sum += g->cn2[l];
    p->gamma.resize(g->L);
    for (int l = 0; l < g->L; ++l) p->gamma[l] = g->cn2[l] / sum;

    int nl = 0, nn = 0;
    for (int i = 0; i < g->G; ++i) (g->kind[i] == SAFR_LGS ? nl : nn) += 1;
    p->mixed = nl > 0 && nn > 0;
    p->remove_tt = p->mixed && g->remove_tt;

    // groups: LGS first (Section 3.3)
    const int kinds[2] = {SAFR_LGS, SAFR_NGS};
    int row0 = 0;
    for (int kk = 0; kk < 2; ++kk) {
        const int cnt = kinds[kk] == SAFR_LGS ? nl : nn;
        if (!cnt) continue;
        safr::Group &gr = p->grp[p->ngroups++];
        gr.kind = kinds[kk];
        gr.G = cnt;
        for (int i = 0; i < g->G; ++i)
            if (g->kind[i] == kinds[kk]) gr.stars.push_back(i);
        gr.c.resize(g->L);
        for (int l = 0; l < g->L; ++l) gr.c[l] = gr.kind == SAFR_LGS ? 1.0 - g->h_m[l] / g->h_lgs_m : 1.0;
        gr.sx.resize((size_t)cnt * g->L);
        gr.sy.resize((size_t)cnt * g->L);
        for (int t = 0; t < cnt; ++t)
            for (int l = 0; l < g->L; ++l) {
                const int s = gr.stars[t];
                gr.sx[(size_t)t * g->L + l] = g->dir_x[s] * g->h_m[l] / (gr.c[l] * g->pitch_m);
                gr.sy[(size_t)t * g->L + l] = g->dir_y[s] * g->h_m[l] / (gr.c[l] * g->pitch_m);
            }
        // alpha_TT for the tip-tilt stars of a mixed plan (Algorithm 3, line 4)
        gr.alpha = (p->mixed && gr.kind == SAFR_NGS) ? g->alpha_tt : g->alpha;
        gr.b_row0 = row0;
        row0 += g->L * cnt;
        gr.resample = gr.kind == SAFR_LGS && p->output_metric;
    }
    p->warnings |= safr::containment_warnings(p);  // Section 2 containment, per axis
    p->sumLG = row0;

    // removeTT: the tip b and tilt c of the least-squares plane a + b x + c y
    // over the pupil mask are linear in psi: (a, b, c) = N^{-1} sum_mask (1, x, y) psi,
    // N = sum_mask (1, x, y)^T (1, x, y).  The two weight images are formed here in FP64.
    p->star_tt.assign(g->G, 0);
    std::vector<unsigned char> mask((size_t)g->P * g->P, 1);
    std::vector<double> ttw(2 * (size_t)g->P * g->P, 0.0);
    if (p->remove_tt) {
        const double ro = g->diameter_m / 2.0, ri = g->obstruction * g->diameter_m / 2.0;
        double N[3][3] = {{0}};
        for (int a = 0; a < g->P; ++a)
            for (int b = 0; b < g->P; ++b) {
                const double x = (a - (g->P - 1) / 2.0) * g->pitch_m, y = (b - (g->P - 1) / 2.0) * g->pitch_m;
                const double r2 = x * x + y * y;
                const unsigned char m = g->diameter_m <= 0 ? 1 : (r2 <= ro * ro && r2 >= ri * ri);
                mask[(size_t)a * g->P + b] = m;
                if (!m) continue;
                const double f[3] = {1.0, x, y};
                for (int u = 0; u < 3; ++u)
                    for (int v = 0; v < 3; ++v) N[u][v] += f[u] * f[v];
            }
        double inv[3][3];
        if (!invert3(N, inv)) return SAFR_ERR_INVALID_ARG;
        const size_t PP = (size_t)g->P * g->P;
        for (int a = 0; a < g->P; ++a)
            for (int b = 0; b < g->P; ++b) {
                const size_t i = (size_t)a * g->P + b;
                if (!mask[i]) continue;
                const double x = (a - (g->P - 1) / 2.0) * g->pitch_m, y = (b - (g->P - 1) / 2.0) * g->pitch_m;
                ttw[i] = inv[1][0] + inv[1][1] * x + inv[1][2] * y;
                ttw[PP + i] = inv[2][0] + inv[2][1] * x + inv[2][2] * y;
            }
        for (int i = 0; i < g->G; ++i) p->star_tt[i] = g->kind[i] == SAFR_LGS;
        // the same functionals in closed form for the persistent kernel: w_b = mask (n10 + n11 x + n12 y),
        // w_c = mask (n20 + n21 x + n22 y), and the mask as one bit per pixel
        for (int v = 0; v < 3; ++v) {
            p->tt_n[v] = inv[1][v];
            p->tt_n[3 + v] = inv[2][v];
        }
        const int words = (g->P + 31) / 32;
        p->mask_bits.assign((size_t)g->P * words, 0u);
        for (int a = 0; a < g->P; ++a)
            for (int b = 0; b < g->P; ++b)
                if (mask[(size_t)a * g->P + b]) p->mask_bits[(size_t)a * words + (b >> 5)] |= 1u << (b & 31);
    }

    // ---------------- device memory ----------------
    const int M = p->M, Mh = p->Mh, L = p->L;
    const size_t cs = p->precision == SAFR_FP64 ? 16 : 8;
    const size_t rs = p->precision == SAFR_FP64 ? 8 : 4;
    cudaError_t e;
#define SAFR_TRY(x)                                                                        \
    do {                                                                                   \
        e = (x);                                                                           \
        if (e != cudaSuccess) return e == cudaErrorMemoryAllocation ? SAFR_ERR_OOM : SAFR_ERR_CUDA; \
    } while (0)

    p->b_bytes = (size_t)Mh * p->sumLG * M * cs;
    SAFR_TRY(cudaMalloc(&p->d_B, p->b_bytes));
    const size_t w1 = (size_t)p->G * p->P * Mh * cs;
    const size_t w2 = (size_t)p->ngroups * L * M * Mh * cs;
    const size_t en = (size_t)p->ngroups * L * Mh * sizeof(float);
    p->ws_bytes = w1 + w2 + en;
    SAFR_TRY(cudaMalloc(&p->d_w1, w1));
    SAFR_TRY(cudaMalloc(&p->d_w2, w2));
    SAFR_TRY(cudaMalloc((void **)&p->d_energy, en));
    SAFR_TRY(cudaMemset(p->d_energy, 0, en));

    // twiddles exp(-2 pi i t / M) from FP64
    if (p->precision == SAFR_FP64) {
        std::vector<double2> tw(M);
        for (int t = 0; t < M; ++t) tw[t] = make_double2(std::cos(2 * kPi * t / M), -std::sin(2 * kPi * t / M));
        SAFR_TRY(upload((double2 **)&p->d_tw, tw));
    } else {
        std::vector<float2> tw(M);
        for (int t = 0; t < M; ++t)
            tw[t] = make_float2((float)std::cos(2 * kPi * t / M), (float)-std::sin(2 * kPi * t / M));
        SAFR_TRY(upload((float2 **)&p->d_tw, tw));
    }

    // metric resample tables of the LGS group: u = M/2 + (p - M/2)/c_l
    std::vector<int> i0((size_t)L * M, 0);
    std::vector<double> fw((size_t)L * M, 0.0);
    for (int gi = 0; gi < p->ngroups; ++gi) {
        if (!p->grp[gi].resample) continue;
        for (int l = 0; l < L; ++l)
            for (int q = 0; q < M; ++q) {
                const double u = M / 2.0 + (q - M / 2.0) / p->grp[gi].c[l];
                const double f = std::floor(u);
                i0[(size_t)l * M + q] = (int)f;
                fw[(size_t)l * M + q] = u - f;
            }
    }
    SAFR_TRY(upload(&p->d_rs_i0, i0));
    if (p->precision == SAFR_FP64) {
        SAFR_TRY(upload((double **)&p->d_rs_w, fw));
    } else {
        std::vector<float> ff(fw.begin(), fw.end());
        SAFR_TRY(upload((float **)&p->d_rs_w, ff));
    }
    SAFR_TRY(upload(&p->d_mask, mask));
    if (!p->mask_bits.empty()) SAFR_TRY(upload(&p->d_mask_bits, p->mask_bits));
    {  // sample points of the POLC operator (loop.cu)
        std::vector<unsigned char> tab;
        safr::polc_table(p, tab);
        SAFR_TRY(upload(&p->d_polc, tab));
    }
    if (p->precision == SAFR_FP64) {
        SAFR_TRY(upload((double **)&p->d_tt_w, ttw));
    } else {
        std::vector<float> tf(ttw.begin(), ttw.end());
        SAFR_TRY(upload((float **)&p->d_tt_w, tf));
    }
    // spectra of x and y on the pupil mask, placed in the padded grid, for the
    // frequency-domain removeTT of the persistent kernel: DFT2(psi - b x - c y)
    // = DFT2(psi) - b X - c Y
    {
        std::vector<double> xm((size_t)M * M, 0.0), ym((size_t)M * M, 0.0);
        if (p->remove_tt)
            for (int a = 0; a < g->P; ++a)
                for (int bq = 0; bq < g->P; ++bq) {
                    if (!mask[(size_t)a * g->P + bq]) continue;
                    xm[(size_t)(a + p->o) * M + bq + p->o] = (a - (g->P - 1) / 2.0) * g->pitch_m;
                    ym[(size_t)(a + p->o) * M + bq + p->o] = (bq - (g->P - 1) / 2.0) * g->pitch_m;
                }
        const size_t half = (size_t)Mh * M;
        std::vector<std::complex<double>> xs, ys;
        if (p->remove_tt) {
            xs = host_dft2_half(xm, M);
            ys = host_dft2_half(ym, M);
        } else {
            xs.assign(half, 0.0);
            ys.assign(half, 0.0);
        }
        // stored with j in the persistent kernel's warp-FFT order: entry [k][pos] is frequency (j(pos), k)
        auto src = [&](size_t i) {
            const size_t k = i / M, pos = i % M;
            return k * M + (size_t)safr::wfft_j_of_pos((int)pos, M);
        };
        if (p->precision == SAFR_FP64) {
            std::vector<double2> h(2 * half);
            for (size_t i = 0; i < half; ++i) {
                h[i] = make_double2(xs[src(i)].real(), xs[src(i)].imag());
                h[half + i] = make_double2(ys[src(i)].real(), ys[src(i)].imag());
            }
            SAFR_TRY(upload((double2 **)&p->d_xy_hat, h));
        } else {
            std::vector<float2> h(2 * half);
            for (size_t i = 0; i < half; ++i) {
                h[i] = make_float2((float)xs[src(i)].real(), (float)xs[src(i)].imag());
                h[half + i] = make_float2((float)ys[src(i)].real(), (float)ys[src(i)].imag());
            }
            SAFR_TRY(upload((float2 **)&p->d_xy_hat, h));
        }
    }
    {   // warp-FFT twiddles of the persistent kernel, from FP64
        std::vector<double> tr, ti;
        safr::frame2_twiddles(M, tr, ti);
        const size_t nt = tr.size();
        if (p->precision == SAFR_FP64) {
            std::vector<double2> h(nt);
            for (size_t i = 0; i < nt; ++i) h[i] = make_double2(tr[i], ti[i]);
            SAFR_TRY(upload((double2 **)&p->d_twq, h));
        } else {
            std::vector<float2> h(nt);
            for (size_t i = 0; i < nt; ++i) h[i] = make_float2((float)tr[i], (float)ti[i]);
            SAFR_TRY(upload((float2 **)&p->d_twq, h));
        }
    }
    SAFR_TRY(cudaMalloc(&p->d_pm, (size_t)p->G * p->P * 2 * rs));
    SAFR_TRY(cudaMemset(p->d_pm, 0, (size_t)p->G * p->P * 2 * rs));
    SAFR_TRY(cudaMalloc((void **)&p->d_bar, 2 * sizeof(unsigned long long)));
    SAFR_TRY(cudaMemset(p->d_bar, 0, 2 * sizeof(unsigned long long)));

    // precompute inputs: per group sx, sy [G][L], sw [L], tau [L]
    SAFR_TRY(upload(&p->d_pre, safr::pre_inputs(p)));

    SAFR_TRY(cudaMalloc((void **)&p->d_status, sizeof(int)));
    SAFR_TRY(cudaMemset(p->d_status, 0, sizeof(int)));

    // staging for safr_reconstruct_host
    const size_t es = elem_size(p->precision);
    p->in_bytes = (size_t)p->G * p->P * p->P * es;
    p->out_bytes = (size_t)L * M * M * es;
    SAFR_TRY(cudaMalloc(&p->d_in_stage, p->in_bytes));
    SAFR_TRY(cudaMalloc(&p->d_out_stage, p->out_bytes));
    SAFR_TRY(cudaMalloc((void **)&p->d_in_scales_stage, (size_t)p->G * sizeof(float)));
    SAFR_TRY(cudaMalloc((void **)&p->d_out_scales_stage, (size_t)L * sizeof(float)));

    const safr_status ks = safr::configure_frame_kernels(p);
    if (ks != SAFR_OK) return ks;
    p->fused_ok = safr::configure_fused(p) ? 1 : 0;
    cudaGetLastError();
    p->cl_ok = safr::configure_cluster(p) ? 1 : 0;
    cudaGetLastError();
#undef SAFR_TRY
    return SAFR_OK;
}

cudaError_t dispatch(safr_plan_s *p, const void *in, const float *in_scales, void *out, float *out_scales,
                     cudaStream_t st)
{
    if (safr::use_cluster(p)) return safr::launch_cluster(p, in, in_scales, out, out_scales, st);
    if (safr::use_fused(p)) return safr::launch_fused(p, in, in_scales, out, out_scales, st);
    return safr::launch_frame(p, in, in_scales, out, out_scales, st);
}

}  // namespace

extern "C" {

safr_status safr_plan_create(const safr_geometry *geom, int cuda_device, safr_plan_t *out)
{
    if (!out) return SAFR_ERR_INVALID_ARG;
    *out = nullptr;
    safr_status s = validate(geom);
    if (s != SAFR_OK) return s;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || cuda_device < 0 || cuda_device >= ndev) {
        cudaGetLastError();
        return SAFR_ERR_CUDA;
    }
    DeviceGuard guard(cuda_device);
    if (!guard.ok) return SAFR_ERR_CUDA;
    safr_plan_s *p = new (std::nothrow) safr_plan_s();
    if (!p) return SAFR_ERR_OOM;
    p->device = cuda_device;
    s = build_plan(geom, p);
    if (s != SAFR_OK) {
        free_plan_memory(p);
        delete p;
        cudaGetLastError();
        return s;
    }
    *out = p;
    return SAFR_OK;
}

safr_status safr_precompute(safr_plan_t plan, cudaStream_t stream)
{
    if (!plan) return SAFR_ERR_INVALID_ARG;
    DeviceGuard guard(plan->device);
    if (!guard.ok) return SAFR_ERR_CUDA;
    if (safr::launch_precompute(plan, stream) != cudaSuccess) return SAFR_ERR_CUDA;
    plan->precomputed = 1;
    return SAFR_OK;
}

safr_status safr_reconstruct(safr_plan_t plan, const void *d_wavefronts, const float *d_in_scales, void *d_layers,
                             float *d_out_scales, cudaStream_t stream)
{
    if (!plan || !d_wavefronts || !d_layers) return SAFR_ERR_INVALID_ARG;
    if (!plan->precomputed) return SAFR_ERR_NOT_PRECOMPUTED;
    if (plan->precision == SAFR_FP16_STORAGE && !d_out_scales) return SAFR_ERR_INVALID_ARG;
    if (plan->precision != SAFR_FP16_STORAGE && (d_in_scales || d_out_scales)) return SAFR_ERR_INVALID_ARG;
    if (!aligned16(d_wavefronts) || !aligned16(d_layers) || (d_in_scales && !aligned16(d_in_scales)) ||
        (d_out_scales && !aligned16(d_out_scales)))
        return SAFR_ERR_MISALIGNED;
    DeviceGuard guard(plan->device);
    if (!guard.ok) return SAFR_ERR_CUDA;
    if (dispatch(plan, d_wavefronts, d_in_scales, d_layers, d_out_scales, stream) != cudaSuccess) return SAFR_ERR_CUDA;
    return SAFR_OK;
}

safr_status safr_reconstruct_frames(safr_plan_t plan, int n, const void *d_wavefronts, const float *d_in_scales,
                                    void *d_layers, float *d_out_scales, cudaStream_t stream)
{
    if (!plan || n < 1 || !d_wavefronts || !d_layers) return SAFR_ERR_INVALID_ARG;
    if (!plan->precomputed) return SAFR_ERR_NOT_PRECOMPUTED;
    if (plan->precision == SAFR_FP16_STORAGE && !d_out_scales) return SAFR_ERR_INVALID_ARG;
    if (plan->precision != SAFR_FP16_STORAGE && (d_in_scales || d_out_scales)) return SAFR_ERR_INVALID_ARG;
    if (!aligned16(d_wavefronts) || !aligned16(d_layers) || (d_in_scales && !aligned16(d_in_scales)) ||
        (d_out_scales && !aligned16(d_out_scales)))
        return SAFR_ERR_MISALIGNED;
    const bool one_launch = safr::use_fused(plan) && plan->f2_frames_ok;
    // frame by frame (other schedules): every frame's buffers must be aligned as safr_reconstruct's
    if (!one_launch && n > 1 &&
        (plan->in_bytes % 16 || plan->out_bytes % 16 || (d_in_scales && (plan->G * sizeof(float)) % 16) ||
         (d_out_scales && (plan->L * sizeof(float)) % 16)))
        return SAFR_ERR_MISALIGNED;
    DeviceGuard guard(plan->device);
    if (!guard.ok) return SAFR_ERR_CUDA;
    if (one_launch) {
        if (safr::launch_fused_frames(plan, d_wavefronts, d_in_scales, d_layers, d_out_scales, n, stream) !=
            cudaSuccess)
            return SAFR_ERR_CUDA;
        return SAFR_OK;
    }
    for (int f = 0; f < n; ++f) {
        const void *in = (const unsigned char *)d_wavefronts + (size_t)f * plan->in_bytes;
        void *out = (unsigned char *)d_layers + (size_t)f * plan->out_bytes;
        const float *isc = d_in_scales ? d_in_scales + (size_t)f * plan->G : nullptr;
        float *osc = d_out_scales ? d_out_scales + (size_t)f * plan->L : nullptr;
        if (dispatch(plan, in, isc, out, osc, stream) != cudaSuccess) return SAFR_ERR_CUDA;
    }
    return SAFR_OK;
}

// The device address of a page-locked, mapped host buffer (16-byte aligned), else null: the GPU
// then reads and writes it directly over the host link (NVLink-C2C on Grace) without staging copies.
const void *host_alias(const void *h)
{
    if (!h) return nullptr;
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, h) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    if (a.type != cudaMemoryTypeHost || !a.devicePointer || !aligned16(a.devicePointer)) return nullptr;
    return a.devicePointer;
}

safr_status safr_reconstruct_host(safr_plan_t plan, const void *h_wavefronts, const float *h_in_scales,
                                  void *h_layers, float *h_out_scales, cudaStream_t stream)
{
    if (!plan || !h_wavefronts || !h_layers) return SAFR_ERR_INVALID_ARG;
    if (!plan->precomputed) return SAFR_ERR_NOT_PRECOMPUTED;
    const bool fp16 = plan->precision == SAFR_FP16_STORAGE;
    if (fp16 && !h_out_scales) return SAFR_ERR_INVALID_ARG;
    if (!fp16 && (h_in_scales || h_out_scales)) return SAFR_ERR_INVALID_ARG;
    DeviceGuard guard(plan->device);
    if (!guard.ok) return SAFR_ERR_CUDA;
    const size_t nsc_in = (size_t)plan->G * sizeof(float), nsc_out = (size_t)plan->L * sizeof(float);
    {  // page-locked buffers: the kernels read and write them in place
        const void *din = host_alias(h_wavefronts), *dout = host_alias(h_layers);
        const void *dsi = host_alias(h_in_scales), *dso = host_alias(h_out_scales);
        if (din && dout && (!h_in_scales || dsi) && (!h_out_scales || dso)) {
            if (dispatch(plan, din, (const float *)dsi, (void *)dout, (float *)dso, stream) != cudaSuccess ||
                cudaStreamSynchronize(stream) != cudaSuccess)
                return SAFR_ERR_CUDA;
            return SAFR_OK;
        }
    }
    if (cudaMemcpyAsync(plan->d_in_stage, h_wavefronts, plan->in_bytes, cudaMemcpyHostToDevice, stream) != cudaSuccess)
        return SAFR_ERR_CUDA;
    if (h_in_scales && cudaMemcpyAsync(plan->d_in_scales_stage, h_in_scales, nsc_in, cudaMemcpyHostToDevice,
                                       stream) != cudaSuccess)
        return SAFR_ERR_CUDA;
    if (dispatch(plan, plan->d_in_stage, h_in_scales ? plan->d_in_scales_stage : nullptr, plan->d_out_stage,
                 fp16 ? plan->d_out_scales_stage : nullptr, stream) != cudaSuccess)
        return SAFR_ERR_CUDA;
    if (cudaMemcpyAsync(h_layers, plan->d_out_stage, plan->out_bytes, cudaMemcpyDeviceToHost, stream) != cudaSuccess)
        return SAFR_ERR_CUDA;
    if (fp16 && cudaMemcpyAsync(h_out_scales, plan->d_out_scales_stage, nsc_out, cudaMemcpyDeviceToHost, stream) !=
                    cudaSuccess)
        return SAFR_ERR_CUDA;
    if (cudaStreamSynchronize(stream) != cudaSuccess) return SAFR_ERR_CUDA;
    return SAFR_OK;
}

safr_status safr_get_status(safr_plan_t plan)
{
    if (!plan) return SAFR_ERR_INVALID_ARG;
    DeviceGuard guard(plan->device);
    if (!guard.ok) return SAFR_ERR_CUDA;
    if (cudaDeviceSynchronize() != cudaSuccess) return SAFR_ERR_CUDA;
    int st = 0;
    if (cudaMemcpy(&st, plan->d_status, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) return SAFR_ERR_CUDA;
    if (st != 0) {
        // clear the sticky word and re-arm the grid barrier that a timeout left half-counted
        if (cudaMemset(plan->d_status, 0, sizeof(int)) != cudaSuccess) return SAFR_ERR_CUDA;
        if (cudaMemset(plan->d_bar, 0, 2 * sizeof(unsigned long long)) != cudaSuccess) return SAFR_ERR_CUDA;
        if (cudaDeviceSynchronize() != cudaSuccess) return SAFR_ERR_CUDA;
    }
    return (safr_status)st;
}

safr_status safr_get_plan_info(safr_plan_t plan, safr_plan_info *info)
{
    if (!plan || !info) return SAFR_ERR_INVALID_ARG;
    std::memset(info, 0, sizeof(*info));
    info->M = plan->M;
    info->P = plan->P;
    info->L = plan->L;
    info->G = plan->G;
    info->ngroups = plan->ngroups;
    for (int gi = 0; gi < plan->ngroups; ++gi) {
        info->group_kind[gi] = plan->grp[gi].kind;
        info->group_G[gi] = plan->grp[gi].G;
    }
    info->b_bytes = plan->b_bytes;
    info->workspace_bytes = plan->ws_bytes;
    info->in_bytes = plan->in_bytes;
    info->out_bytes = plan->out_bytes;
    info->warnings = plan->warnings;
    info->precomputed = plan->precomputed;
    info->path = safr::path_in_use(plan);
    info->tile_rows = plan->f2_rt3;
    info->autotuned = plan->autotuned;
    return SAFR_OK;
}

safr_status safr_copy_B(safr_plan_t plan, int group, double *dst)
{
    if (!plan || !dst || group < 0 || group >= plan->ngroups) return SAFR_ERR_INVALID_ARG;
    if (!plan->precomputed) return SAFR_ERR_NOT_PRECOMPUTED;
    DeviceGuard guard(plan->device);
    if (!guard.ok) return SAFR_ERR_CUDA;
    if (cudaDeviceSynchronize() != cudaSuccess) return SAFR_ERR_CUDA;
    const int M = plan->M, Mh = plan->Mh;
    const size_t rows = (size_t)plan->L * plan->grp[group].G;
    const bool f64 = plan->precision == SAFR_FP64;
    const size_t cs = f64 ? 16 : 8;
    std::vector<unsigned char> buf(rows * M * cs);
    for (int k = 0; k < Mh; ++k) {
        const size_t off = ((size_t)k * plan->sumLG + plan->grp[group].b_row0) * M * cs;
        if (cudaMemcpy(buf.data(), (const unsigned char *)plan->d_B + off, buf.size(), cudaMemcpyDeviceToHost) !=
            cudaSuccess)
            return SAFR_ERR_CUDA;
        double *d = dst + (size_t)k * rows * M * 2;
        for (size_t i = 0; i < rows * M; ++i) {
            // device storage is in the warp-FFT order along j; hand it back in natural order
            const size_t row = i / M, pos = i % M;
            const size_t o = row * M + (size_t)safr::wfft_j_of_pos((int)pos, M);
            if (f64) {
                const double2 v = ((const double2 *)buf.data())[i];
                d[2 * o] = v.x;
                d[2 * o + 1] = v.y;
            } else {
                const float2 v = ((const float2 *)buf.data())[i];
                d[2 * o] = v.x;
                d[2 * o + 1] = v.y;
            }
        }
    }
    return SAFR_OK;
}

safr_status safr_trace(safr_plan_t plan, int enable)
{
    if (!plan) return SAFR_ERR_INVALID_ARG;
    DeviceGuard guard(plan->device);
    if (!guard.ok) return SAFR_ERR_CUDA;
    if (enable && !plan->ev[0])
        for (auto &e : plan->ev)
            if (cudaEventCreate(&e) != cudaSuccess) return SAFR_ERR_CUDA;
    if (enable && !plan->d_stamps && plan->f2_grid > 0) {  // sized for one CTA per SM, the largest grid
        int nsm = plan->f2_grid;
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, plan->device);
        const size_t nst = (size_t)std::max(nsm, plan->f2_grid) * SAFR_TRACE_MARKS * sizeof(unsigned long long);
        if (cudaMalloc((void **)&plan->d_stamps, nst) != cudaSuccess) return SAFR_ERR_OOM;
        if (cudaMemset(plan->d_stamps, 0, nst) != cudaSuccess) return SAFR_ERR_CUDA;
    }
    plan->trace = enable ? 1 : 0;
    plan->traced = 0;
    return SAFR_OK;
}

safr_status safr_trace_read(safr_plan_t plan, float *ms, int n, int *n_out)
{
    if (!plan || (!ms && n > 0)) return SAFR_ERR_INVALID_ARG;
    if (n_out) *n_out = 0;
    if (!plan->traced) return SAFR_ERR_INVALID_ARG;
    DeviceGuard guard(plan->device);
    if (!guard.ok) return SAFR_ERR_CUDA;
    const int nph = safr::launches_per_frame(plan);
    if (cudaEventSynchronize(plan->ev[nph]) != cudaSuccess) return SAFR_ERR_CUDA;
    for (int i = 0; i < nph && i < n; ++i)
        if (cudaEventElapsedTime(&ms[i], plan->ev[i], plan->ev[i + 1]) != cudaSuccess) return SAFR_ERR_CUDA;
    if (n_out) *n_out = nph;
    return SAFR_OK;
}

int safr_launches_per_frame(safr_plan_t plan) { return plan ? safr::launches_per_frame(plan) : 0; }

safr_status safr_trace_phases(safr_plan_t plan, double *us, int n, int *n_out)
{
    if (!plan || (!us && n > 0)) return SAFR_ERR_INVALID_ARG;
    if (n_out) *n_out = 0;
    if (!plan->traced || !(safr::use_fused(plan) || safr::use_cluster(plan)) || !plan->d_stamps)
        return SAFR_ERR_INVALID_ARG;
    DeviceGuard guard(plan->device);
    if (!guard.ok) return SAFR_ERR_CUDA;
    if (cudaEventSynchronize(plan->ev[1]) != cudaSuccess) return SAFR_ERR_CUDA;
    const int K = SAFR_TRACE_MARKS;
    const int grid = safr::use_cluster(plan) ? plan->cl_cs : plan->f2_grid;
    std::vector<unsigned long long> st((size_t)grid * K);
    if (cudaMemcpy(st.data(), plan->d_stamps, st.size() * sizeof(unsigned long long), cudaMemcpyDeviceToHost) !=
        cudaSuccess)
        return SAFR_ERR_CUDA;
    // mark i: latest CTA to reach it, in microseconds from the earliest CTA start
    // (marks a CTA never reaches, e.g. a CTA with no phase-2 column, stay 0)
    unsigned long long t0 = ~0ull;
    for (int b = 0; b < grid; ++b) t0 = std::min(t0, st[(size_t)b * K]);
    double v[SAFR_TRACE_MARKS];
    for (int i = 0; i < K; ++i) {
        unsigned long long last = 0;
        for (int b = 0; b < grid; ++b) last = std::max(last, st[(size_t)b * K + i]);
        v[i] = last > t0 ? 1e-3 * (double)(last - t0) : 0.0;
    }
    for (int i = 0; i < K && i < n; ++i) us[i] = v[i];
    if (n_out) *n_out = K;
    return SAFR_OK;
}

safr_status safr_trace_stamps(safr_plan_t plan, double *us, int n, int *n_cta)
{
    if (!plan || (!us && n > 0)) return SAFR_ERR_INVALID_ARG;
    if (n_cta) *n_cta = 0;
    if (!plan->traced || !(safr::use_fused(plan) || safr::use_cluster(plan)) || !plan->d_stamps)
        return SAFR_ERR_INVALID_ARG;
    DeviceGuard guard(plan->device);
    if (!guard.ok) return SAFR_ERR_CUDA;
    if (cudaEventSynchronize(plan->ev[1]) != cudaSuccess) return SAFR_ERR_CUDA;
    const int K = SAFR_TRACE_MARKS;
    const int grid = safr::use_cluster(plan) ? plan->cl_cs : plan->f2_grid;
    std::vector<unsigned long long> st((size_t)grid * K);
    if (cudaMemcpy(st.data(), plan->d_stamps, st.size() * sizeof(unsigned long long), cudaMemcpyDeviceToHost) !=
        cudaSuccess)
        return SAFR_ERR_CUDA;
    unsigned long long t0 = ~0ull;
    for (int b = 0; b < grid; ++b) t0 = std::min(t0, st[(size_t)b * K]);
    for (size_t i = 0; i < st.size() && (long)i < n; ++i) us[i] = st[i] > t0 ? 1e-3 * (double)(st[i] - t0) : 0.0;
    if (n_cta) *n_cta = grid;
    return SAFR_OK;
}

safr_status safr_set_path(safr_plan_t plan, int path)
{
    if (!plan || path < SAFR_PATH_AUTO || path > SAFR_PATH_CLUSTER) return SAFR_ERR_INVALID_ARG;
    if (path == SAFR_PATH_FUSED && !plan->fused_ok) return SAFR_ERR_UNSUPPORTED_SIZE;
    if (path == SAFR_PATH_CLUSTER && !plan->cl_ok) return SAFR_ERR_UNSUPPORTED_SIZE;
    plan->path = path;
    plan->traced = 0;
    return SAFR_OK;
}

safr_status safr_set_grid(safr_plan_t plan, int ctas)
{
    if (!plan || ctas < 0) return SAFR_ERR_INVALID_ARG;
    if (!plan->fused_ok) return SAFR_ERR_UNSUPPORTED_SIZE;
    DeviceGuard guard(plan->device);
    if (!guard.ok) return SAFR_ERR_CUDA;
    const int old = plan->f2_grid_force;
    plan->f2_grid_force = ctas;
    if (!safr::configure_fused(plan)) {  // the shape cannot run on that grid: keep the previous one
        plan->f2_grid_force = old;
        safr::configure_fused(plan);
        return SAFR_ERR_UNSUPPORTED_SIZE;
    }
    plan->traced = 0;
    return SAFR_OK;
}

int safr_get_grid(safr_plan_t plan) { return plan ? plan->f2_grid : 0; }

safr_status safr_set_tile_rows(safr_plan_t plan, int rows)
{
    if (!plan || rows < 0 || (rows & 1) || rows > std::min(32, plan->M)) return SAFR_ERR_INVALID_ARG;
    if (!plan->fused_ok) return SAFR_ERR_UNSUPPORTED_SIZE;
    DeviceGuard guard(plan->device);
    if (!guard.ok) return SAFR_ERR_CUDA;
    const int old = plan->f2_rt_force;
    plan->f2_rt_force = rows;
    if (!safr::configure_fused(plan)) {  // the tile does not fit: keep the previous choice
        plan->f2_rt_force = old;
        safr::configure_fused(plan);
        return SAFR_ERR_UNSUPPORTED_SIZE;
    }
    plan->traced = 0;
    return SAFR_OK;
}

int safr_get_path(safr_plan_t plan)
{
    if (!plan) return -1;
    return safr::path_in_use(plan);
}

safr_status safr_debug_skip_barrier(safr_plan_t plan, int cta, double timeout_s)
{
    if (!plan || cta < -1) return SAFR_ERR_INVALID_ARG;
    plan->debug_skip_cta = cta;
    plan->barrier_timeout_ns = timeout_s > 0 ? (unsigned long long)(timeout_s * 1e9) : 1000000000ull;
    return SAFR_OK;
}

safr_status safr_destroy(safr_plan_t plan)
{
    if (!plan) return SAFR_ERR_INVALID_ARG;
    {
        DeviceGuard guard(plan->device);
        cudaDeviceSynchronize();
        free_plan_memory(plan);
    }
    delete plan;
    return SAFR_OK;
}

const char *safr_status_string(safr_status s)
{
    switch (s) {
    case SAFR_OK: return "SAFR_OK";
    case SAFR_ERR_INVALID_ARG: return "SAFR_ERR_INVALID_ARG: invalid argument or geometry";
    case SAFR_ERR_UNSUPPORTED_SIZE: return "SAFR_ERR_UNSUPPORTED_SIZE: grid, layer or star count outside the supported range";
    case SAFR_ERR_MISALIGNED: return "SAFR_ERR_MISALIGNED: device pointer not 16-byte aligned";
    case SAFR_ERR_NOT_PRECOMPUTED: return "SAFR_ERR_NOT_PRECOMPUTED: call safr_precompute first";
    case SAFR_ERR_OOM: return "SAFR_ERR_OOM: device allocation failed";
    case SAFR_ERR_CUDA: return "SAFR_ERR_CUDA: CUDA runtime error";
    case SAFR_ERR_TIMEOUT: return "SAFR_ERR_TIMEOUT: a bounded device-side wait gave up";
    case SAFR_ERR_DEVICE: return "SAFR_ERR_DEVICE: a device-side check failed";
    case SAFR_ERR_IO: return "SAFR_ERR_IO: plan file not written or read, or not a valid plan file";
    }
    return "unknown safr_status";
}

}  // extern "C"
