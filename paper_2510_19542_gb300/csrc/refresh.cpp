// Soft real-time work on an existing plan (Algorithm 2 and Section 3.4: B is
// recomputed whenever parameters at the telescope or in the atmosphere
// change) and plan files.
//
// safr_refresh takes new Cn2 weights, star directions and regularisation
// parameters, rewrites the derived tables in the plan's existing buffers and
// reruns the precompute kernel in place, allocating nothing.  safr_plan_save
// and safr_plan_load write and read a plan's geometry and B.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <vector>

#include "plan.h"
#include "safr.h"

namespace safr {

// Inputs of the precompute kernel, per group: sx [G][L], sy [G][L], sw [L] = gamma_l^{1/2} / c_l,
// tau [L] = pi^2 / (c_l T)^2.
std::vector<double> pre_inputs(const safr_plan_s *p)
{
    const double pi = 3.14159265358979323846;
    std::vector<double> pre;
    for (int gi = 0; gi < p->ngroups; ++gi) {
        const Group &gr = p->grp[gi];
        pre.insert(pre.end(), gr.sx.begin(), gr.sx.end());
        pre.insert(pre.end(), gr.sy.begin(), gr.sy.end());
        for (int l = 0; l < p->L; ++l) pre.push_back(std::sqrt(p->gamma[l]) / gr.c[l]);
        for (int l = 0; l < p->L; ++l) pre.push_back(pi * pi / ((gr.c[l] * p->T) * (gr.c[l] * p->T)));
    }
    return pre;
}

// SAFR_WARN_CONTAINMENT if some c_l Omega_A + alpha_g h_l leaves c_l Omega_T (Section 2), per axis.
int containment_warnings(const safr_plan_s *p)
{
    const double ra = 0.5 * p->P * p->delta;
    for (int gi = 0; gi < p->ngroups; ++gi) {
        const Group &gr = p->grp[gi];
        for (int t = 0; t < gr.G; ++t)
            for (int l = 0; l < p->L; ++l) {
                const int s = gr.stars[t];
                const double c = gr.c[l];
                if (c * ra + std::fabs(p->geo_dir_x[s] * p->h[l]) > c * p->T ||
                    c * ra + std::fabs(p->geo_dir_y[s] * p->h[l]) > c * p->T)
                    return SAFR_WARN_CONTAINMENT;
            }
    }
    return 0;
}

}  // namespace safr

namespace {

struct RefreshDeviceGuard {
    int prev = -1;
    bool ok = false;
    explicit RefreshDeviceGuard(int dev)
    {
        if (cudaGetDevice(&prev) != cudaSuccess) return;
        if (prev != dev && cudaSetDevice(dev) != cudaSuccess) return;
        ok = true;
    }
    ~RefreshDeviceGuard()
    {
        if (ok && prev >= 0) cudaSetDevice(prev);
    }
};

// FNV-1a, 64 bits
uint64_t fnv1a(const unsigned char *p, size_t n, uint64_t h = 0xcbf29ce484222325ull)
{
    for (size_t i = 0; i < n; ++i) {
        h ^= p[i];
        h *= 0x100000001b3ull;
    }
    return h;
}

const char kMagic[8] = {'S', 'A', 'F', 'R', 'P', 'L', 'N', '1'};
constexpr uint32_t kVersion = 1;

template <typename T>
void put(std::vector<unsigned char> &b, const T &v)
{
    const unsigned char *p = (const unsigned char *)&v;
    b.insert(b.end(), p, p + sizeof(T));
}

template <typename T>
void put_n(std::vector<unsigned char> &b, const T *v, size_t n)
{
    const unsigned char *p = (const unsigned char *)v;
    b.insert(b.end(), p, p + n * sizeof(T));
}

struct Reader {
    const std::vector<unsigned char> &b;
    size_t pos = 0;
    bool ok = true;
    template <typename T>
    T get()
    {
        T v{};
        if (pos + sizeof(T) > b.size()) {
            ok = false;
            return v;
        }
        std::memcpy(&v, b.data() + pos, sizeof(T));
        pos += sizeof(T);
        return v;
    }
    template <typename T>
    void get_n(std::vector<T> &v, size_t n)
    {
        if (n > (b.size() - pos) / sizeof(T)) {
            ok = false;
            return;
        }
        v.resize(n);
        std::memcpy(v.data(), b.data() + pos, n * sizeof(T));
        pos += n * sizeof(T);
    }
};

}  // namespace

extern "C" {

safr_status safr_refresh(safr_plan_t pl, const safr_update *u, cudaStream_t stream)
{
    if (!pl || !u) return SAFR_ERR_INVALID_ARG;
    if ((u->dir_x == nullptr) != (u->dir_y == nullptr)) return SAFR_ERR_INVALID_ARG;
    const int L = pl->L, G = pl->G;
    if (u->cn2)
        for (int l = 0; l < L; ++l)
            if (!(u->cn2[l] > 0) || !std::isfinite(u->cn2[l])) return SAFR_ERR_INVALID_ARG;
    if (u->dir_x)
        for (int g = 0; g < G; ++g)
            if (!std::isfinite(u->dir_x[g]) || !std::isfinite(u->dir_y[g])) return SAFR_ERR_INVALID_ARG;
    if (!std::isfinite(u->alpha) || !std::isfinite(u->alpha_tt)) return SAFR_ERR_INVALID_ARG;
    RefreshDeviceGuard guard(pl->device);
    if (!guard.ok) return SAFR_ERR_CUDA;

    // the new parameters
    if (u->cn2) {
        pl->geo_cn2.assign(u->cn2, u->cn2 + L);
        double sum = 0;
        for (int l = 0; l < L; ++l) sum += u->cn2[l];
        for (int l = 0; l < L; ++l) pl->gamma[l] = u->cn2[l] / sum;
    }
    if (u->alpha > 0) pl->geo.alpha = u->alpha;
    if (u->alpha_tt > 0) pl->geo.alpha_tt = u->alpha_tt;
    if (u->dir_x) {
        pl->geo_dir_x.assign(u->dir_x, u->dir_x + G);
        pl->geo_dir_y.assign(u->dir_y, u->dir_y + G);
    }
    for (int gi = 0; gi < pl->ngroups; ++gi) {
        safr::Group &gr = pl->grp[gi];
        for (int t = 0; t < gr.G; ++t)
            for (int l = 0; l < L; ++l) {
                const int s = gr.stars[t];
                gr.sx[(size_t)t * L + l] = pl->geo_dir_x[s] * pl->h[l] / (gr.c[l] * pl->delta);
                gr.sy[(size_t)t * L + l] = pl->geo_dir_y[s] * pl->h[l] / (gr.c[l] * pl->delta);
            }
        gr.alpha = (pl->mixed && gr.kind == SAFR_NGS) ? pl->geo.alpha_tt : pl->geo.alpha;
    }
    pl->warnings = (pl->warnings & ~SAFR_WARN_CONTAINMENT) | safr::containment_warnings(pl);

    // tables into the existing buffers, then Algorithm 2 in place
    const std::vector<double> pre = safr::pre_inputs(pl);
    std::vector<unsigned char> tab;
    safr::polc_table(pl, tab);
    if (cudaMemcpyAsync(pl->d_pre, pre.data(), pre.size() * sizeof(double), cudaMemcpyHostToDevice, stream) !=
            cudaSuccess ||
        cudaMemcpyAsync(pl->d_polc, tab.data(), tab.size(), cudaMemcpyHostToDevice, stream) != cudaSuccess)
        return SAFR_ERR_CUDA;
    safr::filter_invalidate(pl);
    if (safr::launch_precompute(pl, stream) != cudaSuccess) return SAFR_ERR_CUDA;
    pl->precomputed = 1;
    return SAFR_OK;
}

safr_status safr_plan_save(safr_plan_t pl, const char *path)
{
    if (!pl || !path) return SAFR_ERR_INVALID_ARG;
    if (!pl->precomputed) return SAFR_ERR_NOT_PRECOMPUTED;
    RefreshDeviceGuard guard(pl->device);
    if (!guard.ok) return SAFR_ERR_CUDA;
    const safr_geometry &g = pl->geo;
    std::vector<unsigned char> b;
    put_n(b, kMagic, 8);
    put(b, kVersion);
    const int32_t ints[8] = {g.M, g.P, g.L, g.G, g.precision, g.output_grid, g.remove_tt, pl->filter_learned};
    put_n(b, ints, 8);
    const double dbl[7] = {g.pitch_m, g.diameter_m, g.obstruction, g.h_lgs_m, g.alpha, g.alpha_tt, g.beta};
    put_n(b, dbl, 7);
    put_n(b, pl->h.data(), g.L);
    put_n(b, pl->geo_cn2.data(), g.L);
    put_n(b, pl->geo_dir_x.data(), g.G);
    put_n(b, pl->geo_dir_y.data(), g.G);
    std::vector<int32_t> kind(pl->geo_kind.begin(), pl->geo_kind.end());
    put_n(b, kind.data(), g.G);
    put(b, fnv1a(b.data(), b.size()));
    const size_t nb = pl->b_bytes;
    put(b, (uint64_t)nb);
    const size_t at = b.size();
    b.resize(at + nb);
    if (cudaDeviceSynchronize() != cudaSuccess || cudaMemcpy(b.data() + at, pl->d_B, nb, cudaMemcpyDeviceToHost) !=
                                                      cudaSuccess)
        return SAFR_ERR_CUDA;
    put(b, fnv1a(b.data() + at, nb));
    FILE *f = std::fopen(path, "wb");
    if (!f) return SAFR_ERR_IO;
    const bool ok = std::fwrite(b.data(), 1, b.size(), f) == b.size();
    return (std::fclose(f) == 0 && ok) ? SAFR_OK : SAFR_ERR_IO;
}

safr_status safr_plan_load(const char *path, int cuda_device, safr_plan_t *out)
{
    if (!path || !out) return SAFR_ERR_INVALID_ARG;
    *out = nullptr;
    FILE *f = std::fopen(path, "rb");
    if (!f) return SAFR_ERR_IO;
    std::vector<unsigned char> b;
    unsigned char chunk[1 << 16];
    size_t n;
    while ((n = std::fread(chunk, 1, sizeof(chunk), f)) > 0) b.insert(b.end(), chunk, chunk + n);
    const bool read_err = std::ferror(f) != 0;
    std::fclose(f);
    if (read_err) return SAFR_ERR_IO;

    Reader r{b};
    std::vector<char> magic;
    r.get_n(magic, 8);
    if (!r.ok || std::memcmp(magic.data(), kMagic, 8) != 0 || r.get<uint32_t>() != kVersion) return SAFR_ERR_IO;
    std::vector<int32_t> ints;
    std::vector<double> dbl;
    r.get_n(ints, 8);
    r.get_n(dbl, 7);
    if (!r.ok) return SAFR_ERR_IO;
    const int L = ints[2], G = ints[3];
    if (L < 1 || L > SAFR_MAX_L || G < 1 || G > SAFR_MAX_G) return SAFR_ERR_IO;
    std::vector<double> h, cn2, dx, dy;
    std::vector<int32_t> kind;
    r.get_n(h, L);
    r.get_n(cn2, L);
    r.get_n(dx, G);
    r.get_n(dy, G);
    r.get_n(kind, G);
    if (!r.ok) return SAFR_ERR_IO;
    const size_t geo_end = r.pos;
    const uint64_t ghash = r.get<uint64_t>();
    const uint64_t nb = r.get<uint64_t>();
    if (!r.ok || ghash != fnv1a(b.data(), geo_end) || nb > b.size() - r.pos || b.size() - r.pos - nb != 8)
        return SAFR_ERR_IO;
    const size_t b_at = r.pos;
    r.pos += nb;
    if (r.get<uint64_t>() != fnv1a(b.data() + b_at, nb)) return SAFR_ERR_IO;

    safr_geometry g{};
    g.M = ints[0];
    g.P = ints[1];
    g.L = L;
    g.G = G;
    g.precision = ints[4];
    g.output_grid = ints[5];
    g.remove_tt = ints[6];
    g.pitch_m = dbl[0];
    g.diameter_m = dbl[1];
    g.obstruction = dbl[2];
    g.h_lgs_m = dbl[3];
    g.alpha = dbl[4];
    g.alpha_tt = dbl[5];
    g.beta = dbl[6];
    g.h_m = h.data();
    g.cn2 = cn2.data();
    g.dir_x = dx.data();
    g.dir_y = dy.data();
    std::vector<int> k(kind.begin(), kind.end());
    g.kind = k.data();
    safr_plan_t pl = nullptr;
    safr_status s = safr_plan_create(&g, cuda_device, &pl);
    if (s != SAFR_OK) return s;
    if (pl->b_bytes != nb) {
        safr_destroy(pl);
        return SAFR_ERR_IO;
    }
    {
        RefreshDeviceGuard guard(pl->device);
        if (!guard.ok || cudaMemcpy(pl->d_B, b.data() + b_at, nb, cudaMemcpyHostToDevice) != cudaSuccess) {
            safr_destroy(pl);
            return SAFR_ERR_CUDA;
        }
    }
    pl->precomputed = 1;
    pl->filter_learned = ints[7] ? 1 : 0;
    *out = pl;
    return SAFR_OK;
}

}  // extern "C"
