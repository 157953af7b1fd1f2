// Batched frames and the schedule autotuner.
//
// safr_batch_*: n frames, frame i reconstructed by plans[i] (plans may differ in
// geometry).  FP32 frames whose plan runs the persistent kernel are grouped by
// grid size M; each group is ONE persistent cooperative launch that runs its
// frames one after the other on the whole grid (k_frame2_batch), so a CTA
// starts the next frame's loads while others finish the last one and there is
// no launch gap between frames.  The parameter copy and the group launches are
// captured once into a CUDA graph and replayed by every later call.  Frames of
// other plans (FP16 storage, FP64, the three-pass schedule) are launched on
// the stream after the graph.
//
// safr_autotune: times the candidate schedules of a plan (persistent kernel
// with each feasible phase-3 tile height, and the three-pass schedule) on the
// plan's own device buffers and keeps the fastest; results are cached per
// plan shape and device, so plans of the same shape are tuned once.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <tuple>
#include <vector>

#include "frame_impl.cuh"
#include "plan.h"
#include "safr.h"

namespace safr {
bool frame2_configure_f32(safr_plan_s *pl, int nsm);
bool configure_fused(safr_plan_s *pl);
cudaError_t launch_fused(safr_plan_s *pl, const void *in, const float *in_scales, void *out, float *out_scales,
                         cudaStream_t stream);
}  // namespace safr

namespace {

using safr::Frame2Params;

// grid sizes with a batch kernel instance (FP32)
template <int M>
struct BatchInst {
    static void *kernel() { return (void *)safr::k_frame2_batch<M>; }
    static Frame2Params<float> params(safr_plan_s *pl, const void *in, void *out)
    {
        return safr::Frame2Host<M, float>::params(pl, in, nullptr, out, nullptr);
    }
};

template <typename F>
bool with_batch_m(int M, F &&f)
{
    switch (M) {
    case 32: f(BatchInst<32>{}); return true;
    case 64: f(BatchInst<64>{}); return true;
    case 128: f(BatchInst<128>{}); return true;
    case 256: f(BatchInst<256>{}); return true;
    case 512: f(BatchInst<512>{}); return true;
    default: return false;
    }
}

bool aligned16(const void *p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

// ---------------------------------------------------------------------------
// autotune cache: plan shape and device -> (path, phase-3 tile rows)
// ---------------------------------------------------------------------------
using TuneKey = std::tuple<int, int, int, int, int, int, int, int, int, int, int>;
std::mutex g_tune_mutex;
std::map<TuneKey, std::pair<int, int>> g_tune;

TuneKey tune_key(const safr_plan_s *pl)
{
    int nsm = 0;
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, pl->device);
    const int g0 = pl->ngroups > 0 ? pl->grp[0].G : 0, g1 = pl->ngroups > 1 ? pl->grp[1].G : 0;
    const int rs = pl->ngroups > 0 && pl->grp[0].resample ? 1 : 0;
    return TuneKey(pl->device, nsm, pl->M, pl->P, pl->L, g0, g1, pl->precision, pl->remove_tt, rs, pl->ngroups);
}

}  // namespace

// ---------------------------------------------------------------------------
// batch object
// ---------------------------------------------------------------------------
struct safr_batch_s {
    struct Group {
        int M = 0;
        void *kernel = nullptr;
        std::vector<int> frames;  // indices into the batch
        size_t smem = 0;
        size_t first = 0;         // first parameter slot of the group
        unsigned long long *d_bar = nullptr;
    };
    int device = 0, n = 0, grid = 0;
    std::vector<safr_plan_s *> plans;
    std::vector<Group> groups;
    std::vector<int> loose;  // frames launched one by one through safr_reconstruct
    size_t nslots = 0;
    Frame2Params<float> *h_params[2] = {nullptr, nullptr};  // page-locked
    Frame2Params<float> *d_params[2] = {nullptr, nullptr};
    cudaEvent_t done[2] = {nullptr, nullptr};
    cudaGraphExec_t exec[2] = {nullptr, nullptr};
    bool tried[2] = {false, false};
    cudaStream_t cap = nullptr;
    unsigned long long calls = 0;
};

namespace {

struct BatchDeviceGuard {
    int prev = -1;
    bool ok = false;
    explicit BatchDeviceGuard(int dev)
    {
        if (cudaGetDevice(&prev) != cudaSuccess) return;
        if (prev != dev && cudaSetDevice(dev) != cudaSuccess) return;
        ok = true;
    }
    ~BatchDeviceGuard()
    {
        if (ok && prev >= 0) cudaSetDevice(prev);
    }
};

void batch_free(safr_batch_s *b)
{
    for (auto &g : b->groups)
        if (g.d_bar) cudaFree(g.d_bar);
    for (int c = 0; c < 2; ++c) {
        if (b->h_params[c]) cudaFreeHost(b->h_params[c]);
        if (b->d_params[c]) cudaFree(b->d_params[c]);
        if (b->done[c]) cudaEventDestroy(b->done[c]);
        if (b->exec[c]) cudaGraphExecDestroy(b->exec[c]);
    }
    if (b->cap) cudaStreamDestroy(b->cap);
}

// One cooperative launch of a group's batch kernel on `st`.
cudaError_t launch_group(const safr_batch_s *b, const safr_batch_s::Group &g, int c, cudaStream_t st)
{
    const Frame2Params<float> *dp = b->d_params[c] + g.first;
    int nfr = (int)g.frames.size();
    unsigned long long *bar = g.d_bar;
    void *args[] = {(void *)&dp, (void *)&nfr, (void *)&bar};
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(b->grid);
    cfg.blockDim = dim3(safr::frame2_threads(g.M));
    cfg.dynamicSmemBytes = g.smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelExC(&cfg, g.kernel, args);
}

// parameter copy + group launches, on `st`
cudaError_t enqueue_groups(const safr_batch_s *b, int c, cudaStream_t st)
{
    cudaError_t e = cudaMemcpyAsync(b->d_params[c], b->h_params[c], b->nslots * sizeof(Frame2Params<float>),
                                    cudaMemcpyHostToDevice, st);
    for (const auto &g : b->groups)
        if (e == cudaSuccess) e = launch_group(b, g, c, st);
    return e;
}

// Capture the copy and the group launches of parameter buffer c into a graph.
void capture(safr_batch_s *b, int c)
{
    b->tried[c] = true;
    cudaGraph_t graph = nullptr;
    if (cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
        cudaGetLastError();
        return;
    }
    const cudaError_t e = enqueue_groups(b, c, b->cap);
    const cudaError_t e2 = cudaStreamEndCapture(b->cap, &graph);
    if (e != cudaSuccess || e2 != cudaSuccess || !graph ||
        cudaGraphInstantiate(&b->exec[c], graph, 0) != cudaSuccess) {
        b->exec[c] = nullptr;
        cudaGetLastError();
    }
    if (graph) cudaGraphDestroy(graph);
}

}  // namespace

extern "C" {

safr_status safr_batch_create(const safr_plan_t *plans, int n, safr_batch_t *out)
{
    if (!out) return SAFR_ERR_INVALID_ARG;
    *out = nullptr;
    if (!plans || n < 1) return SAFR_ERR_INVALID_ARG;
    for (int i = 0; i < n; ++i)
        if (!plans[i] || plans[i]->device != plans[0]->device) return SAFR_ERR_INVALID_ARG;
    BatchDeviceGuard guard(plans[0]->device);
    if (!guard.ok) return SAFR_ERR_CUDA;
    safr_batch_s *b = new (std::nothrow) safr_batch_s();
    if (!b) return SAFR_ERR_OOM;
    b->device = plans[0]->device;
    b->n = n;
    b->plans.assign(plans, plans + n);
    auto fail = [&](safr_status s) {
        batch_free(b);
        delete b;
        cudaGetLastError();
        return s;
    };
    // FP32 frames on the persistent kernel, grouped by grid size; the rest go one by one
    for (int i = 0; i < n; ++i) {
        safr_plan_s *pl = plans[i];
        bool grouped = false;
        if (pl->precision == SAFR_FP32 && safr::use_fused(pl)) {
            with_batch_m(pl->M, [&](auto inst) {
                using I = decltype(inst);
                auto it = std::find_if(b->groups.begin(), b->groups.end(),
                                       [&](const safr_batch_s::Group &g) { return g.M == pl->M; });
                if (it == b->groups.end()) {
                    safr_batch_s::Group g;
                    g.M = pl->M;
                    g.kernel = I::kernel();
                    b->groups.push_back(g);
                    it = b->groups.end() - 1;
                }
                it->frames.push_back(i);
                it->smem = std::max(it->smem, pl->f2_smem);
                b->grid = pl->f2_grid;
                grouped = true;
            });
        }
        if (!grouped) b->loose.push_back(i);
    }
    for (auto &g : b->groups) {
        g.first = b->nslots;
        b->nslots += g.frames.size();
        if (!safr::smem_limit_allows(g.kernel, g.smem)) return fail(SAFR_ERR_UNSUPPORTED_SIZE);
        int occ = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, g.kernel, safr::frame2_threads(g.M), g.smem) !=
                cudaSuccess ||
            occ < 1)
            return fail(SAFR_ERR_UNSUPPORTED_SIZE);
        if (cudaMalloc((void **)&g.d_bar, 2 * sizeof(unsigned long long)) != cudaSuccess) return fail(SAFR_ERR_OOM);
        if (cudaMemset(g.d_bar, 0, 2 * sizeof(unsigned long long)) != cudaSuccess) return fail(SAFR_ERR_CUDA);
    }
    if (b->nslots > 0)
        for (int c = 0; c < 2; ++c) {
            if (cudaMallocHost((void **)&b->h_params[c], b->nslots * sizeof(Frame2Params<float>)) != cudaSuccess)
                return fail(SAFR_ERR_OOM);
            if (cudaMalloc((void **)&b->d_params[c], b->nslots * sizeof(Frame2Params<float>)) != cudaSuccess)
                return fail(SAFR_ERR_OOM);
        }
    for (int c = 0; c < 2; ++c)
        if (cudaEventCreateWithFlags(&b->done[c], cudaEventDisableTiming) != cudaSuccess) return fail(SAFR_ERR_CUDA);
    if (cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking) != cudaSuccess) return fail(SAFR_ERR_CUDA);
    *out = b;
    return SAFR_OK;
}

safr_status safr_batch_reconstruct(safr_batch_t b, const void *const *d_wavefronts, const float *const *d_in_scales,
                                   void *const *d_layers, float *const *d_out_scales, cudaStream_t stream)
{
    if (!b || !d_wavefronts || !d_layers) return SAFR_ERR_INVALID_ARG;
    for (int i = 0; i < b->n; ++i) {
        const safr_plan_s *pl = b->plans[i];
        if (!pl->precomputed) return SAFR_ERR_NOT_PRECOMPUTED;
        if (!d_wavefronts[i] || !d_layers[i]) return SAFR_ERR_INVALID_ARG;
        if (!aligned16(d_wavefronts[i]) || !aligned16(d_layers[i])) return SAFR_ERR_MISALIGNED;
        const bool fp16 = pl->precision == SAFR_FP16_STORAGE;
        if (fp16 && (!d_out_scales || !d_out_scales[i])) return SAFR_ERR_INVALID_ARG;
    }
    for (const auto &g : b->groups)  // schedules fixed when the batch was created (autotune first)
        for (int i : g.frames)
            if (!safr::use_fused(b->plans[i]) || b->plans[i]->f2_smem > g.smem) return SAFR_ERR_INVALID_ARG;
    BatchDeviceGuard guard(b->device);
    if (!guard.ok) return SAFR_ERR_CUDA;
    const int c = (int)(b->calls & 1u);
    // the call that last used parameter buffer c has finished with it
    if (b->calls >= 2 && cudaEventSynchronize(b->done[c]) != cudaSuccess) return SAFR_ERR_CUDA;
    for (const auto &g : b->groups)
        for (size_t s = 0; s < g.frames.size(); ++s) {
            const int i = g.frames[s];
            safr_plan_s *pl = b->plans[i];
            Frame2Params<float> fp{};
            with_batch_m(g.M, [&](auto inst) { fp = decltype(inst)::params(pl, d_wavefronts[i], d_layers[i]); });
            fp.bar = g.d_bar;
            fp.stamps = nullptr;
            fp.skip_cta = -1;
            b->h_params[c][g.first + s] = fp;
        }
    if (b->nslots > 0) {
        if (!b->tried[c]) capture(b, c);
        const cudaError_t e = b->exec[c] ? cudaGraphLaunch(b->exec[c], stream) : enqueue_groups(b, c, stream);
        if (e != cudaSuccess) {
            cudaGetLastError();
            return SAFR_ERR_CUDA;
        }
    }
    for (int i : b->loose) {
        const safr_status s = safr_reconstruct(b->plans[i], d_wavefronts[i], d_in_scales ? d_in_scales[i] : nullptr,
                                               d_layers[i], d_out_scales ? d_out_scales[i] : nullptr, stream);
        if (s != SAFR_OK) return s;
    }
    if (cudaEventRecord(b->done[c], stream) != cudaSuccess) return SAFR_ERR_CUDA;
    ++b->calls;
    return SAFR_OK;
}

safr_status safr_batch_get_status(safr_batch_t b)
{
    if (!b) return SAFR_ERR_INVALID_ARG;
    BatchDeviceGuard guard(b->device);
    if (!guard.ok) return SAFR_ERR_CUDA;
    safr_status first = SAFR_OK;
    for (int i = 0; i < b->n; ++i) {
        const safr_status s = safr_get_status(b->plans[i]);
        if (first == SAFR_OK) first = s;
    }
    if (first != SAFR_OK)  // re-arm the groups' barriers, which a timeout leaves half-counted
        for (auto &g : b->groups)
            if (cudaMemset(g.d_bar, 0, 2 * sizeof(unsigned long long)) != cudaSuccess) return SAFR_ERR_CUDA;
    if (cudaDeviceSynchronize() != cudaSuccess) return SAFR_ERR_CUDA;
    return first;
}

int safr_batch_launches(safr_batch_t b)
{
    if (!b) return 0;
    int n = (int)b->groups.size();
    for (int i : b->loose) n += safr_launches_per_frame(b->plans[i]);
    return n;
}

safr_status safr_batch_destroy(safr_batch_t b)
{
    if (!b) return SAFR_ERR_INVALID_ARG;
    {
        BatchDeviceGuard guard(b->device);
        cudaDeviceSynchronize();
        batch_free(b);
    }
    delete b;
    return SAFR_OK;
}

}  // extern "C"

namespace {

// Apply a schedule: path, and the phase-3 tile rows of the persistent kernel (0: cost model).
bool apply_schedule(safr_plan_s *pl, int path, int rt)
{
    if (pl->fused_ok) {
        pl->f2_rt_force = rt;
        if (!safr::configure_fused(pl)) {
            pl->f2_rt_force = 0;
            safr::configure_fused(pl);
            cudaGetLastError();
            return false;
        }
    }
    pl->path = path;
    pl->traced = 0;
    return true;
}

}  // namespace

extern "C" safr_status safr_autotune(safr_plan_t pl, cudaStream_t stream)
{
    if (!pl) return SAFR_ERR_INVALID_ARG;
    if (!pl->precomputed) return SAFR_ERR_NOT_PRECOMPUTED;
    BatchDeviceGuard guard(pl->device);
    if (!guard.ok) return SAFR_ERR_CUDA;
    const TuneKey key = tune_key(pl);
    {
        std::lock_guard<std::mutex> lock(g_tune_mutex);
        auto it = g_tune.find(key);
        if (it != g_tune.end()) {
            apply_schedule(pl, it->second.first, it->second.second);
            pl->autotuned = 1;
            return SAFR_OK;
        }
    }
    // candidates: the persistent kernel with every feasible phase-3 tile height, the three passes
    std::vector<std::pair<int, int>> cand;
    if (pl->fused_ok)
        for (int rt = std::min(32, pl->M); rt >= 2; rt -= 2)
            if (apply_schedule(pl, SAFR_PATH_FUSED, rt) && pl->f2_rt3 == rt) cand.emplace_back(SAFR_PATH_FUSED, rt);
    cand.emplace_back(SAFR_PATH_PASSES, 0);
    // timing buffers (set-up call: it allocates and synchronises)
    const bool fp16 = pl->precision == SAFR_FP16_STORAGE;
    void *d_in = nullptr, *d_out = nullptr;
    float *d_osc = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    safr_status st = SAFR_OK;
    if (cudaMalloc(&d_in, pl->in_bytes) != cudaSuccess || cudaMalloc(&d_out, pl->out_bytes) != cudaSuccess ||
        (fp16 && cudaMalloc((void **)&d_osc, (size_t)pl->L * sizeof(float)) != cudaSuccess))
        st = SAFR_ERR_OOM;
    if (st == SAFR_OK && (cudaMemsetAsync(d_in, 0, pl->in_bytes, stream) != cudaSuccess ||
                          cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess))
        st = SAFR_ERR_CUDA;
    std::pair<int, int> best(pl->fused_ok ? SAFR_PATH_FUSED : SAFR_PATH_PASSES, 0);
    float best_ms = 1e30f;
    const int trace = pl->trace;
    pl->trace = 0;
    for (size_t ci = 0; st == SAFR_OK && ci < cand.size(); ++ci) {
        if (!apply_schedule(pl, cand[ci].first, cand[ci].second)) continue;
        for (int w = 0; w < 3 && st == SAFR_OK; ++w)
            st = safr_reconstruct(pl, d_in, nullptr, d_out, d_osc, stream);
        if (st != SAFR_OK) break;
        const int reps = 10;
        if (cudaEventRecord(e0, stream) != cudaSuccess) st = SAFR_ERR_CUDA;
        for (int r = 0; r < reps && st == SAFR_OK; ++r) st = safr_reconstruct(pl, d_in, nullptr, d_out, d_osc, stream);
        float ms = 0;
        if (st == SAFR_OK && (cudaEventRecord(e1, stream) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
                              cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess))
            st = SAFR_ERR_CUDA;
        if (st == SAFR_OK && ms < best_ms) {
            best_ms = ms;
            best = cand[ci];
        }
    }
    pl->trace = trace;
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (d_in) cudaFree(d_in);
    if (d_out) cudaFree(d_out);
    if (d_osc) cudaFree(d_osc);
    apply_schedule(pl, best.first, best.second);
    if (st != SAFR_OK) {
        cudaGetLastError();
        return st;
    }
    pl->autotuned = 1;
    std::lock_guard<std::mutex> lock(g_tune_mutex);
    g_tune[key] = best;
    return SAFR_OK;
}
