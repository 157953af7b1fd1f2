// Batched frames and the schedule autotuner.
//
// safr_batch_*: n frames, frame i reconstructed by plans[i] (plans may differ in
// geometry, precision and schedule).  Every frame's launches (one persistent
// cooperative kernel, or the three passes) are captured into ONE CUDA graph;
// each call replays it with a single graph launch.  The graph bakes in the
// frames' buffer pointers, so a call with other pointers captures it again.
// Frames of grids up to 256 may run on K concurrent chains of the graph, each
// on 1/K of the SMs; K in {1, 2, 4, 8} is timed at the first capture.
//
// A single persistent launch that loops over a device array of frame
// parameters was built and measured slower than this graph (4.49 ms against
// 3.83 ms per batch of the 64-frame uneven workload): its frame parameters
// come from memory instead of the constant bank that holds kernel arguments,
// which costs registers (spills at M = 512) and load latency in every phase.
//
// safr_autotune: times the candidate schedules of a plan (persistent kernel
// with each feasible phase-3 tile height, and the three-pass schedule) on the
// plan's own device and keeps the fastest; results are cached per plan shape
// and device, so plans of the same shape are tuned once.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <map>
#include <mutex>
#include <new>
#include <tuple>
#include <vector>

#include "plan.h"
#include "safr.h"

namespace {

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

bool aligned16(const void *p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

}  // namespace

// ---------------------------------------------------------------------------
// batch object
// ---------------------------------------------------------------------------
struct safr_batch_s {
    int device = 0, n = 0;
    std::vector<safr_plan_s *> plans;
    cudaGraphExec_t exec = nullptr;
    bool graph_failed = false;
    std::vector<const void *> key;  // buffer pointers and schedules the graph was captured with
    cudaStream_t cap = nullptr;
    int chains = 0;                    // concurrent chains of the graph (0: not chosen yet)
    std::vector<cudaStream_t> side;    // capture-side streams of chains 1..
    std::vector<cudaEvent_t> ev;       // fork / join events
};

namespace {

// the frames' launches on `st`, in order
safr_status enqueue_frames(safr_batch_s *b, const void *const *in, const float *const *isc, void *const *out,
                           float *const *osc, cudaStream_t st)
{
    for (int i = 0; i < b->n; ++i) {
        const safr_status s =
            safr_reconstruct(b->plans[i], in[i], isc ? isc[i] : nullptr, out[i], osc ? osc[i] : nullptr, st);
        if (s != SAFR_OK) return s;
    }
    return SAFR_OK;
}

// Frames that may run K at a time: persistent-kernel plans of grids up to 256 (latency-bound: on
// 1/K of the SMs each, K of them finish sooner than one after the other), and one-cluster plans
// (a cluster of at most 16 SMs each).  Larger frames run alone on the whole GPU.  A plan that
// appears twice keeps the batch sequential.
bool concurrent_frame(const safr_plan_s *pl)
{
    return (safr::use_fused(pl) && pl->M <= 256) || safr::use_cluster(pl);
}

int concurrent_count(const safr_batch_s *b)
{
    std::vector<const safr_plan_s *> seen;
    int n = 0;
    for (const safr_plan_s *pl : b->plans) {
        if (std::find(seen.begin(), seen.end(), pl) != seen.end()) return 0;
        seen.push_back(pl);
        n += concurrent_frame(pl) ? 1 : 0;
    }
    return n;
}

// Capture the frames' launches into a graph (trace events left out).  K = 1: one chain, frame after
// frame.  K > 1: the large frames one after the other, then the concurrent frames on K chains at
// 1/K of the SMs each, assigned greedily by an estimate of their cost.
bool capture_k(safr_batch_s *b, int K, const void *const *in, const float *const *isc, void *const *out,
               float *const *osc, cudaGraphExec_t *exec_out)
{
    *exec_out = nullptr;
    std::vector<int> trace(b->n);
    for (int i = 0; i < b->n; ++i) {
        trace[i] = b->plans[i]->trace;
        b->plans[i]->trace = 0;
    }
    int nsm = 0;
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, b->device);
    // the concurrent frames' plans on 1/K of the SMs, with their phase-3 tiling kept (every layer
    // sample is then computed by the same arithmetic as on the plan's own grid); set up before the
    // capture and put back after it (the captured launches keep their own copies of the parameters)
    struct Saved {
        safr_plan_s *pl;
        int grid, rt, pdl;
    };
    std::vector<Saved> saved;
    bool conf_ok = true;
    if (K > 1)
        for (safr_plan_s *pl : b->plans)
            if (concurrent_frame(pl) && safr::use_fused(pl)) {  // a one-cluster frame keeps its cluster
                saved.push_back({pl, pl->f2_grid_force, pl->f2_rt_force, pl->f2_pdl});
                pl->f2_grid_force = nsm / K;
                pl->f2_rt_force = pl->f2_rt3;
                pl->f2_pdl = 0;  // no early CTAs holding SMs the other chains could use
                conf_ok = conf_ok && safr::configure_fused(pl) && safr::use_fused(pl);
            }
    cudaGraph_t graph = nullptr;
    bool ok = false;
    if (conf_ok && cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal) == cudaSuccess) {
        safr_status s = SAFR_OK;
        if (K <= 1) {
            s = enqueue_frames(b, in, isc, out, osc, b->cap);
        } else {
            for (int i = 0; i < b->n && s == SAFR_OK; ++i)
                if (!concurrent_frame(b->plans[i]))
                    s = safr_reconstruct(b->plans[i], in[i], isc ? isc[i] : nullptr, out[i], osc ? osc[i] : nullptr,
                                         b->cap);
            // fork: chains 1..K-1 start after the large frames
            if (s == SAFR_OK && cudaEventRecord(b->ev[0], b->cap) != cudaSuccess) s = SAFR_ERR_CUDA;
            for (int c = 1; c < K && s == SAFR_OK; ++c)
                if (cudaStreamWaitEvent(b->side[c - 1], b->ev[0], 0) != cudaSuccess) s = SAFR_ERR_CUDA;
            // greedy: largest frames first, each to the chain with the least work so far
            std::vector<int> idx;
            for (int i = 0; i < b->n; ++i)
                if (concurrent_frame(b->plans[i])) idx.push_back(i);
            auto cost = [&](int i) {
                const safr_plan_s *pl = b->plans[i];
                return (double)pl->M * pl->M * (pl->sumLG + pl->L + pl->G);
            };
            std::sort(idx.begin(), idx.end(), [&](int x, int y) { return cost(x) > cost(y); });
            std::vector<double> load(K, 0.0);
            for (int i : idx) {
                if (s != SAFR_OK) break;
                const int c = (int)(std::min_element(load.begin(), load.end()) - load.begin());
                load[c] += cost(i);
                s = safr_reconstruct(b->plans[i], in[i], isc ? isc[i] : nullptr, out[i], osc ? osc[i] : nullptr,
                                     c == 0 ? b->cap : b->side[c - 1]);
            }
            // join
            for (int c = 1; c < K && s == SAFR_OK; ++c)
                if (cudaEventRecord(b->ev[c], b->side[c - 1]) != cudaSuccess ||
                    cudaStreamWaitEvent(b->cap, b->ev[c], 0) != cudaSuccess)
                    s = SAFR_ERR_CUDA;
        }
        const cudaError_t e = cudaStreamEndCapture(b->cap, &graph);
        ok = s == SAFR_OK && e == cudaSuccess && graph && cudaGraphInstantiate(exec_out, graph, 0) == cudaSuccess;
        if (!ok) *exec_out = nullptr;
        if (graph) cudaGraphDestroy(graph);
    }
    cudaGetLastError();
    for (const Saved &v : saved) {
        v.pl->f2_grid_force = v.grid;
        v.pl->f2_rt_force = v.rt;
        v.pl->f2_pdl = v.pdl;
        safr::configure_fused(v.pl);
    }
    cudaGetLastError();
    for (int i = 0; i < b->n; ++i) b->plans[i]->trace = trace[i];
    return ok;
}

// Median time of three replays (after one) of a captured batch on the capture stream, in ms; < 0 on error.
float time_graph(safr_batch_s *b, cudaGraphExec_t ex)
{
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) return -1.0f;
    std::vector<float> t;
    for (int r = 0; r < 4; ++r) {
        float ms = -1.0f;
        if (cudaEventRecord(e0, b->cap) != cudaSuccess || cudaGraphLaunch(ex, b->cap) != cudaSuccess ||
            cudaEventRecord(e1, b->cap) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
            cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess)
            ms = -1.0f;
        if (r > 0) t.push_back(ms);
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    std::sort(t.begin(), t.end());
    return t[0] < 0 ? -1.0f : t[1];
}

// (Re)capture the batch's graph.  The first time, every chain count K in {1, 2, 4, 8} that the batch
// can use is captured and timed, and the fastest is kept for later captures.
void capture(safr_batch_s *b, const void *const *in, const float *const *isc, void *const *out, float *const *osc)
{
    if (b->exec) cudaGraphExecDestroy(b->exec);
    b->exec = nullptr;
    b->graph_failed = true;
    const int nconc = concurrent_count(b);
    if (b->side.empty() && nconc >= 2) {  // streams and events of up to 8 chains
        b->side.assign(7, nullptr);
        b->ev.assign(8, nullptr);
        bool ok = true;
        for (auto &st : b->side) ok = ok && cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) == cudaSuccess;
        for (auto &e : b->ev) ok = ok && cudaEventCreateWithFlags(&e, cudaEventDisableTiming) == cudaSuccess;
        if (!ok) {
            cudaGetLastError();
            b->chains = 1;
        }
    }
    if (nconc < 2) b->chains = 1;
    if (b->chains == 0) {
        int best_k = 1;
        float best_t = -1.0f;
        cudaGraphExec_t best = nullptr;
        for (int K : {1, 2, 4, 8}) {
            if (K > 1 && nconc < K) continue;
            cudaGraphExec_t ex = nullptr;
            if (!capture_k(b, K, in, isc, out, osc, &ex)) continue;
            const float t = time_graph(b, ex);
            if (t >= 0.0f && (best_t < 0.0f || t < best_t)) {
                if (best) cudaGraphExecDestroy(best);
                best = ex;
                best_t = t;
                best_k = K;
            } else {
                cudaGraphExecDestroy(ex);
            }
        }
        b->chains = best_k;
        b->exec = best;
    } else {
        capture_k(b, b->chains, in, isc, out, osc, &b->exec);
    }
    b->graph_failed = b->exec == nullptr;
    cudaGetLastError();
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
    if (cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking) != cudaSuccess) {
        cudaGetLastError();
        delete b;
        return SAFR_ERR_CUDA;
    }
    *out = b;
    return SAFR_OK;
}

safr_status safr_batch_reconstruct(safr_batch_t b, const void *const *d_wavefronts, const float *const *d_in_scales,
                                   void *const *d_layers, float *const *d_out_scales, cudaStream_t stream)
{
    if (!b || !d_wavefronts || !d_layers) return SAFR_ERR_INVALID_ARG;
    std::vector<const void *> key;
    key.reserve((size_t)b->n * 6);
    for (int i = 0; i < b->n; ++i) {
        const safr_plan_s *pl = b->plans[i];
        if (!pl->precomputed) return SAFR_ERR_NOT_PRECOMPUTED;
        if (!d_wavefronts[i] || !d_layers[i]) return SAFR_ERR_INVALID_ARG;
        if (!aligned16(d_wavefronts[i]) || !aligned16(d_layers[i])) return SAFR_ERR_MISALIGNED;
        const bool fp16 = pl->precision == SAFR_FP16_STORAGE;
        const float *isc = d_in_scales ? d_in_scales[i] : nullptr;
        float *osc = d_out_scales ? d_out_scales[i] : nullptr;
        if (fp16 && !osc) return SAFR_ERR_INVALID_ARG;
        if (!fp16 && (isc || osc)) return SAFR_ERR_INVALID_ARG;
        if ((isc && !aligned16(isc)) || (osc && !aligned16(osc))) return SAFR_ERR_MISALIGNED;
        key.push_back(d_wavefronts[i]);
        key.push_back(isc);
        key.push_back(d_layers[i]);
        key.push_back(osc);
        key.push_back((const void *)(uintptr_t)(safr::use_cluster(pl) ? 1 : (safr::use_fused(pl) ? 2 + pl->f2_rt3 : 0)));
        key.push_back((const void *)(uintptr_t)pl->f2_smem);
    }
    BatchDeviceGuard guard(b->device);
    if (!guard.ok) return SAFR_ERR_CUDA;
    if (key != b->key) {  // other buffers or schedules: capture again
        b->key = key;
        capture(b, d_wavefronts, d_in_scales, d_layers, d_out_scales);
    }
    if (b->exec) {
        if (cudaGraphLaunch(b->exec, stream) != cudaSuccess) {
            cudaGetLastError();
            return SAFR_ERR_CUDA;
        }
        return SAFR_OK;
    }
    return enqueue_frames(b, d_wavefronts, d_in_scales, d_layers, d_out_scales, stream);
}

safr_status safr_batch_get_status(safr_batch_t b)
{
    if (!b) return SAFR_ERR_INVALID_ARG;
    safr_status first = SAFR_OK;
    for (int i = 0; i < b->n; ++i) {
        const safr_status s = safr_get_status(b->plans[i]);
        if (first == SAFR_OK) first = s;
    }
    return first;
}

int safr_batch_launches(safr_batch_t b)
{
    if (!b) return 0;
    int n = 0;
    for (int i = 0; i < b->n; ++i) n += safr_launches_per_frame(b->plans[i]);
    return n;
}

int safr_batch_graph(safr_batch_t b) { return b && b->exec ? 1 : 0; }

int safr_batch_chains(safr_batch_t b) { return b ? b->chains : 0; }

safr_status safr_batch_set_chains(safr_batch_t b, int chains)
{
    if (!b || !(chains == 0 || chains == 1 || chains == 2 || chains == 4 || chains == 8)) return SAFR_ERR_INVALID_ARG;
    b->chains = chains;
    b->key.clear();  // the next call captures the graph again
    return SAFR_OK;
}

safr_status safr_batch_destroy(safr_batch_t b)
{
    if (!b) return SAFR_ERR_INVALID_ARG;
    {
        BatchDeviceGuard guard(b->device);
        cudaDeviceSynchronize();
        if (b->exec) cudaGraphExecDestroy(b->exec);
        if (b->cap) cudaStreamDestroy(b->cap);
        for (auto st : b->side)
            if (st) cudaStreamDestroy(st);
        for (auto e : b->ev)
            if (e) cudaEventDestroy(e);
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
    // candidates: the one-cluster kernel, the persistent kernel with every feasible phase-3 tile
    // height, the three passes
    std::vector<std::pair<int, int>> cand;
    if (pl->cl_ok) cand.emplace_back(SAFR_PATH_CLUSTER, 0);
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
    std::pair<int, int> best(pl->cl_ok ? SAFR_PATH_CLUSTER : (pl->fused_ok ? SAFR_PATH_FUSED : SAFR_PATH_PASSES), 0);
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
