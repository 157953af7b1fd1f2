// safr_reconstruct_noalloc: the FP32 persistent frame kernel run without any
// device allocation.  The paper has no counterpart; this is a deployment form
// of the same reconstruction.
//
// Some callers cannot call cudaMalloc: a hard-real-time control thread (an
// allocation may synchronise the device and has no latency bound), a plugin
// inside a host framework that hands out all device memory from its own pool,
// or software whose rules forbid dynamic allocation after start-up.  A plan
// (safr_plan_create) allocates B, its tables and its workspaces, so those
// callers cannot use one.  Here the caller passes every input (the wavefronts
// and B) and every output (the layers and a status word) in memory it owns.
// The kernel's scratch (the row and layer spectra between its phases, its
// twiddle table and its grid-barrier counters) lives in the file-scope
// device array below.  That array is part of the library image, so every GPU
// that loads the library holds it until the process exits.
#include <cuda_runtime.h>

#include <cstdint>
#include <cstring>
#include <mutex>

#include "frame_impl.cuh"
#include "freqorder.h"
#include "plan.h"
#include "safr.h"

namespace safr {
bool frame2_configure_f32(safr_plan_s *pl, int nsm);
void *frame2_kernel_f32(int M);
}  // namespace safr

namespace {

static_assert(SAFR_NOALLOC_SCRATCH_BYTES % 256 == 0, "scratch size must be a multiple of 256 bytes");

// The shared scratch of every safr_reconstruct_noalloc call on a device.
static __device__ __align__(256) unsigned char g_noalloc_scratch[SAFR_NOALLOC_SCRATCH_BYTES];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mutex;
void *g_scratch_dev[kMaxDevices] = {};  // device address of g_noalloc_scratch, per device

// Launch shapes configured by earlier calls, per (device, M, P, L, G): a later call with the same
// shape makes no configuration queries (kernel attributes, occupancy).  Fixed size, no heap use;
// when it is full, the oldest entry is replaced.
struct ShapeEntry {
    int dev = -1, M = 0, P = 0, L = 0, G = 0;
    int grid = 0, stage_b = 0, rt3 = 0, cap3 = 0, tiles3 = 0, n3 = 0, st3[2] = {0, 0}, nsrc3[2] = {0, 0};
    unsigned off_rs = 0, off_tw = 0, off_b = 0, off_d = 0, off_xy = 0, off_s3 = 0;
    size_t smem = 0;
};
constexpr int kShapes = 32;
ShapeEntry g_shapes[kShapes];
int g_shapes_next = 0;

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

// Warp-FFT twiddles from FP64 sincospi: W_M^(t k) at [k * LW + t] for k < M / LW,
// then W_LW^e at [M + e] (LW = min(M, 32)); and the grid-barrier counters
// cleared for this call.
__global__ void k_noalloc_prepare(float2 *twq, int M, int LW, unsigned long long *bar)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    double s = 0.0, c = 1.0;
    if (i < M) {
        const int k = i / LW, t = i - k * LW;
        const long long e = ((long long)t * k) % M;
        sincospi(2.0 * (double)e / (double)M, &s, &c);
        twq[i] = make_float2((float)c, (float)-s);
    } else if (i < M + LW) {
        sincospi(2.0 * (double)(i - M) / (double)LW, &s, &c);
        twq[i] = make_float2((float)c, (float)-s);
    }
    if (i == 0) {
        bar[0] = 0ull;
        bar[1] = 0ull;
    }
}

bool aligned(const void *p, uintptr_t a) { return (reinterpret_cast<uintptr_t>(p) & (a - 1)) == 0; }

}  // namespace

extern "C" safr_status safr_reconstruct_noalloc(int cuda_device, int M, int P, int L, int G, const void *d_B,
                                                const float *d_wavefronts, float *d_layers, int *d_status,
                                                cudaStream_t stream)
{
    if (M < 8 || M > SAFR_MAX_M || (M & (M - 1))) return SAFR_ERR_UNSUPPORTED_SIZE;
    if (P < 1 || P > M || L < 1 || G < 1) return SAFR_ERR_INVALID_ARG;
    if (L > SAFR_MAX_L || G > SAFR_MAX_GROUP_G) return SAFR_ERR_UNSUPPORTED_SIZE;
    if (!d_B || !d_wavefronts || !d_layers || !d_status) return SAFR_ERR_INVALID_ARG;
    if (!aligned(d_B, 16) || !aligned(d_wavefronts, 16) || !aligned(d_layers, 16) || !aligned(d_status, 4))
        return SAFR_ERR_MISALIGNED;
    const int Mh = M / 2;
    // scratch carve-up: barrier counters | twiddles | row spectra w1 | layer spectra w2
    const size_t off_twq = 256;
    const int LW = safr::wfft_lanes(M);
    const size_t off_w1 = off_twq + align256((size_t)(M + LW) * sizeof(float2));
    const size_t off_w2 = off_w1 + align256((size_t)G * Mh * P * sizeof(float2));
    const size_t need = off_w2 + align256((size_t)L * Mh * M * sizeof(float2));
    if (need > (size_t)SAFR_NOALLOC_SCRATCH_BYTES) return SAFR_ERR_UNSUPPORTED_SIZE;

    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || cuda_device < 0 || cuda_device >= ndev ||
        cuda_device >= kMaxDevices) {
        cudaGetLastError();
        return SAFR_ERR_CUDA;
    }
    int prev = -1;
    if (cudaGetDevice(&prev) != cudaSuccess) return SAFR_ERR_CUDA;
    if (prev != cuda_device && cudaSetDevice(cuda_device) != cudaSuccess) return SAFR_ERR_CUDA;
    struct Restore {
        int dev, prev;
        ~Restore()
        {
            if (prev >= 0 && prev != dev) cudaSetDevice(prev);
        }
    } restore{cuda_device, prev};

    // set-up, once per device with that device current: the device address of the scratch array
    unsigned char *scratch = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_setup_mutex);
        if (!g_scratch_dev[cuda_device]) {
            void *ptr = nullptr;
            if (cudaGetSymbolAddress(&ptr, g_noalloc_scratch) != cudaSuccess || !ptr) {
                cudaGetLastError();
                return SAFR_ERR_CUDA;
            }
            g_scratch_dev[cuda_device] = ptr;
        }
        scratch = (unsigned char *)g_scratch_dev[cuda_device];
    }

    // launch shape of the persistent kernel for one star group: from the cache, else configured on a
    // plan on the stack (no heap use) and cached
    void *kernel = safr::frame2_kernel_f32(M);
    if (!kernel) return SAFR_ERR_UNSUPPORTED_SIZE;
    ShapeEntry sh;
    bool cached = false;
    {
        std::lock_guard<std::mutex> lock(g_setup_mutex);
        for (const ShapeEntry &e : g_shapes)
            if (e.dev == cuda_device && e.M == M && e.P == P && e.L == L && e.G == G) {
                sh = e;
                cached = true;
                break;
            }
    }
    if (!cached) {
        int nsm = 0, coop = 0;
        if (cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, cuda_device) != cudaSuccess ||
            cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, cuda_device) != cudaSuccess || !coop)
            return SAFR_ERR_CUDA;
        safr_plan_s pl;
        pl.device = cuda_device;
        pl.M = M;
        pl.P = P;
        pl.L = L;
        pl.G = G;
        pl.Mh = Mh;
        pl.o = (M - P) / 2;
        pl.precision = SAFR_FP32;
        pl.ngroups = 1;
        pl.grp[0].G = G;
        pl.grp[0].b_row0 = 0;
        pl.grp[0].resample = false;
        pl.sumLG = L * G;
        pl.f2_ck_allow = 0;  // the one-column kernel instance is the one launched below
        if (!safr::frame2_configure_f32(&pl, nsm)) return SAFR_ERR_UNSUPPORTED_SIZE;
        sh.dev = cuda_device;
        sh.M = M;
        sh.P = P;
        sh.L = L;
        sh.G = G;
        sh.grid = pl.f2_grid;
        sh.stage_b = pl.f2_stage_b;
        sh.rt3 = pl.f2_rt3;
        sh.cap3 = pl.f2_cap3;
        sh.tiles3 = pl.f2_tiles3;
        sh.n3 = pl.f2_n3;
        for (int gi = 0; gi < 2; ++gi) {
            sh.st3[gi] = pl.f2_st3[gi];
            sh.nsrc3[gi] = pl.f2_nsrc3[gi];
        }
        sh.off_rs = pl.f2_off_rs;
        sh.off_tw = pl.f2_off_tw;
        sh.off_b = pl.f2_off_b;
        sh.off_d = pl.f2_off_d;
        sh.off_xy = pl.f2_off_xy;
        sh.off_s3 = pl.f2_off_s3;
        sh.smem = pl.f2_smem;
        std::lock_guard<std::mutex> lock(g_setup_mutex);
        g_shapes[g_shapes_next] = sh;
        g_shapes_next = (g_shapes_next + 1) % kShapes;
    }

    using C = float2;
    safr::Frame2Params<float> fp;
    std::memset(&fp, 0, sizeof(fp));
    fp.P = P;
    fp.L = L;
    fp.G = G;
    fp.o = (M - P) / 2;
    fp.ngroups = 1;
    fp.sumLG = L * G;
    fp.npr = (P + 1) / 2;
    fp.n1 = G * fp.npr;
    fp.ntask2 = L;
    fp.rt3 = sh.rt3;
    fp.cap3 = sh.cap3;
    fp.tiles3 = sh.tiles3;
    fp.n3 = sh.n3;
    for (int gi = 0; gi < 2; ++gi) {
        fp.st3[gi] = sh.st3[gi];
        fp.nsrc3[gi] = sh.nsrc3[gi];
    }
    fp.any_tt = 0;
    fp.any_resample = 0;
    fp.stage_b = sh.stage_b;
    fp.skip_cta = -1;
    fp.timeout_ns = 1000000000ull;
    fp.inv_M2 = (float)(1.0 / ((double)M * M));
    fp.off_rs = sh.off_rs;
    fp.off_tw = sh.off_tw;
    fp.off_b = sh.off_b;
    fp.off_d = sh.off_d;
    fp.off_xy = sh.off_xy;
    fp.off_s3 = sh.off_s3;
    fp.in = d_wavefronts;
    fp.out = d_layers;
    fp.B = (const C *)d_B;
    fp.w1 = (C *)(scratch + off_w1);
    fp.w2 = (C *)(scratch + off_w2);
    fp.twq = (const C *)(scratch + off_twq);
    fp.bar = (unsigned long long *)scratch;
    fp.status = d_status;
    fp.grp[0].G = G;
    fp.grp[0].b_row0 = 0;
    fp.grp[0].resample = 0;
    for (int g = 0; g < G; ++g) fp.grp[0].star[g] = g;

    // the launches report their own errors (the caller's pending error state is left alone)
    float2 *twq = (float2 *)(scratch + off_twq);
    unsigned long long *bar = (unsigned long long *)scratch;
    int m_arg = M, lw_arg = LW;
    void *pargs[] = {&twq, &m_arg, &lw_arg, &bar};
    if (cudaLaunchKernel((const void *)k_noalloc_prepare, dim3((M + LW + 255) / 256), dim3(256), pargs, 0, stream) !=
        cudaSuccess)
        return SAFR_ERR_CUDA;
    void *args[] = {&fp};
    if (cudaLaunchCooperativeKernel(kernel, dim3(sh.grid), dim3(safr::frame2_threads(M)), args, sh.smem, stream) !=
        cudaSuccess)
        return SAFR_ERR_CUDA;
    return SAFR_OK;
}
