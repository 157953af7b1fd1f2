// Host entry points of the one-cluster frame kernel (grids up to 64):
// configuration at plan creation and the per-frame launch (with trace events).
#include <cuda_runtime.h>

#include "cluster_impl.cuh"
#include "plan.h"

namespace safr {

template <typename R, typename TIN, typename TOUT, int M>
struct ClusterInst {
    static void *kernel() { return (void *)k_cluster<M, R, TIN, TOUT>; }
};

template <typename R, typename TIN, typename TOUT>
static void *cluster_kernel_of(int M)
{
    switch (M) {
    case 8: return ClusterInst<R, TIN, TOUT, 8>::kernel();
    case 16: return ClusterInst<R, TIN, TOUT, 16>::kernel();
    case 32: return ClusterInst<R, TIN, TOUT, 32>::kernel();
    case 64: return ClusterInst<R, TIN, TOUT, 64>::kernel();
    default: return nullptr;
    }
}

static void *cluster_kernel(const safr_plan_s *pl)
{
    if (pl->precision == SAFR_FP64) return cluster_kernel_of<double, double, double>(pl->M);
    if (pl->precision == SAFR_FP16_STORAGE) return cluster_kernel_of<float, __half, __half>(pl->M);
    return cluster_kernel_of<float, float, float>(pl->M);
}

template <typename R>
static bool configure_m(safr_plan_s *pl, void *k)
{
    switch (pl->M) {
    case 8: return ClusterHost<8, R>::configure(pl, k);
    case 16: return ClusterHost<16, R>::configure(pl, k);
    case 32: return ClusterHost<32, R>::configure(pl, k);
    case 64: return ClusterHost<64, R>::configure(pl, k);
    default: return false;
    }
}

template <typename R>
static cudaError_t launch_m(void *k, safr_plan_s *pl, const void *in, const float *isc, void *out, float *osc,
                            cudaStream_t st)
{
    switch (pl->M) {
    case 8: return ClusterHost<8, R>::launch(k, pl, in, isc, out, osc, st);
    case 16: return ClusterHost<16, R>::launch(k, pl, in, isc, out, osc, st);
    case 32: return ClusterHost<32, R>::launch(k, pl, in, isc, out, osc, st);
    case 64: return ClusterHost<64, R>::launch(k, pl, in, isc, out, osc, st);
    default: return cudaErrorInvalidValue;
    }
}

bool configure_cluster(safr_plan_s *pl)
{
    int dev = 0, cl = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&cl, cudaDevAttrClusterLaunch, dev) != cudaSuccess || !cl) {
        cudaGetLastError();
        return false;
    }
    void *k = cluster_kernel(pl);
    if (!k) return false;
    const bool ok = pl->precision == SAFR_FP64 ? configure_m<double>(pl, k) : configure_m<float>(pl, k);
    cudaGetLastError();
    return ok;
}

cudaError_t launch_cluster(safr_plan_s *pl, const void *in, const float *in_scales, void *out, float *out_scales,
                           cudaStream_t st)
{
    void *k = cluster_kernel(pl);
    if (!k) return cudaErrorInvalidValue;
    if (pl->trace) cudaEventRecord(pl->ev[0], st);
    const cudaError_t e = pl->precision == SAFR_FP64 ? launch_m<double>(k, pl, in, in_scales, out, out_scales, st)
                                                     : launch_m<float>(k, pl, in, in_scales, out, out_scales, st);
    if (pl->trace) {
        cudaEventRecord(pl->ev[1], st);
        pl->traced = 1;
    }
    return e;
}

}  // namespace safr
