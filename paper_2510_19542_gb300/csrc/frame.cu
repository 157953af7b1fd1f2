// Host entry points of the persistent frame kernel: configuration at plan
// creation and the per-frame launch (with trace events).
#include <cuda_runtime.h>

#include "frame_impl.cuh"
#include "plan.h"

namespace safr {

bool frame2_configure_f32(safr_plan_s *pl, int nsm);
bool frame2_configure_f16(safr_plan_s *pl, int nsm);
bool frame2_configure_f64(safr_plan_s *pl, int nsm);
cudaError_t frame2_launch_f32(safr_plan_s *, const void *, const float *, void *, float *, cudaStream_t);
cudaError_t frame2_launch_f16(safr_plan_s *, const void *, const float *, void *, float *, cudaStream_t);
cudaError_t frame2_launch_f64(safr_plan_s *, const void *, const float *, void *, float *, cudaStream_t);
cudaError_t frame2_launch_frames_f32(safr_plan_s *, const void *, const float *, void *, float *, int, cudaStream_t);
cudaError_t frame2_launch_frames_f16(safr_plan_s *, const void *, const float *, void *, float *, int, cudaStream_t);
cudaError_t frame2_launch_frames_f64(safr_plan_s *, const void *, const float *, void *, float *, int, cudaStream_t);

void frame2_twiddles(int M, std::vector<double> &re, std::vector<double> &im) { frame2_twiddles_impl(M, re, im); }

bool configure_fused(safr_plan_s *pl)
{
    int dev = 0, nsm = 0, coop = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return false;
    if (cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return false;
    if (cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev) != cudaSuccess || !coop) return false;
    if (pl->f2_grid_force > 0 && pl->f2_grid_force < nsm) nsm = pl->f2_grid_force;  // safr_set_grid
    bool ok = false;
    if (pl->precision == SAFR_FP64)
        ok = frame2_configure_f64(pl, nsm);
    else if (pl->precision == SAFR_FP16_STORAGE)
        ok = frame2_configure_f16(pl, nsm);
    else
        ok = frame2_configure_f32(pl, nsm);
    cudaGetLastError();
    return ok;
}

cudaError_t launch_fused(safr_plan_s *pl, const void *in, const float *in_scales, void *out, float *out_scales,
                         cudaStream_t st)
{
    if (pl->trace) cudaEventRecord(pl->ev[0], st);
    cudaError_t e;
    if (pl->precision == SAFR_FP64)
        e = frame2_launch_f64(pl, in, in_scales, out, out_scales, st);
    else if (pl->precision == SAFR_FP16_STORAGE)
        e = frame2_launch_f16(pl, in, in_scales, out, out_scales, st);
    else
        e = frame2_launch_f32(pl, in, in_scales, out, out_scales, st);
    if (pl->trace) {
        cudaEventRecord(pl->ev[1], st);
        pl->traced = 1;
    }
    return e;
}

// n frames of the plan in one launch of the persistent kernel (contiguous arrays)
cudaError_t launch_fused_frames(safr_plan_s *pl, const void *in, const float *in_scales, void *out, float *out_scales,
                                int n, cudaStream_t st)
{
    if (pl->trace) cudaEventRecord(pl->ev[0], st);
    cudaError_t e;
    if (pl->precision == SAFR_FP64)
        e = frame2_launch_frames_f64(pl, in, in_scales, out, out_scales, n, st);
    else if (pl->precision == SAFR_FP16_STORAGE)
        e = frame2_launch_frames_f16(pl, in, in_scales, out, out_scales, n, st);
    else
        e = frame2_launch_frames_f32(pl, in, in_scales, out, out_scales, n, st);
    if (pl->trace) {
        cudaEventRecord(pl->ev[1], st);
        pl->traced = 1;
    }
    return e;
}

}  // namespace safr
