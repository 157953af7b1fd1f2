// Persistent frame kernel, FP16 storage (per-star / per-layer scales), FP32 arithmetic, M = 8 .. 1024.
#include "frame_dispatch.cuh"

namespace safr {
using Frame2F16 = Frame2Table<float, __half, __half, 8, 16, 32, 64, 128, 256, 512, 1024>;
bool frame2_configure_f16(safr_plan_s *pl, int nsm) { return Frame2F16::configure(pl, nsm); }
cudaError_t frame2_launch_f16(safr_plan_s *pl, const void *in, const float *isc, void *out, float *osc,
                              cudaStream_t st)
{
    return Frame2F16::launch(pl, in, isc, out, osc, st);
}
cudaError_t frame2_launch_frames_f16(safr_plan_s *pl, const void *in, const float *isc, void *out, float *osc, int n,
                                     cudaStream_t st)
{
    return Frame2F16::launch_frames(pl, in, isc, out, osc, n, st);
}
}  // namespace safr
