// Persistent frame kernel, FP32 storage and arithmetic, M = 8 .. 1024.
#include "frame_dispatch.cuh"

namespace safr {
using Frame2F32 = Frame2Table<float, float, float, 8, 16, 32, 64, 128, 256, 512, 1024>;
bool frame2_configure_f32(safr_plan_s *pl, int nsm) { return Frame2F32::configure(pl, nsm); }
cudaError_t frame2_launch_f32(safr_plan_s *pl, const void *in, const float *isc, void *out, float *osc,
                              cudaStream_t st)
{
    return Frame2F32::launch(pl, in, isc, out, osc, st);
}
}  // namespace safr
