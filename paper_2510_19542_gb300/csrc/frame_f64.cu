// Persistent frame kernel, FP64 storage and arithmetic, M = 8 .. 256 (larger
// FP64 grids use the three-pass schedule).
#include "frame_dispatch.cuh"

namespace safr {
using Frame2F64 = Frame2Table<double, double, double, 8, 16, 32, 64, 128, 256>;
bool frame2_configure_f64(safr_plan_s *pl, int nsm) { return Frame2F64::configure(pl, nsm); }
cudaError_t frame2_launch_f64(safr_plan_s *pl, const void *in, const float *isc, void *out, float *osc,
                              cudaStream_t st)
{
    return Frame2F64::launch(pl, in, isc, out, osc, st);
}
cudaError_t frame2_launch_frames_f64(safr_plan_s *pl, const void *in, const float *isc, void *out, float *osc, int n,
                                     cudaStream_t st)
{
    return Frame2F64::launch_frames(pl, in, isc, out, osc, n, st);
}
}  // namespace safr
