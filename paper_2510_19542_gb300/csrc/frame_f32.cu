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
cudaError_t frame2_launch_frames_f32(safr_plan_s *pl, const void *in, const float *isc, void *out, float *osc, int n,
                                     cudaStream_t st)
{
    return Frame2F32::launch_frames(pl, in, isc, out, osc, n, st);
}
}  // namespace safr

namespace safr {
// The FP32 persistent kernel for grid size M (nullptr if M has no instance).
template <int... Ms>
static void *frame2_kernel_f32_of(int M)
{
    void *k = nullptr;
    ((k = (M == Ms) ? Frame2Inst<float, float, float, Ms>::kernel() : k), ...);
    return k;
}
void *frame2_kernel_f32(int M) { return frame2_kernel_f32_of<8, 16, 32, 64, 128, 256, 512, 1024>(M); }
}  // namespace safr
