// Internal plan of the SAFR library: host-side geometry and the device
// buffers that one plan owns.  Not part of the C ABI.
#pragma once

#include <cuda_runtime.h>

#include <type_traits>
#include <vector>

#include "safr.h"

// timestamps a traced persistent-kernel frame records per CTA
#define SAFR_TRACE_MARKS 23

namespace safr {

// One star group of the split tomography (Section 3.3): all LGS stars, or all
// NGS stars.
struct Group {
    int kind = SAFR_NGS;
    int G = 0;
    std::vector<int> stars;  // star indices in geometry order
    std::vector<double> c;   // [L] cone coefficient c_l (Section 2)
    std::vector<double> sx;  // [G][L] alpha_g^x h_l / (c_l delta): shift in layer pixels
    std::vector<double> sy;  // [G][L]
    double alpha = 0;        // Tikhonov parameter of the group
    int b_row0 = 0;          // first B row of this group inside a column block
    bool resample = false;   // layers move from pitch c_l*delta to delta (metric output)
};

// Geometry of one group handed to the precompute kernel (device pointers).
struct PreGroupDev {
    int G, L, b_row0;
    double alpha;
    const double *sx, *sy;  // [G][L]
    const double *sw;       // [L] gamma_l^{1/2} / c_l
    const double *tau;      // [L] pi^2 / (c_l T)^2
};

// Per-group data the frame kernels need.
struct GroupDev {
    int G;
    int b_row0;
    int resample;
    int star[SAFR_MAX_GROUP_G];
};

// Everything the three frame kernels read, passed by value.
template <typename R>
struct FrameParams {
    using C = typename std::conditional<sizeof(R) == 8, double2, float2>::type;
    int M, P, L, G, Mh, o, ngroups, sumLG, logM;
    int lchunk;       // layers per inverse-FFT chunk in the column pass
    int rows_per_cta; // output rows per CTA in the inverse row pass
    int src_pairs;    // row pairs of smem per group in the inverse row pass
    R delta;
    R inv_M2;         // 1 / M^2 of IDFT2
    const void *in;
    const float *in_scales;
    void *out;
    float *out_scales;
    const C *B;       // [Mh][sumLG][M]
    C *w1;            // [G][P][Mh]     row spectra of the padded wavefronts
    C *w2;            // [ngroups][L][M][Mh]  layer spectra after the inverse column pass
    float *energy;    // [ngroups][L][Mh] Parseval partial sums (FP16 storage only)
    const C *tw;      // [M] exp(-2 pi i t / M) from host FP64
    const int *rs_i0; // [L][M] floor(M/2 + (p - M/2)/c_l), unwrapped (LGS group)
    const R *rs_w;    // [L][M] fractional part
    const unsigned char *mask; // [P][P] pupil mask (removeTT)
    const R *tt_w;    // [2][P][P] tip and tilt of the least-squares plane as linear functionals of psi
    const char *prefetch;      // B, prefetched into L2 by the first pass
    size_t prefetch_bytes;
    int star_tt[SAFR_MAX_G];   // 1: remove this star's tip/tilt
    GroupDev grp[2];
    int *status;
};

}  // namespace safr

struct safr_plan_s {
    int device = 0;
    int M = 0, P = 0, L = 0, G = 0, Mh = 0, o = 0;
    int precision = SAFR_FP32, output_metric = 0, mixed = 0, remove_tt = 0;
    double delta = 0, T = 0, beta = 0;
    double diameter = 0, obstruction = 0;  // pupil annulus (diameter <= 0: the whole P x P square)
    std::vector<double> h, gamma;
    safr_geometry geo{};  // the geometry as given; its arrays point into h and the geo_* vectors
    std::vector<double> geo_cn2, geo_dir_x, geo_dir_y;
    std::vector<int> geo_kind;
    int ngroups = 0;
    safr::Group grp[2];
    int sumLG = 0;
    int warnings = 0;
    int precomputed = 0;
    std::vector<int> star_tt;

    // launch shapes chosen at plan creation
    int lchunk = 1, rows_per_cta = 8, src_pairs = 4;
    int pdl = 1;  // programmatic dependent launch between the three passes
    int path = SAFR_PATH_AUTO;  // requested kernel schedule
    int fused_ok = 0;           // the persistent kernel fits this plan
    // persistent-kernel shapes (frame_impl.cuh)
    int f2_grid = 0, f2_stage_b = 0, f2_rt3 = 2, f2_tiles3 = 1, f2_n3 = 1, f2_cap3 = 1;
    int f2_st3[2] = {0, 0}, f2_nsrc3[2] = {0, 0};
    unsigned f2_off_rs = 0, f2_off_tw = 0, f2_off_b = 0, f2_off_d = 0, f2_off_s3 = 0, f2_off_xy = 0;
    size_t f2_smem = 0;
    int f2_rt_force = 0;        // phase-3 tile rows chosen by the autotuner (0: cost model)
    int f2_grid_force = 0;      // CTAs of the persistent kernel (0: one per SM)
    int f2_ck = 1;              // phase-2 columns per pass
    int f2_ck_allow = 1;        // 0: one column per pass (schedule choice)
    int f2_pdl = 1;             // launch with programmatic stream serialization (0: plain launch)
    int f2_frames_ok = 0;       // the several-frames instance has its shared-memory limit raised
    int autotuned = 0;          // 1 after safr_autotune
    // one-cluster kernel for grids up to 64 (cluster_impl.cuh)
    int cl_ok = 0;              // the one-cluster kernel fits this plan
    int cl_auto = 0;            // ... and SAFR_PATH_AUTO prefers it
    int cl_cs = 0, cl_ncol = 0, cl_slots1 = 0, cl_stage_b = 0;
    unsigned cl_off[11] = {0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0};
    size_t cl_smem = 0;
    int debug_skip_cta = -1;
    unsigned long long barrier_timeout_ns = 1000000000ull;  // 1 s
    int gmax = 16; // compile-time bound on stars per group of the column pass
    size_t smem_k1 = 0, smem_k2 = 0, smem_k3 = 0;
    int k1_rows = 8;

    // device memory owned by the plan
    void *d_B = nullptr;  // [Mh][sumLG][M], j in the warp-FFT order of freqorder.h
    size_t b_bytes = 0;
    void *d_w1 = nullptr, *d_w2 = nullptr;
    float *d_energy = nullptr;
    size_t ws_bytes = 0;
    void *d_tw = nullptr;
    int *d_rs_i0 = nullptr;
    void *d_rs_w = nullptr;
    unsigned char *d_mask = nullptr;
    double tt_n[6] = {0, 0, 0, 0, 0, 0};  // rows b and c of the removeTT normal-equation inverse
    std::vector<unsigned> mask_bits;      // [P][(P + 31) / 32] pupil mask, one bit per pixel
    unsigned *d_mask_bits = nullptr;
    void *d_tt_w = nullptr;
    void *d_twq = nullptr;     // [M + min(M, 32)] warp-FFT twiddles of the persistent kernel
    void *d_xy_hat = nullptr;  // [2][Mh][M] DFT2 of x and y on the pupil mask (frequency-domain removeTT), j permuted
    void *d_pm = nullptr;      // [G][P][2] per-row tip/tilt functionals
    unsigned long long *d_bar = nullptr; // grid barrier: arrival count, launch epoch
    unsigned long long *d_stamps = nullptr;  // [grid][SAFR_TRACE_MARKS] timestamps of traced fused frames
    double *d_pre = nullptr;  // shifts, sw, tau of both groups (precompute)
    unsigned char *d_polc = nullptr;  // POLC sample points on the output grid and the pupil (loop.cu)
    int loop_blend = 0;       // set by safr_loop_step around its persistent-kernel launch
    double loop_gain = 0;     // integrator gain of that launch
    const void *loop_polc_psi = nullptr;  // wavefronts of that launch's POLC phase (null: no phase 0)
    int *d_status = nullptr;
    void *d_in_stage = nullptr, *d_out_stage = nullptr;
    float *d_in_scales_stage = nullptr, *d_out_scales_stage = nullptr;
    size_t in_bytes = 0, out_bytes = 0;

    // learned spectral filter (learned.cu): device state, allocated on first use
    void *filter = nullptr;
    int filter_learned = 0;  // 1: B holds the learned filter's inverse

    // tracing
    int trace = 0;
    int traced = 0;
    cudaEvent_t ev[4] = {nullptr, nullptr, nullptr, nullptr};
};

namespace safr {
// Launchers (reconstruct.cu, precompute.cu).
cudaError_t launch_precompute(safr_plan_s *plan, cudaStream_t stream);
cudaError_t launch_frame(safr_plan_s *plan, const void *in, const float *in_scales, void *out,
                         float *out_scales, cudaStream_t stream);
safr_status configure_frame_kernels(safr_plan_s *plan);
int launches_per_frame(const safr_plan_s *plan);
bool configure_fused(safr_plan_s *plan);
cudaError_t launch_fused(safr_plan_s *plan, const void *in, const float *in_scales, void *out, float *out_scales,
                         cudaStream_t stream);
cudaError_t launch_fused_frames(safr_plan_s *plan, const void *in, const float *in_scales, void *out,
                                float *out_scales, int n, cudaStream_t stream);
void frame2_twiddles(int M, std::vector<double> &re, std::vector<double> &im);
void filter_free(safr_plan_s *plan);
void filter_invalidate(safr_plan_s *plan);  // the SVD basis is stale (the geometry changed)
void polc_table(const safr_plan_s *plan, std::vector<unsigned char> &bytes);
std::vector<double> pre_inputs(const safr_plan_s *plan);    // refresh.cpp
int containment_warnings(const safr_plan_s *plan);          // refresh.cpp
bool configure_cluster(safr_plan_s *plan);
cudaError_t launch_cluster(safr_plan_s *plan, const void *in, const float *in_scales, void *out, float *out_scales,
                           cudaStream_t stream);
// the schedule safr_reconstruct runs: the one-cluster kernel when the plan fits it and the path is
// SAFR_PATH_CLUSTER, or SAFR_PATH_AUTO on a plan small enough for it; else the persistent kernel
// when it fits and the path is not SAFR_PATH_PASSES; else the three passes
inline bool use_cluster(const safr_plan_s *plan)
{
    return plan->cl_ok && (plan->path == SAFR_PATH_CLUSTER || (plan->path == SAFR_PATH_AUTO && plan->cl_auto));
}
inline bool use_fused(const safr_plan_s *plan)
{
    return plan->fused_ok && !use_cluster(plan) && plan->path != SAFR_PATH_PASSES;
}
inline int path_in_use(const safr_plan_s *plan)
{
    return use_cluster(plan) ? SAFR_PATH_CLUSTER : (use_fused(plan) ? SAFR_PATH_FUSED : SAFR_PATH_PASSES);
}
}  // namespace safr
