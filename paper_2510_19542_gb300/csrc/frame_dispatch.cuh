// Per-precision instantiation and dispatch of the persistent frame kernel:
// one instance per supported grid size M (compile-time FFT shapes).
#pragma once

#include "frame_impl.cuh"

namespace safr {

template <typename R, typename TIN, typename TOUT, int M>
struct Frame2Inst {
    // the one-column-per-pass kernel, and (M >= 512 only) the two-column one; each as one frame per
    // launch or as several frames per launch
    static void *kernel() { return (void *)k_frame2<M, R, TIN, TOUT, 1>; }
    static void *kernel_ck(int ck)
    {
        if constexpr (M >= 512)
            if (ck == 2) return (void *)k_frame2<M, R, TIN, TOUT, 2>;
        return kernel();
    }
    static void *kernel_frames_ck(int ck)
    {
        if constexpr (M >= 512)
            if (ck == 2) return (void *)k_frame2_frames<M, R, TIN, TOUT, 2>;
        return (void *)k_frame2_frames<M, R, TIN, TOUT, 1>;
    }
    static bool configure(safr_plan_s *pl, int nsm)
    {
        if (!Frame2Host<M, R>::configure(pl, nsm, kernel())) return false;
        // the other instances need the same shared-memory limit
        if (pl->f2_ck == 2 && !smem_limit_allows(kernel_ck(2), pl->f2_smem)) pl->f2_ck = 1;
        pl->f2_frames_ok = smem_limit_allows(kernel_frames_ck(pl->f2_ck), pl->f2_smem) ? 1 : 0;
        return true;
    }
    static cudaError_t launch(safr_plan_s *pl, const void *in, const float *isc, void *out, float *osc,
                              cudaStream_t st)
    {
        Frame2Params<R> fp = Frame2Host<M, R>::params(pl, in, isc, out, osc);
        void *args[] = {&fp};
        // one CTA per SM at most (configure), so every CTA of the grid is resident once the SMs are
        // free; launched as an ordinary kernel with programmatic stream serialization so that a frame
        // right after another one overlaps its launch and prologue with that frame's end (a
        // cooperative launch does not overlap).  The batch graph's concurrent chains launch without
        // it: there a frame's early CTAs, waiting for the frame before them, would hold SMs that the
        // other chains' frames could use (measured 2.5% slower on the 64-frame batch).
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3(pl->f2_grid);
        cfg.blockDim = dim3(frame2_threads(M));
        cfg.dynamicSmemBytes = pl->f2_smem;
        cfg.stream = st;
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
        attr[0].val.programmaticStreamSerializationAllowed = 1;
        cfg.attrs = attr;
        cfg.numAttrs = pl->f2_pdl ? 1 : 0;
        return cudaLaunchKernelExC(&cfg, kernel_ck(pl->f2_ck), args);
    }
    // `n` frames in one launch (contiguous arrays), launched like one frame
    static cudaError_t launch_frames(safr_plan_s *pl, const void *in, const float *isc, void *out, float *osc, int n,
                                     cudaStream_t st)
    {
        Frame2Params<R> fp = Frame2Host<M, R>::params(pl, in, isc, out, osc);
        int nf = n;
        void *args[] = {&fp, &nf};
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3(pl->f2_grid);
        cfg.blockDim = dim3(frame2_threads(M));
        cfg.dynamicSmemBytes = pl->f2_smem;
        cfg.stream = st;
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
        attr[0].val.programmaticStreamSerializationAllowed = 1;
        cfg.attrs = attr;
        cfg.numAttrs = pl->f2_pdl ? 1 : 0;
        return cudaLaunchKernelExC(&cfg, kernel_frames_ck(pl->f2_ck), args);
    }
};

// Walks the compile-time list of grid sizes.
template <typename R, typename TIN, typename TOUT, int... Ms>
struct Frame2Table;
template <typename R, typename TIN, typename TOUT>
struct Frame2Table<R, TIN, TOUT> {
    static bool configure(safr_plan_s *, int) { return false; }
    static cudaError_t launch(safr_plan_s *, const void *, const float *, void *, float *, cudaStream_t)
    {
        return cudaErrorInvalidValue;
    }
    static cudaError_t launch_frames(safr_plan_s *, const void *, const float *, void *, float *, int, cudaStream_t)
    {
        return cudaErrorInvalidValue;
    }
};
template <typename R, typename TIN, typename TOUT, int M0, int... Ms>
struct Frame2Table<R, TIN, TOUT, M0, Ms...> {
    static bool configure(safr_plan_s *pl, int nsm)
    {
        if (pl->M == M0) return Frame2Inst<R, TIN, TOUT, M0>::configure(pl, nsm);
        return Frame2Table<R, TIN, TOUT, Ms...>::configure(pl, nsm);
    }
    static cudaError_t launch(safr_plan_s *pl, const void *in, const float *isc, void *out, float *osc,
                              cudaStream_t st)
    {
        if (pl->M == M0) return Frame2Inst<R, TIN, TOUT, M0>::launch(pl, in, isc, out, osc, st);
        return Frame2Table<R, TIN, TOUT, Ms...>::launch(pl, in, isc, out, osc, st);
    }
    static cudaError_t launch_frames(safr_plan_s *pl, const void *in, const float *isc, void *out, float *osc, int n,
                                     cudaStream_t st)
    {
        if (pl->M == M0) return Frame2Inst<R, TIN, TOUT, M0>::launch_frames(pl, in, isc, out, osc, n, st);
        return Frame2Table<R, TIN, TOUT, Ms...>::launch_frames(pl, in, isc, out, osc, n, st);
    }
};

}  // namespace safr
