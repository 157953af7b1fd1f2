/*
 * safr.h -- C ABI of the GB300 (sm_103a) SAFR library.
 *
 * SAFR (Singular value-based Atmospheric tomography with Fourier domain
 * Regularization, arXiv 2510.19542) reconstructs L turbulence layers from G
 * guide-star wavefronts.  Per frame (Algorithm 1, "hard real-time"):
 *
 *     d_g    = DFT2(Psi_g)                       g = 1..G
 *     b_l(n) = sum_g B_lg(n) d_g(n)             every frequency n, l = 1..L
 *     Phi_l  = IDFT2(b_l)                         l = 1..L
 *
 * with DFT2 unnormalised and IDFT2 carrying 1/M^2 (Section 3.2).  B is the
 * block-diagonal-in-frequency matrix of Eq. (sparseM), precomputed once per
 * geometry (Algorithm 2, "soft real-time"):
 *
 *     A_n[g][l] = s_l(n) exp(i pi n.(alpha_g h_l) / (c_l T))     (Section 3.1)
 *     s_l(n)    = gamma_l^{1/2} / c_l (1 + tau_l |n|^2)^{-beta/2}, tau_l = pi^2/(c_l T)^2
 *     B_n       = diag(s(n)) R_alpha(A_n),  R_alpha = V g_alpha(Sigma^T) U^H,
 *     g_alpha(s)= s / (s^2 + alpha)                                   (Tikhonov)
 *
 * Mixed LGS + NGS asterisms use split tomography (Section 3.3, Algorithm 3):
 * the tip/tilt of each LGS wavefront is removed, the LGS group (c_l = 1 -
 * h_l/h_LGS) and the NGS group (c_l = 1, regularisation alpha_TT) are
 * reconstructed separately and the layers are added.
 *
 * Conventions (all arrays row-major, C order):
 *   - a wavefront Psi_g is P x P pupil samples, first index p <-> x, second
 *     q <-> y; it is zero-extended (Section 2) into the periodic M x M grid at
 *     offset o = (M-P)/2 on both axes;
 *   - the grid pitch is delta = 2T/M (Section 3.2); layer l of an LGS group is
 *     natively sampled at pitch c_l*delta (x^l_p = c_l x_p);
 *   - frequencies with |n_x| or |n_y| = M/2 (the Nyquist row and column of an
 *     even grid) are not reconstructed: B is zero there, which keeps the
 *     output real (the paper's symmetric truncation assumes odd M = 2m+1).
 *
 * Ownership: the plan owns B, its workspaces and its staging buffers (device
 * memory allocated in safr_plan_create).  The caller owns every buffer passed
 * to safr_reconstruct.  All device work is ordered on the caller's stream.
 *
 * Errors: argument errors are returned synchronously and nothing is launched.
 * Errors found on the device are recorded in the plan's sticky status word,
 * read by safr_get_status.  No call ever traps or spins without a bound.
 */
#ifndef SAFR_H
#define SAFR_H

#include <cuda_runtime_api.h>
#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct safr_plan_s *safr_plan_t;

typedef enum {
    SAFR_OK = 0,
    SAFR_ERR_INVALID_ARG = 1,      /* null pointer, bad size, bad geometry          */
    SAFR_ERR_UNSUPPORTED_SIZE = 2, /* M not a power of two in [8, 1024], L or G too large */
    SAFR_ERR_MISALIGNED = 3,       /* a device pointer not 16-byte aligned          */
    SAFR_ERR_NOT_PRECOMPUTED = 4,  /* safr_reconstruct before safr_precompute       */
    SAFR_ERR_OOM = 5,              /* cudaMalloc failed in safr_plan_create         */
    SAFR_ERR_CUDA = 6,             /* a CUDA runtime call failed (no device, launch) */
    SAFR_ERR_TIMEOUT = 7,          /* a bounded device-side wait gave up            */
    SAFR_ERR_DEVICE = 8,           /* a device-side check failed (see safr_get_status) */
    SAFR_ERR_IO = 9                /* a plan file could not be written or read, or is not a valid plan file */
} safr_status;

enum { SAFR_NGS = 0, SAFR_LGS = 1 };                           /* guide-star kind          */
enum { SAFR_FP32 = 0, SAFR_FP16_STORAGE = 1, SAFR_FP64 = 2 };  /* precision                */
enum { SAFR_NATIVE = 0, SAFR_METRIC = 1 };                     /* output grid              */

/* Limits of one plan. */
#define SAFR_MAX_M 1024
#define SAFR_MAX_L 64
#define SAFR_MAX_G 32       /* stars per plan                   */
#define SAFR_MAX_GROUP_G 16 /* stars per group (LGS or NGS)     */

/* Kernel schedules of safr_reconstruct (safr_set_path). */
enum {
    SAFR_PATH_AUTO = 0,    /* the one-cluster kernel on small plans (grids up to 64 whose last two
                              phases take one round of transforms per CTA), else the persistent
                              kernel when it fits, else the three passes                        */
    SAFR_PATH_FUSED = 1,   /* one persistent cooperative kernel with two grid barriers          */
    SAFR_PATH_PASSES = 2,  /* three kernels chained by programmatic dependent launch           */
    SAFR_PATH_CLUSTER = 3  /* grids up to 64: one thread-block cluster of up to 16 CTAs holds the
                              whole frame in shared memory; the CTAs exchange the row and column
                              spectra through distributed shared memory and two cluster barriers */
};

/* Warning bits of safr_plan_info.warnings. */
#define SAFR_WARN_CONTAINMENT 1 /* c_l Omega_A + alpha_g h_l is not inside c_l Omega_T (Section 2) */

/*
 * Telescope, asterism and atmosphere (Section 2).  Arrays are read during
 * safr_plan_create only (copied).
 */
typedef struct {
    int M;                 /* periodic grid size: power of two, 8 <= M <= 1024            */
    int P;                 /* pupil samples across, 1 <= P <= M                           */
    double pitch_m;        /* grid pitch delta = 2T/M in metres (T = M delta / 2)          */
    double diameter_m;     /* pupil diameter D (annulus mask: removeTT, learned-filter training); <= 0: square */
    double obstruction;    /* central obstruction as a fraction of D                      */
    int L;                 /* number of layers, 1 <= L <= SAFR_MAX_L                      */
    const double *h_m;     /* [L] layer heights, ascending, 0 <= h_l < h_lgs_m             */
    const double *cn2;     /* [L] layer weights gamma_l > 0; normalised to sum 1 here      */
    int G;                 /* number of guide stars, 1 <= G <= SAFR_MAX_G                 */
    const double *dir_x;   /* [G] direction vectors alpha_g^x (Section 2: (ax, ay, 1) points at the star) */
    const double *dir_y;   /* [G] alpha_g^y                                               */
    const int *kind;       /* [G] SAFR_NGS or SAFR_LGS                                    */
    double h_lgs_m;        /* sodium-layer height h_LGS (about 90 km)                     */
    double alpha;          /* Tikhonov parameter of the LGS group, or of the single group */
    double alpha_tt;       /* Tikhonov parameter of the NGS (tip-tilt star) group of a mixed plan */
    double beta;           /* Sobolev smoothness beta >= 0                                */
    int precision;         /* SAFR_FP32, SAFR_FP16_STORAGE or SAFR_FP64                   */
    int output_grid;       /* SAFR_NATIVE or SAFR_METRIC (mixed plans need SAFR_METRIC)    */
    int remove_tt;         /* mixed plans: remove LGS tip/tilt (Algorithm 3, line 3)      */
} safr_geometry;

typedef struct {
    int M, P, L, G;
    int ngroups;            /* 1 or 2 (LGS group first)                            */
    int group_kind[2];      /* SAFR_LGS / SAFR_NGS                                 */
    int group_G[2];         /* stars per group                                    */
    size_t b_bytes;         /* bytes of B on the device                           */
    size_t workspace_bytes; /* bytes of the inter-pass workspaces                 */
    size_t in_bytes;        /* bytes of one frame of wavefronts                   */
    size_t out_bytes;       /* bytes of one frame of layers                       */
    int warnings;           /* SAFR_WARN_* bits                                   */
    int precomputed;        /* 1 after safr_precompute                            */
    int path;               /* schedule safr_reconstruct uses: SAFR_PATH_CLUSTER, _FUSED or _PASSES */
    int tile_rows;          /* output rows per phase-3 item of the persistent kernel */
    int autotuned;          /* 1 after safr_autotune                              */
} safr_plan_info;

/*
 * Validate the geometry (Section 2: ascending heights below h_LGS, weights
 * gamma_l > 0; P <= M), split the stars into an LGS and an NGS group
 * (Section 3.3), derive c_l, the per-(star, layer) shifts alpha_g h_l /
 * (c_l delta) and the resample tables, and allocate B and the workspaces on
 * `cuda_device`.  On success *out is a new plan; on failure *out is NULL and
 * nothing stays allocated.  A mixed plan with SAFR_NATIVE output is rejected.
 * Besides the limits above, the three-pass kernels, which every plan keeps as
 * its fallback schedule, must fit in one SM's shared memory: their column pass
 * holds (3 Gmax + 1) M complex values (Gmax = stars in the larger group), so at
 * M = 1024 a group may have at most 9 stars in FP32 and 4 in FP64, and the
 * resampling pass of a mixed FP64 plan does not fit at M = 1024.  Such a shape
 * returns SAFR_ERR_UNSUPPORTED_SIZE.
 */
safr_status safr_plan_create(const safr_geometry *geom, int cuda_device, safr_plan_t *out);

/*
 * Algorithm 2: compute B for every stored frequency of every group on the
 * GPU in FP64 (stored in FP32, or FP64 for SAFR_FP64).  The regularised
 * inverse is evaluated as diag(s) A^H (A A^H + alpha I)^{-1}, which equals
 * diag(s) V g_alpha(Sigma^T) U^H for the Tikhonov filter (Section 3.1).
 * Asynchronous on `stream`; re-run it whenever alpha, gamma or the asterism
 * changes (the soft real-time step of Section 3.2).
 */
safr_status safr_precompute(safr_plan_t plan, cudaStream_t stream);

/*
 * Algorithm 1 (plus removeTT and the group sum of Algorithm 3 for mixed
 * plans) on device buffers.  Asynchronous on `stream`, no host
 * synchronisation, no allocation.
 *
 *   d_wavefronts [G][P][P]: float (SAFR_FP32), __half (SAFR_FP16_STORAGE) or
 *                double (SAFR_FP64), stars in the geometry's order.
 *   d_in_scales  [G] float or NULL: SAFR_FP16_STORAGE only; Psi_g = value * scale_g
 *                (NULL means 1).
 *   d_layers     [L][M][M]: float, __half or double.  Layer l is sampled at
 *                pitch c_l*delta (SAFR_NATIVE, single group) or delta (SAFR_METRIC).
 *   d_out_scales [L] float: SAFR_FP16_STORAGE only (required there);
 *                Phi_l = value * scale_l, scale_l a power of two chosen from the
 *                layer's energy (Parseval).
 * Every pointer must be 16-byte aligned device memory.
 */
safr_status safr_reconstruct(safr_plan_t plan, const void *d_wavefronts, const float *d_in_scales,
                             void *d_layers, float *d_out_scales, cudaStream_t stream);

/*
 * n frames of one plan (Algorithm 1 for each; the paper reconstructs one frame
 * at a time and has no counterpart of the multi-frame launch).  The arrays are
 * contiguous: d_wavefronts [n][G][P][P], d_layers [n][L][M][M], d_in_scales
 * [n][G], d_out_scales [n][L] (FP16 storage), element types as for
 * safr_reconstruct; frame f's layers are exactly those safr_reconstruct gives
 * for frame f.  On the persistent kernel the n frames run in ONE launch, one
 * after the other, each CTA starting the next frame as soon as it has finished
 * the last phase of the previous one (no launch, no prologue wait between
 * frames); the plan's workspaces serve every frame.  On the other schedules the
 * frames are launched one by one, and every frame's buffers must then be
 * 16-byte aligned (SAFR_ERR_MISALIGNED otherwise, nothing launched).  The base
 * pointers must be 16-byte aligned device memory.  Asynchronous on `stream`,
 * no allocation, no host synchronisation.  SAFR_ERR_INVALID_ARG for n < 1 or a
 * NULL buffer; errors as safr_reconstruct otherwise.
 */
safr_status safr_reconstruct_frames(safr_plan_t plan, int n, const void *d_wavefronts, const float *d_in_scales,
                                    void *d_layers, float *d_out_scales, cudaStream_t stream);

/*
 * End-to-end form of safr_reconstruct for host buffers, synchronising
 * `stream` before returning.  When every buffer is page-locked, mapped host
 * memory (cudaHostAlloc, cudaHostRegister) aligned to 16 bytes, the kernels
 * read the frame from `h_wavefronts` (and `h_in_scales`) and write the layers
 * (and scales) to `h_layers` / `h_out_scales` in place over the host link
 * (NVLink-C2C on Grace), with no staging copies.  Otherwise the frame is
 * copied to plan-owned device staging buffers, reconstructed, and copied
 * back; pageable memory works that way.
 */
safr_status safr_reconstruct_host(safr_plan_t plan, const void *h_wavefronts, const float *h_in_scales,
                                  void *h_layers, float *h_out_scales, cudaStream_t stream);

/*
 * Sticky device-side status of the plan (synchronises the plan's device).
 * Reading a non-OK status clears it and re-arms the plan's grid barrier.
 */
safr_status safr_get_status(safr_plan_t plan);

/* Sizes, groups and warnings of a plan (host only, no synchronisation). */
safr_status safr_get_plan_info(safr_plan_t plan, safr_plan_info *info);

/*
 * Copy group `group`'s B to host memory as complex FP64 pairs (re, im),
 * layout [k][l][g][j] for k in [0, M/2), l in [0, L), g over the group's stars
 * in geometry order, j in [0, M): entry B_lg at frequency (j, k), the n(j),
 * n(k) labels of Section 3.2.  `dst` holds 2*(M/2)*L*G_group*M doubles.
 * Synchronises the plan's device.  For inspection and tests.
 */
safr_status safr_copy_B(safr_plan_t plan, int group, double *dst);

/*
 * Per-phase timing of the next calls: when `enable` is non-zero,
 * safr_reconstruct records CUDA events around each of its kernels on its
 * stream.  safr_trace_read synchronises on the last recorded event and
 * writes up to `n` kernel durations in milliseconds of the last traced call:
 * one for SAFR_PATH_FUSED (the whole frame), three for SAFR_PATH_PASSES
 * (pad+row FFT, column FFT+apply+inverse column FFT, inverse row
 * FFT+resample+store; traced calls run them without programmatic overlap);
 * returns the number of durations in *n_out.
 */
safr_status safr_trace(safr_plan_t plan, int enable);
safr_status safr_trace_read(safr_plan_t plan, float *ms, int n, int *n_out);

/*
 * Inside the last traced SAFR_PATH_FUSED frame, in microseconds from the
 * first CTA's start (read from %globaltimer), the time the last CTA reached
 * each of 23 marks (0 for a mark no CTA reached):
 *    0 start                          12 phase 2: first inverse transforms done
 *    1 prologue issued                13 phase 2: layer spectra stored
 *    2 phase 1: frame data in         14 phase 2 done
 *    3 phase 1: B copy issued         15 grid barrier 2: arrival
 *    4 phase 1: first row transforms  16 grid barrier 2: released
 *    5 phase 1 done                   17 phase 3: resample tables ready
 *    6 grid barrier 1: arrival        18 phase 3: source rows staged
 *    7 grid barrier 1: released       19 phase 3: row transforms done
 *    8 phase 2: star transforms done  20 phase 3: block synchronised
 *    9 phase 2: spectra synchronised  21 phase 3: first item stored
 *   10 phase 2: B block landed        22 phase 3 done
 *   11 phase 2: first apply done
 * (marks 2-4, 8-13 and 17-21 are taken on the CTA's first batch, column or
 * item).  For a SAFR_PATH_CLUSTER frame the marks are:
 *    0 start                          7 phase 2: first column done
 *    1 prologue issued                8 phase 2 done
 *    2 phase 1: frame data in         9 cluster barrier 2 passed
 *    3 phase 1 done                  10 phase 3: first round transformed
 *    4 cluster barrier 1 passed      11 phase 3 done
 *    5 phase 2: star transforms done 12 last cluster barrier passed
 *    6 phase 2: B landed             13 bulk copies issued (thread 0)
 *                                    15 phase 3: first round stored
 * and marks 14, 16-22 are 0.  Writes up to `n` values; *n_out = 23.
 * SAFR_ERR_INVALID_ARG if there is no traced persistent-kernel or one-cluster
 * frame.
 */
safr_status safr_trace_phases(safr_plan_t plan, double *us, int n, int *n_out);

/*
 * The raw timestamps of the last traced persistent-kernel or one-cluster frame: us[b * 23 + i]
 * = mark i of CTA b in microseconds from the earliest CTA start (0 where the
 * CTA never reached the mark), for the n_cta CTAs of the launch; writes at
 * most n values, *n_cta = the grid size.  Errors as safr_trace_phases.
 */
safr_status safr_trace_stamps(safr_plan_t plan, double *us, int n, int *n_cta);

/* Number of kernel launches one safr_reconstruct makes for this plan. */
int safr_launches_per_frame(safr_plan_t plan);

/*
 * Choose the kernel schedule of the next calls (SAFR_PATH_*).  Every schedule
 * computes the same layers.  SAFR_PATH_FUSED on a plan the persistent kernel
 * cannot hold, or SAFR_PATH_CLUSTER on a plan the one-cluster kernel cannot
 * hold (grids above 64, or shared memory), returns SAFR_ERR_UNSUPPORTED_SIZE
 * and leaves the choice as it was.  safr_get_path returns the schedule that
 * safr_reconstruct will use (SAFR_PATH_CLUSTER, SAFR_PATH_FUSED or
 * SAFR_PATH_PASSES), or -1 for a NULL plan.
 */
safr_status safr_set_path(safr_plan_t plan, int path);

/*
 * CTAs of the persistent kernel (the paper fixes no launch shape): 0 (the
 * default) is one per SM; a smaller grid leaves SMs free for another frame's
 * kernel on another stream, and each phase's work is shared among the CTAs
 * launched.  Values above the SM count mean one per SM.  The layers do not
 * depend on it.  SAFR_ERR_UNSUPPORTED_SIZE (choice unchanged) when the plan
 * has no persistent kernel or its shape does not fit the grid.
 * safr_get_grid returns the CTAs of the next launch (0 for NULL).
 */
safr_status safr_set_grid(safr_plan_t plan, int ctas);
int safr_get_grid(safr_plan_t plan);
int safr_get_path(safr_plan_t plan);

/*
 * Output rows per phase-3 item of the persistent kernel (the paper fixes no
 * tiling): 0 (the default) lets the cost model choose; an even value from 2
 * to min(32, M) forces it (safr_autotune sets it the same way).  The layers
 * depend on it only through rounding: rows are paired into complex
 * transforms from the top of each tile.  SAFR_ERR_INVALID_ARG for any other
 * value; SAFR_ERR_UNSUPPORTED_SIZE (choice unchanged) when the plan has no
 * persistent kernel or the tile does not fit in shared memory.
 * safr_get_plan_info reports the height in use (tile_rows).
 */
safr_status safr_set_tile_rows(safr_plan_t plan, int rows);

/*
 * Test hook for the bounded grid barrier of SAFR_PATH_FUSED: with cta >= 0,
 * that CTA leaves the next frames before the first barrier, so every other
 * CTA's wait runs out after timeout_s seconds and the kernel records
 * SAFR_ERR_TIMEOUT (read by safr_get_status) instead of hanging.  cta = -1
 * restores normal operation; timeout_s <= 0 restores the default limit (1 s).
 * The frames computed meanwhile are invalid.
 */
safr_status safr_debug_skip_barrier(safr_plan_t plan, int cta, double timeout_s);

/*
 * No counterpart in the paper: a deployment form of safr_reconstruct for
 * callers that cannot call cudaMalloc.  Examples are a hard-real-time
 * control thread (an allocation may synchronise the device and has no
 * latency bound), a plugin inside a host framework that hands out all device
 * memory from its own pool, or software whose rules forbid dynamic allocation
 * after start-up.  A plan allocates B, its tables and its workspaces, so such
 * callers cannot create one.  This entry point needs no plan and allocates
 * nothing: no cudaMalloc, no cudaFree, no allocating library routine.
 *
 * It runs the FP32 persistent frame kernel for ONE star group with native
 * output: all NGS, or all LGS with layers at pitch c_l*delta.  There is no
 * removeTT, no resample and no second group.  The caller owns every buffer:
 *   d_B          [M/2][L*G][M] float2 (16-byte aligned): B_lg at frequency
 *                (j, k) in row l*G + g of column block k, for k < M/2, at
 *                position pos(j) of the row: the values safr_copy_B returns
 *                for the group, rounded to FP32, in the frame kernel's
 *                frequency order.  With LW = min(M, 32), R = M / LW and
 *                brev(m) the reversal of the log2(LW) bits of m:
 *                pos(j) = (j mod R) * LW + brev(j div R);
 *   d_wavefronts [G][P][P] float (16-byte aligned);
 *   d_layers     [L][M][M] float (16-byte aligned), sampled at pitch c_l*delta;
 *   d_status     one int (device memory), which the caller sets to 0.  A
 *                bounded device-side wait that gives up writes a non-zero
 *                safr_status (SAFR_ERR_TIMEOUT) there.  It is never cleared.
 * The kernel's scratch is a file-scope device array of
 * SAFR_NOALLOC_SCRATCH_BYTES: the grid-barrier counters, the twiddle table,
 * the row spectra (G*(M/2)*P complex) and the layer spectra (L*(M/2)*M
 * complex), each rounded up to 256 bytes.  A size that does not fit returns
 * SAFR_ERR_UNSUPPORTED_SIZE, before anything is launched.  So does a shape
 * the kernel cannot hold.  Every GPU that loads the library holds the array
 * until the process exits.
 *
 * The first call on a device looks up the array's device address
 * (cudaGetSymbolAddress, with that device current); make that first call
 * before any stream capture.  The first call with a given (device, M, P, L,
 * G) also sizes the kernel's launch (kernel attributes and occupancy
 * queries); later calls with that shape reuse it from a fixed table of 32
 * shapes and make no query.  Launch failures are returned as SAFR_ERR_CUDA
 * from the launch calls' own status; an error the caller had pending is
 * neither read nor cleared.  Every call on a device shares the one array,
 * and each call re-initialises the parts that must start from zero.  Calls
 * that overlap on the GPU (other streams, or other threads) race on it and
 * give wrong layers.  Asynchronous on `stream`; argument errors are returned
 * synchronously with nothing launched.
 */
#define SAFR_NOALLOC_SCRATCH_BYTES (8u << 20) /* 8 MiB */
safr_status safr_reconstruct_noalloc(int cuda_device, int M, int P, int L, int G, const void *d_B,
                                     const float *d_wavefronts, float *d_layers, int *d_status,
                                     cudaStream_t stream);

/*
 * Schedule autotuner (the paper has no counterpart; its algorithm fixes no
 * kernel schedule).  Times every candidate schedule of the plan on `stream`:
 * the persistent kernel with each feasible phase-3 tile height (output rows
 * per item), and the three-pass schedule.  Keeps the fastest (read back by
 * safr_get_plan_info: path, tile_rows).  The result is cached for the process
 * per device and plan shape (M, P, L, stars per group, precision, removeTT,
 * resample), so later plans of the same shape are not timed again.  A set-up
 * call: it allocates timing buffers, synchronises `stream` and overwrites the
 * plan's workspaces.  The layers it produces differ only by rounding.
 */
safr_status safr_autotune(safr_plan_t plan, cudaStream_t stream);

/*
 * Batched frames (the paper has no counterpart; it reconstructs one frame at
 * a time): frame i is reconstructed by plans[i], and the plans may differ in
 * geometry, precision and schedule.  Every frame's launches (its persistent
 * kernel, or its three passes) are captured once into ONE CUDA graph, and each
 * call replays it with a single graph launch, so the frames run back to back
 * with no host submission between them.  The graph holds the frames' buffer
 * pointers and schedules: a call with other pointers, or after a plan's
 * schedule changed (safr_autotune, safr_set_path), captures it again.  If a
 * capture fails the frames are launched one by one on the stream.  The layers
 * are exactly those of safr_reconstruct for each frame.
 *
 * safr_batch_create: `plans` [n] are borrowed (they must outlive the batch,
 * be precomputed before safr_batch_reconstruct, and not be reconstructed
 * concurrently on another stream, since the frames use their plans'
 * workspaces); allocates a capture stream.
 * safr_batch_reconstruct: arrays of n pointers, as for safr_reconstruct
 * (d_in_scales / d_out_scales may be NULL when no plan uses FP16 storage);
 * asynchronous on `stream`, no host synchronisation.  A capture (first call,
 * new pointers) makes the call slower on the host.
 * safr_batch_get_status: sticky device status of the batch's plans
 * (synchronises and clears them, as safr_get_status).
 * safr_batch_launches: kernel launches one safr_batch_reconstruct makes.
 * safr_batch_graph: 1 if the last call ran as a graph launch.
 */
typedef struct safr_batch_s *safr_batch_t;
safr_status safr_batch_create(const safr_plan_t *plans, int n, safr_batch_t *out);
safr_status safr_batch_reconstruct(safr_batch_t batch, const void *const *d_wavefronts,
                                   const float *const *d_in_scales, void *const *d_layers,
                                   float *const *d_out_scales, cudaStream_t stream);
safr_status safr_batch_get_status(safr_batch_t batch);
int safr_batch_launches(safr_batch_t batch);
int safr_batch_graph(safr_batch_t batch);
/* Concurrent chains of the batch's graph: frames of grids up to 256 on the
 * persistent kernel may run K at a time, each on 1/K of the SMs (one-cluster
 * frames keep their cluster), with the larger frames first on the whole GPU.  K in {1, 2, 4, 8} is chosen at the
 * first capture by timing each graph (that call replays the batch a few times
 * on its own stream and synchronises); the layers do not depend on K.
 * Returns 0 before the first call. */
int safr_batch_chains(safr_batch_t batch);
/* Force the chain count K of the next captures (1, 2, 4 or 8), or 0 to choose
 * it again by timing at the next capture; the next call captures the graph
 * again.  A batch with fewer than two concurrent frames (or a plan that appears
 * twice) keeps one chain whatever is asked.  SAFR_ERR_INVALID_ARG for other
 * values or a NULL batch. */
safr_status safr_batch_set_chains(safr_batch_t batch, int chains);
safr_status safr_batch_destroy(safr_batch_t batch);

/*
 * Learned spectral filter.  Section 3.1 writes the regularised inverse as
 * B(n) = diag(s) V g(Sigma) U^H for any regularising filter g of the singular
 * values of A(n) = U Sigma V^H (its experiments use Tikhonov,
 * g(s) = s / (s^2 + alpha)).  Here the filter factor phi in (0, 1) of singular
 * direction r in layer l comes from a small MLP of four features:
 *
 *   x = (|n| / (M/2), h_l / 20 km, (log10 sigma_r + 4) / 4, noise level / 0.05)
 *   phi = logistic(W3 gelu(W2 gelu(W1 gelu(W0 x + b0) + b1) + b2) + b3)
 *   B_lg(n) = s_l(n) sum_r V_lr(n) (phi / sigma_r) conj(U_gr(n))
 *
 * (phi = 1 gives the pseudo-inverse, phi = sigma^2 / (sigma^2 + alpha)
 * Tikhonov).  Hidden width 64, GELU in its exact erf form.  The parameters
 * are BF16 on the GPU and the arithmetic FP32; the SVD of every A(n) is FP64.
 * Parameter layout, SAFR_FILTER_PARAMS floats, row-major W[out][in]:
 *   W0[64][4], b0[64], W1[64][64], b1[64], W2[64][64], b2[64], W3[64], b3.
 * Only plans with one star group (no split tomography) take a learned filter
 * (SAFR_ERR_UNSUPPORTED_SIZE otherwise), and the plan must be precomputed.
 * The frame kernels are unchanged: only B is replaced.
 */
#define SAFR_FILTER_PARAMS 8705

typedef struct {
    double r0;          /* Fried parameter of the whole profile [m] of the training screens */
    double L0;          /* outer scale [m] */
    double noise_level; /* per-pixel noise std as a fraction of the noise-free wavefront RMS */
    int train_frames;   /* distinct training frames (drawn again each epoch) */
    int valid_frames;   /* held-out frames judging learned against plain SAFR */
    int epochs;
    double lr;          /* Adam learning rate */
    unsigned long long seed;
} safr_filter_config;

typedef struct {
    double train_loss_first;   /* relative squared layer error on the first training frames, initial weights */
    double train_loss_last;    /* the same after training */
    double valid_loss_learned; /* relative squared layer error on the held-out frames, learned filter */
    double valid_loss_plain;   /* the same with plain SAFR's Tikhonov filter */
    long steps;                /* Adam steps (256 frames each) */
    int used_learned;          /* 1: B now holds the learned filter's inverse */
    int nonfinite;             /* 1: the MLP gave a non-finite weight */
} safr_filter_result;

/*
 * safr_filter_train: trains the MLP on the GPU.  Training frames follow the
 * layered model of Section 2 through the aperture: layer spectra phi_l of
 * von Karman screens (cfg r0, L0, the plan's Cn2 weights and layer periods),
 * the noise-free data spectrum c_g(n) = sum_l exp(i theta_gl(n)) phi_l(n),
 * the wavefront psi_g = IDFT2(c_g) restricted to the plan's pupil (the P x P
 * square at offset (M - P)/2, masked by the annulus when a diameter is
 * given), plus white noise on the pupil pixels with a std of
 * cfg->noise_level x the RMS of the masked noise-free wavefront (per frame
 * and star), and d_g = DFT2 of that.  Random numbers come from
 * Philox4x32-10 (Salmon et al., SC 2011) and Box-Muller: frame F takes
 * phi_l(n), n = (j, k) with k < M/2, from counter (F, k M + j, l, 0), the
 * row k = 0 holding conjugate pairs (j > M/2 is the conjugate of M - j), and
 * the noise at grid pixel (p, q) of star g from the first normal of counter
 * (F, p M + q, g, 1).  Training frames use key (seed mod 2^32,
 * (seed >> 32) xor 0x5AFE), held-out frames key (seed mod 2^32 + 1,
 * (seed >> 32) xor 0x5AFE).  E|phi_l(n)|^2 = M^4 PSD_l(|n| / (2 c_l T)) /
 * (2 (2 c_l T)^2), half the power per complex coefficient of a real screen.
 * Training needs M <= 64 (SAFR_ERR_UNSUPPORTED_SIZE otherwise).  Frames are
 * processed 256 at a time, so held-out frames are taken in multiples of 256
 * (indices wrap modulo valid_frames).  The loss is
 * the relative squared error of the reconstructed
 * layer spectra, minimised by Adam (FP32 master weights, BF16 copy used by
 * the MLP) over ceil(train_frames / 256) * epochs steps of 256 frames.
 * Held-out frames (another key) then compare the learned filter with plain
 * SAFR: B becomes the learned filter's inverse only if its held-out error is
 * lower and every weight it gives is finite; otherwise plain SAFR's B is
 * rebuilt (the fallback).  weights_out [SAFR_FILTER_PARAMS] (may be NULL)
 * receives the trained parameters rounded to BF16; res (may be NULL) the
 * figures above.  Synchronises `stream`; allocates the filter's buffers on
 * first use (freed with the plan).
 *
 * safr_filter_apply: builds B from given parameters (host, rounded to BF16)
 * at noise level `noise_level`.  If the MLP gives a non-finite weight, plain
 * SAFR's B is rebuilt and SAFR_ERR_DEVICE returned.  Synchronises `stream`.
 *
 * safr_filter_reset: rebuilds plain SAFR's B (as safr_precompute).
 */
safr_status safr_filter_train(safr_plan_t plan, const safr_filter_config *cfg, float *weights_out,
                              safr_filter_result *res, cudaStream_t stream);
safr_status safr_filter_apply(safr_plan_t plan, const float *weights, double noise_level, cudaStream_t stream);
safr_status safr_filter_reset(safr_plan_t plan, cudaStream_t stream);

/*
 * The steps of the three-step AO loop around SAFR (Algorithm 3): pseudo open
 * loop control (line 2) and the integrator (line 5).  The mirror/layer state
 * a is L layers on the plan's output grid, [L][M][M] in the plan's precision
 * (FP32 or FP64; plans with FP16 storage return SAFR_ERR_UNSUPPORTED_SIZE),
 * the same layout safr_reconstruct writes.  Wavefront reconstruction from
 * sensor data (CuReD) and the two-step delay of the loop are the caller's.
 *
 * safr_polc: psi~_g = psi_g + A_g a on the pupil, zero off it (the zero
 * extension of Section 2), with the tomography operator of Section 2,
 * (A_g a)(r) = sum_l a_l(c_l r + alpha_g h_l), evaluated matrix-free by
 * bilinear interpolation of the layer samples (the O(N) evaluation of the
 * paper's cost analysis).  For star g, layer l and pupil pixel (p, q) the
 * sample point in output-grid pixels is, per axis,
 *   native output grid:  u = o + p + s_gl
 *   metric output grid:  u = M/2 + c_l (o + p - M/2 + s_gl)
 * with s_gl = alpha_g h_l / (c_l delta), o = (M - P)/2, wrapped periodically
 * onto [0, M).  d_wavefronts and d_out are [G][P][P] (geometry star order)
 * and may not overlap d_a; d_out may equal d_wavefronts.
 *
 * safr_integrate: a <- (1 - gain) a + gain Phi over the L M^2 samples,
 * 0 <= gain <= 1.
 *
 * safr_loop_step: one loop iteration on the plan's staging buffers: POLC of
 * d_wavefronts with the current state d_a, SAFR (safr_reconstruct, with the
 * LGS tip/tilt removal of a mixed plan), then the integrator into d_a.
 * All three are asynchronous on `stream` and launch kernels only.
 */
safr_status safr_polc(safr_plan_t plan, const void *d_wavefronts, const void *d_a, void *d_out,
                      cudaStream_t stream);
safr_status safr_integrate(safr_plan_t plan, const void *d_layers, void *d_a, double gain, cudaStream_t stream);
safr_status safr_loop_step(safr_plan_t plan, const void *d_wavefronts, void *d_a, double gain,
                           cudaStream_t stream);

/*
 * Soft real-time refresh (Algorithm 2; Section 3.4: B is recomputed whenever
 * parameters at the telescope or in the atmosphere change, e.g. guide-star
 * positions or the turbulence profile).  safr_refresh sets new layer weights
 * (cn2 [L], normalised to sum 1 as at creation), new star directions
 * (dir_x, dir_y [G], both or neither; the kinds of the stars are kept) and
 * new regularisation parameters (alpha, alpha_tt; <= 0 keeps the current
 * value).  NULL arrays keep the current values.  Layer heights, grid, pupil and
 * star kinds cannot change (create a new plan).  The derived tables are
 * copied into the plan's existing buffers and B is recomputed in place on
 * `stream`: no allocation, and frames issued later on the same stream use the
 * new B.  A learned filter's B is replaced by plain SAFR's (train or apply
 * it again).  Argument errors are returned before anything changes.
 */
typedef struct {
    const double *cn2;   /* [L] or NULL */
    const double *dir_x; /* [G] or NULL */
    const double *dir_y; /* [G] or NULL */
    double alpha;        /* > 0 to change */
    double alpha_tt;     /* > 0 to change */
} safr_update;
safr_status safr_refresh(safr_plan_t plan, const safr_update *update, cudaStream_t stream);

/*
 * Plan files.  safr_plan_save writes the plan's geometry and its B (as
 * stored on the device, so a learned filter's B is kept) to `path`;
 * synchronises the plan's device.  safr_plan_load reads such a file, creates
 * the plan on `cuda_device` and uploads B without recomputing it; the new
 * plan is precomputed.  Format (little-endian, packed):
 *   char[8] "SAFRPLN1", u32 version = 1,
 *   i32 M, P, L, G, precision, output_grid, remove_tt, learned (1: B is a learned filter's),
 *   f64 pitch_m, diameter_m, obstruction, h_lgs_m, alpha, alpha_tt, beta,
 *   f64 h_m[L], cn2[L], dir_x[G], dir_y[G], i32 kind[G],
 *   u64 FNV-1a-64 of every byte above (the geometry hash),
 *   u64 n, n bytes of B ([M/2][sum_groups L G_group][M] complex in the plan's
 *   B precision, j in the frame kernels' order), u64 FNV-1a-64 of those n bytes.
 * A file that cannot be read or written, a wrong magic, version, size or
 * hash returns SAFR_ERR_IO; the file is checked before any device work.  A
 * geometry that safr_plan_create rejects returns its status.
 */
safr_status safr_plan_save(safr_plan_t plan, const char *path);
safr_status safr_plan_load(const char *path, int cuda_device, safr_plan_t *out);

/* Free every device and host resource of the plan (synchronises its device). */
safr_status safr_destroy(safr_plan_t plan);

/* Static, human-readable name of a status code. */
const char *safr_status_string(safr_status status);

#ifdef __cplusplus
}
#endif

#endif /* SAFR_H */
