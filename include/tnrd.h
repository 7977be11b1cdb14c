/*
 * tnrd.h -- C ABI of the GB300 (sm_103a) TRDMD despeckling library, libtnrd.so.
 *
 * The method (Feng & Chen, "Speckle Reduction with Trained Nonlinear Diffusion
 * Filtering", Sec. 3.1, Eq. diffusionprocessfinal) runs T stages from u_0 = f:
 *
 *     u~_t = u_{t-1} - sum_{i<N_k} K_i^T phi_i^t(K_i^t u_{t-1})
 *     u_t  = (u~_t + sqrt(u~_t^2 + 8 (1+2 lam_t) lam_t f^2)) / (2 (1+2 lam_t))
 *
 * K_i is true 2-D convolution with the ksize x ksize filter k_i over the
 * half-sample symmetric padded image (edge pixel repeated), K_i^T its exact
 * transpose (the rotated-kernel convolution of Eq. diffusion, with the border
 * folded back), and phi_i(z) = sum_j w_ij exp(-(z - mu_j)^2 / (2 gamma^2)) with
 * mu_j = rbf_mu0 + j * rbf_delta.  The prox is Eq. subproblemGIdiv.
 *
 * Conventions for every entry point:
 *  - All array pointers are DEVICE pointers unless stated; the caller owns all
 *    memory.  Images are float32, row-major, `pitch` floats between rows
 *    (pitch >= W, pitch % 4 == 0, base pointers 16-byte aligned); a batch of N
 *    images of one size is contiguous with stride H * pitch floats.
 *  - Every call is asynchronous on `stream`, never synchronises the host, and
 *    launches nothing when it returns an error status.  Calls made from one
 *    host thread that fail leave a message for tnrd_last_error().
 *  - `workspace` is caller-allocated device scratch of at least the size that
 *    tnrd_workspace_size() returns for the same arguments; it may be reused
 *    between calls on the same stream.
 *  - Supported models: (ksize, nfilt) in {(3,4), (5,24), (7,48)}, nrbf <= 64,
 *    rbf_delta >= rbf_gamma > 0 (the RBF sum is evaluated over the 13 centres
 *    nearest to z; the dropped terms are below 1.4e-9 * max|w|).  Images need
 *    H >= ksize and W >= ksize; N == 0 is a no-op.
 */
#ifndef TNRD_H
#define TNRD_H

#include <stddef.h>
#include <cuda_runtime_api.h>

#if defined(__GNUC__)
#define TNRD_API __attribute__((visibility("default")))
#else
#define TNRD_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    TNRD_OK = 0,
    TNRD_ERR_INVALID_ARG = 1,   /* null pointer, bad size, pitch or alignment      */
    TNRD_ERR_UNSUPPORTED = 2,   /* (ksize, nfilt, nrbf, rbf spacing) not built      */
    TNRD_ERR_CUDA = 3,          /* a CUDA runtime call failed; see tnrd_last_error */
    TNRD_ERR_TIMEOUT = 4,       /* a bounded device-side wait expired              */
    TNRD_ERR_WORKSPACE = 5      /* workspace null or smaller than required          */
} tnrd_status;

/* How the stage is computed.  All give the same result within the stated
 * tolerances; FUSED and UNFUSED compute in FP32, the tensor-core variants run
 * the filter bank and its adjoint with TF32 / BF16 operands and FP32
 * accumulation, phi and the prox in FP32.  TNRD_ALGO_TC_TF32: the filter bank
 * and the adjoint run as tcgen05 implicit GEMMs with TF32 operands (u, the
 * filters and phi's outputs rounded to TF32, 10-bit mantissa); its error
 * against the FP64 result is larger than the FP32 paths' (see the tests).
 * TNRD_ALGO_TC_BF16: the same GEMMs with BF16 operands (8-bit mantissa, round
 * to nearest even) and FP32 accumulation; error larger again.
 * TNRD_ALGO_TC_TF32X3: the tensor-core GEMMs at FP32 accuracy: every operand x
 * is split into hi = tf32(x) and lo = tf32(x - hi) and each product taken as
 * lo*hi + hi*lo + hi*hi (three TF32 MMAs, FP32 accumulation; the dropped
 * lo*lo term is below 2^-22 of the product), so its error against the FP64
 * result is that of the FP32 paths (see the tests). */
typedef enum {
    TNRD_ALGO_FUSED = 0,      /* one kernel per stage, responses kept on chip      */
    TNRD_ALGO_UNFUSED = 1,    /* three kernels per stage, N_k response planes in HBM */
    TNRD_ALGO_TC_TF32 = 2,
    TNRD_ALGO_TC_BF16 = 3,
    TNRD_ALGO_TC_TF32X3 = 4
} tnrd_algo;

/* Data term (reaction force) of every stage of a model.  With
 * u~ = u_{t-1} - sum_i K_i^T phi_i(K_i u_{t-1}):
 *   TNRD_DATA_IDIV  despeckling (Eq. diffusionprocessfinal): u_t = prox of
 *                   G = lam <u^2 - 2 f^2 log u, 1> at u~ (Eq. subproblemGIdiv);
 *   TNRD_DATA_GAUSS TNRD Gaussian denoising (Sec. 2.2.1, G = 0, A = I):
 *                   u_t = u~ - lam (u_{t-1} - f);
 *   TNRD_DATA_PROJ  explicit despeckling step with projection (Eq.
 *                   diffusion_backP): u_t = max(u~ - (lam / u_{t-1})
 *                   (1 - f^2 / u_{t-1}^2), proj_c); requires f > 0.
 * A zero-initialised tnrd_params selects TNRD_DATA_IDIV. */
typedef enum {
    TNRD_DATA_IDIV = 0,
    TNRD_DATA_GAUSS = 1,
    TNRD_DATA_PROJ = 2
} tnrd_data_term;

/* Parameters of a T-stage model (Sec. 3.2: Theta_t = {lam_t, phi_i^t, k_i^t}). */
typedef struct {
    int T;                  /* number of stages, >= 1                              */
    int ksize;              /* filter side k (odd)                                 */
    int nfilt;              /* N_k filters per stage                               */
    int nrbf;               /* Gaussian RBFs per influence function                */
    float rbf_mu0;          /* centre of the first RBF                             */
    float rbf_delta;        /* spacing of the centres                              */
    float rbf_gamma;        /* RBF width gamma                                     */
    const float* filters;   /* device [T][nfilt][ksize][ksize], k[a][b] row-major  */
    const float* rbf_w;     /* device [T][nfilt][nrbf]                             */
    const float* lambda;    /* device [T], lam_t >= 0 (> 0 for tnrd_backward)      */
    int data_term;          /* tnrd_data_term; 0 (despeckling prox) when zeroed     */
    float proj_c;           /* projection floor c > 0 of TNRD_DATA_PROJ (paper: 1)  */
} tnrd_params;

typedef enum { TNRD_OP_FORWARD = 0, TNRD_OP_BACKWARD = 1 } tnrd_op;

/* Bytes of device workspace that `op` needs for N images of H x W (pitch in
 * floats).  `keep_stages` as in tnrd_forward.  Returns 0 on invalid arguments. */
TNRD_API size_t tnrd_workspace_size(tnrd_op op, const tnrd_params* params, int N, int H, int W,
                           int pitch, int keep_stages, tnrd_algo algo);

/* Forward cascade, Eq. diffusion with the stage of Eq. diffusionprocessfinal.
 *   f      [N][H][pitch]  noisy input (also u_0 and the data term's f)
 *   u      keep_stages != 0: [T+1][N][H][pitch] receives u_0 = f, u_1 .. u_T
 *                            (the checkpoints tnrd_backward needs);
 *          keep_stages == 0: [N][H][pitch] receives u_T only.
 * u must not overlap f.  Padding columns (W..pitch) of u_1..u_T are not
 * written; u_0 is a byte copy of f, padding included. */
TNRD_API tnrd_status tnrd_forward(const tnrd_params* params, int N, int H, int W, int pitch,
                         const float* f, float* u, int keep_stages, tnrd_algo algo,
                         void* workspace, size_t workspace_bytes, cudaStream_t stream);

/* Describes the stage kernel tnrd_forward would launch for this shape and
 * algo (kernel name, tile geometry and, for the fused stages, how the haloed
 * u_{t-1} tile reaches shared memory: "tma staging" -- a bulk tensor copy, the
 * out-of-image halo mirrored in shared memory -- or "gather staging" when
 * TNRD_TMA=0), as a NUL-terminated string of at most
 * len - 1 characters written to buf.  Host-only: launches nothing.  Returns
 * TNRD_ERR_INVALID_ARG for a null or empty buf, otherwise the status
 * tnrd_forward's parameter checks would return. */
TNRD_API tnrd_status tnrd_forward_kernel(const tnrd_params* params, int N, int H, int W,
                                         tnrd_algo algo, char* buf, size_t len);

/* Gradients of a loss L through the cascade (Sec. 3.2, Eq. iterstep), for the
 * images of a batch summed (the loss of Eq. learning sums over samples).
 *   u_stages  [T+1][N][H][pitch] from tnrd_forward(keep_stages = 1)
 *   grad_uT   [N][H][pitch] dL/du_T (u_T - u_gt for the loss of Eq. learning)
 * Outputs (overwritten, not accumulated):
 *   grad_u0      [N][H][pitch] dL/du_0 along the state path, f held fixed
 *                in the data term (nullable: not computed)
 *   grad_filters [T][nfilt][ksize][ksize]  dL/dk (raw coefficients)
 *   grad_rbf_w   [T][nfilt][nrbf]           dL/dw
 *   grad_lambda  [T]                         dL/dlam (dL/dbeta = lam dL/dlam
 *                for lam = e^beta, Eq. derv5)
 * Requires lam_t > 0.  algo: TNRD_ALGO_FUSED (every kernel on the CUDA cores,
 * FP32), TNRD_ALGO_TC_TF32X3 (the adjoint dL/du_{t-1} = d + sum_i K_i^T c_i
 * of Eq. derv1-1 as a tensor-core GEMM on split TF32 operands, FP32 accuracy;
 * the rest as FUSED) or TNRD_ALGO_TC_TF32 (the same adjoint, and the filter
 * gradient dL/dk as a tensor-core GEMM over the pixels, with TF32 operands;
 * error larger, see the tests); others are TNRD_ERR_UNSUPPORTED.  A tensor-core
 * wait that gave up sets the word tnrd_device_status reads.  The parameter
 * gradients are reduced in a fixed order: repeated calls give identical bits. */
TNRD_API tnrd_status tnrd_backward(const tnrd_params* params, int N, int H, int W, int pitch,
                          const float* f, const float* u_stages, const float* grad_uT,
                          float* grad_u0, float* grad_filters, float* grad_rbf_w,
                          float* grad_lambda, tnrd_algo algo,
                          void* workspace, size_t workspace_bytes, cudaStream_t stream);

/* ---- Batched forward over images of different sizes ---------------------
 * A plan describes a fixed batch: every image with its own size, input and
 * output buffers and one of several parameter sets (e.g. one per number of
 * looks L).  With TNRD_ALGO_FUSED, tnrd_batch_forward runs all T stages of all
 * images either in ONE persistent kernel launch -- CTAs take (stage, image,
 * tile) items from a stage-major queue; a tile of stage t waits until the 3 x 3
 * neighbouring tiles of its image have finished stage t-1 (each wait bounded,
 * see tnrd_plan_set_wait_limit) -- or in one launch per stage over all images'
 * tiles, or in one launch per stage over tiles of the column-pair kernel (two
 * z-columns per lane, 64 - 2R columns per tile, a cluster of two CTAs per
 * tile), whichever the autotuner measured faster (tnrd_plan_launches,
 * tnrd_plan_tile_width; the persistent launch without autotune).  The first
 * two give the same bits; the third the bits of tnrd_forward's column-pair
 * kernel at the same tile height.
 * With TNRD_ALGO_TC_TF32 / _BF16 / _TF32X3 it runs one
 * tensor-core launch per stage over all images' tiles (mixed precision as in
 * tnrd_forward).  The launches are recorded in a CUDA graph at plan creation
 * and replayed by tnrd_batch_forward. */
typedef struct {
    const float* f;     /* device [H][pitch] noisy input (u_0)                 */
    float* u;           /* device [H][pitch] receives u_T; must not overlap f   */
    int H, W, pitch;    /* pitch in floats, multiple of 4, >= W                 */
    int param_set;      /* index into the plan's parameter sets                */
} tnrd_image;

typedef struct tnrd_plan tnrd_plan;

/* Creates a plan for `nimg` images (host array, copied) and `nsets` parameter
 * sets (host array of tnrd_params with device arrays, copied; all sets must
 * share T, ksize, nfilt, nrbf).  algo: TNRD_ALGO_FUSED, _TC_TF32, _TC_BF16 or
 * _TC_TF32X3
 * (TNRD_ALGO_UNFUSED is not batched).  This is the one
 * call that allocates device memory (work lists, per-tile stage counters, the
 * inter-stage images, a status word).  With autotune != 0 it times each
 * compiled tile height (and, for TNRD_ALGO_FUSED, all three schedules) on the
 * actual images (running the forward, which writes the outputs) on `stream`
 * and keeps the fastest; otherwise a size heuristic picks the tile height.
 * Synchronises `stream`. */
TNRD_API tnrd_status tnrd_plan_create(tnrd_plan** plan, const tnrd_image* images, int nimg,
                                      const tnrd_params* sets, int nsets, tnrd_algo algo,
                                      int autotune, cudaStream_t stream);

/* Runs the planned batch on `stream` (asynchronous; graph replay, or a direct
 * launch when `stream` is being captured).  Device-side failures (a wait that
 * hit its limit) are reported by tnrd_plan_status, not here. */
TNRD_API tnrd_status tnrd_batch_forward(const tnrd_plan* plan, cudaStream_t stream);

/* Synchronous: TNRD_OK, or TNRD_ERR_TIMEOUT if a tile of the last
 * tnrd_batch_forward gave up waiting for its neighbours (persistent schedule),
 * for the bulk tensor copy of its u_{t-1} tile (per-stage schedule) or, in
 * tensor-core plans, for its tensor-core operations (its outputs are then
 * incomplete). */
TNRD_API tnrd_status tnrd_plan_status(const tnrd_plan* plan);

/* Bound, in SM clock cycles, on each wait of a tile for its neighbours
 * (default 2e9, about one second).  0 makes every wait give up at once, which
 * tests the error path.  Synchronous. */
TNRD_API tnrd_status tnrd_plan_set_wait_limit(tnrd_plan* plan, long long cycles);

/* Tile height the plan uses (tensor-core plans: 16 NB - 2 (ksize / 2), NB = 2
 * for TF32 and 3 for BF16), and its tile width: 32 - 2 (ksize / 2), or
 * 64 - 2 (ksize / 2) for the column-pair schedule.  0 for a null plan. */
TNRD_API int tnrd_plan_tile_height(const tnrd_plan* plan);
TNRD_API int tnrd_plan_tile_width(const tnrd_plan* plan);

/* Kernel launches per tnrd_batch_forward of the plan: 1 for the persistent
 * schedule, T for one launch per stage (tensor-core plans, and fused plans
 * whose autotuner found that schedule faster). */
TNRD_API int tnrd_plan_launches(const tnrd_plan* plan);

/* Frees the plan's device memory and graph (synchronous). */
TNRD_API void tnrd_plan_destroy(tnrd_plan* plan);

/* Quality indexes of Sec. 4 for N images of H x W (pitch in floats), FP64
 * results in out (device, [N][TNRD_QUALITY_COUNT] doubles, in this order):
 *   psnr    10 log10(peak^2 / mean (ref - img)^2)
 *   mssim   mean SSIM over the 11 x 11 windows inside the image (Gaussian
 *           weights, sigma 1.5, summing to 1; C1 = (0.01 peak)^2,
 *           C2 = (0.03 peak)^2; windowed variance E[x^2] - mean^2); NaN when
 *           H or W < 11
 *   ec      correlation coefficient of the 3 x 3 Laplacians [0 1 0; 1 -4 1; 0 1 0]
 *           of ref and img (half-sample symmetric borders)
 *   ri_mean, ri_var   mean and population variance of the ratio image noisy / img
 *   cv      population standard deviation over mean of img
 * ref (nullable: psnr, mssim and ec are NaN) and img are [N][H][pitch]; noisy
 * (nullable: ri_mean and ri_var are NaN) likewise, with img > 0 where it is
 * given.  peak is the intensity range (255 on the [0, 255] scale).  The sums
 * are FP64 in a fixed order (repeatable bits).  Workspace: at least
 * tnrd_quality_workspace_size(N, H, W) bytes. */
#define TNRD_QUALITY_COUNT 6
TNRD_API size_t tnrd_quality_workspace_size(int N, int H, int W);
TNRD_API tnrd_status tnrd_quality(const float* ref, const float* img, const float* noisy, int N,
                                  int H, int W, int pitch, float peak, double* out,
                                  void* workspace, size_t workspace_bytes, cudaStream_t stream);

/* Largest batch (N * H * pitch floats) that tnrd_forward_noalloc accepts:
 * 4 Mi floats = 16 MiB, e.g. one 2048 x 2048 image or four 1024 x 1024. */
#define TNRD_NOALLOC_MAX_FLOATS (1u << 22)

/* Forward cascade for callers that cannot allocate device memory.  The paper
 * has no counterpart; this is a deployment convenience.  Some hosts own all
 * device memory and forbid a library from calling cudaMalloc (plugin and
 * media frameworks with a fixed memory budget, hard real-time loops where an
 * allocation may stall or fail), so they cannot supply tnrd_forward's
 * workspace.  This entry point computes exactly what
 * tnrd_forward(params, N, H, W, pitch, f, u, keep_stages = 0,
 * TNRD_ALGO_FUSED, ...) computes, with the image between stages held in a
 * scratch array built into the library instead of a caller workspace:
 *  - the array is TNRD_NOALLOC_MAX_FLOATS floats; every GPU that loads the
 *    library holds it until the process exits;
 *  - N * H * pitch above TNRD_NOALLOC_MAX_FLOATS returns TNRD_ERR_INVALID_ARG
 *    and launches nothing;
 *  - the first call on a device looks up the array's device address with
 *    that device current, and so does the first call in a new context of that
 *    device (after cudaDeviceReset the array may sit at another address); make
 *    that first call before any stream capture;
 *  - every call shares the one array, so calls that overlap on the GPU (two
 *    streams, two host threads) race and give wrong results: serialise them;
 *  - it calls no cudaMalloc, cudaFree or other allocating routine. */
TNRD_API tnrd_status tnrd_forward_noalloc(const tnrd_params* params, int N, int H, int W,
                                          int pitch, const float* f, float* u,
                                          cudaStream_t stream);

/* Synchronous: TNRD_OK, or TNRD_ERR_TIMEOUT if a stage launched since the
 * last call gave up waiting for its tensor-core operations or (fused stages)
 * for the bulk tensor copy of its u_{t-1} tile (bounded waits; the affected
 * tile's output is then not written).  Reading clears the device-side word. */
TNRD_API tnrd_status tnrd_device_status(void);

/* Test hook for the bounded waits of the fused stages' tile copies (the
 * one-column, pair and cluster-pair kernels of tnrd_forward) and of the grid
 * barriers between the stages of a small image's one-launch cascade: `cycles`
 * is the limit of each wait in SM cycles (default 2^31, about one second; >= 0;
 * a barrier wait that runs out records TNRD_ERR_TIMEOUT, the CTAs still run
 * every stage and barrier, and the output is not valid), and
 * never_complete != 0 arms each copy's mbarrier for 16 bytes more than the copy
 * brings, so that every wait runs out: each tile records TNRD_ERR_TIMEOUT (read
 * by tnrd_device_status), waits the limit once more for its copy still in
 * flight, and writes no output.  The copies themselves complete normally and
 * the context stays usable.  Process-wide, read when a launch is issued; not
 * for concurrent use.  TNRD_ERR_INVALID_ARG for a negative limit. */
TNRD_API tnrd_status tnrd_stage_wait_test(long long cycles, int never_complete);

/* Message describing the last error status returned on this host thread. */
TNRD_API const char* tnrd_last_error(void);

/* Library version, major * 10000 + minor * 100 + patch. */
TNRD_API int tnrd_version(void);

#ifdef __cplusplus
}
#endif
#endif /* TNRD_H */
