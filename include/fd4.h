/*
 * fd4 -- multi-scale anisotropic fourth-order diffusion (MAFOD) on one GPU.
 *
 * C ABI of the GB300 (sm_103a) library.  The method is the filter of
 * Gorgi Zadeh, Didas, Wintergerst and Schultz, "Multi-Scale Anisotropic
 * Fourth-Order Diffusion Improves Ridge and Valley Localization"
 * (arXiv:1611.06906); section and equation numbers below refer to it.
 *
 * Conventions shared by every entry point
 *   - Images are single-channel float32, row-major; pixel (x, y) of an image
 *     with row pitch `pitch` (in elements) is p[y * pitch + x], x the column.
 *     Every per-pixel array of one call (image, scale index map, tensor field,
 *     V map) uses the same `pitch`, counted in elements of its own type.
 *     pitch >= w and pitch % 4 == 0 (16-byte rows); device pointers 16-byte
 *     aligned.  Minimum image size is 3 x 3.
 *   - Names starting with d_ are device pointers, h_ host pointers.
 *   - The caller owns every buffer.  Entry points never allocate memory;
 *     scratch comes from a caller-provided workspace d_ws of at least
 *     fd4_workspace_bytes(...) bytes (256-byte aligned).  A workspace may be
 *     reused by later calls on the same stream, not by concurrent ones.
 *   - All device work is enqueued on `stream` (NULL = legacy default stream)
 *     and is asynchronous; the functions return once it is enqueued.
 *   - Return value: FD4_OK (0) or a negative fd4_status.  Argument errors are
 *     detected on the host before anything is enqueued.  FD4_ERR_CUDA means
 *     a CUDA runtime call failed; cudaGetLastError() is left set.
 *   - The parity tolerance the library is tested to (max-abs 1e-4 against an
 *     FP64 evaluation of the same method) assumes intensities in [0, 1].
 */
#ifndef FD4_H
#define FD4_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* A cudaStream_t (the runtime's stream handle); NULL is the legacy stream. */
typedef struct CUstream_st *fd4_stream_t;

typedef enum fd4_status {
    FD4_OK = 0,
    FD4_ERR_BAD_ARG = -1,          /* null pointer, size or parameter out of range  */
    FD4_ERR_UNSTABLE_TAU = -2,     /* 3T/(M(n^2+n)) > tau_max, or tau_max > 1/17    */
    FD4_ERR_TOO_MANY_SIGMAS = -3,  /* n_sigma > FD4_MAX_SIGMAS                      */
    FD4_ERR_PITCH = -4,            /* pitch < w or pitch % 4 != 0                   */
    FD4_ERR_WS_TOO_SMALL = -5,     /* ws_bytes < fd4_workspace_bytes(...)           */
    FD4_ERR_TIMEOUT = -6,          /* a bounded device-side wait gave up            */
    FD4_ERR_CUDA = -7,             /* a CUDA runtime call failed                    */
    FD4_ERR_ALIGN = -8,            /* device pointer not 16-byte aligned            */
    FD4_ERR_SIGMA_RANGE = -9,      /* sigma <= 0, sigma > FD4_MAX_SIGMA, unsorted   */
    FD4_ERR_NOT_IMPLEMENTED = -10
} fd4_status;

/* Which creases are enhanced (Sec. 3.2, the paragraph after Eq. 7) and which
 * polarity the vesselness accepts (Sec. 3.3, Eq. 9 and its valley analogue). */
typedef enum fd4_mode { FD4_RIDGE = 0, FD4_VALLEY = 1, FD4_BOTH = 2 } fd4_mode;

/* Boundary of the discrete operator (Sec. 3.4).  NATURAL: a derivative row
 * exists only where its 3x3 stencil fits in the image (per stencil); the
 * scheme then conserves the mean grey value.  PERIODIC: wrap-around, meant for
 * tests (the Fourier analysis of the biharmonic special case).              */
typedef enum fd4_boundary { FD4_BC_NATURAL = 0, FD4_BC_PERIODIC = 1 } fd4_boundary;

#define FD4_MAX_SIGMAS 32          /* scale-set size limit (uint8 index map)     */
#define FD4_MAX_SIGMA 12.0f        /* largest sigma: kernel radius ceil(4 sigma) <= 48 */
#define FD4_MAX_FED_STEPS 4096     /* longest FED cycle                          */

typedef struct fd4_params {
    float lambda;            /* contrast lambda of Eq. 7 (default 0.005)          */
    float rho;               /* integration scale of Eq. 6 (default 0.5)          */
    float beta;              /* Frangi beta of Eq. 9 (default 0.5)                */
    float c;                 /* Frangi c of Eq. 9; <= 0: half the maximum of S
                                over all scales and pixels of the image (default) */
    float gamma;             /* scale normalisation sigma^(2 gamma) (default 1)    */
    float tau_max;           /* stable explicit step (default 0.05, Sec. 3.5)      */
    int mode;                /* fd4_mode (default FD4_BOTH, Sec. 3.2)              */
    int boundary;            /* fd4_boundary (default FD4_BC_NATURAL)              */
    int kappa;               /* FED step ordering: 0 = automatic, else i -> kappa*i mod n */
    int grad_norm_squared;   /* 0: 1/sqrt(1+|grad|) as printed in Eq. 6 (default);
                                1: 1/sqrt(1+|grad|^2)                              */
    int fed_steps_per_launch;/* FED kernel schedule (no effect on the result beyond
                                FP32 rounding): 0 = library default (2),
                                1 = one launch per explicit step, 2..4 = that many
                                steps fused per launch (see fd4_autotune_batched) */
    int reselect_each_cycle; /* whole filters (fd4_filter, fd4_filter_batched,
                                fd4_graph_create): 0 = the scale image is selected
                                once, on the input (default); 1 = selected again
                                on the current image u^k before every cycle's
                                tensor build (the other reading of Eq. 21, where
                                sigma* is part of P(u^k)).  Ignored when the
                                caller gives the scale image.                    */
    int postprocess_scales;  /* whole filters: 0 = the scale image as selected
                                (default); 1 = every selection is followed by
                                the scale-image post-processing of Sec. 3.3 (see
                                fd4_postprocess_scales).  Ignored when the caller
                                gives the scale image.                           */
    float theta;             /* vesselness threshold of the post-processing's
                                vessel mask, in [0, 1] (default 0.2, the paper's
                                synthetic setting; 0.13 for its fundus images)   */
    int model;               /* whole filters: fd4_model (default FD4_MODEL_MAFOD) */
    float ifod_sigma;        /* FD4_MODEL_IFOD: the regularisation scale of
                                H(u_sigma) (default 1.0, the paper's setting;
                                at most FD4_MAX_SIGMA)                           */
    int fed_tile_rows;       /* FED schedule, 2 or 4 steps per launch under the
                                natural boundary: rows of the 64-column regions
                                a block advances in shared memory, 64 or 32
                                (0 = library default, 64)                        */
    int fed_quads_per_thread;/* FED schedule, as above: row quads (4 adjacent
                                pixels) each thread owns, 1 or 2 (0 = library
                                default, 2)                                      */
} fd4_params;

/* The filter a whole-filter call runs.  MAFOD: the paper's method (scale
 * selection, tensor D from N at the selected scales).  IFOD: its isotropic
 * fourth-order comparator (Eq. 2): D = g(|H(u_sigma)|_F^2) I with the
 * Perona-Malik g of Eq. 7 at the one scale ifod_sigma, rebuilt from u^k every
 * cycle, the same FED cycles; the scale set and scale image are not used (a
 * valid scale set is still required by the argument checks).               */
typedef enum fd4_model { FD4_MODEL_MAFOD = 0, FD4_MODEL_IFOD = 1 } fd4_model;

/* Fills *p with the defaults listed above. */
void fd4_default_params(fd4_params *p);

/* Human-readable name of a status code (static storage). */
const char *fd4_strerror(int status);

/* Library version as 10000*major + 100*minor + patch. */
int fd4_version(void);

/* FED step sizes (Sec. 3.5, Eq. 22-23), on the host in float64.
 *   n = ceil(-1/2 + 1/2 sqrt(1 + 12 T / (M tau_max)))  when n_in == 0, else n_in;
 *   tau_i = 3T / (2 M (n^2 + n) cos^2(pi (2i+1) / (4n+2))),  i = 0..n-1.
 * The paper reorders the steps with the kappa cycles of the FED authors'
 * code, which it does not print.  This library orders them as
 * tau_out[i] = tau_{kappa i mod n} with gcd(kappa, n) = 1.  kappa_in = 1 keeps
 * the natural order; kappa_in = 0 picks the kappa with the smallest
 * rounding-error growth bound
 *     A(kappa) = max_j max_p |prod_{l<j} (1 - tau_pi(l) p)| * max_q |prod_{l>=j} (1 - tau_pi(l) q)|
 * over p, q on 4096 points of [0, 34] (34 bounds the operator norm, Sec. 3.4),
 * ties to the smaller kappa.
 * tau_out: host array of tau_cap doubles; *n_out = n; kappa_out nullable.
 * Errors: BAD_ARG (T <= 0, M <= 0, tau_max <= 0, n_in < 0, kappa not coprime
 * to n, n > tau_cap or > FD4_MAX_FED_STEPS), UNSTABLE_TAU (tau_max > 1/17, or
 * n_in given with 3T/(M(n^2+n)) > tau_max).                                  */
int fd4_fed_taus(double T, int M, double tau_max, int n_in, int kappa_in,
                 double *tau_out, int tau_cap, int *n_out, int *kappa_out);

/* Workspace sizes.  op selects the entry point; the size covers a w x h image
 * with pitch roundup(w, 4) and n_sigma scales.                               */
typedef enum fd4_op {
    FD4_OP_SELECT_SCALES = 0,
    FD4_OP_BUILD_TENSOR = 1,
    FD4_OP_FED_CYCLE = 2,
    FD4_OP_FILTER = 3,
    FD4_OP_POSTPROCESS = 4,
    FD4_OP_CREASES = 5
} fd4_op;
size_t fd4_workspace_bytes(int op, int w, int h, int n_sigma);

/* Per-pixel scale selection (Sec. 3.3, Eq. 9).
 * For each sigma of h_sigmas (host, n_sigma values, strictly increasing, each
 * in (0, FD4_MAX_SIGMA]): the Hessian of u_sigma = u * G_sigma (sampled
 * Gaussian-derivative kernels of radius ceil(4 sigma), half-sample mirror
 * border), its eigenvalues scaled by sigma^(2 gamma) and ordered
 * |nu1| <= |nu2| (equal magnitudes: nu2 the negative one), S and R_B = nu1/nu2.
 * V = 0 for the wrong polarity (RIDGE: nu2 > 0, VALLEY: nu2 < 0), else
 * exp(-R_B^2/(2 beta^2)) (1 - exp(-S^2/(2 c^2))).  c = params->c if > 0, else
 * half the maximum of S over all scales and pixels.
 * Output d_sigma_idx[y*pitch+x] = argmax_s V (uint8, ties to the smaller
 * sigma); d_vmax (nullable, float) = the maximum V.
 * d_img: device float image.  params: host, nullable (defaults).           */
int fd4_select_scales(const float *d_img, int w, int h, int pitch,
                      const float *h_sigmas, int n_sigma, const fd4_params *params,
                      uint8_t *d_sigma_idx, float *d_vmax,
                      void *d_ws, size_t ws_bytes, fd4_stream_t stream);

/* Scale-image post-processing (Sec. 3.3, the paragraphs after Eq. 9), in place
 * on d_sigma_idx: the pixels whose vesselness d_vmax exceeds params->theta form
 * the vessel mask; each of them takes the scale of the set nearest to the mean
 * scale of its vessel cross-section.  The cross-section is traced from the
 * pixel along the eigenvector of the Hessian of u_sigma at the pixel's selected
 * scale that belongs to the eigenvalue of largest magnitude (the negative one
 * on a tie): the digital line with one pixel per unit step along its major
 * axis (minor coordinate rounded half up), walked both ways while it stays in
 * the image and the mask, at most ceil(4 sigma_max) pixels per side.  Pixels
 * outside the mask, pixels whose Hessian has equal eigenvalues and pixels
 * whose index is not < n_sigma keep their index; an index not < n_sigma also
 * ends a walk.  All pixels are updated from the scale image as given.
 *   d_u          image the scales were selected on, float32 (h, pitch)
 *   d_sigma_idx  uint8 (h, pitch): selected scale indices in, post-processed out
 *   d_vmax       float32 (h, pitch): max_sigma V_sigma (fd4_select_scales' v_max)
 *   workspace    fd4_workspace_bytes(FD4_OP_POSTPROCESS, pitch, h, n_sigma)
 * Errors as for fd4_select_scales; nothing is written on an error.          */
int fd4_postprocess_scales(const float *d_u, int w, int h, int pitch, uint8_t *d_sigma_idx,
                           const float *d_vmax, const float *h_sigmas, int n_sigma,
                           const fd4_params *params, void *d_ws, size_t ws_bytes, fd4_stream_t stream);

/* IFOD tensor field (Eq. 2): D = g I as (1, 0, g, g) per pixel with
 * g = 1 / (1 + |H(u_s)|_F^2 / lambda^2), |H|_F^2 = u_xx^2 + 2 u_xy^2 + u_yy^2
 * at s = params->ifod_sigma (Gaussian derivatives as in fd4_select_scales).
 * d_tensor: 4 floats per pixel, row pitch `pitch` pixels.  No workspace.    */
int fd4_build_tensor_ifod(const float *d_u, int w, int h, int pitch, const fd4_params *params,
                          float *d_tensor, fd4_stream_t stream);

/* Crease extraction (Sec. 4, ridge and valley extraction): the zero contour of
 * d = det(g | Hg), g the gradient and H the Hessian of u_s at s = sigma
 * (0 < sigma <= 4; derivatives as in fd4_select_scales), by marching squares on
 * the pixel grid.  Cell (i, j) has the corners (i, j), (i+1, j), (i+1, j+1),
 * (i, j+1) (x to the right, y down); a corner is inside where d > 0; edge
 * crossings are linearly interpolated; a saddle cell is resolved by the mean
 * of its corners (mean > 0: the inside corners are connected).  The zero set
 * of d is a superset of the creases: a cell's segments are kept where the
 * mean over its corners of the strongest Hessian eigenvalue (the one of
 * largest magnitude, the negative one on a tie) is negative (FD4_RIDGE),
 * positive (FD4_VALLEY) or non-zero (FD4_BOTH).
 *   d_segs   4 floats per segment (x0, y0, x1, y1, pixel units), 16-byte aligned
 *   d_keys   one int per segment: 2 * (j * (w - 1) + i) + k, k = 0 or 1 (a
 *            saddle cell has two segments), ordering the segments by cell
 *   d_count  one device int: the number of segments found (the first
 *            max_segs of them, in any order, are written)
 *   workspace fd4_workspace_bytes(FD4_OP_CREASES, pitch, h, 0)
 * Errors: FD4_ERR_BAD_ARG for sigma outside (0, 4], a bad mode, null outputs
 * or max_segs < 0, otherwise as for fd4_select_scales.                      */
int fd4_extract_creases(const float *d_u, int w, int h, int pitch, float sigma, int mode, float *d_segs,
                        int *d_keys, int max_segs, int *d_count, void *d_ws, size_t ws_bytes,
                        fd4_stream_t stream);

/* Fourth-order diffusion tensor field (Sec. 3.1 Eq. 6, Sec. 3.2 Eq. 7-8).
 * N = H(u_s) / sqrt(1 + |grad u_s|) at s = h_sigmas[d_sigma_idx[p]] per pixel
 * (|grad u_s|^2 under the root if params->grad_norm_squared), then
 * N_rho = G_rho * N componentwise (radius ceil(4 rho), mirror border), the
 * eigen-decomposition N_rho = nu1 e1 e1^T + nu2 e2 e2^T with nu1 >= nu2, and
 * mu_i = 1 / (1 + nu_i^2 / lambda^2), set to 1 where RIDGE and nu_i >= 0 or
 * VALLEY and nu_i <= 0.  D has eigentensors e1e1, e2e2, sym(e1e2),
 * antisym(e1e2) with eigenvalues mu1, mu2, (mu1+mu2)/2, 0.
 * Output d_tensor: 4 floats per pixel (cos 2t, sin 2t, mu1, mu2),
 * e1 = (cos t, sin t); (1, 0) where nu1 == nu2.  Row pitch `pitch` pixels
 * (4*pitch floats).  d_sigma_idx entries must be < n_sigma.               */
int fd4_build_tensor(const float *d_u, int w, int h, int pitch,
                     const uint8_t *d_sigma_idx, const float *h_sigmas, int n_sigma,
                     const fd4_params *params, float *d_tensor,
                     void *d_ws, size_t ws_bytes, fd4_stream_t stream);

/* One FED cycle (Sec. 3.5, Eq. 21): u <- (I - tau_{n-1} P) ... (I - tau_0 P) u
 * with P = L^T D L (Sec. 3.4, Eq. 17), Hajiaboli stencils at unit spacing,
 * D from d_tensor (as written by fd4_build_tensor) frozen over the cycle.
 * d_u is updated in place.  h_tau: host, n step sizes in execution order
 * (for instance from fd4_fed_taus); each step is applied exactly as given.
 * boundary: fd4_boundary.                                                   */
int fd4_fed_cycle(float *d_u, int w, int h, int pitch, const float *d_tensor,
                  const double *h_tau, int n, int boundary,
                  void *d_ws, size_t ws_bytes, fd4_stream_t stream);

/* fd4_fed_cycle with an explicit kernel schedule (no counterpart in the
 * paper): steps_per_launch, tile_rows and quads_per_thread as the fd4_params
 * fields of those names (0 = the library default).  Every schedule applies
 * the same steps; results differ by FP32 rounding only.  Errors as
 * fd4_fed_cycle, and FD4_ERR_BAD_ARG for a schedule outside those ranges.   */
int fd4_fed_cycle_sched(float *d_u, int w, int h, int pitch, const float *d_tensor,
                        const double *h_tau, int n, int boundary, int steps_per_launch, int tile_rows,
                        int quads_per_thread, void *d_ws, size_t ws_bytes, fd4_stream_t stream);

/* The whole filter (Sec. 3): step sizes from (T, M, n_in, params->tau_max,
 * params->kappa) as in fd4_fed_taus; sigma* once on the input (unless
 * sigma_given, in which case d_sigma_idx is read); then M cycles of
 * fd4_build_tensor on the current image followed by one fd4_fed_cycle.
 * Where the FED schedule runs the TMA kernel (2 or 4 steps per launch, the
 * natural boundary), each cycle's tensor build leaves, in the workspace, the
 * three coefficients that kernel reads -- (mu1 + mu2) / 2, q cos 2t and
 * q sin 2t with q = (mu1 - mu2) / 4 -- instead of the float4 field: the same
 * arithmetic, 12 instead of 16 bytes per pixel for the FED steps to read.
 * d_in is not modified; d_out receives the result (may equal d_in).
 * d_sigma_idx: nullable when !sigma_given (then kept in the workspace);
 * otherwise receives / supplies sigma*.                                     */
int fd4_filter(const float *d_in, float *d_out, int w, int h, int pitch,
               const float *h_sigmas, int n_sigma, const fd4_params *params,
               double T, int M, int n_in, uint8_t *d_sigma_idx, int sigma_given,
               void *d_ws, size_t ws_bytes, fd4_stream_t stream);

/* ------------------------------------------------------------------------ */
/* Batches: many images of uneven sizes, one persistent launch per stage.     */

typedef struct fd4_image {
    const float *d_in;       /* device input image (not modified unless == d_out) */
    float *d_out;            /* device output image; may equal d_in                */
    uint8_t *d_sigma_idx;    /* nullable unless sigma_given: receives / supplies sigma* */
    int w, h, pitch;         /* as for the single-image calls                      */
} fd4_image;

#define FD4_MAX_BATCH 65536

/* Workspace for fd4_filter_batched / fd4_graph_create on this list of images. */
size_t fd4_batch_workspace_bytes(const fd4_image *h_imgs, int n_images, int n_sigma);

/* fd4_filter on every image of the host array h_imgs (n_images entries), with
 * one launch per stage covering all images: each stage kernel walks a flat
 * list of tiles spanning the batch.  Results are those of fd4_filter on each
 * image separately (identical arithmetic per pixel).  Errors as fd4_filter;
 * every image is validated before anything is enqueued.  Without re-selection,
 * a cycle whose FED steps end in the workspace's FED plane leaves the current
 * image there and the next cycle starts from it, so d_out holds the result
 * once the stream has passed the call, not between cycles.                  */
int fd4_filter_batched(const fd4_image *h_imgs, int n_images, const float *h_sigmas, int n_sigma,
                       const fd4_params *params, double T, int M, int n_in, int sigma_given,
                       void *d_ws, size_t ws_bytes, fd4_stream_t stream);

/* The schedule of fd4_filter_batched (descriptor upload, selection, input
 * copy, M cycles of tensor build and FED cycle) captured once into a CUDA
 * graph and replayed by fd4_graph_launch.  `stages` selects what is captured:
 * FD4_STAGES_ALL for the filter; a subset replays only those stages on the
 * current workspace contents (for timing one stage: FD4_STAGE_FED alone runs
 * M FED cycles on the images with the tensor fields left by a previous run;
 * the scale-image post-processing, which reads the copied input, runs only
 * when FD4_STAGE_COPY is captured too).
 * The graph keeps the device pointers of h_imgs and d_ws: those buffers must
 * stay allocated while the graph exists; their contents are read at each
 * launch.  The host arrays may be freed after the call.                     */
#define FD4_STAGE_SELECT 1
#define FD4_STAGE_COPY 2
#define FD4_STAGE_TENSOR 4
#define FD4_STAGE_FED 8
#define FD4_STAGES_ALL 15
/* Option bit for fd4_graph_create with FD4_STAGES_ALL: capture the batch as two
 * image groups on two streams (balanced pixel counts), the second starting
 * after the first group's first tensor build, so the FMA-bound tensor builds
 * of one group overlap the latency-bound FED steps of the other.  Results are
 * identical to the one-stream graph.                                        */
#define FD4_GRAPH_TWO_STREAMS 16
typedef struct fd4_graph_st *fd4_graph;
int fd4_graph_create(const fd4_image *h_imgs, int n_images, const float *h_sigmas, int n_sigma,
                     const fd4_params *params, double T, int M, int n_in, int sigma_given, int stages,
                     void *d_ws, size_t ws_bytes, fd4_graph *out);
int fd4_graph_launch(fd4_graph g, fd4_stream_t stream);
/* Number of kernel launches one fd4_graph_launch performs (the kernel nodes
 * of the captured graph; every one is a kernel of this library).  No
 * counterpart in the paper: launch accounting for benchmarks.               */
int fd4_graph_kernel_count(fd4_graph g, int *n_kernels);
int fd4_graph_destroy(fd4_graph g);

/* One FED kernel schedule and its measured time (fd4_autotune_batched). */
typedef struct fd4_fed_schedule {
    int steps_per_launch;    /* as fd4_params.fed_steps_per_launch (1..4)      */
    int tile_rows;           /* as fd4_params.fed_tile_rows (64 or 32; 0 where
                                the schedule has no such choice)                */
    int quads_per_thread;    /* as fd4_params.fed_quads_per_thread (1 or 2; 0
                                where the schedule has no such choice)          */
    float ms;                /* time of one FED cycle over the batch            */
} fd4_fed_schedule;

#define FD4_AUTOTUNE_CANDIDATES 10

/* Autotuner for the FED kernel schedule (no counterpart in the paper): runs
 * the selection and one tensor build of the batch, then times one FED cycle
 * with each of the FD4_AUTOTUNE_CANDIDATES schedules -- 1 and 3 steps per
 * launch, and 2 and 4 steps per launch on regions of 64 or 32 rows with 1 or
 * 2 quads per thread (the halo depth is 2 pixels per step) -- with CUDA
 * events on `stream` (synchronising it), after one untimed cycle each; a
 * cycle is timed as the batched filter runs it, without a copy of the result
 * back into d_out.  *best receives the fastest; tried (nullable, FD4_AUTOTUNE_CANDIDATES
 * entries) every candidate with its time.  The schedule is copied into a
 * fd4_params by the caller.  The images' d_out buffers are overwritten.     */
int fd4_autotune_batched(const fd4_image *h_imgs, int n_images, const float *h_sigmas, int n_sigma,
                         const fd4_params *params, double T, int M, int n_in, void *d_ws, size_t ws_bytes,
                         fd4_stream_t stream, fd4_fed_schedule *best, fd4_fed_schedule *tried);

/* ------------------------------------------------------------------------ */
/* Learned scale selector.  No counterpart in the paper: a small network that
 * predicts the per-pixel scale index the vesselness argmax (Sec. 3.3) would
 * select, trained on labels the plain selection produces, with the plain
 * selection as fallback and reference.  Network: four dilated 3x3 convolutions
 * (dilations 1, 2, 4, 8; channels 1-32-32-32-16; zero padding), ReLU between
 * them, softmax over the first n_bins outputs (one bin per scale of the set,
 * 2 <= n_bins <= FD4_SELECTOR_MAX_BINS; the other outputs are unused).  BF16
 * weights and activations, FP32 accumulation on the tensor cores (tcgen05).
 * Parameters live in a caller-owned device buffer of
 * fd4_selector_param_bytes() bytes (256-byte aligned): FP32 master weights
 * (order: per layer W[ky][kx][co][ci] then b[co]), Adam moments, accumulated
 * gradients, and the BF16 kernel layouts derived from the master weights.
 * Image stacks are n_img images of w x h, row pitch `pitch`, image after image
 * (h * pitch floats apart).                                                  */
#define FD4_SELECTOR_MAX_BINS 16
size_t fd4_selector_param_bytes(void);
/* Workspace of fd4_selector_grad (training: every layer's input is kept). */
size_t fd4_selector_workspace_bytes(int n_img, int w, int h, int pitch);
/* Workspace of fd4_selector_forward and fd4_selector_predict (inference). */
size_t fd4_selector_infer_workspace_bytes(int n_img, int w, int h, int pitch);
/* He-normal weights from a seed, zero biases, zero moments (synchronous). */
int fd4_selector_init(void *d_params, unsigned long long seed, fd4_stream_t stream);
/* Master weights from / to the host (synchronous); which: 0 weights,
 * 1 and 2 Adam moments, 3 accumulated gradients.                            */
int fd4_selector_set_weights(void *d_params, const float *h_weights, fd4_stream_t stream);
int fd4_selector_get_weights(const void *d_params, float *h_weights, int which, fd4_stream_t stream);
/* Logits (n_bins floats per pixel, pixel layout of the stack) of every image. */
int fd4_selector_forward(const void *d_params, const float *d_imgs, int n_img, int w, int h, int pitch,
                         int n_bins, float *d_logits, void *d_ws, size_t ws_bytes, fd4_stream_t stream);
/* Forward and backward pass: adds the gradient of the mean cross-entropy of
 * the softmax over n_bins against d_labels (uint8 bin per pixel, stack
 * layout; labels >= n_bins count as n_bins - 1) to the accumulated gradients,
 * and the mean loss to *d_loss.                                             */
int fd4_selector_grad(void *d_params, const float *d_imgs, const uint8_t *d_labels, int n_img, int w, int h,
                      int pitch, int n_bins, float *d_loss, void *d_ws, size_t ws_bytes, fd4_stream_t stream);
/* Adam step (beta 0.9 / 0.999, eps 1e-8) on the accumulated gradients, which
 * are then cleared; step counts from 1.                                     */
int fd4_selector_update(void *d_params, float lr, int step, fd4_stream_t stream);
/* Scale index (argmax of the n_bins logits, ties to the smaller) and
 * confidence (its softmax probability, nullable) per pixel of every image of
 * the stack (one launch per layer for the whole stack); d_idx and d_conf in
 * the stack's pixel layout.                                                 */
int fd4_selector_predict(const void *d_params, const float *d_imgs, int n_img, int w, int h, int pitch, int n_bins,
                         uint8_t *d_idx, float *d_conf, void *d_ws, size_t ws_bytes, fd4_stream_t stream);
/* Learned selection with the plain selection as fallback and reference.  The
 * network predicts a scale index and a confidence (its softmax probability)
 * per pixel; every 32 x 64 tile whose least confident pixel is below
 * conf_threshold is recomputed with the plain vesselness selection
 * (fd4_select_scales restricted to those tiles).  Reading for the restricted
 * selection: c = half the maximum of S over the recomputed tiles (with every
 * tile recomputed this is exactly fd4_select_scales).  The network's bins are
 * the n_sigma scales (2 <= n_sigma <= FD4_SELECTOR_MAX_BINS); d_conf (nullable)
 * receives the confidences, d_n_fallback (nullable, device int) the number of
 * recomputed tiles.                                                         */
size_t fd4_select_learned_workspace_bytes(int w, int h, int pitch, int n_sigma);
int fd4_select_scales_learned(const void *d_params, const float *d_img, int w, int h, int pitch,
                              const float *h_sigmas, int n_sigma, const fd4_params *params, float conf_threshold,
                              uint8_t *d_sigma_idx, float *d_conf, int *d_n_fallback, void *d_ws,
                              size_t ws_bytes, fd4_stream_t stream);

/* Library-wide device status word of the FED kernels: FD4_ERR_TIMEOUT after a
 * bounded wait of the TMA-staged FED kernel on a tile's copies gave up (the
 * kernel then stops its work and returns), FD4_OK otherwise.  Synchronous
 * (waits for the device); reset != 0 clears it after reading.  No
 * counterpart in the paper: failure reporting of the device-side waits.     */
int fd4_device_status(int *status, int reset);

/* Device status word of a selector workspace (FD4_ERR_TIMEOUT if a bounded
 * wait in a tensor-core kernel gave up), read synchronously.                */
int fd4_selector_status(const void *d_ws, int *status, fd4_stream_t stream);

/* Failure-detection self-test (no counterpart in the paper): launches the
 * tensor-core convolution with its MMA commit withheld, so the kernel's
 * bounded wait (about one second) runs out; the kernel records
 * FD4_ERR_TIMEOUT in the workspace status word, frees its tensor memory and
 * returns, leaving the context usable.  *status receives the status word read
 * back (FD4_ERR_TIMEOUT when detection works).  Synchronous; d_ws needs
 * fd4_selector_workspace_bytes(1, 128, 4, 128) bytes.                       */
int fd4_selftest_wait_timeout(void *d_ws, size_t ws_bytes, int *status, fd4_stream_t stream);

/* FP32 FMA rate of the current GPU, measured (no counterpart in the paper):
 * the denominator of the fractions quoted for the FMA-bound kernels.  Times
 * a kernel of independent FMA chains on every SM in the scalar form and in
 * packed pairs (two FP32 lanes per instruction), best of three launches after
 * one warm-up, with CUDA events on `stream` (synchronous).  *scalar_tfma and
 * *pair_tfma receive the rates in 1e12 FMA/s.  d_scratch: device memory of at
 * least 8 x 4 x (the SM count) bytes (a sink the kernels never write).      */
int fd4_measure_fma_rate(void *d_scratch, size_t scratch_bytes, double *scalar_tfma, double *pair_tfma,
                         fd4_stream_t stream);

/* Failure-detection self-test of the FED kernels (no counterpart in the
 * paper): one launch of the TMA-staged FED kernel on the image d_u with the
 * tile copies withheld (the tile barrier is armed for bytes that never come)
 * and every bounded wait limited to 10 ms, so the first wait runs out; the
 * kernel records FD4_ERR_TIMEOUT in the device status word (fd4_device_status)
 * and returns without writing d_u, leaving the context usable.  *status
 * receives the status word read back with reset (FD4_ERR_TIMEOUT when
 * detection works).  No copy is ever in flight.  Synchronous; the workspace
 * is that of fd4_fed_cycle.                                                 */
int fd4_selftest_fed_wait_timeout(float *d_u, int w, int h, int pitch, const float *d_tensor, void *d_ws,
                                  size_t ws_bytes, int *status, fd4_stream_t stream);

/* Allocation-free FED cycle.  The paper has no counterpart: this entry point
 * exists for callers that cannot allocate device memory -- host applications
 * that own all device memory and pass a library only the buffers it works on,
 * and programs that must not call cudaMalloc after start-up (it can
 * synchronise the device, and some run under a no-allocation policy).  It
 * computes exactly what fd4_fed_cycle computes, with the same arguments minus
 * the workspace: its scratch plane is a static array inside the library,
 * FD4_NOALLOC_MAX_PIXELS floats (16 MiB) per GPU, held by every GPU that loads
 * the library until the process exits.
 *   - h * pitch must not exceed FD4_NOALLOC_MAX_PIXELS, else
 *     FD4_ERR_WS_TOO_SMALL (the built-in scratch is too small for the image).
 *   - The first call on a device looks up the scratch array's device address
 *     (with that device current) and caches it for the device's context; make
 *     that first call before any stream capture.  After a device reset
 *     (cudaDeviceReset) the next call finds a new context and looks the
 *     address up again, so it too should come before any capture.
 *   - All calls share the one scratch array, which keeps the last call's
 *     contents; nothing in it has to start at zero.  Calls whose work overlaps
 *     on the GPU (different streams, or different host threads on one device)
 *     race on it and must be serialised by the caller.
 *   - It calls no cudaMalloc, cudaFree or allocating library routine.        */
#define FD4_NOALLOC_MAX_PIXELS (4 * 1024 * 1024)
int fd4_fed_cycle_noalloc(float *d_u, int w, int h, int pitch, const float *d_tensor,
                          const double *h_tau, int n, int boundary, fd4_stream_t stream);

#ifdef __cplusplus
}
#endif
#endif /* FD4_H */
