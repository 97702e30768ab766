/*
 * gmr.h -- C ABI of the Gaussian Mesh Renderer hot path (CUDA, sm_103a).
 *
 * The library turns every triangle of a mesh into one planar 3D Gaussian
 * (paper Sec. 2.2, Eq. 3-16) and renders those Gaussians with 3DGS-style tile
 * rasterization (Sec. 2.1): EWA projection to the image plane, binning into
 * screen tiles sorted by (tile, depth, face index), and front-to-back alpha
 * compositing. The backward pass returns dL/d(vertex positions) and
 * dL/d(per-face or per-vertex colour, per-face opacity) from dL/d(image).
 *
 * Conventions for every entry point
 *  - Array arguments are DEVICE pointers unless stated otherwise, contiguous,
 *    FP32 (or int32 for indices), owned by the caller and never freed or
 *    retained by the library beyond what is stated.
 *  - Work is enqueued asynchronously on the given stream; outputs are valid
 *    once that stream reaches the call's end. A NULL stream is the legacy
 *    default stream.
 *  - Errors found on the host are returned at once and nothing is enqueued.
 *    Errors found on the device (face index out of range, pair buffer too
 *    small) set bits of a device status word that gmr_get_device_status()
 *    returns; no kernel traps, asserts or spins without bound.
 *  - A context is not thread-safe: use one context per host thread.
 *  - Images are packed view after view; view c occupies pixels
 *    [off[c], off[c+1]) of the packed buffer (see gmr_image_offsets), rows
 *    top to bottom, 3 floats (RGB) per pixel.
 *  - The kernels of one forward and one backward may be launched with
 *    programmatic dependent launch (each may start while the one before it
 *    on the stream finishes, and waits for it on the device before touching
 *    memory); the ordering the caller sees is plain stream order. Setting
 *    GMR_PDL=0 in the environment (read once per process) launches them
 *    without it.
 */
#ifndef GMR_H_
#define GMR_H_

#include <stdint.h>

#if defined(__GNUC__)
#define GMR_API __attribute__((visibility("default")))
#else
#define GMR_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

/* ABI-identical to cudaStream_t / CUstream. */
typedef struct CUstream_st* gmr_stream;

typedef enum {
  GMR_OK = 0,
  GMR_ERR_INVALID_ARG = 1, /* bad pointer, size, configuration or face index */
  GMR_ERR_CUDA = 2,        /* a CUDA runtime call failed; see gmr_last_error */
  GMR_ERR_OOM = 3,         /* device allocation of the workspace failed */
  GMR_ERR_CAPACITY = 4,    /* a workspace buffer was too small (no-sync mode) */
  GMR_ERR_TIMEOUT = 5,     /* a bounded device-side wait expired */
  GMR_ERR_STATE = 6        /* call order: e.g. backward without a forward */
} gmr_status;

/* Device status bits reported by gmr_get_device_status. */
#define GMR_DEV_BAD_FACE_INDEX 1u /* a face referenced a vertex outside [0, V) */
#define GMR_DEV_PAIR_OVERFLOW 2u  /* more (tile, Gaussian) pairs than capacity */

/* Sec. 2.2: which 3D covariance a facet becomes. */
typedef enum {
  GMR_COV_AREA = 0,     /* Eq. 13: area-matched scales kappa*lambda, s_z = 1e-6 */
  GMR_COV_EMBED_RAW = 1 /* Eq. 15 literally: Sigma2D embedded, zero normal variance */
} gmr_cov_mode;

/* Sec. 2.2, colour assignment. */
typedef enum {
  GMR_COLOR_PER_FACE = 0,   /* rgb is F x 3 */
  GMR_COLOR_PER_VERTEX = 1, /* rgb is V x 3; face colour = mean of its 3 vertices (Eq. 16) */
  GMR_COLOR_SH = 2          /* view-dependent colour, the extension the colour assignment of
                               Sec. 2.2 names: rgb is F x K x 3 (K = (L + 1)^2, L =
                               gmr_config.sh_degree <= 3) coefficients of the real spherical
                               harmonics Y_k (no Condon-Shortley phase, order (l, m) = (0, 0),
                               (1, -1), (1, 0), (1, 1), (2, -2), ...); the colour of a facet in a
                               view is max(0, sum_k a_k Y_k(d) + 1/2) per channel, d the unit
                               vector from the camera centre to the facet's centroid */
} gmr_color_mode;

/* Pinhole camera (76 bytes, no padding). World-to-camera rotation R
 * (row-major) and translation t: x_cam = R x + t; OpenCV axes (x right, y
 * down, z forward); pixel (px, py) has its centre at (px + 0.5, py + 0.5);
 * u = fx * x/z + cx, v = fy * y/z + cy. Faces whose centroid depth is not
 * above znear are culled. */
typedef struct {
  float R[9];
  float t[3];
  float fx, fy, cx, cy;
  int32_t width, height;
  float znear;
} gmr_camera;

/* Renderer configuration. Compositing constants are those of the standard
 * 3DGS rasterizer the paper renders with (Sec. 2.1): alpha = min(0.99,
 * o * G), Gaussians with alpha < 1/255 are skipped, a pixel stops before the
 * Gaussian that would take its transmittance below 1e-4, and a 0.3 px^2
 * low-pass term is added to every projected covariance. */
typedef struct {
  int32_t tile;       /* tile edge in pixels: 8, 16 or 32 (finer tiles give
                         shorter lists where Gaussians cover few pixels) */
  int32_t threads;    /* forward threads per tile: 32 or 64 (8x8 tiles), 64, 128
                         or 256 (16x16), 256 (32x32); each thread composites
                         tile^2 / threads pixels */
  int32_t threads_bwd; /* backward threads per tile, same choices */
  int32_t batch;      /* Gaussians staged per shared-memory batch: 64, 128 or 256 */
  int32_t cov_mode;   /* gmr_cov_mode */
  int32_t color_mode; /* gmr_color_mode */
  float bg[3];        /* background colour added as T_final * bg */
  int32_t flags;      /* GMR_FLAG_* */
  uint32_t profile_stages; /* under GMR_FLAG_PROFILE: bit s set = time gmr_stage s;
                              0 = time every stage */
  int32_t sh_degree;  /* GMR_COLOR_SH: degree L of the spherical harmonics, 0..3 */
} gmr_config;

/* With this flag the forward reads the pair count back to the host once
 * (one stream synchronisation) and grows the pair buffers when needed.
 * Without it the forward never synchronises (it may be captured in a CUDA
 * graph) and an undersized buffer sets GMR_DEV_PAIR_OVERFLOW instead. */
#define GMR_FLAG_SYNC_CHECK 1

/* With this flag every stage of the forward and backward (or those selected
 * by profile_stages) is bracketed by CUDA events on the call's stream (also
 * inside a captured graph), and gmr_get_stage_times returns their
 * durations. */
#define GMR_FLAG_PROFILE 2

/* With this flag the forward also records, per pixel, how many Gaussians
 * contributed and an order-sensitive hash of their face ids (returned by
 * gmr_debug_forward_state); for tests that need to know whether a
 * perturbation changed any discrete decision or the compositing order. */
#define GMR_FLAG_DEBUG_COUNTS 4

/* With this flag the two compositing kernels run as persistent grids: as
 * many CTAs as fit on the device at once, each taking the next tile (in the
 * heaviest-first compositing order) from a device counter until none is
 * left, instead of one CTA per tile. Results are identical either way. */
#define GMR_FLAG_PERSISTENT 8

/* With these flags the forward / backward compositing kernel uses the
 * half-warp layout: each 16-lane half of a warp composites its own 4x4-pixel
 * units and walks its own list of the Gaussians that can reach them, so a
 * warp serves two Gaussians per step where they cover few pixels (dense
 * meshes). 16x16 tiles with 128 or 256 threads, or 8x8 tiles, not with
 * GMR_FLAG_PERSISTENT (GMR_ERR_INVALID_ARG otherwise). Images are identical
 * bit for bit; gradients agree up to the order of the float atomics. */
#define GMR_FLAG_HALF_WARP_FWD 16
#define GMR_FLAG_HALF_WARP_BWD 32

/* With these flags the forward / backward compositing kernel uses the
 * warp-staged layout: each warp loads the tile's list of Gaussians itself, 32
 * at a time, keeps those that can reach its pixels and composites them, with
 * no barrier of the thread block inside the tile (the batch size is unused).
 * Any tile size and thread count; not with GMR_FLAG_PERSISTENT, and not
 * together with the half-warp flag of the same direction
 * (GMR_ERR_INVALID_ARG otherwise). Images are identical bit for bit;
 * gradients agree up to the order of the float atomics. */
#define GMR_FLAG_WARP_STAGE_FWD 64
#define GMR_FLAG_WARP_STAGE_BWD 128

/* With this flag (set for the forward: the backward follows the forward's
 * configuration) every gradient sum of the backward is formed in a fixed
 * order, so identical inputs give bit-identical gradients (same launch
 * shape, same device): the compositing backward writes the sums of each
 * (tile, Gaussian) pair to the pair's own slot, adding the shares of the
 * thread block's warps in warp order (no float atomics); the projection
 * backward adds a record's slots in the order of its tiles and a face's
 * records in view order; each vertex's gradient (and, with per-vertex
 * colours, its colour gradient) is gathered over its incident faces in
 * face order through a vertex-to-face incidence list that the backward
 * builds. The backward then runs block-staged with at most 128 Gaussians
 * per batch (a larger batch is taken as 128; the flag is refused together
 * with GMR_FLAG_HALF_WARP_BWD or GMR_FLAG_WARP_STAGE_BWD) and is slower; the
 * workspace grows by 4 bytes per record, 48 bytes per pair and 4 + 12 +
 * 64 bytes per vertex / face. Graph capture of such a backward needs
 * gmr_reserve (which sizes the vertex buffers for up to 3 max_faces
 * vertices) or an earlier uncaptured backward of at least the same sizes.
 * Images do not change. */
#define GMR_FLAG_DETERMINISTIC 256

/* Stages timed under GMR_FLAG_PROFILE. */
typedef enum {
  GMR_STAGE_PROJECT = 0,      /* conversion fused with EWA projection, tile counts (Sec. 2.2, 2.1) */
  GMR_STAGE_SCAN = 1,         /* per-tile counts -> tile segments, total pairs */
  GMR_STAGE_BIN = 2,          /* keys into segments, per-tile radix sort, ranges */
  GMR_STAGE_RASTER_FWD = 3,   /* front-to-back compositing */
  GMR_STAGE_LOSS = 4,         /* gmr_l2_loss */
  GMR_STAGE_RASTER_BWD = 5,   /* compositing backward */
  GMR_STAGE_PROJECT_BWD = 6,  /* projection + conversion backward, vertex scatter */
  GMR_NUM_STAGES = 7
} gmr_stage;

typedef struct gmr_ctx gmr_ctx;

/* Counters of the last forward/backward (host copies; see gmr_get_stats). */
typedef struct {
  int64_t n_records;     /* views x faces */
  int64_t n_pairs;       /* (tile, Gaussian) pairs of the last forward */
  int64_t n_tiles;       /* tiles over all views */
  int64_t n_pixels;      /* pixels over all views */
  int64_t evals_fwd;     /* (pixel, Gaussian) evaluations, last forward */
  int64_t evals_bwd;     /* (pixel, Gaussian) evaluations, last backward */
  int64_t contribs;      /* (pixel, Gaussian) pairs that contributed, last forward */
  int64_t launches;      /* kernels launched by this context since creation */
  int64_t pair_capacity; /* current pair buffer capacity */
  int64_t workspace_bytes; /* device memory the context's workspace holds */
} gmr_stats;

/* Fills *cfg with the defaults: tile 16, 128 threads (forward and backward),
 * batch 256, GMR_COV_AREA,
 * GMR_COLOR_PER_FACE, black background, GMR_FLAG_SYNC_CHECK. */
GMR_API gmr_status gmr_config_default(gmr_config* cfg);

/* Creates a context on the current CUDA device. The context owns its
 * workspace (device memory, grown on demand outside stream capture) and the
 * forward state that gmr_render_bwd consumes. cfg may be NULL (defaults). */
GMR_API gmr_status gmr_create(const gmr_config* cfg, gmr_ctx** out);

/* Frees the context and its workspace. The caller must make sure no work
 * using the context is still running. */
GMR_API gmr_status gmr_destroy(gmr_ctx* ctx);

/* Replaces the configuration (validated). Invalidates the forward state. */
GMR_API gmr_status gmr_set_config(gmr_ctx* ctx, const gmr_config* cfg);

/* Message of the last host-side error of this context ("" if none). */
GMR_API const char* gmr_last_error(const gmr_ctx* ctx);

/* Name of a status code. */
GMR_API const char* gmr_status_string(gmr_status s);

/* Packed image layout: offsets[c] = first pixel of view c, offsets[C] =
 * total pixels. cams and offsets are HOST arrays. */
GMR_API gmr_status gmr_image_offsets(const gmr_camera* cams, int32_t C, int64_t* offsets);

/* Pre-sizes the workspace for up to max_faces faces, max_views views,
 * max_pixels total pixels and max_pairs (tile, Gaussian) pairs, so that
 * later calls within these limits allocate nothing (needed before stream
 * capture; the tile count is bounded for the configured tile size and
 * views of sides up to 16384 px, the vertex count by 3 max_faces). If it
 * has to grow the workspace, the last
 * forward's state is dropped: gmr_render_bwd then returns GMR_ERR_STATE
 * until the next forward. */
GMR_API gmr_status gmr_reserve(gmr_ctx* ctx, int64_t max_faces, int32_t max_views, int64_t max_pixels,
                       int64_t max_pairs);

/* Caps the device memory the context's workspace may hold at max_bytes (0:
 * no cap, the default). A call that would grow the workspace beyond the cap
 * returns GMR_ERR_OOM, as when cudaMalloc fails, with nothing enqueued and
 * the context still usable (a larger cap, or smaller inputs, let the next
 * call proceed). Memory already held is not released by a lower cap. */
GMR_API gmr_status gmr_set_workspace_limit(gmr_ctx* ctx, int64_t max_bytes);

/* Mesh-to-Gaussian conversion alone (Sec. 2.2, Eq. 3-16).
 *  verts   V x 3, faces F x 3 (int32 vertex indices in [0, V)),
 *  rgb     F x 3 (per-face mode) or V x 3 (per-vertex mode, Eq. 16),
 *  opacity F per-face opacities, or NULL for 1 (the paper's o = 1);
 *          values are clamped to [0, 1].
 * Outputs (any may be NULL): means F x 3 (centroid, Eq. 3-4), cov F x 6
 * (xx, xy, xz, yy, yz, zz of Eq. 13 or Eq. 15 per cov_mode), face_rgb F x 3
 * (Eq. 16), face_opacity F. Faces with an index outside [0, V) set
 * GMR_DEV_BAD_FACE_INDEX and get zero outputs. With GMR_COLOR_SH the colour
 * depends on the view: face_rgb must then be NULL (GMR_ERR_INVALID_ARG). */
GMR_API gmr_status gmr_convert(gmr_ctx* ctx, const float* verts, int32_t V, const int32_t* faces, int32_t F,
                       const float* rgb, const float* opacity, float* means, float* cov, float* face_rgb,
                       float* face_opacity, gmr_stream stream);

/* Forward render of C views (Sec. 2.1-2.2): conversion fused with EWA
 * projection, binning, sorting by (tile, depth, face), compositing.
 *  cams     HOST array of C cameras (copied; under stream capture they must
 *           equal those of the previous call on this context).
 *  images   packed RGB output, offsets[C] x 3 floats.
 *  t_final  packed final transmittance, offsets[C] floats, or NULL.
 * verts, faces, rgb and opacity must stay valid and unchanged until the
 * matching gmr_render_bwd has been enqueued. C = 1 in a loop is the
 * per-view form; one call with all views is the batched form. */
GMR_API gmr_status gmr_render_fwd(gmr_ctx* ctx, const float* verts, int32_t V, const int32_t* faces, int32_t F,
                          const float* rgb, const float* opacity, const gmr_camera* cams, int32_t C,
                          float* images, float* t_final, gmr_stream stream);

/* gmr_render_fwd followed by the squared-error image loss, with the loss
 * computed in the compositing kernel's epilogue (the rendered image is not
 * read back from memory): as gmr_render_fwd, plus
 *  target   packed RGB target image, offsets[C] x 3 floats (device),
 *  dL_dimg  output, 2 (images - target), same layout (device),
 *  loss     output, one double (device): sum of (images - target)^2, each
 *           square in FP32, summed in FP32 per thread and warp and in FP64
 *           above that (relative error below 1.3e-6).
 * Same values as gmr_render_fwd + gmr_l2_loss (dL_dimg bit for bit, loss up
 * to those FP32 partial sums). The paper optimises an image loss of the rendered views;
 * fusing it saves one pass over the images. */
GMR_API gmr_status gmr_render_fwd_l2(gmr_ctx* ctx, const float* verts, int32_t V, const int32_t* faces, int32_t F,
                             const float* rgb, const float* opacity, const gmr_camera* cams, int32_t C,
                             float* images, float* t_final, const float* target, float* dL_dimg, double* loss,
                             gmr_stream stream);

/* Backward of the last forward on this context. The per-pixel compositing is
 * recomputed back to front from the stored final transmittance and last
 * contributor; no per-pixel lists are kept.
 *  dL_dimages    packed, same layout as images.
 *  dL_dverts     V x 3 (may be NULL).
 *  dL_drgb       shape of rgb (may be NULL; with GMR_COLOR_SH the
 *                coefficients' gradient, F x K x 3).
 *  dL_dopacity   F (may be NULL; ignored when the forward had opacity NULL).
 *  accumulate    0: outputs are overwritten; 1: gradients are added to them.
 */
GMR_API gmr_status gmr_render_bwd(gmr_ctx* ctx, const float* dL_dimages, float* dL_dverts, float* dL_drgb,
                          float* dL_dopacity, int32_t accumulate, gmr_stream stream);

/* gmr_render_bwd with, in addition, the gradient of the loss with respect
 * to the final transmittance of every pixel (the silhouette loss of Sec. 3.1
 * compares the rendered mask 1 - T_final with the target silhouette):
 *  dL_dimages   as in gmr_render_bwd, or NULL for zero,
 *  dL_dtfinal   packed, offsets[C] floats (same layout as t_final), or NULL
 *               for zero; not both NULL.
 * Since T_final = prod_j (1 - alpha_j), dL/dalpha_i gains
 * -dL/dT_final T_final / (1 - alpha_i); colours are unaffected. */
GMR_API gmr_status gmr_render_bwd_ex(gmr_ctx* ctx, const float* dL_dimages, const float* dL_dtfinal,
                                     float* dL_dverts, float* dL_drgb, float* dL_dopacity, int32_t accumulate,
                                     gmr_stream stream);

/* Backward of the squared-error image loss of the last forward, with the
 * loss formed inside the compositing backward (one pass over the images
 * fewer than gmr_l2_loss + gmr_render_bwd):
 *  images       the images the last forward wrote (packed, device),
 *  target       the target images (same layout, device),
 *  loss         output, one device double: sum of (images - target)^2
 *               (each square in FP32, summed in FP32 per thread and warp and
 *               in double-float above: relative error below 1.3e-6),
 *  dL_dtfinal   as in gmr_render_bwd_ex, or NULL,
 *  the rest     as in gmr_render_bwd.
 * The gradients equal those of gmr_render_bwd_ex with dL_dimages =
 * 2 (images - target) (bit for bit up to the order of the float atomics);
 * no dL/dimages buffer is written. */
GMR_API gmr_status gmr_render_bwd_l2(gmr_ctx* ctx, const float* images, const float* target, double* loss,
                                     const float* dL_dtfinal, float* dL_dverts, float* dL_drgb,
                                     float* dL_dopacity, int32_t accumulate, gmr_stream stream);

/* Silhouette loss (Sec. 3.1: binary cross-entropy between the rendered mask
 * and the target silhouette) over n pixels, the rendered mask being
 * M = 1 - T_final clamped to [1e-6, 1 - 1e-6]:
 * loss = -(weight/n) sum (m log M + (1 - m) log(1 - M)) (device double,
 * FP32 terms and partial sums, FP64 above the warp), and dL_dtfinal =
 * (weight/n) (m / M - (1 - m) / (1 - M)) where M is not clamped, 0 where it
 * is. t_final, mask and dL_dtfinal are n device floats (mask in [0, 1]). */
GMR_API gmr_status gmr_silhouette_bce(gmr_ctx* ctx, const float* t_final, const float* mask, int64_t n,
                                      float weight, float* dL_dtfinal, double* loss, gmr_stream stream);

/* Squared-error loss sum((img - target)^2) over n floats and its gradient
 * 2 (img - target). loss is a device double (overwritten); dL_dimg may
 * alias neither input. Deterministic (fixed reduction order for a given n);
 * FP32 sums of 8 squares, double-float across a thread's chunks of 16 and
 * the warp, FP64 above that (relative error below 1.3e-6). */
GMR_API gmr_status gmr_l2_loss(gmr_ctx* ctx, const float* img, const float* target, int64_t n, float* dL_dimg,
                       double* loss, gmr_stream stream);

/* gmr_l2_loss without a context and without allocating anything: the same
 * loss sum((img - target)^2) (device double, overwritten) and gradient
 * 2 (img - target) (dL_dimg, n floats), for callers that must not call
 * cudaMalloc where they compute the loss (latency-critical loops, where an
 * allocation may synchronise the device; processes whose device memory is
 * owned by their own pool or by a framework's caching allocator). The
 * paper has no counterpart; this is an interface convenience. The reduction's
 * partial sums live in a fixed array inside the library on each GPU (593
 * doubles, 4,744 bytes: one per block of the loss kernel's grid, which has
 * at most 592 blocks whatever n). n is bounded by GMR_L2_NOALLOC_MAX_ELEMS
 * (2^26 floats per operand, so one call moves at most ~0.8 GB), a bound of
 * this entry point rather than of the array: larger n returns
 * GMR_ERR_CAPACITY before anything is enqueued. The array's address is
 * looked up on the first call on each device and kept for the life of the
 * process: make that call before any stream capture, and do not call this
 * entry point on a device after cudaDeviceReset() of it (the address is then
 * stale). Calls on one GPU share the array, so calls that can run
 * concurrently on the same GPU race; order them. Bad pointers or n < 0 return
 * GMR_ERR_INVALID_ARG; a failing CUDA call returns GMR_ERR_CUDA. */
#define GMR_L2_NOALLOC_MAX_ELEMS 67108864
GMR_API gmr_status gmr_l2_loss_noalloc(const float* img, const float* target, int64_t n, float* dL_dimg,
                                       double* loss, gmr_stream stream);

/* Host-to-device copy of `bytes` bytes from page-locked host memory `src`
 * (allocated with cudaHostAlloc / cudaMallocHost, or registered) to device
 * memory `dst`, asynchronously on `stream`: below 64 MiB by a kernel that
 * reads the host buffer directly over the bus (faster than the copy engine
 * for such sizes on the hosts measured), from 64 MiB up by the copy engine
 * (one cudaMemcpyAsync). No context: any device.
 * Returns GMR_ERR_INVALID_ARG when src is not page-locked memory mapped into
 * the device's address space (nothing is launched then), GMR_ERR_CUDA when
 * the launch fails. 16-byte aligned buffers take the vector path; the rest
 * is copied byte by byte. src must stay valid and unmodified until the copy
 * has run. */
GMR_API gmr_status gmr_copy_h2d(void* dst, const void* src, int64_t bytes, gmr_stream stream);

/* One optimiser step of the fitting loop around the renderer (Sec. 3.1) on
 * n device floats, in place: params -= lr m_hat / (sqrt(v_hat) + eps) with
 * m = beta1 m + (1 - beta1) g, v = beta2 v + (1 - beta2) g^2, m_hat =
 * m / (1 - beta1^step), v_hat = v / (1 - beta2^step) (Adam, Kingma and Ba
 * 2015). group = 3 is VectorAdam, the optimiser the paper uses: params are
 * 3-vectors (n a multiple of 3) and v holds one entry per 3-vector, updated
 * with the squared norm |g|^2. m (n floats) and v (n / group floats) are
 * caller-owned and zero before step 1; step counts from 1. */
GMR_API gmr_status gmr_adam_step(gmr_ctx* ctx, float* params, const float* grads, float* m, float* v, int64_t n,
                                 int32_t group, float lr, float beta1, float beta2, float eps, int32_t step,
                                 gmr_stream stream);

/* The two mesh regularisers of the fitting loop (Sec. 3.1: edge length and
 * Laplacian smoothing), with these readings:
 *  losses[0] = (1/3F) sum over the 3F face edges of (l - mean l)^2 (the
 *              variance of the edge lengths: uniform edges),
 *  losses[1] = (1/V) sum_v |v - n_v|^2, n_v the mean of the two other
 *              vertices of every face at v (uniform weights),
 * both unweighted, as device doubles; w_edge * dlosses[0]/dverts +
 * w_lap * dlosses[1]/dverts is ADDED to dL_dverts (V x 3, may be NULL:
 * losses only). Faces with an index outside [0, V) are skipped. */
GMR_API gmr_status gmr_mesh_regularizers(gmr_ctx* ctx, const float* verts, int32_t V, const int32_t* faces,
                                         int32_t F, float w_edge, float w_lap, float* dL_dverts, double* losses,
                                         gmr_stream stream);

/* Chamfer distance (the paper's CD, Sec. 3.1) between two device point sets
 * a (na x 3) and b (nb x 3), by brute force over all pairs:
 * out[0] = mean over a of min over b |a - b|^2, out[1] = the same from b to
 * a (device doubles; CD = out[0] + out[1]). Distances in FP32, means summed
 * in double-float arithmetic. */
GMR_API gmr_status gmr_chamfer(gmr_ctx* ctx, const float* a, int64_t na, const float* b, int64_t nb, double* out,
                               gmr_stream stream);

/* Synchronises the stream, returns and clears the device status bits
 * (GMR_DEV_*) accumulated since the last call. */
GMR_API gmr_status gmr_get_device_status(gmr_ctx* ctx, gmr_stream stream, uint32_t* status);

/* Synchronises the stream and returns the counters. */
GMR_API gmr_status gmr_get_stats(gmr_ctx* ctx, gmr_stream stream, gmr_stats* out);

/* Synchronises the stream and writes, for each gmr_stage, the duration in
 * milliseconds between its two events as last recorded (eagerly or by a
 * replayed graph captured under GMR_FLAG_PROFILE); -1 for a stage that never
 * ran under profiling. ms has GMR_NUM_STAGES entries. */
GMR_API gmr_status gmr_get_stage_times(gmr_ctx* ctx, gmr_stream stream, float* ms);

/* Introspection of the last forward, for tests (device outputs, copied on
 * the stream):
 *  depth_bits  C*F   FP32 depth key bits per (view, face), view-major
 *  rects       C*F*4 inclusive tile rectangle (x0, x1, y0, y1); x0 > x1 when
 *                    the Gaussian is culled or off-screen
 *  tile_ids, face_ids  n_pairs sorted pairs (cap entries available)
 *  ranges      n_tiles*2 [start, end) per global tile
 *  rec_u       C*F*4 image-plane mean as (x_hi, y_hi, x_lo, y_lo), the mean
 *                    being x_hi + x_lo (float pair)
 *  rec_conic   C*F*4 (a, b, c, 0) of the conic Sigma'^-1 = [[a, b], [b, c]]
 *  n_last      n_pixels  list position + 1 of the last contributor
 *  n_contrib   2*n_pixels  contributors per pixel, then a hash of the ordered
 *                          contributor face ids (needs GMR_FLAG_DEBUG_COUNTS)
 * Any pointer may be NULL. n_pairs (host) receives the pair count. */
GMR_API gmr_status gmr_debug_forward_state(gmr_ctx* ctx, uint32_t* depth_bits, int32_t* rects, uint32_t* tile_ids,
                                   uint32_t* face_ids, int64_t cap, uint32_t* ranges, float* rec_u,
                                   float* rec_conic, uint32_t* n_last, uint32_t* n_contrib, int64_t* n_pairs,
                                   gmr_stream stream);

#ifdef __cplusplus
}
#endif

#endif /* GMR_H_ */
