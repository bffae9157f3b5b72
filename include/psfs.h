/*
 * psfs.h -- C ABI of libpsfs: probabilistic shape-from-silhouette (PSFS) on
 * GB300 (sm_103a).
 *
 * The library computes, per frame, the reconstruction stage of Song, Bian,
 * Yan, Zhao, Liu, "Digitize Your Body and Action in 3-D at Over 10 FPS"
 * (Section 2.2.2):
 *
 *   1. per pixel, the silhouette likelihood SLM = P(F = 1 | I) of a single
 *      Gaussian colour background against a uniform foreground with equal
 *      priors (Eq. 1-2);
 *   2. per voxel, the projection of its centre into every camera (Eq. 3),
 *      the sensor model with a latent occluder marginalised out (Eq. 5-9,
 *      generalised with a detection rate P_D and a false-alarm rate P_FA),
 *      and the posterior as a product over cameras (Eq. 3-4), evaluated as a
 *      sum of per-camera log ratios;
 *   3. thresholding of the posterior ("perform a thresholding process",
 *      end of Section 2.2.2) and stream compaction of the occupied voxels
 *      into a list.
 *
 * Conventions used by every call:
 *   - grid: voxel (i, j, k) has its centre at
 *       origin + (i + 1/2, j + 1/2, k + 1/2) * voxel_size
 *     and linear index i + nx * (j + ny * k) (x fastest);
 *   - camera: x_cam = R X + t, (u, v, w) = K x_cam; a point is seen iff
 *     w > 0 and 0 <= u/w < width and 0 <= v/w < height; it then falls in
 *     pixel (floor(u/w), floor(v/w)).  A camera that does not see a voxel
 *     centre contributes no factor to that voxel;
 *   - images: uint8 [n_cams][height][width][3] (RGB interleaved); background
 *     mean and variance: float32 [n_cams][height][width][3]; every camera of
 *     a handle has the same width and height;
 *   - occupancy: float32 [nz][ny][nx]; the voxel list holds uint32 linear
 *     indices in unspecified order.
 *
 * Memory: "device" arguments are CUDA device pointers of the handle's device;
 * "host" arguments are host pointers (pinned memory gives the fastest copies).
 * Device arrays must be 16-byte aligned, except the voxel list and the count
 * (4-byte aligned).  The caller owns every buffer
 * it passes; the handle owns its scratch (likelihood maps, packed background,
 * status word) and frees it in psfs_destroy.
 *
 * Asynchrony and errors: every call checks its arguments on the host and
 * returns PSFS_ERR_INVALID_ARG at once if one is wrong.  Calls that take
 * device pointers only enqueue work on the handle's stream and return; a
 * problem found on the device (voxel list overflow) is recorded in the
 * handle's status word and reported by the next psfs_sync.  Calls taking host
 * pointers synchronise the stream before they return and report device
 * problems themselves.  A handle is not thread-safe; use one per stream.
 */
#ifndef PSFS_H
#define PSFS_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define PSFS_MAX_CAMS 32

typedef enum {
    PSFS_OK = 0,
    PSFS_ERR_INVALID_ARG = 1,  /* an argument failed the host-side checks        */
    PSFS_ERR_NOT_READY = 2,    /* psfs_set_background has not succeeded yet      */
    PSFS_ERR_CAPACITY = 3,     /* voxel list overflow: count holds the true count */
    PSFS_ERR_CUDA = 4,         /* a CUDA runtime call failed                      */
    PSFS_ERR_TIMEOUT = 5,      /* a bounded device-side wait ran out              */
    PSFS_ERR_NOMEM = 6,        /* device or pinned allocation failed              */
    PSFS_ERR_BOUNDS = 7        /* bounds-checked build only: a device-side index
                                  check failed and the access was skipped       */
} psfs_status;

typedef enum {
    PSFS_MAP_F32 = 0,   /* likelihood maps stored as float32                      */
    PSFS_MAP_F16 = 1,   /* stored as IEEE half; accumulation stays float32        */
    PSFS_MAP_BF16 = 2   /* stored as bfloat16; accumulation stays float32         */
} psfs_map_dtype;

/* Regular voxel grid (Section 2.2.2, "volume of interest"). */
typedef struct {
    int32_t nx, ny, nz;     /* voxels per axis, each >= 1, product < 2^32        */
    double origin[3];       /* world position of the grid's minimum corner (m)   */
    double voxel_size;      /* edge length (m), > 0                               */
} psfs_grid;

/* Calibrated pinhole camera (perspective projection, Section 2.2.1). */
typedef struct {
    int32_t width, height;  /* pixels, >= 1                                       */
    double K[9];            /* intrinsics, row-major                              */
    double R[9];            /* world-to-camera rotation, row-major                */
    double t[3];            /* world-to-camera translation                        */
} psfs_camera;

/* Model parameters. */
typedef struct {
    double p_detect;        /* P_D in [0, 1]: P(S | something on the line) uses
                               P_D s + (1 - P_D)(1 - s)                  (Eq. 7-9) */
    double p_false_alarm;   /* P_FA in [0, 1]: P(S | nothing on the line) uses
                               P_FA s + (1 - P_FA)(1 - s)                   (Eq. 6) */
    double prior;           /* P(V = 1) in (0, 1)                          (Eq. 3) */
    double threshold;       /* occupied iff posterior > threshold, in (0, 1)       */
    double log_fg_density;  /* log U of the uniform foreground colour density
                               (Eq. 1); -3 log 256 = uniform over the RGB cube     */
    int32_t map_dtype;      /* psfs_map_dtype of the stored likelihood maps        */
} psfs_params;

/* Launch shapes (speed only, never results).  The voxel tile one CTA of the
 * fusion kernel owns: a warp covers lanes_x voxels along x by 32 / lanes_x
 * along y, a CTA `warps` warps stacked along y, and each thread walks
 * voxels_z voxels along z; supported: lanes_x in {8, 16, 32}, warps = 4,
 * voxels_z in {2, 4, 8, 16} (8 or 16 when staged).  staged = 1 selects the
 * persistent kernel that copies
 * each tile's image footprint per camera into shared memory (bulk copies,
 * double-buffered) before gathering; 0 gathers from global memory.
 * seq_likelihood_ctas: CTAs per SM of the likelihood grid on the sequence
 * path, 1 to 4 (0 in psfs_set_fuse_config keeps the current value).
 * frames_per_group: frames per launch on the sequence path: 1 = one frame
 * per likelihood and fusion launch; 2, 4, 8, 16 or 32 = frame groups, where
 * one likelihood launch reads the background once for the whole group and
 * writes the group's maps as pixel records of seq_record_bytes bytes holding
 * P frames (P = seq_record_bytes / map element size, the group size when
 * smaller), one plane of records per P frames; one fusion launch per plane
 * projects each voxel once per camera and gathers the plane's P frames with
 * one 32-byte vector load per lane (two lanes per voxel for a 64-byte
 * record; each frame's results are bit-identical to one frame per launch).
 * Groups need staged = 0, lanes_x 8 or 16, and voxels_z 2 or 4, or 8 when a
 * lane holds at most 8 frames, or 16 when at most 4 (2 or 4 with 64-byte
 * records); with another shape the sequence path runs one frame per launch.
 * Trailing frames that do not fill a group run in the largest smaller groups
 * that fit, the last odd frame alone.  0 in psfs_set_fuse_config keeps the
 * current value.  The batch entry points ignore this field.
 * cameras_per_block (batch entry points only; handles report 1): a batched
 * fusion item issues the map loads of that many cameras together before it
 * adds them, still camera by camera in the order 0 .. n_cams - 1, so the
 * results do not change; 1, 2 (lanes_x 8 or 16, voxels_z 4 or 8) or 4
 * (lanes_x 8 or 16, voxels_z 4); 0 in psfs_batch_set_config means 1.
 * batch_launch (batch entry points only): 0 = one persistent kernel whose
 * work list interleaves the frames' likelihood chunks and fusion tiles (the
 * tile shape and camera block above apply); 1 = a graph of each frame's own
 * likelihood and fusion launches (the kernels of psfs_reconstruct, each
 * frame with its handle's one-frame tile shape, a direct one if that is
 * staged), frame f on stream f mod 4, so that frames' likelihoods run
 * beside earlier frames' fusions and small frames share the GPU.  Results
 * are the same bits either way.
 * seq_lanes_x, seq_voxels_z: the tile shape of the sequence path (warps 4,
 * staged 0) when it differs from the one-frame-per-call shape above: 0 in
 * psfs_set_fuse_config makes the sequence path use lanes_x / voxels_z;
 * psfs_get_fuse_config reports the shape the sequence path uses (and
 * frames_per_group is checked against it).
 * seq_record_bytes: 32 or 64, the pixel record of the sequence path's map
 * planes (0 in psfs_set_fuse_config keeps the current value; default 32).
 * A 32-byte record is one L2 sector per (voxel, camera) and plane; a 64-byte
 * record holds twice the frames per plane, read by two lanes in one warp
 * request (one L1 wavefront for both sectors of the line), in planes of
 * twice the size. */
typedef struct {
    int32_t lanes_x;
    int32_t warps;
    int32_t voxels_z;
    int32_t staged;
    int32_t seq_likelihood_ctas;
    int32_t frames_per_group;
    int32_t cameras_per_block;
    int32_t seq_lanes_x;
    int32_t seq_voxels_z;
    int32_t seq_record_bytes;
    int32_t batch_launch;
} psfs_fuse_config;

typedef struct psfs_handle psfs_handle;

/* Fills `p` with P_D = 0.9, P_FA = 0.1, prior = 0.5, threshold = 0.5,
 * log U = -3 log 256, float32 maps.  With P_D = 1 and P_FA = 0 the sensor
 * model is Eq. 6-9 of the paper verbatim. */
void psfs_params_default(psfs_params *p);

/* Creates a handle for one grid and one camera rig on the current CUDA
 * device.  `stream` is a cudaStream_t (NULL = the legacy default stream) on
 * which every later call enqueues its work.  Requirements: 1 <= n_cams <=
 * PSFS_MAX_CAMS, all cameras of the same size, finite matrices, valid
 * parameters with (P_D + P_FA) / 2 strictly between 0 and 1.  Allocates the
 * handle's device scratch.  On success *out receives the handle.
 * Errors: INVALID_ARG, NOMEM, CUDA. */
psfs_status psfs_create(const psfs_grid *grid, const psfs_camera *cams, int32_t n_cams,
                        const psfs_params *params, void *stream, psfs_handle **out);

/* Sets the per-pixel background model of Eq. 1: `mean` and `var` are device
 * float32 [n_cams][height][width][3]; each variance must be finite and in
 * [1e-6, 1e12], each mean finite.  The handle keeps a packed copy (mean and
 * 1 / (2 var)), so the caller may free its buffers afterwards.  Synchronises
 * the stream.  Errors: INVALID_ARG (also for out-of-range values found on the
 * device), CUDA. */
psfs_status psfs_set_background(psfs_handle *h, const float *mean, const float *var);

/* One frame of the reconstruction (Eq. 1-9, threshold, compaction).
 *   images     device uint8 [n_cams][height][width][3]
 *   occupancy  device float32 [nz][ny][nx], posterior P(V = 1 | S)   (Eq. 3)
 *   voxel_list device uint32 [capacity], linear indices of the voxels with
 *              posterior > threshold, unspecified order (may be NULL if
 *              capacity == 0)
 *   count      device uint32 [1], number of occupied voxels (even beyond
 *              capacity; only the first `capacity` are written)
 * Enqueues two kernels and returns.  Overflow is reported by psfs_sync as
 * PSFS_ERR_CAPACITY.  Errors: INVALID_ARG, NOT_READY, CUDA. */
psfs_status psfs_reconstruct(psfs_handle *h, const uint8_t *images, float *occupancy,
                             uint32_t *voxel_list, uint32_t capacity, uint32_t *count);

/* psfs_reconstruct over n_frames frames of this rig, one call: frame f reads
 * images + f * (n_cams * height * width * 3) and writes
 * occupancy + f * (nx * ny * nz), voxel_lists + f * capacity and counts[f].
 * Frames run in units of frames_per_group frames (psfs_fuse_config; one
 * likelihood launch and one fusion launch per plane of pixel records per
 * unit).  The likelihood stage of unit
 * u + 1 runs on a second stream concurrently with the fusion stage of unit u
 * (two map buffers), so that the HBM-bound and the gather-bound kernels
 * overlap; the whole sequence is ordered after earlier work on the handle's
 * stream and later work waits for it.  The frame size in bytes and the voxel
 * count must be multiples of 16 and 4.  The first call with frame groups
 * allocates two group map buffers (n_cams * height * width * frames_per_group
 * map elements each).  Errors: INVALID_ARG, NOT_READY, NOMEM, CUDA. */
psfs_status psfs_reconstruct_sequence(psfs_handle *h, int32_t n_frames, const uint8_t *images,
                                      float *occupancy, uint32_t *voxel_lists, uint32_t capacity,
                                      uint32_t *counts);

/* psfs_reconstruct_sequence from and to host memory, synchronous: frame f
 * reads h_images + f * (n_cams * height * width * 3) and writes
 * h_occupancy + f * (nx * ny * nz) (h_occupancy may be NULL: no occupancy
 * copy), h_counts[f] and the first min(h_counts[f], capacity) entries of
 * h_lists + f * capacity.  Frames go through three device staging slots of
 * 4 frames each (allocated on first use, grown on demand): the copy in of
 * one slot and the copy out of another overlap the kernels of the third.  Pinned
 * host buffers (cudaHostAlloc / cudaHostRegister) let the copies run
 * asynchronously; pageable ones work but serialise them.  Returns after the
 * last copy.  Errors: INVALID_ARG, NOT_READY, NOMEM, CUDA, CAPACITY (some
 * frame had more occupied voxels than `capacity`; its count is still exact). */
psfs_status psfs_reconstruct_sequence_host(psfs_handle *h, int32_t n_frames, const uint8_t *h_images,
                                           float *h_occupancy, uint32_t *h_lists, uint32_t capacity,
                                           uint32_t *h_counts);

/* Particle weights of the tracker (Section 2.3.2, Eq. 14-16; Section 3.3.3,
 * the sum-squared-difference steps b-d): how well each particle's projected
 * body matches the voxel silhouettes (psfs_reproject) and their edges in
 * every camera of this handle's rig.  The paper gives the weights but not
 * the sample points; here:
 *   cylinders  device f32 [n_particles][n_cyl][7]: endpoints a, b (world
 *              xyz) and radius r of each body cylinder
 *   samples    per cylinder and camera, with C the camera centre, u = b - a,
 *              n = unit(u x ((a + b) / 2 - C)): silhouette samples a + t u +
 *              w r n at t = (k + 1/2) / kt, w = (2 l + 1) / kw - 1 (k < kt,
 *              l < kw); edge samples at the same t with w = -1 and +1
 *   value      the bit of the pixel a sample projects into: the silhouette
 *              bit, or for edge samples the edge bit (a set pixel with a
 *              4-neighbour inside the image that is not set); 0 behind the
 *              camera or outside the image
 *   masks      device uint8 [n_cams][height][width] silhouettes (0 / 1)
 *   terms      device f32 [n_particles][n_cams][2] or NULL: S_e, S_r of
 *              Eq. 14-15, the mean of (1 - value) over the edge / silhouette
 *              samples of all cylinders
 *   weights    device f32 [n_particles]: exp(-sum over cameras of
 *              (S_e + S_r)) (Eq. 16)
 * Samples are projected in float32: one whose projection lies within about
 * 1e-3 px of a pixel edge may read the neighbouring pixel.
 * Errors: INVALID_ARG (n_cyl, kt or kw outside [1, 64], NULL pointers),
 * CUDA. */
psfs_status psfs_particle_weights(psfs_handle *h, int32_t n_particles, int32_t n_cyl, const float *cylinders,
                                  int32_t kt, int32_t kw, const uint8_t *masks, float *weights, float *terms);

/* Silhouettes of the reconstructed voxels in every camera (Section 2.3: the
 * projection of the voxels is the tracker's prior knowledge; Section 3.3.3,
 * voxel projection): pixel (x, y) of camera c is set iff the ray from the
 * camera centre through the pixel centre (x + 1/2, y + 1/2) meets, in front
 * of the camera, the cube of a listed voxel (origin + [i, i+1] x [j, j+1] x
 * [k, k+1] * voxel_size).  For n_frames frames of this handle's rig:
 *   voxel_lists   device uint32, frame f's voxels (linear indices, any order;
 *                 the surface list of psfs_surface gives the same silhouette
 *                 as the occupied list, with less work) at voxel_lists +
 *                 f * list_stride
 *   counts        device uint32 [n_frames] (entries beyond list_stride are
 *                 not read)
 *   masks         device uint8 [n_frames][n_cams][height][width], written
 *                 completely (0 or 1)
 * Rays are tested in float32: pixels whose centre ray passes within about
 * 1e-3 voxel of a cube's edge may differ from an exact evaluation.
 * Errors: INVALID_ARG, CUDA. */
psfs_status psfs_reproject(psfs_handle *h, int32_t n_frames, const uint32_t *voxel_lists, uint32_t list_stride,
                           const uint32_t *counts, uint8_t *masks);

/* Smoothing of the voxel probabilities before the threshold (end of Section
 * 2.2.2, which filters the probabilities and then thresholds them; step (d)
 * of Section 3.3.3).  The paper does not give the filter; this is the
 * 3 x 3 x 3 box mean over the neighbours inside the grid (a voxel's
 * 27-neighbourhood clipped to the grid, divided by the number of voxels in
 * it, summed along x, then y, then z in FP32), followed by the strict
 * threshold smoothed > params.threshold and the compaction.  For n_frames
 * frames of this handle's grid:
 *   occupancy      device f32, frame f's posterior grid [nz][ny][nx] (as
 *                  psfs_reconstruct* write it) at occupancy + f * n_vox
 *   smoothed       device f32 or NULL, frame f's smoothed grid at
 *                  smoothed + f * n_vox
 *   voxel_lists    device uint32, frame f's voxels above the threshold at
 *                  voxel_lists + f * capacity (order unspecified; only the
 *                  first `capacity` are written)
 *   counts         device uint32 [n_frames], set to the full counts; overflow
 *                  is reported by psfs_sync as PSFS_ERR_CAPACITY
 * One launch for all frames; each probability is read once from memory.
 * Errors: INVALID_ARG (NULL or misaligned pointers, more than
 * 65535 / ceil(nz / 32) frames), CUDA. */
psfs_status psfs_smooth(psfs_handle *h, int32_t n_frames, const float *occupancy, float *smoothed,
                        uint32_t *voxel_lists, uint32_t capacity, uint32_t *counts);

/* Inner-voxel removal (end of Section 2.2.2 and step (e) of Section 3.3.3 of
 * the paper, which removes the voxels inside the body and keeps the surface
 * voxels): for each of n_frames frames of this handle's grid, the surface
 * voxels are the listed (occupied) voxels with at least one of their six face
 * neighbours not listed; a neighbour outside the grid counts as not listed.
 *   voxel_lists      device uint32, frame f's occupied voxels (linear indices,
 *                    any order, as psfs_reconstruct* write them) at
 *                    voxel_lists + f * list_stride
 *   counts           device uint32 [n_frames]; counts[f] > list_stride (an
 *                    overflowed list) makes the frame's result incomplete and
 *                    is reported by psfs_sync as PSFS_ERR_CAPACITY
 *   surface_lists    device uint32, frame f's surface voxels at
 *                    surface_lists + f * surface_capacity (order unspecified;
 *                    only the first surface_capacity are written)
 *   surface_counts   device uint32 [n_frames], the surface voxel counts (even
 *                    beyond surface_capacity; overflow is reported by psfs_sync)
 * Work is proportional to the listed voxels: one occupancy bitmask per frame
 * (n_vox / 8 bytes of handle scratch per frame, grown on demand) is built
 * from the lists and probed for the six neighbours.  Enqueued on the
 * handle's stream after earlier work.  Errors: INVALID_ARG, NOMEM, CUDA. */
psfs_status psfs_surface(psfs_handle *h, int32_t n_frames, const uint32_t *voxel_lists, uint32_t list_stride,
                         const uint32_t *counts, uint32_t *surface_lists, uint32_t surface_capacity,
                         uint32_t *surface_counts);

/* Keeps the packed background (24 bytes per pixel) resident in L2 for the
 * likelihood stage of psfs_reconstruct_sequence (enable = 1), through an L2
 * access-policy window on the sequence path's own likelihood stream; frames
 * after the first then read it from L2 instead of HBM.  Raises the
 * process's persisting-L2 limit (cudaLimitPersistingL2CacheSize) to the
 * background size if it is lower (capped by the device maximum); the limit
 * belongs to this process's CUDA context and ends with it.  enable = 0
 * removes the window.  Errors: INVALID_ARG, NOMEM, CUDA. */
psfs_status psfs_set_background_l2(psfs_handle *h, int32_t enable);

/* psfs_reconstruct with HOST buffers: copies the images to the device, runs
 * the frame, copies the occupancy, the count and min(count, capacity) list
 * entries back, and synchronises.  Host buffers have the shapes of
 * psfs_reconstruct; h_occupancy may be NULL to skip its copy.  Returns
 * PSFS_ERR_CAPACITY on overflow (the list then holds `capacity` entries).
 * Errors: INVALID_ARG, NOT_READY, CAPACITY, NOMEM, CUDA. */
psfs_status psfs_reconstruct_host(psfs_handle *h, const uint8_t *h_images, float *h_occupancy,
                                  uint32_t *h_list, uint32_t capacity, uint32_t *h_count);

/* Steps 2-3 only, from caller-supplied likelihood maps: `slm` is device
 * float32 [n_cams][height][width] holding SLM = P(F = 1 | I) in [0, 1]
 * (Eq. 2).  Outputs as psfs_reconstruct.  Values outside [0, 1] give
 * unspecified results.  Errors: INVALID_ARG, CUDA. */
psfs_status psfs_fuse_slm(psfs_handle *h, const float *slm, float *occupancy,
                          uint32_t *voxel_list, uint32_t capacity, uint32_t *count);

/* The silhouette likelihood maps SLM (Eq. 2) of a frame, float32
 * [n_cams][height][width] into device `slm_out`.  For inspection and tests;
 * the reconstruction stores log-ratio maps internally instead.
 * Errors: INVALID_ARG, NOT_READY, CUDA. */
psfs_status psfs_get_likelihood(psfs_handle *h, const uint8_t *images, float *slm_out);

/* The per-pixel log ratios g = log(a(s) / b(s)) of Eq. 5-9 exactly as the
 * reconstruction stores them for the frame `images`: [n_cams][height][width]
 * elements of the handle's map_dtype (float32, IEEE half or bfloat16) written
 * to device `map_out` (16-byte aligned).  For inspection and tests (the
 * fusion of Eq. 3-4 sums these stored values).
 * Errors: INVALID_ARG, NOT_READY, CUDA. */
psfs_status psfs_get_log_ratio(psfs_handle *h, const uint8_t *images, void *map_out);

/* Adjoint of psfs_reconstruct (the paper runs the forward only; this is the
 * gradient of a loss on the posterior of Eq. 3-4).  Given d_occ = dLoss/d
 * occupancy (device float32 [nz][ny][nx]) for the frame `images`, recomputes
 * the forward (maps, then the log-odds of every voxel) and writes (each may
 * be NULL to skip it)
 *   d_slm   device float32 [n_cams][height][width]     dLoss/dSLM
 *   d_mean  device float32 [n_cams][height][width][3]  dLoss/d mean
 *   d_var   device float32 [n_cams][height][width][3]  dLoss/d var
 * Pixels that no voxel centre projects to get exactly zero.  Deterministic:
 * each pixel's sum over the voxels that project into it is formed by the
 * thread that owns the pixel, in ascending voxel order, without float
 * atomics.  The first adjoint call of a handle builds its owner lists (for
 * every pixel, the voxels whose centre the forward projects into it: 4 bytes
 * per (voxel, camera) pair plus 4 per pixel, kept until psfs_destroy); it
 * needs nx * ny * nz * n_cams < 2^32 (else INVALID_ARG).
 * Errors: INVALID_ARG, NOT_READY, NOMEM, CUDA. */
psfs_status psfs_backward(psfs_handle *h, const uint8_t *images, const float *d_occ,
                          float *d_slm, float *d_mean, float *d_var);

/* psfs_backward over n_frames frames of this rig, one call: frame f reads
 * images + f * (n_cams * height * width * 3) and d_occ + f * (nx * ny * nz)
 * (device, 16-byte aligned), and writes d_slm + f * (n_cams * height * width)
 * (may be NULL).  d_mean and d_var (may be NULL) receive the sum over the
 * frames of each frame's gradient, added in frame order (the background model
 * is shared by the frames).  Frames go in groups of up to 16, each in one or
 * two parts of up to 8: per part the recomputed forward reads the background
 * once for up to 8 frames and gathers each voxel's log ratios of those frames
 * with one load per camera, and dLoss/dL goes into 32-byte per-voxel records
 * of the part's frames; one per-pixel owner pass then reads one record per
 * part and owned voxel for the whole group, so the owner lists, background
 * and d_mean / d_var are read once per 16 frames.  The records alternate
 * between two buffers, so that one group's
 * recomputed forward (one stream) overlaps the previous group's owner pass (a
 * second stream); the call is ordered after earlier work on the handle's
 * stream and later work waits for it.  Each frame's d_slm is bit-identical
 * to psfs_backward's; d_mean and d_var equal the FP32 sum, in frame order, of
 * psfs_backward's.  Scratch (first call): 2 * 16 * nx * ny * nz floats, maps
 * of 8 frames, a tile plan, the sequence streams, and the owner lists of
 * psfs_backward.  Requirements as psfs_reconstruct_sequence (frame size and
 * voxel count multiples of 16 and 4).  Errors: INVALID_ARG, NOT_READY, NOMEM,
 * CUDA. */
psfs_status psfs_backward_sequence(psfs_handle *h, int32_t n_frames, const uint8_t *images,
                                   const float *d_occ, float *d_slm, float *d_mean, float *d_var);

/* The adjoint of psfs_reconstruct / psfs_reconstruct_sequence from the
 * forward's own output: `occupancy` (device float32 [n_frames][nz][ny][nx])
 * must be what the forward gave for these `images` on this handle with its
 * current background.  dLoss/dL = d_occ occ (1 - occ) is then formed
 * elementwise, so the maps and the log-odds are not recomputed; the pixel
 * passes and the outputs are those of psfs_backward (n_frames = 1) and
 * psfs_backward_sequence (n_frames > 1: d_slm per frame [n_frames][n_cams]
 * [height][width], d_mean and d_var summed over the frames; the records of
 * consecutive groups alternate between two buffers, one group's records
 * formed while the previous group's owner pass runs), with the same bits when
 * `occupancy` is the forward's.  Errors: INVALID_ARG, NOT_READY, NOMEM,
 * CUDA. */
psfs_status psfs_backward_from_occupancy(psfs_handle *h, int32_t n_frames, const uint8_t *images,
                                         const float *occupancy, const float *d_occ, float *d_slm,
                                         float *d_mean, float *d_var);

/* Adjoint of psfs_fuse_slm: given the SLM maps `slm` of the forward (device
 * float32 [n_cams][height][width]) and d_occ, writes dLoss/dSLM to d_slm
 * (device float32 [n_cams][height][width]).  Recomputes the forward.
 * Errors: INVALID_ARG, CUDA. */
psfs_status psfs_backward_slm(psfs_handle *h, const float *slm, const float *d_occ, float *d_slm);

/* Selects the tile shape of the fusion kernel (re-plans the handle; waits for
 * its stream).  Errors: INVALID_ARG (unsupported shape), NOMEM, CUDA. */
psfs_status psfs_set_fuse_config(psfs_handle *h, const psfs_fuse_config *cfg);

/* The tile shape in use.  Errors: INVALID_ARG. */
psfs_status psfs_get_fuse_config(psfs_handle *h, psfs_fuse_config *cfg);

/* Autotuner: times every supported tile shape on the frame `images` (device,
 * as psfs_reconstruct) with CUDA events, `reps` launches each, keeps the
 * fastest and writes it to *best (may be NULL) and the mean milliseconds of
 * each candidate to candidate_ms[PSFS_N_FUSE_CANDIDATES] (may be NULL; order:
 * staged 0 with lanes_x 8, 16, 32 and voxels_z 2, 4, 8, 16, then staged 1
 * with lanes_x 8, 16, 32 and voxels_z 8, 16; small grids favour the short
 * tiles, which give more CTAs); then times the
 * sequence path on 64 frames (32 above 2^23 voxels; copies of the frame at
 * distinct addresses) with 1 to 4 likelihood CTAs per SM at one frame per
 * launch, and frame groups of 2, 4, 8, 16 and 32 frames (direct tile shapes,
 * voxels_z 2, 4, 8 and 16, 1 to 3 likelihood CTAs per SM, pixel records of 32
 * and, where a group fills more than 32 bytes per pixel, 64 bytes), and keeps
 * the fastest sequence configuration.  The best one-frame shape stays the handle's tile
 * shape for one frame per call; when frame groups win with another shape,
 * the sequence path gets that shape and a tile plan of its own.  The choices are
 * remembered for handles of the same grid size, camera count, image size and
 * map type created later in the process.  Allocates and frees its own scratch; waits for the stream.
 * Errors: INVALID_ARG, NOT_READY, NOMEM, CUDA. */
#define PSFS_N_FUSE_CANDIDATES 18
psfs_status psfs_autotune(psfs_handle *h, const uint8_t *images, int32_t reps, psfs_fuse_config *best,
                          float *candidate_ms);

/* The autotuner's choices as a file, so that later processes start with them.
 * psfs_autotune remembers, per (grid size, camera count, image size, map
 * type), the tile shape for one frame per call and the sequence path's
 * configuration; psfs_create applies them to handles of that kind.
 * psfs_tune_cache_save writes every remembered choice to `path` as text: a
 * line "psfs-tune 1", then one line per kind of 19 integers: nx ny nz n_cams
 * width height map_dtype, lanes_x warps voxels_z staged (one frame per call),
 * seq_likelihood_ctas frames_per_group, own_sequence_shape (0 or 1), lanes_x
 * warps voxels_z staged (sequence path), seq_record_bytes.
 * psfs_tune_cache_load reads such a file and adds its choices (replacing
 * those of the same kinds); it changes nothing unless every line is valid
 * (supported shapes and sizes).  Handles created earlier keep their
 * configuration.  psfs_tune_cache_clear forgets every choice;
 * psfs_tune_cache_entries returns how many kinds are remembered.  The cache
 * is shared by the threads of the process (guarded).  Errors: INVALID_ARG
 * (NULL path, a file that cannot be opened, read or written, or an invalid
 * line; the message names the line). */
psfs_status psfs_tune_cache_save(const char *path);
psfs_status psfs_tune_cache_load(const char *path);
void psfs_tune_cache_clear(void);
int32_t psfs_tune_cache_entries(void);

/* Waits for the handle's stream, then returns and clears the first problem
 * recorded on the device since the last psfs_sync (PSFS_ERR_CAPACITY), or
 * PSFS_OK.  Errors: CUDA. */
psfs_status psfs_sync(psfs_handle *h);

/* Frees the handle and its scratch (after waiting for its stream).  NULL is a
 * no-op. */
void psfs_destroy(psfs_handle *h);

/* Stages timed by the profiler below. */
typedef enum {
    PSFS_STAGE_LIKELIHOOD = 0,   /* per-pixel kernel (Eq. 1-2 and log ratio)        */
    PSFS_STAGE_FUSE = 1,         /* per-voxel kernel (Eq. 3-9, threshold, list)     */
    PSFS_STAGE_BACKWARD_VOXEL = 2,  /* adjoint: recomputed log-odds -> dLoss/dL     */
    PSFS_STAGE_BACKWARD_PIXEL = 3,  /* adjoint: per-pixel owner pass + chain rule   */
    PSFS_STAGE_BATCH = 4,        /* batched persistent launch                       */
    PSFS_STAGE_SURFACE = 5,      /* inner-voxel removal (psfs_surface)              */
    PSFS_STAGE_SMOOTH = 6,       /* smoothing + threshold (psfs_smooth)             */
    PSFS_STAGE_REPROJECT = 7,    /* voxel silhouettes (psfs_reproject)              */
    PSFS_N_STAGES = 8
} psfs_stage;

/* Tracing: with max_launches > 0, every later kernel launch of the handle is
 * bracketed by two CUDA events on its stream (a pool sized for max_launches
 * launches between two reads; launches beyond it are not timed).  0 turns it
 * off and frees the pool.  Errors: INVALID_ARG, CUDA. */
psfs_status psfs_profile_enable(psfs_handle *h, int32_t max_launches);

/* Waits for the stream and writes, per psfs_stage, the summed device time in
 * milliseconds and the number of timed launches since the previous read
 * (arrays of PSFS_N_STAGES entries), then resets them.  Errors: INVALID_ARG,
 * CUDA. */
psfs_status psfs_profile_read(psfs_handle *h, double *ms, int32_t *launches);

/* ---- Batched persistent launch (no counterpart in the paper, which runs one
 * frame at a time): many frames, each with its own rig (grid size, camera
 * count, image size, background: its handle), in one persistent kernel
 * captured in a CUDA graph.  The kernel interleaves the likelihood chunks of
 * frame f with the fusion tiles of frame f - 1, so that HBM-bound and
 * gather-bound work share the SMs; a fusion tile waits (bounded, 1 s, then
 * PSFS_ERR_TIMEOUT from psfs_batch_sync) for its frame's maps.  Results are
 * those of psfs_reconstruct on each frame. */
typedef struct {
    psfs_handle *handle;     /* the frame's rig; its background must be set;
                                must outlive the batch                        */
    const uint8_t *images;   /* device, as psfs_reconstruct                   */
    float *occupancy;        /* device outputs, as psfs_reconstruct           */
    uint32_t *voxel_list;
    uint32_t capacity;
    uint32_t *count;
} psfs_frame;

typedef struct psfs_batch psfs_batch;

/* Plans every frame, allocates one map buffer per frame, builds the work
 * list and captures the graph.  The buffers named in `frames` are fixed: a
 * run reads whatever they hold when it executes.  All handles must share the
 * map type and device.  `stream` is where psfs_batch_run enqueues.
 * Errors: INVALID_ARG, NOT_READY, NOMEM, CUDA. */
psfs_status psfs_batch_create(const psfs_frame *frames, int32_t n_frames, void *stream, psfs_batch **out);

/* Launches the captured graph (all frames) on the batch's stream. */
psfs_status psfs_batch_run(psfs_batch *b);

/* Waits for the batch's stream; returns and clears the first device-side
 * problem (PSFS_ERR_TIMEOUT, PSFS_ERR_CAPACITY, PSFS_ERR_BOUNDS) or PSFS_OK. */
psfs_status psfs_batch_sync(psfs_batch *b);

/* The batch's launch form (batch_launch) and, for the persistent kernel, the
 * tile shape of its fusion items (staged must be 0) and camera block;
 * re-plans and re-captures. */
psfs_status psfs_batch_set_config(psfs_batch *b, const psfs_fuse_config *cfg);

/* Autotuner of the batch: times the whole graph for each of
 * PSFS_N_BATCH_CANDIDATES candidates (order: the persistent kernel with
 * lanes_x 8, 16, 32 x voxels_z 8, 16 and one camera per load block; then
 * camera blocks of 2 with lanes_x 8, 16 x voxels_z 4, 8; then camera blocks
 * of 4 with lanes_x 8, 16 and voxels_z 4; last the graph of per-frame
 * launches; times in candidate_ms if not NULL), keeps the fastest and
 * reports it in *best (batch_launch 1 for the last candidate). */
#define PSFS_N_BATCH_CANDIDATES 13
psfs_status psfs_batch_autotune(psfs_batch *b, int32_t reps, psfs_fuse_config *best, float *candidate_ms);

/* Failure detection of the batched launch.  A fusion item waits for every
 * likelihood chunk of its frame (items of other CTAs, counted on the device);
 * the wait is bounded: after `limit_ns` (default 1 s) the item records a
 * timeout, which psfs_batch_sync returns as PSFS_ERR_TIMEOUT, and once one
 * wait has run out every later wait of the launch gives up at once.  This
 * sets that limit (1 us to 10 s) and, for tests of the timeout path only,
 * `hold_frame`: a frame whose items then wait for one chunk more than the
 * frame has, so that their wait must run out (-1: none; the results of a
 * launch with a held frame are invalid).  Re-plans and re-captures the graph
 * as the persistent kernel (the per-frame launch graph has no device-side
 * waits).  Errors: INVALID_ARG, CUDA, NOMEM. */
psfs_status psfs_batch_set_wait_limit(psfs_batch *b, uint64_t limit_ns, int32_t hold_frame);

void psfs_batch_destroy(psfs_batch *b);

/* Largest n_cams * height * width that psfs_reconstruct_noalloc accepts. */
#define PSFS_NOALLOC_MAX_PIXELS (4 * 1024 * 1024)

/* One frame of the reconstruction for callers that cannot allocate device
 * memory: hosts that own every byte of device memory and hand this code fixed
 * buffers, or latency-critical loops that must not pay the implicit
 * synchronisation of cudaMalloc.  (The paper has no counterpart; this is a
 * deployment form of psfs_reconstruct.)
 *   grid, cams, n_cams, params  as psfs_create (params->map_dtype must be
 *                               PSFS_MAP_F32); read on the host, not kept
 *   mean, var                   device float32 [n_cams][height][width][3],
 *                               values as psfs_set_background requires (not
 *                               checked here)
 *   images, occupancy, voxel_list, capacity, count
 *                               as psfs_reconstruct (4-byte aligned device
 *                               pointers).  The call never returns
 *                               PSFS_ERR_CAPACITY: an overflow shows only as
 *                               count > capacity once the kernels have run,
 *                               with the first capacity entries in the list
 *   stream                      cudaStream_t to enqueue on (NULL = legacy)
 * Allocates nothing: its only scratch (the frame's log-ratio maps and a status
 * word) is a fixed __device__ array of PSFS_NOALLOC_MAX_PIXELS floats plus 256
 * bytes that every GPU loading the library holds until the process exits.
 * The first call on a device looks up that array's device address (set-up
 * per device), so make it before any stream capture.  Calls share the array:
 * calls that overlap on the GPU race and give wrong results; order them on
 * one stream.  Same results as psfs_reconstruct.  Enqueues two kernels and
 * returns.  Errors (described by psfs_last_error_message): INVALID_ARG (as
 * psfs_create, including a grid axis longer than 2^24, and also n_cams *
 * height * width > PSFS_NOALLOC_MAX_PIXELS), CUDA. */
psfs_status psfs_reconstruct_noalloc(const psfs_grid *grid, const psfs_camera *cams, int32_t n_cams,
                                     const psfs_params *params, const float *mean, const float *var,
                                     const uint8_t *images, float *occupancy, uint32_t *voxel_list,
                                     uint32_t capacity, uint32_t *count, void *stream);

/* Measurement of the gather rate that bounds the fusion kernels (Eq. 3: each
 * voxel reads the pixel record at its projection in every camera).  Reads the
 * rows idx[0 .. n) of `rows` with the fusion kernels' own loads — one 256-bit
 * read-only load per lane and 32-byte half of a row, two rows in flight per
 * lane — and XORs every 32-bit word read into *checksum, which it does not
 * clear.  Nothing else is computed, so rows gathered per second over a given
 * index list is the device's ceiling for the fusion's reads of the same rows.
 *   rows         device, n_rows rows of record_bytes (32 or 64) bytes,
 *                aligned to record_bytes
 *   idx          device int32 [n] row indices; entries outside [0, n_rows)
 *                are skipped (read nothing)
 *   stream       cudaStream_t to enqueue on (NULL = legacy default stream)
 *   checksum     device uint32, 4-byte aligned
 * Enqueues one kernel on the current device and returns.  Errors (described
 * by psfs_last_error_message): INVALID_ARG, CUDA. */
psfs_status psfs_gather_rows(const void *rows, int64_t n_rows, int32_t record_bytes, const int32_t *idx, int64_t n,
                             void *stream, uint32_t *checksum);

/* Static English name of a status code. */
const char *psfs_status_string(psfs_status s);

/* Text describing the last failure returned to the calling thread (which
 * argument, which CUDA call).  Valid until the thread's next failing call. */
const char *psfs_last_error_message(void);

#ifdef __cplusplus
}
#endif

#endif /* PSFS_H */
