// psfs_internal.cuh -- shared declarations of libpsfs (kernels + host side).
//
// Numerical form used on the device (Section 2.2.2 of the paper, restated):
//
//   Eq. 1-2   SLM s = U / (U + N), N = prod_c (2 pi var_c)^(-1/2)
//             exp(-(I_c - mu_c)^2 / (2 var_c)).  Written with r = log U - log N
//             this is s = sigmoid(r), and with h_c = 1 / (2 var_c)
//               r = log U + 1.5 log(pi) - 0.5 log(h0 h1 h2) + sum_c (I_c - mu_c)^2 h_c.
//   Eq. 5-9   a(s) = P_D s + (1 - P_D)(1 - s)           = P(S | V = 1)
//             f(s) = P_FA s + (1 - P_FA)(1 - s)
//             b(s) = (a + f) / 2                         = P(S | V = 0)
//             With s = sigmoid(r) the common factor 1 / (1 + e^r) cancels:
//               g(r) = log(a / b) = log(P_D e^r + 1 - P_D) - log(q e^r + 1 - q),
//             q = (P_D + P_FA) / 2.  The likelihood kernel stores g per pixel.
//   Eq. 3-4   log-odds L_v = logit(prior) + sum over cameras that see v of g
//             at the pixel of v; posterior = 1 / (1 + exp(-L_v)); occupied iff
//             L_v > logit(threshold).
#pragma once

#include <cuda.h>   // CUtensorMap (type only; the encoder is fetched through the runtime)
#include <cuda_runtime.h>
#include <cuda_fp16.h>
#include <cuda_bf16.h>
#include <stdint.h>

#include <vector>

#include "psfs.h"

namespace psfs {

constexpr uint32_t kStatusCapacity = 1u;
constexpr uint32_t kStatusTimeout = 2u;
constexpr uint32_t kStatusBadValue = 4u;
constexpr uint32_t kStatusBounds = 8u;   // an access outside its buffer was skipped (bounds-checked build)

// The bounds-checked build (-DPSFS_BOUNDS_CHECK): at the accesses whose index
// rests on the kernels' own arithmetic or on a host-side proof (a pixel the
// planner proved inside the image, an owner's voxel index, a silhouette row),
// the index is tested; a failing access is skipped and kStatusBounds recorded
// in the status word (psfs_sync then returns PSFS_ERR_BOUNDS).  In the normal
// build PSFS_IN_BOUNDS is the constant true and compiles to nothing.
#ifdef PSFS_BOUNDS_CHECK
__device__ __forceinline__ bool psfs_in_bounds(bool ok, uint32_t *status)
{
    if (!ok && status) atomicOr(status, kStatusBounds);
    return ok;
}
#define PSFS_IN_BOUNDS(cond, status) ::psfs::psfs_in_bounds((cond), (status))
#else
#define PSFS_IN_BOUNDS(cond, status) true
#endif

// Projection of voxel index space into one camera: (u, v, w) = M (i', j', k', 1)
// with i' = i - (nx - 1) / 2 (likewise j', k'), rows u, v, w of 4 floats.
struct CamMat {
    float m[12];
};

// Constants of g(r) above.
struct SensorConsts {
    float pd, one_minus_pd;   // A(r) = P_D e^r + (1 - P_D)
    float q, one_minus_q;     // B(r) = q e^r + (1 - q)
    int a_zero_const_pos;     // P_D == 0: for r > 0, A e^-r = e^-r exactly
    int a_zero_const_neg;     // P_D == 1: for r <= 0, A = e^r exactly
};

struct LikelihoodArgs {
    const uint8_t *img;       // [n_pix][3]
    const float *mean;        // [n_pix][3]
    const float *hinv;        // [n_pix][3], 1 / (2 var)
    int64_t n_pix;
    float c0;                 // log U + 1.5 log(pi)
    SensorConsts sc;
    void *out;                // [n_pix] map of g (f32 / f16 / bf16) or of s (f32)
    uint32_t *zero_word;      // if non-null, set to 0 by one thread
    uint32_t *status;         // device status word (bounded-wait timeouts)
    // frame groups (sequence path): img is frame 0 of the group, frame f at
    // img + f * img_fstride bytes; out is [n_pix][F]; the F words
    // zero_word + f * zero_fstride are set to 0
    int64_t img_fstride;
    int64_t zero_fstride;
};

struct SlmToMapArgs {
    const float *slm;         // [n_pix] s in [0, 1]
    int64_t n_pix;
    float da, one_minus_pd;   // a(s) = (1 - P_D) + (2 P_D - 1) s
    float db, one_minus_q;    // b(s) = (1 - q) + (2 q - 1) s
    void *out;
    uint32_t *zero_word;
};

// Per (tile, camera) record prepared on the host at handle creation, in
// double precision from the 8 corner voxel centres of the tile (int4):
//   x, y   first column (rounded down to a 16-byte boundary) and row of the
//          image box that the tile's seen voxel centres project into (1 px
//          margin)
//   z      width of that box clipped to the image, in map elements
//          | width class << 16 (tensor-map box width 32 << class)
//          | number of 16-row boxes << 18
//   w      height of the box clipped to the image, in rows | flags << 16
constexpr int kTcStaged = 1;   // the staged kernel copies the box to shared memory
constexpr int kTcInside = 2;   // every voxel centre of the tile is in front of the
                               // camera and inside the image, with margin for the
                               // float32 rounding of the kernel
constexpr int kTcSkip = 4;     // the camera sees no voxel centre of the tile

struct FuseArgs {
    const void *maps;         // [n_cams][H][W] of g, dtype per map_dtype
    int W, H;
    int64_t map_stride;       // W * H
    int n_cams;
    int nx, ny, nz;
    float ci, cj, ck;         // (n - 1) / 2 per axis
    const uint64_t *tiles;    // packed tile coordinates, Morton order
    const int4 *tilecam;      // [n_tiles][n_cams] records
    int n_tiles;
    float logit_prior, logit_tau;
    float *occ;               // [nz][ny][nx]
    uint32_t *list;
    uint32_t capacity;
    uint32_t *count;
    uint32_t *status;
    int tmap_ok;              // the tensor maps below describe `maps`
    // frame groups (sequence path): maps are [n_cams][H][W][F]; the outputs of
    // frame f are occ + f * occ_fstride, list + f * list_fstride and
    // count + f * count_fstride
    int64_t occ_fstride, list_fstride, count_fstride;
    CamMat cam[PSFS_MAX_CAMS];
    // 3-D tensor maps {W, H, n_cams} of `maps` with boxes of (32 << class) x 16
    // x 1 elements, for the staged kernel
    CUtensorMap tmap[3];
};

// Height of one staged box (rows) and the widths of the three box classes.
constexpr int kBoxRows = 16;
constexpr int kBoxClasses = 3;

// Encodes the three tensor maps of a [n_cams][H][W] map buffer; false when
// the rows are not 16-byte aligned or the encoder is unavailable.
bool encode_map_tensors(void *maps, int map_dtype, int W, int H, int n_cams, CUtensorMap *out);

// Encodes a 4-D tensor map {nx, ny, nz, n_frames} of float32 grids with boxes
// of box_x x box_y x 1 x 1 elements (elements outside the grids read as
// zero); false when the rows are not 16-byte multiples, the base is not
// 16-byte aligned or the encoder is unavailable.
bool encode_grid_tensor(const float *grids, int nx, int ny, int nz, int n_frames, int box_x, int box_y,
                        CUtensorMap *out);

// Tile shape of the fuse kernel (see psfs_fuse_config): a warp is LX voxels
// along x by 32 / LX along y, a CTA WY warps along y, TZ voxels per thread
// along z.
// `staged` selects the persistent kernel that copies each (tile, camera) image
// box into shared memory with bulk copies (double-buffered across cameras)
// and gathers from there; otherwise every CTA gathers from global memory.
struct FuseShape {
    int lx, wy, tz, staged;
    int tile_x() const { return lx; }
    int tile_y() const { return (32 / lx) * wy; }
    int tile_z() const { return tz; }
};
constexpr FuseShape kDefaultFuseShape = {8, 4, 16, 0};
bool fuse_shape_supported(const FuseShape &s);

// Shared-memory staging of the staged fusion kernel: two buffers of
// kStageBytes (each holds the boxes of one (tile, camera) step), three CTAs
// per SM.
constexpr int kStageBytes = 32 * 1024;
constexpr int kStagedCtasPerSm = 3;
inline int stage_cap_elems(int map_dtype) { return kStageBytes / (map_dtype == PSFS_MAP_F32 ? 4 : 2); }

__host__ __device__ inline uint64_t pack_tile(uint32_t tx, uint32_t ty, uint32_t tz)
{
    return (uint64_t)tx | ((uint64_t)ty << 21) | ((uint64_t)tz << 42);
}

// ---------------------------------------------------------------------------
// device helpers shared by the forward and adjoint kernels
// ---------------------------------------------------------------------------
__device__ __forceinline__ float rcp_approx(float x)
{
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

// The hardware approximations of 2^x and log2(x) with denormals flushed
// (PTX ex2 / lg2 .approx.ftz), and e^x, log(x), a / b and the logistic
// function built from them: e^x = 2^(x log2 e), log x = ln 2 log2 x,
// a / b = a (1 / b).  Every kernel that evaluates these quantities (forward,
// frame groups, adjoint) goes through these functions, so their results agree
// bit for bit.
constexpr float kLog2e = 1.44269504088896341f;
constexpr float kLn2 = 0.693147180559945309f;

__device__ __forceinline__ float ex2_approx(float x)
{
    float r;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

__device__ __forceinline__ float lg2_approx(float x)
{
    float r;
    asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

__device__ __forceinline__ float exp_fast(float x) { return ex2_approx(x * kLog2e); }
__device__ __forceinline__ float log_fast(float x) { return lg2_approx(x) * kLn2; }
__device__ __forceinline__ float div_fast(float a, float b) { return a * rcp_approx(b); }

// posterior 1 / (1 + e^-lo) of log-odds lo (Eq. 3-4 in log form)
__device__ __forceinline__ float posterior_of_logodds(float lo) { return rcp_approx(1.0f + exp_fast(-lo)); }

// the silhouette likelihood s = 1 / (1 + e^-r) of Eq. 2, without overflow
__device__ __forceinline__ float sigmoid_fast(float r)
{
    if (r > 0.0f) return rcp_approx(1.0f + exp_fast(-r));
    const float e = exp_fast(r);
    return div_fast(e, 1.0f + e);
}

// Pixel coordinate with a bias: fma with round-down of u * rw + 1.5 * 2^23
// leaves floor(u * rw) in the low mantissa bits, so the bit pattern minus
// kFloorBias is floor(u / w) for |u / w| < 2^22.  Outside that range, and for
// inf / NaN, the unsigned difference is >= 2^22, larger than any image side,
// so a single unsigned compare both floors and bounds-checks.
constexpr float kFloorMagic = 12582912.0f;   // 1.5 * 2^23
constexpr uint32_t kFloorBias = 0x4B400000u; // its bit pattern

__device__ __forceinline__ uint32_t biased_floor(float u, float rw)
{
    return __float_as_uint(__fmaf_rd(u, rw, kFloorMagic));
}

// Projection of voxel (fi, fj, fk) (centred index coordinates) into camera
// `m`: the homogeneous image position (u, v, w) = M (fi, fj, fk, 1), its
// reciprocal depth and the biased pixel coordinates.  Every kernel that maps a
// voxel to a pixel (forward and adjoint) goes through this function, so their
// pixel choices are identical bit for bit.
struct Proj {
    float w;
    uint32_t bx, by;   // biased floor(u / w), floor(v / w)
};

__device__ __forceinline__ Proj project_biased(const float *m, float bu, float bv, float bw, float fk)
{
    Proj p;
    const float u = fmaf(m[2], fk, bu);
    const float v = fmaf(m[6], fk, bv);
    p.w = fmaf(m[10], fk, bw);
    const float rw = rcp_approx(p.w);
    p.bx = biased_floor(u, rw);
    p.by = biased_floor(v, rw);
    return p;
}

// The k-independent part of the projection of row (fi, fj).
__device__ __forceinline__ void project_base(const float *m, float fi, float fj, float *bu, float *bv,
                                             float *bw)
{
    *bu = fmaf(m[0], fi, fmaf(m[1], fj, m[3]));
    *bv = fmaf(m[4], fi, fmaf(m[5], fj, m[7]));
    *bw = fmaf(m[8], fi, fmaf(m[9], fj, m[11]));
}

// Seen test and pixel offset py * W + px of a projected voxel centre.
__device__ __forceinline__ bool proj_pixel(const Proj &p, uint32_t W, uint32_t H, int *pix)
{
    const uint32_t ix = p.bx - kFloorBias, iy = p.by - kFloorBias;
    *pix = (int)(iy * W + ix);
    return (p.w > 0.0f) & (ix < W) & (iy < H);
}

__device__ __forceinline__ bool project_voxel(const float *m, float fi, float fj, float fk,
                                              uint32_t W, uint32_t H, int *pix)
{
    float bu, bv, bw;
    project_base(m, fi, fj, &bu, &bv, &bw);
    return proj_pixel(project_biased(m, bu, bv, bw, fk), W, H, pix);
}

// ---------------------------------------------------------------------------
// mbarrier + bulk-copy (TMA) helpers, inline PTX for sm_90+ / sm_103a
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void *p)
{
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_fence_init()
{
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t *bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];\n" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

// One box of a 3-D tensor map, global -> shared (TMA), completion counted on
// `bar`.  x must be a multiple of 16 bytes / element size; rows and cameras
// outside the tensor are filled with zeros.
__device__ __forceinline__ void tma_load_3d(void *dst, const CUtensorMap *tmap, int x, int y, int z, uint64_t *bar)
{
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], "
        "[%5];\n" ::"r"(smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(tmap)), "r"(x), "r"(y), "r"(z), "r"(smem_u32(bar))
        : "memory");
}

// One bulk copy global -> shared, completion counted on `bar` (bytes and both
// addresses multiples of 16).
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *bar)
{
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(
            smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity)
{
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return done != 0;
}

__device__ __forceinline__ uint64_t globaltimer_ns()
{
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;\n" : "=l"(t));
    return t;
}

// Bounded wait for phase `parity` of `bar`.  After kWaitNs of polling it
// records kStatusTimeout, waits once more up to kWaitNs for the copies still
// in flight, and returns false.  Callers then carry on with whatever the
// buffer holds, so that every thread still reaches every barrier; the status
// word marks the result invalid.
constexpr uint64_t kWaitNs = 1000000000ull;   // 1 s

__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, uint32_t parity, uint32_t *status)
{
    if (mbar_try_wait(bar, parity)) return true;
    const uint64_t t0 = globaltimer_ns();
    for (;;) {
        for (int n = 0; n < 64; ++n)
            if (mbar_try_wait(bar, parity)) return true;
        if (globaltimer_ns() - t0 > kWaitNs) break;
    }
    if (status) atomicOr(status, kStatusTimeout);
    const uint64_t t1 = globaltimer_ns();
    while (globaltimer_ns() - t1 < kWaitNs)
        if (mbar_try_wait(bar, parity)) break;
    return false;
}

// Map loads through the coherent path, for maps written earlier in the same
// kernel by other CTAs (the batched kernel); map_load below uses the
// read-only path, valid when the maps come from an earlier kernel.
__device__ __forceinline__ float map_load_coherent(const float *p) { return *p; }
__device__ __forceinline__ float map_load_coherent(const __half *p) { return __half2float(*p); }
__device__ __forceinline__ float map_load_coherent(const __nv_bfloat16 *p) { return __bfloat162float(*p); }

template <typename T>
__device__ __forceinline__ float map_load(const T *p);
template <>
__device__ __forceinline__ float map_load<float>(const float *p) { return __ldg(p); }
template <>
__device__ __forceinline__ float map_load<__half>(const __half *p) { return __half2float(__ldg(p)); }
template <>
__device__ __forceinline__ float map_load<__nv_bfloat16>(const __nv_bfloat16 *p)
{
    return __bfloat162float(__ldg(p));
}

// r = log U - log N (Eq. 1) for one pixel, from its colour, mean and
// h = 1 / (2 var):  r = c0 - 0.5 log(h0 h1 h2) + sum_c (I_c - mu_c)^2 h_c,
// c0 = log U + 1.5 log(pi).  The forward and the adjoint both call this.
// The pixel's colour-independent part c0 - log(det)/2 and the quadratic form
// sum (I - mu)^2 h; r is their sum.  Kernels that evaluate one pixel for
// several frames compute the first part once and add it the same way.
__device__ __forceinline__ float pixel_log_base(float h0, float h1, float h2, float c0)
{
    return c0 - 0.5f * log_fast(h0 * h1 * h2);
}

__device__ __forceinline__ float pixel_quad(float i0, float i1, float i2, float m0, float m1, float m2, float h0,
                                            float h1, float h2)
{
    const float d0 = i0 - m0, d1 = i1 - m1, d2 = i2 - m2;
    return fmaf(d0 * d0, h0, fmaf(d1 * d1, h1, d2 * d2 * h2));
}

__device__ __forceinline__ float pixel_log_odds(float i0, float i1, float i2, float m0, float m1,
                                                float m2, float h0, float h1, float h2, float c0)
{
    return pixel_log_base(h0, h1, h2, c0) + pixel_quad(i0, i1, i2, m0, m1, m2, h0, h1, h2);
}

// g(r) = log(P_D e^r + 1 - P_D) - log(q e^r + 1 - q), evaluated with
// e^-|r| only, so it neither overflows nor loses the constant terms.  The
// hardware approximations (ex2 / lg2 / rcp) keep the absolute error of g near
// 2e-7: A / B stays bounded away from 0 and infinity unless P_D
// is 0 or 1, which takes the branch without the ratio.
__device__ __forceinline__ float log_ratio_of_r(float r, const SensorConsts &c)
{
    const float ar = fabsf(r);
    const float u = exp_fast(-ar);
    // r > 0: both terms divided by e^r.  Operand selects, not branches.
    const bool pos = r > 0.0f;
    const float A = fmaf(pos ? c.one_minus_pd : c.pd, u, pos ? c.pd : c.one_minus_pd);
    const float B = fmaf(pos ? c.one_minus_q : c.q, u, pos ? c.q : c.one_minus_q);
    if (c.a_zero_const_pos | c.a_zero_const_neg) {   // P_D in {0, 1} (uniform across the launch)
        if (pos ? c.a_zero_const_pos : c.a_zero_const_neg) return -ar - log_fast(B);   // A = e^-|r| exactly
    }
    return log_fast(div_fast(A, B));
}

// The text that psfs_last_error_message returns: every failing entry point
// records it (per calling thread) and returns the status it is given
// (psfs_api.cu).
psfs_status record_failure(psfs_status s, const char *what);
psfs_status record_cuda_failure(cudaError_t e, const char *where);
const char *last_failure();

// Streaming multiprocessors of the current device (cached per device).
int device_sm_count();

// ---------------------------------------------------------------------------
// launchers (defined in the .cu files)
// ---------------------------------------------------------------------------
cudaError_t launch_pack_background(const float *mean, const float *var, int64_t n_pix,
                                   float *mean_out, float *hinv_out, uint32_t *bad,
                                   cudaStream_t s);
// ctas_per_sm: CTAs of the persistent likelihood grid per SM (1..4); fewer
// leave room for fusion CTAs of another frame running concurrently.
cudaError_t launch_likelihood(const LikelihoodArgs &a, int map_dtype, bool slm_out, cudaStream_t s,
                              int ctas_per_sm = 4);
cudaError_t launch_slm_to_map(const SlmToMapArgs &a, int map_dtype, cudaStream_t s);

// A camera seen from its pixels (for the silhouettes of listed voxels): the
// ray of a pixel in voxel-index coordinates.
struct PixelInv {
    float qc[3];    // camera centre in continuous voxel-index coordinates (voxel centres at integers)
    float minv[9];  // pixel (x, y, 1) -> ray direction in voxel-index coordinates, row-major
    float margin;   // pixels: frustum widening that covers the float32 error of the forward projection
};

// Silhouettes of listed voxels (psfs_reproject.cu): frame f's list at lists +
// f * list_stride with counts[f] entries; masks [n_frames][n_cams][H][W]
// bytes (zeroed by the launcher).
struct ReprojectArgs {
    CamMat cam[PSFS_MAX_CAMS];
    PixelInv inv[PSFS_MAX_CAMS];
    const uint32_t *lists;
    uint32_t list_stride;
    const uint32_t *counts;
    uint8_t *masks;
    int n_cams, W, H, nx, ny, nz;
    float ci, cj, ck;
    uint32_t n_vox;
    uint32_t *status;   // status word (bounds-checked build)
};
cudaError_t launch_reproject(const ReprojectArgs &a, int n_frames, cudaStream_t s);

// Particle weights of the tracker (psfs_weights.cu): world -> pixel
// matrices P = K [R | t] and camera centres per camera; particle p's
// cylinders at cyl + p * n_cyl * 7 (a xyz, b xyz, r); silhouettes
// [n_cams][H][W]; weights [P]; terms [P][n_cams][2] (S_e, S_r) or null.
struct WeightArgs {
    float P[PSFS_MAX_CAMS][12];
    float C[PSFS_MAX_CAMS][3];
    int n_cams, W, H;
    int n_cyl, kt, kw;
    const float *cyl;
    const uint8_t *masks;
    float *weights;
    float *terms;
};
cudaError_t launch_weights(const WeightArgs &a, int n_particles, cudaStream_t s);

// Frames per record of dLoss/dL in the batched adjoint (a pixel pass reads
// one or two planes of such records): frame f of voxel v at dl[v * kBwRecord
// + f], 32 bytes per voxel.
constexpr int kBwRecord = 8;

// Adjoint (psfs_backward.cu, psfs_owners.cu).  The voxel pass recomputes the
// log-odds of every voxel from the maps (exactly as the forward) and writes
// dLoss/dL = dLoss/docc occ (1 - occ); the pixel pass forms per pixel the sum
// of dLoss/dL over the voxels whose centre projects into it (its owner list),
// then the chain rule to the SLM, mean and variance.
struct BackwardArgs {
    FuseArgs f;                   // grid, cameras, maps (for the voxel pass), tiles
    const float *d_occ;           // [n_vox]
    float *dl;                    // dLoss/dL scratch: voxel v at dl[v * dl_stride]
    int dl_stride;                // 1 (one frame) or kBwRecord (records of the batched adjoint)
    // pixel pass
    const uint8_t *img;           // [n_pix][3] (NULL: `slm` given instead)
    const float *slm;             // [n_pix] caller-supplied SLM (psfs_backward_slm)
    const float *mean, *hinv;     // packed background
    float c0;
    SensorConsts sc;
    float da, one_minus_pd, db, one_minus_q;   // a(s), b(s) of Eq. 5-9
    float *d_slm, *d_mean, *d_var;             // outputs, any may be NULL
    int64_t n_pix;
};

cudaError_t launch_backward_voxel(const BackwardArgs &a, const FuseShape &shape, int map_dtype, cudaStream_t s);

// Batched persistent launch (psfs_batch.cu).  One kernel walks a list of work
// items over many frames, each frame with its own grid, cameras and
// background: likelihood chunks (kind 0) and fusion tiles (kind 1).  A fusion
// tile of frame f waits until every chunk of frame f is done (per-frame
// counter); items are ordered so that every item depends only on items with
// smaller indices, so the persistent grid always makes progress.
struct BatchFrame {
    FuseArgs fa;            // grid, cameras, tile plan, maps (batch-owned), outputs
    const uint8_t *img;     // [n_pix][3]
    const float *mean;      // packed background of the frame's handle
    const float *hinv;
    int64_t n_pix;
    uint32_t n_chunks;
    uint32_t wait_chunks;   // chunk count the fusion tiles wait for (n_chunks; more only in the hold test)
    float c0;
    SensorConsts sc;
};

constexpr int kBatchChunk = 512;   // pixels per likelihood item

__host__ __device__ inline uint64_t pack_item(uint32_t frame, uint32_t kind, uint64_t index)
{
    return ((uint64_t)frame << 40) | ((uint64_t)kind << 39) | index;
}

struct BatchLaunch {
    const BatchFrame *frames;   // device
    const uint64_t *items;      // device
    int64_t n_items;
    uint32_t *done;             // device, [n_frames] completed chunks (zeroed before the launch)
    uint32_t *status;
    int blocks;
    uint64_t wait_ns;           // limit of a fusion tile's wait for its frame's chunks
};

// cameras_per_block: the fusion items issue the loads of that many cameras
// together (1, 2 or 4; the sum stays in camera order); batch_shape_supported
// lists the instantiated combinations.
bool batch_shape_supported(const FuseShape &shape, int cameras_per_block);
cudaError_t launch_batch(const BatchLaunch &b, const FuseShape &shape, int cameras_per_block, int map_dtype,
                         cudaStream_t s);
void plan_pixel_rays(const psfs_grid &grid, const psfs_camera *cams, int n_cams, const FuseArgs &f,
                     PixelInv *inv);
// Owner lists of the adjoint's pixel pass (psfs_owners.cu): for every pixel
// of every camera, the voxels whose centre the forward projects into it, in
// ascending order: segment p is vox[off[p] .. off[p + 1]).  Buffers: cnt
// [n_pix], sums [ceil((n_pix + 1) / 4096)], off [n_pix + 1], vox [n_vox *
// n_cams].  Supported while n_vox * n_cams < 2^32.
bool owner_lists_supported(const FuseArgs &a, int64_t n_pix);
cudaError_t launch_build_owners(const FuseArgs &a, int64_t n_pix, uint32_t *cnt, uint32_t *sums, uint32_t *off,
                                uint32_t *vox, cudaStream_t s);
// Pixel pass of one frame (b.dl dense, dl_stride 1), and of n_frames <=
// 2 kBwRecord frames of records (frame f's colour at b.img + f img_fstride;
// frames kBwRecord and up in a second plane of records at b.dl + n_vox
// kBwRecord).
cudaError_t launch_owner_pixel(const BackwardArgs &b, const uint32_t *off, const uint32_t *vox, cudaStream_t s);
// dLoss/dL = d_occ occ (1 - occ) of n_frames frames (occ and d_occ [n_frames][n_vox]) from a given
// occupancy: dl[v * dl_stride + f] (dl_stride 1 with one frame, or kBwRecord).
cudaError_t launch_dl_from_occ(const float *occ, const float *d_occ, float *dl, int64_t n_vox, int n_frames,
                               int dl_stride, cudaStream_t s);
cudaError_t launch_owner_pixel_group(const BackwardArgs &b, const uint32_t *off, const uint32_t *vox, int n_frames,
                                     int64_t img_fstride, bool accumulate, cudaStream_t s);
cudaError_t launch_fuse(const FuseArgs &a, const FuseShape &shape, int map_dtype, cudaStream_t s);
cudaError_t launch_fuse_staged(const FuseArgs &a, const FuseShape &shape, int map_dtype, cudaStream_t s);

// Inner-voxel removal over the occupied-voxel lists of n frames
// (psfs_surface.cu): frame f's list at lists + f * list_stride with counts[f]
// entries, its occupancy bitmask at masks + f * mask_words (mask_words =
// ceil(n_vox / 32), zeroed by the launcher), its surface voxels appended at
// surface_lists + f * surface_capacity, counted in surface_counts[f].
struct SurfaceArgs {
    const uint32_t *lists;
    uint32_t list_stride;
    const uint32_t *counts;
    uint32_t *surface_lists;
    uint32_t surface_capacity;
    uint32_t *surface_counts;
    uint32_t *masks;
    uint32_t mask_words;
    uint32_t n_vox;
    int nx, ny, nz;
    uint32_t *status;
};
cudaError_t launch_surface(const SurfaceArgs &a, int n_frames, cudaStream_t s);

// Smoothing before the threshold (psfs_smooth.cu): frame f's probabilities at
// prob + f * n_vox, its smoothed grid (if not null) at smoothed + f * n_vox,
// its list at lists + f * capacity, its count at counts[f] (zeroed by the
// launcher).
struct SmoothArgs {
    CUtensorMap tmap;   // {nx, ny, nz, n_frames} over prob, boxes of 136 x 10 (smooth_tma_kernel)
    const float *prob;
    float *smoothed;
    uint32_t *lists;
    uint32_t capacity;
    uint32_t *counts;
    int nx, ny, nz;
    float threshold;
    uint32_t *status;
};
cudaError_t launch_smooth(const SmoothArgs &a, int n_frames, cudaStream_t s);

// Frame groups of the sequence path (psfs_group.cu), F = 2, 4, 8, 16 or 32
// frames: the F frames share one pass over the background (likelihood), and
// the fusion projects each voxel once per camera for all frames of a pixel
// record of `rec` = 32 or 64 bytes.  The group's maps are planes of such
// records: a record holds P = min(F, rec / map_elem) frames, plane q (frames
// qP to qP + P - 1) is [n_cams][H][W][P], and the F / P planes follow one
// another; one fusion launch per plane (two lanes per voxel when a record is
// 64 bytes).  Each frame's arithmetic is that of the single-frame kernels.
constexpr int kMaxGroup = 32;
inline int group_plane_frames(int frames, int map_elem, int rec = 32)
{
    return frames < rec / map_elem ? frames : rec / map_elem;
}
bool group_size_supported(int frames);
bool group_shape_supported(const FuseShape &s, int frames, int map_elem, int rec = 32);
cudaError_t launch_likelihood_group(const LikelihoodArgs &a, int frames, int map_dtype, cudaStream_t s,
                                    int ctas_per_sm, int rec = 32);
cudaError_t launch_fuse_group(const FuseArgs &a, const FuseShape &shape, int frames, int map_dtype,
                              cudaStream_t s, int rec = 32);
// The adjoint's voxel pass over a unit of `frames` (2, 4 or 8) frames whose
// maps are one plane of records ([n_pix][frames], b.f.maps), tile shape
// lanes_x 8 or 16, voxels_z 4: dLoss/dL of frame f into slot f of each
// voxel's record (b.dl points at the unit's first slot).
cudaError_t launch_backward_voxel_group(const BackwardArgs &b, const FuseShape &shape, int frames, int map_dtype,
                                        int64_t docc_fstride, cudaStream_t s);

// Host planning (psfs_plan.cu): projection matrices, tile order and staging
// records of the fuse kernel for one grid and camera rig.
void plan_fuse(const psfs_grid &grid, const psfs_camera *cams, int n_cams, const psfs_params &params,
               const FuseShape &shape, FuseArgs *out, std::vector<uint64_t> *tiles,
               std::vector<int4> *tilecam);

}  // namespace psfs
