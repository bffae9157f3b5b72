// psfs_noalloc.cu -- psfs_reconstruct_noalloc: one frame of the
// reconstruction without any device (or host heap) allocation.
//
// Some callers cannot call cudaMalloc: hosts that own every byte of device
// memory and hand plug-ins fixed buffers, or latency-critical capture loops
// that must not hit the implicit synchronisation of an allocation.  For them
// this entry point takes the grid, cameras, parameters, background, image and
// output buffers as arguments and keeps its only scratch (the per-pixel log
// ratio maps of one frame and a status word) in a file-scope __device__ array
// of fixed size.  Every GPU that loads the library holds that array
// (PSFS_NOALLOC_MAX_PIXELS floats plus 256 bytes) until the process exits.
//
// All calls share the array and it keeps the last call's contents: the
// status word and the caller's count are cleared by the first kernel of each
// call, and the maps are fully rewritten before they are read.  The status
// word only gives the fusion epilogue somewhere to record an overflow; no
// call reads it back, so a caller learns of an overflow from count >
// capacity alone.  Calls that
// overlap on the GPU (different streams, no ordering between them) race on
// the maps and give wrong results; order them on one stream.
//
// The arithmetic is that of psfs_reconstruct (same formulas, same camera
// order), computed with plain loads: the background is read as mean and
// variance (h = 1/(2 var) formed per pixel, as psfs_set_background forms it),
// tiles are taken in raster order and every camera takes the checked
// visibility test.
#include <cmath>
#include <cstring>
#include <mutex>

#include "psfs_fuse_common.cuh"

namespace psfs {

namespace {

constexpr int kNoallocHeaderWords = 64;   // word 0: status word; 256 bytes keep the maps aligned
constexpr int kNoallocLX = 8, kNoallocWY = 4, kNoallocTZ = 16;

// The scratch of psfs_reconstruct_noalloc.  Host code must not use this name
// as an address: it is a host-side stand-in for the device symbol; the device
// address comes from cudaGetSymbolAddress (scratch_on_current_device).
static __device__ __align__(256) uint32_t g_noalloc_scratch[kNoallocHeaderWords + PSFS_NOALLOC_MAX_PIXELS];

// Eq. 1-2 and the log ratio of Eq. 5-9 per pixel, from the raw background.
__global__ void __launch_bounds__(256) noalloc_likelihood_kernel(const uint8_t *img, const float *mean,
                                                                 const float *var, int64_t n_pix, float c0,
                                                                 SensorConsts sc, float *maps, uint32_t *count,
                                                                 uint32_t *status)
{
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        *count = 0u;
        *status = 0u;
    }
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < n_pix; p += stride) {
        const float h0 = 0.5f / var[3 * p], h1 = 0.5f / var[3 * p + 1], h2 = 0.5f / var[3 * p + 2];
        const float r = pixel_log_odds((float)img[3 * p], (float)img[3 * p + 1], (float)img[3 * p + 2], mean[3 * p],
                                       mean[3 * p + 1], mean[3 * p + 2], h0, h1, h2, c0);
        maps[p] = log_ratio_of_r(r, sc);
    }
}

// Eq. 3-9, threshold and compaction over raster-ordered tiles of 8 x 16 x 16
// voxels, every camera with the visibility test.
__global__ void __launch_bounds__(32 * kNoallocWY) noalloc_fuse_kernel(const __grid_constant__ FuseArgs a, int ntx,
                                                                       int nty)
{
    __shared__ uint32_t s_warp_off[kNoallocWY];
    __shared__ uint32_t s_base;
    const int lane = threadIdx.x, wy = threadIdx.y;
    const int b = blockIdx.x;
    const uint64_t tc = pack_tile((uint32_t)(b % ntx), (uint32_t)((b / ntx) % nty), (uint32_t)(b / (ntx * nty)));
    TileCoords<kNoallocLX, kNoallocWY, kNoallocTZ> t;
    t.init(a, tc, lane, wy);
    const uint32_t W = (uint32_t)a.W, H = (uint32_t)a.H;
    const float *maps = reinterpret_cast<const float *>(a.maps);
    float L[kNoallocTZ];
#pragma unroll
    for (int z = 0; z < kNoallocTZ; ++z) L[z] = 0.0f;
    for (int c = 0; c < a.n_cams; ++c) {
        float m[12];
#pragma unroll
        for (int q = 0; q < 12; ++q) m[q] = a.cam[c].m[q];
        float bu, bv, bw;
        project_base(m, t.fi, t.fj, &bu, &bv, &bw);
        gather_global<float, kNoallocTZ>(m, bu, bv, bw, t.fk, maps + (int64_t)c * a.map_stride, W, H, false, L);
    }
    tile_epilogue<kNoallocWY, kNoallocTZ>(a, t.i, t.j, t.k0, L, lane, wy, s_warp_off, &s_base);
}

// Device address of the scratch on the current device, set up once per
// device (the first call on a device does it).
std::mutex g_noalloc_mu;
uint32_t *g_noalloc_ptr[64] = {nullptr};

cudaError_t scratch_on_current_device(uint32_t **out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    if (!g_noalloc_ptr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return e;
        g_noalloc_ptr[dev] = reinterpret_cast<uint32_t *>(p);
    }
    *out = g_noalloc_ptr[dev];
    return cudaSuccess;
}

bool finite_n(const double *v, int n)
{
    for (int i = 0; i < n; ++i)
        if (!std::isfinite(v[i])) return false;
    return true;
}

bool aligned4(const void *p) { return ((uintptr_t)p & 3u) == 0; }

}  // namespace

}  // namespace psfs

using namespace psfs;

extern "C" psfs_status psfs_reconstruct_noalloc(const psfs_grid *grid, const psfs_camera *cams, int32_t n_cams,
                                                const psfs_params *params, const float *mean, const float *var,
                                                const uint8_t *images, float *occupancy, uint32_t *voxel_list,
                                                uint32_t capacity, uint32_t *count, void *stream)
{
    // argument checks: those psfs_create and psfs_reconstruct make, each
    // recorded for psfs_last_error_message
    auto bad = [](const char *what) { return record_failure(PSFS_ERR_INVALID_ARG, what); };
    if (!grid || !cams || !params) return bad("grid, cams or params is NULL");
    if (!mean || !var || !images || !occupancy || !count) return bad("a device buffer is NULL");
    if (capacity > 0 && !voxel_list) return bad("voxel_list is NULL with capacity > 0");
    if (!aligned4(mean) || !aligned4(var) || !aligned4(occupancy) || !aligned4(count) ||
        (voxel_list && !aligned4(voxel_list)))
        return bad("a float or uint32 device buffer is not 4-byte aligned");
    if (n_cams < 1 || n_cams > PSFS_MAX_CAMS) return bad("n_cams outside [1, PSFS_MAX_CAMS]");
    if (params->map_dtype != PSFS_MAP_F32) return bad("params->map_dtype must be PSFS_MAP_F32");
    const double pv[5] = {params->p_detect, params->p_false_alarm, params->prior, params->threshold,
                          params->log_fg_density};
    if (!finite_n(pv, 5) || params->p_detect < 0 || params->p_detect > 1 || params->p_false_alarm < 0 ||
        params->p_false_alarm > 1 || !(params->prior > 0 && params->prior < 1) ||
        !(params->threshold > 0 && params->threshold < 1))
        return bad("params out of range (rates in [0, 1], prior and threshold in (0, 1), all finite)");
    const double pd = params->p_detect, q = 0.5 * (params->p_detect + params->p_false_alarm);
    if (!(q > 0 && q < 1)) return bad("(p_detect + p_false_alarm) / 2 must lie in (0, 1)");
    if (grid->nx < 1 || grid->ny < 1 || grid->nz < 1 || !finite_n(grid->origin, 3) ||
        !std::isfinite(grid->voxel_size) || !(grid->voxel_size > 0))
        return bad("grid sizes < 1, or origin / voxel_size not finite and positive");
    // tile coordinates are packed in 21 bits per axis and voxel indices must
    // stay exact in float32 (the same limit as psfs_create)
    if (grid->nx > (1 << 24) || grid->ny > (1 << 24) || grid->nz > (1 << 24))
        return bad("grid axis longer than 2^24");
    if ((uint64_t)grid->nx * grid->ny * grid->nz >= (1ull << 32)) return bad("grid has 2^32 or more voxels");
    const int W = cams[0].width, H = cams[0].height;
    if (W < 1 || H < 1 || W > 16384 || H > 16384) return bad("image size outside [1, 16384]");
    for (int c = 0; c < n_cams; ++c)
        if (cams[c].width != W || cams[c].height != H || !finite_n(cams[c].K, 9) || !finite_n(cams[c].R, 9) ||
            !finite_n(cams[c].t, 3))
            return bad("cameras differ in image size or have non-finite K, R or t");
    const int64_t n_pix = (int64_t)n_cams * W * H;
    if (n_pix > (int64_t)PSFS_NOALLOC_MAX_PIXELS)
        return bad("n_cams * height * width exceeds PSFS_NOALLOC_MAX_PIXELS (the fixed scratch)");

    uint32_t *scratch = nullptr;
    {
        const cudaError_t e = scratch_on_current_device(&scratch);
        if (e != cudaSuccess) return record_cuda_failure(e, "device address of the no-alloc scratch");
    }
    uint32_t *status = scratch;
    float *maps = reinterpret_cast<float *>(scratch + kNoallocHeaderWords);

    // kernel arguments, formed on the stack in double precision as psfs_create forms them
    SensorConsts sc{};
    sc.pd = (float)pd;
    sc.one_minus_pd = (float)(1.0 - pd);
    sc.q = (float)q;
    sc.one_minus_q = (float)(1.0 - q);
    sc.a_zero_const_pos = (pd == 0.0);
    sc.a_zero_const_neg = (pd == 1.0);
    const float c0 = (float)(params->log_fg_density + 1.5 * std::log(M_PI));
    FuseArgs f{};
    std::memset(&f, 0, sizeof(f));
    f.maps = maps;
    f.W = W;
    f.H = H;
    f.map_stride = (int64_t)W * H;
    f.n_cams = n_cams;
    f.nx = grid->nx;
    f.ny = grid->ny;
    f.nz = grid->nz;
    f.ci = 0.5f * (float)(grid->nx - 1);
    f.cj = 0.5f * (float)(grid->ny - 1);
    f.ck = 0.5f * (float)(grid->nz - 1);
    const double vs = grid->voxel_size;
    const double centre[3] = {grid->origin[0] + 0.5 * grid->nx * vs, grid->origin[1] + 0.5 * grid->ny * vs,
                              grid->origin[2] + 0.5 * grid->nz * vs};
    for (int c = 0; c < n_cams; ++c) {
        const double *K = cams[c].K, *R = cams[c].R, *t = cams[c].t;
        double KR[9], xc[3];
        for (int r = 0; r < 3; ++r) {
            for (int col = 0; col < 3; ++col)
                KR[3 * r + col] = K[3 * r + 0] * R[0 + col] + K[3 * r + 1] * R[3 + col] + K[3 * r + 2] * R[6 + col];
            xc[r] = R[3 * r + 0] * centre[0] + R[3 * r + 1] * centre[1] + R[3 * r + 2] * centre[2] + t[r];
        }
        for (int r = 0; r < 3; ++r) {
            for (int col = 0; col < 3; ++col) f.cam[c].m[4 * r + col] = (float)(KR[3 * r + col] * vs);
            f.cam[c].m[4 * r + 3] = (float)(K[3 * r + 0] * xc[0] + K[3 * r + 1] * xc[1] + K[3 * r + 2] * xc[2]);
        }
    }
    f.logit_prior = (float)std::log(params->prior / (1.0 - params->prior));
    f.logit_tau = (float)std::log(params->threshold / (1.0 - params->threshold));
    f.occ = occupancy;
    f.list = voxel_list;
    f.capacity = capacity;
    f.count = count;
    f.status = status;
    const int ntx = (grid->nx + kNoallocLX - 1) / kNoallocLX;
    const int nty = (grid->ny + (32 / kNoallocLX) * kNoallocWY - 1) / ((32 / kNoallocLX) * kNoallocWY);
    const int ntz = (grid->nz + kNoallocTZ - 1) / kNoallocTZ;
    const int64_t n_tiles = (int64_t)ntx * nty * ntz;
    if (n_tiles > 0x7FFFFFFF) return bad("grid has too many tiles for one launch");
    f.n_tiles = (int)n_tiles;

    cudaStream_t s = (cudaStream_t)stream;
    int64_t blocks = (n_pix + 255) / 256;
    const int64_t cap = 8 * (int64_t)device_sm_count();   // grid-stride loop: any size is correct
    if (blocks > cap) blocks = cap;
    noalloc_likelihood_kernel<<<(int)blocks, 256, 0, s>>>(images, mean, var, n_pix, c0, sc, maps, count, status);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return record_cuda_failure(e, "no-alloc likelihood launch");
    noalloc_fuse_kernel<<<(int)n_tiles, dim3(32, kNoallocWY), 0, s>>>(f, ntx, nty);
    e = cudaGetLastError();
    if (e != cudaSuccess) return record_cuda_failure(e, "no-alloc fusion launch");
    return PSFS_OK;
}
