// psfs_fuse.cu -- per-voxel stage of the reconstruction: projection of every
// voxel centre into every camera (Eq. 3), gather of the per-pixel log ratio,
// sum over cameras (log form of the product of Eq. 4), posterior, strict
// threshold and compaction of the occupied voxels.
//
// Work decomposition.  A CTA owns a tile of 32 (x) x WY (y) x TZ (z) voxels:
// each warp is one run of 32 voxels along x (128-byte occupancy stores) and
// each thread walks TZ voxels along z, sharing the x/y part of the
// projection.  CTAs are issued in Morton order of their tiles.
//
// Gather.  For each camera the CTA copies the image box that its voxel
// centres project into (computed on the host per tile and camera, 16-byte
// aligned rows) from the L2-resident map into shared memory with cp.async,
// then every voxel reads its pixel from shared memory.  A box that does not
// fit the buffer falls back to gathers from global memory.  When the host
// has proven that every voxel centre of the tile is in front of the camera
// and inside the image, the per-voxel visibility test is skipped.
//
// Compaction: per warp a ballot per z step, per CTA one atomicAdd on the
// global count, then each warp writes its indices at its prefix offset.
#include "psfs_internal.cuh"

namespace psfs {

namespace {

__device__ __forceinline__ void cp_async16(void *smem, const void *gmem)
{
    const uint32_t s = (uint32_t)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem) : "memory");
}

__device__ __forceinline__ void cp_async_wait_all()
{
    asm volatile("cp.async.commit_group;\ncp.async.wait_group 0;\n" ::: "memory");
}

template <typename T>
__device__ __forceinline__ float smem_load(const T *p);
template <>
__device__ __forceinline__ float smem_load<float>(const float *p) { return *p; }
template <>
__device__ __forceinline__ float smem_load<__half>(const __half *p) { return __half2float(*p); }
template <>
__device__ __forceinline__ float smem_load<__nv_bfloat16>(const __nv_bfloat16 *p)
{
    return __bfloat162float(*p);
}

template <typename MapT, int WY, int TZ>
__global__ void __launch_bounds__(32 * WY) fuse_kernel(const __grid_constant__ FuseArgs a)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    MapT *sbuf = reinterpret_cast<MapT *>(smem_raw);
    __shared__ uint32_t s_warp_off[WY];
    __shared__ uint32_t s_base;

    const int lane = threadIdx.x;
    const int wy = threadIdx.y;
    const int tid = wy * 32 + lane;
    const uint64_t tc = a.tiles[blockIdx.x];
    const int tx = (int)(tc & 0x1FFFFFu);
    const int ty = (int)((tc >> 21) & 0x1FFFFFu);
    const int tz = (int)(tc >> 42);
    const int i = tx * 32 + lane;
    const int j = ty * WY + wy;
    const int k0 = tz * TZ;
    // Lanes past the grid edge (ragged tiles) project the nearest voxel of the
    // grid instead, so every projection stays inside the tile's staged box;
    // their results are discarded below.
    const float fi = (float)min(i, a.nx - 1) - a.ci;
    const float fj = (float)min(j, a.ny - 1) - a.cj;
    const uint32_t W = (uint32_t)a.W, H = (uint32_t)a.H;
    constexpr int kChunk = 16 / (int)sizeof(MapT);   // elements per 16-byte copy

    float fk[TZ];
    float L[TZ];
#pragma unroll
    for (int t = 0; t < TZ; ++t) {
        fk[t] = (float)min(k0 + t, a.nz - 1) - a.ck;
        L[t] = 0.0f;
    }

    const MapT *maps = reinterpret_cast<const MapT *>(a.maps);
    const int4 *tcrec = a.tilecam + (int64_t)blockIdx.x * a.n_cams;
    for (int c = 0; c < a.n_cams; ++c) {
        const int4 rec = __ldg(tcrec + c);
        const int flags = rec.w >> 16;
        if (flags & kTcSkip) continue;
        const float *m = a.cam[c].m;
        const MapT *map = maps + (int64_t)c * a.map_stride;
        float bu, bv, bw;
        project_base(m, fi, fj, &bu, &bv, &bw);
        if (flags & kTcStaged) {
            const int bx0 = rec.x, by0 = rec.y, sw = rec.z, sh = rec.w & 0xFFFF;
            __syncthreads();   // the previous camera's gathers are done with the buffer
            const MapT *src = map + (int64_t)by0 * W + bx0;
            const int row_chunks = sw / kChunk;
            for (int r = wy; r < sh; r += WY)
                for (int q = lane; q < row_chunks; q += 32)
                    cp_async16(sbuf + r * sw + q * kChunk, src + (int64_t)r * W + q * kChunk);
            cp_async_wait_all();
            __syncthreads();
            const uint32_t ox = kFloorBias + (uint32_t)bx0, oy = kFloorBias + (uint32_t)by0;
            if (flags & kTcInside) {
                // the host proved every centre of the tile lands in the box; the
                // min() only keeps a violated proof from leaving the buffer
                const uint32_t last = (uint32_t)(sw * sh - 1);
#pragma unroll
                for (int t = 0; t < TZ; ++t) {
                    const Proj p = project_biased(m, bu, bv, bw, fk[t]);
                    L[t] += smem_load<MapT>(sbuf + min((p.by - oy) * (uint32_t)sw + (p.bx - ox), last));
                }
            } else {
#pragma unroll
                for (int t = 0; t < TZ; ++t) {
                    const Proj p = project_biased(m, bu, bv, bw, fk[t]);
                    const uint32_t sx = p.bx - ox, sy = p.by - oy;
                    if ((sx < (uint32_t)sw) & (sy < (uint32_t)sh)) L[t] += smem_load<MapT>(sbuf + sy * (uint32_t)sw + sx);
                }
            }
        } else {
#pragma unroll
            for (int t = 0; t < TZ; ++t) {
                int pix;
                if (proj_pixel(project_biased(m, bu, bv, bw, fk[t]), W, H, &pix)) L[t] += map_load<MapT>(map + pix);
            }
        }
    }
    (void)tid;

    // posterior, threshold, compaction
    const bool in_xy = (i < a.nx) && (j < a.ny);
    uint32_t ballots[TZ];
    uint32_t warp_count = 0;
#pragma unroll
    for (int t = 0; t < TZ; ++t) {
        const int k = k0 + t;
        const bool valid = in_xy && (k < a.nz);
        const float lo = L[t] + a.logit_prior;
        if (valid) {
            const uint32_t lin = (uint32_t)i + (uint32_t)a.nx * ((uint32_t)j + (uint32_t)a.ny * (uint32_t)k);
            __stcs(a.occ + lin, __fdividef(1.0f, 1.0f + __expf(-lo)));
        }
        ballots[t] = __ballot_sync(0xFFFFFFFFu, valid && (lo > a.logit_tau));
        warp_count += __popc(ballots[t]);
    }
    if (lane == 0) s_warp_off[wy] = warp_count;
    __syncthreads();
    if (wy == 0 && lane == 0) {
        uint32_t total = 0;
#pragma unroll
        for (int w = 0; w < WY; ++w) {
            const uint32_t cnt = s_warp_off[w];
            s_warp_off[w] = total;
            total += cnt;
        }
        uint32_t base = 0;
        if (total) {
            base = atomicAdd(a.count, total);
            if ((uint64_t)base + total > (uint64_t)a.capacity) atomicOr(a.status, kStatusCapacity);
        }
        s_base = base;
    }
    __syncthreads();
    uint32_t pos = s_base + s_warp_off[wy];
    const uint32_t lt_mask = (1u << lane) - 1u;
#pragma unroll
    for (int t = 0; t < TZ; ++t) {
        const uint32_t b = ballots[t];
        if ((b >> lane) & 1u) {
            const uint32_t p = pos + __popc(b & lt_mask);
            if (p < a.capacity) {
                const int k = k0 + t;
                a.list[p] = (uint32_t)i + (uint32_t)a.nx * ((uint32_t)j + (uint32_t)a.ny * (uint32_t)k);
            }
        }
        pos += __popc(b);
    }
}

template <typename MapT>
cudaError_t launch_typed(const FuseArgs &a, cudaStream_t s)
{
    auto kern = fuse_kernel<MapT, FUSE_WY, FUSE_TZ>;
    const int smem = a.smem_cap * (int)sizeof(MapT);
    static bool configured[64] = {false};
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev >= 0 && dev < 64 && !configured[dev]) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, FUSE_SMEM_BYTES);
        if (e != cudaSuccess) return e;
        configured[dev] = true;
    }
    kern<<<a.n_tiles, dim3(32, FUSE_WY), smem, s>>>(a);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_fuse(const FuseArgs &a, int map_dtype, cudaStream_t s)
{
    if (a.n_tiles <= 0) return cudaSuccess;
    if (map_dtype == PSFS_MAP_F16) return launch_typed<__half>(a, s);
    if (map_dtype == PSFS_MAP_BF16) return launch_typed<__nv_bfloat16>(a, s);
    return launch_typed<float>(a, s);
}

}  // namespace psfs
