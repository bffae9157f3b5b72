// psfs_fuse.cu -- per-voxel stage of the reconstruction: projection of every
// voxel centre into every camera (Eq. 3), gather of the per-pixel log ratio,
// sum over cameras (log form of the product of Eq. 4), posterior, strict
// threshold and compaction of the occupied voxels.
//
// Work decomposition.  A CTA owns a tile of 32 (x) x FUSE_WY (y) x FUSE_TZ (z)
// voxels: each warp is one run of 32 voxels along x, so the occupancy stores
// of a warp are 128 contiguous bytes and its 32 gathers of one camera land in
// a short projected segment of that camera's map; each thread walks FUSE_TZ
// voxels along z, sharing the x/y part of the projection.  CTAs are issued in
// Morton order of their tiles so that neighbouring CTAs gather neighbouring
// map regions.  Cameras are looped inside the thread; the per-voxel sum stays
// in registers.
//
// Compaction: per warp a ballot per z step, per CTA one atomicAdd on the
// global count, then each warp writes its indices at its prefix offset.
#include "psfs_internal.cuh"

namespace psfs {

namespace {

template <typename MapT, int WY, int TZ>
__global__ void __launch_bounds__(32 * WY) fuse_kernel(const __grid_constant__ FuseArgs a)
{
    __shared__ uint32_t s_warp_off[WY];
    __shared__ uint32_t s_base;

    const int lane = threadIdx.x;
    const int wy = threadIdx.y;
    const uint64_t tc = a.tiles[blockIdx.x];
    const int tx = (int)(tc & 0x1FFFFFu);
    const int ty = (int)((tc >> 21) & 0x1FFFFFu);
    const int tz = (int)(tc >> 42);
    const int i = tx * 32 + lane;
    const int j = ty * WY + wy;
    const int k0 = tz * TZ;
    const float fi = (float)i - a.ci;
    const float fj = (float)j - a.cj;
    const float Wf = (float)a.W, Hf = (float)a.H;

    float L[TZ];
#pragma unroll
    for (int t = 0; t < TZ; ++t) L[t] = 0.0f;

    const MapT *maps = reinterpret_cast<const MapT *>(a.maps);
    for (int c = 0; c < a.n_cams; ++c) {
        const float *m = a.cam[c].m;
        const MapT *map = maps + (int64_t)c * a.map_stride;
#pragma unroll
        for (int t = 0; t < TZ; ++t) {
            const float fk = (float)(k0 + t) - a.ck;
            int pix;
            if (project_voxel(m, fi, fj, fk, Wf, Hf, a.W, &pix)) L[t] += map_load<MapT>(map + pix);
        }
    }

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
            __stcs(a.occ + lin, 1.0f / (1.0f + expf(-lo)));
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
            const uint32_t c = s_warp_off[w];
            s_warp_off[w] = total;
            total += c;
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

}  // namespace

cudaError_t launch_fuse(const FuseArgs &a, int map_dtype, cudaStream_t s)
{
    if (a.n_tiles <= 0) return cudaSuccess;
    const dim3 block(32, FUSE_WY);
    if (map_dtype == PSFS_MAP_F16) {
        fuse_kernel<__half, FUSE_WY, FUSE_TZ><<<a.n_tiles, block, 0, s>>>(a);
    } else if (map_dtype == PSFS_MAP_BF16) {
        fuse_kernel<__nv_bfloat16, FUSE_WY, FUSE_TZ><<<a.n_tiles, block, 0, s>>>(a);
    } else {
        fuse_kernel<float, FUSE_WY, FUSE_TZ><<<a.n_tiles, block, 0, s>>>(a);
    }
    return cudaGetLastError();
}

}  // namespace psfs
