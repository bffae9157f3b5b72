// psfs_fuse.cu -- per-voxel stage of the reconstruction: projection of every
// voxel centre into every camera (Eq. 3), gather of the per-pixel log ratio,
// sum over cameras (log form of the product of Eq. 4), posterior, strict
// threshold and compaction of the occupied voxels.
//
// Work decomposition.  A CTA owns a tile of LX (x) x (32/LX) WY (y) x TZ (z)
// voxels: each warp is an LX x 32/LX patch of one z-slice and each thread
// walks TZ voxels along z, sharing the x/y part of the projection.  With the
// cameras on a ring around the grid, a z-slice maps to a band of a few image
// rows, so a square-ish patch (LX = 8) gathers from a handful of 32-byte
// sectors per warp where a 32-voxel row along x spans over a hundred pixels.
// Occupancy stores stay whole sectors (LX consecutive floats per row).  CTAs
// are issued in Morton order of their tiles, so that neighbouring CTAs gather
// from neighbouring parts of the (L2-resident) maps.
//
// Gather.  The instruction stream per voxel and camera is kept minimal:
// three fma for (u, v, w), one approximate reciprocal, two fma with
// round-down that floor u / w and v / w into biased integers, one integer
// multiply-add for the pixel offset, one load, one add.  The host proves per
// (tile, camera) when every voxel centre is in front of the camera and inside
// the image; only the other tiles pay for the visibility test, and cameras
// that see nothing of a tile are skipped.
//
// Compaction: per warp a ballot per z step, per CTA one atomicAdd on the
// global count, then each warp writes its indices at its prefix offset.
#include "psfs_fuse_common.cuh"

namespace psfs {

namespace {

template <typename MapT, int LX, int WY, int TZ>
__global__ void __launch_bounds__(32 * WY) fuse_kernel(const __grid_constant__ FuseArgs a)
{
    __shared__ int s_flags[PSFS_MAX_CAMS];
    __shared__ uint32_t s_warp_off[WY];
    __shared__ uint32_t s_base;

    const int lane = threadIdx.x;
    const int wy = threadIdx.y;
    const int tid = wy * 32 + lane;
    if (tid < a.n_cams) s_flags[tid] = __ldg(&a.tilecam[(int64_t)blockIdx.x * a.n_cams + tid].w) >> 16;

    TileCoords<LX, WY, TZ> tc;
    tc.init(a, a.tiles[blockIdx.x], lane, wy);
    const uint32_t W = (uint32_t)a.W, H = (uint32_t)a.H;
    float L[TZ];
#pragma unroll
    for (int t = 0; t < TZ; ++t) L[t] = 0.0f;
    __syncthreads();

    const MapT *maps = reinterpret_cast<const MapT *>(a.maps);
    const uint32_t last_pix = W * H - 1u;
    const uint32_t bias_off = 0u - (kFloorBias * W + kFloorBias);
    int c = 0;
    while (c < a.n_cams) {
        const int flags = s_flags[c];
        const int flags1 = c + 1 < a.n_cams ? s_flags[c + 1] : kTcSkip;
        if ((flags & kTcInside) && (flags1 & kTcInside)) {
            // two proven cameras at once: all 2 TZ gathers in flight before
            // any add; the adds keep the camera order of the sequential sum
            float m0[12], m1[12];
#pragma unroll
            for (int q = 0; q < 12; ++q) {
                m0[q] = a.cam[c].m[q];
                m1[q] = a.cam[c + 1].m[q];
            }
            float bu0, bv0, bw0, bu1, bv1, bw1;
            project_base(m0, tc.fi, tc.fj, &bu0, &bv0, &bw0);
            project_base(m1, tc.fi, tc.fj, &bu1, &bv1, &bw1);
            const MapT *map0 = maps + (int64_t)c * a.map_stride, *map1 = map0 + a.map_stride;
            float g0[TZ], g1[TZ];
#pragma unroll
            for (int t = 0; t < TZ; ++t) {
                const Proj p0 = project_biased(m0, bu0, bv0, bw0, tc.fk[t]);
                const Proj p1 = project_biased(m1, bu1, bv1, bw1, tc.fk[t]);
                // the host proved both pixels lie in the image; min() only guards the buffer
                g0[t] = PSFS_IN_BOUNDS(proved_inside(p0, W, H), a.status)
                            ? map_load<MapT>(map0 + min(p0.by * W + p0.bx + bias_off, last_pix)) : 0.0f;
                g1[t] = PSFS_IN_BOUNDS(proved_inside(p1, W, H), a.status)
                            ? map_load<MapT>(map1 + min(p1.by * W + p1.bx + bias_off, last_pix)) : 0.0f;
            }
#pragma unroll
            for (int t = 0; t < TZ; ++t) L[t] = (L[t] + g0[t]) + g1[t];
            c += 2;
            continue;
        }
        if (!(flags & kTcSkip)) {
            float m[12];
#pragma unroll
            for (int q = 0; q < 12; ++q) m[q] = a.cam[c].m[q];
            float bu, bv, bw;
            project_base(m, tc.fi, tc.fj, &bu, &bv, &bw);
            gather_global<MapT, TZ>(m, bu, bv, bw, tc.fk, maps + (int64_t)c * a.map_stride, W, H,
                                    (flags & kTcInside) != 0, L, a.status);
        }
        ++c;
    }
    tile_epilogue<WY, TZ>(a, tc.i, tc.j, tc.k0, L, lane, wy, s_warp_off, &s_base);
}

}  // namespace

namespace {

template <typename MapT, int LX, int TZ>
cudaError_t launch_typed(const FuseArgs &a, cudaStream_t s)
{
    fuse_kernel<MapT, LX, 4, TZ><<<a.n_tiles, dim3(32, 4), 0, s>>>(a);
    return cudaGetLastError();
}

template <typename MapT>
cudaError_t launch_shape(const FuseArgs &a, const FuseShape &sh, cudaStream_t s)
{
    if (sh.wy != 4) return cudaErrorInvalidValue;
    if (sh.lx == 8) {
        if (sh.tz == 2) return launch_typed<MapT, 8, 2>(a, s);
        if (sh.tz == 4) return launch_typed<MapT, 8, 4>(a, s);
        if (sh.tz == 8) return launch_typed<MapT, 8, 8>(a, s);
        if (sh.tz == 16) return launch_typed<MapT, 8, 16>(a, s);
        return cudaErrorInvalidValue;
    }
    if (sh.lx == 16) {
        if (sh.tz == 2) return launch_typed<MapT, 16, 2>(a, s);
        if (sh.tz == 4) return launch_typed<MapT, 16, 4>(a, s);
        if (sh.tz == 8) return launch_typed<MapT, 16, 8>(a, s);
        if (sh.tz == 16) return launch_typed<MapT, 16, 16>(a, s);
        return cudaErrorInvalidValue;
    }
    if (sh.lx == 32) {
        if (sh.tz == 2) return launch_typed<MapT, 32, 2>(a, s);
        if (sh.tz == 4) return launch_typed<MapT, 32, 4>(a, s);
        if (sh.tz == 8) return launch_typed<MapT, 32, 8>(a, s);
        if (sh.tz == 16) return launch_typed<MapT, 32, 16>(a, s);
        return cudaErrorInvalidValue;
    }
    return cudaErrorInvalidValue;
}

}  // namespace

cudaError_t launch_fuse(const FuseArgs &a, const FuseShape &shape, int map_dtype, cudaStream_t s)
{
    if (a.n_tiles <= 0) return cudaSuccess;
    if (shape.staged) return launch_fuse_staged(a, shape, map_dtype, s);
    if (map_dtype == PSFS_MAP_F16) return launch_shape<__half>(a, shape, s);
    if (map_dtype == PSFS_MAP_BF16) return launch_shape<__nv_bfloat16>(a, shape, s);
    return launch_shape<float>(a, shape, s);
}

}  // namespace psfs
