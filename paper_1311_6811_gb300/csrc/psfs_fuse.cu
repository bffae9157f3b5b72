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
#include "psfs_internal.cuh"

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

    const uint64_t tc = a.tiles[blockIdx.x];
    const int tx = (int)(tc & 0x1FFFFFu);
    const int ty = (int)((tc >> 21) & 0x1FFFFFu);
    const int tz = (int)(tc >> 42);
    constexpr int LY = 32 / LX;
    const int i = tx * LX + (lane % LX);
    const int j = ty * (LY * WY) + wy * LY + lane / LX;
    const int k0 = tz * TZ;
    // Lanes past the grid edge (ragged tiles) project the nearest voxel of the
    // grid instead, so that the host's per-tile proofs cover them; their
    // results are discarded below.
    const float fi = (float)min(i, a.nx - 1) - a.ci;
    const float fj = (float)min(j, a.ny - 1) - a.cj;
    const uint32_t W = (uint32_t)a.W, H = (uint32_t)a.H;
    const uint32_t last_pix = W * H - 1u;
    // pixel offset from biased coordinates: (by - B) W + (bx - B) = by W + bx + bias_off (mod 2^32)
    const uint32_t bias_off = 0u - (kFloorBias * W + kFloorBias);

    float fk[TZ];
    float L[TZ];
#pragma unroll
    for (int t = 0; t < TZ; ++t) {
        fk[t] = (float)min(k0 + t, a.nz - 1) - a.ck;
        L[t] = 0.0f;
    }
    __syncthreads();

    const MapT *maps = reinterpret_cast<const MapT *>(a.maps);
    for (int c = 0; c < a.n_cams; ++c) {
        const int flags = s_flags[c];
        if (flags & kTcSkip) continue;
        float m[12];
#pragma unroll
        for (int q = 0; q < 12; ++q) m[q] = a.cam[c].m[q];
        const MapT *map = maps + (int64_t)c * a.map_stride;
        float bu, bv, bw;
        project_base(m, fi, fj, &bu, &bv, &bw);
        if (flags & kTcInside) {
#pragma unroll
            for (int t = 0; t < TZ; ++t) {
                const Proj p = project_biased(m, bu, bv, bw, fk[t]);
                // the host proved the pixel lies in the image; min() only guards the buffer
                L[t] += map_load<MapT>(map + min(p.by * W + p.bx + bias_off, last_pix));
            }
        } else {
#pragma unroll
            for (int t = 0; t < TZ; ++t) {
                int pix;
                if (proj_pixel(project_biased(m, bu, bv, bw, fk[t]), W, H, &pix)) L[t] += map_load<MapT>(map + pix);
            }
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
            __stcs(a.occ + lin, __fdividef(1.0f, 1.0f + __expf(-lo)));
        }
        ballots[t] = __ballot_sync(0xFFFFFFFFu, valid && (lo > a.logit_tau));
        warp_count += __popc(ballots[t]);
    }
    if (lane == 0) s_warp_off[wy] = warp_count;
    __syncthreads();
    if (tid == 0) {
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
    if (sh.lx == 8) return sh.tz == 8 ? launch_typed<MapT, 8, 8>(a, s) : launch_typed<MapT, 8, 16>(a, s);
    if (sh.lx == 16) return sh.tz == 8 ? launch_typed<MapT, 16, 8>(a, s) : launch_typed<MapT, 16, 16>(a, s);
    if (sh.lx == 32) return sh.tz == 8 ? launch_typed<MapT, 32, 8>(a, s) : launch_typed<MapT, 32, 16>(a, s);
    return cudaErrorInvalidValue;
}

}  // namespace

cudaError_t launch_fuse(const FuseArgs &a, const FuseShape &shape, int map_dtype, cudaStream_t s)
{
    if (a.n_tiles <= 0) return cudaSuccess;
    if (map_dtype == PSFS_MAP_F16) return launch_shape<__half>(a, shape, s);
    if (map_dtype == PSFS_MAP_BF16) return launch_shape<__nv_bfloat16>(a, shape, s);
    return launch_shape<float>(a, shape, s);
}

}  // namespace psfs
