// psfs_fuse_common.cuh -- pieces shared by the two fusion kernels (direct
// gathers and shared-memory staged gathers): the voxel coordinates a thread
// owns in a tile, and the tile epilogue (posterior, strict threshold,
// compaction of the occupied voxels).
#pragma once

#include "psfs_internal.cuh"

namespace psfs {

// Voxel coordinates of a thread in tile `tc`: lane % LX along x, lane / LX
// and the warp index along y, TZ consecutive voxels along z.  Lanes past the
// grid edge (ragged tiles) project the nearest voxel of the grid instead, so
// that the host's per-tile proofs cover them; their results are discarded by
// the epilogue.
template <int LX, int WY, int TZ>
struct TileCoords {
    int i, j, k0;
    float fi, fj;
    float fk[TZ];

    __device__ __forceinline__ void init(const FuseArgs &a, uint64_t tc, int lane, int wy)
    {
        constexpr int LY = 32 / LX;
        const int tx = (int)(tc & 0x1FFFFFu);
        const int ty = (int)((tc >> 21) & 0x1FFFFFu);
        const int tz = (int)(tc >> 42);
        i = tx * LX + (lane % LX);
        j = ty * (LY * WY) + wy * LY + lane / LX;
        k0 = tz * TZ;
        fi = (float)min(i, a.nx - 1) - a.ci;
        fj = (float)min(j, a.ny - 1) - a.cj;
#pragma unroll
        for (int t = 0; t < TZ; ++t) fk[t] = (float)min(k0 + t, a.nz - 1) - a.ck;
    }
};

// Posterior 1 / (1 + e^-L) (written to the occupancy grid), strict
// threshold L > logit(threshold), and compaction: a ballot per z step per
// warp, one atomicAdd per CTA on the global count, then each warp writes its
// indices at its prefix offset.  Contains two __syncthreads.
template <int WY, int TZ>
__device__ __forceinline__ void tile_epilogue_to(const FuseArgs &a, float *occ, uint32_t *list, uint32_t *count,
                                                 int i, int j, int k0, const float *L, int lane, int wy,
                                                 uint32_t *s_warp_off, uint32_t *s_base)
{
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
            __stcs(occ + lin, posterior_of_logodds(lo));
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
            base = atomicAdd(count, total);
            if ((uint64_t)base + total > (uint64_t)a.capacity) atomicOr(a.status, kStatusCapacity);
        }
        *s_base = base;
    }
    __syncthreads();
    uint32_t pos = *s_base + s_warp_off[wy];
    const uint32_t lt_mask = (1u << lane) - 1u;
#pragma unroll
    for (int t = 0; t < TZ; ++t) {
        const uint32_t b = ballots[t];
        if ((b >> lane) & 1u) {
            const uint32_t p = pos + __popc(b & lt_mask);
            if (p < a.capacity) {
                const int k = k0 + t;
                list[p] = (uint32_t)i + (uint32_t)a.nx * ((uint32_t)j + (uint32_t)a.ny * (uint32_t)k);
            }
        }
        pos += __popc(b);
    }
}

// The epilogue into the frame's own outputs a.occ, a.list, a.count.
template <int WY, int TZ>
__device__ __forceinline__ void tile_epilogue(const FuseArgs &a, int i, int j, int k0, const float *L, int lane,
                                              int wy, uint32_t *s_warp_off, uint32_t *s_base)
{
    tile_epilogue_to<WY, TZ>(a, a.occ, a.list, a.count, i, j, k0, L, lane, wy, s_warp_off, s_base);
}

// One camera's contribution to the TZ voxels of a thread, gathering from
// global memory.  `inside`: the host proved every voxel centre of the tile is
// in front of the camera and inside the image, so no test is made.
// kCoherent: load the maps through the coherent path (maps written by other
// CTAs of the same kernel).
template <typename MapT, int TZ, bool kCoherent = false>
__device__ __forceinline__ float gather_load(const MapT *p)
{
    if (kCoherent) return map_load_coherent(p);
    return map_load<MapT>(p);
}

// The planner's claim for a tile and camera marked inside: the voxel's pixel
// lies in the image (tested in the bounds-checked build only).
__device__ __forceinline__ bool proved_inside(const Proj &p, uint32_t W, uint32_t H)
{
    return (p.bx - kFloorBias) < W && (p.by - kFloorBias) < H;
}

template <typename MapT, int TZ, bool kCoherent = false>
__device__ __forceinline__ void gather_global(const float *m, float bu, float bv, float bw, const float *fk,
                                              const MapT *map, uint32_t W, uint32_t H, bool inside, float *L,
                                              uint32_t *status = nullptr)
{
    (void)status;
    if (inside) {
        const uint32_t last_pix = W * H - 1u;
        // (by - B) W + (bx - B) = by W + bx + bias_off (mod 2^32)
        const uint32_t bias_off = 0u - (kFloorBias * W + kFloorBias);
#pragma unroll
        for (int t = 0; t < TZ; ++t) {
            const Proj p = project_biased(m, bu, bv, bw, fk[t]);
            // the host proved the pixel lies in the image; min() only guards the buffer
            if (PSFS_IN_BOUNDS(proved_inside(p, W, H), status))
                L[t] += gather_load<MapT, TZ, kCoherent>(map + min(p.by * W + p.bx + bias_off, last_pix));
        }
    } else {
#pragma unroll
        for (int t = 0; t < TZ; ++t) {
            int pix;
            if (proj_pixel(project_biased(m, bu, bv, bw, fk[t]), W, H, &pix))
                L[t] += gather_load<MapT, TZ, kCoherent>(map + pix);
        }
    }
}

}  // namespace psfs
