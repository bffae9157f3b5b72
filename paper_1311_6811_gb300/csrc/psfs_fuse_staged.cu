// psfs_fuse_staged.cu -- the fusion stage (Eq. 3-9, threshold, compaction)
// with the gathers served from shared memory.
//
// A persistent grid (three CTAs per SM) walks its tiles round-robin; for each
// tile it visits the cameras in order.  Every (tile, camera) step has an
// image box planned on the host (the pixels its voxel centres project into,
// 16-byte aligned origin).  One thread copies the box of step s + 2 into one
// of two shared-memory buffers as a few tensor-map boxes (TMA: 16 rows of 32,
// 64 or 128 elements each, stacked so that the buffer is a dense
// [rows][box width] array), signalled on an mbarrier, while all threads
// gather step s from the other buffer.  A warp's 32 gathers then cost a
// shared-memory wavefront or two instead of the dozen 32-byte L1 sectors that
// the same gathers touch in global memory.  Steps whose box is too wide or
// too tall for a buffer gather from global memory within the same pipeline;
// steps whose camera sees nothing of the tile do nothing.
#include <algorithm>

#include "psfs_fuse_common.cuh"

namespace psfs {

namespace {

template <typename T>
__device__ __forceinline__ float smem_load(const T *p);
template <>
__device__ __forceinline__ float smem_load<float>(const float *p) { return *p; }
template <>
__device__ __forceinline__ float smem_load<__half>(const __half *p) { return __half2float(*p); }
template <>
__device__ __forceinline__ float smem_load<__nv_bfloat16>(const __nv_bfloat16 *p) { return __bfloat162float(*p); }

template <typename MapT, int LX, int WY, int TZ>
__global__ void __launch_bounds__(32 * WY) fuse_staged_kernel(const __grid_constant__ FuseArgs a)
{
    extern __shared__ __align__(128) unsigned char smem_raw[];
    // tensor copies land on 128-byte boundaries: round the dynamic window up
    unsigned char *smem = smem_raw + ((128u - (smem_u32(smem_raw) & 127u)) & 127u);
    auto buf = [&](int b) { return reinterpret_cast<MapT *>(smem + b * kStageBytes); };
    uint64_t *bars = reinterpret_cast<uint64_t *>(smem + 2 * kStageBytes);
    __shared__ uint32_t s_warp_off[WY];
    __shared__ uint32_t s_base;

    const int lane = threadIdx.x;
    const int wy = threadIdx.y;
    const int tid = wy * 32 + lane;
    const int K = a.n_cams;
    const uint32_t W = (uint32_t)a.W, H = (uint32_t)a.H;
    const MapT *maps = reinterpret_cast<const MapT *>(a.maps);

    if (tid == 0) {
        mbar_init(&bars[0], 1);
        mbar_init(&bars[1], 1);
        mbar_fence_init();
    }
    __syncthreads();

    const int64_t my_tiles =
        (int64_t)blockIdx.x < a.n_tiles ? ((int64_t)a.n_tiles - 1 - blockIdx.x) / gridDim.x + 1 : 0;
    const int64_t n_steps = my_tiles * K;

    // step s: tile blockIdx.x + (s / K) * gridDim.x, camera s % K, buffer s & 1
    const bool use_tma = a.tmap_ok != 0;
    auto issue = [&](int64_t s) {
        const int b = (int)(s & 1);
        const int64_t tile = (int64_t)blockIdx.x + (s / K) * gridDim.x;
        const int c = (int)(s % K);
        const int4 rec = __ldg(&a.tilecam[tile * K + c]);
        const int flags = rec.w >> 16;
        if (use_tma && (flags & kTcStaged)) {
            const int cls = (rec.z >> 16) & 3, nby = rec.z >> 18;
            const uint32_t box_bytes = (uint32_t)((32 << cls) * kBoxRows * (int)sizeof(MapT));
            mbar_arrive_expect_tx(&bars[b], box_bytes * (uint32_t)nby);
            for (int q = 0; q < nby; ++q)
                tma_load_3d(reinterpret_cast<unsigned char *>(buf(b)) + (size_t)q * box_bytes, &a.tmap[cls], rec.x,
                            rec.y + q * kBoxRows, c, &bars[b]);
        } else {
            mbar_arrive(&bars[b]);   // nothing to copy: complete the phase at once
        }
    };
    if (tid == 0)
        for (int64_t s = 0; s < 2 && s < n_steps; ++s) issue(s);

    TileCoords<LX, WY, TZ> tc;
    float L[TZ];
    for (int64_t s = 0; s < n_steps; ++s) {
        const int c = (int)(s % K);
        const int64_t tile = (int64_t)blockIdx.x + (s / K) * gridDim.x;
        if (c == 0) {
            tc.init(a, a.tiles[tile], lane, wy);
#pragma unroll
            for (int t = 0; t < TZ; ++t) L[t] = 0.0f;
        }
        const int b = (int)(s & 1);
        mbar_wait_bounded(&bars[b], (uint32_t)((s >> 1) & 1), a.status);
        const int4 rec = __ldg(&a.tilecam[tile * K + c]);
        const int flags = rec.w >> 16;
        if (!(flags & kTcSkip)) {
            float m[12];
#pragma unroll
            for (int q = 0; q < 12; ++q) m[q] = a.cam[c].m[q];
            float bu, bv, bw;
            project_base(m, tc.fi, tc.fj, &bu, &bv, &bw);
            if (use_tma && (flags & kTcStaged)) {
                const MapT *sb = buf(b);
                // clipped extents; the buffer is [nby * 16 rows][32 << cls]
                const uint32_t sw = (uint32_t)(rec.z & 0xFFFF), sh = (uint32_t)(rec.w & 0xFFFF);
                const uint32_t pitch = 32u << ((rec.z >> 16) & 3);
                const uint32_t ox = kFloorBias + (uint32_t)rec.x, oy = kFloorBias + (uint32_t)rec.y;
                if (flags & kTcInside) {
                    // the host proved every centre lands in the box; min() only guards the buffer
                    const uint32_t last = (uint32_t)(rec.z >> 18) * kBoxRows * pitch - 1u;
#pragma unroll
                    for (int t = 0; t < TZ; ++t) {
                        const Proj p = project_biased(m, bu, bv, bw, tc.fk[t]);
                        L[t] += smem_load<MapT>(sb + min((p.by - oy) * pitch + (p.bx - ox), last));
                    }
                } else {
                    // the box is the seen part of the tile's footprint, clipped to the image
#pragma unroll
                    for (int t = 0; t < TZ; ++t) {
                        const Proj p = project_biased(m, bu, bv, bw, tc.fk[t]);
                        const uint32_t sx = p.bx - ox, sy = p.by - oy;
                        if ((sx < sw) & (sy < sh)) L[t] += smem_load<MapT>(sb + sy * pitch + sx);
                    }
                }
            } else {
                gather_global<MapT, TZ>(m, bu, bv, bw, tc.fk, maps + (int64_t)c * a.map_stride, W, H,
                                        (flags & kTcInside) != 0, L, a.status);
            }
        }
        __syncthreads();   // every thread is done with buffer b
        if (tid == 0 && s + 2 < n_steps) issue(s + 2);
        if (c == K - 1) tile_epilogue<WY, TZ>(a, tc.i, tc.j, tc.k0, L, lane, wy, s_warp_off, &s_base);
    }
}

template <typename MapT, int LX, int TZ>
cudaError_t launch_typed(const FuseArgs &a, cudaStream_t s)
{
    auto kern = fuse_staged_kernel<MapT, LX, 4, TZ>;
    constexpr int smem = 2 * kStageBytes + 16 + 128;
    static bool configured[64] = {false};
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev >= 0 && dev < 64 && !configured[dev]) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        if (e != cudaSuccess) return e;
        configured[dev] = true;
    }
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int blocks = std::max(1, std::min(a.n_tiles, kStagedCtasPerSm * std::max(sms, 1)));
    kern<<<blocks, dim3(32, 4), smem, s>>>(a);
    return cudaGetLastError();
}

template <typename MapT>
cudaError_t launch_shape(const FuseArgs &a, const FuseShape &sh, cudaStream_t s)
{
    if (sh.wy != 4) return cudaErrorInvalidValue;
    if (sh.lx == 8 && (sh.tz == 8 || sh.tz == 16))
        return sh.tz == 8 ? launch_typed<MapT, 8, 8>(a, s) : launch_typed<MapT, 8, 16>(a, s);
    if (sh.lx == 16 && (sh.tz == 8 || sh.tz == 16))
        return sh.tz == 8 ? launch_typed<MapT, 16, 8>(a, s) : launch_typed<MapT, 16, 16>(a, s);
    if (sh.lx == 32 && (sh.tz == 8 || sh.tz == 16))
        return sh.tz == 8 ? launch_typed<MapT, 32, 8>(a, s) : launch_typed<MapT, 32, 16>(a, s);
    return cudaErrorInvalidValue;
}

}  // namespace

cudaError_t launch_fuse_staged(const FuseArgs &a, const FuseShape &shape, int map_dtype, cudaStream_t s)
{
    if (a.n_tiles <= 0) return cudaSuccess;
    if (map_dtype == PSFS_MAP_F16) return launch_shape<__half>(a, shape, s);
    if (map_dtype == PSFS_MAP_BF16) return launch_shape<__nv_bfloat16>(a, shape, s);
    return launch_shape<float>(a, shape, s);
}

}  // namespace psfs
