// psfs_batch.cu -- many frames in one persistent launch.
//
// Frames may differ in grid size, camera count, image size and background
// (each has its own handle); the likelihood maps of every frame live in
// batch-owned buffers.  The work list interleaves the likelihood chunks of
// frame f with the fusion tiles of frame f - 1, so that HBM-bound and
// gather-bound items run side by side on every SM; a fusion tile first waits
// (bounded) until the per-frame counter says all chunks of its frame are
// done.  Every item depends only on items listed before it and each CTA walks
// its items in list order, so the item with the smallest unfinished index can
// always proceed: the grid never deadlocks as long as all its CTAs are
// resident, which the launch guarantees by sizing the grid from the
// occupancy calculator.
#include <algorithm>

#include "psfs_fuse_common.cuh"

namespace psfs {

namespace {

__device__ __forceinline__ uint32_t ld_acquire(const uint32_t *p)
{
    uint32_t v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];\n" : "=r"(v) : "l"(p) : "memory");
    return v;
}

template <typename T>
__device__ __forceinline__ void store_map(T *out, int64_t p, float v);
template <>
__device__ __forceinline__ void store_map<float>(float *out, int64_t p, float v) { out[p] = v; }
template <>
__device__ __forceinline__ void store_map<__half>(__half *out, int64_t p, float v) { out[p] = __float2half_rn(v); }
template <>
__device__ __forceinline__ void store_map<__nv_bfloat16>(__nv_bfloat16 *out, int64_t p, float v)
{
    out[p] = __float2bfloat16_rn(v);
}

// Pixels of likelihood chunk `idx` of a frame.
__device__ __forceinline__ int64_t chunk_pixels(const BatchFrame &fr, int64_t idx)
{
    return min((int64_t)kBatchChunk, fr.n_pix - idx * kBatchChunk);
}

template <typename MapT, int LX, int TZ, int CB>
__global__ void __launch_bounds__(128) batch_kernel(const BatchLaunch b)
{
    constexpr int WY = 4;
    __shared__ int s_flags[PSFS_MAX_CAMS];
    __shared__ uint32_t s_warp_off[WY];
    __shared__ uint32_t s_base;
    const int lane = threadIdx.x, wy = threadIdx.y, tid = wy * 32 + lane;

    for (int64_t it = blockIdx.x; it < b.n_items; it += gridDim.x) {
        const uint64_t e = b.items[it];
        const uint32_t f = (uint32_t)(e >> 40);
        const uint32_t kind = (uint32_t)((e >> 39) & 1u);
        const int64_t idx = (int64_t)(e & ((1ull << 39) - 1));
        const BatchFrame &fr = b.frames[f];
        if (kind == 0) {
            // Eq. 1-2 and the log ratio, pixels [idx * chunk, ...) of frame f
            const int64_t p0 = idx * kBatchChunk;
            const int64_t np = chunk_pixels(fr, idx);
            MapT *out = reinterpret_cast<MapT *>(const_cast<void *>(fr.fa.maps));
            // plain loads: staging the chunk in shared memory with bulk copies
            // measured 9 % slower for the whole launch (28 KB of shared
            // memory per CTA take the L1 capacity the fusion items' gathers use)
            for (int64_t q = tid; q < np; q += 128) {
                const int64_t p = p0 + q;
                const uint8_t *im = fr.img + 3 * p;
                const float *mu = fr.mean + 3 * p, *hv = fr.hinv + 3 * p;
                const float r = pixel_log_odds((float)im[0], (float)im[1], (float)im[2], mu[0], mu[1], mu[2], hv[0],
                                               hv[1], hv[2], fr.c0);
                store_map<MapT>(out, p, log_ratio_of_r(r, fr.sc));
            }
            if (idx == 0 && tid == 0) *fr.fa.count = 0u;
            __syncthreads();
            if (tid == 0) {
                __threadfence();
                atomicAdd(&b.done[f], 1u);
            }
        } else {
            const FuseArgs &a = fr.fa;
            if (tid == 0) {
                // wait, at most b.wait_ns, for every likelihood chunk of this
                // frame; once any wait of the launch has run out the others
                // give up at once (the launch's results are already invalid),
                // so a stuck frame costs one wait limit, not one per tile
                if (ld_acquire(&b.done[f]) < fr.wait_chunks) {
                    const uint64_t t0 = globaltimer_ns();
                    while (ld_acquire(&b.done[f]) < fr.wait_chunks) {
                        __nanosleep(256);
                        if ((ld_acquire(b.status) & kStatusTimeout) || globaltimer_ns() - t0 > b.wait_ns) {
                            atomicOr(b.status, kStatusTimeout);
                            break;
                        }
                    }
                }
            }
            if (tid < a.n_cams) s_flags[tid] = a.tilecam[idx * a.n_cams + tid].w >> 16;
            __syncthreads();
            TileCoords<LX, WY, TZ> tc;
            tc.init(a, a.tiles[idx], lane, wy);
            const uint32_t W = (uint32_t)a.W, H = (uint32_t)a.H;
            float L[TZ];
#pragma unroll
            for (int t = 0; t < TZ; ++t) L[t] = 0.0f;
            const MapT *maps = reinterpret_cast<const MapT *>(a.maps);
            if (CB == 1) {
                for (int c = 0; c < a.n_cams; ++c) {
                    const int flags = s_flags[c];
                    if (flags & kTcSkip) continue;
                    float m[12];
#pragma unroll
                    for (int q = 0; q < 12; ++q) m[q] = a.cam[c].m[q];
                    float bu, bv, bw;
                    project_base(m, tc.fi, tc.fj, &bu, &bv, &bw);
                    gather_global<MapT, TZ, true>(m, bu, bv, bw, tc.fk, maps + (int64_t)c * a.map_stride, W, H,
                                                  (flags & kTcInside) != 0, L, a.status);
                }
            } else {
                // camera blocks: the loads of CB cameras are issued together,
                // then added camera by camera, so the sum runs over the
                // cameras in the order 0 .. n_cams - 1 as in every other kernel
                for (int c0 = 0; c0 < a.n_cams; c0 += CB) {
                    float g[CB][TZ];
                    bool seen[CB][TZ];
#pragma unroll
                    for (int cb = 0; cb < CB; ++cb) {
                        const int c = c0 + cb;
                        const bool use = c < a.n_cams && !(s_flags[min(c, a.n_cams - 1)] & kTcSkip);
#pragma unroll
                        for (int t = 0; t < TZ; ++t) seen[cb][t] = false;
                        if (use) {
                            float m[12];
#pragma unroll
                            for (int q = 0; q < 12; ++q) m[q] = a.cam[c].m[q];
                            float bu, bv, bw;
                            project_base(m, tc.fi, tc.fj, &bu, &bv, &bw);
                            const MapT *map = maps + (int64_t)c * a.map_stride;
#pragma unroll
                            for (int t = 0; t < TZ; ++t) {
                                int pix;
                                seen[cb][t] = proj_pixel(project_biased(m, bu, bv, bw, tc.fk[t]), W, H, &pix);
                                g[cb][t] = seen[cb][t] ? map_load_coherent(map + pix) : 0.0f;
                            }
                        }
                    }
#pragma unroll
                    for (int cb = 0; cb < CB; ++cb)
#pragma unroll
                        for (int t = 0; t < TZ; ++t)
                            if (seen[cb][t]) L[t] += g[cb][t];
                }
            }
            tile_epilogue<WY, TZ>(a, tc.i, tc.j, tc.k0, L, lane, wy, s_warp_off, &s_base);
        }
        __syncthreads();   // s_flags / s_warp_off are reused by the next item
    }
}

template <typename MapT, int LX, int TZ, int CB>
cudaError_t launch_typed(const BatchLaunch &b, cudaStream_t s)
{
    auto kern = batch_kernel<MapT, LX, TZ, CB>;
    int per_sm = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, 128, 0);
    if (e != cudaSuccess) return e;
    // every CTA must be resident at once (items wait on items of other CTAs)
    int blocks = std::max(1, per_sm) * device_sm_count();
    if (b.blocks > 0) blocks = std::min(blocks, b.blocks);
    if ((int64_t)blocks > b.n_items) blocks = (int)std::max<int64_t>(1, b.n_items);
    kern<<<blocks, dim3(32, 4), 0, s>>>(b);
    return cudaGetLastError();
}

template <typename MapT, int LX>
cudaError_t launch_tz(const BatchLaunch &b, int tz, int cb, cudaStream_t s)
{
    if (cb == 1) {
        if (tz == 2) return launch_typed<MapT, LX, 2, 1>(b, s);
        if (tz == 4) return launch_typed<MapT, LX, 4, 1>(b, s);
        if (tz == 8) return launch_typed<MapT, LX, 8, 1>(b, s);
        if (tz == 16) return launch_typed<MapT, LX, 16, 1>(b, s);
        return cudaErrorInvalidValue;
    }
    if constexpr (LX != 32) {
        if (cb == 2) {
            if (tz == 4) return launch_typed<MapT, LX, 4, 2>(b, s);
            if (tz == 8) return launch_typed<MapT, LX, 8, 2>(b, s);
        }
        if (cb == 4 && tz == 4) return launch_typed<MapT, LX, 4, 4>(b, s);
    }
    return cudaErrorInvalidValue;
}

template <typename MapT>
cudaError_t launch_shape(const BatchLaunch &b, const FuseShape &sh, int cb, cudaStream_t s)
{
    if (sh.wy != 4) return cudaErrorInvalidValue;
    if (sh.lx == 8) return launch_tz<MapT, 8>(b, sh.tz, cb, s);
    if (sh.lx == 16) return launch_tz<MapT, 16>(b, sh.tz, cb, s);
    if (sh.lx == 32) return launch_tz<MapT, 32>(b, sh.tz, cb, s);
    return cudaErrorInvalidValue;
}

}  // namespace

bool batch_shape_supported(const FuseShape &sh, int cb)
{
    if (sh.wy != 4 || sh.staged || !(sh.lx == 8 || sh.lx == 16 || sh.lx == 32)) return false;
    if (cb == 1) return sh.tz == 2 || sh.tz == 4 || sh.tz == 8 || sh.tz == 16;
    if (sh.lx == 32) return false;
    return (cb == 2 && (sh.tz == 4 || sh.tz == 8)) || (cb == 4 && sh.tz == 4);
}

cudaError_t launch_batch(const BatchLaunch &b, const FuseShape &shape, int cameras_per_block, int map_dtype,
                         cudaStream_t s)
{
    if (b.n_items <= 0) return cudaSuccess;
    if (map_dtype == PSFS_MAP_F16) return launch_shape<__half>(b, shape, cameras_per_block, s);
    if (map_dtype == PSFS_MAP_BF16) return launch_shape<__nv_bfloat16>(b, shape, cameras_per_block, s);
    return launch_shape<float>(b, shape, cameras_per_block, s);
}

}  // namespace psfs
