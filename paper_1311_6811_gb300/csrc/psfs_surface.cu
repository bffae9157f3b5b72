// psfs_surface.cu -- inner-voxel removal (end of Section 2.2.2; step (e) of
// Section 3.3.3, which the paper kept on the CPU): the surface voxels of a
// frame are its occupied voxels with at least one face neighbour that is not
// occupied (outside the grid counts as not occupied).
//
// Input is the compacted occupied-voxel list the fusion kernels write, so the
// work is proportional to the occupied voxels (~1-3 % of the grid), not to
// the grid: one pass sets one bit per listed voxel in a per-frame occupancy
// bitmask (zeroed by a memset, 32 voxels per word, L2-resident: 256 KB for
// 128^3), a second pass tests each listed voxel's six neighbours in the
// bitmask and appends the surface voxels with one atomicAdd per warp.  Both
// passes cover every frame of a call in one launch (grid.y = frame).
#include <algorithm>

#include "psfs_internal.cuh"

namespace psfs {

namespace {

constexpr int kSurfThreads = 256;

__global__ void __launch_bounds__(kSurfThreads) surface_mark_kernel(SurfaceArgs a)
{
    const int f = blockIdx.y;
    const uint32_t *list = a.lists + (size_t)f * a.list_stride;
    uint32_t *mask = a.masks + (size_t)f * a.mask_words;
    const uint32_t n = __ldg(a.counts + f);
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        a.surface_counts[f] = 0u;
        if (n > a.list_stride) atomicOr(a.status, kStatusCapacity);   // the list is incomplete
    }
    const uint32_t m = min(n, a.list_stride);
    for (uint32_t e = blockIdx.x * kSurfThreads + threadIdx.x; e < m; e += gridDim.x * kSurfThreads) {
        const uint32_t v = __ldg(list + e);
        if (v < a.n_vox) atomicOr(mask + (v >> 5), 1u << (v & 31u));
    }
}

__device__ __forceinline__ bool mask_bit(const uint32_t *mask, uint32_t v)
{
    return (__ldg(mask + (v >> 5)) >> (v & 31u)) & 1u;
}

__global__ void __launch_bounds__(kSurfThreads) surface_test_kernel(SurfaceArgs a)
{
    const int f = blockIdx.y;
    const uint32_t *list = a.lists + (size_t)f * a.list_stride;
    const uint32_t *mask = a.masks + (size_t)f * a.mask_words;
    uint32_t *out = a.surface_lists + (size_t)f * a.surface_capacity;
    const uint32_t m = min(__ldg(a.counts + f), a.list_stride);
    const uint32_t nx = (uint32_t)a.nx, ny = (uint32_t)a.ny, nz = (uint32_t)a.nz, nxy = nx * ny;
    const uint32_t lane = threadIdx.x & 31u;
    const uint32_t warp0 = (blockIdx.x * kSurfThreads + threadIdx.x) & ~31u;
    const uint32_t wstride = gridDim.x * kSurfThreads;
    // every lane of a warp runs the same iterations (the ballot needs them all)
    for (uint32_t base = warp0; base < m; base += wstride) {
        const uint32_t e = base + lane;
        bool surf = false;
        uint32_t v = 0;
        if (e < m) {
            v = __ldg(list + e);
            if (v < a.n_vox) {
                const uint32_t k = v / nxy, r = v - k * nxy, j = r / nx, i = r - j * nx;
                surf = i == 0 || i + 1 == nx || j == 0 || j + 1 == ny || k == 0 || k + 1 == nz ||
                       !mask_bit(mask, v - 1) || !mask_bit(mask, v + 1) || !mask_bit(mask, v - nx) ||
                       !mask_bit(mask, v + nx) || !mask_bit(mask, v - nxy) || !mask_bit(mask, v + nxy);
            }
        }
        const uint32_t b = __ballot_sync(0xFFFFFFFFu, surf);
        if (!b) continue;
        uint32_t pos = 0;
        if (lane == 0) {
            pos = atomicAdd(a.surface_counts + f, (uint32_t)__popc(b));
            if ((uint64_t)pos + __popc(b) > (uint64_t)a.surface_capacity) atomicOr(a.status, kStatusCapacity);
        }
        pos = __shfl_sync(0xFFFFFFFFu, pos, 0) + __popc(b & ((1u << lane) - 1u));
        if (surf && pos < a.surface_capacity) out[pos] = v;
    }
}

}  // namespace

cudaError_t launch_surface(const SurfaceArgs &a, int n_frames, cudaStream_t s)
{
    if (n_frames <= 0) return cudaSuccess;
    cudaError_t e = cudaMemsetAsync(a.masks, 0, (size_t)n_frames * a.mask_words * sizeof(uint32_t), s);
    if (e != cudaSuccess) return e;
    // blocks per frame: about four per SM in total (a handful of frames
    // still fills the GPU), at most one per 256 list entries
    int sms = 0, dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const uint32_t want = (uint32_t)std::max(1, 4 * std::max(sms, 1) / n_frames);
    const uint32_t per_frame =
        std::max<uint32_t>(1, std::min<uint32_t>(std::min<uint32_t>(want, 64), (a.list_stride + kSurfThreads - 1) / kSurfThreads));
    const dim3 grid(per_frame, (unsigned)n_frames);
    surface_mark_kernel<<<grid, kSurfThreads, 0, s>>>(a);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    surface_test_kernel<<<grid, kSurfThreads, 0, s>>>(a);
    return cudaGetLastError();
}

}  // namespace psfs
