// psfs_smooth.cu -- smoothing of the voxel probabilities before the threshold
// (end of Section 2.2.2: the probabilities are filtered, then thresholded;
// step (d) of Section 3.3.3 merges the smoothing with the voxel generation).
// The paper does not give the filter; this is the 3 x 3 x 3 box mean over
// the neighbours inside the grid (a voxel's 27-neighbourhood clipped to the
// grid, divided by the number of voxels in it), then the strict threshold
// smoothed > tau and the compaction of the voxels above it.
//
// One CTA owns 32 (x) x 8 (y) columns over 32 planes (z) of one frame.  The
// planes, each with its one-voxel halo (34 x 10, zeros outside the grid),
// stream through shared memory in z order, the next plane's loads in flight
// while the current one is summed: the 3-sums along x in shared memory, the
// 3-sums along y per thread, and the 3-sums along z from the y-sums of the
// last three planes kept in registers: ((x-sums) y-sums) z-sums, the same
// order for every voxel.  The scaling by the reciprocal of
// the clipped count (the FP32 reciprocal of an integer: one rounding more
// than a division), the optional store of
// the smoothed value, the threshold and the warp-aggregated compaction (one
// atomicAdd per CTA) follow in the same pass, so the frame's probabilities are
// read once and the smoothed grid is written at most once.
#include "psfs_internal.cuh"

namespace psfs {

namespace {

constexpr int kSX = 32, kSY = 8, kSZ = 32;   // outputs per CTA: 32 x 8 columns, 32 planes
constexpr int kHX = kSX + 2, kHY = kSY + 2;   // one plane with its halo: 34 x 10
constexpr int kPlane = kHX * kHY;             // 340 floats
constexpr int kThreads = kSX * kSY;
constexpr int kPerThread = (kPlane + kThreads - 1) / kThreads;   // 2

__global__ void __launch_bounds__(kThreads) smooth_kernel(const SmoothArgs a, int tiles_z)
{
    __shared__ float v[kPlane];
    __shared__ float sx[kHY][kSX];
    __shared__ uint32_t s_bal[kSZ][kSY];   // each warp's ballot per output plane
    __shared__ uint32_t s_off[kSY];
    __shared__ uint32_t s_base;

    const int tid = threadIdx.x;
    const int lx = tid & 31, ly = tid >> 5;   // lane = x, warp = y (8 warps)
    const int f = blockIdx.z / tiles_z;
    const int x0 = blockIdx.x * kSX, y0 = blockIdx.y * kSY, z0 = (blockIdx.z - f * tiles_z) * kSZ;
    const int nx = a.nx, ny = a.ny, nz = a.nz;
    const size_t n_vox = (size_t)nx * ny * nz;
    const float *prob = a.prob + (size_t)f * n_vox;
    const int gx = x0 + lx, gy = y0 + ly;
    const bool in_xy = gx < nx && gy < ny;
    // 1 / (number of in-grid voxels of the clipped neighbourhood), per z case
    const int cxy = (1 + (gx > 0) + (gx + 1 < nx)) * (1 + (gy > 0) + (gy + 1 < ny));
    const float inv1 = 1.0f / (float)cxy, inv2 = 1.0f / (float)(2 * cxy), inv3 = 1.0f / (float)(3 * cxy);
    float *out = a.smoothed ? a.smoothed + (size_t)f * n_vox : nullptr;
    const size_t col = (size_t)gx + (size_t)nx * gy;   // this thread's column

    // This thread's halo elements e = tid + k * 256 of every plane (row
    // e / 34, column e % 34): their in-plane offset and in-grid test are the
    // same for all planes.
    const size_t nxy = (size_t)nx * ny;
    size_t off[kPerThread];
    bool ok[kPerThread];
#pragma unroll
    for (int k = 0; k < kPerThread; ++k) {
        const int e = tid + k * kThreads;
        const int y = e / kHX, x = e - y * kHX;
        const int ex = x0 - 1 + x, ey = y0 - 1 + y;
        ok[k] = e < kPlane && ex >= 0 && ey >= 0 && ex < nx && ey < ny;
        off[k] = ok[k] ? (size_t)ex + (size_t)nx * ey : 0;
    }
    auto load_plane = [&](int gz, float (&r)[kPerThread]) {
        const bool okz = gz >= 0 && gz < nz;
        const float *pl = prob + (okz ? (size_t)gz * nxy : 0);
#pragma unroll
        for (int k = 0; k < kPerThread; ++k) r[k] = (okz && ok[k]) ? __ldg(pl + off[k]) : 0.0f;
    };
    // Planes z0 - 1 .. z0 + kSZ stream through shared memory; the next
    // plane's loads are in flight while the current one is summed.  A thread
    // keeps the y-sums of the last three planes: output plane z = p - 1 is
    // (ys[z - 1] + ys[z]) + ys[z + 1].
    float cur[kPerThread], nxt[kPerThread];
    load_plane(z0 - 1, cur);
    float y_a = 0.0f, y_b = 0.0f;   // y-sums of planes p - 2, p - 1
    uint32_t warp_count = 0;
#pragma unroll 1
    for (int q = 0; q < kSZ + 2; ++q) {
        const int p = z0 - 1 + q;
#pragma unroll
        for (int k = 0; k < kPerThread; ++k)
            if (tid + k * kThreads < kPlane) v[tid + k * kThreads] = cur[k];
        if (q + 1 < kSZ + 2) load_plane(p + 1, nxt);
        __syncthreads();
        // 3-sums along x of the plane's ten halo rows
        for (int e = tid; e < kHY * kSX; e += kThreads) {
            const int y = e >> 5, x = e & 31;
            sx[y][x] = (v[y * kHX + x] + v[y * kHX + x + 1]) + v[y * kHX + x + 2];
        }
        __syncthreads();
        const float y_c = (sx[ly][lx] + sx[ly + 1][lx]) + sx[ly + 2][lx];
        if (q >= 2) {
            const int t = q - 2, gz = z0 + t;
            const bool valid = in_xy && gz < nz;
            const float sum = (y_a + y_b) + y_c;
            const int cz = 1 + (gz > 0) + (gz + 1 < nz);
            const float sm = sum * (cz == 3 ? inv3 : cz == 2 ? inv2 : inv1);
            if (valid && out) __stcs(out + col + (size_t)gz * nxy, sm);
            const uint32_t b = __ballot_sync(0xFFFFFFFFu, valid && sm > a.threshold);
            if (lx == 0) s_bal[t][ly] = b;
            warp_count += __popc(b);
        }
        y_a = y_b;
        y_b = y_c;
#pragma unroll
        for (int k = 0; k < kPerThread; ++k) cur[k] = nxt[k];
        // the next plane overwrites v only after every thread has left the x-sums
        // (ordered by the barrier above); sx is rewritten after the next barrier
    }

    // compaction of the CTA's voxels above the threshold: one atomicAdd
    if (lx == 0) s_off[ly] = warp_count;
    __syncthreads();
    if (tid == 0) {
        uint32_t total = 0;
#pragma unroll
        for (int w = 0; w < kSY; ++w) {
            const uint32_t c = s_off[w];
            s_off[w] = total;
            total += c;
        }
        uint32_t base = 0;
        if (total) {
            base = atomicAdd(a.counts + f, total);
            if ((uint64_t)base + total > (uint64_t)a.capacity) atomicOr(a.status, kStatusCapacity);
        }
        s_base = base;
    }
    __syncthreads();
    uint32_t pos = s_base + s_off[ly];
    uint32_t *list = a.lists + (size_t)f * a.capacity;
#pragma unroll
    for (int t = 0; t < kSZ; ++t) {
        const uint32_t b = s_bal[t][ly];
        if ((b >> lx) & 1u) {
            const uint32_t pp = pos + __popc(b & ((1u << lx) - 1u));
            if (pp < a.capacity)
                list[pp] = (uint32_t)gx + (uint32_t)nx * ((uint32_t)gy + (uint32_t)ny * (uint32_t)(z0 + t));
        }
        pos += __popc(b);
    }
}

}  // namespace

cudaError_t launch_smooth(const SmoothArgs &a, int n_frames, cudaStream_t s)
{
    if (n_frames <= 0) return cudaSuccess;
    cudaError_t e = cudaMemsetAsync(a.counts, 0, (size_t)n_frames * sizeof(uint32_t), s);
    if (e != cudaSuccess) return e;
    const int tx = (a.nx + kSX - 1) / kSX, ty = (a.ny + kSY - 1) / kSY, tz = (a.nz + kSZ - 1) / kSZ;
    if ((int64_t)tz * n_frames > 65535) return cudaErrorInvalidValue;
    smooth_kernel<<<dim3(tx, ty, tz * n_frames), kSX * kSY, 0, s>>>(a, tz);
    return cudaGetLastError();
}

}  // namespace psfs
