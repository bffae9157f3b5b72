// psfs_smooth.cu -- smoothing of the voxel probabilities before the threshold
// (end of Section 2.2.2: the probabilities are filtered, then thresholded;
// step (d) of Section 3.3.3 merges the smoothing with the voxel generation).
// The paper does not give the filter; this is the 3 x 3 x 3 box mean over
// the neighbours inside the grid (a voxel's 27-neighbourhood clipped to the
// grid, divided by the number of voxels in it), then the strict threshold
// smoothed > tau and the compaction of the voxels above it.
//
// One CTA owns a 32 (x) x 8 (y) x 8 (z) block of one frame.  It loads the
// block and a one-voxel halo (34 x 10 x 10, zeros outside the grid) into
// shared memory with row-coalesced loads and forms the 3-sums along x there;
// each thread then takes its (x, y) column, forms the 3-sums along y of the
// ten halo planes and the 3-sums along z in registers: ((x-sums) y-sums)
// z-sums, the same order for every voxel.  The scaling by the reciprocal of
// the clipped count (the FP32 reciprocal of an integer: one rounding more
// than a division), the optional store of
// the smoothed value, the threshold and the warp-aggregated compaction (one
// atomicAdd per CTA) follow in the same pass, so the frame's probabilities are
// read once and the smoothed grid is written at most once.
#include "psfs_internal.cuh"

namespace psfs {

namespace {

constexpr int kSX = 32, kSY = 8, kSZ = 8;                     // outputs per CTA
constexpr int kHX = kSX + 2, kHY = kSY + 2, kHZ = kSZ + 2;    // with the halo

__global__ void __launch_bounds__(kSX * kSY) smooth_kernel(const SmoothArgs a, int tiles_z)
{
    constexpr int kRows = kHZ * kHY;   // halo rows (z, y), row r = z * kHY + y
    __shared__ float v[kRows][kHX];
    __shared__ float sx[kRows][kSX];
    __shared__ uint32_t s_off[kSY];
    __shared__ uint32_t s_base;

    const int tid = threadIdx.x;
    const int lx = tid & 31, ly = tid >> 5;   // lane = x, warp = y (8 warps)
    const int f = blockIdx.z / tiles_z;
    const int x0 = blockIdx.x * kSX, y0 = blockIdx.y * kSY, z0 = (blockIdx.z - f * tiles_z) * kSZ;
    const int nx = a.nx, ny = a.ny, nz = a.nz;
    const size_t n_vox = (size_t)nx * ny * nz;
    const float *prob = a.prob + (size_t)f * n_vox;

    // halo rows of 34 floats: warp w takes rows w, w + 8, ...; lane l loads
    // x = l and lanes 0, 1 also x = 32, 33.  All loads of a thread are issued
    // before the first shared-memory store.
    {
        constexpr int kPerWarp = (kRows + kSY - 1) / kSY;
        const int gxa = x0 - 1 + lx, gxb = x0 + 31 + lx;
        const bool oka = gxa >= 0 && gxa < nx, okb = lx < 2 && gxb < nx;
        float va[kPerWarp], vb[kPerWarp];
#pragma unroll
        for (int q = 0; q < kPerWarp; ++q) {
            const int row = ly + q * kSY;
            const int z = row / kHY, y = row - z * kHY;
            const int gy = y0 - 1 + y, gz = z0 - 1 + z;
            const bool okr = row < kRows && gy >= 0 && gz >= 0 && gy < ny && gz < nz;
            const size_t rbase = okr ? (size_t)nx * ((size_t)gy + (size_t)ny * gz) : 0;
            va[q] = (okr && oka) ? __ldg(prob + rbase + gxa) : 0.0f;
            vb[q] = (okr && okb) ? __ldg(prob + rbase + gxb) : 0.0f;
        }
#pragma unroll
        for (int q = 0; q < kPerWarp; ++q) {
            const int row = ly + q * kSY;
            if (row < kRows) {
                v[row][lx] = va[q];
                if (lx < 2) v[row][32 + lx] = vb[q];
            }
        }
    }
    __syncthreads();
    // 3-sums along x of every halo row
#pragma unroll
    for (int q = 0; q < (kRows + kSY - 1) / kSY; ++q) {
        const int row = ly + q * kSY;
        if (row < kRows) sx[row][lx] = (v[row][lx] + v[row][lx + 1]) + v[row][lx + 2];
    }
    __syncthreads();
    // this thread's column (x0 + lx, y0 + ly): 3-sums along y for the kHZ
    // halo planes, then along z
    float ys[kHZ];
#pragma unroll
    for (int z = 0; z < kHZ; ++z)
        ys[z] = (sx[z * kHY + ly][lx] + sx[z * kHY + ly + 1][lx]) + sx[z * kHY + ly + 2][lx];

    const int gx = x0 + lx, gy = y0 + ly;
    const bool in_xy = gx < nx && gy < ny;
    // 1 / (number of in-grid voxels of the clipped neighbourhood), per z case
    const int cxy = (1 + (gx > 0) + (gx + 1 < nx)) * (1 + (gy > 0) + (gy + 1 < ny));
    const float inv1 = 1.0f / (float)cxy, inv2 = 1.0f / (float)(2 * cxy), inv3 = 1.0f / (float)(3 * cxy);
    float *out = a.smoothed ? a.smoothed + (size_t)f * n_vox : nullptr;
    uint32_t ballots[kSZ];
    uint32_t warp_count = 0;
#pragma unroll
    for (int t = 0; t < kSZ; ++t) {
        const int gz = z0 + t;
        const bool valid = in_xy && gz < nz;
        const float sum = (ys[t] + ys[t + 1]) + ys[t + 2];
        const int cz = 1 + (gz > 0) + (gz + 1 < nz);
        const float sm = sum * (cz == 3 ? inv3 : cz == 2 ? inv2 : inv1);
        const size_t lin = (size_t)gx + (size_t)nx * ((size_t)gy + (size_t)ny * gz);
        if (valid && out) __stcs(out + lin, sm);
        ballots[t] = __ballot_sync(0xFFFFFFFFu, valid && sm > a.threshold);
        warp_count += __popc(ballots[t]);
    }
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
        const uint32_t b = ballots[t];
        if ((b >> lx) & 1u) {
            const uint32_t p = pos + __popc(b & ((1u << lx) - 1u));
            if (p < a.capacity)
                list[p] = (uint32_t)gx + (uint32_t)nx * ((uint32_t)gy + (uint32_t)ny * (uint32_t)(z0 + t));
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
