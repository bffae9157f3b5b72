// psfs_smooth.cu -- smoothing of the voxel probabilities before the threshold
// (end of Section 2.2.2: the probabilities are filtered, then thresholded;
// step (d) of Section 3.3.3 merges the smoothing with the voxel generation).
// The paper does not give the filter; this is the 3 x 3 x 3 box mean over
// the neighbours inside the grid (a voxel's 27-neighbourhood clipped to the
// grid, divided by the number of voxels in it), then the strict threshold
// smoothed > tau and the compaction of the voxels above it.
//
// One CTA owns 32 (x) x 16 (y) columns over 32 planes (z) of one frame; a
// thread owns the columns (x, y) and (x, y + 8).  The planes, each with its
// one-voxel halo (34 x 18, zeros outside the grid), stream through two
// shared-memory buffers in z order with one barrier per plane: the 3-sums
// along x of plane p are formed while plane p + 1 is stored and plane p + 2
// is loaded; after the barrier each thread forms its 3-sums along y, and the
// 3-sums along z come from the y-sums of the last three planes kept in
// registers: ((x-sums) y-sums) z-sums, the same order for every voxel.  The
// scaling by the FP32 reciprocal of the clipped count (one rounding more than
// a division), the optional store of the smoothed value, the threshold and
// the warp-aggregated compaction (one atomicAdd per CTA) follow in the same
// pass, so the frame's probabilities are read once and the smoothed grid is
// written at most once.
//
// When the rows are 16-byte multiples (nx % 4 == 0) smooth_tma_kernel does
// the same sums with fewer instructions: a CTA owns 128 (x) x 8 (y) columns
// over 32 planes; warp w the row y0 + w, lane l the columns x0 + 4 l .. x0 +
// 4 l + 3.  Each plane with its halo (columns x0 - 4 .. x0 + 131, rows y0 - 1
// .. y0 + 8; zeros outside the grid) arrives as one 2-D tensor box (TMA)
// through a 4-stage mbarrier ring issued by one thread; each thread forms
// the x-sums of its four columns in the three rows it needs straight from
// shared memory (16-byte reads), their y-sum, and the z-sum from the y-sums
// of the last two planes kept in registers: the same ((x-sums) y-sums)
// z-sums and the same scaling as smooth_kernel, so the same bits.
#include <climits>

#include "psfs_internal.cuh"

namespace psfs {

namespace {

constexpr int kSX = 32, kSY = 16, kSZ = 32;   // outputs per CTA: 32 x 16 columns, 32 planes
constexpr int kHX = kSX + 2, kHY = kSY + 2;    // one plane with its halo: 34 x 18
constexpr int kPlane = kHX * kHY;              // 612 floats
constexpr int kThreads = 256;                  // 8 warps, rows y and y + 8
constexpr int kPerThread = (kPlane + kThreads - 1) / kThreads;   // 3
constexpr int kSums = kHY * kSX;               // 576 x-sums per plane
constexpr int kSumsPerThread = (kSums + kThreads - 1) / kThreads;   // 3

__global__ void __launch_bounds__(kThreads) smooth_kernel(const SmoothArgs a, int tiles_z)
{
    __shared__ float v[2][kPlane];
    __shared__ float sx[2][kSums];                // [kHY][kSX] x-sums per buffer
    __shared__ uint32_t s_bal[kSZ][2][8];   // ballot per output plane, row half and warp
    __shared__ uint32_t s_off[2][8];
    __shared__ uint32_t s_base;

    const int tid = threadIdx.x;
    const int lx = tid & 31, ly = tid >> 5;
    const int f = blockIdx.z / tiles_z;
    const int x0 = blockIdx.x * kSX, y0 = blockIdx.y * kSY, z0 = (blockIdx.z - f * tiles_z) * kSZ;
    const int nx = a.nx, ny = a.ny, nz = a.nz;
    // per-frame indices fit 32 bits (the handle's voxel count does)
    const uint32_t nxy = (uint32_t)nx * (uint32_t)ny, n_vox = nxy * (uint32_t)nz;
    const float *prob = a.prob + (size_t)f * n_vox;
    float *out = a.smoothed ? a.smoothed + (size_t)f * n_vox : nullptr;

    // this thread's halo elements e = tid + k * 256 of every plane (row e / 34,
    // column e % 34): in-plane offset and in-grid test, the same for all planes
    uint32_t off[kPerThread];
    bool ok[kPerThread];
#pragma unroll
    for (int k = 0; k < kPerThread; ++k) {
        const int e = tid + k * kThreads;
        const int y = e / kHX, x = e - y * kHX;
        const int ex = x0 - 1 + x, ey = y0 - 1 + y;
        ok[k] = e < kPlane && ex >= 0 && ey >= 0 && ex < nx && ey < ny;
        off[k] = ok[k] ? (uint32_t)ex + (uint32_t)nx * (uint32_t)ey : 0u;
    }
    // this thread's x-sums e = tid + k * 256 (row e / 32, column e % 32): the
    // sum's index in sx is e, its first term's index in v is e + 2 (e / 32)
    int vsrc[kSumsPerThread];
#pragma unroll
    for (int k = 0; k < kSumsPerThread; ++k) {
        const int e = tid + k * kThreads;
        vsrc[k] = e + 2 * (e >> 5);
    }
    auto load_plane = [&](int gz, float (&r)[kPerThread]) {
        const bool okz = gz >= 0 && gz < nz;
        const uint32_t zoff = okz ? (uint32_t)gz * nxy : 0u;
#pragma unroll
        for (int k = 0; k < kPerThread; ++k) r[k] = (okz && ok[k]) ? __ldg(prob + (zoff + off[k])) : 0.0f;
    };
    auto store_plane = [&](int buf, const float (&r)[kPerThread]) {
#pragma unroll
        for (int k = 0; k < kPerThread; ++k)
            if (k * kThreads + kThreads <= kPlane || tid + k * kThreads < kPlane) v[buf][tid + k * kThreads] = r[k];
    };

    // the two columns: clipped neighbourhood counts and output offsets
    const int gx = x0 + lx;
    int gy[2] = {y0 + ly, y0 + ly + 8};
    bool in_xy[2];
    float inv1[2], inv2[2], inv3[2];
    uint32_t col[2];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        in_xy[h] = gx < nx && gy[h] < ny;
        const int cxy = (1 + (gx > 0) + (gx + 1 < nx)) * (1 + (gy[h] > 0) + (gy[h] + 1 < ny));
        inv1[h] = 1.0f / (float)cxy;
        inv2[h] = 1.0f / (float)(2 * cxy);
        inv3[h] = 1.0f / (float)(3 * cxy);
        col[h] = (uint32_t)gx + (uint32_t)nx * (uint32_t)gy[h];
    }

    // prologue: plane z0 - 1 in buffer 0, plane z0 in registers
    float cur[kPerThread], nxt[kPerThread];
    load_plane(z0 - 1, nxt);
    store_plane(0, nxt);
    load_plane(z0, cur);
    __syncthreads();

    float ya[2] = {0.0f, 0.0f}, yb[2] = {0.0f, 0.0f};   // y-sums of planes p - 2, p - 1
    uint32_t warp_count[2] = {0u, 0u};
    // kSZ + 2 = 34 planes: unrolled by two, so that the buffer of each copy
    // (q & 1) is a compile-time constant
#pragma unroll 2
    for (int q = 0; q < kSZ + 2; ++q) {
        const int buf = q & 1;
        // x-sums of plane p = z0 - 1 + q (in v[buf]) into sx[buf]
#pragma unroll
        for (int k = 0; k < kSumsPerThread; ++k) {
            if (k * kThreads + kThreads <= kSums || tid + k * kThreads < kSums) {
                const float *vp = &v[buf][vsrc[k]];
                sx[buf][tid + k * kThreads] = (vp[0] + vp[1]) + vp[2];
            }
        }
        // plane p + 1 into the other buffer, plane p + 2 in flight
        if (q + 1 < kSZ + 2) store_plane(buf ^ 1, cur);
        if (q + 2 < kSZ + 2) load_plane(z0 + 1 + q, nxt);
        __syncthreads();
        // y-sums of this thread's two columns; z-sums of plane p - 1
        const int t = q - 2, gz = z0 + t;
        const int cz = 1 + (gz > 0) + (gz + 1 < nz);
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const float *sp = &sx[buf][tid + 256 * h];
            const float yc = (sp[0] + sp[kSX]) + sp[2 * kSX];
            if (q >= 2) {
                const bool valid = in_xy[h] && gz < nz;
                const float sum = (ya[h] + yb[h]) + yc;
                const float sm = sum * (cz == 3 ? inv3[h] : cz == 2 ? inv2[h] : inv1[h]);
                if (valid && out) __stcs(out + (col[h] + (uint32_t)gz * nxy), sm);
                const uint32_t b = __ballot_sync(0xFFFFFFFFu, valid && sm > a.threshold);
                if (lx == 0) s_bal[t][h][ly] = b;
                warp_count[h] += __popc(b);
            }
            ya[h] = yb[h];
            yb[h] = yc;
        }
#pragma unroll
        for (int k = 0; k < kPerThread; ++k) cur[k] = nxt[k];
    }

    // compaction of the CTA's voxels above the threshold: one atomicAdd
    if (lx == 0) {
        s_off[0][ly] = warp_count[0];
        s_off[1][ly] = warp_count[1];
    }
    __syncthreads();
    if (tid == 0) {
        uint32_t total = 0;
#pragma unroll
        for (int h = 0; h < 2; ++h)
#pragma unroll
            for (int w = 0; w < 8; ++w) {
                const uint32_t c = s_off[h][w];
                s_off[h][w] = total;
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
    uint32_t *list = a.lists + (size_t)f * a.capacity;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        uint32_t pos = s_base + s_off[h][ly];
#pragma unroll 4
        for (int t = 0; t < kSZ; ++t) {
            const uint32_t b = s_bal[t][h][ly];
            if ((b >> lx) & 1u) {
                const uint32_t pp = pos + __popc(b & ((1u << lx) - 1u));
                if (pp < a.capacity)
                    list[pp] = (uint32_t)gx + (uint32_t)nx * ((uint32_t)gy[h] + (uint32_t)ny * (uint32_t)(z0 + t));
            }
            pos += __popc(b);
        }
    }
}

// ---------------------------------------------------------------------------
// Tensor-box variant (rows of 16-byte multiples)
// ---------------------------------------------------------------------------
constexpr int kTX = 128, kTY = 8, kTZ = 32;         // outputs per CTA
constexpr int kBoxX = kTX + 8, kBoxY = kTY + 2;     // plane box: columns x0 - 4 .. x0 + 131, rows y0 - 1 .. y0 + 8
constexpr int kBoxFloats = kBoxX * kBoxY;           // 1360
constexpr int kBoxStride = 1376;                    // floats per stage: 5504 bytes, a multiple of 128
constexpr int kTStages = 4;
constexpr int kTThreads = 32 * kTY;                 // one warp per output row

// One box of a 4-D tensor map (x, y, z, frame), global -> shared, completion
// counted on `bar`; x a multiple of 4 floats, elements outside the tensor
// read as zero.
__device__ __forceinline__ void tma_load_4d(void *dst, const CUtensorMap *tmap, int x, int y, int z, int w,
                                            uint64_t *bar)
{
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, "
        "%5}], [%6];\n" ::"r"(smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(tmap)), "r"(x), "r"(y), "r"(z), "r"(w), "r"(smem_u32(bar))
        : "memory");
}

__global__ void __launch_bounds__(kTThreads) smooth_tma_kernel(const __grid_constant__ SmoothArgs a, int tiles_x,
                                                               int tiles_y)
{
    __shared__ __align__(128) float box[kTStages][kBoxStride];   // stages start 128-byte aligned
    __shared__ __align__(8) uint64_t bars[kTStages];
    __shared__ uint32_t s_bal[kTZ][kTY][4];   // ballot per output plane, warp and quad position
    __shared__ uint32_t s_off[kTY];
    __shared__ uint32_t s_base;

    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    const int f = blockIdx.y;
    const int t = blockIdx.x;
    const int tx = t % tiles_x, ty = (t / tiles_x) % tiles_y, tz = t / (tiles_x * tiles_y);
    const int x0 = tx * kTX, y0 = ty * kTY, z0 = tz * kTZ;
    const int nx = a.nx, ny = a.ny, nz = a.nz;
    const uint32_t nxy = (uint32_t)nx * (uint32_t)ny, n_vox = nxy * (uint32_t)nz;
    float *out = a.smoothed ? a.smoothed + (size_t)f * n_vox : nullptr;
    const bool vec_out = (reinterpret_cast<uintptr_t>(a.smoothed) & 15u) == 0;
    const int x = x0 + 4 * lane, y = y0 + w;
    const bool in_xy = y < ny && x < nx;

    // clipped counts along x (per column) and y (the warp's row)
    // and the reciprocals of the whole counts for 1, 2 and 3 planes along z
    float inv[3][4];
    const int cy = 1 + (y > 0) + (y + 1 < ny);
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const int cxy = (1 + (x + k > 0) + (x + k + 1 < nx)) * cy;
#pragma unroll
        for (int c = 0; c < 3; ++c) inv[c][k] = 1.0f / (float)((c + 1) * cxy);
    }

    constexpr int kPlanes = kTZ + 2;   // z0 - 1 .. z0 + kTZ
    if (tid == 0) {
        for (int s = 0; s < kTStages; ++s) mbar_init(&bars[s], 1);
        mbar_fence_init();
    }
    __syncthreads();
    auto issue = [&](int q) {   // plane z0 - 1 + q into stage q % kTStages
        const int s = q % kTStages;
        mbar_arrive_expect_tx(&bars[s], (uint32_t)(kBoxFloats * 4));
        tma_load_4d(box[s], &a.tmap, x0 - 4, y0 - 1, z0 - 1 + q, f, &bars[s]);
    };
    if (tid == 0)
        for (int q = 0; q < kTStages && q < kPlanes; ++q) issue(q);

    float ya[4] = {0.0f, 0.0f, 0.0f, 0.0f}, yb[4] = {0.0f, 0.0f, 0.0f, 0.0f};   // y-sums of planes p - 2, p - 1
    uint32_t warp_count = 0;
    for (int q = 0; q < kPlanes; ++q) {
        const int s = q % kTStages;
        mbar_wait_bounded(&bars[s], (uint32_t)((q / kTStages) & 1), a.status);
        // y-sum of this thread's four columns in plane p = z0 - 1 + q: the
        // x-sums of rows y - 1, y, y + 1 (box rows w, w + 1, w + 2; box column
        // c holds x0 - 4 + c)
        float yc[4] = {0.0f, 0.0f, 0.0f, 0.0f};
        float xs[3][4];
#pragma unroll
        for (int r = 0; r < 3; ++r) {
            const float *row = box[s] + (w + r) * kBoxX + 4 * lane;
            const float4 v = *reinterpret_cast<const float4 *>(row + 4);
            const float left = row[3], right = row[8];
            xs[r][0] = (left + v.x) + v.y;
            xs[r][1] = (v.x + v.y) + v.z;
            xs[r][2] = (v.y + v.z) + v.w;
            xs[r][3] = (v.z + v.w) + right;
        }
#pragma unroll
        for (int k = 0; k < 4; ++k) yc[k] = (xs[0][k] + xs[1][k]) + xs[2][k];
        __syncthreads();   // every thread is done with stage s
        if (tid == 0 && q + kTStages < kPlanes) issue(q + kTStages);
        // z-sums of plane p - 1
        if (q >= 2) {
            const int tq = q - 2, gz = z0 + tq;
            const int cz = 1 + (gz > 0) + (gz + 1 < nz);
            const bool valid_z = gz < nz;
            float sm[4];
            uint32_t b[4];
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const float sum = (ya[k] + yb[k]) + yc[k];
                sm[k] = sum * (cz == 3 ? inv[2][k] : (cz == 2 ? inv[1][k] : inv[0][k]));
                b[k] = __ballot_sync(0xFFFFFFFFu, valid_z && in_xy && x + k < nx && sm[k] > a.threshold);
                warp_count += __popc(b[k]);
            }
            if (lane < 4) s_bal[tq][w][lane] = lane == 0 ? b[0] : lane == 1 ? b[1] : lane == 2 ? b[2] : b[3];
            if (out && valid_z && in_xy) {
                float *o = out + ((uint32_t)gz * nxy + (uint32_t)y * (uint32_t)nx + (uint32_t)x);
                if (vec_out && x + 3 < nx) {
                    __stcs(reinterpret_cast<float4 *>(o), make_float4(sm[0], sm[1], sm[2], sm[3]));
                } else {
#pragma unroll
                    for (int k = 0; k < 4; ++k)
                        if (x + k < nx) __stcs(o + k, sm[k]);
                }
            }
        }
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            ya[k] = yb[k];
            yb[k] = yc[k];
        }
    }

    // compaction of the CTA's voxels above the threshold: one atomicAdd
    if (lane == 0) s_off[w] = warp_count;
    __syncthreads();
    if (tid == 0) {
        uint32_t total = 0;
#pragma unroll
        for (int k = 0; k < kTY; ++k) {
            const uint32_t c = s_off[k];
            s_off[k] = total;
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
    uint32_t *list = a.lists + (size_t)f * a.capacity;
    uint32_t pos = s_base + s_off[w];
    const uint32_t lt_mask = (1u << lane) - 1u;
    for (int tq = 0; tq < kTZ; ++tq) {
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const uint32_t b = s_bal[tq][w][k];
            if ((b >> lane) & 1u) {
                const uint32_t pp = pos + __popc(b & lt_mask);
                if (pp < a.capacity)
                    list[pp] = (uint32_t)(x + k) + (uint32_t)nx * ((uint32_t)y + (uint32_t)ny * (uint32_t)(z0 + tq));
            }
            pos += __popc(b);
        }
    }
}

}  // namespace

cudaError_t launch_smooth(const SmoothArgs &a_in, int n_frames, cudaStream_t s)
{
    if (n_frames <= 0) return cudaSuccess;
    cudaError_t e = cudaMemsetAsync(a_in.counts, 0, (size_t)n_frames * sizeof(uint32_t), s);
    if (e != cudaSuccess) return e;
    // rows of 16-byte multiples: the tensor-box kernel
    SmoothArgs a = a_in;
    const int64_t ttx = (a.nx + kTX - 1) / kTX, tty = (a.ny + kTY - 1) / kTY, ttz = (a.nz + kTZ - 1) / kTZ;
    if (n_frames <= 65535 && ttx * tty * ttz <= INT_MAX &&
        encode_grid_tensor(a.prob, a.nx, a.ny, a.nz, n_frames, kBoxX, kBoxY, &a.tmap)) {
        smooth_tma_kernel<<<dim3((unsigned)(ttx * tty * ttz), (unsigned)n_frames), kTThreads, 0, s>>>(a, (int)ttx,
                                                                                                        (int)tty);
        return cudaGetLastError();
    }
    const int tx = (a.nx + kSX - 1) / kSX, ty = (a.ny + kSY - 1) / kSY, tz = (a.nz + kSZ - 1) / kSZ;
    if ((int64_t)tz * n_frames > 65535) return cudaErrorInvalidValue;
    smooth_kernel<<<dim3(tx, ty, tz * n_frames), kThreads, 0, s>>>(a, tz);
    return cudaGetLastError();
}

}  // namespace psfs
