// psfs_reproject.cu -- silhouettes of the reconstructed voxels in every camera
// (Section 2.3: the projection of the voxels is the tracker's prior knowledge,
// matched against the particles' projected body models; Section 3.3.3,
// "Voxel Projection").  Pixel (x, y) of camera c is set iff the ray from the
// camera centre through the pixel centre meets, in front of the camera, the
// cube of a listed voxel.
//
// One thread per (camera, listed voxel): the eight cube corners are projected
// with the forward kernels' matrices, the pixels whose centres can fall
// inside that projection (its bounding box, widened against float32
// rounding) are tested with a float32 slab test of their centre rays in
// voxel-index coordinates, and a hit stores 1 (every writer stores the same
// value, so no atomics are needed).  Run on the surface list, the work is
// proportional to the body's surface; the silhouette of a solid equals that
// of its surface voxels.
#include <algorithm>

#include "psfs_internal.cuh"

namespace psfs {

namespace {

constexpr int kRpThreads = 256;

__global__ void __launch_bounds__(kRpThreads) reproject_kernel(const __grid_constant__ ReprojectArgs a)
{
    const int f = blockIdx.y;
    const uint32_t m_cnt = min(__ldg(a.counts + f), a.list_stride);
    const uint32_t *list = a.lists + (size_t)f * a.list_stride;
    const int K = a.n_cams, W = a.W, H = a.H;
    uint8_t *masks = a.masks + (size_t)f * K * W * H;
    const uint32_t nx = (uint32_t)a.nx, nxy = (uint32_t)a.nx * (uint32_t)a.ny;
    const uint64_t n_items = (uint64_t)m_cnt * K;
    for (uint64_t it = (uint64_t)blockIdx.x * kRpThreads + threadIdx.x; it < n_items;
         it += (uint64_t)gridDim.x * kRpThreads) {
        // camera-major: the lanes of a warp take consecutive listed voxels of
        // one camera.  Consecutive voxels of a list are neighbours in space
        // (the fusion compacts tile by tile), so their pixel boxes overlap
        // and a warp's byte stores land in few sectors; the camera's
        // matrices are the same for the whole warp.
        const int c = (int)(it / m_cnt);
        const uint32_t e = (uint32_t)(it - (uint64_t)c * m_cnt);
        const uint32_t v = __ldg(list + e);
        if (v >= a.n_vox) continue;
        const uint32_t kz = v / nxy, r = v - kz * nxy, jy = r / nx, ix = r - jy * nx;
        float m[12];
#pragma unroll
        for (int q = 0; q < 12; ++q) m[q] = a.cam[c].m[q];
        // projected corners (centred index coordinates)
        const float x0 = (float)ix - a.ci, y0 = (float)jy - a.cj, z0 = (float)kz - a.ck;
        float umin = INFINITY, umax = -INFINITY, vmin = INFINITY, vmax = -INFINITY;
        bool behind = false;
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            const float X = x0 + ((q & 1) ? 0.5f : -0.5f), Y = y0 + ((q & 2) ? 0.5f : -0.5f),
                        Z = z0 + ((q & 4) ? 0.5f : -0.5f);
            const float u = fmaf(m[0], X, fmaf(m[1], Y, fmaf(m[2], Z, m[3])));
            const float vv = fmaf(m[4], X, fmaf(m[5], Y, fmaf(m[6], Z, m[7])));
            const float w = fmaf(m[8], X, fmaf(m[9], Y, fmaf(m[10], Z, m[11])));
            behind |= !(w > 0.0f);
            const float iw = 1.0f / w;
            umin = fminf(umin, u * iw);
            umax = fmaxf(umax, u * iw);
            vmin = fminf(vmin, vv * iw);
            vmax = fmaxf(vmax, vv * iw);
        }
        // candidate pixels: centres x + 1/2 within the box, widened by 0.01 px
        // plus a relative float32 margin; the whole image when a corner is not
        // in front of the camera (the per-pixel test decides)
        int xa = 0, xb = W - 1, ya = 0, yb = H - 1;
        if (!behind) {
            const float du = 0.01f + 1e-5f * fmaxf(fabsf(umin), fabsf(umax));
            const float dv = 0.01f + 1e-5f * fmaxf(fabsf(vmin), fabsf(vmax));
            xa = max(xa, (int)fmaxf(ceilf(umin - 0.5f - du), -1.0f));
            xb = min(xb, (int)fminf(floorf(umax - 0.5f + du), (float)W));
            ya = max(ya, (int)fmaxf(ceilf(vmin - 0.5f - dv), -1.0f));
            yb = min(yb, (int)fminf(floorf(vmax - 0.5f + dv), (float)H));
        }
        // this camera's inverse projection and the cube's slab offsets from the
        // camera centre, in registers for the pixel loop
        float mi[9], o1[3];
#pragma unroll
        for (int q = 0; q < 9; ++q) mi[q] = a.inv[c].minv[q];
        o1[0] = (float)ix - 0.5f - a.inv[c].qc[0];
        o1[1] = (float)jy - 0.5f - a.inv[c].qc[1];
        o1[2] = (float)kz - 0.5f - a.inv[c].qc[2];
        const float o2[3] = {o1[0] + 1.0f, o1[1] + 1.0f, o1[2] + 1.0f};
        uint8_t *mask = masks + (size_t)c * W * H;
        for (int y = ya; y <= yb; ++y) {
            const float py = (float)y + 0.5f;
            for (int x = xa; x <= xb; ++x) {
                const float px = (float)x + 0.5f;
                float t_in = 0.0f, t_out = INFINITY;
#pragma unroll
                for (int ax = 0; ax < 3; ++ax) {
                    const float d = fmaf(mi[3 * ax], px, fmaf(mi[3 * ax + 1], py, mi[3 * ax + 2]));
                    // hardware reciprocal (about 1 ulp; 1/0 = inf as with the
                    // division): the slab distances move by far less than
                    // the 2e-3 voxel the silhouettes are checked against
                    const float id = rcp_approx(d);
                    const float t1 = o1[ax] * id, t2 = o2[ax] * id;
                    t_in = fmaxf(t_in, fminf(t1, t2));
                    t_out = fminf(t_out, fmaxf(t1, t2));
                }
                if (t_in <= t_out) mask[(size_t)y * W + x] = 1;
            }
        }
    }
}

}  // namespace

cudaError_t launch_reproject(const ReprojectArgs &a, int n_frames, cudaStream_t s)
{
    if (n_frames <= 0) return cudaSuccess;
    cudaError_t e = cudaMemsetAsync(a.masks, 0, (size_t)n_frames * a.n_cams * a.W * a.H, s);
    if (e != cudaSuccess) return e;
    int sms = 0, dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const uint64_t max_items = (uint64_t)a.list_stride * a.n_cams;
    const uint32_t want = (uint32_t)std::max(1, 8 * std::max(sms, 1) / n_frames);
    const uint32_t per_frame =
        (uint32_t)std::max<uint64_t>(1, std::min<uint64_t>(want, (max_items + kRpThreads - 1) / kRpThreads));
    reproject_kernel<<<dim3(per_frame, (unsigned)n_frames), kRpThreads, 0, s>>>(a);
    return cudaGetLastError();
}

}  // namespace psfs
