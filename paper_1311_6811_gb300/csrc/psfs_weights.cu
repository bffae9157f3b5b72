// psfs_weights.cu -- particle weights of the tracker (Section 2.3.2, Eq.
// 14-16; Section 3.3.3, "Compute Sum-squared Difference" steps b-d): how well
// each particle's projected body model matches the voxel silhouettes and
// their edges in every camera.
//
// A particle is n_cyl cylinders (a, b, r).  For a cylinder and a camera
// centre C, the outline seen from C runs along a + t (b - a) +- r n with n
// the unit vector across the axis and the line of sight, n = unit(u x (m - C))
// (u = b - a, m the midpoint).  Silhouette samples sit at t = (k + 1/2) / kt
// and w = (2 l + 1) / kw - 1 across (a + t u + w r n), edge samples at the
// same t on the two outline lines (w = -1, +1).  A sample's value is the
// silhouette (or edge) bit of the pixel its projection falls in, 0 behind the
// camera or outside the image; an edge pixel is a set pixel with a 4-neighbour
// inside the image that is not set.  Per camera S_r = misses / (n_cyl kt kw),
// S_e = misses / (2 n_cyl kt) (Eq. 14-15), weight = exp(-sum_c (S_e + S_r))
// (Eq. 16).
//
// One CTA per particle: its threads take the (camera, cylinder, sample)
// items, count misses per camera with shared-memory integer atomics (exact,
// so the order does not matter), and one thread forms the terms and the
// weight in camera order.
#include "psfs_internal.cuh"

namespace psfs {

namespace {

constexpr int kWThreads = 256;

__device__ __forceinline__ bool mask_at(const uint8_t *m, int W, int x, int y) { return m[(size_t)y * W + x] != 0; }

__global__ void __launch_bounds__(kWThreads) weights_kernel(const __grid_constant__ WeightArgs a)
{
    __shared__ int s_miss_r[PSFS_MAX_CAMS], s_miss_e[PSFS_MAX_CAMS];
    const int p = blockIdx.x;
    const int K = a.n_cams, W = a.W, H = a.H;
    if (threadIdx.x < PSFS_MAX_CAMS) {
        s_miss_r[threadIdx.x] = 0;
        s_miss_e[threadIdx.x] = 0;
    }
    __syncthreads();
    const int per_cyl = a.kt * a.kw + 2 * a.kt;
    const int n_items = K * a.n_cyl * per_cyl;
    const float *cyl0 = a.cyl + (size_t)p * a.n_cyl * 7;
    for (int it = threadIdx.x; it < n_items; it += kWThreads) {
        const int c = it / (a.n_cyl * per_cyl);
        const int r0 = it - c * (a.n_cyl * per_cyl);
        const int q = r0 / per_cyl, smp = r0 - q * per_cyl;
        const float *cy = cyl0 + q * 7;
        const float ax = cy[0], ay = cy[1], az = cy[2];
        const float ux = cy[3] - ax, uy = cy[4] - ay, uz = cy[5] - az, rad = cy[6];
        const float vx = ax + 0.5f * ux - a.C[c][0], vy = ay + 0.5f * uy - a.C[c][1], vz = az + 0.5f * uz - a.C[c][2];
        float nx = uy * vz - uz * vy, ny = uz * vx - ux * vz, nz = ux * vy - uy * vx;
        const float nn = sqrtf(nx * nx + ny * ny + nz * nz);
        const float in = nn > 0.0f ? 1.0f / nn : 0.0f;
        nx *= in;
        ny *= in;
        nz *= in;
        bool edge;
        float t, w;
        if (smp < a.kt * a.kw) {   // silhouette sample (k, l)
            const int k = smp / a.kw, l = smp - k * a.kw;
            t = ((float)k + 0.5f) / (float)a.kt;
            w = (2.0f * (float)l + 1.0f) / (float)a.kw - 1.0f;
            edge = false;
        } else {                   // edge sample (k, side)
            const int e = smp - a.kt * a.kw, k = e >> 1;
            t = ((float)k + 0.5f) / (float)a.kt;
            w = (e & 1) ? 1.0f : -1.0f;
            edge = true;
        }
        const float X = ax + t * ux + w * rad * nx, Y = ay + t * uy + w * rad * ny, Z = az + t * uz + w * rad * nz;
        const float *P = a.P[c];
        const float pu = fmaf(P[0], X, fmaf(P[1], Y, fmaf(P[2], Z, P[3])));
        const float pv = fmaf(P[4], X, fmaf(P[5], Y, fmaf(P[6], Z, P[7])));
        const float pw = fmaf(P[8], X, fmaf(P[9], Y, fmaf(P[10], Z, P[11])));
        bool hit = false;
        if (pw > 0.0f) {
            const float xf = pu / pw, yf = pv / pw;
            if (xf >= 0.0f && xf < (float)W && yf >= 0.0f && yf < (float)H) {
                const int x = min((int)xf, W - 1), y = min((int)yf, H - 1);
                const uint8_t *m = a.masks + (size_t)c * W * H;
                hit = mask_at(m, W, x, y);
                if (edge && hit)
                    hit = (x > 0 && !mask_at(m, W, x - 1, y)) || (x + 1 < W && !mask_at(m, W, x + 1, y)) ||
                          (y > 0 && !mask_at(m, W, x, y - 1)) || (y + 1 < H && !mask_at(m, W, x, y + 1));
            }
        }
        if (!hit) atomicAdd(edge ? &s_miss_e[c] : &s_miss_r[c], 1);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        const float inv_r = 1.0f / (float)(a.n_cyl * a.kt * a.kw), inv_e = 1.0f / (float)(2 * a.n_cyl * a.kt);
        float total = 0.0f;
        for (int c = 0; c < K; ++c) {
            const float se = (float)s_miss_e[c] * inv_e, sr = (float)s_miss_r[c] * inv_r;
            if (a.terms) {
                a.terms[((size_t)p * K + c) * 2 + 0] = se;
                a.terms[((size_t)p * K + c) * 2 + 1] = sr;
            }
            total += se + sr;
        }
        a.weights[p] = expf(-total);
    }
}

}  // namespace

cudaError_t launch_weights(const WeightArgs &a, int n_particles, cudaStream_t s)
{
    if (n_particles <= 0) return cudaSuccess;
    weights_kernel<<<n_particles, kWThreads, 0, s>>>(a);
    return cudaGetLastError();
}

}  // namespace psfs
