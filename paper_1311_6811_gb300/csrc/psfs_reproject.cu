// psfs_reproject.cu -- silhouettes of the reconstructed voxels in every camera
// (Section 2.3: the projection of the voxels is the tracker's prior knowledge,
// matched against the particles' projected body models; Section 3.3.3,
// "Voxel Projection").  Pixel (x, y) of camera c is set iff the ray from the
// camera centre through the pixel centre meets, in front of the camera, the
// cube of a listed voxel.
//
// One thread per (camera, listed voxel), with the forward kernels' matrices;
// a CTA takes chunks of 256 consecutive listed voxels of one camera.  When
// all eight cube corners lie in front of the camera, a centre ray meets the
// cube iff the pixel centre lies in the cube's projection: a convex polygon
// whose vertices are the projections of the cube's silhouette loop (the
// corners between faces turned towards the camera and faces turned away).
// Which corners form that loop, and in which cyclic order, depends only on
// where the camera centre lies relative to the cube's three slabs (below,
// within or above each: 26 cases outside the cube), so a table made once on
// the host gives the 4 or 6 corners to project.  A row of pixel centres
// meets the polygon in one interval whose ends are the row's crossings with
// its edges.  The chunk's intervals are set in shared memory when the union
// of their boxes fits the stage, and each non-zero 4-byte word of the stage
// is then OR-ed into the mask once; otherwise each interval is stored
// directly (4-byte stores where whole aligned words are covered).  Cubes not
// wholly in front of the camera, and projections too large for float32 rows,
// take a float32 slab test of the centre ray of every pixel whose centre can
// fall inside the projection's bounding box.  Every writer writes 1, so no
// value is lost between writers.  Run on the surface list, the work is
// proportional to the body's surface; the silhouette of a solid equals that
// of its surface voxels.
#include <algorithm>
#include <climits>
#include <cmath>

#include "psfs_internal.cuh"

namespace psfs {

namespace {

constexpr int kRpThreads = 256;

// Silhouette loops of a unit cube by camera region: entry (rx + 1) + 3 (ry +
// 1) + 9 (rz + 1), r = -1 / 0 / +1 for a camera centre below / within /
// above the slab of that axis; bits 0-3 the corner count n (4 or 6; 0 for
// the cube's interior), then n corners of 3 bits each (corner q = bx + 2 by +
// 4 bz) in cyclic order.
struct SilTable {
    uint32_t e[27];
};

// Projects the unit cube's corners from a point of each region (along each
// axis 3 cube sizes below the lower face, at the centre, or 3 above the
// upper face) along the view towards the cube's centre and keeps the convex
// hull of the projections (Andrew's monotone chain), in order.
SilTable make_sil_table()
{
    SilTable t{};
    const double pos[3] = {-3.0, 0.5, 4.0};
    for (int code = 0; code < 27; ++code) {
        const int r[3] = {code % 3, (code / 3) % 3, code / 9};
        if (r[0] == 1 && r[1] == 1 && r[2] == 1) continue;   // inside the cube
        const double P[3] = {pos[r[0]], pos[r[1]], pos[r[2]]};
        double d[3] = {0.5 - P[0], 0.5 - P[1], 0.5 - P[2]};
        const double dn = std::sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
        for (double &x : d) x /= dn;
        // a basis (e1, e2) of the image plane: e1 = unit(d x a) with a the axis least aligned with d
        int ax = 0;
        for (int k = 1; k < 3; ++k)
            if (std::fabs(d[k]) < std::fabs(d[ax])) ax = k;
        double a[3] = {0.0, 0.0, 0.0};
        a[ax] = 1.0;
        double e1[3] = {d[1] * a[2] - d[2] * a[1], d[2] * a[0] - d[0] * a[2], d[0] * a[1] - d[1] * a[0]};
        const double n1 = std::sqrt(e1[0] * e1[0] + e1[1] * e1[1] + e1[2] * e1[2]);
        for (double &x : e1) x /= n1;
        const double e2[3] = {d[1] * e1[2] - d[2] * e1[1], d[2] * e1[0] - d[0] * e1[2], d[0] * e1[1] - d[1] * e1[0]};
        double px[8], py[8];
        int idx[8];
        for (int q = 0; q < 8; ++q) {
            const double X[3] = {(double)(q & 1) - P[0], (double)((q >> 1) & 1) - P[1], (double)((q >> 2) & 1) - P[2]};
            const double z = X[0] * d[0] + X[1] * d[1] + X[2] * d[2];
            px[q] = (X[0] * e1[0] + X[1] * e1[1] + X[2] * e1[2]) / z;
            py[q] = (X[0] * e2[0] + X[1] * e2[1] + X[2] * e2[2]) / z;
            idx[q] = q;
        }
        std::sort(idx, idx + 8, [&](int i, int j) { return px[i] < px[j] || (px[i] == px[j] && py[i] < py[j]); });
        auto cross = [&](int o, int i, int j) {
            return (px[i] - px[o]) * (py[j] - py[o]) - (py[i] - py[o]) * (px[j] - px[o]);
        };
        int hull[16], k = 0;
        for (int i = 0; i < 8; ++i) {   // lower chain
            while (k >= 2 && cross(hull[k - 2], hull[k - 1], idx[i]) <= 1e-12) --k;
            hull[k++] = idx[i];
        }
        for (int i = 6, lo = k + 1; i >= 0; --i) {   // upper chain
            while (k >= lo && cross(hull[k - 2], hull[k - 1], idx[i]) <= 1e-12) --k;
            hull[k++] = idx[i];
        }
        const int n = k - 1;   // the last point repeats the first
        uint32_t ent = (uint32_t)n;
        for (int i = 0; i < n && i < 6; ++i) ent |= (uint32_t)hull[i] << (4 + 3 * i);
        t.e[code] = n <= 6 ? ent : 0u;
    }
    return t;
}

// Sets the pixels [x0, x1] of one mask row to 1: single bytes up to and after
// the whole aligned 4-byte words in between (`words`: the row starts 4-byte
// aligned), which get one 32-bit store each.
__device__ __forceinline__ void set_run(uint8_t *row, int x0, int x1, bool words)
{
    int x = x0;
    if (words) {
        for (; x <= x1 && (x & 3); ++x) row[x] = 1;
        for (; x + 3 <= x1; x += 4) *reinterpret_cast<uint32_t *>(row + x) = 0x01010101u;
    }
    for (; x <= x1; ++x) row[x] = 1;
}

// The projection of one listed voxel's cube in camera c: the silhouette
// polygon (n >= 3 corners, a 4-corner loop padded with its first corner, so
// that zero-length edges cross no row), the du/dv of its edges and the
// range of pixel rows and columns whose centres it can hold; n = 0 when a
// corner is not in front of the camera or the projection is too large for
// float32 rows (the caller then takes the slab test).
struct CubeProj {
    float pu[6], pv[6], sl[6];
    int n;
    int xa, xb, ya, yb;   // candidate pixels (the slab test's box when n = 0 and the cube is in front)
    bool behind;
    float o1[3];          // the cube's lower faces minus the camera centre (index coordinates)
};

__device__ __forceinline__ void project_cube(const ReprojectArgs &a, const SilTable &sil, int c, uint32_t v,
                                             CubeProj &P)
{
    const uint32_t nx = (uint32_t)a.nx, nxy = (uint32_t)a.nx * (uint32_t)a.ny;
    const uint32_t kz = v / nxy, r = v - kz * nxy, jy = r / nx, ix = r - jy * nx;
    const int W = a.W, H = a.H;
    float m[12];
#pragma unroll
    for (int q = 0; q < 12; ++q) m[q] = a.cam[c].m[q];
    // centred index coordinates of the cube's centre
    const float x0 = (float)ix - a.ci, y0 = (float)jy - a.cj, z0 = (float)kz - a.ck;
    bool behind = false;
#pragma unroll
    for (int q = 0; q < 8; ++q) {
        const float X = x0 + ((q & 1) ? 0.5f : -0.5f), Y = y0 + ((q & 2) ? 0.5f : -0.5f),
                    Z = z0 + ((q & 4) ? 0.5f : -0.5f);
        behind |= !(fmaf(m[8], X, fmaf(m[9], Y, fmaf(m[10], Z, m[11]))) > 0.0f);
    }
    P.behind = behind;
    P.o1[0] = (float)ix - 0.5f - a.inv[c].qc[0];
    P.o1[1] = (float)jy - 0.5f - a.inv[c].qc[1];
    P.o1[2] = (float)kz - 0.5f - a.inv[c].qc[2];
    P.n = 0;
    P.xa = 0;
    P.xb = W - 1;
    P.ya = 0;
    P.yb = H - 1;
    if (behind) return;   // the whole image: the per-pixel test decides
    int code = 0;
#pragma unroll
    for (int ax = 2; ax >= 0; --ax)
        code = 3 * code + (P.o1[ax] > 0.0f ? 0 : (P.o1[ax] + 1.0f < 0.0f ? 2 : 1));
    const uint32_t ent = sil.e[code];
    const int n = (int)(ent & 15u);
    float umin = INFINITY, umax = -INFINITY, vmin = INFINITY, vmax = -INFINITY;
#pragma unroll
    for (int k = 0; k < 6; ++k) {
        const int q = (int)((ent >> (4 + 3 * (k < n ? k : 0))) & 7u);
        const float X = x0 + ((q & 1) ? 0.5f : -0.5f), Y = y0 + ((q & 2) ? 0.5f : -0.5f),
                    Z = z0 + ((q & 4) ? 0.5f : -0.5f);
        const float u = fmaf(m[0], X, fmaf(m[1], Y, fmaf(m[2], Z, m[3])));
        const float vv = fmaf(m[4], X, fmaf(m[5], Y, fmaf(m[6], Z, m[7])));
        // hardware reciprocal (about 1 ulp): the corners move by ~1e-7 of their
        // distance from the principal point, far below the 2e-3 voxel the
        // silhouettes are checked against
        const float iw = rcp_approx(fmaf(m[8], X, fmaf(m[9], Y, fmaf(m[10], Z, m[11]))));
        P.pu[k] = u * iw;
        P.pv[k] = vv * iw;
        umin = fminf(umin, P.pu[k]);
        umax = fmaxf(umax, P.pu[k]);
        vmin = fminf(vmin, P.pv[k]);
        vmax = fmaxf(vmax, P.pv[k]);
    }
    if (n >= 3 && fmaxf(fmaxf(fabsf(umin), fabsf(umax)), fmaxf(fabsf(vmin), fabsf(vmax))) < 1e5f) {
        P.n = n;
#pragma unroll
        for (int k = 0; k < 6; ++k) {
            const int j = (k + 1) % 6;
            const float dv = P.pv[j] - P.pv[k];
            P.sl[k] = dv != 0.0f ? div_fast(P.pu[j] - P.pu[k], dv) : 0.0f;
        }
        P.xa = max((int)ceilf(umin - 0.5f), 0);
        P.xb = min((int)floorf(umax - 0.5f), W - 1);
        P.ya = max((int)ceilf(vmin - 0.5f), 0);
        P.yb = min((int)floorf(vmax - 0.5f), H - 1);
        return;
    }
    // the slab test's candidates: centres within the box, widened by 0.01 px
    // plus a relative float32 margin
    const float du = 0.01f + 1e-5f * fmaxf(fabsf(umin), fabsf(umax));
    const float dv = 0.01f + 1e-5f * fmaxf(fabsf(vmin), fabsf(vmax));
    P.xa = max(0, (int)fmaxf(ceilf(umin - 0.5f - du), -1.0f));
    P.xb = min(W - 1, (int)fminf(floorf(umax - 0.5f + du), (float)W));
    P.ya = max(0, (int)fmaxf(ceilf(vmin - 0.5f - dv), -1.0f));
    P.yb = min(H - 1, (int)fminf(floorf(vmax - 0.5f + dv), (float)H));
}

// Row y of the silhouette polygon: the columns [xs, xe] whose centres it
// holds (xs > xe: none), kept within the polygon's column range [xa, xb] (a
// rounded crossing may fall just outside its corners' extent).
__device__ __forceinline__ void polygon_row(const CubeProj &P, int y, int &xs, int &xe)
{
    const float yc = (float)y + 0.5f;
    float lo = INFINITY, hi = -INFINITY;
#pragma unroll
    for (int k = 0; k < 6; ++k) {
        const int j = (k + 1) % 6;
        if ((P.pv[k] <= yc) != (P.pv[j] <= yc)) {
            const float x = fmaf(yc - P.pv[k], P.sl[k], P.pu[k]);
            lo = fminf(lo, x);
            hi = fmaxf(hi, x);
        }
    }
    xs = 1;
    xe = 0;
    if (lo <= hi) {
        xs = max((int)ceilf(lo - 0.5f), P.xa);
        xe = min((int)floorf(hi - 0.5f), P.xb);
    }
}

// Slab test of the centre rays of the box's pixels (cubes not wholly in
// front of the camera, or projections too large for float32 rows), stored
// straight to the mask.
__device__ void slab_test_pixels(const ReprojectArgs &a, int c, const CubeProj &P, uint8_t *mask)
{
    float mi[9];
#pragma unroll
    for (int q = 0; q < 9; ++q) mi[q] = a.inv[c].minv[q];
    const float o2[3] = {P.o1[0] + 1.0f, P.o1[1] + 1.0f, P.o1[2] + 1.0f};
    for (int y = P.ya; y <= P.yb; ++y) {
        const float py = (float)y + 0.5f;
        for (int x = P.xa; x <= P.xb; ++x) {
            const float px = (float)x + 0.5f;
            float t_in = 0.0f, t_out = INFINITY;
#pragma unroll
            for (int ax = 0; ax < 3; ++ax) {
                const float d = fmaf(mi[3 * ax], px, fmaf(mi[3 * ax + 1], py, mi[3 * ax + 2]));
                // hardware reciprocal (about 1 ulp; 1/0 = inf as with the
                // division): the slab distances move by far less than the
                // 2e-3 voxel the silhouettes are checked against
                const float id = rcp_approx(d);
                const float t1 = P.o1[ax] * id, t2 = o2[ax] * id;
                t_in = fmaxf(t_in, fminf(t1, t2));
                t_out = fminf(t_out, fmaxf(t1, t2));
            }
            if (t_in <= t_out) mask[(size_t)y * a.W + x] = 1;
        }
    }
}

constexpr int kStageBytes = 32768;   // a CTA's staged mask region

// A CTA takes chunks of kRpThreads consecutive listed voxels of one camera
// (neighbours in space: the fusion compacts tile by tile), one voxel per
// thread.  When the union of the chunk's polygon boxes fits kStageBytes
// (rows of whole aligned 4-byte words), the chunk's rows are set in shared
// memory and each non-zero word of the region is OR-ed into the mask once
// (one atomicOr per word instead of a store per row run and voxel: the
// projections of neighbouring surface voxels overlap several times);
// otherwise each thread stores its runs directly.
__global__ void __launch_bounds__(kRpThreads, 4) reproject_kernel(const __grid_constant__ ReprojectArgs a,
                                                                  const __grid_constant__ SilTable sil)
{
    __shared__ __align__(16) uint32_t stage[kStageBytes / 4];
    __shared__ int s_box[4];   // -xa, xb, -ya, yb of the chunk
    const int f = blockIdx.y;
    const uint32_t m_cnt = min(__ldg(a.counts + f), a.list_stride);
    const uint32_t *list = a.lists + (size_t)f * a.list_stride;
    const int K = a.n_cams, W = a.W, H = a.H;
    uint8_t *masks = a.masks + (size_t)f * K * W * H;
    const bool words = (W % 4 == 0) && ((reinterpret_cast<uintptr_t>(a.masks) & 3u) == 0);
    const uint32_t per_cam = (m_cnt + kRpThreads - 1) / kRpThreads;
    const uint64_t n_chunks = (uint64_t)per_cam * K;
    const int tid = threadIdx.x;
    for (uint64_t ch = blockIdx.x; ch < n_chunks; ch += gridDim.x) {
        const int c = (int)(ch / per_cam);
        const uint32_t e = (uint32_t)(ch - (uint64_t)c * per_cam) * kRpThreads + tid;
        uint8_t *mask = masks + (size_t)c * W * H;
        CubeProj P;
        P.n = 0;
        bool have = false;
        if (e < m_cnt) {
            const uint32_t v = __ldg(list + e);
            if (v < a.n_vox) {
                project_cube(a, sil, c, v, P);
                have = true;
            }
        }
        const bool poly = have && P.n >= 3 && P.xa <= P.xb && P.ya <= P.yb;
        // the chunk's box over its polygons (integer atomics in shared memory)
        if (tid == 0) {
            s_box[0] = s_box[1] = s_box[2] = s_box[3] = INT_MIN;
        }
        __syncthreads();
        if (poly) {
            atomicMax(&s_box[0], -P.xa);
            atomicMax(&s_box[1], P.xb);
            atomicMax(&s_box[2], -P.ya);
            atomicMax(&s_box[3], P.yb);
        }
        __syncthreads();
        int X0 = 0, Y0 = 0, rw = 0, rh = 0;
        bool staged = false;
        if (words && s_box[1] != INT_MIN) {
            X0 = (-s_box[0]) & ~3;
            const int X1 = s_box[1] | 3;   // W % 4 == 0: still inside the row
            Y0 = -s_box[2];
            rw = X1 - X0 + 1;
            rh = s_box[3] - Y0 + 1;
            staged = (int64_t)rw * rh <= kStageBytes;
        }
        if (staged) {
            const int n_words = rw * rh / 4;
            for (int w = tid; w < n_words; w += kRpThreads) stage[w] = 0u;
            __syncthreads();
            if (poly) {
                uint8_t *st = reinterpret_cast<uint8_t *>(stage);
                for (int y = P.ya; y <= P.yb; ++y) {
                    int xs, xe;
                    polygon_row(P, y, xs, xe);
                    if (xs > xe ||
                        !PSFS_IN_BOUNDS(y >= Y0 && y - Y0 < rh && xs >= X0 && xe - X0 < rw, a.status))
                        continue;
                    uint8_t *row = st + (y - Y0) * rw - X0;
                    for (int x = xs; x <= xe; ++x) row[x] = 1;
                }
            }
            __syncthreads();
            const int row_words = rw / 4;
            for (int w = tid; w < n_words; w += kRpThreads) {
                const uint32_t val = stage[w];
                if (val) {
                    const int yy = w / row_words, xx = X0 + 4 * (w - yy * row_words);
                    atomicOr(reinterpret_cast<unsigned int *>(mask + (size_t)(Y0 + yy) * W + xx), val);
                }
            }
        } else if (poly) {
            for (int y = P.ya; y <= P.yb; ++y) {
                int xs, xe;
                polygon_row(P, y, xs, xe);
                if (xs <= xe && PSFS_IN_BOUNDS(y >= 0 && y < H && xs >= 0 && xe < W, a.status))
                    set_run(mask + (size_t)y * W, xs, xe, words);
            }
        }
        if (have && P.n < 3) slab_test_pixels(a, c, P, mask);
        __syncthreads();   // the stage and the box are reused by the next chunk
    }
}

}  // namespace

cudaError_t launch_reproject(const ReprojectArgs &a, int n_frames, cudaStream_t s)
{
    if (n_frames <= 0) return cudaSuccess;
    static const SilTable sil = make_sil_table();
    cudaError_t e = cudaMemsetAsync(a.masks, 0, (size_t)n_frames * a.n_cams * a.W * a.H, s);
    if (e != cudaSuccess) return e;
    const int sms = device_sm_count();
    // CTAs per frame: about 4 per SM over all frames, at most one per chunk
    const uint64_t max_chunks = (uint64_t)((a.list_stride + kRpThreads - 1) / kRpThreads) * a.n_cams;
    const uint32_t want = (uint32_t)std::max(1, 4 * std::max(sms, 1) / n_frames);
    const uint32_t per_frame = (uint32_t)std::max<uint64_t>(1, std::min<uint64_t>(want, max_chunks));
    reproject_kernel<<<dim3(per_frame, (unsigned)n_frames), kRpThreads, 0, s>>>(a, sil);
    return cudaGetLastError();
}

}  // namespace psfs
