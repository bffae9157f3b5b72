// psfs_backward.cu -- adjoint of the reconstruction (no counterpart in the
// paper, which only runs the forward; this is the gradient of a loss on the
// posterior of Eq. 3-4 with respect to the maps of Eq. 2 and the background
// model of Eq. 1).
//
// Loss gradient d_occ per voxel in, gradients per pixel out:
//   dLoss/dL_v   = d_occ_v occ_v (1 - occ_v)                     (voxel pass)
//   dLoss/dg_kp  = sum over voxels v whose centre projects to pixel p of
//                  camera k of dLoss/dL_v                         (pixel pass)
//   dLoss/ds     = dLoss/dg ((2 P_D - 1) / a - (2 q - 1) / b)
//   dLoss/dr     = dLoss/dg dg/dr,  r = log U - log N
//   dLoss/dmu_c  = dLoss/dr (-(I_c - mu_c) / var_c)
//   dLoss/dvar_c = dLoss/dr (1 / (2 var_c) - (I_c - mu_c)^2 / (2 var_c^2))
//
// The forward is recomputed (maps, then the log-odds of every voxel), not
// stored.  The pixel pass owns one pixel per thread and gathers, in a fixed
// order, the voxels that project into it: no atomics, deterministic.  To find
// them it walks the slices of the grid across the pixel's ray along the grid
// axis closest to the ray, and in each slice tests the lattice points inside
// the pixel's (slightly widened) frustum with the exact projection arithmetic
// of the forward kernels, so the ownership is the forward's bit for bit.  The
// walk marks the slices with candidates in a 64-bit mask per block of 64
// slices (one branch-free pass the whole warp runs in step) and then visits
// only the marked slices.
#include "psfs_fuse_common.cuh"

namespace psfs {

namespace {

constexpr int kBwGroup = 8;   // frames per pixel pass of psfs_backward_sequence

template <typename MapT, int LX, int WY, int TZ>
__global__ void __launch_bounds__(32 * WY) backward_voxel_kernel(const __grid_constant__ BackwardArgs b)
{
    const FuseArgs &a = b.f;
    __shared__ int s_flags[PSFS_MAX_CAMS];
    const int lane = threadIdx.x;
    const int wy = threadIdx.y;
    const int tid = wy * 32 + lane;
    if (tid < a.n_cams) s_flags[tid] = __ldg(&a.tilecam[(int64_t)blockIdx.x * a.n_cams + tid].w) >> 16;
    TileCoords<LX, WY, TZ> tc;
    tc.init(a, a.tiles[blockIdx.x], lane, wy);
    const uint32_t W = (uint32_t)a.W, H = (uint32_t)a.H;
    float L[TZ];
#pragma unroll
    for (int t = 0; t < TZ; ++t) L[t] = 0.0f;
    __syncthreads();
    const MapT *maps = reinterpret_cast<const MapT *>(a.maps);
    for (int c = 0; c < a.n_cams; ++c) {
        const int flags = s_flags[c];
        if (flags & kTcSkip) continue;
        float m[12];
#pragma unroll
        for (int q = 0; q < 12; ++q) m[q] = a.cam[c].m[q];
        float bu, bv, bw;
        project_base(m, tc.fi, tc.fj, &bu, &bv, &bw);
        gather_global<MapT, TZ>(m, bu, bv, bw, tc.fk, maps + (int64_t)c * a.map_stride, W, H,
                                (flags & kTcInside) != 0, L);
    }
    if (tc.i >= a.nx || tc.j >= a.ny) return;
#pragma unroll
    for (int t = 0; t < TZ; ++t) {
        const int k = tc.k0 + t;
        if (k >= a.nz) break;
        const uint32_t lin = (uint32_t)tc.i + (uint32_t)a.nx * ((uint32_t)tc.j + (uint32_t)a.ny * (uint32_t)k);
        const float occ = posterior_of_logodds(L[t] + a.logit_prior);
        b.dl[lin] = __ldg(b.d_occ + lin) * occ * (1.0f - occ);
    }
}

__device__ __forceinline__ int ceil_i(float x) { return (int)ceilf(x); }
__device__ __forceinline__ int floor_i(float x) { return (int)floorf(x); }

// The owner walk of pixel p (camera p / (W H)): calls on_voxel(lin) for every
// voxel whose centre the forward projects into that pixel, in a fixed order
// (slices ascending, then the lattice rows and columns of each slice).
template <typename OnVoxel>
__device__ __forceinline__ void owner_walk(const BackwardArgs &b, int64_t p, OnVoxel &&on_voxel)
{
    const FuseArgs &a = b.f;
    const int nn[3] = {a.nx, a.ny, a.nz};
    const float cc[3] = {a.ci, a.cj, a.ck};
    const int cam = (int)(p / a.map_stride);
    const int pix = (int)(p - (int64_t)cam * a.map_stride);
    const int y = pix / a.W, x = pix - y * a.W;
    const PixelInv &iv = b.inv[cam];
    const float *mi = iv.minv;
    // ray direction through the pixel centre, voxel-index coordinates
    const float px = (float)x + 0.5f, py = (float)y + 0.5f;
    float d[3];
#pragma unroll
    for (int r = 0; r < 3; ++r) d[r] = fmaf(mi[3 * r], px, fmaf(mi[3 * r + 1], py, mi[3 * r + 2]));
    // slice along the axis most aligned with the ray
    int ax = 0;
    if (fabsf(d[1]) > fabsf(d[ax])) ax = 1;
    if (fabsf(d[2]) > fabsf(d[ax])) ax = 2;
    const int bx = ax == 0 ? 1 : 0, cx = ax == 2 ? 1 : 2;
    const float inv_da = 1.0f / d[ax];
    // centre ray meets slice plane q_ax = s at (A_b + s B_b, A_c + s B_c)
    const float Bb = d[bx] * inv_da, Bc = d[cx] * inv_da;
    const float qa = iv.qc[ax];
    const float Ab = iv.qc[bx] - qa * Bb, Ac = iv.qc[cx] - qa * Bc;
    // half-extent of the widened frustum per unit of |s - q_a|, from the 4 corners
    float rb = 0.0f, rc = 0.0f;
    const float lo = -0.5f - iv.margin, hi = 0.5f + iv.margin;
#pragma unroll
    for (int corner = 0; corner < 4; ++corner) {
        const float ox = (corner & 1) ? hi : lo, oy = (corner & 2) ? hi : lo;
        float e[3];
#pragma unroll
        for (int r = 0; r < 3; ++r) e[r] = fmaf(mi[3 * r], px + ox, fmaf(mi[3 * r + 1], py + oy, mi[3 * r + 2]));
        const float ia = 1.0f / e[ax];
        rb = fmaxf(rb, fabsf(e[bx] * ia - Bb));
        rc = fmaxf(rc, fabsf(e[cx] * ia - Bc));
    }
    // slices in front of the camera: sign(s - q_a) = sign(d_ax) = sg
    int s_lo = 0, s_hi = nn[ax] - 1;
    const float sg = d[ax] > 0.0f ? 1.0f : -1.0f;
    if (d[ax] > 0.0f) s_lo = max(s_lo, floor_i(qa) + 1);
    else s_hi = min(s_hi, ceil_i(qa) - 1);
    // Slices whose widened window can hold a lattice point of the grid:
    // with |s - q_a| = sg (s - q_a) the window edges are linear in s, and
    // lo_edge(s) <= n - 1, hi_edge(s) >= 0 are linear constraints on s.
    // The range is widened by one slice each way against rounding (it
    // only skips slices; every candidate is still tested exactly).
    {
        const float nbx = (float)(nn[bx] - 1), ncx = (float)(nn[cx] - 1);
        float s_min = (float)s_lo, s_max = (float)s_hi;
        // edge(s) = A + s B +- (sg (s - q_a) r + 1e-3) = k0 + k1 s
        auto clip = [&](float A, float B, float r, float hi_bound) {
            // hi edge >= 0:  (A - sg q_a r + 1e-3) + s (B + sg r) >= 0
            const float k0h = A - sg * qa * r + 1e-3f, k1h = B + sg * r;
            // lo edge <= hi_bound:  (A + sg q_a r - 1e-3) + s (B - sg r) <= hi_bound
            const float k0l = A + sg * qa * r - 1e-3f, k1l = B - sg * r;
            if (fabsf(k1h) > 1e-6f) {
                const float t = -k0h / k1h;
                if (k1h > 0.0f) s_min = fmaxf(s_min, floorf(t) - 1.0f);
                else s_max = fminf(s_max, ceilf(t) + 1.0f);
            } else if (k0h < -1.0f) {
                s_max = -1.0f;   // never reaches the grid
            }
            if (fabsf(k1l) > 1e-6f) {
                const float t = (hi_bound - k0l) / k1l;
                if (k1l > 0.0f) s_max = fminf(s_max, ceilf(t) + 1.0f);
                else s_min = fmaxf(s_min, floorf(t) - 1.0f);
            } else if (k0l > hi_bound + 1.0f) {
                s_max = -1.0f;
            }
        };
        clip(Ab, Bb, rb, nbx);
        clip(Ac, Bc, rc, ncx);
        if (!(s_min <= s_max)) {   // also NaN: the ray misses the grid
            s_lo = 1;
            s_hi = 0;
        } else {
            const float top = (float)nn[ax];
            s_lo = max(s_lo, (int)fminf(fmaxf(s_min, -1.0f), top));
            s_hi = min(s_hi, (int)fminf(fmaxf(s_max, -1.0f), top));
        }
    }
    const float* m = a.cam[cam].m;
    const float nb1 = (float)(nn[bx] - 1), nc1 = (float)(nn[cx] - 1);
    // The window of slice s: centre (b0, c0), half-widths (eb, ec).
    auto window = [&](int s, float &b0, float &c0, float &eb, float &ec) {
        const float fs = (float)s;
        b0 = fmaf(fs, Bb, Ab);
        c0 = fmaf(fs, Bc, Ac);
        const float ds = fabsf(fs - qa);
        eb = fmaf(ds, rb, 1e-3f);
        ec = fmaf(ds, rc, 1e-3f);
    };
    // Slices go in blocks of 64: a branch-free pass marks, in a 64-bit mask,
    // the slices whose windows hold a lattice point of the grid; a second
    // pass visits only the marked slices, in ascending order, and tests
    // their lattice points exactly.  The whole warp runs the first pass
    // in step, and the second only as often as its busiest lane needs.
    for (int s0 = s_lo; s0 <= s_hi; s0 += 64) {
        const int n_s = min(64, s_hi - s0 + 1);
        uint64_t mask = 0;
        for (int q = 0; q < n_s; ++q) {
            float b0, c0, eb, ec;
            window(s0 + q, b0, c0, eb, ec);
            // an integer in [lo, hi] <=> floor(hi) >= lo.  The grid bounds
            // are left to the visit below (it clips the lattice range), so
            // this marks a superset of the slices with in-grid candidates
            // for fewer instructions per slice
            const bool hit = floorf(b0 + eb) >= b0 - eb && floorf(c0 + ec) >= c0 - ec;
            mask |= (uint64_t)hit << q;
        }
        while (mask) {
            const int q = __ffsll((long long)mask) - 1;
            mask &= mask - 1;
            const int s = s0 + q;
            float b0, c0, eb, ec;
            window(s, b0, c0, eb, ec);
            const int b_lo = (int)fmaxf(ceilf(b0 - eb), 0.0f), b_hi = (int)fminf(floorf(b0 + eb), nb1);
            const int c_lo = (int)fmaxf(ceilf(c0 - ec), 0.0f), c_hi = (int)fminf(floorf(c0 + ec), nc1);
            for (int ib = b_lo; ib <= b_hi; ++ib)
                for (int ic = c_lo; ic <= c_hi; ++ic) {
                    int idx[3];
                    idx[ax] = s;
                    idx[bx] = ib;
                    idx[cx] = ic;
                    int pix2;
                    if (project_voxel(m, (float)idx[0] - cc[0], (float)idx[1] - cc[1], (float)idx[2] - cc[2],
                                      (uint32_t)a.W, (uint32_t)a.H, &pix2) &&
                        pix2 == pix) {
                        const uint32_t lin = (uint32_t)idx[0] +
                                             (uint32_t)a.nx * ((uint32_t)idx[1] + (uint32_t)a.ny * (uint32_t)idx[2]);
                        on_voxel(lin);
                    }
                }
        }
    }
}

// Chain rule of pixel p for one frame: dLoss/dg = acc to the SLM and, from
// the frame's colour `img` ([n_pix][3]; NULL: the caller's SLM), to the
// background mean and variance.
__device__ __forceinline__ void chain_rule(const BackwardArgs &b, int64_t p, const uint8_t *img, float acc,
                                           float &dslm, float (&dm)[3], float (&dv)[3])
{
    dslm = 0.0f;
#pragma unroll
    for (int c = 0; c < 3; ++c) dm[c] = dv[c] = 0.0f;
    if (acc != 0.0f) {
        float s_val;
        float r = 0.0f, dd[3] = {0.0f, 0.0f, 0.0f}, hh[3] = {0.0f, 0.0f, 0.0f};
        if (img) {
            const uint8_t *im = img + 3 * p;
            const float *mu = b.mean + 3 * p, *hv = b.hinv + 3 * p;
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                dd[c] = (float)im[c] - mu[c];
                hh[c] = hv[c];
            }
            r = pixel_log_odds((float)im[0], (float)im[1], (float)im[2], mu[0], mu[1], mu[2], hh[0], hh[1], hh[2],
                               b.c0);
            s_val = sigmoid_fast(r);
        } else {
            s_val = __ldg(b.slm + p);
        }
        const float av = fmaf(b.da, s_val, b.one_minus_pd), bv = fmaf(b.db, s_val, b.one_minus_q);
        dslm = acc * (b.da / av - b.db / bv);
        if (img) {
            const float dr = acc * dlog_ratio_dr(r, b.sc);
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                dm[c] = -2.0f * dr * dd[c] * hh[c];
                dv[c] = dr * hh[c] * (1.0f - 2.0f * dd[c] * dd[c] * hh[c]);
            }
        }
    }
}

__global__ void __launch_bounds__(256) backward_pixel_kernel(const __grid_constant__ BackwardArgs b)
{
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < b.n_pix; p += stride) {
        float acc = 0.0f;
        owner_walk(b, p, [&](uint32_t lin) { acc += __ldg(b.dl + lin); });
        float dslm, dm[3], dv[3];
        chain_rule(b, p, b.img, acc, dslm, dm, dv);
        if (b.d_slm) b.d_slm[p] = dslm;
        if (b.d_mean)
            for (int c = 0; c < 3; ++c) b.d_mean[3 * p + c] = dm[c];
        if (b.d_var)
            for (int c = 0; c < 3; ++c) b.d_var[3 * p + c] = dv[c];
    }
}

// The pixel pass of up to kBwGroup frames of one rig at once: one owner walk
// per pixel serves every frame (frame f's dLoss/dL at b.dl + f dl_fstride,
// its colour at b.img + f img_fstride).  Per frame the sums and the chain
// rule are those of backward_pixel_kernel, so d_slm (frame f at
// b.d_slm + f n_pix) is bit-identical to one frame per call; d_mean and d_var
// receive the frames' gradients added in frame order to 0 (or, with
// `accumulate`, to what they hold).
__global__ void __launch_bounds__(256) backward_pixel_group_kernel(const __grid_constant__ BackwardArgs b,
                                                                   int n_frames, int64_t img_fstride,
                                                                   int64_t dl_fstride, int accumulate)
{
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < b.n_pix; p += stride) {
        float acc[kBwGroup];
#pragma unroll
        for (int f = 0; f < kBwGroup; ++f) acc[f] = 0.0f;
        owner_walk(b, p, [&](uint32_t lin) {
#pragma unroll
            for (int f = 0; f < kBwGroup; ++f)
                if (f < n_frames) acc[f] += __ldg(b.dl + f * dl_fstride + lin);
        });
        float tm[3] = {0.0f, 0.0f, 0.0f}, tv[3] = {0.0f, 0.0f, 0.0f};
        if (accumulate) {
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                if (b.d_mean) tm[c] = b.d_mean[3 * p + c];
                if (b.d_var) tv[c] = b.d_var[3 * p + c];
            }
        }
#pragma unroll
        for (int f = 0; f < kBwGroup; ++f) {
            if (f < n_frames) {
                float dslm, dm[3], dv[3];
                chain_rule(b, p, b.img + f * img_fstride, acc[f], dslm, dm, dv);
                if (b.d_slm) b.d_slm[f * b.n_pix + p] = dslm;
                // separate round-to-nearest adds: the compiler may not fuse
                // them with the products above, so the sums are those of the
                // per-frame gradients as psfs_backward stores them
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    tm[c] = __fadd_rn(tm[c], dm[c]);
                    tv[c] = __fadd_rn(tv[c], dv[c]);
                }
            }
        }
        if (b.d_mean)
            for (int c = 0; c < 3; ++c) b.d_mean[3 * p + c] = tm[c];
        if (b.d_var)
            for (int c = 0; c < 3; ++c) b.d_var[3 * p + c] = tv[c];
    }
}

template <typename MapT, int LX, int TZ>
cudaError_t launch_voxel_typed(const BackwardArgs &b, cudaStream_t s)
{
    backward_voxel_kernel<MapT, LX, 4, TZ><<<b.f.n_tiles, dim3(32, 4), 0, s>>>(b);
    return cudaGetLastError();
}

template <typename MapT>
cudaError_t launch_voxel_shape(const BackwardArgs &b, const FuseShape &sh, cudaStream_t s)
{
    if (sh.wy != 4) return cudaErrorInvalidValue;
    if (sh.lx == 8) {
        if (sh.tz == 4) return launch_voxel_typed<MapT, 8, 4>(b, s);
        if (sh.tz == 8) return launch_voxel_typed<MapT, 8, 8>(b, s);
        if (sh.tz == 16) return launch_voxel_typed<MapT, 8, 16>(b, s);
        return cudaErrorInvalidValue;
    }
    if (sh.lx == 16) {
        if (sh.tz == 4) return launch_voxel_typed<MapT, 16, 4>(b, s);
        if (sh.tz == 8) return launch_voxel_typed<MapT, 16, 8>(b, s);
        if (sh.tz == 16) return launch_voxel_typed<MapT, 16, 16>(b, s);
        return cudaErrorInvalidValue;
    }
    if (sh.lx == 32) {
        if (sh.tz == 4) return launch_voxel_typed<MapT, 32, 4>(b, s);
        if (sh.tz == 8) return launch_voxel_typed<MapT, 32, 8>(b, s);
        if (sh.tz == 16) return launch_voxel_typed<MapT, 32, 16>(b, s);
        return cudaErrorInvalidValue;
    }
    return cudaErrorInvalidValue;
}

}  // namespace

cudaError_t launch_backward_voxel(const BackwardArgs &b, const FuseShape &shape, int map_dtype, cudaStream_t s)
{
    if (b.f.n_tiles <= 0) return cudaSuccess;
    if (map_dtype == PSFS_MAP_F16) return launch_voxel_shape<__half>(b, shape, s);
    if (map_dtype == PSFS_MAP_BF16) return launch_voxel_shape<__nv_bfloat16>(b, shape, s);
    return launch_voxel_shape<float>(b, shape, s);
}

cudaError_t launch_backward_pixel(const BackwardArgs &b, cudaStream_t s)
{
    int64_t blocks = (b.n_pix + 255) / 256;
    const int64_t cap = 8 * (int64_t)device_sm_count();
    if (blocks > cap) blocks = cap;
    if (blocks < 1) blocks = 1;
    backward_pixel_kernel<<<(int)blocks, 256, 0, s>>>(b);
    return cudaGetLastError();
}

cudaError_t launch_backward_pixel_group(const BackwardArgs &b, int n_frames, int64_t img_fstride,
                                        int64_t dl_fstride, bool accumulate, cudaStream_t s)
{
    if (n_frames < 1 || n_frames > kBwGroup || !b.img) return cudaErrorInvalidValue;
    int64_t blocks = (b.n_pix + 255) / 256;
    const int64_t cap = 8 * (int64_t)device_sm_count();
    if (blocks > cap) blocks = cap;
    if (blocks < 1) blocks = 1;
    backward_pixel_group_kernel<<<(int)blocks, 256, 0, s>>>(b, n_frames, img_fstride, dl_fstride,
                                                           accumulate ? 1 : 0);
    return cudaGetLastError();
}

}  // namespace psfs
