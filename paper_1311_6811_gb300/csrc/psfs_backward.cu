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
//   dLoss/dr     = dLoss/ds s (1 - s),  s = sigmoid(r), r = log U - log N
//   dLoss/dmu_c  = dLoss/dr (-(I_c - mu_c) / var_c)
//   dLoss/dvar_c = dLoss/dr (1 / (2 var_c) - (I_c - mu_c)^2 / (2 var_c^2))
//
// The forward is recomputed (maps, then the log-odds of every voxel), not
// stored.  This file holds the voxel pass; the pixel pass, which sums each
// pixel's owners in a fixed order from per-handle owner lists, is in
// psfs_owners.cu.
#include "psfs_fuse_common.cuh"

namespace psfs {

namespace {

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
                                (flags & kTcInside) != 0, L, a.status);
    }
    if (tc.i >= a.nx || tc.j >= a.ny) return;
#pragma unroll
    for (int t = 0; t < TZ; ++t) {
        const int k = tc.k0 + t;
        if (k >= a.nz) break;
        const uint32_t lin = (uint32_t)tc.i + (uint32_t)a.nx * ((uint32_t)tc.j + (uint32_t)a.ny * (uint32_t)k);
        const float occ = posterior_of_logodds(L[t] + a.logit_prior);
        b.dl[(size_t)lin * b.dl_stride] = __ldg(b.d_occ + lin) * occ * (1.0f - occ);
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
        if (sh.tz == 2) return launch_voxel_typed<MapT, 8, 2>(b, s);
        if (sh.tz == 4) return launch_voxel_typed<MapT, 8, 4>(b, s);
        if (sh.tz == 8) return launch_voxel_typed<MapT, 8, 8>(b, s);
        if (sh.tz == 16) return launch_voxel_typed<MapT, 8, 16>(b, s);
        return cudaErrorInvalidValue;
    }
    if (sh.lx == 16) {
        if (sh.tz == 2) return launch_voxel_typed<MapT, 16, 2>(b, s);
        if (sh.tz == 4) return launch_voxel_typed<MapT, 16, 4>(b, s);
        if (sh.tz == 8) return launch_voxel_typed<MapT, 16, 8>(b, s);
        if (sh.tz == 16) return launch_voxel_typed<MapT, 16, 16>(b, s);
        return cudaErrorInvalidValue;
    }
    if (sh.lx == 32) {
        if (sh.tz == 2) return launch_voxel_typed<MapT, 32, 2>(b, s);
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

}  // namespace psfs
