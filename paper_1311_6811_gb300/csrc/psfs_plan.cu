// psfs_plan.cu -- host-side planning of the fuse kernel for one grid and
// camera rig, done once at handle creation in double precision:
//   * the 3x4 projection matrix of every camera in centred voxel-index space;
//   * the voxel tiles in Morton order;
//   * per (tile, camera) the record (image box, staged / skip / inside
//     flags) that the fusion kernels read.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <utility>
#include <vector>

#include "psfs_internal.cuh"

namespace psfs {

namespace {

uint64_t spread3(uint64_t x)
{
    // spread the low 21 bits of x to every third bit
    x &= 0x1FFFFFull;
    x = (x | (x << 32)) & 0x1F00000000FFFFull;
    x = (x | (x << 16)) & 0x1F0000FF0000FFull;
    x = (x | (x << 8)) & 0x100F00F00F00F00Full;
    x = (x | (x << 4)) & 0x10C30C30C30C30C3ull;
    x = (x | (x << 2)) & 0x1249249249249249ull;
    return x;
}

// Records of every (tile, camera) pair; see FuseArgs in psfs_internal.cuh.
// Everything here is double precision on the host.  A tile is marked
// "inside" (no per-voxel test in the kernel) or "skip" (camera ignored) only
// where a bound on the float32 projection error of the kernel stays below a
// quarter pixel, well inside the one-pixel margin each decision keeps.
void build_tilecam(const psfs_grid &g, const psfs_camera *cams, int n_cams, const FuseArgs &f,
                   const FuseShape &shape, int map_dtype, const std::vector<uint64_t> &tiles,
                   std::vector<int4> &out)
{
    const int W = cams[0].width, H = cams[0].height;
    const int elem = map_dtype == PSFS_MAP_F32 ? 4 : 2;
    const int chunk = 16 / elem;
    const bool can_stage = shape.staged && ((int64_t)W * elem) % 16 == 0;
    const double vs = g.voxel_size;
    const double eps32 = std::ldexp(1.0, -24);
    // per camera: magnitude bounds of the float32 projection sums
    std::vector<double> Su(n_cams), Sv(n_cams), Sw(n_cams);
    const double half[3] = {0.5 * g.nx + 1, 0.5 * g.ny + 1, 0.5 * g.nz + 1};
    for (int c = 0; c < n_cams; ++c) {
        const float *m = f.cam[c].m;
        double su = std::fabs(m[3]), sv = std::fabs(m[7]), sw = std::fabs(m[11]);
        for (int a = 0; a < 3; ++a) {
            su += std::fabs(m[a]) * half[a];
            sv += std::fabs(m[4 + a]) * half[a];
            sw += std::fabs(m[8 + a]) * half[a];
        }
        Su[c] = su;
        Sv[c] = sv;
        Sw[c] = sw;
    }
    out.assign(tiles.size() * (size_t)n_cams, make_int4(0, 0, 0, 0));
    for (size_t n = 0; n < tiles.size(); ++n) {
        const uint64_t tc = tiles[n];
        const int tx = (int)(tc & 0x1FFFFF), ty = (int)((tc >> 21) & 0x1FFFFF), tz = (int)(tc >> 42);
        const int TX = shape.tile_x(), TY = shape.tile_y(), TZ = shape.tile_z();
        const int i0 = tx * TX, i1 = std::min(g.nx, i0 + TX) - 1;
        const int j0 = ty * TY, j1 = std::min(g.ny, j0 + TY) - 1;
        const int k0 = tz * TZ, k1 = std::min(g.nz, k0 + TZ) - 1;
        for (int c = 0; c < n_cams; ++c) {
            const double *K = cams[c].K, *R = cams[c].R, *t = cams[c].t;
            double wmin = 1e300, wmax = -1e300, xmin = 1e300, xmax = -1e300, ymin = 1e300, ymax = -1e300;
            for (int corner = 0; corner < 8; ++corner) {
                const int ii = (corner & 1) ? i1 : i0, jj = (corner & 2) ? j1 : j0, kk = (corner & 4) ? k1 : k0;
                const double X[3] = {g.origin[0] + (ii + 0.5) * vs, g.origin[1] + (jj + 0.5) * vs,
                                     g.origin[2] + (kk + 0.5) * vs};
                double xc[3], uvw[3];
                for (int r = 0; r < 3; ++r) xc[r] = R[3 * r] * X[0] + R[3 * r + 1] * X[1] + R[3 * r + 2] * X[2] + t[r];
                for (int r = 0; r < 3; ++r) uvw[r] = K[3 * r] * xc[0] + K[3 * r + 1] * xc[1] + K[3 * r + 2] * xc[2];
                wmin = std::min(wmin, uvw[2]);
                wmax = std::max(wmax, uvw[2]);
                if (uvw[2] > 0) {
                    const double x = uvw[0] / uvw[2], y = uvw[1] / uvw[2];
                    xmin = std::min(xmin, x);
                    xmax = std::max(xmax, x);
                    ymin = std::min(ymin, y);
                    ymax = std::max(ymax, y);
                }
            }
            int4 &rec = out[n * (size_t)n_cams + c];
            const double dw = 8 * eps32 * Sw[c];   // bound on the float32 error of w
            if (wmax < -2 * dw) {   // every centre behind the camera, also in float32
                rec.w = kTcSkip << 16;
                continue;
            }
            if (wmin <= 1e-3 * Sw[c]) continue;   // near or across the camera plane: checked global path
            const double xa = std::max(std::fabs(xmin), std::fabs(xmax)), ya = std::max(std::fabs(ymin), std::fabs(ymax));
            const double ex = 2 * ((8 * eps32 * Su[c] + xa * dw) / wmin + xa * std::ldexp(1.0, -21));
            const double ey = 2 * ((8 * eps32 * Sv[c] + ya * dw) / wmin + ya * std::ldexp(1.0, -21));
            if (!(ex < 0.25 && ey < 0.25) || xa > 1e6 || ya > 1e6) continue;
            const int64_t xlo = (int64_t)std::floor(xmin) - 1, xhi = (int64_t)std::floor(xmax) + 2;
            const int64_t ylo = (int64_t)std::floor(ymin) - 1, yhi = (int64_t)std::floor(ymax) + 2;
            const bool inside = xlo >= 0 && xhi <= W && ylo >= 0 && yhi <= H;
            const int64_t cx0 = std::max<int64_t>(0, xlo), cx1 = std::min<int64_t>(W, xhi);
            const int64_t cy0 = std::max<int64_t>(0, ylo), cy1 = std::min<int64_t>(H, yhi);
            if (cx0 >= cx1 || cy0 >= cy1) {
                rec.w = kTcSkip << 16;
                continue;
            }
            const int64_t ax0 = cx0 / chunk * chunk;
            const int64_t sw = cx1 - ax0, sh = cy1 - cy0;   // clipped extents from the box origin
            int cls = 0;
            while (cls < kBoxClasses && (32 << cls) < sw) ++cls;
            const int64_t nby = (sh + kBoxRows - 1) / kBoxRows;
            const bool staged = can_stage && cls < kBoxClasses &&
                                (int64_t)(32 << cls) * nby * kBoxRows * elem <= (int64_t)kStageBytes;
            rec.x = (int)ax0;
            rec.y = (int)cy0;
            rec.z = (int)sw | (staged ? (cls << 16) | ((int)nby << 18) : 0);
            rec.w = (int)sh | (((inside ? kTcInside : 0) | (staged ? kTcStaged : 0)) << 16);
        }
    }
}

}  // namespace

namespace {

using EncodeTiledFn = CUresult (*)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                   const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                   CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encoder()
{
    static EncodeTiledFn fn = nullptr;
    static bool tried = false;
    if (!tried) {
        tried = true;
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiledFn>(p);
    }
    return fn;
}

}  // namespace

bool encode_map_tensors(void *maps, int map_dtype, int W, int H, int n_cams, CUtensorMap *out)
{
    const int elem = map_dtype == PSFS_MAP_F32 ? 4 : 2;
    if (((int64_t)W * elem) % 16 != 0 || ((uintptr_t)maps & 15u)) return false;
    EncodeTiledFn fn = encoder();
    if (!fn) return false;
    const CUtensorMapDataType dt = map_dtype == PSFS_MAP_F32   ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32
                                   : map_dtype == PSFS_MAP_F16 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT16
                                                               : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16;
    const cuuint64_t dims[3] = {(cuuint64_t)W, (cuuint64_t)H, (cuuint64_t)n_cams};
    const cuuint64_t strides[2] = {(cuuint64_t)W * elem, (cuuint64_t)W * H * elem};
    const cuuint32_t estr[3] = {1, 1, 1};
    for (int cls = 0; cls < kBoxClasses; ++cls) {
        const cuuint32_t box[3] = {(cuuint32_t)(32 << cls), (cuuint32_t)kBoxRows, 1};
        if (fn(&out[cls], dt, 3, maps, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
               CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
            return false;
    }
    return true;
}

bool encode_grid_tensor(const float *grids, int nx, int ny, int nz, int n_frames, int box_x, int box_y,
                        CUtensorMap *out)
{
    if (((int64_t)nx * 4) % 16 != 0 || ((uintptr_t)grids & 15u) || box_x > 256 || box_y > 256 || (box_x * 4) % 16)
        return false;
    EncodeTiledFn fn = encoder();
    if (!fn) return false;
    const cuuint64_t dims[4] = {(cuuint64_t)nx, (cuuint64_t)ny, (cuuint64_t)nz, (cuuint64_t)n_frames};
    const cuuint64_t strides[3] = {(cuuint64_t)nx * 4, (cuuint64_t)nx * ny * 4, (cuuint64_t)nx * ny * nz * 4};
    const cuuint32_t box[4] = {(cuuint32_t)box_x, (cuuint32_t)box_y, 1, 1};
    const cuuint32_t estr[4] = {1, 1, 1, 1};
    return fn(out, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, const_cast<float *>(grids), dims, strides, box, estr,
              CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

bool fuse_shape_supported(const FuseShape &s)
{
    return (s.lx == 8 || s.lx == 16 || s.lx == 32) && s.wy == 4 &&
           ((s.staged == 0 && (s.tz == 2 || s.tz == 4 || s.tz == 8 || s.tz == 16)) ||
            (s.staged == 1 && (s.tz == 8 || s.tz == 16)));
}

void plan_fuse(const psfs_grid &grid, const psfs_camera *cams, int n_cams, const psfs_params &params,
               const FuseShape &shape, FuseArgs *out, std::vector<uint64_t> *tiles_out,
               std::vector<int4> *tilecam_out)
{
    FuseArgs &f = *out;
    std::memset(&f, 0, sizeof(f));
    const int W = cams[0].width, H = cams[0].height;
    f.W = W;
    f.H = H;
    f.map_stride = (int64_t)W * H;
    f.n_cams = n_cams;
    f.nx = grid.nx;
    f.ny = grid.ny;
    f.nz = grid.nz;
    f.ci = 0.5f * (float)(grid.nx - 1);
    f.cj = 0.5f * (float)(grid.ny - 1);
    f.ck = 0.5f * (float)(grid.nz - 1);
    // voxel (i, j, k) sits at centre + voxel_size * (i - ci, j - cj, k - ck)
    const double vs = grid.voxel_size;
    const double centre[3] = {grid.origin[0] + 0.5 * grid.nx * vs, grid.origin[1] + 0.5 * grid.ny * vs,
                              grid.origin[2] + 0.5 * grid.nz * vs};
    for (int c = 0; c < n_cams; ++c) {
        const double *K = cams[c].K, *R = cams[c].R, *t = cams[c].t;
        double KR[9], xc[3];
        for (int r = 0; r < 3; ++r) {
            for (int col = 0; col < 3; ++col)
                KR[3 * r + col] = K[3 * r + 0] * R[0 + col] + K[3 * r + 1] * R[3 + col] + K[3 * r + 2] * R[6 + col];
            xc[r] = R[3 * r + 0] * centre[0] + R[3 * r + 1] * centre[1] + R[3 * r + 2] * centre[2] + t[r];
        }
        for (int r = 0; r < 3; ++r) {
            for (int col = 0; col < 3; ++col) f.cam[c].m[4 * r + col] = (float)(KR[3 * r + col] * vs);
            f.cam[c].m[4 * r + 3] = (float)(K[3 * r + 0] * xc[0] + K[3 * r + 1] * xc[1] + K[3 * r + 2] * xc[2]);
        }
    }
    f.logit_prior = (float)std::log(params.prior / (1.0 - params.prior));
    f.logit_tau = (float)std::log(params.threshold / (1.0 - params.threshold));

    const int ntx = (grid.nx + shape.tile_x() - 1) / shape.tile_x();
    const int nty = (grid.ny + shape.tile_y() - 1) / shape.tile_y();
    const int ntz = (grid.nz + shape.tile_z() - 1) / shape.tile_z();
    std::vector<std::pair<uint64_t, uint64_t>> order;
    order.reserve((size_t)ntx * nty * ntz);
    for (int z = 0; z < ntz; ++z)
        for (int y = 0; y < nty; ++y)
            for (int x = 0; x < ntx; ++x)
                order.emplace_back(spread3(x) | (spread3(y) << 1) | (spread3(z) << 2), pack_tile(x, y, z));
    std::sort(order.begin(), order.end());
    tiles_out->resize(order.size());
    for (size_t n = 0; n < order.size(); ++n) (*tiles_out)[n] = order[n].second;
    f.n_tiles = (int)tiles_out->size();
    build_tilecam(grid, cams, n_cams, f, shape, params.map_dtype, *tiles_out, *tilecam_out);
}

void plan_pixel_rays(const psfs_grid &grid, const psfs_camera *cams, int n_cams, const FuseArgs &f,
                     PixelInv *inv)
{
    const double vs = grid.voxel_size;
    const double eps32 = std::ldexp(1.0, -24);
    const double half[3] = {0.5 * grid.nx + 1, 0.5 * grid.ny + 1, 0.5 * grid.nz + 1};
    for (int c = 0; c < n_cams; ++c) {
        const double *K = cams[c].K, *R = cams[c].R, *t = cams[c].t;
        // K^-1 by cofactors
        const double det = K[0] * (K[4] * K[8] - K[5] * K[7]) - K[1] * (K[3] * K[8] - K[5] * K[6]) +
                           K[2] * (K[3] * K[7] - K[4] * K[6]);
        double Ki[9] = {(K[4] * K[8] - K[5] * K[7]) / det, (K[2] * K[7] - K[1] * K[8]) / det,
                        (K[1] * K[5] - K[2] * K[4]) / det, (K[5] * K[6] - K[3] * K[8]) / det,
                        (K[0] * K[8] - K[2] * K[6]) / det, (K[2] * K[3] - K[0] * K[5]) / det,
                        (K[3] * K[7] - K[4] * K[6]) / det, (K[1] * K[6] - K[0] * K[7]) / det,
                        (K[0] * K[4] - K[1] * K[3]) / det};
        // pixel (x, y, 1) -> world direction R^T K^-1 (x, y, 1), then / voxel_size
        for (int r = 0; r < 3; ++r)
            for (int col = 0; col < 3; ++col) {
                double v = 0.0;
                for (int q = 0; q < 3; ++q) v += R[3 * q + r] * Ki[3 * q + col];
                inv[c].minv[3 * r + col] = (float)(v / vs);
            }
        // camera centre C = -R^T t in voxel-index coordinates (voxel centres at integers)
        for (int r = 0; r < 3; ++r) {
            double C = 0.0;
            for (int q = 0; q < 3; ++q) C -= R[3 * q + r] * t[q];
            inv[c].qc[r] = (float)((C - grid.origin[r]) / vs - 0.5);
        }
        // frustum widening: a bound on the float32 error of the forward
        // projection over the grid (as the planner bounds it per tile), x4,
        // at least 0.05 px; 0.5 px if the grid reaches behind the camera
        const float *m = f.cam[c].m;
        double su = std::fabs(m[3]), sv = std::fabs(m[7]), sw = std::fabs(m[11]);
        for (int a = 0; a < 3; ++a) {
            su += std::fabs(m[a]) * half[a];
            sv += std::fabs(m[4 + a]) * half[a];
            sw += std::fabs(m[8 + a]) * half[a];
        }
        double wmin = 1e300, xa = 0.0, ya = 0.0;
        for (int corner = 0; corner < 8; ++corner) {
            const int ii = (corner & 1) ? grid.nx - 1 : 0, jj = (corner & 2) ? grid.ny - 1 : 0,
                      kk = (corner & 4) ? grid.nz - 1 : 0;
            const double X[3] = {grid.origin[0] + (ii + 0.5) * vs, grid.origin[1] + (jj + 0.5) * vs,
                                 grid.origin[2] + (kk + 0.5) * vs};
            double xc[3], uvw[3];
            for (int r = 0; r < 3; ++r) xc[r] = R[3 * r] * X[0] + R[3 * r + 1] * X[1] + R[3 * r + 2] * X[2] + t[r];
            for (int r = 0; r < 3; ++r) uvw[r] = K[3 * r] * xc[0] + K[3 * r + 1] * xc[1] + K[3 * r + 2] * xc[2];
            wmin = std::min(wmin, uvw[2]);
            if (uvw[2] > 0) {
                xa = std::max(xa, std::fabs(uvw[0] / uvw[2]));
                ya = std::max(ya, std::fabs(uvw[1] / uvw[2]));
            }
        }
        double margin = 0.5;
        if (wmin > 1e-3 * sw) {
            const double dw = 8 * eps32 * sw;
            const double ex = 2 * ((8 * eps32 * su + xa * dw) / wmin + xa * std::ldexp(1.0, -21));
            const double ey = 2 * ((8 * eps32 * sv + ya * dw) / wmin + ya * std::ldexp(1.0, -21));
            margin = std::min(0.5, std::max(0.05, 4 * std::max(ex, ey)));
        }
        inv[c].margin = (float)margin;
    }
}

}  // namespace psfs
