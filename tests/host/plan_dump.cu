// Host-only test driver: runs the fuse planner of libpsfs (psfs_plan.cu) on a
// grid and camera rig read from a text file and prints the projection
// matrices and every (tile, camera) record, so that a test can check the
// records against the voxel projections without a GPU.
//
// input:  nx ny nz ox oy oz voxel_size n_cams map_dtype lanes_x warps voxels_z staged
//         then per camera: width height K[9] R[9] t[3]
// output: "TX TY TZ", n_cams lines of 12 matrix entries, then per record
//         "tile c x y z w" (flags in the high half of w)
#include <cstdio>
#include <vector>

#include "psfs_internal.cuh"

int main(int argc, char **argv)
{
    if (argc < 2) return 2;
    FILE *f = std::fopen(argv[1], "r");
    if (!f) return 2;
    psfs_grid g;
    int n = 0, map_dtype = 0;
    psfs::FuseShape shape;
    if (std::fscanf(f, "%d %d %d %lf %lf %lf %lf %d %d %d %d %d %d", &g.nx, &g.ny, &g.nz, &g.origin[0],
                    &g.origin[1], &g.origin[2], &g.voxel_size, &n, &map_dtype, &shape.lx, &shape.wy, &shape.tz,
                    &shape.staged) != 13)
        return 2;
    if (!psfs::fuse_shape_supported(shape)) return 3;
    std::vector<psfs_camera> cams(n);
    for (int c = 0; c < n; ++c) {
        if (std::fscanf(f, "%d %d", &cams[c].width, &cams[c].height) != 2) return 2;
        for (int q = 0; q < 9; ++q) std::fscanf(f, "%lf", &cams[c].K[q]);
        for (int q = 0; q < 9; ++q) std::fscanf(f, "%lf", &cams[c].R[q]);
        for (int q = 0; q < 3; ++q) std::fscanf(f, "%lf", &cams[c].t[q]);
    }
    std::fclose(f);
    psfs_params p;
    psfs_params_default(&p);
    p.map_dtype = map_dtype;
    psfs::FuseArgs fa;
    std::vector<uint64_t> tiles;
    std::vector<int4> rec;
    psfs::plan_fuse(g, cams.data(), n, p, shape, &fa, &tiles, &rec);
    std::printf("%d %d %d %d\n", shape.tile_x(), shape.tile_y(), shape.tile_z(), psfs::stage_cap_elems(map_dtype));
    for (int c = 0; c < n; ++c) {
        for (int q = 0; q < 12; ++q) std::printf("%.9g ", fa.cam[c].m[q]);
        std::printf("\n");
    }
    for (size_t t = 0; t < tiles.size(); ++t)
        for (int c = 0; c < n; ++c) {
            const int4 r = rec[t * n + c];
            std::printf("%llu %d %d %d %d %d\n", (unsigned long long)tiles[t], c, r.x, r.y, r.z, r.w);
        }
    return 0;
}
