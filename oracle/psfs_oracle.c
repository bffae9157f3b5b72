/*
 * psfs_oracle.c -- FP64 CPU oracle for probabilistic shape-from-silhouette.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the plain, slow, obviously correct
 * statement of what the reconstruction computes, written from the paper
 * (Section 2.2.2, Eq. 1-9).  Only the test suite, the smoke check and the CPU
 * baseline leg of the benchmark may load it.  The CUDA library never links,
 * includes or calls it, and it shares no header, helper or constant with it.
 *
 * Every quantity is double precision.  Nothing here is blocked, fused or
 * reordered: each function follows the equations in the paper's order.
 *
 * Conventions (the readings of the paper where it is silent or ambiguous,
 * each with the passage it rests on):
 *   - pixel colour I is an RGB triple; the background likelihood is a single
 *     Gaussian per pixel with independent channels (diagonal covariance,
 *     variance given per channel)                               (Eq. 1, text)
 *   - the foreground likelihood is uniform over the RGB cube, density U,
 *     passed as log U (default -3 log 256)                      (Eq. 1, text)
 *   - equal priors P(F=1) = P(F=0) = 1/2                        (Eq. 1-2)
 *   - camera: x_cam = R X + t, (u, v, w) = K x_cam, image point (u/w, v/w);
 *     pixel (x, y) covers [x, x+1) x [y, y+1); the voxel centre is projected
 *     and looked up in the pixel containing it                  (Eq. 3 text)
 *   - a camera in which the voxel centre is behind the camera or outside the
 *     image contributes no factor                               (silent)
 *   - sensor model with detection rate P_D and false-alarm rate P_FA; with
 *     P_D = 1, P_FA = 0 it is exactly Eq. 6-9                   (Eq. 5-9)
 *   - occupied  <=>  posterior > threshold (strict)             (Sec. 2.2.2 end)
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* camera record: K[9], R[9], t[3] (row-major), 21 doubles per camera */
#define ORACLE_CAM_STRIDE 21

/* --------------------------------------------------------------------- */
/* Eq. 1-2: silhouette likelihood map.                                    */
/*   N = prod_c (2 pi var_c)^(-1/2) exp(-(I_c - mu_c)^2 / (2 var_c))      */
/*   SLM = U P(F=1) / (U P(F=1) + N P(F=0)) = U / (U + N)   (priors 1/2)  */
/* --------------------------------------------------------------------- */
void oracle_slm(int64_t n_pix, const uint8_t *img, const float *mean, const float *var,
                double log_fg_density, double *slm)
{
    const double U = exp(log_fg_density);
    const double pi = 3.14159265358979323846;
    for (int64_t p = 0; p < n_pix; ++p) {
        double N = 1.0;
        for (int c = 0; c < 3; ++c) {
            double I = (double)img[3 * p + c];
            double mu = (double)mean[3 * p + c];
            double v = (double)var[3 * p + c];
            double d = I - mu;
            N *= exp(-d * d / (2.0 * v)) / sqrt(2.0 * pi * v);
        }
        double pf1 = 0.5, pf0 = 0.5;
        slm[p] = U * pf1 / (U * pf1 + N * pf0);
    }
}

/* --------------------------------------------------------------------- */
/* Projection of a world point (the "projection of voxel V_i", Eq. 3).    */
/* Returns 1 and the pixel if the point is in front of the camera and     */
/* inside the image; *xy gets the continuous image position either way    */
/* (when w > 0).  Returns 0 if not seen.                                  */
/* --------------------------------------------------------------------- */
int oracle_project(const double *cam, int W, int H, const double X[3],
                   int *px, int *py, double xy[2], double *w_out)
{
    const double *K = cam, *R = cam + 9, *t = cam + 18;
    double xc[3];
    for (int r = 0; r < 3; ++r)
        xc[r] = R[3 * r + 0] * X[0] + R[3 * r + 1] * X[1] + R[3 * r + 2] * X[2] + t[r];
    double uvw[3];
    for (int r = 0; r < 3; ++r)
        uvw[r] = K[3 * r + 0] * xc[0] + K[3 * r + 1] * xc[1] + K[3 * r + 2] * xc[2];
    *w_out = uvw[2];
    if (!(uvw[2] > 0.0)) return 0;
    double x = uvw[0] / uvw[2];
    double y = uvw[1] / uvw[2];
    xy[0] = x;
    xy[1] = y;
    if (!(x >= 0.0 && x < (double)W && y >= 0.0 && y < (double)H)) return 0;
    *px = (int)floor(x);
    *py = (int)floor(y);
    return 1;
}

static double dist_to_integer(double x)
{
    return fabs(x - floor(x + 0.5));
}

/* --------------------------------------------------------------------- */
/* Eq. 5 with Eq. 6-9 generalised by the rates:                           */
/*   P(S | O=0, V=0) = P_FA s + (1 - P_FA)(1 - s)          ("nothing")     */
/*   P(S | O, V) with O = 1 or V = 1 = P_D s + (1 - P_D)(1 - s)            */
/*   P(S | V=1) = sum_O P(S | O, V=1) P(O) = a                             */
/*   P(S | V=0) = P(O=0) f + P(O=1) a = (f + a) / 2                        */
/* --------------------------------------------------------------------- */
static void sensor_terms(double s, double pd, double pfa, double *a, double *b)
{
    double p_o1 = 0.5, p_o0 = 0.5;
    double something = pd * s + (1.0 - pd) * (1.0 - s);   /* V = 1 or O = 1 */
    double nothing = pfa * s + (1.0 - pfa) * (1.0 - s);   /* V = 0 and O = 0 */
    *a = something * p_o0 + something * p_o1;              /* V = 1 */
    *b = nothing * p_o0 + something * p_o1;                /* V = 0 */
}

/* --------------------------------------------------------------------- */
/* Eq. 3-4: voxel posterior, literal product over the cameras.            */
/*   occ = prior prod a / (prior prod a + (1 - prior) prod b)             */
/* Outputs per voxel (linear index i + nx (j + ny k)):                     */
/*   occ, logodds = log(prior prod a) - log((1-prior) prod b),            */
/*   occupied = occ > threshold, boundary = 1 if in some camera the        */
/*   continuous projection lies within edge_eps px of a pixel edge or of   */
/*   the image border, n_seen = number of cameras that see the centre.     */
/* --------------------------------------------------------------------- */
void oracle_fuse(int nx, int ny, int nz, const double origin[3], double voxel_size,
                 int n_cams, const int *wh, const double *cams, const double *slm,
                 double pd, double pfa, double prior, double threshold, double edge_eps,
                 double *occ, double *logodds, uint8_t *occupied, uint8_t *boundary,
                 uint8_t *n_seen)
{
    /* per-camera offsets into the concatenated maps */
    int64_t *map_off = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n_cams > 0 ? n_cams : 1));
    int64_t off = 0;
    for (int c = 0; c < n_cams; ++c) {
        map_off[c] = off;
        off += (int64_t)wh[2 * c] * wh[2 * c + 1];
    }
    for (int k = 0; k < nz; ++k)
        for (int j = 0; j < ny; ++j)
            for (int i = 0; i < nx; ++i) {
                int64_t v = (int64_t)i + (int64_t)nx * ((int64_t)j + (int64_t)ny * k);
                double X[3] = {origin[0] + (i + 0.5) * voxel_size,
                               origin[1] + (j + 0.5) * voxel_size,
                               origin[2] + (k + 0.5) * voxel_size};
                double A = 1.0, B = 1.0;   /* P({S}|V=1), P({S}|V=0), Eq. 4 */
                int bnd = 0, seen = 0;
                for (int c = 0; c < n_cams; ++c) {
                    int W = wh[2 * c], H = wh[2 * c + 1];
                    int px = 0, py = 0;
                    double xy[2] = {-1e300, -1e300}, w = 0.0;
                    int vis = oracle_project(cams + ORACLE_CAM_STRIDE * c, W, H, X, &px, &py, xy, &w);
                    if (w > 0.0 && xy[0] >= -edge_eps && xy[0] <= W + edge_eps &&
                        xy[1] >= -edge_eps && xy[1] <= H + edge_eps &&
                        (dist_to_integer(xy[0]) < edge_eps || dist_to_integer(xy[1]) < edge_eps))
                        bnd = 1;
                    if (!vis) continue;
                    ++seen;
                    double s = slm[map_off[c] + (int64_t)py * W + px];
                    double a, b;
                    sensor_terms(s, pd, pfa, &a, &b);
                    A *= a;
                    B *= b;
                }
                double num = prior * A;
                double den = prior * A + (1.0 - prior) * B;
                occ[v] = num / den;
                logodds[v] = log(prior * A) - log((1.0 - prior) * B);
                occupied[v] = occ[v] > threshold ? 1 : 0;
                boundary[v] = (uint8_t)bnd;
                n_seen[v] = (uint8_t)(seen > 255 ? 255 : seen);
            }
    free(map_off);
}

/* Thresholded voxels as ascending linear indices; returns the count. */
int64_t oracle_compact(int64_t n_vox, const uint8_t *occupied, uint32_t *list)
{
    int64_t n = 0;
    for (int64_t v = 0; v < n_vox; ++v)
        if (occupied[v]) list[n++] = (uint32_t)v;
    return n;
}

/* --------------------------------------------------------------------- */
/* Particle weights of the tracker (Sec. 2.3.2, Eq. 14-16): the match of  */
/* each particle's projected body model with the voxel silhouettes and    */
/* their edges in every camera.                                            */
/*   Edge map: a pixel is an edge iff it is set in the silhouette and one  */
/*   of its 4 neighbours inside the image is not.                          */
/*   A particle is n_cyl cylinders (a[3], b[3], r), 7 values each.  For a  */
/*   cylinder and camera centre C = -R^T t: u = (b - a) / |b - a|, n =     */
/*   unit(u x (m - C)) with m = (a + b) / 2 (the direction of the outline  */
/*   seen from C).  Silhouette samples: a + t (b - a) + w r n with         */
/*   t = (k + 1/2) / kt, w = (2 l + 1) / kw - 1; edge samples: the same t, */
/*   w = -1 and +1.  A sample is looked up in the pixel containing its     */
/*   projection; behind the camera or outside the image its value is 0.    */
/*   S_r = (1 / N_r) sum (1 - p_r), S_e = (1 / N_e) sum (1 - p_e) per      */
/*   camera (Eq. 14-15), weight = exp(-sum_c (S_e + S_r)) (Eq. 16).        */
/*   ambiguous[p * n_cams + c] counts the samples whose projection is      */
/*   within edge_eps px of a pixel edge (the looked-up pixel may differ in */
/*   another precision).                                                   */
/* --------------------------------------------------------------------- */
void oracle_edges(int n_cams, int W, int H, const uint8_t *masks, uint8_t *edges)
{
    for (int c = 0; c < n_cams; ++c) {
        const uint8_t *m = masks + (int64_t)c * W * H;
        uint8_t *e = edges + (int64_t)c * W * H;
        for (int y = 0; y < H; ++y)
            for (int x = 0; x < W; ++x) {
                int edge = 0;
                if (m[(int64_t)y * W + x]) {
                    if (x > 0 && !m[(int64_t)y * W + x - 1]) edge = 1;
                    if (x + 1 < W && !m[(int64_t)y * W + x + 1]) edge = 1;
                    if (y > 0 && !m[(int64_t)(y - 1) * W + x]) edge = 1;
                    if (y + 1 < H && !m[(int64_t)(y + 1) * W + x]) edge = 1;
                }
                e[(int64_t)y * W + x] = (uint8_t)edge;
            }
    }
}

static int sample_value(const double *cam, int W, int H, const uint8_t *map, const double X[3], double edge_eps,
                        int *ambiguous)
{
    int px, py;
    double xy[2], w;
    int vis = oracle_project(cam, W, H, X, &px, &py, xy, &w);
    if (w > 0.0 && (dist_to_integer(xy[0]) < edge_eps || dist_to_integer(xy[1]) < edge_eps)) ++*ambiguous;
    if (!vis) return 0;
    return map[(int64_t)py * W + px] != 0;
}

void oracle_particle_weights(int n_cams, const int *wh, const double *cams, const uint8_t *masks,
                             int64_t n_particles, int n_cyl, const double *cyl, int kt, int kw, double edge_eps,
                             double *weights, double *terms, int *ambiguous)
{
    const int W = wh[0], H = wh[1];
    uint8_t *edges = (uint8_t *)malloc((size_t)n_cams * W * H);
    oracle_edges(n_cams, W, H, masks, edges);
    for (int64_t p = 0; p < n_particles; ++p) {
        double total = 0.0;
        for (int c = 0; c < n_cams; ++c) {
            const double *cam = cams + ORACLE_CAM_STRIDE * c, *R = cam + 9, *t = cam + 18;
            const uint8_t *mask = masks + (int64_t)c * W * H, *edge = edges + (int64_t)c * W * H;
            double C[3];
            for (int r = 0; r < 3; ++r) C[r] = -(R[r] * t[0] + R[3 + r] * t[1] + R[6 + r] * t[2]);
            int miss_r = 0, miss_e = 0, amb = 0;
            for (int q = 0; q < n_cyl; ++q) {
                const double *cy = cyl + ((size_t)p * n_cyl + q) * 7;
                const double *A = cy, *B = cy + 3, rad = cy[6];
                double u[3], mid[3], view[3], n[3];
                for (int r = 0; r < 3; ++r) {
                    u[r] = B[r] - A[r];
                    mid[r] = 0.5 * (A[r] + B[r]);
                    view[r] = mid[r] - C[r];
                }
                n[0] = u[1] * view[2] - u[2] * view[1];
                n[1] = u[2] * view[0] - u[0] * view[2];
                n[2] = u[0] * view[1] - u[1] * view[0];
                double nn = sqrt(n[0] * n[0] + n[1] * n[1] + n[2] * n[2]);
                for (int r = 0; r < 3; ++r) n[r] = nn > 0.0 ? n[r] / nn : 0.0;
                for (int k = 0; k < kt; ++k) {
                    const double tt = (k + 0.5) / kt;
                    for (int l = 0; l < kw; ++l) {
                        const double ww = (2.0 * l + 1.0) / kw - 1.0;
                        double X[3];
                        for (int r = 0; r < 3; ++r) X[r] = A[r] + tt * u[r] + ww * rad * n[r];
                        miss_r += 1 - sample_value(cam, W, H, mask, X, edge_eps, &amb);
                    }
                    for (int side = -1; side <= 1; side += 2) {
                        double X[3];
                        for (int r = 0; r < 3; ++r) X[r] = A[r] + tt * u[r] + side * rad * n[r];
                        miss_e += 1 - sample_value(cam, W, H, edge, X, edge_eps, &amb);
                    }
                }
            }
            const double s_r = (double)miss_r / (n_cyl * kt * kw), s_e = (double)miss_e / (n_cyl * kt * 2);
            if (terms) {
                terms[(p * n_cams + c) * 2 + 0] = s_e;
                terms[(p * n_cams + c) * 2 + 1] = s_r;
            }
            if (ambiguous) ambiguous[p * n_cams + c] = amb;
            total += s_e + s_r;
        }
        weights[p] = exp(-total);
    }
    free(edges);
}

/* --------------------------------------------------------------------- */
/* Silhouettes of a voxel set (Sec. 2.3: the projection of the voxels in  */
/* each camera is the tracker's prior knowledge, matched against the      */
/* particles' projected models).  Pixel (x, y) of camera c is set iff the */
/* ray from the camera centre C = -R^T t through the pixel centre         */
/* (x + 1/2, y + 1/2) meets, at a positive ray parameter, the cube of a   */
/* listed voxel: origin + [i, i+1] x [j, j+1] x [k, k+1] * voxel_size,    */
/* grown by `grow` voxel sizes on every side (grow = 0: the cube itself). */
/* Brute force: every pixel against every listed voxel, slab test.        */
/* masks: [n_cams][H][W] bytes.                                           */
/* --------------------------------------------------------------------- */
static void inverse3(const double *A, double *Ai)
{
    double det = A[0] * (A[4] * A[8] - A[5] * A[7]) - A[1] * (A[3] * A[8] - A[5] * A[6]) +
                 A[2] * (A[3] * A[7] - A[4] * A[6]);
    Ai[0] = (A[4] * A[8] - A[5] * A[7]) / det;
    Ai[1] = (A[2] * A[7] - A[1] * A[8]) / det;
    Ai[2] = (A[1] * A[5] - A[2] * A[4]) / det;
    Ai[3] = (A[5] * A[6] - A[3] * A[8]) / det;
    Ai[4] = (A[0] * A[8] - A[2] * A[6]) / det;
    Ai[5] = (A[2] * A[3] - A[0] * A[5]) / det;
    Ai[6] = (A[3] * A[7] - A[4] * A[6]) / det;
    Ai[7] = (A[1] * A[6] - A[0] * A[7]) / det;
    Ai[8] = (A[0] * A[4] - A[1] * A[3]) / det;
}

/* does C + t d, t > 0, meet the box [lo, hi]? */
static int ray_hits_box(const double C[3], const double d[3], const double lo[3], const double hi[3])
{
    double t_in = 0.0, t_out = INFINITY;
    for (int a = 0; a < 3; ++a) {
        if (d[a] == 0.0) {
            if (C[a] < lo[a] || C[a] > hi[a]) return 0;
            continue;
        }
        double t1 = (lo[a] - C[a]) / d[a], t2 = (hi[a] - C[a]) / d[a];
        if (t1 > t2) {
            double tmp = t1;
            t1 = t2;
            t2 = tmp;
        }
        if (t1 > t_in) t_in = t1;
        if (t2 < t_out) t_out = t2;
    }
    return t_in <= t_out;
}

void oracle_reproject(int nx, int ny, int nz, const double origin[3], double voxel_size, int n_cams,
                      const int *wh, const double *cams, int64_t n_list, const uint32_t *list, double grow,
                      uint8_t *masks)
{
    int64_t off = 0;
    for (int c = 0; c < n_cams; ++c) {
        const int W = wh[2 * c], H = wh[2 * c + 1];
        const double *K = cams + ORACLE_CAM_STRIDE * c, *R = K + 9, *t = K + 18;
        double Ki[9], C[3];
        inverse3(K, Ki);
        for (int r = 0; r < 3; ++r) C[r] = -(R[r] * t[0] + R[3 + r] * t[1] + R[6 + r] * t[2]);
        for (int y = 0; y < H; ++y)
            for (int x = 0; x < W; ++x) {
                const double p[3] = {x + 0.5, y + 0.5, 1.0};
                double q[3], d[3];
                for (int r = 0; r < 3; ++r) q[r] = Ki[3 * r] * p[0] + Ki[3 * r + 1] * p[1] + Ki[3 * r + 2] * p[2];
                for (int r = 0; r < 3; ++r) d[r] = R[r] * q[0] + R[3 + r] * q[1] + R[6 + r] * q[2];
                uint8_t hit = 0;
                for (int64_t e = 0; e < n_list && !hit; ++e) {
                    const int64_t v = list[e];
                    const int i = (int)(v % nx), j = (int)((v / nx) % ny), k = (int)(v / ((int64_t)nx * ny));
                    if (k >= nz) continue;
                    const double lo[3] = {origin[0] + (i - grow) * voxel_size, origin[1] + (j - grow) * voxel_size,
                                          origin[2] + (k - grow) * voxel_size};
                    const double hi[3] = {origin[0] + (i + 1 + grow) * voxel_size,
                                          origin[1] + (j + 1 + grow) * voxel_size,
                                          origin[2] + (k + 1 + grow) * voxel_size};
                    hit = (uint8_t)ray_hits_box(C, d, lo, hi);
                }
                masks[off + (int64_t)y * W + x] = hit;
            }
        off += (int64_t)W * H;
    }
}

/* --------------------------------------------------------------------- */
/* Spatial smoothing of the voxel probabilities before the threshold      */
/* (end of Sec. 2.2.2; Sec. 3.3.3 step (d)).  The paper does not give the */
/* filter; this is the 3 x 3 x 3 box mean over the neighbours inside the  */
/* grid (each voxel's own 27-neighbourhood clipped to the grid, divided   */
/* by the number of voxels in it).  occupied <=> smoothed > threshold.    */
/* --------------------------------------------------------------------- */
void oracle_smooth(int nx, int ny, int nz, const double *prob, double threshold, double *smoothed,
                   uint8_t *occupied)
{
    for (int k = 0; k < nz; ++k)
        for (int j = 0; j < ny; ++j)
            for (int i = 0; i < nx; ++i) {
                double sum = 0.0;
                int n = 0;
                for (int dk = -1; dk <= 1; ++dk)
                    for (int dj = -1; dj <= 1; ++dj)
                        for (int di = -1; di <= 1; ++di) {
                            int a = i + di, b = j + dj, c = k + dk;
                            if (a < 0 || b < 0 || c < 0 || a >= nx || b >= ny || c >= nz) continue;
                            sum += prob[(int64_t)a + (int64_t)nx * ((int64_t)b + (int64_t)ny * c)];
                            ++n;
                        }
                int64_t v = (int64_t)i + (int64_t)nx * ((int64_t)j + (int64_t)ny * k);
                smoothed[v] = sum / n;
                occupied[v] = smoothed[v] > threshold;
            }
}

/* --------------------------------------------------------------------- */
/* Inner-voxel removal (end of Sec. 2.2.2; Sec. 3.3.3 step (e)): the      */
/* surface voxels are the occupied voxels with at least one of their six  */
/* face neighbours not occupied; a neighbour outside the grid counts as   */
/* not occupied.  Ascending linear indices; returns the count.            */
/* --------------------------------------------------------------------- */
static int occupied_at(int nx, int ny, int nz, const uint8_t *occupied, int i, int j, int k)
{
    if (i < 0 || j < 0 || k < 0 || i >= nx || j >= ny || k >= nz) return 0;
    return occupied[(int64_t)i + (int64_t)nx * ((int64_t)j + (int64_t)ny * k)] != 0;
}

int64_t oracle_surface(int nx, int ny, int nz, const uint8_t *occupied, uint32_t *list)
{
    int64_t n = 0;
    for (int k = 0; k < nz; ++k)
        for (int j = 0; j < ny; ++j)
            for (int i = 0; i < nx; ++i) {
                if (!occupied_at(nx, ny, nz, occupied, i, j, k)) continue;
                int inner = occupied_at(nx, ny, nz, occupied, i - 1, j, k) &&
                            occupied_at(nx, ny, nz, occupied, i + 1, j, k) &&
                            occupied_at(nx, ny, nz, occupied, i, j - 1, k) &&
                            occupied_at(nx, ny, nz, occupied, i, j + 1, k) &&
                            occupied_at(nx, ny, nz, occupied, i, j, k - 1) &&
                            occupied_at(nx, ny, nz, occupied, i, j, k + 1);
                if (!inner) list[n++] = (uint32_t)((int64_t)i + (int64_t)nx * ((int64_t)j + (int64_t)ny * k));
            }
    return n;
}

/* --------------------------------------------------------------------- */
/* Adjoint of Eq. 3-4 with respect to the maps.                           */
/* Given dLoss/docc per voxel:                                            */
/*   dLoss/dlogodds_v = docc_v occ_v (1 - occ_v)                          */
/*   dlogodds_v/ds = (da/ds)/a - (db/ds)/b at the pixel v projects to,    */
/*   da/ds = 2 P_D - 1, df/ds = 2 P_FA - 1, db/ds = (da/ds + df/ds) / 2   */
/*   dLoss/ds_p = sum over voxels that project to p (free scatter here).  */
/* --------------------------------------------------------------------- */
void oracle_backward_slm(int nx, int ny, int nz, const double origin[3], double voxel_size,
                         int n_cams, const int *wh, const double *cams, const double *slm,
                         double pd, double pfa, double prior, const double *d_occ,
                         double *d_slm)
{
    int64_t *map_off = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n_cams > 0 ? n_cams : 1));
    int64_t off = 0;
    for (int c = 0; c < n_cams; ++c) {
        map_off[c] = off;
        off += (int64_t)wh[2 * c] * wh[2 * c + 1];
    }
    memset(d_slm, 0, sizeof(double) * (size_t)off);
    int *pxs = (int *)malloc(sizeof(int) * (size_t)(n_cams > 0 ? n_cams : 1));
    int *pys = (int *)malloc(sizeof(int) * (size_t)(n_cams > 0 ? n_cams : 1));
    int *vis = (int *)malloc(sizeof(int) * (size_t)(n_cams > 0 ? n_cams : 1));
    const double da = 2.0 * pd - 1.0, df = 2.0 * pfa - 1.0, db = 0.5 * (da + df);
    for (int k = 0; k < nz; ++k)
        for (int j = 0; j < ny; ++j)
            for (int i = 0; i < nx; ++i) {
                int64_t v = (int64_t)i + (int64_t)nx * ((int64_t)j + (int64_t)ny * k);
                double X[3] = {origin[0] + (i + 0.5) * voxel_size,
                               origin[1] + (j + 0.5) * voxel_size,
                               origin[2] + (k + 0.5) * voxel_size};
                double A = 1.0, B = 1.0;
                for (int c = 0; c < n_cams; ++c) {
                    double xy[2], w;
                    vis[c] = oracle_project(cams + ORACLE_CAM_STRIDE * c, wh[2 * c], wh[2 * c + 1],
                                            X, &pxs[c], &pys[c], xy, &w);
                    if (!vis[c]) continue;
                    double s = slm[map_off[c] + (int64_t)pys[c] * wh[2 * c] + pxs[c]];
                    double a, b;
                    sensor_terms(s, pd, pfa, &a, &b);
                    A *= a;
                    B *= b;
                }
                double occ = prior * A / (prior * A + (1.0 - prior) * B);
                double dl = d_occ[v] * occ * (1.0 - occ);
                for (int c = 0; c < n_cams; ++c) {
                    if (!vis[c]) continue;
                    int64_t p = map_off[c] + (int64_t)pys[c] * wh[2 * c] + pxs[c];
                    double s = slm[p];
                    double a, b;
                    sensor_terms(s, pd, pfa, &a, &b);
                    d_slm[p] += dl * (da / a - db / b);
                }
            }
    free(pxs);
    free(pys);
    free(vis);
    free(map_off);
}

/* --------------------------------------------------------------------- */
/* Adjoint of Eq. 1-2 with respect to the background mean and variance.  */
/*   ds/dmu_c  = -s (1 - s) (I_c - mu_c) / var_c                           */
/*   ds/dvar_c =  s (1 - s) (1 / (2 var_c) - (I_c - mu_c)^2 / (2 var_c^2)) */
/* --------------------------------------------------------------------- */
void oracle_backward_background(int64_t n_pix, const uint8_t *img, const float *mean,
                                const float *var, const double *slm, const double *d_slm,
                                double *d_mean, double *d_var)
{
    for (int64_t p = 0; p < n_pix; ++p) {
        double s = slm[p];
        double g = d_slm[p] * s * (1.0 - s);
        for (int c = 0; c < 3; ++c) {
            double d = (double)img[3 * p + c] - (double)mean[3 * p + c];
            double v = (double)var[3 * p + c];
            d_mean[3 * p + c] = -g * d / v;
            d_var[3 * p + c] = g * (1.0 / (2.0 * v) - d * d / (2.0 * v * v));
        }
    }
}

/* --------------------------------------------------------------------- */
/* Eq. 3-4 for a list of voxels only (same arithmetic as oracle_fuse, for */
/* finite differences on large grids, where only the voxels that project */
/* into a perturbed pixel change).                                        */
/* --------------------------------------------------------------------- */
void oracle_fuse_subset(int nx, int ny, int nz, const double origin[3], double voxel_size,
                        int n_cams, const int *wh, const double *cams, const double *slm,
                        double pd, double pfa, double prior, int64_t n_sub, const int64_t *idx,
                        double *occ)
{
    int64_t *map_off = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n_cams > 0 ? n_cams : 1));
    int64_t off = 0;
    for (int c = 0; c < n_cams; ++c) {
        map_off[c] = off;
        off += (int64_t)wh[2 * c] * wh[2 * c + 1];
    }
    for (int64_t n = 0; n < n_sub; ++n) {
        int64_t v = idx[n];
        int i = (int)(v % nx), j = (int)((v / nx) % ny), k = (int)(v / ((int64_t)nx * ny));
        (void)nz;
        double X[3] = {origin[0] + (i + 0.5) * voxel_size, origin[1] + (j + 0.5) * voxel_size,
                       origin[2] + (k + 0.5) * voxel_size};
        double A = 1.0, B = 1.0;
        for (int c = 0; c < n_cams; ++c) {
            int W = wh[2 * c], px = 0, py = 0;
            double xy[2], w;
            if (!oracle_project(cams + ORACLE_CAM_STRIDE * c, W, wh[2 * c + 1], X, &px, &py, xy, &w)) continue;
            double s = slm[map_off[c] + (int64_t)py * W + px];
            double a, b;
            sensor_terms(s, pd, pfa, &a, &b);
            A *= a;
            B *= b;
        }
        occ[n] = prior * A / (prior * A + (1.0 - prior) * B);
    }
    free(map_off);
}

/* Pixel offset (py * W + px) of every voxel centre in every camera, -1 where
 * the camera does not see it: out[c * n_vox + v]. */
void oracle_voxel_pixels(int nx, int ny, int nz, const double origin[3], double voxel_size, int n_cams,
                         const int *wh, const double *cams, int32_t *out)
{
    int64_t n_vox = (int64_t)nx * ny * nz;
    for (int k = 0; k < nz; ++k)
        for (int j = 0; j < ny; ++j)
            for (int i = 0; i < nx; ++i) {
                int64_t v = (int64_t)i + (int64_t)nx * ((int64_t)j + (int64_t)ny * k);
                double X[3] = {origin[0] + (i + 0.5) * voxel_size, origin[1] + (j + 0.5) * voxel_size,
                               origin[2] + (k + 0.5) * voxel_size};
                for (int c = 0; c < n_cams; ++c) {
                    int px = 0, py = 0;
                    double xy[2], w;
                    int vis = oracle_project(cams + ORACLE_CAM_STRIDE * c, wh[2 * c], wh[2 * c + 1], X, &px, &py, xy, &w);
                    out[(int64_t)c * n_vox + v] = vis ? py * wh[2 * c] + px : -1;
                }
            }
}
