// psfs_owners.cu -- owner lists and the pixel pass of the adjoint.
//
// The adjoint of the fusion (Eq. 3-4 summed in log space) sends dLoss/dL of
// every voxel back to the one pixel per camera that the voxel's centre
// projects into (Eq. 3):  dLoss/dg_kp = sum over voxels v with pix_k(v) = p
// of dLoss/dL_v.  Which voxels a pixel owns depends on the grid and the rig
// only, so it is worked out once per handle, with the forward's own float32
// projection (project_voxel, the same helper and the same arithmetic as the
// fusion kernels, so the ownership is the forward's bit for bit):
//
//   count  one thread per voxel, per camera the pixel it falls in, an integer
//          atomicAdd on that pixel's count;
//   scan   exclusive prefix sum of the counts: the offsets of each pixel's
//          segment (a two-level block scan);
//   fill   the same projection again; each voxel claims a slot of its
//          pixel's segment (integer atomics, so the order is arbitrary);
//   sort   one thread per pixel sorts its segment by voxel index.
//
// The pixel pass of every frame then owns one pixel per thread and adds the
// dLoss/dL of its segment's voxels in ascending voxel order: no float
// atomics, the same order on every run and in every form (one frame per call
// or eight frames per pass), so the gradients are deterministic and the
// batched pass is bit-identical to one frame per call.  The work is one load
// per (voxel, camera) pair, instead of a walk along each pixel's ray.
#include "psfs_fuse_common.cuh"

namespace psfs {

namespace {

constexpr int kScanThreads = 1024;
constexpr int kScanItems = 4;
constexpr int kScanChunk = kScanThreads * kScanItems;   // entries per block of the first level
constexpr int kScanTopItems = 64;                       // second level: one block, 64 sums per thread

// Voxel v's centre in the centred index coordinates of the fusion kernels.
__device__ __forceinline__ void voxel_coords(const FuseArgs &a, uint64_t v, float &fi, float &fj, float &fk)
{
    const uint64_t nxy = (uint64_t)a.nx * (uint64_t)a.ny;
    const uint32_t k = (uint32_t)(v / nxy);
    const uint32_t r = (uint32_t)(v - (uint64_t)k * nxy);
    const uint32_t j = r / (uint32_t)a.nx;
    const uint32_t i = r - j * (uint32_t)a.nx;
    fi = (float)i - a.ci;
    fj = (float)j - a.cj;
    fk = (float)k - a.ck;
}

__global__ void __launch_bounds__(256) owner_count_kernel(const __grid_constant__ FuseArgs a, uint32_t *cnt)
{
    const uint64_t n_vox = (uint64_t)a.nx * a.ny * a.nz;
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t v = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n_vox; v += stride) {
        float fi, fj, fk;
        voxel_coords(a, v, fi, fj, fk);
        for (int c = 0; c < a.n_cams; ++c) {
            int pix;
            if (project_voxel(a.cam[c].m, fi, fj, fk, (uint32_t)a.W, (uint32_t)a.H, &pix))
                atomicAdd(cnt + (int64_t)c * a.map_stride + pix, 1u);
        }
    }
}

__global__ void __launch_bounds__(256) owner_fill_kernel(const __grid_constant__ FuseArgs a, const uint32_t *off,
                                                         uint32_t *cursor, uint32_t *vox)
{
    const uint64_t n_vox = (uint64_t)a.nx * a.ny * a.nz;
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t v = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n_vox; v += stride) {
        float fi, fj, fk;
        voxel_coords(a, v, fi, fj, fk);
        for (int c = 0; c < a.n_cams; ++c) {
            int pix;
            if (project_voxel(a.cam[c].m, fi, fj, fk, (uint32_t)a.W, (uint32_t)a.H, &pix)) {
                const int64_t p = (int64_t)c * a.map_stride + pix;
                const uint32_t e = off[p] + atomicAdd(cursor + p, 1u);
                if (e < off[p + 1]) vox[e] = (uint32_t)v;   // the count pass made room: e is always inside
            }
        }
    }
}

// Insertion sort of each pixel's segment (segments hold a few voxels, the
// voxels along the pixel's ray; this runs once per handle).
__global__ void __launch_bounds__(256) owner_sort_kernel(const uint32_t *off, uint32_t *vox, int64_t n_pix)
{
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < n_pix; p += stride) {
        const uint32_t e0 = off[p], e1 = off[p + 1];
        for (uint32_t e = e0 + 1; e < e1; ++e) {
            const uint32_t x = vox[e];
            uint32_t q = e;
            while (q > e0 && vox[q - 1] > x) {
                vox[q] = vox[q - 1];
                --q;
            }
            vox[q] = x;
        }
    }
}

// Exclusive scan of one block's kScanThreads values in registers.
__device__ __forceinline__ uint32_t block_exclusive_scan(uint32_t x, uint32_t *s_warp, uint32_t *total)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t inc = x;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, inc, d);
        if (lane >= d) inc += y;
    }
    if (lane == 31) s_warp[warp] = inc;
    __syncthreads();
    if (warp == 0) {
        const uint32_t w = lane < (kScanThreads / 32) ? s_warp[lane] : 0u;
        uint32_t winc = w;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, winc, d);
            if (lane >= d) winc += y;
        }
        s_warp[lane] = winc - w;   // exclusive prefix of each warp
        if (lane == 31) *total = winc;
    }
    __syncthreads();
    return s_warp[warp] + inc - x;
}

// First level: out[i] = sum of in[chunk start .. i) for i < n_in, in[i >= n_in]
// read as 0; the chunk's total goes to sums[blockIdx.x].  n_out entries.
__global__ void __launch_bounds__(kScanThreads) scan_chunks_kernel(const uint32_t *in, int64_t n_in, uint32_t *out,
                                                                   int64_t n_out, uint32_t *sums)
{
    __shared__ uint32_t s_warp[32];
    __shared__ uint32_t s_total;
    const int64_t base = (int64_t)blockIdx.x * kScanChunk + (int64_t)threadIdx.x * kScanItems;
    uint32_t v[kScanItems];
    uint32_t t = 0;
#pragma unroll
    for (int q = 0; q < kScanItems; ++q) {
        v[q] = base + q < n_in ? in[base + q] : 0u;
        t += v[q];
    }
    uint32_t run = block_exclusive_scan(t, s_warp, &s_total);
#pragma unroll
    for (int q = 0; q < kScanItems; ++q) {
        if (base + q < n_out) out[base + q] = run;
        run += v[q];
    }
    if (threadIdx.x == 0) sums[blockIdx.x] = s_total;
}

// Second level, one block: exclusive scan of the chunk totals in place.
__global__ void __launch_bounds__(kScanThreads) scan_top_kernel(uint32_t *sums, int64_t n)
{
    __shared__ uint32_t s_warp[32];
    __shared__ uint32_t s_total;
    const int64_t base = (int64_t)threadIdx.x * kScanTopItems;
    uint32_t t = 0;
    for (int q = 0; q < kScanTopItems; ++q)
        if (base + q < n) t += sums[base + q];
    uint32_t run = block_exclusive_scan(t, s_warp, &s_total);
    for (int q = 0; q < kScanTopItems; ++q)
        if (base + q < n) {
            const uint32_t x = sums[base + q];
            sums[base + q] = run;
            run += x;
        }
}

__global__ void __launch_bounds__(256) scan_add_kernel(uint32_t *out, int64_t n, const uint32_t *sums)
{
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride)
        out[i] += sums[i / kScanChunk];
}

// Chain rule of one frame from the pixel's background loaded once (mu, h =
// 1 / (2 var), base = c0 - log(h0 h1 h2) / 2 = pixel_log_base, so that r =
// base + pixel_quad is pixel_log_odds bit for bit):
//   s = sigmoid(r) (the bits of sigmoid_fast), from u = e^-|r|;
//   dLoss/ds = acc (da / a(s) - db / b(s))            (Eq. 5-9, a, b linear in s)
//   dLoss/dr = dLoss/ds s (1 - s), with s (1 - s) = u / (1 + u)^2 (no cancellation)
//   dLoss/dmu_c, dLoss/dvar_c from dLoss/dr (Eq. 1).
__device__ __forceinline__ void chain_rule_pre(const BackwardArgs &b, const uint8_t *im, const float (&mu)[3],
                                               const float (&hh)[3], float base, float acc, float &dslm,
                                               float (&dm)[3], float (&dv)[3])
{
    dslm = 0.0f;
#pragma unroll
    for (int c = 0; c < 3; ++c) dm[c] = dv[c] = 0.0f;
    if (acc != 0.0f) {
        float dd[3];
#pragma unroll
        for (int c = 0; c < 3; ++c) dd[c] = (float)im[c] - mu[c];
        const float r = base + pixel_quad((float)im[0], (float)im[1], (float)im[2], mu[0], mu[1], mu[2], hh[0],
                                          hh[1], hh[2]);
        const float u = exp_fast(-fabsf(r));
        const float inv = rcp_approx(1.0f + u);
        const float s_val = r > 0.0f ? inv : u * inv;
        const float av = fmaf(b.da, s_val, b.one_minus_pd), bv = fmaf(b.db, s_val, b.one_minus_q);
        dslm = acc * (div_fast(b.da, av) - div_fast(b.db, bv));
        const float dr = dslm * (u * inv * inv);
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            dm[c] = -2.0f * dr * dd[c] * hh[c];
            dv[c] = dr * hh[c] * (1.0f - 2.0f * dd[c] * dd[c] * hh[c]);
        }
    }
}

// dLoss/dSLM of pixel p from a caller-supplied SLM (psfs_backward_slm).
__device__ __forceinline__ float chain_rule_slm(const BackwardArgs &b, int64_t p, float acc)
{
    if (acc == 0.0f) return 0.0f;
    const float s_val = __ldg(b.slm + p);
    const float av = fmaf(b.da, s_val, b.one_minus_pd), bv = fmaf(b.db, s_val, b.one_minus_q);
    return acc * (div_fast(b.da, av) - div_fast(b.db, bv));
}

// One frame: pixel p sums b.dl over its segment in ascending voxel order.
__global__ void __launch_bounds__(256) owner_pixel_kernel(const __grid_constant__ BackwardArgs b, const uint32_t *off,
                                                          const uint32_t *vox)
{
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < b.n_pix; p += stride) {
        const uint32_t e0 = __ldg(off + p);
        uint32_t e1 = __ldg(off + p + 1);
#ifdef PSFS_BOUNDS_CHECK
        {   // the pixel's segment lies in the lists and names voxels of the grid
            const uint64_t n_vox = (uint64_t)b.f.nx * b.f.ny * b.f.nz;
            bool seg_ok = PSFS_IN_BOUNDS(e0 <= e1 && e1 <= __ldg(off + b.n_pix), b.f.status);
            for (uint32_t e = e0; seg_ok && e < e1; ++e) seg_ok = PSFS_IN_BOUNDS(__ldg(vox + e) < n_vox, b.f.status);
            if (!seg_ok) e1 = e0;
        }
#endif
        float acc = 0.0f;
        // four owners at a time: their index and dL loads are independent,
        // so they are in flight together; the adds stay in ascending order
        uint32_t e = e0;
        for (; e + 4 <= e1; e += 4) {
            const uint32_t v0 = __ldg(vox + e), v1 = __ldg(vox + e + 1), v2 = __ldg(vox + e + 2),
                           v3 = __ldg(vox + e + 3);
            const float d0 = __ldg(b.dl + v0), d1 = __ldg(b.dl + v1), d2 = __ldg(b.dl + v2), d3 = __ldg(b.dl + v3);
            acc += d0;
            acc += d1;
            acc += d2;
            acc += d3;
        }
        for (; e < e1; ++e) acc += __ldg(b.dl + __ldg(vox + e));
        float dslm, dm[3], dv[3];
        if (b.img) {
            float mu[3] = {0.0f, 0.0f, 0.0f}, hh[3] = {0.0f, 0.0f, 0.0f}, base = 0.0f;
            if (acc != 0.0f) {
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    mu[c] = __ldg(b.mean + 3 * p + c);
                    hh[c] = __ldg(b.hinv + 3 * p + c);
                }
                base = pixel_log_base(hh[0], hh[1], hh[2], b.c0);
            }
            chain_rule_pre(b, b.img + 3 * p, mu, hh, base, acc, dslm, dm, dv);
        } else {
            dslm = chain_rule_slm(b, p, acc);
#pragma unroll
            for (int c = 0; c < 3; ++c) dm[c] = dv[c] = 0.0f;
        }
        if (b.d_slm) b.d_slm[p] = dslm;
        if (b.d_mean)
            for (int c = 0; c < 3; ++c) b.d_mean[3 * p + c] = dm[c];
        if (b.d_var)
            for (int c = 0; c < 3; ++c) b.d_var[3 * p + c] = dv[c];
    }
}

// One voxel's 32-byte record of dLoss/dL (kBwRecord frames) with one 256-bit
// read-only load.
__device__ __forceinline__ void load_record(const float *rec, uint32_t (&w)[8])
{
    asm("ld.global.nc.L1::no_allocate.v8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
        : "=r"(w[0]), "=r"(w[1]), "=r"(w[2]), "=r"(w[3]), "=r"(w[4]), "=r"(w[5]), "=r"(w[6]), "=r"(w[7])
        : "l"(rec));
}

// Adds K consecutive owners (vox[e .. e + K)) of R record planes: their
// loads are issued together, then added in ascending owner order per frame.
template <int R, int K>
__device__ __forceinline__ void add_owners(const float *dl, size_t plane, const uint32_t *vox, uint32_t e,
                                           float (&acc)[R * kBwRecord])
{
    uint32_t v[K];
#pragma unroll
    for (int k = 0; k < K; ++k) v[k] = __ldg(vox + e + k);
    uint32_t w[K][R][8];
#pragma unroll
    for (int k = 0; k < K; ++k)
#pragma unroll
        for (int r = 0; r < R; ++r) load_record(dl + r * plane + (size_t)v[k] * kBwRecord, w[k][r]);
#pragma unroll
    for (int k = 0; k < K; ++k)
#pragma unroll
        for (int r = 0; r < R; ++r)
#pragma unroll
            for (int f = 0; f < kBwRecord; ++f) acc[r * kBwRecord + f] += __uint_as_float(w[k][r][f]);
}

// Up to R * kBwRecord frames: b.dl holds R planes of records of kBwRecord
// floats per voxel (frame r * kBwRecord + f of voxel v at b.dl[r * n_vox *
// kBwRecord + v * kBwRecord + f]); one 32-byte load per owned voxel and
// plane serves its frames, so the owner list, the background and d_mean /
// d_var are read once per R * kBwRecord frames.  Per frame the sum (same
// voxels, same order) and the chain rule are those of owner_pixel_kernel, so
// d_slm (frame f at b.d_slm + f n_pix) is bit-identical to one frame per
// call; d_mean and d_var receive the frames' gradients added in frame order
// to 0 (or, with `accumulate`, to what they hold).
template <int R>
__global__ void __launch_bounds__(256) owner_pixel_group_kernel(const __grid_constant__ BackwardArgs b,
                                                                const uint32_t *off, const uint32_t *vox,
                                                                int n_frames, int64_t img_fstride, int accumulate)
{
    constexpr int kF = R * kBwRecord;
    const size_t plane = (size_t)b.f.nx * b.f.ny * b.f.nz * kBwRecord;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < b.n_pix; p += stride) {
        const uint32_t e0 = __ldg(off + p);
        uint32_t e1 = __ldg(off + p + 1);
#ifdef PSFS_BOUNDS_CHECK
        {   // the pixel's segment lies in the lists and names voxels of the grid
            const uint64_t n_vox = (uint64_t)b.f.nx * b.f.ny * b.f.nz;
            bool seg_ok = PSFS_IN_BOUNDS(e0 <= e1 && e1 <= __ldg(off + b.n_pix), b.f.status);
            for (uint32_t e = e0; seg_ok && e < e1; ++e) seg_ok = PSFS_IN_BOUNDS(__ldg(vox + e) < n_vox, b.f.status);
            if (!seg_ok) e1 = e0;
        }
#endif
        float acc[kF];
#pragma unroll
        for (int f = 0; f < kF; ++f) acc[f] = 0.0f;
        // four record loads in flight (four owners of one plane, two of two
        // planes), then the rest two and one at a time
        uint32_t e = e0;
        if constexpr (R == 1) {
            for (; e + 4 <= e1; e += 4) add_owners<R, 4>(b.dl, plane, vox, e, acc);
        }
        for (; e + 2 <= e1; e += 2) add_owners<R, 2>(b.dl, plane, vox, e, acc);
        if (e < e1) add_owners<R, 1>(b.dl, plane, vox, e, acc);
        float tm[3] = {0.0f, 0.0f, 0.0f}, tv[3] = {0.0f, 0.0f, 0.0f};
        if (accumulate) {
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                if (b.d_mean) tm[c] = b.d_mean[3 * p + c];
                if (b.d_var) tv[c] = b.d_var[3 * p + c];
            }
        }
        bool any = false;
#pragma unroll
        for (int f = 0; f < kF; ++f) any |= (f < n_frames) & (acc[f] != 0.0f);
        float mu[3] = {0.0f, 0.0f, 0.0f}, hh[3] = {0.0f, 0.0f, 0.0f}, base = 0.0f;
        if (any) {
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                mu[c] = __ldg(b.mean + 3 * p + c);
                hh[c] = __ldg(b.hinv + 3 * p + c);
            }
            base = pixel_log_base(hh[0], hh[1], hh[2], b.c0);
        }
#pragma unroll
        for (int f = 0; f < kF; ++f) {
            if (f < n_frames) {
                float dslm, dm[3], dv[3];
                chain_rule_pre(b, b.img + f * img_fstride + 3 * p, mu, hh, base, acc[f], dslm, dm, dv);
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

// dLoss/dL = d_occ occ (1 - occ) from the forward's own occupancy (the
// expression of the voxel passes, so the same bits as their recomputation):
// n_frames frames of n_vox voxels, frame f's value into slot f of each
// voxel's 8-slot record (slots n_frames .. 7 set to 0; the whole 32-byte
// record in one vector store), or densely (dl_stride 1, one frame).
__global__ void __launch_bounds__(256) dl_from_occ_kernel(const float *occ, const float *d_occ, float *dl,
                                                          int64_t n_vox, int n_frames, int dl_stride)
{
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n_vox; v += stride) {
        if (dl_stride == kBwRecord) {
            float r[kBwRecord];
#pragma unroll
            for (int f = 0; f < kBwRecord; ++f) {
                r[f] = 0.0f;
                if (f < n_frames) {
                    const float o = __ldg(occ + f * n_vox + v);
                    r[f] = __ldg(d_occ + f * n_vox + v) * o * (1.0f - o);
                }
            }
            float4 *rec = reinterpret_cast<float4 *>(dl + v * kBwRecord);
            rec[0] = make_float4(r[0], r[1], r[2], r[3]);
            rec[1] = make_float4(r[4], r[5], r[6], r[7]);
        } else {
            for (int f = 0; f < n_frames; ++f) {
                const float o = __ldg(occ + f * n_vox + v);
                dl[v * dl_stride + f] = __ldg(d_occ + f * n_vox + v) * o * (1.0f - o);
            }
        }
    }
}

int64_t grid_for(int64_t n, int per_sm = 8)
{
    int64_t blocks = (n + 255) / 256;
    const int64_t cap = (int64_t)per_sm * device_sm_count();
    if (blocks > cap) blocks = cap;
    return blocks < 1 ? 1 : blocks;
}

}  // namespace

bool owner_lists_supported(const FuseArgs &a, int64_t n_pix)
{
    const uint64_t pairs = (uint64_t)a.nx * a.ny * a.nz * (uint64_t)a.n_cams;
    const int64_t n_chunks = (n_pix + 1 + kScanChunk - 1) / kScanChunk;
    return pairs < (1ull << 32) && n_chunks <= (int64_t)kScanThreads * kScanTopItems;
}

cudaError_t launch_build_owners(const FuseArgs &a, int64_t n_pix, uint32_t *cnt, uint32_t *sums, uint32_t *off,
                                uint32_t *vox, cudaStream_t s)
{
    if (!owner_lists_supported(a, n_pix)) return cudaErrorInvalidValue;
    const uint64_t n_vox = (uint64_t)a.nx * a.ny * a.nz;
    const int64_t vox_blocks = grid_for((int64_t)n_vox, 16);
    cudaError_t e = cudaMemsetAsync(cnt, 0, (size_t)n_pix * sizeof(uint32_t), s);
    if (e != cudaSuccess) return e;
    owner_count_kernel<<<(int)vox_blocks, 256, 0, s>>>(a, cnt);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    // offsets: n_pix + 1 entries, the last one the total
    const int64_t n_chunks = (n_pix + 1 + kScanChunk - 1) / kScanChunk;
    scan_chunks_kernel<<<(int)n_chunks, kScanThreads, 0, s>>>(cnt, n_pix, off, n_pix + 1, sums);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    scan_top_kernel<<<1, kScanThreads, 0, s>>>(sums, n_chunks);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    scan_add_kernel<<<(int)grid_for(n_pix + 1), 256, 0, s>>>(off, n_pix + 1, sums);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    e = cudaMemsetAsync(cnt, 0, (size_t)n_pix * sizeof(uint32_t), s);
    if (e != cudaSuccess) return e;
    owner_fill_kernel<<<(int)vox_blocks, 256, 0, s>>>(a, off, cnt, vox);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    owner_sort_kernel<<<(int)grid_for(n_pix), 256, 0, s>>>(off, vox, n_pix);
    return cudaGetLastError();
}

cudaError_t launch_dl_from_occ(const float *occ, const float *d_occ, float *dl, int64_t n_vox, int n_frames,
                               int dl_stride, cudaStream_t s)
{
    if (n_frames < 1 || n_frames > dl_stride) return cudaErrorInvalidValue;
    if (dl_stride == kBwRecord && ((uintptr_t)dl & 31u)) return cudaErrorMisalignedAddress;
    dl_from_occ_kernel<<<(int)grid_for(n_vox), 256, 0, s>>>(occ, d_occ, dl, n_vox, n_frames, dl_stride);
    return cudaGetLastError();
}

cudaError_t launch_owner_pixel(const BackwardArgs &b, const uint32_t *off, const uint32_t *vox, cudaStream_t s)
{
    owner_pixel_kernel<<<(int)grid_for(b.n_pix), 256, 0, s>>>(b, off, vox);
    return cudaGetLastError();
}

cudaError_t launch_owner_pixel_group(const BackwardArgs &b, const uint32_t *off, const uint32_t *vox, int n_frames,
                                     int64_t img_fstride, bool accumulate, cudaStream_t s)
{
    if (n_frames < 1 || n_frames > 2 * kBwRecord || !b.img || ((uintptr_t)b.dl & 31u))
        return cudaErrorInvalidValue;
    if (n_frames > kBwRecord)
        owner_pixel_group_kernel<2><<<(int)grid_for(b.n_pix), 256, 0, s>>>(b, off, vox, n_frames, img_fstride,
                                                                             accumulate ? 1 : 0);
    else
        owner_pixel_group_kernel<1><<<(int)grid_for(b.n_pix), 256, 0, s>>>(b, off, vox, n_frames, img_fstride,
                                                                             accumulate ? 1 : 0);
    return cudaGetLastError();
}

}  // namespace psfs
