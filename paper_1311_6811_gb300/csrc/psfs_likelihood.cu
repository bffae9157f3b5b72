// psfs_likelihood.cu -- per-pixel stage of the reconstruction (Eq. 1-2 and
// the per-camera log ratio of Eq. 5-9), plus the background packing kernel.
//
// Streaming, HBM-bound: per pixel 3 B of image + 24 B of packed background in,
// 4 B (f32) or 2 B (f16/bf16) of map out.  A persistent grid (four CTAs per
// SM) walks 512-pixel chunks; one thread per CTA streams each chunk's image
// bytes, means and inverse variances into shared memory with bulk copies
// (TMA) through a four-stage mbarrier ring, so that up to 220 KB per SM are
// in flight independently of registers, while all threads compute from the
// previous stages and write the map with coalesced stores.
#include <algorithm>

#include "psfs_internal.cuh"

namespace psfs {

namespace {

template <typename OutT>
__device__ __forceinline__ void store1(OutT *out, int64_t p, float a);
template <>
__device__ __forceinline__ void store1<float>(float *out, int64_t p, float a) { out[p] = a; }
template <>
__device__ __forceinline__ void store1<__half>(__half *out, int64_t p, float a) { out[p] = __float2half_rn(a); }
template <>
__device__ __forceinline__ void store1<__nv_bfloat16>(__nv_bfloat16 *out, int64_t p, float a)
{
    out[p] = __float2bfloat16_rn(a);
}

constexpr int kLkChunk = 512;                       // pixels per chunk (multiple of 16)
constexpr int kLkImgBytes = 3 * kLkChunk;             // 1536
constexpr int kLkBgBytes = 12 * kLkChunk;             // 6144 (3 floats per pixel)
constexpr int kLkStageBytes = kLkImgBytes + 2 * kLkBgBytes;
constexpr int kLkCtasPerSm = 4;                     // at most 4 x 55 KB of shared memory per SM
// Two shapes: 256 threads with a 4-stage ring (2 to 4 CTAs per SM), or one
// CTA per SM of 512 threads with a 6-stage ring (83 KB in flight), which
// leaves most of the SM to fusion CTAs of another frame on the sequence path.
template <int kStages>
constexpr int lk_smem_bytes() { return kStages * kLkStageBytes + kStages * 8; }

template <typename OutT, bool kSlm>
__device__ __forceinline__ void likelihood_pixel(const LikelihoodArgs &a, OutT *out, int64_t p, float i0,
                                                 float i1, float i2, const float *m, const float *h)
{
    const float r = pixel_log_odds(i0, i1, i2, m[0], m[1], m[2], h[0], h[1], h[2], a.c0);
    store1<OutT>(out, p, kSlm ? sigmoid_fast(r) : log_ratio_of_r(r, a.sc));
}

// n_tma_pix = n_pix rounded down to 16 pixels (48 image bytes), so every
// bulk copy has a size and offsets that are multiples of 16 bytes; the last
// < 16 pixels are read with plain loads by CTA 0.
template <typename OutT, bool kSlm, int kLkThreads, int kLkStages>
__global__ void __launch_bounds__(kLkThreads) likelihood_kernel(const LikelihoodArgs a, int64_t n_tma_pix)
{
    extern __shared__ __align__(128) unsigned char smem[];
    uint64_t *bars = reinterpret_cast<uint64_t *>(smem + kLkStages * kLkStageBytes);
    OutT *out = reinterpret_cast<OutT *>(a.out);
    const int tid = threadIdx.x;
    if (a.zero_word && blockIdx.x == 0 && tid == 0) *a.zero_word = 0u;
    if (tid == 0) {
        for (int s = 0; s < kLkStages; ++s) mbar_init(&bars[s], 1);
        mbar_fence_init();
    }
    __syncthreads();

    const int64_t n_chunks = (n_tma_pix + kLkChunk - 1) / kLkChunk;
    const int64_t my_chunks =
        (int64_t)blockIdx.x < n_chunks ? (n_chunks - 1 - blockIdx.x) / gridDim.x + 1 : 0;
    auto stage_img = [&](int s) { return smem + s * kLkStageBytes; };
    auto stage_mean = [&](int s) { return reinterpret_cast<float *>(smem + s * kLkStageBytes + kLkImgBytes); };
    auto stage_hinv = [&](int s) {
        return reinterpret_cast<float *>(smem + s * kLkStageBytes + kLkImgBytes + kLkBgBytes);
    };
    auto issue = [&](int64_t k) {
        const int s = (int)(k % kLkStages);
        const int64_t p0 = ((int64_t)blockIdx.x + k * gridDim.x) * kLkChunk;
        const uint32_t np = (uint32_t)min((int64_t)kLkChunk, n_tma_pix - p0);
        mbar_arrive_expect_tx(&bars[s], 27u * np);
        bulk_g2s(stage_img(s), a.img + 3 * p0, 3u * np, &bars[s]);
        bulk_g2s(stage_mean(s), a.mean + 3 * p0, 12u * np, &bars[s]);
        bulk_g2s(stage_hinv(s), a.hinv + 3 * p0, 12u * np, &bars[s]);
    };
    if (tid == 0)
        for (int64_t k = 0; k < my_chunks && k < kLkStages; ++k) issue(k);

    for (int64_t k = 0; k < my_chunks; ++k) {
        const int s = (int)(k % kLkStages);
        mbar_wait_bounded(&bars[s], (uint32_t)((k / kLkStages) & 1), a.status);
        const int64_t p0 = ((int64_t)blockIdx.x + k * gridDim.x) * kLkChunk;
        const int np = (int)min((int64_t)kLkChunk, n_tma_pix - p0);
        const unsigned char *im = stage_img(s);
        const float *mu = stage_mean(s);
        const float *hv = stage_hinv(s);
        for (int q = tid; q < np; q += kLkThreads)
            likelihood_pixel<OutT, kSlm>(a, out, p0 + q, (float)im[3 * q], (float)im[3 * q + 1],
                                         (float)im[3 * q + 2], mu + 3 * q, hv + 3 * q);
        __syncthreads();   // every thread is done with stage s before it is refilled
        if (tid == 0 && k + kLkStages < my_chunks) issue(k + kLkStages);
    }

    if (blockIdx.x == 0) {
        for (int64_t p = n_tma_pix + tid; p < a.n_pix; p += kLkThreads) {
            const uint8_t *im = a.img + 3 * p;
            likelihood_pixel<OutT, kSlm>(a, out, p, (float)im[0], (float)im[1], (float)im[2], a.mean + 3 * p,
                                         a.hinv + 3 * p);
        }
    }
}

// s -> g(s) = log(a(s) / b(s)) for caller-supplied SLM maps (Eq. 5-9).
template <typename OutT>
__global__ void __launch_bounds__(256) slm_to_map_kernel(const SlmToMapArgs a)
{
    if (a.zero_word && blockIdx.x == 0 && threadIdx.x == 0) *a.zero_word = 0u;
    OutT *out = reinterpret_cast<OutT *>(a.out);
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < a.n_pix; p += stride) {
        float s = __ldg(a.slm + p);
        float av = fmaf(a.da, s, a.one_minus_pd);
        float bv = fmaf(a.db, s, a.one_minus_q);
        store1<OutT>(out, p, logf(av) - logf(bv));
    }
}

// Copies the mean, stores h = 1 / (2 var), counts invalid entries.
__global__ void __launch_bounds__(256) pack_background_kernel(const float *mean, const float *var,
                                                              int64_t n, float *mean_out,
                                                              float *hinv_out, uint32_t *bad)
{
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    uint32_t nbad = 0;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += stride) {
        float m = mean[e], v = var[e];
        bool ok = isfinite(m) && isfinite(v) && v >= 1e-6f && v <= 1e12f;
        mean_out[e] = m;
        hinv_out[e] = ok ? 0.5f / v : 0.0f;
        nbad += ok ? 0u : 1u;
    }
    if (nbad) atomicAdd(bad, nbad);
}

int grid_for(int64_t work, int threads)
{
    int64_t blocks = (work + threads - 1) / threads;
    int64_t cap = (int64_t)device_sm_count() * 8;
    if (blocks > cap) blocks = cap;
    if (blocks < 1) blocks = 1;
    return (int)blocks;
}

template <typename OutT, bool kSlm, int kThreads, int kStages>
cudaError_t launch_likelihood_shape(const LikelihoodArgs &a, cudaStream_t s, int ctas_per_sm)
{
    auto kern = likelihood_kernel<OutT, kSlm, kThreads, kStages>;
    constexpr int smem = lk_smem_bytes<kStages>();
    static bool configured[64] = {false};
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev >= 0 && dev < 64 && !configured[dev]) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        if (e != cudaSuccess) return e;
        configured[dev] = true;
    }
    const int64_t n_tma_pix = a.n_pix / 16 * 16;
    const int64_t n_chunks = (n_tma_pix + kLkChunk - 1) / kLkChunk;
    int64_t blocks = std::min<int64_t>(n_chunks, ctas_per_sm * (int64_t)device_sm_count());
    if (blocks < 1) blocks = 1;
    kern<<<(int)blocks, kThreads, smem, s>>>(a, n_tma_pix);
    return cudaGetLastError();
}

template <typename OutT, bool kSlm>
cudaError_t launch_likelihood_typed(const LikelihoodArgs &a, cudaStream_t s, int ctas_per_sm)
{
    // bulk copies need 16-byte aligned sources: refuse rather than fault
    if (((uintptr_t)a.img | (uintptr_t)a.mean | (uintptr_t)a.hinv) & 15u) return cudaErrorMisalignedAddress;
    ctas_per_sm = std::max(1, std::min(ctas_per_sm, kLkCtasPerSm));
    if (ctas_per_sm == 1) return launch_likelihood_shape<OutT, kSlm, 512, 6>(a, s, 1);
    return launch_likelihood_shape<OutT, kSlm, 256, 4>(a, s, ctas_per_sm);
}

}  // namespace

cudaError_t launch_pack_background(const float *mean, const float *var, int64_t n_pix,
                                   float *mean_out, float *hinv_out, uint32_t *bad, cudaStream_t s)
{
    const int64_t n = 3 * n_pix;
    pack_background_kernel<<<grid_for(n, 256), 256, 0, s>>>(mean, var, n, mean_out, hinv_out, bad);
    return cudaGetLastError();
}

cudaError_t launch_likelihood(const LikelihoodArgs &a, int map_dtype, bool slm_out, cudaStream_t s,
                              int ctas_per_sm)
{
    if (slm_out) return launch_likelihood_typed<float, true>(a, s, ctas_per_sm);
    if (map_dtype == PSFS_MAP_F16) return launch_likelihood_typed<__half, false>(a, s, ctas_per_sm);
    if (map_dtype == PSFS_MAP_BF16) return launch_likelihood_typed<__nv_bfloat16, false>(a, s, ctas_per_sm);
    return launch_likelihood_typed<float, false>(a, s, ctas_per_sm);
}

cudaError_t launch_slm_to_map(const SlmToMapArgs &a, int map_dtype, cudaStream_t s)
{
    const int blocks = grid_for(a.n_pix, 256);
    if (map_dtype == PSFS_MAP_F16) {
        slm_to_map_kernel<__half><<<blocks, 256, 0, s>>>(a);
    } else if (map_dtype == PSFS_MAP_BF16) {
        slm_to_map_kernel<__nv_bfloat16><<<blocks, 256, 0, s>>>(a);
    } else {
        slm_to_map_kernel<float><<<blocks, 256, 0, s>>>(a);
    }
    return cudaGetLastError();
}

}  // namespace psfs
