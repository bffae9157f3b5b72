// psfs_likelihood.cu -- per-pixel stage of the reconstruction (Eq. 1-2 and
// the per-camera log ratio of Eq. 5-9), plus the background packing kernel.
//
// Streaming, HBM-bound: per pixel 3 B of image + 24 B of packed background in,
// 4 B (f32) or 2 B (f16/bf16) of map out.  One thread handles 4 consecutive
// pixels: 12 image bytes as three 32-bit loads, 12 means and 12 inverse
// variances as three 128-bit loads each, and one 128-bit (or 64-bit) store.
#include "psfs_internal.cuh"

namespace psfs {

namespace {

int sm_count()
{
    static int cached[64] = {0};
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 0 || dev >= 64) return 152;
    if (!cached[dev]) {
        int n = 0;
        cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
        cached[dev] = n > 0 ? n : 152;
    }
    return cached[dev];
}

// Exact float of byte `sel` of w: build the bit pattern 0x4B0000bb (2^23 + b)
// with one byte permute, then subtract 2^23.
__device__ __forceinline__ float byte_to_float(uint32_t w, uint32_t sel)
{
    return __uint_as_float(__byte_perm(w, 0x4B000000u, sel)) - 8388608.0f;
}

// r = log U - log N (Eq. 1) for one pixel, from its colour, mean and
// h = 1 / (2 var):  r = c0 - 0.5 log(h0 h1 h2) + sum_c (I_c - mu_c)^2 h_c.
__device__ __forceinline__ float pixel_log_odds(float i0, float i1, float i2, float m0, float m1,
                                                float m2, float h0, float h1, float h2, float c0)
{
    float d0 = i0 - m0, d1 = i1 - m1, d2 = i2 - m2;
    float quad = fmaf(d0 * d0, h0, fmaf(d1 * d1, h1, d2 * d2 * h2));
    return (c0 - 0.5f * logf(h0 * h1 * h2)) + quad;
}

__device__ __forceinline__ float sigmoid(float r)
{
    if (r > 0.0f) return 1.0f / (1.0f + expf(-r));
    float e = expf(r);
    return e / (1.0f + e);
}

template <typename OutT>
__device__ __forceinline__ void store4(OutT *out, int64_t q, float a, float b, float c, float d);

template <>
__device__ __forceinline__ void store4<float>(float *out, int64_t q, float a, float b, float c, float d)
{
    reinterpret_cast<float4 *>(out)[q] = make_float4(a, b, c, d);
}

template <>
__device__ __forceinline__ void store4<__half>(__half *out, int64_t q, float a, float b, float c, float d)
{
    __half2 lo = __floats2half2_rn(a, b), hi = __floats2half2_rn(c, d);
    uint2 v;
    v.x = *reinterpret_cast<uint32_t *>(&lo);
    v.y = *reinterpret_cast<uint32_t *>(&hi);
    reinterpret_cast<uint2 *>(out)[q] = v;
}

template <>
__device__ __forceinline__ void store4<__nv_bfloat16>(__nv_bfloat16 *out, int64_t q, float a, float b,
                                                      float c, float d)
{
    __nv_bfloat162 lo = __floats2bfloat162_rn(a, b), hi = __floats2bfloat162_rn(c, d);
    uint2 v;
    v.x = *reinterpret_cast<uint32_t *>(&lo);
    v.y = *reinterpret_cast<uint32_t *>(&hi);
    reinterpret_cast<uint2 *>(out)[q] = v;
}

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

template <typename OutT, bool kSlm>
__global__ void __launch_bounds__(256) likelihood_kernel(const LikelihoodArgs a)
{
    if (a.zero_word && blockIdx.x == 0 && threadIdx.x == 0) *a.zero_word = 0u;
    OutT *out = reinterpret_cast<OutT *>(a.out);
    const int64_t n_quads = a.n_pix >> 2;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const uint32_t *img = reinterpret_cast<const uint32_t *>(a.img);
    const float4 *mean = reinterpret_cast<const float4 *>(a.mean);
    const float4 *hinv = reinterpret_cast<const float4 *>(a.hinv);
    for (int64_t q = tid; q < n_quads; q += stride) {
        uint32_t w0 = __ldcs(img + 3 * q), w1 = __ldcs(img + 3 * q + 1), w2 = __ldcs(img + 3 * q + 2);
        float4 ma = __ldg(mean + 3 * q), mb = __ldg(mean + 3 * q + 1), mc = __ldg(mean + 3 * q + 2);
        float4 ha = __ldg(hinv + 3 * q), hb = __ldg(hinv + 3 * q + 1), hc = __ldg(hinv + 3 * q + 2);
        // channel c of pixel p sits at position 3 p + c of the 12 values
        float r0 = pixel_log_odds(byte_to_float(w0, 0x7440), byte_to_float(w0, 0x7441),
                                  byte_to_float(w0, 0x7442), ma.x, ma.y, ma.z, ha.x, ha.y, ha.z, a.c0);
        float r1 = pixel_log_odds(byte_to_float(w0, 0x7443), byte_to_float(w1, 0x7440),
                                  byte_to_float(w1, 0x7441), ma.w, mb.x, mb.y, ha.w, hb.x, hb.y, a.c0);
        float r2 = pixel_log_odds(byte_to_float(w1, 0x7442), byte_to_float(w1, 0x7443),
                                  byte_to_float(w2, 0x7440), mb.z, mb.w, mc.x, hb.z, hb.w, hc.x, a.c0);
        float r3 = pixel_log_odds(byte_to_float(w2, 0x7441), byte_to_float(w2, 0x7442),
                                  byte_to_float(w2, 0x7443), mc.y, mc.z, mc.w, hc.y, hc.z, hc.w, a.c0);
        if (kSlm) {
            store4<OutT>(out, q, sigmoid(r0), sigmoid(r1), sigmoid(r2), sigmoid(r3));
        } else {
            store4<OutT>(out, q, log_ratio_of_r(r0, a.sc), log_ratio_of_r(r1, a.sc),
                         log_ratio_of_r(r2, a.sc), log_ratio_of_r(r3, a.sc));
        }
    }
    // ragged tail (n_pix not a multiple of 4): scalar loads
    const int64_t rem = a.n_pix - 4 * n_quads;
    if (tid < rem) {
        const int64_t p = 4 * n_quads + tid;
        const float *m = a.mean + 3 * p, *hh = a.hinv + 3 * p;
        const uint8_t *im = a.img + 3 * p;
        float r = pixel_log_odds((float)im[0], (float)im[1], (float)im[2], m[0], m[1], m[2], hh[0],
                                 hh[1], hh[2], a.c0);
        store1<OutT>(out, p, kSlm ? sigmoid(r) : log_ratio_of_r(r, a.sc));
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
    int64_t cap = (int64_t)sm_count() * 8;
    if (blocks > cap) blocks = cap;
    if (blocks < 1) blocks = 1;
    return (int)blocks;
}

}  // namespace

cudaError_t launch_pack_background(const float *mean, const float *var, int64_t n_pix,
                                   float *mean_out, float *hinv_out, uint32_t *bad, cudaStream_t s)
{
    const int64_t n = 3 * n_pix;
    pack_background_kernel<<<grid_for(n, 256), 256, 0, s>>>(mean, var, n, mean_out, hinv_out, bad);
    return cudaGetLastError();
}

cudaError_t launch_likelihood(const LikelihoodArgs &a, int map_dtype, bool slm_out, cudaStream_t s)
{
    const int64_t work = (a.n_pix >> 2) > 0 ? (a.n_pix >> 2) : 1;
    const int blocks = grid_for(work, 256);
    if (slm_out) {
        likelihood_kernel<float, true><<<blocks, 256, 0, s>>>(a);
    } else if (map_dtype == PSFS_MAP_F16) {
        likelihood_kernel<__half, false><<<blocks, 256, 0, s>>>(a);
    } else if (map_dtype == PSFS_MAP_BF16) {
        likelihood_kernel<__nv_bfloat16, false><<<blocks, 256, 0, s>>>(a);
    } else {
        likelihood_kernel<float, false><<<blocks, 256, 0, s>>>(a);
    }
    return cudaGetLastError();
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
