// psfs_group.cu -- frame groups of the sequence path.
//
// The rig, grid and background are fixed across the frames of a sequence, so
// F consecutive frames can share the work that does not depend on the image:
//
//   * likelihood: one pass over the packed background (24 B per pixel, the
//     largest input) computes the log ratio g of Eq. 5-9 for all F frames of
//     the group.  The maps are written as pixel records of RB = 32 or 64 bytes
//     holding P frames (P = RB / element size, F when F is smaller):
//     [F / P planes][n_cams][H][W][P], one or two vector stores per pixel and
//     plane.
//   * fusion, one launch per plane: each voxel centre is projected into each
//     camera once (Eq. 3) and vector loads gather g of that pixel for the P
//     frames of the plane; every frame keeps its own log-odds accumulator,
//     output grid and list.  A 32-byte record is one sector per (voxel,
//     camera), and a plane of a 128^3 x 8 x 640 x 480 rig (79 MB) stays in
//     L2.  A 64-byte record is read by two lanes (one 32-byte half each) in
//     the same warp request: the L1 serves both sectors of the line in one
//     wavefront, so a plane costs half the wavefronts per frame, with planes
//     of twice the size.  Groups of more frames only add planes, so the
//     background pass is shared by more frames at the same fusion cost.
//
// Per frame and per pixel / voxel the arithmetic is exactly that of the
// single-frame kernels (the same helper functions, the same camera order of
// the sum), so each frame's occupancy, list and count are bit-identical to a
// single-frame reconstruction; the group only removes repeated background
// reads, projections and load instructions.
#include <algorithm>

#include "psfs_fuse_common.cuh"

namespace psfs {

namespace {

// ---------------------------------------------------------------------------
// F-wide map vectors
// ---------------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ T to_map(float g);
template <>
__device__ __forceinline__ float to_map<float>(float g) { return g; }
template <>
__device__ __forceinline__ __half to_map<__half>(float g) { return __float2half_rn(g); }
template <>
__device__ __forceinline__ __nv_bfloat16 to_map<__nv_bfloat16>(float g) { return __float2bfloat16_rn(g); }

template <typename T>
__device__ __forceinline__ uint32_t map_bits(T v);
template <>
__device__ __forceinline__ uint32_t map_bits<float>(float v) { return __float_as_uint(v); }
template <>
__device__ __forceinline__ uint32_t map_bits<__half>(__half v) { return __half_as_ushort(v); }
template <>
__device__ __forceinline__ uint32_t map_bits<__nv_bfloat16>(__nv_bfloat16 v) { return __bfloat16_as_ushort(v); }

template <typename T>
__device__ __forceinline__ float map_value(uint32_t bits);
template <>
__device__ __forceinline__ float map_value<float>(uint32_t bits) { return __uint_as_float(bits); }
template <>
__device__ __forceinline__ float map_value<__half>(uint32_t bits)
{
    return __half2float(__ushort_as_half((unsigned short)bits));
}
template <>
__device__ __forceinline__ float map_value<__nv_bfloat16>(uint32_t bits)
{
    return __bfloat162float(__ushort_as_bfloat16((unsigned short)bits));
}

// Packs F map values into 32-bit words (element e in the low half first for
// 16-bit types, the little-endian order of a [F] array).
template <typename T, int F>
struct GroupWords {
    static constexpr int kWords = (F * (int)sizeof(T) + 3) / 4;
    uint32_t w[kWords];

    __device__ __forceinline__ void set(int e, T v)
    {
        if (sizeof(T) == 4) {
            w[e] = map_bits<T>(v);
        } else {
            const uint32_t b = map_bits<T>(v) & 0xFFFFu;
            w[e >> 1] = (e & 1) ? (w[e >> 1] | (b << 16)) : b;
        }
    }
    __device__ __forceinline__ float get(int e) const
    {
        if (sizeof(T) == 4) return map_value<T>(w[e]);
        return map_value<T>((w[e >> 1] >> (16 * (e & 1))) & 0xFFFFu);
    }
};


// L += g for two 16-bit map values packed in one word (low half first), one
// mixed-precision add each (sm_100+): the 16-bit value is widened exactly
// and added in FP32 with one rounding, so the sum is that of converting
// first and adding, in one instruction instead of two.
template <typename T>
__device__ __forceinline__ void add_pair(uint32_t w, float &a, float &b);
template <>
__device__ __forceinline__ void add_pair<__half>(uint32_t w, float &a, float &b)
{
    asm("{\n .reg .f16 lo, hi;\n mov.b32 {lo, hi}, %2;\n add.rn.f32.f16 %0, lo, %0;\n add.rn.f32.f16 %1, hi, %1;\n}\n"
        : "+f"(a), "+f"(b) : "r"(w));
}
template <>
__device__ __forceinline__ void add_pair<__nv_bfloat16>(uint32_t w, float &a, float &b)
{
    asm("{\n .reg .b16 lo, hi;\n mov.b32 {lo, hi}, %2;\n add.rn.f32.bf16 %0, lo, %0;\n add.rn.f32.bf16 %1, hi, %1;\n}\n"
        : "+f"(a), "+f"(b) : "r"(w));
}

// L[f][t] += frame f's log ratio of one gathered record, for the F frames.
template <typename MapT, int F, int TZ>
__device__ __forceinline__ void add_words(const GroupWords<MapT, F> &g, float (&L)[F][TZ], int t)
{
    if constexpr (sizeof(MapT) == 4) {
#pragma unroll
        for (int f = 0; f < F; ++f) L[f][t] += g.get(f);
    } else {
        static_assert(F % 2 == 0, "16-bit records hold pairs of frames");
#pragma unroll
        for (int q = 0; q < F / 2; ++q) add_pair<MapT>(g.w[q], L[2 * q][t], L[2 * q + 1][t]);
    }
}

// Vector store / read-only vector load of the F * sizeof(T) bytes of one
// pixel (4, 8, 16 or 32 bytes; the address is a multiple of that size, the
// buffers are 256-byte aligned).
template <int kWords>
__device__ __forceinline__ void store_words(uint32_t *dst, const uint32_t *w)
{
    if constexpr (kWords % 8 == 0) {
#pragma unroll
        for (int q = 0; q < kWords; q += 8)
            asm volatile("st.global.v8.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8};" ::"l"(dst + q), "r"(w[q]),
                         "r"(w[q + 1]), "r"(w[q + 2]), "r"(w[q + 3]), "r"(w[q + 4]), "r"(w[q + 5]), "r"(w[q + 6]),
                         "r"(w[q + 7])
                         : "memory");
    } else if constexpr (kWords == 1) {
        *dst = w[0];
    } else if constexpr (kWords == 2) {
        *reinterpret_cast<uint2 *>(dst) = make_uint2(w[0], w[1]);
    } else {
        static_assert(kWords % 4 == 0, "group vector of 16-byte words");
#pragma unroll
        for (int q = 0; q < kWords; q += 4)
            *reinterpret_cast<uint4 *>(dst + q) = make_uint4(w[q], w[q + 1], w[q + 2], w[q + 3]);
    }
}

template <int kWords>
__device__ __forceinline__ void load_words(const uint32_t *src, uint32_t *w)
{
    if constexpr (kWords % 8 == 0) {
        // 256-bit read-only loads (sm_100+): each a whole 32-byte sector of
        // the lane's group vector in one request.  Lanes rarely share a
        // sector (about 13 % L1 hits), so the line is not kept in L1.
#pragma unroll
        for (int q = 0; q < kWords; q += 8)
            asm("ld.global.nc.L1::no_allocate.v8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
                : "=r"(w[q]), "=r"(w[q + 1]), "=r"(w[q + 2]), "=r"(w[q + 3]), "=r"(w[q + 4]), "=r"(w[q + 5]),
                  "=r"(w[q + 6]), "=r"(w[q + 7])
                : "l"(src + q));
    } else if constexpr (kWords == 1) {
        w[0] = __ldg(src);
    } else if constexpr (kWords == 2) {
        const uint2 v = __ldg(reinterpret_cast<const uint2 *>(src));
        w[0] = v.x;
        w[1] = v.y;
    } else {
        static_assert(kWords % 4 == 0, "group vector of 16-byte words");
#pragma unroll
        for (int q = 0; q < kWords; q += 4) {
            const uint4 v = __ldg(reinterpret_cast<const uint4 *>(src + q));
            w[q] = v.x;
            w[q + 1] = v.y;
            w[q + 2] = v.z;
            w[q + 3] = v.w;
        }
    }
}

// ---------------------------------------------------------------------------
// Likelihood of a frame group
// ---------------------------------------------------------------------------
constexpr int kGThreads = 256;
constexpr int kPairWarps = 8;   // warps of fuse_pair_kernel: 4 warps' voxel columns, two lanes per column
template <int F>
struct GLayout {
    static constexpr int kChunk = F >= 32 ? 256 : 512;              // pixels per chunk (multiple of 16)
    static constexpr int kImgBytes = 3 * kChunk;                    // one frame's colours
    static constexpr int kBgBytes = 12 * kChunk;                    // 3 floats per pixel
    static constexpr int kStages = F >= 32 ? 3 : (F >= 16 ? 2 : 4); // ring depth (16 frames: 74 KB, 32: 92 KB)
    static constexpr int kStage = F * kImgBytes + 2 * kBgBytes;     // bytes per ring stage
    static constexpr int kSmem = kStages * kStage + kStages * 8;    // + mbarriers
};

template <typename OutT, int F, int RB>
__device__ __forceinline__ void group_pixel(const LikelihoodArgs &a, OutT *out, int64_t p, const unsigned char *im,
                                            int64_t im_stride, const float *m, const float *h)
{
    const float m0 = m[0], m1 = m[1], m2 = m[2], h0 = h[0], h1 = h[1], h2 = h[2];
    const float base = pixel_log_base(h0, h1, h2, a.c0);   // r = base + quad, as pixel_log_odds
    // planes of RB-byte records (one plane [n_pix][F] when the F frames fit
    // one record): each plane's record is stored as soon as its frames are
    // formed, so only one record's words are live (a 32-frame group in one
    // record array held 80 registers per thread, which the fusion kernel
    // running beside it on the SM then lacked)
    constexpr int kP = RB / (int)sizeof(OutT);
    constexpr int kPlane = F < kP ? F : kP;
    constexpr int kWords = GroupWords<OutT, kPlane>::kWords;
#pragma unroll
    for (int q = 0; q < F / kPlane; ++q) {
        GroupWords<OutT, kPlane> pk;
#pragma unroll
        for (int e = 0; e < kPlane; ++e) {
            const unsigned char *px = im + (q * kPlane + e) * im_stride;
            const float r = base + pixel_quad((float)px[0], (float)px[1], (float)px[2], m0, m1, m2, h0, h1, h2);
            pk.set(e, to_map<OutT>(log_ratio_of_r(r, a.sc)));
        }
        store_words<kWords>(reinterpret_cast<uint32_t *>(out + ((int64_t)q * a.n_pix + p) * kPlane), pk.w);
    }
}

// Persistent grid over 512-pixel chunks (256 for 32 frames); one thread per CTA streams each
// chunk's F image slices, means and inverse variances into shared memory
// with bulk copies through a 4-stage mbarrier ring.  n_tma_pix = n_pix
// rounded down to 16 pixels; CTA 0 computes the last < 16 pixels with plain
// loads.
template <typename OutT, int F, int RB>
__global__ void __launch_bounds__(kGThreads) likelihood_group_kernel(const LikelihoodArgs a, int64_t n_tma_pix)
{
    extern __shared__ __align__(128) unsigned char smem[];
    uint64_t *bars = reinterpret_cast<uint64_t *>(smem + GLayout<F>::kStages * GLayout<F>::kStage);
    OutT *out = reinterpret_cast<OutT *>(a.out);
    const int tid = threadIdx.x;
    if (a.zero_word && blockIdx.x == 0 && tid < F) a.zero_word[(int64_t)tid * a.zero_fstride] = 0u;
    if (tid == 0) {
        for (int s = 0; s < GLayout<F>::kStages; ++s) mbar_init(&bars[s], 1);
        mbar_fence_init();
    }
    __syncthreads();

    const int64_t n_chunks = (n_tma_pix + GLayout<F>::kChunk - 1) / GLayout<F>::kChunk;
    const int64_t my_chunks =
        (int64_t)blockIdx.x < n_chunks ? (n_chunks - 1 - blockIdx.x) / gridDim.x + 1 : 0;
    auto stage_img = [&](int s) { return smem + s * GLayout<F>::kStage; };
    auto stage_mean = [&](int s) {
        return reinterpret_cast<float *>(smem + s * GLayout<F>::kStage + F * GLayout<F>::kImgBytes);
    };
    auto stage_hinv = [&](int s) {
        return reinterpret_cast<float *>(smem + s * GLayout<F>::kStage + F * GLayout<F>::kImgBytes + GLayout<F>::kBgBytes);
    };
    auto issue = [&](int64_t k) {
        const int s = (int)(k % GLayout<F>::kStages);
        const int64_t p0 = ((int64_t)blockIdx.x + k * gridDim.x) * GLayout<F>::kChunk;
        const uint32_t np = (uint32_t)min((int64_t)GLayout<F>::kChunk, n_tma_pix - p0);
        mbar_arrive_expect_tx(&bars[s], (3u * F + 24u) * np);
#pragma unroll
        for (int f = 0; f < F; ++f)
            bulk_g2s(stage_img(s) + f * GLayout<F>::kImgBytes, a.img + f * a.img_fstride + 3 * p0, 3u * np, &bars[s]);
        bulk_g2s(stage_mean(s), a.mean + 3 * p0, 12u * np, &bars[s]);
        bulk_g2s(stage_hinv(s), a.hinv + 3 * p0, 12u * np, &bars[s]);
    };
    if (tid == 0)
        for (int64_t k = 0; k < my_chunks && k < GLayout<F>::kStages; ++k) issue(k);

    for (int64_t k = 0; k < my_chunks; ++k) {
        const int s = (int)(k % GLayout<F>::kStages);
        mbar_wait_bounded(&bars[s], (uint32_t)((k / GLayout<F>::kStages) & 1), a.status);
        const int64_t p0 = ((int64_t)blockIdx.x + k * gridDim.x) * GLayout<F>::kChunk;
        const int np = (int)min((int64_t)GLayout<F>::kChunk, n_tma_pix - p0);
        const unsigned char *im = stage_img(s);
        const float *mu = stage_mean(s);
        const float *hv = stage_hinv(s);
        for (int q = tid; q < np; q += kGThreads)
            group_pixel<OutT, F, RB>(a, out, p0 + q, im + 3 * q, GLayout<F>::kImgBytes, mu + 3 * q, hv + 3 * q);
        __syncthreads();   // every thread is done with stage s before it is refilled
        if (tid == 0 && k + GLayout<F>::kStages < my_chunks) issue(k + GLayout<F>::kStages);
    }

    if (blockIdx.x == 0) {
        for (int64_t p = n_tma_pix + tid; p < a.n_pix; p += kGThreads)
            group_pixel<OutT, F, RB>(a, out, p, a.img + 3 * p, a.img_fstride, a.mean + 3 * p, a.hinv + 3 * p);
    }
}

template <typename OutT, int F, int RB>
cudaError_t launch_lk_group(const LikelihoodArgs &a, cudaStream_t s, int ctas_per_sm)
{
    auto kern = likelihood_group_kernel<OutT, F, RB>;
    constexpr int smem = GLayout<F>::kSmem;
    static bool configured[64] = {false};
    static int max_ctas[64] = {0};
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    if (!configured[dev]) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        if (e != cudaSuccess) return e;
        int n = 0;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, kern, kGThreads, smem);
        if (e != cudaSuccess) return e;
        max_ctas[dev] = std::max(1, n);
        configured[dev] = true;
    }
    const int per_sm = std::max(1, std::min(ctas_per_sm, max_ctas[dev]));
    const int64_t n_tma_pix = a.n_pix / 16 * 16;
    const int64_t n_chunks = (n_tma_pix + GLayout<F>::kChunk - 1) / GLayout<F>::kChunk;
    int64_t blocks = std::min<int64_t>(n_chunks, (int64_t)per_sm * device_sm_count());
    if (blocks < 1) blocks = 1;
    kern<<<(int)blocks, kGThreads, smem, s>>>(a, n_tma_pix);
    return cudaGetLastError();
}

template <typename OutT>
cudaError_t launch_lk_group_typed(const LikelihoodArgs &a, int frames, cudaStream_t s, int ctas_per_sm, int rec)
{
    // bulk copies need 16-byte aligned sources and sizes: refuse rather than fault
    if (((uintptr_t)a.img | (uintptr_t)a.mean | (uintptr_t)a.hinv | (uintptr_t)a.img_fstride) & 15u)
        return cudaErrorMisalignedAddress;
    if (((uintptr_t)a.out) & (uintptr_t)(frames * sizeof(OutT) - 1)) return cudaErrorMisalignedAddress;
    if (rec != 32 && rec != 64) return cudaErrorInvalidValue;
    // the record size only matters once the F frames fill more than 32 bytes
    const bool wide = rec == 64 && frames * (int)sizeof(OutT) > 32;
    if (frames == 2) return launch_lk_group<OutT, 2, 32>(a, s, ctas_per_sm);
    if (frames == 4) return launch_lk_group<OutT, 4, 32>(a, s, ctas_per_sm);
    if (frames == 8) return launch_lk_group<OutT, 8, 32>(a, s, ctas_per_sm);
    if (frames == 16)
        return wide ? launch_lk_group<OutT, 16, 64>(a, s, ctas_per_sm) : launch_lk_group<OutT, 16, 32>(a, s, ctas_per_sm);
    if (frames == 32)
        return wide ? launch_lk_group<OutT, 32, 64>(a, s, ctas_per_sm) : launch_lk_group<OutT, 32, 32>(a, s, ctas_per_sm);
    return cudaErrorInvalidValue;
}

// ---------------------------------------------------------------------------
// Fusion of a frame group
// ---------------------------------------------------------------------------
// Epilogue of a frame group: per frame the posterior, threshold and
// compaction of tile_epilogue (the same per-voxel arithmetic), with the F
// frames' counts taken together: two barriers per tile, and F threads each
// reserve one frame's list range with one atomicAdd.
template <int WY, int TZ, int F>
__device__ __forceinline__ void group_epilogue(const FuseArgs &a, int i, int j, int k0, const float (&L)[F][TZ],
                                               int lane, int wy, uint32_t (*s_off)[WY], uint32_t *s_base)
{
    const bool in_xy = (i < a.nx) && (j < a.ny);
    const uint32_t zstride = (uint32_t)a.nx * (uint32_t)a.ny;
    const uint32_t lin0 = (uint32_t)i + (uint32_t)a.nx * ((uint32_t)j + (uint32_t)a.ny * (uint32_t)k0);
#pragma unroll
    for (int f = 0; f < F; ++f) {
        float *occ = a.occ + f * a.occ_fstride;
        uint32_t cnt = 0;
#pragma unroll
        for (int t = 0; t < TZ; ++t) {
            const bool valid = in_xy && (k0 + t < a.nz);
            const float lo = L[f][t] + a.logit_prior;
            if (valid) __stcs(occ + lin0 + (uint32_t)t * zstride, posterior_of_logodds(lo));
            cnt += __popc(__ballot_sync(0xFFFFFFFFu, valid && (lo > a.logit_tau)));
        }
        if (lane == 0) s_off[f][wy] = cnt;
    }
    __syncthreads();
    const int tid = wy * 32 + lane;
    if (tid < F) {
        uint32_t total = 0;
#pragma unroll
        for (int w = 0; w < WY; ++w) {
            const uint32_t c = s_off[tid][w];
            s_off[tid][w] = total;
            total += c;
        }
        uint32_t base = 0;
        if (total) {
            base = atomicAdd(a.count + tid * a.count_fstride, total);
            if ((uint64_t)base + total > (uint64_t)a.capacity) atomicOr(a.status, kStatusCapacity);
        }
        s_base[tid] = base;
    }
    __syncthreads();
    const uint32_t lt_mask = (1u << lane) - 1u;
#pragma unroll
    for (int f = 0; f < F; ++f) {
        uint32_t *list = a.list + f * a.list_fstride;
        uint32_t pos = s_base[f] + s_off[f][wy];
#pragma unroll
        for (int t = 0; t < TZ; ++t) {
            const bool valid = in_xy && (k0 + t < a.nz);
            const float lo = L[f][t] + a.logit_prior;
            const uint32_t b = __ballot_sync(0xFFFFFFFFu, valid && (lo > a.logit_tau));
            if ((b >> lane) & 1u) {
                const uint32_t p = pos + __popc(b & lt_mask);
                if (p < a.capacity) list[p] = lin0 + (uint32_t)t * zstride;
            }
            pos += __popc(b);
        }
    }
}

// The tile decomposition, per-tile camera records and projection are those of
// the direct fuse kernel; a thread holds F x TZ log-odds accumulators.  The
// gather of one tile: every camera in order 0 .. n_cams - 1, one vector load
// of the F frames' log ratios per (voxel, camera).  A pixel record holds S
// such F-frame parts (S lanes share a voxel); this lane reads part `part`.
// s_flags must hold the tile's camera flags (a barrier after they were
// written).
template <typename MapT, int LX, int WY, int TZ, int F, int S = 1>
__device__ __forceinline__ void group_gather(const FuseArgs &a, const TileCoords<LX, WY, TZ> &tc,
                                             const int *s_flags, float (&L)[F][TZ], int part = 0)
{
    using Words = GroupWords<MapT, F>;
    constexpr int kRec = S * Words::kWords;   // words per pixel record
    const uint32_t W = (uint32_t)a.W, H = (uint32_t)a.H;
#pragma unroll
    for (int f = 0; f < F; ++f)
#pragma unroll
        for (int t = 0; t < TZ; ++t) L[f][t] = 0.0f;
    const uint32_t *maps = reinterpret_cast<const uint32_t *>(a.maps);
    const uint32_t last_pix = W * H - 1u;
    const uint32_t bias_off = 0u - (kFloorBias * W + kFloorBias);
    for (int c = 0; c < a.n_cams; ++c) {
        const int flags = s_flags[c];
        if (flags & kTcSkip) continue;
        float m[12];
#pragma unroll
        for (int q = 0; q < 12; ++q) m[q] = a.cam[c].m[q];
        float bu, bv, bw;
        project_base(m, tc.fi, tc.fj, &bu, &bv, &bw);
        const uint32_t *map = maps + (int64_t)c * a.map_stride * kRec + part * Words::kWords;
        if (flags & kTcInside) {
#pragma unroll
            for (int t = 0; t < TZ; ++t) {
                const Proj p = project_biased(m, bu, bv, bw, tc.fk[t]);
                // the host proved the pixel lies in the image; min() only guards the buffer
                const uint32_t pix = min(p.by * W + p.bx + bias_off, last_pix);
                if (!PSFS_IN_BOUNDS(proved_inside(p, W, H), a.status)) continue;
                Words g;
                load_words<Words::kWords>(map + (size_t)pix * kRec, g.w);
                add_words<MapT, F, TZ>(g, L, t);
            }
        } else {
#pragma unroll
            for (int t = 0; t < TZ; ++t) {
                int pix;
                if (proj_pixel(project_biased(m, bu, bv, bw, tc.fk[t]), W, H, &pix)) {
                    Words g;
                    load_words<Words::kWords>(map + (size_t)pix * kRec, g.w);
                    add_words<MapT, F, TZ>(g, L, t);
                }
            }
        }
    }
}

template <typename MapT, int LX, int WY, int TZ, int F>
__global__ void __launch_bounds__(32 * WY) fuse_group_kernel(const __grid_constant__ FuseArgs a)
{
    __shared__ int s_flags[PSFS_MAX_CAMS];
    __shared__ uint32_t s_off[F][WY];
    __shared__ uint32_t s_base[F];

    const int lane = threadIdx.x;
    const int wy = threadIdx.y;
    const int tid = wy * 32 + lane;
    if (tid < a.n_cams) s_flags[tid] = __ldg(&a.tilecam[(int64_t)blockIdx.x * a.n_cams + tid].w) >> 16;

    TileCoords<LX, WY, TZ> tc;
    tc.init(a, a.tiles[blockIdx.x], lane, wy);
    float L[F][TZ];
    __syncthreads();
    group_gather<MapT, LX, WY, TZ, F>(a, tc, s_flags, L);
    group_epilogue<WY, TZ, F>(a, tc.i, tc.j, tc.k0, L, lane, wy, s_off, s_base);
}

// Epilogue of a plane of 64-byte records: the two half-warps hold frames
// 0 .. FL - 1 and FL .. 2 FL - 1 of the same 16 voxel columns.  Per frame the
// posterior, threshold and compaction of group_epilogue (the same per-voxel
// arithmetic); a ballot serves both halves' frames (low and high 16 bits).
template <int TZ, int FL>
__device__ __forceinline__ void pair_epilogue(const FuseArgs &a, int i, int j, int k0, const float (&L)[FL][TZ],
                                              int lane, int wy, int half, uint32_t (*s_off)[kPairWarps],
                                              uint32_t *s_base)
{
    constexpr int P = 2 * FL;
    const bool in_xy = (i < a.nx) && (j < a.ny);
    const uint32_t zstride = (uint32_t)a.nx * (uint32_t)a.ny;
    const uint32_t lin0 = (uint32_t)i + (uint32_t)a.nx * ((uint32_t)j + (uint32_t)a.ny * (uint32_t)k0);
#pragma unroll
    for (int e = 0; e < FL; ++e) {
        float *occ = a.occ + (half * FL + e) * a.occ_fstride;
        uint32_t c_lo = 0, c_hi = 0;
#pragma unroll
        for (int t = 0; t < TZ; ++t) {
            const bool valid = in_xy && (k0 + t < a.nz);
            const float lo = L[e][t] + a.logit_prior;
            if (valid) __stcs(occ + lin0 + (uint32_t)t * zstride, posterior_of_logodds(lo));
            const uint32_t b = __ballot_sync(0xFFFFFFFFu, valid && (lo > a.logit_tau));
            c_lo += __popc(b & 0xFFFFu);
            c_hi += __popc(b >> 16);
        }
        if (lane == 0) {
            s_off[e][wy] = c_lo;
            s_off[FL + e][wy] = c_hi;
        }
    }
    __syncthreads();
    const int tid = wy * 32 + lane;
    if (tid < P) {
        uint32_t total = 0;
#pragma unroll
        for (int w = 0; w < kPairWarps; ++w) {
            const uint32_t c = s_off[tid][w];
            s_off[tid][w] = total;
            total += c;
        }
        uint32_t base = 0;
        if (total) {
            base = atomicAdd(a.count + tid * a.count_fstride, total);
            if ((uint64_t)base + total > (uint64_t)a.capacity) atomicOr(a.status, kStatusCapacity);
        }
        s_base[tid] = base;
    }
    __syncthreads();
    const uint32_t lt_mask = (1u << lane) - 1u;
    const uint32_t half_mask = half ? 0xFFFF0000u : 0x0000FFFFu;
#pragma unroll
    for (int e = 0; e < FL; ++e) {
        const int f = half * FL + e;
        uint32_t *list = a.list + f * a.list_fstride;
        uint32_t pos = s_base[f] + s_off[f][wy];
#pragma unroll
        for (int t = 0; t < TZ; ++t) {
            const bool valid = in_xy && (k0 + t < a.nz);
            const float lo = L[e][t] + a.logit_prior;
            const uint32_t b = __ballot_sync(0xFFFFFFFFu, valid && (lo > a.logit_tau)) & half_mask;
            if ((b >> lane) & 1u) {
                const uint32_t q = pos + __popc(b & lt_mask);
                if (q < a.capacity) list[q] = lin0 + (uint32_t)t * zstride;
            }
            pos += __popc(b);
        }
    }
}

// Fusion of one plane of 64-byte records (16 FP32 or 32 16-bit frames per
// pixel).  kPairWarps warps cover the tile of the 4-warp fuse_group_kernel:
// lane l of warp w takes the voxel column of that kernel's thread
// 16 w + (l & 15) and the frames of record half l >> 4, so both 32-byte
// halves of a record are loaded by the same warp request.
template <typename MapT, int LX, int TZ, int FL>
__global__ void __launch_bounds__(32 * kPairWarps) fuse_pair_kernel(const __grid_constant__ FuseArgs a)
{
    __shared__ int s_flags[PSFS_MAX_CAMS];
    __shared__ uint32_t s_off[2 * FL][kPairWarps];
    __shared__ uint32_t s_base[2 * FL];

    const int lane = threadIdx.x;
    const int wy = threadIdx.y;
    const int tid = wy * 32 + lane;
    const int half = lane >> 4;
    const int vt = wy * 16 + (lane & 15);   // thread of the 4-warp tile whose voxel column this lane takes
    if (tid < a.n_cams) s_flags[tid] = __ldg(&a.tilecam[(int64_t)blockIdx.x * a.n_cams + tid].w) >> 16;

    TileCoords<LX, 4, TZ> tc;
    tc.init(a, a.tiles[blockIdx.x], vt & 31, vt >> 5);
    float L[FL][TZ];
    __syncthreads();
    group_gather<MapT, LX, 4, TZ, FL, 2>(a, tc, s_flags, L, half);
    pair_epilogue<TZ, FL>(a, tc.i, tc.j, tc.k0, L, lane, wy, half, s_off, s_base);
}

// The adjoint's voxel pass over F frames of records (psfs_backward_sequence):
// the log-odds of the F frames exactly as fuse_group_kernel forms them, then
// per voxel and frame dLoss/dL = d_occ occ (1 - occ), written to slots 0 ..
// F - 1 of the voxel's record at b.dl + lin * kBwRecord (b.dl already points
// at the unit's first slot; F <= kBwRecord).  Frame f's d_occ is at b.d_occ +
// f * docc_fstride.
template <typename MapT, int LX, int WY, int TZ, int F>
__global__ void __launch_bounds__(32 * WY) backward_voxel_group_kernel(const __grid_constant__ BackwardArgs b,
                                                                       int64_t docc_fstride)
{
    static_assert(F <= kBwRecord, "a unit fills at most one record");
    const FuseArgs &a = b.f;
    __shared__ int s_flags[PSFS_MAX_CAMS];
    const int lane = threadIdx.x;
    const int wy = threadIdx.y;
    const int tid = wy * 32 + lane;
    if (tid < a.n_cams) s_flags[tid] = __ldg(&a.tilecam[(int64_t)blockIdx.x * a.n_cams + tid].w) >> 16;
    TileCoords<LX, WY, TZ> tc;
    tc.init(a, a.tiles[blockIdx.x], lane, wy);
    float L[F][TZ];
    __syncthreads();
    group_gather<MapT, LX, WY, TZ, F>(a, tc, s_flags, L);
    if (tc.i >= a.nx || tc.j >= a.ny) return;
#pragma unroll
    for (int t = 0; t < TZ; ++t) {
        const int k = tc.k0 + t;
        if (k >= a.nz) break;
        const uint32_t lin = (uint32_t)tc.i + (uint32_t)a.nx * ((uint32_t)tc.j + (uint32_t)a.ny * (uint32_t)k);
        float *rec = b.dl + (size_t)lin * kBwRecord;
#pragma unroll
        for (int f = 0; f < F; ++f) {
            const float occ = posterior_of_logodds(L[f][t] + a.logit_prior);
            rec[f] = __ldg(b.d_occ + f * docc_fstride + lin) * occ * (1.0f - occ);
        }
    }
}

template <typename MapT, int LX, int TZ, int F>
cudaError_t launch_fg(const FuseArgs &a, cudaStream_t s)
{
    fuse_group_kernel<MapT, LX, 4, TZ, F><<<a.n_tiles, dim3(32, 4), 0, s>>>(a);
    return cudaGetLastError();
}

template <typename MapT, int LX, int F>
cudaError_t launch_fg_tz(const FuseArgs &a, int tz, cudaStream_t s)
{
    // F x TZ accumulators per thread: at most 64 (TZ = 2 with up to 16 frames: 32)
    if (tz == 2) return launch_fg<MapT, LX, 2, F>(a, s);
    if (tz == 4) return launch_fg<MapT, LX, 4, F>(a, s);
    if constexpr (F <= 8) {
        if (tz == 8) return launch_fg<MapT, LX, 8, F>(a, s);
    }
    if constexpr (F <= 4) {
        if (tz == 16) return launch_fg<MapT, LX, 16, F>(a, s);
    }
    return cudaErrorInvalidValue;
}

template <typename MapT, int F>
cudaError_t launch_fg_shape(const FuseArgs &a, const FuseShape &sh, cudaStream_t s)
{
    if (sh.wy != 4 || sh.staged) return cudaErrorInvalidValue;
    if (sh.lx == 8) return launch_fg_tz<MapT, 8, F>(a, sh.tz, s);
    if (sh.lx == 16) return launch_fg_tz<MapT, 16, F>(a, sh.tz, s);
    return cudaErrorInvalidValue;
}

template <typename MapT, int LX, int TZ>
cudaError_t launch_fp(const FuseArgs &a, cudaStream_t s)
{
    constexpr int FL = 32 / (int)sizeof(MapT);   // frames per lane: one 32-byte half of the record
    fuse_pair_kernel<MapT, LX, TZ, FL><<<a.n_tiles, dim3(32, kPairWarps), 0, s>>>(a);
    return cudaGetLastError();
}

// One plane of 64-byte records.
template <typename MapT>
cudaError_t launch_fp_typed(const FuseArgs &a, const FuseShape &sh, cudaStream_t s)
{
    if (((uintptr_t)a.maps) & 63u) return cudaErrorMisalignedAddress;
    if (sh.wy != 4 || sh.staged || (sh.lx != 8 && sh.lx != 16)) return cudaErrorInvalidValue;
    // FL x TZ accumulators per thread: at most 32
    if (sh.tz == 2) return sh.lx == 8 ? launch_fp<MapT, 8, 2>(a, s) : launch_fp<MapT, 16, 2>(a, s);
    if (sh.tz == 4) return sh.lx == 8 ? launch_fp<MapT, 8, 4>(a, s) : launch_fp<MapT, 16, 4>(a, s);
    return cudaErrorInvalidValue;
}

// One plane of P frames (records of at most 32 bytes).
template <typename MapT>
cudaError_t launch_fg_typed(const FuseArgs &a, const FuseShape &sh, int frames, cudaStream_t s)
{
    if (((uintptr_t)a.maps) & (uintptr_t)(frames * sizeof(MapT) - 1)) return cudaErrorMisalignedAddress;
    if (frames == 2) return launch_fg_shape<MapT, 2>(a, sh, s);
    if (frames == 4) return launch_fg_shape<MapT, 4>(a, sh, s);
    if (frames == 8) return launch_fg_shape<MapT, 8>(a, sh, s);
    if constexpr (sizeof(MapT) == 2) {
        if (frames == 16) return launch_fg_shape<MapT, 16>(a, sh, s);
    }
    return cudaErrorInvalidValue;
}

template <typename MapT, int F>
cudaError_t launch_bvg(const BackwardArgs &b, const FuseShape &sh, int64_t docc_fstride, cudaStream_t s)
{
    if (sh.wy != 4 || sh.staged || sh.tz != 4) return cudaErrorInvalidValue;
    if (sh.lx == 8)
        backward_voxel_group_kernel<MapT, 8, 4, 4, F><<<b.f.n_tiles, dim3(32, 4), 0, s>>>(b, docc_fstride);
    else if (sh.lx == 16)
        backward_voxel_group_kernel<MapT, 16, 4, 4, F><<<b.f.n_tiles, dim3(32, 4), 0, s>>>(b, docc_fstride);
    else
        return cudaErrorInvalidValue;
    return cudaGetLastError();
}

template <typename MapT>
cudaError_t launch_bvg_typed(const BackwardArgs &b, const FuseShape &sh, int frames, int64_t docc_fstride,
                             cudaStream_t s)
{
    if (((uintptr_t)b.f.maps) & (uintptr_t)(frames * sizeof(MapT) - 1)) return cudaErrorMisalignedAddress;
    if (frames == 2) return launch_bvg<MapT, 2>(b, sh, docc_fstride, s);
    if (frames == 4) return launch_bvg<MapT, 4>(b, sh, docc_fstride, s);
    if (frames == 8) return launch_bvg<MapT, 8>(b, sh, docc_fstride, s);
    return cudaErrorInvalidValue;
}

}  // namespace

cudaError_t launch_backward_voxel_group(const BackwardArgs &b, const FuseShape &shape, int frames, int map_dtype,
                                        int64_t docc_fstride, cudaStream_t s)
{
    if (b.f.n_tiles <= 0) return cudaSuccess;
    if (map_dtype == PSFS_MAP_F16) return launch_bvg_typed<__half>(b, shape, frames, docc_fstride, s);
    if (map_dtype == PSFS_MAP_BF16) return launch_bvg_typed<__nv_bfloat16>(b, shape, frames, docc_fstride, s);
    return launch_bvg_typed<float>(b, shape, frames, docc_fstride, s);
}

bool group_size_supported(int frames)
{
    return frames == 2 || frames == 4 || frames == 8 || frames == 16 || frames == kMaxGroup;
}

bool group_shape_supported(const FuseShape &s, int frames, int map_elem, int rec)
{
    if (rec != 32 && rec != 64) return false;
    // a thread holds (frames per lane) x TZ accumulators: at most 64 with
    // 32-byte records (32 with 64-byte records, two lanes per voxel)
    const int P = group_plane_frames(frames, map_elem, rec);
    const bool pair = P * map_elem == 64;
    if (!(group_size_supported(frames) && s.wy == 4 && s.staged == 0 && (s.lx == 8 || s.lx == 16))) return false;
    if (pair) return s.tz == 2 || s.tz == 4;
    return s.tz == 2 || s.tz == 4 || (s.tz == 8 && P <= 8) || (s.tz == 16 && P <= 4);
}

cudaError_t launch_likelihood_group(const LikelihoodArgs &a, int frames, int map_dtype, cudaStream_t s,
                                    int ctas_per_sm, int rec)
{
    if (map_dtype == PSFS_MAP_F16) return launch_lk_group_typed<__half>(a, frames, s, ctas_per_sm, rec);
    if (map_dtype == PSFS_MAP_BF16) return launch_lk_group_typed<__nv_bfloat16>(a, frames, s, ctas_per_sm, rec);
    return launch_lk_group_typed<float>(a, frames, s, ctas_per_sm, rec);
}

cudaError_t launch_fuse_group(const FuseArgs &a, const FuseShape &shape, int frames, int map_dtype,
                              cudaStream_t s, int rec)
{
    if (a.n_tiles <= 0) return cudaSuccess;
    const bool half = map_dtype == PSFS_MAP_F16 || map_dtype == PSFS_MAP_BF16;
    const int elem = half ? 2 : 4;
    const int P = group_plane_frames(frames, elem, rec);
    const bool pair = P * elem == 64;
    const int64_t plane_bytes = (int64_t)a.n_cams * a.map_stride * P * elem;
    for (int q = 0; q * P < frames; ++q) {
        // plane q: frames qP to qP + P - 1
        FuseArgs fq = a;
        fq.maps = static_cast<const char *>(a.maps) + q * plane_bytes;
        fq.occ = a.occ + (int64_t)q * P * a.occ_fstride;
        fq.list = a.list + (int64_t)q * P * a.list_fstride;
        fq.count = a.count + (int64_t)q * P * a.count_fstride;
        cudaError_t e;
        if (map_dtype == PSFS_MAP_F16)
            e = pair ? launch_fp_typed<__half>(fq, shape, s) : launch_fg_typed<__half>(fq, shape, P, s);
        else if (map_dtype == PSFS_MAP_BF16)
            e = pair ? launch_fp_typed<__nv_bfloat16>(fq, shape, s) : launch_fg_typed<__nv_bfloat16>(fq, shape, P, s);
        else
            e = pair ? launch_fp_typed<float>(fq, shape, s) : launch_fg_typed<float>(fq, shape, P, s);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

}  // namespace psfs
