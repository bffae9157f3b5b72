// psfs_gather.cu -- the gather rate that bounds the fusion kernels.
//
// The fusion kernels read, per (voxel, camera), the pixel record of the
// camera's map at the voxel's projection (Eq. 3): scattered 32- or 64-byte
// rows, one 256-bit read-only load per lane and 32-byte half.  Their rate is
// set by how fast the memory system delivers such scattered rows into
// registers, which a plain HBM copy does not measure.  psfs_gather_rows
// performs only those loads (the same instruction, two rows in flight per
// lane as a fusion thread's two voxels) over caller-given row indices, so
// that a measurement can set the fusion's achieved gather rate against the
// device's own ceiling for that access.
#include "psfs_internal.cuh"

namespace psfs {

namespace {

__device__ __forceinline__ void load_v8(const uint32_t *p, uint32_t (&w)[8])
{
    asm volatile("ld.global.nc.L1::no_allocate.v8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
                 : "=r"(w[0]), "=r"(w[1]), "=r"(w[2]), "=r"(w[3]), "=r"(w[4]), "=r"(w[5]), "=r"(w[6]), "=r"(w[7])
                 : "l"(p));
}

// kHalves lanes per row (1: 32-byte rows, 2: 64-byte rows); a warp request
// covers 32 / kHalves rows, each lane keeps two requests in flight.
template <int kHalves>
__global__ void __launch_bounds__(256) gather_rows_kernel(const uint32_t *rows, int64_t n_rows, const int32_t *idx,
                                                          int64_t n, uint32_t *checksum)
{
    constexpr int kRows = 32 / kHalves;      // rows per warp request
    constexpr int kWords = 8 * kHalves;      // 32-bit words per row
    const int lane = threadIdx.x & 31;
    const int half = lane / kRows, slot = lane % kRows;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t n_warps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    uint32_t x = 0;
    for (int64_t base = warp * 2 * kRows; base < n; base += n_warps * 2 * kRows) {
        const int64_t ia = base + slot, ib = base + kRows + slot;
        const int32_t ra = ia < n ? __ldg(idx + ia) : -1, rb = ib < n ? __ldg(idx + ib) : -1;
        uint32_t a[8] = {0, 0, 0, 0, 0, 0, 0, 0}, b[8] = {0, 0, 0, 0, 0, 0, 0, 0};
        if (ra >= 0 && ra < n_rows) load_v8(rows + (size_t)ra * kWords + 8 * half, a);
        if (rb >= 0 && rb < n_rows) load_v8(rows + (size_t)rb * kWords + 8 * half, b);
#pragma unroll
        for (int k = 0; k < 8; ++k) x ^= a[k] ^ b[k];
    }
    x = __reduce_xor_sync(0xFFFFFFFFu, x);
    if (lane == 0) atomicXor(checksum, x);
}

}  // namespace

}  // namespace psfs

using namespace psfs;

extern "C" psfs_status psfs_gather_rows(const void *rows, int64_t n_rows, int32_t record_bytes, const int32_t *idx,
                                        int64_t n, void *stream, uint32_t *checksum)
{
    if (record_bytes != 32 && record_bytes != 64)
        return record_failure(PSFS_ERR_INVALID_ARG, "record_bytes not 32 or 64");
    if (n_rows < 0 || n < 0) return record_failure(PSFS_ERR_INVALID_ARG, "n_rows or n < 0");
    if (!rows || (reinterpret_cast<uintptr_t>(rows) & (uintptr_t)(record_bytes - 1)))
        return record_failure(PSFS_ERR_INVALID_ARG, "rows NULL or not aligned to record_bytes");
    if (n > 0 && (!idx || (reinterpret_cast<uintptr_t>(idx) & 3u)))
        return record_failure(PSFS_ERR_INVALID_ARG, "idx NULL or not 4-byte aligned");
    if (!checksum || (reinterpret_cast<uintptr_t>(checksum) & 3u))
        return record_failure(PSFS_ERR_INVALID_ARG, "checksum NULL or not 4-byte aligned");
    if (n == 0) return PSFS_OK;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int blocks = device_sm_count() * 8;   // 8 CTAs of 8 warps per SM, grid-stride
    const uint32_t *r = static_cast<const uint32_t *>(rows);
    if (record_bytes == 64)
        gather_rows_kernel<2><<<blocks, 256, 0, s>>>(r, n_rows, idx, n, checksum);
    else
        gather_rows_kernel<1><<<blocks, 256, 0, s>>>(r, n_rows, idx, n, checksum);
    const cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? PSFS_OK : record_cuda_failure(e, "gather_rows_kernel launch");
}
