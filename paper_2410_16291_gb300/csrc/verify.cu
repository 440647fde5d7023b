// Device-side check of summed-area tables against their image by the
// recurrence that defines them (Section II-B):
//
//   S[y][x] - S[y][x-1] - S[y-1][x] + S[y-1][x-1] = I[y][x]   (mod 2^64)
//
// with index -1 reading as 0, and Q likewise with I^2.  If every entry passes,
// the table is the image's summed-area table modulo 2^64 (induction over y,
// then x), hence exactly, since no entry reaches 2^64 (the overflow bound).
// The check reads each table about twice and the image once, so the 95 GB
// tables of a 70,000 x 85,000 image are checked in place, without a copy to
// the host.
#include <cuda_runtime.h>
#include <stdint.h>

#include "swa_internal.h"

namespace swa {
namespace {

constexpr int kVerifyThreads = 256;
constexpr int kVerifyCols = 8;                  // consecutive columns per thread

template <typename T>
__device__ __forceinline__ uint64_t pixel(const char *row, int64_t x)
{
    return (uint64_t)reinterpret_cast<const T *>(row)[x];
}

// Blocks take rows (grid-stride); a thread checks 8 consecutive entries of
// its row, carrying the left neighbours along.
template <typename T>
__global__ void __launch_bounds__(kVerifyThreads)
k_verify(const char *img, int64_t pitch, int64_t rows, int64_t cols, const uint64_t *S,
         const uint64_t *Q, int64_t ld, unsigned long long *out)
{
    unsigned long long bad_s = 0, bad_q = 0, first = ~0ull;
    for (int64_t y = blockIdx.x; y < rows; y += gridDim.x) {
        const char *irow = img + y * pitch;
        const uint64_t *s1 = S + y * ld, *s0 = y ? S + (y - 1) * ld : nullptr;
        const uint64_t *q1 = Q ? Q + y * ld : nullptr;
        const uint64_t *q0 = (Q && y) ? Q + (y - 1) * ld : nullptr;
        for (int64_t x0 = (int64_t)threadIdx.x * kVerifyCols; x0 < cols;
             x0 += (int64_t)kVerifyThreads * kVerifyCols) {
            uint64_t ls = x0 ? s1[x0 - 1] : 0, uls = (x0 && s0) ? s0[x0 - 1] : 0;
            uint64_t lq = (Q && x0) ? q1[x0 - 1] : 0, ulq = (Q && x0 && q0) ? q0[x0 - 1] : 0;
#pragma unroll
            for (int k = 0; k < kVerifyCols; ++k) {
                const int64_t x = x0 + k;
                if (x >= cols) break;
                const uint64_t v = pixel<T>(irow, x);
                const uint64_t s = s1[x], us = s0 ? s0[x] : 0;
                if (s - ls - us + uls != v) {
                    ++bad_s;
                    first = min(first, (unsigned long long)(y * cols + x));
                }
                ls = s;
                uls = us;
                if (Q) {
                    const uint64_t q = q1[x], uq = q0 ? q0[x] : 0;
                    if (q - lq - uq + ulq != v * v) {
                        ++bad_q;
                        first = min(first, (unsigned long long)(y * cols + x));
                    }
                    lq = q;
                    ulq = uq;
                }
            }
        }
    }
    if (bad_s) atomicAdd(&out[0], bad_s);
    if (bad_q) atomicAdd(&out[1], bad_q);
    if (first != ~0ull) atomicMin(&out[2], first);
}

}  // namespace
}  // namespace swa

extern "C" swa_status swa_verify_tables(const void *d_image, int64_t rows, int64_t cols,
                                        int64_t pitch_bytes, swa_dtype dtype,
                                        const uint64_t *d_S, const uint64_t *d_Q, int64_t ld,
                                        uint64_t *d_counts, swa_stream stream)
{
    using namespace swa;
    if (!d_image || !d_S || !d_counts || rows <= 0 || cols <= 0 ||
        (dtype != SWA_U8 && dtype != SWA_U16) || pitch_bytes < cols * pixel_bytes(dtype) ||
        ld < cols) {
        set_error("bad arguments to swa_verify_tables");
        return SWA_EINVAL;
    }
    if (dtype == SWA_U16 && ((uintptr_t)d_image % 2 || pitch_bytes % 2)) {
        set_error("uint16 images need a 2-byte aligned base and an even pitch");
        return SWA_EINVAL;
    }
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    cudaError_t e;
    if ((e = cudaMemsetAsync(d_counts, 0, 2 * sizeof(uint64_t), s)) != cudaSuccess ||
        (e = cudaMemsetAsync(d_counts + 2, 0xff, sizeof(uint64_t), s)) != cudaSuccess)
        return cuda_fail(e, "cudaMemsetAsync");
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int64_t blocks = rows < (int64_t)sms * 8 ? rows : (int64_t)sms * 8;
    auto *out = reinterpret_cast<unsigned long long *>(d_counts);
    const char *img = static_cast<const char *>(d_image);
    {
        LaunchScope ls("verify_tables", s);
        if (dtype == SWA_U8)
            k_verify<uint8_t><<<(unsigned)blocks, kVerifyThreads, 0, s>>>(
                img, pitch_bytes, rows, cols, d_S, d_Q, ld, out);
        else
            k_verify<uint16_t><<<(unsigned)blocks, kVerifyThreads, 0, s>>>(
                img, pitch_bytes, rows, cols, d_S, d_Q, ld, out);
    }
    if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(e, "verify launch");
    return SWA_OK;
}
