// transpose.cu -- out = in^T for a row-major R x C matrix of 1-, 2- or
// 4-byte elements.  The library uses it to lay a volume out in another axis
// order (one transpose of the N x N^2 or N^2 x N view moves one axis to the
// front or the back), so that a transform's ingest reads contiguous runs.
#include "internal.cuh"

namespace drt3d {
namespace {

// Generic: 32 x 32 tiles in shared memory, one element per thread and step.
template <typename T>
__global__ void __launch_bounds__(256) transpose_tile32(const T* __restrict__ in, T* __restrict__ out, long long R,
                                                        int C, long long tilesC) {
    pdl_wait_and_release();
    __shared__ T tile[32][33];
    const long long b = blockIdx.x;
    const long long r0 = (b / tilesC) * 32;
    const int c0 = (int)(b % tilesC) * 32;
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
#pragma unroll
    for (int k = ty; k < 32; k += 8) {
        const long long r = r0 + k;
        const int c = c0 + tx;
        if (r < R && c < C) tile[k][tx] = in[r * C + c];
    }
    __syncthreads();
#pragma unroll
    for (int k = ty; k < 32; k += 8) {
        const int c = c0 + k;
        const long long r = r0 + tx;
        if (r < R && c < C) out[(long long)c * R + r] = tile[tx][k];
    }
}

// Bytes, R and C multiples of 64: 64 x 64 tiles moved as 16-byte vectors.
// Load: thread t reads bytes 16 (t % 4) .. + 15 of tile row t / 4.  Store:
// thread t = 64 p + c gathers tile rows 16 p .. 16 p + 15 of column c (a warp
// reads 32 neighbouring bytes of one row per step: no bank conflicts) and
// writes them as one vector of output row c.
constexpr int kPitch8 = 80;  // bytes per shared tile row (16-byte aligned)

__global__ void __launch_bounds__(256) transpose_u8_tile64(const uint8_t* __restrict__ in, uint8_t* __restrict__ out,
                                                           long long R, long long C, long long tilesC) {
    pdl_wait_and_release();
    __shared__ __align__(16) uint8_t tile[64 * kPitch8];
    const long long b = blockIdx.x;
    const long long r0 = (b / tilesC) * 64;
    const long long c0 = (b % tilesC) * 64;
    const int t = threadIdx.x;
    {
        const int row = t >> 2, col = (t & 3) * 16;
        const uint4 w = __ldg(reinterpret_cast<const uint4*>(in + (r0 + row) * C + c0 + col));
        *reinterpret_cast<uint4*>(tile + row * kPitch8 + col) = w;
    }
    __syncthreads();
    const int c = t & 63, p = t >> 6;
    uint32_t w[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const uint8_t* s = tile + (16 * p + 4 * q) * kPitch8 + c;
        w[q] = (uint32_t)s[0] | ((uint32_t)s[kPitch8] << 8) | ((uint32_t)s[2 * kPitch8] << 16) |
               ((uint32_t)s[3 * kPitch8] << 24);
    }
    *reinterpret_cast<uint4*>(out + (c0 + c) * R + r0 + 16 * p) = make_uint4(w[0], w[1], w[2], w[3]);
}

}  // namespace

cudaError_t launch_transpose2d(const void* in, void* out, long long R, int C, int esz, cudaStream_t s) {
    if (esz == 1 && R % 64 == 0 && C % 64 == 0) {
        const long long tilesC = C / 64;
        return launch_chained(transpose_u8_tile64, dim3((unsigned)((R / 64) * tilesC)), dim3(256), 0, s,
                              static_cast<const uint8_t*>(in), static_cast<uint8_t*>(out), R, C, tilesC);
    }
    const long long tilesC = (C + 31) / 32;
    const dim3 grid((unsigned)(((R + 31) / 32) * tilesC));
    switch (esz) {
    case 1:
        return launch_chained(transpose_tile32<uint8_t>, grid, dim3(256), 0, s, static_cast<const uint8_t*>(in),
                              static_cast<uint8_t*>(out), R, C, tilesC);
    case 2:
        return launch_chained(transpose_tile32<uint16_t>, grid, dim3(256), 0, s, static_cast<const uint16_t*>(in),
                              static_cast<uint16_t*>(out), R, C, tilesC);
    case 4:
        return launch_chained(transpose_tile32<uint32_t>, grid, dim3(256), 0, s, static_cast<const uint32_t*>(in),
                              static_cast<uint32_t*>(out), R, C, tilesC);
    default:
        return cudaErrorInvalidValue;
    }
}

}  // namespace drt3d
