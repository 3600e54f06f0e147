// press.cu -- element-wise and stencil kernels of the iterative inverse of
// the planes transform (Section 5.2): the high-pass filter h, the
// prolongation P, the restriction S, the exact N = 1 solve, residuals and
// the norms of the power iteration that sets the step sizes.  The forward and
// adjoint transforms they are combined with are the library's own kernels;
// the host side (api.cu) sequences them.
//
// The filter h of Section 5.2 is delta - k (x) k (x) k with k = (1/4, 1/2,
// 1/4): weight 7/8 at the centre, -1/16 at the 6 face neighbours, -1/32 at
// the 12 edge neighbours and -1/64 at the 8 corners.  Borders are mirrored: a
// neighbour outside the cube takes the nearest voxel inside.
#include "internal.cuh"

namespace drt3d {
namespace {

constexpr int kThreads = 256;

// y = c * (h (*) b) (+ y when ACC); one thread per voxel, neighbours through
// the read-only cache.  The 27 terms are summed in a fixed order: the
// smoothing k (x) k (x) k first (integer weights 1, 2, 1 per axis, the 1/64
// applied once at the end), then subtracted from the centre value.
template <bool ACC>
__global__ void __launch_bounds__(kThreads) press_filter(const float* __restrict__ b, float* __restrict__ y, int N,
                                                         float c) {
    pdl_wait_and_release();
    const long long i = (long long)blockIdx.x * kThreads + threadIdx.x;
    const long long NN = (long long)N * N;
    if (i >= NN * N) return;
    const int x0 = (int)(i / NN), x1 = (int)((i / N) % N), x2 = (int)(i % N);
    const int a0[3] = {max(x0 - 1, 0), x0, min(x0 + 1, N - 1)};
    const int a1[3] = {max(x1 - 1, 0), x1, min(x1 + 1, N - 1)};
    const int a2[3] = {max(x2 - 1, 0), x2, min(x2 + 1, N - 1)};
    const float w[3] = {1.f, 2.f, 1.f};
    float s = 0.f;
#pragma unroll
    for (int p = 0; p < 3; ++p) {
        float sp = 0.f;
#pragma unroll
        for (int q = 0; q < 3; ++q) {
            const float* row = b + (a0[p] * NN + (long long)a1[q] * N);
            const float sq = __ldg(row + a2[0]) + 2.f * __ldg(row + a2[1]) + __ldg(row + a2[2]);
            sp += w[q] * sq;
        }
        s += w[p] * sp;
    }
    const float hb = __ldg(b + i) - s * (1.f / 64.f);
    y[i] = ACC ? y[i] + c * hb : c * hb;
}

// Fine voxel (i, j, k) <- coarse voxel (i/2, j/2, k/2); N is the fine size.
__global__ void __launch_bounds__(kThreads) press_prolong(const float* __restrict__ xc, float* __restrict__ x, int N) {
    pdl_wait_and_release();
    const long long i = (long long)blockIdx.x * kThreads + threadIdx.x;
    const long long NN = (long long)N * N;
    if (i >= NN * N) return;
    const int x0 = (int)(i / NN), x1 = (int)((i / N) % N), x2 = (int)(i % N);
    const int M = N / 2;
    x[i] = __ldg(xc + ((long long)(x0 >> 1) * M + (x1 >> 1)) * M + (x2 >> 1));
}

// Per dodecant, Rc(s1, s2, d) = (R(2s1, 2s2, 2d) + R(2s1, 2s2, 2d+1)) / 8 for
// d in [0, 3Nc); R has pitch 3N = 6Nc.
__global__ void __launch_bounds__(kThreads) press_restrict(const float* __restrict__ R, float* __restrict__ Rc,
                                                           int Nc) {
    pdl_wait_and_release();
    const long long i = (long long)blockIdx.x * kThreads + threadIdx.x;
    const int Wc = 3 * Nc, W = 6 * Nc, N = 2 * Nc;
    const long long per = (long long)Nc * Nc * Wc;
    if (i >= 12 * per) return;
    const int k = (int)(i / per);
    const long long r = i % per;
    const int d = (int)(r % Wc);
    const int s2 = (int)((r / Wc) % Nc), s1 = (int)(r / ((long long)Wc * Nc));
    const float* src = R + (((long long)k * N + 2 * s1) * N + 2 * s2) * W + 2 * d;
    Rc[i] = (__ldg(src) + __ldg(src + 1)) * 0.125f;
}

// Exact solve at N = 1: the voxel is at d = 2 of each dodecant's column;
// average the twelve values in dodecant order.
__global__ void press_coarsest(const float* __restrict__ R1, float* __restrict__ x1) {
    pdl_wait_and_release();
    float s = 0.f;
    for (int k = 0; k < 12; ++k) s += R1[k * 3 + 2];
    x1[0] = s / 12.f;
}

// t = r - t (t holds A x on entry).
__global__ void __launch_bounds__(kThreads) press_residual(const float* __restrict__ r, float* __restrict__ t,
                                                           long long n) {
    pdl_wait_and_release();
    const long long i = (long long)blockIdx.x * kThreads + threadIdx.x;
    if (i < n) t[i] = __ldg(r + i) - t[i];
}

// y += x.
__global__ void __launch_bounds__(kThreads) press_add(const float* __restrict__ x, float* __restrict__ y,
                                                      long long n) {
    pdl_wait_and_release();
    const long long i = (long long)blockIdx.x * kThreads + threadIdx.x;
    if (i < n) y[i] += __ldg(x + i);
}

// Per-block partial sums of squares (in double), block b covering a fixed
// contiguous range, so the total does not depend on scheduling.
__global__ void __launch_bounds__(kThreads) press_sumsq(const float* __restrict__ y, long long n, long long chunk,
                                                        double* __restrict__ partial) {
    pdl_wait_and_release();
    __shared__ double red[kThreads];
    const long long lo = (long long)blockIdx.x * chunk;
    const long long hi = min(n, lo + chunk);
    double s = 0.0;
    for (long long i = lo + threadIdx.x; i < hi; i += kThreads) {
        const double v = y[i];
        s += v * v;
    }
    red[threadIdx.x] = s;
    __syncthreads();
    for (int w = kThreads / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) partial[blockIdx.x] = red[0];
}

// x = y / ||y|| with ||y||^2 the sum of the partials (summed in block order by
// every block); block 0 also stores ||y|| in *norm.
__global__ void __launch_bounds__(kThreads) press_normalize(const float* __restrict__ y, float* __restrict__ x,
                                                            long long n, const double* __restrict__ partial,
                                                            int nparts, double* __restrict__ norm) {
    pdl_wait_and_release();
    __shared__ float inv;
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int p = 0; p < nparts; ++p) t += partial[p];
        const double nr = sqrt(t);
        inv = nr > 0.0 ? (float)(1.0 / nr) : 0.f;
        if (blockIdx.x == 0) *norm = nr;
    }
    __syncthreads();
    for (long long i = (long long)blockIdx.x * kThreads + threadIdx.x; i < n; i += (long long)gridDim.x * kThreads)
        x[i] = y[i] * inv;
}

unsigned blocks_for(long long n) { return (unsigned)((n + kThreads - 1) / kThreads); }

}  // namespace

cudaError_t launch_press_filter(const float* b, float* y, int N, float c, bool accumulate, cudaStream_t s) {
    const long long n = (long long)N * N * N;
    if (accumulate) return launch_chained(press_filter<true>, dim3(blocks_for(n)), dim3(kThreads), 0, s, b, y, N, c);
    return launch_chained(press_filter<false>, dim3(blocks_for(n)), dim3(kThreads), 0, s, b, y, N, c);
}

cudaError_t launch_press_prolong(const float* xc, float* x, int N, cudaStream_t s) {
    return launch_chained(press_prolong, dim3(blocks_for((long long)N * N * N)), dim3(kThreads), 0, s, xc, x, N);
}

cudaError_t launch_press_restrict(const float* R, float* Rc, int Nc, cudaStream_t s) {
    return launch_chained(press_restrict, dim3(blocks_for(12LL * Nc * Nc * 3 * Nc)), dim3(kThreads), 0, s, R, Rc, Nc);
}

cudaError_t launch_press_coarsest(const float* R1, float* x1, cudaStream_t s) {
    return launch_chained(press_coarsest, dim3(1), dim3(1), 0, s, R1, x1);
}

cudaError_t launch_press_residual(const float* r, float* t, long long n, cudaStream_t s) {
    return launch_chained(press_residual, dim3(blocks_for(n)), dim3(kThreads), 0, s, r, t, n);
}

cudaError_t launch_press_add(const float* x, float* y, long long n, cudaStream_t s) {
    return launch_chained(press_add, dim3(blocks_for(n)), dim3(kThreads), 0, s, x, y, n);
}

cudaError_t launch_press_normalize(const float* y, float* x, long long n, double* partial, double* norm,
                                   cudaStream_t s) {
    const long long chunk = (n + kPressNormParts - 1) / kPressNormParts;
    const cudaError_t e = launch_chained(press_sumsq, dim3(kPressNormParts), dim3(kThreads), 0, s, y, n, chunk, partial);
    if (e != cudaSuccess) return e;
    const unsigned nb = (unsigned)std::min<long long>(blocks_for(n), 4096);
    return launch_chained(press_normalize, dim3(nb), dim3(kThreads), 0, s, y, x, n, partial, kPressNormParts, norm);
}

}  // namespace drt3d
