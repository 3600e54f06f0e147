// djt_adjoint.cu -- adjoint (backprojection) of the 3D DJT of lines
// (eq.(invmap3DJsummation): Algorithm 3's stage loop reversed), integer.
//
// Stage m + 1 -> m undoes one stage of eq.(map3DJ) as a transpose.  In the
// row layout of the forward kernels (row ((S1 << m) + S2) << (n - m) | v,
// plane window [base_m, 2N)^2), the forward stage is
//     out[(2 S1 + t1, 2 S2 + t2, w)][d1][d2] = in[(S1, S2, 2w)][d1][d2]
//                        + in[(S1, S2, 2w + 1)][d1 + S1 + t1][d2 + S2 + t2],
// so its transpose gathers, for every stage-m row pair,
//     in_bar[(S1, S2, 2w)][e1][e2]     = sum_{t1,t2} out_bar[(2S1+t1, 2S2+t2, w)][e1][e2]
//     in_bar[(S1, S2, 2w + 1)][e1][e2] = sum_{t1,t2} out_bar[...][e1 - S1 - t1][e2 - S2 - t2]
// with out_bar zero outside its window.  Only the window of stage m is
// computed: the forward never writes outside it, so nothing else can reach
// the volume.  Stage 0's window [N, 2N)^2 is the sector-frame volume; a last
// kernel sums the selected sectors' frame volumes back into the original
// frame voxel by voxel (a gather: no atomics, a fixed sector order).
#include "internal.cuh"

namespace drt3d {
namespace {

constexpr int kAdjK = 4;      // displacements per lane
constexpr int kAdjWarps = 8;

__global__ void __launch_bounds__(kAdjWarps * 32) djt_adj_stage(const __grid_constant__ DjtAdjLaunch L) {
    pdl_wait_and_release();
    const int lane = threadIdx.x & 31;
    long long w = (long long)blockIdx.x * kAdjWarps + (threadIdx.x >> 5);
    if (w >= L.items) return;
    const int n = L.n, m = L.m, N = L.N;
    const int dmax = 2 * N;
    const int tile = (int)(w % L.ntiles); w /= L.ntiles;
    const int e1 = L.out_base + (int)(w % L.D1); w /= L.D1;
    const int wb = n - m - 1;
    const int wq = (int)(w & ((1LL << wb) - 1)); w >>= wb;
    const int sg2 = (int)(w & ((1LL << m) - 1));
    const int sg1 = (int)(w >> m);
    const int e2 = L.out_base + tile * 32 * kAdjK + lane * kAdjK;
    if (e2 >= dmax) return;

    const uint32_t* in = L.in[blockIdx.y];
    uint32_t a0[kAdjK] = {0u, 0u, 0u, 0u}, a1[kAdjK] = {0u, 0u, 0u, 0u};
#pragma unroll
    for (int t1 = 0; t1 < 2; ++t1)
#pragma unroll
        for (int t2 = 0; t2 < 2; ++t2) {
            const long long orow = ((long long)(((2 * sg1 + t1) << (m + 1)) + (2 * sg2 + t2)) << wb) | wq;
            const uint32_t* P = in + orow * L.in_plane;
            // bit 0: unshifted (e1, e2 lie inside the larger window of stage m + 1)
            const uint4 u = __ldg(reinterpret_cast<const uint4*>(P + (long long)(e1 - L.in_base) * L.in_pitch +
                                                                  (e2 - L.in_base)));
            a0[0] += u.x; a0[1] += u.y; a0[2] += u.z; a0[3] += u.w;
            // bit 1: shifted back by (S1 + t1, S2 + t2)
            const int r1 = e1 - sg1 - t1;
            if (r1 >= L.in_base) {
                const uint32_t* row = P + (long long)(r1 - L.in_base) * L.in_pitch - L.in_base;
#pragma unroll
                for (int i = 0; i < kAdjK; ++i) {
                    const int c = e2 + i - sg2 - t2;
                    if (c >= L.in_base) a1[i] += __ldg(row + c);
                }
            }
        }
    uint32_t* out = L.out[blockIdx.y];
    const long long r0 = ((long long)((sg1 << m) + sg2) << (n - m)) | (2 * wq);
    uint32_t* d0 = out + r0 * L.out_plane + (long long)(e1 - L.out_base) * L.out_pitch + (e2 - L.out_base);
    uint32_t* d1 = d0 + L.out_plane;  // row 2w + 1 follows row 2w
    *reinterpret_cast<uint4*>(d0) = make_uint4(a0[0], a0[1], a0[2], a0[3]);
    *reinterpret_cast<uint4*>(d1) = make_uint4(a1[0], a1[1], a1[2], a1[3]);
}

// Original-frame voxel (x0, x1, x2) = sum over the selected sectors of the
// sector-frame volume at (x', y', z'): x' = x_a, y' = x_b (reversed by flip
// bit 0), z' = x_c (reversed by flip bit 1), (a, b, c) cyclic from the
// sector's driving axis a.  The frame volume is stage 0's row x' at
// displacements (N + y', N + z') of its window.
__global__ void __launch_bounds__(256) djt_adj_gather(const __grid_constant__ DjtAdjGather L) {
    pdl_wait_and_release();
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const int N = L.N;
    const long long NN = (long long)N * N;
    if (i >= NN * N) return;
    const int X[3] = {(int)(i / NN), (int)((i / N) % N), (int)(i % N)};
    uint32_t acc = 0u;
    for (int s = 0; s < L.nslots; ++s) {
        const int k = L.sector[s];
        const int a = k >> 2, b = (a + 1) % 3, c = (a + 2) % 3;
        const int xp = X[a];
        const int yp = (k & 1) ? N - 1 - X[b] : X[b];
        const int zp = (k & 2) ? N - 1 - X[c] : X[c];
        acc += __ldg(L.frame[s] + ((long long)xp * L.pitch + (N + yp - L.base)) * L.pitch + (N + zp - L.base));
    }
    L.out[i] = (int32_t)acc;
}

}  // namespace

cudaError_t launch_djt_adj_stage(const DjtAdjLaunch& L, int nslots, cudaStream_t s) {
    const long long blocks = (L.items + kAdjWarps - 1) / kAdjWarps;
    return launch_chained(djt_adj_stage, dim3((unsigned)blocks, (unsigned)nslots), dim3(kAdjWarps * 32), 0, s, L);
}

cudaError_t launch_djt_adj_gather(const DjtAdjGather& L, cudaStream_t s) {
    const long long total = (long long)L.N * L.N * L.N;
    return launch_chained(djt_adj_gather, dim3((unsigned)((total + 255) / 256)), dim3(256), 0, s, L);
}

int djt_adj_lanes_k() { return kAdjK; }

}  // namespace drt3d
