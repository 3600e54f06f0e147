// adjoint_sum.cu -- sum of the dodecants' backprojected frame volumes into
// the volume (the last step of the planes adjoint, Section 5.1).
//
// One CTA owns a C^3 cube of the volume (C = min(16, N)).  A dodecant's map
// is a signed permutation of the axes, so the cube's preimage in each frame
// is again an aligned C^3 cube.  The CTA reads it with loads that run along
// the frame's contiguous axis z', parks it in shared memory with padded
// strides (1, C + 1, C (C + 1) + 1: odd, so a warp walking along any one frame
// axis touches distinct banks), and every thread adds the elements of its
// voxels, which run along the volume's contiguous axis z.  Frame i + 1's
// cube is loaded into registers while frame i's is being added; the sum runs
// in increasing i, the order in which the dodecants were selected.
#include "adjoint_sum.cuh"

#include <cstdlib>

namespace drt3d {
namespace {

constexpr int kSumThreads = 256;

// c[a] for a in {0, 1, 2} without a runtime-indexed array (kept in registers).
__device__ __forceinline__ int pick(int a, int c0, int c1, int c2) { return a == 0 ? c0 : a == 1 ? c1 : c2; }

template <int C>
struct Cube {
    static constexpr int V = C * C * C;                              // voxels
    static constexpr int PER = (V + kSumThreads - 1) / kSumThreads;  // voxels per thread
    static constexpr int SY = C + 1;                                 // padded shared-memory strides
    static constexpr int SX = C * (C + 1) + 1;
    static constexpr int WORDS = C * SX;
};

template <typename T, int C>
__global__ void __launch_bounds__(kSumThreads)
frames_sum_kernel(const __grid_constant__ FramesSum S) {
    pdl_wait_and_release();
    using Q = Cube<C>;
    __shared__ T cube[Q::WORDS];
    const int N = S.N;
    const int nc = N / C;  // cubes per axis
    const int b = (int)blockIdx.x;
    const int cx = (b / (nc * nc)) * C, cy = ((b / nc) % nc) * C, cz = (b % nc) * C;  // volume cube origin
    const int t = (int)threadIdx.x;

    // Element e = t + 256 r of a cube is (x, y, z) = (xt + r XS, yt, zt): a
    // thread's elements differ only in x, and y, z, xt depend on t alone.
    constexpr int XS = kSumThreads / (C * C);
    static_assert(kSumThreads % (C * C) == 0, "a cube layer divides the block");
    const int xt = t / (C * C), yt = (t / C) % C, zt = t % C;
    const bool live = Q::V >= kSumThreads || t < Q::V;

    T next[Q::PER];
    auto load = [&](int i) {
        // frame cube origin (ox, oy, oz); the thread's elements along x'
        const int vx = pick(S.vaxis[i][0], cx, cy, cz), vy = pick(S.vaxis[i][1], cx, cy, cz),
                  vz = pick(S.vaxis[i][2], cx, cy, cz);
        const int ox = S.flip[i][0] ? N - C - vx : vx, oy = S.flip[i][1] ? N - C - vy : vy,
                  oz = S.flip[i][2] ? N - C - vz : vz;
        const T* F = static_cast<const T*>(S.frame[i]) + ((long long)(ox + xt) * N + (oy + yt)) * N + (oz + zt);
        const long long layer = (long long)XS * N * N;
#pragma unroll
        for (int r = 0; r < Q::PER; ++r)
            if (live) next[r] = F[r * layer];
    };

    T acc[Q::PER];
    load(0);
#pragma unroll 1
    for (int i = 0; i < S.nslots; ++i) {
        if (live) {
#pragma unroll
            for (int r = 0; r < Q::PER; ++r) cube[(xt + r * XS) * Q::SX + yt * Q::SY + zt] = next[r];
        }
        __syncthreads();
        if (i + 1 < S.nslots) load(i + 1);
        // Shared-memory offset of the thread's volume-local voxel (xt + r XS,
        // yt, zt) in frame i's cube: frame axis a holds volume axis vaxis[a]
        // (reversed when flipped), so the offset is base + r dstep, dstep the
        // step of the frame axis that holds volume x.
        int base = 0, dstep = 0;
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            const int va = S.vaxis[i][a];
            const int pa = pick(va, xt, yt, zt);
            const int st = a == 0 ? Q::SX : a == 1 ? Q::SY : 1;
            const bool f = S.flip[i][a] != 0;
            base += (f ? C - 1 - pa : pa) * st;
            if (va == 0) dstep = (f ? -st : st) * XS;
        }
        if (live) {
#pragma unroll
            for (int r = 0; r < Q::PER; ++r) {
                const T val = cube[base + r * dstep];
                acc[r] = i == 0 ? val : T(acc[r] + val);
            }
        }
        __syncthreads();
    }

    T* vol = static_cast<T*>(S.vol) + ((long long)(cx + xt) * N + (cy + yt)) * N + (cz + zt);
    if (live) {
#pragma unroll
        for (int r = 0; r < Q::PER; ++r) vol[(long long)r * XS * N * N] = acc[r];
    }
}

template <typename T>
cudaError_t launch_t(const FramesSum& S, cudaStream_t s) {
    const int C = S.N < 16 ? S.N : 16;
    const int nc = S.N / C;
    const unsigned blocks = (unsigned)nc * nc * nc;
    switch (C) {
    case 2: return launch_chained(frames_sum_kernel<T, 2>, dim3(blocks), dim3(kSumThreads), 0, s, S);
    case 4: return launch_chained(frames_sum_kernel<T, 4>, dim3(blocks), dim3(kSumThreads), 0, s, S);
    case 8: return launch_chained(frames_sum_kernel<T, 8>, dim3(blocks), dim3(kSumThreads), 0, s, S);
    case 16: return launch_chained(frames_sum_kernel<T, 16>, dim3(blocks), dim3(kSumThreads), 0, s, S);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace

void frames_sum_axes(const Affine& A, int N, int i, FramesSum* S) {
    const long long st[3] = {A.sx, A.sy, A.sz};
    for (int a = 0; a < 3; ++a) {
        const long long m = std::llabs(st[a]);
        S->vaxis[i][a] = (signed char)(m == 1 ? 2 : m == N ? 1 : 0);
        S->flip[i][a] = (signed char)(st[a] < 0);
    }
}

cudaError_t launch_frames_sum(const FramesSum& S, bool is_float, cudaStream_t s) {
    if (S.nslots < 1 || S.nslots > kMaxSlots || S.N < 2 || (S.N & (S.N - 1))) return cudaErrorInvalidValue;
    return is_float ? launch_t<float>(S, s) : launch_t<uint32_t>(S, s);
}

}  // namespace drt3d
