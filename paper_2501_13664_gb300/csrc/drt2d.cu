// drt2d.cu -- the 2D DRT of lines (Section 2.1, eq.(map2D)) of a batch of
// images over up to four quadrants (Section 2.2).
//
// The n stages are grouped into passes of G <= 4 stages.  A pass works on
// units (sg, w) exactly as the one-axis planes passes do (rows sg + 2^m0 v
// before the pass, new slope bits appended below the old ones after it, so
// the last pass leaves row s = the paper's slope), one warp per unit and
// tile of displacements: it loads the unit's 2^G rows sheared by sg * u, runs
// the register transform of warp_drt.cuh and stores the valid prefix.  The
// first pass reads the image through the quadrant's orientation with the
// image embedded at d in [N, 2N); later passes read the compact rows
// [base, 2N) of the previous one.  Slots are (image, quadrant) pairs of one
// chunk of images; grid.y runs over them.
#include <cstring>
#include <type_traits>

#include "internal.cuh"
#include "warp_drt.cuh"

namespace drt3d {
namespace {

constexpr int kWarps2 = 8;  // warps per block
constexpr int kK2 = 4;      // displacements per lane

template <typename TIn, typename T>
__device__ __forceinline__ T widen(TIn x) {
    if constexpr (std::is_same<T, float>::value) {
        return (T)x;
    } else {
        return (T)(int32_t)x;  // zero/sign extension into the int32 ring
    }
}

template <int B> struct VecOf;
template <> struct VecOf<2> { using type = unsigned short; };
template <> struct VecOf<4> { using type = unsigned int; };
template <> struct VecOf<8> { using type = uint2; };
template <> struct VecOf<16> { using type = uint4; };

// CNT contiguous values from p with vector loads of up to 16 bytes; p must be
// aligned to min(16, CNT * sizeof(TIn)) bytes.
template <typename TIn, int CNT>
__device__ __forceinline__ void load_run(const TIn* p, TIn (&out)[CNT]) {
    constexpr int B = CNT * (int)sizeof(TIn);
    constexpr int W = B >= 16 ? 16 : B;
    using V = typename VecOf<W>::type;
#pragma unroll
    for (int c = 0; c < B / W; ++c) {
        const V x = __ldg(reinterpret_cast<const V*>(p) + c);
        memcpy(reinterpret_cast<char*>(out) + c * W, &x, W);
    }
}

template <typename TIn, typename T, int G, bool INGEST>
__global__ void __launch_bounds__(kWarps2 * 32) drt2d_pass(const __grid_constant__ Drt2dLaunch L) {
    constexpr int K = kK2;
    constexpr int R = 1 << G;
    const int lane = threadIdx.x & 31;
    const long long w = (long long)blockIdx.x * kWarps2 + (threadIdx.x >> 5);
    if (w >= L.warps) return;
    const int slot = blockIdx.y;
    const int tile = (int)(w % L.ntiles);
    const int unit = (int)(w / L.ntiles);
    const int sg = unit & ((1 << L.m0) - 1);
    const int wq = unit >> L.m0;
    const int N = L.N, W = 2 * N;
    const int d0 = L.out_base + tile * L.V;
    const int pos0 = d0 + lane * K;

    T v[R][K];
    if constexpr (INGEST) {
        const int q = L.quad[slot % L.nq];
        const TIn* img = static_cast<const TIn*>(L.in) + (long long)(slot / L.nq) * N * N;
        if (L.vec_ingest) {
            // The first pass has m0 = 0, so sg = 0: rows a0 + u, unsheared,
            // and a lane's K displacements map to K pixels y0 .. y0 + K - 1,
            // all inside the image or all outside (y0 and N multiples of K).
            const int a0 = wq << G;
            const int y0 = pos0 - N;
            if (q & 2) {
                // f_q(u, y) = f(y or N-1-y, a0 + u): for each y the R values
                // are contiguous in image row y.
#pragma unroll
                for (int i = 0; i < K; ++i) {
                    const int y = y0 + i;
                    TIn run[R];
                    if ((unsigned)y < (unsigned)N) {
                        load_run<TIn, R>(img + (long long)((q & 1) ? N - 1 - y : y) * N + a0, run);
                    } else {
#pragma unroll
                        for (int u = 0; u < R; ++u) run[u] = TIn(0);
                    }
#pragma unroll
                    for (int u = 0; u < R; ++u) v[u][i] = widen<TIn, T>(run[u]);
                }
            } else {
                // f_q(u, y) = f(a0 + u, y or N-1-y): K contiguous values per row.
                const bool in = (unsigned)y0 < (unsigned)N;
#pragma unroll
                for (int u = 0; u < R; ++u) {
                    TIn run[K];
                    if (in) {
                        load_run<TIn, K>(img + (long long)(a0 + u) * N + ((q & 1) ? N - K - y0 : y0), run);
                    } else {
#pragma unroll
                        for (int i = 0; i < K; ++i) run[i] = TIn(0);
                    }
                    if (q & 1) {
#pragma unroll
                        for (int i = 0; i < K; ++i) v[u][i] = widen<TIn, T>(run[K - 1 - i]);
                    } else {
#pragma unroll
                        for (int i = 0; i < K; ++i) v[u][i] = widen<TIn, T>(run[i]);
                    }
                }
            }
        } else {
            // Quadrant q sees f_q(u, y): bit 1 swaps the axes, bit 0 reverses
            // the non-driving one.
            const int step_u = (q & 2) ? 1 : N;
            const int step_y = ((q & 2) ? N : 1) * ((q & 1) ? -1 : 1);
            const int y_org = (q & 1) ? (N - 1) * ((q & 2) ? N : 1) : 0;
#pragma unroll
            for (int u = 0; u < R; ++u) {
                const int a = sg + (u << L.m0) + (wq << (L.m0 + G));
                const TIn* row = img + a * step_u + y_org;
                const int y0 = pos0 + sg * u - N;
#pragma unroll
                for (int i = 0; i < K; ++i) {
                    const int y = y0 + i;
                    v[u][i] = ((unsigned)y < (unsigned)N) ? widen<TIn, T>(__ldg(row + y * step_y)) : T(0);
                }
            }
        }
    } else {
        const T* buf = static_cast<const T*>(L.in) + slot * L.in_slot - L.in_base;
#pragma unroll
        for (int u = 0; u < R; ++u) {
            const int a = sg + (u << L.m0) + (wq << (L.m0 + G));
            const T* row = buf + (long long)a * L.in_pitch;
            const int ds = pos0 + sg * u;
#pragma unroll
            for (int i = 0; i < K; ++i) {
                const int d = ds + i;
                v[u][i] = (d >= L.in_base && d < W) ? __ldg(row + d) : T(0);
            }
        }
    }

    fwd_all<G, K>(v);

    // V and every base, pitch and slot stride are multiples of 4: a lane's K
    // displacements are valid together and 16-byte aligned.
    if (lane * K >= L.V || pos0 >= W) return;
    T* out = static_cast<T*>(L.out) + slot * L.out_slot - L.out_base + pos0;
#pragma unroll
    for (int t = 0; t < R; ++t) {
        const int o = t + (sg << G) + (wq << (L.m0 + G));
        if constexpr (std::is_same<T, float>::value) {
            *reinterpret_cast<float4*>(out + (long long)o * L.out_pitch) = make_float4(v[t][0], v[t][1], v[t][2], v[t][3]);
        } else {
            *reinterpret_cast<uint4*>(out + (long long)o * L.out_pitch) = make_uint4(v[t][0], v[t][1], v[t][2], v[t][3]);
        }
    }
}

template <typename TIn, typename T, bool INGEST>
cudaError_t launch_g(const Drt2dLaunch& L, int G, int nslots, cudaStream_t s) {
    const dim3 grid((unsigned)((L.warps + kWarps2 - 1) / kWarps2), (unsigned)nslots);
    switch (G) {
    case 1: drt2d_pass<TIn, T, 1, INGEST><<<grid, kWarps2 * 32, 0, s>>>(L); break;
    case 2: drt2d_pass<TIn, T, 2, INGEST><<<grid, kWarps2 * 32, 0, s>>>(L); break;
    case 3: drt2d_pass<TIn, T, 3, INGEST><<<grid, kWarps2 * 32, 0, s>>>(L); break;
    case 4: drt2d_pass<TIn, T, 4, INGEST><<<grid, kWarps2 * 32, 0, s>>>(L); break;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

}  // namespace

int drt2d_tile_valid(int G) { return (32 * kK2 - ((1 << G) - 1)) & ~3; }

cudaError_t launch_drt2d_pass(const Drt2dLaunch& L, int G, drt3d_dtype in_dtype, bool ingest, int nslots,
                              cudaStream_t s) {
    if (!ingest)
        return in_dtype == DRT3D_F32 ? launch_g<float, float, false>(L, G, nslots, s)
                                     : launch_g<uint32_t, uint32_t, false>(L, G, nslots, s);
    switch (in_dtype) {
    case DRT3D_U8: return launch_g<uint8_t, uint32_t, true>(L, G, nslots, s);
    case DRT3D_I16: return launch_g<int16_t, uint32_t, true>(L, G, nslots, s);
    case DRT3D_I32: return launch_g<int32_t, uint32_t, true>(L, G, nslots, s);
    case DRT3D_F32: return launch_g<float, float, true>(L, G, nslots, s);
    }
    return cudaErrorInvalidValue;
}

}  // namespace drt3d
