// drt2d.cu -- the 2D DRT of lines (Section 2.1, eq.(map2D)) of a batch of
// images over up to four quadrants (Section 2.2).
//
// The n stages are grouped into passes of G <= 4 stages.  A pass works on
// units (sg, w) with the row numbering of internal.cuh (rows sg + 2^m0 v
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
    pdl_wait_and_release();
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
    case 1: return launch_chained(drt2d_pass<TIn, T, 1, INGEST>, grid, dim3(kWarps2 * 32), 0, s, L);
    case 2: return launch_chained(drt2d_pass<TIn, T, 2, INGEST>, grid, dim3(kWarps2 * 32), 0, s, L);
    case 3: return launch_chained(drt2d_pass<TIn, T, 3, INGEST>, grid, dim3(kWarps2 * 32), 0, s, L);
    case 4: return launch_chained(drt2d_pass<TIn, T, 4, INGEST>, grid, dim3(kWarps2 * 32), 0, s, L);
    default: return cudaErrorInvalidValue;
    }
}

// Whole transform of one (image, quadrant) per CTA, for uint8 images with
// N = 2^(G1 + G2) <= 256 and a two-group schedule.  Every partial sum is at
// most N * 255 <= 65280, so the first group's output rows -- N rows over
// [base1, 2N) -- stay in shared memory as 16-bit values; the second group
// reads them back and writes the final rows.  Warp work items are (unit,
// tile) pairs of each group, exactly as in drt2d_pass.
template <int G1, int G2, int NW>
__global__ void __launch_bounds__(NW * 32, NW >= 16 ? 1 : 2) drt2d_fused(const __grid_constant__ Drt2dLaunch L) {
    pdl_wait_and_release();
    constexpr int K = kK2;
    constexpr int R1 = 1 << G1, R2 = 1 << G2;
    constexpr int N = R1 * R2, W = 2 * N;
    constexpr int base1 = (N + 1 - R1) & ~3;  // nothing below is non-zero after G1 stages
    constexpr int W1 = W - base1;
    constexpr int P1 = (W1 + 7) & ~7;         // 16-byte rows
    constexpr int V1 = (32 * K - (R1 - 1)) & ~3, T1 = (W1 + V1 - 1) / V1;
    constexpr int V2 = (32 * K - (R2 - 1)) & ~3, T2 = (W + V2 - 1) / V2;
    extern __shared__ __align__(16) uint16_t rows1[];  // [N][P1], element d at d - base1
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int slot = blockIdx.x;
    const int q = L.quad[slot % L.nq];
    const uint8_t* img = static_cast<const uint8_t*>(L.in) + (long long)(slot / L.nq) * N * N;

    // ---- group 1: G1 stages from the image (sg = 0: rows a0 + u, unsheared)
#pragma unroll 1
    for (int it = warp; it < (N / R1) * T1; it += NW) {
        const int wq = it / T1, tile = it - wq * T1;
        const int pos0 = base1 + tile * V1 + lane * K;
        const int a0 = wq * R1;
        const int y0 = pos0 - N;  // a multiple of K, as N is: all K pixels in or all out
        uint32_t v[R1][K];
        if (q & 2) {
#pragma unroll
            for (int i = 0; i < K; ++i) {
                const int y = y0 + i;
                uint8_t run[R1];
                if ((unsigned)y < (unsigned)N) {
                    load_run<uint8_t, R1>(img + ((q & 1) ? N - 1 - y : y) * N + a0, run);
                } else {
#pragma unroll
                    for (int u = 0; u < R1; ++u) run[u] = 0;
                }
#pragma unroll
                for (int u = 0; u < R1; ++u) v[u][i] = run[u];
            }
        } else {
            const bool in = (unsigned)y0 < (unsigned)N;
#pragma unroll
            for (int u = 0; u < R1; ++u) {
                uint8_t run[K];
                if (in) {
                    load_run<uint8_t, K>(img + (a0 + u) * N + ((q & 1) ? N - K - y0 : y0), run);
                } else {
#pragma unroll
                    for (int i = 0; i < K; ++i) run[i] = 0;
                }
                if (q & 1) {
#pragma unroll
                    for (int i = 0; i < K; ++i) v[u][i] = run[K - 1 - i];
                } else {
#pragma unroll
                    for (int i = 0; i < K; ++i) v[u][i] = run[i];
                }
            }
        }
        fwd_all<G1, K>(v);
        if (lane * K < V1 && pos0 < W) {
#pragma unroll
            for (int t = 0; t < R1; ++t) {
                const uint2 w = make_uint2(v[t][0] | (v[t][1] << 16), v[t][2] | (v[t][3] << 16));
                *reinterpret_cast<uint2*>(rows1 + (a0 + t) * P1 + (pos0 - base1)) = w;
            }
        }
    }
    __syncthreads();

    // ---- group 2: G2 stages, slopes so far sg < R1, rows sg + u R1 sheared by sg u
    uint32_t* out = static_cast<uint32_t*>(L.out) + (long long)slot * N * W;
#pragma unroll 1
    for (int it = warp; it < R1 * T2; it += NW) {
        const int sg = it / T2, tile = it - sg * T2;
        const int pos0 = tile * V2 + lane * K;
        uint32_t v[R2][K];
#pragma unroll
        for (int u = 0; u < R2; ++u) {
            const uint16_t* row = rows1 + (sg + u * R1) * P1 - base1;
            const int ds = pos0 + sg * u;
#pragma unroll
            for (int i = 0; i < K; ++i) {
                const int d = ds + i;
                v[u][i] = (d >= base1 && d < W) ? (uint32_t)row[d] : 0u;
            }
        }
        fwd_all<G2, K>(v);
        if (lane * K < V2 && pos0 < W) {
#pragma unroll
            for (int t = 0; t < R2; ++t)
                *reinterpret_cast<uint4*>(out + (long long)(t + (sg << G2)) * W + pos0) =
                    make_uint4(v[t][0], v[t][1], v[t][2], v[t][3]);
        }
    }
}

template <int G1, int G2, int NW>
cudaError_t launch_fused2(const Drt2dLaunch& L, int nslots, cudaStream_t s) {
    constexpr int N = 1 << (G1 + G2);
    constexpr int base1 = (N + 1 - (1 << G1)) & ~3;
    constexpr int P1 = (2 * N - base1 + 7) & ~7;
    constexpr size_t smem = (size_t)N * P1 * 2;
    auto kern = drt2d_fused<G1, G2, NW>;
    if (smem > 48 * 1024) {
        static DeviceOnce attr_done;  // per instantiation
        int dev = 0;
        cudaGetDevice(&dev);
        if (!attr_done.done(dev)) {
            const cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            if (e != cudaSuccess) return e;
            attr_done.mark(dev);
        }
    }
    return launch_chained(kern, dim3((unsigned)nslots), dim3(NW * 32), smem, s, L);
}

}  // namespace

bool drt2d_fused_supported(int N, drt3d_dtype dtype) {
    return dtype == DRT3D_U8 && N >= 32 && N <= 256;
}

cudaError_t launch_drt2d_fused(const Drt2dLaunch& L, int nslots, cudaStream_t s) {
    switch (L.N) {
    case 32: return launch_fused2<3, 2, 8>(L, nslots, s);
    case 64: return launch_fused2<3, 3, 8>(L, nslots, s);
    case 128: return launch_fused2<4, 3, 8>(L, nslots, s);
    case 256: return launch_fused2<4, 4, 16>(L, nslots, s);
    }
    return cudaErrorInvalidValue;
}

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
