// planes_pass.cu -- one pass of the planes schedule (forward and adjoint).
//
// Forward pass (Algorithm 1's stage loop, G stages of eq.(map3D) along one
// axis, grouped as described in internal.cuh): one warp computes one unit
// (sg, w, j) over a tile of 32K - (2^G - 1) displacements.  It loads the
// unit's 2^G rows sheared by sg * u (zero outside the stored range, or,
// for the first pass, straight from the volume through the dodecant map with
// the volume at d in [2N, 3N)), runs the register transform of warp_drt.cuh
// and stores the valid prefix of the 2^G output rows.
//
// Adjoint pass (Section 5.1: the stage loop reversed with
// eq.(invmap3Dsummation)): the transpose of the forward pass.  It loads the
// unit's 2^G cotangent rows unsheared, runs the transposed register
// transform and stores row u shifted by sg * u.  The transpose of the first
// pass writes rows d in [2N, 3N) only: given the row geometry (base 2N,
// pitch N) it writes the dodecant's frame volume F[x'][y'][z'], which the
// caller then sums over the dodecants through their maps.
#include <type_traits>

#include "internal.cuh"
#include "warp_drt.cuh"

namespace drt3d {
namespace {

constexpr int kWarps = 4;  // warps per block
constexpr int kK = 4;      // displacements per lane

template <typename TIn, typename T>
__device__ __forceinline__ T to_acc(TIn x) {
    if constexpr (sizeof(T) == 4 && !std::is_same<T, float>::value) {
        return (T)(int32_t)x;  // zero/sign extension to the int32 ring
    } else {
        return (T)x;
    }
}

template <typename T>
__device__ __forceinline__ T from_bits(uint32_t x) {
    if constexpr (std::is_same<T, float>::value) {
        return __uint_as_float(x);
    } else {
        return (T)x;
    }
}

template <typename TIn, typename T, int G, bool INGEST>
__global__ void __launch_bounds__(kWarps * 32)
planes_fwd_pass(const __grid_constant__ PassLaunch L) {
    constexpr int K = kK;
    constexpr int R = 1 << G;
    const int lane = threadIdx.x & 31;
    const long long w = (long long)blockIdx.x * kWarps + (threadIdx.x >> 5);
    if (w >= L.warps) return;
    const SlotPtrs& sp = L.slot[blockIdx.y];
    const int tile = (int)(w % L.ntiles);
    long long unit = w / L.ntiles;
    const int sg = (int)(unit & ((1 << L.m0) - 1));
    unit >>= L.m0;
    const int wb = L.n - L.m0 - G;
    const int wq = (int)(unit & ((1 << wb) - 1));
    const int j = (int)(unit >> wb);
    const int N = L.N;
    const int d0 = L.gout.base + tile * L.V;
    const int pos0 = d0 + lane * K;

    T v[R][K];
#pragma unroll
    for (int u = 0; u < R; ++u) {
        const int a = sg + (u << L.m0) + (wq << (L.m0 + G));
        const int dsh = pos0 + sg * u;
        if constexpr (INGEST) {
            const int xp = L.axis == 0 ? a : j;
            const int yp = L.axis == 0 ? j : a;
            const TIn* vol = static_cast<const TIn*>(sp.in);
            const long long rowoff = sp.map.o0 + xp * sp.map.sx + yp * sp.map.sy;
#pragma unroll
            for (int i = 0; i < K; ++i) {
                const int z = dsh + i - 2 * N;
                v[u][i] = (z >= 0 && z < N) ? to_acc<TIn, T>(vol[rowoff + z * sp.map.sz]) : T(0);
            }
        } else {
            const T* buf = static_cast<const T*>(sp.in);
            const long long row = L.axis == 0 ? ((long long)a * N + j) : ((long long)j * N + a);
            const long long rbase = row * L.gin.pitch - L.gin.base;
#pragma unroll
            for (int i = 0; i < K; ++i) {
                const int d = dsh + i;
                v[u][i] = (d >= L.gin.base && d < L.dmax) ? buf[rbase + d] : T(0);
            }
        }
    }

    fwd_all<G, K>(v);

    T* outb = static_cast<T*>(sp.out);
#pragma unroll
    for (int t = 0; t < R; ++t) {
        const int o = t + (sg << G) + (wq << (L.m0 + G));
        const long long row = L.axis == 0 ? ((long long)o * N + j) : ((long long)j * N + o);
        const long long rbase = row * L.gout.pitch - L.gout.base;
#pragma unroll
        for (int i = 0; i < K; ++i) {
            const int p = lane * K + i;
            const int d = d0 + p;
            if (p < L.V && d < L.dmax) outb[rbase + d] = v[t][i];
        }
    }
}

// Transpose of planes_fwd_pass.  Tile positions p are in the cotangent's
// (output) frame; row u's result at p belongs to displacement
// d0 + p + sg * u of the input frame.  Valid positions are
// p in [2^G - 1, 2^G - 1 + V).  The input-frame rows produced are
// d in [gin.base, 3N).
template <typename T, int G>
__global__ void __launch_bounds__(kWarps * 32)
planes_adj_pass(const __grid_constant__ PassLaunch L) {
    constexpr int K = kK;
    constexpr int R = 1 << G;
    constexpr int P0 = R - 1;
    const int lane = threadIdx.x & 31;
    const long long w = (long long)blockIdx.x * kWarps + (threadIdx.x >> 5);
    if (w >= L.warps) return;
    const SlotPtrs& sp = L.slot[blockIdx.y];
    const int tile = (int)(w % L.ntiles);
    long long unit = w / L.ntiles;
    const int sg = (int)(unit & ((1 << L.m0) - 1));
    unit >>= L.m0;
    const int wb = L.n - L.m0 - G;
    const int wq = (int)(unit & ((1 << wb) - 1));
    const int j = (int)(unit >> wb);
    const int N = L.N;
    // Input-frame range this pass must produce.
    const int e_lo = L.gin.base;
    // Tiles start low enough that row R-1 (shifted by sg*(R-1)) still
    // reaches e_lo: d0 = e_lo - P0 - sg_max*(R-1) + tile*V.
    const int sg_max = (1 << L.m0) - 1;
    const int d0 = e_lo - P0 - sg_max * (R - 1) + tile * L.V;
    if (d0 + P0 >= L.dmax) return;                           // nothing left for any row
    if (d0 + P0 + L.V + sg * (R - 1) <= e_lo) return;        // below the range for every row
    const int pos0 = d0 + lane * K;

    T v[R][K];
    const T* cot = static_cast<const T*>(sp.in);
    static_assert(K == 4, "one 16-byte vector per lane and row");
#pragma unroll
    for (int t = 0; t < R; ++t) {
        const int o = t + (sg << G) + (wq << (L.m0 + G));
        const long long row = L.axis == 0 ? ((long long)o * N + j) : ((long long)j * N + o);
        const T* rp = cot + (row * L.gout.pitch - L.gout.base);  // element d of the row at rp[d]
        // A lane's four elements lie inside the stored row and start on a
        // 16-byte boundary whenever the tile origin is a multiple of 4 (m0 >= 2):
        // one vector load; otherwise element by element.
        if (pos0 >= L.gout.base && pos0 + K <= L.dmax && (reinterpret_cast<uintptr_t>(rp + pos0) & 15u) == 0) {
            const uint4 w = __ldg(reinterpret_cast<const uint4*>(rp + pos0));
            v[t][0] = from_bits<T>(w.x);
            v[t][1] = from_bits<T>(w.y);
            v[t][2] = from_bits<T>(w.z);
            v[t][3] = from_bits<T>(w.w);
        } else {
#pragma unroll
            for (int i = 0; i < K; ++i) {
                const int d = pos0 + i;
                v[t][i] = (d >= L.gout.base && d < L.dmax) ? rp[d] : T(0);
            }
        }
    }

    adj_all<G, K>(v);

#pragma unroll
    for (int u = 0; u < R; ++u) {
        const int a = sg + (u << L.m0) + (wq << (L.m0 + G));
#pragma unroll
        for (int i = 0; i < K; ++i) {
            const int p = lane * K + i;
            const int e = d0 + p + sg * u;
            const bool ok = p >= P0 && p < P0 + L.V && e >= e_lo && e < L.dmax;
            T* buf = static_cast<T*>(sp.out);
            const long long row = L.axis == 0 ? ((long long)a * N + j) : ((long long)j * N + a);
            if (ok) buf[row * L.gin.pitch + (e - L.gin.base)] = v[u][i];
        }
    }
}

template <typename TIn, typename T, bool INGEST>
cudaError_t fwd_dispatch(const PassLaunch& L, int G, int nslots, cudaStream_t s) {
    const long long blocks = (L.warps + kWarps - 1) / kWarps;
    dim3 grid((unsigned)blocks, (unsigned)nslots);
    switch (G) {
    case 1: planes_fwd_pass<TIn, T, 1, INGEST><<<grid, kWarps * 32, 0, s>>>(L); break;
    case 2: planes_fwd_pass<TIn, T, 2, INGEST><<<grid, kWarps * 32, 0, s>>>(L); break;
    case 3: planes_fwd_pass<TIn, T, 3, INGEST><<<grid, kWarps * 32, 0, s>>>(L); break;
    case 4: planes_fwd_pass<TIn, T, 4, INGEST><<<grid, kWarps * 32, 0, s>>>(L); break;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

template <typename T>
cudaError_t adj_dispatch(const PassLaunch& L, int G, int nslots, cudaStream_t s) {
    const long long blocks = (L.warps + kWarps - 1) / kWarps;
    dim3 grid((unsigned)blocks, (unsigned)nslots);
    switch (G) {
    case 1: planes_adj_pass<T, 1><<<grid, kWarps * 32, 0, s>>>(L); break;
    case 2: planes_adj_pass<T, 2><<<grid, kWarps * 32, 0, s>>>(L); break;
    case 3: planes_adj_pass<T, 3><<<grid, kWarps * 32, 0, s>>>(L); break;
    case 4: planes_adj_pass<T, 4><<<grid, kWarps * 32, 0, s>>>(L); break;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

}  // namespace

int planes_pass_lanes_k() { return kK; }

cudaError_t launch_planes_pass(const PassLaunch& L, int G, drt3d_dtype in_dtype, bool ingest,
                               bool is_float, int nslots, cudaStream_t s) {
    if (!ingest) {
        return is_float ? fwd_dispatch<float, float, false>(L, G, nslots, s)
                        : fwd_dispatch<uint32_t, uint32_t, false>(L, G, nslots, s);
    }
    switch (in_dtype) {
    case DRT3D_U8: return fwd_dispatch<uint8_t, uint32_t, true>(L, G, nslots, s);
    case DRT3D_I16: return fwd_dispatch<int16_t, uint32_t, true>(L, G, nslots, s);
    case DRT3D_I32: return fwd_dispatch<int32_t, uint32_t, true>(L, G, nslots, s);
    case DRT3D_F32: return fwd_dispatch<float, float, true>(L, G, nslots, s);
    }
    return cudaErrorInvalidValue;
}

cudaError_t launch_planes_adjoint_pass(const PassLaunch& L, int G, bool is_float, int nslots, cudaStream_t s) {
    return is_float ? adj_dispatch<float>(L, G, nslots, s) : adj_dispatch<uint32_t>(L, G, nslots, s);
}

}  // namespace drt3d
