// planes_adjoint_fused.cu -- the transpose of one fused planes pass: the
// backprojection of Section 5.1 (eq.(invmap3Dsummation)), G stages on both
// axes at a time, run in reverse pass order.
//
// A fused forward pass maps the 2^G x 2^G input rows (u1, u2) of a unit to
// its output rows (t1, t2) by
//     out[t1][t2][d] = sum_{u1,u2} in[u1][u2][d + sg1 u1 + sg2 u2
//                                            + l^G_{t1}(u1) + l^G_{t2}(u2)]
// (see planes_fused.cu), so its transpose is
//     in_bar[u1][u2][f + sg1 u1 + sg2 u2]
//         = sum_{t1} Y[t1][u2][f - l^G_{t1}(u1)],
//     Y[t1][u2][g] = sum_{t2} out_bar[t1][t2][g - l^G_{t2}(u2)],
// with both sums taken in the cotangent's frame f: the shear sg1 u1 + sg2 u2
// only moves where an output row's values land.  Reads below displacement 0
// or outside a stored row are zero, which makes it the exact transpose.
//
// One CTA holds one unit over a tile of 32 K displacements of that frame:
//   phase A: warp t1 loads the cotangent rows (t1, t2) as 16-byte vectors,
//            runs the transposed register transform (warp_drt.cuh) along
//            axis 2 and parks rows (u2, t1) in shared memory;
//   phase B: warp u2 reads rows (u2, t1), runs the transposed transform along
//            axis 1 and stores row (u1, u2) at displacement f + sg1 u1 + sg2 u2.
// The transposed transform pulls from lower lanes, so its first 2^G - 1
// positions are invalid; after both phases positions p >= PB are valid, and
// a tile stores V of them.  Tiles step by V in the cotangent frame from below
// e_lo - PB - (sg1 + sg2)(2^G - 1), so every output row is covered exactly
// once over [e_lo, 3N).  With m0 = 0 there is no shear and rows are stored as
// 16-byte vectors; otherwise the per-row offset makes them element stores.
#include <type_traits>

#include "fused_cta.cuh"

namespace drt3d {
namespace {

using namespace fused;

// First valid (stored) phase-B position, stored positions per tile, first
// phase-A position that phase B reads, and the shared-memory row width, for
// lanes of KK positions (a warp tile of 32 KK).  All are multiples of KK, so
// a lane's positions lie wholly inside or outside each range; with KK = 5
// (G <= 3: rows of up to 140 stored positions in one tile, where 4-wide
// lanes store at most 120) the stored width is also a multiple of 4, so tile
// origins stay 16-byte aligned.
template <int G, int KK> __host__ __device__ constexpr int adj_pb() {
    return KK == 4 ? (2 * ((1 << G) - 1) + 3) & ~3 : (2 * ((1 << G) - 1) + KK - 1) / KK * KK;
}
template <int G, int KK> __host__ __device__ constexpr int adj_v() {
    return KK == 4 ? (G >= 4 ? 92 : 32 * KK - adj_pb<G, KK>()) : (32 * KK - adj_pb<G, KK>()) / 20 * 20;
}
template <int G, int KK> __host__ __device__ constexpr int adj_sa() {
    return (adj_pb<G, KK>() - ((1 << G) - 1)) / KK * KK;
}
template <int G, int KK> __host__ __device__ constexpr int adj_ws() {
    return adj_pb<G, KK>() + adj_v<G, KK>() - adj_sa<G, KK>();
}

template <typename T>
__device__ __forceinline__ T from_u32(uint32_t x) {
    if constexpr (std::is_same<T, float>::value) return __uint_as_float(x);
    else return x;
}
template <typename T>
__device__ __forceinline__ uint32_t to_u32(T x) {
    if constexpr (std::is_same<T, float>::value) return __float_as_uint(x);
    else return x;
}

// Cotangent rows and tile origin of CTA (x, slot) of a launch.
struct AdjTile {
    long long o1base, o2base;  // rows o1 = o1base + t1, o2 = o2base + t2
    int d0;
};

template <int G, int KK>
__device__ __forceinline__ AdjTile adj_tile(const FusedLaunch& L, unsigned x) {
    constexpr int PB = adj_pb<G, KK>();
    const unsigned ntiles = (unsigned)L.ntiles;
    unsigned unit = x / ntiles;
    const int tile = (int)(x - unit * ntiles);
    const int m0 = L.m0, wb = L.n - m0 - G;
    const int sg1 = (int)(unit & ((1u << m0) - 1)); unit >>= m0;
    const int wq1 = (int)(unit & ((1u << wb) - 1)); unit >>= wb;
    const int sg2 = (int)(unit & ((1u << m0) - 1)); unit >>= m0;
    const int wq2 = (int)unit;
    AdjTile a;
    a.o1base = (sg1 << G) + ((long long)wq1 << (m0 + G));
    a.o2base = (sg2 << G) + ((long long)wq2 << (m0 + G));
    a.d0 = ((L.gout.base - PB - (sg1 + sg2) * ((1 << G) - 1)) & ~3) + tile * adj_v<G, KK>();
    return a;
}

template <typename T, int G, int KK>
__global__ void __launch_bounds__(32 * fused_warps<G>(), (G >= 4 ? 2 : 1))
planes_adj_fused(const __grid_constant__ FusedLaunch L) {
    pdl_wait_and_release();
    constexpr int K = KK;        // positions per lane (shadows the forward passes' 4)
    constexpr int WT = 32 * KK;  // positions per warp tile
    constexpr bool VEC = KK == 4;
    constexpr int R = 1 << G;
    constexpr int NW = fused_warps<G>();
    constexpr int GPW = R / NW > 0 ? R / NW : 1;  // row groups per warp
    constexpr int P0 = R - 1;
    constexpr int PB = adj_pb<G, KK>(), V = adj_v<G, KK>(), SA = adj_sa<G, KK>(), WS = adj_ws<G, KK>();
    static_assert(PB + V <= WT && SA + WS <= WT && (!VEC || WS % 4 == 0) && V % 4 == 0, "tile layout");
    static_assert(PB % K == 0 && SA % K == 0 && V % K == 0, "lanes wholly inside or outside each range");
    extern __shared__ __align__(16) unsigned char smem_raw[];
    uint32_t* S = reinterpret_cast<uint32_t*>(smem_raw);  // [u2][t1][WS], position p at p - SA

    const FusedSlot& sp = L.slot[launch_slot(L.reverse_slots, blockIdx.y, gridDim.y)];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const bool active = warp < NW;
    const int m0 = L.m0, N = L.N;
    const unsigned ntiles = (unsigned)L.ntiles;
    unsigned unit = blockIdx.x / ntiles;
    const int tile = (int)(blockIdx.x - unit * ntiles);
    const int wb = L.n - m0 - G;
    const int sg1 = (int)(unit & ((1u << m0) - 1)); unit >>= m0;
    const int wq1 = (int)(unit & ((1u << wb) - 1)); unit >>= wb;
    const int sg2 = (int)(unit & ((1u << m0) - 1)); unit >>= m0;
    const int wq2 = (int)unit;
    const int e_lo = L.gout.base;
    const int d0 = ((e_lo - PB - (sg1 + sg2) * P0) & ~3) + tile * V;  // tile origin, cotangent frame
    if (d0 + PB >= L.dmax) return;  // every row's first stored displacement lies past 3N
    const int p0 = lane * K;        // this lane's first position in the tile
    const bool vec_in = VEC && (L.gin.pitch & 3) == 0 && (L.gin.base & 3) == 0 && (L.dmax & 3) == 0;
    const bool vec_out = VEC && (L.gout.pitch & 3) == 0 && (e_lo & 3) == 0 && (L.dmax & 3) == 0;

    // Warm L2 with the cotangent rows of the CTA `prefetch_ahead` places later
    // in launch order (about one wave of resident CTAs): its loads then hit L2
    // instead of waiting on DRAM.  One row window per thread; a hint only.
    if (L.prefetch_ahead > 0 && (L.gin.pitch & 3) == 0 && (L.gin.base & 3) == 0 && (L.dmax & 3) == 0 &&
        threadIdx.x < R * R) {
        const unsigned long long next =
            (unsigned long long)blockIdx.y * gridDim.x + blockIdx.x + (unsigned)L.prefetch_ahead;
        const unsigned ny = (unsigned)(next / gridDim.x), nx = (unsigned)(next % gridDim.x);
        if (ny < gridDim.y) {
            const AdjTile a = adj_tile<G, KK>(L, nx);
            const int lo = max(a.d0, L.gin.base), hi = min(a.d0 + WT, L.dmax);
            if (a.d0 + PB < L.dmax && lo < hi) {
                const int t1 = threadIdx.x / R, t2 = threadIdx.x % R;
                const T* cot = static_cast<const T*>(L.slot[launch_slot(L.reverse_slots, ny, gridDim.y)].in);
                const T* rp = cot + ((a.o1base + t1) * N + a.o2base + t2) * L.gin.pitch - L.gin.base;
                tma::prefetch_l2(rp + lo, (uint32_t)(hi - lo) * 4u);
            }
        }
    }

    // ---------------- phase A: along axis 2, warp = t1 ----------------
#pragma unroll 1
    for (int gi = 0; gi < (active ? GPW : 0); ++gi) {
        const int t1 = warp + gi * NW;
        const long long o1 = t1 + (sg1 << G) + (wq1 << (m0 + G));
        const T* cot = static_cast<const T*>(sp.in);
        T v[R][K];
        const int pos = d0 + p0;
#pragma unroll
        for (int t2 = 0; t2 < R; ++t2) {
            const long long o2 = t2 + (sg2 << G) + (wq2 << (m0 + G));
            const T* rp = cot + (o1 * N + o2) * L.gin.pitch - L.gin.base;  // element d at rp[d]
            if (vec_in) {
                const bool in = pos >= L.gin.base && pos < L.dmax;
                const uint4 w = in ? __ldg(reinterpret_cast<const uint4*>(rp + pos)) : make_uint4(0u, 0u, 0u, 0u);
                const uint32_t e[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
                for (int i = 0; i < K; ++i) v[t2][i] = from_u32<T>(e[i % 4]);
            } else {
#pragma unroll
                for (int i = 0; i < K; ++i) {
                    const int d = pos + i;
                    v[t2][i] = (d >= L.gin.base && d < L.dmax) ? rp[d] : T(0);
                }
            }
        }
        adj_all<G, K>(v);  // rows t2 -> u2
        if (p0 >= SA && p0 < SA + WS) {
#pragma unroll
            for (int u2 = 0; u2 < R; ++u2) {
                uint32_t* dst = S + (u2 * R + t1) * WS + (p0 - SA);
                if constexpr (VEC) {
                    *reinterpret_cast<uint4*>(dst) =
                        make_uint4(to_u32(v[u2][0]), to_u32(v[u2][1 % K]), to_u32(v[u2][2 % K]), to_u32(v[u2][3 % K]));
                } else {
#pragma unroll
                    for (int i = 0; i < K; ++i) dst[i] = to_u32(v[u2][i]);
                }
            }
        }
    }
    __syncthreads();

    // ---------------- phase B: along axis 1, warp = u2 ----------------
    const int q = p0 >= SA && p0 < SA + WS ? p0 - SA : 0;  // lanes below SA feed only invalid positions
#pragma unroll 1
    for (int gi = 0; gi < (active ? GPW : 0); ++gi) {
        const int u2 = warp + gi * NW;
        T v[R][K];
#pragma unroll
        for (int t1 = 0; t1 < R; ++t1) {
            const uint32_t* src = S + (u2 * R + t1) * WS + q;
            if constexpr (VEC) {
                const uint4 w = *reinterpret_cast<const uint4*>(src);
                const uint32_t e[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
                for (int i = 0; i < K; ++i) v[t1][i] = from_u32<T>(e[i % 4]);
            } else {
#pragma unroll
                for (int i = 0; i < K; ++i) v[t1][i] = from_u32<T>(src[i]);
            }
        }
        adj_all<G, K>(v);  // rows t1 -> u1
        const long long a2 = sg2 + (u2 << m0) + (wq2 << (m0 + G));
        T* out = static_cast<T*>(sp.out);
        if (p0 < PB || p0 >= PB + V) continue;
        if (m0 == 0 && vec_out) {
            // no shear: the lane's four positions are one aligned vector of the row
            const int e = d0 + p0;
            if (e < e_lo || e >= L.dmax) continue;
#pragma unroll
            for (int u1 = 0; u1 < R; ++u1) {
                const long long a1 = u1 + (wq1 << G);
                T* dst = out + (a1 * N + a2) * L.gout.pitch + (e - e_lo);
                *reinterpret_cast<uint4*>(dst) =
                    make_uint4(to_u32(v[u1][0]), to_u32(v[u1][1 % K]), to_u32(v[u1][2 % K]), to_u32(v[u1][3 % K]));
            }
        } else {
#pragma unroll
            for (int u1 = 0; u1 < R; ++u1) {
                const long long a1 = sg1 + (u1 << m0) + (wq1 << (m0 + G));
                const int e0 = d0 + p0 + sg1 * u1 + sg2 * u2;
                T* row = out + (a1 * N + a2) * L.gout.pitch - e_lo;  // element e at row[e]
#pragma unroll
                for (int i = 0; i < K; ++i)
                    if (e0 + i >= e_lo && e0 + i < L.dmax) row[e0 + i] = v[u1][i];
            }
        }
    }
}

template <typename T, int G, int KK>
cudaError_t launch_adj_g(const FusedLaunch& Lin, int nslots, cudaStream_t s) {
    const size_t smem = (size_t)(1 << (2 * G)) * adj_ws<G, KK>() * 4;
    auto kern = planes_adj_fused<T, G, KK>;
    static DeviceOnce attr_done;           // per instantiation
    static std::atomic<int> wave[64] = {};  // resident CTAs of the device, written before the flag
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    if (!attr_done.done(dev)) {
        e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        int sms = 0, per = 0;
        e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (e != cudaSuccess) return e;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kern, 32 * fused_warps<G>(), smem);
        if (e != cudaSuccess) return e;
        wave[dev].store(per * sms, std::memory_order_relaxed);
        attr_done.mark(dev);
    }
    FusedLaunch L = Lin;
    L.prefetch_ahead = wave[dev].load(std::memory_order_relaxed);  // one wave ahead
    dim3 grid((unsigned)L.ctas, (unsigned)nslots);
    return launch_chained(kern, grid, dim3(32 * fused_warps<G>()), smem, s, L);
}

template <typename T>
cudaError_t launch_adj_t(const FusedLaunch& L, int G, int KK, int nslots, cudaStream_t s) {
    if (KK == 5) {
        switch (G) {
        case 2: return launch_adj_g<T, 2, 5>(L, nslots, s);
        case 3: return launch_adj_g<T, 3, 5>(L, nslots, s);
        }
        return cudaErrorInvalidValue;
    }
    switch (G) {
    case 1: return launch_adj_g<T, 1, 4>(L, nslots, s);
    case 2: return launch_adj_g<T, 2, 4>(L, nslots, s);
    case 3: return launch_adj_g<T, 3, 4>(L, nslots, s);
    case 4: return launch_adj_g<T, 4, 4>(L, nslots, s);
    }
    return cudaErrorInvalidValue;
}

}  // namespace

// Tile parameters of the fused adjoint with lanes of KK positions (4, or 5
// at G = 2, 3): stored positions per tile, and the first stored position (the
// tile origin sits that far below the first displacement it stores for the
// unshifted row).  False for an unsupported (G, KK).
bool adjoint_fused_tile(int G, int KK, int* V, int* PB) {
    if (KK == 5) {
        switch (G) {
        case 2: *V = adj_v<2, 5>(); *PB = adj_pb<2, 5>(); return true;
        case 3: *V = adj_v<3, 5>(); *PB = adj_pb<3, 5>(); return true;
        }
        return false;
    }
    if (KK != 4) return false;
    switch (G) {
    case 1: *V = adj_v<1, 4>(); *PB = adj_pb<1, 4>(); return true;
    case 2: *V = adj_v<2, 4>(); *PB = adj_pb<2, 4>(); return true;
    case 3: *V = adj_v<3, 4>(); *PB = adj_pb<3, 4>(); return true;
    case 4: *V = adj_v<4, 4>(); *PB = adj_pb<4, 4>(); return true;
    }
    return false;
}

cudaError_t launch_planes_adjoint_fused(const FusedLaunch& L, int G, int KK, bool is_float, int nslots,
                                        cudaStream_t s) {
    return is_float ? launch_adj_t<float>(L, G, KK, nslots, s) : launch_adj_t<uint32_t>(L, G, KK, nslots, s);
}

}  // namespace drt3d
