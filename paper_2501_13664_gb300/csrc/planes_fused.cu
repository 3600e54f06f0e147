// planes_fused.cu -- forward planes pass applying G stages of eq.(map3D)
// along both axes in one CTA (Algorithm 1's stage loop, G stages at a time).
//
// A unit is (sg1, w1, sg2, w2): slope-so-far and remaining position bits on
// the two axes (see internal.cuh).  Its 2^G x 2^G input rows (u1, u2) map to
// 2^G x 2^G output rows (t1, t2) by
//     out[t1][t2][d] = sum_{u1,u2} in[u1][u2][d + sg1 u1 + sg2 u2
//                                             + l^G_{t1}(u1) + l^G_{t2}(u2)],
// which is separable: a 2^G-point transform along axis 1 for every u2,
// then one along axis 2 for every t1.  One CTA holds one unit over a tile of
// 32*K displacements:
//   phase 1: warp u2 loads rows (u1, u2) sheared by sg2 u2 + sg1 u1, runs the
//            register transform along axis 1 and parks its 2^G result rows
//            t1 in shared memory (tile origin d0 + sg2 u2);
//   phase 2: warp t1 reads rows (t1, u2) from shared memory -- already
//            sheared by sg2 u2 -- runs the transform along axis 2 and stores
//            rows (t1, t2) for the first V = 32K - 2(2^G - 1) displacements.
// The first pass reads the volume through the dodecant map with the volume at
// d in [2N, 3N) (Algorithm 1's embedding), using aligned vector loads: either
// the frame's d axis z' is contiguous in memory (dodecants 0-3), or the
// 2^G-row block of the phase-1 axis is (the others; the host swaps the axis
// order per dodecant so that this holds -- the two half-stage axes commute).
#include <type_traits>

#include "fused_cta.cuh"

namespace drt3d {
namespace {

using namespace fused;

template <typename TIn, typename TOut, typename T, typename TS, int G, bool INGEST>
__global__ void __launch_bounds__(32 * fused_warps<G>(), (G >= 4 ? 2 : 1))
planes_fused(const __grid_constant__ FusedLaunch L) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    fused_cta<TIn, TOut, T, TS, G, INGEST, false>(L, L.slot[blockIdx.y], blockIdx.x, smem_raw);
}

template <typename TIn, typename TOut, typename T, typename TS, int G, bool INGEST>
cudaError_t launch_g(const FusedLaunch& L, int nslots, cudaStream_t s) {
    const size_t smem = ((size_t)(1 << (2 * G)) * fused_ws<G>() + K) * sizeof(TS);
    auto kern = planes_fused<TIn, TOut, T, TS, G, INGEST>;
    static unsigned long long attr_done = 0;  // per instantiation, one bit per device
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev >= 64 || !((attr_done >> dev) & 1ull)) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        if (dev < 64) attr_done |= 1ull << dev;
    }
    dim3 grid((unsigned)L.ctas, (unsigned)nslots);
    kern<<<grid, 32 * fused_warps<G>(), smem, s>>>(L);
    return cudaGetLastError();
}

// Shared-memory element type: 16 bits when the phase-1 results provably fit
// (first pass of a uint8 volume: sums of at most 2^G <= 16 voxels of 255).
template <typename TIn, typename TOut, typename T, bool INGEST>
cudaError_t launch_fused_t(const FusedLaunch& L, int G, int nslots, cudaStream_t s) {
    constexpr bool narrow = INGEST && std::is_same<TIn, uint8_t>::value;
    using TS = typename std::conditional<narrow, uint16_t, T>::type;
    switch (G) {
    case 1: return launch_g<TIn, TOut, T, TS, 1, INGEST>(L, nslots, s);
    case 2: return launch_g<TIn, TOut, T, TS, 2, INGEST>(L, nslots, s);
    case 3: return launch_g<TIn, TOut, T, TS, 3, INGEST>(L, nslots, s);
    case 4: return launch_g<TIn, TOut, T, TS, 4, INGEST>(L, nslots, s);
    }
    return cudaErrorInvalidValue;
}

}  // namespace

int fused_lanes_k() { return K; }
int fused_valid(int G) {
    switch (G) {
    case 1: return fused_v<1>();
    case 2: return fused_v<2>();
    case 3: return fused_v<3>();
    default: return fused_v<4>();
    }
}

// in_kind / out_kind: element type read / written (see ElemKind).
cudaError_t launch_planes_fused(const FusedLaunch& L, int G, ElemKind in_kind, ElemKind out_kind,
                                bool ingest, int nslots, cudaStream_t s) {
    const bool fl = out_kind == ElemKind::F32;
    if (fl) {
        if (ingest) return launch_fused_t<float, float, float, true>(L, G, nslots, s);
        return launch_fused_t<float, float, float, false>(L, G, nslots, s);
    }
    if (ingest) {
        switch (in_kind) {
        case ElemKind::U8:
            return out_kind == ElemKind::U16 ? launch_fused_t<uint8_t, uint16_t, uint32_t, true>(L, G, nslots, s)
                                             : launch_fused_t<uint8_t, uint32_t, uint32_t, true>(L, G, nslots, s);
        case ElemKind::I16: return launch_fused_t<int16_t, uint32_t, uint32_t, true>(L, G, nslots, s);
        case ElemKind::I32: return launch_fused_t<int32_t, uint32_t, uint32_t, true>(L, G, nslots, s);
        default: return cudaErrorInvalidValue;
        }
    }
    if (in_kind == ElemKind::U16) {
        return out_kind == ElemKind::U16 ? launch_fused_t<uint16_t, uint16_t, uint32_t, false>(L, G, nslots, s)
                                         : launch_fused_t<uint16_t, uint32_t, uint32_t, false>(L, G, nslots, s);
    }
    if (in_kind == ElemKind::I32) {
        return out_kind == ElemKind::U16 ? cudaErrorInvalidValue
                                         : launch_fused_t<uint32_t, uint32_t, uint32_t, false>(L, G, nslots, s);
    }
    return cudaErrorInvalidValue;
}

}  // namespace drt3d
