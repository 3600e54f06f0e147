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

// SQ: float32 final pass that also sums the squared residual (one partial
// per CTA, see fused_cta).
template <typename TIn, typename TOut, typename T, typename TS, int G, bool INGEST, bool SQ = false>
__global__ void __launch_bounds__(32 * fused_warps<G>(), (G >= 4 ? 2 : 1))
planes_fused(const __grid_constant__ FusedLaunch L) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    pdl_wait_and_release();
    const int sl = launch_slot(L.reverse_slots, blockIdx.y, gridDim.y);
    if constexpr (INGEST && G == 4 && std::is_same<TIn, uint8_t>::value && std::is_same<TS, uint16_t>::value) {
        if (!L.global_layout && !L.slot[sl].sub)  // 16-bit sums: two groups per register
            fused_cta_u8x2<TOut, G>(L, L.slot[sl], blockIdx.x, smem_raw);
        else
            fused_cta<TIn, TOut, T, TS, G, INGEST, false>(L, L.slot[sl], blockIdx.x, smem_raw);
    } else {
        fused_cta<TIn, TOut, T, TS, G, INGEST, false, false, true, SQ>(L, L.slot[sl], blockIdx.x, smem_raw);
    }
}

template <typename TIn, typename TOut, typename T, typename TS, int G, bool INGEST, bool SQ = false>
cudaError_t launch_g(const FusedLaunch& Lin, int nslots, cudaStream_t s) {
    const size_t smem = ((size_t)(1 << (2 * G)) * fused_ws<G>() + fused_pad<G>()) * sizeof(TS);
    auto kern = planes_fused<TIn, TOut, T, TS, G, INGEST, SQ>;
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
    // 32-bit buffer input read by the register loader: prefetch one wave ahead
    L.prefetch_ahead = (!INGEST && sizeof(TIn) == 4) ? wave[dev].load(std::memory_order_relaxed) : 0;
    dim3 grid((unsigned)L.ctas, (unsigned)nslots);
    return launch_chained(kern, grid, dim3(32 * fused_warps<G>()), smem, s, L);
}

// Pass over buffer rows (16-bit, or 32-bit at G = 3) with the phase-1 input
// staged by TMA: one 1-row box per (u2, u1) row window, landing in the
// group's block of phase-1 results; one mbarrier per group counts the bytes.
// T is the arithmetic type (uint32 ring or float), TIn the stored one.  At
// G = 3 four CTAs share an SM (64 registers: the 32-bit variants spill a few
// words, and still beat three CTAs at 80 registers, 1.21 -> 1.17 ms for the
// final float32 pass of 8 volumes of 128^3).
template <typename TIn, typename T, typename TOut, int G, bool SQ = false>
__global__ void __launch_bounds__(32 * fused_warps<G>(), (G >= 4 ? 2 : 4))
planes_fused_tma(const __grid_constant__ FusedLaunch L, const __grid_constant__ CUtensorMap tmap) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    __shared__ __align__(8) uint64_t mbar[1 << G];
    pdl_wait_and_release();
    // TMA destinations are kept 128-byte aligned.
    unsigned char* sm = smem_raw + ((128u - (tma::smem_u32(smem_raw) & 127u)) & 127u);
    const int sl = launch_slot(L.reverse_slots, blockIdx.y, gridDim.y);
    fused_cta<TIn, TOut, T, T, G, false, false, true, true, SQ>(L, L.slot[sl], blockIdx.x, sm, &tmap, sl, mbar);
}

template <typename TIn, typename T, typename TOut, int G, bool SQ = false>
cudaError_t launch_tma_g(const FusedLaunch& L, const CUtensorMap& map, int nslots, cudaStream_t s) {
    const size_t smem = ((size_t)(1 << G) * group_elems<TIn, G, true>() + fused_pad<G>()) * 4 + 128;
    auto kern = planes_fused_tma<TIn, T, TOut, G, SQ>;
    static DeviceOnce attr_done;  // per instantiation
    int dev = 0;
    cudaGetDevice(&dev);
    if (!attr_done.done(dev)) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        attr_done.mark(dev);
    }
    dim3 grid((unsigned)L.ctas, (unsigned)nslots);
    return launch_chained(kern, grid, dim3(32 * fused_warps<G>()), smem, s, L, map);
}

using EncodeTiledFn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                   const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                   CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

// The driver's tensor-map encoder, looked up once through the runtime.
EncodeTiledFn encode_tiled() {
    static EncodeTiledFn fn = [] {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q{};
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) !=
                cudaSuccess ||
            q != cudaDriverEntryPointSuccess)
            return (EncodeTiledFn) nullptr;
        return reinterpret_cast<EncodeTiledFn>(p);
    }();
    return fn;
}

// Shared-memory element type: 16 bits when the phase-1 results provably fit
// (first pass of a uint8 volume: sums of at most 2^G <= 16 voxels of 255).
template <typename TIn, typename TOut, typename T, bool INGEST>
cudaError_t launch_fused_t(const FusedLaunch& L, int G, int nslots, cudaStream_t s) {
    constexpr bool narrow = INGEST && std::is_same<TIn, uint8_t>::value;
    using TS = typename std::conditional<narrow, uint16_t, T>::type;
    if constexpr (std::is_same<TOut, float>::value) {
        if (L.slot[0].sq) {  // final float32 pass summing the squared residual
            switch (G) {
            case 1: return launch_g<TIn, TOut, T, TS, 1, INGEST, true>(L, nslots, s);
            case 2: return launch_g<TIn, TOut, T, TS, 2, INGEST, true>(L, nslots, s);
            case 3: return launch_g<TIn, TOut, T, TS, 3, INGEST, true>(L, nslots, s);
            case 4: return launch_g<TIn, TOut, T, TS, 4, INGEST, true>(L, nslots, s);
            }
            return cudaErrorInvalidValue;
        }
    }
    switch (G) {
    case 1: return launch_g<TIn, TOut, T, TS, 1, INGEST>(L, nslots, s);
    case 2: return launch_g<TIn, TOut, T, TS, 2, INGEST>(L, nslots, s);
    case 3: return launch_g<TIn, TOut, T, TS, 3, INGEST>(L, nslots, s);
    case 4: return launch_g<TIn, TOut, T, TS, 4, INGEST>(L, nslots, s);
    }
    return cudaErrorInvalidValue;
}

// loss[0] = 0.5 * sum of part[0 .. n): one block; thread t adds the entries
// t + j 1024 into accumulator j mod 4 (four independent chains, loads in
// flight together), then the four in order and a fixed tree over the threads
// (the same sum on every run).
constexpr int kLossThreads = 1024;
__global__ void __launch_bounds__(kLossThreads) residual_loss_sum(const double* __restrict__ part, long long n,
                                                                  double* __restrict__ loss) {
    pdl_wait_and_release();
    __shared__ double red[kLossThreads];
    double a[4] = {0.0, 0.0, 0.0, 0.0};
    for (long long i = threadIdx.x; i < n; i += 4LL * kLossThreads) {
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const long long k = i + (long long)j * kLossThreads;
            if (k < n) a[j] += part[k];
        }
    }
    red[threadIdx.x] = (a[0] + a[1]) + (a[2] + a[3]);
    __syncthreads();
#pragma unroll 1
    for (int h = kLossThreads / 2; h > 0; h >>= 1) {
        if ((int)threadIdx.x < h) red[threadIdx.x] += red[threadIdx.x + h];
        __syncthreads();
    }
    if (threadIdx.x == 0) loss[0] = 0.5 * red[0];
}

}  // namespace

cudaError_t launch_residual_loss(const double* part, long long n, double* loss, cudaStream_t s) {
    return launch_chained(residual_loss_sum, dim3(1), dim3(kLossThreads), 0, s, part, n, loss);
}

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

// 16-bit rows at G >= 3; 32-bit rows at G = 3 (at G = 4 their staging would
// outgrow two CTAs' shared memory).
bool fused_uses_tma(int G, ElemKind in_kind, bool ingest) {
    if (ingest) return false;
    if (in_kind == ElemKind::U16) return G >= 3;
    return (in_kind == ElemKind::I32 || in_kind == ElemKind::F32) && G == 3;
}

cudaError_t encode_fused_tmap(const FusedLaunch& L, const void* in_base, size_t slot_stride, int nslots,
                              int elem_bytes, CUtensorMap* map) {
    EncodeTiledFn enc = encode_tiled();
    if (!enc) return cudaErrorNotSupported;
    // 3-D view of the slots' input rows: x = displacement - base (the stored
    // width), y = row, z = slot.  Elements outside it read as zero.
    const cuuint64_t dims[3] = {(cuuint64_t)(L.dmax - L.gin.base), (cuuint64_t)L.N * L.N, (cuuint64_t)nslots};
    if (elem_bytes != 2 && elem_bytes != 4) return cudaErrorInvalidValue;
    const cuuint64_t strides[2] = {(cuuint64_t)L.gin.pitch * elem_bytes, (cuuint64_t)slot_stride};
    const cuuint32_t box[3] = {(cuuint32_t)(elem_bytes == 2 ? Stage<uint16_t>::ELEMS : Stage<uint32_t>::ELEMS), 1, 1};
    const cuuint32_t estr[3] = {1, 1, 1};
    const CUresult r = enc(map, elem_bytes == 2 ? CU_TENSOR_MAP_DATA_TYPE_UINT16 : CU_TENSOR_MAP_DATA_TYPE_UINT32, 3,
                           const_cast<void*>(in_base), dims, strides, box,
                           estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                           CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

cudaError_t launch_planes_fused_tma(const FusedLaunch& L, int G, ElemKind in_kind, ElemKind out_kind,
                                    const void* in_base, size_t slot_stride, int nslots, cudaStream_t s) {
    if (!fused_uses_tma(G, in_kind, false)) return cudaErrorInvalidValue;
    CUtensorMap map;
    const cudaError_t e = encode_fused_tmap(L, in_base, slot_stride, nslots, elem_bytes(in_kind), &map);
    if (e != cudaSuccess) return e;
    if (in_kind == ElemKind::U16) {
        const bool to16 = out_kind == ElemKind::U16;
        if (G == 3)
            return to16 ? launch_tma_g<uint16_t, uint32_t, uint16_t, 3>(L, map, nslots, s)
                        : launch_tma_g<uint16_t, uint32_t, uint32_t, 3>(L, map, nslots, s);
        return to16 ? launch_tma_g<uint16_t, uint32_t, uint16_t, 4>(L, map, nslots, s)
                    : launch_tma_g<uint16_t, uint32_t, uint32_t, 4>(L, map, nslots, s);
    }
    if (in_kind == ElemKind::F32) {
        if (out_kind != ElemKind::F32) return cudaErrorInvalidValue;
        return L.slot[0].sq ? launch_tma_g<float, float, float, 3, true>(L, map, nslots, s)
                            : launch_tma_g<float, float, float, 3>(L, map, nslots, s);
    }
    return out_kind == ElemKind::I32 ? launch_tma_g<uint32_t, uint32_t, uint32_t, 3>(L, map, nslots, s)
                                     : cudaErrorInvalidValue;
}

}  // namespace drt3d
