// djt.cu -- forward 3D discrete John transform of lines (Algorithm 3 per
// sector, stage map eq.(map3DJ), Section 4.1).
//
// A stage of eq.(map3DJ) sums two sub-lines: the row with position bit 0 and
// the row with bit 1 shifted by (s1 + l1, s2 + l2) in (d1, d2).  A group of
// G stages starting after m0 works on units (sg1, sg2, w) -- slopes so far
// and the remaining position bits -- with 2^G input planes u and 4^G output
// planes (t1, t2).  Unrolling eq.(digitalLine) over the G position bits gives
//     out[t1][t2][d1][d2] = sum_u in[u][d1 + sg1 u + l^G_{t1}(u)]
//                                      [d2 + sg2 u + l^G_{t2}(u)].
// For a fixed output x-slope t1 and output row d1 this is the sheared
// 2^G-point transform along d2 of the input rows taken at
// d1 + sg1 u + l^G_{t1}(u): one warp computes it in registers (warp_drt.cuh)
// for all t2 at once.
//
// Storage: after m stages a plane (d1, d2) is non-zero only on
// [N + 1 - 2^m, 2N)^2; intermediates keep a square window from base =
// (N + 1 - 2^m) rounded down to 4, pitch 2N - base.  Plane rows follow
// Algorithm 3's index split: ((S1 << m) + S2) << (n - m) | v, v the
// remaining position bits (first one lowest).  The final planes are
// J[s1][s2][d1][d2] with d1, d2 in [0, 2N) (separateS1S2: s1 + (s2 << n)).
#include "internal.cuh"
#include "warp_drt.cuh"

namespace drt3d {
namespace {

constexpr int kDjtWarps = 8;

// l^G_t(u) of eq.(digitalLine): bit G-1-i of u weighted by
// floor((floor(t / 2^i) + 1) / 2).
__device__ __forceinline__ int lline_dev(int G, int t, int u) {
    int acc = 0;
#pragma unroll
    for (int i = 0; i < 4; ++i)
        if (i < G) acc += ((u >> (G - 1 - i)) & 1) * (((t >> i) + 1) >> 1);
    return acc;
}

template <typename TIn, int G, int K, bool INGEST, bool FINAL>
__global__ void __launch_bounds__(kDjtWarps * 32)
djt_pass(const __grid_constant__ DjtLaunch L) {
    pdl_wait_and_release();
    constexpr int R = 1 << G;
    const int lane = threadIdx.x & 31;
    long long w = (long long)blockIdx.x * kDjtWarps + (threadIdx.x >> 5);
    if (w >= L.warps) return;
    const DjtSlot& sp = L.slot[blockIdx.y];
    const int N = L.N, m0 = L.m0;
    const int tile = (int)(w % L.ntiles); w /= L.ntiles;
    const int d1 = L.out_base + (int)(w % L.D1); w /= L.D1;
    const int t1 = (int)(w % R); w /= R;
    const int wb = L.n - m0 - G;
    const int wq = (int)(w & ((1LL << wb) - 1)); w >>= wb;
    const int sg2 = (int)(w & ((1LL << m0) - 1));
    const int sg1 = (int)(w >> m0);
    const int dmax = 2 * N;
    const int d2_0 = L.out_base + tile * L.V;
    const bool last = d2_0 + 32 * K >= dmax;

    uint32_t v[R][K];
#pragma unroll
    for (int u = 0; u < R; ++u) {
        const int d1i = d1 + sg1 * u + lline_dev(G, t1, u);
        const int q0 = d2_0 + sg2 * u + lane * K;
        const int vv = u + (wq << G);
        if constexpr (INGEST) {
            // Algorithm 3's embedding: plane row x' = v, (d1, d2) = (y' + N, z' + N).
            const TIn* vol = static_cast<const TIn*>(sp.in);
            const int yp = d1i - N;
            const bool rok = yp >= 0 && yp < N;
            const long long rb = sp.map.o0 + (long long)vv * sp.map.sx + (long long)(rok ? yp : 0) * sp.map.sy;
            const int z0 = q0 - N;  // z' of the lane's first element
            if (sp.map.sz == 1 || sp.map.sz == -1) {
                // z' runs along memory: one row pointer, and no per-element
                // bounds test for a lane whose K elements all lie inside
                const TIn* rp = vol + rb + (long long)z0 * sp.map.sz;
                const bool all_in = rok && z0 >= 0 && z0 + K <= N;
                if (all_in) {
                    if (sp.map.sz == 1) {
#pragma unroll
                        for (int i = 0; i < K; ++i) v[u][i] = (uint32_t)(int32_t)rp[i];
                    } else {
#pragma unroll
                        for (int i = 0; i < K; ++i) v[u][i] = (uint32_t)(int32_t)rp[-i];
                    }
                } else {
#pragma unroll
                    for (int i = 0; i < K; ++i) {
                        const bool ok = rok && z0 + i >= 0 && z0 + i < N;
                        v[u][i] = ok ? (uint32_t)(int32_t)rp[(int)sp.map.sz * i] : 0u;
                    }
                }
            } else {
#pragma unroll
                for (int i = 0; i < K; ++i) {
                    const int zp = z0 + i;
                    const bool ok = rok && zp >= 0 && zp < N;
                    v[u][i] = ok ? (uint32_t)(int32_t)vol[rb + (long long)zp * sp.map.sz] : 0u;
                }
            }
        } else {
            const uint32_t* in = static_cast<const uint32_t*>(sp.in);
            const long long row = ((long long)((sg1 << m0) + sg2) << (L.n - m0)) | vv;
            const bool rok = d1i >= L.in_base && d1i < dmax;
            const uint32_t* rp = in + row * L.in_plane + (long long)(rok ? d1i - L.in_base : 0) * L.in_pitch - L.in_base;
#pragma unroll
            for (int i = 0; i < K; ++i) {
                const int d2 = q0 + i;
                const bool ok = rok && d2 >= L.in_base && d2 < dmax;
                v[u][i] = ok ? __ldg(rp + d2) : 0u;
            }
        }
    }

    fwd_all<G, K, 0, true>(v);

    const int S1 = t1 + (sg1 << G);
    const int p0 = lane * K;
    const int vmax = last ? 32 * K : L.V;
    const int m1 = m0 + G;
#pragma unroll
    for (int t2 = 0; t2 < R; ++t2) {
        const int S2 = t2 + (sg2 << G);
        uint32_t* dst;
        if constexpr (FINAL) {
            // J[s1][s2][d1][d2], pitch 2N, displacements from 0
            dst = static_cast<uint32_t*>(sp.out) + ((long long)((S1 << L.n) + S2) * dmax + d1) * dmax + d2_0 + p0;
        } else {
            const long long row = ((long long)((S1 << m1) + S2) << (L.n - m1)) | wq;
            dst = static_cast<uint32_t*>(sp.out) + row * L.out_plane + (long long)(d1 - L.out_base) * L.out_pitch +
                  (d2_0 - L.out_base) + p0;
        }
        const bool full = K % 4 == 0 && p0 + K <= vmax && d2_0 + p0 + K <= dmax;
        if (K == 8 && full && (reinterpret_cast<uintptr_t>(dst) & 31u) == 0) {
            // a lane's eight displacements as one 32-byte store: every sector is
            // written whole by one instruction
            asm volatile("st.global.v8.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8};" ::"l"(dst), "r"(v[t2][0]),
                         "r"(v[t2][1 % K]), "r"(v[t2][2 % K]), "r"(v[t2][3 % K]), "r"(v[t2][4 % K]), "r"(v[t2][5 % K]),
                         "r"(v[t2][6 % K]), "r"(v[t2][7 % K])
                         : "memory");
        } else if (full) {
#pragma unroll
            for (int c = 0; c < K / 4; ++c) {
                uint4 x = make_uint4(v[t2][4 * c], v[t2][4 * c + 1], v[t2][4 * c + 2], v[t2][4 * c + 3]);
                *reinterpret_cast<uint4*>(dst + 4 * c) = x;
            }
        } else if (p0 + K <= vmax && d2_0 + p0 + K <= dmax) {
#pragma unroll
            for (int i = 0; i < K; ++i) dst[i] = v[t2][i];
        } else {
#pragma unroll
            for (int i = 0; i < K; ++i)
                if (p0 + i < vmax && d2_0 + p0 + i < dmax) dst[i] = v[t2][i];
        }
    }
}

template <typename TIn, int G, int K, bool INGEST, bool FINAL>
cudaError_t launch_k(const DjtLaunch& L, int nslots, cudaStream_t s) {
    const long long blocks = (L.warps + kDjtWarps - 1) / kDjtWarps;
    return launch_chained(djt_pass<TIn, G, K, INGEST, FINAL>, dim3((unsigned)blocks, (unsigned)nslots),
                          dim3(kDjtWarps * 32), 0, s, L);
}

template <typename TIn, bool INGEST, bool FINAL>
cudaError_t launch_gk(const DjtLaunch& L, int G, int K, int nslots, cudaStream_t s) {
#define DJT_CASE(g, k) \
    if (G == g && K == k) return launch_k<TIn, g, k, INGEST, FINAL>(L, nslots, s);
    DJT_CASE(1, 1) DJT_CASE(1, 2) DJT_CASE(1, 4) DJT_CASE(1, 8)
    DJT_CASE(2, 1) DJT_CASE(2, 2) DJT_CASE(2, 4) DJT_CASE(2, 8)
    DJT_CASE(3, 1) DJT_CASE(3, 2) DJT_CASE(3, 3) DJT_CASE(3, 4) DJT_CASE(3, 8)
    DJT_CASE(4, 1) DJT_CASE(4, 2) DJT_CASE(4, 4) DJT_CASE(4, 5)
#undef DJT_CASE
    return cudaErrorInvalidValue;
}

}  // namespace

// Lane width K of a DJT pass writing rows of `width` displacements: of the
// compiled widths (1, 2, 4, 5 for G = 4; 1, 2, 3, 4, 8 below), the one with
// the fewest lane positions over all tiles of a row (each tile after the
// first repeats 2^G - 1 positions), the fewer tiles (warps) on a tie.
int djt_lanes_k(int G, int width) {
    static const int k4[] = {1, 2, 4, 5};
    static const int k3[] = {1, 2, 3, 4, 8};
    const int* ks = G >= 4 ? k4 : k3;
    const int nk = G >= 4 ? 4 : 5;
    int best = ks[0], best_tiles = 0;
    long long best_cost = -1;
    for (int j = 0; j < nk; ++j) {
        const int K = ks[j];
        const int V = (32 * K - ((1 << G) - 1)) & ~3;
        if (V <= 0) continue;
        const int tiles = 32 * K >= width ? 1 : 1 + (width - 32 * K + V - 1) / V;
        const long long cost = (long long)tiles * 32 * K;
        if (best_cost < 0 || cost < best_cost || (cost == best_cost && tiles < best_tiles)) {
            best_cost = cost;
            best = K;
            best_tiles = tiles;
        }
    }
    return best;
}

cudaError_t launch_djt_pass(const DjtLaunch& L, int G, int K, drt3d_dtype in_dtype, bool ingest, bool final_,
                            int nslots, cudaStream_t s) {
    if (ingest) {
        switch (in_dtype) {
        case DRT3D_U8:
            return final_ ? launch_gk<uint8_t, true, true>(L, G, K, nslots, s)
                          : launch_gk<uint8_t, true, false>(L, G, K, nslots, s);
        case DRT3D_I16:
            return final_ ? launch_gk<int16_t, true, true>(L, G, K, nslots, s)
                          : launch_gk<int16_t, true, false>(L, G, K, nslots, s);
        case DRT3D_I32:
            return final_ ? launch_gk<int32_t, true, true>(L, G, K, nslots, s)
                          : launch_gk<int32_t, true, false>(L, G, K, nslots, s);
        default:
            return cudaErrorInvalidValue;
        }
    }
    return final_ ? launch_gk<uint32_t, false, true>(L, G, K, nslots, s)
                  : launch_gk<uint32_t, false, false>(L, G, K, nslots, s);
}

}  // namespace drt3d
