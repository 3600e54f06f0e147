// warp_drt.cuh -- a 2^G-point multiscale transform held in one warp's
// registers.
//
// Layout: lane L holds K consecutive displacements L*K .. L*K+K-1 of every
// one of the 2^G rows, v[row][i].  Because the per-unit shear has already
// been applied by the loads, every shift of the 2^G-point transform is a
// compile-time constant: stage J pairs rows tau + (q << (J+1)) (position bit
// 0) and tau + 2^J + (q << (J+1)) (position bit 1) and writes
//     row lsb + 2 tau + (q << (J+1)) :  lo[d] + hi[d + tau + lsb]
// (eq.(map2D) restricted to the unit, slope so far tau, new slope bit lsb).
// Values that a shift pulls from beyond the lane come from the next lanes by
// shuffles; the last lanes of the warp receive stale values, so only
// positions p < 32K - (2^G - 1) of the result are valid.
//
// The adjoint stage is the transpose (eq.(invmap3Dsummation) restricted to
// the unit): row bit 0 receives out0[d] + out1[d], row bit 1 receives
// out0[d - tau] + out1[d - tau - 1]; there the first 2^G - 1 positions are
// the invalid ones.
#pragma once

#include <cstdint>

namespace drt3d {

__device__ __forceinline__ uint32_t shfl_down(uint32_t v, int d) {
    return __shfl_down_sync(0xffffffffu, v, d);
}
__device__ __forceinline__ float shfl_down(float v, int d) {
    return __shfl_down_sync(0xffffffffu, v, d);
}
__device__ __forceinline__ uint32_t shfl_up(uint32_t v, int d) {
    return __shfl_up_sync(0xffffffffu, v, d);
}
__device__ __forceinline__ float shfl_up(float v, int d) {
    return __shfl_up_sync(0xffffffffu, v, d);
}

// ZB ("zero beyond"): values pulled from past the last lane read as zero
// instead of stale, so a tile whose input is zero past its end is valid in
// every position.
template <int G, int K, int J, bool ZB = false, typename T>
__device__ __forceinline__ void fwd_stage(T (&v)[1 << G][K]) {
    constexpr int R = 1 << G;
    constexpr int HALF = 1 << J;
    T nv[R][K];
#pragma unroll
    for (int q = 0; q < (R >> (J + 1)); ++q) {
#pragma unroll
        for (int tau = 0; tau < HALF; ++tau) {
            const int a = tau + (q << (J + 1));
            const int b = a + HALF;
            // ext[p] = hi at position L*K + p for p in [0, K + tau]
            T ext[K + HALF];
#pragma unroll
            for (int i = 0; i < K; ++i) ext[i] = v[b][i];
#pragma unroll
            for (int e = 0; e < HALF; ++e)
                if (e <= tau) {
                    ext[K + e] = shfl_down(v[b][e % K], 1 + e / K);
                    if (ZB && (int)(threadIdx.x & 31) + 1 + e / K >= 32) ext[K + e] = T(0);
                }
#pragma unroll
            for (int lsb = 0; lsb < 2; ++lsb)
#pragma unroll
                for (int i = 0; i < K; ++i)
                    nv[lsb + 2 * tau + (q << (J + 1))][i] = v[a][i] + ext[i + tau + lsb];
        }
    }
#pragma unroll
    for (int r = 0; r < R; ++r)
#pragma unroll
        for (int i = 0; i < K; ++i) v[r][i] = nv[r][i];
}

// Stage 0 with the value one position past the lane's last of each odd row
// supplied by the caller (nxt[q] for row 2q + 1, read along with the row)
// instead of taken from the next lane by a shuffle.
template <int G, int K, typename T>
__device__ __forceinline__ void fwd_stage0_nxt(T (&v)[1 << G][K], const T (&nxt)[1 << (G - 1)]) {
    constexpr int R = 1 << G;
    T nv[R][K];
#pragma unroll
    for (int q = 0; q < R / 2; ++q) {
        T ext[K + 1];
#pragma unroll
        for (int i = 0; i < K; ++i) ext[i] = v[2 * q + 1][i];
        ext[K] = nxt[q];
#pragma unroll
        for (int lsb = 0; lsb < 2; ++lsb)
#pragma unroll
            for (int i = 0; i < K; ++i) nv[2 * q + lsb][i] = v[2 * q][i] + ext[i + lsb];
    }
#pragma unroll
    for (int r = 0; r < R; ++r)
#pragma unroll
        for (int i = 0; i < K; ++i) v[r][i] = nv[r][i];
}

template <int G, int K, int J = 0, bool ZB = false, typename T>
__device__ __forceinline__ void fwd_all(T (&v)[1 << G][K]) {
    if constexpr (J < G) {
        fwd_stage<G, K, J, ZB>(v);
        fwd_all<G, K, J + 1, ZB>(v);
    }
}

// Value at position L*K + i - s (s >= 0) of a row: from this lane's
// registers or, when it falls below, from a lower lane.
template <int K, typename T>
__device__ __forceinline__ T take_lower(const T (&x)[K], int i, int s) {
    const int p = i - s;
    if (p >= 0) return x[p];
    const int c = (K - 1 - p) / K;
    return shfl_up(x[p + c * K], c);
}

template <int G, int K, int J, typename T>
__device__ __forceinline__ void adj_stage(T (&v)[1 << G][K]) {
    constexpr int R = 1 << G;
    constexpr int HALF = 1 << J;
    T nv[R][K];
#pragma unroll
    for (int q = 0; q < (R >> (J + 1)); ++q) {
#pragma unroll
        for (int tau = 0; tau < HALF; ++tau) {
            const int r0 = 2 * tau + (q << (J + 1));
            const int r1 = r0 + 1;
            const int a = tau + (q << (J + 1));
            const int b = a + HALF;
#pragma unroll
            for (int i = 0; i < K; ++i) {
                nv[a][i] = v[r0][i] + v[r1][i];
                nv[b][i] = take_lower<K>(v[r0], i, tau) + take_lower<K>(v[r1], i, tau + 1);
            }
        }
    }
#pragma unroll
    for (int r = 0; r < R; ++r)
#pragma unroll
        for (int i = 0; i < K; ++i) v[r][i] = nv[r][i];
}

template <int G, int K, int J = G - 1, typename T>
__device__ __forceinline__ void adj_all(T (&v)[1 << G][K]) {
    if constexpr (J >= 0) {
        adj_stage<G, K, J>(v);
        adj_all<G, K, J - 1>(v);
    }
}

}  // namespace drt3d
