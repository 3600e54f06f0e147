// planes_inverse.cu -- exact integer inverse of one dodecant's planes
// transform.
//
// The paper's own inverse is iterative (Section 5.2).  This one follows from
// the stage map eq.(map3D) and Algorithm 1's zero embedding: a stage is a
// half-stage along s1 followed by one along s2, and a half-stage with
// slope-so-far S and new bit l maps the position pair (lo, hi) to
//     out_l[d] = lo[d] + hi[d + S + l],       hi[d] = 0 for d >= 3N.
// With Delta = out_1 - out_0 and the suffix sum
//     T[i] = sum_{i <= i' <= 3N-1-S} Delta[i']
// the pair is recovered as
//     hi[e] = -T[e - S]  (e >= S; 0 below),  lo[d] = out_0[d] + T[d],
// and data in the range of the forward map has Delta[i] = 0 for
// i > 3N-1-S and, after the last stage, zeros outside d in [2N, 3N).  All
// arithmetic is modulo 2^32.
//
// One CTA undoes a group of G half-stages along one axis for one unit: the
// unit's 2^G rows over the whole stored displacement range sit in shared
// memory, each of the 2^(G-1) pairs of a stage is one warp, and the suffix
// sum of a segment of up to 1024 displacements is a register suffix sum over
// each lane's contiguous chunk plus one warp shuffle scan of the chunk totals.
// Recovered pairs overwrite the slots of the rows they came from.
#include "internal.cuh"

namespace drt3d {
namespace {

constexpr int kInvWarps = 8;

__device__ __forceinline__ void flag(int* status, int code) {
    if (*status == 0) atomicCAS(status, 0, code);
}

// Shared rows are stored in chunks of 32 displacements with one pad word per
// chunk: element i of a row sits at (i / 32) * 33 + i % 32.  Lane L owns
// chunk L during a scan, so "element k of every lane's chunk" falls on 32
// distinct banks, and the lane-consecutive element i = lane + 32 * c used for
// copies lands on consecutive words of chunk c.
constexpr int kCh = 32;
constexpr int kCs = 33;
constexpr int kMaxChunks = 32;  // rows of up to 1024 displacements per segment

// T is stored with a prefix of kPre chunks below index 0 holding the values
// hi reads there: T[0] for displacements >= 0, 0 below (kPre * 32 >= the
// largest slope-so-far S of any half-stage, N/2 - 1 <= 511).
constexpr int kPre = 16;

template <int G>
__global__ void __launch_bounds__(kInvWarps * 32, 2)
planes_inv_pass(const __grid_constant__ InvLaunch L) {
    constexpr int R = 1 << G;
    constexpr int PAIRS = R / 2;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int W = L.dmax - L.gin.base;   // stored row length of the input geometry
    const int NC = (W + kCh - 1) / kCh;  // chunks per row
    const int WS = NC * kCs;
    const int TS = (NC + kPre) * kCs;    // per-pair T buffer with its prefix
    uint32_t* rows = reinterpret_cast<uint32_t*>(smem_raw);  // [R][WS]
    uint32_t* scan = rows + R * WS;                          // [PAIRS][TS]
    __shared__ int slot[R];

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int N = L.N, m0 = L.m0;
    unsigned unit = blockIdx.x;
    const int sg = (int)(unit & ((1u << m0) - 1)); unit >>= m0;
    const int wb = L.n - m0 - G;
    const int wq = (int)(unit & ((1u << wb) - 1));
    const int j = (int)(unit >> wb);
    const long long rs_axis = L.axis == 0 ? N : 1;   // row stride of the undone axis
    const long long rs_other = L.axis == 0 ? 1 : N;

    // Load the unit's output rows o(t) = t + (sg << G) + (w << (m0 + G)),
    // zero-padding the last chunk.
    const uint32_t* in = static_cast<const uint32_t*>(L.in);
    for (int t = warp; t < R; t += kInvWarps) {
        const long long row = (long long)(t + (sg << G) + (wq << (m0 + G))) * rs_axis + (long long)j * rs_other;
        const uint32_t* src = in + row * L.gin.pitch + lane;
        uint32_t* dst = rows + t * WS + lane;
        for (int c0 = 0; c0 < NC; c0 += 16) {
            uint32_t v[16];
#pragma unroll
            for (int c = 0; c < 16; ++c)
                v[c] = (c0 + c) * kCh + lane < W ? __ldg(src + (c0 + c) * kCh) : 0u;
#pragma unroll
            for (int c = 0; c < 16; ++c)
                if (c0 + c < NC) dst[(c0 + c) * kCs] = v[c];
        }
    }
    if (threadIdx.x < R) slot[threadIdx.x] = threadIdx.x;
    __syncthreads();

    const int base = L.gin.base;
    const int top = L.dmax;  // 3N
    // Rows whose length is a whole number of chunks need no masking at all.
    const bool whole = (W & (kCh - 1)) == 0;
#pragma unroll 1
    for (int J = G - 1; J >= 0; --J) {
        const int half = 1 << J;
        if (warp < PAIRS) {
            const int q = warp >> J, tau = warp & (half - 1);
            const int r0 = 2 * tau + (q << (J + 1));      // rows of stage J+1 (within the unit)
            const int S = (sg << J) + tau;                 // slope so far at global stage m0 + J
            uint32_t* o0 = rows + slot[r0] * WS;
            uint32_t* o1 = rows + slot[r0 + 1] * WS;
            uint32_t* T = scan + warp * TS + kPre * kCs;   // T[0] after the prefix
            const int lim = top - 1 - S - base;            // last stored index with a free Delta
            // Data in the range has Delta = 0 past lim; check it there (the
            // scan below does not mask it: for such data masking changes
            // nothing, and other data is reported and left undefined).
            bool bad = false;
            for (int i = lim + 1 + lane; i < W; i += 32) bad |= o1[(i >> 5) * kCs + (i & 31)] != o0[(i >> 5) * kCs + (i & 31)];
            if (__any_sync(0xffffffffu, bad) && lane == 0) flag(L.status, DRT3D_ERR_NOT_IN_RANGE);
            uint32_t seg_carry = 0;
            // Segments of kMaxChunks chunks from the top; lane L owns chunk
            // seg * 32 + L of the segment.
            const int nseg = (NC + kMaxChunks - 1) / kMaxChunks;
#pragma unroll 1
            for (int sgm = nseg - 1; sgm >= 0; --sgm) {
                const int c = sgm * kMaxChunks + lane;
                const bool live = c < NC;
                uint32_t* p0 = o0 + (live ? c : 0) * kCs;
                uint32_t* p1 = o1 + (live ? c : 0) * kCs;
                uint32_t a[kCh], x[kCh];
#pragma unroll
                for (int k = 0; k < kCh; ++k) {
                    a[k] = p0[k];
                    x[k] = live ? p1[k] - a[k] : 0u;
                }
#pragma unroll
                for (int k = kCh - 2; k >= 0; --k) x[k] += x[k + 1];
                const uint32_t tot = x[0];
                uint32_t y = tot;
#pragma unroll
                for (int off = 1; off < 32; off <<= 1) {
                    const uint32_t z = __shfl_down_sync(0xffffffffu, y, off);
                    if (lane + off < 32) y += z;
                }
                const uint32_t carry = y - tot + seg_carry;
                if (live) {
                    uint32_t* pt = T + c * kCs;
#pragma unroll
                    for (int k = 0; k < kCh; ++k) {
                        const uint32_t t = x[k] + carry;
                        pt[k] = t;
                        p0[k] = a[k] + t;  // lo[d] = out0[d] + T[d]
                    }
                }
                seg_carry += __shfl_sync(0xffffffffu, y, 0);
            }
            __syncwarp();
            // Prefix below T[0]: T is constant (= T[0]) below the stored range,
            // where Delta vanishes, and hi is 0 below displacement 0.
            const uint32_t T0 = T[0];
            for (int jj = -(lane + 1); jj >= -S; jj -= 32)
                T[(jj >> 5) * kCs + (jj & 31)] = (base + jj >= 0) ? T0 : 0u;
            __syncwarp();
            // hi[i] = -T[i - S]
            for (int c = lane; c < NC; c += 32) {
                const int i0 = c * kCh;
                uint32_t* p1 = o1 + c * kCs;
                const int jb = i0 - S;  // source index of element 0 (>= -S)
                const int rb = jb & 31;
                const uint32_t* ps = T + (jb >> 5) * kCs + rb;  // element k: next chunk once rb + k >= 32
                if (whole || i0 + kCh <= W) {
#pragma unroll
                    for (int k = 0; k < kCh; ++k) p1[k] = 0u - ps[k + (k >= 32 - rb ? 1 : 0)];
                } else {
#pragma unroll
                    for (int k = 0; k < kCh; ++k)
                        if (i0 + k < W) p1[k] = 0u - ps[k + (k >= 32 - rb ? 1 : 0)];
                }
            }
        }
        __syncthreads();
        if (threadIdx.x < 32) {
            // new slot of every row of stage J (computed by one warp, lane r)
            const int r = threadIdx.x;
            int ns = 0;
            if (r < R) {
                const int hi = (r >> J) & 1;        // position bit J of the stage-J row
                const int a = r - (hi << J);        // its lo partner
                const int q = a >> (J + 1), tau = a & (half - 1);
                const int r0 = 2 * tau + (q << (J + 1));
                ns = slot[r0 + hi];
            }
            __syncwarp();
            if (r < R) slot[r] = ns;
        }
        __syncthreads();
    }

    // Store the unit's input rows a(u) = sg + (u << m0) + (w << (m0 + G)).
    // Recovered values below the output geometry's lower bound must vanish.
    const int lo_out = L.lo_out;
    for (int u = warp; u < R; u += kInvWarps) {
        const int a = sg + (u << m0) + (wq << (m0 + G));
        const uint32_t* srow = rows + slot[u] * WS + lane;
        bool bad = false;
        if (L.scatter) {
            // Stage 0 rows: the volume sits at d in [2N, 3N) of the frame row (x', y').
            const int xp = L.axis == 0 ? a : j, yp = L.axis == 0 ? j : a;
            int32_t* vol = static_cast<int32_t*>(L.out);
            const long long rb = L.map.o0 + xp * L.map.sx + yp * L.map.sy;
            for (int c = 0; c < NC; ++c) {
                const int i = c * kCh + lane;
                if (i >= W) break;
                const int d = base + i;
                const uint32_t v = srow[c * kCs];
                if (d < 2 * N) bad |= v != 0u;
                else vol[rb + (long long)(d - 2 * N) * L.map.sz] = (int32_t)v;
            }
        } else {
            const long long row = (long long)a * rs_axis + (long long)j * rs_other;
            uint32_t* dst = static_cast<uint32_t*>(L.out) + row * L.gout.pitch - L.gout.base + base + lane;
            for (int c = 0; c < NC; ++c) {
                const int i = c * kCh + lane;
                if (i >= W) break;
                const int d = base + i;
                const uint32_t v = srow[c * kCs];
                if (d < lo_out) bad |= v != 0u;
                if (d >= L.gout.base) dst[c * kCh] = v;
            }
        }
        if (__any_sync(0xffffffffu, bad) && lane == 0) flag(L.status, DRT3D_ERR_NOT_IN_RANGE);
    }
}

size_t inv_smem(int G, int W) {
    const int NC = (W + kCh - 1) / kCh;
    return ((size_t)(1 << G) * NC + (size_t)((1 << G) / 2) * (NC + kPre)) * kCs * 4;
}

template <int G>
cudaError_t launch_inv_g(const InvLaunch& L, cudaStream_t s) {
    const int W = L.dmax - L.gin.base;
    const size_t smem = inv_smem(G, W);
    auto kern = planes_inv_pass<G>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const unsigned units = (unsigned)((long long)L.N << (L.n - G));
    kern<<<units, kInvWarps * 32, smem, s>>>(L);
    return cudaGetLastError();
}

}  // namespace

size_t inverse_smem_bytes(int N, int G, int base) {
    const int W = 3 * N - base;
    return inv_smem(G, W);
}

cudaError_t launch_planes_inverse_pass(const InvLaunch& L, int G, cudaStream_t s) {
    switch (G) {
    case 1: return launch_inv_g<1>(L, s);
    case 2: return launch_inv_g<2>(L, s);
    case 3: return launch_inv_g<3>(L, s);
    case 4: return launch_inv_g<4>(L, s);
    }
    return cudaErrorInvalidValue;
}

}  // namespace drt3d
