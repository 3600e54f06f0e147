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
// memory for the whole group, and each of the 2^(G-1) pairs of a stage is one
// warp.  A lane holds a CH-displacement chunk of both rows of its pair in
// registers (CH = 8, 16 or 32; rows of more than 32 chunks are scanned in
// segments of 32 chunks from the top, carrying the sum down), forms
// nD = out_0 - out_1 and the chunk's suffix sums; one warp shuffle scan of the
// chunk totals turns them into nT = -T.  lo = out_0 - nT goes back over out_0
// and nT over out_1.  hi[e] = nT[e - S] is not copied: the slot records the
// offset S, and whoever reads the row later (the next stage, the range check,
// the final store) reads element e at e - S.  A stage's pair is either two
// unshifted rows or two rows at offsets (S, S + 1) (the hi rows of two
// neighbouring pairs of the previous stage); shifted rows are read as 16-byte
// vectors from the aligned element below and unpacked at a compile-time
// misalignment.
//
// Shared layout: a row slot holds P prefix chunks (displacements below the
// stored range, which the shifted copy reads) and NC chunks of CH words.
// Chunks are CH + 4 words apart, and (CH/4 + 1) is odd: vector k of chunk c
// then falls in 16-byte bank group (c (CH/4 + 1) + k) mod 8, so the three
// access patterns -- lane = chunk, lane = consecutive vector, lane = chunk at
// a common shifted offset -- each touch 8 distinct groups per quarter warp,
// and a lane's vectors of one chunk sit at fixed offsets from its start.  Lanes whose chunk lies past the row
// take part in the shuffle scans only: they read the last chunk's addresses
// (served by broadcast, no extra traffic) and store nothing.
#include "internal.cuh"
#include "tma.cuh"

namespace drt3d {
namespace {

__host__ __device__ constexpr int inv_warps(int G) { return G >= 4 ? 8 : (1 << (G - 1)); }

// Chunk width: 8 up to 384 displacements (one or two segments; four CTAs
// fit an SM), 16 up to 1024 (one or two segments: three CTAs per SM, which
// beats one segment of 24-wide chunks at two), 32 beyond.  The second
// segment of a short row keeps only a few lanes busy, but the shorter chains
// and higher occupancy more than pay for it.
__host__ __device__ inline int inv_chunk_width(int W) { return W <= 384 ? 8 : W <= 1024 ? 16 : 32; }

// Prefix chunks of a slot: the shifted copy of a half-stage with slope so
// far S reads down to displacement -(S + 3); S < 2^(m0 + G - 1).
__host__ __device__ inline int inv_pre_chunks(int m0, int G, int CH) { return ((1 << (m0 + G - 1)) + 2 + CH - 1) / CH; }

__host__ __device__ inline int inv_slot_words(int W, int m0, int G, int CH) {
    return (inv_pre_chunks(m0, G, CH) + (W + CH - 1) / CH) * (CH + 4) + 4;
}

__device__ __forceinline__ void flag(int* status, int code) {
    if (*status == 0) atomicCAS(status, 0, code);
}

// Word offset, within a slot, of element i (i >= -CH P).
template <int CH>
__device__ __forceinline__ int word_off(int i, int P) {
    const int j = i + P * CH;  // >= 0
    const int c = j / CH;
    return c * (CH + 4) + (j - c * CH);
}

__device__ __forceinline__ uint4 lds4(const uint32_t* s, int off) { return *reinterpret_cast<const uint4*>(s + off); }
__device__ __forceinline__ void sts4(uint32_t* s, int off, uint4 v) { *reinterpret_cast<uint4*>(s + off) = v; }

// The 4 * NVEC elements of a row from the 4-aligned physical element
// `start` (>= -CH P), NVEC = CH/4 or CH/4 + 1: crosses at most one chunk
// boundary.
template <int CH, int NVEC>
__device__ __forceinline__ void read_window(const uint32_t* s, int start, int P, uint32_t (&src)[4 * NVEC]) {
    constexpr int VPC = CH / 4;
    const int w0 = word_off<CH>(start, P);
    const int kb = VPC - (((start + P * CH) % CH) >> 2);  // vectors before the next chunk starts
#pragma unroll
    for (int t = 0; t < NVEC; ++t) {
        const uint4 w = lds4(s, w0 + 4 * t + (t >= kb ? 4 : 0));
        src[4 * t] = w.x; src[4 * t + 1] = w.y; src[4 * t + 2] = w.z; src[4 * t + 3] = w.w;
    }
}

// Logical chunk c of both rows of a pair: a = out_0, x = out_0 - out_1.
// SH: the rows sit at offsets (off0, off0 + 1) with RR0 = (-off0) & 3;
// otherwise both are unshifted.
template <int CH, bool SH, int RR0>
__device__ __forceinline__ void load_pair(const uint32_t* s0, const uint32_t* s1, int c, int off0, int P,
                                          uint32_t (&a)[CH], uint32_t (&x)[CH]) {
    constexpr int VPC = CH / 4;
    if constexpr (!SH) {
        const int cw = (c + P) * (CH + 4);
#pragma unroll
        for (int kv = 0; kv < VPC; ++kv) {
            const uint4 A = lds4(s0, cw + 4 * kv);
            const uint4 B = lds4(s1, cw + 4 * kv);
            a[4 * kv] = A.x; a[4 * kv + 1] = A.y; a[4 * kv + 2] = A.z; a[4 * kv + 3] = A.w;
            x[4 * kv] = A.x - B.x; x[4 * kv + 1] = A.y - B.y; x[4 * kv + 2] = A.z - B.z; x[4 * kv + 3] = A.w - B.w;
        }
    } else {
        constexpr int RR1 = (RR0 + 3) & 3;  // (-(off0 + 1)) & 3
        constexpr int N0 = RR0 ? VPC + 1 : VPC, N1 = RR1 ? VPC + 1 : VPC;
        uint32_t w0[4 * N0], w1[4 * N1];
        read_window<CH, N0>(s0, CH * c - off0 - RR0, P, w0);
        read_window<CH, N1>(s1, CH * c - off0 - 1 - RR1, P, w1);
#pragma unroll
        for (int k = 0; k < CH; ++k) {
            a[k] = w0[k + RR0];
            x[k] = w0[k + RR0] - w1[k + RR1];
        }
    }
}

// One pair of one stage: lo over out_0's slot, nT over out_1's slot (with
// its prefix below the stored range).  Segments of 32 chunks from the top;
// inside one, every lane reads before any lane writes (shifted reads reach
// lower chunks, writes go to the lane's own chunk).
template <int CH, bool MULTI, bool SH, int RR0>
__device__ __forceinline__ void stage_pair(uint32_t* s0, uint32_t* s1, int off0, int P, int NC, int base, int lane) {
    constexpr int VPC = CH / 4;
    constexpr int RUN = CH / 4;  // suffix-sum run length (4 runs per chunk)
    const int nseg = MULTI ? (NC + 31) / 32 : 1;
    uint32_t seg_carry = 0, first = 0;
#pragma unroll 1
    for (int sgm = nseg - 1; sgm >= 0; --sgm) {
        const int c = sgm * 32 + lane;
        const bool live = c < NC;
        uint32_t a[CH], x[CH];
        load_pair<CH, SH, RR0>(s0, s1, live ? c : NC - 1, off0, P, a, x);
        // Chunk suffix sums as 4 independent runs (short dependency chains),
        // then the runs' carries.
#pragma unroll
        for (int k = RUN - 2; k >= 0; --k)
#pragma unroll
            for (int b = 0; b < 4; ++b) x[RUN * b + k] += x[RUN * b + k + 1];
        uint32_t rc[4];
        rc[3] = 0u;
        rc[2] = x[3 * RUN];
        rc[1] = rc[2] + x[2 * RUN];
        rc[0] = rc[1] + x[RUN];
        const uint32_t tot = live ? x[0] + rc[0] : 0u;
        uint32_t y = tot;
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const uint32_t z = __shfl_down_sync(0xffffffffu, y, off);
            if (lane + off < 32) y += z;
        }
        const uint32_t carry = y - tot + seg_carry;
#pragma unroll
        for (int b = 0; b < 4; ++b) rc[b] += carry;
#pragma unroll
        for (int k = 0; k < CH; ++k) {
            x[k] += rc[k / RUN];  // nT
            a[k] -= x[k];         // lo = out_0 + T
        }
        first = x[0];
        if constexpr (SH) __syncwarp();  // all shifted reads of the segment before its writes
        if (live) {
            const int cw = (c + P) * (CH + 4);
#pragma unroll
            for (int kv = 0; kv < VPC; ++kv) {
                sts4(s0, cw + 4 * kv, make_uint4(a[4 * kv], a[4 * kv + 1], a[4 * kv + 2], a[4 * kv + 3]));
                sts4(s1, cw + 4 * kv, make_uint4(x[4 * kv], x[4 * kv + 1], x[4 * kv + 2], x[4 * kv + 3]));
            }
        }
        seg_carry += __shfl_sync(0xffffffffu, y, 0);
        if constexpr (SH && MULTI) __syncwarp();
    }
    // Prefix below the stored range: T is constant (= T[0]) there, where
    // Delta vanishes, and hi is 0 below displacement 0.
    const uint32_t nT0 = __shfl_sync(0xffffffffu, first, 0);
#pragma unroll
    for (int it = 0; it < 2; ++it) {
        const int v = lane + 32 * it;
        const int i = -CH * P + 4 * v;
        const uint32_t f = base + i >= 0 ? nT0 : 0u;
        if (v < VPC * P) sts4(s1, word_off<CH>(i, P), make_uint4(f, f, f, f));
    }
    for (int v = lane + 64; v < VPC * P; v += 32) {
        const int i = -CH * P + 4 * v;
        const uint32_t f = base + i >= 0 ? nT0 : 0u;
        sts4(s1, word_off<CH>(i, P), make_uint4(f, f, f, f));
    }
}

// MULTI: rows of more than 32 chunks, scanned in segments of 32 chunks from
// the top with a carry; otherwise one segment.
template <int G, int CH, bool MULTI>
__global__ void __launch_bounds__(inv_warps(G) * 32, (G >= 4 ? (CH <= 8 ? 4 : CH <= 16 ? 3 : 2) : 4))
planes_inv_pass(const __grid_constant__ InvLaunch L) {
    pdl_wait_and_release();
    constexpr int R = 1 << G;
    constexpr int NW = inv_warps(G);
    constexpr int NT = NW * 32;
    constexpr int VPC = CH / 4;
    constexpr int RUN = CH / 4;  // suffix-sum run length (4 runs per chunk)
    extern __shared__ __align__(16) unsigned char smem_raw[];
    uint32_t* rows = reinterpret_cast<uint32_t*>(smem_raw);
    __shared__ int slot[R];
    __shared__ int slot_off[R];  // offset of the row a slot holds (element e at e - offset)

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int N = L.N, m0 = L.m0;
    const int base = L.gin.base;
    const int W = L.dmax - base;       // stored row length of the input geometry
    const int NC = (W + CH - 1) / CH;  // chunks per row
    const int P = inv_pre_chunks(m0, G, CH);
    const int RS = inv_slot_words(W, m0, G, CH);
    unsigned unit = blockIdx.x;
    const int sg = (int)(unit & ((1u << m0) - 1)); unit >>= m0;
    const int wb = L.n - m0 - G;
    const int wq = (int)(unit & ((1u << wb) - 1));
    const int j = (int)(unit >> wb);
    const long long rs_axis = L.axis == 0 ? N : 1;  // row stride of the undone axis
    const long long rs_other = L.axis == 0 ? 1 : N;

    // ---- load the unit's output rows o(t) = t + (sg << G) + (w << (m0 + G)),
    // zeros past the stored width in the last chunk
    {
        const uint32_t* in = static_cast<const uint32_t*>(L.in);
        const bool vec_in = (L.gin.pitch & 3) == 0;
        const int NV = NC * VPC;  // 16-byte vectors per row
        constexpr int B = 8;      // vectors in flight per lane
        for (int t = warp; t < R; t += NW) {
            const long long row = (long long)(t + (sg << G) + (wq << (m0 + G))) * rs_axis + (long long)j * rs_other;
            const uint32_t* src = in + row * L.gin.pitch;
            uint32_t* dst = rows + t * RS;
            for (int v0 = lane; v0 < NV; v0 += B * 32) {
                uint4 w[B];
#pragma unroll
                for (int b = 0; b < B; ++b) {
                    const int i = 4 * (v0 + 32 * b);
                    w[b] = make_uint4(0u, 0u, 0u, 0u);
                    if (vec_in && i + 4 <= W) {
                        w[b] = __ldg(reinterpret_cast<const uint4*>(src + i));
                    } else if (i < W) {
                        w[b].x = __ldg(src + i);
                        if (i + 1 < W) w[b].y = __ldg(src + i + 1);
                        if (i + 2 < W) w[b].z = __ldg(src + i + 2);
                        if (i + 3 < W) w[b].w = __ldg(src + i + 3);
                    }
                }
#pragma unroll
                for (int b = 0; b < B; ++b)
                    if (v0 + 32 * b < NV) sts4(dst, word_off<CH>(4 * (v0 + 32 * b), P), w[b]);
            }
        }
    }
    if (threadIdx.x < R) {
        slot[threadIdx.x] = threadIdx.x;
        slot_off[threadIdx.x] = 0;
    }
    __syncthreads();

#pragma unroll 1
    for (int J = G - 1; J >= 0; --J) {
        const int half = 1 << J;
        {
            const int p = warp;  // one pair per warp
            const int q = p >> J, tau = p & (half - 1);
            const int r0 = 2 * tau + (q << (J + 1));  // rows of stage J+1 (within the unit)
            const int S = (sg << J) + tau;            // slope so far at global stage m0 + J
            const int sl0 = slot[r0], sl1 = slot[r0 + 1];
            uint32_t* s0 = rows + sl0 * RS;
            uint32_t* s1 = rows + sl1 * RS;
            const int off1 = slot_off[sl1];
            const int off0 = off1 ? off1 - 1 : 0;  // the pair is (0, 0) or (off, off + 1)

            // Data in the range has Delta = 0 past 3N - 1 - S; check it there.
            {
                bool bad = false;
                const int from = W - S > 0 ? W - S : 0;
#pragma unroll
                for (int it = 0; it < 4; ++it) {  // S < 128: at most 4 rounds
                    const int i = from + lane + 32 * it;
                    if (i < W) bad |= s0[word_off<CH>(i - off0, P)] != s1[word_off<CH>(i - off1, P)];
                }
                for (int i = from + 128 + lane; i < W; i += 32)
                    bad |= s0[word_off<CH>(i - off0, P)] != s1[word_off<CH>(i - off1, P)];
                if (__any_sync(0xffffffffu, bad) && lane == 0) flag(L.status, DRT3D_ERR_NOT_IN_RANGE);
            }
            __syncwarp();
            if (off1 == 0) {
                stage_pair<CH, MULTI, false, 0>(s0, s1, 0, P, NC, base, lane);
            } else {
                switch ((-off0) & 3) {
                case 0: stage_pair<CH, MULTI, true, 0>(s0, s1, off0, P, NC, base, lane); break;
                case 1: stage_pair<CH, MULTI, true, 1>(s0, s1, off0, P, NC, base, lane); break;
                case 2: stage_pair<CH, MULTI, true, 2>(s0, s1, off0, P, NC, base, lane); break;
                default: stage_pair<CH, MULTI, true, 3>(s0, s1, off0, P, NC, base, lane); break;
                }
            }
            if (lane == 0) {
                slot_off[sl0] = 0;  // lo, in place
                slot_off[sl1] = S;  // hi[e] = nT[e - S]
            }
        }
        __syncthreads();
        if (threadIdx.x < 32) {
            // new slot of every row of stage J (lane r)
            const int r = threadIdx.x;
            int ns = 0;
            if (r < R) {
                const int hb = (r >> J) & 1;   // position bit J of the stage-J row
                const int a = r - (hb << J);   // its lo partner
                const int q = a >> (J + 1), tau = a & (half - 1);
                ns = slot[2 * tau + (q << (J + 1)) + hb];
            }
            __syncwarp();
            if (r < R) slot[r] = ns;
        }
        __syncthreads();
    }

    // ---- store the unit's input rows a(u) = sg + (u << m0) + (w << (m0 + G)).
    // Recovered values below the output geometry's lower bound must vanish.
    // A row at offset `off` holds element i at i - off.
    bool bad = false;
    if (!L.scatter) {
        const int lo_out = L.lo_out;
        const bool vec_out = (L.gout.pitch & 3) == 0;
        uint32_t* out = static_cast<uint32_t*>(L.out);
        for (int u = warp; u < R; u += NW) {
            const int a = sg + (u << m0) + (wq << (m0 + G));
            const long long row = (long long)a * rs_axis + (long long)j * rs_other;
            uint32_t* dst = out + row * L.gout.pitch - L.gout.base + base;  // element i of the stored row
            const uint32_t* srow = rows + slot[u] * RS;
            const int off = slot_off[slot[u]];
            for (int v = lane; 4 * v < W; v += 32) {
                const int i = 4 * v;
                const int d = base + i;
                uint32_t e[4];
                if ((off & 3) == 0) {
                    const uint4 w = lds4(srow, word_off<CH>(i - off, P));
                    e[0] = w.x; e[1] = w.y; e[2] = w.z; e[3] = w.w;
                } else {
#pragma unroll
                    for (int k = 0; k < 4; ++k) e[k] = srow[word_off<CH>(i + k - off, P)];
                }
                if (d < lo_out) {
#pragma unroll
                    for (int k = 0; k < 4; ++k)
                        if (d + k < lo_out) bad |= e[k] != 0u;
                }
                if (d >= L.gout.base) {
                    if (vec_out && i + 4 <= W) {
                        *reinterpret_cast<uint4*>(dst + i) = make_uint4(e[0], e[1], e[2], e[3]);
                    } else {
#pragma unroll
                        for (int k = 0; k < 4; ++k)
                            if (i + k < W) dst[i + k] = e[k];
                    }
                }
            }
        }
    } else {
        // Stage-0 rows: the volume sits at d in [2N, 3N) of frame row (x', y').
        int32_t* vol = static_cast<int32_t*>(L.out);
        const Affine& M = L.map;
        const long long s_row = L.axis == 0 ? M.sx : M.sy;  // volume stride between rows u, u + 1
        if (M.sz == 1 || (s_row != 1 && s_row != -1)) {
            // lanes along d
            for (int u = warp; u < R; u += NW) {
                const int a = sg + (u << m0) + (wq << (m0 + G));
                const int xp = L.axis == 0 ? a : j, yp = L.axis == 0 ? j : a;
                const long long rb = M.o0 + xp * M.sx + yp * M.sy;
                const uint32_t* srow = rows + slot[u] * RS;
                const int off = slot_off[slot[u]];
                for (int v = lane; 4 * v < W; v += 32) {
                    const int i = 4 * v;
                    const int d = base + i;
                    uint32_t e[4];
                    if ((off & 3) == 0) {
                        const uint4 w = lds4(srow, word_off<CH>(i - off, P));
                        e[0] = w.x; e[1] = w.y; e[2] = w.z; e[3] = w.w;
                    } else {
#pragma unroll
                        for (int k = 0; k < 4; ++k) e[k] = srow[word_off<CH>(i + k - off, P)];
                    }
                    if (M.sz == 1 && d >= 2 * N && i + 4 <= W && ((rb + d - 2 * N) & 3) == 0) {
                        *reinterpret_cast<uint4*>(vol + rb + (d - 2 * N)) = make_uint4(e[0], e[1], e[2], e[3]);
                    } else {
#pragma unroll
                        for (int k = 0; k < 4; ++k) {
                            if (i + k >= W) break;
                            if (d + k < 2 * N) bad |= e[k] != 0u;
                            else vol[rb + (long long)(d + k - 2 * N) * M.sz] = (int32_t)e[k];
                        }
                    }
                }
            }
        } else {
            // lanes along the rows u (unit stride in the volume)
            for (int idx = threadIdx.x; idx < R * W; idx += NT) {
                const int i = idx / R, u = idx - i * R;
                const int d = base + i;
                const uint32_t e = rows[slot[u] * RS + word_off<CH>(i - slot_off[slot[u]], P)];
                if (d < 2 * N) {
                    bad |= e != 0u;
                } else {
                    const int a = sg + (u << m0) + (wq << (m0 + G));
                    const int xp = L.axis == 0 ? a : j, yp = L.axis == 0 ? j : a;
                    vol[M.o0 + xp * M.sx + yp * M.sy + (long long)(d - 2 * N) * M.sz] = (int32_t)e;
                }
            }
        }
    }
    if (__any_sync(0xffffffffu, bad) && lane == 0) flag(L.status, DRT3D_ERR_NOT_IN_RANGE);
}

// ---------------------------------------------------------------------------
// Aligned-row variant (rows of at most 896 displacements, i.e. N <= 256).
//
// Same stage algebra as above, but every row is kept physically aligned in
// shared memory: element i of a slot is displacement base + i.  The shift of
// hi (hi[i] = nT[i - S]) is applied once, when hi is written: lane l holds
// nT over its chunk [l CH, l CH + CH) and writes the aligned block
// [l CH + sa, l CH + sa + CH), sa = S & ~3, whose first r = S & 3 elements
// are the last r of lane l - 1's chunk (one shuffle each); below the
// stored window T is constant (Delta vanishes there), so hi[i] for i < S is
// nT[0] while base + i - S >= 0 and 0 below displacement 0.  Every later
// access is then an aligned 16-byte vector at the lane's own chunk.  CH is
// 4 VPL with VPL odd, so the 8 lanes of each quarter-warp phase of an LDS.128
// or STS.128 at a stride of CH words touch 8 distinct bank groups (an even
// VPL = 6 for rows of 768 was a third slower with its two-way conflicts).  A
// pair is undone by a warp (LPP = 32 lanes) or, for rows of at most 320, by
// a half-warp (LPP = 16: the narrowest span LPP CH >= W wins).
//
// The slots hold LPP CH words (the lanes' chunks) plus room for the shifted
// block of the last lane.  Positions in [W, LPP CH) are zero at load; lo stays
// zero there and hi is zero there whenever the pair passes the range check
// (nT must vanish above W - 1 - S), so they never disturb the suffix sums of
// data in the range of the forward map.
template <int CH>
__device__ __forceinline__ void load_chunk(const uint32_t* s, int c0, uint32_t (&v)[CH]) {
#pragma unroll
    for (int k = 0; k < CH / 4; ++k) {
        const uint4 w = lds4(s, c0 + 4 * k);
        v[4 * k] = w.x; v[4 * k + 1] = w.y; v[4 * k + 2] = w.z; v[4 * k + 3] = w.w;
    }
}

template <int CH>
__device__ __forceinline__ void store_chunk(uint32_t* s, int c0, const uint32_t (&v)[CH]) {
#pragma unroll
    for (int k = 0; k < CH / 4; ++k) sts4(s, c0 + 4 * k, make_uint4(v[4 * k], v[4 * k + 1], v[4 * k + 2], v[4 * k + 3]));
}

// hi over the lane's aligned block at c0 + sa: element j is nT[c0 + j - RR]
// (j >= RR, this lane) or the previous lane's nT[c0 - RR + j] (j < RR); for
// lane 0 those positions lie below S and take the fill value (nT[0] from
// position fill_from on, 0 below).
template <int CH, int RR, int LPP>
__device__ __forceinline__ void realign(const uint32_t (&x)[CH], int lane, int sa, uint32_t nt0, int fill_from,
                                        uint32_t (&e)[CH]) {
#pragma unroll
    for (int j = 0; j < RR; ++j) {
        const uint32_t p = __shfl_up_sync(0xffffffffu, x[CH - RR + j], 1, LPP);
        e[j] = lane > 0 ? p : (sa + j >= fill_from ? nt0 : 0u);
    }
#pragma unroll
    for (int j = RR; j < CH; ++j) e[j] = x[j - RR];
}

// The same with the previous lane's last three elements already shuffled in
// (prev[k] = its x[CH - 3 + k]): no shuffle inside the branch on r.
template <int CH, int RR>
__device__ __forceinline__ void realign_from(const uint32_t (&x)[CH], const uint32_t (&prev)[3], int lane, int sa,
                                             uint32_t nt0, int fill_from, uint32_t (&e)[CH]) {
#pragma unroll
    for (int j = 0; j < RR; ++j) e[j] = lane > 0 ? prev[3 - RR + j] : (sa + j >= fill_from ? nt0 : 0u);
#pragma unroll
    for (int j = RR; j < CH; ++j) e[j] = x[j - RR];
}

// r = S & 3 is uniform over a warp when a pair is the whole warp; with
// half-warp pairs the two pairs of a warp have different slopes, so the
// shuffles are done by every lane before branching on r.
template <int CH, int LPP>
__device__ __forceinline__ void realign_any(int r, const uint32_t (&x)[CH], int lane, int sa, uint32_t nt0,
                                            int fill_from, uint32_t (&e)[CH]) {
    if constexpr (LPP == 32) {
        switch (r) {
        case 0: realign<CH, 0, LPP>(x, lane, sa, nt0, fill_from, e); break;
        case 1: realign<CH, 1, LPP>(x, lane, sa, nt0, fill_from, e); break;
        case 2: realign<CH, 2, LPP>(x, lane, sa, nt0, fill_from, e); break;
        default: realign<CH, 3, LPP>(x, lane, sa, nt0, fill_from, e); break;
        }
    } else {
        uint32_t prev[3];
#pragma unroll
        for (int k = 0; k < 3; ++k) prev[k] = __shfl_up_sync(0xffffffffu, x[CH - 3 + k], 1, LPP);
        switch (r) {
        case 0: realign_from<CH, 0>(x, prev, lane, sa, nt0, fill_from, e); break;
        case 1: realign_from<CH, 1>(x, prev, lane, sa, nt0, fill_from, e); break;
        case 2: realign_from<CH, 2>(x, prev, lane, sa, nt0, fill_from, e); break;
        default: realign_from<CH, 3>(x, prev, lane, sa, nt0, fill_from, e); break;
        }
    }
}

// Upper bound (ns) on the wait for a bulk row copy: a copy that has not
// landed by then is reported as a time-out.
constexpr unsigned long long kBulkWaitNs = 200000000ull;

// Physical slot of logical row r once stages G-1 .. J1 have been undone.
// Undoing stage J keeps lo in out_0's slot and hi in out_1's: the row with
// position bit J = hb and low bits tau came from stage-(J+1) row
// 2 tau + hb of its block, i.e. the low J + 1 bits rotated left by one.
template <int G, int J1>
__device__ __forceinline__ int phys_slot(int r) {
#pragma unroll
    for (int J = J1; J < G; ++J) {
        constexpr int one = 1;
        const int m = (2 * one << J) - 1;
        r = (r & ~m) | (((r << 1) | ((r >> J) & 1)) & m);
    }
    return r;
}

// Per-CTA constants of the aligned-row kernel (lane: within the pair's LPP
// lanes; pair: the pair of a stage this thread's lanes undo).
struct InvCtx {
    uint32_t* rows;  // slot 0
    int RS, W, base, sg, wq, j, m0, c0, lane, pair, LO, dlt;
    long long rs_axis, rs_other;
    bool direct;
};

// Undo stage J of the group (one pair per LPP lanes), in place in the slots;
// the group's last stage (J = 0) with `direct` sends both rows out by bulk
// copies.
template <int G, int VPL, int J, int LPP>
__device__ __forceinline__ void inv_stage(const InvLaunch& L, const InvCtx& C, bool& bad) {
    constexpr int CH = 4 * VPL;
    constexpr int RUN = VPL;  // suffix-sum run length (4 runs per chunk)
    constexpr int LOG_LPP = LPP == 32 ? 5 : 4;
    constexpr int half = 1 << J;
    const int lane = C.lane, c0 = C.c0, W = C.W;
    const int p = C.pair;
    const int q = p >> J, tau = p & (half - 1);
    const int r0 = 2 * tau + (q << (J + 1));
    const int S = (C.sg << J) + tau;  // slope so far at global stage m0 + J
    uint32_t a[CH], x[CH];
    uint32_t* s0 = C.rows + phys_slot<G, J + 1>(r0) * C.RS;
    uint32_t* s1 = C.rows + phys_slot<G, J + 1>(r0 + 1) * C.RS;
    load_chunk<CH>(s0, c0, a);
    load_chunk<CH>(s1, c0, x);
    // data in the range has Delta = 0 above W - 1 - S (S < 2^(m0 + J))
    {
        bool top_bad = false;
        if (C.m0 + J <= LOG_LPP) {
            if (lane < S) top_bad = s0[W - S + lane] != s1[W - S + lane];
        } else {
            for (int i = W - S + lane; i < W; i += LPP) top_bad |= s0[i] != s1[i];
        }
        if (__any_sync(0xffffffffu, top_bad) && lane == 0) flag(L.status, DRT3D_ERR_NOT_IN_RANGE);
    }
    __syncwarp();  // both rows read by every lane before any lane writes
#pragma unroll
    for (int k = 0; k < CH; ++k) x[k] = a[k] - x[k];  // out_0 - out_1 = -Delta
    // chunk suffix sums as 4 independent runs, then the runs' carries
#pragma unroll
    for (int k = RUN - 2; k >= 0; --k)
#pragma unroll
        for (int b = 0; b < 4; ++b) x[RUN * b + k] += x[RUN * b + k + 1];
    uint32_t rc[4];
    rc[3] = 0u;
    rc[2] = x[3 * RUN];
    rc[1] = rc[2] + x[2 * RUN];
    rc[0] = rc[1] + x[RUN];
    const uint32_t tot = x[0] + rc[0];
    uint32_t y = tot;
#pragma unroll
    for (int off = 1; off < LPP; off <<= 1) {
        const uint32_t z = __shfl_down_sync(0xffffffffu, y, off, LPP);
        if (lane + off < LPP) y += z;
    }
    const uint32_t carry = y - tot;  // chunks above this lane's
#pragma unroll
    for (int b = 0; b < 4; ++b) rc[b] += carry;
#pragma unroll
    for (int k = 0; k < CH; ++k) {
        x[k] += rc[k / RUN];  // nT = -T
        a[k] -= x[k];         // lo = out_0 + T
    }
    store_chunk<CH>(s0, c0, a);
    const uint32_t nt0 = __shfl_sync(0xffffffffu, x[0], 0, LPP);
    const int r = S & 3, sa = S - r;
    const int fill_from = S - C.base;  // hi[i] = nT[0] for S - base <= i < S, 0 below
    {
        uint32_t e[CH];
        realign_any<CH, LPP>(r, x, lane, sa, nt0, fill_from, e);  // hi over [c0 + sa, c0 + sa + CH)
        store_chunk<CH>(s1, c0 + sa, e);
    }
    // positions [0, sa) of hi lie below S
    if (4 * lane < sa) {
        for (int v = lane; 4 * v < sa; v += LPP) {
            uint32_t f[4];
#pragma unroll
            for (int k = 0; k < 4; ++k) f[k] = 4 * v + k >= fill_from ? nt0 : 0u;
            sts4(s1, 4 * v, make_uint4(f[0], f[1], f[2], f[3]));
        }
    }
    if (J > 0 || !C.direct) {
        __syncthreads();
        return;
    }
    // Stage 0 of the group: lo is input row a(2p), hi input row a(2p + 1).
    // Values below LO must vanish; [dlt, W) of both rows leaves by two bulk
    // copies once this warp's writes are visible to the async proxy.
    __syncwarp();
    for (int i = 4 * lane; i < C.LO; i += 4 * LPP) {
        const uint4 u0 = lds4(s0, i), u1 = lds4(s1, i);
        const uint32_t e0[4] = {u0.x | u1.x, u0.y | u1.y, u0.z | u1.z, u0.w | u1.w};
#pragma unroll
        for (int k = 0; k < 4; ++k) bad |= i + k < C.LO && e0[k] != 0u;
    }
    tma::fence_proxy_async_shared();
    __syncwarp();
    if (lane == 0) {
        const int m0 = C.m0;
        const int ua = C.sg + ((2 * p) << m0) + (C.wq << (m0 + G));
        const int ub = ua + (1 << m0);
        uint32_t *da, *db;
        if (!L.scatter) {
            uint32_t* out = static_cast<uint32_t*>(L.out);
            da = out + ((long long)ua * C.rs_axis + (long long)C.j * C.rs_other) * L.gout.pitch;
            db = out + ((long long)ub * C.rs_axis + (long long)C.j * C.rs_other) * L.gout.pitch;
        } else {
            const Affine& M = L.map;
            uint32_t* vol = static_cast<uint32_t*>(L.out);
            const long long ra = M.o0 + (L.axis == 0 ? (long long)ua * M.sx + (long long)C.j * M.sy
                                                     : (long long)C.j * M.sx + (long long)ua * M.sy);
            da = vol + ra;
            db = vol + ra + (L.axis == 0 ? M.sx : M.sy) * (long long)(1 << m0);
        }
        tma::bulk_store(da, s0 + C.dlt, (W - C.dlt) * 4u);
        tma::bulk_store(db, s1 + C.dlt, (W - C.dlt) * 4u);
        tma::bulk_commit();
        tma::bulk_wait_read();  // shared memory stays valid until the copies have read it
    }
}

template <int G, int VPL, int J, int LPP>
__device__ __forceinline__ void inv_stages(const InvLaunch& L, const InvCtx& C, bool& bad) {
    inv_stage<G, VPL, J, LPP>(L, C, bad);
    if constexpr (J > 0) inv_stages<G, VPL, J - 1, LPP>(L, C, bad);
}

// Warps of the aligned-row kernel: 2^(G-1) pairs per stage, LPP lanes each.
__host__ __device__ constexpr int inv_group_warps(int G, int LPP) { return (1 << (G - 1)) * LPP / 32; }

// Minimum resident CTAs of the aligned-row kernel (register budget).
__host__ __device__ constexpr int inv_group_min_ctas(int G, int VPL, int LPP) {
    return LPP == 16 ? 8 : G >= 4 ? (VPL >= 7 ? 3 : 4) : (VPL >= 7 ? 5 : 8);
}

// LPP: lanes per pair, 32 (a warp) or 16 (a half-warp, for rows of at most
// 64 VPL displacements: each lane then holds a wider chunk, fewer lanes idle
// past the row, and the scans take four shuffle steps).
template <int G, int VPL, int LPP>
__global__ void __launch_bounds__(inv_group_warps(G, LPP) * 32, inv_group_min_ctas(G, VPL, LPP))
planes_inv_group(const __grid_constant__ InvLaunch L) {
    pdl_wait_and_release();
    static_assert(LPP == 32 || (LPP == 16 && G >= 2), "a pair is a warp or a half-warp");
    constexpr int R = 1 << G;
    constexpr int NW = inv_group_warps(G, LPP);
    constexpr int NP = R / 2;  // pairs per stage
    constexpr int CH = 4 * VPL;
    constexpr int SPAN = LPP * CH;
    extern __shared__ __align__(16) uint32_t rows_al[];
    __shared__ __align__(8) uint64_t bar[NP];  // one per pair: its two input rows

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int pl = lane % LPP;                       // lane within the pair
    const int pair = warp * (32 / LPP) + lane / LPP;  // the pair these lanes undo
    const int N = L.N, m0 = L.m0;
    const int base = L.gin.base;
    const int W = L.dmax - base;  // stored row length (a multiple of 4, at most SPAN)
    const int RS = SPAN + (((1 << (m0 + G - 1)) + 3) & ~3);  // slot words
    unsigned unit = blockIdx.x;
    const int sg = (int)(unit & ((1u << m0) - 1)); unit >>= m0;
    const int wb = L.n - m0 - G;
    const int wq = (int)(unit & ((1u << wb) - 1));
    const int j = (int)(unit >> wb);
    const long long rs_axis = L.axis == 0 ? N : 1;
    const long long rs_other = L.axis == 0 ? 1 : N;
    const int c0 = pl * CH;
    const Affine& M = L.map;
    // Final rows leave by bulk copies: buffer rows, or volume rows whose z'
    // runs forward in memory from a 16-byte-aligned start.
    const bool direct = !L.scatter || (M.sz == 1 && ((M.o0 | M.sx | M.sy) & 3) == 0);
    // Positions below LO must vanish after the group; only [dlt, W) is stored.
    const int LO = L.scatter ? 2 * N - base : L.lo_out - base;
    const int dlt = L.scatter ? 2 * N - base : L.gout.base - base;
    bool bad = false;

    // ---- the pair of the group's first stage: input rows o(2p), o(2p + 1)
    // into slots 2p, 2p + 1 by two bulk copies; zeros past W.
    {
        const int p = pair;
        uint32_t* s0 = rows_al + (2 * p) * RS;
        uint32_t* s1 = s0 + RS;
        if (pl == 0) {
            tma::mbar_init(&bar[p], 1);
            tma::fence_barrier_init();
            const uint32_t* in = static_cast<const uint32_t*>(L.in);
            const long long orow = (long long)(2 * p + (sg << G) + (wq << (m0 + G))) * rs_axis + (long long)j * rs_other;
            const uint32_t* g0 = in + orow * L.gin.pitch;
            tma::mbar_arrive_expect_tx(&bar[p], 2u * W * 4u);
            tma::bulk_load(s0, g0, W * 4u, &bar[p]);
            tma::bulk_load(s1, g0 + rs_axis * L.gin.pitch, W * 4u, &bar[p]);
        }
        for (int i = W + 4 * pl; i < SPAN; i += 4 * LPP) {
            sts4(s0, i, make_uint4(0u, 0u, 0u, 0u));
            sts4(s1, i, make_uint4(0u, 0u, 0u, 0u));
        }
        __syncwarp();
        if (!tma::mbar_wait(&bar[p], 0, kBulkWaitNs)) {
            if (pl == 0) flag(L.status, DRT3D_ERR_TIMEOUT);
            tma::mbar_wait(&bar[p], 0, kBulkWaitNs);  // once more for the copies in flight
        }
    }

    {
        InvCtx C;
        C.rows = rows_al;
        C.RS = RS; C.W = W; C.base = base; C.sg = sg; C.wq = wq; C.j = j; C.m0 = m0;
        C.c0 = c0; C.lane = pl; C.pair = pair; C.LO = LO; C.dlt = dlt;
        C.rs_axis = rs_axis; C.rs_other = rs_other;
        C.direct = direct;
        inv_stages<G, VPL, G - 1, LPP>(L, C, bad);
    }

    if (!direct) {
        // Volume rows not contiguous along z' (or reversed): from shared
        // memory through the dodecant map.  Stage-0 rows hold the volume at d
        // in [2N, 3N) of frame row (x', y').
        int32_t* vol = static_cast<int32_t*>(L.out);
        const long long s_row = L.axis == 0 ? M.sx : M.sy;  // volume stride between rows u, u + 1
        if (s_row != 1 && s_row != -1) {
#pragma unroll 1
            for (int u = warp; u < R; u += NW) {
                const int a = sg + (u << m0) + (wq << (m0 + G));
                const int xp = L.axis == 0 ? a : j, yp = L.axis == 0 ? j : a;
                const long long rb = M.o0 + xp * M.sx + yp * M.sy;
                const uint32_t* srow = rows_al + phys_slot<G, 0>(u) * RS;
                for (int i = lane; i < W; i += 32) {
                    const int d = base + i;
                    const uint32_t e = srow[i];
                    if (d < 2 * N) bad |= e != 0u;
                    else vol[rb + (long long)(d - 2 * N) * M.sz] = (int32_t)e;
                }
            }
        } else {
            // lanes along the rows u (unit stride in the volume)
            constexpr int NT = NW * 32;
            for (int idx = threadIdx.x; idx < R * W; idx += NT) {
                const int i = idx / R, u = idx - i * R;
                const int d = base + i;
                const uint32_t e = rows_al[phys_slot<G, 0>(u) * RS + i];
                if (d < 2 * N) {
                    bad |= e != 0u;
                } else {
                    const int a = sg + (u << m0) + (wq << (m0 + G));
                    const int xp = L.axis == 0 ? a : j, yp = L.axis == 0 ? j : a;
                    vol[M.o0 + xp * M.sx + yp * M.sy + (long long)(d - 2 * N) * M.sz] = (int32_t)e;
                }
            }
        }
    }
    if (__any_sync(0xffffffffu, bad) && lane == 0) flag(L.status, DRT3D_ERR_NOT_IN_RANGE);
}

// Lanes per pair and chunk vectors per lane of the aligned-row kernel for rows
// of W displacements: the narrowest span LPP * 4 VPL >= W (VPL odd, so the
// lanes of a quarter-warp phase of a 16-byte access hit distinct bank groups;
// half-warp pairs only for spans up to 320), a warp per pair on ties.
// {0, 0} when the rows are too long or not made of whole 16-byte vectors.
struct InvShape {
    int lpp, vpl;
};
InvShape inv_group_shape(int W, int G, const InvLaunch& L) {
    if (W % 4 != 0 || L.gin.pitch % 4 != 0 || (!L.scatter && (L.gout.pitch % 4 != 0 || L.gout.base % 4 != 0)))
        return {0, 0};
    InvShape best{0, 0};
    for (InvShape c : {InvShape{32, 1}, InvShape{32, 3}, InvShape{32, 5}, InvShape{32, 7}, InvShape{16, 3},
                       InvShape{16, 5}}) {
        if (c.lpp == 16 && G < 2) continue;
        const int span = c.lpp * 4 * c.vpl;
        if (span >= W && (best.lpp == 0 || span < best.lpp * 4 * best.vpl)) best = c;
    }
    return best;
}

size_t inv_group_smem(int G, int m0, int vpl, int lpp) {
    return (size_t)(1 << G) * (lpp * 4 * vpl + (((1 << (m0 + G - 1)) + 3) & ~3)) * 4;
}

template <int G, int VPL, int LPP>
cudaError_t launch_inv_group(const InvLaunch& L, cudaStream_t s) {
    const size_t smem = inv_group_smem(G, L.m0, VPL, LPP);
    auto kern = planes_inv_group<G, VPL, LPP>;
    static DeviceOnce attr_done;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (!attr_done.done(dev)) {
        // the largest slot set this instantiation can need (m0 + G <= 10)
        e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)inv_group_smem(G, 10 - G, VPL, LPP));
        if (e != cudaSuccess) return e;
        attr_done.mark(dev);
    }
    const unsigned units = (unsigned)((long long)L.N << (L.n - G));
    return launch_chained(kern, dim3(units), dim3(inv_group_warps(G, LPP) * 32), smem, s, L);
}

template <int G>
cudaError_t launch_inv_group_g(const InvLaunch& L, InvShape sh, cudaStream_t s) {
    if constexpr (G >= 2) {
        if (sh.lpp == 16) return sh.vpl == 3 ? launch_inv_group<G, 3, 16>(L, s) : launch_inv_group<G, 5, 16>(L, s);
    }
    switch (sh.vpl) {
    case 1: return launch_inv_group<G, 1, 32>(L, s);
    case 3: return launch_inv_group<G, 3, 32>(L, s);
    case 5: return launch_inv_group<G, 5, 32>(L, s);
    default: return launch_inv_group<G, 7, 32>(L, s);
    }
}

size_t inv_smem(int G, int W, int m0) {
    return (size_t)(1 << G) * inv_slot_words(W, m0, G, inv_chunk_width(W)) * 4;
}

template <int G, int CH, bool MULTI>
cudaError_t launch_inv_gc(const InvLaunch& L, cudaStream_t s) {
    const int W = L.dmax - L.gin.base;
    const size_t smem = inv_smem(G, W, L.m0);
    auto kern = planes_inv_pass<G, CH, MULTI>;
    // The size cap is per device: raise it once to the device's opt-in
    // maximum (occupancy follows the size each launch asks for).
    static DeviceOnce attr_done;
    static std::atomic<int> optin_max[64] = {};  // written before the device's flag is set
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    if (!attr_done.done(dev)) {
        int mx = 0;
        e = cudaDeviceGetAttribute(&mx, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
        if (e != cudaSuccess) return e;
        cudaFuncAttributes fa{};
        e = cudaFuncGetAttributes(&fa, kern);
        if (e != cudaSuccess) return e;
        mx -= (int)fa.sharedSizeBytes;  // the cap counts dynamic memory only, beside the static
        e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
        if (e != cudaSuccess) return e;
        optin_max[dev].store(mx, std::memory_order_relaxed);
        attr_done.mark(dev);
    }
    if (smem > (size_t)optin_max[dev].load(std::memory_order_relaxed)) return cudaErrorInvalidValue;
    const unsigned units = (unsigned)((long long)L.N << (L.n - G));
    return launch_chained(kern, dim3(units), dim3(inv_warps(G) * 32), smem, s, L);
}

template <int G>
cudaError_t launch_inv_g(const InvLaunch& L, cudaStream_t s) {
    const int W = L.dmax - L.gin.base;
    switch (inv_chunk_width(W)) {
    case 8:
        return (W + 7) / 8 > 32 ? launch_inv_gc<G, 8, true>(L, s) : launch_inv_gc<G, 8, false>(L, s);
    case 16:
        return (W + 15) / 16 > 32 ? launch_inv_gc<G, 16, true>(L, s) : launch_inv_gc<G, 16, false>(L, s);
    default:
        return (W + 31) / 32 > 32 ? launch_inv_gc<G, 32, true>(L, s) : launch_inv_gc<G, 32, false>(L, s);
    }
}

}  // namespace

size_t inverse_smem_bytes(int N, int G, int base, int m0) { return inv_smem(G, 3 * N - base, m0); }

cudaError_t launch_planes_inverse_pass(const InvLaunch& L, int G, cudaStream_t s) {
    const InvShape sh = inv_group_shape(L.dmax - L.gin.base, G, L);
    if (sh.vpl > 0) {
        switch (G) {
        case 1: return launch_inv_group_g<1>(L, sh, s);
        case 2: return launch_inv_group_g<2>(L, sh, s);
        case 3: return launch_inv_group_g<3>(L, sh, s);
        case 4: return launch_inv_group_g<4>(L, sh, s);
        }
        return cudaErrorInvalidValue;
    }
    switch (G) {
    case 1: return launch_inv_g<1>(L, s);
    case 2: return launch_inv_g<2>(L, s);
    case 3: return launch_inv_g<3>(L, s);
    case 4: return launch_inv_g<4>(L, s);
    }
    return cudaErrorInvalidValue;
}

}  // namespace drt3d
