// fused_cta.cuh -- the CTA body of a fused planes pass (G stages of
// eq.(map3D) on both axes), shared by the per-pass kernel (planes_fused.cu)
// and the batched persistent kernel (planes_batched.cu).  See
// planes_fused.cu for the algorithm.
#pragma once

#include <type_traits>

#include "internal.cuh"
#include "tma.cuh"
#include "warp_drt.cuh"

namespace drt3d {
namespace fused {

constexpr int K = 4;       // displacements per lane
constexpr int WT = 32 * K; // displacements per warp tile

template <typename TIn, typename T>
__device__ __forceinline__ T to_acc(TIn x) {
    if constexpr (std::is_same<T, float>::value) {
        return (T)x;
    } else {
        return (T)(int32_t)x;  // zero/sign extension into the int32 ring
    }
}

// Load `n` elements of TIn starting at p (aligned to min(n*sizeof, 16) bytes).
template <typename TIn, int NE>
__device__ __forceinline__ void load_run(const TIn* p, TIn (&dst)[NE]) {
    constexpr int BYTES = NE * (int)sizeof(TIn);
    if constexpr (BYTES >= 16) {
        const uint4* q = reinterpret_cast<const uint4*>(p);
#pragma unroll
        for (int c = 0; c < BYTES / 16; ++c) {
            uint4 w = __ldg(q + c);
            memcpy(reinterpret_cast<char*>(dst) + 16 * c, &w, 16);
        }
    } else if constexpr (BYTES == 8) {
        uint2 w = __ldg(reinterpret_cast<const uint2*>(p));
        memcpy(dst, &w, 8);
    } else if constexpr (BYTES == 4) {
        unsigned w = __ldg(reinterpret_cast<const unsigned*>(p));
        memcpy(dst, &w, 4);
    } else if constexpr (BYTES == 2) {
        unsigned short w = __ldg(reinterpret_cast<const unsigned short*>(p));
        memcpy(dst, &w, 2);
    } else {
#pragma unroll
        for (int e = 0; e < NE; ++e) dst[e] = p[e];
    }
}

// Number of warps of the fused CTA for a G-stage group: one warp per row
// group up to 8; with G = 4 each warp handles two groups per phase, so two
// CTAs (2 x 256 threads, <= 128 registers each) fit on one SM.
template <int G> __host__ __device__ constexpr int fused_warps() { return G >= 3 ? 8 : (1 << G); }
// Displacements of a phase-1 result row that phase 2 consumes: V valid
// outputs plus the 2^G - 1 the phase-2 shifts reach past them.
template <int G> __host__ __device__ constexpr int fused_v() { return (WT - 2 * ((1 << G) - 1)) & ~3; }
template <int G> __host__ __device__ constexpr int fused_ws() { return (fused_v<G>() + (1 << G) - 1 + 3) & ~3; }
// Elements after the last phase-1 row that its lanes past WS read (they read
// on into the next row; for the last row, into this pad).
template <int G> __host__ __device__ constexpr int fused_pad() { return WT - fused_ws<G>() > K ? WT - fused_ws<G>() : K; }

// Staged (TMA) input of one phase-1 group: 2^G rows, each the window
// [q, q + WT) of a row rounded out to 16-byte boundaries (WT + 16 / size
// elements), rows ROW_BYTES apart (a multiple of 128 bytes, the alignment kept
// for TMA destinations).  The staging of group u2 sits at the start of that
// group's block of phase-1 results, which overwrites it once the group's warp
// has read it; a group's block is the larger of the two (group_elems).
template <typename TIn>
struct Stage {
    static constexpr int ELEMS = WT + 16 / (int)sizeof(TIn);
    static constexpr int ROW_BYTES = (ELEMS * (int)sizeof(TIn) + 127) / 128 * 128;
};

// Elements (of the 32-bit phase-1 result type when staged) of one group's
// block of shared memory: its 2^G result rows of WS, or its staging if that is
// larger (32-bit rows).
template <typename TIn, int G, bool TMA>
__host__ __device__ constexpr int group_elems() {
    return (!TMA || (1 << G) * fused_ws<G>() >= (1 << G) * Stage<TIn>::ROW_BYTES / 4)
               ? (1 << G) * fused_ws<G>()
               : (1 << G) * Stage<TIn>::ROW_BYTES / 4;
}
// Upper bound on a stalled transaction-count wait (ns): a load that has not
// landed by then is reported as a time-out.
constexpr unsigned long long kTmaWaitNs = 200000000ull;

// Buffer rows are stored on [base, base + pitch) with base and pitch
// multiples of 8 and hold zeros outside [base, dmax) (dmax a multiple of 4).
// A lane's window [q, q + K) is covered by the two aligned 4-element chunks
// starting at q & ~3; each chunk is entirely inside or entirely outside the
// valid range, so it is one predicated vector load.  r = q & 3 is the same
// for all lanes of a row.  Loads are issued for all rows first, then the
// windows are extracted branch-free.
struct Chunks16 { uint2 c[2]; };   // 8 x 16-bit
struct Chunks32 { uint4 c[2]; };   // 8 x 32-bit

template <typename TIn>
using ChunksOf = typename std::conditional<sizeof(TIn) == 2, Chunks16, Chunks32>::type;

// Global loads: the read-only path, or (COHERENT) an L2-coherent load.  Both
// name the global space explicitly, so pointers that come from a table in
// memory (not kernel parameters) still compile to global accesses.
template <typename V, bool COHERENT>
__device__ __forceinline__ V ld_vec(const V* p) {
    if constexpr (COHERENT) return __ldcg(p);
    else return __ldg(p);
}

// Global stores with the address space named explicitly.
__device__ __forceinline__ void st_global(uint4* p, uint4 v) { __stcg(p, v); }
__device__ __forceinline__ void st_global(uint2* p, uint2 v) { __stcg(p, v); }
__device__ __forceinline__ void st_global(uint32_t* p, uint32_t v) { __stcg(p, v); }
__device__ __forceinline__ void st_global(uint16_t* p, uint16_t v) { __stcg(reinterpret_cast<unsigned short*>(p), v); }
__device__ __forceinline__ void st_global(float* p, float v) { __stcg(p, v); }

template <typename TIn, bool COHERENT>
__device__ __forceinline__ ChunksOf<TIn> load_chunks(const TIn* row, int base, int dmax, int q) {
    ChunksOf<TIn> w;
    const int qa = q & ~3;
#pragma unroll
    for (int c = 0; c < 2; ++c) {
        const int dc = qa + 4 * c;
        const bool in = dc >= base && dc < dmax;
        const TIn* p = row + (in ? dc - base : 0);
        if constexpr (sizeof(TIn) == 2) {
            const uint2 x = ld_vec<uint2, COHERENT>(reinterpret_cast<const uint2*>(p));
            w.c[c] = in ? x : make_uint2(0, 0);
        } else {
            const uint4 x = ld_vec<uint4, COHERENT>(reinterpret_cast<const uint4*>(p));
            w.c[c] = in ? x : make_uint4(0, 0, 0, 0);
        }
    }
    return w;
}

// Elements r .. r+3 of the 8 loaded ones, as accumulator values.
template <typename TIn, typename T>
__device__ __forceinline__ void extract4(const ChunksOf<TIn>& w, int r, T (&v)[K]) {
    if constexpr (sizeof(TIn) == 2) {
        const uint32_t x0 = w.c[0].x, x1 = w.c[0].y, x2 = w.c[1].x, x3 = w.c[1].y;
        const bool hi = (r & 2) != 0;
        const uint32_t a0 = hi ? x1 : x0, a1 = hi ? x2 : x1, a2 = hi ? x3 : x2;
        const uint32_t sh = (uint32_t)(r & 1) * 16u;
        const uint32_t o0 = __funnelshift_r(a0, a1, sh);
        const uint32_t o1 = __funnelshift_r(a1, a2, sh);
        const uint32_t e[4] = {o0 & 0xFFFFu, o0 >> 16, o1 & 0xFFFFu, o1 >> 16};
#pragma unroll
        for (int i = 0; i < K; ++i) v[i] = to_acc<TIn, T>((TIn)e[i]);
    } else {
        const uint32_t x[8] = {w.c[0].x, w.c[0].y, w.c[0].z, w.c[0].w, w.c[1].x, w.c[1].y, w.c[1].z, w.c[1].w};
        uint32_t t[5];
#pragma unroll
        for (int j = 0; j < 5; ++j) t[j] = (r & 2) ? x[j + 2] : x[j];
#pragma unroll
        for (int i = 0; i < K; ++i) {
            const uint32_t bits = (r & 1) ? t[i + 1] : t[i];
            TIn e;
            memcpy(&e, &bits, 4);
            v[i] = to_acc<TIn, T>(e);
        }
    }
}

// 16-bit buffer input of phase 1.  A row's window [q, q + 4) lies in the
// two aligned 4-element chunks starting at q & ~3; `lo` is the offset of the
// first chunk from the row's first stored element and `width` the stored
// width (both multiples of 4).  A chunk outside [0, width) reads as zero, so
// each chunk is one predicated load.  The in-chunk offset q & 3 is the same
// for all lanes and repeats with u1 mod 4, so rows are loaded by residue
// class, and the window is unpacked with its offset fixed at compile time.
template <bool COHERENT>
__device__ __forceinline__ Chunks16 load_pair_u16(const uint16_t* c0, int lo, int width) {
    Chunks16 w;
    w.c[0] = make_uint2(0u, 0u);
    w.c[1] = make_uint2(0u, 0u);
    if ((unsigned)lo < (unsigned)width) w.c[0] = ld_vec<uint2, COHERENT>(reinterpret_cast<const uint2*>(c0));
    if ((unsigned)(lo + 4) < (unsigned)width) w.c[1] = ld_vec<uint2, COHERENT>(reinterpret_cast<const uint2*>(c0 + 4));
    return w;
}

template <int RR, typename T>
__device__ __forceinline__ void unpack_u16(const Chunks16& w, T (&v)[K]) {
    const uint32_t x[4] = {w.c[0].x, w.c[0].y, w.c[1].x, w.c[1].y};
#pragma unroll
    for (int i = 0; i < K; ++i) {
        const int e = RR + i;  // element of the 8 loaded
        const uint32_t word = x[e >> 1];
        v[i] = to_acc<uint16_t, T>((uint16_t)((e & 1) ? (word >> 16) : (word & 0xFFFFu)));
    }
}

template <typename T>
__device__ __forceinline__ T from_bits(uint32_t x) {
    if constexpr (std::is_same<T, float>::value) return __uint_as_float(x);
    else return (T)x;
}

// Words LO .. HI of a staged row from q, each read with the widest aligned
// shared-memory access up to MAXV words (q is aligned to MAXV words).
template <int LO, int HI, int MAXV>
__device__ __forceinline__ void lds_words(const uint32_t* q, uint32_t (&w)[8]) {
    if constexpr (LO <= HI) {
        if constexpr (MAXV >= 4 && LO % 4 == 0 && LO + 3 <= HI) {
            const uint4 x = *reinterpret_cast<const uint4*>(q + LO);
            w[LO] = x.x; w[LO + 1] = x.y; w[LO + 2] = x.z; w[LO + 3] = x.w;
            lds_words<LO + 4, HI, MAXV>(q, w);
        } else if constexpr (MAXV >= 2 && LO % 2 == 0 && LO + 1 <= HI) {
            const uint2 x = *reinterpret_cast<const uint2*>(q + LO);
            w[LO] = x.x; w[LO + 1] = x.y;
            lds_words<LO + 2, HI, MAXV>(q, w);
        } else {
            w[LO] = q[LO];
            lds_words<LO + 1, HI, MAXV>(q, w);
        }
    }
}

// Staged 32-bit rows of residue class J (u1 = J mod 4): the box starts at the
// 4-aligned element below the window, so lane L's chunk is at 4L and its
// elements are rr .. rr + 3 of the eight there, read as whole 16-byte chunks
// (lanes 16 bytes apart: a narrower read would conflict on the banks and cost
// as many wavefronts); the second chunk only when rr > 0.  The odd rows also
// give stage 0 the element after the window: element rr + 4 of the chunks
// when rr > 0, else the next lane's first element, shuffled (rr is the same
// for the whole warp).
template <int J, int G, typename T>
__device__ __forceinline__ void stage_class_u32(int rr, const uint32_t* st, int lane, T (&v)[1 << G][K],
                                                T (&nxt)[1 << (G - 1)]) {
    constexpr int RW = Stage<uint32_t>::ROW_BYTES / 4;  // words between staged rows
    constexpr bool ODD = (J & 1) != 0;
#define DRT3D_STAGE_CLASS(RRV)                                                                 \
    _Pragma("unroll") for (int u1 = J; u1 < (1 << G); u1 += 4) {                               \
        uint32_t w[8];                                                                         \
        lds_words<0, ((RRV) > 0 ? 7 : 3), 4>(st + u1 * RW + lane * K, w);                        \
        _Pragma("unroll") for (int i = 0; i < K; ++i) v[u1][i] = from_bits<T>(w[(RRV) + i]);  \
        if constexpr (ODD) {                                                                   \
            if constexpr ((RRV) > 0) nxt[u1 >> 1] = from_bits<T>(w[(RRV) + K]);               \
            else nxt[u1 >> 1] = shfl_down(v[u1][0], 1);                                        \
        }                                                                                      \
    }
    switch (rr) {
    case 0: DRT3D_STAGE_CLASS(0) break;
    case 1: DRT3D_STAGE_CLASS(1) break;
    case 2: DRT3D_STAGE_CLASS(2) break;
    default: DRT3D_STAGE_CLASS(3) break;
    }
#undef DRT3D_STAGE_CLASS
}

__device__ __forceinline__ uint32_t u16_at(const uint32_t (&w)[8], int e) {
    return (e & 1) ? (w[e >> 1] >> 16) : (w[e >> 1] & 0xFFFFu);
}

// Staged 16-bit rows of residue class J (u1 = J mod 4) at window offset rr:
// each row's K elements, and for the odd rows also the element after them
// (stage 0 adds it instead of shuffling it from the next lane).  Lanes are
// 8 bytes apart, so a 4- or 8-byte read costs two wavefronts: the words the
// window needs take two (rr = 0, four elements) or four, never more than the
// two 8-byte reads of the whole chunk pair.
template <int J, int G, typename T>
__device__ __forceinline__ void stage_class_u16(int rr, const uint16_t* st, int g_lo, int sg1, int lane,
                                                T (&v)[1 << G][K], T (&nxt)[1 << (G - 1)]) {
    constexpr int RW = Stage<uint16_t>::ROW_BYTES / 2;  // elements between staged rows
    constexpr int NE = (J & 1) ? K + 1 : K;
#define DRT3D_STAGE_U16(RRV)                                                             \
    _Pragma("unroll") for (int u1 = J; u1 < (1 << G); u1 += 4) {                         \
        uint32_t w[8];                                                                   \
        lds_words<(RRV) / 2, ((RRV) + NE - 1) / 2, 2>(                                   \
            reinterpret_cast<const uint32_t*>(st + u1 * RW + ((g_lo + sg1 * u1) & 4) + lane * K), w); \
        _Pragma("unroll") for (int i = 0; i < K; ++i)                                    \
            v[u1][i] = to_acc<uint16_t, T>((uint16_t)u16_at(w, RRV + i));                \
        if constexpr ((J & 1) != 0) nxt[u1 >> 1] = to_acc<uint16_t, T>((uint16_t)u16_at(w, RRV + K)); \
    }
    switch (rr) {
    case 0: DRT3D_STAGE_U16(0) break;
    case 1: DRT3D_STAGE_U16(1) break;
    case 2: DRT3D_STAGE_U16(2) break;
    default: DRT3D_STAGE_U16(3) break;
    }
#undef DRT3D_STAGE_U16
}

template <int J, int G, typename T>
__device__ __forceinline__ void unpack_class_u16(int rr, const Chunks16 (&w)[1 << G], T (&v)[1 << G][K]) {
#define DRT3D_UNPACK_CLASS(RRV)                                  \
    _Pragma("unroll") for (int u1 = J; u1 < (1 << G); u1 += 4) \
        unpack_u16<RRV, T>(w[u1], v[u1]);
    switch (rr) {
    case 0: DRT3D_UNPACK_CLASS(0) break;
    case 1: DRT3D_UNPACK_CLASS(1) break;
    case 2: DRT3D_UNPACK_CLASS(2) break;
    default: DRT3D_UNPACK_CLASS(3) break;
    }
#undef DRT3D_UNPACK_CLASS
}

// Phase-2 store of output rows (t1, t2), t2 < 2^G, over the tile's first V
// displacements.  d0, V, base and dmax are multiples of 4, so a lane's K = 4
// values are either all valid or all past the tile: lanes past it return at
// once, the others store one aligned vector per row (element stores only when
// the output pitch rules vectors out).
// With SQ (float32 residual stores), returns the sum of the squares of the
// residual cells this lane stored, else 0.
template <typename TOut, typename T, int G, bool SQ = false>
__device__ __forceinline__ float store_rows(const FusedLaunch& L, const FusedSlot& sp, const T (&v)[1 << G][K],
                                            int t1, int sg1, int wq1, int sg2, int wq2, int rs1, int rs2,
                                            int d0, int lane) {
    constexpr int R = 1 << G;
    constexpr bool FSQ = SQ && std::is_same<TOut, float>::value;
    const int p0 = lane * K;
    const int d = d0 + p0;
    float sq = 0.f;
    if (p0 >= L.V || d >= L.dmax) return sq;
    const int m0 = L.m0;
    const int o1 = t1 + (sg1 << G) + (wq1 << (m0 + G));
    const long long orow0 = (long long)o1 * rs1 + (long long)((sg2 << G) + (wq2 << (m0 + G))) * rs2;
    if constexpr (sizeof(TOut) == 4) {
        if (L.global_layout) {
            // Algorithm 2's array: row g0 + s1 g1 + s2 g2, pitch 3N - 2, the
            // displacement index shifted down by 2 (rows 0 and 1 are dropped).
            const int gp = 3 * L.N - 2;
            TOut* gout = static_cast<TOut*>(sp.out);
#pragma unroll
            for (int t2 = 0; t2 < R; ++t2) {
                const long long r = orow0 + (long long)t2 * rs2;
                const long long grow = sp.g0 + (r >> L.n) * sp.g1 + (r & (L.N - 1)) * sp.g2;
                TOut* dst = gout + grow * gp + (d - 2);
                TOut e[K];
#pragma unroll
                for (int i = 0; i < K; ++i) e[i] = (TOut)v[t2][i];
                if (d >= 2) {
                    uint2 w0, w1;
                    memcpy(&w0, e, 8);
                    memcpy(&w1, e + 2, 8);
                    st_global(reinterpret_cast<uint2*>(dst), w0);
                    st_global(reinterpret_cast<uint2*>(dst + 2), w1);
                } else {
                    st_global(dst + 2, e[2]);
                    st_global(dst + 3, e[3]);
                }
            }
            return sq;
        }
    }
    TOut* out = static_cast<TOut*>(sp.out) + (d - L.gout.base);
    const long long rstride = (long long)rs2 * L.gout.pitch;
    TOut* dst = out + orow0 * L.gout.pitch;
    // residual epilogue: the target cell at the same offset as the output's
    const TOut* sub = sp.sub ? static_cast<const TOut*>(sp.sub) + (dst - static_cast<TOut*>(sp.out)) : nullptr;
    if constexpr (sizeof(TOut) == 4) {
        if (sub && L.vec_store) {
            // The target rows are read in batches of up to 8 before the batch's
            // stores (the target may be the output itself, so a store may not
            // pass a later row's read: reading first keeps the loads in flight).
            constexpr int BT = R < 8 ? R : 8;
#pragma unroll
            for (int t0 = 0; t0 < R; t0 += BT) {
                uint4 bw[BT];
#pragma unroll
                for (int j = 0; j < BT; ++j) bw[j] = __ldcs(reinterpret_cast<const uint4*>(sub + (long long)(t0 + j) * rstride));
#pragma unroll
                for (int j = 0; j < BT; ++j) {
                    TOut e[K], b[K];
                    memcpy(b, &bw[j], 16);
#pragma unroll
                    for (int i = 0; i < K; ++i) {
                        e[i] = (TOut)v[t0 + j][i] - b[i];
                        if constexpr (FSQ) sq += e[i] * e[i];
                    }
                    uint4 w;
                    memcpy(&w, e, 16);
                    st_global(reinterpret_cast<uint4*>(dst + (long long)(t0 + j) * rstride), w);
                }
            }
            return sq;
        }
    }
    if (L.vec_store) {
#pragma unroll
        for (int t2 = 0; t2 < R; ++t2, dst += rstride) {
            TOut e[K];
#pragma unroll
            for (int i = 0; i < K; ++i) e[i] = (TOut)v[t2][i];
            if constexpr (sizeof(TOut) == 4) {
                uint4 w;
                memcpy(&w, e, 16);
                st_global(reinterpret_cast<uint4*>(dst), w);
            } else {
                uint2 w;
                memcpy(&w, e, 8);
                st_global(reinterpret_cast<uint2*>(dst), w);
            }
        }
    } else {
#pragma unroll
        for (int t2 = 0; t2 < R; ++t2, dst += rstride)
#pragma unroll
            for (int i = 0; i < K; ++i)
                if (d + i < L.dmax) {
                    TOut e = (TOut)v[t2][i];
                    if (sub) {
                        e = e - sub[(long long)t2 * rstride + i];
                        if constexpr (FSQ) sq += e * e;
                    }
                    st_global(dst + i, e);
                }
    }
    return sq;
}

// The CTA's sum of its threads' squared residuals, written by thread 0: a
// butterfly within each warp, then the warps in order (the same sum on every
// run).  Every thread of the block must call it.
template <int NW>
__device__ __forceinline__ void write_cta_sq(double* dst, float s) {
    __shared__ double red[NW];
    double t = s;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = t;
    __syncthreads();
    if (threadIdx.x == 0) {
        double a = 0.0;
#pragma unroll
        for (int w = 0; w < NW; ++w) a += red[w];
        *dst = a;
    }
}

// One CTA of a fused pass: unit/tile `cta` of slot `sp`.  All threads of
// the block must call it (it synchronises); warps at or past fused_warps<G>()
// idle.  With COHERENT the input is read with plain loads instead of the
// read-only path (the batched kernel reads buffers other CTAs of the same
// launch wrote).  PF compiles the launch-order L2 prefetch in (it reads
// L.slot at a run-time index; a caller that keeps L in registers leaves it
// out).  SQ (float32 final passes with a residual target) writes the CTA's
// sum of squared residual cells to sp.sq[cta]; then every warp of the block
// must be one of the 2^G / GPW working warps.
template <typename TIn, typename TOut, typename T, typename TS, int G, bool INGEST, bool COHERENT, bool TMA = false,
          bool PF = true, bool SQ = false>
__device__ __forceinline__ void fused_cta(const FusedLaunch& L, const FusedSlot& sp, unsigned cta,
                                          unsigned char* smem_raw, const CUtensorMap* tmap = nullptr,
                                          int slot_z = 0, uint64_t* mbar = nullptr) {
    static_assert(!TMA || (!INGEST && sizeof(TS) == 4 && G >= 3 && (sizeof(TIn) == 2 || sizeof(TIn) == 4)),
                  "TMA staging: 16- or 32-bit buffer input, 32-bit phase-1 results, G >= 3");
    // With TMA, `smem_raw` is 128-byte aligned and `mbar` holds 2^G barriers.
    constexpr int R = 1 << G;
    constexpr int NW = fused_warps<G>();
    constexpr int GPW = R / NW > 0 ? R / NW : 1;  // row groups per warp
    constexpr int WS = fused_ws<G>();
    constexpr int GB = group_elems<TIn, G, TMA>();  // elements of one group's block
    TS* S = reinterpret_cast<TS*>(smem_raw);  // [u2: GB][t1][WS] (+ pad)
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const bool active = warp < NW;
    const int m0 = L.m0;
    const int N = L.N;
    const unsigned ntiles = (unsigned)L.ntiles;
    unsigned unit = cta / ntiles;
    const int tile = (int)(cta - unit * ntiles);
    const int wb = L.n - m0 - G;
    const int sg1 = (int)(unit & ((1u << m0) - 1)); unit >>= m0;
    const int wq1 = (int)(unit & ((1u << wb) - 1)); unit >>= wb;
    const int sg2 = (int)(unit & ((1u << m0) - 1)); unit >>= m0;
    const int wq2 = (int)unit;
    const int d0 = L.gout.base + tile * L.V;
    const bool swap = sp.swap != 0;
    // Row strides (in rows) of the two axes within the [i1][i2] layout.
    const int rs1 = swap ? 1 : N, rs2 = swap ? N : 1;
    // An output row with slopes-so-far (s1, s2) vanishes below d = 2N - s1 - s2
    // (every digital-line value l^m_s(u) is at most s).  A tile that lies below
    // that bound for the unit's largest slopes is all zeros: store them and
    // skip the loads and both transforms.
    const int smax1 = (sg1 << G) + (1 << G) - 1, smax2 = (sg2 << G) + (1 << G) - 1;
    const bool zero_tile = d0 + L.V <= 2 * N - smax1 - smax2;

    if (sp.sub && threadIdx.x < R * R && sizeof(TOut) == 4 && L.vec_store) {
        // Residual: warm L2 with this tile's target rows (one row window per
        // thread), read again by the stores at the end of phase 2.
        const int t1 = threadIdx.x / R, t2 = threadIdx.x % R;
        const int o1 = t1 + (sg1 << G) + (wq1 << (m0 + G)), o2 = t2 + (sg2 << G) + (wq2 << (m0 + G));
        const int hi = min(d0 + L.V, L.dmax);
        if (d0 < hi)
            tma::prefetch_l2(static_cast<const TOut*>(sp.sub) +
                                 ((long long)o1 * rs1 + (long long)o2 * rs2) * L.gout.pitch + (d0 - L.gout.base),
                             (uint32_t)(hi - d0) * (uint32_t)sizeof(TOut));
    }


    if (zero_tile) {
        if (!active) return;
        float sq = 0.f;
#pragma unroll 1
        for (int gi = 0; gi < GPW; ++gi) {
            const int t1 = warp + gi * NW;
            T v[R][K];
#pragma unroll
            for (int r = 0; r < R; ++r)
#pragma unroll
                for (int i = 0; i < K; ++i) v[r][i] = T(0);
            sq += store_rows<TOut, T, G, SQ>(L, sp, v, t1, sg1, wq1, sg2, wq2, rs1, rs2, d0, lane);
        }
        if constexpr (SQ) write_cta_sq<NW>(sp.sq + cta, sq);
        return;
    }

    if constexpr (PF && !INGEST && !TMA && sizeof(TIn) == 4) {
        // Warm L2 with the input rows of the CTA `prefetch_ahead` places later
        // in launch order (about one wave of resident CTAs): one sheared row
        // window per thread, in 16-byte units; a hint only.  A zero tile is
        // not prefetched.
        constexpr int EA = 16 / (int)sizeof(TIn);  // elements per 16 bytes
        if (L.prefetch_ahead > 0 && threadIdx.x < R * R && L.gin.pitch % EA == 0 && L.gin.base % EA == 0 &&
            L.dmax % EA == 0) {
            const unsigned long long nxt =
                (unsigned long long)blockIdx.y * gridDim.x + blockIdx.x + (unsigned)L.prefetch_ahead;
            const unsigned ny = (unsigned)(nxt / gridDim.x), nc = (unsigned)(nxt % gridDim.x);
            if (ny < gridDim.y) {
                const int nsl = launch_slot(L.reverse_slots, ny, gridDim.y);
                unsigned nu = nc / ntiles;
                const int ntile = (int)(nc - nu * ntiles);
                const int nsg1 = (int)(nu & ((1u << m0) - 1)); nu >>= m0;
                const int nwq1 = (int)(nu & ((1u << wb) - 1)); nu >>= wb;
                const int nsg2 = (int)(nu & ((1u << m0) - 1)); nu >>= m0;
                const int nwq2 = (int)nu;
                const int nd0 = L.gout.base + ntile * L.V;
                const int nsmax = (nsg1 << G) + (nsg2 << G) + 2 * (R - 1);
                if (nd0 + L.V > 2 * N - nsmax) {
                    const int u1 = threadIdx.x % R, u2 = threadIdx.x / R;
                    const int q = nd0 + nsg2 * u2 + nsg1 * u1;
                    // the loads read [q rounded down to 16 bytes, + WT + 16 bytes)
                    const int lo = max(q & ~(EA - 1), L.gin.base), hi = min(lo + WT + 2 * EA, L.dmax);
                    const FusedSlot& ns = L.slot[nsl];
                    const bool nswap = ns.swap != 0;
                    const int nrs1 = nswap ? 1 : N, nrs2 = nswap ? N : 1;
                    const long long row = (long long)(nsg1 + (u1 << m0) + (nwq1 << (m0 + G))) * nrs1 +
                                          (long long)(nsg2 + (u2 << m0) + (nwq2 << (m0 + G))) * nrs2;
                    if (lo < hi)
                        tma::prefetch_l2(static_cast<const TIn*>(ns.in) + row * L.gin.pitch + (lo - L.gin.base),
                                         (uint32_t)(hi - lo) * (uint32_t)sizeof(TIn));
                }
            }
        }
    }

    if constexpr (TMA) {
        // Stage every group's rows: one 1-row box per (u2, u1); a group whose
        // windows all miss the stored range issues nothing (its warp parks
        // zeros below, the same test decides both).  A group's barrier is
        // used by its own warp only (initialised, armed, waited on and
        // retired there), so no block-wide barrier precedes the loads.
        if (active) {
            if (lane == 0) {
#pragma unroll 1
                for (int gi = 0; gi < GPW; ++gi) tma::mbar_init(&mbar[warp + gi * NW], 1);
                tma::fence_barrier_init();
            }
            __syncwarp();
#pragma unroll 1
            for (int gi = 0; gi < GPW; ++gi) {
                const int u2 = warp + gi * NW;
                const int g_lo = d0 + sg2 * u2, g_hi = g_lo + sg1 * (R - 1) + WT + 4;
                if (g_hi <= L.gin.base || g_lo >= L.dmax) continue;
                if (lane == 0) tma::mbar_arrive_expect_tx(&mbar[u2], R * Stage<TIn>::ELEMS * (int)sizeof(TIn));
                __syncwarp();
                if (lane < R) {
                    if constexpr (COHERENT) tma::fence_proxy_async_global();  // rows other CTAs wrote
                    const int u1 = lane;
                    const int a2 = sg2 + (u2 << m0) + (wq2 << (m0 + G));
                    const long long row =
                        (long long)(sg1 + (wq1 << (m0 + G))) * rs1 + (long long)a2 * rs2 + (long long)(u1 * rs1 << m0);
                    const int q = g_lo + sg1 * u1;
                    unsigned char* dst = smem_raw + (size_t)u2 * GB * sizeof(TS) + u1 * Stage<TIn>::ROW_BYTES;
                    constexpr int EA = 16 / (int)sizeof(TIn);  // elements per 16 bytes
                    tma::load_3d(dst, tmap, (q & ~(EA - 1)) - L.gin.base, (int)row, slot_z, &mbar[u2]);
                }
            }
        }
    }

    // ---------------- phase 1: transform along axis 1, warp = u2 ----------
#pragma unroll 1
    for (int gi = 0; gi < (active ? GPW : 0); ++gi) {
        const int u2 = warp + gi * NW;
        const int a2 = sg2 + (u2 << m0) + (wq2 << (m0 + G));
        const int start = d0 + sg2 * u2 + lane * K;
        T v[R][K];
        if constexpr (INGEST) {
            // m0 == 0 here: no shear, rows a1 = u1 + (wq1 << G).
            const TIn* vol = static_cast<const TIn*>(sp.in);
            const int z0 = start - 2 * N;
            const long long sx = swap ? sp.map.sy : sp.map.sx;   // stride of the phase-1 axis
            const long long s2 = swap ? sp.map.sx : sp.map.sy;   // stride of the phase-2 axis
            const long long rowbase = sp.map.o0 + (long long)a2 * s2 + (long long)(wq1 << G) * sx;
            if (sp.mode == kIngestZ) {
                // K consecutive z' of each row are contiguous (stride +-1).
                const bool in = z0 >= 0 && z0 < N;
                const int zc = in ? z0 : 0;  // clamp: always a valid, aligned address
#pragma unroll
                for (int u1 = 0; u1 < R; ++u1) {
                    TIn e[K];
                    {
                        const long long b = rowbase + (long long)u1 * sx + (long long)zc * sp.map.sz;
                        load_run<TIn, K>(vol + (sp.reverse ? b - (K - 1) : b), e);
                    }
#pragma unroll
                    for (int i = 0; i < K; ++i)
                        v[u1][i] = in ? to_acc<TIn, T>(sp.reverse ? e[K - 1 - i] : e[i]) : T(0);
                }
            } else if (sp.mode == kIngestRun) {
                // The R rows of the block are contiguous at every z'.
#pragma unroll
                for (int i = 0; i < K; ++i) {
                    const int z = z0 + i;
                    TIn e[R];
                    const bool in = z >= 0 && z < N;
                    {
                        const long long b = rowbase + (long long)(in ? z : 0) * sp.map.sz;
                        load_run<TIn, R>(vol + (sp.reverse ? b - (R - 1) : b), e);
                    }
#pragma unroll
                    for (int u1 = 0; u1 < R; ++u1)
                        v[u1][i] = in ? to_acc<TIn, T>(sp.reverse ? e[R - 1 - u1] : e[u1]) : T(0);
                }
            } else {
#pragma unroll
                for (int u1 = 0; u1 < R; ++u1)
#pragma unroll
                    for (int i = 0; i < K; ++i) {
                        const int z = z0 + i;
                        v[u1][i] = (z >= 0 && z < N)
                                       ? to_acc<TIn, T>(vol[rowbase + (long long)u1 * sx + (long long)z * sp.map.sz])
                                       : T(0);
                    }
            }
        } else {
            // A group whose sheared windows all miss the stored range [base, dmax)
            // reads only zeros: park zeros and skip the loads and the transform.
            const int g_lo = d0 + sg2 * u2, g_hi = g_lo + sg1 * (R - 1) + WT + 4;
            if (g_hi <= L.gin.base || g_lo >= L.dmax) {
                if (lane * K < WS) {
#pragma unroll
                    for (int t1 = 0; t1 < R; ++t1) {
                        TS* dst = S + (u2 * GB + t1 * WS + lane * K);
#pragma unroll
                        for (int i = 0; i < K; ++i) dst[i] = TS(0);
                    }
                }
                if constexpr (TMA) {
                    if (lane == 0) tma::mbar_inval(&mbar[u2]);  // never armed
                }
                continue;
            }
            const TIn* buf = static_cast<const TIn*>(sp.in);
            const long long row0 = (long long)(sg1 + (wq1 << (m0 + G))) * rs1 + (long long)a2 * rs2;
            const long long rstep = (long long)rs1 << m0;  // rows between u1 and u1 + 1
            if constexpr (TMA) {
                // Wait for the group's staged rows, then read each lane's 4
                // elements at the row's offset inside its 16-byte-aligned box.
                const bool landed = tma::mbar_wait(&mbar[u2], 0, kTmaWaitNs);
                if (!landed && L.status) atomicCAS(L.status, 0, (int)DRT3D_ERR_TIMEOUT);
                // Retire the group's barrier once every lane has seen it
                // complete (after a time-out a load may still be pending:
                // leave it).
                if (__all_sync(0xffffffffu, landed) && lane == 0) tma::mbar_inval(&mbar[u2]);
                const int a = sg1 & 3, c = g_lo & 3;
                if constexpr (sizeof(TIn) == 2) {
                    // Two 8-byte reads per row from the 4-aligned element below
                    // the window; the in-chunk offset repeats with u1 mod 4 (as
                    // for the register path) and is unpacked at a compile-time
                    // offset.
                    // Each row's words are read at a compile-time offset per
                    // class; the odd rows also supply the element past the
                    // lane's window, which stage 0 takes instead of a shuffle.
                    const uint16_t* st = reinterpret_cast<const uint16_t*>(smem_raw + (size_t)u2 * GB * sizeof(TS));
                    T nxt[R / 2];
                    stage_class_u16<0, G>(c, st, g_lo, sg1, lane, v, nxt);
                    stage_class_u16<1, G>((c + a) & 3, st, g_lo, sg1, lane, v, nxt);
                    stage_class_u16<2, G>((c + 2 * a) & 3, st, g_lo, sg1, lane, v, nxt);
                    stage_class_u16<3, G>((c + 3 * a) & 3, st, g_lo, sg1, lane, v, nxt);
                    __syncwarp();  // the group's results overwrite its staging
                    fwd_stage0_nxt<G, K>(v, nxt);
                } else {
                    // 32-bit rows: one or two 16-byte reads per row at the
                    // lane's chunk, taken by residue class at a compile-time
                    // offset.
                    const uint32_t* st = reinterpret_cast<const uint32_t*>(smem_raw + (size_t)u2 * GB * sizeof(TS));
                    T nxt[R / 2];
                    stage_class_u32<0, G>(c, st, lane, v, nxt);
                    stage_class_u32<1, G>((c + a) & 3, st, lane, v, nxt);
                    stage_class_u32<2, G>((c + 2 * a) & 3, st, lane, v, nxt);
                    stage_class_u32<3, G>((c + 3 * a) & 3, st, lane, v, nxt);
                    __syncwarp();  // the group's results overwrite its staging
                    fwd_stage0_nxt<G, K>(v, nxt);
                }
            } else if constexpr (sizeof(TIn) == 2) {
                const int L0 = start - L.gin.base;  // window offset of row u1 = 0
                const int width = L.dmax - L.gin.base;
                const long long step = rstep * L.gin.pitch + sg1;  // window step per u1
                const uint16_t* q0 = reinterpret_cast<const uint16_t*>(buf) + row0 * L.gin.pitch + L0;
                const int a = sg1 & 3, c = L0 & 3;
                Chunks16 w[R];
#pragma unroll
                for (int j = 0; j < (R < 4 ? R : 4); ++j) {
                    const int rr = (c + a * j) & 3;
                    const uint16_t* pj = q0 + (long long)j * step - rr;
                    const int lo_j = L0 + j * sg1 - rr;
#pragma unroll
                    for (int u1 = j; u1 < R; u1 += 4)
                        w[u1] = load_pair_u16<COHERENT>(pj + (long long)(u1 - j) * step, lo_j + (u1 - j) * sg1, width);
                }
                unpack_class_u16<0, G>(c, w, v);
                if constexpr (R > 1) unpack_class_u16<1, G>((c + a) & 3, w, v);
                if constexpr (R > 2) unpack_class_u16<2, G>((c + 2 * a) & 3, w, v);
                if constexpr (R > 3) unpack_class_u16<3, G>((c + 3 * a) & 3, w, v);
            } else {
                // Issue the loads of up to 8 x 32-bit rows, then extract.
                constexpr int BATCH = R < 8 ? R : 8;
#pragma unroll
                for (int b0 = 0; b0 < R; b0 += BATCH) {
                    ChunksOf<TIn> w[BATCH];
#pragma unroll
                    for (int j = 0; j < BATCH; ++j) {
                        const int u1 = b0 + j;
                        const TIn* rowp = buf + (row0 + u1 * rstep) * L.gin.pitch;
                        w[j] = load_chunks<TIn, COHERENT>(rowp, L.gin.base, L.dmax, start + sg1 * u1);
                    }
#pragma unroll
                    for (int j = 0; j < BATCH; ++j) {
                        const int u1 = b0 + j;
                        extract4<TIn, T>(w[j], (start + sg1 * u1) & 3, v[u1]);
                    }
                }
            }
        }
        if constexpr (TMA) fwd_all<G, K, 1>(v);  // stage 0 done with the staged reads
        else fwd_all<G, K>(v);
        if (lane * K < WS) {
#pragma unroll
            for (int t1 = 0; t1 < R; ++t1) {
                TS* dst = S + (u2 * GB + t1 * WS + lane * K);
                TS e[K];
#pragma unroll
                for (int i = 0; i < K; ++i) e[i] = (TS)v[t1][i];
                if constexpr (sizeof(TS) == 4) {
                    uint4 w;
                    memcpy(&w, e, 16);
                    *reinterpret_cast<uint4*>(dst) = w;
                } else {
                    uint2 w;
                    memcpy(&w, e, 8);
                    *reinterpret_cast<uint2*>(dst) = w;
                }
            }
        }
    }
    __syncthreads();

    // ---------------- phase 2: transform along axis 2, warp = t1 ----------
    float sq = 0.f;
#pragma unroll 1
    for (int gi = 0; gi < (active ? GPW : 0); ++gi) {
        const int t1 = warp + gi * NW;
        T v[R][K];
#pragma unroll
        for (int u2 = 0; u2 < R; ++u2) {
            // lanes past WS read the next row (or the pad): values they feed are invalid
            const TS* src = S + (u2 * GB + t1 * WS + lane * K);
            TS e[K];
            if constexpr (sizeof(TS) == 4) {
                uint4 w = *reinterpret_cast<const uint4*>(src);
                memcpy(e, &w, 16);
            } else {
                uint2 w = *reinterpret_cast<const uint2*>(src);
                memcpy(e, &w, 8);
            }
#pragma unroll
            for (int i = 0; i < K; ++i) v[u2][i] = (T)e[i];
        }
        fwd_all<G, K>(v);
        sq += store_rows<TOut, T, G, SQ>(L, sp, v, t1, sg1, wq1, sg2, wq2, rs1, rs2, d0, lane);
    }
    if constexpr (SQ) write_cta_sq<NW>(sp.sq + cta, sq);
}

// ---------------------------------------------------------------------------
// First pass of a uint8 volume with two row groups per register.
//
// With G = 4 every phase-1 value is a sum of at most 16 voxels (<= 4080) and
// every phase-2 value a sum of at most 256 (<= 65280): both fit 16 bits.  A
// warp's two phase-1 groups (u2 = warp, warp + 8) see identical shifts (the
// shear is applied by the loads, and it is zero at m0 = 0), and so do its two
// phase-2 groups (t1 = warp, warp + 8).  So each 32-bit register carries one
// value of each group, low and high half, and one 32-bit add adds both with no
// carry between the halves: half the adds and shuffles of the plain path.

// [A_e0, 0, B_e0, 0] and [A_e1, 0, B_e1, 0] from t = [A_e0, B_e0, A_e1, B_e1].
__device__ __forceinline__ uint32_t spread_lo(uint32_t t) { return __byte_perm(t, 0u, 0x4140); }
__device__ __forceinline__ uint32_t spread_hi(uint32_t t) { return __byte_perm(t, 0u, 0x4342); }

template <typename TOut, int G>
__device__ __forceinline__ void store_rows_x2(const FusedLaunch& L, const FusedSlot& sp,
                                              const uint32_t (&v)[1 << G][K], int t1A, int t1B, int wq1, int wq2,
                                              int rs1, int rs2, int d0, int lane) {
    constexpr int R = 1 << G;
    const int p0 = lane * K;
    const int d = d0 + p0;
    if (p0 >= L.V || d >= L.dmax) return;
    // m0 = 0: slopes so far are zero
    TOut* out = static_cast<TOut*>(sp.out) + (d - L.gout.base);
    const long long colr = (long long)(wq2 << G) * rs2;
    const long long rstride = (long long)rs2 * L.gout.pitch;
    TOut* dA = out + ((long long)(t1A + (wq1 << G)) * rs1 + colr) * L.gout.pitch;
    TOut* dB = out + ((long long)(t1B + (wq1 << G)) * rs1 + colr) * L.gout.pitch;
    if (L.vec_store) {
#pragma unroll
        for (int t2 = 0; t2 < R; ++t2, dA += rstride, dB += rstride) {
            if constexpr (sizeof(TOut) == 2) {
                st_global(reinterpret_cast<uint2*>(dA), make_uint2(__byte_perm(v[t2][0], v[t2][1], 0x5410),
                                                                   __byte_perm(v[t2][2], v[t2][3], 0x5410)));
                st_global(reinterpret_cast<uint2*>(dB), make_uint2(__byte_perm(v[t2][0], v[t2][1], 0x7632),
                                                                   __byte_perm(v[t2][2], v[t2][3], 0x7632)));
            } else {
                st_global(reinterpret_cast<uint4*>(dA), make_uint4(v[t2][0] & 0xFFFFu, v[t2][1] & 0xFFFFu,
                                                                   v[t2][2] & 0xFFFFu, v[t2][3] & 0xFFFFu));
                st_global(reinterpret_cast<uint4*>(dB), make_uint4(v[t2][0] >> 16, v[t2][1] >> 16, v[t2][2] >> 16,
                                                                   v[t2][3] >> 16));
            }
        }
    } else {
#pragma unroll
        for (int t2 = 0; t2 < R; ++t2, dA += rstride, dB += rstride)
#pragma unroll
            for (int i = 0; i < K; ++i)
                if (d + i < L.dmax) {
                    st_global(dA + i, (TOut)(v[t2][i] & 0xFFFFu));
                    st_global(dB + i, (TOut)(v[t2][i] >> 16));
                }
    }
}

template <typename TOut, int G>
__device__ __forceinline__ void fused_cta_u8x2(const FusedLaunch& L, const FusedSlot& sp, unsigned cta,
                                               unsigned char* smem_raw) {
    static_assert(G == 4, "two groups per warp needs G = 4");
    constexpr int R = 1 << G;
    constexpr int NW = fused_warps<G>();
    constexpr int WS = fused_ws<G>();
    uint16_t* S = reinterpret_cast<uint16_t*>(smem_raw);  // [u2][t1][WS] (+ pad)
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int N = L.N;
    const unsigned ntiles = (unsigned)L.ntiles;
    unsigned unit = cta / ntiles;
    const int tile = (int)(cta - unit * ntiles);
    const int wb = L.n - G;  // m0 = 0
    const int wq1 = (int)(unit & ((1u << wb) - 1));
    const int wq2 = (int)(unit >> wb);
    const int d0 = L.gout.base + tile * L.V;
    const bool swap = sp.swap != 0;
    const int rs1 = swap ? 1 : N, rs2 = swap ? N : 1;

    if (d0 + L.V <= 2 * N - 2 * (R - 1)) {  // all-zero tile (slopes so far are zero)
        uint32_t z[R][K];
#pragma unroll
        for (int r = 0; r < R; ++r)
#pragma unroll
            for (int i = 0; i < K; ++i) z[r][i] = 0u;
        store_rows_x2<TOut, G>(L, sp, z, warp, warp + NW, wq1, wq2, rs1, rs2, d0, lane);
        return;
    }

    // ---- phase 1: groups u2 = warp (low halves) and warp + 8 (high halves)
    {
        const uint8_t* vol = static_cast<const uint8_t*>(sp.in);
        const int z0 = d0 + lane * K - 2 * N;
        const long long sx = swap ? sp.map.sy : sp.map.sx;  // stride of the phase-1 axis
        const long long s2 = swap ? sp.map.sx : sp.map.sy;  // stride of the phase-2 axis
        const long long rowA = sp.map.o0 + (long long)(warp + (wq2 << G)) * s2 + (long long)(wq1 << G) * sx;
        const long long offB = (long long)NW * s2;
        // byte selectors pairing element i of A with element i of B, in load order
        const uint32_t sel0 = sp.reverse ? 0x6273u : 0x5140u;
        const uint32_t sel1 = sp.reverse ? 0x4051u : 0x7362u;
        uint32_t v[R][K];
        if (sp.mode == kIngestZ) {
            const bool in = z0 >= 0 && z0 < N;
            const int zc = in ? z0 : 0;
#pragma unroll
            for (int u1 = 0; u1 < R; ++u1) {
                long long b = rowA + (long long)u1 * sx + (long long)zc * sp.map.sz;
                if (sp.reverse) b -= K - 1;
                uint32_t wA = __ldg(reinterpret_cast<const unsigned*>(vol + b));
                uint32_t wB = __ldg(reinterpret_cast<const unsigned*>(vol + b + offB));
                wA = in ? wA : 0u;
                wB = in ? wB : 0u;
                const uint32_t t0 = __byte_perm(wA, wB, sel0), t1 = __byte_perm(wA, wB, sel1);
                v[u1][0] = spread_lo(t0);
                v[u1][1] = spread_hi(t0);
                v[u1][2] = spread_lo(t1);
                v[u1][3] = spread_hi(t1);
            }
        } else if (sp.mode == kIngestRun) {
#pragma unroll
            for (int i = 0; i < K; ++i) {
                const int z = z0 + i;
                const bool in = z >= 0 && z < N;
                long long b = rowA + (long long)(in ? z : 0) * sp.map.sz;
                if (sp.reverse) b -= R - 1;
                uint4 qa = __ldg(reinterpret_cast<const uint4*>(vol + b));
                uint4 qb = __ldg(reinterpret_cast<const uint4*>(vol + b + offB));
                uint32_t wa[4] = {qa.x, qa.y, qa.z, qa.w}, wbv[4] = {qb.x, qb.y, qb.z, qb.w};
#pragma unroll
                for (int wi = 0; wi < 4; ++wi) {
                    // rows 4 wi .. 4 wi + 3: word wi, or word 3 - wi read backwards
                    const uint32_t a = in ? (sp.reverse ? wa[3 - wi] : wa[wi]) : 0u;
                    const uint32_t bb = in ? (sp.reverse ? wbv[3 - wi] : wbv[wi]) : 0u;
                    const uint32_t t0 = __byte_perm(a, bb, sel0), t1 = __byte_perm(a, bb, sel1);
                    v[4 * wi][i] = spread_lo(t0);
                    v[4 * wi + 1][i] = spread_hi(t0);
                    v[4 * wi + 2][i] = spread_lo(t1);
                    v[4 * wi + 3][i] = spread_hi(t1);
                }
            }
        } else {
#pragma unroll
            for (int u1 = 0; u1 < R; ++u1)
#pragma unroll
                for (int i = 0; i < K; ++i) {
                    const int z = z0 + i;
                    const bool in = z >= 0 && z < N;
                    const long long b = rowA + (long long)u1 * sx + (long long)(in ? z : 0) * sp.map.sz;
                    const uint32_t a = in ? (uint32_t)vol[b] : 0u;
                    const uint32_t bb = in ? (uint32_t)vol[b + offB] : 0u;
                    v[u1][i] = a | (bb << 16);
                }
        }
        fwd_all<G, K>(v);
        if (lane * K < WS) {
#pragma unroll
            for (int t1 = 0; t1 < R; ++t1) {
                const uint2 lo = make_uint2(__byte_perm(v[t1][0], v[t1][1], 0x5410), __byte_perm(v[t1][2], v[t1][3], 0x5410));
                const uint2 hi = make_uint2(__byte_perm(v[t1][0], v[t1][1], 0x7632), __byte_perm(v[t1][2], v[t1][3], 0x7632));
                *reinterpret_cast<uint2*>(S + ((warp * R + t1) * WS + lane * K)) = lo;
                *reinterpret_cast<uint2*>(S + (((warp + NW) * R + t1) * WS + lane * K)) = hi;
            }
        }
    }
    __syncthreads();

    // ---- phase 2: t1 = warp (low halves) and warp + 8 (high halves)
    {
        uint32_t v[R][K];
#pragma unroll
        for (int u2 = 0; u2 < R; ++u2) {
            // lanes past WS read the next row (or the pad): values they feed are invalid
            const uint2 a = *reinterpret_cast<const uint2*>(S + ((u2 * R + warp) * WS + lane * K));
            const uint2 b = *reinterpret_cast<const uint2*>(S + ((u2 * R + warp + NW) * WS + lane * K));
            v[u2][0] = __byte_perm(a.x, b.x, 0x5410);
            v[u2][1] = __byte_perm(a.x, b.x, 0x7632);
            v[u2][2] = __byte_perm(a.y, b.y, 0x5410);
            v[u2][3] = __byte_perm(a.y, b.y, 0x7632);
        }
        fwd_all<G, K>(v);
        store_rows_x2<TOut, G>(L, sp, v, warp, warp + NW, wq1, wq2, rs1, rs2, d0, lane);
    }
}

}  // namespace fused
}  // namespace drt3d
