// api.cu -- the extern "C" boundary of libdrt3d: plans, argument checks,
// workspace carving and the pass schedules of the planes transforms.
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <algorithm>
#include <new>

#include "internal.cuh"
#include "adjoint_sum.cuh"

namespace drt3d {

// Algorithm 2's InOrder table with the reading documented in drt3d.h: new
// axis i of dodecant k is original axis |e_i| - 1, and original axis a is
// reversed when its own entry e_a is negative.  Rows 5, 6, 9, 10 carry the
// single-sign corrections that make the twelve sectors distinct.
static const int kInOrder[12][3] = {
    {1, 2, 3},   {-2, 1, 3},  {-1, -2, 3}, {2, -1, 3},   {-1, -3, -2}, {-3, 1, 2},
    {3, -1, 2},  {1, 3, -2},  {-3, -2, -1}, {2, -3, 1},  {-2, 3, 1},   {3, 2, -1},
};

Affine dodecant_affine(int N, int k) {
    const long long stride[3] = {(long long)N * N, (long long)N, 1};
    long long s[3];
    Affine A{0, 0, 0, 0};
    for (int i = 0; i < 3; ++i) {
        const int a = std::abs(kInOrder[k][i]) - 1;
        if (kInOrder[k][a] < 0) {
            A.o0 += (long long)(N - 1) * stride[a];
            s[i] = -stride[a];
        } else {
            s[i] = stride[a];
        }
    }
    A.sx = s[0];
    A.sy = s[1];
    A.sz = s[2];
    return A;
}

Affine sector_affine(int N, int k) {
    const long long stride[3] = {(long long)N * N, (long long)N, 1};
    const int a = k >> 2, flips = k & 3;
    Affine A{0, stride[a], 0, 0};
    const int b = (a + 1) % 3, c = (a + 2) % 3;
    if (flips & 1) { A.o0 += (long long)(N - 1) * stride[b]; A.sy = -stride[b]; }
    else A.sy = stride[b];
    if (flips & 2) { A.o0 += (long long)(N - 1) * stride[c]; A.sz = -stride[c]; }
    else A.sz = stride[c];
    return A;
}

static Geo planes_geo(int N, int mx, int my) {
    const int lo = 2 * N + 2 - (1 << mx) - (1 << my);
    Geo g;
    g.base = lo & ~7;
    g.pitch = (int)align_up((size_t)(3 * N - g.base), 8);
    return g;
}

static ElemKind kind_of(drt3d_dtype d) {
    switch (d) {
    case DRT3D_U8: return ElemKind::U8;
    case DRT3D_I16: return ElemKind::I16;
    case DRT3D_I32: return ElemKind::I32;
    default: return ElemKind::F32;
    }
}

bool make_fused_schedule_groups(int N, drt3d_dtype dtype, int ng, const int* G, FusedSchedule* out) {
    FusedSchedule S{};
    if (ng < 1 || ng > 8) return false;
    int m = 0;
    size_t maxb = 0;
    for (int g = 0; g < ng; ++g) {
        if (G[g] < 1 || G[g] > 4) return false;
        FusedPass& P = S.pass[g];
        P.G = G[g];
        P.m0 = m;
        P.ingest = (g == 0);
        P.in = (g == 0) ? Geo{0, 0} : S.pass[g - 1].out;
        P.in_kind = (g == 0) ? kind_of(dtype) : S.pass[g - 1].out_kind;
        m += P.G;
        P.final_ = (g == ng - 1);
        if (P.final_) {
            P.out = Geo{0, 3 * N};
            P.out_kind = dtype == DRT3D_F32 ? ElemKind::F32 : ElemKind::I32;
        } else {
            P.out = planes_geo(N, m, m);
            // u8 volumes: every intermediate value is a sum of 4^m voxels of at
            // most 255, so it is exact in 16 bits while 255 * 4^m < 2^16.
            if (dtype == DRT3D_U8 && 255L * (1L << (2 * m)) <= 65535L) P.out_kind = ElemKind::U16;
            else P.out_kind = dtype == DRT3D_F32 ? ElemKind::F32 : ElemKind::I32;
            const size_t b = align_up((size_t)N * N * P.out.pitch * elem_bytes(P.out_kind), 256);
            if (b > maxb) maxb = b;
        }
    }
    if ((1 << m) != N) return false;
    S.npass = ng;
    S.buf_bytes = maxb;
    *out = S;
    return true;
}

// Default split: ceil(n / 4) groups of near-equal size, larger ones first.
FusedSchedule make_fused_schedule(int N, drt3d_dtype dtype) {
    const int n = ilog2(N);
    const int ng = (n + 3) / 4;
    int G[8];
    for (int g = 0; g < ng; ++g) G[g] = n / ng + (g < n % ng ? 1 : 0);
    FusedSchedule S{};
    make_fused_schedule_groups(N, dtype, ng, G, &S);
    return S;
}

// Ingest mode of dodecant k's first pass (see planes_fused.cu).
void fused_ingest_mode(int N, const Affine& A, FusedSlot& fs) {
    fs.swap = 0;
    fs.reverse = 0;
    fs.mode = kIngestGeneric;
    if (N >= 4 && (A.sz == 1 || A.sz == -1)) {
        fs.mode = kIngestZ;
        fs.reverse = A.sz < 0;
    } else if (A.sx == 1 || A.sx == -1) {
        fs.mode = kIngestRun;
        fs.reverse = A.sx < 0;
    } else if (A.sy == 1 || A.sy == -1) {
        fs.mode = kIngestRun;
        fs.swap = 1;
        fs.reverse = A.sy < 0;
    }
}

// Exact-inverse schedule: per axis the n stages are undone in groups of at
// most Gmax (so a unit's rows over the full 3N range fit in shared memory),
// last group first, the s2 axis before the s1 axis within each group.
struct InvStep { int axis, G, m0, mx_in, my_in, mx_out, my_out; };
static int inverse_steps(int N, InvStep* steps) {
    const int n = ilog2(N);
    const int gmax = N <= 512 ? 4 : 3;
    const int ng = (n + gmax - 1) / gmax;
    int sz[12], M[13];
    M[0] = 0;
    for (int g = 0; g < ng; ++g) {
        sz[g] = n / ng + (g < n % ng ? 1 : 0);
        M[g + 1] = M[g] + sz[g];
    }
    int c = 0;
    for (int g = ng - 1; g >= 0; --g) {
        steps[c++] = InvStep{1, sz[g], M[g], M[g + 1], M[g + 1], M[g + 1], M[g]};
        steps[c++] = InvStep{0, sz[g], M[g], M[g + 1], M[g], M[g], M[g]};
    }
    return c;
}

// Inverse intermediates: base rounded down to 32 so that (for N >= 32) rows
// are whole 32-element chunks of the inverse kernel.
static Geo inv_geo(int N, int mx, int my) {
    if (mx == ilog2(N) && my == ilog2(N)) return Geo{0, 3 * N};
    const int lo = 2 * N + 2 - (1 << mx) - (1 << my);
    Geo g;
    g.base = lo & ~31;
    g.pitch = (int)align_up((size_t)(3 * N - g.base), 8);
    return g;
}

static size_t inverse_buf_bytes(int N) {
    InvStep st[24];
    const int c = inverse_steps(N, st);
    size_t mx = 0;
    for (int i = 0; i + 1 < c; ++i) {
        const Geo g = inv_geo(N, st[i].mx_out, st[i].my_out);
        mx = std::max(mx, align_up((size_t)N * N * g.pitch * 4, 256));
    }
    return mx;
}

// Lines schedule: n <= 4 in one pass, else two passes (ceil(n/2), floor(n/2)),
// the larger first so that the last (output-writing) pass keeps G <= 3 and
// one warp tile spans a whole output row where possible.
static int djt_groups(int N, int* G) {
    const int n = ilog2(N);
    if (n <= 4) { G[0] = n; return 1; }
    G[0] = (n + 1) / 2;
    G[1] = n / 2;
    return 2;
}
static int djt_base(int N, int m) { return (N + 1 - (1 << m)) & ~3; }
// Lines forward: the volume rearranged into the frames of the y- and
// z-driven sectors (x' = y, y' = z, z' = x and x' = z, y' = x, z' = y), so
// that every sector's ingest reads runs of z' contiguously.  One copy each.
static size_t djt_frame_copy_bytes(int N, drt3d_dtype dt) {
    const size_t esz = dt == DRT3D_U8 ? 1 : dt == DRT3D_I16 ? 2 : 4;
    return align_up((size_t)N * N * N * esz, 256);
}

static size_t djt_buf_bytes(int N) {
    int G[2];
    if (djt_groups(N, G) < 2) return 0;
    const int n = ilog2(N), m = G[0];
    const long long pitch = 2LL * N - djt_base(N, m);
    return align_up((size_t)(1LL << (n + m)) * pitch * pitch * 4, 256);
}

// Lines adjoint: stage m's window [base_m, 2N)^2 (full at m = n), rows
// 2^(n + m); per slot two buffers for the alternating stages n-1, n-2, ...
static int djt_adj_base(int N, int m) { return m >= ilog2(N) ? 0 : djt_base(N, m); }
static size_t djt_adj_stage_bytes(int N, int m) {
    const long long pitch = 2LL * N - djt_adj_base(N, m);
    return align_up((size_t)(1LL << (ilog2(N) + m)) * pitch * pitch * 4, 256);
}
static size_t djt_adj_slot_bytes(int N) {
    const int n = ilog2(N);
    return djt_adj_stage_bytes(N, n - 1) + (n >= 2 ? djt_adj_stage_bytes(N, n - 2) : 0);
}

// One intermediate buffer of the planes adjoint: a fused pass's 32-bit rows,
// or the dodecant's frame volume that the last pass writes.
static const FusedSchedule& adjoint_schedule(const drt3d_plan* P) { return P->has_adj ? P->adj : P->fused; }

// Partial sums of the squared residual that the final forward pass writes for
// one dodecant slot (drt3d_planes_forward_residual_loss): one per CTA of that
// pass.
static long long residual_partials_per_slot(const drt3d_plan* P) {
    const FusedPass& ps = P->fused.pass[P->fused.npass - 1];
    const int V = fused_valid(ps.G);
    const long long ntiles = (3LL * P->N - ps.out.base + V - 1) / V;
    const long long per_axis = 1LL << (P->n - ps.G);
    return per_axis * per_axis * ntiles;
}

static size_t adjoint_buf_bytes(const drt3d_plan* P) {
    return std::max(adjoint_schedule(P).buf_bytes, align_up((size_t)P->N * P->N * P->N * 4, 256));
}

static bool aligned16(const void* p) { return ((uintptr_t)p & 15u) == 0; }

static int popcount12(uint32_t m) {
    int c = 0;
    for (int k = 0; k < 12; ++k) c += (m >> k) & 1;
    return c;
}



// Profiling helpers: no-ops unless drt3d_set_profiling(plan, 1).
static void prof_begin(const drt3d_plan* P, cudaStream_t s, const char* name, double bytes) {
    Profiler& pr = P->prof;
    if (!pr.on || pr.count >= kMaxLaunch) return;
    cudaEventRecord(pr.ev[2 * pr.count], s);
    pr.bytes[pr.count] = bytes;
    std::snprintf(pr.name[pr.count], sizeof(pr.name[0]), "%s", name);
}
static void prof_end(const drt3d_plan* P, cudaStream_t s) {
    Profiler& pr = P->prof;
    if (!pr.on || pr.count >= kMaxLaunch) return;
    cudaEventRecord(pr.ev[2 * pr.count + 1], s);
    ++pr.count;
}

// Algorithmic bytes of one fused pass for one dodecant (compact rows read at
// their element size, or the volume; rows written at their element size).
static double fused_pass_bytes(const drt3d_plan* P, const FusedPass& ps) {
    const double N = P->N;
    const int m1 = ps.m0 + ps.G;
    const double lo_in = 2 * N + 2 - 2.0 * (1 << ps.m0);
    const double lo_out = 2 * N + 2 - 2.0 * (1 << m1);
    const double in_b = ps.ingest ? N * N * N * elem_bytes(ps.in_kind)
                                  : N * N * (3 * N - lo_in) * elem_bytes(ps.in_kind);
    const double out_b = ps.final_ ? N * N * 3 * N * 4.0 : N * N * (3 * N - lo_out) * elem_bytes(ps.out_kind);
    return in_b + out_b;
}

// 2D DRT of lines: the n stages split into ceil(n / 4) near-equal groups; the
// rows after m stages are stored over d in [base, 2N) (nothing below
// N + 1 - 2^m can be non-zero), base rounded down to 4, pitch up to 4.
static int drt2d_groups(int n, int* G) {
    const int ng = (n + 3) / 4;
    for (int g = 0; g < ng; ++g) G[g] = n / ng + (g < n % ng ? 1 : 0);
    return ng;
}
static int drt2d_base(int N, int m) { return m >= ilog2(N) ? 0 : (N + 1 - (1 << m)) & ~3; }
static int drt2d_pitch(int N, int m) { return (int)align_up((size_t)(2 * N - drt2d_base(N, m)), 4); }
// Bytes of one (image, quadrant) slot of the largest intermediate, and how
// many intermediates are live at once.
static size_t drt2d_slot_bytes(int N, int* nbuf) {
    int G[4];
    const int ng = drt2d_groups(ilog2(N), G);
    size_t mx = 0;
    for (int g = 0, m = 0; g + 1 < ng; ++g) {
        m += G[g];
        mx = std::max(mx, (size_t)N * drt2d_pitch(N, m) * 4);
    }
    *nbuf = ng <= 1 ? 0 : (ng == 2 ? 1 : 2);
    return mx;
}
// Images per chunk for a workspace of `ws` bytes (0 if none fits).
static long long drt2d_chunk(int N, int nq, int B, size_t ws) {
    int nbuf;
    const size_t slot = drt2d_slot_bytes(N, &nbuf);
    if (nbuf == 0) return std::min<long long>(B, 65535 / nq);
    const long long c = (long long)(ws / ((size_t)nbuf * nq * slot));
    return std::min<long long>(std::min<long long>(c, B), 65535 / nq);
}
// Default workspace: chunks whose intermediates stay near 32 MiB, so that a
// pass's output is still in L2 when the next pass reads it.
constexpr size_t kDrt2dChunkTarget = 32u << 20;
static int quad_count(uint32_t m) { return ((m >> 0) & 1) + ((m >> 1) & 1) + ((m >> 2) & 1) + ((m >> 3) & 1); }

}  // namespace drt3d

using namespace drt3d;

extern "C" {

int drt3d_version(void) { return 100; }

const char* drt3d_status_string(drt3d_status s) {
    switch (s) {
    case DRT3D_OK: return "DRT3D_OK";
    case DRT3D_ERR_INVALID_ARG: return "DRT3D_ERR_INVALID_ARG";
    case DRT3D_ERR_SIZE: return "DRT3D_ERR_SIZE";
    case DRT3D_ERR_DTYPE: return "DRT3D_ERR_DTYPE";
    case DRT3D_ERR_ALIGN: return "DRT3D_ERR_ALIGN";
    case DRT3D_ERR_WORKSPACE: return "DRT3D_ERR_WORKSPACE";
    case DRT3D_ERR_NOT_IN_RANGE: return "DRT3D_ERR_NOT_IN_RANGE";
    case DRT3D_ERR_TIMEOUT: return "DRT3D_ERR_TIMEOUT";
    case DRT3D_ERR_BOUNDS: return "DRT3D_ERR_BOUNDS";
    case DRT3D_ERR_CUDA: return "DRT3D_ERR_CUDA";
    case DRT3D_ERR_NO_MEMORY: return "DRT3D_ERR_NO_MEMORY";
    case DRT3D_ERR_SCRATCH_LIMIT: return "DRT3D_ERR_SCRATCH_LIMIT";
    }
    return "DRT3D_ERR_UNKNOWN";
}

drt3d_status drt3d_plan_create(drt3d_plan** plan, int N, drt3d_dtype in_dtype, unsigned flags) {
    if (!plan) return DRT3D_ERR_INVALID_ARG;
    *plan = nullptr;
    if (flags != 0) return DRT3D_ERR_INVALID_ARG;
    if (N < 2 || N > kMaxN || (N & (N - 1)) != 0) return DRT3D_ERR_SIZE;
    if (in_dtype != DRT3D_U8 && in_dtype != DRT3D_I16 && in_dtype != DRT3D_I32 && in_dtype != DRT3D_F32)
        return DRT3D_ERR_DTYPE;
    drt3d_plan* P = new (std::nothrow) drt3d_plan();
    if (!P) return DRT3D_ERR_NO_MEMORY;
    P->N = N;
    P->n = ilog2(N);
    P->dtype = in_dtype;
    P->flags = flags;
    if (cudaGetDevice(&P->device) != cudaSuccess) { delete P; return DRT3D_ERR_CUDA; }
    if (cudaMalloc(&P->d_status, sizeof(int)) != cudaSuccess) { delete P; return DRT3D_ERR_NO_MEMORY; }
    if (cudaMemset(P->d_status, 0, sizeof(int)) != cudaSuccess) {
        cudaFree(P->d_status);
        delete P;
        return DRT3D_ERR_CUDA;
    }
    P->fused = make_fused_schedule(N, in_dtype);
    *plan = P;
    return DRT3D_OK;
}

drt3d_status drt3d_plan_destroy(drt3d_plan* plan) {
    if (!plan) return DRT3D_OK;
    for (std::atomic<drt3d_plan*>& lp : plan->levels) drt3d_plan_destroy(lp.exchange(nullptr));
    if (plan->prof.events_made)
        for (int i = 0; i < 2 * kMaxLaunch; ++i) cudaEventDestroy(plan->prof.ev[i]);
    if (plan->d_status && !plan->borrowed_status) cudaFree(plan->d_status);
    delete plan;
    return DRT3D_OK;
}

drt3d_status drt3d_planes_out_shape(const drt3d_plan* P, int64_t dims[4]) {
    if (!P || !dims) return DRT3D_ERR_INVALID_ARG;
    dims[0] = 12; dims[1] = P->N; dims[2] = P->N; dims[3] = 3 * (int64_t)P->N;
    return DRT3D_OK;
}

drt3d_status drt3d_lines_out_shape(const drt3d_plan* P, int64_t dims[5]) {
    if (!P || !dims) return DRT3D_ERR_INVALID_ARG;
    dims[0] = 12; dims[1] = P->N; dims[2] = P->N; dims[3] = 2 * (int64_t)P->N; dims[4] = 2 * (int64_t)P->N;
    return DRT3D_OK;
}

// --------------------------------------------------------------------------
// Iterative inverse (Section 5.2): float32 plans of the coarser sizes and the
// workspace layout.
// --------------------------------------------------------------------------
static drt3d_plan* level_plan(const drt3d_plan* P, int l) {
    if (l == P->n) return const_cast<drt3d_plan*>(P);
    drt3d_plan* have = P->levels[l].load(std::memory_order_acquire);
    if (!have) {
        drt3d_plan* q = new (std::nothrow) drt3d_plan();
        if (!q) return nullptr;
        q->N = 1 << l;
        q->n = l;
        q->dtype = DRT3D_F32;
        q->flags = 0;
        q->device = P->device;
        q->d_status = P->d_status;
        q->borrowed_status = true;
        q->fused = make_fused_schedule(q->N, DRT3D_F32);
        if (P->levels[l].compare_exchange_strong(have, q, std::memory_order_acq_rel))
            return q;
        delete q;  // another thread installed the level first (`have` now holds it)
    }
    return have;
}

struct PressLayout {
    size_t r[11];  // restricted residual of each level 2^l (r[n]: top-level residual)
    size_t t;      // A x of the level being smoothed
    size_t x[11];  // solution of each level
    size_t b;      // backprojection
    size_t partial, norm;
    size_t tws;    // forward / adjoint workspace
    size_t tws_bytes;
    size_t total;
};
static PressLayout press_layout(const drt3d_plan* P) {
    PressLayout Lo{};
    const int N = P->N, n = P->n;
    size_t off = 0;
    auto take = [&](size_t bytes) {
        const size_t o = off;
        off += align_up(bytes, 256);
        return o;
    };
    for (int l = 0; l <= n; ++l) {
        const size_t L = (size_t)1 << l;
        Lo.r[l] = take(12 * L * L * 3 * L * 4);
    }
    Lo.t = take((size_t)12 * N * N * 3 * N * 4);
    for (int l = 0; l <= n; ++l) {
        const size_t L = (size_t)1 << l;
        Lo.x[l] = take(L * L * L * 4);
    }
    Lo.b = take((size_t)N * N * N * 4);
    Lo.partial = take(kPressNormParts * sizeof(double));
    Lo.norm = take(sizeof(double));
    Lo.tws_bytes = std::max((size_t)kMaxSlots * 2 * P->fused.buf_bytes, (size_t)kMaxSlots * 2 * adjoint_buf_bytes(P));
    Lo.tws = take(Lo.tws_bytes);
    Lo.total = off;
    return Lo;
}

drt3d_status drt3d_workspace_bytes(const drt3d_plan* P, int op, size_t* bytes) {
    if (!P || !bytes) return DRT3D_ERR_INVALID_ARG;
    switch (op) {
    case DRT3D_OP_PLANES_FORWARD:
    case DRT3D_OP_PLANES_ADJOINT:
        *bytes = (size_t)kMaxSlots * 2 * (op == DRT3D_OP_PLANES_FORWARD ? P->fused.buf_bytes : adjoint_buf_bytes(P));
        return DRT3D_OK;
    case DRT3D_OP_PLANES_INVERSE:
        *bytes = 2 * inverse_buf_bytes(P->N);
        return DRT3D_OK;
    case DRT3D_OP_PLANES_RESIDUAL_LOSS:
        *bytes = align_up((size_t)kMaxSlots * 2 * P->fused.buf_bytes, 256) +
                 (size_t)kMaxSlots * residual_partials_per_slot(P) * sizeof(double);
        return DRT3D_OK;
    case DRT3D_OP_LINES_FORWARD:
        *bytes = (size_t)kMaxSlots * djt_buf_bytes(P->N);
        if (*bytes) *bytes += 2 * djt_frame_copy_bytes(P->N, P->dtype);
        return DRT3D_OK;
    case DRT3D_OP_LINES_ADJOINT:
        *bytes = (size_t)kMaxSlots * djt_adj_slot_bytes(P->N);
        return DRT3D_OK;
    case DRT3D_OP_PLANES_PRESS:
        if (P->dtype != DRT3D_F32) return DRT3D_ERR_DTYPE;
        *bytes = press_layout(P).total;
        return DRT3D_OK;
    }
    return DRT3D_ERR_INVALID_ARG;
}

// Algorithm 2's output tables (OutOrder with 1-based dimension numbers, a
// negative entry flipping that output dimension after the permutation, and
// DodecantCoords), as printed in the paper.
static const int kOutOrder[12][2] = {{-2, -1}, {-1, 2}, {2, 1}, {1, -2}, {2, 1}, {1, -2},
                                     {-1, 2}, {-2, -1}, {2, 1}, {-1, 2}, {1, -2}, {-2, -1}};
static const int kDodecantCoords[12][2] = {{1, 1}, {1, 2}, {2, 2}, {2, 1}, {0, 2}, {0, 1},
                                           {3, 2}, {3, 1}, {2, 0}, {1, 0}, {2, 3}, {1, 3}};

// Row of dodecant k's (s1, s2) in the 4N x 4N global array, as
// g0 + s1 g1 + s2 g2: output dimension i takes (s1, s2)[|OutOrder[k][i]| - 1],
// reversed when the entry is negative, inside block DodecantCoords[k].
static void global_row_map(int N, int k, FusedSlot& fs) {
    long long c[2];
    long long a[2][2];  // a[i][j]: coefficient of (s1, s2)[j] in output index i
    for (int i = 0; i < 2; ++i) {
        const int e = kOutOrder[k][i];
        const int src = (e < 0 ? -e : e) - 1;
        a[i][0] = a[i][1] = 0;
        a[i][src] = e < 0 ? -1 : 1;
        c[i] = e < 0 ? N - 1 : 0;
    }
    const long long W = 4LL * N;
    fs.g0 = ((long long)kDodecantCoords[k][0] * N + c[0]) * W + (long long)kDodecantCoords[k][1] * N + c[1];
    fs.g1 = (int)(a[0][0] * W + a[1][0]);
    fs.g2 = (int)(a[0][1] * W + a[1][1]);
}

// d_sub: residual target of the final pass (or null); d_sq: with d_sub and a
// float32 plan, its per-CTA partial sums of the squared residual,
// residual_partials_per_slot per slot (or null).
static drt3d_status planes_forward_impl(const drt3d_plan* P, const void* d_in, void* d_out, uint32_t mask,
                                        void* d_ws, size_t ws_bytes, cudaStream_t stream, bool global,
                                        const void* d_sub = nullptr, double* d_sq = nullptr) {
    if (!P || !d_in || !d_out) return DRT3D_ERR_INVALID_ARG;
    if (d_sub && (global || !aligned16(d_sub))) return d_sub && global ? DRT3D_ERR_INVALID_ARG : DRT3D_ERR_ALIGN;
    if (!device_is_current(P->device)) return DRT3D_ERR_INVALID_ARG;
    if (mask == 0 || (mask & ~DRT3D_ALL_DODECANTS)) return DRT3D_ERR_INVALID_ARG;
    if (!aligned16(d_in) || !aligned16(d_out) || !aligned16(d_ws)) return DRT3D_ERR_ALIGN;
    const FusedSchedule& S = P->fused;
    const size_t buf = S.buf_bytes;
    const int nslots = popcount12(mask);
    if (S.npass > 1 && (!d_ws || ws_bytes < (size_t)nslots * 2 * buf)) return DRT3D_ERR_WORKSPACE;
    const int N = P->N;
    const size_t out_block = (size_t)N * N * 3 * N * 4;
    char* ws = static_cast<char*>(d_ws);
    FusedLaunch L{};
    L.N = N;
    L.n = P->n;
    L.dmax = 3 * N;
    L.status = P->d_status;
    for (int p = 0; p < S.npass; ++p) {
        const FusedPass& ps = S.pass[p];
        int i = 0;
        for (int k = 0; k < 12; ++k) {
            if (!((mask >> k) & 1)) continue;
            char* bufA = ws + (size_t)i * 2 * buf;
            char* bufB = bufA + buf;
            FusedSlot& fs = L.slot[i];
            fs.map = dodecant_affine(N, k);
            fused_ingest_mode(N, fs.map, fs);
            fs.in = (p == 0) ? d_in : ((p & 1) ? (const void*)bufA : (const void*)bufB);
            fs.out = ps.final_ ? (void*)(static_cast<char*>(d_out) + (global ? 0 : (size_t)i * out_block))
                               : ((p & 1) ? (void*)bufB : (void*)bufA);
            fs.sub = (ps.final_ && d_sub) ? (const void*)(static_cast<const char*>(d_sub) + (size_t)i * out_block)
                                          : nullptr;
            fs.sq = (ps.final_ && d_sub && d_sq) ? d_sq + (size_t)i * residual_partials_per_slot(P) : nullptr;
            if (global) global_row_map(N, k, fs);
            ++i;
        }
        L.m0 = ps.m0;
        L.gin = ps.in;
        L.gout = ps.out;
        L.V = fused_valid(ps.G);
        L.ntiles = (3 * N - ps.out.base + L.V - 1) / L.V;
        const long long per_axis = 1LL << (P->n - ps.G);
        L.ctas = per_axis * per_axis * L.ntiles;
        L.vec_store = (ps.out.pitch % 4 == 0) && (ps.out.base % 4 == 0) && (3 * N) % 4 == 0;
        L.global_layout = (global && ps.final_) ? 1 : 0;
        // Dispatch order of the slots alternates between passes, the last pass
        // last to first: each pass starts on the slots whose input the previous
        // pass wrote last (still in L2), and the first slot's output is the
        // freshest in L2 when the call ends (a round trip inverts dodecant 0
        // by default).
        L.reverse_slots = ((S.npass - 1 - p) & 1) == 0 ? 1 : 0;
        char nm[40];
        std::snprintf(nm, sizeof nm, "planes_fused G=%d m0=%d", ps.G, ps.m0);
        prof_begin(P, stream, nm, nslots * fused_pass_bytes(P, ps));
        cudaError_t e;
        if (fused_uses_tma(ps.G, ps.in_kind, ps.ingest))
            e = launch_planes_fused_tma(L, ps.G, ps.in_kind, ps.out_kind, L.slot[0].in, 2 * buf, nslots, stream);
        else
            e = launch_planes_fused(L, ps.G, ps.in_kind, ps.out_kind, ps.ingest, nslots, stream);
        if (e != cudaSuccess) return DRT3D_ERR_CUDA;
        prof_end(P, stream);
    }
    return DRT3D_OK;
}

drt3d_status drt3d_planes_forward(const drt3d_plan* P, const void* d_in, void* d_out, uint32_t mask,
                                  void* d_ws, size_t ws_bytes, cudaStream_t stream) {
    return planes_forward_impl(P, d_in, d_out, mask, d_ws, ws_bytes, stream, false);
}

drt3d_status drt3d_planes_forward_residual(const drt3d_plan* P, const void* d_in, const void* d_target, void* d_out,
                                           uint32_t mask, void* d_ws, size_t ws_bytes, cudaStream_t stream) {
    if (!d_target) return DRT3D_ERR_INVALID_ARG;
    return planes_forward_impl(P, d_in, d_out, mask, d_ws, ws_bytes, stream, false, d_target);
}

drt3d_status drt3d_planes_forward_residual_loss(const drt3d_plan* P, const void* d_in, const void* d_target,
                                                void* d_out, uint32_t mask, double* d_loss, void* d_ws,
                                                size_t ws_bytes, cudaStream_t stream) {
    if (!P || !d_target || !d_loss) return DRT3D_ERR_INVALID_ARG;
    if (P->dtype != DRT3D_F32) return DRT3D_ERR_DTYPE;
    if (reinterpret_cast<uintptr_t>(d_loss) & 7) return DRT3D_ERR_ALIGN;
    if (mask == 0 || (mask & ~DRT3D_ALL_DODECANTS)) return DRT3D_ERR_INVALID_ARG;
    const size_t fwd = align_up((size_t)kMaxSlots * 2 * P->fused.buf_bytes, 256);
    const long long per = residual_partials_per_slot(P);
    if (!d_ws || ws_bytes < fwd + (size_t)kMaxSlots * per * sizeof(double)) return DRT3D_ERR_WORKSPACE;
    if (!aligned16(d_ws)) return DRT3D_ERR_ALIGN;
    double* part = reinterpret_cast<double*>(static_cast<char*>(d_ws) + fwd);
    const drt3d_status st = planes_forward_impl(P, d_in, d_out, mask, d_ws, fwd, stream, false, d_target, part);
    if (st != DRT3D_OK) return st;
    prof_begin(P, stream, "planes_residual_loss", (double)popcount12(mask) * per * sizeof(double));
    if (launch_residual_loss(part, (long long)popcount12(mask) * per, d_loss, stream) != cudaSuccess)
        return DRT3D_ERR_CUDA;
    prof_end(P, stream);
    return DRT3D_OK;
}

drt3d_status drt3d_planes_forward_global(const drt3d_plan* P, const void* d_in, void* d_out, void* d_ws,
                                         size_t ws_bytes, cudaStream_t stream) {
    if (!P || !d_in || !d_out) return DRT3D_ERR_INVALID_ARG;
    if (!device_is_current(P->device)) return DRT3D_ERR_INVALID_ARG;
    if (P->N < 4) return DRT3D_ERR_SIZE;
    if (!aligned16(d_out)) return DRT3D_ERR_ALIGN;
    const int N = P->N;
    const size_t gp = (size_t)(3 * N - 2) * 4;  // bytes per global row
    // The four corner blocks hold no dodecant: zero them.
    for (int b0 : {0, 3})
        for (int b1 : {0, 3}) {
            char* blk = static_cast<char*>(d_out) + ((size_t)b0 * N * 4 * N + (size_t)b1 * N) * gp;
            if (cudaMemset2DAsync(blk, 4 * (size_t)N * gp, 0, (size_t)N * gp, N, stream) != cudaSuccess)
                return DRT3D_ERR_CUDA;
        }
    return planes_forward_impl(P, d_in, d_out, DRT3D_ALL_DODECANTS, d_ws, ws_bytes, stream, true);
}

drt3d_status drt3d_planes_adjoint(const drt3d_plan* P, const void* d_cot, void* d_vol, uint32_t mask,
                                  void* d_ws, size_t ws_bytes, cudaStream_t stream) {
    if (!P || !d_cot || !d_vol) return DRT3D_ERR_INVALID_ARG;
    if (!device_is_current(P->device)) return DRT3D_ERR_INVALID_ARG;
    if (P->dtype != DRT3D_I32 && P->dtype != DRT3D_F32) return DRT3D_ERR_DTYPE;
    if (mask == 0 || (mask & ~DRT3D_ALL_DODECANTS)) return DRT3D_ERR_INVALID_ARG;
    if (!aligned16(d_cot) || !aligned16(d_vol) || !aligned16(d_ws)) return DRT3D_ERR_ALIGN;
    const size_t buf = adjoint_buf_bytes(P);
    const int nslots = popcount12(mask);
    if (!d_ws || ws_bytes < (size_t)nslots * 2 * buf) return DRT3D_ERR_WORKSPACE;
    const int N = P->N;
    const bool is_float = P->dtype == DRT3D_F32;
    const size_t cot_block = (size_t)N * N * 3 * N * 4;
    const FusedSchedule& S = adjoint_schedule(P);
    char* ws = static_cast<char*>(d_ws);

    FusedLaunch L{};
    L.N = N;
    L.n = P->n;
    L.dmax = 3 * N;
    L.status = P->d_status;
    // The fused forward passes transposed, last first; q counts adjoint passes
    // done so the ping-pong of buffers is independent of the pass count.
    for (int p = S.npass - 1, q = 0; p >= 0; --p, ++q) {
        const FusedPass& ps = S.pass[p];
        L.m0 = ps.m0;
        L.gin = ps.out;                                // the forward pass's output rows
        L.gout = p == 0 ? Geo{2 * N, N} : ps.in;       // its input rows, or the frame volume
        // Lanes of 4 positions (vector loads and stores), or of 5 where that
        // cuts the positions computed by a quarter or more (a row that one
        // 5-wide tile covers but 4-wide tiles need two for, as the frame rows
        // of N = 128).
        const int R1 = (1 << ps.G) - 1;
        const int off_max = 2 * ((1 << ps.m0) - 1) * R1;
        int KK = 4, V = 0, PB = 0;
        adjoint_fused_tile(ps.G, 4, &V, &PB);
        int ntiles = (3 * N - PB - ((L.gout.base - PB - off_max) & ~3) + V - 1) / V;
        {
            int V5 = 0, PB5 = 0;
            if (adjoint_fused_tile(ps.G, 5, &V5, &PB5)) {
                const int nt5 = (3 * N - PB5 - ((L.gout.base - PB5 - off_max) & ~3) + V5 - 1) / V5;
                if (4 * (nt5 * 160) <= 3 * (ntiles * 128)) {
                    KK = 5;
                    V = V5;
                    PB = PB5;
                    ntiles = nt5;
                }
            }
        }
        L.V = V;
        L.ntiles = ntiles;
        const long long per_axis = 1LL << (P->n - ps.G);
        L.ctas = per_axis * per_axis * L.ntiles;
        // slots first to last on the first adjoint pass (a forward's last pass
        // ends on the first slot), then alternating (see planes_forward_impl)
        L.reverse_slots = q & 1;
        FramesSum FS{};
        for (int k = 0, i = 0; k < 12; ++k) {
            if (!((mask >> k) & 1)) continue;
            char* bufA = ws + (size_t)i * 2 * buf;
            char* bufB = bufA + buf;
            FusedSlot& fs = L.slot[i];
            fs.in = (q == 0) ? (const void*)(static_cast<const char*>(d_cot) + (size_t)i * cot_block)
                             : ((q & 1) ? (const void*)bufA : (const void*)bufB);
            fs.out = (q & 1) ? (void*)bufB : (void*)bufA;
            if (p == 0) {
                FS.frame[i] = fs.out;
                frames_sum_axes(dodecant_affine(N, k), N, i, &FS);
            }
            ++i;
        }
        char nm[40];
        std::snprintf(nm, sizeof nm, "planes_adj_fused G=%d m0=%d", ps.G, ps.m0);
        const double lo_in = 2.0 * N + 2 - 2.0 * (1 << ps.m0), lo_out = 2.0 * N + 2 - 2.0 * (1 << (ps.m0 + ps.G));
        const double rd = ps.final_ ? (double)N * N * 3 * N * 4 : (double)N * N * (3 * N - lo_out) * 4;
        const double wr = p == 0 ? (double)N * N * N * 4 : (double)N * N * (3 * N - lo_in) * 4;
        prof_begin(P, stream, nm, nslots * (rd + wr));
        if (launch_planes_adjoint_fused(L, ps.G, KK, is_float, nslots, stream) != cudaSuccess) return DRT3D_ERR_CUDA;
        prof_end(P, stream);
        if (p == 0) {
            // the frames summed through the dodecant maps, in increasing k so
            // that the float sum has a fixed order
            FS.vol = d_vol;
            FS.N = N;
            FS.nslots = nslots;
            const double vox = (double)N * N * N * 4;
            prof_begin(P, stream, "planes_adj_sum", (nslots + 1) * vox);
            if (launch_frames_sum(FS, is_float, stream) != cudaSuccess) return DRT3D_ERR_CUDA;
            prof_end(P, stream);
        }
    }
    return DRT3D_OK;
}

drt3d_status drt3d_planes_inverse(const drt3d_plan* P, const int32_t* d_R, int dodecant, int32_t* d_vol,
                                  void* d_ws, size_t ws_bytes, cudaStream_t stream) {
    if (!P || !d_R || !d_vol) return DRT3D_ERR_INVALID_ARG;
    if (!device_is_current(P->device)) return DRT3D_ERR_INVALID_ARG;
    if (dodecant < 0 || dodecant >= 12) return DRT3D_ERR_INVALID_ARG;
    if (P->dtype == DRT3D_F32) return DRT3D_ERR_DTYPE;
    if (!aligned16(d_R) || !aligned16(d_vol) || !aligned16(d_ws)) return DRT3D_ERR_ALIGN;
    const int N = P->N;
    const size_t buf = inverse_buf_bytes(N);
    InvStep st[24];
    const int c = inverse_steps(N, st);
    if (c > 1 && (!d_ws || ws_bytes < 2 * buf)) return DRT3D_ERR_WORKSPACE;
    char* ws = static_cast<char*>(d_ws);
    InvLaunch L{};
    L.status = P->d_status;
    L.map = dodecant_affine(N, dodecant);
    L.N = N;
    L.n = P->n;
    L.dmax = 3 * N;
    for (int i = 0; i < c; ++i) {
        const InvStep& t = st[i];
        L.axis = t.axis;
        L.m0 = t.m0;
        L.gin = inv_geo(N, t.mx_in, t.my_in);
        L.gout = inv_geo(N, t.mx_out, t.my_out);
        L.lo_out = 2 * N + 2 - (1 << t.mx_out) - (1 << t.my_out);
        L.scatter = (i == c - 1);
        L.in = (i == 0) ? (const void*)d_R : (const void*)(ws + (size_t)((i - 1) & 1) * buf);
        L.out = L.scatter ? (void*)d_vol : (void*)(ws + (size_t)(i & 1) * buf);
        char nm[40];
        std::snprintf(nm, sizeof nm, "planes_inverse %c G=%d m0=%d", t.axis ? 'y' : 'x', t.G, t.m0);
        const double W = 3.0 * N - L.gin.base;
        const double outb = L.scatter ? (double)N * N * N * 4 : (double)N * N * (3.0 * N - L.lo_out) * 4;
        prof_begin(P, stream, nm, (double)N * N * W * 4 + outb);
        if (launch_planes_inverse_pass(L, t.G, stream) != cudaSuccess) return DRT3D_ERR_CUDA;
        prof_end(P, stream);
    }
    return DRT3D_OK;
}

drt3d_status djt3d_lines_forward(const drt3d_plan* P, const void* d_in, int32_t* d_out, uint32_t mask,
                                 void* d_ws, size_t ws_bytes, cudaStream_t stream) {
    if (!P || !d_in || !d_out) return DRT3D_ERR_INVALID_ARG;
    if (!device_is_current(P->device)) return DRT3D_ERR_INVALID_ARG;
    if (mask == 0 || (mask & ~DRT3D_ALL_SECTORS)) return DRT3D_ERR_INVALID_ARG;
    if (P->dtype == DRT3D_F32) return DRT3D_ERR_DTYPE;
    if (P->N > 256) return DRT3D_ERR_SIZE;
    if (!aligned16(d_in) || !aligned16(d_out) || !aligned16(d_ws)) return DRT3D_ERR_ALIGN;
    const int N = P->N, n = P->n;
    int G[2];
    const int npass = djt_groups(N, G);
    const size_t buf = djt_buf_bytes(N);
    const int nslots = popcount12(mask);
    if (npass > 1 && (!d_ws || ws_bytes < (size_t)nslots * buf)) return DRT3D_ERR_WORKSPACE;
    const long long out_block = 4LL * N * N * N * N;  // elements per sector
    // With room in the workspace, y- and z-driven sectors read frame copies
    // of the volume (z' contiguous) instead of gathering across it.
    const size_t fcb = djt_frame_copy_bytes(N, P->dtype);
    const bool need_y = (mask & 0x0F0u) != 0, need_z = (mask & 0xF00u) != 0;
    const bool copies = npass > 1 && (need_y || need_z) && ws_bytes >= 2 * fcb + (size_t)nslots * buf;
    char* ws = static_cast<char*>(d_ws);
    char* slots = ws + (copies ? 2 * fcb : 0);
    if (copies) {
        const int esz = P->dtype == DRT3D_U8 ? 1 : P->dtype == DRT3D_I16 ? 2 : 4;
        const long long NN = (long long)N * N;
        prof_begin(P, stream, "djt_frame_copies", (double)(need_y + need_z) * 2 * NN * N * esz);
        // y-driven frame [y][z][x]: the volume as an N x N^2 matrix, transposed
        if (need_y && launch_transpose2d(d_in, ws, N, (int)NN, esz, stream) != cudaSuccess) return DRT3D_ERR_CUDA;
        // z-driven frame [z][x][y]: the volume as an N^2 x N matrix, transposed
        if (need_z && launch_transpose2d(d_in, ws + fcb, NN, N, esz, stream) != cudaSuccess) return DRT3D_ERR_CUDA;
        prof_end(P, stream);
    }
    DjtLaunch L{};
    L.N = N;
    L.n = n;
    int m0 = 0;
    for (int p = 0; p < npass; ++p) {
        const bool ingest = p == 0, final_ = p == npass - 1;
        const int m1 = m0 + G[p];
        int i = 0;
        for (int k = 0; k < 12; ++k) {
            if (!((mask >> k) & 1)) continue;
            DjtSlot& sl = L.slot[i];
            const int a = k >> 2;
            const void* src = d_in;
            if (copies && a > 0) {
                // the frame copy is g[x'][y'][z'] with strides N^2, N, 1; the
                // sector's flips reverse y' (bit 0) and z' (bit 1)
                src = ws + (a == 1 ? 0 : fcb);
                sl.map = sector_affine(N, k & 3);
            } else {
                sl.map = sector_affine(N, k);
            }
            char* b = slots + (size_t)i * buf;
            sl.in = ingest ? src : (const void*)b;
            sl.out = final_ ? (void*)(d_out + (size_t)i * out_block) : (void*)b;
            ++i;
        }
        L.m0 = m0;
        L.in_base = ingest ? N : djt_base(N, m0);
        L.in_pitch = 2 * N - L.in_base;
        L.in_plane = (long long)L.in_pitch * L.in_pitch;
        L.out_base = final_ ? 0 : djt_base(N, m1);
        L.out_pitch = 2 * N - L.out_base;
        L.out_plane = (long long)L.out_pitch * L.out_pitch;
        L.D1 = 2 * N - L.out_base;
        const int width = 2 * N - L.out_base;
        const int K = djt_lanes_k(G[p], width);
        L.V = (32 * K - ((1 << G[p]) - 1)) & ~3;
        L.ntiles = (32 * K >= width) ? 1 : 1 + (width - 32 * K + L.V - 1) / L.V;
        L.warps = (1LL << (2 * m0 + (n - m1))) * (1LL << G[p]) * L.D1 * L.ntiles;
        char nm[40];
        std::snprintf(nm, sizeof nm, "djt_pass G=%d m0=%d", G[p], m0);
        const double item = P->dtype == DRT3D_U8 ? 1 : P->dtype == DRT3D_I16 ? 2 : 4;
        const double in_b = ingest ? (double)N * N * N * item
                                   : (double)(1LL << (n + m0)) * (N + (1 << m0) - 1.0) * (N + (1 << m0) - 1.0) * 4;
        const double out_b = final_ ? (double)out_block * 4
                                    : (double)(1LL << (n + m1)) * (N + (1 << m1) - 1.0) * (N + (1 << m1) - 1.0) * 4;
        prof_begin(P, stream, nm, nslots * (in_b + out_b));
        if (launch_djt_pass(L, G[p], K, P->dtype, ingest, final_, nslots, stream) != cudaSuccess)
            return DRT3D_ERR_CUDA;
        prof_end(P, stream);
        m0 = m1;
    }
    return DRT3D_OK;
}

drt3d_status djt3d_lines_adjoint(const drt3d_plan* P, const int32_t* d_cot, int32_t* d_vol, uint32_t mask,
                                 void* d_ws, size_t ws_bytes, cudaStream_t stream) {
    if (!P || !d_cot || !d_vol) return DRT3D_ERR_INVALID_ARG;
    if (!device_is_current(P->device)) return DRT3D_ERR_INVALID_ARG;
    if (mask == 0 || (mask & ~DRT3D_ALL_SECTORS)) return DRT3D_ERR_INVALID_ARG;
    if (P->dtype != DRT3D_I32) return DRT3D_ERR_DTYPE;
    if (P->N > 256) return DRT3D_ERR_SIZE;
    if (!aligned16(d_cot) || !aligned16(d_vol) || !aligned16(d_ws)) return DRT3D_ERR_ALIGN;
    const int N = P->N, n = P->n;
    const int nslots = popcount12(mask);
    const size_t slot_bytes = djt_adj_slot_bytes(N);
    if (!d_ws || ws_bytes < (size_t)nslots * slot_bytes) return DRT3D_ERR_WORKSPACE;
    const long long cot_block = 4LL * N * N * N * N;  // elements per sector
    char* ws = static_cast<char*>(d_ws);
    // stage m lives in buffer (n - 1 - m) & 1 of its slot
    auto stage_buf = [&](int slot, int m) -> uint32_t* {
        char* b = ws + (size_t)slot * slot_bytes + (((n - 1 - m) & 1) ? djt_adj_stage_bytes(N, n - 1) : 0);
        return reinterpret_cast<uint32_t*>(b);
    };
    DjtAdjGather Gt{};
    int i = 0;
    for (int k = 0; k < 12; ++k) {
        if (!((mask >> k) & 1)) continue;
        Gt.sector[i] = k;
        ++i;
    }
    for (int m = n - 1; m >= 0; --m) {
        DjtAdjLaunch L{};
        for (int s = 0; s < nslots; ++s) {
            L.in[s] = (m == n - 1) ? reinterpret_cast<const uint32_t*>(d_cot + (size_t)s * cot_block)
                                   : stage_buf(s, m + 1);
            L.out[s] = stage_buf(s, m);
        }
        L.N = N;
        L.n = n;
        L.m = m;
        L.in_base = djt_adj_base(N, m + 1);
        L.in_pitch = 2 * N - L.in_base;
        L.in_plane = (long long)L.in_pitch * L.in_pitch;
        L.out_base = djt_adj_base(N, m);
        L.out_pitch = 2 * N - L.out_base;
        L.out_plane = (long long)L.out_pitch * L.out_pitch;
        L.D1 = 2 * N - L.out_base;
        const int lanes_w = 32 * djt_adj_lanes_k();
        L.ntiles = (L.out_pitch + lanes_w - 1) / lanes_w;
        L.items = (1LL << (2 * m)) * (1LL << (n - m - 1)) * L.D1 * L.ntiles;
        char nm[40];
        std::snprintf(nm, sizeof nm, "djt_adj_stage m=%d", m);
        const double in_b = (double)(1LL << (n + m + 1)) * L.in_plane * 4;
        const double out_b = (double)(1LL << (n + m)) * L.out_plane * 4;
        prof_begin(P, stream, nm, nslots * (in_b + out_b));
        if (launch_djt_adj_stage(L, nslots, stream) != cudaSuccess) return DRT3D_ERR_CUDA;
        prof_end(P, stream);
    }
    for (int s = 0; s < nslots; ++s) Gt.frame[s] = stage_buf(s, 0);
    Gt.nslots = nslots;
    Gt.N = N;
    Gt.base = djt_adj_base(N, 0);
    Gt.pitch = 2 * N - Gt.base;
    Gt.out = d_vol;
    prof_begin(P, stream, "djt_adj_gather", (double)nslots * N * N * N * 4 + (double)N * N * N * 4);
    if (launch_djt_adj_gather(Gt, stream) != cudaSuccess) return DRT3D_ERR_CUDA;
    prof_end(P, stream);
    return DRT3D_OK;
}

// One smoothing step at level l: x += c * h (*) A^T (r - A x).
static drt3d_status press_smooth(const drt3d_plan* P, int l, const float* r, float* x, float c, char* ws,
                                 const PressLayout& Lo, cudaStream_t stream) {
    const drt3d_plan* lp = level_plan(P, l);
    if (!lp) return DRT3D_ERR_NO_MEMORY;
    const int L = 1 << l;
    float* t = reinterpret_cast<float*>(ws + Lo.t);
    float* b = reinterpret_cast<float*>(ws + Lo.b);
    drt3d_status st = planes_forward_impl(lp, x, t, DRT3D_ALL_DODECANTS, ws + Lo.tws, Lo.tws_bytes, stream, false);
    if (st != DRT3D_OK) return st;
    if (launch_press_residual(r, t, 12LL * L * L * 3 * L, stream) != cudaSuccess) return DRT3D_ERR_CUDA;
    st = drt3d_planes_adjoint(lp, t, b, DRT3D_ALL_DODECANTS, ws + Lo.tws, Lo.tws_bytes, stream);
    if (st != DRT3D_OK) return st;
    if (launch_press_filter(b, x, L, c, true, stream) != cudaSuccess) return DRT3D_ERR_CUDA;
    return DRT3D_OK;
}

static bool press_args_ok(const drt3d_plan* P, void* d_ws, size_t ws_bytes, drt3d_status* err) {
    if (P->dtype != DRT3D_F32) { *err = DRT3D_ERR_DTYPE; return false; }
    if (!aligned16(d_ws)) { *err = DRT3D_ERR_ALIGN; return false; }
    if (!d_ws || ws_bytes < press_layout(P).total) { *err = DRT3D_ERR_WORKSPACE; return false; }
    for (int l = 1; l < P->n; ++l)
        if (!level_plan(P, l)) { *err = DRT3D_ERR_NO_MEMORY; return false; }
    return true;
}

drt3d_status drt3d_planes_press_inverse(const drt3d_plan* P, const float* d_R, float* d_vol, int iterations,
                                        int smooth, const float* steps, void* d_ws, size_t ws_bytes,
                                        cudaStream_t stream) {
    if (!P || !d_R || !d_vol || !steps || iterations < 0 || smooth < 1) return DRT3D_ERR_INVALID_ARG;
    if (!device_is_current(P->device)) return DRT3D_ERR_INVALID_ARG;
    if (!aligned16(d_R) || !aligned16(d_vol)) return DRT3D_ERR_ALIGN;
    drt3d_status st;
    if (!press_args_ok(P, d_ws, ws_bytes, &st)) return st;
    for (int l = 1; l <= P->n; ++l)
        if (!(steps[l] > 0.f)) return DRT3D_ERR_INVALID_ARG;
    const int N = P->N, n = P->n;
    const long long vox = (long long)N * N * N;
    const PressLayout Lo = press_layout(P);
    char* ws = static_cast<char*>(d_ws);
    auto fbuf = [&](size_t off) { return reinterpret_cast<float*>(ws + off); };
    if (cudaMemsetAsync(d_vol, 0, (size_t)vox * 4, stream) != cudaSuccess) return DRT3D_ERR_CUDA;
    for (int it = 0; it < iterations; ++it) {
        // residual of the current solution (the data itself for f_0 = 0)
        const float* rN = d_R;
        if (it > 0) {
            st = planes_forward_impl(P, d_vol, fbuf(Lo.r[n]), DRT3D_ALL_DODECANTS, ws + Lo.tws, Lo.tws_bytes,
                                     stream, false);
            if (st != DRT3D_OK) return st;
            if (launch_press_residual(d_R, fbuf(Lo.r[n]), 12LL * N * N * 3 * N, stream) != cudaSuccess)
                return DRT3D_ERR_CUDA;
            rN = fbuf(Lo.r[n]);
        }
        // restrict down to N = 1 and solve there exactly
        for (int l = n - 1; l >= 0; --l)
            if (launch_press_restrict(l == n - 1 ? rN : fbuf(Lo.r[l + 1]), fbuf(Lo.r[l]), 1 << l, stream) !=
                cudaSuccess)
                return DRT3D_ERR_CUDA;
        if (launch_press_coarsest(fbuf(Lo.r[0]), fbuf(Lo.x[0]), stream) != cudaSuccess) return DRT3D_ERR_CUDA;
        // prolongate and smooth level by level
        for (int l = 1; l <= n; ++l) {
            if (launch_press_prolong(fbuf(Lo.x[l - 1]), fbuf(Lo.x[l]), 1 << l, stream) != cudaSuccess)
                return DRT3D_ERR_CUDA;
            const float* rl = l == n ? rN : fbuf(Lo.r[l]);
            for (int j = 0; j < smooth; ++j) {
                st = press_smooth(P, l, rl, fbuf(Lo.x[l]), steps[l], ws, Lo, stream);
                if (st != DRT3D_OK) return st;
            }
        }
        if (launch_press_add(fbuf(Lo.x[n]), d_vol, vox, stream) != cudaSuccess) return DRT3D_ERR_CUDA;
    }
    return DRT3D_OK;
}

drt3d_status drt3d_press_spectral_radius(const drt3d_plan* P, int level, const float* d_start, int iterations,
                                         double* lambda, void* d_ws, size_t ws_bytes, cudaStream_t stream) {
    if (!P || !d_start || !lambda || iterations < 1 || level < 1 || level > P->n) return DRT3D_ERR_INVALID_ARG;
    if (!device_is_current(P->device)) return DRT3D_ERR_INVALID_ARG;
    if (!aligned16(d_start)) return DRT3D_ERR_ALIGN;
    drt3d_status st;
    if (!press_args_ok(P, d_ws, ws_bytes, &st)) return st;
    const drt3d_plan* lp = level_plan(P, level);
    const int L = 1 << level;
    const long long vox = (long long)L * L * L;
    const PressLayout Lo = press_layout(P);
    char* ws = static_cast<char*>(d_ws);
    float* x = reinterpret_cast<float*>(ws + Lo.x[level]);
    float* t = reinterpret_cast<float*>(ws + Lo.t);
    float* b = reinterpret_cast<float*>(ws + Lo.b);
    double* partial = reinterpret_cast<double*>(ws + Lo.partial);
    double* norm = reinterpret_cast<double*>(ws + Lo.norm);
    if (launch_press_normalize(d_start, x, vox, partial, norm, stream) != cudaSuccess) return DRT3D_ERR_CUDA;
    for (int it = 0; it < iterations; ++it) {
        st = planes_forward_impl(lp, x, t, DRT3D_ALL_DODECANTS, ws + Lo.tws, Lo.tws_bytes, stream, false);
        if (st != DRT3D_OK) return st;
        st = drt3d_planes_adjoint(lp, t, b, DRT3D_ALL_DODECANTS, ws + Lo.tws, Lo.tws_bytes, stream);
        if (st != DRT3D_OK) return st;
        if (launch_press_filter(b, x, L, 1.f, false, stream) != cudaSuccess) return DRT3D_ERR_CUDA;
        if (launch_press_normalize(x, x, vox, partial, norm, stream) != cudaSuccess) return DRT3D_ERR_CUDA;
    }
    if (cudaMemcpyAsync(lambda, norm, sizeof(double), cudaMemcpyDeviceToHost, stream) != cudaSuccess)
        return DRT3D_ERR_CUDA;
    if (cudaStreamSynchronize(stream) != cudaSuccess) return DRT3D_ERR_CUDA;
    return DRT3D_OK;
}

drt3d_status drt2d_workspace_bytes(const drt3d_plan* P, int B, uint32_t qmask, size_t* bytes) {
    if (!P || !bytes || B < 0 || qmask == 0 || (qmask & ~DRT2D_ALL_QUADRANTS)) return DRT3D_ERR_INVALID_ARG;
    int nbuf;
    const size_t slot = drt2d_slot_bytes(P->N, &nbuf);
    const int nq = quad_count(qmask);
    if (nbuf == 0 || B == 0 || drt2d_fused_supported(P->N, P->dtype)) {
        *bytes = 0;
        return DRT3D_OK;
    }
    const long long per_image = (long long)nbuf * nq * slot;
    long long c = std::max<long long>(1, (long long)(kDrt2dChunkTarget / (size_t)per_image));
    c = std::min<long long>(std::min<long long>(c, B), 65535 / nq);
    *bytes = (size_t)(c * per_image);
    return DRT3D_OK;
}

drt3d_status drt2d_forward(const drt3d_plan* P, const void* d_img, int B, void* d_out, uint32_t qmask, void* d_ws,
                           size_t ws_bytes, cudaStream_t stream) {
    if (!P || B < 0 || qmask == 0 || (qmask & ~DRT2D_ALL_QUADRANTS)) return DRT3D_ERR_INVALID_ARG;
    if (!device_is_current(P->device)) return DRT3D_ERR_INVALID_ARG;
    if (B == 0) return DRT3D_OK;
    if (!d_img || !d_out) return DRT3D_ERR_INVALID_ARG;
    if (!aligned16(d_img) || !aligned16(d_out) || !aligned16(d_ws)) return DRT3D_ERR_ALIGN;
    const int N = P->N, n = P->n;
    const int nq = quad_count(qmask);
    if (drt2d_fused_supported(N, P->dtype)) {
        // one CTA per (image, quadrant), intermediates in shared memory
        Drt2dLaunch F{};
        F.in = d_img;
        F.out = d_out;
        F.N = N;
        F.n = n;
        F.nq = nq;
        for (int q = 0, i = 0; q < 4; ++q)
            if ((qmask >> q) & 1) F.quad[i++] = q;
        const long long nslots = (long long)B * nq;
        if (nslots > 0x7fffffffLL) return DRT3D_ERR_INVALID_ARG;
        prof_begin(P, stream, "drt2d_fused", (double)B * N * N + (double)nslots * N * 2 * N * 4);
        if (launch_drt2d_fused(F, (int)nslots, stream) != cudaSuccess) return DRT3D_ERR_CUDA;
        prof_end(P, stream);
        return DRT3D_OK;
    }
    int nbuf;
    const size_t slot_bytes = drt2d_slot_bytes(N, &nbuf);
    const long long chunk = drt2d_chunk(N, nq, B, ws_bytes);
    if (nbuf > 0 && (!d_ws || chunk < 1)) return DRT3D_ERR_WORKSPACE;
    int G[4];
    const int ng = drt2d_groups(n, G);
    const int esz = P->dtype == DRT3D_U8 ? 1 : P->dtype == DRT3D_I16 ? 2 : 4;
    Drt2dLaunch L{};
    L.N = N;
    L.n = n;
    L.nq = nq;
    L.vec_ingest = N >= 4 && (N * esz) % 16 == 0;
    for (int q = 0, i = 0; q < 4; ++q)
        if ((qmask >> q) & 1) L.quad[i++] = q;
    const long long out_per_image = (long long)nq * N * 2 * N;  // elements
    char* bufs[2] = {static_cast<char*>(d_ws), static_cast<char*>(d_ws) + (size_t)chunk * nq * slot_bytes};
    for (long long b0 = 0; b0 < B; b0 += chunk) {
        const int nimg = (int)std::min<long long>(chunk, B - b0);
        const int nslots = nimg * nq;
        for (int g = 0, m = 0; g < ng; m += G[g], ++g) {
            const bool first = g == 0, last = g + 1 == ng;
            L.m0 = m;
            L.in = first ? static_cast<const void*>(static_cast<const char*>(d_img) + (size_t)b0 * N * N * esz)
                         : static_cast<const void*>(bufs[(g - 1) & 1]);
            L.in_base = drt2d_base(N, m);
            L.in_pitch = drt2d_pitch(N, m);
            L.in_slot = (long long)slot_bytes / 4;
            L.out = last ? static_cast<void*>(static_cast<char*>(d_out) + (size_t)b0 * out_per_image * 4)
                         : static_cast<void*>(bufs[g & 1]);
            L.out_base = last ? 0 : drt2d_base(N, m + G[g]);
            L.out_pitch = last ? 2 * N : drt2d_pitch(N, m + G[g]);
            L.out_slot = last ? (long long)N * 2 * N : (long long)slot_bytes / 4;
            L.V = drt2d_tile_valid(G[g]);
            L.ntiles = (2 * N - L.out_base + L.V - 1) / L.V;
            L.warps = (1LL << (n - G[g])) * L.ntiles;
            char nm[40];
            std::snprintf(nm, sizeof nm, "drt2d_pass G=%d m0=%d", G[g], m);
            const double in_b = first ? (double)N * N * esz : (double)N * (2 * N - L.in_base) * 4;
            const double out_b = (double)N * (2 * N - L.out_base) * 4;
            prof_begin(P, stream, nm, (first ? (double)nimg * in_b : (double)nslots * in_b) + nslots * out_b);
            if (launch_drt2d_pass(L, G[g], P->dtype, first, nslots, stream) != cudaSuccess) return DRT3D_ERR_CUDA;
            prof_end(P, stream);
        }
    }
    return DRT3D_OK;
}

drt3d_status drt3d_plan_set_schedule(drt3d_plan* P, int ngroups, const int* G) {
    if (!P || !G) return DRT3D_ERR_INVALID_ARG;
    FusedSchedule S{};
    if (!make_fused_schedule_groups(P->N, P->dtype, ngroups, G, &S)) return DRT3D_ERR_INVALID_ARG;
    P->fused = S;
    return DRT3D_OK;
}

drt3d_status drt3d_plan_get_schedule(const drt3d_plan* P, int* ngroups, int G[8]) {
    if (!P || !ngroups || !G) return DRT3D_ERR_INVALID_ARG;
    *ngroups = P->fused.npass;
    for (int g = 0; g < P->fused.npass; ++g) G[g] = P->fused.pass[g].G;
    return DRT3D_OK;
}

drt3d_status drt3d_plan_set_adjoint_schedule(drt3d_plan* P, int ngroups, const int* G) {
    if (!P) return DRT3D_ERR_INVALID_ARG;
    if (ngroups == 0) {
        P->has_adj = false;
        return DRT3D_OK;
    }
    if (!G) return DRT3D_ERR_INVALID_ARG;
    FusedSchedule S{};
    if (!make_fused_schedule_groups(P->N, P->dtype, ngroups, G, &S)) return DRT3D_ERR_INVALID_ARG;
    P->adj = S;
    P->has_adj = true;
    return DRT3D_OK;
}

drt3d_status drt3d_plan_get_adjoint_schedule(const drt3d_plan* P, int* ngroups, int G[8]) {
    if (!P || !ngroups || !G) return DRT3D_ERR_INVALID_ARG;
    const FusedSchedule& S = adjoint_schedule(P);
    *ngroups = S.npass;
    for (int g = 0; g < S.npass; ++g) G[g] = S.pass[g].G;
    return DRT3D_OK;
}

drt3d_status drt3d_set_profiling(drt3d_plan* P, int enable) {
    if (!P) return DRT3D_ERR_INVALID_ARG;
    Profiler& pr = P->prof;
    if (enable && !pr.events_made) {
        for (int i = 0; i < 2 * kMaxLaunch; ++i)
            if (cudaEventCreate(&pr.ev[i]) != cudaSuccess) return DRT3D_ERR_CUDA;
        pr.events_made = true;
    }
    pr.on = enable != 0;
    pr.count = 0;
    return DRT3D_OK;
}

drt3d_status drt3d_profiled_launches(const drt3d_plan* P, float* ms, double* algo_bytes, int capacity, int* count) {
    if (!P || !count) return DRT3D_ERR_INVALID_ARG;
    const Profiler& pr = P->prof;
    *count = pr.count;
    if (pr.count == 0) return DRT3D_OK;
    if (cudaEventSynchronize(pr.ev[2 * pr.count - 1]) != cudaSuccess) return DRT3D_ERR_CUDA;
    for (int i = 0; i < pr.count && i < capacity; ++i) {
        if (ms && cudaEventElapsedTime(&ms[i], pr.ev[2 * i], pr.ev[2 * i + 1]) != cudaSuccess)
            return DRT3D_ERR_CUDA;
        if (algo_bytes) algo_bytes[i] = pr.bytes[i];
    }
    return DRT3D_OK;
}

const char* drt3d_profiled_launch_name(const drt3d_plan* P, int i) {
    if (!P || i < 0 || i >= P->prof.count) return "";
    return P->prof.name[i];
}

drt3d_status drt3d_get_device_error(const drt3d_plan* P, cudaStream_t stream) {
    if (!P) return DRT3D_ERR_INVALID_ARG;
    if (!drt3d::device_is_current(P->device)) return DRT3D_ERR_INVALID_ARG;
    if (cudaStreamSynchronize(stream) != cudaSuccess) return DRT3D_ERR_CUDA;
    int h = 0;
    if (cudaMemcpy(&h, P->d_status, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) return DRT3D_ERR_CUDA;
    if (h != 0 && cudaMemset(P->d_status, 0, sizeof(int)) != cudaSuccess) return DRT3D_ERR_CUDA;
    return (drt3d_status)h;
}

}  // extern "C"
