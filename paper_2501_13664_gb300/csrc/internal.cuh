// internal.cuh -- shared declarations of libdrt3d's CUDA implementation.
//
// Buffer geometry used by every planes kernel
// -------------------------------------------
// The planes recursion of Algorithm 1 keeps an N x N x 3N buffer per stage.
// Here the two half-stage axes are scheduled separately (a stage of
// eq.(map3D) is exactly a half-stage along s1 followed by one along s2), and
// consecutive half-stages are grouped: a pass applies G >= 1 stages along one
// axis.  After mx stages along x and my along y, only displacements
// d >= lo = 2N + 2 - 2^mx - 2^my can be non-zero (the volume starts at 2N and
// every stage shifts reads upward by at most the slope-so-far plus one), so
// an intermediate stores rows (i1, i2) over d in [base, 3N) with
// base = lo rounded down to 8 and an 8-aligned pitch:
//     element (i1, i2, d) at ((i1 * N + i2) * pitch + d - base).
// Reads outside [base, 3N) are zero.  The final output uses base 0 and pitch
// 3N, the layout of the public ABI.
//
// A pass of G stages along one axis, starting after m0 stages on that axis,
// works on units (sg, w) with sg < 2^m0 (slope so far) and w < 2^(n-m0-G)
// (remaining position bits).  The unit's 2^G input rows are
//     a(u) = sg + (u << m0) + (w << (m0 + G)),   u < 2^G,
// and its 2^G output rows are o(t) = t + (sg << G) + (w << (m0 + G)).
// Unrolling eq.(digitalLine) over the G position bits gives
//     out[o(t)][d] = sum_u in[a(u)][d + sg * u + l^G_t(u)],
// i.e. a shear of row u by sg * u followed by a plain 2^G-point transform
// whose shifts are compile-time constants.
#pragma once

#include <cstddef>
#include <cstdint>

#include <cuda_runtime.h>

#include <cuda.h>

#include <algorithm>
#include <atomic>
#include <utility>

#include "drt3d.h"

namespace drt3d {

constexpr int kMaxN = 1024;

// One flag per device (ordinals 0..63; higher ones never read as set), e.g.
// "this kernel's dynamic shared-memory cap has been raised there".  Host
// threads launching through the same plan may test and set it concurrently.
struct DeviceOnce {
    std::atomic<unsigned long long> bits{0};
    bool done(int dev) const { return dev >= 0 && dev < 64 && ((bits.load(std::memory_order_acquire) >> dev) & 1ull); }
    void mark(int dev) {
        if (dev >= 0 && dev < 64) bits.fetch_or(1ull << dev, std::memory_order_release);
    }
};
// Whether `device` is the calling thread's current device: a plan's status
// word and the tables its launches read live there, so compute calls made
// with another device current are rejected as an argument error.
inline bool device_is_current(int device) {
    int cur = -1;
    return cudaGetDevice(&cur) == cudaSuccess && cur == device;
}

// Programmatic dependent launch.  A kernel of a pass chain is launched with
// programmatic stream serialisation: it may be scheduled while the previous
// kernel of the stream is still running its last CTAs, and it waits for that
// kernel's completion (and its memory) before it touches global memory.
// Each kernel of the chain lets its own dependents launch as soon as all of
// its CTAs have started.  Both instructions are no-ops for kernels launched
// the ordinary way.
__device__ __forceinline__ void pdl_wait_and_release() {
    asm volatile("griddepcontrol.wait;" ::: "memory");
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

template <typename... KArgs, typename... Args>
cudaError_t launch_chained(void (*kern)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                           Args&&... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kern, std::forward<Args>(args)...);
}

constexpr int kMaxSlots = 12;
constexpr int kMaxPasses = 12;

struct Geo {
    int base;   // first stored displacement
    int pitch;  // elements per row
};

// Affine map from a frame coordinate (x', y', z') to a flat index of the
// original volume: o0 + x' sx + y' sy + z' sz.
struct Affine {
    long long o0, sx, sy, sz;
};

// Dodecant k's frame (Algorithm 2's InOrder, see drt3d.h) and sector k's
// frame (Section 4.1), as affine maps for an N^3 volume.
Affine dodecant_affine(int N, int k);
Affine sector_affine(int N, int k);

inline int ilog2(int N) {
    int n = 0;
    while ((1 << n) < N) ++n;
    return n;
}

inline size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

// Element type of a buffer read or written by a fused pass.
enum class ElemKind : int { U8 = 0, I16 = 1, I32 = 2, F32 = 3, U16 = 4 };
inline int elem_bytes(ElemKind k) {
    return k == ElemKind::U8 ? 1 : (k == ElemKind::I16 || k == ElemKind::U16) ? 2 : 4;
}

// How the first fused pass reads the volume for one dodecant.
constexpr int kIngestGeneric = 0;  // scalar gathers
constexpr int kIngestZ = 1;        // the frame's z' axis is contiguous in memory
constexpr int kIngestRun = 2;      // the phase-1 axis is contiguous in memory

struct FusedSlot {
    const void* in;
    void* out;
    Affine map;
    int swap;     // 1: phase 1 runs along the second frame axis (y')
    int mode;     // kIngest* (first pass only)
    int reverse;  // the contiguous axis runs backwards in memory
    // Global layout (last pass only): output row (s1, s2) goes to row
    // g0 + s1 g1 + s2 g2 of the 4N x 4N x (3N - 2) array.
    long long g0;
    int g1, g2;
    // Final pass only: when set, each output cell is stored minus the cell at
    // the same offset of this array (the residual of a least-squares fit).
    const void* sub;
    // Final pass with `sub`, float32 only: when set, CTA c writes the sum of
    // the squares of the residual cells it stored to sq[c].
    double* sq;
};

struct FusedLaunch {
    FusedSlot slot[kMaxSlots];
    int N, n;
    int m0;          // stages already done on each axis
    Geo gin, gout;
    int dmax;        // 3N
    int V;           // valid displacements per CTA tile
    int ntiles;
    long long ctas;  // CTAs per slot
    int vec_store;   // output rows allow aligned vector stores
    int* status;     // device status word (time-outs of staged loads), may be null
    int global_layout;  // last pass writes Algorithm 2's 4N x 4N x (3N - 2) array
    int prefetch_ahead;  // CTAs (in launch order) whose input rows a CTA prefetches into L2, 0 = none
    // CTAs with blockIdx.y = j take slot nslots - 1 - j: the slots are
    // dispatched last to first (an order only; buffers stay indexed by slot).
    int reverse_slots;
};

// Slot of a CTA of a launch over `gridDim.y` slots (see reverse_slots).
__device__ __forceinline__ int launch_slot(int reverse, unsigned y, unsigned ny) {
    return reverse ? (int)(ny - 1 - y) : (int)y;
}

// One fused pass: G stages of eq.(map3D) (both axes).
struct FusedPass {
    int G, m0;
    Geo in, out;
    ElemKind in_kind, out_kind;
    bool ingest, final_;
};

struct FusedSchedule {
    int npass;
    FusedPass pass[8];
    size_t buf_bytes;  // bytes of one intermediate buffer (256-aligned)
};

FusedSchedule make_fused_schedule(int N, drt3d_dtype dtype);
// Schedule from an explicit split of the n stages into ng groups (each 1..4).
bool make_fused_schedule_groups(int N, drt3d_dtype dtype, int ng, const int* G, FusedSchedule* out);
// Ingest mode (vector load pattern, axis order) of one dodecant's first pass.
void fused_ingest_mode(int N, const Affine& A, FusedSlot& fs);

// Launchers (implemented per .cu file); return cudaGetLastError().
// One pass of the exact inverse: undo G half-stages along one axis.
struct InvLaunch {
    const void* in;   // rows of the later stage (geometry gin)
    void* out;        // rows of the earlier stage (geometry gout) or the volume
    int* status;      // device status word
    Affine map;       // dodecant map (scatter pass)
    int N, n;
    int axis, m0;     // axis undone; stages on that axis before the group
    Geo gin, gout;
    int dmax;         // 3N
    int lo_out;       // values below this displacement must vanish after the pass
    int scatter;      // last pass: write the volume through the dodecant map
};
size_t inverse_smem_bytes(int N, int G, int base, int m0);
cudaError_t launch_planes_inverse_pass(const InvLaunch& L, int G, cudaStream_t s);

// One pass of the lines transform (djt.cu).
struct DjtSlot {
    const void* in;
    void* out;
    Affine map;  // sector frame (first pass)
};
struct DjtLaunch {
    DjtSlot slot[kMaxSlots];
    int N, n, m0;
    int in_base, in_pitch;   // input plane window [in_base, 2N)^2
    long long in_plane;      // elements per input plane
    int out_base, out_pitch; // output plane window (final: 0, 2N)
    long long out_plane;
    int D1;                  // output rows d1 per plane (2N - out_base)
    int V, ntiles;           // d2 tiling: valid displacements of a non-last tile
    long long warps;         // warps per slot
};
int djt_lanes_k(int G, int width);
// out = in^T for an R x C row-major matrix of esz-byte elements (transpose.cu).
cudaError_t launch_transpose2d(const void* in, void* out, long long R, int C, int esz, cudaStream_t s);

// One stage of the lines adjoint, stage m + 1 -> m (djt_adjoint.cu).
struct DjtAdjLaunch {
    const uint32_t* in[kMaxSlots];  // stage m + 1 rows per slot
    uint32_t* out[kMaxSlots];       // stage m rows per slot
    int N, n, m;
    int in_base, in_pitch;          // stage m + 1 window [in_base, 2N)^2
    long long in_plane;
    int out_base, out_pitch;        // stage m window
    long long out_plane;
    int D1, ntiles;                 // e1 rows and e2 tiles of a stage-m plane
    long long items;                // warps per slot
};
// Sum of the selected sectors' frame volumes (stage-0 windows) in the
// original frame.
struct DjtAdjGather {
    const uint32_t* frame[kMaxSlots];
    int sector[kMaxSlots];
    int nslots, N;
    int base, pitch;                // stage-0 window
    int32_t* out;
};
cudaError_t launch_djt_adj_stage(const DjtAdjLaunch& L, int nslots, cudaStream_t s);
cudaError_t launch_djt_adj_gather(const DjtAdjGather& L, cudaStream_t s);
int djt_adj_lanes_k();
cudaError_t launch_djt_pass(const DjtLaunch& L, int G, int K, drt3d_dtype in_dtype, bool ingest, bool final_,
                            int nslots, cudaStream_t s);

// One pass of the 2D DRT of lines (drt2d.cu).  Slot i of the launch is
// (image i / nq, quadrant quad[i % nq]) of one chunk of images.
struct Drt2dLaunch {
    const void* in;          // images (first pass) or the previous pass's rows
    void* out;               // rows of this pass, or the final (s, d) arrays
    int N, n, m0;            // stages before the pass
    int in_base, in_pitch;   // input rows: d in [in_base, 2N)
    long long in_slot;       // elements per input slot
    int out_base, out_pitch;
    long long out_slot;
    int V, ntiles;           // valid displacements per warp tile, tiles per row
    long long warps;         // warps per slot
    int nq;
    int quad[4];
    int vec_ingest;          // first pass: image rows allow 16-byte vector loads
};
int drt2d_tile_valid(int G);
// The whole transform of each (image, quadrant) in one CTA (uint8 images,
// 32 <= N <= 256: first-group rows kept as 16 bits in shared memory).  Slot i
// of L reads image i / nq and writes its (N, 2N) block at out + i N 2N.
bool drt2d_fused_supported(int N, drt3d_dtype dtype);
cudaError_t launch_drt2d_fused(const Drt2dLaunch& L, int nslots, cudaStream_t s);
cudaError_t launch_drt2d_pass(const Drt2dLaunch& L, int G, drt3d_dtype in_dtype, bool ingest, int nslots,
                              cudaStream_t s);

// Kernels of the iterative inverse (press.cu).  Volumes are N^3 float32,
// transforms 12 dodecants of N x N x 3N float32.
constexpr int kPressNormParts = 256;  // partial sums of one norm
cudaError_t launch_press_filter(const float* b, float* y, int N, float c, bool accumulate, cudaStream_t s);
cudaError_t launch_press_prolong(const float* xc, float* x, int N, cudaStream_t s);
cudaError_t launch_press_restrict(const float* R, float* Rc, int Nc, cudaStream_t s);
cudaError_t launch_press_coarsest(const float* R1, float* x1, cudaStream_t s);
cudaError_t launch_press_residual(const float* r, float* t, long long n, cudaStream_t s);
cudaError_t launch_press_add(const float* x, float* y, long long n, cudaStream_t s);
// x = y / ||y||, ||y|| also stored (double) in *norm; partial holds
// kPressNormParts doubles.
cudaError_t launch_press_normalize(const float* y, float* x, long long n, double* partial, double* norm,
                                   cudaStream_t s);

int fused_valid(int G);  // valid displacements per CTA tile of a G-stage fused pass
cudaError_t launch_planes_fused(const FusedLaunch& L, int G, ElemKind in_kind, ElemKind out_kind,
                                bool ingest, int nslots, cudaStream_t s);
// Whether a fused pass stages its input through TMA boxes (16-bit buffer
// input at G >= 3, 32-bit at G = 3), and that launch: `in_base` is slot 0's
// input buffer, the other slots follow at `slot_stride` bytes.
bool fused_uses_tma(int G, ElemKind in_kind, bool ingest);
// loss[0] = 0.5 * sum of the n per-warp partial sums `part` (fixed order).
cudaError_t launch_residual_loss(const double* part, long long n, double* loss, cudaStream_t s);
cudaError_t launch_planes_fused_tma(const FusedLaunch& L, int G, ElemKind in_kind, ElemKind out_kind,
                                    const void* in_base, size_t slot_stride, int nslots, cudaStream_t s);
// The tensor map of those staged loads (x = displacement - base, y = row,
// z = slot; elements of elem_bytes = 2 or 4), for launches that keep it in
// global memory.
cudaError_t encode_fused_tmap(const FusedLaunch& L, const void* in_base, size_t slot_stride, int nslots,
                              int elem_bytes, CUtensorMap* map);
// The transpose of one fused pass (planes_adjoint_fused.cu): reads the
// forward pass's output rows (geometry gin) as cotangent and writes its input
// rows (geometry gout; the frame volume, base 2N and pitch N, for the first
// pass).  `V` stored positions per tile; tile origins are placed by the kernel.
bool adjoint_fused_tile(int G, int KK, int* V, int* PB);
cudaError_t launch_planes_adjoint_fused(const FusedLaunch& L, int G, int KK, bool is_float, int nslots,
                                        cudaStream_t s);

}  // namespace drt3d

namespace drt3d {
constexpr int kMaxLaunch = 2048;
struct Profiler {
    bool on = false;
    bool events_made = false;
    int count = 0;
    cudaEvent_t ev[2 * kMaxLaunch];
    double bytes[kMaxLaunch];
    char name[kMaxLaunch][40];
};
}  // namespace drt3d

struct drt3d_plan {
    mutable drt3d::Profiler prof;
    int N;
    int n;
    drt3d_dtype dtype;
    unsigned flags;
    int device;
    int* d_status;  // device status word (drt3d_status), 0 = OK
    drt3d::FusedSchedule fused;    // two-axis passes (forward)
    // Passes of the adjoint when set (its own split of the stages: any split
    // gives the same operator), else the forward's transposed.
    drt3d::FusedSchedule adj;
    bool has_adj = false;
    // Float32 plans of the coarser sizes N/2, N/4, ..., 2 used by the
    // iterative inverse, indexed by log2 of their size; host-only, created on
    // first use (by whichever host thread gets there first), sharing this
    // plan's status word.
    mutable std::atomic<drt3d_plan*> levels[11] = {};
    bool borrowed_status = false;
};
