/*
 * drt3d.h -- C ABI of libdrt3d, a GB300 (sm_103a) library for the 3D
 * multiscale discrete Radon transform (DRT) of planes and discrete John
 * transform (DJT) of lines of Marichal-Hernandez et al., "Three-dimensional
 * multiscale discrete Radon and John transforms" (arXiv 2501.13664).
 *
 * General conventions
 * -------------------
 *  - Every function returns a drt3d_status and never throws.  Argument errors
 *    are detected and returned synchronously, before anything is enqueued.
 *  - All compute is enqueued asynchronously on the caller's CUDA stream
 *    (0 = legacy default stream).  Errors raised inside a kernel (for example
 *    an inverse input that is not in the range of the forward map) are
 *    recorded in a device status word and read back by
 *    drt3d_get_device_error().
 *  - The caller owns every device buffer (inputs, outputs, workspaces).  The
 *    library allocates no device memory on any compute call; a plan owns only
 *    host metadata and one small device status word allocated at creation.
 *  - Device pointers must be 16-byte aligned.
 *  - A plan (and a batch plan) belongs to the device that was current when
 *    it was created.  Compute calls and status reads must be made with that
 *    device current; otherwise they return DRT3D_ERR_INVALID_ARG and enqueue
 *    nothing.
 *  - Compute calls may be made from several host threads at once, with one
 *    plan or several, on any streams (drt3d_planes_forward_noalloc excepted:
 *    its calls share one scratch array).  A plan's device status word is then
 *    shared: an error recorded by one call is reported by whichever
 *    drt3d_get_device_error() on that plan comes next.  Plan creation and
 *    destruction, the schedule setters and the profiling calls are not
 *    thread-safe for the same plan.
 *  - N = 2^n with 2 <= N <= 1024 (Algorithms 1 and 3 take log2 N stages;
 *    non-cubic sizes are left as future work in the paper's conclusions).
 *  - Integer arithmetic is two's-complement int32 and wraps modulo 2^32, so
 *    results are defined bit for bit for any input.
 *
 * Memory layouts (all C-contiguous)
 * ---------------------------------
 *  - Input volume f[x][y][z], N^3 elements of the plan's dtype.
 *  - Planes output, one block per selected dodecant, in increasing dodecant
 *    order: R[k][s1][s2][d], s1, s2 in [0, N), d in [0, 3N).  In dodecant k's
 *    frame the cell sums the digital plane z' = l_{s1}(x') + l_{s2}(y') +
 *    d - 2N (eq.(3DfDRT) with Algorithm 1's storage index, Section 3.1);
 *    d = 0 and d = 1 are always zero.  Dodecant k's frame is
 *    g_k(x', y', z') = f(...) given by Algorithm 2's InOrder table read as
 *    "flip original axis j where entry j < 0, then new axis i takes original
 *    axis |entry i|", with the rows of dodecants 5, 6, 9 and 10 taken as
 *    [-3,1,2], [3,-1,2], [2,-3,1] and [-2,3,1] (the printed rows repeat two
 *    sectors and miss two).
 *  - Lines output, one block per selected sector, in increasing sector
 *    order: J[k][s1][s2][d1][d2], d1, d2 in [0, 2N).  The cell sums the
 *    digital line y' = l_{s1}(x') + d1 - N, z' = l_{s2}(x') + d2 - N
 *    (eq.(3DfDJT), Algorithm 3's storage index, Section 4.1).  Sector
 *    k = 4a + b drives along axis a (x, y, z); the two other axes follow in
 *    cyclic order and bit 0 / bit 1 of b reverse the first / second of them.
 *
 * Digital line (eq.(digitalLine), Section 2.1):
 *   l^n_s(u) = sum_{i=0}^{n-1} u_{n-1-i} * floor((floor(s / 2^i) + 1) / 2).
 */
#ifndef DRT3D_H
#define DRT3D_H

#include <stddef.h>
#include <stdint.h>

#include <cuda_runtime_api.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum drt3d_status {
    DRT3D_OK = 0,
    DRT3D_ERR_INVALID_ARG = 1,  /* null plan/pointer, bad mask or dodecant index */
    DRT3D_ERR_SIZE = 2,         /* N not a power of two, N < 2 or N > 1024 */
    DRT3D_ERR_DTYPE = 3,        /* dtype not supported by this operation */
    DRT3D_ERR_ALIGN = 4,        /* a device pointer is not 16-byte aligned */
    DRT3D_ERR_WORKSPACE = 5,    /* workspace null or smaller than required */
    DRT3D_ERR_NOT_IN_RANGE = 6, /* inverse input is not a forward transform */
    DRT3D_ERR_TIMEOUT = 7,      /* a bounded device-side wait gave up */
    DRT3D_ERR_BOUNDS = 8,       /* a device-side bounds check failed */
    DRT3D_ERR_CUDA = 9,         /* a CUDA runtime call failed */
    DRT3D_ERR_NO_MEMORY = 10,   /* host allocation or plan status word failed */
    DRT3D_ERR_SCRATCH_LIMIT = 11 /* call needs more than the fixed no-alloc scratch */
} drt3d_status;

typedef enum drt3d_dtype {
    DRT3D_U8 = 0,
    DRT3D_I16 = 1,
    DRT3D_I32 = 2,
    DRT3D_F32 = 3
} drt3d_dtype;

/* Operation codes for drt3d_workspace_bytes(). */
typedef enum drt3d_op {
    DRT3D_OP_PLANES_FORWARD = 0,
    DRT3D_OP_PLANES_ADJOINT = 1,
    DRT3D_OP_PLANES_INVERSE = 2,
    DRT3D_OP_LINES_FORWARD = 3,
    DRT3D_OP_LINES_ADJOINT = 4,
    DRT3D_OP_PLANES_PRESS = 5,
    DRT3D_OP_PLANES_RESIDUAL_LOSS = 6
} drt3d_op;

#define DRT3D_ALL_DODECANTS 0xFFFu
#define DRT3D_ALL_SECTORS 0xFFFu
#define DRT2D_ALL_QUADRANTS 0xFu

typedef struct drt3d_plan drt3d_plan;

/* Create a plan for N^3 volumes of dtype `in_dtype`.  Planes forward accepts
 * U8/I16/I32 (int32 output) and F32 (float output); the adjoint takes I32 or
 * F32 plans; the inverse and the lines forward are integer only.  `flags` is
 * reserved and must be 0.  On success *plan owns a 4-byte device status word
 * on the current device.  Errors: INVALID_ARG (plan null, flags != 0), SIZE,
 * DTYPE, NO_MEMORY, CUDA. */
drt3d_status drt3d_plan_create(drt3d_plan** plan, int N, drt3d_dtype in_dtype, unsigned flags);

/* Release a plan (NULL is accepted).  Waits for nothing: the caller must not
 * destroy a plan while work that uses it is still in flight. */
drt3d_status drt3d_plan_destroy(drt3d_plan* plan);

/* Shape of the full 12-dodecant planes output: {12, N, N, 3N}. */
drt3d_status drt3d_planes_out_shape(const drt3d_plan* plan, int64_t dims[4]);

/* Shape of the full 12-sector lines output: {12, N, N, 2N, 2N}. */
drt3d_status drt3d_lines_out_shape(const drt3d_plan* plan, int64_t dims[5]);

/* Bytes of device workspace an operation needs for all 12 dodecants or
 * sectors (a smaller mask never needs more).  `op` is a drt3d_op. */
drt3d_status drt3d_workspace_bytes(const drt3d_plan* plan, int op, size_t* bytes);

/* Forward 3D DRT of planes (Algorithm 1 per dodecant, Algorithm 2's twelve
 * dodecants; stage map eq.(map3D), Section 3.1).
 *   d_in   : N^3 volume of the plan's dtype, f[x][y][z].
 *   d_out  : popcount(dodecant_mask) blocks of N*N*3N int32 (integer plans)
 *            or float (F32 plans), R[k][s1][s2][d], overwritten.
 *   dodecant_mask : bit k selects dodecant k (1..0xFFF).
 *   d_ws, ws_bytes: workspace, >= drt3d_workspace_bytes(PLANES_FORWARD).
 * Integer results are exact (wrapping int32); F32 results are rounded sums.
 * Passes over 16-bit intermediates stage their rows in shared memory with
 * TMA loads whose completion is awaited for at most 0.2 s; a load still
 * outstanding then leaves the output undefined and records DRT3D_ERR_TIMEOUT
 * in the device status word (drt3d_get_device_error).
 * Errors: INVALID_ARG, ALIGN, WORKSPACE, CUDA. */
drt3d_status drt3d_planes_forward(const drt3d_plan* plan, const void* d_in, void* d_out,
                                  uint32_t dodecant_mask, void* d_ws, size_t ws_bytes,
                                  cudaStream_t stream);

/* The 3D DRT of a cube in Algorithm 2's global layout: all 12 dodecants merged
 * into one 4N x 4N x (3N-2) array.  Dodecant k's output R_k[s1][s2][d] goes to
 * block DodecantCoords[k] (N x N cells), its two slope dimensions permuted by
 * |OutOrder[k]| and reversed where OutOrder[k] is negative (OutOrder and
 * DodecantCoords as printed in Algorithm 2), displacement d at index d - 2
 * (d = 0, 1 are always zero and are dropped; d is not reversed).  The four
 * corner blocks, which no dodecant uses, are zeroed.  The remap is done by the
 * last pass's stores; nothing is copied.
 *   d_out : 16 N^2 (3N - 2) int32 (or float for F32 plans), overwritten.
 *   d_ws, ws_bytes: as drt3d_planes_forward with all 12 dodecants.
 * N >= 4.  Errors: INVALID_ARG, SIZE, ALIGN, WORKSPACE, CUDA. */
drt3d_status drt3d_planes_forward_global(const drt3d_plan* plan, const void* d_in, void* d_out, void* d_ws,
                                         size_t ws_bytes, cudaStream_t stream);

/* Residual of the planes forward against a target: d_out = A d_in - d_target
 * cell by cell, with A the transform of drt3d_planes_forward (same inputs,
 * masks, workspace and layouts).  The subtraction happens as the last pass
 * stores each cell, so the transform itself is never written out: this is
 * the residual of the least-squares fit of a volume to a target transform
 * (the gradient of 0.5 ||A x - b||^2 is the adjoint of the residual).
 *   d_target : popcount(dodecant_mask) blocks of N*N*3N elements of the output
 *              type, R[k][s1][s2][d] layout, 16-byte aligned; it may be d_out
 *              itself (each cell is read before it is overwritten by the same
 *              thread).
 * Float32 results equal the forward's cell minus the target cell rounded once
 * (bit for bit the forward followed by a subtraction); integer results wrap.
 * The paper has no counterpart: its method stops at the transform and its
 * backprojection.
 * Errors: as drt3d_planes_forward; INVALID_ARG when d_target is NULL. */
drt3d_status drt3d_planes_forward_residual(const drt3d_plan* plan, const void* d_in, const void* d_target,
                                           void* d_out, uint32_t dodecant_mask, void* d_ws, size_t ws_bytes,
                                           cudaStream_t stream);

/* drt3d_planes_forward_residual, and the least-squares loss of that residual:
 *   d_loss[0] = 0.5 * sum over the stored cells of (A x - b)^2   (double).
 * Each cell's square is added as the last pass stores it (per thread in
 * float, per CTA in double into the workspace), then one small launch adds
 * the partial sums in a fixed order, so the loss is the same on every run
 * and no extra pass reads the residual.  Float32 plans only; d_loss is
 * device memory (8-byte aligned).  The workspace must hold
 * drt3d_workspace_bytes(plan, DRT3D_OP_PLANES_RESIDUAL_LOSS) bytes (the
 * forward's, then the partial sums).  No paper counterpart: the loss of
 * Section 5.2's fit written into the transform's epilogue.
 * Errors: as drt3d_planes_forward_residual; DTYPE for non-float plans,
 * INVALID_ARG when d_loss is NULL. */
drt3d_status drt3d_planes_forward_residual_loss(const drt3d_plan* plan, const void* d_in, const void* d_target,
                                                void* d_out, uint32_t dodecant_mask, double* d_loss, void* d_ws,
                                                size_t ws_bytes, cudaStream_t stream);

/* Adjoint (backprojection) of drt3d_planes_forward (Section 5.1, stage loop
 * reversed with eq.(invmap3Dsummation); reads below d = 0 are zero):
 *   d_vol = sum over selected k, in increasing k, of g_k^T(A_k^T d_cot[k]).
 *   d_cot : popcount(mask) blocks of N*N*3N (int32 or float per the plan).
 *   d_vol : N^3 int32 or float, overwritten.
 * Plan dtype must be I32 or F32.  The dodecant sum has a fixed order, so F32
 * results are deterministic.  Errors: INVALID_ARG, DTYPE, ALIGN, WORKSPACE,
 * CUDA. */
drt3d_status drt3d_planes_adjoint(const drt3d_plan* plan, const void* d_cot, void* d_vol,
                                  uint32_t dodecant_mask, void* d_ws, size_t ws_bytes,
                                  cudaStream_t stream);

/* Exact inverse of one dodecant's planes transform (not printed in the
 * paper: derived from eq.(map2D)/eq.(map3D) and Algorithm 1's zero embedding;
 * the paper's own inverse is the iterative scheme of Section 5.2).  Each
 * half-stage is undone by a suffix sum of out1 - out0 along d.
 *   d_R   : N*N*3N int32, dodecant `dodecant`'s block of the forward output.
 *   d_vol : N^3 int32 volume f[x][y][z] (original frame), overwritten.
 * If d_R is not in the range of the forward map the volume is undefined and
 * DRT3D_ERR_NOT_IN_RANGE is recorded in the device status word (read it with
 * drt3d_get_device_error).  Integer plans only.  Errors: INVALID_ARG, DTYPE,
 * ALIGN, WORKSPACE, CUDA. */
drt3d_status drt3d_planes_inverse(const drt3d_plan* plan, const int32_t* d_R, int dodecant,
                                  int32_t* d_vol, void* d_ws, size_t ws_bytes, cudaStream_t stream);

/* Forward 3D DJT of lines (Algorithm 3 per sector; stage map eq.(map3DJ),
 * Section 4.1).
 *   d_in  : N^3 volume of the plan's dtype (U8, I16 or I32).
 *   d_out : popcount(sector_mask) blocks of N*N*2N*2N int32, overwritten.
 *   d_ws, ws_bytes: N >= 32 needs one intermediate buffer per selected
 *           sector; drt3d_workspace_bytes(LINES_FORWARD) adds room for two
 *           transposed copies of the volume that the y- and z-driven sectors
 *           then read instead of gathering across it (same result, faster).
 * N <= 256.  Errors: INVALID_ARG, DTYPE, SIZE, ALIGN, WORKSPACE, CUDA. */
drt3d_status djt3d_lines_forward(const drt3d_plan* plan, const void* d_in, int32_t* d_out,
                                 uint32_t sector_mask, void* d_ws, size_t ws_bytes,
                                 cudaStream_t stream);

/* Adjoint (backprojection) of djt3d_lines_forward (eq.(invmap3DJsummation):
 * Algorithm 3's stage loop reversed; reads below displacement 0 are zero):
 *   d_vol = sum over selected k, in increasing k, of (sector k's frame map)^T
 *           (J_k^T d_cot[k]).
 *   d_cot : popcount(sector_mask) blocks of N*N*2N*2N int32, J[k][s1][s2][d1][d2].
 *   d_vol : N^3 int32 volume f[x][y][z] (original frame), overwritten.
 *   d_ws, ws_bytes: workspace, >= drt3d_workspace_bytes(LINES_ADJOINT)
 *            (two stage buffers per sector: 1.6 GB per sector at N = 128).
 * Plan dtype must be I32; N <= 256.  Exact in wrapping int32 and deterministic
 * (every output is a gather; no atomics).  Errors: INVALID_ARG, DTYPE, SIZE,
 * ALIGN, WORKSPACE, CUDA. */
drt3d_status djt3d_lines_adjoint(const drt3d_plan* plan, const int32_t* d_cot, int32_t* d_vol,
                                 uint32_t sector_mask, void* d_ws, size_t ws_bytes, cudaStream_t stream);

/* Iterative inverse of the planes transform (Section 5.2: the adjoint
 * followed by the high-pass filter h as an approximate inverse, improved
 * iteratively with a multigrid of prolongations P and restrictions S).
 * With A the twelve-dodecant forward and B_L r = steps[l] * h (*) A_L^T r at
 * size L = 2^l (h with mirrored borders: an outside neighbour takes the
 * nearest voxel inside):
 *   f_0 = 0;  f_{k+1} = f_k + M_N(d_R - A f_k)  for k < iterations, where
 *   M_N(r): r_N = r, r_{L/2} = S r_L down to L = 1; x_1 = mean over the
 *   twelve dodecants of r_1(0, 0, 2) (exact at N = 1); then for L = 2 .. N:
 *   x_L = P x_{L/2} and `smooth` times x_L += B_L (r_L - A_L x_L).
 *   S: r_{L/2}(s1, s2, d) = (r_L(2s1, 2s2, 2d) + r_L(2s1, 2s2, 2d + 1)) / 8;
 *   P: x_L(i, j, k) = x_{L/2}(i/2, j/2, k/2).
 *   d_R   : 12 blocks of N*N*3N float32 (all dodecants, drt3d_planes_forward's
 *           layout).
 *   d_vol : N^3 float32, overwritten with f_iterations (zero for 0 iterations).
 *   steps : host array of n + 1 floats, steps[l] > 0 for l = 1..n (entry 0
 *           unused); steps[l] = factor / drt3d_press_spectral_radius(l) with
 *           factor < 2 makes each smoothing step contract.
 *   d_ws, ws_bytes: >= drt3d_workspace_bytes(PLANES_PRESS): about 320 N^3
 *           bytes (residuals of every level, one transform-sized buffer,
 *           per-level solutions) plus the larger of the forward's and the
 *           adjoint's workspace; N = 1024 does not fit a 288 GB device.
 * Plan dtype must be F32.  The coarser levels' plans are created (host
 * memory only) on first use and released with the plan.  Errors:
 * INVALID_ARG, DTYPE, ALIGN, WORKSPACE, NO_MEMORY, CUDA. */
drt3d_status drt3d_planes_press_inverse(const drt3d_plan* plan, const float* d_R, float* d_vol, int iterations,
                                        int smooth, const float* steps, void* d_ws, size_t ws_bytes,
                                        cudaStream_t stream);

/* Spectral radius of h (*) A_L^T A_L at size L = 2^level (1 <= level <= n)
 * by `iterations` steps of the power iteration from d_start (L^3 float32,
 * non-zero): x = start / ||start||, then y = h (*) A^T A x, x = y / ||y||;
 * *lambda = ||y|| of the last step.  Synchronises `stream` to return the
 * value.  Same plan and workspace as drt3d_planes_press_inverse.  Errors:
 * INVALID_ARG, DTYPE, ALIGN, WORKSPACE, NO_MEMORY, CUDA. */
drt3d_status drt3d_press_spectral_radius(const drt3d_plan* plan, int level, const float* d_start, int iterations,
                                         double* lambda, void* d_ws, size_t ws_bytes, cudaStream_t stream);

/* 2D DRT of lines (Section 2.1: the stage recursion eq.(map2D); the four
 * quadrants of Section 2.2), for a batch of images, using the plan's N and
 * input dtype.
 *   d_img : B images f[b][x][y], N x N each, of the plan's dtype.
 *   d_out : B blocks of popcount(quadrant_mask) arrays R[q][s][d] of N x 2N
 *           int32 (float32 for an F32 plan), quadrants in increasing order,
 *           overwritten.  The cell sums the digital line
 *           y' = l_s(u) + d - N over u of quadrant q's view f_q(u, y') of the
 *           image: f(u, y'), f(u, N-1-y'), f(y', u), f(N-1-y', u) for
 *           q = 0..3 (bit 1 swaps the axes, bit 0 reverses the other one).
 *           d = 0 is always zero.
 *   quadrant_mask : bits 0..3, non-zero.
 *   d_ws, ws_bytes: workspace for the intermediate stages of one chunk of
 *           images; drt2d_workspace_bytes() gives a size that keeps a chunk's
 *           intermediates near 32 MiB.  Any size that holds one image works
 *           (images are processed in chunks of what fits).  None is needed
 *           for N <= 16, nor for uint8 images with N <= 256 (each image and
 *           quadrant is transformed by one CTA with its intermediate rows in
 *           shared memory as 16-bit values, exact since N * 255 < 2^16).
 *   B = 0 is a no-op.  Integer input is exact in wrapping int32; float input
 *   is summed in float32 in a fixed order.  Errors: INVALID_ARG, ALIGN,
 *   WORKSPACE, CUDA. */
drt3d_status drt2d_forward(const drt3d_plan* plan, const void* d_img, int B, void* d_out, uint32_t quadrant_mask,
                           void* d_ws, size_t ws_bytes, cudaStream_t stream);
drt3d_status drt2d_workspace_bytes(const drt3d_plan* plan, int B, uint32_t quadrant_mask, size_t* bytes);

/* Stage-fusion schedule of the planes forward: the n = log2 N stages of
 * eq.(map3D) run in `ngroups` passes of G[0], G[1], ... stages on both axes
 * (each 1..4, summing to n).  The default is ceil(n/4) near-equal groups;
 * an autotuner may set another split.  Changing it changes the workspace
 * sizes (query drt3d_workspace_bytes again); integer results never change,
 * float32 results only through the order of the additions.
 * Errors: INVALID_ARG (bad split). */
drt3d_status drt3d_plan_set_schedule(drt3d_plan* plan, int ngroups, const int* G);
drt3d_status drt3d_plan_get_schedule(const drt3d_plan* plan, int* ngroups, int G[8]);
/* Stage-fusion schedule of the planes adjoint (eq.(invmap3Dsummation)): the
 * adjoint runs the transposes of the passes of this split, last first.  Every
 * split of the stages gives the same operator, so the adjoint's split may
 * differ from the forward's (an autotuner picks each for speed; integer
 * results are identical, float32 results differ only in the order of the
 * additions).  ngroups = 0 (G may be null) makes the adjoint follow the
 * forward's schedule again (the default).  The get call reports the split
 * in effect.  Changes the adjoint's workspace size.  Not thread-safe for the
 * same plan.  Errors: INVALID_ARG (bad split). */
drt3d_status drt3d_plan_set_adjoint_schedule(drt3d_plan* plan, int ngroups, const int* G);
drt3d_status drt3d_plan_get_adjoint_schedule(const drt3d_plan* plan, int* ngroups, int G[8]);

/* ---------------------------------------------------------------------
 * Batched planes forward: many uint8 volumes of sizes N in {16,...,256} in
 * one persistent kernel launch (not in the paper, which transforms one cube).
 * Work items are the CTAs of every pass of every volume and dodecant; a
 * second-pass item waits for its (volume, dodecant)'s first pass through a
 * device counter, with a bounded wait (default 2 s) after which the launch
 * records DRT3D_ERR_TIMEOUT and skips the remaining dependent work.
 *   1. drt3d_batch_plan_create(&bp, count, Ns, DRT3D_U8, 0)
 *   2. optionally drt3d_batch_set_schedule(bp, N, ngroups, G) and
 *      drt3d_batch_set_item_tiles(bp, N, npass, tiles) per size
 *   3. drt3d_batch_workspace_bytes(bp, &bytes); allocate it
 *   4. drt3d_batch_bind(bp, descs, d_ws, bytes): uploads the work tables
 *      (allocates small device tables; not for capture)
 *   5. drt3d_planes_forward_batched(bp, stream): one cudaMemsetAsync and one
 *      kernel launch, no host synchronisation -- capturable in a CUDA graph
 *   6. drt3d_batch_get_device_error(bp, stream)
 * Outputs: descs[i].d_out holds all 12 dodecants of volume i in the layout
 * of drt3d_planes_forward, bit-identical to it.
 * --------------------------------------------------------------------- */
typedef struct drt3d_vol_desc {
    const void* d_in;  /* N^3 uint8 volume */
    int32_t* d_out;    /* 12 * N * N * 3N int32 */
} drt3d_vol_desc;

typedef struct drt3d_batch_plan drt3d_batch_plan;

drt3d_status drt3d_batch_plan_create(drt3d_batch_plan** plan, int count, const int* Ns, drt3d_dtype dtype,
                                     unsigned flags);
drt3d_status drt3d_batch_plan_destroy(drt3d_batch_plan* plan);
drt3d_status drt3d_batch_set_schedule(drt3d_batch_plan* plan, int N, int ngroups, const int* G);
/* Work-item size of the persistent launch (mode 0) for the batch's volumes of
 * size N: tiles[p] consecutive unit-tiles of pass p per claimed item (a unit
 * is one 2^G x 2^G row block of a fused pass, processed over its displacement
 * tiles one after another; units follow each other in row-major order); 0
 * keeps the default (8 tiles at G = 4, whole units grouped to at least 256
 * rows below).  npass = the number of passes of N's batched schedule; a later
 * drt3d_batch_set_schedule for N clears the setting.  Not a paper quantity: a
 * scheduling parameter for the autotuner.  Takes effect at the next bind.
 * Errors: INVALID_ARG (null, npass mismatch, negative entry), SIZE (no volume
 * of size N in the batch). */
drt3d_status drt3d_batch_set_item_tiles(drt3d_batch_plan* plan, int N, int npass, const int* tiles);
drt3d_status drt3d_batch_workspace_bytes(const drt3d_batch_plan* plan, size_t* bytes);
drt3d_status drt3d_batch_bind(drt3d_batch_plan* plan, const drt3d_vol_desc* descs, void* d_ws, size_t ws_bytes);
/* How drt3d_planes_forward_batched runs the bound batch.
 *   mode 0 (default): one memset and one persistent kernel for every pass of
 *           every volume (work items claimed from a counter, dependencies
 *           through completion counters with bounded waits).
 *   mode 1: each volume's passes as ordinary kernel launches, the volumes
 *           spread over `nstreams` (1..8) internal streams, largest first onto
 *           the least loaded; the streams are forked from and joined back into
 *           the caller's stream, so the call stays capturable in a CUDA graph.
 * Results are identical in both modes.  Errors: INVALID_ARG, CUDA. */
drt3d_status drt3d_batch_set_mode(drt3d_batch_plan* plan, int mode, int nstreams);
drt3d_status drt3d_planes_forward_batched(const drt3d_batch_plan* plan, cudaStream_t stream);
drt3d_status drt3d_batch_get_device_error(const drt3d_batch_plan* plan, cudaStream_t stream);
/* Test and tuning hook: bounded-wait limit in nanoseconds; (withhold_vol,
 * withhold_dodecant) >= 0 makes that first-pass signal never arrive, so the
 * dependent waits time out (exercises the error path without a GPU fault). */
drt3d_status drt3d_batch_set_wait_limit(drt3d_batch_plan* plan, unsigned long long ns, int withhold_vol,
                                        int withhold_dodecant);

/* Synchronise `stream`, read and clear the plan's device status word.
 * Returns DRT3D_OK if no kernel recorded an error since the last call. */
drt3d_status drt3d_get_device_error(const drt3d_plan* plan, cudaStream_t stream);

/* Human-readable name of a status code (static storage). */
const char* drt3d_status_string(drt3d_status status);

/* Diagnostics.  While profiling is enabled, every compute call made with the
 * plan records a CUDA event pair around each of its kernel launches on the
 * caller's stream (up to 2048 launches after enabling), with a short name and
 * the launch's algorithmic bytes (compact rows read plus rows written: the
 * HBM floor of that launch).  drt3d_set_profiling(plan, 1) clears the record;
 * enabling creates events (no device memory).  Profiling state lives in the
 * plan and is not thread-safe.
 * drt3d_profiled_launches(): synchronises on the last recorded event, fills
 * up to `capacity` entries of ms[] and algo_bytes[] (either may be NULL) and
 * sets *count to the number of recorded launches. */
drt3d_status drt3d_set_profiling(drt3d_plan* plan, int enable);
drt3d_status drt3d_profiled_launches(const drt3d_plan* plan, float* ms, double* algo_bytes, int capacity,
                                     int* count);
/* Name of recorded launch i ("" if out of range). */
const char* drt3d_profiled_launch_name(const drt3d_plan* plan, int i);

/* Forward planes transform that allocates nothing and takes no workspace.
 * The paper has no counterpart: this is a service for callers that cannot
 * allocate device memory where they run the transform (host callbacks or
 * real-time loops that must stay out of the allocator, plug-in hosts that
 * hand out only input and output buffers, processes whose device memory is
 * reserved up front by another framework).  Same arguments, layouts and
 * results as drt3d_planes_forward, minus the workspace.
 *   Scratch: a fixed library-owned device array of
 *            drt3d_noalloc_scratch_bytes() = 16 MiB, held by every GPU on
 *            which the library is loaded until the process exits.  A call
 *            needing more (two intermediate buffers per selected dodecant,
 *            e.g. all 12 dodecants at N = 64 with 32-bit input or at N >= 128)
 *            returns DRT3D_ERR_SCRATCH_LIMIT without enqueuing anything;
 *            N <= 16 needs none.
 *   Set-up:  the first call on a device looks up the array's device address
 *            (cudaGetSymbolAddress) and caches it; make that first call
 *            before any stream capture.
 *   Sharing: all calls use the same array and nothing in it must start at
 *            zero (every element is written before it is read), but calls
 *            that overlap on the GPU race on it: serialise them.
 * Errors: INVALID_ARG, ALIGN, SCRATCH_LIMIT, CUDA. */
drt3d_status drt3d_planes_forward_noalloc(const drt3d_plan* plan, const void* d_in, void* d_out,
                                          uint32_t dodecant_mask, cudaStream_t stream);

/* Size in bytes of the fixed scratch used by drt3d_planes_forward_noalloc. */
size_t drt3d_noalloc_scratch_bytes(void);

/* Library version, major * 10000 + minor * 100 + patch. */
int drt3d_version(void);

#ifdef __cplusplus
}
#endif

#endif /* DRT3D_H */
