// adjoint_sum.cuh -- the last step of the planes adjoint: the sum over the
// selected dodecants of their backprojected frame volumes (Section 5.1's
// adjoint summed over the 12 dodecants of Algorithm 2).
#pragma once

#include "internal.cuh"

namespace drt3d {

// Frame i (the i-th selected dodecant, increasing k) holds the volume in that
// dodecant's frame, F_i[x'][y'][z'] (C-contiguous, N^3 elements).  Frame axis
// a (0: x', 1: y', 2: z') runs along volume axis vaxis[i][a] (0: x, 1: y,
// 2: z), reversed when flip[i][a] != 0.
struct FramesSum {
    const void* frame[kMaxSlots];
    signed char vaxis[kMaxSlots][3];
    signed char flip[kMaxSlots][3];
    void* vol;   // N^3 int32 or float32, overwritten
    int N;
    int nslots;
};

// The frame layout of dodecant k's affine map (A.sx, A.sy, A.sz are signed
// volume strides N^2, N or 1).
void frames_sum_axes(const Affine& A, int N, int i, FramesSum* S);

// vol = sum over i = 0 .. nslots-1 of frame i read through its axes, added
// in increasing i (a fixed order, so float sums are deterministic).
cudaError_t launch_frames_sum(const FramesSum& S, bool is_float, cudaStream_t s);

}  // namespace drt3d
