"""Small fixed workloads for profiling one kernel family at a time.

    python -m paper_2501_13664_gb300.profile_cases CASE [--reps R] [--schedule 4,4]

Each case builds its inputs with the seeded generators of ``synth``, runs the
transform ``reps`` times on the current stream, synchronises, checks the
device status word and prints one line.  The cases are sized for kernel
profilers: inputs larger than the 129 MB L2 where the kernel streams, a few GB
on the device at most.

    fused-n256-d1   N=256 uint8 volume (1% sparse + 8 digital planes of 255),
                    forward DRT of planes of dodecant 0 (both fused passes)
    fused-n256      the same volume, all 12 dodecants (2.4 GB of int32 out)
    inverse-n256    forward of dodecant 0, then its exact inverse
    lines-n64-s0    N=64 int16 volume (uniform 0..1023 + 32 lines), DJT of
                    sector 0 (268 MB of int32 out)
    lines-n128-s0   the config-3 volume (N=128 int16), DJT of sector 0
                    (4.3 GB of int32 out; first pass G = 4, second G = 3)
    batched-c4-n64  80 uint8 volumes with the N <= 64 sizes of the 96-volume
                    mixed batch, one persistent launch after one memset
    lines-adj-n64   the lines-n64-s0 transform, then its adjoint (backprojection)
    drt2d-n256      64 uint8 images of 256^2, 2D DRT over four quadrants
                    (134 MB of int32 out)
    press-n64       N=64 float32 phantom, two iterations of the multigrid
                    inverse (step sizes from the power iteration first)
    adj-f32-n128    N=128 float32 cotangent of all 12 dodecants (302 MB),
                    planes adjoint (backprojection) to the volume
    fwd-f32-n128    one config-5 volume (N=128 float32, N(0,1)), forward of all
                    12 dodecants (302 MB of float32 out)
"""
from __future__ import annotations

import argparse

import torch


def _sched(s: str):
    return tuple(int(x) for x in s.split(",")) if s else None


def main(argv=None) -> int:
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("case", choices=["fused-n256-d1", "fused-n256", "inverse-n256", "lines-n64-s0", "batched-c4-n64",
                                     "lines-adj-n64", "drt2d-n256", "press-n64", "adj-f32-n128",
                                     "lines-n128-s0", "fwd-f32-n128"])
    ap.add_argument("--reps", type=int, default=3)
    ap.add_argument("--schedule", type=str, default="4,4", help="stage-fusion split of the N=256 planes cases")
    args = ap.parse_args(argv)

    import synth

    from . import (ALL, BatchPlan, drt2d_forward, get_plan, lines_adjoint, lines_forward, planes_adjoint,
                   planes_forward, planes_inverse, planes_press_inverse, press_step_sizes)

    dev = torch.device("cuda", 0)
    sched = _sched(args.schedule)
    status = 0
    if args.case.startswith("fused") or args.case == "inverse-n256":
        N = 256
        vol = torch.from_numpy(synth.c2_volume(N)).to(dev)
        plan = get_plan(N, torch.uint8)
        if sched:
            plan.set_schedule(sched)
        mask = ALL if args.case == "fused-n256" else 1
        out = torch.empty((bin(mask).count("1"), N, N, 3 * N), dtype=torch.int32, device=dev)
        ws = plan.workspace("planes_forward")
        if args.case == "inverse-n256":
            planes_forward(vol, mask, out=out, workspace=ws)
            iplan = get_plan(N, torch.int32)
            iws = iplan.workspace("planes_inverse")
            f = torch.empty((N, N, N), dtype=torch.int32, device=dev)
            for _ in range(args.reps):
                planes_inverse(out[0], 0, out=f, workspace=iws, check=False)
            torch.cuda.synchronize()
            status = iplan.device_error()
            ok = bool(torch.equal(f, vol.to(torch.int32)))
            print(f"{args.case}: reps={args.reps} status={status} round_trip_equal={ok}")
            return 0 if (status == 0 and ok) else 1
        for _ in range(args.reps):
            planes_forward(vol, mask, out=out, workspace=ws)
        torch.cuda.synchronize()
        status = plan.device_error()
        print(f"{args.case}: reps={args.reps} schedule={plan.schedule()} status={status} sum={int(out[0].sum())}")
    elif args.case == "lines-adj-n64":
        N = 64
        vol = torch.from_numpy(synth.c3_volume(N)).to(dev)
        J = lines_forward(vol, [0])
        plan = get_plan(N, torch.int32)
        ws = plan.workspace("lines_adjoint")
        back = torch.empty((N, N, N), dtype=torch.int32, device=dev)
        for _ in range(args.reps):
            lines_adjoint(J, [0], out=back, workspace=ws)
        torch.cuda.synchronize()
        status = plan.device_error()
        print(f"{args.case}: reps={args.reps} status={status} sum={int(back.sum())}")
    elif args.case == "drt2d-n256":
        imgs = torch.from_numpy(synth.images_2d(256, 64)).to(dev)
        out = torch.empty((64, 4, 256, 512), dtype=torch.int32, device=dev)
        for _ in range(args.reps):
            drt2d_forward(imgs, range(4), out=out)
        torch.cuda.synchronize()
        print(f"{args.case}: reps={args.reps} sum={int(out.sum())}")
    elif args.case == "press-n64":
        N = 64
        f = torch.from_numpy(synth.phantom(N)).to(dev)
        R = planes_forward(f)
        steps = press_step_sizes(N)
        out = torch.empty_like(f)
        for _ in range(args.reps):
            planes_press_inverse(R, 2, 2, steps, out=out)
        torch.cuda.synchronize()
        err = float(torch.sqrt(torch.mean((out - f) ** 2)) / (f.max() - f.min()))
        print(f"{args.case}: reps={args.reps} nrmsd={err:.3e}")
    elif args.case == "adj-f32-n128":
        N = 128
        cot = torch.from_numpy(synth.random_float((12, N, N, 3 * N), 16)).to(dev)
        plan = get_plan(N, torch.float32)
        ws = plan.workspace("planes_adjoint")
        back = torch.empty((N, N, N), dtype=torch.float32, device=dev)
        for _ in range(args.reps):
            planes_adjoint(cot, ALL, out=back, workspace=ws)
        torch.cuda.synchronize()
        status = plan.device_error()
        print(f"{args.case}: reps={args.reps} status={status} sum={float(back.double().sum()):.6e}")
    elif args.case == "fwd-f32-n128":
        N = 128
        x = torch.from_numpy(synth.c5_batch(N=N, batch=1)[0]).to(dev)
        plan = get_plan(N, torch.float32)
        ws = plan.workspace("planes_forward")
        out = torch.empty((12, N, N, 3 * N), dtype=torch.float32, device=dev)
        for _ in range(args.reps):
            planes_forward(x, ALL, out=out, workspace=ws)
        torch.cuda.synchronize()
        status = plan.device_error()
        print(f"{args.case}: reps={args.reps} schedule={plan.schedule()} status={status} "
              f"sum={float(out.double().sum()):.6e}")
    elif args.case in ("lines-n64-s0", "lines-n128-s0"):
        N = 64 if args.case == "lines-n64-s0" else 128
        vol = torch.from_numpy(synth.c3_volume(N)).to(dev)
        plan = get_plan(N, torch.int16)
        out = torch.empty((1, N, N, 2 * N, 2 * N), dtype=torch.int32, device=dev)
        ws = plan.workspace("lines_forward")
        for _ in range(args.reps):
            lines_forward(vol, [0], out=out, workspace=ws)
        torch.cuda.synchronize()
        status = plan.device_error()
        print(f"{args.case}: reps={args.reps} status={status} sum={int(out[0].sum())}")
    else:
        sizes = [N for N in synth.c4_sizes() if N <= 64]
        vols = [torch.from_numpy(v).to(dev) for v in synth.c4_batch(sizes=sizes)]
        bp = BatchPlan(sizes)
        bp.bind(vols)
        for _ in range(args.reps):
            bp.run()
        torch.cuda.synchronize()
        status = bp.device_error()
        print(f"{args.case}: reps={args.reps} volumes={len(sizes)} status={status}")
    return 0 if status == 0 else 1


if __name__ == "__main__":
    raise SystemExit(main())
