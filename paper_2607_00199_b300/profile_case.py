"""Minimal driver for profiler captures of the stage kernels on the benchmark
workload (K = 131072 jittered triangles, N = 4): set-up, `--warmup` steps, then
`--steps` steps, with as few other launches as possible.

    python -m paper_2607_00199_b300.profile_case --precision mixed|fp64 [--steps 2] [--warmup 2] [--n 256] [--warps 4]

The mixed kernel's launch shape is fixed by --warps (no tuning launches) so that
launch indices in a capture are the same from run to run: set-up launches, then
4 stage launches and one vertex update per step.
"""
import argparse

import torch

from paper_2607_00199_b300 import gb, inputs, state


def main():
    p = argparse.ArgumentParser()
    p.add_argument('--precision', choices=['mixed', 'fp64'], default='mixed')
    p.add_argument('--steps', type=int, default=2)
    p.add_argument('--warmup', type=int, default=2)
    p.add_argument('--n', type=int, default=256)
    p.add_argument('--N', type=int, default=4)
    p.add_argument('--warps', type=int, default=4, choices=[1, 2, 4])
    a = p.parse_args()
    prec = gb.GB_MIXED if a.precision == 'mixed' else gb.GB_FP64
    mesh = inputs.periodic_square_mesh(a.n, jitter=0.1)
    s = gb.Solver(mesh, a.N, 0.1, 1000.0, precision=prec, stream=torch.cuda.current_stream().cuda_stream)
    s.set_motion(0.05, 1.0)
    if prec == gb.GB_MIXED:
        s.set_launch_config(a.warps)
    s.set_graph(False)
    xy = s.nodes()
    rho, u, v = inputs.taylor_green(xy[..., 0], xy[..., 1], 0.1)
    s.set_fields(state.equilibrium_fields(rho, u, v, s.c), 0.0)
    dt = inputs.cfl_dt(mesh, a.N, s.c, 0.5)
    s.step(dt, a.warmup)
    s.sync()
    ms = s.step_timed(dt, a.steps)
    print('kernel ms per step:', [round(x / a.steps, 4) for x in ms])


if __name__ == '__main__':
    main()
