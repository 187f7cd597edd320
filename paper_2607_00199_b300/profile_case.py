"""Minimal driver for profiler captures of the stage kernels on the benchmark
workload (K = 131072 jittered triangles, N = 4): set-up, `--warmup` steps, then
`--steps` steps, with as few other launches as possible.

    python -m paper_2607_00199_b300.profile_case --precision mixed|fp64 [--steps 2] [--warmup 2] [--n 256] [--warps 8]
    python -m paper_2607_00199_b300.profile_case --dim 3 --precision mixed|fp64 [--nx 64 --ny 16 --nz 16] [--N 3] [--shape3 1..8|16]
    python -m paper_2607_00199_b300.profile_case --airfoil [--no-pml] --precision mixed|fp64

With --airfoil the case is the plunging NACA 0012 O-grid (256 x 192 quads, K = 98304, N = 4)
with the outer 3-chord perfectly matched layer (r = 17..20 about mid-chord).
With --dim 3 the case is the deforming-channel workload (periodic box [0,8]x[0,2]x[0,2]
of nx x ny x nz hexes, 6 tetrahedra each, travelling-wave motion).

The mixed kernel's launch shape is fixed by --warps (8: the tcgen05 kernel; 1, 2, 4: the
mma.sync kernel's warps per CTA; no tuning launches) so that
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
    p.add_argument('--N', type=int, default=None, help='order (default 4 in 2D, 3 in 3D)')
    p.add_argument('--warps', type=int, default=8, choices=[1, 2, 4, 8], help='launch shape of the mixed kernel (8: tcgen05)')
    p.add_argument('--dim', type=int, default=2, choices=[2, 3])
    p.add_argument('--shape3', type=int, default=None, choices=[1, 2, 3, 4, 5, 6, 7, 8, 16],
                   help='dim 3, mixed: launch shape (1..8 the tensor-core kernel, warps per CTA; 16 one thread per node)')
    p.add_argument('--nx', type=int, default=64)
    p.add_argument('--ny', type=int, default=16)
    p.add_argument('--nz', type=int, default=16)
    p.add_argument('--airfoil', action='store_true')
    p.add_argument('--no-pml', action='store_true')
    a = p.parse_args()
    prec = gb.GB_MIXED if a.precision == 'mixed' else gb.GB_FP64
    if a.N is None:
        a.N = 4 if a.dim == 2 else 3
    if a.dim == 3:
        return main3(a, prec)
    if a.airfoil:
        return main_airfoil(a, prec)
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


def main_airfoil(a, prec):
    import math
    mesh = inputs.naca_ogrid_mesh(256, 192)
    far = (1.0, 1.0, 0.0)
    s = gb.Solver(mesh, a.N, 0.1, 1000.0, precision=prec, stream=torch.cuda.current_stream().cuda_stream,
                  far_state=far)
    s.set_motion(0.25, 2.0, kind=gb.GB_MOTION_PLUNGE)
    if not a.no_pml:
        c = s.c
        sigma_max = 3.0 * math.sqrt(3.0) * c * math.log(1e6) / (2.0 * 3.0)
        s.set_pml(gb.GB_PML_RADIAL, centre=(0.5, 0.0), r0=17.0, d=3.0, sigma_max=sigma_max, power=2.0, alpha=1.0)
    if prec == gb.GB_MIXED:
        s.set_launch_config(a.warps if a.warps != 8 else 4)   # boundary faces: the mma.sync kernel
    s.set_graph(False)
    xy = s.nodes()
    rho, u, v = inputs.free_stream(xy[..., 0], xy[..., 1], far[1], far[2])
    s.set_fields(state.equilibrium_fields(rho, u, v, s.c), 0.0)
    dt = inputs.cfl_dt(mesh, a.N, s.c, 0.5)
    s.step(dt, a.warmup)
    s.sync()
    ms = s.step_timed(dt, a.steps)
    print('kernel ms per step:', [round(x / a.steps, 4) for x in ms])


def main3(a, prec):
    import math
    mesh = inputs.periodic_box_tet_mesh(a.nx, a.ny, a.nz, L=(8.0, 2.0, 2.0))
    s = gb.Solver(mesh, a.N, 0.1, 500.0, precision=prec, stream=torch.cuda.current_stream().cuda_stream)
    s.set_wave_motion(0.02, 0.08, 8.0, 1.0, 2 * math.pi, 0.25, 1.0, 1.0)
    if prec == gb.GB_MIXED and a.shape3 is not None:
        s.set_launch_config(a.shape3)
    s.set_graph(False)
    xyz = s.nodes()
    rho, u, v, w = inputs.channel_flow_3d(xyz[..., 0], xyz[..., 1], xyz[..., 2], 0.1)
    s.set_fields(state.equilibrium_fields3(rho, u, v, w, s.c), 0.0)
    dt = inputs.cfl_dt_3d(mesh, a.N, s.c, 0.5)
    s.step(dt, a.warmup)
    s.sync()
    ms = s.step_timed(dt, a.steps)
    print('kernel ms per step:', [round(x / a.steps, 4) for x in ms])


if __name__ == '__main__':
    main()
