#!/usr/bin/env python
"""Benchmark of the SARK step on the 2D moving Taylor-Green vortex workload.

Workload: periodic [0, 2 pi]^2, 256 x 256 quads split into K = 131072
triangles with vertices jittered by +-10% of h (seeded), N = 4 (Np = 15),
6 Galerkin-Boltzmann fields, Ma = 0.1, Re = 1000, vertex motion
x = X + 0.05 sin(X) sin(Y) sin(2 pi t), CFL 0.5.  A "step" is one full SARK
step (4 stages: vertex positions, geometric factors, volume, surface,
cubature and update for every element).  Metric: DOF-stage updates/s with
DOF = K Np 6 and 4 stages per step.

Two paths are timed: GB_MIXED (FP32 perturbation fields, FP64 geometry and
SARK coefficients; the headline `value`) and GB_FP64 (the reference form).
Both start from the same state and take the same steps; the mixed path's
error against the FP64 path is reported.  Under torchrun each rank runs an
independent replica on its own GPU (no collective on the data path).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
"""
import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOAD = dict(n=256, N=4, Ma=0.1, Re=1000.0, A=0.05, T=1.0, jitter=0.1, cfl=0.5)
WORKLOAD_NAME = ('2D moving Taylor-Green vortex: periodic [0,2pi]^2, 256x256 quads -> K=131072 triangles, '
                 'vertices jittered +-10% h (seed 260700199), N=4 (Np=15), 6 fields, Ma=0.1, Re=1000, '
                 'motion A=0.05 T=1, CFL 0.5')
PEAKS_FILE = os.path.join(ROOT, 'MEASURED_PEAKS.json')
TRAFFIC_FILE = os.path.join(ROOT, 'profiles', 'stage_kernel_traffic.json')
# FP64 pipe: 2 FMA per clock per SM on B300 (measured 1.127 TFLOP/s at 1935 MHz with the
# FMA probe in paper_2607_00199_b300/csrc/peak_probe.cu); peak = 148 SMs x 4 flop x 2032 MHz.
FP64_FLOP_PER_CLK_SM = 4.0


def run_serving(torch, n_req=256, steps=500, rate=50.0, budget_gib=None):
    """Serving stream of independent moving-mesh simulations: n_req requests with Poisson
    arrivals, K in {2048 .. 131072}, N in {2 .. 5}, random motion and Re, `steps` SARK
    steps each (GB_MIXED), admitted against a device-memory budget (default: 80% of the
    free device memory) and stepped by the continuous-batching loop: small requests in
    groups per (N, size class), large ones alone, every unit on its own stream at its own
    cadence.  Baselines: the same requests run one after another alone, in GB_FP64 and in
    GB_MIXED (tuned launch shape), from per-(K, N) step times measured here first; each
    request's slowdown is its completion latency over its time alone in GB_MIXED."""
    from paper_2607_00199_b300 import gb, inputs, serve, state
    reqs = inputs.serving_requests(n_req, rate=rate, seed=1)
    stream = torch.cuda.Stream()
    setup = torch.cuda.Stream()
    # per-bucket step times of a request running alone
    alone = {}
    for prec, name, nst in ((gb.GB_FP64, 'fp64', 2), (gb.GB_MIXED, 'mixed', 10)):
        for K in sorted({r['K'] for r in reqs}):
            for N in sorted({r['N'] for r in reqs}):
                spec = {'id': -1, 'arrival': 0.0, 'n': int(round(math.sqrt(K / 2))), 'N': N, 'A': 0.05, 'T': 1.0,
                        'Re': 1000.0, 'Ma': 0.1}
                rq = serve.Request(spec, stream.cuda_stream, precision=prec)
                rq.solver.step(rq.dt, 2)
                stream.synchronize()
                t0 = time.perf_counter()
                rq.solver.step(rq.dt, nst)
                rq.solver.sync()
                alone[(name, K, N)] = (time.perf_counter() - t0) / nst
                rq.solver.close()
    alone_ms = {(K, N): alone[('mixed', K, N)] * 1e3 for (nm, K, N) in alone if nm == 'mixed'}
    budget = None if budget_gib is None else int(budget_gib * 2 ** 30)
    srv = serve.Server(budget, stream.cuda_stream, steps_per_request=steps, setup_stream=setup.cuda_stream,
                       alone_ms=alone_ms)
    stats = srv.run(reqs)
    work = sum(2 * r['n'] ** 2 * ((r['N'] + 1) * (r['N'] + 2) // 2) * 6 * 4 * steps for r in reqs)
    t_fp64 = sum(alone[('fp64', r['K'], r['N'])] * steps for r in reqs)
    t_mixed = sum(alone[('mixed', r['K'], r['N'])] * steps for r in reqs)
    return {'workload': '%d requests, Poisson %.0f/s (seed 1), K in {2048,8192,32768,131072}, N in {2,3,4,5}, '
                        'A~U[0.01,0.08], T~U[0.5,2], Re~U[100,2000], Ma 0.1, %d SARK steps each, GB_MIXED; '
                        'device-memory budget %.1f GiB (%s); small requests grouped per (N, size class), '
                        'K >= 32768 alone, every unit on its own stream'
                        % (n_req, rate, steps, stats['budget_bytes'] / 2 ** 30,
                           'given' if budget_gib is not None else '80% of the free device memory'),
            'dof_stage_per_s': stats['dof_stage_per_s'], 'wall_s': stats['wall_s'], 'launches': stats['launches'],
            'step_latency_ms': stats['step_latency_ms'], 'completion_latency_s': stats['completion_latency_s'],
            'slowdown_vs_alone': stats.get('slowdown_vs_alone'),
            'peak_device_bytes': stats['peak_device_bytes'], 'budget_bytes': stats['budget_bytes'],
            'alone_fp64_dof_stage_per_s': work / t_fp64, 'alone_mixed_dof_stage_per_s': work / t_mixed,
            'speedup_vs_alone_fp64': (work / stats['wall_s']) / (work / t_fp64),
            'speedup_vs_alone_mixed': (work / stats['wall_s']) / (work / t_mixed),
            'note': 'aggregate rate = all DOF-stage updates / wall time from the first arrival to the last '
                    'completion (includes set-up of each request and idle time before arrivals); slowdown = '
                    'completion latency (arrival to last step) / the request\'s steps x its alone step time'}


WORKLOAD3 = dict(dims=(64, 16, 16), L=(8.0, 2.0, 2.0), N=3, Ma=0.1, Re=500.0, cfl=0.5,
                 wave=dict(A0=0.02, A1=0.08, Lx=8.0, wavelength=1.0, omega=2 * math.pi, r0sq=0.25, yc=1.0, zc=1.0))
WORKLOAD3_NAME = ('3D deforming channel: periodic box [0,8]x[0,2]x[0,2], 64x16x16 hexes -> K=98304 tetrahedra '
                  '(6 per hex), N=3 (Np=20), 10 fields, Ma=0.1, Re=500, y += (0.02+0.08x/8) sin(2 pi x - 2 pi t) '
                  'exp(-r^2/0.25), CFL 0.5, uniform stream u=1 with a small transverse disturbance')


WORKLOAD_TGV = dict(n=24, N=3, Ma=0.1, Re=1600.0, cfl=0.5, A=math.pi / 6, T=20.0, L=2 * math.pi)
WORKLOAD_TGV_NAME = ('3D moving Taylor-Green vortex at the paper\'s per-GPU load: periodic cube [-pi,pi]^3, 24^3 hexes '
                     '-> K=82944 tetrahedra (6 per hex), N=3 (Np=20), 10 fields, Ma=0.1, Re=1600, deformation '
                     'x_d += (pi/6) sin(2 pi t/20) S(X_a) S(X_b), S(s) = sin(2 pi (s + pi)/(2 pi)), CFL 0.5, '
                     'Taylor-Green initial state')
# the paper's only timing (Sec. 7.2 weak-scaling table): 82944 tetrahedra per GPU, N = 3, one node of
# 4 NVIDIA H100 (MareNostrum 5), mean t_step over 1000 SARK steps; context, another machine
PAPER_TGV_T_STEP_MS = 14.18


def sizes3(N):
    Np, Nfp = (N + 1) * (N + 2) * (N + 3) // 6, (N + 1) * (N + 2) // 2
    qc = (3 * N + 2) // 2
    return Np, Nfp, qc ** 3


def flops3_per_element_stage(N):
    """Algorithmic flops (FMA = 2) of one tetrahedron-stage of the fused 3D RHS + update."""
    Np, Nfp, Nc = sizes3(N)
    macs = 3 * 10 * Np * Np + 10 * Np * 4 * Nfp + 4 * Nc * Np + 6 * Np * Nc   # Dr Ds Dt, LIFT, I, P
    volume = Np * 250         # chain rule 180, v_G interpolation 8, At_x/y/z products 42, sums 20
    surface = 4 * Nfp * 190   # jump 10, four At_n products 120, upwind/ALE combination 60
    cubature = Nc * 24        # Ntilde with one division
    update = 10 * Np * 4
    return 2 * macs + volume + surface + cubature + update


def bytes3_per_step(K, N, nv, elem_bytes):
    """Algorithmic HBM bytes of the 4 stage launches of one 3D step: 18 field arrays,
    plus per launch the 48-byte mesh record of every element and x_n (24 B) and the
    velocity shapes S1, S2 (48 B) of every unique vertex."""
    Np, _, _ = sizes3(N)
    return 18 * K * 10 * Np * elem_bytes + 4 * (48 * K + 72 * nv)


def run_3d(torch, steps_fp64=10, steps_mixed=50, warmup=3, tgv=False):
    """A 3D workload, FP64 and GB_MIXED (the tuned one of the two mixed kernels: the
    tensor-core kernel, mma.sync TF32 split products in 16-element warp tiles, or the FP32
    one-thread-per-node kernel; both are timed and reported), timed like the 2D headline
    (CUDA-graph step replay between CUDA events), with the mixed path's error against the FP64
    path after the same steps: the deforming channel, or (tgv) the moving Taylor-Green vortex
    at the per-GPU load of the paper's timing."""
    from paper_2607_00199_b300 import gb, inputs, state
    W = WORKLOAD_TGV if tgv else WORKLOAD3
    mesh = inputs.tgv_box_tet_mesh(W['n']) if tgv else inputs.periodic_box_tet_mesh(*W['dims'], L=W['L'])
    tstream = torch.cuda.Stream()
    N = W['N']
    Np, Nfp, Nc = sizes3(N)
    hbm, sm_max, peak_kind = load_peaks()
    res = {}
    qend = {}
    shapes = {}
    for name, prec, steps in (('fp64', gb.GB_FP64, steps_fp64), ('mixed', gb.GB_MIXED, steps_mixed),
                              ('mixed_other', gb.GB_MIXED, steps_mixed)):
        s = gb.Solver(mesh, N, W['Ma'], W['Re'], precision=prec, stream=tstream.cuda_stream)
        if name == 'mixed_other':
            other = 16 if shapes['mixed'] != 16 else 7
            try:
                s.set_launch_config(other)
            except gb.GBError:
                s.close()
                continue
        xyz = s.nodes()
        if tgv:
            s.set_tgv_motion(W['A'], W['T'], W['L'])
            rho, u, v, w = inputs.taylor_green_3d(xyz[..., 0], xyz[..., 1], xyz[..., 2], W['Ma'])
        else:
            s.set_wave_motion(**W['wave'])
            rho, u, v, w = inputs.channel_flow_3d(xyz[..., 0], xyz[..., 1], xyz[..., 2], W['Ma'])
        q0 = state.equilibrium_fields3(rho, u, v, w, s.c)
        dt = inputs.cfl_dt_3d(mesh, N, s.c, W['cfl'])
        ms, kms = time_path(torch, s, q0, dt, steps, warmup, lambda: None, tstream)
        shapes[name] = s.launch_config()
        if name == 'mixed_other':
            res['mixed']['other_kernel'] = {'launch_shape': shapes[name], 'ms_per_step': ms / steps,
                                            'mean_launch_ms': float(sum(kms[:4])) / (4 * steps)}
            s.close()
            continue
        # same state and steps for the error comparison
        s.set_vertices(mesh['X'])
        s.set_fields(q0, 0.0)
        s.step(dt, 10)
        qend[name], _ = s.fields()
        stage_ms = float(sum(kms[:4]))
        dof = s.K * Np * 10
        ebytes = 8 if prec == gb.GB_FP64 else 4
        alg = bytes3_per_step(s.K, N, s.nv, ebytes)
        fl = flops3_per_element_stage(N) * s.K * 4
        gbs = alg * steps / (stage_ms / 1e3) / 1e9
        tfl = fl * steps / (stage_ms / 1e3) / 1e12
        r = {'value': dof * 4 * steps / (ms / 1e3), 'ms_per_step': ms / steps, 'steps': steps, 'warmup': warmup,
             'kernel_ms_per_step': [x / steps for x in kms], 'mean_launch_ms': stage_ms / (4 * steps),
             'hbm': {'achieved_gbs': gbs, 'peak_gbs': hbm, 'frac': gbs / hbm, 'algorithmic_bytes_per_step': alg},
             'algorithmic_flops_per_element_stage': flops3_per_element_stage(N)}
        if prec == gb.GB_FP64:
            peak = 148 * FP64_FLOP_PER_CLK_SM * sm_max * 1e6 / 1e12
            r['roofline'] = {'bound': 'alu', 'achieved': tfl, 'peak': peak, 'unit': 'TFLOP/s', 'frac': tfl / peak,
                             'kernel': 'stage3_kernel<double,3,*>',
                             'peak_source': 'FP64 pipe: 148 SMs x 2 FMA/clk x 2 flop x %.0f MHz' % sm_max}
        else:
            shape = shapes[name]
            r['launch_shape'] = shape
            r['kernel'] = ('stage3_kernel<float,3,*> (FP32, one thread per node)' if shape == 16 else
                           'tc3_stage_kernel<3,*> (mma.sync TF32 split products, %d warps per CTA)' % shape)
            r['roofline'] = {'bound': 'hbm', 'achieved': gbs, 'peak': hbm, 'unit': 'GB/s', 'frac': gbs / hbm,
                             'kernel': r['kernel'], 'peak_source': '%s hbm_gbs (MEASURED_PEAKS.json)' % peak_kind}
        res[name] = r
        K, nv = s.K, s.nv
        s.close()
    rest = np.zeros_like(qend['fp64'])
    rest[:, 0, :] = 1.0
    dq = qend['mixed'] - qend['fp64']
    out = {'workload': WORKLOAD_TGV_NAME if tgv else WORKLOAD3_NAME, 'K': K, 'n_vert': nv, 'N': N, 'Np': Np,
           'fields': 10, 'dof': K * Np * 10}
    if tgv:
        out['paper_context'] = {
            't_step_ms': PAPER_TGV_T_STEP_MS, 'hardware': '4x NVIDIA H100 (one MareNostrum 5 node), 82944 tets per GPU',
            'precision': 'not stated', 'ratio_fp64': PAPER_TGV_T_STEP_MS / res['fp64']['ms_per_step'],
            'ratio_mixed': PAPER_TGV_T_STEP_MS / res['mixed']['ms_per_step'],
            'note': 'paper t_step / this t_step on one B300; another machine and a multi-GPU run: context, not a target'}
    return dict(out, **{
            'metric': 'DOF-stage updates/s', 'fp64': res['fp64'], 'mixed': res['mixed'],
            'mixed_speedup_vs_fp64': res['mixed']['value'] / res['fp64']['value'],
            'mixed_error': {'rel_l2_fields': float(np.linalg.norm(dq) / np.linalg.norm(qend['fp64'])),
                            'rel_l2_perturbation': float(np.linalg.norm(dq) / np.linalg.norm(qend['fp64'] - rest)),
                            'steps': 10, 'against': 'GB_FP64 3D path (oracle-parity-tested) from the same state'},
            'timing': 'ms_per_step: gb_step (CUDA graph replay) between CUDA events; inputs larger than L2 '
                      '(FP64 state %d MB per array, FP32 %d MB)' % (K * Np * 80 // 10 ** 6, K * Np * 40 // 10 ** 6)})


WORKLOAD_AF = dict(ni=256, nj=192, R=20.0, N=4, Ma=0.1, Re=1000.0, A=0.25, T=2.0, far=(1.0, 1.0, 0.0), cfl=0.5,
                   pml=dict(r0=17.0, d=3.0, power=2.0, alpha=1.0, reflection=1e-6))
WORKLOAD_AF_NAME = ('2D plunging NACA 0012 airfoil: O-grid of 256 wrap-around x 192 radial quads (geometric growth 1.02, '
                    'radius 20 chords) -> K=98304 triangles, N=4, 6 fields, Ma=0.1, Re=1000, rigid plunge '
                    'h(t)=0.25 sin(2 pi 0.5 t), walls on the airfoil (bounce-back about the wall velocity), outer 3-chord '
                    'perfectly matched layer (radial, r = 17..20 about mid-chord, sigma ~ ((r-17)/3)^2, auxiliary fields '
                    'on the layer elements) in front of the free-stream far field, whole SARK step captured as a CUDA graph')


def run_airfoil(torch, steps=50, warmup=3):
    """The plunging-airfoil workload (throughput; the paper's drag and lift comparisons need
    its published curves): GB_MIXED and GB_FP64, timed like the headline."""
    from paper_2607_00199_b300 import gb, inputs, state
    W = WORKLOAD_AF
    mesh = inputs.naca_ogrid_mesh(W['ni'], W['nj'], R=W['R'])
    tstream = torch.cuda.Stream()
    Np, _, _ = sizes(W['N'])
    hbm, sm_max, _ = load_peaks()
    out = {'workload': WORKLOAD_AF_NAME, 'K': int(mesh['EToV'].shape[0]), 'N': W['N'], 'Np': Np, 'fields': 6}
    P = W['pml']
    c = 1.0 / W['Ma']
    # sigma_max for the continuous layer's normal-incidence round trip exp(-2 int sigma / (sqrt3 c)) = R
    sigma_max = (P['power'] + 1.0) * math.sqrt(3.0) * c * math.log(1.0 / P['reflection']) / (2.0 * P['d'])
    out['pml'] = dict(P, sigma_max=sigma_max, centre=(0.5, 0.0))
    legs = (('mixed', gb.GB_MIXED, steps, True), ('mixed_no_pml', gb.GB_MIXED, steps, False),
            ('fp64', gb.GB_FP64, max(4, steps // 10), True))
    for name, prec, nst, layer in legs:
        s = gb.Solver(mesh, W['N'], W['Ma'], W['Re'], precision=prec, stream=tstream.cuda_stream, far_state=W['far'])
        s.set_motion(W['A'], W['T'], kind=gb.GB_MOTION_PLUNGE)
        if layer:
            s.set_pml(gb.GB_PML_RADIAL, centre=(0.5, 0.0), r0=P['r0'], d=P['d'], sigma_max=sigma_max,
                      power=P['power'], alpha=P['alpha'])
            out['pml']['n_layer_elements'] = int(s.pml_fields()[1].shape[0])
        xy = s.nodes()
        rho, u, v = inputs.free_stream(xy[..., 0], xy[..., 1], W['far'][1], W['far'][2])
        q0 = state.equilibrium_fields(rho, u, v, s.c)
        dt = inputs.cfl_dt(mesh, W['N'], s.c, W['cfl'])
        ms, kms = time_path(torch, s, q0, dt, nst, warmup, lambda: None, tstream)
        dof = s.K * Np * 6
        stage_ms = float(sum(kms[:4]))
        r = {'value': dof * 4 * nst / (ms / 1e3), 'ms_per_step': ms / nst, 'steps': nst, 'warmup': warmup,
             'kernel_ms_per_step': [x / nst for x in kms], 'pml': layer}
        if name == 'mixed_no_pml':
            out[name] = {'ms_per_step': ms / nst, 'value': r['value']}
            s.close()
            continue
        if prec == gb.GB_MIXED:
            alg = bytes_per_step(s.K, W['N'], s.nv, 4)
            gbs = alg * nst / (stage_ms / 1e3) / 1e9
            r['roofline'] = {'bound': 'hbm', 'achieved': gbs, 'peak': hbm, 'unit': 'GB/s', 'frac': gbs / hbm,
                             'kernel': 'tc_stage_kernel<4,*,BC> + pml_stage_kernel (4 + 4 launches per step)'}
        else:
            fl = flops_per_element_stage(W['N']) * s.K * 4 * nst / (stage_ms / 1e3) / 1e12
            peak = 148 * FP64_FLOP_PER_CLK_SM * sm_max * 1e6 / 1e12
            r['roofline'] = {'bound': 'alu', 'achieved': fl, 'peak': peak, 'unit': 'TFLOP/s', 'frac': fl / peak,
                             'kernel': 'stage_kernel<double,4,*,BC>'}
        out[name] = r
        s.close()
    out['mixed_speedup_vs_fp64'] = out['mixed']['value'] / out['fp64']['value']
    out['pml_overhead_mixed'] = out['mixed']['ms_per_step'] / out['mixed_no_pml']['ms_per_step'] - 1.0
    out['note'] = ('throughput only; dt from CFL 0.5 on the thinnest O-grid cell, so a step covers little physical '
                   'time; the per-step cost is what is measured')
    return out


def parse():
    p = argparse.ArgumentParser()
    p.add_argument('--gpus', type=int, default=1)
    p.add_argument('--steps', type=int, default=100)
    p.add_argument('--warmup', type=int, default=5)
    p.add_argument('--impl', choices=['ours', 'reference'], default='ours')
    p.add_argument('--no-cpu-baseline', action='store_true')
    p.add_argument('--no-long-error', action='store_true', help='skip the 1000-step mixed-vs-FP64 error run')
    p.add_argument('--no-serve', action='store_true', help='skip the serving-stream measurement')
    p.add_argument('--serve-only', action='store_true', help='only the serving-stream measurement')
    p.add_argument('--no-3d', action='store_true',
                   help='skip the 3D measurements (deforming channel, moving Taylor-Green vortex)')
    p.add_argument('--no-airfoil', action='store_true', help='skip the plunging-airfoil measurement')
    p.add_argument('--serve-requests', type=int, default=256)
    p.add_argument('--serve-steps', type=int, default=500)
    return p.parse_args()


# ---------------------------------------------------------------------------
# algorithmic work per element-stage: the operations and bytes each stage kernel must do and move
# ---------------------------------------------------------------------------
def sizes(N):
    Np, Nfp = (N + 1) * (N + 2) // 2, N + 1
    qc = (3 * N + 2) // 2
    return Np, Nfp, qc * qc


def flops_per_element_stage(N):
    """Algorithmic flops (FMA = 2) of one element-stage of the fused RHS + update."""
    Np, Nfp, Nc = sizes(N)
    macs = 2 * 6 * Np * Np + 6 * Np * 3 * Nfp + 3 * Nc * Np + 3 * Np * Nc   # Dr, Ds, LIFT, I, P
    volume = Np * 86          # chain rule 36, flux terms 16, v_G . grad 24, v_G interpolation 10
    surface = 3 * Nfp * 95    # jump 6, upwind blocks 64, ALE 12, v_G . n 13
    cubature = Nc * 12        # Ntilde with one division
    update = 6 * Np * 4
    return 2 * macs + volume + surface + cubature + update


def bytes_per_step(K, N, nv, elem_bytes):
    """Algorithmic HBM bytes of the 4 stage launches of one step: 18 field arrays
    (3 + 5 + 6 + 4 reads/writes), plus per launch the 32-byte mesh record of every
    element and x_n and S(X) (32 bytes) of every unique vertex."""
    Np, _, _ = sizes(N)
    return 18 * K * 6 * Np * elem_bytes + 4 * (32 * K + 32 * nv)


# ---------------------------------------------------------------------------
# environment helpers
# ---------------------------------------------------------------------------
def max_over_ranks(dist, x, device='cuda'):
    """The largest value of x over the ranks (the job's timed region ends when the
    slowest replica ends); x itself without a process group."""
    if dist is None:
        return x
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def aggregate_rate(world_size, units_per_rank, seconds):
    """Whole-job throughput of independent replicas: every rank processes the same
    units (weak scaling), divided by the max-over-ranks time."""
    return world_size * units_per_rank / seconds


def dist_env():
    ws = int(os.environ.get('WORLD_SIZE', '1'))
    rank = int(os.environ.get('RANK', '0'))
    local = int(os.environ.get('LOCAL_RANK', '0'))
    return ws, rank, local


class ClockSampler:
    """nvidia-smi clock/throttle samples every 200 ms while running."""
    FIELDS = ('index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,'
              'clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,'
              'clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap')

    def __init__(self, index):
        self.index = index
        self.file = tempfile.NamedTemporaryFile('w+', suffix='.csv', delete=False)
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(['nvidia-smi', '--query-gpu=' + self.FIELDS, '--format=csv,noheader,nounits',
                                          '-lms', '200', '-i', str(self.index)],
                                         stdout=self.file, stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        self.file.flush()
        rows = []
        try:
            with open(self.file.name) as f:
                for line in f:
                    parts = [x.strip() for x in line.split(',')]
                    if len(parts) >= 9 and parts[1].replace('.', '').isdigit():
                        rows.append(parts)
        except OSError:
            pass
        finally:
            try:
                os.unlink(self.file.name)
            except OSError:
                pass
        if not rows:
            return {'sm_mhz': None, 'sm_max_mhz': None, 'reasons': ['unavailable'], 'samples': 0}
        sm = [float(r[1]) for r in rows]
        reasons = set()
        names = ['hw_slowdown', 'hw_thermal_slowdown', 'sw_thermal_slowdown', 'sw_power_cap']
        for r in rows:
            for k, nm in enumerate(names):
                if r[5 + k].lower().startswith('active'):
                    reasons.add(nm)
        return {'sm_mhz': statistics.median(sm), 'sm_max_mhz': float(rows[0][2]), 'reasons': sorted(reasons),
                'samples': len(rows), 'power_w_max': max(float(r[3]) for r in rows if r[3].replace('.', '').isdigit())}


def load_peaks():
    try:
        with open(PEAKS_FILE) as f:
            d = json.load(f)
        return float(d['hbm_gbs']), float(d.get('sm_max_mhz', 2032.0)), 'measured'
    except (OSError, KeyError, ValueError):
        return 6400.0, 2032.0, 'fallback'


def recorded_traffic(key):
    """DRAM bytes per launch (average over the 4 stage launches of a step) of the
    stage kernel from a committed ncu capture ('mixed': the warp-tile mma.sync kernel,
    'mixed_um': the tcgen05 kernel, 'fp64'), or None if that kernel's source file
    changed since the capture was taken."""
    try:
        with open(TRAFFIC_FILE) as f:
            d = json.load(f)[key]
        src = os.path.join(ROOT, d['kernel_source'])
        if hashlib.sha256(open(src, 'rb').read()).hexdigest() != d['kernel_source_sha256']:
            return None
        return d['dram_bytes_per_launch_avg']
    except (OSError, KeyError, ValueError):
        return None


# ---------------------------------------------------------------------------
# our arm
# ---------------------------------------------------------------------------
def make_case(gb, inputs, state, precision, stream):
    W = WORKLOAD
    mesh = inputs.periodic_square_mesh(W['n'], jitter=W['jitter'])
    s = gb.Solver(mesh, W['N'], W['Ma'], W['Re'], precision=precision, stream=stream)
    s.set_motion(W['A'], W['T'])
    xy = s.nodes()
    rho, u, v = inputs.taylor_green(xy[..., 0], xy[..., 1], W['Ma'])
    q0 = state.equilibrium_fields(rho, u, v, s.c)
    dt = inputs.cfl_dt(mesh, W['N'], s.c, W['cfl'])
    return s, q0, dt


def time_path(torch, s, q0, dt, steps, warmup, barrier, stream):
    """Timed region 1 (the reported time): `steps` SARK steps through gb_step, which
    replays one captured CUDA graph per step, bracketed by CUDA events on the
    solver's stream.  Timed region 2 (the per-kernel breakdown for the roofline):
    the same number of steps through gb_step_timed, which records an event pair
    around every kernel launch (direct launches)."""
    s.set_fields(q0, 0.0)
    s.step(dt, warmup)
    s.sync()
    barrier()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    s.step(dt, steps)
    e1.record(stream)
    torch.cuda.synchronize()
    barrier()
    ms = e0.elapsed_time(e1)
    s.set_fields(q0, 0.0)
    s.step(dt, warmup)
    s.sync()
    kernel_ms = s.step_timed(dt, steps)
    torch.cuda.synchronize()
    return ms, kernel_ms


class _SingleThreadBLAS:
    """Limit BLAS threads when threadpoolctl is available (the oracle's einsum and
    batched small linalg calls are single-threaded either way)."""

    def __enter__(self):
        try:
            from threadpoolctl import threadpool_limits
            self._ctx = threadpool_limits(1)
        except ImportError:
            self._ctx = None
        return self

    def __exit__(self, *exc):
        if self._ctx is not None:
            self._ctx.__exit__(*exc)


def _cores_used(cpu_s, wall_s):
    return max(1, int(round(cpu_s / max(wall_s, 1e-9))))


def _oracle_replica(job):
    """One replica of the oracle sample (a spawned process): set up, wait for the others,
    time `steps` SARK steps; returns (DOF-stage updates, seconds)."""
    n, steps, barrier = job if len(job) == 3 else (job[0], job[1], None)
    import sys
    sys.path.insert(0, ROOT)
    from oracle import physics
    from oracle.solver import Motion, OracleSolver
    from paper_2607_00199_b300 import inputs
    W = WORKLOAD
    with _SingleThreadBLAS():
        mesh = inputs.periodic_square_mesh(n, jitter=W['jitter'])
        o = OracleSolver(mesh, W['N'], Ma=W['Ma'], Re=W['Re'], motion=Motion(W['A'], W['T']))
        xn = o.node_coords(o.X)
        rho, u, v = inputs.taylor_green(xn[..., 0], xn[..., 1], W['Ma'])
        q = np.ascontiguousarray(physics.equilibrium_state(rho, u, v, o.c).transpose(0, 2, 1))
        dt = inputs.cfl_dt(mesh, W['N'], o.c, W['cfl'])
        if barrier is not None:
            barrier.wait()
        t0 = time.perf_counter()
        o.run(q, o.X.copy(), 0.0, dt, steps)
        el = time.perf_counter() - t0
    Np, _, _ = sizes(W['N'])
    return o.K * Np * 6 * 4 * steps, el


def cpu_baseline_all_cores(steps_sample=2, n_sample=64):
    """The oracle as it stands on every host core: one replica per core (spawned processes,
    a common start), each running the bounded sample; rate = all updates over the longest
    replica's time."""
    import multiprocessing as mp
    ctx = mp.get_context('spawn')
    P = os.cpu_count() or 1
    mgr = ctx.Manager()
    bar = mgr.Barrier(P)
    with ctx.Pool(P) as pool:
        res = pool.map(_oracle_replica, [(n_sample, steps_sample, bar)] * P)
    mgr.shutdown()
    work = sum(r[0] for r in res)
    el = max(r[1] for r in res)
    return {'value': work / el, 'unit': 'DOF-stage updates/s', 'cores': P, 'kind': 'oracle', 'nproc': P,
            'sample': '%d replicas (one per host core, spawned processes, common start), each %d SARK steps '
                      'of the same method on a %dx%d jittered mesh (K=%d, N=%d), numpy FP64 on one thread; '
                      'longest replica %.1f s' % (P, steps_sample, n_sample, n_sample, 2 * n_sample ** 2,
                                                  WORKLOAD['N'], el)}


def cpu_baseline(steps_sample=2, n_sample=128):
    """The oracle, as it stands, on a bounded sample of the workload (one host core)."""
    from oracle import physics
    from oracle.solver import Motion, OracleSolver
    from paper_2607_00199_b300 import inputs
    W = WORKLOAD
    with _SingleThreadBLAS():
        mesh = inputs.periodic_square_mesh(n_sample, jitter=W['jitter'])
        o = OracleSolver(mesh, W['N'], Ma=W['Ma'], Re=W['Re'], motion=Motion(W['A'], W['T']))
        xn = o.node_coords(o.X)
        rho, u, v = inputs.taylor_green(xn[..., 0], xn[..., 1], W['Ma'])
        q = np.ascontiguousarray(physics.equilibrium_state(rho, u, v, o.c).transpose(0, 2, 1))
        dt = inputs.cfl_dt(mesh, W['N'], o.c, W['cfl'])
        c0, t0 = time.process_time(), time.perf_counter()
        o.run(q, o.X.copy(), 0.0, dt, steps_sample)
        el, cpu = time.perf_counter() - t0, time.process_time() - c0
    Np, _, _ = sizes(W['N'])
    dof = o.K * Np * 6
    return {'value': dof * 4 * steps_sample / el, 'unit': 'DOF-stage updates/s', 'cores': _cores_used(cpu, el),
            'kind': 'oracle',
            'nproc': os.cpu_count(),
            'sample': '%d SARK steps of the same method on a %dx%d jittered mesh (K=%d, N=%d), numpy FP64 on '
                      'one thread; %.1f s wall, %.1f s CPU (cores = CPU/wall, rounded)'
                      % (steps_sample, n_sample, n_sample, o.K, W['N'], el, cpu)}


def long_error(results, steps):
    """The error of the mixed path after `steps` SARK steps of the benchmark workload,
    against the FP64 path run from the same initial state (the FP64 path matches the oracle
    to 1e-10 after 100 steps and at full size per step, in the GPU parity tests)."""
    out = {}
    q = {}
    for name in ('mixed', 'fp64'):
        r = results[name]
        s = r['solver']
        s.set_fields(r['q0'], 0.0)
        t0 = time.perf_counter()
        s.step(r['dt'], steps)
        q[name], _ = s.fields()
        out['%s_s' % name] = time.perf_counter() - t0
    qm, qf = q['mixed'], q['fp64']
    rest = np.zeros_like(qf)
    rest[:, 0, :] = 1.0
    dq = qm - qf
    out.update({'steps': steps, 'rel_l2_fields': float(np.linalg.norm(dq) / np.linalg.norm(qf)),
                'rel_l2_perturbation': float(np.linalg.norm(dq) / np.linalg.norm(qf - rest)),
                'max_abs_over_max_perturbation': float(np.abs(dq).max() / np.abs(qf - rest).max()),
                'against': 'GB_FP64 path from the same state'})
    return out


def run_ours(args):
    import torch
    ws, rank, local = dist_env()
    if ws != args.gpus:
        raise SystemExit('--gpus %d but WORLD_SIZE %d' % (args.gpus, ws))
    torch.cuda.set_device(local)
    dist = None
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group('nccl', device_id=torch.device('cuda', local))
    barrier = (lambda: dist.barrier()) if dist else (lambda: None)

    from paper_2607_00199_b300 import gb, inputs, state
    W = WORKLOAD
    tstream = torch.cuda.Stream()          # a non-default stream: gb_step replays CUDA graphs
    stream = tstream.cuda_stream
    Np, Nfp, Nc = sizes(W['N'])
    results = {}
    sampler = ClockSampler(local)
    with sampler:
        for name, prec in (('mixed', gb.GB_MIXED), ('fp64', gb.GB_FP64)):
            s, q0, dt = make_case(gb, inputs, state, prec, stream)
            ms, kms = time_path(torch, s, q0, dt, args.steps, args.warmup, barrier, tstream)
            q_end, _ = s.fields()
            results[name] = dict(ms=ms, kernel_ms=kms, solver=s, q_end=q_end, q0=q0, dt=dt,
                                 warps=s.launch_config())
    clocks = sampler.summary()

    K = results['mixed']['solver'].K
    nv = results['mixed']['solver'].nv
    dof = K * Np * 6
    hbm, sm_max, peak_kind = load_peaks()
    out = {}
    for name in ('mixed', 'fp64'):
        r = results[name]
        ms = max_over_ranks(dist, r['ms'])
        stage_ms = float(sum(r['kernel_ms'][:4]))
        v = aggregate_rate(ws, dof * 4 * args.steps, ms / 1e3)
        ebytes = 4 if name == 'mixed' else 8
        if name == 'mixed':
            # the stage kernels' time inside the graph-timed steps: ms_per_step times the
            # stage kernels' share of the per-launch event pass (the vertex update is the rest),
            # so that the kernel time never exceeds the step it is part of
            event_ms = float(sum(r['kernel_ms']))
            share = stage_ms / event_ms if event_ms > 0 else 1.0
            kern_ms = ms * share
            alg = bytes_per_step(K, W['N'], nv, ebytes) * args.steps
            achieved = alg / (kern_ms / 1e3) / 1e9
            um = r['warps'] == 8
            traffic = recorded_traffic('mixed_um' if um else 'mixed')
            kname = ('um_stage_kernel<4> (tcgen05, 128-element CTA tiles; 4 launches per step)' if um
                     else 'tc_stage_kernel<4,*> (mma.sync, %d-warp CTAs; 4 launches per step)' % r['warps'])
            roof = {'bound': 'hbm', 'achieved': achieved, 'peak': hbm, 'unit': 'GB/s', 'frac': achieved / hbm,
                    'traffic': traffic, 'kernel': kname,
                    'algorithmic_bytes_per_launch_avg': bytes_per_step(K, W['N'], nv, ebytes) / 4,
                    'mean_launch_ms': kern_ms / (4 * args.steps),
                    'mean_launch_ms_event_pass': stage_ms / (4 * args.steps),
                    'kernel_time': 'graph-timed steps x the stage kernels\' share of the event-per-launch pass',
                    'peak_source': '%s hbm_gbs (MEASURED_PEAKS.json)' % peak_kind if peak_kind == 'measured'
                    else 'fallback 6400 GB/s',
                    'algorithmic_bytes_per_step': bytes_per_step(K, W['N'], nv, ebytes)}
        else:
            fl = flops_per_element_stage(W['N']) * K * 4 * args.steps
            achieved = fl / (stage_ms / 1e3) / 1e12
            peak = 148 * FP64_FLOP_PER_CLK_SM * sm_max * 1e6 / 1e12
            roof = {'bound': 'alu', 'achieved': achieved, 'peak': peak, 'unit': 'TFLOP/s', 'frac': achieved / peak,
                    'traffic': recorded_traffic('fp64'), 'kernel': 'stage_kernel<double,4,*> (4 launches per step)',
                    'mean_launch_ms': stage_ms / (4 * args.steps),
                    'peak_source': 'FP64 pipe: 148 SMs x 2 FMA/clk x 2 flop x %.0f MHz' % sm_max,
                    'algorithmic_flops_per_element_stage': flops_per_element_stage(W['N'])}
        out[name] = {'value': v, 'ms_per_step': ms / args.steps, 'roofline': roof,
                     'kernel_ms_per_step': [x / args.steps for x in r['kernel_ms']],
                     'stage_kernel_share': min(1.0, stage_ms / ms),
                     'timing': 'ms_per_step: gb_step (CUDA graph replay); kernel_ms_per_step: gb_step_timed',
                     'launch_shape': (('tcgen05 128-element CTA tiles (shape 8)' if r['warps'] == 8 else
                                       'mma.sync 16-element warp tiles, %d warps per CTA' % r['warps'])
                                      if name == 'mixed' else None)}
    qm, qf = results['mixed']['q_end'], results['fp64']['q_end']
    rest = np.zeros_like(qf)
    rest[:, 0, :] = 1.0
    err = {'rel_l2_fields': float(np.linalg.norm(qm - qf) / np.linalg.norm(qf)),
           'rel_l2_perturbation': float(np.linalg.norm(qm - qf) / np.linalg.norm(qf - rest)),
           'steps': args.warmup + args.steps, 'against': 'GB_FP64 path (oracle-parity-tested) from the same state'}
    if not args.no_long_error:
        err['run_1000'] = long_error(results, 1000)

    # end to end through the public API: pinned host state in, steps, pinned host state out
    s = results['mixed']['solver']
    q0 = results['mixed']['q0']
    pin_in = torch.empty(q0.shape, dtype=torch.float64, pin_memory=True).numpy()
    pin_in[...] = q0
    pin_out = torch.empty(q0.shape, dtype=torch.float64, pin_memory=True).numpy()
    barrier()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    s.set_fields(pin_in, 0.0)
    s.step(results['mixed']['dt'], args.steps)
    s.fields(out=pin_out)
    e2e_s = max_over_ranks(dist, time.perf_counter() - t0)
    nbytes = q0.nbytes
    e2e = {'value': aggregate_rate(ws, dof * 4 * args.steps, e2e_s), 'unit': 'DOF-stage updates/s',
           'h2d_bytes_per_step': nbytes / args.steps, 'd2h_bytes_per_step': nbytes / args.steps,
           'note': 'gb_set_fields (pinned host FP64 state) + gb_step x K + gb_fields (pinned host), wall clock'}

    if rank != 0:
        return
    line = {
        'metric': 'DOF-stage updates/s', 'value': out['mixed']['value'], 'unit': 'DOF-stage updates/s',
        'n_gpus': ws, 'steps': args.steps, 'warmup': args.warmup, 'ms_per_step': out['mixed']['ms_per_step'],
        'higher_is_better': True, 'scaling': 'weak', 'vs_baseline': None, 'dtype': 'f32',
        'data': 'synthetic: seeded jittered periodic mesh, Taylor-Green initial state, prescribed motion',
        'config': {'workload': WORKLOAD_NAME, 'K': K, 'N': W['N'], 'Np': Np, 'fields': 6, 'dof': dof,
                   'precision': 'GB_MIXED: FP32 perturbation fields, FP64 geometry and SARK coefficients',
                   'l2': 'inputs larger than L2: state arrays 5 x %.0f MB (FP32)' % (dof * 4 / 1e6),
                   'parallelism': 'replicas' if ws > 1 else 'single GPU'},
        'roofline': out['mixed']['roofline'],
        'e2e': e2e,
        'gpu_launches': 5 * args.steps,
        'launch_shape': out['mixed']['launch_shape'],   # the tuner's pick for this (N, size class)
        'clocks': clocks,
        'fp64': out['fp64'],
        'mixed': {k: v for k, v in out['mixed'].items() if k != 'roofline'},
        'mixed_speedup_vs_fp64': out['mixed']['value'] / out['fp64']['value'],
        'mixed_error': err,
    }
    if ws == 1 and not args.no_3d:
        line['d3'] = run_3d(torch)
        line['tgv3d'] = run_3d(torch, tgv=True)
    if ws == 1 and not args.no_airfoil:
        line['airfoil'] = run_airfoil(torch)
    if ws == 1 and not args.no_serve:
        line['serving'] = run_serving(torch, args.serve_requests, args.serve_steps)
    if ws == 1 and not args.no_cpu_baseline:
        line['cpu_baseline'] = cpu_baseline()
        line['cpu_baseline_all_cores'] = cpu_baseline_all_cores()
    print(json.dumps(line))


# ---------------------------------------------------------------------------
# reference arm: the oracle on the host cores
# ---------------------------------------------------------------------------
def run_reference(args):
    ws, rank, local = dist_env()
    if rank != 0:
        return
    from oracle import physics
    from oracle.solver import Motion, OracleSolver
    from paper_2607_00199_b300 import inputs
    W = WORKLOAD
    # bounded sample per step: a smaller jittered mesh of the same workload, sized so
    # that warmup + steps stays within a couple of minutes (~0.16 ms per element-step)
    budget_s = 120.0
    per_elem = 1.6e-4
    k_target = max(512, min(32768, budget_s / max(1, args.steps + args.warmup) / per_elem))
    n = max(16, int(math.sqrt(k_target / 2)))
    with _SingleThreadBLAS():
        mesh = inputs.periodic_square_mesh(n, jitter=W['jitter'])
        o = OracleSolver(mesh, W['N'], Ma=W['Ma'], Re=W['Re'], motion=Motion(W['A'], W['T']))
        xn = o.node_coords(o.X)
        rho, u, v = inputs.taylor_green(xn[..., 0], xn[..., 1], W['Ma'])
        q = np.ascontiguousarray(physics.equilibrium_state(rho, u, v, o.c).transpose(0, 2, 1))
        dt = inputs.cfl_dt(mesh, W['N'], o.c, W['cfl'])
        x, t = o.X.copy(), 0.0
        for _ in range(args.warmup):
            q, x = o.step(q, x, t, dt)
            t += dt
        c0, t0 = time.process_time(), time.perf_counter()
        for _ in range(args.steps):
            q, x = o.step(q, x, t, dt)
            t += dt
        el, cpu = time.perf_counter() - t0, time.process_time() - c0
    Np, _, _ = sizes(W['N'])
    dof = o.K * Np * 6
    v = dof * 4 * args.steps / el
    sample = ('each step: one SARK step of the same method on a %dx%d jittered mesh (K=%d, N=%d) '
              'instead of 256x256, numpy FP64' % (n, n, o.K, W['N']))
    line = {'impl': 'reference', 'metric': 'DOF-stage updates/s', 'value': v, 'unit': 'DOF-stage updates/s',
            'n_gpus': ws, 'steps': args.steps, 'warmup': args.warmup, 'ms_per_step': el / args.steps * 1e3,
            'higher_is_better': True, 'scaling': 'weak', 'vs_baseline': None, 'dtype': 'f64',
            'data': 'synthetic: seeded jittered periodic mesh, Taylor-Green initial state, prescribed motion',
            'config': {'workload': WORKLOAD_NAME, 'K': 131072, 'N': W['N'], 'sample_K': o.K},
            'cpu_baseline': {'value': v, 'unit': 'DOF-stage updates/s', 'cores': _cores_used(cpu, el), 'kind': 'oracle',
                             'sample': sample},
            'e2e': {'value': v, 'unit': 'DOF-stage updates/s', 'h2d_bytes_per_step': 0, 'd2h_bytes_per_step': 0}}
    print(json.dumps(line))


if __name__ == '__main__':
    a = parse()
    if a.serve_only:
        import torch
        print(json.dumps(run_serving(torch, a.serve_requests, a.serve_steps)))
    elif a.impl == 'reference':
        run_reference(a)
    else:
        run_ours(a)
