"""Pin: the oracle's right-hand side does not depend on how the mesh is numbered, wherever
the method itself does not.

Listing the elements in another order and each element's vertices in another
orientation-preserving order leaves the nodal basis (the node sets are symmetric), the face
pairing, the normals and the upwind fluxes unchanged at every physical node, so the volume
and surface terms must agree at the same physical node up to rounding.  The collision term
P Ntilde(I q) goes through the conical-product cubature, which is not symmetric under a
change of the collapsed vertex: it is exact, and hence independent of the numbering, only
while Ntilde is a polynomial of degree <= 3N.  So the cases here either switch collisions
off (general state) or hold q1 = 1, where Ntilde is quadratic in q2..q4 (degree 2N); a third
case shows that a general state with collisions does depend on the numbering, at the level
of the rule's error for a rational integrand.  The renumbered meshes make faces meet in every
pairing of local face numbers, which the generated meshes alone do not (a split quad grid
never joins two faces of the same local number), so a wrong face, node or normal index in
the connectivity fails here.
"""
import math

import numpy as np
import pytest

from oracle import physics, physics3d
from oracle.solver import Motion, OracleSolver
from oracle.solver3d import OracleSolver3D, WaveMotion
from paper_2607_00199_b300 import inputs

WAVE = dict(A0=0.02, A1=0.08, Lx=8.0, wavelength=1.0, omega=2 * math.pi, r0sq=0.25, yc=1.0, zc=1.0)


def _node_map(xa, xb):
    """m with xb[m[n]] == xa[n] (node coordinates of one element in two numberings)."""
    d = np.sqrt(((xa[:, None, :] - xb[None, :, :]) ** 2).sum(-1))
    m = np.argmin(d, axis=1)
    assert d[np.arange(len(m)), m].max() < 1e-12
    assert len(set(m.tolist())) == len(m)
    return m


def _compare(o_old, o_new, order, F_old, F_new, xv_old, xv_new):
    xo, xn = o_old.node_coords(xv_old), o_new.node_coords(xv_new)
    scale = np.abs(F_old).max()
    worst = 0.0
    for i in range(o_new.K):
        m = _node_map(xn[i], xo[order[i]])
        worst = max(worst, float(np.abs(F_new[i] - F_old[order[i]][:, m]).max()))
    assert worst <= 1e-12 * scale, worst / scale


def _face_pairs(o, nfaces):
    pairs = set()
    for e in range(o.K):
        for f in range(nfaces):
            if o.nbr_elem[e, f] >= 0:
                pairs.add((f, int(o.nbr_face[e, f])))
    return pairs


def _state2(o, xv, flow):
    xn = o.node_coords(xv)
    rho, u, v = flow(xn[..., 0], xn[..., 1])
    return np.ascontiguousarray(physics.equilibrium_state(rho, u, v, o.c).transpose(0, 2, 1))


def _pair2(mesh, new, N, motion, collide, **kw):
    tau = {} if collide else {'c': 10.0, 'tau': float('inf')}
    args = {'Ma': 0.1, 'Re': 100.0} if collide else {}
    return (OracleSolver(mesh, N, motion=motion, **args, **tau, **kw),
            OracleSolver(new, N, motion=motion, **args, **tau, **kw))


@pytest.mark.parametrize('case', ['collisions off', 'q1 = 1'])
@pytest.mark.parametrize('N', [1, 3])
def test_renumbered_periodic_mesh_gives_the_same_rhs(N, case):
    mesh = inputs.periodic_square_mesh(4, jitter=0.1)
    new, order = inputs.renumber_mesh(mesh, seed=5)
    assert not np.array_equal(order, np.arange(len(order)))
    motion = Motion(0.05, 1.0)
    o_old, o_new = _pair2(mesh, new, N, motion, case == 'q1 = 1')
    assert len(_face_pairs(o_old, 3)) == 6 and len(_face_pairs(o_new, 3)) == 9
    t = 0.3
    xv = o_old.X + motion.displacement(o_old.X, t)
    vv = motion.velocity(o_old.X, t)
    flow = lambda x, y: inputs.random_flow(x, y, 7)
    q_old, q_new = _state2(o_old, xv, flow), _state2(o_new, xv, flow)
    if case == 'q1 = 1':
        q_old[:, 0], q_new[:, 0] = 1.0, 1.0
    F_old = o_old.rhs(q_old, xv, vv)
    F_new = o_new.rhs(q_new, xv, vv)
    if case == 'q1 = 1':
        assert np.abs(F_old[:, 3:]).max() > 1e-2 * np.abs(F_old).max()    # the collision term is there
    _compare(o_old, o_new, order, F_old, F_new, xv, xv)


def test_collision_term_of_a_general_state_depends_on_the_collapsed_vertex():
    """Not a defect: the cubature's error for the rational Ntilde changes with the numbering,
    and shrinks as N grows (the rule is exact to degree 3N)."""
    mesh = inputs.periodic_square_mesh(4, jitter=0.1)
    new, order = inputs.renumber_mesh(mesh, seed=5)
    motion = Motion(0.05, 1.0)
    gaps = []
    for N in (2, 4):
        o_old, o_new = _pair2(mesh, new, N, motion, True)
        flow = lambda x, y: (1.0 + 0.3 * np.sin(x) * np.cos(y), 0.1 * np.cos(x), 0.1 * np.sin(y))
        F_old = o_old.rhs(_state2(o_old, o_old.X, flow), o_old.X, 0 * o_old.X)
        F_new = o_new.rhs(_state2(o_new, o_old.X, flow), o_old.X, 0 * o_old.X)
        xo, xn = o_old.node_coords(o_old.X), o_new.node_coords(o_old.X)
        gap = max(float(np.abs(F_new[i] - F_old[order[i]][:, _node_map(xn[i], xo[order[i]])]).max())
                  for i in range(o_new.K))
        gaps.append(gap / np.abs(F_old).max())
    assert gaps[0] > 1e-9 and gaps[1] < gaps[0] / 10, gaps


def test_renumbered_bounded_mesh_gives_the_same_rhs():
    """Walls and far field on a plunging channel: the boundary tags follow their faces."""
    mesh = inputs.wall_channel_mesh(4, 3, 2.0, 1.5)
    mesh['bc'] = mesh['bc'].copy()
    mesh['bc'][1::2][mesh['bc'][1::2] > 0] = inputs.BC_FARFIELD     # far field at x = 0, wall at x = Lx
    new, order = inputs.renumber_mesh(mesh, seed=9)
    motion = Motion(0.1, 2.0, kind='plunge')
    far = (1.0, 0.5, 0.1)
    o_old, o_new = _pair2(mesh, new, 3, motion, True, far_state=far)
    assert (o_new.bc == inputs.BC_WALL).sum() == (o_old.bc == inputs.BC_WALL).sum() > 0
    assert (o_new.bc == inputs.BC_FARFIELD).sum() == (o_old.bc == inputs.BC_FARFIELD).sum() > 0
    t = 0.4
    xv = o_old.X + motion.displacement(o_old.X, t)
    vv = motion.velocity(o_old.X, t)
    flow = lambda x, y: (1.0 + 0.02 * np.sin(x + 2 * y), 0.5 + 0.1 * np.cos(y), 0.1 + 0.05 * np.sin(x))
    q_old, q_new = _state2(o_old, xv, flow), _state2(o_new, xv, flow)
    q_old[:, 0], q_new[:, 0] = 1.0, 1.0             # Ntilde polynomial: the cubature is exact
    F_old = o_old.rhs(q_old, xv, vv)
    F_new = o_new.rhs(q_new, xv, vv)
    _compare(o_old, o_new, order, F_old, F_new, xv, xv)


def test_renumbered_tetrahedral_mesh_gives_the_same_rhs():
    mesh = inputs.periodic_box_tet_mesh(3, 3, 3, jitter=0.1)
    new, order = inputs.renumber_mesh(mesh, seed=3)
    motion = WaveMotion(**WAVE)
    o_old = OracleSolver3D(mesh, 2, Ma=0.1, Re=500.0, motion=motion)
    o_new = OracleSolver3D(new, 2, Ma=0.1, Re=500.0, motion=motion)     # q1 = 1 below: exact cubature
    assert len(_face_pairs(o_new, 4)) == 16 > len(_face_pairs(o_old, 4))
    t = 0.3
    xv = o_old.X + motion.displacement(o_old.X, t)
    vv = motion.velocity(o_old.X, t)

    def state(o):
        xn = o.node_coords(xv)
        rho, u, v, w = inputs.random_flow_3d(xn[..., 0], xn[..., 1], xn[..., 2], 13)
        q = np.ascontiguousarray(physics3d.equilibrium_state(rho, u, v, w, o.c).transpose(0, 2, 1))
        q[:, 0] = 1.0
        return q

    F_old = o_old.rhs(state(o_old), xv, vv)
    F_new = o_new.rhs(state(o_new), xv, vv)
    _compare(o_old, o_new, order, F_old, F_new, xv, xv)
