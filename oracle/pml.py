"""Perfectly matched layer (PML) of the airfoil case's outer boundary (oracle; test
infrastructure only).

The paper runs the plunging airfoil with a PML carrying auxiliary fields but prints no PML
equations.  Reading used here: complex stretching of one direction e(x) (the radial
direction of the O-grid's outer layer; a fixed direction for a slab), in the planar
approximation (the stretching of the tangential 1/r factor is neglected), with a
frequency shift alpha (the complex-frequency-shifted form):

    d/de  ->  d/de (s + alpha) / (s + alpha + sigma),   s the Laplace variable.

Split the advective operator of the semi-discrete form, L(q) = volume + surface terms, into
its part along e and the rest, L = R_e + R_t.  Since (s + alpha)/(s + alpha + sigma) =
1 - sigma/(s + alpha + sigma), the stretched system is, with Phi the auxiliary fields
(6 per node, zero outside the layer):

    dq/dt   = L(q) + Ntilde(q) - sigma Phi          (fields 4..6 keep their exact -q/tau)
    dPhi/dt = R_e(q) - (alpha + sigma) Phi

R_e in the DG form:
  volume   (A_e + (v_G . e)) d_e q,  A_e = e_x A_x + e_y A_y,  d_e q = e . grad q,
           e taken at each node;
  surface  the upwind flux of L is 1/2 (A_n + v_n) dq + 1/2 (c |At_n| + |v_n|) dq with
           A_n + v_n = (n.e)(A_e + v_e) + (n.t)(A_t + v_t): the central part along e is
           1/2 (n.e)(A_e + v_e) dq (the DG derivative along e with a central trace), the
           upwind dissipation is shared with weights (n.e)^2 and (n.t)^2 (t the tangential
           direction); both pieces sum with the t-part to L exactly.
Phi is advanced by the same RK4 stages as the grid (gamma = 0), the -sigma Phi term joins
the non-stiff F of every field in the SARK stages.

Profiles (sigma(r) = sigma_max ((r - r0)/d)^p for r > r0, zero inside; r and e from the
Lagrangian node position X): 'radial' r = |X - centre|, e = (X - centre)/r (the O-grid's
outer ring); 'slab' r = |(X - centre) . e0|, e = sign((X - centre) . e0) e0 (two layers
facing away from the centre line); 'uniform' sigma = sigma_max and e = e0 everywhere (a
test configuration: the whole mesh is the layer).  Elements with a node where sigma > 0
form the layer.

Pins (tests/test_oracle_pml.py): on a periodic mesh with a uniform layer along x, the DG
solution converges to the exact solution of the stretched system for a Fourier mode
(matrix exponential of the 12 x 12 mode system), q at rate N+1 and Phi (the time integral
of a DG directional derivative) at rate N; the split R_e + R_t = L is exact; sigma = 0
leaves q bit for bit as without the layer; a uniform stream is steady with the layer;
slab layers cut the reflection error of far-field ends against a wider domain.
"""
import math

import numpy as np


class PML:
    """sigma and direction fields of a layer, evaluated at Lagrangian node positions."""

    def __init__(self, kind='radial', centre=(0.5, 0.0), r0=17.0, d=3.0, sigma_max=1.0, power=2.0,
                 alpha=0.0, direction=(1.0, 0.0)):
        if kind not in ('radial', 'slab', 'uniform'):
            raise ValueError('kind must be radial, slab or uniform')
        self.kind = kind
        self.centre = np.asarray(centre, dtype=np.float64)
        self.r0, self.d = float(r0), float(d)
        self.sigma_max, self.power, self.alpha = float(sigma_max), float(power), float(alpha)
        e = np.asarray(direction, dtype=np.float64)
        self.direction = e / np.sqrt((e * e).sum())

    def fields(self, Xn):
        """sigma (...,) and unit direction e (..., 2) at positions Xn (..., 2)."""
        if self.kind == 'uniform':
            sigma = np.full(Xn.shape[:-1], self.sigma_max)
            e = np.broadcast_to(self.direction, Xn.shape).copy()
            return sigma, e
        rel = Xn - self.centre
        if self.kind == 'radial':
            r = np.sqrt((rel * rel).sum(-1))
            e = rel / np.where(r > 0, r, 1.0)[..., None]
        else:
            s = rel @ self.direction
            r = np.abs(s)
            e = np.where(s < 0, -1.0, 1.0)[..., None] * self.direction
        depth = np.clip((r - self.r0) / self.d, 0.0, None)
        sigma = self.sigma_max * depth ** self.power
        return sigma, e


def sigma_max_for_reflection(c, d, power=2.0, reflection=1e-6):
    """sigma_max giving the continuous layer of depth d the round-trip reflection
    `reflection` for normal incidence at the fastest speed sqrt(3) c of the 2D moment
    system: exp(-2 int_0^d sigma / lambda) = R with sigma = sigma_max (x/d)^p."""
    lam = math.sqrt(3.0) * c
    return (power + 1.0) * lam * math.log(1.0 / reflection) / (2.0 * d)
