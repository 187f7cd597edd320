"""ALE right-hand side and SARK step on a moving periodic tetrahedral mesh, 10 fields
(oracle; test infrastructure only).

The 3D form of oracle.solver, step for step (paper Secs. 2-5; the paper runs the same
scheme on tetrahedra):
  Sec. 5   grid velocity prescribed at the vertices, linear (P1) in each element;
           vertices advanced with the same RK stages as the fields.
  Sec. 3   G = dx/d(r,s,t), J = det G, recomputed from the stage vertex positions at
           every stage (GCL); normals and Fscale from Nanson's relation.
  Sec. 2-3 dq/dt = (A + v_G) . D_x q + LIFT (F (q* - q^-)) + P Ntilde(I q), with the
           upwind fluxes F_S (q* - q^-) = c/2 (|At_n| - At_n)(q^+ - q^-) and
           F_ALE (q* - q^-) = max(v_G . n, 0)(q^+ - q^-) (the 2D readings).
  Sec. 4   SARK stages, gamma = 0 for fields 1..4 and -dt/tau for fields 5..10.

Layout: q has shape (K, 10, Np).  Vertex arrays (n_vert, 3); element vertex k of
element e is at x[EToV[e, k]] + shift[e, k].

Motions: TGVMotion3D, the deformation of the moving 3D Taylor-Green vortex (Sec. 7.2),
and WaveMotion, the deforming-channel workload: the vertex with Lagrangian position X moves in
y by d(X, t) = A(X) sin(2 pi X/lambda - omega t) exp(-r^2/r0sq), A(X) = A0 + A1 X/Lx,
r^2 = (Y - yc)^2 + (Z - zc)^2; its velocity is the time derivative of d at the same X
(Sec. 5: velocity of the Lagrangian point).

Pins (tests/test_oracle_solver3d.py): free-stream preservation on the deforming mesh,
N+1 convergence of an exact plane wave with the collision term off (static and moving
meshes), mass conservation on a static mesh, shear-wave decay at the rate nu k^2
(nu = tau RT), connectivity an involution.
"""
import math

import numpy as np

from . import physics3d
from .sark import RK4_A, RK4_B, RK4_C, sark_coefficients
from .tet import FACE_VERTS, REF_FACE_JAC, REF_NORMALS, ReferenceTet


class WaveMotion:
    """Traveling-wave lateral displacement of the deforming channel (module doc); A0 = A1 = 0 is static."""

    def __init__(self, A0=0.0, A1=0.0, Lx=8.0, wavelength=1.0, omega=2.0 * math.pi, r0sq=0.25, yc=1.0, zc=1.0):
        self.A0, self.A1, self.Lx = float(A0), float(A1), float(Lx)
        self.k = 2.0 * math.pi / float(wavelength)
        self.omega, self.r0sq, self.yc, self.zc = float(omega), float(r0sq), float(yc), float(zc)

    def _amp(self, X):
        r2 = (X[:, 1] - self.yc) ** 2 + (X[:, 2] - self.zc) ** 2
        return (self.A0 + self.A1 * X[:, 0] / self.Lx) * np.exp(-r2 / self.r0sq)

    def displacement(self, X, t):
        d = np.zeros_like(X)
        d[:, 1] = self._amp(X) * np.sin(self.k * X[:, 0] - self.omega * t)
        return d

    def velocity(self, X, t):
        v = np.zeros_like(X)
        v[:, 1] = -self.omega * self._amp(X) * np.cos(self.k * X[:, 0] - self.omega * t)
        return v


class TGVMotion3D:
    """Deformation of the moving 3D Taylor-Green vortex (Sec. 7.2, Eq. TGV_deformation): each
    coordinate of the vertex with Lagrangian position X moves by
    A sin(2 pi t / T) S(a) S(b), (a, b) the other two Lagrangian coordinates,
    S(s) = sin(2 pi (s + L/2) / L); L = 2 pi, A = pi / 6, T = 20 in the paper."""

    def __init__(self, A=math.pi / 6.0, T=20.0, L=2.0 * math.pi):
        self.A, self.T, self.L = float(A), float(T), float(L)

    def _shape(self, X):
        S = np.sin(2.0 * math.pi * (X + 0.5 * self.L) / self.L)
        return np.stack([S[:, 1] * S[:, 2], S[:, 0] * S[:, 2], S[:, 0] * S[:, 1]], axis=1)

    def displacement(self, X, t):
        return self.A * math.sin(2.0 * math.pi * t / self.T) * self._shape(X)

    def velocity(self, X, t):
        w = 2.0 * math.pi / self.T
        return self.A * w * math.cos(w * t) * self._shape(X)


class OracleSolver3D:
    """Plain FP64 ALE-DG Galerkin-Boltzmann solver on a periodic tetrahedral mesh.

    mesh: dict with X (n_vert, 3), EToV (K, 4), shift (K, 4, 3), L (3,).  (Ma, Re) or
    (c, tau); tau = inf switches the collision term off (test-only knob).
    """

    def __init__(self, mesh, N, Ma=None, Re=None, c=None, tau=None, motion=None):
        self.ref = ReferenceTet(N)
        self.N = N
        if c is None:
            c, tau = 1.0 / Ma, Ma * Ma / Re
        self.c = float(c)
        self.tau = float(tau)
        self.X = np.asarray(mesh['X'], dtype=np.float64)
        self.EToV = np.asarray(mesh['EToV'], dtype=np.int64)
        self.shift = np.asarray(mesh['shift'], dtype=np.float64)
        self.L = np.asarray(mesh['L'], dtype=np.float64)
        self.K = self.EToV.shape[0]
        self.motion = motion if motion is not None else WaveMotion()
        self._connect()

    def element_vertices(self, xv):
        return xv[self.EToV] + self.shift

    def node_coords(self, xv):
        return np.einsum('nv,evd->end', self.ref.bary, self.element_vertices(xv))

    def _connect(self):
        """Face neighbours by shared vertex-id triples; node pairing by physical
        position modulo the periods."""
        ref = self.ref
        K, Nfp = self.K, ref.Nfp
        faces = {}
        for e in range(K):
            for f, fv in enumerate(FACE_VERTS):
                key = tuple(sorted(int(self.EToV[e, v]) for v in fv))
                faces.setdefault(key, []).append((e, f))
        self.nbr_elem = np.zeros((K, 4), dtype=np.int64)
        self.nbr_face = np.zeros((K, 4), dtype=np.int64)
        for key, lst in faces.items():
            if len(lst) != 2:
                raise ValueError('face %s shared by %d elements' % (key, len(lst)))
            (e1, f1), (e2, f2) = lst
            self.nbr_elem[e1, f1], self.nbr_face[e1, f1] = e2, f2
            self.nbr_elem[e2, f2], self.nbr_face[e2, f2] = e1, f1
        xn = self.node_coords(self.X)
        self.nbr_node = np.zeros((K, 4, Nfp), dtype=np.int64)
        for e in range(K):
            for f in range(4):
                e2, f2 = self.nbr_elem[e, f], self.nbr_face[e, f]
                mine = xn[e, ref.fmask[f]]
                theirs = xn[e2, ref.fmask[f2]]
                d = mine[:, None, :] - theirs[None, :, :]
                d = d - self.L * np.round(d / self.L)
                dist = np.sqrt((d ** 2).sum(-1))
                k2 = np.argmin(dist, axis=1)
                if dist[np.arange(Nfp), k2].max() > 1e-8 * max(self.L):
                    raise ValueError('face nodes of element %d face %d do not match' % (e, f))
                self.nbr_node[e, f] = ref.fmask[f2][k2]

    def geometry(self, xv):
        """G^-1 (rows r_x.., s_x.., t_x..), J, unit outward normals (K, 4, 3), Fscale (K, 4)."""
        P = self.element_vertices(xv)
        G = np.stack([(P[:, 1] - P[:, 0]) / 2.0, (P[:, 2] - P[:, 0]) / 2.0, (P[:, 3] - P[:, 0]) / 2.0], axis=2)
        J = np.linalg.det(G)
        Ginv = np.linalg.inv(G)
        m = np.einsum('eji,fj->efi', Ginv, REF_NORMALS)          # G^-T n_hat
        mlen = np.sqrt((m ** 2).sum(-1))
        return Ginv, J, m / mlen[..., None], mlen * REF_FACE_JAC[None, :]

    def rhs(self, q, xv, vv):
        """F(q) = volume + surface + P Ntilde(I q) at vertex positions xv, velocities vv."""
        ref = self.ref
        K, Np, Nfp = self.K, ref.Np, ref.Nfp
        Ginv, J, normals, fscale = self.geometry(xv)
        vg = np.einsum('nv,evd->end', ref.bary, vv[self.EToV])          # (K, Np, 3)
        qd = [np.einsum('ij,efj->efi', D, q) for D in (ref.Dr, ref.Ds, ref.Dt)]
        grad = [sum(Ginv[:, a, d][:, None, None] * qd[a] for a in range(3)) for d in range(3)]
        F = np.zeros_like(q)
        for d, At in enumerate((physics3d.ATX, physics3d.ATY, physics3d.ATZ)):
            F += -self.c * np.einsum('gf,efi->egi', At, grad[d]) + vg[:, None, :, d] * grad[d]
        fm = np.concatenate(ref.fmask)
        qM = q[:, :, fm].reshape(K, 10, 4, Nfp)
        qP = np.transpose(q[self.nbr_elem[:, :, None], :, self.nbr_node], (0, 3, 1, 2))
        dq = qP - qM
        An = np.einsum('efd,dgh->efgh', normals, np.stack([physics3d.ATX, physics3d.ATY, physics3d.ATZ]))
        absAn = physics3d.abs_normal_matrix(normals)
        fluxS = 0.5 * self.c * np.einsum('efgh,ehfk->egfk', absAn - An, dq)
        vgf = vg[:, fm, :].reshape(K, 4, Nfp, 3)
        vn = np.einsum('efkd,efd->efk', vgf, normals)
        fluxA = np.maximum(vn, 0.0)[:, None, :, :] * dq
        flux = (fscale[:, None, :, None] * (fluxS + fluxA)).reshape(K, 10, 4 * Nfp)
        F = F + np.einsum('im,egm->egi', ref.LIFT, flux)
        if np.isfinite(self.tau):
            qc = np.einsum('cj,efj->efc', ref.I, q[:, 0:4])
            nt = physics3d.ntilde(qc[:, 0], qc[:, 1], qc[:, 2], qc[:, 3], self.tau)
            F[:, 4:10] += np.einsum('jc,efc->efj', ref.P, np.stack(nt, axis=1))
        return F

    def field_coefficients(self, dt):
        gamma = 0.0 if not np.isfinite(self.tau) else -dt / self.tau
        E0, A0, B0 = sark_coefficients(0.0)
        E1, A1, B1 = sark_coefficients(gamma)
        cls = np.array([0] * 4 + [1] * 6)
        E = np.array([E0, E1])[cls].T
        A = np.transpose(np.array([A0, A1])[cls], (1, 2, 0))
        B = np.array([B0, B1])[cls].T
        return E, A, B

    def step(self, q, xv, t, dt):
        """One SARK step from (q_n, x_n, t_n); returns (q_{n+1}, x_{n+1})."""
        E, A, B = self.field_coefficients(dt)
        Fs, vs = [], []
        qi = q
        for i in range(4):
            ti = t + RK4_C[i] * dt
            xi = xv + dt * sum(RK4_A[i][j] * vs[j] for j in range(i)) if i else xv
            vs.append(self.motion.velocity(self.X, ti))
            Fs.append(self.rhs(qi, xi, vs[i]))
            if i < 3:
                qi = E[i + 1][None, :, None] * q + dt * sum(A[i + 1, j][None, :, None] * Fs[j] for j in range(i + 1))
        qn = E[4][None, :, None] * q + dt * sum(B[j][None, :, None] * Fs[j] for j in range(4))
        xn = xv + dt * sum(RK4_B[j] * vs[j] for j in range(4))
        return qn, xn

    def run(self, q, xv, t, dt, nsteps):
        for _ in range(nsteps):
            q, xv = self.step(q, xv, t, dt)
            t = t + dt
        return q, xv, t

    def integral(self, f, xv):
        """int f over the mesh for nodal f (K, Np): sum_e J_e 1^T Mhat f_e."""
        _, J, _, _ = self.geometry(xv)
        return float(np.einsum('e,ij,ej->', J, self.ref.M, f))

    def diagnostics(self, q, xv):
        """Integrals of the state (Sec. 7.2 kinetic energy with rho_inf = 1), each the exact
        integral of the nodal interpolant of its integrand: mass int rho,
        E_K = (1/|Omega|) int rho |u|^2 / 2, momentum int rho u, int rho v, int rho w and
        the volume |Omega|.  q has shape (K, 10, Np)."""
        rho, mu, mv, mw = physics3d.macroscopic(np.moveaxis(q, 1, -1), self.c)
        vol = self.integral(np.ones_like(rho), xv)
        ke = self.integral(0.5 * (mu * mu + mv * mv + mw * mw) / rho, xv)
        return {'mass': self.integral(rho, xv), 'kinetic_energy': ke / vol, 'momentum_x': self.integral(mu, xv),
                'momentum_y': self.integral(mv, xv), 'momentum_z': self.integral(mw, xv), 'volume': vol}
