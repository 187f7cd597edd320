"""ALE right-hand side and SARK step on a moving periodic triangle mesh (oracle; test infrastructure only).

Follows the paper in order:
  Sec. 5   grid velocity: prescribed at the vertices, linear (P1) inside each
           element; vertices advanced with the same RK stages as the fields.
  Sec. 3   geometric factors G = [[x_r, x_s], [y_r, y_s]], J = det G, recomputed
           from the stage vertex positions at every stage (GCL, Sec. 5).
  Sec. 2-3 semi-discrete form
             dq/dt = (A + v_G) . D_x q + LIFT (F (q* - q^-)) + P Ntilde(I q),
           with F = A.n + v_G.n and the upwind fluxes of Sec. 3.
  Sec. 4   SARK stages with gamma = 0 for fields 1..3 and gamma = -dt/tau for
           fields 4..6.

Layout: q has shape (K, 6, Np) (element, field, node); node order as in
oracle.basis.  Vertex arrays have shape (n_vert, 2) over unique vertex ids;
element vertex coordinates are x[EToV] + shift (periodic unwrap offsets).

Readings (paper silent or ambiguous):
 * upwinding is physical: the residual flux is
   F_S (q* - q^-) = c/2 (|At_n| - At_n)(q^+ - q^-) and
   F_ALE (q* - q^-) = max(v_G.n, 0)(q^+ - q^-), upwinded separately as printed.
   (The literal "Lambda^+ acts on q^-" with Lambda the eigenvalues of A.n = -c At_n
   would be anti-upwind, because A carries the factor -c.)
 * the collision term J P N(I q) uses the reference projection: for an affine
   element the J of the paper's P^e = (M^e)^-1 I^T W cancels the J in front.
 * only the non-stiff Ntilde goes through the cubature; -Lambda q is integrated
   exactly by the exponentials (Sec. 4).
 * the grid motion of the free-stream test is evaluated at the Lagrangian
   (initial) vertex position X and displaces x and y by the same function.
 * stage i uses the vertex positions x_i of that stage and the vertex velocity
   v(X, t_n + c_i dt).

Pins (tests/test_oracle_solver.py): free-stream preservation on the deforming
mesh (Sec. 5 argument, Table 2 scale), N+1 convergence of an exact plane wave
with the collision term off, decay of the incompressible Taylor-Green vortex,
mass conservation on a static mesh.
"""
import math

import numpy as np

from . import physics
from .operators import REF_FACE_JAC, REF_NORMALS, ReferenceElement
from .sark import RK4_A, RK4_B, RK4_C, sark_coefficients

# d(lambda_v)/dr and d(lambda_v)/ds of the P1 barycentric map
_DLAM_DR = np.array([-0.5, 0.5, 0.0])
_DLAM_DS = np.array([-0.5, 0.0, 0.5])


class Motion:
    """Prescribed vertex displacement d(X, t) = A sin(2 pi t/T) S(X).  kind 'sinxy': S(X) =
    sin(2 pi X/Lx) sin(2 pi Y/Ly) for both x and y (free-stream test of Sec. 7.1); kind
    'plunge': S = (0, 1), the rigid plunge h(t) = A sin(2 pi t/T) of the airfoil case (Sec. 7).
    A = 0 is a static mesh."""

    def __init__(self, A=0.0, T=1.0, Lx=2.0 * math.pi, Ly=2.0 * math.pi, kind='sinxy'):
        self.A, self.T, self.Lx, self.Ly = float(A), float(T), float(Lx), float(Ly)
        self.kind = kind

    def shape(self, X):
        if self.kind == 'plunge':
            return np.stack([np.zeros(X.shape[0]), np.ones(X.shape[0])], axis=1)
        sxy = np.sin(2.0 * math.pi * X[:, 0] / self.Lx) * np.sin(2.0 * math.pi * X[:, 1] / self.Ly)
        return np.stack([sxy, sxy], axis=1)

    def velocity(self, X, t):
        w = 2.0 * math.pi / self.T
        return self.A * w * math.cos(w * t) * self.shape(X)

    def displacement(self, X, t):
        return self.A * math.sin(2.0 * math.pi * t / self.T) * self.shape(X)


class OracleSolver:
    """Plain FP64 ALE-DG Galerkin-Boltzmann solver on a periodic triangle mesh.

    mesh: dict with X (n_vert, 2), EToV (K, 3), shift (K, 3, 2), L (Lx, Ly).
    Either (Ma, Re) or (c, tau) is given; tau = inf switches the collision term
    off (a test-only knob that makes the system linear).
    """

    def __init__(self, mesh, N, Ma=None, Re=None, c=None, tau=None, motion=None, far_state=(1.0, 1.0, 0.0),
                 pml=None):
        self.ref = ReferenceElement(N)
        self.N = N
        if c is None:
            c, tau = physics.sound_speed_and_tau(Ma, Re)
        self.c = float(c)
        self.tau = float(tau)
        self.X = np.asarray(mesh['X'], dtype=np.float64)
        self.EToV = np.asarray(mesh['EToV'], dtype=np.int64)
        self.shift = np.asarray(mesh['shift'], dtype=np.float64)
        self.L = np.asarray(mesh['L'], dtype=np.float64)
        self.K = self.EToV.shape[0]
        self.motion = motion if motion is not None else Motion(0.0)
        # boundary faces (reading, see physics.wall_ghost): per face 0 interior or periodic,
        # 1 wall, 2 far field with the free-stream equilibrium of far_state = (rho, u, v)
        self.bc = np.asarray(mesh.get('bc', np.zeros((self.K, 3))), dtype=np.int64)
        self.q_far = physics.equilibrium_state(*far_state, self.c)
        self._connect()
        # perfectly matched layer (oracle.pml): sigma and direction at the Lagrangian nodes
        self.pml = pml
        if pml is not None:
            self.pml_sigma, self.pml_dir = pml.fields(self.node_coords(self.X))
            self.pml_layer = (self.pml_sigma > 0).any(axis=1)

    # ---- mesh -----------------------------------------------------------
    def element_vertices(self, xv):
        """Unwrapped vertex coordinates of every element, (K, 3, 2)."""
        return xv[self.EToV] + self.shift

    def node_coords(self, xv):
        """Physical node coordinates (K, Np, 2) from the P1 map of the vertices."""
        return np.einsum('nv,evd->end', self.ref.bary, self.element_vertices(xv))

    def _connect(self):
        """Face neighbours by shared vertex ids; node pairing by physical position
        modulo the periods (independent of any node-ordering convention)."""
        ref = self.ref
        K, Nfp = self.K, ref.Nfp
        faces = {}
        for e in range(K):
            for f in range(3):
                if self.bc[e, f]:
                    continue
                key = tuple(sorted((int(self.EToV[e, f]), int(self.EToV[e, (f + 1) % 3]))))
                faces.setdefault(key, []).append((e, f))
        self.nbr_elem = np.full((K, 3), -1, dtype=np.int64)
        self.nbr_face = np.zeros((K, 3), dtype=np.int64)
        for key, lst in faces.items():
            if len(lst) != 2:
                raise ValueError('face %s shared by %d elements (mesh must be closed/periodic)' % (key, len(lst)))
            (e1, f1), (e2, f2) = lst
            self.nbr_elem[e1, f1], self.nbr_face[e1, f1] = e2, f2
            self.nbr_elem[e2, f2], self.nbr_face[e2, f2] = e1, f1
        xn = self.node_coords(self.X)
        self.nbr_node = np.zeros((K, 3, Nfp), dtype=np.int64)
        per = np.where(self.L > 0, self.L, 1.0)
        scale = max(float(np.max(self.L)), float(np.ptp(self.X)))
        for e in range(K):
            for f in range(3):
                e2, f2 = self.nbr_elem[e, f], self.nbr_face[e, f]
                if e2 < 0:
                    self.nbr_node[e, f] = ref.fmask[f]   # unused: the exterior state comes from the boundary condition
                    continue
                mine = xn[e, ref.fmask[f]]              # (Nfp, 2)
                theirs = xn[e2, ref.fmask[f2]]
                d = mine[:, None, :] - theirs[None, :, :]
                d = d - np.where(self.L > 0, self.L * np.round(d / per), 0.0)
                dist = np.sqrt((d ** 2).sum(-1))
                k2 = np.argmin(dist, axis=1)
                if dist[np.arange(Nfp), k2].max() > 1e-8 * scale:
                    raise ValueError('face nodes of element %d face %d do not match' % (e, f))
                self.nbr_node[e, f] = ref.fmask[f2][k2]

    # ---- geometry (Sec. 3 and 5) ----------------------------------------
    def geometry(self, xv):
        """Per element: G^-1 = [[r_x, r_y], [s_x, s_y]] and J; per face: unit
        outward normal and Fscale = sJ / J, from Nanson's relation
        n ds = J G^-T nhat dshat."""
        P = self.element_vertices(xv)
        G = np.empty((self.K, 2, 2))
        G[:, 0, 0] = P[:, :, 0] @ _DLAM_DR
        G[:, 0, 1] = P[:, :, 0] @ _DLAM_DS
        G[:, 1, 0] = P[:, :, 1] @ _DLAM_DR
        G[:, 1, 1] = P[:, :, 1] @ _DLAM_DS
        J = np.linalg.det(G)
        Ginv = np.linalg.inv(G)
        GinvT = np.transpose(Ginv, (0, 2, 1))
        m = np.einsum('eij,fj->efi', GinvT, REF_NORMALS)       # (K, 3, 2)
        mlen = np.sqrt((m ** 2).sum(-1))
        normals = m / mlen[..., None]
        fscale = mlen * REF_FACE_JAC[None, :]
        return Ginv, J, normals, fscale

    # ---- right-hand side F = L(q) + Ntilde(q) (Secs. 3-4) -----------------
    def rhs(self, q, xv, vv, along_pml=False):
        """F(q) = volume + surface + P Ntilde(I q) at vertex positions xv and vertex
        velocities vv; the stiff -Lambda q part is not included (Sec. 4).  along_pml:
        also return R_e, the part of the advective terms along the layer direction e
        (oracle.pml)."""
        ref = self.ref
        K, Np, Nfp = self.K, ref.Np, ref.Nfp
        Ax, Ay = physics.flux_matrices(self.c)
        Ginv, J, normals, fscale = self.geometry(xv)
        rx, ry = Ginv[:, 0, 0], Ginv[:, 0, 1]
        sx, sy = Ginv[:, 1, 0], Ginv[:, 1, 1]
        # grid velocity at the nodes (P1 interpolation of vertex velocities)
        vg = np.einsum('nv,evd->end', ref.bary, vv[self.EToV])            # (K, Np, 2)
        # volume term: (A + v_G) . grad q
        qr = np.einsum('ij,efj->efi', ref.Dr, q)
        qs = np.einsum('ij,efj->efi', ref.Ds, q)
        qx = rx[:, None, None] * qr + sx[:, None, None] * qs
        qy = ry[:, None, None] * qr + sy[:, None, None] * qs
        F = (np.einsum('gf,efi->egi', Ax, qx) + np.einsum('gf,efi->egi', Ay, qy)
             + vg[:, None, :, 0] * qx + vg[:, None, :, 1] * qy)
        # surface term: LIFT of the upwind flux jump
        fm = np.concatenate(ref.fmask)                                      # (3 Nfp,)
        qM = q[:, :, fm].reshape(K, 6, 3, Nfp)
        qP = q[np.maximum(self.nbr_elem, 0)[:, :, None], :, self.nbr_node]  # (K, 3, Nfp, 6)
        vgf = vg[:, fm, :].reshape(K, 3, Nfp, 2)
        wall = self.bc == 1
        if wall.any():
            qm_w = np.transpose(qM, (0, 2, 3, 1))[wall]                      # (nw, Nfp, 6)
            qP[wall] = physics.wall_ghost(qm_w, vgf[wall][..., 0] / self.c, vgf[wall][..., 1] / self.c)
        far = self.bc == 2
        if far.any():
            qP[far] = self.q_far
        qP = np.transpose(qP, (0, 3, 1, 2))
        dq = qP - qM
        An = (normals[..., 0, None, None] * physics.ATX + normals[..., 1, None, None] * physics.ATY)
        absAn = physics.abs_normal_matrix(normals[..., 0], normals[..., 1])  # (K, 3, 6, 6)
        fluxS = 0.5 * self.c * np.einsum('efgh,ehfk->egfk', absAn - An, dq)
        vn = vgf[..., 0] * normals[:, :, None, 0] + vgf[..., 1] * normals[:, :, None, 1]
        fluxA = np.maximum(vn, 0.0)[:, None, :, :] * dq
        flux = (fscale[:, None, :, None] * (fluxS + fluxA)).reshape(K, 6, 3 * Nfp)
        F = F + np.einsum('im,egm->egi', ref.LIFT, flux)
        if along_pml:
            ex, ey = self.pml_dir[..., 0][:, None, :], self.pml_dir[..., 1][:, None, :]    # (K, 1, Np)
            qe = ex * qx + ey * qy                                                       # e . grad q
            vge = (vg[..., 0] * self.pml_dir[..., 0] + vg[..., 1] * self.pml_dir[..., 1])[:, None, :]
            R = (ex * np.einsum('gf,efi->egi', Ax, qe) + ey * np.einsum('gf,efi->egi', Ay, qe) + vge * qe)
            # face terms: the flux is 1/2 (A_n + v_n) dq (central) + 1/2 (c |At_n| + |v_n|) dq
            # (upwind dissipation); A_n + v_n = (n.e)(A_e + v_e) + (n.t)(A_t + v_t) gives the
            # central part along e exactly, the dissipation is shared with weights (n.e)^2
            ef = self.pml_dir[:, fm, :].reshape(K, 3, Nfp, 2)                            # e at the face nodes
            ne = np.einsum('efkd,efd->efk', ef, normals)                                 # n . e
            Ae = (ef[..., 0, None, None] * Ax + ef[..., 1, None, None] * Ay)              # (K, 3, Nfp, 6, 6)
            ve = (vgf * ef).sum(-1)                                                      # v_G . e
            cen = 0.5 * ne[:, None] * (np.einsum('efkgh,ehfk->egfk', Ae, dq) + ve[:, None] * dq)
            dis = 0.5 * (self.c * np.einsum('efgh,ehfk->egfk', absAn, dq) + np.abs(vn)[:, None] * dq)
            fe = (fscale[:, None, :, None] * (cen + (ne ** 2)[:, None] * dis)).reshape(K, 6, 3 * Nfp)
            R = R + np.einsum('im,egm->egi', ref.LIFT, fe)
        # collision term through the cubature: fields 4..6 get P Ntilde(I q)
        if np.isfinite(self.tau):
            qc = np.einsum('cj,efj->efc', ref.I, q[:, 0:3])
            n4, n5, n6 = physics.ntilde(qc[:, 0], qc[:, 1], qc[:, 2], self.tau)
            F[:, 3:6] += np.einsum('jc,efc->efj', ref.P, np.stack([n4, n5, n6], axis=1))
        return (F, R) if along_pml else F

    # ---- SARK step (Sec. 4) with RK4 vertex motion (Sec. 5) ----------------
    def field_coefficients(self, dt):
        """Per-field SARK coefficients: arrays E (5, 6), A (4, 4, 6), B (4, 6)."""
        gamma = 0.0 if not np.isfinite(self.tau) else -dt / self.tau
        E0, A0, B0 = sark_coefficients(0.0)
        E1, A1, B1 = sark_coefficients(gamma)
        cls = np.array([0, 0, 0, 1, 1, 1])
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
                qi = E[i + 1][None, :, None] * q + dt * sum(
                    A[i + 1, j][None, :, None] * Fs[j] for j in range(i + 1))
        qn = E[4][None, :, None] * q + dt * sum(B[j][None, :, None] * Fs[j] for j in range(4))
        xn = xv + dt * sum(RK4_B[j] * vs[j] for j in range(4))
        return qn, xn

    def run(self, q, xv, t, dt, nsteps):
        for _ in range(nsteps):
            q, xv = self.step(q, xv, t, dt)
            t = t + dt
        return q, xv, t

    def step_pml(self, q, phi, xv, t, dt):
        """One SARK step with the perfectly matched layer (oracle.pml): F_i gets -sigma Phi_i
        in every field, Phi advances by the RK4 stages with dPhi/dt = R_e - (alpha + sigma) Phi
        on the layer's elements (zero elsewhere).  Returns (q_{n+1}, Phi_{n+1}, x_{n+1})."""
        E, A, B = self.field_coefficients(dt)
        sig = self.pml_sigma[:, None, :]
        lay = self.pml_layer[:, None, None]
        Fs, Gs, vs = [], [], []
        qi, phii = q, phi
        for i in range(4):
            ti = t + RK4_C[i] * dt
            xi = xv + dt * sum(RK4_A[i][j] * vs[j] for j in range(i)) if i else xv
            vs.append(self.motion.velocity(self.X, ti))
            F, R = self.rhs(qi, xi, vs[i], along_pml=True)
            Fs.append(F - sig * phii)
            Gs.append(np.where(lay, R - (self.pml.alpha + sig) * phii, 0.0))
            if i < 3:
                qi = E[i + 1][None, :, None] * q + dt * sum(
                    A[i + 1, j][None, :, None] * Fs[j] for j in range(i + 1))
                phii = phi + dt * sum(RK4_A[i + 1][j] * Gs[j] for j in range(i + 1))
        qn = E[4][None, :, None] * q + dt * sum(B[j][None, :, None] * Fs[j] for j in range(4))
        phin = phi + dt * sum(RK4_B[j] * Gs[j] for j in range(4))
        xn = xv + dt * sum(RK4_B[j] * vs[j] for j in range(4))
        return qn, phin, xn

    def run_pml(self, q, phi, xv, t, dt, nsteps):
        for _ in range(nsteps):
            q, phi, xv = self.step_pml(q, phi, xv, t, dt)
            t = t + dt
        return q, phi, xv, t

    # ---- diagnostics ------------------------------------------------------
    def integral(self, f, xv):
        """int f over the mesh for nodal f of shape (K, Np): sum_e J_e 1^T Mhat f_e."""
        _, J, _, _ = self.geometry(xv)
        return float(np.einsum('e,ij,ej->', J, self.ref.M, f))

    def diagnostics(self, q, xv):
        """Integrals of the state (Sec. 7.2 kinetic energy, rho_inf = 1), each the
        exact integral of the nodal interpolant of its integrand:
        mass int rho, E_K = (1/|Omega|) int rho |u|^2 / 2, momentum int rho u,
        int rho v, and the area |Omega|.  q has shape (K, 6, Np)."""
        rho, mu, mv = physics.macroscopic(np.moveaxis(q, 1, -1), self.c)
        area = self.integral(np.ones_like(rho), xv)
        ke = self.integral(0.5 * (mu * mu + mv * mv) / rho, xv)
        return {'mass': self.integral(rho, xv), 'kinetic_energy': ke / area,
                'momentum_x': self.integral(mu, xv), 'momentum_y': self.integral(mv, xv), 'area': area}
