"""Seeded synthetic inputs: meshes, motion parameters, initial flows, request streams.

This module holds none of the method's arithmetic.  It is the one piece shared
by the CUDA library's tests and benchmark and by the CPU oracle's tests: it
only generates the inputs both sides receive.

Random numbers come from splitmix64 (Steele, Lea and Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014) used as a counter-based
generator: draw k of stream `seed` is mix(seed + (k + 1) * 0x9E3779B97F4A7C15).
"""
import math

import numpy as np

GOLDEN = np.uint64(0x9E3779B97F4A7C15)
DEFAULT_SEED = 260700199


def splitmix64(counter, seed=DEFAULT_SEED):
    """splitmix64 output for integer counters (array), as uint64."""
    with np.errstate(over='ignore'):
        z = np.uint64(seed) + (np.asarray(counter, dtype=np.uint64) + np.uint64(1)) * GOLDEN
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
        z = z ^ (z >> np.uint64(31))
    return z


def uniform(counter, seed=DEFAULT_SEED, lo=0.0, hi=1.0):
    """Uniform doubles in [lo, hi) from the top 53 bits of splitmix64."""
    u = (splitmix64(counter, seed) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)
    return lo + (hi - lo) * u


def periodic_square_mesh(n, L=2.0 * math.pi, jitter=0.0, seed=DEFAULT_SEED):
    """Periodic [0, L]^2 with n x n square cells, each split along its (0,0)-(1,1)
    diagonal into two counter-clockwise triangles; K = 2 n^2.

    Unique vertices are the n^2 grid points (periodic images share an id).
    jitter > 0 moves every unique vertex by independent U[-jitter h, jitter h]
    offsets in x and y (h = L/n), drawn with splitmix64 (x: counter 2 id,
    y: counter 2 id + 1).

    Returns a dict: X (n^2, 2) float64 vertex coordinates, EToV (K, 3) int32,
    shift (K, 3, 2) float64 periodic unwrap offsets (element vertex k of
    element e sits at X[EToV[e, k]] + shift[e, k]), L (2,) periods, n.
    """
    if n < 3:
        raise ValueError('n >= 3 is needed so that every face has a unique vertex pair')
    h = L / n
    ii, jj = np.meshgrid(np.arange(n), np.arange(n), indexing='ij')
    X = np.zeros((n * n, 2))
    vid = (ii + n * jj).ravel()
    X[vid, 0] = (ii * h).ravel()
    X[vid, 1] = (jj * h).ravel()
    if jitter > 0.0:
        ids = np.arange(n * n, dtype=np.uint64)
        X[:, 0] += uniform(2 * ids, seed, -jitter * h, jitter * h)
        X[:, 1] += uniform(2 * ids + 1, seed, -jitter * h, jitter * h)
    # cells in row-major order (j outer, i inner), two triangles per cell
    j, i = np.meshgrid(np.arange(n), np.arange(n), indexing='ij')
    i = i.ravel()
    j = j.ravel()
    corners = np.array([[(0, 0), (1, 0), (1, 1)], [(0, 0), (1, 1), (0, 1)]])
    a = i[:, None, None] + corners[None, :, :, 0]
    b = j[:, None, None] + corners[None, :, :, 1]
    EToV = ((a % n) + n * (b % n)).reshape(-1, 3).astype(np.int32)
    shift = np.stack([(a // n) * L, (b // n) * L], axis=-1).reshape(-1, 3, 2).astype(np.float64)
    return {'X': X, 'EToV': EToV, 'shift': shift, 'L': np.array([L, L]), 'n': n}


def min_altitude(mesh):
    """Smallest triangle altitude of the mesh at its Lagrangian positions."""
    P = mesh['X'][mesh['EToV']] + mesh['shift']
    e = [P[:, (k + 1) % 3] - P[:, k] for k in range(3)]
    area2 = np.abs(e[0][:, 0] * e[1][:, 1] - e[0][:, 1] * e[1][:, 0])
    longest = np.max(np.stack([np.hypot(v[:, 0], v[:, 1]) for v in e]), axis=0)
    return float(np.min(area2 / longest))


def cfl_dt(mesh, N, c, cfl):
    """Run parameter: dt = cfl * h_min / (sqrt(3) c (N+1)^2), with sqrt(3) c the
    largest characteristic speed and h_min the smallest altitude.  The paper does
    not define its time step; this helper fixes one, passed to both sides."""
    return cfl * min_altitude(mesh) / (math.sqrt(3.0) * c * (N + 1) ** 2)


def taylor_green(x, y, Ma):
    """Incompressible 2D Taylor-Green vortex: u = sin x cos y, v = -cos x sin y,
    rho = 1 + Ma^2/4 (cos 2x + cos 2y).  Returns (rho, u, v)."""
    u = np.sin(x) * np.cos(y)
    v = -np.cos(x) * np.sin(y)
    rho = 1.0 + Ma * Ma * 0.25 * (np.cos(2.0 * x) + np.cos(2.0 * y))
    return rho, u, v


def free_stream(x, y, u0=1.0, v0=0.0):
    """Uniform flow rho = 1, (u, v) = (u0, v0)."""
    return np.ones_like(x), np.full_like(x, u0), np.full_like(x, v0)


def random_flow(x, y, seed, amp=0.05):
    """Smooth seeded periodic perturbation of the rest state (for parity tests)."""
    k = uniform(np.arange(12), seed)
    rho = 1.0 + amp * (np.sin(x + 6.0 * k[0]) * np.cos(y + 6.0 * k[1]) + 0.5 * np.sin(2 * x + 6.0 * k[2]))
    u = 0.5 * np.sin(y + 6.0 * k[3]) + 0.3 * np.cos(x + 2 * y + 6.0 * k[4])
    v = 0.5 * np.cos(x + 6.0 * k[5]) - 0.3 * np.sin(2 * x - y + 6.0 * k[6])
    return rho, u, v


def serving_requests(n=256, rate=50.0, seed=1):
    """Request stream: Poisson arrivals (mean `rate`/s) with K in
    {2048, 8192, 32768, 131072} (as n x n x 2 meshes), N in {2, 3, 4, 5},
    motion amplitude U[0.01, 0.08], period U[0.5, 2], Re U[100, 2000], Ma = 0.1."""
    ids = np.arange(n, dtype=np.uint64)
    u = [uniform(8 * ids + k, seed) for k in range(6)]
    gaps = -np.log1p(-u[0]) / rate
    arrival = np.cumsum(gaps)
    Ks = np.array([2048, 8192, 32768, 131072])
    Ns = np.array([2, 3, 4, 5])
    out = []
    for r in range(n):
        K = int(Ks[min(int(u[1][r] * 4), 3)])
        out.append({'id': r, 'arrival': float(arrival[r]), 'K': K, 'n': int(round(math.sqrt(K / 2))),
                    'N': int(Ns[min(int(u[2][r] * 4), 3)]),
                    'A': 0.01 + 0.07 * float(u[3][r]), 'T': 0.5 + 1.5 * float(u[4][r]),
                    'Re': 100.0 + 1900.0 * float(u[5][r]), 'Ma': 0.1})
    return out


# ---- three dimensions: periodic box of tetrahedra ------------------------------------

# Kuhn (Freudenthal) subdivision of the unit cube: one tetrahedron per ordering of the
# three axes, walking from corner (0,0,0) to (1,1,1) along unit steps.  The same split
# in every cell makes the faces of neighbouring cells (and of periodic copies) match.
_KUHN_ORDERS = ((0, 1, 2), (0, 2, 1), (1, 0, 2), (1, 2, 0), (2, 0, 1), (2, 1, 0))


def _even_permutations(n):
    """The orientation-preserving vertex orders of a simplex with n vertices."""
    import itertools
    out = []
    for p in itertools.permutations(range(n)):
        inversions = sum(1 for a in range(n) for b in range(a + 1, n) if p[a] > p[b])
        if inversions % 2 == 0:
            out.append(p)
    return np.array(out, dtype=np.int64)


def renumber_mesh(mesh, seed=DEFAULT_SEED):
    """The same mesh with its elements listed in a seeded random order and each element's
    vertices in a seeded random orientation-preserving order (a cyclic rotation of a
    triangle, an even permutation of a tetrahedron).  The geometry is unchanged; the
    numbering of elements, of their faces and of their nodes is not, so that faces meet in
    every pairing of local face numbers.  Returns (new mesh, order): element i of the new
    mesh is element order[i] of the old one.  Per-face boundary tags (2D 'bc', face f
    running from vertex f to f + 1) follow their faces.
    Draws: splitmix64 stream `seed`, counters 2 e (order key) and 2 e + 1 (vertex order)."""
    EToV = np.asarray(mesh['EToV'])
    K, nv = EToV.shape
    e = np.arange(K, dtype=np.uint64)
    order = np.argsort(splitmix64(2 * e, seed), kind='stable')
    perms = np.array([[(j + r) % 3 for j in range(3)] for r in range(3)]) if nv == 3 else _even_permutations(4)
    choice = (splitmix64(2 * e + np.uint64(1), seed) % np.uint64(len(perms))).astype(np.int64)[order]
    p = perms[choice]                                                       # (K, nv): new slot -> old slot
    rows = np.arange(K)[:, None]
    out = dict(mesh)
    out['EToV'] = EToV[order][rows, p].astype(EToV.dtype)
    out['shift'] = np.asarray(mesh['shift'])[order][rows, p]
    if 'bc' in mesh:
        if nv != 3:
            raise ValueError('boundary tags are defined for triangles only')
        # new face f joins new vertices f, f + 1 = old vertices r + f, r + f + 1: old face (f + r) mod 3
        out['bc'] = np.asarray(mesh['bc'])[order][rows, p]
    return out, order


def periodic_box_tet_mesh(nx, ny, nz, L=(8.0, 2.0, 2.0), jitter=0.0, seed=DEFAULT_SEED, origin=(0.0, 0.0, 0.0)):
    """Periodic box origin + [0, Lx] x [0, Ly] x [0, Lz] with nx x ny x nz hexahedral
    cells, each split into 6 tetrahedra (Kuhn subdivision); K = 6 nx ny nz.

    Unique vertices are the nx ny nz grid points, id = i + nx (j + ny k).  Every
    tetrahedron is listed with positive orientation (det[v1-v0, v2-v0, v3-v0] > 0).
    jitter > 0 moves every unique vertex by independent U[-jitter h_d, jitter h_d]
    offsets per direction d (h_d = L_d / n_d), splitmix64 counter 3 id + d.

    Returns a dict: X (n_vert, 3), EToV (K, 4) int32, shift (K, 4, 3) periodic unwrap
    offsets (vertex k of element e sits at X[EToV[e, k]] + shift[e, k]), L (3,), dims.
    """
    if min(nx, ny, nz) < 3:
        raise ValueError('at least 3 cells per direction are needed so that faces have unique vertex triples')
    L = np.asarray(L, dtype=np.float64)
    n = np.array([nx, ny, nz])
    h = L / n
    i, j, k = np.meshgrid(np.arange(nx), np.arange(ny), np.arange(nz), indexing='ij')
    vid = (i + nx * (j + ny * k)).ravel()
    X = np.zeros((nx * ny * nz, 3))
    X[vid, 0] = (i * h[0]).ravel()
    X[vid, 1] = (j * h[1]).ravel()
    X[vid, 2] = (k * h[2]).ravel()
    X += np.asarray(origin, dtype=np.float64)[None, :]
    if jitter > 0.0:
        ids = np.arange(nx * ny * nz, dtype=np.uint64)
        for d in range(3):
            X[:, d] += uniform(3 * ids + d, seed, -jitter * h[d], jitter * h[d])
    # cells in order (k outer, j, i inner), six tetrahedra per cell
    kk, jj, ii = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing='ij')
    cell = np.stack([ii.ravel(), jj.ravel(), kk.ravel()], axis=1)          # (ncell, 3)
    corners = []
    for order in _KUHN_ORDERS:
        c = [np.zeros(3, dtype=np.int64)]
        for ax in order:
            nxt = c[-1].copy()
            nxt[ax] += 1
            c.append(nxt)
        # det[e_o0, e_o1, e_o2] is the sign of the axis permutation; fix odd ones
        sign = np.linalg.det(np.eye(3)[list(order)])
        if sign < 0:
            c[2], c[3] = c[3], c[2]
        corners.append(np.stack(c))
    corners = np.stack(corners)                                              # (6, 4, 3)
    g = cell[:, None, None, :] + corners[None, :, :, :]                      # (ncell, 6, 4, 3)
    wrap = g // n
    gm = g % n
    EToV = (gm[..., 0] + nx * (gm[..., 1] + ny * gm[..., 2])).reshape(-1, 4).astype(np.int32)
    shift = (wrap * L).reshape(-1, 4, 3).astype(np.float64)
    return {'X': X, 'EToV': EToV, 'shift': shift, 'L': L.copy(), 'dims': (nx, ny, nz)}


def min_altitude_3d(mesh):
    """Smallest tetrahedron altitude (3 volume / largest face area) at the Lagrangian positions."""
    P = mesh['X'][mesh['EToV']] + mesh['shift']
    vol = np.abs(np.einsum('ei,ei->e', P[:, 1] - P[:, 0], np.cross(P[:, 2] - P[:, 0], P[:, 3] - P[:, 0]))) / 6.0
    faces = ((0, 1, 2), (0, 1, 3), (1, 2, 3), (0, 2, 3))
    area = np.stack([0.5 * np.linalg.norm(np.cross(P[:, b] - P[:, a], P[:, c] - P[:, a]), axis=1) for a, b, c in faces])
    return float(np.min(3.0 * vol / area.max(axis=0)))


def cfl_dt_3d(mesh, N, c, cfl):
    """dt = cfl * h_min / (sqrt(3) c (N+1)^2) on a tetrahedral mesh (the 2D rule of cfl_dt)."""
    return cfl * min_altitude_3d(mesh) / (math.sqrt(3.0) * c * (N + 1) ** 2)


def random_flow_3d(x, y, z, seed, amp=0.05, L=(8.0, 2.0, 2.0)):
    """Smooth seeded periodic perturbation of the rest state on the box (rho, u, v, w)."""
    k = uniform(np.arange(16), seed)
    ax, ay, az = (2.0 * math.pi / Ld for Ld in L)
    rho = 1.0 + amp * (np.sin(ax * x + 6 * k[0]) * np.cos(ay * y + 6 * k[1]) + 0.5 * np.sin(az * z + 6 * k[2]))
    u = 0.5 * np.sin(ay * y + 6 * k[3]) + 0.3 * np.cos(ax * x + az * z + 6 * k[4])
    v = 0.5 * np.cos(az * z + 6 * k[5]) - 0.3 * np.sin(ax * x - ay * y + 6 * k[6])
    w = 0.4 * np.sin(ax * x + 6 * k[7]) + 0.2 * np.cos(ay * y + az * z + 6 * k[8])
    return rho, u, v, w


def channel_flow_3d(x, y, z, Ma, L=(8.0, 2.0, 2.0), eps=0.05):
    """Uniform stream u = 1 along x with a small smooth transverse disturbance (the
    deforming-channel workload's initial state): v, w of amplitude eps, rho from p' = c^2 rho'."""
    ax, ay, az = (2.0 * math.pi / Ld for Ld in L)
    u = np.ones_like(x)
    v = eps * np.sin(ax * x) * np.cos(az * z)
    w = eps * np.cos(ax * x) * np.sin(ay * y)
    rho = 1.0 + Ma * Ma * eps * np.cos(ax * x) * np.cos(ay * y)
    return rho, u, v, w


def taylor_green_3d(x, y, z, Ma, U0=1.0):
    """Initial state of the 3D Taylor-Green vortex (Sec. 7.2): u = U0 sin x cos y cos z,
    v = -U0 cos x sin y cos z, w = 0 on [-pi, pi]^3 (length scale 1); the paper gives no
    density, so rho carries the incompressible pressure of this field,
    p' = U0^2 (cos 2x + cos 2y)(cos 2z + 2) / 16, through p' = c^2 rho' with c = U0 / Ma."""
    u = U0 * np.sin(x) * np.cos(y) * np.cos(z)
    v = -U0 * np.cos(x) * np.sin(y) * np.cos(z)
    w = np.zeros_like(x)
    rho = 1.0 + Ma * Ma / 16.0 * (np.cos(2.0 * x) + np.cos(2.0 * y)) * (np.cos(2.0 * z) + 2.0)
    return rho, u, v, w


def tgv_box_tet_mesh(n, jitter=0.0, seed=DEFAULT_SEED):
    """The moving 3D Taylor-Green vortex mesh (Sec. 7.2): the periodic cube [-pi, pi]^3 of
    n^3 hexahedra, 6 tetrahedra each (K = 6 n^3; n = 32 gives the paper's 196608)."""
    return periodic_box_tet_mesh(n, n, n, L=(2 * math.pi,) * 3, jitter=jitter, seed=seed, origin=(-math.pi,) * 3)


# ---- two dimensions with boundaries: O-grid around a symmetric airfoil ------------------

BC_INTERIOR, BC_WALL, BC_FARFIELD = 0, 1, 2


def naca4_thickness(x, t=0.12):
    """Half-thickness of the symmetric NACA 4-digit section with the closed trailing edge
    (x in [0, 1], chord 1): 5 t (0.2969 sqrt x - 0.1260 x - 0.3516 x^2 + 0.2843 x^3 - 0.1036 x^4)."""
    x = np.asarray(x, dtype=np.float64)
    return 5.0 * t * (0.2969 * np.sqrt(x) - 0.1260 * x - 0.3516 * x ** 2 + 0.2843 * x ** 3 - 0.1036 * x ** 4)


def naca_ogrid_mesh(ni=256, nj=192, R=20.0, t=0.12, growth=1.02):
    """O-grid of ni wrap-around x nj radial quads around the NACA 00xx section (chord 1,
    leading edge at the origin), out to the circle of radius R about the mid-chord,
    each quad split into two counter-clockwise triangles; K = 2 ni nj.

    Surface point i sits at x = (1 + cos phi_i)/2, y = +-thickness (upper for
    sin phi > 0), phi_i = 2 pi i / ni; radial line i runs straight to the circle point at
    the same angle with geometric spacing (cell lengths grow by `growth` per cell).  Vertex id = i + ni j (i wraps around).  Returns the periodic-
    mesh dict of periodic_square_mesh plus bc (K, 3): per face (face f from local vertex f
    to f + 1) BC_WALL on the airfoil, BC_FARFIELD on the circle, BC_INTERIOR otherwise.
    """
    phi = 2.0 * math.pi * np.arange(ni) / ni
    xs = (1.0 + np.cos(phi)) / 2.0
    ys = np.sign(np.sin(phi)) * naca4_thickness(xs, t)
    cx = 0.5 + R * np.cos(phi)
    cy = R * np.sin(phi)
    q = float(growth)
    s = (q ** np.arange(nj + 1) - 1.0) / (q ** nj - 1.0) if q != 1.0 else np.linspace(0.0, 1.0, nj + 1)
    X = np.zeros((ni * (nj + 1), 2))
    for j in range(nj + 1):
        X[j * ni:(j + 1) * ni, 0] = xs + (cx - xs) * s[j]
        X[j * ni:(j + 1) * ni, 1] = ys + (cy - ys) * s[j]
    vid = lambda i, j: (i % ni) + ni * j
    tris, bcs = [], []
    for j in range(nj):
        for i in range(ni):
            a, b, c, d = vid(i, j), vid(i + 1, j), vid(i + 1, j + 1), vid(i, j + 1)
            for tri, fbc in (((a, b, c), (BC_WALL if j == 0 else 0, 0, 0)),
                             ((a, c, d), (0, BC_FARFIELD if j == nj - 1 else 0, 0))):
                P = X[list(tri)]
                area2 = (P[1, 0] - P[0, 0]) * (P[2, 1] - P[0, 1]) - (P[2, 0] - P[0, 0]) * (P[1, 1] - P[0, 1])
                if area2 < 0:   # reverse to counter-clockwise; face f runs from vertex f to f + 1
                    tri = (tri[0], tri[2], tri[1])
                    fbc = (fbc[2], fbc[1], fbc[0])
                tris.append(tri)
                bcs.append(fbc)
    EToV = np.array(tris, dtype=np.int32)
    return {'X': X, 'EToV': EToV, 'shift': np.zeros((EToV.shape[0], 3, 2)), 'L': np.array([0.0, 0.0]),
            'bc': np.array(bcs, dtype=np.int8), 'dims': (ni, nj)}


def wall_channel_mesh(nx, ny, Lx=1.0, Ly=1.0):
    """Box [0, Lx] x [0, Ly] of nx x ny squares split along the (0,0)-(1,1) diagonal into
    counter-clockwise triangles, walls at x = 0 and x = Lx, periodic in y; K = 2 nx ny.
    Vertex id = i + (nx + 1) j, j wrapping.  Same dict as naca_ogrid_mesh (bc per face)."""
    if ny < 3:
        raise ValueError('ny >= 3 is needed for unique periodic vertex pairs')
    hx, hy = Lx / nx, Ly / ny
    X = np.zeros(((nx + 1) * ny, 2))
    for j in range(ny):
        for i in range(nx + 1):
            X[i + (nx + 1) * j] = (i * hx, j * hy)
    vid = lambda i, j: i + (nx + 1) * (j % ny)
    tris, bcs, shifts = [], [], []
    for j in range(ny):
        for i in range(nx):
            wrap = lambda jj: (jj // ny) * Ly
            # (0,0),(1,0),(1,1): face 0 on y = const, face 1 on x = i + 1, face 2 the diagonal
            tris.append((vid(i, j), vid(i + 1, j), vid(i + 1, j + 1)))
            shifts.append(((0, wrap(j)), (0, wrap(j)), (0, wrap(j + 1))))
            bcs.append((0, BC_WALL if i + 1 == nx else 0, 0))
            # (0,0),(1,1),(0,1): face 0 the diagonal, face 1 on y = const, face 2 on x = i
            tris.append((vid(i, j), vid(i + 1, j + 1), vid(i, j + 1)))
            shifts.append(((0, wrap(j)), (0, wrap(j + 1)), (0, wrap(j + 1))))
            bcs.append((0, 0, BC_WALL if i == 0 else 0))
    return {'X': X, 'EToV': np.array(tris, dtype=np.int32), 'shift': np.array(shifts, dtype=np.float64),
            'L': np.array([0.0, Ly]), 'bc': np.array(bcs, dtype=np.int8), 'dims': (nx, ny)}
