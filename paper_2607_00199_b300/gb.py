"""Thin ctypes binding of libgb (C ABI in include/gb.h).

Argument marshalling only: every step of the solver runs in the library's
CUDA kernels.  Importing this module loads libgb.so and fails loudly if the
library has not been built (python -m paper_2607_00199_b300.build); there is
no fallback implementation.

Device arrays may be passed as torch CUDA tensors (their data_ptr() is used)
or as raw integer addresses.
"""
import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, 'libgb.so')

GB_OK, GB_EINVAL, GB_ENOMEM, GB_ECUDA, GB_EMESH, GB_ENAN = 0, -1, -2, -3, -4, -5
GB_FP64, GB_MIXED = 0, 1
GB_MOTION_STATIC, GB_MOTION_SINXY, GB_MOTION_PLUNGE, GB_MOTION_TGV3D = 0, 1, 2, 3
GB_BC_INTERIOR, GB_BC_WALL, GB_BC_FARFIELD = 0, 1, 2
GB_PML_RADIAL, GB_PML_SLAB, GB_PML_UNIFORM = 0, 1, 2
_NAMES = {GB_EINVAL: 'GB_EINVAL', GB_ENOMEM: 'GB_ENOMEM', GB_ECUDA: 'GB_ECUDA', GB_EMESH: 'GB_EMESH', GB_ENAN: 'GB_ENAN'}

_dp = ctypes.POINTER(ctypes.c_double)
_ip = ctypes.POINTER(ctypes.c_int32)


class GbMesh(ctypes.Structure):
    _fields_ = [('dim', ctypes.c_int32), ('n_vert', ctypes.c_int64), ('X', _dp),
                ('n_elem', ctypes.c_int64), ('EToV', _ip), ('elem_shift', _dp)]


class GbMotion(ctypes.Structure):
    _fields_ = [('kind', ctypes.c_int32), ('A', ctypes.c_double), ('T', ctypes.c_double),
                ('Lx', ctypes.c_double), ('Ly', ctypes.c_double)]


class GbWaveMotion(ctypes.Structure):
    _fields_ = [(k, ctypes.c_double) for k in ('A0', 'A1', 'Lx', 'wavelength', 'omega', 'r0sq', 'yc', 'zc')]


class GbPml(ctypes.Structure):
    _fields_ = [('kind', ctypes.c_int32)] + [(k, ctypes.c_double) for k in
                                             ('cx', 'cy', 'ex', 'ey', 'r0', 'd', 'sigma_max', 'power', 'alpha')]


class GBError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__('%s: %s' % (_NAMES.get(code, str(code)), msg))
        self.code = code


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError('libgb.so is not built (run python -m paper_2607_00199_b300.build): %s' % LIB_PATH)
    lib = ctypes.CDLL(LIB_PATH)
    vp, i64, c_int, c_double = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int, ctypes.c_double
    sig = {
        'gb_create': ([ctypes.POINTER(GbMesh), c_int, c_double, c_double, c_int, vp, ctypes.POINTER(vp)], c_int),
        'gb_create_bounded': ([ctypes.POINTER(GbMesh), ctypes.POINTER(ctypes.c_int8), _dp, c_int, c_double, c_double,
                               c_int, vp, ctypes.POINTER(vp)], c_int),
        'gb_set_motion': ([vp, ctypes.POINTER(GbMotion)], c_int),
        'gb_set_fields': ([vp, _dp, c_double], c_int),
        'gb_fields': ([vp, _dp, _dp], c_int),
        'gb_set_vertices': ([vp, _dp], c_int),
        'gb_vertices': ([vp, _dp], c_int),
        'gb_nodes': ([vp, _dp], c_int),
        'gb_rhs': ([vp, c_double, vp, vp], c_int),
        'gb_rhs_noalloc': ([vp, c_double, vp, vp], c_int),
        'gb_step': ([vp, c_double, i64], c_int),
        'gb_step_timed': ([vp, c_double, i64, _dp], c_int),
        'gb_sync': ([vp], c_int),
        'gb_set_stream': ([vp, vp], c_int),
        'gb_set_graph': ([vp, c_int], c_int),
        'gb_diagnostics': ([vp, _dp], c_int),
        'gb_diagnostics3d': ([vp, _dp], c_int),
        'gb_set_pml': ([vp, ctypes.POINTER(GbPml)], c_int),
        'gb_pml_fields': ([vp, _dp, ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int64)], c_int),
        'gb_set_diagnostics': ([vp, c_int, ctypes.c_int64], c_int),
        'gb_diagnostics_history': ([vp, _dp, ctypes.c_int64, ctypes.POINTER(ctypes.c_int64),
                                    ctypes.POINTER(ctypes.c_int64)], c_int),
        'gb_launch_config': ([vp, ctypes.POINTER(c_int)], c_int),
        'gb_group_launch_config': ([vp, c_int, ctypes.POINTER(c_int)], c_int),
        'gb_group_set_launch_config': ([vp, c_int, c_int], c_int),
        'gb_set_launch_config': ([vp, c_int], c_int),
        'gb_info': ([vp, ctypes.POINTER(c_int), ctypes.POINTER(c_int), ctypes.POINTER(c_int),
                     ctypes.POINTER(i64), ctypes.POINTER(i64), _dp, _dp, ctypes.POINTER(i64)], c_int),
        'gb_state_ptr': ([vp, ctypes.POINTER(vp)], c_int),
        'gb_destroy': ([vp], c_int),
        'gb_last_error': ([vp], ctypes.c_char_p),
        'gb_reference_operators': ([c_int] + [_dp] * 10 + [ctypes.POINTER(c_int)], c_int),
        'gb_sark_coefficients': ([c_double, _dp, _dp, _dp], c_int),
        'gb_set_wave_motion': ([vp, ctypes.POINTER(GbWaveMotion)], c_int),
        'gb_reference_operators3d': ([c_int] + [_dp] * 13 + [ctypes.POINTER(c_int)], c_int),
        'gb_group_create': ([c_int, vp, ctypes.POINTER(vp)], c_int),
        'gb_group_step': ([vp, ctypes.POINTER(vp), _dp, c_int, i64], c_int),
        'gb_group_destroy': ([vp], c_int),
        'gb_group_last_error': ([vp], ctypes.c_char_p),
    }
    for name, (args, res) in sig.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = res
    return lib


lib = _load()


def _ptr(a):
    return a.ctypes.data_as(_dp)


def _addr(x):
    """Device address of a torch tensor or an int."""
    if x is None:
        return None
    if hasattr(x, 'data_ptr'):
        return ctypes.c_void_p(x.data_ptr())
    return ctypes.c_void_p(int(x))


def _check(rc, handle=None):
    if rc != GB_OK:
        raise GBError(rc, lib.gb_last_error(handle).decode())
    return rc


def reference_operators(N):
    """The library's order-N reference operators (host computation, no GPU)."""
    Np, Nfp = (N + 1) * (N + 2) // 2, N + 1
    nc = ctypes.c_int(0)
    _check(lib.gb_reference_operators(N, *([None] * 10), ctypes.byref(nc)))
    Nc = nc.value
    out = {'r': np.zeros(Np), 's': np.zeros(Np), 'Dr': np.zeros((Np, Np)), 'Ds': np.zeros((Np, Np)),
           'LIFT': np.zeros((Np, 3 * Nfp)), 'I': np.zeros((Nc, Np)), 'P': np.zeros((Np, Nc)),
           'cr': np.zeros(Nc), 'cs': np.zeros(Nc), 'cw': np.zeros(Nc)}
    keys = ['r', 's', 'Dr', 'Ds', 'LIFT', 'I', 'P', 'cr', 'cs', 'cw']
    _check(lib.gb_reference_operators(N, *[_ptr(out[k]) for k in keys], ctypes.byref(nc)))
    out['Nc'] = Nc
    return out


def reference_operators3d(N):
    """The library's order-N tetrahedral reference operators (host computation, no GPU)."""
    Np, Nfp = (N + 1) * (N + 2) * (N + 3) // 6, (N + 1) * (N + 2) // 2
    nc = ctypes.c_int(0)
    _check(lib.gb_reference_operators3d(N, *([None] * 13), ctypes.byref(nc)))
    Nc = nc.value
    out = {'r': np.zeros(Np), 's': np.zeros(Np), 't': np.zeros(Np), 'Dr': np.zeros((Np, Np)),
           'Ds': np.zeros((Np, Np)), 'Dt': np.zeros((Np, Np)), 'LIFT': np.zeros((Np, 4 * Nfp)),
           'I': np.zeros((Nc, Np)), 'P': np.zeros((Np, Nc)), 'cr': np.zeros(Nc), 'cs': np.zeros(Nc),
           'ct': np.zeros(Nc), 'cw': np.zeros(Nc)}
    keys = ['r', 's', 't', 'Dr', 'Ds', 'Dt', 'LIFT', 'I', 'P', 'cr', 'cs', 'ct', 'cw']
    _check(lib.gb_reference_operators3d(N, *[_ptr(out[k]) for k in keys], ctypes.byref(nc)))
    out['Nc'] = Nc
    return out


def sark_coefficients(gamma):
    """(E[5], A[4,4], B[4]) from the library (host computation, no GPU)."""
    E, A, B = np.zeros(5), np.zeros(16), np.zeros(4)
    _check(lib.gb_sark_coefficients(float(gamma), _ptr(E), _ptr(A), _ptr(B)))
    return E, A.reshape(4, 4), B


class Solver:
    """Owns one gb_solver.  mesh is a dict with X, EToV, shift (see inputs.py); the
    dimension follows from X: (n_vert, 2) triangles with 6 fields, (n_vert, 3)
    tetrahedra with 10 fields.  A 2D mesh with a 'bc' array (n_elem x 3 face tags) is
    created with gb_create_bounded and the free stream far_state = (rho, u, v)."""

    def __init__(self, mesh, N, Ma, Re, precision=GB_FP64, stream=None, far_state=(1.0, 1.0, 0.0)):
        self._X = np.ascontiguousarray(mesh['X'], dtype=np.float64)
        self._EToV = np.ascontiguousarray(mesh['EToV'], dtype=np.int32)
        shift = mesh.get('shift')
        self._shift = None if shift is None else np.ascontiguousarray(shift, dtype=np.float64)
        self.dim = int(self._X.shape[1])
        self.nfields = 6 if self.dim == 2 else 10
        m = GbMesh(self.dim, self._X.shape[0], _ptr(self._X), self._EToV.shape[0],
                   self._EToV.ctypes.data_as(_ip), None if self._shift is None else _ptr(self._shift))
        h = ctypes.c_void_p(None)
        st = None if stream is None else ctypes.c_void_p(int(stream))
        if mesh.get('bc') is not None:
            self._bc = np.ascontiguousarray(mesh['bc'], dtype=np.int8)
            self._far = np.ascontiguousarray(far_state, dtype=np.float64)
            _check(lib.gb_create_bounded(ctypes.byref(m), self._bc.ctypes.data_as(ctypes.POINTER(ctypes.c_int8)),
                                         _ptr(self._far), int(N), float(Ma), float(Re), int(precision), st,
                                         ctypes.byref(h)))
        else:
            _check(lib.gb_create(ctypes.byref(m), int(N), float(Ma), float(Re), int(precision), st, ctypes.byref(h)))
        self.h = h
        self.N = int(N)
        self.precision = int(precision)
        np_, nfp, nc = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        K, nv, c, tau, nb = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_double(), ctypes.c_double(), ctypes.c_int64()
        _check(lib.gb_info(h, ctypes.byref(np_), ctypes.byref(nfp), ctypes.byref(nc), ctypes.byref(K),
                           ctypes.byref(nv), ctypes.byref(c), ctypes.byref(tau), ctypes.byref(nb)), h)
        self.Np, self.Nfp, self.Nc = np_.value, nfp.value, nc.value
        self.K, self.nv, self.c, self.tau = K.value, nv.value, c.value, tau.value
        self.device_bytes = nb.value

    def _c(self, rc):
        return _check(rc, self.h)

    def set_motion(self, A=0.0, T=1.0, Lx=2 * np.pi, Ly=2 * np.pi, kind=None):
        if kind is None:
            kind = GB_MOTION_SINXY if A != 0.0 else GB_MOTION_STATIC
        m = GbMotion(kind, float(A), float(T), float(Lx), float(Ly))
        self._c(lib.gb_set_motion(self.h, ctypes.byref(m)))

    def set_tgv_motion(self, A=np.pi / 6, T=20.0, L=2 * np.pi):
        """Deformation of the moving 3D Taylor-Green vortex (GB_MOTION_TGV3D, dim = 3)."""
        self.set_motion(A, T, L, 0.0, kind=GB_MOTION_TGV3D)

    def set_wave_motion(self, A0, A1=0.0, Lx=8.0, wavelength=1.0, omega=2 * np.pi, r0sq=0.25, yc=1.0, zc=1.0):
        """Travelling-wave lateral motion of a dim = 3 solver (gb_set_wave_motion)."""
        m = GbWaveMotion(float(A0), float(A1), float(Lx), float(wavelength), float(omega), float(r0sq),
                         float(yc), float(zc))
        self._c(lib.gb_set_wave_motion(self.h, ctypes.byref(m)))

    def set_pml(self, kind=GB_PML_RADIAL, centre=(0.5, 0.0), r0=17.0, d=3.0, sigma_max=1.0, power=2.0,
                alpha=0.0, direction=(1.0, 0.0)):
        """Perfectly matched layer (gb_set_pml, dim = 2); kind None removes it."""
        if kind is None:
            self._c(lib.gb_set_pml(self.h, None))
            return
        p = GbPml(int(kind), float(centre[0]), float(centre[1]), float(direction[0]), float(direction[1]),
                  float(r0), float(d), float(sigma_max), float(power), float(alpha))
        self._c(lib.gb_set_pml(self.h, ctypes.byref(p)))

    def pml_fields(self):
        """(Phi_n of the layer's elements (n_layer, 6, Np), their canonical ids ascending)."""
        n = ctypes.c_int64()
        self._c(lib.gb_pml_fields(self.h, None, None, ctypes.byref(n)))
        phi = np.zeros((n.value, 6, self.Np))
        ids = np.zeros(n.value, dtype=np.int64)
        if n.value:
            self._c(lib.gb_pml_fields(self.h, _ptr(phi), ids.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)),
                                      ctypes.byref(n)))
        return phi, ids

    def set_fields(self, q, t=0.0):
        q = np.ascontiguousarray(q, dtype=np.float64)
        if q.size != self.K * self.nfields * self.Np:
            raise ValueError('q must hold K*nfields*Np values')
        self._c(lib.gb_set_fields(self.h, _ptr(q), float(t)))

    def fields(self, out=None):
        q = out if out is not None else np.empty((self.K, self.nfields, self.Np))
        t = ctypes.c_double()
        self._c(lib.gb_fields(self.h, _ptr(q), ctypes.byref(t)))
        return q, t.value

    def set_vertices(self, x):
        x = np.ascontiguousarray(x, dtype=np.float64)
        if x.size != self.dim * self.nv:
            raise ValueError('x must hold n_vert*dim values')
        self._c(lib.gb_set_vertices(self.h, _ptr(x)))

    def vertices(self):
        x = np.empty((self.nv, self.dim))
        self._c(lib.gb_vertices(self.h, _ptr(x)))
        return x

    def nodes(self):
        xy = np.empty((self.K, self.Np, self.dim))
        self._c(lib.gb_nodes(self.h, _ptr(xy)))
        return xy

    def rhs(self, t, q_dev, F_dev):
        self._c(lib.gb_rhs(self.h, float(t), _addr(q_dev), _addr(F_dev)))

    def rhs_noalloc(self, t, q_dev, F_dev):
        """gb_rhs_noalloc: GB_MIXED right-hand side with a static scratch array (no allocation)."""
        self._c(lib.gb_rhs_noalloc(self.h, float(t), _addr(q_dev), _addr(F_dev)))

    def step(self, dt, nsteps=1):
        self._c(lib.gb_step(self.h, float(dt), int(nsteps)))

    def step_timed(self, dt, nsteps=1):
        """Steps with a CUDA event pair around every kernel; returns the summed device
        milliseconds per kernel kind: [stage 0, stage 1, stage 2, stage 3, vertex update]."""
        ms = np.zeros(5)
        self._c(lib.gb_step_timed(self.h, float(dt), int(nsteps), _ptr(ms)))
        return ms

    def diagnostics(self):
        """dict: mass, kinetic_energy (per unit area or volume), momentum_x, momentum_y and
        area (2D) or momentum_z and volume (3D)."""
        if self.dim == 3:
            out = np.zeros(6)
            self._c(lib.gb_diagnostics3d(self.h, _ptr(out)))
            keys = ('mass', 'kinetic_energy', 'momentum_x', 'momentum_y', 'momentum_z', 'volume')
            return {k: out[i] for i, k in enumerate(keys)}
        out = np.zeros(5)
        self._c(lib.gb_diagnostics(self.h, _ptr(out)))
        return {'mass': out[0], 'kinetic_energy': out[1], 'momentum_x': out[2], 'momentum_y': out[3], 'area': out[4]}

    def set_diagnostics(self, every, capacity=4096):
        """Record the diagnostics on the device after every `every`-th step (0: off)."""
        self._c(lib.gb_set_diagnostics(self.h, int(every), int(capacity)))
        self._diag_cap = int(capacity) if every else 0

    def diagnostics_history(self):
        """Recorded diagnostics, oldest first: dict of arrays t, mass, kinetic_energy,
        momentum_x, momentum_y, area (the volume in 3D), plus 'total' (records written
        since enabled)."""
        cap = getattr(self, '_diag_cap', 0)
        out = np.zeros((max(cap, 1), 6))
        n, tot = ctypes.c_int64(), ctypes.c_int64()
        self._c(lib.gb_diagnostics_history(self.h, _ptr(out), cap, ctypes.byref(n), ctypes.byref(tot)))
        r = out[:n.value]
        keys = ('t', 'mass', 'kinetic_energy', 'momentum_x', 'momentum_y', 'area')
        d = {k: r[:, i].copy() for i, k in enumerate(keys)}
        d['total'] = tot.value
        return d

    def launch_config(self):
        """The GB_MIXED launch shape (tuned at the first step; 0 for GB_FP64): in 2D the
        mma.sync kernel's warps per CTA (1, 2, 4) or 8 for the tcgen05 kernel; in 3D the
        tensor-core kernel's warps per CTA (1..8, N <= 3) or 16 for the FP32 kernel."""
        w = ctypes.c_int()
        self._c(lib.gb_launch_config(self.h, ctypes.byref(w)))
        return w.value

    def set_launch_config(self, warps_per_cta):
        """Fix the GB_MIXED launch shape instead of tuning.  2D: 1, 2 or 4 warps per CTA of
        the mma.sync kernel, or 8 for the tcgen05 kernel (N <= 4, no boundary faces).  3D: 1..8
        warps per CTA of the tensor-core kernel (N <= 3, at most as many as fit: 7 at N = 3),
        or 16 for the FP32 one-thread-per-node kernel."""
        self._c(lib.gb_set_launch_config(self.h, int(warps_per_cta)))

    def set_graph(self, enable):
        """Capture each step as a CUDA graph in step() (default on)."""
        self._c(lib.gb_set_graph(self.h, int(bool(enable))))

    def set_stream(self, stream):
        """Finish pending work, then use `stream` (a cudaStream_t address) from now on."""
        self._c(lib.gb_set_stream(self.h, None if stream is None else ctypes.c_void_p(int(stream))))

    def sync(self):
        self._c(lib.gb_sync(self.h))

    def state_ptr(self):
        p = ctypes.c_void_p()
        self._c(lib.gb_state_ptr(self.h, ctypes.byref(p)))
        return p.value

    def close(self):
        if getattr(self, 'h', None) is not None and self.h.value is not None:
            lib.gb_destroy(self.h)
            self.h = ctypes.c_void_p(None)

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Group:
    """Owns one gb_group: steps several GB_MIXED solvers of one order together."""

    def __init__(self, capacity, stream=None):
        h = ctypes.c_void_p(None)
        st = None if stream is None else ctypes.c_void_p(int(stream))
        rc = lib.gb_group_create(int(capacity), st, ctypes.byref(h))
        if rc != GB_OK:
            raise GBError(rc, lib.gb_group_last_error(None).decode())
        self.h = h
        self.capacity = int(capacity)

    def step(self, solvers, dts, nsteps=1):
        n = len(solvers)
        arr = (ctypes.c_void_p * n)(*[s.h.value for s in solvers])
        d = np.ascontiguousarray(dts, dtype=np.float64)
        rc = lib.gb_group_step(self.h, arr, _ptr(d), n, int(nsteps))
        if rc != GB_OK:
            raise GBError(rc, lib.gb_group_last_error(self.h).decode())

    def launch_config(self, N):
        """Warps per CTA of the group kernel last used for order N (0: not stepped yet)."""
        w = ctypes.c_int(0)
        rc = lib.gb_group_launch_config(self.h, int(N), ctypes.byref(w))
        if rc != GB_OK:
            raise GBError(rc, 'gb_group_launch_config: bad order')
        return w.value

    def set_launch_config(self, N, warps_per_cta):
        """Fix the group kernel's warps per CTA (1, 2 or 4) for order N and skip its tuner."""
        rc = lib.gb_group_set_launch_config(self.h, int(N), int(warps_per_cta))
        if rc != GB_OK:
            raise GBError(rc, 'gb_group_set_launch_config: bad order or shape')

    def close(self):
        if getattr(self, 'h', None) is not None and self.h.value is not None:
            lib.gb_group_destroy(self.h)
            self.h = ctypes.c_void_p(None)

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

