"""Python access to the FP64 CPU oracle (``oracle/hs3d_oracle.c``).

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the CPU
baseline leg of ``bench.py`` use this module; the product library never does.
The C source is compiled with gcc (``-O2 -fopenmp``, plain IEEE arithmetic, no
fast-math) into ``oracle/_build/liboracle.so`` on first use.

Array layouts (numpy, float64, C order):
  u, dudt      [E, 5, n, n, n]   (last axis is i, the xi direction)
  X            [E, 3, n, n, n]
  Ja           [E, 3(d), 3(c), n, n, n]   Ja[e, d, c] = J d xi_d / d x_c
  J            [E, n, n, n]
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "hs3d_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

PHYSICS = {"euler": 0, "ns": 1}
SURFACE = {"lf": 0, "roe": 1, "ec": 2, "rusanov": 3, "ldroe": 4, "matrix": 5}
VOLUME = {"standard": 0, "ec": 1, "kg": 2, "pirozzoli": 3, "ducros": 4, "morinishi": 5, "ir": 6}
TIME = {"rk3": 0, "rk4": 1}


def build(force: bool = False) -> str:
    """Compile the oracle shared library; returns its path."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-std=c11", "-D_GNU_SOURCE", "-shared", "-fPIC",
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


class _Box(C.Structure):
    _fields_ = [("ex", C.c_int), ("ey", C.c_int), ("ez", C.c_int), ("N", C.c_int),
                ("lo", C.c_double * 3), ("hi", C.c_double * 3), ("amp", C.c_double), ("nodes", C.c_int)]

NODES = {"lobatto": 0, "gauss": 1}


class _Cfg(C.Structure):
    _fields_ = [("physics", C.c_int), ("surface_flux", C.c_int), ("volume_form", C.c_int),
                ("gamma", C.c_double), ("Re", C.c_double), ("Pr", C.c_double), ("cfl", C.c_double),
                ("time_scheme", C.c_int)]


_dp = np.ctypeslib.ndpointer(dtype=np.float64, flags="C_CONTIGUOUS")


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = C.CDLL(build())
            L.orc_lgl.argtypes = [C.c_int, _dp, _dp]
            L.orc_dmatrix.argtypes = [C.c_int, _dp, _dp]
            L.orc_mesh_create.argtypes = [C.POINTER(_Box), C.c_void_p]
            L.orc_mesh_create.restype = C.c_void_p
            L.orc_mesh_destroy.argtypes = [C.c_void_p]
            L.orc_mesh_E.argtypes = [C.c_void_p]
            L.orc_mesh_arrays.argtypes = [C.c_void_p] + [C.c_void_p] * 6
            L.orc_neighbour.argtypes = [C.c_void_p, C.c_int, C.c_int, C.c_int]
            L.orc_metrics.argtypes = [C.c_int, C.c_int, _dp, _dp, _dp, _dp]
            for name in ("orc_flux_lf", "orc_flux_roe", "orc_flux_ec", "orc_flux_rusanov", "orc_flux_ldroe",
                         "orc_flux_matrix", "orc_flux_morinishi", "orc_flux_ir"):
                getattr(L, name).argtypes = [_dp, _dp, _dp, C.c_double, _dp]
            L.orc_flux_roe_signed.argtypes = [_dp, _dp, _dp, C.c_double, _dp, C.c_int]
            L.orc_flux_euler.argtypes = [_dp, _dp, C.c_double, _dp]
            L.orc_flux_visc.argtypes = [_dp, _dp, C.c_double, C.c_double, _dp, _dp]
            L.orc_entropy_vars.argtypes = [_dp, C.c_double, _dp]
            L.orc_logmean.argtypes = [C.c_double, C.c_double]
            L.orc_logmean.restype = C.c_double
            L.orc_residual.argtypes = [C.c_void_p, C.POINTER(_Cfg), _dp, _dp]
            L.orc_residual_nodal.argtypes = [C.c_void_p, C.POINTER(_Cfg), _dp, _dp]
            L.orc_gauss.argtypes = [C.c_int, _dp, _dp]
            L.orc_lagrange_at.argtypes = [C.c_int, _dp, C.c_double, _dp]
            L.orc_mesh_faces.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]
            L.orc_gradients.argtypes = [C.c_void_p, C.POINTER(_Cfg), _dp, _dp]
            L.orc_dt.argtypes = [C.c_void_p, C.POINTER(_Cfg), _dp]
            L.orc_dt.restype = C.c_double
            L.orc_rk3_step.argtypes = [C.c_void_p, C.POINTER(_Cfg), _dp, _dp, C.c_double, C.POINTER(C.c_double)]
            L.orc_rk3_coefficients.argtypes = [_dp, _dp, _dp]
            L.orc_rk4_coefficients.argtypes = [_dp, _dp, _dp]
            L.orc_lsrk_stage.argtypes = [C.c_int, C.c_longlong, C.c_int, C.c_double, _dp, _dp, _dp]
            L.orc_flux_split.argtypes = [C.c_int, _dp, _dp, _dp, C.c_double, _dp]
            L.orc_lsrk3_stage.argtypes = [C.c_longlong, C.c_int, C.c_double, _dp, _dp, _dp]
            L.orc_ic_vortex.argtypes = [C.c_void_p, C.c_double, C.c_double, C.c_double, C.c_double,
                                        C.c_double, C.c_double, _dp]
            L.orc_ic_tgv.argtypes = [C.c_void_p, C.c_double, C.c_double, _dp]
            L.orc_integrals.argtypes = [C.c_void_p, C.c_double, _dp, C.c_void_p, _dp]
            L.orc_mortar_matrices.argtypes = [C.c_int, C.c_int, _dp, _dp]
            L.orc_pmesh_create.argtypes = [C.POINTER(_Box), C.c_void_p]
            L.orc_pmesh_create.restype = C.c_void_p
            L.orc_pmesh_create3.argtypes = [C.POINTER(_Box), C.c_void_p]
            L.orc_pmesh_create3.restype = C.c_void_p
            L.orc_pmesh_destroy.argtypes = [C.c_void_p]
            L.orc_pmesh_Ngeo.argtypes = [C.c_void_p]
            L.orc_pmesh_arrays.argtypes = [C.c_void_p] + [C.c_void_p] * 5
            L.orc_presidual.argtypes = [C.c_void_p, C.POINTER(_Cfg), _dp, _dp]
            L.orc_pgradients.argtypes = [C.c_void_p, C.POINTER(_Cfg), _dp, _dp]
            L.orc_pdt.argtypes = [C.c_void_p, C.POINTER(_Cfg), _dp]
            L.orc_pdt.restype = C.c_double
            L.orc_prk_step.argtypes = [C.c_void_p, C.POINTER(_Cfg), _dp, _dp, C.c_double, C.POINTER(C.c_double)]
            L.orc_pic.argtypes = [C.c_void_p, C.c_int, _dp, _dp]
            L.orc_pintegrals.argtypes = [C.c_void_p, C.c_double, _dp, C.c_void_p, _dp]
            _lib = L
    return _lib


# --------------------------------------------------------------------------- 1-D operators

def lgl(N: int):
    """Gauss-Lobatto nodes and weights on [-1, 1] (ascending)."""
    x = np.zeros(N + 1)
    w = np.zeros(N + 1)
    if lib().orc_lgl(N, x, w) != 0:
        raise ValueError("N must be >= 1")
    return x, w


def gauss(N: int):
    x, w = np.zeros(N + 1), np.zeros(N + 1)
    lib().orc_gauss(N, x, w)
    return x, w


def lagrange_at(x, y):
    x = np.ascontiguousarray(x, dtype=np.float64)
    out = np.zeros(x.size)
    lib().orc_lagrange_at(x.size, x, float(y), out)
    return out


def dmatrix(N: int, x=None):
    """Nodal derivative matrix D[i, j] = l_j'(x_i) on the Gauss-Lobatto nodes (or given x)."""
    if x is None:
        x, _ = lgl(N)
    D = np.zeros((N + 1, N + 1))
    lib().orc_dmatrix(N, np.ascontiguousarray(x, dtype=np.float64), D)
    return D


# --------------------------------------------------------------------------- configuration

class Cfg:
    def __init__(self, physics="euler", surface="lf", volume="standard", gamma=1.4, Re=1600.0, Pr=0.72, cfl=0.5,
                 time="rk3"):
        self.physics, self.surface, self.volume = physics, surface, volume
        self.gamma, self.Re, self.Pr, self.cfl, self.time = gamma, Re, Pr, cfl, time

    def c(self):
        return _Cfg(PHYSICS[self.physics], SURFACE[self.surface], VOLUME[self.volume],
                    self.gamma, self.Re, self.Pr, self.cfl, TIME[self.time])


class Mesh:
    """Oracle mesh of an ex*ey*ez periodic box with Gauss-Lobatto nodes of degree N."""

    def __init__(self, ex, ey, ez, N, lo=(0.0, 0.0, 0.0), hi=(1.0, 1.0, 1.0), amp=0.0, X=None, nodes="lobatto"):
        """X, if given, holds the Gauss-Lobatto geometry nodes; `nodes` picks
        the solution nodes ("lobatto" or "gauss")."""
        self.ex, self.ey, self.ez, self.N = ex, ey, ez, N
        self.n = N + 1
        self.E = ex * ey * ez
        self.lo, self.hi, self.amp = tuple(lo), tuple(hi), amp
        self.nodes = nodes
        box = _Box(ex, ey, ez, N, (C.c_double * 3)(*lo), (C.c_double * 3)(*hi), amp, NODES[nodes])
        Xp = None
        if X is not None:
            X = np.ascontiguousarray(X, dtype=np.float64)
            assert X.shape == (self.E, 3, self.n, self.n, self.n)
            Xp = X.ctypes.data
        self._h = lib().orc_mesh_create(C.byref(box), Xp)
        if not self._h:
            raise ValueError("bad mesh description")
        n = self.n
        self.xi = np.zeros(n)
        self.w = np.zeros(n)
        self.D = np.zeros((n, n))
        self.X = np.zeros((self.E, 3, n, n, n))
        self.Ja = np.zeros((self.E, 3, 3, n, n, n))
        self.J = np.zeros((self.E, n, n, n))
        lib().orc_mesh_arrays(self._h, *(a.ctypes.data for a in (self.xi, self.w, self.D, self.X, self.Ja, self.J)))
        self.Sf = np.zeros((self.E, 3, 2, 3, n, n))   # own face metrics [e][d][side -1/+1][c][tb][ta]
        self.lb = np.zeros(n)
        self.rb = np.zeros(n)
        lib().orc_mesh_faces(self._h, self.Sf.ctypes.data, self.lb.ctypes.data, self.rb.ctypes.data)

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            lib().orc_mesh_destroy(h)
            self._h = None

    @property
    def shape(self):
        return (self.E, 5, self.n, self.n, self.n)

    def neighbour(self, e, d, side):
        return lib().orc_neighbour(self._h, e, d, side)

    # ---- initial conditions
    def ic_vortex(self, gamma=1.4, Ma=0.5, beta=5.0, xc=None, yc=None, t=0.0):
        if xc is None:
            xc = 0.5 * (self.lo[0] + self.hi[0])
        if yc is None:
            yc = 0.5 * (self.lo[1] + self.hi[1])
        u = np.zeros(self.shape)
        lib().orc_ic_vortex(self._h, gamma, Ma, beta, xc, yc, t, u)
        return u

    def ic_tgv(self, gamma=1.4, Ma=0.1):
        u = np.zeros(self.shape)
        lib().orc_ic_tgv(self._h, gamma, Ma, u)
        return u

    # ---- operators
    def residual(self, cfg: Cfg, u):
        u = np.ascontiguousarray(u, dtype=np.float64)
        out = np.zeros(self.shape)
        if lib().orc_residual(self._h, C.byref(cfg.c()), u, out) != 0:
            raise ValueError("residual: unsupported configuration for these nodes")
        return out

    def residual_nodal(self, cfg: Cfg, u):
        """The interpolated-trace form of the residual (any nodes)."""
        u = np.ascontiguousarray(u, dtype=np.float64)
        out = np.zeros(self.shape)
        if lib().orc_residual_nodal(self._h, C.byref(cfg.c()), u, out) != 0:
            raise ValueError("residual: unsupported configuration")
        return out

    def gradients(self, cfg: Cfg, u):
        """BR1 gradients [E, 4(v1,v2,v3,T), 3(x,y,z), n, n, n]."""
        u = np.ascontiguousarray(u, dtype=np.float64)
        out = np.zeros((self.E, 4, 3, self.n, self.n, self.n))
        lib().orc_gradients(self._h, C.byref(cfg.c()), u, out)
        return out

    def dt(self, cfg: Cfg, u):
        return lib().orc_dt(self._h, C.byref(cfg.c()), np.ascontiguousarray(u, dtype=np.float64))

    def rk3_step(self, cfg: Cfg, u, g=None, dt=0.0):
        """One Williamson RK3 step in place on u (and g); returns the dt used."""
        if g is None:
            g = np.zeros_like(u)
        used = C.c_double(0.0)
        lib().orc_rk3_step(self._h, C.byref(cfg.c()), u, g, dt, C.byref(used))
        return used.value

    def integrals(self, gamma, u, dudt=None):
        """[sum J w u_v (or dudt_v) for v in 0..4, entropy rate, entropy-rate magnitude scale]."""
        out = np.zeros(7)
        u = np.ascontiguousarray(u, dtype=np.float64)
        dp = None
        if dudt is not None:
            dudt = np.ascontiguousarray(dudt, dtype=np.float64)
            dp = dudt.ctypes.data
        lib().orc_integrals(self._h, gamma, u, dp, out)
        return out


# --------------------------------------------------------------------------- point functions

def _v(a, k=5):
    a = np.ascontiguousarray(a, dtype=np.float64)
    assert a.shape == (k,)
    return a


def flux_euler(u, a, gamma=1.4):
    f = np.zeros(5)
    lib().orc_flux_euler(_v(u), _v(a, 3), gamma, f)
    return f


def flux_lf(uL, uR, nh, gamma=1.4):
    f = np.zeros(5)
    lib().orc_flux_lf(_v(uL), _v(uR), _v(nh, 3), gamma, f)
    return f


def flux_roe(uL, uR, nh, gamma=1.4):
    f = np.zeros(5)
    lib().orc_flux_roe(_v(uL), _v(uR), _v(nh, 3), gamma, f)
    return f


def roe_wave_sum(uL, uR, nh, gamma=1.4):
    """sum_k lambda_k alpha_k r_k with signed eigenvalues."""
    f = np.zeros(5)
    lib().orc_flux_roe_signed(_v(uL), _v(uR), _v(nh, 3), gamma, f, 1)
    return f


def flux_ec(uL, uR, a, gamma=1.4):
    f = np.zeros(5)
    lib().orc_flux_ec(_v(uL), _v(uR), _v(a, 3), gamma, f)
    return f


def flux_visc(q, G, mu, kappa, a):
    f = np.zeros(5)
    lib().orc_flux_visc(_v(q, 4), np.ascontiguousarray(G, dtype=np.float64).reshape(12), mu, kappa, _v(a, 3), f)
    return f


def entropy_vars(u, gamma=1.4):
    w = np.zeros(5)
    lib().orc_entropy_vars(_v(u), gamma, w)
    return w


def logmean(a, b):
    return lib().orc_logmean(a, b)


def flux_split(kind, uL, uR, a, gamma=1.4):
    """Two-point split-form flux: kind "kg", "pirozzoli", "ducros",
    "morinishi", "ir" (Ismail-Roe) or "ec" (Chandrashekar)."""
    f = np.zeros(5)
    if kind == "ec":
        lib().orc_flux_ec(_v(uL), _v(uR), _v(a, 3), gamma, f)
    elif kind in ("morinishi", "ir"):
        getattr(lib(), "orc_flux_" + kind)(_v(uL), _v(uR), _v(a, 3), gamma, f)
    else:
        lib().orc_flux_split(VOLUME[kind], _v(uL), _v(uR), _v(a, 3), gamma, f)
    return f


def flux_surface(kind, uL, uR, nh, gamma=1.4):
    """Surface flux with unit normal nh: "lf", "roe", "rusanov", "ldroe",
    "matrix" (entropy-stable matrix dissipation) or "ec"."""
    f = np.zeros(5)
    getattr(lib(), "orc_flux_" + kind)(_v(uL), _v(uR), _v(nh, 3), gamma, f)
    return f


def rk4_coefficients():
    A, B, Cc = np.zeros(5), np.zeros(5), np.zeros(5)
    lib().orc_rk4_coefficients(A, B, Cc)
    return A, B, Cc


def lsrk_stage(scheme, k, dt, u, g, R):
    u = np.ascontiguousarray(u, dtype=np.float64)
    lib().orc_lsrk_stage(TIME[scheme], u.size, k, dt, u, g, np.ascontiguousarray(R, dtype=np.float64))


def rk3_coefficients():
    A, B, Cc = np.zeros(3), np.zeros(3), np.zeros(3)
    lib().orc_rk3_coefficients(A, B, Cc)
    return A, B, Cc


def lsrk3_stage(k, dt, u, g, R):
    u = np.ascontiguousarray(u, dtype=np.float64)
    lib().orc_lsrk3_stage(u.size, k, dt, u, g, np.ascontiguousarray(R, dtype=np.float64))


# --------------------------------------------------------------------------- per-element degree (Sec. 3.6)

def mortar_matrices(Ns: int, Nm: int):
    """(Pi, P): interpolation from degree Ns to the mortar degree Nm >= Ns
    ([Nm+1, Ns+1]) and the L2 projection back ([Ns+1, Nm+1])."""
    Pi = np.zeros((Nm + 1, Ns + 1))
    P = np.zeros((Ns + 1, Nm + 1))
    if lib().orc_mortar_matrices(Ns, Nm, Pi, P) != 0:
        raise ValueError("need 1 <= Ns <= Nm")
    return Pi, P


class PMesh:
    """Oracle mesh of an ex*ey*ez periodic box whose elements carry their own
    degrees (Gauss-Lobatto nodes), coupled by mortars.  `degrees` is one
    degree per element (isotropic, shape (E,)) or one per element and
    reference direction (anisotropic, shape (E, 3): P_x, P_y, P_z).

    The state is one flat float64 vector of element blocks
    [5, n_z, n_y, n_x] in element order; `block(u, e)` views element e's
    block."""

    def __init__(self, ex, ey, ez, degrees, lo=(0.0, 0.0, 0.0), hi=(1.0, 1.0, 1.0), amp=0.0):
        self.ex, self.ey, self.ez = ex, ey, ez
        self.E = ex * ey * ez
        d = np.asarray(degrees, dtype=np.int32)
        if d.ndim == 2:
            assert d.shape == (self.E, 3)
            deg3 = np.ascontiguousarray(d)
        else:
            d = d.reshape(-1)
            assert d.size == self.E
            deg3 = np.ascontiguousarray(np.repeat(d[:, None], 3, axis=1))
        self.degrees3 = deg3.copy()
        self.isotropic = bool(np.all(deg3 == deg3[:, :1]))
        self.degrees = deg3[:, 0].copy() if self.isotropic else None
        self.lo, self.hi, self.amp = tuple(lo), tuple(hi), amp
        box = _Box(ex, ey, ez, 0, (C.c_double * 3)(*lo), (C.c_double * 3)(*hi), amp, 0)
        if d.ndim == 2:
            self._h = lib().orc_pmesh_create3(C.byref(box), deg3.ctypes.data)
        else:
            dd = np.ascontiguousarray(d)
            self._h = lib().orc_pmesh_create(C.byref(box), dd.ctypes.data)
        if not self._h:
            raise ValueError("bad p-mesh description")
        self.Ngeo = lib().orc_pmesh_Ngeo(self._h)
        self.off = np.zeros(self.E + 1, dtype=np.int64)
        self.noff = np.zeros(self.E + 1, dtype=np.int64)
        lib().orc_pmesh_arrays(self._h, self.off.ctypes.data, self.noff.ctypes.data, None, None, None)
        nodes = int(self.noff[-1])
        self._X = np.zeros(3 * nodes)
        self._Ja = np.zeros(9 * nodes)
        self._J = np.zeros(nodes)
        lib().orc_pmesh_arrays(self._h, None, None, self._X.ctypes.data, self._Ja.ctypes.data, self._J.ctypes.data)
        self.size = int(self.off[-1])

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            lib().orc_pmesh_destroy(h)
            self._h = None

    def n(self, e):
        """Nodes per direction of an isotropic element."""
        nx, ny, nz = self.shape3(e)
        assert nx == ny == nz
        return nx

    def shape3(self, e):
        """(n_x, n_y, n_z) of element e."""
        return tuple(int(x) + 1 for x in self.degrees3[e])

    def _dims(self, e):
        nx, ny, nz = self.shape3(e)
        return (nz, ny, nx)

    def block(self, u, e):
        return u[self.off[e]:self.off[e + 1]].reshape(5, *self._dims(e))

    def X(self, e):
        return self._X[3 * self.noff[e]:3 * self.noff[e + 1]].reshape(3, *self._dims(e))

    def Ja(self, e):
        return self._Ja[9 * self.noff[e]:9 * self.noff[e + 1]].reshape(3, 3, *self._dims(e))

    def J(self, e):
        return self._J[self.noff[e]:self.noff[e + 1]].reshape(*self._dims(e))

    def neighbour(self, e, d, side):
        ab = [e % self.ex, (e // self.ex) % self.ey, e // (self.ex * self.ey)]
        ab[d] = (ab[d] + side) % (self.ex, self.ey, self.ez)[d]
        return ab[0] + self.ex * (ab[1] + self.ey * ab[2])

    def empty(self):
        return np.zeros(self.size)

    def ic_tgv(self, gamma=1.4, Ma=0.1):
        u = self.empty()
        lib().orc_pic(self._h, 0, np.array([gamma, Ma, 0.0, 0.0, 0.0]), u)
        return u

    def ic_vortex(self, gamma=1.4, Ma=0.5, beta=5.0, xc=None, yc=None):
        xc = 0.5 * (self.lo[0] + self.hi[0]) if xc is None else xc
        yc = 0.5 * (self.lo[1] + self.hi[1]) if yc is None else yc
        u = self.empty()
        lib().orc_pic(self._h, 1, np.array([gamma, Ma, beta, xc, yc]), u)
        return u

    def residual(self, cfg: Cfg, u):
        u = np.ascontiguousarray(u, dtype=np.float64)
        out = self.empty()
        if lib().orc_presidual(self._h, C.byref(cfg.c()), u, out) != 0:
            raise MemoryError("residual")
        return out

    def gradients(self, cfg: Cfg, u):
        """BR1 gradients, flat: element e's [4, 3, n, n, n] block at 12 noff[e]."""
        out = np.zeros(12 * int(self.noff[-1]))
        lib().orc_pgradients(self._h, C.byref(cfg.c()), np.ascontiguousarray(u, dtype=np.float64), out)
        return out

    def dt(self, cfg: Cfg, u):
        return lib().orc_pdt(self._h, C.byref(cfg.c()), np.ascontiguousarray(u, dtype=np.float64))

    def rk_step(self, cfg: Cfg, u, g, dt=0.0):
        """One low-storage RK step in place on u and g; returns the dt used."""
        used = C.c_double(0.0)
        lib().orc_prk_step(self._h, C.byref(cfg.c()), u, g, dt, C.byref(used))
        return used.value

    def integrals(self, gamma, u, dudt=None):
        out = np.zeros(7)
        dp = None
        if dudt is not None:
            dudt = np.ascontiguousarray(dudt, dtype=np.float64)
            dp = dudt.ctypes.data
        lib().orc_pintegrals(self._h, gamma, np.ascontiguousarray(u, dtype=np.float64), dp, out)
        return out
