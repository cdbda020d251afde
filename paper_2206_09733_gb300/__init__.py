"""hs3d: GB300-native DGSEM residual and low-storage RK3 for compressible Euler/Navier-Stokes.

A thin ctypes binding over the C-ABI in ``include/hs3d.h`` (``libhs3d.so``,
built in-tree by ``paper_2206_09733_gb300.build``).  It only marshals
arguments: device arrays are torch CUDA tensors (float64, contiguous) passed
by pointer together with the current torch stream; every step of the
computation runs in the library's CUDA kernels.  There is no CPU fallback --
without the built library or a GPU, calls raise.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libhs3d.so")

OK, PENDING = 0, 1
ERR_INVALID, ERR_NOMEM, ERR_CUDA, ERR_TIMEOUT, ERR_NONPHYSICAL, ERR_UNSUPPORTED = -1, -2, -3, -4, -5, -6
STATUS_NAMES = {0: "OK", 1: "PENDING", -1: "INVALID", -2: "NOMEM", -3: "CUDA", -4: "TIMEOUT",
                -5: "NONPHYSICAL", -6: "UNSUPPORTED"}
EULER, NS = 0, 1
FLUX_LF, FLUX_ROE, FLUX_EC, FLUX_RUSANOV, FLUX_LDROE, FLUX_MATRIX = 0, 1, 2, 3, 4, 5
VOL_STANDARD, VOL_EC, VOL_KG, VOL_PIROZZOLI, VOL_DUCROS, VOL_MORINISHI, VOL_IR = 0, 1, 2, 3, 4, 5, 6
TIME_RK3, TIME_RK4 = 0, 1
NODES_LOBATTO, NODES_GAUSS = 0, 1
FP64, MIXED32, MIXED_TC = 0, 1, 2
IC_VORTEX, IC_TGV = 0, 1

PHYSICS = {"euler": EULER, "ns": NS}
SURFACE = {"lf": FLUX_LF, "roe": FLUX_ROE, "ec": FLUX_EC, "rusanov": FLUX_RUSANOV, "ldroe": FLUX_LDROE,
           "matrix": FLUX_MATRIX}
VOLUME = {"standard": VOL_STANDARD, "ec": VOL_EC, "kg": VOL_KG, "pirozzoli": VOL_PIROZZOLI, "ducros": VOL_DUCROS,
          "morinishi": VOL_MORINISHI, "ir": VOL_IR}
TIME = {"rk3": TIME_RK3, "rk4": TIME_RK4}
NODES = {"lobatto": NODES_LOBATTO, "gauss": NODES_GAUSS}
PRECISION = {"fp64": FP64, "mixed32": MIXED32, "mixed_tc": MIXED_TC}

# every entry point declared in include/hs3d.h
EXPORTS = ["hs3d_mesh_create", "hs3d_mesh_destroy", "hs3d_mesh_info", "hs3d_mesh_geometry", "hs3d_init_state",
           "hs3d_residual", "hs3d_rk3_step", "hs3d_rk3_run", "hs3d_dt", "hs3d_clock", "hs3d_diagnostics",
           "hs3d_server_create", "hs3d_server_destroy", "hs3d_server_set_launch_mode", "hs3d_submit", "hs3d_poll",
           "hs3d_server_stats",
           "hs3d_last_error", "hs3d_version", "hs3d_rk3_step_profiled", "hs3d_alu_peaks",
           "hs3d_diagnostics_noalloc", "hs3d_autotune", "hs3d_check_rounding", "hs3d_pmesh_create", "hs3d_pmesh_create3",
           "hs3d_pmesh_destroy", "hs3d_pmesh_layout", "hs3d_pmesh_geometry", "hs3d_pmesh_init_state",
           "hs3d_pmesh_residual", "hs3d_pmesh_run", "hs3d_pmesh_clock", "hs3d_pmesh_diagnostics"]


class HS3DError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"hs3d {STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


class MeshDesc(C.Structure):
    _fields_ = [("ex", C.c_int), ("ey", C.c_int), ("ez", C.c_int), ("N", C.c_int),
                ("lo", C.c_double * 3), ("hi", C.c_double * 3), ("periodic", C.c_int * 3),
                ("perturb_amp", C.c_double), ("node_xyz", C.c_void_p), ("nodes", C.c_int)]


class SolverCfg(C.Structure):
    _fields_ = [("physics", C.c_int), ("surface_flux", C.c_int), ("volume_form", C.c_int), ("precision", C.c_int),
                ("gamma", C.c_double), ("Re", C.c_double), ("Pr", C.c_double), ("Ma", C.c_double),
                ("cfl", C.c_double), ("time_scheme", C.c_int)]


class IC(C.Structure):
    _fields_ = [("kind", C.c_int), ("gamma", C.c_double), ("Ma", C.c_double), ("beta", C.c_double),
                ("xc", C.c_double), ("yc", C.c_double), ("t", C.c_double)]


class Request(C.Structure):
    _fields_ = [("mesh", MeshDesc), ("cfg", SolverCfg), ("ic", IC), ("t_final", C.c_double),
                ("n_steps", C.c_int), ("result_host", C.c_void_p)]


class Result(C.Structure):
    _fields_ = [("status", C.c_int), ("t_sim", C.c_double), ("steps", C.c_int64), ("dof", C.c_int64),
                ("t_submit", C.c_double), ("t_admit", C.c_double), ("t_done", C.c_double),
                ("device_bytes", C.c_size_t)]


_lib = None
_lock = threading.Lock()


def lib():
    """Load libhs3d.so (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise HS3DError(ERR_CUDA, f"{LIB_PATH} missing: run paper_2206_09733_gb300.build")
            L = C.CDLL(LIB_PATH)
            vp, i, d = C.c_void_p, C.c_int, C.c_double
            sig = {
                "hs3d_mesh_create": [C.POINTER(MeshDesc), C.POINTER(vp)],
                "hs3d_mesh_destroy": [vp],
                "hs3d_mesh_info": [vp, C.POINTER(C.c_int64), C.POINTER(i), C.POINTER(C.c_size_t)],
                "hs3d_mesh_geometry": [vp, vp, vp, vp, vp],
                "hs3d_init_state": [vp, C.POINTER(IC), vp, vp],
                "hs3d_residual": [vp, C.POINTER(SolverCfg), vp, vp, vp],
                "hs3d_rk3_step": [vp, C.POINTER(SolverCfg), vp, vp, d, vp],
                "hs3d_rk3_run": [vp, C.POINTER(SolverCfg), vp, vp, d, i, vp],
                "hs3d_dt": [vp, C.POINTER(SolverCfg), vp, vp, vp],
                "hs3d_clock": [vp, C.POINTER(d), C.POINTER(C.c_int64), i, vp],
                "hs3d_diagnostics": [vp, C.POINTER(SolverCfg), vp, vp, vp, vp],
                "hs3d_server_create": [C.c_size_t, i, C.POINTER(vp)],
                "hs3d_server_destroy": [vp],
                "hs3d_server_set_launch_mode": [vp, i],
                "hs3d_submit": [vp, C.POINTER(Request), C.POINTER(C.c_uint64)],
                "hs3d_poll": [vp, C.c_uint64, C.POINTER(Result)],
                "hs3d_server_stats": [vp, C.POINTER(C.c_int64), C.POINTER(C.c_int64), C.POINTER(C.c_int64),
                                      C.POINTER(C.c_size_t)],
                "hs3d_rk3_step_profiled": [vp, C.POINTER(SolverCfg), vp, vp, d, C.POINTER(d), vp],
                "hs3d_alu_peaks": [C.POINTER(d), vp],
                "hs3d_diagnostics_noalloc": [i, C.c_int64, d, i, vp, vp, vp, vp, vp],
                "hs3d_autotune": [vp, C.POINTER(SolverCfg), C.POINTER(i), vp],
                "hs3d_check_rounding": [vp, C.c_int64, vp, vp],
                "hs3d_pmesh_create": [C.POINTER(MeshDesc), vp, C.POINTER(vp)],
                "hs3d_pmesh_create3": [C.POINTER(MeshDesc), vp, C.POINTER(vp)],
                "hs3d_pmesh_destroy": [vp],
                "hs3d_pmesh_layout": [vp, vp, C.POINTER(i)],
                "hs3d_pmesh_geometry": [vp, vp, vp, vp],
                "hs3d_pmesh_init_state": [vp, C.POINTER(IC), vp, vp],
                "hs3d_pmesh_residual": [vp, C.POINTER(SolverCfg), vp, vp, vp],
                "hs3d_pmesh_run": [vp, C.POINTER(SolverCfg), vp, vp, d, i, vp],
                "hs3d_pmesh_clock": [vp, C.POINTER(d), C.POINTER(C.c_int64), i, vp],
                "hs3d_pmesh_diagnostics": [vp, C.POINTER(SolverCfg), vp, vp, vp, vp],
                "hs3d_last_error": [],
                "hs3d_version": [],
            }
            for name, args in sig.items():
                f = getattr(L, name)
                f.argtypes = args
                f.restype = C.c_int
            L.hs3d_mesh_destroy.restype = None
            L.hs3d_pmesh_destroy.restype = None
            L.hs3d_server_destroy.restype = None
            L.hs3d_last_error.restype = C.c_char_p
            L.hs3d_version.restype = C.c_char_p
            _lib = L
    return _lib


def check(status):
    if status not in (OK, PENDING):
        raise HS3DError(status, lib().hs3d_last_error().decode())
    return status


def _stream(stream=None):
    if stream is not None:
        return C.c_void_p(stream if isinstance(stream, int) else stream.cuda_stream)
    import torch
    return C.c_void_p(torch.cuda.current_stream().cuda_stream)


def _ptr(t, name="tensor"):
    import torch
    if t is None:
        return None
    if not (t.is_cuda and t.dtype == torch.float64 and t.is_contiguous()):
        raise HS3DError(ERR_INVALID, f"{name} must be a contiguous float64 CUDA tensor")
    return C.c_void_p(t.data_ptr())


def solver_cfg(physics="euler", surface="lf", volume="standard", precision="fp64", gamma=1.4, Re=1600.0,
               Pr=0.72, Ma=0.1, cfl=0.5, time="rk3") -> SolverCfg:
    return SolverCfg(PHYSICS[physics], SURFACE[surface], VOLUME[volume], PRECISION[precision],
                     gamma, Re, Pr, Ma, cfl, TIME[time])


def mesh_desc(ex, ey, ez, N, lo=(0.0, 0.0, 0.0), hi=(1.0, 1.0, 1.0), amp=0.0, node_xyz=None,
              nodes="lobatto") -> MeshDesc:
    return MeshDesc(ex, ey, ez, N, (C.c_double * 3)(*lo), (C.c_double * 3)(*hi), (C.c_int * 3)(1, 1, 1),
                    amp, node_xyz, NODES[nodes])


class Mesh:
    """A library-owned mesh on the current CUDA device (``hs3d_mesh_create``)."""

    def __init__(self, ex, ey, ez, N, lo=(0.0, 0.0, 0.0), hi=(1.0, 1.0, 1.0), amp=0.0, node_xyz=None,
                 nodes="lobatto"):
        self.ex, self.ey, self.ez, self.N = ex, ey, ez, N
        self.nodes = nodes
        self.n = N + 1
        self.E = ex * ey * ez
        self.lo, self.hi = tuple(lo), tuple(hi)
        keep = None
        xyz = None
        if node_xyz is not None:
            import numpy as np
            keep = np.ascontiguousarray(node_xyz, dtype=np.float64)
            xyz = keep.ctypes.data
        d = mesh_desc(ex, ey, ez, N, lo, hi, amp, xyz, nodes)
        h = C.c_void_p()
        check(lib().hs3d_mesh_create(C.byref(d), C.byref(h)))
        self._h = h
        del keep

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value:
            lib().hs3d_mesh_destroy(h)
            self._h = None

    @property
    def handle(self):
        return self._h

    @property
    def shape(self):
        return (self.E, 5, self.n, self.n, self.n)

    def info(self):
        E, N, b = C.c_int64(), C.c_int(), C.c_size_t()
        check(lib().hs3d_mesh_info(self._h, C.byref(E), C.byref(N), C.byref(b)))
        return E.value, N.value, b.value

    def empty_state(self):
        import torch
        return torch.empty(self.shape, dtype=torch.float64, device="cuda")

    def geometry(self, stream=None):
        import torch
        n = self.n
        X = torch.empty((self.E, 3, n, n, n), dtype=torch.float64, device="cuda")
        Ja = torch.empty((self.E, 3, 3, n, n, n), dtype=torch.float64, device="cuda")
        J = torch.empty((self.E, n, n, n), dtype=torch.float64, device="cuda")
        check(lib().hs3d_mesh_geometry(self._h, _ptr(X), _ptr(Ja), _ptr(J), _stream(stream)))
        return X, Ja, J

    def init_state(self, u, kind="vortex", gamma=1.4, Ma=0.5, beta=5.0, xc=None, yc=None, t=0.0, stream=None):
        if xc is None:
            xc = 0.5 * (self.lo[0] + self.hi[0])
        if yc is None:
            yc = 0.5 * (self.lo[1] + self.hi[1])
        ic = IC({"vortex": IC_VORTEX, "tgv": IC_TGV}[kind], gamma, Ma, beta, xc, yc, t)
        check(lib().hs3d_init_state(self._h, C.byref(ic), _ptr(u, "u"), _stream(stream)))
        return u

    def residual(self, cfg: SolverCfg, u, dudt, stream=None):
        check(lib().hs3d_residual(self._h, C.byref(cfg), _ptr(u, "u"), _ptr(dudt, "dudt"), _stream(stream)))
        return dudt

    def rk3_step(self, cfg: SolverCfg, u, g, dt=0.0, stream=None):
        check(lib().hs3d_rk3_step(self._h, C.byref(cfg), _ptr(u, "u"), _ptr(g, "g"), float(dt), _stream(stream)))

    def rk3_run(self, cfg: SolverCfg, u, g, nsteps, dt=0.0, stream=None):
        """nsteps RK steps (hs3d_rk3_run): dt > 0 fixed, dt == 0 from the
        CFL rule, dt < 0 continue the previous run of this same state."""
        check(lib().hs3d_rk3_run(self._h, C.byref(cfg), _ptr(u, "u"), _ptr(g, "g"), float(dt), int(nsteps),
                                 _stream(stream)))

    def rk3_step_profiled(self, cfg: SolverCfg, u, g, dt=0.0, stream=None):
        """One eager RK3 step with per-kernel event timing; returns
        {"dt": ms, "grad": ms, "face": ms, "volume": ms, "step": ms}."""
        ms = (C.c_double * 5)()
        check(lib().hs3d_rk3_step_profiled(self._h, C.byref(cfg), _ptr(u, "u"), _ptr(g, "g"), float(dt), ms,
                                           _stream(stream)))
        return dict(zip(("dt", "grad", "face", "volume", "step"), list(ms)))

    def dt(self, cfg: SolverCfg, u, out, stream=None):
        check(lib().hs3d_dt(self._h, C.byref(cfg), _ptr(u, "u"), _ptr(out, "dt_out"), _stream(stream)))
        return out

    def clock(self, reset=False, stream=None, check_state=True):
        """(simulated time, steps) of this mesh's clock; raises on a
        non-physical state unless check_state=False, which returns
        (time, steps, status) instead."""
        t, s = C.c_double(), C.c_int64()
        st = lib().hs3d_clock(self._h, C.byref(t), C.byref(s), int(reset), _stream(stream))
        if not check_state:
            return t.value, s.value, st
        check(st)
        return t.value, s.value

    def autotune(self, cfg: SolverCfg, stream=None):
        """Pick the fastest elements-per-CTA of the gradient and element
        kernels for this mesh and cfg; returns (gradient, element)."""
        ch = (C.c_int * 2)()
        check(lib().hs3d_autotune(self._h, C.byref(cfg), ch, _stream(stream)))
        return ch[0], ch[1]

    def diagnostics(self, cfg: SolverCfg, u, out, dudt=None, stream=None):
        check(lib().hs3d_diagnostics(self._h, C.byref(cfg), _ptr(u, "u"), _ptr(dudt, "dudt"), _ptr(out, "out"),
                                     _stream(stream)))
        return out


class PMesh:
    """A mesh whose elements carry their own polynomial degree, coupled by
    mortars (``hs3d_pmesh_create``, Sec. 3.6).  ``degrees``: one per element
    (shape (E,)), or one per element and reference direction (shape (E, 3):
    P_x, P_y, P_z, ``hs3d_pmesh_create3``).

    States are flat float64 CUDA tensors of ``size`` doubles; element e's
    block [5, n_z, n_y, n_x] starts at ``offset[e]`` (see
    ``hs3d_pmesh_layout``)."""

    def __init__(self, ex, ey, ez, degrees, lo=(0.0, 0.0, 0.0), hi=(1.0, 1.0, 1.0), amp=0.0):
        import numpy as np
        self.ex, self.ey, self.ez = ex, ey, ez
        self.E = ex * ey * ez
        dg = np.asarray(degrees, dtype=np.int32)
        if dg.ndim == 2:
            if dg.shape != (self.E, 3):
                raise HS3DError(ERR_INVALID, "three degrees per element")
            deg3 = np.ascontiguousarray(dg)
        else:
            if dg.size != self.E:
                raise HS3DError(ERR_INVALID, "one degree per element")
            deg3 = np.ascontiguousarray(np.repeat(dg.reshape(-1)[:, None], 3, axis=1))
        self.degrees3 = deg3.copy()
        self.degrees = deg3[:, 0].copy() if bool(np.all(deg3 == deg3[:, :1])) else None
        self.lo, self.hi = tuple(lo), tuple(hi)
        d = mesh_desc(ex, ey, ez, 1, lo, hi, amp)
        h = C.c_void_p()
        if dg.ndim == 2:
            check(lib().hs3d_pmesh_create3(C.byref(d), C.c_void_p(deg3.ctypes.data), C.byref(h)))
        else:
            deg = np.ascontiguousarray(dg.reshape(-1))
            check(lib().hs3d_pmesh_create(C.byref(d), C.c_void_p(deg.ctypes.data), C.byref(h)))
        self._h = h
        off = np.zeros(self.E + 1, dtype=np.int64)
        ng = C.c_int()
        check(lib().hs3d_pmesh_layout(h, C.c_void_p(off.ctypes.data), C.byref(ng)))
        self.offset = off
        self.size = int(off[-1])
        self.Ngeo = ng.value

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value:
            lib().hs3d_pmesh_destroy(h)
            self._h = None

    def n(self, e):
        """Nodes per direction of an element of equal degrees."""
        nx, ny, nz = self.shape3(e)
        if not nx == ny == nz:
            raise HS3DError(ERR_INVALID, "element with per-direction degrees: use shape3")
        return nx

    def shape3(self, e):
        """(n_x, n_y, n_z) of element e."""
        return tuple(int(x) + 1 for x in self.degrees3[e])

    def empty_state(self):
        import torch
        return torch.zeros(self.size, dtype=torch.float64, device="cuda")

    def block(self, u, e):
        """View of element e's block [5, n_z, n_y, n_x] of a flat state (tensor or array)."""
        nx, ny, nz = self.shape3(e)
        o = int(self.offset[e])
        return u[o:o + 5 * nx * ny * nz].reshape(5, nz, ny, nx)

    def geometry(self, stream=None):
        """(X, J) as flat tensors: element e's X [3, n^3] at 3 offset[e]/5, J [n^3] at offset[e]/5."""
        import torch
        X = torch.zeros(3 * self.size // 5, dtype=torch.float64, device="cuda")
        J = torch.zeros(self.size // 5, dtype=torch.float64, device="cuda")
        check(lib().hs3d_pmesh_geometry(self._h, _ptr(X), _ptr(J), _stream(stream)))
        return X, J

    def init_state(self, u, kind="tgv", gamma=1.4, Ma=0.1, beta=5.0, xc=None, yc=None, t=0.0, stream=None):
        if xc is None:
            xc = 0.5 * (self.lo[0] + self.hi[0])
        if yc is None:
            yc = 0.5 * (self.lo[1] + self.hi[1])
        ic = IC({"vortex": IC_VORTEX, "tgv": IC_TGV}[kind], gamma, Ma, beta, xc, yc, t)
        check(lib().hs3d_pmesh_init_state(self._h, C.byref(ic), _ptr(u, "u"), _stream(stream)))
        return u

    def residual(self, cfg: SolverCfg, u, dudt, stream=None):
        check(lib().hs3d_pmesh_residual(self._h, C.byref(cfg), _ptr(u, "u"), _ptr(dudt, "dudt"), _stream(stream)))
        return dudt

    def run(self, cfg: SolverCfg, u, g, nsteps, dt=0.0, stream=None):
        """nsteps RK steps (hs3d_pmesh_run): dt > 0 fixed, dt == 0 the CFL rule,
        dt < 0 continue the previous run of this same state."""
        check(lib().hs3d_pmesh_run(self._h, C.byref(cfg), _ptr(u, "u"), _ptr(g, "g"), float(dt), int(nsteps),
                                   _stream(stream)))

    def diagnostics(self, cfg: SolverCfg, u, out, dudt=None, stream=None):
        """hs3d_pmesh_diagnostics into out (7 float64 on the device)."""
        check(lib().hs3d_pmesh_diagnostics(self._h, C.byref(cfg), _ptr(u, "u"), _ptr(dudt, "dudt"),
                                           _ptr(out, "out"), _stream(stream)))
        return out

    def clock(self, reset=False, stream=None):
        t, s = C.c_double(), C.c_int64()
        check(lib().hs3d_pmesh_clock(self._h, C.byref(t), C.byref(s), int(reset), _stream(stream)))
        return t.value, s.value


class Server:
    """Continuous-batching solve server (hs3d_server_create / hs3d_submit / hs3d_poll)."""

    def __init__(self, hbm_budget_bytes=0, max_batch=0, launch_mode="grid"):
        h = C.c_void_p()
        check(lib().hs3d_server_create(int(hbm_budget_bytes), int(max_batch), C.byref(h)))
        self._h = h
        self._keep = {}
        if launch_mode != "grid":
            self.set_launch_mode(launch_mode)

    def set_launch_mode(self, mode):
        """"grid" (a CTA per tile, binary search for the request) or
        "persistent" (work table + persistent grids); hs3d_server_set_launch_mode."""
        check(lib().hs3d_server_set_launch_mode(self._h, {"grid": 0, "persistent": 1}[mode]))

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            lib().hs3d_server_destroy(self._h)
            self._h = None

    def __del__(self):
        self.close()

    def submit(self, mesh: MeshDesc, cfg: SolverCfg, ic: IC, t_final=0.0, n_steps=0, result=None):
        """Queue a solve; `result` (a C-contiguous float64 numpy array of
        E*5*n^3 values) receives the final state.  Returns the ticket."""
        ptr = None
        if result is not None:
            if not (result.flags["C_CONTIGUOUS"] and result.dtype.name == "float64"):
                raise HS3DError(ERR_INVALID, "result must be a C-contiguous float64 array")
            ptr = result.ctypes.data
        req = Request(mesh, cfg, ic, float(t_final), int(n_steps), ptr)
        t = C.c_uint64()
        check(lib().hs3d_submit(self._h, C.byref(req), C.byref(t)))
        self._keep[t.value] = result
        return t.value

    def poll(self, ticket):
        """(status, Result): status is PENDING, OK or the request's error code."""
        res = Result()
        st = lib().hs3d_poll(self._h, C.c_uint64(ticket), C.byref(res))
        if st != PENDING:
            self._keep.pop(ticket, None)
        return st, res

    def stats(self):
        q, r, f, b = C.c_int64(), C.c_int64(), C.c_int64(), C.c_size_t()
        check(lib().hs3d_server_stats(self._h, C.byref(q), C.byref(r), C.byref(f), C.byref(b)))
        return {"queued": q.value, "running": r.value, "finished": f.value, "bytes_in_use": b.value}


def diagnostics_noalloc(N, E, gamma, J, u, out, dudt=None, nodes="lobatto", stream=None):
    """hs3d_diagnostics_noalloc: the quadrature diagnostics with no device
    allocation (for callers that cannot allocate; see include/hs3d.h);
    `nodes` names the solution nodes of the mesh J and u belong to."""
    check(lib().hs3d_diagnostics_noalloc(int(N), int(E), float(gamma), NODES[nodes], _ptr(J, "J"), _ptr(u, "u"),
                                         _ptr(dudt, "dudt"), _ptr(out, "out"), _stream(stream)))
    return out


def check_rounding(x, stream=None):
    """Counts from hs3d_check_rounding for a float64 CUDA tensor x:
    (d2f mismatches, widening mismatches, inputs below the FP32 normal range,
    float-float split low-part mismatches)."""
    import torch
    counts = torch.zeros(4, dtype=torch.int64, device=x.device)
    check(lib().hs3d_check_rounding(_ptr(x, "x"), x.numel(), C.c_void_p(counts.data_ptr()), _stream(stream)))
    torch.cuda.synchronize()
    return tuple(int(v) for v in counts.cpu())


def ic_desc(kind="vortex", gamma=1.4, Ma=0.5, beta=5.0, xc=5.0, yc=5.0, t=0.0) -> IC:
    return IC({"vortex": IC_VORTEX, "tgv": IC_TGV}[kind], gamma, Ma, beta, xc, yc, t)


def alu_peaks(stream=None):
    """Measured FP64 and FP32 FMA throughput in TFLOP/s (hs3d_alu_peaks)."""
    out = (C.c_double * 2)()
    check(lib().hs3d_alu_peaks(out, _stream(stream)))
    return {"fp64_tflops": out[0], "fp32_tflops": out[1]}


def version() -> str:
    return lib().hs3d_version().decode()
