"""ctypes binding of libsexpe.so (argument marshalling only).

Every computation runs in the library: the FP64 setup on the host inside the
library, every step in its CUDA kernels.  There is no Python or CPU fallback:
if the library is missing, ``lib()`` raises.

Device arrays are passed as torch CUDA tensors (``data_ptr()``) on the current
torch stream, or as raw integer device pointers; the library never sees torch
types.
"""
import ctypes
import os
import re

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "lib", "libsexpe.so")
HEADER = os.path.join(os.path.dirname(_HERE), "include", "sexpe.h")

GEOMETRY = {"disk": 0, "sphere": 1, "ball": 2, "cylinder": 3}
PRECISION = {"fp64": 0, "split_tf32": 1, "unsplit_fp64": 2}
REACTION = {"none": 0, "schnakenberg": 1, "gray_scott": 2, "linear_cubic": 3, "bvam": 4, "bvam_manufactured": 5,
            "linear": 6}
ZBC = {"neumann": 0, "paper": 1}
AXIS = {"theta": 0, "rho2": 1, "rho3": 2, "phi": 3, "z_neumann": 4, "z_paper": 5}
STATUS = {0: "SEXPE_OK", 1: "SEXPE_EINVAL", 2: "SEXPE_ENOMEM", 3: "SEXPE_ECUDA", 4: "SEXPE_ETIMEOUT",
          5: "SEXPE_EUNSUPPORTED", 6: "SEXPE_ENUMERIC"}


class SexpeError(RuntimeError):
    def __init__(self, status, where):
        self.status = status
        super().__init__(f"{where}: {STATUS.get(status, status)} ({_lib.sexpe_status_string(status).decode()})")


class Grid(ctypes.Structure):
    _fields_ = [("geometry", ctypes.c_int32), ("n", ctypes.c_int32 * 3), ("rho_star", ctypes.c_double),
                ("z_star", ctypes.c_double), ("z_bc", ctypes.c_int32), ("rho_op", ctypes.c_int32),
                ("lam", ctypes.c_double)]


class Species(ctypes.Structure):
    _fields_ = [("n_species", ctypes.c_int32), ("d_host", ctypes.POINTER(ctypes.c_double)),
                ("reaction", ctypes.c_int32), ("n_params", ctypes.c_int32),
                ("params_host", ctypes.POINTER(ctypes.c_double)), ("offset_host", ctypes.POINTER(ctypes.c_double))]


COUPLING = {"schnakenberg_ball": 0, "dib_cylinder": 1}


class Coupling(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("zeta", ctypes.c_double * 5), ("eta", ctypes.c_double * 5),
                ("alpha3", ctypes.c_double), ("beta3", ctypes.c_double), ("u_top", ctypes.c_double),
                ("v_top", ctypes.c_double)]


def _coupling_struct(c):
    """c: dict with 'kind' (default 'schnakenberg_ball'), zeta1..zeta5, eta1..eta5 (missing ones 0),
    alpha3, beta3, u_top, v_top."""
    z = [float(c.get(f"zeta{q}", 0.0)) for q in range(1, 6)]
    e = [float(c.get(f"eta{q}", 0.0)) for q in range(1, 6)]
    return Coupling(COUPLING[c.get("kind", "schnakenberg_ball")], (ctypes.c_double * 5)(*z),
                    (ctypes.c_double * 5)(*e), float(c.get("alpha3", 0.0)), float(c.get("beta3", 0.0)),
                    float(c.get("u_top", 0.0)), float(c.get("v_top", 0.0)))


class PlanInfo(ctypes.Structure):
    _fields_ = [("geometry", ctypes.c_int32), ("precision", ctypes.c_int32), ("n_species", ctypes.c_int32),
                ("ndim", ctypes.c_int32), ("n", ctypes.c_int32 * 3), ("n_instances", ctypes.c_int32),
                ("kernels_per_step", ctypes.c_int32), ("npts", ctypes.c_int64), ("state_elems", ctypes.c_int64),
                ("workspace_bytes", ctypes.c_int64), ("setup_ms", ctypes.c_double),
                ("stencil_tile_j", ctypes.c_int32), ("ring_slots", ctypes.c_int32 * 2),
                ("stencil_tile_us", ctypes.c_float), ("stencil_planes", ctypes.c_int32),
                ("stencil_ctas_per_sm", ctypes.c_int32), ("theta_split", ctypes.c_int32),
                ("batch_order", ctypes.c_int32), ("batch_step_us", ctypes.c_float)]


_lib = None
_P = ctypes.c_void_p
_DP = ctypes.POINTER(ctypes.c_double)


def lib():
    """Open libsexpe.so (built in-tree by __graft_entry__.build()); raise if it is missing."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is not built; run __graft_entry__.build()")
        L = ctypes.CDLL(LIB_PATH)
        L.sexpe_status_string.restype = ctypes.c_char_p
        L.sexpe_status_string.argtypes = [ctypes.c_int32]
        L.sexpe_setup.argtypes = [ctypes.POINTER(Grid), ctypes.POINTER(Species), ctypes.c_double, ctypes.c_int32,
                                  _P, ctypes.POINTER(_P)]
        L.sexpe_batch_setup.argtypes = [ctypes.c_int32, ctypes.POINTER(Grid), ctypes.POINTER(Species),
                                        ctypes.c_double, ctypes.c_int32, _P, ctypes.POINTER(_P)]
        L.sexpe_coupled_setup.argtypes = [ctypes.POINTER(Grid), ctypes.POINTER(Species), ctypes.POINTER(Species),
                                          ctypes.POINTER(Coupling), ctypes.c_double, ctypes.c_int32, _P,
                                          ctypes.POINTER(_P)]
        L.sexpe_coupling_terms.argtypes = [ctypes.POINTER(Grid), ctypes.POINTER(Species), ctypes.POINTER(Coupling),
                                           ctypes.c_int64] + [_DP] * 8
        L.sexpe_state_offsets.argtypes = [_P, ctypes.POINTER(ctypes.c_int64)]
        L.sexpe_step.argtypes = [_P, _P, ctypes.c_int64, _P]
        L.sexpe_step_host.argtypes = [_P, _DP, ctypes.c_int64, _P]
        L.sexpe_step_noalloc.argtypes = [_P, _P, ctypes.c_int64, _P]
        L.sexpe_synchronize.argtypes = [_P, _P]
        L.sexpe_plan_get_info.argtypes = [_P, ctypes.POINTER(PlanInfo)]
        L.sexpe_set_stencil.argtypes = [_P, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32]
        L.sexpe_set_theta_split.argtypes = [_P, ctypes.c_int32]
        L.sexpe_selftest_wait_timeout.argtypes = [_P]
        L.sexpe_set_time.argtypes = [_P, ctypes.c_double, _P]
        L.sexpe_destroy.argtypes = [_P]
        L.sexpe_step_checkpointed.argtypes = [_P, _P, ctypes.c_int64, ctypes.c_int32, _P, _P]
        L.sexpe_adjoint.argtypes = [_P, _P, ctypes.c_int32, ctypes.c_int32, _P, _P, _DP, _P]
        L.sexpe_profile_begin.argtypes = [_P, ctypes.c_int32]
        L.sexpe_profile_end.argtypes = [_P, _DP, ctypes.POINTER(ctypes.c_int32), ctypes.c_int32]
        L.sexpe_axis_matrix.argtypes = [ctypes.c_int32, ctypes.c_int32, ctypes.c_double, _DP]
        L.sexpe_axis_phi1.argtypes = [ctypes.c_int32, ctypes.c_int32, ctypes.c_double, ctypes.c_double, _DP]
        L.sexpe_axis_eigen.argtypes = [ctypes.c_int32, ctypes.c_int32, ctypes.c_double, _DP, _DP, _DP]
        for name in ["sexpe_setup", "sexpe_batch_setup", "sexpe_state_offsets", "sexpe_step", "sexpe_step_host",
                     "sexpe_synchronize", "sexpe_plan_get_info", "sexpe_destroy", "sexpe_axis_matrix",
                     "sexpe_profile_begin", "sexpe_profile_end", "sexpe_step_noalloc",
                     "sexpe_step_checkpointed", "sexpe_adjoint", "sexpe_set_stencil",
                     "sexpe_set_theta_split", "sexpe_selftest_wait_timeout", "sexpe_set_time",
                     "sexpe_axis_phi1", "sexpe_axis_eigen", "sexpe_coupled_setup",
                     "sexpe_coupling_terms"]:
            getattr(L, name).restype = ctypes.c_int32
        _lib = L
    return _lib


def header_functions():
    """Names of the functions include/sexpe.h declares."""
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(sexpe_\w+)\s*\(", text)))


def selftest_wait_timeout(stream=None):
    """sexpe_selftest_wait_timeout: returns the status (SEXPE_ETIMEOUT = 4 when the bounded wait
    gave up and reported as designed)."""
    return int(lib().sexpe_selftest_wait_timeout(_stream_ptr(stream)))


def _check(status, where):
    if status != 0:
        raise SexpeError(status, where)


def _dptr(x):
    return ctypes.cast(np.ascontiguousarray(x, dtype=np.float64).ctypes.data, _DP)


def _stream_ptr(stream):
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def _data_ptr(x):
    if isinstance(x, int):
        return x
    import torch
    if not (isinstance(x, torch.Tensor) and x.is_cuda and x.dtype == torch.float64 and x.is_contiguous()):
        raise TypeError("state must be a contiguous CUDA float64 tensor or a device pointer")
    return x.data_ptr()


def _grid_struct(geometry, n, rho_star=1.0, z_star=1.0, z_bc="neumann"):
    nn = list(n) + [1] * (3 - len(n))
    return Grid(GEOMETRY[geometry], (ctypes.c_int32 * 3)(*nn), float(rho_star), float(z_star), ZBC[z_bc])


class Plan:
    """A plan of the split exponential Euler step (wraps sexpe_setup / sexpe_batch_setup)."""

    def __init__(self, geometry, n, d, reaction="none", params=(), tau=1e-3, precision="split_tf32",
                 rho_star=1.0, z_star=1.0, z_bc="neumann", stream=None, lam=None, offsets=None):
        """lam: exponent of the anomalous operator Delta_lambda on the disk (Dirichlet at rho_*);
        offsets: per-species lifting constants the reactions add to the state."""
        L = lib()
        self._d = np.ascontiguousarray(d, dtype=np.float64)
        self._p = np.ascontiguousarray(params if len(params) else [0.0], dtype=np.float64)
        grid = _grid_struct(geometry, n, rho_star, z_star, z_bc)
        if lam is not None:
            grid.rho_op, grid.lam = 1, float(lam)
        self._off = None if offsets is None else np.ascontiguousarray(offsets, dtype=np.float64)
        sp = Species(len(self._d), _dptr(self._d), REACTION[reaction], len(params), _dptr(self._p),
                     None if self._off is None else _dptr(self._off))
        h = _P()
        st = _stream_ptr(stream) if stream is not None else 0
        _check(L.sexpe_setup(ctypes.byref(grid), ctypes.byref(sp), float(tau), PRECISION[precision], st,
                             ctypes.byref(h)), "sexpe_setup")
        self.handle = h
        self.geometry, self.n, self.S = geometry, tuple(n), len(self._d)
        self._p_list = list(params)

    @classmethod
    def from_workload(cls, w, precision="split_tf32", stream=None):
        return cls(w["geometry"], w["n"], w["d"], w["reaction"], w["params"], w["tau"], precision,
                   stream=stream, lam=w.get("lam"), offsets=w.get("offsets"))

    def info(self):
        inf = PlanInfo()
        _check(lib().sexpe_plan_get_info(self.handle, ctypes.byref(inf)), "sexpe_plan_get_info")
        return {f: (list(getattr(inf, f)) if f in ("n", "ring_slots") else getattr(inf, f)) for f, _ in PlanInfo._fields_}

    def set_time(self, t, stream=None):
        """sexpe_set_time: time of the next step (plans with time-dependent sources)."""
        _check(lib().sexpe_set_time(self.handle, float(t), _stream_ptr(stream)), "sexpe_set_time")

    def set_stencil(self, tile_j, planes=0, ctas_per_sm=1):
        """sexpe_set_stencil: override the measured stencil configuration."""
        _check(lib().sexpe_set_stencil(self.handle, int(tile_j), int(planes), int(ctas_per_sm)), "sexpe_set_stencil")

    def set_theta_split(self, split):
        """sexpe_set_theta_split: override the measured theta-kernel column split of a sphere plan."""
        _check(lib().sexpe_set_theta_split(self.handle, int(split)), "sexpe_set_theta_split")

    def step(self, state, n_steps, stream=None):
        _check(lib().sexpe_step(self.handle, _data_ptr(state), int(n_steps), _stream_ptr(stream)), "sexpe_step")

    def step_noalloc(self, state, n_steps, stream=None):
        """sexpe_step_noalloc: the split-TF32 step with scratch in the library's static device array."""
        _check(lib().sexpe_step_noalloc(self.handle, _data_ptr(state), int(n_steps), _stream_ptr(stream)),
               "sexpe_step_noalloc")

    def step_host(self, state_host, n_steps, stream=None):
        """state_host: C-contiguous float64 numpy array (or pinned CPU tensor), updated in place."""
        if hasattr(state_host, "data_ptr"):
            ptr = ctypes.cast(state_host.data_ptr(), _DP)
        else:
            assert state_host.dtype == np.float64 and state_host.flags["C_CONTIGUOUS"]
            ptr = ctypes.cast(state_host.ctypes.data, _DP)
        _check(lib().sexpe_step_host(self.handle, ptr, int(n_steps), _stream_ptr(stream)), "sexpe_step_host")

    def synchronize(self, stream=None):
        _check(lib().sexpe_synchronize(self.handle, _stream_ptr(stream)), "sexpe_synchronize")

    def step_checkpointed(self, state, n_steps, every, checkpoints, stream=None):
        """Advance `state` n_steps steps, storing the state before every `every`-th step in `checkpoints`
        (a CUDA float64 tensor of ceil(n_steps/every) states)."""
        _check(lib().sexpe_step_checkpointed(self.handle, _data_ptr(state), int(n_steps), int(every),
                                             _data_ptr(checkpoints), _stream_ptr(stream)), "sexpe_step_checkpointed")

    def adjoint(self, checkpoints, n_ckpt, every, dL_dWT, dL_dW0, stream=None):
        """sexpe_adjoint: writes dL/dW0 into dL_dW0 and returns the parameter gradient
        (reaction parameters, then the diffusion of every species) as a numpy array."""
        out = np.zeros(len(self._p_list) + self.S)
        _check(lib().sexpe_adjoint(self.handle, _data_ptr(checkpoints), int(n_ckpt), int(every), _data_ptr(dL_dWT),
                                   _data_ptr(dL_dW0), _dptr_out(out), _stream_ptr(stream)), "sexpe_adjoint")
        return out

    def profile_begin(self, max_steps):
        _check(lib().sexpe_profile_begin(self.handle, int(max_steps)), "sexpe_profile_begin")

    def profile_end(self):
        """Average duration (ms) of each kernel slot of a step over the profiled steps."""
        out = np.zeros(16)
        n = ctypes.c_int32(0)
        _check(lib().sexpe_profile_end(self.handle, _dptr_out(out), ctypes.byref(n), 16), "sexpe_profile_end")
        return out[:n.value].tolist()

    def close(self):
        if getattr(self, "handle", None):
            lib().sexpe_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class BatchPlan(Plan):
    """Many independent disks stepped together (wraps sexpe_batch_setup).

    `workloads` is a list of workload dicts (disk, 2 species); the state is the
    concatenation of the instances' states (see offsets())."""

    def __init__(self, workloads, precision="split_tf32", stream=None):
        L = lib()
        count = len(workloads)
        grids = (Grid * count)()
        specs = (Species * count)()
        self._keep = []
        for q, w in enumerate(workloads):
            grids[q] = _grid_struct(w["geometry"], w["n"], w.get("rho_star", 1.0))
            d = np.ascontiguousarray(w["d"], dtype=np.float64)
            prm = np.ascontiguousarray(w["params"] if len(w["params"]) else [0.0], dtype=np.float64)
            self._keep += [d, prm]
            specs[q] = Species(len(d), _dptr(d), REACTION[w["reaction"]], len(w["params"]), _dptr(prm))
        h = _P()
        st = _stream_ptr(stream) if stream is not None else 0
        _check(L.sexpe_batch_setup(count, grids, specs, float(workloads[0]["tau"]), PRECISION[precision], st,
                                   ctypes.byref(h)), "sexpe_batch_setup")
        self.handle = h
        self.geometry, self.n, self.S = "disk", None, 2
        self._p_list = []
        self.count = count

    def offsets(self):
        out = (ctypes.c_int64 * (self.count + 1))()
        _check(lib().sexpe_state_offsets(self.handle, out), "sexpe_state_offsets")
        return list(out)


class CoupledPlan(Plan):
    """A bulk-surface coupled plan (wraps sexpe_coupled_setup).  Section 5.5: the ball
    n = (n_rho, n_theta, n_phi) and its boundary sphere, state [u][v] (ball layout) then [r][s] (sphere
    layout, theta fastest).  Section 5.6 (coupling kind 'dib_cylinder', geometry 'cylinder'): the
    cylinder n = (n_rho, n_theta, n_z) with the Dirichlet top of eq. A_z, its state lifted by
    (u_top, v_top), and the bottom disk, state [w_u][w_v] (cylinder layout) then [r][s] (disk layout)."""

    def __init__(self, n, d_bulk, bulk_params, d_surface, surface_params, coupling, tau, rho_star=1.0,
                 precision="fp64", stream=None, reaction="schnakenberg", surface_reaction=None,
                 geometry="ball", z_star=1.0, z_bc=None):
        L = lib()
        self._keep = [np.ascontiguousarray(x if len(x) else [0.0], dtype=np.float64)
                      for x in (d_bulk, bulk_params, d_surface, surface_params)]
        db, pb, ds, ps = self._keep
        if z_bc is None:
            z_bc = "paper" if geometry == "cylinder" else "neumann"
        grid = _grid_struct(geometry, n, rho_star, z_star, z_bc)
        srx = reaction if surface_reaction is None else surface_reaction
        bulk = Species(len(d_bulk), _dptr(db), REACTION[reaction], len(bulk_params), _dptr(pb))
        surf = Species(len(d_surface), _dptr(ds), REACTION[srx], len(surface_params), _dptr(ps))
        cp = _coupling_struct(coupling)
        h = _P()
        st = _stream_ptr(stream) if stream is not None else 0
        _check(L.sexpe_coupled_setup(ctypes.byref(grid), ctypes.byref(bulk), ctypes.byref(surf), ctypes.byref(cp),
                                     float(tau), PRECISION[precision], st, ctypes.byref(h)), "sexpe_coupled_setup")
        self.handle = h
        self.geometry, self.n, self.S = geometry + "+surface", tuple(n), len(d_bulk) + len(d_surface)
        self._p_list = []
        self.n_bulk = int(np.prod(n))
        self.n_surface = int(n[1]) * int(n[2]) if geometry == "ball" else int(n[0]) * int(n[1])


def coupling_terms(geometry, n, d_bulk, coupling, ub, vb, r, s, rho_star=1.0, z_star=1.0):
    """sexpe_coupling_terms: the additions to the bulk F (boundary node) and to the surface F at each
    of len(ub) surface points, as four numpy arrays (host evaluation, no GPU)."""
    L = lib()
    d = np.ascontiguousarray(d_bulk, dtype=np.float64)
    grid = _grid_struct(geometry, n, rho_star, z_star, "paper" if geometry == "cylinder" else "neumann")
    sp = Species(len(d), _dptr(d), REACTION["none"], 0, None)
    cp = _coupling_struct(coupling)
    ins = [np.ascontiguousarray(x, dtype=np.float64).ravel() for x in (ub, vb, r, s)]
    outs = [np.zeros_like(ins[0]) for _ in range(4)]
    _check(L.sexpe_coupling_terms(ctypes.byref(grid), ctypes.byref(sp), ctypes.byref(cp), len(ins[0]),
                                  *[_dptr(x) for x in ins], *[_dptr_out(x) for x in outs]), "sexpe_coupling_terms")
    return outs


def coupled_setup_status(*args, **kw):
    """Status code of sexpe_coupled_setup for the given arguments (the plan is destroyed again)."""
    try:
        p = CoupledPlan(*args, **kw)
    except SexpeError as e:
        return e.status
    p.close()
    return 0


def batch_setup_status(workloads, precision="split_tf32"):
    try:
        p = BatchPlan(workloads, precision)
    except SexpeError as e:
        return e.status
    p.close()
    return 0


def setup_status(geometry, n, d, reaction="none", params=(), tau=1e-3, precision="split_tf32", **kw):
    """Status code of sexpe_setup for the given arguments (the plan is destroyed again)."""
    try:
        p = Plan(geometry, n, d, reaction, params, tau, precision, **kw)
    except SexpeError as e:
        return e.status
    p.close()
    return 0


def axis_matrix(axis, n, extent=1.0):
    out = np.zeros((n, n))
    _check(lib().sexpe_axis_matrix(AXIS[axis], n, extent, _dptr_out(out)), "sexpe_axis_matrix")
    return out


def axis_phi1(axis, n, t, extent=1.0):
    out = np.zeros((n, n))
    _check(lib().sexpe_axis_phi1(AXIS[axis], n, extent, t, _dptr_out(out)), "sexpe_axis_phi1")
    return out


def axis_eigen(axis, n, extent=1.0):
    lam, V, Vinv = np.zeros(n), np.zeros((n, n)), np.zeros((n, n))
    _check(lib().sexpe_axis_eigen(AXIS[axis], n, extent, _dptr_out(lam), _dptr_out(V), _dptr_out(Vinv)),
           "sexpe_axis_eigen")
    return lam, V, Vinv


def _dptr_out(a):
    assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]
    return ctypes.cast(a.ctypes.data, _DP)


def _autograd_function():
    import torch

    class SplitEulerEvolve(torch.autograd.Function):
        """W_N = (n_steps split exponential Euler steps)(W_0) with the library's
        checkpointed forward and discrete adjoint.  `params` is a CPU float64
        tensor holding the values the plan was built with (reaction parameters,
        then the diffusion coefficients); its gradient is the adjoint's
        parameter gradient.  FP64 plans, and split-TF32 sphere plans."""

        @staticmethod
        def forward(ctx, W0, params, plan, n_steps, every):
            n_ckpt = -(-n_steps // every)
            ckpt = torch.empty((n_ckpt,) + tuple(W0.shape), dtype=torch.float64, device=W0.device)
            W = W0.detach().clone().contiguous()
            plan.step_checkpointed(W, n_steps, every, ckpt)
            ctx.plan, ctx.every, ctx.n_ckpt = plan, every, n_ckpt
            ctx.save_for_backward(ckpt)
            if n_steps != n_ckpt * every:
                raise ValueError("n_steps must be a multiple of every")
            return W

        @staticmethod
        def backward(ctx, gW):
            (ckpt,) = ctx.saved_tensors
            g0 = torch.empty_like(gW)
            gp = ctx.plan.adjoint(ckpt, ctx.n_ckpt, ctx.every, gW.contiguous(), g0)
            return g0, torch.from_numpy(gp), None, None, None

    return SplitEulerEvolve


def evolve(plan, W0, params, n_steps, every):
    """Differentiable n_steps-step evolution (see SplitEulerEvolve)."""
    return _autograd_function().apply(W0, params, plan, n_steps, every)
