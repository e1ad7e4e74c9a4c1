"""Python binding of libalbm.so (argument marshalling only).

Every step of the method runs in the library's CUDA kernels; this module
only converts a :class:`~paper_1501_04741_gb300.inputs.Problem` into the C
``lbm_params`` struct, passes pointers of torch tensors (device) or numpy
arrays (host) and the current torch CUDA stream, and turns status codes into
exceptions.  Importing it loads the library and raises when it is missing;
there is no fallback path.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from .inputs import Problem

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "lib", "libalbm.so")

LATTICE = {"D2Q9": 0, "D3Q19": 1}
COLLISION = {"BGK": 0, "MRT": 1}
PRECISION = {"fp32": 0, "bf16": 1, "fp16": 2}
POROSITY = {"linear": 0, "power": 1, "ramp": 2}
OBJECTIVE = {"none": 0, "dissipation": 1, "variance": 2, "heatflux_dp": 3, "mixflux": 4,
             "heatflux": 5}
SCALAR_INLET = {"zero": 0, "halves": 1, "signed": 2}
KERNEL = {"auto": 0, "plain": 1, "tiles": 2, "async": 3}
ADJOINT_MODE = {"unsteady": 0, "frozen": 1}
INLET = {"velocity": 0, "pressure": 1}
STATUS = {0: "LBM_OK", 1: "LBM_ERR_ARG", 2: "LBM_ERR_OOM", 3: "LBM_ERR_CUDA",
          4: "LBM_ERR_NONFINITE", 5: "LBM_ERR_TIMEOUT", 6: "LBM_ERR_STATE"}

# symbols declared in include/albm.h
EXPORTS = ["lbm_create", "lbm_destroy", "lbm_last_error", "lbm_set_theta", "lbm_reset",
           "lbm_primal_step", "lbm_time", "lbm_objective", "lbm_adjoint_step",
           "lbm_adjoint_seed", "lbm_adjoint_time", "lbm_run", "lbm_gradient",
           "lbm_get_populations", "lbm_get_populations_at", "lbm_set_populations", "lbm_get_adjoint", "lbm_get_flags",
           "lbm_check_finite", "lbm_sizes", "lbm_last_timing", "lbm_profile",
           "lbm_profile_read", "lbm_recompute_steps", "lbm_batch_primal_step",
           "lbm_batch_adjoint_step", "lbm_set_design", "lbm_oneshot_reset",
           "lbm_oneshot_step", "lbm_oneshot_eval", "lbm_threshold_scan",
           "lbm_threshold_apply", "lbm_get_theta", "lbm_mma_reset", "lbm_mma_update",
           "lbm_mma_update_with", "lbm_state_objective_noalloc",
           "lbm_noalloc_last_error", "lbm_set_stream", "lbm_batch_primal_steps",
           "lbm_batch_adjoint_steps", "lbm_set_wait_polls"]


class LbmParams(C.Structure):
    _fields_ = [
        ("lattice", C.c_int), ("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int),
        ("collision", C.c_int), ("tau", C.c_double), ("s_other", C.c_double),
        ("force", C.c_double * 3), ("walls", C.c_int), ("inlet_outlet", C.c_int),
        ("u_in", C.c_double), ("rho_out", C.c_double), ("nscalars", C.c_int),
        ("alpha_fluid", C.c_double), ("alpha_solid", C.c_double), ("scalar_inlet", C.c_int),
        ("hot", C.c_int * 4), ("T_hot", C.c_double), ("porosity", C.c_int),
        ("porosity_q", C.c_double), ("objective", C.c_int), ("obj_window", C.c_int),
        ("nsteps", C.c_int), ("precision", C.c_int), ("ckpt_every", C.c_int),
        ("mem_budget", C.c_double), ("kernel", C.c_int), ("adjoint_mode", C.c_int),
        ("inlet_kind", C.c_int), ("dp", C.c_double),
    ]


class AlbmError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{STATUS.get(code, code)}: {msg}")
        self.code = code


_lib = None


def lib():
    """Load libalbm.so once (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"libalbm.so not built ({LIB_PATH}); run "
                               "`python -m paper_1501_04741_gb300.build`")
        L = C.CDLL(LIB_PATH)
        vp, i, d = C.c_void_p, C.c_int, C.c_double
        L.lbm_create.argtypes = [C.POINTER(vp), C.POINTER(LbmParams), vp, vp, vp]
        L.lbm_destroy.argtypes = [vp]
        L.lbm_destroy.restype = None
        L.lbm_last_error.argtypes = [vp]
        L.lbm_last_error.restype = C.c_char_p
        for name in ("lbm_set_theta", "lbm_adjoint_seed", "lbm_set_populations"):
            getattr(L, name).argtypes = [vp, vp]
        for name in ("lbm_reset", "lbm_run"):
            getattr(L, name).argtypes = [vp]
        for name in ("lbm_primal_step", "lbm_adjoint_step", "lbm_profile"):
            getattr(L, name).argtypes = [vp, i]
        L.lbm_time.argtypes = [vp]
        L.lbm_adjoint_time.argtypes = [vp]
        L.lbm_objective.argtypes = [vp, C.POINTER(d)]
        L.lbm_gradient.argtypes = [vp, vp]
        L.lbm_get_populations.argtypes = [vp, vp, i]
        L.lbm_get_populations_at.argtypes = [vp, i, vp, i]
        L.lbm_get_adjoint.argtypes = [vp, vp]
        L.lbm_get_flags.argtypes = [vp, vp]
        L.lbm_check_finite.argtypes = [vp, C.POINTER(C.c_longlong)]
        L.lbm_sizes.argtypes = [vp, C.POINTER(i), C.POINTER(C.c_longlong)]
        L.lbm_last_timing.argtypes = [vp, C.POINTER(C.c_float), C.POINTER(C.c_float)]
        L.lbm_profile_read.argtypes = [vp, C.POINTER(d)]
        L.lbm_recompute_steps.argtypes = [vp]
        L.lbm_recompute_steps.restype = C.c_longlong
        L.lbm_batch_primal_step.argtypes = [C.POINTER(vp), i, i]
        L.lbm_batch_adjoint_step.argtypes = [C.POINTER(vp), i, i]
        L.lbm_batch_primal_steps.argtypes = [C.POINTER(vp), i, C.POINTER(i)]
        L.lbm_batch_adjoint_steps.argtypes = [C.POINTER(vp), i, C.POINTER(i)]
        L.lbm_set_design.argtypes = [vp, vp]
        L.lbm_oneshot_reset.argtypes = [vp]
        L.lbm_oneshot_step.argtypes = [vp, i, d, d, i]
        L.lbm_oneshot_eval.argtypes = [vp, C.POINTER(d), C.POINTER(d)]
        L.lbm_threshold_scan.argtypes = [vp, C.POINTER(d), i, i, C.POINTER(d)]
        L.lbm_threshold_apply.argtypes = [vp, d]
        L.lbm_get_theta.argtypes = [vp, vp]
        L.lbm_mma_reset.argtypes = [vp]
        L.lbm_mma_update.argtypes = [vp, i, d]
        L.lbm_mma_update_with.argtypes = [vp, vp, i, d]
        L.lbm_set_stream.argtypes = [vp, vp]
        L.lbm_set_wait_polls.argtypes = [vp, C.c_longlong]
        L.lbm_state_objective_noalloc.argtypes = [C.POINTER(LbmParams), vp, vp, vp, vp,
                                                  C.POINTER(d)]
        L.lbm_noalloc_last_error.argtypes = []
        L.lbm_noalloc_last_error.restype = C.c_char_p
        _lib = L
    return _lib


def make_params(P: Problem, mem_budget: float = 0.0) -> LbmParams:
    p = LbmParams()
    p.lattice = LATTICE[P.lattice]
    p.nx, p.ny, p.nz = (int(v) for v in P.dims)
    p.collision = COLLISION[P.collision]
    p.tau = float(P.tau)
    p.s_other = float(P.s_other)
    for a in range(3):
        p.force[a] = float(P.force[a])
    p.walls = (1 if "y" in P.walls else 0) | (2 if "z" in P.walls else 0)
    p.inlet_outlet = 1 if P.channel == "inlet_outlet" else 0
    p.u_in = float(P.u_in)
    p.rho_out = float(P.rho_out)
    p.nscalars = int(P.nscalars)
    p.alpha_fluid = float(P.alpha_fluid)
    p.alpha_solid = float(P.alpha_solid)
    p.scalar_inlet = SCALAR_INLET[P.scalar_inlet]
    hot = tuple(P.hot) if P.hot else (0, 0, 0, 0)
    for a in range(4):
        p.hot[a] = int(hot[a])
    p.T_hot = float(P.T_hot)
    p.porosity = POROSITY[P.porosity]
    p.porosity_q = float(P.porosity_q)
    p.objective = OBJECTIVE[P.objective]
    p.obj_window = int(P.obj_window)
    p.nsteps = int(P.nsteps)
    p.precision = PRECISION[P.precision]
    p.ckpt_every = int(P.ckpt_every)
    p.mem_budget = float(mem_budget)
    p.kernel = KERNEL[P.kernel]
    p.adjoint_mode = ADJOINT_MODE[P.adjoint_mode]
    p.inlet_kind = INLET[P.inlet]
    p.dp = float(P.dp)
    return p


def _ptr(x):
    """Raw pointer of a torch tensor or a C-contiguous numpy array."""
    if isinstance(x, np.ndarray):
        if not x.flags["C_CONTIGUOUS"]:
            raise ValueError("numpy array must be C-contiguous")
        return x.ctypes.data
    if not x.is_contiguous():
        raise ValueError("tensor must be contiguous")
    return x.data_ptr()


def _stream_ptr(stream):
    if stream is None:
        import torch
        stream = torch.cuda.current_stream()
    return getattr(stream, "cuda_stream", stream)


class Solver:
    """One adjoint-LBM problem on the GPU (a handle of the C library)."""

    def __init__(self, P: Problem, theta, flags=None, stream=None, mem_budget: float = 0.0):
        import torch
        self.P = P
        self._L = lib()
        self._h = C.c_void_p()
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        self._params = make_params(P, mem_budget)
        th = self._as_f32(theta)
        self._sync_in()
        fl = None if flags is None else np.ascontiguousarray(flags, dtype=np.uint8)
        code = self._L.lbm_create(C.byref(self._h), C.byref(self._params), _ptr(th),
                                  None if fl is None else _ptr(fl), _stream_ptr(self.stream))
        if code != 0:
            msg = self._L.lbm_last_error(self._h).decode() if self._h else "lbm_create failed"
            if self._h:
                self._L.lbm_destroy(self._h)
                self._h = C.c_void_p()
            raise AlbmError(code, msg)
        M = C.c_int()
        N = C.c_longlong()
        self._check(self._L.lbm_sizes(self._h, C.byref(M), C.byref(N)))
        self.M, self.N = M.value, N.value

    # ---- helpers ---------------------------------------------------------------
    # The library works on the solver's stream; torch tensors are produced and
    # consumed on torch's current stream.  Device inputs are made visible to
    # the solver's stream before a call reads them, and device outputs to the
    # current stream after a call writes them.
    def _sync_in(self):
        import torch
        if isinstance(self.stream, torch.cuda.Stream):
            cur = torch.cuda.current_stream()
            if self.stream != cur:
                self.stream.wait_stream(cur)

    def _sync_out(self):
        import torch
        if isinstance(self.stream, torch.cuda.Stream):
            cur = torch.cuda.current_stream()
            if self.stream != cur:
                cur.wait_stream(self.stream)

    def _as_f32(self, theta):
        import torch
        if isinstance(theta, torch.Tensor):
            t = theta.detach().to(torch.float32).contiguous().reshape(-1)
            self._keep = t  # keep alive until the async copy is done
            return t
        return np.ascontiguousarray(np.asarray(theta, dtype=np.float32).reshape(-1))

    def _check(self, code):
        if code != 0:
            raise AlbmError(code, self._L.lbm_last_error(self._h).decode())

    def close(self):
        if getattr(self, "_h", None):
            self._L.lbm_destroy(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    # ---- the C ABI --------------------------------------------------------------
    def set_theta(self, theta):
        th = self._as_f32(theta)
        self._sync_in()
        self._check(self._L.lbm_set_theta(self._h, _ptr(th)))

    def reset(self):
        self._check(self._L.lbm_reset(self._h))

    def primal_step(self, k: int = 1):
        self._check(self._L.lbm_primal_step(self._h, int(k)))

    def adjoint_step(self, k: int = 1):
        self._check(self._L.lbm_adjoint_step(self._h, int(k)))

    def adjoint_seed(self, lam):
        self._sync_in()
        self._check(self._L.lbm_adjoint_seed(self._h, _ptr(lam)))

    def run(self):
        self._check(self._L.lbm_run(self._h))

    @property
    def time(self) -> int:
        return int(self._L.lbm_time(self._h))

    @property
    def adjoint_time(self) -> int:
        return int(self._L.lbm_adjoint_time(self._h))

    def objective(self) -> float:
        J = C.c_double()
        self._check(self._L.lbm_objective(self._h, C.byref(J)))
        return J.value

    def gradient(self, out=None):
        """dJ/dtheta as float64: into ``out`` (tensor or array) or a new device tensor."""
        import torch
        if out is None:
            out = torch.empty(self.N, dtype=torch.float64, device="cuda")
        self._sync_in()
        self._check(self._L.lbm_gradient(self._h, _ptr(out)))
        self._sync_out()
        return out

    def populations(self, which: int = 0, out=None):
        """(M, N) float32 full populations: which=0 pre-collision f^n, 1 post-collision."""
        import torch
        if out is None:
            out = torch.empty((self.M, self.N), dtype=torch.float32, device="cuda")
        self._sync_in()
        self._check(self._L.lbm_get_populations(self._h, _ptr(out), int(which)))
        self._sync_out()
        return out

    def populations_at(self, time: int, which: int = 0, out=None):
        """Populations of an earlier time the handle still holds."""
        import torch
        if out is None:
            out = torch.empty((self.M, self.N), dtype=torch.float32, device="cuda")
        self._sync_in()
        self._check(self._L.lbm_get_populations_at(self._h, int(time), _ptr(out), int(which)))
        self._sync_out()
        return out

    def set_populations(self, f):
        self._sync_in()
        self._check(self._L.lbm_set_populations(self._h, _ptr(f)))

    def adjoint(self, out=None):
        import torch
        if out is None:
            out = torch.empty((self.M, self.N), dtype=torch.float32, device="cuda")
        self._sync_in()
        self._check(self._L.lbm_get_adjoint(self._h, _ptr(out)))
        self._sync_out()
        return out

    def set_wait_polls(self, polls: int):
        """Bound of the tile-staged kernels' waits (< 0: the default)."""
        self._check(self._L.lbm_set_wait_polls(self._h, int(polls)))

    def set_stream(self, stream):
        """Move the handle to ``stream`` (a torch.cuda.Stream); its queued work
        is ordered before later work on the new stream."""
        if stream is self.stream:
            return
        self._check(self._L.lbm_set_stream(self._h, _stream_ptr(stream)))
        self.stream = stream

    def flags(self) -> np.ndarray:
        out = np.empty(self.N, dtype=np.uint8)
        self._check(self._L.lbm_get_flags(self._h, _ptr(out)))
        return out

    def check_finite(self) -> int:
        c = C.c_longlong()
        code = self._L.lbm_check_finite(self._h, C.byref(c))
        if code not in (0, 4):
            self._check(code)
        return c.value

    def last_timing(self):
        a, b = C.c_float(), C.c_float()
        self._check(self._L.lbm_last_timing(self._h, C.byref(a), C.byref(b)))
        return a.value, b.value

    def profile(self, enable: bool = True):
        self._check(self._L.lbm_profile(self._h, 1 if enable else 0))

    def profile_read(self) -> dict:
        out = (C.c_double * 8)()
        self._check(self._L.lbm_profile_read(self._h, out))
        v = list(out)
        return {"primal": (int(v[0]), v[1]), "recompute": (int(v[2]), v[3]),
                "adjoint": (int(v[4]), v[5]), "other_launches": int(v[6]),
                "launches": int(v[7])}

    def recompute_steps(self) -> int:
        return int(self._L.lbm_recompute_steps(self._h))

    # ---- one-shot optimisation (Sec. 3.3) and threshold (Sec. 3.2) ---------------
    def set_design(self, mask=None):
        """Design mask (N values, nonzero = updated) or None for the FLUID nodes."""
        import torch
        if mask is None:
            self._check(self._L.lbm_set_design(self._h, None))
            return
        if isinstance(mask, torch.Tensor):
            m = mask.detach().to(torch.uint8).contiguous().reshape(-1)
            self._keep_mask = m
            self._sync_in()
        else:
            m = np.ascontiguousarray(np.asarray(mask).reshape(-1).astype(np.uint8))
        self._check(self._L.lbm_set_design(self._h, _ptr(m)))

    def oneshot_reset(self):
        self._check(self._L.lbm_oneshot_reset(self._h))

    def oneshot_step(self, iters: int, zeta: float, penalty: float = 0.0, maximize: bool = True):
        self._check(self._L.lbm_oneshot_step(self._h, int(iters), float(zeta), float(penalty),
                                             1 if maximize else 0))

    def oneshot_eval(self):
        """(J of the current state, penalty P over the design nodes)."""
        J, P = C.c_double(), C.c_double()
        self._check(self._L.lbm_oneshot_eval(self._h, C.byref(J), C.byref(P)))
        return J.value, P.value

    def threshold_scan(self, etas, nsteps: int):
        e = (C.c_double * len(etas))(*[float(v) for v in etas])
        out = (C.c_double * len(etas))()
        self._check(self._L.lbm_threshold_scan(self._h, e, len(etas), int(nsteps), out))
        return list(out)

    def threshold_apply(self, eta: float):
        self._check(self._L.lbm_threshold_apply(self._h, float(eta)))

    # ---- MMA design iterations (Sec. 3.3) --------------------------------------
    def mma_reset(self):
        self._check(self._L.lbm_mma_reset(self._h))

    def mma_update(self, maximize: bool = True, move: float = 0.5):
        """One MMA update of theta with dJ/dtheta of the completed solve."""
        self._check(self._L.lbm_mma_update(self._h, 1 if maximize else 0, float(move)))

    def mma_update_with(self, grad, maximize: bool = True, move: float = 0.5):
        """One MMA update with a caller's gradient (N float64, tensor or array)."""
        import torch
        if isinstance(grad, torch.Tensor):
            g = grad.detach().to(torch.float64).contiguous().reshape(-1)
            self._keep_grad = g
            self._sync_in()
        else:
            g = np.ascontiguousarray(np.asarray(grad, dtype=np.float64).reshape(-1))
        self._check(self._L.lbm_mma_update_with(self._h, _ptr(g), 1 if maximize else 0,
                                                float(move)))

    def theta(self, out=None):
        """The handle's current theta (N float32) into ``out`` or a new device tensor."""
        import torch
        if out is None:
            out = torch.empty(self.N, dtype=torch.float32, device="cuda")
        self._sync_in()
        self._check(self._L.lbm_get_theta(self._h, _ptr(out)))
        self._sync_out()
        return out


def state_objective_noalloc(P: Problem, f, theta, flags, stream=None) -> float:
    """F(f) of one pre-collision state through the allocation-free entry point.

    For callers that cannot allocate device memory when they need an
    objective value (a process whose device memory is reserved in advance, a
    host framework that owns the allocator).  ``f`` (M x N float32),
    ``theta`` (N float32) and ``flags`` (N uint8) must be contiguous CUDA
    tensors of exactly those sizes: the C entry point takes no buffer sizes,
    so they are checked here before the call.  The library allocates no
    device memory for this call (its scratch is a fixed static device
    array); calls on one device must not overlap.
    """
    import torch
    Q = 9 if P.lattice == "D2Q9" else 19
    Qs = 9 if P.lattice == "D2Q9" else 7
    M = Q + int(P.nscalars) * Qs
    N = P.n_nodes
    for name, t, dtype, n in (("f", f, torch.float32, M * N), ("theta", theta, torch.float32, N),
                              ("flags", flags, torch.uint8, N)):
        if not isinstance(t, torch.Tensor) or not t.is_cuda:
            raise ValueError(f"{name} must be a CUDA tensor")
        if t.dtype != dtype or t.numel() != n or not t.is_contiguous():
            raise ValueError(f"{name} must be a contiguous {dtype} tensor of {n} elements "
                             f"(got {t.dtype}, {t.numel()} elements)")
    L = lib()
    p = make_params(P)
    F = C.c_double()
    code = L.lbm_state_objective_noalloc(C.byref(p), _ptr(f), _ptr(theta), _ptr(flags),
                                         _stream_ptr(stream), C.byref(F))
    if code != 0:
        raise AlbmError(code, L.lbm_noalloc_last_error().decode())
    return F.value


def _handles(solvers):
    arr = (C.c_void_p * len(solvers))()
    for k, s in enumerate(solvers):
        arr[k] = s._h.value
    return arr


def _steps(k, n):
    """A step count for every solver: one int for all, or a list of n."""
    if isinstance(k, (list, tuple)):
        if len(k) != n:
            raise ValueError("one step count per solver is required")
        return (C.c_int * n)(*[int(v) for v in k])
    return None


def batch_primal_step(solvers, k=1):
    """Advance every solver by up to k primal steps in batched launches (k an
    int, or a list with one count per solver)."""
    L = lib()
    ks = _steps(k, len(solvers))
    code = (L.lbm_batch_primal_steps(_handles(solvers), len(solvers), ks) if ks is not None
            else L.lbm_batch_primal_step(_handles(solvers), len(solvers), int(k)))
    if code != 0:
        raise AlbmError(code, L.lbm_last_error(solvers[0]._h).decode())


def batch_adjoint_step(solvers, k=1):
    """Run up to k adjoint steps on every solver in batched launches (k an int,
    or a list with one count per solver)."""
    L = lib()
    ks = _steps(k, len(solvers))
    code = (L.lbm_batch_adjoint_steps(_handles(solvers), len(solvers), ks) if ks is not None
            else L.lbm_batch_adjoint_step(_handles(solvers), len(solvers), int(k)))
    if code != 0:
        raise AlbmError(code, L.lbm_last_error(solvers[0]._h).decode())
